"""Pins of the oracle's lattice part against closed forms and invariants.

Eq lbm2 / lbm2.5 (BGK update), Eq lbm2.6 / lbm2.7 (relaxation times), Eq lbm3
(flow equilibrium), Eq lbm3.5 read on D2Q5/D3Q7, Eq lbm9 (forcing) and the
halfway / anti-bounce-back walls are checked here without re-typing them: the
expected values are the analytic solutions of the Navier-Stokes and heat
equations that the scheme approximates, and conservation laws it must obey.
"""
import numpy as np
import pytest

import oracle
import workloads as W


E15 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 1), (-1, -1, -1),
       (1, 1, -1), (-1, -1, 1), (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1)]
W15 = [2 / 9] + [1 / 9] * 6 + [1 / 72] * 8


def _poiseuille_err(ny, nu, steps, dim=2, flow_q=0):
    case = W.poiseuille(ny=ny, nu=nu, dim=dim, nz=3 if dim == 3 else 1)
    case["flow_q"] = flow_q
    o = oracle.Oracle(case)
    o.step(steps)
    ux = o.field("ux")[0, :, 0]
    F = case["body_force"][0]
    y = np.arange(ny)
    exact = F / (2 * o.relaxation()["nu"]) * (y + 0.5) * (ny - 0.5 - y)
    return np.max(np.abs(ux - exact)) / exact.max(), o


@pytest.mark.parametrize("dim,flow_q", [(2, 0), (3, 0), (3, 15)])
def test_poiseuille_exact_at_magic_tau(dim, flow_q):
    # Halfway bounce-back + BGK reproduces the parabola exactly when
    # tau_f = 1/2 + sqrt(3/16): walls at y = -1/2 and ny - 1/2 (D2Q9, D3Q19
    # and the paper's D3Q15)
    err, o = _poiseuille_err(16, np.sqrt(3.0 / 16.0) / 3.0, 20000, dim, flow_q)
    assert abs(o.relaxation()["tau_f"] - (0.5 + np.sqrt(3.0 / 16.0))) < 1e-15
    assert err < 1e-9
    if dim == 3:
        assert np.max(np.abs(o.field("uz"))) < 1e-15


def test_poiseuille_second_order():
    errs = [_poiseuille_err(n, 0.5, int(6 * n * n / 0.5))[0] for n in (8, 16, 32)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2, errs


@pytest.mark.parametrize("dim", [2, 3])
def test_conduction_linear_profile(dim):
    case = W.conduction(ny=16, alpha=0.1, T_lo=1.0, T_hi=0.0, dim=dim, nz=3 if dim == 3 else 1)
    o = oracle.Oracle(case)
    o.step(8000)
    T = o.field("T")
    y = np.arange(16)
    exact = 1.0 + (0.0 - 1.0) * (y + 0.5) / 16.0
    assert np.max(np.abs(T - exact[None, :, None])) < 1e-12
    assert np.max(np.abs(o.field("uy"))) == 0.0


def _totals(o):
    f, g = o.populations()
    E = np.array(W.D2Q9_E if o.dim == 2 else (E15 if o.Q == 15 else W.D3Q19_E), dtype=np.float64)
    mass = f.sum()
    mom = E.T @ f.reshape(f.shape[0], -1).sum(axis=1)
    return mass, mom, g.sum()


@pytest.mark.parametrize("dim,shape,flow_q", [(2, (16, 12, 1), 0), (3, (6, 5, 4), 0), (3, (6, 5, 4), 15)])
def test_periodic_box_invariants(dim, shape, flow_q):
    case = W.periodic_box(shape=shape, dim=dim, buoyancy=True)
    case["flow_q"] = flow_q
    o = oracle.Oracle(case)
    f, g = W.random_populations(case)
    o.set_populations(f.ravel(), g.ravel())
    N = np.prod(shape)
    m0, j0, e0 = _totals(o)
    buoy = o.relaxation()["buoy"]
    up = np.zeros(3)
    up[case["gravity_axis"]] = 1.0
    for _ in range(200):
        o.step(1)
    m1, j1, e1 = _totals(o)
    assert abs(m1 - m0) / m0 < 1e-13
    assert abs(e1 - e0) / e0 < 1e-13
    # momentum gains the total force every step: buoyancy (U_c^2/L_c)(T - T_ref)
    # summed over nodes, with sum T conserved
    expect = j0 + 200 * buoy * (e0 - N * case["T_ref"]) * up
    assert np.max(np.abs(j1 - expect)) < 1e-12 * max(1.0, np.abs(expect).max())


def test_body_force_momentum_balance():
    case = W.periodic_box(shape=(10, 8, 1), dim=2, buoyancy=False, body=(1e-5, -2e-5, 0.0))
    o = oracle.Oracle(case)
    f, g = W.random_populations(case)
    o.set_populations(f.ravel(), g.ravel())
    _, j0, _ = _totals(o)
    o.step(50)
    _, j1, _ = _totals(o)
    assert np.allclose(j1 - j0, 50 * 80 * np.array([1e-5, -2e-5, 0.0]), rtol=1e-10, atol=1e-16)


def test_shear_wave_viscosity():
    # u_x = A sin(k y) decays as exp(-nu k^2 t), nu = U_c L_c sqrt(Pr/Ra) (Eq lbm2.6)
    ny = 64
    case = W.periodic_box(shape=(4, ny, 1), dim=2, buoyancy=False)
    case.update(Ra=1e4, Pr=0.71, U_c=0.1, L_c=64.0)
    o = oracle.Oracle(case)
    nu = o.relaxation()["nu"]
    assert abs(nu - 0.1 * 64 * np.sqrt(0.71 / 1e4)) < 1e-15
    k = 2 * np.pi / ny
    y = np.arange(ny)
    ux = 1e-4 * np.sin(k * (y + 0.0))
    E = np.array(W.D2Q9_E, dtype=float)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = w[:, None, None, None] * (1 + 3 * E[:, 0, None, None, None] * ux[None, None, :, None])
    f = np.broadcast_to(f, (9, 1, ny, 4)).copy()
    o.set_populations(f.ravel(), None)
    o.step(200)
    a1 = np.sum(o.field("ux")[0, :, 0] * np.sin(k * y))
    o.step(1000)
    a2 = np.sum(o.field("ux")[0, :, 0] * np.sin(k * y))
    rate = -np.log(a2 / a1) / 1000
    assert abs(rate / (nu * k * k) - 1) < 5e-3


@pytest.mark.parametrize("dim", [2, 3])
def test_thermal_diffusivity(dim):
    # T = T0 + A sin(k x) decays as exp(-alpha k^2 t), alpha = nu / Pr (Eq lbm2.7)
    nx = 48
    shape = (nx, 3, 1) if dim == 2 else (nx, 3, 3)
    case = W.periodic_box(shape=shape, dim=dim, buoyancy=False)
    case.update(Ra=1e4, Pr=0.71, U_c=0.1, L_c=64.0)
    o = oracle.Oracle(case)
    alpha = o.relaxation()["alpha"]
    k = 2 * np.pi / nx
    x = np.arange(nx)
    T = 0.5 + 1e-2 * np.sin(k * x)
    wg = np.array([1 / 3] + [1 / 6] * 4) if dim == 2 else np.array([1 / 4] + [1 / 8] * 6)
    g = wg[:, None, None, None] * T[None, None, None, :] * np.ones((1,) + shape[::-1])
    o.set_populations(None, g.ravel())
    o.step(100)
    a1 = np.sum((o.field("T")[0, 0, :] - 0.5) * np.sin(k * x))
    o.step(600)
    a2 = np.sum((o.field("T")[0, 0, :] - 0.5) * np.sin(k * x))
    rate = -np.log(a2 / a1) / 600
    assert abs(rate / (alpha * k * k) - 1) < 5e-3


def test_shear_wave_viscosity_d3q15():
    # the paper's 3-D lattice: u_x = A sin(k z) decays as exp(-nu k^2 t) with
    # nu = (tau_f - 1/2) / 3 (c_s^2 = 1/3 on D3Q15 as on D3Q19)
    nz = 48
    case = W.periodic_box(shape=(3, 3, nz), dim=3, buoyancy=False)
    case.update(Ra=1e4, Pr=0.71, U_c=0.1, L_c=64.0, flow_q=15)
    o = oracle.Oracle(case)
    nu = o.relaxation()["nu"]
    k = 2 * np.pi / nz
    z = np.arange(nz)
    ux = 1e-4 * np.sin(k * z)
    E = np.array(E15, dtype=float)
    f = np.array(W15)[:, None, None, None] * (1 + 3 * E[:, 0, None, None, None] * ux[None, :, None, None])
    f = np.broadcast_to(f, (15, nz, 3, 3)).copy()
    o.set_populations(f.ravel(), None)
    o.step(100)
    a1 = np.sum(o.field("ux")[:, 0, 0] * np.sin(k * z))
    o.step(600)
    a2 = np.sum(o.field("ux")[:, 0, 0] * np.sin(k * z))
    rate = -np.log(a2 / a1) / 600
    assert abs(rate / (nu * k * k) - 1) < 5e-3


def test_rest_state_is_stationary():
    case = W.sed2d(nx=32, ny=48, n_p=0)
    case["particles"] = None
    case["buoyancy"] = False
    o = oracle.Oracle(case)
    f0, g0 = o.populations()
    o.step(20)
    f1, g1 = o.populations()
    assert np.max(np.abs(f1 - f0)) < 1e-15
    # cold walls on a symmetric box: the temperature field keeps the box's mirror symmetries
    T = o.field("T")[0]
    assert np.max(np.abs(T - T[:, ::-1])) < 1e-14
    assert np.max(np.abs(T - T[::-1, :])) < 1e-14
    assert T.min() < 0.1 and abs(T[24, 16] - 0.5) < 1e-3
