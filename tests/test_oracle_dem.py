"""Pins of the oracle's DEM part (Eq demgov and the Hertz / Mindlin-Deresiewicz
and spring-dashpot contact laws): brute-force contact search, conservation
laws, and closed-form collision results.  The fluid coupling is switched off
so that only the particle equations act."""
import numpy as np
import pytest

import oracle
import workloads as W


def _dem_case(shape, dim, parts, law, substeps=10, g=(0.0, 0.0, 0.0)):
    case = W.periodic_box(shape=shape, dim=dim, buoyancy=False)
    case["walls"] = [(1, 1, 0.0)] * (2 * dim)
    case["pibm"] = False
    case["contact"] = law
    case["dem_substeps"] = substeps
    case["g_particle"] = list(g)
    case["particles"] = parts
    return case


def _random_cluster(dim, n, R, box, seed, vel=0.01, gap=None):
    gen = W.rng(seed)
    if gap is None:
        X = np.zeros((n, 3))
        X[:, :dim] = box[0] + gen.random((n, dim)) * (box[1] - box[0])
    else:  # dense packing with small overlaps
        X = W.rsa_positions(gen, n, R, [box[0]] * dim, [box[1]] * dim, gap=gap)
    U = np.zeros((n, 3))
    U[:, :dim] = gen.normal(size=(n, dim)) * vel
    Wv = np.zeros((n, 3))
    if dim == 2:
        Wv[:, 2] = gen.normal(size=n) * vel / R
    else:
        Wv[:] = gen.normal(size=(n, 3)) * vel / R
    Rs = R * (0.8 + 0.4 * gen.random(n)) if gap is None else R * (0.95 + 0.1 * gen.random(n))
    return dict(X=X, U=U, W=Wv, R=Rs, rho_p=np.full(n, 1.5), T_p=np.zeros(n))


@pytest.mark.parametrize("dim", [2, 3])
def test_cell_list_matches_brute_force(dim):
    shape = (40, 36, 1) if dim == 2 else (20, 18, 16)
    n = 64
    parts = _random_cluster(dim, n, 2.0, (2.0, 14.0), seed=21)
    o = oracle.Oracle(_dem_case(shape, dim, parts, W.spring_dashpot()))
    cl = o.contacts()
    bf = o.contacts_bruteforce()
    assert len(bf) > 20
    assert np.array_equal(cl, bf)
    cells, nc = o.cells()
    side = [shape[a] / nc[a] for a in range(3)]
    X = parts["X"]
    for a in range(dim):
        c = (cells // ([1, nc[0], nc[0] * nc[1]][a])) % nc[a]
        assert np.all(c * side[a] - 0.5 <= X[:, a] + 1e-12)
        assert np.all(X[:, a] < (c + 1) * side[a] - 0.5 + 1e-12)
    assert min(side[:dim]) >= 2 * parts["R"].max()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("law", ["sd", "hertz"])
def test_momentum_and_angular_momentum_conserved(dim, law):
    shape = (48, 48, 1) if dim == 2 else (32, 32, 32)
    n = 20 if dim == 2 else 30
    parts = _random_cluster(dim, n, 2.0, (14.0, 34.0) if dim == 2 else (8.0, 24.0), seed=31, gap=-0.3)
    contact = (W.spring_dashpot(kn=5.0, kt=1.5, gamma_n=0.5, gamma_t=0.1, mu=0.5) if law == "sd"
               else W.hertz(E=50.0, mu=0.5, gamma_n=0.5, gamma_t=0.1))
    o = oracle.Oracle(_dem_case(shape, dim, parts, contact, substeps=10))
    m = parts["rho_p"] * (np.pi * parts["R"] ** 2 if dim == 2 else 4 / 3 * np.pi * parts["R"] ** 3)
    I = (0.5 if dim == 2 else 0.4) * m * parts["R"] ** 2

    def totals():
        p = o.particles()
        P = (m[:, None] * p["U"]).sum(axis=0)
        L = (m[:, None] * np.cross(p["X"], p["U"]) + I[:, None] * p["W"]).sum(axis=0)
        return P, L, np.abs(m[:, None] * p["U"]).sum()

    P0, L0, scale = totals()
    o.step(20)
    P1, L1, _ = totals()
    assert len(o.contacts()) > 0
    assert np.max(np.abs(P1 - P0)) < 1e-13 * scale
    assert np.max(np.abs(L1 - L0)) < 1e-13 * scale * 20


def _head_on(E, substeps, max_steps, R=4.0, v=0.1):
    parts = dict(X=[[6.0, 8.0, 8.0], [14.25, 8.0, 8.0]], U=[[v / 2, 0, 0], [-v / 2, 0, 0]],
                 R=[R, R], rho_p=[1.2, 1.2], T_p=[0, 0])
    o = oracle.Oracle(_dem_case((24, 16, 16), 3, parts, W.hertz(E=E, poisson=0.33, mu=0.0),
                                substeps=substeps))
    dmax, touching = 0.0, 0
    for _ in range(max_steps):
        o.step(1)
        X = o.particles()["X"]
        overlap = 2 * R - (X[1, 0] - X[0, 0])
        dmax = max(dmax, overlap)
        touching += overlap > 0
        if touching and overlap < -0.05:
            break
    m = 1.2 * 4 / 3 * np.pi * R ** 3
    return o.particles(), m, dmax, touching


def test_hertz_elastic_head_on_energy():
    # Two equal spheres, mu = 0, no damping: kinetic energy is conserved and the velocities swap
    v = 0.1
    p, m, _, touching = _head_on(2000.0, 160, 40)
    ke0 = 2 * 0.5 * m * (v / 2) ** 2
    ke1 = 0.5 * m * (p["U"] ** 2).sum()
    assert touching > 0
    assert abs(ke1 / ke0 - 1) < 2e-6  # velocity Verlet, ~160 substeps per contact
    assert abs(p["U"][0, 0] + v / 2) < 1e-6 and abs(p["U"][1, 0] - v / 2) < 1e-6


def test_hertz_overlap_and_contact_time():
    # delta_max = (15 m* v^2 / (16 E* sqrt(R*)))^(2/5), t_c = 2.9432 delta_max / v,
    # with 1/E* = (1 - nu^2)/E + (1 - nu^2)/E (text after Eq demgov)
    E, R, v = 5.0, 4.0, 0.1
    _, m, dmax, touching = _head_on(E, 40, 80)
    Estar = E / (2 * (1 - 0.33 ** 2))
    dth = (15 * (m / 2) * v * v / (16 * Estar * np.sqrt(R / 2))) ** 0.4
    assert abs(dmax / dth - 1) < 1e-2  # sampled once per lattice step
    tc = 2.9432 * dth / v
    assert abs(touching - tc) <= 1.0  # sampled once per lattice step


def test_spring_dashpot_restitution():
    # linear spring-dashpot: e = exp(-pi zeta / sqrt(1 - zeta^2)), zeta = gamma / (2 sqrt(m* k))
    R, v = 5.0, 0.05
    kn, gn = 100.0, 5.15
    parts = dict(X=[[10.0, 12.0, 0.0], [20.2, 12.0, 0.0]], U=[[v / 2, 0, 0], [-v / 2, 0, 0]],
                 R=[R, R], rho_p=[1.5, 1.5], T_p=[0, 0])
    law = W.spring_dashpot(kn=kn, kt=0.0, gamma_n=gn, mu=0.0)
    o = oracle.Oracle(_dem_case((32, 24, 1), 2, parts, law, substeps=200))
    o.step(30)
    p = o.particles()
    assert 2 * R - (p["X"][1, 0] - p["X"][0, 0]) < 0  # separated again
    e = (p["U"][1, 0] - p["U"][0, 0]) / v
    m = 1.5 * np.pi * R ** 2
    zeta = gn / (2 * np.sqrt(m / 2 * kn))
    assert abs(e / np.exp(-np.pi * zeta / np.sqrt(1 - zeta ** 2)) - 1) < 1e-3


def test_free_fall_exact():
    # constant acceleration (1 - rho_f/rho_p) g: velocity Verlet is exact
    g = np.array([0.0, -1e-3, 0.0])
    parts = dict(X=[[8.0, 12.0, 0.0]], U=[[0.002, 0.0, 0.0]], R=[2.0], rho_p=[2.0], T_p=[0])
    o = oracle.Oracle(_dem_case((16, 24, 1), 2, parts, W.spring_dashpot(), substeps=10, g=g))
    o.step(40)
    p = o.particles()
    a = 0.5 * g
    assert np.allclose(p["U"][0], [0.002, 0, 0] + a * 40, rtol=0, atol=1e-15)
    assert np.allclose(p["X"][0], [8.0 + 0.002 * 40, 12.0, 0] + 0.5 * a * 40 ** 2, rtol=0, atol=1e-12)


def test_wall_bounce_elastic():
    R, v = 4.0, 0.08
    parts = dict(X=[[8.0, 4.2, 8.0]], U=[[0, -v, 0]], R=[R], rho_p=[1.2], T_p=[0])
    o = oracle.Oracle(_dem_case((16, 16, 16), 3, parts, W.hertz(E=2000.0, mu=0.0), substeps=100))
    o.step(20)
    p = o.particles()
    assert abs(p["U"][0, 1] / v - 1) < 5e-6
    assert p["X"][0, 1] > 4.0


def test_sliding_disk_reaches_rolling():
    # A disk sliding on the floor without spin: Coulomb friction (mu F_n, the cap
    # of the tangential spring) slows it and spins it up until it rolls; with
    # I = m R^2 / 2 the rolling speed is 2/3 of the initial speed.
    R, v0, rho = 5.0, 0.01, 2.0
    m = rho * np.pi * R ** 2
    g = 1e-2
    kn = 100.0
    delta = m * (1 - 1 / rho) * g / kn
    parts = dict(X=[[10.0, -0.5 + R - delta, 0.0]], U=[[v0, 0, 0]], R=[R], rho_p=[rho], T_p=[0])
    law = W.spring_dashpot(kn=kn, kt=30.0, gamma_n=5.0, gamma_t=5.0, mu=0.3)
    o = oracle.Oracle(_dem_case((64, 16, 1), 2, parts, law, substeps=20, g=(0, -g, 0)))
    o.step(20)
    v, wr = [], []
    for _ in range(60):  # the stuck tangential spring oscillates about the rolling state
        o.step(1)
        p = o.particles()
        v.append(p["U"][0, 0])
        wr.append(-p["W"][0, 2] * R)
    assert abs(np.mean(v) / (2 * v0 / 3) - 1) < 0.02
    assert abs(np.mean(wr) / np.mean(v) - 1) < 0.02  # rolling without slip, clockwise
