"""Pins of the surrogate's reference (oracle/surrogate.py) against closed forms:
region statistics of uniform and rigidly rotating fields, gaps of a known
arrangement, the coupling's load as the exact linear function of the
coupling-weighted features (Eqs lbm7, lbm7.5, lbm8, lbm13 at a frozen fluid
state), backpropagation against central differences, the least-squares linear
path on exactly linear data, the first Adam step, BF16 rounding, and the
secant Jacobian of a network whose answer is known."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import surrogate as S


def _fields(shape_zyx, fn):
    nz, ny, nx = shape_zyx
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ux, uy, uz, T = fn(x.astype(float), y.astype(float), z.astype(float))
    return {"rho": np.ones(shape_zyx), "ux": ux, "uy": uy, "uz": uz, "T": T}


@pytest.mark.parametrize("dim", [2, 3])
def test_region_statistics_of_uniform_flow_and_rigid_rotation(dim):
    # a uniform stream plus a rigid rotation about the particle centre: the
    # rigid-motion fit returns both exactly on any (asymmetric) region, so a
    # particle moving with the stream and spinning with the fluid has zero
    # relative velocity and spin
    Xc = np.array([10.3, 11.7, 9.4 if dim == 3 else 0.0])
    U0 = np.array([0.01, -0.02, 0.005 if dim == 3 else 0.0])
    Om = np.array([0.003, -0.001, 0.002]) if dim == 3 else np.array([0.0, 0.0, 0.002])
    shape = (21, 23, 22) if dim == 3 else (1, 23, 22)

    def fn(x, y, z):
        d = np.stack([x - Xc[0], y - Xc[1], (z - Xc[2]) if dim == 3 else 0 * z], axis=-1)
        u = U0 + np.cross(Om, d)
        return u[..., 0], u[..., 1], u[..., 2], 0.7 + 0 * x

    f = _fields(shape, fn)
    feat = S.features(f, np.array([Xc]), np.array([U0]), np.array([Om]), np.array([3.2]), np.array([1.0]), dim)
    assert np.max(np.abs(feat[0, 0:6])) < 1e-15
    assert abs(feat[0, 6] - 0.3) < 1e-14
    # moving particle: the relative velocity is U_p minus the stream
    feat = S.features(f, np.array([Xc]), np.array([U0 + 0.1]), np.array([Om]), np.array([3.2]), np.array([1.0]), dim)
    assert np.allclose(feat[0, 0:dim], 0.1, atol=1e-14)


def test_region_is_the_covered_disk():
    nodes = S.region(np.array([5.0, 5.0, 0.0]), 2.0, (11, 11, 1), 2)
    r = np.hypot(nodes[:, 0] - 5.0, nodes[:, 1] - 5.0)
    # x^2 + y^2 < 6.25: r^2 in {0, 1, 2, 4, 5}: 1 + 4 + 4 + 4 + 8 points
    assert np.all(r < 2.5) and len(nodes) == 21


def test_gaps_and_solid_fraction_of_a_row():
    # equal spheres on a line at spacing 2R + g: gaps of the middle one are g, g,
    # 2R + 2g capped at 2R, ...; phi counts the neighbours closer than 4R
    R, g = 2.0, 0.5
    n = 5
    X = np.zeros((n, 3))
    X[:, 0] = 10 + np.arange(n) * (2 * R + g)
    f = _fields((20, 20, 40), lambda x, y, z: (0 * x, 0 * x, 0 * x, 0 * x))
    feat = S.features(f, X + np.array([0, 10, 10]), np.zeros((n, 3)), np.zeros((n, 3)), np.full(n, R), np.zeros(n), 3)
    mid = feat[2]
    assert np.allclose(mid[8:12], [g, g, 2 * R, 2 * R])
    # centres within 4R = 8 of the middle one: the two at 4.5 (the next at 9 is out)
    assert abs(mid[7] - 2 * (R / (4 * R)) ** 3) < 1e-15
    end = feat[0]
    assert np.allclose(end[8:12], [g, 2 * R, 2 * R, 2 * R])


def test_backprop_matches_central_differences():
    gen = np.random.default_rng(3)
    params = S.init_params(11)
    params = [(W, gen.normal(size=b.shape) * 0.1) for W, b in params]
    params[4] = (gen.normal(size=(S.N_OUT, S.N_FEAT)) * 0.1, np.zeros(0))  # the linear path
    X = gen.normal(size=(9, S.N_FEAT))
    Y = gen.normal(size=(9, S.N_OUT))
    loss, grads = S.loss_and_grads(params, X, Y)
    flat = S.flatten(params)
    gflat = S.flatten(grads)
    h = 1e-6
    for k in gen.choice(len(flat), 40, replace=False):
        e = np.zeros_like(flat)
        e[k] = h
        lp, _ = S.loss_and_grads(S.unflatten(flat + e), X, Y)
        lm, _ = S.loss_and_grads(S.unflatten(flat - e), X, Y)
        assert abs((lp - lm) / (2 * h) - gflat[k]) < 1e-7 * max(1.0, abs(gflat[k])), k
    assert len(flat) == S.N_PARAMS


def test_first_adam_step_is_signed_learning_rate():
    params = S.init_params(1)
    grads = [(np.full_like(W, 3.0), np.full_like(b, -2.0)) for W, b in params]
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    new, m, v = S.adam(params, grads, zeros, zeros, 1, 1e-3)
    for (W0, b0), (W1, b1) in zip(params, new):
        assert np.allclose(W1 - W0, -1e-3 * 3 / (3 + 1e-8)) and np.allclose(b1 - b0, 1e-3 * 2 / (2 + 1e-8))


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, -2.5, 3.0e38])
    exp = np.array([1.0, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5, 2.9980e38])
    got = S.to_bf16(vals)
    assert np.array_equal(got[:5], exp[:5])
    assert abs(got[5] / 3.0e38 - 1) < 2 ** -8


def test_secant_jacobian_of_a_linear_network():
    # a network with tiny first-layer weights is linear to first order; make it
    # exactly linear by checking the secant against forward differences of the
    # same network and the de-standardisation by a known scale
    params = S.init_params(5)
    gen = np.random.default_rng(2)
    params[4] = (gen.normal(size=(S.N_OUT, S.N_FEAT)) * 0.3, np.zeros(0))
    Xraw = gen.normal(size=(4, S.N_FEAT))
    xmu, xsd = np.zeros(S.N_FEAT), np.full(S.N_FEAT, 2.0)
    ymu, ysd = np.zeros(S.N_OUT), np.full(S.N_OUT, 3.0)
    Y, J = S.jacobian(params, xmu, xsd, ymu, ysd, Xraw, delta=1e-6)
    # analytical derivative of the FP64 network by forward differences on the raw input
    for b in range(3):
        Xp = Xraw.copy()
        Xp[:, b] += 1e-6 * 2.0
        Yp = S.forward(params, (Xp - xmu) / xsd)[-1] * ysd + ymu
        assert np.allclose(J[:, b:9:3], (Yp[:, 0:3] - Y[:, 0:3]) / (1e-6 * 2.0), rtol=1e-6, atol=1e-8)
    for b in range(3):  # torque in spin
        Xp = Xraw.copy()
        Xp[:, 3 + b] += 1e-6 * 2.0
        Yp = S.forward(params, (Xp - xmu) / xsd)[-1] * ysd + ymu
        assert np.allclose(J[:, 9 + b:18:3], (Yp[:, 3:6] - Y[:, 3:6]) / (1e-6 * 2.0), rtol=1e-6, atol=1e-8)
    Xp = Xraw.copy()  # heat flux in the particle temperature
    Xp[:, 6] += 1e-6 * 2.0
    Yp = S.forward(params, (Xp - xmu) / xsd)[-1] * ysd + ymu
    assert np.allclose(J[:, 18], (Yp[:, 6] - Y[:, 6]) / (1e-6 * 2.0), rtol=1e-6, atol=1e-8)
    assert J.shape == (4, 19)
    assert np.allclose(Y, S.forward(params, (Xraw - xmu) / xsd)[-1] * ysd + ymu)
    assert S.gate_error(Y[:, 0:3], Y[:, 0:3]) == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_raw_fields_of_linear_equilibrium(dim):
    # first-order equilibrium populations f_i = w_i rho (1 + 3 e_i.u) carry
    # exactly the momentum rho u; g_k = w_k T sums to T
    gen = np.random.default_rng(8)
    E = np.asarray(S._E2 if dim == 2 else S._E3, dtype=float)
    w = (np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4) if dim == 2
         else np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12))
    shape = (1, 5, 6) if dim == 2 else (4, 5, 6)
    rho = 1 + 0.01 * gen.random(shape)
    u = 0.01 * gen.normal(size=(3,) + shape)
    if dim == 2:
        u[2] = 0
    f = w[:, None, None, None] * rho[None] * (1 + 3 * np.einsum("qa,a...->q...", E, u))
    T = gen.random(shape)
    g = np.stack([T * wk for wk in ([1 / 3] + [1 / 6] * 4 if dim == 2 else [1 / 4] + [1 / 8] * 6)])
    r = S.raw_fields(f, g, dim)
    assert np.allclose(r["rho"], rho, rtol=1e-14) and np.allclose(r["T"], T, rtol=1e-14)
    for a, k in enumerate(("ux", "uy", "uz")):
        assert np.allclose(r[k], u[a], atol=1e-16)


def test_owned_regions_partition_overlapping_footprints():
    # two overlapping disks: the owned node sets are disjoint, their union is
    # every node either covers, and a node goes to the disk with the larger
    # covered fraction (the lower index on a tie)
    X = np.array([[10.2, 10.0, 0.0], [14.0, 10.3, 0.0]])
    R = np.array([3.0, 2.5])
    a = S.owned(S.region(X[0], R[0], (30, 30, 1), 2), 0, X, R, 2)
    b = S.owned(S.region(X[1], R[1], (30, 30, 1), 2), 1, X, R, 2)
    sa, sb = {tuple(v) for v in a}, {tuple(v) for v in b}
    assert not (sa & sb)
    ua = {tuple(v) for v in S.region(X[0], R[0], (30, 30, 1), 2)}
    ub = {tuple(v) for v in S.region(X[1], R[1], (30, 30, 1), 2)}
    assert sa | sb == ua | ub and (ua & ub)
    for v in ua & ub:
        n = np.array([v])
        e0, e1 = S._eps(n, X[0], R[0], 2)[0], S._eps(n, X[1], R[1], 2)[0]
        assert (v in sa) == (e0 >= e1)


def test_linear_path_least_squares_recovers_linear_data():
    # targets exactly affine in the inputs: the least-squares linear path
    # reproduces them (the ridge, 1e-8 per row, moves the answer by ~1e-8)
    gen = np.random.default_rng(12)
    X = gen.normal(size=(500, S.N_FEAT))
    A = gen.normal(size=(S.N_OUT, S.N_FEAT))
    c = gen.normal(size=S.N_OUT)
    Y = X @ A.T + c
    p = S.linear_fit(S.init_params(2), X, Y)
    assert np.max(np.abs(S.forward(p, X)[-1] - Y)) < 1e-6
    assert np.allclose(p[4][0], A, atol=1e-6) and np.allclose(p[3][1], c, atol=1e-6)
    assert not np.any(p[3][0])  # the hidden layers start switched off


def test_coupling_load_is_linear_in_the_weighted_features():
    """With the coupling's own weights (epsilon rho for the rigid-motion fit,
    epsilon for the fluid temperature) the oracle's coupling of a state equals
    F = -2 m (U - V) - 2 (omega - Om) x D, tau = -2 D x (U - V) - 2 M (omega -
    Om), H = 2 kappa_T (sum epsilon) (T_p - T_s) to round-off, with m, D, M the
    weighted moments of the owned nodes.  The load comes from the oracle's C
    coupling, the features from the Python reference: an unweighted fit, a
    dropped epsilon or a sign error on either side fails by far more."""
    case = W.sed3d(nx=32, ny=32, nz=40, n_p=6, d=7.0, config_index=11, T_p_random=True)
    case["g_particle"] = [0.0, 0.0, -5e-4]
    o = oracle.Oracle(case)
    o.step(6)
    f, g = o.populations()
    fl = S.raw_fields(f, g, 3)
    p = o.particles()
    R = case["particles"]["R"]
    load = o.particle_forces()
    feat = S.features(fl, p["X"], p["U"], p["W"], R, p["T_p"], 3)
    o.close()
    kappa = case.get("kappa_T", 1.0)
    for q in range(len(R)):
        nodes = S.owned(S.region(p["X"][q], R[q], (32, 32, 40), 3), q, p["X"], R, 3)
        eps = S._eps(nodes, p["X"][q], R[q], 3)
        w = eps * fl["rho"][nodes[:, 2], nodes[:, 1], nodes[:, 0]]
        d = nodes - p["X"][q][None, :]
        m, D = np.sum(w), (w[:, None] * d).sum(axis=0)
        M = np.sum(w * np.sum(d * d, axis=1)) * np.eye(3) - (w[:, None] * d).T @ d
        dU, dW, dT = feat[q, 0:3], feat[q, 3:6], feat[q, 6]
        F = -2.0 * m * dU - 2.0 * np.cross(dW, D)
        T = -2.0 * np.cross(D, dU) - 2.0 * M @ dW
        H = 2.0 * kappa * np.sum(eps) * dT
        scale = np.linalg.norm(load["F"][q]) + 1e-30
        assert np.linalg.norm(F - load["F"][q]) < 1e-9 * scale, q
        assert np.linalg.norm(T - load["T"][q]) < 1e-9 * (np.linalg.norm(load["T"][q]) + 1e-30) + 1e-15, q
        assert abs(H - load["H"][q]) < 1e-9 * abs(load["H"][q]) + 1e-15, q
        assert scale > 1e-8  # a moving particle: the check is not trivially zero


def test_closed_form_jacobian_stabilises_light_spheres():
    """With the weighted features the coupling's load is linear in the particle's
    velocity and spin (test above), so the Jacobian the DEM should apply is known
    in closed form: half of dF/dU = -2 m and dtau/domega = -2 M, with m and M the
    eps rho-weighted mass and inertia moments of the covered fluid (rho ~ 1 at
    rest).  Applied from the first step by the oracle, it keeps spheres of
    diameter 8 at rho_p / rho_f = 0.6 bounded over 200 steps, where the plain
    explicit coupling diverges within 60."""
    case = W.sed3d(nx=40, ny=40, nz=56, n_p=12, d=8.0, config_index=31, rho_ratio=0.6)
    case["g_particle"] = [0.0, 0.0, -2e-4]
    X, R = np.asarray(case["particles"]["X"]), np.asarray(case["particles"]["R"])
    n = len(R)

    def run(J, steps):
        o = oracle.Oracle(case)
        if J is not None:
            o.set_hydro_jacobian(J)
        for k in range(steps // 20):
            o.step(20)
            U = o.particles()["U"]
            if not np.all(np.isfinite(U)) or np.max(np.abs(U)) > 1.0:
                o.close()
                return None
        o.close()
        return float(np.max(np.abs(U)))

    assert run(None, 60) is None  # the plain method diverges
    J = np.zeros((n, 19))
    for q in range(n):
        nodes = S.region(X[q], R[q], case["shape"], 3)
        eps = S._eps(nodes, X[q], R[q], 3)
        d = nodes - X[q][None, :]
        M = np.sum(eps * np.sum(d * d, axis=1)) * np.eye(3) - (eps[:, None] * d).T @ d
        J[q, 0:9] = (-np.sum(eps) * np.eye(3)).ravel()
        J[q, 9:18] = (-M).ravel()
    umax = run(J, 200)
    assert umax is not None and umax < 0.02


def test_secant_steps_survive_bf16_inputs():
    # near 0 the step is delta; far out in the tails it widens to two BF16
    # spacings, so the two BF16 inputs of the secant always differ
    x = np.array([0.0, 0.3, -1.7, 40.0, 100.0, -3000.0], dtype=np.float32)
    st = S.secant_steps(x, 0.25)
    assert st[0] == 0.25 and st[1] == 0.25 and st[2] == 0.25
    assert st[4] == 1.0  # 100 lies in [64, 128): BF16 spacing 0.5
    dq = S.to_bf16(x + st) - S.to_bf16(x)
    assert np.all(dq > 0) and np.all(dq <= 4 * st)
    # the plain step would vanish out there
    assert S.to_bf16(np.float32(100.0) + np.float32(0.25)) == S.to_bf16(np.float32(100.0))


def test_admissible_jacobian_blocks():
    m, I, h = np.array([10.0] * 5), np.array([4.0] * 5), 0.1
    J = np.zeros((5, 19))
    phys = -3.0 * np.eye(3) + 0.2 * (np.ones((3, 3)) - np.eye(3))
    for p in range(5):
        J[p, 0:9] = phys.ravel()
        J[p, 9:18] = (-2.0 * np.eye(3)).ravel()
    J[1, 4] = 0.5                 # a positive diagonal entry
    J[2, 1] = 5.0                 # a row no longer diagonally dominant
    J[3, 9:18] = (-100.0 * np.eye(3)).ravel()  # |J| h = 10 >= 2 I: an unstable substep
    A = S.admissible(J, m, I, h, 3)
    assert np.array_equal(A[0], J[0])
    assert not np.any(A[1, 0:9]) and np.array_equal(A[1, 9:18], J[1, 9:18])
    assert not np.any(A[2, 0:9])
    assert np.array_equal(A[3, 0:9], J[3, 0:9]) and not np.any(A[3, 9:18])
    # 2-D: only x, y of J_FU and z of J_TW can move; a bad z row of J_FU is ignored
    J2 = J[:1].copy()
    J2[0, 8] = 7.0
    assert np.array_equal(S.admissible(J2, m, I, h, 2), J2)
    assert not np.any(S.admissible(J2, m, I, h, 3)[0, 0:9])
