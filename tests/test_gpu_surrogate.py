"""Learned coupling surrogate on the GPU against its FP64 reference
(oracle/surrogate.py) and the C oracle: features, FP32 training gradients,
the least-squares linear path, BF16 tensor-core inference, the
hydrodynamic-Jacobian correction inside the DEM substeps and in the
thermosensitive update, the device-side Jacobian and gate, and what the
trained network gains over the plain method (stable light particles, stable
particles of small heat capacity), with the gate at its 1 % bound."""
import numpy as np
import pytest

import oracle
import workloads as W
from _util import POS_ATOL, build_library
from oracle import surrogate as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def _sim(case):
    from paper_1502_01159_gb300 import Simulation
    return Simulation(case)


def _case(dim, seed=21, rho_ratio=None):
    if dim == 2:
        case = W.sed2d(nx=96, ny=128, n_p=14, d=10.0, config_index=seed, rho_ratio=rho_ratio or 1.5)
        case["g_particle"] = [0.0, -2e-4, 0.0]
    else:
        case = W.sed3d(nx=40, ny=40, nz=56, n_p=12, d=8.0, config_index=seed, rho_ratio=rho_ratio or 1.2)
        case["g_particle"] = [0.0, 0.0, -2e-4]
    return case


def _oracle_features(orc, dim):
    f, g = orc.populations()
    fields = S.raw_fields(f, g, dim)
    p = orc.particles()
    R = np.asarray(orc.case["particles"]["R"])
    return S.features(fields, p["X"], p["U"], p["W"], R, p["T_p"], dim)


@pytest.mark.parametrize("dim", [2, 3])
def test_features_match_reference(dim):
    case = _case(dim)
    sim, orc = _sim(case), oracle.Oracle(case)
    sim.step(30)
    orc.step(30)
    fg = sim.read_features()
    fo = _oracle_features(orc, dim)
    # columns 0-6 come from FP32 node arithmetic on the raw moments: the
    # velocity differences (~1e-6) carry ~1e-10 absolute from FP32 moments of
    # ~1e-3; the neighbour columns 7-11 are FP64 from the positions
    for k in range(12):
        scale = max(np.max(np.abs(fo[:, k])), 1e-12)
        tol = 1e-4 * scale + 1e-9 if k < 7 else 1e-5 * scale + 1e-6
        assert np.max(np.abs(fg[:, k] - fo[:, k])) <= tol, (k, np.max(np.abs(fg[:, k] - fo[:, k])), scale)
    assert np.max(np.abs(fo[:, 0:3])) > 0  # the particles move relative to the fluid


@pytest.mark.parametrize("dim", [2, 3])
def test_features_with_one_cell_match_reference(dim):
    # a cell as large as the box: the neighbour features take the all-pairs
    # kernels instead of the cell scan (and the DEM's neighbour list holds every
    # pair); the result is the same reference
    case = _case(dim, seed=27)
    case["cell_size"] = 1000.0
    sim, orc = _sim(case), oracle.Oracle(case)
    sim.step(10)
    orc.step(10)
    fg = sim.read_features()
    fo = _oracle_features(orc, dim)
    for k in range(7, 12):
        scale = max(np.max(np.abs(fo[:, k])), 1e-12)
        assert np.max(np.abs(fg[:, k] - fo[:, k])) <= 1e-5 * scale + 1e-6, (k, np.max(np.abs(fg[:, k] - fo[:, k])))


def test_training_gradient_matches_fp64_backprop():
    sim = _sim(_case(3))
    gen = np.random.default_rng(5)
    params = S.init_params(7)
    params = [(Wm, gen.normal(size=b.shape) * 0.1) for Wm, b in params]
    params[4] = (gen.normal(size=(S.N_OUT, S.N_FEAT)) * 0.1, np.zeros(0))  # the linear path
    flat = S.flatten(params).astype(np.float32)
    norm = np.concatenate([np.zeros(12), np.ones(12), np.zeros(7), np.ones(7)]).astype(np.float32)
    sim.surrogate_set_params(flat, norm)
    for B in (1, 77, 1000):
        X = gen.normal(size=(B, 12)).astype(np.float32)
        Y = gen.normal(size=(B, 7)).astype(np.float32)
        g, loss = sim.surrogate_gradient(X, Y)
        lo, go = S.loss_and_grads(S.unflatten(flat.astype(np.float64)), X.astype(np.float64), Y.astype(np.float64))
        gflat = S.flatten(go)
        assert abs(loss - lo) <= 1e-5 * lo, (B, loss, lo)
        err = np.max(np.abs(g - gflat)) / np.max(np.abs(gflat))
        print("gradient", B, err)
        assert err < 1e-4, (B, err)


def test_tensor_core_inference_matches_bf16_reference():
    sim = _sim(_case(3))
    gen = np.random.default_rng(9)
    params = S.init_params(3)
    params = [(Wm, gen.normal(size=b.shape) * 0.2) for Wm, b in params]
    params[4] = (gen.normal(size=(S.N_OUT, S.N_FEAT)) * 0.2, np.zeros(0))  # the linear path
    flat = S.flatten(params).astype(np.float32)
    norm = np.concatenate([np.zeros(12), np.ones(12), np.zeros(7), np.ones(7)]).astype(np.float32)
    sim.surrogate_set_params(flat, norm)
    for rows in (1, 128, 1000):  # one partial tile, one full tile, several tiles with a ragged tail
        X = gen.normal(size=(rows, 12)).astype(np.float32)
        Yg = sim.surrogate_infer(X)
        p32 = S.unflatten(flat.astype(np.float64))
        Yb = S.forward_bf16(p32, X.astype(np.float64))
        Y64 = S.forward(p32, X.astype(np.float64))[-1]
        scale = np.max(np.abs(Y64))
        e_b = np.max(np.abs(Yg - Yb)) / scale
        e_64 = np.max(np.abs(Yg - Y64)) / scale
        print("inference", rows, e_b, e_64)
        # same BF16 quantisation points as the reference: within one tile the
        # result is the reference's up to the FP32 accumulation of 64 + 16
        # products (bound ~80 x 2^-24 = 5e-6 of the scale; measured 1e-7 to
        # 8e-7); over many rows the accumulation order now and then decides a
        # BF16 rounding of a hidden activation (measured ~5e-4 at 1 000 rows)
        assert e_b < (2e-6 if rows <= 128 else 1e-3), (rows, e_b)
        assert np.mean(np.abs(Yg - Yb)) / scale < 1e-5
        assert e_64 < 5e-2, (rows, e_64)  # BF16 against exact arithmetic


@pytest.mark.parametrize("dim", [2, 3])
def test_fixed_jacobian_matches_oracle(dim):
    # the in-step correction F_held + J_FU (U - U0), tau_held + J_TW (omega - omega0)
    case = _case(dim, seed=23)
    n = len(case["particles"]["R"])
    gen = np.random.default_rng(4)
    J = np.zeros((n, 19))
    for p in range(n):
        J[p, 0:9] = (-0.4 * np.eye(3) + 0.05 * gen.normal(size=(3, 3))).ravel()
        J[p, 9:18] = (-2.0 * np.eye(3) + 0.1 * gen.normal(size=(3, 3))).ravel()
        J[p, 18] = 30.0 + 10.0 * gen.random()  # no effect here: no heat capacity
    J = J.astype(np.float32).astype(np.float64)  # the device keeps it in FP32
    sim, orc = _sim(case), oracle.Oracle(case)
    sim.set_hydro_jacobian(J)
    orc.set_hydro_jacobian(J)
    plain = oracle.Oracle(case)
    sim.step(100)
    orc.step(100)
    plain.step(100)
    ps, po, pp = sim.read_particles(), orc.particles(), plain.particles()
    dX = np.max(np.abs(ps["X"] - po["X"]))
    print("fixed J", dim, dX, np.max(np.abs(po["U"] - pp["U"])))
    assert dX < POS_ATOL
    assert np.max(np.abs(ps["W"] - po["W"])) < 1e-6
    assert np.max(np.abs(po["U"] - pp["U"])) > 1e-7  # the correction changes the motion
    Jr, on = sim.read_hydro_jacobian()
    assert on and np.array_equal(Jr, J)


def _thermo_case(Cp, seed=51, rho_ratio=1.5):
    """2-D: 14 disks of diameter 10 with random initial temperatures and heat
    capacity Cp each (thermosensitive)."""
    case = _case(2, seed=seed, rho_ratio=rho_ratio)
    n = len(case["particles"]["R"])
    case["particles"]["heat_cap"] = np.full(n, float(Cp))
    case["particles"]["T_p"] = W.rng(seed + 100).random(n)
    return case


K_DISK = 157.629  # 2 kappa_T sum eps over the nodes a disk of diameter 10 covers (about 2 pi 25)


def test_fixed_heat_jacobian_matches_oracle():
    # the heat row: C_p (T_new - T) = -(H_held + J_HT (T_new - T)) at C_p = 10,
    # where the explicit update (J_HT = 0) diverges within 10 steps (a = k /
    # (2 C_p) = 7.9 > 1; oracle pin test_heat_jacobian_stabilises_small_heat_capacity)
    case = _thermo_case(10.0)
    n = len(case["particles"]["R"])
    J = np.zeros((n, 19))
    J[:, 18] = np.float32(0.5 * K_DISK)
    sim, orc = _sim(case), oracle.Oracle(case)
    sim.set_hydro_jacobian(J)
    orc.set_hydro_jacobian(J)
    sim.step(100)
    orc.step(100)
    Ts, To = sim.read_particles()["T_p"], orc.particles()["T_p"]
    print("heat Jacobian: max |dT_p|", np.max(np.abs(Ts - To)), "range", To.min(), To.max())
    assert np.all(np.isfinite(Ts)) and np.max(np.abs(To - 0.5)) < 0.5
    assert np.max(np.abs(Ts - To)) < 1e-5
    assert np.max(np.abs(sim.read_particles()["X"] - orc.particles()["X"])) < POS_ATOL


def _collect(case, steps):
    """Features and PIBM coupling (force, torque, heat flux) of each state."""
    sim = _sim(case)
    feats, targs = [], []
    for k in range(steps):
        sim.step(1)
        F = sim.read_particle_forces()
        feats.append(sim.read_features())
        targs.append(S.targets(F["F"], F["T"], F["H"]))
    sim.close()
    return np.concatenate(feats), np.concatenate(targs)


def test_training_and_device_jacobian_and_gate():
    case = _case(3, seed=25)
    feat, targ = _collect(case, 120)
    sim = _sim(case)
    # zero epochs: the least-squares linear path alone, against the FP64 reference
    sim.surrogate_train(feat, targ, epochs=0, batch=128, lr=2e-3, seed=1)
    p0, norm0 = sim.surrogate_get_params()
    mu, sd = S.standardise(feat)
    ymu, ysd = S.standardise(targ)
    ref = S.linear_fit(S.init_params(1), (feat - mu) / sd, (targ - ymu) / ysd)
    got = S.unflatten(p0.astype(np.float64))
    scale = np.max(np.abs(ref[4][0]))  # standardised data: the bias is ~0, the linear path O(1)
    for a_, b_ in ((got[4][0], ref[4][0]), (got[3][1], ref[3][1])):
        print("linear path vs reference", np.max(np.abs(a_ - b_)) / scale)
        assert np.max(np.abs(a_ - b_)) <= 1e-4 * scale
    assert not np.any(got[3][0])  # W4 = 0
    losses = sim.surrogate_train(feat, targ, epochs=40, batch=128, lr=1e-3, seed=1)
    print("loss by epoch", losses[[0, 9, 19, 39]])
    assert losses[-1] < losses[0]
    params, norm = sim.surrogate_get_params()
    # the standardisation is the training set's
    assert np.allclose(norm[:12], mu, rtol=1e-5, atol=1e-9) and np.allclose(norm[12:24], sd, rtol=1e-5)
    sim.step(20)
    # device Jacobian and gate against the reference arithmetic on the device's features;
    # the gate at its 1 % bound opens on this state
    sim.surrogate_enable(True, bound=0.01, delta=0.25)
    fg = sim.read_features()
    Jd, on = sim.read_hydro_jacobian()
    p64 = S.unflatten(params.astype(np.float64))
    xmu, xsd = norm[:12].astype(np.float64), norm[12:24].astype(np.float64)
    ymu, ysd = norm[24:31].astype(np.float64), norm[31:38].astype(np.float64)
    Yr, Jr = S.jacobian(p64, xmu, xsd, ymu, ysd, fg, delta=0.25, infer=S.forward_bf16)
    R, rho_p = np.asarray(case["particles"]["R"]), np.asarray(case["particles"]["rho_p"])
    mass = rho_p * 4.0 / 3.0 * np.pi * R ** 3
    Jr = S.admissible(S.applied_jacobian(Jr), mass, 0.4 * mass * R ** 2, 1.0 / case["dem_substeps"], 3)
    scale = np.max(np.abs(Jr))
    print("device Jacobian vs reference", np.max(np.abs(Jd - Jr)) / scale)
    assert np.max(np.abs(Jd - Jr)) / scale < 1e-4
    F = sim.read_particle_forces()["F"]
    e_ref = S.gate_error(Yr[:, 0:3], F)
    st = sim.surrogate_stats()
    print("gate", st, e_ref)
    assert abs(st["last_error"] - e_ref) < 1e-3 * e_ref + 1e-9
    assert on and st["last_error"] < 0.01 and st["on_steps"] == 1
    # bound 0: the gate always falls back, and the run is the plain method bit for bit
    ref = _sim(case)
    ref.step(20)
    sim2 = _sim(case)
    sim2.surrogate_set_params(params, norm)
    sim2.step(20)
    sim2.surrogate_enable(True, bound=0.0, delta=0.25)
    sim2.step(30)
    ref.step(30)
    a, b = sim2.read_particles(), ref.read_particles()
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["U"], b["U"])
    st2 = sim2.surrogate_stats()
    assert st2["on_steps"] == 0 and st2["off_steps"] == 31


def test_network_stabilises_light_particles():
    # What the trained network gains over the method without it.  The plain
    # coupling is explicit: the load held over a step was computed before the
    # particle moved, so for particles lighter than the fluid the exchange of
    # momentum with the covered fluid overshoots and grows (the oracle: at
    # rho_p / rho_f = 0.6 the velocities blow up within 60 steps).  The network
    # is trained only on runs the plain method can do -- density ratios 0.8 to
    # 1.5, each within its stable window -- and learns the coupling's stiffness
    # dF/dU (about -2 rho_f V); half of it, applied inside the substeps, keeps
    # the light particles bounded over 300 steps.
    feats, targs = [], []
    for rr, steps, seed in ((0.8, 110, 41), (1.0, 150, 42), (1.5, 150, 43), (0.9, 130, 44)):
        f_, t_ = _collect(_case(2, seed=seed, rho_ratio=rr), steps)
        feats.append(f_)
        targs.append(t_)
    feat, targ = np.concatenate(feats), np.concatenate(targs)
    light = _case(2, seed=31, rho_ratio=0.6)
    orc = oracle.Oracle(light)
    diverged = False
    for _ in range(15):
        orc.step(20)
        U = orc.particles()["U"]
        if not np.all(np.isfinite(U)) or np.max(np.abs(U)) > 1.0:
            diverged = True
            break
    assert diverged, "the plain method was expected to diverge for light particles"
    sim = _sim(light)
    losses = sim.surrogate_train(feat, targ, epochs=60, batch=128, lr=1e-3, seed=4)
    sim.surrogate_enable(True, bound=0.01, delta=0.25)
    J, on = sim.read_hydro_jacobian()
    rhoV = np.pi * 25.0  # fluid mass a disk of diameter 10 covers
    print("light particles: loss", losses[0], losses[-1], "applied diag J_FU / (rho_f V)", np.mean(J[:, [0, 4]]) / rhoV)
    umax = 0.0
    for k in range(15):
        sim.step(20)
        U = sim.read_particles()["U"]
        assert np.all(np.isfinite(U))
        umax = max(umax, float(np.max(np.abs(U))))
        assert umax < 0.02, (k, umax)  # stop early instead of running a diverging case on
    st = sim.surrogate_stats()
    print("light particles with the network: max |U| %.3g over 300 steps; gate" % umax, st)
    # the gate at its 1 % bound keeps the network in use on most steps (measured 205
    # to 217 of 301: the light particles sit at the edge of the training data, where
    # the network's force error is 0.5-1 %); the fallback steps do not let the run
    # diverge
    assert st["on_steps"] >= 180


def test_network_stabilises_light_spheres_3d():
    # The same gain in 3-D: spheres of diameter 8 at rho_p / rho_f = 0.6.  The
    # network is trained on 3-D runs the plain method can do (0.9, 1.0, 1.5 for
    # 120 steps).  The light spheres start moving: 20 steps at 1.2, then the
    # density set to 0.6 (same positions and velocities, the fluid kept), where
    # the plain method diverges within 50 steps (the oracle).  From rest the
    # coupling's force is zero and the relative gate stays shut until the spheres
    # move, which in 3-D is too late for this density; with the Jacobian from the
    # first step (the closed form, applied by the oracle) the run from rest
    # stays bounded too (test_closed_form_jacobian_stabilises_light_spheres).
    from paper_1502_01159_gb300 import PibmError
    feats, targs = [], []
    for rr, seed in ((0.9, 41), (1.0, 42), (1.5, 43)):
        f_, t_ = _collect(_case(3, seed=seed, rho_ratio=rr), 120)
        feats.append(f_)
        targs.append(t_)
    feat, targ = np.concatenate(feats), np.concatenate(targs)

    def switched(seed=31):
        case = _case(3, seed=seed, rho_ratio=1.2)
        s_ = _sim(case)
        s_.step(20)
        p = s_.read_particles()
        parts = dict(case["particles"])
        parts.update(X=p["X"], U=p["U"], W=p["W"], T_p=p["T_p"], rho_p=np.full(len(p["T_p"]), 0.6))
        s_.set_particles(parts)
        return s_

    plain = switched()
    try:
        plain.step(60)
        U = plain.read_particles()["U"]
        diverged = not np.all(np.isfinite(U)) or np.max(np.abs(U)) > 1.0
    except PibmError:
        diverged = True  # the runaway velocities tripped the DEM's displacement check
    assert diverged, "the plain method was expected to diverge for light spheres"
    plain.close()
    sim = switched()
    # few Adam epochs: the load is linear in these features, and the least-squares
    # path carries it; long training of the tanh layers on the heavier runs'
    # range extrapolates worse to the light spheres' (the gate then shuts)
    sim.surrogate_train(feat, targ, epochs=5, batch=128, lr=5e-4, seed=6)
    sim.surrogate_enable(True, bound=0.01, delta=0.25)
    J, on = sim.read_hydro_jacobian()
    umax = 0.0
    for k in range(15):
        sim.step(20)
        U = sim.read_particles()["U"]
        assert np.all(np.isfinite(U))
        umax = max(umax, float(np.max(np.abs(U))))
        print("light spheres, step", 20 * (k + 1), "max |U| %.4g" % umax, sim.surrogate_stats())
        assert umax < 0.02, (k, umax)
    st = sim.surrogate_stats()
    print("light spheres with the network: applied diag J_FU %.4g, max |U| %.3g over 300 steps; gate"
          % (np.mean(J[:, [0, 4, 8]]), umax), st)
    assert st["on_steps"] >= 200


def test_network_stabilises_small_heat_capacity():
    # The heat row.  The thermosensitive update is explicit too: below C_p = k / 2
    # (k = dH/dT_p = 2 kappa_T sum eps, 158 for these disks) the particle
    # temperature overshoots the fluid's and grows.  The network is trained on
    # runs with heat capacities the plain method can do (500 and 2 000).  A run
    # at C_p = 500 is stepped until the particles move, then its particles are
    # given C_p = 10 (same positions, velocities, spins, temperatures; the fluid
    # kept): the plain update then diverges within a few steps, while half the
    # network's dH/dT_p, applied in the update with the gate at its 1 % bound,
    # keeps the temperatures bounded.
    from paper_1502_01159_gb300 import PibmError
    feats, targs = [], []
    for Cp, seed in ((500.0, 61), (2000.0, 62)):
        f_, t_ = _collect(_thermo_case(Cp, seed=seed), 120)
        feats.append(f_)
        targs.append(t_)
    feat, targ = np.concatenate(feats), np.concatenate(targs)

    def switched(seed=63):
        case = _thermo_case(500.0, seed=seed)
        s_ = _sim(case)
        s_.step(20)
        p = s_.read_particles()
        parts = dict(case["particles"])
        parts.update(X=p["X"], U=p["U"], W=p["W"], T_p=p["T_p"], heat_cap=np.full(len(p["T_p"]), 10.0))
        s_.set_particles(parts)
        return s_

    plain = switched()
    try:
        plain.step(6)
        Tp = plain.read_particles()["T_p"]
        diverged = not np.all(np.isfinite(Tp)) or np.max(np.abs(Tp)) > 100.0
    except PibmError:
        diverged = True  # the runaway temperature drove the flow until the DEM's displacement check tripped
    assert diverged, "the plain update was expected to diverge"
    plain.close()
    sim = switched()
    sim.surrogate_train(feat, targ, epochs=20, batch=128, lr=1e-3, seed=5)
    sim.surrogate_enable(True, bound=0.01, delta=0.25)
    J, on = sim.read_hydro_jacobian()
    print("small heat capacity: applied J_HT / (k/2)", np.mean(J[:, 18]) / (0.5 * K_DISK), "gate on", on)
    for k in range(10):
        sim.step(20)
        Tp = sim.read_particles()["T_p"]
        assert np.all(np.isfinite(Tp)) and np.max(np.abs(Tp - 0.5)) < 0.6, (k, Tp.min(), Tp.max())
    st = sim.surrogate_stats()
    print("small heat capacity with the network: T_p in [%.3f, %.3f] after 200 steps; gate" % (Tp.min(), Tp.max()), st)
    assert st["on_steps"] >= 190
