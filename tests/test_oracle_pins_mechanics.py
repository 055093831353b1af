"""Pins of three oracle functions against results that mechanics fixes, not
against the oracle's own formulas.

1. Mindlin tangential stiffness k_t = 8 G* r_a (Section 2.3, the tangential
   increment after Eq demgov, loading branch): a sphere resting on the floor
   under gravity with a stuck tangential spring oscillates at
   omega^2 = k_t (1/m + a^2/I).
2. Thermosensitive particle update (C_p dT_p/dt = -H_p, once per lattice step,
   with the load of a step taken as the mean of the couplings of t and t-1):
   in an adiabatic closed box the heat of the fluid plus that of the particle
   obeys an exact discrete balance.
3. The in-step Jacobian kick (Eq demgov with a held hydrodynamic load
   corrected by J_FU (U - U_start)): one free particle under a constant load
   follows the closed-form solution of the kick recurrence and converges to
   the solution of the ODE m dU/dt = F_0 + J_FU (U - U_0).

Each test also shows that the plausible mistakes named in its docstring
would fail it."""
import numpy as np
import pytest

import oracle
import workloads as W


def _box(shape, dim=3):
    case = W.periodic_box(shape=shape, dim=dim, buoyancy=False)
    case["walls"] = [(1, 0, 0.0)] * (2 * dim)
    return case


# ---------------------------------------------------------------- 1. Mindlin
def _hertz_constants(E, nu):
    """Hertz / Mindlin-Deresiewicz constants of two bodies of one material
    (Section 2.3): 1/E* = 2 (1 - nu^2)/E, 1/G* = 2 (1 - nu^2)/G, G = E/(2(1+nu))."""
    G = E / (2.0 * (1.0 + nu))
    return E / (2.0 * (1.0 - nu * nu)), G / (2.0 * (1.0 - nu * nu)), G


def test_mindlin_stiffness_from_stuck_oscillation():
    """A sphere resting on the floor, pushed sideways, with friction high enough
    that the contact never slides.  With v_t = U_x - a omega_y the tangential
    spring F = -k_t xi (xi' = v_t) drives m U_x' = F and I omega_y' = -a F, so
    xi'' = -k_t (1/m + a^2/I) xi: v_t oscillates at omega^2 = k_t (1/m + a^2/I)
    with a = R - delta/2 and k_t = 8 G* sqrt(delta R) (wall: R* = R).  delta
    comes from the static Hertz balance 4/3 E* sqrt(R) delta^1.5 = m (1 - 1/rho_p) g.
    A missing factor 8 changes omega by sqrt(8); the usual 1/G* = 2 (2 - nu)/G
    by a factor 1.37: both fail the 1% bar."""
    E, nu, R, rho_p, g, nsub = 100.0, 0.33, 3.0, 10.0, 1e-4, 10
    Estar, Gstar, G = _hertz_constants(E, nu)
    m = rho_p * 4.0 / 3.0 * np.pi * R ** 3
    I = 0.4 * m * R * R
    Fn = m * (1.0 - 1.0 / rho_p) * g
    delta = (Fn / (4.0 / 3.0 * Estar * np.sqrt(R))) ** (2.0 / 3.0)
    a = R - 0.5 * delta
    kt = 8.0 * Gstar * np.sqrt(delta * R)
    omega = np.sqrt(kt * (1.0 / m + a * a / I))

    case = _box((24, 24, 20))
    case.update(pibm=False, dem_substeps=nsub, g_particle=[0.0, 0.0, -g],
                contact=W.hertz(E=E, poisson=nu, mu=50.0))
    X = np.array([[11.5, 11.5, -0.5 + R - delta]])
    u0 = 1e-5
    case["particles"] = dict(X=X, U=np.array([[u0, 0.0, 0.0]]), R=np.array([R]), rho_p=np.array([rho_p]),
                             T_p=np.zeros(1))
    o = oracle.Oracle(case)
    steps = 300
    vt = np.empty(steps + 1)
    p = o.particles()
    vt[0] = p["U"][0, 0] - a * p["W"][0, 1]
    for k in range(steps):
        o.step(1)
        p = o.particles()
        vt[k + 1] = p["U"][0, 0] - a * p["W"][0, 1]
    # the normal overlap stays at the static balance (the first half kick,
    # before any contact force exists, starts a vertical ripple of ~1e-6)
    assert abs(p["X"][0, 2] - X[0, 2]) < 1e-3 * delta
    # zero crossings of v_t, linearly interpolated between lattice steps
    s = np.sign(vt)
    idx = np.nonzero(s[:-1] * s[1:] < 0)[0]
    tz = idx + vt[idx] / (vt[idx] - vt[idx + 1])
    assert len(tz) >= 10
    period = 2.0 * (tz[-1] - tz[0]) / (len(tz) - 1)
    measured = 2.0 * np.pi / period
    assert abs(measured / omega - 1.0) < 1e-2, (measured, omega)
    # v_t stays bounded by its initial amplitude (stuck: no slip, no damping)
    assert np.max(np.abs(vt)) < 1.01 * u0
    # the plausible mistakes would not pass
    assert abs(measured / (omega / np.sqrt(8.0)) - 1.0) > 0.5
    G_std = G / (2.0 * (2.0 - nu))
    omega_std = np.sqrt(8.0 * G_std * np.sqrt(delta * R) * (1.0 / m + a * a / I))
    assert abs(measured / omega_std - 1.0) > 0.2


# -------------------------------------------------------- 2. thermosensitive
def test_thermosensitive_heat_balance():
    """Adiabatic closed box (bounce-back of g at every wall), one fixed hot
    particle with heat capacity C_p.  The collision adds Q_B(r) to sum_k g_k at
    every node (sum_k g_eq = T = sum g + Q_B/2, so the BGK part adds Q_B/(2 tau)
    and the source (1 - 1/(2 tau)) Q_B), streaming with bounce-back conserves
    the sum, and sum_r Q_B(r) = sum_l A_l Q_l = H (delta_h is a partition of
    unity away from the walls).  So with S(t) = sum_r sum_k g_k(r, t):
        S(t+1) = S(t) + H(t),  C_p T_p(t+1) = C_p T_p(t) - (H(t) + H(t-1))/2
    (H(t-1) := H(t) on the first step), and
        S(t) + C_p T_p(t) - H(t-1)/2
    is the same at every t >= 1, and S + C_p T_p is unchanged over the first
    step.  A sign error in the update, a missing 1/C_p or the raw H(t) instead
    of the mean breaks the balance by O(H) per step."""
    case = _box((28, 28, 28))
    case["pibm"] = True
    # C_p large against dH/dT_p (about 2 x the covered volume): the explicit
    # update then relaxes monotonically
    R, Cp = 4.0, 8000.0
    case["particles"] = dict(X=np.array([[13.7, 14.2, 13.9]]), R=np.array([R]), rho_p=np.array([1.2]),
                             T_p=np.array([1.0]), heat_cap=np.array([Cp]), fixed=np.array([1], dtype=np.uint8))
    o = oracle.Oracle(case)

    def S():
        return float(np.sum(o.populations()[1]))

    S0, T0 = S(), float(o.particles()["T_p"][0])
    H0 = float(o.particle_forces()["H"][0])
    assert H0 > 0.0  # the hot particle heats the fluid
    o.step(1)
    S1, T1 = S(), float(o.particles()["T_p"][0])
    assert abs(S1 - (S0 + H0)) < 1e-11 * S0
    assert abs((S1 + Cp * T1) - (S0 + Cp * T0)) < 1e-11 * S0
    Hprev = H0
    inv = S1 + Cp * T1 - 0.5 * Hprev
    Ts = [T0, T1]
    for k in range(60):
        Hk = float(o.particle_forces()["H"][0])
        Sk = S()
        o.step(1)
        S2, T2 = S(), float(o.particles()["T_p"][0])
        assert abs(S2 - (Sk + Hk)) < 1e-11 * S0
        assert abs((S2 + Cp * T2 - 0.5 * Hk) - inv) < 1e-11 * S0, k
        Ts.append(T2)
    Ts = np.array(Ts)
    # the hot particle cools: monotonically once the covered fluid has taken
    # the particle's temperature (the first steps ripple as H(t) settles)
    assert np.all(np.diff(Ts[10:]) < 0.0)
    assert Ts[-1] < Ts[0] - 0.05
    assert Ts[-1] > 0.5  # and not below the fluid's initial temperature


def _heat_capacity_run(Cp, J_HT, steps):
    case = _box((28, 28, 28))
    case["pibm"] = True
    case["particles"] = dict(X=np.array([[13.7, 14.2, 13.9]]), R=np.array([4.0]), rho_p=np.array([1.2]),
                             T_p=np.array([1.0]), heat_cap=np.array([Cp]), fixed=np.array([1], dtype=np.uint8))
    o = oracle.Oracle(case)
    if J_HT is not None:
        J = np.zeros((1, 19))
        J[0, 18] = J_HT
        o.set_hydro_jacobian(J)
    Ts = [float(o.particles()["T_p"][0])]
    for _ in range(steps):
        o.step(1)
        Ts.append(float(o.particles()["T_p"][0]))
    o.close()
    return np.array(Ts)


def test_heat_jacobian_stabilises_small_heat_capacity():
    """The heat row of the Jacobian in the thermosensitive update: C_p (T_new -
    T) = -(H_held + J_HT (T_new - T)).  At a frozen fluid state the coupling's
    heat flux is H = k (T_p - T_s) with k = 2 kappa_T sum epsilon (Eq lbm7.5
    summed over the covered nodes), and the held flux is the mean of two
    couplings, so the explicit update (J_HT = 0) has the recurrence
    x^2 - (1 - a) x + a = 0, a = k / (2 C_p), unstable once C_p < k / 2; with
    the applied J_HT = k / 2 the coefficient becomes k / (2 C_p + k) < 1 and the
    update is stable for any C_p.  A particle with C_p = k / 14 in an adiabatic
    box (the covered fluid responds too, so the decay rings): without the heat
    row its temperature departs from the fluid's by orders of magnitude within
    12 steps; with it, the ripple never exceeds the initial offset and decays
    toward the fluid's temperature; a negative J_HT is taken as 0."""
    from oracle import surrogate as S
    nodes = S.region(np.array([13.7, 14.2, 13.9]), 4.0, (28, 28, 28), 3)
    k = 2.0 * 1.0 * np.sum(S._eps(nodes, np.array([13.7, 14.2, 13.9]), 4.0, 3))
    Cp = k / 14.0
    plain = _heat_capacity_run(Cp, None, 12)
    assert not np.all(np.isfinite(plain)) or np.max(np.abs(plain - 0.5)) > 100.0
    held = _heat_capacity_run(Cp, 0.5 * k, 80)
    assert np.all(np.isfinite(held))
    assert np.max(np.abs(held - 0.5)) <= 0.5 + 1e-12  # never beyond the initial offset
    assert np.max(np.abs(np.diff(held[-10:]))) < 5e-3  # the ripple has decayed to under 1 %
    assert 0.5 < np.mean(held[-10:]) < 0.55  # near the fluid's temperature, above it
    flipped = _heat_capacity_run(Cp, -0.5 * k, 12)  # taken as 0: the explicit update
    assert np.array_equal(flipped, plain)


# --------------------------------------------------------- 3. Jacobian kick
M_FREE = 2.0 * 4.0 / 3.0 * np.pi * 8.0  # rho_p (4/3) pi R^3 of the free particle below


def _free_particle(nsub, J):
    case = _box((16, 16, 16))
    rho_p, g = 2.0, np.array([3e-4, -2e-4, -5e-4])
    case.update(pibm=False, dem_substeps=nsub, g_particle=list(g), contact=W.hertz())
    U0 = np.array([[2e-3, -1e-3, 5e-4]])
    case["particles"] = dict(X=np.array([[7.5, 7.5, 7.5]]), U=U0, R=np.array([2.0]), rho_p=np.array([rho_p]),
                             T_p=np.zeros(1))
    o = oracle.Oracle(case)
    Jfull = np.zeros((1, 19))
    Jfull[0, :9] = J.ravel()
    o.set_hydro_jacobian(Jfull)
    m = rho_p * 4.0 / 3.0 * np.pi * 8.0
    F0 = m * (1.0 - 1.0 / rho_p) * g
    o.step(1)
    return o.particles()["U"][0], U0[0], F0, m


def test_jacobian_kick_diagonal_closed_form():
    """J_FU = -c m I, constant load F_0, no contacts, no fluid.  Each half kick
    of velocity Verlet is U <- U + (h/2)(F_0 + J (U - U_0))/m, evaluated at the
    start of the half kick, so over one lattice step (2 n_sub half kicks of
    h/2 = 1/(2 n_sub)) the velocity change is exactly
        V = (F_0/(m c)) (1 - (1 - c/(2 n_sub))^(2 n_sub)),
    which tends to the ODE solution (F_0/(m c)) (1 - e^-c) at first order in
    1/n_sub (the half kicks are explicit in U)."""
    c = 0.7
    errs = []
    for nsub in (5, 10, 20, 40):
        # J in force per unit velocity (dF_a/dU_b)
        U, U0, F0, m = _free_particle(nsub, -c * np.eye(3) * M_FREE)
        V = U - U0
        exact_discrete = F0 / (m * c) * (1.0 - (1.0 - c / (2 * nsub)) ** (2 * nsub))
        assert np.max(np.abs(V - exact_discrete)) < 1e-14
        ode = F0 / (m * c) * (1.0 - np.exp(-c))
        errs.append(np.max(np.abs(V - ode)) / np.max(np.abs(ode)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 2.0) < 0.15), ratios  # first order
    assert errs[-1] < 1e-2
    # a sign error (J = +c m I) would grow the velocity instead
    Ubad, U0, F0, m = _free_particle(10, c * np.eye(3) * M_FREE)
    assert np.max(np.abs((Ubad - U0) - F0 / (m * c) * (1.0 - np.exp(-c)))) > 0.3 * np.max(np.abs(F0 / m))


def test_jacobian_kick_full_matrix_converges_to_ode():
    """A non-symmetric J_FU (so a transposed J or a swapped index fails): the
    velocity change over one lattice step converges to the ODE solution
    V(1) = B^-1 (e^B - I) F_0/m with B = J_FU / m, first order in 1/n_sub, and
    the Richardson combination 2 V(2n) - V(n) matches it at second order."""
    from scipy.linalg import expm
    m = M_FREE
    B = np.array([[-0.9, 0.3, 0.0], [-0.2, -0.5, 0.25], [0.1, 0.0, -1.3]])
    ode = None
    V = {}
    for nsub in (10, 20, 40):
        U, U0, F0, mm = _free_particle(nsub, B * m)
        assert abs(mm - m) < 1e-12 * m
        a = F0 / m
        ode = np.linalg.solve(B, (expm(B) - np.eye(3)) @ a)
        V[nsub] = U - U0
    e = {k: np.max(np.abs(v - ode)) for k, v in V.items()}
    assert 1.8 < e[10] / e[20] < 2.2 and 1.8 < e[20] / e[40] < 2.2, e
    rich = 2.0 * V[40] - V[20]
    assert np.max(np.abs(rich - ode)) < 0.05 * e[40]
    # the transposed Jacobian gives a different answer, outside the first-order error
    odeT = np.linalg.solve(B.T, (expm(B.T) - np.eye(3)) @ a)
    assert np.max(np.abs(odeT - ode)) > 20 * e[40]
