"""Pins of the oracle's Mindlin-Deresiewicz loading history (Section 2.3: the
tangential increment 8 G* r_a theta_k dd_t + (-1)^k mu dF_n (1 - theta_k) after
Eq demgov; theta_k by the closure of Thornton and Yin for loading, unloading and
reloading) against the closed forms of Mindlin and Deresiewicz for a contact
under a constant normal force N, stiffness k0 = 8 G* a, slip displacement
d_max = 3 mu N / (2 k0) (= 3 mu N / (16 G* a)):

  loading from rest      T = mu N [1 - (1 - d / d_max)^(3/2)]
  unloading from T*, d*  T = T* - 2 mu N [1 - (1 - (d* - d) / (2 d_max))^(3/2)]
  reloading from T**     T = T** + 2 mu N [1 - (1 - (d - d**) / (2 d_max))^(3/2)]

and a load-unload-reload cycle between +d* and -d* closes (the hysteresis
loop returns to T* at d*).  The update is explicit in the displacement, so the
closed forms are reached at first order in the increment: 1e-3 of mu N with
d_max / 20000 increments.  A missing cube root, a factor 2 dropped from the
unloading branch or a wrong turning point fails these by far more."""
import numpy as np
import pytest

import oracle
import workloads as W

E, NU, MU, N, A = 500.0, 0.3, 0.4, 0.05, 0.7


def _oracle():
    case = W.periodic_box(shape=(8, 8, 8), dim=3, buoyancy=False)
    case["contact"] = dict(law=2, E=E, poisson=NU, mu=MU, kn=0.0, kt=0.0, gamma_n=0.0, gamma_t=0.0)
    return oracle.Oracle(case)


def _k0():
    G = E / (2.0 * (1.0 + NU))
    return 8.0 * G / (2.0 * (1.0 - NU * NU)) * A


def _run(o, increments):
    """increments along x (negative: T grows along +x first); returns the x
    component of the tangential force after each update and the displacement."""
    ds = np.zeros((len(increments), 3))
    ds[:, 0] = -np.asarray(increments)
    T = o.md_path([0.0, 0.0, 1.0], A, np.full(len(increments), N), ds)
    return T[:, 0], np.cumsum(increments)


def test_loading_curve():
    o = _oracle()
    dmax = 1.5 * MU * N / _k0()
    h = dmax / 20000
    T, d = _run(o, np.full(19000, h))
    closed = MU * N * (1.0 - (1.0 - d / dmax) ** 1.5)
    assert np.max(np.abs(T - closed)) < 1e-3 * MU * N
    # the same increments with the no-slip spring (theta = 1) would be linear
    assert abs(T[9999] - _k0() * d[9999]) > 0.05 * MU * N


@pytest.mark.parametrize("frac", [0.3, 0.7])
def test_unloading_and_reloading_curves(frac):
    o = _oracle()
    k0 = _k0()
    dmax = 1.5 * MU * N / k0
    h = dmax / 20000
    nload = int(frac * 20000)
    nun = int(1.2 * 20000)
    nre = int(0.8 * 20000)
    inc = np.concatenate([np.full(nload, h), np.full(nun, -h), np.full(nre, h)])
    T, d = _run(o, inc)
    Ts, ds_ = T[nload - 1], d[nload - 1]
    assert abs(Ts - MU * N * (1.0 - (1.0 - ds_ / dmax) ** 1.5)) < 1e-3 * MU * N
    u = slice(nload, nload + nun)
    x = ds_ - d[u]
    unload = Ts - 2.0 * MU * N * (1.0 - np.clip(1.0 - x / (2.0 * dmax), 0.0, None) ** 1.5)
    unload = np.maximum(unload, -MU * N)  # full reverse slip
    assert np.max(np.abs(T[u] - unload)) < 1e-3 * MU * N
    Tss, dss = T[nload + nun - 1], d[nload + nun - 1]
    r = slice(nload + nun, nload + nun + nre)
    y = d[r] - dss
    reload = Tss + 2.0 * MU * N * (1.0 - np.clip(1.0 - y / (2.0 * dmax), 0.0, None) ** 1.5)
    # reloading meets the loading curve at T*, then follows it (capped at mu N)
    on_reload = reload <= Ts
    assert np.max(np.abs(T[r][on_reload] - reload[on_reload])) < 1e-3 * MU * N
    # a unloading branch without the factor 2 would differ grossly
    wrong = Ts - MU * N * (1.0 - np.clip(1.0 - x / dmax, 0.0, None) ** 1.5)
    assert np.max(np.abs(T[u] - wrong)) > 0.05 * MU * N


def test_hysteresis_loop_closes():
    o = _oracle()
    dmax = 1.5 * MU * N / _k0()
    h = dmax / 20000
    n1 = 6000  # d* = 0.3 d_max
    inc = np.concatenate([np.full(n1, h), np.full(2 * n1, -h), np.full(2 * n1, h)])
    T, d = _run(o, inc)
    Ts = T[n1 - 1]
    assert abs(T[3 * n1 - 1] + Ts) < 2e-3 * MU * N    # unloaded to -T* at -d*
    assert abs(T[5 * n1 - 1] - Ts) < 2e-3 * MU * N    # reloaded back to T* at d*
    # the loop dissipates: the work sum T dd over the cycle is positive, the
    # ascending branch lies above the descending one (at d = 0 the closed forms
    # give -/+ (2 mu N (1 - (1 - d*/(2 d_max))^1.5) - T*) = -/+ 0.0183 mu N)
    i_un = n1 + n1 - 1          # d = 0 on the way down
    i_re = 3 * n1 + n1 - 1      # d = 0 on the way up
    x = 0.3 / 2.0
    gap = 2.0 * MU * N * (1.0 - (1.0 - x) ** 1.5) - MU * N * (1.0 - 0.7 ** 1.5)
    assert abs(T[i_re] - gap) < 2e-3 * MU * N and abs(T[i_un] + gap) < 2e-3 * MU * N
    work = np.sum(T[n1:] * np.diff(d)[n1 - 1:])
    assert work > 0.0


def test_first_contact_update_has_no_history_increment():
    # a new contact (previous normal force zero) with a tangential increment:
    # T = k0 d on its first update, not a jump to mu N
    o = _oracle()
    ds = np.array([[-1e-6, 0.0, 0.0]])
    T = o.md_path([0.0, 0.0, 1.0], A, [N], ds)
    assert abs(T[0, 0] - _k0() * 1e-6) < 1e-9 * _k0() * 1e-6 + 1e-18


def _departure(case, steps, eps=1e-15):
    """max |dX| between the oracle on `case` and on `case` with its positions
    scaled by (1 + eps), after `steps` steps"""
    import copy
    other = copy.deepcopy(case)
    other["particles"]["X"] = other["particles"]["X"] * (1.0 + eps)
    a, b = oracle.Oracle(case), oracle.Oracle(other)
    a.step(steps)
    b.step(steps)
    d = np.max(np.abs(a.particles()["X"] - b.particles()["X"]))
    a.close()
    b.close()
    return d


def test_history_trajectory_conditioning():
    """The explicit theta_k update maps T to T + 8 G* a theta(T) dd, whose
    slope 1 - 8 G* a |dd| / (3 theta^2 mu F_n) leaves [-1, 1] near full slip:
    there the update amplifies differences, and the cube root turns a rounding
    residual eps of the slip condition into eps^(1/3).  On the dense pile,
    whose contacts sit at or near slip, a 1e-15 change of the positions moves
    the law-2 trajectory by more than 1e-7 within one step, where law 1
    (theta = 1) stays below 1e-10; on the dilute colliding gas law 2 stays
    below 1e-9 over 100 steps.  Element-by-element parity of law 2 is
    therefore checked on the gas, and on the pile only the whole state."""
    assert _departure(W.dense_pile(law=2), 1) > 1e-7
    assert _departure(W.dense_pile(law=1), 10) < 1e-10
    assert _departure(W.colliding_gas(law=2), 100) < 1e-9
