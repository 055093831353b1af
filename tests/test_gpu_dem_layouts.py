"""Parity of the DEM kernel's thread layouts with the FP64 oracle on a dense
3-D Hertz / Mindlin-Deresiewicz cluster (Section 2.3: Hertz normal force and
the tangential increment after Eq demgov, with friction and damping).

The DEM kernel gives each particle 4, 2 or 1 threads depending on how many
particles one CTA of its cluster holds (up to 64, up to 128, more).  The
particles-per-CTA tuning knob selects each of the three layouts on the same
294-sphere pile: 20 per CTA (15 CTAs, 4 threads per particle), 100 (3 CTAs,
98 each, 2 threads) and 150 (2 CTAs, 147 each, 1 thread).  The pile rests on
the floor of a walled box under gravity with every sphere in contact from the
start, so contacts (pairs and walls) load, slide and unload throughout.

Bars: contact lists bit-exact and non-empty at every checked step; positions
and spins within 1e-6 after 100 steps.  A coupled sedimentation case (fluid on)
with 130 spheres in one CTA runs the one-thread layout with the PIBM load."""
import numpy as np
import pytest

import oracle
import workloads as W
from _util import FIELD_RTOL, POS_ATOL, build_library, rel_l2

pytestmark = pytest.mark.gpu

CHECKS = (25, 50, 75, 100)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def dense_pile(seed=71):
    """7 x 7 x 6 spheres on a square lattice of spacing 4.98 resting on the
    floor, diameters 4.94 .. 5.02 (neighbours overlap by up to 0.04 or sit up to
    0.04 apart), small random velocities and spins; Hertz E = 200, nu = 0.33,
    mu = 0.3, normal and tangential damping; gravity 1e-3 along -z; no fluid."""
    gen = W.rng(seed)
    nxs, nys, nzs, s, L = 7, 7, 6, 4.98, 36
    idx = np.array([(i, j, k) for k in range(nzs) for j in range(nys) for i in range(nxs)], dtype=float)
    n = len(idx)
    X = np.zeros((n, 3))
    X[:, 0] = (L - 1) / 2.0 + (idx[:, 0] - (nxs - 1) / 2.0) * s + 0.02 * (gen.random(n) - 0.5)
    X[:, 1] = (L - 1) / 2.0 + (idx[:, 1] - (nys - 1) / 2.0) * s + 0.02 * (gen.random(n) - 0.5)
    X[:, 2] = 2.0 + idx[:, 2] * s + 0.02 * (gen.random(n) - 0.5)
    U = gen.normal(size=(n, 3)) * 2e-3
    Wv = gen.normal(size=(n, 3)) * 1e-3
    R = 2.47 + 0.04 * W.rng(seed + 1).random(n)
    case = W.periodic_box(shape=(L, L, 40), dim=3, buoyancy=False)
    case.update(walls=[(1, 1, 0.0)] * 6, pibm=False, g_particle=[0.0, 0.0, -1e-3],
                contact=W.hertz(E=200.0, poisson=0.33, mu=0.3, gamma_n=10.0, gamma_t=2.0),
                particles=dict(X=X, U=U, W=Wv, R=R, rho_p=np.full(n, 1.5), T_p=np.zeros(n)))
    return case


@pytest.fixture(scope="module")
def pile_reference():
    case = dense_pile()
    o = oracle.Oracle(case)
    ref = {0: dict(contacts=o.contacts(), **o.particles())}
    t = 0
    for tc in CHECKS:
        o.step(tc - t)
        t = tc
        ref[tc] = dict(contacts=o.contacts(), **o.particles())
    o.close()
    return case, ref


@pytest.mark.parametrize("per_cta,threads_per_particle", [(20, 4), (100, 2), (150, 1)])
def test_dense_hertz_mindlin_pile_layouts(pile_reference, per_cta, threads_per_particle):
    from paper_1502_01159_gb300 import TUNE_DEM_PARTICLES_PER_CTA, Simulation
    case, ref = pile_reference
    n = len(case["particles"]["R"])
    cs = min(16, -(-n // per_cta))
    per = -(-n // cs)
    assert (4 if per <= 64 else (2 if per <= 128 else 1)) == threads_per_particle
    sim = Simulation(case)
    sim.set_tuning(TUNE_DEM_PARTICLES_PER_CTA, per_cta)
    assert np.array_equal(sim.read_contacts(), ref[0]["contacts"])
    t = 0
    for tc in CHECKS:
        sim.step(tc - t)
        t = tc
        c = sim.read_contacts()
        assert len(ref[tc]["contacts"]) > 100  # the pile stays in contact
        assert np.array_equal(c, ref[tc]["contacts"]), (tc, len(c), len(ref[tc]["contacts"]))
    p = sim.read_particles()
    dX = np.max(np.abs(p["X"] - ref[100]["X"]))
    dW = np.max(np.abs(p["W"] - ref[100]["W"]))
    print(f"pile, {threads_per_particle} threads per particle: max |dX| {dX:.3g}, max |dW| {dW:.3g}")
    assert np.max(np.abs(ref[100]["X"] - case["particles"]["X"])) > 0.1  # the pile did settle
    assert dX < POS_ATOL
    assert dW < 1e-6
    sim.close()


def test_coupled_sedimentation_one_thread_per_particle():
    """Fluid on: 130 spheres of diameter 6 in one DEM CTA (one thread per
    particle), 100 steps against the oracle."""
    from paper_1502_01159_gb300 import TUNE_DEM_PARTICLES_PER_CTA, Simulation
    case = W.sed3d(nx=64, ny=64, nz=80, n_p=130, d=6.0, config_index=9)
    case["g_particle"] = [0.0, 0.0, -2e-4]
    sim = Simulation(case)
    sim.set_tuning(TUNE_DEM_PARTICLES_PER_CTA, 130)
    orc = oracle.Oracle(case)
    sim.step(100)
    orc.step(100)
    for name in ("rho", "T"):
        assert rel_l2(sim.read_field(name), orc.field(name)) < FIELD_RTOL, name
    u_s = np.stack([sim.read_field(c) for c in ("ux", "uy", "uz")])
    u_o = np.stack([orc.field(c) for c in ("ux", "uy", "uz")])
    assert rel_l2(u_s, u_o) < FIELD_RTOL
    ps, po = sim.read_particles(), orc.particles()
    assert np.max(np.abs(po["X"] - case["particles"]["X"])) > 1e-3
    assert np.max(np.abs(ps["X"] - po["X"])) < POS_ATOL
    assert np.max(np.abs(ps["W"] - po["W"])) < 1e-6
    sim.close()
