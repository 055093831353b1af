"""Batched ensemble (pibm_ensemble_*): uneven boxes of thermosensitive sphere
sedimentation with different Rayleigh numbers, advanced by one graph launch
per step.  Each box must match the FP64 oracle under the same bars as a
single context, match stepping the box alone bit for bit, and be unchanged
by the autotuner's choice of launch shapes."""
import numpy as np
import pytest

import oracle
import workloads as W
from _util import FIELD_RTOL, POS_ATOL, build_library, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def _cases(seed=5):
    return W.ensemble(n_boxes=4, edges=(24, 32, 40), n_range=(6, 20), config_index=seed)


def _state(sim):
    f, g = sim.read_populations()
    p = sim.read_particles()
    return f, g, p


def test_ensemble_matches_oracle_per_box():
    from paper_1502_01159_gb300 import Ensemble
    cases = _cases()
    assert len({c["shape"] for c in cases}) > 1 and len({c["Ra"] for c in cases}) == len(cases)
    ens = Ensemble(cases)
    ens.step(100)
    assert ens.t == 100
    for b, case in enumerate(cases):
        orc = oracle.Oracle(case)
        orc.step(100)
        sim = ens.boxes[b]
        errs = {k: rel_l2(sim.read_field(k), orc.field(k)) for k in ("rho", "T")}
        errs["u"] = rel_l2(np.stack([sim.read_field(c) for c in ("ux", "uy", "uz")]),
                           np.stack([orc.field(c) for c in ("ux", "uy", "uz")]))
        ps, po = sim.read_particles(), orc.particles()
        dX = float(np.max(np.abs(ps["X"] - po["X"])))
        dT = float(np.max(np.abs(ps["T_p"] - po["T_p"])))
        print("box", b, case["shape"], len(case["particles"]["R"]), f"Ra {case['Ra']:.3g}", errs, dX, dT)
        for k, v in errs.items():
            assert v < FIELD_RTOL, (b, k, v)
        assert dX < POS_ATOL, (b, dX)
        assert dT < 1e-6, (b, dT)
        # thermosensitive: the particle temperatures moved from their initial values
        assert np.max(np.abs(ps["T_p"] - case["particles"]["T_p"])) > 1e-4
    ens.close()


def test_ensemble_equals_boxes_stepped_alone():
    from paper_1502_01159_gb300 import Ensemble, Simulation
    cases = _cases(seed=6)
    ens = Ensemble(cases)
    ens.step(1)
    ens.step(1)
    ens.step(48)
    for b, case in enumerate(cases):
        alone = Simulation(case)
        alone.step(50)
        fa, ga, pa = _state(ens.boxes[b])
        fb_, gb_, pb = _state(alone)
        assert np.array_equal(fa, fb_) and np.array_equal(ga, gb_), b
        for k in ("X", "U", "W", "T_p"):
            assert np.array_equal(pa[k], pb[k]), (b, k)
        alone.close()
    ens.close()


def test_autotune_changes_no_result():
    from paper_1502_01159_gb300 import Ensemble
    cases = _cases(seed=7)
    tuned, plain = Ensemble(cases), Ensemble(cases)
    choice = tuned.autotune(reps=1)
    steps = 5 * 1 + 16 * (1 + 4)
    assert len(choice) == len(cases) and all(len(c) == 3 for c in choice) and tuned.t == steps
    print("autotune choices", choice)
    plain.step(steps)
    tuned.step(20)
    plain.step(20)
    for b in range(len(cases)):
        fa, ga, pa = _state(tuned.boxes[b])
        fb_, gb_, pb = _state(plain.boxes[b])
        assert np.array_equal(fa, fb_) and np.array_equal(ga, gb_), b
        assert np.array_equal(pa["X"], pb["X"]) and np.array_equal(pa["T_p"], pb["T_p"]), b
    assert tuned.kernels_per_step() >= 4 * len(cases)
    tuned.close()
    plain.close()


def test_ensemble_rejects_boxes_at_different_times():
    from paper_1502_01159_gb300 import Ensemble, PibmError
    cases = _cases(seed=8)[:2]
    ens = Ensemble(cases)
    ens.boxes[0].step(1)
    with pytest.raises(PibmError):
        ens.step(1)
    ens.boxes[1].step(1)
    ens.step(2)
    assert ens.t == 3
    ens.close()


def test_ensemble_recaptures_after_box_setup_change():
    # changing a box's set-up between ensemble steps invalidates the ensemble
    # graph; the next step must use the new set-up (compare with a box alone)
    from paper_1502_01159_gb300 import Ensemble, Simulation
    cases = _cases(seed=9)[:2]
    ens = Ensemble(cases)
    ens.step(10)
    new_wall = (1, 1, 0.3)
    ens.boxes[1].set_wall(5, *new_wall)
    ens.step(10)
    alone = Simulation(cases[1])
    alone.step(10)
    alone.set_wall(5, *new_wall)
    alone.step(10)
    fa, ga, _ = _state(ens.boxes[1])
    fb_, gb_, _ = _state(alone)
    assert np.array_equal(fa, fb_) and np.array_equal(ga, gb_)
    alone.close()
    ens.close()
