"""Failure detection of the library, exercised without any GPU fault:

- a non-finite value planted in the populations on the host is reported by
  pibm_diagnostics as PIBM_ERR_UNSTABLE, and the state stays readable;
- an allocator hook that fails at its k-th call makes pibm_create (or
  pibm_set_particles) return PIBM_ERR_OOM, and every block the hook handed out
  is given back (no leak);
- the bounded wait of the tensor-core inference kernel, given a poll limit of
  0, gives up: the call returns PIBM_ERR_TIMEOUT, the kernel drains its own
  work and frees its tensor memory, and the context keeps working."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from _util import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def _small_case():
    case = W.sed3d(nx=32, ny=32, nz=48, n_p=6, d=8.0, config_index=2)
    case["g_particle"] = [0.0, 0.0, -2e-4]
    return case


def test_nonfinite_population_reported_unstable():
    from paper_1502_01159_gb300 import PibmError, Simulation
    from paper_1502_01159_gb300._native import PIBM_ERR_UNSTABLE
    case = _small_case()
    sim = Simulation(case)
    sim.step(3)
    assert sim.diagnostics()["nonfinite"] == 0
    f, g = sim.read_populations()
    f = f.copy()
    f[4, 20, 10, 11] = np.nan  # one population of one node, planted on the host
    sim.set_populations(f.ravel(), g.ravel())
    sim.step(2)
    with pytest.raises(PibmError) as ei:
        sim.diagnostics()
    assert ei.value.status == PIBM_ERR_UNSTABLE
    # the state is kept for inspection: the field reads back, with the NaN spread
    rho = sim.read_field("rho")
    assert np.isnan(rho).any() and np.isfinite(rho).any()
    sim.close()


class CountingAllocator:
    """Device memory from torch, failing from the `fail_at`-th request on;
    counts live blocks so that a leak shows."""

    def __init__(self, fail_at):
        import torch
        from paper_1502_01159_gb300._native import ALLOC_FN, FREE_FN, pibm_allocator
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = pibm_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, user):
        self.calls += 1
        if self.calls >= self.fail_at:
            return None
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _do_free(self, ptr, user):
        self.live.pop(ptr, None)


@pytest.mark.parametrize("fail_at", [1, 2, 5, 9])
def test_allocator_failure_in_create_reports_oom_without_leak(fail_at):
    from paper_1502_01159_gb300._native import PIBM_ERR_OOM, desc_from_case, load
    L = load()
    alloc = CountingAllocator(fail_at)
    d = desc_from_case(_small_case())
    h = C.c_void_p()
    st = L.pibm_create(C.byref(d), None, C.byref(alloc.struct), C.byref(h))
    assert st == PIBM_ERR_OOM
    assert not h.value
    assert alloc.calls >= fail_at
    assert alloc.live == {}  # every block handed out was given back


def test_allocator_failure_in_set_particles_reports_oom_without_leak():
    from paper_1502_01159_gb300._native import PIBM_ERR_OOM, PIBM_OK, desc_from_case, load, _dp, _f64
    L = load()
    alloc = CountingAllocator(10 ** 9)
    case = _small_case()
    d = desc_from_case(case)
    h = C.c_void_p()
    assert L.pibm_create(C.byref(d), None, C.byref(alloc.struct), C.byref(h)) == PIBM_OK
    for face, (kind, thermal, Tw) in enumerate(case["walls"]):  # particles need walls on every axis
        assert L.pibm_set_wall(h, face, kind, thermal, float(Tw)) == PIBM_OK
    n_create = len(alloc.live)
    alloc.fail_at = alloc.calls + 3  # the third buffer of the particle set fails
    p = case["particles"]
    X = _f64(p["X"], (-1, 3))
    n = X.shape[0]
    z3 = np.zeros((n, 3))
    R, rho, Tp = _f64(p["R"]), _f64(p["rho_p"]), _f64(p["T_p"])
    st = L.pibm_set_particles(h, n, _dp(X), _dp(z3), _dp(z3), _dp(R), _dp(rho), _dp(Tp), None, None)
    assert st == PIBM_ERR_OOM
    assert len(alloc.live) == n_create  # the partial particle buffers were released
    assert L.pibm_step(h, 2) == PIBM_OK  # the context still steps (with no particles)
    assert L.pibm_destroy(h) == PIBM_OK
    assert alloc.live == {}


def test_tensor_core_wait_timeout_is_reported_and_recovers():
    from paper_1502_01159_gb300 import PibmError, Simulation, TUNE_TC_WAIT_POLLS
    from paper_1502_01159_gb300._native import PIBM_ERR_TIMEOUT
    case = _small_case()
    sim = Simulation(case)
    gen = np.random.default_rng(5)
    n_params = 12 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 7 + 7  # the 12-64-64-64-7 network
    params = (gen.standard_normal(n_params) * 0.1).astype(np.float32)
    norm = np.concatenate([np.zeros(12), np.ones(12), np.zeros(7), np.ones(7)]).astype(np.float32)
    sim.surrogate_set_params(params, norm)
    Xn = gen.standard_normal((300, 12)).astype(np.float32)
    ref = sim.surrogate_infer(Xn)
    sim.set_tuning(TUNE_TC_WAIT_POLLS, 0)
    with pytest.raises(PibmError) as ei:
        sim.surrogate_infer(Xn)
    assert ei.value.status == PIBM_ERR_TIMEOUT
    # back to the default limit: the same inference gives the same result again
    sim.set_tuning(TUNE_TC_WAIT_POLLS, 1 << 22)
    again = sim.surrogate_infer(Xn)
    assert np.array_equal(ref, again)
    sim.step(2)
    assert sim.diagnostics()["nonfinite"] == 0
    sim.close()
