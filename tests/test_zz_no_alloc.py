"""The allocation-free contact search (pibm_contacts_static) against the
context's own contact read-back (pibm_read_contacts) on the same positions.

pibm_contacts_static exists for callers that cannot allocate device memory
(code inside another framework's memory pool, plug-ins whose host owns every
allocation, processes with their device memory reserved up front); it keeps
its working arrays in one fixed device array that every call shares.  This
file is collected last so that a run stopping at the first failure has run
every other test; it passes alone in a fresh process and after the others."""
import numpy as np
import pytest

import workloads as W
from _util import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()


def _particles(dim, n, shape, seed, rmin=2.0):
    gen = W.rng(seed)
    R = rmin + gen.random(n)
    X = np.zeros((n, 3))
    X[:, :dim] = 4.0 + gen.random((n, dim)) * (np.array(shape[:dim]) - 9.0)
    return X, R


def _library_contacts(dim, shape, X, R):
    from paper_1502_01159_gb300 import Simulation
    case = W.periodic_box(shape=shape, dim=dim, buoyancy=False)
    case.update(walls=[(1, 1, 0.0)] * (2 * dim), pibm=False, contact=W.hertz(),
                particles=dict(X=X, R=R, rho_p=np.full(len(R), 1.2)))
    sim = Simulation(case)
    pairs = sim.read_contacts()
    sim.close()
    return pairs


def test_static_contacts_match_library_on_two_calls_in_a_row():
    import torch

    from paper_1502_01159_gb300._native import contacts_static
    # two different particle sets, the static search called on them back to
    # back: the second call must not see the first call's cell counts or
    # offsets left in the shared array
    sets = []
    for dim, n, shape, seed in [(3, 600, (48, 40, 52), 71), (2, 250, (120, 90, 1), 72)]:
        X, R = _particles(dim, n, shape, seed)
        expect = _library_contacts(dim, shape, X, R)
        assert len(expect) > 20
        Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
        Rd = torch.tensor(R, dtype=torch.float64, device="cuda")
        sets.append((dim, shape, Xd, Rd, 2.0 * R.max() + 1.5, expect))  # the library's default cell side
    results = [contacts_static(Xd, Rd, dim, shape, cell) for dim, shape, Xd, Rd, cell, _ in sets]
    for (got, flag), (*_, expect) in zip(results, sets):
        assert flag == 0
        assert np.array_equal(got.cpu().numpy(), expect)


def test_static_contacts_reject_sizes_beyond_the_limit():
    import torch

    from paper_1502_01159_gb300._native import PibmError, contacts_static
    n = 16385
    X = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    R = torch.ones(n, dtype=torch.float64, device="cuda")
    with pytest.raises(PibmError, match="16384"):
        contacts_static(X, R, 3, (64, 64, 64), 3.5)
