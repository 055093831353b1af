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


def _call_static(X, R, dim, shape, cell, pairs, count):
    """One pibm_contacts_static call on caller-owned buffers (no torch allocation here)."""
    import ctypes as C

    import torch

    from paper_1502_01159_gb300._native import PIBM_OK, load
    L = load()
    nl = (C.c_int32 * 3)(*shape)
    s = torch.cuda.current_stream()
    st = L.pibm_contacts_static(C.c_void_p(X.data_ptr()), C.c_void_p(R.data_ptr()), int(R.numel()), dim, nl,
                                float(cell), C.c_void_p(pairs.data_ptr()), pairs.numel() // 2,
                                C.c_void_p(count.data_ptr()), C.c_void_p(s.cuda_stream))
    assert st == PIBM_OK
    s.synchronize()


def test_static_contacts_allocate_nothing():
    import torch
    X, R = _particles(3, 500, (48, 40, 52), 73)
    Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    Rd = torch.tensor(R, dtype=torch.float64, device="cuda")
    pairs = torch.zeros(2 * 4000, dtype=torch.int32, device="cuda")
    count = torch.zeros(2, dtype=torch.int32, device="cuda")
    cell = 2.0 * R.max() + 1.5
    _call_static(Xd, Rd, 3, (48, 40, 52), cell, pairs, count)  # warm-up (module load, address lookup)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        _call_static(Xd, Rd, 3, (48, 40, 52), cell, pairs, count)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # no device memory taken by the calls
    expect = _library_contacts(3, (48, 40, 52), X, R)
    total, flag = (int(v) for v in count.tolist())
    assert flag == 0 and total == len(expect)
    assert np.array_equal(pairs[: 2 * total].view(-1, 2).cpu().numpy(), expect)


def test_static_contacts_cap_and_flags():
    import torch

    from paper_1502_01159_gb300._native import contacts_static
    # cap below the pair count: the first cap pairs in (i, j) order, count = all pairs
    X, R = _particles(3, 400, (40, 36, 44), 74)
    expect = _library_contacts(3, (40, 36, 44), X, R)
    Xd = torch.tensor(X, dtype=torch.float64, device="cuda")
    Rd = torch.tensor(R, dtype=torch.float64, device="cuda")
    cap = len(expect) // 3
    got, flag = contacts_static(Xd, Rd, 3, (40, 36, 44), 2.0 * R.max() + 1.5, cap=cap)
    assert flag == 0 and len(got) == cap
    assert np.array_equal(got.cpu().numpy(), expect[:cap])
    # a cell side below the largest diameter: flag bit 2
    _, flag = contacts_static(Xd, Rd, 3, (40, 36, 44), 2.0 * R.max() - 0.5)
    assert flag & 2
    # one large particle touching 80 small ones (indices above it): 64 of its
    # pairs are kept, flag bit 1, and the pairs written are sorted and exact
    n_small = 80
    k = np.arange(n_small) + 0.5
    phi = np.arccos(1.0 - 2.0 * k / n_small)
    theta = np.pi * (1.0 + 5.0 ** 0.5) * k
    c = np.array([23.0, 23.0, 23.0])
    Xs = c + 9.0 * np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], axis=1)
    Xb = np.vstack([c, Xs])
    Rb = np.concatenate([[10.0], np.full(n_small, 0.5)])
    assert len(oracle_pairs(Xb, Rb)) == n_small  # the small ones touch only the large one
    got, flag = contacts_static(torch.tensor(Xb, dtype=torch.float64, device="cuda"),
                                torch.tensor(Rb, dtype=torch.float64, device="cuda"), 3, (48, 48, 48), 21.5)
    got = got.cpu().numpy()
    assert flag == 1 and len(got) == 64
    assert np.all(got[:, 0] == 0) and np.all(np.diff(got[:, 1]) > 0) and got[:, 1].min() >= 1


def oracle_pairs(X, R):
    import oracle
    return oracle.point_contacts(X, R)
