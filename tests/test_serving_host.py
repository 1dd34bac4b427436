"""CPU checks of the serving layer's host logic: the admission rule
(hz_select_evictions) against an exhaustive search, and argument validation of
the server entry points that needs no device."""
import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


def _fits(bytes_, chosen, resident, need, budget):
    return resident - sum(bytes_[i] for i in chosen) + need <= budget


def test_select_evictions_against_exhaustive_search(hzmod):
    rng = np.random.default_rng(3)
    for trial in range(300):
        k = int(rng.integers(0, 7))
        b = rng.integers(1, 50, k)
        lu = rng.permutation(k).astype(np.float64) if k else np.zeros(0)
        ev = rng.integers(0, 2, k)
        resident = int(b.sum())
        need = int(rng.integers(0, 60))
        budget = int(rng.integers(1, 150))
        got = hzmod.select_evictions(b, lu, ev, resident, need, budget)
        cand = [i for i in range(k) if ev[i]]
        feasible = _fits(b, cand, resident, need, budget)
        if not feasible:
            assert got is None
            continue
        assert got is not None
        assert all(ev[i] for i in got) and len(set(got)) == len(got)
        assert _fits(b, got, resident, need, budget)
        # least recently used first: the choice is the shortest prefix of the
        # evictable residents in increasing last use that makes room
        order = sorted(cand, key=lambda i: lu[i])
        assert got == order[:len(got)]
        assert len(got) == 0 or not _fits(b, got[:-1], resident, need, budget)


def test_select_evictions_edge_cases(hzmod):
    assert hzmod.select_evictions([], [], [], 0, 10, 100) == []
    assert hzmod.select_evictions([], [], [], 0, 10, 5) is None            # alone over budget
    assert hzmod.select_evictions([5], [1.0], [1], 5, 10, 0) == []        # no budget: no limit
    assert hzmod.select_evictions([5], [1.0], [0], 5, 10, 12) is None     # busy resident
    # ties in last use keep index order
    assert hzmod.select_evictions([4, 4, 4], [1.0, 1.0, 1.0], [1, 1, 1], 12, 4, 8) == [0, 1]


def test_every_exhaustive_subset_is_no_smaller(hzmod):
    """No eviction set of fewer residents fits when the LRU prefix needs k of them
    and the residents have equal sizes."""
    b = [7, 7, 7, 7]
    lu = [3.0, 0.0, 2.0, 1.0]
    got = hzmod.select_evictions(b, lu, [1, 1, 1, 1], 28, 14, 28)
    assert got == [1, 3]
    for r in range(len(got)):
        for sub in itertools.combinations(range(4), r):
            assert not _fits(b, sub, 28, 14, 28)


def test_server_create_rejects_bad_options(hzmod):
    import ctypes as C
    lib = hzmod.lib()
    o = hzmod.ServerOptions()
    o.slots, o.precision = 1, hzmod.HZ_MIXED
    h = C.c_void_p()
    assert lib.hz_server_create(C.byref(o), C.byref(h)) == hzmod.HZ_ERR_ARG
    o.slots, o.precision = 4, 7
    assert lib.hz_server_create(C.byref(o), C.byref(h)) == hzmod.HZ_ERR_ARG
    assert lib.hz_server_create(None, C.byref(h)) == hzmod.HZ_ERR_ARG
    lib.hz_server_free(None)                                              # NULL-safe
    assert lib.hz_server_wait(None, 1, 0.0, None) == hzmod.HZ_ERR_ARG
    assert lib.hz_server_ndofs(None, 0) == -1
