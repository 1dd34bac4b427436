"""GPU tests of the serving layer (hz_server_*): continuous batching over cached
per-(mesh, frequency) factors under an HBM budget.

Every source is one slot of its problem's pseudo-block FGMRES and follows the
same per-right-hand-side recurrence whatever shares its steps, so a request's
solutions are bitwise the same alone and in a mix of other requests (the
required bar is the solver tolerance; bitwise is what the design gives).  Every
solution is also checked against the tolerance with the oracle's FP64 operator.
"""
import numpy as np
import pytest

import synth
from oracle.solver import OracleSolver

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


@pytest.fixture(scope="module")
def probs():
    pa = synth.small_overthrust(seed=0, levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    pb = synth.small_overthrust(seed=1, levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    return pa, pb


@pytest.fixture(scope="module")
def oracles(probs):
    return [OracleSolver(p) for p in probs]


def _pts(p, rel):
    return np.asarray(rel, np.float64) * p.mesh.xyz.max(axis=0)


def _check_residuals(S, pts, X, tol=TOL):
    B = S.rhs(pts)
    for j in range(B.shape[1]):
        r = np.linalg.norm(B[:, j] - S.A @ X[:, j]) / np.linalg.norm(B[:, j])
        assert r <= tol, (j, r)


def test_same_alone_and_in_the_mix(hzmod, probs, oracles):
    pa, pb = probs
    srv = hzmod.Server(slots=4, precision=hzmod.HZ_MIXED)
    a = srv.add_problem(pa)
    b = srv.add_problem(pb)
    R = _pts(pa, [[0.3, 0.4, 0.3], [0.6, 0.5, 0.5], [0.45, 0.7, 0.4]])
    X_alone, inf_alone, t_alone = srv.wait(srv.submit(a, R, TOL), timeout=900)
    assert all(s == 0 for _, s, _ in inf_alone)
    # the same request again, now among requests on both problems submitted before
    # and after it: its sources share steps with other sources and take other slots
    rng = np.random.default_rng(7)
    before = [srv.submit(b, _pts(pb, rng.uniform(0.1, 0.9, (2, 3))), TOL),
              srv.submit(a, _pts(pa, rng.uniform(0.1, 0.9, (2, 3))), TOL)]
    again = srv.submit(a, R, TOL)
    after = [srv.submit(a, _pts(pa, rng.uniform(0.1, 0.9, (5, 3))), TOL),
             srv.submit(b, _pts(pb, rng.uniform(0.1, 0.9, (3, 3))), TOL)]
    X_mix, inf_mix, t_mix = srv.wait(again, timeout=900)
    assert [i for i, _, _ in inf_mix] == [i for i, _, _ in inf_alone]
    assert np.array_equal(X_alone, X_mix)
    d = np.linalg.norm(X_mix - X_alone) / np.linalg.norm(X_alone)
    assert d <= TOL
    _check_residuals(oracles[0], R, X_mix)
    for req in before + after:
        X, inf, t = srv.wait(req, timeout=900)
        assert all(s == 0 for _, s, _ in inf)
        assert t["admit_s"] >= t["submit_s"] and t["done_s"] >= t["admit_s"]
    st = srv.stats()
    assert st["analyses"] == 2 and st["factorisations"] == 2 and st["evictions"] == 0
    assert st["requests_done"] == 6 and st["rhs_done"] == 3 + 3 + 2 + 2 + 5 + 3
    assert 0 < st["p50_latency_s"] <= st["p99_latency_s"]
    srv.close()


def test_results_meet_tolerance_fp64_and_mixed(hzmod, probs, oracles):
    pa, pb = probs
    for prec in (hzmod.HZ_FP64, hzmod.HZ_MIXED):
        srv = hzmod.Server(slots=8, precision=prec)
        ids = [srv.add_problem(p) for p in probs]
        reqs = []
        for k in range(4):
            p = probs[k % 2]
            pts = _pts(p, np.random.default_rng(k).uniform(0.1, 0.9, (1 + 3 * k, 3)))
            reqs.append((k % 2, pts, srv.submit(ids[k % 2], pts, TOL)))
        lat = []
        for which, pts, req in reqs:
            X, inf, t = srv.wait(req, timeout=900)
            assert all(s == 0 for _, s, _ in inf)
            _check_residuals(oracles[which], pts, X)
            lat.append(t["latency_s"])
        st = srv.stats()
        # nearest-rank percentiles over the finished requests
        ls = np.sort(lat)
        assert st["p50_latency_s"] == pytest.approx(ls[int(np.ceil(0.5 * len(ls))) - 1])
        assert st["p99_latency_s"] == pytest.approx(ls[int(np.ceil(0.99 * len(ls))) - 1])
        assert st["rhs_done"] == sum(1 + 3 * k for k in range(4))
        srv.close()


def test_eviction_under_a_budget(hzmod, probs, oracles):
    # planned bytes of a load (persistent + factorisation workspace) and the bytes each
    # problem actually keeps resident afterwards
    need = []
    for p in probs:
        st = hzmod.plan(p, precision=hzmod.HZ_MIXED, block_size=16)
        need.append(st["device_bytes"] + int(1.1 * st["front_bytes"]) + 1)
    srv = hzmod.Server(slots=16, precision=hzmod.HZ_MIXED)
    ids = [srv.add_problem(p) for p in probs]
    kept = []
    for i, p in zip(ids, probs):
        srv.wait(srv.submit(i, _pts(p, [[0.5, 0.5, 0.5]]), TOL), timeout=900)
        kept.append(srv.stats()["resident_bytes"] - sum(kept))
    srv.close()
    # room for either load alone, never for one load beside the other resident problem
    # (1 KB below the sum covers the rounding of the planned workspace)
    budget = min(kept[0] + need[1], kept[1] + need[0]) - 1024
    assert budget >= max(need)
    srv = hzmod.Server(slots=16, precision=hzmod.HZ_MIXED, hbm_budget=budget)
    ids = [srv.add_problem(p) for p in probs]
    for k in range(4):
        which = k % 2
        pts = _pts(probs[which], [[0.35, 0.45, 0.4], [0.65, 0.3, 0.6]])
        X, inf, t = srv.wait(srv.submit(ids[which], pts, TOL), timeout=900)
        assert all(s == 0 for _, s, _ in inf)
        _check_residuals(oracles[which], pts, X)
    st = srv.stats()
    ctx = (need, kept, budget, st)
    assert st["analyses"] == 2, ctx                 # analysis kept across evictions
    assert st["factorisations"] == 4 and st["evictions"] == 3, ctx
    assert st["peak_resident_bytes"] <= budget
    srv.close()


def test_problem_over_budget_and_bad_requests(hzmod, probs):
    pa, pb = probs
    srv = hzmod.Server(slots=4, precision=hzmod.HZ_MIXED, hbm_budget=1 << 20)
    a = srv.add_problem(pa)
    with pytest.raises(hzmod.HzError) as e:
        srv.submit(a + 5, _pts(pa, [[0.5, 0.5, 0.5]]))
    assert e.value.status == hzmod.HZ_ERR_ARG
    X, inf, t = srv.wait(srv.submit(a, _pts(pa, [[0.5, 0.5, 0.5]])), timeout=900)
    assert inf[0][1] == hzmod.HZ_ERR_OOM and t["status"] == hzmod.HZ_ERR_OOM
    srv.close()
    srv = hzmod.Server(slots=4, precision=hzmod.HZ_MIXED)
    a = srv.add_problem(pa)
    pts = np.vstack([_pts(pa, [[0.5, 0.5, 0.5]]), [[-50.0, 0.0, 1.0]]])   # second one outside
    X, inf, t = srv.wait(srv.submit(a, pts), timeout=900)
    assert inf[0][1] == 0 and inf[1][1] == hzmod.HZ_ERR_ARG
    X, inf, t = srv.wait(srv.submit(a, np.zeros((0, 3))), timeout=60)   # empty request
    assert X.shape[1] == 0 and inf == []
    srv.close()


def test_same_alone_and_in_the_mix_at_55k_dofs(hzmod):
    """The alone-against-mix property on two 54,925-dof Overthrust-shaped problems (1.25 Hz,
    coarse (16, 16, 3) cells, 8 subdomains) with 8 slots: a 5-source request solved alone,
    then again among 4 other requests on both problems, gives bitwise the same solutions
    and iteration counts; both meet the tolerance with the oracle's operator."""
    pa = synth.overthrust_problem(seed=0, freq=1.25, nsub=8, overlap=2, restart=50, levels=2)
    pb = synth.overthrust_problem(seed=1, freq=1.25, nsub=8, overlap=2, restart=50, levels=2)
    srv = hzmod.Server(slots=8, precision=hzmod.HZ_MIXED)
    try:
        a = srv.add_problem(pa)
        b = srv.add_problem(pb)
        R = _pts(pa, [[0.2, 0.3, 0.1], [0.6, 0.5, 0.3], [0.45, 0.7, 0.2], [0.8, 0.2, 0.4], [0.3, 0.9, 0.1]])
        X_alone, inf_alone, _ = srv.wait(srv.submit(a, R, TOL), timeout=900)
        assert all(s == 0 for _, s, _ in inf_alone)
        rng = np.random.default_rng(3)
        others = [srv.submit(b, _pts(pb, rng.uniform(0.1, 0.9, (4, 3))), TOL),
                  srv.submit(a, _pts(pa, rng.uniform(0.1, 0.9, (3, 3))), TOL)]
        again = srv.submit(a, R, TOL)
        others += [srv.submit(a, _pts(pa, rng.uniform(0.1, 0.9, (6, 3))), TOL),
                   srv.submit(b, _pts(pb, rng.uniform(0.1, 0.9, (2, 3))), TOL)]
        X_mix, inf_mix, _ = srv.wait(again, timeout=900)
        assert [i for i, _, _ in inf_mix] == [i for i, _, _ in inf_alone]
        assert np.array_equal(X_alone, X_mix)
        for req in others:
            X, inf, t = srv.wait(req, timeout=900)
            assert all(s == 0 for _, s, _ in inf)
    finally:
        srv.close()
    _check_residuals(OracleSolver(pa), R, X_mix)


def test_problem_over_the_budget_fails_while_others_stay_resident(hzmod):
    """A problem that needs more than the whole HBM budget ends its requests with
    HZ_ERR_OOM at once, even while another problem stays resident and idle (that one is
    never evicted for it, since evicting it could not make room); the resident problem
    keeps serving afterwards."""
    small = synth.small_overthrust(seed=0, levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    big = synth.overthrust_problem(seed=0, freq=1.25, nsub=8, overlap=2, restart=50, levels=2)
    srv = hzmod.Server(slots=4, precision=hzmod.HZ_MIXED, hbm_budget=800 * 10**6)
    try:
        a = srv.add_problem(small)
        b = srv.add_problem(big)
        X, inf, _ = srv.wait(srv.submit(a, _pts(small, [[0.3, 0.4, 0.3]]), TOL), timeout=300)
        assert inf[0][1] == 0
        X, inf, _ = srv.wait(srv.submit(b, _pts(big, [[0.3, 0.4, 0.1], [0.6, 0.5, 0.2]]), TOL), timeout=300)
        assert [s for _, s, _ in inf] == [hzmod.HZ_ERR_OOM] * 2
        assert "over the budget" in srv.last_error()
        X, inf, _ = srv.wait(srv.submit(a, _pts(small, [[0.5, 0.5, 0.5]]), TOL), timeout=300)
        assert inf[0][1] == 0
        st = srv.stats()
        assert st["evictions"] == 0 and st["factorisations"] == 1
    finally:
        srv.close()
