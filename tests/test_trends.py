"""GPU checks of the qualitative results of the experiments section on synthetic
Overthrust-shaped models (the real model is not available): the two-level method
needs fewer iterations than the one-level method, the one-level count grows with
frequency (Table 1), and attenuation lowers the iteration count.  Mixed precision
through the C ABI, tol 1e-6."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


def _iterations(hz, p):
    G = hz.Solver(p, precision=hz.HZ_MIXED)
    G.factor()
    b = G.point_sources(p.sources)[:, 0].copy()
    x, info = G.solve(b)
    G.close()
    assert info[0][1] == 0
    return info[0][0]


def test_two_levels_beat_one_and_one_level_grows_with_frequency(hzmod):
    """At these small sizes (11-30k dofs) both counts are pre-asymptotic; the growth
    of the two counts with frequency at 0.3-2M dofs is measured by
    ``bench.py --workload trends``."""
    it = {}
    for f, cells, nsub in [(0.6, (6, 6, 3), 8), (1.2, (12, 12, 3), 16)]:
        for lv in (1, 2):
            p = synth.overthrust_problem(seed=0, freq=f, cells=cells, nsub=nsub, overlap=2, levels=lv)
            it[(f, lv)] = _iterations(hzmod, p)
    for f in (0.6, 1.2):
        assert it[(f, 2)] < it[(f, 1)], it
    assert it[(1.2, 1)] > it[(0.6, 1)], it


def test_attenuation_lowers_iterations(hzmod):
    its = []
    for Q in (20.0, 1000.0):
        p = synth.overthrust_problem(seed=0, freq=1.2, cells=(12, 12, 3), nsub=16, overlap=2, levels=2, Q=Q)
        its.append(_iterations(hzmod, p))
    assert its[0] <= its[1], its
