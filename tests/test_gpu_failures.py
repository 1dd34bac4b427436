"""Device-reported failure statuses, made to happen without faulting the GPU.

- HZ_ERR_TIMEOUT: the complex64 factorisation's tensor-core Schur update waits on an
  mbarrier for its MMAs with a bounded poll loop.  ``tc_wait_limit < 0`` gives the first
  wait no polls, so it runs out at once; the kernel then drains the MMAs it issued with
  its full-length second wait before it frees its tensor memory and returns, and
  hz_factor reports the timeout.  The context is left unfactored (hz_solve answers
  HZ_ERR_STATE), the device stays usable, and a context with the normal limit factors
  and solves the same problem.
- HZ_ERR_ZERO_PIVOT: a host-built singular input.  With a wave speed of 1e30 km/s the
  mass and absorbing terms vanish to rounding (c^-2 = 1e-60, c^-1 = 1e-30), and with
  every boundary face absorbing there is no Dirichlet row, so A = K up to 1e-30: the
  Neumann stiffness matrix, singular by the constants.  One subdomain holds all of it,
  so the last LDL^T pivot of the FP64 factor is rounding noise, far below
  1e-13 max|A_i|."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


def test_tensor_core_wait_timeout_is_reported_and_the_device_recovers(hzmod):
    import torch
    hz = hzmod
    p = synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=8)
    b = np.zeros(0)
    G = hz.Solver(p, precision=hz.HZ_MIXED, tc_wait_limit=-1)
    try:
        assert G.stats()["tc_tiles"] > 0                     # the update runs on tensor cores
        for _ in range(2):                                    # deterministic, and repeatable
            with pytest.raises(hz.HzError) as e:
                G.factor()
            assert e.value.status == hz.HZ_ERR_TIMEOUT
        b = G.point_sources()[:, 0]
        with pytest.raises(hz.HzError) as e:
            G.solve(b)
        assert e.value.status == hz.HZ_ERR_STATE              # no factor after a timeout
    finally:
        G.close()
    t = torch.arange(1000, device="cuda", dtype=torch.float64)
    assert float(t.sum()) == 499500.0                        # the context still works
    G = hz.Solver(p, precision=hz.HZ_MIXED)
    try:
        G.factor()
        x, info = G.solve(b)
        assert info[0][1] == hz.HZ_OK and info[0][2] <= p.tol
    finally:
        G.close()


def test_singular_local_matrix_gives_zero_pivot(hzmod):
    hz = hzmod
    p = synth.unit_cube_problem(n=4, nsub=1, overlap=0)
    p.c = np.full(len(p.c), 1e30 + 0j)
    p.mesh.face_tag = np.full(len(p.mesh.face_tag), 1, np.int8)   # HZ_TAG_ABC everywhere
    G = hz.Solver(p)
    try:
        with pytest.raises(hz.HzError) as e:
            G.factor()
        assert e.value.status == hz.HZ_ERR_ZERO_PIVOT
    finally:
        G.close()
    # the same mesh with its Dirichlet top restored factors
    q = synth.unit_cube_problem(n=4, nsub=1, overlap=0)
    G = hz.Solver(q)
    try:
        G.factor()
    finally:
        G.close()
