"""hz_cgs2_noalloc -- the CGS2 step for callers that cannot allocate device memory
(its partial sums live in a fixed file-scope device array instead of a context
workspace).  Checked through the C ABI against hz_cgs2 on two calls in a row,
which also shows that the contents the first call leaves in the shared array do
not leak into the second.  Collected last, so that a failure here comes after
every other test has run."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_cgs2_matches_context_cgs2():
    import torch
    from paper_2004_06309_gb300 import build, hz
    build.build()
    lib = hz.lib()
    p = synth.small_overthrust(levels=2, cells=(4, 4, 2), freq=0.5, nsub=8)
    G = hz.Solver(p)
    n = G.n
    rng = np.random.default_rng(11)
    for call, ncols in enumerate((13, 40)):
        V = rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))
        V, _ = np.linalg.qr(V)
        w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        Vd = torch.from_numpy(V).cuda()
        # existing entry point (context workspace)
        w_ref = torch.from_numpy(w).cuda()
        h_ref, nrm_ref = G.cgs2(Vd, w_ref)
        # scratch-free entry point, twice in a row on fresh copies of w
        Vt = Vd.T.contiguous()
        for rep in range(2):
            w_na = torch.from_numpy(w).cuda()
            h_na = torch.empty(ncols, dtype=torch.complex128, device="cuda")
            nrm_na = torch.empty(1, dtype=torch.float64, device="cuda")
            s = lib.hz_cgs2_noalloc(C.c_void_p(Vt.data_ptr()), n, n, ncols, C.c_void_p(w_na.data_ptr()),
                                    C.c_void_p(h_na.data_ptr()), C.c_void_p(nrm_na.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream or None))
            assert s == hz.HZ_OK
            torch.cuda.synchronize()
            tol = 1e-12
            assert torch.allclose(h_na, h_ref, rtol=0, atol=tol * float(h_ref.abs().max()))
            assert torch.allclose(w_na, w_ref, rtol=0, atol=tol * float(abs(w).max()))
            assert abs(float(nrm_na[0]) - nrm_ref) <= tol * nrm_ref
    # the widest call the fixed scratch holds (64 columns), with V stored at a padded
    # leading dimension, against hz_cgs2 with the same layout
    ncols, ldv = 64, n + 7
    V = rng.standard_normal((n, ncols)) + 1j * rng.standard_normal((n, ncols))
    V, _ = np.linalg.qr(V)
    Vpad = np.zeros((ncols, ldv), np.complex128)           # column-major n x ncols, ld = n + 7
    Vpad[:, :n] = V.T
    Vp = torch.from_numpy(Vpad).cuda()
    w = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w_ref = torch.from_numpy(w).cuda()
    h_ref = torch.empty(ncols, dtype=torch.complex128, device="cuda")
    nrm_ref = C.c_double()
    assert lib.hz_cgs2(G.h, C.c_void_p(Vp.data_ptr()), ldv, ncols, C.c_void_p(w_ref.data_ptr()),
                       C.c_void_p(h_ref.data_ptr()), C.byref(nrm_ref)) == hz.HZ_OK
    w_na = torch.from_numpy(w).cuda()
    h_na = torch.empty(ncols, dtype=torch.complex128, device="cuda")
    nrm_na = torch.empty(1, dtype=torch.float64, device="cuda")
    s = lib.hz_cgs2_noalloc(C.c_void_p(Vp.data_ptr()), n, ldv, ncols, C.c_void_p(w_na.data_ptr()),
                            C.c_void_p(h_na.data_ptr()), C.c_void_p(nrm_na.data_ptr()),
                            C.c_void_p(torch.cuda.current_stream().cuda_stream or None))
    assert s == hz.HZ_OK
    torch.cuda.synchronize()
    tol = 1e-12
    assert torch.allclose(h_na, h_ref, rtol=0, atol=tol * float(h_ref.abs().max()))
    assert torch.allclose(w_na, w_ref, rtol=0, atol=tol * float(abs(w).max()))
    assert abs(float(nrm_na[0]) - nrm_ref.value) <= tol * nrm_ref.value
    # sizes outside [1, 64] columns are rejected
    for bad_cols in (65, 0):
        bad = lib.hz_cgs2_noalloc(C.c_void_p(Vt.data_ptr()), n, n, bad_cols, C.c_void_p(w_na.data_ptr()),
                                  C.c_void_p(h_na.data_ptr()), C.c_void_p(nrm_na.data_ptr()), None)
        assert bad == hz.HZ_ERR_ARG
    G.close()
