"""Thin ctypes binding of the hz C ABI (``include/hz.h``).

Argument marshalling only: every step of setup, factorisation and solve runs in
``libhz.so``.  Importing this module loads the library and raises if it is
missing -- there is no fallback path.  PyTorch is used only for device memory
and streams (CUDA tensors are passed by ``data_ptr()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhz.so")

HZ_OK = 0
HZ_ERR_ARG = 1
HZ_ERR_STATE = 2
HZ_ERR_OOM = 3
HZ_ERR_CUDA = 4
HZ_ERR_ZERO_PIVOT = 5
HZ_ERR_BREAKDOWN = 6
HZ_ERR_NOT_CONVERGED = 7
HZ_ERR_TIMEOUT = 8
HZ_FP64 = 0
HZ_MIXED = 1
HZ_COARSE_DIRECT = 0
HZ_COARSE_ORAS = 1
HZ_KRYLOV_PSEUDO_BLOCK = 0
HZ_KRYLOV_BLOCK = 1


class MeshDesc(C.Structure):
    _fields_ = [
        ("nv", C.c_int64), ("ne", C.c_int64), ("nf", C.c_int64),
        ("xyz", C.c_void_p), ("tets", C.c_void_p), ("faces", C.c_void_p),
        ("face_tag", C.c_void_p), ("c_re", C.c_void_p), ("c_im", C.c_void_p),
        ("order", C.c_int32),
        ("coarse_nv", C.c_int64), ("coarse_ne", C.c_int64), ("coarse_nf", C.c_int64),
        ("coarse_xyz", C.c_void_p), ("coarse_tets", C.c_void_p), ("coarse_faces", C.c_void_p),
        ("coarse_face_tag", C.c_void_p), ("fine_parent", C.c_void_p),
    ]


class Options(C.Structure):
    _fields_ = [
        ("nsub", C.c_int32), ("overlap", C.c_int32), ("levels", C.c_int32),
        ("restart", C.c_int32), ("precision", C.c_int32), ("max_iter", C.c_int32),
        ("leaf_size", C.c_int32), ("max_snode", C.c_int32),
        ("hbm_budget", C.c_uint64), ("elem_part", C.c_void_p), ("stream", C.c_void_p),
        ("block_size", C.c_int32), ("spmv_lanes", C.c_int32), ("coarse_solver", C.c_int32),
        ("coarse_maxit", C.c_int32), ("coarse_tol", C.c_double), ("recycle", C.c_int32),
        ("sweep_tasks", C.c_int32), ("bwd_chunk", C.c_int32), ("tc_wait_limit", C.c_int32),
        ("factor_group", C.c_int32), ("krylov", C.c_int32), ("tune_sweeps", C.c_int32),
        ("recycle_keep", C.c_int32),
    ]


class RhsInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("rel_residual", C.c_double)]


class Stats(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("nnz", C.c_int64), ("n_coarse", C.c_int64), ("nnz_coarse", C.c_int64),
        ("sum_ni", C.c_int64), ("nnz_local", C.c_int64), ("nnz_factor", C.c_int64),
        ("nnz_factor_coarse", C.c_int64), ("nsupernodes", C.c_int64), ("nlevels", C.c_int32),
        ("nlevels_coarse", C.c_int32), ("front_bytes", C.c_int64), ("device_bytes", C.c_int64),
        ("factor_flops", C.c_double), ("setup_seconds", C.c_double), ("factor_seconds", C.c_double),
        ("min_pivot", C.c_double), ("launches", C.c_int64), ("coarse_solves", C.c_int64),
        ("coarse_iterations", C.c_int64), ("recycle_dim", C.c_int64),
        ("fwd_levels_wide", C.c_int32), ("fwd_levels_narrow", C.c_int32), ("bwd_levels_wide", C.c_int32),
        ("bwd_levels_narrow", C.c_int32), ("bwd_split_blocks", C.c_int64), ("tc_tiles", C.c_int64),
        ("tc_multi_fronts", C.c_int64), ("tc_max_kstages", C.c_int32), ("max_snode_width", C.c_int32),
        ("sweep_chunk", C.c_int32), ("sweep_scale", C.c_double),
        ("coarse_solve_levels", C.c_int32), ("coarse_merged_chains", C.c_int32),
        ("coarse_merged_bytes", C.c_int64),
        ("solve_levels", C.c_int32), ("merged_chains", C.c_int32), ("merged_bytes", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PHASES = ["spmv", "coarse", "restrict", "local_solve", "prolong", "cgs2", "precond", "iteration"]


class Profile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("bytes", C.c_double * 8), ("flops", C.c_double * 8),
                ("launches", C.c_int64 * 8)]


class ServerOptions(C.Structure):
    _fields_ = [("hbm_budget", C.c_uint64), ("slots", C.c_int32), ("precision", C.c_int32),
                ("device", C.c_int32)]


class RequestTimes(C.Structure):
    _fields_ = [("submit_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("latency_s", C.c_double), ("nsrc", C.c_int32), ("status", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(C.Structure):
    _fields_ = [
        ("requests_done", C.c_int64), ("rhs_done", C.c_int64), ("p50_latency_s", C.c_double),
        ("p99_latency_s", C.c_double), ("rhs_per_s", C.c_double), ("analyses", C.c_int64),
        ("factorisations", C.c_int64), ("evictions", C.c_int64), ("resident_bytes", C.c_int64),
        ("peak_resident_bytes", C.c_int64), ("budget_bytes", C.c_int64), ("steps", C.c_int64),
        ("factor_seconds", C.c_double), ("launches", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every exported symbol and its signature: (restype, argtypes).
SIGNATURES = {
    "hz_setup_mesh": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "hz_factor": (C.c_int, [C.c_void_p, C.c_double]),
    "hz_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_double, C.c_void_p, C.c_int32,
                           C.POINTER(RhsInfo)]),
    "hz_point_sources": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "hz_apply_A": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hz_apply_M": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "hz_plan": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(Options), C.POINTER(Stats)]),
    "hz_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "hz_profile": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Profile)]),
    "hz_cgs2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                          C.POINTER(C.c_double)]),
    "hz_cgs2_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "hz_dense_eig": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "hz_ndofs": (C.c_int64, [C.c_void_p]),
    "hz_status_string": (C.c_char_p, [C.c_int]),
    "hz_last_error": (C.c_char_p, [C.c_void_p]),
    "hz_free": (None, [C.c_void_p]),
    "hz_server_create": (C.c_int, [C.POINTER(ServerOptions), C.POINTER(C.c_void_p)]),
    "hz_server_add_problem": (C.c_int, [C.c_void_p, C.POINTER(MeshDesc), C.POINTER(Options), C.c_double,
                                        C.POINTER(C.c_int32)]),
    "hz_server_submit": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_double,
                                   C.POINTER(C.c_uint64)]),
    "hz_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(RequestTimes)]),
    "hz_server_collect": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(RhsInfo),
                                    C.POINTER(RequestTimes)]),
    "hz_server_ndofs": (C.c_int64, [C.c_void_p, C.c_int32]),
    "hz_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "hz_server_last_error": (C.c_char_p, [C.c_void_p]),
    "hz_server_free": (None, [C.c_void_p]),
    "hz_select_evictions": (C.c_int32, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                                        C.c_int64, C.c_void_p]),
}


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"libhz.so not built ({path}); run paper_2004_06309_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


class HzError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class _MeshArrays:
    """Owns contiguous copies of the mesh arrays for the duration of a call."""

    def __init__(self, mesh, c, order, coarse=None, fine_parent=None):
        self.xyz = _c(mesh.xyz, np.float64)
        self.tets = _c(mesh.tets, np.int32)
        self.faces = _c(mesh.faces, np.int32)
        self.tag = _c(mesh.face_tag, np.int8)
        c = np.asarray(c, np.complex128)
        self.cre = _c(c.real, np.float64)
        self.cim = _c(c.imag, np.float64)
        d = MeshDesc()
        d.nv, d.ne, d.nf = len(self.xyz), len(self.tets), len(self.faces)
        d.xyz, d.tets, d.faces, d.face_tag = _ptr(self.xyz), _ptr(self.tets), _ptr(self.faces), _ptr(self.tag)
        d.c_re, d.c_im = _ptr(self.cre), _ptr(self.cim)
        d.order = int(order)
        if coarse is not None:
            self.cxyz = _c(coarse.xyz, np.float64)
            self.ctets = _c(coarse.tets, np.int32)
            self.cfaces = _c(coarse.faces, np.int32)
            self.ctag = _c(coarse.face_tag, np.int8)
            self.parent = _c(fine_parent, np.int32)
            d.coarse_nv, d.coarse_ne, d.coarse_nf = len(self.cxyz), len(self.ctets), len(self.cfaces)
            d.coarse_xyz, d.coarse_tets = _ptr(self.cxyz), _ptr(self.ctets)
            d.coarse_faces, d.coarse_face_tag = _ptr(self.cfaces), _ptr(self.ctag)
            d.fine_parent = _ptr(self.parent)
        self.desc = d


def make_options(nsub, overlap, levels, restart, precision=HZ_FP64, max_iter=2000, leaf_size=0,
                 max_snode=0, hbm_budget=0, elem_part=None, stream=0, block_size=0, spmv_lanes=0,
                 coarse_solver=0, coarse_maxit=0, coarse_tol=0.0, recycle=0, sweep_tasks=0, bwd_chunk=0,
                 tc_wait_limit=0, factor_group=0, krylov=0, tune_sweeps=0, recycle_keep=0):
    o = Options()
    o.nsub, o.overlap, o.levels, o.restart = int(nsub), int(overlap), int(levels), int(restart)
    o.precision, o.max_iter = int(precision), int(max_iter)
    o.leaf_size, o.max_snode = int(leaf_size), int(max_snode)
    o.hbm_budget = int(hbm_budget)
    part = None if elem_part is None else _c(elem_part, np.int32)
    o.elem_part = _ptr(part)
    o.stream = int(stream) if stream else None
    o.block_size = int(block_size)
    o.spmv_lanes = int(spmv_lanes)
    o.coarse_solver, o.coarse_maxit, o.coarse_tol = int(coarse_solver), int(coarse_maxit), float(coarse_tol)
    o.recycle = int(recycle)
    o.sweep_tasks, o.bwd_chunk, o.tc_wait_limit = int(sweep_tasks), int(bwd_chunk), int(tc_wait_limit)
    o.factor_group = int(factor_group)
    o.krylov = int(krylov)
    o.tune_sweeps = int(tune_sweeps)
    o.recycle_keep = int(recycle_keep)
    return o, part


def _problem_args(p):
    coarse = p.coarse if p.levels == 2 else None
    parent = p.fine_parent if p.levels == 2 else None
    return _MeshArrays(p.mesh, p.c, p.order, coarse, parent)


def plan(problem, precision=HZ_FP64, use_partition=True, **kw):
    """Host-only analysis of ``problem``: sizes and device bytes (no GPU needed)."""
    ma = _problem_args(problem)
    o, part = make_options(problem.nsub, problem.overlap, problem.levels, problem.restart, precision,
                           elem_part=problem.elem_part if use_partition else None, **kw)
    st = Stats()
    s = lib().hz_plan(C.byref(ma.desc), C.byref(o), C.byref(st))
    if s != HZ_OK:
        raise HzError(s, "hz_plan failed: " + lib().hz_status_string(s).decode())
    return st.as_dict()


class Solver:
    """One context: mesh + decomposition + factors + Krylov workspace on the GPU."""

    def __init__(self, problem, precision=HZ_FP64, stream=None, use_partition=True, **kw):
        import torch  # device memory and streams only
        self.torch = torch
        self.problem = problem
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ma = _problem_args(problem)
        o, part = make_options(problem.nsub, problem.overlap, problem.levels, problem.restart,
                               precision, elem_part=problem.elem_part if use_partition else None,
                               stream=self.stream.cuda_stream, **kw)
        h = C.c_void_p()
        s = lib().hz_setup_mesh(C.byref(ma.desc), C.byref(o), C.byref(h))
        if s != HZ_OK:
            raise HzError(s, "hz_setup_mesh failed: " + lib().hz_status_string(s).decode())
        self.h = h
        self.n = int(lib().hz_ndofs(h))

    def _check(self, s, what):
        if s not in (HZ_OK,):
            msg = lib().hz_last_error(self.h).decode()
            raise HzError(s, f"{what}: {lib().hz_status_string(s).decode()}: {msg}")

    def close(self):
        if getattr(self, "h", None):
            lib().hz_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, freq=None):
        freq = self.problem.freq if freq is None else freq
        self._check(lib().hz_factor(self.h, float(freq)), "hz_factor")

    def stats(self):
        st = Stats()
        self._check(lib().hz_get_stats(self.h, C.byref(st)), "hz_get_stats")
        return st.as_dict()

    def profile(self, reps=5):
        """Per-phase device time (ms), algorithmic bytes, flops and launches of one iteration."""
        pr = Profile()
        self._check(lib().hz_profile(self.h, int(reps), C.byref(pr)), "hz_profile")
        return {name: dict(ms=pr.ms[i], bytes=pr.bytes[i], flops=pr.flops[i], launches=pr.launches[i])
                for i, name in enumerate(PHASES)}

    def point_sources(self, pts=None, device=False):
        pts = self.problem.sources if pts is None else pts
        pts = _c(np.atleast_2d(pts), np.float64)
        if device:
            out = self.torch.empty((len(pts), self.n), dtype=self.torch.complex128, device="cuda")
            self._check(lib().hz_point_sources(self.h, _ptr(pts), len(pts), C.c_void_p(out.data_ptr()), 1),
                        "hz_point_sources")
            return out.T
        out = np.zeros((len(pts), self.n), np.complex128)
        self._check(lib().hz_point_sources(self.h, _ptr(pts), len(pts), _ptr(out), 0), "hz_point_sources")
        return out.T

    def solve(self, B, tol=None, check=True):
        """B: (n,) or (n, nrhs) numpy (host path) or CUDA tensor (device path).
        Returns (X, list of (iterations, status, rel_residual))."""
        tol = self.problem.tol if tol is None else tol
        torch = self.torch
        one = B.ndim == 1
        if isinstance(B, np.ndarray):
            Bc = np.asfortranarray(B.reshape(self.n, -1).astype(np.complex128))
            nrhs = Bc.shape[1]
            X = np.zeros((self.n, nrhs), np.complex128, order="F")
            info = (RhsInfo * nrhs)()
            s = lib().hz_solve(self.h, _ptr(Bc), nrhs, float(tol), _ptr(X), 0, info)
        else:
            Bt = B.reshape(self.n, -1).to(torch.complex128).T.contiguous()   # (nrhs, n) = column-major
            nrhs = Bt.shape[0]
            Xt = torch.empty_like(Bt)
            info = (RhsInfo * nrhs)()
            s = lib().hz_solve(self.h, C.c_void_p(Bt.data_ptr()), nrhs, float(tol),
                               C.c_void_p(Xt.data_ptr()), 1, info)
            X = Xt.T
        if check and s not in (HZ_OK, HZ_ERR_NOT_CONVERGED):
            self._check(s, "hz_solve")
        inf = [(info[j].iterations, info[j].status, info[j].rel_residual) for j in range(nrhs)]
        if one:
            X = X[:, 0]
        return X, inf

    def cgs2(self, V, w):
        """One CGS2 step: w (CUDA, length n) is orthogonalised in place against the columns of
        V (CUDA, n x ncols); returns (h, ||w||)."""
        Vt = V.T.contiguous() if V.dim() == 2 else V          # column-major storage
        ncols = Vt.shape[0]
        h = self.torch.empty(ncols, dtype=self.torch.complex128, device=w.device)
        nrm = C.c_double()
        self._check(lib().hz_cgs2(self.h, C.c_void_p(Vt.data_ptr()), self.n, ncols, C.c_void_p(w.data_ptr()),
                                  C.c_void_p(h.data_ptr()), C.byref(nrm)), "hz_cgs2")
        return h, nrm.value

    def apply_A(self, x):
        y = self.torch.empty_like(x)
        self._check(lib().hz_apply_A(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr())), "hz_apply_A")
        return y

    def apply_M(self, v):
        z = self.torch.empty_like(v)
        self._check(lib().hz_apply_M(self.h, C.c_void_p(v.data_ptr()), C.c_void_p(z.data_ptr())), "hz_apply_M")
        return z


def dense_eig(A):
    """Eigenvalues and unit right eigenvectors of a complex square matrix (hz_dense_eig)."""
    A = np.asfortranarray(np.asarray(A, np.complex128))
    n = A.shape[0]
    w = np.zeros(n, np.complex128)
    V = np.zeros((n, n), np.complex128, order="F")
    s = lib().hz_dense_eig(n, _ptr(A), _ptr(w), _ptr(V))
    if s != HZ_OK:
        raise HzError(s, "hz_dense_eig failed")
    return w, V


def select_evictions(bytes_, last_use, evictable, resident, need, budget):
    """The server's admission rule (hz_select_evictions): indices to evict, or None."""
    b = _c(bytes_, np.int64)
    lu = _c(last_use, np.float64)
    ev = _c(evictable, np.int32)
    out = np.zeros(max(len(b), 1), np.int32)
    k = lib().hz_select_evictions(len(b), _ptr(b), _ptr(lu), _ptr(ev), int(resident), int(need), int(budget),
                                  _ptr(out))
    return None if k < 0 else [int(i) for i in out[:k]]


class Server:
    """Continuous-batching solve server over cached per-(mesh, frequency) factors.

    ``add_problem`` registers a ``synth`` problem (its mesh, options and frequency);
    ``submit`` queues point sources and returns a request id at once; ``wait`` returns
    ``(X (n, nsrc), [(iterations, status, rel_residual)], times)``.  Both native threads
    (loader, solver) run inside libhz.so."""

    def __init__(self, slots=8, precision=HZ_MIXED, hbm_budget=0, device=0):
        o = ServerOptions()
        o.hbm_budget, o.slots, o.precision, o.device = int(hbm_budget), int(slots), int(precision), int(device)
        h = C.c_void_p()
        s = lib().hz_server_create(C.byref(o), C.byref(h))
        if s != HZ_OK:
            raise HzError(s, "hz_server_create failed: " + lib().hz_status_string(s).decode())
        self.h = h
        self.problems = []

    def add_problem(self, problem, freq=None, use_partition=True, **kw):
        ma = _problem_args(problem)
        o, part = make_options(problem.nsub, problem.overlap, problem.levels, problem.restart,
                               elem_part=problem.elem_part if use_partition else None, **kw)
        pid = C.c_int32()
        freq = problem.freq if freq is None else freq
        s = lib().hz_server_add_problem(self.h, C.byref(ma.desc), C.byref(o), float(freq), C.byref(pid))
        if s != HZ_OK:
            raise HzError(s, "hz_server_add_problem failed")
        self.problems.append(problem)
        return pid.value

    def submit(self, pid, pts, tol=1e-6):
        pts = _c(np.atleast_2d(pts), np.float64).reshape(-1, 3)
        rid = C.c_uint64()
        s = lib().hz_server_submit(self.h, int(pid), _ptr(pts), len(pts), float(tol), C.byref(rid))
        if s != HZ_OK:
            raise HzError(s, "hz_server_submit failed")
        return rid.value, len(pts), int(pid)

    def wait(self, req, timeout=0.0):
        """Blocks until the request finishes; returns (X (n, nsrc), info, times)."""
        rid, nsrc, pid = req
        times = RequestTimes()
        s = lib().hz_server_wait(self.h, rid, float(timeout), C.byref(times))
        if s != HZ_OK:
            raise HzError(s, "hz_server_wait: " + lib().hz_status_string(s).decode())
        n = self.ndofs(pid)
        X = np.zeros((nsrc, max(n, 0)), np.complex128)
        info = (RhsInfo * max(nsrc, 1))()
        lib().hz_server_collect(self.h, rid, _ptr(X) if n > 0 else None, info, C.byref(times))
        inf = [(info[j].iterations, info[j].status, info[j].rel_residual) for j in range(nsrc)]
        return X.T, inf, times.as_dict()

    def ndofs(self, pid):
        return int(lib().hz_server_ndofs(self.h, int(pid)))

    def stats(self):
        st = ServerStats()
        s = lib().hz_server_get_stats(self.h, C.byref(st))
        if s != HZ_OK:
            raise HzError(s, "hz_server_get_stats failed")
        return st.as_dict()

    def last_error(self):
        return lib().hz_server_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None):
            lib().hz_server_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
