"""Oracle: one- and two-level ORAS preconditioners and the full solve.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

One level, Eq. (4):   M_1^{-1} t = sum_i R_i^T D_i A_i^{-1} R_i t.
Two levels, Eq. (3):  M^{-1} v = M_1^{-1} (v - A y) + y,  y = Z E^{-1} Z^T v.

The local and coarse inverses are applied with a sparse direct solver
(SuperLU through scipy), the "direct solver" of the method; they are
computed once per frequency.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import coarse, dd, fem, krylov


class OracleSolver:
    """``coarse_solver="direct"`` solves E by a sparse direct solver; ``"oras"`` by the
    paper's inner GMRES with one-level ORAS on the coarse mesh (tolerance
    ``coarse_tol``, at most ``coarse_m`` iterations)."""

    def __init__(self, problem, robin=True, coarse_solver="direct", coarse_tol=1e-2, coarse_m=30):
        self.p = problem
        self.robin = robin
        self.coarse_solver = coarse_solver
        self.coarse_tol = coarse_tol
        self.coarse_m = coarse_m
        self.coarse_its = []
        self.A, self.dm, self.ddofs = fem.global_system(problem)
        self.n = self.dm.n
        self.subs = dd.grow_subdomains(problem.mesh, problem.elem_part, problem.nsub,
                                       problem.overlap, self.dm)
        self.Z = None
        if problem.levels == 2:
            self.Z, self.cdm, self.ckeep = coarse.interpolation(problem, self.dm)
            if coarse_solver == "oras":
                self.cor = coarse.CoarseORAS(problem, self.dm, self.Z, self.cdm, self.ckeep)
        self.freq = None

    def factor(self, freq=None):
        freq = self.p.freq if freq is None else freq
        if freq != self.p.freq:
            dm, K, Mp, Bp = fem.assemble_parts(self.p.mesh, self.p.c, self.p.order, dm=self.dm)
            self.A = fem.apply_dirichlet(fem.helmholtz_matrix(K, Mp, Bp, freq), self.ddofs)
        dd.build_local_matrices(self.p, self.dm, self.subs, self.ddofs, freq, robin=self.robin)
        self.lu = [spla.splu(s.A.tocsc()) for s in self.subs]
        if self.Z is not None:
            self.E = coarse.coarse_operator(self.Z, self.A)
            if self.coarse_solver == "oras":
                self.cor.factor(freq)
            else:
                self.Elu = spla.splu(self.E.tocsc())
        self.freq = freq

    # --- operators -------------------------------------------------------
    def apply_A(self, x):
        return self.A @ x

    def apply_M1(self, t):
        z = np.zeros(self.n, np.complex128)
        for s, lu in zip(self.subs, self.lu):
            xi = lu.solve(t[s.dofs])
            z[s.dofs] += s.D * xi
        return z

    def coarse_correction(self, v):
        rH = self.Z.T @ v
        if self.coarse_solver == "oras":
            yH, its = self.cor.solve(self.E, rH, self.coarse_tol, self.coarse_m)
            self.coarse_its.append(its)
            return self.Z @ yH
        return self.Z @ self.Elu.solve(rH)

    def apply_M(self, v):
        if self.Z is None:
            return self.apply_M1(v)
        y = self.coarse_correction(v)
        t = v - self.A @ y
        return self.apply_M1(t) + y

    # --- inputs / solve --------------------------------------------------
    def rhs(self, pts=None):
        pts = self.p.sources if pts is None else pts
        return fem.point_sources(self.p, self.dm, self.ddofs, pts)

    def solve(self, B, tol=None, m=None, maxit=2000, history=None):
        tol = self.p.tol if tol is None else tol
        m = self.p.restart if m is None else m
        B = np.asarray(B, np.complex128)
        one = B.ndim == 1
        if one:
            B = B[:, None]
        X = np.zeros_like(B)
        its, rels, conv = [], [], []
        for j in range(B.shape[1]):
            x, it, rel, ok = krylov.fgmres(self.apply_A, self.apply_M, B[:, j], tol=tol, m=m,
                                           maxit=maxit, history=history)
            X[:, j] = x
            its.append(it)
            rels.append(rel)
            conv.append(ok)
        if one:
            return X[:, 0], its[0], rels[0], conv[0]
        return X, its, rels, conv
