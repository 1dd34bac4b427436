"""Independent quadrature used only by tests to pin the oracle's exact integrals.

Collapsed-coordinate (Duffy) tensor Gauss-Legendre rules on the reference
tetrahedron and triangle: exact for polynomials up to degree 2q-1 - (the
Jacobian degree), here used with q large enough for every integrand.
"""
import numpy as np


def tet_rule(q=8):
    """Points as barycentric coordinates (npts, 4) and weights summing to 1."""
    g, w = np.polynomial.legendre.leggauss(q)
    t = 0.5 * (g + 1.0)
    wt = 0.5 * w
    U, V, W = np.meshgrid(t, t, t, indexing="ij")
    WU, WV, WW = np.meshgrid(wt, wt, wt, indexing="ij")
    x = U
    y = V * (1 - U)
    z = W * (1 - U) * (1 - V)
    jac = (1 - U) ** 2 * (1 - V)
    wts = (WU * WV * WW * jac).ravel() * 6.0          # normalise: reference volume 1/6
    lam = np.stack([1 - x - y - z, x, y, z], axis=-1).reshape(-1, 4)
    return lam, wts


def tri_rule(q=8):
    g, w = np.polynomial.legendre.leggauss(q)
    t = 0.5 * (g + 1.0)
    wt = 0.5 * w
    U, V = np.meshgrid(t, t, indexing="ij")
    WU, WV = np.meshgrid(wt, wt, indexing="ij")
    x = U
    y = V * (1 - U)
    jac = 1 - U
    wts = (WU * WV * jac).ravel() * 2.0
    lam = np.stack([1 - x - y, x, y], axis=-1).reshape(-1, 3)
    return lam, wts
