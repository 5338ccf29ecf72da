"""Global step: the least-squares problem of Eq. 8 with targets fixed.

Test infrastructure only (see the package docstring).

With P_e, R and v_c fixed by the local step, Eq. 8 is quadratic in the vertex
positions:  sum_e w_e |S_e X N - P_e|^2 + k sum_{v in V_col} |x_v - v_c|^2,
S_e selecting the 4 vertices of e.  N is symmetric and idempotent and every
target is centered (P_e N = P_e), so the normal equations are

    A = sum_e w_e S_e^T N S_e + k diag(mask),   b = sum_e w_e S_e^T P_e^T + k c,

with fixed vertices moved to the right-hand side.  The three coordinate columns
share A.  The oracle solves them exactly with a sparse LU factorisation.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import N4


def laplacian(tets: np.ndarray, omega: np.ndarray, n_verts: int) -> sp.csr_matrix:
    """L_w = sum_e w_e S_e^T N S_e (entries 3/4 w on the diagonal, -1/4 w off)."""
    rows = np.repeat(tets, 4, axis=1).ravel()
    cols = np.tile(tets, (1, 4)).ravel()
    vals = (omega[:, None] * N4.ravel()[None, :]).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(n_verts, n_verts)).tocsr()


def assemble(tets, omega, P, n_verts, spring_verts, spring_targets, k):
    """Full (n_v x n_v) A and (n_v x 3) b of the normal equations."""
    A = laplacian(tets, omega, n_verts)
    b = np.zeros((n_verts, 3))
    for j in range(4):
        np.add.at(b, tets[:, j], omega[:, None] * P[:, :, j])
    if len(spring_verts):
        d = np.zeros(n_verts)
        np.add.at(d, spring_verts, k)
        A = A + sp.diags(d)
        np.add.at(b, spring_verts, k * spring_targets)
    return A.tocsr(), b


def solve(A, b, X, fixed):
    """Minimise over the free vertices with fixed ones held at X; returns the
    new positions (fixed rows copied from X)."""
    free = ~fixed.astype(bool)
    Aff = A[free][:, free].tocsc()
    Afx = A[free][:, ~free]
    rhs = b[free] - Afx @ X[~free]
    lu = spla.splu(Aff)
    Xn = X.copy()
    Xn[free] = lu.solve(rhs)
    return Xn
