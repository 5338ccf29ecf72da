"""Local projection step (Sec. II-A, Sec. III-A, Eq. 6, Eq. 7).

Test infrastructure only (see the package docstring).

For every tet with centered deformed shape X_c = V^d N and centered rest shape
T_c = V N:

* R is the rotation that best aligns R T_c with X_c (the "rotation matrix
  computed by SVD" of Eq. 1): with D = X_c T_c^T = U S V^T,
  R = U diag(1, 1, sign det(U V^T)) V^T (Kabsch; proper rotation).
* Chamber element of group g (Sec. III-A.1): every vertex of the target is the
  rest vertex scaled by cbrt(alpha_g), so P = cbrt(alpha_g) R T_c.
* Body element (Eq. 6): V_blend = (1 - w) R^T X_c + w T_c in the rest frame;
  in the deformed frame B = (1 - w) X_c + w R T_c, with w = R_omega(eps_e).
  The strain measure eps_e is the relative Procrustes misfit
  sqrt(max(0, |X_c|^2 + |T_c|^2 - 2 tr(R^T D))) / |T_c| (this library's
  reading: the paper defers R_omega and the strain to another work).
* Volume scaling (Eq. 7, read without its circular right-hand side and with
  the cube root that makes the volume ratio exact): P = s B with
  s = cbrt(Vol(T_c) / Vol(B)) when Vol(B) > 1e-3 Vol(T_c), else s = 1.
"""
from __future__ import annotations

import numpy as np

from .mesh import centered, element_matrices, signed_volume


def kabsch_rotation(D: np.ndarray):
    """Proper rotation maximising tr(R^T D) for a batch of 3x3 matrices, and
    that maximal trace sigma1 + sigma2 + d sigma3.  Uses LAPACK's SVD."""
    U, S, Vt = np.linalg.svd(D)
    d = np.sign(np.linalg.det(U @ Vt))
    d[d == 0] = 1.0
    Dg = np.zeros_like(D)
    Dg[:, 0, 0] = 1.0
    Dg[:, 1, 1] = 1.0
    Dg[:, 2, 2] = d
    R = U @ Dg @ Vt
    tr = S[:, 0] + S[:, 1] + d * S[:, 2]
    return R, tr


def w_of_eps(eps: np.ndarray, knots) -> np.ndarray:
    """Piecewise-linear stiffness table w(eps) through (eps_i, w_i), clamped
    to the end values outside the knot range."""
    xs = np.array([k[0] for k in knots], dtype=np.float64)
    ys = np.array([k[1] for k in knots], dtype=np.float64)
    return np.interp(eps, xs, ys)


def local_step(X, tets, T_c, vol0, group, alpha, knots):
    """Targets P_e (n_t, 3, 4) for the current positions X, plus R, eps_e, w_e.

    ``alpha`` are per-group volume ratios; chamber targets scale by cbrt(alpha).
    """
    X_c = centered(element_matrices(X, tets))
    D = X_c @ T_c.transpose(0, 2, 1)
    R, tr = kabsch_rotation(D)
    RT = R @ T_c
    n_t = tets.shape[0]
    P = np.empty((n_t, 3, 4))
    chamber = group >= 0
    if np.any(chamber):
        scale = np.cbrt(np.asarray(alpha, dtype=np.float64)[group[chamber]])
        P[chamber] = scale[:, None, None] * RT[chamber]
    body = ~chamber
    xx = np.einsum("nij,nij->n", X_c, X_c)
    tt = np.einsum("nij,nij->n", T_c, T_c)
    eps = np.sqrt(np.maximum(0.0, xx + tt - 2.0 * tr)) / np.sqrt(tt)
    w = w_of_eps(eps, knots)
    if np.any(body):
        wb = w[body][:, None, None]
        B = (1.0 - wb) * X_c[body] + wb * RT[body]
        volB = signed_volume(B)
        v0 = vol0[body]
        s = np.ones_like(volB)
        ok = volB > 1e-3 * v0
        s[ok] = np.cbrt(v0[ok] / volB[ok])
        P[body] = s[:, None, None] * B
    return P, R, eps, w


def elastic_energy(X, tets, P, omega):
    """sum_e omega_e |V^d N - P_e|_F^2, the element part of Eq. 8."""
    X_c = centered(element_matrices(X, tets))
    return float(np.sum(omega * np.einsum("nij,nij->n", X_c - P, X_c - P)))
