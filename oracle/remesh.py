"""Remesh trigger and progressive actuation (Sec. III-C, Algorithm 1 outer loop).

Test infrastructure only (see the package docstring).

Remeshing itself (re-tetrahedralising the chamber region) is not part of the
built path; this module computes what decides it and the outer loop around
the inner local-global loop.

* ``remesh_flags``: for every chamber element e (group >= 0) and a reference
  shape (the rest shape, or the shape at the previous outer step as in
  Algorithm 1's Vol(e_{k+1}) / Vol(e_k)), the affine map F taking the
  reference element to the deformed one, F = D_d D_r^-1 with D the matrix of
  edge vectors (v1 - v0, v2 - v0, v3 - v0).  Flag bit 1: volume change
  Vol(e_d) / Vol(e_r) = det F > alpha_max; flag bit 2: distortion, the
  largest singular value of F (the norm of the diagonal factor of its SVD)
  > d_max.  The paper writes the map "from V^d to V"; read as the map
  relating the two shapes in the direction whose stretch grows with the
  expansion the passage describes (the inverse map would flag compression).
  Body elements are never flagged.  Also returns, per chamber group, the
  chamber volume ratio sum_e Vol(e_d) / sum_e Vol(e_r).
* ``progressive``: Algorithm 1's outer loop without the remeshing step:
  outer step k = 1, 2, ... applies the ratios a_g = min(alpha_g, k alpha_step)
  (alpha_k = k alpha_max, capped at the target so the last step applies
  exactly alpha), runs ``n_inner`` inner iterations from the previous shape
  and spring records, then records the flags against the previous outer
  step's shape and the chamber volume ratios against the rest shape; it stops
  once every group's target is applied (or after ``max_outer`` steps).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from . import loop, springs

FLAG_VOLUME = 1
FLAG_DISTORTION = 2


def edge_matrices(X: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """(n_t, 3, 3): columns v1 - v0, v2 - v0, v3 - v0."""
    V = X[tets]                          # (n_t, 4, 3)
    return (V[:, 1:, :] - V[:, :1, :]).transpose(0, 2, 1)


def remesh_flags(X, ref, tets, group, alpha_max=4.0, d_max=4.0):
    """Returns (flags uint8 (n_t,), ratio (n_t,), sigma_max (n_t,), group_volume_ratio dict g -> ratio)."""
    tets = np.asarray(tets, dtype=np.int64)
    group = np.asarray(group)
    n_t = tets.shape[0]
    flags = np.zeros(n_t, np.uint8)
    ratio = np.zeros(n_t)
    smax = np.zeros(n_t)
    ch = np.nonzero(group >= 0)[0]
    gvr = {}
    if ch.size:
        Dd = edge_matrices(np.asarray(X, np.float64), tets[ch])
        Dr = edge_matrices(np.asarray(ref, np.float64), tets[ch])
        F = Dd @ np.linalg.inv(Dr)
        ratio[ch] = np.linalg.det(F)
        smax[ch] = np.linalg.svd(F, compute_uv=False)[:, 0]
        flags[ch] = (np.where(ratio[ch] > alpha_max, FLAG_VOLUME, 0) |
                     np.where(smax[ch] > d_max, FLAG_DISTORTION, 0)).astype(np.uint8)
        vd = np.linalg.det(Dd) / 6.0
        vr = np.linalg.det(Dr) / 6.0
        for g in np.unique(group[ch]):
            sel = group[ch] == g
            gvr[int(g)] = float(vd[sel].sum() / vr[sel].sum())
    return flags, ratio, smax, gvr


@dataclass
class OuterRecord:
    k: int
    applied: np.ndarray          # ratios applied at this outer step (per group)
    n_volume: int                # chamber elements flagged for volume change
    n_distortion: int            # chamber elements flagged for distortion
    n_flagged: int               # chamber elements with any flag
    chamber_volume_ratio: dict   # per group, against the rest shape


def progressive(m, alpha_target, alpha_step, n_inner, max_outer=64, alpha_max=4.0, d_max=4.0,
                prep=None):
    """Algorithm 1's outer loop (no remeshing) on a generator ``Mesh``.
    Returns (X, records)."""
    prep = prep or loop.prepare(m.rest, m.tets, m.group, m.fixed)
    target = np.asarray(alpha_target, dtype=np.float64)
    X = np.array(m.rest, dtype=np.float64)
    st = springs.SpringState.empty(prep.query.shape[0])
    spheres = np.zeros((0, 4)) if m.spheres is None else np.asarray(m.spheres, np.float64)
    recs: List[OuterRecord] = []
    for k in range(1, max_outer + 1):
        applied = np.minimum(target, k * alpha_step)
        Xk = X.copy()
        for _ in range(n_inner):
            X, st, _rec, _ps, _po = loop.iterate(prep, X, st, applied, spheres, m.w_knots, m.k_spring, m.eps,
                                                 m.collision)
        flags, _r, _s, _ = remesh_flags(X, Xk, m.tets, m.group, alpha_max, d_max)
        _f, _r2, _s2, gvr = remesh_flags(X, m.rest, m.tets, m.group, alpha_max, d_max)
        recs.append(OuterRecord(k, applied, int(np.count_nonzero(flags & FLAG_VOLUME)),
                                int(np.count_nonzero(flags & FLAG_DISTORTION)), int(np.count_nonzero(flags)), gvr))
        if np.all(applied == target):
            break
    return X, recs
