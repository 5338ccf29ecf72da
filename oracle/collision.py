"""Brute-force collision detection (Sec. II-B, Eq. 3, Eq. 4).

Test infrastructure only (see the package docstring).

The paper's plain definition: check every tetrahedron for every surface vertex
(Sec. II-B).  Following Eq. 3 (read as "no boundary vertex lies inside any
other element", the equation labels being swapped in the text), the self set is

    P_self = {(v, e) : v a non-fixed boundary vertex, v not a vertex of e,
                        v strictly inside e},

"strictly inside" meaning all four barycentric signs are positive, evaluated
exactly (a point on a face, edge or vertex is not inside).  Eq. 4's obstacle
set for spheres (c_j, r_j) is

    P_obs = {(v, j) : |x_v - c_j|^2 < r_j^2},

evaluated in FP64 in the fixed order ((dx*dx + dy*dy) + dz*dz) < r*r.

The orientation sign uses Shewchuk's floating-point filter (Shewchuk 1997,
"Adaptive precision floating-point arithmetic and fast robust geometric
predicates": error bound (7 + 56 eps) eps times the permanent, eps = 2^-53)
and falls back to exact rational arithmetic (``fractions.Fraction``) when the
filter cannot decide.  Exact rejections come first: a point strictly inside a tet lies in the tet's
closed bounding box, and so in the tet's slab range along one axis.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

_EPS = 2.0 ** -53
_O3D_BOUND_A = (7.0 + 56.0 * _EPS) * _EPS


def _orient_filter(q0, q1, q2, q3):
    """det[q1-q0, q2-q0, q3-q0] in double plus Shewchuk's error bound."""
    u = q1 - q0
    v = q2 - q0
    w = q3 - q0
    m1 = v[:, 1] * w[:, 2]
    m2 = v[:, 2] * w[:, 1]
    m3 = w[:, 1] * u[:, 2]
    m4 = w[:, 2] * u[:, 1]
    m5 = u[:, 1] * v[:, 2]
    m6 = u[:, 2] * v[:, 1]
    det = u[:, 0] * (m1 - m2) + v[:, 0] * (m3 - m4) + w[:, 0] * (m5 - m6)
    perm = ((np.abs(m1) + np.abs(m2)) * np.abs(u[:, 0])
            + (np.abs(m3) + np.abs(m4)) * np.abs(v[:, 0])
            + (np.abs(m5) + np.abs(m6)) * np.abs(w[:, 0]))
    return det, _O3D_BOUND_A * perm


def orient_exact_one(q0, q1, q2, q3) -> int:
    """Exact sign of det[q1-q0, q2-q0, q3-q0] for double inputs."""
    a = [Fraction(float(x)) for x in q0]
    b = [Fraction(float(x)) for x in q1]
    c = [Fraction(float(x)) for x in q2]
    d = [Fraction(float(x)) for x in q3]
    u = [b[i] - a[i] for i in range(3)]
    v = [c[i] - a[i] for i in range(3)]
    w = [d[i] - a[i] for i in range(3)]
    det = (u[0] * (v[1] * w[2] - v[2] * w[1])
           + v[0] * (w[1] * u[2] - w[2] * u[1])
           + w[0] * (u[1] * v[2] - u[2] * v[1]))
    return (det > 0) - (det < 0)


def orient_sign(q0, q1, q2, q3) -> np.ndarray:
    """Exact signs (-1, 0, +1) of det[q1-q0, q2-q0, q3-q0], batched."""
    det, bound = _orient_filter(q0, q1, q2, q3)
    sign = np.where(det > bound, 1, np.where(-det > bound, -1, 0)).astype(np.int8)
    unsure = np.nonzero(~((det > bound) | (-det > bound)))[0]
    for i in unsure:
        sign[i] = orient_exact_one(q0[i], q1[i], q2[i], q3[i])
    return sign


def strictly_inside(p, a, b, c, d) -> np.ndarray:
    """p strictly inside the positively oriented tet (a, b, c, d): all four
    sub-tets obtained by replacing one vertex with p have positive volume."""
    s0 = orient_sign(p, b, c, d)
    s1 = orient_sign(a, p, c, d)
    s2 = orient_sign(a, b, p, d)
    s3 = orient_sign(a, b, c, p)
    return (s0 > 0) & (s1 > 0) & (s2 > 0) & (s3 > 0)


def self_pairs(X: np.ndarray, tets: np.ndarray, query: np.ndarray, chunk: int = 64,
               n_slabs: int = 64) -> np.ndarray:
    """All (v, e) with v in ``query`` strictly inside tet e not containing v,
    sorted by (v, e); returns an (m, 2) int64 array.

    Every (vertex, tet) pair is decided by the exact predicate after two exact
    rejections: the tet's closed bounding box, and before it a 1-D slab test
    along the longest axis (p can lie in a tet only if lo_a <= p_a <= hi_a, and
    floor((x - base) / width) is monotone in x, so such a tet is listed in p's
    slab)."""
    E = X[tets]                      # (n_t, 4, 3)
    lo = E.min(axis=1)
    hi = E.max(axis=1)
    query = np.asarray(query, dtype=np.int64)
    if query.size == 0 or tets.shape[0] == 0:
        return np.zeros((0, 2), dtype=np.int64)
    ext = hi.max(axis=0) - lo.min(axis=0)
    ax = int(np.argmax(ext))
    base = float(lo[:, ax].min())
    width = max(float(ext[ax]) / n_slabs, 1e-300)
    s_lo = np.floor((lo[:, ax] - base) / width).astype(np.int64)
    s_hi = np.floor((hi[:, ax] - base) / width).astype(np.int64)
    s_q = np.floor((X[query, ax] - base) / width).astype(np.int64)
    out = []
    for sl in np.unique(s_q):
        cand = np.nonzero((s_lo <= sl) & (s_hi >= sl))[0]
        if cand.size == 0:
            continue
        qs = query[s_q == sl]
        lo_c, hi_c = lo[cand], hi[cand]
        for s in range(0, qs.shape[0], chunk):
            vs = qs[s:s + chunk]
            p = X[vs]                    # (c, 3)
            box = np.all((p[:, None, :] >= lo_c[None]) & (p[:, None, :] <= hi_c[None]), axis=2)
            vi, ci = np.nonzero(box)
            if vi.size == 0:
                continue
            v = vs[vi]
            ei = cand[ci]
            keep = np.all(tets[ei] != v[:, None], axis=1)
            v, ei = v[keep], ei[keep]
            if v.size == 0:
                continue
            t = tets[ei]
            ins = strictly_inside(X[v], X[t[:, 0]], X[t[:, 1]], X[t[:, 2]], X[t[:, 3]])
            if np.any(ins):
                out.append(np.stack([v[ins], ei[ins]], axis=1))
    if not out:
        return np.zeros((0, 2), dtype=np.int64)
    pairs = np.concatenate(out).astype(np.int64)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order]


def sphere_pairs(X: np.ndarray, query: np.ndarray, spheres: np.ndarray) -> np.ndarray:
    """All (v, j) with |x_v - c_j|^2 < r_j^2 in the fixed FP64 order, sorted."""
    out = []
    query = np.asarray(query, dtype=np.int64)
    p = X[query]
    for j in range(spheres.shape[0]):
        cx, cy, cz, r = (float(t) for t in spheres[j])
        dx = p[:, 0] - cx
        dy = p[:, 1] - cy
        dz = p[:, 2] - cz
        d2 = (dx * dx + dy * dy) + dz * dz
        ins = d2 < r * r
        if np.any(ins):
            out.append(np.stack([query[ins], np.full(int(ins.sum()), j)], axis=1))
    if not out:
        return np.zeros((0, 2), dtype=np.int64)
    pairs = np.concatenate(out).astype(np.int64)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order]
