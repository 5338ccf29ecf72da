"""Virtual-spring collision response (Sec. II-C, Eq. 5, Sec. III-A.3).

Test infrastructure only (see the package docstring).

Each non-fixed boundary vertex v carries at most one spring (v, v_c) with
energy k |v - v_c|^2 (Eq. 5).  Per iteration, after detection:

* v inside an obstacle sphere: an obstacle spring to the closest point of the
  sphere grown by eps, v_c = c_j + (r_j + eps) u, u = (x_v - c_j)/|x_v - c_j|
  (u = -n(v) when x_v = c_j); with several spheres the nearest surface
  (smallest |x_v - c_j| - r_j, then lowest j) wins.  The obstacle takes
  precedence over self-collision.
* else v in a self pair: a self spring.  The correspondence is found by
  searching from x_v along -n(v) (Sec. II-C): the ray hits the boundary faces
  f not containing v whose outward normal points along the ray
  ((-n(v)) . n_f > 0, "exit" faces); the hit with the smallest t > 0 and
  inclusive barycentrics wins (ties: lower face id), using the Moller-Trumbore
  ray-triangle test (Moller and Trumbore 1997).  With no hit, the closest
  point over boundary faces not containing v is used.  The stored record is
  (face f, barycentrics beta1, beta2) and v_c = b + eps n_f, b the hit point
  and n_f the unit face normal.
* v inside the tetrahedral obstacle (``oracle.obstacle``): a spring to the
  closest point of the obstacle's boundary offset by eps along that face's
  outward normal (Sec. II-C), record (face, beta1, beta2).  When v is inside
  spheres and the mesh obstacle, the obstacle whose signed surface distance
  is smallest wins (|x_v - c_j| - r_j for a sphere, minus the distance to the
  boundary for the mesh; spheres first on ties).
* else an existing spring is released or kept by the paper's release
  condition (v outside the obstacle and its normal distance to the contact
  surface above eps), read as: obstacle spring released iff
  |x_v - c_j| - r_j > eps; self spring released iff n_f . (x_v - b) > eps,
  with b and n_f re-evaluated from the stored (f, beta) at the current
  positions.  A kept spring is re-targeted from its stored record.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KIND_SELF = 0
KIND_OBSTACLE = 1       # sphere obstacle: face = sphere id
KIND_MESH_OBSTACLE = 2  # tetrahedral obstacle: face = obstacle boundary face id, bary on it


@dataclass
class SpringState:
    """Per-query-vertex spring records (query = sorted non-fixed surface verts)."""

    active: np.ndarray   # (n_q,) bool
    kind: np.ndarray     # (n_q,) int8: 0 self, 1 obstacle
    face: np.ndarray     # (n_q,) int64: boundary face id, or sphere id
    bary: np.ndarray     # (n_q, 2) float64
    target: np.ndarray   # (n_q, 3) float64
    fallback: np.ndarray = None  # (n_q,) bool: this update's self target came from the closest point

    def __post_init__(self):
        if self.fallback is None:
            self.fallback = np.zeros(self.active.shape[0], bool)

    @staticmethod
    def empty(n_q: int) -> "SpringState":
        return SpringState(np.zeros(n_q, bool), np.zeros(n_q, np.int8), np.full(n_q, -1, np.int64),
                           np.zeros((n_q, 2)), np.zeros((n_q, 3)))

    def copy(self) -> "SpringState":
        return SpringState(self.active.copy(), self.kind.copy(), self.face.copy(),
                           self.bary.copy(), self.target.copy(), self.fallback.copy())


def _cross_rows(a, b):
    """Row-wise cross products of (n, 3) arrays, written out component by
    component (a_y b_z - a_z b_y, a_z b_x - a_x b_z, a_x b_y - a_y b_x)."""
    return np.stack([a[..., 1] * b[..., 2] - a[..., 2] * b[..., 1],
                     a[..., 2] * b[..., 0] - a[..., 0] * b[..., 2],
                     a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]], axis=-1)


def _dot_rows(a, b):
    """Row-wise dot products a_x b_x + a_y b_y + a_z b_z, summed left to right."""
    return a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1] + a[..., 2] * b[..., 2]


def _ray_triangles(o, d, q0, q1, q2):
    """Moller-Trumbore (Moller and Trumbore 1997) for one ray o + t d against
    many triangles (rows of q0, q1, q2): (hit, t, beta1, beta2) per triangle,
    barycentrics inclusive, t > 0; a triangle parallel to the ray (det = 0)
    is not hit."""
    e1 = q1 - q0
    e2 = q2 - q0
    pv = _cross_rows(np.broadcast_to(d, e2.shape), e2)
    det = _dot_rows(e1, pv)
    ok = det != 0.0
    inv = np.zeros_like(det)
    inv[ok] = 1.0 / det[ok]
    tv = o[None, :] - q0
    b1 = _dot_rows(tv, pv) * inv
    qv = _cross_rows(tv, e1)
    b2 = _dot_rows(np.broadcast_to(d, qv.shape), qv) * inv
    t = _dot_rows(e2, qv) * inv
    hit = ok & (b1 >= 0.0) & (b2 >= 0.0) & (b1 + b2 <= 1.0) & (t > 0.0)
    return hit, t, b1, b2


def _closest_on_segment(p, a, b):
    ab = b - a
    den = float(np.dot(ab, ab))
    s = 0.0 if den == 0.0 else min(1.0, max(0.0, float(np.dot(p - a, ab)) / den))
    return a + s * ab, s


def closest_point_triangle(p, q0, q1, q2):
    """Closest point of triangle q0 q1 q2 to p and its barycentrics (b1, b2)
    (weights of q1 and q2): the plane projection when it falls inside,
    otherwise the nearest of the three edge projections."""
    e1 = q1 - q0
    e2 = q2 - q0
    n = np.cross(e1, e2)
    nn = float(np.dot(n, n))
    if nn > 0.0:
        x = p - (float(np.dot(p - q0, n)) / nn) * n
        # barycentrics of x by the 2x2 normal equations
        d11, d12, d22 = float(np.dot(e1, e1)), float(np.dot(e1, e2)), float(np.dot(e2, e2))
        r = x - q0
        r1, r2 = float(np.dot(r, e1)), float(np.dot(r, e2))
        den = d11 * d22 - d12 * d12
        b1 = (d22 * r1 - d12 * r2) / den
        b2 = (d11 * r2 - d12 * r1) / den
        if b1 >= 0.0 and b2 >= 0.0 and b1 + b2 <= 1.0:
            return x, b1, b2
    best = None
    for (a, b, wa) in ((q0, q1, 0), (q1, q2, 1), (q2, q0, 2)):
        c, s = _closest_on_segment(p, a, b)
        dd = float(np.dot(p - c, p - c))
        if wa == 0:
            bb = (s, 0.0)
        elif wa == 1:
            bb = (1.0 - s, s)
        else:
            bb = (0.0, 1.0 - s)
        if best is None or dd < best[0]:
            best = (dd, c, bb)
    return best[1], best[2][0], best[2][1]


def _face_point(X, face_verts, b1, b2):
    q0, q1, q2 = X[face_verts[0]], X[face_verts[1]], X[face_verts[2]]
    return (1.0 - b1 - b2) * q0 + b1 * q1 + b2 * q2


def _face_unit_normal(X, face_verts):
    q0, q1, q2 = X[face_verts[0]], X[face_verts[1]], X[face_verts[2]]
    n = np.cross(q1 - q0, q2 - q0)
    return n / np.linalg.norm(n)


def ray_cast_target(X, v, nrm_v, faces, fnormals):
    """Self-collision correspondence of vertex v: (face id, b1, b2, fell back
    to the closest point).

    Every exit face (not containing v, outward normal along the ray -n(v)) is
    tested; among the hits the smallest t wins, then the lowest face id.  With
    no hit, the closest point over all boundary faces not containing v wins
    (smallest squared distance, then the lowest face id)."""
    d = -nrm_v
    o = X[v]
    free = np.all(faces != v, axis=1)
    cand = np.nonzero((fnormals @ d > 0.0) & free)[0]
    if cand.size:
        hit, t, b1, b2 = _ray_triangles(o, d, X[faces[cand, 0]], X[faces[cand, 1]], X[faces[cand, 2]])
        if np.any(hit):
            h = np.nonzero(hit)[0]
            k = h[np.lexsort((cand[h], t[h]))[0]]
            return int(cand[k]), float(b1[k]), float(b2[k]), False
    # no exit face hit: closest point over boundary faces not containing v
    best = None
    for f in np.nonzero(free)[0]:
        x, b1, b2 = closest_point_triangle(o, X[faces[f, 0]], X[faces[f, 1]], X[faces[f, 2]])
        dd = float(np.dot(o - x, o - x))
        if best is None or dd < best[0]:
            best = (dd, int(f), b1, b2)
    return best[1], best[2], best[3], True


def _sphere_target(x, c, r, eps, nrm_v):
    u = x - c
    nu = float(np.linalg.norm(u))
    u = -nrm_v if nu == 0.0 else u / nu
    return c + (r + eps) * u


def update_springs(X, query, prev: SpringState, self_pairs, sphere_pairs, spheres,
                   faces, vnormals, eps, obstacle=None, obstacle_pairs=None) -> SpringState:
    """One spring update (create, re-target or release) for every query vertex."""
    from . import obstacle as obst

    st = prev.copy()
    st.fallback[:] = False
    fn = np.cross(X[faces[:, 1]] - X[faces[:, 0]], X[faces[:, 2]] - X[faces[:, 0]])
    in_self = np.zeros(query.shape[0], bool)
    in_mesh = np.zeros(query.shape[0], bool)
    pos = {int(v): i for i, v in enumerate(query)}
    for v, _e in self_pairs:
        in_self[pos[int(v)]] = True
    if obstacle_pairs is not None:
        for v, _e in obstacle_pairs:
            in_mesh[pos[int(v)]] = True
    obs_hits = {}
    for v, j in sphere_pairs:
        obs_hits.setdefault(pos[int(v)], []).append(int(j))
    for i, v in enumerate(query):
        x = X[v]
        sphere = None
        if i in obs_hits:
            js = obs_hits[i]
            dists = [float(np.linalg.norm(x - spheres[j, :3])) - float(spheres[j, 3]) for j in js]
            k = int(np.argmin(dists))
            sphere = (js[k], dists[k])
        mesh_hit = None
        if in_mesh[i]:
            f, b1, b2, d2 = obst.closest_boundary_point(x, obstacle)
            mesh_hit = (f, b1, b2, -float(np.sqrt(d2)))
        if sphere is not None and (mesh_hit is None or sphere[1] <= mesh_hit[3]):
            j = sphere[0]
            st.active[i] = True
            st.kind[i] = KIND_OBSTACLE
            st.face[i] = j
            st.bary[i] = 0.0
            st.target[i] = _sphere_target(x, spheres[j, :3], float(spheres[j, 3]), eps, vnormals[v])
        elif mesh_hit is not None:
            f, b1, b2, _d = mesh_hit
            st.active[i] = True
            st.kind[i] = KIND_MESH_OBSTACLE
            st.face[i] = f
            st.bary[i] = (b1, b2)
            st.target[i] = obst.target(obstacle, f, b1, b2, eps)
        elif in_self[i]:
            f, b1, b2, fb = ray_cast_target(X, v, vnormals[v], faces, fn)
            st.fallback[i] = fb
            st.active[i] = True
            st.kind[i] = KIND_SELF
            st.face[i] = f
            st.bary[i] = (b1, b2)
            b = _face_point(X, faces[f], b1, b2)
            st.target[i] = b + eps * _face_unit_normal(X, faces[f])
        elif st.active[i]:
            if st.kind[i] == KIND_OBSTACLE:
                j = int(st.face[i])
                c, r = spheres[j, :3], float(spheres[j, 3])
                if float(np.linalg.norm(x - c)) - r > eps:
                    st.active[i] = False
                else:
                    st.target[i] = _sphere_target(x, c, r, eps, vnormals[v])
            elif st.kind[i] == KIND_MESH_OBSTACLE:
                f = int(st.face[i])
                b1, b2 = st.bary[i]
                if obst.released(x, obstacle, f, b1, b2, eps):
                    st.active[i] = False
                else:
                    st.target[i] = obst.target(obstacle, f, b1, b2, eps)
            else:
                f = int(st.face[i])
                b = _face_point(X, faces[f], st.bary[i, 0], st.bary[i, 1])
                nf = _face_unit_normal(X, faces[f])
                if float(np.dot(nf, x - b)) > eps:
                    st.active[i] = False
                else:
                    st.target[i] = b + eps * nf
    st.face[~st.active] = -1
    st.bary[~st.active] = 0.0
    st.target[~st.active] = 0.0
    return st


def spring_energy(X, query, st: SpringState, k):
    """k sum_{v in V_col} |x_v - v_c|^2 (Eq. 5 summed, Eq. 8 second term)."""
    a = st.active
    d = X[query[a]] - st.target[a]
    return float(k * np.sum(d * d))
