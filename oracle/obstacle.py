"""Rigid tetrahedral obstacles (Sec. II-B, Eq. 4; Sec. II-C).

Test infrastructure only (see the package docstring).

The paper builds AABB trees over the robot M and over the obstacle O_obs,
whose leaves hold one tetrahedron each (Sec. II-B), so the obstacle is a
tetrahedral mesh like the robot.  Eq. 4 (M does not intersect O_obs) is read
for the robot's non-fixed boundary vertices: the obstacle pairs are

    P_mesh = {(v, e) : v a non-fixed robot boundary vertex, e an obstacle
                       tetrahedron, v strictly inside e (exact signs)},

and a robot vertex inside the obstacle gets a spring to the closest point of
the obstacle's boundary, offset by eps along that face's outward normal
(Sec. II-C: "the closest point on the boundary of the collided region", the
boundary offset by eps).  The closest point is taken over all boundary
triangles of the obstacle; among equal squared distances the lowest face id
wins.  A kept spring is released when the vertex lies more than eps outside
the stored face point along the face normal, as for self springs.  The
obstacle does not move.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import collision, mesh
from .springs import _cross_rows, _dot_rows


@dataclass
class Obstacle:
    X: np.ndarray       # (n_o, 3) fixed positions
    tets: np.ndarray    # (m, 4) positively oriented
    faces: np.ndarray   # (n_f, 3) boundary faces, outward, ordered by (tet, local face)


def prepare(X, tets) -> Obstacle:
    tets = np.asarray(tets, dtype=np.int64)
    return Obstacle(np.asarray(X, dtype=np.float64), tets, mesh.boundary_faces(tets))


def pairs(Xr: np.ndarray, query: np.ndarray, obs: Obstacle) -> np.ndarray:
    """All (v, e) with robot vertex v in ``query`` strictly inside obstacle
    tet e, sorted by (v, e); the exact test of the self-collision check on the
    robot and obstacle positions side by side (no obstacle tet contains a
    robot vertex id, so none is skipped)."""
    n = Xr.shape[0]
    Xc = np.concatenate([Xr, obs.X])
    return collision.self_pairs(Xc, obs.tets + n, query)


def closest_points(p: np.ndarray, q0: np.ndarray, q1: np.ndarray, q2: np.ndarray):
    """Closest points of many triangles (rows of q0, q1, q2) to one point p,
    with their barycentric weights (b1, b2) of q1, q2: the projection onto the
    triangle's plane when it falls inside, otherwise the nearest of the three
    edge projections (the rule of ``springs.closest_point_triangle``, written
    for arrays)."""
    e1 = q1 - q0
    e2 = q2 - q0
    nrm = _cross_rows(e1, e2)
    nn = _dot_rows(nrm, nrm)
    ok = nn > 0.0
    t = np.zeros_like(nn)
    t[ok] = _dot_rows(p[None, :] - q0, nrm)[ok] / nn[ok]
    x = p[None, :] - t[:, None] * nrm
    d11, d12, d22 = _dot_rows(e1, e1), _dot_rows(e1, e2), _dot_rows(e2, e2)
    r = x - q0
    r1, r2 = _dot_rows(r, e1), _dot_rows(r, e2)
    den = d11 * d22 - d12 * d12
    with np.errstate(divide="ignore", invalid="ignore"):
        c1 = (d22 * r1 - d12 * r2) / den
        c2 = (d11 * r2 - d12 * r1) / den
    inside = ok & (c1 >= 0.0) & (c2 >= 0.0) & (c1 + c2 <= 1.0)
    best_x = np.where(inside[:, None], x, 0.0)
    best_b1 = np.where(inside, c1, 0.0)
    best_b2 = np.where(inside, c2, 0.0)
    best_d = np.where(inside, np.inf, np.inf)
    # edges (q0, q1), (q1, q2), (q2, q0), first one wins ties
    for k, (a, b) in enumerate(((q0, q1), (q1, q2), (q2, q0))):
        ab = b - a
        den_e = _dot_rows(ab, ab)
        with np.errstate(divide="ignore", invalid="ignore"):
            s = np.where(den_e == 0.0, 0.0, np.clip(_dot_rows(p[None, :] - a, ab) / den_e, 0.0, 1.0))
        c = a + s[:, None] * ab
        dd = _dot_rows(p[None, :] - c, p[None, :] - c)
        if k == 0:
            bb1, bb2 = s, np.zeros_like(s)
        elif k == 1:
            bb1, bb2 = 1.0 - s, s
        else:
            bb1, bb2 = np.zeros_like(s), 1.0 - s
        take = ~inside & (dd < best_d)
        best_d = np.where(take, dd, best_d)
        best_x = np.where(take[:, None], c, best_x)
        best_b1 = np.where(take, bb1, best_b1)
        best_b2 = np.where(take, bb2, best_b2)
    return best_x, best_b1, best_b2


def closest_boundary_point(x: np.ndarray, obs: Obstacle):
    """(face id, b1, b2, squared distance) of the closest point of the
    obstacle's boundary to x; ties go to the lowest face id."""
    f = obs.faces
    c, b1, b2 = closest_points(x, obs.X[f[:, 0]], obs.X[f[:, 1]], obs.X[f[:, 2]])
    d2 = _dot_rows(x[None, :] - c, x[None, :] - c)
    k = int(np.lexsort((np.arange(f.shape[0]), d2))[0])
    return k, float(b1[k]), float(b2[k]), float(d2[k])


def face_point_and_normal(obs: Obstacle, f: int, b1: float, b2: float):
    q0, q1, q2 = (obs.X[obs.faces[f, k]] for k in range(3))
    n = np.cross(q1 - q0, q2 - q0)
    return (1.0 - b1 - b2) * q0 + b1 * q1 + b2 * q2, n / np.linalg.norm(n)


def target(obs: Obstacle, f: int, b1: float, b2: float, eps: float) -> np.ndarray:
    """Spring target: the face point offset by eps along the outward normal."""
    b, n = face_point_and_normal(obs, f, b1, b2)
    return b + eps * n


def released(x: np.ndarray, obs: Obstacle, f: int, b1: float, b2: float, eps: float) -> bool:
    """Release test of a kept obstacle spring: x more than eps outside the
    stored face point along the face's outward normal."""
    b, n = face_point_and_normal(obs, f, b1, b2)
    return float(np.dot(n, x - b)) > eps

