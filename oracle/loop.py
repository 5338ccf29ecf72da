"""The collision-aware local-global loop (Algorithm 1, inner while-loop).

Test infrastructure only (see the package docstring).

Algorithm 1 alternates local projection, global blending and collision
checking.  Its loop guard ("while V_coll is non-empty and i < i_max") would not
run when the collided set starts empty, and it checks collision on M^i after
computing M^{i+1}; this oracle reads it as exactly ``n_iters`` iterations, each

    detection on X_i -> spring update -> local step on X_i -> global step -> X_{i+1}

so that the first iteration already sees contacts.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import collision, global_step, local, mesh, springs


@dataclass
class Prepared:
    """Derived mesh quantities (O1) used by every iteration."""

    tets: np.ndarray
    group: np.ndarray
    fixed: np.ndarray
    T_c: np.ndarray
    vol0: np.ndarray
    omega: np.ndarray
    faces: np.ndarray
    query: np.ndarray          # sorted non-fixed surface vertices
    n_verts: int


def prepare(rest, tets, group, fixed) -> Prepared:
    tets = np.asarray(tets, dtype=np.int64)
    T_c, vol0, omega = mesh.rest_quantities(rest, tets)
    faces = mesh.boundary_faces(tets)
    surf = mesh.surface_vertices(faces)
    query = surf[fixed[surf] == 0]
    return Prepared(tets, np.asarray(group), np.asarray(fixed), T_c, vol0, omega, faces, query,
                    rest.shape[0])


@dataclass
class IterRecord:
    energy: float              # E_i of Eq. 8 at X_i with the targets of iteration i
    n_self_pairs: int
    n_obstacle_pairs: int
    n_springs: int


@dataclass
class RunResult:
    X: np.ndarray
    springs: springs.SpringState
    history: List[IterRecord] = field(default_factory=list)
    self_pairs: Optional[np.ndarray] = None
    sphere_pairs: Optional[np.ndarray] = None


def iterate(prep: Prepared, X, st, alpha, spheres, knots, k, eps, collision_mode, obstacle=None):
    """One outer iteration from X_i (and the spring records of iteration i-1).

    Returns X_{i+1}, the updated springs, the iteration record and the pairs
    (self pairs; sphere pairs followed by tetrahedral-obstacle pairs)."""
    if collision_mode >= 1:
        sp_self = collision.self_pairs(X, prep.tets, prep.query)
    else:
        sp_self = np.zeros((0, 2), np.int64)
    if collision_mode >= 2 and spheres.shape[0] > 0:
        sp_obs = collision.sphere_pairs(X, prep.query, spheres)
    else:
        sp_obs = np.zeros((0, 2), np.int64)
    sp_mesh = None
    if collision_mode >= 2 and obstacle is not None:
        from . import obstacle as obst

        sp_mesh = obst.pairs(X, prep.query, obstacle)
    if collision_mode >= 1:
        vn = mesh.vertex_normals(X, prep.faces, prep.n_verts)
        st = springs.update_springs(X, prep.query, st, sp_self, sp_obs, spheres, prep.faces, vn, eps,
                                    obstacle, sp_mesh)
    P, _R, _eps, _w = local.local_step(X, prep.tets, prep.T_c, prep.vol0, prep.group, alpha, knots)
    sv = prep.query[st.active]
    stg = st.target[st.active]
    energy = local.elastic_energy(X, prep.tets, P, prep.omega) + springs.spring_energy(X, prep.query, st, k)
    A, b = global_step.assemble(prep.tets, prep.omega, P, prep.n_verts, sv, stg, k)
    Xn = global_step.solve(A, b, X, prep.fixed)
    n_obs = int(sp_obs.shape[0]) + (0 if sp_mesh is None else int(sp_mesh.shape[0]))
    rec = IterRecord(energy, int(sp_self.shape[0]), n_obs, int(st.active.sum()))
    if sp_mesh is not None:
        sp_obs = (sp_obs, sp_mesh)
    return Xn, st, rec, sp_self, sp_obs


def run(rest, tets, group, fixed, alpha, n_iters, spheres=None, knots=((0.0, 1.0),), k=1.0,
        eps=0.005, collision_mode=1, X0=None, springs0=None, prep=None, obstacle=None) -> RunResult:
    """Run ``n_iters`` iterations from X0 (default: rest) and springs0."""
    prep = prep or prepare(rest, tets, group, fixed)
    spheres = np.zeros((0, 4)) if spheres is None else np.asarray(spheres, dtype=np.float64)
    X = np.array(rest if X0 is None else X0, dtype=np.float64)
    st = springs0.copy() if springs0 is not None else springs.SpringState.empty(prep.query.shape[0])
    res = RunResult(X, st)
    for _ in range(n_iters):
        X, st, rec, ps, po = iterate(prep, X, st, alpha, spheres, knots, k, eps, collision_mode, obstacle)
        res.history.append(rec)
        res.self_pairs, res.sphere_pairs = ps, po
    res.X, res.springs = X, st
    return res


def run_mesh(m, n_iters=None, X0=None, springs0=None, prep=None, knots=None) -> RunResult:
    """Convenience wrapper for a generator ``Mesh`` (its tetrahedral obstacle
    included when it has one)."""
    obstacle = None
    if getattr(m, "obstacle_X", None) is not None:
        from . import obstacle as obst

        obstacle = obst.prepare(m.obstacle_X, m.obstacle_tets)
    return run(m.rest, m.tets, m.group, m.fixed, m.alpha, m.n_iters if n_iters is None else n_iters,
               spheres=m.spheres, knots=m.w_knots if knots is None else knots, k=m.k_spring,
               eps=m.eps, collision_mode=m.collision, X0=X0, springs0=springs0, prep=prep, obstacle=obstacle)
