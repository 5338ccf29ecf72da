"""Reverse-mode derivative of the unrolled local-global loop (oracle side).

Test infrastructure only (see the package docstring).

The loss is L(X_n) = sum over loss vertices of |x_v - t_v|^2 after n
iterations from the rest shape; the parameters are the chamber volume ratios
alpha_g (Eq. 2, Sec. III-A.1).  The loop's discrete decisions -- which
vertices carry springs, of which kind, on which face or sphere, and whether a
self spring was re-cast this iteration or kept its stored barycentrics -- are
taken from a plain forward run of the numpy oracle and held fixed; the
continuous map between them is then re-expressed in PyTorch (float64, CPU) and
differentiated by autograd:

* local step: the rotation from the SVD of D = X_c T_c^T (Kabsch sign fix),
  chamber target cbrt(alpha) R T_c, body blend with w = R_omega(eps) and the
  volume scaling of Eq. 7;
* spring targets: sphere closest point; a self spring's target is the point of
  its face with the barycentric weights of the hit of the ray x_v - t n(v)
  with the face's plane, taken at the iteration that cast the ray (and kept,
  with their dependence on that iteration's positions, while the spring is
  kept), offset by eps along the face normal; when the ray met no exit face
  and the closest point was used instead, the weights are held constant (the
  projection onto the nearest face is not differentiated);
* global step: the Eq. 8 normal equations solved exactly (sparse LU), with the
  reverse pass solving the transposed (here identical) system.

It is pinned against central finite differences of the numpy oracle itself.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

from . import global_step, loop, springs

N4 = torch.eye(4, dtype=torch.float64) - 0.25


@dataclass
class IterDecisions:
    """Discrete state of one iteration, recorded by the numpy forward pass."""

    active: np.ndarray      # (n_q,) bool, springs after the update
    kind: np.ndarray        # (n_q,) 0 self, 1 sphere obstacle, 2 tetrahedral obstacle
    face: np.ndarray        # (n_q,) face id or sphere id
    bary: np.ndarray        # (n_q, 2)
    recast: np.ndarray      # (n_q,) bool: self spring cast this iteration (vertex in a pair) by a ray hit
    cast: np.ndarray = None  # (n_q,) bool: self spring cast this iteration (ray hit or closest point)


def _obstacle_of(m):
    """The generator mesh's tetrahedral obstacle, if it has one."""
    if getattr(m, "obstacle_X", None) is None:
        return None
    from . import obstacle

    return obstacle.prepare(m.obstacle_X, m.obstacle_tets)


def record_forward(m, n_iters, prep=None):
    """Numpy oracle forward from rest; returns (X_n, decisions per iteration)."""
    prep = prep or loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X = m.rest.copy()
    st = springs.SpringState.empty(prep.query.shape[0])
    dec: List[IterDecisions] = []
    obs = _obstacle_of(m)
    for _ in range(n_iters):
        Xn, st, rec, ps, po = loop.iterate(prep, X, st, m.alpha, m.spheres, m.w_knots, m.k_spring, m.eps, m.collision,
                                           obs)
        if isinstance(po, tuple):
            po = np.concatenate(po)
        in_self = np.isin(prep.query, ps[:, 0]) if ps.shape[0] else np.zeros(prep.query.shape[0], bool)
        in_obs = np.isin(prep.query, po[:, 0]) if po.shape[0] else np.zeros(prep.query.shape[0], bool)
        cast = st.active & (st.kind == springs.KIND_SELF) & in_self & ~in_obs
        dec.append(IterDecisions(st.active.copy(), st.kind.copy(), st.face.copy(), st.bary.copy(),
                                 cast & ~st.fallback, cast.copy()))
        X = Xn
    return X, dec, prep


class _SparseSolve(torch.autograd.Function):
    """x = A^-1 b for a fixed sparse SPD A (LU factor reused in reverse)."""

    @staticmethod
    def forward(ctx, b, lu):
        ctx.lu = lu
        return torch.from_numpy(lu.solve(b.detach().numpy()))

    @staticmethod
    def backward(ctx, g):
        return torch.from_numpy(ctx.lu.solve(g.detach().numpy())), None


def _w_table(eps, knots):
    xs = [k[0] for k in knots]
    ys = [k[1] for k in knots]
    out = torch.full_like(eps, ys[0])
    for i in range(len(xs) - 1):
        sel = (eps > xs[i]) & (eps <= xs[i + 1])
        val = ys[i] + (eps - xs[i]) * (ys[i + 1] - ys[i]) / (xs[i + 1] - xs[i])
        out = torch.where(sel, val, out)
    out = torch.where(eps > xs[-1], torch.full_like(eps, ys[-1]), out)
    return out


def _local_targets(X, tets, T_c, vol0, group, alpha, knots):
    Xc = X[tets].transpose(1, 2) @ N4
    D = Xc @ T_c.transpose(1, 2)
    U, S, Vh = torch.linalg.svd(D)
    det = torch.linalg.det(U @ Vh)
    sgn = torch.where(det < 0, -torch.ones_like(det), torch.ones_like(det))
    Dg = torch.diag_embed(torch.stack([torch.ones_like(sgn), torch.ones_like(sgn), sgn], dim=1))
    R = U @ Dg @ Vh
    RT = R @ T_c
    ch = group >= 0
    P = torch.empty_like(Xc)
    if ch.any():
        scale = alpha[group[ch]] ** (1.0 / 3.0)
        P[ch] = scale[:, None, None] * RT[ch]
    body = ~ch
    if body.any():
        diff = Xc[body] - RT[body]
        tt = (T_c[body] ** 2).sum(dim=(1, 2))
        eps = torch.sqrt((diff ** 2).sum(dim=(1, 2)) / tt)
        w = _w_table(eps, knots)[:, None, None]
        B = (1 - w) * Xc[body] + w * RT[body]
        E = B[:, :, 1:] - B[:, :, :1]
        volB = torch.linalg.det(E) / 6.0
        v0 = vol0[body]
        ok = volB > 1e-3 * v0
        s = torch.where(ok, torch.pow(torch.where(ok, v0 / volB, torch.ones_like(volB)), 1.0 / 3.0),
                        torch.ones_like(volB))
        P[body] = s[:, None, None] * B
    return P


def _bary(b, q0, q1, q2):
    """Barycentric weights (of q1, q2) of a point b of the triangle's plane."""
    e1, e2, r = q1 - q0, q2 - q0, b - q0
    d11, d12, d22 = torch.dot(e1, e1), torch.dot(e1, e2), torch.dot(e2, e2)
    r1, r2 = torch.dot(r, e1), torch.dot(r, e2)
    den = d11 * d22 - d12 * d12
    return torch.stack([(d22 * r1 - d12 * r2) / den, (d11 * r2 - d12 * r1) / den])


def _spring_targets(X, prep, dec: IterDecisions, spheres, eps, bary_t, obs=None):
    """Targets c_v (n_active, 3) and their vertex ids, for the fixed decisions.

    ``bary_t`` maps a query index to the barycentric weights (a tensor) of its
    self spring's correspondence: set when the spring's ray is cast, reused
    while the spring is kept, so the weights carry their dependence on the
    positions of the iteration that cast them."""
    faces = torch.from_numpy(prep.faces)
    q = torch.from_numpy(prep.query)
    act = np.nonzero(dec.active)[0]
    if act.size == 0:
        return torch.zeros((0, 3), dtype=torch.float64), np.zeros(0, np.int64)
    # vertex normals n(v): sum of unnormalised incident face normals
    fn_all = torch.cross(X[faces[:, 1]] - X[faces[:, 0]], X[faces[:, 2]] - X[faces[:, 0]], dim=1)
    vn = torch.zeros_like(X).index_add(0, faces[:, 0], fn_all).index_add(0, faces[:, 1], fn_all) \
        .index_add(0, faces[:, 2], fn_all)
    out = []
    for qi in act.tolist():
        v = int(q[qi])
        x = X[v]
        if dec.kind[qi] == springs.KIND_MESH_OBSTACLE:
            # a point of the rigid tetrahedral obstacle: constant
            from . import obstacle

            b1, b2 = dec.bary[qi]
            out.append(torch.from_numpy(obstacle.target(obs, int(dec.face[qi]), float(b1), float(b2), eps)))
            continue
        if dec.kind[qi] == springs.KIND_OBSTACLE:
            c = torch.from_numpy(spheres[dec.face[qi], :3])
            r = float(spheres[dec.face[qi], 3])
            u = x - c
            out.append(c + (r + eps) * u / torch.linalg.norm(u))
            continue
        f = prep.faces[dec.face[qi]]
        q0, q1, q2 = X[f[0]], X[f[1]], X[f[2]]
        n = torch.cross(q1 - q0, q2 - q0, dim=0)
        nh = n / torch.linalg.norm(n)
        if (dec.cast[qi] and not dec.recast[qi]) or qi not in bary_t:
            # closest-point fallback (this iteration or at the spring's cast):
            # weights held constant
            bary_t[qi] = torch.tensor(np.asarray(dec.bary[qi], dtype=np.float64))
        if dec.recast[qi]:
            d = -vn[v] / torch.linalg.norm(vn[v])
            t = torch.dot(n, q0 - x) / torch.dot(n, d)
            bt = _bary(x + t * d, q0, q1, q2)
            bary_t[qi] = bt
        bt = bary_t[qi]
        b = (1 - bt[0] - bt[1]) * q0 + bt[0] * q1 + bt[1] * q2
        out.append(b + eps * nh)
    return torch.stack(out), prep.query[act]


def loss_and_grad(m, n_iters, loss_verts, targets, prep=None):
    """FP64 loss and dL/dalpha of the unrolled loop (decisions from numpy)."""
    X_np, dec, prep = record_forward(m, n_iters, prep)
    obs = _obstacle_of(m)
    tets = torch.from_numpy(prep.tets)
    T_c = torch.from_numpy(prep.T_c)
    vol0 = torch.from_numpy(prep.vol0)
    group = torch.from_numpy(np.asarray(prep.group, dtype=np.int64))
    omega = prep.omega
    alpha = torch.tensor(np.asarray(m.alpha, dtype=np.float64), requires_grad=True)
    free = prep.fixed == 0
    X = torch.from_numpy(m.rest.copy())
    n_v = m.n_verts
    L0 = global_step.laplacian(prep.tets, omega, n_v)
    Xfix = torch.from_numpy(m.rest[~free])
    bary_t = {}
    for it in range(n_iters):
        P = _local_targets(X, tets, T_c, vol0, group, alpha, m.w_knots)
        for qi in list(bary_t):
            if not dec[it].active[qi] or dec[it].kind[qi] != springs.KIND_SELF:
                del bary_t[qi]
        c, sv = _spring_targets(X, prep, dec[it], m.spheres, m.eps, bary_t, obs)
        om = torch.from_numpy(omega)[:, None, None]
        bw = (om * P).transpose(1, 2)             # (n_t, 4, 3)
        b = torch.zeros((n_v, 3), dtype=torch.float64).index_add(0, tets.reshape(-1), bw.reshape(-1, 3))
        A = L0
        if sv.size:
            kd = np.zeros(n_v)
            np.add.at(kd, sv, m.k_spring)
            A = (L0 + sp.diags(kd)).tocsr()
            b = b.index_add(0, torch.from_numpy(sv), m.k_spring * c)
        Aff = A[free][:, free].tocsc()
        Afx = A[free][:, ~free]
        rhs = b[torch.from_numpy(free)] - torch.from_numpy(Afx @ Xfix.numpy())
        lu = spla.splu(Aff)
        xf = _SparseSolve.apply(rhs, lu)
        Xn = X.clone()
        Xn[torch.from_numpy(free)] = xf
        X = Xn
    tv = torch.from_numpy(np.asarray(loss_verts, dtype=np.int64))
    L = ((X[tv] - torch.from_numpy(targets)) ** 2).sum()
    L.backward()
    return float(L.item()), alpha.grad.numpy().copy(), X.detach().numpy(), X_np


def loss_numpy(m, n_iters, loss_verts, targets, alpha=None, prep=None):
    """The same loss evaluated by the numpy oracle's forward pass."""
    a = m.alpha if alpha is None else alpha
    r = loop.run(m.rest, m.tets, m.group, m.fixed, a, n_iters, spheres=m.spheres, knots=m.w_knots, k=m.k_spring,
                 eps=m.eps, collision_mode=m.collision, prep=prep, obstacle=_obstacle_of(m))
    d = r.X[loss_verts] - targets
    return float(np.sum(d * d)), r
