"""Anderson acceleration of the local-global loop (Sec. III-B; Peng et al. 2018).

Test infrastructure only (see the package docstring).

One iteration of the loop is a map G taking positions x to G(x) (collision
check, spring update, local step, global step).  Anderson acceleration with
memory m (Anderson 1965; Walker and Ni 2011) keeps the last m + 1 evaluated
pairs (x_j, g_j = G(x_j)) with residuals f_j = g_j - x_j and, after
evaluating g_k, solves the small least-squares problem

    theta = argmin || f_k - dF theta ||,   dF = [f_{j+1} - f_j]  (m columns)

through its normal equations with a Tikhonov term
(dF^T dF + lambda I) theta = dF^T f_k, lambda = 1e-12 trace(dF^T dF) / m,
and proposes x_acc = g_k - dG theta, dG = [g_{j+1} - g_j].

Safeguard (the energy test of Peng et al. 2018): the proposal is taken only
if its energy is below that of the point it came from, E(x_acc) < E(x_k), both
evaluated with the local projections at the point and the spring records of
iteration k (the iteration that evaluated G(x_k), so the two energies use the
same springs); otherwise x_{k+1} = g_k, the plain iterate.  The history keeps
every evaluated pair whichever point is taken.  With m = 0 this is the plain
loop.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from . import local, loop, springs


def aa_proposal(F: List[np.ndarray], Gs: List[np.ndarray]) -> np.ndarray:
    """x_acc from the last m + 1 residuals F and images Gs (oldest first),
    each flattened to a vector."""
    f, g = F[-1], Gs[-1]
    if len(F) < 2:
        return g.copy()
    dF = np.stack([F[j + 1] - F[j] for j in range(len(F) - 1)], axis=1)
    dG = np.stack([Gs[j + 1] - Gs[j] for j in range(len(Gs) - 1)], axis=1)
    M = dF.T @ dF
    m = M.shape[0]
    lam = 1e-12 * np.trace(M) / m
    theta = np.linalg.solve(M + lam * np.eye(m), dF.T @ f)
    return g - dG @ theta


def anderson_fixed_point(G, x0, m, n_steps):
    """Plain AA(m) on a fixed-point map G (no safeguard): the iterates."""
    x = np.asarray(x0, dtype=np.float64).copy()
    F, Gs, xs = [], [], [x.copy()]
    for _ in range(n_steps):
        g = G(x)
        F.append(g - x)
        Gs.append(g)
        F, Gs = F[-(m + 1):], Gs[-(m + 1):]
        x = aa_proposal(F, Gs) if m > 0 else g
        xs.append(x.copy())
    return xs


def energy(prep, X, st, alpha, knots, k_spring):
    """Eq. 8 energy with the local projections at X and the given spring records."""
    P, _R, _e, _w = local.local_step(X, prep.tets, prep.T_c, prep.vol0, prep.group, alpha, knots)
    return local.elastic_energy(X, prep.tets, P, prep.omega) + springs.spring_energy(X, prep.query, st, k_spring)


@dataclass
class AAStep:
    e_prev: float       # E(x_k)
    e_acc: float        # E(x_acc) (NaN when no proposal was formed)
    accepted: bool      # x_{k+1} = x_acc


def run_anderson(m_mesh, n_steps, m, X0=None, prep=None):
    """n_steps iterations of the safeguarded accelerated loop on a generator
    ``Mesh``; returns (X, spring records, per-step records)."""
    mm = m_mesh
    prep = prep or loop.prepare(mm.rest, mm.tets, mm.group, mm.fixed)
    spheres = np.zeros((0, 4)) if mm.spheres is None else np.asarray(mm.spheres, np.float64)
    x = np.array(mm.rest if X0 is None else X0, dtype=np.float64)
    st = springs.SpringState.empty(prep.query.shape[0])
    F, Gs, recs = [], [], []
    for _ in range(n_steps):
        g, st, _rec, _ps, _po = loop.iterate(prep, x, st, mm.alpha, spheres, mm.w_knots, mm.k_spring, mm.eps,
                                             mm.collision)
        F.append((g - x).ravel())
        Gs.append(g.ravel())
        F, Gs = F[-(m + 1):], Gs[-(m + 1):]
        if m > 0 and len(F) >= 2:
            xa = aa_proposal(F, Gs).reshape(g.shape)
            ep = energy(prep, x, st, mm.alpha, mm.w_knots, mm.k_spring)
            ea = energy(prep, xa, st, mm.alpha, mm.w_knots, mm.k_spring)
            acc = ea < ep
            recs.append(AAStep(ep, ea, acc))
            x = xa if acc else g
        else:
            recs.append(AAStep(np.nan, np.nan, False))
            x = g
    return x, st, recs
