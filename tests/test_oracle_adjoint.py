"""Pins of the oracle's adjoint: its PyTorch re-expression reproduces the
numpy oracle's forward pass, and its gradient matches central finite
differences of the numpy oracle (FP64, exact solves, h = 1e-4) where the
spring decisions at alpha +- h are the same."""
import numpy as np
import pytest

from paper_2203_02054_gb300 import synth
from oracle import adjoint, loop


def _case(n_iters=8, nx=20, n_ch=4, seed=7):
    m = synth.small_finger(nx=nx, ny=4, nz=4, n_ch=n_ch, seed=seed, n_iters=n_iters,
                           precision=synth.PRECISION_FP64)
    # loss on the tip face (x = nx) vertices, targets = rest + seeded offsets
    tips = np.nonzero(np.isclose(m.rest[:, 0], nx * m.h))[0]
    rng = np.random.default_rng(seed)
    targets = m.rest[tips] + rng.normal(size=(tips.size, 3)) * 0.5
    return m, tips, targets


def test_torch_forward_reproduces_numpy_oracle():
    m, tips, targets = _case()
    L, g, X_t, X_np = adjoint.loss_and_grad(m, 8, tips, targets)
    assert np.abs(X_t - X_np).max() < 1e-10
    L_np, _ = adjoint.loss_numpy(m, 8, tips, targets)
    assert abs(L - L_np) <= 1e-10 * max(1.0, abs(L_np))


def test_adjoint_matches_central_differences():
    m, tips, targets = _case()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    L, g, _, _ = adjoint.loss_and_grad(m, 8, tips, targets, prep=prep)
    h = 1e-4
    _, r0 = adjoint.loss_numpy(m, 8, tips, targets, prep=prep)
    n0 = [hh.n_springs for hh in r0.history]
    assert max(n0) > 0          # the case exercises the spring terms
    checked = 0
    for gi in range(m.n_groups):
        ap = m.alpha.copy()
        am = m.alpha.copy()
        ap[gi] += h
        am[gi] -= h
        Lp, rp = adjoint.loss_numpy(m, 8, tips, targets, alpha=ap, prep=prep)
        Lm, rm = adjoint.loss_numpy(m, 8, tips, targets, alpha=am, prep=prep)
        same = ([hh.n_springs for hh in rp.history] == n0 and [hh.n_springs for hh in rm.history] == n0
                and np.array_equal(rp.springs.active, r0.springs.active)
                and np.array_equal(rm.springs.active, r0.springs.active))
        if not same:
            continue
        fd = (Lp - Lm) / (2 * h)
        assert abs(g[gi] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(g).max()), (gi, g[gi], fd)
        checked += 1
    assert checked >= m.n_groups - 1
