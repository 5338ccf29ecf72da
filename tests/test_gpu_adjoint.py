"""Adjoint (reverse pass of the unrolled loop) on the GPU: dL/dalpha for a
loss on tip-vertex positions, against the oracle's FP64 adjoint and against
central finite differences of the GPU's own FP64 forward pass (h = 1e-4,
only where the spring decisions at alpha +- h are identical)."""
import numpy as np
import pytest

from paper_2203_02054_gb300 import casim, synth
from oracle import adjoint as oadj
from oracle import loop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    casim.load_library()


def _finger(nx, ny, nz, n_ch, seed, precision, n_iters):
    m = synth.small_finger(nx=nx, ny=ny, nz=nz, n_ch=n_ch, seed=seed, n_iters=n_iters, precision=precision)
    tips = np.nonzero(np.isclose(m.rest[:, 0], nx * m.h))[0]
    rng = np.random.default_rng(seed)
    targets = m.rest[tips] + rng.normal(size=(tips.size, 3)) * 0.5
    return m, tips, targets


def _gpu_grad(sim, m, tips, targets, n_iters, every):
    casim.casim_set_actuation(sim.h, m.alpha)
    sim.reset()
    casim.casim_forward_ckpt(sim.h, n_iters, every)
    assert sim.sync() == 0
    X = sim.positions()
    gX = np.zeros_like(X)
    gX[tips] = 2.0 * (X[tips] - targets)
    L = float(np.sum((X[tips] - targets) ** 2))
    return L, casim.casim_backward(sim.h, gX, m.n_groups), X


def test_gpu_adjoint_matches_oracle_adjoint_fp64():
    m, tips, targets = _finger(20, 4, 4, 4, 7, synth.PRECISION_FP64, 8)
    sim = casim.Sim(m)
    L, g, X = _gpu_grad(sim, m, tips, targets, 8, 3)
    Lo, go, Xo, _ = oadj.loss_and_grad(m, 8, tips, targets)
    assert np.abs(X - Xo).max() < 1e-9
    assert abs(L - Lo) <= 1e-9 * abs(Lo)
    assert np.allclose(g, go, rtol=1e-7, atol=1e-9 * np.abs(go).max()), (g, go)
    sim.close()


def test_gpu_adjoint_independent_of_checkpoint_interval():
    m, tips, targets = _finger(20, 4, 4, 4, 7, synth.PRECISION_MIXED, 10)
    sim = casim.Sim(m)
    grads = [_gpu_grad(sim, m, tips, targets, 10, every)[1] for every in (1, 4, 10)]
    assert np.array_equal(grads[0], grads[1]) and np.array_equal(grads[0], grads[2])
    sim.close()


def test_gpu_adjoint_mixed_close_to_fp64():
    m, tips, targets = _finger(20, 4, 4, 4, 7, synth.PRECISION_MIXED, 8)
    sim = casim.Sim(m)
    _, g32, _ = _gpu_grad(sim, m, tips, targets, 8, 4)
    sim.close()
    m64, _, _ = _finger(20, 4, 4, 4, 7, synth.PRECISION_FP64, 8)
    sim = casim.Sim(m64)
    _, g64, _ = _gpu_grad(sim, m64, tips, targets, 8, 4)
    sim.close()
    assert np.allclose(g32, g64, rtol=2e-3, atol=2e-3 * np.abs(g64).max())


def _decisions(sim):
    sp = sim.springs()
    hist = sim.history()
    return ([h["n_self_pairs"] for h in hist][-20:], [h["n_springs"] for h in hist][-20:],
            sp["active"].tolist(), sp["kind"].tolist(), sp["face"].tolist())


def test_gpu_adjoint_central_differences_on_20k_copy():
    """The 20,736-tet copy of the adjoint workload (96x6x6 voxels, 16
    chambers), FP64 forward, 20 iterations, checkpoints every 5.  A group is
    compared only when every recorded decision (pair and spring counts of all
    iterations, final spring records) is the same at alpha +- h."""
    m = synth.config5_adjoint(nx=96, ny=6, nz=6, n_ch=16, n_iters=20)
    m.precision = synth.PRECISION_FP64
    tips, targets = m.tip_verts, m.tip_targets
    sim = casim.Sim(m)
    L, g, _ = _gpu_grad(sim, m, tips, targets, 20, 5)
    sim.reset()
    casim.casim_set_actuation(sim.h, m.alpha)
    sim.step(20)
    sim.sync()
    base = _decisions(sim)
    h = 1e-4
    checked = 0
    for gi in range(m.n_groups):
        vals = []
        same = True
        for sgn in (1.0, -1.0):
            a = m.alpha.copy()
            a[gi] += sgn * h
            casim.casim_set_actuation(sim.h, a)
            sim.reset()
            sim.step(20)
            assert sim.sync() == 0
            X = sim.positions()
            vals.append(float(np.sum((X[tips] - targets) ** 2)))
            same = same and _decisions(sim) == base
        if not same:
            continue
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g[gi] - fd) <= 1e-4 * max(abs(fd), 1e-2 * np.abs(g).max()), (gi, g[gi], fd)
        checked += 1
    assert checked >= 4
    sim.close()


def test_gpu_adjoint_matches_oracle_adjoint_on_20k_copy():
    m = synth.config5_adjoint(nx=96, ny=6, nz=6, n_ch=16, n_iters=10)
    m.precision = synth.PRECISION_FP64
    tips, targets = m.tip_verts, m.tip_targets
    sim = casim.Sim(m)
    L, g, X = _gpu_grad(sim, m, tips, targets, 10, 5)
    sim.close()
    Lo, go, Xo, _ = oadj.loss_and_grad(m, 10, tips, targets)
    assert np.abs(X - Xo).max() < 1e-8
    assert np.allclose(g, go, rtol=1e-6, atol=1e-8 * np.abs(go).max()), np.abs(g - go).max()


def test_autograd_function_matches_backward():
    import torch

    m, tips, targets = _finger(20, 4, 4, 4, 7, synth.PRECISION_FP64, 6)
    sim = casim.Sim(m)
    a = torch.tensor(m.alpha, dtype=torch.float64, requires_grad=True)
    X = casim.actuation_to_positions(sim, a, 6, ckpt_every=2)
    t = torch.from_numpy(targets)
    loss = ((X[torch.from_numpy(tips)] - t) ** 2).sum()
    loss.backward()
    _, g, _ = _gpu_grad(sim, m, tips, targets, 6, 2)
    assert np.allclose(a.grad.numpy(), g, rtol=1e-12, atol=0)
    sim.close()
