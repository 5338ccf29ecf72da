"""Pins of the Anderson-accelerated loop (Sec. III-B): on a linear fixed-point
map, AA with memory n terminates at the fixed point within n + 1 steps (its
equivalence with GMRES, Walker and Ni 2011); memory 0 is the plain loop; the
safeguard never takes a point of higher energy than the one it came from; and on
a finger the accelerated loop shrinks the fixed-point residual faster."""
import numpy as np

from oracle import anderson, loop
from paper_2203_02054_gb300 import synth


def test_linear_map_terminates_in_n_plus_one_steps():
    rng = np.random.default_rng(0)
    n = 6
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    M = Q @ np.diag(np.linspace(-0.9, 0.9, n)) @ Q.T
    b = rng.normal(size=n)
    x_star = np.linalg.solve(np.eye(n) - M, b)
    xs = anderson.anderson_fixed_point(lambda x: M @ x + b, np.zeros(n), m=n, n_steps=n + 1)
    assert np.linalg.norm(xs[n + 1] - x_star) <= 1e-8 * np.linalg.norm(x_star)
    assert np.linalg.norm(xs[n] - x_star) > 1e-3        # not before: the finite termination is the pin
    plain = anderson.anderson_fixed_point(lambda x: M @ x + b, np.zeros(n), m=0, n_steps=n + 1)
    assert np.linalg.norm(plain[-1] - x_star) > 0.1 * np.linalg.norm(x_star)


def test_memory_zero_is_the_plain_loop():
    m = synth.small_finger(nx=16, ny=4, nz=4, n_ch=3, seed=5, n_iters=8, precision=synth.PRECISION_FP64)
    X, _st, recs = anderson.run_anderson(m, 8, 0)
    ref = loop.run_mesh(m, n_iters=8)
    assert np.array_equal(X, ref.X)
    assert not any(r.accepted for r in recs)


def test_safeguard_and_acceleration():
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, seed=7, n_iters=40, precision=synth.PRECISION_FP64,
                           collision=synth.COLLISION_OFF)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    res = {}
    for mem in (0, 5):
        X, st, recs = anderson.run_anderson(m, 40, mem, prep=prep)
        for r in recs:
            if r.accepted:
                assert r.e_acc < r.e_prev
        g, *_ = loop.iterate(prep, X, st, m.alpha, np.zeros((0, 4)), m.w_knots, m.k_spring, m.eps, m.collision)
        res[mem] = (np.abs(g - X).max(), sum(r.accepted for r in recs))
    assert res[5][1] > 0
    assert res[5][0] < 0.5 * res[0][0]
