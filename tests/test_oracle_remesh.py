"""Pins of the remesh trigger and the progressive outer loop (Sec. III-C,
Algorithm 1): closed forms of affine maps with known singular values and
volume change, invariants (rotations, body elements, identity reference), and
the one-step outer loop reproducing the plain inner loop."""
import numpy as np

from oracle import loop, remesh
from paper_2203_02054_gb300 import synth


def _tet_mesh(n=6, seed=3):
    """A few random positively oriented tets sharing no vertices."""
    rng = np.random.default_rng(seed)
    X, T = [], []
    for e in range(n):
        base = rng.normal(size=3) * 5.0
        while True:
            P = base + rng.normal(size=(4, 3))
            if np.linalg.det((P[1:] - P[0]).T) > 0.3:
                break
        X.append(P)
        T.append([4 * e, 4 * e + 1, 4 * e + 2, 4 * e + 3])
    return np.concatenate(X), np.array(T)


def _rot(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _apply(X, F, t=np.zeros(3)):
    return X @ F.T + t


def test_uniform_scaling_and_rotation():
    X, T = _tet_mesh()
    g = np.zeros(T.shape[0], int)
    for s, expect in ((1.5, 0), (1.6, remesh.FLAG_VOLUME)):       # s^3 = 3.375 / 4.096 against 4
        Y = _apply(X, s * _rot(11), np.array([0.3, -2.0, 1.0]))
        flags, ratio, smax, gvr = remesh.remesh_flags(Y, X, T, g)
        assert np.allclose(ratio, s ** 3, rtol=1e-12)
        assert np.allclose(smax, s, rtol=1e-12)
        assert np.all(flags == expect)
        assert abs(gvr[0] - s ** 3) < 1e-12 * s ** 3


def test_stretch_flags_both():
    X, T = _tet_mesh()
    g = np.zeros(T.shape[0], int)
    Y = _apply(X, _rot(5) @ np.diag([5.0, 1.0, 1.0]))
    flags, ratio, smax, _ = remesh.remesh_flags(Y, X, T, g)
    assert np.allclose(ratio, 5.0, rtol=1e-12) and np.allclose(smax, 5.0, rtol=1e-12)
    assert np.all(flags == remesh.FLAG_VOLUME | remesh.FLAG_DISTORTION)


def test_shear_singular_value_closed_form():
    """F = [[1, gamma, 0], [0, 1, 0], [0, 0, 1]]: det 1, and the 2x2 block's
    largest singular value is (gamma + sqrt(gamma^2 + 4)) / 2."""
    X, T = _tet_mesh()
    g = np.zeros(T.shape[0], int)
    for gamma, expect in ((3.5, 0), (3.8, remesh.FLAG_DISTORTION)):
        F = np.array([[1.0, gamma, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
        Y = _apply(X, _rot(7) @ F)
        flags, ratio, smax, _ = remesh.remesh_flags(Y, X, T, g)
        assert np.allclose(ratio, 1.0, rtol=1e-12)
        assert np.allclose(smax, (gamma + np.sqrt(gamma * gamma + 4.0)) / 2.0, rtol=1e-12)
        assert np.all(flags == expect)


def test_thresholds_are_parameters_and_body_is_never_flagged():
    X, T = _tet_mesh()
    g = np.array([-1, 0, -1, 1, 1, -1])
    Y = _apply(X, np.diag([6.0, 6.0, 6.0]))
    flags, ratio, _, gvr = remesh.remesh_flags(Y, X, T, g)
    assert np.all(flags[g < 0] == 0) and np.all(ratio[g < 0] == 0)
    assert np.all(flags[g >= 0] == remesh.FLAG_VOLUME | remesh.FLAG_DISTORTION)
    assert set(gvr) == {0, 1}
    flags2, _, _, _ = remesh.remesh_flags(Y, X, T, g, alpha_max=300.0, d_max=7.0)
    assert np.all(flags2 == 0)
    flags3, ratio3, smax3, gvr3 = remesh.remesh_flags(Y, Y, T, g)     # identity reference
    assert np.all(flags3 == 0) and np.allclose(ratio3[g >= 0], 1.0) and np.allclose(smax3[g >= 0], 1.0)
    assert all(abs(v - 1.0) < 1e-12 for v in gvr3.values())


def test_one_outer_step_is_the_plain_loop():
    m = synth.small_finger(nx=16, ny=4, nz=4, n_ch=3, seed=5, n_iters=6, precision=synth.PRECISION_FP64)
    X1, recs = remesh.progressive(m, m.alpha, alpha_step=10.0, n_inner=6)
    ref = loop.run_mesh(m, n_iters=6)
    assert len(recs) == 1 and np.array_equal(recs[0].applied, m.alpha)
    assert np.array_equal(X1, ref.X)


def test_outer_steps_cap_at_the_target():
    m = synth.small_finger(nx=16, ny=4, nz=4, n_ch=3, seed=5, n_iters=4, precision=synth.PRECISION_FP64)
    step = float(np.max(m.alpha)) / 2.0 + 1e-9
    X, recs = remesh.progressive(m, m.alpha, alpha_step=step, n_inner=4, alpha_max=1.05, d_max=1.05)
    assert len(recs) == 2
    assert np.allclose(recs[0].applied, np.minimum(m.alpha, step))
    assert np.array_equal(recs[-1].applied, m.alpha)
    # the chambers expand: their volume ratio against rest grows from the first outer step to the second
    for gk, v in recs[-1].chamber_volume_ratio.items():
        assert v > recs[0].chamber_volume_ratio[gk] > 1.0
    assert recs[0].n_flagged > 0
