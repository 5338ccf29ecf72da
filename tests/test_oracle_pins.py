"""Pins of the FP64 oracle against facts that do not come from the oracle:
closed forms, invariants the paper states, an independent rotation method,
brute force and exact rational arithmetic.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2203_02054_gb300 import synth
from oracle import collision, global_step, local, loop, mesh, springs

W1 = ((0.0, 1.0),)   # w == 1: the body target is the rotated rest shape


def _rot(axis, ang):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _single_tet():
    rest = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    tets = np.array([[0, 1, 2, 3]])
    return rest, tets


# ---------------------------------------------------------------- O1 / mesh
def test_kuhn_mesh_orientation_and_volume():
    m = synth.config1_beam()
    V = mesh.element_matrices(m.rest, m.tets.astype(np.int64))
    vol = mesh.signed_volume(V)
    assert np.all(vol > 0)
    assert np.allclose(vol, m.h ** 3 / 6.0, rtol=0, atol=1e-15)
    # 6 Kuhn tets tile each voxel exactly
    assert math.isclose(vol.sum(), 20 * 4 * 4 * m.h ** 3, rel_tol=1e-13)


def test_boundary_faces_of_block_and_slits():
    # a solid block: 2 triangles per boundary voxel face; outward normals sum to 0
    m = synth.config1_beam()
    f = mesh.boundary_faces(m.tets.astype(np.int64))
    assert f.shape[0] == 2 * 2 * (20 * 4 + 20 * 4 + 4 * 4)
    fn = mesh.face_normals(m.rest, f)
    assert np.allclose(fn.sum(axis=0), 0, atol=1e-12)
    # each outward normal points away from the centroid of its tet
    c = m.rest.mean(axis=0)
    tri_c = m.rest[f].mean(axis=1)
    # divergence theorem: sum over faces of (centroid . n)/3*... = 3 * volume / ...
    vol = np.sum(np.einsum("ij,ij->i", tri_c, fn)) / 6.0
    assert math.isclose(vol, 20 * 4 * 4 * m.h ** 3, rel_tol=1e-12)
    del c
    # slit finger: the slit adds 2 x (plane faces) boundary triangles
    fm = synth.small_finger()
    lay = synth.finger_layout(20, 4, 4, 4)
    ff = mesh.boundary_faces(fm.tets.astype(np.int64))
    n_plain = 2 * 2 * (20 * 4 + 20 * 4 + 4 * 4)
    per_slit = 2 * 2 * 4 * (4 - lay["s"])
    assert ff.shape[0] == n_plain + per_slit * len(lay["slits"])


# ---------------------------------------------------------------- O2 / local
def test_kabsch_known_factors_and_reflection():
    rng = np.random.default_rng(1)
    for refl in (False, True):
        U = _rot(rng.normal(size=3), 0.7)
        V = _rot(rng.normal(size=3), -1.3)
        sig = np.array([3.0, 1.5, 0.4])
        if refl:
            U = U @ np.diag([1, 1, -1.0])   # det(U V^T) = -1
        D = U @ np.diag(sig) @ V.T
        R, tr = local.kabsch_rotation(D[None])
        if not refl:
            assert np.allclose(R[0], U @ V.T, atol=1e-13)
            assert math.isclose(tr[0], sig.sum(), rel_tol=1e-13)
        else:
            assert np.allclose(R[0], U @ np.diag([1, 1, -1.0]) @ V.T, atol=1e-13)
            assert math.isclose(tr[0], 3.0 + 1.5 - 0.4, rel_tol=1e-13)
        assert math.isclose(np.linalg.det(R[0]), 1.0, rel_tol=1e-13)


def _horn_rotation(D):
    """Independent rotation fit: Horn's unit-quaternion method (Horn 1987).
    The rotation maximising tr(R^T D) is given by the eigenvector of the
    largest eigenvalue of a symmetric 4x4 matrix built from D."""
    # tr(R^T D) = sum_ij R_ij D_ij;  build N so that q^T N q = tr(R(q)^T D)
    Sxx, Sxy, Sxz = D[0]
    Syx, Syy, Syz = D[1]
    Szx, Szy, Szz = D[2]
    Nm = np.array([
        [Sxx + Syy + Szz, Szy - Syz, Sxz - Szx, Syx - Sxy],
        [Szy - Syz, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz],
        [Sxz - Szx, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy],
        [Syx - Sxy, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz]])
    w, v = np.linalg.eigh(Nm)
    q0, qx, qy, qz = v[:, -1]
    return np.array([
        [q0 * q0 + qx * qx - qy * qy - qz * qz, 2 * (qx * qy - q0 * qz), 2 * (qx * qz + q0 * qy)],
        [2 * (qy * qx + q0 * qz), q0 * q0 - qx * qx + qy * qy - qz * qz, 2 * (qy * qz - q0 * qx)],
        [2 * (qz * qx - q0 * qy), 2 * (qz * qy + q0 * qx), q0 * q0 - qx * qx - qy * qy + qz * qz]]), w[-1]


def test_kabsch_matches_horn_quaternion_method():
    rng = np.random.default_rng(2)
    D = rng.normal(size=(200, 3, 3))
    R, tr = local.kabsch_rotation(D)
    for i in range(D.shape[0]):
        Rh, lam = _horn_rotation(D[i])
        assert np.allclose(R[i], Rh, atol=1e-9)
        assert math.isclose(tr[i], lam, rel_tol=1e-10, abs_tol=1e-12)


def test_local_step_targets_closed_forms():
    rest, tets = _single_tet()
    T_c, vol0, _ = mesh.rest_quantities(rest, tets)
    Q = _rot([1, 2, 3], 0.9)
    X = (Q @ rest.T).T * 1.1 + np.array([5.0, -2, 1])
    # chamber: target = cbrt(alpha) R T_c with R = Q (the element is a similarity)
    P, R, eps, _ = local.local_step(X, tets, T_c, vol0, np.array([0]), [2.0], W1)
    assert np.allclose(R[0], Q, atol=1e-13)
    assert np.allclose(P[0], 2.0 ** (1 / 3) * Q @ T_c[0], atol=1e-13)
    assert math.isclose(mesh.signed_volume(P)[0], 2.0 * vol0[0], rel_tol=1e-12)
    # body: strain = 0.1 (relative Procrustes misfit of a 1.1 scaling)
    P, R, eps, w = local.local_step(X, tets, T_c, vol0, np.array([-1]), [], synth.SOFT_W_KNOTS)
    assert math.isclose(eps[0], 0.1, rel_tol=1e-12)
    assert math.isclose(w[0], 0.6 + 0.1 * (0.9 - 0.6) / 0.5, rel_tol=1e-12)
    assert math.isclose(mesh.signed_volume(P)[0], vol0[0], rel_tol=1e-12)  # Eq. 7 volume


def test_body_volume_preservation_random():
    m = synth.small_finger()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X = synth.perturbed_positions(m, 0.2, seed=3)
    P, R, eps, w = local.local_step(X, prep.tets, prep.T_c, prep.vol0, prep.group, m.alpha, m.w_knots)
    body = prep.group < 0
    volP = mesh.signed_volume(P)
    volB = volP  # s scales the blend to the rest volume unless the guard triggers
    assert np.allclose(volB[body], prep.vol0[body], rtol=1e-11)
    ch = ~body
    assert np.allclose(volP[ch], m.alpha[prep.group[ch]] * prep.vol0[ch], rtol=1e-11)
    # R are proper rotations
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)


def test_body_target_w1_is_rotated_rest():
    m = synth.small_finger()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X = synth.perturbed_positions(m, 0.2, seed=4)
    P, R, eps, w = local.local_step(X, prep.tets, prep.T_c, prep.vol0, prep.group, m.alpha, W1)
    body = prep.group < 0
    assert np.allclose(P[body], (R @ prep.T_c)[body], atol=1e-12)


# ---------------------------------------------------------------- O5 / global
def test_global_step_single_tet_closed_form():
    rest, tets = _single_tet()
    rng = np.random.default_rng(5)
    P = rng.normal(size=(1, 3, 4))
    P = P - P.mean(axis=2, keepdims=True)
    X = rest + rng.normal(size=rest.shape)
    fixed = np.array([1, 1, 1, 0], np.uint8)
    A, b = global_step.assemble(tets, np.array([1.0]), P, 4, np.zeros(0, int), np.zeros((0, 3)), 1.0)
    Xn = global_step.solve(A, b, X, fixed)
    expect = (4 * P[0, :, 3] + X[0] + X[1] + X[2]) / 3.0
    assert np.allclose(Xn[3], expect, atol=1e-13)
    assert np.allclose(Xn[:3], X[:3])


def test_laplacian_row_sums_and_symmetry():
    m = synth.small_finger()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    L = global_step.laplacian(prep.tets, prep.omega, m.n_verts)
    assert np.allclose(np.asarray(L.sum(axis=1)).ravel(), 0, atol=1e-13)
    assert abs(L - L.T).max() == 0


def test_global_step_minimises_eq8_energy():
    """The solved positions make the Eq. 8 energy (evaluated from its
    definition, not from the assembled system) stationary and minimal."""
    m = synth.small_finger()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X = synth.perturbed_positions(m, 0.2, seed=6)
    P, *_ = local.local_step(X, prep.tets, prep.T_c, prep.vol0, prep.group, m.alpha, m.w_knots)
    rng = np.random.default_rng(7)
    sv = prep.query[:20]
    stg = X[sv] + rng.normal(size=(20, 3)) * 0.1
    k = 1.0
    A, b = global_step.assemble(prep.tets, prep.omega, P, m.n_verts, sv, stg, k)
    Xs = global_step.solve(A, b, X, prep.fixed)

    def energy(Y):
        ee = local.elastic_energy(Y, prep.tets, P, prep.omega)
        return ee + k * float(np.sum((Y[sv] - stg) ** 2))

    e0 = energy(Xs)
    free = np.nonzero(prep.fixed == 0)[0]
    for trial in range(5):
        d = np.zeros_like(Xs)
        d[free] = rng.normal(size=(free.size, 3)) * 1e-3
        assert energy(Xs + d) >= e0
        # central difference of the energy along d vanishes at the minimum
        g = (energy(Xs + d) - energy(Xs - d)) / 2.0
        assert abs(g) < 1e-10


# ---------------------------------------------------------------- O6 / loop
def test_rest_is_fixed_point():
    m = synth.small_finger(n_iters=3)
    ones = np.ones_like(m.alpha)
    r = loop.run(m.rest, m.tets, m.group, m.fixed, ones, 3, knots=m.w_knots, eps=m.eps, collision_mode=1)
    # exact up to the rounding of the sparse direct solve
    assert np.abs(r.X - m.rest).max() < 1e-10
    assert all(h.n_self_pairs == 0 and h.n_springs == 0 for h in r.history)
    assert all(abs(h.energy) < 1e-20 for h in r.history)


def test_uniform_scaling_gives_similar_shape():
    m = synth.config1_beam()
    group = np.zeros(m.n_tets, np.int32)
    fixed = np.zeros(m.n_verts, np.uint8)
    fixed[0] = 1
    alpha = 1.7
    r = loop.run(m.rest, m.tets, group, fixed, [alpha], 1, knots=W1, collision_mode=0)
    x0 = m.rest[0]
    expect = x0 + alpha ** (1 / 3) * (m.rest - x0)
    assert np.abs(r.X - expect).max() < 1e-11
    # second iteration: energy is zero
    r2 = loop.run(m.rest, m.tets, group, fixed, [alpha], 2, knots=W1, collision_mode=0)
    assert r2.history[1].energy < 1e-20


def test_energy_nonincreasing_w1():
    m = synth.config1_beam()
    r = loop.run(m.rest, m.tets, m.group, m.fixed, m.alpha, 30, knots=W1, collision_mode=0)
    E = [h.energy for h in r.history]
    for a, b in zip(E, E[1:]):
        assert b <= a * (1 + 1e-12)
    assert E[-1] < E[0]


def test_rigid_motion_equivariance():
    m = synth.config1_beam()
    Q = _rot([0.3, -1, 2], 1.1)
    t = np.array([3.0, -7.0, 2.5])
    r1 = loop.run(m.rest, m.tets, m.group, m.fixed, m.alpha, 5, knots=m.w_knots, collision_mode=0)
    rest2 = m.rest @ Q.T + t
    r2 = loop.run(rest2, m.tets, m.group, m.fixed, m.alpha, 5, knots=m.w_knots, collision_mode=0)
    assert np.abs(r2.X - (r1.X @ Q.T + t)).max() < 1e-10
    assert np.allclose([h.energy for h in r1.history], [h.energy for h in r2.history], rtol=1e-9)


def test_scale_equivariance_with_collision():
    m = synth.small_finger(n_iters=4)
    lam = 2.0   # a power of two keeps every coordinate exact
    r1 = loop.run_mesh(m)
    r2 = loop.run(m.rest * lam, m.tets, m.group, m.fixed, m.alpha, 4, knots=m.w_knots,
                  eps=m.eps * lam, collision_mode=1)
    assert np.abs(r2.X - lam * r1.X).max() < 1e-9
    assert [h.n_self_pairs for h in r1.history] == [h.n_self_pairs for h in r2.history]


# ---------------------------------------------------------------- O3 / collision
def test_orient_sign_exact_on_integer_grid():
    rng = np.random.default_rng(8)
    q = rng.integers(-4, 5, size=(4000, 4, 3)).astype(np.float64)
    # force many exactly-coplanar cases
    q[::3, 3] = q[::3, 0] + (q[::3, 1] - q[::3, 0]) * 2 - (q[::3, 2] - q[::3, 0])
    s = collision.orient_sign(q[:, 0], q[:, 1], q[:, 2], q[:, 3])
    qi = q.astype(np.int64)
    u, v, w = qi[:, 1] - qi[:, 0], qi[:, 2] - qi[:, 0], qi[:, 3] - qi[:, 0]
    det = np.einsum("ij,ij->i", u, np.cross(v, w))
    assert np.array_equal(s, np.sign(det))
    assert np.sum(det == 0) > 1000


def test_orient_sign_near_degenerate_tiny_offsets():
    # points a few ulps off a plane: the filter cannot decide, the exact path must
    rng = np.random.default_rng(9)
    a = np.array([0.1, 0.2, 0.3])
    b = np.array([1.3, 0.7, -0.2])
    c = np.array([-0.4, 1.1, 0.9])
    out = []
    for _ in range(200):
        t1, t2 = rng.uniform(-1, 2, size=2)
        p = a + t1 * (b - a) + t2 * (c - a)
        p = p + rng.integers(-3, 4, size=3) * np.spacing(p)
        s = collision.orient_sign(a[None], b[None], c[None], p[None])[0]
        fa, fb, fc, fp = ([Fraction(float(x)) for x in pt] for pt in (a, b, c, p))
        u = [fb[i] - fa[i] for i in range(3)]
        v = [fc[i] - fa[i] for i in range(3)]
        w = [fp[i] - fa[i] for i in range(3)]
        det = u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) \
            + u[2] * (v[0] * w[1] - v[1] * w[0])
        out.append(s == ((det > 0) - (det < 0)))
    assert all(out)


def test_strict_inside_special_points():
    a, b, c, d = (np.array(p, float) for p in ([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]))
    pts = {
        "centroid": ([0.25, 0.25, 0.25], True),
        "inside": ([0.1, 0.2, 0.3], True),
        "on_face": ([0.0, 0.3, 0.3], False),
        "on_slanted_face": ([0.25, 0.25, 0.5], False),
        "on_edge": ([0.5, 0.5, 0.0], False),
        "at_vertex": ([1.0, 0.0, 0.0], False),
        "outside": ([0.5, 0.5, 0.5], False),
    }
    for name, (p, exp) in pts.items():
        got = collision.strictly_inside(np.array([p]), a[None], b[None], c[None], d[None])[0]
        assert got == exp, name


def test_self_pairs_brute_force_vs_barycentric_loop():
    """The vectorised brute force equals a per-pair loop over all (v, e) using
    exact barycentric signs from rational arithmetic."""
    m = synth.small_finger(nx=10, ny=4, nz=4, n_ch=2)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X = synth.perturbed_positions(m, 0.3, seed=10)
    pairs = collision.self_pairs(X, prep.tets, prep.query)
    got = set(map(tuple, pairs.tolist()))
    expect = set()
    Xf = [[Fraction(float(x)) for x in row] for row in X]

    def det3(u, v, w):
        return (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
                + u[2] * (v[0] * w[1] - v[1] * w[0]))

    def vol(p0, p1, p2, p3):
        return det3([p1[i] - p0[i] for i in range(3)], [p2[i] - p0[i] for i in range(3)],
                    [p3[i] - p0[i] for i in range(3)])

    lo = X[prep.tets].min(axis=1)
    hi = X[prep.tets].max(axis=1)
    for v in prep.query.tolist():
        for e in range(prep.tets.shape[0]):
            t = prep.tets[e].tolist()
            if v in t:
                continue
            if np.any(X[v] < lo[e] - 1e-9) or np.any(X[v] > hi[e] + 1e-9):
                continue
            P = [Xf[i] for i in t]
            p = Xf[v]
            if (vol(p, P[1], P[2], P[3]) > 0 and vol(P[0], p, P[2], P[3]) > 0
                    and vol(P[0], P[1], p, P[3]) > 0 and vol(P[0], P[1], P[2], p) > 0):
                expect.add((v, e))
    assert got == expect
    assert len(expect) >= 5


def test_slit_mesh_rest_has_no_contacts():
    m = synth.small_finger()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    assert collision.self_pairs(m.rest, prep.tets, prep.query).shape[0] == 0


def test_sphere_boundary_is_not_inside():
    X = np.array([[3.0, 0, 0], [2.999, 0, 0], [0, 0, 0], [0, 3.0, 0.0], [1, 2, 2.0]])
    pairs = collision.sphere_pairs(X, np.arange(5), np.array([[0.0, 0, 0, 3.0]]))
    assert pairs[:, 0].tolist() == [1, 2]


# ---------------------------------------------------------------- O4 / springs
def test_ray_cast_across_slit_closed_form():
    rest, tets, group, fixed = synth._voxel_kuhn(2, 2, 2, 1.0, slit_levels=[1], s=-1)
    # slit at x = 1 for all z levels (s = -1): left block x in [0,1], right x in [1,2]
    prep = loop.prepare(rest, tets, group, np.zeros(rest.shape[0], np.uint8))
    # left-block vertex at (1, 1, 1): the centre of the slit face, left copy
    v = int(np.nonzero((rest == [1.0, 1.0, 1.0]).all(axis=1))[0][0])
    assert v < 27   # base (left) copy
    X = rest.copy()
    X[v] += np.array([0.125, 0.03, 0.07])   # off the voxel edge lines
    pairs = collision.self_pairs(X, prep.tets, prep.query)
    assert v in set(pairs[:, 0].tolist())
    vn = mesh.vertex_normals(X, prep.faces, X.shape[0])
    eps = 0.01
    st = springs.update_springs(X, prep.query, springs.SpringState.empty(prep.query.size), pairs,
                                np.zeros((0, 2), int), np.zeros((0, 4)), prep.faces, vn, eps)
    i = int(np.nonzero(prep.query == v)[0][0])
    assert st.active[i] and st.kind[i] == springs.KIND_SELF
    # the hit point lies on the right block's slit face x = 1, the target eps outside it
    face = prep.faces[st.face[i]]
    assert np.allclose(X[face][:, 0], 1.0)
    n = mesh.face_normals(X, face[None])[0]
    assert n[0] < 0
    tgt = st.target[i]
    assert math.isclose(tgt[0], 1.0 - eps, rel_tol=0, abs_tol=1e-12)
    # the ray runs along -n(v); n(v) is the normal of the pushed vertex's faces
    o = X[v]
    d = -vn[v]
    tpar = (1.0 - o[0]) / d[0]
    hit = o + tpar * d
    assert np.allclose(tgt[1:], hit[1:], atol=1e-12)
    # release: pulled back 2 eps outside -> released; 0.5 eps outside -> kept
    for back, keep in ((2 * eps, False), (0.5 * eps, True)):
        X2 = X.copy()
        X2[v, 0] = 1.0 - back
        vn2 = mesh.vertex_normals(X2, prep.faces, X2.shape[0])
        st2 = springs.update_springs(X2, prep.query, st, np.zeros((0, 2), int), np.zeros((0, 2), int),
                                     np.zeros((0, 4)), prep.faces, vn2, eps)
        assert bool(st2.active[i]) == keep


def test_sphere_target_closed_form_and_release():
    X = np.array([[1.0, 0.5, -0.25]])
    sph = np.array([[0.0, 0.0, 0.0, 2.0]])
    faces = np.zeros((0, 3), int)
    pairs = collision.sphere_pairs(X, np.array([0]), sph)
    st = springs.update_springs(X, np.array([0]), springs.SpringState.empty(1), np.zeros((0, 2), int),
                                pairs, sph, faces, np.zeros((1, 3)), 0.01)
    u = X[0] / np.linalg.norm(X[0])
    assert st.active[0] and st.kind[0] == springs.KIND_OBSTACLE
    assert np.allclose(st.target[0], 2.01 * u, atol=1e-15)
    Xo = (2.0 + 0.02) * u[None]
    st2 = springs.update_springs(Xo, np.array([0]), st, np.zeros((0, 2), int), np.zeros((0, 2), int),
                                 sph, faces, np.zeros((1, 3)), 0.01)
    assert not st2.active[0]
    Xk = (2.0 + 0.005) * u[None]
    st3 = springs.update_springs(Xk, np.array([0]), st, np.zeros((0, 2), int), np.zeros((0, 2), int),
                                 sph, faces, np.zeros((1, 3)), 0.01)
    assert st3.active[0]


def test_closest_point_triangle_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(50):
        q = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 2
        x, b1, b2 = springs.closest_point_triangle(p, *q)
        assert np.allclose(x, (1 - b1 - b2) * q[0] + b1 * q[1] + b2 * q[2], atol=1e-12)
        # brute force over a fine barycentric grid
        g = np.linspace(0, 1, 201)
        B1, B2 = np.meshgrid(g, g)
        ok = B1 + B2 <= 1
        pts = (1 - B1[ok] - B2[ok])[:, None] * q[0] + B1[ok][:, None] * q[1] + B2[ok][:, None] * q[2]
        dmin = np.min(np.linalg.norm(pts - p, axis=1))
        assert np.linalg.norm(x - p) <= dmin + 1e-12


def test_slab_prefilter_equals_plain_all_pairs():
    m = synth.small_finger(nx=16, ny=4, nz=4, n_ch=3)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X = synth.perturbed_positions(m, 0.35, seed=13)
    a = collision.self_pairs(X, prep.tets, prep.query)
    b = collision.self_pairs(X, prep.tets, prep.query, n_slabs=1)
    assert np.array_equal(a, b) and a.shape[0] > 0


# ------------------------------------------------- vertex normals (reading G18)
def test_vertex_normal_is_area_weighted_closed_form():
    """Corner vertex of the right-angle tet (0,0,0), (a,0,0), (0,b,0), (0,0,c)
    with a, b, c unequal: its three boundary faces lie in the coordinate
    planes with outward normals -z, -x, -y and areas ab/2, bc/2, ac/2, so the
    normalised sum of the unnormalised face normals is -(bc, ac, ab)/|.|.
    A uniform or angle weighting gives -(1, 1, 1)/sqrt(3) here (the three
    face angles at the corner are all 90 degrees), and a missing
    normalisation gives the wrong length."""
    a, b, c = 1.0, 2.0, 4.0
    X = np.array([[0.0, 0, 0], [a, 0, 0], [0, b, 0], [0, 0, c]])
    tets = np.array([[0, 1, 2, 3]])
    faces = mesh.boundary_faces(tets)
    vn = mesh.vertex_normals(X, faces, 4)
    expect = -np.array([b * c, a * c, a * b])
    expect /= np.linalg.norm(expect)
    assert np.allclose(vn[0], expect, rtol=0, atol=1e-15)
    assert math.isclose(np.linalg.norm(vn[0]), 1.0, rel_tol=0, abs_tol=1e-15)
    assert not np.allclose(vn[0], -np.ones(3) / math.sqrt(3.0), atol=1e-3)
    # the ray from the corner along -n(v) runs along the normal of the
    # opposite face x/a + y/b + z/c = 1 and hits it at the foot of the
    # perpendicular from the origin: abc (bc, ac, ab) / (b^2c^2 + a^2c^2 + a^2b^2)
    fn = mesh.face_normals(X, faces)
    f, b1, b2, fb = springs.ray_cast_target(X, 0, vn[0], faces, fn)
    assert not fb
    assert sorted(faces[f].tolist()) == [1, 2, 3]
    hit = (1 - b1 - b2) * X[faces[f, 0]] + b1 * X[faces[f, 1]] + b2 * X[faces[f, 2]]
    den = (b * c) ** 2 + (a * c) ** 2 + (a * b) ** 2
    foot = a * b * c * np.array([b * c, a * c, a * b]) / den
    assert np.allclose(hit, foot, rtol=0, atol=1e-14)


def test_vertex_normal_of_a_skewed_corner():
    """A corner where two incident faces meet at 60 degrees with areas in the
    ratio 1 : 3: a vertex at the origin of the tet (0,0,0), (1,0,0),
    (cos60, sin60, 0) * 3, (0,0,1) has faces in the plane z = 0 (area 3/2 sin60,
    outward -z), in the plane y = 0 (area 1/2, outward -y) and in the plane
    through the z axis at 60 degrees (area 3/2, outward normal
    (sin60, -cos60, 0)); the area-weighted normal is the normalised sum of
    area * unit normal."""
    s, co = math.sin(math.pi / 3), math.cos(math.pi / 3)
    X = np.array([[0.0, 0, 0], [1, 0, 0], [3 * co, 3 * s, 0], [0, 0, 1]])
    tets = np.array([[0, 1, 2, 3]])
    faces = mesh.boundary_faces(tets)
    vn = mesh.vertex_normals(X, faces, 4)
    acc = 1.5 * s * np.array([0, 0, -1.0]) + 0.5 * np.array([0, -1.0, 0]) + 1.5 * np.array([-s, co, 0])
    assert np.allclose(vn[0], acc / np.linalg.norm(acc), rtol=0, atol=1e-15)


# ------------------------------------------ ray cast against a linear solve
def _ray_tri_solve(o, d, q0, q1, q2):
    """o + t d = q0 + b1 (q1 - q0) + b2 (q2 - q0) as a 3x3 linear system."""
    M = np.stack([d, -(q1 - q0), -(q2 - q0)], axis=1)
    t, b1, b2 = np.linalg.solve(M, q0 - o)
    return t, b1, b2


def test_ray_triangle_test_equals_linear_solve():
    rng = np.random.default_rng(21)
    o = rng.normal(size=3)
    d = rng.normal(size=3)
    q = rng.normal(size=(400, 3, 3)) * 2.0
    hit, t, b1, b2 = springs._ray_triangles(o, d, q[:, 0], q[:, 1], q[:, 2])
    n_hit = 0
    for k in range(q.shape[0]):
        ts, s1, s2 = _ray_tri_solve(o, d, *q[k])
        margin = min(s1, s2, 1 - s1 - s2, ts)
        if abs(margin) < 1e-9:
            continue
        assert bool(hit[k]) == (margin > 0), k
        assert np.allclose([t[k], b1[k], b2[k]], [ts, s1, s2], rtol=1e-9, atol=1e-12)
        n_hit += int(margin > 0)
    assert n_hit > 10


def test_ray_cast_target_equals_brute_force_on_a_penetrating_finger():
    """Every self-pair vertex of a perturbed small finger: the first exit face
    along -n(v) found by solving each face's 3x3 system one by one."""
    m = synth.small_finger(nx=16, ny=4, nz=4, n_ch=3)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X = synth.perturbed_positions(m, 0.35, seed=13)
    pairs = collision.self_pairs(X, prep.tets, prep.query)
    vn = mesh.vertex_normals(X, prep.faces, X.shape[0])
    fn = mesh.face_normals(X, prep.faces)
    checked = 0
    for v in np.unique(pairs[:, 0]):
        d = -vn[v]
        best = None
        for f in range(prep.faces.shape[0]):
            fv = prep.faces[f]
            if v in fv or float(fn[f] @ d) <= 0.0:
                continue
            t, s1, s2 = _ray_tri_solve(X[v], d, X[fv[0]], X[fv[1]], X[fv[2]])
            if min(s1, s2, 1 - s1 - s2) >= -1e-12 and t > 0 and (best is None or t < best[0] - 1e-12):
                best = (t, f, s1, s2)
        f, b1, b2, fb = springs.ray_cast_target(X, v, vn[v], prep.faces, fn)
        if best is None:
            assert fb
            continue
        assert not fb and f == best[1], v
        assert np.allclose([b1, b2], best[2:], atol=1e-9)
        checked += 1
    assert checked >= 5


# ------------------------------------------------ tetrahedral obstacle (Eq. 4)
def test_closest_points_array_rule_equals_scalar_rule():
    from oracle import obstacle

    rng = np.random.default_rng(31)
    for _ in range(20):
        q = rng.normal(size=(50, 3, 3))
        p = rng.normal(size=3) * 1.5
        x, b1, b2 = obstacle.closest_points(p, q[:, 0], q[:, 1], q[:, 2])
        for k in range(q.shape[0]):
            xs, s1, s2 = springs.closest_point_triangle(p, *q[k])
            assert np.allclose(x[k], xs, atol=1e-12)
            assert abs(b1[k] - s1) <= 1e-9 and abs(b2[k] - s2) <= 1e-9


def test_box_obstacle_pairs_closest_point_target_and_release():
    """Unit-cube obstacle (one voxel, 6 Kuhn tets): a generic point inside lies
    in exactly one tet; the closest boundary point is the projection onto the
    nearest cube face (closed form: distance min(x, 1-x, y, 1-y, z, 1-z)); the
    target is that point moved eps outward; the release test flips between
    0.5 eps and 2 eps outside."""
    from oracle import obstacle

    X, tets = synth.box_obstacle(1, 1, 1, 1.0, (0.0, 0.0, 0.0))
    obs = obstacle.prepare(X, tets)
    assert obs.faces.shape[0] == 12
    rng = np.random.default_rng(5)
    P = rng.uniform(0.02, 0.98, size=(40, 3))
    outside = np.array([[1.5, 0.5, 0.5], [-0.1, 0.2, 0.3], [0.5, 0.5, 1.0 + 1e-9]])
    Xr = np.concatenate([P, outside])
    pr = obstacle.pairs(Xr, np.arange(Xr.shape[0]), obs)
    counts = np.bincount(pr[:, 0], minlength=Xr.shape[0])
    assert np.all(counts[:40] == 1) and np.all(counts[40:] == 0)
    eps = 0.01
    for p in P:
        f, b1, b2, d2 = obstacle.closest_boundary_point(p, obs)
        dist = np.array([p[0], 1 - p[0], p[1], 1 - p[1], p[2], 1 - p[2]])
        j = int(np.argmin(dist))
        assert math.isclose(math.sqrt(d2), dist[j], rel_tol=0, abs_tol=1e-12)
        ax, side = j // 2, j % 2
        foot = p.copy()
        foot[ax] = float(side)
        b, n = obstacle.face_point_and_normal(obs, f, b1, b2)
        assert np.allclose(b, foot, atol=1e-12)
        out = np.zeros(3)
        out[ax] = 1.0 if side == 1 else -1.0
        assert np.allclose(n, out, atol=1e-12)
        assert np.allclose(obstacle.target(obs, f, b1, b2, eps), foot + eps * out, atol=1e-12)
        assert obstacle.released(foot + 2 * eps * out, obs, f, b1, b2, eps)
        assert not obstacle.released(foot + 0.5 * eps * out, obs, f, b1, b2, eps)


def test_obstacle_spring_update_precedence_and_kinds():
    """A vertex inside the box obstacle gets a mesh-obstacle spring; inside
    both a sphere and the box, the smaller signed surface distance wins."""
    from oracle import obstacle

    X, tets = synth.box_obstacle(2, 2, 2, 0.5, (0.0, 0.0, 0.0))
    obs = obstacle.prepare(X, tets)
    Xr = np.array([[0.3, 0.45, 0.52], [0.47, 0.53, 0.05]])
    q = np.arange(2)
    pm = obstacle.pairs(Xr, q, obs)
    assert sorted(set(pm[:, 0].tolist())) == [0, 1]
    # sphere around vertex 1 only, reaching far inside: |x - c| - r = -0.25,
    # while vertex 1 is 0.05 from the box bottom (signed distance -0.05)
    sph = np.array([[0.47, 0.53, 0.05, 0.25]])
    ps = collision.sphere_pairs(Xr, q, sph)
    st = springs.update_springs(Xr, q, springs.SpringState.empty(2), np.zeros((0, 2), int), ps, sph,
                                np.zeros((0, 3), int), np.zeros((2, 3)), 0.01, obs, pm)
    assert st.kind[0] == springs.KIND_MESH_OBSTACLE and st.active[0]
    assert st.kind[1] == springs.KIND_OBSTACLE and st.face[1] == 0
    # vertex 0 is 0.3 from x = 0, 0.48 from z = 1 ... nearest face x = 0 at distance 0.3
    assert np.allclose(st.target[0], [-0.01, 0.45, 0.52], atol=1e-12)
