"""Parity at the full workload sizes, in the launch configuration the
benchmark times (default parameters: auto PCG kernel, CUDA graph).

The oracle cannot run hundreds of iterations at 50k-200k tets in a test, so
these tests compare single iterations from seeded states, sample the contact
check vertex by vertex, and check properties of full-length runs that hold at
any size (convergence of every global solve, determinism, finiteness)."""
import numpy as np
import pytest

from paper_2203_02054_gb300 import casim, synth
from oracle import collision, global_step, local, loop, springs as osprings

pytestmark = pytest.mark.gpu
POS_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    casim.load_library()


def _one_iteration(m, X0):
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    sim = casim.Sim(m)
    sim.set_positions(X0)
    sim.step(1)
    status = sim.sync()
    Xn, st, rec, ps, po = loop.iterate(prep, X0, osprings.SpringState.empty(prep.query.shape[0]), m.alpha,
                                       m.spheres, m.w_knots, m.k_spring, m.eps, m.collision)
    return sim, prep, status, Xn, st, ps, po


def test_finger_51840_tets_one_iteration_replay():
    m = synth.config2_finger()
    X0 = synth.perturbed_positions(m, 0.25, seed=101, dtype=np.float32)
    sim, prep, status, Xn, st, ps, po = _one_iteration(m, X0)
    assert status == 0
    pairs, _ = sim.contacts()
    assert ps.shape[0] > 100
    assert np.array_equal(pairs, ps)
    sp = sim.springs()
    assert np.array_equal(sp["active"], st.active)
    assert np.allclose(sp["target"], st.target, atol=1e-9)
    assert np.abs(sim.positions() - Xn).max() <= POS_TOL * m.bbox_diag()
    sim.close()


def test_gripper_193920_tets_first_iteration_and_sampled_contacts():
    m = synth.config3_gripper()
    # first iteration from rest (touching slit faces are not contacts)
    sim, prep, status, Xn, st, ps, po = _one_iteration(m, m.rest.copy())
    assert status == 0 and ps.shape[0] == 0
    assert np.abs(sim.positions() - Xn).max() <= POS_TOL * m.bbox_diag()
    sim.close()
    # a perturbed state with the sphere pushed into one finger: contacts of a
    # seeded sample of vertices, decided one by one by the oracle
    m.spheres = np.array([[6.5, 0.0, -10.0, 3.0]])
    X0 = synth.perturbed_positions(m, 0.3, seed=102, dtype=np.float32)
    sim = casim.Sim(m)
    sim.set_positions(X0)
    sim.step(1)
    assert sim.sync() in (0, casim.CASIM_W_PCG_MAXIT)
    pairs, obs = sim.contacts()
    rng = np.random.default_rng(103)
    sample = np.sort(rng.choice(prep.query, size=1500, replace=False))
    expect = collision.self_pairs(X0, prep.tets, sample)
    got = pairs[np.isin(pairs[:, 0], sample)]
    assert expect.shape[0] > 10
    assert np.array_equal(got, expect)
    eo = collision.sphere_pairs(X0, prep.query, m.spheres)
    assert eo.shape[0] > 0 and np.array_equal(obs, np.unique(eo[:, 0]))
    sim.close()


def test_gripper_full_run_properties():
    """200 iterations of the benchmark workload: every PCG solve converges to
    its tolerance, nothing turns non-finite, contacts arise and are resolved
    by springs, and a second run is bitwise identical."""
    m = synth.config3_gripper()
    outs = []
    for _ in range(2):
        sim = casim.Sim(m)
        sim.step(m.n_iters)
        assert sim.sync() == 0
        hist = sim.history()
        X = sim.positions()
        assert np.all(np.isfinite(X))
        assert len(hist) == m.n_iters
        assert all(h["pcg_rel_residual"] <= 1e-6 for h in hist)
        assert all(np.isfinite(h["energy"]) for h in hist)
        assert max(h["n_springs"] for h in hist) > 0
        outs.append(X)
        sim.close()
    assert np.array_equal(outs[0], outs[1])


def test_gripper_graph_branches_match_one_stream():
    """The CUDA graph runs the local step on a branch beside the spring update
    and the ray casts; eager launches on one stream (stats=2) run the same
    kernels in sequence.  Every reduction has a fixed order, so any race
    between the branches would show as a difference: positions, spring
    records and every iteration's record must agree bit for bit."""
    m = synth.config3_gripper()
    n = 60
    runs = []
    for stats in (1, 2):
        sim = casim.Sim(m, stats=stats)
        sim.step(n)
        assert sim.sync() == 0
        runs.append((sim.positions(), sim.springs(), sim.history()))
        sim.close()
    (xa, sa, ha), (xb, sb, hb) = runs
    assert np.array_equal(xa, xb)
    for key in ("active", "kind", "face", "bary", "target"):
        assert np.array_equal(sa[key], sb[key]), key
    assert len(ha) == len(hb) == n
    assert ha == hb
    assert max(h["n_springs"] for h in ha) > 0


def _oracle_springs(prep, rec):
    st = osprings.SpringState.empty(prep.query.shape[0])
    assert np.array_equal(rec["verts"], prep.query)
    st.active = rec["active"].copy()
    st.kind = rec["kind"].astype(np.int8)
    st.face = rec["face"].astype(np.int64)
    st.bary = rec["bary"].copy()
    st.target = rec["target"].copy()
    return st


def _oracle_global_with(prep, m, X, rec):
    """The oracle's local and global steps from X with the spring set of
    another update (active vertices and their targets) held as given."""
    P, *_ = local.local_step(X, prep.tets, prep.T_c, prep.vol0, prep.group, m.alpha, m.w_knots)
    act = rec["active"]
    A, b = global_step.assemble(prep.tets, prep.omega, P, prep.n_verts, prep.query[act], rec["target"][act],
                                m.k_spring)
    return global_step.solve(A, b, X, prep.fixed)


def _ray_t(X, v, nrm, face):
    q0, q1, q2 = X[face[0]], X[face[1]], X[face[2]]
    M = np.stack([-nrm, -(q1 - q0), -(q2 - q0)], axis=1)
    return float(np.linalg.solve(M, q0 - X[v])[0])


def _replay_along_trajectory(m, checkpoints):
    """Runs the GPU loop from rest; at each checkpoint k it takes the GPU's
    state (X_k and the spring records of iteration k-1), runs one more GPU
    iteration and the oracle's iteration k from the same state, and compares:
    pair sets bit for bit, obstacle vertices, spring decisions (a decision may
    differ only where the oracle's release test is within 1e-5 cm of its
    threshold), targets of equal decisions (1e-9; a different hit face only
    where the two faces' ray parameters tie within 1e-9), and X_{k+1} within
    1e-5 of the bounding-box diagonal against the oracle's solve with the
    GPU's spring set (and against the oracle's own X_{k+1} when every
    decision agrees)."""
    from test_gpu_parity import _release_margin

    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    sim = casim.Sim(m)
    done = 0
    tol = POS_TOL * m.bbox_diag()
    out = []
    for k in checkpoints:
        sim.step(k - done)
        assert sim.sync() == 0
        Xk = sim.positions()
        st_prev = _oracle_springs(prep, sim.springs())
        sim.step(1)
        done = k + 1
        assert sim.sync() == 0
        pairs, obs = sim.contacts()
        rec = sim.springs()
        Xg = sim.positions()
        Xn, stn, orec, ps, po = loop.iterate(prep, Xk, st_prev, m.alpha, m.spheres, m.w_knots, m.k_spring, m.eps,
                                             m.collision)
        assert np.array_equal(pairs, ps), k
        assert np.array_equal(obs, np.unique(po[:, 0]) if po.shape[0] else obs[:0]), k
        diff = np.nonzero(rec["active"] != stn.active)[0]
        for qi in diff:
            assert st_prev.active[qi], (k, qi)
            assert abs(_release_margin(Xk, prep, st_prev, qi, m.spheres, m.eps)) < 1e-5, (k, qi)
        same = np.nonzero(rec["active"] & stn.active)[0]
        assert np.array_equal(rec["kind"][same], stn.kind[same].astype(np.int32)), k
        face_diff = same[rec["face"][same] != stn.face[same]]
        vn = None
        if face_diff.size:
            from oracle import mesh as omesh

            vn = omesh.vertex_normals(Xk, prep.faces, prep.n_verts)
        for qi in face_diff:
            v = prep.query[qi]
            ta = _ray_t(Xk, v, -vn[v], prep.faces[rec["face"][qi]])
            tb = _ray_t(Xk, v, -vn[v], prep.faces[stn.face[qi]])
            assert abs(ta - tb) <= 1e-9 * max(1.0, abs(tb)), (k, qi, ta, tb)
        eq = np.setdiff1d(same, face_diff)
        assert np.abs(rec["target"][eq] - stn.target[eq]).max(initial=0.0) <= 1e-9, k
        Xs = _oracle_global_with(prep, m, Xk, rec)
        err_s = float(np.abs(Xg - Xs).max())
        assert err_s <= tol, (k, err_s)
        if diff.size == 0 and face_diff.size == 0:
            assert float(np.abs(Xg - Xn).max()) <= tol, k
        out.append(dict(k=k, pairs=int(ps.shape[0]), obstacle_pairs=int(po.shape[0]),
                        springs=int(rec["active"].sum()), decision_ties=int(diff.size),
                        face_ties=int(face_diff.size), err=err_s))
    sim.close()
    return out


def test_gripper_mid_trajectory_replay_with_contacts():
    """The benchmark workload (193,920 tets) at outer iterations 50, 100 and
    199, with self and obstacle springs active."""
    m = synth.config3_gripper()
    res = _replay_along_trajectory(m, [50, 100, 199])
    print(res)
    assert all(r["pairs"] > 100 and r["springs"] > 100 for r in res)
    assert res[-1]["obstacle_pairs"] > 0 and res[-2]["obstacle_pairs"] > 0


def test_finger_mid_trajectory_replay_with_contacts():
    """The 51,840-tet finger at outer iterations 50 and 99."""
    m = synth.config2_finger()
    res = _replay_along_trajectory(m, [50, 99])
    print(res)
    assert all(r["pairs"] > 100 and r["springs"] > 100 for r in res)
