"""AABB-tree broad phase (Sec. II-B: trees over the robot and the obstacle,
built once, boxes refitted as the body deforms) and the rigid tetrahedral
obstacle (Eq. 4, Sec. II-C closest-point response), against the oracle's
brute-force definitions and against the spatial-hash broad phase."""
import numpy as np
import pytest

from paper_2203_02054_gb300 import casim, synth
from oracle import collision, loop
from oracle import obstacle as oobst
from oracle import springs as osprings

pytestmark = pytest.mark.gpu
POS_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    casim.load_library()


def _one(m, X0, broad, st0=None):
    sim = casim.Sim(m, broad_phase=broad)
    sim.set_positions(X0)
    if st0 is not None:
        sim.set_springs(st0["verts"], st0["active"], st0["kind"], st0["face"], st0["bary"], st0["target"])
    sim.step(1)
    assert sim.sync() in (0, casim.CASIM_W_PCG_MAXIT)
    out = dict(pairs=sim.contacts()[0], obs=sim.contacts()[1], springs=sim.springs(), X=sim.positions())
    sim.close()
    return out


@pytest.mark.parametrize("amp,seed", [(0.3, 1), (0.45, 2)])
def test_tree_pairs_springs_and_step_equal_oracle(amp, seed):
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4)
    X0 = synth.perturbed_positions(m, amp, seed=seed, dtype=np.float32)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    Xn, st, rec, ps, po = loop.iterate(prep, X0, osprings.SpringState.empty(prep.query.shape[0]), m.alpha,
                                       m.spheres, m.w_knots, m.k_spring, m.eps, m.collision)
    tree = _one(m, X0, 1)
    hsh = _one(m, X0, 0)
    assert ps.shape[0] > 10
    assert np.array_equal(tree["pairs"], ps)
    assert np.array_equal(tree["pairs"], hsh["pairs"])
    sp = tree["springs"]
    assert np.array_equal(sp["active"], st.active)
    assert np.array_equal(sp["face"][st.active], st.face[st.active])
    assert np.allclose(sp["target"], st.target, atol=1e-9)
    assert np.abs(tree["X"] - Xn).max() <= POS_TOL * m.bbox_diag()


def test_tree_whole_loop_fp64_equals_oracle():
    m = synth.small_finger(n_iters=20, precision=synth.PRECISION_FP64)
    sim = casim.Sim(m, broad_phase=1)
    sim.step(m.n_iters)
    assert sim.sync() == 0
    hist = sim.history()
    ref = loop.run_mesh(m)
    assert np.abs(sim.positions() - ref.X).max() <= 1e-9 * m.bbox_diag()
    assert [h["n_self_pairs"] for h in hist] == [h.n_self_pairs for h in ref.history]
    assert [h["n_springs"] for h in hist] == [h.n_springs for h in ref.history]
    assert max(h.n_springs for h in ref.history) > 0
    sim.close()


def _finger_with_box(precision):
    """A small finger whose chambers press against a box obstacle above its
    top surface (the box's lower face 0.05 cm below the finger's rest top, so
    the top vertices start inside it)."""
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, precision=precision,
                           collision=synth.COLLISION_SELF_OBSTACLE, n_iters=12)
    dt = np.float32 if precision == synth.PRECISION_MIXED else np.float64
    OX, otets = synth.box_obstacle(4, 3, 2, 0.5, (4.13, -0.21, 1.95), dtype=dt)
    m.obstacle_X, m.obstacle_tets = OX, otets
    return m


def test_tetrahedral_obstacle_whole_loop_fp64_both_broad_phases():
    m = _finger_with_box(synth.PRECISION_FP64)
    ref = loop.run_mesh(m)
    assert max(h.n_obstacle_pairs for h in ref.history) > 0
    assert np.any(ref.springs.kind == osprings.KIND_MESH_OBSTACLE)
    for broad in (0, 1):
        sim = casim.Sim(m, broad_phase=broad)
        sim.step(m.n_iters)
        assert sim.sync() == 0
        hist = sim.history()
        assert [h["n_obstacle_pairs"] for h in hist] == [h.n_obstacle_pairs for h in ref.history], broad
        assert [h["n_springs"] for h in hist] == [h.n_springs for h in ref.history], broad
        sp = sim.springs()
        assert np.array_equal(sp["kind"][sp["active"]], ref.springs.kind[ref.springs.active].astype(np.int32))
        assert np.abs(sim.positions() - ref.X).max() <= 1e-9 * m.bbox_diag(), broad
        sim.close()


def test_tetrahedral_obstacle_mixed_replay():
    m = _finger_with_box(synth.PRECISION_MIXED)
    X0 = synth.perturbed_positions(m, 0.2, seed=17, dtype=np.float32)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    obs = oobst.prepare(m.obstacle_X, m.obstacle_tets)
    Xn, st, rec, ps, po = loop.iterate(prep, X0, osprings.SpringState.empty(prep.query.shape[0]), m.alpha,
                                       m.spheres, m.w_knots, m.k_spring, m.eps, m.collision, obs)
    sph_pairs, mesh_pairs = po
    assert mesh_pairs.shape[0] > 0
    for broad in (0, 1):
        out = _one(m, X0, broad)
        assert np.array_equal(out["pairs"], ps)
        assert np.array_equal(out["obs"], np.unique(mesh_pairs[:, 0]))
        sp = out["springs"]
        assert np.array_equal(sp["active"], st.active)
        assert np.array_equal(sp["kind"], st.kind.astype(np.int32))
        assert np.array_equal(sp["face"][st.active], st.face[st.active])
        assert np.allclose(sp["target"], st.target, atol=1e-9)
        assert np.abs(out["X"] - Xn).max() <= POS_TOL * m.bbox_diag()


def test_tree_equals_hash_on_gripper_trajectory():
    """The benchmark gripper (193,920 tets) at iterations 60 and 120 of a
    hash-mode run: the tree broad phase finds the same pairs, obstacle
    vertices and spring records from the same state, and the pairs of a
    seeded sample of vertices equal the oracle's brute force."""
    m = synth.config3_gripper()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    run = casim.Sim(m)
    done = 0
    rng = np.random.default_rng(7)
    for k in (60, 120):
        run.step(k - done)
        done = k
        assert run.sync() == 0
        Xk = run.positions()
        st_prev = run.springs()
        outs = [_one(m, Xk, broad, st_prev) for broad in (0, 1)]
        assert np.array_equal(outs[0]["pairs"], outs[1]["pairs"]), k
        assert np.array_equal(outs[0]["obs"], outs[1]["obs"]), k
        for key in ("active", "kind", "face"):
            assert np.array_equal(outs[0]["springs"][key], outs[1]["springs"][key]), (k, key)
        assert np.allclose(outs[0]["springs"]["target"], outs[1]["springs"]["target"], atol=1e-12)
        sample = np.sort(rng.choice(prep.query, size=800, replace=False))
        expect = collision.self_pairs(Xk, prep.tets, sample)
        got = outs[1]["pairs"][np.isin(outs[1]["pairs"][:, 0], sample)]
        assert expect.shape[0] > 10 and np.array_equal(got, expect), k
    run.close()


def _stacked_tets(n_over):
    """Tet 0 has one free vertex near the origin; tets 1..n_over are fixed,
    slightly differently scaled copies of the unit corner tet, shifted so
    that each strictly contains the free vertex."""
    rest = [[0.001, 0.0013, 0.0017], [0.6, 0.0, 0.0], [0.0, 0.6, 0.0], [0.0, 0.0, 0.6]]
    tets = [[0, 1, 2, 3]]
    for k in range(1, n_over + 1):
        s = 1.0 + 0.01 * k
        base = len(rest)
        for c in ([0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]):
            rest.append([s * (c[0] - 0.2), s * (c[1] - 0.2), s * (c[2] - 0.2)])
        tets.append([base, base + 1, base + 2, base + 3])
    rest = np.array(rest, np.float64)
    fixed = np.ones(rest.shape[0], np.uint8)
    fixed[0] = 0
    return synth.Mesh(name="stacked", rest=rest, tets=np.array(tets, np.int32),
                      group=np.full(len(tets), -1, np.int32), fixed=fixed, alpha=np.zeros(0), n_iters=1)


@pytest.mark.parametrize("max_pairs", [8, 16])
def test_truncated_pair_list_keeps_the_smallest_tets(max_pairs):
    """A vertex strictly inside 20 tets: both broad phases keep the max_pairs
    smallest tet ids of the brute-force pair set and raise the truncation
    warning."""
    m = _stacked_tets(20)
    expect = collision.self_pairs(m.rest, m.tets, np.array([0]))
    assert expect.shape[0] == 20
    for broad in (0, 1):
        sim = casim.Sim(m, broad_phase=broad, max_pairs=max_pairs)
        sim.step(1)
        assert sim.sync() in (casim.CASIM_W_PCG_MAXIT, casim.CASIM_W_PAIRS_TRUNCATED), broad
        assert sim.stats().status_bits & 16, broad  # a pair list was truncated
        assert np.array_equal(sim.contacts()[0], expect[:max_pairs]), broad
        sim.close()
