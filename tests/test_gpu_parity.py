"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bars: contact pair sets bit-exact on identical positions; final positions
within 1e-5 of the bounding-box diagonal (the FP64 path is held to 1e-9);
element targets within the FP32 rounding of the MIXED path."""
import numpy as np
import pytest

from paper_2203_02054_gb300 import casim, synth
from oracle import collision, local, loop, mesh as omesh, springs as osprings

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5      # x bounding-box diagonal


@pytest.fixture(scope="module", autouse=True)
def _lib():
    casim.load_library()


def _oracle_springs_from(prep, rec):
    """Spring records of the C ABI's layout as an oracle SpringState."""
    st = osprings.SpringState.empty(prep.query.shape[0])
    assert np.array_equal(rec["verts"], prep.query)
    st.active = rec["active"].copy()
    st.kind = rec["kind"].astype(np.int8)
    st.face = rec["face"].astype(np.int64)
    st.bary = rec["bary"].copy()
    st.target = rec["target"].copy()
    return st


# ------------------------------------------------------------ whole loop
def test_beam_fp64_matches_oracle():
    m = synth.config1_beam()
    sim = casim.Sim(m)
    sim.step(m.n_iters)
    assert sim.sync() == 0
    Xg = sim.positions()
    hist = sim.history()
    ref = loop.run_mesh(m)
    diag = m.bbox_diag()
    err = np.abs(Xg - ref.X).max()
    assert err <= 1e-9 * diag, err
    Eg = np.array([h["energy"] for h in hist])
    Eo = np.array([h.energy for h in ref.history])
    assert np.allclose(Eg, Eo, rtol=1e-9, atol=1e-12)
    assert all(h["pcg_rel_residual"] <= 1e-12 for h in hist)
    sim.close()


def test_small_finger_fp64_whole_loop_with_collision_matches_oracle():
    """FP64 path, 30 free-running iterations with self-collision: same contact
    and spring counts every iteration and positions within 1e-9 diag."""
    m = synth.small_finger(n_iters=30, precision=synth.PRECISION_FP64)
    sim = casim.Sim(m)
    sim.step(m.n_iters)
    assert sim.sync() == 0
    hist = sim.history()
    ref = loop.run_mesh(m)
    assert np.abs(sim.positions() - ref.X).max() <= 1e-9 * m.bbox_diag()
    assert [h["n_self_pairs"] for h in hist] == [h.n_self_pairs for h in ref.history]
    assert [h["n_springs"] for h in hist] == [h.n_springs for h in ref.history]
    assert max(h.n_springs for h in ref.history) > 0
    sim.close()


def _release_margin(X, prep, st, qi, spheres, eps):
    """Oracle-side distance of spring qi's release test from its threshold."""
    v = prep.query[qi]
    if st.kind[qi] == osprings.KIND_OBSTACLE:
        c, r = spheres[st.face[qi], :3], spheres[st.face[qi], 3]
        return float(np.linalg.norm(X[v] - c) - r - eps)
    f = prep.faces[st.face[qi]]
    q0, q1, q2 = X[f[0]], X[f[1]], X[f[2]]
    b1, b2 = st.bary[qi]
    bp = (1 - b1 - b2) * q0 + b1 * q1 + b2 * q2
    n = np.cross(q1 - q0, q2 - q0)
    n = n / np.linalg.norm(n)
    return float(np.dot(n, X[v] - bp) - eps)


def test_small_finger_mixed_replay_every_iteration():
    """MIXED path along the oracle's 30-iteration trajectory: from each oracle
    state (rounded to FP32) one GPU iteration must give the same pair set bit
    for bit, the same spring decisions (a decision may differ only where the
    oracle's release test is within 1e-5 cm of its threshold) and positions
    within 1e-5 of the bounding-box diagonal."""
    m = synth.small_finger(n_iters=30)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    sim = casim.Sim(m)
    X = m.rest.copy()
    st = osprings.SpringState.empty(prep.query.shape[0])
    compared = 0
    for i in range(m.n_iters):
        Xf = X.astype(np.float32).astype(np.float64)
        sim.set_positions(Xf)
        sim.set_springs(prep.query.astype(np.int32), st.active, st.kind.astype(np.int32), st.face.astype(np.int32),
                        st.bary, st.target)
        sim.step(1)
        assert sim.sync() == 0
        Xn, stn, rec, ps, po = loop.iterate(prep, Xf, st, m.alpha, m.spheres, m.w_knots, m.k_spring, m.eps,
                                            m.collision)
        assert np.array_equal(sim.contacts()[0], ps), i
        sp = sim.springs()
        diff = np.nonzero(sp["active"] != stn.active)[0]
        for qi in diff:
            assert st.active[qi], (i, qi)          # only a release decision can tie
            assert abs(_release_margin(Xf, prep, st, qi, m.spheres, m.eps)) < 1e-5, (i, qi)
        if diff.size == 0:
            same = stn.active
            assert np.allclose(sp["target"][same], stn.target[same], atol=1e-9)
            err = np.abs(sim.positions() - Xn).max()
            assert err <= POS_TOL * m.bbox_diag(), (i, err)
            compared += 1
        X, st = Xn, stn
    assert compared >= m.n_iters - 2
    sim.close()


def test_finger_ragged_sizes_mixed():
    # odd sizes: several thread blocks plus ragged tails everywhere
    m = synth.small_finger(nx=23, ny=5, nz=5, n_ch=3, seed=21, n_iters=12)
    sim = casim.Sim(m)
    sim.step(m.n_iters)
    assert sim.sync() == 0
    ref = loop.run_mesh(m)
    err = np.abs(sim.positions() - ref.X).max()
    assert err <= POS_TOL * m.bbox_diag(), err
    sim.close()


# ------------------------------------------------------------ replay parity
def _replay_one(m, X0, sim=None):
    """One GPU iteration from X0 (already FP32-exact for MIXED) with no prior
    springs, and the oracle's same iteration."""
    sim = sim or casim.Sim(m)
    sim.set_positions(X0)
    sim.step(1)
    assert sim.sync() in (0, casim.CASIM_W_PCG_MAXIT)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    Xn, st, rec, ps, po = loop.iterate(prep, X0, osprings.SpringState.empty(prep.query.shape[0]), m.alpha,
                                       m.spheres, m.w_knots, m.k_spring, m.eps, m.collision)
    return sim, prep, Xn, st, rec, ps, po


@pytest.mark.parametrize("amp,seed", [(0.25, 1), (0.4, 2)])
def test_replay_pairs_bit_exact_and_step_parity(amp, seed):
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4)
    X0 = synth.perturbed_positions(m, amp, seed=seed, dtype=np.float32)
    sim, prep, Xn, st, rec, ps, po = _replay_one(m, X0)
    pairs, obs = sim.contacts()
    assert ps.shape[0] > 0
    assert np.array_equal(pairs, ps)                      # bit-exact pair set
    sp = sim.springs()
    assert np.array_equal(sp["active"], st.active)
    assert np.array_equal(sp["kind"][st.active], st.kind[st.active])
    assert np.array_equal(sp["face"][st.active], st.face[st.active])
    assert np.allclose(sp["target"], st.target, atol=1e-9)
    assert np.allclose(sp["bary"], st.bary, atol=1e-9)
    # local step targets (FP32 rotation fit vs LAPACK FP64)
    P_or, *_ = local.local_step(X0, prep.tets, prep.T_c, prep.vol0, prep.group, m.alpha, m.w_knots)
    P_gpu = sim.targets()
    assert np.abs(P_gpu - P_or).max() <= 2e-5 * m.h * 10
    err = np.abs(sim.positions() - Xn).max()
    assert err <= POS_TOL * m.bbox_diag(), err
    sim.close()


def test_replay_fp64_targets_tight():
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, precision=synth.PRECISION_FP64)
    X0 = synth.perturbed_positions(m, 0.3, seed=5)
    sim, prep, Xn, st, rec, ps, po = _replay_one(m, X0)
    pairs, _ = sim.contacts()
    assert np.array_equal(pairs, ps)
    P_or, *_ = local.local_step(X0, prep.tets, prep.T_c, prep.vol0, prep.group, m.alpha, m.w_knots)
    assert np.abs(sim.targets() - P_or).max() <= 1e-12
    assert np.abs(sim.positions() - Xn).max() <= 1e-9 * m.bbox_diag()
    sim.close()


def test_replay_with_prior_springs_release_and_retarget():
    """Two oracle iterations give springs that the third releases or keeps;
    the GPU, handed the same state, must update them identically."""
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    X0 = synth.perturbed_positions(m, 0.3, seed=9, dtype=np.float32)
    r = loop.run_mesh(m, n_iters=2, X0=X0, prep=prep)
    X2 = r.X.astype(np.float32).astype(np.float64)
    st2 = r.springs
    sim = casim.Sim(m)
    sim.set_positions(X2)
    sim.set_springs(prep.query.astype(np.int32), st2.active, st2.kind.astype(np.int32), st2.face.astype(np.int32),
                    st2.bary, st2.target)
    sim.step(1)
    assert sim.sync() == 0
    Xn, st3, rec, ps, po = loop.iterate(prep, X2, st2, m.alpha, m.spheres, m.w_knots, m.k_spring, m.eps, m.collision)
    sp = sim.springs()
    assert np.array_equal(sim.contacts()[0], ps)
    assert np.array_equal(sp["active"], st3.active)
    assert np.allclose(sp["target"], st3.target, atol=1e-9)
    assert np.abs(sim.positions() - Xn).max() <= POS_TOL * m.bbox_diag()
    sim.close()


def test_sphere_obstacle_replay():
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, collision=synth.COLLISION_SELF_OBSTACLE)
    # two spheres overlapping the finger's top and side surfaces
    m.spheres = np.array([[5.0, 1.0, 2.6, 0.8], [7.5, -0.4, 1.0, 0.7]])
    X0 = synth.perturbed_positions(m, 0.2, seed=12, dtype=np.float32)
    sim, prep, Xn, st, rec, ps, po = _replay_one(m, X0)
    pairs, obs = sim.contacts()
    assert po.shape[0] > 0
    assert np.array_equal(obs, np.unique(po[:, 0]))
    assert np.array_equal(pairs, ps)
    sp = sim.springs()
    assert np.array_equal(sp["active"], st.active)
    assert np.array_equal(sp["kind"], st.kind.astype(np.int32))
    assert np.allclose(sp["target"], st.target, atol=1e-9)
    assert np.abs(sim.positions() - Xn).max() <= POS_TOL * m.bbox_diag()
    sim.close()


def test_integer_grid_exact_predicates():
    """Positions on an integer lattice put many query vertices exactly on
    faces, edges and vertices of other tets; the exact predicates must agree."""
    m = synth.small_finger(nx=12, ny=4, nz=4, n_ch=2, precision=synth.PRECISION_FP64)
    rng = np.random.default_rng(3)
    X0 = m.rest.copy()
    free = m.fixed == 0
    X0[free] += rng.integers(-1, 2, size=(int(free.sum()), 3)) * 0.25
    sim = casim.Sim(m)
    sim.set_positions(X0)
    sim.step(1)
    sim.sync()
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    ps = collision.self_pairs(X0, prep.tets, prep.query)
    assert np.array_equal(sim.contacts()[0], ps)
    sim.close()


def test_rest_state_is_fixed_point_on_gpu():
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4)
    m.alpha = np.ones_like(m.alpha)
    sim = casim.Sim(m, knots=((0.0, 1.0),))
    X0 = sim.positions()
    sim.step(3)
    assert sim.sync() == 0
    hist = sim.history()
    assert all(h["n_self_pairs"] == 0 and h["n_springs"] == 0 for h in hist)
    assert np.abs(sim.positions() - X0).max() <= 1e-5 * m.h
    sim.close()


# ------------------------------------------------------------ system behaviour
def test_deterministic_and_checkpoint_resume():
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, n_iters=10)
    a = casim.Sim(m)
    a.step(4)
    a.sync()
    blob = casim.casim_save_state(a.h)
    a.step(6)
    a.sync()
    Xa = a.positions()
    b = casim.Sim(m)
    b.step(10)
    b.sync()
    assert np.array_equal(Xa, b.positions())       # bitwise determinism
    c = casim.Sim(m)
    casim.casim_load_state(c.h, blob)
    c.step(6)
    c.sync()
    assert np.array_equal(Xa, c.positions())       # resume from checkpoint
    for s in (a, b, c):
        s.close()


def test_pcg_cap_warning():
    m = synth.config2_finger()
    sim = casim.Sim(m, pcg_max_iter=1)
    sim.step(1)
    assert sim.sync() == casim.CASIM_W_PCG_MAXIT
    sim.close()


@pytest.mark.parametrize("kernel", [2, 5])
def test_pcg_wait_gives_up_with_timeout_status(kernel):
    """A wait for a block that does not exist (the grid barrier of kernel 2,
    the partial poll of kernel 5) must give up after its clock budget (~10 ms
    here) with a timeout status; the context stays usable afterwards."""
    m = synth.config2_finger()
    sim = casim.Sim(m, wait_budget_cycles=20_000_000, debug_flags=casim.CASIM_DEBUG_BARRIER_NEVER_COMPLETES,
                    pcg_kernel=kernel)
    assert sim.stats().pcg_kernel == kernel
    sim.step(1)
    with pytest.raises(casim.CasimError) as ei:
        sim.sync()
    assert ei.value.code == casim.CASIM_E_TIMEOUT
    sim.close()
    sim = casim.Sim(m)
    sim.step(1)
    assert sim.sync() == 0
    sim.close()


def test_host_validation_rejects_bad_input_before_launch():
    m = synth.config1_beam()
    sim = casim.Sim(m)
    X = m.rest.copy()
    X[3, 1] = np.nan
    with pytest.raises(casim.CasimError) as ei:
        sim.set_positions(X)
    assert ei.value.code == casim.CASIM_E_INVALID
    bad = m.tets.copy()
    bad[0, 0] = m.n_verts + 5
    with pytest.raises(casim.CasimError):
        casim.casim_upload_mesh(sim.h, m.rest, bad, m.group, m.fixed)
    free = np.zeros(m.n_verts, np.uint8)
    with pytest.raises(casim.CasimError) as ei:
        casim.casim_upload_mesh(sim.h, m.rest, m.tets, m.group, free)
    assert ei.value.code == casim.CASIM_E_SINGULAR
    sim.close()


@pytest.mark.parametrize("kernel", [1, 2, 3, 5])
def test_both_pcg_kernels_match_oracle(kernel):
    m = synth.small_finger(nx=24, ny=4, nz=4, n_ch=4, seed=31, n_iters=8)
    sim = casim.Sim(m, pcg_kernel=kernel)
    assert sim.stats().pcg_kernel == kernel
    sim.step(m.n_iters)
    assert sim.sync() == 0
    ref = loop.run_mesh(m)
    err = np.abs(sim.positions() - ref.X).max()
    assert err <= POS_TOL * m.bbox_diag(), err
    sim.close()
