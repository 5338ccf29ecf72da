"""Anderson-accelerated loop on the GPU (Sec. III-B) against the FP64 oracle:
the same proposals, energies and safeguard decisions step by step, and the
same positions; memory 0 is the plain loop."""
import numpy as np
import pytest

from oracle import anderson
from paper_2203_02054_gb300 import casim, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    casim.load_library()


@pytest.mark.parametrize("collision", [synth.COLLISION_OFF, synth.COLLISION_SELF])
def test_anderson_matches_oracle_fp64(collision):
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, seed=7, n_iters=16, precision=synth.PRECISION_FP64,
                           collision=collision)
    mem, n = 5, 16
    X_o, _st, recs_o = anderson.run_anderson(m, n, mem)
    sim = casim.Sim(m)
    recs, n_acc = sim.step_anderson(n, mem)
    assert sim.sync() >= 0
    assert n_acc == sum(r["accepted"] for r in recs) == sum(r.accepted for r in recs_o)
    assert n_acc > 0
    for r, ro in zip(recs, recs_o):
        if np.isnan(ro.e_prev):
            assert not r["proposed"]
            continue
        assert r["proposed"]
        assert abs(r["e_prev"] - ro.e_prev) <= 1e-9 * abs(ro.e_prev)
        assert abs(r["e_acc"] - ro.e_acc) <= 1e-9 * abs(ro.e_acc)
        # decisions taken in FP64 on both sides; no near-tie in this run
        assert abs(ro.e_acc - ro.e_prev) > 1e-8 * abs(ro.e_prev)
        assert bool(r["accepted"]) == ro.accepted
    X = sim.positions()
    assert np.abs(X - X_o).max() <= 1e-8 * m.bbox_diag()
    sim.close()


def test_memory_zero_is_plain_step():
    m = synth.small_finger(nx=16, ny=4, nz=4, n_ch=3, seed=5, n_iters=6)
    a = casim.Sim(m)
    recs, n_acc = a.step_anderson(6, 0)
    assert n_acc == 0 and not any(r["proposed"] for r in recs)
    b = casim.Sim(m)
    b.step(6)
    assert a.sync() >= 0 and b.sync() >= 0
    assert np.array_equal(a.positions(), b.positions())
    a.close()
    b.close()
