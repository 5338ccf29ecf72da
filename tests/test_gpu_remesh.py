"""Remesh trigger and progressive actuation on the GPU (Sec. III-C,
Algorithm 1 outer loop) against the FP64 oracle.  The flags are integer
decisions taken in FP64 on both sides from the same positions; elements
within 1e-9 (relative) of a threshold, where the two FP64 evaluations may
round differently, are excluded from the bit-exact comparison."""
import numpy as np
import pytest

from oracle import remesh
from paper_2203_02054_gb300 import casim, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    casim.load_library()


def _clear(ratio, smax, amax, dmax, group):
    return (group >= 0) & (np.abs(ratio - amax) > 1e-9 * amax) & (np.abs(smax - dmax) > 1e-9 * dmax)


@pytest.mark.parametrize("precision", [synth.PRECISION_MIXED, synth.PRECISION_FP64])
def test_flags_match_oracle_on_the_same_positions(precision):
    m = synth.small_finger(nx=24, ny=4, nz=4, n_ch=4, seed=31, n_iters=8, precision=precision)
    sim = casim.Sim(m)
    sim.step(8)
    assert sim.sync() >= 0
    X = sim.positions()
    amax, dmax = 1.3, 1.15
    flags, n_flagged, gvr = sim.remesh_flags(None, amax, dmax)
    oflags, ratio, smax, ogvr = remesh.remesh_flags(X, m.rest, m.tets, m.group, amax, dmax)
    ok = _clear(ratio, smax, amax, dmax, m.group)
    assert np.array_equal(flags[ok], oflags[ok])
    assert np.all(flags[m.group < 0] == 0)
    assert n_flagged == int(np.count_nonzero(flags))
    assert n_flagged > 0 and np.count_nonzero(flags & remesh.FLAG_DISTORTION) > 0
    assert np.count_nonzero(flags & remesh.FLAG_VOLUME) > 0
    for g, v in ogvr.items():
        assert abs(gvr[g] - v) <= 1e-12 * abs(v)
    # an explicit reference equal to the rest shape gives the same answer
    flags2, n2, gvr2 = sim.remesh_flags(m.rest, amax, dmax)
    assert np.array_equal(flags2, flags) and n2 == n_flagged and np.array_equal(gvr2, gvr)
    # against the current shape itself nothing changes
    flags3, n3, gvr3 = sim.remesh_flags(X, amax, dmax)
    assert n3 == 0 and np.allclose(gvr3, 1.0, rtol=1e-12)
    sim.close()


def test_progressive_matches_oracle_fp64():
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4, seed=7, n_iters=5, precision=synth.PRECISION_FP64)
    target = np.asarray(m.alpha, dtype=np.float64)
    step = 1.2   # ratios 1.2, 2.4, ... capped at the targets (1.5 to 2.5 here)
    amax, dmax = 1.05, 1.05
    X_o, recs_o = remesh.progressive(m, target, step, n_inner=5, alpha_max=amax, d_max=dmax)
    sim = casim.Sim(m)
    recs = sim.progressive(target, step, n_inner=5, alpha_max=amax, d_max=dmax)
    assert len(recs) == len(recs_o) == int(np.ceil(target.max() / step))
    X = sim.positions()
    assert np.abs(X - X_o).max() <= 1e-9 * m.bbox_diag()
    for r, ro in zip(recs, recs_o):
        assert r["k"] == ro.k and r["status"] >= 0
        assert r["applied_max"] == float(np.max(ro.applied))
        lo, hi = min(ro.chamber_volume_ratio.values()), max(ro.chamber_volume_ratio.values())
        assert abs(r["chamber_volume_ratio_min"] - lo) <= 1e-9 * lo
        assert abs(r["chamber_volume_ratio_max"] - hi) <= 1e-9 * hi
        assert r["n_flagged"] == ro.n_flagged and r["n_volume"] == ro.n_volume
        assert r["n_distortion"] == ro.n_distortion
    assert recs_o[0].n_flagged > 0
    # the targets are applied at the end
    assert recs[-1]["applied_max"] == float(target.max())
    sim.close()


def test_remesh_arguments_are_validated():
    m = synth.small_finger(nx=16, ny=4, nz=4, n_ch=3, seed=5, n_iters=2)
    sim = casim.Sim(m)
    with pytest.raises(casim.CasimError):
        sim.remesh_flags(None, -1.0, 4.0)
    with pytest.raises(casim.CasimError):
        casim.casim_progressive(sim.h, np.ones(m.n_groups + 1), 2.0, 1)
    with pytest.raises(casim.CasimError):
        sim.progressive(np.asarray(m.alpha), 0.0, 1)
    sim.close()
