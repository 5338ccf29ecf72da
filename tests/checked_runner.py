"""Runs small cases on the bounds-checked library (libcasim_checked.so) in its
own process (the binding loads one library per process) and prints one JSON
line of results; tests/test_gpu_checked.py drives it."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import loop  # noqa: E402
from oracle import springs as osprings  # noqa: E402
from paper_2203_02054_gb300 import casim, synth  # noqa: E402


def main():
    casim.load_library(casim.LIB_CHECKED_PATH)
    out = {"checked": int(casim.load_library().casim_build_checked())}
    # FP64 finger with self collision against the oracle's whole run
    m = synth.small_finger(n_iters=20, precision=synth.PRECISION_FP64)
    sim = casim.Sim(m)
    sim.step(m.n_iters)
    out["fp64_status"] = sim.sync()
    ref = loop.run_mesh(m)
    out["fp64_err"] = float(np.abs(sim.positions() - ref.X).max() / m.bbox_diag())
    out["fp64_springs"] = [h["n_springs"] for h in sim.history()] == [h.n_springs for h in ref.history]
    sim.close()
    # MIXED: one iteration from a perturbed state against the oracle
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4)
    X0 = synth.perturbed_positions(m, 0.3, seed=5, dtype=np.float32)
    prep = loop.prepare(m.rest, m.tets, m.group, m.fixed)
    Xn, st, rec, ps, po = loop.iterate(prep, X0, osprings.SpringState.empty(prep.query.shape[0]), m.alpha,
                                       m.spheres, m.w_knots, m.k_spring, m.eps, m.collision)
    sim = casim.Sim(m)
    sim.set_positions(X0)
    sim.step(1)
    out["mixed_status"] = sim.sync()
    out["mixed_pairs_equal"] = bool(np.array_equal(sim.contacts()[0], ps)) and ps.shape[0] > 0
    out["mixed_err"] = float(np.abs(sim.positions() - Xn).max() / m.bbox_diag())
    sim.close()
    # the benchmark gripper (dataflow PCG, full collision path), 20 iterations
    m = synth.config3_gripper()
    sim = casim.Sim(m)
    sim.step(20)
    out["gripper_status"] = sim.sync()
    out["gripper_finite"] = bool(np.all(np.isfinite(sim.positions())))
    sim.close()
    # a small batch (segmented PCG), 5 iterations
    batch = synth.config4_batch(n_robots=8, n_iters=5)
    sim = casim.Sim(batch)
    sim.step(5)
    out["batch_status"] = sim.sync()
    sim.close()
    # fault injection: an out-of-range incidence entry planted on the device
    m = synth.small_finger(n_iters=2)
    sim = casim.Sim(m, debug_flags=casim.CASIM_DEBUG_CORRUPT_INCIDENCE)
    sim.step(1)
    try:
        out["corrupt_status"] = sim.sync()
    except casim.CasimError as e:
        out["corrupt_status"] = e.code
    out["corrupt_bits"] = int(sim.stats().status_bits)
    sim.close()
    # the context stays usable
    sim = casim.Sim(m)
    sim.step(2)
    out["after_status"] = sim.sync()
    sim.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
