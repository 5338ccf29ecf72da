"""Autotuner of the simulator's kernel choices and launch shapes.

Host logic only: every candidate configuration is a simulation created
through the C ABI and timed with CUDA events on its stream, so what is
measured is exactly what a user of that configuration runs.  The tuned
dimensions are

* the global-step kernel and its preconditioner (``pcg_kernel``,
  ``pcg_precond``: for one robot the dataflow kernel with the two-level or the
  Jacobi preconditioner, the register-resident and the streaming kernels; for
  a batch the segmented and the cluster kernels) and the dataflow kernel's
  rows per block (``pcg_block``),
* the collision broad phase (``broad_phase``: spatial hash or AABB trees) and
  the hash cell edge (``cell_scale`` times the voxel edge),
* the thread-block sizes of the local step, the RHS gather and the narrow
  phase (``local_block``, ``rhs_block``, ``narrow_block``),

searched one dimension at a time from the defaults (coordinate descent; a
value replaces the current one only when it is faster by more than 1%).  A
candidate counts only if its run ends with device status 0 and finite
positions.  The winners are cached per GPU name and workload shape (vertex,
tet and robot counts, precision, collision mode) in a JSON file;
``apply_cached`` copies them into a ``casim_params`` before upload.

    python -m paper_2203_02054_gb300.autotune --workload gripper --iters 20
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from typing import Dict, List, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE_PATH = os.path.join(HERE, "tuned.json")

PARAM_KEYS = ("pcg_kernel", "pcg_precond", "pcg_block", "broad_phase", "cell_scale", "local_block", "rhs_block",
              "narrow_block")
DEFAULTS = dict(pcg_kernel=0, pcg_precond=0, pcg_block=0, broad_phase=0, cell_scale=1.0, local_block=0,
                rhs_block=0, narrow_block=0)


def gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name(torch.cuda.current_device())


def workload_key(mesh) -> str:
    """Shape of a workload: a generator Mesh or a list of them (a batch)."""
    ms = list(mesh) if isinstance(mesh, (list, tuple)) else [mesh]
    nv = sum(m.n_verts for m in ms)
    nt = sum(m.n_tets for m in ms)
    return "v%d_t%d_r%d_p%d_c%d" % (nv, nt, len(ms), ms[0].precision, ms[0].collision)


def dimensions(mesh) -> List[List[Dict]]:
    """Candidate values per dimension, in search order."""
    from . import synth

    batch = isinstance(mesh, (list, tuple))
    first = mesh[0] if batch else mesh
    if batch:
        pcg = [dict(pcg_kernel=0, pcg_precond=0), dict(pcg_kernel=3, pcg_precond=0)]
    else:
        pcg = [dict(pcg_kernel=0, pcg_precond=0), dict(pcg_kernel=2, pcg_precond=0), dict(pcg_kernel=1, pcg_precond=0)]
        if first.precision == synth.PRECISION_MIXED:
            pcg.insert(1, dict(pcg_kernel=0, pcg_precond=1))
    dims = [pcg]
    if not batch and first.precision == synth.PRECISION_MIXED:
        dims.append([dict(pcg_block=b) for b in (0, 288, 384)])
    if first.collision >= 1:
        # the hash's cell edge first, then the tree against the tuned hash
        dims.append([dict(cell_scale=c) for c in (1.0, 0.75, 1.5, 2.0)])
        dims.append([dict(broad_phase=0), dict(broad_phase=1)])
        dims.append([dict(narrow_block=b) for b in (0, 128, 512)])
    dims.append([dict(local_block=b) for b in (0, 64, 256)])
    dims.append([dict(rhs_block=b) for b in (0, 128, 512)])
    return dims


def measure(mesh, cfg: Dict, iters: int, stream) -> Optional[float]:
    """Milliseconds per outer iteration of ``iters`` iterations from rest
    (after 3 warm-up iterations), or None when the configuration is refused
    at upload or its run does not end cleanly."""
    import torch

    from . import casim

    kw = {k: cfg[k] for k in PARAM_KEYS}
    try:
        sim = casim.Sim(mesh, stream=stream.cuda_stream, stats=0, **kw)
    except casim.CasimError:
        return None
    try:
        sim.step(3)
        sim.sync()
        sim.reset()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        sim.step(iters)
        b.record(stream)
        torch.cuda.synchronize()
        if sim.sync() != 0 or not np.all(np.isfinite(sim.positions())):
            return None
        return a.elapsed_time(b) / iters
    except casim.CasimError:
        return None
    finally:
        sim.close()


def tune(mesh, iters: int = 20, log=print, measure_fn=None) -> Dict:
    """Coordinate descent over ``dimensions(mesh)``; returns the record that
    ``save`` stores (winners, their time, the defaults' time, every trial).
    ``measure_fn(mesh, cfg, iters)`` replaces the GPU timing (tests)."""
    if measure_fn is None:
        import torch

        stream = torch.cuda.current_stream()
        measure_fn = lambda m, c, n: measure(m, c, n, stream)  # noqa: E731
    best = dict(DEFAULTS)
    t_best = measure_fn(mesh, best, iters)
    if t_best is None:
        raise RuntimeError("the default configuration does not run cleanly")
    t_default = t_best
    trials = [dict(best, ms_per_iter=t_best)]
    log("default: %.4f ms/iter" % t_best)
    for dim in dimensions(mesh):
        for cand in dim:
            cfg = dict(best, **cand)
            if all(cfg[k] == best[k] for k in PARAM_KEYS):
                continue
            if cfg["broad_phase"] == 1 and cfg["cell_scale"] != best["cell_scale"]:
                continue  # the cell edge only matters to the hash
            t = measure_fn(mesh, cfg, iters)
            trials.append(dict(cfg, ms_per_iter=t))
            log("%s: %s" % (cand, "refused" if t is None else "%.4f ms/iter" % t))
            if t is not None and t < 0.99 * t_best:
                best, t_best = cfg, t
    return dict(params=best, ms_per_iter=t_best, default_ms_per_iter=t_default, iters=iters, trials=trials,
                when=time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()))


def load(path: str = CACHE_PATH) -> Dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save(record: Dict, mesh, path: str = CACHE_PATH, gpu: Optional[str] = None) -> None:
    data = load(path)
    data.setdefault(gpu or gpu_name(), {})[workload_key(mesh)] = record
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cached(mesh, path: str = CACHE_PATH, gpu: Optional[str] = None) -> Optional[Dict]:
    try:
        name = gpu or gpu_name()
    except Exception:
        return None
    return load(path).get(name, {}).get(workload_key(mesh))


def apply_cached(params, mesh, path: str = CACHE_PATH) -> Optional[Dict]:
    """Copies the cached winners for this GPU and workload shape into the
    ctypes ``casim_params`` (the cell edge as a multiple of the current one);
    returns the applied parameters, or None when nothing is cached."""
    rec = cached(mesh, path)
    if not rec:
        return None
    p = rec["params"]
    for k in ("pcg_kernel", "pcg_precond", "pcg_block", "broad_phase", "local_block", "rhs_block", "narrow_block"):
        setattr(params, k, int(p.get(k, 0)))
    params.cell_size = params.cell_size * float(p["cell_scale"])
    return dict(p)


def _workload(name: str):
    from . import synth

    if name == "gripper":
        return synth.config3_gripper()
    if name == "finger":
        return synth.config2_finger()
    if name == "beam":
        return synth.config1_beam()
    if name == "batch":
        return synth.config4_batch()
    raise ValueError(name)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", action="append", required=True,
                    choices=["gripper", "finger", "beam", "batch"])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--cache", default=CACHE_PATH)
    args = ap.parse_args(argv)
    import torch

    from . import casim

    casim.load_library()
    torch.cuda.set_device(0)
    for w in args.workload:
        m = _workload(w)
        print("== %s (%s) on %s" % (w, workload_key(m), gpu_name()), flush=True)
        rec = tune(m, args.iters, log=lambda s: print("  " + s, flush=True))
        save(rec, m, args.cache)
        print("  winner %s: %.4f ms/iter (default %.4f)" % (rec["params"], rec["ms_per_iter"],
                                                           rec["default_ms_per_iter"]), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
