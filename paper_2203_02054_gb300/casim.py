"""Python binding of the casim C ABI (``include/casim.h``): argument marshalling only.

Every function named ``casim_*`` here calls the C entry point of the same name
in ``libcasim.so``; every step of the simulation runs in the CUDA library.
Loading fails loudly (``ImportError``) when the library has not been built:
there is no fallback implementation.

``Sim`` is a small convenience wrapper that owns a handle and converts numpy
arrays; device outputs may be any CUDA pointer (for example a torch tensor's
``data_ptr()``).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcasim.so")
# the same library with every gather index of the hot kernels bounds-checked
# on the device (built alongside it; see casim_build_checked)
LIB_CHECKED_PATH = os.path.join(HERE, "libcasim_checked.so")

CASIM_OK = 0
CASIM_E_INVALID = -1
CASIM_E_CUDA = -2
CASIM_E_SINGULAR = -3
CASIM_E_STATE = -4
CASIM_E_CAPACITY = -5
CASIM_E_NONFINITE = -6
CASIM_E_TIMEOUT = -7
CASIM_E_OVERFLOW = -8
CASIM_E_BOUNDS = -9
CASIM_W_PCG_MAXIT = 1
CASIM_W_PAIRS_TRUNCATED = 2

CASIM_FP64 = 0
CASIM_MIXED = 1
CASIM_DEBUG_BARRIER_NEVER_COMPLETES = 1
CASIM_DEBUG_CORRUPT_INCIDENCE = 2

EXPORTS = [
    "casim_default_params", "casim_create", "casim_upload_mesh", "casim_upload_batch", "casim_set_actuation",
    "casim_set_spheres", "casim_set_obstacle_mesh", "casim_set_positions", "casim_reset", "casim_step", "casim_forward_ckpt",
    "casim_backward", "casim_sync", "casim_get_positions",
    "casim_get_contacts", "casim_get_springs", "casim_set_springs", "casim_get_targets",
    "casim_get_history", "casim_get_stats", "casim_save_state", "casim_load_state",
    "casim_get_sizes", "casim_get_phase_times", "casim_contacts_noalloc", "casim_remesh_flags",
    "casim_progressive", "casim_step_anderson", "casim_destroy", "casim_last_error", "casim_build_checked",
]


class casim_params(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("collision", ctypes.c_int32),
        ("k_spring", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("pcg_tol", ctypes.c_double),
        ("pcg_max_iter", ctypes.c_int32),
        ("n_w_knots", ctypes.c_int32),
        ("w_knots", ctypes.POINTER(ctypes.c_double)),
        ("cell_size", ctypes.c_double),
        ("stats", ctypes.c_int32),
        ("max_pairs_per_vertex", ctypes.c_int32),
        ("wait_budget_cycles", ctypes.c_uint64),
        ("pcg_kernel", ctypes.c_int32),
        ("debug_flags", ctypes.c_int32),
        ("pcg_precond", ctypes.c_int32),
        ("broad_phase", ctypes.c_int32),
        ("local_block", ctypes.c_int32),
        ("rhs_block", ctypes.c_int32),
        ("narrow_block", ctypes.c_int32),
        ("pcg_block", ctypes.c_int32),
    ]


class casim_iter_record(ctypes.Structure):
    _fields_ = [
        ("energy", ctypes.c_double),
        ("pcg_rel_residual", ctypes.c_double),
        ("n_self_pairs", ctypes.c_int32),
        ("n_obstacle_pairs", ctypes.c_int32),
        ("n_springs", ctypes.c_int32),
        ("pcg_iters", ctypes.c_int32),
        ("knot_signature", ctypes.c_uint64),
        ("spring_signature", ctypes.c_uint64),
    ]


class casim_stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int64),
        ("total_pcg_iters", ctypes.c_int64),
        ("last", casim_iter_record),
        ("status", ctypes.c_int32),
        ("pcg_kernel", ctypes.c_int32),
        ("status_bits", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class casim_outer_record(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("n_volume", ctypes.c_int32),
        ("n_distortion", ctypes.c_int32),
        ("n_flagged", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("applied_max", ctypes.c_double),
        ("chamber_volume_ratio_min", ctypes.c_double),
        ("chamber_volume_ratio_max", ctypes.c_double),
    ]


class casim_aa_record(ctypes.Structure):
    _fields_ = [
        ("e_prev", ctypes.c_double),
        ("e_acc", ctypes.c_double),
        ("accepted", ctypes.c_int32),
        ("proposed", ctypes.c_int32),
    ]


class casim_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("n_verts", ctypes.c_int32),
        ("rest_xyz", ctypes.POINTER(ctypes.c_double)),
        ("n_tets", ctypes.c_int32),
        ("tets", ctypes.POINTER(ctypes.c_int32)),
        ("tet_group", ctypes.POINTER(ctypes.c_int32)),
        ("fixed", ctypes.POINTER(ctypes.c_uint8)),
    ]


class CasimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("casim error %d: %s" % (code, msg))
        self.code = code


_lib: Optional[ctypes.CDLL] = None

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libcasim.so and declares every entry point's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libcasim.so is not built (%s); run __graft_entry__.build()" % path)
    L = ctypes.CDLL(path)
    L.casim_default_params.argtypes = [ctypes.POINTER(casim_params)]
    L.casim_default_params.restype = None
    L.casim_create.argtypes = [ctypes.POINTER(casim_params), _P, ctypes.POINTER(_P)]
    L.casim_upload_mesh.argtypes = [_P, ctypes.c_int32, _D, ctypes.c_int32, _I32, _I32, _U8]
    L.casim_upload_batch.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(casim_mesh_desc)]
    L.casim_set_actuation.argtypes = [_P, ctypes.c_int32, _D]
    L.casim_set_spheres.argtypes = [_P, ctypes.c_int32, _D]
    L.casim_set_obstacle_mesh.argtypes = [_P, ctypes.c_int32, _D, ctypes.c_int32, _I32]
    L.casim_set_positions.argtypes = [_P, _D]
    L.casim_reset.argtypes = [_P]
    L.casim_step.argtypes = [_P, ctypes.c_int32]
    L.casim_forward_ckpt.argtypes = [_P, ctypes.c_int32, ctypes.c_int32]
    L.casim_backward.argtypes = [_P, _D, _D]
    L.casim_sync.argtypes = [_P]
    L.casim_get_positions.argtypes = [_P, _D, _P]
    L.casim_get_contacts.argtypes = [_P, _I32, _I64, _I32, _I64]
    L.casim_get_springs.argtypes = [_P, _I64, _I32, _U8, _I32, _I32, _D, _D]
    L.casim_set_springs.argtypes = [_P, ctypes.c_int64, _I32, _U8, _I32, _I32, _D, _D]
    L.casim_get_targets.argtypes = [_P, _D]
    L.casim_get_history.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(casim_iter_record), _I32]
    L.casim_get_stats.argtypes = [_P, ctypes.POINTER(casim_stats)]
    L.casim_save_state.argtypes = [_P, _P, ctypes.POINTER(ctypes.c_size_t)]
    L.casim_load_state.argtypes = [_P, _P, ctypes.c_size_t]
    L.casim_get_sizes.argtypes = [_P, _I32, _I32, _I32, _I32, _I32]
    L.casim_get_phase_times.argtypes = [_P, _D]
    L.casim_contacts_noalloc.argtypes = [ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_int32, _P,
                                         ctypes.c_double, ctypes.c_int32, _P, _P, _P]
    L.casim_remesh_flags.argtypes = [_P, _D, ctypes.c_double, ctypes.c_double, _U8, _I32, ctypes.c_int32, _D]
    L.casim_progressive.argtypes = [_P, ctypes.c_int32, _D, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_double, ctypes.POINTER(casim_outer_record), _I32]
    L.casim_step_anderson.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(casim_aa_record), _I32]
    L.casim_destroy.argtypes = [_P]
    L.casim_build_checked.argtypes = []
    L.casim_destroy.restype = None
    L.casim_last_error.argtypes = [_P]
    L.casim_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        f = getattr(L, name)
        if name not in ("casim_default_params", "casim_destroy", "casim_last_error"):
            f.restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check(rc: int, sim=None, allow_warning: bool = True) -> int:
    if rc < 0 or (rc > 0 and not allow_warning):
        msg = load_library().casim_last_error(sim).decode()
        raise CasimError(rc, msg)
    return rc


# ---- same-name wrappers ---------------------------------------------------
def casim_default_params() -> casim_params:
    p = casim_params()
    load_library().casim_default_params(ctypes.byref(p))
    return p


def casim_create(params: casim_params, stream: int = 0):
    h = _P()
    rc = load_library().casim_create(ctypes.byref(params), _P(stream or None), ctypes.byref(h))
    _check(rc, None)
    return h


def casim_upload_mesh(sim, rest, tets, group, fixed):
    rest = np.ascontiguousarray(rest, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    group = np.ascontiguousarray(group, dtype=np.int32)
    fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
    rc = load_library().casim_upload_mesh(sim, rest.shape[0], _ptr(rest, ctypes.c_double), tets.shape[0],
                                          _ptr(tets, ctypes.c_int32), _ptr(group, ctypes.c_int32),
                                          _ptr(fixed, ctypes.c_uint8))
    return _check(rc, sim)


def casim_upload_batch(sim, meshes):
    """meshes: sequence of (rest, tets, group, fixed) array tuples."""
    keep = []
    descs = (casim_mesh_desc * len(meshes))()
    for i, (rest, tets, group, fixed) in enumerate(meshes):
        rest = np.ascontiguousarray(rest, dtype=np.float64)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        group = np.ascontiguousarray(group, dtype=np.int32)
        fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
        keep.append((rest, tets, group, fixed))
        descs[i] = casim_mesh_desc(rest.shape[0], _ptr(rest, ctypes.c_double), tets.shape[0],
                                   _ptr(tets, ctypes.c_int32), _ptr(group, ctypes.c_int32),
                                   _ptr(fixed, ctypes.c_uint8))
    rc = load_library().casim_upload_batch(sim, len(meshes), descs)
    del keep
    return _check(rc, sim)


def casim_set_actuation(sim, alpha):
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    return _check(load_library().casim_set_actuation(sim, a.shape[0], _ptr(a, ctypes.c_double)), sim)


def casim_set_spheres(sim, spheres):
    s = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    return _check(load_library().casim_set_spheres(sim, s.shape[0], _ptr(s, ctypes.c_double)), sim)


def casim_set_obstacle_mesh(sim, xyz, tets):
    x = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    t = np.ascontiguousarray(np.asarray(tets, dtype=np.int32).reshape(-1, 4))
    return _check(load_library().casim_set_obstacle_mesh(sim, x.shape[0], _ptr(x, ctypes.c_double), t.shape[0],
                                                         _ptr(t, ctypes.c_int32)), sim)


def casim_set_positions(sim, xyz):
    x = np.ascontiguousarray(xyz, dtype=np.float64)
    return _check(load_library().casim_set_positions(sim, _ptr(x, ctypes.c_double)), sim)


def casim_reset(sim):
    return _check(load_library().casim_reset(sim), sim)


def casim_step(sim, n_iters: int):
    return _check(load_library().casim_step(sim, int(n_iters)), sim)


def casim_forward_ckpt(sim, n_iters: int, ckpt_every: int):
    return _check(load_library().casim_forward_ckpt(sim, int(n_iters), int(ckpt_every)), sim)


def casim_backward(sim, dL_dX, n_groups: int) -> np.ndarray:
    g = np.ascontiguousarray(dL_dX, dtype=np.float64)
    out = np.zeros(max(n_groups, 1), dtype=np.float64)
    _check(load_library().casim_backward(sim, _ptr(g, ctypes.c_double), _ptr(out, ctypes.c_double)), sim)
    return out[:n_groups]


def casim_sync(sim) -> int:
    """Returns the device status (0 or a positive warning); raises on errors."""
    return _check(load_library().casim_sync(sim), sim)


def casim_get_sizes(sim):
    v = [ctypes.c_int32() for _ in range(5)]
    _check(load_library().casim_get_sizes(sim, *[ctypes.byref(x) for x in v]), sim)
    return dict(zip(["n_verts", "n_tets", "n_free", "n_boundary_faces", "n_query_verts"], [x.value for x in v]))


def casim_get_positions(sim, n_verts: int, dev_out: int = 0) -> Optional[np.ndarray]:
    if dev_out:
        _check(load_library().casim_get_positions(sim, None, _P(dev_out)), sim)
        return None
    out = np.empty((n_verts, 3), dtype=np.float64)
    _check(load_library().casim_get_positions(sim, _ptr(out, ctypes.c_double), None), sim)
    return out


def casim_get_contacts(sim):
    L = load_library()
    npairs = ctypes.c_int64(0)
    nobs = ctypes.c_int64(0)
    rc = L.casim_get_contacts(sim, None, ctypes.byref(npairs), None, ctypes.byref(nobs))
    if rc not in (CASIM_OK, CASIM_E_CAPACITY):
        _check(rc, sim)
    pairs = np.empty((max(npairs.value, 1), 2), dtype=np.int32)
    obs = np.empty(max(nobs.value, 1), dtype=np.int32)
    cp = ctypes.c_int64(pairs.shape[0])
    co = ctypes.c_int64(obs.shape[0])
    _check(L.casim_get_contacts(sim, _ptr(pairs, ctypes.c_int32), ctypes.byref(cp), _ptr(obs, ctypes.c_int32),
                                ctypes.byref(co)), sim)
    return pairs[:cp.value].astype(np.int64), obs[:co.value].astype(np.int64)


def casim_get_springs(sim, n_q: int):
    verts = np.empty(n_q, np.int32)
    active = np.empty(n_q, np.uint8)
    kind = np.empty(n_q, np.int32)
    face = np.empty(n_q, np.int32)
    bary = np.empty((n_q, 2), np.float64)
    target = np.empty((n_q, 3), np.float64)
    n = ctypes.c_int64(n_q)
    _check(load_library().casim_get_springs(sim, ctypes.byref(n), _ptr(verts, ctypes.c_int32),
                                            _ptr(active, ctypes.c_uint8), _ptr(kind, ctypes.c_int32),
                                            _ptr(face, ctypes.c_int32), _ptr(bary, ctypes.c_double),
                                            _ptr(target, ctypes.c_double)), sim)
    return dict(verts=verts, active=active.astype(bool), kind=kind, face=face, bary=bary, target=target)


def casim_set_springs(sim, verts, active, kind, face, bary, target):
    verts = np.ascontiguousarray(verts, np.int32)
    active = np.ascontiguousarray(active, np.uint8)
    kind = np.ascontiguousarray(kind, np.int32)
    face = np.ascontiguousarray(face, np.int32)
    bary = np.ascontiguousarray(bary, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    return _check(load_library().casim_set_springs(
        sim, verts.shape[0], _ptr(verts, ctypes.c_int32), _ptr(active, ctypes.c_uint8), _ptr(kind, ctypes.c_int32),
        _ptr(face, ctypes.c_int32), _ptr(bary, ctypes.c_double), _ptr(target, ctypes.c_double)), sim)


def casim_get_targets(sim, n_tets: int) -> np.ndarray:
    out = np.empty((n_tets, 3, 4), np.float64)
    _check(load_library().casim_get_targets(sim, _ptr(out, ctypes.c_double)), sim)
    return out


def casim_get_history(sim, cap: int = 4096):
    arr = (casim_iter_record * max(cap, 1))()
    n = ctypes.c_int32(0)
    _check(load_library().casim_get_history(sim, cap, arr, ctypes.byref(n)), sim)
    return [dict(energy=r.energy, pcg_rel_residual=r.pcg_rel_residual, n_self_pairs=r.n_self_pairs,
                 n_obstacle_pairs=r.n_obstacle_pairs, n_springs=r.n_springs, pcg_iters=r.pcg_iters,
                 knot_signature=r.knot_signature, spring_signature=r.spring_signature)
            for r in arr[:n.value]]


def casim_get_stats(sim) -> casim_stats:
    s = casim_stats()
    _check(load_library().casim_get_stats(sim, ctypes.byref(s)), sim)
    return s


def casim_save_state(sim) -> bytes:
    L = load_library()
    n = ctypes.c_size_t(0)
    _check(L.casim_save_state(sim, None, ctypes.byref(n)), sim)
    buf = ctypes.create_string_buffer(n.value)
    _check(L.casim_save_state(sim, ctypes.cast(buf, _P), ctypes.byref(n)), sim)
    return buf.raw[:n.value]


def casim_load_state(sim, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    return _check(load_library().casim_load_state(sim, ctypes.cast(buf, _P), len(blob)), sim)


def casim_get_phase_times(sim) -> np.ndarray:
    out = np.zeros(5, np.float64)
    _check(load_library().casim_get_phase_times(sim, _ptr(out, ctypes.c_double)), sim)
    return out


def casim_contacts_noalloc(n_verts: int, dev_xyz: int, n_tets: int, dev_tets: int, n_query: int, dev_query: int,
                           cell_size: float, max_pairs: int, dev_pair_count: int, dev_pair_tet: int,
                           stream: int = 0) -> int:
    """Allocation-free contact check on caller-owned device buffers (pointers
    as integers, e.g. torch ``data_ptr()``); returns the C status code."""
    return load_library().casim_contacts_noalloc(
        int(n_verts), _P(dev_xyz), int(n_tets), _P(dev_tets), int(n_query), _P(dev_query), float(cell_size),
        int(max_pairs), _P(dev_pair_count), _P(dev_pair_tet), _P(stream or None))


def casim_remesh_flags(sim, n_tets: int, n_groups: int, ref_xyz=None, alpha_max: float = 4.0, d_max: float = 4.0):
    """(flags uint8 (n_tets,), n_flagged, group volume ratios (n_groups,))."""
    flags = np.zeros(n_tets, np.uint8)
    nf = np.zeros(1, np.int32)
    gvr = np.zeros(max(n_groups, 1), np.float64)
    ref = None
    if ref_xyz is not None:
        ref = np.ascontiguousarray(np.asarray(ref_xyz, dtype=np.float64).reshape(-1))
    _check(load_library().casim_remesh_flags(sim, None if ref is None else _ptr(ref, ctypes.c_double), alpha_max,
                                             d_max, _ptr(flags, ctypes.c_uint8), _ptr(nf, ctypes.c_int32), n_groups,
                                             _ptr(gvr, ctypes.c_double) if n_groups else None), sim)
    return flags, int(nf[0]), gvr[:n_groups]


def casim_progressive(sim, alpha_target, alpha_step: float, n_inner: int, max_outer: int = 64,
                      alpha_max: float = 4.0, d_max: float = 4.0):
    """List of per-outer-step dicts (casim_outer_record fields)."""
    a = np.ascontiguousarray(np.asarray(alpha_target, dtype=np.float64))
    recs = (casim_outer_record * max_outer)()
    n = np.zeros(1, np.int32)
    _check(load_library().casim_progressive(sim, a.shape[0], _ptr(a, ctypes.c_double), alpha_step, n_inner,
                                            max_outer, alpha_max, d_max, recs, _ptr(n, ctypes.c_int32)), sim)
    names = [f[0] for f in casim_outer_record._fields_ if f[0] != "pad"]
    return [{k: getattr(recs[i], k) for k in names} for i in range(int(n[0]))]


def casim_step_anderson(sim, n_iters: int, m: int):
    """(list of per-iteration dicts (casim_aa_record fields), number of accepted proposals)."""
    recs = (casim_aa_record * max(n_iters, 1))()
    n = np.zeros(1, np.int32)
    _check(load_library().casim_step_anderson(sim, n_iters, m, recs, _ptr(n, ctypes.c_int32)), sim)
    names = [f[0] for f in casim_aa_record._fields_]
    return [{k: getattr(recs[i], k) for k in names} for i in range(n_iters)], int(n[0])


def casim_destroy(sim):
    load_library().casim_destroy(sim)


def casim_last_error(sim=None) -> str:
    return load_library().casim_last_error(sim).decode()


# ---- convenience wrapper ---------------------------------------------------
class Sim:
    """Owns one casim handle built from a generator ``Mesh``, or from a list of
    them (a batch of independent robots; parameters from the first)."""

    def __init__(self, mesh, precision=None, collision=None, stream: int = 0, stats: int = 1,
                 pcg_tol=None, pcg_max_iter=1000, knots=None, max_pairs=8, wait_budget_cycles=0,
                 pcg_kernel=0, debug_flags=0, pcg_precond=0, broad_phase=None, local_block=0, rhs_block=0,
                 narrow_block=0, cell_scale=1.0, tuned=False, pcg_block=0):
        load_library()
        self.batch = None
        if isinstance(mesh, (list, tuple)):
            self.batch = list(mesh)
            mesh = self.batch[0]
        p = casim_default_params()
        p.precision = mesh.precision if precision is None else precision
        p.collision = mesh.collision if collision is None else collision
        p.k_spring = mesh.k_spring
        p.eps = mesh.eps
        p.pcg_tol = (1e-12 if p.precision == CASIM_FP64 else 1e-6) if pcg_tol is None else pcg_tol
        p.pcg_max_iter = pcg_max_iter
        kn = np.ascontiguousarray(np.array(mesh.w_knots if knots is None else knots, dtype=np.float64).ravel())
        self._knots = kn
        p.n_w_knots = kn.shape[0] // 2
        p.w_knots = _ptr(kn, ctypes.c_double)
        p.cell_size = mesh.cell_size * cell_scale
        p.stats = stats
        p.max_pairs_per_vertex = max_pairs
        p.wait_budget_cycles = wait_budget_cycles
        p.pcg_kernel = pcg_kernel
        p.debug_flags = debug_flags
        p.pcg_precond = pcg_precond
        if broad_phase is not None:
            p.broad_phase = broad_phase
        p.local_block = local_block
        p.rhs_block = rhs_block
        p.narrow_block = narrow_block
        p.pcg_block = pcg_block
        self.tuned_from = None
        if tuned:
            from . import autotune

            self.tuned_from = autotune.apply_cached(p, self.batch if self.batch is not None else mesh)
        self.params = p
        self.mesh = mesh
        self.h = casim_create(p, stream)
        try:
            if self.batch is None:
                casim_upload_mesh(self.h, mesh.rest, mesh.tets, mesh.group, mesh.fixed)
                alpha = mesh.alpha
            else:
                casim_upload_batch(self.h, [(b.rest, b.tets, b.group, b.fixed) for b in self.batch])
                alpha = np.concatenate([b.alpha for b in self.batch])
            if len(alpha):
                casim_set_actuation(self.h, alpha)
            if mesh.spheres is not None and len(mesh.spheres):
                casim_set_spheres(self.h, mesh.spheres)
            if getattr(mesh, "obstacle_X", None) is not None:
                casim_set_obstacle_mesh(self.h, mesh.obstacle_X, mesh.obstacle_tets)
        except Exception:
            casim_destroy(self.h)
            self.h = None
            raise
        self.sizes = casim_get_sizes(self.h)
        self.n_groups = int(len(alpha))

    def step(self, n: int):
        casim_step(self.h, n)

    def step_anderson(self, n: int, m: int):
        return casim_step_anderson(self.h, n, m)

    def remesh_flags(self, ref=None, alpha_max=4.0, d_max=4.0):
        return casim_remesh_flags(self.h, self.sizes["n_tets"], self.n_groups, ref, alpha_max, d_max)

    def progressive(self, alpha_target, alpha_step, n_inner, max_outer=64, alpha_max=4.0, d_max=4.0):
        return casim_progressive(self.h, alpha_target, alpha_step, n_inner, max_outer, alpha_max, d_max)

    def reset(self):
        casim_reset(self.h)

    def sync(self) -> int:
        return casim_sync(self.h)

    def positions(self) -> np.ndarray:
        return casim_get_positions(self.h, self.sizes["n_verts"])

    def set_positions(self, X):
        casim_set_positions(self.h, X)

    def contacts(self):
        return casim_get_contacts(self.h)

    def springs(self):
        return casim_get_springs(self.h, self.sizes["n_query_verts"])

    def set_springs(self, verts, active, kind, face, bary, target):
        casim_set_springs(self.h, verts, active, kind, face, bary, target)

    def targets(self) -> np.ndarray:
        return casim_get_targets(self.h, self.sizes["n_tets"])

    def history(self, cap=4096):
        return casim_get_history(self.h, cap)

    def stats(self):
        return casim_get_stats(self.h)

    def close(self):
        if self.h is not None:
            casim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def actuation_to_positions(sim: "Sim", alpha, n_iters: int, ckpt_every: int = 10):
    """Differentiable map alpha -> final positions (torch tensors, CPU, float64)
    through ``casim_forward_ckpt`` / ``casim_backward``: every forward call
    resets the simulation to its rest state, sets the ratios and runs
    ``n_iters`` iterations with checkpoints; the backward pass returns
    dL/dalpha from the library's adjoint."""
    import torch

    class _ActuationToPositions(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a):
            an = a.detach().cpu().double().numpy()
            casim_set_actuation(sim.h, an)
            casim_reset(sim.h)
            casim_forward_ckpt(sim.h, n_iters, ckpt_every)
            casim_sync(sim.h)
            return torch.from_numpy(sim.positions())

        @staticmethod
        def backward(ctx, gX):
            ga = casim_backward(sim.h, gX.detach().cpu().double().numpy(), sim.n_groups)
            return torch.from_numpy(ga)

    return _ActuationToPositions.apply(alpha)
