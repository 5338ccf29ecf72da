"""Seeded synthetic soft-robot inputs (voxel Kuhn tetrahedral meshes).

This module only builds inputs: rest vertex positions, tetrahedra, chamber
group ids, fixed-vertex masks, actuation ratios, spheres, loss targets and
perturbed replay states.  It holds none of the simulation arithmetic (no
targets, rotations, collision tests or solves), so both the CUDA library and
the FP64 oracle can consume it without sharing any method code.

The paper's meshes (twisting robot, soft finger, membrane; Sec. IV) are not
available, so pneumatic fingers built from voxels stand in for them:

* voxel edge ``h`` (0.5 cm, exact in binary); vertex id ``i + (nx+1)(j + (ny+1)k)``;
* every voxel is split into 6 Kuhn tetrahedra around its (0,0,0)-(1,1,1)
  diagonal, one per axis permutation in lexicographic order, with tet id
  ``6 * voxel + perm`` and positive orientation;
* a finger has a spine (voxel z < s), ``n_ch`` chamber boxes above it whose
  voxels are chamber elements (the chamber region is tetrahedralised too,
  Sec. II-A), 2-voxel gaps between chambers, and a zero-width slit on the
  mid-plane of each gap above the spine (duplicated vertices), so that the
  "teeth" of the pneu-net touch at rest and collide when the chambers inflate;
* vertices on the x = 0 plane are fixed.

Random draws use SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) with ``u = (next >> 11) * 2^-53``
and Box-Muller for normal deviates.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MASK64 = (1 << 64) - 1

# Kuhn split: one tetrahedron per permutation of the three axes, in
# lexicographic order of the permutation.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_PERM_EVEN = [True, False, False, True, True, False]

# Body-element stiffness table w(eps): piecewise linear knots, clamped.  The
# paper defines R_omega only by reference to another publication, so this
# "soft" preset is this library's reading (see the design notes).
SOFT_W_KNOTS = ((0.0, 0.6), (0.5, 0.9), (1.0, 1.0))

PRECISION_FP64 = 0
PRECISION_MIXED = 1

COLLISION_OFF = 0
COLLISION_SELF = 1
COLLISION_SELF_OBSTACLE = 2


class SplitMix64:
    """SplitMix64 generator (Steele et al. 2014) with a 64-bit state."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (2.0 ** -53)
        return a + (b - a) * u

    def randint(self, a: int, b: int) -> int:
        """Uniform integer in [a, b] inclusive."""
        u = (self.next_u64() >> 11) * (2.0 ** -53)
        return a + min(int(u * (b - a + 1)), b - a)

    def normal(self) -> float:
        """One standard normal deviate by Box-Muller (cosine branch)."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 2.0 ** -53)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclass
class Mesh:
    """One tetrahedral soft-robot mesh plus its actuation and solver settings."""

    name: str
    rest: np.ndarray          # (n_v, 3) float64, cm
    tets: np.ndarray          # (n_t, 4) int32, positively oriented
    group: np.ndarray         # (n_t,) int32: -1 body, g >= 0 chamber group g
    fixed: np.ndarray         # (n_v,) uint8
    alpha: np.ndarray         # (n_groups,) float64 volume ratios
    h: float = 0.5
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))
    n_iters: int = 50
    precision: int = PRECISION_MIXED
    collision: int = COLLISION_SELF
    k_spring: float = 1.0
    w_knots: tuple = SOFT_W_KNOTS
    tip_verts: Optional[np.ndarray] = None     # (m,) int32 loss vertices
    tip_targets: Optional[np.ndarray] = None   # (m, 3) float64
    obstacle_X: Optional[np.ndarray] = None    # (n_o, 3) rigid tetrahedral obstacle positions
    obstacle_tets: Optional[np.ndarray] = None # (m_o, 4) int32, positively oriented

    @property
    def n_verts(self) -> int:
        return int(self.rest.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.alpha.shape[0])

    @property
    def eps(self) -> float:
        return self.h / 100.0

    @property
    def cell_size(self) -> float:
        return self.h

    @property
    def pcg_tol(self) -> float:
        return 1e-12 if self.precision == PRECISION_FP64 else 1e-6

    def bbox_diag(self) -> float:
        lo = self.rest.min(axis=0)
        hi = self.rest.max(axis=0)
        return float(np.linalg.norm(hi - lo))


def _voxel_kuhn(nx, ny, nz, h, slit_levels=(), s=0, group_of_voxel=None):
    """Voxel block split into Kuhn tets, with optional zero-width slits.

    ``slit_levels`` are vertex x-levels P at which voxels with i >= P use
    duplicated copies of the plane vertices above vertex level ``s``.
    Returns rest (n_v,3), tets (n_t,4), group (n_t,), fixed (n_v,).
    """
    nvx, nvy, nvz = nx + 1, ny + 1, nz + 1
    n_base = nvx * nvy * nvz
    K, J, I = np.meshgrid(np.arange(nvz), np.arange(nvy), np.arange(nvx), indexing="ij")
    base_xyz = np.stack([I.ravel() * h, J.ravel() * h, K.ravel() * h], axis=1).astype(np.float64)

    slit_levels = list(slit_levels)
    n_lev = nz - s
    dup_rows = []
    for P in slit_levels:
        for kk in range(s + 1, nz + 1):
            for jj in range(ny + 1):
                dup_rows.append(P + nvx * (jj + nvy * kk))
    rest = np.concatenate([base_xyz, base_xyz[np.array(dup_rows, dtype=np.int64)]], axis=0) \
        if dup_rows else base_xyz

    slit_index = {P: q for q, P in enumerate(slit_levels)}
    # voxel grid in (k, j, i) order, i fastest: voxel index i + nx (j + ny k)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    if group_of_voxel is None:
        gvox = np.full(ii.shape[0], -1, dtype=np.int32)
    else:
        gvox = np.array([group_of_voxel(a, b, c) for a, b, c in zip(ii.tolist(), jj.tolist(), kk.tolist())],
                        dtype=np.int32)

    def vid(I_, J_, K_):
        """Vertex ids of corner levels (I_, J_, K_) for voxels with x index ii."""
        out = I_ + nvx * (J_ + nvy * K_)
        for P, q in slit_index.items():
            sel = (I_ == P) & (ii == P) & (K_ > s)
            out = np.where(sel, n_base + q * n_lev * nvy + (K_ - s - 1) * nvy + J_, out)
        return out

    tets = np.empty((nx * ny * nz, 6, 4), dtype=np.int64)
    for p, (a, b, _c) in enumerate(_PERMS):
        c1 = [0, 0, 0]
        c1[a] = 1
        c2 = list(c1)
        c2[b] = 1
        corners = [(0, 0, 0), tuple(c1), tuple(c2), (1, 1, 1)]
        ids = [vid(ii + dd[0], jj + dd[1], kk + dd[2]) for dd in corners]
        if not _PERM_EVEN[p]:
            ids[1], ids[2] = ids[2], ids[1]
        tets[:, p, :] = np.stack(ids, axis=1)
    tets = tets.reshape(-1, 4).astype(np.int32)
    group = np.repeat(gvox, 6).astype(np.int32)
    fixed = np.zeros(rest.shape[0], dtype=np.uint8)
    fixed[np.isclose(rest[:, 0], 0.0) & (np.arange(rest.shape[0]) < n_base)] = 1
    return rest, tets, group, fixed


def finger_layout(nx, ny, nz, n_ch):
    """Chamber boxes and slit planes of the finger family (integers only)."""
    s = nz // 4
    w = max(1, ny // 6)
    t = max(1, nz // 12)
    c0 = max(1, ny // 4)
    gap = 2
    L = (nx - 2 * c0 - gap * (n_ch - 1)) // n_ch
    if L < 1:
        raise ValueError("finger too short for %d chambers" % n_ch)
    starts = [c0 + c * (L + gap) for c in range(n_ch)]
    slits = [starts[c] + L + 1 for c in range(n_ch - 1)]
    return dict(s=s, w=w, t=t, c0=c0, L=L, starts=starts, slits=slits)


def max_chambers(nx, ny, nz):
    n = 1
    while True:
        c0 = max(1, ny // 4)
        L = (nx - 2 * c0 - 2 * n) // (n + 1)
        if L < 1:
            return n
        n += 1


def finger_mesh(nx, ny, nz, n_ch, h=0.5, group_base=0):
    lay = finger_layout(nx, ny, nz, n_ch)
    s, w, t, L = lay["s"], lay["w"], lay["t"], lay["L"]

    def gov(i, j, k):
        if not (w <= j < ny - w and s <= k < nz - t):
            return -1
        for c, x0 in enumerate(lay["starts"]):
            if x0 <= i < x0 + L:
                return group_base + c
        return -1

    return _voxel_kuhn(nx, ny, nz, h, slit_levels=lay["slits"], s=s, group_of_voxel=gov)


def config1_beam() -> Mesh:
    """Cantilever beam 20x4x4 voxels; top voxel layer is chamber group 0 with
    volume ratio 1.3; x = 0 fixed; FP64, no collision, 50 iterations."""
    nx, ny, nz = 20, 4, 4
    rest, tets, group, fixed = _voxel_kuhn(
        nx, ny, nz, 0.5, group_of_voxel=lambda i, j, k: 0 if k == nz - 1 else -1)
    return Mesh("beam_20x4x4", rest, tets, group, fixed, np.array([1.3]),
                n_iters=50, precision=PRECISION_FP64, collision=COLLISION_OFF)


def config2_finger(nx=60, ny=12, nz=12, n_ch=8, seed=1002, lo=1.5, hi=2.5, n_iters=100) -> Mesh:
    """Pneumatic bending finger (60x12x12, 8 chambers, ~52k tets), ratios U(1.5,2.5)."""
    rng = SplitMix64(seed)
    rest, tets, group, fixed = finger_mesh(nx, ny, nz, n_ch)
    alpha = np.array([rng.uniform(lo, hi) for _ in range(n_ch)])
    return Mesh("finger_%dx%dx%d_c%d" % (nx, ny, nz, n_ch), rest, tets, group, fixed, alpha,
                n_iters=n_iters, precision=PRECISION_MIXED, collision=COLLISION_SELF)


def _place_finger(rest, nx, ny, nz, h, theta, radius, root_z):
    """Map finger-local (x along length, y width, z toward chambers) to world:
    x -> -Z (hanging below the plate), z -> radially outward at angle theta,
    y -> tangential.  The map is a proper rotation plus a translation."""
    er = np.array([math.cos(theta), math.sin(theta), 0.0])
    et = np.array([-math.sin(theta), math.cos(theta), 0.0])
    ez = np.array([0.0, 0.0, 1.0])
    lx, ly, lz = rest[:, 0], rest[:, 1], rest[:, 2]
    return ((radius + (lz - nz * h / 2))[:, None] * er[None, :]
            + (ly - ny * h / 2)[:, None] * et[None, :]
            + (root_z - lx)[:, None] * ez[None, :])


def config3_gripper(seed=1003, n_iters=200) -> Mesh:
    """Three 60x12x12 fingers at 0/120/240 degrees (centre-line radius 8 cm)
    hanging 0.25 cm below a 40x40x4-voxel plate whose top is fixed, plus a
    rigid sphere of radius 3 cm in one finger's closing path; 24 chamber
    ratios U(1.2,2.5); ~194k tets.  Draw order: ratios, object finger,
    radial offset, depth."""
    rng = SplitMix64(seed)
    nx, ny, nz, n_ch, h = 60, 12, 12, 8, 0.5
    alpha = np.array([rng.uniform(1.2, 2.5) for _ in range(3 * n_ch)])
    # The sphere (the grasped object) sits in the closing path of a seeded
    # finger f near the fingertips: centre at radius rho toward finger f, so
    # that the sphere's surface lies within 0.25 cm inside that finger's inner
    # face (radius 5 cm at rest; not touching), at depth 28-31 cm below the
    # plate (the tips hang at 30.25 cm).  The finger curls onto it within the
    # first tens of iterations.
    f_obj = rng.randint(0, 2)
    rho = 2.0 - rng.uniform(0.0, 0.25)
    depth = rng.uniform(28.0, 31.0)
    th = 2.0 * math.pi * f_obj / 3.0
    sphere = np.array([[rho * math.cos(th), rho * math.sin(th), -depth, 3.0]])
    rests, tetss, groups, fixeds = [], [], [], []
    off = 0
    for f in range(3):
        r, t, g, fx = finger_mesh(nx, ny, nz, n_ch, h, group_base=f * n_ch)
        rests.append(_place_finger(r, nx, ny, nz, h, 2.0 * math.pi * f / 3.0, 8.0, -0.25))
        tetss.append(t + off)
        groups.append(g)
        fixeds.append(fx)
        off += r.shape[0]
    pr, pt, pg, _ = _voxel_kuhn(40, 40, 4, h)
    pr = pr + np.array([-10.0, -10.0, 0.0])
    pf = np.zeros(pr.shape[0], dtype=np.uint8)
    pf[np.isclose(pr[:, 2], 2.0)] = 1
    rests.append(pr)
    tetss.append(pt + off)
    groups.append(pg)
    fixeds.append(pf)
    return Mesh("gripper3_plate_sphere", np.concatenate(rests), np.concatenate(tetss).astype(np.int32),
                np.concatenate(groups).astype(np.int32), np.concatenate(fixeds), alpha,
                spheres=sphere, n_iters=n_iters, precision=PRECISION_MIXED,
                collision=COLLISION_SELF_OBSTACLE)


def config4_batch(n_robots=256, seed=1004, n_iters=100) -> List[Mesh]:
    """Batch of independent fingers: scale k ~ U{1..4} -> (20k, 4k, 4k) voxels,
    chambers U{4..10} clipped to the largest count with chamber length >= 1,
    ratios U(1.2,2.5).  Draw order per robot: k, n_ch, then its ratios."""
    rng = SplitMix64(seed)
    out = []
    for r in range(n_robots):
        k = rng.randint(1, 4)
        n_ch = rng.randint(4, 10)
        nx, ny, nz = 20 * k, 4 * k, 4 * k
        n_ch = min(n_ch, max_chambers(nx, ny, nz))
        alpha = np.array([rng.uniform(1.2, 2.5) for _ in range(n_ch)])
        rest, tets, group, fixed = finger_mesh(nx, ny, nz, n_ch)
        out.append(Mesh("batch%03d_finger_%dx%dx%d_c%d" % (r, nx, ny, nz, n_ch), rest, tets, group,
                        fixed, alpha, n_iters=n_iters, precision=PRECISION_MIXED,
                        collision=COLLISION_SELF))
    return out


def config5_adjoint(nx=160, ny=32, nz=32, n_ch=16, seed=1005, n_iters=100) -> Mesh:
    """Adjoint workload: finger (160x32x32, 16 chambers), ratios U(1.2,2.5);
    loss vertices = the tip-face (x = nx) vertex sub-grid with stride ny/8
    (64 vertices at 32x32), each with target rest + N(0, 1 cm^2) per axis."""
    rng = SplitMix64(seed)
    rest, tets, group, fixed = finger_mesh(nx, ny, nz, n_ch)
    alpha = np.array([rng.uniform(1.2, 2.5) for _ in range(n_ch)])
    stride = max(1, ny // 8)
    nvx, nvy = nx + 1, ny + 1
    tips = [nx + nvx * (jj + nvy * kk)
            for kk in range(0, nz, stride) for jj in range(0, ny, stride)]
    tips = np.array(tips[:64], dtype=np.int32)
    targets = rest[tips] + np.array([[rng.normal() for _ in range(3)] for _ in range(len(tips))])
    return Mesh("adjoint_finger_%dx%dx%d_c%d" % (nx, ny, nz, n_ch), rest, tets, group, fixed, alpha,
                n_iters=n_iters, precision=PRECISION_MIXED, collision=COLLISION_SELF,
                tip_verts=tips, tip_targets=targets)


def small_finger(nx=20, ny=4, nz=4, n_ch=4, seed=7, lo=1.5, hi=2.5, n_iters=30,
                 precision=PRECISION_MIXED, collision=COLLISION_SELF) -> Mesh:
    """A small member of the finger family for tests that the oracle finishes
    in seconds (several thread blocks plus a ragged tail)."""
    m = config2_finger(nx, ny, nz, n_ch, seed=seed, lo=lo, hi=hi, n_iters=n_iters)
    m.precision = precision
    m.collision = collision
    return m


def box_obstacle(nx, ny, nz, h, origin, dtype=np.float64):
    """A rigid box obstacle: an nx x ny x nz block of voxels of edge h, split
    into Kuhn tets, translated to ``origin``; optionally rounded to float32 so
    that a MIXED-precision consumer sees the identical coordinates."""
    rest, tets, _g, _f = _voxel_kuhn(nx, ny, nz, h)
    X = rest + np.asarray(origin, dtype=np.float64)[None, :]
    if dtype == np.float32:
        X = X.astype(np.float32).astype(np.float64)
    return X, tets


def perturbed_positions(mesh: Mesh, amplitude: float, seed: int, dtype=np.float64) -> np.ndarray:
    """Replay state: rest + seeded uniform noise of +-amplitude*h per axis on
    free vertices (fixed vertices stay at rest).  Optionally rounded to
    float32 so that a MIXED-precision consumer sees the identical values."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.uniform(-1.0, 1.0, size=mesh.rest.shape) * amplitude * mesh.h
    d[mesh.fixed.astype(bool)] = 0.0
    x = mesh.rest + d
    if dtype == np.float32:
        x = x.astype(np.float32).astype(np.float64)
    return x


CONFIGS = {
    "beam": config1_beam,
    "finger": config2_finger,
    "gripper": config3_gripper,
    "adjoint": config5_adjoint,
}
