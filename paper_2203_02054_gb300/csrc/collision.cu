// Collision check (Sec. II-B, Eq. 3, Eq. 4) and spring update (Sec. II-C,
// Eq. 5, Sec. III-A.3) kernels.
//
// Broad phase: one spatial hash over tets and one over boundary faces, rebuilt
// every iteration from the current positions (counting sort: count, scan,
// fill).  A point strictly inside a tet lies in the tet's closed bounding box,
// whose cell range covers the point's cell, so the hash never drops a pair;
// hash collisions only add candidates.
//
// Narrow phase: one warp per non-fixed boundary vertex tests the tets of its
// cell with exact orientation signs (predicates.cuh), so the pair set equals
// the brute-force definition bit for bit.
//
// Spring update: one thread per non-fixed boundary vertex for obstacle
// targets (closed form) and the paper's release condition; self-collision
// targets by a ray cast along -n(v) (3D-DDA cell walk of Amanatides and Woo
// 1987 over the face hash, Moller-Trumbore 1997 ray-triangle test), one warp
// per casting vertex.  All spring geometry is evaluated in FP64.
#include <algorithm>

#include "bvh.cuh"
#include "common.cuh"
#include "kernels.h"
#include "predicates.cuh"

namespace casim {

static constexpr int MAX_CELLS_PER_ITEM = 4096;
static constexpr int MAX_DDA_STEPS = 4096;

template <typename T>
__device__ __forceinline__ void load3(const R4<T>* X, int v, double& x, double& y, double& z) {
  const R4<T> a = X[v];
  x = (double)a.x;
  y = (double)a.y;
  z = (double)a.z;
}

// Bounding box of item i: tets are items [0, n_t), boundary faces [n_t, n_t + n_f),
// in the positions' own precision.
template <typename T>
__device__ __forceinline__ bool item_box_t(const Dev<T>& d, int i, T lo[3], T hi[3]) {
  int vs[4];
  int nv;
  if (i < d.n_t) {
    const int4 t = chk_idx4(d.ctrl, d.tet[i], d.n_v);
    vs[0] = t.x; vs[1] = t.y; vs[2] = t.z; vs[3] = t.w;
    nv = 4;
  } else {
    const int4 f = chk_face(d.ctrl, d.faces[i - d.n_t], d.n_v);
    vs[0] = f.x; vs[1] = f.y; vs[2] = f.z;
    nv = 3;
  }
  // min/max in the positions' own precision, converted once (exact)
  const R4<T> a0 = d.X[vs[0]];
  T l[3] = {a0.x, a0.y, a0.z}, h[3] = {a0.x, a0.y, a0.z};
  bool ok = isfinite(a0.x) && isfinite(a0.y) && isfinite(a0.z);
  for (int k = 1; k < nv; ++k) {
    const R4<T> a = d.X[vs[k]];
    const T c[3] = {a.x, a.y, a.z};
    for (int j = 0; j < 3; ++j) {
      ok = ok && isfinite(c[j]);
      l[j] = fmin(l[j], c[j]);
      h[j] = fmax(h[j], c[j]);
    }
  }
  for (int j = 0; j < 3; ++j) {
    lo[j] = l[j];
    hi[j] = h[j];
  }
  return ok;
}

// Cell coordinate in FP32 for FP32 positions, used for the tets and for the
// narrow phase's point lookups only: it is monotone in x, so the cells of a
// tet's box corners bound the cell of every point in the box, the property
// the point-in-tet search needs.  The boundary faces keep FP64 cells
// (cell_coord), the model of the ray walk and of the shell search.
__device__ __forceinline__ int cell_coord_f(float x, float inv_cell) {
  float c = floorf(x * inv_cell);
  c = fminf(fmaxf(c, -1.0e6f), 1.0e6f);
  return (int)c;
}

// Block-reduced bounding box of the valid item boxes (count pass only).
// Warps without a valid item skip the shuffles, and blocks without one skip
// the atomics (only the boundary faces' blocks contribute).
__device__ __forceinline__ void reduce_box(Ctrl* c, bool valid, const double lo[3], const double hi[3]) {
  __shared__ long long s_lo[3][8], s_hi[3][8];
  constexpr long long kLo = 0x7FFFFFFFFFFFFFFFLL, kHi = (long long)0x8000000000000000ULL;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool any = __any_sync(0xffffffffu, valid);
  for (int j = 0; j < 3; ++j) {
    long long a = kLo, b = kHi;
    if (any) {
      a = valid ? order_code(lo[j]) : kLo;
      b = valid ? order_code(hi[j]) : kHi;
      for (int o = 16; o > 0; o >>= 1) {
        a = min(a, __shfl_down_sync(0xffffffffu, a, o));
        b = max(b, __shfl_down_sync(0xffffffffu, b, o));
      }
    }
    if (lane == 0) {
      s_lo[j][wid] = a;
      s_hi[j][wid] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int j = threadIdx.x;
    long long a = s_lo[j][0], b = s_hi[j][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      a = min(a, s_lo[j][w]);
      b = max(b, s_hi[j][w]);
    }
    if (a != kLo) atomicMin(&c->box_lo[j], a);
    if (b != kHi) atomicMax(&c->box_hi[j], b);
  }
}

template <typename T, bool FILL>
__global__ void __launch_bounds__(256) k_grid_bin(Dev<T> d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = d.n_t + d.n_f;
  T lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  const bool ok = i < n && item_box_t(d, i, lo, hi);
  if (!FILL) {
    // the box of the boundary faces bounds the ray walks (no face lies beyond it)
    const bool face = ok && i >= d.n_t;
    double lod[3] = {0.0, 0.0, 0.0}, hid[3] = {0.0, 0.0, 0.0};
    if (face)
      for (int j = 0; j < 3; ++j) {
        lod[j] = (double)lo[j];
        hid[j] = (double)hi[j];
      }
    reduce_box(d.ctrl, face, lod, hid);
  }
  if (i >= n) return;
  if (!ok) {
    if (!FILL) set_status(d.ctrl, ST_NONFINITE);
    return;
  }
  int c0[3], c1[3];
  const bool is_tet = i < d.n_t;
  if (std::is_same<T, float>::value && is_tet) {
    const float inv_f = (float)d.inv_cell;
    for (int j = 0; j < 3; ++j) {
      c0[j] = cell_coord_f((float)lo[j], inv_f);
      c1[j] = cell_coord_f((float)hi[j], inv_f);
    }
  } else {
    for (int j = 0; j < 3; ++j) {
      c0[j] = cell_coord((double)lo[j], d.inv_cell);
      c1[j] = cell_coord((double)hi[j], d.inv_cell);
    }
  }
  const long long ncell =
      (long long)(c1[0] - c0[0] + 1) * (c1[1] - c0[1] + 1) * (c1[2] - c0[2] + 1);
  if (ncell > MAX_CELLS_PER_ITEM) {
    if (!FILL) set_status(d.ctrl, ST_OVERFLOW);
    return;
  }
  const unsigned base = is_tet ? 0u : d.H_t;
  const unsigned mask = (is_tet ? d.H_t : d.H_f) - 1u;
  const int robot = is_tet ? (d.robot_of_tet ? d.robot_of_tet[i] : 0) : (d.robot_of_face ? d.robot_of_face[i - d.n_t] : 0);
  for (int cz = c0[2]; cz <= c1[2]; ++cz)
    for (int cy = c0[1]; cy <= c1[1]; ++cy)
      for (int cx = c0[0]; cx <= c1[0]; ++cx) {
        const unsigned h = base + (hash_cell(cx, cy, cz, robot) & mask);
        if (!FILL) {
          atomicAdd(&d.cell_count[h], 1);
        } else {
          const int pos = d.cell_start[h] + atomicAdd(&d.cell_cursor[h], 1);
          if (pos < d.cap_items) d.items[pos] = i;
        }
      }
}

// ---- exclusive scan of cell_count into cell_start (three small kernels) ----
static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_PER_THREAD = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__global__ void k_scan_tiles(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ tile_sums,
                             int n) {
  __shared__ int sh[SCAN_THREADS];
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_PER_THREAD;
  int v[SCAN_PER_THREAD];
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {
    int t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - s;  // exclusive prefix of this thread
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = sh[threadIdx.x];
}

// Single block: exclusive scan of the tile sums in place, total into *total.
__global__ void k_scan_top(int* tile_sums, int n_tiles, int* total_out, Ctrl* ctrl, int cap) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n_tiles; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = (i < n_tiles) ? tile_sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n_tiles) tile_sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total_out = carry;
    if (ctrl) {
      ctrl->n_items = carry;
      if (carry > cap) atomicOr(&ctrl->status, ST_OVERFLOW);
    }
  }
}

__global__ void k_scan_add(int* out, const int* tile_sums, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_sums[i / SCAN_TILE];
}

// ---- single-pass exclusive scan with decoupled look-back -----------------
// (Merrill and Garland 2016).  Each block takes a tile ticket (so every
// smaller tile belongs to a block that is already running), scans its tile,
// publishes the tile's sum as a status word (flag 1: the tile's own sum,
// flag 2: the inclusive prefix up to and including the tile), and warp 0
// walks back over the predecessors' words, 32 at a time, adding own sums
// until it meets an inclusive prefix.  Waits for a predecessor's word are
// bounded by the clock budget (then ST_TIMEOUT).  Integer sums, so the result
// is the same as any other scan order.  The status words and the ticket are
// zeroed with the count array before each use; the last tile resets nothing
// and writes the total (with the capacity check).
__device__ __forceinline__ unsigned long long scan_word(unsigned flag, int v) {
  return ((unsigned long long)flag << 62) | (unsigned)v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_lookback(const int* __restrict__ in, int* __restrict__ out, int n,
                                                                unsigned long long* status, unsigned* ticket,
                                                                int* total_out, Ctrl* ctrl, int cap,
                                                                unsigned long long budget) {
  __shared__ int sh[SCAN_THREADS];
  __shared__ int s_tile, s_prefix;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  const int tile = s_tile;
  const int base = tile * SCAN_TILE + threadIdx.x * SCAN_PER_THREAD;
  int v[SCAN_PER_THREAD];
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {
    const int t = (threadIdx.x >= off) ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  const int agg = sh[SCAN_THREADS - 1];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int prefix = 0;
    if (tile == 0) {
      if (lane == 0) st_relaxed_u64(status + tile, scan_word(2u, agg));
    } else {
      if (lane == 0) st_relaxed_u64(status + tile, scan_word(1u, agg));
      long long t0 = 0;
      unsigned polls = 0;
      bool failed = false;
      for (int j = tile - 1; j >= 0 && !failed; j -= 32) {
        const int q = j - lane;  // predecessor this lane reads (nearest first)
        unsigned long long w = q >= 0 ? ld_relaxed_u64(status + q) : scan_word(1u, 0);
        // wait until every word of the window is published
        while (__any_sync(0xffffffffu, (w >> 62) == 0ull)) {
          if ((++polls & 31u) == 0) {
            const long long now = clock64();
            if (t0 == 0) t0 = now;
            else if ((unsigned long long)(now - t0) > budget) {
              failed = true;
              break;
            }
          }
          if ((w >> 62) == 0ull) w = ld_relaxed_u64(status + q);
        }
        if (failed) break;
        const unsigned incl = __ballot_sync(0xffffffffu, (w >> 62) == 2ull);
        const int stop = incl ? __ffs(incl) - 1 : 32;  // nearest inclusive prefix in the window
        int part = (lane <= stop && q >= 0) ? (int)(unsigned)(w & 0xFFFFFFFFull) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        prefix += __shfl_sync(0xffffffffu, part, 0);
        if (incl) break;
      }
      if (failed && lane == 0) atomicOr(&ctrl->status, ST_TIMEOUT);
      if (lane == 0) st_relaxed_u64(status + tile, scan_word(2u, prefix + agg));
    }
    if (lane == 0) s_prefix = prefix;
  }
  __syncthreads();
  int run = s_prefix + sh[threadIdx.x] - s;  // exclusive prefix of this thread
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) {
    const int tot = s_prefix + agg;
    *total_out = tot;
    if (ctrl) {
      ctrl->n_items = tot;
      if (tot > cap) atomicOr(&ctrl->status, ST_OVERFLOW);
    }
  }
}

int scan_lookback_extra_ints(int n) { return 2 + 2 * (scan_tiles(n) + 1) + 2; }

// ---- narrow phase ----
__device__ __forceinline__ int orient_t(float ax, float ay, float az, float bx, float by, float bz, float cx, float cy,
                                        float cz, float dx, float dy, float dz) {
  return orient_sign_f(ax, ay, az, bx, by, bz, cx, cy, cz, dx, dy, dz);
}
__device__ __forceinline__ int orient_t(double ax, double ay, double az, double bx, double by, double bz, double cx,
                                        double cy, double cz, double dx, double dy, double dz) {
  return orient_sign(ax, ay, az, bx, by, bz, cx, cy, cz, dx, dy, dz);
}

template <typename T>
__device__ __forceinline__ T min4(T a, T b, T c, T e) {
  return fmin(fmin(a, b), fmin(c, e));
}
template <typename T>
__device__ __forceinline__ T max4(T a, T b, T c, T e) {
  return fmax(fmax(a, b), fmax(c, e));
}

// p strictly inside tet t, evaluated in the positions' own precision (the
// box reject compares exactly; the orientation signs are exact).
template <typename T>
__device__ __forceinline__ bool strictly_inside_at(const R4<T>* X, T px, T py, T pz, int4 t) {
  const R4<T> a = X[t.x], b = X[t.y], c = X[t.z], e = X[t.w];
  // A point strictly inside a tet lies strictly inside its box: the tet
  // reaches its extreme coordinates only on its boundary.  The open box test
  // is exact and rejects the many points on a box face (vertices of
  // axis-aligned meshes), whose orientation signs would be exact zeros.
  if (!(px > min4(a.x, b.x, c.x, e.x) && px < max4(a.x, b.x, c.x, e.x))) return false;
  if (!(py > min4(a.y, b.y, c.y, e.y) && py < max4(a.y, b.y, c.y, e.y))) return false;
  if (!(pz > min4(a.z, b.z, c.z, e.z) && pz < max4(a.z, b.z, c.z, e.z))) return false;
  // p strictly inside iff each sub-tet with one vertex replaced by p is
  // positive; for FP32 positions every sign first gets the FP32 filter, so a
  // certified negative sign ends the test before any FP64 or exact work
  if constexpr (std::is_same<T, float>::value) {
    const int s0 = orient_filter_f(px, py, pz, b.x, b.y, b.z, c.x, c.y, c.z, e.x, e.y, e.z);
    const int s1 = orient_filter_f(a.x, a.y, a.z, px, py, pz, c.x, c.y, c.z, e.x, e.y, e.z);
    const int s2 = orient_filter_f(a.x, a.y, a.z, b.x, b.y, b.z, px, py, pz, e.x, e.y, e.z);
    const int s3 = orient_filter_f(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, px, py, pz);
    if (s0 < 0 || s1 < 0 || s2 < 0 || s3 < 0) return false;
  }
  if (orient_t(px, py, pz, b.x, b.y, b.z, c.x, c.y, c.z, e.x, e.y, e.z) <= 0) return false;
  if (orient_t(a.x, a.y, a.z, px, py, pz, c.x, c.y, c.z, e.x, e.y, e.z) <= 0) return false;
  if (orient_t(a.x, a.y, a.z, b.x, b.y, b.z, px, py, pz, e.x, e.y, e.z) <= 0) return false;
  if (orient_t(a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, px, py, pz) <= 0) return false;
  return true;
}
template <typename T>
__device__ __forceinline__ bool strictly_inside(const Dev<T>& d, T px, T py, T pz, int4 t) {
  return strictly_inside_at(d.X, px, py, pz, t);
}

// Obstacle tests of one query point (Eq. 4): the sphere whose signed surface
// distance |x - c_j| - r_j is smallest among those strictly containing it
// (ties: lowest j), how many spheres contain it, and how many tetrahedra of
// the rigid tetrahedral obstacle strictly contain it (exact signs, AABB tree
// of the obstacle).  Spheres use the fixed FP64 evaluation order.
template <typename T>
__device__ __forceinline__ void obstacle_tests(const Dev<T>& d, T px, T py, T pz, int& best, int& n_sph,
                                               int& n_mesh) {
  best = -1;
  n_sph = 0;
  n_mesh = 0;
  if (d.collision < 2) return;
  double bestd = 0.0;
  for (int j = 0; j < d.n_spheres; ++j) {
    // FP32 reject first: a point farther than r from the centre along one axis
    // is outside; the margins (1e-5 relative to the magnitudes involved) cover
    // the FP32 rounding of the centre, the radius and the difference, so only
    // points near the sphere reach the FP64 test (on this part an FP64
    // instruction costs about as much in one lane as in thirty-two)
    {
      const float rf = d.spheres_f[4 * j + 3];
      const float cf[3] = {d.spheres_f[4 * j], d.spheres_f[4 * j + 1], d.spheres_f[4 * j + 2]};
      const float pf[3] = {(float)px, (float)py, (float)pz};
      bool far = false;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        far |= fabsf(pf[k] - cf[k]) > rf * 1.00001f + 1e-5f * (fabsf(cf[k]) + fabsf(pf[k]));
      if (far) continue;
    }
    const double cx = d.spheres[4 * j], cy = d.spheres[4 * j + 1], cz = d.spheres[4 * j + 2];
    const double r = d.spheres[4 * j + 3];
    const double dx = __dsub_rn((double)px, cx), dy = __dsub_rn((double)py, cy), dz = __dsub_rn((double)pz, cz);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (d2 < __dmul_rn(r, r)) {
      ++n_sph;
      const double dist = sqrt(d2) - r;
      if (best < 0 || dist < bestd) {
        best = j;
        bestd = dist;
      }
    }
  }
  if (d.ot.n > 0)
    bvh_point_query(d.ot, 0, (double)px, (double)py, (double)pz, [&](int e) {
      if (strictly_inside_at(d.OX, px, py, pz, d.ot.prim[e])) ++n_mesh;
    });
}

template <typename T>
__device__ void spring_update_vertex(const Dev<T>& d, int qi, int& active_out, unsigned long long& ssig);

// One warp per query vertex: the lanes test the candidates of the vertex's
// hash bucket in parallel; hits are merged by lane 0 into the vertex's sorted,
// duplicate-free pair list.
// Block totals of one narrow-phase-and-spring-update launch into this
// iteration's record: self pairs, obstacle pairs, finished springs and the
// springs' signature.
template <typename T>
__device__ __forceinline__ void narrow_block_totals(const Dev<T>& d, int n_self, int n_obs, int n_spr,
                                                   unsigned long long ssig, int* shi) {
  if (d.stats) warp_add_u64(ssig, &(d.hist + (d.ctrl->iter % d.hist_cap))->spring_sig);
  const int s1 = block_sum_int(n_self, shi);
  const int s2 = block_sum_int(n_obs, shi);
  const int s3 = block_sum_int(n_spr, shi);
  if (threadIdx.x == 0 && (s1 | s2 | s3)) {
    IterRec* rec = d.hist + (d.ctrl->iter % d.hist_cap);
    if (s1) atomicAdd(&rec->n_self_pairs, s1);
    if (s2) atomicAdd(&rec->n_obstacle_pairs, s2);
    if (s3) atomicAdd(&rec->n_springs, s3);
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(BS) k_narrow(Dev<T> d) {
  __shared__ int shi[32];
  const int lane = threadIdx.x & 31;
  const int qi = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  int n_self = 0, n_obs = 0, n_spr = 0;
  unsigned long long ssig = 0;
  if (qi < d.n_q) {
    const int v = d.q_verts[qi];
    const R4<T> pv = d.X[v];
    const T px = pv.x, py = pv.y, pz = pv.z;
    int cnt = 0;
    bool over = false;
    int* out = d.pair_tet + (size_t)qi * d.max_pairs;
    const int rv = d.robot_of_vert ? d.robot_of_vert[v] : 0;
    if (d.collision >= 1 && isfinite(px) && isfinite(py) && isfinite(pz)) {
      int cp[3];
      if constexpr (std::is_same<T, float>::value) {
        const float inv_f = (float)d.inv_cell;
        cp[0] = cell_coord_f(px, inv_f);
        cp[1] = cell_coord_f(py, inv_f);
        cp[2] = cell_coord_f(pz, inv_f);
      } else {
        cp[0] = cell_coord((double)px, d.inv_cell);
        cp[1] = cell_coord((double)py, d.inv_cell);
        cp[2] = cell_coord((double)pz, d.inv_cell);
      }
      const unsigned h = hash_cell(cp[0], cp[1], cp[2], rv) & (d.H_t - 1u);
      const int b0 = d.cell_start[h];
      const int b1 = min(d.cell_start[h + 1], d.cap_items);
      for (int base = b0; base < b1; base += 32) {
        const int k = base + lane;
        int e = -1;
        bool hit = false;
        if (k < b1) {
          e = chk_idx(d.ctrl, d.items[k], d.n_t);
          const int4 t = chk_idx4(d.ctrl, d.tet[e], d.n_v);
          const bool same_robot = !d.robot_of_tet || d.robot_of_tet[e] == rv;
          if (same_robot && t.x != v && t.y != v && t.z != v && t.w != v) hit = strictly_inside(d, px, py, pz, t);
        }
        unsigned m = __ballot_sync(0xffffffffu, hit);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const int eh = __shfl_sync(0xffffffffu, e, src);
          if (lane == 0) {
            // sorted insert without duplicates (a tet may repeat in a bucket)
            int pos = 0;
            while (pos < cnt && out[pos] < eh) ++pos;
            if (!(pos < cnt && out[pos] == eh)) {
              bool ins = true;
              if (cnt == d.max_pairs) {
                over = true;
                if (pos == cnt) ins = false;
                else --cnt;  // drop the largest to keep the smallest ids
              }
              if (ins) {
                for (int j = cnt; j > pos; --j) out[j] = out[j - 1];
                out[pos] = eh;
                ++cnt;
              }
            }
          }
        }
      }
    }
    if (lane == 0) {
      if (over) set_status(d.ctrl, ST_PAIRS_TRUNC);
      d.pair_count[qi] = cnt;
      n_self = cnt;
      int best, n_sph, n_mesh;
      obstacle_tests(d, px, py, pz, best, n_sph, n_mesh);
      n_obs = n_sph + n_mesh;
      d.obs_sphere[qi] = best;
      if (d.obs_mesh) d.obs_mesh[qi] = n_mesh;
    }
  }
  narrow_block_totals(d, n_self, n_obs, n_spr, ssig, shi);
}

// ---- AABB trees: refit and point queries ----
// Refit after the positions moved (the tree's structure is kept, Sec. II-B):
// one thread per leaf computes its box and climbs; at every internal node the
// first of the two arriving threads stops, the second forms the union of the
// two children's boxes (the sibling's box was written before its arrival,
// fenced) and continues toward the root.
template <typename T>
__global__ void __launch_bounds__(256) k_bvh_refit(BvhDev b, const R4<T>* __restrict__ X) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= b.n) return;
  float4 lo, hi;
  prim_box(b, X, p, lo, hi);
  int me = ~p;
  int node = b.parent[b.n - 1 + p];
  while (node >= 0) {
    __threadfence();
    if (atomicAdd(&b.flag[node], 1) == 0) return;
    __threadfence();
    const int2 c = b.child[node];
    const int other = c.x == me ? c.y : c.x;
    float4 olo, ohi;
    if (other < 0) {
      prim_box(b, X, ~other, olo, ohi);
    } else {
      olo = __ldcg(&b.lo[other]);
      ohi = __ldcg(&b.hi[other]);
    }
    lo = make_float4(fminf(lo.x, olo.x), fminf(lo.y, olo.y), fminf(lo.z, olo.z), 0.0f);
    hi = make_float4(fmaxf(hi.x, ohi.x), fmaxf(hi.y, ohi.y), fmaxf(hi.z, ohi.z), 0.0f);
    __stcg(&b.lo[node], lo);
    __stcg(&b.hi[node], hi);
    me = node;
    node = b.parent[node];
  }
}

// Narrow phase over the robot's AABB tree (broad phase 1): one thread per
// query vertex descends through the boxes containing it and tests the tets
// at the leaves exactly; the pair list is the same sorted, duplicate-free
// list as the hash path's (at most max_pairs, the smallest tet ids).
static constexpr int NARROW_BVH_THREADS = 128;

template <typename T>
__global__ void __launch_bounds__(NARROW_BVH_THREADS) k_narrow_bvh(Dev<T> d) {
  __shared__ int shi[32];
  const int qi = blockIdx.x * blockDim.x + threadIdx.x;
  int n_self = 0, n_obs = 0, n_spr = 0;
  unsigned long long ssig = 0;
  if (qi < d.n_q) {
    const int v = d.q_verts[qi];
    const R4<T> pv = d.X[v];
    const T px = pv.x, py = pv.y, pz = pv.z;
    int cnt = 0;
    bool over = false;
    int* out = d.pair_tet + (size_t)qi * d.max_pairs;
    const int rv = d.robot_of_vert ? d.robot_of_vert[v] : 0;
    if (d.collision >= 1 && isfinite(px) && isfinite(py) && isfinite(pz)) {
      bvh_point_query(d.bt, rv, (double)px, (double)py, (double)pz, [&](int e) {
        const int4 t = chk_idx4(d.ctrl, d.tet[e], d.n_v);
        if (d.robot_of_tet && d.robot_of_tet[e] != rv) return;
        if (t.x == v || t.y == v || t.z == v || t.w == v) return;
        if (!strictly_inside(d, px, py, pz, t)) return;
        int pos = 0;
        while (pos < cnt && out[pos] < e) ++pos;
        if (pos < cnt && out[pos] == e) return;
        if (cnt == d.max_pairs) {
          over = true;
          if (pos == cnt) return;
          --cnt;
        }
        for (int j = cnt; j > pos; --j) out[j] = out[j - 1];
        out[pos] = e;
        ++cnt;
      });
    }
    if (over) set_status(d.ctrl, ST_PAIRS_TRUNC);
    d.pair_count[qi] = cnt;
    n_self = cnt;
    int best, n_sph, n_mesh;
    if (isfinite(px) && isfinite(py) && isfinite(pz)) {
      obstacle_tests(d, px, py, pz, best, n_sph, n_mesh);
    } else {
      best = -1;
      n_sph = n_mesh = 0;
      set_status(d.ctrl, ST_NONFINITE);
    }
    n_obs = n_sph + n_mesh;
    d.obs_sphere[qi] = best;
    if (d.obs_mesh) d.obs_mesh[qi] = n_mesh;
    if (d.sp.active) spring_update_vertex(d, qi, n_spr, ssig);
  }
  narrow_block_totals(d, n_self, n_obs, n_spr, ssig, shi);
}

// ---- spring update ----
struct V3 {
  double x, y, z;
};
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 scl(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(V3 a) { return sqrt(dot(a, a)); }

template <typename T>
__device__ __forceinline__ V3 pos(const Dev<T>& d, int v) {
  const R4<T> a = d.X[v];
  return {(double)a.x, (double)a.y, (double)a.z};
}

// Moller-Trumbore with inclusive barycentrics and t > 0.
__device__ __forceinline__ bool ray_tri(V3 o, V3 dir, V3 q0, V3 q1, V3 q2, double& t, double& b1,
                                        double& b2) {
  const V3 e1 = sub(q1, q0), e2 = sub(q2, q0);
  const V3 pv = cross(dir, e2);
  const double det = dot(e1, pv);
  if (det == 0.0) return false;
  const double inv = 1.0 / det;
  const V3 tv = sub(o, q0);
  b1 = dot(tv, pv) * inv;
  const V3 qv = cross(tv, e1);
  b2 = dot(dir, qv) * inv;
  t = dot(e2, qv) * inv;
  return b1 >= 0.0 && b2 >= 0.0 && b1 + b2 <= 1.0 && t > 0.0;
}

// Closest point of a triangle: plane projection when inside, else the nearest
// edge projection.  Returns the barycentric weights of q1, q2.
__device__ __forceinline__ V3 closest_tri(V3 p, V3 q0, V3 q1, V3 q2, double& b1, double& b2) {
  const V3 e1 = sub(q1, q0), e2 = sub(q2, q0);
  const V3 n = cross(e1, e2);
  const double nn = dot(n, n);
  if (nn > 0.0) {
    const V3 x = sub(p, scl(dot(sub(p, q0), n) / nn, n));
    const double d11 = dot(e1, e1), d12 = dot(e1, e2), d22 = dot(e2, e2);
    const V3 r = sub(x, q0);
    const double r1 = dot(r, e1), r2 = dot(r, e2);
    const double den = d11 * d22 - d12 * d12;
    const double c1 = (d22 * r1 - d12 * r2) / den, c2 = (d11 * r2 - d12 * r1) / den;
    if (c1 >= 0.0 && c2 >= 0.0 && c1 + c2 <= 1.0) {
      b1 = c1;
      b2 = c2;
      return x;
    }
  }
  double bestd = 0.0;
  V3 best = q0;
  const V3 A[3] = {q0, q1, q2};
  const V3 B[3] = {q1, q2, q0};
  for (int k = 0; k < 3; ++k) {
    const V3 ab = sub(B[k], A[k]);
    const double den = dot(ab, ab);
    const double s = den == 0.0 ? 0.0 : fmin(1.0, fmax(0.0, dot(sub(p, A[k]), ab) / den));
    const V3 c = add(A[k], scl(s, ab));
    const V3 dd = sub(p, c);
    const double d2 = dot(dd, dd);
    if (k == 0 || d2 < bestd) {
      bestd = d2;
      best = c;
      if (k == 0) { b1 = s; b2 = 0.0; }
      else if (k == 1) { b1 = 1.0 - s; b2 = s; }
      else { b1 = 0.0; b2 = 1.0 - s; }
    }
  }
  return best;
}

template <typename T>
__device__ void face_verts(const Dev<T>& d, int f, V3& q0, V3& q1, V3& q2, int4& fv) {
  fv = chk_face(d.ctrl, d.faces[chk_idx(d.ctrl, f, d.n_f)], d.n_v);
  q0 = pos(d, fv.x);
  q1 = pos(d, fv.y);
  q2 = pos(d, fv.z);
}

// Warp argmin of (key, face id) over the lanes (face id < 0: no candidate);
// every lane ends with the minimum and its barycentrics.  The order is total,
// so the result does not depend on which lane held which face.
// Keys are non-negative doubles (ray parameters t > 0, squared distances), so
// their bit patterns order like their values and the comparisons run on the
// integer pipes: every lane of the warp takes part, and FP64 instructions
// with 32 active lanes are what the narrow FP64 pipe of this part is slowest
// at.
__device__ __forceinline__ unsigned long long key_bits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ void warp_argmin(int& f, double& key, double& b1, double& b2) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int of = __shfl_xor_sync(0xffffffffu, f, o);
    const double ok = __shfl_xor_sync(0xffffffffu, key, o);
    const double o1 = __shfl_xor_sync(0xffffffffu, b1, o);
    const double o2 = __shfl_xor_sync(0xffffffffu, b2, o);
    const unsigned long long kb = key_bits(key), okb = key_bits(ok);
    if (of >= 0 && (f < 0 || okb < kb || (okb == kb && of < f))) {
      f = of;
      key = ok;
      b1 = o1;
      b2 = o2;
    }
  }
}

// Closest-point candidate of face f for point o (lane-local running minimum).
template <typename T>
__device__ __forceinline__ void closest_candidate(const Dev<T>& d, int v, int rv, int f, V3 o, int& lf, double& ld,
                                                  double& l1, double& l2) {
  if (d.robot_of_face && d.robot_of_face[f] != rv) return;
  V3 q0, q1, q2;
  int4 fv;
  face_verts(d, f, q0, q1, q2, fv);
  if (fv.x == v || fv.y == v || fv.z == v) return;
  double b1, b2;
  const V3 x = closest_tri(o, q0, q1, q2, b1, b2);
  const V3 dd = sub(o, x);
  const double d2 = dot(dd, dd);
  if (lf < 0 || d2 < ld || (d2 == ld && f < lf)) {
    lf = f;
    ld = d2;
    l1 = b1;
    l2 = b2;
  }
}

// Self-collision correspondence of vertex v: first exit-face hit along dir,
// by one warp.  Every lane walks the same cells (3D-DDA); the faces listed in
// a cell are split over the lanes and the cell's first hit is the warp
// minimum of (t, face id), merged into the running first hit.  The result is
// the same as a serial walk's.
template <typename T>
__device__ int ray_cast_warp(const Dev<T>& d, int v, int rv, V3 o, V3 dir, double& rb1, double& rb2,
                             int& fell_back) {
  const int lane = threadIdx.x & 31;
  fell_back = 0;
  int best_f = -1;
  double best_t = 0.0;
  unsigned long long best_lim = 0;  // bits of best_t (1 + 1e-9)
  rb1 = rb2 = 0.0;
  // DDA set-up: lane a < 3 forms axis a's start cell, step, first boundary
  // parameter and increment, and its bound on the ray parameter from the
  // bounding box of this iteration's boundary faces (the ray can meet no face
  // beyond it); the warp shares them by shuffles, so the FP64 divisions run once per
  // axis, not once per lane.  tbox is the minimum over the axes.
  int cell[3], step[3];
  double tmax[3], tdel[3], tbox;
  {
    const int a = lane < 3 ? lane : 0;
    const double dva = a == 0 ? dir.x : a == 1 ? dir.y : dir.z;
    const double ova = a == 0 ? o.x : a == 1 ? o.y : o.z;
    int c_a = 0, st_a = 0;
    double tm_a = INFINITY, td_a = INFINITY, tb_a = INFINITY;
    if (lane < 3) {
      c_a = cell_coord(ova, d.inv_cell);
      const double blo = order_decode(d.ctrl->box_lo[a]) - d.cell, bhi = order_decode(d.ctrl->box_hi[a]) + d.cell;
      if (dva > 0.0) {
        st_a = 1;
        tm_a = ((c_a + 1) * d.cell - ova) / dva;
        td_a = d.cell / dva;
        tb_a = (bhi - ova) / dva;
      } else if (dva < 0.0) {
        st_a = -1;
        tm_a = (c_a * d.cell - ova) / dva;
        td_a = -d.cell / dva;
        tb_a = (blo - ova) / dva;
      }
      // ray parameters of the walk are compared by their bit patterns below,
      // so they are made non-negative: a start within rounding of a cell face
      // can give -0.0 or a tiny negative first boundary (either way the walk
      // first steps across it), and the walk starts inside the faces' box
      tm_a = tm_a > 0.0 ? tm_a : 0.0;
      tb_a = tb_a > 0.0 ? tb_a : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cell[k] = __shfl_sync(0xffffffffu, c_a, k);
      step[k] = __shfl_sync(0xffffffffu, st_a, k);
      tmax[k] = __shfl_sync(0xffffffffu, tm_a, k);
      tdel[k] = __shfl_sync(0xffffffffu, td_a, k);
    }
    tbox = fmin(fmin(__shfl_sync(0xffffffffu, tb_a, 0), __shfl_sync(0xffffffffu, tb_a, 1)),
                __shfl_sync(0xffffffffu, tb_a, 2));
  }
  for (int it = 0; it < MAX_DDA_STEPS; ++it) {
    const unsigned h = d.H_t + (hash_cell(cell[0], cell[1], cell[2], rv) & (d.H_f - 1u));
    const int k0 = d.cell_start[h], k1 = min(d.cell_start[h + 1], d.cap_items);
    int lf = -1;
    double lt = 0.0, l1 = 0.0, l2 = 0.0;
    for (int k = k0 + lane; k < k1; k += 32) {
      const int f = d.items[k] - d.n_t;
      if (d.robot_of_face && d.robot_of_face[f] != rv) continue;
      V3 q0, q1, q2;
      int4 fv;
      face_verts(d, f, q0, q1, q2, fv);
      if (fv.x == v || fv.y == v || fv.z == v) continue;
      if (!(dot(dir, cross(sub(q1, q0), sub(q2, q0))) > 0.0)) continue;
      double t, b1, b2;
      if (!ray_tri(o, dir, q0, q1, q2, t, b1, b2)) continue;
      if (lf < 0 || t < lt || (t == lt && f < lf)) {
        lf = f;
        lt = t;
        l1 = b1;
        l2 = b2;
      }
    }
    if (__any_sync(0xffffffffu, lf >= 0)) {
      warp_argmin(lf, lt, l1, l2);
      if (best_f < 0 || key_bits(lt) < key_bits(best_t) || (lt == best_t && lf < best_f)) {
        best_f = lf;
        best_t = lt;
        rb1 = l1;
        rb2 = l2;
        best_lim = key_bits(best_t * (1.0 + 1e-9));
      }
    }
    const unsigned long long m0 = key_bits(tmax[0]), m1 = key_bits(tmax[1]), m2 = key_bits(tmax[2]);
    const unsigned long long texit = m0 < m1 ? (m0 < m2 ? m0 : m2) : (m1 < m2 ? m1 : m2);
    if (best_f >= 0 && best_lim < texit) return best_f;
    if (texit >= key_bits(INFINITY) || texit > key_bits(tbox)) break;
    const int a = (m0 <= m1 && m0 <= m2) ? 0 : (m1 <= m2 ? 1 : 2);
    cell[a] += step[a];
    tmax[a] += tdel[a];
  }
  if (best_f >= 0) return best_f;
  fell_back = 1;
  // No exit face hit: the closest point over the boundary faces not
  // containing v, found by scanning cubic shells of cells around v's cell
  // (the cells of a shell split over the lanes).  After shell k every face
  // with a point within k cells has been seen, so the search stops once the
  // best distance is at most k cell edges.
  const int c0[3] = {cell_coord(o.x, d.inv_cell), cell_coord(o.y, d.inv_cell), cell_coord(o.z, d.inv_cell)};
  double bestd = 0.0;
  for (int k = 0; k <= 64; ++k) {
    const int side = 2 * k + 1;
    const int ncell = side * side * side;
    int lf = -1;
    double ld = 0.0, l1 = 0.0, l2 = 0.0;
    for (int idx = lane; idx < ncell; idx += 32) {
      const int dx = idx % side - k, dy = (idx / side) % side - k, dz = idx / (side * side) - k;
      if (max(abs(dx), max(abs(dy), abs(dz))) != k) continue;
      const unsigned h = d.H_t + (hash_cell(c0[0] + dx, c0[1] + dy, c0[2] + dz, rv) & (d.H_f - 1u));
      const int k0 = d.cell_start[h], k1 = min(d.cell_start[h + 1], d.cap_items);
      for (int q = k0; q < k1; ++q) closest_candidate(d, v, rv, d.items[q] - d.n_t, o, lf, ld, l1, l2);
    }
    warp_argmin(lf, ld, l1, l2);
    if (lf >= 0 && (best_f < 0 || ld < bestd || (ld == bestd && lf < best_f))) {
      best_f = lf;
      bestd = ld;
      rb1 = l1;
      rb2 = l2;
    }
    if (best_f >= 0 && sqrt(bestd) <= k * d.cell) return best_f;
  }
  if (best_f >= 0) return best_f;
  // the shell search found nothing within 64 cells: every face (rare)
  int lf = -1;
  double ld = 0.0, l1 = 0.0, l2 = 0.0;
  for (int f = lane; f < d.n_f; f += 32) closest_candidate(d, v, rv, f, o, lf, ld, l1, l2);
  warp_argmin(lf, ld, l1, l2);
  rb1 = l1;
  rb2 = l2;
  return lf;
}

template <typename T>
__device__ __forceinline__ V3 face_point(const Dev<T>& d, int f, double b1, double b2, V3& nunit) {
  V3 q0, q1, q2;
  int4 fv;
  face_verts(d, f, q0, q1, q2, fv);
  V3 n = cross(sub(q1, q0), sub(q2, q0));
  nunit = scl(1.0 / norm(n), n);
  return add(add(scl(1.0 - b1 - b2, q0), scl(b1, q1)), scl(b2, q2));
}

// Point and unit outward normal of boundary face f of the tetrahedral
// obstacle at barycentrics (b1, b2).
template <typename T>
__device__ __forceinline__ V3 obstacle_face_point(const Dev<T>& d, int f, double b1, double b2, V3& nunit) {
  const int4 fv = d.oface[f];
  const R4<T> a = d.OX[fv.x], b = d.OX[fv.y], c = d.OX[fv.z];
  const V3 q0 = {(double)a.x, (double)a.y, (double)a.z}, q1 = {(double)b.x, (double)b.y, (double)b.z},
           q2 = {(double)c.x, (double)c.y, (double)c.z};
  const V3 n = cross(sub(q1, q0), sub(q2, q0));
  nunit = scl(1.0 / norm(n), n);
  return add(add(scl(1.0 - b1 - b2, q0), scl(b1, q1)), scl(b2, q2));
}

// Closest point of the tetrahedral obstacle's boundary to x (Sec. II-C,
// robot-obstacle response): the face with the smallest squared distance,
// ties to the lowest face id, found through the obstacle's face tree.
template <typename T>
__device__ __forceinline__ int obstacle_closest(const Dev<T>& d, V3 x, double& b1, double& b2, double& d2) {
  int bf = -1;
  double bd = INFINITY, c1 = 0.0, c2 = 0.0;
  bvh_nearest(
      d.of, 0, x.x, x.y, x.z,
      [&](int f) {
        const int4 fv = d.oface[f];
        const R4<T> a = d.OX[fv.x], b = d.OX[fv.y], c = d.OX[fv.z];
        const V3 q0 = {(double)a.x, (double)a.y, (double)a.z}, q1 = {(double)b.x, (double)b.y, (double)b.z},
                 q2 = {(double)c.x, (double)c.y, (double)c.z};
        double e1, e2;
        const V3 p = closest_tri(x, q0, q1, q2, e1, e2);
        const V3 dd = sub(x, p);
        const double dist2 = dot(dd, dd);
        if (bf < 0 || dist2 < bd || (dist2 == bd && f < bf)) {
          bf = f;
          bd = dist2;
          c1 = e1;
          c2 = e2;
        }
      },
      [&]() { return bd; });
  b1 = c1;
  b2 = c2;
  d2 = bd;
  return bf;
}

// Spring update, one thread per query vertex.  A vertex in a self pair (and
// in no obstacle) needs a ray cast: it is appended to the cast list with its
// unit normal and finished by k_cast (or k_cast_bvh); every other vertex is
// finished by the update itself.
static constexpr int CAST_THREADS = 256;

// Signature term of one spring record (see sig_mix): query index and the
// decision code (0 a self spring kept from its record, 1 a sphere spring, 2 a
// tetrahedral-obstacle spring, 3 a self spring cast in this iteration) with
// the face, sphere or obstacle face id.
__device__ __forceinline__ unsigned long long spring_term(int qi, int code, int face) {
  return sig_mix((unsigned)qi, ((unsigned)code << 30) ^ (unsigned)(face + 1));
}

// Spring update of query vertex qi, by one thread, once its contacts of this
// iteration are known (pair_count, obs_sphere, obs_mesh): creates, re-targets
// or releases its spring, or queues it for a ray cast.  Adds 1 to active_out
// for a finished active spring and its signature term to ssig.
template <typename T>
__device__ void spring_update_vertex(const Dev<T>& d, int qi, int& active_out, unsigned long long& ssig) {
  {
    const int v = d.q_verts[qi];
    // area-weighted unit vertex normal of the incident boundary faces, formed
    // only where it is used (a queued ray cast, a sphere spring whose vertex
    // sits at the centre): most vertices have no contact, and this FP64
    // work is the costliest part of the update
    auto normal = [&]() {
      V3 n = {0.0, 0.0, 0.0};
      for (int k = d.qf_ptr[qi]; k < d.qf_ptr[qi + 1]; ++k) {
        V3 q0, q1, q2;
        int4 fv;
        face_verts(d, d.qf[k], q0, q1, q2, fv);
        n = add(n, cross(sub(q1, q0), sub(q2, q0)));
      }
      const double nl = norm(n);
      return nl > 0.0 ? scl(1.0 / nl, n) : V3{0.0, 0.0, 0.0};
    };
    int active = d.sp.active[qi];
    int kind = d.sp.kind[qi];
    int face = d.sp.face[qi];
    double b1 = d.sp.bary[2 * qi], b2 = d.sp.bary[2 * qi + 1];
    V3 tgt = {0.0, 0.0, 0.0};
    int js = d.obs_sphere[qi];
    const double eps = d.eps;
    bool deferred = false;
    const bool in_mesh = d.obs_mesh && d.obs_mesh[qi] > 0;
    // the position in FP64, read only by a vertex with an obstacle contact or
    // a spring to re-target (the conversions are FP64 instructions)
    V3 x = {0.0, 0.0, 0.0};
    if (in_mesh || js >= 0 || active) x = pos(d, v);
    // inside the tetrahedral obstacle: its closest boundary point, unless a
    // containing sphere's surface is at least as near (signed distances
    // |x - c| - r and minus the distance to the obstacle's boundary)
    int mf = -1;
    double m1 = 0.0, m2 = 0.0;
    if (in_mesh) {
      double md2;
      mf = obstacle_closest(d, x, m1, m2, md2);
      if (js >= 0 && mf >= 0) {
        const V3 c = {d.spheres[4 * js], d.spheres[4 * js + 1], d.spheres[4 * js + 2]};
        if (!(norm(sub(x, c)) - d.spheres[4 * js + 3] <= -sqrt(md2))) js = -1;
        else mf = -1;
      }
    }
    if (js >= 0) {
      const V3 c = {d.spheres[4 * js], d.spheres[4 * js + 1], d.spheres[4 * js + 2]};
      const double r = d.spheres[4 * js + 3];
      V3 u = sub(x, c);
      const double nu = norm(u);
      u = nu == 0.0 ? scl(-1.0, normal()) : scl(1.0 / nu, u);
      active = 1;
      kind = 1;
      face = js;
      b1 = b2 = 0.0;
      tgt = add(c, scl(r + eps, u));
    } else if (mf >= 0) {
      V3 nf;
      const V3 bp = obstacle_face_point(d, mf, m1, m2, nf);
      active = 1;
      kind = 2;
      face = mf;
      b1 = m1;
      b2 = m2;
      tgt = add(bp, scl(eps, nf));
    } else if (d.pair_count[qi] > 0) {
      deferred = true;
      const int slot = atomicAdd(&d.ctrl->n_cast, 1);  // < n_q: each vertex enters once
      d.cast_list[slot] = qi;
      const V3 n = normal();
      d.cast_nrm[3 * qi] = n.x;
      d.cast_nrm[3 * qi + 1] = n.y;
      d.cast_nrm[3 * qi + 2] = n.z;
    } else if (active) {
      if (kind == 1) {
        const V3 c = {d.spheres[4 * face], d.spheres[4 * face + 1], d.spheres[4 * face + 2]};
        const double r = d.spheres[4 * face + 3];
        V3 u = sub(x, c);
        const double nu = norm(u);
        if (nu - r > eps) {
          active = 0;
        } else {
          u = nu == 0.0 ? scl(-1.0, normal()) : scl(1.0 / nu, u);
          tgt = add(c, scl(r + eps, u));
        }
      } else if (kind == 2) {
        V3 nf;
        const V3 bp = obstacle_face_point(d, face, b1, b2, nf);
        if (dot(nf, sub(x, bp)) > eps) {
          active = 0;
        } else {
          tgt = add(bp, scl(eps, nf));
        }
      } else {
        V3 nf;
        const V3 bp = face_point(d, face, b1, b2, nf);
        if (dot(nf, sub(x, bp)) > eps) {
          active = 0;
        } else {
          tgt = add(bp, scl(eps, nf));
        }
      }
    }
    if (!deferred) {
      if (!active) {
        kind = 0;
        face = -1;
        b1 = b2 = 0.0;
        tgt = {0.0, 0.0, 0.0};
      }
      d.sp.active[qi] = active;
      d.sp.fallback[qi] = 0;
      d.sp.kind[qi] = kind;
      d.sp.face[qi] = face;
      d.sp.bary[2 * qi] = b1;
      d.sp.bary[2 * qi + 1] = b2;
      d.sp.target[3 * qi] = tgt.x;
      d.sp.target[3 * qi + 1] = tgt.y;
      d.sp.target[3 * qi + 2] = tgt.z;
      d.spring_c[v] = R4<double>{tgt.x, tgt.y, tgt.z, active ? 1.0 : 0.0};
      active_out += active;
      if (active) ssig += spring_term(qi, kind, face);
    }
  }
}

// Spring update of every query vertex, one thread each (the hash broad
// phase's narrow phase runs one warp per vertex, which would leave 31 lanes
// idle during this FP64 work; the tree's narrow phase runs one thread per
// vertex and does the update in the same launch).
template <typename T>
__global__ void __launch_bounds__(128) k_springs(Dev<T> d) {
  __shared__ int shi[32];
  const int qi = blockIdx.x * blockDim.x + threadIdx.x;
  int n_spr = 0;
  unsigned long long ssig = 0;
  if (qi < d.n_q) spring_update_vertex(d, qi, n_spr, ssig);
  narrow_block_totals(d, 0, 0, n_spr, ssig, shi);
}

// Self springs of the listed vertices: one warp per vertex shares the ray
// cast (persistent grid, warps stride over the list); lane 0 writes the
// spring record, v_c = hit point + eps n_f.
template <typename T>
__global__ void __launch_bounds__(CAST_THREADS) k_cast(Dev<T> d) {
  __shared__ int shi[32];
  const int lane = threadIdx.x & 31;
  const int n_warps = gridDim.x * (CAST_THREADS / 32);
  const int n_cast = d.ctrl->n_cast;
  int active_out = 0;
  for (int j = (int)((blockIdx.x * (unsigned)CAST_THREADS + threadIdx.x) >> 5); j < n_cast; j += n_warps) {
    const int qi = chk_idx(d.ctrl, d.cast_list[j], d.n_q);
    const int v = d.q_verts[qi];
    const V3 x = pos(d, v);
    const V3 n = {d.cast_nrm[3 * qi], d.cast_nrm[3 * qi + 1], d.cast_nrm[3 * qi + 2]};
    const int rv = d.robot_of_vert ? d.robot_of_vert[v] : 0;
    double b1, b2;
    int fell_back;
    const int f = ray_cast_warp(d, v, rv, x, scl(-1.0, n), b1, b2, fell_back);
    if (lane == 0) {
      V3 tgt = {0.0, 0.0, 0.0};
      if (f >= 0) {
        V3 nf;
        const V3 bp = face_point(d, f, b1, b2, nf);
        tgt = add(bp, scl(d.eps, nf));
      } else {
        b1 = b2 = 0.0;
      }
      const int active = f >= 0;
      d.sp.active[qi] = active;
      d.sp.fallback[qi] = fell_back;
      d.sp.kind[qi] = 0;
      d.sp.face[qi] = f;
      d.sp.bary[2 * qi] = b1;
      d.sp.bary[2 * qi + 1] = b2;
      d.sp.target[3 * qi] = tgt.x;
      d.sp.target[3 * qi + 1] = tgt.y;
      d.sp.target[3 * qi + 2] = tgt.z;
      d.spring_c[v] = R4<double>{tgt.x, tgt.y, tgt.z, active ? 1.0 : 0.0};
      active_out += active;
      if (active && d.stats) atomicAdd(&(d.hist + (d.ctrl->iter % d.hist_cap))->spring_sig, spring_term(qi, 3, f));
    }
  }
  const int ns = block_sum_int(active_out, shi);
  if (threadIdx.x == 0 && ns) atomicAdd(&(d.hist + (d.ctrl->iter % d.hist_cap))->n_springs, ns);
}

// Self springs of the listed vertices with the robot's face tree (broad
// phase 1): one thread per casting vertex finds the first exit face along
// -n(v) (smallest t, then the lowest face id; the tree prunes boxes entered
// beyond the best hit), else the closest point over the boundary faces not
// containing v (smallest squared distance, then the lowest face id).
template <typename T>
__global__ void __launch_bounds__(CAST_THREADS) k_cast_bvh(Dev<T> d) {
  __shared__ int shi[32];
  const int n_cast = d.ctrl->n_cast;
  int active_out = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_cast; j += gridDim.x * blockDim.x) {
    const int qi = chk_idx(d.ctrl, d.cast_list[j], d.n_q);
    const int v = d.q_verts[qi];
    const V3 x = pos(d, v);
    const V3 dir = {-d.cast_nrm[3 * qi], -d.cast_nrm[3 * qi + 1], -d.cast_nrm[3 * qi + 2]};
    const int rv = d.robot_of_vert ? d.robot_of_vert[v] : 0;
    int bf = -1, fell_back = 0;
    double bt = INFINITY, b1 = 0.0, b2 = 0.0;
    const double o[3] = {x.x, x.y, x.z}, dv[3] = {dir.x, dir.y, dir.z};
    bvh_ray(
        d.bf, rv, o, dv,
        [&](int f) {
          if (d.robot_of_face && d.robot_of_face[f] != rv) return;
          V3 q0, q1, q2;
          int4 fv;
          face_verts(d, f, q0, q1, q2, fv);
          if (fv.x == v || fv.y == v || fv.z == v) return;
          if (!(dot(dir, cross(sub(q1, q0), sub(q2, q0))) > 0.0)) return;
          double t, e1, e2;
          if (!ray_tri(x, dir, q0, q1, q2, t, e1, e2)) return;
          if (bf < 0 || t < bt || (t == bt && f < bf)) {
            bf = f;
            bt = t;
            b1 = e1;
            b2 = e2;
          }
        },
        [&]() { return bt; });
    if (bf < 0) {
      fell_back = 1;
      double bd = INFINITY;
      bvh_nearest(
          d.bf, rv, x.x, x.y, x.z,
          [&](int f) {
            if (d.robot_of_face && d.robot_of_face[f] != rv) return;
            V3 q0, q1, q2;
            int4 fv;
            face_verts(d, f, q0, q1, q2, fv);
            if (fv.x == v || fv.y == v || fv.z == v) return;
            double e1, e2;
            const V3 p = closest_tri(x, q0, q1, q2, e1, e2);
            const V3 dd = sub(x, p);
            const double dist2 = dot(dd, dd);
            if (bf < 0 || dist2 < bd || (dist2 == bd && f < bf)) {
              bf = f;
              bd = dist2;
              b1 = e1;
              b2 = e2;
            }
          },
          [&]() { return bd; });
    }
    V3 tgt = {0.0, 0.0, 0.0};
    if (bf >= 0) {
      V3 nf;
      const V3 bp = face_point(d, bf, b1, b2, nf);
      tgt = add(bp, scl(d.eps, nf));
    } else {
      b1 = b2 = 0.0;
    }
    const int active = bf >= 0;
    d.sp.active[qi] = active;
    d.sp.fallback[qi] = fell_back;
    d.sp.kind[qi] = 0;
    d.sp.face[qi] = bf;
    d.sp.bary[2 * qi] = b1;
    d.sp.bary[2 * qi + 1] = b2;
    d.sp.target[3 * qi] = tgt.x;
    d.sp.target[3 * qi + 1] = tgt.y;
    d.sp.target[3 * qi + 2] = tgt.z;
    d.spring_c[v] = R4<double>{tgt.x, tgt.y, tgt.z, active ? 1.0 : 0.0};
    active_out += active;
    if (active && d.stats) atomicAdd(&(d.hist + (d.ctrl->iter % d.hist_cap))->spring_sig, spring_term(qi, 3, bf));
  }
  const int ns = block_sum_int(active_out, shi);
  if (threadIdx.x == 0 && ns) atomicAdd(&(d.hist + (d.ctrl->iter % d.hist_cap))->n_springs, ns);
}

// ---- launchers ----
template <typename T>
void launch_bvh_refit(const BvhDev& b, const R4<T>* X, cudaStream_t st) {
  if (b.n < 2 || !b.flag) return;
  cudaMemsetAsync(b.flag, 0, sizeof(int) * (size_t)(b.n - 1), st);
  k_bvh_refit<T><<<(b.n + 255) / 256, 256, 0, st>>>(b, X);
}

template <typename T>
void launch_collision(const Dev<T>& d, const CollisionScratch& cs, cudaStream_t st) {
  if (d.broad == 1) {
    // AABB trees: refit the tet and face trees to this iteration's positions
    launch_bvh_refit<T>(d.bt, d.X, st);
    launch_bvh_refit<T>(d.bf, d.X, st);
    if (d.n_q > 0)
      k_narrow_bvh<T><<<(d.n_q + NARROW_BVH_THREADS - 1) / NARROW_BVH_THREADS, NARROW_BVH_THREADS, 0, st>>>(d);
    return;
  }
  const int n_items = d.n_t + d.n_f;
  const int H = (int)(d.H_t + d.H_f);
  // with the single-pass scan its status words and ticket follow the counts
  // and are zeroed by the same memset
  const size_t n_zero = (size_t)(H + 1) + (cs.tile_status ? (size_t)scan_lookback_extra_ints(H + 1) : 0);
  cudaMemsetAsync(d.cell_count, 0, sizeof(int) * n_zero, st);
  cudaMemsetAsync(d.cell_cursor, 0, sizeof(int) * (size_t)H, st);
  k_grid_bin<T, false><<<(n_items + 255) / 256, 256, 0, st>>>(d);
  const int n_scan = H + 1;
  const int n_tiles = (n_scan + SCAN_TILE - 1) / SCAN_TILE;
  if (cs.tile_status) {
    k_scan_lookback<<<n_tiles, SCAN_THREADS, 0, st>>>(d.cell_count, d.cell_start, n_scan, cs.tile_status, cs.ticket,
                                                       cs.total, d.ctrl, d.cap_items, d.wait_budget);
  } else {
    k_scan_tiles<<<n_tiles, SCAN_THREADS, 0, st>>>(d.cell_count, d.cell_start, cs.tile_sums, n_scan);
    k_scan_top<<<1, 1024, 0, st>>>(cs.tile_sums, n_tiles, cs.total, d.ctrl, d.cap_items);
    k_scan_add<<<(n_scan + 255) / 256, 256, 0, st>>>(d.cell_start, cs.tile_sums, n_scan);
  }
  k_grid_bin<T, true><<<(n_items + 255) / 256, 256, 0, st>>>(d);
  if (d.n_q > 0) {
    const long long threads = 32LL * d.n_q;
    const int bs = d.narrow_threads > 0 ? d.narrow_threads : 256;
    const unsigned nb = (unsigned)((threads + bs - 1) / bs);
    if (bs == 128)
      k_narrow<T, 128><<<nb, 128, 0, st>>>(d);
    else if (bs == 512)
      k_narrow<T, 512><<<nb, 512, 0, st>>>(d);
    else
      k_narrow<T, 256><<<nb, 256, 0, st>>>(d);
  }
}

// The spring update (a separate launch after the hash's narrow phase, inside
// the tree's narrow phase), then the ray casts of the vertices it queued.
template <typename T>
void launch_springs(const Dev<T>& d, cudaStream_t st) {
  if (d.n_q <= 0) return;
  if (d.broad != 1) k_springs<T><<<(d.n_q + 127) / 128, 128, 0, st>>>(d);
  // enough warps for one pass over a list of up to 8,192 casts
  if (d.broad == 1) {
    k_cast_bvh<T><<<std::min((d.n_q + CAST_THREADS - 1) / CAST_THREADS, 1024), CAST_THREADS, 0, st>>>(d);
    return;
  }
  const int per_block = CAST_THREADS / 32;
  const int blocks = std::min((d.n_q + per_block - 1) / per_block, 1024);
  k_cast<T><<<blocks, CAST_THREADS, 0, st>>>(d);
}
int scan_tiles(int n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

void launch_scan_exclusive(const int* in, int* out, int n, int* tile_sums, int* total, cudaStream_t st) {
  if (n <= 0) return;
  const int n_tiles = scan_tiles(n);
  k_scan_tiles<<<n_tiles, SCAN_THREADS, 0, st>>>(in, out, tile_sums, n);
  k_scan_top<<<1, 1024, 0, st>>>(tile_sums, n_tiles, total, nullptr, 0);
  k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(out, tile_sums, n);
}

template void launch_bvh_refit<float>(const BvhDev&, const R4<float>*, cudaStream_t);
template void launch_bvh_refit<double>(const BvhDev&, const R4<double>*, cudaStream_t);
template void launch_collision<float>(const Dev<float>&, const CollisionScratch&, cudaStream_t);
template void launch_collision<double>(const Dev<double>&, const CollisionScratch&, cudaStream_t);
template void launch_springs<float>(const Dev<float>&, cudaStream_t);
template void launch_springs<double>(const Dev<double>&, cudaStream_t);

}  // namespace casim
