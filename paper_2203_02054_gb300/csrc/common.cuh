// Device-side data layout and helpers shared by the casim CUDA kernels.
//
// Layout in HBM (per simulation, T = float in MIXED mode, double in FP64):
//   vertices  X[n_v] as R4<T> (x, y, z, pad); internal order = free vertices
//             first (robot by robot, each robot's in recursive coordinate
//             bisection order of the rest positions), then the fixed ones in
//             the caller's relative order;
//   elements  tet[n_t] int4 internal vertex ids (caller's tet order),
//             Tc[3 n_t] rows x/y/z of the centered rest shape V N (Eq. 1),
//             tinfo[n_t] (omega_e, Vol_e, |T_c|^2, group id as T),
//             P[4 n_t] omega_e-weighted target columns written by the local step;
//   system    incidence CSR of free vertices (tet*4 + slot), constant
//             Laplacian off-diagonals in sliced ELL (32-row slices,
//             column-major inside a slice), diagonal separate;
//   PCG       r, u, p, s, w, dx vectors R4<T>[n_free], FP64 block partials;
//             right-hand side b and the fixed-vertex term in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace casim {

template <typename T>
struct __align__(4 * sizeof(T)) R4 {
  T x, y, z, w;
};

// Device status bits (OR-ed by kernels, mapped to CASIM_* codes on the host).
enum : int {
  ST_NONFINITE = 1,
  ST_TIMEOUT = 2,
  ST_PCG_MAXIT = 4,
  ST_OVERFLOW = 8,
  ST_PAIRS_TRUNC = 16,   // a vertex had more self pairs than max_pairs_per_vertex
  ST_BAD_INPUT = 32,     // an input id out of range (checked on the device before use)
  ST_BOUNDS = 64,        // a gather index out of range (builds with -DCASIM_CHECKED only)
};

struct IterRec {
  double energy;
  double pcg_rel_residual;
  int n_self_pairs;
  int n_obstacle_pairs;
  int n_springs;
  int pcg_iters;
  unsigned long long knot_sig;    // sum over body tets of sig_mix(tet, w-table interval of its strain)
  unsigned long long spring_sig;  // sum over active springs of sig_mix(query index, kind and face / sphere)
};

// Order-independent signatures of the discrete state of an iteration: a sum
// (mod 2^64) of the SplitMix64 output function (Steele, Lea and Flood 2014)
// applied to (index, state) pairs.  Equal signatures mean equal states with
// overwhelming probability; the sum does not depend on the order of the adds.
__host__ __device__ inline unsigned long long sig_mix(unsigned a, unsigned b) {
  unsigned long long z = ((unsigned long long)a << 32 | b) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#ifdef __CUDACC__
// Adds v (summed over the warp first) to *dst from lane 0; all lanes call it.
__device__ inline void warp_add_u64(unsigned long long v, unsigned long long* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}
#endif

struct Ctrl {
  int status;            // ST_* bits
  int abort;             // set when a grid barrier gives up
  unsigned bar_count;    // grid barrier arrival counter (top bit = round parity)
  unsigned queue;        // next robot for the cluster PCG work queue
  long long iter;        // outer iterations completed (history index)
  long long total_pcg;   // PCG iterations summed over outer iterations
  int n_items;           // spatial-hash entries of this iteration
  int n_cast;            // ray-cast list length of this iteration (reset at its end)
  long long box_lo[3];   // bounding box of all item boxes of this iteration,
  long long box_hi[3];   //   as order-preserving integer codes of doubles
};

// Order-preserving map between doubles and 64-bit integers (for atomic
// min / max of doubles).
__host__ __device__ inline long long order_code(double v) {
  union {
    double d;
    long long i;
  } u;
  u.d = v;
  return u.i >= 0 ? u.i : (u.i ^ 0x7FFFFFFFFFFFFFFFLL);
}
__host__ __device__ inline double order_decode(long long c) {
  union {
    double d;
    long long i;
  } u;
  u.i = c >= 0 ? c : (c ^ 0x7FFFFFFFFFFFFFFFLL);
  return u.d;
}

// AABB trees (layout in bvh.cuh): n primitives, one tree per robot.
struct BvhDev {
  int n;               // primitives; 0 = no tree
  int nv;              // vertices per primitive: 4 (tets) or 3 (faces)
  const int2* child;   // n - 1
  const int* parent;   // 2 n - 1
  float4* lo;          // n - 1 internal boxes
  float4* hi;
  int* flag;           // n - 1 refit arrival counters (zeroed before each refit)
  const int4* prim;    // primitive vertex ids
  const int* root;     // per robot: root code of its tree (null: one tree rooted at node 0)
};

struct SpringDev {
  int* active;           // n_q
  int* kind;             // n_q: 0 self, 1 sphere obstacle, 2 tetrahedral obstacle
  int* face;             // n_q: face id / sphere id / obstacle face id / -1
  double* bary;          // 2 n_q
  double* target;        // 3 n_q
  int* fallback;         // n_q: 1 if this update's self target is a closest point
};

template <typename T>
struct Dev {
  int n_v, n_t, n_free, n_q, n_f, n_groups, n_spheres, n_knots;
  // vertices and elements
  R4<T>* X;
  const int4* tet;
  const R4<T>* Tc;
  const R4<T>* tinfo;
  R4<T>* P;
  const T* cbrt_alpha;   // per chamber group
  const double* knots;   // 2 n_knots
  // system
  const int* inc_ptr;    // n_free + 1
  const int* inc;        // tet*4 + slot
  const T* diagL;        // n_free
  const R4<double>* bfix; // n_free, FP64
  R4<double>* b;          // n_free, FP64 right-hand side
  T* diag;               // n_free (Laplacian diagonal + k mask)
  int n_slices;
  const int* sl_ptr;     // n_slices + 1 (entries)
  const int* sl_col;     // entries
  const T* sl_val;       // entries
  R4<T>* r;
  R4<T>* u;
  R4<T>* p;
  R4<T>* s;
  R4<T>* w;
  R4<T>* dx;             // PCG correction (streaming kernel)
  R4<T>* xstep;          // dataflow PCG of an outer iteration: x_i - x_(i-1) per free row; the solve starts
                         //   from x_i + xstep instead of x_i (null: from x_i)
  double* partials;      // 2 x 4 x pcg grid
  unsigned long long* df_u;  // dataflow PCG: 2 x n_free x 2 epoch-tagged words of u
  unsigned long long* df_p;  // dataflow PCG: 2 x (grid + 1) x 4 epoch-tagged partial words
  const int* halo_ptr;   // dataflow PCG: per block, start of its halo in halo_rows
  const int* halo_rows;  //   distinct rows each block's SpMV reads: its own rows, then the
                         //   others (each part ascending)
  const int* halo_own;   //   per block, how many of its halo rows are its own
  const int* halo_self;  //   per free row, its index in its block's halo (-1: not read)
  const int* sl_lcol;    //   per sliced-ELL entry: the column's index in its block's halo
  int halo_max;          //   longest halo (rows)
  int df_rows;           //   rows (threads) per block: 288 or 384
  const float* cg_ainv;  // dataflow PCG coarse correction: A_c^-1 (n_agg x n_agg, row-major)
  int n_agg;             //   aggregates of 128 consecutive free rows; 0 = Jacobi only
  // collision
  const int* q_verts;    // n_q internal vertex ids, in ascending caller id
  const int* qf_ptr;     // n_q + 1 incident boundary faces
  const int* qf;         // face ids
  const int4* faces;     // n_f (v0, v1, v2, owning tet)
  const double* spheres; // 4 n_spheres
  const float* spheres_f; // the same, rounded to FP32 (the reject test before the FP64 one)
  unsigned H_t, H_f;     // hash sizes (powers of two)
  int* cell_count;       // H_t + H_f (+1)
  int* cell_start;       // H_t + H_f + 1
  int* cell_cursor;      // H_t + H_f
  int* items;            // cap_items
  int cap_items;
  int* pair_count;       // n_q
  int* pair_tet;         // n_q * max_pairs
  int* obs_sphere;       // n_q: sphere id or -1
  int max_pairs;
  SpringDev sp;
  int* cast_list;        // n_q: query indices whose spring needs a ray cast
  double* cast_nrm;      // 3 n_q: unit vertex normal of each listed query vertex
  R4<double>* spring_c;  // n_free: (c, mask), FP64
  // AABB trees (broad phase 1) and the rigid tetrahedral obstacle
  int broad;             // 0 spatial hash, 1 AABB trees refitted every iteration
  BvhDev bt, bf;         // robot tets, robot boundary faces
  BvhDev ot, of;         // obstacle tets, obstacle boundary faces (static)
  const R4<T>* OX;       // obstacle positions (the working precision)
  const int4* oface;     // obstacle boundary faces (v0, v1, v2, owning tet)
  int n_of;
  int* obs_mesh;         // n_q: obstacle tets strictly containing the vertex
  // parameters
  double k_spring, eps, cell, inv_cell, tol2;
  int max_iter, collision, stats;
  int local_threads, rhs_threads, narrow_threads;  // launch shapes (autotuned)
  int rhs_in_pcg;        // 1: the dataflow PCG forms b, the diagonal and the iteration's record itself
  int n_robots;          // independent systems (robots) in the mesh
  const int* robot_row;  // n_robots + 1: first free row of each robot
  int cl_rows_cap;       // rows per CTA the cluster PCG's shared memory holds
  const int* robot_of_vert;  // n_v (internal order); null for a single robot
  const int* robot_of_tet;   // n_t; null for a single robot
  const int* robot_of_face;  // n_f; null for a single robot
  const int* seg_lo;     // segmented PCG: per block, first row
  const int* seg_hi;     //   one past the last row
  const int* seg_rb0;    //   first block of the block's robot
  const int* seg_rb1;    //   one past the robot's last block
  const int* seg_robot;  //   the block's robot
  int seg_coarse;        //   1: per-robot two-level preconditioner (MIXED)
  const int* seg_agg_base;       // per robot: first aggregate (global index); + 1 entries
  const long long* seg_ainv_off; // per robot: offset of its A_c^-1 (n_agg^2 floats, row-major)
  const float* seg_ainv;
  float* seg_aggsum;     //   per aggregate: sums of w (3) and r (3) of the last pass
  unsigned bar_extra;    // 0; 1 = test-only: the barrier expects one more block
  unsigned long long wait_budget;
  // control and statistics
  Ctrl* ctrl;
  IterRec* hist;
  int hist_cap;
  double* e_partials;    // energy partials (local-step blocks + RHS blocks, whose
                         //   rows carry the spring energy)
  int n_e_local, n_e_spring;
};

__host__ __device__ inline unsigned hash_cell(int cx, int cy, int cz, int robot = 0) {
  // Spatial hash of Teschner et al. 2003 ("Optimized spatial hashing for
  // collision detection of deformable objects"), with the robot id mixed in
  // so that robots placed at the same location do not share buckets.
  return ((unsigned)cx * 73856093u) ^ ((unsigned)cy * 19349663u) ^ ((unsigned)cz * 83492791u) ^
         ((unsigned)robot * 2654435761u);
}

// Cell coordinate of one coordinate value: floor(x / cell), clamped so that
// far-away or non-finite values cannot overflow the integer range.  The map is
// monotone in x, so a point inside a closed box maps into the box's cell range.
__device__ inline int cell_coord(double x, double inv_cell) {
  double c = floor(x * inv_cell);
  c = fmin(fmax(c, -1.0e6), 1.0e6);
  return (int)c;
}

template <typename T>
__device__ inline bool finite4(const R4<T>& a) {
  return isfinite((double)a.x) && isfinite((double)a.y) && isfinite((double)a.z);
}

__device__ inline void set_status(Ctrl* c, int bits) { atomicOr(&c->status, bits); }

// Gather index check.  In builds with -DCASIM_CHECKED (the stand-in for a
// memory checker, which this pool does not offer) an index outside [0, n)
// sets ST_BOUNDS and is replaced by 0, so the access stays inside its array
// and the step ends with CASIM_E_BOUNDS; other builds use the index as is.
#ifdef CASIM_CHECKED
__device__ __forceinline__ int chk_idx(Ctrl* c, int i, int n) {
  if ((unsigned)i >= (unsigned)n) {
    atomicOr(&c->status, ST_BOUNDS);
    return 0;
  }
  return i;
}
#else
__device__ __forceinline__ int chk_idx(Ctrl*, int i, int) { return i; }
#endif
__device__ __forceinline__ int4 chk_idx4(Ctrl* c, int4 t, int n) {
  return make_int4(chk_idx(c, t.x, n), chk_idx(c, t.y, n), chk_idx(c, t.z, n), chk_idx(c, t.w, n));
}
// a boundary face (x, y, z vertices, w its tet): the three vertex indices
__device__ __forceinline__ int4 chk_face(Ctrl* c, int4 f, int n_v) {
  return make_int4(chk_idx(c, f.x, n_v), chk_idx(c, f.y, n_v), chk_idx(c, f.z, n_v), f.w);
}

// Block-wide sum of one double (blockDim.x a multiple of 32, <= 1024); the
// result is valid in thread 0.  Fixed reduction order -> deterministic.
__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t += sh[i];
  }
  return t;
}

__device__ inline int block_sum_int(int v, int* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int t = 0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t += sh[i];
  }
  return t;
}

}  // namespace casim
