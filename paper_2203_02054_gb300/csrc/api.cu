// casim C ABI: host-side mesh preparation, validation, device memory and the
// CUDA graph that runs one outer iteration of the collision-aware
// local-global loop (Algorithm 1, inner while-loop).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstddef>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <limits>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "casim.h"
#include "common.cuh"
#include "kernels.h"

using namespace casim;

namespace {

thread_local std::string g_create_error;

// Outward faces of a positively oriented tet (v0, v1, v2, v3): face k is the
// face opposite local vertex k, counter-clockwise seen from outside.
const int kTetFace[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};

size_t pow2_at_least(size_t n) {
  size_t p = 1024;
  while (p < n) p <<= 1;
  return p;
}

// Recursive coordinate bisection of the vertices idx[0..n) by their rest
// positions: split along the longest extent of the set's bounding box so that
// the first part holds a multiple of `leaf` vertices (about half), order
// each part recursively; ties by vertex id, so the order is deterministic.
void rcb_order(const double* xyz, int* idx, int n, int leaf) {
  if (n <= leaf) {
    std::sort(idx, idx + n);
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], xyz[3 * (size_t)idx[i] + c]);
      hi[c] = std::max(hi[c], xyz[3 * (size_t)idx[i] + c]);
    }
  int ax = 0;
  for (int c = 1; c < 3; ++c)
    if (hi[c] - lo[c] > hi[ax] - lo[ax]) ax = c;
  const int nl = leaf * ((n + 2 * leaf - 1) / (2 * leaf));
  std::nth_element(idx, idx + nl, idx + n, [&](int a, int b) {
    const double xa = xyz[3 * (size_t)a + ax], xb = xyz[3 * (size_t)b + ax];
    return xa < xb || (xa == xb && a < b);
  });
  rcb_order(xyz, idx, nl, leaf);
  rcb_order(xyz, idx + nl, n - nl, leaf);
}

// AABB trees over n primitives with centroids cen (3 per primitive), one tree
// per group (robot): median split along the longest extent of the centroids'
// box (ties by primitive id), built once (Sec. II-B keeps the trees and
// refits their boxes).  Internal nodes in preorder, group after group; child
// codes >= 0 internal, < 0 leaf ~prim; parent[i] of internal node i,
// parent[n - 1 + p] of leaf p; root[g] the root code of group g (the
// minimum int for an empty group).
struct BvhHost {
  std::vector<int2> child;
  std::vector<int> parent;
  std::vector<int> root;
};
void bvh_build(const std::vector<double>& cen, int n, const int* group, int n_groups, BvhHost& out) {
  out.child.assign(std::max(n - 1, 1), make_int2(0, 0));
  out.parent.assign(std::max(2 * n - 1, 1), -1);
  out.root.assign(std::max(n_groups, 1), -2147483647 - 1);
  if (n < 1) return;
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  if (group) std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return group[a] < group[b]; });
  int next = 0;
  std::function<int(int, int, int)> build = [&](int a, int b, int par) -> int {
    if (b - a == 1) {
      out.parent[n - 1 + idx[a]] = par;
      return ~idx[a];
    }
    const int node = next++;
    out.parent[node] = par;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = a; i < b; ++i)
      for (int c = 0; c < 3; ++c) {
        lo[c] = std::min(lo[c], cen[3 * (size_t)idx[i] + c]);
        hi[c] = std::max(hi[c], cen[3 * (size_t)idx[i] + c]);
      }
    int ax = 0;
    for (int c = 1; c < 3; ++c)
      if (hi[c] - lo[c] > hi[ax] - lo[ax]) ax = c;
    const int m = a + (b - a) / 2;
    std::nth_element(idx.begin() + a, idx.begin() + m, idx.begin() + b, [&](int p, int q) {
      const double xp = cen[3 * (size_t)p + ax], xq = cen[3 * (size_t)q + ax];
      return xp < xq || (xp == xq && p < q);
    });
    const int l = build(a, m, node);
    const int r = build(m, b, node);
    out.child[node] = make_int2(l, r);
    return node;
  };
  for (int a = 0; a < n;) {
    const int g = group ? group[idx[a]] : 0;
    int b = a + 1;
    while (b < n && (group ? group[idx[b]] : 0) == g) ++b;
    out.root[g] = build(a, b, -1);
    a = b;
  }
}

// Boundary faces of a tet mesh: faces of exactly one tet, oriented outward
// (face k of a tet is opposite its local vertex k), ordered by (tet, k), as
// (v0, v1, v2, owning tet).
void boundary_faces4(const int32_t* tets, int n_t, std::vector<int>& faces4) {
  faces4.clear();
  std::vector<std::array<int, 4>> keys(4 * (size_t)n_t);
  for (int e = 0; e < n_t; ++e)
    for (int k = 0; k < 4; ++k) {
      int t3[3] = {tets[4 * e + kTetFace[k][0]], tets[4 * e + kTetFace[k][1]], tets[4 * e + kTetFace[k][2]]};
      std::sort(t3, t3 + 3);
      keys[4 * (size_t)e + k] = {t3[0], t3[1], t3[2], 4 * e + k};
    }
  std::sort(keys.begin(), keys.end());
  std::vector<char> once(4 * (size_t)n_t, 0);
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j][0] == keys[i][0] && keys[j][1] == keys[i][1] && keys[j][2] == keys[i][2]) ++j;
    if (j - i == 1) once[keys[i][3]] = 1;
    i = j;
  }
  for (int id = 0; id < 4 * n_t; ++id)
    if (once[id]) {
      const int e = id / 4, k = id % 4;
      faces4.push_back(tets[4 * e + kTetFace[k][0]]);
      faces4.push_back(tets[4 * e + kTetFace[k][1]]);
      faces4.push_back(tets[4 * e + kTetFace[k][2]]);
      faces4.push_back(e);
    }
}

// In-place inverse of the SPD n x n matrix A (row-major) by its Cholesky
// factor L (A = L L^T, A^-1 = L^-T L^-1); false if a pivot is not positive.
bool cholesky_inverse(std::vector<double>& A, int n) {
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double dsum = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) dsum -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(dsum > 0.0)) return false;
    const double ljj = std::sqrt(dsum);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / ljj;
    }
  }
  // columns of L^-1 by forward substitution, then A^-1 = L^-T L^-1
  std::vector<double> Li((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    for (int i = c; i < n; ++i) {
      double t = i == c ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) t -= L[(size_t)i * n + k] * Li[(size_t)k * n + c];
      Li[(size_t)i * n + c] = t / L[(size_t)i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) {
      double t = 0.0;
      for (int k = i; k < n; ++k) t += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
      A[(size_t)i * n + j] = A[(size_t)j * n + i] = t;
    }
  return true;
}

}  // namespace

namespace casim {
void set_handle_free_error(const char* msg) { g_create_error = msg ? msg : ""; }
const char* handle_free_error() { return g_create_error.c_str(); }
}  // namespace casim

// Device buffers of the Anderson-accelerated loop (allocated on first use,
// for memory up to m_cap): positions x_k and the proposal (all vertices), the
// residual and previous residual / image, the history rings dF, dG, and small
// tables for the dot and combine kernels.
struct AAState {
  int m_cap = 0;
  void *x = nullptr, *xa = nullptr, *f = nullptr, *fprev = nullptr, *gprev = nullptr;
  std::vector<void*> dF, dG;
  void** vec_tab = nullptr;
  void** dg_tab = nullptr;
  int* pairs = nullptr;
  double* theta = nullptr;
  double* partials = nullptr;
};

struct casim_sim {
  casim_params params{};
  std::vector<double> knots;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  // graph capture only: the local step's branch, forked from and joined back
  // into cap_stream
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
  int device = 0;
  bool has_mesh = false;
  bool has_act = false;
  // host-side mesh
  int n_v = 0, n_t = 0, n_free = 0, n_q = 0, n_f = 0, n_groups = 0, n_spheres = 0;
  int n_qf = 0;  // incidences (query vertex, boundary face)
  std::vector<int> int_of_user, user_of_int;
  std::vector<double> omega;
  std::vector<int> q_verts;  // internal ids
  std::vector<int> fx_ptr, fx_col;
  std::vector<double> fx_val;
  std::vector<double> X_fixed;  // internal order of fixed vertices, 3 per vertex
  std::vector<double> spheres;
  // device memory
  std::vector<void*> allocs;
  size_t rs = 4;  // bytes per real
  void *X = nullptr, *Tc = nullptr, *tinfo = nullptr, *P = nullptr, *cbrt_alpha = nullptr;
  void *diagL = nullptr, *bfix = nullptr, *b = nullptr, *diag = nullptr, *sl_val = nullptr;
  void *r = nullptr, *u = nullptr, *p = nullptr, *s = nullptr, *w = nullptr, *dx = nullptr, *spring_c = nullptr;
  void* pos_out = nullptr;
  void* X0 = nullptr;  // positions restored by casim_reset
  void* xstep = nullptr;  // the last outer iteration's step per free row (MIXED warm start of the dataflow and batch PCG)
  int4 *tet = nullptr, *faces = nullptr;
  int *inc_ptr = nullptr, *inc = nullptr, *sl_ptr = nullptr, *sl_col = nullptr;
  int *q_verts_d = nullptr, *qf_ptr = nullptr, *qf = nullptr;
  int *cell_count = nullptr, *cell_start = nullptr, *cell_cursor = nullptr, *items = nullptr;
  int *pair_count = nullptr, *pair_tet = nullptr, *obs_sphere = nullptr, *int_of_user_d = nullptr;
  int* cast_list = nullptr;
  double* cast_nrm = nullptr;
  double *knots_d = nullptr, *spheres_d = nullptr, *partials = nullptr, *e_partials = nullptr;
  float* spheres_fd = nullptr;
  SpringDev sp{};
  Ctrl* ctrl = nullptr;
  IterRec* hist = nullptr;
  int hist_cap = 4096;
  CollisionScratch cs{};
  unsigned H_t = 0, H_f = 0;
  int cap_items = 0, n_slices = 0, pcg_grid = 1, n_e_local = 0, n_e_spring = 0;
  bool pcg_rr = false;  // register-resident PCG (one row per thread)
  bool pcg_cl = false;  // cluster PCG (one cluster per robot, work queue)
  int pcg_variant = 1;  // whole-grid kernel: 1 streaming, 2 register-resident, 5 dataflow
  unsigned long long *df_u = nullptr, *df_p = nullptr;  // dataflow PCG: epoch-tagged words
  int *halo_ptr = nullptr, *halo_rows = nullptr, *sl_lcol = nullptr;  // dataflow PCG: block halos
  int *halo_own = nullptr, *halo_self = nullptr;
  std::vector<int> halo_ptr_h, halo_rows_h, sl_lcol_h, halo_own_h, halo_self_h;
  int halo_max = 0;
  int df_rows = 384;  // rows per block of the dataflow PCG
  std::vector<float> cg_ainv_h;  // dataflow PCG coarse correction: A_c^-1, row-major
  int n_agg = 0;
  float* cg_ainv = nullptr;
  bool pcg_seg = false; // segmented streaming PCG (batches: blocks per robot)
  int seg_blocks = 0;
  std::vector<int> seg_h;  // 5 x seg_blocks: lo, hi, rb0, rb1, robot
  int* seg_d = nullptr;
  // segmented PCG coarse correction (per robot): aggregate offsets, inverse
  // offsets, the inverses (FP32), and the per-aggregate sums exchanged
  bool seg_coarse = false;
  std::vector<int> seg_agg_base_h;
  std::vector<long long> seg_ainv_off_h;
  std::vector<float> seg_ainv_h;
  int* seg_agg_base = nullptr;
  long long* seg_ainv_off = nullptr;
  float* seg_ainv = nullptr;
  float* seg_aggsum = nullptr;
  int pcg_clusters = 0, cl_rows_cap = 0, n_robots = 1;
  // AABB trees (broad phase 1) of the robot's tets and boundary faces
  BvhHost bvh_t_h, bvh_f_h;
  BvhDev bt{}, bf{};
  int* obs_mesh = nullptr;  // n_q
  // rigid tetrahedral obstacle (its own allocations, replaced as a whole)
  std::vector<void*> obs_allocs;
  BvhDev ot{}, of{};
  void* OX = nullptr;
  int4* oface = nullptr;
  int n_ov = 0, n_ot = 0, n_of = 0;
  void free_obstacle() {
    for (void* q : obs_allocs) cudaFree(q);
    obs_allocs.clear();
    ot = BvhDev{};
    of = BvhDev{};
    OX = nullptr;
    oface = nullptr;
    n_ov = n_ot = n_of = 0;
  }
  int* robot_row = nullptr;
  std::vector<int> robot_row_h;
  std::vector<int> robot_of_vert_h, robot_of_tet_h, robot_of_face_h;
  int *robot_of_vert = nullptr, *robot_of_tet = nullptr, *robot_of_face = nullptr;
  // graph of one iteration
  cudaGraphExec_t gexec = nullptr;
  bool graph_dirty = true;
  bool no_graph = false;  // capture refused: launch the iteration eagerly
  long long iters = 0;
  int last_status = 0;
  int status_bits = 0;  // OR of the device status words read by casim_sync
  double phase_ms[5] = {0, 0, 0, 0, 0};
  std::vector<double> alpha_h;  // current volume ratios (host copy, for the adjoint)
  std::vector<double> rest_h;   // rest positions, internal order, FP64 (remesh trigger reference)
  std::vector<int> group_h;     // group of every tet (caller's tet order)
  double *rm_ref = nullptr, *rm_rest = nullptr, *rm_vols = nullptr;  // remesh trigger buffers (on first use)
  unsigned char* rm_flags = nullptr;
  AAState aa;                   // Anderson acceleration buffers (on first use)
  // adjoint: checkpoints of the last casim_forward_ckpt and reverse-pass buffers
  struct Adj {
    int n_iters = 0, every = 0, n_ckpt = 0, cap_ckpt = 0, cap_every = 0;
    bool valid = false;
    void* ckX = nullptr;      // n_ckpt x n_v positions
    int *ck_act = nullptr, *ck_kind = nullptr, *ck_face = nullptr;
    double *ck_bary = nullptr, *ck_tgt = nullptr;
    void* segX = nullptr;     // every x n_v positions of a recomputed segment
    int *seg_act = nullptr, *seg_kind = nullptr, *seg_face = nullptr, *seg_flag = nullptr;
    double* seg_bary = nullptr;
    void* mu = nullptr;
    R4<double>* g = nullptr;
    R4<double>* xbar_tet = nullptr;
    double *betabar = nullptr, *alpha_part = nullptr, *alpha_d = nullptr, *abar = nullptr;
    int *em_vert = nullptr, *em_cnt = nullptr, *em_start = nullptr, *em_cur = nullptr, *em_list = nullptr;
    int *em_tiles = nullptr, *em_total = nullptr;
    R4<double>* em_val = nullptr;
    int n_slots = 0;
    void* finX = nullptr;     // final forward state, restored after the reverse pass
    int *fin_act = nullptr, *fin_kind = nullptr, *fin_face = nullptr;
    double *fin_bary = nullptr, *fin_tgt = nullptr;
    std::vector<void*> allocs;
  } adj;
  void free_adj() {
    for (void* q : adj.allocs) cudaFree(q);
    adj = Adj();
  }

  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  template <class X>
  X* dalloc(size_t n) {
    void* q = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&q, n * sizeof(X)) != cudaSuccess) return nullptr;
    allocs.push_back(q);
    return static_cast<X*>(q);
  }
  void* dalloc_bytes(size_t n) {
    void* q = nullptr;
    if (n == 0) n = 16;
    if (cudaMalloc(&q, n) != cudaSuccess) return nullptr;
    allocs.push_back(q);
    return q;
  }
  void free_all() {
    free_adj();
    free_obstacle();
    bt = BvhDev{};
    bf = BvhDev{};
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    for (void* q : allocs) cudaFree(q);
    allocs.clear();
    rm_ref = rm_rest = rm_vols = nullptr;
    rm_flags = nullptr;
    aa = AAState{};
    graph_dirty = true;
  }
};

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return sim->fail(CASIM_E_CUDA, std::string(#call) + ": " + \
                                                              cudaGetErrorString(e_)); \
  } while (0)

namespace {

template <typename T>
Dev<T> make_dev(casim_sim* sim) {
  Dev<T> d{};
  d.n_v = sim->n_v;
  d.n_t = sim->n_t;
  d.n_free = sim->n_free;
  d.n_q = sim->n_q;
  d.n_f = sim->n_f;
  d.n_groups = sim->n_groups;
  d.n_spheres = sim->params.collision >= 2 ? sim->n_spheres : 0;
  d.n_knots = (int)sim->knots.size() / 2;
  d.X = (R4<T>*)sim->X;
  d.tet = sim->tet;
  d.Tc = (const R4<T>*)sim->Tc;
  d.tinfo = (const R4<T>*)sim->tinfo;
  d.P = (R4<T>*)sim->P;
  d.cbrt_alpha = (const T*)sim->cbrt_alpha;
  d.knots = sim->knots_d;
  d.inc_ptr = sim->inc_ptr;
  d.inc = sim->inc;
  d.diagL = (const T*)sim->diagL;
  d.bfix = (const R4<double>*)sim->bfix;
  d.b = (R4<double>*)sim->b;
  d.diag = (T*)sim->diag;
  d.n_slices = sim->n_slices;
  d.sl_ptr = sim->sl_ptr;
  d.sl_col = sim->sl_col;
  d.sl_val = (const T*)sim->sl_val;
  d.r = (R4<T>*)sim->r;
  d.u = (R4<T>*)sim->u;
  d.p = (R4<T>*)sim->p;
  d.s = (R4<T>*)sim->s;
  d.w = (R4<T>*)sim->w;
  d.dx = (R4<T>*)sim->dx;
  d.partials = sim->partials;
  d.df_u = sim->df_u;
  d.df_p = sim->df_p;
  d.halo_ptr = sim->halo_ptr;
  d.halo_rows = sim->halo_rows;
  d.halo_own = sim->halo_own;
  d.halo_self = sim->halo_self;
  d.sl_lcol = sim->sl_lcol;
  d.halo_max = sim->halo_max;
  d.df_rows = sim->df_rows;
  d.cg_ainv = sim->cg_ainv;
  d.n_agg = sim->n_agg;
  d.q_verts = sim->q_verts_d;
  d.qf_ptr = sim->qf_ptr;
  d.qf = sim->qf;
  d.faces = sim->faces;
  d.spheres = sim->spheres_d;
  d.spheres_f = sim->spheres_fd;
  d.H_t = sim->H_t;
  d.H_f = sim->H_f;
  d.cell_count = sim->cell_count;
  d.cell_start = sim->cell_start;
  d.cell_cursor = sim->cell_cursor;
  d.items = sim->items;
  d.cap_items = sim->cap_items;
  d.pair_count = sim->pair_count;
  d.pair_tet = sim->pair_tet;
  d.obs_sphere = sim->obs_sphere;
  d.max_pairs = sim->params.max_pairs_per_vertex;
  d.sp = sim->sp;
  d.cast_list = sim->cast_list;
  d.cast_nrm = sim->cast_nrm;
  d.spring_c = (R4<double>*)sim->spring_c;
  d.broad = sim->params.broad_phase;
  d.bt = sim->bt;
  d.bf = sim->bf;
  d.ot = sim->ot;
  d.of = sim->of;
  d.OX = (const R4<T>*)sim->OX;
  d.oface = sim->oface;
  d.n_of = sim->n_of;
  d.obs_mesh = sim->obs_mesh;
  d.k_spring = sim->params.k_spring;
  d.eps = sim->params.eps;
  d.cell = sim->params.cell_size;
  d.inv_cell = 1.0 / sim->params.cell_size;
  d.tol2 = sim->params.pcg_tol * sim->params.pcg_tol;
  d.max_iter = sim->params.pcg_max_iter;
  d.collision = sim->params.collision;
  d.stats = sim->params.stats;
  d.bar_extra = (sim->params.debug_flags & CASIM_DEBUG_BARRIER_NEVER_COMPLETES) ? 1u : 0u;
  d.n_robots = sim->n_robots;
  d.robot_of_vert = sim->robot_of_vert;
  d.robot_of_tet = sim->robot_of_tet;
  d.robot_of_face = sim->robot_of_face;
  d.seg_lo = sim->seg_d;
  d.seg_hi = sim->seg_d ? sim->seg_d + sim->seg_blocks : nullptr;
  d.seg_rb0 = sim->seg_d ? sim->seg_d + 2 * sim->seg_blocks : nullptr;
  d.seg_rb1 = sim->seg_d ? sim->seg_d + 3 * sim->seg_blocks : nullptr;
  d.seg_robot = sim->seg_d ? sim->seg_d + 4 * sim->seg_blocks : nullptr;
  d.seg_coarse = sim->seg_coarse ? 1 : 0;
  d.seg_agg_base = sim->seg_agg_base;
  d.seg_ainv_off = sim->seg_ainv_off;
  d.seg_ainv = sim->seg_ainv;
  d.seg_aggsum = sim->seg_aggsum;
  d.robot_row = sim->robot_row;
  d.cl_rows_cap = sim->cl_rows_cap;
  d.wait_budget = sim->params.wait_budget_cycles ? sim->params.wait_budget_cycles : 4000000000ull;
  d.ctrl = sim->ctrl;
  d.hist = sim->hist;
  d.hist_cap = sim->hist_cap;
  d.e_partials = sim->e_partials;
  d.local_threads = sim->params.local_block ? sim->params.local_block : LOCAL_THREADS;
  d.rhs_threads = sim->params.rhs_block ? sim->params.rhs_block : RHS_THREADS;
  d.narrow_threads = sim->params.narrow_block ? sim->params.narrow_block : 256;
  d.n_e_local = local_blocks(sim->n_t, d.local_threads);
  d.n_e_spring = rhs_blocks(sim->n_free, d.rhs_threads);
  return d;
}

// Forgets the last outer iteration's step: the next solve starts from x_i.
// Called wherever the positions are set other than by an outer iteration.
cudaError_t clear_xstep(casim_sim* sim) {
  if (!sim->xstep) return cudaSuccess;
  return cudaMemsetAsync(sim->xstep, 0, 4 * sim->rs * (size_t)std::max(sim->n_free, 1), sim->stream);
}

// The last step in caller order (n_v*3 doubles; zero for fixed vertices and
// where none is kept): out != NULL reads it from the device, else it is set
// from in.
template <typename T>
int xstep_io(casim_sim* sim, double* out, const double* in) {
  const int nf = sim->n_free;
  if (!sim->xstep || nf == 0) {
    if (out) std::fill(out, out + 3 * (size_t)sim->n_v, 0.0);
    return CASIM_OK;
  }
  std::vector<R4<T>> h(nf);
  if (out) {
    CK(cudaStreamSynchronize(sim->stream));
    CK(cudaMemcpy(h.data(), sim->xstep, sizeof(R4<T>) * nf, cudaMemcpyDeviceToHost));
    std::fill(out, out + 3 * (size_t)sim->n_v, 0.0);
    for (int i = 0; i < nf; ++i) {
      const size_t uv = (size_t)sim->user_of_int[i];
      out[3 * uv] = (double)h[i].x;
      out[3 * uv + 1] = (double)h[i].y;
      out[3 * uv + 2] = (double)h[i].z;
    }
  } else {
    for (int i = 0; i < nf; ++i) {
      const size_t uv = (size_t)sim->user_of_int[i];
      h[i] = R4<T>{(T)in[3 * uv], (T)in[3 * uv + 1], (T)in[3 * uv + 2], T(0)};
    }
    CK(cudaMemcpyAsync(sim->xstep, h.data(), sizeof(R4<T>) * nf, cudaMemcpyHostToDevice, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
  }
  return CASIM_OK;
}

// Copies the obstacle spheres to the device: the FP64 values the tests use and
// their round-to-nearest FP32 images for the reject test that precedes them.
cudaError_t upload_spheres(casim_sim* sim) {
  const int n = sim->n_spheres;
  std::vector<float> f(sim->spheres.begin(), sim->spheres.begin() + 4 * n);
  cudaError_t e = cudaMemcpy(sim->spheres_d, sim->spheres.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(sim->spheres_fd, f.data(), sizeof(float) * 4 * n, cudaMemcpyHostToDevice);
  return e;
}

// Enqueues one outer iteration on stream st (used for graph capture and for
// the timed eager path).  With a side stream (graph capture) the local step
// runs on it, concurrently with the spring update and the ray casts: it
// reads only the positions, which no collision kernel writes, and writes
// only the projections P and its energy partials, which the collision
// kernels do not read; the iteration's record takes both sides' terms by
// integer atomics.  The global solve waits for both branches.
// NVTX range for profilers (a no-op unless a tool is attached); in graph
// replay the ranges mark the capture, in eager mode every iteration.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

template <typename T>
cudaError_t enqueue_iteration(casim_sim* sim, cudaStream_t st, cudaEvent_t* ev, cudaStream_t side = nullptr) {
  NvtxRange outer("casim iteration");
  const Dev<T> d = make_dev<T>(sim);
  if (ev) cudaEventRecord(ev[0], st);
  if (d.collision >= 1 && d.n_q > 0) {
    NvtxRange r("collision check");
    launch_collision<T>(d, sim->cs, st);
  }
  if (ev) cudaEventRecord(ev[1], st);
  if (side) {
    cudaEventRecord(sim->ev_fork, st);
    cudaStreamWaitEvent(side, sim->ev_fork, 0);
    NvtxRange r("local step");
    launch_local<T>(d, side);
    cudaEventRecord(sim->ev_join, side);
  }
  if (d.collision >= 1 && d.n_q > 0) {
    NvtxRange r("spring update");
    launch_springs<T>(d, st);
  }
  if (ev) cudaEventRecord(ev[2], st);
  if (side) {
    cudaStreamWaitEvent(st, sim->ev_join, 0);
  } else {
    NvtxRange r("local step");
    launch_local<T>(d, st);
  }
  if (ev) cudaEventRecord(ev[3], st);
  // the dataflow PCG forms the right-hand side, the diagonal and the
  // iteration's record itself (one launch instead of three)
  const bool fused = !sim->pcg_seg && !sim->pcg_cl && sim->pcg_variant == 5;
  if (!fused) {
    NvtxRange r("rhs gather");
    launch_rhs<T>(d, st);
  }
  if (ev) cudaEventRecord(ev[4], st);
  NvtxRange rp("global solve");
  // reset the grid-barrier words (abort, count, generation) before the PCG
  cudaMemsetAsync(reinterpret_cast<char*>(sim->ctrl) + offsetof(Ctrl, abort), 0, 3 * sizeof(int), st);
  Dev<T> dp = d;
  dp.rhs_in_pcg = fused ? 1 : 0;
  dp.xstep = (fused || sim->pcg_seg) ? (R4<T>*)sim->xstep : nullptr;
  cudaError_t e = sim->pcg_seg  ? launch_pcg_seg<T>(dp, sim->seg_blocks, st)
                  : sim->pcg_cl ? launch_pcg_cluster<T>(d, sim->pcg_clusters, st)
                                : launch_pcg<T>(dp, sim->pcg_grid, sim->pcg_variant, st);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[5], st);
  if (!fused) launch_finalize<T>(d, st);
  return cudaGetLastError();
}

template <typename T>
void to_real(const std::vector<double>& a, std::vector<T>& out) {
  out.resize(a.size());
  for (size_t i = 0; i < a.size(); ++i) out[i] = (T)a[i];
}

template <typename T>
int upload_typed(casim_sim* sim, const std::vector<double>& rest_int, const std::vector<int>& tets_int,
                 const std::vector<int>& group, const std::vector<double>& Tc, const std::vector<double>& vol0,
                 const std::vector<double>& tt, const std::vector<int>& faces4, const std::vector<int>& qf_ptr,
                 const std::vector<int>& qf, const std::vector<int>& inc_ptr, const std::vector<int>& inc,
                 const std::vector<double>& diagL, const std::vector<int>& sl_ptr,
                 const std::vector<int>& sl_col, const std::vector<double>& sl_val) {
  const int n_v = sim->n_v, n_t = sim->n_t, n_free = sim->n_free, n_q = sim->n_q, n_f = sim->n_f;
  sim->X = sim->dalloc<R4<T>>(n_v);
  sim->X0 = sim->dalloc<R4<T>>(n_v);
  sim->pos_out = sim->dalloc<T>(3 * (size_t)n_v);
  sim->tet = sim->dalloc<int4>(n_t);
  sim->Tc = sim->dalloc<R4<T>>(3 * (size_t)n_t);
  sim->tinfo = sim->dalloc<R4<T>>(n_t);
  sim->P = sim->dalloc<R4<T>>(4 * (size_t)n_t);
  sim->cbrt_alpha = sim->dalloc<T>(std::max(1, sim->n_groups));
  sim->knots_d = sim->dalloc<double>(sim->knots.size());
  sim->inc_ptr = sim->dalloc<int>(n_free + 1);
  sim->inc = sim->dalloc<int>(inc.size());
  sim->diagL = sim->dalloc<T>(n_free);
  sim->bfix = sim->dalloc<R4<double>>(n_free);
  sim->b = sim->dalloc<R4<double>>(n_free);
  sim->diag = sim->dalloc<T>(n_free);
  sim->sl_ptr = sim->dalloc<int>(sl_ptr.size());
  sim->sl_col = sim->dalloc<int>(sl_col.size());
  sim->sl_val = sim->dalloc<T>(sl_val.size());
  sim->r = sim->dalloc<R4<T>>(n_free);
  sim->u = sim->dalloc<R4<T>>(n_free);
  sim->p = sim->dalloc<R4<T>>(n_free);
  sim->s = sim->dalloc<R4<T>>(n_free);
  sim->w = sim->dalloc<R4<T>>(n_free);
  sim->dx = sim->dalloc<R4<T>>(n_free);
  // the step that the next solve starts from (MIXED; dataflow and batch PCG)
  sim->xstep = std::is_same<T, float>::value && (sim->pcg_variant == 5 || sim->pcg_seg)
                   ? sim->dalloc<R4<T>>(std::max(n_free, 1))
                   : nullptr;
  sim->spring_c = sim->dalloc<R4<double>>(n_free);
  sim->partials = sim->dalloc<double>(2 * 4 * (size_t)std::max(sim->pcg_grid, 1));
  if (sim->pcg_variant == 5) {
    sim->df_u = sim->dalloc<unsigned long long>(4 * (size_t)std::max(n_free, 1));
    sim->df_p = sim->dalloc<unsigned long long>((size_t)PCG_DF_REPLICAS * 2 * 16 * ((size_t)sim->pcg_grid + 1));
    if (sim->n_agg > 0) sim->cg_ainv = sim->dalloc<float>((size_t)sim->n_agg * sim->n_agg);
    sim->halo_ptr = sim->dalloc<int>(sim->halo_ptr_h.size());
    sim->halo_rows = sim->dalloc<int>(std::max<size_t>(sim->halo_rows_h.size(), 1));
    sim->sl_lcol = sim->dalloc<int>(std::max<size_t>(sim->sl_lcol_h.size(), 1));
    sim->halo_own = sim->dalloc<int>(std::max<size_t>(sim->halo_own_h.size(), 1));
    sim->halo_self = sim->dalloc<int>(std::max<size_t>(sim->halo_self_h.size(), 1));
  }
  sim->q_verts_d = sim->dalloc<int>(n_q);
  sim->qf_ptr = sim->dalloc<int>(n_q + 1);
  sim->qf = sim->dalloc<int>(qf.size());
  sim->faces = sim->dalloc<int4>(n_f);
  sim->spheres_d = sim->dalloc<double>(4 * 64);
  sim->spheres_fd = sim->dalloc<float>(4 * 64);
  const size_t H = (size_t)sim->H_t + sim->H_f;
  // the count array is followed by the single-pass scan's status words and
  // ticket (8-byte aligned), which its memset zeroes as well
  sim->cell_count = sim->dalloc<int>(H + 1 + scan_lookback_extra_ints((int)H + 1));
  {
    const size_t off = ((H + 1 + 1) / 2) * 2;  // ints, rounded up to 8 bytes
    sim->cs.tile_status = reinterpret_cast<unsigned long long*>(sim->cell_count + off);
    sim->cs.ticket = reinterpret_cast<unsigned*>(sim->cs.tile_status + (scan_tiles((int)H + 1) + 1));
  }
  sim->cell_start = sim->dalloc<int>(H + 1);
  sim->cell_cursor = sim->dalloc<int>(H);
  sim->items = sim->dalloc<int>(sim->cap_items);
  sim->cs.tile_sums = sim->dalloc<int>(scan_tiles((int)H + 1) + 1);
  sim->cs.total = sim->dalloc<int>(1);
  sim->pair_count = sim->dalloc<int>(n_q);
  sim->pair_tet = sim->dalloc<int>((size_t)n_q * sim->params.max_pairs_per_vertex);
  sim->obs_sphere = sim->dalloc<int>(n_q);
  sim->obs_mesh = sim->dalloc<int>(n_q);
  auto alloc_bvh = [&](const BvhHost& h, int n, int nv, const int4* prim, BvhDev& b) {
    b = BvhDev{};
    if (sim->params.broad_phase != 1 || n <= 0) return;
    b.n = n;
    b.nv = nv;
    b.prim = prim;
    b.root = sim->dalloc<int>(h.root.size());
    b.child = sim->dalloc<int2>(std::max(n - 1, 1));
    b.parent = sim->dalloc<int>(2 * (size_t)n);
    b.lo = sim->dalloc<float4>(std::max(n - 1, 1));
    b.hi = sim->dalloc<float4>(std::max(n - 1, 1));
    b.flag = sim->dalloc<int>(std::max(n - 1, 1));
  };
  sim->sp.active = sim->dalloc<int>(n_q);
  sim->sp.kind = sim->dalloc<int>(n_q);
  sim->sp.face = sim->dalloc<int>(n_q);
  sim->sp.bary = sim->dalloc<double>(2 * (size_t)n_q);
  sim->sp.target = sim->dalloc<double>(3 * (size_t)n_q);
  sim->sp.fallback = sim->dalloc<int>(n_q);
  sim->cast_list = sim->dalloc<int>(n_q);
  sim->cast_nrm = sim->dalloc<double>(3 * (size_t)n_q);
  sim->int_of_user_d = sim->dalloc<int>(n_v);
  sim->robot_row = sim->dalloc<int>(sim->robot_row_h.size());
  sim->seg_d = sim->seg_blocks ? sim->dalloc<int>(sim->seg_h.size()) : nullptr;
  if (sim->seg_coarse) {
    sim->seg_agg_base = sim->dalloc<int>(sim->seg_agg_base_h.size());
    sim->seg_ainv_off = sim->dalloc<long long>(sim->seg_ainv_off_h.size());
    sim->seg_ainv = sim->dalloc<float>(std::max<size_t>(sim->seg_ainv_h.size(), 1));
    sim->seg_aggsum = sim->dalloc<float>(6 * (size_t)std::max(sim->seg_agg_base_h.back(), 1));
  } else {
    sim->seg_agg_base = nullptr;
    sim->seg_ainv_off = nullptr;
    sim->seg_ainv = nullptr;
    sim->seg_aggsum = nullptr;
  }
  if (sim->n_robots > 1) {
    sim->robot_of_vert = sim->dalloc<int>(n_v);
    sim->robot_of_tet = sim->dalloc<int>(n_t);
    sim->robot_of_face = sim->dalloc<int>(std::max(n_f, 1));
  } else {
    sim->robot_of_vert = sim->robot_of_tet = sim->robot_of_face = nullptr;
  }
  sim->ctrl = sim->dalloc<Ctrl>(1);
  sim->hist = sim->dalloc<IterRec>(sim->hist_cap);
  // energy partials: room for the smallest allowed block sizes
  sim->n_e_local = local_blocks(n_t, 64);
  sim->n_e_spring = rhs_blocks(n_free, 128);
  sim->e_partials = sim->dalloc<double>(sim->n_e_local + sim->n_e_spring + 1);
  alloc_bvh(sim->bvh_t_h, n_t, 4, sim->tet, sim->bt);
  alloc_bvh(sim->bvh_f_h, n_f, 3, sim->faces, sim->bf);
  for (void* q : sim->allocs)
    if (!q) return sim->fail(CASIM_E_CUDA, "cudaMalloc failed");
  if (!sim->X || !sim->items || !sim->P || !sim->e_partials || !sim->hist)
    return sim->fail(CASIM_E_CUDA, "device allocation failed");

  std::vector<R4<T>> Xh(n_v);
  for (int i = 0; i < n_v; ++i) Xh[i] = R4<T>{(T)rest_int[3 * i], (T)rest_int[3 * i + 1], (T)rest_int[3 * i + 2], T(0)};
  std::vector<int4> th(n_t);
  for (int e = 0; e < n_t; ++e) th[e] = make_int4(tets_int[4 * e], tets_int[4 * e + 1], tets_int[4 * e + 2], tets_int[4 * e + 3]);
  std::vector<R4<T>> Tch(3 * (size_t)n_t), info(n_t);
  for (int e = 0; e < n_t; ++e) {
    for (int i = 0; i < 3; ++i)
      Tch[3 * (size_t)e + i] = R4<T>{(T)Tc[12 * (size_t)e + 4 * i], (T)Tc[12 * (size_t)e + 4 * i + 1],
                                     (T)Tc[12 * (size_t)e + 4 * i + 2], (T)Tc[12 * (size_t)e + 4 * i + 3]};
    info[e] = R4<T>{(T)sim->omega[e], (T)vol0[e], (T)tt[e], (T)group[e]};
  }
  std::vector<int4> fh(n_f);
  for (int f = 0; f < n_f; ++f) fh[f] = make_int4(faces4[4 * f], faces4[4 * f + 1], faces4[4 * f + 2], faces4[4 * f + 3]);
  std::vector<T> dl, slv;
  to_real(diagL, dl);
  to_real(sl_val, slv);
  cudaStream_t st = sim->stream;
  CK(cudaMemcpyAsync(sim->X, Xh.data(), sizeof(R4<T>) * n_v, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->X0, Xh.data(), sizeof(R4<T>) * n_v, cudaMemcpyHostToDevice, st));
  if (sim->xstep) CK(cudaMemsetAsync(sim->xstep, 0, sizeof(R4<T>) * std::max(n_free, 1), st));
  CK(cudaMemcpyAsync(sim->tet, th.data(), sizeof(int4) * n_t, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->Tc, Tch.data(), sizeof(R4<T>) * 3 * (size_t)n_t, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->tinfo, info.data(), sizeof(R4<T>) * n_t, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->knots_d, sim->knots.data(), sizeof(double) * sim->knots.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->inc_ptr, inc_ptr.data(), sizeof(int) * inc_ptr.size(), cudaMemcpyHostToDevice, st));
  if (!inc.empty()) {
    if (sim->params.debug_flags & CASIM_DEBUG_CORRUPT_INCIDENCE) {
      // test-only (checked builds): one incidence entry out of range on the
      // device, which the checked gathers must catch
      std::vector<int> bad(inc);
      bad[0] = 4 * n_t + 7;
      CK(cudaMemcpyAsync(sim->inc, bad.data(), sizeof(int) * bad.size(), cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
    } else {
      CK(cudaMemcpyAsync(sim->inc, inc.data(), sizeof(int) * inc.size(), cudaMemcpyHostToDevice, st));
    }
  }
  if (!dl.empty()) CK(cudaMemcpyAsync(sim->diagL, dl.data(), sizeof(T) * dl.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->sl_ptr, sl_ptr.data(), sizeof(int) * sl_ptr.size(), cudaMemcpyHostToDevice, st));
  if (!sl_col.empty()) {
    CK(cudaMemcpyAsync(sim->sl_col, sl_col.data(), sizeof(int) * sl_col.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sim->sl_val, slv.data(), sizeof(T) * slv.size(), cudaMemcpyHostToDevice, st));
  }
  if (sim->pcg_variant == 5) {
    CK(cudaMemcpyAsync(sim->halo_ptr, sim->halo_ptr_h.data(), sizeof(int) * sim->halo_ptr_h.size(),
                       cudaMemcpyHostToDevice, st));
    if (!sim->halo_rows_h.empty())
      CK(cudaMemcpyAsync(sim->halo_rows, sim->halo_rows_h.data(), sizeof(int) * sim->halo_rows_h.size(),
                         cudaMemcpyHostToDevice, st));
    if (!sim->sl_lcol_h.empty())
      CK(cudaMemcpyAsync(sim->sl_lcol, sim->sl_lcol_h.data(), sizeof(int) * sim->sl_lcol_h.size(),
                         cudaMemcpyHostToDevice, st));
    if (!sim->halo_own_h.empty())
      CK(cudaMemcpyAsync(sim->halo_own, sim->halo_own_h.data(), sizeof(int) * sim->halo_own_h.size(),
                         cudaMemcpyHostToDevice, st));
    if (!sim->halo_self_h.empty())
      CK(cudaMemcpyAsync(sim->halo_self, sim->halo_self_h.data(), sizeof(int) * sim->halo_self_h.size(),
                         cudaMemcpyHostToDevice, st));
    if (sim->n_agg > 0)
      CK(cudaMemcpyAsync(sim->cg_ainv, sim->cg_ainv_h.data(), sizeof(float) * sim->cg_ainv_h.size(),
                         cudaMemcpyHostToDevice, st));
  }
  if (n_q) {
    CK(cudaMemcpyAsync(sim->q_verts_d, sim->q_verts.data(), sizeof(int) * n_q, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(sim->qf_ptr, qf_ptr.data(), sizeof(int) * qf_ptr.size(), cudaMemcpyHostToDevice, st));
  if (!qf.empty()) CK(cudaMemcpyAsync(sim->qf, qf.data(), sizeof(int) * qf.size(), cudaMemcpyHostToDevice, st));
  if (n_f) CK(cudaMemcpyAsync(sim->faces, fh.data(), sizeof(int4) * n_f, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->int_of_user_d, sim->int_of_user.data(), sizeof(int) * n_v, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(sim->robot_row, sim->robot_row_h.data(), sizeof(int) * sim->robot_row_h.size(), cudaMemcpyHostToDevice, st));
  if (sim->seg_blocks)
    CK(cudaMemcpyAsync(sim->seg_d, sim->seg_h.data(), sizeof(int) * sim->seg_h.size(), cudaMemcpyHostToDevice, st));
  if (sim->seg_coarse) {
    CK(cudaMemcpyAsync(sim->seg_agg_base, sim->seg_agg_base_h.data(), sizeof(int) * sim->seg_agg_base_h.size(),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sim->seg_ainv_off, sim->seg_ainv_off_h.data(),
                       sizeof(long long) * sim->seg_ainv_off_h.size(), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sim->seg_ainv, sim->seg_ainv_h.data(), sizeof(float) * sim->seg_ainv_h.size(),
                       cudaMemcpyHostToDevice, st));
  }
  if (sim->n_robots > 1) {
    CK(cudaMemcpyAsync(sim->robot_of_vert, sim->robot_of_vert_h.data(), sizeof(int) * n_v, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sim->robot_of_tet, sim->robot_of_tet_h.data(), sizeof(int) * n_t, cudaMemcpyHostToDevice, st));
    if (n_f)
      CK(cudaMemcpyAsync(sim->robot_of_face, sim->robot_of_face_h.data(), sizeof(int) * n_f, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemsetAsync(sim->spring_c, 0, sizeof(R4<double>) * std::max(n_free, 1), st));
  CK(cudaMemsetAsync(sim->sp.active, 0, sizeof(int) * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->sp.kind, 0, sizeof(int) * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->sp.face, 0xff, sizeof(int) * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->sp.bary, 0, sizeof(double) * 2 * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->sp.target, 0, sizeof(double) * 3 * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->sp.fallback, 0, sizeof(int) * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->pair_count, 0, sizeof(int) * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->obs_sphere, 0xff, sizeof(int) * std::max(n_q, 1), st));
  CK(cudaMemsetAsync(sim->obs_mesh, 0, sizeof(int) * std::max(n_q, 1), st));
  for (auto pr : {std::make_pair(&sim->bvh_t_h, &sim->bt), std::make_pair(&sim->bvh_f_h, &sim->bf)}) {
    const BvhHost& h = *pr.first;
    BvhDev& b = *pr.second;
    if (b.n >= 1) {
      CK(cudaMemcpyAsync((void*)b.child, h.child.data(), sizeof(int2) * h.child.size(), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync((void*)b.parent, h.parent.data(), sizeof(int) * h.parent.size(), cudaMemcpyHostToDevice,
                         st));
      CK(cudaMemcpyAsync((void*)b.root, h.root.data(), sizeof(int) * h.root.size(), cudaMemcpyHostToDevice, st));
    }
  }
  {
    Ctrl c0{};
    for (int j = 0; j < 3; ++j) {
      c0.box_lo[j] = 0x7FFFFFFFFFFFFFFFLL;
      c0.box_hi[j] = (long long)0x8000000000000000ULL;
    }
    CK(cudaMemcpyAsync(sim->ctrl, &c0, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  CK(cudaMemsetAsync(sim->hist, 0, sizeof(IterRec) * sim->hist_cap, st));
  CK(cudaMemsetAsync(sim->e_partials, 0, sizeof(double) * (sim->n_e_local + sim->n_e_spring + 1), st));
  CK(cudaMemsetAsync(sim->P, 0, sizeof(R4<T>) * 4 * (size_t)std::max(n_t, 1), st));
  CK(cudaStreamSynchronize(st));
  return CASIM_OK;
}

// bfix_v = sum over fixed u of A_vu x_u for every free row (constant between
// position uploads).
template <typename T>
int upload_bfix(casim_sim* sim) {
  std::vector<R4<double>> bf(std::max(sim->n_free, 1));
  for (int v = 0; v < sim->n_free; ++v) {
    double a[3] = {0, 0, 0};
    for (int k = sim->fx_ptr[v]; k < sim->fx_ptr[v + 1]; ++k) {
      const int u = sim->fx_col[k] - sim->n_free;
      for (int c = 0; c < 3; ++c) a[c] += sim->fx_val[k] * sim->X_fixed[3 * (size_t)u + c];
    }
    bf[v] = R4<double>{a[0], a[1], a[2], 0.0};
  }
  CK(cudaMemcpyAsync(sim->bfix, bf.data(), sizeof(R4<double>) * sim->n_free, cudaMemcpyHostToDevice, sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  return CASIM_OK;
}

template <typename T>
int set_positions_typed(casim_sim* sim, const double* xyz) {
  std::vector<R4<T>> Xh(sim->n_v);
  for (int uv = 0; uv < sim->n_v; ++uv) {
    const int i = sim->int_of_user[uv];
    Xh[i] = R4<T>{(T)xyz[3 * (size_t)uv], (T)xyz[3 * (size_t)uv + 1], (T)xyz[3 * (size_t)uv + 2], T(0)};
  }
  for (int i = sim->n_free; i < sim->n_v; ++i)
    for (int c = 0; c < 3; ++c) sim->X_fixed[3 * (size_t)(i - sim->n_free) + c] = (double)(&Xh[i].x)[c];
  CK(cudaMemcpyAsync(sim->X, Xh.data(), sizeof(R4<T>) * sim->n_v, cudaMemcpyHostToDevice, sim->stream));
  CK(cudaMemcpyAsync(sim->X0, Xh.data(), sizeof(R4<T>) * sim->n_v, cudaMemcpyHostToDevice, sim->stream));
  CK(clear_xstep(sim));
  return upload_bfix<T>(sim);
}

template <typename T>
int get_positions_typed(casim_sim* sim, double* host_out, void* dev_out) {
  const Dev<T> d = make_dev<T>(sim);
  launch_gather_positions<T>(d, sim->int_of_user_d, sim->n_v, (T*)sim->pos_out, sim->stream);
  CK(cudaGetLastError());
  if (dev_out)
    CK(cudaMemcpyAsync(dev_out, sim->pos_out, sizeof(T) * 3 * (size_t)sim->n_v, cudaMemcpyDeviceToDevice,
                       sim->stream));
  if (host_out) {
    std::vector<T> h(3 * (size_t)sim->n_v);
    CK(cudaMemcpyAsync(h.data(), sim->pos_out, sizeof(T) * h.size(), cudaMemcpyDeviceToHost, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));
    for (size_t i = 0; i < h.size(); ++i) host_out[i] = (double)h[i];
  }
  return CASIM_OK;
}

template <typename T>
int get_targets_typed(casim_sim* sim, double* out) {
  std::vector<R4<T>> h(4 * (size_t)sim->n_t);
  CK(cudaMemcpyAsync(h.data(), sim->P, sizeof(R4<T>) * h.size(), cudaMemcpyDeviceToHost, sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  for (int e = 0; e < sim->n_t; ++e) {
    const double om = sim->omega[e];
    for (int k = 0; k < 4; ++k) {
      const R4<T>& c = h[4 * (size_t)e + k];
      out[12 * (size_t)e + 0 * 4 + k] = (double)c.x / om;
      out[12 * (size_t)e + 1 * 4 + k] = (double)c.y / om;
      out[12 * (size_t)e + 2 * 4 + k] = (double)c.z / om;
    }
  }
  return CASIM_OK;
}

template <typename T>
int set_actuation_typed(casim_sim* sim, const std::vector<double>& alpha) {
  std::vector<T> c(std::max<size_t>(alpha.size(), 1), T(1));
  for (size_t g = 0; g < alpha.size(); ++g) c[g] = (T)std::cbrt(alpha[g]);
  CK(cudaMemcpyAsync(sim->cbrt_alpha, c.data(), sizeof(T) * c.size(), cudaMemcpyHostToDevice, sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  return CASIM_OK;
}

template <typename T>
int capture_graph(casim_sim* sim) {
  if (sim->gexec) {
    cudaGraphExecDestroy(sim->gexec);
    sim->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(sim->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_iteration<T>(sim, sim->cap_stream, nullptr, sim->side_stream);
  cudaError_t e2 = cudaStreamEndCapture(sim->cap_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return sim->fail(CASIM_E_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  }
  if (e2 != cudaSuccess) return sim->fail(CASIM_E_CUDA, std::string("end capture: ") + cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&sim->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return sim->fail(CASIM_E_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
  sim->graph_dirty = false;
  return CASIM_OK;
}

template <typename T>
int step_typed(casim_sim* sim, int n_iters) {
  if (sim->params.stats >= 2) {
    // eager launches with events between the phases (diagnostic timing)
    cudaEvent_t ev[6];
    for (auto& x : ev) CK(cudaEventCreate(&x));
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < n_iters; ++i) {
      cudaError_t e = enqueue_iteration<T>(sim, sim->stream, ev);
      if (e != cudaSuccess) return sim->fail(CASIM_E_CUDA, cudaGetErrorString(e));
      CK(cudaEventSynchronize(ev[5]));
      for (int k = 0; k < 5; ++k) {
        float ms = 0;
        cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
        acc[k] += ms;
      }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    for (int k = 0; k < 5; ++k) sim->phase_ms[k] = acc[k];
    sim->iters += n_iters;
    return CASIM_OK;
  }
  if (sim->graph_dirty && !sim->no_graph) {
    if (capture_graph<T>(sim) != CASIM_OK) {
      cudaGetLastError();
      sim->no_graph = true;
    }
  }
  if (sim->no_graph) {
    for (int i = 0; i < n_iters; ++i) {
      cudaError_t e = enqueue_iteration<T>(sim, sim->stream, nullptr);
      if (e != cudaSuccess) return sim->fail(CASIM_E_CUDA, cudaGetErrorString(e));
    }
    sim->iters += n_iters;
    return CASIM_OK;
  }
  for (int i = 0; i < n_iters; ++i) CK(cudaGraphLaunch(sim->gexec, sim->stream));
  sim->iters += n_iters;
  return CASIM_OK;
}

struct Triplet {
  int r, c;
  double v;
};

}  // namespace

// 1 in builds with -DCASIM_CHECKED (every gather index of the hot kernels
// bounds-checked on the device, failures reported as CASIM_E_BOUNDS)
#ifdef CASIM_CHECKED
static constexpr int kCheckedBuild = 1;
#else
static constexpr int kCheckedBuild = 0;
#endif

extern "C" {

void casim_default_params(casim_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->precision = CASIM_MIXED;
  p->collision = CASIM_COLLISION_SELF;
  p->k_spring = 1.0;
  p->eps = 0.005;
  p->pcg_tol = 1e-6;
  p->pcg_max_iter = 1000;
  p->n_w_knots = 0;
  p->w_knots = nullptr;
  p->cell_size = 0.5;
  p->stats = 1;
  p->max_pairs_per_vertex = 8;
  p->wait_budget_cycles = 0;
}

int casim_create(const casim_params* params, void* cuda_stream, casim_sim** out) {
  if (!params || !out) {
    g_create_error = "null argument";
    return CASIM_E_INVALID;
  }
  *out = nullptr;
  const casim_params& p = *params;
  std::string why;
  if (p.precision != CASIM_FP64 && p.precision != CASIM_MIXED) why = "precision";
  else if (p.collision < 0 || p.collision > 2) why = "collision";
  else if (!(p.k_spring >= 0.0) || !std::isfinite(p.k_spring)) why = "k_spring";
  else if (!(p.eps >= 0.0) || !std::isfinite(p.eps)) why = "eps";
  else if (!(p.pcg_tol > 0.0) || !std::isfinite(p.pcg_tol)) why = "pcg_tol";
  else if (p.pcg_max_iter < 1) why = "pcg_max_iter";
  else if (p.n_w_knots < 0 || (p.n_w_knots > 0 && !p.w_knots) || p.n_w_knots > 64) why = "w_knots";
  else if (!(p.cell_size > 0.0) || !std::isfinite(p.cell_size)) why = "cell_size";
  else if (p.max_pairs_per_vertex < 1 || p.max_pairs_per_vertex > 16) why = "max_pairs_per_vertex";
  else if (p.pcg_kernel < 0 || p.pcg_kernel > 5) why = "pcg_kernel";
  else if (p.debug_flags & ~(CASIM_DEBUG_BARRIER_NEVER_COMPLETES | (kCheckedBuild ? CASIM_DEBUG_CORRUPT_INCIDENCE : 0)))
    why = "debug_flags";
  else if (p.pcg_precond < 0 || p.pcg_precond > 1) why = "pcg_precond";
  else if (p.broad_phase < 0 || p.broad_phase > 1) why = "broad_phase";
  else if (p.pcg_block != 0 && p.pcg_block != 288 && p.pcg_block != 384) why = "pcg_block";
  else if (p.local_block != 0 && p.local_block != 64 && p.local_block != 128 && p.local_block != 256)
    why = "local_block";
  else if (p.rhs_block != 0 && p.rhs_block != 128 && p.rhs_block != 256 && p.rhs_block != 512) why = "rhs_block";
  else if (p.narrow_block != 0 && p.narrow_block != 128 && p.narrow_block != 256 && p.narrow_block != 512)
    why = "narrow_block";
  if (why.empty() && p.n_w_knots > 1) {
    for (int i = 0; i + 1 < p.n_w_knots; ++i)
      if (!(p.w_knots[2 * i + 2] > p.w_knots[2 * i])) why = "w_knots must be strictly ascending";
  }
  if (!why.empty()) {
    g_create_error = "invalid parameter: " + why;
    return CASIM_E_INVALID;
  }
  casim_sim* sim = new (std::nothrow) casim_sim();
  if (!sim) {
    g_create_error = "out of host memory";
    return CASIM_E_INVALID;
  }
  sim->params = p;
  if (p.n_w_knots > 0)
    sim->knots.assign(p.w_knots, p.w_knots + 2 * p.n_w_knots);
  else
    sim->knots = {0.0, 1.0};
  sim->params.w_knots = nullptr;
  sim->params.n_w_knots = (int)sim->knots.size() / 2;
  sim->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&sim->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sim->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sim->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sim->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&sim->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    g_create_error = "CUDA unavailable";
    if (sim->cap_stream) cudaStreamDestroy(sim->cap_stream);
    if (sim->side_stream) cudaStreamDestroy(sim->side_stream);
    if (sim->ev_fork) cudaEventDestroy(sim->ev_fork);
    delete sim;
    return CASIM_E_CUDA;
  }
  *out = sim;
  return CASIM_OK;
}

}  // extern "C"


// ---- adjoint: checkpointed forward and reverse pass ------------------------
namespace {

template <class X>
X* adj_alloc(casim_sim* sim, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, (n ? n : 1) * sizeof(X)) != cudaSuccess) return nullptr;
  sim->adj.allocs.push_back(q);
  return static_cast<X*>(q);
}

template <typename T>
int adj_reserve(casim_sim* sim, int n_ckpt, int every) {
  auto& A = sim->adj;
  if (A.allocs.size() && A.cap_ckpt >= n_ckpt && A.cap_every >= every) return CASIM_OK;
  sim->free_adj();
  const size_t nv = sim->n_v, nq = std::max(sim->n_q, 1), nt = sim->n_t, nf = std::max(sim->n_free, 1);
  const int ng = std::max(sim->n_groups, 1);
  A.ckX = adj_alloc<R4<T>>(sim, (size_t)n_ckpt * nv);
  A.ck_act = adj_alloc<int>(sim, (size_t)n_ckpt * nq);
  A.ck_kind = adj_alloc<int>(sim, (size_t)n_ckpt * nq);
  A.ck_face = adj_alloc<int>(sim, (size_t)n_ckpt * nq);
  A.ck_bary = adj_alloc<double>(sim, (size_t)n_ckpt * 2 * nq);
  A.ck_tgt = adj_alloc<double>(sim, (size_t)n_ckpt * 3 * nq);
  A.segX = adj_alloc<R4<T>>(sim, (size_t)every * nv);
  A.seg_act = adj_alloc<int>(sim, (size_t)every * nq);
  A.seg_kind = adj_alloc<int>(sim, (size_t)every * nq);
  A.seg_face = adj_alloc<int>(sim, (size_t)every * nq);
  A.seg_flag = adj_alloc<int>(sim, (size_t)every * nq);
  A.seg_bary = adj_alloc<double>(sim, (size_t)every * 2 * nq);
  A.mu = adj_alloc<R4<T>>(sim, nf);
  A.g = adj_alloc<R4<double>>(sim, nf);
  A.xbar_tet = adj_alloc<R4<double>>(sim, 4 * nt);
  A.n_slots = 4 * sim->n_q + 3 * sim->n_qf;
  const size_t ns = std::max(A.n_slots, 1);
  A.em_vert = adj_alloc<int>(sim, ns);
  A.em_val = adj_alloc<R4<double>>(sim, ns);
  A.em_list = adj_alloc<int>(sim, ns);
  A.em_cnt = adj_alloc<int>(sim, nf + 1);
  A.em_start = adj_alloc<int>(sim, nf + 1);
  A.em_cur = adj_alloc<int>(sim, nf + 1);
  A.em_tiles = adj_alloc<int>(sim, scan_tiles((int)nf + 1) + 1);
  A.em_total = adj_alloc<int>(sim, 1);
  A.betabar = adj_alloc<double>(sim, 2 * nq);
  A.alpha_part = adj_alloc<double>(sim, (size_t)local_blocks(sim->n_t) * ng);
  A.alpha_d = adj_alloc<double>(sim, ng);
  A.abar = adj_alloc<double>(sim, ng);
  A.finX = adj_alloc<R4<T>>(sim, nv);
  A.fin_act = adj_alloc<int>(sim, nq);
  A.fin_kind = adj_alloc<int>(sim, nq);
  A.fin_face = adj_alloc<int>(sim, nq);
  A.fin_bary = adj_alloc<double>(sim, 2 * nq);
  A.fin_tgt = adj_alloc<double>(sim, 3 * nq);
  for (void* q : A.allocs)
    if (!q) {
      sim->free_adj();
      return sim->fail(CASIM_E_CUDA, "cudaMalloc failed (adjoint buffers)");
    }
  A.cap_ckpt = n_ckpt;
  A.cap_every = every;
  return CASIM_OK;
}

// copies (positions, spring records) between the live state and a slot
template <typename T>
cudaError_t adj_copy_state(casim_sim* sim, void* X, int* act, int* kind, int* face, double* bary, double* tgt,
                           bool save) {
  const size_t nv = sim->n_v, nq = sim->n_q;
  cudaStream_t st = sim->stream;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
  };
  cudaError_t e = save ? cp(X, sim->X, sizeof(R4<T>) * nv) : cp(sim->X, X, sizeof(R4<T>) * nv);
  if (e || nq == 0) return e;
  if (save) {
    if ((e = cp(act, sim->sp.active, sizeof(int) * nq))) return e;
    if ((e = cp(kind, sim->sp.kind, sizeof(int) * nq))) return e;
    if ((e = cp(face, sim->sp.face, sizeof(int) * nq))) return e;
    if ((e = cp(bary, sim->sp.bary, sizeof(double) * 2 * nq))) return e;
    if (tgt) e = cp(tgt, sim->sp.target, sizeof(double) * 3 * nq);
  } else {
    if ((e = cp(sim->sp.active, act, sizeof(int) * nq))) return e;
    if ((e = cp(sim->sp.kind, kind, sizeof(int) * nq))) return e;
    if ((e = cp(sim->sp.face, face, sizeof(int) * nq))) return e;
    if ((e = cp(sim->sp.bary, bary, sizeof(double) * 2 * nq))) return e;
    if (tgt) e = cp(sim->sp.target, tgt, sizeof(double) * 3 * nq);
  }
  return e;
}

template <typename T>
int forward_ckpt_typed(casim_sim* sim, int n_iters, int every) {
  const int n_ckpt = (n_iters + every - 1) / every;
  int rc = adj_reserve<T>(sim, n_ckpt, every);
  if (rc) return rc;
  auto& A = sim->adj;
  const size_t nv = sim->n_v, nq = std::max(sim->n_q, 1);
  int done = 0;
  for (int c = 0; c < n_ckpt; ++c) {
    CK((adj_copy_state<T>(sim, (R4<T>*)A.ckX + c * nv, A.ck_act + c * nq, A.ck_kind + c * nq, A.ck_face + c * nq,
                          A.ck_bary + c * 2 * nq, A.ck_tgt + c * 3 * nq, true)));
    // every solve of the adjoint's forward pass starts from x_i, so that the
    // map x_i -> x_(i+1) (and its recomputation in the backward pass) does
    // not depend on where the checkpoints fall
    const int m = std::min(every, n_iters - done);
    for (int j = 0; j < m; ++j) {
      CK(clear_xstep(sim));
      rc = step_typed<T>(sim, 1);
      if (rc) return rc;
    }
    done += m;
  }
  CK((adj_copy_state<T>(sim, A.finX, A.fin_act, A.fin_kind, A.fin_face, A.fin_bary, A.fin_tgt, true)));
  A.n_iters = n_iters;
  A.every = every;
  A.n_ckpt = n_ckpt;
  A.valid = true;
  return CASIM_OK;
}

template <typename T>
int backward_typed(casim_sim* sim, const double* dL_dX, double* dL_dalpha) {
  auto& A = sim->adj;
  cudaStream_t st = sim->stream;
  const size_t nv = sim->n_v, nq = std::max(sim->n_q, 1);
  const int nf = sim->n_free, ng = sim->n_groups;
  // g = dL/dX_n on the free rows (internal order)
  std::vector<R4<double>> gh(std::max(nf, 1));
  for (int uv = 0; uv < sim->n_v; ++uv) {
    const int i = sim->int_of_user[uv];
    if (i < nf) gh[i] = R4<double>{dL_dX[3 * (size_t)uv], dL_dX[3 * (size_t)uv + 1], dL_dX[3 * (size_t)uv + 2], 0.0};
  }
  CK(cudaMemcpyAsync(A.g, gh.data(), sizeof(R4<double>) * std::max(nf, 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(A.abar, 0, sizeof(double) * std::max(ng, 1), st));
  CK(cudaMemsetAsync(A.betabar, 0, sizeof(double) * 2 * nq, st));
  if (ng) CK(cudaMemcpyAsync(A.alpha_d, sim->alpha_h.data(), sizeof(double) * ng, cudaMemcpyHostToDevice, st));
  // keep the history counters of the forward pass
  Ctrl saved;
  CK(cudaMemcpyAsync(&saved, sim->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  Dev<T> d = make_dev<T>(sim);
  Dev<T> dpcg = d;
  dpcg.X = (R4<T>*)A.mu;
  dpcg.b = A.g;
  for (int c = A.n_ckpt - 1; c >= 0; --c) {
    const int first = c * A.every;
    const int m = std::min(A.every, A.n_iters - first);
    CK((adj_copy_state<T>(sim, (R4<T>*)A.ckX + c * nv, A.ck_act + c * nq, A.ck_kind + c * nq, A.ck_face + c * nq,
                          A.ck_bary + c * 2 * nq, A.ck_tgt + c * 3 * nq, false)));
    // recompute the segment, keeping X_i and the spring decisions of each iteration
    for (int j = 0; j < m; ++j) {
      CK(cudaMemcpyAsync((R4<T>*)A.segX + j * nv, sim->X, sizeof(R4<T>) * nv, cudaMemcpyDeviceToDevice, st));
      CK(clear_xstep(sim));
      int rc = step_typed<T>(sim, 1);
      if (rc) return rc;
      if (sim->n_q) {
        CK(cudaMemcpyAsync(A.seg_act + j * nq, sim->sp.active, sizeof(int) * nq, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(A.seg_kind + j * nq, sim->sp.kind, sizeof(int) * nq, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(A.seg_face + j * nq, sim->sp.face, sizeof(int) * nq, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(A.seg_bary + j * 2 * nq, sim->sp.bary, sizeof(double) * 2 * nq, cudaMemcpyDeviceToDevice,
                           st));
        launch_adjoint_flags<T>(d, A.seg_flag + j * nq, st);
      } else {
        CK(cudaMemsetAsync(A.seg_act + j * nq, 0, sizeof(int) * nq, st));
      }
    }
    // reverse through the segment
    for (int j = m - 1; j >= 0; --j) {
      AdjDev<T> a{};
      a.Xi = (const R4<T>*)A.segX + j * nv;
      a.mu = (const R4<T>*)A.mu;
      a.sp_active = A.seg_act + j * nq;
      a.sp_kind = A.seg_kind + j * nq;
      a.sp_face = A.seg_face + j * nq;
      a.sp_bary = A.seg_bary + j * 2 * nq;
      a.sp_flag = A.seg_flag + j * nq;
      a.xbar_tet = A.xbar_tet;
      a.em_vert = A.em_vert;
      a.em_val = A.em_val;
      a.em_cnt = A.em_cnt;
      a.em_start = A.em_start;
      a.em_cur = A.em_cur;
      a.em_list = A.em_list;
      a.em_tiles = A.em_tiles;
      a.em_total = A.em_total;
      a.n_slots = (sim->params.collision == 0 || sim->n_q == 0) ? 0 : A.n_slots;
      a.betabar = A.betabar;
      a.alpha_part = A.alpha_part;
      a.alpha = A.alpha_d;
      a.abar = A.abar;
      a.g = A.g;
      a.n_groups = ng;
      if (sim->params.collision == 0 || sim->n_q == 0) {
        CK(cudaMemsetAsync(A.seg_act + j * nq, 0, sizeof(int) * nq, st));
      }
      launch_adjoint_diag<T>(d, a, st);
      CK(cudaMemsetAsync(A.mu, 0, sizeof(R4<T>) * std::max(nf, 1), st));
      CK(cudaMemsetAsync(reinterpret_cast<char*>(sim->ctrl) + offsetof(Ctrl, abort), 0, 3 * sizeof(int), st));
      cudaError_t e = sim->pcg_seg  ? launch_pcg_seg<T>(dpcg, sim->seg_blocks, st)
                      : sim->pcg_cl ? launch_pcg_cluster<T>(dpcg, sim->pcg_clusters, st)
                                    : launch_pcg<T>(dpcg, sim->pcg_grid, sim->pcg_variant, st);
      if (e != cudaSuccess) return sim->fail(CASIM_E_CUDA, std::string("adjoint solve: ") + cudaGetErrorString(e));
      launch_adjoint_step<T>(d, a, st);
      CK(cudaGetLastError());
    }
  }
  std::vector<double> ab(std::max(ng, 1));
  if (ng) CK(cudaMemcpyAsync(ab.data(), A.abar, sizeof(double) * ng, cudaMemcpyDeviceToHost, st));
  // restore the final forward state and the counters
  CK((adj_copy_state<T>(sim, A.finX, A.fin_act, A.fin_kind, A.fin_face, A.fin_bary, A.fin_tgt, false)));
  int st_bits = 0;
  CK(cudaMemcpyAsync(&st_bits, &sim->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  saved.status |= st_bits;
  CK(cudaMemcpy(sim->ctrl, &saved, sizeof(Ctrl), cudaMemcpyHostToDevice));
  // the recomputation used the history slots from here on: clear the next one
  CK(cudaMemset(sim->hist + (saved.iter % sim->hist_cap), 0, sizeof(IterRec)));
  for (int gi = 0; gi < ng; ++gi) dL_dalpha[gi] = ab[gi];
  if (st_bits & (ST_TIMEOUT | ST_NONFINITE)) return sim->fail(CASIM_E_NONFINITE, "adjoint pass: device status");
  return CASIM_OK;
}

}  // namespace

// Upload of R >= 1 independent robots given as one concatenated mesh
// (robot_of_tet says which robot each tet belongs to; robots share no vertex).
static int upload_robots(casim_sim* sim, int32_t n_verts, const double* rest_xyz, int32_t n_tets, const int32_t* tets,
                         const int32_t* tet_group, const uint8_t* fixed, int n_robots, const int* robot_of_tet) {
  if (!sim) return CASIM_E_INVALID;
  if (n_verts <= 0 || n_tets <= 0 || !rest_xyz || !tets || !tet_group || !fixed)
    return sim->fail(CASIM_E_INVALID, "empty mesh or null pointer");
  for (long long i = 0; i < 3LL * n_verts; ++i)
    if (!std::isfinite(rest_xyz[i])) return sim->fail(CASIM_E_INVALID, "non-finite rest position");
  int max_group = -1;
  for (int e = 0; e < n_tets; ++e) {
    for (int k = 0; k < 4; ++k)
      if (tets[4 * e + k] < 0 || tets[4 * e + k] >= n_verts)
        return sim->fail(CASIM_E_INVALID, "tet vertex id out of range at tet " + std::to_string(e));
    for (int k = 0; k < 4; ++k)
      for (int j = k + 1; j < 4; ++j)
        if (tets[4 * e + k] == tets[4 * e + j])
          return sim->fail(CASIM_E_INVALID, "repeated vertex in tet " + std::to_string(e));
    if (tet_group[e] < -1) return sim->fail(CASIM_E_INVALID, "group id < -1");
    max_group = std::max(max_group, (int)tet_group[e]);
  }
  sim->free_all();
  sim->has_mesh = false;
  sim->has_act = false;
  const int n_v = n_verts, n_t = n_tets;
  // ---- rest element quantities (FP64) ----
  std::vector<double> Tc(12 * (size_t)n_t), vol0(n_t), tt(n_t);
  double vsum = 0.0;
  for (int e = 0; e < n_t; ++e) {
    double V[3][4];
    for (int k = 0; k < 4; ++k)
      for (int i = 0; i < 3; ++i) V[i][k] = rest_xyz[3 * (size_t)tets[4 * e + k] + i];
    const double a0 = V[0][1] - V[0][0], a1 = V[1][1] - V[1][0], a2 = V[2][1] - V[2][0];
    const double b0 = V[0][2] - V[0][0], b1 = V[1][2] - V[1][0], b2 = V[2][2] - V[2][0];
    const double c0 = V[0][3] - V[0][0], c1 = V[1][3] - V[1][0], c2 = V[2][3] - V[2][0];
    const double vol = (a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0)) / 6.0;
    if (!(vol > 0.0)) return sim->fail(CASIM_E_INVALID, "non-positive rest volume at tet " + std::to_string(e));
    vol0[e] = vol;
    vsum += vol;
    double s2 = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double m = 0.25 * (V[i][0] + V[i][1] + V[i][2] + V[i][3]);
      for (int k = 0; k < 4; ++k) {
        const double c = V[i][k] - m;
        Tc[12 * (size_t)e + 4 * i + k] = c;
        s2 += c * c;
      }
    }
    tt[e] = s2;
  }
  (void)vsum;
  // omega_e = Vol(e) / mean Vol over the tet's own robot
  std::vector<double> rsum(n_robots, 0.0);
  std::vector<long long> rcnt(n_robots, 0);
  for (int e = 0; e < n_t; ++e) {
    rsum[robot_of_tet[e]] += vol0[e];
    rcnt[robot_of_tet[e]] += 1;
  }
  sim->omega.resize(n_t);
  for (int e = 0; e < n_t; ++e) sim->omega[e] = vol0[e] / (rsum[robot_of_tet[e]] / rcnt[robot_of_tet[e]]);
  // robot of every vertex (from its tets; robots must not share vertices)
  std::vector<int> robot_of_vert_user(n_v, -1);
  for (int e = 0; e < n_t; ++e)
    for (int k = 0; k < 4; ++k) {
      int& rv = robot_of_vert_user[tets[4 * e + k]];
      if (rv >= 0 && rv != robot_of_tet[e]) return sim->fail(CASIM_E_INVALID, "robots share a vertex");
      rv = robot_of_tet[e];
    }
  // ---- connected components must each hold a fixed vertex ----
  {
    std::vector<int> parent(n_v);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int x) {
      while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
      }
      return x;
    };
    std::vector<char> used(n_v, 0);
    for (int e = 0; e < n_t; ++e) {
      for (int k = 0; k < 4; ++k) used[tets[4 * e + k]] = 1;
      const int a = find(tets[4 * e]);
      for (int k = 1; k < 4; ++k) {
        const int b = find(tets[4 * e + k]);
        if (a != b) parent[b] = a;
      }
    }
    std::vector<char> has_fixed(n_v, 0);
    for (int v = 0; v < n_v; ++v)
      if (fixed[v]) has_fixed[find(v)] = 1;
    for (int v = 0; v < n_v; ++v) {
      if (!used[v] && !fixed[v])
        return sim->fail(CASIM_E_SINGULAR, "free vertex " + std::to_string(v) + " belongs to no tet");
      if (used[v] && !has_fixed[find(v)])
        return sim->fail(CASIM_E_SINGULAR, "component of vertex " + std::to_string(v) + " has no fixed vertex");
    }
  }
  // ---- internal numbering: free vertices first, robot by robot, each
  // robot's free vertices in recursive-coordinate-bisection order of their
  // rest positions (so that consecutive rows, and with them the PCG's thread
  // blocks and coarse aggregates, are compact pieces of the body); then the
  // fixed vertices in the caller's order ----
  sim->n_v = n_v;
  sim->n_t = n_t;
  sim->int_of_user.assign(n_v, -1);
  sim->user_of_int.assign(n_v, -1);
  int nf = 0;
  {
    // rows per block of the dataflow PCG (single robot, MIXED): 288 (9 warps,
    // more blocks, fewer rows each) when the system fits 152 such blocks,
    // else 384; the bisection leaves are its aggregates (a third of a block)
    int n_free_all = 0;
    for (int v = 0; v < n_v; ++v) n_free_all += !fixed[v];
    const int pb = sim->params.pcg_block;
    sim->df_rows = (pb == PCG_DF_THREADS || (pb == 0 && n_free_all > pcg_df_max_rows(PCG_DF_ROWS_SMALL)))
                       ? PCG_DF_THREADS
                       : PCG_DF_ROWS_SMALL;
    const int leaf = n_robots == 1 ? sim->df_rows / 3 : 128;
    std::vector<std::vector<int>> per_robot(n_robots);
    for (int v = 0; v < n_v; ++v)
      if (!fixed[v]) per_robot[std::max(0, robot_of_vert_user[v])].push_back(v);
    for (int r = 0; r < n_robots; ++r) {
      std::vector<int>& L = per_robot[r];
      rcb_order(rest_xyz, L.data(), (int)L.size(), leaf);
      for (int v : L) sim->int_of_user[v] = nf++;
    }
  }
  sim->n_free = nf;
  int nx = nf;
  for (int v = 0; v < n_v; ++v)
    if (fixed[v]) sim->int_of_user[v] = nx++;
  for (int v = 0; v < n_v; ++v) sim->user_of_int[sim->int_of_user[v]] = v;
  const int n_free = nf;
  // free rows of each robot are contiguous (robots occupy increasing id ranges)
  sim->n_robots = n_robots;
  sim->robot_row_h.assign(n_robots + 1, 0);
  {
    int prev = 0;
    for (int i = 0; i < n_free; ++i) {
      int r = robot_of_vert_user[sim->user_of_int[i]];
      if (r < 0) r = prev;
      if (r < prev) return sim->fail(CASIM_E_INVALID, "robot vertex ranges must be contiguous and ascending");
      prev = r;
      sim->robot_row_h[r + 1]++;
    }
    for (int r = 0; r < n_robots; ++r) sim->robot_row_h[r + 1] += sim->robot_row_h[r];
  }
  sim->robot_of_vert_h.assign(n_v, 0);
  for (int v = 0; v < n_v; ++v) sim->robot_of_vert_h[sim->int_of_user[v]] = std::max(0, robot_of_vert_user[v]);
  sim->robot_of_tet_h.assign(robot_of_tet, robot_of_tet + n_t);
  std::vector<int> tets_int(4 * (size_t)n_t);
  for (size_t i = 0; i < tets_int.size(); ++i) tets_int[i] = sim->int_of_user[tets[i]];
  std::vector<int> group(tet_group, tet_group + n_t);
  sim->n_groups = max_group + 1;
  std::vector<double> rest_int(3 * (size_t)n_v);
  for (int v = 0; v < n_v; ++v)
    for (int c = 0; c < 3; ++c) rest_int[3 * (size_t)sim->int_of_user[v] + c] = rest_xyz[3 * (size_t)v + c];
  sim->rest_h = rest_int;
  sim->group_h = group;
  sim->X_fixed.assign(3 * (size_t)(n_v - n_free), 0.0);
  for (int i = n_free; i < n_v; ++i)
    for (int c = 0; c < 3; ++c) sim->X_fixed[3 * (size_t)(i - n_free) + c] = rest_int[3 * (size_t)i + c];
  // ---- boundary faces: faces of exactly one tet, ordered by (tet, k) ----
  std::vector<int> faces4;
  boundary_faces4(tets, n_t, faces4);
  for (size_t i = 0; i < faces4.size(); i += 4)
    for (int k = 0; k < 3; ++k) faces4[i + k] = sim->int_of_user[faces4[i + k]];
  sim->n_f = (int)(faces4.size() / 4);
  sim->robot_of_face_h.resize(sim->n_f);
  for (int f = 0; f < sim->n_f; ++f) sim->robot_of_face_h[f] = robot_of_tet[faces4[4 * f + 3]];
  // ---- query vertices (non-fixed boundary vertices) and incident faces ----
  std::vector<char> on_surf(n_v, 0);
  for (int f = 0; f < sim->n_f; ++f)
    for (int k = 0; k < 3; ++k) on_surf[faces4[4 * f + k]] = 1;
  // (listed in ascending caller vertex id, so that contacts and spring
  // records come out in the caller's order)
  sim->q_verts.clear();
  std::vector<int> qidx(n_v, -1);
  for (int uv = 0; uv < n_v; ++uv) {
    const int i = sim->int_of_user[uv];
    if (i < n_free && on_surf[i]) {
      qidx[i] = (int)sim->q_verts.size();
      sim->q_verts.push_back(i);
    }
  }
  sim->n_q = (int)sim->q_verts.size();
  std::vector<int> qf_ptr(sim->n_q + 1, 0), qf;
  for (int f = 0; f < sim->n_f; ++f)
    for (int k = 0; k < 3; ++k)
      if (qidx[faces4[4 * f + k]] >= 0) qf_ptr[qidx[faces4[4 * f + k]] + 1]++;
  for (int q = 0; q < sim->n_q; ++q) qf_ptr[q + 1] += qf_ptr[q];
  qf.assign(qf_ptr[sim->n_q], 0);
  sim->n_qf = qf_ptr[sim->n_q];
  {
    std::vector<int> cur(qf_ptr.begin(), qf_ptr.end() - 1);
    for (int f = 0; f < sim->n_f; ++f)
      for (int k = 0; k < 3; ++k) {
        const int q = qidx[faces4[4 * f + k]];
        if (q >= 0) qf[cur[q]++] = f;
      }
  }
  // ---- incidence CSR of free vertices: entries tet*4 + slot, by tet ----
  std::vector<int> inc_ptr(n_free + 1, 0), inc;
  for (int e = 0; e < n_t; ++e)
    for (int k = 0; k < 4; ++k)
      if (tets_int[4 * e + k] < n_free) inc_ptr[tets_int[4 * e + k] + 1]++;
  for (int v = 0; v < n_free; ++v) inc_ptr[v + 1] += inc_ptr[v];
  inc.assign(inc_ptr[n_free], 0);
  {
    std::vector<int> cur(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int e = 0; e < n_t; ++e)
      for (int k = 0; k < 4; ++k) {
        const int v = tets_int[4 * e + k];
        if (v < n_free) inc[cur[v]++] = 4 * e + k;
      }
  }
  // ---- Laplacian L_w: 3/4 w on the diagonal, -1/4 w per element edge ----
  std::vector<double> diagL(n_free, 0.0);
  std::vector<int> rptr(n_free + 1, 0);
  for (int e = 0; e < n_t; ++e)
    for (int a = 0; a < 4; ++a)
      if (tets_int[4 * e + a] < n_free) rptr[tets_int[4 * e + a] + 1] += 3;
  for (int v = 0; v < n_free; ++v) rptr[v + 1] += rptr[v];
  std::vector<std::pair<int, double>> ent(rptr[n_free]);
  {
    std::vector<int> cur(rptr.begin(), rptr.end() - 1);
    for (int e = 0; e < n_t; ++e) {
      const double w = sim->omega[e];
      for (int a = 0; a < 4; ++a) {
        const int va = tets_int[4 * e + a];
        if (va >= n_free) continue;
        diagL[va] += 0.75 * w;
        for (int b = 0; b < 4; ++b)
          if (b != a) ent[cur[va]++] = {tets_int[4 * e + b], -0.25 * w};
      }
    }
  }
  std::vector<int> row_len(n_free, 0);
  std::vector<std::vector<std::pair<int, double>>> rows_ff(n_free);
  sim->fx_ptr.assign(n_free + 1, 0);
  sim->fx_col.clear();
  sim->fx_val.clear();
  for (int v = 0; v < n_free; ++v) {
    auto beg = ent.begin() + rptr[v], end = ent.begin() + rptr[v + 1];
    std::sort(beg, end, [](const std::pair<int, double>& x, const std::pair<int, double>& y) { return x.first < y.first; });
    std::vector<std::pair<int, double>> merged;
    for (auto it = beg; it != end; ++it) {
      if (!merged.empty() && merged.back().first == it->first)
        merged.back().second += it->second;
      else
        merged.push_back(*it);
    }
    for (auto& m : merged) {
      if (m.first < n_free)
        rows_ff[v].push_back(m);
      else {
        sim->fx_col.push_back(m.first);
        sim->fx_val.push_back(m.second);
      }
    }
    sim->fx_ptr[v + 1] = (int)sim->fx_col.size();
  }
  // ---- sliced ELL (32-row slices, column-major inside a slice) ----
  sim->n_slices = (n_free + 31) / 32;
  std::vector<int> sl_ptr(sim->n_slices + 1, 0), sl_col;
  std::vector<double> sl_val;
  for (int s = 0; s < sim->n_slices; ++s) {
    int width = 0;
    for (int l = 0; l < 32 && 32 * s + l < n_free; ++l) width = std::max(width, (int)rows_ff[32 * s + l].size());
    sl_ptr[s + 1] = sl_ptr[s] + 32 * width;
  }
  sl_col.assign(sl_ptr[sim->n_slices], 0);
  sl_val.assign(sl_ptr[sim->n_slices], 0.0);
  for (int s = 0; s < sim->n_slices; ++s) {
    const int width = (sl_ptr[s + 1] - sl_ptr[s]) / 32;
    for (int l = 0; l < 32; ++l) {
      const int row = 32 * s + l;
      for (int j = 0; j < width; ++j) {
        const size_t k = sl_ptr[s] + (size_t)j * 32 + l;
        if (row < n_free && j < (int)rows_ff[row].size()) {
          sl_col[k] = rows_ff[row][j].first;
          sl_val[k] = rows_ff[row][j].second;
        } else {
          sl_col[k] = row < n_free ? row : 0;
          sl_val[k] = 0.0;
        }
      }
    }
  }
  // ---- AABB trees of the tets and boundary faces (broad phase 1) ----
  sim->bvh_t_h = BvhHost{};
  sim->bvh_f_h = BvhHost{};
  if (sim->params.broad_phase == 1) {
    std::vector<double> cen(3 * (size_t)n_t);
    for (int e = 0; e < n_t; ++e)
      for (int c = 0; c < 3; ++c) {
        double a = 0.0;
        for (int k = 0; k < 4; ++k) a += rest_int[3 * (size_t)tets_int[4 * e + k] + c];
        cen[3 * (size_t)e + c] = 0.25 * a;
      }
    bvh_build(cen, n_t, robot_of_tet, n_robots, sim->bvh_t_h);
    cen.assign(3 * (size_t)sim->n_f, 0.0);
    for (int f = 0; f < sim->n_f; ++f)
      for (int c = 0; c < 3; ++c) {
        double a = 0.0;
        for (int k = 0; k < 3; ++k) a += rest_int[3 * (size_t)faces4[4 * f + k] + c];
        cen[3 * (size_t)f + c] = a / 3.0;
      }
    bvh_build(cen, sim->n_f, sim->robot_of_face_h.data(), n_robots, sim->bvh_f_h);
  }
  // ---- spatial hash sizes ----
  sim->H_t = (unsigned)pow2_at_least(2 * (size_t)n_t);
  sim->H_f = (unsigned)pow2_at_least(2 * (size_t)std::max(sim->n_f, 1));
  sim->cap_items = (int)std::min<long long>(16LL * (n_t + sim->n_f) + 4096, 2000000000LL);
  // ---- PCG grid: co-resident blocks, no more than the rows need ----
  int max_width = 0;
  for (int s = 0; s < sim->n_slices; ++s) max_width = std::max(max_width, (sl_ptr[s + 1] - sl_ptr[s]) / 32);
  const bool fp64 = sim->params.precision == CASIM_FP64;
  const int rr_rows = fp64 ? pcg_rr_max_rows<double>() : pcg_rr_max_rows<float>();
  const bool rr_fits = max_width <= PCG_RR_MAXW && n_free <= rr_rows;
  // dataflow PCG (FP32 vectors only): one row per thread, one block per SM.
  // Block b owns rows [b R, (b + 1) R), R = df_rows (whole slices); its
  // halo is the list of distinct columns its rows read, its own rows first
  // (each row writes its value there itself, from its registers), then the
  // other blocks' rows it loads, each part ascending; every sliced-ELL entry
  // also gets its column's index in that list.
  const int R_df = sim->df_rows;
  bool df_fits = !fp64 && max_width <= PCG_RR_MAXW && n_free <= pcg_df_max_rows(R_df);
  sim->halo_ptr_h.clear();
  sim->halo_rows_h.clear();
  sim->sl_lcol_h.clear();
  sim->halo_own_h.clear();
  sim->halo_self_h.clear();
  sim->halo_max = 0;
  if (df_fits) {
    const int spb = R_df / 32;
    const int nbk = (n_free + R_df - 1) / R_df;
    sim->halo_ptr_h.assign(nbk + 1, 0);
    sim->halo_own_h.assign(nbk, 0);
    sim->halo_self_h.assign(n_free, -1);
    sim->sl_lcol_h.assign(sl_col.size(), 0);
    std::vector<int> cols, own, other;
    for (int b = 0; b < nbk; ++b) {
      const int s0 = b * spb, s1 = std::min(sim->n_slices, s0 + spb);
      const int r0 = b * R_df, r1 = r0 + R_df;
      cols.clear();
      for (int s = s0; s < s1; ++s)
        for (int k = sl_ptr[s]; k < sl_ptr[s + 1]; ++k)
          if (32 * s + (k - sl_ptr[s]) % 32 < n_free) cols.push_back(sl_col[k]);
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      own.clear();
      other.clear();
      for (int c : cols) (c >= r0 && c < r1 ? own : other).push_back(c);
      const int n_own = (int)own.size();
      for (int j = 0; j < n_own; ++j) sim->halo_self_h[own[j]] = j;
      for (int s = s0; s < s1; ++s)
        for (int k = sl_ptr[s]; k < sl_ptr[s + 1]; ++k)
          if (32 * s + (k - sl_ptr[s]) % 32 < n_free) {
            const int c = sl_col[k];
            sim->sl_lcol_h[k] =
                c >= r0 && c < r1 ? (int)(std::lower_bound(own.begin(), own.end(), c) - own.begin())
                                  : n_own + (int)(std::lower_bound(other.begin(), other.end(), c) - other.begin());
          }
      sim->halo_rows_h.insert(sim->halo_rows_h.end(), own.begin(), own.end());
      sim->halo_rows_h.insert(sim->halo_rows_h.end(), other.begin(), other.end());
      sim->halo_ptr_h[b + 1] = (int)sim->halo_rows_h.size();
      sim->halo_own_h[b] = n_own;
      sim->halo_max = std::max(sim->halo_max, (int)cols.size());
    }
    if ((size_t)sim->halo_max * 16 > PCG_DF_HALO_MAX_BYTES) df_fits = false;
  }
  // two-level preconditioner of the dataflow kernel: Galerkin coarse matrix
  // A_c = Z^T L Z of the free-row Laplacian over aggregates of consecutive
  // rows (a = row / R), inverted here in FP64 (Cholesky)
  sim->n_agg = 0;
  sim->cg_ainv_h.clear();
  if (df_fits && n_robots == 1 && sim->params.pcg_precond == 0) {
    const int R = R_df / 3;
    const int na = (n_free + R - 1) / R;
    std::vector<double> Ac((size_t)na * na, 0.0);
    for (int v = 0; v < n_free; ++v) {
      const int a = v / R;
      Ac[(size_t)a * na + a] += diagL[v];
      for (const auto& e : rows_ff[v]) Ac[(size_t)a * na + e.first / R] += e.second;
    }
    if (cholesky_inverse(Ac, na)) {
      sim->n_agg = na;
      sim->cg_ainv_h.assign(Ac.begin(), Ac.end());
    }
  }
  if (df_fits && !pcg_df_prepare(R_df, 16 * sim->halo_max + (int)sizeof(float) * 3 * sim->n_agg)) df_fits = false;
  // cluster PCG: every robot's rows must fit the cluster's shared memory
  int max_robot_rows = 0;
  for (int r = 0; r < sim->n_robots; ++r)
    max_robot_rows = std::max(max_robot_rows, sim->robot_row_h[r + 1] - sim->robot_row_h[r]);
  const int cap = fp64 ? pcg_cluster_rows_cap<double>() : pcg_cluster_rows_cap<float>();
  const int need = (((max_robot_rows + PCG_CL_SIZE - 1) / PCG_CL_SIZE) + 31) & ~31;
  int max_clusters = 0;
  if (need <= cap) max_clusters = fp64 ? pcg_cluster_max_clusters<double>(cap) : pcg_cluster_max_clusters<float>(cap);
  const bool cl_fits = need <= cap && max_clusters > 0;
  const int kern = sim->params.pcg_kernel;
  if ((kern == 2 && !rr_fits) || (kern == 3 && !cl_fits) || (kern == 5 && !df_fits))
    return sim->fail(CASIM_E_INVALID, "requested PCG kernel does not fit this mesh (" + std::to_string(n_free) +
                                          " rows, width " + std::to_string(max_width) + ")");
  // auto: a single system runs fastest on the whole-grid register-resident
  // kernel (latency bound); several robots share the GPU through the cluster
  // kernel's work queue
  const bool many = sim->n_robots > 1;
  // segmented streaming PCG: every robot needs at least one co-resident block
  const int seg_max = fp64 ? pcg_seg_max_blocks<double>() : pcg_seg_max_blocks<float>();
  const bool seg_fits = sim->n_robots <= seg_max && seg_max > 0;
  if (kern == 4 && !seg_fits) return sim->fail(CASIM_E_INVALID, "segmented PCG: more robots than co-resident blocks");
  sim->pcg_seg = (kern == 4) || (kern == 0 && many && seg_fits);
  sim->seg_h.clear();
  sim->seg_blocks = 0;
  if (sim->pcg_seg) {
    // blocks per robot: one each, the rest in proportion to the robot's work,
    // rows x (expected CG iterations).  A launch lasts until the slowest robot
    // converges, and Jacobi-CG on these slender bodies needs iterations in
    // proportion to the body's length in elements, so the weight is the rows
    // times the longest extent of the robot's rest box over its mean edge.
    const int R = sim->n_robots;
    std::vector<double> wgt(R, 0.0);
    {
      std::vector<double> lo(3 * (size_t)R, 1e300), hi(3 * (size_t)R, -1e300), esum(R, 0.0);
      std::vector<long long> ecnt(R, 0);
      for (int v = 0; v < n_free; ++v) {
        const int r = sim->robot_of_vert_h[v];
        for (int c = 0; c < 3; ++c) {
          lo[3 * (size_t)r + c] = std::min(lo[3 * (size_t)r + c], rest_int[3 * (size_t)v + c]);
          hi[3 * (size_t)r + c] = std::max(hi[3 * (size_t)r + c], rest_int[3 * (size_t)v + c]);
        }
      }
      for (int e = 0; e < n_t; ++e) {
        const int r = robot_of_tet[e];
        const int a = tets_int[4 * e], b = tets_int[4 * e + 1];
        double dd = 0.0;
        for (int c = 0; c < 3; ++c) {
          const double t = rest_int[3 * (size_t)a + c] - rest_int[3 * (size_t)b + c];
          dd += t * t;
        }
        esum[r] += std::sqrt(dd);
        ecnt[r] += 1;
      }
      for (int r = 0; r < R; ++r) {
        const double rows = sim->robot_row_h[r + 1] - sim->robot_row_h[r];
        double ext = 0.0;
        for (int c = 0; c < 3; ++c) ext = std::max(ext, hi[3 * (size_t)r + c] - lo[3 * (size_t)r + c]);
        const double edge = ecnt[r] ? esum[r] / ecnt[r] : 1.0;
        wgt[r] = rows * std::max(1.0, edge > 0.0 ? ext / edge : 1.0);
      }
    }
    double wtot = 0.0;
    for (double w : wgt) wtot += w;
    std::vector<int> nb(R);
    int used = 0;
    for (int r = 0; r < R; ++r) {
      const long long rows = sim->robot_row_h[r + 1] - sim->robot_row_h[r];
      nb[r] = 1 + (int)(wgt[r] * (double)(seg_max - R) / std::max(wtot, 1e-300));
      nb[r] = (int)std::min<long long>(nb[r], std::max<long long>(1, rows));
      used += nb[r];
    }
    // Block boundaries fall on whole aggregates of SA rows counted from the
    // robot's first row (a block owns at most SEG_AGG_MAX aggregates), so the
    // per-robot coarse correction below can be summed block by block.
    const int SA = 128;  // the segmented kernel's aggregate rows
    bool coarse_ok = !fp64 && sim->params.pcg_precond == 0;
    used = 0;
    for (int r = 0; r < R; ++r) {
      const int rows = sim->robot_row_h[r + 1] - sim->robot_row_h[r];
      const int na = std::max(1, (rows + SA - 1) / SA);
      nb[r] = std::max(1, std::min(nb[r], na));
      if ((na + nb[r] - 1) / nb[r] > PCG_SEG_AGG_MAX) coarse_ok = false;
      used += nb[r];
    }
    std::vector<int> lo, hi, rb0, rb1, rob;
    int bidx = 0;
    for (int r = 0; r < R; ++r) {
      const int r0 = sim->robot_row_h[r], rows = sim->robot_row_h[r + 1] - r0;
      const int na = std::max(1, (rows + SA - 1) / SA);
      const int first = bidx;
      for (int k = 0; k < nb[r]; ++k) {
        lo.push_back(std::min(r0 + SA * (int)((long long)na * k / nb[r]), r0 + rows));
        hi.push_back(std::min(r0 + SA * (int)((long long)na * (k + 1) / nb[r]), r0 + rows));
        rob.push_back(r);
        ++bidx;
      }
      for (int k = 0; k < nb[r]; ++k) {
        rb0.push_back(first);
        rb1.push_back(bidx);
      }
    }
    sim->seg_blocks = used;
    sim->seg_h.reserve(5 * used);
    sim->seg_h.insert(sim->seg_h.end(), lo.begin(), lo.end());
    sim->seg_h.insert(sim->seg_h.end(), hi.begin(), hi.end());
    sim->seg_h.insert(sim->seg_h.end(), rb0.begin(), rb0.end());
    sim->seg_h.insert(sim->seg_h.end(), rb1.begin(), rb1.end());
    sim->seg_h.insert(sim->seg_h.end(), rob.begin(), rob.end());
    sim->pcg_grid = std::max(sim->pcg_grid, used);
    // per-robot Galerkin coarse matrices of the Laplacian over the robot's
    // aggregates, inverted (Cholesky, FP64) and kept as FP32
    sim->seg_agg_base_h.assign(R + 1, 0);
    sim->seg_ainv_off_h.assign(R + 1, 0);
    sim->seg_ainv_h.clear();
    if (coarse_ok) {
      for (int r = 0; r < R && coarse_ok; ++r) {
        const int r0 = sim->robot_row_h[r], rows = sim->robot_row_h[r + 1] - r0;
        const int na = std::max(1, (rows + SA - 1) / SA);
        std::vector<double> Ac((size_t)na * na, 0.0);
        for (int v = r0; v < r0 + rows; ++v) {
          const int a = (v - r0) / SA;
          Ac[(size_t)a * na + a] += diagL[v];
          for (const auto& e : rows_ff[v]) Ac[(size_t)a * na + (e.first - r0) / SA] += e.second;
        }
        if (!cholesky_inverse(Ac, na)) coarse_ok = false;
        sim->seg_agg_base_h[r + 1] = sim->seg_agg_base_h[r] + na;
        sim->seg_ainv_off_h[r + 1] = sim->seg_ainv_off_h[r] + (long long)na * na;
        sim->seg_ainv_h.insert(sim->seg_ainv_h.end(), Ac.begin(), Ac.end());
      }
    }
    sim->seg_coarse = coarse_ok;
    if (!coarse_ok) sim->seg_ainv_h.clear();
  }
  sim->pcg_cl = !sim->pcg_seg && ((kern == 3) || (kern == 0 && cl_fits && (many || !rr_fits)));
  const bool df = !sim->pcg_cl && !sim->pcg_seg && ((kern == 5) || (kern == 0 && !many && df_fits));
  sim->pcg_rr = !df && !sim->pcg_cl && !sim->pcg_seg && ((kern == 2) || (kern == 0 && rr_fits));
  sim->pcg_variant = df ? 5 : sim->pcg_rr ? 2 : 1;
  sim->cl_rows_cap = cap;
  sim->pcg_clusters = std::max(1, std::min(max_clusters, sim->n_robots));
  if (sim->pcg_seg) {
    // partials buffer is sized by pcg_grid (already >= seg_blocks)
  } else if (sim->pcg_variant == 5) {
    sim->pcg_grid = std::max(1, (n_free + R_df - 1) / R_df);
  } else if (sim->pcg_rr) {
    sim->pcg_grid = std::max(1, (n_free + PCG_RR_THREADS - 1) / PCG_RR_THREADS);
  } else {
    const int maxg = fp64 ? pcg_max_grid<double>() : pcg_max_grid<float>();
    sim->pcg_grid = std::max(1, std::min(maxg, (n_free + PCG_THREADS - 1) / PCG_THREADS));
  }
  sim->rs = sim->params.precision == CASIM_FP64 ? 8 : 4;
  int rc;
  if (sim->params.precision == CASIM_FP64)
    rc = upload_typed<double>(sim, rest_int, tets_int, group, Tc, vol0, tt, faces4, qf_ptr, qf, inc_ptr, inc, diagL,
                              sl_ptr, sl_col, sl_val);
  else
    rc = upload_typed<float>(sim, rest_int, tets_int, group, Tc, vol0, tt, faces4, qf_ptr, qf, inc_ptr, inc, diagL,
                             sl_ptr, sl_col, sl_val);
  if (rc) {
    sim->free_all();
    return rc;
  }
  rc = sim->params.precision == CASIM_FP64 ? upload_bfix<double>(sim) : upload_bfix<float>(sim);
  if (rc) {
    sim->free_all();
    return rc;
  }
  if (!sim->spheres.empty()) CK(upload_spheres(sim));
  sim->iters = 0;
  sim->status_bits = 0;
  sim->has_mesh = true;
  sim->graph_dirty = true;
  if (sim->n_groups == 0) {
    std::vector<double> none;
    rc = sim->params.precision == CASIM_FP64 ? set_actuation_typed<double>(sim, none)
                                             : set_actuation_typed<float>(sim, none);
    if (rc) return rc;
    sim->has_act = true;
  }
  return CASIM_OK;
}

extern "C" {

int casim_upload_mesh(casim_sim* sim, int32_t n_verts, const double* rest_xyz, int32_t n_tets, const int32_t* tets,
                      const int32_t* tet_group, const uint8_t* fixed) {
  if (!sim) return CASIM_E_INVALID;
  if (n_tets <= 0) return sim->fail(CASIM_E_INVALID, "empty mesh or null pointer");
  std::vector<int> robot(n_tets, 0);
  return upload_robots(sim, n_verts, rest_xyz, n_tets, tets, tet_group, fixed, 1, robot.data());
}

int casim_upload_batch(casim_sim* sim, int32_t n_robots, const casim_mesh_desc* robots) {
  if (!sim) return CASIM_E_INVALID;
  if (n_robots < 1 || !robots) return sim->fail(CASIM_E_INVALID, "n_robots >= 1 and robots required");
  long long nv = 0, nt = 0;
  for (int r = 0; r < n_robots; ++r) {
    const casim_mesh_desc& m = robots[r];
    if (m.n_verts <= 0 || m.n_tets <= 0 || !m.rest_xyz || !m.tets || !m.tet_group || !m.fixed)
      return sim->fail(CASIM_E_INVALID, "robot " + std::to_string(r) + ": empty mesh or null pointer");
    nv += m.n_verts;
    nt += m.n_tets;
  }
  if (nv > 2000000000LL || nt > 500000000LL) return sim->fail(CASIM_E_INVALID, "batch too large");
  std::vector<double> rest(3 * (size_t)nv);
  std::vector<int> tets(4 * (size_t)nt), group(nt), robot(nt);
  std::vector<uint8_t> fixed(nv);
  long long vo = 0, to = 0;
  int go = 0;
  for (int r = 0; r < n_robots; ++r) {
    const casim_mesh_desc& m = robots[r];
    std::copy(m.rest_xyz, m.rest_xyz + 3 * (size_t)m.n_verts, rest.begin() + 3 * vo);
    std::copy(m.fixed, m.fixed + m.n_verts, fixed.begin() + vo);
    int gmax = -1;
    for (int e = 0; e < m.n_tets; ++e) {
      for (int k = 0; k < 4; ++k) {
        const int v = m.tets[4 * e + k];
        if (v < 0 || v >= m.n_verts)
          return sim->fail(CASIM_E_INVALID, "robot " + std::to_string(r) + ": tet vertex id out of range");
        tets[4 * (to + e) + k] = (int)(v + vo);
      }
      const int g = m.tet_group[e];
      if (g < -1) return sim->fail(CASIM_E_INVALID, "group id < -1");
      group[to + e] = g < 0 ? -1 : g + go;
      robot[to + e] = r;
      gmax = std::max(gmax, g);
    }
    go += gmax + 1;
    vo += m.n_verts;
    to += m.n_tets;
  }
  return upload_robots(sim, (int)nv, rest.data(), (int)nt, tets.data(), group.data(), fixed.data(), n_robots,
                       robot.data());
}

int casim_set_actuation(casim_sim* sim, int32_t n_groups, const double* alpha) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  if (n_groups != sim->n_groups) return sim->fail(CASIM_E_INVALID, "n_groups must equal 1 + the largest group id");
  if (n_groups > 0 && !alpha) return sim->fail(CASIM_E_INVALID, "null alpha");
  std::vector<double> a(alpha, alpha + n_groups);
  for (double x : a)
    if (!(x > 0.0) || !std::isfinite(x)) return sim->fail(CASIM_E_INVALID, "volume ratio must be positive");
  const int rc = sim->params.precision == CASIM_FP64 ? set_actuation_typed<double>(sim, a)
                                                     : set_actuation_typed<float>(sim, a);
  if (rc) return rc;
  sim->alpha_h = a;
  sim->adj.valid = false;
  sim->has_act = true;
  return CASIM_OK;
}

int casim_set_spheres(casim_sim* sim, int32_t n, const double* cxyzr) {
  if (!sim) return CASIM_E_INVALID;
  if (n < 0 || n > 64 || (n > 0 && !cxyzr)) return sim->fail(CASIM_E_INVALID, "0 <= n <= 64 spheres");
  for (int i = 0; i < 4 * n; ++i)
    if (!std::isfinite(cxyzr[i])) return sim->fail(CASIM_E_INVALID, "non-finite sphere");
  for (int i = 0; i < n; ++i)
    if (!(cxyzr[4 * i + 3] > 0.0)) return sim->fail(CASIM_E_INVALID, "sphere radius must be positive");
  sim->spheres.assign(cxyzr, cxyzr + 4 * n);
  sim->n_spheres = n;
  if (sim->has_mesh && n > 0) CK(upload_spheres(sim));
  sim->graph_dirty = true;
  return CASIM_OK;
}

}  // extern "C"

namespace {
template <typename T>
int set_obstacle_typed(casim_sim* sim, int32_t n_verts, const double* xyz, int32_t n_tets, const int32_t* tets) {
  sim->free_obstacle();
  if (n_tets == 0) {
    sim->graph_dirty = true;
    return CASIM_OK;
  }
  std::vector<int> faces4;
  boundary_faces4(tets, n_tets, faces4);
  const int n_of = (int)(faces4.size() / 4);
  BvhHost ht, hf;
  std::vector<double> cen(3 * (size_t)n_tets);
  for (int e = 0; e < n_tets; ++e)
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int k = 0; k < 4; ++k) a += xyz[3 * (size_t)tets[4 * e + k] + c];
      cen[3 * (size_t)e + c] = 0.25 * a;
    }
  bvh_build(cen, n_tets, nullptr, 1, ht);
  cen.assign(3 * (size_t)n_of, 0.0);
  for (int f = 0; f < n_of; ++f)
    for (int c = 0; c < 3; ++c) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += xyz[3 * (size_t)faces4[4 * f + k] + c];
      cen[3 * (size_t)f + c] = a / 3.0;
    }
  bvh_build(cen, n_of, nullptr, 1, hf);
  auto oalloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    sim->obs_allocs.push_back(q);
    return q;
  };
  std::vector<R4<T>> Xh(n_verts);
  for (int i = 0; i < n_verts; ++i)
    Xh[i] = R4<T>{(T)xyz[3 * (size_t)i], (T)xyz[3 * (size_t)i + 1], (T)xyz[3 * (size_t)i + 2], T(0)};
  std::vector<int4> th(n_tets), fh(n_of);
  for (int e = 0; e < n_tets; ++e) th[e] = make_int4(tets[4 * e], tets[4 * e + 1], tets[4 * e + 2], tets[4 * e + 3]);
  for (int f = 0; f < n_of; ++f)
    fh[f] = make_int4(faces4[4 * f], faces4[4 * f + 1], faces4[4 * f + 2], faces4[4 * f + 3]);
  void* OX = oalloc(sizeof(R4<T>) * n_verts);
  int4* otet = (int4*)oalloc(sizeof(int4) * n_tets);
  int4* oface = (int4*)oalloc(sizeof(int4) * std::max(n_of, 1));
  auto mk = [&](const BvhHost& h, int n, int nv, const int4* prim, BvhDev& b) -> bool {
    b = BvhDev{};
    b.n = n;
    b.nv = nv;
    b.prim = prim;
    if (n < 1) return true;
    b.root = (int*)oalloc(sizeof(int) * h.root.size());
    b.child = (int2*)oalloc(sizeof(int2) * std::max(n - 1, 1));
    b.parent = (int*)oalloc(sizeof(int) * (2 * (size_t)n - 1));
    b.lo = (float4*)oalloc(sizeof(float4) * std::max(n - 1, 1));
    b.hi = (float4*)oalloc(sizeof(float4) * std::max(n - 1, 1));
    b.flag = (int*)oalloc(sizeof(int) * std::max(n - 1, 1));
    return b.root && b.child && b.parent && b.lo && b.hi && b.flag;
  };
  bool ok = OX && otet && oface && mk(ht, n_tets, 4, otet, sim->ot) && mk(hf, n_of, 3, oface, sim->of);
  if (!ok) {
    sim->free_obstacle();
    return sim->fail(CASIM_E_CUDA, "cudaMalloc failed (obstacle)");
  }
  cudaStream_t st = sim->stream;
  CK(cudaMemcpyAsync(OX, Xh.data(), sizeof(R4<T>) * n_verts, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(otet, th.data(), sizeof(int4) * n_tets, cudaMemcpyHostToDevice, st));
  if (n_of) CK(cudaMemcpyAsync(oface, fh.data(), sizeof(int4) * n_of, cudaMemcpyHostToDevice, st));
  for (auto pr : {std::make_pair(&ht, &sim->ot), std::make_pair(&hf, &sim->of)}) {
    const BvhHost& h = *pr.first;
    BvhDev& b = *pr.second;
    if (b.n >= 1) {
      CK(cudaMemcpyAsync((void*)b.child, h.child.data(), sizeof(int2) * h.child.size(), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync((void*)b.parent, h.parent.data(), sizeof(int) * h.parent.size(), cudaMemcpyHostToDevice,
                         st));
      CK(cudaMemcpyAsync((void*)b.root, h.root.data(), sizeof(int) * h.root.size(), cudaMemcpyHostToDevice, st));
    }
  }
  // the obstacle does not move: its boxes are fitted once
  launch_bvh_refit<T>(sim->ot, (const R4<T>*)OX, st);
  launch_bvh_refit<T>(sim->of, (const R4<T>*)OX, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  sim->OX = OX;
  sim->oface = oface;
  sim->n_ov = n_verts;
  sim->n_ot = n_tets;
  sim->n_of = n_of;
  sim->graph_dirty = true;
  return CASIM_OK;
}
}  // namespace

extern "C" {

int casim_set_obstacle_mesh(casim_sim* sim, int32_t n_verts, const double* xyz, int32_t n_tets,
                            const int32_t* tets) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "upload the robot mesh first");
  if (n_tets < 0 || n_verts < 0 || (n_tets > 0 && (!xyz || !tets || n_verts < 4)))
    return sim->fail(CASIM_E_INVALID, "obstacle: bad sizes or null pointer");
  for (long long i = 0; i < 3LL * n_verts; ++i)
    if (!std::isfinite(xyz[i])) return sim->fail(CASIM_E_INVALID, "obstacle: non-finite position");
  for (int e = 0; e < n_tets; ++e) {
    for (int k = 0; k < 4; ++k)
      if (tets[4 * e + k] < 0 || tets[4 * e + k] >= n_verts)
        return sim->fail(CASIM_E_INVALID, "obstacle: vertex id out of range at tet " + std::to_string(e));
    double V[4][3];
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) V[k][c] = xyz[3 * (size_t)tets[4 * e + k] + c];
    const double a[3] = {V[1][0] - V[0][0], V[1][1] - V[0][1], V[1][2] - V[0][2]};
    const double b[3] = {V[2][0] - V[0][0], V[2][1] - V[0][1], V[2][2] - V[0][2]};
    const double c[3] = {V[3][0] - V[0][0], V[3][1] - V[0][1], V[3][2] - V[0][2]};
    const double vol = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                       a[2] * (b[0] * c[1] - b[1] * c[0]);
    if (!(vol > 0.0)) return sim->fail(CASIM_E_INVALID, "obstacle: non-positive volume at tet " + std::to_string(e));
  }
  return sim->params.precision == CASIM_FP64 ? set_obstacle_typed<double>(sim, n_verts, xyz, n_tets, tets)
                                             : set_obstacle_typed<float>(sim, n_verts, xyz, n_tets, tets);
}

}  // extern "C"

extern "C" {

int casim_set_positions(casim_sim* sim, const double* xyz) {
  if (!sim) return CASIM_E_INVALID;
  sim->adj.valid = false;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  if (!xyz) return sim->fail(CASIM_E_INVALID, "null positions");
  for (long long i = 0; i < 3LL * sim->n_v; ++i)
    if (!std::isfinite(xyz[i])) return sim->fail(CASIM_E_INVALID, "non-finite position");
  return sim->params.precision == CASIM_FP64 ? set_positions_typed<double>(sim, xyz)
                                             : set_positions_typed<float>(sim, xyz);
}

int casim_reset(casim_sim* sim) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  const size_t nq = std::max(sim->n_q, 1);
  CK(cudaMemcpyAsync(sim->X, sim->X0, 4 * sim->rs * (size_t)sim->n_v, cudaMemcpyDeviceToDevice, sim->stream));
  CK(clear_xstep(sim));
  CK(cudaMemsetAsync(sim->spring_c, 0, sizeof(R4<double>) * (size_t)std::max(sim->n_free, 1), sim->stream));
  CK(cudaMemsetAsync(sim->sp.active, 0, sizeof(int) * nq, sim->stream));
  CK(cudaMemsetAsync(sim->sp.kind, 0, sizeof(int) * nq, sim->stream));
  CK(cudaMemsetAsync(sim->sp.face, 0xff, sizeof(int) * nq, sim->stream));
  CK(cudaMemsetAsync(sim->sp.bary, 0, sizeof(double) * 2 * nq, sim->stream));
  CK(cudaMemsetAsync(sim->sp.target, 0, sizeof(double) * 3 * nq, sim->stream));
  return CASIM_OK;
}

int casim_step(casim_sim* sim, int32_t n_iters) {
  NvtxRange r("casim_step");
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  if (!sim->has_act) return sim->fail(CASIM_E_STATE, "no actuation set");
  if (n_iters < 0) return sim->fail(CASIM_E_INVALID, "n_iters < 0");
  if (n_iters == 0) return CASIM_OK;
  return sim->params.precision == CASIM_FP64 ? step_typed<double>(sim, n_iters) : step_typed<float>(sim, n_iters);
}

int casim_forward_ckpt(casim_sim* sim, int32_t n_iters, int32_t ckpt_every) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  if (!sim->has_act) return sim->fail(CASIM_E_STATE, "no actuation set");
  if (n_iters < 1 || ckpt_every < 1) return sim->fail(CASIM_E_INVALID, "n_iters and ckpt_every must be >= 1");
  return sim->params.precision == CASIM_FP64 ? forward_ckpt_typed<double>(sim, n_iters, ckpt_every)
                                             : forward_ckpt_typed<float>(sim, n_iters, ckpt_every);
}

int casim_backward(casim_sim* sim, const double* dL_dX, double* dL_dalpha) {
  NvtxRange r("casim_backward");
  if (!sim || !dL_dX || (!dL_dalpha && sim->n_groups > 0)) return CASIM_E_INVALID;
  if (!sim->has_mesh || !sim->adj.valid)
    return sim->fail(CASIM_E_STATE, "casim_backward needs a preceding casim_forward_ckpt with the same actuation");
  return sim->params.precision == CASIM_FP64 ? backward_typed<double>(sim, dL_dX, dL_dalpha)
                                             : backward_typed<float>(sim, dL_dX, dL_dalpha);
}

int casim_sync(casim_sim* sim) {
  if (!sim) return CASIM_E_INVALID;
  CK(cudaStreamSynchronize(sim->stream));
  if (!sim->has_mesh) return CASIM_OK;
  int st = 0;
  CK(cudaMemcpy(&st, &sim->ctrl->status, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(&sim->ctrl->status, 0, sizeof(int)));
  sim->status_bits |= st;
  int rc = CASIM_OK;
  if (st & ST_BOUNDS) rc = CASIM_E_BOUNDS;
  else if (st & ST_TIMEOUT) rc = CASIM_E_TIMEOUT;
  else if (st & ST_NONFINITE) rc = CASIM_E_NONFINITE;
  else if (st & ST_OVERFLOW) rc = CASIM_E_OVERFLOW;
  else if (st & ST_PCG_MAXIT) rc = CASIM_W_PCG_MAXIT;
  else if (st & ST_PAIRS_TRUNC) rc = CASIM_W_PAIRS_TRUNCATED;
  sim->last_status = rc;
  if (rc < 0) sim->err = "device status " + std::to_string(st);
  return rc;
}

int casim_get_positions(casim_sim* sim, double* host_out, void* dev_out) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  return sim->params.precision == CASIM_FP64 ? get_positions_typed<double>(sim, host_out, dev_out)
                                             : get_positions_typed<float>(sim, host_out, dev_out);
}

int casim_get_contacts(casim_sim* sim, int32_t* pairs, int64_t* n_pairs, int32_t* obstacle_verts, int64_t* n_obst) {
  if (!sim || !n_pairs || !n_obst) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  const int n_q = sim->n_q, mp = sim->params.max_pairs_per_vertex;
  std::vector<int> cnt(std::max(n_q, 1)), pt((size_t)std::max(n_q, 1) * mp), obs(std::max(n_q, 1)),
      obm(std::max(n_q, 1));
  CK(cudaStreamSynchronize(sim->stream));
  if (n_q) {
    CK(cudaMemcpy(cnt.data(), sim->pair_count, sizeof(int) * n_q, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(pt.data(), sim->pair_tet, sizeof(int) * (size_t)n_q * mp, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(obs.data(), sim->obs_sphere, sizeof(int) * n_q, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(obm.data(), sim->obs_mesh, sizeof(int) * n_q, cudaMemcpyDeviceToHost));
  }
  const int64_t cap_p = *n_pairs, cap_o = *n_obst;
  int64_t np = 0, no = 0;
  for (int q = 0; q < n_q; ++q) {
    const int uv = sim->user_of_int[sim->q_verts[q]];
    const int c = std::min(cnt[q], mp);
    for (int j = 0; j < c; ++j) {
      if (pairs && np < cap_p) {
        pairs[2 * np] = uv;
        pairs[2 * np + 1] = pt[(size_t)q * mp + j];
      }
      ++np;
    }
    if (obs[q] >= 0 || obm[q] > 0) {
      if (obstacle_verts && no < cap_o) obstacle_verts[no] = uv;
      ++no;
    }
  }
  *n_pairs = np;
  *n_obst = no;
  if (np > cap_p || no > cap_o) return sim->fail(CASIM_E_CAPACITY, "contact buffer too small");
  return CASIM_OK;
}

int casim_get_springs(casim_sim* sim, int64_t* n, int32_t* verts, uint8_t* active, int32_t* kind, int32_t* face,
                      double* bary, double* target) {
  if (!sim || !n) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  const int n_q = sim->n_q;
  if (*n < n_q) {
    *n = n_q;
    return sim->fail(CASIM_E_CAPACITY, "spring buffer too small");
  }
  *n = n_q;
  if (n_q == 0) return CASIM_OK;
  std::vector<int> a(n_q), k(n_q), f(n_q);
  std::vector<double> b(2 * (size_t)n_q), t(3 * (size_t)n_q);
  CK(cudaStreamSynchronize(sim->stream));
  CK(cudaMemcpy(a.data(), sim->sp.active, sizeof(int) * n_q, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(k.data(), sim->sp.kind, sizeof(int) * n_q, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(f.data(), sim->sp.face, sizeof(int) * n_q, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(b.data(), sim->sp.bary, sizeof(double) * 2 * n_q, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(t.data(), sim->sp.target, sizeof(double) * 3 * n_q, cudaMemcpyDeviceToHost));
  for (int q = 0; q < n_q; ++q) {
    if (verts) verts[q] = sim->user_of_int[sim->q_verts[q]];
    if (active) active[q] = (uint8_t)(a[q] != 0);
    if (kind) kind[q] = k[q];
    if (face) face[q] = f[q];
    if (bary) {
      bary[2 * q] = b[2 * q];
      bary[2 * q + 1] = b[2 * q + 1];
    }
    if (target)
      for (int c = 0; c < 3; ++c) target[3 * q + c] = t[3 * q + c];
  }
  return CASIM_OK;
}

int casim_set_springs(casim_sim* sim, int64_t n, const int32_t* verts, const uint8_t* active, const int32_t* kind,
                      const int32_t* face, const double* bary, const double* target) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  const int n_q = sim->n_q;
  if (n != n_q || !verts || !active || !kind || !face || !bary || !target)
    return sim->fail(CASIM_E_INVALID, "spring records must cover every non-fixed boundary vertex");
  std::vector<int> a(n_q), k(n_q), f(n_q);
  for (int q = 0; q < n_q; ++q) {
    if (verts[q] != sim->user_of_int[sim->q_verts[q]]) return sim->fail(CASIM_E_INVALID, "spring vertex order");
    a[q] = active[q] ? 1 : 0;
    k[q] = kind[q];
    f[q] = face[q];
    if (a[q] && (k[q] < 0 || k[q] > 2)) return sim->fail(CASIM_E_INVALID, "spring kind");
    if (a[q] && k[q] == 2 && (f[q] < 0 || f[q] >= sim->n_of)) return sim->fail(CASIM_E_INVALID, "obstacle face id");
    if (a[q] && k[q] == 0 && (f[q] < 0 || f[q] >= sim->n_f)) return sim->fail(CASIM_E_INVALID, "spring face id");
    if (a[q] && k[q] == 1 && (f[q] < 0 || f[q] >= sim->n_spheres)) return sim->fail(CASIM_E_INVALID, "spring sphere id");
  }
  if (n_q == 0) return CASIM_OK;
  CK(cudaMemcpy(sim->sp.active, a.data(), sizeof(int) * n_q, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sim->sp.kind, k.data(), sizeof(int) * n_q, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sim->sp.face, f.data(), sizeof(int) * n_q, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sim->sp.bary, bary, sizeof(double) * 2 * n_q, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(sim->sp.target, target, sizeof(double) * 3 * n_q, cudaMemcpyHostToDevice));
  return CASIM_OK;
}

int casim_get_targets(casim_sim* sim, double* host_out) {
  if (!sim || !host_out) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  return sim->params.precision == CASIM_FP64 ? get_targets_typed<double>(sim, host_out)
                                             : get_targets_typed<float>(sim, host_out);
}

int casim_get_history(casim_sim* sim, int32_t cap, casim_iter_record* out, int32_t* n) {
  if (!sim || !n || cap < 0 || (cap > 0 && !out)) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  CK(cudaStreamSynchronize(sim->stream));
  long long done = 0;
  CK(cudaMemcpy(&done, &sim->ctrl->iter, sizeof(long long), cudaMemcpyDeviceToHost));
  std::vector<IterRec> h(sim->hist_cap);
  CK(cudaMemcpy(h.data(), sim->hist, sizeof(IterRec) * sim->hist_cap, cudaMemcpyDeviceToHost));
  const long long avail = std::min<long long>(done, sim->hist_cap);
  const long long m = std::min<long long>(avail, cap);
  for (long long j = 0; j < m; ++j) {
    const IterRec& r = h[(done - m + j) % sim->hist_cap];
    out[j].energy = r.energy;
    out[j].pcg_rel_residual = r.pcg_rel_residual;
    out[j].n_self_pairs = r.n_self_pairs;
    out[j].n_obstacle_pairs = r.n_obstacle_pairs;
    out[j].n_springs = r.n_springs;
    out[j].pcg_iters = r.pcg_iters;
    out[j].knot_signature = r.knot_sig;
    out[j].spring_signature = r.spring_sig;
  }
  *n = (int32_t)m;
  return CASIM_OK;
}

int casim_get_stats(casim_sim* sim, casim_stats* out) {
  if (!sim || !out) return CASIM_E_INVALID;
  std::memset(out, 0, sizeof(*out));
  if (!sim->has_mesh) return CASIM_OK;
  CK(cudaStreamSynchronize(sim->stream));
  Ctrl c;
  CK(cudaMemcpy(&c, sim->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  out->iterations = c.iter;
  out->total_pcg_iters = c.total_pcg;
  out->status = sim->last_status;
  out->pcg_kernel = sim->pcg_seg ? 4 : sim->pcg_cl ? 3 : sim->pcg_variant;
  out->status_bits = sim->status_bits;
  if (c.iter > 0) {
    IterRec r;
    CK(cudaMemcpy(&r, sim->hist + ((c.iter - 1) % sim->hist_cap), sizeof(IterRec), cudaMemcpyDeviceToHost));
    out->last.energy = r.energy;
    out->last.pcg_rel_residual = r.pcg_rel_residual;
    out->last.n_self_pairs = r.n_self_pairs;
    out->last.n_obstacle_pairs = r.n_obstacle_pairs;
    out->last.n_springs = r.n_springs;
    out->last.pcg_iters = r.pcg_iters;
    out->last.knot_signature = r.knot_sig;
    out->last.spring_signature = r.spring_sig;
  }
  return CASIM_OK;
}

// Checkpoint layout: header (magic, version, precision, n_v, n_q), positions
// (n_v*3 doubles, caller order), then per spring vertex active, kind, face
// (int32), bary (2 doubles), target (3 doubles); version 2 appends the last
// outer iteration's step x_i - x_(i-1) (n_v*3 doubles, caller order, zero
// where the solver keeps none), from which the next solve starts.  Version 1
// states load with a zero step.
namespace {
struct StateHeader {
  uint32_t magic, version;
  int32_t precision, n_v, n_q, pad;
};
const uint32_t kMagic = 0x4d495343u;  // "CSIM"

}  // namespace

int casim_save_state(casim_sim* sim, void* buf, size_t* len) {
  if (!sim || !len) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  const size_t nq = sim->n_q;
  const size_t need =
      sizeof(StateHeader) + 2 * sizeof(double) * 3 * sim->n_v + nq * (3 * sizeof(int32_t) + 5 * sizeof(double));
  if (!buf) {
    *len = need;
    return CASIM_OK;
  }
  if (*len < need) {
    *len = need;
    return sim->fail(CASIM_E_CAPACITY, "state buffer too small");
  }
  char* o = static_cast<char*>(buf);
  StateHeader h{kMagic, 2u, sim->params.precision, sim->n_v, sim->n_q, 0};
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  int rc = casim_get_positions(sim, reinterpret_cast<double*>(o), nullptr);
  if (rc) return rc;
  o += sizeof(double) * 3 * sim->n_v;
  std::vector<int32_t> verts(nq), kind(nq), face(nq);
  std::vector<uint8_t> act(nq);
  std::vector<double> bary(2 * nq), tgt(3 * nq);
  int64_t n = (int64_t)nq;
  rc = casim_get_springs(sim, &n, verts.data(), act.data(), kind.data(), face.data(), bary.data(), tgt.data());
  if (rc) return rc;
  for (size_t q = 0; q < nq; ++q) {
    const int32_t a = act[q];
    std::memcpy(o, &a, 4);
    std::memcpy(o + 4, &kind[q], 4);
    std::memcpy(o + 8, &face[q], 4);
    std::memcpy(o + 12, &bary[2 * q], 16);
    std::memcpy(o + 28, &tgt[3 * q], 24);
    o += 52;
  }
  std::vector<double> step(3 * (size_t)sim->n_v);
  rc = sim->params.precision == CASIM_FP64 ? xstep_io<double>(sim, step.data(), nullptr)
                                           : xstep_io<float>(sim, step.data(), nullptr);
  if (rc) return rc;
  std::memcpy(o, step.data(), sizeof(double) * step.size());
  *len = need;
  return CASIM_OK;
}

int casim_load_state(casim_sim* sim, const void* buf, size_t len) {
  if (!sim || !buf) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  const size_t nq = sim->n_q;
  const size_t need1 = sizeof(StateHeader) + sizeof(double) * 3 * sim->n_v + nq * 52;
  if (len < need1) return sim->fail(CASIM_E_INVALID, "state buffer too short");
  const char* o = static_cast<const char*>(buf);
  StateHeader h;
  std::memcpy(&h, o, sizeof(h));
  if (h.magic != kMagic || (h.version != 1u && h.version != 2u) || h.n_v != sim->n_v || h.n_q != sim->n_q)
    return sim->fail(CASIM_E_INVALID, "state does not match this mesh");
  if (h.version == 2u && len < need1 + sizeof(double) * 3 * sim->n_v)
    return sim->fail(CASIM_E_INVALID, "state buffer too short");
  o += sizeof(h);
  std::vector<double> X(3 * (size_t)sim->n_v);
  std::memcpy(X.data(), o, sizeof(double) * X.size());
  o += sizeof(double) * X.size();
  int rc = casim_set_positions(sim, X.data());
  if (rc) return rc;
  std::vector<int32_t> verts(nq), kind(nq), face(nq);
  std::vector<uint8_t> act(nq);
  std::vector<double> bary(2 * nq), tgt(3 * nq);
  for (size_t q = 0; q < nq; ++q) {
    int32_t a;
    std::memcpy(&a, o, 4);
    act[q] = (uint8_t)(a != 0);
    std::memcpy(&kind[q], o + 4, 4);
    std::memcpy(&face[q], o + 8, 4);
    std::memcpy(&bary[2 * q], o + 12, 16);
    std::memcpy(&tgt[3 * q], o + 28, 24);
    verts[q] = sim->user_of_int[sim->q_verts[q]];
    o += 52;
  }
  rc = casim_set_springs(sim, (int64_t)nq, verts.data(), act.data(), kind.data(), face.data(), bary.data(), tgt.data());
  if (rc || h.version < 2u) return rc;  // a version 1 state keeps the zero step set by casim_set_positions
  std::vector<double> step(3 * (size_t)sim->n_v);
  std::memcpy(step.data(), o, sizeof(double) * step.size());
  return sim->params.precision == CASIM_FP64 ? xstep_io<double>(sim, nullptr, step.data())
                                             : xstep_io<float>(sim, nullptr, step.data());
}

int casim_get_sizes(casim_sim* sim, int32_t* n_verts, int32_t* n_tets, int32_t* n_free, int32_t* n_boundary_faces,
                    int32_t* n_query_verts) {
  if (!sim) return CASIM_E_INVALID;
  if (n_verts) *n_verts = sim->n_v;
  if (n_tets) *n_tets = sim->n_t;
  if (n_free) *n_free = sim->n_free;
  if (n_boundary_faces) *n_boundary_faces = sim->n_f;
  if (n_query_verts) *n_query_verts = sim->n_q;
  return CASIM_OK;
}

int casim_get_phase_times(casim_sim* sim, double* ms_out5) {
  if (!sim || !ms_out5) return CASIM_E_INVALID;
  for (int k = 0; k < 5; ++k) ms_out5[k] = sim->phase_ms[k];
  return CASIM_OK;
}

// ---- remesh trigger and progressive actuation (Sec. III-C, Algorithm 1) ----
}  // extern "C"

namespace {

// Flags and element volumes of every tet against the reference in sim->rm_ref
// (internal order, FP64) or the rest shape; synchronous on the sim's stream.
template <typename T>
int remesh_eval_typed(casim_sim* sim, bool against_rest, double amax, double dmax, std::vector<uint8_t>& flags,
                      std::vector<double>& vols) {
  const Dev<T> d = make_dev<T>(sim);
  launch_remesh_flags<T>(d, against_rest ? sim->rm_rest : sim->rm_ref, amax, dmax, sim->rm_flags, sim->rm_vols,
                         sim->stream);
  flags.resize(sim->n_t);
  vols.resize(2 * (size_t)sim->n_t);
  CK(cudaMemcpyAsync(flags.data(), sim->rm_flags, (size_t)sim->n_t, cudaMemcpyDeviceToHost, sim->stream));
  CK(cudaMemcpyAsync(vols.data(), sim->rm_vols, sizeof(double) * 2 * sim->n_t, cudaMemcpyDeviceToHost, sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  return CASIM_OK;
}

int remesh_prepare(casim_sim* sim) {
  if (!sim->rm_rest) {
    sim->rm_ref = sim->dalloc<double>(3 * (size_t)sim->n_v);
    sim->rm_rest = sim->dalloc<double>(3 * (size_t)sim->n_v);
    sim->rm_vols = sim->dalloc<double>(2 * (size_t)std::max(sim->n_t, 1));
    sim->rm_flags = sim->dalloc<unsigned char>(std::max(sim->n_t, 1));
    if (!sim->rm_ref || !sim->rm_rest || !sim->rm_vols || !sim->rm_flags)
      return sim->fail(CASIM_E_CUDA, "cudaMalloc failed");
    CK(cudaMemcpyAsync(sim->rm_rest, sim->rest_h.data(), sizeof(double) * sim->rest_h.size(), cudaMemcpyHostToDevice,
                       sim->stream));
  }
  return CASIM_OK;
}

int remesh_eval(casim_sim* sim, bool against_rest, double amax, double dmax, std::vector<uint8_t>& flags,
                std::vector<double>& vols) {
  return sim->params.precision == CASIM_FP64 ? remesh_eval_typed<double>(sim, against_rest, amax, dmax, flags, vols)
                                             : remesh_eval_typed<float>(sim, against_rest, amax, dmax, flags, vols);
}

// per-group chamber volume ratios: sums of deformed over reference volumes, in tet order
void group_volume_ratios(const casim_sim* sim, const std::vector<double>& vols, std::vector<double>& out) {
  std::vector<double> num(sim->n_groups, 0.0), den(sim->n_groups, 0.0);
  for (int e = 0; e < sim->n_t; ++e) {
    const int g = sim->group_h[e];
    if (g < 0) continue;
    num[g] += vols[2 * (size_t)e];
    den[g] += vols[2 * (size_t)e + 1];
  }
  out.assign(sim->n_groups, 0.0);
  for (int g = 0; g < sim->n_groups; ++g) out[g] = den[g] != 0.0 ? num[g] / den[g] : 0.0;
}

}  // namespace

extern "C" {

int casim_remesh_flags(casim_sim* sim, const double* ref_xyz, double alpha_max, double d_max, uint8_t* flags_out,
                       int32_t* n_flagged, int32_t n_groups, double* group_volume_ratio) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  if (!flags_out) return sim->fail(CASIM_E_INVALID, "null flags_out");
  if (!(alpha_max > 0.0) || !(d_max > 0.0) || !std::isfinite(alpha_max) || !std::isfinite(d_max))
    return sim->fail(CASIM_E_INVALID, "alpha_max and d_max must be positive");
  if (group_volume_ratio && n_groups != sim->n_groups)
    return sim->fail(CASIM_E_INVALID, "n_groups must equal 1 + the largest group id");
  int rc = remesh_prepare(sim);
  if (rc) return rc;
  if (ref_xyz) {
    std::vector<double> ref(3 * (size_t)sim->n_v);
    for (int v = 0; v < sim->n_v; ++v)
      for (int c = 0; c < 3; ++c) {
        const double x = ref_xyz[3 * (size_t)v + c];
        if (!std::isfinite(x)) return sim->fail(CASIM_E_INVALID, "non-finite reference position");
        ref[3 * (size_t)sim->int_of_user[v] + c] = x;
      }
    CK(cudaMemcpyAsync(sim->rm_ref, ref.data(), sizeof(double) * ref.size(), cudaMemcpyHostToDevice, sim->stream));
    CK(cudaStreamSynchronize(sim->stream));  // ref is a local buffer
  }
  std::vector<uint8_t> flags;
  std::vector<double> vols;
  rc = remesh_eval(sim, ref_xyz == nullptr, alpha_max, d_max, flags, vols);
  if (rc) return rc;
  int count = 0;
  for (int e = 0; e < sim->n_t; ++e) {
    flags_out[e] = flags[e];
    count += flags[e] != 0;
  }
  if (n_flagged) *n_flagged = count;
  if (group_volume_ratio) {
    std::vector<double> gvr;
    group_volume_ratios(sim, vols, gvr);
    std::copy(gvr.begin(), gvr.end(), group_volume_ratio);
  }
  return CASIM_OK;
}

int casim_progressive(casim_sim* sim, int32_t n_groups, const double* alpha_target, double alpha_step,
                      int32_t n_inner, int32_t max_outer, double alpha_max, double d_max,
                      casim_outer_record* records, int32_t* n_outer) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  if (n_groups != sim->n_groups) return sim->fail(CASIM_E_INVALID, "n_groups must equal 1 + the largest group id");
  if (n_groups > 0 && !alpha_target) return sim->fail(CASIM_E_INVALID, "null alpha_target");
  if (!(alpha_step > 0.0) || !std::isfinite(alpha_step))
    return sim->fail(CASIM_E_INVALID, "alpha_step must be positive");
  if (n_inner < 0 || max_outer < 1 || !records)
    return sim->fail(CASIM_E_INVALID, "need n_inner >= 0, max_outer >= 1 and a records array");
  if (!(alpha_max > 0.0) || !(d_max > 0.0)) return sim->fail(CASIM_E_INVALID, "alpha_max and d_max must be positive");
  for (int g = 0; g < n_groups; ++g)
    if (!(alpha_target[g] > 0.0) || !std::isfinite(alpha_target[g]))
      return sim->fail(CASIM_E_INVALID, "volume ratio must be positive");
  int rc = remesh_prepare(sim);
  if (rc) return rc;
  std::vector<double> applied(n_groups);
  std::vector<uint8_t> flags;
  std::vector<double> vols, gvr;
  int done = 0;
  for (int k = 1; k <= max_outer; ++k) {
    bool last = true;
    double amax_applied = 0.0;
    for (int g = 0; g < n_groups; ++g) {
      applied[g] = std::min(alpha_target[g], k * alpha_step);
      last = last && applied[g] == alpha_target[g];
      amax_applied = std::max(amax_applied, applied[g]);
    }
    if ((rc = casim_set_actuation(sim, n_groups, applied.data()))) return rc;
    // the reference of this outer step's flags: the shape it starts from
    if (sim->params.precision == CASIM_FP64)
      launch_positions_f64<double>(make_dev<double>(sim), sim->n_v, sim->rm_ref, sim->stream);
    else
      launch_positions_f64<float>(make_dev<float>(sim), sim->n_v, sim->rm_ref, sim->stream);
    if ((rc = casim_step(sim, n_inner))) return rc;
    const int st = casim_sync(sim);
    if (st < 0) return st;
    if ((rc = remesh_eval(sim, false, alpha_max, d_max, flags, vols))) return rc;
    casim_outer_record& r = records[done++];
    r.k = k;
    r.status = st;
    r.n_volume = r.n_distortion = r.n_flagged = 0;
    for (int e = 0; e < sim->n_t; ++e) {
      r.n_volume += (flags[e] & 1) != 0;
      r.n_distortion += (flags[e] & 2) != 0;
      r.n_flagged += flags[e] != 0;
    }
    r.pad = 0;
    r.applied_max = amax_applied;
    if ((rc = remesh_eval(sim, true, alpha_max, d_max, flags, vols))) return rc;
    group_volume_ratios(sim, vols, gvr);
    r.chamber_volume_ratio_min = r.chamber_volume_ratio_max = gvr.empty() ? 0.0 : gvr[0];
    for (double v : gvr) {
      r.chamber_volume_ratio_min = std::min(r.chamber_volume_ratio_min, v);
      r.chamber_volume_ratio_max = std::max(r.chamber_volume_ratio_max, v);
    }
    if (last) break;
  }
  if (n_outer) *n_outer = done;
  return CASIM_OK;
}

// ---- Anderson acceleration (Sec. III-B) ----
}  // extern "C"

namespace {

int aa_prepare(casim_sim* sim, int m) {
  AAState& A = sim->aa;
  const size_t rs = 4 * (size_t)sim->rs;  // bytes of one R4<T>
  const size_t nf = std::max(sim->n_free, 1), nv = std::max(sim->n_v, 1);
  if (A.m_cap >= m && A.x) return CASIM_OK;
  const int cap = std::max(m, 1);
  A.x = sim->dalloc<unsigned char>(rs * nv);
  A.xa = sim->dalloc<unsigned char>(rs * nv);
  A.f = sim->dalloc<unsigned char>(rs * nf);
  A.fprev = sim->dalloc<unsigned char>(rs * nf);
  A.gprev = sim->dalloc<unsigned char>(rs * nf);
  A.dF.assign(cap, nullptr);
  A.dG.assign(cap, nullptr);
  for (int j = 0; j < cap; ++j) {
    A.dF[j] = sim->dalloc<unsigned char>(rs * nf);
    A.dG[j] = sim->dalloc<unsigned char>(rs * nf);
  }
  const int max_pairs = cap * (cap + 1) / 2 + cap;
  A.vec_tab = sim->dalloc<void*>(cap + 1);
  A.dg_tab = sim->dalloc<void*>(cap);
  A.pairs = sim->dalloc<int>(2 * max_pairs);
  A.theta = sim->dalloc<double>(cap);
  A.partials = sim->dalloc<double>((size_t)max_pairs * aa_dot_blocks(sim->n_free));
  if (!A.x || !A.xa || !A.f || !A.fprev || !A.gprev || !A.vec_tab || !A.dg_tab || !A.pairs || !A.theta || !A.partials)
    return sim->fail(CASIM_E_CUDA, "cudaMalloc failed");
  for (int j = 0; j < cap; ++j)
    if (!A.dF[j] || !A.dG[j]) return sim->fail(CASIM_E_CUDA, "cudaMalloc failed");
  A.m_cap = cap;
  return CASIM_OK;
}

// Eq. 8 energy at the positions in Xbuf (all vertices) with the local
// projections there and the current spring targets: the local step's element
// energies plus the spring energies, summed on the host in partial order.
template <typename T>
int aa_energy(casim_sim* sim, void* Xbuf, double& E) {
  Dev<T> d = make_dev<T>(sim);
  d.X = (R4<T>*)Xbuf;
  d.stats = 1;
  launch_local<T>(d, sim->stream);
  launch_spring_energy<T>(d.X, d.spring_c, d.k_spring, sim->n_free, sim->e_partials + d.n_e_local, sim->stream);
  std::vector<double> parts(d.n_e_local + spring_energy_blocks(sim->n_free));
  CK(cudaMemcpyAsync(parts.data(), sim->e_partials, sizeof(double) * parts.size(), cudaMemcpyDeviceToHost,
                     sim->stream));
  CK(cudaStreamSynchronize(sim->stream));
  E = 0.0;
  for (double p : parts) E += p;
  return CASIM_OK;
}

// Cholesky solve of the small SPD system M theta = r (row-major n x n); false
// if a pivot is not positive.
bool small_spd_solve(std::vector<double> M, std::vector<double> r, int n, std::vector<double>& theta) {
  for (int j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int k = 0; k < j; ++k) s -= M[j * n + k] * M[j * n + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    M[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = t / ljj;
    }
  }
  for (int i = 0; i < n; ++i) {  // L y = r
    double t = r[i];
    for (int k = 0; k < i; ++k) t -= M[i * n + k] * r[k];
    r[i] = t / M[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {  // L^T theta = y
    double t = r[i];
    for (int k = i + 1; k < n; ++k) t -= M[k * n + i] * r[k];
    r[i] = t / M[i * n + i];
  }
  theta = r;
  return true;
}

template <typename T>
int step_anderson_typed(casim_sim* sim, int n_iters, int m, casim_aa_record* recs, int* n_accepted) {
  AAState& A = sim->aa;
  cudaStream_t st = sim->stream;
  const int nf = sim->n_free;
  const size_t row = sizeof(R4<T>);
  CK(cudaMemcpyAsync(A.xa, sim->X, row * sim->n_v, cudaMemcpyDeviceToDevice, st));  // fixed rows of the proposal
  int head = 0, n_hist = 0, have_prev = 0, accepted = 0;
  for (int k = 0; k < n_iters; ++k) {
    CK(cudaMemcpyAsync(A.x, sim->X, row * sim->n_v, cudaMemcpyDeviceToDevice, st));  // x_k (all vertices)
    int rc = step_typed<T>(sim, 1);                                            // X = g_k = G(x_k)
    if (rc) return rc;
    const int slot = head;
    launch_aa_update<T>((const R4<T>*)sim->X, (const R4<T>*)A.x, (R4<T>*)A.f, (R4<T>*)A.fprev, (R4<T>*)A.gprev,
                        (R4<T>*)A.dF[slot], (R4<T>*)A.dG[slot], nf, have_prev, st);
    if (have_prev && m > 0) {
      head = (head + 1) % m;
      n_hist = std::min(n_hist + 1, m);
    }
    have_prev = 1;
    casim_aa_record r;
    r.e_prev = r.e_acc = std::numeric_limits<double>::quiet_NaN();
    r.accepted = 0;
    r.proposed = 0;
    if (m > 0 && n_hist > 0) {
      // columns oldest first; vector table: dF columns, then f
      const int h = n_hist;
      std::vector<int> cols(h);
      for (int j = 0; j < h; ++j) cols[j] = (head - h + j + m) % m;
      std::vector<void*> vtab(h + 1), gtab(h);
      for (int j = 0; j < h; ++j) {
        vtab[j] = A.dF[cols[j]];
        gtab[j] = A.dG[cols[j]];
      }
      vtab[h] = A.f;
      std::vector<int> pairs;
      for (int i = 0; i < h; ++i)
        for (int j = i; j < h; ++j) {
          pairs.push_back(i);
          pairs.push_back(j);
        }
      for (int i = 0; i < h; ++i) {
        pairs.push_back(i);
        pairs.push_back(h);
      }
      const int np = (int)pairs.size() / 2, nb = aa_dot_blocks(nf);
      CK(cudaMemcpyAsync(A.vec_tab, vtab.data(), sizeof(void*) * vtab.size(), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(A.pairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice, st));
      launch_aa_dot<T>((const R4<T>* const*)A.vec_tab, A.pairs, np, nf, A.partials, st);
      std::vector<double> parts((size_t)np * nb);
      CK(cudaMemcpyAsync(parts.data(), A.partials, sizeof(double) * parts.size(), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      std::vector<double> dots(np, 0.0);
      for (int p = 0; p < np; ++p)
        for (int b = 0; b < nb; ++b) dots[p] += parts[(size_t)p * nb + b];
      std::vector<double> M(h * h), rhs(h), theta;
      int p = 0;
      for (int i = 0; i < h; ++i)
        for (int j = i; j < h; ++j, ++p) M[i * h + j] = M[j * h + i] = dots[p];
      for (int i = 0; i < h; ++i, ++p) rhs[i] = dots[p];
      double tr = 0.0;
      for (int i = 0; i < h; ++i) tr += M[i * h + i];
      for (int i = 0; i < h; ++i) M[i * h + i] += 1e-12 * tr / h;
      if (tr > 0.0 && small_spd_solve(M, rhs, h, theta)) {
        CK(cudaMemcpyAsync(A.dg_tab, gtab.data(), sizeof(void*) * gtab.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(A.theta, theta.data(), sizeof(double) * h, cudaMemcpyHostToDevice, st));
        launch_aa_combine<T>((const R4<T>*)sim->X, (const R4<T>* const*)A.dg_tab, A.theta, h, nf, (R4<T>*)A.xa, st);
        // safeguard: the proposal must lower the energy of the point it came
        // from (both with iteration k's springs); else x_{k+1} = g_k
        double ep = 0.0, ea = 0.0;
        if ((rc = aa_energy<T>(sim, A.x, ep))) return rc;
        if ((rc = aa_energy<T>(sim, A.xa, ea))) return rc;
        r.e_prev = ep;
        r.e_acc = ea;
        r.proposed = 1;
        if (ea < ep) {
          CK(cudaMemcpyAsync(sim->X, A.xa, row * nf, cudaMemcpyDeviceToDevice, st));
          CK(clear_xstep(sim));  // the accepted proposal is not the last solve's end point
          r.accepted = 1;
          ++accepted;
        }
      }
    }
    if (recs) recs[k] = r;
  }
  CK(cudaStreamSynchronize(st));
  if (n_accepted) *n_accepted = accepted;
  return CASIM_OK;
}

}  // namespace

extern "C" {

int casim_step_anderson(casim_sim* sim, int32_t n_iters, int32_t m, casim_aa_record* records, int32_t* n_accepted) {
  if (!sim) return CASIM_E_INVALID;
  if (!sim->has_mesh) return sim->fail(CASIM_E_STATE, "no mesh uploaded");
  if (!sim->has_act) return sim->fail(CASIM_E_STATE, "no actuation set");
  if (n_iters < 0 || m < 0 || m > CASIM_AA_MAX_M) return sim->fail(CASIM_E_INVALID, "need n_iters >= 0, 0 <= m <= 16");
  if (n_iters == 0) {
    if (n_accepted) *n_accepted = 0;
    return CASIM_OK;
  }
  int rc = aa_prepare(sim, m);
  if (rc) return rc;
  sim->adj.valid = false;
  return sim->params.precision == CASIM_FP64 ? step_anderson_typed<double>(sim, n_iters, m, records, n_accepted)
                                             : step_anderson_typed<float>(sim, n_iters, m, records, n_accepted);
}

void casim_destroy(casim_sim* sim) {
  if (!sim) return;
  cudaStreamSynchronize(sim->stream);
  sim->free_all();
  if (sim->cap_stream) cudaStreamDestroy(sim->cap_stream);
  if (sim->side_stream) cudaStreamDestroy(sim->side_stream);
  if (sim->ev_fork) cudaEventDestroy(sim->ev_fork);
  if (sim->ev_join) cudaEventDestroy(sim->ev_join);
  delete sim;
}

int casim_build_checked(void) { return kCheckedBuild; }

const char* casim_last_error(const casim_sim* sim) {
  if (!sim) return g_create_error.c_str();
  return sim->err.c_str();
}

}  // extern "C"
