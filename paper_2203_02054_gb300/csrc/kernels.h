// Internal launcher declarations of the casim CUDA kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace casim {

struct CollisionScratch {
  int* tile_sums;  // scan tiles of the hash count array
  int* total;      // total hash entries
  // single-pass scan (null: the three-kernel scan): per-tile status words and
  // the tile ticket, stored right after the hash count array so that its one
  // memset zeroes them too
  unsigned long long* tile_status;
  unsigned* ticket;
};

static constexpr int LOCAL_THREADS = 128;
static constexpr int RHS_THREADS = 256;
static constexpr int PCG_THREADS = 512;
static constexpr int PCG_RR_THREADS = 256;
static constexpr int PCG_RR_MAXW = 16;   // widest sliced-ELL row kept in registers
static constexpr int PCG_CL_THREADS = 1024;
static constexpr int PCG_SEG_THREADS = 256;
static constexpr int PCG_SEG_AGG_MAX = 64;  // aggregates per block of the segmented PCG's coarse correction
static constexpr int PCG_DF_THREADS = 384;     // rows (threads) per block of the dataflow PCG
static constexpr int PCG_DF_ROWS_SMALL = 288;  // the same with 9 warps, for systems that fit 152 such blocks
static constexpr int PCG_DF_REPLICAS = 4;  // copies of the dataflow PCG's reduction slots
static constexpr size_t PCG_DF_HALO_MAX_BYTES = 160 * 1024;  // halo words in shared memory
static constexpr int PCG_CL_SIZE = 16;   // CTAs per cluster (non-portable size)

template <typename T>
void launch_collision(const Dev<T>& d, const CollisionScratch& cs, cudaStream_t st);
template <typename T>
void launch_springs(const Dev<T>& d, cudaStream_t st);
template <typename T>
void launch_bvh_refit(const BvhDev& b, const R4<T>* X, cudaStream_t st);
template <typename T>
void launch_local(const Dev<T>& d, cudaStream_t st);
template <typename T>
void launch_rhs(const Dev<T>& d, cudaStream_t st);
template <typename T>
cudaError_t launch_pcg(const Dev<T>& d, int grid, int variant, cudaStream_t st);
template <typename T>
int pcg_rr_max_rows();
int pcg_df_max_rows(int rows);
bool pcg_df_prepare(int rows, int smem_bytes);
template <typename T>
int pcg_seg_max_blocks();
template <typename T>
cudaError_t launch_pcg_seg(const Dev<T>& d, int blocks, cudaStream_t st);
template <typename T>
int pcg_cluster_rows_cap();
template <typename T>
int pcg_cluster_max_clusters(int rows_cap);
template <typename T>
cudaError_t launch_pcg_cluster(const Dev<T>& d, int n_clusters, cudaStream_t st);
template <typename T>
void launch_finalize(const Dev<T>& d, cudaStream_t st);
template <typename T>
void launch_gather_positions(const Dev<T>& d, const int* int_of_user, int n_user, T* out,
                             cudaStream_t st);
template <typename T>
int pcg_max_grid();
template <typename T>
void launch_remesh_flags(const Dev<T>& d, const double* ref, double alpha_max, double d_max, unsigned char* flags,
                         double* vols, cudaStream_t st);
template <typename T>
void launch_positions_f64(const Dev<T>& d, int n_v, double* out, cudaStream_t st);
int aa_dot_blocks(int n);
int spring_energy_blocks(int n);
template <typename T>
void launch_aa_update(const R4<T>* g, const R4<T>* x, R4<T>* f, R4<T>* f_prev, R4<T>* g_prev, R4<T>* dF, R4<T>* dG,
                      int n, int have_prev, cudaStream_t st);
template <typename T>
void launch_aa_dot(const R4<T>* const* vec, const int* pairs, int n_pairs, int n, double* partials, cudaStream_t st);
template <typename T>
void launch_aa_combine(const R4<T>* g, const R4<T>* const* dG, const double* theta, int m, int n, R4<T>* xa,
                       cudaStream_t st);
template <typename T>
void launch_spring_energy(const R4<T>* X, const R4<double>* spring_c, double k_spring, int n, double* partials,
                          cudaStream_t st);

// Device view of one reverse step of the adjoint (iteration i of a segment).
template <typename T>
struct AdjDev {
  const R4<T>* Xi;        // positions X_i (n_v)
  const R4<T>* mu;        // A_i^-1 g on the free rows
  const int* sp_active;   // spring records after iteration i's update (n_q)
  const int* sp_kind;
  const int* sp_face;
  const double* sp_bary;  // 2 n_q
  const int* sp_flag;     // self spring cast in iteration i: 1 by a ray hit, 2 by the closest point
  R4<double>* xbar_tet;   // 4 n_t per-tet pullbacks
  // Spring pullbacks, gathered deterministically: spring qi writes its
  // contributions to the slots [4 qi + 3 qf_ptr[qi], ...) (destination vertex
  // and value; at most 4 + 3 x its incident boundary faces), then the slots
  // are grouped by destination (count, scan, fill) and every vertex adds its
  // contributions in slot order.
  int* em_vert;           // n_slots destination vertex, -1 = unused
  R4<double>* em_val;     // n_slots contributions
  int* em_cnt;            // n_free + 1 counts per destination
  int* em_start;          // n_free + 1 exclusive offsets
  int* em_cur;            // n_free fill cursors
  int* em_list;           // n_slots slot ids grouped by destination
  int* em_tiles;          // scan tiles
  int* em_total;          // 1
  int n_slots;
  double* betabar;        // 2 n_q barycentric adjoints of kept springs
  double* alpha_part;     // local blocks x n_groups
  const double* alpha;    // n_groups
  double* abar;           // n_groups, accumulated dL/dalpha
  R4<double>* g;          // n_free: dL/dX_i on exit
  int n_groups;
};

template <typename T>
void launch_adjoint_step(const Dev<T>& d, const AdjDev<T>& a, cudaStream_t st);
template <typename T>
void launch_adjoint_diag(const Dev<T>& d, const AdjDev<T>& a, cudaStream_t st);
template <typename T>
void launch_adjoint_flags(const Dev<T>& d, int* flag, cudaStream_t st);

// Message of the last failure of a call that has no handle (casim_create,
// casim_contacts_noalloc) on the calling host thread; casim_last_error(NULL)
// returns it.
void set_handle_free_error(const char* msg);
const char* handle_free_error();

void launch_scan_exclusive(const int* in, int* out, int n, int* tile_sums, int* total, cudaStream_t st);

int local_blocks(int n_t);
int rhs_blocks(int n_free);
int local_blocks(int n_t, int threads);
int rhs_blocks(int n_free, int threads);
int scan_tiles(int n);
// ints to allocate after an (n + 1)-int count array for the single-pass scan
int scan_lookback_extra_ints(int n);

}  // namespace casim
