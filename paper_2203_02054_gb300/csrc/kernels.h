// Internal launcher declarations of the casim CUDA kernels (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace casim {

struct CollisionScratch {
  int* tile_sums;  // scan tiles of the hash count array
  int* total;      // total hash entries
};

static constexpr int LOCAL_THREADS = 128;
static constexpr int RHS_THREADS = 256;
static constexpr int PCG_THREADS = 512;
static constexpr int PCG_RR_THREADS = 256;
static constexpr int PCG_RR_MAXW = 16;   // widest sliced-ELL row kept in registers
static constexpr int PCG_CL_THREADS = 1024;
static constexpr int PCG_CL_SIZE = 16;   // CTAs per cluster (non-portable size)

template <typename T>
void launch_collision(const Dev<T>& d, const CollisionScratch& cs, cudaStream_t st);
template <typename T>
void launch_springs(const Dev<T>& d, cudaStream_t st);
template <typename T>
void launch_local(const Dev<T>& d, cudaStream_t st);
template <typename T>
void launch_rhs(const Dev<T>& d, cudaStream_t st);
template <typename T>
cudaError_t launch_pcg(const Dev<T>& d, int grid, int variant, cudaStream_t st);
template <typename T>
int pcg_rr_max_rows();
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

int spring_blocks(int n_q);
int local_blocks(int n_t);
int scan_tiles(int n);

}  // namespace casim
