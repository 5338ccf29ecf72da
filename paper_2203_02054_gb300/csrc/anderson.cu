// Anderson acceleration of the local-global loop (Sec. III-B; Peng et al.
// 2018): vector kernels of one accelerated step.  The host drives the step
// (api.cu, casim_step_anderson): after an iteration has produced
// g_k = G(x_k), k_aa_update forms the residual f_k = g_k - x_k and the newest
// columns dF = f_k - f_{k-1}, dG = g_k - g_{k-1} of the history rings;
// k_aa_dot gives per-block FP64 partials of the Gram entries dF_i . dF_j and
// dF_i . f_k (summed on the host in block order); the host solves the m x m
// normal equations; k_aa_combine forms the proposal x_acc = g_k - dG theta;
// k_spring_energy supplies the spring part of the energy used by the
// safeguard.  All vectors cover the free rows only (fixed rows never move).
#include "common.cuh"
#include "kernels.h"

namespace casim {

static constexpr int AA_THREADS = 256;

// f = g - x; if have_prev, dF[slot] = f - f_prev and dG[slot] = g - g_prev;
// then f_prev = f, g_prev = g.
template <typename T>
__global__ void __launch_bounds__(AA_THREADS) k_aa_update(const R4<T>* __restrict__ g, const R4<T>* __restrict__ x,
                                                          R4<T>* __restrict__ f, R4<T>* __restrict__ f_prev,
                                                          R4<T>* __restrict__ g_prev, R4<T>* __restrict__ dF,
                                                          R4<T>* __restrict__ dG, int n, int have_prev) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R4<T> gi = g[i], xi = x[i];
  R4<T> fi;
  fi.x = gi.x - xi.x;
  fi.y = gi.y - xi.y;
  fi.z = gi.z - xi.z;
  fi.w = T(0);
  if (have_prev) {
    const R4<T> fp = f_prev[i], gp = g_prev[i];
    dF[i] = R4<T>{fi.x - fp.x, fi.y - fp.y, fi.z - fp.z, T(0)};
    dG[i] = R4<T>{gi.x - gp.x, gi.y - gp.y, gi.z - gp.z, T(0)};
  }
  f[i] = fi;
  f_prev[i] = fi;
  g_prev[i] = gi;
}

// Block partials of a . b over the free rows: blockIdx.y selects the pair
// (pairs[2 p], pairs[2 p + 1]) of vectors from the table vec; partial sums
// are FP64, reduced by a fixed tree (deterministic).
template <typename T>
__global__ void __launch_bounds__(AA_THREADS) k_aa_dot(const R4<T>* const* __restrict__ vec,
                                                       const int* __restrict__ pairs, int n,
                                                       double* __restrict__ partials) {
  __shared__ double sh[32];
  const R4<T>* a = vec[pairs[2 * blockIdx.y]];
  const R4<T>* b = vec[pairs[2 * blockIdx.y + 1]];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const R4<T> u = a[i], v = b[i];
    s += (double)u.x * v.x + (double)u.y * v.y + (double)u.z * v.z;
  }
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

// x_acc = g - sum_j theta_j dG_j over the free rows (theta in FP64).
template <typename T>
__global__ void __launch_bounds__(AA_THREADS) k_aa_combine(const R4<T>* __restrict__ g,
                                                           const R4<T>* const* __restrict__ dG,
                                                           const double* __restrict__ theta, int m, int n,
                                                           R4<T>* __restrict__ xa) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R4<T> gi = g[i];
  double x = gi.x, y = gi.y, z = gi.z;
  for (int j = 0; j < m; ++j) {
    const R4<T> d = dG[j][i];
    x -= theta[j] * (double)d.x;
    y -= theta[j] * (double)d.y;
    z -= theta[j] * (double)d.z;
  }
  xa[i] = R4<T>{(T)x, (T)y, (T)z, T(0)};
}

// Spring part of the Eq. 8 energy at positions X with the current spring
// targets: k mask_v |x_v - c_v|^2 summed per block in row order.
template <typename T>
__global__ void __launch_bounds__(AA_THREADS) k_spring_energy(const R4<T>* __restrict__ X,
                                                              const R4<double>* __restrict__ spring_c,
                                                              double k_spring, int n,
                                                              double* __restrict__ partials) {
  __shared__ double sh[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e = 0.0;
  if (i < n) {
    const R4<double> c = spring_c[i];
    if (c.w != 0.0) {
      const R4<T> x = X[i];
      const double ex = (double)x.x - c.x, ey = (double)x.y - c.y, ez = (double)x.z - c.z;
      e = k_spring * c.w * (ex * ex + ey * ey + ez * ez);
    }
  }
  const double s = block_sum(e, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

int aa_blocks(int n) { return (n + AA_THREADS - 1) / AA_THREADS; }
int spring_energy_blocks(int n) { return n <= 0 ? 0 : aa_blocks(n); }
int aa_dot_blocks(int n) { return std::max(1, std::min(256, (n + AA_THREADS - 1) / AA_THREADS)); }

template <typename T>
void launch_aa_update(const R4<T>* g, const R4<T>* x, R4<T>* f, R4<T>* f_prev, R4<T>* g_prev, R4<T>* dF, R4<T>* dG,
                      int n, int have_prev, cudaStream_t st) {
  if (n <= 0) return;
  k_aa_update<T><<<aa_blocks(n), AA_THREADS, 0, st>>>(g, x, f, f_prev, g_prev, dF, dG, n, have_prev);
}

template <typename T>
void launch_aa_dot(const R4<T>* const* vec, const int* pairs, int n_pairs, int n, double* partials, cudaStream_t st) {
  if (n_pairs <= 0) return;
  k_aa_dot<T><<<dim3(aa_dot_blocks(n), n_pairs), AA_THREADS, 0, st>>>(vec, pairs, n, partials);
}

template <typename T>
void launch_aa_combine(const R4<T>* g, const R4<T>* const* dG, const double* theta, int m, int n, R4<T>* xa,
                       cudaStream_t st) {
  if (n <= 0) return;
  k_aa_combine<T><<<aa_blocks(n), AA_THREADS, 0, st>>>(g, dG, theta, m, n, xa);
}

template <typename T>
void launch_spring_energy(const R4<T>* X, const R4<double>* spring_c, double k_spring, int n, double* partials,
                          cudaStream_t st) {
  if (n <= 0) return;
  k_spring_energy<T><<<aa_blocks(n), AA_THREADS, 0, st>>>(X, spring_c, k_spring, n, partials);
}

template void launch_aa_update<float>(const R4<float>*, const R4<float>*, R4<float>*, R4<float>*, R4<float>*,
                                      R4<float>*, R4<float>*, int, int, cudaStream_t);
template void launch_aa_update<double>(const R4<double>*, const R4<double>*, R4<double>*, R4<double>*,
                                       R4<double>*, R4<double>*, R4<double>*, int, int, cudaStream_t);
template void launch_aa_dot<float>(const R4<float>* const*, const int*, int, int, double*, cudaStream_t);
template void launch_aa_dot<double>(const R4<double>* const*, const int*, int, int, double*, cudaStream_t);
template void launch_aa_combine<float>(const R4<float>*, const R4<float>* const*, const double*, int, int,
                                       R4<float>*, cudaStream_t);
template void launch_aa_combine<double>(const R4<double>*, const R4<double>* const*, const double*, int, int,
                                        R4<double>*, cudaStream_t);
template void launch_spring_energy<float>(const R4<float>*, const R4<double>*, double, int, double*, cudaStream_t);
template void launch_spring_energy<double>(const R4<double>*, const R4<double>*, double, int, double*,
                                           cudaStream_t);

}  // namespace casim
