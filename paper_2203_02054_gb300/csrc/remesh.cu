// Remesh trigger (Sec. III-C; Algorithm 1, the check after the inner loop).
//
// A chamber element is flagged for remeshing when its volume grows by more
// than alpha_max against a reference shape (the rest shape, or the shape at
// the previous outer step: Vol(e_{k+1}) / Vol(e_k)), or when its shape is
// distorted by more than d_max, read as the largest singular value of the
// affine map F taking the reference element to the deformed one
// (F = D_d D_r^-1 with D the matrix of edge vectors v1 - v0, v2 - v0, v3 - v0).
// One thread per element, in FP64: the singular value comes from cyclic
// Jacobi sweeps on F^T F (its largest eigenvalue is sigma_max^2).  Remeshing
// itself is not part of this library.
#include "common.cuh"
#include "kernels.h"
#include "svd3.cuh"

namespace casim {

__device__ __forceinline__ double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

template <typename T>
__global__ void __launch_bounds__(256) k_remesh_flags(const R4<T>* __restrict__ X, const double* __restrict__ ref,
                                                      const int4* __restrict__ tet, const R4<T>* __restrict__ tinfo,
                                                      int n_t, double alpha_max, double d_max,
                                                      unsigned char* __restrict__ flags, double* __restrict__ vols) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_t) return;
  const int g = (int)tinfo[e].w;
  if (g < 0) {
    flags[e] = 0;
    vols[2 * e] = 0.0;
    vols[2 * e + 1] = 0.0;
    return;
  }
  const int4 t = tet[e];
  const int v[4] = {t.x, t.y, t.z, t.w};
  double Dd[3][3], Dr[3][3];
  const R4<T> x0 = X[v[0]];
  const double r0[3] = {ref[3 * (size_t)v[0]], ref[3 * (size_t)v[0] + 1], ref[3 * (size_t)v[0] + 2]};
  for (int k = 1; k < 4; ++k) {
    const R4<T> xk = X[v[k]];
    Dd[0][k - 1] = (double)xk.x - (double)x0.x;
    Dd[1][k - 1] = (double)xk.y - (double)x0.y;
    Dd[2][k - 1] = (double)xk.z - (double)x0.z;
    for (int c = 0; c < 3; ++c) Dr[c][k - 1] = ref[3 * (size_t)v[k] + c] - r0[c];
  }
  const double dd = det3(Dd), dr = det3(Dr);
  // D_r^-1 = adj(D_r) / det(D_r)
  double Ri[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
      Ri[i][j] = (Dr[i1][j1] * Dr[i2][j2] - Dr[i1][j2] * Dr[i2][j1]) / dr;
    }
  double F[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) F[i][j] = Dd[i][0] * Ri[0][j] + Dd[i][1] * Ri[1][j] + Dd[i][2] * Ri[2][j];
  double S[3][3], V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) S[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
  for (int sweep = 0; sweep < 8; ++sweep) {
    jacobi_rotate<double>(S, V, 0, 1);
    jacobi_rotate<double>(S, V, 0, 2);
    jacobi_rotate<double>(S, V, 1, 2);
  }
  const double lam = fmax(S[0][0], fmax(S[1][1], S[2][2]));
  const double smax = sqrt(fmax(lam, 0.0));
  const double ratio = dd / dr;
  flags[e] = (unsigned char)((ratio > alpha_max ? 1 : 0) | (smax > d_max ? 2 : 0));
  vols[2 * e] = dd / 6.0;
  vols[2 * e + 1] = dr / 6.0;
}

template <typename T>
__global__ void k_positions_f64(const R4<T>* __restrict__ X, int n_v, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  const R4<T> x = X[i];
  out[3 * (size_t)i] = (double)x.x;
  out[3 * (size_t)i + 1] = (double)x.y;
  out[3 * (size_t)i + 2] = (double)x.z;
}

template <typename T>
void launch_remesh_flags(const Dev<T>& d, const double* ref, double alpha_max, double d_max, unsigned char* flags,
                         double* vols, cudaStream_t st) {
  if (d.n_t <= 0) return;
  k_remesh_flags<T><<<(d.n_t + 255) / 256, 256, 0, st>>>(d.X, ref, d.tet, d.tinfo, d.n_t, alpha_max, d_max, flags,
                                                         vols);
}

template <typename T>
void launch_positions_f64(const Dev<T>& d, int n_v, double* out, cudaStream_t st) {
  if (n_v <= 0) return;
  k_positions_f64<T><<<(n_v + 255) / 256, 256, 0, st>>>(d.X, n_v, out);
}

template void launch_remesh_flags<float>(const Dev<float>&, const double*, double, double, unsigned char*, double*,
                                         cudaStream_t);
template void launch_remesh_flags<double>(const Dev<double>&, const double*, double, double, unsigned char*,
                                          double*, cudaStream_t);
template void launch_positions_f64<float>(const Dev<float>&, int, double*, cudaStream_t);
template void launch_positions_f64<double>(const Dev<double>&, int, double*, cudaStream_t);

}  // namespace casim
