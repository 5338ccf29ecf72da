// Rotation fit of one element by a signed 3x3 SVD (the "rotation computed by
// SVD" of Eq. 1 in the paper).
//
// For D = X_c T_c^T, returns the proper rotation R = U V^T of the signed SVD
// D = U diag(s1, s2, s3) V^T with U, V in SO(3), s1 >= s2 >= |s3| and s3 of
// either sign; R maximises tr(R^T D) over SO(3) (Kabsch) and that maximum is
// s1 + s2 + s3.  Steps (the structure of McAdams et al. 2011, "Computing the
// singular value decomposition of 3x3 matrices with minimal branching and
// elementary floating point operations", with exact Jacobi angles instead of
// their approximate quaternion rotations):
//   1. cyclic Jacobi on the symmetric S = D^T D (Golub and Van Loan,
//      symmetric Schur rotations), accumulating V;
//   2. sort the eigenvalues descending, permuting the columns of V with one
//      sign flip per swap so that det V stays +1;
//   3. Givens QR of B = D V = U Sigma: U is a product of rotations and the
//      diagonal of the triangular factor holds the signed singular values.
#pragma once

#include <cuda_runtime.h>

namespace casim {

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

// One Jacobi rotation zeroing S[p][q] of the symmetric 3x3 S; V <- V J.
template <typename T>
__device__ __forceinline__ void jacobi_rotate(T S[3][3], T V[3][3], int p, int q) {
  const T spq = S[p][q];
  if (spq == T(0)) return;
  const T tau = (S[q][q] - S[p][p]) / (T(2) * spq);
  const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
  const T c = rsqrt_t<T>(T(1) + t * t);
  const T s = t * c;
  // S <- J^T S J with J the rotation in the (p, q) plane
  for (int k = 0; k < 3; ++k) {
    const T skp = S[k][p], skq = S[k][q];
    S[k][p] = c * skp - s * skq;
    S[k][q] = s * skp + c * skq;
  }
  for (int k = 0; k < 3; ++k) {
    const T spk = S[p][k], sqk = S[q][k];
    S[p][k] = c * spk - s * sqk;
    S[q][k] = s * spk + c * sqk;
  }
  S[p][q] = T(0);
  S[q][p] = T(0);
  for (int k = 0; k < 3; ++k) {
    const T vkp = V[k][p], vkq = V[k][q];
    V[k][p] = c * vkp - s * vkq;
    V[k][q] = s * vkp + c * vkq;
  }
}

template <typename T>
__device__ __forceinline__ void swap_cols_neg(T V[3][3], T lam[3], int a, int b) {
  T tl = lam[a];
  lam[a] = lam[b];
  lam[b] = tl;
  for (int k = 0; k < 3; ++k) {
    T t = V[k][a];
    V[k][a] = V[k][b];
    V[k][b] = -t;
  }
}

// Givens rotation acting on rows p, q of B (3x3) zeroing B[q][col]; U <- U G^T.
template <typename T>
__device__ __forceinline__ void givens_rows(T B[3][3], T U[3][3], int p, int q, int col) {
  const T a = B[p][col], b = B[q][col];
  const T r2 = a * a + b * b;
  if (!(r2 > T(0))) return;
  const T ir = rsqrt_t<T>(r2);
  const T c = a * ir, s = b * ir;
  for (int k = 0; k < 3; ++k) {
    const T bp = B[p][k], bq = B[q][k];
    B[p][k] = c * bp + s * bq;
    B[q][k] = -s * bp + c * bq;
  }
  B[q][col] = T(0);
  for (int k = 0; k < 3; ++k) {
    const T up = U[k][p], uq = U[k][q];
    U[k][p] = c * up + s * uq;
    U[k][q] = -s * up + c * uq;
  }
}

// R = U V^T (row-major 3x3) and tr(R^T D) for one D (row-major).
template <typename T, int SWEEPS>
__device__ __forceinline__ void kabsch_rotation(const T D[3][3], T R[3][3], T& trace) {
  T S[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      S[i][j] = D[0][i] * D[0][j] + D[1][i] * D[1][j] + D[2][i] * D[2][j];
      V[i][j] = (i == j) ? T(1) : T(0);
    }
#pragma unroll
  for (int sweep = 0; sweep < SWEEPS; ++sweep) {
    jacobi_rotate<T>(S, V, 0, 1);
    jacobi_rotate<T>(S, V, 0, 2);
    jacobi_rotate<T>(S, V, 1, 2);
  }
  T lam[3] = {S[0][0], S[1][1], S[2][2]};
  if (lam[0] < lam[1]) swap_cols_neg<T>(V, lam, 0, 1);
  if (lam[0] < lam[2]) swap_cols_neg<T>(V, lam, 0, 2);
  if (lam[1] < lam[2]) swap_cols_neg<T>(V, lam, 1, 2);
  T B[3][3], U[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      B[i][j] = D[i][0] * V[0][j] + D[i][1] * V[1][j] + D[i][2] * V[2][j];
      U[i][j] = (i == j) ? T(1) : T(0);
    }
  givens_rows<T>(B, U, 0, 1, 0);
  givens_rows<T>(B, U, 0, 2, 0);
  givens_rows<T>(B, U, 1, 2, 1);
  // B is now upper triangular: B[0][0] >= 0, B[1][1] >= 0, B[2][2] signed
  trace = B[0][0] + B[1][1] + B[2][2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = U[i][0] * V[j][0] + U[i][1] * V[j][1] + U[i][2] * V[j][2];
}

}  // namespace casim
