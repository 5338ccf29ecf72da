// Exact orientation sign on the GPU.
//
// sign(det[q1-q0, q2-q0, q3-q0]) for double inputs, evaluated with a
// floating-point filter and an exact fallback, following the method of
// Shewchuk 1997 ("Adaptive precision floating-point arithmetic and fast
// robust geometric predicates"):
//   * filter: the determinant in double, each operation rounded separately
//     (no contraction), accepted when |det| exceeds (7 + 56 e) e * permanent,
//     e = 2^-53;
//   * fallback: every difference as an exact two-term expansion, every triple
//     product as an exact four-term expansion (FMA gives the rounding error of
//     a product exactly), all summed into a nonoverlapping expansion whose
//     largest component carries the sign.
// For float inputs an FP32 stage runs first (orient_sign_f): the same
// determinant and permanent in single precision with the same bound for unit
// roundoff e = 2^-24; what it cannot certify goes to the FP64 stages.
#pragma once

#include <cuda_runtime.h>

namespace casim {

__device__ __forceinline__ void two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  double bv = __dsub_rn(x, a);
  double av = __dsub_rn(x, bv);
  double br = __dsub_rn(b, bv);
  double ar = __dsub_rn(a, av);
  y = __dadd_rn(ar, br);
}

__device__ __forceinline__ void two_diff(double a, double b, double& x, double& y) {
  x = __dsub_rn(a, b);
  double bv = __dsub_rn(a, x);
  double av = __dadd_rn(x, bv);
  double br = __dsub_rn(bv, b);
  double ar = __dsub_rn(a, av);
  y = __dadd_rn(ar, br);
}

__device__ __forceinline__ void two_prod(double a, double b, double& x, double& y) {
  x = __dmul_rn(a, b);
  y = fma(a, b, -x);
}

// Adds b to the nonoverlapping expansion e[0..n) (increasing magnitude),
// dropping zero components; returns the new length.
__device__ __forceinline__ int grow_expansion_zeroelim(double* e, int n, double b) {
  double q = b;
  int m = 0;
  for (int i = 0; i < n; ++i) {
    double qn, h;
    two_sum(q, e[i], qn, h);
    q = qn;
    if (h != 0.0) e[m++] = h;
  }
  if (q != 0.0 || m == 0) e[m++] = q;
  return m;
}

// Exact sign of det[u, v, w] where u = b - a, v = c - a, w = d - a.
__device__ __noinline__ int orient_exact(double ax, double ay, double az, double bx, double by,
                                         double bz, double cx, double cy, double cz, double dx,
                                         double dy, double dz) {
  double U[3][2], V[3][2], W[3][2];
  two_diff(bx, ax, U[0][0], U[0][1]);
  two_diff(by, ay, U[1][0], U[1][1]);
  two_diff(bz, az, U[2][0], U[2][1]);
  two_diff(cx, ax, V[0][0], V[0][1]);
  two_diff(cy, ay, V[1][0], V[1][1]);
  two_diff(cz, az, V[2][0], V[2][1]);
  two_diff(dx, ax, W[0][0], W[0][1]);
  two_diff(dy, ay, W[1][0], W[1][1]);
  two_diff(dz, az, W[2][0], W[2][1]);
  // Leibniz terms: +u0 v1 w2, -u0 v2 w1, -u1 v0 w2, +u1 v2 w0, +u2 v0 w1, -u2 v1 w0
  const int ia[6] = {0, 0, 1, 1, 2, 2};
  const int ib[6] = {1, 2, 0, 2, 0, 1};
  const int ic[6] = {2, 1, 2, 0, 1, 0};
  const double sg[6] = {1.0, -1.0, -1.0, 1.0, 1.0, -1.0};
  double e[200];
  int n = 0;
  for (int t = 0; t < 6; ++t) {
    for (int i = 0; i < 2; ++i) {
      double a = U[ia[t]][i];
      if (a == 0.0) continue;
      for (int j = 0; j < 2; ++j) {
        double b = V[ib[t]][j];
        if (b == 0.0) continue;
        for (int k = 0; k < 2; ++k) {
          double c = W[ic[t]][k];
          if (c == 0.0) continue;
          double p1, p0, q1, q0, r1, r0;
          two_prod(a, b, p1, p0);
          two_prod(p1, c, q1, q0);
          two_prod(p0, c, r1, r0);
          const double s = sg[t];
          if (q0 != 0.0) n = grow_expansion_zeroelim(e, n, s * q0);
          if (r0 != 0.0) n = grow_expansion_zeroelim(e, n, s * r0);
          if (r1 != 0.0) n = grow_expansion_zeroelim(e, n, s * r1);
          if (q1 != 0.0) n = grow_expansion_zeroelim(e, n, s * q1);
          if (n > 192) n = 192;  // cannot happen: at most 192 terms are added
        }
      }
    }
  }
  if (n == 0) return 0;
  double top = e[n - 1];
  return (top > 0.0) - (top < 0.0);
}

// Filtered exact orientation sign.
__device__ __forceinline__ int orient_sign(double ax, double ay, double az, double bx, double by,
                                           double bz, double cx, double cy, double cz, double dx,
                                           double dy, double dz) {
  const double ux = __dsub_rn(bx, ax), uy = __dsub_rn(by, ay), uz = __dsub_rn(bz, az);
  const double vx = __dsub_rn(cx, ax), vy = __dsub_rn(cy, ay), vz = __dsub_rn(cz, az);
  const double wx = __dsub_rn(dx, ax), wy = __dsub_rn(dy, ay), wz = __dsub_rn(dz, az);
  const double m1 = __dmul_rn(vy, wz), m2 = __dmul_rn(vz, wy);
  const double m3 = __dmul_rn(wy, uz), m4 = __dmul_rn(wz, uy);
  const double m5 = __dmul_rn(uy, vz), m6 = __dmul_rn(uz, vy);
  const double det = __dadd_rn(__dadd_rn(__dmul_rn(ux, __dsub_rn(m1, m2)), __dmul_rn(vx, __dsub_rn(m3, m4))),
                               __dmul_rn(wx, __dsub_rn(m5, m6)));
  const double perm =
      __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(fabs(m1), fabs(m2)), fabs(ux)),
                          __dmul_rn(__dadd_rn(fabs(m3), fabs(m4)), fabs(vx))),
                __dmul_rn(__dadd_rn(fabs(m5), fabs(m6)), fabs(wx)));
  const double eps = 1.1102230246251565e-16;  // 2^-53
  const double bound = __dmul_rn((7.0 + 56.0 * eps) * eps, perm);
  if (det > bound) return 1;
  if (-det > bound) return -1;
  return orient_exact(ax, ay, az, bx, by, bz, cx, cy, cz, dx, dy, dz);
}

// The FP32 stage alone: +1 or -1 when the FP32 filter certifies the sign, 0
// when it does not (the sign may still be anything, zero included).
__device__ __forceinline__ int orient_filter_f(float ax, float ay, float az, float bx, float by, float bz,
                                               float cx, float cy, float cz, float dx, float dy, float dz) {
  const float ux = __fsub_rn(bx, ax), uy = __fsub_rn(by, ay), uz = __fsub_rn(bz, az);
  const float vx = __fsub_rn(cx, ax), vy = __fsub_rn(cy, ay), vz = __fsub_rn(cz, az);
  const float wx = __fsub_rn(dx, ax), wy = __fsub_rn(dy, ay), wz = __fsub_rn(dz, az);
  const float m1 = __fmul_rn(vy, wz), m2 = __fmul_rn(vz, wy);
  const float m3 = __fmul_rn(wy, uz), m4 = __fmul_rn(wz, uy);
  const float m5 = __fmul_rn(uy, vz), m6 = __fmul_rn(uz, vy);
  const float det = __fadd_rn(__fadd_rn(__fmul_rn(ux, __fsub_rn(m1, m2)), __fmul_rn(vx, __fsub_rn(m3, m4))),
                              __fmul_rn(wx, __fsub_rn(m5, m6)));
  const float perm = __fadd_rn(__fadd_rn(__fmul_rn(__fadd_rn(fabsf(m1), fabsf(m2)), fabsf(ux)),
                                         __fmul_rn(__fadd_rn(fabsf(m3), fabsf(m4)), fabsf(vx))),
                               __fmul_rn(__fadd_rn(fabsf(m5), fabsf(m6)), fabsf(wx)));
  const float bound = __fmul_rn(0x1.c0000ep-22f, perm);  // (7 + 56 e) e, e = 2^-24
  if (perm >= 0x1p-60f) {
    if (det > bound) return 1;
    if (-det > bound) return -1;
  }
  return 0;
}

// Filtered exact orientation sign for float inputs.  The FP32 stage is
// Shewchuk's error analysis with e = 2^-24: |det| > (7 + 56 e) e * permanent
// certifies the sign.  That analysis assumes no underflow, so a permanent
// below 2^-60 is not certified (for coordinates below 2^20 any underflowed
// product then contributes far less than the bound); NaN or infinite values
// fail both comparisons.  Uncertified cases take the FP64 filter and the exact
// fallback on the exactly converted inputs, so the sign is always exact.
__device__ __forceinline__ int orient_sign_f(float ax, float ay, float az, float bx, float by, float bz, float cx,
                                             float cy, float cz, float dx, float dy, float dz) {
  const float ux = __fsub_rn(bx, ax), uy = __fsub_rn(by, ay), uz = __fsub_rn(bz, az);
  const float vx = __fsub_rn(cx, ax), vy = __fsub_rn(cy, ay), vz = __fsub_rn(cz, az);
  const float wx = __fsub_rn(dx, ax), wy = __fsub_rn(dy, ay), wz = __fsub_rn(dz, az);
  const float m1 = __fmul_rn(vy, wz), m2 = __fmul_rn(vz, wy);
  const float m3 = __fmul_rn(wy, uz), m4 = __fmul_rn(wz, uy);
  const float m5 = __fmul_rn(uy, vz), m6 = __fmul_rn(uz, vy);
  const float det = __fadd_rn(__fadd_rn(__fmul_rn(ux, __fsub_rn(m1, m2)), __fmul_rn(vx, __fsub_rn(m3, m4))),
                              __fmul_rn(wx, __fsub_rn(m5, m6)));
  const float perm = __fadd_rn(__fadd_rn(__fmul_rn(__fadd_rn(fabsf(m1), fabsf(m2)), fabsf(ux)),
                                         __fmul_rn(__fadd_rn(fabsf(m3), fabsf(m4)), fabsf(vx))),
                               __fmul_rn(__fadd_rn(fabsf(m5), fabsf(m6)), fabsf(wx)));
  const float errbound_f = 0x1.c0000ep-22f;  // (7 + 56 e) e for e = 2^-24, exact in FP32
  const float bound = __fmul_rn(errbound_f, perm);
  if (perm >= 0x1p-60f) {
    if (det > bound) return 1;
    if (-det > bound) return -1;
  }
  return orient_sign((double)ax, (double)ay, (double)az, (double)bx, (double)by, (double)bz, (double)cx,
                     (double)cy, (double)cz, (double)dx, (double)dy, (double)dz);
}

}  // namespace casim
