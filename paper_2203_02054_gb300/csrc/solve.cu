// Local step (Sec. III-A, Eq. 6, Eq. 7), right-hand-side gather and the
// global step solve (Sec. III-B, Eq. 8) on the GPU.
//
// Global step: the normal equations of Eq. 8 are A X = b with
//   A = L_w + k diag(mask),  L_w = sum_e w_e S_e^T N S_e  (3/4 w on the
//   diagonal, -1/4 w per shared edge), b = sum_e w_e S_e^T P_e^T + k c - A_fx x_fixed,
// the three coordinate columns sharing A.  They are solved together by
// Jacobi-preconditioned conjugate gradients in the single-reduction form of
// Chronopoulos and Gear (1989), inside one persistent cooperative kernel.
// Per iteration the neighbours' preconditioned residual u must be visible to
// the SpMV and one grid reduction produces (r.u, w.u, r.r) to FP64 accuracy:
// the barrier kernels publish u with a grid barrier, the dataflow kernel
// (MIXED precision) with epoch-tagged words that readers wait for.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "svd3.cuh"

namespace casim {

// ---- FP64-grade dot products
// The CG dot products are accumulated to FP64 accuracy.  FP64 arithmetic is
// slow on this part (a dependent FP64 add takes about 64 cycles and an SM
// retires about two FP64 lanes per cycle, against 4.5 cycles and 128 lanes for
// FP32), so for FP32 vectors the per-row products and the in-block trees use
// double-word (float-float) arithmetic built from error-free transformations
// on the FP32 pipes:
//   TwoProd by FMA (the rounding error of a*b is fma(a, b, -a*b)),
//   TwoSum (Knuth) and Fast2Sum (Dekker),
//   the compensated dot product Dot2 of Ogita, Rump and Oishi (2005), kept
//   unrounded as a double word,
//   the double-word addition of Joldes, Muller and Popescu (2017) in its
//   11-operation form (below), relative error a few u^2 (u = 2^-24).
// Every operation is an explicitly rounded intrinsic, so the compiler can
// neither contract nor reassociate them.  Block partials are summed in block
// order (FP64 in the barrier kernels, double words in the dataflow kernel).
struct DW {
  float hi, lo;
};

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// requires a == 0 or exponent(a) >= exponent(b)
__device__ __forceinline__ void fast_two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Sloppy double-word addition (Joldes, Muller, Popescu 2017, Algorithm 5):
// 11 operations; for operands of the same sign the relative error is at most
// 3u^2, otherwise the error is at most about u^2 (|x| + |y|), the same kind of
// bound as an FP64 sum has.
__device__ __forceinline__ DW dw_add_sloppy(DW x, DW y) {
  float sh, sl;
  two_sum_f(x.hi, y.hi, sh, sl);
  const float v = __fadd_rn(x.lo, y.lo);
  const float w = __fadd_rn(sl, v);
  DW z;
  fast_two_sum_f(sh, w, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ DW dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
  float p = __fmul_rn(a0, b0);
  float e = __fmaf_rn(a0, b0, -p);
  const float h1 = __fmul_rn(a1, b1), q1 = __fmaf_rn(a1, b1, -h1);
  const float h2 = __fmul_rn(a2, b2), q2 = __fmaf_rn(a2, b2, -h2);
  float s, t;
  two_sum_f(p, h1, s, t);
  p = s;
  e = __fadd_rn(e, __fadd_rn(q1, t));
  two_sum_f(p, h2, s, t);
  p = s;
  e = __fadd_rn(e, __fadd_rn(q2, t));
  DW z;
  two_sum_f(p, e, z.hi, z.lo);
  return z;
}

// Double-word product: the exact product of the high parts by TwoProd (FMA),
// the cross terms added in FP32, renormalised by Fast2Sum (relative error a
// few u^2; the neglected lo * lo term is below u^2 of the result).
__device__ __forceinline__ DW dw_mul(DW a, DW b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  DW z;
  fast_two_sum_f(p, e, z.hi, z.lo);
  return z;
}
__device__ __forceinline__ DW dw_neg(DW a) { return DW{-a.hi, -a.lo}; }
// s += x for an FP32 x: the high parts by TwoSum, its error into the low part
// (renormalised once at the end by dw_norm).
__device__ __forceinline__ void dw_acc(DW& s, float x) {
  float h, e;
  two_sum_f(s.hi, x, h, e);
  s.hi = h;
  s.lo = __fadd_rn(s.lo, e);
}
// s += a b, the product exact by TwoProd (FMA)
__device__ __forceinline__ void dw_acc_prod(DW& s, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = __fmaf_rn(a, b, -p);
  float h, e;
  two_sum_f(s.hi, p, h, e);
  s.hi = h;
  s.lo = __fadd_rn(s.lo, __fadd_rn(e, pe));
}
__device__ __forceinline__ DW dw_norm(DW s) {
  DW z;
  fast_two_sum_f(s.hi, s.lo, z.hi, z.lo);
  return z;
}
// an FP64 value as a double word (hi = its FP32 rounding, lo = the rest rounded)
__device__ __forceinline__ DW dw_from(double x) {
  const float h = (float)x;
  return DW{h, (float)(x - (double)h)};
}


// Double-word quotient by one correction step: q = a.hi / b.hi in FP32, the
// remainder a - q b formed from the exact product q * b.hi (TwoProd; a.hi -
// q b.hi is exact by Sterbenz's lemma, q b.hi being within an ulp of a.hi)
// and the low parts, then q + remainder / b.hi renormalised (relative error a
// few u^2 for b not near the FP32 range limits).
__device__ __forceinline__ DW dw_div(DW a, DW b) {
  const float q = __fdiv_rn(a.hi, b.hi);
  const float p = __fmul_rn(q, b.hi);
  const float pe = __fmaf_rn(q, b.hi, -p);
  float r = __fsub_rn(a.hi, p);
  r = __fsub_rn(r, pe);
  r = __fadd_rn(r, a.lo);
  r = __fmaf_rn(-q, b.lo, r);
  DW z;
  fast_two_sum_f(q, __fdiv_rn(r, b.hi), z.hi, z.lo);
  return z;
}

__device__ __forceinline__ double dot3(double a0, double a1, double a2, double b0, double b1, double b2) {
  return fma(a2, b2, fma(a1, b1, a0 * b0));
}

__device__ __forceinline__ DW acc_add(DW a, DW b) { return dw_add_sloppy(a, b); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ DW shfl_down(DW v, int o) {
  return DW{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ DW shfl_xor(DW v, int o) {
  return DW{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double acc_to_f64(DW a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double acc_to_f64(double a) { return a; }

template <typename A>
__device__ __forceinline__ A acc_zero();
template <>
__device__ __forceinline__ DW acc_zero<DW>() { return DW{0.0f, 0.0f}; }
template <>
__device__ __forceinline__ double acc_zero<double>() { return 0.0; }


// Block sums of NV per-thread values by fixed shuffle trees (within each warp,
// then over the NW warp sums, padded with zeros to a power of two); the FP64
// result is valid in lane 0 of warp 0.
// Contains one __syncthreads; sh holds at least 32 * NV doubles.
template <int NV, int NW, typename A>
__device__ __forceinline__ void block_sums(A (&v)[NV], double* sh, double (&bs)[NV]) {
  static_assert(sizeof(A) == sizeof(double), "accumulator must fit a double slot");
  static_assert(NW >= 1 && NW <= 32, "at most 32 warps per block");
  constexpr int NW2 = NW <= 1 ? 1 : NW <= 2 ? 2 : NW <= 4 ? 4 : NW <= 8 ? 8 : NW <= 16 ? 16 : 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  A* sa = reinterpret_cast<A*>(sh);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = acc_add(v[k], shfl_down(v[k], o));
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sa[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      A t = lane < NW ? sa[k * 32 + lane] : acc_zero<A>();
#pragma unroll
      for (int o = NW2 >> 1; o > 0; o >>= 1) t = acc_add(t, shfl_down(t, o));
      bs[k] = acc_to_f64(t);
    }
  }
}

// Warp sums of NV <= 4 double words by one butterfly that halves the values
// each lane carries at every level (a warp reduce-scatter): lanes exchange
// the half they give up at distance 16, then 8 (NV > 2), and every lane then
// finishes its one value with the remaining levels.  The pairs added are
// those of a shuffle-down tree over distances 16, 8, 4, 2, 1 (the sloppy
// addition is commutative bit for bit: TwoSum's error term is exact), so each
// sum equals that tree's, with 6 instead of 15 exchanges for NV = 3.  Value k
// ends in lanes [k L, (k + 1) L), L = 32 / (NV rounded up to a power of two).
template <int NV>
__device__ __forceinline__ DW warp_sums_dw_rs(const DW (&v)[NV]) {
  static_assert(NV >= 1 && NV <= 4, "one to four values");
  const int lane = threadIdx.x & 31;
  if constexpr (NV == 1) {
    DW x = v[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = dw_add_sloppy(x, shfl_xor(x, o));
    return x;
  } else if constexpr (NV == 2) {
    const bool up = lane & 16;
    DW x = dw_add_sloppy(up ? v[1] : v[0], shfl_xor(up ? v[0] : v[1], 16));
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) x = dw_add_sloppy(x, shfl_xor(x, o));
    return x;
  } else {
    const DW z{0.0f, 0.0f};
    const DW a2 = v[2], a3 = NV > 3 ? v[NV > 3 ? 3 : 0] : z;
    const bool up = lane & 16;
    const DW k0 = dw_add_sloppy(up ? a2 : v[0], shfl_xor(up ? v[0] : a2, 16));
    const DW k1 = dw_add_sloppy(up ? a3 : v[1], shfl_xor(up ? v[1] : a3, 16));
    const bool up8 = lane & 8;
    DW x = dw_add_sloppy(up8 ? k1 : k0, shfl_xor(up8 ? k0 : k1, 8));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) x = dw_add_sloppy(x, shfl_xor(x, o));
    return x;
  }
}

// Block sums of NV per-thread double words by fixed trees of sloppy
// double-word additions (the warp butterfly above, then warp 0 over the
// warps' sums); the double-word result is valid in lane 0 of warp 0.
// Contains one __syncthreads; sh holds at least 32 * NV doubles.
template <int NV, int NW>
__device__ __forceinline__ void block_sums_dw(DW (&v)[NV], double* sh, DW (&bs)[NV]) {
  static_assert(NW >= 1 && NW <= 32, "at most 32 warps per block");
  constexpr int NW2 = NW <= 1 ? 1 : NW <= 2 ? 2 : NW <= 4 ? 4 : NW <= 8 ? 8 : NW <= 16 ? 16 : 32;
  constexpr int L = NV == 1 ? 32 : NV == 2 ? 16 : 8;  // lanes per value after the butterfly
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  DW* sa = reinterpret_cast<DW*>(sh);
  const DW x = warp_sums_dw_rs<NV>(v);
  if (lane % L == 0 && lane / L < NV) sa[(lane / L) * 32 + wid] = x;
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      DW t = lane < NW ? sa[k * 32 + lane] : DW{0.0f, 0.0f};
#pragma unroll
      for (int o = NW2 >> 1; o > 0; o >>= 1) t = dw_add_sloppy(t, shfl_down(t, o));
      bs[k] = t;
    }
  }
}

// ---------------------------------------------------------------- local step
template <typename T>
__device__ __forceinline__ T cbrt_t(T x);
template <>
__device__ __forceinline__ float cbrt_t<float>(float x) { return cbrtf(x); }
template <>
__device__ __forceinline__ double cbrt_t<double>(double x) { return cbrt(x); }

__device__ __forceinline__ double w_table(const double* knots, int n, double eps, int& seg) {
  // piecewise linear through (eps_i, w_i), clamped at both ends; seg = the
  // interval used (0 below the first knot, i + 1 for [eps_i, eps_i+1), n above)
  seg = 0;
  if (eps <= knots[0]) return knots[1];
  for (int i = 0; i + 1 < n; ++i) {
    const double x0 = knots[2 * i], x1 = knots[2 * i + 2];
    if (eps < x1) {
      const double y0 = knots[2 * i + 1], y1 = knots[2 * i + 3];
      seg = i + 1;
      return y0 + (eps - x0) * (y1 - y0) / (x1 - x0);
    }
  }
  seg = n;
  return knots[2 * n - 1];
}

// The same table in FP32 (knots rounded to FP32), for FP32 positions.
__device__ __forceinline__ float w_table_f(const float* knots, int n, float eps, int& seg) {
  seg = 0;
  if (eps <= knots[0]) return knots[1];
  for (int i = 0; i + 1 < n; ++i) {
    const float x0 = knots[2 * i], x1 = knots[2 * i + 2];
    if (eps < x1) {
      const float y0 = knots[2 * i + 1], y1 = knots[2 * i + 3];
      seg = i + 1;
      return y0 + (eps - x0) * (y1 - y0) / (x1 - x0);
    }
  }
  seg = n;
  return knots[2 * n - 1];
}

// One thread per tet.  For FP32 positions the strain, w(eps) and the energy
// statistic stay on the FP32 pipes (FP32 strain and table, energy in double
// words); FP64 positions use FP64 throughout.
template <typename T, int SWEEPS, int BS>
__global__ void __launch_bounds__(BS) k_local(Dev<T> d) {
  constexpr bool F32 = std::is_same<T, float>::value;
  __shared__ double shd[32];
  __shared__ float s_kn[F32 ? 128 : 1];  // the knot table in FP32 (at most 64 knots)
  if constexpr (F32) {
    for (int k = threadIdx.x; k < 2 * d.n_knots; k += BS) s_kn[k] = (float)d.knots[k];
    __syncthreads();
  }
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double en = 0.0;
  DW en_w{0.0f, 0.0f};
  unsigned long long ksig = 0;
  if (e < d.n_t) {
    const int4 t = chk_idx4(d.ctrl, d.tet[e], d.n_v);
    const R4<T> x0 = d.X[t.x], x1 = d.X[t.y], x2 = d.X[t.z], x3 = d.X[t.w];
    // centered deformed shape X_c = V^d N, formed from differences to x0
    T Xc[3][4];
    {
      const T r1[3] = {x1.x - x0.x, x1.y - x0.y, x1.z - x0.z};
      const T r2[3] = {x2.x - x0.x, x2.y - x0.y, x2.z - x0.z};
      const T r3[3] = {x3.x - x0.x, x3.y - x0.y, x3.z - x0.z};
      for (int i = 0; i < 3; ++i) {
        const T m = (r1[i] + r2[i] + r3[i]) * T(0.25);
        Xc[i][0] = -m;
        Xc[i][1] = r1[i] - m;
        Xc[i][2] = r2[i] - m;
        Xc[i][3] = r3[i] - m;
      }
    }
    const R4<T> tx = d.Tc[3 * (size_t)e], ty = d.Tc[3 * (size_t)e + 1], tz = d.Tc[3 * (size_t)e + 2];
    const T Tm[3][4] = {{tx.x, tx.y, tx.z, tx.w}, {ty.x, ty.y, ty.z, ty.w}, {tz.x, tz.y, tz.z, tz.w}};
    T D[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        D[i][j] = Xc[i][0] * Tm[j][0] + Xc[i][1] * Tm[j][1] + Xc[i][2] * Tm[j][2] + Xc[i][3] * Tm[j][3];
    T R[3][3], tr;
    kabsch_rotation<T, SWEEPS>(D, R, tr);
    T RT[3][4];
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 4; ++k) RT[i][k] = R[i][0] * Tm[0][k] + R[i][1] * Tm[1][k] + R[i][2] * Tm[2][k];
    const R4<T> info = d.tinfo[e];
    const T omega = info.x, vol0 = info.y, tt = info.z;
    const int g = (int)info.w;
    T P[3][4];
    if (g >= 0) {
      // chamber element: every target vertex is the rest vertex scaled by cbrt(alpha_g)
      const T s = d.cbrt_alpha[g];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) P[i][k] = s * RT[i][k];
    } else {
      // body element: blend with w = R_omega(eps), then volume scaling (Eq. 6, Eq. 7)
      T mis = T(0);
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) {
          const T q = Xc[i][k] - RT[i][k];
          mis += q * q;
        }
      int seg;
      T w;
      if constexpr (F32) {
        w = w_table_f(s_kn, d.n_knots, sqrtf(mis / tt), seg);
      } else {
        w = w_table(d.knots, d.n_knots, sqrt(mis / tt), seg);
      }
      if (d.stats) ksig = sig_mix((unsigned)e, (unsigned)seg);
      T B[3][4];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) B[i][k] = (T(1) - w) * Xc[i][k] + w * RT[i][k];
      const T a0 = B[0][1] - B[0][0], a1 = B[1][1] - B[1][0], a2 = B[2][1] - B[2][0];
      const T b0 = B[0][2] - B[0][0], b1 = B[1][2] - B[1][0], b2 = B[2][2] - B[2][0];
      const T c0 = B[0][3] - B[0][0], c1 = B[1][3] - B[1][0], c2 = B[2][3] - B[2][0];
      const T volB = (a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0)) / T(6);
      const T s = (volB > T(1e-3) * vol0) ? cbrt_t<T>(vol0 / volB) : T(1);
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) P[i][k] = s * B[i][k];
    }
    if (d.stats) {
      if constexpr (F32) {
        // sum of (Xc - P)^2 with each difference exact as a double word
        DW acc{0.0f, 0.0f};
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 4; ++k) {
            float qh, ql;
            two_sum_f(Xc[i][k], -P[i][k], qh, ql);
            dw_acc_prod(acc, qh, qh);
            acc.lo = __fmaf_rn(__fmul_rn(2.0f, qh), ql, acc.lo);
          }
        en_w = dw_mul(DW{omega, 0.0f}, dw_norm(acc));
      } else {
        double acc = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 4; ++k) {
            const double q = (double)Xc[i][k] - (double)P[i][k];
            acc += q * q;
          }
        en = (double)omega * acc;
      }
    }
    R4<T>* out = d.P + 4 * (size_t)e;
    for (int k = 0; k < 4; ++k) {
      R4<T> c;
      c.x = omega * P[0][k];
      c.y = omega * P[1][k];
      c.z = omega * P[2][k];
      c.w = T(0);
      out[k] = c;
    }
  }
  if (d.stats) warp_add_u64(ksig, &(d.hist + (d.ctrl->iter % d.hist_cap))->knot_sig);
  if constexpr (F32) {
    DW v[1] = {en_w}, bs[1];
    block_sums_dw<1, BS / 32>(v, shd, bs);
    if (threadIdx.x == 0) d.e_partials[blockIdx.x] = acc_to_f64(bs[0]);
  } else {
    const double s = block_sum(en, shd);
    if (threadIdx.x == 0) d.e_partials[blockIdx.x] = s;
  }
}

// ------------------------------------------------------------ RHS gather
// b_v = sum over incident (e, slot) of w_e P_e[:, slot] + k mask_v c_v - bfix_v,
// accumulated in FP64 (the products of the FP32 targets need no rounding).
// The rows also carry the spring energy k mask_v |x_v - c_v|^2 (Eq. 5) of
// this iteration's springs (positions are unchanged since the spring update),
// summed per block in row order.
// One row of the right-hand side and of the diagonal: b_i, A_ii and the row's
// spring energy (see above).
template <typename T>
__device__ __forceinline__ void rhs_row(const Dev<T>& d, int i, R4<double>& b, T& diag, double& es) {
  double bx = 0.0, by = 0.0, bz = 0.0;
  const int k1 = d.inc_ptr[i + 1];
  for (int k = d.inc_ptr[i]; k < k1; ++k) {
    const R4<T> p = d.P[chk_idx(d.ctrl, d.inc[k], 4 * d.n_t)];
    bx += (double)p.x;
    by += (double)p.y;
    bz += (double)p.z;
  }
  const R4<double> sc = d.spring_c[i];
  const double km = d.k_spring * sc.w;
  const R4<double> bf = d.bfix[i];
  b = R4<double>{bx + km * sc.x - bf.x, by + km * sc.y - bf.y, bz + km * sc.z - bf.z, 0.0};
  diag = d.diagL[i] + (T)km;
  es = 0.0;
  if (sc.w != 0.0) {
    const R4<T> xi = d.X[i];
    const double ex = (double)xi.x - sc.x, ey = (double)xi.y - sc.y, ez = (double)xi.z - sc.z;
    es = km * (ex * ex + ey * ey + ez * ez);
  }
}

// The same row for FP32 positions with the FP32 terms added as double words
// (TwoSum) and the FP64 spring and fixed-vertex terms only on the rows that
// have them; the spring energy as a double word.
__device__ __forceinline__ void rhs_row_dw(const Dev<float>& d, int i, R4<double>& b, float& diag, DW& es) {
  DW bx{0.0f, 0.0f}, by{0.0f, 0.0f}, bz{0.0f, 0.0f};
  const int k1 = d.inc_ptr[i + 1];
#pragma unroll 4
  for (int k = d.inc_ptr[i]; k < k1; ++k) {
    const R4<float> p = d.P[chk_idx(d.ctrl, d.inc[k], 4 * d.n_t)];
    dw_acc(bx, p.x);
    dw_acc(by, p.y);
    dw_acc(bz, p.z);
  }
  bx = dw_norm(bx);
  by = dw_norm(by);
  bz = dw_norm(bz);
  b = R4<double>{(double)bx.hi + (double)bx.lo, (double)by.hi + (double)by.lo, (double)bz.hi + (double)bz.lo, 0.0};
  const R4<double> sc = d.spring_c[i];
  const double km = d.k_spring * sc.w;
  const R4<double> bf = d.bfix[i];
  diag = d.diagL[i] + (float)km;
  es = DW{0.0f, 0.0f};
  if (km != 0.0) {
    b.x += km * sc.x;
    b.y += km * sc.y;
    b.z += km * sc.z;
    const R4<float> xi = d.X[i];
    const double ex = (double)xi.x - sc.x, ey = (double)xi.y - sc.y, ez = (double)xi.z - sc.z;
    es = dw_from(km * (ex * ex + ey * ey + ez * ez));
  }
  if (bf.x != 0.0 || bf.y != 0.0 || bf.z != 0.0) {
    b.x -= bf.x;
    b.y -= bf.y;
    b.z -= bf.z;
  }
}

template <typename T, int BS>
__global__ void __launch_bounds__(BS) k_rhs(Dev<T> d) {
  __shared__ double shd[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (std::is_same<T, float>::value) {
    DW es[1] = {{0.0f, 0.0f}}, bs[1];
    if (i < d.n_free) {
      R4<double> b;
      float dg;
      rhs_row_dw(d, i, b, dg, es[0]);
      d.b[i] = b;
      d.diag[i] = dg;
    }
    block_sums_dw<1, BS / 32>(es, shd, bs);
    if (threadIdx.x == 0) d.e_partials[d.n_e_local + blockIdx.x] = acc_to_f64(bs[0]);
  } else {
    double es = 0.0;
    if (i < d.n_free) {
      R4<double> b;
      T dg;
      rhs_row(d, i, b, dg, es);
      d.b[i] = b;
      d.diag[i] = dg;
    }
    const double s = block_sum(es, shd);
    if (threadIdx.x == 0) d.e_partials[d.n_e_local + blockIdx.x] = s;
  }
}

// End of an outer iteration (one thread): the energy into this iteration's
// record, the iteration count, and the per-iteration words reset.
template <typename T>
__device__ __forceinline__ void finalize_iteration(const Dev<T>& d, double energy) {
  Ctrl* c = d.ctrl;
  IterRec* rec = d.hist + (c->iter % d.hist_cap);
  rec->energy = energy;
  if (!isfinite(energy) && d.stats) c->status |= ST_NONFINITE;
  c->iter += 1;
  c->n_cast = 0;
  for (int j = 0; j < 3; ++j) {
    c->box_lo[j] = 0x7FFFFFFFFFFFFFFFLL;
    c->box_hi[j] = (long long)0x8000000000000000ULL;
  }
  IterRec* nx = d.hist + (c->iter % d.hist_cap);
  nx->energy = 0.0;
  nx->pcg_rel_residual = 0.0;
  nx->n_self_pairs = 0;
  nx->n_obstacle_pairs = 0;
  nx->n_springs = 0;
  nx->pcg_iters = 0;
  nx->knot_sig = 0;
  nx->spring_sig = 0;
}

// ------------------------------------------------------------------ PCG
//
// The PCG kernels solve for the correction d of the warm start x:
//   r0 = b - A x  in FP64 (FP32 products are exact in FP64),
//   A d = r0      by Jacobi-preconditioned CG in the working precision,
//   x <- x + d    once at the end,
// so that the rounding of the working precision applies to the small
// correction, not to the positions (one step of mixed-precision iterative
// refinement per outer iteration).  The stopping test ||r|| <= tol ||b|| is the
// same as for the plain system.
//
// Per CG iteration there are two grid barriers: one publishes the new
// preconditioned residual u for the neighbours' SpMV, one completes the
// reduction of (r.u, w.u, r.r).
//
// Grid barrier: one arrival counter whose top bit flips once per round.
// Block 0 adds 0x80000000 - (nblocks - 1) and every other block adds 1, so a
// full round adds exactly 0x80000000: the low bits return to their value and
// the top bit changes, which every block waits for (no reset, one atomic per
// block).  Every wait is bounded by a clock budget, after which the kernel
// records ST_TIMEOUT, raises the abort word and returns.
//
// Reductions: each block forms its sums (below), lane 0 of warp 0 stores them
// as the block's partials and arrives; after the barrier warp 0 alone adds the
// partials in block order (deterministic), computes the CG scalars once for
// the block and hands them to the other warps through shared memory.  Partials
// are stored value-major, partials[(parity * 4 + k) * nblocks + block], in two
// buffers chosen by the barrier count's parity.
struct GridCtx {
  Ctrl* ctrl;
  double* partials;
  unsigned nblocks;
  unsigned long long budget;
  unsigned extra;  // test-only: arrivals expected beyond the grid (never come)
};

// One thread of the block arrives and waits for the round to complete.
// Returns 0 when the wait gave up (timeout) or another block aborted.
__device__ __forceinline__ int arrive_and_wait(const GridCtx& g) {
  const unsigned add = blockIdx.x == 0 ? (0x80000000u - (g.nblocks - 1u + g.extra)) : 1u;
  __threadfence();
  const unsigned old = atomicAdd(&g.ctrl->bar_count, add);
  volatile unsigned* vc = &g.ctrl->bar_count;
  int ok = 1;
  if (((old ^ *vc) & 0x80000000u) == 0) {
    const long long t0 = clock64();
    unsigned spins = 0;
    while (((old ^ *vc) & 0x80000000u) == 0) {
      if ((++spins & 63u) == 0) {
        if (*(volatile int*)&g.ctrl->abort) {
          ok = 0;
          break;
        }
        if ((unsigned long long)(clock64() - t0) > g.budget) {
          atomicExch(&g.ctrl->abort, 1);
          atomicOr(&g.ctrl->status, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
  }
  __threadfence();
  return ok;
}

// Plain grid barrier (makes every block's prior global writes visible).
__device__ __forceinline__ bool grid_barrier(const GridCtx& g, unsigned& epoch, int* shf) {
  ++epoch;
  __syncthreads();
  if (threadIdx.x == 0) *shf = arrive_and_wait(g);
  __syncthreads();
  return *shf != 0;
}

// per-thread accumulator of the CG dot products for vectors of type T
template <typename T>
struct DotAcc;
template <>
struct DotAcc<float> {
  using type = DW;
};
template <>
struct DotAcc<double> {
  using type = double;
};

// Called by all of warp 0 after block_sums.  Lane 0 stores the block's sums
// as its partials, arrives and waits; the warp then adds the partials of
// blocks [b0, b1) in block order: each lane its blocks in increasing order,
// then a fixed shuffle tree.  tot is valid in lane 0.  Returns false
// (warp-uniform) when the wait gave up or another block aborted.
template <int NV>
__device__ __forceinline__ bool warp0_reduce(const GridCtx& g, unsigned& epoch, const double (&bs)[NV], int b0,
                                             int b1, double (&tot)[NV]) {
  ++epoch;
  const int lane = threadIdx.x & 31;
  const size_t nb = g.nblocks;
  const double* buf = g.partials + (size_t)(epoch & 1u) * 4 * nb;
  int ok = 1;
  if (lane == 0) {
    double* wb = g.partials + (size_t)(epoch & 1u) * 4 * nb;
#pragma unroll
    for (int k = 0; k < NV; ++k) wb[k * nb + blockIdx.x] = bs[k];
    ok = arrive_and_wait(g);
  }
  __syncwarp();
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return false;
  double a[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) a[k] = 0.0;
#pragma unroll 2
  for (int b = b0 + lane; b < b1; b += 32) {
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] += __ldcg(buf + k * nb + b);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    tot[k] = a[k];
  }
  return true;
}

enum { CG_CONTINUE = 0, CG_DONE = 1, CG_NONFINITE = 2, CG_ABORT = 3 };

// CG scalars after the reduction of (gamma_k, delta_k, rr), by all of warp 0
// (inputs read from lane 0, outputs in every lane).
// alpha_k = gamma_k / (delta_k - beta_k gamma_k / alpha_{k-1}) with
// beta_k = gamma_k / gamma_{k-1}, rearranged with q = gamma_{k-1} alpha_{k-1}
// to alpha_k = gamma_k q / (delta_k q - gamma_k^2); lanes 0 and 1 form
// alpha_k's and beta_k's quotients in the same division, so one FP64
// division lies on the dependent path.
__device__ __forceinline__ int cg_scalars_warp(const double (&t)[3], double bb_l0, double tol2, double& gamma,
                                               double& alpha, double& beta, double& rr) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const double gnew = __shfl_sync(full, t[0], 0), delta = __shfl_sync(full, t[1], 0);
  const double bb = __shfl_sync(full, bb_l0, 0);
  const double g = __shfl_sync(full, gamma, 0), a = __shfl_sync(full, alpha, 0);
  rr = __shfl_sync(full, t[2], 0);
  gamma = g;
  alpha = a;
  if (!isfinite(gnew) || !isfinite(delta) || !isfinite(rr)) return CG_NONFINITE;
  if (rr <= tol2 * bb) return CG_DONE;
  const double q = g * a;
  const double num = lane == 1 ? gnew : gnew * q;
  const double den = lane == 1 ? g : delta * q - gnew * gnew;
  const double quo = num / den;
  beta = __shfl_sync(full, quo, 1);
  alpha = __shfl_sync(full, quo, 0);
  gamma = gnew;
  return CG_CONTINUE;
}

// The same CG scalars in double-word arithmetic on the FP32 pipes, for the
// dataflow kernel (its dot sums are double words already): an FP64 division
// and the FP64 products around it form a long dependent chain on this part,
// which every CG iteration waits for.  The state (gamma, alpha) lives in
// shared memory (st[0], st[1]); the stopping test compares ||r||^2 with the
// FP32 threshold thr = tol^2 ||b||^2.  Inputs from lane 0, by all of warp 0;
// lane 0 stores the new state and rr (st[2]).  Outputs: alpha_k and beta_k
// rounded to FP32 (valid in every lane).
__device__ __forceinline__ int cg_scalars_dw(const DW (&t)[3], float thr, DW* st, float& ta, float& tb) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const DW gnew{__shfl_sync(full, t[0].hi, 0), __shfl_sync(full, t[0].lo, 0)};
  const DW delta{__shfl_sync(full, t[1].hi, 0), __shfl_sync(full, t[1].lo, 0)};
  const DW rr{__shfl_sync(full, t[2].hi, 0), __shfl_sync(full, t[2].lo, 0)};
  if (lane == 0) st[2] = rr;
  if (!isfinite(gnew.hi) || !isfinite(delta.hi) || !isfinite(rr.hi)) return CG_NONFINITE;
  if (rr.hi <= thr) return CG_DONE;
  const DW g = st[0], a = st[1];
  const DW q = dw_mul(g, a);
  const DW num = lane == 1 ? gnew : dw_mul(gnew, q);
  const DW den = lane == 1 ? g : dw_add_sloppy(dw_mul(delta, q), dw_neg(dw_mul(gnew, gnew)));
  const DW quo = dw_div(num, den);
  const DW alpha{__shfl_sync(full, quo.hi, 0), __shfl_sync(full, quo.lo, 0)};
  tb = __shfl_sync(full, quo.hi, 1);
  ta = alpha.hi;
  if (lane == 0) {
    st[0] = gnew;
    st[1] = alpha;
  }
  return CG_CONTINUE;
}

// shared state of one block of a PCG kernel
template <typename T>
struct CgShared {
  double sh[96];
  T ta, tb;
  int flag;
  int ok;
};

template <typename T>
__device__ __forceinline__ R4<T> ld_cg(const R4<T>* a);
template <>
__device__ __forceinline__ R4<float> ld_cg<float>(const R4<float>* a) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(a));
  return R4<float>{v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ R4<double> ld_cg<double>(const R4<double>* a) {
  const double2 v0 = __ldcg(reinterpret_cast<const double2*>(a));
  const double2 v1 = __ldcg(reinterpret_cast<const double2*>(a) + 1);
  return R4<double>{v0.x, v0.y, v1.x, v1.y};
}

__device__ __forceinline__ void write_pcg_record(const Ctrl* c, IterRec* hist, int cap, Ctrl* cw, int it, double rr,
                                                 double bb) {
  IterRec* rec = hist + (c->iter % cap);
  rec->pcg_iters = it;
  cw->total_pcg += it;
  rec->pcg_rel_residual = bb > 0.0 ? sqrt(rr / bb) : 0.0;
}

// The solve's starting point for free row i: x_i, plus the last outer
// iteration's step x_i - x_(i-1) where one is kept (an outer iteration's
// solve in MIXED mode; null otherwise).  The local-global iteration
// approaches its fixed point along a slowly turning direction, so
// x_i + (x_i - x_(i-1)) is a closer guess for x_(i+1) than x_i: the solve
// still stops at the same relative residual, from a smaller first one.  The
// same rounded sums in every row that reads it.
template <typename T>
__device__ __forceinline__ R4<T> warm_start(const Dev<T>& d, int i, R4<T> xi) {
  if (d.xstep) {
    const R4<T> s = d.xstep[i];
    xi.x += s.x;
    xi.y += s.y;
    xi.z += s.z;
  }
  return xi;
}

// r_i = b_i - (A x)_i in FP64, x the solve's starting point, and ||b_i||^2,
// ||r_i||^2 (the first residual of the correction form; X is read-only while
// it is formed).
template <typename T>
__device__ __forceinline__ void residual_row_f64(const Dev<T>& d, int i, T dg, double (&rv)[3], double (&a0)[2],
                                                 const R4<double>* b_in = nullptr) {
  const R4<T> xi = warm_start(d, i, d.X[i]);
  double ax = (double)dg * xi.x, ay = (double)dg * xi.y, az = (double)dg * xi.z;
  const int sl = i >> 5, lane = i & 31;
  const int k1 = d.sl_ptr[sl + 1];
  for (int k = d.sl_ptr[sl] + lane; k < k1; k += 32) {
    const double a = (double)d.sl_val[k];
    const int col = chk_idx(d.ctrl, d.sl_col[k], d.n_free);
    const R4<T> xc = warm_start(d, col, d.X[col]);
    ax += a * xc.x;
    ay += a * xc.y;
    az += a * xc.z;
  }
  const R4<double> bi = b_in ? *b_in : d.b[i];
  rv[0] = bi.x - ax;
  rv[1] = bi.y - ay;
  rv[2] = bi.z - az;
  a0[0] += bi.x * bi.x + bi.y * bi.y + bi.z * bi.z;
  a0[1] += rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2];
}

// Right-hand side, diagonal and first residual of row i for FP32 positions,
// in double-word arithmetic on the FP32 pipes (FP64 arithmetic is scarce on
// this part, and these rows lie on every block's path to the first
// reduction): b_i = sum of the row's P_e columns (FP32 values added by
// TwoSum) + k mask_i c_i - bfix_i (the last two in FP64, only where nonzero),
// A_ii = diagL_i + k mask_i, r_i = b_i - (A x)_i with the products exact
// (TwoProd), and the row's ||b_i||^2, ||r_i||^2 and spring energy as double
// words.  val holds the row's off-diagonal values (sliced ELL, `width`
// entries); about 48 significant bits throughout, far beyond what the FP32
// CG needs from its right-hand side.
template <int MAXW>
__device__ __forceinline__ void rhs_residual_row_dw(const Dev<float>& d, int i, const float (&val)[MAXW], int width,
                                                    float& dg, float (&r)[3], DW (&a0)[3]) {
  DW b[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  const int k1 = d.inc_ptr[i + 1];
#pragma unroll 8
  for (int k = d.inc_ptr[i]; k < k1; ++k) {
    const R4<float> p = d.P[chk_idx(d.ctrl, d.inc[k], 4 * d.n_t)];
    dw_acc(b[0], p.x);
    dw_acc(b[1], p.y);
    dw_acc(b[2], p.z);
  }
  const R4<double> sc = d.spring_c[i];
  const double km = d.k_spring * sc.w;
  const R4<double> bf = d.bfix[i];
  const R4<float> xi = d.X[i];
  const R4<float> xs = warm_start(d, i, xi);  // the solve's starting point
  dg = d.diagL[i] + (float)km;
  DW es{0.0f, 0.0f};
  if (km != 0.0) {
    const double cv[3] = {sc.x, sc.y, sc.z};
    for (int c = 0; c < 3; ++c) b[c] = dw_add_sloppy(dw_norm(b[c]), dw_from(km * cv[c]));
    const double ex = (double)xi.x - sc.x, ey = (double)xi.y - sc.y, ez = (double)xi.z - sc.z;
    es = dw_from(km * (ex * ex + ey * ey + ez * ez));
  }
  if (bf.x != 0.0 || bf.y != 0.0 || bf.z != 0.0) {
    const double fv[3] = {bf.x, bf.y, bf.z};
    for (int c = 0; c < 3; ++c) b[c] = dw_add_sloppy(dw_norm(b[c]), dw_neg(dw_from(fv[c])));
  }
  DW ax[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  dw_acc_prod(ax[0], dg, xs.x);
  dw_acc_prod(ax[1], dg, xs.y);
  dw_acc_prod(ax[2], dg, xs.z);
  const int sl = i >> 5, ln = i & 31;
  const int base = d.sl_ptr[sl];
#pragma unroll
  for (int j = 0; j < MAXW; ++j) {
    if (j < width) {
      const int col = chk_idx(d.ctrl, d.sl_col[base + j * 32 + ln], d.n_free);
      const R4<float> xc = warm_start(d, col, d.X[col]);
      dw_acc_prod(ax[0], val[j], xc.x);
      dw_acc_prod(ax[1], val[j], xc.y);
      dw_acc_prod(ax[2], val[j], xc.z);
    }
  }
  DW rw[3];
  for (int c = 0; c < 3; ++c) {
    b[c] = dw_norm(b[c]);
    rw[c] = dw_add_sloppy(b[c], dw_neg(dw_norm(ax[c])));
    r[c] = rw[c].hi;
  }
  a0[0] = dot3(b[0].hi, b[1].hi, b[2].hi, b[0].hi, b[1].hi, b[2].hi);
  a0[1] = dot3(rw[0].hi, rw[1].hi, rw[2].hi, rw[0].hi, rw[1].hi, rw[2].hi);
  a0[2] = es;
}

// Streaming variant: any number of rows per thread (grid-stride); vectors in
// HBM/L2, off-diagonals read from the sliced-ELL arrays every SpMV.
template <typename T>
__device__ __forceinline__ void spmv_row(const Dev<T>& d, int i, const R4<T>* __restrict__ src, T dg,
                                         const R4<T>& self, T& ax, T& ay, T& az) {
  ax = dg * self.x;
  ay = dg * self.y;
  az = dg * self.z;
  const int s = i >> 5, lane = i & 31;
  const int k1 = d.sl_ptr[s + 1];
  for (int k = d.sl_ptr[s] + lane; k < k1; k += 32) {
    const int c = chk_idx(d.ctrl, d.sl_col[k], d.n_v);
    const T a = d.sl_val[k];
    const R4<T> x = ld_cg<T>(src + c);
    ax += a * x.x;
    ay += a * x.y;
    az += a * x.z;
  }
}

template <typename T>
__global__ void __launch_bounds__(PCG_THREADS, 1) k_pcg(Dev<T> d) {
  using A = typename DotAcc<T>::type;
  constexpr int NW = PCG_THREADS / 32;
  __shared__ CgShared<T> cs;
  const GridCtx g{d.ctrl, d.partials, gridDim.x, d.wait_budget, d.bar_extra};
  unsigned epoch = 0;
  const int lane = threadIdx.x & 31;
  const bool w0 = threadIdx.x < 32;
  const int n = d.n_free;
  const int G = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  R4<T>* __restrict__ X = d.X;
  R4<T>* __restrict__ r = d.r;
  R4<T>* __restrict__ u = d.u;
  R4<T>* __restrict__ p = d.p;
  R4<T>* __restrict__ s = d.s;
  R4<T>* __restrict__ w = d.w;
  R4<T>* __restrict__ dx = d.dx;
  const R4<T> zero = {T(0), T(0), T(0), T(0)};
  // CG scalars: meaningful in lane 0 of warp 0
  double bb = 0.0, rr = 0.0, gamma = 0.0, alpha = 0.0, beta = 0.0;

  // r = b - A x in FP64, u = M^-1 r, d = 0
  double a0[2] = {0.0, 0.0};
  for (int i = tid; i < n; i += G) {
    const T dg = d.diag[i];
    double rv[3];
    residual_row_f64(d, i, dg, rv, a0);
    R4<T> ri, ui;
    ri.x = (T)rv[0]; ri.y = (T)rv[1]; ri.z = (T)rv[2]; ri.w = T(0);
    ui.x = ri.x / dg; ui.y = ri.y / dg; ui.z = ri.z / dg; ui.w = T(0);
    r[i] = ri;
    u[i] = ui;
    dx[i] = zero;
  }
  {
    double bs[2], t[2];
    block_sums<2, NW>(a0, cs.sh, bs);
    if (w0) {
      const bool ok = warp0_reduce<2>(g, epoch, bs, 0, gridDim.x, t);
      if (lane == 0) {
        bb = t[0];
        rr = t[1];
        cs.flag = !ok ? CG_ABORT : ((bb > 0.0 && rr > d.tol2 * bb) ? CG_CONTINUE : CG_DONE);
      }
    }
    __syncthreads();
  }
  if (cs.flag == CG_ABORT) return;
  int it = 0;
  if (cs.flag == CG_CONTINUE) {
    A a1[2] = {acc_zero<A>(), acc_zero<A>()};
    for (int i = tid; i < n; i += G) {
      const T dg = d.diag[i];
      const R4<T> ui = u[i], ri = r[i];
      T ax, ay, az;
      spmv_row(d, i, u, dg, ui, ax, ay, az);
      R4<T> wi;
      wi.x = ax; wi.y = ay; wi.z = az; wi.w = T(0);
      w[i] = wi;
      a1[0] = acc_add(a1[0], dot3(ri.x, ri.y, ri.z, ui.x, ui.y, ui.z));
      a1[1] = acc_add(a1[1], dot3(ax, ay, az, ui.x, ui.y, ui.z));
    }
    {
      double bs[2], t[2];
      block_sums<2, NW>(a1, cs.sh, bs);
      if (w0) {
        const bool ok = warp0_reduce<2>(g, epoch, bs, 0, gridDim.x, t);
        if (lane == 0) {
          if (ok) {
            gamma = t[0];
            alpha = gamma / t[1];
            cs.ta = (T)alpha;
            cs.tb = T(0);
          }
          cs.flag = ok ? CG_CONTINUE : CG_ABORT;
        }
      }
      __syncthreads();
    }
    if (cs.flag == CG_ABORT) return;
    T ta = cs.ta, tb = T(0);
    bool first = true;
    for (it = 1; it <= d.max_iter; ++it) {
      for (int i = tid; i < n; i += G) {
        const R4<T> ui = u[i], wi = w[i];
        R4<T> pi, si;
        if (first) {
          pi = ui;
          si = wi;
        } else {
          const R4<T> po = p[i], so = s[i];
          pi.x = ui.x + tb * po.x; pi.y = ui.y + tb * po.y; pi.z = ui.z + tb * po.z;
          si.x = wi.x + tb * so.x; si.y = wi.y + tb * so.y; si.z = wi.z + tb * so.z;
        }
        pi.w = T(0);
        si.w = T(0);
        p[i] = pi;
        s[i] = si;
        R4<T> di = dx[i], ri = r[i];
        di.x += ta * pi.x; di.y += ta * pi.y; di.z += ta * pi.z;
        ri.x -= ta * si.x; ri.y -= ta * si.y; ri.z -= ta * si.z;
        dx[i] = di;
        r[i] = ri;
        const T dg = d.diag[i];
        R4<T> un;
        un.x = ri.x / dg; un.y = ri.y / dg; un.z = ri.z / dg; un.w = T(0);
        u[i] = un;
      }
      if (!grid_barrier(g, epoch, &cs.ok)) return;
      A a2[3] = {acc_zero<A>(), acc_zero<A>(), acc_zero<A>()};
      for (int i = tid; i < n; i += G) {
        const T dg = d.diag[i];
        const R4<T> ui = u[i], ri = r[i];
        T ax, ay, az;
        spmv_row(d, i, u, dg, ui, ax, ay, az);
        R4<T> wi;
        wi.x = ax; wi.y = ay; wi.z = az; wi.w = T(0);
        w[i] = wi;
        a2[0] = acc_add(a2[0], dot3(ri.x, ri.y, ri.z, ui.x, ui.y, ui.z));
        a2[1] = acc_add(a2[1], dot3(ax, ay, az, ui.x, ui.y, ui.z));
        a2[2] = acc_add(a2[2], dot3(ri.x, ri.y, ri.z, ri.x, ri.y, ri.z));
      }
      {
        double bs[3], t[3];
        block_sums<3, NW>(a2, cs.sh, bs);
        if (w0) {
          const bool ok = warp0_reduce<3>(g, epoch, bs, 0, gridDim.x, t);
          int f = CG_ABORT;
          if (ok) f = cg_scalars_warp(t, bb, d.tol2, gamma, alpha, beta, rr);
          if (lane == 0) {
            if (ok) {
              if (f == CG_NONFINITE && blockIdx.x == 0) set_status(d.ctrl, ST_NONFINITE);
              cs.ta = (T)alpha;
              cs.tb = (T)beta;
            }
            cs.flag = f;
          }
        }
        __syncthreads();
      }
      const int f = cs.flag;
      if (f == CG_ABORT) return;
      if (f != CG_CONTINUE) break;
      ta = cs.ta;
      tb = cs.tb;
      first = false;
    }
    if (it > d.max_iter) {
      it = d.max_iter;
      if (tid == 0) set_status(d.ctrl, ST_PCG_MAXIT);
    }
    for (int i = tid; i < n; i += G) {
      R4<T> xi = X[i];
      const R4<T> di = dx[i];
      xi.x += di.x; xi.y += di.y; xi.z += di.z;
      X[i] = xi;
    }
  }
  if (tid == 0) write_pcg_record(d.ctrl, d.hist, d.hist_cap, d.ctrl, it, rr, bb);
}

// Register-resident variant: one row per thread.  The thread keeps its
// sliced-ELL row, diagonal and all CG vectors in registers for the whole
// solve; per iteration only the preconditioned residual u is written to
// memory and the neighbours' values are gathered from L2.
template <typename T, int MAXW>
__global__ void __launch_bounds__(PCG_RR_THREADS, 2) k_pcg_rr(Dev<T> d) {
  using A = typename DotAcc<T>::type;
  constexpr int NW = PCG_RR_THREADS / 32;
  __shared__ CgShared<T> cs;
  const GridCtx g{d.ctrl, d.partials, gridDim.x, d.wait_budget, d.bar_extra};
  unsigned epoch = 0;
  const int lane = threadIdx.x & 31;
  const bool w0 = threadIdx.x < 32;
  const int n = d.n_free;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < n;
  int col[MAXW];
  T val[MAXW];
  int width = 0;
  T dg = T(1);
  T x[3] = {T(0), T(0), T(0)};
  if (act) {
    const int sl = i >> 5, ln = i & 31;
    const int base = d.sl_ptr[sl];
    width = (d.sl_ptr[sl + 1] - base) >> 5;
#pragma unroll
    for (int j = 0; j < MAXW; ++j) {
      if (j < width) {
        col[j] = d.sl_col[base + j * 32 + ln];
        val[j] = d.sl_val[base + j * 32 + ln];
      } else {
        col[j] = i;
        val[j] = T(0);
      }
    }
    dg = d.diag[i];
    const R4<T> xi = d.X[i];
    x[0] = xi.x; x[1] = xi.y; x[2] = xi.z;
  }
  auto spmv = [&](const R4<T>* src, const T (&self)[3], T (&ax)[3]) {
    ax[0] = dg * self[0];
    ax[1] = dg * self[1];
    ax[2] = dg * self[2];
#pragma unroll
    for (int j = 0; j < MAXW; ++j) {
      if (j < width) {
        const R4<T> v = ld_cg<T>(src + col[j]);
        ax[0] += val[j] * v.x;
        ax[1] += val[j] * v.y;
        ax[2] += val[j] * v.z;
      }
    }
  };
  auto store_u = [&](const T (&uu)[3]) {
    R4<T> t;
    t.x = uu[0]; t.y = uu[1]; t.z = uu[2]; t.w = T(0);
    d.u[i] = t;
  };
  // CG scalars: meaningful in lane 0 of warp 0
  double bb = 0.0, rr = 0.0, gamma = 0.0, alpha = 0.0, beta = 0.0;
  T r[3], u[3], w[3], p[3], s[3], dd[3] = {T(0), T(0), T(0)};
  double a0[2] = {0.0, 0.0};
  if (act) {
    double rv[3];
    residual_row_f64(d, i, dg, rv, a0);
    for (int c = 0; c < 3; ++c) {
      r[c] = (T)rv[c];
      u[c] = r[c] / dg;
    }
    store_u(u);
  }
  {
    double bs[2], t[2];
    block_sums<2, NW>(a0, cs.sh, bs);
    if (w0) {
      const bool ok = warp0_reduce<2>(g, epoch, bs, 0, gridDim.x, t);
      if (lane == 0) {
        bb = t[0];
        rr = t[1];
        cs.flag = !ok ? CG_ABORT : ((bb > 0.0 && rr > d.tol2 * bb) ? CG_CONTINUE : CG_DONE);
      }
    }
    __syncthreads();
  }
  if (cs.flag == CG_ABORT) return;
  int it = 0;
  if (cs.flag == CG_CONTINUE) {
    A a1[2] = {acc_zero<A>(), acc_zero<A>()};
    if (act) {
      spmv(d.u, u, w);
      a1[0] = dot3(r[0], r[1], r[2], u[0], u[1], u[2]);
      a1[1] = dot3(w[0], w[1], w[2], u[0], u[1], u[2]);
      for (int c = 0; c < 3; ++c) {
        p[c] = u[c];
        s[c] = w[c];
      }
    }
    {
      double bs[2], t[2];
      block_sums<2, NW>(a1, cs.sh, bs);
      if (w0) {
        const bool ok = warp0_reduce<2>(g, epoch, bs, 0, gridDim.x, t);
        if (lane == 0) {
          if (ok) {
            gamma = t[0];
            alpha = gamma / t[1];
            cs.ta = (T)alpha;
          }
          cs.flag = ok ? CG_CONTINUE : CG_ABORT;
        }
      }
      __syncthreads();
    }
    if (cs.flag == CG_ABORT) return;
    T ta = cs.ta;
    for (it = 1; it <= d.max_iter; ++it) {
      if (act) {
        for (int c = 0; c < 3; ++c) {
          dd[c] += ta * p[c];
          r[c] -= ta * s[c];
          u[c] = r[c] / dg;
        }
        store_u(u);
      }
      if (!grid_barrier(g, epoch, &cs.ok)) return;
      A a2[3] = {acc_zero<A>(), acc_zero<A>(), acc_zero<A>()};
      if (act) {
        spmv(d.u, u, w);
        a2[0] = dot3(r[0], r[1], r[2], u[0], u[1], u[2]);
        a2[1] = dot3(w[0], w[1], w[2], u[0], u[1], u[2]);
        a2[2] = dot3(r[0], r[1], r[2], r[0], r[1], r[2]);
      }
      {
        double bs[3], t[3];
        block_sums<3, NW>(a2, cs.sh, bs);
        if (w0) {
          const bool ok = warp0_reduce<3>(g, epoch, bs, 0, gridDim.x, t);
          int f = CG_ABORT;
          if (ok) f = cg_scalars_warp(t, bb, d.tol2, gamma, alpha, beta, rr);
          if (lane == 0) {
            if (ok) {
              if (f == CG_NONFINITE && blockIdx.x == 0) set_status(d.ctrl, ST_NONFINITE);
              cs.ta = (T)alpha;
              cs.tb = (T)beta;
            }
            cs.flag = f;
          }
        }
        __syncthreads();
      }
      const int f = cs.flag;
      if (f == CG_ABORT) return;
      if (f != CG_CONTINUE) break;
      ta = cs.ta;
      const T tb = cs.tb;
      if (act)
        for (int c = 0; c < 3; ++c) {
          p[c] = u[c] + tb * p[c];
          s[c] = w[c] + tb * s[c];
        }
    }
    if (it > d.max_iter) {
      it = d.max_iter;
      if (i == 0) set_status(d.ctrl, ST_PCG_MAXIT);
    }
    if (act) {
      R4<T> t;
      t.x = x[0] + dd[0]; t.y = x[1] + dd[1]; t.z = x[2] + dd[2]; t.w = T(0);
      d.X[i] = t;
    }
  }
  if (i == 0) write_pcg_record(d.ctrl, d.hist, d.hist_cap, d.ctrl, it, rr, bb);
}

// ------------------------------------------------------- dataflow PCG (FP32)
// Register-resident CG (one row per thread) with one grid-wide wait per
// iteration instead of two.  The preconditioned residual u that neighbours
// read is published as epoch-tagged words: each row as two 8-byte words, a
// 16-bit epoch tag over 48 bits of payload (x, y, z in FP32).  Aligned 8-byte
// accesses are single-copy atomic, so a word whose tag matches holds that
// epoch's payload; a reader re-reads words that still carry an older tag
// (bounded waits), so the SpMV waits only for the rows it reads and needs no
// grid barrier.  Each block copies its halo (the distinct rows its SpMV
// reads, listed at upload) into shared memory with mostly contiguous loads,
// then multiplies from shared memory.  The reduction of (r.u, w.u, r.r) is
// one arrival on the grid counter (relaxed: no fences) after the block has
// stored its partials as tagged words; once the round completes, warp 0
// reads the partials (re-reading any whose tag is not yet current) and sums
// them in block order.  Words are double-buffered by epoch parity and zeroed
// before each launch.  No block is ever more than one epoch ahead of a
// reader of its words (it cannot pass a reduction before the reader has
// arrived, after its last read of the older epoch), so a stale word is at
// most two epochs old and its tag cannot match.  Sums and CG scalars are
// formed as in the barrier kernels (block order, fixed trees), so results do
// not depend on timing.
__device__ __forceinline__ void st_v2_relaxed(unsigned long long* p, unsigned long long a, unsigned long long b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void ld_v2_relaxed(const unsigned long long* p, unsigned long long& a,
                                              unsigned long long& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p));
}

// same load with the address base + 16 * idx formed inside the asm, so that
// the compiler keeps one index register per row, not one 64-bit address
__device__ __forceinline__ void ld_v2_relaxed_at(const unsigned long long* base, int idx, unsigned long long& a,
                                                 unsigned long long& b) {
  asm volatile(
      "{\n\t.reg .u64 ad;\n\t"
      "mad.wide.s32 ad, %2, 16, %3;\n\t"
      "ld.relaxed.gpu.global.v2.u64 {%0, %1}, [ad];\n\t}"
      : "=l"(a), "=l"(b)
      : "r"(idx), "l"(base));
}

__device__ __forceinline__ unsigned long long df_tag(unsigned e) { return (unsigned long long)(e & 0xFFFFu) << 48; }
__device__ __forceinline__ bool df_has(unsigned long long w, unsigned long long tag) {
  return (w & 0xFFFF000000000000ull) == tag;
}

// u row: w0 = tag | x | y[31:16], w1 = tag | y[15:0] | z
__device__ __forceinline__ void df_pack_u(unsigned long long tag, float x, float y, float z, unsigned long long& w0,
                                          unsigned long long& w1) {
  const unsigned bx = __float_as_uint(x), by = __float_as_uint(y), bz = __float_as_uint(z);
  w0 = tag | ((unsigned long long)bx << 16) | (by >> 16);
  w1 = tag | ((unsigned long long)(by & 0xFFFFu) << 32) | bz;
}
__device__ __forceinline__ void df_unpack_u(unsigned long long w0, unsigned long long w1, float& x, float& y,
                                            float& z) {
  x = __uint_as_float((unsigned)(w0 >> 16));
  y = __uint_as_float((((unsigned)w0 & 0xFFFFu) << 16) | ((unsigned)(w1 >> 32) & 0xFFFFu));
  z = __uint_as_float((unsigned)w1);
}

// three doubles (192 bits) as four 48-bit chunks under one tag each
__device__ __forceinline__ void df_pack_3d(unsigned long long tag, const double (&v)[3], unsigned long long (&w)[4]) {
  const unsigned long long b0 = __double_as_longlong(v[0]), b1 = __double_as_longlong(v[1]),
                           b2 = __double_as_longlong(v[2]);
  const unsigned long long m48 = 0xFFFFFFFFFFFFull;
  w[0] = tag | (b0 >> 16);
  w[1] = tag | ((b0 & 0xFFFFull) << 32) | (b1 >> 32);
  w[2] = tag | ((b1 & 0xFFFFFFFFull) << 16) | (b2 >> 48);
  w[3] = tag | (b2 & m48);
}
__device__ __forceinline__ void df_unpack_3d(const unsigned long long (&w)[4], double (&v)[3]) {
  const unsigned long long m48 = 0xFFFFFFFFFFFFull;
  const unsigned long long c0 = w[0] & m48, c1 = w[1] & m48, c2 = w[2] & m48, c3 = w[3] & m48;
  v[0] = __longlong_as_double((long long)((c0 << 16) | (c1 >> 32)));
  v[1] = __longlong_as_double((long long)(((c1 & 0xFFFFFFFFull) << 32) | (c2 >> 16)));
  v[2] = __longlong_as_double((long long)(((c2 & 0xFFFFull) << 48) | c3));
}

// Bounded polling: every 32nd poll checks the abort word and the clock budget
// (on expiry records ST_TIMEOUT and raises abort).  Returns false to stop.
struct DfWait {
  long long t0 = 0;
  unsigned n = 0;
  __device__ __forceinline__ bool again(Ctrl* c, unsigned long long budget) {
    if ((++n & 31u) != 0) return true;
    if (*(volatile int*)&c->abort) return false;
    const long long now = clock64();
    if (t0 == 0) {
      t0 = now;
      return true;
    }
    if ((unsigned long long)(now - t0) > budget) {
      atomicExch(&c->abort, 1);
      atomicOr(&c->status, ST_TIMEOUT);
      return false;
    }
    return true;
  }
};

static constexpr int DF_MAXQ = 5;  // partial slots per lane of warp 0: up to 160 blocks

// Warp 0: lane 0 stores the block's sums under epoch e and arrives on the
// grid counter, then waits for the round to complete.  The arrival is a
// fire-and-forget add: after round e (counted from 1 in each launch) the
// counter's top bit equals e & 1, because the counter starts at zero and
// every complete round adds 2^31 (block 0 adds 2^31 - (nblocks - 1), the
// others 1), so the top bit flips exactly when a round's last arrival lands.
// Once the round is complete every lane reads its blocks' slots (lane,
// lane + 32, ...), re-reading any that do not yet carry epoch e, and adds them
// in block order; a fixed shuffle tree gives tot in lane 0.  The sums are FP64
// (S = double) or double words added on the FP32 pipes (S = DW; three DW
// values fill the same four words).  Returns false (warp-uniform) when a wait
// gave up or another block aborted.
__device__ __forceinline__ void df_pack(unsigned long long tag, const double (&v)[3], unsigned long long (&w)[4]) {
  df_pack_3d(tag, v, w);
}
__device__ __forceinline__ void df_pack(unsigned long long tag, const DW (&v)[3], unsigned long long (&w)[4]) {
  double x[3];
  for (int k = 0; k < 3; ++k)
    x[k] = __longlong_as_double((long long)(((unsigned long long)__float_as_uint(v[k].hi) << 32) |
                                            __float_as_uint(v[k].lo)));
  df_pack_3d(tag, x, w);
}
__device__ __forceinline__ void df_unpack(const unsigned long long (&w)[4], double (&v)[3]) { df_unpack_3d(w, v); }
__device__ __forceinline__ void df_unpack(const unsigned long long (&w)[4], DW (&v)[3]) {
  double x[3];
  df_unpack_3d(w, x);
  for (int k = 0; k < 3; ++k) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[k]);
    v[k] = DW{__uint_as_float((unsigned)(b >> 32)), __uint_as_float((unsigned)b)};
  }
}
__device__ __forceinline__ double df_add(double a, double b) { return a + b; }
__device__ __forceinline__ DW df_add(DW a, DW b) { return dw_add_sloppy(a, b); }

template <typename S>
__device__ __forceinline__ bool df_reduce(const Dev<float>& d, unsigned e, const S (&bs)[3], S (&tot)[3]) {
  const int lane = threadIdx.x & 31;
  const int nb = gridDim.x;
  unsigned long long* buf = d.df_p + (size_t)(e & 1u) * 4 * (size_t)nb;
  const unsigned long long tag = df_tag(e);
  int arrived = 1;
  if (lane == 0) {
    unsigned long long w[4];
    df_pack(tag, bs, w);
    st_v2_relaxed(buf + 4 * (size_t)blockIdx.x, w[0], w[1]);
    st_v2_relaxed(buf + 4 * (size_t)blockIdx.x + 2, w[2], w[3]);
    const unsigned add = blockIdx.x == 0 ? (0x80000000u - ((unsigned)nb - 1u + d.bar_extra)) : 1u;
    atomicAdd(&d.ctrl->bar_count, add);  // result unused: issued as a reduction
    const unsigned want = (e & 1u) << 31;
    volatile unsigned* vc = &d.ctrl->bar_count;
    DfWait wt;
    while ((*vc & 0x80000000u) != want)
      if (!wt.again(d.ctrl, d.wait_budget)) {
        arrived = 0;
        break;
      }
  }
  if (!__shfl_sync(0xffffffffu, arrived, 0)) return false;
  unsigned long long w[DF_MAXQ][4];
#pragma unroll
  for (int q = 0; q < DF_MAXQ; ++q) {
    const int b = lane + 32 * q;
    if (b < nb) {
      ld_v2_relaxed(buf + 4 * (size_t)b, w[q][0], w[q][1]);
      ld_v2_relaxed(buf + 4 * (size_t)b + 2, w[q][2], w[q][3]);
    }
  }
  // slots whose store is not yet visible: re-read them all, then re-check
  auto fresh = [&](int q) {
    return df_has(w[q][0], tag) && df_has(w[q][1], tag) && df_has(w[q][2], tag) && df_has(w[q][3], tag);
  };
  unsigned stale = 0;
#pragma unroll
  for (int q = 0; q < DF_MAXQ; ++q)
    if (lane + 32 * q < nb && !fresh(q)) stale |= 1u << q;
  DfWait wt;
  while (stale != 0 && wt.again(d.ctrl, d.wait_budget)) {
#pragma unroll
    for (int q = 0; q < DF_MAXQ; ++q)
      if (stale & (1u << q)) {
        const int b = lane + 32 * q;
        ld_v2_relaxed(buf + 4 * (size_t)b, w[q][0], w[q][1]);
        ld_v2_relaxed(buf + 4 * (size_t)b + 2, w[q][2], w[q][3]);
      }
#pragma unroll
    for (int q = 0; q < DF_MAXQ; ++q)
      if ((stale & (1u << q)) && fresh(q)) stale &= ~(1u << q);
  }
  if (!__all_sync(0xffffffffu, stale == 0)) return false;
  S a[3] = {acc_zero<S>(), acc_zero<S>(), acc_zero<S>()};
#pragma unroll
  for (int q = 0; q < DF_MAXQ; ++q) {
    if (lane + 32 * q < nb) {
      S v[3];
      df_unpack(w[q], v);
      a[0] = df_add(a[0], v[0]);
      a[1] = df_add(a[1], v[1]);
      a[2] = df_add(a[2], v[2]);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] = df_add(a[k], shfl_down(a[k], o));
    tot[k] = a[k];
  }
  return true;
}


// ---- two-level preconditioner of the dataflow kernel ----------------------
// M^-1 = D^-1 + Z A_c^-1 Z^T: Jacobi plus an additive coarse correction over
// aggregates of ROWS / 3 consecutive rows (compact pieces of the body: the
// free rows are numbered by recursive coordinate bisection), Z the 0/1
// aggregation matrix and A_c = Z^T L Z the Galerkin coarse matrix of the
// spring-free Laplacian (both SPD, so M is SPD: A + k diag(mask) >= L only
// makes the coarse part an approximation).  A_c^-1 is formed once at upload.
// Per CG iteration every block needs g_i = (A_c^-1 Z^T v)_{a_i} for its own
// aggregates a_i and v = r_{k+1}, before r_{k+1}'s SpMV.  With
// r_{k+1} = r_k - alpha_k s_k and s_k = w_k + beta_k s_{k-1} (w = A u),
// g(r_{k+1}) = g(r_k) - alpha_k g(s_k) and g(s_k) = g(w_k) + beta_k g(s_{k-1}):
// every block adds its aggregates' sums of w_k and r_k to the slot it
// publishes in the reduction it already makes, so g(r_k) and g(w_k) are
// formed fresh from that round's sums (only g(s) is carried, like s itself),
// and the coarse correction costs no extra grid-wide wait.
static constexpr int DF_AGG = 3;                 // aggregates per block (of ROWS / 3 rows each)
static constexpr int DF_SLOT_C = 4 + 4 * DF_AGG;  // slot words with the aggregate sums
static constexpr int SEG_AGG_ROWS = 128;         // aggregate rows of the segmented batch kernel

// All threads: per-warp sums of w and r over the warp's rows (fixed shuffle
// trees), stored by lane 0 in sz[warp]; call before block_sums*, whose
// __syncthreads publishes them.
__device__ __forceinline__ void agg_warp_sums(const float (&w)[3], const float (&r)[3], float (*sz)[6]) {
  // reduce-scatter butterfly over the six values (padded to eight): the
  // lanes give up half their values at distances 16, 8 and 4 and finish the
  // one left at 2 and 1; the pairs added, and so the sums, are those of a
  // shuffle-down tree over distances 16, 8, 4, 2, 1 (9 exchanges instead of
  // 30); value c ends in lanes 4c .. 4c + 3
  const int lane = threadIdx.x & 31;
  const float a[8] = {w[0], w[1], w[2], r[0], r[1], r[2], 0.0f, 0.0f};
  float b[4], c2[2];
  const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    b[k] = __fadd_rn(u16 ? a[4 + k] : a[k], __shfl_xor_sync(0xffffffffu, u16 ? a[k] : a[4 + k], 16));
#pragma unroll
  for (int k = 0; k < 2; ++k)
    c2[k] = __fadd_rn(u8 ? b[2 + k] : b[k], __shfl_xor_sync(0xffffffffu, u8 ? b[k] : b[2 + k], 8));
  float x = __fadd_rn(u4 ? c2[1] : c2[0], __shfl_xor_sync(0xffffffffu, u4 ? c2[0] : c2[1], 4));
  x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, 2));
  x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, 1));
  if ((lane & 3) == 0 && (lane >> 2) < 6) sz[threadIdx.x >> 5][lane >> 2] = x;
}

// The slots are stored in PCG_DF_REPLICAS copies and block b reads copy
// b % PCG_DF_REPLICAS: every block reads every slot once per round, and
// spreading those reads over copies at different addresses (different L2
// slices) shortens the queue of reads of one slot.
__device__ __forceinline__ unsigned long long* df_slots(const Dev<float>& d, unsigned e, int copy) {
  const size_t nb = gridDim.x;
  return d.df_p + ((size_t)copy * 2 + (e & 1u)) * DF_SLOT_C * (nb + 1);
}
__device__ __forceinline__ double shfl0(double v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ DW shfl0(DW v) {
  return DW{__shfl_sync(0xffffffffu, v.hi, 0), __shfl_sync(0xffffffffu, v.lo, 0)};
}

// Warp 0: lanes 0..PCG_DF_REPLICAS-1 store the block's sums bs (valid in
// lane 0) and its aggregates' sums (warps 4k..4k+3 of aggregate k, added in
// order) as one slot of epoch e, one copy each; lane 0 then arrives on the
// grid counter and waits for the round to complete.  Returns false
// (warp-uniform) when the wait gave up or another block aborted.
template <int WPA, typename S>
__device__ __forceinline__ bool df_publish_c(const Dev<float>& d, unsigned e, const S (&bs_l0)[3],
                                             const float (*sz)[6]) {
  const int lane = threadIdx.x & 31;
  const int nb = gridDim.x;
  const unsigned long long tag = df_tag(e);
  int arrived = 1;
  const S bs[3] = {shfl0(bs_l0[0]), shfl0(bs_l0[1]), shfl0(bs_l0[2])};
  if (lane < PCG_DF_REPLICAS) {
    unsigned long long w[4];
    df_pack(tag, bs, w);
    unsigned long long* slot = df_slots(d, e, lane) + DF_SLOT_C * (size_t)blockIdx.x;
    st_v2_relaxed(slot, w[0], w[1]);
    st_v2_relaxed(slot + 2, w[2], w[3]);
#pragma unroll
    for (int k = 0; k < DF_AGG; ++k) {
      float z[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        float t = sz[WPA * k][c];
#pragma unroll
        for (int q = 1; q < WPA; ++q) t = __fadd_rn(t, sz[WPA * k + q][c]);
        z[c] = t;
      }
      unsigned long long a, b;
      df_pack_u(tag, z[0], z[1], z[2], a, b);
      st_v2_relaxed(slot + 4 + 4 * k, a, b);
      df_pack_u(tag, z[3], z[4], z[5], a, b);
      st_v2_relaxed(slot + 6 + 4 * k, a, b);
    }
  }
  __syncwarp();
  if (lane == 0) {
    const unsigned add = blockIdx.x == 0 ? (0x80000000u - ((unsigned)nb - 1u + d.bar_extra)) : 1u;
    atomicAdd(&d.ctrl->bar_count, add);
    const unsigned want = (e & 1u) << 31;
    volatile unsigned* vc = &d.ctrl->bar_count;
    DfWait wt;
    while ((*vc & 0x80000000u) != want)
      if (!wt.again(d.ctrl, d.wait_budget)) {
        arrived = 0;
        break;
      }
  }
  return __shfl_sync(0xffffffffu, arrived, 0) != 0;
}

// Warp 0 after the round: the dot sums of all slots of epoch e, each lane its
// slots (lane, lane + 32, ...) in block order, then a fixed shuffle tree;
// tot is valid in lane 0.  Re-reads slots whose words are not yet current.
template <typename S>
__device__ __forceinline__ bool df_gather_dots_c(const Dev<float>& d, unsigned e, S (&tot)[3]) {
  const int lane = threadIdx.x & 31;
  const int nb = gridDim.x;
  const unsigned long long* buf = df_slots(d, e, blockIdx.x % PCG_DF_REPLICAS);
  const unsigned long long tag = df_tag(e);
  unsigned long long w[DF_MAXQ][4];
#pragma unroll
  for (int q = 0; q < DF_MAXQ; ++q) {
    const int b = lane + 32 * q;
    if (b < nb) {
      ld_v2_relaxed(buf + DF_SLOT_C * (size_t)b, w[q][0], w[q][1]);
      ld_v2_relaxed(buf + DF_SLOT_C * (size_t)b + 2, w[q][2], w[q][3]);
    }
  }
  auto fresh = [&](int q) {
    return df_has(w[q][0], tag) && df_has(w[q][1], tag) && df_has(w[q][2], tag) && df_has(w[q][3], tag);
  };
  unsigned stale = 0;
#pragma unroll
  for (int q = 0; q < DF_MAXQ; ++q)
    if (lane + 32 * q < nb && !fresh(q)) stale |= 1u << q;
  DfWait wt;
  while (stale != 0 && wt.again(d.ctrl, d.wait_budget)) {
#pragma unroll
    for (int q = 0; q < DF_MAXQ; ++q)
      if (stale & (1u << q)) {
        const int b = lane + 32 * q;
        ld_v2_relaxed(buf + DF_SLOT_C * (size_t)b, w[q][0], w[q][1]);
        ld_v2_relaxed(buf + DF_SLOT_C * (size_t)b + 2, w[q][2], w[q][3]);
      }
#pragma unroll
    for (int q = 0; q < DF_MAXQ; ++q)
      if ((stale & (1u << q)) && fresh(q)) stale &= ~(1u << q);
  }
  if (!__all_sync(0xffffffffu, stale == 0)) return false;
  S a[3] = {acc_zero<S>(), acc_zero<S>(), acc_zero<S>()};
#pragma unroll
  for (int q = 0; q < DF_MAXQ; ++q) {
    if (lane + 32 * q < nb) {
      S v[3];
      df_unpack(w[q], v);
      a[0] = df_add(a[0], v[0]);
      a[1] = df_add(a[1], v[1]);
      a[2] = df_add(a[2], v[2]);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] = df_add(a[k], shfl_down(a[k], o));
    tot[k] = a[k];
  }
  return true;
}

// Warps 1..5 after the round (threads 32..191, one slot each): thread t reads
// slot t's aggregate sums of w and r and forms its part of
// g_i = sum_j Ainv[i][j] z_j for the block's aggregates i (ainv: DF_AGG rows
// of A_c^-1 in shared memory); the parts are added by fixed trees (warp
// shuffles, then the five warp totals in order) into g[0] (from w) and g[1]
// (from r).  Uses named barrier 1 (160 threads).
__device__ __forceinline__ void df_gather_coarse(const Dev<float>& d, unsigned e, const float* ainv,
                                                 float (*part)[6 * DF_AGG], float (*g)[DF_AGG][3]) {
  const int t = (int)threadIdx.x - 32;
  const int nb = gridDim.x;
  float c[DF_AGG][6];
#pragma unroll
  for (int i = 0; i < DF_AGG; ++i)
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) c[i][cc] = 0.0f;
  if (t < nb) {
    const unsigned long long* slot = df_slots(d, e, blockIdx.x % PCG_DF_REPLICAS) + DF_SLOT_C * (size_t)t + 4;
    const unsigned long long tag = df_tag(e);
    unsigned long long w[4 * DF_AGG];
#pragma unroll
    for (int k = 0; k < 2 * DF_AGG; ++k) ld_v2_relaxed(slot + 2 * k, w[2 * k], w[2 * k + 1]);
    DfWait wt;
    for (;;) {
      bool ok = true;
#pragma unroll
      for (int k = 0; k < 4 * DF_AGG; ++k) ok = ok && df_has(w[k], tag);
      if (ok || !wt.again(d.ctrl, d.wait_budget)) break;
#pragma unroll
      for (int k = 0; k < 2 * DF_AGG; ++k) ld_v2_relaxed(slot + 2 * k, w[2 * k], w[2 * k + 1]);
    }
#pragma unroll
    for (int k = 0; k < DF_AGG; ++k) {
      const int j = DF_AGG * t + k;
      if (j >= d.n_agg) break;
      float z[6];
      df_unpack_u(w[4 * k], w[4 * k + 1], z[0], z[1], z[2]);
      df_unpack_u(w[4 * k + 2], w[4 * k + 3], z[3], z[4], z[5]);
#pragma unroll
      for (int i = 0; i < DF_AGG; ++i) {
        const float a = ainv[i * d.n_agg + j];
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) c[i][cc] = __fmaf_rn(a, z[cc], c[i][cc]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < DF_AGG; ++i)
#pragma unroll
    for (int cc = 0; cc < 6; ++cc)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c[i][cc] = __fadd_rn(c[i][cc], __shfl_down_sync(0xffffffffu, c[i][cc], o));
  const int wq = t >> 5;
  if ((t & 31) == 0)
#pragma unroll
    for (int i = 0; i < DF_AGG; ++i)
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) part[wq][6 * i + cc] = c[i][cc];
  asm volatile("bar.sync 1, 160;" ::: "memory");
  if (t < 6 * DF_AGG) {
    float s = part[0][t];
#pragma unroll
    for (int q = 1; q < 5; ++q) s = __fadd_rn(s, part[q][t]);
    const int i = t / 6, cc = t % 6;
    g[cc / 3][i][cc % 3] = s;
  }
}

template <int MAXW, bool COARSE, int ROWS>
__global__ void __launch_bounds__(ROWS, 1) k_pcg_df(Dev<float> d) {
  constexpr int NW = ROWS / 32;
  constexpr int AGG_ROWS = ROWS / DF_AGG;
  static_assert(AGG_ROWS % 32 == 0, "aggregates of whole warps");
  __shared__ CgShared<float> cs;
  __shared__ double sc[2];  // bb, rr of the first reduction: used by lane 0 of warp 0 only
  __shared__ DW s_st[3];    // gamma, alpha, rr of the CG recurrence (double words)
  __shared__ float s_thr;   // tol^2 ||b||^2 in FP32
  __shared__ double s_es;   // the iteration's spring energy (fused right-hand side)
  extern __shared__ unsigned long long halo[];  // 2 tagged words per halo row (+ coarse rows)
  const int lane = threadIdx.x & 31;
  const bool w0 = threadIdx.x < 32;
  const int n = d.n_free;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i < n;
  const size_t ustride = 2 * (size_t)n;  // words of one parity buffer of u
  int lcol[MAXW];  // columns as indices into the block's halo
  float val[MAXW];
  int width = 0;
  float dg = 1.0f, idg = 1.0f;  // the row's diagonal and its reciprocal (the Jacobi part of the preconditioner)
  if (act) {
    const int sl = i >> 5, ln = i & 31;
    const int base = d.sl_ptr[sl];
    width = (d.sl_ptr[sl + 1] - base) >> 5;
#pragma unroll
    for (int j = 0; j < MAXW; ++j) {
      lcol[j] = j < width ? chk_idx(d.ctrl, d.sl_lcol[base + j * 32 + ln], d.halo_max) : 0;
      val[j] = j < width ? d.sl_val[base + j * 32 + ln] : 0.0f;
    }
  }
  // coarse correction state (COARSE only): per-warp aggregate sums, the
  // parts of warps 1..5, the block's g values, this block's rows of A_c^-1
  __shared__ float s_zw[COARSE ? NW : 1][6];
  __shared__ float s_part[COARSE ? 5 : 1][6 * DF_AGG];
  __shared__ float s_g[2][DF_AGG][3];  // g(w), g(r) of the block's aggregates
  __shared__ int s_ok;
  float* ainv = reinterpret_cast<float*>(halo + 2 * (size_t)d.halo_max);
  const int ia = (int)threadIdx.x / AGG_ROWS;  // this row's aggregate within the block
  if constexpr (COARSE) {
    for (int k = threadIdx.x; k < DF_AGG * d.n_agg; k += ROWS) {
      const int r = k / d.n_agg, j = k - r * d.n_agg;
      const int a = DF_AGG * (int)blockIdx.x + r;
      ainv[k] = a < d.n_agg ? d.cg_ainv[(size_t)a * d.n_agg + j] : 0.0f;
    }
  }
  auto store_u = [&](unsigned e, const float (&uu)[3]) {
    unsigned long long a, b;
    df_pack_u(df_tag(e), uu[0], uu[1], uu[2], a, b);
    st_v2_relaxed(d.df_u + (size_t)(e & 1u) * ustride + 2 * (size_t)i, a, b);
  };
  const int h0 = d.halo_ptr[blockIdx.x], nh = d.halo_ptr[blockIdx.x + 1] - h0;
  const int n_own = d.halo_own[blockIdx.x];  // the halo's first n_own rows are this block's
  const int hself = act ? d.halo_self[i] : -1;
  // A u for this row from the neighbours' u of epoch e.  Called by every
  // thread of the block with its own u of epoch e: each row that the block
  // reads writes its own value into the halo, the block copies the other
  // blocks' rows of epoch e (re-reading rows whose words are not yet
  // current), then each active row multiplies from shared memory.
  // Each halo row is unpacked once, into a float4 in place of its two words,
  // so the multiply reads one 16-byte shared-memory word per entry.
  float4* const halo4 = reinterpret_cast<float4*>(halo);
  auto spmv = [&](unsigned e, const float (&self)[3], float (&ax)[3]) {
    const unsigned long long* buf = d.df_u + (size_t)(e & 1u) * ustride;
    const unsigned long long tag = df_tag(e);
    unsigned long long stale = 0;  // bit q: this thread's row n_own + threadIdx.x + q * ROWS is not yet current
    if (hself >= 0) halo4[chk_idx(d.ctrl, hself, d.halo_max)] = make_float4(self[0], self[1], self[2], 0.0f);
#pragma unroll 4
    for (int k = n_own + (int)threadIdx.x, q = 0; k < nh; k += ROWS, ++q) {
      unsigned long long w0, w1;
      ld_v2_relaxed_at(buf, chk_idx(d.ctrl, d.halo_rows[h0 + k], n), w0, w1);
      if (df_has(w0, tag) && df_has(w1, tag)) {
        float vx, vy, vz;
        df_unpack_u(w0, w1, vx, vy, vz);
        halo4[k] = make_float4(vx, vy, vz, 0.0f);
      } else {
        stale |= 1ull << q;
      }
    }
    if (stale) {
      DfWait wt;
      for (int k = n_own + (int)threadIdx.x, q = 0; k < nh; k += ROWS, ++q) {
        if (!(stale & (1ull << q))) continue;
        unsigned long long w0, w1;
        do {
          ld_v2_relaxed_at(buf, chk_idx(d.ctrl, d.halo_rows[h0 + k], n), w0, w1);
        } while (!(df_has(w0, tag) && df_has(w1, tag)) && wt.again(d.ctrl, d.wait_budget));
        float vx, vy, vz;
        df_unpack_u(w0, w1, vx, vy, vz);
        halo4[k] = make_float4(vx, vy, vz, 0.0f);
      }
      // a wait that gave up leaves the abort word raised: the next reduction
      // cannot complete, so every block leaves at its next reduction
    }
    __syncthreads();
    if (act) {
      ax[0] = dg * self[0];
      ax[1] = dg * self[1];
      ax[2] = dg * self[2];
#pragma unroll
      for (int j = 0; j < MAXW; ++j) {
        if (j < width) {
          const float4 v = halo4[lcol[j]];
          ax[0] += val[j] * v.x;
          ax[1] += val[j] * v.y;
          ax[2] += val[j] * v.z;
        }
      }
    }
    __syncthreads();  // the halo is rewritten by the next call
  };
  // COARSE: the reduction of epoch e with the aggregate sums of zv.  Warp 0
  // publishes the slot and waits for the round; after a block-wide barrier
  // warp 0 sums the dot words (dots(), which also sets cs.flag) while warps
  // 1..5 form the block's coarse values g (into s_g); a second barrier
  // publishes both.  Returns false (block-uniform) when the round was not
  // completed.
  auto reduce_c = [&](unsigned e, const auto (&bs)[3], auto dots) -> bool {
    if (w0) {
      const bool ok = df_publish_c<AGG_ROWS / 32>(d, e, bs, s_zw);
      if (lane == 0) s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;
    if (w0)
      dots();
    else if (threadIdx.x < 32 * 6)
      df_gather_coarse(d, e, ainv, s_part, s_g);
    __syncthreads();
    return true;
  };
  unsigned ue = 0, re = 0;  // epochs of u and of the reductions (the same in every thread)
  float r[3] = {0.0f, 0.0f, 0.0f}, u[3], w[3] = {0.0f, 0.0f, 0.0f}, p[3], s[3], dd[3] = {0.0f, 0.0f, 0.0f};
  float gr[3] = {0.0f, 0.0f, 0.0f}, gs[3] = {0.0f, 0.0f, 0.0f};  // g(r), g(s) of this row's aggregate
  DW a0[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
  ++ue;
  if (act) {
    if (d.rhs_in_pcg) {
      rhs_residual_row_dw(d, i, val, width, dg, r, a0);
    } else {
      dg = d.diag[i];
      double rv[3];
      double a01[2] = {0.0, 0.0};
      residual_row_f64(d, i, dg, rv, a01);
      a0[0] = dw_from(a01[0]);
      a0[1] = dw_from(a01[1]);
      for (int c = 0; c < 3; ++c) r[c] = (float)rv[c];
    }
    idg = 1.0f / dg;
    for (int c = 0; c < 3; ++c) u[c] = r[c] * idg;
    if constexpr (!COARSE) store_u(ue, u);
  }
  {
    // (||b||^2, ||r0||^2, spring energy) summed over the grid
    DW bs[3], t[3] = {};
    if constexpr (COARSE) agg_warp_sums(w, r, s_zw);  // w is zero here
    block_sums_dw<3, NW>(a0, cs.sh, bs);
    ++re;
    auto first = [&](bool ok) {
      if (lane == 0) {
        const double bb = acc_to_f64(t[0]), rr = acc_to_f64(t[1]);
        sc[0] = bb;
        sc[1] = rr;
        s_es = acc_to_f64(t[2]);
        s_thr = (float)(d.tol2 * bb);
        cs.flag = !ok ? CG_ABORT : ((bb > 0.0 && rr > d.tol2 * bb) ? CG_CONTINUE : CG_DONE);
      }
    };
    if constexpr (!COARSE) {
      if (w0) first(df_reduce(d, re, bs, t));
      __syncthreads();
    } else {
      if (!reduce_c(re, bs, [&] { first(df_gather_dots_c(d, re, t)); }))
        return;
      for (int c = 0; c < 3; ++c) gr[c] = s_g[1][ia][c];
    }
  }
  if (cs.flag == CG_ABORT) return;
  int it = 0;
  if (cs.flag == CG_CONTINUE) {
    DW a1[2] = {acc_zero<DW>(), acc_zero<DW>()};
    if constexpr (COARSE) {
      if (act) {
        for (int c = 0; c < 3; ++c) u[c] = r[c] * idg + gr[c];
        store_u(ue, u);
      }
    }
    spmv(ue, u, w);
    if (act) {
      a1[0] = dot3(r[0], r[1], r[2], u[0], u[1], u[2]);
      a1[1] = dot3(w[0], w[1], w[2], u[0], u[1], u[2]);
      for (int c = 0; c < 3; ++c) {
        p[c] = u[c];
        s[c] = w[c];
      }
    }
    {
      DW bs2[2], t[3] = {};
      if constexpr (COARSE) agg_warp_sums(w, r, s_zw);
      block_sums_dw<2, NW>(a1, cs.sh, bs2);
      ++re;
      const DW bs[3] = {bs2[0], bs2[1], DW{0.0f, 0.0f}};
      auto first_scalars = [&](bool ok) {
        if (lane == 0) {
          if (ok) {
            const DW a = dw_div(t[0], t[1]);
            s_st[0] = t[0];
            s_st[1] = a;
            cs.ta = a.hi;
          }
          cs.flag = ok ? CG_CONTINUE : CG_ABORT;
        }
      };
      if constexpr (!COARSE) {
        if (w0) first_scalars(df_reduce(d, re, bs, t));
        __syncthreads();
      } else {
        if (!reduce_c(re, bs, [&] { first_scalars(df_gather_dots_c(d, re, t)); })) return;
        for (int c = 0; c < 3; ++c) {
          gs[c] = s_g[0][ia][c];  // s_0 = w_0
          gr[c] = s_g[1][ia][c];
        }
      }
    }
    if (cs.flag == CG_ABORT) return;
    float ta = cs.ta;
    for (it = 1; it <= d.max_iter; ++it) {
      ++ue;
      if constexpr (COARSE)
        for (int c = 0; c < 3; ++c) gr[c] -= ta * gs[c];
      if (act) {
        for (int c = 0; c < 3; ++c) {
          dd[c] += ta * p[c];
          r[c] -= ta * s[c];
          u[c] = r[c] * idg;
          if constexpr (COARSE) u[c] += gr[c];
        }
        store_u(ue, u);
      }
      DW a2[3] = {acc_zero<DW>(), acc_zero<DW>(), acc_zero<DW>()};
      spmv(ue, u, w);
      if (act) {
        a2[0] = dot3(r[0], r[1], r[2], u[0], u[1], u[2]);
        a2[1] = dot3(w[0], w[1], w[2], u[0], u[1], u[2]);
        a2[2] = dot3(r[0], r[1], r[2], r[0], r[1], r[2]);
      }
      {
        DW bs[3], tw[3] = {};
        if constexpr (COARSE) agg_warp_sums(w, r, s_zw);
        block_sums_dw<3, NW>(a2, cs.sh, bs);
        ++re;
        auto scalars = [&](bool ok) {
          int f = CG_ABORT;
          float fa = 0.0f, fb = 0.0f;
          if (ok) f = cg_scalars_dw(tw, s_thr, s_st, fa, fb);
          if (lane == 0) {
            if (ok) {
              if (f == CG_NONFINITE && blockIdx.x == 0) set_status(d.ctrl, ST_NONFINITE);
              cs.ta = fa;
              cs.tb = fb;
            }
            cs.flag = f;
          }
        };
        if constexpr (!COARSE) {
          if (w0) scalars(df_reduce(d, re, bs, tw));
          __syncthreads();
        } else {
          if (!reduce_c(re, bs, [&] { scalars(df_gather_dots_c(d, re, tw)); })) return;
        }
      }
      const int f = cs.flag;
      if (f == CG_ABORT) return;
      if (f != CG_CONTINUE) break;
      ta = cs.ta;
      const float tb = cs.tb;
      if constexpr (COARSE)
        for (int c = 0; c < 3; ++c) {
          gs[c] = s_g[0][ia][c] + tb * gs[c];  // g(s_k) = g(w_k) + beta_k g(s_k-1)
          gr[c] = s_g[1][ia][c];               // g(r_k), fresh from this round's sums
        }
      if (act)
        for (int c = 0; c < 3; ++c) {
          p[c] = u[c] + tb * p[c];
          s[c] = w[c] + tb * s[c];
        }
    }
    if (it > d.max_iter) {
      it = d.max_iter;
      if (i == 0) set_status(d.ctrl, ST_PCG_MAXIT);
    }
    if (act) {
      // x_(i+1) = start + correction; the step x_(i+1) - x_i is kept for the
      // next outer iteration's start
      const R4<float> x0 = d.X[i];
      R4<float> t = warm_start(d, i, x0);
      t.x += dd[0]; t.y += dd[1]; t.z += dd[2];
      d.X[i] = t;
      if (d.xstep) d.xstep[i] = R4<float>{t.x - x0.x, t.y - x0.y, t.z - x0.z, 0.0f};
    }
  }
  if (blockIdx.x == 0) {
    // the record of this outer iteration; with the fused right-hand side
    // also what a separate finalize launch would do: the Eq. 8 energy (the
    // local step's partials, summed by the whole block in a fixed order, plus
    // the spring energy of the first reduction), the iteration count, and the
    // per-iteration words reset for the next iteration
    double el[1] = {0.0}, e_loc[1];
    if (d.rhs_in_pcg && d.stats)
      for (int k = threadIdx.x; k < d.n_e_local; k += ROWS) el[0] += d.e_partials[k];
    block_sums<1, NW>(el, cs.sh, e_loc);
    if (threadIdx.x == 0) {
      const double rr = it > 0 ? (double)s_st[2].hi + (double)s_st[2].lo : sc[1];
      write_pcg_record(d.ctrl, d.hist, d.hist_cap, d.ctrl, it, rr, sc[0]);
      if (d.rhs_in_pcg) finalize_iteration(d, d.stats ? e_loc[0] + s_es : 0.0);
    }
  }
}

// Segmented streaming variant for batches: block b works on a contiguous row
// range of one robot (every robot owns at least one block; blocks are given
// to robots in proportion to their rows), so each robot runs its own CG with
// its own scalars and stopping test while all robots share the two grid
// barriers of an iteration.  Robot totals are the sums of the partials of the
// robot's blocks in block order (deterministic).  A robot that has converged
// stops updating; the launch ends when every robot has converged (a counter
// that the robot's first block increments, read after the next barrier so
// every block sees the same value) or at the iteration cap.
// Per-robot coarse correction of the segmented kernel (COARSE): the same
// additive two-level preconditioner as the dataflow kernel's, per robot, with
// aggregates of SEG_AGG_ROWS rows counted from the robot's first row and block
// boundaries on whole aggregates.  In a pass, round m of the block's threads
// covers the rows lo + 256 m + t, i.e. the block's local aggregates 2m (warps
// 0..3) and 2m + 1 (warps 4..7); each warp adds its rows' values by a fixed
// shuffle tree and the four warp sums of an aggregate are added in order.
static constexpr int SEG_WPA = SEG_AGG_ROWS / 32;  // warps per aggregate

template <int NV>
__device__ __forceinline__ void seg_agg_partial(const float (&v)[NV], int m, float (*zp)[PCG_SEG_THREADS / 32][6],
                                                int off) {
  float a[NV];
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    a[c] = v[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[c] = __fadd_rn(a[c], __shfl_down_sync(0xffffffffu, a[c], o));
  }
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    const int agg = 2 * m + wid / SEG_WPA;
    if (agg < PCG_SEG_AGG_MAX)
#pragma unroll
      for (int c = 0; c < NV; ++c) zp[agg][wid % SEG_WPA][off + c] = a[c];
  }
}

template <typename T, bool COARSE>
__global__ void __launch_bounds__(PCG_SEG_THREADS, 4) k_pcg_seg(Dev<T> d) {
  using A = typename DotAcc<T>::type;
  constexpr int NW = PCG_SEG_THREADS / 32;
  __shared__ CgShared<T> cs;
  // coarse state of the block's aggregates: warp partial sums of a pass,
  // fresh g(w) and g(r) of the last reduction, the carried g(s)
  __shared__ float s_zp[COARSE ? PCG_SEG_AGG_MAX : 1][PCG_SEG_THREADS / 32][6];
  __shared__ float s_gw[COARSE ? PCG_SEG_AGG_MAX : 1][3];
  __shared__ float s_gr[COARSE ? PCG_SEG_AGG_MAX : 1][3];
  __shared__ float s_gs[COARSE ? PCG_SEG_AGG_MAX : 1][3];
  const GridCtx g{d.ctrl, d.partials, gridDim.x, d.wait_budget, d.bar_extra};
  unsigned epoch = 0;
  const int lane = threadIdx.x & 31;
  const bool w0 = threadIdx.x < 32;
  const int b = blockIdx.x;
  const int lo = d.seg_lo[b], hi = d.seg_hi[b];
  const int rb0 = d.seg_rb0[b], rb1 = d.seg_rb1[b];
  const bool lead = b == rb0 && threadIdx.x == 0;  // the robot's first block, lane 0
  R4<T>* __restrict__ X = d.X;
  R4<T>* __restrict__ r = d.r;
  R4<T>* __restrict__ u = d.u;
  R4<T>* __restrict__ p = d.p;
  R4<T>* __restrict__ s = d.s;
  R4<T>* __restrict__ w = d.w;
  R4<T>* __restrict__ dx = d.dx;
  const R4<T> zero = {T(0), T(0), T(0), T(0)};
  // robot CG scalars: meaningful in lane 0 of warp 0
  double bb = 0.0, rr = 0.0, gamma = 0.0, alpha = 0.0, beta = 0.0;
  int it_done = 0;
  // coarse bookkeeping
  int rob = 0, r0 = 0, ga0 = 0, na_r = 0, na_b = 0;
  const float* ainv = nullptr;
  if constexpr (COARSE) {
    rob = d.seg_robot[b];
    r0 = d.robot_row[rob];
    na_r = d.seg_agg_base[rob + 1] - d.seg_agg_base[rob];
    ga0 = d.seg_agg_base[rob] + (lo - r0) / SEG_AGG_ROWS;
    na_b = (hi - lo + SEG_AGG_ROWS - 1) / SEG_AGG_ROWS;
    ainv = d.seg_ainv + d.seg_ainv_off[rob] + (size_t)((lo - r0) / SEG_AGG_ROWS) * na_r;
  }
  // the block's aggregate sums of this pass into the global exchange array
  // (call after a __syncthreads that follows the pass); which = 0 w, 1 r
  auto agg_store = [&](int which) {
    for (int k = threadIdx.x; k < na_b * 3; k += blockDim.x) {
      const int a = k / 3, c = k % 3;
      float t = s_zp[a][0][3 * which + c];
#pragma unroll
      for (int q = 1; q < SEG_WPA; ++q) t = __fadd_rn(t, s_zp[a][q][3 * which + c]);
      d.seg_aggsum[6 * (size_t)(ga0 + a) + 3 * which + c] = t;
    }
  };
  // g = A_c^-1 Z^T v for the block's aggregates from the robot's exchanged
  // sums (after the reduction made them visible): which = 0 w into s_gw, 1 r
  // into s_gr; one thread per (aggregate, column, which), robot-order sums
  auto agg_coarse = [&]() {
    const int base = d.seg_agg_base[rob];
    for (int k = threadIdx.x; k < na_b * 6; k += blockDim.x) {
      const int a = k / 6, which = (k % 6) / 3, c = k % 3;
      const float* row = ainv + (size_t)a * na_r;
      float t = 0.0f;
      for (int j = 0; j < na_r; ++j)
        t = __fmaf_rn(row[j], __ldcg(&d.seg_aggsum[6 * (size_t)(base + j) + 3 * which + c]), t);
      if (which == 0)
        s_gw[a][c] = t;
      else
        s_gr[a][c] = t;
    }
  };

  double a0[2] = {0.0, 0.0};
  for (int i = lo + (int)threadIdx.x, m = 0; i < hi || (COARSE && m * (int)blockDim.x < hi - lo);
       i += blockDim.x, ++m) {
    float rz[3] = {0.0f, 0.0f, 0.0f};
    if (i < hi) {
      const T dg = d.diag[i];
      double rv[3];
      residual_row_f64(d, i, dg, rv, a0);
      R4<T> ri, ui;
      ri.x = (T)rv[0]; ri.y = (T)rv[1]; ri.z = (T)rv[2]; ri.w = T(0);
      const T idg = T(1) / dg;
      ui.x = ri.x * idg; ui.y = ri.y * idg; ui.z = ri.z * idg; ui.w = T(0);
      r[i] = ri;
      u[i] = ui;
      dx[i] = zero;
      rz[0] = (float)ri.x; rz[1] = (float)ri.y; rz[2] = (float)ri.z;
    }
    if constexpr (COARSE) {
      const float wz[3] = {0.0f, 0.0f, 0.0f};
      seg_agg_partial<3>(wz, m, s_zp, 0);
      seg_agg_partial<3>(rz, m, s_zp, 3);
    }
  }
  if constexpr (COARSE) {
    __syncthreads();
    agg_store(0);
    agg_store(1);
  }
  {
    double bs[2], t[2];
    block_sums<2, NW>(a0, cs.sh, bs);
    if (w0) {
      const bool ok = warp0_reduce<2>(g, epoch, bs, rb0, rb1, t);
      if (lane == 0) {
        bb = t[0];
        rr = t[1];
        const bool conv = !(bb > 0.0 && rr > d.tol2 * bb);
        if (ok && conv && b == rb0) atomicAdd(&d.ctrl->queue, 1u);
        cs.flag = !ok ? CG_ABORT : (conv ? CG_DONE : CG_CONTINUE);
      }
    }
    __syncthreads();
  }
  if (cs.flag == CG_ABORT) return;
  bool done = cs.flag != CG_CONTINUE;
  if constexpr (COARSE) {
    // u_0 = D^-1 r_0 + Z g(r_0): one more pass and a grid barrier before the
    // first SpMV reads the neighbours' u
    if (!done) agg_coarse();
    __syncthreads();
    if (!done)
      for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
        const int a = (i - lo) / SEG_AGG_ROWS;
        R4<T> ui = u[i];
        ui.x += (T)s_gr[a][0];
        ui.y += (T)s_gr[a][1];
        ui.z += (T)s_gr[a][2];
        u[i] = ui;
      }
    if (!grid_barrier(g, epoch, &cs.ok)) return;
  }
  A a1[2] = {acc_zero<A>(), acc_zero<A>()};
  if (!done) {
    for (int i = lo + (int)threadIdx.x, m = 0; i < hi || (COARSE && m * (int)blockDim.x < hi - lo);
         i += blockDim.x, ++m) {
      float wz[3] = {0.0f, 0.0f, 0.0f}, rz[3] = {0.0f, 0.0f, 0.0f};
      if (i < hi) {
        const T dg = d.diag[i];
        const R4<T> ui = u[i], ri = r[i];
        T ax, ay, az;
        spmv_row(d, i, u, dg, ui, ax, ay, az);
        R4<T> wi;
        wi.x = ax; wi.y = ay; wi.z = az; wi.w = T(0);
        w[i] = wi;
        a1[0] = acc_add(a1[0], dot3(ri.x, ri.y, ri.z, ui.x, ui.y, ui.z));
        a1[1] = acc_add(a1[1], dot3(ax, ay, az, ui.x, ui.y, ui.z));
        wz[0] = (float)ax; wz[1] = (float)ay; wz[2] = (float)az;
        rz[0] = (float)ri.x; rz[1] = (float)ri.y; rz[2] = (float)ri.z;
      }
      if constexpr (COARSE) {
        seg_agg_partial<3>(wz, m, s_zp, 0);
        seg_agg_partial<3>(rz, m, s_zp, 3);
      }
    }
  }
  if constexpr (COARSE) {
    __syncthreads();
    if (!done) {
      agg_store(0);
      agg_store(1);
    }
  }
  {
    double bs[2], t[2];
    block_sums<2, NW>(a1, cs.sh, bs);
    if (w0) {
      const bool ok = warp0_reduce<2>(g, epoch, bs, rb0, rb1, t);
      if (lane == 0) {
        if (ok && !done) {
          gamma = t[0];
          alpha = gamma / t[1];
        }
        cs.ta = (T)alpha;
        cs.tb = T(0);
        cs.flag = ok ? CG_CONTINUE : CG_ABORT;
      }
    }
    __syncthreads();
  }
  if (cs.flag == CG_ABORT) return;
  T ta = cs.ta, tb = T(0);
  if constexpr (COARSE) {
    if (!done) agg_coarse();  // g(w_0), g(r_0)
    __syncthreads();
  }
  bool first = true;
  int it = 1;
  for (;; ++it) {
    if constexpr (COARSE) {
      // g(s_k) = g(w_k) + beta_k g(s_k-1); g(r_k+1) = g(r_k) - alpha_k g(s_k)
      if (!done)
        for (int k = threadIdx.x; k < na_b * 3; k += blockDim.x) {
          const int a = k / 3, c = k % 3;
          const float gs = first ? s_gw[a][c] : s_gw[a][c] + (float)tb * s_gs[a][c];
          s_gs[a][c] = gs;
          s_gr[a][c] = s_gr[a][c] - (float)ta * gs;
        }
      __syncthreads();
    }
    // r.u and r.r of the new residual are formed in the update pass, so the
    // SpMV pass does not read r again (same values, same order of rows)
    A a_ru = acc_zero<A>(), a_rr = acc_zero<A>();
    if (!done) {
      for (int i = lo + (int)threadIdx.x, m = 0; i < hi || (COARSE && m * (int)blockDim.x < hi - lo);
           i += blockDim.x, ++m) {
        float rz[3] = {0.0f, 0.0f, 0.0f};
        if (i < hi) {
          const R4<T> ui = u[i], wi = w[i];
          R4<T> pi, si;
          if (first) {
            pi = ui;
            si = wi;
          } else {
            const R4<T> po = p[i], so = s[i];
            pi.x = ui.x + tb * po.x; pi.y = ui.y + tb * po.y; pi.z = ui.z + tb * po.z;
            si.x = wi.x + tb * so.x; si.y = wi.y + tb * so.y; si.z = wi.z + tb * so.z;
          }
          pi.w = T(0);
          si.w = T(0);
          p[i] = pi;
          s[i] = si;
          R4<T> di = dx[i], ri = r[i];
          di.x += ta * pi.x; di.y += ta * pi.y; di.z += ta * pi.z;
          ri.x -= ta * si.x; ri.y -= ta * si.y; ri.z -= ta * si.z;
          dx[i] = di;
          r[i] = ri;
          const T idg = T(1) / d.diag[i];
          R4<T> un;
          un.x = ri.x * idg; un.y = ri.y * idg; un.z = ri.z * idg; un.w = T(0);
          if constexpr (COARSE) {
            const int a = (i - lo) / SEG_AGG_ROWS;
            un.x += (T)s_gr[a][0];
            un.y += (T)s_gr[a][1];
            un.z += (T)s_gr[a][2];
          }
          u[i] = un;
          a_ru = acc_add(a_ru, dot3(ri.x, ri.y, ri.z, un.x, un.y, un.z));
          a_rr = acc_add(a_rr, dot3(ri.x, ri.y, ri.z, ri.x, ri.y, ri.z));
          rz[0] = (float)ri.x; rz[1] = (float)ri.y; rz[2] = (float)ri.z;
        }
        if constexpr (COARSE) seg_agg_partial<3>(rz, m, s_zp, 3);
      }
    }
    if (!grid_barrier(g, epoch, &cs.ok)) return;
    // every block reads the same count: increments happen before this barrier
    const unsigned n_done = __ldcg(&d.ctrl->queue);
    if ((int)n_done >= d.n_robots || it > d.max_iter) break;
    A a2[3] = {a_ru, acc_zero<A>(), a_rr};
    if (!done) {
      for (int i = lo + (int)threadIdx.x, m = 0; i < hi || (COARSE && m * (int)blockDim.x < hi - lo);
           i += blockDim.x, ++m) {
        float wz[3] = {0.0f, 0.0f, 0.0f};
        if (i < hi) {
          const T dg = d.diag[i];
          const R4<T> ui = u[i];
          T ax, ay, az;
          spmv_row(d, i, u, dg, ui, ax, ay, az);
          R4<T> wi;
          wi.x = ax; wi.y = ay; wi.z = az; wi.w = T(0);
          w[i] = wi;
          a2[1] = acc_add(a2[1], dot3(ax, ay, az, ui.x, ui.y, ui.z));
          wz[0] = (float)ax; wz[1] = (float)ay; wz[2] = (float)az;
        }
        if constexpr (COARSE) seg_agg_partial<3>(wz, m, s_zp, 0);
      }
    }
    if constexpr (COARSE) {
      __syncthreads();
      if (!done) {
        agg_store(0);
        agg_store(1);
      }
    }
    {
      double bs[3], t[3];
      block_sums<3, NW>(a2, cs.sh, bs);
      if (w0) {
        const bool ok = warp0_reduce<3>(g, epoch, bs, rb0, rb1, t);
        int f = CG_ABORT;
        if (ok) f = done ? CG_DONE : cg_scalars_warp(t, bb, d.tol2, gamma, alpha, beta, rr);
        if (lane == 0) {
          if (ok) {
            if (!done) {
              if (f == CG_NONFINITE && b == rb0) set_status(d.ctrl, ST_NONFINITE);
              if (f != CG_CONTINUE) {
                it_done = it;
                if (b == rb0) atomicAdd(&d.ctrl->queue, 1u);
              }
            }
            cs.ta = (T)alpha;
            cs.tb = (T)beta;
          }
          cs.flag = f;
        }
      }
      __syncthreads();
    }
    const int f = cs.flag;
    if (f == CG_ABORT) return;
    if (f != CG_CONTINUE) done = true;
    ta = cs.ta;
    tb = cs.tb;
    first = false;
    if constexpr (COARSE) {
      if (!done) agg_coarse();  // g(w_k+1) and a fresh g(r_k+1)
      __syncthreads();
    }
  }
  if (!done && lead) {
    it_done = d.max_iter;
    set_status(d.ctrl, ST_PCG_MAXIT);
  }
  for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) {
    // x_(i+1) = start + correction; the step is kept for the next start
    const R4<T> x0 = X[i];
    R4<T> xi = warm_start(d, i, x0);
    const R4<T> di = dx[i];
    xi.x += di.x; xi.y += di.y; xi.z += di.z;
    X[i] = xi;
    if (d.xstep) d.xstep[i] = R4<T>{xi.x - x0.x, xi.y - x0.y, xi.z - x0.z, T(0)};
  }
  if (lead) {
    IterRec* rec = d.hist + (d.ctrl->iter % d.hist_cap);
    atomicMax(&rec->pcg_iters, it_done);
    atomicAdd(reinterpret_cast<unsigned long long*>(&d.ctrl->total_pcg), (unsigned long long)it_done);
    const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    atomicMax(reinterpret_cast<unsigned long long*>(&rec->pcg_rel_residual),
              (unsigned long long)__double_as_longlong(rel));
  }
}

// Cluster variant: one thread-block cluster of PCG_CL_SIZE CTAs solves one
// robot's system at a time, taking robots from a work queue (one persistent
// launch serves any number of independent robots).  Each CTA owns a
// contiguous range of the robot's rows and keeps all of its CG vectors in
// shared memory; the preconditioned residual u of neighbouring rows is read
// from the owning CTA's shared memory (distributed shared memory), and the
// FP64 reductions exchange one partial per CTA through distributed shared
// memory.  All synchronisation is the cluster's hardware barrier.
namespace cgx = cooperative_groups;

template <typename T>
__global__ void __launch_bounds__(PCG_CL_THREADS, 1) k_pcg_cluster(Dev<T> d) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[96];
  __shared__ double part[4];
  __shared__ double tot[4];
  __shared__ int s_robot;
  cgx::cluster_group cl = cgx::this_cluster();
  const int crank = (int)cl.block_rank();
  const int csz = (int)cl.num_blocks();
  const int cap = d.cl_rows_cap;
  R4<T>* su = reinterpret_cast<R4<T>*>(smem);
  T* sr = reinterpret_cast<T*>(su + cap);
  T* sp = sr + 3 * cap;
  T* ss = sp + 3 * cap;
  T* sw = ss + 3 * cap;
  T* sd = sw + 3 * cap;
  T* sg = sd + 3 * cap;  // diagonal

  // cluster-wide FP64 sums of nv values: block sums in one shared-memory
  // round, one partial per CTA exchanged through distributed shared memory,
  // summed by a fixed shuffle tree over the ranks (deterministic)
  auto cluster_reduce = [&](const double* v, int nv) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double t[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < nv; ++k) {
      t[k] = v[k];
      for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
    }
    __syncthreads();
    if (lane == 0)
      for (int k = 0; k < nv; ++k) sh[k * 32 + wid] = t[k];
    __syncthreads();
    if (threadIdx.x < 3 && threadIdx.x < nv) {
      double a = 0.0;
      const int nw = (blockDim.x + 31) >> 5;
      for (int i = 0; i < nw; ++i) a += sh[threadIdx.x * 32 + i];
      part[threadIdx.x] = a;
    }
    cl.sync();
    if (threadIdx.x < 32) {
      double a[3] = {0.0, 0.0, 0.0};
      if (lane < csz) {
        const double* rp = cl.map_shared_rank(part, lane);
        for (int k = 0; k < nv; ++k) a[k] = rp[k];
      }
      for (int k = 0; k < nv; ++k) {
        for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
        if (lane == 0) tot[k] = a[k];
      }
    }
    __syncthreads();
  };

  while (true) {
    if (crank == 0 && threadIdx.x == 0) s_robot = (int)atomicAdd(&d.ctrl->queue, 1u);
    cl.sync();
    const int robot = *cl.map_shared_rank(&s_robot, 0);
    cl.sync();  // every rank has read rank 0's word before any rank moves on or exits
    if (robot >= d.n_robots) break;
    const int row0 = d.robot_row[robot];
    const int n = d.robot_row[robot + 1] - row0;
    const int rpc = (((n + csz - 1) / csz) + 31) & ~31;  // rows per CTA (host checks rpc <= cap)
    const int my0 = crank * rpc;
    const int my1 = min(n, my0 + rpc);
    const int nmine = my1 > my0 ? my1 - my0 : 0;
    // SpMV of local rows: diag * own + sum of off-diagonals over neighbours' u
    auto spmv_u = [&](int j, T& ax, T& ay, T& az) {
      const int i = row0 + my0 + j;
      const T dg = sg[j];
      const R4<T> self = su[j];
      ax = dg * self.x;
      ay = dg * self.y;
      az = dg * self.z;
      const int sl = i >> 5, lane = i & 31;
      const int base = d.sl_ptr[sl] + lane;
      const int width = (d.sl_ptr[sl + 1] - d.sl_ptr[sl]) >> 5;
      // chunks of 8 entries: all column/value loads first, then the
      // distributed-shared-memory gathers, so the loads overlap
      for (int j0 = 0; j0 < width; j0 += 8) {
        int cc[8];
        T aa[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (j0 + q < width) {
            cc[q] = d.sl_col[base + (j0 + q) * 32];
            aa[q] = d.sl_val[base + (j0 + q) * 32];
          } else {
            cc[q] = row0 + my0 + j;
            aa[q] = T(0);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int c = cc[q] - row0;
          const int owner = c / rpc;
          const R4<T> v = cl.map_shared_rank(su, owner)[c - owner * rpc];
          ax += aa[q] * v.x;
          ay += aa[q] * v.y;
          az += aa[q] * v.z;
        }
      }
    };
    // r = b - A x in FP64, u = r / diag, correction d = 0
    double a0[2] = {0.0, 0.0};
    for (int j = threadIdx.x; j < nmine; j += blockDim.x) {
      const int i = row0 + my0 + j;
      const T dg = d.diag[i];
      sg[j] = dg;
      const R4<T> xi = d.X[i];
      double ax = (double)dg * xi.x, ay = (double)dg * xi.y, az = (double)dg * xi.z;
      const int sl = i >> 5, lane = i & 31;
      const int k1 = d.sl_ptr[sl + 1];
      for (int k = d.sl_ptr[sl] + lane; k < k1; k += 32) {
        const double a = (double)d.sl_val[k];
        const R4<T> xc = d.X[d.sl_col[k]];
        ax += a * xc.x;
        ay += a * xc.y;
        az += a * xc.z;
      }
      const R4<double> bi = d.b[i];
      const double rx = bi.x - ax, ry = bi.y - ay, rz = bi.z - az;
      sr[3 * j] = (T)rx;
      sr[3 * j + 1] = (T)ry;
      sr[3 * j + 2] = (T)rz;
      su[j] = R4<T>{sr[3 * j] / dg, sr[3 * j + 1] / dg, sr[3 * j + 2] / dg, T(0)};
      sd[3 * j] = sd[3 * j + 1] = sd[3 * j + 2] = T(0);
      a0[0] += bi.x * bi.x + bi.y * bi.y + bi.z * bi.z;
      a0[1] += rx * rx + ry * ry + rz * rz;
    }
    cluster_reduce(a0, 2);  // also publishes u
    const double bb = tot[0];
    double rr = tot[1];
    int it = 0;
    if (bb > 0.0 && rr > d.tol2 * bb) {
      double a1[2] = {0.0, 0.0};
      for (int j = threadIdx.x; j < nmine; j += blockDim.x) {
        T ax, ay, az;
        spmv_u(j, ax, ay, az);
        const R4<T> uj = su[j];
        sw[3 * j] = ax; sw[3 * j + 1] = ay; sw[3 * j + 2] = az;
        sp[3 * j] = uj.x; sp[3 * j + 1] = uj.y; sp[3 * j + 2] = uj.z;
        ss[3 * j] = ax; ss[3 * j + 1] = ay; ss[3 * j + 2] = az;
        a1[0] += (double)sr[3 * j] * uj.x + (double)sr[3 * j + 1] * uj.y + (double)sr[3 * j + 2] * uj.z;
        a1[1] += (double)ax * uj.x + (double)ay * uj.y + (double)az * uj.z;
      }
      cluster_reduce(a1, 2);
      double gamma = tot[0];
      double alpha = gamma / tot[1];
      for (it = 1; it <= d.max_iter; ++it) {
        const T ta = (T)alpha;
        for (int j = threadIdx.x; j < nmine; j += blockDim.x) {
          const T dg = sg[j];
          T un[3];
          for (int c = 0; c < 3; ++c) {
            sd[3 * j + c] += ta * sp[3 * j + c];
            sr[3 * j + c] -= ta * ss[3 * j + c];
            un[c] = sr[3 * j + c] / dg;
          }
          su[j] = R4<T>{un[0], un[1], un[2], T(0)};
        }
        cl.sync();  // u published to the cluster
        double a2[3] = {0.0, 0.0, 0.0};
        for (int j = threadIdx.x; j < nmine; j += blockDim.x) {
          T ax, ay, az;
          spmv_u(j, ax, ay, az);
          const R4<T> uj = su[j];
          sw[3 * j] = ax; sw[3 * j + 1] = ay; sw[3 * j + 2] = az;
          const T r0 = sr[3 * j], r1 = sr[3 * j + 1], r2 = sr[3 * j + 2];
          a2[0] += (double)r0 * uj.x + (double)r1 * uj.y + (double)r2 * uj.z;
          a2[1] += (double)ax * uj.x + (double)ay * uj.y + (double)az * uj.z;
          a2[2] += (double)r0 * r0 + (double)r1 * r1 + (double)r2 * r2;
        }
        cluster_reduce(a2, 3);
        const double gnew = tot[0], delta = tot[1];
        rr = tot[2];
        if (!isfinite(gnew) || !isfinite(delta) || !isfinite(rr)) {
          if (crank == 0 && threadIdx.x == 0) set_status(d.ctrl, ST_NONFINITE);
          break;
        }
        if (rr <= d.tol2 * bb) break;
        const double beta = gnew / gamma;
        alpha = gnew / (delta - beta * gnew / alpha);
        gamma = gnew;
        const T tb = (T)beta;
        for (int j = threadIdx.x; j < nmine; j += blockDim.x) {
          const R4<T> uj = su[j];
          const T uu[3] = {uj.x, uj.y, uj.z};
          for (int c = 0; c < 3; ++c) {
            sp[3 * j + c] = uu[c] + tb * sp[3 * j + c];
            ss[3 * j + c] = sw[3 * j + c] + tb * ss[3 * j + c];
          }
        }
      }
      if (it > d.max_iter) {
        it = d.max_iter;
        if (crank == 0 && threadIdx.x == 0) set_status(d.ctrl, ST_PCG_MAXIT);
      }
      for (int j = threadIdx.x; j < nmine; j += blockDim.x) {
        const int i = row0 + my0 + j;
        R4<T> xi = d.X[i];
        xi.x += sd[3 * j];
        xi.y += sd[3 * j + 1];
        xi.z += sd[3 * j + 2];
        d.X[i] = xi;
      }
    }
    if (crank == 0 && threadIdx.x == 0) {
      IterRec* rec = d.hist + (d.ctrl->iter % d.hist_cap);
      atomicMax(&rec->pcg_iters, it);
      atomicAdd(reinterpret_cast<unsigned long long*>(&d.ctrl->total_pcg), (unsigned long long)it);
      const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
      atomicMax(reinterpret_cast<unsigned long long*>(&rec->pcg_rel_residual),
                (unsigned long long)__double_as_longlong(rel));
    }
    cl.sync();  // shared memory is reused by the next robot
  }
}

// --------------------------------------------------------------- finalize
template <typename T>
__global__ void k_finalize(Dev<T> d) {
  __shared__ double sh[32];
  const int n = d.n_e_local + d.n_e_spring;
  // fixed-order sum: eight interleaved thread-strided chains (so that the
  // loads overlap), added in a fixed order, then a fixed tree
  constexpr int K = 8;
  double a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
  const int step = (int)blockDim.x * K;
  for (int i0 = threadIdx.x; i0 < n; i0 += step) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = i0 + k * (int)blockDim.x;
      if (i < n) a[k] += d.e_partials[i];
    }
  }
  double at = 0.0;
#pragma unroll
  for (int k = 0; k < K; ++k) at += a[k];
  const double t = block_sum(at, sh);
  if (threadIdx.x == 0) finalize_iteration(d, t);
}

template <typename T>
__global__ void k_gather_positions(const R4<T>* X, const int* int_of_user, int n, T* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const R4<T> x = X[int_of_user[i]];
  out[3 * (size_t)i] = x.x;
  out[3 * (size_t)i + 1] = x.y;
  out[3 * (size_t)i + 2] = x.z;
}

// ---------------------------------------------------------------- launchers
int local_blocks(int n_t, int threads) { return (n_t + threads - 1) / threads; }
int rhs_blocks(int n_free, int threads) { return (n_free + threads - 1) / threads; }
int local_blocks(int n_t) { return local_blocks(n_t, LOCAL_THREADS); }
int rhs_blocks(int n_free) { return rhs_blocks(n_free, RHS_THREADS); }

// The block sizes are launch-shape choices of the autotuner: each allowed
// size is its own instantiation (compiled with its own launch bound).
template <typename T>
void launch_local(const Dev<T>& d, cudaStream_t st) {
  if (d.n_t == 0) return;
  const int bs = d.local_threads > 0 ? d.local_threads : LOCAL_THREADS;
  const int nb = local_blocks(d.n_t, bs);
  constexpr int SW = sizeof(T) == 4 ? 4 : 6;
  if (bs == 64)
    k_local<T, SW, 64><<<nb, 64, 0, st>>>(d);
  else if (bs == 256)
    k_local<T, SW, 256><<<nb, 256, 0, st>>>(d);
  else
    k_local<T, SW, 128><<<nb, 128, 0, st>>>(d);
}

template <typename T>
void launch_rhs(const Dev<T>& d, cudaStream_t st) {
  if (d.n_free == 0) return;
  const int bs = d.rhs_threads > 0 ? d.rhs_threads : RHS_THREADS;
  const int nb = rhs_blocks(d.n_free, bs);
  if (bs == 128)
    k_rhs<T, 128><<<nb, 128, 0, st>>>(d);
  else if (bs == 512)
    k_rhs<T, 512><<<nb, 512, 0, st>>>(d);
  else
    k_rhs<T, 256><<<nb, 256, 0, st>>>(d);
}

template <typename T>
int pcg_max_grid() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg<T>, PCG_THREADS, 0);
  return sms * (per > 0 ? per : 1);
}

template <typename T>
int pcg_rr_max_rows() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_rr<T, PCG_RR_MAXW>, PCG_RR_THREADS, 0);
  return sms * per * PCG_RR_THREADS;
}

template <int ROWS>
static bool pcg_df_prepare_rows(int smem_bytes) {
  return cudaFuncSetAttribute(k_pcg_df<PCG_RR_MAXW, false, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_bytes) == cudaSuccess &&
         cudaFuncSetAttribute(k_pcg_df<PCG_RR_MAXW, true, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_bytes) == cudaSuccess;
}
bool pcg_df_prepare(int rows, int smem_bytes) {
  return rows == PCG_DF_ROWS_SMALL ? pcg_df_prepare_rows<PCG_DF_ROWS_SMALL>(smem_bytes)
                                   : pcg_df_prepare_rows<PCG_DF_THREADS>(smem_bytes);
}

int pcg_df_max_rows(int rows) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (rows == PCG_DF_ROWS_SMALL)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_df<PCG_RR_MAXW, true, PCG_DF_ROWS_SMALL>, rows, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_df<PCG_RR_MAXW, true, PCG_DF_THREADS>, rows, 0);
  const int blocks = std::min(sms * per, 32 * DF_MAXQ);
  return blocks * rows;
}

template <typename T>
cudaError_t launch_pcg(const Dev<T>& d, int grid, int variant, cudaStream_t st) {
  if (d.n_free == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(variant == 5 ? d.df_rows : variant == 2 ? PCG_RR_THREADS : PCG_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (variant == 5) {
    if constexpr (std::is_same<T, float>::value) {
      // epoch-tagged words start from zero in every launch
      cudaError_t e = cudaMemsetAsync(d.df_u, 0, sizeof(unsigned long long) * 4 * (size_t)d.n_free, st);
      if (e == cudaSuccess)
        e = cudaMemsetAsync(d.df_p, 0,
                            sizeof(unsigned long long) * PCG_DF_REPLICAS * 2 * DF_SLOT_C * (size_t)(grid + 1), st);
      if (e != cudaSuccess) return e;
      cfg.dynamicSmemBytes = 16 * (size_t)d.halo_max;
      const bool small = d.df_rows == PCG_DF_ROWS_SMALL;
      if (d.n_agg > 0) {
        cfg.dynamicSmemBytes += sizeof(float) * DF_AGG * (size_t)d.n_agg;
        return small ? cudaLaunchKernelEx(&cfg, k_pcg_df<PCG_RR_MAXW, true, PCG_DF_ROWS_SMALL>, d)
                     : cudaLaunchKernelEx(&cfg, k_pcg_df<PCG_RR_MAXW, true, PCG_DF_THREADS>, d);
      }
      return small ? cudaLaunchKernelEx(&cfg, k_pcg_df<PCG_RR_MAXW, false, PCG_DF_ROWS_SMALL>, d)
                   : cudaLaunchKernelEx(&cfg, k_pcg_df<PCG_RR_MAXW, false, PCG_DF_THREADS>, d);
    } else {
      return cudaErrorInvalidValue;
    }
  }
  if (variant == 2) return cudaLaunchKernelEx(&cfg, k_pcg_rr<T, PCG_RR_MAXW>, d);
  return cudaLaunchKernelEx(&cfg, k_pcg<T>, d);
}

template <typename T>
void launch_finalize(const Dev<T>& d, cudaStream_t st) {
  k_finalize<T><<<1, 1024, 0, st>>>(d);
}

template <typename T>
void launch_gather_positions(const Dev<T>& d, const int* int_of_user, int n_user, T* out,
                             cudaStream_t st) {
  if (n_user == 0) return;
  k_gather_positions<T><<<(n_user + 255) / 256, 256, 0, st>>>(d.X, int_of_user, n_user, out);
}

template <typename T>
int pcg_cluster_rows_cap() {
  // per row: u (R4) + r, p, s, w, d, diag (3+3+3+3+3+1 values)
  const size_t per_row = sizeof(R4<T>) + 16 * sizeof(T);
  const size_t avail = 220 * 1024;
  return (int)((avail / per_row) & ~size_t(31));
}

template <typename T>
int pcg_cluster_max_clusters(int rows_cap) {
  const size_t smem = (sizeof(R4<T>) + 16 * sizeof(T)) * (size_t)rows_cap;
  if (cudaFuncSetAttribute(k_pcg_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cudaFuncSetAttribute(k_pcg_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PCG_CL_SIZE);
  cfg.blockDim = dim3(PCG_CL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PCG_CL_SIZE;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_pcg_cluster<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T>
cudaError_t launch_pcg_cluster(const Dev<T>& d, int n_clusters, cudaStream_t st) {
  if (d.n_free == 0) return cudaSuccess;
  const size_t smem = (sizeof(R4<T>) + 16 * sizeof(T)) * (size_t)d.cl_rows_cap;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(PCG_CL_SIZE * n_clusters);
  cfg.blockDim = dim3(PCG_CL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = PCG_CL_SIZE;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_pcg_cluster<T>, d);
}

template <typename T>
int pcg_seg_max_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_seg<T, std::is_same<T, float>::value>,
                                                PCG_SEG_THREADS, 0);
  return sms * per;
}

template <typename T>
cudaError_t launch_pcg_seg(const Dev<T>& d, int blocks, cudaStream_t st) {
  if (d.n_free == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(PCG_SEG_THREADS);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if constexpr (std::is_same<T, float>::value) {
    if (d.seg_coarse) return cudaLaunchKernelEx(&cfg, k_pcg_seg<T, true>, d);
  }
  return cudaLaunchKernelEx(&cfg, k_pcg_seg<T, false>, d);
}

template int pcg_seg_max_blocks<float>();
template int pcg_seg_max_blocks<double>();
template cudaError_t launch_pcg_seg<float>(const Dev<float>&, int, cudaStream_t);
template cudaError_t launch_pcg_seg<double>(const Dev<double>&, int, cudaStream_t);
template int pcg_cluster_rows_cap<float>();
template int pcg_cluster_rows_cap<double>();
template int pcg_cluster_max_clusters<float>(int);
template int pcg_cluster_max_clusters<double>(int);
template cudaError_t launch_pcg_cluster<float>(const Dev<float>&, int, cudaStream_t);
template cudaError_t launch_pcg_cluster<double>(const Dev<double>&, int, cudaStream_t);
template void launch_local<float>(const Dev<float>&, cudaStream_t);
template void launch_local<double>(const Dev<double>&, cudaStream_t);
template void launch_rhs<float>(const Dev<float>&, cudaStream_t);
template void launch_rhs<double>(const Dev<double>&, cudaStream_t);
template cudaError_t launch_pcg<float>(const Dev<float>&, int, int, cudaStream_t);
template cudaError_t launch_pcg<double>(const Dev<double>&, int, int, cudaStream_t);
template int pcg_rr_max_rows<float>();
template int pcg_rr_max_rows<double>();
template int pcg_max_grid<float>();
template int pcg_max_grid<double>();
template void launch_finalize<float>(const Dev<float>&, cudaStream_t);
template void launch_finalize<double>(const Dev<double>&, cudaStream_t);
template void launch_gather_positions<float>(const Dev<float>&, const int*, int, float*, cudaStream_t);
template void launch_gather_positions<double>(const Dev<double>&, const int*, int, double*,
                                              cudaStream_t);

}  // namespace casim
