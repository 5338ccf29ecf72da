// Reverse pass of the unrolled local-global loop: gradients of a loss on the
// final positions with respect to the chamber volume ratios alpha_g.
//
// One outer iteration maps X_i to X_{i+1} = A_i^-1 b(X_i, alpha, S_i) with
// the spring decisions S_i (which vertices carry springs, kind, face or
// sphere) held fixed (they are discrete).  Given g = dL/dX_{i+1} on the free
// rows, the reverse of iteration i is
//   mu = A_i^-1 g                       (A_i symmetric; same PCG kernels),
//   Pbar_e[:, j] = w_e mu_{v_j},  cbar_v = k mu_v,
//   Xbar_i = (local-step VJP) + (spring-target VJP),  abar_g += (1/3) a^(-2/3) <Pbar_e, R_e T_c>.
// Local-step VJP (per tet): the rotation R = polar(D), D = X_c T_c^T, S = R^T D,
// has the derivative dR = R [w]x with (tr(S) I - S) w = vec(R^T dD), so a
// gradient Rbar pulls back to Dbar = R [y]x with (tr(S) I - S) y = vec(R^T Rbar);
// the body blend, the strain table w(eps) (eps's dependence on R vanishes at
// the optimal rotation) and the volume scaling of Eq. 7 are differentiated
// directly.  Spring-target VJP (per spring): sphere projection; face point
// with barycentric weights plus eps times the unit face normal; for a spring
// whose ray was cast this iteration, the barycentric weights of the ray-plane
// hit x_v + t d, d = -n(v)/|n(v)|, through the vertex normal n(v) of the
// incident boundary faces.  Barycentric adjoints of kept springs accumulate
// across iterations until the iteration that cast them.  Every sum is formed
// in a fixed order (per-tet pullbacks by incidence, spring pullbacks by
// emission slot), so the reverse pass is bitwise reproducible.
#include "common.cuh"
#include "kernels.h"
#include "svd3.cuh"

namespace casim {

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return {x, y, z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dotd(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 crossd(D3 a, D3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double normd(D3 a) { return sqrt(dotd(a, a)); }

template <typename T>
__device__ __forceinline__ D3 posd(const R4<T>* X, int v) {
  const R4<T> a = X[v];
  return {(double)a.x, (double)a.y, (double)a.z};
}

// One spring's contributions go to consecutive slots starting at its base.
struct Emit {
  int* vert;
  R4<double>* val;
  size_t pos;
  __device__ __forceinline__ void put(int v, D3 a) {
    vert[pos] = v;
    val[pos] = R4<double>{a.x, a.y, a.z, 0.0};
    ++pos;
  }
};

// slope of the piecewise-linear w(eps) table at eps (0 where clamped)
__device__ __forceinline__ double w_and_slope(const double* k, int n, double eps, double& slope) {
  slope = 0.0;
  if (eps <= k[0]) return k[1];
  for (int i = 0; i + 1 < n; ++i) {
    const double x0 = k[2 * i], x1 = k[2 * i + 2];
    if (eps < x1) {
      const double y0 = k[2 * i + 1], y1 = k[2 * i + 3];
      slope = (y1 - y0) / (x1 - x0);
      return y0 + (eps - x0) * slope;
    }
  }
  return k[2 * n - 1];
}

template <typename T, int SWEEPS>
__global__ void __launch_bounds__(128) k_adj_local(Dev<T> d, AdjDev<T> a) {
  __shared__ double s_contrib[128];
  __shared__ int s_group[128];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double acontrib = 0.0;
  int grp = -1;
  if (e < d.n_t) {
    const int4 t = d.tet[e];
    const int tv[4] = {t.x, t.y, t.z, t.w};
    // forward recomputation (in the working precision, as the forward did)
    const R4<T> x0 = a.Xi[t.x], x1 = a.Xi[t.y], x2 = a.Xi[t.z], x3 = a.Xi[t.w];
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
    T Rt[3][3], trt;
    kabsch_rotation<T, SWEEPS>(D, Rt, trt);
    // from here on FP64
    double R[3][3], X[3][4], Tc[3][4], RT[3][4];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) R[i][j] = (double)Rt[i][j];
      for (int k = 0; k < 4; ++k) {
        X[i][k] = (double)Xc[i][k];
        Tc[i][k] = (double)Tm[i][k];
      }
    }
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 4; ++k) RT[i][k] = R[i][0] * Tc[0][k] + R[i][1] * Tc[1][k] + R[i][2] * Tc[2][k];
    const R4<T> info = d.tinfo[e];
    const double omega = (double)info.x, vol0 = (double)info.y, tt = (double)info.z;
    const int g = (int)info.w;
    double Pb[3][4];
    for (int k = 0; k < 4; ++k) {
      const int v = tv[k];
      double mx = 0.0, my = 0.0, mz = 0.0;
      if (v < d.n_free) {
        const R4<T> mv = a.mu[v];
        mx = mv.x;
        my = mv.y;
        mz = mv.z;
      }
      Pb[0][k] = omega * mx;
      Pb[1][k] = omega * my;
      Pb[2][k] = omega * mz;
    }
    double Rb[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double Xb[3][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};
    if (g >= 0) {
      const double al = a.alpha[g];
      const double c = cbrt(al);
      double pr = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) pr += Pb[i][k] * RT[i][k];
      acontrib = pr * c / (3.0 * al);  // d cbrt(a)/da = cbrt(a) / (3a)
      grp = g;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double s = 0.0;
          for (int k = 0; k < 4; ++k) s += Pb[i][k] * Tc[j][k];
          Rb[i][j] = c * s;
        }
    } else {
      double mis = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) {
          const double q = X[i][k] - RT[i][k];
          mis += q * q;
        }
      const double eps = sqrt(mis / tt);
      double slope;
      const double w = w_and_slope(d.knots, d.n_knots, eps, slope);
      double B[3][4];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) B[i][k] = (1.0 - w) * X[i][k] + w * RT[i][k];
      const D3 e1 = d3(B[0][1] - B[0][0], B[1][1] - B[1][0], B[2][1] - B[2][0]);
      const D3 e2 = d3(B[0][2] - B[0][0], B[1][2] - B[1][0], B[2][2] - B[2][0]);
      const D3 e3 = d3(B[0][3] - B[0][0], B[1][3] - B[1][0], B[2][3] - B[2][0]);
      const double volB = dotd(e1, crossd(e2, e3)) / 6.0;
      const bool scaled = volB > 1e-3 * vol0;
      const double s = scaled ? cbrt(vol0 / volB) : 1.0;
      double Bb[3][4];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) Bb[i][k] = s * Pb[i][k];
      if (scaled) {
        double sb = 0.0;
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 4; ++k) sb += Pb[i][k] * B[i][k];
        const double volb = sb * (-s / (3.0 * volB));
        const D3 g1 = (1.0 / 6.0) * crossd(e2, e3), g2 = (1.0 / 6.0) * crossd(e3, e1),
                 g3 = (1.0 / 6.0) * crossd(e1, e2);
        const D3 gs[3] = {g1, g2, g3};
        for (int k = 1; k < 4; ++k) {
          Bb[0][k] += volb * gs[k - 1].x;
          Bb[1][k] += volb * gs[k - 1].y;
          Bb[2][k] += volb * gs[k - 1].z;
        }
        const D3 g0 = d3(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
        Bb[0][0] += volb * g0.x;
        Bb[1][0] += volb * g0.y;
        Bb[2][0] += volb * g0.z;
      }
      double wb = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 4; ++k) {
          Xb[i][k] += (1.0 - w) * Bb[i][k];
          wb += Bb[i][k] * (RT[i][k] - X[i][k]);
        }
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double sacc = 0.0;
          for (int k = 0; k < 4; ++k) sacc += Bb[i][k] * Tc[j][k];
          Rb[i][j] = w * sacc;
        }
      if (eps > 0.0) {
        const double eb = wb * slope;
        const double f = eb / (tt * eps);
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 4; ++k) Xb[i][k] += f * (X[i][k] - RT[i][k]);
      }
    }
    // polar-factor pullback: Dbar = R [y]x, (tr(S) I - S) y = vec(R^T Rbar), S = R^T D
    double S[3][3], M[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < 3; ++k) {
          s1 += R[k][i] * (double)D[k][j];
          s2 += R[k][i] * Rb[k][j];
        }
        S[i][j] = s1;
        M[i][j] = s2;
      }
    // symmetrise S (equal to R^T D up to rounding)
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j) {
        const double m = 0.5 * (S[i][j] + S[j][i]);
        S[i][j] = S[j][i] = m;
      }
    const double av[3] = {M[2][1] - M[1][2], M[0][2] - M[2][0], M[1][0] - M[0][1]};
    const double trS = S[0][0] + S[1][1] + S[2][2];
    double K[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) K[i][j] = (i == j ? trS : 0.0) - S[i][j];
    const double det = K[0][0] * (K[1][1] * K[2][2] - K[1][2] * K[2][1]) -
                       K[0][1] * (K[1][0] * K[2][2] - K[1][2] * K[2][0]) +
                       K[0][2] * (K[1][0] * K[2][1] - K[1][1] * K[2][0]);
    double y[3] = {0.0, 0.0, 0.0};
    if (det != 0.0) {
      double Ki[3][3];
      Ki[0][0] = (K[1][1] * K[2][2] - K[1][2] * K[2][1]) / det;
      Ki[0][1] = (K[0][2] * K[2][1] - K[0][1] * K[2][2]) / det;
      Ki[0][2] = (K[0][1] * K[1][2] - K[0][2] * K[1][1]) / det;
      Ki[1][0] = (K[1][2] * K[2][0] - K[1][0] * K[2][2]) / det;
      Ki[1][1] = (K[0][0] * K[2][2] - K[0][2] * K[2][0]) / det;
      Ki[1][2] = (K[0][2] * K[1][0] - K[0][0] * K[1][2]) / det;
      Ki[2][0] = (K[1][0] * K[2][1] - K[1][1] * K[2][0]) / det;
      Ki[2][1] = (K[0][1] * K[2][0] - K[0][0] * K[2][1]) / det;
      Ki[2][2] = (K[0][0] * K[1][1] - K[0][1] * K[1][0]) / det;
      for (int i = 0; i < 3; ++i) y[i] = Ki[i][0] * av[0] + Ki[i][1] * av[1] + Ki[i][2] * av[2];
    }
    const double Y[3][3] = {{0.0, -y[2], y[1]}, {y[2], 0.0, -y[0]}, {-y[1], y[0], 0.0}};
    double Db[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Db[i][j] = R[i][0] * Y[0][j] + R[i][1] * Y[1][j] + R[i][2] * Y[2][j];
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 4; ++k) Xb[i][k] += Db[i][0] * Tc[0][k] + Db[i][1] * Tc[1][k] + Db[i][2] * Tc[2][k];
    // X_c = X_e N  ->  Xbar_e = Xbar_c N (N symmetric)
    for (int i = 0; i < 3; ++i) {
      const double m = 0.25 * (Xb[i][0] + Xb[i][1] + Xb[i][2] + Xb[i][3]);
      for (int k = 0; k < 4; ++k) Xb[i][k] -= m;
    }
    for (int k = 0; k < 4; ++k) a.xbar_tet[4 * (size_t)e + k] = R4<double>{Xb[0][k], Xb[1][k], Xb[2][k], 0.0};
  }
  // deterministic per-block sums of the alpha contributions, group by group
  s_contrib[threadIdx.x] = acontrib;
  s_group[threadIdx.x] = grp;
  __syncthreads();
  if (threadIdx.x < a.n_groups) {
    double sacc = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i)
      if (s_group[i] == (int)threadIdx.x) sacc += s_contrib[i];
    a.alpha_part[(size_t)blockIdx.x * a.n_groups + threadIdx.x] = sacc;
  }
}

// Barycentric weights (of q1, q2) of a point b in the triangle's plane, and
// the pullback of their adjoint bb onto b and the three vertices.
__device__ __forceinline__ void bary_vjp(D3 b, D3 q0, D3 q1, D3 q2, double bb1, double bb2, D3& gb, D3& g0,
                                         D3& g1, D3& g2) {
  const D3 e1 = q1 - q0, e2 = q2 - q0, r = b - q0;
  const double d11 = dotd(e1, e1), d12 = dotd(e1, e2), d22 = dotd(e2, e2);
  const double r1 = dotd(r, e1), r2 = dotd(r, e2);
  const double den = d11 * d22 - d12 * d12;
  const double be1 = (d22 * r1 - d12 * r2) / den, be2 = (d11 * r2 - d12 * r1) / den;
  const double rb1 = (bb1 * d22 - bb2 * d12) / den;
  const double rb2 = (-bb1 * d12 + bb2 * d11) / den;
  const double db11 = (bb1 * (-be1 * d22) + bb2 * (r2 - be2 * d22)) / den;
  const double db12 = (bb1 * (-r2 + 2.0 * be1 * d12) + bb2 * (-r1 + 2.0 * be2 * d12)) / den;
  const double db22 = (bb1 * (r1 - be1 * d11) + bb2 * (-be2 * d11)) / den;
  D3 ge1 = (2.0 * db11) * e1 + db12 * e2 + rb1 * r;
  D3 ge2 = (2.0 * db22) * e2 + db12 * e1 + rb2 * r;
  const D3 gr = rb1 * e1 + rb2 * e2;
  gb = gr;
  g1 = ge1;
  g2 = ge2;
  g0 = d3(0, 0, 0) - gr - ge1 - ge2;
}

// pullback of n = (q1 - q0) x (q2 - q0) onto the vertices
__device__ __forceinline__ void cross_vjp(D3 q0, D3 q1, D3 q2, D3 nb, D3& g0, D3& g1, D3& g2) {
  const D3 e1 = q1 - q0, e2 = q2 - q0;
  const D3 ge1 = crossd(e2, nb), ge2 = crossd(nb, e1);
  g1 = ge1;
  g2 = ge2;
  g0 = d3(0, 0, 0) - ge1 - ge2;
}

template <typename T>
__global__ void __launch_bounds__(128) k_adj_springs(Dev<T> d, AdjDev<T> a) {
  const int qi = blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= d.n_q) return;
  if (!a.sp_active[qi]) {
    a.betabar[2 * qi] = 0.0;
    a.betabar[2 * qi + 1] = 0.0;
    return;
  }
  if (a.sp_kind[qi] == 2) {
    // tetrahedral-obstacle spring: the target is a point of the rigid
    // obstacle, held constant (its weights are not differentiated)
    a.betabar[2 * qi] = 0.0;
    a.betabar[2 * qi + 1] = 0.0;
    return;
  }
  const int v = d.q_verts[qi];
  Emit em{a.em_vert, a.em_val, 4 * (size_t)qi + 3 * (size_t)d.qf_ptr[qi]};
  const R4<T> mv = a.mu[v];
  const D3 cb = (double)d.k_spring * d3(mv.x, mv.y, mv.z);
  const D3 x = posd(a.Xi, v);
  const double eps = d.eps;
  if (a.sp_kind[qi] == 1) {
    const int j = a.sp_face[qi];
    const D3 c = d3(d.spheres[4 * j], d.spheres[4 * j + 1], d.spheres[4 * j + 2]);
    const double r = d.spheres[4 * j + 3];
    const D3 u = x - c;
    const double nu = normd(u);
    if (nu > 0.0) {
      const D3 uh = (1.0 / nu) * u;
      em.put(v, ((r + eps) / nu) * (cb - dotd(uh, cb) * uh));
    }
    a.betabar[2 * qi] = 0.0;
    a.betabar[2 * qi + 1] = 0.0;
    return;
  }
  const int f = a.sp_face[qi];
  const int4 fv = d.faces[f];
  const D3 q0 = posd(a.Xi, fv.x), q1 = posd(a.Xi, fv.y), q2 = posd(a.Xi, fv.z);
  const double b1 = a.sp_bary[2 * qi], b2 = a.sp_bary[2 * qi + 1];
  // c = (1 - b1 - b2) q0 + b1 q1 + b2 q2 + eps n / |n|
  D3 g0 = (1.0 - b1 - b2) * cb, g1 = b1 * cb, g2 = b2 * cb;
  double bb1 = a.betabar[2 * qi] + dotd(q1 - q0, cb);
  double bb2 = a.betabar[2 * qi + 1] + dotd(q2 - q0, cb);
  const D3 n = crossd(q1 - q0, q2 - q0);
  const double nn = normd(n);
  const D3 nh = (1.0 / nn) * n;
  D3 nb = (eps / nn) * (cb - dotd(nh, cb) * nh);
  if (a.sp_flag[qi] == 1) {
    // weights from this iteration's ray cast: b = x + t d, t = n.(q0 - x) / n.d
    D3 m = d3(0, 0, 0);
    for (int k = d.qf_ptr[qi]; k < d.qf_ptr[qi + 1]; ++k) {
      const int4 gv = d.faces[d.qf[k]];
      const D3 p0 = posd(a.Xi, gv.x), p1 = posd(a.Xi, gv.y), p2 = posd(a.Xi, gv.z);
      m = m + crossd(p1 - p0, p2 - p0);
    }
    const double mn = normd(m);
    const D3 mh = (1.0 / mn) * m;
    const D3 dir = d3(0, 0, 0) - mh;
    const double Nn = dotd(n, q0 - x), Dn = dotd(n, dir);
    const double t = Nn / Dn;
    const D3 hit = x + t * dir;
    D3 gb, h0, h1, h2;
    bary_vjp(hit, q0, q1, q2, bb1, bb2, gb, h0, h1, h2);
    g0 = g0 + h0;
    g1 = g1 + h1;
    g2 = g2 + h2;
    D3 xb = gb;
    D3 db = t * gb;
    const double tb = dotd(gb, dir);
    const double Nb = tb / Dn, Db = -tb * t / Dn;
    nb = nb + Nb * (q0 - x) + Db * dir;
    g0 = g0 + Nb * n;
    xb = xb - Nb * n;
    db = db + Db * n;
    // dir = -m / |m|
    const D3 mb = (-1.0 / mn) * (db - dotd(mh, db) * mh);
    for (int k = d.qf_ptr[qi]; k < d.qf_ptr[qi + 1]; ++k) {
      const int4 gv = d.faces[d.qf[k]];
      const D3 p0 = posd(a.Xi, gv.x), p1 = posd(a.Xi, gv.y), p2 = posd(a.Xi, gv.z);
      D3 r0, r1, r2;
      cross_vjp(p0, p1, p2, mb, r0, r1, r2);
      em.put(gv.x, r0);
      em.put(gv.y, r1);
      em.put(gv.z, r2);
    }
    em.put(v, xb);
    bb1 = 0.0;
    bb2 = 0.0;
  } else if (a.sp_flag[qi] == 2) {
    // weights of a closest-point fallback: constant, their adjoint ends here
    bb1 = 0.0;
    bb2 = 0.0;
  }
  D3 c0, c1, c2;
  cross_vjp(q0, q1, q2, nb, c0, c1, c2);
  em.put(fv.x, g0 + c0);
  em.put(fv.y, g1 + c1);
  em.put(fv.z, g2 + c2);
  a.betabar[2 * qi] = bb1;
  a.betabar[2 * qi + 1] = bb2;
}

// Grouping of the spring contributions by destination row (contributions to
// fixed vertices are dropped: they have no row).
__global__ void k_em_count(const int* __restrict__ em_vert, int n_slots, int n_free, int* cnt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const int u = em_vert[s];
  if (u >= 0 && u < n_free) atomicAdd(&cnt[u], 1);
}
__global__ void k_em_fill(const int* __restrict__ em_vert, int n_slots, int n_free, const int* __restrict__ start,
                          int* cur, int* list) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const int u = em_vert[s];
  if (u >= 0 && u < n_free) list[start[u] + atomicAdd(&cur[u], 1)] = s;
}

// g_v = (spring contributions to v, added in slot order) + (sum over incident
// (tet, slot) of Xbar_tet, in incidence order).  The fill order of a row's
// slot list depends on timing, so each row sorts its list first (insertion
// sort; a row receives a few tens of contributions at most); the result is
// independent of the launch's timing.
template <typename T>
__global__ void __launch_bounds__(256) k_adj_gather(Dev<T> d, AdjDev<T> a) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= d.n_free) return;
  int* L = a.em_list + a.em_start[v];
  const int n = a.em_start[v + 1] - a.em_start[v];
  for (int i = 1; i < n; ++i) {
    const int key = L[i];
    int j = i - 1;
    while (j >= 0 && L[j] > key) {
      L[j + 1] = L[j];
      --j;
    }
    L[j + 1] = key;
  }
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int i = 0; i < n; ++i) {
    const R4<double> c = a.em_val[L[i]];
    gx += c.x;
    gy += c.y;
    gz += c.z;
  }
  for (int k = d.inc_ptr[v]; k < d.inc_ptr[v + 1]; ++k) {
    const R4<double> c = a.xbar_tet[d.inc[k]];
    gx += c.x;
    gy += c.y;
    gz += c.z;
  }
  a.g[v] = R4<double>{gx, gy, gz, 0.0};
}

// diagonal of A_i = L + k diag(mask_i): the Laplacian diagonal first, then
// (second kernel) the springs of iteration i
template <typename T>
__global__ void k_adj_diag_base(Dev<T> d) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < d.n_free) d.diag[v] = d.diagL[v];
}

template <typename T>
__global__ void k_adj_diag_springs(Dev<T> d, AdjDev<T> a) {
  const int qi = blockIdx.x * blockDim.x + threadIdx.x;
  if (qi < d.n_q && a.sp_active[qi]) {
    const int u = d.q_verts[qi];
    d.diag[u] = d.diagL[u] + (T)d.k_spring;
  }
}

// Cast of query vertex qi's spring in this iteration: 1 by a ray hit (self
// spring of a vertex found in a self pair and in no sphere), 2 by the
// closest-point fallback (weights held constant in the reverse pass), 0 none
template <typename T>
__global__ void k_adj_flags(Dev<T> d, int* flag) {
  const int qi = blockIdx.x * blockDim.x + threadIdx.x;
  if (qi >= d.n_q) return;
  const bool cast = d.sp.active[qi] && d.sp.kind[qi] == 0 && d.pair_count[qi] > 0 && d.obs_sphere[qi] < 0;
  flag[qi] = cast ? (d.sp.fallback[qi] ? 2 : 1) : 0;
}

__global__ void k_adj_alpha_reduce(const double* part, int n_blocks, int n_groups, double* abar) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  double s = 0.0;
  for (int b = 0; b < n_blocks; ++b) s += part[(size_t)b * n_groups + g];
  abar[g] += s;
}

template <typename T>
void launch_adjoint_step(const Dev<T>& d, const AdjDev<T>& a, cudaStream_t st) {
  const int nb = local_blocks(d.n_t);
  if (sizeof(T) == 4)
    k_adj_local<T, 4><<<nb, 128, 0, st>>>(d, a);
  else
    k_adj_local<T, 6><<<nb, 128, 0, st>>>(d, a);
  if (a.n_groups > 0) k_adj_alpha_reduce<<<(a.n_groups + 63) / 64, 64, 0, st>>>(a.alpha_part, nb, a.n_groups, a.abar);
  cudaMemsetAsync(a.em_cnt, 0, sizeof(int) * ((size_t)d.n_free + 1), st);
  cudaMemsetAsync(a.em_cur, 0, sizeof(int) * ((size_t)d.n_free + 1), st);
  if (a.n_slots > 0) {
    cudaMemsetAsync(a.em_vert, 0xff, sizeof(int) * (size_t)a.n_slots, st);
    if (d.n_q > 0) k_adj_springs<T><<<(d.n_q + 127) / 128, 128, 0, st>>>(d, a);
    k_em_count<<<(a.n_slots + 255) / 256, 256, 0, st>>>(a.em_vert, a.n_slots, d.n_free, a.em_cnt);
  }
  launch_scan_exclusive(a.em_cnt, a.em_start, d.n_free + 1, a.em_tiles, a.em_total, st);
  if (a.n_slots > 0)
    k_em_fill<<<(a.n_slots + 255) / 256, 256, 0, st>>>(a.em_vert, a.n_slots, d.n_free, a.em_start, a.em_cur,
                                                        a.em_list);
  if (d.n_free > 0) k_adj_gather<T><<<(d.n_free + 255) / 256, 256, 0, st>>>(d, a);
}

template <typename T>
void launch_adjoint_diag(const Dev<T>& d, const AdjDev<T>& a, cudaStream_t st) {
  if (d.n_free > 0) k_adj_diag_base<T><<<(d.n_free + 255) / 256, 256, 0, st>>>(d);
  if (d.n_q > 0) k_adj_diag_springs<T><<<(d.n_q + 255) / 256, 256, 0, st>>>(d, a);
}

template <typename T>
void launch_adjoint_flags(const Dev<T>& d, int* flag, cudaStream_t st) {
  if (d.n_q > 0) k_adj_flags<T><<<(d.n_q + 255) / 256, 256, 0, st>>>(d, flag);
}

template void launch_adjoint_step<float>(const Dev<float>&, const AdjDev<float>&, cudaStream_t);
template void launch_adjoint_step<double>(const Dev<double>&, const AdjDev<double>&, cudaStream_t);
template void launch_adjoint_diag<float>(const Dev<float>&, const AdjDev<float>&, cudaStream_t);
template void launch_adjoint_diag<double>(const Dev<double>&, const AdjDev<double>&, cudaStream_t);
template void launch_adjoint_flags<float>(const Dev<float>&, int*, cudaStream_t);
template void launch_adjoint_flags<double>(const Dev<double>&, int*, cudaStream_t);

}  // namespace casim
