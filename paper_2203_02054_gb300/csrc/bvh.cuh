// Bounding-volume hierarchies of axis-aligned boxes (Sec. II-B: AABB trees
// over the robot and the obstacle, leaves of one element each; the tree is
// built once and only its boxes are refitted as the body deforms).
//
// Layout: n primitives (leaves) in one tree per robot (a forest), n - R
// internal nodes for R robots with primitives; root[r] is robot r's root code
// (node 0 for a single robot).  child[i] = (left, right): a value >= 0 is an
// internal node, a value < 0 the leaf ~prim.  parent[i] for internal node i
// and parent[n - 1 + p] for leaf p (-1 at a root).  Internal boxes are floats rounded outward from the
// positions (exact for FP32 positions), so every query below is conservative
// and the exact tests at the leaves decide.
#pragma once

#include "common.cuh"

namespace casim {

__device__ __forceinline__ float f_lo(float x) { return x; }
__device__ __forceinline__ float f_hi(float x) { return x; }
__device__ __forceinline__ float f_lo(double x) { return __double2float_rd(x); }
__device__ __forceinline__ float f_hi(double x) { return __double2float_ru(x); }

// Box of primitive p from positions X, rounded outward to float.
template <typename T>
__device__ __forceinline__ void prim_box(const BvhDev& b, const R4<T>* X, int p, float4& lo, float4& hi) {
  const int4 q = b.prim[p];
  const int vs[4] = {q.x, q.y, q.z, q.w};
  const R4<T> a0 = X[vs[0]];
  T l[3] = {a0.x, a0.y, a0.z}, h[3] = {a0.x, a0.y, a0.z};
  for (int k = 1; k < b.nv; ++k) {
    const R4<T> a = X[vs[k]];
    l[0] = fmin(l[0], a.x);
    l[1] = fmin(l[1], a.y);
    l[2] = fmin(l[2], a.z);
    h[0] = fmax(h[0], a.x);
    h[1] = fmax(h[1], a.y);
    h[2] = fmax(h[2], a.z);
  }
  lo = make_float4(f_lo(l[0]), f_lo(l[1]), f_lo(l[2]), 0.0f);
  hi = make_float4(f_hi(h[0]), f_hi(h[1]), f_hi(h[2]), 0.0f);
}

// Box tests run in FP32 (FP64 arithmetic is scarce on this part) and are
// conservative: a query point is carried as the FP32 interval [lo, hi] that
// contains it, and every distance or ray parameter is rounded toward
// accepting the box; only the exact tests at the leaves decide.
struct PtF {
  float lx, ly, lz, hx, hy, hz;
};
__device__ __forceinline__ PtF pt_f(double x, double y, double z) {
  return {__double2float_rd(x), __double2float_rd(y), __double2float_rd(z),
          __double2float_ru(x), __double2float_ru(y), __double2float_ru(z)};
}

__device__ __forceinline__ bool box_has(const float4& lo, const float4& hi, const PtF& p) {
  return p.hx >= lo.x && p.lx <= hi.x && p.hy >= lo.y && p.ly <= hi.y && p.hz >= lo.z && p.lz <= hi.z;
}

// A lower bound of the squared distance from the point to the box (0 when
// they touch), rounded down.
__device__ __forceinline__ float box_d2(const float4& lo, const float4& hi, const PtF& p) {
  const float dx = fmaxf(fmaxf(__fsub_rd(lo.x, p.hx), __fsub_rd(p.lx, hi.x)), 0.0f);
  const float dy = fmaxf(fmaxf(__fsub_rd(lo.y, p.hy), __fsub_rd(p.ly, hi.y)), 0.0f);
  const float dz = fmaxf(fmaxf(__fsub_rd(lo.z, p.hz), __fsub_rd(p.lz, hi.z)), 0.0f);
  return __fadd_rd(__fadd_rd(__fmul_rd(dx, dx), __fmul_rd(dy, dy)), __fmul_rd(dz, dz));
}

// Ray in FP32 for box tests: origin interval and reciprocal direction.
struct RayF {
  PtF o;
  float inv[3];
};

// A lower bound of the ray parameter at which the ray o + t d (t >= 0)
// enters the box, widened by a relative margin so that rounding cannot drop
// a box the ray touches; +inf when the ray misses it.
__device__ __forceinline__ float ray_box_t(const float4& lo, const float4& hi, const RayF& r) {
  const float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
  const float ol[3] = {r.o.lx, r.o.ly, r.o.lz}, oh[3] = {r.o.hx, r.o.hy, r.o.hz};
  float t0 = 0.0f, t1 = INFINITY;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float m = 1e-5f * (fabsf(l[a]) + fabsf(h[a]) + (h[a] - l[a])) + 1e-30f;
    const float lo_a = l[a] - m, hi_a = h[a] + m;
    if (isinf(r.inv[a])) {
      if (oh[a] < lo_a || ol[a] > hi_a) return INFINITY;
      continue;
    }
    // entry and exit over the origin interval, widened
    float ta, tb;
    if (r.inv[a] > 0.0f) {
      ta = (lo_a - oh[a]) * r.inv[a];
      tb = (hi_a - ol[a]) * r.inv[a];
    } else {
      ta = (hi_a - ol[a]) * r.inv[a];
      tb = (lo_a - oh[a]) * r.inv[a];
    }
    t0 = fmaxf(t0, ta * (ta > 0.0f ? 0.9999f : 1.0001f));
    t1 = fminf(t1, tb * (tb > 0.0f ? 1.0001f : 0.9999f));
  }
  return t0 <= t1 ? t0 : INFINITY;
}

static constexpr int BVH_STACK = 64;
static constexpr int BVH_EMPTY = (-2147483647 - 1);  // root code of a robot without primitives

// Calls leaf(p) for every primitive whose ancestors' boxes all contain
// (x, y, z) (the leaf's own box is left to the caller's exact test).
template <typename Leaf>
__device__ __forceinline__ void bvh_point_query(const BvhDev& b, int tree, double x, double y, double z, Leaf leaf) {
  if (b.n <= 0) return;
  const int root = b.root ? b.root[tree] : 0;
  if (root == BVH_EMPTY) return;
  if (root < 0) {
    leaf(~root);
    return;
  }
  const PtF pf = pt_f(x, y, z);
  int stack[BVH_STACK];
  int sp = 0;
  if (!box_has(b.lo[root], b.hi[root], pf)) return;
  stack[sp++] = root;
  while (sp > 0) {
    const int node = stack[--sp];
    const int2 c = b.child[node];
    const int cs[2] = {c.x, c.y};
    for (int k = 0; k < 2; ++k) {
      const int ch = cs[k];
      if (ch < 0) {
        leaf(~ch);
      } else if (box_has(b.lo[ch], b.hi[ch], pf) && sp < BVH_STACK) {
        stack[sp++] = ch;
      }
    }
  }
}

// Nearest primitive: leaf(p) returns the primitive's squared distance (or a
// negative value to skip it) and records it; bound() gives the best squared
// distance so far.  A subtree is skipped only when its box is strictly
// farther than the best, so equal distances still reach every candidate and
// the caller's tie rule decides.
template <typename Leaf, typename Bound>
__device__ __forceinline__ void bvh_nearest(const BvhDev& b, int tree, double x, double y, double z, Leaf leaf,
                                            Bound bound) {
  if (b.n <= 0) return;
  const int root = b.root ? b.root[tree] : 0;
  if (root == BVH_EMPTY) return;
  if (root < 0) {
    leaf(~root);
    return;
  }
  const PtF pf = pt_f(x, y, z);
  int stack[BVH_STACK];
  int sp = 0;
  stack[sp++] = root;
  while (sp > 0) {
    const int node = stack[--sp];
    if ((double)box_d2(b.lo[node], b.hi[node], pf) > bound()) continue;
    const int2 c = b.child[node];
    // visit the nearer child first (pushed last)
    const int cs[2] = {c.x, c.y};
    double dc[2];
    for (int k = 0; k < 2; ++k) dc[k] = cs[k] < 0 ? 0.0 : (double)box_d2(b.lo[cs[k]], b.hi[cs[k]], pf);
    const int first = dc[1] < dc[0] ? 1 : 0;
    for (int j = 0; j < 2; ++j) {
      const int k = j == 0 ? 1 - first : first;
      const int ch = cs[k];
      if (ch < 0) {
        leaf(~ch);
      } else if (dc[k] <= bound() && sp < BVH_STACK) {
        stack[sp++] = ch;
      }
    }
  }
}

// First hit along a ray: leaf(p) tests primitive p and records a hit; tbest()
// gives the best ray parameter so far (+inf before any hit).  Boxes entered
// beyond the best hit (with a relative margin) are skipped.
template <typename Leaf, typename Best>
__device__ __forceinline__ void bvh_ray(const BvhDev& b, int tree, const double (&o)[3], const double (&dir)[3],
                                        Leaf leaf, Best tbest) {
  if (b.n <= 0) return;
  const int root = b.root ? b.root[tree] : 0;
  if (root == BVH_EMPTY) return;
  if (root < 0) {
    leaf(~root);
    return;
  }
  RayF r;
  r.o = pt_f(o[0], o[1], o[2]);
  for (int a = 0; a < 3; ++a) {
    const float df = (float)dir[a];
    r.inv[a] = df != 0.0f ? 1.0f / df : INFINITY;
  }
  int stack[BVH_STACK];
  float node_t[BVH_STACK];  // entry parameter of each stacked node
  int sp = 0;
  const float t_root = ray_box_t(b.lo[root], b.hi[root], r);
  if (t_root == INFINITY) return;
  node_t[sp] = t_root;
  stack[sp++] = root;
  while (sp > 0) {
    const int node = stack[--sp];
    if ((double)node_t[sp] > tbest() * (1.0 + 1e-6) + 1e-9) continue;  // a nearer hit was found meanwhile
    const int2 c = b.child[node];
    const int cs[2] = {c.x, c.y};
    float te[2];
    for (int k = 0; k < 2; ++k) {
      if (cs[k] < 0) {
        leaf(~cs[k]);
        te[k] = INFINITY;
      } else {
        te[k] = ray_box_t(b.lo[cs[k]], b.hi[cs[k]], r);
      }
    }
    // push the farther child first, so the nearer one is visited next
    const int nearer = te[1] < te[0] ? 1 : 0;
    for (int j = 0; j < 2; ++j) {
      const int k = j == 0 ? 1 - nearer : nearer;
      if (cs[k] >= 0 && te[k] < INFINITY && (double)te[k] <= tbest() * (1.0 + 1e-6) + 1e-9 && sp < BVH_STACK) {
        node_t[sp] = te[k];
        stack[sp++] = cs[k];
      }
    }
  }
}

}  // namespace casim
