// Bounding-volume hierarchies of axis-aligned boxes (Sec. II-B: AABB trees
// over the robot and the obstacle, leaves of one element each; the tree is
// built once and only its boxes are refitted as the body deforms).
//
// Layout: n primitives (leaves) and n - 1 internal nodes, node 0 the root.
// child[i] = (left, right): a value >= 0 is an internal node, a value < 0 the
// leaf ~prim.  parent[i] for internal node i and parent[n - 1 + p] for leaf p
// (-1 at the root).  Internal boxes are floats rounded outward from the
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

__device__ __forceinline__ bool box_has(const float4& lo, const float4& hi, double x, double y, double z) {
  return x >= (double)lo.x && x <= (double)hi.x && y >= (double)lo.y && y <= (double)hi.y && z >= (double)lo.z &&
         z <= (double)hi.z;
}

// Squared distance from a point to a box (0 inside), in FP64.
__device__ __forceinline__ double box_d2(const float4& lo, const float4& hi, double x, double y, double z) {
  const double dx = fmax(fmax((double)lo.x - x, x - (double)hi.x), 0.0);
  const double dy = fmax(fmax((double)lo.y - y, y - (double)hi.y), 0.0);
  const double dz = fmax(fmax((double)lo.z - z, z - (double)hi.z), 0.0);
  return dx * dx + dy * dy + dz * dz;
}

// Entry parameter of the ray o + t d (t >= 0) into a box, widened by a
// relative margin so that rounding cannot drop a box the ray touches;
// +inf when the ray misses it.
__device__ __forceinline__ double ray_box_t(const float4& lo, const float4& hi, const double (&o)[3],
                                            const double (&inv)[3]) {
  const double l[3] = {(double)lo.x, (double)lo.y, (double)lo.z};
  const double h[3] = {(double)hi.x, (double)hi.y, (double)hi.z};
  double t0 = 0.0, t1 = INFINITY;
  for (int a = 0; a < 3; ++a) {
    const double m = 1e-7 * (fabs(l[a]) + fabs(h[a]) + (h[a] - l[a])) + 1e-30;
    const double lo_a = l[a] - m, hi_a = h[a] + m;
    if (isinf(inv[a])) {
      if (o[a] < lo_a || o[a] > hi_a) return INFINITY;
      continue;
    }
    double ta = (lo_a - o[a]) * inv[a], tb = (hi_a - o[a]) * inv[a];
    if (ta > tb) {
      const double s = ta;
      ta = tb;
      tb = s;
    }
    t0 = fmax(t0, ta);
    t1 = fmin(t1, tb);
  }
  return t0 <= t1 ? t0 : INFINITY;
}

static constexpr int BVH_STACK = 64;

// Calls leaf(p) for every primitive whose ancestors' boxes all contain
// (x, y, z) (the leaf's own box is left to the caller's exact test).
template <typename Leaf>
__device__ __forceinline__ void bvh_point_query(const BvhDev& b, double x, double y, double z, Leaf leaf) {
  if (b.n <= 0) return;
  if (b.n == 1) {
    leaf(0);
    return;
  }
  int stack[BVH_STACK];
  int sp = 0;
  if (!box_has(b.lo[0], b.hi[0], x, y, z)) return;
  stack[sp++] = 0;
  while (sp > 0) {
    const int node = stack[--sp];
    const int2 c = b.child[node];
    const int cs[2] = {c.x, c.y};
    for (int k = 0; k < 2; ++k) {
      const int ch = cs[k];
      if (ch < 0) {
        leaf(~ch);
      } else if (box_has(b.lo[ch], b.hi[ch], x, y, z) && sp < BVH_STACK) {
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
__device__ __forceinline__ void bvh_nearest(const BvhDev& b, double x, double y, double z, Leaf leaf, Bound bound) {
  if (b.n <= 0) return;
  if (b.n == 1) {
    leaf(0);
    return;
  }
  int stack[BVH_STACK];
  int sp = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    const int node = stack[--sp];
    if (box_d2(b.lo[node], b.hi[node], x, y, z) > bound()) continue;
    const int2 c = b.child[node];
    // visit the nearer child first (pushed last)
    const int cs[2] = {c.x, c.y};
    double dc[2];
    for (int k = 0; k < 2; ++k) dc[k] = cs[k] < 0 ? 0.0 : box_d2(b.lo[cs[k]], b.hi[cs[k]], x, y, z);
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
__device__ __forceinline__ void bvh_ray(const BvhDev& b, const double (&o)[3], const double (&dir)[3], Leaf leaf,
                                        Best tbest) {
  if (b.n <= 0) return;
  if (b.n == 1) {
    leaf(0);
    return;
  }
  double inv[3];
  for (int a = 0; a < 3; ++a) inv[a] = dir[a] != 0.0 ? 1.0 / dir[a] : INFINITY;
  int stack[BVH_STACK];
  int sp = 0;
  if (ray_box_t(b.lo[0], b.hi[0], o, inv) == INFINITY) return;
  stack[sp++] = 0;
  while (sp > 0) {
    const int node = stack[--sp];
    const int2 c = b.child[node];
    const int cs[2] = {c.x, c.y};
    for (int k = 0; k < 2; ++k) {
      const int ch = cs[k];
      if (ch < 0) {
        leaf(~ch);
      } else {
        const double te = ray_box_t(b.lo[ch], b.hi[ch], o, inv);
        if (te < INFINITY && te <= tbest() * (1.0 + 1e-9) + 1e-12 && sp < BVH_STACK) stack[sp++] = ch;
      }
    }
  }
}

}  // namespace casim
