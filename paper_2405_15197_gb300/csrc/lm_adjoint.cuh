// Adjoint of the triangulated area and enclosed volume (no counterpart in
// the paper, which has no gradients): d(w_area area + w_vol volume) / d(node
// position, node radius) of the mesh of Section 5 at resolution k, with the
// discrete structure held fixed (vertex generators, arcs, loops, holes,
// segment counts, stitching order, fan-centre rule).
//
// Two stages.
//  1. Point adjoints.  Every triangle adds, for each of its corners p,
//       w_area * dA/dp + w_vol * dV/dp,
//     dA/dp_a = 1/2 (p_b - p_c) x n^ (and cyclically) for A = |n|/2,
//     n = (p_b - p_a) x (p_c - p_a); and, because the mesh is closed, the
//     divergence-theorem volume has dV/dp = (sum over the triangles around p
//     of n)/6, so each triangle adds n/6 to each corner (local, free of the
//     cancellation of the per-triangle form (p_b x p_c)/6).  Corners are
//     identified by point ids: a meta-mesh vertex, an interior subdivision
//     point of an arc, or a hole's fan centre.
//  2. Parameter adjoints, one node at a time.  Every point of a node is a
//     function of the node's position and radius and of the positions and
//     radii of its neighbours (the strut ends of the node).  The node's
//     geometry is recomputed in forward-mode dual numbers seeded with W of
//     those 4 + 4d parameters at a time, and each point's tangents are
//     contracted with its adjoint.  Nothing per node is stored between the
//     forward pass and this one.
#pragma once
#include "lm_geom.cuh"

namespace lm {

// value + W tangents (forward mode)
template <int W>
struct Dual {
  float v;
  float t[W];
  __device__ Dual() : v(0.0f) {
#pragma unroll
    for (int i = 0; i < W; i++) t[i] = 0.0f;
  }
  __device__ Dual(float x) : v(x) {
#pragma unroll
    for (int i = 0; i < W; i++) t[i] = 0.0f;
  }
  __device__ Dual(int x) : Dual((float)x) {}
  __device__ Dual(bool x) : Dual(x ? 1.0f : 0.0f) {}
  __device__ explicit Dual(double x) : Dual((float)x) {}
  __device__ explicit operator float() const { return v; }
};

template <int W>
__device__ __forceinline__ Dual<W> operator+(const Dual<W>& a, const Dual<W>& b) {
  Dual<W> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.t[i] + b.t[i];
  return r;
}
template <int W>
__device__ __forceinline__ Dual<W> operator-(const Dual<W>& a, const Dual<W>& b) {
  Dual<W> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.t[i] - b.t[i];
  return r;
}
template <int W>
__device__ __forceinline__ Dual<W> operator-(const Dual<W>& a) {
  Dual<W> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = -a.t[i];
  return r;
}
template <int W>
__device__ __forceinline__ Dual<W> operator*(const Dual<W>& a, const Dual<W>& b) {
  Dual<W> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.v * b.t[i] + b.v * a.t[i];
  return r;
}
template <int W>
__device__ __forceinline__ Dual<W> operator/(const Dual<W>& a, const Dual<W>& b) {
  Dual<W> r;
  float ib = 1.0f / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = (a.t[i] - r.v * b.t[i]) * ib;
  return r;
}
template <int W>
__device__ __forceinline__ bool operator<(const Dual<W>& a, const Dual<W>& b) { return a.v < b.v; }
template <int W>
__device__ __forceinline__ bool operator>(const Dual<W>& a, const Dual<W>& b) { return a.v > b.v; }
template <int W>
__device__ __forceinline__ bool operator<=(const Dual<W>& a, const Dual<W>& b) { return a.v <= b.v; }
template <int W>
__device__ __forceinline__ bool operator>=(const Dual<W>& a, const Dual<W>& b) { return a.v >= b.v; }

template <int W>
__device__ __forceinline__ Dual<W> lm_sqrt(const Dual<W>& a) {
  Dual<W> r;
  r.v = a.v > 0.0f ? sqrtf(a.v) : 0.0f;
  float h = r.v > 0.0f ? 0.5f / r.v : 0.0f;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.t[i] * h;
  return r;
}
template <int W>
__device__ __forceinline__ Dual<W> lm_atan2(const Dual<W>& y, const Dual<W>& x) {
  Dual<W> r;
  r.v = atan2f(y.v, x.v);
  float ir = 1.0f / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = (x.v * y.t[i] - y.v * x.t[i]) * ir;
  return r;
}
template <int W>
__device__ __forceinline__ void lm_sincos(const Dual<W>& a, Dual<W>* s, Dual<W>* c) {
  float sv, cv;
  sincosf(a.v, &sv, &cv);
  s->v = sv;
  c->v = cv;
#pragma unroll
  for (int i = 0; i < W; i++) {
    s->t[i] = cv * a.t[i];
    c->t[i] = -sv * a.t[i];
  }
}

// a constant shifted by a value-only offset (continuous angle tracking)
template <int W>
__device__ __forceinline__ Dual<W> shift(const Dual<W>& a, float d) {
  Dual<W> r = a;
  r.v += d;
  return r;
}

// Strut end `end_id` of node `node` as a function of seeded inputs: the
// node's centre c and radius R, the far node's centre cf and radius Rf (the
// same arithmetic as make_end; the frame axis is a discrete choice, taken on
// the input values).
template <typename T, typename U>
__device__ EndG<U> end_from(const LatDev<T>& L, int64_t node, int32_t end_id, V3<U> c, U R, V3<U> cf, U Rf) {
  EndG<U> e;
  int32_t strut = end_id >> 1;
  int32_t a = L.ends[2 * (int64_t)strut], b = L.ends[2 * (int64_t)strut + 1];
  e.end_id = end_id;
  e.far = (end_id & 1) ? a : b;
  int32_t lo = a < b ? a : b, hi = a < b ? b : a;
  e.at_lo = (node == lo);
  V3<U> d = e.at_lo ? cf - c : c - cf;
  e.L = norm3(d);
  U il = U(1) / e.L;
  V3<U> ue = d * il;
  e.u = e.at_lo ? ue : ue * U(-1);
  e.s = (R - Rf) * il;
  e.co = lm_sqrt(U(1) - e.s * e.s);
  e.ico = U(1) / e.co;
  int ax = frame_axis(L, lo, hi);
  V3<U> Ex = mk3<U>(U(ax == 0), U(ax == 1), U(ax == 2));
  V3<U> c1 = cross(ue, Ex);
  e.e1 = c1 * (U(1) / norm3(c1));
  e.e2 = cross(ue, e.e1);
  return e;
}

}  // namespace lm
