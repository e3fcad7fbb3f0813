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
#include <type_traits>

#include "lm_geom.cuh"

namespace lm {

// scalar helpers: the FP32 path calls the single-precision functions, the
// FP64 path the double ones
__device__ __forceinline__ float sc_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double sc_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ void sc_sincos(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sc_sincos(double a, double* s, double* c) { sincos(a, s, c); }
__device__ __forceinline__ float sc_rem2pi(float a) { return remainderf(a, (float)PI2); }
__device__ __forceinline__ double sc_rem2pi(double a) { return remainder(a, PI2); }

// value + W tangents (forward mode) in scalar S (the lattice's precision)
template <int W, typename S = float>
struct Dual {
  S v;
  S t[W];
  __device__ Dual() : v(S(0)) {
#pragma unroll
    for (int i = 0; i < W; i++) t[i] = S(0);
  }
  __device__ Dual(S x) : v(x) {
#pragma unroll
    for (int i = 0; i < W; i++) t[i] = S(0);
  }
  __device__ Dual(int x) : Dual((S)x) {}
  __device__ Dual(bool x) : Dual(x ? S(1) : S(0)) {}
  template <typename X, typename = typename std::enable_if<std::is_floating_point<X>::value &&
                                                           !std::is_same<X, S>::value>::type>
  __device__ explicit Dual(X x) : Dual((S)x) {}
  __device__ explicit operator S() const { return v; }
};

template <int W, typename S>
__device__ __forceinline__ Dual<W, S> operator+(const Dual<W, S>& a, const Dual<W, S>& b) {
  Dual<W, S> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.t[i] + b.t[i];
  return r;
}
template <int W, typename S>
__device__ __forceinline__ Dual<W, S> operator-(const Dual<W, S>& a, const Dual<W, S>& b) {
  Dual<W, S> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.t[i] - b.t[i];
  return r;
}
template <int W, typename S>
__device__ __forceinline__ Dual<W, S> operator-(const Dual<W, S>& a) {
  Dual<W, S> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = -a.t[i];
  return r;
}
template <int W, typename S>
__device__ __forceinline__ Dual<W, S> operator*(const Dual<W, S>& a, const Dual<W, S>& b) {
  Dual<W, S> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.v * b.t[i] + b.v * a.t[i];
  return r;
}
template <int W, typename S>
__device__ __forceinline__ Dual<W, S> operator/(const Dual<W, S>& a, const Dual<W, S>& b) {
  Dual<W, S> r;
  S ib = S(1) / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = (a.t[i] - r.v * b.t[i]) * ib;
  return r;
}
template <int W, typename S>
__device__ __forceinline__ bool operator<(const Dual<W, S>& a, const Dual<W, S>& b) { return a.v < b.v; }
template <int W, typename S>
__device__ __forceinline__ bool operator>(const Dual<W, S>& a, const Dual<W, S>& b) { return a.v > b.v; }
template <int W, typename S>
__device__ __forceinline__ bool operator<=(const Dual<W, S>& a, const Dual<W, S>& b) { return a.v <= b.v; }
template <int W, typename S>
__device__ __forceinline__ bool operator>=(const Dual<W, S>& a, const Dual<W, S>& b) { return a.v >= b.v; }

template <int W, typename S>
__device__ __forceinline__ Dual<W, S> lm_sqrt(const Dual<W, S>& a) {
  Dual<W, S> r;
  r.v = a.v > S(0) ? lm_sqrt(a.v) : S(0);
  S h = r.v > S(0) ? S(0.5) / r.v : S(0);
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = a.t[i] * h;
  return r;
}
template <int W, typename S>
__device__ __forceinline__ Dual<W, S> lm_atan2(const Dual<W, S>& y, const Dual<W, S>& x) {
  Dual<W, S> r;
  r.v = sc_atan2(y.v, x.v);
  S ir = S(1) / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int i = 0; i < W; i++) r.t[i] = (x.v * y.t[i] - y.v * x.t[i]) * ir;
  return r;
}
template <int W, typename S>
__device__ __forceinline__ void lm_sincos(const Dual<W, S>& a, Dual<W, S>* s, Dual<W, S>* c) {
  S sv, cv;
  sc_sincos(a.v, &sv, &cv);
  s->v = sv;
  c->v = cv;
#pragma unroll
  for (int i = 0; i < W; i++) {
    s->t[i] = cv * a.t[i];
    c->t[i] = -sv * a.t[i];
  }
}

// a constant shifted by a value-only offset (continuous angle tracking)
template <int W, typename S>
__device__ __forceinline__ Dual<W, S> shift(const Dual<W, S>& a, S d) {
  Dual<W, S> r = a;
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
