// Strut / plane / arc geometry of the lattice meta-mesh, templated on the
// arithmetic type U (float for the bulk, double for stability steps).
//
// Paper: arXiv 2405.15197.  Section 4.1 (struts tangent to nodal spheres),
// Section 4.3.1 (auxiliary planes P_ij from the planar-conic property,
// strut-plane ellipses, ellipse-plane trimming Eq. arc-range /
// overlap-vertices), Section 5 (subdivision Eq. sampling / parameter-range,
// hole filling).
//
// Notation at a node with centre c and radius R, for an incident strut end:
//   u   outward unit axis, L strut length, s = (R - R_far)/L = sin(alpha),
//   co  = cos(alpha), ico = 1/co;
//   frame e1, e2 built from the strut's lo->hi axis (lo = lower node id), so
//   both ends of a strut share the angle phi;
//   rho(phi) = cos(phi) e1 + sin(phi) e2,
//   w(phi) = s u + co rho(phi)  (sphere normal on the tangency circle),
//   g(phi) = co u - s rho(phi)  (generator direction),
//   surface point c + R w(phi) + t g(phi), t >= 0 (generator coordinate);
//   generator coordinate of any point z (relative to c): G(z) = (u.z - R s)/co.
// The surfaces of two struts meeting at the node intersect (near the node) on
// the plane P_ij : G_i(z) = G_j(z); a point of strut i's surface is inside
// strut l iff G_l(z) > G_i(z).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lm_df.cuh"

namespace lm {

constexpr double PI2 = 6.283185307179586476925286766559;

// Decision thresholds (readings of ties the paper is silent on).
constexpr double ETA_SIGMA = 1e-9;  // x R: a strut passes through a vertex
constexpr double ETA_DEDUP = 1e-3;  // x R: candidates with one key are one vertex
constexpr double ETA_PHI = 1e-9;    // rad: angle ties; relative angles wrap to [-ETA_PHI, 2pi - ETA_PHI)
constexpr double PHI_CUT = 0.0009765625;  // rad (2^-10): absolute angles in [-PHI_CUT, 2pi - PHI_CUT)
constexpr double ETA_ZIP = 0.015625;  // rad (2^-6): stitching tie band
constexpr double TAU_COUNT = 0.0009765625;  // segment count offset (2^-10)
constexpr double ETA_BARY = 1e-4;   // x R: hole barycentre at the centre
constexpr double EPS_PAR = 1e-6;    // 1 - c^2 below this: (anti)parallel pair
constexpr double EPS_TAN = 1e-6;    // tangency measure: node exempt from exact parity

// FP32 safety margins: an FP32 quantity closer than this to a decision
// threshold, or computed from an ill-conditioned configuration, is decided
// again in FP64 from the inputs.
constexpr float M_LEN = 1e-4f;   // x R (FP32 candidate error <= ~1e-5 R once conditioned)
constexpr float M_ANG = 1e-5f;   // rad (loop angles of the meta-mesh)
constexpr float M_ZIP = 2e-5f;   // rad (stitching order, about ETA_ZIP; FP32 angle error <= ~2e-6)
constexpr float M_COND = 1e-2f;  // conditioning floor of q, |v|^2, |A|, D/R^2, g2
constexpr float M_CNT = 2e-5f;   // rad: arc extent, for the segment count (x k / 2pi)
constexpr float M_POS = 1e-1f;   // conditioning floor for keeping an FP32 circle-point position
// A triple point keeps its FP32 position when its first-order sensitivity to
// unit-roundoff perturbations of the strut axes (the dominant FP32 error: the
// line P_ij n P_ik moves with the plane normals and meets the cone at an
// angle) stays below M_SENS R per unit roundoff, i.e. about 3e-6 R.
constexpr float M_SENS = 50.0f;
// An elliptical arc whose points t(phi) = (n0 + n1 c + n2 s) / (d0 + d1 c +
// d2 s) come close to the pole of that ratio is subdivided in FP64 from the
// inputs.  The strut kernels form n0 and d0 without cancellation (1 - u_i.u_j
// as |u_i - u_j|^2 / 2, co_j - co_i as a product over a sum), so every
// coefficient is accurate relative to its own size; what is left is the
// sensitivity of t near the pole, about 3e-7 (R + |t|) (1 + |N| / R) / |D|.
// Arcs on which |D| drops below D_ILL are taken in FP64: above it the FP32
// points measured within 3.3e-6 (|z| + R) over 370,000 arcs of three
// irregular lattices (radii at 0.3 and 0.06 of the mean strut length), 98.5 %
// of them above the floor (below 1e-3 the error reaches 1e-2).  Regular
// lattices stay far above it (BCC 2/3, octet 1/2).
constexpr float D_ILL = 0.0078125f;

// node flags (same bits as LM_NODE_* in liblm.h)
constexpr uint32_t NF_NEAR_TANGENT = 1u, NF_DEGENERATE = 2u, NF_INCONSISTENT = 4u,
                   NF_BEYOND = 8u, NF_STEEP = 16u, NF_SEAM_CUT = 32u, NF_ANGLE_TIE = 64u,
                   NF_ALONG = 128u, NF_OVERFLOW = 256u;
constexpr uint32_t VF_SPHERE = 1u, VF_SEAM = 2u;

template <typename U>
struct V3 {
  U x, y, z;
};
template <typename U>
__host__ __device__ __forceinline__ V3<U> mk3(U x, U y, U z) {
  return V3<U>{x, y, z};
}
template <typename U>
__device__ __forceinline__ V3<U> operator+(V3<U> a, V3<U> b) {
  return mk3(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <typename U>
__device__ __forceinline__ V3<U> operator-(V3<U> a, V3<U> b) {
  return mk3(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <typename U>
__device__ __forceinline__ V3<U> operator*(V3<U> a, U s) {
  return mk3(a.x * s, a.y * s, a.z * s);
}
template <typename U>
__device__ __forceinline__ U dot(V3<U> a, V3<U> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename U>
__device__ __forceinline__ V3<U> cross(V3<U> a, V3<U> b) {
  return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <typename U, typename S>
__device__ __forceinline__ V3<U> cvt3(V3<S> a) {
  return mk3((U)a.x, (U)a.y, (U)a.z);
}
__device__ __forceinline__ float lm_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double lm_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ df lm_sqrt(df x) { return df_sqrt(x); }
__device__ __forceinline__ float lm_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double lm_rsqrt(double x) { return 1.0 / sqrt(x); }
// FP32 atan2 from atan(r) ~ r P(r^2) on r = min/max in [0, 1] (P of degree 7
// in r^2; minimax coefficients from Lawson's iteratively reweighted least
// squares, rounded to FP32: paper_2405_15197_gb300/fit_atan.py reproduces
// them; FP32 Horner evaluation error at most 1.23e-7 rad on [0, 1]) and the
// octant identities (each adds at most 1.5e-7 rad: the FP32 constants pi/2
// and pi and one rounding).  Every FP32 angle decision has a margin of at
// least 1e-5 rad.
__device__ __forceinline__ float lm_atan2(float y, float x) {
  float ax = fabsf(x), ay = fabsf(y);
  float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  if (mx == 0.0f) return 0.0f;
  float r = mn / mx, t = r * r;
  float p = -0.004054488614201546f;
  p = fmaf(p, t, 0.021862687543034554f);
  p = fmaf(p, t, -0.05591195821762085f);
  p = fmaf(p, t, 0.09642171859741211f);
  p = fmaf(p, t, -0.13908620178699493f);
  p = fmaf(p, t, 0.19946563243865967f);
  p = fmaf(p, t, -0.33329859375953674f);
  p = fmaf(p, t, 0.9999993443489075f);
  float a = r * p;
  if (ay > ax) a = 1.5707963267948966f - a;
  if (x < 0.0f) a = 3.1415926535897932f - a;
  return y < 0.0f ? -a : a;
}
__device__ __forceinline__ double lm_atan2(double y, double x) { return atan2(y, x); }
// FP32 sin/cos: reduction by the nearest multiple of 2 pi in two parts
// (Cody and Waite's split: 6.28125, exact in a few bits, then the rest of
// 2 pi), then the hardware approximation on [-pi, pi] (absolute error about
// 2^-21.4).  Arguments stay within a few turns; with the rounding of the
// reduced argument the absolute error stays below 7e-7 (tested against FP64
// sine and cosine).
__device__ __forceinline__ void lm_sincos(float a, float* s, float* c) {
  float k = rintf(a * 0.15915494309189535f);
  float r = fmaf(-k, 6.28125f, a);
  r = fmaf(-k, 0.0019353071795864769f, r);
  __sincosf(r, s, c);
}
__device__ __forceinline__ void lm_sincos(double a, double* s, double* c) { sincos(a, s, c); }
template <typename U>
__device__ __forceinline__ U norm3(V3<U> a) {
  return lm_sqrt(dot(a, a));
}

// Lattice inputs on the device (dtype T of the caller's arrays).
template <typename T>
struct LatDev {
  const T* xyz;          // [N][3]
  const int32_t* ends;   // [E][2]
  const T* node_R;       // [N] (derived from the per-end radii)
  const int64_t* row_ptr;
  const int32_t* adj;
  int64_t n_nodes, n_struts;
};

template <typename T, typename U>
__device__ __forceinline__ V3<U> node_xyz(const LatDev<T>& L, int64_t n) {
  return mk3((U)L.xyz[3 * n], (U)L.xyz[3 * n + 1], (U)L.xyz[3 * n + 2]);
}

// One strut end as seen from its node.
template <typename U>
struct EndG {
  V3<U> u, e1, e2;
  U s, co, ico, L;
  int32_t end_id, far;
  int32_t at_lo;
};

// Frame axis: the coordinate axis of smallest |x_hi - x_lo| (ties -> lowest),
// decided on the exact differences of the inputs.  For FP32 inputs the
// difference a - b is held exactly as s + e (error-free 2Sum); for FP64 the
// computed difference is the one the FP64 reference uses.
struct ExactDiff {
  float s, e;
};
__device__ __forceinline__ ExactDiff exact_abs_diff(float a, float b) {
  float s = a - b;
  float bb = s - a;
  float e = (a - (s - bb)) + (-b - bb);
  if (s < 0.0f || (s == 0.0f && e < 0.0f)) {
    s = -s;
    e = -e;
  }
  return ExactDiff{s, e};
}
__device__ __forceinline__ bool exact_less(ExactDiff x, ExactDiff y) {
  return x.s < y.s || (x.s == y.s && x.e < y.e);
}
template <typename T>
__device__ __forceinline__ int frame_axis(const LatDev<T>& L, int32_t lo, int32_t hi) {
  if constexpr (sizeof(T) == 4) {
    ExactDiff d0 = exact_abs_diff((float)L.xyz[3 * hi], (float)L.xyz[3 * lo]);
    ExactDiff d1 = exact_abs_diff((float)L.xyz[3 * hi + 1], (float)L.xyz[3 * lo + 1]);
    ExactDiff d2 = exact_abs_diff((float)L.xyz[3 * hi + 2], (float)L.xyz[3 * lo + 2]);
    int ax = 0;
    ExactDiff best = d0;
    if (exact_less(d1, best)) { ax = 1; best = d1; }
    if (exact_less(d2, best)) ax = 2;
    return ax;
  } else {
    double d0 = fabs((double)L.xyz[3 * hi] - (double)L.xyz[3 * lo]);
    double d1 = fabs((double)L.xyz[3 * hi + 1] - (double)L.xyz[3 * lo + 1]);
    double d2 = fabs((double)L.xyz[3 * hi + 2] - (double)L.xyz[3 * lo + 2]);
    int ax = 0;
    double best = d0;
    if (d1 < best) { ax = 1; best = d1; }
    if (d2 < best) ax = 2;
    return ax;
  }
}

// Strut end `end_id` at node `node` (Section 4.3.1: strut S_i with ends
// v_i^0, v_i^1 and radii r_i^0, r_i^1; the cone half-angle is read as
// alpha = asin((R_node - R_far)/L)).
template <typename T, typename U>
__device__ EndG<U> make_end(const LatDev<T>& L, int64_t node, int32_t end_id) {
  EndG<U> e;
  int32_t strut = end_id >> 1;
  int32_t a = L.ends[2 * (int64_t)strut], b = L.ends[2 * (int64_t)strut + 1];
  e.end_id = end_id;
  e.far = (end_id & 1) ? a : b;
  int32_t lo = a < b ? a : b, hi = a < b ? b : a;
  e.at_lo = (node == lo);
  V3<U> d = node_xyz<T, U>(L, hi) - node_xyz<T, U>(L, lo);
  e.L = norm3(d);
  U il = U(1) / e.L;
  V3<U> ue = d * il;
  e.u = e.at_lo ? ue : ue * U(-1);
  U R = (U)L.node_R[node], Rf = (U)L.node_R[e.far];
  e.s = (R - Rf) * il;
  e.co = lm_sqrt(U(1) - e.s * e.s);
  e.ico = U(1) / e.co;
  int ax = frame_axis(L, lo, hi);
  V3<U> E = mk3<U>(ax == 0, ax == 1, ax == 2);
  V3<U> c1 = cross(ue, E);
  e.e1 = c1 * (U(1) / norm3(c1));
  e.e2 = cross(ue, e.e1);
  return e;
}

template <typename U>
__device__ __forceinline__ V3<U> rho_dir(const EndG<U>& e, U c, U s) {
  return e.e1 * c + e.e2 * s;
}

// h_j(phi) on strut end i: generator coordinate where the generator at phi
// crosses plane P_ij (the ellipse of Section 4.3.1 in i's angle).
template <typename U>
__device__ __forceinline__ U hval(const EndG<U>& i, const EndG<U>& j, U cph, U sph, U R) {
  V3<U> r = rho_dir(i, cph, sph);
  V3<U> w = i.u * i.s + r * i.co;
  V3<U> g = i.u * i.co - r * i.s;
  return R * (dot(j.u, w) - j.s) / (j.co - dot(j.u, g));
}

// node-relative surface point of strut end e at angle phi, generator coord t
template <typename U>
__device__ __forceinline__ V3<U> surf_point(const EndG<U>& e, U cph, U sph, U t, U R) {
  V3<U> r = rho_dir(e, cph, sph);
  V3<U> w = e.u * e.s + r * e.co;
  V3<U> g = e.u * e.co - r * e.s;
  return w * R + g * t;
}

// raw angle of a node-relative point around strut end e, in (-pi, pi]
template <typename U>
__device__ __forceinline__ U raw_angle(const EndG<U>& e, V3<U> z) {
  return lm_atan2(dot(z, e.e2), dot(z, e.e1));
}

// generator code: type (0 circle point, 1 triple point, 2 seam) | root << 2 |
// i << 3 | j << 9 | k << 15 (local strut-end indices)
__host__ __device__ __forceinline__ uint32_t gen_code(int type, int root, int i, int j, int k) {
  return (uint32_t)type | ((uint32_t)root << 2) | ((uint32_t)i << 3) | ((uint32_t)j << 9) |
         ((uint32_t)k << 15);
}

// Result of one generator (pair or triple of strut ends): up to two roots.
template <typename U>
struct GenOut {
  V3<U> z[2];
  U t0[2];
  uint64_t key[2];
  uint8_t sphere[2];
  uint8_t state[2];   // 0 rejected, 1 kept, 2 uncertain (decide in FP64)
  uint8_t tangent[2];
  uint8_t nroot;      // 0 or 2 (roots produced, before screening)
  uint8_t unc;        // whole generator uncertain in this precision
  uint8_t refine;     // decisions certain, but recompute positions in FP64
  uint32_t nflags;    // node flags raised independent of survival
  uint32_t kflags[2]; // node flags raised if the root is kept as a new vertex
  uint64_t umask[2];  // FP32: strut ends whose screening decision was uncertain
};

// What an FP32 evaluation already decided, for a higher-precision
// re-decision of the same generator: per root its FP32 state (0 rejected,
// 1 kept, 2 uncertain, 3 duplicate of a vertex found earlier) and the strut
// ends whose screening was uncertain.  Every other screening decision was
// certain (beyond its margin) and is not repeated.
struct GenHint {
  uint8_t st[2];
  uint64_t umask[2];
};

// Candidates of one generator with screening (trimming) against every strut
// end of the node.  F64 = true: all decisions exact (thresholds only).
// F64 = false: decisions within the FP32 margins are reported uncertain.
template <typename U, bool F64>
__device__ void eval_gen(const EndG<U>* E, int d, U R, uint32_t gcode, GenOut<U>& o,
                         const GenHint* hint = nullptr) {
  o.nroot = 0;
  o.unc = 0;
  o.refine = 0;
  o.nflags = 0;
  int type = gcode & 3, i = (gcode >> 3) & 63, j = (gcode >> 9) & 63, k = (gcode >> 15) & 63;
  uint64_t gmask;
  bool sph0;
  U tanq;
  bool well = true;                  // FP32 circle points accurate to ~1e-6 R
  bool wellr[2] = {true, true};      // FP32 triple points accurate to ~3e-6 R
  if (type == 0) {
    // circle points: unit n with u_i.n = s_i, u_j.n = s_j (two tangency
    // circles on the nodal sphere)
    U c = dot(E[i].u, E[j].u);
    U q = U(1) - c * c;
    if (F64) {
      if (q < U(EPS_PAR)) return;
    } else {
      if (q < U(0.5 * EPS_PAR)) return;
      if (q < U(M_COND)) { o.unc = 1; return; }
    }
    U iq = U(1) / q;
    U al = (E[i].s - c * E[j].s) * iq;
    U be = (E[j].s - c * E[i].s) * iq;
    U g2 = U(1) - (al * al + be * be + U(2) * al * be * c);
    if (F64) {
      if (g2 <= U(0)) {
        if (g2 > U(-EPS_TAN)) o.nflags |= NF_NEAR_TANGENT;
        return;
      }
    } else {
      U mag = U(1) + al * al + be * be;
      if (g2 < U(-1e-3) * mag) return;
      if (g2 < U(M_COND) * mag) { o.unc = 1; return; }
    }
    if constexpr (!F64) well = q >= U(M_POS) && g2 >= U(M_POS) * (U(1) + al * al + be * be);
    V3<U> w = cross(E[i].u, E[j].u);
    w = w * (U(1) / norm3(w));
    U g = lm_sqrt(g2);
    V3<U> base = E[i].u * al + E[j].u * be;
    o.z[0] = (base - w * g) * R;
    o.z[1] = (base + w * g) * R;
    o.t0[0] = o.t0[1] = U(0);
    gmask = (1ull << i) | (1ull << j);
    sph0 = true;
    tanq = g2 - U(EPS_TAN);
  } else {
    // triple points: line P_ij n P_ik cut with the cone of i
    V3<U> mj = E[i].u * E[i].ico - E[j].u * E[j].ico;
    V3<U> mk = E[i].u * E[i].ico - E[k].u * E[k].ico;
    U dj = R * (E[i].s * E[i].ico - E[j].s * E[j].ico);
    U dk = R * (E[i].s * E[i].ico - E[k].s * E[k].ico);
    V3<U> v = cross(mj, mk);
    U vv = dot(v, v);
    U mm = dot(mj, mj) * dot(mk, mk);
    if (F64) {
      if (vv < U(EPS_PAR) * mm) return;
    } else {
      if (vv < U(0.5 * EPS_PAR) * mm) return;
      if (vv < U(M_COND) * mm) { o.unc = 1; return; }
    }
    U ivv = U(1) / vv;
    V3<U> z0 = (cross(mk, v) * dj - cross(mj, v) * dk) * ivv;
    V3<U> vh = v * lm_sqrt(ivv);
    U G0 = (dot(E[i].u, z0) - R * E[i].s) * E[i].ico;
    U G1 = dot(E[i].u, vh) * E[i].ico;
    U A = U(1) - G1 * G1;
    U B = -G0 * G1;
    U C = dot(z0, z0) - R * R - G0 * G0;
    if (F64) {
      if (fabs(A) < U(1e-12)) {
        o.nflags |= NF_DEGENERATE | NF_ALONG;
        return;
      }
    } else if (fabsf((float)A) < M_COND) {
      o.unc = 1;
      return;
    }
    U D = B * B - A * C;
    U R2 = R * R;
    if (F64) {
      if (D <= U(0)) {
        if (D > U(-EPS_TAN) * R2) o.nflags |= NF_NEAR_TANGENT;
        return;
      }
    } else {
      U mag = B * B + fabs(A * C) + R2;
      if (D < U(-1e-3) * mag) return;
      if (D < U(M_COND) * R2 || D < U(1e-3) * mag) { o.unc = 1; return; }
    }
    U sq = lm_sqrt(D);
    U lam0, lam1;
    if (B >= U(0)) {
      U q = -(B + sq);
      lam0 = q / A;
      lam1 = C / q;
    } else {
      U q = -B + sq;
      lam1 = q / A;
      lam0 = C / q;
    }
    o.z[0] = z0 + vh * lam0;
    o.z[1] = z0 + vh * lam1;
    o.t0[0] = G0 + lam0 * G1;
    o.t0[1] = G0 + lam1 * G1;
    if constexpr (!F64) {
      // z solves (G_i - G_j, G_i - G_k, |z|^2 - R^2 - G_i^2) = 0 with Jacobian
      // rows mj, mk, nc = z - G_i ico_i u_i; a perturbation of the axes by one
      // roundoff moves the residuals by about |z| ico (|t| ico for the cone
      // row), and the Jacobian inverse is adj / (v . nc)
      U icom = fmax(E[i].ico, fmax(E[j].ico, E[k].ico));
      U svv = lm_sqrt(vv);
#pragma unroll
      for (int r = 0; r < 2; r++) {
        V3<U> nc = o.z[r] - E[i].u * (o.t0[r] * E[i].ico);
        U num = norm3(o.z[r]) * (norm3(cross(mk, nc)) + norm3(cross(nc, mj))) +
                svv * norm3(nc) * fabs(o.t0[r]) * icom;
        wellr[r] = icom * num <= U(M_SENS) * R * fabs(dot(v, nc));
      }
    }
    gmask = (1ull << i) | (1ull << j) | (1ull << k);
    sph0 = false;
    tanq = D - U(EPS_TAN) * R2;
  }
  o.nroot = 2;
  const U M = F64 ? U(0) : U(M_LEN) * R;
  const U eta = U(ETA_SIGMA) * R;
  for (int r = 0; r < 2; r++) {
    o.state[r] = 0;
    o.key[r] = gmask;
    o.sphere[r] = sph0;
    o.tangent[r] = tanq < U(0);
    o.kflags[r] = 0;
    o.umask[r] = 0;
    if (hint && (hint->st[r] == 0 || hint->st[r] == 3)) {
      o.state[r] = hint->st[r];
      continue;
    }
    U t0 = o.t0[r];
    V3<U> z = o.z[r];
    // certain rejections first (inside the sphere side, wrong nappe, inside
    // another strut), then uncertainty, then the exact decisions
    bool rej = false, unc = false;
    uint64_t key = gmask;
    if (t0 < -eta - M) rej = true;
    else if (t0 < -eta + M && !F64) unc = true;
    for (int l = 0; l < d && !rej; l++) {
      if (hint && !((hint->umask[r] >> l) & 1ull)) continue;  // certain in FP32
      if (gmask >> l & 1ull) {
        U np = R - E[l].s * dot(E[l].u, z);
        if (np <= -M) rej = true;
        else if (np <= M) {
          if (F64) rej = true;
          else {
            unc = true;
            o.umask[r] |= 1ull << l;
          }
        }
        continue;
      }
      U sg = (dot(E[l].u, z) - R * E[l].s) * E[l].ico - t0;
      if (sg > eta + M) rej = true;
      else if (sg >= -eta - M) {
        if (F64) key |= 1ull << l;
        else {
          unc = true;
          o.umask[r] |= 1ull << l;
        }
      }
    }
    if (rej) continue;
    bool sph = sph0;
    if (!sph0) {
      if (!F64 && fabs(t0) <= M + eta) unc = true;
      sph = fabs(t0) <= eta;
    }
    uint32_t kf = 0;
    for (int l = 0; l < d; l++) {
      if (!(key >> l & 1ull)) continue;
      U lim = E[l].L * E[l].co;
      if (!F64 && fabs(t0 - lim) <= M) unc = true;
      if (t0 > lim) kf |= NF_DEGENERATE | NF_BEYOND;
    }
    if (unc || !well || !wellr[r]) {
      o.state[r] = 2;
      continue;
    }
    o.key[r] = key;
    o.sphere[r] = sph;
    o.state[r] = 1;
    o.kflags[r] = kf | (o.tangent[r] ? NF_NEAR_TANGENT : 0u);
  }
}

// Re-decision of a triple-point root whose FP32 screening was uncertain
// (partially: the generator itself was well conditioned), without
// recomputing the point from scratch.  Newton steps from its FP32 position
// zf on F(z) = (G_i - G_j, G_i - G_k, |z|^2 - R^2 - G_i^2) = 0, the residual
// in double-float and the correction from the FP32 Jacobian J (rows m_j,
// m_k, 2 (z - G_i ico_i u_i)) taken at zf.  A point is accepted once the
// first-order error bound |J^-1| |F| (row by row) times (1 + max ico) is
// below 1e-12 R, three orders inside the tie tolerance ETA_SIGMA R: after at
// most two steps (the FP32 error ~1e-6 R shrinks by the Jacobian's relative
// error ~1e-7 per step, plus a quadratic term ~|e|^2 / R).  If J is ill
// conditioned or the bound is not met, false is returned and the caller
// recomputes the generator in double-float.  Otherwise the screening
// decisions of the ends in umask and the root-level decisions are taken as
// eval_gen does in exact mode.  Outputs: state (0 rejected, 1 kept), key,
// sphere flag, node flags if kept, the refined position.
__device__ __forceinline__ bool rescreen_triple_df(const EndG<df>* E, const EndG<float>* EF, int d, float Rf,
                                                       uint32_t gcode, V3<float> zf, uint64_t umask,
                                                       uint8_t& state, uint64_t& key, uint8_t& sphere,
                                                       uint32_t& kflags, V3<float>& zout) {
  const int i = (gcode >> 3) & 63, j = (gcode >> 9) & 63, k = (gcode >> 15) & 63;
  const df R(Rf);
  auto G = [&](int l, const V3<df>& p) { return (dot(E[l].u, p) - R * E[l].s) * E[l].ico; };
  const float tf = (dot(EF[i].u, zf) - Rf * EF[i].s) * EF[i].ico;
  const V3<float> a = EF[i].u * EF[i].ico - EF[j].u * EF[j].ico;
  const V3<float> b = EF[i].u * EF[i].ico - EF[k].u * EF[k].ico;
  const V3<float> c = (zf - EF[i].u * (tf * EF[i].ico)) * 2.0f;
  const V3<float> bc = cross(b, c), ca = cross(c, a), ab = cross(a, b);
  const float det = dot(a, bc);
  if (!(fabsf(det) > 1e-3f * norm3(a) * norm3(b) * norm3(c))) return false;
  const float idet = 1.0f / det;
  const float nbc = norm3(bc), nca = norm3(ca), nab = norm3(ab);
  const float tol = 1e-12f * Rf * fabsf(det) / (1.0f + fmaxf(EF[i].ico, fmaxf(EF[j].ico, EF[k].ico)));
  V3<df> z = mk3(df(zf.x), df(zf.y), df(zf.z));
  df t0;
  for (int it = 0;; it++) {
    t0 = G(i, z);
    const float F0 = (float)(t0 - G(j, z)), F1 = (float)(t0 - G(k, z));
    const float F2 = (float)(dot(z, z) - R * R - t0 * t0);
    if (nbc * fabsf(F0) + nca * fabsf(F1) + nab * fabsf(F2) <= tol) break;
    if (it == 2) return false;
    const V3<float> dz = (bc * F0 + ca * F1 + ab * F2) * (-idet);
    z = z + mk3(df(dz.x), df(dz.y), df(dz.z));
  }
  const uint64_t gmask = (1ull << i) | (1ull << j) | (1ull << k);
  const df eta = df(ETA_SIGMA) * R;
  zout = mk3((float)z.x, (float)z.y, (float)z.z);
  state = 0;
  if (t0 < -eta) return true;
  key = gmask;
  for (int l = 0; l < d; l++) {
    if (!((umask >> l) & 1ull)) continue;
    if ((gmask >> l) & 1ull) {
      if (R - E[l].s * dot(E[l].u, z) <= df(0.0f)) return true;  // wrong nappe
      continue;
    }
    const df sg = G(l, z) - t0;
    if (sg > eta) return true;
    if (sg >= -eta) key |= 1ull << l;
  }
  sphere = fabs(t0) <= eta;
  uint32_t kf = 0;
  for (int l = 0; l < d; l++)
    if (((key >> l) & 1ull) && t0 > E[l].L * E[l].co) kf |= NF_DEGENERATE | NF_BEYOND;
  kflags = kf;
  state = 1;
  return true;
}

// Recompute vertex `gcode` (a kept candidate root, or a seam) in precision U.
template <typename U>
__device__ V3<U> vertex_from_gen(const EndG<U>* E, int d, U R, uint32_t gcode) {
  int type = gcode & 3, root = (gcode >> 2) & 1;
  if (type == 2) {
    int i = (gcode >> 3) & 63, lab = (gcode >> 9) & 63;
    bool has = (gcode >> 21) & 1;
    U t = has ? hval(E[i], E[lab], U(1), U(0), R) : U(0);
    return surf_point(E[i], U(1), U(0), t, R);
  }
  GenOut<U> o;
  eval_gen<U, true>(E, d, R, gcode & ~4u, o);
  return o.z[root];
}

__device__ __forceinline__ uint64_t warp_or64(uint64_t x) {
  uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)x);
  uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(x >> 32));
  return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ int warp_excl_scan(int x, int lane) {
  int v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v - x;
}

template <typename T>
__device__ __forceinline__ T norm_angle(T a) {
  return a < T(-PHI_CUT) ? a + T(PI2) : a;
}

// x moved by a multiple of 2pi into [lo, lo + 2pi) (one floor, no loop)
template <typename T>
__device__ __forceinline__ T wrap_from(T x, T lo) {
  T r = x - T(PI2) * floor((x - lo) * T(1.0 / PI2));
  if (r < lo) r += T(PI2);
  if (r >= lo + T(PI2)) r -= T(PI2);
  return r;
}

// Largest generator coordinate t of the elliptical arc of plane P_ij on
// strut end i over angles [phi0, phi0 + dphi]: h = (n0 + n1 c + n2 s) /
// (d0 + d1 c + d2 s) has its interior extrema where P c + Q s = W.
template <typename U>
__device__ U arc_tmax(const EndG<U>& Ei, const EndG<U>& Ej, U R, U phi0, U dphi) {
  U cij = dot(Ei.u, Ej.u), a1 = dot(Ej.u, Ei.e1), a2 = dot(Ej.u, Ei.e2);
  U n0 = R * (Ei.s * cij - Ej.s), n1 = R * Ei.co * a1, n2 = R * Ei.co * a2;
  U d0 = Ej.co - Ei.co * cij, d1 = Ei.s * a1, d2 = Ei.s * a2;
  U c, s;
  lm_sincos(phi0, &s, &c);
  U tmax = hval(Ei, Ej, c, s, R);
  lm_sincos(phi0 + dphi, &s, &c);
  U t1 = hval(Ei, Ej, c, s, R);
  if (t1 > tmax) tmax = t1;
  U P = n2 * d0 - n0 * d2, Q = n0 * d1 - n1 * d0, W = n1 * d2 - n2 * d1;
  U rr = lm_sqrt(P * P + Q * Q);
  if (rr > fabs(W) && rr > U(0)) {
    U base = lm_atan2(Q, P);
    U off = acos(W / rr);
    for (int sg = -1; sg <= 1; sg += 2) {
      U ph = base + U(sg) * off;
      U rel = ph - phi0;
      rel -= U(PI2) * floor(rel * U(1.0 / PI2));
      if (rel < dphi) {
        lm_sincos(phi0 + rel, &s, &c);
        U t = hval(Ei, Ej, c, s, R);
        if (t > tmax) tmax = t;
      }
    }
  }
  return tmax;
}

// FP32 strut-end data promoted to FP64 (for FP64 arithmetic on FP32 inputs)
__device__ __forceinline__ EndG<double> promote(const EndG<float>& a) {
  EndG<double> e;
  e.u = cvt3<double>(a.u);
  e.e1 = cvt3<double>(a.e1);
  e.e2 = cvt3<double>(a.e2);
  e.s = a.s;
  e.co = a.co;
  e.ico = 1.0 / (double)a.co;
  e.L = a.L;
  e.end_id = a.end_id;
  e.far = a.far;
  e.at_lo = a.at_lo;
  return e;
}
__device__ __forceinline__ EndG<double> promote(const EndG<double>& a) { return a; }

// Candidate positions of generator gcode in FP64 arithmetic, without
// screening (the decisions were certain; only the positions need accuracy).
template <typename U>
__device__ __noinline__ void gen_points64(const EndG<U>* E, U R, uint32_t gcode, V3<double> z[2],
                                          double t0[2]) {
  int type = gcode & 3, i = (gcode >> 3) & 63, j = (gcode >> 9) & 63, k = (gcode >> 15) & 63;
  EndG<double> Ei = promote(E[i]), Ej = promote(E[j]);
  double Rd = (double)R;
  if (type == 0) {
    double c = dot(Ei.u, Ej.u), q = 1.0 - c * c, iq = 1.0 / q;
    double al = (Ei.s - c * Ej.s) * iq, be = (Ej.s - c * Ei.s) * iq;
    double g2 = 1.0 - (al * al + be * be + 2.0 * al * be * c);
    V3<double> w = cross(Ei.u, Ej.u);
    w = w * (1.0 / norm3(w));
    double g = sqrt(g2 > 0.0 ? g2 : 0.0);
    V3<double> base = Ei.u * al + Ej.u * be;
    z[0] = (base - w * g) * Rd;
    z[1] = (base + w * g) * Rd;
    t0[0] = t0[1] = 0.0;
    return;
  }
  EndG<double> Ek = promote(E[k]);
  V3<double> mj = Ei.u * Ei.ico - Ej.u * Ej.ico;
  V3<double> mk = Ei.u * Ei.ico - Ek.u * Ek.ico;
  double dj = Rd * (Ei.s * Ei.ico - Ej.s * Ej.ico);
  double dk = Rd * (Ei.s * Ei.ico - Ek.s * Ek.ico);
  V3<double> v = cross(mj, mk);
  double ivv = 1.0 / dot(v, v);
  V3<double> z0 = (cross(mk, v) * dj - cross(mj, v) * dk) * ivv;
  V3<double> vh = v * sqrt(ivv);
  double G0 = (dot(Ei.u, z0) - Rd * Ei.s) * Ei.ico;
  double G1 = dot(Ei.u, vh) * Ei.ico;
  double A = 1.0 - G1 * G1, B = -G0 * G1, C = dot(z0, z0) - Rd * Rd - G0 * G0;
  double D = B * B - A * C;
  double sq = sqrt(D > 0.0 ? D : 0.0);
  double lam0, lam1;
  if (B >= 0.0) {
    double q = -(B + sq);
    lam0 = q / A;
    lam1 = C / q;
  } else {
    double q = -B + sq;
    lam1 = q / A;
    lam0 = C / q;
  }
  z[0] = z0 + vh * lam0;
  z[1] = z0 + vh * lam1;
  t0[0] = G0 + lam0 * G1;
  t0[1] = G0 + lam1 * G1;
}

// Compact geometry of one arc for point evaluation: owner frame and the
// plane ratio t(phi) = (n0 + n1 c + n2 s) / (d0 + d1 c + d2 s) (t = 0 on a
// circular arc).  Point: (R s + t co) u + (R co - t s) rho(phi).
template <typename T>
struct ArcGeo {
  V3<T> u, e1, e2;
  T Rs, Rco, co, s;
  T n0, n1, n2, d0, d1, d2;
};

template <typename T>
__device__ __forceinline__ ArcGeo<T> arc_geo(const EndG<T>& o, const EndG<T>* ot, T R) {
  ArcGeo<T> g;
  g.u = o.u;
  g.e1 = o.e1;
  g.e2 = o.e2;
  g.Rs = R * o.s;
  g.Rco = R * o.co;
  g.co = o.co;
  g.s = o.s;
  if (ot) {
    T cij = dot(o.u, ot->u), a1 = dot(ot->u, o.e1), a2 = dot(ot->u, o.e2);
    g.n0 = R * (o.s * cij - ot->s);
    g.n1 = R * o.co * a1;
    g.n2 = R * o.co * a2;
    g.d0 = ot->co - o.co * cij;
    g.d1 = o.s * a1;
    g.d2 = o.s * a2;
  } else {
    g.n0 = g.n1 = g.n2 = T(0);
    g.d0 = T(1);
    g.d1 = g.d2 = T(0);
  }
  return g;
}

template <typename T>
__device__ __forceinline__ V3<T> geo_point(const ArcGeo<T>& g, T phi) {
  T c, s;
  lm_sincos(phi, &s, &c);
  T t = (g.n0 + g.n1 * c + g.n2 * s) / (g.d0 + g.d1 * c + g.d2 * s);
  V3<T> r = g.e1 * c + g.e2 * s;
  return g.u * (g.Rs + t * g.co) + r * (g.Rco - t * g.s);
}

// Whether an elliptical arc [phi0, phi0 + dphi] of geometry g is
// ill-conditioned in the sense of D_ILL: D(phi) = d0 + rho cos(phi - phi_d)
// is bounded on the arc by its values at the ends and at its interior
// extremes.
template <typename T>
__device__ __forceinline__ bool arc_ill(const ArcGeo<T>& g, T phi0, T dphi) {
  const T rho = lm_sqrt(g.d1 * g.d1 + g.d2 * g.d2);
  // D keeps |D| >= D_ILL on the whole circle
  if (fabs(g.d0) - rho >= T(D_ILL)) return false;
  T c, s;
  lm_sincos(phi0, &s, &c);
  const T D0 = g.d0 + g.d1 * c + g.d2 * s;
  lm_sincos(phi0 + dphi, &s, &c);
  const T D1 = g.d0 + g.d1 * c + g.d2 * s;
  T lo = fmin(D0, D1), hi = fmax(D0, D1);
  if (rho > T(0)) {
    const T pd = lm_atan2(g.d2, g.d1);
    T r = pd - phi0;
    r -= T(PI2) * floor(r * T(1.0 / PI2));
    if (r <= dphi) hi = fmax(hi, g.d0 + rho);
    r = pd + T(0.5 * PI2) - phi0;
    r -= T(PI2) * floor(r * T(1.0 / PI2));
    if (r <= dphi) lo = fmin(lo, g.d0 - rho);
  }
  return lo < T(D_ILL) && hi > -T(D_ILL);
}

// Exactly rounded operations: no contraction or reassociation is left to the
// compiler, so an expression gives the same bits wherever it is inlined.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
// a / b within 2 ulp (FP32: reciprocal approximation times a; the same two
// instructions wherever it is inlined)
__device__ __forceinline__ float div_fast(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_fast(double a, double b) { return __ddiv_rn(a, b); }

// Subdivision point m of N of an arc (node-relative; Section 5: uniform in the
// owner's angle, phi = phi0 + dphi m / N, also returned) with every operation
// explicitly rounded (the two quotients within 2 ulp): the kernels that emit a shared point (the two struts of
// an elliptical arc, a strut and a hole fan of a circular arc) write the same
// bits.
template <typename T>
__device__ __forceinline__ V3<T> arc_point_rn(const ArcGeo<T>& g, T phi0, T dphi, int m, int N, T& phi) {
  phi = add_rn(phi0, div_fast(mul_rn(dphi, (T)m), (T)N));
  T c, s;
  lm_sincos(phi, &s, &c);
  const T t = div_fast(fma_rn(g.n2, s, fma_rn(g.n1, c, g.n0)), fma_rn(g.d2, s, fma_rn(g.d1, c, g.d0)));
  const T a = fma_rn(t, g.co, g.Rs), b = fma_rn(-t, g.s, g.Rco);
  V3<T> z;
  z.x = fma_rn(fma_rn(g.e2.x, s, mul_rn(g.e1.x, c)), b, mul_rn(g.u.x, a));
  z.y = fma_rn(fma_rn(g.e2.y, s, mul_rn(g.e1.y, c)), b, mul_rn(g.u.y, a));
  z.z = fma_rn(fma_rn(g.e2.z, s, mul_rn(g.e1.z, c)), b, mul_rn(g.u.z, a));
  return z;
}

// Node-relative point of vertex generator `gcode` from the node's strut ends
// (no screening: the vertex is known to be kept).  Circle point: unit n with
// u_i.n = s_i and u_j.n = s_j, times R.  Triple point: line P_ij n P_ik cut
// with cone i, root (-B -/+ sqrt(B^2 - A C))/A in the stable form.  Seam:
// generator at angle 0 of strut end i, cut by plane P_ij when labelled.
template <typename U>
__device__ V3<U> gen_point(const EndG<U>* E, U R, uint32_t gcode) {
  int type = gcode & 3, root = (gcode >> 2) & 1;
  int i = (gcode >> 3) & 63, j = (gcode >> 9) & 63, k = (gcode >> 15) & 63;
  if (type == 0) {
    U c = dot(E[i].u, E[j].u);
    U q = U(1) - c * c;
    U al = (E[i].s - c * E[j].s) / q;
    U be = (E[j].s - c * E[i].s) / q;
    U g2 = U(1) - (al * al + be * be + U(2) * al * be * c);
    V3<U> w = cross(E[i].u, E[j].u);
    w = w * (U(1) / norm3(w));
    U g = lm_sqrt(g2);
    V3<U> base = E[i].u * al + E[j].u * be;
    return (root == 0 ? base - w * g : base + w * g) * R;
  }
  if (type == 1) {
    V3<U> mj = E[i].u * E[i].ico - E[j].u * E[j].ico;
    V3<U> mk = E[i].u * E[i].ico - E[k].u * E[k].ico;
    U dj = R * (E[i].s * E[i].ico - E[j].s * E[j].ico);
    U dk = R * (E[i].s * E[i].ico - E[k].s * E[k].ico);
    V3<U> v = cross(mj, mk);
    U ivv = U(1) / dot(v, v);
    V3<U> z0 = (cross(mk, v) * dj - cross(mj, v) * dk) * ivv;
    V3<U> vh = v * lm_sqrt(ivv);
    U G0 = (dot(E[i].u, z0) - R * E[i].s) * E[i].ico;
    U G1 = dot(E[i].u, vh) * E[i].ico;
    U A = U(1) - G1 * G1, B = -(G0 * G1), C = dot(z0, z0) - R * R - G0 * G0;
    U sq = lm_sqrt(B * B - A * C);
    U lam;
    if (B >= U(0)) {
      U q = -(B + sq);
      lam = root == 0 ? q / A : C / q;
    } else {
      U q = sq - B;
      lam = root == 1 ? q / A : C / q;
    }
    return z0 + vh * lam;
  }
  U t = U(0);
  if ((gcode >> 21) & 1) t = hval(E[i], E[j], U(1), U(0), R);
  return surf_point(E[i], U(1), U(0), t, R);
}

// Position of a stored vertex recomputed in FP64 from the inputs, using only
// the strut ends that generated it (no screening: the vertex is known kept).
template <typename T>
__device__ __noinline__ V3<double> vertex_pos64(const LatDev<T>& L, int64_t node, uint32_t gcode) {
  int64_t b = L.row_ptr[node];
  int type = gcode & 3, root = (gcode >> 2) & 1;
  int i = (gcode >> 3) & 63, j = (gcode >> 9) & 63, k = (gcode >> 15) & 63;
  double R = (double)L.node_R[node];
  EndG<double> Ei = make_end<T, double>(L, node, L.adj[b + i]);
  if (type == 2) {
    bool has = (gcode >> 21) & 1;
    double t = 0.0;
    if (has) {
      EndG<double> Ej = make_end<T, double>(L, node, L.adj[b + j]);
      t = hval(Ei, Ej, 1.0, 0.0, R);
    }
    return surf_point(Ei, 1.0, 0.0, t, R);
  }
  EndG<double> Ej = make_end<T, double>(L, node, L.adj[b + j]);
  EndG<double> E3[3];
  E3[0] = Ei;
  E3[1] = Ej;
  V3<double> z[2];
  double t0[2];
  if (type == 0) {
    gen_points64<double>(E3, R, gen_code(0, 0, 0, 1, 0), z, t0);
  } else {
    E3[2] = make_end<T, double>(L, node, L.adj[b + k]);
    gen_points64<double>(E3, R, gen_code(1, 0, 0, 1, 2), z, t0);
  }
  return z[root];
}

}  // namespace lm
