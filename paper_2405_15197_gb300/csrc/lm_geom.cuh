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

namespace lm {

constexpr double PI2 = 6.283185307179586476925286766559;

// Decision thresholds (readings of ties the paper is silent on).
constexpr double ETA_SIGMA = 1e-9;  // x R: a strut passes through a vertex
constexpr double ETA_DEDUP = 1e-3;  // x R: candidates with one key are one vertex
constexpr double ETA_PHI = 1e-9;    // rad: angles normalised to [-ETA_PHI, 2pi - ETA_PHI)
constexpr double ETA_ZIP = 1e-9;    // rad: stitching tie
constexpr double TAU_COUNT = 1e-6;  // segment count offset
constexpr double ETA_BARY = 1e-4;   // x R: hole barycentre at the centre
constexpr double EPS_PAR = 1e-6;    // 1 - c^2 below this: (anti)parallel pair
constexpr double EPS_TAN = 1e-6;    // tangency measure: node exempt from exact parity

// FP32 safety margins: an FP32 quantity closer than this to a decision
// threshold, or computed from an ill-conditioned configuration, is decided
// again in FP64 from the inputs.
constexpr float M_LEN = 1e-3f;   // x R
constexpr float M_ANG = 1e-4f;   // rad
constexpr float M_COND = 1e-2f;  // conditioning floor of q, |v|^2, |A|, D/R^2, g2
constexpr float M_CNT = 1e-3f;   // segment-count fraction
constexpr float M_POS = 1e-1f;   // conditioning floor for keeping an FP32 vertex position

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
__device__ __forceinline__ float lm_atan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double lm_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ void lm_sincos(float a, float* s, float* c) { sincosf(a, s, c); }
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

// Frame axis: the coordinate axis of smallest |x_hi - x_lo| (ties -> lowest).
// FP32 differences decide when strictly ordered; a tie is re-decided on the
// exact FP64 differences of the inputs.
template <typename T>
__device__ __forceinline__ int frame_axis(const LatDev<T>& L, int32_t lo, int32_t hi) {
  float a0 = fabsf((float)L.xyz[3 * hi] - (float)L.xyz[3 * lo]);
  float a1 = fabsf((float)L.xyz[3 * hi + 1] - (float)L.xyz[3 * lo + 1]);
  float a2 = fabsf((float)L.xyz[3 * hi + 2] - (float)L.xyz[3 * lo + 2]);
  if (a0 != a1 && a0 != a2 && a1 != a2 && sizeof(T) == 4) {
    int ax = 0;
    if (a1 < a0) ax = 1;
    if (a2 < (ax == 0 ? a0 : a1)) ax = 2;
    return ax;
  }
  double d0 = fabs((double)L.xyz[3 * hi] - (double)L.xyz[3 * lo]);
  double d1 = fabs((double)L.xyz[3 * hi + 1] - (double)L.xyz[3 * lo + 1]);
  double d2 = fabs((double)L.xyz[3 * hi + 2] - (double)L.xyz[3 * lo + 2]);
  int ax = 0;
  double best = d0;
  if (d1 < best) { ax = 1; best = d1; }
  if (d2 < best) ax = 2;
  return ax;
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
  uint32_t nflags;    // node flags raised independent of survival
  uint32_t kflags[2]; // node flags raised if the root is kept as a new vertex
};

// Candidates of one generator with screening (trimming) against every strut
// end of the node.  F64 = true: all decisions exact (thresholds only).
// F64 = false: decisions within the FP32 margins are reported uncertain.
template <typename U, bool F64>
__device__ void eval_gen(const EndG<U>* E, int d, U R, uint32_t gcode, GenOut<U>& o) {
  o.nroot = 0;
  o.unc = 0;
  o.nflags = 0;
  int type = gcode & 3, i = (gcode >> 3) & 63, j = (gcode >> 9) & 63, k = (gcode >> 15) & 63;
  uint64_t gmask;
  bool sph0;
  U tanq;
  bool well = true;  // FP32 positions accurate to ~1e-6 R
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
    if (!F64) well = q >= U(M_POS) && g2 >= U(M_POS) * (U(1) + al * al + be * be);
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
      if (fabs((double)A) < 1e-12) {
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
    if (!F64)
      well = vv >= U(M_POS) * mm && fabs(A) >= U(M_POS) && D >= U(M_POS) * R2 &&
             D >= U(M_POS) * (B * B + fabs(A * C) + R2);
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
    U t0 = o.t0[r];
    V3<U> z = o.z[r];
    // certain rejections first (inside the sphere side, wrong nappe, inside
    // another strut), then uncertainty, then the exact decisions
    bool rej = false, unc = false;
    uint64_t key = gmask;
    if (t0 < -eta - M) rej = true;
    else if (t0 < -eta + M && !F64) unc = true;
    for (int l = 0; l < d && !rej; l++) {
      if (gmask >> l & 1ull) {
        U np = R - E[l].s * dot(E[l].u, z);
        if (np <= -M) rej = true;
        else if (np <= M) {
          if (F64) rej = true;
          else unc = true;
        }
        continue;
      }
      U sg = (dot(E[l].u, z) - R * E[l].s) * E[l].ico - t0;
      if (sg > eta + M) rej = true;
      else if (sg >= -eta - M) {
        if (F64) key |= 1ull << l;
        else unc = true;
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
    if (unc || !well) {
      o.state[r] = 2;
      continue;
    }
    o.key[r] = key;
    o.sphere[r] = sph;
    o.state[r] = 1;
    o.kflags[r] = kf | (o.tangent[r] ? NF_NEAR_TANGENT : 0u);
  }
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
  return a < T(-ETA_PHI) ? a + T(PI2) : a;
}

// x moved by a multiple of 2pi into [lo, lo + 2pi) (one floor, no loop)
template <typename T>
__device__ __forceinline__ T wrap_from(T x, T lo) {
  T r = x - T(PI2) * floor((x - lo) * T(1.0 / PI2));
  if (r < lo) r += T(PI2);
  if (r >= lo + T(PI2)) r -= T(PI2);
  return r;
}

}  // namespace lm
