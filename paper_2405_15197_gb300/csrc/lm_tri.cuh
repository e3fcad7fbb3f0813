// Resolution-k triangulation of the meta-mesh (Section 5 of arXiv
// 2405.15197, Algorithm 1), on the GPU.
//
//  * segment count per arc: Eq. sampling with chord error CE = 1 - cos(pi/k),
//    read as N = max(1, ceil(dphi k / 2pi - TAU_COUNT));
//  * subdivision points uniform in the owner strut's angle (Eq.
//    parameter-range, sampled on the strut's end circle and mapped onto the
//    arc), evaluated once per shared arc in the owner's frame so both struts
//    emit bit-identical coordinates;
//  * strut stitching: a zipper between the strut's two arc loops in the
//    strut angle, computed with ranks (each lane places its own triangles);
//  * hole filling: fan from the barycentre projected onto the nodal sphere.
// Triangles are written as 50-byte binary-STL records staged in shared
// memory and stored with 16-byte vector stores.
#pragma once
#include "lm_geom.cuh"

namespace lm {

template <typename T>
struct TriArgs {
  LatDev<T> lat;
  const int64_t *vtx_off, *arc_off, *end_off, *node_hole_off, *hole_off;
  const T* vtx_z;
  const uint32_t* vtx_gen;
  const uint32_t* arc_vtx;  // v0 | v1<<8 | owner_local<<16 | (other_local+1)<<24
  const T* arc_phi;
  const uint32_t* loop_ent;
  const uint32_t* hole_ent;
  int k;
  int32_t* item_cnt;       // count pass: [E+N]
  const int64_t* tri_off;  // [E+N+1]
  int64_t item_begin, item_end, out_first, capacity;
  uint8_t* out;            // STL records (NULL: objective only)
  double* acc;             // area, volume accumulators (NULL: none)
  int* queue;
  int* err;
  int pmax;                // points per loop capacity
  int emax;                // loop entries capacity
  int dmax;                // largest node valence
  int* max_pts;            // count pass: max points of one loop / one node's holes
  unsigned long long* fb;  // FP64 stability-step counters (8: segments, 9: start angle,
                           // 10: stitching order, 11: fan centre)
  // device-side item range [2] (chunks replayed from one CUDA graph), or NULL:
  // item_begin / item_end and first_ptr then apply
  const int64_t* range;
  // [N]: the hole items of nodes whose mask is 0 have no triangles (NULL:
  // every node's holes are filled)
  const uint8_t* node_mask;
  // struts deferred to the FP64 stitching pass, listed: [0] count, then up to
  // rcap strut ids (NULL: the pass scans the deferral bitmap instead; so it
  // does when the count exceeds rcap)
  unsigned long long* rlist;
  int64_t rcap;
  // adjoint (point adjoints instead of records)
  T* adj;                     // [n_vtx + interior arc points][3]
  const int64_t* arc_pt_off;  // [A + 1] first interior point of each arc
  int64_t n_vtx;
  double w_area, w_vol;
};

__device__ __forceinline__ void tfb_add(unsigned long long* fb, int which, bool pred,
                                        unsigned mask = 0xffffffffu) {
  uint32_t m = __ballot_sync(mask, pred);
  if (fb && m && (threadIdx.x & 31) == (__ffs(m) - 1)) atomicAdd(fb + which, (unsigned long long)__popc(m));
}

// ---- segment count (Eq. sampling) with an FP64 recheck flag
template <typename T>
__device__ __forceinline__ int seg_count(T dphi, int k, bool& unc) {
  T y = dphi * (T)k * T(1.0 / PI2) - T(TAU_COUNT);
  T c = ceil(y);
  unc = sizeof(T) == 4 && fabs(y - rint(y)) <= T(M_CNT) * (T)k * T(1.0 / PI2);
  int n = (int)c;
  return n < 1 ? 1 : n;
}

// FP64 context of a node: its strut ends in FP64, built on demand.
struct Node64 {
  EndG<double> E[64];
  int d;
  double R;
  int64_t node;
};

template <typename T>
__device__ __noinline__ void load_node64(const LatDev<T>& L, int64_t n, Node64* ctx, int lane) {
  int64_t b = L.row_ptr[n];
  int d = (int)(L.row_ptr[n + 1] - b);
  for (int li = lane; li < d; li += 32) ctx->E[li] = make_end<T, double>(L, n, L.adj[b + li]);
  if (lane == 0) {
    ctx->d = d;
    ctx->R = (double)L.node_R[n];
    ctx->node = n;
  }
  __syncwarp();
}

// exact angular length of arc (node-local id a) in its owner's frame
template <typename T>
__device__ __noinline__ double arc_dphi64(const TriArgs<T>& A, const Node64* ctx, int64_t ga,
                                          double* a0_out) {
  if (ctx->node < 0 || ctx->d < 1 || ctx->d > 64) {
    // context not loaded for this node: keep the FP32 values, report
    atomicCAS(A.err, 0, 6);
    if (a0_out) *a0_out = (double)A.arc_phi[2 * ga];
    return (double)A.arc_phi[2 * ga + 1];
  }
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255, o = (av >> 16) & 255;
  int64_t vo = A.vtx_off[ctx->node];
  V3<double> z0 = vertex_from_gen<double>(ctx->E, ctx->d, ctx->R, A.vtx_gen[vo + v0]);
  V3<double> z1 = vertex_from_gen<double>(ctx->E, ctx->d, ctx->R, A.vtx_gen[vo + v1]);
  double a0 = raw_angle(ctx->E[o], z0), a1 = raw_angle(ctx->E[o], z1);
  if (a0 < -PHI_CUT) a0 += PI2;
  if (a1 < -PHI_CUT) a1 += PI2;
  double dd = a1 - a0;
  if (v0 == v1) dd = PI2;
  else if (dd <= 0.0) dd += PI2;
  if (a0_out) *a0_out = a0;
  return dd;
}

template <typename T>
__device__ int arc_segments(const TriArgs<T>& A, int64_t node, int64_t ga, Node64* ctx,
                            int lane_unused) {
  bool unc;
  int N = seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
  if (!unc) return N;
  if (ctx->node != node) {
    atomicCAS(A.err, 0, 6);
    return N;
  }
  // exact re-decision from the inputs
  double dd = arc_dphi64(A, ctx, ga, nullptr);
  bool u2;
  return seg_count<double>(dd, A.k, u2);
}

// ---------------------------------------------------------------- counts
// Triangle counts of items [b, e) into cnt[item - b] and the largest point
// count of one loop (or of one node's holes) into *max_pts (atomic max).
// One FP64 context per warp in scratch (the grid has at most as many warps).
template <typename T>
__global__ void __launch_bounds__(256) k_tri_count(TriArgs<T> A, Node64* scratch, int64_t b, int64_t e,
                                                   int32_t* cnt, int* max_pts) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  Node64* ctx = scratch + gw;
  const int64_t E = A.lat.n_struts;
  const int64_t n_items = e;
  // one thread per item, lanes of a warp on consecutive items; an exact
  // recount (rare) loads the node's FP64 context warp-cooperatively
  for (int64_t base = b + (int64_t)gw * 32; base < n_items; base += (int64_t)nwarps * 32) {
    int64_t it = base + lane;
    int64_t cs[2] = {0, 0};
    bool need = false;
    int64_t nodes[2] = {-1, -1};
    if (it < n_items) {
      if (it < E) {
        for (int s = 0; s < 2; s++) {
          int64_t nd = A.lat.ends[2 * it + s];
          int64_t eid = 2 * it + s;
          int64_t ao = A.arc_off[nd];
          for (int64_t q = A.end_off[eid]; q < A.end_off[eid + 1]; q++) {
            int64_t ga = ao + (A.loop_ent[q] & 0x7fffffffu);
            bool unc;
            cs[s] += seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
            if (unc) { need = true; nodes[s] = nd; }
          }
        }
      } else if (!A.node_mask || A.node_mask[it - E]) {
        int64_t nd = it - E;
        int64_t ao = A.arc_off[nd];
        for (int64_t h = A.node_hole_off[nd]; h < A.node_hole_off[nd + 1]; h++)
          for (int64_t q = A.hole_off[h]; q < A.hole_off[h + 1]; q++) {
            int64_t ga = ao + (A.hole_ent[q] & 0x7fffffffu);
            bool unc;
            cs[0] += seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
            if (unc) { need = true; nodes[0] = nd; }
          }
      }
    }
    uint32_t m = __ballot_sync(0xffffffffu, need);
    while (m) {
      int src = __ffs(m) - 1;
      m &= m - 1;
      int64_t it2 = __shfl_sync(0xffffffffu, it, src);
      for (int s = 0; s < 2; s++) {
        int64_t nd = __shfl_sync(0xffffffffu, nodes[s], src);
        if (nd < 0) continue;
        load_node64(A.lat, nd, ctx, lane);
        __syncwarp();
        if (lane == src) {
          int64_t ao = A.arc_off[nd];
          // recount the entries of this node exactly
          if (it2 < E) {
            int64_t eid = 2 * it2 + s;
            for (int64_t q = A.end_off[eid]; q < A.end_off[eid + 1]; q++) {
              int64_t ga = ao + (A.loop_ent[q] & 0x7fffffffu);
              bool unc;
              int n32 = seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
              if (unc) cs[s] += arc_segments<T>(A, nd, ga, ctx, 0) - n32;
            }
          } else {
            for (int64_t h = A.node_hole_off[nd]; h < A.node_hole_off[nd + 1]; h++)
              for (int64_t q = A.hole_off[h]; q < A.hole_off[h + 1]; q++) {
                int64_t ga = ao + (A.hole_ent[q] & 0x7fffffffu);
                bool unc;
                int n32 = seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
                if (unc) cs[0] += arc_segments<T>(A, nd, ga, ctx, 0) - n32;
              }
          }
        }
        __syncwarp();
      }
    }
    int64_t c = cs[0] + cs[1];
    int mx = (int)(cs[0] > cs[1] ? cs[0] : cs[1]);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0 && mx > 0) atomicMax(max_pts, mx);
    if (it < n_items) cnt[it - b] = (int32_t)c;
  }
}

// Geometry of the arc owned by strut end `oid` (cut by the plane of `otid`, or
// circular when otid < 0) at a node, with every operation explicitly rounded:
// every kernel that subdivides the arc starts from the same bits (the same
// arithmetic as make_end and arc_geo, in a fixed order).
template <typename T>
__device__ __forceinline__ T dot_rn(V3<T> a, V3<T> b) {
  return fma_rn(a.z, b.z, fma_rn(a.y, b.y, mul_rn(a.x, b.x)));
}
template <typename T>
__device__ __forceinline__ V3<T> cross_rn(V3<T> a, V3<T> b) {
  return mk3(fma_rn(a.y, b.z, -mul_rn(a.z, b.y)), fma_rn(a.z, b.x, -mul_rn(a.x, b.z)),
             fma_rn(a.x, b.y, -mul_rn(a.y, b.x)));
}
template <typename T>
__device__ __forceinline__ V3<T> scale_rn(V3<T> a, T k) {
  return mk3(mul_rn(a.x, k), mul_rn(a.y, k), mul_rn(a.z, k));
}
template <typename T>
struct EndRn {
  V3<T> u, e1, e2;
  T s, co;
};
template <typename T>
__device__ __forceinline__ EndRn<T> end_rn(const LatDev<T>& L, int64_t node, int32_t end_id) {
  const int32_t strut = end_id >> 1;
  const int32_t a = L.ends[2 * (int64_t)strut], b = L.ends[2 * (int64_t)strut + 1];
  const int32_t far = (end_id & 1) ? a : b, lo = a < b ? a : b, hi = a < b ? b : a;
  const V3<T> d = mk3(add_rn(L.xyz[3 * (int64_t)hi], -L.xyz[3 * (int64_t)lo]),
                      add_rn(L.xyz[3 * (int64_t)hi + 1], -L.xyz[3 * (int64_t)lo + 1]),
                      add_rn(L.xyz[3 * (int64_t)hi + 2], -L.xyz[3 * (int64_t)lo + 2]));
  const T il = div_rn(T(1), lm_sqrt(dot_rn(d, d)));
  const V3<T> ue = scale_rn(d, il);
  EndRn<T> e;
  e.u = node == lo ? ue : scale_rn(ue, T(-1));
  e.s = mul_rn(add_rn(L.node_R[node], -L.node_R[far]), il);
  e.co = lm_sqrt(fma_rn(-e.s, e.s, T(1)));
  const int ax = frame_axis(L, lo, hi);
  const V3<T> c1 = cross_rn(ue, mk3<T>(ax == 0, ax == 1, ax == 2));
  e.e1 = scale_rn(c1, div_rn(T(1), lm_sqrt(dot_rn(c1, c1))));
  e.e2 = cross_rn(ue, e.e1);
  return e;
}
template <typename T>
__device__ __forceinline__ ArcGeo<T> node_arc_geo(const LatDev<T>& L, int64_t node, int32_t oid, int32_t otid, T R) {
  const EndRn<T> o = end_rn<T>(L, node, oid);
  ArcGeo<T> g;
  g.u = o.u;
  g.e1 = o.e1;
  g.e2 = o.e2;
  g.Rs = mul_rn(R, o.s);
  g.Rco = mul_rn(R, o.co);
  g.co = o.co;
  g.s = o.s;
  if (otid >= 0) {
    const EndRn<T> t = end_rn<T>(L, node, otid);
    const T a1 = dot_rn(t.u, o.e1), a2 = dot_rn(t.u, o.e2);
    // n0 = R (s_o c - s_t) and d0 = co_t - co_o c (c = u_o.u_t) without the
    // cancellation of nearly parallel struts: 1 - c = |u_o - u_t|^2 / 2 and
    // co_t - co_o = (s_o - s_t)(s_o + s_t) / (co_o + co_t), each accurate
    // relative to its own size
    const V3<T> w = mk3(add_rn(o.u.x, -t.u.x), add_rn(o.u.y, -t.u.y), add_rn(o.u.z, -t.u.z));
    const T h = mul_rn(T(0.5), dot_rn(w, w));
    const T ds = add_rn(o.s, -t.s);
    const T dco = div_rn(mul_rn(ds, add_rn(o.s, t.s)), add_rn(o.co, t.co));
    g.n0 = mul_rn(R, fma_rn(-o.s, h, ds));
    g.n1 = mul_rn(g.Rco, a1);
    g.n2 = mul_rn(g.Rco, a2);
    g.d0 = fma_rn(o.co, h, dco);
    g.d1 = mul_rn(o.s, a1);
    g.d2 = mul_rn(o.s, a2);
  } else {
    g.n0 = g.n1 = g.n2 = T(0);
    g.d0 = T(1);
    g.d1 = g.d2 = T(0);
  }
  return g;
}

// ------------------------------------------------------- strut stitching
// Per-warp shared workspace for one strut (dynamic size from pmax, emax).
template <typename T>
struct EntryS {
  ArcGeo<T> g;
  T phi0, dphi, psi;
  int N, pre;
  int64_t ga;
  uint8_t rev, own;
};

// node-relative point s of an entry and its angle around the own strut (T);
// shared by the strut and hole kernels so shared points are bit-identical
template <typename T>
__device__ __forceinline__ void entry_point(const TriArgs<T>& A, int64_t node, const EntryS<T>& e,
                                            const EndG<T>* own, int s, V3<T>& z, T& th) {
  int m = e.rev ? e.N - s : s;
  if (s == 0 || m == 0 || m == e.N) {
    uint32_t av = A.arc_vtx[e.ga];
    int64_t vi = A.vtx_off[node] + (m == 0 ? (av & 255) : ((av >> 8) & 255));
    z = mk3(A.vtx_z[3 * vi], A.vtx_z[3 * vi + 1], A.vtx_z[3 * vi + 2]);
    th = e.psi;
    if (s != 0 && own) th = e.psi + wrap_from(raw_angle(*own, z) - e.psi, T(-ETA_PHI));
    return;
  }
  T phi;
  z = arc_point_rn(e.g, e.phi0, e.dphi, m, e.N, phi);
  if (e.own) th = phi;
  else if (own) th = e.psi + wrap_from(raw_angle(*own, z) - e.psi, T(-ETA_PHI));
  else th = T(0);
}

// STL record of triangle (a, b, c): relative points (to centre o) for the
// normal, area and volume; absolute points pa, pb, pc for the record
template <typename T>
__device__ __forceinline__ void stl_record(unsigned char* dst, V3<T> o, V3<T> ra, V3<T> rb, V3<T> rc,
                                           V3<T> pa, V3<T> pb, V3<T> pc, double* area, double* vol) {
  V3<T> cr = cross(rb - ra, rc - ra);
  T len = norm3(cr);
  V3<T> nn = len > T(0) ? cr * (T(1) / len) : mk3(T(0), T(0), T(0));
  if (dst) {
    float f[12] = {(float)nn.x, (float)nn.y, (float)nn.z, (float)pa.x, (float)pa.y, (float)pa.z,
                   (float)pb.x, (float)pb.y, (float)pb.z, (float)pc.x, (float)pc.y, (float)pc.z};
    uint16_t* d16 = reinterpret_cast<uint16_t*>(dst);
    const uint16_t* s16 = reinterpret_cast<const uint16_t*>(f);
#pragma unroll
    for (int q = 0; q < 24; q++) d16[q] = s16[q];
    d16[24] = 0;
  }
  *area = 0.5 * (double)len;
  *vol = ((double)dot(ra, cross(rb, rc)) + dot(mk3((double)o.x, (double)o.y, (double)o.z),
                                               mk3((double)cr.x, (double)cr.y, (double)cr.z))) /
         6.0;
}

// copy `nbytes` (even) from shared staging to global dst (2-byte aligned):
// 2-byte head/tail, 16-byte body
__device__ __forceinline__ void flush_stage(unsigned char* gdst, const unsigned char* st, int nbytes,
                                            int lane, int width = 32) {
  uintptr_t ga = (uintptr_t)gdst;
  int head = (int)((16 - (ga & 15)) & 15);
  if (head > nbytes) head = nbytes;
  head &= ~1;
  for (int q = lane; q < head / 2; q += width)
    reinterpret_cast<uint16_t*>(gdst)[q] = reinterpret_cast<const uint16_t*>(st)[q];
  int body = ((nbytes - head) / 16) * 16;
  for (int q = lane; q < body / 16; q += width) {
    const uint16_t* s = reinterpret_cast<const uint16_t*>(st + head + 16 * q);
    uint4 v;
    v.x = (uint32_t)s[0] | ((uint32_t)s[1] << 16);
    v.y = (uint32_t)s[2] | ((uint32_t)s[3] << 16);
    v.z = (uint32_t)s[4] | ((uint32_t)s[5] << 16);
    v.w = (uint32_t)s[6] | ((uint32_t)s[7] << 16);
    reinterpret_cast<uint4*>(gdst + head)[q] = v;
  }
  int tail = nbytes - head - body;
  for (int q = lane; q < tail / 2; q += width)
    reinterpret_cast<uint16_t*>(gdst + head + body)[q] =
        reinterpret_cast<const uint16_t*>(st + head + body)[q];
}

// ------------------------------------------- thread-per-strut stitching
// One thread per strut: the strut's two loops are walked by iterators that
// compute each subdivision point once, and the zipper runs exactly as the
// FP64 reference does.  Records are staged per lane in shared memory and
// leave in aligned groups of 8 (400 bytes = 25 x 16-byte stores).

// FP64 angle of loop point s of arc ga around own end `own_eid` (rare path)
template <typename T>
__device__ __noinline__ double theta64_thread(const TriArgs<T>& A, int64_t node, int32_t own_eid, int64_t ga,
                                              int N, int rev, int s) {
  const LatDev<T>& L = A.lat;
  int64_t b = L.row_ptr[node];
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255;
  int o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
  int64_t vo = A.vtx_off[node];
  double R = (double)L.node_R[node];
  EndG<double> me = make_end<T, double>(L, node, own_eid);
  EndG<double> Eo = make_end<T, double>(L, node, L.adj[b + o]);
  V3<double> z0 = vertex_pos64(L, node, A.vtx_gen[vo + v0]);
  V3<double> z1 = v1 == v0 ? z0 : vertex_pos64(L, node, A.vtx_gen[vo + v1]);
  double a0 = norm_angle(raw_angle(Eo, z0)), a1 = norm_angle(raw_angle(Eo, z1));
  double dd = a1 - a0;
  if (v0 == v1) dd = PI2;
  else if (dd <= 0.0) dd += PI2;
  V3<double> zs = rev ? z1 : z0;
  double psi = norm_angle(raw_angle(me, zs));
  if (s == 0) return psi;
  int m = rev ? N - s : s;
  double phi = a0 + dd * (double)m / (double)N;
  if (Eo.end_id == own_eid) return phi;
  double c, sn;
  sincos(phi, &sn, &c);
  double t = 0.0;
  if (ot >= 0) {
    EndG<double> Et = make_end<T, double>(L, node, L.adj[b + ot]);
    t = hval(Eo, Et, c, sn, R);
  }
  V3<double> z = surf_point(Eo, c, sn, t, R);
  return psi + wrap_from(raw_angle(me, z) - psi, -ETA_PHI);
}

// exact segment count of arc ga (rare path)
template <typename T>
__device__ __noinline__ int segments64_thread(const TriArgs<T>& A, int64_t node, int64_t ga) {
  const LatDev<T>& L = A.lat;
  int64_t b = L.row_ptr[node];
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255, o = (av >> 16) & 255;
  int64_t vo = A.vtx_off[node];
  EndG<double> Eo = make_end<T, double>(L, node, L.adj[b + o]);
  double dd = PI2;
  if (v0 != v1) {
    double a0 = norm_angle(raw_angle(Eo, vertex_pos64(L, node, A.vtx_gen[vo + v0])));
    double a1 = norm_angle(raw_angle(Eo, vertex_pos64(L, node, A.vtx_gen[vo + v1])));
    dd = a1 - a0;
    if (dd <= 0.0) dd += PI2;
  }
  bool u;
  return seg_count<double>(dd, A.k, u);
}

template <typename T>
struct LoopIt {
  int64_t node, q0, ao;
  int32_t eid;
  int ne;
  T R;
  V3<T> me1, me2;  // own frame
  // current entry
  int q, s, N;
  uint8_t rev, own;
  int64_t ga;
  T phi0, dphi, psi;
  ArcGeo<T>* g;  // per-thread slot in shared memory
};

template <typename T>
__device__ __forceinline__ int it_segments(const TriArgs<T>& A, const LoopIt<T>& it, int64_t ga) {
  bool unc;
  int N = seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
  if (unc) N = segments64_thread<T>(A, it.node, ga);
  return N;
}

template <typename T>
__device__ __noinline__ void it_load(const TriArgs<T>& A, LoopIt<T>& it, int q) {
  const LatDev<T>& L = A.lat;
  it.q = q;
  it.s = 0;
  uint32_t en = A.loop_ent[it.q0 + q];
  it.ga = it.ao + (en & 0x7fffffffu);
  it.rev = (uint8_t)(en >> 31);
  uint32_t av = A.arc_vtx[it.ga];
  int o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
  it.phi0 = A.arc_phi[2 * it.ga];
  it.dphi = A.arc_phi[2 * it.ga + 1];
  it.N = it_segments(A, it, it.ga);
  int64_t b = L.row_ptr[it.node];
  int32_t oid = L.adj[b + o];
  *it.g = node_arc_geo<T>(L, it.node, oid, ot >= 0 ? L.adj[b + ot] : -1, it.R);
  it.own = (oid == it.eid);
  if (it.own && !it.rev) {
    it.psi = it.phi0;
  } else {
    int vs = it.rev ? ((av >> 8) & 255) : (av & 255);
    int64_t vi = A.vtx_off[it.node] + vs;
    V3<T> zs = mk3(A.vtx_z[3 * vi], A.vtx_z[3 * vi + 1], A.vtx_z[3 * vi + 2]);
    T a = lm_atan2(dot(zs, it.me2), dot(zs, it.me1));
    if (sizeof(T) == 4 && fabs(a + T(PHI_CUT)) <= T(M_ANG)) {
      EndG<double> me = make_end<T, double>(L, it.node, it.eid);
      a = (T)norm_angle(raw_angle(me, vertex_pos64(L, it.node, A.vtx_gen[vi])));
    }
    it.psi = norm_angle(a);
  }
}

template <typename T>
__device__ void it_init(const TriArgs<T>& A, LoopIt<T>& it, int64_t node, int32_t eid, ArcGeo<T>* slot) {
  const LatDev<T>& L = A.lat;
  it.g = slot;
  it.node = node;
  it.eid = eid;
  it.q0 = A.end_off[eid];
  it.ne = (int)(A.end_off[eid + 1] - it.q0);
  it.ao = A.arc_off[node];
  it.R = L.node_R[node];
  EndG<T> me = make_end<T, T>(L, node, eid);
  it.me1 = me.e1;
  it.me2 = me.e2;
  it_load(A, it, 0);
}

// current point of the iterator (node-relative) and its own-frame angle
template <typename T>
__device__ __forceinline__ void it_point(const TriArgs<T>& A, const LoopIt<T>& it, V3<T>& z, T& th) {
  int m = it.rev ? it.N - it.s : it.s;
  if (it.s == 0) {
    uint32_t av = A.arc_vtx[it.ga];
    int64_t vi = A.vtx_off[it.node] + (m == 0 ? (av & 255) : ((av >> 8) & 255));
    z = mk3(A.vtx_z[3 * vi], A.vtx_z[3 * vi + 1], A.vtx_z[3 * vi + 2]);
    th = it.psi;
    return;
  }
  T phi;
  z = arc_point_rn(*it.g, it.phi0, it.dphi, m, it.N, phi);
  if (it.own) th = phi;
  else th = it.psi + wrap_from(lm_atan2(dot(z, it.me2), dot(z, it.me1)) - it.psi, T(-ETA_PHI));
}

template <typename T>
__device__ __forceinline__ void it_next(const TriArgs<T>& A, LoopIt<T>& it) {
  if (++it.s >= it.N) it_load(A, it, it.q + 1 < it.ne ? it.q + 1 : 0);
}

template <typename T>
__device__ __forceinline__ double it_theta64(const TriArgs<T>& A, const LoopIt<T>& it) {
  return theta64_thread<T>(A, it.node, it.eid, it.ga, it.N, it.rev, it.s);
}

// 50-byte record into (2-byte aligned) shared memory
__device__ __forceinline__ void rec_store(unsigned char* dst, const float f[12]) {
  if (((uintptr_t)dst & 3) == 0) {
    uint32_t* d32 = reinterpret_cast<uint32_t*>(dst);
#pragma unroll
    for (int q = 0; q < 12; q++) d32[q] = __float_as_uint(f[q]);
    reinterpret_cast<uint16_t*>(dst)[24] = 0;
  } else {
    uint16_t* d16 = reinterpret_cast<uint16_t*>(dst);
#pragma unroll
    for (int q = 0; q < 12; q++) {
      uint32_t u = __float_as_uint(f[q]);
      d16[2 * q] = (uint16_t)(u & 0xffffu);
      d16[2 * q + 1] = (uint16_t)(u >> 16);
    }
    d16[24] = 0;
  }
}

// one record at any 2-byte aligned dst with 13 stores (12 words + 1
// halfword) whatever dst mod 4: at dst = 2 mod 4 the words pair the high half
// of value q with the low half of value q + 1
__device__ __forceinline__ void rec_store_any(unsigned char* dst, const float f[12]) {
  const bool odd = ((uintptr_t)dst & 2) != 0;
  uint32_t* w = reinterpret_cast<uint32_t*>(dst + (odd ? 2 : 0));
#pragma unroll
  for (int q = 0; q < 12; q++) {
    const uint32_t u = __float_as_uint(f[q]), un = q < 11 ? __float_as_uint(f[q + 1]) : 0u;
    w[q] = odd ? __byte_perm(u, un, 0x5432) : u;
  }
  *reinterpret_cast<uint16_t*>(odd ? dst : dst + 48) = odd ? (uint16_t)(__float_as_uint(f[0]) & 0xffffu) : (uint16_t)0;
}

// copy `nbytes` (even) staged at offset sh (even, < 16) of a 16-byte aligned
// shared buffer to global gdst, where gdst = sh mod 16: 16-byte loads and
// stores for the body, halfwords for the head and tail
__device__ __forceinline__ void flush_congruent(unsigned char* gdst, const unsigned char* st, int sh, int nbytes,
                                                int lane, int width) {
  const int end = sh + nbytes;
  const int cf = (sh + 15) >> 4, ce = end >> 4;  // full 16-byte chunks [cf, ce)
  if (cf >= ce) {
    for (int q = lane; q < nbytes / 2; q += width)
      reinterpret_cast<uint16_t*>(gdst)[q] = reinterpret_cast<const uint16_t*>(st + sh)[q];
    return;
  }
  for (int c = cf + lane; c < ce; c += width)
    *reinterpret_cast<uint4*>(gdst + 16 * c - sh) = *reinterpret_cast<const uint4*>(st + 16 * c);
  const int hh = (16 * cf - sh) >> 1, th = (end - 16 * ce) >> 1;
  for (int q = lane; q < hh + th; q += width) {
    const int off = q < hh ? sh + 2 * q : 16 * ce + 2 * (q - hh);
    *reinterpret_cast<uint16_t*>(gdst + off - sh) = *reinterpret_cast<const uint16_t*>(st + off);
  }
}

constexpr int REC_LANE_STRIDE = 404;  // 8 records + pad (odd word count: no bank conflicts)
// per-thread shared slot: the two loops' arc geometry (8-byte aligned for
// FP64), then 8 staged records; the stride is a multiple of 8 bytes with an
// odd number of 8-byte words
template <typename T>
__host__ __device__ constexpr int tri_geo_bytes() {
  return ((2 * (int)sizeof(ArcGeo<T>) + 15) / 16) * 16;
}
template <typename T>
__host__ __device__ constexpr int tri_lane_stride() {
  return (((tri_geo_bytes<T>() + 400 + 7) / 8) % 2 == 1) ? ((tri_geo_bytes<T>() + 400 + 7) / 8) * 8
                                                          : ((tri_geo_bytes<T>() + 400 + 7) / 8) * 8 + 8;
}

template <typename T, bool OBJ>
__global__ void __launch_bounds__(128, 3) k_tri_thread(TriArgs<T> A, const int64_t* first_ptr) {
  extern __shared__ __align__(16) unsigned char stage[];
  const int64_t out_first = first_ptr ? *first_ptr : 0;
  const LatDev<T>& L = A.lat;
  const int64_t E = L.n_struts;
  const int64_t e_end = A.item_end < E ? A.item_end : E;
  ArcGeo<T>* gslot = reinterpret_cast<ArcGeo<T>*>(stage + threadIdx.x * tri_lane_stride<T>());
  unsigned char* my = stage + threadIdx.x * tri_lane_stride<T>() + tri_geo_bytes<T>();
  const bool vec_ok = A.out && (((uintptr_t)A.out) & 15) == 0;
  double sa = 0.0, sv = 0.0;
  for (int64_t e = A.item_begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e_end;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = L.ends[2 * e], b = L.ends[2 * e + 1];
    int32_t lo = a < b ? a : b, hi = a < b ? b : a;
    int side_lo = (a == lo) ? 0 : 1;
    int32_t eA = (int32_t)(2 * e + side_lo), eB = (int32_t)(2 * e + 1 - side_lo);
    LoopIt<T> IA, IB;
    it_init(A, IA, lo, eA, gslot);
    it_init(A, IB, hi, eB, gslot + 1);
    // loop sizes
    int nA = 0, nB = 0;
    for (int q = 0; q < IA.ne; q++) nA += it_segments(A, IA, IA.ao + (A.loop_ent[IA.q0 + q] & 0x7fffffffu));
    for (int q = 0; q < IB.ne; q++) nB += it_segments(A, IB, IB.ao + (A.loop_ent[IB.q0 + q] & 0x7fffffffu));
    // A's first point (kept for the wrap)
    V3<T> a0z;
    T thA0;
    it_point(A, IA, a0z, thA0);
    double thA0_64 = 0.0;
    bool have_a0_64 = false;
    auto a0_64 = [&]() {
      if (!have_a0_64) {
        uint32_t en = A.loop_ent[IA.q0];
        int64_t ga0 = IA.ao + (en & 0x7fffffffu);
        thA0_64 = theta64_thread<T>(A, IA.node, IA.eid, ga0, 1, (int)(en >> 31), 0);
        have_a0_64 = true;
      }
      return thA0_64;
    };
    // key of a B point in the window [thA0 - ETA_ZIP, thA0 + 2pi - ETA_ZIP)
    auto keyB = [&](const LoopIt<T>& I, T th, bool& exact, double& k64) -> T {
      T x = wrap_from(th, thA0 - T(ETA_ZIP));
      exact = false;
      if (sizeof(T) == 4 && (x - (thA0 - T(ETA_ZIP)) <= T(M_ZIP) || thA0 + T(PI2 - ETA_ZIP) - x <= T(M_ZIP))) {
        k64 = wrap_from(it_theta64(A, I), a0_64() - ETA_ZIP);
        exact = true;
        x = (T)k64;
      }
      return x;
    };
    // rotation of B: its first key within ETA_PHI of the smallest (one pass
    // for the smallest key, one to find the start, keeping the point before
    // it; the whole loop when the start is point 0)
    V3<T> bprev = mk3(T(0), T(0), T(0));
    int sB = 0;
    {
      T kmin = T(0);
      for (int j = 0; j < nB; j++) {
        V3<T> z;
        T th;
        it_point(A, IB, z, th);
        bool ex;
        double k64;
        T kj = keyB(IB, th, ex, k64);
        if (j == 0 || kj < kmin) kmin = kj;
        it_next(A, IB);
      }
      it_load(A, IB, 0);
      bool found = false;
      for (int j = 0; j < nB; j++) {
        V3<T> z;
        T th;
        it_point(A, IB, z, th);
        bool ex;
        double k64;
        T kj = keyB(IB, th, ex, k64);
        if (!found && kj <= kmin + T(ETA_PHI)) {
          found = true;
          sB = j;
          if (j > 0) break;  // the iterator stays at the start point
        }
        bprev = z;
        it_next(A, IB);
      }
      if (sB == 0) it_load(A, IB, 0);  // bprev is the loop's last point
    }
    // zipper (ties advance A)
    const int64_t t0 = A.tri_off[e] - out_first;
    const int ntri = nA + nB;
    V3<T> cA = node_xyz<T, T>(L, lo), cB = node_xyz<T, T>(L, hi);
    V3<T> dAB = cB - cA;
    V3<T> acur = a0z, bcur = bprev;
    it_next(A, IA);
    V3<T> anext;
    T thAn;
    if (nA > 1) it_point(A, IA, anext, thAn);
    else { anext = a0z; thAn = thA0 + T(PI2); }
    int ia = 0, ib = -1;
    V3<T> bnext;
    T thBn;
    it_point(A, IB, bnext, thBn);
    bool exB;
    double kB64;
    T kBn = keyB(IB, thBn, exB, kB64);
    for (int t = 0; t < ntri; t++) {
      bool takeA;
      if (ib == nB - 1) takeA = true;
      else if (ia >= nA) takeA = false;
      else {
        T xa = ia + 1 < nA ? thAn : thA0 + T(PI2);
        if (sizeof(T) == 4 && fabs(xa - kBn - T(ETA_ZIP)) <= T(M_ZIP)) {
          double xa64 = ia + 1 < nA ? it_theta64(A, IA) : a0_64() + PI2;
          double kb = exB ? kB64 : wrap_from(it_theta64(A, IB), a0_64() - ETA_ZIP);
          takeA = xa64 <= kb + ETA_ZIP;
        } else {
          takeA = xa <= kBn + T(ETA_ZIP);
        }
      }
      V3<T> ra, rb, rc, pa, pb, pc;
      if (takeA) {
        ra = acur;
        rb = anext;
        rc = dAB + bcur;
        pa = cA + acur;
        pb = cA + anext;
        pc = cB + bcur;
        acur = anext;
        ia++;
        if (ia < nA) {
          it_next(A, IA);
          if (ia + 1 < nA) it_point(A, IA, anext, thAn);
          else { anext = a0z; thAn = thA0 + T(PI2); }
        }
      } else {
        ra = acur;
        rb = dAB + bnext;
        rc = dAB + bcur;
        pa = cA + acur;
        pb = cB + bnext;
        pc = cB + bcur;
        bcur = bnext;
        ib++;
        if (ib < nB - 1) {
          it_next(A, IB);
          it_point(A, IB, bnext, thBn);
          kBn = keyB(IB, thBn, exB, kB64);
        }
      }
      // record
      V3<T> cr = cross(rb - ra, rc - ra);
      T len = norm3(cr);
      V3<T> nn = len > T(0) ? cr * (T(1) / len) : mk3(T(0), T(0), T(0));
      if (OBJ) {
        sa += 0.5 * (double)len;
        sv += ((double)dot(ra, cross(rb, rc)) +
               dot(mk3((double)cA.x, (double)cA.y, (double)cA.z), mk3((double)cr.x, (double)cr.y, (double)cr.z))) *
              (1.0 / 6.0);
      }
      if (A.out) {
        int64_t u = t0 + t;
        int slot = (int)(u & 7);
        float f[12] = {(float)nn.x, (float)nn.y, (float)nn.z, (float)pa.x, (float)pa.y, (float)pa.z,
                       (float)pb.x, (float)pb.y, (float)pb.z, (float)pc.x, (float)pc.y, (float)pc.z};
        rec_store(my + 50 * slot, f);
        if (slot == 7 || t == ntri - 1) {
          int first_slot = (int)((u - (int64_t)(t < slot ? t : slot)) & 7);
          int nrec = slot - first_slot + 1;
          int64_t ustart = u - (nrec - 1);
          if (ustart + nrec > A.capacity) {
            atomicCAS(A.err, 0, 4);
          } else if (vec_ok && nrec == 8) {
            uint4* dst = reinterpret_cast<uint4*>(A.out + 50 * ustart);
            const uint32_t* src = reinterpret_cast<const uint32_t*>(my);
#pragma unroll 5
            for (int c = 0; c < 25; c++) dst[c] = make_uint4(src[4 * c], src[4 * c + 1], src[4 * c + 2], src[4 * c + 3]);
          } else {
            uint16_t* dst = reinterpret_cast<uint16_t*>(A.out + 50 * ustart);
            const uint16_t* src = reinterpret_cast<const uint16_t*>(my + 50 * first_slot);
            for (int c = 0; c < 25 * nrec; c++) dst[c] = src[c];
          }
        }
      }
    }
  }
  if (OBJ && A.acc) {
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(A.acc, sa);
      atomicAdd(A.acc + 1, sv);
    }
  }
}

// ------------------------------------------------ tile-per-strut stitching
// A tile of TL lanes (8 on the forward path: four struts per warp) stitches one strut.  The
// entries of both loops are set up lane-parallel (their arc geometry goes to
// shared memory), the loop points are evaluated lane-parallel, B's angles are
// moved into A's window and B is rotated to its smallest key, and then each
// lane emits two consecutive triangles per round, finding its place in the
// zipper by a merge-path search.  Records are staged per tile at their
// destination's offset mod 16 and stored with 16-byte vector stores.  Angle decisions that FP32 cannot take safely (keys within
// M_ZIP of each other or of the window edges) are retaken in FP64 from the
// exact vertex generators, recomputed per comparison (they are rare).
// x in [-n, 2n) moved into [0, n) (no integer division)
__device__ __forceinline__ int wrap_idx(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

template <typename T>
struct TileEntry {
  ArcGeo<T> g;
  T phi0, dphi, psi;
  int N, pre;
  int64_t ga;
  uint8_t rev, own, ill, pad1;  // ill: points subdivided in FP64 (arc_ill)
};

struct TileHdr {
  int np[2], ne[2];
  int li[2];     // local index of the strut's end at its lo / hi node (FP64 pass)
  int pad[2];
  double a0_64;  // FP64 angle of A's first point (when some key was flagged)
};

// consecutive triangles per lane and round of the zipper (one merge-path
// search per lane and round, then single comparisons)
constexpr int TILE_RPL = 2;

// per-tile shared memory: header, entries of both loops (the staging of
// TL * TILE_RPL records reuses them: they are dead once the points are evaluated), point
// angles of both loops (B's angles are overwritten by B's keys), point
// positions of both loops; the FP64 pass adds flags per point and its FP64
// data.  Smaller tiles mean more struts in flight per SM.
template <typename T, int TL>
struct TileLayout {
  __host__ __device__ static constexpr size_t r16c(size_t b) { return (b + 15) & ~(size_t)15; }
  int pmax, emax;
  bool exact;  // the FP64 pass also holds FP64 strut ends of both nodes, FP64 arc
               // data per entry and angles per point
  bool adjm;   // adjoint mode: point ids of both loops
  int dmax;    // largest node valence (FP64 strut ends)
  __host__ __device__ size_t ent() const { return r16c(sizeof(TileHdr)); }
  __host__ __device__ size_t ent_bytes() const {
    size_t e = 2 * (size_t)emax * sizeof(TileEntry<T>), st = (size_t)TL * TILE_RPL * 50 + 16;
    return r16c(e > st ? e : st);
  }
  __host__ __device__ size_t th() const { return ent() + ent_bytes(); }
  __host__ __device__ size_t kb() const { return th() + (size_t)pmax * sizeof(T); }
  __host__ __device__ size_t z() const { return th() + r16c(2 * (size_t)pmax * sizeof(T)); }
  __host__ __device__ size_t fl() const { return z() + r16c(2 * (size_t)pmax * sizeof(V3<T>)); }
  __host__ __device__ size_t stage() const { return ent(); }
  // flags per point (FP64 pass) or zipper decisions per triangle (sequential
  // zipper of the FP64 pass and of FP64 lattices)
  __host__ __device__ size_t ea64() const {
    return fl() + ((exact || sizeof(T) == 8) ? r16c(2 * (size_t)pmax) : 0);
  }
  __host__ __device__ size_t th64() const { return ea64() + (exact ? r16c(2 * (size_t)emax * 32) : 0); }
  __host__ __device__ size_t e64() const { return th64() + (exact ? r16c(2 * (size_t)pmax * 8) : 0); }
  __host__ __device__ size_t pid() const {
    return e64() + (exact ? r16c(2 * (size_t)dmax * sizeof(EndG<double>)) : 0);
  }
  __host__ __device__ size_t bytes() const { return pid() + (adjm ? r16c(2 * (size_t)pmax * 8) : 0); }
};

// FP64 data of one loop entry: start angle of its arc in the owner's frame,
// angular extent, and the angle of the entry's first point in the loop's frame
struct Arc64 {
  double a0, dd, psi, pad;
};

template <int TL>
__device__ __forceinline__ unsigned tile_mask(int lane) {
  return TL == 32 ? 0xffffffffu : (((1u << TL) - 1u) << (lane & ~(TL - 1)));
}
template <int TL>
__device__ __forceinline__ int tile_excl_scan(int x, int tl, unsigned m) {
  int v = x;
#pragma unroll
  for (int o = 1; o < TL; o <<= 1) {
    int t = __shfl_up_sync(m, v, o, TL);
    if (tl >= o) v += t;
  }
  return v - x;
}

// entry of point p of a loop (entries hold the exclusive prefix of points)
template <typename T>
__device__ __forceinline__ int tile_entry_of(const TileEntry<T>* ents, int ne, int p) {
  int lq = 0, hq = ne - 1;
  while (lq < hq) {
    int mid = (lq + hq + 1) >> 1;
    if (ents[mid].pre <= p) lq = mid;
    else hq = mid - 1;
  }
  return lq;
}

// FP64 arc data of entry (ga, rev) of the loop of local end `li` (rare
// path); E: the node's strut ends in FP64 (shared memory)
template <typename T>
__device__ __noinline__ Arc64 arc64_data(const TriArgs<T>& A, const EndG<double>* E, int64_t node, int li,
                                         int64_t ga, int rev) {
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255, o = (av >> 16) & 255;
  int64_t vo = A.vtx_off[node];
  double R = (double)A.lat.node_R[node];
  V3<double> z0 = gen_point<double>(E, R, A.vtx_gen[vo + v0]);
  V3<double> z1 = v1 == v0 ? z0 : gen_point<double>(E, R, A.vtx_gen[vo + v1]);
  Arc64 r;
  r.a0 = norm_angle(raw_angle(E[o], z0));
  double a1 = norm_angle(raw_angle(E[o], z1));
  r.dd = a1 - r.a0;
  if (v0 == v1) r.dd = PI2;
  else if (r.dd <= 0.0) r.dd += PI2;
  r.psi = norm_angle(raw_angle(E[li], rev ? z1 : z0));
  r.pad = 0.0;
  return r;
}

// FP64 angle of point s of an entry from its FP64 arc data (rare path)
template <typename T>
__device__ __noinline__ double point64_theta(const TriArgs<T>& A, const EndG<double>* E, int64_t node, int li,
                                             int64_t ga, const Arc64& d, int N, int rev, int s) {
  if (s == 0) return d.psi;
  uint32_t av = A.arc_vtx[ga];
  int o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
  int m = rev ? N - s : s;
  double phi = d.a0 + d.dd * (double)m / (double)N;
  if (o == li) return phi;
  double R = (double)A.lat.node_R[node];
  double c, sn;
  sincos(phi, &sn, &c);
  double t = ot >= 0 ? hval(E[o], E[ot], c, sn, R) : 0.0;
  V3<double> z = surf_point(E[o], c, sn, t, R);
  return d.psi + wrap_from(raw_angle(E[li], z) - d.psi, -ETA_PHI);
}

// FP64 position of subdivision point m of N of arc ga (node-relative), from
// the FP64 strut ends E of its node (rare path: ill-conditioned arcs)
template <typename T>
__device__ __noinline__ V3<double> point64_pos(const TriArgs<T>& A, const EndG<double>* E, int64_t node,
                                               int64_t ga, int N, int m) {
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255, o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
  int64_t vo = A.vtx_off[node];
  double R = (double)A.lat.node_R[node];
  V3<double> z0 = gen_point<double>(E, R, A.vtx_gen[vo + v0]);
  V3<double> z1 = v1 == v0 ? z0 : gen_point<double>(E, R, A.vtx_gen[vo + v1]);
  double a0 = norm_angle(raw_angle(E[o], z0)), a1 = norm_angle(raw_angle(E[o], z1));
  double dd = a1 - a0;
  if (v0 == v1) dd = PI2;
  else if (dd <= 0.0) dd += PI2;
  double phi = a0 + dd * (double)m / (double)N, c, sn;
  sincos(phi, &sn, &c);
  double t = ot >= 0 ? hval(E[o], E[ot], c, sn, R) : 0.0;
  return surf_point(E[o], c, sn, t, R);
}

// exact segment count of arc ga (rare path; E as above)
template <typename T>
__device__ __noinline__ int segments64_cached(const TriArgs<T>& A, const EndG<double>* E, int64_t node,
                                              int64_t ga) {
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255, o = (av >> 16) & 255;
  int64_t vo = A.vtx_off[node];
  double R = (double)A.lat.node_R[node];
  double dd = PI2;
  if (v0 != v1) {
    double a0 = norm_angle(raw_angle(E[o], gen_point<double>(E, R, A.vtx_gen[vo + v0])));
    double a1 = norm_angle(raw_angle(E[o], gen_point<double>(E, R, A.vtx_gen[vo + v1])));
    dd = a1 - a0;
    if (dd <= 0.0) dd += PI2;
  }
  bool u;
  return seg_count<double>(dd, A.k, u);
}

// Set up one loop entry (arc geometry, start angle, segment count) in shared
// memory.  EXACT: decisions that FP32 cannot take safely are retaken in FP64.
// Otherwise an uncertain start angle returns -1 (the strut is deferred) and an
// uncertain segment count returns the FP32 count with SEG_UNC set (the caller
// settles it from the strut's exact triangle count, or defers the strut).
constexpr int SEG_UNC = 1 << 29;
template <typename T, bool EXACT>
__device__ __forceinline__ int tile_entry_setup_impl(const TriArgs<T>& A, int64_t node, int32_t eid, int64_t qi,
                                                     TileEntry<T>* dst, V3<T>& z0, const EndG<double>* E64 = nullptr,
                                                     int li = 0) {
  const LatDev<T>& L = A.lat;
  const int64_t ao = A.arc_off[node], rb = L.row_ptr[node], vo = A.vtx_off[node];
  const T R = L.node_R[node];
  constexpr bool IS64 = sizeof(T) == 8;
  TileEntry<T> en;
  uint32_t ent = A.loop_ent[qi];
  en.ga = ao + (ent & 0x7fffffffu);
  en.rev = (uint8_t)(ent >> 31);
  en.ill = en.pad1 = 0;
  uint32_t av = A.arc_vtx[en.ga];
  int o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
  // the entry's first vertex in loop order (its first point)
  const int64_t vi = vo + (en.rev ? ((av >> 8) & 255) : (av & 255));
  z0 = mk3(A.vtx_z[3 * vi], A.vtx_z[3 * vi + 1], A.vtx_z[3 * vi + 2]);
  en.phi0 = A.arc_phi[2 * en.ga];
  en.dphi = A.arc_phi[2 * en.ga + 1];
  bool unc;
  int Nq = seg_count<T>(en.dphi, A.k, unc);
  if (EXACT && unc) Nq = segments64_cached<T>(A, E64, node, en.ga);
  int32_t oid = L.adj[rb + o];
  en.g = node_arc_geo<T>(L, node, oid, ot >= 0 ? L.adj[rb + ot] : -1, R);
  en.own = (oid == eid);
  // an ill-conditioned elliptical arc is subdivided in FP64 (FP64 pass; both
  // struts of the arc take this decision from the same bits)
  if (!IS64 && ot >= 0 && arc_ill<T>(en.g, en.phi0, en.dphi)) {
    if (!EXACT) return -2;
    en.ill = 1;
  }
  if (en.own && !en.rev) {
    en.psi = en.phi0;
  } else {
    EndG<T> own = make_end<T, T>(L, node, eid);
    T ang = raw_angle(own, z0);
    if (!IS64 && fabs(ang + T(PHI_CUT)) <= T(M_ANG)) {
      if (!EXACT) return -1;
      ang = (T)norm_angle(raw_angle(E64[li], gen_point<double>(E64, (double)R, A.vtx_gen[vi])));
    }
    en.psi = norm_angle(ang);
  }
  en.N = Nq;
  en.pre = 0;
  *dst = en;
  return (!EXACT && unc) ? (Nq | SEG_UNC) : Nq;
}

template <typename T>
__device__ __noinline__ int tile_entry_setup_exact(const TriArgs<T>& A, int64_t node, int32_t eid, int64_t qi,
                                                   TileEntry<T>* dst, V3<T>& z0, const EndG<double>* E64, int li) {
  return tile_entry_setup_impl<T, true>(A, node, eid, qi, dst, z0, E64, li);
}

template <typename T, int TL>
struct TileSmem {
  TileHdr* H;
  TileEntry<T>* ENT;
  T* TH;
  V3<T>* Z;
  T* KB;
  uint8_t* FL;
  unsigned char* STG;
  Arc64* EA64;
  double* TH64;
  EndG<double>* E64;
  int64_t* PID;
  __device__ TileSmem(unsigned char* base, const TileLayout<T, TL>& Lay)
      : H(reinterpret_cast<TileHdr*>(base)),
        ENT(reinterpret_cast<TileEntry<T>*>(base + Lay.ent())),
        TH(reinterpret_cast<T*>(base + Lay.th())),
        Z(reinterpret_cast<V3<T>*>(base + Lay.z())),
        KB(reinterpret_cast<T*>(base + Lay.kb())),
        FL(reinterpret_cast<uint8_t*>(base + Lay.fl())),
        STG(base + Lay.stage()),
        EA64(reinterpret_cast<Arc64*>(base + Lay.ea64())),
        TH64(reinterpret_cast<double*>(base + Lay.th64())),
        E64(reinterpret_cast<EndG<double>*>(base + Lay.e64())),
        PID(reinterpret_cast<int64_t*>(base + Lay.pid())) {}
};

// Point adjoints of one triangle (a, b, c relative to any common origin; n =
// (b - a) x (c - a), nh = n / |n|): each corner p gets
// w_area dA/dp + w_vol n / 6 with dA/da = (b - c) x nh / 2 (cyclically).
template <typename T>
__device__ __forceinline__ void tri_point_adjoints(const TriArgs<T>& A, V3<T> a, V3<T> b, V3<T> c, V3<T> nh,
                                                   V3<T> n, int64_t pa, int64_t pb, int64_t pc) {
  const T wa = T(0.5) * (T)A.w_area, wv = (T)A.w_vol / T(6);
  V3<T> g[3] = {cross(b - c, nh) * wa + n * wv, cross(c - a, nh) * wa + n * wv, cross(a - b, nh) * wa + n * wv};
  int64_t id[3] = {pa, pb, pc};
#pragma unroll
  for (int q = 0; q < 3; q++) {
    atomicAdd(A.adj + 3 * id[q], g[q].x);
    atomicAdd(A.adj + 3 * id[q] + 1, g[q].y);
    atomicAdd(A.adj + 3 * id[q] + 2, g[q].z);
  }
}

// Stitch strut e with one tile.  Returns true (uniformly over the tile) when
// the strut needs FP64 decisions and EXACT is off: nothing was written then.
template <typename T, int TL, bool OBJ, bool EXACT, bool ADJ = false>
__device__ __forceinline__ bool tile_strut(const TriArgs<T>& A, const TileSmem<T, TL>& S, int64_t e,
                                           int64_t out_first, int tl, unsigned m, bool vec_ok, double& sa,
                                           double& sv) {
  constexpr bool IS64 = sizeof(T) == 8;
  constexpr bool FP64_STEPS = EXACT && !IS64;
  const LatDev<T>& L = A.lat;
  TileHdr* H = S.H;
  TileEntry<T>* ENT = S.ENT;
  T* TH = S.TH;
  V3<T>* Z = S.Z;
  T* KB = S.KB;
  uint8_t* FL = S.FL;
  int32_t a = L.ends[2 * e], b = L.ends[2 * e + 1];
  int32_t lo = a < b ? a : b, hi = a < b ? b : a;
  int side_lo = (a == lo) ? 0 : 1;
  const int32_t eA = (int32_t)(2 * e + side_lo), eB = (int32_t)(2 * e + 1 - side_lo);
  bool ok = true, defer = false;
  if constexpr (FP64_STEPS) {
    // FP64 strut ends of both nodes, once per strut (every FP64 step below
    // reads them), and the local index of the strut's end at each node
    const int64_t rb0 = L.row_ptr[lo], rb1 = L.row_ptr[hi];
    const int d0 = (int)(L.row_ptr[lo + 1] - rb0), d1 = (int)(L.row_ptr[hi + 1] - rb1);
    if (d0 > A.dmax || d1 > A.dmax) {
      if (tl == 0) atomicCAS(A.err, 0, 4);
      return false;
    }
    for (int q = tl; q < d0 + d1; q += TL) {
      int X = q < d0 ? 0 : 1, li = X == 0 ? q : q - d0;
      int64_t node = X == 0 ? lo : hi;
      int32_t eid = L.adj[(X == 0 ? rb0 : rb1) + li];
      S.E64[X * A.dmax + li] = make_end<T, double>(L, node, eid);
      if (eid == (X == 0 ? eA : eB)) H->li[X] = li;
    }
    __syncwarp(m);
  }
  // ---- entries of both loops, set up together (lanes over the entries of
  // loop A, then of loop B, so the dependent loads of both overlap)
  {
    const int64_t qa = A.end_off[eA], qb = A.end_off[eB];
    const int neA0 = (int)(A.end_off[eA + 1] - qa), neB0 = (int)(A.end_off[eB + 1] - qb);
    if (neA0 < 1 || neA0 > A.emax || neB0 < 1 || neB0 > A.emax) ok = false;
    int cnt[2] = {0, 0};
    int nunc = 0, uncX = 0, uncQ = 0;  // entries with an uncertain segment count
    const int net = neA0 + neB0;
    for (int c0 = 0; c0 < net && ok; c0 += TL) {
      int q = c0 + tl;
      int Nq = 0, X = 0, qq = q;
      V3<T> z0 = mk3(T(0), T(0), T(0));
      if (q >= neA0) {
        X = 1;
        qq = q - neA0;
      }
      if (q < net) {
        int64_t node = X == 0 ? lo : hi;
        int32_t eid = X == 0 ? eA : eB;
        int64_t qi = (X == 0 ? qa : qb) + qq;
        if (FP64_STEPS)
          Nq = tile_entry_setup_exact<T>(A, node, eid, qi, ENT + X * A.emax + qq, z0, S.E64 + X * A.dmax, H->li[X]);
        else Nq = tile_entry_setup_impl<T, false>(A, node, eid, qi, ENT + X * A.emax + qq, z0);
      }
      if (__any_sync(m, Nq < 0)) {
        tfb_add(A.fb, __any_sync(m, Nq == -2) ? 17 : 12, tl == 0, m);
        defer = true;
        break;
      }
      if (!EXACT) {
        const unsigned ub = __ballot_sync(m, (Nq & SEG_UNC) != 0) >> (TL == 32 ? 0 : (threadIdx.x & 31 & ~(TL - 1)));
        if (ub) {
          nunc += __popc(ub);
          const int qu = c0 + __ffs(ub) - 1;
          uncX = qu < neA0 ? 0 : 1;
          uncQ = qu < neA0 ? qu : qu - neA0;
        }
        Nq &= ~SEG_UNC;
      }
      // per-loop exclusive prefix: scan the round's loop-A and loop-B counts
      // separately (loop B's entries follow loop A's in lane order)
      int nA_ = X == 0 ? Nq : 0, nB_ = X == 1 ? Nq : 0;
      int pa = tile_excl_scan<TL>(nA_, tl, m), pb = tile_excl_scan<TL>(nB_, tl, m);
      if (q < net) {
        // the entry's first point is its first vertex (the points pass skips it)
        const int pre = X == 0 ? cnt[0] + pa : cnt[1] + pb;
        ENT[X * A.emax + qq].pre = pre;
        if (pre < A.pmax) {
          Z[X * A.pmax + pre] = z0;
          TH[X * A.pmax + pre] = ENT[X * A.emax + qq].psi;
        }
      }
      cnt[0] += __shfl_sync(m, pa + nA_, TL - 1, TL);
      cnt[1] += __shfl_sync(m, pb + nB_, TL - 1, TL);
    }
    if (!EXACT && !defer && ok && nunc > 0) {
      // the count pass decided every segment count exactly: with one
      // uncertain entry, the strut's triangle count (points of both loops)
      // fixes it; with more the strut is deferred
      const int diff = (int)(A.tri_off[e + 1] - A.tri_off[e]) - (cnt[0] + cnt[1]);
      __syncwarp(m);
      TileEntry<T>* eu = ENT + uncX * A.emax + uncQ;
      if (nunc > 1 || diff < -1 || diff > 1 || eu->N + diff < 1) {
        tfb_add(A.fb, 12, tl == 0, m);
        defer = true;
      } else if (diff != 0) {
        const int neX = uncX == 0 ? neA0 : neB0;
        for (int q = uncQ + 1 + tl; q < neX; q += TL) ENT[uncX * A.emax + q].pre += diff;
        if (tl == 0) eu->N += diff;
        __syncwarp(m);
        if (tl == 0) {
          // the first points of the later entries move by diff (in the order
          // that reads each before it is overwritten)
          for (int r = 0; r < neX - uncQ - 1; r++) {
            const int q = diff > 0 ? neX - 1 - r : uncQ + 1 + r;
            const int pn = ENT[uncX * A.emax + q].pre, po = pn - diff;
            if (pn >= 0 && pn < A.pmax && po >= 0 && po < A.pmax) {
              Z[uncX * A.pmax + pn] = Z[uncX * A.pmax + po];
              TH[uncX * A.pmax + pn] = TH[uncX * A.pmax + po];
            }
          }
        }
        cnt[uncX] += diff;
      }
    }
    if (cnt[0] > A.pmax || cnt[1] > A.pmax) ok = false;
    if (tl == 0) {
      H->ne[0] = neA0;
      H->ne[1] = neB0;
      H->np[0] = cnt[0];
      H->np[1] = cnt[1];
    }
  }
  if (defer) return true;
  __syncwarp(m);
  if (!ok) {
    if (tl == 0) atomicCAS(A.err, 0, 4);
    return false;
  }
  const int nA = H->np[0], nB = H->np[1];
  const int neA = H->ne[0], neB = H->ne[1];
  // ---- points of both loops, lanes over the points of A then of B (the
  // strut frame e1, e2 -- all raw_angle reads -- is the same at both ends)
  {
    const EndG<T> own = make_end<T, T>(L, lo, eA);
    for (int q = tl; q < nA + nB; q += TL) {
      const int X = q < nA ? 0 : 1, p = X == 0 ? q : q - nA;
      const int64_t node = X == 0 ? lo : hi;
      const int ne = X == 0 ? neA : neB;
      const TileEntry<T>* ents = ENT + X * A.emax;
      const TileEntry<T>& en = ents[tile_entry_of(ents, ne, p)];
      int sidx = p - en.pre;
      int mm = en.rev ? en.N - sidx : sidx;
      if (sidx != 0) {
        T phi;
        V3<T> zz = arc_point_rn(en.g, en.phi0, en.dphi, mm, en.N, phi);
        if constexpr (FP64_STEPS) {
          if (en.ill) {
            const V3<double> z64 = point64_pos<T>(A, S.E64 + X * A.dmax, node, en.ga, en.N, mm);
            zz = mk3((T)z64.x, (T)z64.y, (T)z64.z);
          }
        }
        Z[X * A.pmax + p] = zz;
        TH[X * A.pmax + p] = en.own ? phi : en.psi + wrap_from(raw_angle(own, zz) - en.psi, T(-ETA_PHI));
      }
      if (FP64_STEPS) FL[X * A.pmax + p] = 0;
      if constexpr (ADJ) {
        uint32_t av = A.arc_vtx[en.ga];
        S.PID[X * A.pmax + p] = sidx == 0 ? A.vtx_off[node] + (mm == 0 ? (av & 255) : ((av >> 8) & 255))
                                          : A.n_vtx + A.arc_pt_off[en.ga] + mm - 1;
      }
    }
  }
  __syncwarp(m);
  const T thA0 = TH[0];
  // ---- B keys in A's window [thA0 - ETA_ZIP, thA0 + 2pi - ETA_ZIP)
  bool any = false;
  for (int j = tl; j < nB; j += TL) {
    T x = wrap_from(TH[A.pmax + j], thA0 - T(ETA_ZIP));
    KB[j] = x;
    if (!IS64 && (x - (thA0 - T(ETA_ZIP)) <= T(M_ZIP) || thA0 + T(PI2 - ETA_ZIP) - x <= T(M_ZIP))) {
      if (FP64_STEPS) FL[A.pmax + j] = 2;  // window edge: key retaken in FP64
      any = true;
    }
  }
  if (!IS64 && !EXACT && __any_sync(m, any)) {
    tfb_add(A.fb, 13, tl == 0, m);
    return true;
  }
  __syncwarp(m);
  // B starts at its first key within ETA_PHI of the smallest (ties: loop
  // order); kmin receives the smallest key
  T kmin = T(0);
  auto rotation = [&]() {
    T mn = T(1e30);
    for (int j = tl; j < nB; j += TL) mn = fmin(mn, KB[j]);
#pragma unroll
    for (int o = TL / 2; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(m, mn, o, TL));
    kmin = mn;
    int first = 0x7fffffff;
    for (int j = tl; j < nB; j += TL)
      if (KB[j] <= mn + T(ETA_PHI)) first = min(first, j);
#pragma unroll
    for (int o = TL / 2; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(m, first, o, TL));
    return first == 0x7fffffff ? 0 : first;
  };
  int sB = rotation();
  // The merge-path placement below equals the oracle's sequential zipper only
  // when A's angles and B's rotated keys are both non-decreasing.  On
  // degenerate nodes (sections past a strut's length, steep sections) a loop
  // can turn back in angle: the FP32 pass defers such a strut, and the FP64
  // pass and FP64 lattices run the sequential zipper instead.
  // In FP32 a second key within M_ZIP of the smallest makes the rotation
  // uncertain: it is taken like out-of-order keys, from FP64 keys.
  bool unsorted = false;
  {
    bool u = false;
    int near_min = 0;
    for (int i = tl; i < nA; i += TL)
      if ((i + 1 < nA ? TH[i + 1] : thA0 + T(PI2)) < TH[i]) u = true;
    for (int j = tl; j + 1 < nB; j += TL)
      if (KB[wrap_idx(sB + j + 1, nB)] < KB[wrap_idx(sB + j, nB)]) u = true;
    if (!IS64)
      for (int j = tl; j < nB; j += TL) near_min += KB[j] <= kmin + T(M_ZIP);
#pragma unroll
    for (int o = TL / 2; o > 0; o >>= 1) near_min += __shfl_xor_sync(m, near_min, o, TL);
    unsorted = __any_sync(m, u) || near_min > 1;
  }
  if (!IS64 && !EXACT && unsorted) {
    tfb_add(A.fb, 16, tl == 0, m);
    return true;
  }
  // FP32 strut pass (no adjoint): the comparisons that decide the zipper are
  // checked against the margin where the emission makes them (see below)
  constexpr bool FOLD = !IS64 && !EXACT && !ADJ;
  if (!IS64 && !unsorted && !FOLD) {
    // A points whose angle lies within M_ZIP of some B key + ETA_ZIP: every
    // such pair is decided in FP64 (B keys are sorted after the rotation up
    // to FP32 rounding, so each scan stops at the first key clearly out of
    // range)
    for (int i = tl; i <= nA; i += TL) {
      if (i == 0) continue;
      T x = (i < nA ? TH[i] : thA0 + T(PI2)) - T(ETA_ZIP);
      int lj = 0, hj = nB;
      while (lj < hj) {
        int mid = (lj + hj) >> 1;
        if (KB[wrap_idx(sB + mid, nB)] < x) lj = mid + 1;
        else hj = mid;
      }
      bool hit = false;
      for (int jj = lj - 1; jj >= lj - nB; jj--) {
        int jr = wrap_idx(jj, nB);
        T kv = KB[wrap_idx(sB + jr, nB)] - (jj < 0 ? T(PI2) : T(0));
        if (kv < x - T(2 * M_ZIP)) break;
        if (fabs(kv - x) <= T(M_ZIP)) {
          if (FP64_STEPS) FL[A.pmax + wrap_idx(sB + jr, nB)] |= 1;
          hit = true;
        }
      }
      for (int jj = lj; jj < lj + nB; jj++) {
        int jr = wrap_idx(jj, nB);
        T kv = KB[wrap_idx(sB + jr, nB)] + (jj >= nB ? T(PI2) : T(0));
        if (kv > x + T(2 * M_ZIP)) break;
        if (fabs(kv - x) <= T(M_ZIP)) {
          if (FP64_STEPS) FL[A.pmax + wrap_idx(sB + jr, nB)] |= 1;
          hit = true;
        }
      }
      if (hit) {
        if (FP64_STEPS) FL[i < nA ? i : 0] |= 1;
        any = true;
      }
    }
  }
  const bool anyt = !IS64 && __any_sync(m, any);
  if (!EXACT && anyt) {
    tfb_add(A.fb, 14, tl == 0, m);
    return true;
  }
  if (FP64_STEPS) tfb_add(A.fb, 10, (anyt || unsorted) && tl == 0, m);
  if (FP64_STEPS && (anyt || unsorted)) {
    // out of order: every key is taken in FP64 for the sequential zipper
    if (unsorted) {
      for (int p = tl; p < nA; p += TL) FL[p] = 1;
      for (int j = tl; j < nB; j += TL) FL[A.pmax + j] = 1;
      __syncwarp(m);
    }
    // A's first point fixes the window: always taken in FP64 here
    if (tl == 0) FL[0] |= 4;
    __syncwarp(m);
    // FP64 arc data of every entry that holds a flagged point, then the FP64
    // angle of every flagged point, each computed once
    for (int X = 0; X < 2; X++) {
      int64_t node = X == 0 ? lo : hi;
      int32_t eid = X == 0 ? eA : eB;
      int ne = X == 0 ? neA : neB;
      const TileEntry<T>* ents = ENT + X * A.emax;
      for (int q = tl; q < ne; q += TL) {
        bool need = false;
        for (int p = ents[q].pre; p < ents[q].pre + ents[q].N && !need; p++) need = FL[X * A.pmax + p] != 0;
        if (need)
          S.EA64[X * A.emax + q] = arc64_data<T>(A, S.E64 + X * A.dmax, node, H->li[X], ents[q].ga, ents[q].rev);
      }
    }
    __syncwarp(m);
    for (int X = 0; X < 2; X++) {
      int64_t node = X == 0 ? lo : hi;
      int32_t eid = X == 0 ? eA : eB;
      int np = X == 0 ? nA : nB, ne = X == 0 ? neA : neB;
      const TileEntry<T>* ents = ENT + X * A.emax;
      for (int p = tl; p < np; p += TL) {
        if (!FL[X * A.pmax + p]) continue;
        int q = tile_entry_of(ents, ne, p);
        S.TH64[X * A.pmax + p] = point64_theta<T>(A, S.E64 + X * A.dmax, node, H->li[X], ents[q].ga,
                                                  S.EA64[X * A.emax + q], ents[q].N,
                                                  ents[q].rev, p - ents[q].pre);
      }
    }
    __syncwarp(m);
    const double a0 = S.TH64[0];
    // B keys of flagged points in FP64; window-edge keys replace the FP32
    // ones, then B is rotated again
    for (int j = tl; j < nB; j += TL) {
      uint8_t f = FL[A.pmax + j];
      if (!f) continue;
      double x64 = wrap_from(S.TH64[A.pmax + j], a0 - ETA_ZIP);
      S.TH64[A.pmax + j] = x64;
      if (f & 2) KB[j] = (T)x64;
    }
    __syncwarp(m);
    if (A.fb && !unsorted) {
      // pairs of keys decided in FP64 (within M_ZIP of the tie band's edge)
      int pairs = 0;
      for (int i = tl + 1; i <= nA; i += TL) {
        if (!FL[i < nA ? i : 0]) continue;
        double x = (i < nA ? S.TH64[i] : a0 + PI2) - ETA_ZIP;
        for (int j = 0; j < nB; j++)
          if (FL[A.pmax + j] && fabs(S.TH64[A.pmax + j] - x) <= M_ZIP) pairs++;
      }
      if (pairs) atomicAdd(A.fb + 15, (unsigned long long)pairs);
    }
    __syncwarp(m);
    if (unsorted) {
      // B rotated to its first smallest FP64 key
      double mn = 1e300;
      for (int j = tl; j < nB; j += TL) mn = fmin(mn, S.TH64[A.pmax + j]);
#pragma unroll
      for (int o = TL / 2; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(m, mn, o, TL));
      int first = 0x7fffffff;
      for (int j = tl; j < nB; j += TL)
        if (S.TH64[A.pmax + j] <= mn + ETA_PHI) first = min(first, j);
#pragma unroll
      for (int o = TL / 2; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(m, first, o, TL));
      sB = first == 0x7fffffff ? 0 : first;
    } else {
      sB = rotation();
    }
  }
  const double a0_64 = FP64_STEPS && (anyt || unsorted) ? S.TH64[0] : 0.0;
  const int ntri = nA + nB;
  if (unsorted) {
    // sequential zipper (the oracle's process; ties advance A): the decision
    // of each triangle goes to FL, and lanes place their triangles by prefix
    // counts of the decisions
    if (tl == 0) {
      auto keyA = [&](int i) -> double {
        if constexpr (FP64_STEPS) return i < nA ? S.TH64[i] : a0_64 + PI2;
        else return i < nA ? (double)TH[i] : (double)thA0 + PI2;
      };
      auto keyB = [&](int j) -> double {
        const int jb = wrap_idx(sB + j, nB);
        if constexpr (FP64_STEPS) return S.TH64[A.pmax + jb];
        else return (double)KB[jb];
      };
      int ia = 0, ib = -1;
      for (int p = 0; p < ntri; p++) {
        bool takeA;
        if (ib == nB - 1) takeA = true;
        else if (ia >= nA) takeA = false;
        else takeA = keyA(ia + 1) <= keyB(ib + 1) + ETA_ZIP;
        FL[p] = takeA ? 1 : 0;
        if (takeA) ia++;
        else ib++;
      }
    }
    __syncwarp(m);
  }
  // In the FOLD pass every comparison the placement searches and the walks
  // make is checked against the margin M_ZIP, and a strut with one inside it
  // is deferred to the FP64 pass after its records are written (that pass
  // writes the same range again).  When every comparison made is outside the
  // margin, each has the outcome the FP64 keys give, so the searches and
  // walks follow the FP64 path exactly: this replaces a check of every A-B
  // pair by a check of the pairs that decide the output.
  bool near = false;
  auto a_before_b = [&](int i, int j) -> bool {
    int jb = wrap_idx(sB + j, nB);
    if (FP64_STEPS && anyt && FL[i < nA ? i : 0] && FL[A.pmax + jb]) {
      double x = i < nA ? S.TH64[i] : a0_64 + PI2;
      return x <= S.TH64[A.pmax + jb] + ETA_ZIP;
    }
    T x = i < nA ? TH[i] : thA0 + T(PI2);
    const T y = KB[jb] + T(ETA_ZIP);
    if (FOLD) near |= fabs(x - y) <= T(M_ZIP);
    return x <= y;
  };
  // ---- triangles by merge-path; TL * RPL records per round
  constexpr int RPL = TILE_RPL;
  const int64_t t0 = A.tri_off[e] - out_first;
  V3<T> cA = node_xyz<T, T>(L, lo), cB = node_xyz<T, T>(L, hi);
  V3<T> dAB = cB - cA;
  double sa_s = 0.0, sv_s = 0.0;  // this strut's area and volume terms
  int ibase = 0;  // A events before position c0 (carried from round to round)
  for (int c0 = 0; c0 < ntri; c0 += TL * RPL) {
    const int p = c0 + RPL * tl;  // this lane's first position
    // records staged at the global destination's offset mod 16 (out is
    // 16-byte aligned: 50 t = 2 t mod 16)
    const int sh = vec_ok ? (int)((2 * (t0 + c0)) & 15) : 0;
    int i = ibase;
    if (unsorted) {
      // A events before this lane's first position, from the decisions
      int na_ = 0;
#pragma unroll
      for (int r = 0; r < RPL; r++)
        if (p + r < ntri) na_ += FL[p + r];
      i = ibase + tile_excl_scan<TL>(na_, tl, m);
    }
    if (p < ntri) {
      if (!unsorted) {
        // i = A events among the first p (ties -> A first); i(p) - i(c0) is
        // between 0 and p - c0, so the search spans at most RPL TL + 1 values
        int li_ = p - nB > ibase ? p - nB : ibase, hi_ = ibase + RPL * tl;
        if (hi_ > nA) hi_ = nA;
        while (li_ < hi_) {
          int mid = (li_ + hi_) >> 1;
          if (a_before_b(mid + 1, p - mid - 1)) li_ = mid + 1;
          else hi_ = mid;
        }
        i = li_;
      }
#pragma unroll
      for (int r = 0; r < RPL; r++) {
        if (p + r >= ntri) break;
        const int jn = p + r - i;
        const bool isA = unsorted ? FL[p + r] != 0 : (i < nA) && (jn == nB || a_before_b(i + 1, jn));
        int jp = wrap_idx(sB + jn - 1, nB);
        V3<T> za = Z[i < nA ? i : 0];
        V3<T> zp = Z[A.pmax + jp];
        V3<T> q1 = isA ? Z[i + 1 < nA ? i + 1 : 0] : Z[A.pmax + wrap_idx(sB + jn, nB)];
        V3<T> ra = za, rb = isA ? q1 : dAB + q1, rc = dAB + zp;
        V3<T> pa = cA + za, pb = isA ? cA + q1 : cB + q1, pc = cB + zp;
        V3<T> cr = cross(rb - ra, rc - ra);
        const T l2 = dot(cr, cr);
        // unit normal (one reciprocal square root; the record's normal is
        // informative, its error bound is far above 2 ulp)
        V3<T> nn = l2 > T(0) ? cr * lm_rsqrt(l2) : mk3(T(0), T(0), T(0));
        if constexpr (ADJ) {
          int64_t ia_ = S.PID[i < nA ? i : 0];
          int64_t ib_ = isA ? S.PID[i + 1 < nA ? i + 1 : 0] : S.PID[A.pmax + wrap_idx(sB + jn, nB)];
          int64_t ic_ = S.PID[A.pmax + jp];
          tri_point_adjoints<T>(A, ra, rb, rc, nn, cr, ia_, ib_, ic_);
        } else {
          if (OBJ) {
            sa_s += 0.5 * (double)lm_sqrt(l2);
            sv_s += ((double)dot(ra, cross(rb, rc)) +
                   dot(mk3((double)cA.x, (double)cA.y, (double)cA.z), mk3((double)cr.x, (double)cr.y, (double)cr.z))) *
                  (1.0 / 6.0);
          }
          if (A.out) {
            float f[12] = {(float)nn.x, (float)nn.y, (float)nn.z, (float)pa.x, (float)pa.y, (float)pa.z,
                           (float)pb.x, (float)pb.y, (float)pb.z, (float)pc.x, (float)pc.y, (float)pc.z};
            rec_store_any(S.STG + sh + 50 * (RPL * tl + r), f);
          }
        }
        i += isA ? 1 : 0;
      }
    }
    const int npos = ntri - c0 < TL * RPL ? ntri - c0 : TL * RPL;
    // the lane holding this round's last position fixes the next round's base
    ibase = __shfl_sync(m, i, (npos - 1) / RPL, TL);
    __syncwarp(m);
    if (!ADJ && A.out) {
      const int nrec = npos;
      int64_t gt = t0 + c0;
      if (gt + nrec <= A.capacity) {
        if (vec_ok) flush_congruent(A.out + 50 * gt, S.STG, sh, 50 * nrec, tl, TL);
        else {
          uint16_t* d16 = reinterpret_cast<uint16_t*>(A.out + 50 * gt);
          const uint16_t* s16 = reinterpret_cast<const uint16_t*>(S.STG);
          for (int q = tl; q < 25 * nrec; q += TL) d16[q] = s16[q];
        }
      } else if (tl == 0) {
        atomicCAS(A.err, 0, 4);
      }
    }
    __syncwarp(m);
  }
  if constexpr (FOLD) {
    if (__any_sync(m, near)) {
      tfb_add(A.fb, 14, tl == 0, m);
      return true;
    }
  }
  if (OBJ) {
    sa += sa_s;
    sv += sv_s;
  }
  return false;
}

// Strut pass.  EXACT off: every strut of [item_begin, min(item_end, E)) is
// stitched in the kernel's precision, and a strut that needs an FP64 stability
// step is marked in `redo` (bit e - redo_base) instead.  EXACT on: only the
// marked struts are stitched, with the FP64 steps.
template <typename T, int TL, bool OBJ, bool EXACT, bool ADJ = false>
__global__ void __launch_bounds__(EXACT ? 64 : 128, EXACT ? 4 : 7)
    k_tri_tiles(TriArgs<T> A, const int64_t* first_ptr, uint32_t* redo, int64_t redo_base) {
  if (A.range) {
    A.item_begin = A.range[0];
    A.item_end = A.range[1];
  }
  const int64_t out_first = A.range ? A.tri_off[A.item_begin] : (first_ptr ? *first_ptr : 0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int tl = lane & (TL - 1);
  const unsigned m = tile_mask<TL>(lane);
  const int tile_in_block = threadIdx.x / TL;
  const int64_t gtile = (int64_t)blockIdx.x * (blockDim.x / TL) + tile_in_block;
  const int64_t ntiles = (int64_t)gridDim.x * (blockDim.x / TL);
  TileLayout<T, TL> Lay{A.pmax, A.emax, EXACT, ADJ, A.dmax};
  TileSmem<T, TL> S(smem_raw + (size_t)tile_in_block * Lay.bytes(), Lay);
  const int64_t E = A.lat.n_struts;
  const int64_t e_end = A.item_end < E ? A.item_end : E;
  const bool vec_ok = A.out && (((uintptr_t)A.out) & 15) == 0;
  double sa = 0.0, sv = 0.0;
  if (!EXACT) {
    for (int64_t e = A.item_begin + gtile; e < e_end; e += ntiles) {
      bool d = tile_strut<T, TL, OBJ, false, ADJ>(A, S, e, out_first, tl, m, vec_ok, sa, sv);
      if (d && tl == 0) {
        atomicOr(redo + ((e - redo_base) >> 5), 1u << ((e - redo_base) & 31));
        if (A.rlist) {
          unsigned long long q = atomicAdd(A.rlist, 1ull);
          if (q < (unsigned long long)A.rcap) A.rlist[1 + q] = (unsigned long long)e;
        }
      }
    }
  } else {
    const unsigned long long nl = A.rlist ? A.rlist[0] : 0ull;
    if (A.rlist && nl <= (unsigned long long)A.rcap) {
      // the listed struts, dealt round-robin over the tiles
      for (int64_t i = gtile; i < (int64_t)nl; i += ntiles)
        tile_strut<T, TL, OBJ, true, ADJ>(A, S, (int64_t)A.rlist[1 + i], out_first, tl, m, vec_ok, sa, sv);
    } else {
      // marked struts dealt round-robin over the tiles (marks cluster in space)
      for (int64_t e = A.item_begin + gtile; e < e_end; e += ntiles) {
        if (!((redo[(e - redo_base) >> 5] >> ((e - redo_base) & 31)) & 1u)) continue;
        tile_strut<T, TL, OBJ, true, ADJ>(A, S, e, out_first, tl, m, vec_ok, sa, sv);
      }
    }
  }
  if (OBJ && A.acc) {
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sv += __shfl_xor_sync(0xffffffffu, sv, o);
    }
    if (lane == 0) {
      atomicAdd(A.acc, sa);
      atomicAdd(A.acc + 1, sv);
    }
  }
}

// ------------------------------------------------ chunks replayed by graph
// First node of a chunk graph: the next chunk of this graph's sequence
// (cursor[0], stepped by `stride`) as a device-side item range.
static __global__ void k_chunk_begin(int64_t* cursor, int64_t stride, int64_t chunk, int64_t i0, int64_t i1,
                                     int64_t* range) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t c = cursor[0];
    int64_t b = i0 + c * chunk, e = b + chunk;
    range[0] = b < i1 ? b : i1;
    range[1] = e < i1 ? e : i1;
    cursor[0] = c + stride;
  }
}

// Clear the deferral bitmap words of the struts of a device-side range, and
// the deferral list.
static __global__ void k_redo_clear(const int64_t* range, uint32_t* redo, int64_t base, int64_t n_struts,
                                    unsigned long long* rlist) {
  if (rlist && blockIdx.x == 0 && threadIdx.x == 0) rlist[0] = 0ull;
  int64_t b = range[0], e = range[1] < n_struts ? range[1] : n_struts;
  if (e <= b) return;
  int64_t w0 = (b - base) >> 5, w1 = (e - base + 31) >> 5;
  for (int64_t w = w0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < w1; w += (int64_t)gridDim.x * blockDim.x)
    redo[w] = 0u;
}

// ---------------------------------------------------------- hole fans
// Per-warp shared workspace of the hole kernel: contour points (both
// contours of a band), 32 staged records, FP64 angles or keys of the points,
// and the band's stitching steps.
template <typename T>
__host__ __device__ constexpr size_t holes_ws_q(int pmax) { return (((size_t)pmax * sizeof(V3<T>)) + 15) & ~(size_t)15; }
__host__ __device__ constexpr size_t holes_ws_stage() { return (32 * 50 + 64 + 15) & ~(size_t)15; }
template <typename T>
__host__ __device__ constexpr size_t holes_ws_bytes(int pmax) {
  return holes_ws_q<T>(pmax) + holes_ws_stage() + (((size_t)pmax * 8 + 15) & ~(size_t)15) +
         (((size_t)pmax * 4 + 15) & ~(size_t)15);
}

// Contour points of hole h (node-relative, hole order) into Q[0, cap), lanes
// over each entry's points; returns the contour's point count (points past
// cap are not stored).
template <typename T>
__device__ int hole_contour(const TriArgs<T>& A, int64_t nd, int64_t h, int64_t ao, int64_t rb, T R, Node64* ctx,
                            V3<T>* Q, int cap, int lane) {
  const LatDev<T>& L = A.lat;
  int M = 0;
  for (int64_t q = A.hole_off[h]; q < A.hole_off[h + 1]; q++) {
    uint32_t ent = A.hole_ent[q];
    int64_t ga = ao + (ent & 0x7fffffffu);
    int rev = ent >> 31;
    bool unc;
    int Nq = seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
    if (unc) {  // the same for every lane of the warp
      if (ctx->node != nd) {
        load_node64(L, nd, ctx, lane);
        __syncwarp();
      }
      Nq = arc_segments<T>(A, nd, ga, ctx, 0);
    }
    EntryS<T> en;
    en.g = node_arc_geo<T>(L, nd, L.adj[rb + ((A.arc_vtx[ga] >> 16) & 255)], -1, R);
    en.phi0 = A.arc_phi[2 * ga];
    en.dphi = A.arc_phi[2 * ga + 1];
    en.psi = T(0);
    en.N = Nq;
    en.pre = M;
    en.ga = ga;
    en.rev = (uint8_t)rev;
    en.own = 1;
    for (int s = lane; s < Nq; s += 32) {
      V3<T> z;
      T th;
      if (M + s < cap) {
        entry_point<T>(A, nd, en, nullptr, s, z, th);
        Q[M + s] = z;
      }
    }
    M += Nq;
  }
  return M;
}

// FP64 point s of a hole entry (circular arc ga, owner end o; arc angles a0,
// dd from arc_dphi64) from the node's FP64 strut ends (rare paths)
template <typename T>
__device__ __forceinline__ V3<double> hole_point64(const TriArgs<T>& A, const Node64* ctx, int64_t ga, int rev,
                                                   int Nq, double a0, double dd, int s) {
  const uint32_t av = A.arc_vtx[ga];
  const int o = (av >> 16) & 255;
  const int64_t vo = A.vtx_off[ctx->node];
  const int m = rev ? Nq - s : s;
  if (m == 0) return vertex_from_gen<double>(ctx->E, ctx->d, ctx->R, A.vtx_gen[vo + (av & 255)]);
  if (m == Nq) return vertex_from_gen<double>(ctx->E, ctx->d, ctx->R, A.vtx_gen[vo + ((av >> 8) & 255)]);
  double ph = a0 + dd * (double)m / (double)Nq, cs, sn;
  sincos(ph, &sn, &cs);
  return surf_point(ctx->E[o], cs, sn, 0.0, ctx->R);
}

// Stitching of an annular band (reading 10) from the angles K[0, M0) of
// contour 0 and K[M0, M0 + M1) of contour 1 around the band's axis (both in
// hole order, FP64): checks that contour 0 turns once positively and contour
// 1 once negatively, turns K into the zipper keys (contour 0 relative to its
// first point; contour 1 moved into [th0 - ETA_ZIP, th0 + 2pi - ETA_ZIP), in
// place), rotates contour 1 backward to its smallest key (ties within
// ETA_PHI: the first) and writes the decision of each triangle p to DEC[p]
// (ia << 1 | contour-0 advances).  Returns contour 1's start sB, or -1 when a
// contour does not turn once.  Called by the whole warp.
__device__ __forceinline__ int band_zip(double* K, int M0, int M1, int32_t* DEC, int lane) {
  double t0 = 0.0, t1 = 0.0;
  const double HP = 0.5 * PI2;
  for (int i = lane; i < M0; i += 32) {
    double r = K[i + 1 < M0 ? i + 1 : 0] - K[i];
    while (r <= -HP) r += PI2;
    while (r > HP) r -= PI2;
    t0 += r;
  }
  for (int j = lane; j < M1; j += 32) {
    double r = K[M0 + (j + 1 < M1 ? j + 1 : 0)] - K[M0 + j];
    while (r <= -HP) r += PI2;
    while (r > HP) r -= PI2;
    t1 += r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    t0 += __shfl_xor_sync(0xffffffffu, t0, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
  }
  if (fabs(t0 - PI2) > 1e-6 || fabs(t1 + PI2) > 1e-6) return -1;
  const double th0 = K[0];
  __syncwarp();
  for (int i = lane; i < M0; i += 32) {
    double r = K[i] - th0;
    while (r < -ETA_PHI) r += PI2;
    while (r >= PI2 - ETA_PHI) r -= PI2;
    K[i] = th0 + r;
  }
  double kmin = 1e300;
  for (int x = lane; x < M1; x += 32) {
    double v = K[M0 + x];
    while (v < th0 - ETA_ZIP) v += PI2;
    while (v >= th0 + PI2 - ETA_ZIP) v -= PI2;
    K[M0 + x] = v;
    kmin = fmin(kmin, v);
  }
  for (int o = 16; o > 0; o >>= 1) kmin = fmin(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
  __syncwarp();
  int sB = 0x7fffffff;
  for (int x = lane; x < M1; x += 32)
    if (K[M0 + x] <= kmin + ETA_PHI) sB = min(sB, (M1 - x) % M1);
  for (int o = 16; o > 0; o >>= 1) sB = min(sB, __shfl_xor_sync(0xffffffffu, sB, o));
  if (lane == 0) {
    int ia = 0, ib = -1;
    for (int p = 0; p < M0 + M1; p++) {
      const int xb = M0 + (M1 - ((sB + ib + 1 + M1) % M1)) % M1;
      const bool takeA = (ib == M1 - 1) || (ia < M0 && (ia + 1 < M0 ? K[ia + 1] : th0 + PI2) <= K[xb] + ETA_ZIP);
      DEC[p] = (ia << 1) | (takeA ? 1 : 0);
      if (takeA) ia++;
      else ib++;
    }
  }
  __syncwarp();
  return sB;
}

// position in the contour arrays of point j of contour 1 backward from its
// start sB (j >= -1)
__device__ __forceinline__ int band_bpos(int M0, int M1, int sB, int j) {
  return M0 + (M1 - ((sB + j + M1) % M1)) % M1;
}

// Annular exposed component of node nd (reading 10): two contours bounding
// one component of the nodal sphere are stitched as a band like a strut's
// lateral band: q0 = hole h0 forward, q1 = hole h0 + 1 backward, both in the
// angle around the axis from q0's barycentre to q1's (frame: e1 = a x E_ax
// with ax the axis of smallest |a_ax|, ties lowest; e2 = a x e1); q0 starts
// at its first point, q1's keys are moved into [th0 - ETA_ZIP,
// th0 + 2pi - ETA_ZIP) and q1 starts at its smallest key (ties within
// ETA_PHI: the first); an event of q0 comes first unless it exceeds q1's by
// more than ETA_ZIP.  Every decision is taken in FP64 from points recomputed
// from the inputs; the records use the FP32 contour points, which the struts
// share bit for bit.  Returns the triangles emitted, -1 when the band does
// not apply (barycentres within ETA_BARY R, or a contour that does not turn
// once around the axis: the holes are fanned), -2 on a capacity error.
template <typename T>
__device__ __noinline__ int band_node(const TriArgs<T>& A, int64_t nd, int64_t h0, V3<T> c, T R, int64_t ao,
                                      int64_t rb, Node64* ctx, V3<T>* Q, double* K, int32_t* DEC,
                                      unsigned char* stage, int64_t tbase, int lane, double& sa, double& sv) {
  const LatDev<T>& L = A.lat;
  const int M0 = hole_contour<T>(A, nd, h0, ao, rb, R, ctx, Q, A.pmax, lane);
  const int M1 = hole_contour<T>(A, nd, h0 + 1, ao, rb, R, ctx, Q + (M0 < A.pmax ? M0 : A.pmax),
                                 A.pmax - M0, lane);
  if (M0 < 1 || M1 < 1) return -1;
  if (M0 + M1 > A.pmax) {
    if (lane == 0) atomicCAS(A.err, 0, 4);
    return -2;
  }
  if (ctx->node != nd) load_node64(L, nd, ctx, lane);
  __syncwarp();
  // FP64 points: barycentres (pass 0), then angles around the axis (pass 1)
  V3<double> ax_ = mk3(0.0, 0.0, 0.0), e1 = ax_, e2 = ax_;
  for (int pass = 0; pass < 2; pass++) {
    V3<double> bs[2] = {mk3(0.0, 0.0, 0.0), mk3(0.0, 0.0, 0.0)};
    int p = 0;
    for (int cc = 0; cc < 2; cc++) {
      for (int64_t q = A.hole_off[h0 + cc]; q < A.hole_off[h0 + cc + 1]; q++) {
        const uint32_t ent = A.hole_ent[q];
        const int64_t ga = ao + (ent & 0x7fffffffu);
        const int rev = ent >> 31;
        const int Nq = arc_segments<T>(A, nd, ga, ctx, 0);
        double a0;
        const double dd = arc_dphi64(A, ctx, ga, &a0);
        for (int s = lane; s < Nq; s += 32) {
          const V3<double> z = hole_point64<T>(A, ctx, ga, rev, Nq, a0, dd, s);
          if (pass == 0) bs[cc] = bs[cc] + z;
          else K[p + s] = atan2(dot(z, e2), dot(z, e1));
        }
        p += Nq;
      }
    }
    if (pass == 0) {
      for (int cc = 0; cc < 2; cc++)
        for (int o = 16; o > 0; o >>= 1) {
          bs[cc].x += __shfl_xor_sync(0xffffffffu, bs[cc].x, o);
          bs[cc].y += __shfl_xor_sync(0xffffffffu, bs[cc].y, o);
          bs[cc].z += __shfl_xor_sync(0xffffffffu, bs[cc].z, o);
        }
      const V3<double> a = bs[1] * (1.0 / (double)M1) - bs[0] * (1.0 / (double)M0);
      const double al = norm3(a);
      if (!(al > ETA_BARY * ctx->R)) return -1;
      ax_ = a * (1.0 / al);
      const double aa[3] = {fabs(ax_.x), fabs(ax_.y), fabs(ax_.z)};
      int ax = 0;
      if (aa[1] < aa[ax]) ax = 1;
      if (aa[2] < aa[ax]) ax = 2;
      const V3<double> c1 = cross(ax_, mk3<double>(ax == 0, ax == 1, ax == 2));
      e1 = c1 * (1.0 / norm3(c1));
      e2 = cross(ax_, e1);
    }
  }
  __syncwarp();
  const int sB = band_zip(K, M0, M1, DEC, lane);
  if (sB < 0) return -1;
  auto bpos = [&](int j) { return band_bpos(M0, M1, sB, j); };
  const int ntri = M0 + M1;
  for (int c0 = 0; c0 < ntri; c0 += 32) {
    const int p = c0 + lane;
    if (p < ntri) {
      const int v = DEC[p], ia = v >> 1, ib = p - ia - 1;
      const V3<T> ra = Q[ia % M0];
      const V3<T> rb = (v & 1) ? Q[(ia + 1) % M0] : Q[bpos(ib + 1)];
      const V3<T> rc = Q[bpos(ib)];
      double ar, vo;
      stl_record<T>(A.out ? stage + 50 * lane : nullptr, c, ra, rb, rc, c + ra, c + rb, c + rc, &ar, &vo);
      sa += ar;
      sv += vo;
    }
    __syncwarp();
    if (A.out) {
      const int nrec = ntri - c0 < 32 ? ntri - c0 : 32;
      const int64_t gt = tbase + c0;
      if (gt + nrec <= A.capacity) flush_stage(A.out + 50 * gt, stage, 50 * nrec, lane);
      else if (lane == 0) atomicCAS(A.err, 0, 4);
    }
    __syncwarp();
  }
  return ntri;
}

// ---------------------------------------------------------- hole fans
// One warp per node with holes: for each hole, the contour points (circular arcs in
// hole order), their barycentre b, b_project = o + R (b - o)/|b - o| (Section
// 5), falling back to the direction away from the struts when b sits at the
// centre or outside the hole region; fan triangles (b_project, q_m, q_m+1).
template <typename T>
__global__ void __launch_bounds__(256) k_tri_holes(TriArgs<T> A, Node64* scratch,
                                                    const int64_t* first_ptr) {
  if (A.range) {
    A.item_begin = A.range[0];
    A.item_end = A.range[1];
  }
  const int64_t out_first = A.range ? A.tri_off[A.item_begin] : (first_ptr ? *first_ptr : 0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  unsigned char* base = smem_raw + (size_t)w * holes_ws_bytes<T>(A.pmax);
  V3<T>* Q = reinterpret_cast<V3<T>*>(base);
  unsigned char* stage = base + holes_ws_q<T>(A.pmax);
  double* K = reinterpret_cast<double*>(stage + holes_ws_stage());
  int32_t* DEC = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(K) +
                                            ((((size_t)A.pmax * 8) + 15) & ~(size_t)15));
  Node64* ctx = scratch + 2 * gw;
  const LatDev<T>& L = A.lat;
  const int64_t E = L.n_struts;
  constexpr bool IS64 = sizeof(T) == 8;
  const int64_t n0 = (A.item_begin > E ? A.item_begin : E) - E;
  const int64_t n1 = A.item_end - E;
  // nodes are taken from the queue 32 at a time (most have no hole: one
  // atomic per node would bound the kernel by the counter's throughput); a
  // group is 32 nodes `stride` apart, so that runs of consecutive nodes with
  // holes (a face of the lattice) spread over many groups
  const int64_t stride = (n1 - n0 + 31) / 32;
  unsigned todo = 0;
  int64_t g0 = 0;
  while (true) {
    if (!todo) {
      if (lane == 0) g0 = atomicAdd(A.queue, 1);
      g0 = __shfl_sync(0xffffffffu, g0, 0);
      if (g0 >= stride) break;
      const int64_t mine = n0 + g0 + lane * stride;
      todo = __ballot_sync(0xffffffffu, mine < n1 && A.node_hole_off[mine] != A.node_hole_off[mine + 1] &&
                                            (!A.node_mask || A.node_mask[mine]));
      if (!todo) continue;
    }
    const int64_t nd = n0 + g0 + (__ffs(todo) - 1) * stride;
    todo &= todo - 1;
    int64_t h0 = A.node_hole_off[nd], h1 = A.node_hole_off[nd + 1];
    int64_t ao = A.arc_off[nd];
    int64_t rb = L.row_ptr[nd];
    int d = (int)(L.row_ptr[nd + 1] - rb);
    T R = L.node_R[nd];
    V3<T> c = node_xyz<T, T>(L, nd);
    int64_t tbase = A.tri_off[E + nd] - out_first;
    double sa = 0.0, sv = 0.0;
    // two contours bounding one exposed component (the node's partition of
    // its sphere: V - A + d + 2F - H = 2, so F = 1 when A - V - d + 4 = 2
    // with H = 2): stitched as a band when the geometry allows
    int band = -1;
    if (h1 - h0 == 2 &&
        (A.arc_off[nd + 1] - ao) - (A.vtx_off[nd + 1] - A.vtx_off[nd]) - (int64_t)d + 4 == 2) {
      band = band_node<T>(A, nd, h0, c, R, ao, rb, ctx, Q, K, DEC, stage, tbase, lane, sa, sv);
      __syncwarp();
    }
    for (int64_t h = band == -1 ? h0 : h1; h < h1; h++) {
      // contour points: entries in order, N points each
      int64_t q0 = A.hole_off[h], q1 = A.hole_off[h + 1];
      const int M = hole_contour<T>(A, nd, h, ao, rb, R, ctx, Q, A.pmax, lane);
      if (M > A.pmax) {
        if (lane == 0) atomicCAS(A.err, 0, 4);
        break;
      }
      __syncwarp();
      V3<T> b = mk3(T(0), T(0), T(0));
      for (int m = lane; m < M; m += 32) b = b + Q[m];
      for (int o = 16; o > 0; o >>= 1) {
        b.x += __shfl_xor_sync(0xffffffffu, b.x, o);
        b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
        b.z += __shfl_xor_sync(0xffffffffu, b.z, o);
      }
      b = b * (T(1) / (T)M);
      // direction of the fan centre, with the exact re-decision near the
      // thresholds
      T bl = norm3(b);
      V3<T> dir = mk3(T(0), T(0), T(0));
      bool ok = false, unc = false;
      if (!IS64 && fabs(bl - T(ETA_BARY) * R) <= T(M_LEN) * R * T(0.05)) unc = true;
      if (bl > T(ETA_BARY) * R) {
        dir = b * (T(1) / bl);
        ok = true;
        for (int li = 0; li < d; li++) {
          EndG<T> e = make_end<T, T>(L, nd, L.adj[rb + li]);
          T x = dot(e.u, dir) - e.s;
          if (!IS64 && fabs(x) <= T(M_LEN)) unc = true;
          if (x > T(0)) ok = false;
        }
      }
      if (!ok) {
        V3<T> su = mk3(T(0), T(0), T(0));
        for (int li = 0; li < d; li++) su = su - make_end<T, T>(L, nd, L.adj[rb + li]).u;
        T sl = norm3(su);
        if (!IS64 && fabs(sl - T(ETA_BARY)) <= T(M_LEN)) unc = true;
        if (sl > T(ETA_BARY)) dir = su * (T(1) / sl);
        else if (bl > T(0)) dir = b * (T(1) / bl);
        else dir = make_end<T, T>(L, nd, L.adj[rb]).u * T(-1);
      }
      tfb_add(A.fb, 11, unc && lane == 0);
      if (!IS64 && unc) {
        // exact: contour in FP64 from the inputs
        if (ctx->node != nd) load_node64(L, nd, ctx, lane);
        __syncwarp();
        V3<double> b64 = mk3(0.0, 0.0, 0.0);
        int Mq = 0;
        for (int64_t q = q0; q < q1; q++) {
          uint32_t ent = A.hole_ent[q];
          int64_t ga = ao + (ent & 0x7fffffffu);
          int rev = ent >> 31;
          int Nq = arc_segments<T>(A, nd, ga, ctx, 0);
          uint32_t av = A.arc_vtx[ga];
          int o = (av >> 16) & 255;
          double a0;
          double dd = arc_dphi64(A, ctx, ga, &a0);
          int64_t vo = A.vtx_off[nd];
          for (int s = lane; s < Nq; s += 32) {
            int m = rev ? Nq - s : s;
            V3<double> z;
            if (m == 0) z = vertex_from_gen<double>(ctx->E, ctx->d, ctx->R, A.vtx_gen[vo + (av & 255)]);
            else if (m == Nq) z = vertex_from_gen<double>(ctx->E, ctx->d, ctx->R, A.vtx_gen[vo + ((av >> 8) & 255)]);
            else {
              double ph = a0 + dd * (double)m / (double)Nq, cs, sn;
              sincos(ph, &sn, &cs);
              z = surf_point(ctx->E[o], cs, sn, 0.0, ctx->R);
            }
            b64 = b64 + z;
          }
          Mq += Nq;
        }
        for (int o = 16; o > 0; o >>= 1) {
          b64.x += __shfl_xor_sync(0xffffffffu, b64.x, o);
          b64.y += __shfl_xor_sync(0xffffffffu, b64.y, o);
          b64.z += __shfl_xor_sync(0xffffffffu, b64.z, o);
        }
        b64 = b64 * (1.0 / (double)Mq);
        double R64 = ctx->R, bl64 = norm3(b64);
        V3<double> d64 = mk3(0.0, 0.0, 0.0);
        bool ok64 = false;
        if (bl64 > ETA_BARY * R64) {
          d64 = b64 * (1.0 / bl64);
          ok64 = true;
          for (int li = 0; li < ctx->d; li++)
            if (dot(ctx->E[li].u, d64) > ctx->E[li].s) ok64 = false;
        }
        if (!ok64) {
          V3<double> su = mk3(0.0, 0.0, 0.0);
          for (int li = 0; li < ctx->d; li++) su = su - ctx->E[li].u;
          double sl = norm3(su);
          if (sl > ETA_BARY) d64 = su * (1.0 / sl);
          else if (bl64 > 0.0) d64 = b64 * (1.0 / bl64);
          else d64 = ctx->E[0].u * -1.0;
        }
        dir = mk3((T)d64.x, (T)d64.y, (T)d64.z);
        __syncwarp();
      }
      V3<T> bp = dir * R;
      // fan triangles (bp, q_m, q_m+1), staged 32 at a time
      for (int c0 = 0; c0 < M; c0 += 32) {
        int m = c0 + lane;
        if (m < M) {
          V3<T> qa = Q[m], qb = Q[(m + 1) % M];
          double ar, vo;
          stl_record<T>(A.out ? stage + 50 * lane : nullptr, c, bp, qa, qb, c + bp, c + qa, c + qb, &ar, &vo);
          sa += ar;
          sv += vo;
        }
        __syncwarp();
        if (A.out) {
          int nrec = M - c0 < 32 ? M - c0 : 32;
          int64_t gt = tbase + c0;
          if (gt + nrec <= A.capacity) flush_stage(A.out + 50 * gt, stage, 50 * nrec, lane);
          else if (lane == 0) atomicCAS(A.err, 0, 4);
        }
        __syncwarp();
      }
      tbase += M;
    }
    if (A.acc) {
      for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sv += __shfl_xor_sync(0xffffffffu, sv, o);
      }
      if (lane == 0) {
        atomicAdd(A.acc, sa);
        atomicAdd(A.acc + 1, sv);
      }
    }
  }
}

}  // namespace lm
