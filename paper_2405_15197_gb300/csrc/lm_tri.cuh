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
  int* max_pts;            // count pass: max points of one loop / one node's holes
};

// ---- segment count (Eq. sampling) with an FP64 recheck flag
template <typename T>
__device__ __forceinline__ int seg_count(T dphi, int k, bool& unc) {
  T y = dphi * (T)k * T(1.0 / PI2) - T(TAU_COUNT);
  T c = ceil(y);
  unc = sizeof(T) == 4 && fabs(y - rint(y)) <= T(M_CNT);
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
  if (a0 < -ETA_PHI) a0 += PI2;
  if (a1 < -ETA_PHI) a1 += PI2;
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
template <typename T>
__global__ void __launch_bounds__(256) k_tri_count(TriArgs<T> A, Node64* scratch) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  Node64* ctx = scratch + gw;
  const int64_t E = A.lat.n_struts, N = A.lat.n_nodes;
  const int64_t n_items = E + N;
  // one thread per item, lanes of a warp on consecutive items; an exact
  // recount (rare) loads the node's FP64 context warp-cooperatively
  for (int64_t base = (int64_t)gw * 32; base < n_items; base += (int64_t)nwarps * 32) {
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
      } else {
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
    if (lane == 0 && mx > 0) atomicMax(A.max_pts, mx);
    if (it < n_items) A.item_cnt[it] = (int32_t)c;
  }
}

// ------------------------------------------------------- strut stitching
// Per-warp shared workspace for one strut (dynamic size from pmax, emax).
struct StrutHdr {
  int ne[2], np[2];
  int64_t node[2];
  int32_t own_end[2];
  int own_li[2];
  int sB;
};

template <typename T>
struct StrutWs {
  StrutHdr* h;  // shared scalars of the warp's current strut
  // entry arrays [2][emax]: global arc, N, prefix, rev, start angle
  int64_t* e_ga;
  int* e_n;
  int* e_pre;
  uint8_t* e_rev;
  T* e_psi;
  // point arrays [2][pmax]
  T* th;
  V3<T>* z;
  double* th64;
  uint8_t* fl;   // point needs the exact angle
  T* kB;         // B keys in A's window
  unsigned char* stage;  // 32 STL records + slack
};

__host__ __device__ inline size_t strut_ws_bytes(int pmax, int emax, int elt) {
  size_t b = 64 + 2 * (size_t)emax * (8 + 4 + 4 + 1 + elt) + 2 * (size_t)pmax * (elt + 3 * elt + 8 + 1) +
             (size_t)pmax * elt + 32 * 50 + 256;
  return (b + 15) & ~(size_t)15;
}

template <typename T>
__device__ StrutWs<T> carve_ws(unsigned char* p, int pmax, int emax) {
  StrutWs<T> W;
  W.h = reinterpret_cast<StrutHdr*>(p);
  size_t o = 64;
  auto take = [&](size_t bytes) {
    unsigned char* r = p + o;
    o += (bytes + 7) & ~(size_t)7;
    return r;
  };
  W.e_ga = (int64_t*)take(2 * emax * 8);
  W.e_n = (int*)take(2 * emax * 4);
  W.e_pre = (int*)take(2 * emax * 4);
  W.e_psi = (T*)take(2 * emax * sizeof(T));
  W.e_rev = (uint8_t*)take(2 * emax);
  W.th = (T*)take(2 * pmax * sizeof(T));
  W.z = (V3<T>*)take(2 * pmax * sizeof(V3<T>));
  W.th64 = (double*)take(2 * pmax * 8);
  W.kB = (T*)take(pmax * sizeof(T));
  W.fl = (uint8_t*)take(2 * pmax);
  o = (o + 15) & ~(size_t)15;
  W.stage = p + o;
  return W;
}

// node-relative point s of entry q of a loop and its own-frame angle (T)
template <typename T>
__device__ void loop_point(const TriArgs<T>& A, int64_t node, const EndG<T>& own, int64_t ga, int N,
                           int rev, int s, T psi, V3<T>& z, T& th) {
  const LatDev<T>& L = A.lat;
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255;
  int m = rev ? N - s : s;
  T R = L.node_R[node];
  if (s == 0) {
    int64_t vi = A.vtx_off[node] + (rev ? v1 : v0);
    z = mk3(A.vtx_z[3 * vi], A.vtx_z[3 * vi + 1], A.vtx_z[3 * vi + 2]);
    th = psi;
    return;
  }
  int o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
  int64_t b = L.row_ptr[node];
  EndG<T> Eo = make_end<T, T>(L, node, L.adj[b + o]);
  T phi0 = A.arc_phi[2 * ga], dphi = A.arc_phi[2 * ga + 1];
  T phi = phi0 + dphi * (T)m / (T)N;
  T c, sn;
  lm_sincos(phi, &sn, &c);
  T t = T(0);
  if (ot >= 0) {
    EndG<T> Et = make_end<T, T>(L, node, L.adj[b + ot]);
    t = hval(Eo, Et, c, sn, R);
  }
  z = surf_point(Eo, c, sn, t, R);
  if (Eo.end_id == own.end_id) {
    th = phi;
  } else {
    th = psi + wrap_from(raw_angle(own, z) - psi, T(-ETA_PHI));
  }
}

// exact own-frame angle of the same point (ctx = FP64 context of `node`)
template <typename T>
__device__ __noinline__ double loop_theta64(const TriArgs<T>& A, const Node64* ctx, int own_li,
                                            int64_t ga, int N, int rev, int s) {
  if (ctx->node < 0 || ctx->d < 1 || ctx->d > 64 || own_li < 0 || own_li >= ctx->d) {
    atomicCAS(A.err, 0, 6);
    return 0.0;
  }
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255;
  int o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
  int64_t vo = A.vtx_off[ctx->node];
  double a0;
  double dd = arc_dphi64(A, ctx, ga, &a0);
  const EndG<double>& me = ctx->E[own_li];
  V3<double> zs = vertex_from_gen<double>(ctx->E, ctx->d, ctx->R, A.vtx_gen[vo + (rev ? v1 : v0)]);
  double psi = raw_angle(me, zs);
  if (psi < -ETA_PHI) psi += PI2;
  if (s == 0) return psi;
  int m = rev ? N - s : s;
  double phi = a0 + dd * (double)m / (double)N;
  if (o == own_li) return phi;
  double c, sn;
  sincos(phi, &sn, &c);
  double t = ot >= 0 ? hval(ctx->E[o], ctx->E[ot], c, sn, ctx->R) : 0.0;
  V3<double> z = surf_point(ctx->E[o], c, sn, t, ctx->R);
  return psi + wrap_from(raw_angle(me, z) - psi, -ETA_PHI);
}

// STL record writer: triangle (a, b, c) given node-relative points and the
// node centres they belong to; o = the centre the math is relative to.
template <typename T>
__device__ __forceinline__ void stl_record(unsigned char* dst, V3<T> o, V3<T> ra, V3<T> rb, V3<T> rc,
                                           V3<T> pa, V3<T> pb, V3<T> pc, double* area, double* vol) {
  V3<T> cr = cross(rb - ra, rc - ra);
  T len = norm3(cr);
  V3<T> nn = len > T(0) ? cr * (T(1) / len) : mk3(T(0), T(0), T(0));
  float f[12] = {(float)nn.x, (float)nn.y, (float)nn.z, (float)pa.x, (float)pa.y, (float)pa.z,
                 (float)pb.x, (float)pb.y, (float)pb.z, (float)pc.x, (float)pc.y, (float)pc.z};
  if (dst) {
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
                                            int lane) {
  uintptr_t ga = (uintptr_t)gdst;
  int head = (int)((16 - (ga & 15)) & 15);
  if (head > nbytes) head = nbytes;
  head &= ~1;
  for (int q = lane; q < head / 2; q += 32)
    reinterpret_cast<uint16_t*>(gdst)[q] = reinterpret_cast<const uint16_t*>(st)[q];
  int body = ((nbytes - head) / 16) * 16;
  // shared source may be misaligned relative to 16: assemble from 2-byte words
  for (int q = lane; q < body / 16; q += 32) {
    const uint16_t* s = reinterpret_cast<const uint16_t*>(st + head + 16 * q);
    uint4 v;
    v.x = (uint32_t)s[0] | ((uint32_t)s[1] << 16);
    v.y = (uint32_t)s[2] | ((uint32_t)s[3] << 16);
    v.z = (uint32_t)s[4] | ((uint32_t)s[5] << 16);
    v.w = (uint32_t)s[6] | ((uint32_t)s[7] << 16);
    reinterpret_cast<uint4*>(gdst + head)[q] = v;
  }
  int tail = nbytes - head - body;
  for (int q = lane; q < tail / 2; q += 32)
    reinterpret_cast<uint16_t*>(gdst + head + body)[q] =
        reinterpret_cast<const uint16_t*>(st + head + body)[q];
}

template <typename T>
__global__ void __launch_bounds__(256) k_tri_struts(TriArgs<T> A, Node64* scratch,
                                                     const int64_t* first_ptr) {
  const int64_t out_first = first_ptr ? *first_ptr : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t wsb = strut_ws_bytes(A.pmax, A.emax, sizeof(T));
  StrutWs<T> W = carve_ws<T>(smem_raw + (size_t)w * wsb, A.pmax, A.emax);
  Node64* ctx = scratch + 2 * gw;
  const LatDev<T>& L = A.lat;
  const int64_t E = L.n_struts;
  const int64_t e_end = A.item_end < E ? A.item_end : E;
  constexpr bool IS64 = sizeof(T) == 8;
  while (true) {
    int64_t e = 0;
    if (lane == 0) e = A.item_begin + atomicAdd(A.queue, 1);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e >= e_end) break;
    int32_t a = L.ends[2 * e], b = L.ends[2 * e + 1];
    int32_t lo = a < b ? a : b, hi = a < b ? b : a;
    int side_lo = (a == lo) ? 0 : 1;
    // ---- entries of both loops, segment counts, prefix sums
    bool ovf = false;
    for (int X = 0; X < 2; X++) {
      int64_t node = X == 0 ? lo : hi;
      int32_t eid = (int32_t)(2 * e + (X == 0 ? side_lo : 1 - side_lo));
      int64_t q0 = A.end_off[eid], q1 = A.end_off[eid + 1];
      int ne = (int)(q1 - q0);
      if (ne > A.emax) { ovf = true; break; }
      int64_t ao = A.arc_off[node];
      int cntsum = 0;
      bool need = false;
      for (int c0 = 0; c0 < ne; c0 += 32) {
        int q = c0 + lane;
        int Nq = 0;
        bool unc = false;
        int64_t ga = 0;
        int rev = 0;
        if (q < ne) {
          uint32_t ent = A.loop_ent[q0 + q];
          ga = ao + (ent & 0x7fffffffu);
          rev = ent >> 31;
          Nq = seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
        }
        if (__any_sync(0xffffffffu, unc)) {
          load_node64(L, node, ctx, lane);
          __syncwarp();
          if (unc) Nq = arc_segments<T>(A, node, ga, ctx, 0);
          __syncwarp();
        }
        int pre = warp_excl_scan(Nq, lane) + cntsum;
        if (q < ne) {
          W.e_ga[X * A.emax + q] = ga;
          W.e_n[X * A.emax + q] = Nq;
          W.e_pre[X * A.emax + q] = pre;
          W.e_rev[X * A.emax + q] = (uint8_t)rev;
        }
        cntsum = __shfl_sync(0xffffffffu, pre + Nq, 31);
      }
      if (cntsum > A.pmax) { ovf = true; break; }
      if (lane == 0) {
        W.h->ne[X] = ne;
        W.h->np[X] = cntsum;
        W.h->node[X] = node;
        W.h->own_end[X] = eid;
      }
    }
    if (ovf) {
      if (lane == 0) atomicCAS(A.err, 0, 4);
      continue;
    }
    __syncwarp();
    // ---- own ends, start angles of entries, points
    for (int X = 0; X < 2; X++) {
      int64_t node = W.h->node[X];
      int64_t b0 = L.row_ptr[node];
      int d = (int)(L.row_ptr[node + 1] - b0);
      int li = 0;
      for (int q = lane; q < d; q += 32)
        if (L.adj[b0 + q] == W.h->own_end[X]) li = q + 1;
      li = __reduce_max_sync(0xffffffffu, li) - 1;
      if (lane == 0) W.h->own_li[X] = li;
      EndG<T> own = make_end<T, T>(L, node, W.h->own_end[X]);
      // start angle of each entry: the stored angle for own arcs; otherwise
      // the start vertex's angle, re-decided in FP64 next to the wrap point
      bool pu = false;
      for (int q = lane; q < W.h->ne[X]; q += 32) {
        int64_t ga = W.e_ga[X * A.emax + q];
        uint32_t av = A.arc_vtx[ga];
        int rev = W.e_rev[X * A.emax + q];
        if ((int)((av >> 16) & 255) == li && !rev) {
          W.e_psi[X * A.emax + q] = A.arc_phi[2 * ga];
          continue;
        }
        int64_t vi = A.vtx_off[node] + (rev ? ((av >> 8) & 255) : (av & 255));
        V3<T> zs = mk3(A.vtx_z[3 * vi], A.vtx_z[3 * vi + 1], A.vtx_z[3 * vi + 2]);
        T a = raw_angle(own, zs);
        if (!IS64 && fabs(a + T(ETA_PHI)) <= T(M_ANG)) pu = true;
        W.e_psi[X * A.emax + q] = norm_angle(a);
      }
      if (!IS64 && __any_sync(0xffffffffu, pu)) {
        load_node64(L, node, ctx + X, lane);
        __syncwarp();
        for (int q = lane; q < W.h->ne[X]; q += 32) {
          int64_t ga = W.e_ga[X * A.emax + q];
          uint32_t av = A.arc_vtx[ga];
          int rev = W.e_rev[X * A.emax + q];
          if ((int)((av >> 16) & 255) == li && !rev) continue;
          int64_t vi = A.vtx_off[node] + (rev ? ((av >> 8) & 255) : (av & 255));
          V3<double> z64 = vertex_from_gen<double>(ctx[X].E, ctx[X].d, ctx[X].R, A.vtx_gen[vi]);
          W.e_psi[X * A.emax + q] = (T)norm_angle(raw_angle(ctx[X].E[li], z64));
        }
      }
      __syncwarp();
      int np = W.h->np[X], ne = W.h->ne[X];
      for (int p = lane; p < np; p += 32) {
        // entry containing point p
        int lo_q = 0, hi_q = ne - 1;
        while (lo_q < hi_q) {
          int mid = (lo_q + hi_q + 1) >> 1;
          if (W.e_pre[X * A.emax + mid] <= p) lo_q = mid;
          else hi_q = mid - 1;
        }
        int q = lo_q;
        V3<T> z;
        T th;
        loop_point<T>(A, node, own, W.e_ga[X * A.emax + q], W.e_n[X * A.emax + q],
                      W.e_rev[X * A.emax + q], p - W.e_pre[X * A.emax + q],
                      W.e_psi[X * A.emax + q], z, th);
        W.z[X * A.pmax + p] = z;
        W.th[X * A.pmax + p] = th;
        W.fl[X * A.pmax + p] = 0;
      }
    }
    __syncwarp();
    const int nA = W.h->np[0], nB = W.h->np[1];
    T* thA = W.th;
    T* thB = W.th + A.pmax;
    // ---- exact angles where an A point and a B point are too close to order
    if (!IS64) {
      bool any = false;
      for (int i = lane; i < nA; i += 32) {
        for (int j = 0; j < nB; j++) {
          T dd = thA[i] - thB[j];
          dd -= T(PI2) * rint(dd * T(1.0 / PI2));
          if (fabs(dd) <= T(M_ANG)) {
            W.fl[i] = 1;
            W.fl[A.pmax + j] = 1;
            any = true;
          }
        }
      }
      if (__any_sync(0xffffffffu, any)) {
        __syncwarp();
        for (int X = 0; X < 2; X++) {
          load_node64(L, W.h->node[X], ctx + X, lane);
        }
        __syncwarp();
        for (int X = 0; X < 2; X++) {
          int np = W.h->np[X], ne = W.h->ne[X];
          for (int p = lane; p < np; p += 32) {
            if (!W.fl[X * A.pmax + p]) continue;
            int lo_q = 0, hi_q = ne - 1;
            while (lo_q < hi_q) {
              int mid = (lo_q + hi_q + 1) >> 1;
              if (W.e_pre[X * A.emax + mid] <= p) lo_q = mid;
              else hi_q = mid - 1;
            }
            int q = lo_q;
            W.th64[X * A.pmax + p] =
                loop_theta64<T>(A, ctx + X, W.h->own_li[X], W.e_ga[X * A.emax + q], W.e_n[X * A.emax + q],
                                W.e_rev[X * A.emax + q], p - W.e_pre[X * A.emax + q]);
          }
        }
        __syncwarp();
      }
    }
    // ---- B keys in the window [thA0 - ETA_ZIP, thA0 + 2pi - ETA_ZIP) that
    // starts at A's first point; exact keys for flagged B points
    const T thA0 = thA[0];
    for (int j = lane; j < nB; j += 32) {
      T x = wrap_from(thB[j], thA0 - T(ETA_ZIP));
      if (!IS64 && W.fl[A.pmax + j]) {
        double a0 = W.fl[0] ? W.th64[0] : (double)thA0;
        double x64 = wrap_from(W.th64[A.pmax + j], a0 - ETA_ZIP);
        W.th64[A.pmax + j] = x64;
        x = (T)x64;
      }
      W.kB[j] = x;
    }
    __syncwarp();
    {
      // rotation: first index of the smallest key
      T mn = T(1e30);
      for (int j = lane; j < nB; j += 32) mn = fmin(mn, W.kB[j]);
      for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      int first = 0x7fffffff;
      for (int j = lane; j < nB; j += 32)
        if (W.kB[j] == mn) first = min(first, j);
      first = __reduce_min_sync(0xffffffffu, first);
      if (lane == 0) W.h->sB = first == 0x7fffffff ? 0 : first;
    }
    __syncwarp();
    const int sB = W.h->sB;
    // A event i (1..nA) precedes B event j (0..nB-1) iff thA(i) <= kB(j) + ETA_ZIP
    auto a_before_b = [&](int i, int j) -> bool {
      int ia = i < nA ? i : 0;
      int jb = (sB + j) % nB;
      if (!IS64 && W.fl[ia] && W.fl[A.pmax + jb]) {
        double x = W.th64[ia] + (i < nA ? 0.0 : PI2);
        return x <= W.th64[A.pmax + jb] + ETA_ZIP;
      }
      T x = i < nA ? thA[i] : thA0 + T(PI2);
      return x <= W.kB[jb] + T(ETA_ZIP);
    };
    // ---- triangles: merged sequence of nA + nB events; each lane takes one
    // output position and finds its event by merge-path search
    const int ntri = nA + nB;
    const int64_t t0 = A.tri_off[e] - out_first;
    double sa = 0.0, sv = 0.0;
    V3<T> cA = node_xyz<T, T>(L, lo), cB = node_xyz<T, T>(L, hi);
    V3<T> dAB = cB - cA;
    for (int c0 = 0; c0 < ntri; c0 += 32) {
      int p = c0 + lane;
      if (p < ntri) {
        int lo_i = p - nB > 0 ? p - nB : 0, hi_i = p < nA ? p : nA;
        while (lo_i < hi_i) {
          int mid = (lo_i + hi_i) >> 1;
          bool more = (mid < nA) && (p - mid - 1 >= 0) && a_before_b(mid + 1, p - mid - 1);
          if (more) lo_i = mid + 1;
          else hi_i = mid;
        }
        int i = lo_i, jn = p - i;
        bool isA = (i < nA) && (jn == nB || a_before_b(i + 1, jn));
        V3<T> ra, rb, rc, pa, pb, pc;
        if (isA) {
          int jb = ((sB + jn - 1) % nB + nB) % nB;
          V3<T> zb = W.z[A.pmax + jb];
          ra = W.z[i];
          rb = W.z[(i + 1) % nA];
          rc = dAB + zb;
          pa = cA + ra;
          pb = cA + rb;
          pc = cB + zb;
        } else {
          int jb = (sB + jn) % nB, jp = ((sB + jn - 1) % nB + nB) % nB;
          V3<T> za = W.z[i % nA];
          ra = za;
          rb = dAB + W.z[A.pmax + jb];
          rc = dAB + W.z[A.pmax + jp];
          pa = cA + za;
          pb = cB + W.z[A.pmax + jb];
          pc = cB + W.z[A.pmax + jp];
        }
        double ar, vo;
        stl_record<T>(A.out ? W.stage + 50 * lane : nullptr, cA, ra, rb, rc, pa, pb, pc, &ar, &vo);
        sa += ar;
        sv += vo;
      }
      __syncwarp();
      if (A.out) {
        int nrec = ntri - c0 < 32 ? ntri - c0 : 32;
        int64_t gt = t0 + c0;
        if (gt + nrec <= A.capacity) flush_stage(A.out + 50 * gt, W.stage, 50 * nrec, lane);
        else if (lane == 0) atomicCAS(A.err, 0, 4);
      }
      __syncwarp();
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

// ---------------------------------------------------------- hole fans
// One warp per node: for each hole, the contour points (circular arcs in
// hole order), their barycentre b, b_project = o + R (b - o)/|b - o| (Section
// 5), falling back to the direction away from the struts when b sits at the
// centre or outside the hole region; fan triangles (b_project, q_m, q_m+1).
template <typename T>
__global__ void __launch_bounds__(256) k_tri_holes(TriArgs<T> A, Node64* scratch,
                                                    const int64_t* first_ptr) {
  const int64_t out_first = first_ptr ? *first_ptr : 0;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t wsb = (size_t)A.pmax * sizeof(V3<T>) + 32 * 50 + 64;
  unsigned char* base = smem_raw + (size_t)w * ((wsb + 15) & ~(size_t)15);
  V3<T>* Q = reinterpret_cast<V3<T>*>(base);
  unsigned char* stage = base + (((size_t)A.pmax * sizeof(V3<T>) + 15) & ~(size_t)15);
  Node64* ctx = scratch + 2 * gw;
  const LatDev<T>& L = A.lat;
  const int64_t E = L.n_struts;
  constexpr bool IS64 = sizeof(T) == 8;
  const int64_t n0 = (A.item_begin > E ? A.item_begin : E) - E;
  const int64_t n1 = A.item_end - E;
  while (true) {
    int64_t nd = 0;
    if (lane == 0) nd = n0 + atomicAdd(A.queue, 1);
    nd = __shfl_sync(0xffffffffu, nd, 0);
    if (nd >= n1) break;
    int64_t h0 = A.node_hole_off[nd], h1 = A.node_hole_off[nd + 1];
    if (h0 == h1) continue;
    int64_t ao = A.arc_off[nd];
    int64_t rb = L.row_ptr[nd];
    int d = (int)(L.row_ptr[nd + 1] - rb);
    T R = L.node_R[nd];
    V3<T> c = node_xyz<T, T>(L, nd);
    int64_t tbase = A.tri_off[E + nd] - out_first;
    double sa = 0.0, sv = 0.0;
    for (int64_t h = h0; h < h1; h++) {
      // contour points: entries in order, N points each
      int64_t q0 = A.hole_off[h], q1 = A.hole_off[h + 1];
      int M = 0;
      for (int64_t q = q0; q < q1; q++) {
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
        EndG<T> own = make_end<T, T>(L, nd, L.adj[rb + ((A.arc_vtx[ga] >> 16) & 255)]);
        for (int s = lane; s < Nq; s += 32) {
          V3<T> z;
          T th;
          if (M + s < A.pmax) {
            loop_point<T>(A, nd, own, ga, Nq, rev, s, T(0), z, th);
            Q[M + s] = z;
          }
        }
        M += Nq;
      }
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
