// Adjoint of the triangulated area and volume (see lm_adjoint.cuh for the
// method): kernels and the host code behind lm_metamesh_backward.
#include <cuda_runtime.h>

#include "lm_adjoint.cuh"
#include "lm_internal.h"
#include "lm_scan.cuh"
#include "lm_tri.cuh"

namespace lm {
namespace {

constexpr int BW = 8;  // tangent directions per forward-mode pass

template <typename T>
TriArgs<T> bwd_args(lm_metamesh* mm, int k) {
  TriArgs<T> A{};
  A.lat.xyz = (const T*)mm->xyz;
  A.lat.ends = mm->ends;
  A.lat.node_R = (const T*)mm->node_R;
  A.lat.row_ptr = mm->row_ptr;
  A.lat.adj = mm->adj;
  A.lat.n_nodes = mm->N;
  A.lat.n_struts = mm->E;
  A.vtx_off = mm->vtx_off;
  A.arc_off = mm->arc_off;
  A.end_off = mm->end_off;
  A.node_hole_off = mm->hole_off_n;
  A.hole_off = mm->hole_off;
  A.vtx_z = (const T*)mm->vtx_z;
  A.vtx_gen = mm->vtx_gen;
  A.arc_vtx = mm->arc_vtx;
  A.arc_phi = (const T*)mm->arc_phi;
  A.loop_ent = mm->loop_ent;
  A.hole_ent = mm->hole_ent;
  A.k = k;
  A.tri_off = mm->tri_off;
  A.item_begin = 0;
  A.item_end = mm->E + mm->N;
  A.err = mm->d_err;
  A.pmax = mm->tri_pmax > 0 ? mm->tri_pmax : 1;
  A.emax = mm->max_loop_entries > 0 ? mm->max_loop_entries : 1;
  A.dmax = mm->max_valence > 0 ? mm->max_valence : 1;
  A.n_vtx = mm->V;
  return A;
}

// segment count of every arc (with the FP64 re-decision of the triangulation)
// and its number of interior points; the largest vertex count of a node
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_arc_counts(TriArgs<T> A, int32_t* arc_N, int32_t* arc_np,
                                                        int* max_v) {
  int mv = 0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < A.lat.n_nodes;
       n += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t ga = A.arc_off[n]; ga < A.arc_off[n + 1]; ga++) {
      bool unc;
      int N = seg_count<T>(A.arc_phi[2 * ga + 1], A.k, unc);
      if (unc) N = segments64_thread<T>(A, n, ga);
      arc_N[ga] = N;
      arc_np[ga] = N > 1 ? N - 1 : 0;
    }
    int v = (int)(A.vtx_off[n + 1] - A.vtx_off[n]);
    mv = v > mv ? v : mv;
  }
  mv = __reduce_max_sync(0xffffffffu, mv);
  if ((threadIdx.x & 31) == 0 && mv > 0) atomicMax(max_v, mv);
}

// contour points of hole h (node-relative) and their point ids into
// Q[0, cap), PQ[0, cap); returns the contour's point count
template <typename T>
__device__ int bwd_contour(const TriArgs<T>& A, const int32_t* arc_N, int64_t nd, int64_t h, int64_t ao,
                           int64_t rb, T R, V3<T>* Q, int64_t* PQ, int cap, int lane) {
  const LatDev<T>& L = A.lat;
  int M = 0;
  for (int64_t q = A.hole_off[h]; q < A.hole_off[h + 1]; q++) {
    uint32_t ent = A.hole_ent[q];
    int64_t ga = ao + (ent & 0x7fffffffu);
    int rev = ent >> 31;
    int Nq = arc_N[ga];
    EntryS<T> en;
    en.g = arc_geo<T>(make_end<T, T>(L, nd, L.adj[rb + ((A.arc_vtx[ga] >> 16) & 255)]), nullptr, R);
    en.phi0 = A.arc_phi[2 * ga];
    en.dphi = A.arc_phi[2 * ga + 1];
    en.psi = T(0);
    en.N = Nq;
    en.pre = M;
    en.ga = ga;
    en.rev = (uint8_t)rev;
    en.own = 1;
    uint32_t av = A.arc_vtx[ga];
    for (int s = lane; s < Nq; s += 32) {
      if (M + s >= cap) continue;
      V3<T> z;
      T th;
      entry_point<T>(A, nd, en, nullptr, s, z, th);
      int m = rev ? Nq - s : s;
      Q[M + s] = z;
      PQ[M + s] = (m == 0 || m == Nq) ? A.vtx_off[nd] + (m == 0 ? (av & 255) : ((av >> 8) & 255))
                                      : A.n_vtx + A.arc_pt_off[ga] + m - 1;
    }
    M += Nq;
  }
  return M;
}

// Point adjoints of an annular band (the forward pass's band_node, reading
// 10): the same stitching, with its decisions taken from FP64 angles of the
// contour points in the lattice's precision.  Returns false when the band
// does not apply (the holes are fanned).
template <typename T>
__device__ __noinline__ bool bwd_band(const TriArgs<T>& A, const int32_t* arc_N, int64_t nd, int64_t h0,
                                      int64_t ao, int64_t rb, T R, V3<T>* Q, int64_t* PQ, double* K,
                                      int32_t* DEC, int lane) {
  const int M0 = bwd_contour<T>(A, arc_N, nd, h0, ao, rb, R, Q, PQ, A.pmax, lane);
  const int off = M0 < A.pmax ? M0 : A.pmax;
  const int M1 = bwd_contour<T>(A, arc_N, nd, h0 + 1, ao, rb, R, Q + off, PQ + off, A.pmax - off, lane);
  if (M0 < 1 || M1 < 1 || M0 + M1 > A.pmax) return false;
  __syncwarp();
  V3<double> bs[2] = {mk3(0.0, 0.0, 0.0), mk3(0.0, 0.0, 0.0)};
  for (int p = lane; p < M0 + M1; p += 32) {
    const V3<T> z = Q[p];
    bs[p < M0 ? 0 : 1] = bs[p < M0 ? 0 : 1] + mk3((double)z.x, (double)z.y, (double)z.z);
  }
  for (int cc = 0; cc < 2; cc++)
    for (int o = 16; o > 0; o >>= 1) {
      bs[cc].x += __shfl_xor_sync(0xffffffffu, bs[cc].x, o);
      bs[cc].y += __shfl_xor_sync(0xffffffffu, bs[cc].y, o);
      bs[cc].z += __shfl_xor_sync(0xffffffffu, bs[cc].z, o);
    }
  const V3<double> a = bs[1] * (1.0 / (double)M1) - bs[0] * (1.0 / (double)M0);
  const double al = norm3(a);
  if (!(al > ETA_BARY * (double)R)) return false;
  const V3<double> ua = a * (1.0 / al);
  const double aa[3] = {fabs(ua.x), fabs(ua.y), fabs(ua.z)};
  int ax = 0;
  if (aa[1] < aa[ax]) ax = 1;
  if (aa[2] < aa[ax]) ax = 2;
  const V3<double> c1 = cross(ua, mk3<double>(ax == 0, ax == 1, ax == 2));
  const V3<double> e1 = c1 * (1.0 / norm3(c1)), e2 = cross(ua, e1);
  for (int p = lane; p < M0 + M1; p += 32) {
    const V3<double> z = mk3((double)Q[p].x, (double)Q[p].y, (double)Q[p].z);
    K[p] = atan2(dot(z, e2), dot(z, e1));
  }
  __syncwarp();
  const int sB = band_zip(K, M0, M1, DEC, lane);
  if (sB < 0) return false;
  auto bpos = [&](int j) { return band_bpos(M0, M1, sB, j); };
  const int ntri = M0 + M1;
  for (int p = lane; p < ntri; p += 32) {
    const int v = DEC[p], ia = v >> 1, ib = p - ia - 1;
    const int qa = ia % M0, qb = (v & 1) ? (ia + 1) % M0 : bpos(ib + 1), qc = bpos(ib);
    const V3<T> ra = Q[qa], rb2 = Q[qb], rc = Q[qc];
    V3<T> cr = cross(rb2 - ra, rc - ra);
    T len = norm3(cr);
    V3<T> nh = len > T(0) ? cr * (T(1) / len) : mk3(T(0), T(0), T(0));
    tri_point_adjoints<T>(A, ra, rb2, rc, nh, cr, PQ[qa], PQ[qb], PQ[qc]);
  }
  __syncwarp();
  return true;
}

// Per-warp workspace of k_bwd_holes: contour points, point ids, FP64 keys
// and stitching steps (bands)
template <typename T>
__host__ __device__ constexpr size_t bwd_holes_qb(int pmax) { return ((size_t)pmax * sizeof(V3<T>) + 7) & ~(size_t)7; }
template <typename T>
__host__ __device__ constexpr size_t bwd_holes_ws(int pmax) {
  return (bwd_holes_qb<T>(pmax) + 8 * (size_t)pmax + 8 * (size_t)pmax + 4 * (size_t)pmax + 15) & ~(size_t)15;
}

// Fan triangles of every hole: point adjoints of the contour points and of
// the centre (point id n_vtx + interior points + hole id); the band of an
// annular node instead.  Warp per node.
template <typename T>
__global__ void __launch_bounds__(128) k_bwd_holes(TriArgs<T> A, const int32_t* arc_N, int64_t centre_base) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t qb = bwd_holes_qb<T>(A.pmax);
  const size_t wsb = bwd_holes_ws<T>(A.pmax);
  V3<T>* Q = reinterpret_cast<V3<T>*>(smem_raw + (size_t)w * wsb);
  int64_t* PQ = reinterpret_cast<int64_t*>(smem_raw + (size_t)w * wsb + qb);
  double* K = reinterpret_cast<double*>(smem_raw + (size_t)w * wsb + qb + 8 * (size_t)A.pmax);
  int32_t* DEC = reinterpret_cast<int32_t*>(smem_raw + (size_t)w * wsb + qb + 16 * (size_t)A.pmax);
  const LatDev<T>& L = A.lat;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t nd = gw; nd < L.n_nodes; nd += nw) {
    int64_t h0 = A.node_hole_off[nd], h1 = A.node_hole_off[nd + 1];
    if (h0 == h1) continue;
    int64_t ao = A.arc_off[nd], rb = L.row_ptr[nd];
    int d = (int)(L.row_ptr[nd + 1] - rb);
    T R = L.node_R[nd];
    bool band = false;
    if (h1 - h0 == 2 &&
        (A.arc_off[nd + 1] - ao) - (A.vtx_off[nd + 1] - A.vtx_off[nd]) - (int64_t)d + 4 == 2) {
      band = bwd_band<T>(A, arc_N, nd, h0, ao, rb, R, Q, PQ, K, DEC, lane);
      __syncwarp();
    }
    for (int64_t h = band ? h1 : h0; h < h1; h++) {
      const int M = bwd_contour<T>(A, arc_N, nd, h, ao, rb, R, Q, PQ, A.pmax, lane);
      __syncwarp();
      if (M > A.pmax) {
        if (lane == 0) atomicCAS(A.err, 0, 4);
        break;
      }
      V3<T> b = mk3(T(0), T(0), T(0));
      for (int m = lane; m < M; m += 32) b = b + Q[m];
      for (int o = 16; o > 0; o >>= 1) {
        b.x += __shfl_xor_sync(0xffffffffu, b.x, o);
        b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
        b.z += __shfl_xor_sync(0xffffffffu, b.z, o);
      }
      b = b * (T(1) / (T)M);
      // centre rule of the forward pass (decided in FP32 here)
      T bl = norm3(b);
      V3<T> dir;
      bool ok = false;
      if (bl > T(ETA_BARY) * R) {
        dir = b * (T(1) / bl);
        ok = true;
        for (int li = 0; li < d; li++) {
          EndG<T> e = make_end<T, T>(L, nd, L.adj[rb + li]);
          if (dot(e.u, dir) - e.s > T(0)) ok = false;
        }
      }
      if (!ok) {
        V3<T> su = mk3(T(0), T(0), T(0));
        for (int li = 0; li < d; li++) su = su - make_end<T, T>(L, nd, L.adj[rb + li]).u;
        T sl = norm3(su);
        if (sl > T(ETA_BARY)) dir = su * (T(1) / sl);
        else if (bl > T(0)) dir = b * (T(1) / bl);
        else dir = make_end<T, T>(L, nd, L.adj[rb]).u * T(-1);
      }
      V3<T> bp = dir * R;
      for (int m = lane; m < M; m += 32) {
        int m1 = m + 1 < M ? m + 1 : 0;
        V3<T> qa = Q[m], qb = Q[m1];
        V3<T> cr = cross(qa - bp, qb - bp);
        T len = norm3(cr);
        V3<T> nh = len > T(0) ? cr * (T(1) / len) : mk3(T(0), T(0), T(0));
        tri_point_adjoints<T>(A, bp, qa, qb, nh, cr, centre_base + h, PQ[m], PQ[m1]);
      }
      __syncwarp();
    }
  }
}

template <int W, typename S>
__device__ __forceinline__ void dual_warp_sum(Dual<W, S>& a) {
  for (int o = 16; o > 0; o >>= 1) {
    a.v += __shfl_xor_sync(0xffffffffu, a.v, o);
#pragma unroll
    for (int i = 0; i < W; i++) a.t[i] += __shfl_xor_sync(0xffffffffu, a.t[i], o);
  }
}

// contract a point's tangents with its adjoint
template <int W, typename S>
__device__ __forceinline__ void contract(S acc[W], const V3<Dual<W, S>>& p, const S* g) {
  S gx = g[0], gy = g[1], gz = g[2];
#pragma unroll
  for (int i = 0; i < W; i++) acc[i] += gx * p.x.t[i] + gy * p.y.t[i] + gz * p.z.t[i];
}

// interior point m of arc ga (node-relative), in dual numbers
template <typename T, int W>
__device__ __forceinline__ V3<Dual<W, T>> arc_point_dual(const ArcGeo<Dual<W, T>>& g, const Dual<W, T>& p0,
                                                          const Dual<W, T>& dp, int m, int N) {
  Dual<W, T> phi = p0 + dp * Dual<W, T>((T)m / (T)N);
  return geo_point(g, phi);
}

// angles of arc ga in its owner's frame, followed continuously from the
// stored values (the forward pass's arc data)
template <typename T, int W>
__device__ __forceinline__ void arc_angles_dual(const TriArgs<T>& A, int64_t ga, const EndG<Dual<W, T>>& Eo,
                                                const V3<Dual<W, T>>* Z, Dual<W, T>& p0, Dual<W, T>& dp) {
  uint32_t av = A.arc_vtx[ga];
  int v0 = av & 255, v1 = (av >> 8) & 255;
  T s0 = (T)A.arc_phi[2 * ga], sd = (T)A.arc_phi[2 * ga + 1];
  Dual<W, T> a0 = raw_angle(Eo, Z[v0]);
  p0 = shift(a0, s0 + sc_rem2pi(a0.v - s0) - a0.v);
  if (v0 == v1) {
    dp = Dual<W, T>((T)PI2);
  } else {
    T s1 = s0 + sd;
    Dual<W, T> a1 = raw_angle(Eo, Z[v1]);
    Dual<W, T> p1 = shift(a1, s1 + sc_rem2pi(a1.v - s1) - a1.v);
    dp = p1 - p0;
  }
}

template <typename T>
struct BwdNodeArgs {
  const int32_t* arc_N;
  const T* adj;           // point adjoints [points][3]
  int64_t centre_base;    // point id of hole 0's centre
  double* g_xyz;          // [N][3]
  double* g_R;            // [N]
  int maxd, maxv;
  int* queue;
};

// Parameter adjoints, warp per node, forward mode with W directions per pass.
template <typename T, int W>
__global__ void __launch_bounds__(64) k_bwd_nodes(TriArgs<T> A, BwdNodeArgs<T> B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef Dual<W, T> D;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t eb = (size_t)B.maxd * sizeof(EndG<D>);
  const size_t wsb = ((eb + (size_t)B.maxv * sizeof(V3<D>)) + 15) & ~(size_t)15;
  EndG<D>* E = reinterpret_cast<EndG<D>*>(smem_raw + (size_t)w * wsb);
  V3<D>* Z = reinterpret_cast<V3<D>*>(smem_raw + (size_t)w * wsb + eb);
  const LatDev<T>& L = A.lat;
  while (true) {
    int64_t nd = 0;
    if (lane == 0) nd = atomicAdd(B.queue, 1);
    nd = __shfl_sync(0xffffffffu, nd, 0);
    if (nd >= L.n_nodes) break;
    const int64_t rb = L.row_ptr[nd], vo = A.vtx_off[nd], ao = A.arc_off[nd];
    const int d = (int)(L.row_ptr[nd + 1] - rb);
    const int nv = (int)(A.vtx_off[nd + 1] - vo), na = (int)(A.arc_off[nd + 1] - ao);
    if (d == 0 || d > B.maxd || nv > B.maxv) continue;
    const int np = 4 + 4 * d;
    for (int s0 = 0; s0 < np; s0 += W) {
      // seeded node centre and radius
      V3<D> c = mk3(D((T)L.xyz[3 * nd]), D((T)L.xyz[3 * nd + 1]), D((T)L.xyz[3 * nd + 2]));
      D R = D((T)L.node_R[nd]);
      if (0 >= s0 && 0 < s0 + W) c.x.t[0 - s0] = T(1);
      if (1 >= s0 && 1 < s0 + W) c.y.t[1 - s0] = T(1);
      if (2 >= s0 && 2 < s0 + W) c.z.t[2 - s0] = T(1);
      if (3 >= s0 && 3 < s0 + W) R.t[3 - s0] = T(1);
      for (int li = lane; li < d; li += 32) {
        int32_t eid = L.adj[rb + li];
        int32_t st = eid >> 1;
        int32_t far = (eid & 1) ? L.ends[2 * (int64_t)st] : L.ends[2 * (int64_t)st + 1];
        V3<D> cf = mk3(D((T)L.xyz[3 * far]), D((T)L.xyz[3 * far + 1]), D((T)L.xyz[3 * far + 2]));
        D Rf = D((T)L.node_R[far]);
        int sb = 4 + 4 * li - s0;
        if (sb >= 0 && sb < W) cf.x.t[sb] = T(1);
        if (sb + 1 >= 0 && sb + 1 < W) cf.y.t[sb + 1] = T(1);
        if (sb + 2 >= 0 && sb + 2 < W) cf.z.t[sb + 2] = T(1);
        if (sb + 3 >= 0 && sb + 3 < W) Rf.t[sb + 3] = T(1);
        E[li] = end_from<T, D>(L, nd, eid, c, R, cf, Rf);
      }
      __syncwarp();
      T acc[W];
#pragma unroll
      for (int i = 0; i < W; i++) acc[i] = T(0);
      // vertices
      for (int v = lane; v < nv; v += 32) {
        V3<D> z = gen_point<D>(E, R, A.vtx_gen[vo + v]);
        Z[v] = z;
        contract<W, T>(acc, c + z, B.adj + 3 * (vo + v));
      }
      __syncwarp();
      // interior points of every arc
      for (int a = lane; a < na; a += 32) {
        int64_t ga = ao + a;
        int N = B.arc_N[ga];
        if (N < 2) continue;
        uint32_t av = A.arc_vtx[ga];
        int o = (av >> 16) & 255, ot = (int)((av >> 24) & 255) - 1;
        ArcGeo<D> g = arc_geo<D>(E[o], ot >= 0 ? &E[ot] : nullptr, R);
        D p0, dp;
        arc_angles_dual<T, W>(A, ga, E[o], Z, p0, dp);
        const T* adj = B.adj + 3 * (A.n_vtx + A.arc_pt_off[ga]);
        for (int m = 1; m < N; m++) contract<W, T>(acc, c + arc_point_dual<T, W>(g, p0, dp, m, N), adj + 3 * (m - 1));
      }
      // hole centres: barycentre of the contour, projected as in the forward pass
      for (int64_t h = A.node_hole_off[nd]; h < A.node_hole_off[nd + 1]; h++) {
        V3<D> b = mk3(D(T(0)), D(T(0)), D(T(0)));
        int M = 0;
        for (int64_t q = A.hole_off[h]; q < A.hole_off[h + 1]; q++) {
          uint32_t ent = A.hole_ent[q];
          int64_t ga = ao + (ent & 0x7fffffffu);
          int N = B.arc_N[ga];
          uint32_t av = A.arc_vtx[ga];
          int o = (av >> 16) & 255, rev = ent >> 31;
          // contour points of this entry: s = 0..N-1, m = rev ? N - s : s
          ArcGeo<D> g = arc_geo<D>(E[o], nullptr, R);
          D p0, dp;
          arc_angles_dual<T, W>(A, ga, E[o], Z, p0, dp);
          for (int s = lane; s < N; s += 32) {
            int m = rev ? N - s : s;
            V3<D> z = (m == 0) ? Z[av & 255] : (m == N ? Z[(av >> 8) & 255] : arc_point_dual<T, W>(g, p0, dp, m, N));
            b = b + z;
          }
          M += N;
        }
        dual_warp_sum<W, T>(b.x);
        dual_warp_sum<W, T>(b.y);
        dual_warp_sum<W, T>(b.z);
        b = b * D(T(1) / (T)M);
        T bl = lm_sqrt(b.x.v * b.x.v + b.y.v * b.y.v + b.z.v * b.z.v);
        int rule = 3;
        if (bl > (T)ETA_BARY * R.v) {
          bool ok = true;
          for (int li = 0; li < d; li++) {
            T x = (E[li].u.x.v * b.x.v + E[li].u.y.v * b.y.v + E[li].u.z.v * b.z.v) / bl - E[li].s.v;
            if (x > T(0)) ok = false;
          }
          if (ok) rule = 0;
        }
        V3<D> su = mk3(D(T(0)), D(T(0)), D(T(0)));
        for (int li = 0; li < d; li++) su = su - E[li].u;
        if (rule != 0) {
          T sl = lm_sqrt(su.x.v * su.x.v + su.y.v * su.y.v + su.z.v * su.z.v);
          rule = sl > (T)ETA_BARY ? 1 : (bl > T(0) ? 2 : 3);
        }
        V3<D> dir = rule == 1 ? su * (D(T(1)) / norm3(su))
                              : (rule == 3 ? E[0].u * D(T(-1)) : b * (D(T(1)) / norm3(b)));
        if (lane == 0) contract<W, T>(acc, c + dir * R, B.adj + 3 * (B.centre_base + h));
      }
      // reduce the W tangents and scatter to the parameters they seed
#pragma unroll
      for (int i = 0; i < W; i++)
        for (int o = 16; o > 0; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
      if (lane < W && s0 + lane < np) {
        int sl = s0 + lane;
        T val = T(0);
#pragma unroll
        for (int i = 0; i < W; i++)
          if (i == lane) val = acc[i];
        int64_t node = nd;
        int q = sl;
        if (sl >= 4) {
          int li = (sl - 4) >> 2;
          q = (sl - 4) & 3;
          int32_t eid = L.adj[rb + li];
          int32_t st = eid >> 1;
          node = (eid & 1) ? L.ends[2 * (int64_t)st] : L.ends[2 * (int64_t)st + 1];
        }
        if (q < 3) atomicAdd(B.g_xyz + 3 * node + q, (double)val);
        else atomicAdd(B.g_R + node, (double)val);
      }
      __syncwarp();
    }
  }
}

template <typename T>
__global__ void k_bwd_out(const double* gx, const double* gr, int64_t n, T* out_xyz, T* out_r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (out_xyz) {
      out_xyz[3 * i] += (T)gx[3 * i];
      out_xyz[3 * i + 1] += (T)gx[3 * i + 1];
      out_xyz[3 * i + 2] += (T)gx[3 * i + 2];
    }
    if (out_r) out_r[i] += (T)gr[i];
  }
}

int sms_now() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

#define BK(x)                                     \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) { status = e_; goto done; } \
  } while (0)

}  // namespace

template <typename T>
cudaError_t metamesh_backward(lm_metamesh* mm, int k, double w_area, double w_vol, void* gxyz, void* gr,
                              cudaStream_t st) {
  cudaError_t status = cudaSuccess;
  const int sms = sms_now();
  TriArgs<T> A = bwd_args<T>(mm, k);
  A.w_area = w_area;
  A.w_vol = w_vol;
  const int64_t Na = mm->A, N = mm->N;
  int32_t *arc_N = nullptr, *arc_np = nullptr;
  int64_t *arc_pt_off = nullptr, *ws = nullptr;
  int* misc = nullptr;
  T* adj = nullptr;
  double* g = nullptr;
  uint32_t* redo = nullptr;
  int64_t P = 0;
  int hm[2] = {0, 0};
  BK(cudaMallocAsync((void**)&arc_N, sizeof(int32_t) * (size_t)(Na > 0 ? Na : 1), st));
  BK(cudaMallocAsync((void**)&arc_np, sizeof(int32_t) * (size_t)(Na > 0 ? Na : 1), st));
  BK(cudaMallocAsync((void**)&arc_pt_off, sizeof(int64_t) * (size_t)(Na + 1), st));
  BK(cudaMallocAsync((void**)&ws, sizeof(int64_t) * (size_t)(scan_ws_elems(Na) + 8), st));
  BK(cudaMallocAsync((void**)&misc, sizeof(int) * 4, st));
  BK(cudaMemsetAsync(misc, 0, sizeof(int) * 4, st));
  {
    int64_t grid = (N + 255) / 256;
    if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
    if (grid < 1) grid = 1;
    count_launch();
    k_bwd_arc_counts<T><<<(unsigned)grid, 256, 0, st>>>(A, arc_N, arc_np, misc);
    BK(cudaGetLastError());
  }
  BK(scan_excl<int32_t>(arc_np, 1, Na, arc_pt_off, ws, st));
  BK(cudaMemcpyAsync(&P, arc_pt_off + Na, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  BK(cudaMemcpyAsync(hm, misc, sizeof(int), cudaMemcpyDeviceToHost, st));
  BK(cudaStreamSynchronize(st));
  A.arc_pt_off = arc_pt_off;
  {
    const int64_t npts = mm->V + P + mm->H;
    BK(cudaMallocAsync((void**)&adj, sizeof(T) * 3 * (size_t)(npts > 0 ? npts : 1), st));
    BK(cudaMemsetAsync(adj, 0, sizeof(T) * 3 * (size_t)(npts > 0 ? npts : 1), st));
    BK(cudaMallocAsync((void**)&g, sizeof(double) * 4 * (size_t)(N > 0 ? N : 1), st));
    BK(cudaMemsetAsync(g, 0, sizeof(double) * 4 * (size_t)(N > 0 ? N : 1), st));
    A.adj = adj;
  }
  // 1. point adjoints of the strut bands (the two passes of the forward
  //    stitching, so every stitching decision is the forward's)
  if (mm->E > 0) {
    constexpr int TL = 16;
    TileLayout<T, TL> Lay{A.pmax, A.emax, false, true, A.dmax}, LayX{A.pmax, A.emax, true, true, A.dmax};
    auto tiles_for = [&](size_t bytes) {
      int t = 128 / TL;  // the stitching kernel's block bound
      while (t > 2 && (size_t)t * bytes > 200 * 1024) t >>= 1;
      return (size_t)t * bytes <= 200 * 1024 ? t : 0;
    };
    const int tiles = tiles_for(Lay.bytes());
    const int tilesx = tiles_for(LayX.bytes()) < 64 / TL ? tiles_for(LayX.bytes()) : 64 / TL;
    if (tiles == 0 || tilesx == 0) { status = cudaErrorInvalidValue; goto done; }
    const int64_t words = mm->E / 32 + 1;
    BK(cudaMallocAsync((void**)&redo, sizeof(uint32_t) * (size_t)words, st));
    BK(cudaMemsetAsync(redo, 0, sizeof(uint32_t) * (size_t)words, st));
    A.item_end = mm->E;
    {
      size_t smem = (size_t)tiles * Lay.bytes();
      auto kern = k_tri_tiles<T, TL, false, false, true>;
      BK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int64_t grid = (mm->E + tiles - 1) / tiles;
      if (grid > (int64_t)sms * 32) grid = (int64_t)sms * 32;
      count_launch();
      kern<<<(unsigned)grid, tiles * TL, smem, st>>>(A, nullptr, redo, 0);
      BK(cudaGetLastError());
    }
    if (sizeof(T) == 4) {
      size_t smem = (size_t)tilesx * LayX.bytes();
      auto kx = k_tri_tiles<T, TL, false, true, true>;
      BK(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kx, tilesx * TL, smem);
      int64_t gx = (int64_t)(per_sm > 0 ? per_sm : 1) * sms;
      count_launch();
      kx<<<(unsigned)gx, tilesx * TL, smem, st>>>(A, nullptr, redo, 0);
      BK(cudaGetLastError());
    }
    A.item_end = mm->E + mm->N;
  }
  // 2. point adjoints of the hole fans
  if (mm->H > 0) {
    const size_t wsb = bwd_holes_ws<T>(A.pmax);
    // four warps per block, fewer when a warp's contour points need more
    // shared memory (fine resolutions)
    int warps = 4;
    while (warps > 1 && (size_t)warps * wsb > 200 * 1024) warps >>= 1;
    if (wsb > 200 * 1024) BK(cudaErrorInvalidValue);
    size_t smem = (size_t)warps * wsb;
    BK(cudaFuncSetAttribute(k_bwd_holes<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t grid = (N + warps - 1) / warps;
    if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
    if (grid < 1) grid = 1;
    count_launch();
    k_bwd_holes<T><<<(unsigned)grid, warps * 32, smem, st>>>(A, arc_N, mm->V + P);
    BK(cudaGetLastError());
  }
  // 3. parameter adjoints, node by node
  if (N > 0) {
    BwdNodeArgs<T> B;
    B.arc_N = arc_N;
    B.adj = adj;
    B.centre_base = mm->V + P;
    B.g_xyz = g;
    B.g_R = g + 3 * N;
    B.maxd = mm->max_valence > 0 ? mm->max_valence : 1;
    B.maxv = hm[0] > 0 ? hm[0] : 1;
    B.queue = misc + 1;
    const size_t eb = (size_t)B.maxd * sizeof(EndG<Dual<BW, T>>);
    const size_t wsb = ((eb + (size_t)B.maxv * sizeof(V3<Dual<BW, T>>)) + 15) & ~(size_t)15;
    int warps = 2;
    while (warps > 1 && (size_t)warps * wsb > 200 * 1024) warps--;
    if (wsb > 200 * 1024) { status = cudaErrorInvalidValue; goto done; }
    size_t smem = (size_t)warps * wsb;
    auto kern = k_bwd_nodes<T, BW>;
    BK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)per_sm * sms;
    int64_t need = (N + warps - 1) / warps;
    if (grid > need) grid = need;
    count_launch();
    kern<<<(unsigned)grid, 32 * warps, smem, st>>>(A, B);
    BK(cudaGetLastError());
    int64_t go = (N + 255) / 256;
    if (go > (int64_t)sms * 8) go = (int64_t)sms * 8;
    count_launch();
    k_bwd_out<T><<<(unsigned)go, 256, 0, st>>>(g, g + 3 * N, N, (T*)gxyz, (T*)gr);
    BK(cudaGetLastError());
  }
  BK(cudaStreamSynchronize(st));
done:
  for (void* p : {(void*)arc_N, (void*)arc_np, (void*)arc_pt_off, (void*)ws, (void*)misc, (void*)adj, (void*)g,
                  (void*)redo})
    if (p) cudaFreeAsync(p, st);
  cudaStreamSynchronize(st);
  return status;
}

template cudaError_t metamesh_backward<float>(lm_metamesh*, int, double, double, void*, void*, cudaStream_t);
template cudaError_t metamesh_backward<double>(lm_metamesh*, int, double, double, void*, void*, cudaStream_t);

}  // namespace lm
