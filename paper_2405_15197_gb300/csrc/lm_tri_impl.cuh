// Launchers of the triangulation kernels.
#pragma once
#include <algorithm>
#include "lm_internal.h"
#include "lm_tri.cuh"

namespace lm {

template <typename T>
TriArgs<T> tri_args(const TriLaunch<T>& a) {
  TriArgs<T> A{};
  A.lat.xyz = a.xyz;
  A.lat.ends = a.ends;
  A.lat.node_R = a.node_R;
  A.lat.row_ptr = a.row_ptr;
  A.lat.adj = a.adj;
  A.lat.n_nodes = a.n_nodes;
  A.lat.n_struts = a.n_struts;
  A.vtx_off = a.vtx_off;
  A.arc_off = a.arc_off;
  A.end_off = a.end_off;
  A.node_hole_off = a.node_hole_off;
  A.hole_off = a.hole_off;
  A.vtx_z = a.vtx_z;
  A.vtx_gen = a.vtx_gen;
  A.arc_vtx = a.arc_vtx;
  A.arc_phi = a.arc_phi;
  A.loop_ent = a.loop_ent;
  A.hole_ent = a.hole_ent;
  A.k = a.k;
  A.item_cnt = a.item_cnt;
  A.tri_off = a.tri_off;
  A.item_begin = a.item_begin;
  A.item_end = a.item_end;
  A.out_first = 0;
  A.capacity = a.capacity;
  A.out = a.out;
  A.acc = a.acc;
  A.queue = a.queue;
  A.err = a.err;
  A.pmax = a.pmax;
  A.emax = a.emax;
  A.dmax = a.dmax > 0 ? a.dmax : 1;
  A.max_pts = a.max_pts;
  A.range = a.range;
  A.node_mask = a.node_mask;
  A.rlist = a.rlist;
  A.rcap = a.rlist ? a.rcap : 0;
  A.fb = a.fb;
  return A;
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

template <typename T>
cudaError_t launch_tri_count(const TriLaunch<T>& a, cudaStream_t st) {
  TriArgs<T> A = tri_args(a);
  int threads = 256;
  int64_t warps_needed = (a.n_nodes + a.n_struts + 31) / 32;
  int64_t grid = (warps_needed * 32 + threads - 1) / threads;
  int64_t gmax = a.scratch_warps / (threads / 32);
  if (grid > gmax) grid = gmax;
  if (grid < 1) grid = 1;
  count_launch();
  k_tri_count<T><<<(unsigned)grid, threads, 0, st>>>(A, a.scratch, 0, a.n_nodes + a.n_struts, a.item_cnt,
                                                     a.max_pts);
  return cudaGetLastError();
}

// hole fans of the nodes in the item range (one warp per node with holes)
template <typename T>
cudaError_t launch_tri_holes(const TriLaunch<T>& a, cudaStream_t st) {
  TriArgs<T> A = tri_args(a);
  const int sms = sm_count();
  const size_t wsb = holes_ws_bytes<T>(a.pmax);
  // eight warps per block, fewer when a warp's contour points need more
  // shared memory (fine resolutions)
  int warps = 8;
  while (warps > 1 && (size_t)warps * wsb > 200 * 1024) warps >>= 1;
  if (wsb > 200 * 1024) return cudaErrorInvalidValue;
  const int threads = warps * 32;
  const size_t smem = warps * wsb;
  cudaError_t e = cudaFuncSetAttribute(k_tri_holes<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tri_holes<T>, threads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)per_sm * sms;
  const int64_t gmax = a.scratch_warps / (2 * warps);
  if (grid > gmax) grid = gmax;
  const int64_t nb = a.item_begin > a.n_struts ? a.item_begin : a.n_struts;
  const int64_t n = a.item_end - nb;
  const int64_t gneed = ((n + 31) / 32 + warps - 1) / warps;  // groups of 32 nodes
  if (grid > gneed) grid = gneed;
  if (grid < 1) grid = 1;
  A.queue = a.queue + 1;
  count_launch();
  k_tri_holes<T><<<(unsigned)grid, threads, smem, st>>>(A, a.scratch, a.first_ptr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tri_emit(const TriLaunch<T>& a, cudaStream_t st) {
  TriArgs<T> A = tri_args(a);
  int sms = sm_count();
  cudaError_t e;
  const bool holes = a.item_end > a.n_struts;
  const bool fork = holes && a.aux && a.item_begin < a.n_struts;
  if (fork) {
    // the hole fans are independent of the strut passes: they run on the
    // second stream beside them and the stream joins before returning
    if ((e = cudaEventRecord(a.ev_fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(a.aux, a.ev_fork, 0)) != cudaSuccess) return e;
    if ((e = launch_tri_holes(a, a.aux)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(a.ev_join, a.aux)) != cudaSuccess) return e;
  }
  // struts: one 8-lane tile per strut (four per warp; measured faster than
  // 4, 16 or 32 lanes on octet and BCC lattices at k = 8 and 32) while the
  // per-tile shared memory fits; otherwise (very fine resolutions) one thread
  // per strut that streams its points
  if (a.item_begin < a.n_struts) {
    // the FP64 pass (about 1 % of the struts) is bound by the FP64 pipe (1/64
    // of the FP32 rate) and its steps occupy few lanes: two deferred struts
    // per warp (16-lane tiles) fill its instructions better than one
    constexpr int TL = 8, TLX = 16;
    const int64_t n = (a.item_end < a.n_struts ? a.item_end : a.n_struts) - a.item_begin;
    TileLayout<T, TL> Lay{a.pmax, a.emax, false, false, a.dmax};
    TileLayout<T, TLX> LayX{a.pmax, a.emax, true, false, a.dmax};
    const size_t smem_cap = 200 * 1024;
    auto tiles_for = [&](size_t bytes, int tl) {
      int t = 128 / tl;
      while (t > 2 && (size_t)t * bytes > smem_cap) t >>= 1;
      return (size_t)t * bytes <= smem_cap ? t : 0;
    };
    const int tiles = tiles_for(Lay.bytes(), TL);
    const int tilesx = std::min(tiles_for(LayX.bytes(), TLX), 64 / TLX);
    if (tiles > 0 && tilesx > 0) {
      constexpr bool F32 = sizeof(T) == 4;
      const int64_t e_end = a.item_end < a.n_struts ? a.item_end : a.n_struts;
      const int64_t w0 = (a.item_begin - a.redo_base) >> 5, w1 = (e_end - a.redo_base + 31) >> 5;
      if (F32) {
        if (!a.redo) return cudaErrorInvalidValue;
        if (a.range) {
          int64_t gw = (w1 - w0 + 255) / 256;
          if (gw > (int64_t)sms * 4) gw = (int64_t)sms * 4;
          if (gw < 1) gw = 1;
          count_launch();
          k_redo_clear<<<(unsigned)gw, 256, 0, st>>>(a.range, a.redo, a.redo_base, a.n_struts, a.rlist);
          e = cudaGetLastError();
        } else {
          e = cudaMemsetAsync(a.redo + w0, 0, (size_t)(w1 - w0) * sizeof(uint32_t), st);
          if (e == cudaSuccess && a.rlist) e = cudaMemsetAsync(a.rlist, 0, sizeof(unsigned long long), st);
        }
        if (e != cudaSuccess) return e;
      }
      {
        const int tpb = tiles * TL;
        size_t smem = (size_t)tiles * Lay.bytes();
        auto kern = a.acc ? k_tri_tiles<T, TL, true, false> : k_tri_tiles<T, TL, false, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t grid = (n + tiles - 1) / tiles;
        int64_t gmax = (int64_t)per_sm * sms * 8;
        if (grid > gmax) grid = gmax;
        if (grid < 1) grid = 1;
        count_launch();
        kern<<<(unsigned)grid, tpb, smem, st>>>(A, a.first_ptr, a.redo, a.redo_base);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      if (F32) {
        // the deferred struts, with the FP64 stability steps
        const int tpb = tilesx * TLX;
        size_t smem = (size_t)tilesx * LayX.bytes();
        auto kx = a.acc ? k_tri_tiles<T, TLX, true, true> : k_tri_tiles<T, TLX, false, true>;
        e = cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kx, tpb, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t gx = (int64_t)per_sm * sms;
        if (gx < 1) gx = 1;
        count_launch();
        kx<<<(unsigned)gx, tpb, smem, st>>>(A, a.first_ptr, a.redo, a.redo_base);
      }
    } else {
      const int tpb = 128;
      size_t smem = (size_t)tpb * tri_lane_stride<T>();
      auto kern = a.acc ? k_tri_thread<T, true> : k_tri_thread<T, false>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, smem);
      if (per_sm < 1) per_sm = 1;
      int64_t grid = (n + tpb - 1) / tpb;
      int64_t gmax = (int64_t)per_sm * sms * 8;
      if (grid > gmax) grid = gmax;
      if (grid < 1) grid = 1;
      count_launch();
      kern<<<(unsigned)grid, tpb, smem, st>>>(A, a.first_ptr);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (fork) return cudaStreamWaitEvent(st, a.ev_join, 0);
  if (holes) return launch_tri_holes(a, st);
  return cudaSuccess;
}

}  // namespace lm
