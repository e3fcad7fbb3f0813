// Launchers of the persistent meta-mesh kernel, one instantiation per
// arithmetic type and valence bucket.
#pragma once
#include "lm_internal.h"
#include "lm_metamesh.cuh"

namespace lm {

template <typename T>
int metamesh_ctas_per_sm() {
  const size_t smem = mm_smem_bytes<T>();
  if (cudaFuncSetAttribute(k_metamesh<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_metamesh<T>, MM_BLOCK_WARPS * 32, smem) !=
      cudaSuccess)
    return 0;
  return per_sm;
}

template <typename T>
cudaError_t launch_metamesh(bool emit, const MMLaunch<T>& a, const MMBuckets& bk, int grid_ctas, cudaStream_t st,
                            int* used) {
  MMArgs<T> A{};
  A.lat.xyz = a.xyz;
  A.lat.ends = a.ends;
  A.lat.node_R = a.node_R;
  A.lat.row_ptr = a.row_ptr;
  A.lat.adj = a.adj;
  A.lat.n_nodes = a.n_nodes;
  A.lat.n_struts = a.n_struts;
  A.err = a.err;
  A.node_flags = a.node_flags;
  A.node_cnt = a.node_cnt;
  A.end_cnt = a.end_cnt;
  A.vtx_off = a.vtx_off;
  A.arc_off = a.arc_off;
  A.hole_off_n = a.hole_off_n;
  A.hent_off_n = a.hent_off_n;
  A.end_off = a.end_off;
  A.vtx_z = a.vtx_z;
  A.vtx_key = a.vtx_key;
  A.vtx_flags = a.vtx_flags;
  A.vtx_gen = a.vtx_gen;
  A.arc_vtx = a.arc_vtx;
  A.arc_phi = a.arc_phi;
  A.loop_ent = a.loop_ent;
  A.hole_off = a.hole_off;
  A.hole_ent = a.hole_ent;
  A.overflow = a.overflow;
  A.fb = a.fb;
  A.emit = emit ? 1 : 0;
  A.ar = a.arena;
  const size_t smem = mm_smem_bytes<T>();
  int per_sm = metamesh_ctas_per_sm<T>();
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = grid_ctas > 0 ? grid_ctas : per_sm * sms;
  if (used) *used = grid;
  count_launch();
  k_metamesh<T><<<grid, MM_BLOCK_WARPS * 32, smem, st>>>(A, bk);
  return cudaGetLastError();
}

// One warp per node stored in the arena: its vertices, arcs, holes and hole
// entries move to the node's CSR ranges, its loop entries to the CSR ranges of
// its ends (adjacency order), hole starts become absolute.
template <typename T>
__global__ void __launch_bounds__(256) k_mm_gather(MMLaunch<T> a) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t n = w0; n < a.n_nodes; n += nw) {
    const int64_t at = a.arena.start[n];
    if (at < 0) continue;
    const int64_t vo = a.vtx_off[n], nv = a.vtx_off[n + 1] - vo;
    const int64_t ao = a.arc_off[n], na = a.arc_off[n + 1] - ao;
    const int64_t ho = a.hole_off_n[n], nh = a.hole_off_n[n + 1] - ho;
    const int64_t heo = a.hent_off_n[n], nhe = a.hent_off_n[n + 1] - heo;
    const ArenaBlock B = arena_block(nv, na, nh, nhe, 0, sizeof(T));
    const unsigned char* blk = a.arena.buf + at;
    const T* vz = reinterpret_cast<const T*>(blk + B.vz);
    const uint64_t* vkey = reinterpret_cast<const uint64_t*>(blk + B.vkey);
    const uint8_t* vfl = blk + B.vfl;
    const uint32_t* vgen = reinterpret_cast<const uint32_t*>(blk + B.vgen);
    for (int64_t q = lane; q < 3 * nv; q += 32) a.vtx_z[3 * vo + q] = vz[q];
    for (int64_t v = lane; v < nv; v += 32) {
      a.vtx_key[vo + v] = vkey[v];
      a.vtx_flags[vo + v] = vfl[v];
      a.vtx_gen[vo + v] = vgen[v];
    }
    const uint32_t* avtx = reinterpret_cast<const uint32_t*>(blk + B.avtx);
    const T* aphi = reinterpret_cast<const T*>(blk + B.aphi);
    for (int64_t q = lane; q < 2 * na; q += 32) a.arc_phi[2 * ao + q] = aphi[q];
    for (int64_t q = lane; q < na; q += 32) a.arc_vtx[ao + q] = avtx[q];
    const uint32_t* hos = reinterpret_cast<const uint32_t*>(blk + B.ho);
    const uint32_t* hes = reinterpret_cast<const uint32_t*>(blk + B.he);
    for (int64_t h = lane; h < nh; h += 32) a.hole_off[ho + h] = heo + hos[h];
    for (int64_t q = lane; q < nhe; q += 32) a.hole_ent[heo + q] = hes[q];
    const uint16_t* le = reinterpret_cast<const uint16_t*>(blk + B.le);
    const int64_t rb = a.row_ptr[n], d = a.row_ptr[n + 1] - rb;
    // a lane per strut end: its loop's entries start in the block at the
    // exclusive prefix of the entry counts of the ends before it
    int64_t run0 = 0;
    for (int64_t l0 = 0; l0 < d; l0 += 32) {
      const int64_t li = l0 + lane;
      int64_t eo = 0, ne = 0;
      if (li < d) {
        const int32_t eid = a.adj[rb + li];
        eo = a.end_off[eid];
        ne = a.end_off[eid + 1] - eo;
      }
      int64_t inc = ne;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      const int64_t run = run0 + inc - ne;
      for (int64_t q = 0; q < ne; q++) {
        const uint32_t v = le[run + q];
        a.loop_ent[eo + q] = v == 0xffffu ? 0xffffffffu : (v & 0x7fffu) | ((v & 0x8000u) << 16);
      }
      run0 += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
}

template <typename T>
cudaError_t launch_mm_gather(const MMLaunch<T>& a, cudaStream_t st) {
  if (a.n_nodes <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (a.n_nodes + 7) / 8;
  if (grid > (int64_t)sms * 16) grid = (int64_t)sms * 16;
  count_launch();
  k_mm_gather<T><<<(unsigned)grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lm
