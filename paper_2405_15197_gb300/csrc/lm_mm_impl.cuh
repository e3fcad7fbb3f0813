// Launchers of the persistent meta-mesh kernel, one instantiation per
// arithmetic type and valence bucket.
#pragma once
#include "lm_internal.h"
#include "lm_metamesh.cuh"

namespace lm {

using Cap16 = Cap<16, 64, 192, 160>;
using Cap32 = Cap<32, 128, 384, 320>;
using Cap64 = Cap<64, 224, 640, 480>;

template <typename T, typename C>
cudaError_t go_metamesh(bool emit, const MMArgs<T>& A, int block_warps, int grid_ctas,
                        cudaStream_t st, int* used) {
  size_t per = sizeof(WarpSmem<T, C>);
  if (block_warps <= 0) block_warps = 4;
  while (block_warps > 1 && per * block_warps > 200 * 1024) block_warps >>= 1;
  size_t smem = per * block_warps;
  auto kern = emit ? k_metamesh<T, C, true> : k_metamesh<T, C, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block_warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = grid_ctas > 0 ? grid_ctas : per_sm * sms;
  int64_t need = (A.n_list + (A.nodes_per_task > 0 ? A.nodes_per_task : 1) - 1) /
                 (A.nodes_per_task > 0 ? A.nodes_per_task : 1);
  int64_t maxg = (need + block_warps - 1) / block_warps;
  if (grid > maxg) grid = (int)(maxg > 0 ? maxg : 1);
  if (used) *used = grid;
  count_launch();
  kern<<<grid, block_warps * 32, smem, st>>>(A);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_metamesh(int bucket, bool emit, const MMLaunch<T>& a, int block_warps,
                            int grid_ctas, cudaStream_t st, int* used) {
  MMArgs<T> A{};
  A.lat.xyz = a.xyz;
  A.lat.ends = a.ends;
  A.lat.node_R = a.node_R;
  A.lat.row_ptr = a.row_ptr;
  A.lat.adj = a.adj;
  A.lat.n_nodes = a.n_nodes;
  A.lat.n_struts = a.n_struts;
  A.nodes = a.nodes;
  A.n_list = a.n_list;
  A.queue = a.queue;
  A.nodes_per_task = a.nodes_per_task;
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
  A.arc_ends = a.arc_ends;
  A.arc_vtx = a.arc_vtx;
  A.arc_phi = a.arc_phi;
  A.loop_ent = a.loop_ent;
  A.hole_off = a.hole_off;
  A.hole_ent = a.hole_ent;
  A.overflow = a.overflow;
  A.fb = a.fb;
  A.smask = a.smask;
  A.smask_words = a.smask ? a.smask_words : 0;
  if (A.n_list <= 0) {
    if (used) *used = 0;
    return cudaSuccess;
  }
  switch (bucket) {
    case 0: return go_metamesh<T, Cap16>(emit, A, block_warps, grid_ctas, st, used);
    case 1: return go_metamesh<T, Cap32>(emit, A, block_warps, grid_ctas, st, used);
    default: return go_metamesh<T, Cap64>(emit, A, block_warps, grid_ctas, st, used);
  }
}

}  // namespace lm
