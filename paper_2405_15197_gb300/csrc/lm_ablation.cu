// Warp-centric vs thread-centric trimming (Section 6 of arXiv 2405.15197,
// Fig. thread-vs-warp: the paper's warp-centric meta-meshing kernel ran 35x
// faster than a thread-centric one that allocates a thread per arc
// calculation and lets every thread read the strut parameters it needs from
// global memory by itself).
//
// The step compared is the trimming of Section 4.3.1: on strut end i of a
// node, the kept surface starts at t*(phi) = max(0, max_{j != i} h_j(phi)),
// the envelope of the auxiliary planes P_ij, and its arg-max labels the arc
// the generator at phi ends on.  Both kernels evaluate it at S sample angles
// phi_q = 2 pi q / S of every strut end with the same arithmetic (make_end,
// hval); they differ only in how the work is mapped and where the strut
// parameters come from:
//   * thread-centric: one thread per (strut end, angle); it builds its own
//     end and every other end of its node from the lattice in global memory;
//   * warp-centric: one warp per node; the node's strut ends are built once
//     into shared memory (one per lane), then the lanes sweep (end, angle).
#include <cuda_runtime.h>

#include "lm_geom.cuh"
#include "lm_internal.h"

namespace lm {
namespace {

constexpr double ENV_PI2 = 6.283185307179586476925286766559;

template <typename T>
__device__ __forceinline__ void env_angle(int q, int S, T& c, T& s) {
  const T phi = (T)(ENV_PI2 * (double)q / (double)S);
  lm_sincos(phi, &s, &c);
}

// thread-centric: thread per (strut end, angle), parameters from global memory
template <typename T>
__global__ void __launch_bounds__(256) k_env_thread(LatDev<T> L, int S, T* out_t, int16_t* out_lab) {
  const int64_t n_ends = 2 * L.n_struts;
  const int64_t total = n_ends * (int64_t)S;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = (int32_t)(g / S);
    const int q = (int)(g - (int64_t)e * S);
    const int64_t node = L.ends[e];  // end id 2 strut + side is at node ends[strut][side]
    const EndG<T> Ei = make_end<T, T>(L, node, e);
    const T R = L.node_R[node];
    T c, s;
    env_angle<T>(q, S, c, s);
    const int64_t rb = L.row_ptr[node], re = L.row_ptr[node + 1];
    T best = T(0);
    int lab = -1;
    for (int64_t jj = rb; jj < re; jj++) {
      const int32_t ej = L.adj[jj];
      if (ej == e) continue;
      const EndG<T> Ej = make_end<T, T>(L, node, ej);
      const T hv = hval(Ei, Ej, c, s, R);
      if (hv > best) {
        best = hv;
        lab = (int)(jj - rb);
      }
    }
    out_t[g] = best;
    out_lab[g] = (int16_t)lab;
  }
}

// warp-centric: warp per node, its strut ends staged in shared memory
constexpr int ENV_WARPS = 4;
template <typename T>
__global__ void __launch_bounds__(ENV_WARPS * 32) k_env_warp(LatDev<T> L, int S, T* out_t, int16_t* out_lab,
                                                            int* err) {
  __shared__ EndG<T> sE[ENV_WARPS][LM_MAX_VALENCE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  EndG<T>* E = sE[w];
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t node = gw; node < L.n_nodes; node += nw) {
    const int64_t rb = L.row_ptr[node];
    const int d = (int)(L.row_ptr[node + 1] - rb);
    if (d > LM_MAX_VALENCE) {
      if (lane == 0) atomicCAS(err, 0, LM_ERR_VALENCE);
      continue;
    }
    for (int li = lane; li < d; li += 32) E[li] = make_end<T, T>(L, node, L.adj[rb + li]);
    __syncwarp();
    const T R = L.node_R[node];
    for (int p = lane; p < d * S; p += 32) {
      const int li = p / S, q = p - li * S;
      T c, s;
      env_angle<T>(q, S, c, s);
      T best = T(0);
      int lab = -1;
      for (int j = 0; j < d; j++) {
        if (j == li) continue;
        const T hv = hval(E[li], E[j], c, s, R);
        if (hv > best) {
          best = hv;
          lab = j;
        }
      }
      const int64_t o = (int64_t)E[li].end_id * S + q;
      out_t[o] = best;
      out_lab[o] = (int16_t)lab;
    }
    __syncwarp();
  }
}

template <typename T>
lm_status env_launch(const lm_metamesh* mm, int S, int mode, void* d_t, int16_t* d_label, cudaStream_t st) {
  LatDev<T> L;
  L.xyz = (const T*)mm->xyz;
  L.ends = mm->ends;
  L.node_R = (const T*)mm->node_R;
  L.row_ptr = mm->row_ptr;
  L.adj = mm->adj;
  L.n_nodes = mm->N;
  L.n_struts = mm->E;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (mode == LM_ENV_THREAD) {
    const int64_t total = 2 * mm->E * (int64_t)S;
    int64_t grid = (total + 255) / 256;
    if (grid > (int64_t)sms * 64) grid = (int64_t)sms * 64;
    if (grid < 1) grid = 1;
    count_launch();
    k_env_thread<T><<<(unsigned)grid, 256, 0, st>>>(L, S, (T*)d_t, d_label);
  } else {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_env_warp<T>, ENV_WARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (mm->N + ENV_WARPS - 1) / ENV_WARPS;
    if (grid > (int64_t)per_sm * sms) grid = (int64_t)per_sm * sms;
    if (grid < 1) grid = 1;
    count_launch();
    k_env_warp<T><<<(unsigned)grid, ENV_WARPS * 32, 0, st>>>(L, S, (T*)d_t, d_label, mm->d_err);
  }
  return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

}  // namespace
}  // namespace lm

extern "C" lm_status lm_envelope_samples(const lm_metamesh* mm, int32_t samples, int32_t mode, void* d_t,
                                         int16_t* d_label, void* stream) {
  if (!mm || samples < 1 || samples > 4096 || (mode != LM_ENV_WARP && mode != LM_ENV_THREAD) ||
      (mm->E > 0 && (!d_t || !d_label)))
    return LM_ERR_INVALID_ARG;
  if (mm->E == 0) return LM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return mm->dtype == LM_F32 ? lm::env_launch<float>(mm, samples, mode, d_t, d_label, st)
                             : lm::env_launch<double>(mm, samples, mode, d_t, d_label, st);
}
