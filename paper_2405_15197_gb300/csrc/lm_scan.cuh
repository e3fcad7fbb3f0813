// Exclusive prefix sums for the index regions of the meta-mesh (Section
// 4.3.2: "the index region is a prefix-sum array ... obtained through
// parallel scanning"), written here as a three-phase reduce / scan / apply
// with warp-shuffle block scans.  Input counts are int32 or int64 (strided),
// outputs are int64 offsets with the total appended (n + 1 entries).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "lm_internal.h"

namespace lm {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_excl_scan(int64_t x, int64_t* warp_tot, int64_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_tot[w] = v;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < nw ? warp_tot[lane] : 0;
    int64_t a = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, a, o);
      if (lane >= o) a += t;
    }
    if (lane < nw) warp_tot[lane] = a - s;
    if (lane == 31) *total = a;
  }
  __syncthreads();
  int64_t r = v - x + warp_tot[w];
  __syncthreads();
  return r;
}

template <typename I>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const I* in, int64_t stride, int64_t n,
                                                              int64_t* sums) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; q++) {
    int64_t i = base + (int64_t)q * SCAN_THREADS + threadIdx.x;
    if (i < n) s += (int64_t)in[i * stride];
  }
  block_excl_scan(s, wt, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// apply: out[i] = offset(block) + exclusive scan within the block
template <typename I>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const I* in, int64_t stride, int64_t n,
                                                             const int64_t* block_off, int64_t* out) {
  __shared__ int64_t wt[32];
  __shared__ int64_t tot;
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; q++) {
    int64_t i = base + q;
    v[q] = i < n ? (int64_t)in[i * stride] : 0;
    s += v[q];
  }
  int64_t off = block_excl_scan(s, wt, &tot) + (block_off ? block_off[blockIdx.x] : 0);
#pragma unroll
  for (int q = 0; q < SCAN_ITEMS; q++) {
    int64_t i = base + q;
    if (i < n) out[i] = off;
    off += v[q];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = off;
}

// Workspace (int64 elements) needed by scan_excl for n inputs.
inline int64_t scan_workspace(int64_t n) {
  int64_t w = 0;
  while (n > SCAN_TILE) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    w += nb + 1;
    n = nb;
  }
  return w + 1;
}

// out[0..n] = exclusive scan of in[0], in[stride], ...; out[n] = total
template <typename I>
cudaError_t scan_excl(const I* in, int64_t stride, int64_t n, int64_t* out, int64_t* ws,
                      cudaStream_t st) {
  if (n <= SCAN_TILE) {
    count_launch();
    k_scan_apply<I><<<1, SCAN_THREADS, 0, st>>>(in, stride, n, nullptr, out);
    return cudaGetLastError();
  }
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* sums = ws;
  int64_t* offs = ws + nb;  // nb + 1 entries, followed by deeper workspace
  count_launch(2);
  k_scan_reduce<I><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, stride, n, sums);
  cudaError_t e = scan_excl<int64_t>(sums, 1, nb, offs, ws + 2 * nb + 1, st);
  if (e != cudaSuccess) return e;
  k_scan_apply<I><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, stride, n, offs, out);
  return cudaGetLastError();
}

inline int64_t scan_ws_elems(int64_t n) {
  // sums (nb) + offs (nb+1) per level
  int64_t w = 0;
  while (n > SCAN_TILE) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    w += 2 * nb + 1;
    n = nb;
  }
  return w + 1;
}

}  // namespace lm
