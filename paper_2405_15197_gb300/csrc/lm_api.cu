// liblm C ABI: CSR build, valence bucketing, the two-pass meta-mesh build,
// triangulation, objective, streaming to pinned host memory.
// Paper: arXiv 2405.15197 (Sections 4.2.2, 4.3, 5).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <fcntl.h>
#include <unistd.h>

#include <algorithm>
#include <cerrno>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lm_geom.cuh"
#include "lm_internal.h"
#include "lm_scan.cuh"

using namespace lm;

#include <atomic>
static std::atomic<long long> g_launches{0};
namespace lm {
void count_launch(int n) { g_launches += n; }
}

namespace {

#define LM_CK(x)                                  \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) return st_cuda(e_);   \
  } while (0)

// the CUDA error behind the last LM_ERR_CUDA / LM_ERR_OOM of this thread
thread_local cudaError_t g_last_cuda = cudaSuccess;

// NVTX range of one call or build phase (visible to a profiler attached to
// the process; no effect otherwise)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

lm_status st_cuda(cudaError_t e) {
  g_last_cuda = e;
  if (e == cudaErrorMemoryAllocation) return LM_ERR_OOM;
  return LM_ERR_CUDA;
}

// device allocation on behalf of handle mm, within its test budget
// (lm_options.mem_budget)
cudaError_t mm_malloc(lm_metamesh* mm, void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (mm->opt.mem_budget > 0 && mm->alloc_bytes + (int64_t)bytes > mm->opt.mem_budget)
    return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e == cudaSuccess) mm->alloc_bytes += (int64_t)bytes;
  return e;
}
template <typename X>
cudaError_t dalloc(lm_metamesh* mm, X** p, int64_t n, cudaStream_t st) {
  if (n <= 0) n = 1;
  return mm_malloc(mm, (void**)p, sizeof(X) * (size_t)n, st);
}
template <typename X>
void dfree(X*& p, cudaStream_t st) {
  if (p) cudaFreeAsync((void*)p, st);
  p = nullptr;
}

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }

// ---- validation and CSR (node-sorted adjacency by counting sort)
template <typename T>
__global__ void k_strut_validate(const int32_t* ends, const T* radii, int64_t E, int64_t N, int* deg,
                                 int* err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = ends[2 * e], b = ends[2 * e + 1];
    T ra = radii[2 * e], rb = radii[2 * e + 1];
    bool ok = a >= 0 && a < N && b >= 0 && b < N && a != b && ra > T(0) && rb > T(0) &&
              isfinite((double)ra) && isfinite((double)rb);
    if (!ok) {
      set_err(err, LM_ERR_INVALID_ARG);
      continue;
    }
    atomicAdd(&deg[a], 1);
    atomicAdd(&deg[b], 1);
  }
}

__global__ void k_scatter(const int32_t* ends, int64_t E2, int64_t N, const int64_t* row_ptr, int* fill,
                          int32_t* adj) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E2;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t nd = ends[i];
    // a strut with an invalid end was reported by k_strut_validate and was
    // not counted: none of its ends is placed
    const int32_t a = ends[i & ~(int64_t)1], b = ends[i | 1];
    if (a < 0 || a >= N || b < 0 || b >= N || a == b) continue;
    int pos = atomicAdd(&fill[nd], 1);
    adj[row_ptr[nd] + pos] = (int32_t)i;
  }
}

template <typename T>
__global__ void k_node_finalize(const T* xyz, const T* radii, int64_t N, const int64_t* row_ptr,
                                int32_t* adj, T* node_R, int* err, int* max_deg) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = row_ptr[n];
    int d = (int)(row_ptr[n + 1] - b);
    if (!isfinite((double)xyz[3 * n]) || !isfinite((double)xyz[3 * n + 1]) ||
        !isfinite((double)xyz[3 * n + 2]))
      set_err(err, LM_ERR_INVALID_ARG);
    atomicMax(max_deg, d);
    if (d > LM_MAX_VALENCE) {
      set_err(err, LM_ERR_VALENCE);
      node_R[n] = T(0);
      continue;
    }
    // stable order: ascending strut-end id
    for (int i = 1; i < d; i++) {
      int32_t x = adj[b + i];
      int j = i;
      while (j > 0 && adj[b + j - 1] > x) {
        adj[b + j] = adj[b + j - 1];
        j--;
      }
      adj[b + j] = x;
    }
    if (d == 0) {
      node_R[n] = T(0);
      continue;
    }
    T r0 = radii[adj[b]];
    for (int i = 1; i < d; i++) {
      T r = radii[adj[b + i]];
      if (fabs((double)r0 - (double)r) > 1e-12 * fabs((double)r)) set_err(err, LM_ERR_RADIUS_MISMATCH);
    }
    node_R[n] = r0;
  }
}

template <typename T>
__global__ void k_strut_taper(const T* xyz, const int32_t* ends, const T* node_R, int64_t E, int64_t N, int* err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = ends[2 * e], b = ends[2 * e + 1];
    if (a < 0 || a >= N || b < 0 || b >= N || a == b) continue;  // reported by k_strut_validate
    double dx = (double)xyz[3 * b] - (double)xyz[3 * a], dy = (double)xyz[3 * b + 1] - (double)xyz[3 * a + 1],
           dz = (double)xyz[3 * b + 2] - (double)xyz[3 * a + 2];
    double L = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(fabs((double)node_R[a] - (double)node_R[b]) < L)) set_err(err, LM_ERR_DEGENERATE);
  }
}

// global strut-end ids of every arc (owner, other or -1) from its node-local
// end indices in arc_vtx, one warp per node
__global__ void k_arc_ends(const int64_t* row_ptr, const int32_t* adj, const int64_t* arc_off,
                           const uint32_t* arc_vtx, int64_t N, int32_t* arc_ends) {
  const int lane = threadIdx.x & 31;
  for (int64_t n = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; n < N;
       n += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t rb = row_ptr[n], d = row_ptr[n + 1] - rb;
    for (int64_t a = arc_off[n] + lane; a < arc_off[n + 1]; a += 32) {
      const uint32_t av = arc_vtx[a];
      const int64_t o = (av >> 16) & 255, ot = (int64_t)(av >> 24) - 1;
      arc_ends[2 * a] = o < d ? adj[rb + o] : -1;
      arc_ends[2 * a + 1] = ot >= 0 && ot < d ? adj[rb + ot] : -1;
    }
  }
}

// warp-aggregated bucketing of nodes by valence (keeps runs of nodes)
__global__ void k_bucket(const int64_t* row_ptr, int64_t N, int* cnt, int32_t* lists, int64_t cap) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) & ~31ll; base < N;
       base += (int64_t)gridDim.x * blockDim.x) {
    int64_t n = base + lane;
    int b = -1;
    if (n < N) {
      int d = (int)(row_ptr[n + 1] - row_ptr[n]);
      if (d > 0 && d <= LM_MAX_VALENCE) b = bucket_of(d);
    }
    for (int q = 0; q < NB_BUCKETS; q++) {
      uint32_t m = __ballot_sync(0xffffffffu, b == q);
      if (!m) continue;
      int start = 0;
      if (lane == __ffs(m) - 1) start = atomicAdd(&cnt[q], __popc(m));
      start = __shfl_sync(0xffffffffu, start, __ffs(m) - 1);
      if (b == q) lists[q * cap + start + __popc(m & ((1u << lane) - 1))] = (int32_t)n;
    }
  }
}

__global__ void k_mm_stats(const uint32_t* arc_vtx, int64_t A, const uint32_t* node_flags, int64_t N,
                           const int32_t* end_cnt, int64_t E2, unsigned long long* out) {
  // out: [0] circular arcs, [1] degenerate nodes, [2] flags OR, [3] max loop entries
  unsigned long long circ = 0, deg = 0, fl = 0, mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A; i += (int64_t)gridDim.x * blockDim.x)
    circ += (arc_vtx[i] >> 24) == 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    deg += (node_flags[i] & 2u) != 0;
    fl |= node_flags[i];
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E2; i += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, (unsigned long long)end_cnt[i]);
  for (int o = 16; o > 0; o >>= 1) {
    circ += __shfl_xor_sync(0xffffffffu, circ, o);
    deg += __shfl_xor_sync(0xffffffffu, deg, o);
    fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], circ);
    atomicAdd(&out[1], deg);
    atomicOr(&out[2], fl);
    atomicMax(&out[3], mx);
  }
}

int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

// ---- autotuner of the persistent meta-mesh launch: nodes a warp takes per
// queue access in each bucket and CTAs per SM, per device, lattice dtype and
// valence mix (the bucket shares in eighths); each candidate runs the count
// pass on a sample of every bucket and the fastest is cached for the process.
struct TuneKey {
  int dev, dtype, mix1, mix2, big;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, dtype, mix1, mix2, big) < std::tie(o.dev, o.dtype, o.mix1, o.mix2, o.big);
  }
};
struct TuneVal {
  int npt0, ctas_per_sm;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

template <typename T>
lm_status tune_launch(lm_metamesh* mm, const MMLaunch<T>& L, MMBuckets bk, const int hb[3], cudaStream_t st,
                      TuneVal* out) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int64_t tot = std::max<int64_t>(1, (int64_t)hb[0] + hb[1] + hb[2]);
  TuneKey key{dev, mm->dtype, (int)(8 * (int64_t)hb[1] / tot), (int)(8 * (int64_t)hb[2] / tot), hb[2] > 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *out = it->second;
      return LM_OK;
    }
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = metamesh_ctas_per_sm<T>();
  if (per_sm < 1) return LM_ERR_CUDA;
  // a sample of each bucket in proportion to the mix (the first nodes of
  // each list)
  const int cap = 16384;
  for (int b = 0; b < NB_BUCKETS; b++)
    bk.limit[b] = hb[b] == 0 ? 0 : (int)std::max<int64_t>(64, (int64_t)cap * hb[b] / tot);
  const int cand_npt[4] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  TuneVal bv{1, per_sm};
  for (int rep = 0; rep < 2; rep++)  // the first round warms up
    for (int c = per_sm; c >= std::max(1, per_sm - 2); c--)
      for (int j = 0; j < 4; j++) {
        bk.npt[0] = cand_npt[j];
        LM_CK(cudaMemsetAsync(bk.queues, 0, NB_BUCKETS * sizeof(int), st));
        cudaEventRecord(e0, st);
        LM_CK(launch_metamesh<T>(false, L, bk, c * sms, st, nullptr));
        cudaEventRecord(e1, st);
        LM_CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1 && ms < best) {
          best = ms;
          bv = TuneVal{cand_npt[j], c};
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *out = bv;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = bv;
  return LM_OK;
}

template <typename T>
lm_status build_impl(lm_metamesh* mm, cudaStream_t st) {
  const int64_t N = mm->N, E = mm->E;
  const T* xyz = (const T*)mm->xyz;
  const T* radii = (const T*)mm->radii;
  cudaEvent_t ev[6];
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], st);
  int* deg = nullptr;
  int* fill = nullptr;
  LM_CK(dalloc(mm, &mm->d_err, 4, st));
  LM_CK(dalloc(mm, &mm->d_queue, 8, st));
  LM_CK(dalloc(mm, &mm->d_misc, 8, st));
  LM_CK(dalloc(mm, &mm->d_acc, 4, st));
  LM_CK(dalloc(mm, &mm->d_fb, LM_N_FP64_COUNTS, st));
  LM_CK(cudaMemsetAsync(mm->d_fb, 0, LM_N_FP64_COUNTS * sizeof(unsigned long long), st));
  LM_CK(cudaMemsetAsync(mm->d_err, 0, 4 * sizeof(int), st));
  LM_CK(cudaMemsetAsync(mm->d_misc, 0, 8 * sizeof(int), st));
  LM_CK(cudaMemsetAsync(mm->d_queue, 0, 8 * sizeof(int), st));
  T* node_R = nullptr;
  LM_CK(dalloc(mm, &node_R, N, st));
  mm->node_R = node_R;
  LM_CK(dalloc(mm, &mm->row_ptr, N + 1, st));
  LM_CK(dalloc(mm, &mm->adj, 2 * E, st));
  LM_CK(dalloc(mm, &deg, N, st));
  LM_CK(dalloc(mm, &fill, N, st));
  LM_CK(cudaMemsetAsync(deg, 0, sizeof(int) * N, st));
  LM_CK(cudaMemsetAsync(fill, 0, sizeof(int) * N, st));
  mm->scan_ws_n = scan_ws_elems(std::max<int64_t>(std::max<int64_t>(N + E, 2 * E), 1));
  LM_CK(dalloc(mm, &mm->scan_ws, mm->scan_ws_n, st));
  // CSR build and bucketing, with no host synchronisation: input errors are
  // recorded on the device (every kernel skips invalid ids) and read at the
  // sizing synchronisation below, before anything is allocated from counts
  count_launch(); k_strut_validate<T><<<grid_for(E), 256, 0, st>>>(mm->ends, radii, E, N, deg, mm->d_err);
  LM_CK(cudaGetLastError());
  LM_CK(scan_excl<int>(deg, 1, N, mm->row_ptr, mm->scan_ws, st));
  count_launch(); k_scatter<<<grid_for(2 * E), 256, 0, st>>>(mm->ends, 2 * E, N, mm->row_ptr, fill, mm->adj);
  count_launch(); k_node_finalize<T><<<grid_for(N), 256, 0, st>>>(xyz, radii, N, mm->row_ptr, mm->adj, node_R, mm->d_err,
                                                 mm->d_misc);
  count_launch(); k_strut_taper<T><<<grid_for(E), 256, 0, st>>>(xyz, mm->ends, node_R, E, N, mm->d_err);
  LM_CK(cudaGetLastError());
  dfree(fill, st);
  // valence buckets (device-side counts)
  int32_t* lists = nullptr;
  int* bcnt = mm->d_misc + 4;
  const int64_t cap = std::max<int64_t>(N, 1);
  LM_CK(dalloc(mm, &lists, (int64_t)NB_BUCKETS * cap, st));
  count_launch(); k_bucket<<<grid_for(N), 256, 0, st>>>(mm->row_ptr, N, bcnt, lists, cap);
  LM_CK(cudaGetLastError());
  // ---- count pass
  int32_t *node_cnt = nullptr, *end_cnt = nullptr;
  LM_CK(dalloc(mm, &node_cnt, 4 * N, st));
  LM_CK(dalloc(mm, &end_cnt, 2 * E, st));
  LM_CK(dalloc(mm, &mm->node_flags, N, st));
  LM_CK(cudaMemsetAsync(node_cnt, 0, sizeof(int32_t) * 4 * N, st));
  LM_CK(cudaMemsetAsync(end_cnt, 0, sizeof(int32_t) * 2 * E, st));
  LM_CK(cudaMemsetAsync(mm->node_flags, 0, sizeof(uint32_t) * N, st));
  int* overflow = mm->d_misc + 1;
  MMLaunch<T> L{};
  L.xyz = xyz;
  L.ends = mm->ends;
  L.node_R = node_R;
  L.row_ptr = mm->row_ptr;
  L.adj = mm->adj;
  L.n_nodes = N;
  L.n_struts = E;
  L.err = mm->d_err;
  L.node_flags = mm->node_flags;
  L.node_cnt = node_cnt;
  L.end_cnt = end_cnt;
  L.overflow = overflow;
  L.fb = mm->d_fb;
  MMBuckets bk{};
  bk.lists = lists;
  bk.cap = cap;
  bk.counts = bcnt;
  bk.queues = mm->d_queue + 4;
  for (int b = 0; b < NB_BUCKETS; b++) bk.npt[b] = mm->opt.nodes_per_task > 0 ? mm->opt.nodes_per_task : 1;
  int ctas = mm->opt.grid_ctas;
  // arena of the count pass (replaces the emit pass for the nodes it holds):
  // up to 45 % of the free memory left beside the CSR offsets, at most about
  // 300 B per strut (a node's block is about 50 B per strut end); the CSR
  // arrays, about 1.05 times the arena's content, are allocated beside it
  // (if they do not fit, the arena is released and every node is emitted)
  MMArena arena{};
  void* arena_buf = nullptr;
  const double arena_want = (double)(sizeof(T) == 4 ? 300 : 400) * (double)E + 64.0 * (double)N + 65536.0;
  // per bucket, room to list up to 1/16 of the nodes that the arena could
  // not hold (the emit pass then computes only those)
  const int64_t mcap = N / 16 + 1024;
  auto arena_room = [&]() {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    {
      // memory the default pool keeps mapped but unused (lm_pool_retain) is
      // free for this build's allocations too
      int dev = 0;
      cudaMemPool_t pool;
      unsigned long long resv = 0, inuse = 0;
      if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess &&
          cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &resv) == cudaSuccess &&
          cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &inuse) == cudaSuccess && resv > inuse)
        fr += (size_t)(resv - inuse);
      (void)cudaGetLastError();
    }
    const double offs = 8.0 * (4.0 * (double)(N + 1) + 2.0 * (double)E + 1.0);
    double budget = 0.45 * std::max(0.0, (double)fr - offs);
    if (mm->opt.arena_bytes > 0) budget = std::min(budget, (double)mm->opt.arena_bytes);
    return budget - 8.0 * (double)std::max<int64_t>(N, 1) - 4.0 * NB_BUCKETS * (double)mcap - 4096.0;
  };
  if (mm->opt.arena_bytes >= 0) {
    double capb = std::min(arena_room(), arena_want);
    if (capb > 4096.0) {
      const size_t cap_bytes = ((size_t)capb) & ~(size_t)255;
      const size_t start_off = cap_bytes, ctr_off = start_off + (((size_t)8 * std::max<int64_t>(N, 1) + 255) & ~(size_t)255);
      const size_t ml_off = ctr_off + 256;
      if (mm_malloc(mm, &arena_buf, ml_off + (size_t)4 * NB_BUCKETS * (size_t)mcap, st) == cudaSuccess) {
        unsigned char* b = (unsigned char*)arena_buf;
        arena.buf = b;
        arena.cap = (int64_t)cap_bytes;
        arena.start = (int64_t*)(b + start_off);
        arena.used = (unsigned long long*)(b + ctr_off);
        arena.miss = (int*)(b + ctr_off + 8);
        arena.mcnt = (int*)(b + ctr_off + 16);
        arena.mlist = (int32_t*)(b + ml_off);
        arena.mcap = mcap;
        LM_CK(cudaMemsetAsync(b + ctr_off, 0, 64, st));
      } else {
        (void)cudaGetLastError();
        arena_buf = nullptr;
      }
    }
  }
  if (mm->opt.autotune) {
    // the tuner needs the valence mix and times its samples: the one extra
    // synchronisation of an autotuned build
    int hb[4] = {0, 0, 0, 0};
    int herr = 0;
    LM_CK(cudaMemcpyAsync(hb, bcnt, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CK(cudaMemcpyAsync(&herr, mm->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CK(cudaStreamSynchronize(st));
    if (herr == 0) {
      TuneVal tv{1, 0};
      lm_status ts = tune_launch<T>(mm, L, bk, hb, st, &tv);
      if (ts != LM_OK) return ts;
      if (mm->opt.nodes_per_task <= 0) bk.npt[0] = tv.npt0;
      if (ctas <= 0) {
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        ctas = tv.ctas_per_sm * sms;
      }
      // the sample runs counted their FP64 steps too
      LM_CK(cudaMemsetAsync(mm->d_fb, 0, LM_N_FP64_COUNTS * sizeof(unsigned long long), st));
      LM_CK(cudaMemsetAsync(overflow, 0, sizeof(int), st));
      if (arena_buf) LM_CK(cudaMemsetAsync(arena.used, 0, 64, st));
    }
  }
  for (int b = 0; b < NB_BUCKETS; b++) {
    mm->tuned[b][0] = MM_SLOTS[b];
    mm->tuned[b][1] = bk.npt[b];
  }
  if (arena_buf) L.arena = arena;
  LM_CK(cudaMemsetAsync(bk.queues, 0, NB_BUCKETS * sizeof(int), st));
  int used = 0;
  cudaEventRecord(ev[1], st);
  {
    NvtxRange r("meta-mesh count pass");
    LM_CK(launch_metamesh<T>(false, L, bk, ctas, st, &used));
  }
  cudaEventRecord(ev[2], st);
  // ---- sizing: offsets from the counts, and the one synchronisation
  LM_CK(dalloc(mm, &mm->vtx_off, N + 1, st));
  LM_CK(dalloc(mm, &mm->arc_off, N + 1, st));
  LM_CK(dalloc(mm, &mm->hole_off_n, N + 1, st));
  LM_CK(dalloc(mm, &mm->hent_off_n, N + 1, st));
  LM_CK(dalloc(mm, &mm->end_off, 2 * E + 1, st));
  LM_CK(scan_excl<int32_t>(node_cnt + 0, 4, N, mm->vtx_off, mm->scan_ws, st));
  LM_CK(scan_excl<int32_t>(node_cnt + 1, 4, N, mm->arc_off, mm->scan_ws, st));
  LM_CK(scan_excl<int32_t>(node_cnt + 2, 4, N, mm->hole_off_n, mm->scan_ws, st));
  LM_CK(scan_excl<int32_t>(node_cnt + 3, 4, N, mm->hent_off_n, mm->scan_ws, st));
  LM_CK(scan_excl<int32_t>(end_cnt, 1, 2 * E, mm->end_off, mm->scan_ws, st));
  int64_t tot[5];
  LM_CK(cudaMemcpyAsync(&tot[0], mm->vtx_off + N, 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&tot[1], mm->arc_off + N, 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&tot[2], mm->hole_off_n + N, 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&tot[3], mm->hent_off_n + N, 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&tot[4], mm->end_off + 2 * E, 8, cudaMemcpyDeviceToHost, st));
  int hmisc[4] = {0, 0, 0, 0};  // [0] max valence, [1] overflow
  int herr = 0, arena_miss = 0, mcnt[NB_BUCKETS] = {0, 0, 0};
  LM_CK(cudaMemcpyAsync(hmisc, mm->d_misc, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&herr, mm->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (arena_buf) {
    LM_CK(cudaMemcpyAsync(&arena_miss, arena.miss, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CK(cudaMemcpyAsync(mcnt, arena.mcnt, NB_BUCKETS * sizeof(int), cudaMemcpyDeviceToHost, st));
  }
  LM_CK(cudaStreamSynchronize(st));
  mm->max_valence = hmisc[0];
  if (herr != 0 || hmisc[1] != 0) {
    if (arena_buf) cudaFreeAsync(arena_buf, st);
    dfree(node_cnt, st);
    dfree(end_cnt, st);
    dfree(lists, st);
    dfree(deg, st);
    return herr != 0 ? (lm_status)herr : LM_ERR_CAPACITY;
  }
  mm->V = tot[0];
  mm->A = tot[1];
  mm->H = tot[2];
  mm->HE = tot[3];
  mm->LE = tot[4];
  T *vz = nullptr, *aphi = nullptr;
  auto alloc_out = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = dalloc(mm, &vz, 3 * mm->V, st)) != cudaSuccess) return e;
    if ((e = dalloc(mm, &mm->vtx_key, mm->V, st)) != cudaSuccess) return e;
    if ((e = dalloc(mm, &mm->vtx_flags, mm->V, st)) != cudaSuccess) return e;
    if ((e = dalloc(mm, &mm->vtx_gen, mm->V, st)) != cudaSuccess) return e;
    if ((e = dalloc(mm, &mm->arc_vtx, mm->A, st)) != cudaSuccess) return e;
    if ((e = dalloc(mm, &aphi, 2 * mm->A, st)) != cudaSuccess) return e;
    if ((e = dalloc(mm, &mm->loop_ent, mm->LE, st)) != cudaSuccess) return e;
    if ((e = dalloc(mm, &mm->hole_off, mm->H + 1, st)) != cudaSuccess) return e;
    return dalloc(mm, &mm->hole_ent, mm->HE, st);
  };
  cudaError_t ae = alloc_out();
  if (ae != cudaSuccess && arena_buf) {
    // no room beside the arena: release it and emit every node
    (void)cudaGetLastError();
    dfree(vz, st);
    dfree(mm->vtx_key, st);
    dfree(mm->vtx_flags, st);
    dfree(mm->vtx_gen, st);
    dfree(mm->arc_vtx, st);
    dfree(aphi, st);
    dfree(mm->loop_ent, st);
    dfree(mm->hole_off, st);
    dfree(mm->hole_ent, st);
    cudaFreeAsync(arena_buf, st);
    arena_buf = nullptr;
    arena = MMArena{};
    L.arena = MMArena{};
    ae = alloc_out();
  }
  LM_CK(ae);
  mm->vtx_z = vz;
  mm->arc_phi = aphi;
  LM_CK(cudaMemcpyAsync(mm->hole_off + mm->H, mm->hent_off_n + N, 8, cudaMemcpyDeviceToDevice, st));
  L.vtx_off = mm->vtx_off;
  L.arc_off = mm->arc_off;
  L.hole_off_n = mm->hole_off_n;
  L.hent_off_n = mm->hent_off_n;
  L.end_off = mm->end_off;
  L.vtx_z = vz;
  L.vtx_key = mm->vtx_key;
  L.vtx_flags = mm->vtx_flags;
  L.vtx_gen = mm->vtx_gen;
  L.arc_vtx = mm->arc_vtx;
  L.arc_phi = aphi;
  L.loop_ent = mm->loop_ent;
  L.hole_off = mm->hole_off;
  L.hole_ent = mm->hole_ent;
  // ---- outputs: nodes held by the arena go to their CSR ranges; the emit
  // pass computes only the others (none when the arena held every node)
  cudaEventRecord(ev[3], st);
  if (arena_buf) {
    L.arena = arena;
    LM_CK(launch_mm_gather<T>(L, st));
  }
  cudaEventRecord(ev[4], st);
  mm->emit_nodes = arena_buf ? arena_miss : N;
  mm->emit_listed = 0;
  if (!arena_buf || arena_miss > 0) {
    LM_CK(cudaMemsetAsync(bk.queues, 0, NB_BUCKETS * sizeof(int), st));
    bool listed = arena_buf != nullptr;
    for (int b = 0; b < NB_BUCKETS; b++) listed = listed && mcnt[b] <= mcap;
    mm->emit_listed = listed ? 1 : 0;
    if (listed) {
      // only the listed nodes (those the arena could not hold)
      MMBuckets bm = bk;
      bm.lists = arena.mlist;
      bm.cap = mcap;
      bm.counts = arena.mcnt;
      for (int b = 0; b < NB_BUCKETS; b++) bm.limit[b] = 0;
      LM_CK(launch_metamesh<T>(true, L, bm, ctas, st, &used));
    } else {
      LM_CK(launch_metamesh<T>(true, L, bk, ctas, st, &used));
    }
  }
  cudaEventRecord(ev[5], st);
  if (arena_buf) cudaFreeAsync(arena_buf, st);
  // statistics
  unsigned long long* dstat = nullptr;
  LM_CK(dalloc(mm, &dstat, 4, st));
  LM_CK(cudaMemsetAsync(dstat, 0, 4 * sizeof(unsigned long long), st));
  count_launch(); k_mm_stats<<<grid_for(std::max<int64_t>(std::max<int64_t>(mm->A, N), 2 * E)), 256, 0, st>>>(
      mm->arc_vtx, mm->A, mm->node_flags, N, end_cnt, 2 * E, dstat);
  // FP64 fallback contexts of the triangulation kernels, every context
  // starting as "no node" (node id -1)
  mm->scratch_warps = tri_scratch_warps();
  LM_CK(mm_malloc(mm, (void**)&mm->scratch, node64_bytes() * (size_t)mm->scratch_warps, st));
  LM_CK(cudaMemsetAsync(mm->scratch, 0xff, node64_bytes() * (size_t)mm->scratch_warps, st));
  unsigned long long hs[4];
  LM_CK(cudaMemcpyAsync(hs, dstat, sizeof(hs), cudaMemcpyDeviceToHost, st));
  LM_CK(cudaStreamSynchronize(st));
  mm->n_circ = (int64_t)hs[0];
  mm->n_ell = mm->A - mm->n_circ;
  mm->n_degenerate = (int64_t)hs[1];
  mm->flags_or = (uint32_t)hs[2];
  mm->max_loop_entries = (int)hs[3];
  cudaEventElapsedTime(&mm->t_csr, ev[0], ev[1]);
  cudaEventElapsedTime(&mm->t_count, ev[1], ev[2]);
  cudaEventElapsedTime(&mm->t_size, ev[2], ev[3]);
  cudaEventElapsedTime(&mm->t_gather, ev[3], ev[4]);
  cudaEventElapsedTime(&mm->t_emit, ev[4], ev[5]);
  for (auto& e : ev) cudaEventDestroy(e);
  dfree(dstat, st);
  dfree(node_cnt, st);
  dfree(end_cnt, st);
  dfree(lists, st);
  dfree(deg, st);
  return LM_OK;
}

template <typename T>
TriLaunch<T> tri_launch(lm_metamesh* mm) {
  TriLaunch<T> L{};
  L.xyz = (const T*)mm->xyz;
  L.ends = mm->ends;
  L.node_R = (const T*)mm->node_R;
  L.row_ptr = mm->row_ptr;
  L.adj = mm->adj;
  L.n_nodes = mm->N;
  L.n_struts = mm->E;
  L.vtx_off = mm->vtx_off;
  L.arc_off = mm->arc_off;
  L.end_off = mm->end_off;
  L.node_hole_off = mm->hole_off_n;
  L.hole_off = mm->hole_off;
  L.vtx_z = (const T*)mm->vtx_z;
  L.vtx_gen = mm->vtx_gen;
  L.arc_vtx = mm->arc_vtx;
  L.arc_phi = (const T*)mm->arc_phi;
  L.loop_ent = mm->loop_ent;
  L.hole_ent = mm->hole_ent;
  L.item_cnt = mm->item_cnt;
  L.tri_off = mm->tri_off;
  L.queue = mm->d_queue;
  L.err = mm->d_err;
  L.emax = std::max(mm->max_loop_entries, 1);
  L.pmax = std::max(mm->tri_pmax, 1);
  L.dmax = std::max(mm->max_valence, 1);
  L.max_pts = mm->d_misc + 2;
  L.scratch = mm->scratch;
  L.scratch_warps = mm->scratch_warps;
  L.fb = mm->d_fb;
  L.redo = mm->redo_bits;
  L.redo_base = 0;
  L.rlist = mm->redo_list;
  L.rcap = mm->redo_cap;
  L.aux = mm->aux_st;
  L.ev_fork = mm->ev_fork;
  L.ev_join = mm->ev_join;
  L.node_mask = mm->node_mask;
  return L;
}

// second stream and fork / join events of the hole fans (created once)
cudaError_t ensure_aux(lm_metamesh* mm) {
  if (mm->aux_st) return cudaSuccess;
  cudaError_t e = cudaEventCreateWithFlags(&mm->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mm->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&mm->aux_st, cudaStreamNonBlocking);
  return e;
}

template <typename T>
lm_status tri_count_impl(lm_metamesh* mm, int k, cudaStream_t st, int64_t* total) {
  const int64_t n_items = mm->E + mm->N;
  if (!mm->item_cnt) {
    LM_CK(dalloc(mm, &mm->item_cnt, n_items, st));
    LM_CK(dalloc(mm, &mm->tri_off, n_items + 1, st));
    LM_CK(dalloc(mm, &mm->redo_bits, mm->E / 32 + 1, st));
    // the deferred struts are rare (about 1 % on cone-strut lattices); more
    // than redo_cap in one call fall back to scanning the bitmap
    mm->redo_cap = mm->opt.redo_list_cap > 0
                       ? mm->opt.redo_list_cap
                       : std::min<int64_t>(std::max<int64_t>(mm->E / 32, 65536), (int64_t)1 << 24);
    LM_CK(dalloc(mm, &mm->redo_list, mm->redo_cap + 1, st));
  }
  LM_CK(cudaMemsetAsync(mm->d_misc + 2, 0, sizeof(int), st));
  TriLaunch<T> L = tri_launch<T>(mm);
  L.k = k;
  LM_CK(launch_tri_count<T>(L, st));
  LM_CK(scan_excl<int32_t>(mm->item_cnt, 1, n_items, mm->tri_off, mm->scan_ws, st));
  int64_t tot = 0;
  int mp = 0;
  LM_CK(cudaMemcpyAsync(&tot, mm->tri_off + n_items, 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&mp, mm->d_misc + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  LM_CK(cudaStreamSynchronize(st));
  mm->tri_k = k;
  mm->tri_total = tot;
  mm->tri_pmax = mp + 1;
  if (total) *total = tot;
  return LM_OK;
}

template <typename T>
lm_status tri_emit_impl(lm_metamesh* mm, int k, int64_t b, int64_t e, void* out, int64_t cap,
                        double* acc, cudaStream_t st) {
  LM_CK(ensure_aux(mm));
  LM_CK(cudaMemsetAsync(mm->d_queue, 0, 2 * sizeof(int), st));
  TriLaunch<T> L = tri_launch<T>(mm);
  L.k = k;
  L.item_begin = b;
  L.item_end = e;
  L.capacity = cap;
  L.first_ptr = mm->tri_off + b;
  L.out = (uint8_t*)out;
  L.acc = acc;
  LM_CK(launch_tri_emit<T>(L, st));
  return LM_OK;
}

// Two CUDA graphs for the chunk sequence of lm_triangulate_stream: graph q
// emits chunks q, q + 2, q + 4, ... into dbuf[q].  Its first node takes the
// next chunk of its sequence from a device cursor and writes the item range
// that the emit kernels read, so one instantiated graph replays every chunk
// of its parity with no host work besides the launch.
//   dev: device int64 [6] = cursor[2], range[2][2]
template <typename T>
lm_status chunk_graphs(lm_metamesh* mm, int k, int64_t chunk, int64_t i0, int64_t i1, uint8_t* dbuf[2],
                       int64_t cap, int64_t* dev, cudaGraphExec_t ex[2], long long* kernels_per_launch) {
  LM_CK(ensure_aux(mm));
  cudaStream_t cs;
  LM_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  lm_status s = LM_OK;
  for (int q = 0; q < 2 && s == LM_OK; q++) {
    TriLaunch<T> L = tri_launch<T>(mm);
    L.k = k;
    L.item_begin = i0;
    L.item_end = i1;  // host-side sizing only; the kernels read the range
    L.capacity = cap;
    L.first_ptr = nullptr;
    L.out = dbuf[q];
    L.acc = nullptr;
    L.range = dev + 2 + 2 * q;
    long long n0 = g_launches.load();
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) { s = LM_ERR_CUDA; break; }
    cudaError_t e0 = launch_chunk_begin(dev + q, 2, chunk, i0, i1, dev + 2 + 2 * q, cs);
    cudaError_t e1 = cudaMemsetAsync(mm->d_queue, 0, 2 * sizeof(int), cs);
    cudaError_t e2 = launch_tri_emit<T>(L, cs);
    cudaError_t e3 = cudaStreamEndCapture(cs, &g);
    long long n1 = g_launches.load();
    count_launch((int)-(n1 - n0));  // capture is not execution
    *kernels_per_launch = n1 - n0;
    if (e0 != cudaSuccess || e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || !g) {
      s = LM_ERR_CUDA;
      break;
    }
    if (cudaGraphInstantiate(&ex[q], g, 0) != cudaSuccess) s = LM_ERR_CUDA;
    cudaGraphDestroy(g);
  }
  cudaStreamDestroy(cs);
  return s;
}

bool valid_k(int k) { return k >= 1 && k <= 4096; }

// the library's FP32 angle functions on arrays (for tests of their error)
__global__ void k_eval_angle_fns(const float* y, const float* x, const float* a, int64_t n, float* at, float* sn,
                                 float* cs) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    at[i] = lm::lm_atan2(y[i], x[i]);
    float s, c;
    lm::lm_sincos(a[i], &s, &c);
    sn[i] = s;
    cs[i] = c;
  }
}

}  // namespace

extern "C" {

const char* lm_status_string(lm_status s) {
  switch (s) {
    case LM_OK: return "ok";
    case LM_ERR_INVALID_ARG: return "invalid argument";
    case LM_ERR_RADIUS_MISMATCH: return "strut-end radii disagree at a node";
    case LM_ERR_DEGENERATE: return "strut taper not smaller than its length";
    case LM_ERR_CAPACITY: return "capacity exceeded";
    case LM_ERR_OOM: return "device out of memory";
    case LM_ERR_CUDA: return "CUDA error";
    case LM_ERR_TIMEOUT: return "device wait timed out";
    case LM_ERR_VALENCE: return "node valence above LM_MAX_VALENCE";
    case LM_ERR_STATE: return "call order violated";
    case LM_ERR_IO: return "file could not be opened or written";
  }
  return "unknown status";
}

void lm_metamesh_free(lm_metamesh* mm) {
  if (!mm) return;
  cudaStream_t st = mm->st;
  cudaStreamSynchronize(st);
  void* ptrs[] = {mm->node_R, mm->row_ptr, mm->adj, mm->node_flags, mm->vtx_off, mm->arc_off,
                  mm->hole_off_n, mm->hent_off_n, mm->end_off, mm->vtx_z, mm->vtx_key, mm->vtx_flags,
                  mm->vtx_gen, mm->arc_ends, mm->arc_vtx, mm->arc_phi, mm->loop_ent, mm->hole_off,
                  mm->hole_ent, mm->item_cnt, mm->tri_off, mm->redo_bits, mm->redo_list, mm->scratch, mm->d_err, mm->d_queue,
                  mm->d_misc, mm->d_acc, mm->scan_ws, mm->d_fb};
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, st);
  cudaStreamSynchronize(st);
  if (mm->aux_st) {
    cudaStreamSynchronize(mm->aux_st);
    cudaStreamDestroy(mm->aux_st);
  }
  if (mm->ev_fork) cudaEventDestroy(mm->ev_fork);
  if (mm->ev_join) cudaEventDestroy(mm->ev_join);
  delete mm;
}

lm_status lm_build_metamesh(const lm_lattice* lat, const lm_options* opt, void* stream,
                            lm_metamesh** out) {
  NvtxRange nvtx_("lm_build_metamesh");
  if (!out) return LM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!lat || lat->n_nodes < 0 || lat->n_struts < 0 || (lat->dtype != LM_F32 && lat->dtype != LM_F64))
    return LM_ERR_INVALID_ARG;
  if (lat->n_struts > 0 && (!lat->node_xyz || !lat->strut_ends || !lat->end_radii))
    return LM_ERR_INVALID_ARG;
  if (2 * lat->n_struts >= (int64_t)0x7fffffff || lat->n_nodes >= (int64_t)0x7fffffff)
    return LM_ERR_INVALID_ARG;
  lm_metamesh* mm = new lm_metamesh();
  std::memset((void*)mm, 0, sizeof(*mm));
  mm->dtype = lat->dtype;
  mm->N = lat->n_nodes;
  mm->E = lat->n_struts;
  mm->xyz = lat->node_xyz;
  mm->ends = lat->strut_ends;
  mm->radii = lat->end_radii;
  if (opt) mm->opt = *opt;
  mm->st = (cudaStream_t)stream;
  mm->tri_k = 0;
  lm_status s = lat->dtype == LM_F32 ? build_impl<float>(mm, mm->st) : build_impl<double>(mm, mm->st);
  if (s != LM_OK) {
    lm_metamesh_free(mm);
    return s;
  }
  *out = mm;
  return LM_OK;
}

lm_status lm_metamesh_counts(const lm_metamesh* mm, int64_t out[8]) {
  if (!mm || !out) return LM_ERR_INVALID_ARG;
  out[0] = mm->V;
  out[1] = mm->n_ell;
  out[2] = mm->n_circ;
  out[3] = mm->H;
  out[4] = mm->E + mm->H;
  out[5] = mm->n_degenerate;
  out[6] = mm->max_valence;
  out[7] = mm->flags_or;
  return LM_OK;
}

lm_status lm_metamesh_export(lm_metamesh* mm, lm_metamesh_view* v) {
  if (!mm || !v) return LM_ERR_INVALID_ARG;
  if (!mm->arc_ends && mm->A > 0) {
    cudaStream_t st = mm->st;
    if (dalloc(mm, &mm->arc_ends, 2 * mm->A, st) != cudaSuccess) {
      (void)cudaGetLastError();
      mm->arc_ends = nullptr;
      return LM_ERR_OOM;
    }
    count_launch();
    k_arc_ends<<<grid_for(32 * mm->N), 256, 0, st>>>(mm->row_ptr, mm->adj, mm->arc_off, mm->arc_vtx, mm->N,
                                                     mm->arc_ends);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return st_cuda(e);
  }
  v->n_nodes = mm->N;
  v->n_struts = mm->E;
  v->n_vtx = mm->V;
  v->n_arcs = mm->A;
  v->n_loop_ent = mm->LE;
  v->n_holes = mm->H;
  v->n_hole_ent = mm->HE;
  v->dtype = mm->dtype;
  v->pad_ = 0;
  v->row_ptr = mm->row_ptr;
  v->adj = mm->adj;
  v->node_R = mm->node_R;
  v->node_flags = mm->node_flags;
  v->node_vtx_off = mm->vtx_off;
  v->vtx_z = mm->vtx_z;
  v->vtx_key = mm->vtx_key;
  v->vtx_flags = mm->vtx_flags;
  v->vtx_gen = mm->vtx_gen;
  v->node_arc_off = mm->arc_off;
  v->arc_ends = mm->arc_ends;
  v->arc_vtx = mm->arc_vtx;
  v->arc_phi = mm->arc_phi;
  v->end_loop_off = mm->end_off;
  v->loop_ent = mm->loop_ent;
  v->node_hole_off = mm->hole_off_n;
  v->hole_off = mm->hole_off;
  v->hole_ent = mm->hole_ent;
  return LM_OK;
}

lm_status lm_tri_count(lm_metamesh* mm, int32_t k, void* stream, int64_t* h_total) {
  NvtxRange nvtx_("lm_tri_count");
  if (!mm || !valid_k(k)) return LM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  return mm->dtype == LM_F32 ? tri_count_impl<float>(mm, k, st, h_total)
                             : tri_count_impl<double>(mm, k, st, h_total);
}

lm_status lm_tri_range(const lm_metamesh* mm, int64_t b, int64_t e, int64_t* h_first, int64_t* h_count) {
  if (!mm || b < 0 || e < b || e > mm->E + mm->N) return LM_ERR_INVALID_ARG;
  if (!mm->tri_k) return LM_ERR_STATE;
  int64_t x[2];
  if (cudaMemcpy(&x[0], mm->tri_off + b, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return LM_ERR_CUDA;
  if (cudaMemcpy(&x[1], mm->tri_off + e, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return LM_ERR_CUDA;
  if (h_first) *h_first = x[0];
  if (h_count) *h_count = x[1] - x[0];
  return LM_OK;
}

lm_status lm_triangulate(lm_metamesh* mm, int32_t k, int64_t b, int64_t e, void* d_out, int64_t cap,
                         void* stream) {
  NvtxRange nvtx_("lm_triangulate");
  if (!mm || !valid_k(k) || b < 0 || e < b || e > mm->E + mm->N || cap < 0) return LM_ERR_INVALID_ARG;
  if (mm->tri_k != k) return LM_ERR_STATE;
  if (!d_out && cap > 0) return LM_ERR_INVALID_ARG;
  if (e == b) return LM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  return mm->dtype == LM_F32 ? tri_emit_impl<float>(mm, k, b, e, d_out, cap, nullptr, st)
                             : tri_emit_impl<double>(mm, k, b, e, d_out, cap, nullptr, st);
}

lm_status lm_objective(lm_metamesh* mm, int32_t k, void* stream, double* h_area, double* h_volume) {
  if (!mm || !valid_k(k)) return LM_ERR_INVALID_ARG;
  if (mm->tri_k != k) return LM_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  LM_CK(cudaMemsetAsync(mm->d_acc, 0, 2 * sizeof(double), st));
  lm_status s = mm->dtype == LM_F32
                    ? tri_emit_impl<float>(mm, k, 0, mm->E + mm->N, nullptr, 0, mm->d_acc, st)
                    : tri_emit_impl<double>(mm, k, 0, mm->E + mm->N, nullptr, 0, mm->d_acc, st);
  if (s != LM_OK) return s;
  double h[2];
  LM_CK(cudaMemcpyAsync(h, mm->d_acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  LM_CK(cudaStreamSynchronize(st));
  if (h_area) *h_area = h[0];
  if (h_volume) *h_volume = h[1];
  return LM_OK;
}

lm_status lm_metamesh_build_times(const lm_metamesh* mm, float out[5]) {
  if (!mm || !out) return LM_ERR_INVALID_ARG;
  out[0] = mm->t_csr;
  out[1] = mm->t_count;
  out[2] = mm->t_size;
  out[3] = mm->t_gather;
  out[4] = mm->t_emit;
  return LM_OK;
}

lm_status lm_metamesh_launch_shape(const lm_metamesh* mm, int32_t out[8]) {
  if (!mm || !out) return LM_ERR_INVALID_ARG;
  for (int b = 0; b < 3; b++) {
    out[2 * b] = mm->tuned[b][0];
    out[2 * b + 1] = mm->tuned[b][1];
  }
  out[6] = (int32_t)mm->emit_nodes;
  out[7] = mm->emit_listed;
  return LM_OK;
}

lm_status lm_last_error(lm_metamesh* mm, void* stream) {
  if (!mm) return LM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int e = 0;
  LM_CK(cudaMemcpyAsync(&e, mm->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemsetAsync(mm->d_err, 0, sizeof(int), st));
  LM_CK(cudaStreamSynchronize(st));
  return (lm_status)e;
}

void lm_stl_header(uint8_t hdr[84], int64_t n_tris) {
  std::memset(hdr, 0, 84);
  const char* txt = "liblm binary STL (lattice meta-mesh triangulation)";
  std::memcpy(hdr, txt, std::strlen(txt));
  uint32_t c = n_tris > 0xffffffffll ? 0xffffffffu : (uint32_t)(n_tris < 0 ? 0 : n_tris);
  hdr[80] = c & 255;
  hdr[81] = (c >> 8) & 255;
  hdr[82] = (c >> 16) & 255;
  hdr[83] = (c >> 24) & 255;
}

}  // extern "C"

namespace {
// Writer of a binary-STL file, the third stage of the pipeline of Section
// 4.2.2 (GPU triangulation, device-to-host copy, disk): a host thread takes
// the chunks in order, waits for each chunk's copy into its pinned slot, and
// writes the records at their file offset; the streaming loop reuses a slot
// only once the writer has written it.
struct StlFileSink {
  struct Job {
    int64_t c;
    cudaEvent_t ev;
    const uint8_t* src;
    int64_t nbytes, off;
  };
  int fd = -1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job> q;
  int64_t written = 0;  // chunks written (in order)
  bool closed = false;
  int err = 0;  // errno of the first failed write
  double busy_s = 0.0, wait_s = 0.0;
  int64_t bytes = 0;
  std::thread th;

  static double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  }
  // write all of [p, p + n) at offset off; errno on failure, else 0
  static int write_all(int fd, const uint8_t* p, int64_t n, int64_t off) {
    while (n > 0) {
      const ssize_t r = pwrite(fd, p, (size_t)std::min<int64_t>(n, (int64_t)1 << 30), (off_t)off);
      if (r < 0) {
        if (errno == EINTR) continue;
        return errno;
      }
      if (r == 0) return EIO;
      p += r;
      n -= r;
      off += r;
    }
    return 0;
  }
  void run() {
    while (true) {
      Job j;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return !q.empty() || closed; });
        if (q.empty()) break;
        j = q.front();
        q.pop_front();
      }
      cudaEventSynchronize(j.ev);
      cudaEventDestroy(j.ev);
      int e = 0;
      double t0 = now();
      if (err == 0 && j.nbytes > 0) e = write_all(fd, j.src, j.nbytes, j.off);
      double dt = now() - t0;
      {
        std::lock_guard<std::mutex> lk(mu);
        busy_s += dt;
        if (e == 0 && err == 0) bytes += j.nbytes;
        if (e != 0 && err == 0) err = e;
        written = j.c + 1;
      }
      cv.notify_all();
    }
  }
  void start() { th = std::thread([this] { run(); }); }
  void push(const Job& j) {
    {
      std::lock_guard<std::mutex> lk(mu);
      q.push_back(j);
    }
    cv.notify_all();
  }
  // main thread: block until `n` chunks are written; false on a write error
  bool wait_written(int64_t n) {
    double t0 = now();
    std::unique_lock<std::mutex> lk(mu);
    cv.wait(lk, [&] { return written >= n || err != 0; });
    wait_s += now() - t0;
    return err == 0;
  }
  void close_and_join() {
    {
      std::lock_guard<std::mutex> lk(mu);
      closed = true;
    }
    cv.notify_all();
    if (th.joinable()) th.join();
  }
};

// Chunked triangulation into a pinned host ring (lm_triangulate_stream), the
// chunks handed to the callback or, with `fs`, to a file writer.
lm_status stream_impl(lm_metamesh* mm, int32_t k, int64_t chunk_items, void* h_ring, int64_t slot_bytes,
                      int32_t n_slots, lm_chunk_cb cb, void* user, void* stream, int64_t* h_total,
                      StlFileSink* fs, int64_t i0 = 0, int64_t i1 = -1) {
  cudaStream_t st = (cudaStream_t)stream;
  lm_status s = LM_OK;
  if (mm->tri_k != k) {
    s = lm_tri_count(mm, k, stream, nullptr);
    if (s != LM_OK) return s;
  }
  // items [i0, i1) (default: every item)
  if (i1 < 0) i1 = mm->E + mm->N;
  if (i0 < 0 || i0 > i1 || i1 > mm->E + mm->N) return LM_ERR_INVALID_ARG;
  const int64_t n_items = i1 - i0;
  const int64_t n_chunks = (n_items + chunk_items - 1) / chunk_items;
  // chunk boundaries (host copy of the offsets at chunk starts)
  std::vector<int64_t> bnd(n_chunks + 1);
  for (int64_t c = 0; c <= n_chunks; c++) {
    int64_t it = i0 + std::min(c * chunk_items, n_items);
    if (cudaMemcpyAsync(&bnd[c], mm->tri_off + it, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return LM_ERR_CUDA;
  }
  LM_CK(cudaStreamSynchronize(st));
  int64_t max_tris = 0;
  for (int64_t c = 0; c < n_chunks; c++) max_tris = std::max(max_tris, bnd[c + 1] - bnd[c]);
  if (max_tris * 50 > slot_bytes) return LM_ERR_CAPACITY;
  uint8_t* dbuf[2] = {nullptr, nullptr};
  cudaStream_t cs;
  LM_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t done_comp[2], done_copy[2];
  for (int q = 0; q < 2; q++) {
    LM_CK(cudaMallocAsync((void**)&dbuf[q], (size_t)std::max<int64_t>(max_tris, 1) * 50, st));
    cudaEventCreateWithFlags(&done_comp[q], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&done_copy[q], cudaEventDisableTiming);
  }
  std::vector<cudaEvent_t> copied(n_chunks);
  // chunk graphs: cursors start at chunks 0 and 1
  int64_t* gdev = nullptr;
  cudaGraphExec_t gex[2] = {nullptr, nullptr};
  long long kpl = 0;
  LM_CK(cudaMallocAsync((void**)&gdev, 6 * sizeof(int64_t), st));
  {
    const int64_t init[6] = {0, 1, 0, 0, 0, 0};
    LM_CK(cudaMemcpyAsync(gdev, init, sizeof(init), cudaMemcpyHostToDevice, st));
    LM_CK(cudaStreamSynchronize(st));
    s = mm->dtype == LM_F32 ? chunk_graphs<float>(mm, k, chunk_items, i0, i1, dbuf, max_tris, gdev, gex, &kpl)
                            : chunk_graphs<double>(mm, k, chunk_items, i0, i1, dbuf, max_tris, gdev, gex, &kpl);
  }
  for (int64_t c = 0; c < n_chunks && s == LM_OK; c++) {
    int q = (int)(c & 1);
    if (c >= 2) cudaStreamWaitEvent(st, done_copy[q], 0);
    cudaError_t ge = cudaGraphLaunch(gex[q], st);
    if (ge != cudaSuccess) {
      s = st_cuda(ge);
      break;
    }
    count_launch((int)kpl);
    cudaEventRecord(done_comp[q], st);
    // the host slot of chunk c was last used by chunk c - n_slots: wait for
    // its copy and hand it to the caller first (or, writing a file, wait
    // until the writer has written it)
    if (c >= n_slots && fs) {
      if (!fs->wait_written(c - n_slots + 1)) {
        s = LM_ERR_IO;
        break;
      }
    } else if (c >= n_slots) {
      cudaEventSynchronize(copied[c - n_slots]);
      cudaEventDestroy(copied[c - n_slots]);
      copied[c - n_slots] = nullptr;
      int64_t pc = c - n_slots;
      if (cb) cb(pc, i0 + pc * chunk_items, bnd[pc + 1] - bnd[pc], (uint8_t*)h_ring + (pc % n_slots) * slot_bytes, user);
    }
    cudaStreamWaitEvent(cs, done_comp[q], 0);
    int64_t nb = (bnd[c + 1] - bnd[c]) * 50;
    if (nb > 0) {
      cudaError_t ce = cudaMemcpyAsync((uint8_t*)h_ring + (c % n_slots) * slot_bytes, dbuf[q], nb,
                                       cudaMemcpyDeviceToHost, cs);
      if (ce != cudaSuccess) s = st_cuda(ce);
    }
    cudaEventRecord(done_copy[q], cs);
    cudaEventCreateWithFlags(&copied[c], cudaEventDisableTiming);
    cudaEventRecord(copied[c], cs);
    if (fs) {
      // the writer owns the event from here
      fs->push(StlFileSink::Job{c, copied[c], (const uint8_t*)h_ring + (c % n_slots) * slot_bytes, nb,
                                84 + 50 * bnd[c]});
      copied[c] = nullptr;
    }
  }
  if (fs) {
    fs->close_and_join();
    if (s == LM_OK && fs->err != 0) s = LM_ERR_IO;
  }
  for (int64_t c = std::max<int64_t>(0, n_chunks - n_slots); c < n_chunks && !fs; c++) {
    if (!copied[c]) continue;
    cudaEventSynchronize(copied[c]);
    cudaEventDestroy(copied[c]);
    if (cb && s == LM_OK) cb(c, i0 + c * chunk_items, bnd[c + 1] - bnd[c], (uint8_t*)h_ring + (c % n_slots) * slot_bytes, user);
  }
  cudaStreamSynchronize(cs);
  for (int q = 0; q < 2; q++)
    if (gex[q]) cudaGraphExecDestroy(gex[q]);
  cudaFreeAsync(gdev, st);
  for (int q = 0; q < 2; q++) {
    cudaFreeAsync(dbuf[q], st);
    cudaEventDestroy(done_comp[q]);
    cudaEventDestroy(done_copy[q]);
  }
  cudaStreamSynchronize(st);
  cudaStreamDestroy(cs);
  if (h_total) *h_total = bnd[n_chunks];
  if (s == LM_OK) s = lm_last_error(mm, stream);
  return s;
}

// ---- chunked meta-meshing and streaming (lm_stream_chunked)
// The lattice is meta-meshed in chunks of struts [s0, s1): the sub-lattice of
// a chunk holds its struts and every strut incident to their end nodes (the
// halo), renumbered in increasing global order, so each end node of the
// chunk's struts sees the same incident struts in the same order as in the
// whole lattice and its meta-mesh has the same bits.  The chunk emits its own
// struts and the hole fans of the nodes whose lowest-id strut is its own.

// degree of every node (ends outside [0, N) are reported, not counted)
__global__ void k_ck_deg(const int32_t* ends, int64_t E2, int64_t N, int* deg, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E2; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t n = ends[i];
    if (n < 0 || n >= N) {
      atomicCAS(err, 0, (int)LM_ERR_INVALID_ARG);
      continue;
    }
    atomicAdd(deg + n, 1);
  }
}
// strut ends of every node (order within a node irrelevant here)
__global__ void k_ck_fill(const int32_t* ends, int64_t E2, int64_t N, const int64_t* row, int* fill, int32_t* adj) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E2; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t n = ends[i];
    if (n < 0 || n >= N) continue;
    adj[row[n] + atomicAdd(fill + n, 1)] = (int32_t)i;
  }
}
// mark the struts incident to the end nodes of struts [s0, s1) (their own
// included) and the window of their ids
// the window of ids (below 2^31) seen by the threads of a warp: one atomic
// pair per warp
__device__ __forceinline__ void ck_window(unsigned lo, unsigned hi, unsigned long long* win) {
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0 && lo <= hi) {
    atomicMin(win, (unsigned long long)lo);
    atomicMax(win + 1, (unsigned long long)hi);
  }
}
__global__ void k_ck_mark_struts(const int32_t* ends, int64_t s0, int64_t s1, const int64_t* row,
                                 const int32_t* adj, uint8_t* smark, unsigned long long* win) {
  unsigned lo = 0xffffffffu, hi = 0u;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  // every thread of the grid runs the same number of rounds (the warp
  // reductions below need all lanes)
  for (int64_t s0t = s0 + blockIdx.x * (int64_t)blockDim.x; s0t < s1; s0t += st) {
    const int64_t s = s0t + threadIdx.x;
    if (s >= s1) continue;
    for (int side = 0; side < 2; side++) {
      const int64_t n = ends[2 * s + side];
      for (int64_t q = row[n]; q < row[n + 1]; q++) {
        const unsigned t = (unsigned)(adj[q] >> 1);
        smark[t] = 1;
        lo = t < lo ? t : lo;
        hi = t > hi ? t : hi;
      }
    }
  }
  ck_window(lo, hi, win);
}
// ids (lo + i) of the marked entries of mark[lo, lo + W), in increasing order
__global__ void k_ck_compact(const uint8_t* mark, int64_t lo, int64_t W, const int64_t* pos, int32_t* ids) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < W; i += (int64_t)gridDim.x * blockDim.x)
    if (mark[lo + i]) ids[pos[i]] = (int32_t)(lo + i);
}
// mark the end nodes of the sub-lattice's struts and the window of their ids
__global__ void k_ck_mark_nodes(const int32_t* ends, const int32_t* sub_struts, int64_t Es, uint8_t* nmark,
                                unsigned long long* win) {
  unsigned lo = 0xffffffffu, hi = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Es; i += (int64_t)gridDim.x * blockDim.x)
    for (int side = 0; side < 2; side++) {
      const unsigned n = (unsigned)ends[2 * (int64_t)sub_struts[i] + side];
      nmark[n] = 1;
      lo = n < lo ? n : lo;
      hi = n > hi ? n : hi;
    }
  ck_window(lo, hi, win);
}
// node renumbering and the sub-lattice's arrays
__global__ void k_ck_remap(const int32_t* sub_nodes, int64_t Ns, int32_t* remap) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < Ns; j += (int64_t)gridDim.x * blockDim.x)
    remap[sub_nodes[j]] = (int32_t)j;
}
template <typename T>
__global__ void k_ck_gather(const T* xyz, const int32_t* ends, const T* radii, const int32_t* sub_struts, int64_t Es,
                            const int32_t* sub_nodes, int64_t Ns, const int32_t* remap, T* xyz_s, int32_t* ends_s,
                            T* radii_s) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = tid; j < Ns; j += st)
    for (int c = 0; c < 3; c++) xyz_s[3 * j + c] = xyz[3 * (int64_t)sub_nodes[j] + c];
  for (int64_t i = tid; i < Es; i += st) {
    const int64_t g = sub_struts[i];
    ends_s[2 * i] = remap[ends[2 * g]];
    ends_s[2 * i + 1] = remap[ends[2 * g + 1]];
    radii_s[2 * i] = radii[2 * g];
    radii_s[2 * i + 1] = radii[2 * g + 1];
  }
}
// a node is owned by the chunk whose struts include its lowest-id strut
__global__ void k_ck_owned(const int64_t* row, const int32_t* adj, int64_t Ns, int64_t a, int64_t b, uint8_t* own) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < Ns; n += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = -1;
    for (int64_t q = row[n]; q < row[n + 1]; q++) {
      const int64_t t = adj[q] >> 1;
      if (lo < 0 || t < lo) lo = t;
    }
    own[n] = (uint8_t)(lo >= a && lo < b);
  }
}

// grid of 256-thread blocks for n grid-strided items: at most 32 blocks per SM
int ck_grid(int64_t n) {
  static thread_local int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  }
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)sms * 32) g = (int64_t)sms * 32;
  return (int)(g < 1 ? 1 : g);
}

// one chunk's sub-lattice and meta-mesh
struct CkChunk {
  int64_t s0 = 0, s1 = 0, Es = 0, Ns = 0, a = 0, b = 0;
  void *xyz = nullptr, *radii = nullptr;
  int32_t* ends = nullptr;
  uint8_t* own = nullptr;
  lm_metamesh* mm = nullptr;
  lm_status st = LM_OK;
};

struct CkShared {
  const lm_lattice* lat;
  const lm_options* opt;
  int64_t N, E;
  size_t tsz;
  int64_t *row, *pos, *ws;
  int32_t *adj, *remap, *sub_struts, *sub_nodes;
  uint8_t *smark, *nmark;
  unsigned long long* win;  // [4]: strut window, node window
  cudaStream_t st;
};

lm_status ck_free(CkChunk& c, cudaStream_t st) {
  if (c.mm) lm_metamesh_free(c.mm);
  c.mm = nullptr;
  if (c.xyz) cudaFreeAsync(c.xyz, st);
  if (c.radii) cudaFreeAsync(c.radii, st);
  if (c.ends) cudaFreeAsync(c.ends, st);
  if (c.own) cudaFreeAsync(c.own, st);
  c.xyz = c.radii = nullptr;
  c.ends = nullptr;
  c.own = nullptr;
  return cudaStreamSynchronize(st) == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

// sub-lattice of struts [s0, s1) with its halo, then its meta-mesh and the
// ownership mask of its nodes (every call synchronises sh.st)
lm_status ck_prepare(CkShared& sh, CkChunk& c) {
  NvtxRange nvtx_("chunk build");
  cudaStream_t st = sh.st;
  const unsigned long long init[4] = {~0ull, 0ull, ~0ull, 0ull};
  LM_CK(cudaMemcpyAsync(sh.win, init, sizeof(init), cudaMemcpyHostToDevice, st));
  const int32_t* ends = sh.lat->strut_ends;
  count_launch();
  k_ck_mark_struts<<<ck_grid(c.s1 - c.s0), 256, 0, st>>>(ends, c.s0, c.s1, sh.row, sh.adj, sh.smark, sh.win);
  unsigned long long w[4];
  LM_CK(cudaMemcpyAsync(w, sh.win, sizeof(w), cudaMemcpyDeviceToHost, st));
  LM_CK(cudaStreamSynchronize(st));
  const int64_t slo = (int64_t)w[0], sW = (int64_t)w[1] - slo + 1;
  LM_CK(scan_excl<uint8_t>(sh.smark + slo, 1, sW, sh.pos, sh.ws, st));
  int64_t ab[2];
  LM_CK(cudaMemcpyAsync(&ab[0], sh.pos + (c.s0 - slo), 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&ab[1], sh.pos + sW, 8, cudaMemcpyDeviceToHost, st));
  count_launch();
  k_ck_compact<<<ck_grid(sW), 256, 0, st>>>(sh.smark, slo, sW, sh.pos, sh.sub_struts);
  LM_CK(cudaStreamSynchronize(st));
  c.a = ab[0];
  c.b = c.a + (c.s1 - c.s0);
  c.Es = ab[1];
  // every strut of [s0, s1) is incident to its own end nodes, so all are in
  // the sub-lattice (a defensive check before the ranges are used)
  if (c.b > c.Es || c.a < 0) return LM_ERR_STATE;
  count_launch();
  k_ck_mark_nodes<<<ck_grid(c.Es), 256, 0, st>>>(ends, sh.sub_struts, c.Es, sh.nmark, sh.win + 2);
  LM_CK(cudaMemcpyAsync(w, sh.win, sizeof(w), cudaMemcpyDeviceToHost, st));
  LM_CK(cudaStreamSynchronize(st));
  const int64_t nlo = (int64_t)w[2], nW = (int64_t)w[3] - nlo + 1;
  LM_CK(scan_excl<uint8_t>(sh.nmark + nlo, 1, nW, sh.pos, sh.ws, st));
  LM_CK(cudaMemcpyAsync(&c.Ns, sh.pos + nW, 8, cudaMemcpyDeviceToHost, st));
  count_launch();
  k_ck_compact<<<ck_grid(nW), 256, 0, st>>>(sh.nmark, nlo, nW, sh.pos, sh.sub_nodes);
  LM_CK(cudaStreamSynchronize(st));
  count_launch();
  k_ck_remap<<<ck_grid(c.Ns), 256, 0, st>>>(sh.sub_nodes, c.Ns, sh.remap);
  LM_CK(cudaMallocAsync(&c.xyz, sh.tsz * 3 * (size_t)std::max<int64_t>(c.Ns, 1), st));
  LM_CK(cudaMallocAsync(&c.radii, sh.tsz * 2 * (size_t)std::max<int64_t>(c.Es, 1), st));
  LM_CK(cudaMallocAsync((void**)&c.ends, 8 * (size_t)std::max<int64_t>(c.Es, 1), st));
  count_launch();
  if (sh.tsz == 4)
    k_ck_gather<float><<<ck_grid(std::max(c.Es, c.Ns)), 256, 0, st>>>(
        (const float*)sh.lat->node_xyz, ends, (const float*)sh.lat->end_radii, sh.sub_struts, c.Es, sh.sub_nodes,
        c.Ns, sh.remap, (float*)c.xyz, c.ends, (float*)c.radii);
  else
    k_ck_gather<double><<<ck_grid(std::max(c.Es, c.Ns)), 256, 0, st>>>(
        (const double*)sh.lat->node_xyz, ends, (const double*)sh.lat->end_radii, sh.sub_struts, c.Es, sh.sub_nodes,
        c.Ns, sh.remap, (double*)c.xyz, c.ends, (double*)c.radii);
  LM_CK(cudaGetLastError());
  // clear the marks for the next chunk
  LM_CK(cudaMemsetAsync(sh.smark + slo, 0, (size_t)sW, st));
  LM_CK(cudaMemsetAsync(sh.nmark + nlo, 0, (size_t)nW, st));
  lm_lattice sub{};
  sub.n_nodes = c.Ns;
  sub.n_struts = c.Es;
  sub.dtype = sh.lat->dtype;
  sub.node_xyz = c.xyz;
  sub.strut_ends = c.ends;
  sub.end_radii = c.radii;
  lm_status s = lm_build_metamesh(&sub, sh.opt, (void*)st, &c.mm);
  if (s != LM_OK) return s;
  LM_CK(cudaMallocAsync((void**)&c.own, (size_t)std::max<int64_t>(c.Ns, 1), st));
  count_launch();
  k_ck_owned<<<ck_grid(c.Ns), 256, 0, st>>>(c.mm->row_ptr, c.mm->adj, c.Ns, c.a, c.b, c.own);
  LM_CK(cudaGetLastError());
  LM_CK(cudaStreamSynchronize(st));
  c.mm->node_mask = c.own;
  return LM_OK;
}

struct CkCb {
  lm_kchunk_cb cb;
  void* user;
  int32_t k;
  int64_t* seq;
};
void ck_trampoline(int64_t, int64_t first_item, int64_t n_tris, void* slot, void* u) {
  CkCb* w = (CkCb*)u;
  if (w->cb) w->cb((*w->seq)++, w->k, first_item, n_tris, slot, w->user);
}

// one chunk's triangles at every k: its own struts, then its owned nodes'
// holes, through the ring (items per streamed chunk from the slot and the
// mean triangle count of the range, halved until the largest chunk fits)
lm_status ck_stream(CkChunk& c, const int32_t* ks, int32_t n_k, void* h_ring, int64_t slot_bytes,
                    int32_t n_slots, lm_kchunk_cb cb, void* user, cudaStream_t st, int64_t* seq, int64_t* tris) {
  for (int32_t q = 0; q < n_k; q++) {
    lm_status s = lm_tri_count(c.mm, ks[q], (void*)st, nullptr);
    if (s != LM_OK) return s;
    const int64_t rng[2][2] = {{c.a, c.b}, {c.Es, c.Es + c.Ns}};
    for (int r = 0; r < 2; r++) {
      const int64_t i0 = rng[r][0], i1 = rng[r][1];
      if (i1 <= i0) continue;
      int64_t t0 = 0, t1 = 0;
      LM_CK(cudaMemcpyAsync(&t0, c.mm->tri_off + i0, 8, cudaMemcpyDeviceToHost, st));
      LM_CK(cudaMemcpyAsync(&t1, c.mm->tri_off + i1, 8, cudaMemcpyDeviceToHost, st));
      LM_CK(cudaStreamSynchronize(st));
      if (t1 == t0) continue;
      const double per = std::max(1.0, (double)(t1 - t0) / (double)(i1 - i0));
      int64_t chunk = std::max<int64_t>(1, (int64_t)(0.5 * (double)slot_bytes / (50.0 * per)));
      CkCb w{cb, user, ks[q], seq};
      int64_t got = 0;
      while (true) {
        s = stream_impl(c.mm, ks[q], chunk, h_ring, slot_bytes, n_slots, ck_trampoline, &w, (void*)st, &got,
                        nullptr, i0, i1);
        if (s != LM_ERR_CAPACITY || chunk == 1) break;
        chunk /= 2;
      }
      if (s != LM_OK) return s;
      tris[q] += got - t0;
    }
  }
  return LM_OK;
}
}  // namespace

extern "C" {

lm_status lm_triangulate_stream(lm_metamesh* mm, int32_t k, int64_t chunk_items, void* h_ring,
                                int64_t slot_bytes, int32_t n_slots, lm_chunk_cb cb, void* user,
                                void* stream, int64_t* h_total) {
  NvtxRange nvtx_("lm_triangulate_stream");
  if (!mm || !valid_k(k) || chunk_items <= 0 || !h_ring || slot_bytes <= 0 || n_slots < 2)
    return LM_ERR_INVALID_ARG;
  return stream_impl(mm, k, chunk_items, h_ring, slot_bytes, n_slots, cb, user, stream, h_total, nullptr);
}

lm_status lm_stream_chunked(const lm_lattice* lat, const lm_options* opt, const int32_t* ks, int32_t n_k,
                            int64_t build_struts, void* h_ring, int64_t slot_bytes, int32_t n_slots,
                            lm_kchunk_cb cb, void* user, void* stream, int64_t* h_tris) {
  NvtxRange nvtx_("lm_stream_chunked");
  if (!lat || !ks || n_k < 1 || build_struts < 1 || !h_ring || slot_bytes < 50 || n_slots < 2 || !h_tris ||
      lat->n_nodes < 0 || lat->n_struts < 0 || lat->n_nodes >= 2147483647ll || lat->n_struts >= 1073741823ll ||
      (lat->dtype != LM_F32 && lat->dtype != LM_F64) ||
      (lat->n_struts > 0 && (!lat->node_xyz || !lat->strut_ends || !lat->end_radii)))
    return LM_ERR_INVALID_ARG;
  for (int32_t q = 0; q < n_k; q++) {
    if (!valid_k(ks[q])) return LM_ERR_INVALID_ARG;
    h_tris[q] = 0;
  }
  const int64_t N = lat->n_nodes, E = lat->n_struts;
  if (E == 0) return LM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // the chunk builds run on a stream of their own (on a helper thread, beside
  // the previous chunk's streaming)
  cudaStream_t bst;
  LM_CK(cudaStreamCreateWithFlags(&bst, cudaStreamNonBlocking));
  {
    // the build stream starts after the caller's stream has produced the
    // lattice (a non-blocking stream does not wait for the legacy stream)
    cudaEvent_t ready;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, st) != cudaSuccess || cudaStreamWaitEvent(bst, ready, 0) != cudaSuccess) {
      cudaStreamDestroy(bst);
      return LM_ERR_CUDA;
    }
    cudaEventDestroy(ready);
  }
  CkShared sh{};
  sh.lat = lat;
  sh.opt = opt;
  sh.N = N;
  sh.E = E;
  sh.tsz = lat->dtype == LM_F32 ? 4 : 8;
  sh.st = bst;
  lm_status s = LM_OK;
  int* dev_int = nullptr;  // [N] degrees / fill counters, [1] error
  auto fail = [&](lm_status x) {
    if (s == LM_OK) s = x;
  };
  const int64_t wsn = scan_ws_elems(std::max(N, E) + 1);
  auto al = [&](void** p, size_t b) {
    if (s == LM_OK && cudaMallocAsync(p, std::max<size_t>(b, 1), bst) != cudaSuccess) fail(LM_ERR_OOM);
  };
  al((void**)&dev_int, 4 * (size_t)(N + 1));
  al((void**)&sh.row, 8 * (size_t)(N + 1));
  al((void**)&sh.adj, 4 * (size_t)(2 * E));
  al((void**)&sh.pos, 8 * (size_t)(std::max(N, E) + 1));
  al((void**)&sh.ws, 8 * (size_t)wsn);
  al((void**)&sh.remap, 4 * (size_t)N);
  al((void**)&sh.sub_struts, 4 * (size_t)E);
  al((void**)&sh.sub_nodes, 4 * (size_t)N);
  al((void**)&sh.smark, (size_t)E);
  al((void**)&sh.nmark, (size_t)N);
  al((void**)&sh.win, 4 * sizeof(unsigned long long));
  if (s == LM_OK) {
    // full CSR of the strut ends (the halo of every chunk comes from it)
    int herr = 0;
    if (cudaMemsetAsync(dev_int, 0, 4 * (size_t)(N + 1), bst) != cudaSuccess) fail(LM_ERR_CUDA);
    count_launch();
    k_ck_deg<<<ck_grid(2 * E), 256, 0, bst>>>(lat->strut_ends, 2 * E, N, dev_int, dev_int + N);
    if (s == LM_OK && scan_excl<int>(dev_int, 1, N, sh.row, sh.ws, bst) != cudaSuccess) fail(LM_ERR_CUDA);
    if (s == LM_OK && cudaMemcpyAsync(&herr, dev_int + N, 4, cudaMemcpyDeviceToHost, bst) != cudaSuccess)
      fail(LM_ERR_CUDA);
    if (s == LM_OK && cudaMemsetAsync(dev_int, 0, 4 * (size_t)N, bst) != cudaSuccess) fail(LM_ERR_CUDA);
    count_launch();
    k_ck_fill<<<ck_grid(2 * E), 256, 0, bst>>>(lat->strut_ends, 2 * E, N, sh.row, dev_int, sh.adj);
    if (s == LM_OK && cudaMemsetAsync(sh.smark, 0, (size_t)E, bst) != cudaSuccess) fail(LM_ERR_CUDA);
    if (s == LM_OK && cudaMemsetAsync(sh.nmark, 0, (size_t)N, bst) != cudaSuccess) fail(LM_ERR_CUDA);
    if (cudaStreamSynchronize(bst) != cudaSuccess) fail(LM_ERR_CUDA);
    if (herr != 0) fail((lm_status)herr);
  }
  const int64_t n_chunks = (E + build_struts - 1) / build_struts;
  CkChunk cur, nxt;
  int64_t seq = 0;
  if (s == LM_OK) {
    cur.s0 = 0;
    cur.s1 = std::min(E, build_struts);
    fail(ck_prepare(sh, cur));
  }
  for (int64_t c = 0; c < n_chunks && s == LM_OK; c++) {
    std::thread helper;
    lm_status hs = LM_OK;
    if (c + 1 < n_chunks) {
      nxt = CkChunk{};
      nxt.s0 = (c + 1) * build_struts;
      nxt.s1 = std::min(E, nxt.s0 + build_struts);
      int dev = 0;
      cudaGetDevice(&dev);
      helper = std::thread([&, dev] {
        cudaSetDevice(dev);
        hs = ck_prepare(sh, nxt);
      });
    }
    fail(ck_stream(cur, ks, n_k, h_ring, slot_bytes, n_slots, cb, user, st, &seq, h_tris));
    if (helper.joinable()) helper.join();
    fail(ck_free(cur, bst));
    fail(hs);
    cur = nxt;
    nxt = CkChunk{};
  }
  ck_free(cur, bst);
  ck_free(nxt, bst);
  for (void* p : {(void*)dev_int, (void*)sh.row, (void*)sh.adj, (void*)sh.pos, (void*)sh.ws, (void*)sh.remap,
                  (void*)sh.sub_struts, (void*)sh.sub_nodes, (void*)sh.smark, (void*)sh.nmark, (void*)sh.win})
    if (p) cudaFreeAsync(p, bst);
  cudaStreamSynchronize(bst);
  cudaStreamDestroy(bst);
  return s;
}

lm_status lm_triangulate_to_file(lm_metamesh* mm, int32_t k, const char* path, int64_t chunk_items,
                                 void* h_ring, int64_t slot_bytes, int32_t n_slots, int32_t flags,
                                 void* stream, int64_t* h_total, double h_stats[4]) {
  NvtxRange nvtx_("lm_triangulate_to_file");
  if (!mm || !valid_k(k) || !path || !h_ring || slot_bytes < 50 || n_slots < 2) return LM_ERR_INVALID_ARG;
  lm_status s = LM_OK;
  if (mm->tri_k != k) {
    s = lm_tri_count(mm, k, stream, nullptr);
    if (s != LM_OK) return s;
  }
  const int64_t n_items = mm->E + mm->N;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t total = 0, strut_tris = 0;
  LM_CK(cudaMemcpyAsync(&total, mm->tri_off + n_items, 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaMemcpyAsync(&strut_tris, mm->tri_off + mm->E, 8, cudaMemcpyDeviceToHost, st));
  LM_CK(cudaStreamSynchronize(st));
  if (chunk_items <= 0) {
    // Eq. chunk-size: N_batch = S_buffer / (S_triangle N_strut), with the
    // mean triangle count of a strut for N_strut and 80 % of a slot for
    // S_buffer; halved while some chunk's records would not fit a slot
    const double per_strut = std::max(1.0, (double)strut_tris / (double)std::max<int64_t>(mm->E, 1));
    chunk_items = std::max<int64_t>(1, (int64_t)(0.8 * (double)slot_bytes / (50.0 * per_strut)));
    while (chunk_items > 1) {
      const int64_t nc = (n_items + chunk_items - 1) / chunk_items;
      std::vector<int64_t> b(nc + 1);
      for (int64_t c = 0; c <= nc; c++)
        LM_CK(cudaMemcpyAsync(&b[c], mm->tri_off + std::min(c * chunk_items, n_items), 8, cudaMemcpyDeviceToHost, st));
      LM_CK(cudaStreamSynchronize(st));
      int64_t mx = 0;
      for (int64_t c = 0; c < nc; c++) mx = std::max(mx, b[c + 1] - b[c]);
      if (50 * mx <= slot_bytes) break;
      chunk_items /= 2;
    }
  }
  const int fd = open(path, O_WRONLY | O_CREAT | O_TRUNC, 0644);
  if (fd < 0) return LM_ERR_IO;
  uint8_t hdr[84];
  lm_stl_header(hdr, total);
  StlFileSink fs;
  fs.fd = fd;
  const double t0 = StlFileSink::now();
  if (StlFileSink::write_all(fd, hdr, 84, 0) != 0) {
    close(fd);
    return LM_ERR_IO;
  }
  fs.bytes = 84;
  fs.start();
  int64_t got = 0;
  s = stream_impl(mm, k, chunk_items, h_ring, slot_bytes, n_slots, nullptr, nullptr, stream, &got, &fs);
  fs.close_and_join();
  double sync_s = 0.0;
  if (s == LM_OK && (flags & LM_FILE_SYNC)) {
    const double ts = StlFileSink::now();
    if (fsync(fd) != 0) s = LM_ERR_IO;
    sync_s = StlFileSink::now() - ts;
  }
  if (close(fd) != 0 && s == LM_OK) s = LM_ERR_IO;
  if (h_total) *h_total = got;
  if (h_stats) {
    h_stats[0] = StlFileSink::now() - t0;
    h_stats[1] = fs.busy_s;
    h_stats[2] = fs.wait_s;
    h_stats[3] = sync_s;
  }
  return s;
}

long long lm_launch_count(void) { return g_launches.load(); }

const char* lm_cuda_error_string(void) { return cudaGetErrorString(g_last_cuda); }

lm_status lm_pool_retain(uint64_t bytes) {
  int dev = 0;
  cudaMemPool_t pool;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, dev);
  if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &bytes);
  if (e == cudaSuccess && bytes == 0) e = cudaMemPoolTrimTo(pool, 0);
  return e == cudaSuccess ? LM_OK : st_cuda(e);
}

lm_status lm_eval_angle_fns(const float* d_y, const float* d_x, const float* d_a, int64_t n, float* d_atan2,
                            float* d_sin, float* d_cos, void* stream) {
  if (n < 0 || (n > 0 && (!d_y || !d_x || !d_a || !d_atan2 || !d_sin || !d_cos))) return LM_ERR_INVALID_ARG;
  if (n == 0) return LM_OK;
  count_launch();
  k_eval_angle_fns<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(d_y, d_x, d_a, n, d_atan2, d_sin, d_cos);
  return cudaGetLastError() == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

lm_status lm_fp64_counts(const lm_metamesh* mm, int64_t out[LM_N_FP64_COUNTS]) {
  if (!mm || !out) return LM_ERR_INVALID_ARG;
  unsigned long long h[LM_N_FP64_COUNTS];
  if (cudaMemcpy(h, mm->d_fb, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return LM_ERR_CUDA;
  for (int i = 0; i < LM_N_FP64_COUNTS; i++) out[i] = (int64_t)h[i];
  return LM_OK;
}

lm_status lm_copy_to_host(void* h_dst, const void* d_src, int64_t bytes) {
  if (bytes < 0 || (bytes > 0 && (!h_dst || !d_src))) return LM_ERR_INVALID_ARG;
  if (bytes == 0) return LM_OK;
  return cudaMemcpy(h_dst, d_src, (size_t)bytes, cudaMemcpyDeviceToHost) == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

lm_status lm_metamesh_backward(lm_metamesh* mm, int32_t k, double w_area, double w_vol, void* d_grad_xyz,
                               void* d_grad_r, void* stream, double* h_area, double* h_volume) {
  NvtxRange nvtx_("lm_metamesh_backward");
  if (!mm || !valid_k(k)) return LM_ERR_INVALID_ARG;
  lm_status s = LM_OK;
  if (mm->tri_k != k) {
    s = lm_tri_count(mm, k, stream, nullptr);
    if (s != LM_OK) return s;
  }
  s = lm_objective(mm, k, stream, h_area, h_volume);
  if (s != LM_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = mm->dtype == LM_F32
                      ? lm::metamesh_backward<float>(mm, k, w_area, w_vol, d_grad_xyz, d_grad_r, st)
                      : lm::metamesh_backward<double>(mm, k, w_area, w_vol, d_grad_xyz, d_grad_r, st);
  if (e != cudaSuccess) return st_cuda(e);
  return lm_last_error(mm, stream);
}

}  // extern "C"
