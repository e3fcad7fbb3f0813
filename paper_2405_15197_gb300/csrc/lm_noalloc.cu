// Allocation-free triangulation entry point.
//
// lm_triangulate_noalloc emits the same STL records as lm_tri_count + lm_triangulate
// for one item range, for callers that cannot allocate device memory at that
// point: code that runs while a stream is being captured into a CUDA graph, or
// under an external memory budget / custom allocator that forbids the library
// from calling cudaMalloc.  All scratch it needs (per-item triangle counts and
// offsets of the range, the scan workspace, the FP64 fallback contexts of its
// warps and its work counters) lives in one file-scope __device__ array of
// fixed size, which every GPU that loads the library keeps until exit.
#include <cuda_runtime.h>

#include <mutex>

#include "lm_internal.h"
#include "lm_scan.cuh"
#include "lm_tri.cuh"

using namespace lm;

namespace {

constexpr int64_t NA_MAX_ITEMS = 1 << 18;  // items per call
constexpr int NA_CONTEXTS = 512;           // FP64 contexts: 2 per warp, 256 warps
constexpr int64_t NA_SCAN_WS = 2 * ((NA_MAX_ITEMS + SCAN_TILE - 1) / SCAN_TILE) + 8;

struct NaLayout {
  int32_t cnt[NA_MAX_ITEMS];
  int64_t off[NA_MAX_ITEMS + 1];
  int64_t ws[NA_SCAN_WS];
  uint32_t redo[NA_MAX_ITEMS / 32 + 2];  // struts deferred to the FP64 pass
  unsigned long long rlist[NA_MAX_ITEMS / 16 + 1];  // the same, listed (count first)
  int counters[8];  // [0..1] work queues, [2] max points of one loop
};
constexpr size_t NA_CTX_OFFSET = (sizeof(NaLayout) + 255) & ~(size_t)255;
constexpr size_t NA_BYTES = NA_CTX_OFFSET + (size_t)NA_CONTEXTS * sizeof(Node64);

// the scratch (about 7 MB); host code must not use this name as an address
__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_na_mu;
unsigned char* g_na_ptr[256] = {nullptr};

// device address of the scratch on the current device (set up on first use)
cudaError_t na_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = (unsigned char*)p;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

// triangle count of items [b, e) (same rules as the full count pass)
template <typename T>
__global__ void __launch_bounds__(256) k_count_range(TriArgs<T> A, Node64* ctxs, int64_t b, int64_t e,
                                                     int32_t* cnt, int* max_pts) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  Node64* ctx = ctxs + gw;
  const int64_t E = A.lat.n_struts;
  for (int64_t base = b + (int64_t)gw * 32; base < e; base += (int64_t)nwarps * 32) {
    int64_t it = base + lane;
    int64_t cs[2] = {0, 0};
    bool need = false;
    int64_t nodes[2] = {-1, -1};
    if (it < e) {
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
        if (lane == src) {
          int64_t ao = A.arc_off[nd];
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
    int mx = (int)(cs[0] > cs[1] ? cs[0] : cs[1]);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0 && mx > 0) atomicMax(max_pts, mx);
    if (it < e) cnt[it - b] = (int32_t)(cs[0] + cs[1]);
  }
}

template <typename T>
lm_status run_noalloc(lm_metamesh* mm, int k, int64_t b, int64_t e, void* d_out, int64_t cap,
                      cudaStream_t st, int64_t* h_ntris) {
  unsigned char* base = nullptr;
  if (na_scratch(&base) != cudaSuccess) return LM_ERR_CUDA;
  NaLayout* S = reinterpret_cast<NaLayout*>(base);
  Node64* ctx = reinterpret_cast<Node64*>(base + NA_CTX_OFFSET);
  const int64_t n = e - b;
  // the array keeps the previous call's contents: reset counters and mark
  // every FP64 context empty
  if (cudaMemsetAsync(S->counters, 0, sizeof(S->counters), st) != cudaSuccess) return LM_ERR_CUDA;
  if (cudaMemsetAsync(ctx, 0xff, (size_t)NA_CONTEXTS * sizeof(Node64), st) != cudaSuccess) return LM_ERR_CUDA;
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
  A.err = mm->d_err;
  const int threads = 256;
  int64_t grid = (n + threads - 1) / threads;
  if (grid > NA_CONTEXTS / (threads / 32)) grid = NA_CONTEXTS / (threads / 32);
  if (grid < 1) grid = 1;
  count_launch();
  k_count_range<T><<<(unsigned)grid, threads, 0, st>>>(A, ctx, b, e, S->cnt, &S->counters[2]);
  if (cudaGetLastError() != cudaSuccess) return LM_ERR_CUDA;
  if (scan_excl<int32_t>(S->cnt, 1, n, S->off, S->ws, st) != cudaSuccess) return LM_ERR_CUDA;
  int64_t total = 0;
  int maxp = 0;
  if (cudaMemcpyAsync(&total, &S->off[n], sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&maxp, &S->counters[2], sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return LM_ERR_CUDA;
  if (h_ntris) *h_ntris = total;
  if (n == 0 || total == 0) return LM_OK;
  if (cudaMemsetAsync(ctx, 0xff, (size_t)NA_CONTEXTS * sizeof(Node64), st) != cudaSuccess) return LM_ERR_CUDA;
  TriLaunch<T> L{};
  L.xyz = A.lat.xyz;
  L.ends = A.lat.ends;
  L.node_R = A.lat.node_R;
  L.row_ptr = A.lat.row_ptr;
  L.adj = A.lat.adj;
  L.n_nodes = mm->N;
  L.n_struts = mm->E;
  L.vtx_off = A.vtx_off;
  L.arc_off = A.arc_off;
  L.end_off = A.end_off;
  L.node_hole_off = A.node_hole_off;
  L.hole_off = A.hole_off;
  L.vtx_z = A.vtx_z;
  L.vtx_gen = A.vtx_gen;
  L.arc_vtx = A.arc_vtx;
  L.arc_phi = A.arc_phi;
  L.loop_ent = A.loop_ent;
  L.hole_ent = A.hole_ent;
  L.k = k;
  L.tri_off = S->off - b;  // indexed by global item id
  L.first_ptr = S->off;    // = 0
  L.item_begin = b;
  L.item_end = e;
  L.capacity = cap;
  L.out = (uint8_t*)d_out;
  L.acc = nullptr;
  L.queue = S->counters;
  L.err = mm->d_err;
  L.emax = mm->max_loop_entries > 0 ? mm->max_loop_entries : 1;
  L.pmax = maxp + 1;
  L.dmax = mm->max_valence > 0 ? mm->max_valence : 1;
  L.max_pts = nullptr;
  L.scratch = ctx;
  L.scratch_warps = NA_CONTEXTS;
  L.redo = S->redo;
  L.redo_base = b;
  L.rlist = S->rlist;
  L.rcap = NA_MAX_ITEMS / 16;
  return launch_tri_emit<T>(L, st) == cudaSuccess ? LM_OK : LM_ERR_CUDA;
}

}  // namespace

extern "C" lm_status lm_triangulate_noalloc(lm_metamesh* mm, int32_t k, int64_t item_begin,
                                            int64_t item_end, void* d_out, int64_t capacity_tris,
                                            void* stream, int64_t* h_ntris) {
  if (!mm || k < 1 || k > 4096 || item_begin < 0 || item_end < item_begin ||
      item_end > mm->E + mm->N || capacity_tris < 0 || (!d_out && capacity_tris > 0))
    return LM_ERR_INVALID_ARG;
  if (item_end - item_begin > NA_MAX_ITEMS) return LM_ERR_CAPACITY;
  cudaStream_t st = (cudaStream_t)stream;
  return mm->dtype == LM_F32 ? run_noalloc<float>(mm, k, item_begin, item_end, d_out, capacity_tris, st, h_ntris)
                             : run_noalloc<double>(mm, k, item_begin, item_end, d_out, capacity_tris, st, h_ntris);
}
