// Allocation-free triangulation entry point.
//
// lm_triangulate_noalloc emits the same STL records as lm_tri_count +
// lm_triangulate for one item range without allocating device memory.  It is
// for callers whose device memory is not theirs to request at that point: an
// application whose framework's caching allocator or fixed memory pool owns
// the GPU's memory (a cudaMalloc from the library could fail, or force the
// pool to release cached blocks), or a latency-bound serving loop in which a
// cudaMalloc / cudaFree would stall the device.  All scratch it needs
// (per-item triangle counts and offsets of the range, the scan workspace,
// the FP64 fallback contexts of its warps, its work counters) lives in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "lm_internal.h"
#include "lm_scan.cuh"
#include "lm_tri.cuh"

using namespace lm;

namespace {

constexpr int64_t NA_MAX_ITEMS = 1 << 18;  // items per call
// FP64 contexts (Node64) in the array: the count pass uses one per warp of
// its grid (at most NA_CONTEXTS warps of NA_COUNT_THREADS / 32), the hole
// fans two per warp (launch_tri_holes clamps its grid to scratch_warps / 2
// warps), the FP64 stitching pass none
constexpr int NA_CONTEXTS = 512;
constexpr int NA_COUNT_THREADS = 256;
constexpr int64_t NA_SCAN_WS = 2 * ((NA_MAX_ITEMS + SCAN_TILE - 1) / SCAN_TILE) + 8;

// count-pass grid of n items: one warp per 32 items, at most one FP64
// context per warp
int64_t count_grid(int64_t n) {
  constexpr int64_t max_blocks = NA_CONTEXTS / (NA_COUNT_THREADS / 32);
  static_assert(max_blocks * (NA_COUNT_THREADS / 32) <= NA_CONTEXTS, "count pass: one context per warp");
  int64_t g = (n + NA_COUNT_THREADS - 1) / NA_COUNT_THREADS;
  return g < 1 ? 1 : (g > max_blocks ? max_blocks : g);
}

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
  // the count kernel of lm_tri_count on the range: one FP64 context per warp
  const int64_t grid = count_grid(n);
  count_launch();
  k_tri_count<T><<<(unsigned)grid, NA_COUNT_THREADS, 0, st>>>(A, ctx, b, e, S->cnt, &S->counters[2]);
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
