// Internal declarations shared by the liblm translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/liblm.h"

struct lm_metamesh;

namespace lm {

struct Node64;

// valence buckets of the meta-mesh kernel
enum { NB_BUCKETS = 3 };
// warps of a meta-mesh block working on each bucket: the block's shared
// memory holds four workspaces of the first bucket (d <= 16), two of the
// second (d <= 32) or one of the third (d <= 64)
constexpr int MM_BLOCK_WARPS = 4;
constexpr int MM_SLOTS[3] = {4, 2, 1};
__host__ __device__ inline int bucket_of(int d) { return d <= 16 ? 0 : (d <= 32 ? 1 : 2); }

// Arena of the meta-mesh count pass: each node's output, stashed in one
// atomically reserved block, so that a gather into the CSR layout replaces
// the emit pass (nodes that do not fit go through the emit pass).
struct MMArena {
  unsigned char* buf;
  unsigned long long* used;  // bytes reserved so far
  int64_t cap;               // bytes
  int64_t* start;            // [N] byte offset of each node's block; < 0: not stored
  int* miss;                 // nodes not stored
  // the nodes not stored, listed per valence bucket ([3][mcap]; counts in
  // mcnt[3], which may exceed mcap: the emit pass then takes every node)
  int32_t* mlist;
  int* mcnt;
  int64_t mcap;
};

// Layout of one node's block (byte offsets): vertex positions, keys,
// generators; arc vertices (owner and other local end included: the gather
// derives the arcs' global end ids from them), angles; hole starts (relative
// to the node's first hole entry); hole entries; vertex flags (one byte
// each); loop entries of its ends in adjacency order (last: the other
// offsets do not depend on their number).  Blocks are 8-byte aligned.
struct ArenaBlock {
  int64_t vz, vkey, vgen, avtx, aphi, ho, he, vfl, le, bytes;
};
__host__ __device__ inline int64_t arena_a8(int64_t x) { return (x + 7) & ~(int64_t)7; }
__host__ __device__ inline ArenaBlock arena_block(int64_t nv, int64_t na, int64_t nh, int64_t nhe, int64_t nle,
                                                  int64_t tsz) {
  ArenaBlock b;
  int64_t o = 0;
  b.vz = o;
  o = arena_a8(o + 3 * tsz * nv);
  b.vkey = o;
  o += 8 * nv;
  b.vgen = o;
  o += 4 * nv;
  b.avtx = o;
  o = arena_a8(o + 4 * na);
  b.aphi = o;
  o += 2 * tsz * na;
  b.ho = o;
  o += 4 * nh;
  b.he = o;
  o += 4 * nhe;
  b.vfl = o;
  o = (o + nv + 3) & ~(int64_t)3;
  b.le = o;  // loop entries as 16 bits: node-local arc (< 2^15) | rev << 15, 0xffff unmatched
  o += 2 * nle;
  b.bytes = arena_a8(o);
  return b;
}

// Valence buckets of the persistent meta-mesh launch (device-side counts:
// no host synchronisation between the bucketing and the launch).
struct MMBuckets {
  const int32_t* lists;  // [3][cap] node lists
  int64_t cap;           // stride between the lists
  const int* counts;     // device [3]: nodes in each list
  int limit[3];          // > 0: at most this many nodes of a list (autotuner samples)
  int* queues;           // device [3]: work counters, zero at launch
  int npt[3];            // nodes a warp takes per queue access
};

template <typename T>
struct MMLaunch {
  // inputs
  const T* xyz;
  const int32_t* ends;
  const T* node_R;
  const int64_t* row_ptr;
  const int32_t* adj;
  int64_t n_nodes, n_struts;
  const int* err;  // input errors of the CSR build (the launch does nothing then)
  uint32_t* node_flags;
  int32_t* node_cnt;
  int32_t* end_cnt;
  const int64_t *vtx_off, *arc_off, *hole_off_n, *hent_off_n, *end_off;
  T* vtx_z;
  uint64_t* vtx_key;
  uint32_t* vtx_flags;
  uint32_t* vtx_gen;
  uint32_t* arc_vtx;
  T* arc_phi;
  uint32_t* loop_ent;
  int64_t* hole_off;
  uint32_t* hole_ent;
  int* overflow;
  unsigned long long* fb;
  MMArena arena;  // arena.start NULL: none
};

// the persistent meta-mesh launch over every valence bucket; grid_ctas <= 0:
// resident CTAs x SM count.  Returns the CTAs launched in *used_ctas.
template <typename T>
cudaError_t launch_metamesh(bool emit, const MMLaunch<T>& a, const MMBuckets& bk, int grid_ctas,
                            cudaStream_t st, int* used_ctas);
// resident CTAs per SM of the meta-mesh launch
template <typename T>
int metamesh_ctas_per_sm();
// copy the arena-stored nodes into the CSR layout (the launch's output arrays
// and offsets)
template <typename T>
cudaError_t launch_mm_gather(const MMLaunch<T>& a, cudaStream_t st);

template <typename T>
struct TriLaunch {
  const T* xyz;
  const int32_t* ends;
  const T* node_R;
  const int64_t* row_ptr;
  const int32_t* adj;
  int64_t n_nodes, n_struts;
  const int64_t *vtx_off, *arc_off, *end_off, *node_hole_off, *hole_off;
  const T* vtx_z;
  const uint32_t* vtx_gen;
  const uint32_t* arc_vtx;
  const T* arc_phi;
  const uint32_t* loop_ent;
  const uint32_t* hole_ent;
  int k;
  int32_t* item_cnt;
  const int64_t* tri_off;
  int64_t item_begin, item_end, capacity;
  const int64_t* first_ptr;  // device: tri_off + item_begin
  uint8_t* out;
  double* acc;
  int* queue;  // 2 counters
  int* err;
  int pmax, emax;
  int dmax;  // largest node valence
  int* max_pts;
  Node64* scratch;
  int64_t scratch_warps;
  unsigned long long* fb;
  uint32_t* redo;     // bitmap of struts deferred to the FP64 pass (bit e - redo_base)
  int64_t redo_base;
  unsigned long long* rlist;  // [1 + rcap]: count, then the deferred struts (NULL: bitmap only)
  int64_t rcap;
  const int64_t* range;  // device-side [begin, end) overriding item_begin/end, or NULL
  const uint8_t* node_mask;  // [N]: hole items of nodes with 0 count no triangles (NULL: all)
  // second stream for the hole fans, which then run beside the strut passes
  // (fork and join through the two events); NULL: everything on one stream
  cudaStream_t aux;
  cudaEvent_t ev_fork, ev_join;
};

template <typename T>
cudaError_t launch_tri_count(const TriLaunch<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_tri_emit(const TriLaunch<T>& a, cudaStream_t st);
// adjoint (lm_bwd.cu): gradients of w_area area + w_vol volume at k added
// into gxyz [N][3] and gr [N] (lattice dtype); requires the counts at k
template <typename T>
cudaError_t metamesh_backward(lm_metamesh* mm, int k, double w_area, double w_vol, void* gxyz, void* gr,
                              cudaStream_t st);
// first node of a chunk graph (see lm_triangulate_stream)
cudaError_t launch_chunk_begin(int64_t* cursor, int64_t stride, int64_t chunk, int64_t i0, int64_t i1, int64_t* range,
                               cudaStream_t st);
size_t node64_bytes();
int64_t tri_scratch_warps();
// host-side count of kernels this library launched (all threads)
void count_launch(int n = 1);

}  // namespace lm

struct lm_metamesh {
  int dtype;
  int64_t N, E;
  const void* xyz;
  const int32_t* ends;
  const void* radii;
  lm_options opt;
  cudaStream_t st;
  cudaStream_t aux_st;             // hole fans beside the strut passes (created on first use)
  cudaEvent_t ev_fork, ev_join;
  // CSR and per-node data
  void* node_R;
  int64_t* row_ptr;
  int32_t* adj;
  uint32_t* node_flags;
  int max_valence;
  int max_loop_entries;
  // meta-mesh
  int64_t *vtx_off, *arc_off, *hole_off_n, *hent_off_n, *end_off;
  void* vtx_z;
  uint64_t* vtx_key;
  uint32_t *vtx_flags, *vtx_gen;
  int32_t* arc_ends;  // derived on the first export (not used by the kernels)
  uint32_t* arc_vtx;
  void* arc_phi;
  uint32_t* loop_ent;
  int64_t* hole_off;
  uint32_t* hole_ent;
  int64_t V, A, LE, H, HE;
  const uint8_t* node_mask;  // [N] or NULL: see TriLaunch::node_mask (chunked streaming)
  int64_t emit_nodes;  // nodes the build's emit pass computed again
  int emit_listed;     // the emit pass took only the listed missed nodes
  int64_t n_ell, n_circ, n_degenerate;
  uint32_t flags_or;
  // triangulation state (one k at a time)
  int tri_k;
  int32_t* item_cnt;
  int64_t* tri_off;
  uint32_t* redo_bits;  // [E/32 + 1]: struts deferred to the FP64 stitching pass
  unsigned long long* redo_list;  // [1 + redo_cap]: the same struts, listed
  int64_t redo_cap;
  int64_t tri_total;
  int tri_pmax;
  lm::Node64* scratch;
  int64_t scratch_warps;
  int* d_err;
  int* d_queue;
  int* d_misc;
  double* d_acc;
  int64_t* scan_ws;
  int64_t scan_ws_n;
  // timing of the last build (device ms): csr, count, sizing (scans, host
  // sync, output allocation), arena gather, emit pass
  float t_csr, t_count, t_size, t_gather, t_emit;
  // FP64 stability-step counters: [0..7] meta-mesh build, [8..15] triangulation
  unsigned long long* d_fb;
  // launch shape of the meta-mesh kernel per valence bucket (block warps,
  // nodes per queue access), as used by the last build
  int tuned[3][2];
  // device bytes allocated for this handle so far (cumulative)
  int64_t alloc_bytes;
};
