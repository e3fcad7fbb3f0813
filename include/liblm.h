/*
 * liblm -- GB300-native lattice meta-meshing and resolution-k triangulation.
 *
 * C ABI of the data-parallel hot path of "Warp-centric GPU meta-meshing and
 * fast triangulation of billion-scale lattice structures" (Zou & Gao, CAD;
 * arXiv 2405.15197).  All pointers named d_* are device pointers (CUDA
 * global memory of the current device); h_* are host pointers.  `stream` is
 * a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 * asynchronous on that stream unless documented as synchronising.
 *
 * Ownership: the caller owns every input and output buffer; the library
 * owns the meta-mesh handle and the device memory behind it (allocated with
 * cudaMallocAsync on the call's stream).  The lattice arrays passed to
 * lm_build_metamesh must stay valid and unchanged until lm_metamesh_free,
 * because triangulation and the adjoint re-derive strut geometry from them.
 *
 * Errors: every call returns an lm_status; no exception crosses the ABI.
 * Per-node geometric degeneracies do not fail a call: they are counted and
 * flagged per node (LM_NODE_* bits) and those nodes still produce output.
 *
 * Lattice model (Section 4.1 of the paper): each node is a sphere whose
 * radius is a property of the node; each strut is the cone (a cylinder when
 * both node radii are equal) tangent to the spheres of its two end nodes.
 */
#ifndef LIBLM_H
#define LIBLM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LM_OK = 0,
  LM_ERR_INVALID_ARG = 1,     /* NULL pointer, bad size, node id out of range,
                                 a strut joining a node to itself, radius <= 0
                                 or NaN, coordinate NaN, k out of [1, 4096] */
  LM_ERR_RADIUS_MISMATCH = 2, /* two strut ends at one node carry radii that
                                 differ by more than 1e-12 relative */
  LM_ERR_DEGENERATE = 3,      /* a strut with |R_a - R_b| >= its length */
  LM_ERR_CAPACITY = 4,        /* an output or per-node work buffer too small */
  LM_ERR_OOM = 5,             /* device allocation failed */
  LM_ERR_CUDA = 6,            /* a CUDA runtime call failed */
  LM_ERR_TIMEOUT = 7,         /* reserved: no kernel of this library waits on
                                 another, so no call returns it */
  LM_ERR_VALENCE = 8,         /* a node with more than LM_MAX_VALENCE struts */
  LM_ERR_STATE = 9,           /* call order violated (e.g. triangulate before
                                 lm_tri_count for that k) */
  LM_ERR_IO = 10              /* a file could not be opened or written */
} lm_status;

enum { LM_F32 = 0, LM_F64 = 1 };
enum { LM_MAX_VALENCE = 64 };

/* per-node flag bits (lm_metamesh_view.node_flags) */
enum {
  LM_NODE_NEAR_TANGENT = 1,  /* an active strut pair within 1e-6 of tangency:
                                exempt from bit-exact comparisons */
  LM_NODE_DEGENERATE = 2,    /* the node violates a validity condition of the
                                lattice model (reasons below) */
  LM_NODE_INCONSISTENT = 4,  /* loops of two struts disagree on a shared arc */
  LM_NODE_BEYOND_LENGTH = 8, /* a vertex lies past a strut's far tangency circle */
  LM_NODE_STEEP_PAIR = 16,   /* an active pair whose plane section is not an ellipse */
  LM_NODE_SEAM_CUT = 32,     /* a vertex-free loop lies on a plane, not the sphere */
  LM_NODE_ANGLE_TIE = 64,    /* two vertices of one loop at the same angle */
  LM_NODE_LINE_ALONG_CONE = 128,
  LM_NODE_OVERFLOW = 256     /* node exceeded a per-node work capacity */
};

/* per-vertex flag bits */
enum { LM_VTX_SPHERE = 1, LM_VTX_SEAM = 2 };

/* Input lattice (Section 4.3.1 notation: strut S_i with end vertices
 * v_i^0, v_i^1 and radii r_i^0, r_i^1).
 *   node_xyz   : device, [n_nodes][3] of dtype (float or double)
 *   strut_ends : device, [n_struts][2] int32 node ids
 *   end_radii  : device, [n_struts][2] of dtype; must equal the radius of
 *                the node each end sits on (node property)            */
typedef struct {
  int64_t n_nodes, n_struts;
  int32_t dtype; /* LM_F32 or LM_F64 */
  int32_t pad_;
  const void* node_xyz;
  const int32_t* strut_ends;
  const void* end_radii;
} lm_lattice;

/* Tuning knobs; zero-initialised = library defaults.
 *   autotune      : 1 = time the candidate launch shapes of the persistent
 *                   meta-mesh launch (nodes a warp takes per queue access,
 *                   CTAs per SM) on a sample of the lattice's nodes, once
 *                   per device, dtype and valence mix (the shares of the
 *                   valence buckets), cache the winner (host memory) and use
 *                   it; costs one extra synchronisation per build
 *   block_warps   : unused (the meta-mesh blocks have four warps: four
 *                   workspaces for nodes of valence <= 16, two for <= 32,
 *                   one for <= 64)
 *   grid_ctas     : persistent grid size (0 = resident CTAs x SM count)
 *   nodes_per_task: nodes a warp pops from the work queue at once (0 = 1)
 *   arena_bytes   : device memory for the count pass to keep each node's
 *                   meta-mesh, so that a gather into the CSR layout replaces
 *                   the emit pass for the nodes it holds (0 = up to 45 % of
 *                   the memory free beside the CSR offsets, memory the pool
 *                   keeps mapped included; < 0 = none:
 *                   every node is emitted);
 *                   the result is the same either way
 *   redo_list_cap : capacity of the list of struts the FP32 stitching pass
 *                   defers to the FP64 pass (0 = max(E/32, 65,536), at most
 *                   2^24); a call that defers more scans the deferral bitmap
 *                   instead (same result)
 *   mem_budget    : > 0: device allocations that would take the bytes this
 *                   handle has allocated (cumulative, temporaries included)
 *                   past this budget fail as an out-of-memory device would
 *                   (LM_ERR_OOM); a hook for exercising the failure path    */
typedef struct {
  int32_t autotune;
  int32_t block_warps;
  int32_t grid_ctas;
  int32_t nodes_per_task;
  int64_t arena_bytes;
  int64_t redo_list_cap;
  int64_t mem_budget;
  int64_t reserved[1];
} lm_options;

typedef struct lm_metamesh lm_metamesh;

/* Build the meta-mesh (Section 4.3: auxiliary planes P_ij, strut-plane
 * ellipses, ellipse-plane trimming, arc loops; Section 5: hole flags).
 * Runs the node-sorted CSR build, the valence bucketing and one persistent,
 * work-stealing meta-mesh launch over nodes of every valence (Section
 * 4.3.3's warp scheduling) on `stream` with no host synchronisation between
 * them; synchronises the stream once to size the outputs (input errors are
 * reported then) and once at the end for the totals.
 *   lat  : input lattice (device arrays, see lm_lattice)
 *   opt  : NULL = defaults
 *   out  : receives the handle (NULL on error)                           */
lm_status lm_build_metamesh(const lm_lattice* lat, const lm_options* opt, void* stream,
                            lm_metamesh** out);

/* Totals of the meta-mesh (Section 4.1, "Meta-mesh definition": the
 * vertices, circular / elliptical arcs and trimmed strut surfaces that bound
 * the lattice; Section 5's hole contours are the circular-arc loops left on
 * the nodal spheres).  Host values, read after the build's synchronisation;
 * no device work.
 *   out   : host, 8 int64: [0] vertices, [1] elliptical arcs, [2] circular
 *           arcs, [3] holes, [4] faces (struts + holes), [5] nodes flagged
 *           LM_NODE_DEGENERATE, [6] max valence, [7] OR of all node flags
 * Returns LM_ERR_INVALID_ARG for a NULL handle or array.                 */
lm_status lm_metamesh_counts(const lm_metamesh* mm, int64_t out[8]);

/* Device views of the meta-mesh arrays (Section 4.1's vertices, arcs and arc
 * loops in the layout of Section 4.3.2, "Coalesced-access memory layout": an
 * index region of prefix sums (the *_off arrays, one CSR range per node or
 * strut end) over structure-of-arrays data).  Library-owned device memory,
 * valid until lm_metamesh_free; the call fills `view` on the host.  arc_ends
 * is not kept by the build (no kernel reads it; it follows from arc_vtx and
 * the CSR): the first call derives it on the handle's stream (one allocation
 * of 8 B per arc and one kernel, synchronised), later calls reuse it.
 * Returns LM_ERR_INVALID_ARG for a NULL handle or view, LM_ERR_OOM or
 * LM_ERR_CUDA if that first derivation fails.
 * Node-local vertex and arc ids index from node_vtx_off[n] / node_arc_off[n].
 *   vtx_z     : [V][3] dtype, vertex position relative to its node centre
 *   arc_ends  : [A][2] int32 global strut-end ids (2*strut+side): owner, other
 *               (other = -1 for a circular arc); owner = lower strut id
 *   arc_vtx   : [A] uint32, v0 | v1<<8 | owner_local<<16 | (other_local+1)<<24
 *               (node-local vertex ids and node-local strut-end indices)
 *   arc_phi   : [A][2] dtype, start angle and angular length in the owner's
 *               strut frame
 *   loop_ent  : per strut end (end_loop_off over 2E+1), node-local arc id |
 *               reversed<<31, in increasing strut angle from the first vertex
 *   hole_ent  : per hole (hole_off over H+1), node-local arc id | reversed<<31 */
typedef struct {
  int64_t n_nodes, n_struts, n_vtx, n_arcs, n_loop_ent, n_holes, n_hole_ent;
  int32_t dtype, pad_;
  const int64_t* row_ptr;     /* [N+1] CSR of strut ends per node */
  const int32_t* adj;         /* [2E] strut-end ids, ascending per node */
  const void* node_R;         /* [N] dtype */
  const uint32_t* node_flags; /* [N] */
  const int64_t* node_vtx_off; /* [N+1] */
  const void* vtx_z;
  const uint64_t* vtx_key;    /* [V] bit l = local strut end l meets here */
  const uint32_t* vtx_flags;  /* [V] LM_VTX_* */
  const uint32_t* vtx_gen;    /* [V] generator: type | root<<2 | i<<3 | j<<9 | k<<15 */
  const int64_t* node_arc_off; /* [N+1] */
  const int32_t* arc_ends;
  const uint32_t* arc_vtx;
  const void* arc_phi;
  const int64_t* end_loop_off; /* [2E+1] */
  const uint32_t* loop_ent;
  const int64_t* node_hole_off; /* [N+1] */
  const int64_t* hole_off;      /* [H+1] */
  const uint32_t* hole_ent;
} lm_metamesh_view;

lm_status lm_metamesh_export(lm_metamesh* mm, lm_metamesh_view* view);

/* Triangle counts at resolution k (Section 5, Eq. sampling with chord error
 * CE = 1 - cos(pi/k); Algorithm 1).  Items 0..E-1 are struts (lateral band
 * between the strut's two arc loops), items E..E+N-1 are nodes (hole fans).
 * Computes per-item counts and their exclusive scan in the handle (one k at
 * a time) and synchronises the stream to return the total.
 *   h_total : host, receives the number of triangles of all items        */
lm_status lm_tri_count(lm_metamesh* mm, int32_t k, void* stream, int64_t* h_total);

/* Host-side range query after lm_tri_count(k) (synchronising): first
 * triangle index and triangle count of items [item_begin, item_end).     */
lm_status lm_tri_range(const lm_metamesh* mm, int64_t item_begin, int64_t item_end,
                       int64_t* h_first, int64_t* h_count);

/* Triangulation at resolution k (Section 5: arc subdivision by Eq. sampling
 * and Eq. parameter-range, strut stitching, hole filling; Algorithm 1,
 * subdivide / triangulate / fillHoles, with write(T) here a device buffer in
 * STL layout).  Emits the triangles of items [item_begin, item_end) as
 * binary-STL records (50 bytes: normal f32x3, v0, v1, v2 f32x3, uint16
 * attribute 0; outward counter-clockwise) into d_out, the record of global
 * triangle t at byte 50*(t - first(item_begin)).  Asynchronous; requires
 * lm_tri_count(k) first (else LM_ERR_STATE).  Records beyond capacity_tris
 * are not written and set LM_ERR_CAPACITY, reported by lm_last_error.
 *   d_out : device, >= 50*capacity_tris bytes, any alignment of 2 bytes    */
lm_status lm_triangulate(lm_metamesh* mm, int32_t k, int64_t item_begin, int64_t item_end,
                         void* d_out, int64_t capacity_tris, void* stream);

/* Same triangles streamed through device chunk buffers into a caller-owned
 * pinned host buffer ring on overlapped streams (the heterogeneous pipeline
 * of Section 4.2.2, here GPU triangulation + device-to-host copies).
 * Items are processed in chunks of chunk_items; chunk c is copied to
 * h_ring + (c % n_slots) * slot_bytes.  After each chunk's copy completes,
 * the callback (may be NULL) is invoked on a host thread with (chunk index,
 * first item, triangle count, slot pointer, user).  Synchronising.
 * The per-chunk device work (range set-up, deferral-bitmap reset, strut and
 * fan kernels) is captured once into two CUDA graphs, one per device
 * buffer, whose first node reads the next chunk from a device cursor; each
 * chunk is then one graph launch plus one copy.                          */
typedef void (*lm_chunk_cb)(int64_t chunk, int64_t first_item, int64_t n_tris, void* h_slot,
                            void* user);
lm_status lm_triangulate_stream(lm_metamesh* mm, int32_t k, int64_t chunk_items, void* h_ring,
                                int64_t slot_bytes, int32_t n_slots, lm_chunk_cb cb, void* user,
                                void* stream, int64_t* h_total);

/* The lattice meta-meshed and triangulated chunk by chunk with the build of
 * the next chunk overlapped with the streaming of the current one (the
 * pipeline of Section 4.2.2, Fig. pipeline (a): meta-meshing of one batch
 * beside the triangulation and transfer of the previous one).  Struts are
 * taken in chunks of build_struts; a chunk's sub-lattice holds its struts
 * and every strut incident to their end nodes, in increasing global order,
 * so the meta-mesh of each end node, and every triangle, has the same bits
 * as in a whole-lattice build.  A chunk emits, at each k of ks in turn, its
 * own struts (ascending id) and then the hole fans of the nodes whose
 * lowest-id strut it holds (ascending id); the records go through the
 * caller's pinned ring as in lm_triangulate_stream, and cb (may be NULL)
 * gets (sequence number, k, first item of the streamed piece in the chunk's
 * sub-lattice, triangle count, slot pointer, user) after each piece's copy.
 * The set of records per k equals lm_triangulate's; their order differs.
 * Synchronising; the work starts after the work already queued on `stream`
 * (which may have produced the lattice).
 *   lat         : device arrays as for lm_build_metamesh (fewer than 2^30
 *                 struts, 2^31 nodes); opt: as for lm_build_metamesh
 *   ks, n_k     : resolutions, each emitted per chunk
 *   h_ring      : host, pinned, n_slots (>= 2) x slot_bytes
 *   h_tris      : host, [n_k] triangles emitted per k
 * Returns LM_ERR_INVALID_ARG for an end outside [0, N), LM_ERR_CAPACITY if
 * one strut's or node's records exceed a slot, or a chunk build's status. */
typedef void (*lm_kchunk_cb)(int64_t seq, int32_t k, int64_t first_item, int64_t n_tris, void* h_slot,
                             void* user);
lm_status lm_stream_chunked(const lm_lattice* lat, const lm_options* opt, const int32_t* ks, int32_t n_k,
                            int64_t build_struts, void* h_ring, int64_t slot_bytes, int32_t n_slots,
                            lm_kchunk_cb cb, void* user, void* stream, int64_t* h_tris);

/* The same triangles written to a binary-STL file at `path` (created or
 * truncated) through the three-stage pipeline of Section 4.2.2: GPU
 * triangulation of chunk c + 1, device-to-host copy of chunk c into the
 * caller's pinned ring, and the file write of earlier chunks by a host
 * writer thread, all overlapped (Fig. pipeline (a) and (b)).  The file is the
 * 84-byte header of lm_stl_header followed by every record in triangle
 * order (84 + 50 n bytes).  chunk_items <= 0 sizes the chunks by Eq.
 * chunk-size, N_batch = S_buffer / (S_triangle N_strut), with S_buffer = 80 %
 * of a slot and N_strut = the mean triangle count of an item; a chunk whose
 * records exceed a slot returns LM_ERR_CAPACITY.  Synchronising; runs
 * lm_tri_count(k) first when needed.
 *   h_ring  : host, pinned (cudaHostAlloc), n_slots (>= 2) x slot_bytes, owned
 *             by the caller; its contents are undefined afterwards
 *   flags   : LM_FILE_SYNC: fsync the file before returning
 *   h_total : host, receives the triangle count (may be NULL)
 *   h_stats : host, may be NULL; [0] seconds of the whole call, [1] seconds
 *             the writer spent in write calls, [2] seconds the streaming
 *             loop waited for the writer to free a slot (disk-bound when
 *             large), [3] seconds of the final fsync (0 without the flag)
 * Returns LM_ERR_IO if the file cannot be opened, written or synced (what
 * was written up to the failure stays in the file).                      */
enum { LM_FILE_SYNC = 1 };
lm_status lm_triangulate_to_file(lm_metamesh* mm, int32_t k, const char* path, int64_t chunk_items,
                                 void* h_ring, int64_t slot_bytes, int32_t n_slots, int32_t flags,
                                 void* stream, int64_t* h_total, double h_stats[4]);

/* Binary-STL file header for the records of lm_triangulate (Section 5 and
 * Algorithm 1 write the triangles as STL; Table 1 reports the STL file
 * sizes, 84 + 50 bytes per triangle): 80-byte text header (zero padded) +
 * little-endian uint32 triangle count; counts above 2^32-1 write 0xFFFFFFFF
 * (the true count is the int64 the caller holds).  Host only.
 *   hdr    : host, 84 bytes written
 *   n_tris : triangle count (negative counts write 0)                     */
void lm_stl_header(uint8_t hdr[84], int64_t n_tris);

/* Objective of the triangulated mesh at k: area = sum |(v1-v0)x(v2-v0)|/2,
 * volume = sum v0.(v1 x v2)/6 (divergence theorem), accumulated in FP64.
 * Synchronising; requires lm_tri_count(k).                               */
lm_status lm_objective(lm_metamesh* mm, int32_t k, void* stream, double* h_area,
                       double* h_volume);

/* Adjoint: d(w_area*area + w_vol*volume)/d(node xyz, node radius) of the
 * triangulated mesh at k, with the arc topology and the segment counts held
 * fixed; per-node intermediates are recomputed, not stored.  Gradients are
 * ADDED into d_grad_xyz [n_nodes][3] and d_grad_r [n_nodes] (dtype of the
 * lattice).  Synchronising (returns the objective terms).                */
lm_status lm_metamesh_backward(lm_metamesh* mm, int32_t k, double w_area, double w_vol,
                               void* d_grad_xyz, void* d_grad_r, void* stream, double* h_area,
                               double* h_volume);

/* Launch shape the build used for the persistent meta-mesh kernel, per
 * valence bucket (d <= 16, d <= 32, d <= 64): out[2b] = warps of a block
 * working on the bucket, out[2b+1] = nodes a warp takes per work-queue
 * access.  With
 * lm_options.autotune these are the autotuner's choices (Section 4.3.3's
 * workload balancing, done by measurement); 0 for buckets without nodes.
 * out[6] = nodes the emit pass computed a second time (those the count
 * pass's arena could not hold; every node when the build ran without an
 * arena), out[7] = 1 if the emit pass took only those nodes from the lists
 * the count pass made of them, 0 if it went over every node (no arena, or
 * more nodes missed than the lists hold: 1/16 of the nodes + 1,024 per
 * valence bucket).  Host values; no device work.                        */
lm_status lm_metamesh_launch_shape(const lm_metamesh* mm, int32_t out[8]);

/* Device time of the build's phases, milliseconds from CUDA events on the
 * build's stream: out[0] = input checks, CSR, bucketing and (with
 * lm_options.autotune) the tuner's sample launches; out[1] = the persistent
 * count-pass launch of the meta-mesh kernel alone (every node computed once);
 * out[2] = sizing (offset scans, the one host synchronisation, allocation of
 * the output arrays); out[3] = the arena gather; out[4] = the emit pass of
 * the nodes the arena could not hold.  Host values; no device work.  Returns
 * LM_ERR_INVALID_ARG for a NULL handle or array.                          */
lm_status lm_metamesh_build_times(const lm_metamesh* mm, float out[5]);

/* First asynchronous error recorded on the handle by a device-side check
 * (LM_ERR_CAPACITY); synchronises `stream`, then clears it.              */
lm_status lm_last_error(lm_metamesh* mm, void* stream);

void lm_metamesh_free(lm_metamesh* mm);
const char* lm_status_string(lm_status s);

/* Allocation-free variant of lm_tri_count + lm_triangulate for one item
 * range (the paper has no counterpart: it concerns how this library gets its
 * scratch memory).  For callers that cannot let the library allocate device
 * memory when they triangulate: an application whose GPU memory belongs to a
 * framework's caching allocator or to a pool sized up front (a library
 * cudaMalloc could fail there, or make the pool give back its cache), or a
 * latency-bound loop in which cudaMalloc / cudaFree would stall the device.
 * It calls no cudaMalloc, cudaFree or allocating library routine: every
 * scratch buffer (per-item counts and offsets of the range, scan workspace,
 * FP64 fallback contexts, work counters) lives in one fixed file-scope device
 * array of about 7 MB that each GPU loading the library keeps until process
 * exit.  The records are byte-identical to lm_triangulate's.
 *   item range : at most 262,144 items per call, else LM_ERR_CAPACITY;
 *                chunk larger ranges
 *   d_out      : records of the range from byte 0 (as lm_triangulate)
 *   h_ntris    : host, receives the range's triangle count (may be NULL)
 * Needs only lm_build_metamesh first (no lm_tri_count).  Synchronises the
 * stream once (it reads the range's triangle count back to size the
 * kernel's shared memory).  The first call on each device resolves the
 * array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * last call's contents (the call clears what must start empty): calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Capacity overflow is reported by lm_last_error
 * as for lm_triangulate.                                                 */
lm_status lm_triangulate_noalloc(lm_metamesh* mm, int32_t k, int64_t item_begin, int64_t item_end,
                                 void* d_out, int64_t capacity_tris, void* stream, int64_t* h_ntris);

/* Utility (no counterpart in the paper): synchronous device-to-host copy of
 * `bytes` bytes, for reading the views of lm_metamesh_export.            */
lm_status lm_copy_to_host(void* h_dst, const void* d_src, int64_t bytes);

/* FP64 stability steps (of the FP32 path; no counterpart in the paper): how
 * many decisions were re-taken in higher precision because their FP32 value
 * lay inside a safety margin of its threshold or came from an
 * ill-conditioned configuration.  Candidate re-decisions ([1]) run in
 * double-float arithmetic (about 48 bits), the others in FP64.
 * Synchronous.  Cumulative over the handle's lifetime.
 *   out[0] pair classification, [1] candidate vertex re-decision,
 *   [2] vertex position refinement, [3] deduplication, [4] seam label,
 *   [5] loop angle order / wrap, [6] arc label, [7] arc extent (build);
 *   [8] segment count, [9] start angle, [10] struts stitched with FP64
 *   angles, [11] fan centre (triangulation); struts deferred from the FP32
 *   stitching pass because of [12] an entry's segment count or start
 *   angle, [13] a key at the edge of the angular window, [14] a pair of
 *   keys within the zipper margin, [16] keys out of angular order (a loop
 *   that turns back on a degenerate node; stitched by the sequential zipper
 *   in FP64), [17] an ill-conditioned elliptical arc (a steep section on a
 *   degenerate node; its points are subdivided in FP64); [15] pairs of
 *   zipper keys decided in FP64.                                           */
enum { LM_N_FP64_COUNTS = 18 };
lm_status lm_fp64_counts(const lm_metamesh* mm, int64_t out[LM_N_FP64_COUNTS]);

/* Ablation of Section 6 (Fig. thread-vs-warp: the paper's warp-centric
 * meta-meshing kernel ran 35x faster than a thread-centric one, which
 * allocates a thread per arc calculation and lets every thread read the
 * strut parameters it needs from global memory by itself).  The trimming
 * step of Section 4.3.1 with the same arithmetic in both work mappings: for
 * every strut end i of the handle's lattice and S sample angles
 * phi_q = 2 pi q / S on its end circle (strut frame), t*(phi_q) =
 * max(0, max_{j != i} h_j(phi_q)) -- the generator length where the kept
 * surface starts, the envelope of the auxiliary planes P_ij -- and its
 * arg-max (node-local index of j; -1 where the nodal sphere wins).
 *   mode    : LM_ENV_WARP: one warp per node, its strut ends built once into
 *             shared memory, lanes over (end, angle); LM_ENV_THREAD: one
 *             thread per (end, angle), which builds its own end and every
 *             other end of its node from the lattice in global memory
 *   samples : S, 1..4096
 *   d_t     : device, [2E][S] in the lattice's dtype, index end_id * S + q
 *   d_label : device, [2E][S] int16
 * Asynchronous on `stream`; valences above LM_MAX_VALENCE are reported by
 * lm_last_error (LM_ERR_VALENCE, warp mode).                              */
enum { LM_ENV_WARP = 0, LM_ENV_THREAD = 1 };
lm_status lm_envelope_samples(const lm_metamesh* mm, int32_t samples, int32_t mode, void* d_t,
                              int16_t* d_label, void* stream);

/* Utility (no counterpart in the paper): number of CUDA kernels this library
 * has launched in the process so far (host-side counter).                */
long long lm_launch_count(void);

/* Utility (no counterpart in the paper): the library allocates its device
 * memory from the current device's default memory pool (CUDA's stream-ordered
 * allocator), which by default gives freed memory back to the driver at every
 * synchronisation, so that a build after a freed one maps its memory again.
 * lm_pool_retain(bytes) lets that pool keep up to `bytes` of freed memory
 * mapped for reuse (0 restores the default).  The setting belongs to the pool,
 * so it applies to every user of the current device's default pool; memory it
 * keeps is not available to other allocators (PyTorch's, for one) until the
 * threshold is lowered again.  Returns LM_ERR_CUDA if the pool cannot be
 * queried or set.                                                         */
lm_status lm_pool_retain(uint64_t bytes);

/* Utility (no counterpart in the paper): text of the CUDA error behind the
 * last LM_ERR_CUDA or LM_ERR_OOM that a call of this library returned on the
 * calling thread ("no error" if none).                                    */
const char* lm_cuda_error_string(void);

/* Utility (no counterpart in the paper): the library's FP32 angle functions,
 * evaluated element-wise on device arrays so that their error can be tested
 * against FP64 references: d_atan2[i] = lm_atan2(d_y[i], d_x[i]) (polynomial
 * arctangent, see csrc/lm_geom.cuh), (d_sin[i], d_cos[i]) = lm_sincos(d_a[i])
 * (two-part reduction by 2 pi, then the hardware sine / cosine).  All arrays
 * device, n float32 each; asynchronous on `stream`.                       */
lm_status lm_eval_angle_fns(const float* d_y, const float* d_x, const float* d_a, int64_t n, float* d_atan2,
                            float* d_sin, float* d_cos, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LIBLM_H */
