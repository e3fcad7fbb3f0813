// Warp-per-node meta-meshing (Section 4.3 of arXiv 2405.15197).
//
// One warp owns one node at a time: the node's strut ends are staged in
// shared memory (the paper's "per-node strut lists"), candidate vertices are
// evaluated one generator per lane (the paper's "one ellipse per thread"),
// survivors are compacted with warp ballots in canonical order, loops are
// built one strut end per lane, and per-node counts feed warp-aggregated
// prefix sums.  The same code runs twice: a count pass (sizes only) and an
// emit pass that writes the structure-of-arrays layout at scanned offsets
// (Section 4.3.2's index region + data region, here CSR offsets + SoA).  The
// count pass also keeps each node's output in an arena when it has room; a
// gather then moves those nodes to their CSR ranges and the emit pass
// computes only the others.
//
// Arithmetic is T (float for FP32 lattices, double for FP64 lattices).  For
// FP32 every decision whose FP32 value lies inside a safety margin of its
// threshold, or comes from an ill-conditioned configuration, is taken again
// in FP64 from the inputs (near-parallel pairs, tangencies, angular ties).
#pragma once
#include "lm_geom.cuh"
#include "lm_internal.h"

namespace lm {

template <int MD, int MV, int MLE, int MA>
struct Cap {
  static constexpr int D = MD, V = MV, LE = MLE, A = MA;
};

// A root kept or uncertain after the evaluation of its generator, waiting in
// canonical order for its re-decision and its append.
template <typename T>
struct CandRec {
  V3<T> z;
  uint64_t key, umask;  // key; strut ends whose FP32 screening was uncertain
  uint32_t code;        // generator code | root << 2
  uint32_t kflags;      // node flags raised if kept as a new vertex
  uint8_t state;        // 1 kept, 2 uncertain (0 after a rejection)
  uint8_t sphere, whole, pad;  // whole: the generator was uncertain as a whole
};
// records per warp (a round of 32 generators adds up to 64: the list is
// flushed as often as it fills)
constexpr int CAND_CAP = 32;

template <typename T, typename C>
struct WarpSmem {
  EndG<T> E[C::D];
  EndG<double> E64[sizeof(T) == 4 ? C::D : 1];
  EndG<df> EDF[sizeof(T) == 4 ? C::D : 1];
  uint64_t e64_valid, edf_valid;
  uint64_t tan_small[C::D], tan_neg[C::D], coinc[C::D];
  V3<T> vz[C::V];
  uint64_t vkey[C::V];
  uint32_t vgen[C::V];
  uint8_t vfl[C::V];
  int nv;
  uint32_t nflags;
  uint16_t loop_off[C::D + 1];
  uint8_t le_v[C::LE];
  int8_t le_lab[C::LE];
  uint8_t le_rev[C::LE];
  int16_t le_arc[C::LE];
  T le_ang[C::LE];
  T le_dphi[C::LE];
  uint8_t a_owner[C::A];
  int8_t a_other[C::A];
  uint8_t a_v0[C::A], a_v1[C::A];
  T a_phi0[C::A], a_dphi[C::A];
  int na;
  uint16_t h_off[C::A + 1];
  uint16_t h_ent[C::A];
  int nh, nhe;
  CandRec<T> cand[CAND_CAP];
};

template <typename T>
struct MMArgs {
  LatDev<T> lat;
  const int* err;        // input errors found by the CSR build: skip all work
  uint32_t* node_flags;  // [N]
  // count pass
  int32_t* node_cnt;     // [N][4]: V, A, H, HE
  int32_t* end_cnt;      // [2E]
  // emit pass
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
  unsigned long long* fb;  // FP64 re-decision counters (see FB_*)
  // 0: count pass (sizes, and each node's output stashed in `ar` when it
  // has room); 1: emit pass (CSR outputs of the nodes `ar` does not hold).
  // One kernel instantiation serves both, so both write the same bits.
  int emit;
  // count pass: each node's output stashed in an arena (start NULL: none)
  MMArena ar;
};

// FP64 stability-step counters
enum { FB_PAIR = 0, FB_GEN = 1, FB_REFINE = 2, FB_DEDUP = 3, FB_SEAM = 4, FB_ANGLE = 5,
       FB_LABEL = 6, FB_EXTENT = 7, FB_N = 8 };
__device__ __forceinline__ void fb_add(unsigned long long* fb, int which, bool pred) {
  uint32_t m = __ballot_sync(0xffffffffu, pred);
  if (fb && m && (threadIdx.x & 31) == (__ffs(m) - 1)) atomicAdd(fb + which, (unsigned long long)__popc(m));
}

// FP64 copies of the node's strut ends, built on first use.
template <typename T, typename C>
__device__ void ensure64(WarpSmem<T, C>& S, const LatDev<T>& L, int64_t n, int d, int lane) {
  if (sizeof(T) == 8) return;
  uint64_t all = d >= 64 ? ~0ull : ((1ull << d) - 1);
  uint64_t miss = all & ~S.e64_valid;
  if (!miss) return;
  for (int li = lane; li < d; li += 32)
    if (miss >> li & 1ull) S.E64[li] = make_end<T, double>(L, n, S.E[li].end_id);
  __syncwarp();
  if (lane == 0) S.e64_valid |= miss;
  __syncwarp();
}
// Double-float copies of the node's strut ends (candidate re-decisions),
// built on first use.
template <typename T, typename C>
__device__ void ensure_df(WarpSmem<T, C>& S, const LatDev<T>& L, int64_t n, int d, int lane) {
  if (sizeof(T) == 8) return;
  uint64_t all = d >= 64 ? ~0ull : ((1ull << d) - 1);
  uint64_t miss = all & ~S.edf_valid;
  if (!miss) return;
  for (int li = lane; li < d; li += 32)
    if (miss >> li & 1ull) S.EDF[li] = make_end<T, df>(L, n, S.E[li].end_id);
  __syncwarp();
  if (lane == 0) S.edf_valid |= miss;
  __syncwarp();
}
template <typename T, typename C>
__device__ __forceinline__ const EndG<double>* ends64(WarpSmem<T, C>& S) {
  if constexpr (sizeof(T) == 8) return reinterpret_cast<const EndG<double>*>(S.E);
  else return S.E64;
}

// canonical generator g -> code: pairs (i<j) first, then triples (i<j<k),
// both lexicographic
__device__ __forceinline__ uint32_t decode_gen(int g, int d, int np) {
  if (g < np) {
    int i = 0, rem = g;
    while (rem >= d - 1 - i) { rem -= d - 1 - i; i++; }
    return gen_code(0, 0, i, i + 1 + rem, 0);
  }
  int rem = g - np, i = 0;
  while (true) {
    int m = d - 1 - i;
    int c = m * (m - 1) / 2;
    if (rem < c) break;
    rem -= c;
    i++;
  }
  int j = i + 1;
  while (rem >= d - 1 - j) { rem -= d - 1 - j; j++; }
  return gen_code(1, 0, i, j, j + 1 + rem);
}


// exact (FP64) loop angle of vertex v around local end li
template <typename T, typename C>
__device__ double angle64(WarpSmem<T, C>& S, int d, double R, int li, int v) {
  const EndG<double>* E = ends64(S);
  V3<double> z = vertex_from_gen<double>(E, d, R, S.vgen[v]);
  return (double)norm_angle(raw_angle(E[li], z));
}

// Envelope arg-max among the labels in (cm, cs) at the mid-angle pm, with
// the sequential tie rule (a later label must beat the best by ETA_SIGMA R).
template <typename U>
__device__ int midpoint_label(const EndG<U>* E, int li, uint64_t cm, bool cs, U pm, U R, U& gap) {
  U c, s;
  lm_sincos(pm, &s, &c);
  U best = cs ? U(0) : U(0);
  int label = cs ? -1 : -2;
  U second = U(-1e30);
  for (int j = 0; j < 64; j++) {
    if (!(cm >> j & 1ull)) continue;
    U h = hval(E[li], E[j], c, s, R);
    if (label == -2 || h > best + U(ETA_SIGMA) * R) {
      if (label != -2) second = best;
      best = h;
      label = j;
    } else if (h > second) {
      second = h;
    }
  }
  if (cs && label >= 0 && second < U(0)) second = U(0);
  gap = best - second;
  return label;
}

template <typename T, typename C>
__device__ void node_metamesh(WarpSmem<T, C>& S, const MMArgs<T>& A, int64_t n, int lane) {
  const LatDev<T>& L = A.lat;
  const bool EMIT = A.emit != 0;
  constexpr bool IS64 = sizeof(T) == 8;
  // stored in the arena by the count pass: gathered, not emitted
  if (EMIT && A.ar.start && A.ar.start[n] >= 0) return;
  const int64_t base = L.row_ptr[n];
  const int d = (int)(L.row_ptr[n + 1] - base);
  const T R = L.node_R[n];
  const double R64 = (double)L.node_R[n];
  if (d == 0) {
    if (!EMIT && lane == 0) {
      A.node_flags[n] = 0;
      for (int q = 0; q < 4; q++) A.node_cnt[4 * n + q] = 0;
      if (A.ar.start) A.ar.start[n] = 0;
    }
    return;
  }
  // ---- strut ends of the node
  for (int li = lane; li < d; li += 32) S.E[li] = make_end<T, T>(L, n, L.adj[base + li]);
  for (int li = lane; li < d; li += 32) S.tan_small[li] = S.tan_neg[li] = S.coinc[li] = 0;
  if (lane == 0) {
    S.nv = 0;
    S.nflags = 0;
    S.e64_valid = 0;
    S.edf_valid = 0;
  }
  __syncwarp();

  // ---- pair classification (tangency 1 - max_phi k_j, coincident circles)
  {
    const int npair = d * d;
    for (int c0 = 0; c0 < npair; c0 += 32) {
      int p = c0 + lane;
      int i = p / d, j = p % d;
      bool act = p < npair && i != j;
      bool unc = false;
      bool ts = false, tn = false, co = false;
      if (act) {
        T c = dot(S.E[i].u, S.E[j].u);
        T pr = lm_sqrt(fmax(T(0), T(1) - c * c));
        T tau = T(1) - (S.E[i].co * c + fabs(S.E[i].s) * pr) * S.E[j].ico;
        if (IS64) {
          ts = fabs(tau) < T(EPS_TAN);
          tn = tau <= T(0);
        } else if (tau < T(M_COND)) {
          unc = true;
        }
        if (i < j) {
          T q = T(1) - c * c;
          if (IS64) {
            if (q < T(EPS_PAR)) {
              T coin = c < T(0) ? S.E[i].s + S.E[j].s : S.E[i].s - S.E[j].s;
              co = fabs(coin) < T(EPS_TAN);
            }
          } else if (q < T(0.6 * EPS_PAR)) {
            // certainly (anti)parallel: q's FP32 error is below 4e-7
            T coin = c < T(0) ? S.E[i].s + S.E[j].s : S.E[i].s - S.E[j].s;
            if (fabs(coin) >= T(1.5 * EPS_TAN)) co = false;
            else if (fabs(coin) <= T(0.5 * EPS_TAN)) co = true;
            else unc = true;
          } else if (q < T(M_COND)) {
            unc = true;
          }
        }
      }
      fb_add(A.fb, FB_PAIR, unc);
      if (!IS64 && __any_sync(0xffffffffu, unc)) {
        ensure64(S, L, n, d, lane);
        if (unc) {
          const EndG<double>* E = ends64(S);
          double c = dot(E[i].u, E[j].u);
          double pr = sqrt(fmax(0.0, 1.0 - c * c));
          double tau = 1.0 - (E[i].co * c + fabs(E[i].s) * pr) * E[j].ico;
          ts = fabs(tau) < EPS_TAN;
          tn = tau <= 0.0;
          if (i < j) {
            double q = 1.0 - c * c;
            if (q < EPS_PAR) {
              double coin = c < 0.0 ? E[i].s + E[j].s : E[i].s - E[j].s;
              co = fabs(coin) < EPS_TAN;
            }
          }
        }
      }
      if (act && ts) { atomicOr((unsigned long long*)&S.tan_small[i], 1ull << j); atomicOr((unsigned long long*)&S.tan_small[j], 1ull << i); }
      if (act && tn) { atomicOr((unsigned long long*)&S.tan_neg[i], 1ull << j); atomicOr((unsigned long long*)&S.tan_neg[j], 1ull << i); }
      if (act && co) { atomicOr((unsigned long long*)&S.coinc[i], 1ull << j); atomicOr((unsigned long long*)&S.coinc[j], 1ull << i); }
    }
  }
  __syncwarp();

  // ---- candidate vertices in canonical order, screened, deduplicated.
  // (1) The generators are evaluated in the kernel's precision, 32 at a
  // time; the roots they keep and the roots whose decisions FP32 cannot take
  // safely go to a per-warp list in canonical order.  (2) When the list is
  // full, or the generators are done, its uncertain roots are re-decided in
  // double-float together, a root per lane.  (3) The list is appended in
  // canonical order with the deduplication of the oracle.
  const int np = d * (d - 1) / 2;
  const int nt = d * (d - 1) * (d - 2) / 6;
  const int ng = np + nt;
  bool overflow = false;
  uint32_t nflags = 0;
  int nrec = 0;  // records in S.cand (warp-uniform)
  auto flush = [&]() {
    if constexpr (!IS64) {
      // (2) dense double-float re-decisions of the uncertain roots
      bool need = false;
      for (int q = lane; q < nrec; q += 32) need |= S.cand[q].state == 2;
      if (__any_sync(0xffffffffu, need)) {
        ensure_df(S, L, n, d, lane);
        for (int q0 = 0; q0 < nrec; q0 += 32) {
          const int q = q0 + lane;
          const bool mine = q < nrec && S.cand[q].state == 2;
          fb_add(A.fb, FB_GEN, mine);
          // a partially uncertain triple point at a node of valence <= 8:
          // Newton steps in double-float (there most such roots are exact
          // ties of four struts, as on BCC lattices).  At higher valence the
          // uncertain roots are mostly near-threshold non-ties whose steps
          // fail the error bound about a quarter of the time (irregular
          // lattice at r_scale 0.3), and the full re-evaluation is faster.
          bool done = false;
          if constexpr (sizeof(T) == 4) {
            if (mine && d <= 8 && !S.cand[q].whole && (S.cand[q].code & 3) == 1) {
              CandRec<T>& c = S.cand[q];
              done = rescreen_triple_df(S.EDF, S.E, d, (float)R, c.code,
                                        c.z, c.umask, c.state, c.key, c.sphere, c.kflags, c.z);
            }
          }
          if (mine && !done) {
            CandRec<T>& c = S.cand[q];
            const int r = (c.code >> 2) & 1;
            // a generator uncertain as a whole is redone in full; otherwise
            // only the uncertain screening decisions of this root are retaken
            GenHint hint;
            hint.st[r] = 2;
            hint.st[1 - r] = 0;
            hint.umask[r] = c.umask;
            hint.umask[1 - r] = 0;
            GenOut<df> o64;
            eval_gen<df, true>(S.EDF, d, df(R), c.code & ~4u, o64, c.whole ? nullptr : &hint);
            nflags |= o64.nflags;
            if (o64.nroot == 2) {
              c.z = mk3((T)(float)o64.z[r].x, (T)(float)o64.z[r].y, (T)(float)o64.z[r].z);
              c.key = o64.key[r];
              c.sphere = o64.sphere[r];
              c.state = o64.state[r];
              c.kflags = o64.kflags[r];
            } else {
              c.state = 0;
            }
          }
        }
        __syncwarp();
      }
    }
    // (3) append in canonical order.  A record is dropped as a duplicate of
    // an earlier vertex (same key and sphere flag, within ETA_DEDUP R) or of
    // an earlier record of the list that is kept.  Lane q holds record q and
    // compares it with the vertices already stored and with every earlier
    // kept-or-uncertain record (masks of certain and uncertain matches); the
    // keep decisions are then resolved in canonical order over those masks,
    // which gives the decisions of a one-record-at-a-time append.  A distance
    // the FP32 margins cannot decide is taken in FP64 from the generators.
    static_assert(CAND_CAP <= 32, "one candidate record per lane");
    {
      const int nv0 = S.nv;
      const int q = lane;
      const bool live = q < nrec && S.cand[q].state == 1;
      V3<T> z = mk3(T(0), T(0), T(0));
      uint64_t key = 0;
      int sph = 0;
      bool dpre = false, upre = false;
      uint32_t mm = 0, um = 0;
      if (live) {
        const CandRec<T>& c = S.cand[q];
        z = c.z;
        key = c.key;
        sph = c.sphere;
        for (int v = 0; v < nv0; v++) {
          if (S.vkey[v] != key || ((S.vfl[v] & VF_SPHERE) != 0) != (sph != 0)) continue;
          V3<T> dz = z - S.vz[v];
          T dd = lm_sqrt(dot(dz, dz));
          if (IS64) {
            dpre |= dd <= T(ETA_DEDUP) * R;
          } else {
            if (dd <= T(0.5 * ETA_DEDUP) * R) dpre = true;
            else if (dd <= T(2.0 * ETA_DEDUP) * R) upre = true;
          }
        }
        for (int p = 0; p < q; p++) {
          const CandRec<T>& o = S.cand[p];
          if (o.state != 1 || o.key != key || (o.sphere != 0) != (sph != 0)) continue;
          V3<T> dz = z - o.z;
          T dd = lm_sqrt(dot(dz, dz));
          if (IS64) {
            if (dd <= T(ETA_DEDUP) * R) mm |= 1u << p;
          } else {
            if (dd <= T(0.5 * ETA_DEDUP) * R) mm |= 1u << p;
            else if (dd <= T(2.0 * ETA_DEDUP) * R) um |= 1u << p;
          }
        }
      }
      const uint32_t liveM = __ballot_sync(0xffffffffu, live);
      const uint32_t dpreM = __ballot_sync(0xffffffffu, dpre);
      const uint32_t upreM = __ballot_sync(0xffffffffu, upre);
      // With no FP32-uncertain distance the keep set is the unique solution
      // of K_q = live_q and not dpre_q and (mm_q & K) = 0 over the earlier
      // records; the guess "no earlier live match" is that solution when it
      // satisfies every equation (checked lane-parallel), else the equations
      // are solved in canonical order below.
      uint32_t K = liveM & ~dpreM & ~__ballot_sync(0xffffffffu, (mm & liveM) != 0u);
      const bool fast = !__any_sync(0xffffffffu, upre || um != 0u) &&
                        __all_sync(0xffffffffu, ((K >> q) & 1u) == (uint32_t)(live && !dpre && (mm & K) == 0u));
      if (!fast) K = 0;
      for (int r = 0; r < nrec && !fast; r++) {
        const uint32_t mr = __shfl_sync(0xffffffffu, mm, r);
        const uint32_t ur = __shfl_sync(0xffffffffu, um, r);
        if (!((liveM >> r) & 1u)) continue;
        bool dup = ((dpreM >> r) & 1u) || (mr & K);
        if (!IS64 && !dup && (((upreM >> r) & 1u) || (ur & K))) {
          fb_add(A.fb, FB_DEDUP, lane == 0);
          ensure64(S, L, n, d, lane);
          const CandRec<T>& c = S.cand[r];
          const V3<double> z64 = vertex_from_gen<double>(ends64(S), d, R64, c.code);
          bool d64 = false;
          for (int v = lane; v < nv0 + r; v += 32) {
            uint32_t g;
            if (v < nv0) {
              if (S.vkey[v] != c.key || ((S.vfl[v] & VF_SPHERE) != 0) != (c.sphere != 0)) continue;
              g = S.vgen[v];
            } else {
              const int p = v - nv0;
              if (!((K >> p) & 1u) || S.cand[p].key != c.key || (S.cand[p].sphere != 0) != (c.sphere != 0)) continue;
              g = S.cand[p].code;
            }
            const V3<double> w = vertex_from_gen<double>(ends64(S), d, R64, g);
            const V3<double> dz = z64 - w;
            d64 |= sqrt(dot(dz, dz)) <= ETA_DEDUP * R64;
          }
          dup = __any_sync(0xffffffffu, d64);
        }
        if (!dup) K |= 1u << r;
      }
      const int room = C::V - nv0;
      const int nk = __popc(K);
      if (live && ((K >> q) & 1u)) {
        const int rank = __popc(K & ((1u << q) - 1u));
        if (rank < room) {
          const CandRec<T>& c = S.cand[q];
          S.vz[nv0 + rank] = z;
          S.vkey[nv0 + rank] = key;
          S.vfl[nv0 + rank] = sph ? VF_SPHERE : 0;
          S.vgen[nv0 + rank] = c.code;
          nflags |= c.kflags;
        }
      }
      __syncwarp();
      if (lane == 0) S.nv = nv0 + (nk < room ? nk : room);
      if (nk > room) overflow = true;
    }
    nrec = 0;
    __syncwarp();
  };
  for (int c0 = 0; c0 < ng && !overflow; c0 += 32) {
    // (1) evaluation
    const int g = c0 + lane;
    GenOut<T> o;
    uint32_t code = 0;
    o.nroot = 0;
    o.unc = 0;
    o.nflags = 0;
    if (g < ng) {
      code = decode_gen(g, d, np);
      eval_gen<T, IS64>(S.E, d, R, code, o);
    }
    nflags |= o.nflags;
    // records of this lane: both roots of a generator uncertain as a whole,
    // else the roots kept or uncertain
    const int nr = o.unc ? 2 : (o.nroot == 2 ? (o.state[0] != 0) + (o.state[1] != 0) : 0);
    const int pre = warp_excl_scan(nr, lane);
    const int tot = __shfl_sync(0xffffffffu, pre + nr, 31);
    // the lanes' records go to the list in lane order, as many lanes at a
    // time as the list has room for (the list is flushed when full)
    int done = 0;  // records of this round already in the list
    while (done < tot && !overflow) {
      const bool fits = nr > 0 && pre >= done && pre + nr - done <= CAND_CAP - nrec;
      if (fits) {
        int pos = nrec + pre - done;
        for (int r = 0; r < 2; r++) {
          if (!o.unc && (o.nroot != 2 || o.state[r] == 0)) continue;
          CandRec<T>& c = S.cand[pos++];
          c.code = code | ((uint32_t)r << 2);
          c.whole = o.unc;
          c.state = o.unc ? 2 : o.state[r];
          if (!o.unc) {
            c.z = o.z[r];
            c.key = o.key[r];
            c.umask = o.umask[r];
            c.sphere = o.sphere[r];
            c.kflags = o.kflags[r];
          }
        }
      }
      const int w = __reduce_add_sync(0xffffffffu, fits ? nr : 0);
      nrec += w;
      done += w;
      __syncwarp();
      if (done < tot) flush();
    }
  }
  if (!overflow) flush();
  nflags = __reduce_or_sync(0xffffffffu, nflags);

  // ---- seam vertices for strut ends no vertex touches, in end order: a seam
  // cut by plane P_ij also touches end j, which then needs no seam of its own
  if (!overflow) {
    uint32_t seam_need = 0;
    uint64_t covered = 0;  // ends touched by the seams added so far
    for (int i0 = 0; i0 < d; i0 += 32) {
      int i = i0 + lane;
      bool need = false, unc = false;
      int lab = -1;
      T best = T(0);
      if (i < d) {
        bool has = false;
        for (int v = 0; v < S.nv; v++) has |= (S.vkey[v] >> i) & 1ull;
        need = !has;
        if (need) {
          T top = T(0), second = T(-1e30);
          for (int j = 0; j < d; j++) {
            if (j == i) continue;
            T h = hval(S.E[i], S.E[j], T(1), T(0), R);
            if (h > best + T(ETA_SIGMA) * R) {
              best = h;
              lab = j;
            }
            if (h > top) { second = top; top = h; }
            else if (h > second) second = h;
          }
          if (!IS64 && top - second <= T(M_LEN) * R) unc = true;
        }
      }
      fb_add(A.fb, FB_SEAM, unc);
      if (!IS64 && __any_sync(0xffffffffu, unc)) {
        ensure64(S, L, n, d, lane);
        if (unc) {
          const EndG<double>* E = ends64(S);
          double b = 0.0;
          lab = -1;
          for (int j = 0; j < d; j++) {
            if (j == i) continue;
            double h = hval(E[i], E[j], 1.0, 0.0, R64);
            if (h > b + ETA_SIGMA * R64) { b = h; lab = j; }
          }
          best = (T)b;
        }
      }
      uint32_t m = __ballot_sync(0xffffffffu, need);
      while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        int li = i0 + src;
        int lb = __shfl_sync(0xffffffffu, lab, src);
        T bs = __shfl_sync(0xffffffffu, best, src);
        if ((covered >> li) & 1ull) continue;
        covered |= (1ull << li) | (lb >= 0 ? (1ull << lb) : 0ull);
        int nvc = S.nv;
        if (nvc >= C::V) { overflow = true; break; }
        // a seam cut by a plane lies on a steep section (the node is
        // degenerate): its position is ill-conditioned in FP32 and is taken
        // in FP64 from the inputs
        if (!IS64 && lb >= 0) ensure64(S, L, n, d, lane);
        if (lane == 0) {
          if (!IS64 && lb >= 0) {
            const EndG<double>* E = ends64(S);
            V3<double> z64 = surf_point(E[li], 1.0, 0.0, hval(E[li], E[lb], 1.0, 0.0, R64), R64);
            S.vz[nvc] = mk3((T)z64.x, (T)z64.y, (T)z64.z);
          } else {
            S.vz[nvc] = surf_point(S.E[li], T(1), T(0), bs, R);
          }
          S.vkey[nvc] = (1ull << li) | (lb >= 0 ? (1ull << lb) : 0ull);
          S.vfl[nvc] = VF_SEAM | (lb < 0 ? VF_SPHERE : 0u);
          S.vgen[nvc] = gen_code(2, 0, li, lb < 0 ? 0 : lb, 0) | (lb >= 0 ? (1u << 21) : 0u);
          S.nv = nvc + 1;
        }
        if (lb >= 0) nflags |= NF_DEGENERATE | NF_SEAM_CUT;
        __syncwarp();
      }
      (void)seam_need;
    }
  }
  __syncwarp();

  // ---- loops: per strut end, vertices by angle, arcs labelled
  int nle = 0;
  if (!overflow) {
    int cnt[2] = {0, 0};
    for (int t = 0; t < 2; t++) {
      int i = lane + 32 * t;
      if (i < d)
        for (int v = 0; v < S.nv; v++) cnt[t] += (S.vkey[v] >> i) & 1ull;
    }
    int off0 = warp_excl_scan(cnt[0], lane);
    int tot0 = __shfl_sync(0xffffffffu, off0 + cnt[0], 31);
    int off1 = tot0 + warp_excl_scan(cnt[1], lane);
    nle = __shfl_sync(0xffffffffu, off1 + cnt[1], 31);
    if (nle > C::LE) overflow = true;
    if (!overflow) {
      if (lane < d) S.loop_off[lane] = off0;
      if (lane + 32 < d) S.loop_off[lane + 32] = off1;
      if (lane == 0) S.loop_off[d] = nle;
    }
  }
  __syncwarp();
  if (!overflow) {
    for (int t = 0; t < 2; t++) {
      int i = lane + 32 * t;
      bool unc = false;
      int b0 = 0, nl = 0;
      if (i < d) {
        b0 = S.loop_off[i];
        nl = S.loop_off[i + 1] - b0;
        int q = 0;
        for (int v = 0; v < S.nv; v++) {
          if (!((S.vkey[v] >> i) & 1ull)) continue;
          const V3<T> z = S.vz[v];
          const T zx = dot(z, S.E[i].e1), zy = dot(z, S.E[i].e2);
          T a = lm_atan2(zy, zx);
          if (!IS64 && fabs(a + T(PHI_CUT)) <= T(M_ANG)) unc = true;
          // the angle of a vertex close to the strut's axis relative to its
          // distance from the node (seams of steep sections, vertices past a
          // strut's length: degenerate nodes) amplifies its FP32 position
          // error: the loop is ordered with FP64 angles
          if (!IS64 && T(256) * (zx * zx + zy * zy) < dot(z, z) + R * R) unc = true;
          a = norm_angle(a);
          // stable insertion by angle
          int p = q;
          while (p > 0 && S.le_ang[b0 + p - 1] > a) {
            S.le_ang[b0 + p] = S.le_ang[b0 + p - 1];
            S.le_v[b0 + p] = S.le_v[b0 + p - 1];
            p--;
          }
          S.le_ang[b0 + p] = a;
          S.le_v[b0 + p] = (uint8_t)v;
          q++;
        }
        if (!IS64)
          for (int p = 0; p + 1 < nl; p++)
            if (S.le_ang[b0 + p + 1] - S.le_ang[b0 + p] <= T(M_ANG)) unc = true;
      }
      fb_add(A.fb, FB_ANGLE, unc);
      if (!IS64 && __any_sync(0xffffffffu, unc)) {
        ensure64(S, L, n, d, lane);
        if (unc) {
          // exact angles, stable re-sort by (angle, vertex id)
          double ang[C::V > 64 ? 64 : C::V];
          int vv[C::V > 64 ? 64 : C::V];
          int m = 0;
          for (int v = 0; v < S.nv && m < 64; v++) {
            if (!((S.vkey[v] >> i) & 1ull)) continue;
            double a = angle64(S, d, R64, i, v);
            int p = m;
            while (p > 0 && ang[p - 1] > a) { ang[p] = ang[p - 1]; vv[p] = vv[p - 1]; p--; }
            ang[p] = a;
            vv[p] = v;
            m++;
          }
          for (int p = 0; p < m; p++) {
            S.le_ang[b0 + p] = (T)ang[p];
            S.le_v[b0 + p] = (uint8_t)vv[p];
            if (p + 1 < m && ang[p + 1] - ang[p] <= ETA_PHI) nflags |= NF_DEGENERATE | NF_ANGLE_TIE;
          }
        }
      }
      if (IS64 && i < d)
        for (int p = 0; p + 1 < nl; p++)
          if (S.le_ang[b0 + p + 1] - S.le_ang[b0 + p] <= T(ETA_PHI)) nflags |= NF_DEGENERATE | NF_ANGLE_TIE;
    }
  }
  __syncwarp();
  // labels
  if (!overflow) {
    for (int t = 0; t < 2; t++) {
      int i = lane + 32 * t;
      if (i >= d) continue;
      int b0 = S.loop_off[i], nl = S.loop_off[i + 1] - b0;
      for (int q = 0; q < nl; q++) {
        int va = S.le_v[b0 + q], vb = S.le_v[b0 + (q + 1) % nl];
        T dph = (q + 1 < nl) ? S.le_ang[b0 + q + 1] - S.le_ang[b0 + q]
                             : S.le_ang[b0] + T(PI2) - S.le_ang[b0 + q];
        uint64_t cm = (S.vkey[va] & S.vkey[vb]) & ~(1ull << i);
        bool cs = (S.vfl[va] & VF_SPHERE) && (S.vfl[vb] & VF_SPHERE);
        int ncand = __popcll(cm) + (cs ? 1 : 0);
        int label;
        if (ncand == 1) {
          label = cs ? -1 : __ffsll(cm) - 1;
        } else {
          if (ncand == 0) {
            nflags |= NF_INCONSISTENT;
            cm = (d >= 64 ? ~0ull : ((1ull << d) - 1)) & ~(1ull << i);
            cs = true;
          }
          T gap;
          label = midpoint_label<T>(S.E, i, cm, cs, S.le_ang[b0 + q] + T(0.5) * dph, R, gap);
          if (!IS64 && gap <= T(M_LEN) * R) {
            // exact re-decision (rare; no warp-collective calls here)
            if (A.fb) atomicAdd(A.fb + FB_LABEL, 1ull);
            if (S.e64_valid != ((d >= 64) ? ~0ull : ((1ull << d) - 1))) {
              for (int li = 0; li < d; li++)
                if (!((S.e64_valid >> li) & 1ull)) S.E64[li] = make_end<T, double>(L, n, S.E[li].end_id);
            }
            const EndG<double>* E = ends64(S);
            double a0 = angle64(S, d, R64, i, va);
            double a1 = angle64(S, d, R64, i, vb);
            double dd = a1 - a0;
            if (q + 1 >= nl) dd += PI2;
            double g64;
            label = midpoint_label<double>(E, i, cm, cs, a0 + 0.5 * dd, R64, g64);
          }
        }
        S.le_lab[b0 + q] = (int8_t)label;
        S.le_dphi[b0 + q] = dph;
      }
    }
  }
  nflags = __reduce_or_sync(0xffffffffu, nflags);
  __syncwarp();

  // ---- activity of flagged pairs
  if (!overflow) {
    uint32_t f = 0;
    for (int v = lane; v < S.nv; v += 32) {
      uint64_t key = S.vkey[v];
      for (int i = 0; i < d; i++) {
        if (!((key >> i) & 1ull)) continue;
        if (key & S.tan_small[i]) f |= NF_NEAR_TANGENT;
        if (key & S.tan_neg[i]) f |= NF_DEGENERATE | NF_STEEP;
      }
    }
    uint64_t hc = 0;
    for (int i = lane; i < d; i += 32) {
      int b0 = S.loop_off[i], nl = S.loop_off[i + 1] - b0;
      for (int q = 0; q < nl; q++)
        if (S.le_lab[b0 + q] < 0) hc |= 1ull << i;
    }
    hc = warp_or64(hc);
    for (int i = lane; i < d; i += 32)
      if (((hc >> i) & 1ull) && (S.coinc[i] & hc)) f |= NF_NEAR_TANGENT;
    nflags |= __reduce_or_sync(0xffffffffu, f);
  }

  // ---- node-local arcs: own arcs by (owner end, loop position)
  int na = 0;
  if (!overflow) {
    int own[2] = {0, 0};
    for (int t = 0; t < 2; t++) {
      int i = lane + 32 * t;
      if (i >= d) continue;
      int b0 = S.loop_off[i], nl = S.loop_off[i + 1] - b0;
      int si = S.E[i].end_id >> 1;
      for (int q = 0; q < nl; q++) {
        int lb = S.le_lab[b0 + q];
        if (lb < 0 || si < (S.E[lb].end_id >> 1)) own[t]++;
      }
    }
    int o0 = warp_excl_scan(own[0], lane);
    int t0 = __shfl_sync(0xffffffffu, o0 + own[0], 31);
    int o1 = t0 + warp_excl_scan(own[1], lane);
    na = __shfl_sync(0xffffffffu, o1 + own[1], 31);
    if (na > C::A) overflow = true;
    if (!overflow) {
      for (int t = 0; t < 2; t++) {
        int i = lane + 32 * t;
        if (i >= d) continue;
        int id = t == 0 ? o0 : o1;
        int b0 = S.loop_off[i], nl = S.loop_off[i + 1] - b0;
        int si = S.E[i].end_id >> 1;
        for (int q = 0; q < nl; q++) {
          int lb = S.le_lab[b0 + q];
          if (lb < 0 || si < (S.E[lb].end_id >> 1)) {
            S.a_owner[id] = (uint8_t)i;
            S.a_other[id] = (int8_t)lb;
            S.a_v0[id] = S.le_v[b0 + q];
            S.a_v1[id] = S.le_v[b0 + (q + 1) % nl];
            S.a_phi0[id] = S.le_ang[b0 + q];
            S.a_dphi[id] = S.le_dphi[b0 + q];
            S.le_arc[b0 + q] = (int16_t)id;
            S.le_rev[b0 + q] = 0;
            id++;
          } else {
            S.le_arc[b0 + q] = -1;
          }
        }
      }
    }
  }
  __syncwarp();
  // partner search for non-owner entries
  if (!overflow) {
    uint32_t f = 0;
    for (int t = 0; t < 2; t++) {
      int i = lane + 32 * t;
      if (i >= d) continue;
      int b0 = S.loop_off[i], nl = S.loop_off[i + 1] - b0;
      for (int q = 0; q < nl; q++) {
        if (S.le_arc[b0 + q] >= 0) continue;
        int j = S.le_lab[b0 + q];
        int va = S.le_v[b0 + q], vb = S.le_v[b0 + (q + 1) % nl];
        int found = -1, rev = 0, nf = 0;
        int c0 = S.loop_off[j], cl = S.loop_off[j + 1] - c0;
        for (int q2 = 0; q2 < cl; q2++) {
          int id = S.le_arc[c0 + q2];
          if (id < 0 || S.le_lab[c0 + q2] != i) continue;
          if (S.a_v0[id] == va && S.a_v1[id] == vb) {
            if (found < 0) { found = id; rev = 0; }
            nf++;
          } else if (S.a_v0[id] == vb && S.a_v1[id] == va) {
            if (found < 0) { found = id; rev = 1; }
            nf++;
          }
        }
        if (nf != 1 || va == vb) f |= NF_INCONSISTENT;
        S.le_arc[b0 + q] = (int16_t)(found >= 0 ? found : -2);
        S.le_rev[b0 + q] = (uint8_t)rev;
      }
    }
    nflags |= __reduce_or_sync(0xffffffffu, f);
    __syncwarp();
    // entries without a partner become arcs of their own, appended in
    // (end, loop position) order
    if (lane == 0) {
      for (int i = 0; i < d && !overflow; i++) {
        int b0 = S.loop_off[i], nl = S.loop_off[i + 1] - b0;
        for (int q = 0; q < nl; q++) {
          if (S.le_arc[b0 + q] != -2) continue;
          if (na >= C::A) { overflow = true; break; }
          S.a_owner[na] = (uint8_t)i;
          S.a_other[na] = S.le_lab[b0 + q];
          S.a_v0[na] = S.le_v[b0 + q];
          S.a_v1[na] = S.le_v[b0 + (q + 1) % nl];
          S.a_phi0[na] = S.le_ang[b0 + q];
          S.a_dphi[na] = S.le_dphi[b0 + q];
          S.le_arc[b0 + q] = (int16_t)na;
          S.le_rev[b0 + q] = 0;
          na++;
        }
      }
    }
    na = __shfl_sync(0xffffffffu, na, 0);
    overflow = __shfl_sync(0xffffffffu, (int)overflow, 0);
  }
  __syncwarp();

  // ---- arc extent: every elliptical arc within both struts' lengths
  if (!overflow) {
    uint32_t f = 0;
    bool unc = false;
    for (int a = lane; a < na; a += 32) {
      if (S.a_other[a] < 0) continue;
      const EndG<T>& Ei = S.E[S.a_owner[a]];
      const EndG<T>& Ej = S.E[S.a_other[a]];
      T tm = arc_tmax(Ei, Ej, R, S.a_phi0[a], S.a_dphi[a]);
      T lim = fmin(Ei.L * Ei.co, Ej.L * Ej.co);
      if (!IS64 && fabs(tm - lim) <= T(M_LEN) * R) unc = true;
      else if (tm > lim) f |= NF_DEGENERATE | NF_BEYOND;
    }
    fb_add(A.fb, FB_EXTENT, unc);
    if (!IS64 && __any_sync(0xffffffffu, unc)) {
      ensure64(S, L, n, d, lane);
      const EndG<double>* E = ends64(S);
      for (int a = lane; a < na; a += 32) {
        if (S.a_other[a] < 0) continue;
        const EndG<double>& Ei = E[S.a_owner[a]];
        const EndG<double>& Ej = E[S.a_other[a]];
        T lim32 = fmin(S.E[S.a_owner[a]].L * S.E[S.a_owner[a]].co, S.E[S.a_other[a]].L * S.E[S.a_other[a]].co);
        T tm32 = arc_tmax(S.E[S.a_owner[a]], S.E[S.a_other[a]], R, S.a_phi0[a], S.a_dphi[a]);
        if (fabs(tm32 - lim32) > T(M_LEN) * R) continue;
        double p0 = angle64(S, d, R64, S.a_owner[a], S.a_v0[a]);
        double p1 = angle64(S, d, R64, S.a_owner[a], S.a_v1[a]);
        double dd = S.a_v0[a] == S.a_v1[a] ? PI2 : p1 - p0;
        if (dd <= 0.0) dd += PI2;
        double tm = arc_tmax(Ei, Ej, R64, p0, dd);
        if (tm > fmin(Ei.L * Ei.co, Ej.L * Ej.co)) f |= NF_DEGENERATE | NF_BEYOND;
      }
    }
    nflags |= __reduce_or_sync(0xffffffffu, f);
  }
  __syncwarp();

  // ---- holes: circular arcs chained with the hole on the left seen from
  // outside (lower-id-end frames are right-handed about the outward axis)
  int nh = 0, nhe = 0;
  if (!overflow && lane == 0) {
    uint32_t f = 0;
    uint8_t used[C::A];
    for (int a = 0; a < na; a++) used[a] = 0;
    for (int a0 = 0; a0 < na && !overflow; a0++) {
      if (S.a_other[a0] >= 0 || used[a0]) continue;
      S.h_off[nh] = (uint16_t)nhe;
      int cur = a0;
      auto hs = [&](int a) { return S.E[S.a_owner[a]].at_lo ? S.a_v1[a] : S.a_v0[a]; };
      auto he = [&](int a) { return S.E[S.a_owner[a]].at_lo ? S.a_v0[a] : S.a_v1[a]; };
      while (true) {
        used[cur] = 1;
        S.h_ent[nhe++] = (uint16_t)cur | (S.E[S.a_owner[cur]].at_lo ? 0x8000u : 0u);
        int ev = he(cur);
        if (ev == hs(a0)) break;
        int nxt = -1, cnt = 0;
        for (int a = 0; a < na; a++) {
          if (S.a_other[a] >= 0 || used[a]) continue;
          if (hs(a) == ev) {
            if (nxt < 0) nxt = a;
            cnt++;
          }
        }
        if (cnt != 1) f |= NF_INCONSISTENT;
        if (nxt < 0) break;
        cur = nxt;
      }
      nh++;
    }
    S.h_off[nh] = (uint16_t)nhe;
    S.nh = nh;
    S.nhe = nhe;
    nflags |= f;
  }
  nh = __shfl_sync(0xffffffffu, nh, 0);
  nhe = __shfl_sync(0xffffffffu, nhe, 0);
  nflags = __shfl_sync(0xffffffffu, nflags, 0) | nflags;
  nflags = __reduce_or_sync(0xffffffffu, nflags);
  __syncwarp();

  // ---- outputs
  if (!EMIT) {
    if (overflow) {
      if (lane == 0) {
        A.node_flags[n] = nflags | NF_OVERFLOW;
        for (int q = 0; q < 4; q++) A.node_cnt[4 * n + q] = 0;
        atomicAdd(A.overflow, 1);
        if (A.ar.start) A.ar.start[n] = -1;
      }
      for (int li = lane; li < d; li += 32) A.end_cnt[L.adj[base + li]] = 0;
      return;
    }
    if (lane == 0) {
      A.node_flags[n] = nflags;
      A.node_cnt[4 * n + 0] = S.nv;
      A.node_cnt[4 * n + 1] = na;
      A.node_cnt[4 * n + 2] = nh;
      A.node_cnt[4 * n + 3] = nhe;
    }
    for (int li = lane; li < d; li += 32)
      A.end_cnt[L.adj[base + li]] = S.loop_off[li + 1] - S.loop_off[li];
    if (A.ar.start) {
      // stash the node's output in the arena (one block, or not at all)
      const int nle = S.loop_off[d];
      const ArenaBlock B = arena_block(S.nv, na, nh, nhe, nle, sizeof(T));
      long long at = 0;
      if (lane == 0) {
        at = (long long)atomicAdd(A.ar.used, (unsigned long long)B.bytes);
        if (at + B.bytes > A.ar.cap) {
          at = -1;
          atomicAdd(A.ar.miss, 1);
        }
        A.ar.start[n] = at;
      }
      at = __shfl_sync(0xffffffffu, at, 0);
      if (at >= 0) {
        unsigned char* blk = A.ar.buf + at;
        T* vz = reinterpret_cast<T*>(blk + B.vz);
        uint64_t* vkey = reinterpret_cast<uint64_t*>(blk + B.vkey);
        uint8_t* vfl = blk + B.vfl;
        uint32_t* vgen = reinterpret_cast<uint32_t*>(blk + B.vgen);
        for (int v = lane; v < S.nv; v += 32) {
          vz[3 * v] = S.vz[v].x;
          vz[3 * v + 1] = S.vz[v].y;
          vz[3 * v + 2] = S.vz[v].z;
          vkey[v] = S.vkey[v];
          vfl[v] = S.vfl[v];
          vgen[v] = S.vgen[v];
        }
        uint32_t* avtx = reinterpret_cast<uint32_t*>(blk + B.avtx);
        T* aphi = reinterpret_cast<T*>(blk + B.aphi);
        for (int a = lane; a < na; a += 32) {
          avtx[a] = (uint32_t)S.a_v0[a] | ((uint32_t)S.a_v1[a] << 8) | ((uint32_t)S.a_owner[a] << 16) |
                    ((uint32_t)(S.a_other[a] + 1) << 24);
          aphi[2 * a] = S.a_phi0[a];
          aphi[2 * a + 1] = S.a_dphi[a];
        }
        uint32_t* ho = reinterpret_cast<uint32_t*>(blk + B.ho);
        uint32_t* he = reinterpret_cast<uint32_t*>(blk + B.he);
        uint16_t* le = reinterpret_cast<uint16_t*>(blk + B.le);
        for (int h = lane; h < nh; h += 32) ho[h] = S.h_off[h];
        for (int q = lane; q < nhe; q += 32) {
          uint32_t e = S.h_ent[q];
          he[q] = (e & 0x7fffu) | ((e & 0x8000u) ? 0x80000000u : 0u);
        }
        // 16 bits per entry: arc | rev << 15, 0xffff for an unmatched entry
        // (arc -1, which the emit pass writes as 0xffffffff)
        for (int q = lane; q < nle; q += 32)
          le[q] = S.le_arc[q] < 0 ? (uint16_t)0xffffu
                                  : (uint16_t)((uint32_t)S.le_arc[q] | ((uint32_t)S.le_rev[q] << 15));
      }
    }
    return;
  }
  if (overflow) return;
  const int64_t vo = A.vtx_off[n], ao = A.arc_off[n];
  for (int v = lane; v < S.nv; v += 32) {
    A.vtx_z[3 * (vo + v)] = S.vz[v].x;
    A.vtx_z[3 * (vo + v) + 1] = S.vz[v].y;
    A.vtx_z[3 * (vo + v) + 2] = S.vz[v].z;
    A.vtx_key[vo + v] = S.vkey[v];
    A.vtx_flags[vo + v] = S.vfl[v];
    A.vtx_gen[vo + v] = S.vgen[v];
  }
  for (int a = lane; a < na; a += 32) {
    A.arc_vtx[ao + a] = (uint32_t)S.a_v0[a] | ((uint32_t)S.a_v1[a] << 8) |
                        ((uint32_t)S.a_owner[a] << 16) | ((uint32_t)(S.a_other[a] + 1) << 24);
    A.arc_phi[2 * (ao + a)] = S.a_phi0[a];
    A.arc_phi[2 * (ao + a) + 1] = S.a_dphi[a];
  }
  for (int li = 0; li < d; li++) {
    int32_t eid = S.E[li].end_id;
    int64_t eo = A.end_off[eid];
    int b0 = S.loop_off[li], nl = S.loop_off[li + 1] - b0;
    for (int q = lane; q < nl; q += 32)
      A.loop_ent[eo + q] = (uint32_t)S.le_arc[b0 + q] | ((uint32_t)S.le_rev[b0 + q] << 31);
  }
  const int64_t ho = A.hole_off_n[n], heo = A.hent_off_n[n];
  for (int h = lane; h < nh; h += 32) A.hole_off[ho + h] = heo + S.h_off[h];
  for (int q = lane; q < nhe; q += 32) {
    uint32_t e = S.h_ent[q];
    A.hole_ent[heo + q] = (e & 0x7fffu) | ((e & 0x8000u) ? 0x80000000u : 0u);
  }
}

// capacities of the three valence buckets (d <= 16, <= 32, <= 64): strut
// ends, vertices, loop entries, arcs per node
using Cap16 = Cap<16, 64, 192, 160>;
using Cap32 = Cap<32, 128, 384, 320>;
using Cap64 = Cap<64, 224, 640, 480>;
// arena loop entries hold a node-local arc id in 15 bits (0x7fff and up unused)
static_assert(Cap16::A < 0x7fff && Cap32::A < 0x7fff && Cap64::A < 0x7fff, "arc ids fit 15 bits");

template <typename T>
__host__ __device__ constexpr size_t mm_smem_bytes() {
  return 4 * sizeof(WarpSmem<T, Cap16>) > 2 * sizeof(WarpSmem<T, Cap32>)
             ? (4 * sizeof(WarpSmem<T, Cap16>) > sizeof(WarpSmem<T, Cap64>) ? 4 * sizeof(WarpSmem<T, Cap16>)
                                                                             : sizeof(WarpSmem<T, Cap64>))
             : (2 * sizeof(WarpSmem<T, Cap32>) > sizeof(WarpSmem<T, Cap64>) ? 2 * sizeof(WarpSmem<T, Cap32>)
                                                                             : sizeof(WarpSmem<T, Cap64>));
}

// Work of one bucket: each warp with a workspace pops tasks of npt
// consecutive entries of the bucket's node list from an atomic counter.
template <typename T, typename C, int SLOTS>
__device__ __forceinline__ void mm_bucket(const MMArgs<T>& A, const MMBuckets& Bk, int b, unsigned char* smem,
                                          int w, int lane) {
  if (w >= SLOTS) return;
  if (A.err && *(volatile const int*)A.err != 0) return;  // invalid input: nothing to compute
  WarpSmem<T, C>& S = reinterpret_cast<WarpSmem<T, C>*>(smem)[w];
  int64_t n = Bk.counts[b];
  if (Bk.limit[b] > 0 && n > Bk.limit[b]) n = Bk.limit[b];
  const int npt = Bk.npt[b] > 0 ? Bk.npt[b] : 1;
  const int32_t* list = Bk.lists + (int64_t)b * Bk.cap;
  while (true) {
    int task = 0;
    if (lane == 0) task = atomicAdd(Bk.queues + b, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    const int64_t first = (int64_t)task * npt;
    if (first >= n) break;
    const int64_t last = first + npt < n ? first + npt : n;
    for (int64_t t = first; t < last; t++) {
      const int32_t nd = list[t];
      node_metamesh<T, C>(S, A, nd, lane);
      __syncwarp();
      // count pass: a node the arena could not hold joins its bucket's list
      // for the emit pass (lane 0 wrote its arena start)
      if (!A.emit && A.ar.mlist && lane == 0 && A.ar.start[nd] < 0) {
        const int q = atomicAdd(A.ar.mcnt + b, 1);
        if (q < A.ar.mcap) A.ar.mlist[(int64_t)b * A.ar.mcap + q] = nd;
      }
    }
  }
}

// One persistent, work-stealing launch over nodes of every valence: the
// blocks work through the buckets in turn (a block passes to the next
// bucket once its warps have found the current one's queue empty), each
// warp with the workspace its bucket needs in the block's shared memory.
template <typename T>
__global__ void __launch_bounds__(128, 4) k_metamesh(MMArgs<T> A, MMBuckets Bk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  mm_bucket<T, Cap16, MM_SLOTS[0]>(A, Bk, 0, smem_raw, w, lane);
  __syncthreads();
  mm_bucket<T, Cap32, MM_SLOTS[1]>(A, Bk, 1, smem_raw, w, lane);
  __syncthreads();
  mm_bucket<T, Cap64, MM_SLOTS[2]>(A, Bk, 2, smem_raw, w, lane);
}

}  // namespace lm
