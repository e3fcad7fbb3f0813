// FP64 CPU oracle for lattice meta-meshing and resolution-k triangulation.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
// CUDA path is checked against.  Only the tests, __graft_entry__.smoke() and
// the benchmark's CPU-baseline leg may load it.  It shares no code, header,
// table or constant generator with the CUDA library: every formula below is
// written out again from the paper (arXiv 2405.15197, "Warp-centric GPU
// meta-meshing and fast triangulation of billion-scale lattice structures").
//
// What it computes, step by step, in FP64:
//   * Lattice model (Section 4.1): every node is a sphere of radius R; every
//     strut is the cone (cylinder when its two node radii are equal) tangent
//     to the spheres of its two end nodes.
//   * Auxiliary planes (Section 4.3.1): the surfaces of two struts meeting at
//     a node intersect in a planar conic.  With generator coordinate
//     G_i(z) = (u_i.z - R s_i)/co_i the cone of strut end i is
//     |z|^2 - R^2 - G_i(z)^2 = 0, so the near-node intersection of struts i
//     and j lies on the plane P_ij : G_i(z) = G_j(z).
//   * Trimming (Section 4.3.1, Eq. arc-range / overlap-vertices): a point of
//     strut i's surface is kept iff it is inside no other strut, which on the
//     surface reads G_l(z) <= G_i(z) for every other strut end l.  The arc
//     endpoints are therefore the points where three strut surfaces meet
//     (line P_ij n P_ik cut with the cone; "triple points") and where two
//     tangency circles meet on the nodal sphere ("circle points").
//   * Arc loops (Section 4.3.1, last paragraph): the kept vertices of each
//     strut end, ordered by angle around the strut axis, with each arc
//     labelled by the plane (elliptical arc) or by the nodal sphere (circular
//     arc, the one-bit hole flag of Section 5).
//   * Triangulation (Section 5, Eq. sampling, Eq. parameter-range,
//     Algorithm 1): each arc gets N segments, sampled uniformly in the strut
//     angle and mapped onto the arc; the two loops of a strut are stitched;
//     hole contours are fanned to the barycentre projected on the nodal
//     sphere (Section 5, hole-filling equation).
//   * Annular holes: the hole filling assumes disc-shaped holes; where two
//     contours bound one exposed component of a nodal sphere (two narrowing
//     cones with disjoint caps) the band between them is stitched like a
//     strut's lateral band instead (band_tris).
//
// Readings of points where the paper is silent or garbled (all listed in the
// design notes of the repository):
//   * radius is a node property; per-end radii must agree at each node;
//   * the cone half-angle is alpha = asin((R_near - R_far)/L) (the printed
//     arccos formula is self-contradictory);
//   * subdivision is uniform in the strut angle phi (Section 5 samples on the
//     strut's end circle, then maps onto the arc);
//   * segment count N = max(1, ceil(dphi*k/(2 pi) - TAU)), i.e. Eq. sampling
//     with chord error CE = 1 - cos(pi/k), except that an arc of exactly j
//     sectors gets j segments;
//   * ties are decided with the tolerances ETA_* below and lower-id rules.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

const double PI2 = 6.283185307179586476925286766559;

// Tolerances (readings; the CUDA path decides with the same values).
const double ETA_SIGMA = 1e-9;   // x R: a strut passes through a vertex
const double ETA_DEDUP = 1e-3;   // x R: two candidates with one key are one vertex
const double ETA_PHI = 1e-9;     // rad: angle ties; relative angles wrap to [-ETA_PHI, 2pi-ETA_PHI)
// rad: absolute angles around a strut end are normalised to
// [-PHI_CUT, 2pi - PHI_CUT).  The cut sits away from angle 0, where
// symmetric lattices put vertices, so which end of the range they land on is
// never a rounding question.
const double PHI_CUT = 0.0009765625;  // 2^-10
// rad: zipper tie band.  A point of loop A advances before a point of loop B
// whose angle it exceeds by at most ETA_ZIP.  Points of the two loops of a
// (near-)symmetric strut line up to within far less than this, so they all
// take the same branch; the band is also far from the structural angle
// differences of symmetric lattices (multiples of the point spacing).
const double ETA_ZIP = 0.015625;  // 2^-6
// segment-count offset: an arc whose ratio dphi k / 2pi exceeds an integer n
// by at most TAU_COUNT gets n segments (exact multiples, as on symmetric
// lattices, keep the minimal count; the chord error may exceed its target
// by a relative 2^-10 / n at most)
const double TAU_COUNT = 0.0009765625;  // 2^-10
const double ETA_BARY = 1e-4;    // x R: hole barycentre too close to the centre
const double EPS_PAR = 1e-6;     // 1 - c^2 below this: (anti)parallel pair
const double EPS_TAN = 1e-6;     // tangency measure below this: node exempt

// node flag bits
const uint32_t F_NEAR_TANGENT = 1u;
const uint32_t F_DEGENERATE = 2u;
const uint32_t F_INCONSISTENT = 4u;
// reasons (informative, set together with F_DEGENERATE)
const uint32_t F_BEYOND_LENGTH = 8u;    // a vertex lies past a strut's far tangency circle
const uint32_t F_STEEP_PAIR = 16u;      // an active pair with 1 - max k_j <= 0
const uint32_t F_SEAM_CUT = 32u;        // a vertex-free loop lies on a plane, not the sphere
const uint32_t F_ANGLE_TIE = 64u;       // two vertices of one loop at the same angle
const uint32_t F_LINE_ALONG_CONE = 128u;  // a triple line parallel to a cone generator

// vertex flag bits
const uint32_t VF_SPHERE = 1u;
const uint32_t VF_SEAM = 2u;

struct V3 {
  double x, y, z;
};
inline V3 mk(double x, double y, double z) { return V3{x, y, z}; }
inline V3 add(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
inline V3 sub(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
inline V3 mul(V3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }

struct Lattice {
  int64_t n_nodes, n_struts;
  const double* xyz;      // [n_nodes][3]
  const int32_t* ends;    // [n_struts][2]
  const double* radii;    // [n_struts][2]
};

// One strut end as seen from its node.
struct End {
  int32_t end_id;   // 2*strut + side
  int32_t strut;
  int32_t far_node;
  bool at_lo;       // this node is the strut's lower-id node
  V3 u;             // outward unit axis
  double s, co, L;  // sin / cos of the cone half-angle, strut length
  V3 e1, e2;        // strut frame (built from the lo->hi axis)
};

struct Vertex {
  V3 z;            // position relative to the node centre
  uint64_t key;    // local strut ends meeting here
  uint32_t flags;  // VF_SPHERE, VF_SEAM
  uint32_t gen;    // generator code (type | root | i | j | k)
};

struct Arc {
  int owner;     // local end index owning the arc
  int other;     // local end index of the other strut, -1 = circular arc
  int v0, v1;    // node-local vertex ids, owner's increasing-angle direction
  double phi0, dphi;
};

struct Entry {
  int arc;
  int rev;
};

struct NodeOut {
  uint32_t flags = 0;
  std::vector<Vertex> V;
  std::vector<Arc> A;
  std::vector<std::vector<Entry>> loops;  // per local end
  std::vector<std::vector<Entry>> holes;
};

struct Mesh {
  Lattice lat;
  std::vector<double> node_R;
  std::vector<int64_t> row_ptr;  // CSR: strut-end ids incident to each node
  std::vector<int32_t> adj;
  std::vector<NodeOut> nodes;
  int status = 0;
};

inline V3 node_xyz(const Lattice& L, int64_t n) {
  return mk(L.xyz[3 * n], L.xyz[3 * n + 1], L.xyz[3 * n + 2]);
}

// Strut end data (Section 4.3.1 notation: strut S_i with ends v_i^0, v_i^1
// and radii r_i^0, r_i^1; here the radii are the node radii).
End make_end(const Mesh& M, int64_t node, int32_t end_id) {
  const Lattice& L = M.lat;
  End e;
  e.end_id = end_id;
  e.strut = end_id >> 1;
  int side = end_id & 1;
  int32_t a = L.ends[2 * e.strut], b = L.ends[2 * e.strut + 1];
  e.far_node = side == 0 ? b : a;
  int32_t lo = std::min(a, b), hi = std::max(a, b);
  e.at_lo = (node == lo);
  V3 d = sub(node_xyz(L, hi), node_xyz(L, lo));
  e.L = norm(d);
  V3 ue = mul(d, 1.0 / e.L);
  e.u = e.at_lo ? ue : mul(ue, -1.0);
  double R = M.node_R[node], Rf = M.node_R[e.far_node];
  e.s = (R - Rf) / e.L;
  e.co = std::sqrt(1.0 - e.s * e.s);
  // frame: axis of smallest |d_a| (ties -> lowest a); e1 = ue x E_a, e2 = ue x e1
  double ad[3] = {std::fabs(d.x), std::fabs(d.y), std::fabs(d.z)};
  int ax = 0;
  if (ad[1] < ad[ax]) ax = 1;
  if (ad[2] < ad[ax]) ax = 2;
  V3 E = mk(ax == 0, ax == 1, ax == 2);
  V3 c1 = cross(ue, E);
  e.e1 = mul(c1, 1.0 / norm(c1));
  e.e2 = cross(ue, e.e1);
  return e;
}

inline V3 rho(const End& e, double phi) {
  return add(mul(e.e1, std::cos(phi)), mul(e.e2, std::sin(phi)));
}
inline V3 wdir(const End& e, double phi) { return add(mul(e.u, e.s), mul(rho(e, phi), e.co)); }
inline V3 gdir(const End& e, double phi) { return sub(mul(e.u, e.co), mul(rho(e, phi), e.s)); }
// generator coordinate G_l(z)
inline double G(const End& e, V3 z, double R) { return (dot(e.u, z) - R * e.s) / e.co; }
// h_j(phi) on strut end i: the t where the generator at phi crosses plane P_ij
inline double hval(const End& i, const End& j, double phi, double R) {
  return R * (dot(j.u, wdir(i, phi)) - j.s) / (j.co - dot(j.u, gdir(i, phi)));
}
// angle of a node-relative point around strut end e, in [-PHI_CUT, 2pi-PHI_CUT)
inline double angle(const End& e, V3 z) {
  double p = std::atan2(dot(z, e.e2), dot(z, e.e1));
  if (p < -PHI_CUT) p += PI2;
  return p;
}

struct Cand {
  V3 z;
  double t0;
  uint64_t gen_mask;
  bool sphere;
  uint32_t gen;
  bool tangent;
};

uint32_t gen_code(int type, int root, int i, int j, int k) {
  return (uint32_t)type | ((uint32_t)root << 2) | ((uint32_t)i << 3) | ((uint32_t)j << 9) |
         ((uint32_t)k << 15);
}

// Meta-mesh of one node: Section 4.3.1 (planes, ellipses, trimming, loops)
// and the hole flag of Section 5.
NodeOut node_metamesh(const Mesh& M, int64_t n) {
  NodeOut out;
  int64_t b0 = M.row_ptr[n], b1 = M.row_ptr[n + 1];
  int d = (int)(b1 - b0);
  if (d == 0) return out;
  double R = M.node_R[n];
  std::vector<End> E(d);
  for (int i = 0; i < d; i++) E[i] = make_end(M, n, M.adj[b0 + i]);
  out.loops.resize(d);

  // pair tangency: 1 - max_phi k_j(phi), k_j = u_j.g_i / co_j.  A flagged pair
  // only marks the node when the pair is active (shares a vertex, or, for
  // coincident tangency circles, both loops keep a circular arc).
  std::vector<uint64_t> tan_small(d, 0), tan_neg(d, 0), coinc(d, 0);
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      if (i == j) continue;
      double c = dot(E[i].u, E[j].u);
      double pr = std::sqrt(std::max(0.0, 1.0 - c * c));
      double tau = 1.0 - (E[i].co * c + std::fabs(E[i].s) * pr) / E[j].co;
      if (std::fabs(tau) < EPS_TAN) { tan_small[i] |= 1ull << j; tan_small[j] |= 1ull << i; }
      if (tau <= 0.0) { tan_neg[i] |= 1ull << j; tan_neg[j] |= 1ull << i; }
    }

  // ---- candidate vertices, canonical order: pairs (circle points), then triples
  std::vector<Cand> cand;
  for (int i = 0; i < d; i++)
    for (int j = i + 1; j < d; j++) {
      double c = dot(E[i].u, E[j].u);
      double q = 1.0 - c * c;
      if (q < EPS_PAR) {
        double coin = c < 0 ? E[i].s + E[j].s : E[i].s - E[j].s;
        if (std::fabs(coin) < EPS_TAN) { coinc[i] |= 1ull << j; coinc[j] |= 1ull << i; }
        continue;
      }
      // unit n with u_i.n = s_i and u_j.n = s_j
      double al = (E[i].s - c * E[j].s) / q;
      double be = (E[j].s - c * E[i].s) / q;
      double g2 = 1.0 - (al * al + be * be + 2.0 * al * be * c);
      if (g2 <= 0.0) {
        if (g2 > -EPS_TAN) out.flags |= F_NEAR_TANGENT;
        continue;
      }
      V3 w = cross(E[i].u, E[j].u);
      w = mul(w, 1.0 / norm(w));
      double g = std::sqrt(g2);
      for (int r = 0; r < 2; r++) {
        V3 nrm = add(add(mul(E[i].u, al), mul(E[j].u, be)), mul(w, r == 0 ? -g : g));
        Cand cd;
        cd.z = mul(nrm, R);
        cd.t0 = 0.0;
        cd.gen_mask = (1ull << i) | (1ull << j);
        cd.sphere = true;
        cd.gen = gen_code(0, r, i, j, 0);
        cd.tangent = g2 < EPS_TAN;
        cand.push_back(cd);
      }
    }
  for (int i = 0; i < d; i++)
    for (int j = i + 1; j < d; j++)
      for (int k = j + 1; k < d; k++) {
        // line P_ij n P_ik: m.z = delta
        V3 mj = sub(mul(E[i].u, 1.0 / E[i].co), mul(E[j].u, 1.0 / E[j].co));
        V3 mk_ = sub(mul(E[i].u, 1.0 / E[i].co), mul(E[k].u, 1.0 / E[k].co));
        double dj = R * (E[i].s / E[i].co - E[j].s / E[j].co);
        double dk = R * (E[i].s / E[i].co - E[k].s / E[k].co);
        V3 v = cross(mj, mk_);
        double vv = dot(v, v);
        if (vv < EPS_PAR * dot(mj, mj) * dot(mk_, mk_)) continue;  // parallel planes
        V3 z0 = mul(sub(mul(cross(mk_, v), dj), mul(cross(mj, v), dk)), 1.0 / vv);
        V3 vh = mul(v, 1.0 / std::sqrt(vv));
        // cone i along z0 + lam vh: A lam^2 + 2 B lam + C = 0
        double G0 = (dot(E[i].u, z0) - R * E[i].s) / E[i].co;
        double G1 = dot(E[i].u, vh) / E[i].co;
        double A = 1.0 - G1 * G1;
        double B = -G0 * G1;
        double C = dot(z0, z0) - R * R - G0 * G0;
        if (std::fabs(A) < 1e-12) {
          out.flags |= F_DEGENERATE | F_LINE_ALONG_CONE;
          continue;
        }
        double D = B * B - A * C;
        if (D <= 0.0) {
          if (D > -EPS_TAN * R * R) out.flags |= F_NEAR_TANGENT;
          continue;
        }
        double sq = std::sqrt(D);
        double lam[2];
        if (B >= 0.0) {
          double q = -(B + sq);
          lam[0] = q / A;
          lam[1] = C / q;
        } else {
          double q = -B + sq;
          lam[1] = q / A;
          lam[0] = C / q;
        }
        for (int r = 0; r < 2; r++) {
          Cand cd;
          cd.z = add(z0, mul(vh, lam[r]));
          cd.t0 = G0 + lam[r] * G1;
          cd.gen_mask = (1ull << i) | (1ull << j) | (1ull << k);
          cd.sphere = false;
          cd.gen = gen_code(1, r, i, j, k);
          cd.tangent = D < EPS_TAN * R * R;
          cand.push_back(cd);
        }
      }

  // ---- screening (trimming) and keys; dedup by key + distance
  for (size_t ci = 0; ci < cand.size(); ci++) {
    Cand& cd = cand[ci];
    if (cd.t0 < -ETA_SIGMA * R) continue;  // inside the nodal sphere side
    bool bad = false;
    uint64_t key = cd.gen_mask;
    bool sph = cd.sphere || std::fabs(cd.t0) <= ETA_SIGMA * R;
    for (int l = 0; l < d && !bad; l++) {
      if (cd.gen_mask >> l & 1ull) {
        // correct nappe of every generating cone
        if (R - E[l].s * dot(E[l].u, cd.z) <= 0.0) bad = true;
        continue;
      }
      double sg = G(E[l], cd.z, R) - cd.t0;
      if (sg > ETA_SIGMA * R) bad = true;
      else if (sg >= -ETA_SIGMA * R) key |= 1ull << l;
    }
    if (bad) continue;
    bool dup = false;
    for (auto& v : out.V) {
      if (v.key == key && ((v.flags & VF_SPHERE) != 0) == sph &&
          norm(sub(v.z, cd.z)) <= ETA_DEDUP * R) {
        dup = true;
        break;
      }
    }
    if (dup) continue;
    if (cd.tangent) out.flags |= F_NEAR_TANGENT;
    for (int l = 0; l < d; l++)
      if ((key >> l & 1ull) && cd.t0 > E[l].L * E[l].co) out.flags |= F_DEGENERATE | F_BEYOND_LENGTH;
    Vertex vx;
    vx.z = cd.z;
    vx.key = key;
    vx.flags = sph ? VF_SPHERE : 0u;
    vx.gen = cd.gen;
    out.V.push_back(vx);
  }

  // ---- seam vertices for strut ends that no vertex touches
  for (int i = 0; i < d; i++) {
    bool any = false;
    for (auto& v : out.V)
      if (v.key >> i & 1ull) any = true;
    if (any) continue;
    double best = 0.0;
    int lab = -1;
    for (int j = 0; j < d; j++) {
      if (j == i) continue;
      double h = hval(E[i], E[j], 0.0, R);
      if (h > best + ETA_SIGMA * R) {
        best = h;
        lab = j;
      }
    }
    Vertex vx;
    vx.z = add(mul(wdir(E[i], 0.0), R), mul(gdir(E[i], 0.0), best));
    vx.key = 1ull << i;
    vx.flags = VF_SEAM | (lab < 0 ? VF_SPHERE : 0u);
    if (lab >= 0) {
      vx.key |= 1ull << lab;
      out.flags |= F_DEGENERATE | F_SEAM_CUT;
    }
    vx.gen = gen_code(2, 0, i, lab < 0 ? 0 : lab, 0) | (lab >= 0 ? (1u << 21) : 0u);
    out.V.push_back(vx);
  }

  // ---- loops: per strut end, vertices ordered by angle, arcs labelled
  struct LArc {
    int va, vb, label;  // label: local end or -1 = sphere
    double phia, dphi;
  };
  std::vector<std::vector<LArc>> larcs(d);
  for (int i = 0; i < d; i++) {
    std::vector<std::pair<double, int>> lv;
    for (int v = 0; v < (int)out.V.size(); v++)
      if (out.V[v].key >> i & 1ull) lv.push_back({angle(E[i], out.V[v].z), v});
    std::stable_sort(lv.begin(), lv.end(),
                     [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
                       return a.first < b.first;
                     });
    int nv = (int)lv.size();
    for (int q = 0; q + 1 < nv; q++)
      if (lv[q + 1].first - lv[q].first <= ETA_PHI) out.flags |= F_DEGENERATE | F_ANGLE_TIE;
    for (int q = 0; q < nv; q++) {
      int va = lv[q].second, vb = lv[(q + 1) % nv].second;
      double dph = (q + 1 < nv) ? lv[q + 1].first - lv[q].first : lv[0].first + PI2 - lv[q].first;
      const Vertex& A = out.V[va];
      const Vertex& B = out.V[vb];
      uint64_t cm = (A.key & B.key) & ~(1ull << i);
      bool cs = (A.flags & VF_SPHERE) && (B.flags & VF_SPHERE);
      int ncand = __builtin_popcountll(cm) + (cs ? 1 : 0);
      int label;
      if (ncand == 1) {
        label = cs ? -1 : __builtin_ctzll(cm);
      } else {
        // arg-max of the envelope at the arc's mid-angle, ties -> lowest label
        if (ncand == 0) {
          out.flags |= F_INCONSISTENT;
          cm = ~0ull & ~(1ull << i);
          if (d < 64) cm &= (1ull << d) - 1;
          cs = true;
        }
        double pm = lv[q].first + 0.5 * dph;
        double best = cs ? 0.0 : -INFINITY;
        label = cs ? -1 : -2;
        for (int j = 0; j < d; j++) {
          if (!(cm >> j & 1ull)) continue;
          double h = hval(E[i], E[j], pm, R);
          if (label == -2 || h > best + ETA_SIGMA * R) {
            best = h;
            label = j;
          }
        }
      }
      larcs[i].push_back(LArc{va, vb, label, lv[q].first, dph});
    }
  }

  // ---- activity of flagged pairs
  for (auto& v : out.V)
    for (int i = 0; i < d; i++) {
      if (!(v.key >> i & 1ull)) continue;
      if (v.key & tan_small[i]) out.flags |= F_NEAR_TANGENT;
      if (v.key & tan_neg[i]) out.flags |= F_DEGENERATE | F_STEEP_PAIR;
    }
  {
    uint64_t has_circ = 0;
    for (int i = 0; i < d; i++)
      for (auto& a : larcs[i])
        if (a.label < 0) has_circ |= 1ull << i;
    for (int i = 0; i < d; i++)
      if ((has_circ >> i & 1ull) && (coinc[i] & has_circ)) out.flags |= F_NEAR_TANGENT;
  }

  // ---- node-local arc list: own arcs (circular, or elliptical whose owner is
  // the lower global strut id), ordered by owner then loop position
  std::vector<std::vector<int>> arc_of(d);
  for (int i = 0; i < d; i++) {
    arc_of[i].assign(larcs[i].size(), -1);
    for (size_t q = 0; q < larcs[i].size(); q++) {
      const LArc& a = larcs[i][q];
      bool own = a.label < 0 || E[i].strut < E[a.label].strut;
      if (!own) continue;
      arc_of[i][q] = (int)out.A.size();
      out.A.push_back(Arc{i, a.label, a.va, a.vb, a.phia, a.dphi});
    }
  }
  for (int i = 0; i < d; i++) {
    for (size_t q = 0; q < larcs[i].size(); q++) {
      const LArc& a = larcs[i][q];
      if (arc_of[i][q] >= 0) {
        out.loops[i].push_back(Entry{arc_of[i][q], 0});
        continue;
      }
      int j = a.label, found = -1, rev = 0, nf = 0;
      for (size_t q2 = 0; q2 < larcs[j].size(); q2++) {
        int id = arc_of[j][q2];
        if (id < 0) continue;
        const Arc& o = out.A[id];
        if (o.other != i) continue;
        if (o.v0 == a.va && o.v1 == a.vb) {
          if (found < 0) { found = id; rev = 0; }
          nf++;
        } else if (o.v0 == a.vb && o.v1 == a.va) {
          if (found < 0) { found = id; rev = 1; }
          nf++;
        }
      }
      if (nf != 1 || a.va == a.vb) out.flags |= F_INCONSISTENT;
      if (found < 0) {
        // no partner: keep it as an arc of its own so the loop stays closed
        found = (int)out.A.size();
        out.A.push_back(Arc{i, j, a.va, a.vb, a.phia, a.dphi});
        rev = 0;
      }
      out.loops[i].push_back(Entry{found, rev});
    }
  }

  // ---- arc extent: an elliptical arc must stay within both struts' lengths.
  // h(phi) = (n0 + n1 cos + n2 sin)/(d0 + d1 cos + d2 sin) on the owner i;
  // its extrema satisfy P cos + Q sin = W (derivative of the ratio)
  for (const Arc& a : out.A) {
    if (a.other < 0) continue;
    const End& Ei = E[a.owner];
    const End& Ej = E[a.other];
    double cij = dot(Ei.u, Ej.u), a1 = dot(Ej.u, Ei.e1), a2 = dot(Ej.u, Ei.e2);
    double n0 = R * (Ei.s * cij - Ej.s), n1 = R * Ei.co * a1, n2 = R * Ei.co * a2;
    double d0 = Ej.co - Ei.co * cij, d1 = Ei.s * a1, d2 = Ei.s * a2;
    double tmax = std::max(hval(Ei, Ej, a.phi0, R), hval(Ei, Ej, a.phi0 + a.dphi, R));
    double P = n2 * d0 - n0 * d2, Q = n0 * d1 - n1 * d0, W = n1 * d2 - n2 * d1;
    double rr = std::sqrt(P * P + Q * Q);
    if (rr > std::fabs(W) && rr > 0.0) {
      double base = std::atan2(Q, P), off = std::acos(W / rr);
      for (int sg = -1; sg <= 1; sg += 2) {
        double ph = base + sg * off;
        double rel = std::fmod(ph - a.phi0, PI2);
        if (rel < 0) rel += PI2;
        if (rel < a.dphi) tmax = std::max(tmax, hval(Ei, Ej, a.phi0 + rel, R));
      }
    }
    if (tmax > std::min(Ei.L * Ei.co, Ej.L * Ej.co)) out.flags |= F_DEGENERATE | F_BEYOND_LENGTH;
  }

  // ---- holes: chain circular arcs (hole on the left seen from outside)
  int na = (int)out.A.size();
  std::vector<char> used(na, 0);
  auto hstart = [&](int a) {
    const Arc& x = out.A[a];
    return E[x.owner].at_lo ? x.v1 : x.v0;
  };
  auto hend = [&](int a) {
    const Arc& x = out.A[a];
    return E[x.owner].at_lo ? x.v0 : x.v1;
  };
  for (int a0 = 0; a0 < na; a0++) {
    if (out.A[a0].other >= 0 || used[a0]) continue;
    std::vector<Entry> hole;
    int cur = a0;
    while (true) {
      used[cur] = 1;
      hole.push_back(Entry{cur, E[out.A[cur].owner].at_lo ? 1 : 0});
      int ev = hend(cur);
      if (ev == hstart(a0)) break;
      int nxt = -1, cnt = 0;
      for (int a = 0; a < na; a++) {
        if (out.A[a].other >= 0 || used[a]) continue;
        if (hstart(a) == ev) {
          if (nxt < 0) nxt = a;
          cnt++;
        }
      }
      if (cnt != 1) out.flags |= F_INCONSISTENT;
      if (nxt < 0) break;
      cur = nxt;
    }
    out.holes.push_back(hole);
  }
  return out;
}

// ---------------------------------------------------------------- triangulation

inline int seg_count(double dphi, int k) {
  double x = dphi * (double)k / PI2;
  int n = (int)std::ceil(x - TAU_COUNT);
  return n < 1 ? 1 : n;
}

struct NodeGeo {
  V3 c;
  double R;
  std::vector<End> E;
};

NodeGeo node_geo(const Mesh& M, int64_t n) {
  NodeGeo g;
  g.c = node_xyz(M.lat, n);
  g.R = M.node_R[n];
  for (int64_t b = M.row_ptr[n]; b < M.row_ptr[n + 1]; b++) g.E.push_back(make_end(M, n, M.adj[b]));
  return g;
}

// point m of an arc (Eq. parameter-range, uniform in the owner's angle;
// Section 5: sampled on the strut's end circle and mapped onto the arc)
V3 arc_point(const NodeGeo& g, const NodeOut& no, const Arc& a, int m, int N) {
  if (m == 0) return no.V[a.v0].z;
  if (m == N) return no.V[a.v1].z;
  const End& o = g.E[a.owner];
  double phi = a.phi0 + a.dphi * (double)m / (double)N;
  double t = a.other < 0 ? 0.0 : hval(o, g.E[a.other], phi, g.R);
  return add(mul(wdir(o, phi), g.R), mul(gdir(o, phi), t));
}

struct LoopPts {
  std::vector<V3> z;     // node-relative
  std::vector<double> th;  // unwrapped angle around the strut
};

// Nf: recorded segment counts per node-local arc (frozen topology), or NULL
LoopPts loop_points(const NodeGeo& g, const NodeOut& no, int li, int k, const std::vector<int>* Nf = nullptr) {
  LoopPts P;
  const End& me = g.E[li];
  const std::vector<Entry>& L = no.loops[li];
  for (const Entry& en : L) {
    const Arc& a = no.A[en.arc];
    int N = Nf ? (*Nf)[en.arc] : seg_count(a.dphi, k);
    int vs = en.rev ? a.v1 : a.v0;
    double psi = angle(me, no.V[vs].z);
    for (int s = 0; s < N; s++) {
      int m = en.rev ? N - s : s;
      V3 z = arc_point(g, no, a, m, N);
      double th;
      if (s == 0) {
        th = psi;
      } else if (a.owner == li) {
        th = a.phi0 + a.dphi * (double)m / (double)N;
      } else {
        double r = std::atan2(dot(z, me.e2), dot(z, me.e1)) - psi;
        while (r < -ETA_PHI) r += PI2;
        while (r >= PI2 - ETA_PHI) r -= PI2;
        th = psi + r;
      }
      P.z.push_back(z);
      P.th.push_back(th);
    }
  }
  return P;
}

struct Tri {
  V3 p[3];  // absolute
  V3 n;
  double area, vol;
};

// Discrete structure of a triangulation at k, recorded once and replayed
// with perturbed geometry (the adjoint's reference: topology held fixed).
struct Frozen {
  int k = 0;
  std::vector<std::vector<int>> N;        // [node][arc] segment count
  std::vector<std::vector<uint8_t>> zip;  // [strut] stitching steps, 1 = A advances
  std::vector<std::vector<uint8_t>> fan;  // [node][hole] centre rule (see hole_tris)
  // [node] stitching steps of an annular band (see band_tris), 1 = q0
  // advances; empty: the node's holes are fanned
  std::vector<std::vector<uint8_t>> band;
  std::vector<uint8_t> is_band;  // [node] the two contours were stitched as a band
};

// a, b, c relative to o (an exact node centre) give the STL normal, the area
// and the volume term det(a,b,c) + o.(2 x area vector); pa, pb, pc are the
// absolute coordinates, always formed as (own node centre) + (relative point)
void emit(std::vector<Tri>& T, V3 o, V3 a, V3 b, V3 c, V3 pa, V3 pb, V3 pc) {
  Tri t;
  V3 cr = cross(sub(b, a), sub(c, a));
  double len = norm(cr);
  t.n = len > 0.0 ? mul(cr, 1.0 / len) : mk(0, 0, 0);
  t.area = 0.5 * len;
  t.vol = (dot(a, cross(b, c)) + dot(o, cr)) / 6.0;
  t.p[0] = pa;
  t.p[1] = pb;
  t.p[2] = pc;
  T.push_back(t);
}

// lateral band of strut e: zipper between its loop at the lo node (A) and at
// the hi node (B), both in the strut's angle; ties advance A.
// fz: record the stitching steps into fz (replay = false) or replay them
// and the recorded segment counts (replay = true); NULL: plain evaluation
void strut_tris(const Mesh& M, int64_t e, int k, std::vector<Tri>& T, Frozen* fz = nullptr,
                bool replay = false) {
  int32_t a = M.lat.ends[2 * e], b = M.lat.ends[2 * e + 1];
  int32_t lo = std::min(a, b), hi = std::max(a, b);
  int side_lo = (a == lo) ? 0 : 1;
  int32_t endA = (int32_t)(2 * e + side_lo), endB = (int32_t)(2 * e + (1 - side_lo));
  NodeGeo gA = node_geo(M, lo), gB = node_geo(M, hi);
  int liA = -1, liB = -1;
  for (int64_t q = M.row_ptr[lo]; q < M.row_ptr[lo + 1]; q++)
    if (M.adj[q] == endA) liA = (int)(q - M.row_ptr[lo]);
  for (int64_t q = M.row_ptr[hi]; q < M.row_ptr[hi + 1]; q++)
    if (M.adj[q] == endB) liB = (int)(q - M.row_ptr[hi]);
  const std::vector<int>* NA = replay ? &fz->N[lo] : nullptr;
  const std::vector<int>* NB = replay ? &fz->N[hi] : nullptr;
  LoopPts PA = loop_points(gA, M.nodes[lo], liA, k, NA);
  LoopPts PB = loop_points(gB, M.nodes[hi], liB, k, NB);
  int nA = (int)PA.z.size(), nB = (int)PB.z.size();
  V3 dAB = sub(gB.c, gA.c);
  // B's angles moved into the window [thA0 - ETA_ZIP, thA0 + 2pi - ETA_ZIP)
  // that starts at A's first point; B is rotated to start at its smallest
  // key, and the band starts from the B point just before A's first point.
  // Keys within ETA_PHI of the smallest are ties (the angle tie rule): the
  // first of them in loop order is taken (a loop that runs along an arc and
  // back, on a degenerate node, meets each of its points twice).
  double thA0 = PA.th[0];
  std::vector<double> kB(nB);
  double kmin = INFINITY;
  for (int j = 0; j < nB; j++) {
    double x = PB.th[j];
    while (x < thA0 - ETA_ZIP) x += PI2;
    while (x >= thA0 + PI2 - ETA_ZIP) x -= PI2;
    kB[j] = x;
    kmin = std::min(kmin, x);
  }
  int sB = 0;
  while (kB[sB] > kmin + ETA_PHI) sB++;
  auto thA = [&](int i) { return i < nA ? PA.th[i] : thA0 + PI2; };
  auto thB = [&](int j) { return kB[(sB + j) % nB]; };  // j = 0..nB-1
  auto pA = [&](int i) { return PA.z[i % nA]; };
  auto pB = [&](int j) { return add(dAB, PB.z[(sB + j + nB) % nB]); };
  auto aA = [&](int i) { return add(gA.c, PA.z[i % nA]); };
  auto aB = [&](int j) { return add(gB.c, PB.z[(sB + j + nB) % nB]); };
  // state: current A point ia (0..nA), current B point ib (-1..nB-1);
  // events a_1..a_nA and b_0..b_{nB-1} in key order, ties -> A first
  int ia = 0, ib = -1;
  size_t step = 0;
  if (fz && !replay) fz->zip[e].clear();
  while (ia < nA || ib < nB - 1) {
    bool takeA = (ib == nB - 1) || (ia < nA && thA(ia + 1) <= thB(ib + 1) + ETA_ZIP);
    if (fz && replay) takeA = step < fz->zip[e].size() ? fz->zip[e][step] != 0 : (ia < nA);
    if (fz && !replay) fz->zip[e].push_back(takeA ? 1 : 0);
    step++;
    if (takeA) {
      emit(T, gA.c, pA(ia), pA(ia + 1), pB(ib), aA(ia), aA(ia + 1), aB(ib));
      ia++;
    } else {
      emit(T, gA.c, pA(ia), pB(ib + 1), pB(ib), aA(ia), aB(ib + 1), aB(ib));
      ib++;
    }
  }
}

// Annular exposed component (reading 10): the band between its two contours
// q0 and q1 (node-relative points in hole order, each contour with the
// component on its left seen from outside), stitched like a strut's lateral
// band (reading 8).  Both contours are taken in the angle around the axis a
// from q0's barycentre to q1's (frame as the strut frames: e1 = a x E_ax
// with ax the axis of smallest |a_ax|, e2 = a x e1), q0 forward and q1
// backward, so that both turn once positively; q0 starts at its first point,
// q1's keys are moved into the window [th0 - ETA_ZIP, th0 + 2pi - ETA_ZIP)
// and q1 starts at its smallest key (ties within ETA_PHI: the first); an
// event of q0 comes first unless it exceeds q1's by more than ETA_ZIP.
// Returns false (the holes are then fanned) when the barycentres are within
// ETA_BARY R of each other or a contour does not turn once around a.
// rec / rep: record / replay the stitching steps (frozen structure).
bool band_tris(const NodeGeo& g, const std::vector<V3>& q0, const std::vector<V3>& q1, std::vector<Tri>& T,
               std::vector<uint8_t>* rec, const std::vector<uint8_t>* rep) {
  const int M0 = (int)q0.size(), M1 = (int)q1.size();
  if (M0 < 1 || M1 < 1) return false;
  V3 b0 = mk(0, 0, 0), b1 = mk(0, 0, 0);
  for (const V3& p : q0) b0 = add(b0, p);
  for (const V3& p : q1) b1 = add(b1, p);
  V3 a = sub(mul(b1, 1.0 / M1), mul(b0, 1.0 / M0));
  const double al = norm(a);
  if (!rep && al <= ETA_BARY * g.R) return false;
  a = mul(a, 1.0 / al);
  double aa[3] = {std::fabs(a.x), std::fabs(a.y), std::fabs(a.z)};
  int ax = 0;
  if (aa[1] < aa[ax]) ax = 1;
  if (aa[2] < aa[ax]) ax = 2;
  V3 c1 = cross(a, mk(ax == 0, ax == 1, ax == 2));
  const V3 e1 = mul(c1, 1.0 / norm(c1)), e2 = cross(a, e1);
  auto ang = [&](V3 p) { return std::atan2(dot(p, e2), dot(p, e1)); };
  // q1 backward from its first point
  auto qb = [&](int j) { return q1[((M1 - j) % M1 + M1) % M1]; };
  // each contour turns once positively around a
  auto turn = [&](int M, auto pt) {
    double t = 0.0;
    for (int i = 0; i < M; i++) {
      double r = ang(pt((i + 1) % M)) - ang(pt(i));
      while (r <= -0.5 * PI2) r += PI2;
      while (r > 0.5 * PI2) r -= PI2;
      t += r;
    }
    return t;
  };
  if (!rep && (std::fabs(turn(M0, [&](int i) { return q0[i]; }) - PI2) > 1e-6 ||
               std::fabs(turn(M1, qb) - PI2) > 1e-6))
    return false;
  const double th0 = ang(q0[0]);
  std::vector<double> kA(M0), kB(M1);
  for (int i = 0; i < M0; i++) {
    double r = ang(q0[i]) - th0;
    while (r < -ETA_PHI) r += PI2;
    while (r >= PI2 - ETA_PHI) r -= PI2;
    kA[i] = th0 + r;
  }
  double kmin = INFINITY;
  for (int j = 0; j < M1; j++) {
    double x = ang(qb(j));
    while (x < th0 - ETA_ZIP) x += PI2;
    while (x >= th0 + PI2 - ETA_ZIP) x -= PI2;
    kB[j] = x;
    kmin = std::min(kmin, x);
  }
  int sB = 0;
  while (kB[sB] > kmin + ETA_PHI) sB++;
  auto thA = [&](int i) { return i < M0 ? kA[i] : th0 + PI2; };
  auto thB = [&](int j) { return kB[(sB + j) % M1]; };
  auto pA = [&](int i) { return q0[i % M0]; };
  auto pB = [&](int j) { return qb((sB + j + M1) % M1); };
  int ia = 0, ib = -1;
  size_t step = 0;
  if (rec) rec->clear();
  while (ia < M0 || ib < M1 - 1) {
    bool takeA = (ib == M1 - 1) || (ia < M0 && thA(ia + 1) <= thB(ib + 1) + ETA_ZIP);
    if (rep) takeA = step < rep->size() ? (*rep)[step] != 0 : (ia < M0);
    if (rec) rec->push_back(takeA ? 1 : 0);
    step++;
    if (takeA) {
      emit(T, g.c, pA(ia), pA(ia + 1), pB(ib), add(g.c, pA(ia)), add(g.c, pA(ia + 1)), add(g.c, pB(ib)));
      ia++;
    } else {
      emit(T, g.c, pA(ia), pB(ib + 1), pB(ib), add(g.c, pA(ia)), add(g.c, pB(ib + 1)), add(g.c, pB(ib)));
      ib++;
    }
  }
  return true;
}

// hole fans of node n (Section 5 hole filling)
// fz: record (replay = false) or replay (replay = true) the centre rule of
// every hole and the segment counts; NULL: plain evaluation
void hole_tris(const Mesh& M, int64_t n, int k, std::vector<Tri>& T, Frozen* fz = nullptr,
               bool replay = false) {
  const NodeOut& no = M.nodes[n];
  if (no.holes.empty()) return;
  NodeGeo g = node_geo(M, n);
  if (fz && !replay) fz->fan[n].assign(no.holes.size(), 0);
  // contour points of hole hh (node-relative, hole order)
  auto contour = [&](size_t hh) {
    std::vector<V3> q;
    for (const Entry& en : no.holes[hh]) {
      const Arc& a = no.A[en.arc];
      int N = replay ? fz->N[n][en.arc] : seg_count(a.dphi, k);
      for (int s = 0; s < N; s++) q.push_back(arc_point(g, no, a, en.rev ? N - s : s, N));
    }
    return q;
  };
  // reading 10: two contours that bound one exposed component of the nodal
  // sphere (the node's partition of its sphere into d loops and the exposed
  // components gives V - A + d + 2F - H = 2, so F = 1 when
  // A - V - d + 4 = 2 with H = 2) are stitched as a band
  if (fz && !replay) fz->is_band[n] = 0;
  if (no.holes.size() == 2 && (int64_t)no.A.size() - (int64_t)no.V.size() - (int64_t)g.E.size() + 4 == 2) {
    const bool rep_band = replay && fz->is_band[n];
    if (!replay || rep_band) {
      std::vector<uint8_t>* rec = fz && !replay ? &fz->band[n] : nullptr;
      if (band_tris(g, contour(0), contour(1), T, rec, rep_band ? &fz->band[n] : nullptr)) {
        if (fz && !replay) fz->is_band[n] = 1;
        return;
      }
    }
  }
  for (size_t hh = 0; hh < no.holes.size(); hh++) {
    std::vector<V3> q = contour(hh);
    int Mq = (int)q.size();
    V3 b = mk(0, 0, 0);
    for (auto& p : q) b = add(b, p);
    b = mul(b, 1.0 / Mq);
    // b_project = o + R (b - o)/|b - o|, falling back to the direction away
    // from the struts when b is at the centre or outside the hole region
    auto in_hole = [&](V3 dir) {
      for (const End& e : g.E)
        if (dot(e.u, dir) > e.s) return false;
      return true;
    };
    // rule: 0 barycentre direction, 1 -sum u, 2 barycentre (no -sum u), 3 -u_0
    V3 dir = mk(0, 0, 0);
    double bl = norm(b);
    V3 su = mk(0, 0, 0);
    for (const End& e : g.E) su = sub(su, e.u);
    double sl = norm(su);
    int rule;
    if (replay) {
      rule = fz->fan[n][hh];
    } else {
      rule = -1;
      if (bl > ETA_BARY * g.R && in_hole(mul(b, 1.0 / bl))) rule = 0;
      else if (sl > ETA_BARY) rule = 1;
      else if (bl > 0.0) rule = 2;
      else rule = 3;
      if (fz) fz->fan[n][hh] = (uint8_t)rule;
    }
    if (rule == 0 || rule == 2) dir = mul(b, 1.0 / bl);
    else if (rule == 1) dir = mul(su, 1.0 / sl);
    else dir = mul(g.E[0].u, -1.0);
    V3 bp = mul(dir, g.R);
    for (int m = 0; m < Mq; m++) {
      V3 q1 = q[(m + 1) % Mq];
      emit(T, g.c, bp, q[m], q1, add(g.c, bp), add(g.c, q[m]), add(g.c, q1));
    }
  }
}

// ----------------------------------------------- frozen-topology objective
// Reference of the adjoint: d(area, volume)/d(node positions, radii) with the
// discrete structure held fixed (vertex generators, arcs, loops, holes,
// segment counts, stitching order, fan-centre rule).  Geometry is recomputed
// from perturbed parameters: each vertex from its generator (the formulas of
// node_metamesh: circle point, triple point with the same root, seam), each
// arc's angles from its end vertices (followed continuously from the recorded
// values), then points and triangles as in strut_tris / hole_tris.

// node-relative vertex of generator `gen` from the node's strut ends
V3 vertex_from_gen(const std::vector<End>& E, double R, uint32_t gen) {
  int type = gen & 3, root = (gen >> 2) & 1;
  int i = (gen >> 3) & 63, j = (gen >> 9) & 63, k = (gen >> 15) & 63;
  if (type == 0) {
    double c = dot(E[i].u, E[j].u);
    double q = 1.0 - c * c;
    double al = (E[i].s - c * E[j].s) / q;
    double be = (E[j].s - c * E[i].s) / q;
    double g2 = 1.0 - (al * al + be * be + 2.0 * al * be * c);
    V3 w = cross(E[i].u, E[j].u);
    w = mul(w, 1.0 / norm(w));
    double g = std::sqrt(std::max(g2, 0.0));
    return mul(add(add(mul(E[i].u, al), mul(E[j].u, be)), mul(w, root == 0 ? -g : g)), R);
  }
  if (type == 1) {
    V3 mj = sub(mul(E[i].u, 1.0 / E[i].co), mul(E[j].u, 1.0 / E[j].co));
    V3 mk_ = sub(mul(E[i].u, 1.0 / E[i].co), mul(E[k].u, 1.0 / E[k].co));
    double dj = R * (E[i].s / E[i].co - E[j].s / E[j].co);
    double dk = R * (E[i].s / E[i].co - E[k].s / E[k].co);
    V3 v = cross(mj, mk_);
    double vv = dot(v, v);
    V3 z0 = mul(sub(mul(cross(mk_, v), dj), mul(cross(mj, v), dk)), 1.0 / vv);
    V3 vh = mul(v, 1.0 / std::sqrt(vv));
    double G0 = (dot(E[i].u, z0) - R * E[i].s) / E[i].co;
    double G1 = dot(E[i].u, vh) / E[i].co;
    double A = 1.0 - G1 * G1;
    double B = -G0 * G1;
    double C = dot(z0, z0) - R * R - G0 * G0;
    double sq = std::sqrt(std::max(B * B - A * C, 0.0));
    // roots (-B - sq)/A and (-B + sq)/A, in the stable form
    double lam;
    if (B >= 0.0) {
      double q = -(B + sq);
      lam = root == 0 ? q / A : C / q;
    } else {
      double q = -B + sq;
      lam = root == 1 ? q / A : C / q;
    }
    return add(z0, mul(vh, lam));
  }
  // seam at angle 0 of strut end i, on plane P_ij when labelled
  double t = (gen >> 21) & 1 ? hval(E[i], E[j], 0.0, R) : 0.0;
  return add(mul(wdir(E[i], 0.0), R), mul(gdir(E[i], 0.0), t));
}

inline double wrap_pi(double x) { return x - PI2 * std::nearbyint(x / PI2); }

// geometry of node n recomputed from the (perturbed) lattice of M2, with the
// discrete structure of `base`
void refresh_node(const Mesh& M2, const NodeOut& base, NodeOut& out, int64_t n) {
  if (base.V.empty() && base.A.empty()) return;
  NodeGeo g = node_geo(M2, n);
  for (size_t v = 0; v < base.V.size(); v++) out.V[v].z = vertex_from_gen(g.E, g.R, base.V[v].gen);
  for (size_t a = 0; a < base.A.size(); a++) {
    const Arc& b = base.A[a];
    const End& o = g.E[b.owner];
    auto ang = [&](V3 z) { return std::atan2(dot(z, o.e2), dot(z, o.e1)); };
    double p0 = b.phi0 + wrap_pi(ang(out.V[b.v0].z) - b.phi0);
    double dp = PI2;
    if (b.v0 != b.v1) {
      double e1 = b.phi0 + b.dphi;
      dp = e1 + wrap_pi(ang(out.V[b.v1].z) - e1) - p0;
    }
    out.A[a].phi0 = p0;
    out.A[a].dphi = dp;
  }
}

// items (strut bands, then node holes) whose triangles depend on node v
void items_of(const Mesh& M, int64_t v, std::vector<int64_t>& struts, std::vector<int64_t>& nodes) {
  nodes.clear();
  struts.clear();
  nodes.push_back(v);
  for (int64_t q = M.row_ptr[v]; q < M.row_ptr[v + 1]; q++) {
    int32_t e = M.adj[q] >> 1;
    int32_t a = M.lat.ends[2 * e], b = M.lat.ends[2 * e + 1];
    nodes.push_back(a == v ? b : a);
  }
  for (int64_t w : nodes)
    for (int64_t q = M.row_ptr[w]; q < M.row_ptr[w + 1]; q++) struts.push_back(M.adj[q] >> 1);
  std::sort(struts.begin(), struts.end());
  struts.erase(std::unique(struts.begin(), struts.end()), struts.end());
  std::sort(nodes.begin(), nodes.end());
  nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
}

void sum_items(const Mesh& M2, Frozen* fz, const std::vector<int64_t>& struts,
               const std::vector<int64_t>& nodes, double* acc) {
  std::vector<Tri> T;
  for (int64_t e : struts) {
    T.clear();
    strut_tris(M2, e, fz->k, T, fz, true);
    for (auto& t : T) { acc[0] += t.area; acc[1] += t.vol; }
  }
  for (int64_t n : nodes) {
    T.clear();
    hole_tris(M2, n, fz->k, T, fz, true);
    for (auto& t : T) { acc[0] += t.area; acc[1] += t.vol; }
  }
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

// status: 0 ok, 1 invalid argument, 2 radius mismatch
void* lmo_build(int64_t n_nodes, int64_t n_struts, const double* xyz, const int32_t* ends,
                const double* radii, int* status) {
  Mesh* M = new Mesh();
  M->lat = Lattice{n_nodes, n_struts, xyz, ends, radii};
  *status = 0;
  std::vector<int64_t> deg(n_nodes, 0);
  M->node_R.assign(n_nodes, NAN);
  for (int64_t e = 0; e < n_struts; e++) {
    for (int s = 0; s < 2; s++) {
      int32_t nd = ends[2 * e + s];
      if (nd < 0 || nd >= n_nodes || !(radii[2 * e + s] > 0.0)) {
        *status = 1;
        return M;
      }
      deg[nd]++;
      double r = radii[2 * e + s];
      if (std::isnan(M->node_R[nd])) M->node_R[nd] = r;
      else if (std::fabs(M->node_R[nd] - r) > 1e-12 * std::fabs(r)) {
        *status = 2;
        return M;
      }
    }
    if (ends[2 * e] == ends[2 * e + 1]) {
      *status = 1;
      return M;
    }
  }
  for (int64_t e = 0; e < n_struts; e++) {
    int32_t a = ends[2 * e], b = ends[2 * e + 1];
    V3 d = sub(node_xyz(M->lat, b), node_xyz(M->lat, a));
    if (!(std::fabs(M->node_R[a] - M->node_R[b]) < norm(d))) {
      *status = 3;
      return M;
    }
  }
  M->row_ptr.assign(n_nodes + 1, 0);
  for (int64_t v = 0; v < n_nodes; v++) {
    if (deg[v] > 64) {
      *status = 1;
      return M;
    }
    M->row_ptr[v + 1] = M->row_ptr[v] + deg[v];
  }
  M->adj.assign(2 * n_struts, 0);
  std::vector<int64_t> fill(M->row_ptr.begin(), M->row_ptr.end() - 1);
  for (int64_t e = 0; e < n_struts; e++)
    for (int s = 0; s < 2; s++) M->adj[fill[ends[2 * e + s]]++] = (int32_t)(2 * e + s);
  M->nodes.resize(n_nodes);
  return M;
}

// meta-mesh of nodes [n0, n1) (all nodes: 0, n_nodes)
void lmo_metamesh(void* h, int64_t n0, int64_t n1) {
  Mesh* M = (Mesh*)h;
  for (int64_t n = n0; n < n1; n++) M->nodes[n] = node_metamesh(*M, n);
}

void lmo_free(void* h) { delete (Mesh*)h; }

// per-node sizes: out[n*6 + {0..5}] = flags, V, arcs, loop entries, holes, hole entries
void lmo_node_sizes(void* h, int64_t n0, int64_t n1, int64_t* out) {
  Mesh* M = (Mesh*)h;
  for (int64_t n = n0; n < n1; n++) {
    const NodeOut& no = M->nodes[n];
    int64_t le = 0, he = 0;
    for (auto& l : no.loops) le += (int64_t)l.size();
    for (auto& l : no.holes) he += (int64_t)l.size();
    int64_t* o = out + 6 * (n - n0);
    o[0] = no.flags;
    o[1] = (int64_t)no.V.size();
    o[2] = (int64_t)no.A.size();
    o[3] = le;
    o[4] = (int64_t)no.holes.size();
    o[5] = he;
  }
}

// Export one node.  Arrays sized from lmo_node_sizes.
//   vz[V][3], vkey[V], vflags[V], vgen[V]
//   arc_i[A][4] = owner_end_id, other_end_id(-1), v0, v1 ; arc_f[A][2] = phi0, dphi
//   loop_len[d], loop_ent[le] (arc | rev<<31) in local-end order
//   hole_len[H], hole_ent[he]
void lmo_node_export(void* h, int64_t n, double* vz, uint64_t* vkey, uint32_t* vflags,
                     uint32_t* vgen, int32_t* arc_i, double* arc_f, int32_t* loop_len,
                     uint32_t* loop_ent, int32_t* hole_len, uint32_t* hole_ent) {
  Mesh* M = (Mesh*)h;
  const NodeOut& no = M->nodes[n];
  int64_t b0 = M->row_ptr[n];
  for (size_t v = 0; v < no.V.size(); v++) {
    vz[3 * v] = no.V[v].z.x;
    vz[3 * v + 1] = no.V[v].z.y;
    vz[3 * v + 2] = no.V[v].z.z;
    vkey[v] = no.V[v].key;
    vflags[v] = no.V[v].flags;
    vgen[v] = no.V[v].gen;
  }
  for (size_t a = 0; a < no.A.size(); a++) {
    const Arc& x = no.A[a];
    arc_i[4 * a] = M->adj[b0 + x.owner];
    arc_i[4 * a + 1] = x.other < 0 ? -1 : M->adj[b0 + x.other];
    arc_i[4 * a + 2] = x.v0;
    arc_i[4 * a + 3] = x.v1;
    arc_f[2 * a] = x.phi0;
    arc_f[2 * a + 1] = x.dphi;
  }
  size_t p = 0;
  for (size_t i = 0; i < no.loops.size(); i++) {
    loop_len[i] = (int32_t)no.loops[i].size();
    for (auto& en : no.loops[i]) loop_ent[p++] = (uint32_t)en.arc | ((uint32_t)en.rev << 31);
  }
  p = 0;
  for (size_t hh = 0; hh < no.holes.size(); hh++) {
    hole_len[hh] = (int32_t)no.holes[hh].size();
    for (auto& en : no.holes[hh]) hole_ent[p++] = (uint32_t)en.arc | ((uint32_t)en.rev << 31);
  }
}

// triangle count of items [i0, i1): items 0..E-1 are struts (lateral band),
// E..E+N-1 are nodes (hole fans)
void lmo_tri_counts(void* h, int k, int64_t i0, int64_t i1, int64_t* out) {
  Mesh* M = (Mesh*)h;
  int64_t E = M->lat.n_struts;
  for (int64_t it = i0; it < i1; it++) {
    int64_t c = 0;
    if (it < E) {
      int32_t a = M->lat.ends[2 * it], b = M->lat.ends[2 * it + 1];
      for (int s = 0; s < 2; s++) {
        int32_t nd = s == 0 ? a : b;
        int32_t eid = (int32_t)(2 * it + s);
        const NodeOut& no = M->nodes[nd];
        for (int64_t q = M->row_ptr[nd]; q < M->row_ptr[nd + 1]; q++) {
          if (M->adj[q] != eid) continue;
          for (auto& en : no.loops[q - M->row_ptr[nd]]) c += seg_count(no.A[en.arc].dphi, k);
        }
      }
    } else {
      const NodeOut& no = M->nodes[it - E];
      for (auto& hole : no.holes)
        for (auto& en : hole) c += seg_count(no.A[en.arc].dphi, k);
    }
    out[it - i0] = c;
  }
}

// triangles of items [i0, i1) in output order: tris[t][12] = normal, v0, v1, v2;
// returns the count; area/volume of these triangles added to acc[0], acc[1]
int64_t lmo_triangulate(void* h, int k, int64_t i0, int64_t i1, double* tris, double* acc) {
  Mesh* M = (Mesh*)h;
  int64_t E = M->lat.n_struts;
  int64_t t = 0;
  std::vector<Tri> T;
  for (int64_t it = i0; it < i1; it++) {
    T.clear();
    if (it < E) strut_tris(*M, it, k, T);
    else hole_tris(*M, it - E, k, T);
    for (auto& x : T) {
      if (tris) {
        double* o = tris + 12 * t;
        o[0] = x.n.x; o[1] = x.n.y; o[2] = x.n.z;
        for (int v = 0; v < 3; v++) {
          o[3 + 3 * v] = x.p[v].x;
          o[4 + 3 * v] = x.p[v].y;
          o[5 + 3 * v] = x.p[v].z;
        }
      }
      if (acc) {
        acc[0] += x.area;
        acc[1] += x.vol;
      }
      t++;
    }
  }
  return t;
}

// the N+1 points (node-relative) of node-local arc a of node n at resolution k
int lmo_arc_points(void* h, int64_t n, int a, int k, double* out) {
  Mesh* M = (Mesh*)h;
  const NodeOut& no = M->nodes[n];
  NodeGeo g = node_geo(*M, n);
  const Arc& x = no.A[a];
  int N = seg_count(x.dphi, k);
  for (int m = 0; m <= N; m++) {
    V3 z = arc_point(g, no, x, m, N);
    out[3 * m] = z.x;
    out[3 * m + 1] = z.y;
    out[3 * m + 2] = z.z;
  }
  return N;
}

// envelope t*(phi) = max(0, max_j h_j(phi)) on local end li of node n and its
// arg-max label (-1 = sphere), by direct evaluation (brute-force checks)
void lmo_envelope(void* h, int64_t n, int li, int64_t np, const double* phi, double* t,
                  int32_t* label) {
  Mesh* M = (Mesh*)h;
  NodeGeo g = node_geo(*M, n);
  int d = (int)g.E.size();
  for (int64_t q = 0; q < np; q++) {
    double best = 0.0;
    int lab = -1;
    for (int j = 0; j < d; j++) {
      if (j == li) continue;
      double hv = hval(g.E[li], g.E[j], phi[q], g.R);
      if (hv > best) {
        best = hv;
        lab = j;
      }
    }
    t[q] = best;
    label[q] = lab;
  }
}

// the oracle's CSR, node radii and per-end frames (for host-side checks)
void lmo_csr(void* h, int64_t* row_ptr, int32_t* adj, double* node_R) {
  Mesh* M = (Mesh*)h;
  std::memcpy(row_ptr, M->row_ptr.data(), sizeof(int64_t) * M->row_ptr.size());
  std::memcpy(adj, M->adj.data(), sizeof(int32_t) * M->adj.size());
  std::memcpy(node_R, M->node_R.data(), sizeof(double) * M->node_R.size());
}

// frame of the strut end with local index li at node n: u, e1, e2, s, co
void lmo_end_frame(void* h, int64_t n, int li, double* out) {
  Mesh* M = (Mesh*)h;
  End e = make_end(*M, n, M->adj[M->row_ptr[n] + li]);
  double v[11] = {e.u.x, e.u.y, e.u.z, e.e1.x, e.e1.y, e.e1.z, e.e2.x, e.e2.y, e.e2.z, e.s, e.co};
  std::memcpy(out, v, sizeof(v));
}

// ---- frozen-topology objective (adjoint reference)
// record the discrete structure of the triangulation at k (meta-mesh of all
// nodes must be built)
void* lmo_frozen_record(void* h, int k) {
  Mesh* M = (Mesh*)h;
  Frozen* fz = new Frozen();
  fz->k = k;
  int64_t N = M->lat.n_nodes, E = M->lat.n_struts;
  fz->N.resize(N);
  fz->zip.resize(E);
  fz->fan.resize(N);
  fz->band.resize(N);
  fz->is_band.assign(N, 0);
  for (int64_t n = 0; n < N; n++)
    for (const Arc& a : M->nodes[n].A) fz->N[n].push_back(seg_count(a.dphi, k));
  std::vector<Tri> T;
  for (int64_t e = 0; e < E; e++) { T.clear(); strut_tris(*M, e, k, T, fz, false); }
  for (int64_t n = 0; n < N; n++) { T.clear(); hole_tris(*M, n, k, T, fz, false); }
  return fz;
}

void lmo_frozen_free(void* fz) { delete (Frozen*)fz; }

// area and volume (out[0], out[1]) of the recorded structure evaluated at
// node positions xyz [N][3] and node radii node_R [N]
void lmo_frozen_objective(void* h, void* f, const double* xyz, const double* node_R, double* out) {
  Mesh* M = (Mesh*)h;
  Frozen* fz = (Frozen*)f;
  Mesh M2;
  M2.lat = M->lat;
  M2.lat.xyz = xyz;
  M2.node_R.assign(node_R, node_R + M->lat.n_nodes);
  M2.row_ptr = M->row_ptr;
  M2.adj = M->adj;
  M2.nodes = M->nodes;
  for (int64_t n = 0; n < M->lat.n_nodes; n++) refresh_node(M2, M->nodes[n], M2.nodes[n], n);
  std::vector<int64_t> struts(M->lat.n_struts), nodes(M->lat.n_nodes);
  for (int64_t e = 0; e < M->lat.n_struts; e++) struts[e] = e;
  for (int64_t n = 0; n < M->lat.n_nodes; n++) nodes[n] = n;
  out[0] = out[1] = 0.0;
  sum_items(M2, fz, struts, nodes, out);
}

// central differences with step `step` of the recorded structure's area and
// volume for the nodes in `list`: g[8 q + 0..3] = d area / d(x, y, z, R) of
// node list[q], g[8 q + 4..7] the same for the volume.  Only the items that
// depend on the perturbed node are re-evaluated.
void lmo_frozen_fd(void* h, void* f, double step, const int64_t* list, int64_t n_list, double* g) {
  Mesh* M = (Mesh*)h;
  Frozen* fz = (Frozen*)f;
  int64_t N = M->lat.n_nodes;
  std::vector<double> xyz(M->lat.xyz, M->lat.xyz + 3 * N);
  Mesh M2;
  M2.lat = M->lat;
  M2.lat.xyz = xyz.data();
  M2.node_R = M->node_R;
  M2.row_ptr = M->row_ptr;
  M2.adj = M->adj;
  M2.nodes = M->nodes;
  std::vector<int64_t> struts, nodes;
  for (int64_t q = 0; q < n_list; q++) {
    int64_t v = list[q];
    items_of(*M, v, struts, nodes);
    for (int p = 0; p < 4; p++) {
      double acc[2][2] = {{0, 0}, {0, 0}};
      for (int sg = 0; sg < 2; sg++) {
        double d = sg == 0 ? step : -step;
        if (p < 3) xyz[3 * v + p] = M->lat.xyz[3 * v + p] + d;
        else M2.node_R[v] = M->node_R[v] + d;
        for (int64_t w : nodes) refresh_node(M2, M->nodes[w], M2.nodes[w], w);
        sum_items(M2, fz, struts, nodes, acc[sg]);
      }
      if (p < 3) xyz[3 * v + p] = M->lat.xyz[3 * v + p];
      else M2.node_R[v] = M->node_R[v];
      g[8 * q + p] = (acc[0][0] - acc[1][0]) / (2.0 * step);
      g[8 * q + 4 + p] = (acc[0][1] - acc[1][1]) / (2.0 * step);
    }
    for (int64_t w : nodes) M2.nodes[w] = M->nodes[w];
  }
}

}  // extern "C"
