// Device side of concurrent Bowyer-Watson insertion (Algorithm 1 per point, Section 3 rules).
//
// One insertion round processes R candidate points in three phases separated by kernel
// boundaries (or block barriers), so every read of the triangulation in phases 1-2 sees the
// same state:
//   1. walk (thread per point): visibility walk with orient3d (Section 2.1, ghost rules of
//      Section 2.6) to a tetrahedron in conflict with p;
//   2. cavity (warp per point): breadth-first search over tetrahedra in conflict (perturbed
//      insphere, composite ghost sphere), recording the cavity C and its boundary facets. Each
//      tetrahedron has two claim words, X (priorities of points that delete or touch it) and
//      Y (priorities of points that delete it); a point with priority (round stamp << 32 |
//      point id + 1) raises X and Y on its cavity C and X on its outside neighbours A;
//   3. insert (warp per point): a point wins when X == its priority on all of C and Y is below
//      its priority on all of A. Then no other winner deletes or touches its C and no other
//      winner deletes its A (rules (1a)(1b) of Section 3.2); two winners may share outside
//      tetrahedra, each rewriting a different facet slot. The winner replaces C by
//      the ball B (Section 2.5): one tetrahedron per boundary facet, the cavity tetrahedron
//      with its vertex opposite the facet replaced by p, adjacency to the outside tetrahedron
//      known a priori, adjacencies between new tetrahedra through the n x n edge table of
//      oriented boundary edges (hash fallback for large cavities), slots taken from the
//      cavity first, then from the free list, then from the bump pointer (rule (2)).
// The highest-priority located point of a round always wins, so every round makes progress.
#pragma once
#include "common.cuh"
#include "predicates.cuh"

namespace dtg {

enum CandStatus : uint32_t {
  kCandEmpty = 0,
  kCandLocated = 1,
  kCandWalkLimit = 2,
  kCandDup = 3,
  kCandLost = 4,
  kCandBig = 5,
  kCandInserted = 6,
};

constexpr int kCMax = 64;   // cavity tetrahedra on the shared-memory path
constexpr int kFMax = 60;   // boundary facets on the shared-memory path (<= 32 boundary vertices)
constexpr int kHash = 256;  // visited-set slots per warp (shared-memory path)

struct Ctx {
  Tet* tets;
  unsigned long long* claim;  // claim[2t] = X, claim[2t + 1] = Y of tetrahedron t
  const Pt* pts;   // exact coordinates; .w = input index (the perturbation order)
  const PtF* ptf;  // double-float copy for the FP32 first stage of the predicates
  float eta;       // absolute error of a double-float difference (see predicates.cuh)
  uint32_t* freelist;
  uint32_t* pending;
  uint32_t* cell_hint;    // fine grid: a recent tetrahedron per cell
  uint32_t* cell_hint2;   // coarse grid (8 x 8 x 8 fine cells per coarse cell)
  uint32_t* point_hint;   // per vertex: where its last walk ended / its ball
  DevState* st;
  float lo[3], sc[3];  // hint grid: cell = floor((x - lo) * sc), clamped (a hint, not exact)
  int cb;  // bits per axis of the hint grid
  uint32_t max_walk;
  int coherent;  // 1 when this kernel also writes the tetrahedra it reads (L2 loads)
  uint32_t ntets;  // tetrahedron slots allocated (bounds of every id read from the mesh)
  uint32_t npts;   // vertex slots allocated
  float4* subdet;  // sub-determinant cache of the asynchronous engine (two float4 per slot) or
                   // null; the engines that do not fill it mark the entries they replace invalid
};

// Claim priority of point p in the current round. Section 3.2 settles conflicts by a total
// order of the points, and any strict order yields the same triangulation: the round's stamp
// (so older claims never win), then a scheduling rank (0 unless the learned schedule sets one:
// points expected to have small cavities first), then the point's index.
__device__ __forceinline__ unsigned long long claim_prio(unsigned long long stamp, uint32_t rank8, uint32_t p) {
  return (stamp << 40) | ((unsigned long long)rank8 << 32) | (unsigned long long)(p + 1u);
}

// Training labels of the learned scheduler (DT_FLAG_LOG), kept out of Ctx so the kernels that
// do not log carry no extra registers: the cavity of each insertion and the conflicts a point
// lost on the way.
struct InsertLog {
  uint16_t* nc;   // per vertex: |C| of its insertion (null: not logging)
  uint8_t* lost;  // per vertex: conflicts lost before it (saturating)
};

__device__ __forceinline__ void log_outcome(const InsertLog& g, uint32_t p, uint32_t status, int nc) {
  if (!g.nc) return;
  if (status == kCandInserted) g.nc[p] = (uint16_t)(nc < 65535 ? nc : 65535);
  else if (status == kCandLost && g.lost[p] < 255) g.lost[p] += 1;
}

// A tetrahedron record read from the mesh only references allocated vertices and slots; a
// record that does not raises kErrInternal (the kernels then stop using it) instead of
// letting a bad id reach memory.
__device__ __forceinline__ bool tet_sane(const Ctx& c, const Tet& T) {
  bool ok = true;
  for (int k = 0; k < 4; ++k) {
    uint32_t v = get4(T.v, k), n = get4(T.n, k);
    ok = ok && (v == kGhost || v < c.npts) && n < c.ntets;
  }
  return ok;
}

__device__ __forceinline__ Tet tet_at(const Ctx& c, uint32_t t) {
  return c.coherent ? load_tet_cg(c.tets, t) : load_tet(c.tets, t);
}

__device__ __forceinline__ uint32_t nbr_at(const Ctx& c, uint32_t t, int f) {
  const uint32_t* p = reinterpret_cast<const uint32_t*>(&c.tets[t].n) + f;
  return c.coherent ? __ldcg(p) : __ldg(p);
}

// Working storage of one cavity search (shared memory per warp, or global for large cavities).
struct CavWS {
  uint32_t* hkey;
  uint8_t* hval;  // 1 = in cavity, 2 = outside
  uint32_t hmask;
  uint32_t* clist;
  uint32_t cmax;
  uint32_t* blist;  // boundary facets as 4 * (position of the cavity tetrahedron in clist) + facet
  uint32_t bmax;
};

// Working storage of one ball construction.
struct InsWS {
  uint4* nv;
  uint4* nn;  // neighbours of the new tetrahedra, validated before anything is written
  uint32_t* outh;
  uint32_t* slot;
  uint8_t* ipos;  // facet of new tetrahedron i on the boundary | 4 * the outside tetrahedron's facet
  uint32_t* vkey;  // 32-slot vertex hash: slot = cavity-local vertex index
  uint16_t* tab;   // 32 x 32 edge table: 4 * (new tetrahedron) + facet
  unsigned long long* ekey;
  uint32_t* eval;
  uint32_t* hslot;
  uint32_t* hold;
  uint32_t emask;
};

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Fine and coarse hint-grid cells of P.
__device__ __forceinline__ void cells_of(const Ctx& c, const PtF& P, uint32_t* fine, uint32_t* coarse) {
  const float x[3] = {P.hx, P.hy, P.hz};
  const float lim = (float)((1u << c.cb) - 1u);
  uint32_t q[3];
  for (int k = 0; k < 3; ++k) {
    float f = floorf((x[k] - c.lo[k]) * c.sc[k]);
    f = f < 0.0f ? 0.0f : (f > lim ? lim : f);  // also maps NaN to 0
    q[k] = (uint32_t)f;
  }
  *fine = (q[2] << (2 * c.cb)) | (q[1] << c.cb) | q[0];
  int cc = c.cb > 3 ? c.cb - 3 : 1, sh = c.cb - cc;
  *coarse = ((q[2] >> sh) << (2 * cc)) | ((q[1] >> sh) << cc) | (q[0] >> sh);
}

// Positions (a, b, c) such that (p, w[a], w[b], w[c]) is an even permutation of a tetrahedron
// w with p at position i.
// i = 0: (1,2,3); 1: (0,3,2); 2: (0,1,3); 3: (0,2,1).
__device__ __forceinline__ void after_pos(int i, int& a, int& b, int& c) {
  a = (i == 0) ? 1 : 0;
  b = (i == 0) ? 2 : (i == 1) ? 3 : (i == 2) ? 1 : 2;
  c = (i == 0) ? 3 : (i == 1) ? 2 : (i == 2) ? 3 : 1;
}

__device__ __forceinline__ Pt sel4(int i, int k, Pt P, Pt V) { return i == k ? P : V; }

// ------------------------------------------------------------------ walk (Section 2.1)
__device__ __forceinline__ const PtF& self4(int i, int k, const PtF& P, const PtF& V) { return i == k ? P : V; }

__device__ __forceinline__ bool same_f(const PtF& a, const PtF& b) {
  return a.hx == b.hx && a.hy == b.hy && a.hz == b.hz && a.lx == b.lx && a.ly == b.ly && a.lz == b.lz;
}

__device__ __forceinline__ Pt self4d(int i, int k, const Pt& P, const Pt& V) { return i == k ? P : V; }

// orient3d of tetrahedron vertices v[] with vertex i replaced by the query p (FP32 stage first).
// v must be a finite tetrahedron: all four of its vertices are read on the FP64 path.
// exact = false stops after the filters (FP32, then FP64) and returns 0 when they cannot decide.
__device__ __forceinline__ int orient_replace(const Ctx& c, const uint4& v, int i, uint32_t p, const PtF& FP,
                                              const PtF& F0, const PtF& F1, const PtF& F2, const PtF& F3,
                                              bool exact = true) {
  int o = orient3d_f(self4(i, 0, FP, F0), self4(i, 1, FP, F1), self4(i, 2, FP, F2), self4(i, 3, FP, F3), c.eta);
  if (o != 0) return o;
  Pt P = load_pt(c.pts, p);
  Pt V0 = load_pt(c.pts, v.x), V1 = load_pt(c.pts, v.y), V2 = load_pt(c.pts, v.z), V3 = load_pt(c.pts, v.w);
  const Pt A = self4d(i, 0, P, V0), B = self4d(i, 1, P, V1), C = self4d(i, 2, P, V2), D = self4d(i, 3, P, V3);
  return exact ? orient3d(A, B, C, D, c.st) : orient3d_filter(A, B, C, D);
}

// Returns kCandLocated (*t_out in conflict with p), kCandWalkLimit (*t_out = where it stopped)
// or kCandDup (p equals a vertex of the tetrahedron reached).
static __device__ int walk_point(const Ctx& c, uint32_t p, const PtF& FP, uint32_t start, uint32_t salt, uint32_t anchor,
                          uint32_t max_steps, uint32_t* t_out, uint32_t* steps_out) {
  uint32_t t = start;
  Tet T;
  int hops = 0;
  for (;;) {
    if (t == kNone || t >= c.ntets) t = anchor;
    T = tet_at(c, t);
    if (!tet_dead(T.v)) break;
    t = (++hops > 64) ? anchor : T.n.x;  // dead slot: follow the redirect it keeps
    if (t != kNone && t >= c.ntets) t = anchor;
    if (hops > 66) {
      raise_error(c.st, kErrWalk, t);
      *t_out = anchor;
      *steps_out = 0;
      return kCandWalkLimit;
    }
  }
  if (!tet_sane(c, T)) {
    raise_error(c.st, kErrInternal, 0xA000u);
    *t_out = anchor;
    *steps_out = 0;
    return kCandWalkLimit;
  }
  int g = ghost_pos(T.v);
  if (g >= 0) {  // a ghost start steps into its real neighbour (Section 2.6)
    t = get4(T.n, g);
    T = tet_at(c, t);
    if (!tet_sane(c, T)) {
      raise_error(c.st, kErrInternal, 0xA001u);
      *t_out = anchor;
      *steps_out = 0;
      return kCandWalkLimit;
    }
  }
  uint32_t prev = kNone;
  uint32_t steps = 0;
  for (;;) {
    if (ghost_pos(T.v) >= 0) break;  // entered a ghost through a facet that sees p
    PtF F0 = load_ptf(c.ptf, T.v.x), F1 = load_ptf(c.ptf, T.v.y), F2 = load_ptf(c.ptf, T.v.z),
        F3 = load_ptf(c.ptf, T.v.w);
    int exit = -1;
    int s0 = (salt + steps) & 3;
    // the filters first: any facet p certainly sees is a valid exit, so the exact sign of a
    // facet the filters cannot decide (p on or near its plane: lattices, surfaces) is needed
    // only when no other facet is certainly seen
    unsigned undecided = 0;
    for (int k = 0; k < 4; ++k) {
      int i = (s0 + k) & 3;
      uint32_t nb = get4(T.n, i);
      if (nb == prev) continue;  // p is on this tetrahedron's side of the facet just crossed
      const int o = orient_replace(c, T.v, i, p, FP, F0, F1, F2, F3, false);
      if (o < 0) {
        exit = i;
        break;
      }
      if (o == 0) undecided |= 1u << k;
    }
    for (int k = 0; k < 4 && exit < 0 && undecided; ++k) {
      if (!(undecided & (1u << k))) continue;
      const int i = (s0 + k) & 3;
      if (orient_replace(c, T.v, i, p, FP, F0, F1, F2, F3) < 0) exit = i;
    }
    if (exit < 0) {
      bool dup = false;
      if (same_f(F0, FP) || same_f(F1, FP) || same_f(F2, FP) || same_f(F3, FP)) {
        Pt P = load_pt(c.pts, p);
        for (int k = 0; k < 4; ++k) {
          Pt V = load_pt(c.pts, get4(T.v, k));
          dup = dup || (V.x == P.x && V.y == P.y && V.z == P.z);
        }
      }
      *t_out = t;
      *steps_out = steps;
      return dup ? kCandDup : kCandLocated;
    }
    if (steps >= max_steps) {
      *t_out = t;
      *steps_out = steps;
      return kCandWalkLimit;
    }
    prev = t;
    t = get4(T.n, exit);
    T = tet_at(c, t);
    ++steps;
    if (!tet_sane(c, T) || tet_dead(T.v)) {
      raise_error(c.st, kErrInternal, 0xA002u);
      *t_out = anchor;
      *steps_out = steps;
      return kCandWalkLimit;
    }
  }
  *t_out = t;
  *steps_out = steps;
  return kCandLocated;
}

// ------------------------------------------------------------------ conflict test
// Perturbed insphere of a finite tetrahedron and p: negative = p inside (FP32 stage first).
// FP64 (then exact, then perturbed) insphere, out of line: the FP32 stage settles nearly every
// test, and keeping this path out of the callers keeps their registers for the common case.
static __device__ __noinline__ bool inside_finite_fp64(const Ctx& c, uint4 v, uint32_t p) {
  Pt a = load_pt(c.pts, v.x), b = load_pt(c.pts, v.y), d = load_pt(c.pts, v.z), e = load_pt(c.pts, v.w);
  return insphere_sos(a, b, d, e, load_pt(c.pts, p), c.st) < 0;
}

__device__ __forceinline__ bool inside_finite(const Ctx& c, const uint4& v, uint32_t p, const PtF& FP) {
  PtF A = load_ptf(c.ptf, v.x), B = load_ptf(c.ptf, v.y), C = load_ptf(c.ptf, v.z), D = load_ptf(c.ptf, v.w);
  int s = insphere_f(A, B, C, D, FP, c.eta);
  if (s != 0) return s < 0;
  return inside_finite_fp64(c, v, p);
}

// Membership of tetrahedron u in the cavity of p: perturbed insphere for a finite tetrahedron;
// for a ghost, p strictly beyond its hull facet, or on the facet's plane and inside the
// perturbed sphere of the finite neighbour across it (Section 2.6).
static __device__ bool in_conflict(const Ctx& c, uint32_t u, uint32_t p, const PtF& FP) {
  Tet U = tet_at(c, u);
  if (!tet_sane(c, U) || tet_dead(U.v)) {
    raise_error(c.st, kErrInternal, 0xB000u);
    return false;
  }
  int g = ghost_pos(U.v);
  if (g < 0) return inside_finite(c, U.v, p, FP);
  PtF q[4];
  for (int k = 0; k < 4; ++k) q[k] = (k == g) ? FP : load_ptf(c.ptf, get4(U.v, k));
  int o = orient3d_f(q[0], q[1], q[2], q[3], c.eta);
  if (o == 0) {  // the ghost vertex has no coordinates: only p and the hull facet are read
    Pt r[4];
    for (int k = 0; k < 4; ++k) r[k] = load_pt(c.pts, k == g ? p : get4(U.v, k));
    o = orient3d(r[0], r[1], r[2], r[3], c.st);
  }
  if (o != 0) return o > 0;
  uint32_t rr = get4(U.n, g);
  Tet R = tet_at(c, rr);
  if (!tet_sane(c, R) || ghost_pos(R.v) >= 0) {
    raise_error(c.st, kErrInternal, 0xB001u);
    return false;
  }
  return inside_finite(c, R.v, p, FP);
}

// ------------------------------------------------------------------ visited set
__device__ __forceinline__ uint32_t hash32(uint32_t k) { return k * 0x9E3779B1u; }

// Workspace arrays may live in global memory, where another lane's atomic or store is not
// seen through this SM's L1: lanes read each other's entries with volatile loads.
template <class T>
__device__ __forceinline__ T vld(const T* p) {
  return *reinterpret_cast<const volatile T*>(p);
}

__device__ __forceinline__ int ws_find(const CavWS& w, uint32_t key) {
  uint32_t h = (hash32(key) >> 8) & w.hmask;
  for (uint32_t probe = 0; probe <= w.hmask; ++probe) {
    uint32_t k = vld(&w.hkey[h]);
    if (k == key) return vld(&w.hval[h]);
    if (k == kNone) return 0;
    h = (h + 1) & w.hmask;
  }
  return 0;
}

__device__ __forceinline__ bool ws_insert(const CavWS& w, uint32_t key, uint8_t val) {
  uint32_t h = (hash32(key) >> 8) & w.hmask;
  for (uint32_t probe = 0; probe <= w.hmask; ++probe) {
    uint32_t old = atomicCAS(&w.hkey[h], kNone, key);
    if (old == kNone || old == key) {
      w.hval[h] = val;
      return true;
    }
    h = (h + 1) & w.hmask;
  }
  return false;
}

// ------------------------------------------------------------------ cavity (warp)
// Returns kCandLocated (C in w.clist[0..nc), boundary facets in w.blist[0..nb)), kCandLost
// (saw a higher-priority claim) or kCandBig (exceeds this workspace).
static __device__ int cavity_warp(const Ctx& c, const CavWS& w, uint32_t t0, uint32_t p, const PtF& FP,
                           unsigned long long prio, int* nc_out, int* nb_out) {
  const int lane = threadIdx.x & 31;
  for (uint32_t i = lane; i <= w.hmask; i += 32) w.hkey[i] = kNone;
  __syncwarp();
  int flag = 0;  // 1 lost, 2 big, 4 internal
  if (lane == 0) {
    if (!in_conflict(c, t0, p, FP)) flag |= 4;
    w.clist[0] = t0;
    ws_insert(w, t0, 1);
    if (atomicMax(&c.claim[2 * (size_t)t0], prio) > prio) flag |= 1;
    atomicMax(&c.claim[2 * (size_t)t0 + 1], prio);
  }
  flag = __shfl_sync(kFull, flag, 0);
  if (flag & 4) {
    if (lane == 0) raise_error(c.st, kErrInternal, t0);
    return kCandLost;
  }
  __syncwarp();
  int nc = 1, nb = 0, head = 0;
  while (head < nc && flag == 0) {
    int batch = min(8, nc - head);
    int k = lane >> 2, f = lane & 3;
    bool active = k < batch;
    const int ci = head + k;
    uint32_t t = 0, u = kNone;
    if (active) {
      t = vld(&w.clist[ci]);
      u = nbr_at(c, t, f);
      if (u >= c.ntets) {
        raise_error(c.st, kErrInternal, 0xC000u);
        u = t;
      }
    }
    head += batch;
    int known = active ? ws_find(w, u) : 0;
    bool need = active && known == 0;
    unsigned peers = __match_any_sync(kFull, need ? u : 0xFFFFFFFFu);
    int leader = __ffs(peers) - 1;
    bool is_leader = need && lane == leader;
    int res = 0, myflag = 0;
    if (is_leader) {
      res = in_conflict(c, u, p, FP) ? 1 : 2;
      unsigned long long oldx = atomicMax(&c.claim[2 * (size_t)u], prio);
      if (res == 1) {
        if (oldx > prio) myflag |= 1;  // a higher priority deletes or touches a tetrahedron of C
        atomicMax(&c.claim[2 * (size_t)u + 1], prio);
      } else if (__ldcg(&c.claim[2 * (size_t)u + 1]) > prio) {
        myflag |= 1;  // a higher priority deletes this outside tetrahedron
      }
      if (!ws_insert(w, u, (uint8_t)res)) myflag |= 2;
    }
    int lres = __shfl_sync(kFull, res, leader);
    if (need) res = lres;
    else res = known;
    bool addC = is_leader && res == 1;
    unsigned mC = __ballot_sync(kFull, addC);
    if (addC) {
      int pos = nc + __popc(mC & lanemask_lt());
      if (pos < (int)w.cmax) w.clist[pos] = u;
    }
    nc += __popc(mC);
    bool addB = active && res == 2;
    unsigned mB = __ballot_sync(kFull, addB);
    if (addB) {
      int pos = nb + __popc(mB & lanemask_lt());
      if (pos < (int)w.bmax) w.blist[pos] = 4u * (uint32_t)ci + (uint32_t)f;
    }
    nb += __popc(mB);
    flag = __reduce_or_sync(kFull, myflag);
    if (nc > (int)w.cmax || nb > (int)w.bmax) flag |= 2;
    if (__ldcg(&c.st->error) != 0u) flag |= 1;  // stop on any raised error
    __syncwarp();
  }
  *nc_out = nc;
  *nb_out = nb;
  if (flag & 1) return kCandLost;
  if (flag & 2) return kCandBig;
  return kCandLocated;
}

// ------------------------------------------------------------------ slot allocation
// Virtual slot v of this round: the free list (top first), then the bump pointer.
__device__ __forceinline__ uint32_t virtual_slot(const Ctx& c, unsigned long long v,
                                                 unsigned long long fa, unsigned long long bump,
                                                 unsigned long long cap, bool& fail) {
  if (v < fa) return c.freelist[fa - 1 - v];
  unsigned long long b = bump + (v - fa);
  if (b >= cap) {
    fail = true;
    return kNone;
  }
  return (uint32_t)b;
}

// Empty slot of the vertex hash: never a vertex id (the ghost vertex is kGhost = kNone).
constexpr uint32_t kNoVertex = kDeadMark;

__device__ __forceinline__ int vslot(uint32_t* vkey, uint32_t x) {
  uint32_t h = hash32(x) >> 27;
#pragma unroll 1
  for (int probe = 0; probe < 32; ++probe) {
    uint32_t old = atomicCAS(&vkey[h], kNoVertex, x);
    if (old == kNoVertex || old == x) return (int)h;
    h = (h + 1) & 31u;
  }
  return -1;
}

__device__ __forceinline__ uint32_t edge_slot(const InsWS& w, unsigned long long key) {
  uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & w.emask;
  for (uint32_t probe = 0; probe <= w.emask; ++probe) {
    unsigned long long old = atomicCAS(&w.ekey[h], ~0ull, key);
    if (old == ~0ull || old == key) return h;
    h = (h + 1) & w.emask;
  }
  return kNone;
}

// ------------------------------------------------------------------ ball (warp)
// Verifies the claims of a located point and, if it won, replaces its cavity by the ball.
// Returns kCandInserted or kCandLost. alloc: allocator snapshot of this round.
static __device__ int insert_warp(const Ctx& c, const InsWS& w, uint32_t p, unsigned long long prio,
                           const uint32_t* clist, int nc, const uint32_t* blist, int nb,
                           bool use_table, unsigned long long fa, unsigned long long bump,
                           unsigned long long cap) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int i = lane; i < nc; i += 32)
    if (__ldcg(&c.claim[2 * (size_t)vld(&clist[i])]) != prio) ok = false;
  if (!__all_sync(kFull, ok)) return kCandLost;
  for (int i = lane; i < nb; i += 32) {
    uint32_t e = vld(&blist[i]);
    uint32_t t = vld(&clist[e >> 2]);
    int f = (int)(e & 3u);
    Tet T = load_tet_cg(c.tets, t);
    uint32_t out = get4(T.n, f);
    if (out >= c.ntets || !tet_sane(c, T)) {
      raise_error(c.st, kErrInternal, 0xD000u);
      ok = false;
      out = 0;
    }
    if (__ldcg(&c.claim[2 * (size_t)out + 1]) >= prio) ok = false;
    // the facet of the outside tetrahedron that faces t (read before this warp writes anything;
    // a winner's outside tetrahedra are its own for the round)
    const int back = back_facet(__ldcg(reinterpret_cast<const uint4*>(&c.tets[out].n)), t);
    if (back < 0) ok = false;
    uint4 v = T.v;
    set4(v, f, p);
    w.nv[i] = v;
    w.outh[i] = out;
    w.ipos[i] = (uint8_t)(f | ((back & 3) << 2));
  }
  if (!__all_sync(kFull, ok)) return kCandLost;
  // slots: cavity slots first (Section 2.5), then the allocator (Section 3.6)
  int reuse = min(nc, nb), extra = nb - reuse;
  unsigned long long base = 0;
  if (lane == 0 && extra > 0) base = atomicAdd(&c.st->alloc_cursor, (unsigned long long)extra);
  base = __shfl_sync(kFull, base, 0);
  bool fail = false;
  for (int i = lane; i < nb; i += 32)
    w.slot[i] = (i < reuse) ? vld(&clist[i]) : virtual_slot(c, base + (unsigned long long)(i - reuse), fa, bump, cap, fail);
  if (__any_sync(kFull, fail)) {
    if (lane == 0) raise_error(c.st, kErrCapacity, (unsigned)nb);
    return kCandLost;
  }
  if (use_table)
    for (int i = lane; i < 32; i += 32) w.vkey[i] = kNoVertex;
  else
    for (uint32_t i = lane; i <= w.emask; i += 32) {
      w.ekey[i] = ~0ull;
      w.eval[i] = kNone;
    }
  __syncwarp();
  // record every internal facet: facet a of new tetrahedron i holds the boundary edge b -> c
  if (use_table) {
    bool vfail = false;
    for (int i = lane; i < nb; i += 32) {
      uint4 v = w.nv[i];
      int a, b, cc;
      after_pos(w.ipos[i] & 3, a, b, cc);
      int la = vslot(w.vkey, get4(v, a)), lb = vslot(w.vkey, get4(v, b)), lc = vslot(w.vkey, get4(v, cc));
      if (la < 0 || lb < 0 || lc < 0) {
        vfail = true;
        continue;
      }
      w.tab[lb * 32 + lc] = (uint16_t)((i << 2) | a);
      w.tab[lc * 32 + la] = (uint16_t)((i << 2) | b);
      w.tab[la * 32 + lb] = (uint16_t)((i << 2) | cc);
    }
    if (__any_sync(kFull, vfail)) {
      if (lane == 0) raise_error(c.st, kErrInternal, 0x7AB1u);
      return kCandLost;
    }
  } else {
    bool efail = false;
    for (int i = lane; i < nb; i += 32) {
      uint4 v = w.nv[i];
      int pos[3];
      after_pos(w.ipos[i] & 3, pos[0], pos[1], pos[2]);
      for (int k = 0; k < 3; ++k) {
        uint32_t x = get4(v, pos[(k + 1) % 3]), y = get4(v, pos[(k + 2) % 3]);
        unsigned long long key = ((unsigned long long)min(x, y) << 32) | max(x, y);
        uint32_t s = edge_slot(w, key);
        if (s == kNone) {
          efail = true;
          break;
        }
        w.hslot[3 * i + k] = s;
        w.hold[3 * i + k] = atomicExch(&w.eval[s], (uint32_t)((i << 2) | pos[k]));
      }
    }
    if (__any_sync(kFull, efail)) {
      if (lane == 0) raise_error(c.st, kErrBigCavity, (unsigned)nb);
      return kCandLost;
    }
  }
  __syncwarp();
  // partners of every internal facet; all must name a new tetrahedron before any write
  bool bad = false;
  for (int i = lane; i < nb; i += 32) {
    uint4 v = w.nv[i];
    int ip = w.ipos[i] & 3;
    int a, b, cc;
    after_pos(ip, a, b, cc);
    uint32_t ea, eb, ec;
    if (use_table) {
      int la = vslot(w.vkey, get4(v, a)), lb = vslot(w.vkey, get4(v, b)), lc = vslot(w.vkey, get4(v, cc));
      ea = vld(&w.tab[lc * 32 + lb]);
      eb = vld(&w.tab[la * 32 + lc]);
      ec = vld(&w.tab[lb * 32 + la]);
    } else {
      uint32_t hh[3];
      for (int k = 0; k < 3; ++k) {
        uint32_t old = w.hold[3 * i + k];
        hh[k] = (old != kNone) ? old : vld(&w.eval[w.hslot[3 * i + k]]);
      }
      ea = hh[0];
      eb = hh[1];
      ec = hh[2];
    }
    if ((ea >> 2) >= (uint32_t)nb || (eb >> 2) >= (uint32_t)nb || (ec >> 2) >= (uint32_t)nb ||
        (ea >> 2) == (uint32_t)i || (eb >> 2) == (uint32_t)i || (ec >> 2) == (uint32_t)i) {
      bad = true;
      continue;
    }
    uint4 nn;
    set4(nn, ip, w.outh[i]);
    set4(nn, a, vld(&w.slot[ea >> 2]));
    set4(nn, b, vld(&w.slot[eb >> 2]));
    set4(nn, cc, vld(&w.slot[ec >> 2]));
    w.nn[i] = nn;
  }
  if (__any_sync(kFull, bad)) {
    if (lane == 0) raise_error(c.st, kErrInternal, 0xE000u);
    return kCandLost;
  }
  __syncwarp();
  // write the ball
  for (int i = lane; i < nb; i += 32) {
    uint32_t s = w.slot[i];
    uint4* dst = reinterpret_cast<uint4*>(c.tets + s);
    dst[0] = w.nv[i];
    dst[1] = w.nn[i];
    uint32_t out = w.outh[i];
    reinterpret_cast<uint32_t*>(&c.tets[out].n)[w.ipos[i] >> 2] = s;
    if (c.subdet) c.subdet[2 * (size_t)s + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // cavity slots left over (|C| > |B|) die and join the free list after the round
  int freed = nc - nb;
  if (freed > 0) {
    unsigned long long pb = 0;
    if (lane == 0) pb = atomicAdd(&c.st->pending, (unsigned long long)freed);
    pb = __shfl_sync(kFull, pb, 0);
    uint32_t redirect = vld(&w.slot[0]);
    for (int i = lane; i < freed; i += 32) {
      uint32_t s = vld(&clist[nb + i]);
      uint4* dst = reinterpret_cast<uint4*>(c.tets + s);
      dst[0] = make_uint4(kDeadMark, kDeadMark, kDeadMark, kDeadMark);
      dst[1] = make_uint4(redirect, kNone, kNone, kNone);
      if (pb + i < c.st->free_capacity) c.pending[pb + i] = s;
      else raise_error(c.st, kErrFreeList, 0);
    }
    __threadfence();  // the warp that closes the round reads these entries
  }
  return kCandInserted;
}

// ------------------------------------------------------------------ global-memory workspaces
struct BigWS {
  CavWS cav;
  InsWS ins;
};

// Carves the workspaces of one candidate out of a byte range (global memory).
__host__ __device__ inline size_t carve(char* base, uint32_t hashn, uint32_t cn, uint32_t fn, uint32_t edgen,
                                        BigWS* w) {
  size_t off = 0;
  auto take = [&](size_t n) {
    char* r = base ? base + off : nullptr;
    off += (n + 15) & ~size_t(15);
    return r;
  };
  BigWS x{};
  x.ins.ekey = (unsigned long long*)take((size_t)edgen * 8);
  x.ins.nv = (uint4*)take((size_t)fn * 16);
  x.ins.nn = (uint4*)take((size_t)fn * 16);
  x.cav.hkey = (uint32_t*)take((size_t)hashn * 4);
  x.cav.clist = (uint32_t*)take((size_t)cn * 4);
  x.cav.blist = (uint32_t*)take((size_t)fn * 4);
  x.ins.eval = (uint32_t*)take((size_t)edgen * 4);
  x.ins.hslot = (uint32_t*)take((size_t)fn * 3 * 4);
  x.ins.hold = (uint32_t*)take((size_t)fn * 3 * 4);
  x.ins.outh = (uint32_t*)take((size_t)fn * 4);
  x.ins.slot = (uint32_t*)take((size_t)fn * 4);
  x.ins.vkey = (uint32_t*)take(32 * 4);
  x.ins.tab = (uint16_t*)take(32 * 32 * 2);
  x.cav.hval = (uint8_t*)take(hashn);
  x.ins.ipos = (uint8_t*)take(fn);
  x.cav.hmask = hashn - 1;
  x.cav.cmax = cn;
  x.cav.bmax = fn;
  x.ins.emask = edgen - 1;
  if (w) *w = x;
  return off;
}

// ------------------------------------------------------------------ rounds and init
// Closes a round (run by the last block of the insert kernel): the allocator consumed the top
// of the free list, then the bump pointer; slots freed during the round join the free list;
// the claim stamp advances.
static __device__ void finish_round_block(const Ctx& c) {
  DevState* st = c.st;
  unsigned long long used = __ldcg(&st->alloc_cursor), fa = __ldcg(&st->free_avail);
  unsigned long long np = __ldcg(&st->pending);
  __syncthreads();
  unsigned long long consumed = used < fa ? used : fa;
  unsigned long long nfa = fa - consumed;
  if (nfa + np > st->free_capacity) {
    if (threadIdx.x == 0) raise_error(st, kErrFreeList, 0);
    np = st->free_capacity - nfa;
  }
  for (unsigned long long i = threadIdx.x; i < np; i += blockDim.x) c.freelist[nfa + i] = __ldcg(&c.pending[i]);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->bump += used - consumed;
    st->free_avail = nfa + np;
    st->alloc_cursor = 0;
    st->pending = 0;
    st->stamp += 1;
    st->blocks_done = 0;
    __threadfence();
  }
  __syncthreads();
}

// Closes a round run by a single warp (the serial path, and the last warp of the insert kernel).
static __device__ void finish_round_warp(const Ctx& c) {
  const int lane = threadIdx.x & 31;
  DevState* st = c.st;
  unsigned long long used = __ldcg(&st->alloc_cursor), fa = __ldcg(&st->free_avail);
  unsigned long long np = __ldcg(&st->pending);
  __syncwarp();
  unsigned long long consumed = used < fa ? used : fa;
  unsigned long long nfa = fa - consumed;
  if (nfa + np > st->free_capacity) {
    if (lane == 0) raise_error(st, kErrFreeList, 0);
    np = st->free_capacity - nfa;
  }
  for (unsigned long long i = lane; i < np; i += 32) c.freelist[nfa + i] = __ldcg(&c.pending[i]);
  __syncwarp();
  if (lane == 0) {
    st->bump += used - consumed;
    st->free_avail = nfa + np;
    st->alloc_cursor = 0;
    st->pending = 0;
    st->stamp += 1;
    st->blocks_done = 0;
  }
  __threadfence();
  __syncwarp();
}

// Init (Section 2.1): the first four non-coplanar vertices of the insertion order form a
// positive tetrahedron; four ghost tetrahedra close it (Section 2.6). The five records go to
// slots tbase .. tbase + 4. Returns false (and raises kErrDegenerate) when [vbegin, vend) holds
// fewer than four non-coplanar vertices. One thread.
static __device__ bool init_mesh(const Ctx& c, uint32_t vbegin, uint32_t vend, uint8_t* vflag, uint32_t tbase) {
  uint32_t s = vbegin;
  while (s < vend && vflag[s]) ++s;
  uint32_t i0 = s++;
  while (s < vend && vflag[s]) ++s;
  uint32_t i1 = s++;
  if (i1 >= vend) {
    raise_error(c.st, kErrDegenerate, 0);
    return false;
  }
  Pt A = c.pts[i0], B = c.pts[i1];
  while (s < vend && (vflag[s] || collinear_exact(A, B, c.pts[s], c.st))) ++s;
  uint32_t i2 = s++;
  if (i2 >= vend) {
    raise_error(c.st, kErrDegenerate, 1);
    return false;
  }
  Pt C = c.pts[i2];
  while (s < vend && (vflag[s] || orient3d(A, B, C, c.pts[s], c.st) == 0)) ++s;
  uint32_t i3 = s;
  if (i3 >= vend) {
    raise_error(c.st, kErrDegenerate, 2);
    return false;
  }
  uint32_t v[4] = {i0, i1, i2, i3};
  if (orient3d(A, B, C, c.pts[i3], c.st) < 0) {
    v[2] = i3;
    v[3] = i2;
  }
  uint32_t tv[5][4];
  for (int k = 0; k < 4; ++k) tv[0][k] = v[k];
  for (int i = 0; i < 4; ++i) {
    for (int k = 0; k < 4; ++k) tv[1 + i][k] = v[k];
    tv[1 + i][i] = kGhost;
    int a = (i == 0) ? 1 : 0, b = (i <= 1) ? 2 : 1;
    uint32_t x = tv[1 + i][a];
    tv[1 + i][a] = tv[1 + i][b];
    tv[1 + i][b] = x;
  }
  uint32_t nn[5][4];
  for (int t = 0; t < 5; ++t)
    for (int f = 0; f < 4; ++f) {
      nn[t][f] = kNone;
      for (int u = 0; u < 5 && nn[t][f] == kNone; ++u) {
        if (u == t) continue;
        for (int g = 0; g < 4; ++g) {
          // facet f of t equals facet g of u when the other three vertices coincide as sets
          int match = 0;
          for (int a = 0; a < 4; ++a) {
            if (a == f) continue;
            for (int b = 0; b < 4; ++b)
              if (b != g && tv[t][a] == tv[u][b]) {
                ++match;
                break;
              }
          }
          if (match == 3) {
            nn[t][f] = tbase + u;
            break;
          }
        }
      }
    }
  for (int t = 0; t < 5; ++t) {
    c.tets[tbase + t].v = make_uint4(tv[t][0], tv[t][1], tv[t][2], tv[t][3]);
    c.tets[tbase + t].n = make_uint4(nn[t][0], nn[t][1], nn[t][2], nn[t][3]);
    if (c.subdet) c.subdet[2 * (size_t)(tbase + t) + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  vflag[i0] = vflag[i1] = vflag[i2] = vflag[i3] = 2;
  c.st->bump = tbase + 5;
  c.st->anchor = tbase;
  c.st->n_inserted += 4;
  return true;
}

// Canonical form of a positively oriented tetrahedron (vertex ids r[0..3]): the even permutation
// that brings the smallest id first, then the cyclic turn of the other three that starts at
// their smallest. Orientation is preserved.
__device__ __forceinline__ void canonical_rotation(uint32_t r[4]) {
  int k = 0;
  for (int i = 1; i < 4; ++i)
    if (r[i] < r[k]) k = i;
  uint32_t a[4];
  if (k == 0) { a[0] = r[0]; a[1] = r[1]; a[2] = r[2]; a[3] = r[3]; }
  else if (k == 1) { a[0] = r[1]; a[1] = r[0]; a[2] = r[3]; a[3] = r[2]; }
  else if (k == 2) { a[0] = r[2]; a[1] = r[0]; a[2] = r[1]; a[3] = r[3]; }
  else { a[0] = r[3]; a[1] = r[0]; a[2] = r[2]; a[3] = r[1]; }
  if (a[2] < a[1] && a[2] < a[3]) { uint32_t x = a[1]; a[1] = a[2]; a[2] = a[3]; a[3] = x; }
  else if (a[3] < a[1] && a[3] < a[2]) { uint32_t x = a[3]; a[3] = a[2]; a[2] = a[1]; a[1] = x; }
  for (int i = 0; i < 4; ++i) r[i] = a[i];
}

}  // namespace dtg
