// Asynchronous concurrent insertion: one persistent launch per wave, no rounds.
//
// The paper's threads (Section 3.2) each own a Moore-curve partition of the points and insert
// them one after the other; a thread that would touch a tetrahedron another thread holds aborts
// the insertion and retries it later. Here every warp is such a thread: warp w takes the w-th
// contiguous segment of the wave's Moore order and inserts its points in that order, each walk
// starting from the warp's previous ball (Algorithm 1). Ownership is a 32-bit word per
// tetrahedron slot (0 = free, else the owning warp). One insertion:
//   1. walk (Section 2.1) from the previous ball, reading the mesh without locks;
//   2. cavity search (Section 2.1, Eq. 1) on those unlocked reads: the cavity C, its outside
//      neighbours A and the boundary facets, with every record kept in shared memory;
//   3. lock C, A and the slots the ball needs beyond C (Section 2.5 reuses C's slots first),
//      one compare-and-swap each; any slot held by another warp aborts the insertion (rule
//      (1) of Section 3.2: a thread touches only tetrahedra it owns);
//   4. re-read C (whole records) and A (vertices) under the locks: a difference means another
//      warp changed them between steps 2 and 3, and the insertion starts over from the walk;
//      also read which facet of each tetrahedron of A faces the cavity (neighbour slots hold
//      plain tetrahedron ids: it is the facet whose neighbour is the cavity tetrahedron);
//   5. write the ball (Section 2.5: one tetrahedron per boundary facet, adjacency through the
//      edge table), the back-pointers of A, then release every lock after a fence.
// Aborted points wait in a small per-warp list and are retried after later insertions; what is
// still left when the segment ends goes to the next pass. A cavity larger than the per-warp
// shared-memory workspace is inserted again in a global-memory workspace borrowed from a pool,
// else by a separate large-cavity launch; a predicate the FP32 stage cannot decide hands the
// point to the round-based engine. No warp ever waits on another, so every loop here is
// bounded by the segment length and fixed retry counts.
//
// The triangulation does not depend on the order of insertions (exact predicates and one
// symbolic perturbation, Section 2.4), so this engine gives the same tetrahedra as the
// round-based one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"
#include "predicates.cuh"

namespace dtg {
namespace {

constexpr int kAW = 4;            // warps per block of the shared-memory kernel
constexpr int kADefer = 16;       // aborted points waiting for a retry
constexpr int kARetry = 3;        // immediate restarts after a failed re-read
constexpr uint32_t kAChunk = 32;  // slots taken from the allocator at a time

enum AStatus : int { kAInserted = 0, kALost = 1, kARestart = 2, kABig = 3, kAWalkLimit = 4, kADup = 5, kAExact = 6 };

// Ball adjacency (Section 2.5): the n x n edge table for balls of at most 32 boundary vertices
// (the shared-memory workspaces), an edge hash for larger ones (the global-memory workspaces).
template <bool kTable, int kHashN, int kFMaxN>
struct AWSTail;
template <int kHashN, int kFMaxN>
struct AWSTail<true, kHashN, kFMaxN> {
  // the visited set is needed only while the cavity is searched, the edge table only while the
  // ball is built: they share their bytes
  union {
    struct {
      uint32_t hkey[kHashN];
      uint8_t hval[kHashN];
    };
    uint16_t tab[32 * 32];
  };
};
template <int kHashN, int kFMaxN>
struct AWSTail<false, kHashN, kFMaxN> {
  static constexpr uint32_t kEdgeN = 4096;
  uint32_t hkey[kHashN];
  uint8_t hval[kHashN];
  unsigned long long ekey[kEdgeN];
  uint32_t eval[kEdgeN];
  uint32_t hslot[3 * kFMaxN];
  uint32_t hold[3 * kFMaxN];
};

// Working storage of one warp: the cavity's tetrahedra with their records as read, the outside
// tetrahedra with their vertices as read, the boundary facets, the ball's slots, a private pool
// of free slots, deferred points, and the warp's state (uniform across its lanes, written by
// lane 0). Held: the type of a lane's lock mask (one bit per lock-list entry of the lane).
template <int kHashN, int kCMaxN, int kAMaxN, int kFMaxN, bool kTableB, class HeldT, bool kCacheB>
struct AWS : AWSTail<kTableB, kHashN, kFMaxN> {
  static constexpr int kHash = kHashN, kCMax = kCMaxN, kAMax = kAMaxN, kFMax = kFMaxN;
  static constexpr bool kCache = kCacheB;  // conflict tests through the sub-determinant cache
  static constexpr int kPool = kFMaxN + 36;  // a refill of 32 slots always fits below kFMax
  static constexpr bool kTable = kTableB;
  using Held = HeldT;
  using CI = typename std::conditional<(kCMaxN > 255), uint16_t, uint8_t>::type;
  static_assert(kCMaxN + kAMaxN + kFMaxN <= 32 * 8 * (int)sizeof(HeldT), "lock mask holds every entry");
  uint32_t cl[kCMaxN];       // cavity slots
  Tet cr[kCMaxN];            // their records as read
  uint32_t al[kAMaxN];       // outside slots
  uint4 av[kAMaxN];          // their vertex ids as read
  uint32_t slot[kFMaxN];     // slots of the new tetrahedra
  uint32_t ex[kFMaxN];       // slots beyond the cavity's, taken from the pool
  uint32_t vkey[32];
  uint32_t pool[kPool];
  uint32_t defer[kADefer];
  CI bl_ci[kFMaxN];          // boundary facet: cavity index
  uint8_t bl_f[kFMaxN];      // boundary facet: facet | 4 * the outside tetrahedron's facet
  unsigned long long fa, bump;  // allocator snapshot of the launch
  unsigned int cnt[8];          // inserted, lost, attempts, sum |C|, sum |B|, walk steps, restarts
  uint32_t hint;                // the warp's last ball
  int bn;                       // tetrahedra of the warp's last ball (0: none); slots in slot[]
  int np;                       // slots in the pool
  int nc, na, nb;               // cavity, outside and boundary-facet counts of the last search
};

// Shared-memory workspace of the main kernel (cavities of up to 64 tetrahedra and 60 boundary
// facets) and the global-memory one of the large-cavity kernel.
template <bool kCache>
using SmallWST = AWS<256, 64, 64, 60, true, unsigned, kCache>;
template <bool kCache>
using LargeWST = AWS<4096, 640, 704, 704, false, unsigned long long, kCache>;
using LargeWS = LargeWST<false>;  // the same layout with and without the cache

__device__ __forceinline__ Tet ld_tet(const Tet* T, uint32_t t) { return load_tet_cg(T, t); }

__device__ __forceinline__ bool same_tet(const Tet& a, const Tet& b) {
  return a.v.x == b.v.x && a.v.y == b.v.y && a.v.z == b.v.z && a.v.w == b.v.w && a.n.x == b.n.x &&
         a.n.y == b.n.y && a.n.z == b.n.z && a.n.w == b.n.w;
}

__device__ __forceinline__ bool same_v(const uint4& a, const uint4& b) {
  return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w;
}

// A record that references only allocated vertices and slots (a record being rewritten may be
// read half old, half new; such a read is never followed).
__device__ __forceinline__ bool rec_ok(const Tet& T, uint32_t ntets, uint32_t npts) {
  bool ok = true;
  for (int k = 0; k < 4; ++k) {
    uint32_t v = get4(T.v, k), n = get4(T.n, k);
    ok = ok && (v == kGhost || v < npts) && n < ntets;
  }
  return ok;
}

// The predicates' FP32 stage on the double-float point copy (predicates.cuh: rigorous error
// bounds, Section 2.4's filters moved to FP32). When it cannot decide, the insertion is handed to
// the round-based engine, which runs the whole cascade (FP64 filter, exact arithmetic, symbolic
// perturbation): keeping the exact stages out of this kernel keeps its registers free of the
// save and restore traffic their calls would cost. A return of 0 means "undecided".

__device__ __forceinline__ PtF pick(bool c, const PtF& x, const PtF& y) {
  PtF r;
  r.hx = c ? x.hx : y.hx; r.hy = c ? x.hy : y.hy; r.hz = c ? x.hz : y.hz; r.hw = 0.f;
  r.lx = c ? x.lx : y.lx; r.ly = c ? x.ly : y.ly; r.lz = c ? x.lz : y.lz; r.lw = 0.f;
  return r;
}

// orient3d of (v0, v1, v2, v3) with vertex i replaced by p. Moving p to the last place is an
// odd permutation for i = 0, 2 and an even one for i = 1, 3, so one FP32 evaluation on the other
// three vertices in their order serves every i (one copy of the code: the kernel's instruction
// footprint decides how often its warps wait for instructions).
__device__ __forceinline__ int orient_with_p(const Ctx& c, int i, const PtF& FP, const PtF& F0, const PtF& F1,
                                             const PtF& F2, const PtF& F3) {
  const PtF A = pick(i == 0, F1, F0), B = pick(i <= 1, F2, F1), C = pick(i <= 2, F3, F2);
  const int o = orient3d_f(A, B, C, FP, c.eta);
  return (i & 1) ? o : -o;
}

// Insphere of a finite tetrahedron v and p: -1 inside, 1 outside, 0 undecided.
__device__ __forceinline__ int inside_async(const Ctx& c, const uint4& v, const PtF& FP) {
  PtF A = load_ptf(c.ptf, v.x), B = load_ptf(c.ptf, v.y), C = load_ptf(c.ptf, v.z), D = load_ptf(c.ptf, v.w);
  return insphere_f(A, B, C, D, FP, c.eta);
}

// Sub-determinant cache (Section 2.4; an ablation, off unless the handle allocates it). With
// b, c, d, e the differences of the tetrahedron's other vertices and of p from its first vertex
// a, the insphere determinant expanded along e's row is ex Ax + ey Ay + ez Az + |e|^2 AL, and
// the cofactors A depend on the tetrahedron alone. Two float4 per slot: q0 = (Ax, Ay, Az, AL);
// q1 = (the permanents of Ax and Ay, then of Az and AL, each pair as two bfloat16 rounded up;
// the largest |coordinate| of b, c, d; 1 when the entry is valid). The same monomials as
// insphere_f's with fewer roundings on each (12 against 16), so insphere_f's bound holds;
// rounding the permanents up widens it by at most 2^-7 of itself.
__device__ __forceinline__ uint32_t bf16_up(float x) {  // x >= 0: the bfloat16 at or above x
  return (__float_as_uint(x) + 0xFFFFu) >> 16;
}
__device__ __forceinline__ float bf16_lo(float packed) { return __uint_as_float(__float_as_uint(packed) << 16); }
__device__ __forceinline__ float bf16_hi(float packed) {
  return __uint_as_float(__float_as_uint(packed) & 0xFFFF0000u);
}

__device__ __forceinline__ void subdet_make(const PtF& A, const PtF& B, const PtF& C, const PtF& D, float4& q0,
                                            float4& q1) {
  float bx, by, bz, cx, cy, cz, dx, dy, dz;
  diff_f(B, A, bx, by, bz);
  diff_f(C, A, cx, cy, cz);
  diff_f(D, A, dx, dy, dz);
  const float Lb = bx * bx + by * by + bz * bz, Lc = cx * cx + cy * cy + cz * cz, Ld = dx * dx + dy * dy + dz * dz;
  const float cd0 = cy * dz - cz * dy, cd1 = cx * dz - cz * dx, cd2 = cx * dy - cy * dx;
  const float bd0 = by * dz - bz * dy, bd1 = bx * dz - bz * dx, bd2 = bx * dy - by * dx;
  const float bc0 = by * cz - bz * cy, bc1 = bx * cz - bz * cx, bc2 = bx * cy - by * cx;
  const float pcd0 = fabsf(cy * dz) + fabsf(cz * dy), pcd1 = fabsf(cx * dz) + fabsf(cz * dx),
              pcd2 = fabsf(cx * dy) + fabsf(cy * dx);
  const float pbd0 = fabsf(by * dz) + fabsf(bz * dy), pbd1 = fabsf(bx * dz) + fabsf(bz * dx),
              pbd2 = fabsf(bx * dy) + fabsf(by * dx);
  const float pbc0 = fabsf(by * cz) + fabsf(bz * cy), pbc1 = fabsf(bx * cz) + fabsf(bz * cx),
              pbc2 = fabsf(bx * cy) + fabsf(by * cx);
  q0.x = Lc * bd0 - Lb * cd0 - Ld * bc0;
  q0.y = Lb * cd1 + Ld * bc1 - Lc * bd1;
  q0.z = Lc * bd2 - Lb * cd2 - Ld * bc2;
  q0.w = bx * cd0 - by * cd1 + bz * cd2;
  const float px = Lc * pbd0 + Lb * pcd0 + Ld * pbc0, py = Lc * pbd1 + Lb * pcd1 + Ld * pbc1,
              pz = Lc * pbd2 + Lb * pcd2 + Ld * pbc2;
  const float pl = fabsf(bx) * pcd0 + fabsf(by) * pcd1 + fabsf(bz) * pcd2;
  q1.x = __uint_as_float(bf16_up(px) | (bf16_up(py) << 16));
  q1.y = __uint_as_float(bf16_up(pz) | (bf16_up(pl) << 16));
  q1.z = fmaxf(fmaxf(fmaxf(fabsf(bx), fabsf(by)), fmaxf(fabsf(bz), fabsf(cx))),
               fmaxf(fmaxf(fabsf(cy), fabsf(cz)), fmaxf(fmaxf(fabsf(dx), fabsf(dy)), fabsf(dz))));
  q1.w = 1.f;
}

// insphere_f of the cached tetrahedron (first vertex A) and p: -1 inside, 1 outside, 0 undecided.
__device__ __forceinline__ int insphere_cached(const float4& q0, const float4& q1, const PtF& A, const PtF& FP,
                                               float eta) {
  float ex, ey, ez;
  diff_f(FP, A, ex, ey, ez);
  const float Le = ex * ex + ey * ey + ez * ez;
  const float det = (ex * q0.x + ey * q0.y) + (ez * q0.z + Le * q0.w);
  const float perm = (fabsf(ex) * bf16_lo(q1.x) + fabsf(ey) * bf16_hi(q1.x)) +
                     (fabsf(ez) * bf16_lo(q1.y) + Le * bf16_hi(q1.y));
  const float mm = fmaxf(q1.z, fmaxf(fabsf(ex), fmaxf(fabsf(ey), fabsf(ez)))) + eta, mm2 = mm * mm;
  const float eb = kInsphereCf * perm + 400.0f * eta * (mm2 * mm2);
  if (!(perm > 1e-30f && perm < 1e30f)) return 0;
  return det > eb ? 1 : (det < -eb ? -1 : 0);
}

// The conflict test of a finite tetrahedron u (vertices v) through the cache when its entry
// is valid, else from the coordinates.
__device__ __forceinline__ int inside_maybe_cached(const Ctx& c, uint32_t u, const uint4& v, const PtF& FP) {
  const float4 q1 = __ldcg(c.subdet + 2 * (size_t)u + 1);
  if (q1.w == 0.f) return inside_async(c, v, FP);
  const float4 q0 = __ldcg(c.subdet + 2 * (size_t)u);
  return insphere_cached(q0, q1, load_ptf(c.ptf, v.x), FP, c.eta);
}

// Visibility walk (Section 2.1, ghost rules of Section 2.6) on unlocked reads. Lanes 0-3 test
// the four facets of the current tetrahedron at once (lane i: p against the facet opposite
// vertex i), and the walk leaves through the first facet p sees, in an order that turns with
// the steps. A record that is being rewritten may be read half old, half new: such reads end
// the walk with kARestart (or it runs into its step bound); nothing is trusted before step 4
// re-reads it under a lock. Called by the whole warp; the result is uniform.
__device__ __forceinline__ int walk_async(const Ctx& c, uint32_t p, const PtF& FP, uint32_t start, uint32_t salt,
                                          uint32_t max_steps, uint32_t* t_out, uint32_t* steps_out) {
  const int lane = threadIdx.x & 31;
  uint32_t t = start;
  Tet T;
  *steps_out = 0;
  *t_out = kNone;
  int hops = 0;
  for (;;) {
    if (t == kNone || t >= c.ntets) t = __ldcg(&c.st->anchor);
    if (t >= c.ntets) return kARestart;
    T = ld_tet(c.tets, t);
    if (!tet_dead(T.v)) break;
    t = T.n.x;  // dead slot: follow its redirect
    if (++hops > 64) return kARestart;
  }
  if (!rec_ok(T, c.ntets, c.npts)) return kARestart;
  int g = ghost_pos(T.v);
  if (g >= 0) {
    t = get4(T.n, g);
    T = ld_tet(c.tets, t);
    if (tet_dead(T.v) || !rec_ok(T, c.ntets, c.npts)) return kARestart;
  }
  uint32_t prev = kNone, steps = 0;
  for (;;) {
    if (ghost_pos(T.v) >= 0) break;
    // lane i < 4: orientation of p against the facet opposite vertex i (0: undecided)
    int o = 1;
    if (lane < 4) {
      const PtF F0 = load_ptf(c.ptf, T.v.x), F1 = load_ptf(c.ptf, T.v.y), F2 = load_ptf(c.ptf, T.v.z),
                F3 = load_ptf(c.ptf, T.v.w);
      o = get4(T.n, lane) == prev ? 1 : orient_with_p(c, lane, FP, F0, F1, F2, F3);
    }
    const unsigned sees = __ballot_sync(kFull, lane < 4 && o < 0) & 0xFu;
    // a facet the FP32 stage cannot decide matters only when no other facet is certainly seen:
    // any facet p sees is a valid exit of the visibility walk
    if (sees == 0 && (__ballot_sync(kFull, lane < 4 && o == 0) & 0xFu)) return kAExact;
    if (sees == 0) {
      // p is inside (or on) this tetrahedron: a vertex equal to p would be a duplicate
      bool dup = false;
      if (lane < 4) {
        const PtF V = load_ptf(c.ptf, get4(T.v, lane));
        if (same_f(V, FP)) {
          const Pt P = load_pt(c.pts, p), Q = load_pt(c.pts, get4(T.v, lane));
          dup = Q.x == P.x && Q.y == P.y && Q.z == P.z;
        }
      }
      *t_out = t;
      *steps_out = steps;
      return __any_sync(kFull, dup) ? kADup : kAInserted;
    }
    if (steps >= max_steps) {
      *t_out = t;
      *steps_out = steps;
      return kAWalkLimit;
    }
    // the first facet p sees, starting from a position that turns with the steps
    const unsigned rot = ((sees | (sees << 4)) >> ((salt + steps) & 3)) & 0xFu;
    const int exit = (__ffs(rot) - 1 + (int)((salt + steps) & 3)) & 3;
    prev = t;
    t = get4(T.n, exit);
    T = ld_tet(c.tets, t);
    ++steps;
    if (tet_dead(T.v) || !rec_ok(T, c.ntets, c.npts)) {
      *t_out = t;
      *steps_out = steps;
      return kARestart;
    }
  }
  *t_out = t;
  *steps_out = steps;
  return kAInserted;
}

// Conflict of a record U (already read) with p: 1 in the cavity, 0 outside, -2 undecided by the
// FP32 stage. For a ghost whose hull facet's plane holds p the finite neighbour across the facet
// decides (Section 2.6): that case is left to the round-based engine (-2).
template <bool kCache>
__device__ __forceinline__ int conflict_async(const Ctx& c, uint32_t u, const Tet& U, const PtF& FP) {
  const int g = ghost_pos(U.v);
  if (g < 0) {
    const int s = kCache ? inside_maybe_cached(c, u, U.v, FP) : inside_async(c, U.v, FP);
    return s < 0 ? 1 : (s > 0 ? 0 : -2);
  }
  // orientation of the hull facet's three vertices and p in the ghost's place
  const uint32_t a = g == 0 ? U.v.y : U.v.x, b = g <= 1 ? U.v.z : U.v.y, d = g <= 2 ? U.v.w : U.v.z;
  int o = orient3d_f(load_ptf(c.ptf, a), load_ptf(c.ptf, b), load_ptf(c.ptf, d), FP, c.eta);
  o = (g & 1) ? o : -o;
  if (o != 0) return o > 0 ? 1 : 0;
  // p on the facet's plane as far as the FP32 stage can tell: the exact rule needs the
  // round-based engine (the plane test and the neighbour's perturbed sphere)
  return -2;
}

template <class W>
__device__ __forceinline__ int hfind(const W& w, uint32_t key) {
  uint32_t h = (hash32(key) >> 8) & (W::kHash - 1);
#pragma unroll 1
  for (int probe = 0; probe < W::kHash; ++probe) {
    uint32_t k = vld(&w.hkey[h]);
    if (k == key) return vld(&w.hval[h]);
    if (k == kNone) return 0;
    h = (h + 1) & (W::kHash - 1);
  }
  return 0;
}

template <class W>
__device__ __forceinline__ bool hinsert(W& w, uint32_t key, uint8_t val) {
  uint32_t h = (hash32(key) >> 8) & (W::kHash - 1);
#pragma unroll 1
  for (int probe = 0; probe < W::kHash; ++probe) {
    uint32_t old = atomicCAS(&w.hkey[h], kNone, key);
    if (old == kNone || old == key) {
      w.hval[h] = val;
      return true;
    }
    h = (h + 1) & (W::kHash - 1);
  }
  return false;
}

// Step 2: the cavity of p from t0 on unlocked reads. Returns kAInserted (lists filled),
// kARestart (an inconsistent read), kABig (the workspace is too small) or kAExact. The first
// pass of the loop tests t0 itself (one lane), so the conflict test's code exists once.
template <class W>
__device__ __forceinline__ int cavity_async(const Ctx& c, W& w, uint32_t t0, uint32_t p, const PtF& FP) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < W::kHash; i += 32) w.hkey[i] = kNone;
  __syncwarp();
  int flag = 0;  // 1 restart, 2 big, 4 a predicate the FP32 stage cannot decide
  int nc = 0, na = 0, nb = 0, head = 0;
  bool seed = true;
  while (flag == 0 && (seed || head < nc)) {
    const int k = lane >> 2, f = lane & 3;
    bool active;
    int ci;
    uint32_t u = kNone;
    if (seed) {
      active = lane == 0;
      ci = -1;
      u = t0;
    } else {
      const int batch = min(8, nc - head);
      active = k < batch;
      ci = head + k;
      if (active) {
        u = get4(w.cr[ci].n, f);
        if (u >= c.ntets) {
          flag = 1;
          active = false;
        }
      }
      flag = __reduce_or_sync(kFull, flag);
      if (flag) break;
      head += batch;
    }
    const int known = active ? hfind(w, u) : 0;
    const bool need = active && known == 0;
    const unsigned peers = __match_any_sync(kFull, need ? u : 0xFFFFFFFFu);
    const int leader = __ffs(peers) - 1;
    const bool is_leader = need && lane == leader;
    int res = 0, myflag = 0;
    Tet U;
    if (is_leader) {
      U = ld_tet(c.tets, u);
      const int in = (tet_dead(U.v) || !rec_ok(U, c.ntets, c.npts)) ? -1 : conflict_async<W::kCache>(c, u, U, FP);
      if (in == -2) {
        myflag |= 4;
      } else if (in < 0) {
        myflag |= 1;
      } else {
        res = in ? 1 : 2;
        if (seed && res != 1) myflag |= 1;  // the walk's tetrahedron was read mid-rewrite
        else if (!hinsert(w, u, (uint8_t)res)) myflag |= 2;
      }
    }
    const int lres = __shfl_sync(kFull, res, leader);
    res = need ? lres : known;
    flag = __reduce_or_sync(kFull, myflag);
    if (flag) break;
    const bool addC = is_leader && res == 1;
    const unsigned mC = __ballot_sync(kFull, addC);
    if (addC) {
      const int pos = nc + __popc(mC & lanemask_lt());
      if (pos < W::kCMax) {
        w.cl[pos] = u;
        w.cr[pos] = U;
      }
    }
    nc += __popc(mC);
    // outside tetrahedra (locked and verified)
    const bool addA = is_leader && res == 2;
    const unsigned mA = __ballot_sync(kFull, addA);
    if (addA) {
      const int pos = na + __popc(mA & lanemask_lt());
      if (pos < W::kAMax) {
        w.al[pos] = u;
        w.av[pos] = U.v;
      }
    }
    na += __popc(mA);
    const bool addB = active && ci >= 0 && res == 2;
    const unsigned mB = __ballot_sync(kFull, addB);
    if (addB) {
      const int pos = nb + __popc(mB & lanemask_lt());
      if (pos < W::kFMax) {
        w.bl_ci[pos] = (typename W::CI)ci;
        w.bl_f[pos] = (uint8_t)f;
      }
    }
    nb += __popc(mB);
    if (nc > W::kCMax || na > W::kAMax || nb > W::kFMax) flag |= 2;
    seed = false;
    __syncwarp();
  }
  if (lane == 0) {
    w.nc = nc;
    w.na = na;
    w.nb = nb;
  }
  __syncwarp();
  if (flag & 4) return kAExact;
  if (flag & 1) return kARestart;
  if (flag & 2) return kABig;
  return kAInserted;
}

// Slot of lock-list entry i: cavity slots, then the outside slots, then the ball's extra slots.
template <class W>
__device__ __forceinline__ uint32_t lock_entry(const W& w, int i, int nc, int na, int nx) {
  if (i < nc) return w.cl[i];
  i -= nc;
  if (i < na) return w.al[i];
  i -= na;
  return i < nx ? w.ex[i] : kNone;
}

// Releases the locks of the entries this lane took (bit k of `held` = entry lane + 32 k).
template <class W>
__device__ __forceinline__ void release_held(const W& w, uint32_t* lock, typename W::Held held, int nc, int na,
                                             int nx) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; held; ++k, held >>= 1)
    if (held & 1u) __stcg(&lock[lock_entry(w, lane + 32 * k, nc, na, nx)], 0u);
}

// Takes n slots from the warp's pool into w.ex, refilling it from the allocator (free list,
// then the bump pointer, as in the round-based engine). False when the store is full.
template <class W>
__device__ __forceinline__ bool pool_take(const Ctx& c, W& w, int n) {
  const int lane = threadIdx.x & 31;
  int np = w.np;
  while (np < n) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&c.st->alloc_cursor, (unsigned long long)kAChunk);
    base = __shfl_sync(kFull, base, 0);
    bool fail = false;
    const uint32_t s = virtual_slot(c, base + lane, w.fa, w.bump, c.st->capacity, fail);
    if (__any_sync(kFull, fail)) {
      if (lane == 0) raise_error(c.st, kErrCapacity, 0xA5u);
      return false;
    }
    w.pool[np + lane] = s;  // np < n <= kFMax, so np + 32 <= kPool
    np += 32;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) w.ex[i] = w.pool[np - 1 - i];
  __syncwarp();
  if (lane == 0) w.np = np - n;
  __syncwarp();
  return true;
}

// Puts n slots s[0, n) back into the pool; what does not fit goes to the pending list.
template <class W>
__device__ __forceinline__ void pool_give(const Ctx& c, W& w, const uint32_t* s, int n) {
  const int lane = threadIdx.x & 31;
  const int np = w.np;
  const int keep = min(n, W::kPool - np);
  for (int i = lane; i < keep; i += 32) w.pool[np + i] = s[i];
  if (n > keep) {
    unsigned long long pb = 0;
    if (lane == 0) pb = atomicAdd(&c.st->pending, (unsigned long long)(n - keep));
    pb = __shfl_sync(kFull, pb, 0);
    for (int i = keep + lane; i < n; i += 32) {
      if (pb + (i - keep) < c.st->free_capacity) c.pending[pb + (i - keep)] = s[i];
      else raise_error(c.st, kErrFreeList, 0xA7u);
    }
  }
  __syncwarp();
  if (lane == 0) w.np = np + keep;
  __syncwarp();
}

// One attempt at inserting p (steps 1-5). w.hint is the warp's last ball, updated on success.
template <class W>
__device__ __forceinline__ int try_insert(const Ctx& c, W& w, uint32_t* lock, uint32_t me, uint32_t p,
                                          const InsertLog& lg, bool io_balltest = true) {
  const int lane = threadIdx.x & 31;
  const PtF FP = load_ptf(c.ptf, p);
  for (int attempt = 0; attempt <= kARetry; ++attempt) {
    // 1. a start in conflict with p. Consecutive points of a segment are close, so p is often
    //    inside the circumsphere of a tetrahedron of the previous ball (it will be joined to the
    //    previous point): one insphere test per lane finds it without a walk. Otherwise walk.
    int ws = kAInserted;
    uint32_t t0 = kNone;
    if (attempt == 0 && w.bn > 0 && io_balltest) {
      bool in = false;
      if (lane < w.bn) {
        const uint4 v = __ldcg(reinterpret_cast<const uint4*>(c.tets + w.slot[lane]));
        in = !tet_dead(v) && ghost_pos(v) < 0 && v.x < c.npts && v.y < c.npts && v.z < c.npts && v.w < c.npts &&
             inside_async(c, v, FP) < 0;
      }
      const unsigned m = __ballot_sync(kFull, in);
      if (m) t0 = w.slot[__ffs(m) - 1];
    }
    if (t0 == kNone) {
      uint32_t start = attempt == 0 ? w.hint : kNone;
      if (start == kNone) start = c.point_hint[p];
      if (start == kNone) {
        uint32_t f, g;
        cells_of(c, FP, &f, &g);
        start = c.cell_hint[f];
        if (start == kNone) start = c.cell_hint2[g];
      }
      start = __shfl_sync(kFull, start, 0);
      uint32_t steps = 0;
      ws = walk_async(c, p, FP, start, p * 0x9E3779B1u >> 30, c.max_walk, &t0, &steps);
      if (lane == 0) {
        if (t0 != kNone && t0 < c.ntets) c.point_hint[p] = t0;
        w.cnt[5] += steps;
      }
    }
    if (lane == 0) w.bn = 0;  // used once
    if (ws == kADup || ws == kAWalkLimit || ws == kAExact) return ws;
    if (ws == kARestart) {
      if (lane == 0) w.cnt[6] += 1;
      continue;
    }
    // 2. cavity on unlocked reads
    const int r = cavity_async(c, w, t0, p, FP);
    if (r == kABig || r == kAExact) return r;
    if (r == kARestart) {
      if (lane == 0) w.cnt[6] += 1;
      continue;
    }
    const int nc = w.nc, na = w.na, nb = w.nb;
    const int reuse = min(nc, nb), nx = nb - reuse;
    if (nx > 0 && !pool_take(c, w, nx)) return kALost;
    // 3. lock C, A and the extra slots
    const int nl = nc + na + nx;
    typename W::Held held = 0;
    bool ok = true;
    for (int k = 0; lane + 32 * k < nl; ++k) {
      const uint32_t s = lock_entry(w, lane + 32 * k, nc, na, nx);
      if (s == kNone) continue;
      if (atomicCAS(&lock[s], 0u, me) == 0u) held |= (typename W::Held)1 << k;
      else ok = false;
    }
    if (!__all_sync(kFull, ok)) {
      release_held(w, lock, held, nc, na, nx);
      if (nx > 0) pool_give(c, w, w.ex, nx);
      return kALost;
    }
    __threadfence();
    // 4. re-read under the locks
    bool same = true;
    for (int i = lane; i < nc; i += 32) same = same && same_tet(ld_tet(c.tets, w.cl[i]), w.cr[i]);
    for (int i = lane; i < na; i += 32) {
      const uint32_t a = w.al[i];
      same = same && same_v(__ldcg(reinterpret_cast<const uint4*>(c.tets + a)), w.av[i]);
    }
    // which facet of each outside tetrahedron faces the cavity (it is locked: this stays true)
    for (int i = lane; i < nb; i += 32) {
      const int ci = w.bl_ci[i], f = w.bl_f[i] & 3;
      const uint32_t u = get4(w.cr[ci].n, f);
      const int back = back_facet(__ldcg(reinterpret_cast<const uint4*>(&c.tets[u].n)), w.cl[ci]);
      same = same && back >= 0;
      w.bl_f[i] = (uint8_t)(f | ((back & 3) << 2));
    }
    if constexpr (W::kCache) {
      // the cache's decisions were taken on entries read without locks: each is taken again on
      // the entry as it stands under the locks (an entry changes only with its record)
      for (int i = lane; i < nc; i += 32) {
        const uint4 v = w.cr[i].v;
        if (ghost_pos(v) < 0) same = same && inside_maybe_cached(c, w.cl[i], v, FP) < 0;
      }
      for (int i = lane; i < na; i += 32) {
        const uint4 v = w.av[i];
        if (ghost_pos(v) < 0) same = same && inside_maybe_cached(c, w.al[i], v, FP) > 0;
      }
    }
    if (!__all_sync(kFull, same)) {
      release_held(w, lock, held, nc, na, nx);
      if (nx > 0) pool_give(c, w, w.ex, nx);
      if (lane == 0) w.cnt[6] += 1;
      continue;
    }
    // 5. the ball: cavity slots first, then the extra slots
    for (int i = lane; i < nb; i += 32) w.slot[i] = i < reuse ? w.cl[i] : w.ex[i - reuse];
    w.vkey[lane] = kNoVertex;
    if constexpr (!W::kTable) {
      for (uint32_t i = lane; i < W::kEdgeN; i += 32) {
        w.ekey[i] = ~0ull;
        w.eval[i] = kNone;
      }
    }
    __syncwarp();
    // record every internal facet: facet a of new tetrahedron i holds the boundary edge b -> c
    bool vfail = false;
    // the table path's vertex slots of this lane's facets (lane and lane + 32; nb <= 60), kept
    // for the partner lookups below
    uint32_t vs[2] = {0, 0};
    for (int i = lane; i < nb; i += 32) {
      const int ci = w.bl_ci[i], f = w.bl_f[i] & 3;
      uint4 v = w.cr[ci].v;
      set4(v, f, p);
      int pos[3];
      after_pos(f, pos[0], pos[1], pos[2]);
      if constexpr (W::kTable) {
        const int la = vslot(w.vkey, get4(v, pos[0])), lb = vslot(w.vkey, get4(v, pos[1])),
                  lc = vslot(w.vkey, get4(v, pos[2]));
        if (la < 0 || lb < 0 || lc < 0) {
          vfail = true;
          continue;
        }
        vs[i >> 5] = (uint32_t)la | ((uint32_t)lb << 8) | ((uint32_t)lc << 16);
        w.tab[lb * 32 + lc] = (uint16_t)((i << 2) | pos[0]);
        w.tab[lc * 32 + la] = (uint16_t)((i << 2) | pos[1]);
        w.tab[la * 32 + lb] = (uint16_t)((i << 2) | pos[2]);
      } else {
        for (int k = 0; k < 3; ++k) {
          const uint32_t x = get4(v, pos[(k + 1) % 3]), y = get4(v, pos[(k + 2) % 3]);
          const unsigned long long key = ((unsigned long long)min(x, y) << 32) | max(x, y);
          uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & (W::kEdgeN - 1), sl = kNone;
#pragma unroll 1
          for (uint32_t probe = 0; probe < W::kEdgeN; ++probe) {
            const unsigned long long old = atomicCAS(&w.ekey[h], ~0ull, key);
            if (old == ~0ull || old == key) {
              sl = h;
              break;
            }
            h = (h + 1) & (W::kEdgeN - 1);
          }
          if (sl == kNone) {
            vfail = true;
            break;
          }
          w.hslot[3 * i + k] = sl;
          w.hold[3 * i + k] = atomicExch(&w.eval[sl], (uint32_t)((i << 2) | pos[k]));
        }
      }
    }
    __syncwarp();
    // every internal facet was recorded by its two sides (the cavity was verified under the
    // locks, so its boundary is a closed surface); a lookup that finds no partner is a bug
    bool bad = __any_sync(kFull, vfail);
    for (int i = lane; i < nb && !bad; i += 32) {
      const int ci = w.bl_ci[i], f = w.bl_f[i] & 3, back = w.bl_f[i] >> 2;
      uint4 v = w.cr[ci].v;
      const uint32_t out = get4(w.cr[ci].n, f);
      set4(v, f, p);
      int a, b, cc;
      after_pos(f, a, b, cc);
      uint32_t ea, eb, ec;
      if constexpr (W::kTable) {
        const uint32_t sl = vs[i >> 5];
        const int la = (int)(sl & 0xFFu), lb = (int)((sl >> 8) & 0xFFu), lc = (int)(sl >> 16);
        ea = vld(&w.tab[lc * 32 + lb]);
        eb = vld(&w.tab[la * 32 + lc]);
        ec = vld(&w.tab[lb * 32 + la]);
      } else {
        uint32_t e3[3];
        for (int k = 0; k < 3; ++k) {
          const uint32_t old = w.hold[3 * i + k];
          e3[k] = old != kNone ? old : vld(&w.eval[w.hslot[3 * i + k]]);
        }
        ea = e3[0];
        eb = e3[1];
        ec = e3[2];
      }
      if ((ea >> 2) >= (uint32_t)nb || (eb >> 2) >= (uint32_t)nb || (ec >> 2) >= (uint32_t)nb ||
          (ea >> 2) == (uint32_t)i || (eb >> 2) == (uint32_t)i || (ec >> 2) == (uint32_t)i) {
        bad = true;
        break;
      }
      uint4 n4;
      set4(n4, f, out);
      set4(n4, a, w.slot[ea >> 2]);
      set4(n4, b, w.slot[eb >> 2]);
      set4(n4, cc, w.slot[ec >> 2]);
      const uint32_t s = w.slot[i];
      uint4* dst = reinterpret_cast<uint4*>(c.tets + s);
      __stcg(dst, v);
      __stcg(dst + 1, n4);
      if constexpr (W::kCache) {
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;  // a ghost's entry stays invalid
        if (ghost_pos(v) < 0)
          subdet_make(load_ptf(c.ptf, v.x), load_ptf(c.ptf, v.y), load_ptf(c.ptf, v.z), load_ptf(c.ptf, v.w), q0, q1);
        __stcg(c.subdet + 2 * (size_t)s, q0);
        __stcg(c.subdet + 2 * (size_t)s + 1, q1);
      }
      __stcg(reinterpret_cast<uint32_t*>(&c.tets[out].n) + back, s);
    }
    if (__any_sync(kFull, bad)) {
      if (lane == 0) raise_error(c.st, kErrInternal, 0xA8u);
      release_held(w, lock, held, nc, na, nx);
      return kALost;
    }
    // cavity slots left over (|C| > |B|) die, keep a redirect into the ball, and join the pool
    const int freed = nc - nb;
    if (freed > 0) {
      const uint32_t redirect = w.slot[0];
      for (int i = lane; i < freed; i += 32) {
        uint4* dst = reinterpret_cast<uint4*>(c.tets + w.cl[nb + i]);
        __stcg(dst, make_uint4(kDeadMark, kDeadMark, kDeadMark, kDeadMark));
        __stcg(dst + 1, make_uint4(redirect, kNone, kNone, kNone));
      }
    }
    __threadfence();
    release_held(w, lock, held, nc, na, nx);
    if (freed > 0) pool_give(c, w, w.cl + nb, freed);
    if (lane == 0) {
      const uint32_t s0 = w.slot[0];
      uint32_t f, g;
      cells_of(c, FP, &f, &g);
      c.cell_hint[f] = s0;
      c.cell_hint2[g] = s0;
      c.point_hint[p] = s0;
      // the handle's state shares one cache line with the allocator's atomics: every warp
      // writing it per insertion serialised the whole launch, so it is refreshed now and then
      if ((w.cnt[0] & 63u) == 0) c.st->anchor = s0;
      log_outcome(lg, p, kCandInserted, nc);
      w.hint = s0;
      w.bn = W::kTable ? (nb < 32 ? nb : 32) : 0;
      w.cnt[0] += 1;
      w.cnt[3] += nc;
      w.cnt[4] += nb;
    }
    __syncwarp();
    return kAInserted;
  }
  return kALost;
}

// Hands point p to a queue of the host's next step (0: next pass, 1: large cavities, 2: the
// round-based engine's exact predicates). Lane 0.
__device__ __forceinline__ void to_queue(const AsyncIO& io, const Ctx& c, int q, uint32_t p) {
  uint32_t* out = q == 0 ? io.lose_out : (q == 1 ? io.big_out : io.exact_out);
  const int qi = q == 0 ? io.lose_q : (q == 1 ? io.big_q : io.exact_q);
  const unsigned long long b = atomicAdd(&c.st->q[qi], 1ull);
  out[b] = p;
}

// A cavity too large for the warp's shared-memory workspace: the same insertion again in a
// global-memory workspace borrowed from the launch's pool (tried at a few places, never waited
// for). Returns kABig when none is free or the cavity exceeds it too. The borrowed workspace's
// counters, spare slots and ball hint come back to the warp's own. Out of line: it runs for
// about one point in 1500, and inlined it would double the kernel's instruction footprint.
template <class W>
__device__ __noinline__ int try_insert_large(const Ctx& c, const AsyncIO& io, W& w, uint32_t* lock, uint32_t me,
                                             uint32_t p, const InsertLog& lg) {
  if (!io.big_ws || io.big_n == 0) return kABig;
  const int lane = threadIdx.x & 31;
  int k = -1;
  if (lane == 0)
    for (int t = 0; t < 8 && k < 0; ++t) {
      const uint32_t cand = (me * 0x9E3779B1u + (uint32_t)t * 0x85EBCA6Bu) % io.big_n;
      if (atomicCAS(&io.big_busy[cand], 0u, 1u) == 0u) k = (int)cand;
    }
  k = __shfl_sync(kFull, k, 0);
  if (k < 0) return kABig;
  LargeWST<W::kCache>& L = static_cast<LargeWST<W::kCache>*>(io.big_ws)[k];
  if (lane == 0) {
    L.fa = w.fa;
    L.bump = w.bump;
    L.np = 0;
    L.bn = 0;
    L.hint = w.hint;
    for (int q = 0; q < 8; ++q) L.cnt[q] = 0;
  }
  __syncwarp();
  const int r = try_insert(c, L, lock, me, p, lg);
  pool_give(c, w, L.pool, L.np);
  if (lane == 0) {
    w.cnt[0] += L.cnt[0];
    w.cnt[3] += L.cnt[3];
    w.cnt[4] += L.cnt[4];
    w.cnt[5] += L.cnt[5];
    w.cnt[6] += L.cnt[6];
    if (r == kAInserted) w.hint = L.hint;
    w.bn = 0;
    __threadfence();
    atomicExch(&io.big_busy[k], 0u);
  }
  __syncwarp();
  return r;
}

// One warp's work: segment [b0, e0) of io's list in order, deferred points retried after later
// insertions, then what is left handed on, unused slots returned and counters flushed.
template <class W>
__device__ __forceinline__ void run_segment(const Ctx& c, const AsyncIO& io, W& w, uint32_t* lock, uint32_t me,
                                            uint64_t b0, uint64_t e0, const uint8_t* vflag, const InsertLog& lg) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    w.fa = __ldcg(&c.st->free_avail);
    w.bump = __ldcg(&c.st->bump);
    w.np = 0;
    w.bn = 0;
    for (int k = 0; k < 8; ++k) w.cnt[k] = 0;
    w.hint = b0 < e0 ? c.point_hint[io.q ? io.q[b0] : io.qbase + (uint32_t)b0] : kNone;
  }
  __syncwarp();
  int nd = 0, dhead = 0;
  uint64_t i = b0;
  int since = 0;  // insertions since the last retry of a deferred point
  for (;;) {
    __syncwarp();  // lane 0's writes to the deferred list are seen by every lane below
    uint32_t p;
    bool retried = false;
    if (nd > 0 && (i >= e0 || since >= 4)) {
      p = w.defer[dhead];
      dhead = (dhead + 1) % kADefer;
      --nd;
      retried = true;
      since = 0;
    } else if (i < e0) {
      p = io.q ? io.q[i] : io.qbase + (uint32_t)i;
      ++i;
      if (vflag[p] != 0) continue;
    } else {
      break;
    }
    if (lane == 0) w.cnt[2] += 1;
    int r = try_insert(c, w, lock, me, p, lg, io.ball_start != 0);
    if constexpr (W::kTable) {
      if (r == kABig) r = try_insert_large(c, io, w, lock, me, p, lg);
    }
    // a raised error stops the launch; read every 16 points for the same reason as the anchor
    unsigned err = 0;
    if (lane == 0 && (w.cnt[2] & 15u) == 0) err = __ldcg(&c.st->error);
    if (__shfl_sync(kFull, err, 0) != 0u) break;
    if (r == kAInserted) {
      ++since;
      continue;
    }
    // every lane holds the same r, nd, dhead and `retried`: the decisions below are uniform
    if (r == kALost && lane == 0) {
      w.cnt[1] += 1;
      log_outcome(lg, p, kCandLost, 0);
    }
    if (r == kADup) {
      if (lane == 0) atomicAdd(&c.st->n_dups, 1ull);
    } else if (r == kABig) {
      if (lane == 0) to_queue(io, c, 1, p);
    } else if (r == kAExact) {
      if (lane == 0) to_queue(io, c, 2, p);
    } else if (r == kALost && !retried && nd < kADefer) {
      if (lane == 0) w.defer[(dhead + nd) % kADefer] = p;
      ++nd;
    } else {  // a walk over its step bound, or a point that lost again: the next pass
      if (lane == 0) to_queue(io, c, 0, p);
    }
  }
  __syncwarp();
  // what is left: deferred points to the next pass, unused slots back to the allocator
  if (lane == 0)
    for (int k = 0; k < nd; ++k) to_queue(io, c, 0, w.defer[(dhead + k) % kADefer]);
  const int np = w.np;
  if (np > 0) {
    unsigned long long pb = 0;
    if (lane == 0) pb = atomicAdd(&c.st->pending, (unsigned long long)np);
    pb = __shfl_sync(kFull, pb, 0);
    for (int k = lane; k < np; k += 32) {
      if (pb + k < c.st->free_capacity) c.pending[pb + k] = w.pool[k];
      else raise_error(c.st, kErrFreeList, 0xA9u);
    }
  }
  if (lane == 0) {
    unsigned long long* dst[8] = {&c.st->n_inserted, &c.st->n_conflicts, &c.st->n_attempts, &c.st->sum_cavity,
                                  &c.st->sum_ball, &c.st->sum_walk, &c.st->n_restart, &c.st->n_inserted_async};
    w.cnt[7] = w.cnt[0];
    for (int k = 0; k < 8; ++k)
      if (w.cnt[k]) atomicAdd(dst[k], (unsigned long long)w.cnt[k]);
  }
}

template <int kMinBlocks, bool kCache = false>
__global__ void __launch_bounds__(kAW * 32, kMinBlocks) k_async(Ctx c, AsyncIO io, uint32_t* lock,
                                                               const uint8_t* __restrict__ vflag, InsertLog lg) {
  __shared__ SmallWST<kCache> s_ws[kAW];
  const int wid = threadIdx.x >> 5;
  const uint32_t seg = blockIdx.x * kAW + wid;
  if (seg >= io.W) return;
  uint64_t b0, e0;
  if (io.bounds) {  // segments of equal predicted work (the learned schedule)
    b0 = io.bounds[seg];
    e0 = io.bounds[seg + 1];
  } else {
    b0 = (uint64_t)seg * io.L;
    e0 = b0 + io.L < io.m ? b0 + io.L : io.m;
  }
  run_segment(c, io, s_ws[wid], lock, seg + 1, b0, e0, vflag, lg);
}

// Large cavities (beyond the shared-memory workspaces): the same insertion with each warp's
// workspace in global memory. Owner words are per warp of the launch, and this kernel never
// runs beside k_async, so warp numbers may repeat across the two.
template <bool kCache>
__global__ void __launch_bounds__(128) k_async_big(Ctx c, AsyncIO io, uint32_t* lock, const uint8_t* __restrict__ vflag,
                                                  InsertLog lg, LargeWST<kCache>* ws) {
  const uint32_t seg = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (seg >= io.W) return;
  const uint64_t b0 = (uint64_t)seg * io.L;
  const uint64_t e0 = b0 + io.L < io.m ? b0 + io.L : io.m;
  run_segment(c, io, ws[seg], lock, seg + 1, b0, e0, vflag, lg);
}

// Folds the allocator of the launch into the free list, as a round close does
// (finish_round_block): the slots freed during the launch (pending) follow the free-list
// entries it did not consume. Copy on the whole grid, then the state on one thread.
__global__ void k_async_close_copy(Ctx c) {
  const DevState* st = c.st;
  const unsigned long long used = __ldcg(&st->alloc_cursor), fa = __ldcg(&st->free_avail);
  const unsigned long long consumed = used < fa ? used : fa, nfa = fa - consumed;
  unsigned long long np = __ldcg(&st->pending);
  if (nfa + np > st->free_capacity) np = st->free_capacity - nfa;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < np;
       i += (unsigned long long)gridDim.x * blockDim.x)
    c.freelist[nfa + i] = __ldcg(&c.pending[i]);
}

__global__ void k_async_close_state(Ctx c) {
  DevState* st = c.st;
  const unsigned long long used = st->alloc_cursor, fa = st->free_avail;
  const unsigned long long consumed = used < fa ? used : fa, nfa = fa - consumed;
  unsigned long long np = st->pending;
  if (nfa + np > st->free_capacity) {
    raise_error(st, kErrFreeList, 0xAAu);
    np = st->free_capacity - nfa;
  }
  st->bump += used - consumed;
  st->free_avail = nfa + np;
  st->alloc_cursor = 0;
  st->pending = 0;
  st->stamp += 1;
  st->blocks_done = 0;
}

int g_async_blocks = 0;  // resident blocks per SM the kernel is built for (0: not chosen yet)

int async_blocks_per_sm() {
  if (!g_async_blocks) {
    // 8 resident blocks (32 warps) per SM at 64 registers measured fastest: 255 ms per 1e7 uniform
    // step against 265 (6 blocks, 80 registers), 276 (5, 96) and 301 (4, 128)
    int v = 8;
    if (const char* e = std::getenv("DT_ASYNC_BLOCKS")) v = std::atoi(e);
    g_async_blocks = (v == 4 || v == 5 || v == 6 || v == 7 || v == 8) ? v : 8;
  }
  return g_async_blocks;
}

}  // namespace

int async_launch(const Ctx& c, const AsyncIO& io, uint32_t* lock, const uint8_t* vflag, const InsertLog& lg,
                 cudaStream_t s) {
  if (io.W == 0 || io.m == 0) return DT_OK;
  Ctx cc = c;
  cc.coherent = 1;
  cc.max_walk = io.max_walk;
  const unsigned blocks = (io.W + kAW - 1) / kAW;
  // the sub-determinant cache ablation is built for the default 8 blocks per SM only
  switch (c.subdet ? 0 : async_blocks_per_sm()) {
    case 0: k_async<8, true><<<blocks, kAW * 32, 0, s>>>(cc, io, lock, vflag, lg); break;
    case 4: k_async<4><<<blocks, kAW * 32, 0, s>>>(cc, io, lock, vflag, lg); break;
    case 5: k_async<5><<<blocks, kAW * 32, 0, s>>>(cc, io, lock, vflag, lg); break;
    case 6: k_async<6><<<blocks, kAW * 32, 0, s>>>(cc, io, lock, vflag, lg); break;
    case 7: k_async<7><<<blocks, kAW * 32, 0, s>>>(cc, io, lock, vflag, lg); break;
    default: k_async<8><<<blocks, kAW * 32, 0, s>>>(cc, io, lock, vflag, lg); break;
  }
  k_async_close_copy<<<152, 256, 0, s>>>(cc);
  k_async_close_state<<<1, 1, 0, s>>>(cc);
  g_kernel_launches += 3;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

size_t async_big_ws_bytes() { return sizeof(LargeWS); }

int async_launch_big(const Ctx& c, const AsyncIO& io, uint32_t* lock, const uint8_t* vflag, const InsertLog& lg,
                     void* ws, cudaStream_t s) {
  if (io.W == 0 || io.m == 0) return DT_OK;
  Ctx cc = c;
  cc.coherent = 1;
  cc.max_walk = io.max_walk;
  if (c.subdet)
    k_async_big<true><<<(io.W + 3) / 4, 128, 0, s>>>(cc, io, lock, vflag, lg, static_cast<LargeWST<true>*>(ws));
  else
    k_async_big<false><<<(io.W + 3) / 4, 128, 0, s>>>(cc, io, lock, vflag, lg, static_cast<LargeWS*>(ws));
  k_async_close_copy<<<152, 256, 0, s>>>(cc);
  k_async_close_state<<<1, 1, 0, s>>>(cc);
  g_kernel_launches += 3;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

int async_max_warps() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int mb = async_blocks_per_sm();
    cudaError_t e = mb == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_async<4>, kAW * 32, 0)
                  : mb == 5 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_async<5>, kAW * 32, 0)
                  : mb == 6 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_async<6>, kAW * 32, 0)
                  : mb == 7 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_async<7>, kAW * 32, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_async<8>, kAW * 32, 0);
    if (e != cudaSuccess) per = mb;
    cached = std::max(1, sms * std::max(per, 1) * kAW);
  }
  return cached;
}

}  // namespace dtg
