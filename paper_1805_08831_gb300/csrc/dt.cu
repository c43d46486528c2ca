// Kernels, handle and C ABI of the GB300 Delaunay library (see include/dt.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <new>
#include <vector>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"
#include "predicates.cuh"

namespace dtg {
namespace {

constexpr int kCavWarps = 4;  // candidates per block of the cavity kernel (4 measured faster than 8)
constexpr int kInsWarps = 8;  // candidates per block of the ball kernel
constexpr uint32_t kDefaultWalk = 48;          // walk steps per pass (a longer walk resumes next pass)
constexpr uint32_t kAsyncWalk = 4096;          // walk steps per attempt of the asynchronous engine
constexpr uint32_t kAsyncBigWarps = 512;       // warps (global-memory workspaces) of its large-cavity kernel
constexpr uint32_t kAsyncBorrow = 256;         // large-cavity workspaces the main kernel's warps may borrow
constexpr uint64_t kLongWalkBelow = 8192;      // retry lists shorter than this walk up to
constexpr uint32_t kLongWalkSteps = 1u << 14;  // this many steps per pass
constexpr uint32_t kScratchStride = kCMax + kFMax;

// Queues of points a round hands on (DevState::q).
constexpr int kQNext = 0;   // lost a conflict or hit the walk limit: next pass
constexpr int kQBig = 1;    // cavity too large for shared memory: large-cavity rounds
constexpr int kQBig2 = 2;   // lost a conflict in a large-cavity round: next large-cavity round
constexpr int kQHuge = 3;   // cavity too large even for the large-cavity workspace: serial path
constexpr int kQBigG = 4;   // cavity too large for the shared-memory large rounds: global-memory rounds
constexpr int kQExact = 5;  // the asynchronous engine could not decide a predicate: round-based rounds
constexpr int kNumQueues = 6;
static_assert(sizeof(DevState::q) / sizeof(DevState::q[0]) == kNumQueues, "one length per queue");

// Large-cavity rounds, first tier: one warp per candidate with its workspaces in dynamic shared
// memory (kMedWarps warps per block), for cavities of up to kMedCN tetrahedra and kMedFN
// boundary facets. Hash probes and list appends then cost shared-memory latency instead of an
// L2 round trip; larger cavities go on to the global-memory tier.
constexpr int kMedWarps = 4;
constexpr uint32_t kMedHash = 1024, kMedCN = 256, kMedFN = 192, kMedEdge = 512;

// Large-cavity rounds: per-candidate workspaces in global memory.
constexpr uint32_t kBigR = 1024;      // candidates per large-cavity round
constexpr uint32_t kBigHashN = 4096;  // visited-set slots
constexpr uint32_t kBigCN = 1024;     // cavity tetrahedra
constexpr uint32_t kBigFN = 1024;     // boundary facets
constexpr uint32_t kBigEdgeN = 4096;  // edge-hash slots

// Serial path (one point at a time, one warp): the largest workspaces.
// The serial path's workspace holds cavities of kHugeC tetrahedra at first and grows with the
// tetrahedron store, up to kHugeCMax: points inserted into a mesh with an empty interior (the first
// refinement iterations of a surface) can have cavities of a large share of the mesh.
constexpr uint32_t kHugeC = 1u << 15;
constexpr uint32_t kHugeCMax = 1u << 20;

inline size_t big_stride() { return carve(nullptr, kBigHashN, kBigCN, kBigFN, kBigEdgeN, nullptr); }
__host__ __device__ inline size_t med_stride() { return carve(nullptr, kMedHash, kMedCN, kMedFN, kMedEdge, nullptr); }

// Where the candidates of a round come from and where the ones it does not insert go.
struct RoundIO {
  const uint32_t* q;  // candidate list; nullptr = the vertex range qbase + idx
  uint32_t qbase;
  uint64_t m, L, j;   // segment s of length L offers its point j (Section 3.3 partitions)
  uint32_t R;         // segments = candidates this round
  uint32_t* lose_out;
  int lose_q;
  uint32_t* big_out;
  int big_q;
  const uint8_t* prank;  // per vertex: scheduling rank of its claims (null: 0)
};

// ------------------------------------------------------------------ kernels of one round
__global__ void __launch_bounds__(256) k_walk(Ctx c, RoundIO io, const uint8_t* __restrict__ vflag,
                                              uint32_t* cand_p, uint32_t* cand_t, uint32_t* cand_status) {
  __shared__ unsigned long long s_steps, s_limit;
  __shared__ unsigned int s_max;
  if (threadIdx.x == 0) {
    s_steps = 0;
    s_limit = 0;
    s_max = 0;
  }
  __syncthreads();
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < io.R) {
    uint64_t idx = (uint64_t)s * io.L + io.j;
    uint32_t status = kCandEmpty, p = kNone, t = kNone;
    if (idx < io.m) {
      p = io.q ? io.q[idx] : io.qbase + (uint32_t)idx;
      if (vflag[p] == 0) {
        uint32_t anchor = __ldcg(&c.st->anchor);
        PtF FP = load_ptf(c.ptf, p);
        // hints (Algorithm 1 walks from the previous ball): this point's last stop, then the
        // segment predecessor's, then the fine and coarse grid cells, then any live tetrahedron
        uint32_t hint = c.point_hint[p];
        if (hint == kNone && io.j > 0) {
          uint32_t pp = io.q ? io.q[idx - 1] : io.qbase + (uint32_t)(idx - 1);
          hint = c.point_hint[pp];
        }
        if (hint == kNone) {
          uint32_t f, g;
          cells_of(c, FP, &f, &g);
          hint = c.cell_hint[f];
          if (hint == kNone) hint = c.cell_hint2[g];
        }
        uint32_t steps = 0;
        status = walk_point(c, p, FP, hint, p * 0x9E3779B1u >> 30, anchor, c.max_walk, &t, &steps);
        atomicAdd(&s_steps, (unsigned long long)steps);
        atomicMax(&s_max, steps);
        c.point_hint[p] = t;
        if (status == kCandWalkLimit) atomicAdd(&s_limit, 1ull);
      }
    }
    cand_p[s] = p;
    cand_t[s] = t;
    cand_status[s] = status;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_steps) atomicAdd(&c.st->sum_walk, s_steps);
    if (s_limit) atomicAdd(&c.st->n_walk_limit, s_limit);
    if (s_max) atomicMax(&c.st->max_walk, (unsigned long long)s_max);
  }
}

// kMode 0: the shared-memory path (8 candidates per block); 1: large cavities with
// global-memory workspaces; 2: large cavities with dynamic shared-memory workspaces.
template <int kMode>
__global__ void __launch_bounds__((kCavWarps > kMedWarps ? kCavWarps : kMedWarps) * 32, 32 / kCavWarps) k_cavity(Ctx c, uint32_t R, const uint32_t* __restrict__ cand_p,
                                                const uint32_t* __restrict__ cand_t, uint32_t* cand_status,
                                                uint32_t* cand_nc, uint32_t* cand_nb, uint32_t* scratch,
                                                char* bigmem, size_t bigstride, const uint8_t* __restrict__ prank) {
  constexpr bool kSmall = kMode == 0;
  constexpr int kW = kMode == 2 ? kMedWarps : kCavWarps;
  __shared__ uint32_t s_hkey[kSmall ? kCavWarps : 1][kHash];
  __shared__ uint8_t s_hval[kSmall ? kCavWarps : 1][kHash];
  __shared__ uint32_t s_c[kSmall ? kCavWarps : 1][kCMax];
  __shared__ uint32_t s_b[kSmall ? kCavWarps : 1][kFMax];
  extern __shared__ __align__(16) char s_dyn[];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t cand = blockIdx.x * kW + wid;
  if (cand >= R) return;
  if (cand_status[cand] != kCandLocated) return;
  uint32_t p = cand_p[cand];
  PtF FP = load_ptf(c.ptf, p);
  unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), prank ? prank[p] : 0u, p);
  CavWS w;
  if (kMode == 1) {
    BigWS b;
    carve(bigmem + (size_t)cand * bigstride, kBigHashN, kBigCN, kBigFN, kBigEdgeN, &b);
    w = b.cav;
  } else if (kMode == 2) {
    BigWS b;
    carve(s_dyn + (size_t)wid * med_stride(), kMedHash, kMedCN, kMedFN, kMedEdge, &b);
    w = b.cav;
  } else {
    w = CavWS{s_hkey[wid], s_hval[wid], kHash - 1, s_c[wid], kCMax, s_b[wid], kFMax};
  }
  int nc = 0, nb = 0;
  int r = cavity_warp(c, w, cand_t[cand], p, FP, prio, &nc, &nb);
  if (kMode != 1 && r == kCandLocated) {
    // the lists outlive the block: the ball kernel reads them back
    const uint32_t cap = kMode == 2 ? kMedCN : kCMax;
    uint32_t* dst = scratch + (size_t)cand * (kMode == 2 ? kMedCN + kMedFN : kScratchStride);
    for (int i = lane; i < nc; i += 32) dst[i] = w.clist[i];
    for (int i = lane; i < nb; i += 32) dst[cap + i] = w.blist[i];
  }
  if (lane == 0) {
    cand_status[cand] = (uint32_t)r;
    cand_nc[cand] = (uint32_t)nc;
    cand_nb[cand] = (uint32_t)nb;
  }
}

// Ball phase: each warp verifies and inserts one candidate independently (no block barrier);
// the last warp of each block flushes the block's counters, and the last of those closes the
// round.
template <int kMode>
__global__ void __launch_bounds__((kInsWarps > kMedWarps ? kInsWarps : kMedWarps) * 32) k_insert(Ctx c, RoundIO io, const uint32_t* __restrict__ cand_p,
                                                uint32_t* cand_status, const uint32_t* __restrict__ cand_nc,
                                                const uint32_t* __restrict__ cand_nb,
                                                const uint32_t* __restrict__ scratch, char* bigmem,
                                                size_t bigstride, InsertLog lg) {
  constexpr int W = kMode == 0 ? kInsWarps : 1;
  constexpr int kW = kMode == 2 ? kMedWarps : kInsWarps;  // candidates per block
  extern __shared__ __align__(16) char s_dyn[];
  __shared__ uint4 s_nv[W][kFMax];
  __shared__ uint4 s_nn[W][kFMax];
  __shared__ uint32_t s_out[W][kFMax];
  __shared__ uint32_t s_slot[W][kFMax];
  __shared__ uint8_t s_ipos[W][kFMax + 4];
  __shared__ uint32_t s_vkey[W][32];
  __shared__ uint16_t s_tab[W][32 * 32];
  __shared__ unsigned int s_warps_done, s_nlose, s_nbigq;
  __shared__ uint32_t s_lose[kW], s_bigq[kW];
  __shared__ unsigned long long s_stat[6];  // inserted, conflicts, attempts, cavity, ball, dups
  if (threadIdx.x == 0) {
    s_warps_done = 0;
    s_nlose = 0;
    s_nbigq = 0;
    for (int k = 0; k < 6; ++k) s_stat[k] = 0;
  }
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t cand = blockIdx.x * kW + wid;
  uint32_t status = kCandEmpty, p = kNone;
  if (cand < io.R) {
    status = cand_status[cand];
    p = cand_p[cand];
  }
  if (status == kCandLocated) {
    unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), io.prank ? io.prank[p] : 0u, p);
    int nc = (int)cand_nc[cand], nb = (int)cand_nb[cand];
    const uint32_t* cl;
    const uint32_t* bl;
    InsWS w;
    if (kMode == 1) {
      BigWS b;
      carve(bigmem + (size_t)cand * bigstride, kBigHashN, kBigCN, kBigFN, kBigEdgeN, &b);
      w = b.ins;
      cl = b.cav.clist;
      bl = b.cav.blist;
    } else if (kMode == 2) {
      BigWS b;
      carve(s_dyn + (size_t)wid * med_stride(), kMedHash, kMedCN, kMedFN, kMedEdge, &b);
      w = b.ins;
      cl = scratch + (size_t)cand * (kMedCN + kMedFN);
      bl = cl + kMedCN;
    } else {
      w = InsWS{s_nv[wid], s_nn[wid], s_out[wid], s_slot[wid], s_ipos[wid], s_vkey[wid], s_tab[wid],
                nullptr, nullptr, nullptr, nullptr, 0};
      cl = scratch + (size_t)cand * kScratchStride;
      bl = cl + kCMax;
    }
    status = insert_warp(c, w, p, prio, cl, nc, bl, nb, nb <= kFMax, __ldcg(&c.st->free_avail),
                         __ldcg(&c.st->bump), c.st->capacity);
    if (status == kCandInserted && lane == 0) {
      PtF FP = load_ptf(c.ptf, p);
      uint32_t f, g, s0 = w.slot[0];
      cells_of(c, FP, &f, &g);
      c.cell_hint[f] = s0;
      c.cell_hint2[g] = s0;
      c.point_hint[p] = s0;
      // the handle's state line also takes the allocator's atomics: refresh the anchor rarely
      if ((p & 63u) == 0) c.st->anchor = s0;
      atomicAdd(&s_stat[0], 1ull);
      atomicAdd(&s_stat[3], (unsigned long long)nc);
      atomicAdd(&s_stat[4], (unsigned long long)nb);
    }
  }
  unsigned int closer = 0;
  if (lane == 0) {
    if (cand < io.R && status != kCandEmpty) {
      log_outcome(lg, p, status, status == kCandInserted ? (int)cand_nc[cand] : 0);
      atomicAdd(&s_stat[2], 1ull);
      if (status == kCandLost) atomicAdd(&s_stat[1], 1ull);
      if (status == kCandDup) atomicAdd(&s_stat[5], 1ull);
      if (status == kCandLost || status == kCandWalkLimit) s_lose[atomicAdd(&s_nlose, 1u)] = p;
      else if (status == kCandBig) s_bigq[atomicAdd(&s_nbigq, 1u)] = p;
    }
    __threadfence_block();
    if (atomicAdd(&s_warps_done, 1u) == kW - 1) {
      // every warp of the block has counted itself: flush the block's queues and counters
      closer = 1;
      unsigned nl = s_nlose, nbq = s_nbigq;
      if (nl) {
        unsigned long long b = atomicAdd(&c.st->q[io.lose_q], (unsigned long long)nl);
        for (unsigned k = 0; k < nl; ++k) io.lose_out[b + k] = s_lose[k];
      }
      if (nbq) {
        unsigned long long b = atomicAdd(&c.st->q[io.big_q], (unsigned long long)nbq);
        for (unsigned k = 0; k < nbq; ++k) io.big_out[b + k] = s_bigq[k];
      }
      if (s_stat[0]) atomicAdd(&c.st->n_inserted, s_stat[0]);
      if (s_stat[1]) atomicAdd(&c.st->n_conflicts, s_stat[1]);
      if (s_stat[2]) atomicAdd(&c.st->n_attempts, s_stat[2]);
      if (s_stat[3]) atomicAdd(&c.st->sum_cavity, s_stat[3]);
      if (s_stat[4]) atomicAdd(&c.st->sum_ball, s_stat[4]);
      if (s_stat[5]) atomicAdd(&c.st->n_dups, s_stat[5]);
      if (kMode != 0 && s_stat[0]) atomicAdd(&c.st->n_big, s_stat[0]);
    }
  }
  // the last warp of the last block closes the round
  closer = __shfl_sync(kFull, closer, 0);
  if (closer == 1u) {
    unsigned int last = 0;
    if (lane == 0) {
      __threadfence();
      last = (atomicAdd(&c.st->blocks_done, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    last = __shfl_sync(kFull, last, 0);
    if (last) {
      __threadfence();
      finish_round_warp(c);
    }
  }
}

// Points whose cavity exceeds even the large-cavity workspaces: inserted one at a time by one
// warp with the largest workspaces; nothing else runs concurrently.
__global__ void k_huge(Ctx c, const uint32_t* list, uint32_t n, BigWS ws, InsertLog lg) {
  const int lane = threadIdx.x & 31;
  for (uint32_t k = 0; k < n; ++k) {
    uint32_t p = list[k];
    PtF FP = load_ptf(c.ptf, p);
    uint32_t t = kNone, steps = 0;
    int s = 0;
    if (lane == 0) {
      uint32_t anchor = __ldcg(&c.st->anchor);
      uint32_t hint = c.point_hint[p];
      if (hint == kNone) {
        uint32_t f, g;
        cells_of(c, FP, &f, &g);
        hint = c.cell_hint[f];
      }
      s = walk_point(c, p, FP, hint, 0, anchor, 1u << 22, &t, &steps);
    }
    s = __shfl_sync(kFull, s, 0);
    t = __shfl_sync(kFull, t, 0);
    if (s == kCandDup) {
      if (lane == 0) atomicAdd(&c.st->n_dups, 1ull);
      continue;
    }
    if (s != kCandLocated) {
      if (lane == 0) raise_error(c.st, kErrWalk, p);
      return;
    }
    unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), 0u, p);
    int nc = 0, nb = 0;
    int r = cavity_warp(c, ws.cav, t, p, FP, prio, &nc, &nb);
    if (r != kCandLocated) {
      if (lane == 0) raise_error(c.st, kErrBigCavity, p);
      return;
    }
    r = insert_warp(c, ws.ins, p, prio, ws.cav.clist, nc, ws.cav.blist, nb, nb <= kFMax,
                    __ldcg(&c.st->free_avail), __ldcg(&c.st->bump), c.st->capacity);
    if (r != kCandInserted) {
      if (lane == 0) raise_error(c.st, kErrInternal, p);
      return;
    }
    if (lane == 0) {
      uint32_t f, g, s0 = ws.ins.slot[0];
      cells_of(c, FP, &f, &g);
      c.cell_hint[f] = s0;
      c.cell_hint2[g] = s0;
      c.point_hint[p] = s0;
      c.st->anchor = s0;
      c.st->n_inserted += 1;
      c.st->n_big += 1;
      log_outcome(lg, p, kCandInserted, nc);
      c.st->sum_cavity += nc;
      c.st->sum_ball += nb;
    }
    __threadfence();
    __syncwarp();
    finish_round_warp(c);
  }
}


// ------------------------------------------------------------------ one-block engine
// The first insertions of a cloud (a few thousand points into a mesh that starts with one
// tetrahedron) offer little parallelism and large cavities: one thread block runs all of the
// first BRIO round itself, with block barriers in place of kernel boundaries between the walk,
// cavity and ball phases of a round. It takes the round's waves in order (up to kCtaWarps
// concurrent insertions, alpha * mesh size), then retries the points that lost until none is
// left. Each warp works in its own global-memory workspace, so cavities of up to
// kCtaCN / kCtaFN tetrahedra / facets stay here; larger ones go to the serial path.
constexpr int kCtaWarps = 32;
constexpr uint32_t kCtaHashN = 2048, kCtaCN = 512, kCtaFN = 512, kCtaEdgeN = 2048;

inline size_t cta_stride() { return carve(nullptr, kCtaHashN, kCtaCN, kCtaFN, kCtaEdgeN, nullptr); }

__global__ void __launch_bounds__(kCtaWarps * 32) k_cta_insert(Ctx c, const uint32_t* __restrict__ wlist,
                                                               const uint32_t* __restrict__ cum, int nwaves,
                                                               const uint8_t* __restrict__ vflag,
                                                               uint32_t* list_a, uint32_t* list_b,
                                                               uint32_t* huge_out, char* wsmem, size_t wsstride,
                                                               float alpha, uint32_t max_passes, InsertLog lg) {
  __shared__ uint32_t s_p[kCtaWarps], s_t[kCtaWarps], s_st[kCtaWarps], s_nc[kCtaWarps], s_nb[kCtaWarps];
  __shared__ unsigned int s_nout, s_R, s_err;
  __shared__ unsigned long long s_L, s_N0;
  __shared__ unsigned long long s_stat[6];  // inserted, conflicts, attempts, cavity, ball, walk
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  BigWS ws;
  carve(wsmem + (size_t)wid * wsstride, kCtaHashN, kCtaCN, kCtaFN, kCtaEdgeN, &ws);
  if (tid < 6) s_stat[tid] = 0;
  if (tid == 0) {
    s_N0 = __ldcg(&c.st->n_inserted);
    s_nout = 0;
  }
  __syncthreads();
  // passes: the waves (in order), then retries of the points that lost
  const uint32_t* q = wlist;
  uint64_t m = 0;
  uint32_t* out = list_a;
  int wave = 0;
  uint64_t woff = 0;
  for (uint32_t pass = 0; pass < max_passes; ++pass) {
    if (wave < nwaves) {
      q = wlist + woff;
      m = cum[wave] - woff;
      woff = cum[wave];
      ++wave;
    } else {
      // all waves done: the points that lost during them (or during the last retry)
      q = out;
      m = s_nout;
      out = (out == list_a) ? list_b : list_a;
      __syncthreads();
      if (tid == 0) s_nout = 0;
      if (m == 0) break;
    }
    if (tid == 0) {
      double N = (double)(s_N0 + s_stat[0]);
      uint64_t R = (uint64_t)fmax(1.0, alpha * N);
      R = R > kCtaWarps ? kCtaWarps : R;
      R = R > m ? m : R;
      s_R = (unsigned)(R > 0 ? R : 1);
      s_L = (m + s_R - 1) / s_R;
      s_err = __ldcg(&c.st->error);
    }
    __syncthreads();
    if (s_err) break;
    const uint32_t R = s_R;
    const uint64_t L = s_L;
    for (uint64_t j = 0; j < L; ++j) {
      // walk: one thread per candidate
      if (tid < (int)R) {
        uint64_t idx = (uint64_t)tid * L + j;
        uint32_t status = kCandEmpty, p = kNone, t = kNone;
        if (idx < m) {
          p = q[idx];
          if (vflag[p] == 0) {
            PtF FP = load_ptf(c.ptf, p);
            uint32_t hint = c.point_hint[p];
            if (hint == kNone && j > 0) hint = c.point_hint[q[idx - 1]];
            if (hint == kNone) {
              uint32_t f, g;
              cells_of(c, FP, &f, &g);
              hint = c.cell_hint[f];
              if (hint == kNone) hint = c.cell_hint2[g];
            }
            uint32_t steps = 0;
            status = walk_point(c, p, FP, hint, p * 0x9E3779B1u >> 30, __ldcg(&c.st->anchor), c.max_walk, &t, &steps);
            atomicAdd(&s_stat[5], (unsigned long long)steps);
            c.point_hint[p] = t;
          }
        }
        s_p[tid] = p;
        s_t[tid] = t;
        s_st[tid] = status;
      }
      __syncthreads();
      // cavity: one warp per candidate, in its own workspace
      if (wid < (int)R && s_st[wid] == kCandLocated) {
        uint32_t p = s_p[wid];
        unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), 0u, p);
        int nc = 0, nb = 0;
        int r = cavity_warp(c, ws.cav, s_t[wid], p, load_ptf(c.ptf, p), prio, &nc, &nb);
        if (lane == 0) {
          s_st[wid] = (uint32_t)r;
          s_nc[wid] = (uint32_t)nc;
          s_nb[wid] = (uint32_t)nb;
        }
      }
      __threadfence();
      __syncthreads();
      // ball: the same warp, from its workspace
      if (wid < (int)R && s_st[wid] == kCandLocated) {
        uint32_t p = s_p[wid];
        unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), 0u, p);
        int nc = (int)s_nc[wid], nb = (int)s_nb[wid];
        int r = insert_warp(c, ws.ins, p, prio, ws.cav.clist, nc, ws.cav.blist, nb, nb <= kFMax,
                            __ldcg(&c.st->free_avail), __ldcg(&c.st->bump), c.st->capacity);
        if (lane == 0) {
          s_st[wid] = (uint32_t)r;
          if (r == kCandInserted) {
            PtF FP = load_ptf(c.ptf, p);
            uint32_t f, g, s0 = ws.ins.slot[0];
            cells_of(c, FP, &f, &g);
            c.cell_hint[f] = s0;
            c.cell_hint2[g] = s0;
            c.point_hint[p] = s0;
            c.st->anchor = s0;
            atomicAdd(&s_stat[0], 1ull);
            atomicAdd(&s_stat[3], (unsigned long long)nc);
            atomicAdd(&s_stat[4], (unsigned long long)nb);
          }
        }
      }
      __threadfence();
      __syncthreads();
      if (tid < (int)R) {
        uint32_t st = s_st[tid], p = s_p[tid];
        if (st != kCandEmpty) log_outcome(lg, p, st, (int)s_nc[tid]);
        if (st != kCandEmpty) atomicAdd(&s_stat[2], 1ull);
        if (st == kCandLost) atomicAdd(&s_stat[1], 1ull);
        if (st == kCandLost || st == kCandWalkLimit) out[atomicAdd(&s_nout, 1u)] = p;
        else if (st == kCandBig) huge_out[atomicAdd(&c.st->q[kQHuge], 1ull)] = p;
        else if (st == kCandDup) atomicAdd(&c.st->n_dups, 1ull);
      }
      // the last warp closes the round while the first records this round's outcomes and walks
      // the next: neither touches the allocator or the stamp, and the barrier after the walk
      // orders the close before the next claims
      if (wid == kCtaWarps - 1) finish_round_warp(c);
    }
    __syncthreads();
  }
  if (tid == 0) {
    atomicAdd(&c.st->n_inserted, s_stat[0]);
    atomicAdd(&c.st->n_conflicts, s_stat[1]);
    atomicAdd(&c.st->n_attempts, s_stat[2]);
    atomicAdd(&c.st->sum_cavity, s_stat[3]);
    atomicAdd(&c.st->sum_ball, s_stat[4]);
    atomicAdd(&c.st->sum_walk, s_stat[5]);
    if (s_nout > 0 || wave < nwaves) raise_error(c.st, kErrInternal, 0xF000u);
  }
}

// Wave of each vertex of one BRIO round: its hash rank inside the round (a uniformly random
// order) against the cumulative wave ends; the stable sort by wave keeps the Moore order.
__global__ void k_wave_keys(uint32_t vbegin, uint64_t m, uint64_t base, uint64_t rank0,
                            const uint32_t* __restrict__ perm, const uint32_t* __restrict__ rank,
                            const uint32_t* __restrict__ cum, int nwaves, const uint8_t* __restrict__ risky,
                            uint64_t* keys, uint32_t* vals) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = vbegin + (uint32_t)i;
    uint64_t r = rank[perm[v - base]] - rank0;
    int lo = 0, hi = nwaves - 1;
    while (lo < hi) {
      int mid = (lo + hi) / 2;
      if (r < cum[mid]) hi = mid;
      else lo = mid + 1;
    }
    // with the learned schedule, the points expected to lose go after the rest of their wave
    keys[i] = risky ? 2 * (uint64_t)lo + risky[v] : (uint64_t)lo;
    vals[i] = v;
  }
}

// Init (Section 2.1): the first four non-coplanar vertices of the insertion order form a
// positive tetrahedron; four ghost tetrahedra close it (Section 2.6).
__global__ void k_init(Ctx c, uint32_t vbegin, uint32_t vend, uint8_t* vflag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  init_mesh(c, vbegin, vend, vflag, 0);
}

__device__ __forceinline__ void split_df(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);  // x - hi is exact in double
}

__global__ void k_build_pts(const double* __restrict__ xyz, const uint32_t* __restrict__ perm,
                            const uint8_t* __restrict__ dup, uint64_t n, uint64_t base,
                            Pt* pts, PtF* ptf, uint8_t* vflag, uint32_t* point_hint) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t i = perm[s];
    double x = xyz[3 * (uint64_t)i], y = xyz[3 * (uint64_t)i + 1], z = xyz[3 * (uint64_t)i + 2];
    pts[base + s] = make_pt(x, y, z, (double)(base + i));
    PtF f;
    split_df(x, f.hx, f.lx);
    split_df(y, f.hy, f.ly);
    split_df(z, f.hz, f.lz);
    f.hw = f.lw = 0.0f;
    ptf[base + s] = f;
    vflag[base + s] = dup[i];
    point_hint[base + s] = kNone;
  }
}

// Finite live tetrahedra with vertex ids mapped to input indices; canonical rotation optional.
// One counter update per warp and iteration (ballot, then each lane's rank among the warp's
// kept tetrahedra): a warp's rows land next to each other, and the counter sees 32 times fewer
// atomics. The grid-stride loop runs the same number of times on every lane of a warp.
__global__ void k_collect(const Tet* __restrict__ tets, uint64_t nslots, const Pt* __restrict__ pts,
                          uint64_t npts, uint32_t* out, unsigned long long* count, uint64_t cap,
                          int canonical) {
  const int lane = threadIdx.x & 31;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) - lane;
  for (uint64_t base = warp0; base < nslots; base += stride) {
    const uint64_t t = base + lane;
    bool keep = false;
    uint32_t r[4] = {0, 0, 0, 0};
    if (t < nslots) {
      const uint4 v = tets[t].v;
      keep = !tet_dead(v) && ghost_pos(v) < 0 && v.x < npts && v.y < npts && v.z < npts && v.w < npts;
      if (keep) {
        r[0] = (uint32_t)pts[v.x].w;
        r[1] = (uint32_t)pts[v.y].w;
        r[2] = (uint32_t)pts[v.z].w;
        r[3] = (uint32_t)pts[v.w].w;
        if (canonical) canonical_rotation(r);
      }
    }
    const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
    if (m == 0) continue;
    unsigned long long first = 0;
    if (lane == 0) first = atomicAdd(count, (unsigned long long)__popc(m));
    first = __shfl_sync(0xFFFFFFFFu, first, 0);
    if (keep) {
      const unsigned long long pos = first + __popc(m & ((1u << lane) - 1u));
      if (pos < cap) reinterpret_cast<uint4*>(out)[pos] = make_uint4(r[0], r[1], r[2], r[3]);
    }
  }
}

// Certificate of a mesh (the Delaunay lemma: a closed, consistently oriented complex whose every
// facet is locally Delaunay is the Delaunay triangulation; with the perturbation of the
// insertion predicates it is the unique one). One thread per slot; out[0] live finite
// tetrahedra, out[1] facets whose neighbour is not live or does not share them back, out[2]
// finite tetrahedra not positively oriented, out[3] facets whose neighbour's opposite vertex is
// in conflict with the tetrahedron (Section 2.6 for ghosts), out[4] distinct finite vertices.
__global__ void k_check(Ctx c, uint64_t nslots, uint8_t* seen, unsigned long long* out) {
  unsigned long long live = 0, bad_adj = 0, bad_orient = 0, bad_del = 0;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nslots;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const Tet T = load_tet(c.tets, (uint32_t)t);
    if (tet_dead(T.v)) continue;
    if (!tet_sane(c, T)) {
      bad_adj += 4;
      continue;
    }
    const bool finite = ghost_pos(T.v) < 0;
    if (finite) {
      ++live;
      PtF F[4];
      for (int k = 0; k < 4; ++k) {
        F[k] = load_ptf(c.ptf, get4(T.v, k));
        seen[get4(T.v, k)] = 1;
      }
      if (orient_replace(c, T.v, 0, T.v.x, F[0], F[0], F[1], F[2], F[3]) <= 0) ++bad_orient;
    }
    for (int i = 0; i < 4; ++i) {
      const uint32_t u = get4(T.n, i);
      const Tet U = load_tet(c.tets, u);
      const int k = tet_dead(U.v) ? -1 : back_facet(U.n, (uint32_t)t);
      bool same = k >= 0;
      for (int j = 0; j < 4 && same; ++j) {
        if (j == i) continue;
        const uint32_t x = get4(T.v, j);
        bool found = false;
        for (int m = 0; m < 4; ++m) found = found || (m != k && get4(U.v, m) == x);
        same = found;
      }
      if (!same) {
        ++bad_adj;
        continue;
      }
      const uint32_t q = get4(U.v, k);
      if (q == kGhost) continue;  // the vertex at infinity lies outside every finite sphere
      if (in_conflict(c, (uint32_t)t, q, load_ptf(c.ptf, q))) ++bad_del;
    }
  }
  if (live) atomicAdd(&out[0], live);
  if (bad_adj) atomicAdd(&out[1], bad_adj);
  if (bad_orient) atomicAdd(&out[2], bad_orient);
  if (bad_del) atomicAdd(&out[3], bad_del);
}

__global__ void k_count_seen(const uint8_t* seen, uint64_t n, unsigned long long* out) {
  unsigned long long m = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    m += seen[i];
  if (m) atomicAdd(out, m);
}

__global__ void k_split_keys(const uint4* tets, uint64_t T, uint64_t* khi, uint64_t* klo, uint32_t* idx) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint4 t = tets[i];
    khi[i] = ((uint64_t)t.x << 32) | t.y;
    klo[i] = ((uint64_t)t.z << 32) | t.w;
    idx[i] = (uint32_t)i;
  }
}

__global__ void k_gather_keys(const uint64_t* src, const uint32_t* idx, uint64_t T, uint64_t* dst) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
       i += (uint64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

__global__ void k_gather_tets(const uint4* src, const uint32_t* idx, uint64_t T, uint4* dst) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
       i += (uint64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

__global__ void k_eval_predicates(int kind, const double* pts, const int64_t* ids, int8_t* out, uint64_t n,
                                  DevState* st) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    Pt q[5];
    for (int k = 0; k < 5; ++k)
      q[k] = make_pt(pts[15 * i + 3 * k], pts[15 * i + 3 * k + 1], pts[15 * i + 3 * k + 2],
                          ids ? (double)ids[5 * i + k] : 0.0);
    int s;
    if (kind <= 2) {
      if (kind == 0) s = orient3d(q[0], q[1], q[2], q[3], st);
      else if (kind == 1) s = insphere(q[0], q[1], q[2], q[3], q[4], st);
      else s = insphere_sos(q[0], q[1], q[2], q[3], q[4], st);
    } else {
      // the kernels' pipeline: FP32 stage on the double-float copy, then FP64 + exact
      PtF f[5];
      double cm = 0.0;
      for (int k = 0; k < 5; ++k) {
        split_df(q[k].x, f[k].hx, f[k].lx);
        split_df(q[k].y, f[k].hy, f[k].ly);
        split_df(q[k].z, f[k].hz, f[k].lz);
        cm = fmax(cm, fmax(fabs(q[k].x), fmax(fabs(q[k].y), fabs(q[k].z))));
      }
      float eta = (float)(ldexp(cm, -44) * 1.0001 + 1e-38);
      if (kind == 3) {
        s = orient3d_f(f[0], f[1], f[2], f[3], eta);
        if (s == 0) s = orient3d(q[0], q[1], q[2], q[3], st);
      } else {
        s = insphere_f(f[0], f[1], f[2], f[3], f[4], eta);
        if (s == 0) s = insphere_sos(q[0], q[1], q[2], q[3], q[4], st);
      }
    }
    out[i] = (int8_t)s;
  }
}

// ------------------------------------------------------------------ learned scheduler
// Cell of a point on a 2^g-per-axis grid over the box, rounding each operation separately.
__device__ __forceinline__ void grid_cell(const Pt& P, const double* bb, int g, int q[3], double u[3]) {
  const double G = (double)(1 << g);
  const double c[3] = {P.x, P.y, P.z};
  for (int k = 0; k < 3; ++k) {
    double ext = bb[3 + k] - bb[k];
    double s = ext > 0.0 ? G / ext : 0.0;
    double f = floor(__dmul_rn(__dsub_rn(c[k], bb[k]), s));
    f = f < 0.0 ? 0.0 : (f > G - 1.0 ? G - 1.0 : f);
    q[k] = (int)f;
    double w = ext > 0.0 ? __ddiv_rn(__dsub_rn(c[k], bb[k]), ext) : 0.5;
    u[k] = w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
  }
}

// Points per cell of the grid (vertices [vb, vb + n), duplicates excluded).
__global__ void k_cell_count(const Pt* __restrict__ pts, const uint8_t* __restrict__ dup_of_input,
                             const uint32_t* __restrict__ perm, uint32_t vb, uint64_t n, const double* __restrict__ bb,
                             int g, uint32_t* count) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    if (dup_of_input[perm[s]]) continue;
    int q[3];
    double u[3];
    grid_cell(pts[vb + s], bb, g, q, u);
    atomicAdd(&count[((size_t)q[2] << (2 * g)) | ((size_t)q[1] << g) | (size_t)q[0]], 1u);
  }
}

// The eight features of every vertex of the call (see dt_get_features), x[s * 8 + k].
__global__ void k_features(const Pt* __restrict__ pts, uint32_t vb, uint64_t n, const double* __restrict__ bb, int g,
                           const uint32_t* __restrict__ count, const uint32_t* __restrict__ perm,
                           const uint64_t* __restrict__ keys, const uint8_t* __restrict__ rounds, float* x) {
  const int G = 1 << g;
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    int q[3];
    double u[3];
    grid_cell(pts[vb + s], bb, g, q, u);
    auto at = [&](int a, int b, int c) { return count[((size_t)c << (2 * g)) | ((size_t)b << g) | (size_t)a]; };
    const double nc = at(q[0], q[1], q[2]);
    double sum = 0.0, mx = -1.0, mn = 1e300;
    int k = 0;
    for (int d = 0; d < 3; ++d)
      for (int e = -1; e <= 1; e += 2) {
        int r[3] = {q[0], q[1], q[2]};
        r[d] += e;
        if (r[d] < 0 || r[d] >= G) continue;
        double v = at(r[0], r[1], r[2]);
        sum += v;
        mx = fmax(mx, v);
        mn = fmin(mn, v);
        ++k;
      }
    const double mean = k ? sum / k : nc;
    if (!k) mx = mn = nc;
    const uint32_t i = perm[s];
    const uint64_t key = keys[i];
    double f[8];
    f[0] = log2(1.0 + nc) / 8.0;
    f[1] = log2(1.0 + mean) / 8.0;
    f[2] = (log2(1.0 + mx) - log2(1.0 + mn)) / 8.0;
    f[3] = (nc - mean) / (1.0 + nc + mean);
    f[4] = (double)((key >> 57) & 63) / 64.0;
    f[5] = (double)((key >> 51) & 63) / 64.0;
    f[6] = (double)rounds[i] / 8.0;
    f[7] = 2.0 * fmin(fmin(fmin(u[0], 1.0 - u[0]), fmin(u[1], 1.0 - u[1])), fmin(u[2], 1.0 - u[2]));
    for (int j = 0; j < 8; ++j) x[s * 8 + j] = (float)f[j];
  }
}

// Labels of the call's vertices from the insertion log.
__global__ void k_labels(const uint16_t* __restrict__ log_nc, const uint8_t* __restrict__ log_lost, uint32_t vb,
                         uint64_t n, float* y, uint8_t* valid) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t nc = log_nc[vb + s];
    if (y) {
      y[2 * s] = log2f(1.f + (float)nc);
      y[2 * s + 1] = log_lost[vb + s] ? 1.f : 0.f;
    }
    if (valid) valid[s] = nc > 0 ? 1 : 0;
  }
}

// From the network's outputs: the points expected to lose a conflict (logit above logit_tau),
// and every point's claim rank, 255 - 32 log2(1 + predicted |C|) clamped to [0, 255], so that a
// point expected to have a small cavity wins against one expected to have a large cavity (each
// large cavity that wins knocks out every small one it overlaps).
__global__ void k_risky(const float* __restrict__ pred, uint64_t n, uint32_t vb, float logit_tau, float rank_scale,
                        uint8_t* risky, uint8_t* prank) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    risky[vb + s] = pred[2 * s + 1] > logit_tau ? 1 : 0;
    float r = rintf(255.f - rank_scale * pred[2 * s]);
    prank[vb + s] = (uint8_t)(r < 0.f ? 0.f : (r > 255.f ? 255.f : r));
  }
}

// Histogram of the 2 x (wave) sub-wave keys of a BRIO round.
// Predicted insertion work of each vertex (learned schedule): a fixed part for the walk, the
// locks and the ball, plus a quarter of the predicted cavity size |C| = 2^out0 - 1.
__global__ void k_work(const float* __restrict__ pred, uint64_t n, uint32_t vb, uint8_t* wcost) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n; s += (uint64_t)gridDim.x * blockDim.x) {
    const float c = exp2f(fminf(fmaxf(pred[2 * s], 0.f), 7.f)) - 1.f;
    wcost[vb + s] = (uint8_t)(4.f + rintf(c * 0.25f));
  }
}

__global__ void k_seg_cost(const uint32_t* __restrict__ q, uint32_t qbase, uint64_t m, const uint8_t* __restrict__ wcost,
                           uint32_t* out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = wcost[q ? q[i] : qbase + (uint32_t)i];
}

// bounds[w] = the first list position whose exclusive prefix of work reaches w / W of the total.
__global__ void k_seg_bounds(const uint32_t* __restrict__ prefix, const uint32_t* __restrict__ q, uint32_t qbase,
                             uint64_t m, const uint8_t* __restrict__ wcost, uint32_t W, uint32_t* bounds) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w > W) return;
  const uint64_t total = (uint64_t)prefix[m - 1] + wcost[q ? q[m - 1] : qbase + (uint32_t)(m - 1)];
  const uint64_t target = total * w / W;
  uint64_t lo = 0, hi = m;  // first i in [0, m] with prefix[i] >= target (prefix[m] = total)
  while (lo < hi) {
    const uint64_t mid = (lo + hi) / 2;
    if ((uint64_t)prefix[mid] >= target) hi = mid;
    else lo = mid + 1;
  }
  bounds[w] = (uint32_t)(w == W ? m : lo);
}

__global__ void k_key_hist(const uint64_t* __restrict__ keys, uint64_t m, uint32_t* hist) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[keys[i]], 1u);
}

unsigned grid_for(uint64_t n, int threads) {
  uint64_t b = (n + threads - 1) / threads;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 32));
}

int map_dev_error(unsigned e) {
  switch (e) {
    case kErrNone: return DT_OK;
    case kErrCapacity:
    case kErrFreeList: return DT_ENOMEM;
    case kErrDegenerate: return DT_EDEGENERATE;
    default: return DT_ELIMIT;
  }
}

}  // namespace
}  // namespace dtg

using namespace dtg;

// ------------------------------------------------------------------ handle
struct dt_handle {
  dt_config cfg{};
  cudaStream_t stream = nullptr;
  OrderWS ows;
  RefineWS rws;  // refinement iterations (dt_refine)
  Pt* pts = nullptr;
  PtF* ptf = nullptr;
  double cmax = 0.0;  // largest |coordinate| so far (sets the FP32 stage's eta)
  uint8_t* vflag = nullptr;
  uint32_t* point_hint = nullptr;
  uint64_t n_pts = 0, cap_pts = 0;
  Tet* tets = nullptr;
  unsigned long long* claim = nullptr;
  uint32_t* lock = nullptr;  // asynchronous engine: owner of each slot (0 = free)
  float4* subdet = nullptr;  // sub-determinant cache (ablation, DT_SUBDET=1): two float4 per slot
  double* in_buf = nullptr;    // dt_insert_host: the device copy of the host points, kept between calls
  uint64_t in_cap = 0;         // rows
  uint32_t* out_buf = nullptr; // dt_get_tets_host: the tetrahedra on the device before the copy out
  uint64_t out_cap = 0;        // rows
  bool use_subdet = false;
  uint64_t cap_tets = 0;
  uint32_t* freelist = nullptr;
  uint32_t* pending = nullptr;
  uint64_t cap_free = 0;
  uint32_t* cell_hint = nullptr;
  uint32_t* cell_hint2 = nullptr;
  int cb = 0, cell_hint_cb = -1;
  double lo[3] = {0, 0, 0}, sc[3] = {0, 0, 0};
  DevState* st = nullptr;
  DevState* st_host = nullptr;
  uint32_t Rmax = 0;
  uint32_t *cand_p = nullptr, *cand_t = nullptr, *cand_status = nullptr, *cand_nc = nullptr,
           *cand_nb = nullptr, *scratch = nullptr;
  uint32_t* queue[kNumQueues] = {};  // kQNext .. kQExact
  uint32_t* medscratch = nullptr;  // cavity lists of the shared-memory large rounds
  uint64_t cap_q = 0;
  char* bigmem = nullptr;   // kBigR large-cavity workspaces
  size_t bigstride = 0;
  char* hugemem = nullptr;  // the serial path's workspace
  uint32_t huge_c = 0;      // its cavity capacity (tetrahedra and boundary facets)
  char* ctamem = nullptr;   // the one-block engine's per-warp workspaces
  size_t ctastride = 0;
  BigWS hugews{};
  double* bbox_dev = nullptr;
  bool has_mesh = false;
  uint64_t last_n = 0;
  double alpha = 0.02;   // candidates per round = alpha * mesh vertices (measured best at 1e7 and 1e8)
  double alpha_refine = 0.01;  // the same during dt_refine
  double refine_rebuild = 0.25;  // dt_refine: rebuild the mesh when an iteration adds this share
  bool refine_rebuild_async = true;  // ... and let the rebuild use the asynchronous engine
  double gamma = 0.3;    // wave size = gamma * mesh vertices (round-based and batch engines)
  double gamma_async = 2.0;  // the asynchronous engine's waves (measured: 164.9 ms per 1e7 uniform
                             // step at 2.0 against 166.8 at 1.0, 175.0 at 0.5 and 185.6 at 0.3;
                             // 1e8: 1192 ms at 2.0 against 1264 at 1.0): fewer, longer launches
  double alpha_cta = 0.05; // candidates per round of the one-block engine per mesh vertex (at most 32)
  int walk_threads = 64;   // block size of the thread-per-point walk: small blocks spread a round over every SM
  bool use_async = true;   // waves and long retry lists run on the asynchronous engine (async.cu)
  double alpha_async = 0.05; // concurrent insertions (warps) per mesh vertex of the asynchronous engine
                             // (with its waves of 2x the mesh: 162.1 ms per 1e7 uniform step at 0.05,
                             // 164.9 at 0.1, 169.8 at 0.2; a lost attempt is cheap when nothing waits)
  uint64_t async_min_retry = 1;    // retry lists shorter than this use the round-based engine (1e7
                                   // uniform: 146 ms with every list on the asynchronous engine,
                                   // 147 with lists of 32 or more, 152 with 256, 155 with 2048); a
                                   // retry pass without progress moves the list to the rounds anyway
  uint64_t async_warps = 0;        // cap on the asynchronous engine's warps (0: all that fit)
  bool async_off = false;          // this call's inputs defeat the asynchronous engine's FP32 stage
  uint32_t async_ball_start = 1;   // start from the previous ball's tetrahedra before walking
  double async_handoff_frac = 0.2; // hand-offs per point of a pass that switch it off for the call
                                   // (degenerate mix: 42.8 Mtets/s at 0.2, 34.7 at 0.5; never
                                   // switching off sends points back and forth, 3.2)
  uint64_t async_handoff_min = 4096; // passes shorter than this never switch it off
  uint8_t* wcost = nullptr;        // learned schedule: predicted insertion work per vertex
  bool wcost_ready = false;
  uint32_t* seg_prefix = nullptr;  // prefix sums of a pass's predicted work
  uint64_t cap_seg = 0;
  uint32_t* seg_bounds = nullptr;  // the pass's segment starts
  uint64_t cap_wcost = 0;
  char* async_big_ws = nullptr;    // global-memory workspaces of the asynchronous large-cavity kernel
  char* async_borrow_ws = nullptr; // workspaces the main asynchronous kernel's warps borrow
  unsigned int* async_borrow_busy = nullptr;
  bool big_smem = true;    // large cavities try the shared-memory workspaces first
  int big_smem_skip = 0;   // passes left that go straight to the global-memory tier
  uint32_t* wlist = nullptr;
  uint32_t* wave_cum = nullptr;
  uint64_t cap_w = 0;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> prof_events;
  unsigned long long next_stamp = 1;
  unsigned long long launches0 = 0;
  dt_stats stats{};
  unsigned last_dev_error = 0, last_dev_info = 0;
  // batch of clouds (dt_batch)
  bool batch_mode = false;
  uint32_t n_clouds = 0;
  std::vector<uint64_t> boff;              // input offsets of the clouds
  std::vector<BatchCloud> bclouds_host;    // per-cloud ranges and results
  uint64_t* boff_dev = nullptr;
  BatchCloud* bclouds = nullptr;
  uint32_t* border = nullptr;               // clouds by decreasing size
  uint32_t* bsample = nullptr;              // the autotuner's sample of clouds
  uint64_t cap_bclouds = 0;
  uint32_t* bcid = nullptr;
  uint8_t* bdup = nullptr;                  // duplicate flags by vertex (sorted position)
  uint32_t *blist_a = nullptr, *blist_b = nullptr, *blist_big = nullptr;
  uint64_t cap_bpts = 0;
  uint32_t *bhint_f = nullptr, *bhint_c = nullptr;
  double* bcbox = nullptr;
  DevState* bstates = nullptr;
  uint64_t cap_bstates = 0;
  char* bws = nullptr;
  size_t cap_bws = 0;
  unsigned long long* bstats = nullptr;
  unsigned int* bnext = nullptr;
  int batch_W = 0;                          // autotuned block shape (warps per block), 0 = not tuned
  float batch_alpha = 0.f;                  // autotuned concurrent insertions per mesh vertex
  uint64_t batch_sig = 0;                   // workload signature the tuning belongs to
  double batch_tune_ms = 0.0;
  float* beta = nullptr;                    // device: the batch's FP32 error term
  cudaStream_t bs = nullptr;                // the handle's own stream for batches (capturable)
  cudaEvent_t bev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraph_t bgraph = nullptr;             // the captured steady-state batch
  cudaGraphExec_t bexec = nullptr;
  uint64_t bgraph_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  uint64_t bgraph_kernels = 0;              // kernels in the captured graph
  bool bgraph_used = false;                 // the last batch replayed the graph
  // learned scheduler
  uint16_t* log_nc = nullptr;               // DT_FLAG_LOG: |C| of each vertex's insertion
  uint8_t* log_lost = nullptr;              // DT_FLAG_LOG: conflicts each vertex lost
  uint64_t cap_log = 0;
  float* model = nullptr;                   // DT_MLP_PARAMS parameters (device)
  bool model_loaded = false;
  float* feat = nullptr;                    // features [n, 8] of the call being scheduled
  float* pred = nullptr;                    // network outputs [n, 2]
  uint64_t cap_feat = 0;
  uint32_t* cell_count = nullptr;
  uint64_t cap_cells = 0;
  uint8_t* risky = nullptr;                 // per vertex: expected to lose a conflict
  uint8_t* prank = nullptr;                 // per vertex: claim rank (smaller predicted cavity: higher)
  uint64_t cap_risky = 0;
  bool risky_ready = false;
  bool prank_ready = false;
  bool use_prank = true, use_defer = false;  // uses of the network's predictions (deferral measured slower)
  uint32_t* wave_hist = nullptr;            // sub-wave sizes
  double risky_scale = 0.25;                // concurrency of the expected losers, relative
  float risky_logit = 0.f;                  // logit threshold (0: probability one half)
  float rank_scale = 32.f;                  // claim rank steps per unit of predicted log2(1 + |C|)
  uint64_t last_base = 0;                   // the last dt_insert call's vertices
};

namespace {

template <class T>
cudaError_t grow(T*& p, uint64_t old_n, uint64_t new_n, cudaStream_t s) {
  T* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<uint64_t>(new_n, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (p && old_n) cudaMemcpyAsync(q, p, old_n * sizeof(T), cudaMemcpyDeviceToDevice, s);
  if (p) {
    cudaStreamSynchronize(s);
    cudaFree(p);
  }
  p = q;
  return cudaSuccess;
}

Ctx make_ctx(dt_handle* h) {
  Ctx c;
  c.tets = h->tets;
  c.claim = h->claim;
  c.pts = h->pts;
  c.ptf = h->ptf;
  // eta = 2^-44 max|x| plus the spacing of FP32 subnormals (see predicates.cuh)
  c.eta = (float)(std::ldexp(h->cmax, -44) * 1.0001 + 1e-38);
  c.freelist = h->freelist;
  c.pending = h->pending;
  c.cell_hint = h->cell_hint;
  c.cell_hint2 = h->cell_hint2;
  c.point_hint = h->point_hint;
  c.st = h->st;
  for (int k = 0; k < 3; ++k) {
    c.lo[k] = (float)h->lo[k];
    c.sc[k] = (float)h->sc[k];
  }
  c.cb = h->cb;
  // a walk that has not arrived after this many steps continues in the next pass, from where it
  // stopped, so one long walk does not hold up a whole round
  c.max_walk = h->cfg.max_walk_steps ? h->cfg.max_walk_steps : kDefaultWalk;
  c.coherent = 0;
  c.ntets = (uint32_t)h->cap_tets;
  c.npts = (uint32_t)h->cap_pts;
  c.subdet = h->use_subdet ? h->subdet : nullptr;
  return c;
}

InsertLog make_log(dt_handle* h) {
  const bool logging = (h->cfg.flags & DT_FLAG_LOG) && h->log_nc;
  return InsertLog{logging ? h->log_nc : nullptr, logging ? h->log_lost : nullptr};
}

// Device bytes the handle holds (its arrays at their current capacities; the batch and
// refinement workspaces are counted when they exist).
uint64_t device_bytes(const dt_handle* h) {
  uint64_t b = 0;
  b += h->cap_pts * (sizeof(Pt) + sizeof(PtF) + 1 + 4);             // points, FP32 copy, flag, hint
  b += h->cap_tets * (sizeof(Tet) + 16 + 4);                         // records, claim pair, owner word
  if (h->subdet) b += h->cap_tets * 2 * sizeof(float4);              // sub-determinant cache
  b += h->in_cap * 24 + h->out_cap * 16;                             // host entry points' buffers
  b += h->cap_free * 8;                                              // free list and pending
  if (h->cell_hint_cb > 0) {
    const int cb = h->cell_hint_cb, cbc = cb > 3 ? cb - 3 : 1;
    b += (4ull << (3 * cb)) + (4ull << (3 * cbc));
  }
  b += h->ows.cap * (8 + 8 + 8 + 4 + 4 + 1 + 1 + 4 + 4) + h->ows.hist_cap * 4;
  if (h->cand_p) {
    b += (uint64_t)h->Rmax * (5 * 4 + (uint64_t)kScratchStride * 4);
    b += h->bigstride * kBigR + (uint64_t)kBigR * (kMedCN + kMedFN) * 4 + h->ctastride * kCtaWarps;
  }
  b += h->cap_q * 4 * kNumQueues + h->cap_w * 4;
  if (h->async_big_ws) b += (uint64_t)kAsyncBigWarps * async_big_ws_bytes();
  if (h->async_borrow_ws) b += (uint64_t)kAsyncBorrow * (async_big_ws_bytes() + 4);
  if (h->hugemem) b += carve(nullptr, 4 * h->huge_c, h->huge_c, h->huge_c, 4 * h->huge_c, nullptr);
  b += h->cap_log * 3 + h->cap_feat * (8 + 2) * 4 + h->cap_risky * 2 + h->cap_cells * 4;
  b += h->cap_bpts * 32 + h->cap_bws + h->cap_bstates * sizeof(DevState);
  return b;
}

int sync_state(dt_handle* h) {
  if (cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return DT_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return DT_ECUDA;
  if (h->st_host->error) {
    h->last_dev_error = h->st_host->error;
    h->last_dev_info = h->st_host->error_info;
    return map_dev_error(h->st_host->error);
  }
  return DT_OK;
}

int reserve_points(dt_handle* h, uint64_t total) {
  if (total <= h->cap_pts) return DT_OK;
  uint64_t nc = std::max<uint64_t>(total, h->cap_pts + h->cap_pts / 2);
  if (grow(h->pts, h->n_pts, nc, h->stream) != cudaSuccess) return DT_ENOMEM;
  if (grow(h->ptf, h->n_pts, nc, h->stream) != cudaSuccess) return DT_ENOMEM;
  if (grow(h->vflag, h->n_pts, nc, h->stream) != cudaSuccess) return DT_ENOMEM;
  if (grow(h->point_hint, h->n_pts, nc, h->stream) != cudaSuccess) return DT_ENOMEM;
  h->cap_pts = nc;
  return DT_OK;
}

int reserve_tets(dt_handle* h, uint64_t total_pts) {
  double f = h->cfg.tet_capacity_factor > 0 ? h->cfg.tet_capacity_factor : 8.0;
  uint64_t need = (uint64_t)(f * (double)total_pts) + 4096;
  if (need > kMaxSlots) need = kMaxSlots;
  if (need <= h->cap_tets) return DT_OK;
  unsigned long long bump = h->has_mesh ? h->st_host->bump : 0;
  if (grow(h->tets, bump, need, h->stream) != cudaSuccess) return DT_ENOMEM;
  // slots not yet handed out read as dead (v.x == v.y == 0): the asynchronous engine may read
  // a slot through a freshly written pointer before its record arrives, and must never find an
  // old, self-consistent mesh there
  cudaMemsetAsync(h->tets + bump, 0, (need - bump) * sizeof(Tet), h->stream);
  if (grow(h->claim, 2 * bump, 2 * need, h->stream) != cudaSuccess) return DT_ENOMEM;
  // claim words of slots not yet handed out start at zero (below every priority)
  cudaMemsetAsync(h->claim + 2 * bump, 0, 2 * (need - bump) * sizeof(unsigned long long), h->stream);
  if (h->use_subdet) {
    // cache entries of slots not yet handed out read as invalid
    if (grow(h->subdet, 2 * bump, 2 * need, h->stream) != cudaSuccess) return DT_ENOMEM;
    cudaMemsetAsync(h->subdet + 2 * bump, 0, 2 * (need - bump) * sizeof(float4), h->stream);
  }
  // owner words: every slot free (no lock is held between launches)
  cudaStreamSynchronize(h->stream);
  cudaFree(h->lock);
  h->lock = nullptr;
  if (cudaMalloc(&h->lock, need * sizeof(uint32_t)) != cudaSuccess) return DT_ENOMEM;
  cudaMemsetAsync(h->lock, 0, need * sizeof(uint32_t), h->stream);
  // free list: the slots a round frees, plus every warp's private slots that the asynchronous
  // engine hands back when its launch ends
  uint64_t nf = need / 4 + 4096 + (uint64_t)async_max_warps() * 160;
  uint64_t fold = h->has_mesh ? h->st_host->free_avail : 0;
  if (grow(h->freelist, fold, nf, h->stream) != cudaSuccess) return DT_ENOMEM;
  cudaFree(h->pending);
  h->pending = nullptr;
  if (cudaMalloc(&h->pending, nf * 4) != cudaSuccess) return DT_ENOMEM;
  h->cap_tets = need;
  h->cap_free = nf;
  unsigned long long vals[2] = {need, nf};
  cudaMemcpyAsync(&h->st->capacity, &vals[0], 8, cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(&h->st->free_capacity, &vals[1], 8, cudaMemcpyHostToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  return DT_OK;
}

// The serial path's workspace: cavities of a quarter of the tetrahedron store, between kHugeC
// and kHugeCMax tetrahedra (visited-set and edge hashes four times that).
int reserve_huge(dt_handle* h) {
  uint64_t want = kHugeC;
  while (want < kHugeCMax && want < h->cap_tets / 4) want <<= 1;
  if (h->hugemem && want <= h->huge_c) return DT_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->hugemem);
  h->hugemem = nullptr;
  h->huge_c = 0;
  const uint32_t c = (uint32_t)want;
  size_t bytes = carve(nullptr, 4 * c, c, c, 4 * c, nullptr);
  if (cudaMalloc(&h->hugemem, bytes)) return DT_ENOMEM;
  carve(h->hugemem, 4 * c, c, c, 4 * c, &h->hugews);
  h->huge_c = c;
  return DT_OK;
}

int reserve_rounds(dt_handle* h, uint64_t qcap) {
  if (!h->cand_p) {
    h->Rmax = 1u << 19;
    uint64_t R = h->Rmax;
    if (cudaMalloc(&h->cand_p, R * 4) || cudaMalloc(&h->cand_t, R * 4) || cudaMalloc(&h->cand_status, R * 4) ||
        cudaMalloc(&h->cand_nc, R * 4) || cudaMalloc(&h->cand_nb, R * 4) ||
        cudaMalloc(&h->scratch, R * kScratchStride * 4))
      return DT_ENOMEM;
    h->bigstride = big_stride();
    if (cudaMalloc(&h->bigmem, h->bigstride * kBigR)) return DT_ENOMEM;
    if (cudaMalloc(&h->medscratch, (size_t)kBigR * (kMedCN + kMedFN) * 4)) return DT_ENOMEM;
    const int msmem = (int)(kMedWarps * med_stride());
    if (cudaFuncSetAttribute(k_cavity<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, msmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_insert<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, msmem) != cudaSuccess)
      return DT_ECUDA;
    h->ctastride = cta_stride();
    if (cudaMalloc(&h->ctamem, h->ctastride * kCtaWarps)) return DT_ENOMEM;
  }
  if (!h->wave_cum && cudaMalloc(&h->wave_cum, 256 * 4) != cudaSuccess) return DT_ENOMEM;
  if (!h->wave_hist && cudaMalloc(&h->wave_hist, 512 * 4) != cudaSuccess) return DT_ENOMEM;
  if (qcap > h->cap_w) {
    cudaFree(h->wlist);
    h->wlist = nullptr;
    if (cudaMalloc(&h->wlist, qcap * 4) != cudaSuccess) return DT_ENOMEM;
    h->cap_w = qcap;
  }
  if (qcap > h->cap_q) {
    for (auto& qb : h->queue) {
      cudaFree(qb);
      qb = nullptr;
      if (cudaMalloc(&qb, qcap * 4)) return DT_ENOMEM;
    }
    h->cap_q = qcap;
  }
  return DT_OK;
}

uint32_t choose_segments(dt_handle* h, uint64_t mesh_vertices, uint64_t m, float alpha_scale = 1.f) {
  if (h->cfg.segments) return (uint32_t)std::min<uint64_t>(std::min<uint64_t>(h->cfg.segments, h->Rmax), m);
  double r = h->alpha * alpha_scale * (double)mesh_vertices;
  uint64_t R = (uint64_t)std::max(1.0, r);
  R = std::min<uint64_t>(R, h->Rmax);
  R = std::min<uint64_t>(R, m);
  return (uint32_t)std::max<uint64_t>(R, 1);
}

// One concurrent insertion round: walk, cavity + claims, ball (+ closing the round).
// mode 0: a round of the shared-memory path; 1: large cavities with global-memory workspaces;
// 2: large cavities with shared-memory workspaces.
void launch_round(dt_handle* h, const Ctx& c, const RoundIO& io, int mode, uint64_t j_prof) {
  const bool prof = (h->cfg.flags & DT_FLAG_PROFILE) != 0 && mode == 0;
  cudaStream_t s = h->stream;
  uint32_t R = io.R;
  if (prof) cudaEventRecord(h->prof_events[6 * j_prof], s);
  const unsigned wt = (unsigned)h->walk_threads;
  k_walk<<<(R + wt - 1) / wt, wt, 0, s>>>(c, io, h->vflag, h->cand_p, h->cand_t, h->cand_status);
  ++g_kernel_launches;
  if (prof) {
    cudaEventRecord(h->prof_events[6 * j_prof + 1], s);
    cudaEventRecord(h->prof_events[6 * j_prof + 2], s);
  }
  const unsigned cblocks = (R + kCavWarps - 1) / kCavWarps;
  const unsigned iblocks = (R + kInsWarps - 1) / kInsWarps;
  const unsigned mblocks = (R + kMedWarps - 1) / kMedWarps;
  const size_t msmem = (size_t)kMedWarps * med_stride();
  if (mode == 1)
    k_cavity<1><<<cblocks, kCavWarps * 32, 0, s>>>(c, R, h->cand_p, h->cand_t, h->cand_status, h->cand_nc, h->cand_nb,
                                        h->scratch, h->bigmem, h->bigstride, io.prank);
  else if (mode == 2)
    k_cavity<2><<<mblocks, kMedWarps * 32, msmem, s>>>(c, R, h->cand_p, h->cand_t, h->cand_status, h->cand_nc,
                                                         h->cand_nb, h->medscratch, nullptr, 0, io.prank);
  else
    k_cavity<0><<<cblocks, kCavWarps * 32, 0, s>>>(c, R, h->cand_p, h->cand_t, h->cand_status, h->cand_nc, h->cand_nb,
                                        h->scratch, h->bigmem, h->bigstride, io.prank);
  ++g_kernel_launches;
  if (prof) {
    cudaEventRecord(h->prof_events[6 * j_prof + 3], s);
    cudaEventRecord(h->prof_events[6 * j_prof + 4], s);
  }
  if (mode == 1)
    k_insert<1><<<iblocks, kInsWarps * 32, 0, s>>>(c, io, h->cand_p, h->cand_status, h->cand_nc, h->cand_nb, h->scratch,
                                        h->bigmem, h->bigstride, make_log(h));
  else if (mode == 2)
    k_insert<2><<<mblocks, kMedWarps * 32, msmem, s>>>(c, io, h->cand_p, h->cand_status, h->cand_nc, h->cand_nb,
                                                         h->medscratch, nullptr, 0, make_log(h));
  else
    k_insert<0><<<iblocks, kInsWarps * 32, 0, s>>>(c, io, h->cand_p, h->cand_status, h->cand_nc, h->cand_nb, h->scratch,
                                        h->bigmem, h->bigstride, make_log(h));
  ++g_kernel_launches;
  if (prof) cudaEventRecord(h->prof_events[6 * j_prof + 5], s);
  h->stats.n_rounds++;
  if (mode != 0) h->stats.n_rounds_big++;
}

int set_queue_lengths(dt_handle* h, std::initializer_list<int> which) {
  unsigned long long zero = 0;
  for (int q : which)
    if (cudaMemcpyAsync(&h->st->q[q], &zero, 8, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) return DT_ECUDA;
  return DT_OK;
}

// Large cavities of a pass: rounds of up to kBigR candidates with global-memory workspaces
// (losers retry in the next such round), then the serial path for any larger ones.
int run_big(dt_handle* h, const Ctx& c) {
  // tier 1 (shared-memory workspaces): losers retry in the next tier-1 round, cavities that
  // outgrow the workspace move on to tier 2 (global memory), and from there to the serial path
  // when most of the recent large cavities outgrew the shared-memory workspaces (degenerate
  // inputs), skip that tier for a while instead of paying for two tiers
  const bool smem = h->big_smem && h->big_smem_skip == 0;
  if (h->big_smem_skip > 0) --h->big_smem_skip;
  const uint64_t listed = h->st_host->q[kQBig];
  for (int tier = smem ? 2 : 1; tier >= 1; --tier) {
    const int in_q = kQBig;
    const int out_q = tier == 2 ? kQBigG : kQHuge;
    if (tier == 2) {
      int rc = set_queue_lengths(h, {kQBigG});
      if (rc != DT_OK) return rc;
    } else if (smem) {
      // the cavities the shared-memory tier could not hold become the global tier's list
      std::swap(h->queue[kQBig], h->queue[kQBigG]);
      h->st_host->q[kQBig] = h->st_host->q[kQBigG];
      if (2 * h->st_host->q[kQBig] > listed) h->big_smem_skip = 8;
    }
    uint64_t nbig = h->st_host->q[in_q];
    int guard = 0;
    while (nbig > 0) {
      if (++guard > 100000) {
        h->last_dev_error = 101;  // host-side: large-cavity rounds stopped progressing
        h->last_dev_info = (unsigned)nbig;
        return DT_ELIMIT;
      }
      int rc = set_queue_lengths(h, {kQBig2});
      if (rc != DT_OK) return rc;
      uint32_t R = (uint32_t)std::min<uint64_t>(nbig, kBigR);
      uint64_t L = (nbig + R - 1) / R;
      for (uint64_t j = 0; j < L; ++j) {
        RoundIO io{h->queue[kQBig], 0, nbig, L, j, R, h->queue[kQBig2], kQBig2, h->queue[out_q], out_q,
                   h->prank_ready ? h->prank : nullptr};
        launch_round(h, c, io, tier == 2 ? 2 : 1, 0);
      }
      if ((rc = sync_state(h)) != DT_OK) return rc;
      nbig = h->st_host->q[kQBig2];
      std::swap(h->queue[kQBig], h->queue[kQBig2]);
    }
  }
  uint64_t nhuge = h->st_host->q[kQHuge];
  if (nhuge) {
    int rc = reserve_huge(h);
    if (rc != DT_OK) return rc;
    Ctx cc = c;
    cc.coherent = 1;
    k_huge<<<1, 32, 0, h->stream>>>(cc, h->queue[kQHuge], (uint32_t)nhuge, h->hugews, make_log(h));
    ++g_kernel_launches;
    rc = sync_state(h);
    if (rc != DT_OK) return rc;
  }
  return DT_OK;
}

// Large cavities of an asynchronous pass: the asynchronous kernel with global-memory
// workspaces, again on its losers while that makes progress; whatever is left (and cavities
// beyond those workspaces) goes through the large-cavity rounds and the serial path.
int run_big_async(dt_handle* h, const Ctx& c) {
  uint64_t nbig = h->st_host->q[kQBig];
  if (nbig > 0 && !h->async_big_ws &&
      cudaMalloc(&h->async_big_ws, (size_t)kAsyncBigWarps * async_big_ws_bytes()) != cudaSuccess)
    return DT_ENOMEM;
  for (int iter = 0; nbig > 0 && iter < 8; ++iter) {
    int rc = set_queue_lengths(h, {kQBig2});
    if (rc != DT_OK) return rc;
    uint64_t W = std::min<uint64_t>(nbig, kAsyncBigWarps);
    const uint64_t L = (nbig + W - 1) / W;
    W = (nbig + L - 1) / L;
    AsyncIO io{h->queue[kQBig], 0, nbig, L, (uint32_t)W, h->cfg.max_walk_steps ? h->cfg.max_walk_steps : kAsyncWalk,
               h->queue[kQBig2], kQBig2, h->queue[kQHuge], kQHuge, h->queue[kQExact], kQExact,
               nullptr, nullptr, nullptr, 0, h->async_ball_start};
    if ((rc = async_launch_big(c, io, h->lock, h->vflag, make_log(h), h->async_big_ws, h->stream)) != DT_OK)
      return rc;
    h->stats.n_async++;
    if ((rc = sync_state(h)) != DT_OK) return rc;
    const uint64_t left = h->st_host->q[kQBig2];
    std::swap(h->queue[kQBig], h->queue[kQBig2]);
    h->st_host->q[kQBig] = left;
    if (cudaMemcpyAsync(&h->st->q[kQBig], &left, 8, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return DT_ECUDA;
    if (left >= nbig) break;  // no progress: the rounds below settle the rest
    nbig = left;
  }
  return run_big(h, c);
}

// One pass: rounds over q[0..m) (or the vertex range qbase + [0, m)) split into R segments of
// length L (segment s offers q[s*L + j] in round j), then the large cavities of the pass.
int run_pass(dt_handle* h, const Ctx& c, const uint32_t* q, uint32_t qbase, uint64_t m, bool reset_next,
             float alpha_scale = 1.f, bool rounds_only = false);


int run_pass_async(dt_handle* h, const Ctx& c, const uint32_t* q, uint32_t qbase, uint64_t m, bool reset_next) {
  uint64_t mesh = h->st_host->n_inserted;
  uint64_t W = (uint64_t)std::max(1.0, h->alpha_async * (double)mesh);
  W = std::min<uint64_t>(W, h->async_warps ? h->async_warps : (uint64_t)async_max_warps());
  W = std::min<uint64_t>(W, m);
  const uint64_t L = (m + W - 1) / W;
  W = (m + L - 1) / L;
  int rc = reset_next ? set_queue_lengths(h, {kQNext, kQBig, kQHuge}) : set_queue_lengths(h, {kQBig, kQHuge});
  if (rc != DT_OK) return rc;
  if ((rc = set_queue_lengths(h, {kQExact})) != DT_OK) return rc;
  // learned schedule: segments of equal predicted work (a fixed part plus the predicted cavity)
  const uint32_t* seg_bounds = nullptr;
  if (h->wcost_ready && h->cfg.schedule == DT_SCHED_LEARNED) {
    if (m > h->cap_seg) {
      cudaFree(h->seg_prefix);
      h->seg_prefix = nullptr;
      if (cudaMalloc(&h->seg_prefix, m * 4) != cudaSuccess) return DT_ENOMEM;
      h->cap_seg = m;
    }
    if (!h->seg_bounds && cudaMalloc(&h->seg_bounds, ((size_t)async_max_warps() + 1) * 4) != cudaSuccess)
      return DT_ENOMEM;
    k_seg_cost<<<grid_for(m, 256), 256, 0, h->stream>>>(q, qbase, m, h->wcost, h->seg_prefix);
    prefix_sum_exclusive(h->seg_prefix, m, h->ows.hist, h->stream);
    k_seg_bounds<<<grid_for(W + 1, 256), 256, 0, h->stream>>>(h->seg_prefix, q, qbase, m, h->wcost, (uint32_t)W,
                                                               h->seg_bounds);
    g_kernel_launches += 2;
    seg_bounds = h->seg_bounds;
  }
  if (!h->async_borrow_ws) {
    if (cudaMalloc(&h->async_borrow_ws, (size_t)kAsyncBorrow * async_big_ws_bytes()) != cudaSuccess ||
        cudaMalloc(&h->async_borrow_busy, kAsyncBorrow * sizeof(unsigned int)) != cudaSuccess)
      return DT_ENOMEM;
    cudaMemsetAsync(h->async_borrow_busy, 0, kAsyncBorrow * sizeof(unsigned int), h->stream);
  }
  AsyncIO io{q, qbase, m, L, (uint32_t)W, h->cfg.max_walk_steps ? h->cfg.max_walk_steps : kAsyncWalk,
             h->queue[kQNext], kQNext, h->queue[kQBig], kQBig, h->queue[kQExact], kQExact,
             seg_bounds, h->async_borrow_ws, h->async_borrow_busy, kAsyncBorrow, h->async_ball_start};
  const bool prof = (h->cfg.flags & DT_FLAG_PROFILE) != 0;
  if (prof) cudaEventRecord(h->ev[3], h->stream);
  if ((rc = async_launch(c, io, h->lock, h->vflag, make_log(h), h->stream)) != DT_OK) return rc;
  if (prof) cudaEventRecord(h->ev[4], h->stream);
  h->stats.n_async++;
  h->stats.n_passes++;
  if ((rc = sync_state(h)) != DT_OK) return rc;
  if (prof) {
    float ms = 0;
    cudaEventElapsedTime(&ms, h->ev[3], h->ev[4]);
    h->stats.ms_async += ms;
  }
  // large cavities now (deferring them to the end of the BRIO round was measured slower: they
  // then meet each other, 592 instead of 395 rounds per 1e7 uniform step)
  if ((rc = run_big_async(h, c)) != DT_OK) return rc;
  // points whose predicates the asynchronous engine's FP32 stage could not decide: one
  // round-based pass with the full predicate cascade (its losers join the next pass's list)
  const uint64_t ne = h->st_host->q[kQExact];
  if (ne == 0) return DT_OK;
  h->stats.n_exact_handoff += ne;
  // when the FP32 stage cannot decide for a fifth of a pass's points (near-degenerate inputs:
  // lattices, co-spherical surfaces, refinement centres), the work it did was mostly wasted:
  // the rest of this call runs on the round-based engine. A short retry list says little about
  // the input (its points are the hard ones by selection), so it never decides this
  if (m >= h->async_handoff_min && (double)ne > h->async_handoff_frac * (double)m) h->async_off = true;
  return run_pass(h, c, h->queue[kQExact], 0, ne, false, 1.f, true);
}

int run_pass(dt_handle* h, const Ctx& c, const uint32_t* q, uint32_t qbase, uint64_t m, bool reset_next,
             float alpha_scale, bool rounds_only) {
  if (h->use_async && !h->async_off && !rounds_only && (!reset_next || m >= h->async_min_retry))
    return run_pass_async(h, c, q, qbase, m, reset_next);
  uint64_t& kind_rounds = reset_next ? h->stats.n_rounds_retry : h->stats.n_rounds_wave;
  uint64_t mesh = h->st_host->n_inserted;
  uint32_t R = choose_segments(h, mesh, m, alpha_scale);
  uint64_t L = (m + R - 1) / R;
  int rc = reset_next ? set_queue_lengths(h, {kQNext, kQBig, kQHuge}) : set_queue_lengths(h, {kQBig, kQHuge});
  if (rc != DT_OK) return rc;
  const bool prof = (h->cfg.flags & DT_FLAG_PROFILE) != 0;
  if (prof) {
    while (h->prof_events.size() < 6 * L) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return DT_ECUDA;
      h->prof_events.push_back(e);
    }
  }
  for (uint64_t j = 0; j < L; ++j) {
    RoundIO io{q, qbase, m, L, j, R, h->queue[kQNext], kQNext, h->queue[kQBig], kQBig,
               h->prank_ready ? h->prank : nullptr};
    launch_round(h, c, io, 0, j);
  }
  kind_rounds += L;
  h->stats.n_passes++;
  if ((rc = sync_state(h)) != DT_OK) return rc;
  if (cudaGetLastError() != cudaSuccess) return DT_ECUDA;
  if (prof) {
    for (uint64_t j = 0; j < L; ++j) {
      float a = 0, b = 0, cc = 0;
      cudaEventElapsedTime(&a, h->prof_events[6 * j], h->prof_events[6 * j + 1]);
      cudaEventElapsedTime(&b, h->prof_events[6 * j + 2], h->prof_events[6 * j + 3]);
      cudaEventElapsedTime(&cc, h->prof_events[6 * j + 4], h->prof_events[6 * j + 5]);
      h->stats.ms_walk += a;
      h->stats.ms_cavity += b;
      h->stats.ms_insert_k += cc;
      h->stats.n_profiled++;
    }
  }
  // large cavities of the pass: inserting them now keeps the remaining neighbourhoods small
  return run_big(h, c);
}

// Waves of one BRIO round (see run_brio_round): fills h->wlist with the round's vertices grouped
// by wave, Moore order inside each wave, h->wave_cum with the cumulative wave ends, and returns
// the number of waves.
int make_waves(dt_handle* h, uint32_t vbegin, uint32_t vend, int round, uint64_t base, std::vector<uint32_t>& cum,
               std::vector<float>* scale = nullptr) {
  cudaStream_t s = h->stream;
  uint64_t m = vend - vbegin;
  cum.clear();
  double N = (double)std::max<uint64_t>(h->st_host->n_inserted, 4);
  uint64_t acc = 0;
  while (acc < m && cum.size() < 255) {
    const double gamma = (h->use_async && !h->async_off) ? h->gamma_async : h->gamma;
    uint64_t w = (uint64_t)std::max(1.0, std::ceil(gamma * N));
    acc = std::min<uint64_t>(m, acc + w);
    cum.push_back((uint32_t)acc);
    N += (double)w;
  }
  cum.back() = (uint32_t)m;
  if (cudaMemcpyAsync(h->wave_cum, cum.data(), cum.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return -1;
  uint64_t rank0 = round == 0 ? 0 : brio_round_end(round - 1);
  // learned schedule: every wave splits into the points expected to win, then those expected to
  // lose (inserted with less concurrency)
  const bool split = scale && h->risky_ready;
  k_wave_keys<<<grid_for(m, 256), 256, 0, s>>>(vbegin, m, base, rank0, h->ows.perm, h->ows.rank, h->wave_cum,
                                                (int)cum.size(), split ? h->risky : nullptr, h->ows.k0, h->ows.v0);
  ++g_kernel_launches;
  if (split) {
    const int nk = 2 * (int)cum.size();
    cudaMemsetAsync(h->wave_hist, 0, nk * 4, s);
    k_key_hist<<<grid_for(m, 256), 256, 0, s>>>(h->ows.k0, m, h->wave_hist);
    ++g_kernel_launches;
    std::vector<uint32_t> hist(nk);
    cudaMemcpyAsync(hist.data(), h->wave_hist, nk * 4, cudaMemcpyDeviceToHost, s);
    bool alt = radix_sort_pairs(h->ows.k0, h->ows.v0, h->ows.k1, h->ows.v1, m, 16, h->ows.hist, s);
    cudaMemcpyAsync(h->wlist, alt ? h->ows.v1 : h->ows.v0, m * 4, cudaMemcpyDeviceToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    cum.clear();
    scale->clear();
    uint64_t end = 0;
    for (int k = 0; k < nk; ++k) {
      if (hist[k] == 0) continue;
      end += hist[k];
      cum.push_back((uint32_t)end);
      scale->push_back((k & 1) ? (float)h->risky_scale : 1.f);
    }
    return (int)cum.size();
  }
  if (scale) scale->assign(cum.size(), 1.f);
  bool alt = radix_sort_pairs(h->ows.k0, h->ows.v0, h->ows.k1, h->ows.v1, m, 8, h->ows.hist, s);
  cudaMemcpyAsync(h->wlist, alt ? h->ows.v1 : h->ows.v0, m * 4, cudaMemcpyDeviceToDevice, s);
  return (int)cum.size();
}

// The first BRIO round of a new triangulation on one thread block (see k_cta_insert).
int run_cta_round(dt_handle* h, uint32_t vbegin, uint32_t vend, uint64_t base) {
  Ctx c = make_ctx(h);
  Ctx cc = c;
  cc.coherent = 1;
  int rc = set_queue_lengths(h, {kQBig, kQHuge});
  if (rc != DT_OK) return rc;
  std::vector<uint32_t> cum;
  int nw = make_waves(h, vbegin, vend, 0, base, cum);
  if (nw < 0) return DT_ECUDA;
  cudaEventRecord(h->ev[3], h->stream);
  k_cta_insert<<<1, kCtaWarps * 32, 0, h->stream>>>(cc, h->wlist, h->wave_cum, nw, h->vflag, h->queue[kQNext],
                                                     h->queue[kQBig2], h->queue[kQHuge], h->ctamem, h->ctastride,
                                                     (float)h->alpha_cta, 1u << 16, make_log(h));
  ++g_kernel_launches;
  cudaEventRecord(h->ev[4], h->stream);
  h->stats.n_passes++;
  if ((rc = sync_state(h)) != DT_OK) return rc;
  float ms = 0;
  cudaEventElapsedTime(&ms, h->ev[3], h->ev[4]);
  h->stats.ms_first_round = ms;
  return run_big(h, c);
}

// Inserts the vertices [vbegin, vend) (BRIO round `round`, Moore order). The round is split
// into waves of about gamma * (mesh size) points, each a uniformly random subset kept in
// Moore order, so the number of concurrent insertions can follow the mesh as it grows. Points
// that lose a conflict are retried after the last wave, re-keyed with a re-partition
// transform (Section 3.3) until none is left.
int run_brio_round(dt_handle* h, uint32_t vbegin, uint32_t vend, int round, uint64_t base) {
  Ctx c = make_ctx(h);
  cudaStream_t s = h->stream;
  uint32_t max_rounds = h->cfg.max_rounds ? h->cfg.max_rounds : (1u << 22);
  std::vector<uint32_t> cum;
  std::vector<float> scale;
  if (make_waves(h, vbegin, vend, round, base, cum, &scale) < 0) return DT_ECUDA;
  int rc = set_queue_lengths(h, {kQNext});
  if (rc != DT_OK) return rc;
  uint64_t off = 0;
  for (size_t w = 0; w < cum.size(); ++w) {
    if ((rc = run_pass(h, c, h->wlist + off, 0, cum[w] - off, false, scale[w])) != DT_OK) return rc;
    off = cum[w];
  }
  uint64_t nq = h->st_host->q[kQNext];
  uint32_t pass = 0;
  int stalled = 0;
  while (nq > 0) {
    if (h->stats.n_rounds > max_rounds) {
      h->last_dev_error = 103;  // host-side: round budget exhausted
      return DT_ELIMIT;
    }
    uint64_t before = nq, limited = h->st_host->n_walk_limit;
    transformed_keys(h->pts, h->queue[kQNext], nq, h->bbox_dev, h->cfg.seed + 0x51ED2701ull * (pass + 1) + vbegin,
                     h->ows.k0, h->ows.v0, s);
    // the top 24 bits of the 63-bit key (8 levels of the curve) order the retries well enough
    bool a2 = radix_sort_pairs_bits(h->ows.k0, h->ows.v0, h->ows.k1, h->ows.v1, nq, 39, 63, h->ows.hist, s);
    // a short retry list is cheap per round: let its walks run long instead of over many passes
    Ctx cr = c;
    if (!h->cfg.max_walk_steps && nq < kLongWalkBelow) cr.max_walk = kLongWalkSteps;
    // after a pass that made no progress the round-based engine takes over: its highest-priority
    // located point always wins, where the asynchronous engine's retries might keep colliding
    if ((rc = run_pass(h, cr, a2 ? h->ows.v1 : h->ows.v0, 0, nq, true, 1.f, stalled > 0)) != DT_OK) return rc;
    nq = h->st_host->q[kQNext];
    // every pass shrinks the retry list (its highest-priority located point is inserted, or
    // moves to the large-cavity queue) or advances walks that hit their step limit; three
    // passes that do neither are a bug, not a schedule
    bool walking = h->st_host->n_walk_limit > limited;
    stalled = (nq >= before && !walking) ? stalled + 1 : 0;
    if (stalled >= 3) {
      h->last_dev_error = 102;  // host-side: retry passes stopped progressing
      h->last_dev_info = (unsigned)((nq << 8) | (pass & 255));
      return DT_ELIMIT;
    }
    ++pass;
  }
  return DT_OK;
}

int schedule_learned(dt_handle* h, uint64_t n);

int insert_impl(dt_handle* h, const double* xyz, uint64_t n, bool allow_async = true) {
  if (n == 0) return h->has_mesh ? DT_OK : DT_EDEGENERATE;
  h->async_off = !allow_async;
  if (h->n_pts + n >= 0xFFFFFFF0ull) return DT_EINVAL;
  cudaStream_t s = h->stream;
  cudaEventRecord(h->ev[0], s);
  int rc = order_points(xyz, n, h->cfg.seed, h->ows, s);
  if (rc != DT_OK) return rc;
  cudaEventRecord(h->ev[1], s);
  uint64_t base = h->n_pts;
  if ((rc = reserve_points(h, base + n)) != DT_OK) return rc;
  if ((rc = reserve_tets(h, base + n)) != DT_OK) return rc;
  if ((rc = reserve_rounds(h, n + 1024)) != DT_OK) return rc;
  k_build_pts<<<grid_for(n, 256), 256, 0, s>>>(xyz, h->ows.perm, h->ows.dup, n, base, h->pts, h->ptf,
                                                h->vflag, h->point_hint);
  ++g_kernel_launches;
  h->last_base = base;
  h->risky_ready = false;
  h->prank_ready = false;
  h->wcost_ready = false;
  if (h->cfg.flags & DT_FLAG_LOG) {
    if (h->cap_pts > h->cap_log) {
      uint16_t* a = nullptr;
      uint8_t* b = nullptr;
      if (cudaMalloc(&a, h->cap_pts * 2) != cudaSuccess || cudaMalloc(&b, h->cap_pts) != cudaSuccess) {
        cudaFree(a);
        return DT_ENOMEM;
      }
      if (base) {
        cudaMemcpyAsync(a, h->log_nc, base * 2, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(b, h->log_lost, base, cudaMemcpyDeviceToDevice, s);
      }
      cudaStreamSynchronize(s);
      cudaFree(h->log_nc);
      cudaFree(h->log_lost);
      h->log_nc = a;
      h->log_lost = b;
      h->cap_log = h->cap_pts;
    }
    cudaMemsetAsync(h->log_nc + base, 0, n * 2, s);
    cudaMemsetAsync(h->log_lost + base, 0, n, s);
  }
  if (h->cfg.schedule == DT_SCHED_LEARNED) {
    if (!h->model_loaded) return DT_ESTATE;
    if ((rc = schedule_learned(h, n)) != DT_OK) return rc;
  }
  double bb[6];
  if (cudaMemcpyAsync(bb, h->ows.bbox, 48, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DT_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;
  for (int k = 0; k < 6; ++k) h->cmax = std::max(h->cmax, std::fabs(bb[k]));
  if (!h->has_mesh) {
    if (!h->bbox_dev && cudaMalloc(&h->bbox_dev, 48) != cudaSuccess) return DT_ENOMEM;
    cudaMemcpyAsync(h->bbox_dev, h->ows.bbox, 48, cudaMemcpyDeviceToDevice, s);
    // hint grid: about 8 points per cell, at most 2^24 cells
    int cb = 1;
    while (cb < 8 && (1ull << (3 * (cb + 1))) * 8ull <= n) ++cb;
    h->cb = cb;
    for (int k = 0; k < 3; ++k) {
      h->lo[k] = bb[k];
      double ext = bb[3 + k] - bb[k];
      h->sc[k] = ext > 0 ? (double)(1u << cb) / ext : 0.0;
    }
    int cbc = cb > 3 ? cb - 3 : 1;
    if (h->cell_hint_cb != cb) {
      cudaFree(h->cell_hint);
      cudaFree(h->cell_hint2);
      h->cell_hint = h->cell_hint2 = nullptr;
      if (cudaMalloc(&h->cell_hint, (size_t)4 << (3 * cb)) != cudaSuccess) return DT_ENOMEM;
      if (cudaMalloc(&h->cell_hint2, (size_t)4 << (3 * cbc)) != cudaSuccess) return DT_ENOMEM;
      h->cell_hint_cb = cb;
    }
    cudaMemsetAsync(h->cell_hint, 0xFF, (size_t)4 << (3 * cb), s);
    cudaMemsetAsync(h->cell_hint2, 0xFF, (size_t)4 << (3 * cbc), s);
    // a new mesh: every slot reads as dead until it is handed out (see reserve_tets)
    cudaMemsetAsync(h->tets, 0, h->cap_tets * sizeof(Tet), s);
    if (h->subdet) cudaMemsetAsync(h->subdet, 0, 2 * h->cap_tets * sizeof(float4), s);
    DevState z{};
    z.stamp = h->next_stamp;
    z.capacity = h->cap_tets;
    z.free_capacity = h->cap_free;
    z.anchor = 0;
    std::memcpy(h->st_host, &z, sizeof(z));
    cudaMemcpyAsync(h->st, &z, sizeof(z), cudaMemcpyHostToDevice, s);
    Ctx c = make_ctx(h);
    k_init<<<1, 32, 0, s>>>(c, (uint32_t)base, (uint32_t)(base + n), h->vflag);
    ++g_kernel_launches;
    if ((rc = sync_state(h)) != DT_OK) return rc;
    h->has_mesh = true;
  }
  for (int r = 0;; ++r) {
    uint64_t b = r == 0 ? 0 : brio_round_end(r - 1);
    if (b >= n) break;
    uint64_t e = std::min<uint64_t>(brio_round_end(r), n);
    // the first BRIO round of a new triangulation: the asynchronous engine in waves (measured
    // faster: 181.7 against 197.6 ms per 1e7 uniform step, 31 against 41 ms at 1e5), or the
    // one-block engine when the round-based engine runs alone
    if (r == 0 && h->st_host->n_inserted <= 4 && (!h->use_async || std::getenv("DT_CTA")) && !std::getenv("DT_NO_CTA"))
      rc = run_cta_round(h, (uint32_t)(base + b), (uint32_t)(base + e), base);
    else
      rc = run_brio_round(h, (uint32_t)(base + b), (uint32_t)(base + e), r, base);
    if (rc != DT_OK) return rc;
  }
  cudaEventRecord(h->ev[2], s);
  if ((rc = sync_state(h)) != DT_OK) return rc;
  float ms_sort = 0, ms_ins = 0;
  cudaEventElapsedTime(&ms_sort, h->ev[0], h->ev[1]);
  cudaEventElapsedTime(&ms_ins, h->ev[1], h->ev[2]);
  h->stats.ms_sort = ms_sort;
  h->stats.ms_insert = ms_ins;
  h->n_pts = base + n;
  h->last_n = n;
  return DT_OK;
}

// ------------------------------------------------------------------ batches of clouds
template <class T>
bool realloc_dev(T*& p, uint64_t n) {
  cudaFree(p);
  p = nullptr;
  return cudaMalloc(&p, std::max<uint64_t>(n, 1) * sizeof(T)) == cudaSuccess;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  return n;
}

// Device memory of a batch of nc clouds, N points and T tetrahedron slots (in total).
int batch_reserve(dt_handle* h, uint64_t N, uint32_t nc, uint64_t T) {
  if (reserve_points(h, N) != DT_OK) return DT_ENOMEM;
  if (order_ws_reserve(h->ows, N) != cudaSuccess) return DT_ENOMEM;
  if (N > h->cap_bpts) {
    if (!realloc_dev(h->bcid, N) || !realloc_dev(h->bdup, N) || !realloc_dev(h->blist_a, N) ||
        !realloc_dev(h->blist_b, N) || !realloc_dev(h->blist_big, N))
      return DT_ENOMEM;
    h->cap_bpts = N;
  }
  if (nc > h->cap_bclouds) {
    if (!realloc_dev(h->boff_dev, (uint64_t)nc + 1) || !realloc_dev(h->bclouds, nc) || !realloc_dev(h->border, nc) ||
        !realloc_dev(h->bsample, nc) || !realloc_dev(h->bhint_f, (uint64_t)nc * batch_hint_fine()) ||
        !realloc_dev(h->bhint_c, (uint64_t)nc * batch_hint_coarse()) || !realloc_dev(h->bcbox, 6ull * nc))
      return DT_ENOMEM;
    h->cap_bclouds = nc;
  }
  if (T > h->cap_tets) {
    if (!realloc_dev(h->tets, T) || !realloc_dev(h->claim, 2 * T)) return DT_ENOMEM;
    h->cap_tets = T;
  }
  if (T > h->cap_free) {
    if (!realloc_dev(h->freelist, T) || !realloc_dev(h->pending, T)) return DT_ENOMEM;
    h->cap_free = T;
  }
  if (!h->bstats && (!realloc_dev(h->bstats, kBatchStatSlots) || !realloc_dev(h->bnext, 1))) return DT_ENOMEM;
  // workspaces and states for the largest grid of any block shape
  int shapes[8];
  int ns = batch_shapes(shapes, 8);
  uint64_t states = 0;
  size_t ws = 0;
  const int sms = sm_count();
  for (int i = 0; i < ns; ++i) {
    uint64_t blocks = (uint64_t)std::max(1, batch_blocks_per_sm(shapes[i])) * sms;
    states = std::max(states, blocks);
    ws = std::max(ws, (size_t)blocks * (shapes[i] & 255) * batch_ws_stride());
  }
  if (states > h->cap_bstates) {
    if (!realloc_dev(h->bstates, states)) return DT_ENOMEM;
    cudaMemsetAsync(h->bstates, 0, states * sizeof(DevState), h->stream);
    h->cap_bstates = states;
  }
  if (ws > h->cap_bws) {
    if (!realloc_dev(h->bws, ws)) return DT_ENOMEM;
    h->cap_bws = ws;
  }
  return DT_OK;
}

Ctx batch_ctx(dt_handle* h) {
  Ctx c = make_ctx(h);
  c.coherent = 1;  // a block reads back the tetrahedra it writes
  c.max_walk = h->cfg.max_walk_steps ? h->cfg.max_walk_steps : kDefaultWalk;
  c.subdet = nullptr;  // the batch store has no cache
  return c;
}

// Batched S1..S4, the vertex records and the per-cloud hint grids: enqueued on the batch stream,
// no host synchronisation.
void batch_enqueue_prepare(dt_handle* h, const double* xyz, cudaStream_t s) {
  const uint64_t N = h->boff[h->n_clouds];
  cudaMemsetAsync(h->ows.bad, 0, 4, s);
  order_batch(xyz, N, h->boff_dev, h->n_clouds, h->cfg.seed, h->gamma, h->ows, h->bcid, h->bcbox, s);
  k_build_pts<<<grid_for(N, 256), 256, 0, s>>>(xyz, h->ows.perm, h->ows.dup, N, 0, h->pts, h->ptf, h->vflag,
                                                h->point_hint);
  ++g_kernel_launches;
  cudaMemcpyAsync(h->bdup, h->vflag, N, cudaMemcpyDeviceToDevice, s);
  batch_prepare(h->bclouds, h->bcbox, h->n_clouds, h->beta, s);
}

// Reset of the clouds and the persistent launch over order[0 .. n) with block shape W.
int batch_enqueue_insert(dt_handle* h, int W, float alpha, const uint32_t* order, uint32_t n, bool reset_all,
                         cudaStream_t s) {
  batch_reset(h->bclouds, reset_all ? nullptr : order, reset_all ? h->n_clouds : n, h->claim, h->bhint_f, h->bhint_c,
              h->bdup, h->vflag, h->point_hint, s);
  cudaMemsetAsync(h->bnext, 0, 4, s);
  cudaMemsetAsync(h->bstats, 0, kBatchStatSlots * 8, s);
  const unsigned blocks = (unsigned)std::max(1, batch_blocks_per_sm(W)) * (unsigned)sm_count();
  return batch_launch(W, std::min<unsigned>(blocks, n), batch_ctx(h), h->bclouds, order, n, h->bnext, h->vflag,
                      h->blist_a, h->blist_b, h->blist_big, h->bhint_f, h->bhint_c, h->bstates, h->bws,
                      batch_ws_stride(), alpha, h->gamma, h->beta, h->bstats, s);
}

// One timed launch over order[0 .. n) (the autotuner's trials); device ms, or < 0 on failure.
float batch_run(dt_handle* h, int W, float alpha, const uint32_t* order, uint32_t n, bool reset_all) {
  cudaStream_t s = h->bs;
  cudaEventRecord(h->bev[2], s);
  int rc = batch_enqueue_insert(h, W, alpha, order, n, reset_all, s);
  cudaEventRecord(h->bev[3], s);
  if (rc != DT_OK || cudaStreamSynchronize(s) != cudaSuccess) return -1.f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->bev[2], h->bev[3]);
  return ms;
}

// Autotuner: block shape (warps per block) and round size (concurrent insertions per mesh
// vertex) timed on a sample of the clouds spread over the size order; the fastest is kept for
// batches with the same signature (cloud count and size range).
int batch_tune(dt_handle* h, const std::vector<uint32_t>& by_size, uint64_t sig) {
  const uint32_t nc = h->n_clouds;
  // DT_BATCH_WARPS / DT_BATCH_ALPHA restrict the candidates (warps per block; round size)
  const char* fw = std::getenv("DT_BATCH_WARPS");
  const char* fa = std::getenv("DT_BATCH_ALPHA");
  h->batch_tune_ms = 0.0;
  // the sample: every k-th cloud of the size order, a quarter of the batch (at least enough to
  // fill the GPU several times), so that the trials see the batch's tail as well as its bulk
  const uint32_t want = std::min<uint32_t>(nc, std::max<uint32_t>(8u * (uint32_t)sm_count(), nc / 4));
  const uint32_t step = std::max<uint32_t>(1, nc / std::max<uint32_t>(want, 1));
  std::vector<uint32_t> sample;
  for (uint32_t k = 0; k < nc && sample.size() < want; k += step) sample.push_back(by_size[k]);
  if (cudaMemcpyAsync(h->bsample, sample.data(), sample.size() * 4, cudaMemcpyHostToDevice, h->bs) != cudaSuccess)
    return DT_ECUDA;
  int shapes[8];
  int ns = batch_shapes(shapes, 8);
  if (const char* fs = std::getenv("DT_BATCH_SHAPE")) {  // one exact shape: warps | (min blocks << 8)
    shapes[0] = std::atoi(fs);
    ns = 1;
  }
  std::vector<float> alphas = {0.1f, 0.3f};
  if (fa) alphas = {(float)std::atof(fa)};
  float best = -1.f;
  auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < ns; ++i) {
    if (fw && std::atoi(fw) != (shapes[i] & 255)) continue;
    for (float a : alphas) {
      float ms = batch_run(h, shapes[i], a, h->bsample, (uint32_t)sample.size(), false);
      if (ms < 0.f) return DT_ECUDA;
      if (best < 0.f || ms < best) {
        best = ms;
        h->batch_W = shapes[i];
        h->batch_alpha = a;
      }
    }
  }
  h->batch_tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->batch_sig = sig;
  return h->batch_W ? DT_OK : DT_ELIMIT;
}

int batch_impl(dt_handle* h, const double* xyz, const uint64_t* off, uint32_t nc) {
  const uint64_t N = off[nc];
  double f = h->cfg.tet_capacity_factor > 0 ? h->cfg.tet_capacity_factor : 8.0;
  // slots per cloud: f per point plus room for the first tetrahedra and ghosts
  std::vector<BatchCloud> cl(nc);
  uint64_t T = 0, hash = 1469598103934665603ull;
  for (uint32_t c = 0; c < nc; ++c) {
    uint64_t n = off[c + 1] - off[c];
    uint64_t cap = (uint64_t)(f * (double)n) + 64;
    cl[c] = BatchCloud{};
    cl[c].vb = (uint32_t)off[c];
    cl[c].ve = (uint32_t)off[c + 1];
    cl[c].tb = (uint32_t)T;
    cl[c].tcap = (uint32_t)cap;
    T += cap;
    hash = (hash ^ n) * 1099511628211ull;
  }
  if (T > kMaxSlots) return DT_ENOMEM;
  int rc = batch_reserve(h, N, nc, T);
  if (rc != DT_OK) return rc;
  if (!h->bs) {
    if (cudaStreamCreateWithFlags(&h->bs, cudaStreamNonBlocking) != cudaSuccess) return DT_ECUDA;
    for (auto& e : h->bev)
      if (cudaEventCreate(&e) != cudaSuccess) return DT_ECUDA;
    if (cudaMalloc(&h->beta, sizeof(float)) != cudaSuccess) return DT_ENOMEM;
  }
  cudaStream_t s = h->bs;
  // the batch stream starts after the caller's stream has produced the input
  cudaEventRecord(h->bev[0], h->stream);
  cudaStreamWaitEvent(s, h->bev[0], 0);
  h->n_clouds = nc;
  h->boff.assign(off, off + nc + 1);
  std::vector<uint32_t> by_size(nc);
  for (uint32_t c = 0; c < nc; ++c) by_size[c] = c;
  std::stable_sort(by_size.begin(), by_size.end(), [&](uint32_t a, uint32_t b) {
    return off[a + 1] - off[a] > off[b + 1] - off[b];
  });
  if (cudaMemcpyAsync(h->boff_dev, off, (nc + 1) * 8ull, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(h->bclouds, cl.data(), nc * sizeof(BatchCloud), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(h->border, by_size.data(), nc * 4ull, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DT_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;  // host vectors go out of scope
  h->n_pts = N;
  h->batch_mode = true;
  unsigned int bad = 0;
  // the autotuner needs the ordered points: prepare once eagerly, then time the candidates
  uint64_t big = off[by_size[0] + 1] - off[by_size[0]];
  uint64_t sig = ((uint64_t)nc << 40) ^ ((uint64_t)(64 - __builtin_clzll(N | 1)) << 32) ^
                 (uint64_t)(64 - __builtin_clzll(big | 1));
  const bool fixed = std::getenv("DT_BATCH_WARPS") || std::getenv("DT_BATCH_ALPHA") || std::getenv("DT_BATCH_SHAPE");
  if (fixed || !h->batch_W || h->batch_sig != sig) {
    batch_enqueue_prepare(h, xyz, s);
    cudaMemcpyAsync(&bad, h->ows.bad, 4, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;
    if (bad) return DT_EINVAL;
    if ((rc = batch_tune(h, by_size, sig)) != DT_OK) return rc;
  } else {
    h->batch_tune_ms = 0.0;
  }
  // the steady state: sort, records, reset and the persistent launch, replayed from a CUDA graph
  // while the batch keeps its shape (same input buffer, cloud sizes, block shape and round size)
  const uint64_t key[8] = {(uint64_t)(uintptr_t)xyz, N, nc, hash, (uint64_t)h->batch_W,
                           (uint64_t)(h->batch_alpha * 1e6f), h->cfg.seed, (uint64_t)(h->gamma * 1e9)};
  const bool use_graph = !std::getenv("DT_BATCH_NO_GRAPH");
  h->bgraph_used = false;
  if (use_graph && !(h->bexec && std::equal(key, key + 8, h->bgraph_key))) {
    if (h->bexec) cudaGraphExecDestroy(h->bexec);
    if (h->bgraph) cudaGraphDestroy(h->bgraph);
    h->bexec = nullptr;
    h->bgraph = nullptr;
    unsigned long long k0 = g_kernel_launches;
    bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      // external records: the graph itself records the events, so every replay is timed
      cudaEventRecordWithFlags(h->bev[1], s, cudaEventRecordExternal);
      batch_enqueue_prepare(h, xyz, s);
      cudaEventRecordWithFlags(h->bev[2], s, cudaEventRecordExternal);
      int rl = batch_enqueue_insert(h, h->batch_W, h->batch_alpha, h->border, nc, true, s);
      cudaEventRecordWithFlags(h->bev[3], s, cudaEventRecordExternal);
      ok = cudaStreamEndCapture(s, &h->bgraph) == cudaSuccess && rl == DT_OK;
    }
    if (ok) ok = cudaGraphInstantiate(&h->bexec, h->bgraph, 0) == cudaSuccess;
    if (ok) {
      std::copy(key, key + 8, h->bgraph_key);
      h->bgraph_kernels = g_kernel_launches - k0;
    } else {
      cudaGetLastError();  // capture unsupported here: run the same sequence eagerly
      if (h->bgraph) cudaGraphDestroy(h->bgraph);
      h->bgraph = nullptr;
      h->bexec = nullptr;
    }
    g_kernel_launches = k0;
  }
  if (use_graph && h->bexec) {
    if (cudaGraphLaunch(h->bexec, s) != cudaSuccess) return DT_ECUDA;
    g_kernel_launches += h->bgraph_kernels;
    h->bgraph_used = true;
  } else {
    cudaEventRecord(h->bev[1], s);
    batch_enqueue_prepare(h, xyz, s);
    cudaEventRecord(h->bev[2], s);
    if ((rc = batch_enqueue_insert(h, h->batch_W, h->batch_alpha, h->border, nc, true, s)) != DT_OK) return rc;
    cudaEventRecord(h->bev[3], s);
  }
  // results: per-cloud status and sizes, and the batch counters
  h->bclouds_host.resize(nc);
  unsigned long long st[kBatchStatSlots];
  cudaMemcpyAsync(&bad, h->ows.bad, 4, cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(h->bclouds_host.data(), h->bclouds, nc * sizeof(BatchCloud), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(st, h->bstats, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;
  if (bad) return DT_EINVAL;
  float ms_sort = 0.f, ms_ins = 0.f;
  if (cudaEventElapsedTime(&ms_sort, h->bev[1], h->bev[2]) != cudaSuccess) ms_sort = 0.f;
  if (cudaEventElapsedTime(&ms_ins, h->bev[2], h->bev[3]) != cudaSuccess) ms_ins = 0.f;
  cudaGetLastError();
  DevState agg{};
  uint64_t degenerate = 0, used = 0;
  for (const BatchCloud& b : h->bclouds_host) {
    used += b.used;
    if (b.status == kErrDegenerate) {
      ++degenerate;
    } else if (b.status != 0 && h->last_dev_error == 0) {
      h->last_dev_error = b.status;
      h->last_dev_info = b.info;
    }
  }
  agg.n_inserted = st[0];
  agg.n_conflicts = st[1];
  agg.n_attempts = st[2];
  agg.sum_cavity = st[3];
  agg.sum_ball = st[4];
  agg.sum_walk = st[5];
  agg.n_big = st[7];
  agg.n_exact = st[9];
  agg.n_sos = st[10];
  agg.bump = used;
  std::memcpy(h->st_host, &agg, sizeof(agg));
  h->stats.ms_sort = ms_sort;
  h->stats.ms_insert = ms_ins;
  h->stats.n_rounds = st[8];
  h->stats.n_passes = 0;
  h->stats.n_clouds_degenerate = degenerate;
  h->stats.batch_warps = (uint64_t)(h->batch_W & 255);
  h->stats.batch_min_blocks = (uint64_t)(h->batch_W >> 8);
  h->stats.batch_alpha = h->batch_alpha;
  h->stats.ms_batch_tune = h->batch_tune_ms;
  h->stats.batch_graph = h->bgraph_used ? 1 : 0;
  // DT_EDEGENERATE only when no cloud could be triangulated
  if (h->last_dev_error) return map_dev_error(h->last_dev_error);
  return degenerate == nc ? DT_EDEGENERATE : DT_OK;
}

// Finite tetrahedra of a batch, grouped by cloud (cloud-local ids).
int batch_get_tets(dt_handle* h, uint32_t* tets_dev, uint64_t cap, uint64_t* n_tets, uint64_t* cloud_offsets,
                   int canonical) {
  cudaStream_t s = h->stream;
  const uint32_t nc = h->n_clouds;
  unsigned long long *counts = nullptr, *ooff = nullptr;
  if (cudaMalloc(&counts, nc * 8ull) != cudaSuccess) return DT_ENOMEM;
  if (cudaMalloc(&ooff, (nc + 1) * 8ull) != cudaSuccess) {
    cudaFree(counts);
    return DT_ENOMEM;
  }
  cudaMemsetAsync(counts, 0, nc * 8ull, s);
  batch_collect(h->bclouds, nc, h->tets, h->pts, h->boff_dev, 0, counts, nullptr, nullptr, canonical, s);
  std::vector<unsigned long long> cnt(nc), oo(nc + 1, 0);
  cudaMemcpyAsync(cnt.data(), counts, nc * 8ull, cudaMemcpyDeviceToHost, s);
  int rc = cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
  for (uint32_t c = 0; c < nc; ++c) oo[c + 1] = oo[c] + cnt[c];
  const uint64_t T = oo[nc];
  *n_tets = T;
  h->stats.n_tets = T;
  if (cloud_offsets)
    for (uint32_t c = 0; c <= nc; ++c) cloud_offsets[c] = oo[c];
  if (rc == DT_OK && T > cap) rc = DT_ETOOSMALL;
  // the sorted list needs the unsorted one first; otherwise the rows go straight to the output
  const bool sort = canonical && !(h->cfg.flags & DT_FLAG_NO_CANONICAL_SORT) && T > 1;
  uint32_t* tmp = nullptr;
  if (rc == DT_OK && sort && cudaMalloc(&tmp, T * 16) != cudaSuccess) rc = DT_ENOMEM;
  if (rc == DT_OK && T > 0) {
    cudaMemcpyAsync(ooff, oo.data(), (nc + 1) * 8ull, cudaMemcpyHostToDevice, s);
    batch_collect(h->bclouds, nc, h->tets, h->pts, h->boff_dev, 1, counts, ooff, sort ? tmp : tets_dev, canonical, s);
    if (sort) {
      // lexicographic by (cloud, a, b, c, d): LSD passes on (c, d), then (a, b), then the cloud
      uint64_t *khi = nullptr, *klo = nullptr, *kcl = nullptr, *ka = nullptr;
      uint32_t *idx = nullptr, *ia = nullptr, *hist = nullptr;
      bool ok = cudaMalloc(&khi, T * 8) == cudaSuccess && cudaMalloc(&klo, T * 8) == cudaSuccess &&
                cudaMalloc(&kcl, T * 8) == cudaSuccess && cudaMalloc(&ka, T * 8) == cudaSuccess &&
                cudaMalloc(&idx, T * 4) == cudaSuccess && cudaMalloc(&ia, T * 4) == cudaSuccess &&
                cudaMalloc(&hist, radix_hist_entries(T) * 4) == cudaSuccess;
      if (ok) {
        int cbits = 8;
        while (cbits < 32 && (1ull << cbits) < nc) cbits += 8;
        batch_tet_keys(tmp, T, ooff, nc, khi, klo, kcl, idx, s);
        bool alt = radix_sort_pairs(klo, idx, ka, ia, T, 64, hist, s);
        uint32_t* order = alt ? ia : idx;
        uint32_t* other = alt ? idx : ia;
        k_gather_keys<<<grid_for(T, 256), 256, 0, s>>>(khi, order, T, ka);
        ++g_kernel_launches;
        bool alt2 = radix_sort_pairs(ka, order, klo, other, T, 64, hist, s);
        uint32_t* order2 = alt2 ? other : order;
        uint32_t* other2 = alt2 ? order : other;
        k_gather_keys<<<grid_for(T, 256), 256, 0, s>>>(kcl, order2, T, ka);
        ++g_kernel_launches;
        bool alt3 = radix_sort_pairs_bits(ka, order2, klo, other2, T, 0, cbits, hist, s);
        k_gather_tets<<<grid_for(T, 256), 256, 0, s>>>((const uint4*)tmp, alt3 ? other2 : order2, T,
                                                       (uint4*)tets_dev);
        ++g_kernel_launches;
      } else {
        rc = DT_ENOMEM;
      }
      cudaFree(khi);
      cudaFree(klo);
      cudaFree(kcl);
      cudaFree(ka);
      cudaFree(idx);
      cudaFree(ia);
      cudaFree(hist);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = DT_ECUDA;
  }
  cudaFree(tmp);
  cudaFree(counts);
  cudaFree(ooff);
  return rc;
}


// ------------------------------------------------------------------ learned scheduler (host)
// Feature grid bits: about four points per cell, at most 2^24 cells.
int feature_grid_bits(uint64_t n) {
  int g = 1;
  while (g < 8 && (1ull << (3 * (g + 1))) * 4ull <= n) ++g;
  return g;
}

// Features of the n vertices of the last call into h->feat (grows the buffers).
int compute_features(dt_handle* h, uint64_t n) {
  cudaStream_t s = h->stream;
  if (n > h->cap_feat) {
    if (!realloc_dev(h->feat, n * 8) || !realloc_dev(h->pred, n * 2)) return DT_ENOMEM;
    h->cap_feat = n;
  }
  const int g = feature_grid_bits(n);
  const uint64_t cells = 1ull << (3 * g);
  if (cells > h->cap_cells) {
    if (!realloc_dev(h->cell_count, cells)) return DT_ENOMEM;
    h->cap_cells = cells;
  }
  cudaMemsetAsync(h->cell_count, 0, cells * 4, s);
  const uint32_t vb = (uint32_t)h->last_base;
  k_cell_count<<<grid_for(n, 256), 256, 0, s>>>(h->pts, h->ows.dup, h->ows.perm, vb, n, h->ows.bbox, g, h->cell_count);
  k_features<<<grid_for(n, 256), 256, 0, s>>>(h->pts, vb, n, h->ows.bbox, g, h->cell_count, h->ows.perm, h->ows.keys,
                                              h->ows.rounds, h->feat);
  g_kernel_launches += 2;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

// Learned schedule of the call: features, the network, and the expected losers' flags.
int schedule_learned(dt_handle* h, uint64_t n) {
  int rc = compute_features(h, n);
  if (rc != DT_OK) return rc;
  if (h->last_base + n > h->cap_risky) {
    uint8_t *r = nullptr, *k = nullptr;
    if (cudaMalloc(&r, h->cap_pts) != cudaSuccess || cudaMalloc(&k, h->cap_pts) != cudaSuccess) {
      cudaFree(r);
      return DT_ENOMEM;
    }
    if (h->risky && h->last_base) {
      cudaMemcpyAsync(r, h->risky, h->last_base, cudaMemcpyDeviceToDevice, h->stream);
      cudaMemcpyAsync(k, h->prank, h->last_base, cudaMemcpyDeviceToDevice, h->stream);
    }
    cudaStreamSynchronize(h->stream);
    cudaFree(h->risky);
    cudaFree(h->prank);
    h->risky = r;
    h->prank = k;
    h->cap_risky = h->cap_pts;
  }
  if ((rc = mlp_forward(h->model, h->feat, n, h->pred, h->stream)) != DT_OK) return rc;
  k_risky<<<grid_for(n, 256), 256, 0, h->stream>>>(h->pred, n, (uint32_t)h->last_base,
                                                    h->use_defer ? h->risky_logit : 1e30f, h->rank_scale, h->risky,
                                                    h->prank);
  ++g_kernel_launches;
  if (h->last_base + n > h->cap_wcost) {
    uint8_t* wc = nullptr;
    if (cudaMalloc(&wc, h->cap_pts) != cudaSuccess) return DT_ENOMEM;
    if (h->wcost && h->last_base) cudaMemcpyAsync(wc, h->wcost, h->last_base, cudaMemcpyDeviceToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    cudaFree(h->wcost);
    h->wcost = wc;
    h->cap_wcost = h->cap_pts;
  }
  k_work<<<grid_for(n, 256), 256, 0, h->stream>>>(h->pred, n, (uint32_t)h->last_base, h->wcost);
  ++g_kernel_launches;
  h->wcost_ready = true;
  h->risky_ready = h->use_defer;
  h->prank_ready = h->use_prank;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

void fill_stats(dt_handle* h, dt_stats* o) {
  *o = h->stats;
  o->n_launches = g_kernel_launches - h->launches0;
  o->device_error = h->last_dev_error;
  o->device_error_info = h->last_dev_info;
  const DevState& d = *h->st_host;
  o->n_points = h->n_pts;
  o->n_unique = d.n_inserted;
  o->n_dups = h->n_pts - d.n_inserted;
  o->n_slots = d.bump;
  o->n_attempts = d.n_attempts;
  o->n_conflicts = d.n_conflicts;
  o->n_big = d.n_big;
  o->sum_cavity = d.sum_cavity;
  o->sum_ball = d.sum_ball;
  o->sum_walk = d.sum_walk;
  o->n_exact = d.n_exact;
  o->n_sos = d.n_sos;
  o->n_walk_limit = d.n_walk_limit;
  o->free_slots = d.free_avail;
  o->max_walk = d.max_walk;
  o->n_restarts = d.n_restart;
  o->n_inserted_async = d.n_inserted_async;
  o->device_bytes = device_bytes(h);
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int dt_create(dt_handle** out, const dt_config* cfg) {
  if (!out) return DT_EINVAL;
  *out = nullptr;
  if (cfg) {
    for (uint32_t r : cfg->reserved)
      if (r) return DT_EINVAL;
    if (cfg->schedule > DT_SCHED_LEARNED || cfg->tet_capacity_factor < 0) return DT_EINVAL;
  }
  dt_handle* h = new (std::nothrow) dt_handle();
  if (!h) return DT_ENOMEM;
  if (cfg) h->cfg = *cfg;
  h->stream = (cudaStream_t)h->cfg.stream;
  if (const char* a = std::getenv("DT_ALPHA")) h->alpha = std::atof(a);
  if (const char* a = std::getenv("DT_ALPHA_REFINE")) h->alpha_refine = std::atof(a);
  if (const char* a = std::getenv("DT_REFINE_REBUILD")) h->refine_rebuild = std::atof(a);
  if (const char* a = std::getenv("DT_REFINE_REBUILD_ASYNC")) h->refine_rebuild_async = std::atoi(a) != 0;
  if (const char* g = std::getenv("DT_GAMMA")) h->gamma = std::atof(g);
  if (const char* g = std::getenv("DT_GAMMA_ASYNC")) h->gamma_async = std::atof(g);
  if (const char* a = std::getenv("DT_ALPHA_CTA")) h->alpha_cta = std::atof(a);
  if (const char* b = std::getenv("DT_BIG_SMEM")) h->big_smem = std::atoi(b) != 0;
  if (const char* a = std::getenv("DT_ASYNC")) h->use_async = std::atoi(a) != 0;
  if (const char* a = std::getenv("DT_ALPHA_ASYNC")) h->alpha_async = std::atof(a);
  if (const char* a = std::getenv("DT_ASYNC_MIN_RETRY")) h->async_min_retry = std::strtoull(a, nullptr, 10);
  if (const char* a = std::getenv("DT_ASYNC_WARPS")) h->async_warps = std::strtoull(a, nullptr, 10);
  if (const char* a = std::getenv("DT_ASYNC_HANDOFF")) h->async_handoff_frac = std::atof(a);
  if (const char* a = std::getenv("DT_ASYNC_HANDOFF_MIN")) h->async_handoff_min = std::strtoull(a, nullptr, 10);
  if (const char* a = std::getenv("DT_SUBDET")) h->use_subdet = std::atoi(a) != 0;
  if (const char* a = std::getenv("DT_ASYNC_BALL_START")) h->async_ball_start = (uint32_t)std::atoi(a);
  if (const char* w = std::getenv("DT_WALK_THREADS")) {
    int v = std::atoi(w);
    if (v == 32 || v == 64 || v == 128 || v == 256) h->walk_threads = v;
  }
  bool ok = cudaMalloc(&h->st, sizeof(DevState)) == cudaSuccess &&
            cudaMallocHost(&h->st_host, sizeof(DevState)) == cudaSuccess;
  for (auto& e : h->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  if (!ok) {
    dt_destroy(h);
    return DT_ENOMEM;
  }
  std::memset(h->st_host, 0, sizeof(DevState));
  cudaMemset(h->st, 0, sizeof(DevState));
  h->launches0 = g_kernel_launches;
  *out = h;
  return DT_OK;
}

int clear_mesh(dt_handle* h, bool keep_stats);

int dt_clear(dt_handle* h) {
  if (!h) return DT_EINVAL;
  return clear_mesh(h, false);
}

int clear_mesh(dt_handle* h, bool keep_stats) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  // claim priorities keep growing across triangulations, so stale claims never win
  unsigned long long s = h->has_mesh ? h->st_host->stamp : 0;
  h->next_stamp = std::max(h->next_stamp, s + 1);
  h->has_mesh = false;
  if (h->next_stamp > (1ull << 23) && h->claim) {
    // claim priorities hold the stamp in 24 bits: start over from clear claim words
    if (cudaMemsetAsync(h->claim, 0, 2 * h->cap_tets * sizeof(unsigned long long), h->stream) != cudaSuccess)
      return DT_ECUDA;
    h->next_stamp = 1;
  }
  if (h->batch_mode) {
    // a batch restarts its claim stamps in every cloud: clear the words before anything else
    if (h->claim && cudaMemsetAsync(h->claim, 0, 2 * h->cap_tets * sizeof(unsigned long long), h->stream) != cudaSuccess)
      return DT_ECUDA;
    h->batch_mode = false;
    h->n_clouds = 0;
  }
  h->n_pts = 0;
  h->last_n = 0;
  h->cmax = 0.0;
  h->last_dev_error = h->last_dev_info = 0;
  if (!keep_stats) {
    h->stats = dt_stats{};
    h->launches0 = g_kernel_launches;
  }
  std::memset(h->st_host, 0, sizeof(DevState));
  return cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_insert(dt_handle* h, const double* xyz_dev, uint64_t n) {
  if (!h || (n > 0 && !xyz_dev)) return DT_EINVAL;
  if (h->batch_mode) return DT_ESTATE;
  return insert_impl(h, xyz_dev, n);
}

// The mesh of every point the handle holds plus ns more (device, [ns, 3]), built from scratch:
// the points keep their input indices, so the triangulation (unique under the perturbation) is
// the one inserting the ns points into the current mesh would give. An iteration of dt_refine
// that adds many points into a mesh whose interior is empty meets cavities of thousands of
// tetrahedra; in BRIO order over all points the cavities stay small.
int rebuild_with(dt_handle* h, const double* extra, uint64_t ns, bool allow_async) {
  const uint64_t n0 = h->n_pts, N = n0 + ns;
  double* all = nullptr;
  if (cudaMalloc(&all, N * 24) != cudaSuccess) return DT_ENOMEM;
  int rc = points_out(h->pts, n0, all, n0, h->stream);
  if (rc == DT_OK &&
      cudaMemcpyAsync(all + 3 * n0, extra, ns * 24, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
    rc = DT_ECUDA;
  if (rc == DT_OK) rc = clear_mesh(h, true);
  if (rc == DT_OK) rc = insert_impl(h, all, N, allow_async);
  cudaStreamSynchronize(h->stream);
  cudaFree(all);
  return rc;
}

int dt_refine(dt_handle* h, double size, double ratio, double spacing, const double* box_host, uint32_t max_iters,
              uint64_t* n_added, uint32_t* n_iters) {
  if (n_added) *n_added = 0;
  if (n_iters) *n_iters = 0;
  if (!h || !box_host) return DT_EINVAL;
  if (!(size > 0.0) || !(ratio > 0.0) || !(spacing > 0.0) || !std::isfinite(size * ratio) ||
      !std::isfinite(size * spacing))
    return DT_EINVAL;
  RefineParams p{};
  double ext = 0.0;
  for (int k = 0; k < 3; ++k) {
    p.lo[k] = box_host[k];
    p.hi[k] = box_host[3 + k];
    if (!std::isfinite(p.lo[k]) || !std::isfinite(p.hi[k]) || !(p.lo[k] < p.hi[k])) return DT_EINVAL;
    ext = std::max(ext, p.hi[k] - p.lo[k]);
  }
  if (h->batch_mode || !h->has_mesh) return DT_ESTATE;
  p.thr_r2 = (ratio * size) * (ratio * size);
  p.thr_d2 = (spacing * size) * (spacing * size);
  // filter cells a little wider than spacing * size: a pair closer than that is in neighbouring cells
  p.inv_cell = 1.0 / (spacing * size * (1.0 + 1e-6));
  const double g = std::floor(ext * p.inv_cell) + 2.0;
  if (!(g < (double)(1u << 21))) return DT_EINVAL;
  p.G = (uint32_t)g;
  p.bits = 1;
  while ((1u << p.bits) < p.G) ++p.bits;
  uint64_t added = 0;
  uint32_t iters = 0;
  int rc = DT_OK;
  // the first iterations put every new point into the sparse interior while the concurrency
  // follows the whole (mostly surface) mesh: fewer candidates per vertex collide less
  // (measured 10 % faster at 0.01 than at the default 0.02 on the 1/128 box)
  const double alpha_keep = h->alpha;
  h->alpha = h->alpha_refine;
  while (iters < max_iters) {
    if ((rc = sync_state(h)) != DT_OK) break;
    uint64_t m = 0, ns = 0;
    if ((rc = refine_step(h->rws, h->tets, h->st_host->bump, h->pts, h->n_pts, p, &m, &ns, h->stream)) != DT_OK) break;
    if (ns == 0) break;
    // refinement centres lie almost on the spheres of their neighbours and the first iterations
    // fill an empty interior (cavities of thousands of tetrahedra): the round-based engine,
    // with its full predicate cascade and large-cavity tiers, is faster here (5.9 s against
    // 10.9 s for the 1/128 box)
    // a rebuild pays for the whole mesh again (the boundary points' degenerate predicates
    // included) but keeps every cavity small; inserting a quarter of the mesh's points or more
    // into it measured slower than rebuilding at every iteration of the 1/128 box (requiring
    // also as many new points as refinement had added so far: 1.90 s against 1.75 s)
    if (h->refine_rebuild > 0 && (double)ns >= h->refine_rebuild * (double)h->n_pts) {
      h->alpha = alpha_keep;  // a rebuild is a plain insertion of the whole set
      rc = rebuild_with(h, h->rws.xyz, ns, h->refine_rebuild_async);
      h->alpha = h->alpha_refine;
    }
    else
      rc = insert_impl(h, h->rws.xyz, ns, false);
    if (rc != DT_OK) break;
    added += ns;
    ++iters;
  }
  h->alpha = alpha_keep;
  if (n_added) *n_added = added;
  if (n_iters) *n_iters = iters;
  return rc;
}

int dt_get_points(dt_handle* h, double* xyz_dev, uint64_t rows, uint64_t* n_points) {
  if (!h || (rows > 0 && !xyz_dev)) return DT_EINVAL;
  if (h->batch_mode) return DT_ESTATE;
  if (n_points) *n_points = h->n_pts;
  if (rows == 0) return DT_OK;
  int rc = points_out(h->pts, h->n_pts, xyz_dev, rows, h->stream);
  if (rc != DT_OK) return rc;
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_check(dt_handle* h, uint64_t* out_host) {
  if (!h || !out_host) return DT_EINVAL;
  for (int k = 0; k < 5; ++k) out_host[k] = 0;
  if (h->batch_mode) return DT_ESTATE;
  if (!h->has_mesh) return DT_OK;
  cudaStream_t s = h->stream;
  int rc = sync_state(h);
  if (rc != DT_OK) return rc;
  const uint64_t slots = h->st_host->bump;
  // the predicates count their exact calls and report errors through a DevState: a scratch one
  // keeps the handle's statistics those of its insertions
  char* mem = nullptr;
  const size_t off_out = (sizeof(DevState) + 15) & ~size_t(15), off_seen = off_out + 64;
  if (cudaMalloc(&mem, off_seen + std::max<uint64_t>(h->n_pts, 1)) != cudaSuccess) return DT_ENOMEM;
  cudaMemsetAsync(mem, 0, off_seen + h->n_pts, s);
  Ctx c = make_ctx(h);
  c.st = reinterpret_cast<DevState*>(mem);
  unsigned long long* out = reinterpret_cast<unsigned long long*>(mem + off_out);
  uint8_t* seen = reinterpret_cast<uint8_t*>(mem + off_seen);
  if (slots) {
    k_check<<<grid_for(slots, 256), 256, 0, s>>>(c, slots, seen, out);
    k_count_seen<<<grid_for(h->n_pts, 256), 256, 0, s>>>(seen, h->n_pts, out + 4);
    g_kernel_launches += 2;
  }
  unsigned long long r[5] = {0, 0, 0, 0, 0};
  unsigned int err = 0;
  cudaMemcpyAsync(r, out, sizeof(r), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&err, &c.st->error, 4, cudaMemcpyDeviceToHost, s);
  rc = cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
  cudaFree(mem);
  if (rc != DT_OK) return rc;
  for (int k = 0; k < 5; ++k) out_host[k] = r[k];
  if (err != 0) {
    h->last_dev_error = err;
    return map_dev_error(err);
  }
  return DT_OK;
}

int dt_insert_host(dt_handle* h, const double* xyz_host, uint64_t n) {
  if (!h || (n > 0 && !xyz_host)) return DT_EINVAL;
  if (h->batch_mode) return DT_ESTATE;
  // the device copy lives in a buffer the handle keeps, so a call allocates only when it grows
  if (n > h->in_cap) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->in_buf);
    h->in_buf = nullptr;
    h->in_cap = 0;
    if (cudaMalloc(&h->in_buf, n * 24) != cudaSuccess) return DT_ENOMEM;
    h->in_cap = n;
  }
  if (n && cudaMemcpyAsync(h->in_buf, xyz_host, n * 24, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return DT_ECUDA;
  int rc = insert_impl(h, h->in_buf, n);
  cudaStreamSynchronize(h->stream);
  return rc;
}

int dt_batch(dt_handle* h, const double* xyz_dev, const uint64_t* offsets_host, uint32_t n_clouds) {
  if (!h || !offsets_host || n_clouds == 0 || offsets_host[0] != 0) return DT_EINVAL;
  for (uint32_t c = 0; c < n_clouds; ++c)
    if (offsets_host[c + 1] < offsets_host[c]) return DT_EINVAL;
  const uint64_t N = offsets_host[n_clouds];
  if (N == 0 || !xyz_dev || N >= 0xFFFFFFF0ull) return DT_EINVAL;
  int rc = dt_clear(h);
  if (rc != DT_OK) return rc;
  rc = batch_impl(h, xyz_dev, offsets_host, n_clouds);
  if (rc != DT_OK && rc != DT_EDEGENERATE && h->last_dev_error == 0) h->last_dev_error = 0;
  return rc;
}

int dt_get_tets(dt_handle* h, uint32_t* tets_dev, uint64_t cap, uint64_t* n_tets, uint64_t* cloud_offsets,
                int canonical) {
  if (!h || !n_tets || (cap > 0 && !tets_dev)) return DT_EINVAL;
  *n_tets = 0;
  if (cap > 0) {
    // page-locked host memory is accepted too, through its mapped device address
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, tets_dev) == cudaSuccess) {
      if (at.type == cudaMemoryTypeUnregistered) return DT_EINVAL;  // pageable host memory
      if (at.type == cudaMemoryTypeHost) {
        if (!at.devicePointer) return DT_EINVAL;
        tets_dev = static_cast<uint32_t*>(at.devicePointer);
      }
    }
    cudaGetLastError();  // an unknown pointer leaves an error behind; it is not one
  }
  if (h->batch_mode) return batch_get_tets(h, tets_dev, cap, n_tets, cloud_offsets, canonical);
  if (!h->has_mesh) return DT_OK;
  cudaStream_t s = h->stream;
  int rc = sync_state(h);
  if (rc != DT_OK) return rc;
  uint64_t slots = h->st_host->bump;
  unsigned long long* cnt = nullptr;
  uint32_t* tmp = nullptr;
  if (cudaMalloc(&cnt, 8) != cudaSuccess) return DT_ENOMEM;
  // the sorted list needs the unsorted one first; otherwise the tetrahedra go straight to the
  // caller's buffer (a count alone when it has none)
  const bool sort = canonical && !(h->cfg.flags & DT_FLAG_NO_CANONICAL_SORT) && cap > 0;
  if (sort && cudaMalloc(&tmp, std::max<uint64_t>(slots, 1) * 16) != cudaSuccess) {
    cudaFree(cnt);
    return DT_ENOMEM;
  }
  cudaMemsetAsync(cnt, 0, 8, s);
  k_collect<<<grid_for(slots, 256), 256, 0, s>>>(h->tets, slots, h->pts, h->cap_pts, sort ? tmp : tets_dev, cnt,
                                                 sort ? slots : cap, canonical);
  ++g_kernel_launches;
  unsigned long long T = 0;
  cudaMemcpyAsync(&T, cnt, 8, cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  *n_tets = T;
  h->stats.n_tets = T;
  if (T > cap) {
    cudaFree(cnt);
    cudaFree(tmp);
    return DT_ETOOSMALL;
  }
  if (sort && T > 1) {
    uint64_t *khi = nullptr, *klo = nullptr, *ka = nullptr;
    uint32_t *idx = nullptr, *ia = nullptr, *hist = nullptr;
    bool ok = cudaMalloc(&khi, T * 8) == cudaSuccess && cudaMalloc(&klo, T * 8) == cudaSuccess &&
              cudaMalloc(&ka, T * 8) == cudaSuccess && cudaMalloc(&idx, T * 4) == cudaSuccess &&
              cudaMalloc(&ia, T * 4) == cudaSuccess &&
              cudaMalloc(&hist, radix_hist_entries(T) * 4) == cudaSuccess;
    if (ok) {
      k_split_keys<<<grid_for(T, 256), 256, 0, s>>>((const uint4*)tmp, T, khi, klo, idx);
      ++g_kernel_launches;
      bool alt = radix_sort_pairs(klo, idx, ka, ia, T, 64, hist, s);
      uint32_t* order = alt ? ia : idx;
      uint32_t* other = alt ? idx : ia;
      k_gather_keys<<<grid_for(T, 256), 256, 0, s>>>(khi, order, T, ka);
      ++g_kernel_launches;
      bool alt2 = radix_sort_pairs(ka, order, klo, other, T, 64, hist, s);
      k_gather_tets<<<grid_for(T, 256), 256, 0, s>>>((const uint4*)tmp, alt2 ? other : order, T, (uint4*)tets_dev);
      ++g_kernel_launches;
    } else {
      rc = DT_ENOMEM;
    }
    cudaFree(khi);
    cudaFree(klo);
    cudaFree(ka);
    cudaFree(idx);
    cudaFree(ia);
    cudaFree(hist);
  } else if (sort && T) {
    cudaMemcpyAsync(tets_dev, tmp, T * 16, cudaMemcpyDeviceToDevice, s);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = DT_ECUDA;
  cudaFree(cnt);
  cudaFree(tmp);
  return rc;
}

int dt_get_tets_host(dt_handle* h, uint32_t* tets_host, uint64_t cap, uint64_t* n_tets, int canonical) {
  if (!h || !n_tets || (cap > 0 && !tets_host)) return DT_EINVAL;
  *n_tets = 0;
  if (cap == 0) return dt_get_tets(h, nullptr, 0, n_tets, nullptr, canonical);
  // page-locked host memory is mapped into the device's address space: without the canonical
  // sort the collection writes the rows there directly, and no copy follows
  const bool sort = canonical && !(h->cfg.flags & DT_FLAG_NO_CANONICAL_SORT);
  cudaPointerAttributes at{};
  if (!sort && cudaPointerGetAttributes(&at, tets_host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer) {
    uint64_t T = 0;
    const int rc = dt_get_tets(h, static_cast<uint32_t*>(at.devicePointer), cap, &T, nullptr, canonical);
    *n_tets = T;
    return rc;
  }
  cudaGetLastError();  // a pointer the runtime does not know leaves an error behind; it is not one
  // one collection into a device buffer kept by the handle, then one copy out (fast from
  // page-locked memory)
  if (cap > h->out_cap) {
    cudaFree(h->out_buf);
    h->out_buf = nullptr;
    h->out_cap = 0;
    if (cudaMalloc(&h->out_buf, cap * 16) != cudaSuccess) return DT_ENOMEM;
    h->out_cap = cap;
  }
  uint64_t T = 0;
  int rc = dt_get_tets(h, h->out_buf, cap, &T, nullptr, canonical);
  *n_tets = T;
  if (rc != DT_OK) return rc;
  if (T && cudaMemcpyAsync(tets_host, h->out_buf, T * 16, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return DT_ECUDA;
  return cudaStreamSynchronize(h->stream) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_get_order(dt_handle* h, uint64_t* keys_dev, uint32_t* perm_dev, uint8_t* rounds_dev) {
  if (!h) return DT_EINVAL;
  if (!h->last_n) return DT_ESTATE;
  uint64_t n = h->last_n;
  cudaStream_t s = h->stream;
  if (keys_dev) cudaMemcpyAsync(keys_dev, h->ows.keys, n * 8, cudaMemcpyDeviceToDevice, s);
  if (perm_dev) cudaMemcpyAsync(perm_dev, h->ows.perm, n * 4, cudaMemcpyDeviceToDevice, s);
  if (rounds_dev) cudaMemcpyAsync(rounds_dev, h->ows.rounds, n, cudaMemcpyDeviceToDevice, s);
  return cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_get_stats(dt_handle* h, dt_stats* out) {
  if (!h || !out) return DT_EINVAL;
  if (h->has_mesh) {
    int rc = sync_state(h);
    if (rc != DT_OK && rc != DT_ELIMIT && rc != DT_ENOMEM) return rc;
  }
  fill_stats(h, out);
  return DT_OK;
}

int dt_load_model(dt_handle* h, const float* params_host, uint32_t n_params) {
  if (!h || !params_host || n_params != (uint32_t)mlp_params()) return DT_EINVAL;
  if (!h->model && cudaMalloc(&h->model, n_params * sizeof(float)) != cudaSuccess) return DT_ENOMEM;
  if (cudaMemcpyAsync(h->model, params_host, n_params * sizeof(float), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return DT_ECUDA;
  if (const char* t = std::getenv("DT_RISK_LOGIT")) h->risky_logit = (float)std::atof(t);
  if (const char* r = std::getenv("DT_RISK_SCALE")) h->risky_scale = std::atof(r);
  if (const char* r = std::getenv("DT_RANK_SCALE")) h->rank_scale = (float)std::atof(r);
  if (const char* u = std::getenv("DT_LEARN_USE")) {  // "rank", "defer" or "both"
    h->use_prank = std::strstr(u, "rank") || std::strstr(u, "both");
    h->use_defer = std::strstr(u, "defer") || std::strstr(u, "both");
  }
  h->model_loaded = true;
  return DT_OK;
}

int dt_get_features(dt_handle* h, float* x_dev, float* y_dev, uint8_t* valid_dev, uint64_t n) {
  if (!h || !x_dev || h->batch_mode || !h->has_mesh) return DT_EINVAL;
  if (n != h->last_n) return DT_EINVAL;
  if ((y_dev || valid_dev) && !((h->cfg.flags & DT_FLAG_LOG) && h->log_nc)) return DT_ESTATE;
  cudaStream_t s = h->stream;
  int rc = compute_features(h, n);
  if (rc != DT_OK) return rc;
  cudaMemcpyAsync(x_dev, h->feat, n * 8 * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (y_dev || valid_dev) {
    k_labels<<<grid_for(n, 256), 256, 0, s>>>(h->log_nc, h->log_lost, (uint32_t)h->last_base, n, y_dev, valid_dev);
    ++g_kernel_launches;
  }
  return cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_mlp_forward(const float* params_dev, const float* x_dev, uint64_t n, float* out_dev, void* stream) {
  if (!params_dev || (n && (!x_dev || !out_dev))) return DT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = mlp_forward(params_dev, x_dev, n, out_dev, s);
  if (rc != DT_OK) return rc;
  return cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_mlp_grad(const float* params_dev, const float* x_dev, const float* y_dev, uint64_t n, float* grad_dev,
                float* loss_dev, void* stream) {
  if (!params_dev || !x_dev || !y_dev || !grad_dev || !loss_dev || n == 0) return DT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = mlp_grad(params_dev, x_dev, y_dev, n, grad_dev, loss_dev, s);
  if (rc != DT_OK) return rc;
  return cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_mlp_train(float* params_dev, const float* x_dev, const float* y_dev, uint64_t n, uint32_t steps,
                 uint32_t batch, float lr, uint64_t seed, float* losses_host, void* stream) {
  if (!params_dev || !x_dev || !y_dev || n == 0 || batch == 0 || !(lr > 0.f) || n > 0xFFFFFFFFull) return DT_EINVAL;
  return mlp_train(params_dev, x_dev, y_dev, n, steps, batch, lr, seed, losses_host, (cudaStream_t)stream);
}

void dt_destroy(dt_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  order_ws_free(h->ows);
  refine_ws_free(h->rws);
  cudaFree(h->pts);
  cudaFree(h->ptf);
  cudaFree(h->vflag);
  cudaFree(h->point_hint);
  cudaFree(h->tets);
  cudaFree(h->claim);
  cudaFree(h->lock);
  cudaFree(h->subdet);
  cudaFree(h->in_buf);
  cudaFree(h->out_buf);
  cudaFree(h->async_big_ws);
  cudaFree(h->async_borrow_ws);
  cudaFree(h->async_borrow_busy);
  cudaFree(h->wcost);
  cudaFree(h->seg_prefix);
  cudaFree(h->seg_bounds);
  cudaFree(h->freelist);
  cudaFree(h->pending);
  cudaFree(h->cell_hint);
  cudaFree(h->cell_hint2);
  cudaFree(h->st);
  if (h->st_host) cudaFreeHost(h->st_host);
  cudaFree(h->cand_p);
  cudaFree(h->cand_t);
  cudaFree(h->cand_status);
  cudaFree(h->cand_nc);
  cudaFree(h->cand_nb);
  cudaFree(h->scratch);
  for (auto& qb : h->queue) cudaFree(qb);
  cudaFree(h->wlist);
  cudaFree(h->wave_cum);
  cudaFree(h->bigmem);
  cudaFree(h->medscratch);
  cudaFree(h->hugemem);
  cudaFree(h->ctamem);
  cudaFree(h->bbox_dev);
  cudaFree(h->boff_dev);
  cudaFree(h->bclouds);
  cudaFree(h->border);
  cudaFree(h->bsample);
  cudaFree(h->bcid);
  cudaFree(h->bdup);
  cudaFree(h->blist_a);
  cudaFree(h->blist_b);
  cudaFree(h->blist_big);
  cudaFree(h->bhint_f);
  cudaFree(h->bhint_c);
  cudaFree(h->bcbox);
  cudaFree(h->bstates);
  cudaFree(h->bws);
  cudaFree(h->bstats);
  cudaFree(h->bnext);
  cudaFree(h->beta);
  cudaFree(h->log_nc);
  cudaFree(h->log_lost);
  cudaFree(h->model);
  cudaFree(h->feat);
  cudaFree(h->pred);
  cudaFree(h->cell_count);
  cudaFree(h->risky);
  cudaFree(h->wave_hist);
  if (h->bexec) cudaGraphExecDestroy(h->bexec);
  if (h->bgraph) cudaGraphDestroy(h->bgraph);
  for (auto& e : h->bev)
    if (e) cudaEventDestroy(e);
  if (h->bs) cudaStreamDestroy(h->bs);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->prof_events) cudaEventDestroy(e);
  delete h;
}

const char* dt_strerror(int code) {
  switch (code) {
    case DT_OK: return "ok";
    case DT_EINVAL: return "invalid argument";
    case DT_ENOMEM: return "out of device memory or tetrahedron capacity";
    case DT_ETOOSMALL: return "output buffer too small";
    case DT_EDEGENERATE: return "fewer than four non-coplanar points";
    case DT_ELIMIT: return "a device-side bound was exceeded";
    case DT_ECUDA: return "CUDA runtime error";
    case DT_ESTATE: return "call not valid in the current state";
    default: return "unknown error";
  }
}

int dt_eval_predicates(int kind, const double* pts_dev, const int64_t* ids_dev, int8_t* out_dev, uint64_t n,
                       void* stream) {
  if (kind < 0 || kind > 4 || (n > 0 && (!pts_dev || !out_dev)) || ((kind == 2 || kind == 4) && n > 0 && !ids_dev))
    return DT_EINVAL;
  if (n == 0) return DT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = nullptr;
  if (cudaMalloc(&st, sizeof(DevState)) != cudaSuccess) return DT_ENOMEM;
  cudaMemsetAsync(st, 0, sizeof(DevState), s);
  k_eval_predicates<<<grid_for(n, 128), 128, 0, s>>>(kind, pts_dev, (kind == 2 || kind == 4) ? ids_dev : nullptr,
                                                     out_dev, n, st);
  ++g_kernel_launches;
  DevState hs;
  cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  int rc = cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
  cudaFree(st);
  if (rc == DT_OK && hs.error) rc = map_dev_error(hs.error);
  return rc;
}

}  // extern "C"
