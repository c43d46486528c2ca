// Batches of independent clouds in one persistent launch.
//
// Every thread block takes whole clouds from a device work counter, largest first, and builds
// each one completely by itself: Init, then the cloud's BRIO rounds wave by wave, each wave in
// rounds of up to W concurrent insertions (Algorithm 1 per point, with the claims of Section 3.2
// between the warps of the block), the points that lost retried until none is left, cavities
// too large for a warp's workspace inserted one at a time with the whole block's workspace.
// Block barriers replace the kernel boundaries of the single-cloud engine, so a cloud of a few
// hundred points costs no kernel launches at all, and the clouds of a batch fill every SM.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"
#include "predicates.cuh"

namespace dtg {

namespace {

unsigned grid_for(uint64_t n, int threads) {
  uint64_t b = (n + threads - 1) / threads;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 16));
}

// Per-warp workspace: cavities up to kBatchCN tetrahedra and kBatchFN boundary facets.
constexpr uint32_t kBatchHashN = 2048, kBatchCN = 512, kBatchFN = 512, kBatchEdgeN = 2048;
constexpr uint32_t kBatchLongWalk = 1u << 14;  // walk limit of short retry lists
constexpr uint32_t kBatchStall = 1024;         // retry passes without an insertion before giving up

// Hint grid of a cloud: 8 x 8 x 8 fine cells, 2 x 2 x 2 coarse cells.
constexpr int kBatchCb = 3;
constexpr uint32_t kBatchFine = 1u << (3 * kBatchCb);
constexpr uint32_t kBatchCoarse = 8;

struct BatchArgs {
  BatchCloud* clouds;
  const uint32_t* order;   // clouds in the order blocks take them
  uint32_t n_clouds;
  unsigned int* next;      // work counter
  uint8_t* vflag;
  uint32_t* list_a;        // retry lists (ping-pong) and the large-cavity list, indexed like
  uint32_t* list_b;        //   the vertices: a cloud uses its own range [vb, ve)
  uint32_t* list_big;
  uint32_t* hint_fine;     // kBatchFine per cloud
  uint32_t* hint_coarse;   // kBatchCoarse per cloud
  DevState* states;        // one per block
  char* wsmem;             // W workspaces per block
  size_t wsstride;
  float alpha;
  double gamma;            // wave growth: must equal the ordering's, bit for bit
  const float* eta;        // FP32 stage error term of this batch (computed on the device)
  unsigned long long* stats;  // kBatchStatSlots accumulators
};

// Statistics of a batch: inserted, conflicts, attempts, sum |C|, sum |B|, walk steps, dups,
// large cavities, rounds (kept per block), then exact and perturbed predicate counts.
constexpr int kBatchStats = 9;

template <int W>
struct BlockShared {
  uint32_t p[W], t[W], st[W], nc[W], nb[W];
  unsigned int nout, nbig, R, err, cloud, stop;
  unsigned long long L, stat[kBatchStats];
  unsigned long long mesh;  // vertices of the current cloud's triangulation
};

// One pass over the candidate list q (or the vertex range qbase + [0, m) when q is null):
// rounds of R segments (Section 3.3), segment s offering q[s * L + j] in round j. Losers go to
// out, large cavities to big.
template <int W>
__device__ void batch_pass(const Ctx& c, BlockShared<W>& sh, const BigWS& ws, const uint32_t* q, uint32_t qbase,
                           uint64_t m, uint32_t* out, uint32_t* big, uint8_t* vflag, float alpha, bool last_chance) {
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    double N = (double)sh.mesh;
    uint64_t R = (uint64_t)fmax(1.0, (double)alpha * N);
    R = R > (uint64_t)W ? (uint64_t)W : R;
    R = R > m ? m : R;
    sh.R = (unsigned)(R > 0 ? R : 1);
    sh.L = (m + sh.R - 1) / sh.R;
    sh.err = __ldcg(&c.st->error);
  }
  __syncthreads();
  if (sh.err) return;
  const uint32_t R = sh.R;
  const uint64_t L = sh.L;
  const uint32_t max_walk = last_chance ? kBatchLongWalk : c.max_walk;
  for (uint64_t j = 0; j < L; ++j) {
    // walk: one thread per candidate (the lanes of the first warp walk together)
    if (tid < (int)R) {
      uint64_t idx = (uint64_t)tid * L + j;
      uint32_t status = kCandEmpty, p = kNone, t = kNone;
      if (idx < m) {
        p = q ? q[idx] : qbase + (uint32_t)idx;
        if (vflag[p] == 0) {
          PtF FP = load_ptf(c.ptf, p);
          uint32_t hint = c.point_hint[p];
          if (hint == kNone && j > 0) hint = c.point_hint[q ? q[idx - 1] : qbase + (uint32_t)(idx - 1)];
          if (hint == kNone) {
            uint32_t f, g;
            cells_of(c, FP, &f, &g);
            hint = c.cell_hint[f];
            if (hint == kNone) hint = c.cell_hint2[g];
          }
          uint32_t steps = 0;
          status = walk_point(c, p, FP, hint, p * 0x9E3779B1u >> 30, __ldcg(&c.st->anchor), max_walk, &t, &steps);
          atomicAdd(&sh.stat[5], (unsigned long long)steps);
          c.point_hint[p] = t;
        }
      }
      sh.p[tid] = p;
      sh.t[tid] = t;
      sh.st[tid] = status;
    }
    __syncthreads();
    // cavity and claims: one warp per candidate
    if (wid < (int)R && sh.st[wid] == kCandLocated) {
      uint32_t p = sh.p[wid];
      unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), 0u, p);
      int nc = 0, nb = 0;
      int r = cavity_warp(c, ws.cav, sh.t[wid], p, load_ptf(c.ptf, p), prio, &nc, &nb);
      if (lane == 0) {
        sh.st[wid] = (uint32_t)r;
        sh.nc[wid] = (uint32_t)nc;
        sh.nb[wid] = (uint32_t)nb;
      }
    }
    __threadfence();
    __syncthreads();
    // ball, then the candidate's bookkeeping by the same warp
    if (wid < (int)R) {
      const uint32_t p = sh.p[wid];
      uint32_t s = sh.st[wid];
      if (s == kCandLocated) {
        unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), 0u, p);
        int nc = (int)sh.nc[wid], nb = (int)sh.nb[wid];
        s = (uint32_t)insert_warp(c, ws.ins, p, prio, ws.cav.clist, nc, ws.cav.blist, nb, nb <= kFMax,
                                  __ldcg(&c.st->free_avail), __ldcg(&c.st->bump), c.st->capacity);
        if (lane == 0 && s == kCandInserted) {
          PtF FP = load_ptf(c.ptf, p);
          uint32_t f, g, s0 = ws.ins.slot[0];
          cells_of(c, FP, &f, &g);
          c.cell_hint[f] = s0;
          c.cell_hint2[g] = s0;
          c.point_hint[p] = s0;
          c.st->anchor = s0;
          vflag[p] = 2;
          atomicAdd(&sh.stat[0], 1ull);
          atomicAdd(&sh.mesh, 1ull);
          atomicAdd(&sh.stat[3], (unsigned long long)nc);
          atomicAdd(&sh.stat[4], (unsigned long long)nb);
        }
      }
      if (lane == 0) {
        if (s != kCandEmpty) atomicAdd(&sh.stat[2], 1ull);
        if (s == kCandLost) atomicAdd(&sh.stat[1], 1ull);
        if (s == kCandLost || s == kCandWalkLimit) out[atomicAdd(&sh.nout, 1u)] = p;
        else if (s == kCandBig) big[atomicAdd(&sh.nbig, 1u)] = p;
        else if (s == kCandDup) {
          vflag[p] = 1;
          atomicAdd(&sh.stat[6], 1ull);
        }
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) sh.stat[8] += 1;
    // the last warp closes the round while the first walks the next one: walks do not touch the
    // allocator or the stamp, and the barrier after the walk orders the close before the claims
    if (wid == W - 1) finish_round_warp(c);
  }
  __syncthreads();
}

// The large cavities of a pass, one at a time by warp 0 with the whole block's workspace (the
// other warps wait at the barrier that follows).
template <int W>
__device__ void batch_big(const Ctx& c, BlockShared<W>& sh, const BigWS& wide, uint32_t* big, uint8_t* vflag) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) {
    for (uint32_t k = 0; k < sh.nbig; ++k) {
      int e = __shfl_sync(kFull, lane == 0 ? (int)__ldcg(&c.st->error) : 0, 0);
      if (e) break;
      uint32_t p = big[k];
      PtF FP = load_ptf(c.ptf, p);
      uint32_t t = kNone, steps = 0;
      int s = kCandEmpty;
      if (lane == 0) {
        uint32_t hint = c.point_hint[p];
        s = walk_point(c, p, FP, hint, 0, __ldcg(&c.st->anchor), 1u << 20, &t, &steps);
        sh.stat[5] += steps;
      }
      s = __shfl_sync(kFull, s, 0);
      t = __shfl_sync(kFull, t, 0);
      if (s == kCandDup) {
        if (lane == 0) {
          vflag[p] = 1;
          sh.stat[6] += 1;
        }
        continue;
      }
      if (s != kCandLocated) {
        if (lane == 0) raise_error(c.st, kErrWalk, p);
        break;
      }
      unsigned long long prio = claim_prio(__ldcg(&c.st->stamp), 0u, p);
      int nc = 0, nb = 0;
      int r = cavity_warp(c, wide.cav, t, p, FP, prio, &nc, &nb);
      if (r == kCandLocated)
        r = insert_warp(c, wide.ins, p, prio, wide.cav.clist, nc, wide.cav.blist, nb, nb <= kFMax,
                        __ldcg(&c.st->free_avail), __ldcg(&c.st->bump), c.st->capacity);
      if (r != kCandInserted) {
        if (lane == 0) raise_error(c.st, kErrBigCavity, (unsigned)nb);
        break;
      }
      if (lane == 0) {
        uint32_t s0 = wide.ins.slot[0];
        c.point_hint[p] = s0;
        c.st->anchor = s0;
        vflag[p] = 2;
        sh.stat[0] += 1;
        sh.mesh += 1;
        sh.stat[3] += (unsigned long long)nc;
        sh.stat[4] += (unsigned long long)nb;
        sh.stat[7] += 1;
      }
      finish_round_warp(c);
    }
  }
  __syncthreads();
  if (tid == 0) sh.nbig = 0;
  __syncthreads();
}

template <int W, int MINB>
__global__ void __launch_bounds__(W * 32, MINB) k_batch(Ctx c0, BatchArgs a) {
  __shared__ BlockShared<W> sh;
  const int tid = threadIdx.x, wid = tid >> 5;
  BigWS ws, wide;
  char* base = a.wsmem + (size_t)blockIdx.x * W * a.wsstride;
  carve(base + (size_t)wid * a.wsstride, kBatchHashN, kBatchCN, kBatchFN, kBatchEdgeN, &ws);
  carve(base, W * kBatchHashN, W * kBatchCN, W * kBatchFN, W * kBatchEdgeN, &wide);
  DevState* st = a.states + blockIdx.x;
  const float eta = *a.eta;
  if (tid < kBatchStats) sh.stat[tid] = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) sh.cloud = atomicAdd(a.next, 1u);
    __syncthreads();
    const uint32_t k = sh.cloud;
    if (k >= a.n_clouds) break;
    const uint32_t ci = a.order[k];
    BatchCloud* cl = a.clouds + ci;
    const uint32_t vb = cl->vb, ve = cl->ve, tb = cl->tb;
    Ctx c = c0;
    c.eta = eta;
    c.st = st;
    c.freelist = c0.freelist + tb;
    c.pending = c0.pending + tb;
    c.cell_hint = a.hint_fine + (size_t)ci * kBatchFine;
    c.cell_hint2 = a.hint_coarse + (size_t)ci * kBatchCoarse;
    for (int d = 0; d < 3; ++d) {
      c.lo[d] = cl->lo[d];
      c.sc[d] = cl->sc[d];
    }
    c.cb = kBatchCb;
    if (tid == 0) {
      // a fresh allocator and claim stamp for this cloud's slot range
      st->stamp = 1;
      st->bump = tb;
      st->capacity = (unsigned long long)tb + cl->tcap;
      st->free_avail = 0;
      st->alloc_cursor = 0;
      st->pending = 0;
      st->free_capacity = cl->tcap;
      st->error = 0;
      st->error_info = 0;
      st->anchor = tb;
      st->n_inserted = 0;
      sh.nout = 0;
      sh.nbig = 0;
      sh.err = init_mesh(c, vb, ve, a.vflag, tb) ? 0u : 1u;
      sh.mesh = sh.err ? 0 : 4;
      if (!sh.err) sh.stat[0] += 4;
      __threadfence_block();
    }
    __syncthreads();
    if (sh.err == 0) {
      const uint64_t n = ve - vb;
      for (int r = 0;; ++r) {
        uint64_t b = brio_round_begin(r), e = brio_round_begin(r + 1);
        if (b >= n) break;
        uint64_t m = (e < n ? e : n) - b;
        // waves: contiguous ranges of the (cloud, round, wave, key) order
        uint64_t lo = 0;
        for (int w = 0; w < kMaxWaves && lo < m; ++w) {
          uint64_t hi = wave_end(m, b, a.gamma, w);
          batch_pass<W>(c, sh, ws, nullptr, vb + (uint32_t)(b + lo), hi - lo, a.list_a + vb, a.list_big + vb,
                        a.vflag, a.alpha, false);
          if (sh.nbig) batch_big<W>(c, sh, wide, a.list_big + vb, a.vflag);
          lo = hi;
        }
        // the points that lost (or stopped walking): retried until none is left
        uint32_t* cur = a.list_a + vb;
        uint32_t* nxt = a.list_b + vb;
        // every retry pass inserts its highest-priority located point or advances the walks that
        // hit their step limit; kBatchStall passes without an insertion end the cloud in error
        uint32_t idle = 0;
        for (;;) {
          __syncthreads();
          const uint32_t mq = sh.nout;
          const unsigned long long before = sh.stat[0];
          if (tid == 0) sh.stop = (mq == 0 || __ldcg(&st->error)) ? 1u : 0u;
          __syncthreads();
          if (sh.stop) break;
          if (tid == 0) sh.nout = 0;
          __syncthreads();
          batch_pass<W>(c, sh, ws, cur, 0, mq, nxt, a.list_big + vb, a.vflag, a.alpha, mq < 64);
          if (sh.nbig) batch_big<W>(c, sh, wide, a.list_big + vb, a.vflag);
          __syncthreads();
          idle = (sh.stat[0] == before) ? idle + 1 : 0;
          if (idle >= kBatchStall) {
            if (tid == 0) raise_error(st, kErrInternal, 0xBA7Cu);
            __syncthreads();
            break;
          }
          uint32_t* x = cur;
          cur = nxt;
          nxt = x;
        }
        __syncthreads();
        if (tid == 0) sh.stop = (sh.nout != 0 || __ldcg(&st->error)) ? 1u : 0u;
        __syncthreads();
        if (sh.stop) break;
      }
    }
    __syncthreads();
    if (tid == 0) {
      unsigned e = sh.err ? (unsigned)kErrDegenerate : (unsigned)__ldcg(&st->error);
      if (e == 0 && sh.nout != 0) e = kErrInternal;
      cl->status = e;
      cl->info = sh.err ? 0u : (unsigned)__ldcg(&st->error_info);
      cl->used = (uint32_t)(__ldcg(&st->bump) - tb);
      cl->inserted = (uint32_t)sh.mesh;
      atomicAdd(&a.stats[9], __ldcg(&st->n_exact));
      atomicAdd(&a.stats[10], __ldcg(&st->n_sos));
      st->n_exact = 0;
      st->n_sos = 0;
    }
  }
  __syncthreads();
  if (tid < kBatchStats && sh.stat[tid]) atomicAdd(&a.stats[tid], sh.stat[tid]);
}

// Per-cloud reset before a launch: claim words of the cloud's slots, its hint cells, the
// vertices' flags (duplicates stay flagged) and walk hints.
__global__ void k_batch_reset(const BatchCloud* clouds, const uint32_t* list, uint32_t n_list,
                              unsigned long long* claim, uint32_t* hint_fine, uint32_t* hint_coarse,
                              const uint8_t* dup_sorted, uint8_t* vflag, uint32_t* point_hint) {
  for (uint32_t k = blockIdx.x; k < n_list; k += gridDim.x) {
    const uint32_t ci = list ? list[k] : k;
    const BatchCloud cl = clouds[ci];
    for (uint64_t t = threadIdx.x; t < 2ull * cl.tcap; t += blockDim.x) claim[2ull * cl.tb + t] = 0ull;
    for (uint32_t i = threadIdx.x; i < kBatchFine; i += blockDim.x) hint_fine[(size_t)ci * kBatchFine + i] = kNone;
    if (threadIdx.x < kBatchCoarse) hint_coarse[(size_t)ci * kBatchCoarse + threadIdx.x] = kNone;
    for (uint32_t v = cl.vb + threadIdx.x; v < cl.ve; v += blockDim.x) {
      vflag[v] = dup_sorted[v];
      point_hint[v] = kNone;
    }
  }
}

// Finite tetrahedra of every cloud, vertex ids local to the cloud. Pass 0 counts per cloud;
// pass 1 writes from out_off[cloud] (one block per cloud, order inside a cloud unspecified).
__global__ void k_batch_collect(const BatchCloud* clouds, uint32_t n_clouds, const Tet* __restrict__ tets,
                                const Pt* __restrict__ pts, const uint64_t* __restrict__ in_off, int pass,
                                unsigned long long* counts, const unsigned long long* out_off, uint32_t* out,
                                int canonical) {
  for (uint32_t ci = blockIdx.x; ci < n_clouds; ci += gridDim.x) {
    const BatchCloud cl = clouds[ci];
    if (cl.status != 0) continue;
    unsigned long long pos = 0;
    for (uint64_t t0 = 0; t0 < cl.used; t0 += blockDim.x) {
      uint64_t t = t0 + threadIdx.x;
      bool keep = false;
      uint32_t r[4] = {0, 0, 0, 0};
      if (t < cl.used) {
        uint4 v = tets[cl.tb + t].v;
        keep = !tet_dead(v) && ghost_pos(v) < 0;
        if (keep) {
          r[0] = (uint32_t)((uint64_t)pts[v.x].w - in_off[ci]);
          r[1] = (uint32_t)((uint64_t)pts[v.y].w - in_off[ci]);
          r[2] = (uint32_t)((uint64_t)pts[v.z].w - in_off[ci]);
          r[3] = (uint32_t)((uint64_t)pts[v.w].w - in_off[ci]);
          if (canonical) canonical_rotation(r);
        }
      }
      unsigned bal = __ballot_sync(kFull, keep);
      __shared__ unsigned s_w[32];
      __shared__ unsigned long long s_base;
      const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
      if (lane == 0) s_w[wid] = __popc(bal);
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
          unsigned x = s_w[w];
          s_w[w] = (unsigned)acc;
          acc += x;
        }
        s_base = pos;
        pos += acc;
      }
      __syncthreads();
      if (pass == 1 && keep) {
        unsigned long long at = out_off[ci] + s_base + s_w[wid] + __popc(bal & ((1u << lane) - 1u));
        reinterpret_cast<uint4*>(out)[at] = make_uint4(r[0], r[1], r[2], r[3]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && pass == 0) counts[ci] = pos;
  }
}

// Key of a collected tetrahedron for the canonical order of a batch: (cloud, tetrahedron).
__global__ void k_batch_tet_keys(const uint4* tets, uint64_t T, const unsigned long long* out_off, uint32_t n_clouds,
                                 uint64_t* khi, uint64_t* klo, uint64_t* kcl, uint32_t* idx) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < T;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint4 t = tets[i];
    khi[i] = ((uint64_t)t.x << 32) | t.y;
    klo[i] = ((uint64_t)t.z << 32) | t.w;
    uint32_t lo = 0, hi = n_clouds;  // cloud: last c with out_off[c] <= i
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) / 2;
      if (out_off[mid] <= i) lo = mid;
      else hi = mid;
    }
    kcl[i] = lo;
    idx[i] = (uint32_t)i;
  }
}


// Hint grid of every cloud (8 cells per axis over its box) and the batch's FP32 error term
// eta = 2^-44 max|x| (+ the spacing of FP32 subnormals), as the single-cloud engine sets it.
__global__ void k_batch_prepare(BatchCloud* clouds, const double* __restrict__ cbox, uint32_t n_clouds,
                                float* eta) {
  __shared__ double s_max[256];
  double m = 0.0;
  for (uint32_t c = threadIdx.x; c < n_clouds; c += blockDim.x) {
    const double* B = cbox + 6ull * c;
    for (int k = 0; k < 6; ++k) m = fmax(m, fabs(B[k]));
    for (int k = 0; k < 3; ++k) {
      double ext = B[3 + k] - B[k];
      clouds[c].lo[k] = (float)B[k];
      clouds[c].sc[k] = ext > 0 ? (float)((double)(1u << kBatchCb) / ext) : 0.f;
    }
  }
  s_max[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *eta = (float)(ldexp(s_max[0], -44) * 1.0001 + 1e-38);
}

}  // namespace

size_t batch_ws_stride() { return carve(nullptr, kBatchHashN, kBatchCN, kBatchFN, kBatchEdgeN, nullptr); }
uint32_t batch_hint_fine() { return kBatchFine; }
uint32_t batch_hint_coarse() { return kBatchCoarse; }
int batch_cb() { return kBatchCb; }

// Block shapes the batch kernel is built for: warps per block and the minimum resident blocks
// per SM that bounds its registers (128 registers at 8 warps x 2 blocks, 64 at 32 x 1, 32 at
// 32 x 2). The 32-register shapes spill, but 64 resident warps per SM hide the latency of the
// pointer chasing better than fewer warps without spills, so the autotuner tries both kinds.
// A shape is encoded as warps | (min_blocks << 8).
static const int kShapes[] = {8 | (2 << 8),  8 | (4 << 8),  8 | (8 << 8),  16 | (2 << 8),
                              16 | (4 << 8), 32 | (1 << 8), 32 | (2 << 8)};

int batch_shapes(int* shapes, int max_n) {
  int n = 0;
  for (int s : kShapes)
    if (n < max_n) shapes[n++] = s;
  return n;
}

template <int W, int MINB>
static int occupancy() {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<W, MINB>, W * 32, 0) == cudaSuccess ? nb : 0;
}

// Resident blocks per SM of the batch kernel with the given shape (for sizing its workspaces).
int batch_blocks_per_sm(int shape) {
  switch (shape) {
    case 8 | (2 << 8): return occupancy<8, 2>();
    case 8 | (4 << 8): return occupancy<8, 4>();
    case 8 | (8 << 8): return occupancy<8, 8>();
    case 16 | (2 << 8): return occupancy<16, 2>();
    case 16 | (4 << 8): return occupancy<16, 4>();
    case 32 | (1 << 8): return occupancy<32, 1>();
    case 32 | (2 << 8): return occupancy<32, 2>();
    default: return 0;
  }
}

int batch_launch(int shape, unsigned blocks, const Ctx& c, BatchCloud* clouds, const uint32_t* order, uint32_t n_clouds,
                 unsigned int* next, uint8_t* vflag, uint32_t* list_a, uint32_t* list_b, uint32_t* list_big,
                 uint32_t* hint_fine, uint32_t* hint_coarse, DevState* states, char* wsmem, size_t wsstride,
                 float alpha, double gamma, const float* eta, unsigned long long* stats, cudaStream_t s) {
  BatchArgs a{clouds, order, n_clouds, next, vflag, list_a, list_b, list_big, hint_fine, hint_coarse, states,
              wsmem, wsstride, alpha, gamma, eta, stats};
  switch (shape) {
    case 8 | (2 << 8): k_batch<8, 2><<<blocks, 8 * 32, 0, s>>>(c, a); break;
    case 8 | (4 << 8): k_batch<8, 4><<<blocks, 8 * 32, 0, s>>>(c, a); break;
    case 8 | (8 << 8): k_batch<8, 8><<<blocks, 8 * 32, 0, s>>>(c, a); break;
    case 16 | (2 << 8): k_batch<16, 2><<<blocks, 16 * 32, 0, s>>>(c, a); break;
    case 16 | (4 << 8): k_batch<16, 4><<<blocks, 16 * 32, 0, s>>>(c, a); break;
    case 32 | (1 << 8): k_batch<32, 1><<<blocks, 32 * 32, 0, s>>>(c, a); break;
    case 32 | (2 << 8): k_batch<32, 2><<<blocks, 32 * 32, 0, s>>>(c, a); break;
    default: return DT_EINVAL;
  }
  ++g_kernel_launches;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

void batch_reset(const BatchCloud* clouds, const uint32_t* list, uint32_t n_list, unsigned long long* claim,
                 uint32_t* hint_fine, uint32_t* hint_coarse, const uint8_t* dup_sorted, uint8_t* vflag,
                 uint32_t* point_hint, cudaStream_t s) {
  if (n_list == 0) return;
  k_batch_reset<<<std::min<uint32_t>(n_list, 152u * 8), 256, 0, s>>>(clouds, list, n_list, claim, hint_fine,
                                                                     hint_coarse, dup_sorted, vflag, point_hint);
  ++g_kernel_launches;
}

void batch_prepare(BatchCloud* clouds, const double* cbox, uint32_t n_clouds, float* eta, cudaStream_t s) {
  k_batch_prepare<<<1, 256, 0, s>>>(clouds, cbox, n_clouds, eta);
  ++g_kernel_launches;
}

void batch_collect(const BatchCloud* clouds, uint32_t n_clouds, const Tet* tets, const Pt* pts, const uint64_t* in_off,
                   int pass, unsigned long long* counts, const unsigned long long* out_off, uint32_t* out,
                   int canonical, cudaStream_t s) {
  k_batch_collect<<<std::min<uint32_t>(n_clouds, 152u * 8), 256, 0, s>>>(clouds, n_clouds, tets, pts, in_off, pass,
                                                                        counts, out_off, out, canonical);
  ++g_kernel_launches;
}

void batch_tet_keys(const uint32_t* tets, uint64_t T, const unsigned long long* out_off, uint32_t n_clouds,
                    uint64_t* khi, uint64_t* klo, uint64_t* kcl, uint32_t* idx, cudaStream_t s) {
  k_batch_tet_keys<<<grid_for(T, 256), 256, 0, s>>>((const uint4*)tets, T, out_off, n_clouds, khi, klo, kcl, idx);
  ++g_kernel_launches;
}

}  // namespace dtg
