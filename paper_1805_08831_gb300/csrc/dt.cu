// Kernels, handle and C ABI of the GB300 Delaunay library (see include/dt.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "engine.cuh"
#include "internal.h"
#include "predicates.cuh"

namespace dtg {
namespace {

constexpr int kWarps = 8;  // candidates per 256-thread block in the warp-per-point kernels
constexpr uint32_t kScratchStride = kCMax + kFMax;

// Large-cavity workspace capacities (global memory, one point at a time).
constexpr uint32_t kBigHash = 1u << 17;
constexpr uint32_t kBigC = 1u << 15;
constexpr uint32_t kBigF = 1u << 15;
constexpr uint32_t kBigEdge = 1u << 17;

struct BigWS {
  CavWS cav;
  InsWS ins;
};

// ------------------------------------------------------------------ kernels of one round
__global__ void __launch_bounds__(256) k_walk(Ctx c, const uint32_t* __restrict__ q, uint32_t qbase,
                                              uint64_t m, uint64_t L, uint64_t j, uint32_t R,
                                              const uint8_t* __restrict__ vflag, uint32_t* cand_p,
                                              uint32_t* cand_t, uint32_t* cand_status) {
  __shared__ unsigned long long s_steps, s_limit;
  if (threadIdx.x == 0) {
    s_steps = 0;
    s_limit = 0;
  }
  __syncthreads();
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < R) {
    uint64_t idx = (uint64_t)s * L + j;
    uint32_t status = kCandEmpty, p = kNone, t = kNone;
    if (idx < m) {
      p = q ? q[idx] : qbase + (uint32_t)idx;
      if (vflag[p] == 0) {
        uint32_t anchor = __ldcg(&c.st->anchor);
        Pt P = load_pt(c.pts, p);
        uint32_t hint = c.point_hint[p];
        if (hint == kNone) hint = c.cell_hint[cell_of(c, P)];
        uint32_t steps = 0;
        status = walk_point(c, P, hint, p * 0x9E3779B1u >> 30, anchor, c.max_walk, &t, &steps);
        atomicAdd(&s_steps, (unsigned long long)steps);
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
  }
}

__global__ void __launch_bounds__(256) k_cavity(Ctx c, uint32_t R, const uint32_t* __restrict__ cand_p,
                                                const uint32_t* __restrict__ cand_t, uint32_t* cand_status,
                                                uint32_t* cand_nc, uint32_t* cand_nb, uint32_t* scratch) {
  __shared__ uint32_t s_hkey[kWarps][kHash];
  __shared__ uint8_t s_hval[kWarps][kHash];
  __shared__ uint32_t s_c[kWarps][kCMax];
  __shared__ uint32_t s_b[kWarps][kFMax];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t cand = blockIdx.x * kWarps + wid;
  if (cand >= R) return;
  if (cand_status[cand] != kCandLocated) return;
  uint32_t p = cand_p[cand];
  Pt P = load_pt(c.pts, p);
  unsigned long long prio = (__ldcg(&c.st->stamp) << 32) | (unsigned long long)(p + 1u);
  CavWS w{s_hkey[wid], s_hval[wid], kHash - 1, s_c[wid], kCMax, s_b[wid], kFMax};
  int nc = 0, nb = 0;
  int r = cavity_warp(c, w, cand_t[cand], P, prio, &nc, &nb);
  if (r == kCandLocated) {
    uint32_t* dst = scratch + (size_t)cand * kScratchStride;
    for (int i = lane; i < nc; i += 32) dst[i] = s_c[wid][i];
    for (int i = lane; i < nb; i += 32) dst[kCMax + i] = s_b[wid][i];
  }
  if (lane == 0) {
    cand_status[cand] = (uint32_t)r;
    cand_nc[cand] = (uint32_t)nc;
    cand_nb[cand] = (uint32_t)nb;
  }
}

__global__ void __launch_bounds__(256) k_insert(Ctx c, uint32_t R, const uint32_t* __restrict__ cand_p,
                                                uint32_t* cand_status, const uint32_t* __restrict__ cand_nc,
                                                const uint32_t* __restrict__ cand_nb,
                                                const uint32_t* __restrict__ scratch, uint32_t* qnext,
                                                uint32_t* big) {
  __shared__ uint4 s_nv[kWarps][kFMax];
  __shared__ uint4 s_nn[kWarps][kFMax];
  __shared__ uint32_t s_out[kWarps][kFMax];
  __shared__ uint32_t s_slot[kWarps][kFMax];
  __shared__ uint8_t s_ipos[kWarps][kFMax + 4];
  __shared__ uint32_t s_vkey[kWarps][32];
  __shared__ uint16_t s_tab[kWarps][32 * 32];
  __shared__ unsigned int s_nq, s_nbig;
  __shared__ unsigned long long s_qbase, s_bbase;
  __shared__ unsigned long long s_stat[6];  // inserted, conflicts, attempts, cavity, ball, dups
  if (threadIdx.x == 0) {
    s_nq = 0;
    s_nbig = 0;
    for (int k = 0; k < 6; ++k) s_stat[k] = 0;
  }
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t cand = blockIdx.x * kWarps + wid;
  uint32_t status = kCandEmpty, p = kNone;
  if (cand < R) {
    status = cand_status[cand];
    p = cand_p[cand];
  }
  if (status == kCandLocated) {
    unsigned long long prio = (__ldcg(&c.st->stamp) << 32) | (unsigned long long)(p + 1u);
    InsWS w{s_nv[wid], s_nn[wid], s_out[wid], s_slot[wid], s_ipos[wid], s_vkey[wid], s_tab[wid],
            nullptr, nullptr, nullptr, nullptr, 0};
    int nc = (int)cand_nc[cand], nb = (int)cand_nb[cand];
    const uint32_t* src = scratch + (size_t)cand * kScratchStride;
    status = insert_warp(c, w, p, prio, src, nc, src + kCMax, nb, true, __ldcg(&c.st->free_avail),
                         __ldcg(&c.st->bump), c.st->capacity);
    if (status == kCandInserted && lane == 0) {
      Pt P = load_pt(c.pts, p);
      c.cell_hint[cell_of(c, P)] = s_slot[wid][0];
      c.st->anchor = s_slot[wid][0];
      atomicAdd(&s_stat[0], 1ull);
      atomicAdd(&s_stat[3], (unsigned long long)nc);
      atomicAdd(&s_stat[4], (unsigned long long)nb);
    }
  }
  int qslot = -1, bslot = -1;
  if (lane == 0 && cand < R && status != kCandEmpty) {
    atomicAdd(&s_stat[2], 1ull);
    if (status == kCandLost) atomicAdd(&s_stat[1], 1ull);
    if (status == kCandDup) atomicAdd(&s_stat[5], 1ull);
    if (status == kCandLost || status == kCandWalkLimit) qslot = (int)atomicAdd(&s_nq, 1u);
    else if (status == kCandBig) bslot = (int)atomicAdd(&s_nbig, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_qbase = s_nq ? atomicAdd(&c.st->qnext, (unsigned long long)s_nq) : 0;
    s_bbase = s_nbig ? atomicAdd(&c.st->nbig, (unsigned long long)s_nbig) : 0;
    if (s_stat[0]) atomicAdd(&c.st->n_inserted, s_stat[0]);
    if (s_stat[1]) atomicAdd(&c.st->n_conflicts, s_stat[1]);
    if (s_stat[2]) atomicAdd(&c.st->n_attempts, s_stat[2]);
    if (s_stat[3]) atomicAdd(&c.st->sum_cavity, s_stat[3]);
    if (s_stat[4]) atomicAdd(&c.st->sum_ball, s_stat[4]);
    if (s_stat[5]) atomicAdd(&c.st->n_dups, s_stat[5]);
  }
  __syncthreads();
  if (qslot >= 0) qnext[s_qbase + qslot] = p;
  if (bslot >= 0) big[s_bbase + bslot] = p;
}

// Closes a round: the allocator consumed the top of the free list, then the bump pointer;
// slots freed during the round are appended to the free list; the claim stamp advances.
// Warp version (one warp runs the kernel); k_finish is the block version.
__device__ void finish_round_warp(const Ctx& c) {
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
  }
  __threadfence();
  __syncwarp();
}

__global__ void k_finish(Ctx c) {
  // every thread reads the counters before thread 0 rewrites them
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
  }
}

// Points whose cavity exceeds the shared-memory path: inserted one at a time by one warp,
// with global-memory workspaces; nothing else runs concurrently.
__global__ void k_big(Ctx c, const uint32_t* big, uint32_t nbig, BigWS ws) {
  const int lane = threadIdx.x & 31;
  for (uint32_t k = 0; k < nbig; ++k) {
    uint32_t p = big[k];
    Pt P = load_pt(c.pts, p);
    uint32_t t = kNone, steps = 0;
    int s = 0;
    if (lane == 0) {
      uint32_t anchor = __ldcg(&c.st->anchor);
      uint32_t hint = c.point_hint[p];
      if (hint == kNone) hint = c.cell_hint[cell_of(c, P)];
      s = walk_point(c, P, hint, 0, anchor, 1u << 22, &t, &steps);
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
    unsigned long long prio = (__ldcg(&c.st->stamp) << 32) | (unsigned long long)(p + 1u);
    int nc = 0, nb = 0;
    int r = cavity_warp(c, ws.cav, t, P, prio, &nc, &nb);
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
      c.cell_hint[cell_of(c, P)] = ws.ins.slot[0];
      c.st->anchor = ws.ins.slot[0];
      c.st->n_inserted += 1;
      c.st->n_big += 1;
      c.st->sum_cavity += nc;
      c.st->sum_ball += nb;
    }
    __threadfence();
    __syncwarp();
    finish_round_warp(c);
  }
}

// Init (Section 2.1): the first four non-coplanar vertices of the insertion order form a
// positive tetrahedron; four ghost tetrahedra close it (Section 2.6).
__global__ void k_init(Ctx c, uint32_t vbegin, uint32_t vend, uint8_t* vflag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t s = vbegin;
  while (s < vend && vflag[s]) ++s;
  uint32_t i0 = s++;
  while (s < vend && vflag[s]) ++s;
  uint32_t i1 = s++;
  if (i1 >= vend) {
    raise_error(c.st, kErrDegenerate, 0);
    return;
  }
  Pt A = c.pts[i0], B = c.pts[i1];
  while (s < vend && (vflag[s] || collinear_exact(A, B, c.pts[s], c.st))) ++s;
  uint32_t i2 = s++;
  if (i2 >= vend) {
    raise_error(c.st, kErrDegenerate, 1);
    return;
  }
  Pt C = c.pts[i2];
  while (s < vend && (vflag[s] || orient3d(A, B, C, c.pts[s], c.st) == 0)) ++s;
  uint32_t i3 = s;
  if (i3 >= vend) {
    raise_error(c.st, kErrDegenerate, 2);
    return;
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
            nn[t][f] = 4u * u + g;
            break;
          }
        }
      }
    }
  for (int t = 0; t < 5; ++t) {
    c.tets[t].v = make_uint4(tv[t][0], tv[t][1], tv[t][2], tv[t][3]);
    c.tets[t].n = make_uint4(nn[t][0], nn[t][1], nn[t][2], nn[t][3]);
  }
  vflag[i0] = vflag[i1] = vflag[i2] = vflag[i3] = 2;
  c.st->bump = 5;
  c.st->anchor = 0;
  c.st->n_inserted += 4;
}

__global__ void k_build_pts(const double* __restrict__ xyz, const uint32_t* __restrict__ perm,
                            const uint8_t* __restrict__ dup, uint64_t n, uint64_t base,
                            Pt* pts, uint8_t* vflag, uint32_t* point_hint) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t i = perm[s];
    pts[base + s] = make_pt(xyz[3 * (uint64_t)i], xyz[3 * (uint64_t)i + 1], xyz[3 * (uint64_t)i + 2],
                                 (double)(base + i));
    vflag[base + s] = dup[i];
    point_hint[base + s] = kNone;
  }
}

// Finite live tetrahedra with vertex ids mapped to input indices; canonical rotation optional.
__global__ void k_collect(const Tet* __restrict__ tets, uint64_t nslots, const Pt* __restrict__ pts,
                          uint64_t npts, uint32_t* out, unsigned long long* count, uint64_t cap,
                          int canonical) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nslots;
       t += (uint64_t)gridDim.x * blockDim.x) {
    uint4 v = tets[t].v;
    if (tet_dead(v) || ghost_pos(v) >= 0) continue;
    if (v.x >= npts || v.y >= npts || v.z >= npts || v.w >= npts) continue;
    uint32_t r[4] = {(uint32_t)pts[v.x].w, (uint32_t)pts[v.y].w, (uint32_t)pts[v.z].w, (uint32_t)pts[v.w].w};
    if (canonical) {
      // even permutation bringing the smallest id first, then a cyclic turn of the other three
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
    unsigned long long pos = atomicAdd(count, 1ull);
    if (pos < cap) {
      reinterpret_cast<uint4*>(out)[pos] = make_uint4(r[0], r[1], r[2], r[3]);
    }
  }
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
    if (kind == 0) s = orient3d(q[0], q[1], q[2], q[3], st);
    else if (kind == 1) s = insphere(q[0], q[1], q[2], q[3], q[4], st);
    else s = insphere_sos(q[0], q[1], q[2], q[3], q[4], st);
    out[i] = (int8_t)s;
  }
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
  Pt* pts = nullptr;
  uint8_t* vflag = nullptr;
  uint32_t* point_hint = nullptr;
  uint64_t n_pts = 0, cap_pts = 0;
  Tet* tets = nullptr;
  unsigned long long* claim = nullptr;
  uint64_t cap_tets = 0;
  uint32_t* freelist = nullptr;
  uint32_t* pending = nullptr;
  uint64_t cap_free = 0;
  uint32_t* cell_hint = nullptr;
  int cb = 0, cell_hint_cb = -1;
  double lo[3] = {0, 0, 0}, sc[3] = {0, 0, 0};
  DevState* st = nullptr;
  DevState* st_host = nullptr;
  uint32_t Rmax = 0;
  uint32_t *cand_p = nullptr, *cand_t = nullptr, *cand_status = nullptr, *cand_nc = nullptr,
           *cand_nb = nullptr, *scratch = nullptr;
  uint32_t* qnext = nullptr;
  uint32_t* big = nullptr;
  uint64_t cap_q = 0;
  void* bigmem = nullptr;
  BigWS bigws{};
  double* bbox_dev = nullptr;
  bool has_mesh = false;
  uint64_t last_n = 0;
  double alpha = 0.03;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> prof_events;
  unsigned long long next_stamp = 1;
  unsigned long long launches0 = 0;
  dt_stats stats{};
  unsigned last_dev_error = 0, last_dev_info = 0;
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
  c.freelist = h->freelist;
  c.pending = h->pending;
  c.cell_hint = h->cell_hint;
  c.point_hint = h->point_hint;
  c.st = h->st;
  for (int k = 0; k < 3; ++k) {
    c.lo[k] = h->lo[k];
    c.sc[k] = h->sc[k];
  }
  c.cb = h->cb;
  c.max_walk = h->cfg.max_walk_steps ? h->cfg.max_walk_steps : (1u << 16);
  c.coherent = 0;
  c.ntets = (uint32_t)h->cap_tets;
  c.npts = (uint32_t)h->cap_pts;
  return c;
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
  if (grow(h->vflag, h->n_pts, nc, h->stream) != cudaSuccess) return DT_ENOMEM;
  if (grow(h->point_hint, h->n_pts, nc, h->stream) != cudaSuccess) return DT_ENOMEM;
  h->cap_pts = nc;
  return DT_OK;
}

int reserve_tets(dt_handle* h, uint64_t total_pts) {
  double f = h->cfg.tet_capacity_factor > 0 ? h->cfg.tet_capacity_factor : 8.0;
  uint64_t need = (uint64_t)(f * (double)total_pts) + 4096;
  if (need > 0x3FFFFFFFull) need = 0x3FFFFFFFull;  // 4t + facet fits 32 bits
  if (need <= h->cap_tets) return DT_OK;
  uint64_t old = h->cap_tets;
  unsigned long long bump = h->has_mesh ? h->st_host->bump : 0;
  if (grow(h->tets, bump, need, h->stream) != cudaSuccess) return DT_ENOMEM;
  if (grow(h->claim, bump, need, h->stream) != cudaSuccess) return DT_ENOMEM;
  cudaMemsetAsync(h->claim + old, 0, (need - old) * sizeof(unsigned long long), h->stream);
  uint64_t nf = need / 4 + 4096;
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

int reserve_rounds(dt_handle* h, uint64_t qcap) {
  if (!h->cand_p) {
    h->Rmax = 1u << 19;
    uint64_t R = h->Rmax;
    if (cudaMalloc(&h->cand_p, R * 4) || cudaMalloc(&h->cand_t, R * 4) || cudaMalloc(&h->cand_status, R * 4) ||
        cudaMalloc(&h->cand_nc, R * 4) || cudaMalloc(&h->cand_nb, R * 4) ||
        cudaMalloc(&h->scratch, R * kScratchStride * 4))
      return DT_ENOMEM;
    size_t bytes = (size_t)kBigHash * 4 + kBigHash + (size_t)kBigC * 4 + (size_t)kBigF * 4 +
                   (size_t)kBigF * 32 + (size_t)kBigF * 4 * 2 + kBigF + 32 * 4 + 32 * 32 * 2 +
                   (size_t)kBigEdge * 8 + (size_t)kBigEdge * 4 + (size_t)kBigF * 3 * 4 * 2 + 1024;
    if (cudaMalloc(&h->bigmem, bytes)) return DT_ENOMEM;
    char* b = (char*)h->bigmem;
    auto take = [&](size_t n) {
      char* r = b;
      b += (n + 15) & ~size_t(15);
      return r;
    };
    BigWS& w = h->bigws;
    w.ins.ekey = (unsigned long long*)take((size_t)kBigEdge * 8);
    w.ins.nv = (uint4*)take((size_t)kBigF * 16);
    w.ins.nn = (uint4*)take((size_t)kBigF * 16);
    w.cav.hkey = (uint32_t*)take((size_t)kBigHash * 4);
    w.cav.clist = (uint32_t*)take((size_t)kBigC * 4);
    w.cav.blist = (uint32_t*)take((size_t)kBigF * 4);
    w.ins.eval = (uint32_t*)take((size_t)kBigEdge * 4);
    w.ins.hslot = (uint32_t*)take((size_t)kBigF * 3 * 4);
    w.ins.hold = (uint32_t*)take((size_t)kBigF * 3 * 4);
    w.ins.outh = (uint32_t*)take((size_t)kBigF * 4);
    w.ins.slot = (uint32_t*)take((size_t)kBigF * 4);
    w.ins.vkey = (uint32_t*)take(32 * 4);
    w.ins.tab = (uint16_t*)take(32 * 32 * 2);
    w.cav.hval = (uint8_t*)take(kBigHash);
    w.ins.ipos = (uint8_t*)take(kBigF);
    w.cav.hmask = kBigHash - 1;
    w.cav.cmax = kBigC;
    w.cav.bmax = kBigF;
    w.ins.emask = kBigEdge - 1;
  }
  if (qcap > h->cap_q) {
    cudaFree(h->qnext);
    cudaFree(h->big);
    h->qnext = h->big = nullptr;
    if (cudaMalloc(&h->qnext, qcap * 4) || cudaMalloc(&h->big, qcap * 4)) return DT_ENOMEM;
    h->cap_q = qcap;
  }
  return DT_OK;
}

uint32_t choose_segments(dt_handle* h, uint64_t mesh_vertices, uint64_t m) {
  if (h->cfg.segments) return (uint32_t)std::min<uint64_t>(std::min<uint64_t>(h->cfg.segments, h->Rmax), m);
  double r = h->alpha * (double)mesh_vertices;
  uint64_t R = (uint64_t)std::max(1.0, r);
  R = std::min<uint64_t>(R, h->Rmax);
  R = std::min<uint64_t>(R, m);
  return (uint32_t)std::max<uint64_t>(R, 1);
}

// Inserts the vertices [vbegin, vend) (one BRIO round, Moore order) by passes of concurrent
// rounds; failed points are re-keyed with a re-partition transform and retried (Section 3.3).
int run_brio_round(dt_handle* h, uint32_t vbegin, uint32_t vend) {
  Ctx c = make_ctx(h);
  const uint32_t* q = nullptr;
  uint32_t qbase = vbegin;
  uint64_t m = vend - vbegin;
  uint32_t pass = 0;
  uint32_t max_rounds = h->cfg.max_rounds ? h->cfg.max_rounds : (1u << 22);
  int stalled = 0;
  while (m > 0) {
    uint64_t mesh = h->st_host->n_inserted;
    uint64_t before = h->st_host->n_inserted + h->st_host->n_dups;
    uint32_t R = choose_segments(h, mesh, m);
    uint64_t L = (m + R - 1) / R;
    unsigned long long zero2[2] = {0, 0};
    cudaMemcpyAsync(&h->st->qnext, zero2, 16, cudaMemcpyHostToDevice, h->stream);
    const bool prof = (h->cfg.flags & DT_FLAG_PROFILE) != 0;
    if (prof) {
      while (h->prof_events.size() < 6 * L) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return DT_ECUDA;
        h->prof_events.push_back(e);
      }
    }
    for (uint64_t j = 0; j < L; ++j) {
      if (prof) cudaEventRecord(h->prof_events[6 * j], h->stream);
      k_walk<<<(R + 255) / 256, 256, 0, h->stream>>>(c, q, qbase, m, L, j, R, h->vflag, h->cand_p, h->cand_t,
                                                      h->cand_status);
      ++g_kernel_launches;
      if (prof) cudaEventRecord(h->prof_events[6 * j + 1], h->stream);
      if (prof) cudaEventRecord(h->prof_events[6 * j + 2], h->stream);
      k_cavity<<<(R + kWarps - 1) / kWarps, 256, 0, h->stream>>>(c, R, h->cand_p, h->cand_t, h->cand_status,
                                                                  h->cand_nc, h->cand_nb, h->scratch);
      ++g_kernel_launches;
      if (prof) cudaEventRecord(h->prof_events[6 * j + 3], h->stream);
      if (prof) cudaEventRecord(h->prof_events[6 * j + 4], h->stream);
      k_insert<<<(R + kWarps - 1) / kWarps, 256, 0, h->stream>>>(c, R, h->cand_p, h->cand_status, h->cand_nc,
                                                                  h->cand_nb, h->scratch, h->qnext, h->big);
      ++g_kernel_launches;
      if (prof) cudaEventRecord(h->prof_events[6 * j + 5], h->stream);
      k_finish<<<1, 256, 0, h->stream>>>(c);
      ++g_kernel_launches;
      h->stats.n_rounds++;
    }
    h->stats.n_passes++;
    int rc = sync_state(h);
    if (rc != DT_OK) return rc;
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
    if (cudaGetLastError() != cudaSuccess) return DT_ECUDA;
    uint64_t nbig = h->st_host->nbig, nq = h->st_host->qnext;
    if (nbig) {
      Ctx cb = c;
      cb.coherent = 1;
      k_big<<<1, 32, 0, h->stream>>>(cb, h->big, (uint32_t)nbig, h->bigws);
      ++g_kernel_launches;
      rc = sync_state(h);
      if (rc != DT_OK) return rc;
    }
    if (h->stats.n_rounds > max_rounds) return DT_ELIMIT;
    if (nq == 0) break;
    // a pass that inserted nothing three times in a row is a bug, not a schedule
    stalled = (h->st_host->n_inserted + h->st_host->n_dups == before) ? stalled + 1 : 0;
    if (stalled >= 3) return DT_ELIMIT;
    // re-partition the failed points: transformed keys, then sort (Section 3.3)
    transformed_keys(h->pts, h->qnext, nq, h->bbox_dev, h->cfg.seed + 0x51ED2701ull * (pass + 1) + vbegin,
                     h->ows.k0, h->ows.v0, h->stream);
    bool alt = radix_sort_pairs(h->ows.k0, h->ows.v0, h->ows.k1, h->ows.v1, nq, 64, h->ows.hist, h->stream);
    q = alt ? h->ows.v1 : h->ows.v0;
    m = nq;
    ++pass;
  }
  return DT_OK;
}

int insert_impl(dt_handle* h, const double* xyz, uint64_t n) {
  if (n == 0) return h->has_mesh ? DT_OK : DT_EDEGENERATE;
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
  k_build_pts<<<grid_for(n, 256), 256, 0, s>>>(xyz, h->ows.perm, h->ows.dup, n, base, h->pts, h->vflag,
                                                h->point_hint);
  ++g_kernel_launches;
  if (!h->has_mesh) {
    double bb[6];
    if (cudaMemcpyAsync(bb, h->ows.bbox, 48, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;
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
    if (h->cell_hint_cb != cb) {
      cudaFree(h->cell_hint);
      h->cell_hint = nullptr;
      if (cudaMalloc(&h->cell_hint, (size_t)4 << (3 * cb)) != cudaSuccess) return DT_ENOMEM;
      h->cell_hint_cb = cb;
    }
    cudaMemsetAsync(h->cell_hint, 0xFF, (size_t)4 << (3 * cb), s);
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
    if ((rc = run_brio_round(h, (uint32_t)(base + b), (uint32_t)(base + e))) != DT_OK) return rc;
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
  o->reserved[0] = d.n_walk_limit;
  o->reserved[1] = d.free_avail;
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

int dt_clear(dt_handle* h) {
  if (!h) return DT_EINVAL;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  // claim priorities keep growing across triangulations, so stale claims never win
  unsigned long long s = h->has_mesh ? h->st_host->stamp : 0;
  h->next_stamp = std::max(h->next_stamp, s + 1);
  h->has_mesh = false;
  h->n_pts = 0;
  h->last_n = 0;
  h->last_dev_error = h->last_dev_info = 0;
  h->stats = dt_stats{};
  h->launches0 = g_kernel_launches;
  std::memset(h->st_host, 0, sizeof(DevState));
  return cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream) == cudaSuccess ? DT_OK : DT_ECUDA;
}

int dt_insert(dt_handle* h, const double* xyz_dev, uint64_t n) {
  if (!h || (n > 0 && !xyz_dev)) return DT_EINVAL;
  return insert_impl(h, xyz_dev, n);
}

int dt_insert_host(dt_handle* h, const double* xyz_host, uint64_t n) {
  if (!h || (n > 0 && !xyz_host)) return DT_EINVAL;
  double* d = nullptr;
  if (n && cudaMalloc(&d, n * 24) != cudaSuccess) return DT_ENOMEM;
  if (n && cudaMemcpyAsync(d, xyz_host, n * 24, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
    cudaFree(d);
    return DT_ECUDA;
  }
  int rc = insert_impl(h, d, n);
  cudaStreamSynchronize(h->stream);
  cudaFree(d);
  return rc;
}

int dt_batch(dt_handle* h, const double* xyz_dev, const uint64_t* offsets_host, uint32_t n_clouds) {
  (void)xyz_dev;
  (void)offsets_host;
  (void)n_clouds;
  if (!h) return DT_EINVAL;
  return DT_ESTATE;
}

int dt_get_tets(dt_handle* h, uint32_t* tets_dev, uint64_t cap, uint64_t* n_tets, uint64_t* cloud_offsets,
                int canonical) {
  (void)cloud_offsets;
  if (!h || !n_tets || (cap > 0 && !tets_dev)) return DT_EINVAL;
  *n_tets = 0;
  if (!h->has_mesh) return DT_OK;
  cudaStream_t s = h->stream;
  int rc = sync_state(h);
  if (rc != DT_OK) return rc;
  uint64_t slots = h->st_host->bump;
  unsigned long long* cnt = nullptr;
  uint32_t* tmp = nullptr;
  if (cudaMalloc(&cnt, 8) != cudaSuccess) return DT_ENOMEM;
  if (cudaMalloc(&tmp, std::max<uint64_t>(slots, 1) * 16) != cudaSuccess) {
    cudaFree(cnt);
    return DT_ENOMEM;
  }
  cudaMemsetAsync(cnt, 0, 8, s);
  k_collect<<<grid_for(slots, 256), 256, 0, s>>>(h->tets, slots, h->pts, h->cap_pts, tmp, cnt, slots, canonical);
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
  if (canonical && !(h->cfg.flags & DT_FLAG_NO_CANONICAL_SORT) && T > 1) {
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
  } else if (T) {
    cudaMemcpyAsync(tets_dev, tmp, T * 16, cudaMemcpyDeviceToDevice, s);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = DT_ECUDA;
  cudaFree(cnt);
  cudaFree(tmp);
  return rc;
}

int dt_get_tets_host(dt_handle* h, uint32_t* tets_host, uint64_t cap, uint64_t* n_tets, int canonical) {
  if (!h || !n_tets || (cap > 0 && !tets_host)) return DT_EINVAL;
  uint64_t T = 0;
  int rc = dt_get_tets(h, nullptr, 0, &T, nullptr, canonical);
  *n_tets = T;
  if (rc != DT_OK && rc != DT_ETOOSMALL) return rc;
  if (T > cap) return DT_ETOOSMALL;
  if (T == 0) return DT_OK;
  uint32_t* d = nullptr;
  if (cudaMalloc(&d, T * 16) != cudaSuccess) return DT_ENOMEM;
  rc = dt_get_tets(h, d, T, &T, nullptr, canonical);
  if (rc == DT_OK && cudaMemcpy(tets_host, d, T * 16, cudaMemcpyDeviceToHost) != cudaSuccess) rc = DT_ECUDA;
  cudaFree(d);
  return rc;
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
  if (!h || !params_host || n_params != 1410) return DT_EINVAL;
  return DT_ESTATE;
}

void dt_destroy(dt_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  order_ws_free(h->ows);
  cudaFree(h->pts);
  cudaFree(h->vflag);
  cudaFree(h->point_hint);
  cudaFree(h->tets);
  cudaFree(h->claim);
  cudaFree(h->freelist);
  cudaFree(h->pending);
  cudaFree(h->cell_hint);
  cudaFree(h->st);
  if (h->st_host) cudaFreeHost(h->st_host);
  cudaFree(h->cand_p);
  cudaFree(h->cand_t);
  cudaFree(h->cand_status);
  cudaFree(h->cand_nc);
  cudaFree(h->cand_nb);
  cudaFree(h->scratch);
  cudaFree(h->qnext);
  cudaFree(h->big);
  cudaFree(h->bigmem);
  cudaFree(h->bbox_dev);
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
  if (kind < 0 || kind > 2 || (n > 0 && (!pts_dev || !out_dev)) || (kind == 2 && n > 0 && !ids_dev))
    return DT_EINVAL;
  if (n == 0) return DT_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = nullptr;
  if (cudaMalloc(&st, sizeof(DevState)) != cudaSuccess) return DT_ENOMEM;
  cudaMemsetAsync(st, 0, sizeof(DevState), s);
  k_eval_predicates<<<grid_for(n, 128), 128, 0, s>>>(kind, pts_dev, kind == 2 ? ids_dev : nullptr, out_dev, n, st);
  ++g_kernel_launches;
  DevState hs;
  cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  int rc = cudaStreamSynchronize(s) == cudaSuccess ? DT_OK : DT_ECUDA;
  cudaFree(st);
  if (rc == DT_OK && hs.error) rc = map_dev_error(hs.error);
  return rc;
}

}  // extern "C"
