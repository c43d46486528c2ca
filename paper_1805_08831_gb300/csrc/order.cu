// Spatial order of the points (Section 2.3): bounding box, 21-bit quantisation, 63-bit Moore
// keys, BRIO rounds (sizes of Table 2), a stable LSD radix sort by (round, key, index), and
// exact-duplicate detection on runs of equal keys.
//
// The Moore index follows Hamilton's Gray-code construction of the Hilbert curve (each sub-cube
// curve has an entry corner e and an exit direction d; its cells are visited in Gray-code
// order after the transform rotr(l ^ e, d + 1)), closed into a loop at the top level: the
// octant visited w-th (Gray order) is entered at corner ~gray(w) ^ M[w] and left along the
// axis of M[w] ^ M[w + 1], M = {x, 0, z, 0, y, y|z, z, 0}. Here the per-level rule is
// compiled into a 24-state transition table evaluated per point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace dtg {
namespace {

// ------------------------------------------------------------------ Moore transition tables
struct MooreTab {
  uint16_t step[24 * 8];  // (state, cell bits) -> (digit << 8) | next state; state = 3e + d
  uint16_t top[8];        // top-level cell bits -> (digit << 8) | first state
};

constexpr unsigned gray_of(unsigned i) { return i ^ (i >> 1); }
constexpr unsigned gray_rank(unsigned g) { return g ^ (g >> 1) ^ (g >> 2); }
constexpr unsigned ones_below(unsigned i) {
  unsigned c = 0;
  while (i & 1u) {
    ++c;
    i >>= 1;
  }
  return c;
}
constexpr unsigned rot_right3(unsigned b, unsigned r) {
  r %= 3;
  return ((b >> r) | (b << (3 - r))) & 7u;
}
constexpr unsigned rot_left3(unsigned b, unsigned r) {
  r %= 3;
  return ((b << r) | (b >> (3 - r))) & 7u;
}

constexpr MooreTab build_moore() {
  MooreTab T{};
  for (unsigned e = 0; e < 8; ++e)
    for (unsigned d = 0; d < 3; ++d)
      for (unsigned l = 0; l < 8; ++l) {
        unsigned w = gray_rank(rot_right3(l ^ e, d + 1));
        unsigned entry = w == 0 ? 0u : gray_of(2u * ((w - 1u) / 2u));
        unsigned dir = w == 0 ? 0u : ((w & 1u) ? ones_below(w) : ones_below(w - 1u)) % 3u;
        unsigned e2 = e ^ rot_left3(entry, d + 1);
        unsigned d2 = (d + dir + 1) % 3;
        T.step[(e * 3 + d) * 8 + l] = (uint16_t)((w << 8) | (e2 * 3 + d2));
      }
  const unsigned M[8] = {1u, 0u, 4u, 0u, 2u, 6u, 4u, 0u};
  for (unsigned l = 0; l < 8; ++l) {
    unsigned w = gray_rank(l);
    unsigned e = (~gray_of(w) & 7u) ^ M[w];
    unsigned x = M[w] ^ M[(w + 1) & 7u];
    unsigned d = x == 1u ? 0u : (x == 2u ? 1u : 2u);
    T.top[l] = (uint16_t)((w << 8) | (e * 3 + d));
  }
  return T;
}

__constant__ MooreTab kMoore = build_moore();

constexpr int kLevels = 21;
constexpr double kCells = 2097152.0;  // 2^21

__device__ __forceinline__ uint64_t moore_of_cell(uint32_t qx, uint32_t qy, uint32_t qz,
                                                  const uint16_t* step, const uint16_t* top) {
  int i = kLevels - 1;
  unsigned l = ((qx >> i) & 1u) | (((qy >> i) & 1u) << 1) | (((qz >> i) & 1u) << 2);
  unsigned e = top[l];
  uint64_t key = e >> 8;
  unsigned state = e & 255u;
  for (i = kLevels - 2; i >= 0; --i) {
    l = ((qx >> i) & 1u) | (((qy >> i) & 1u) << 1) | (((qz >> i) & 1u) << 2);
    e = step[state * 8 + l];
    key = (key << 3) | (e >> 8);
    state = e & 255u;
  }
  return key;
}

__device__ __forceinline__ uint32_t quantise(double x, double lo, double scale) {
  double t = __dsub_rn(x, lo);
  double s = __dmul_rn(t, scale);
  double f = floor(s);
  f = f < 0.0 ? 0.0 : (f > kCells - 1.0 ? kCells - 1.0 : f);
  return (uint32_t)f;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ------------------------------------------------------------------ bounding box
constexpr int kBoxThreads = 256;
constexpr int kBoxBlocks = 304;  // 2 x 152 SMs

__global__ void k_bbox_partial(const double* __restrict__ xyz, uint64_t n, double* partial,
                               unsigned int* bad) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool b = false;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < 3; ++k) {
      double x = xyz[3 * i + k];
      if (!(fabs(x) <= 1e30)) b = true;  // also catches NaN
      lo[k] = fmin(lo[k], x);
      hi[k] = fmax(hi[k], x);
    }
  }
  if (b) atomicExch(bad, 1u);
  __shared__ double s[6][kBoxThreads];
  for (int k = 0; k < 3; ++k) {
    s[k][threadIdx.x] = lo[k];
    s[3 + k][threadIdx.x] = hi[k];
  }
  __syncthreads();
  for (int w = kBoxThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + w]);
        s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x < 6) partial[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_bbox_final(const double* partial, int nblocks, double* bbox) {
  int k = threadIdx.x;
  if (k >= 6) return;
  double v = k < 3 ? INFINITY : -INFINITY;
  for (int b = 0; b < nblocks; ++b) v = k < 3 ? fmin(v, partial[b * 6 + k]) : fmax(v, partial[b * 6 + k]);
  bbox[k] = v;
}

// ------------------------------------------------------------------ keys
__global__ void k_moore_keys(const double* __restrict__ xyz, uint64_t n, const double* bbox,
                             uint64_t* keys, uint64_t* skeys, uint32_t* svals) {
  __shared__ uint16_t step[24 * 8];
  __shared__ uint16_t top[8];
  for (int i = threadIdx.x; i < 24 * 8; i += blockDim.x) step[i] = kMoore.step[i];
  if (threadIdx.x < 8) top[threadIdx.x] = kMoore.top[threadIdx.x];
  __syncthreads();
  double lo[3], sc[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = bbox[k];
    double ext = bbox[3 + k] - bbox[k];
    sc[k] = ext > 0.0 ? kCells / ext : 0.0;
  }
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t qx = quantise(xyz[3 * i], lo[0], sc[0]);
    uint32_t qy = quantise(xyz[3 * i + 1], lo[1], sc[1]);
    uint32_t qz = quantise(xyz[3 * i + 2], lo[2], sc[2]);
    uint64_t key = moore_of_cell(qx, qy, qz, step, top);
    keys[i] = key;
    skeys[i] = key;
    svals[i] = (uint32_t)i;
  }
}

// Re-partition keys (Section 3.3): coordinates normalised to the box are compressed below a
// random threshold t and expanded above it (t maps to 1/2), then the curve index is shifted.
__global__ void k_transformed_keys(const Pt* __restrict__ pts, const uint32_t* ids, uint64_t m,
                                   const double* bbox, uint64_t seed, uint64_t* keys,
                                   uint32_t* vals) {
  __shared__ uint16_t step[24 * 8];
  __shared__ uint16_t top[8];
  for (int i = threadIdx.x; i < 24 * 8; i += blockDim.x) step[i] = kMoore.step[i];
  if (threadIdx.x < 8) top[threadIdx.x] = kMoore.top[threadIdx.x];
  __syncthreads();
  double lo[3], inv[3], thr[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = bbox[k];
    double ext = bbox[3 + k] - bbox[k];
    inv[k] = ext > 0.0 ? 1.0 / ext : 0.0;
    thr[k] = 0.25 + 0.5 * (double)(mix64(seed + 11 * k + 1) >> 11) * 0x1p-53;
  }
  uint64_t shift = mix64(seed + 97) & ((1ull << 63) - 1);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = ids[i];
    Pt P = pts[v];
    double c[3] = {P.x, P.y, P.z};
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      double u = (c[k] - lo[k]) * inv[k];
      double w = u < thr[k] ? u * (0.5 / thr[k]) : 0.5 + (u - thr[k]) * (0.5 / (1.0 - thr[k]));
      double f = floor(w * kCells);
      f = f < 0.0 ? 0.0 : (f > kCells - 1.0 ? kCells - 1.0 : f);
      q[k] = (uint32_t)f;
    }
    keys[i] = (moore_of_cell(q[0], q[1], q[2], step, top) + shift) & ((1ull << 63) - 1);
    vals[i] = v;
  }
}

__global__ void k_brio_hash(uint64_t n, uint64_t seed, uint64_t* keys, uint32_t* vals) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    keys[i] = mix64((seed ^ i) + 0x9E3779B97F4A7C15ull);
    vals[i] = (uint32_t)i;
  }
}

__global__ void k_brio_assign(const uint32_t* sorted_idx, uint64_t n, uint8_t* rounds, uint32_t* rank) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
       r += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t end = 2048;
    uint8_t k = 0;
    while (r >= end) {
      end *= 7;
      ++k;
    }
    rounds[sorted_idx[r]] = k;
    rank[sorted_idx[r]] = (uint32_t)r;
  }
}

// Exact duplicates: equal coordinates imply equal keys, so they sit in one run of the key
// order, where input indices ascend (stable sort). Each run is scanned by one thread.
__global__ void k_dedup_runs(const uint64_t* __restrict__ skeys, const uint32_t* __restrict__ svals,
                             uint64_t n, const double* __restrict__ xyz, uint8_t* dup) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    if (s > 0 && skeys[s] == skeys[s - 1]) continue;
    uint64_t e = s + 1;
    while (e < n && skeys[e] == skeys[s]) ++e;
    if (e == s + 1) continue;
    for (uint64_t a = s + 1; a < e; ++a) {
      uint32_t ia = svals[a];
      for (uint64_t b = s; b < a; ++b) {
        uint32_t ib = svals[b];
        if (xyz[3 * (uint64_t)ia] == xyz[3 * (uint64_t)ib] &&
            xyz[3 * (uint64_t)ia + 1] == xyz[3 * (uint64_t)ib + 1] &&
            xyz[3 * (uint64_t)ia + 2] == xyz[3 * (uint64_t)ib + 2]) {
          dup[ia] = 1;
          break;
        }
      }
    }
  }
}

__global__ void k_round_keys(const uint32_t* svals, uint64_t n, const uint8_t* rounds, uint64_t* keys) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x)
    keys[s] = rounds[svals[s]];
}

// ------------------------------------------------------------------ batches of clouds
// Cloud of every input index (cloud c holds input rows offsets[c] .. offsets[c + 1]).
__global__ void k_batch_cid(const uint64_t* __restrict__ offsets, uint32_t n_clouds, uint32_t* cid) {
  for (uint32_t c = blockIdx.x; c < n_clouds; c += gridDim.x)
    for (uint64_t i = offsets[c] + threadIdx.x; i < offsets[c + 1]; i += blockDim.x) cid[i] = c;
}

// Bounding box of every cloud (one block per cloud), and the non-finite coordinate check.
__global__ void k_batch_bbox(const double* __restrict__ xyz, const uint64_t* __restrict__ offsets,
                             uint32_t n_clouds, double* bbox, unsigned int* bad) {
  __shared__ double s[6][kBoxThreads];
  for (uint32_t c = blockIdx.x; c < n_clouds; c += gridDim.x) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool b = false;
    for (uint64_t i = offsets[c] + threadIdx.x; i < offsets[c + 1]; i += blockDim.x)
      for (int k = 0; k < 3; ++k) {
        double x = xyz[3 * i + k];
        if (!(fabs(x) <= 1e30)) b = true;
        lo[k] = fmin(lo[k], x);
        hi[k] = fmax(hi[k], x);
      }
    if (b) atomicExch(bad, 1u);
    for (int k = 0; k < 3; ++k) {
      s[k][threadIdx.x] = lo[k];
      s[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int w = kBoxThreads / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w)
        for (int k = 0; k < 3; ++k) {
          s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + w]);
          s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + w]);
        }
      __syncthreads();
    }
    if (threadIdx.x < 6) bbox[6 * (uint64_t)c + threadIdx.x] = s[threadIdx.x][0];
    __syncthreads();
  }
}

// Moore key of every point on its own cloud's 2^21 grid (the same key dt_insert would give the
// cloud on its own).
__global__ void k_batch_moore(const double* __restrict__ xyz, uint64_t n, const uint32_t* __restrict__ cid,
                              const double* __restrict__ bbox, uint64_t* keys, uint64_t* skeys, uint32_t* svals) {
  __shared__ uint16_t step[24 * 8];
  __shared__ uint16_t top[8];
  for (int i = threadIdx.x; i < 24 * 8; i += blockDim.x) step[i] = kMoore.step[i];
  if (threadIdx.x < 8) top[threadIdx.x] = kMoore.top[threadIdx.x];
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const double* B = bbox + 6 * (uint64_t)cid[i];
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      double ext = B[3 + k] - B[k];
      q[k] = quantise(xyz[3 * i + k], B[k], ext > 0.0 ? kCells / ext : 0.0);
    }
    uint64_t key = moore_of_cell(q[0], q[1], q[2], step, top);
    keys[i] = key;
    skeys[i] = key;
    svals[i] = (uint32_t)i;
  }
}

__global__ void k_batch_gather_cid(const uint32_t* __restrict__ svals, uint64_t n, const uint32_t* __restrict__ cid,
                                   uint64_t* keys) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x)
    keys[s] = cid[svals[s]];
}

// Exact duplicates inside a cloud: they share the cloud and the key, so they sit in one run of
// the (cloud, key) order, input indices ascending.
__global__ void k_batch_dedup(const uint32_t* __restrict__ svals, uint64_t n, const uint64_t* __restrict__ keys,
                              const uint32_t* __restrict__ cid, const double* __restrict__ xyz, uint8_t* dup) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t i = svals[s];
    if (s > 0) {
      uint32_t j = svals[s - 1];
      if (keys[j] == keys[i] && cid[j] == cid[i]) continue;
    }
    uint64_t e = s + 1;
    while (e < n && keys[svals[e]] == keys[i] && cid[svals[e]] == cid[i]) ++e;
    for (uint64_t a = s + 1; a < e; ++a) {
      uint32_t ia = svals[a];
      for (uint64_t b = s; b < a; ++b) {
        uint32_t ib = svals[b];
        if (xyz[3 * (uint64_t)ia] == xyz[3 * (uint64_t)ib] &&
            xyz[3 * (uint64_t)ia + 1] == xyz[3 * (uint64_t)ib + 1] &&
            xyz[3 * (uint64_t)ia + 2] == xyz[3 * (uint64_t)ib + 2]) {
          dup[ia] = 1;
          break;
        }
      }
    }
  }
}

// BRIO keys inside each cloud: (cloud, top 32 bits of the hash of the cloud-local index).
__global__ void k_batch_hash(uint64_t n, const uint32_t* __restrict__ cid, const uint64_t* __restrict__ offsets,
                             uint64_t seed, uint64_t* keys, uint32_t* vals) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c = cid[i];
    uint64_t local = i - offsets[c];
    keys[i] = ((uint64_t)c << 32) | (mix64((seed ^ local) + 0x9E3779B97F4A7C15ull) >> 32);
    vals[i] = (uint32_t)i;
  }
}

// BRIO round of every point from its hash rank inside its cloud (Table 2 sizes).
__global__ void k_batch_assign(const uint32_t* __restrict__ sorted_idx, uint64_t n, const uint32_t* __restrict__ cid,
                               const uint64_t* __restrict__ offsets, uint8_t* rounds, uint32_t* rank) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t i = sorted_idx[s];
    uint64_t r = s - offsets[cid[i]];
    uint64_t end = 2048;
    uint8_t k = 0;
    while (r >= end) {
      end *= 7;
      ++k;
    }
    rounds[i] = k;
    rank[i] = (uint32_t)r;
  }
}

// (cloud, round, wave) of every point in the (cloud, key) order. A round joins a mesh of about
// as many vertices as the rounds before it hold.
__global__ void k_batch_round_keys(const uint32_t* __restrict__ svals, uint64_t n, const uint32_t* __restrict__ cid,
                                   const uint64_t* __restrict__ offsets, const uint8_t* __restrict__ rounds,
                                   const uint32_t* __restrict__ rank, double gamma, uint64_t* keys) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < n;
       s += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t i = svals[s];
    uint32_t c = cid[i];
    int r = rounds[i];
    uint64_t nc = offsets[c + 1] - offsets[c];
    uint64_t b = brio_round_begin(r), e = brio_round_begin(r + 1);
    uint64_t m = (e < nc ? e : nc) - b;
    int w = wave_of(rank[i] - b, m, b, gamma);
    keys[s] = ((uint64_t)c << 16) | ((uint64_t)r << 8) | (uint64_t)w;
  }
}

// ------------------------------------------------------------------ radix sort
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys,
                                                             uint64_t n, int shift, uint32_t* hist,
                                                             uint32_t ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  uint64_t start = (uint64_t)blockIdx.x * kTile;
  for (int c = 0; c < kSortItems; ++c) {
    uint64_t i = start + (uint64_t)c * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n, int shift,
    const uint32_t* __restrict__ offs, uint32_t ntiles, uint64_t* okeys, uint32_t* ovals) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wc[kSortThreads / 32][256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  base[tid] = offs[(uint64_t)tid * ntiles + blockIdx.x];
  uint64_t start = (uint64_t)blockIdx.x * kTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kSortItems; ++c) {
    for (int w = 0; w < kSortThreads / 32; ++w) wc[w][tid] = 0;
    __syncthreads();
    uint64_t i = start + (uint64_t)c * kSortThreads + tid;
    bool valid = i < n;
    uint64_t k = valid ? keys[i] : 0;
    uint32_t v = valid ? vals[i] : 0;
    unsigned d = valid ? (unsigned)((k >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t s = base[tid];
      for (int w = 0; w < kSortThreads / 32; ++w) {
        uint32_t x = wc[w][tid];
        wc[w][tid] = s;
        s += x;
      }
      base[tid] = s;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = wc[warp][d] + rank;
      okeys[pos] = k;
      ovals[pos] = v;
    }
    __syncthreads();
  }
}

// The same pass with the tile ranked in shared memory first: every element gets its stable
// position inside the tile's digit runs (chunks, then warps, then lanes in order, as above), and
// the runs are then written out contiguously, so consecutive threads write consecutive addresses
// of one digit's run instead of one scattered element each.
constexpr size_t kScatterSmem = (size_t)kTile * 8 + (size_t)kTile * 4 + (size_t)(kSortThreads / 32) * 256 * 4 +
                                3 * 256 * 4;

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter_tiled(
    const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n, int shift,
    const uint32_t* __restrict__ offs, uint32_t ntiles, uint64_t* okeys, uint32_t* ovals) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(sm);
  uint32_t* sv = reinterpret_cast<uint32_t*>(sm + (size_t)kTile * 8);
  uint32_t(*wc)[256] = reinterpret_cast<uint32_t(*)[256]>(sm + (size_t)kTile * 12);
  uint32_t* lstart = reinterpret_cast<uint32_t*>(sm + (size_t)kTile * 12 + (size_t)(kSortThreads / 32) * 1024);
  uint32_t* lnext = lstart + 256;
  uint32_t* gbase = lnext + 256;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t start = (uint64_t)blockIdx.x * kTile;
  const uint32_t tn = (uint32_t)((n - start) < (uint64_t)kTile ? (n - start) : (uint64_t)kTile);
  gbase[tid] = offs[(uint64_t)tid * ntiles + blockIdx.x];
  // the tile's digit counts, then their exclusive scan: where each digit's run starts in the tile
  lnext[tid] = 0;
  __syncthreads();
  for (int c = 0; c < kSortItems; ++c) {
    const uint32_t j = (uint32_t)c * kSortThreads + tid;
    if (j < tn) atomicAdd(&lnext[(keys[start + j] >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (warp == 0) {
    uint32_t v[8], acc = 0;
    for (int k = 0; k < 8; ++k) v[k] = lnext[lane * 8 + k];
    for (int k = 0; k < 8; ++k) acc += v[k];
    uint32_t incl = acc;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t run = incl - acc;
    for (int k = 0; k < 8; ++k) {
      lstart[lane * 8 + k] = run;
      run += v[k];
    }
  }
  __syncthreads();
  lnext[tid] = lstart[tid];
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kSortItems; ++c) {
    for (int w = 0; w < kSortThreads / 32; ++w) wc[w][tid] = 0;
    __syncthreads();
    const uint32_t j = (uint32_t)c * kSortThreads + tid;
    const bool valid = j < tn;
    const uint64_t k = valid ? keys[start + j] : 0;
    const uint32_t v = valid ? vals[start + j] : 0;
    const unsigned d = valid ? (unsigned)((k >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    const unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wc[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t x0 = lnext[tid];
      for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t x = wc[w][tid];
        wc[w][tid] = x0;
        x0 += x;
      }
      lnext[tid] = x0;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wc[warp][d] + rank;
      sk[pos] = k;
      sv[pos] = v;
    }
    __syncthreads();
  }
  // the runs, in order: position j of the tile holds digit d's (j - lstart[d])-th element
  for (uint32_t j = tid; j < tn; j += kSortThreads) {
    const uint64_t k = sk[j];
    const unsigned d = (unsigned)((k >> shift) & 255u);
    const uint64_t g = (uint64_t)gbase[d] + (j - lstart[d]);
    okeys[g] = k;
    ovals[g] = sv[j];
  }
}

// Exclusive scan of a uint32 array, 4096 elements per block, recursive on block sums.
constexpr int kScanThreads = 1024;
constexpr int kScanTile = kScanThreads * 4;

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(uint32_t* data, uint64_t len, uint32_t* sums) {
  __shared__ uint32_t ws[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t i0 = (uint64_t)blockIdx.x * kScanTile + 4 * (uint64_t)tid;
  uint32_t v[4];
  uint32_t tot = 0;
  for (int k = 0; k < 4; ++k) {
    v[k] = (i0 + k < len) ? data[i0 + k] : 0u;
    uint32_t x = v[k];
    v[k] = tot;
    tot += x;
  }
  uint32_t inc = tot;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    uint32_t x = ws[lane];
    uint32_t y = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t z = __shfl_up_sync(0xFFFFFFFFu, y, o);
      if (lane >= o) y += z;
    }
    ws[lane] = y - x;
    if (lane == 31) sums[blockIdx.x] = y;
  }
  __syncthreads();
  uint32_t off = ws[warp] + inc - tot;
  for (int k = 0; k < 4; ++k)
    if (i0 + k < len) data[i0 + k] = v[k] + off;
}

__global__ void k_scan_add(uint32_t* data, uint64_t len, const uint32_t* sums) {
  uint32_t add = sums[blockIdx.x];
  uint64_t i0 = (uint64_t)blockIdx.x * kScanTile;
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (i0 + k < len) data[i0 + k] += add;
}

void scan_exclusive(uint32_t* data, uint64_t len, uint32_t* scratch, cudaStream_t s) {
  uint64_t nb = (len + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, s>>>(data, len, scratch);
  ++g_kernel_launches;
  if (nb > 1) {
    scan_exclusive(scratch, nb, scratch + nb, s);
    k_scan_add<<<(unsigned)nb, 256, 0, s>>>(data, len, scratch);
    ++g_kernel_launches;
  }
}

unsigned grid_for(uint64_t n, int threads) {
  uint64_t b = (n + threads - 1) / threads;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 16));
}

}  // namespace

unsigned long long g_kernel_launches = 0;

uint64_t brio_round_end(int r) {
  uint64_t e = 2048;
  for (int i = 0; i < r; ++i) e *= 7;
  return e;
}

// Histogram and scan entries of one radix sort of n keys (compile-time, so fixed scratch areas
// can be checked against it).
constexpr uint64_t radix_hist_entries_for(uint64_t n) {
  uint64_t tiles = (n + kTile - 1) / kTile;
  uint64_t len = 256 * (tiles > 1 ? tiles : 1);
  uint64_t extra = 0, l = len;
  while (l > 1) {
    l = (l + kScanTile - 1) / kScanTile;
    extra += l;
  }
  return len + extra + 64;
}

uint64_t radix_hist_entries(uint64_t n) { return radix_hist_entries_for(n); }

void prefix_sum_exclusive(uint32_t* data, uint64_t len, uint32_t* scratch, cudaStream_t s) {
  if (len) scan_exclusive(data, len, scratch, s);
}

bool radix_sort_pairs(uint64_t* k, uint32_t* v, uint64_t* ka, uint32_t* va, uint64_t n, int bits,
                      uint32_t* hist, cudaStream_t s) {
  return radix_sort_pairs_bits(k, v, ka, va, n, 0, bits, hist, s);
}

// The tiled scatter needs more than the default 48 KB of dynamic shared memory: opt in once per
// process (every device of this library runs the same build).
bool tiled_scatter_ready() {
  static int state = 0;  // 0 unknown, 1 ready, -1 not available
  if (state == 0) {
    if (std::getenv("DT_SORT_SCATTER_PLAIN")) state = -1;
    else state = cudaFuncSetAttribute(k_radix_scatter_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kScatterSmem) == cudaSuccess ? 1 : -1;
  }
  return state == 1;
}

bool radix_sort_pairs_bits(uint64_t* k, uint32_t* v, uint64_t* ka, uint32_t* va, uint64_t n, int lo_bit,
                           int hi_bit, uint32_t* hist, cudaStream_t s) {
  if (n <= 1) return false;
  uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
  uint64_t len = 256ull * ntiles;
  bool alt = false;
  for (int shift = lo_bit; shift < hi_bit; shift += 8) {
    uint64_t* sk = alt ? ka : k;
    uint32_t* sv = alt ? va : v;
    uint64_t* dk = alt ? k : ka;
    uint32_t* dv = alt ? v : va;
    k_radix_hist<<<ntiles, kSortThreads, 0, s>>>(sk, n, shift, hist, ntiles);
    ++g_kernel_launches;
    scan_exclusive(hist, len, hist + len, s);
    if (tiled_scatter_ready())
      k_radix_scatter_tiled<<<ntiles, kSortThreads, kScatterSmem, s>>>(sk, sv, n, shift, hist, ntiles, dk, dv);
    else
      k_radix_scatter<<<ntiles, kSortThreads, 0, s>>>(sk, sv, n, shift, hist, ntiles, dk, dv);
    ++g_kernel_launches;
    alt = !alt;
  }
  return alt;
}

cudaError_t order_ws_reserve(OrderWS& ws, uint64_t n) {
  if (n <= ws.cap && ws.keys) return cudaSuccess;
  order_ws_free(ws);
  uint64_t c = std::max<uint64_t>(n, 1024);
  cudaError_t e;
  if ((e = cudaMalloc(&ws.keys, c * 8)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.k0, c * 8)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.k1, c * 8)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.v0, c * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.v1, c * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.rounds, c)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.dup, c)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.perm, c * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.rank, c * 4)) != cudaSuccess) return e;
  ws.hist_cap = radix_hist_entries(c);
  if ((e = cudaMalloc(&ws.hist, ws.hist_cap * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.bbox, 6 * 8)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.partial, kBoxBlocks * 6 * 8)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ws.bad, 4)) != cudaSuccess) return e;
  ws.cap = c;
  return cudaSuccess;
}

void order_ws_free(OrderWS& ws) {
  cudaFree(ws.keys);
  cudaFree(ws.k0);
  cudaFree(ws.k1);
  cudaFree(ws.v0);
  cudaFree(ws.v1);
  cudaFree(ws.rounds);
  cudaFree(ws.dup);
  cudaFree(ws.perm);
  cudaFree(ws.rank);
  cudaFree(ws.hist);
  cudaFree(ws.bbox);
  cudaFree(ws.partial);
  cudaFree(ws.bad);
  ws = OrderWS();
}

// S1..S4 on a workspace that already holds room for n points (allocates nothing).
int order_points_ws(const double* xyz, uint64_t n, uint64_t seed, OrderWS& ws, cudaStream_t s) {
  if (n == 0) return DT_OK;
  cudaMemsetAsync(ws.bad, 0, 4, s);
  cudaMemsetAsync(ws.dup, 0, n, s);
  k_bbox_partial<<<kBoxBlocks, kBoxThreads, 0, s>>>(xyz, n, ws.partial, ws.bad);
  ++g_kernel_launches;
  k_bbox_final<<<1, 32, 0, s>>>(ws.partial, kBoxBlocks, ws.bbox);
  ++g_kernel_launches;
  unsigned g = grid_for(n, 256);
  k_moore_keys<<<g, 256, 0, s>>>(xyz, n, ws.bbox, ws.keys, ws.k0, ws.v0);
  ++g_kernel_launches;
  // global Moore order (stable, so input indices ascend inside runs of equal keys)
  bool alt = radix_sort_pairs(ws.k0, ws.v0, ws.k1, ws.v1, n, 64, ws.hist, s);
  uint64_t* sk = alt ? ws.k1 : ws.k0;
  uint32_t* sv = alt ? ws.v1 : ws.v0;
  k_dedup_runs<<<g, 256, 0, s>>>(sk, sv, n, xyz, ws.dup);
  ++g_kernel_launches;
  // keep the key order in perm while the BRIO ranks use the sort buffers
  cudaMemcpyAsync(ws.perm, sv, n * 4, cudaMemcpyDeviceToDevice, s);
  k_brio_hash<<<g, 256, 0, s>>>(n, seed, ws.k0, ws.v0);
  ++g_kernel_launches;
  bool alt2 = radix_sort_pairs(ws.k0, ws.v0, ws.k1, ws.v1, n, 64, ws.hist, s);
  k_brio_assign<<<g, 256, 0, s>>>(alt2 ? ws.v1 : ws.v0, n, ws.rounds, ws.rank);
  ++g_kernel_launches;
  // stable sort of the key order by round
  k_round_keys<<<g, 256, 0, s>>>(ws.perm, n, ws.rounds, ws.k0);
  ++g_kernel_launches;
  cudaMemcpyAsync(ws.v0, ws.perm, n * 4, cudaMemcpyDeviceToDevice, s);
  bool alt3 = radix_sort_pairs(ws.k0, ws.v0, ws.k1, ws.v1, n, 8, ws.hist, s);
  cudaMemcpyAsync(ws.perm, alt3 ? ws.v1 : ws.v0, n * 4, cudaMemcpyDeviceToDevice, s);
  unsigned int bad = 0;
  cudaMemcpyAsync(&bad, ws.bad, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;
  if (bad) return DT_EINVAL;
  return DT_OK;
}

int order_points(const double* xyz, uint64_t n, uint64_t seed, OrderWS& ws, cudaStream_t s) {
  if (n == 0) return DT_OK;
  if (order_ws_reserve(ws, n) != cudaSuccess) return DT_ENOMEM;
  return order_points_ws(xyz, n, seed, ws, s);
}

int order_batch(const double* xyz, uint64_t n, const uint64_t* offsets_dev, uint32_t n_clouds, uint64_t seed,
                double gamma, OrderWS& ws, uint32_t* cid, double* cbox, cudaStream_t s) {
  if (n == 0) return DT_OK;
  int cbits = 8;
  while (cbits < 32 && (1ull << cbits) < n_clouds) cbits += 8;
  cudaMemsetAsync(ws.bad, 0, 4, s);
  cudaMemsetAsync(ws.dup, 0, n, s);
  unsigned gc = (unsigned)std::min<uint32_t>(n_clouds, 152u * 16);
  k_batch_cid<<<gc, 256, 0, s>>>(offsets_dev, n_clouds, cid);
  k_batch_bbox<<<gc, kBoxThreads, 0, s>>>(xyz, offsets_dev, n_clouds, cbox, ws.bad);
  unsigned g = grid_for(n, 256);
  k_batch_moore<<<g, 256, 0, s>>>(xyz, n, cid, cbox, ws.keys, ws.k0, ws.v0);
  g_kernel_launches += 3;
  // (cloud, key, index) order: Moore keys, then a stable sort by cloud
  bool alt = radix_sort_pairs(ws.k0, ws.v0, ws.k1, ws.v1, n, 64, ws.hist, s);
  uint32_t* sv = alt ? ws.v1 : ws.v0;
  uint32_t* ov = alt ? ws.v0 : ws.v1;
  uint64_t* sk = alt ? ws.k1 : ws.k0;
  uint64_t* ok = alt ? ws.k0 : ws.k1;
  k_batch_gather_cid<<<g, 256, 0, s>>>(sv, n, cid, sk);
  ++g_kernel_launches;
  bool alt2 = radix_sort_pairs_bits(sk, sv, ok, ov, n, 0, cbits, ws.hist, s);
  uint32_t* kv = alt2 ? ov : sv;
  k_batch_dedup<<<g, 256, 0, s>>>(kv, n, ws.keys, cid, xyz, ws.dup);
  ++g_kernel_launches;
  cudaMemcpyAsync(ws.perm, kv, n * 4, cudaMemcpyDeviceToDevice, s);
  // BRIO ranks inside each cloud
  k_batch_hash<<<g, 256, 0, s>>>(n, cid, offsets_dev, seed, ws.k0, ws.v0);
  ++g_kernel_launches;
  bool alt3 = radix_sort_pairs_bits(ws.k0, ws.v0, ws.k1, ws.v1, n, 0, 32 + cbits, ws.hist, s);
  k_batch_assign<<<g, 256, 0, s>>>(alt3 ? ws.v1 : ws.v0, n, cid, offsets_dev, ws.rounds, ws.rank);
  ++g_kernel_launches;
  // stable sort of the (cloud, key) order by (cloud, round, wave)
  k_batch_round_keys<<<g, 256, 0, s>>>(ws.perm, n, cid, offsets_dev, ws.rounds, ws.rank, gamma, ws.k0);
  ++g_kernel_launches;
  cudaMemcpyAsync(ws.v0, ws.perm, n * 4, cudaMemcpyDeviceToDevice, s);
  bool alt4 = radix_sort_pairs_bits(ws.k0, ws.v0, ws.k1, ws.v1, n, 0, cbits + 16, ws.hist, s);
  cudaMemcpyAsync(ws.perm, alt4 ? ws.v1 : ws.v0, n * 4, cudaMemcpyDeviceToDevice, s);
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

void transformed_keys(const Pt* pts, const uint32_t* ids, uint64_t m, const double* bbox,
                      uint64_t seed, uint64_t* keys_out, uint32_t* vals_out, cudaStream_t s) {
  if (m == 0) return;
  k_transformed_keys<<<grid_for(m, 256), 256, 0, s>>>(pts, ids, m, bbox, seed, keys_out, vals_out);
  ++g_kernel_launches;
}

}  // namespace dtg

// ------------------------------------------------------------------ ordering without allocation
// Scratch of dt_order_noalloc: a file-scope device array, present on every device that loads
// the library, reused by every call (see include/dt.h).
namespace dtg {
namespace {

constexpr uint64_t kNoAllocMax = DT_NOALLOC_MAX_POINTS;
constexpr uint64_t kNoAllocHist = radix_hist_entries_for(kNoAllocMax);
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffK0 = 0;
constexpr size_t kOffK1 = kOffK0 + align256(kNoAllocMax * 8);
constexpr size_t kOffV0 = kOffK1 + align256(kNoAllocMax * 8);
constexpr size_t kOffV1 = kOffV0 + align256(kNoAllocMax * 4);
constexpr size_t kOffDup = kOffV1 + align256(kNoAllocMax * 4);
constexpr size_t kOffHist = kOffDup + align256(kNoAllocMax);
constexpr size_t kOffBox = kOffHist + align256(kNoAllocHist * 4);
constexpr size_t kOffPart = kOffBox + align256(6 * 8);
constexpr size_t kOffBad = kOffPart + align256(kBoxBlocks * 6 * 8);
constexpr size_t kOffRank = kOffBad + 256;
constexpr size_t kNoAllocBytes = kOffRank + align256(kNoAllocMax * 4);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[1024] = {};

// Host address of the device array on the current device, looked up once per device.
int noalloc_scratch(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 1024) return DT_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DT_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = static_cast<char*>(g_noalloc_ptr[dev]);
  return DT_OK;
}

}  // namespace
}  // namespace dtg

extern "C" int dt_order_noalloc(const double* xyz_dev, uint64_t n, uint64_t seed, uint64_t* keys_dev,
                                uint32_t* perm_dev, uint8_t* rounds_dev, void* stream) {
  using namespace dtg;
  if (n > kNoAllocMax) return DT_EINVAL;
  if (n > 0 && (!xyz_dev || !keys_dev || !perm_dev || !rounds_dev)) return DT_EINVAL;
  if (n == 0) return DT_OK;
  char* base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != DT_OK) return rc;
  OrderWS ws;
  ws.cap = kNoAllocMax;
  ws.keys = keys_dev;
  ws.perm = perm_dev;
  ws.rounds = rounds_dev;
  ws.k0 = reinterpret_cast<uint64_t*>(base + kOffK0);
  ws.k1 = reinterpret_cast<uint64_t*>(base + kOffK1);
  ws.v0 = reinterpret_cast<uint32_t*>(base + kOffV0);
  ws.v1 = reinterpret_cast<uint32_t*>(base + kOffV1);
  ws.dup = reinterpret_cast<uint8_t*>(base + kOffDup);
  ws.hist = reinterpret_cast<uint32_t*>(base + kOffHist);
  ws.hist_cap = kNoAllocHist;
  ws.bbox = reinterpret_cast<double*>(base + kOffBox);
  ws.partial = reinterpret_cast<double*>(base + kOffPart);
  ws.bad = reinterpret_cast<unsigned int*>(base + kOffBad);
  ws.rank = reinterpret_cast<uint32_t*>(base + kOffRank);
  return order_points_ws(xyz_dev, n, seed, ws, static_cast<cudaStream_t>(stream));
}
