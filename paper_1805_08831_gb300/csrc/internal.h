// Host-side declarations shared by the translation units of the library (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dt.h"
#include "common.cuh"

namespace dtg {

// Kernels launched by this library (all handles), for the launch counts the bench reports.
extern unsigned long long g_kernel_launches;

// ---------------------------------------------------------------- order.cu (S1-S4)
// Device workspace for ordering up to `cap` points.
struct OrderWS {
  uint64_t cap = 0;
  uint64_t* keys = nullptr;      // Moore key per input index
  uint64_t* k0 = nullptr;        // sort ping-pong keys
  uint64_t* k1 = nullptr;
  uint32_t* v0 = nullptr;        // sort ping-pong values
  uint32_t* v1 = nullptr;
  uint8_t* rounds = nullptr;     // BRIO round per input index
  uint8_t* dup = nullptr;        // 1 = exact duplicate of a smaller input index
  uint32_t* perm = nullptr;      // insertion order: s-th point -> input index
  uint32_t* rank = nullptr;      // BRIO hash rank per input index
  uint32_t* hist = nullptr;      // radix histograms / scan scratch
  uint64_t hist_cap = 0;
  double* bbox = nullptr;        // [6] lo xyz, hi xyz
  double* partial = nullptr;     // per-block bbox partials
  unsigned int* bad = nullptr;   // non-finite or out-of-range coordinate seen
};

cudaError_t order_ws_reserve(OrderWS& ws, uint64_t n);
void order_ws_free(OrderWS& ws);

// S1..S4 for n points xyz (device, [n,3]). Fills ws.keys, ws.rounds, ws.dup (by input index)
// and ws.perm (insertion order). Returns DT_OK, DT_EINVAL (bad coordinates) or DT_ECUDA.
int order_points(const double* xyz, uint64_t n, uint64_t seed, OrderWS& ws, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on bits [0, bits) of the keys. Ping-pongs between
// (k, v) and (ka, va); returns true when the sorted result ended in (ka, va).
bool radix_sort_pairs(uint64_t* k, uint32_t* v, uint64_t* ka, uint32_t* va, uint64_t n, int bits,
                      uint32_t* hist, cudaStream_t s);
// The same on bits [lo_bit, hi_bit) only (a stable sort by those bits).
bool radix_sort_pairs_bits(uint64_t* k, uint32_t* v, uint64_t* ka, uint32_t* va, uint64_t n, int lo_bit,
                           int hi_bit, uint32_t* hist, cudaStream_t s);
uint64_t radix_hist_entries(uint64_t n);

// Cumulative end of BRIO round r (Section 2.3 / Table 2): 2048 * 7^r.
uint64_t brio_round_end(int r);

// Keys under a re-partition transform (Section 3.3): per-axis piecewise-linear compression
// below a random threshold and expansion above it, then a circular shift of the curve.
void transformed_keys(const Pt* pts, const uint32_t* ids, uint64_t m, const double* bbox,
                      uint64_t seed, uint64_t* keys_out, uint32_t* vals_out, cudaStream_t s);

}  // namespace dtg
