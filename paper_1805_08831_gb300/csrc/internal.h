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

// ---------------------------------------------------------------- waves (both engines)
// A BRIO round of m points joins a mesh of about n0 vertices in waves: each wave takes
// ceil(gamma * N) more points of the round (N = mesh size before the wave), so the number of
// concurrent insertions can follow the mesh as it grows. Points go to waves by their hash rank
// inside the round (a uniformly random subset per wave). At most kMaxWaves waves per round.
constexpr int kMaxWaves = 255;

// End (exclusive, in ranks) of wave k of a round of m points joining n0 vertices.
__host__ __device__ inline uint64_t wave_end(uint64_t m, uint64_t n0, double gamma, int k) {
  double N = (double)(n0 < 4 ? 4 : n0);
  uint64_t acc = 0;
  for (int i = 0; i <= k && acc < m; ++i) {
    double w = ceil(gamma * N);
    uint64_t wi = w < 1.0 ? 1 : (uint64_t)w;
    acc = (i == kMaxWaves - 1 || acc + wi > m) ? m : acc + wi;
    N += (double)wi;
  }
  return acc;
}

// Wave of the point of rank r (0 <= r < m) inside its round.
__host__ __device__ inline int wave_of(uint64_t r, uint64_t m, uint64_t n0, double gamma) {
  double N = (double)(n0 < 4 ? 4 : n0);
  uint64_t acc = 0;
  for (int i = 0; i < kMaxWaves; ++i) {
    double w = ceil(gamma * N);
    uint64_t wi = w < 1.0 ? 1 : (uint64_t)w;
    acc = (i == kMaxWaves - 1 || acc + wi > m) ? m : acc + wi;
    if (r < acc) return i;
    N += (double)wi;
  }
  return kMaxWaves - 1;
}

// First input rank of BRIO round r (cumulative sizes of Table 2: 2048, x 7 per round).
__host__ __device__ inline uint64_t brio_round_begin(int r) {
  uint64_t e = 0, s = 2048;
  for (int i = 0; i < r; ++i) {
    e = s;
    s *= 7;
  }
  return e;
}

// ---------------------------------------------------------------- batch of clouds
// One cloud of a batch. Its vertices are the sorted positions [vb, ve) (the same rows as its
// input), its tetrahedra the slots [tb, tb + tcap).
struct BatchCloud {
  uint32_t vb, ve;
  uint32_t tb, tcap;
  float lo[3], sc[3];  // 8 x 8 x 8 hint grid over the cloud's box
  uint32_t used;       // out: slots used (from tb)
  uint32_t status;     // out: 0 = triangulated, else the device error code (kErr*)
  uint32_t info;       // out: the error's detail
  uint32_t inserted;   // out: vertices in the triangulation
};

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

// S1..S4 for a batch of n_clouds clouds back to back (cloud c = input rows offsets_dev[c] ..
// offsets_dev[c + 1], device array): each cloud gets its own box, Moore keys, duplicates and
// BRIO ranks (ws.keys, ws.dup, ws.rounds, ws.rank by input index), and ws.perm orders the points
// by (cloud, round, wave, key, index), so every cloud keeps its input rows' positions and every
// wave (wave_of with gamma, n0 = the round's first rank) is a contiguous range. cid [n] and
// cbox [6 n_clouds] (device) receive the cloud of every input index and every cloud's box.
// Enqueues only (no host synchronisation, so it can be captured into a graph): ws.bad becomes
// non-zero on a non-finite or |x| > 1e30 coordinate.
int order_batch(const double* xyz, uint64_t n, const uint64_t* offsets_dev, uint32_t n_clouds, uint64_t seed,
                double gamma, OrderWS& ws, uint32_t* cid, double* cbox, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on bits [0, bits) of the keys. Ping-pongs between
// (k, v) and (ka, va); returns true when the sorted result ended in (ka, va).
bool radix_sort_pairs(uint64_t* k, uint32_t* v, uint64_t* ka, uint32_t* va, uint64_t n, int bits,
                      uint32_t* hist, cudaStream_t s);
// The same on bits [lo_bit, hi_bit) only (a stable sort by those bits).
bool radix_sort_pairs_bits(uint64_t* k, uint32_t* v, uint64_t* ka, uint32_t* va, uint64_t n, int lo_bit,
                           int hi_bit, uint32_t* hist, cudaStream_t s);
uint64_t radix_hist_entries(uint64_t n);
// In-place exclusive prefix sum of data[0, len) (device); scratch holds radix_hist_entries(len).
void prefix_sum_exclusive(uint32_t* data, uint64_t len, uint32_t* scratch, cudaStream_t s);

// Cumulative end of BRIO round r (Section 2.3 / Table 2): 2048 * 7^r.
uint64_t brio_round_end(int r);

// Keys under a re-partition transform (Section 3.3): per-axis piecewise-linear compression
// below a random threshold and expansion above it, then a circular shift of the curve.
void transformed_keys(const Pt* pts, const uint32_t* ids, uint64_t m, const double* bbox,
                      uint64_t seed, uint64_t* keys_out, uint32_t* vals_out, cudaStream_t s);

// ---------------------------------------------------------------- async.cu (one launch per pass)
struct Ctx;
struct InsertLog;
// Points q[0, m) (or the vertex range qbase + [0, m) when q is null) in W contiguous segments
// of L points, segment w inserted by warp w in order. Points that lose or walk past max_walk
// steps go to lose_out (queue lose_q), cavities too large for a warp's workspace to big_out.
struct AsyncIO {
  const uint32_t* q;
  uint32_t qbase;
  uint64_t m, L;
  uint32_t W;
  uint32_t max_walk;
  uint32_t* lose_out;
  int lose_q;
  uint32_t* big_out;
  int big_q;
  uint32_t* exact_out;  // predicates the FP32 stage cannot decide: the round-based engine's
  int exact_q;
  const uint32_t* bounds;  // W + 1 segment starts (learned schedule), or null: equal segments of L
  void* big_ws;         // global-memory workspaces a warp may borrow for a large cavity (or null)
  unsigned int* big_busy;  // one word per workspace: 0 free, 1 borrowed
  uint32_t big_n;       // workspaces
  uint32_t ball_start;  // 1: try the previous ball's tetrahedra as the start before walking
};
// Enqueues the asynchronous insertion of one pass and the close of its allocator. lock: one
// word per tetrahedron slot, all zero before and after.
int async_launch(const Ctx& c, const AsyncIO& io, uint32_t* lock, const uint8_t* vflag, const InsertLog& lg,
                 cudaStream_t s);
// Warps of the asynchronous kernel that can be resident on the current device at once.
int async_max_warps();
// The same insertion for cavities beyond the main kernel's shared-memory workspaces: io.W warps
// with one global-memory workspace of async_big_ws_bytes() each at ws (device). Points whose
// cavities exceed even these go to io.big_out.
size_t async_big_ws_bytes();
int async_launch_big(const Ctx& c, const AsyncIO& io, uint32_t* lock, const uint8_t* vflag, const InsertLog& lg,
                     void* ws, cudaStream_t s);

// ---------------------------------------------------------------- batch.cu (dt_batch)
size_t batch_ws_stride();       // bytes of one warp's workspace
uint32_t batch_hint_fine();     // fine hint cells per cloud
uint32_t batch_hint_coarse();   // coarse hint cells per cloud
int batch_cb();                 // bits per axis of a cloud's fine hint grid
int batch_shapes(int* shapes, int max_n);  // block shapes: warps | (min blocks per SM << 8)
int batch_blocks_per_sm(int shape);         // resident blocks per SM of a shape
constexpr int kBatchStatSlots = 11;      // accumulators batch_launch adds into
// One persistent launch over the clouds order[0 .. n_clouds) (see batch.cu); *next must be 0.
int batch_launch(int shape, unsigned blocks, const Ctx& c, BatchCloud* clouds, const uint32_t* order, uint32_t n_clouds,
                 unsigned int* next, uint8_t* vflag, uint32_t* list_a, uint32_t* list_b, uint32_t* list_big,
                 uint32_t* hint_fine, uint32_t* hint_coarse, DevState* states, char* wsmem, size_t wsstride,
                 float alpha, double gamma, const float* eta, unsigned long long* stats, cudaStream_t s);
// Per-cloud hint grids from the clouds' boxes cbox [6 n_clouds], and the FP32 stage's error
// term eta (from the largest |coordinate| of the batch) into *eta, on the device.
void batch_prepare(BatchCloud* clouds, const double* cbox, uint32_t n_clouds, float* eta, cudaStream_t s);
// Resets the clouds list[0 .. n_list) (all clouds when list is null) for a new launch.
void batch_reset(const BatchCloud* clouds, const uint32_t* list, uint32_t n_list, unsigned long long* claim,
                 uint32_t* hint_fine, uint32_t* hint_coarse, const uint8_t* dup_sorted, uint8_t* vflag,
                 uint32_t* point_hint, cudaStream_t s);
// Finite tetrahedra per cloud with cloud-local ids: pass 0 counts into counts[c], pass 1
// writes cloud c's from out_off[c].
void batch_collect(const BatchCloud* clouds, uint32_t n_clouds, const Tet* tets, const Pt* pts, const uint64_t* in_off,
                   int pass, unsigned long long* counts, const unsigned long long* out_off, uint32_t* out,
                   int canonical, cudaStream_t s);
// Sort keys of collected tetrahedra: (a, b), (c, d) and the cloud.
void batch_tet_keys(const uint32_t* tets, uint64_t T, const unsigned long long* out_off, uint32_t n_clouds,
                    uint64_t* khi, uint64_t* klo, uint64_t* kcl, uint32_t* idx, cudaStream_t s);
// ---------------------------------------------------------------- mlp.cu (learned scheduler)
// ---------------------------------------------------------------- refinement (refine.cu)
// Parameters of one refinement iteration (Section 4): thresholds (ratio h)^2 and (spacing h)^2,
// the box, and the filter grid (cells of 1 / inv_cell >= spacing h, G per axis, bits per axis).
struct RefineParams {
  double lo[3], hi[3];
  double thr_r2, thr_d2, inv_cell;
  uint32_t G;
  int bits;
};
// Device workspace of the refinement iterations, grown on demand and kept by the handle.
struct RefineWS {
  double4_32a* cand = nullptr;  // candidate centre x, y, z and r^2
  uint4* tup = nullptr;     // sorted input-index tuple of the candidate's tetrahedron
  uint8_t* ok = nullptr;    // passed the existing-point filter
  uint32_t* surv = nullptr; // survivors
  double* xyz = nullptr;    // survivors' coordinates in insertion order [n, 3]
  uint64_t *k0 = nullptr, *k1 = nullptr;
  uint32_t *v0 = nullptr, *v1 = nullptr, *hist = nullptr;
  unsigned long long* count = nullptr;  // candidates, survivors
  uint64_t cap_cand = 0, cap_xyz = 0, cap_grid = 0, hist_cap = 0;
};
void refine_ws_free(RefineWS& w);
// Samples and filters one iteration on tetrahedron slots [0, nslots) of the points pts[0, npts):
// *n_cand candidates, *n_new survivors whose coordinates are left in w.xyz in insertion order.
int refine_step(RefineWS& w, const Tet* tets, uint64_t nslots, const Pt* pts, uint64_t npts, const RefineParams& p,
                uint64_t* n_cand, uint64_t* n_new, cudaStream_t s);
// Writes the coordinates of pts[0, npts) to row (input index) of xyz[rows, 3].
int points_out(const Pt* pts, uint64_t npts, double* xyz, uint64_t rows, cudaStream_t s);

int mlp_params();
int mlp_forward(const float* params, const float* x, uint64_t n, float* out, cudaStream_t s);
int mlp_grad(const float* params, const float* x, const float* y, uint64_t n, float* grad, float* loss,
             cudaStream_t s);
int mlp_train(float* params, const float* x, const float* y, uint64_t n, uint32_t steps, uint32_t batch, float lr,
              uint64_t seed, float* losses_host, cudaStream_t s);

}  // namespace dtg
