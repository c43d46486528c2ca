// Delaunay refinement inside a box (Section 4, Algorithm 2: the loop of SamplePoints,
// FilterPoints and InsertPoints), the sampling and filtering half. The insertion is the
// library's concurrent insertion, called by the host loop in dt.cu with the survivors found here.
//
// One iteration on the current tetrahedra:
//   sample  a finite live tetrahedron with r^2 > (ratio h)^2 gives a candidate at its
//           circumcentre when that lies strictly inside the box;
//   filter  (1) a candidate at squared distance < (spacing h)^2 from an existing point is
//           dropped: the circumcentre of a near-flat tetrahedron is dominated by rounding and can
//           sit next to a vertex (the paper aborts such a cavity instead); (2) a remaining
//           candidate at squared distance < (spacing h)^2 from a remaining candidate of higher
//           priority (larger r^2, then the smaller sorted input-index tuple) is dropped;
//   order   the survivors by their tetrahedra's sorted input-index tuples.
// Every floating-point operation is rounded on its own, in a fixed order (no contraction), so the
// candidates, the filters' decisions and the order are a fixed function of the points and the
// tetrahedra, whatever the slot layout or the thread schedule.
//
// Both filters use one uniform grid over the points and the candidates, with cells slightly
// wider than spacing h, sorted by cell key: a pair closer than spacing h lies in neighbouring
// cells, and the three cells of a row of neighbours are contiguous in key order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"

namespace dtg {
namespace {

constexpr int kThreads = 256;

unsigned grid_of(uint64_t n) {
  uint64_t b = (n + kThreads - 1) / kThreads;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 32));
}

struct V3 {
  double x, y, z;
};

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }

// (p.x q.x + p.y q.y) + p.z q.z
__device__ __forceinline__ double dot(const V3& p, const V3& q) {
  return add(add(mul(p.x, q.x), mul(p.y, q.y)), mul(p.z, q.z));
}

__device__ __forceinline__ V3 cross(const V3& p, const V3& q) {
  return {sub(mul(p.y, q.z), mul(p.z, q.y)), sub(mul(p.z, q.x), mul(p.x, q.z)), sub(mul(p.x, q.y), mul(p.y, q.x))};
}

__device__ __forceinline__ V3 diff(const Pt& p, const Pt& q) { return {sub(p.x, q.x), sub(p.y, q.y), sub(p.z, q.z)}; }

// Circumcentre and squared circumradius of the tetrahedron a, b, c, d (given in increasing input
// index): with u = b - a, v = c - a, w = d - a,
//   o = ((|u|^2 (v x w) + |v|^2 (w x u)) + |w|^2 (u x v)) / (2 u . (v x w)),  centre = a + o.
__device__ void circumcentre(const Pt& a, const Pt& b, const Pt& c, const Pt& d, V3& centre, double& r2) {
  const V3 u = diff(b, a), v = diff(c, a), w = diff(d, a);
  const double lu = dot(u, u), lv = dot(v, v), lw = dot(w, w);
  const V3 vw = cross(v, w), wu = cross(w, u), uv = cross(u, v);
  const double den = mul(2.0, dot(u, vw));
  const V3 o = {__ddiv_rn(add(add(mul(lu, vw.x), mul(lv, wu.x)), mul(lw, uv.x)), den),
                __ddiv_rn(add(add(mul(lu, vw.y), mul(lv, wu.y)), mul(lw, uv.y)), den),
                __ddiv_rn(add(add(mul(lu, vw.z), mul(lv, wu.z)), mul(lw, uv.z)), den)};
  centre = {add(a.x, o.x), add(a.y, o.y), add(a.z, o.z)};
  r2 = dot(o, o);
}

__device__ __forceinline__ void order2(Pt& p, Pt& q) {
  if (q.w < p.w) {
    Pt t = p;
    p = q;
    q = t;
  }
}

__global__ void __launch_bounds__(kThreads) k_refine_sample(const Tet* __restrict__ tets, uint64_t nslots,
                                                            const Pt* __restrict__ pts, uint64_t npts, RefineParams p,
                                                            double4_32a* __restrict__ cand, uint4* __restrict__ tup,
                                                            unsigned long long* count, uint64_t cap) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nslots; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 v = tets[t].v;
    if (tet_dead(v) || ghost_pos(v) >= 0) continue;
    if (v.x >= npts || v.y >= npts || v.z >= npts || v.w >= npts) continue;
    Pt q0 = pts[v.x], q1 = pts[v.y], q2 = pts[v.z], q3 = pts[v.w];
    // the four vertices in increasing input index (a sorting network)
    order2(q0, q1);
    order2(q2, q3);
    order2(q0, q2);
    order2(q1, q3);
    order2(q1, q2);
    V3 c;
    double r2;
    circumcentre(q0, q1, q2, q3, c, r2);
    if (!(r2 > p.thr_r2)) continue;
    if (!(p.lo[0] < c.x && c.x < p.hi[0] && p.lo[1] < c.y && c.y < p.hi[1] && p.lo[2] < c.z && c.z < p.hi[2]))
      continue;
    const unsigned long long k = atomicAdd(count, 1ull);
    if (k < cap) {
      cand[k] = make_double4_32a(c.x, c.y, c.z, r2);
      tup[k] = make_uint4((uint32_t)q0.w, (uint32_t)q1.w, (uint32_t)q2.w, (uint32_t)q3.w);
    }
  }
}

__device__ __forceinline__ uint32_t cell_of(double x, double lo, double inv, uint32_t G) {
  const double f = mul(sub(x, lo), inv);
  if (!(f > 0.0)) return 0;  // below the box (or NaN)
  if (f >= (double)G) return G - 1;
  return (uint32_t)f;
}

__device__ __forceinline__ uint64_t cell_key(uint32_t x, uint32_t y, uint32_t z, int bits) {
  return ((uint64_t)z << (2 * bits)) | ((uint64_t)y << bits) | x;
}

// Grid entries: points 0 .. npts-1, then candidates npts .. npts+m-1.
__global__ void k_refine_grid_keys(const Pt* __restrict__ pts, uint64_t npts, const double4_32a* __restrict__ cand,
                                   uint64_t m, RefineParams p, uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
  const uint64_t E = npts + m;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < E; e += (uint64_t)gridDim.x * blockDim.x) {
    double x, y, z;
    if (e < npts) {
      const Pt q = pts[e];
      x = q.x, y = q.y, z = q.z;
    } else {
      const double4_32a c = cand[e - npts];
      x = c.x, y = c.y, z = c.z;
    }
    key[e] = cell_key(cell_of(x, p.lo[0], p.inv_cell, p.G), cell_of(y, p.lo[1], p.inv_cell, p.G),
                      cell_of(z, p.lo[2], p.inv_cell, p.G), p.bits);
    val[e] = (uint32_t)e;
  }
}

__device__ __forceinline__ uint64_t lower_bound(const uint64_t* __restrict__ key, uint64_t E, uint64_t k) {
  uint64_t lo = 0, hi = E;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (key[mid] < k)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Calls f(entry) for every grid entry in the 27 cells around c, until f returns false.
template <class F>
__device__ void for_near(const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, uint64_t E,
                         const RefineParams& p, const double4_32a& c, F f) {
  const uint32_t cx = cell_of(c.x, p.lo[0], p.inv_cell, p.G), cy = cell_of(c.y, p.lo[1], p.inv_cell, p.G),
                 cz = cell_of(c.z, p.lo[2], p.inv_cell, p.G);
  const uint32_t x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < p.G ? cx + 1 : cx;
  for (int dz = -1; dz <= 1; ++dz) {
    const int64_t z = (int64_t)cz + dz;
    if (z < 0 || z >= p.G) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int64_t y = (int64_t)cy + dy;
      if (y < 0 || y >= p.G) continue;
      const uint64_t k1 = cell_key(x1, (uint32_t)y, (uint32_t)z, p.bits);
      for (uint64_t e = lower_bound(key, E, cell_key(x0, (uint32_t)y, (uint32_t)z, p.bits)); e < E && key[e] <= k1; ++e)
        if (!f(val[e])) return;
    }
  }
}

__device__ __forceinline__ double dist2(const double4_32a& a, double x, double y, double z) {
  const V3 d = {sub(a.x, x), sub(a.y, y), sub(a.z, z)};
  return dot(d, d);
}

// Filter 1: no existing point at squared distance < thr_d2.
__global__ void __launch_bounds__(kThreads) k_refine_near_points(const double4_32a* __restrict__ cand, uint64_t m,
                                                                 const Pt* __restrict__ pts, uint64_t npts,
                                                                 const uint64_t* __restrict__ key,
                                                                 const uint32_t* __restrict__ val, RefineParams p,
                                                                 uint8_t* __restrict__ ok) {
  const uint64_t E = npts + m;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const double4_32a c = cand[i];
    bool good = true;
    for_near(key, val, E, p, c, [&](uint32_t e) {
      if (e >= npts) return true;
      const Pt q = pts[e];
      if (dist2(c, q.x, q.y, q.z) < p.thr_d2) good = false;
      return good;
    });
    ok[i] = good ? 1 : 0;
  }
}

__device__ __forceinline__ bool tuple_less(const uint4& a, const uint4& b) {
  if (a.x != b.x) return a.x < b.x;
  if (a.y != b.y) return a.y < b.y;
  if (a.z != b.z) return a.z < b.z;
  return a.w < b.w;
}

// Filter 2: no remaining candidate of higher priority at squared distance < thr_d2. Survivors are
// appended to surv (their order there does not matter: they are sorted next).
__global__ void __launch_bounds__(kThreads) k_refine_filter(const double4_32a* __restrict__ cand,
                                                            const uint4* __restrict__ tup, uint64_t m, uint64_t npts,
                                                            const uint64_t* __restrict__ key,
                                                            const uint32_t* __restrict__ val, RefineParams p,
                                                            const uint8_t* __restrict__ ok, uint32_t* __restrict__ surv,
                                                            unsigned long long* count) {
  const uint64_t E = npts + m;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!ok[i]) continue;
    const double4_32a c = cand[i];
    const uint4 ti = tup[i];
    bool keep = true;
    for_near(key, val, E, p, c, [&](uint32_t e) {
      if (e < npts) return true;
      const uint64_t j = e - npts;
      if (j == i || !ok[j]) return true;
      const double4_32a cj = cand[j];
      if (!(dist2(c, cj.x, cj.y, cj.z) < p.thr_d2)) return true;
      if (cj.w > c.w || (cj.w == c.w && tuple_less(tup[j], ti))) keep = false;
      return keep;
    });
    if (keep) surv[atomicAdd(count, 1ull)] = (uint32_t)i;
  }
}

// Keys of the survivors' tuples, (t.z, t.w) or (t.x, t.y) packed on 2 * bits bits, in the order
// of ids.
__global__ void k_refine_tuple_keys(const uint32_t* __restrict__ ids, uint64_t n, const uint4* __restrict__ tup,
                                    int bits, int high, uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t id = ids[k];
    const uint4 t = tup[id];
    key[k] = high ? ((uint64_t)t.x << bits) | t.y : ((uint64_t)t.z << bits) | t.w;
    val[k] = id;
  }
}

__global__ void k_refine_gather(const uint32_t* __restrict__ ids, uint64_t n, const double4_32a* __restrict__ cand,
                                double* __restrict__ xyz) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const double4_32a c = cand[ids[k]];
    xyz[3 * k] = c.x;
    xyz[3 * k + 1] = c.y;
    xyz[3 * k + 2] = c.z;
  }
}

__global__ void k_points_out(const Pt* __restrict__ pts, uint64_t npts, double* __restrict__ xyz, uint64_t rows) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < npts; i += (uint64_t)gridDim.x * blockDim.x) {
    const Pt q = pts[i];
    const uint64_t r = (uint64_t)q.w;
    if (r < rows) {
      xyz[3 * r] = q.x;
      xyz[3 * r + 1] = q.y;
      xyz[3 * r + 2] = q.z;
    }
  }
}

template <class T>
cudaError_t grow(T*& p, uint64_t& cap, uint64_t need) {
  if (need <= cap && p) return cudaSuccess;
  cudaFree(p);
  p = nullptr;
  cap = 0;
  const uint64_t c = std::max<uint64_t>(need + need / 4, 1024);
  cudaError_t e = cudaMalloc(&p, c * sizeof(T));
  if (e == cudaSuccess) cap = c;
  return e;
}

int bits_for(uint64_t n) {
  int b = 1;
  while (b < 64 && (n >> b)) ++b;
  return b;
}

}  // namespace

void refine_ws_free(RefineWS& w) {
  cudaFree(w.cand);
  cudaFree(w.tup);
  cudaFree(w.ok);
  cudaFree(w.k0);
  cudaFree(w.k1);
  cudaFree(w.v0);
  cudaFree(w.v1);
  cudaFree(w.hist);
  cudaFree(w.surv);
  cudaFree(w.xyz);
  cudaFree(w.count);
  w = RefineWS();
}

int refine_step(RefineWS& w, const Tet* tets, uint64_t nslots, const Pt* pts, uint64_t npts, const RefineParams& p,
                uint64_t* n_cand, uint64_t* n_new, cudaStream_t s) {
  *n_cand = 0;
  *n_new = 0;
  if (nslots > w.cap_cand || !w.cand) {
    uint64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    cudaFree(w.cand), cudaFree(w.tup), cudaFree(w.ok), cudaFree(w.surv);
    w.cand = nullptr, w.tup = nullptr, w.ok = nullptr, w.surv = nullptr, w.cap_cand = 0;
    if (grow(w.cand, c0, nslots) != cudaSuccess || grow(w.tup, c1, nslots) != cudaSuccess ||
        grow(w.ok, c2, nslots) != cudaSuccess || grow(w.surv, c3, nslots) != cudaSuccess)
      return DT_ENOMEM;
    w.cap_cand = c0;
  }
  if (grow(w.xyz, w.cap_xyz, 3 * nslots) != cudaSuccess) return DT_ENOMEM;
  if (!w.count && cudaMalloc(&w.count, 16) != cudaSuccess) return DT_ENOMEM;
  cudaMemsetAsync(w.count, 0, 16, s);
  k_refine_sample<<<grid_of(nslots), kThreads, 0, s>>>(tets, nslots, pts, npts, p, w.cand, w.tup, w.count, nslots);
  ++g_kernel_launches;
  unsigned long long cnt[2] = {0, 0};
  if (cudaMemcpyAsync(cnt, w.count, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DT_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;
  const uint64_t m = cnt[0];
  *n_cand = m;
  if (m == 0) return DT_OK;
  if (npts + m >= 0xFFFFFFF0ull) return DT_EINVAL;
  // the grid over points and candidates, sorted by cell key
  const uint64_t E = npts + m;
  if (E > w.cap_grid || !w.k0) {
    uint64_t g0 = 0, g1 = 0, g2 = 0, g3 = 0;
    cudaFree(w.k0), cudaFree(w.k1), cudaFree(w.v0), cudaFree(w.v1);
    w.k0 = nullptr, w.k1 = nullptr, w.v0 = nullptr, w.v1 = nullptr, w.cap_grid = 0;
    if (grow(w.k0, g0, E) != cudaSuccess || grow(w.k1, g1, E) != cudaSuccess || grow(w.v0, g2, E) != cudaSuccess ||
        grow(w.v1, g3, E) != cudaSuccess)
      return DT_ENOMEM;
    w.cap_grid = g0;
  }
  if (grow(w.hist, w.hist_cap, radix_hist_entries(E)) != cudaSuccess) return DT_ENOMEM;
  k_refine_grid_keys<<<grid_of(E), kThreads, 0, s>>>(pts, npts, w.cand, m, p, w.k0, w.v0);
  ++g_kernel_launches;
  const bool alt = radix_sort_pairs(w.k0, w.v0, w.k1, w.v1, E, 3 * p.bits, w.hist, s);
  const uint64_t* key = alt ? w.k1 : w.k0;
  const uint32_t* val = alt ? w.v1 : w.v0;
  k_refine_near_points<<<grid_of(m), kThreads, 0, s>>>(w.cand, m, pts, npts, key, val, p, w.ok);
  k_refine_filter<<<grid_of(m), kThreads, 0, s>>>(w.cand, w.tup, m, npts, key, val, p, w.ok, w.surv, w.count + 1);
  g_kernel_launches += 2;
  if (cudaMemcpyAsync(cnt + 1, w.count + 1, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return DT_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DT_ECUDA;
  const uint64_t ns = cnt[1];
  if (ns == 0) return DT_OK;
  // survivors in increasing tuple order: a stable sort by (z, w), then by (x, y)
  const int b = bits_for(npts);
  const int kb = std::min(64, 2 * b);
  k_refine_tuple_keys<<<grid_of(ns), kThreads, 0, s>>>(w.surv, ns, w.tup, b, 0, w.k0, w.v0);
  ++g_kernel_launches;
  bool a1 = radix_sort_pairs(w.k0, w.v0, w.k1, w.v1, ns, kb, w.hist, s);
  uint32_t* ids = a1 ? w.v1 : w.v0;
  uint64_t* kbuf = a1 ? w.k1 : w.k0;
  uint64_t* kalt = a1 ? w.k0 : w.k1;
  uint32_t* valt = a1 ? w.v0 : w.v1;
  k_refine_tuple_keys<<<grid_of(ns), kThreads, 0, s>>>(ids, ns, w.tup, b, 1, kbuf, valt);
  ++g_kernel_launches;
  const bool a2 = radix_sort_pairs(kbuf, valt, kalt, ids, ns, kb, w.hist, s);
  const uint32_t* order = a2 ? ids : valt;
  k_refine_gather<<<grid_of(ns), kThreads, 0, s>>>(order, ns, w.cand, w.xyz);
  ++g_kernel_launches;
  if (cudaPeekAtLastError() != cudaSuccess) return DT_ECUDA;
  *n_new = ns;
  return DT_OK;
}

int points_out(const Pt* pts, uint64_t npts, double* xyz, uint64_t rows, cudaStream_t s) {
  if (npts == 0) return DT_OK;
  k_points_out<<<grid_of(npts), kThreads, 0, s>>>(pts, npts, xyz, rows);
  ++g_kernel_launches;
  return cudaPeekAtLastError() == cudaSuccess ? DT_OK : DT_ECUDA;
}

}  // namespace dtg
