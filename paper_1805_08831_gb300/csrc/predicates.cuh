// Robust geometric predicates on the GPU (Section 2.4, "Implementation details").
//
// Strategy of the paper: evaluate in floating point, trust the sign when a filter proves it,
// otherwise evaluate exactly, and break exact ties with a symbolic perturbation.
//
//  * Filter: semi-static. With d = q - a (computed), mx, my, mz the largest |d| per axis and
//    md = max(mx, my, mz), every monomial of the expanded determinant is bounded by
//    mx*my*mz (orient3d, 6 monomials) or md^2*mx*my*mz (insphere, 4 * 3 * 6 = 72 monomials).
//    Along the evaluation tree below each monomial meets at most 8 (orient3d) or 17 (insphere)
//    roundings (an FMA contraction only removes roundings), so |error| <= 8*6 eps or
//    17*72 eps times that bound (eps = 2^-53), up to (1 + O(eps)) factors. The constants
//    below add margin: 50 eps and 1300 eps. Magnitudes outside [1e-290, 1e290] go exact.
//  * Exact: expansion arithmetic (Shewchuk, "Adaptive precision floating-point arithmetic and
//    fast robust geometric predicates", 1997): error-free sum and FMA product, Grow-Expansion,
//    Scale-Expansion and Compress, restated below. Exact only while no product underflows
//    or overflows; such an event raises kErrExactRange instead of returning a wrong sign.
//  * Perturbation: the lifted coordinate |p|^2 of point i is raised by eps_i, larger for a
//    larger input index (stored in .w of the point). Expanding the 5x5 lifted determinant
//    along the lifted column, a zero insphere becomes sum_i (-1)^i eps_i O_i with O_i the
//    orient3d of the other four points in order (i = 0..4 for a, b, c, d, e); the sign is
//    that of the first non-zero O_i in decreasing input-index order.
//
// Conventions: orient3d(a,b,c,d) = sign det[b-a; c-a; d-a] (positive tetrahedron > 0);
// insphere(a,b,c,d,e) = sign of the 4x4 determinant of Section 2.4 with rows (q-a, |q-a|^2),
// negative when e is inside the circumsphere of the positive tetrahedron abcd.
#pragma once
#include "common.cuh"

namespace dtg {

constexpr double kEps = 1.1102230246251565e-16;  // 2^-53
constexpr double kOrientC = 50.0 * kEps;
constexpr double kInsphereC = 1300.0 * kEps;
constexpr double kBoundLo = 1e-290;
constexpr double kBoundHi = 1e290;

// ----------------------------------------------------------------- error-free transformations
__device__ __forceinline__ void two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  double bv = __dsub_rn(x, a);
  double av = __dsub_rn(x, bv);
  y = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  y = __dsub_rn(b, __dsub_rn(x, a));
}

__device__ __forceinline__ void two_prod(double a, double b, double& x, double& y, bool& bad) {
  x = __dmul_rn(a, b);
  y = __fma_rn(a, b, -x);
  double ax = fabs(x);
  if ((x != 0.0 && ax < 0x1p-969) || !(ax <= 1.7976931348623157e308)) bad = true;
}

// ----------------------------------------------------------------- expansions
// An expansion is an array of non-overlapping doubles in increasing magnitude whose exact
// sum is the value; zero components are dropped and zero is the single component 0.0.

// h <- h + b in place (Grow-Expansion with zero elimination); returns the new length.
__device__ __forceinline__ int ex_grow(double* h, int nh, double b) {
  double Q = b;
  int k = 0;
  for (int i = 0; i < nh; ++i) {
    double s, e;
    two_sum(Q, h[i], s, e);
    Q = s;
    if (e != 0.0) h[k++] = e;
  }
  if (Q != 0.0 || k == 0) h[k++] = Q;
  return k;
}

// h <- e * b (Scale-Expansion with zero elimination); at most 2*ne components.
__device__ __forceinline__ int ex_scale(const double* e, int ne, double b, double* h, bool& bad) {
  int k = 0;
  double Q, lo;
  two_prod(e[0], b, Q, lo, bad);
  if (lo != 0.0) h[k++] = lo;
  for (int i = 1; i < ne; ++i) {
    double p1, p0, s, t;
    two_prod(e[i], b, p1, p0, bad);
    two_sum(Q, p0, s, t);
    if (t != 0.0) h[k++] = t;
    fast_two_sum(p1, s, Q, t);
    if (t != 0.0) h[k++] = t;
  }
  if (Q != 0.0 || k == 0) h[k++] = Q;
  return k;
}

// Compress in place: same value, usually far fewer components.
__device__ __forceinline__ int ex_compress(double* e, int ne) {
  int bottom = ne - 1;
  double Q = e[bottom];
  for (int i = ne - 2; i >= 0; --i) {
    double s, q;
    fast_two_sum(Q, e[i], s, q);
    if (q != 0.0) {
      e[bottom--] = s;
      Q = q;
    } else {
      Q = s;
    }
  }
  int top = 0;
  for (int i = bottom + 1; i < ne; ++i) {
    double s, q;
    fast_two_sum(e[i], Q, s, q);
    if (q != 0.0) e[top++] = q;
    Q = s;
  }
  e[top] = Q;
  return top + 1;
}

// h += f (in place); -1 when the result could exceed cap.
__device__ __forceinline__ int ex_add_into(double* h, int nh, const double* f, int nf, int cap) {
  if (nh + nf > cap) return -1;
  for (int j = 0; j < nf; ++j) nh = ex_grow(h, nh, f[j]);
  return nh;
}

// h = e * f using tmp (>= 2*ne doubles); -1 when the result could exceed cap.
__device__ __forceinline__ int ex_mul(const double* e, int ne, const double* f, int nf, double* h,
                                      int cap, double* tmp, bool& bad) {
  if (2 * ne * nf > cap) return -1;
  int nh = 1;
  h[0] = 0.0;
  for (int j = 0; j < nf; ++j) {
    int nt = ex_scale(e, ne, f[j], tmp, bad);
    for (int k = 0; k < nt; ++k) nh = ex_grow(h, nh, tmp[k]);
  }
  return nh;
}

__device__ __forceinline__ void ex_negate(double* e, int ne) {
  for (int i = 0; i < ne; ++i) e[i] = -e[i];
}

__device__ __forceinline__ int ex_sign(const double* e, int ne) {
  double top = e[ne - 1];
  return top > 0.0 ? 1 : (top < 0.0 ? -1 : 0);
}

// Exact difference a - b as an expansion of at most 2 components.
struct Ex2 {
  double c[2];
  int n;
};

__device__ __forceinline__ Ex2 ex_diff(double a, double b) {
  Ex2 r;
  double x, y;
  two_sum(a, -b, x, y);
  if (y != 0.0) {
    r.c[0] = y;
    r.c[1] = x;
    r.n = 2;
  } else {
    r.c[0] = x;
    r.n = 1;
  }
  return r;
}

// out = a*b - c*d, compressed (at most 16 components). Returns length (-1 on overflow).
__device__ __forceinline__ int ex_minor(const Ex2& a, const Ex2& b, const Ex2& c, const Ex2& d,
                                        double* out, bool& bad) {
  double p[8], q[8], tmp[4];
  int np = ex_mul(a.c, a.n, b.c, b.n, p, 8, tmp, bad);
  int nq = ex_mul(c.c, c.n, d.c, d.n, q, 8, tmp, bad);
  ex_negate(q, nq);
  for (int i = 0; i < np; ++i) out[i] = p[i];
  int n = ex_add_into(out, np, q, nq, 16);
  return ex_compress(out, n);
}

// out = det[r0; r1; r2] for rows of exact differences, compressed; at most 193 components.
static __device__ __noinline__ int ex_det3(const Ex2* r0, const Ex2* r1, const Ex2* r2, double* out,
                                    bool& bad) {
  double m[16], t[64], tmp[4];
  int n = 1;
  out[0] = 0.0;
  // r0.x * (r1.y r2.z - r1.z r2.y)
  int nm = ex_minor(r1[1], r2[2], r1[2], r2[1], m, bad);
  int nt = ex_mul(r0[0].c, r0[0].n, m, nm, t, 64, tmp, bad);
  n = ex_add_into(out, n, t, nt, 200);
  // - r0.y * (r1.x r2.z - r1.z r2.x)
  nm = ex_minor(r1[0], r2[2], r1[2], r2[0], m, bad);
  nt = ex_mul(r0[1].c, r0[1].n, m, nm, t, 64, tmp, bad);
  ex_negate(t, nt);
  n = ex_add_into(out, n, t, nt, 200);
  // + r0.z * (r1.x r2.y - r1.y r2.x)
  nm = ex_minor(r1[0], r2[1], r1[1], r2[0], m, bad);
  nt = ex_mul(r0[2].c, r0[2].n, m, nm, t, 64, tmp, bad);
  n = ex_add_into(out, n, t, nt, 200);
  return ex_compress(out, n);
}

// ----------------------------------------------------------------- exact stage on integers
// When every coordinate of the points of a predicate is an integer multiple of one power of two
// 2^E with at most 62 significant bits after scaling (lattice, grid and most clustered inputs),
// the coordinates divided by 2^E are exact 64-bit integers, and both determinants are exact
// polynomials in them: sums of products of at most five factors, a 3 x 3 minor (< 2^192) times
// a squared length (< 2^128). They are evaluated in two's-complement arithmetic on 64-bit limbs
// (4 limbs for orient3d, 6 for insphere) on the integer pipes, which GB300 runs far faster than
// its FP64 pipe. Subnormal coordinates or exponents spread over more than about 9 bits keep the
// expansion arithmetic below.
struct IntCoord {
  uint64_t mag;  // odd significand (0 for a zero coordinate)
  int lo;        // exponent of its lowest bit
  int bits;      // significant bits
  bool neg;
};

__device__ __forceinline__ bool int_coord(double x, IntCoord& c) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  uint64_t m = b & 0xFFFFFFFFFFFFFull;
  c.neg = (b >> 63) != 0;
  if (ex == 0 && m == 0) {
    c.mag = 0;
    c.lo = 0x7FFFFFFF;
    c.bits = 0;
    return true;
  }
  if (ex == 0 || ex == 0x7FF) return false;  // subnormal, infinite or NaN
  m |= 1ull << 52;
  const int tz = __ffsll((long long)m) - 1;
  c.mag = m >> tz;
  c.lo = ex - 1075 + tz;
  c.bits = 64 - __clzll((long long)c.mag);
  return true;
}

// The n coordinates as integers of one common power of two (false if one needs > 62 bits).
__device__ __forceinline__ bool int_scale(const IntCoord* c, int n, long long* X) {
  int E = 0x7FFFFFFF;
  for (int i = 0; i < n; ++i) E = min(E, c[i].lo);
  for (int i = 0; i < n; ++i) {
    if (c[i].mag == 0) {
      X[i] = 0;
      continue;
    }
    const int sh = c[i].lo - E;
    if (sh > 62 || c[i].bits + sh > 62) return false;
    const long long v = (long long)(c[i].mag << sh);
    X[i] = c[i].neg ? -v : v;
  }
  return true;
}

// acc (N limbs, two's complement) += m or -= m (m: an nm-limb magnitude).
template <int N>
__device__ __forceinline__ void wide_add(uint64_t* acc, const uint64_t* m, int nm, bool sub) {
  uint64_t c = 0;
  for (int i = 0; i < N; ++i) {
    const uint64_t mi = i < nm ? m[i] : 0ull;
    if (!sub) {
      const uint64_t s = acc[i] + mi;
      const uint64_t c1 = s < mi;
      const uint64_t s2 = s + c;
      c = c1 | (s2 < c);
      acc[i] = s2;
    } else {
      const uint64_t dd = acc[i] - mi;
      const uint64_t b1 = acc[i] < mi;
      const uint64_t d2 = dd - c;
      c = b1 | (dd < c);
      acc[i] = d2;
    }
  }
}

// out[0 .. nm] = m[0 .. nm) * v (magnitudes).
__device__ __forceinline__ void mag_mul1(const uint64_t* m, int nm, uint64_t v, uint64_t* out) {
  uint64_t carry = 0;
  for (int i = 0; i < nm; ++i) {
    uint64_t lo = m[i] * v;
    uint64_t hi = __umul64hi(m[i], v);
    lo += carry;
    hi += (lo < carry);
    out[i] = lo;
    carry = hi;
  }
  out[nm] = carry;
}

__device__ __forceinline__ uint64_t mag64(long long x) { return x < 0 ? (uint64_t)(-x) : (uint64_t)x; }

// det[u; v; w] of integer rows into a 4-limb two's-complement accumulator.
__device__ __forceinline__ void int_det3(const long long* u, const long long* v, const long long* w, uint64_t* acc) {
  for (int i = 0; i < 4; ++i) acc[i] = 0;
  const long long t[6][3] = {{u[0], v[1], w[2]}, {u[0], v[2], w[1]}, {u[1], v[0], w[2]},
                             {u[1], v[2], w[0]}, {u[2], v[0], w[1]}, {u[2], v[1], w[0]}};
  const bool minus[6] = {false, true, true, false, false, true};
  for (int k = 0; k < 6; ++k) {
    const long long a = t[k][0], b = t[k][1], c = t[k][2];
    if (a == 0 || b == 0 || c == 0) continue;
    const bool neg = minus[k] ^ (a < 0) ^ (b < 0) ^ (c < 0);
    const uint64_t ab[2] = {mag64(a) * mag64(b), __umul64hi(mag64(a), mag64(b))};
    uint64_t abc[3];
    mag_mul1(ab, 2, mag64(c), abc);
    wide_add<4>(acc, abc, 3, neg);
  }
}

template <int N>
__device__ __forceinline__ int wide_sign(const uint64_t* acc) {
  if (acc[N - 1] >> 63) return -1;
  for (int i = 0; i < N; ++i)
    if (acc[i]) return 1;
  return 0;
}

// Exact orient3d in integers: true (and *s) when the coordinates fit.
__device__ __forceinline__ bool orient3d_int(const Pt& a, const Pt& b, const Pt& c, const Pt& d, int* s) {
  const double v[12] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, d.x, d.y, d.z};
  IntCoord ic[12];
  for (int i = 0; i < 12; ++i)
    if (!int_coord(v[i], ic[i])) return false;
  long long X[12];
  if (!int_scale(ic, 12, X)) return false;
  long long r[3][3];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) r[i][k] = X[3 * (i + 1) + k] - X[k];
  uint64_t acc[4];
  int_det3(r[0], r[1], r[2], acc);
  *s = wide_sign<4>(acc);
  return true;
}

// Exact insphere in integers (the same determinant as insphere below): true when the
// coordinates fit.
__device__ __forceinline__ bool insphere_int(const Pt& a, const Pt& b, const Pt& c, const Pt& d, const Pt& e,
                                             int* s) {
  const double v[15] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z, d.x, d.y, d.z, e.x, e.y, e.z};
  IntCoord ic[15];
  for (int i = 0; i < 15; ++i)
    if (!int_coord(v[i], ic[i])) return false;
  long long X[15];
  if (!int_scale(ic, 15, X)) return false;
  long long D[4][3];
  uint64_t L[4][2];
  for (int i = 0; i < 4; ++i) {
    L[i][0] = L[i][1] = 0;
    for (int k = 0; k < 3; ++k) {
      D[i][k] = X[3 * (i + 1) + k] - X[k];
      const uint64_t m = mag64(D[i][k]);
      const uint64_t sq[2] = {m * m, __umul64hi(m, m)};
      wide_add<2>(L[i], sq, 2, false);  // < 3 * 2^126: no carry out of two limbs
    }
  }
  uint64_t acc[6] = {0, 0, 0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) {
    int r[3], j = 0;
    for (int i = 0; i < 4; ++i)
      if (i != k) r[j++] = i;
    uint64_t M[4];
    int_det3(D[r[0]], D[r[1]], D[r[2]], M);
    const int sm = wide_sign<4>(M);
    if (sm == 0 || (L[k][0] | L[k][1]) == 0) continue;
    if (sm < 0) {  // magnitude of M
      for (int i = 0; i < 4; ++i) M[i] = ~M[i];
      const uint64_t one = 1;
      wide_add<4>(M, &one, 1, false);
    }
    uint64_t p0[5], p1[5], prod[6];
    mag_mul1(M, 4, L[k][0], p0);
    mag_mul1(M, 4, L[k][1], p1);
    for (int i = 0; i < 6; ++i) prod[i] = 0;
    wide_add<6>(prod, p0, 5, false);
    wide_add<5>(prod + 1, p1, 5, false);
    // sign of the term: (-1)^(k+1) times the sign of the minor
    const bool neg = ((k == 0 || k == 2) ? true : false) ^ (sm < 0);
    wide_add<6>(acc, prod, 6, neg);
  }
  *s = wide_sign<6>(acc);
  return true;
}

static __device__ __noinline__ int orient3d_exact(Pt a, Pt b, Pt c, Pt d,
                                           DevState* st) {
  atomicAdd(&st->n_exact, 1ull);
  int s;
  if (orient3d_int(a, b, c, d, &s)) return s;
  bool bad = false;
  Ex2 u[3] = {ex_diff(b.x, a.x), ex_diff(b.y, a.y), ex_diff(b.z, a.z)};
  Ex2 v[3] = {ex_diff(c.x, a.x), ex_diff(c.y, a.y), ex_diff(c.z, a.z)};
  Ex2 w[3] = {ex_diff(d.x, a.x), ex_diff(d.y, a.y), ex_diff(d.z, a.z)};
  double det[200];
  int n = ex_det3(u, v, w, det, bad);
  if (bad) raise_error(st, kErrExactRange, 1);
  return ex_sign(det, n);
}

static __device__ __noinline__ int insphere_exact(Pt a, Pt b, Pt c, Pt d, Pt e,
                                           DevState* st) {
  atomicAdd(&st->n_exact, 1ull);
  int s;
  if (insphere_int(a, b, c, d, e, &s)) return s;
  bool bad = false;
  const Pt q[4] = {b, c, d, e};
  Ex2 D[4][3];
  double L[4][26];
  int nL[4];
  double tmp[48];
  for (int i = 0; i < 4; ++i) {
    D[i][0] = ex_diff(q[i].x, a.x);
    D[i][1] = ex_diff(q[i].y, a.y);
    D[i][2] = ex_diff(q[i].z, a.z);
    int n = 1;
    L[i][0] = 0.0;
    for (int k = 0; k < 3; ++k) {
      double sq[8];
      int ns = ex_mul(D[i][k].c, D[i][k].n, D[i][k].c, D[i][k].n, sq, 8, tmp, bad);
      n = ex_add_into(L[i], n, sq, ns, 26);
    }
    nL[i] = ex_compress(L[i], n);
  }
  double acc[128], M[200], T[256];
  int nacc = 1;
  acc[0] = 0.0;
  for (int k = 0; k < 4; ++k) {
    int r[3], j = 0;
    for (int i = 0; i < 4; ++i)
      if (i != k) r[j++] = i;
    int nM = ex_det3(D[r[0]], D[r[1]], D[r[2]], M, bad);
    if (2 * nL[k] > 48) {
      bad = true;
      break;
    }
    int nT = ex_mul(L[k], nL[k], M, nM, T, 256, tmp, bad);
    if (nT < 0) {
      bad = true;
      break;
    }
    nT = ex_compress(T, nT);
    if (k == 0 || k == 2) ex_negate(T, nT);  // (-1)^(k+3)
    nacc = ex_add_into(acc, nacc, T, nT, 128);
    if (nacc < 0) {
      bad = true;
      break;
    }
    nacc = ex_compress(acc, nacc);
  }
  if (bad) {
    raise_error(st, kErrExactRange, 2);
    return 0;
  }
  return ex_sign(acc, nacc);
}

// Exact test that c lies on the line ab: every component of (b-a) x (c-a) is zero.
static __device__ __noinline__ bool collinear_exact(Pt a, Pt b, Pt c, DevState* st) {
  bool bad = false;
  Ex2 u[3] = {ex_diff(b.x, a.x), ex_diff(b.y, a.y), ex_diff(b.z, a.z)};
  Ex2 v[3] = {ex_diff(c.x, a.x), ex_diff(c.y, a.y), ex_diff(c.z, a.z)};
  double m[16];
  bool zero = true;
  int n = ex_minor(u[1], v[2], u[2], v[1], m, bad);
  zero = zero && ex_sign(m, n) == 0;
  n = ex_minor(u[2], v[0], u[0], v[2], m, bad);
  zero = zero && ex_sign(m, n) == 0;
  n = ex_minor(u[0], v[1], u[1], v[0], m, bad);
  zero = zero && ex_sign(m, n) == 0;
  if (bad) raise_error(st, kErrExactRange, 3);
  return zero;
}

// ----------------------------------------------------------------- FP32 first stage
// GB300 runs FP64 at about 1/64 of the FP32 rate, and converting FP64 to FP32 costs as much as
// an FP64 operation. So every vertex also carries a double-float copy x = hi + lo (+ r,
// |r| <= 2^-48 |x|), and the predicates first run in FP32 on it:
//   differences D = fl(fl(hi_q - hi_a) + fl(lo_q - lo_a)) satisfy
//   |D - (q - a)| <= 2.01 u |D| + eta,  u = 2^-24, eta = 2^-44 max|x| (+ subnormal slack);
//   the determinant and its permanent P (sum of |monomials|) are evaluated in FP32; with
//   k input factors and r roundings per monomial, |det_f - det| <= (2.01 k + r) u P +
//   (k * #monomials) eta mmax^(k-1) to first order. orient3d: k = 3, r = 8, 6 monomials;
//   insphere: k = 5, r = 16, 72 monomials. The constants below round these up (15 u, 28 u;
//   20 eta, 400 eta). When the sign is not certain (or magnitudes leave FP32's normal range)
//   the FP64 stage below decides.
struct __align__(16) PtF {
  float hx, hy, hz, hw;
  float lx, ly, lz, lw;
};

constexpr float kU = 5.9604645e-08f;  // 2^-24
constexpr float kOrientCf = 15.0f * kU;
constexpr float kInsphereCf = 28.0f * kU;

__device__ __forceinline__ PtF load_ptf(const PtF* P, uint32_t v) {
  const float4* q = reinterpret_cast<const float4*>(P + v);
  float4 a = __ldg(q), b = __ldg(q + 1);
  PtF r;
  r.hx = a.x; r.hy = a.y; r.hz = a.z; r.hw = a.w;
  r.lx = b.x; r.ly = b.y; r.lz = b.z; r.lw = b.w;
  return r;
}

__device__ __forceinline__ void diff_f(const PtF& q, const PtF& a, float& x, float& y, float& z) {
  x = (q.hx - a.hx) + (q.lx - a.lx);
  y = (q.hy - a.hy) + (q.ly - a.ly);
  z = (q.hz - a.hz) + (q.lz - a.lz);
}

// 1 / -1 when certain, 0 when the FP64 stage must decide.
__device__ __forceinline__ int orient3d_f(const PtF& a, const PtF& b, const PtF& c, const PtF& d, float eta) {
  float ux, uy, uz, vx, vy, vz, wx, wy, wz;
  diff_f(b, a, ux, uy, uz);
  diff_f(c, a, vx, vy, vz);
  diff_f(d, a, wx, wy, wz);
  float m0 = vy * wz - vz * wy, m1 = vx * wz - vz * wx, m2 = vx * wy - vy * wx;
  float det = ux * m0 - uy * m1 + uz * m2;
  float perm = fabsf(ux) * (fabsf(vy * wz) + fabsf(vz * wy)) + fabsf(uy) * (fabsf(vx * wz) + fabsf(vz * wx)) +
               fabsf(uz) * (fabsf(vx * wy) + fabsf(vy * wx));
  float mm = fmaxf(fmaxf(fmaxf(fabsf(ux), fabsf(uy)), fmaxf(fabsf(uz), fabsf(vx))),
                   fmaxf(fmaxf(fabsf(vy), fabsf(vz)), fmaxf(fmaxf(fabsf(wx), fabsf(wy)), fabsf(wz)))) + eta;
  float eb = kOrientCf * perm + 20.0f * eta * mm * mm;
  if (!(perm > 1e-30f && perm < 1e30f)) return 0;
  return det > eb ? 1 : (det < -eb ? -1 : 0);
}

__device__ __forceinline__ int insphere_f(const PtF& a, const PtF& b, const PtF& c, const PtF& d, const PtF& e,
                                          float eta) {
  float bx, by, bz, cx, cy, cz, dx, dy, dz, ex, ey, ez;
  diff_f(b, a, bx, by, bz);
  diff_f(c, a, cx, cy, cz);
  diff_f(d, a, dx, dy, dz);
  diff_f(e, a, ex, ey, ez);
  float Lb = bx * bx + by * by + bz * bz, Lc = cx * cx + cy * cy + cz * cz;
  float Ld = dx * dx + dy * dy + dz * dz, Le = ex * ex + ey * ey + ez * ez;
  // 3x3 minors of the x,y,z columns and their permanents
  float cd0 = cy * dz - cz * dy, cd1 = cx * dz - cz * dx, cd2 = cx * dy - cy * dx;
  float pcd0 = fabsf(cy * dz) + fabsf(cz * dy), pcd1 = fabsf(cx * dz) + fabsf(cz * dx),
        pcd2 = fabsf(cx * dy) + fabsf(cy * dx);
  float ce0 = cy * ez - cz * ey, ce1 = cx * ez - cz * ex, ce2 = cx * ey - cy * ex;
  float pce0 = fabsf(cy * ez) + fabsf(cz * ey), pce1 = fabsf(cx * ez) + fabsf(cz * ex),
        pce2 = fabsf(cx * ey) + fabsf(cy * ex);
  float de0 = dy * ez - dz * ey, de1 = dx * ez - dz * ex, de2 = dx * ey - dy * ex;
  float pde0 = fabsf(dy * ez) + fabsf(dz * ey), pde1 = fabsf(dx * ez) + fabsf(dz * ex),
        pde2 = fabsf(dx * ey) + fabsf(dy * ex);
  float M0 = cx * de0 - cy * de1 + cz * de2;  // rows c, d, e
  float M1 = bx * de0 - by * de1 + bz * de2;  // rows b, d, e
  float M2 = bx * ce0 - by * ce1 + bz * ce2;  // rows b, c, e
  float M3 = bx * cd0 - by * cd1 + bz * cd2;  // rows b, c, d
  float P0 = fabsf(cx) * pde0 + fabsf(cy) * pde1 + fabsf(cz) * pde2;
  float P1 = fabsf(bx) * pde0 + fabsf(by) * pde1 + fabsf(bz) * pde2;
  float P2 = fabsf(bx) * pce0 + fabsf(by) * pce1 + fabsf(bz) * pce2;
  float P3 = fabsf(bx) * pcd0 + fabsf(by) * pcd1 + fabsf(bz) * pcd2;
  float det = (Lc * M1 - Lb * M0) + (Le * M3 - Ld * M2);
  float perm = (Lc * P1 + Lb * P0) + (Le * P3 + Ld * P2);
  float mm = fmaxf(fmaxf(fmaxf(fabsf(bx), fabsf(by)), fmaxf(fabsf(bz), fabsf(cx))),
                   fmaxf(fmaxf(fabsf(cy), fabsf(cz)), fmaxf(fabsf(dx), fabsf(dy))));
  mm = fmaxf(mm, fmaxf(fmaxf(fabsf(dz), fabsf(ex)), fmaxf(fabsf(ey), fabsf(ez)))) + eta;
  float mm2 = mm * mm;
  float eb = kInsphereCf * perm + 400.0f * eta * (mm2 * mm2);
  if (!(perm > 1e-30f && perm < 1e30f)) return 0;
  return det > eb ? 1 : (det < -eb ? -1 : 0);
}

// ----------------------------------------------------------------- filtered predicates
__device__ __forceinline__ double absmax3(double a, double b, double c) {
  return fmax(fmax(fabs(a), fabs(b)), fabs(c));
}

// The FP64 filter of orient3d alone: the sign, or 0 when it cannot be certain.
__device__ __forceinline__ int orient3d_filter(const Pt& a, const Pt& b, const Pt& c, const Pt& d) {
  double ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
  double vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
  double wx = d.x - a.x, wy = d.y - a.y, wz = d.z - a.z;
  double det = ux * (vy * wz - vz * wy) - uy * (vx * wz - vz * wx) + uz * (vx * wy - vy * wx);
  double mx = absmax3(ux, vx, wx), my = absmax3(uy, vy, wy), mz = absmax3(uz, vz, wz);
  double bound = mx * my * mz;
  if (bound > kBoundLo && bound < kBoundHi) {
    double eb = kOrientC * bound;
    if (det > eb) return 1;
    if (det < -eb) return -1;
  }
  return 0;
}

__device__ __forceinline__ int orient3d(Pt a, Pt b, Pt c, Pt d, DevState* st) {
  const int s = orient3d_filter(a, b, c, d);
  return s != 0 ? s : orient3d_exact(a, b, c, d, st);
}

__device__ __forceinline__ double det3d(double ax, double ay, double az, double bx, double by,
                                        double bz, double cx, double cy, double cz) {
  return ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
}

__device__ __forceinline__ int insphere(Pt a, Pt b, Pt c, Pt d, Pt e,
                                        DevState* st) {
  double bx = b.x - a.x, by = b.y - a.y, bz = b.z - a.z;
  double cx = c.x - a.x, cy = c.y - a.y, cz = c.z - a.z;
  double dx = d.x - a.x, dy = d.y - a.y, dz = d.z - a.z;
  double ex = e.x - a.x, ey = e.y - a.y, ez = e.z - a.z;
  double Lb = bx * bx + by * by + bz * bz;
  double Lc = cx * cx + cy * cy + cz * cz;
  double Ld = dx * dx + dy * dy + dz * dz;
  double Le = ex * ex + ey * ey + ez * ez;
  double M0 = det3d(cx, cy, cz, dx, dy, dz, ex, ey, ez);
  double M1 = det3d(bx, by, bz, dx, dy, dz, ex, ey, ez);
  double M2 = det3d(bx, by, bz, cx, cy, cz, ex, ey, ez);
  double M3 = det3d(bx, by, bz, cx, cy, cz, dx, dy, dz);
  double det = (Lc * M1 - Lb * M0) + (Le * M3 - Ld * M2);
  double mx = fmax(absmax3(bx, cx, dx), fabs(ex));
  double my = fmax(absmax3(by, cy, dy), fabs(ey));
  double mz = fmax(absmax3(bz, cz, dz), fabs(ez));
  double md = fmax(fmax(mx, my), mz);
  double bound = md * md * (mx * my * mz);
  if (bound > kBoundLo && bound < kBoundHi) {
    double eb = kInsphereC * bound;
    if (det > eb) return 1;
    if (det < -eb) return -1;
  }
  return insphere_exact(a, b, c, d, e, st);
}

// Perturbed insphere: never 0 when abcd is a positive (non-flat) tetrahedron.
__device__ __forceinline__ int insphere_sos(Pt a, Pt b, Pt c, Pt d, Pt e,
                                            DevState* st) {
  int s = insphere(a, b, c, d, e, st);
  if (s != 0) return s;
  atomicAdd(&st->n_sos, 1ull);
  Pt p[5] = {a, b, c, d, e};
  unsigned used = 0;
  for (int t = 0; t < 5; ++t) {
    int best = -1;
    for (int i = 0; i < 5; ++i)
      if (!(used & (1u << i)) && (best < 0 || p[i].w > p[best].w)) best = i;
    used |= 1u << best;
    Pt o[4];
    int j = 0;
    for (int k = 0; k < 5; ++k)
      if (k != best) o[j++] = p[k];
    int s4 = orient3d(o[0], o[1], o[2], o[3], st);
    if (s4 != 0) return (best & 1) ? -s4 : s4;
  }
  return 0;
}

}  // namespace dtg
