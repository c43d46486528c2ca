// Serial CPU oracle for the Delaunay kernel of arXiv 1805.08831 (Marot, Pellerin, Remacle).
//
// TEST INFRASTRUCTURE ONLY: used by the tests, the package smoke check and the CPU-baseline leg
// of the benchmark. It shares no code with the GPU library. Each function restates a passage of
// the paper in the plainest form that still finishes on 1e5..1e7 points:
//   - predicates (Section 2.4): a double-precision filter with a deliberately loose bound
//     (1e-12 of the permanent for orient3d, 1e-11 for insphere, several thousand times the
//     rounding error), and otherwise big-integer arithmetic on the exact dyadic values;
//   - symbolic perturbation of the lifting (Section 2.4, item 3): the sign of a zero insphere
//     determinant is the sign of the first non-zero perturbation coefficient;
//   - ghost tetrahedra and their composite circumsphere (Section 2.6);
//   - Algorithm 1 (Init, Sort, Walk, Cavity, DelaunayBall) with a sort-based facet matcher in
//     place of the n x n table of Section 2.5;
//   - the Moore curve index (Section 2.3) from Hamilton's Gray-code construction;
//   - BRIO rounds with the sizes of Table 2.
// Compile with -ffp-contract=off so the quantisation rounds each operation separately.
#include "oracle.h"

#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <utility>
#include <vector>

namespace {

int g_mut = 0;  // planted mistake for mutation tests (0 = none)

constexpr uint32_t GHOST = 0xFFFFFFFFu;
constexpr uint32_t NONE = 0xFFFFFFFFu;

// Predicate counters of the calling thread (the threaded baseline calls the predicates from
// several threads; the serial oracle runs on one).
struct Counters {
  int64_t insphere = 0, exact = 0, sos = 0;
};
thread_local Counters g_cnt;

// ------------------------------------------------------------------ big integers
// Sign-magnitude integers with little-endian 32-bit limbs; schoolbook arithmetic.
struct Big {
  int sign = 0;
  std::vector<uint32_t> mag;
};

void trim(std::vector<uint32_t>& m) {
  while (!m.empty() && m.back() == 0) m.pop_back();
}

int cmp_mag(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

std::vector<uint32_t> add_mag(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  std::vector<uint32_t> r(std::max(a.size(), b.size()) + 1, 0);
  uint64_t carry = 0;
  for (size_t i = 0; i < r.size(); ++i) {
    uint64_t s = carry;
    if (i < a.size()) s += a[i];
    if (i < b.size()) s += b[i];
    r[i] = (uint32_t)s;
    carry = s >> 32;
  }
  trim(r);
  return r;
}

// Requires |a| >= |b|.
std::vector<uint32_t> sub_mag(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  std::vector<uint32_t> r(a.size(), 0);
  int64_t borrow = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    int64_t d = (int64_t)a[i] - borrow - (i < b.size() ? (int64_t)b[i] : 0);
    if (d < 0) {
      d += (int64_t)1 << 32;
      borrow = 1;
    } else {
      borrow = 0;
    }
    r[i] = (uint32_t)d;
  }
  trim(r);
  return r;
}

std::vector<uint32_t> mul_mag(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  if (a.empty() || b.empty()) return {};
  std::vector<uint32_t> r(a.size() + b.size(), 0);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      uint64_t cur = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)cur;
      carry = cur >> 32;
    }
    size_t k = i + b.size();
    while (carry) {
      uint64_t cur = (uint64_t)r[k] + carry;
      r[k] = (uint32_t)cur;
      carry = cur >> 32;
      ++k;
    }
  }
  trim(r);
  return r;
}

Big add(const Big& a, const Big& b) {
  if (a.sign == 0) return b;
  if (b.sign == 0) return a;
  Big r;
  if (a.sign == b.sign) {
    r.sign = a.sign;
    r.mag = add_mag(a.mag, b.mag);
    return r;
  }
  int c = cmp_mag(a.mag, b.mag);
  if (c == 0) return r;
  if (c > 0) {
    r.sign = a.sign;
    r.mag = sub_mag(a.mag, b.mag);
  } else {
    r.sign = b.sign;
    r.mag = sub_mag(b.mag, a.mag);
  }
  return r;
}

Big neg(Big a) {
  a.sign = -a.sign;
  return a;
}

Big sub(const Big& a, const Big& b) { return add(a, neg(b)); }

Big mul(const Big& a, const Big& b) {
  Big r;
  if (a.sign == 0 || b.sign == 0) return r;
  r.mag = mul_mag(a.mag, b.mag);
  r.sign = a.sign * b.sign;
  return r;
}

// Exponent of the last mantissa bit: x = M * 2^ulp_exp(x) with M a 53-bit integer.
int ulp_exp(double x) {
  int e;
  std::frexp(std::fabs(x), &e);
  return e - 53;
}

int common_exp(const double* v, int k) {
  int E = INT_MAX;
  for (int i = 0; i < k; ++i)
    if (v[i] != 0.0) E = std::min(E, ulp_exp(v[i]));
  return E == INT_MAX ? 0 : E;
}

// The integer x / 2^E (exact because E <= ulp_exp(x)).
Big big_from_double(double x, int E) {
  Big r;
  if (x == 0.0) return r;
  int e;
  double f = std::frexp(std::fabs(x), &e);
  uint64_t M = (uint64_t)std::ldexp(f, 53);
  int shift = e - 53 - E;
  r.sign = x < 0 ? -1 : 1;
  r.mag.assign((size_t)(shift / 32), 0u);
  int bits = shift % 32;
  uint64_t lo = M << bits;                              // low 64 bits of M * 2^bits
  uint64_t hi = bits ? (M >> (64 - bits)) : 0;          // bits above 64
  r.mag.push_back((uint32_t)lo);
  r.mag.push_back((uint32_t)(lo >> 32));
  r.mag.push_back((uint32_t)hi);
  trim(r.mag);
  return r;
}

// value * 2^scale rounded to double through the top limbs (exact for small values).
double big_to_double(const Big& b, int scale) {
  if (b.sign == 0) return 0.0;
  long double acc = 0.0L;
  size_t top = b.mag.size();
  size_t lo = top > 4 ? top - 4 : 0;
  for (size_t i = top; i-- > lo;) acc = acc * 4294967296.0L + (long double)b.mag[i];
  return (double)(b.sign * std::ldexp(acc, (int)(32 * lo) + scale));
}

// ------------------------------------------------------------------ predicates (Section 2.4)
// orient3d(a,b,c,d) = sign det[b-a; c-a; d-a]  (positive tetrahedron convention).
int orient3d_exact(const double* a, const double* b, const double* c, const double* d,
                   double* value = nullptr) {
  ++g_cnt.exact;
  double all[12];
  for (int k = 0; k < 3; ++k) {
    all[k] = a[k];
    all[3 + k] = b[k];
    all[6 + k] = c[k];
    all[9 + k] = d[k];
  }
  int E = common_exp(all, 12);
  Big u[3], v[3], w[3];
  for (int k = 0; k < 3; ++k) {
    Big A = big_from_double(a[k], E);
    u[k] = sub(big_from_double(b[k], E), A);
    v[k] = sub(big_from_double(c[k], E), A);
    w[k] = sub(big_from_double(d[k], E), A);
  }
  Big det = add(sub(mul(u[0], sub(mul(v[1], w[2]), mul(v[2], w[1]))),
                    mul(u[1], sub(mul(v[0], w[2]), mul(v[2], w[0])))),
                mul(u[2], sub(mul(v[0], w[1]), mul(v[1], w[0]))));
  if (value) *value = big_to_double(det, 3 * E);
  return det.sign;
}

int orient3d(const double* a, const double* b, const double* c, const double* d) {
  if (g_mut == 4) std::swap(c, d);
  double u0 = b[0] - a[0], u1 = b[1] - a[1], u2 = b[2] - a[2];
  double v0 = c[0] - a[0], v1 = c[1] - a[1], v2 = c[2] - a[2];
  double w0 = d[0] - a[0], w1 = d[1] - a[1], w2 = d[2] - a[2];
  double det = u0 * (v1 * w2 - v2 * w1) - u1 * (v0 * w2 - v2 * w0) + u2 * (v0 * w1 - v1 * w0);
  double perm = std::fabs(u0) * (std::fabs(v1 * w2) + std::fabs(v2 * w1)) +
                std::fabs(u1) * (std::fabs(v0 * w2) + std::fabs(v2 * w0)) +
                std::fabs(u2) * (std::fabs(v0 * w1) + std::fabs(v1 * w0));
  if (perm > 1e-250 && perm < 1e250 && std::fabs(det) > 1e-12 * perm) return det > 0 ? 1 : -1;
  return orient3d_exact(a, b, c, d);
}

// 3x3 determinant of rows r0, r1, r2 (doubles), with its permanent.
double det3(const double* r0, const double* r1, const double* r2, double* perm) {
  double m0 = r1[1] * r2[2] - r1[2] * r2[1];
  double m1 = r1[0] * r2[2] - r1[2] * r2[0];
  double m2 = r1[0] * r2[1] - r1[1] * r2[0];
  *perm = std::fabs(r0[0]) * (std::fabs(r1[1] * r2[2]) + std::fabs(r1[2] * r2[1])) +
          std::fabs(r0[1]) * (std::fabs(r1[0] * r2[2]) + std::fabs(r1[2] * r2[0])) +
          std::fabs(r0[2]) * (std::fabs(r1[0] * r2[1]) + std::fabs(r1[1] * r2[0]));
  return r0[0] * m0 - r0[1] * m1 + r0[2] * m2;
}

// The 4x4 determinant of Section 2.4 with rows (q-a, |q-a|^2), q = b, c, d, e, expanded along
// the lifted column: D4 = sum_k (-1)^(k+3) L_k M_k, M_k = det of the x,y,z part without row k.
int insphere_exact(const double* const p[5], double* value = nullptr) {
  ++g_cnt.exact;
  double all[15];
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 3; ++k) all[3 * i + k] = p[i][k];
  int E = common_exp(all, 15);
  Big D[4][3], L[4];
  for (int q = 0; q < 4; ++q) {
    for (int k = 0; k < 3; ++k)
      D[q][k] = sub(big_from_double(p[q + 1][k], E), big_from_double(p[0][k], E));
    L[q] = add(add(mul(D[q][0], D[q][0]), mul(D[q][1], D[q][1])), mul(D[q][2], D[q][2]));
  }
  Big total;
  for (int k = 0; k < 4; ++k) {
    if (g_mut == 3 && k == 0) continue;
    int r[3], j = 0;
    for (int q = 0; q < 4; ++q)
      if (q != k) r[j++] = q;
    const Big* R0 = D[r[0]];
    const Big* R1 = D[r[1]];
    const Big* R2 = D[r[2]];
    Big M = add(sub(mul(R0[0], sub(mul(R1[1], R2[2]), mul(R1[2], R2[1]))),
                    mul(R0[1], sub(mul(R1[0], R2[2]), mul(R1[2], R2[0])))),
                mul(R0[2], sub(mul(R1[0], R2[1]), mul(R1[1], R2[0]))));
    Big term = mul(L[k], M);
    total = ((k + 3) % 2 == 0) ? add(total, term) : sub(total, term);
  }
  if (value) *value = big_to_double(total, 5 * E);
  return total.sign;
}

int insphere(const double* const p[5]) {
  ++g_cnt.insphere;
  double D[4][3], L[4];
  for (int q = 0; q < 4; ++q) {
    for (int k = 0; k < 3; ++k) D[q][k] = p[q + 1][k] - p[0][k];
    L[q] = D[q][0] * D[q][0] + D[q][1] * D[q][1] + D[q][2] * D[q][2];
  }
  double total = 0.0, perm = 0.0;
  for (int k = 0; k < 4; ++k) {
    if (g_mut == 3 && k == 0) continue;
    int r[3], j = 0;
    for (int q = 0; q < 4; ++q)
      if (q != k) r[j++] = q;
    double pm;
    double M = det3(D[r[0]], D[r[1]], D[r[2]], &pm);
    double term = L[k] * M;
    total = ((k + 3) % 2 == 0) ? total + term : total - term;
    perm += std::fabs(L[k]) * pm;
  }
  if (perm > 1e-250 && perm < 1e250 && std::fabs(total) > 1e-11 * perm) return total > 0 ? 1 : -1;
  return insphere_exact(p);
}

// Perturbed insphere (Section 2.4 item 3). With the lifting |p_i|^2 + eps_i, the determinant
// gains sum_i (-1)^i eps_i O_i where O_i is orient3d of the other four points in their order
// (i = 0..4 for a, b, c, d, e). eps_i is larger for larger input index, so the first non-zero
// O_i in decreasing-index order gives the sign. Negative result = inside.
int insphere_sos(const double* const p[5], const int64_t id[5]) {
  int s = insphere(p);
  if (s != 0) return s;
  ++g_cnt.sos;
  int ord[5] = {0, 1, 2, 3, 4};
  std::sort(ord, ord + 5, [&](int x, int y) {
    return g_mut == 2 ? id[x] < id[y] : id[x] > id[y];
  });
  for (int t = 0; t < 5; ++t) {
    int i = ord[t];
    const double* q[4];
    int j = 0;
    for (int k = 0; k < 5; ++k)
      if (k != i) q[j++] = p[k];
    int o = orient3d(q[0], q[1], q[2], q[3]);
    int sg = (i % 2 == 0) ? 1 : -1;
    if (g_mut == 1 && i == 4) sg = -sg;
    if (o != 0) return sg * o;
  }
  return 0;
}

// Exact test that c lies on the line ab: every component of (b-a) x (c-a) is zero.
bool collinear_exact(const double* a, const double* b, const double* c) {
  double all[9];
  for (int k = 0; k < 3; ++k) {
    all[k] = a[k];
    all[3 + k] = b[k];
    all[6 + k] = c[k];
  }
  int E = common_exp(all, 9);
  Big u[3], v[3];
  for (int k = 0; k < 3; ++k) {
    Big A = big_from_double(a[k], E);
    u[k] = sub(big_from_double(b[k], E), A);
    v[k] = sub(big_from_double(c[k], E), A);
  }
  return sub(mul(u[1], v[2]), mul(u[2], v[1])).sign == 0 &&
         sub(mul(u[2], v[0]), mul(u[0], v[2])).sign == 0 &&
         sub(mul(u[0], v[1]), mul(u[1], v[0])).sign == 0;
}

// ------------------------------------------------------------------ Moore curve (Section 2.3)
// Hamilton's Gray-code Hilbert construction in 3 dimensions, bit 0 = x, 1 = y, 2 = z.
// A sub-cube curve has state (e, d): it enters at corner e and leaves at corner e ^ (1 << d).
// The closed (Moore) curve visits the 8 octants in Gray-code order; the octant visited w-th is
// entered at corner ~gray(w) ^ M[w] and left at ~gray(w) ^ M[w+1] (indices mod 8), with
// M = {x, 0, z, 0, y, y|z, z, 0}; consecutive octants then meet in face-adjacent cells and the
// last octant meets the first.
unsigned gray(unsigned i) { return i ^ (i >> 1); }
unsigned gray_inverse(unsigned g) { return g ^ (g >> 1) ^ (g >> 2); }
unsigned trailing_ones(unsigned i) {
  unsigned c = 0;
  while (i & 1u) {
    ++c;
    i >>= 1;
  }
  return c;
}
unsigned rotr3(unsigned b, unsigned r) {
  r %= 3;
  return ((b >> r) | (b << (3 - r))) & 7u;
}
unsigned rotl3(unsigned b, unsigned r) {
  r %= 3;
  return ((b << r) | (b >> (3 - r))) & 7u;
}
unsigned hilbert_entry(unsigned w) { return w == 0 ? 0u : gray(2u * ((w - 1u) / 2u)); }
unsigned hilbert_dir(unsigned w) {
  if (w == 0) return 0u;
  return (w % 2 == 0) ? trailing_ones(w - 1) % 3 : trailing_ones(w) % 3;
}
const unsigned kMooreM[8] = {1u, 0u, 4u, 0u, 2u, 6u, 4u, 0u};
unsigned axis_of(unsigned onehot) { return onehot == 1u ? 0u : (onehot == 2u ? 1u : 2u); }

uint64_t moore_index(uint32_t x, uint32_t y, uint32_t z, int m) {
  auto bits = [&](int i) -> unsigned {
    return ((x >> i) & 1u) | (((y >> i) & 1u) << 1) | (((z >> i) & 1u) << 2);
  };
  unsigned w = gray_inverse(bits(m - 1));
  uint64_t key = w;
  unsigned e = ((~gray(w)) & 7u) ^ kMooreM[w];
  unsigned d = axis_of(kMooreM[w] ^ kMooreM[(w + 1) % 8]);
  for (int i = m - 2; i >= 0; --i) {
    unsigned t = rotr3(bits(i) ^ e, g_mut == 6 ? d : d + 1);
    unsigned v = gray_inverse(t);
    key = (key << 3) | v;
    e ^= rotl3(hilbert_entry(v), d + 1);
    d = (d + hilbert_dir(v) + 1) % 3;
  }
  return key;
}

constexpr int kLevels = 21;

void moore_keys(const double* xyz, int64_t n, uint64_t* keys) {
  double mn[3], mx[3], scale[3];
  for (int k = 0; k < 3; ++k) {
    mn[k] = INFINITY;
    mx[k] = -INFINITY;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      mn[k] = std::min(mn[k], xyz[3 * i + k]);
      mx[k] = std::max(mx[k], xyz[3 * i + k]);
    }
  const double cells = g_mut == 8 ? 1048576.0 : 2097152.0;  // 2^21
  for (int k = 0; k < 3; ++k) {
    double ext = mx[k] - mn[k];
    scale[k] = ext > 0.0 ? cells / ext : 0.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      double t = xyz[3 * i + k] - mn[k];
      double s = t * scale[k];
      double f = std::floor(s);
      if (f < 0.0) f = 0.0;
      if (f > 2097151.0) f = 2097151.0;
      q[k] = (uint32_t)f;
    }
    keys[i] = moore_index(q[0], q[1], q[2], kLevels);
  }
}

// ------------------------------------------------------------------ BRIO (Section 2.3, Table 2)
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
uint64_t brio_hash(uint64_t seed, uint64_t i) { return mix64((seed ^ i) + 0x9E3779B97F4A7C15ull); }

void brio_rounds(int64_t n, uint64_t seed, uint8_t* rounds) {
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::vector<uint64_t> h(n);
  for (int64_t i = 0; i < n; ++i) h[i] = brio_hash(seed, (uint64_t)i);
  std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    return h[a] != h[b] ? h[a] < h[b] : a < b;
  });
  for (int64_t rank = 0; rank < n; ++rank) {
    int r = 0;
    int64_t end = g_mut == 7 ? 2047 : 2048;
    while (rank >= end) {
      ++r;
      end *= 7;
    }
    rounds[idx[rank]] = (uint8_t)r;
  }
}

void insertion_order(const double* xyz, int64_t n, uint64_t seed, std::vector<int64_t>& order) {
  std::vector<uint64_t> keys(n);
  std::vector<uint8_t> rounds(n);
  moore_keys(xyz, n, keys.data());
  brio_rounds(n, seed, rounds.data());
  order.resize(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    if (rounds[a] != rounds[b]) return rounds[a] < rounds[b];
    if (keys[a] != keys[b]) return keys[a] < keys[b];
    return a < b;
  });
}

void dedup(const double* xyz, int64_t n, std::vector<int64_t>& rep) {
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  auto less = [&](int64_t a, int64_t b) {
    for (int k = 0; k < 3; ++k)
      if (xyz[3 * a + k] != xyz[3 * b + k]) return xyz[3 * a + k] < xyz[3 * b + k];
    return a < b;
  };
  std::sort(idx.begin(), idx.end(), less);
  rep.assign(n, -1);
  for (int64_t s = 0; s < n;) {
    int64_t e = s + 1;
    while (e < n && xyz[3 * idx[e]] == xyz[3 * idx[s]] && xyz[3 * idx[e] + 1] == xyz[3 * idx[s] + 1] &&
           xyz[3 * idx[e] + 2] == xyz[3 * idx[s] + 2])
      ++e;
    for (int64_t k = s; k < e; ++k) rep[idx[k]] = idx[s];
    s = e;
  }
}

bool finite_input(const double* xyz, int64_t n) {
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(xyz[i])) return false;
  return true;
}

// ------------------------------------------------------------------ canonical output
void canonical(uint32_t t[4]) {
  int k = 0;
  for (int i = 1; i < 4; ++i)
    if (t[i] < t[k]) k = i;
  // even permutation bringing position k to the front
  static const int perm[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 0, 1, 3}, {3, 0, 2, 1}};
  uint32_t r[4];
  for (int i = 0; i < 4; ++i) r[i] = t[perm[k][i]];
  // cyclic rotation of positions 1..3 (even) so the smallest of them comes first
  int j = 1;
  for (int i = 2; i < 4; ++i)
    if (r[i] < r[j]) j = i;
  uint32_t a = r[1], b = r[2], c = r[3];
  if (j == 2) {
    r[1] = b; r[2] = c; r[3] = a;
  } else if (j == 3) {
    r[1] = c; r[2] = a; r[3] = b;
  }
  std::memcpy(t, r, sizeof(r));
}

void sort_tets(std::vector<std::array<uint32_t, 4>>& tets) { std::sort(tets.begin(), tets.end()); }

// ------------------------------------------------------------------ mesh and Algorithm 1
struct Mesh {
  const double* xyz;
  std::vector<std::array<uint32_t, 4>> v;  // vertex ids (input indices), GHOST for the ghost
  std::vector<std::array<uint32_t, 4>> n;  // neighbours 4*t + facet (Section 2.2)
  std::vector<uint8_t> alive;
  std::vector<uint32_t> free_slots;
  std::vector<uint64_t> stamp;
  uint64_t cur_stamp = 0;

  const double* P(uint32_t id) const { return xyz + 3 * (size_t)id; }
  int gpos(uint32_t t) const {
    for (int k = 0; k < 4; ++k)
      if (v[t][k] == GHOST) return k;
    return -1;
  }
  uint32_t alloc() {
    if (!free_slots.empty()) {
      uint32_t s = free_slots.back();
      free_slots.pop_back();
      return s;
    }
    v.push_back({0, 0, 0, 0});
    n.push_back({NONE, NONE, NONE, NONE});
    alive.push_back(0);
    stamp.push_back(0);
    return (uint32_t)(v.size() - 1);
  }
  int orient_with(const std::array<uint32_t, 4>& q) const {
    return orient3d(P(q[0]), P(q[1]), P(q[2]), P(q[3]));
  }
  int insphere_with(const std::array<uint32_t, 4>& t, uint32_t p) const {
    const double* pts[5] = {P(t[0]), P(t[1]), P(t[2]), P(t[3]), P(p)};
    int64_t ids[5] = {t[0], t[1], t[2], t[3], p};
    return insphere_sos(pts, ids);
  }
  // Cavity membership (Section 2.1; ghosts per Section 2.6).
  bool conflict(uint32_t t, uint32_t p) const {
    int k = gpos(t);
    if (k < 0) return insphere_with(v[t], p) < 0;
    std::array<uint32_t, 4> q = v[t];
    q[k] = p;
    int o = orient_with(q);
    if (o != 0) return o > 0;
    if (g_mut == 5) return false;
    uint32_t r = n[t][k] >> 2;
    return insphere_with(v[r], p) < 0;
  }
};

// Fills n[] for the tetrahedra listed in `ts` by matching facets with equal vertex sets.
void match_facets(Mesh& M, const std::vector<uint32_t>& ts) {
  std::vector<std::pair<std::array<uint32_t, 3>, uint32_t>> f;
  for (uint32_t t : ts)
    for (int i = 0; i < 4; ++i) {
      std::array<uint32_t, 3> key;
      int j = 0;
      for (int k = 0; k < 4; ++k)
        if (k != i) key[j++] = M.v[t][k];
      std::sort(key.begin(), key.end());
      f.push_back({key, 4 * t + (uint32_t)i});
    }
  std::sort(f.begin(), f.end());
  for (size_t i = 0; i + 1 < f.size(); ++i)
    if (f[i].first == f[i + 1].first) {
      uint32_t a = f[i].second, b = f[i + 1].second;
      M.n[a >> 2][a & 3] = b;
      M.n[b >> 2][b & 3] = a;
      ++i;
    }
}

struct Insert {
  Mesh& M;
  uint32_t last = 0;
  int64_t walk_steps = 0, cav = 0, ball = 0;
  std::vector<uint32_t> C;
  std::vector<std::pair<uint32_t, int>> B;

  explicit Insert(Mesh& m) : M(m) {}

  // Walk (Section 2.1, with the ghost rules of Section 2.6).
  int64_t locate(uint32_t p, uint32_t* out) {
    uint32_t t = last;
    int k = M.gpos(t);
    if (k >= 0) t = M.n[t][k] >> 2;
    int64_t steps = 0, limit = 4 * (int64_t)M.v.size() + 1000;
    for (;;) {
      if (M.gpos(t) >= 0) break;
      bool moved = false;
      for (int i = 0; i < 4; ++i) {
        std::array<uint32_t, 4> q = M.v[t];
        q[i] = p;
        if (M.orient_with(q) < 0) {
          t = M.n[t][i] >> 2;
          moved = true;
          break;
        }
      }
      if (!moved) break;
      if (++steps > limit) return -1;
    }
    *out = t;
    return steps;
  }

  int insert(uint32_t p) {
    uint32_t t0;
    int64_t steps = locate(p, &t0);
    if (steps < 0) return ORACLE_EINTERNAL;
    walk_steps += steps;
    // Cavity: breadth-first search over tetrahedra in conflict with p.
    ++M.cur_stamp;
    C.clear();
    B.clear();
    if (!M.conflict(t0, p)) return ORACLE_EINTERNAL;
    C.push_back(t0);
    M.stamp[t0] = M.cur_stamp;
    for (size_t q = 0; q < C.size(); ++q) {
      uint32_t t = C[q];
      for (int i = 0; i < 4; ++i) {
        uint32_t u = M.n[t][i] >> 2;
        if (M.stamp[u] == M.cur_stamp) continue;
        if (M.conflict(u, p)) {
          M.stamp[u] = M.cur_stamp;
          C.push_back(u);
        } else {
          B.push_back({t, i});
        }
      }
    }
    cav += (int64_t)C.size();
    ball += (int64_t)B.size();
    // DelaunayBall: one new tetrahedron per boundary facet, the cavity tetrahedron with its
    // vertex opposite that facet replaced by p (Section 2.5).
    struct NewTet {
      std::array<uint32_t, 4> v;
      int i;
      uint32_t out;
    };
    std::vector<NewTet> nt;
    nt.reserve(B.size());
    for (auto& b : B) {
      std::array<uint32_t, 4> q = M.v[b.first];
      q[b.second] = p;
      nt.push_back({q, b.second, M.n[b.first][b.second]});
    }
    for (uint32_t t : C) {
      M.alive[t] = 0;
      M.free_slots.push_back(t);
    }
    std::vector<uint32_t> slots(nt.size());
    std::vector<std::pair<std::pair<uint32_t, uint32_t>, uint32_t>> inner;
    for (size_t k = 0; k < nt.size(); ++k) {
      uint32_t s = M.alloc();
      slots[k] = s;
      M.v[s] = nt[k].v;
      M.alive[s] = 1;
      M.n[s] = {NONE, NONE, NONE, NONE};
      M.n[s][nt[k].i] = nt[k].out;
      M.n[nt[k].out >> 2][nt[k].out & 3] = 4 * s + (uint32_t)nt[k].i;
    }
    // Adjacencies between new tetrahedra: facet j != i holds p and an edge of the boundary.
    for (size_t k = 0; k < nt.size(); ++k)
      for (int j = 0; j < 4; ++j) {
        if (j == nt[k].i) continue;
        uint32_t e[2];
        int m = 0;
        for (int l = 0; l < 4; ++l)
          if (l != j && l != nt[k].i) e[m++] = nt[k].v[l];
        inner.push_back({{std::min(e[0], e[1]), std::max(e[0], e[1])}, 4 * slots[k] + (uint32_t)j});
      }
    std::sort(inner.begin(), inner.end());
    if (inner.size() % 2) return ORACLE_EINTERNAL;
    for (size_t k = 0; k < inner.size(); k += 2) {
      if (inner[k].first != inner[k + 1].first) return ORACLE_EINTERNAL;
      uint32_t a = inner[k].second, b = inner[k + 1].second;
      M.n[a >> 2][a & 3] = b;
      M.n[b >> 2][b & 3] = a;
    }
    last = slots.empty() ? last : slots[0];
    return ORACLE_OK;
  }
};

int64_t validate(const Mesh& M, int64_t* ghosts_out, int64_t* hullv_out) {
  int64_t flags = 0, ghosts = 0;
  std::vector<uint32_t> hv;
  for (uint32_t t = 0; t < M.v.size(); ++t) {
    if (!M.alive[t]) continue;
    int k = M.gpos(t);
    if (k < 0) {
      if (M.orient_with(M.v[t]) <= 0) flags |= ORACLE_BAD_ORIENT;
    } else {
      ++ghosts;
      for (int i = 0; i < 4; ++i)
        if (i != k) hv.push_back(M.v[t][i]);
      uint32_t h = M.n[t][k];
      uint32_t r = h >> 2;
      if (h == NONE || M.gpos(r) >= 0) {
        flags |= ORACLE_BAD_GHOST;
      } else {
        std::array<uint32_t, 4> q = M.v[t];
        q[k] = M.v[r][h & 3];
        if (M.orient_with(q) >= 0) flags |= ORACLE_BAD_GHOST;
      }
    }
    for (int i = 0; i < 4; ++i) {
      uint32_t h = M.n[t][i];
      if (h == NONE) {
        flags |= ORACLE_BAD_ADJACENCY;
        continue;
      }
      uint32_t u = h >> 2, j = h & 3;
      if (u >= M.v.size() || !M.alive[u] || M.n[u][j] != 4 * t + (uint32_t)i) {
        flags |= ORACLE_BAD_ADJACENCY;
        continue;
      }
      std::array<uint32_t, 3> a, b;
      int x = 0, y = 0;
      for (int l = 0; l < 4; ++l) {
        if (l != i) a[x++] = M.v[t][l];
        if (l != (int)j) b[y++] = M.v[u][l];
      }
      std::sort(a.begin(), a.end());
      std::sort(b.begin(), b.end());
      if (a != b) flags |= ORACLE_BAD_ADJACENCY;
      if (k < 0 && M.gpos(u) < 0 && M.insphere_with(M.v[t], M.v[u][j]) <= 0)
        flags |= ORACLE_BAD_DELAUNAY;
    }
  }
  std::sort(hv.begin(), hv.end());
  hv.erase(std::unique(hv.begin(), hv.end()), hv.end());
  if (ghosts != 2 * (int64_t)hv.size() - 4) flags |= ORACLE_BAD_HULLCOUNT;
  *ghosts_out = ghosts;
  *hullv_out = (int64_t)hv.size();
  return flags;
}

int64_t write_out(std::vector<std::array<uint32_t, 4>>& tets, uint32_t* out, int64_t cap,
                  oracle_stats* st) {
  for (auto& t : tets) canonical(t.data());
  sort_tets(tets);
  if (st) st->n_tets = (int64_t)tets.size();
  if ((int64_t)tets.size() > cap) return ORACLE_ETOOSMALL;
  for (size_t i = 0; i < tets.size(); ++i)
    for (int k = 0; k < 4; ++k) out[4 * i + k] = tets[i][k];
  return (int64_t)tets.size();
}

int64_t delaunay(const double* xyz, int64_t n, uint64_t seed, const int64_t* order_in,
                 uint32_t* out, int64_t cap, int do_validate, oracle_stats* st) {
  if (n < 0 || (n > 0 && !xyz) || n >= (int64_t)0xFFFFFFFF) return ORACLE_EINVAL;
  if (!finite_input(xyz, n)) return ORACLE_EINVAL;
  g_cnt = Counters();
  std::vector<int64_t> rep;
  dedup(xyz, n, rep);
  std::vector<int64_t> order;
  if (order_in) {
    std::vector<uint8_t> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
      if (order_in[i] < 0 || order_in[i] >= n || seen[order_in[i]]) return ORACLE_EINVAL;
      seen[order_in[i]] = 1;
    }
    order.assign(order_in, order_in + n);
  } else {
    insertion_order(xyz, n, seed, order);
  }
  std::vector<uint32_t> seq;
  for (int64_t i : order)
    if (rep[i] == i) seq.push_back((uint32_t)i);
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->n_points = n;
    st->n_unique = (int64_t)seq.size();
    st->n_dups = n - (int64_t)seq.size();
  }
  // Init (Section 2.1): the first four non-coplanar vertices of the order.
  if (seq.size() < 4) return ORACLE_EDEGENERATE;
  Mesh M;
  M.xyz = xyz;
  // Storage only: a uniform cloud ends with about 6.8 slots per point; reserving them up front
  // keeps a 1e8-point run from doubling its vectors past the host's memory.
  const size_t slots_hint = 7 * seq.size() + 64;
  M.v.reserve(slots_hint);
  M.n.reserve(slots_hint);
  M.alive.reserve(slots_hint);
  M.stamp.reserve(slots_hint);
  size_t k2 = 2;
  while (k2 < seq.size() && collinear_exact(M.P(seq[0]), M.P(seq[1]), M.P(seq[k2]))) ++k2;
  if (k2 >= seq.size()) return ORACLE_EDEGENERATE;
  size_t k3 = k2 + 1;
  while (k3 < seq.size() && orient3d(M.P(seq[0]), M.P(seq[1]), M.P(seq[k2]), M.P(seq[k3])) == 0) ++k3;
  if (k3 >= seq.size()) return ORACLE_EDEGENERATE;
  std::array<uint32_t, 4> t0 = {seq[0], seq[1], seq[k2], seq[k3]};
  if (M.orient_with(t0) < 0) std::swap(t0[2], t0[3]);
  std::vector<uint32_t> first;
  uint32_t s0 = M.alloc();
  M.v[s0] = t0;
  M.alive[s0] = 1;
  first.push_back(s0);
  for (int i = 0; i < 4; ++i) {
    // ghost over facet i: the ghost vertex replaces vertex i and two others swap, so that a
    // point beyond the hull facet makes the tetrahedron positive.
    std::array<uint32_t, 4> g = t0;
    g[i] = GHOST;
    int a = (i == 0) ? 1 : 0, b = (i == 1 || i == 0) ? 2 : 1;
    std::swap(g[a], g[b]);
    uint32_t s = M.alloc();
    M.v[s] = g;
    M.alive[s] = 1;
    first.push_back(s);
  }
  match_facets(M, first);
  Insert I(M);
  I.last = s0;
  for (size_t q = 0; q < seq.size(); ++q) {
    if (q == 0 || q == 1 || q == k2 || q == k3) continue;
    int rc = I.insert(seq[q]);
    if (rc != ORACLE_OK) return rc;
  }
  int64_t ghosts = 0, hullv = 0;
  int64_t flags = 0;
  if (do_validate) flags = validate(M, &ghosts, &hullv);
  if (st) {
    st->sum_cavity = I.cav;
    st->sum_ball = I.ball;
    st->sum_walk = I.walk_steps;
    st->n_insphere = g_cnt.insphere;
    st->n_exact = g_cnt.exact;
    st->n_sos = g_cnt.sos;
    st->validate_flags = flags;
    st->n_ghosts = ghosts;
    st->n_hull_vertices = hullv;
  }
  // Output: the finite tetrahedra go straight into the caller's buffer, canonical and sorted
  // there, after the mesh is released (storage only; the same list as collecting them first).
  int64_t T = 0;
  for (uint32_t t = 0; t < M.v.size(); ++t)
    if (M.alive[t] && M.gpos(t) < 0) ++T;
  if (st) st->n_tets = T;
  if (T > cap || !out) return ORACLE_ETOOSMALL;
  int64_t w = 0;
  for (uint32_t t = 0; t < M.v.size(); ++t)
    if (M.alive[t] && M.gpos(t) < 0) {
      for (int k = 0; k < 4; ++k) out[4 * w + k] = M.v[t][k];
      canonical(out + 4 * w);
      ++w;
    }
  { Mesh empty; std::swap(M.v, empty.v); std::swap(M.n, empty.n); std::swap(M.alive, empty.alive);
    std::swap(M.stamp, empty.stamp); }
  static_assert(sizeof(std::array<uint32_t, 4>) == 16, "rows are four packed ids");
  auto* rows = reinterpret_cast<std::array<uint32_t, 4>*>(out);
  std::sort(rows, rows + T);
  return T;
}

int64_t brute_force(const double* xyz, int64_t n, uint32_t* out, int64_t cap) {
  if (n < 0 || n > 200 || (n > 0 && !xyz) || !finite_input(xyz, n)) return ORACLE_EINVAL;
  std::vector<int64_t> rep;
  dedup(xyz, n, rep);
  std::vector<uint32_t> u;
  for (int64_t i = 0; i < n; ++i)
    if (rep[i] == i) u.push_back((uint32_t)i);
  const double* X = xyz;
  auto P = [&](uint32_t id) { return X + 3 * (size_t)id; };
  std::vector<std::array<uint32_t, 4>> tets;
  size_t m = u.size();
  for (size_t a = 0; a < m; ++a)
    for (size_t b = a + 1; b < m; ++b)
      for (size_t c = b + 1; c < m; ++c)
        for (size_t d = c + 1; d < m; ++d) {
          std::array<uint32_t, 4> t = {u[a], u[b], u[c], u[d]};
          int o = orient3d(P(t[0]), P(t[1]), P(t[2]), P(t[3]));
          if (o == 0) continue;
          if (o < 0) std::swap(t[2], t[3]);
          bool empty = true;
          for (size_t e = 0; e < m && empty; ++e) {
            uint32_t q = u[e];
            if (q == t[0] || q == t[1] || q == t[2] || q == t[3]) continue;
            const double* pts[5] = {P(t[0]), P(t[1]), P(t[2]), P(t[3]), P(q)};
            int64_t ids[5] = {t[0], t[1], t[2], t[3], q};
            if (insphere_sos(pts, ids) < 0) empty = false;
          }
          if (empty) tets.push_back(t);
        }
  return write_out(tets, out, cap, nullptr);
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int oracle_moore_keys(const double* xyz, int64_t n, uint64_t* keys) {
  if (n < 0 || (n > 0 && (!xyz || !keys)) || !finite_input(xyz, n)) return ORACLE_EINVAL;
  moore_keys(xyz, n, keys);
  return ORACLE_OK;
}

int oracle_moore_index(const uint32_t* q, int64_t n, int m, uint64_t* keys) {
  if (n < 0 || m < 1 || m > 21 || (n > 0 && (!q || !keys))) return ORACLE_EINVAL;
  for (int64_t i = 0; i < n; ++i) keys[i] = moore_index(q[3 * i], q[3 * i + 1], q[3 * i + 2], m);
  return ORACLE_OK;
}

int oracle_brio_rounds(int64_t n, uint64_t seed, uint8_t* rounds) {
  if (n < 0 || (n > 0 && !rounds)) return ORACLE_EINVAL;
  try {
    brio_rounds(n, seed, rounds);
  } catch (const std::bad_alloc&) {
    return ORACLE_EINTERNAL;
  }
  return ORACLE_OK;
}

int oracle_insertion_order(const double* xyz, int64_t n, uint64_t seed, uint32_t* perm) {
  if (n < 0 || (n > 0 && (!xyz || !perm)) || !finite_input(xyz, n)) return ORACLE_EINVAL;
  try {
    std::vector<int64_t> order;
    insertion_order(xyz, n, seed, order);
    for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)order[i];
  } catch (const std::bad_alloc&) {
    return ORACLE_EINTERNAL;
  }
  return ORACLE_OK;
}

int oracle_dedup(const double* xyz, int64_t n, uint32_t* rep) {
  if (n < 0 || (n > 0 && (!xyz || !rep))) return ORACLE_EINVAL;
  std::vector<int64_t> r;
  dedup(xyz, n, r);
  for (int64_t i = 0; i < n; ++i) rep[i] = (uint32_t)r[i];
  return ORACLE_OK;
}

int oracle_orient3d(const double* p) { return orient3d(p, p + 3, p + 6, p + 9); }

int oracle_insphere(const double* p) {
  const double* q[5] = {p, p + 3, p + 6, p + 9, p + 12};
  return insphere(q);
}

int oracle_insphere_sos(const double* p, const int64_t* ids) {
  const double* q[5] = {p, p + 3, p + 6, p + 9, p + 12};
  return insphere_sos(q, ids);
}

double oracle_insphere_value(const double* p) {
  const double* q[5] = {p, p + 3, p + 6, p + 9, p + 12};
  double v = 0.0;
  insphere_exact(q, &v);
  return v;
}

double oracle_orient3d_value(const double* p) {
  double v = 0.0;
  orient3d_exact(p, p + 3, p + 6, p + 9, &v);
  return v;
}

int64_t oracle_delaunay(const double* xyz, int64_t n, uint64_t seed, const int64_t* order,
                        uint32_t* tets_out, int64_t cap, int validate_mesh, oracle_stats* stats) {
  try {
    return delaunay(xyz, n, seed, order, tets_out, cap, validate_mesh, stats);
  } catch (const std::bad_alloc&) {
    return ORACLE_EINTERNAL;
  }
}

int64_t oracle_brute_force(const double* xyz, int64_t n, uint32_t* tets_out, int64_t cap) {
  try {
    return brute_force(xyz, n, tets_out, cap);
  } catch (const std::bad_alloc&) {
    return ORACLE_EINTERNAL;
  }
}

int oracle_adjacency(const uint32_t* tets, int64_t T, uint32_t* nbr) {
  if (T < 0 || (T > 0 && (!tets || !nbr))) return ORACLE_EINVAL;
  Mesh M;
  M.xyz = nullptr;
  std::vector<uint32_t> ts;
  for (int64_t t = 0; t < T; ++t) {
    uint32_t s = M.alloc();
    for (int k = 0; k < 4; ++k) M.v[s][k] = tets[4 * t + k];
    ts.push_back(s);
  }
  match_facets(M, ts);
  for (int64_t t = 0; t < T; ++t)
    for (int k = 0; k < 4; ++k) nbr[4 * t + k] = M.n[t][k];
  return ORACLE_OK;
}

void oracle_set_mutation(int k) { g_mut = k; }

}  // extern "C"
