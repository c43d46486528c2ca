// The paper's CPU parallel insertion (Section 3.2 to 3.4) as a second host baseline beside the
// serial oracle: TEST AND BASELINE INFRASTRUCTURE ONLY (used by the tests and the benchmark's CPU
// legs; it shares no code with the GPU library).
//
// It reuses the serial oracle's predicates, Moore index, BRIO rounds, duplicate removal and
// canonical output (the oracle's source is included below) and adds the thread scheme:
//   - the points to insert are sorted by Moore index and cut into one range of equal count per
//     thread; every vertex (inserted or not) belongs to the range its index falls in; the ghost
//     vertex belongs to none;
//   - a tetrahedron belongs to a thread when at least three of its vertices are in its range,
//     otherwise it is in the buffer zone (Fig. 5);
//   - a thread aborts a point when its cavity touches a tetrahedron that is not its own, or when
//     its walk ends on one; aborted points are retried in the next pass, with partitions from
//     the transformed curve (coordinates compressed below and expanded above a random threshold
//     per axis, the index circularly shifted; Fig. 6);
//   - the first BRIO round is inserted by one thread; the thread count halves when the success
//     ratio falls below 1/5 or a thread would get fewer than 3000 points, and one thread takes
//     the rest when the ratio falls to 1/threads or less;
//   - each thread reuses only the slots it freed, new slots come in chunks from one atomic
//     counter (Section 3.4's rule that two threads never create tetrahedra at one index).
// Every field another thread can be writing is read through relaxed atomics, so a walk may cross
// other threads' tetrahedra and see them half-updated; it only proposes a start, which the thread
// must own, and everything the cavity touches is then the thread's own and stable. (The paper
// stops walks at the partition border; a walk here may cross it, which keeps hints useful after
// re-partitioning.) The result equals the serial oracle's: the perturbed Delaunay triangulation
// is unique, whatever the insertion order.
#include "oracle.cpp"

#include <atomic>
#include <memory>
#include <random>
#include <system_error>
#include <thread>

namespace {

constexpr uint64_t kChunk = 256;

// The curve of one pass (pass 0: the plain curve of the oracle's insertion order): per axis,
// u = (x - min) / extent is compressed below a random threshold th and expanded above it
// (u < th: u / (2 th), else 1/2 + (u - th) / (2 (1 - th))), quantised to 21 bits and indexed, and
// the index is shifted circularly by a random amount. bound holds the first index of ranges
// 1 .. T-1.
struct Curve {
  const double* xyz = nullptr;
  double mn[3], ext[3], th[3] = {0.5, 0.5, 0.5};
  uint64_t shift = 0, pass = 0;
  std::vector<uint64_t> bound;

  Curve(const double* x, const double* lo, const double* e, int p, uint64_t seed) : xyz(x), pass((uint64_t)p) {
    for (int k = 0; k < 3; ++k) mn[k] = lo[k], ext[k] = e[k];
    if (p > 0) {
      std::mt19937_64 rng(seed * 0x9E3779B97F4A7C15ull + (uint64_t)p);
      for (int k = 0; k < 3; ++k) th[k] = 0.25 + 0.5 * (double)(rng() >> 11) * 0x1.0p-53;
      shift = rng() & ((1ull << 63) - 1);
    }
  }
  uint64_t key(uint32_t id) const {
    const double* x = xyz + 3 * (size_t)id;
    uint32_t qc[3];
    for (int k = 0; k < 3; ++k) {
      double u = ext[k] > 0.0 ? (x[k] - mn[k]) / ext[k] : 0.0;
      if (pass > 0) u = u < th[k] ? u / (2.0 * th[k]) : 0.5 + (u - th[k]) / (2.0 * (1.0 - th[k]));
      double f = std::floor(u * 2097152.0);
      if (!(f >= 0.0)) f = 0.0;
      if (f > 2097151.0) f = 2097151.0;
      qc[k] = (uint32_t)f;
    }
    return (moore_index(qc[0], qc[1], qc[2], kLevels) + shift) & ((1ull << 63) - 1);
  }
  uint32_t range_of_key(uint64_t k) const {
    return (uint32_t)(std::upper_bound(bound.begin(), bound.end(), k) - bound.begin());
  }
};

struct PMesh {
  const double* xyz = nullptr;
  uint64_t cap = 0;
  std::unique_ptr<std::atomic<uint32_t>[]> V, N;  // 4 per slot: vertex ids, neighbours 4 t + facet
  std::unique_ptr<std::atomic<uint8_t>[]> alive;
  std::unique_ptr<uint64_t[]> stamp;  // touched only by the thread that owns the slot
  std::atomic<uint64_t> bump{0};
  // Range of every point (input index) under the current pass's partition, computed on first
  // use in a pass: (pass + 1) << 32 | range.
  std::unique_ptr<std::atomic<uint64_t>[]> tag;
  const struct Curve* curve = nullptr;

  const double* P(uint32_t id) const { return xyz + 3 * (size_t)id; }
  void getv(uint32_t t, uint32_t q[4]) const {
    for (int k = 0; k < 4; ++k) q[k] = V[4 * (size_t)t + k].load(std::memory_order_relaxed);
  }
  uint32_t getn(uint32_t t, int k) const { return N[4 * (size_t)t + k].load(std::memory_order_relaxed); }
  void setv(uint32_t t, const std::array<uint32_t, 4>& q) {
    for (int k = 0; k < 4; ++k) V[4 * (size_t)t + k].store(q[k], std::memory_order_relaxed);
  }
  void setn(uint32_t t, int k, uint32_t x) { N[4 * (size_t)t + k].store(x, std::memory_order_relaxed); }
  // A live slot at or after `from` (wrapping), or cap when there is none.
  uint64_t find_live(uint64_t from) const {
    const uint64_t used = std::min<uint64_t>(bump.load(std::memory_order_relaxed), cap);
    for (uint64_t k = 0; k < used; ++k) {
      const uint64_t s = (from + k) % used;
      if (alive[s].load(std::memory_order_relaxed)) return s;
    }
    return cap;
  }
  uint32_t part_of(uint32_t id) const {
    const uint64_t now = (curve->pass + 1) << 32;
    uint64_t t = tag[id].load(std::memory_order_relaxed);
    if ((t & ~0xFFFFFFFFull) == now) return (uint32_t)t;
    const uint32_t r = curve->range_of_key(curve->key(id));
    tag[id].store(now | r, std::memory_order_relaxed);
    return r;
  }
};

int gpos4(const uint32_t q[4]) {
  for (int k = 0; k < 4; ++k)
    if (q[k] == GHOST) return k;
  return -1;
}

struct Worker {
  PMesh& M;
  int me = 0;
  uint32_t last = 0;
  std::vector<uint32_t> free_slots;
  uint64_t lo = 0, hi = 0;  // the current chunk of fresh slots
  int64_t walk = 0, cav = 0, ball = 0;
  uint64_t stamp_seq = 0;  // visit stamps (me + 1) << 48 | sequence: unique across threads
  std::vector<uint32_t> C;
  std::vector<std::pair<uint32_t, int>> B;
  struct NewTet {
    std::array<uint32_t, 4> v;
    int i;
    uint32_t out;
  };
  std::vector<NewTet> nt;  // reused by every insertion of the thread
  std::vector<uint32_t> slots;
  std::vector<std::pair<std::pair<uint32_t, uint32_t>, uint32_t>> inner;

  explicit Worker(PMesh& m) : M(m) {}

  bool mine(const uint32_t q[4]) const {
    int c = 0;
    for (int k = 0; k < 4; ++k)
      if (q[k] != GHOST && M.part_of(q[k]) == (uint32_t)me) ++c;
    return c >= 3;
  }
  bool owned(uint32_t t) const {
    if (t >= M.cap || !M.alive[t].load(std::memory_order_relaxed)) return false;
    uint32_t q[4];
    M.getv(t, q);
    return mine(q);
  }
  bool alloc(uint32_t* s) {
    if (!free_slots.empty()) {
      *s = free_slots.back();
      free_slots.pop_back();
      return true;
    }
    if (lo == hi) {
      lo = M.bump.fetch_add(kChunk);
      hi = lo + kChunk;
      if (hi > M.cap) return false;
    }
    *s = (uint32_t)lo++;
    return true;
  }
  int orient4(const uint32_t q[4]) const { return orient3d(M.P(q[0]), M.P(q[1]), M.P(q[2]), M.P(q[3])); }
  bool in_sphere(const uint32_t q[4], uint32_t p) const {
    const double* pts[5] = {M.P(q[0]), M.P(q[1]), M.P(q[2]), M.P(q[3]), M.P(p)};
    int64_t ids[5] = {q[0], q[1], q[2], q[3], p};
    return insphere_sos(pts, ids) < 0;
  }
  // Cavity membership of an owned tetrahedron (Sections 2.1, 2.6). *ok turns false when the
  // decision needs a tetrahedron this thread does not own.
  bool conflict(uint32_t t, uint32_t p, bool* ok) const {
    uint32_t q[4];
    M.getv(t, q);
    int k = gpos4(q);
    if (k < 0) return in_sphere(q, p);
    uint32_t r[4] = {q[0], q[1], q[2], q[3]};
    r[k] = p;
    int o = orient4(r);
    if (o != 0) return o > 0;
    uint32_t u = M.getn(t, k) >> 2;
    if (!owned(u)) {
      *ok = false;
      return false;
    }
    M.getv(u, q);
    return in_sphere(q, p);
  }

  // 1: inserted; 0: aborted (another thread's tetrahedron or the buffer zone); < 0: error.
  int insert(uint32_t p) {
    // walk (Section 2.1) from the last tetrahedron this thread created
    if (last >= M.cap || !M.alive[last].load(std::memory_order_relaxed)) {
      const uint64_t s = M.find_live(last < M.cap ? last : 0);
      if (s >= M.cap) return ORACLE_EINTERNAL;
      last = (uint32_t)s;
    }
    uint32_t t = last, q[4];
    M.getv(t, q);
    int g = gpos4(q);
    if (g >= 0) t = M.getn(t, g) >> 2;
    int64_t steps = 0;
    const int64_t limit = 4 * (int64_t)M.bump.load(std::memory_order_relaxed) + 1000;
    for (;;) {
      if (t >= M.cap) return 0;
      M.getv(t, q);
      if (gpos4(q) >= 0) break;
      bool moved = false;
      for (int i = 0; i < 4; ++i) {
        uint32_t r[4] = {q[0], q[1], q[2], q[3]};
        r[i] = p;
        if (orient4(r) < 0) {
          t = M.getn(t, i) >> 2;
          moved = true;
          break;
        }
      }
      if (!moved) break;
      if (++steps > limit) return 0;
    }
    walk += steps;
    if (!owned(t)) return 0;
    bool ok = true;
    if (!conflict(t, p, &ok) || !ok) return 0;
    // cavity: breadth-first search, every tetrahedron read must be this thread's own
    const uint64_t st = ((uint64_t)(me + 1) << 48) | ++stamp_seq;
    C.clear();
    B.clear();
    C.push_back(t);
    M.stamp[t] = st;
    for (size_t k = 0; k < C.size(); ++k) {
      uint32_t c = C[k];
      for (int i = 0; i < 4; ++i) {
        uint32_t u = M.getn(c, i) >> 2;
        if (!owned(u)) return 0;
        if (M.stamp[u] == st) continue;
        bool in = conflict(u, p, &ok);
        if (!ok) return 0;
        if (in) {
          M.stamp[u] = st;
          C.push_back(u);
        } else {
          B.push_back({c, i});
        }
      }
    }
    // ball (Section 2.5): one new tetrahedron per boundary facet
    nt.clear();
    for (auto& b : B) {
      uint32_t r[4];
      M.getv(b.first, r);
      std::array<uint32_t, 4> v = {r[0], r[1], r[2], r[3]};
      v[b.second] = p;
      nt.push_back({v, b.second, M.getn(b.first, b.second)});
    }
    for (uint32_t c : C) {
      M.alive[c].store(0, std::memory_order_relaxed);
      free_slots.push_back(c);
    }
    slots.resize(nt.size());
    inner.clear();
    for (size_t k = 0; k < nt.size(); ++k) {
      uint32_t s;
      if (!alloc(&s)) return ORACLE_EINTERNAL;
      slots[k] = s;
      M.setv(s, nt[k].v);
      for (int j = 0; j < 4; ++j) M.setn(s, j, NONE);
      M.setn(s, nt[k].i, nt[k].out);
      M.setn(nt[k].out >> 2, nt[k].out & 3, 4 * s + (uint32_t)nt[k].i);
      M.stamp[s] = 0;
      M.alive[s].store(1, std::memory_order_relaxed);
    }
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
      M.setn(a >> 2, a & 3, b);
      M.setn(b >> 2, b & 3, a);
    }
    cav += (int64_t)C.size();
    ball += (int64_t)B.size();
    last = slots[0];
    return 1;
  }
};

// Runs f(a, b) on [0, n) cut into T contiguous pieces, one thread each.
template <class F>
void parallel_for(size_t n, int T, F f) {
  if (T <= 1 || n < 4096) {
    f((size_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  for (int w = 1; w < T; ++w) th.emplace_back(f, n * w / T, n * (w + 1) / T);
  f((size_t)0, n / T);
  for (auto& x : th) x.join();
}

// Sorts with T threads: pieces sorted in parallel, then merged pairwise in parallel rounds. The
// comparators used here are strict total orders (ties broken by index), so the result is the
// one std::sort gives.
template <class T_, class Cmp>
void parallel_sort(std::vector<T_>& v, int T, Cmp cmp) {
  const size_t n = v.size();
  if (T <= 1 || n < 65536) {
    std::sort(v.begin(), v.end(), cmp);
    return;
  }
  std::vector<size_t> b(T + 1);
  for (int i = 0; i <= T; ++i) b[i] = n * (size_t)i / (size_t)T;
  {
    std::vector<std::thread> th;
    for (int i = 0; i < T; ++i) th.emplace_back([&, i] { std::sort(v.begin() + b[i], v.begin() + b[i + 1], cmp); });
    for (auto& x : th) x.join();
  }
  for (int width = 1; width < T; width *= 2) {
    std::vector<std::thread> th;
    for (int i = 0; i + width < T; i += 2 * width) {
      const size_t lo = b[i], mid = b[i + width], hi = b[std::min(i + 2 * width, T)];
      th.emplace_back([&, lo, mid, hi] { std::inplace_merge(v.begin() + lo, v.begin() + mid, v.begin() + hi, cmp); });
    }
    for (auto& x : th) x.join();
  }
}

// The insertion order of the serial oracle (duplicates dropped, BRIO rounds of Table 2, Moore
// index of the 21-bit quantised coordinates, ties by index), computed with T threads.
void parallel_order(const double* xyz, int64_t n, uint64_t seed, int T, std::vector<uint32_t>& seq,
                    std::vector<uint8_t>& rounds) {
  // duplicates: sort by coordinates, then index; the first of a run represents it
  std::vector<uint32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0u);
  parallel_sort(idx, T, [&](uint32_t a, uint32_t b) {
    for (int k = 0; k < 3; ++k)
      if (xyz[3 * (size_t)a + k] != xyz[3 * (size_t)b + k]) return xyz[3 * (size_t)a + k] < xyz[3 * (size_t)b + k];
    return a < b;
  });
  std::vector<uint8_t> dup(n, 0);
  for (int64_t s = 1; s < n; ++s) {
    const double* p = xyz + 3 * (size_t)idx[s];
    const double* q = xyz + 3 * (size_t)idx[s - 1];
    if (p[0] == q[0] && p[1] == q[1] && p[2] == q[2]) dup[idx[s]] = 1;
  }
  // Moore keys on the box of all points
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      mn[k] = std::min(mn[k], xyz[3 * i + k]);
      mx[k] = std::max(mx[k], xyz[3 * i + k]);
    }
  double scale[3];
  for (int k = 0; k < 3; ++k) scale[k] = mx[k] - mn[k] > 0.0 ? 2097152.0 / (mx[k] - mn[k]) : 0.0;
  std::vector<uint64_t> key(n), h(n);
  parallel_for((size_t)n, T, [&](size_t a, size_t b) {
    for (size_t i = a; i < b; ++i) {
      uint32_t q[3];
      for (int k = 0; k < 3; ++k) {
        double f = std::floor((xyz[3 * i + k] - mn[k]) * scale[k]);
        if (f < 0.0) f = 0.0;
        if (f > 2097151.0) f = 2097151.0;
        q[k] = (uint32_t)f;
      }
      key[i] = moore_index(q[0], q[1], q[2], kLevels);
      h[i] = brio_hash(seed, (uint64_t)i);
    }
  });
  // BRIO rounds from the rank of the hash
  std::iota(idx.begin(), idx.end(), 0u);
  parallel_sort(idx, T, [&](uint32_t a, uint32_t b) { return h[a] != h[b] ? h[a] < h[b] : a < b; });
  rounds.assign(n, 0);
  parallel_for((size_t)n, T, [&](size_t a, size_t b) {
    for (size_t rank = a; rank < b; ++rank) {
      int r = 0;
      uint64_t end = 2048;
      while (rank >= end) {
        ++r;
        end *= 7;
      }
      rounds[idx[rank]] = (uint8_t)r;
    }
  });
  // order by (round, key, index), duplicates left out
  std::iota(idx.begin(), idx.end(), 0u);
  parallel_sort(idx, T, [&](uint32_t a, uint32_t b) {
    if (rounds[a] != rounds[b]) return rounds[a] < rounds[b];
    if (key[a] != key[b]) return key[a] < key[b];
    return a < b;
  });
  seq.clear();
  seq.reserve(n);
  for (uint32_t i : idx)
    if (!dup[i]) seq.push_back(i);
}

struct ParStats {
  int64_t passes = 0, aborted = 0, sequential_passes = 0, max_threads = 0;
};

// Inserts `todo` with up to T threads, passes of re-partitioned retries until none is left.
int insert_parallel(PMesh& M, std::vector<Worker>& W, std::vector<uint32_t> todo, int T, int64_t min_per_thread,
                    const double mn[3], const double ext[3], uint64_t seed, int* pass_counter, ParStats& ps) {
  std::vector<uint64_t> key_todo;
  while (!todo.empty()) {
    const int pass = (*pass_counter)++;
    ++ps.passes;
    while (T > 1 && (int64_t)todo.size() < min_per_thread * (int64_t)T) T /= 2;
    // partition: equal counts of the points to insert along the pass's curve; the mesh vertices
    // get their ranges on first use (PMesh::part_of)
    Curve curve(M.xyz, mn, ext, pass, seed);
    key_todo.resize(todo.size());
    {
      auto keys = [&](size_t a, size_t b) {
        for (size_t s = a; s < b; ++s) key_todo[s] = curve.key(todo[s]);
      };
      std::vector<std::thread> th;
      const size_t m = todo.size(), nt = (size_t)std::max(1, T);
      for (size_t w = 1; w < nt; ++w) th.emplace_back(keys, m * w / nt, m * (w + 1) / nt);
      keys(0, m / nt);
      for (auto& x : th) x.join();
    }
    std::vector<size_t> idx(todo.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
      return key_todo[a] != key_todo[b] ? key_todo[a] < key_todo[b] : todo[a] < todo[b];
    });
    for (int r = 1; r < T; ++r) curve.bound.push_back(key_todo[idx[todo.size() * r / T]]);
    M.curve = &curve;
    std::vector<std::vector<uint32_t>> mine(T);
    for (size_t s : idx) {
      const uint32_t r = curve.range_of_key(key_todo[s]);
      M.tag[todo[s]].store(((uint64_t)(pass + 1) << 32) | r, std::memory_order_relaxed);
      mine[r].push_back(todo[s]);
    }
    if (T == 1) ++ps.sequential_passes;
    ps.max_threads = std::max<int64_t>(ps.max_threads, T);
    std::vector<std::vector<uint32_t>> fail(T);
    std::vector<int> rc(T, ORACLE_OK);
    auto run = [&](int w) {
      Worker& X = W[w];
      X.me = w;
      for (uint32_t p : mine[w]) {
        int r = X.insert(p);
        if (r < 0) {
          rc[w] = r;
          return;
        }
        if (r == 0) fail[w].push_back(p);
      }
    };
    if (T == 1) {
      run(0);
    } else {
      std::vector<std::thread> th;
      for (int w = 0; w < T; ++w) th.emplace_back(run, w);
      for (auto& x : th) x.join();
    }
    M.curve = nullptr;  // the pass's curve ends here
    size_t failed = 0;
    for (int w = 0; w < T; ++w) {
      if (rc[w] != ORACLE_OK) return rc[w];
      failed += fail[w].size();
    }
    if (T == 1 && failed) return ORACLE_EINTERNAL;  // one thread owns every tetrahedron
    ps.aborted += (int64_t)failed;
    const double rho = 1.0 - (double)failed / (double)todo.size();
    std::vector<uint32_t> next;
    for (int w = 0; w < T; ++w) next.insert(next.end(), fail[w].begin(), fail[w].end());
    if (T > 1 && rho <= 1.0 / T)
      T = 1;
    else if (rho < 0.2)
      T = std::max(1, T / 2);
    todo.swap(next);
  }
  return ORACLE_OK;
}

int64_t delaunay_parallel(const double* xyz, int64_t n, uint64_t seed, int threads, int64_t min_per_thread,
                          uint32_t* out, int64_t cap, int64_t* stats) {
  if (n < 0 || (n > 0 && !xyz) || n >= (int64_t)0xFFFFFFF0 || threads < 1 || min_per_thread < 1) return ORACLE_EINVAL;
  if (!finite_input(xyz, n)) return ORACLE_EINVAL;
  std::vector<uint32_t> seq;
  std::vector<uint8_t> rounds;
  parallel_order(xyz, n, seed, threads, seq, rounds);
  if (seq.size() < 4) return ORACLE_EDEGENERATE;
  PMesh M;
  M.xyz = xyz;
  M.cap = 10 * (uint64_t)seq.size() + 64 * kChunk * (uint64_t)threads + 4096;
  M.V.reset(new std::atomic<uint32_t>[4 * M.cap]);
  M.N.reset(new std::atomic<uint32_t>[4 * M.cap]);
  M.alive.reset(new std::atomic<uint8_t>[M.cap]);
  M.stamp.reset(new uint64_t[M.cap]);
  parallel_for(M.cap, threads, [&](size_t a, size_t b) {
    for (size_t s = a; s < b; ++s) {
      for (int k = 0; k < 4; ++k) {
        M.V[4 * s + k].store(0, std::memory_order_relaxed);
        M.N[4 * s + k].store(NONE, std::memory_order_relaxed);
      }
      M.alive[s].store(0, std::memory_order_relaxed);
      M.stamp[s] = 0;
    }
  });
  M.tag.reset(new std::atomic<uint64_t>[n]);
  for (int64_t i = 0; i < n; ++i) M.tag[i].store(0, std::memory_order_relaxed);
  // Init (Section 2.1), as the serial oracle: the first four non-coplanar points of the order
  size_t k2 = 2;
  while (k2 < seq.size() && collinear_exact(M.P(seq[0]), M.P(seq[1]), M.P(seq[k2]))) ++k2;
  if (k2 >= seq.size()) return ORACLE_EDEGENERATE;
  size_t k3 = k2 + 1;
  while (k3 < seq.size() && orient3d(M.P(seq[0]), M.P(seq[1]), M.P(seq[k2]), M.P(seq[k3])) == 0) ++k3;
  if (k3 >= seq.size()) return ORACLE_EDEGENERATE;
  std::array<uint32_t, 4> t0 = {seq[0], seq[1], seq[k2], seq[k3]};
  if (orient3d(M.P(t0[0]), M.P(t0[1]), M.P(t0[2]), M.P(t0[3])) < 0) std::swap(t0[2], t0[3]);
  {
    Mesh S;  // the oracle's own initial tetrahedron and ghosts, copied into the shared store
    S.xyz = xyz;
    std::vector<uint32_t> first;
    uint32_t s0 = S.alloc();
    S.v[s0] = t0;
    S.alive[s0] = 1;
    first.push_back(s0);
    for (int i = 0; i < 4; ++i) {
      std::array<uint32_t, 4> g = t0;
      g[i] = GHOST;
      int a = (i == 0) ? 1 : 0, b = (i == 1 || i == 0) ? 2 : 1;
      std::swap(g[a], g[b]);
      uint32_t s = S.alloc();
      S.v[s] = g;
      S.alive[s] = 1;
      first.push_back(s);
    }
    match_facets(S, first);
    for (uint32_t s : first) {
      M.setv(s, S.v[s]);
      for (int k = 0; k < 4; ++k) M.setn(s, k, S.n[s][k]);
      M.alive[s].store(1, std::memory_order_relaxed);
    }
    M.bump.store(first.size());
  }
  double mn[3], mx[3], ext[3];
  for (int k = 0; k < 3; ++k) {
    mn[k] = INFINITY;
    mx[k] = -INFINITY;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) {
      mn[k] = std::min(mn[k], xyz[3 * i + k]);
      mx[k] = std::max(mx[k], xyz[3 * i + k]);
    }
  for (int k = 0; k < 3; ++k) ext[k] = mx[k] - mn[k];
  std::vector<Worker> W;
  W.reserve(threads);
  for (int w = 0; w < threads; ++w) W.emplace_back(M);
  for (auto& X : W) X.last = 0;
  ParStats ps;
  int pass = 0;
  // BRIO rounds: the first by one thread, the others with the thread scheme
  size_t q = 0;
  int rc = ORACLE_OK;
  while (q < seq.size() && rc == ORACLE_OK) {
    const uint8_t r = rounds[seq[q]];
    std::vector<uint32_t> todo;
    for (; q < seq.size() && rounds[seq[q]] == r; ++q) {
      if (q == 0 || q == 1 || q == k2 || q == k3) continue;
      todo.push_back(seq[q]);
    }
    rc = insert_parallel(M, W, std::move(todo), r == 0 ? 1 : threads, min_per_thread, mn, ext, seed, &pass, ps);
  }
  if (rc != ORACLE_OK) return rc;
  // output: the finite live tetrahedra, canonical and sorted (threads over slot ranges)
  const uint64_t used = std::min<uint64_t>(M.bump.load(), M.cap);
  std::vector<std::vector<std::array<uint32_t, 4>>> part(threads);
  {
    std::vector<std::thread> th;
    auto collect = [&](int w) {
      for (uint64_t s = used * w / threads; s < used * (w + 1) / threads; ++s) {
        if (!M.alive[s].load(std::memory_order_relaxed)) continue;
        uint32_t v[4];
        M.getv((uint32_t)s, v);
        if (gpos4(v) >= 0) continue;
        canonical(v);
        part[w].push_back({v[0], v[1], v[2], v[3]});
      }
    };
    for (int w = 1; w < threads; ++w) th.emplace_back(collect, w);
    collect(0);
    for (auto& x : th) x.join();
  }
  std::vector<std::array<uint32_t, 4>> tets;
  for (auto& v : part) tets.insert(tets.end(), v.begin(), v.end());
  parallel_sort(tets, threads, [](const std::array<uint32_t, 4>& a, const std::array<uint32_t, 4>& b) { return a < b; });
  if (stats) {
    int64_t walk = 0, cav = 0, ball = 0;
    for (auto& X : W) walk += X.walk, cav += X.cav, ball += X.ball;
    stats[0] = (int64_t)seq.size();
    stats[1] = (int64_t)tets.size();
    stats[2] = ps.passes;
    stats[3] = ps.aborted;
    stats[4] = ps.sequential_passes;
    stats[5] = ps.max_threads;
    stats[6] = cav;
    stats[7] = ball;
    stats[8] = walk;
  }
  if ((int64_t)tets.size() > cap) return ORACLE_ETOOSMALL;
  for (size_t t = 0; t < tets.size(); ++t)
    for (int k = 0; k < 4; ++k) out[4 * t + k] = tets[t][k];
  return (int64_t)tets.size();
}

}  // namespace

extern "C" {

// The paper's parallel insertion with up to `threads` threads, halving while a thread would get
// fewer than min_per_thread points (3000 in the paper). Output as oracle_delaunay (the canonical
// sorted finite tetrahedra). stats (may be NULL), 9 entries: unique points, tetrahedra, passes,
// aborted insertions, one-thread passes, most threads used, summed cavity and ball sizes, walk
// steps.
int64_t paper_cpu_delaunay(const double* xyz, int64_t n, uint64_t seed, int threads, int64_t min_per_thread,
                           uint32_t* tets_out, int64_t cap, int64_t* stats) {
  try {
    return delaunay_parallel(xyz, n, seed, threads, min_per_thread, tets_out, cap, stats);
  } catch (const std::bad_alloc&) {
    return ORACLE_EINTERNAL;
  } catch (const std::system_error&) {
    return ORACLE_EINTERNAL;
  }
}

}  // extern "C"
