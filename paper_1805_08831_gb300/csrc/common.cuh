// Shared device types of the GB300 Delaunay library.
//
// Tetrahedron store (Section 2.2, adapted for coalesced 32-byte sectors): one record of
//   v[4]  vertex ids (vertex id = position in the insertion order; kGhost for the ghost vertex)
//   n[4]  neighbour slots (facet i is opposite vertex i, Fig. 2): n[i] is the tetrahedron
//         across facet i. Which of its facets faces back is not stored: it is the one whose
//         neighbour is this tetrahedron (two tetrahedra share at most one facet), so ids use
//         all 32 bits and a mesh may hold up to kMaxSlots records.
// Both halves of a record share one 32-byte DRAM sector, so a cavity test reads one sector.
// A dead slot has v.x == v.y (a live tetrahedron never repeats a vertex) and keeps in n.x the
// id of a tetrahedron created when it died (a redirect for stale walk hints).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dtg {

constexpr uint32_t kGhost = 0xFFFFFFFFu;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kDeadMark = 0xFFFFFFFEu;
// Largest number of tetrahedron slots of one mesh: below the two markers above, with room for a
// grid-stride loop over the slots to step past the end without wrapping 32 bits.
constexpr uint64_t kMaxSlots = 0xF0000000ull;

// A vertex: coordinates and, in .w, its input index (the order of the perturbation).
struct __align__(32) Pt {
  double x, y, z, w;
};

__host__ __device__ __forceinline__ Pt make_pt(double x, double y, double z, double w) {
  Pt p;
  p.x = x;
  p.y = y;
  p.z = z;
  p.w = w;
  return p;
}

struct __align__(16) Tet {
  uint4 v;
  uint4 n;
};

// Device error codes (mapped to DT_E* on the host).
enum DevError : unsigned int {
  kErrNone = 0,
  kErrCapacity = 1,   // tetrahedron store full
  kErrFreeList = 2,   // free-list array full
  kErrExactRange = 3, // exact arithmetic left its exact range (underflow/overflow) or workspace
  kErrInternal = 4,   // inconsistent topology (never expected)
  kErrBigCavity = 5,  // cavity exceeds even the large-cavity workspace
  kErrDegenerate = 6, // no initial tetrahedron
  kErrWalk = 7,       // walk could not find a live start tetrahedron
};

// Counters and per-round allocator state, one instance in device memory per handle.
struct DevState {
  unsigned long long stamp;          // round stamp: upper 32 bits of claim priorities
  unsigned long long bump;           // first never-used tetrahedron slot
  unsigned long long capacity;       // tetrahedron slots allocated
  unsigned long long free_avail;     // free-list entries usable this round
  unsigned long long alloc_cursor;   // virtual allocation cursor of this round
  unsigned long long pending;        // slots freed this round (appended after the round)
  unsigned long long free_capacity;  // size of the free-list array
  unsigned long long q[6];           // queue lengths: 0 next pass, 1 large cavities,
                                     // 2 large-cavity retries, 3 serial path,
                                     // 4 cavities too large for the shared-memory large rounds,
                                     // 5 points the asynchronous engine hands to the rounds
  unsigned int blocks_done;          // blocks of the insert kernel that finished this round
  unsigned int pad1;
  unsigned int error;                // first DevError raised
  unsigned int error_info;
  unsigned int anchor;               // a tetrahedron known to be live
  unsigned int pad0;
  // statistics
  unsigned long long n_inserted, n_conflicts, n_attempts, n_walk_limit, n_big, n_dups;
  unsigned long long sum_cavity, sum_ball, sum_walk, n_exact, n_sos, max_walk;
  unsigned long long n_restart;  // asynchronous insertions restarted after a failed re-read
  unsigned long long n_inserted_async;  // insertions made by the asynchronous engine
};

__device__ __forceinline__ void raise_error(DevState* st, unsigned int code, unsigned int info) {
  if (atomicCAS(&st->error, 0u, code) == 0u) st->error_info = info;
}

__device__ __forceinline__ bool tet_dead(const uint4& v) { return v.x == v.y; }

__device__ __forceinline__ int ghost_pos(const uint4& v) {
  return v.x == kGhost ? 0 : v.y == kGhost ? 1 : v.z == kGhost ? 2 : v.w == kGhost ? 3 : -1;
}

__device__ __forceinline__ uint32_t get4(const uint4& a, int i) {
  return i == 0 ? a.x : i == 1 ? a.y : i == 2 ? a.z : a.w;
}

__device__ __forceinline__ void set4(uint4& a, int i, uint32_t x) {
  if (i == 0) a.x = x;
  else if (i == 1) a.y = x;
  else if (i == 2) a.z = x;
  else a.w = x;
}

// The facet of a tetrahedron (neighbour ids n) whose neighbour is t, or -1.
__device__ __forceinline__ int back_facet(const uint4& n, uint32_t t) {
  return n.x == t ? 0 : n.y == t ? 1 : n.z == t ? 2 : n.w == t ? 3 : -1;
}

__device__ __forceinline__ Tet load_tet(const Tet* T, uint32_t t) {
  Tet r;
  const uint4* p = reinterpret_cast<const uint4*>(T + t);
  r.v = __ldg(p);
  r.n = __ldg(p + 1);
  return r;
}

// Coherent (L2) load of a record that other blocks of the same kernel may write.
__device__ __forceinline__ Tet load_tet_cg(const Tet* T, uint32_t t) {
  Tet r;
  const uint4* p = reinterpret_cast<const uint4*>(T + t);
  r.v = __ldcg(p);
  r.n = __ldcg(p + 1);
  return r;
}

__device__ __forceinline__ Pt load_pt(const Pt* P, uint32_t v) {
  const double2* q = reinterpret_cast<const double2*>(P + v);
  double2 a = __ldg(q), b = __ldg(q + 1);
  return make_pt(a.x, a.y, b.x, b.y);
}

}  // namespace dtg
