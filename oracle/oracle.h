/* Serial CPU oracle for the 3D Delaunay kernel of Marot, Pellerin, Remacle,
 * "One machine, one minute, three billion tetrahedra" (arXiv 1805.08831).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The GPU library never links or calls it and the
 * two share no source, header, table or helper.
 *
 * Every routine is a plain, slow, serial restatement of the paper (section / equation /
 * algorithm cited next to each declaration). Predicates are exact: a loose double-precision
 * filter, then big-integer evaluation on the dyadic values of the doubles.
 *
 * Conventions (shared with the GPU library only through this written specification):
 *  - a tetrahedron (a,b,c,d) is positive iff det[b-a; c-a; d-a] > 0;
 *  - for a positive tetrahedron, e is inside its circumsphere iff the 4x4 determinant of
 *    Section 2.4 (rows q-a, |q-a|^2 for q = b,c,d,e) is negative;
 *  - degenerate insphere tests are decided by perturbing the lifted coordinate |p|^2 of each
 *    point by eps^k with k decreasing in the input index (the point with the largest input
 *    index carries the dominant perturbation);
 *  - exact duplicates keep the smallest input index; the others are not inserted;
 *  - output tetrahedra are finite, positively oriented, rotated by an even permutation so that
 *    the smallest id comes first and the remaining three start at their smallest, and the list
 *    is sorted lexicographically.
 */
#ifndef DT_ORACLE_H
#define DT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_EDEGENERATE (-2)
#define ORACLE_ETOOSMALL (-3)
#define ORACLE_EINTERNAL (-4)

typedef struct {
  int64_t n_points;        /* input points */
  int64_t n_unique;        /* points after exact-duplicate removal */
  int64_t n_dups;          /* duplicates dropped */
  int64_t n_tets;          /* finite tetrahedra in the result */
  int64_t n_ghosts;        /* ghost tetrahedra = convex-hull facets */
  int64_t n_hull_vertices; /* distinct vertices of hull facets */
  int64_t sum_cavity;      /* sum over insertions of |C| (deleted tetrahedra, ghosts included) */
  int64_t sum_ball;        /* sum over insertions of |B| (created tetrahedra) */
  int64_t sum_walk;        /* sum over insertions of walk steps */
  int64_t n_insphere;      /* insphere evaluations */
  int64_t n_exact;         /* predicate evaluations that needed big integers */
  int64_t n_sos;           /* insphere evaluations decided by the perturbation */
  int64_t validate_flags;  /* 0 = every requested check passed; bit set = failed check */
} oracle_stats;

/* Validation bits (oracle_delaunay with validate != 0). */
#define ORACLE_BAD_ORIENT 1       /* a finite tetrahedron is not positive */
#define ORACLE_BAD_ADJACENCY 2    /* nbr[nbr[s]] != s or the shared facet differs */
#define ORACLE_BAD_DELAUNAY 4     /* an interior facet is not locally Delaunay (perturbed) */
#define ORACLE_BAD_GHOST 8        /* a ghost is mis-oriented or not on a hull facet */
#define ORACLE_BAD_HULLCOUNT 16   /* ghosts != 2 * hull vertices - 4 */

/* S1+S2, Section 2.3: per-axis bounding box, 21-bit quantisation
 * q = floor((x - min) * (2^21 / (max - min))) clamped to [0, 2^21 - 1], then the 63-bit Moore
 * index of cell q (closed Hilbert curve, Hamilton's construction). */
int oracle_moore_keys(const double* xyz, int64_t n, uint64_t* keys);

/* Moore index of explicit integer cells q (n x 3, each < 2^m) on an m-level curve. */
int oracle_moore_index(const uint32_t* q, int64_t n, int m, uint64_t* keys);

/* S3, Section 2.3 and Table 2: BRIO round of each input index. Points are ranked by
 * splitmix64(seed ^ index); round r holds ranks [2048*7^(r-1), 2048*7^r), round 0 the first
 * 2048, and the last round all the remaining ranks. */
int oracle_brio_rounds(int64_t n, uint64_t seed, uint8_t* rounds);

/* S4, Section 2.3: insertion order = input indices sorted by (round, Moore key, index). */
int oracle_insertion_order(const double* xyz, int64_t n, uint64_t seed, uint32_t* perm);

/* Exact duplicates: rep[i] = smallest input index with the same coordinates as i. */
int oracle_dedup(const double* xyz, int64_t n, uint32_t* rep);

/* Exact predicate signs (Section 2.4). pts = consecutive xyz triples. */
int oracle_orient3d(const double* pts12);
int oracle_insphere(const double* pts15);
int oracle_insphere_sos(const double* pts15, const int64_t* ids5);
/* Exact value of the 4x4 insphere determinant, rounded to double. */
double oracle_insphere_value(const double* pts15);
/* Exact value of det[b-a; c-a; d-a], rounded to double. */
double oracle_orient3d_value(const double* pts12);

/* Algorithm 1 with ghost tetrahedra (Section 2.6): serial Bowyer-Watson insertion. Points are
 * inserted in the S4 order (or in `order`, a permutation of 0..n-1, when not NULL) after
 * removing exact duplicates. Writes the canonical sorted list of finite tetrahedra (input
 * indices) and returns its length, or a negative ORACLE_E* code. With cap too small returns
 * ORACLE_ETOOSMALL and stats->n_tets holds the required count. */
int64_t oracle_delaunay(const double* xyz, int64_t n, uint64_t seed, const int64_t* order,
                        uint32_t* tets_out, int64_t cap, int validate, oracle_stats* stats);

/* Definition of DT (Section 2): every non-flat 4-subset whose perturbed circumsphere holds no
 * other point. O(n^5); for n <= 40. Canonical sorted output, duplicates removed first. */
int64_t oracle_brute_force(const double* xyz, int64_t n, uint32_t* tets_out, int64_t cap);

/* Adjacency encoding of Section 2.2 (Fig. 2): nbr[4t+i] = 4u+j when facet i of t (opposite its
 * vertex i) is facet j of u; 0xFFFFFFFF on unmatched facets. */
int oracle_adjacency(const uint32_t* tets, int64_t T, uint32_t* nbr);

/* Plants a known mistake (k > 0) for the tests that show the pins catch it; 0 = none. */
void oracle_set_mutation(int k);

#ifdef __cplusplus
}
#endif
#endif
