/* dt.h — C ABI of the GB300 (sm_103a) concurrent 3D Delaunay kernel.
 *
 * The library builds DT(S), the Delaunay triangulation of a 3D point set S, by incremental
 * Bowyer–Watson insertion as defined in Section 2.1, Eq. (1) of Marot, Pellerin, Remacle,
 * "One machine, one minute, three billion tetrahedra": DT_{k+1} = DT_k - C(DT_k, p) + B(DT_k, p),
 * where the cavity C holds every tetrahedron whose circumsphere contains p and the ball B fills
 * the hole with tetrahedra joining p to the cavity boundary. Many points are inserted
 * concurrently per round; a point whose cavity overlaps another's (the conflict rules of
 * Section 3.2) retries in a later round. Because the predicates are exact and degeneracies
 * are resolved by one symbolic perturbation that depends only on point identity, the result is
 * the unique perturbed Delaunay triangulation, independent of the schedule.
 *
 * Conventions used throughout:
 *  - points are float64 triples, row-major [n, 3]; coordinates must be finite;
 *  - vertex ids in outputs are 0-based input indices (global across successive dt_insert calls
 *    on one handle, local to the cloud in dt_batch);
 *  - output tetrahedra are finite (ghost tetrahedra of Section 2.6 are dropped) and positively
 *    oriented, det[b-a; c-a; d-a] > 0; the canonical form rotates each by an even permutation
 *    so the smallest id is first and the other three start at their smallest, and sorts the
 *    list lexicographically;
 *  - exact duplicate points keep the smallest input index; the others are not inserted and are
 *    counted in dt_stats.n_dups;
 *  - "device" pointers are CUDA global-memory pointers of the current device; "host" pointers
 *    are ordinary (preferably pinned) host memory. The caller owns every buffer it passes;
 *    the library reads inputs during the call (stream-ordered) and copies what it keeps;
 *  - every function returns DT_OK (0) or a negative DT_E* code, never traps or aborts; device
 *    loops are bounded and report DT_ELIMIT instead of hanging;
 *  - a handle is not thread-safe: one host thread at a time.
 */
#ifndef DT_GB300_H
#define DT_GB300_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DT_OK 0
#define DT_EINVAL (-1)      /* bad argument (null pointer, non-finite coordinate, bad sizes) */
#define DT_ENOMEM (-2)      /* device allocation failed or tetrahedron capacity exhausted */
#define DT_ETOOSMALL (-3)   /* output capacity too small; *n_tets holds the required count */
#define DT_EDEGENERATE (-4) /* fewer than four non-coplanar points */
#define DT_ELIMIT (-5)      /* a device-side bound tripped (walk, cavity, rounds, exact workspace) */
#define DT_ECUDA (-6)       /* a CUDA runtime call failed */
#define DT_ESTATE (-7)      /* call not valid in the handle's current state */

#define DT_SCHED_PLAIN 0    /* Moore segments + rescaling/shift re-partition (Section 3.3) */
#define DT_SCHED_LEARNED 1  /* claim ranks from the learned cavity-size model (a loaded model is
                               required, dt_load_model); the same tetrahedra as the plain schedule */

#define DT_FLAG_NO_CANONICAL_SORT 1u /* dt_get_tets(canonical=1) rotates but does not sort */
#define DT_FLAG_PROFILE 2u           /* time each launch of the round kernels with CUDA events */
#define DT_FLAG_LOG 4u               /* log per point: cavity size of its insertion, conflicts lost
                                        (the learned scheduler's training labels, dt_get_features) */

#define DT_MLP_PARAMS 1410u          /* parameters of the learned scheduler's network */
#define DT_FEATURES 8u               /* inputs per point */

typedef struct {
  double tet_capacity_factor; /* tetrahedron slots reserved per point; 0 = 8.0 */
  uint64_t seed;              /* BRIO hash and re-partition randomness */
  void* stream;               /* cudaStream_t to run on; NULL = the default stream */
  uint32_t schedule;          /* DT_SCHED_PLAIN or DT_SCHED_LEARNED */
  uint32_t max_walk_steps;    /* per walk attempt (a longer walk resumes next pass); 0 = 48 */
  uint32_t max_rounds;        /* insertion rounds per call before DT_ELIMIT; 0 = 1 << 22 */
  uint32_t segments;          /* concurrent insertions per round; 0 = chosen per round */
  uint32_t flags;             /* DT_FLAG_* */
  uint32_t reserved[5];       /* must be zero */
} dt_config;

typedef struct {
  uint64_t n_points;      /* points given to the handle so far */
  uint64_t n_unique;      /* points inserted (duplicates excluded) */
  uint64_t n_dups;        /* exact duplicates not inserted */
  uint64_t n_tets;        /* finite tetrahedra in the current triangulation */
  uint64_t n_slots;       /* tetrahedron slots in use (finite + ghost + free) */
  uint64_t n_rounds;      /* concurrent insertion rounds launched */
  uint64_t n_passes;      /* re-partition passes (Section 3.3) */
  uint64_t n_attempts;    /* insertion attempts (successes + retries) */
  uint64_t n_conflicts;   /* attempts lost to a higher-priority cavity */
  uint64_t n_big;         /* cavities too large for the shared-memory path */
  uint64_t sum_cavity;    /* sum of |C| over successful insertions */
  uint64_t sum_ball;      /* sum of |B| over successful insertions */
  uint64_t sum_walk;      /* sum of walk steps over all attempts */
  uint64_t n_exact;       /* predicate evaluations that needed exact arithmetic */
  uint64_t n_sos;         /* insphere evaluations decided by the perturbation */
  double ms_sort;         /* device time of keys + sort + dedup (last call) */
  double ms_insert;       /* device time of the insertion rounds (last call) */
  uint64_t n_launches;    /* kernels launched by the handle so far */
  double ms_walk, ms_cavity, ms_insert_k; /* summed launch times of the three round kernels
                                             (DT_FLAG_PROFILE only) */
  uint64_t n_profiled;    /* launches of each round kernel that were timed */
  uint64_t device_error;  /* first device-side error code of the last failing call (0 = none) */
  uint64_t device_error_info;
  uint64_t n_rounds_wave;  /* rounds of the waves of BRIO rounds */
  uint64_t n_rounds_retry; /* rounds of the retry passes */
  uint64_t n_rounds_big;   /* large-cavity rounds */
  double ms_first_round;   /* device time of the one-block engine (first BRIO round, last call) */
  uint64_t n_walk_limit;   /* walks stopped at max_walk_steps (each resumes in a later pass) */
  uint64_t free_slots;     /* slots on the free list after the last round */
  uint64_t max_walk;       /* longest single walk (steps) */
  uint64_t n_clouds_degenerate; /* dt_batch: clouds with fewer than four non-coplanar points */
  uint64_t batch_warps;    /* dt_batch: block shape used (warps per block, autotuned) */
  double batch_alpha;      /* dt_batch: concurrent insertions per mesh vertex used (autotuned) */
  double ms_batch_tune;    /* dt_batch: host time of the autotuning in the last call (0 = reused) */
  uint64_t batch_graph;    /* dt_batch: 1 if the last call replayed its captured CUDA graph */
  uint64_t batch_min_blocks; /* dt_batch: resident blocks per SM the chosen shape was built for */
  double ms_async;         /* summed device time of the asynchronous insertion launches
                              (DT_FLAG_PROFILE only) */
  uint64_t n_async;        /* asynchronous insertion launches (one per wave or retry pass) */
  uint64_t n_restarts;     /* asynchronous insertions that found their cavity changed under the
                              locks and started over */
  uint64_t device_bytes;   /* device memory the handle holds */
  uint64_t n_exact_handoff; /* points the asynchronous engine handed to the round-based engine
                               because its FP32 predicate stage could not decide a test */
  uint64_t n_inserted_async; /* insertions made by the asynchronous engine */
  uint64_t reserved[2];
} dt_stats;

typedef struct dt_handle dt_handle;

/* Creates an empty triangulation on the current CUDA device. cfg may be NULL (defaults).
 * *out receives the handle; release it with dt_destroy. */
int dt_create(dt_handle** out, const dt_config* cfg);

/* Inserts n points (device pointer, [n, 3] float64 row-major) into the handle's triangulation:
 * Moore keys of the 21-bit quantised coordinates (Section 2.3), BRIO rounds (Table 2 sizes),
 * radix sort by (round, key, index), then concurrent insertion rounds (Algorithm 1 per point,
 * Section 3 conflict rules). The first call needs at least four non-coplanar points
 * (DT_EDEGENERATE otherwise). Later calls extend the same triangulation; the result equals one
 * call with all points. Input indices of this call start at the number of points given before.
 * Stream-ordered on cfg->stream; returns after the triangulation is complete. */
int dt_insert(dt_handle* h, const double* xyz_dev, uint64_t n);

/* Same as dt_insert, with host input: the points are copied to the device inside the call, into
 * a device buffer the handle keeps for later calls (n * 24 bytes, freed by dt_destroy; counted
 * in dt_stats.device_bytes). Page-locked host memory makes the copy fastest. */
int dt_insert_host(dt_handle* h, const double* xyz_host, uint64_t n);

/* Triangulates n_clouds independent clouds: one batched sort (each cloud gets its own box,
 * Moore keys, duplicates and BRIO rounds, exactly as dt_insert would give it alone), then ONE
 * persistent kernel launch in which every thread block takes whole clouds from a device work
 * counter (largest first) and runs Algorithm 1 for all of a cloud's points with its warps
 * inserting concurrently (the Section 3.2 conflict rules between them). The block shape (warps
 * per block) and the round size are chosen by an autotuner that times candidates on a sample of
 * the clouds the first time a batch of this kind (cloud count, size range) is seen.
 *  - xyz_dev: the clouds back to back, [sum n_i, 3] float64 (device);
 *  - offsets_host: n_clouds + 1 ascending entries (host), offsets_host[0] = 0; cloud c is rows
 *    offsets_host[c] .. offsets_host[c + 1].
 * Replaces the handle's content (dt_insert returns DT_ESTATE until dt_clear). A cloud with fewer
 * than four non-coplanar points gets no tetrahedra and is counted in n_clouds_degenerate; the
 * call returns DT_EDEGENERATE only if every cloud is so. Vertex ids in dt_get_tets are local to
 * each cloud. Each cloud's tetrahedra are those of dt_insert on that cloud alone. */
int dt_batch(dt_handle* h, const double* xyz_dev, const uint64_t* offsets_host, uint32_t n_clouds);

/* Delaunay refinement of the current triangulation inside an axis-aligned box (Section 4,
 * Algorithm 2: SamplePoints, FilterPoints, InsertPoints, repeated). The box should be the hull
 * of the points already inserted (for instance their 8 corners are among them): boundary
 * recovery is not part of this call. One iteration:
 *  - sample: each finite tetrahedron with circumradius r, r^2 > (ratio * size)^2, gives a
 *    candidate at its circumcentre when that lies strictly inside the box. The circumcentre of
 *    the tetrahedron a, b, c, d (vertices in increasing input index) is computed in float64 with
 *    every operation rounded on its own: u = b - a, v = c - a, w = d - a,
 *    o = ((|u|^2 (v x w) + |v|^2 (w x u)) + |w|^2 (u x v)) / (2 u . (v x w)), centre = a + o,
 *    r^2 = o . o, each dot product summed as (x + y) + z;
 *  - filter: a candidate at squared distance < (spacing * size)^2 from an existing point is
 *    dropped; of the rest, one at squared distance < (spacing * size)^2 from a remaining
 *    candidate of higher priority (larger r^2, then the lexicographically smaller sorted tuple
 *    of its tetrahedron's input indices) is dropped;
 *  - insert: the survivors, in increasing order of those tuples, are inserted as by dt_insert
 *    (their input indices follow the last point given before).
 * The paper's values are ratio = 1.4 and spacing = 0.7. Stops after an iteration with no
 * survivor or after max_iters iterations that inserted points. *n_added (may be NULL) receives
 * the points added, *n_iters (may be NULL) the iterations that inserted points.
 *  - box_host: 6 float64 (host): lo x, y, z, hi x, y, z, lo < hi on every axis.
 * DT_EINVAL for a non-positive or non-finite size, ratio or spacing, a bad box, or a box wider
 * than 2^21 filter cells (spacing * size) per axis; DT_ESTATE without a triangulation or after
 * dt_batch. Insertion errors are returned as by dt_insert, with the counts reached so far.
 * An iteration that adds at least a quarter as many points as the mesh holds rebuilds the mesh
 * from all its points (same input indices, so the same triangulation); after an error in that
 * step the handle holds the part of the rebuild that was reached, as after a failed dt_insert. */
int dt_refine(dt_handle* h, double size, double ratio, double spacing, const double* box_host, uint32_t max_iters,
              uint64_t* n_added, uint32_t* n_iters);

/* Coordinates of every point given to the handle (dt_insert calls and dt_refine), by input
 * index: row i of xyz_dev ([rows, 3] float64, device) receives point i when i < rows. *n_points
 * (may be NULL) receives the number of points; rows = 0 only queries it. DT_ESTATE after
 * dt_batch. */
int dt_get_points(dt_handle* h, double* xyz_dev, uint64_t rows, uint64_t* n_points);

/* Copies the finite tetrahedra of the current triangulation into tets_dev ([cap, 4] uint32,
 * device memory, or page-locked host memory that the kernels write through its mapped device
 * address; pageable host memory gives DT_EINVAL). canonical != 0 rotates and sorts them (see
 * conventions); 0 writes them positively
 * oriented in an unspecified order. *n_tets receives the count; DT_ETOOSMALL if cap < count.
 * After dt_batch, cloud_offsets (host, n_clouds + 1 entries, may be NULL) receives where each
 * cloud's tetrahedra start; each cloud's block is canonical on its own. */
int dt_get_tets(dt_handle* h, uint32_t* tets_dev, uint64_t cap, uint64_t* n_tets,
                uint64_t* cloud_offsets, int canonical);

/* Certificate of the current triangulation, checked on the device at any size. A closed,
 * consistently oriented complex of tetrahedra (the ghost ones included) whose every facet is
 * locally Delaunay is the Delaunay triangulation of its vertices (the Delaunay lemma; Section
 * 2.1's empty-sphere property follows). With the insertion predicates' perturbation (Section 2.4)
 * that triangulation is unique, so a certificate without faults identifies it. out_host (host,
 * 5 entries) receives:
 *   [0] live finite tetrahedra (the count dt_get_tets returns),
 *   [1] (tetrahedron, facet) pairs whose neighbour is dead, or does not name the tetrahedron
 *       back, or does not share the facet's three vertices,
 *   [2] finite tetrahedra whose orientation is not positive (exact),
 *   [3] facets whose neighbour's opposite vertex is in conflict with the tetrahedron (exact
 *       perturbed insphere; for a ghost, the hull facet's side and Section 2.6's rule),
 *   [4] distinct points that are vertices of finite tetrahedra (the points given minus the
 *       duplicates dropped).
 * A Delaunay triangulation gives [1] = [2] = [3] = 0. The handle's statistics do not change.
 * DT_ESTATE after dt_batch; DT_ENOMEM if the scratch (n_points bytes) cannot be allocated. */
int dt_check(dt_handle* h, uint64_t* out_host);

/* Host variant of dt_get_tets: tets_host is host memory ([cap, 4] uint32). Without the
 * canonical sort, page-locked memory (cudaHostAlloc, cudaHostRegister) receives the rows
 * straight from the collecting kernel through its mapped device address. Otherwise the
 * tetrahedra are collected once into a device buffer the handle keeps (cap * 16 bytes, freed by
 * dt_destroy; counted in dt_stats.device_bytes) and copied out in one transfer. cap = 0 only
 * counts. DT_ETOOSMALL (with *n_tets the count) if cap is too small. */
int dt_get_tets_host(dt_handle* h, uint32_t* tets_host, uint64_t cap, uint64_t* n_tets, int canonical);

/* The sort of the last dt_insert call (Section 2.3): keys_dev[i] = 63-bit Moore key of input
 * point i, perm_dev[s] = input index of the s-th point in (round, key, index) order, and
 * rounds_dev[i] = BRIO round of point i. Any pointer may be NULL. Indices are call-local. */
int dt_get_order(dt_handle* h, uint64_t* keys_dev, uint32_t* perm_dev, uint8_t* rounds_dev);

/* Counters of the handle (see dt_stats). */
int dt_get_stats(dt_handle* h, dt_stats* out);

/* Loads the learned scheduler's parameters (float32, host): W1[8x32], b1[32], W2[32x32], b2[32],
 * W3[32x2], b3[2] row-major in that order (W[i][j]: input i -> output j), n_params = 1410.
 * Used by dt_insert when cfg.schedule = DT_SCHED_LEARNED (DT_ESTATE if none is loaded). The
 * network maps a point's features (dt_get_features) to out[0] = predicted log2(1 + |C|) and
 * out[1] = the logit of the probability that the point loses a conflict; points predicted to
 * have small cavities claim with a higher priority than points expected to have large ones
 * (conflicts are settled by any strict total order of the points, Section 3.2; a large cavity
 * that wins knocks out every small one it overlaps, so fewer attempts are lost). The tetrahedra
 * do not depend on the schedule. */
int dt_load_model(dt_handle* h, const float* params_host, uint32_t n_params);

/* Per-point features and labels of the last dt_insert call, in insertion order (the order of
 * dt_get_order's perm): x_dev [n, 8] float32 (device) = log2-scaled point count of the point's
 * cell of a ~4-points-per-cell grid, the mean / spread of its 6 face neighbours' counts, the
 * density contrast, two 6-bit fields of the Moore key, the BRIO round / 8 and the distance to
 * the box boundary (fraction of the half-extent). With DT_FLAG_LOG, y_dev [n, 2] receives the
 * labels (log2(1 + |C|) of the point's insertion, 1 if it lost a conflict first) and valid_dev
 * [n] (uint8) 1 where the point was inserted by a concurrent round (0: init, duplicate, or the
 * label is missing). y_dev and valid_dev may be NULL. n must equal the call's point count. */
int dt_get_features(dt_handle* h, float* x_dev, float* y_dev, uint8_t* valid_dev, uint64_t n);

/* The network on n feature rows (device): out_dev [n, 2] float32. */
int dt_mlp_forward(const float* params_dev, const float* x_dev, uint64_t n, float* out_dev, void* stream);

/* Mean loss over n samples, (out0 - y0)^2 + softplus(out1) - y1 * out1, into *loss_dev, and its
 * gradient with respect to the 1410 parameters into grad_dev (all device, float32). */
int dt_mlp_grad(const float* params_dev, const float* x_dev, const float* y_dev, uint64_t n, float* grad_dev,
                float* loss_dev, void* stream);

/* Trains params_dev in place on the GPU: `steps` Adam steps (learning rate lr) on minibatches of
 * `batch` samples drawn from the n rows by a counter-based hash of (seed, step). losses_host
 * (may be NULL) receives each step's minibatch loss. */
int dt_mlp_train(float* params_dev, const float* x_dev, const float* y_dev, uint64_t n, uint32_t steps,
                 uint32_t batch, float lr, uint64_t seed, float* losses_host, void* stream);

/* Forgets the triangulation and the points but keeps the device memory, so the next dt_insert
 * starts a new triangulation without allocating (used between repeated runs). */
int dt_clear(dt_handle* h);

/* Releases the handle and all its device memory. NULL is a no-op. */
void dt_destroy(dt_handle* h);

/* Static description of an error code. */
const char* dt_strerror(int code);

/* Largest point count dt_order_noalloc accepts. */
#define DT_NOALLOC_MAX_POINTS 262144u

/* The spatial order of dt_get_order (Moore keys, BRIO rounds, insertion permutation) computed
 * without allocating any device memory. The paper has no counterpart; this entry point exists
 * for callers that cannot call cudaMalloc: hosts whose device memory is all owned by another
 * allocator (a framework's caching pool or a fixed arena that may not be bypassed), and code
 * under a device-memory budget that a new allocation could break. The call synchronises its
 * stream before it returns (it reads back the coordinate check).
 *  - xyz_dev: [n, 3] float64 row-major (device); n <= DT_NOALLOC_MAX_POINTS, else DT_EINVAL.
 *  - keys_dev [n] uint64, perm_dev [n] uint32, rounds_dev [n] uint8: device outputs, owned by
 *    the caller; same values as dt_get_order after dt_insert of the same points and seed.
 *  - stream: cudaStream_t (NULL = default stream); the call returns after the stream is done.
 * The working memory is one file-scope device array of about 7.7 MB that every device loading
 * the library holds until the process exits. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture begins. All calls share the array and each leaves its contents
 * behind (the parts that must start at zero are cleared at the start of every call): calls
 * that overlap on the GPU, from several host threads or streams, race and must be serialised
 * by the caller. The looked-up address is kept for the life of the process: do not use this
 * entry point after cudaDeviceReset on that device. Errors: DT_EINVAL (bad pointer, size over the limit, non-finite or
 * |x| > 1e30 coordinate), DT_ECUDA. */
int dt_order_noalloc(const double* xyz_dev, uint64_t n, uint64_t seed, uint64_t* keys_dev, uint32_t* perm_dev,
                     uint8_t* rounds_dev, void* stream);

/* Exact predicate signs on the device, for testing the predicates in isolation (Section 2.4):
 * for each of n tuples, kind 0 = orient3d(a,b,c,d) (4 points), 1 = insphere(a,b,c,d,e) (5 points,
 * unperturbed), 2 = perturbed insphere with ids_dev giving the 5 point identities; kinds 3
 * (orient3d) and 4 (perturbed insphere) run the insertion kernels' full pipeline: the FP32
 * stage on a double-float copy of the points, then the FP64 filter, then exact arithmetic.
 * pts_dev: [n, 5, 3] float64 (unused slots ignored); ids_dev: [n, 5] int64 (kind 2 only, else
 * NULL); out_dev: [n] int8 signs. */
int dt_eval_predicates(int kind, const double* pts_dev, const int64_t* ids_dev, int8_t* out_dev,
                       uint64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif
