/*
 * mf.h -- C ABI of the GB300 manifold-tracing and certification library
 * (libmf.so).  A from-scratch implementation of the hot path of
 * "Scaling Motion Planning Infeasibility Proofs" (Li & Dantam, arXiv 2406.04795):
 * tracing the zero set of a learned RBF decision function over the Coxeter
 * (Ã_d) triangulation in permutahedral representation (Sec. II-B, IV-A),
 * the crossing n-simplices (Sec. IV-C), and the forward-kinematics / capsule
 * collision check that certifies the traced points (Sec. V-C, App. A).
 *
 * Conventions for every entry point
 *  - Return value: MF_OK (0) or a negative MF_ERR_* code; mf_last_error(ctx)
 *    then holds a one-line message.  No entry point aborts the process.
 *  - Pointers documented "device" must point to memory of the context's
 *    device (cudaMalloc, torch CUDA tensors, ...); "host" pointers to host
 *    memory.  The caller owns every buffer it passes; the library never frees
 *    or keeps a caller pointer beyond the call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls enqueue their kernels on it and return after the counts
 *    they report are known (they synchronise that stream).
 *  - The context owns its resident device memory (hash tables, frontier and
 *    vertex lists, cell lists) inside the HBM budget given at creation.
 *  - Multi-dimensional arrays are row-major.  d is the configuration-space
 *    dimension, 2 <= d <= MF_MAXD.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MF_MAXD 8

#define MF_OK 0
#define MF_ERR_INVALID (-1)   /* bad argument: d out of range, lambda <= 0, NaN, NULL */
#define MF_ERR_DOMAIN (-2)    /* lattice keys of this domain / lambda do not fit 64 bits */
#define MF_ERR_OOM (-3)       /* the request does not fit the context's HBM budget */
#define MF_ERR_CAPACITY (-4)  /* an output buffer is too small; counts hold the sizes needed */
#define MF_ERR_MAXEDGES (-5)  /* traced set exceeded opts.max_edges; result is partial */
#define MF_ERR_TIMEOUT (-6)   /* a bounded device-side wait gave up */
#define MF_ERR_CUDA (-7)      /* a CUDA runtime call failed */
#define MF_ERR_DEVICE (-8)    /* a device-side check failed (hash probe limit, index) */

/* Arithmetic of the RBF evaluation.  The mixed paths re-evaluate in FP64 every
 * vertex whose sign their error bound cannot decide, so all three trace the
 * same set. */
#define MF_FP64 0        /* FP64 differences and exp */
#define MF_MIXED_BF16 1  /* distance GEMM on tcgen05 tensor cores (BF16 split, FP32
                            accumulate), FP32 exp, FP64 recheck of |f~| <= band */
#define MF_MIXED_FP32 2  /* FP32 SIMT distance and exp, FP64 recheck of |f~| <= band */

/* mf_trace_opts.flags */
#define MF_WANT_ROOTS 1u /* solve t and the intersection point of every traced edge */
#define MF_WANT_CELLS 2u /* crossing n-simplices and the cell -> edge CSR */
/* Root accuracy.  The FP64 path solves every root to |t - t*| <= 1e-9.  The
 * mixed paths solve to |t - t*| <= 1e-6 (their stated tolerance): FP32
 * iterations, then one FP64 Newton step that takes in FP64 the terms that can
 * exceed 1e-5 and sums the rest in FP32 under a bound that moves t by at most
 * 1e-7.  This flag gives a mixed path the FP64 path's 1e-9 root solve. */
#define MF_ROOTS_FP64_EXACT 4u
/* Sorted output (mf_trace and mf_trace_fetch; the batched, served and
 * allocation-free entry points reject it): edges in increasing order of their
 * 64-bit edge key (mf_vertex_keys(y) * 2^d + mask), cells in increasing order
 * of (vertex key of z, pi read as base-8 digits with pi_0 most significant),
 * and the cell -> edge CSR in the new orders (each row keeps its pairs in
 * vertex order).  Without it the order is the search's insertion order,
 * which depends on the scheduling of atomics. */
#define MF_SORT_OUTPUT 8u

typedef struct mf_ctx mf_ctx;

/* The learned manifold: f(q) = sum_i alpha_i exp(-gamma |q - s_i|^2) + b, the
 * decision function of an RBF-kernel SVM (Sec. IV-A; ThunderSVM, Sec. VI). */
typedef struct {
  int32_t d;
  int64_t n_sv;
  const double *sv;    /* device [n_sv][d] support vectors */
  const double *alpha; /* device [n_sv] signed dual weights */
  double gamma;        /* > 0 */
  double b;
} mf_rbf;

/* The traced region: the closed box [lo, hi]^d of C-space, and the lattice
 * offset o of the triangulation x = lambda * L * y + o (L = I - c 1 1^T,
 * c = (1 - 1/sqrt(d+1))/d, the Ã_d realisation of the Freudenthal-Kuhn
 * lattice).  An edge is traced only if both its vertices lie in the box. */
typedef struct {
  double lo[MF_MAXD], hi[MF_MAXD];
  double offset[MF_MAXD];
} mf_domain;

typedef struct {
  double lambda;           /* triangulation scale lambda_T (Sec. IV-A), > 0 */
  int64_t batch_cap_edges; /* frontier edges expanded per BFS chunk; 0 = 2^24 */
  int32_t precision;       /* MF_FP64 / MF_MIXED_BF16 / MF_MIXED_FP32 */
  double recheck_band;     /* mixed paths: vertices with |f~| <= max(bound, band)
                              are re-evaluated in FP64; 0 = 1e-3 */
  double root_tol;         /* root solve stops when |Newton step| <= root_tol; 0 = 1e-12 */
  int64_t max_edges;       /* capacity of the resident edge table; 0 = 2^24 */
  int64_t max_vertices;    /* capacity of the vertex table; 0 = max_edges */
  int64_t max_cells;       /* capacity of the cell list; 0 = 2 * max_edges */
  uint32_t flags;          /* MF_WANT_ROOTS | MF_WANT_CELLS */
} mf_trace_opts;

/* Results of mf_trace.  Array fields are caller-owned DEVICE buffers of the
 * given capacities (NULL with capacity 0 = not wanted).  If a capacity is too
 * small the call returns MF_ERR_CAPACITY after filling the counts; the result
 * stays in the context, and mf_trace_fetch copies it into larger buffers
 * without tracing again.  The order of edges and cells is unspecified (each
 * BFS level is contiguous); compare them as sets. */
typedef struct {
  int64_t cap_edges;
  int32_t *edge_y;        /* [cap_edges][d] first vertex y of each traced edge */
  uint32_t *edge_mask;    /* [cap_edges] first part p1 of the edge's ordered
                             partition (p1, p2), as a mask over {0..d-1}; the
                             second vertex is y + sum_{i in p1} e_i */
  double *edge_f;         /* [cap_edges][2] f at the two vertices */
  double *edge_t;         /* [cap_edges] root parameter t in [0,1] (MF_WANT_ROOTS) */
  double *points;         /* [cap_edges][d] intersection point x(y) + t (x(y') - x(y)) */
  int64_t cap_cells;
  int32_t *cell_y;        /* [cap_cells][d] vertex of each crossing n-simplex */
  uint8_t *cell_perm;     /* [cap_cells][d] order of its singleton parts before {d} */
  int64_t *cell_edge_off; /* [cap_cells + 1] CSR offsets into cell_edge_idx */
  int64_t cap_cell_edges;
  int64_t *cell_edge_idx; /* [cap_cell_edges] indices of the traced edges of each cell */
  /* counts written by the library */
  int64_t n_edges, n_cells, n_cell_edges;
  int64_t n_vertices;     /* distinct lattice vertices at which f was evaluated */
  int64_t n_near_zero;    /* of those, |f| < 1e-12 */
  int64_t n_recheck;      /* mixed paths: vertices re-evaluated in FP64 */
  int64_t n_boundary;     /* (traced edge, 2-coface) pairs whose new vertex lies outside the box */
  int64_t n_dead_seeds;   /* seeds whose n-simplex has no traced edge */
  int64_t levels;         /* BFS levels (level 0 = seed edges) */
  int64_t root_evals;     /* f evaluations spent by the root solve */
} mf_trace_out;

/* Serial arm for certification: frame T_{i+1} = T_i Rz(q_i + theta_i) Tz(d_i)
 * Tx(a_i) Rx(alpha_i), T_0 = identity; link i is the capsule between the
 * origins of T_i and T_{i+1} with radius radius[i].  The robot's elements are
 * its link capsules (elements 0 .. n_links-1, when radius is given) followed
 * by its spheres.  Spheres are the paper's robot model (Sec. VI: each link
 * as a set of spheres): sphere s rides on link sphere_link[s] (the body that
 * joint sphere_link[s] turns) with its centre given in that link's frame
 * T_{link+1}.  A zero-initialised tail (n_spheres = 0) means capsules only;
 * radius = NULL means spheres only. */
typedef struct {
  int32_t n_links;        /* == d of the points */
  const double *dh;       /* device [n_links][4]: theta_i, d_i, a_i, alpha_i */
  const double *radius;   /* device [n_links] capsule radii, or NULL: no capsules */
  int32_t n_spheres;      /* 0 .. MF_MAX_SPHERES */
  const int32_t *sphere_link;   /* device [n_spheres], in [0, n_links) */
  const double *sphere_center;  /* device [n_spheres][3], in frame T_{link+1} */
  const double *sphere_radius;  /* device [n_spheres] */
} mf_robot;
#define MF_MAX_SPHERES 64

#define MF_BOX 0
#define MF_SPHERE 1
#define MF_CYLINDER 2
typedef struct {
  int32_t n;
  const int32_t *type;    /* device [n]: MF_BOX / MF_SPHERE / MF_CYLINDER */
  const double *pose;     /* device [n][12]: rotation R (row-major, obstacle frame
                             -> world) followed by the translation t */
  const double *dims;     /* device [n][3]: box side lengths; sphere radius in [0];
                             cylinder radius in [0] and height in [1], centred on
                             the frame origin with the local z axis as its axis
                             (App. A, sphere vs cylinder) */
} mf_scene;

/* Creates a context on `device` whose resident allocations never exceed
 * hbm_budget_bytes (0 = 90% of free memory).  *out receives the context. */
int mf_ctx_create(int device, size_t hbm_budget_bytes, mf_ctx **out);
void mf_ctx_destroy(mf_ctx *ctx);
/* One-line description of the last error on this context ("" if none). */
const char *mf_last_error(mf_ctx *ctx);
/* Device bytes currently held by the context. */
size_t mf_ctx_bytes(mf_ctx *ctx);

/* Query type 1 (Sec. IV-A): the n-simplex of the Ã_d triangulation holding
 * each point.  points: device [n][d]; y_out: device [n][d] vertex; perm_out:
 * device [n][d] the singleton parts in walk order before {d}.  Ties among the
 * fractional lattice coordinates go to the lower index. */
int mf_locate(mf_ctx *ctx, int32_t d, double lambda, const double *offset_host,
              const double *points, int64_t n, int32_t *y_out, uint8_t *perm_out, void *stream);

/* The exact domain test the tracing kernels use, as a table (host only, no
 * GPU needed).  For s = sum(y) in [*smin, *smin + *span) and axis i, entries
 * tab[(s - *smin) * d * 2 + 2i] and [... + 1] are the lowest and highest y_i
 * whose coordinate x_i = lambda * (y_i - c s) + o_i (Ã_d map, rounded as the
 * kernels round it) lies in [lo_i, hi_i]; an empty range has low > high.  A
 * lattice vertex is in the box iff every y_i is in its range for s = sum(y).
 * tab may be NULL to query the size (span * d * 2 int32); cap is tab's length.
 * MF_ERR_DOMAIN if the table would exceed 2^22 rows. */
int mf_domain_table(int32_t d, double lambda, const mf_domain *dom, int32_t *smin, int32_t *span,
                    int32_t *tab, int64_t cap);

/* The 64-bit vertex keys of the tracing hash tables (host only, no GPU
 * needed).  y: host [n][d] lattice vertices; keys: host [n]; in_range: host
 * [n] or NULL, 1 where y lies inside the key packing (keys of such vertices
 * are distinct), else 0 (the key aliases another vertex).  The packing covers
 * every vertex within three lattice steps of the box; edge keys are
 * key * 2^d + mask.  MF_ERR_DOMAIN when edge keys of this domain and lambda
 * would not fit 64 bits. */
int mf_vertex_keys(int32_t d, double lambda, const mf_domain *dom, const int32_t *y, int64_t n,
                   uint64_t *keys, uint8_t *in_range);

/* f at n arbitrary points (the RBF kernel evaluation of the traced path).
 * q: device [n][d]; f_out: device [n].  precision as in mf_trace_opts; the
 * mixed paths apply the same FP64 recheck band (band <= 0 means 1e-3). */
int mf_eval(mf_ctx *ctx, const mf_rbf *rbf, const double *q, int64_t n, int32_t precision,
            double band, double *f_out, void *stream);

/* Manifold tracing (Sec. IV-A, Figs. 3-4) from n_seeds points: locate each
 * seed's n-simplex, keep its crossing edges, then breadth-first search over
 * shared 2-simplex cofaces until the frontier is empty; then the root of f
 * on every traced edge and the crossing n-simplices (Sec. IV-C).
 * seeds: device [n_seeds][d]. */
int mf_trace(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom, const mf_trace_opts *opts,
             const double *seeds, int64_t n_seeds, mf_trace_out *out, void *stream);

/* Copies the last mf_trace result of this context into `out` (two-call
 * pattern after MF_ERR_CAPACITY). */
int mf_trace_fetch(mf_ctx *ctx, mf_trace_out *out, void *stream);

/* Many independent traces (Sec. IV-A tracing, Sec. IV-C cells) in one launch:
 * trace t has its own RBF rbfs[t] (any d, support-vector count, gamma), domain
 * doms[t], options opts[t] (lambda, precision, capacities, flags) and seeds
 * seeds[t] (a host array of n device pointers to [n_seeds[t]][d_t]).  All
 * traces advance together: one CUDA-graph launch (a conditional WHILE loop
 * over breadth-first steps) runs every level of every trace, with the work
 * items of all traces sharing each kernel.  Results go to outs[t] exactly as
 * mf_trace writes them; a trace whose buffers are too small gets its counts
 * and the call returns MF_ERR_CAPACITY (call again with larger buffers).
 * 1 <= n <= 1024.  Capacities default to 2^20 edges per trace. */
int mf_trace_batch(mf_ctx *ctx, int32_t n, const mf_rbf *rbfs, const mf_domain *doms,
                   const mf_trace_opts *opts, const double *const *seeds, const int64_t *n_seeds,
                   mf_trace_out *outs, void *stream);

/* Batch triangulation (Sec. V-B, Figs. 5-6, Eqs. bc and local).  The
 * manifold is traced at the coarse scale k * opts->lambda (same offset); each
 * crossing n-simplex (z, pi) of that trace is then subdivided into the
 * triangulation of scale opts->lambda inside it: the local vertices v' with
 * k >= v'_0 >= ... >= v'_{d-1} >= 0 (Eq. local, read as the closed simplex),
 * mapped to the lattice vertices y = k z + sum_j v'_j e(pi_j) (Eq. bc), and
 * the local edges between them, the same template for every n-simplex.  The
 * result is every such edge with both vertices in the box and a sign change,
 * with its root as mf_trace solves it.  It is the direct trace at
 * opts->lambda wherever the coarse trace's n-simplices cover the manifold;
 * it misses fine crossings inside coarse n-simplices whose vertices all
 * share one sign.
 *
 * mf_subdiv_begin runs the coarse trace (capacities from opts, cells wanted)
 * and keeps its n-simplices in the context; *n_coarse_cells receives their
 * number.  Each mf_subdiv_next then processes the next cells_per_batch of
 * them (0 = all at once) into `out` as mf_trace does (edges, end values,
 * roots and points when opts asks for roots; no cells), with fine tables of
 * opts->max_edges / max_vertices that start empty every batch: the memory
 * is bounded by the batch, and an edge on a face shared by n-simplices of
 * two batches is reported by both.  *cells_left receives the n-simplices
 * still to do (0: finished; further calls return empty batches).  Any other
 * tracing, evaluation or tuning call on the context ends the subdivision.
 * k: 1 .. 16. */
int mf_subdiv_begin(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom, const mf_trace_opts *opts,
                    int32_t k, const double *seeds, int64_t n_seeds, int64_t cells_per_batch,
                    int64_t *n_coarse_cells, void *stream);
int mf_subdiv_next(mf_ctx *ctx, mf_trace_out *out, int64_t *cells_left, void *stream);

/* Proof server (continuous batching of tracing requests; the paper's
 * planner-side loop is out of scope, this is the serving runtime around the
 * traced path).  The server holds up to max_slots concurrent traces in an HBM
 * arena of hbm_bytes (one server per context).  Requests queue FIFO; each
 * mf_server_step admits queued requests while a slot is free and the
 * request's buffers (sized from its opts capacities, defaults 2^20 edges) fit
 * the arena, runs up to MF_SERVER_STEPS breadth-first steps of every running
 * trace in one launch of a CUDA graph built at creation (a conditional loop
 * whose body is one step of every slot), and finishes traces whose search ended
 * (roots, cells, CSR over just those slots).  A trace gives its slot back
 * when it finishes or fails; its results stay in the arena until fetched, so
 * a caller that never fetches eventually blocks admission by memory.  The
 * caller keeps each request's inputs (support vectors, alpha, seeds) alive
 * until the request is done, and passes the same stream to every step and
 * fetch of one server (memory handed back is reused in stream order). */
typedef struct mf_server mf_server;
#define MF_SERVER_STEPS 16 /* breadth-first steps per mf_server_step (fewer when all finish) */
int mf_server_create(mf_ctx *ctx, int32_t max_slots, size_t hbm_bytes, mf_server **out);
void mf_server_destroy(mf_server *s);
/* Queues a request; *id receives its handle. */
int mf_server_submit(mf_server *s, const mf_rbf *rbf, const mf_domain *dom,
                     const mf_trace_opts *opts, const double *seeds, int64_t n_seeds, int64_t *id);
/* One scheduling round (see above); reports running and queued requests. */
int mf_server_step(mf_server *s, void *stream, int32_t *n_running, int32_t *n_queued);
/* Ids (host, up to cap) of requests that finished or failed since the last
 * call, oldest first; *n receives how many were written. */
int mf_server_done(mf_server *s, int64_t *ids, int32_t cap, int32_t *n);
/* state: 0 queued, 1 running, 2 done, < 0 the request's error code; times are
 * host steady-clock seconds at submission, admission and completion. */
int mf_server_status(mf_server *s, int64_t id, int32_t *state, double *t_submit, double *t_admit,
                     double *t_done);
/* Copies a done request's results (as mf_trace does) and releases its
 * memory; a failed request returns its error code and is forgotten. */
int mf_server_fetch(mf_server *s, int64_t id, mf_trace_out *out, void *stream);
/* Runs mf_server_step until request id is done or has failed, or until
 * timeout_ms of host wall time have passed (MF_ERR_TIMEOUT; the request keeps
 * running and can be waited for again).  *state receives its state as
 * mf_server_status reports it.  Requests finished meanwhile are reported by
 * mf_server_done as usual. */
int mf_server_wait(mf_server *s, int64_t id, double timeout_ms, void *stream, int32_t *state);

/* Certification (Sec. V-C, App. A): forward kinematics of every point, exact
 * capsule/box and capsule/sphere distances, per-point margin
 * max_{link,obstacle}(radius - distance) and verdict (1 = in collision, i.e.
 * the point is in C_obs, iff margin >= 0), and per cell the AND of the
 * verdicts of its points.  points: device [n_points][d]; cell CSR: device
 * (n_cells may be 0 and the CSR pointers NULL); outputs: device
 * point_verdict [n_points], margin [n_points], cell_verdict [n_cells].
 * n_points must be below 2^32 (MF_ERR_INVALID otherwise); the context's
 * scratch holds 4 bytes per point for the points left to the full search. */
int mf_certify(mf_ctx *ctx, const mf_robot *robot, const mf_scene *scene, const double *points,
               int64_t n_points, int32_t d, const int64_t *cell_edge_off,
               const int64_t *cell_edge_idx, int64_t n_cells, uint8_t *point_verdict,
               double *margin, uint8_t *cell_verdict, void *stream);

/* Outputs of mf_certify_ex (caller-owned device buffers; NULL = not wanted,
 * except point_verdict and margin). */
typedef struct {
  uint8_t *point_verdict; /* [n_points] 1 iff the point is in collision (C_obs) */
  double *margin;         /* [n_points] max over elements and obstacles of radius - distance */
  int16_t *element;       /* [n_points] the deciding element (capsules, then spheres): the
                             lowest index whose margin is within 1e-9 of the maximum */
  uint8_t *cell_verdict;  /* [n_cells] AND of the verdicts of the cell's points */
  uint8_t *cell_whole;    /* [n_cells] 1 iff the whole-cell certificate holds (below) */
  double *cell_slack;     /* [n_cells] the certificate's slack (>= 0: certified) */
} mf_certify_out;

/* Certification as mf_certify, with the robot's spheres, cylinder obstacles,
 * the deciding element of every point, and the whole-cell certificate (the
 * rigorous form of the cell check that the paper's prior work uses, Sec.
 * IV-A; the paper itself checks points, Sec. V-C).  A cell's piece of the
 * traced manifold is the convex hull of its points.  Turning joint k by dq
 * moves a point of element e by at most L[e][k] |dq|, with L[e][k] the sum of
 * the link lengths sqrt(d_m^2 + a_m^2), m = k .. link(e) (plus |centre| for a
 * sphere; 0 for joints after the element's link).  So with span_jk the
 * largest |p_lk - p_jk| over the cell's points, every configuration of the
 * piece keeps element e_j's margin at least margin_j - sum_k L[e_j][k]
 * span_jk; slack = the maximum over the cell's points of margin_j - 1e-9 -
 * sum_k L[e_j][k] span_jk (the 1e-9 covers the deciding element's own margin,
 * within 1e-9 of margin_j), and cell_whole = (slack >= 0) certifies the whole
 * piece in collision.  The margin stops at the element's radius inside an
 * obstacle (distances are 0 there), which bounds what a cell can certify. */
int mf_certify_ex(mf_ctx *ctx, const mf_robot *robot, const mf_scene *scene, const double *points,
                  int64_t n_points, int32_t d, const int64_t *cell_edge_off,
                  const int64_t *cell_edge_idx, int64_t n_cells, const mf_certify_out *out,
                  void *stream);

/* Size of the fixed device array used by mf_trace_noalloc (64 MiB). */
#define MF_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* mf_trace without any allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code running
 * under another framework's memory pool, real-time loops that forbid
 * allocation after start-up, processes whose device memory is reserved by
 * someone else.  It computes what mf_trace computes (same arguments and
 * outputs, no context) with all scratch (hash tables, lists, counters,
 * prepared support vectors) carved from one file-scope device array of
 * MF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * exit.  It calls no cudaMalloc/cudaFree and no allocating library routine.
 *  - Runs on the current device.  Its first call on a device looks up the
 *    array's address (cudaGetSymbolAddress); make that call before any stream
 *    capture.  Under CUDA's lazy module loading the array is reserved on a
 *    device when the library's device code is loaded there: by that first
 *    call, or earlier by any launch of the library's kernels on the device.
 *    Make the first call at start-up, before device memory is reserved
 *    elsewhere; if the module cannot be loaded then, the call returns
 *    MF_ERR_CUDA (not MF_ERR_OOM).
 *  - Capacities: opts->max_edges / max_vertices / max_cells, or (when 0) the
 *    largest default that fits.  Requests whose tables and lists exceed the
 *    array return MF_ERR_OOM; output buffers that are too small return
 *    MF_ERR_CAPACITY with the counts filled (call again with larger ones).
 *  - All calls on a device share the array: each clears what must start
 *    empty, and calls that overlap on the GPU race and must not be issued.
 *  - No context means no mf_last_error message: the return code is the
 *    whole diagnosis. */
int mf_trace_noalloc(const mf_rbf *rbf, const mf_domain *dom, const mf_trace_opts *opts,
                     const double *seeds, int64_t n_seeds, mf_trace_out *out, void *stream);

/* Native per-phase profiling (CUDA events recorded on the call's stream
 * around every kernel launch of the library; no effect on results). */
#define MF_PHASES 12
enum {
  MF_PH_PREPARE = 0,   /* RBF preparation */
  MF_PH_SEEDS = 1,     /* locate edges (Fig. 3) */
  MF_PH_EXPAND_V = 2,  /* BFS: new vertices of 2-cofaces */
  MF_PH_EVAL = 3,      /* f at new vertices (incl. FP64 recheck) */
  MF_PH_EXPAND_E = 4,  /* BFS: new crossing edges, dedup */
  MF_PH_ROOTS = 5,     /* root solve on every traced edge */
  MF_PH_CELLS = 6,     /* n-cofaces of traced edges, dedup */
  MF_PH_CSR = 7,       /* cell -> edge CSR (count, scan, fill) */
  MF_PH_COPY = 8,      /* copies into caller buffers */
  MF_PH_CERT_PTS = 9,  /* FK + capsule/obstacle distances */
  MF_PH_CERT_CELLS = 10,
  MF_PH_OTHER = 11
};
typedef struct {
  double ms[MF_PHASES];        /* device time summed over the phase's launches */
  int64_t launches[MF_PHASES]; /* kernel launches of the phase */
  int64_t units[MF_PHASES];    /* work items: seeds, frontier edges, edges solved, points ... */
  int64_t terms[MF_PHASES];    /* strong RBF terms: FP64 exp (eval phase; the root
                                  step's full FP64 re-evaluations) or double-float
                                  (the root step's lane-per-chunk sums) */
  int64_t terms_weak[MF_PHASES]; /* RBF terms in FP32 with ex2: weak terms, the tensor-
                                    core tiles' terms, the root solve's FP32 Halley steps */
} mf_stats;

/* Enables (1) or disables (0) profiling on the context; enabling clears the stats. */
int mf_ctx_set_profiling(mf_ctx *ctx, int enable);
/* Copies the accumulated stats (zeros when profiling is off). */
int mf_ctx_get_stats(mf_ctx *ctx, mf_stats *out);

/* Autotuning (batched multi-trace and single traces; no counterpart in the
 * paper, which runs fixed launch shapes).  mf_autotune traces the request
 * once per BFS-chunk candidate (roots and cells off), then times on that
 * trace the launch variants of the root solve (register cap x grid x group
 * screen size), of the
 * FP64 vertex evaluation (grid) and, for MF_MIXED_BF16, of the tensor-core
 * chunk width (64 or 128 support vectors per MMA).  The fastest of each is
 * kept in the context and used by every later mf_trace on it; *out (host)
 * receives the choices and their times.  Results of earlier traces are
 * invalidated (mf_trace_fetch fails until the next mf_trace). */
typedef struct {
  int32_t roots_variant;       /* 0: up to 128 registers (2 blocks/SM), 1: 3 blocks/SM */
  int32_t roots_blocks_per_sm; /* root-solve grid = this x SMs */
  int32_t eval_blocks_per_sm;  /* FP64 vertex-evaluation grid = this x SMs */
  int32_t tc_chunk;            /* support vectors per tensor-core MMA: 64 or 128 */
  int64_t frontier_chunk;      /* edges per BFS expansion step; 0 = the batch cap */
  double ms_bfs;               /* measured: breadth-first search with the chosen chunk */
  double ms_roots;             /* measured: root solve of the sampled edges */
  double ms_eval;              /* measured: evaluation of every traced vertex */
  int32_t n_candidates;        /* launch variants timed */
  int32_t roots_group;         /* consecutive edges sharing one group screen (1: none) */
} mf_tune;
int mf_autotune(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom, const mf_trace_opts *opts,
                const double *seeds, int64_t n_seeds, mf_tune *out, void *stream);
/* Applies launch choices (NULL restores the defaults) / reads the current ones
 * (the ms_* and n_candidates fields are ignored / zero). */
int mf_ctx_set_tune(mf_ctx *ctx, const mf_tune *t);
int mf_ctx_get_tune(mf_ctx *ctx, mf_tune *out);

/* Measured throughput of the pipes that bound the traced path on this GPU
 * (no counterpart in the paper; the denominators of the roofline the
 * benchmark reports).  Each probe kernel runs independent chains on every SM
 * (8 blocks of 256 threads per SM) and the best of three timed launches is
 * kept.  Rates are thread-level operations per second. */
typedef struct {
  double fp64_fma_per_s;  /* FP64 fused multiply-adds */
  double fp32_fma_per_s;  /* FP32 fused multiply-adds */
  double ex2_per_s;       /* FP32 ex2.approx (MUFU) */
  double exp_neg_per_s;   /* the FP64 table-driven exp of the RBF terms */
  int32_t sm_count;
  double sm_clock_mhz;    /* the device's nominal SM clock */
} mf_rates;
int mf_probe_rates(mf_ctx *ctx, mf_rates *out, void *stream);

/* Accuracy diagnostic of the FP64 exp the RBF kernels use (Tang's
 * table-driven method, ACM TOMS 15(2), 1989): y_table[i] = that exp of x[i],
 * y_lib[i] = CUDA's exp(x[i]), for comparison on the host.  x, y_*: device
 * [n]; meant for x in [-708, 0] (the kernels' arguments are -gamma r^2). */
int mf_diag_exp(mf_ctx *ctx, const double *x, int64_t n, double *y_table, double *y_lib,
                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MF_H */
