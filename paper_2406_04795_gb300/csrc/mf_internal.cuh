// mf_internal.cuh -- device-side building blocks shared by the library's
// translation units: the lattice frame of one trace, integer simplex keys,
// open-addressing hash tables, and the trace's device counters.
#pragma once
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mf.h"

#define MF_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

// Lattice frame of one trace: the Ã_d realisation x = lam * (y - c * sum(y)) + o
// (Sec. II-B; L = I - c 1 1^T, c = (1 - 1/sqrt(d+1))/d), the closed C-space box,
// and the packing of lattice vertices into 64-bit keys.
struct MfFrame {
  int32_t d;
  double lam, c, cinv;  // cinv = c * sqrt(d+1): L^-1 = I + cinv 1 1^T
  double o[MF_MAXD], lo[MF_MAXD], hi[MF_MAXD];
  int32_t ymin[MF_MAXD];    // bounding box of the box's lattice coordinates,
  int32_t range[MF_MAXD];   // with a margin of 3 (domain-table search range)
  // Vertex keys, a sheared mixed radix: with s = sum(y) and
  // q(s) = floor(s * qc / 2^32) ~ c s, the digits are s - kmin_s and
  // y_i - q(s) - zmin[i] for i < d-1 (y_{d-1} follows from s).  y_i - q(s)
  // tracks (x_i - o_i) / lam, so the key space spans the box itself, not the
  // bounding box of its lattice coordinates (smaller by ~(1 + d cinv)^d / sqrt(d+1)).
  uint32_t qc;
  int32_t kmin_s, kspan_s;
  int32_t zmin[MF_MAXD];
  uint64_t kstride[MF_MAXD];  // place value of digit i < d-1
  uint64_t sstride;           // place value of the s digit
  // Optional exact domain table: for s = sum(y) in [smin, smin + sspan) and
  // each axis i, the interval of y_i whose x_i (computed as mf_vertex_x does)
  // lies in [lo_i, hi_i].  NULL: the domain test evaluates x in FP64.
  const int2 *dom_tab;      // [sspan][d]
  int32_t smin, sspan;
};

// Device counters of one trace; read back by the host once per BFS level.
struct MfCounters {
  unsigned long long n_edges;      // edges appended to the edge list
  unsigned long long n_vertices;   // vertices appended to the vertex list
  unsigned long long v_evaluated;  // vertex list prefix whose f is final
  unsigned long long n_cells;
  unsigned long long n_boundary;
  unsigned long long n_near_zero;
  unsigned long long n_dead_seeds;
  unsigned long long n_recheck;    // mixed: vertices queued for FP64 recheck
  unsigned long long n_recheck_done;
  unsigned long long root_evals;
  unsigned long long n_cell_edges;
  unsigned long long eval_terms;   // RBF terms with FP64 exp, vertex evaluation
  unsigned long long root_terms;   // RBF terms with FP64 exp, root solve
  unsigned long long eval_terms_weak;  // RBF terms with the reduced-cost exp, vertex evaluation
  unsigned long long root_terms_weak;  // RBF terms with the reduced-cost exp, root solve
  unsigned long long n_vlist;      // entries taken from the per-vertex list pool
  unsigned long long root_overflow;  // edges whose screen lists overflowed (full re-evaluation)
  unsigned long long n_defer;      // root steps handed to the lane-per-edge FP64 kernel
  unsigned long long n_defer_list; // their strong-term list entries
  unsigned long long n_redo;       // deferred steps not accepted (solved again in full)
  unsigned long long n_items;      // expand items of the current chunk given a vertex slot
  unsigned int err_table_full;     // a hash probe ran past the table
  unsigned int err_overflow;       // a list ran past its capacity
  unsigned int err_missing;        // a vertex expected in the table was absent
  unsigned int err_timeout;        // a bounded device-side wait gave up
};

// Pointers of one trace's resident device state (all owned by the context).
struct MfTraceBufs {
  // edge hash table: key -> index into the edge list
  // 16-byte slots (key word, then the value word), so that a probe that
  // finds its key has the value in the same memory sector
  unsigned long long *etab_key;  // [TE][2]: key, edge-list index (u32)
  uint64_t etab_mask;
  // vertex hash table: key -> f
  unsigned long long *vtab_key;  // [TV][2]: key, f (f64)
  uint64_t vtab_mask;
  // cell hash table (keys only; winners append to the cell list)
  // edge list (insertion order; each BFS level is a contiguous range)
  int32_t *edge_y;     // [ME][d]
  uint32_t *edge_mask; // [ME]
  double *edge_f;      // [ME][2]
  double *edge_t;      // [ME]
  double *edge_pt;     // [ME][d]
  uint64_t max_edges;
  // vertex list (insertion order): lattice vertex and its table slot
  int32_t *vert_y;     // [MV][d]
  uint32_t *vert_slot; // [MV]
  uint64_t max_vertices;
  // mixed path: recheck queue of vertex-list indices
  uint32_t *recheck;   // [MV]
  // cell list
  int32_t *cell_y;     // [MC][d]
  uint8_t *cell_perm;  // [MC][d]
  int64_t *cell_off;   // [MC+1]
  uint32_t *cell_sgn;  // [MC] per cell vertex i: bit i = in the vertex table, bit 16+i = f >= 0
  int64_t *cell_idx;   // [MC * (d+1)d/2]
  uint64_t max_cells;
  MfCounters *cnt;
  // Per-vertex support-vector lists for the root screen (FP64 path; NULL:
  // none).  Vertex i's list holds every vector within sqrt(list_r2) of it,
  // a radius that covers the screen radius around any point of an edge
  // leaving the vertex.
  uint32_t *vtab_idx;   // [vertex table size] vertex-list index of each slot
  int32_t *vlist;       // pool of vector indices
  uint64_t *vlist_off;  // [MV] offset of vertex i's list in the pool
  uint32_t *vlist_n;    // [MV] its length, MF_NO_LIST when it has none
  uint64_t vlist_cap;   // pool capacity (entries)
  float list_r2;
  // Deferred FP64 root steps of one chunk of edges (NULL: none): records of
  // the edges whose single FP64 Newton step runs lane per edge, their
  // strong-term lists in 8-entry chunks (-1 pads a list), the queue of edges
  // to solve again in full, the chunk's end points in FP32 for the warp
  // kernel, and the steps' evaluation points and chunk sums.
  void *defer_rec;          // [defer_cap] records (32 bytes each)
  int32_t *defer_list;      // [defer_list_cap] support-vector indices
  uint64_t *redo;           // [defer_cap] edge indices
  float *ep32;              // [defer_cap][MF_EP_ROW(d)]: x1 hi, x1 lo, dir, f(x1), f(x2),
                            // [f(x1) >= 0], base vertex's list length and offset (bits)
  double *defer_x;          // [defer_cap][2d] FP64 x1, dir
  float *defer_x3;          // [defer_cap][3d] step points, each coordinate as three floats
  float *defer_bnd;         // [defer_list_cap / 8] error weight of each chunk (see k_roots_terms)
  double *defer_part;       // [defer_list_cap / 8] FP64 sum of each chunk
  uint32_t *defer_chunk;    // [defer_list_cap / 8] record of each chunk (~0: none)
  uint64_t defer_cap, defer_list_cap;
  // vertex slots of the expand items of the whole search: k_expand_vertices
  // records the slot of item j of warp w of a chunk at
  // item_slot[warp_base[w] + j] (~0u: outside the domain) and the first item
  // of each edge in edge_item_off (~0: not recorded); k_expand_edges and the
  // cell enumeration's link tables read them instead of looking the
  // vertices up (warp_base[w] = ~0: the warp's items did not fit, look them
  // up); absent when null
  uint32_t *item_slot;
  unsigned long long *warp_base;
  unsigned long long *edge_item_off;
  uint64_t item_cap;
};
#define MF_NO_LIST 0xFFFFFFFFu
#define MF_EP_ROW(d) (3 * (d) + 6)

// Prepared RBF: structure-of-arrays copies for coalesced streaming.
struct MfRbfDev {
  int32_t d;
  int32_t n;
  const float *sv32;   // [d][n] FP32 rounding of the coordinates
  const float *svlo32; // [d][n] s - (double)sv32: the low part of a hi/lo split
  const double *sv64;  // [d][n]
  const double *alpha; // [n]
  const float *alpha32;// [n]
  const float *strong32; // [n] ln(|alpha| / tau): term needs the FP64 exp iff gamma r^2 below
  const double *exp_tab; // [64] 2^(j/64), the table of mf_exp_neg
  // row-major copies for gathers (one support vector per 64-byte row):
  const double *sv64r;   // [n][8] coordinates, zero-padded
  const float *svhl;     // [n][16] (hi, lo) FP32 pairs of the coordinates; for d < 8
                         // the pair after them holds (alpha, strong32)
  // double-float (FP32 pair) forms for the root step's strong terms:
  const float *sv3;        // [n][24] each coordinate as three floats s1 + s2 + s3 (exact)
  const float *alpha_lo32; // [n] alpha - (double)alpha32
  const float2 *exp_df;    // [1024] 2^(-j/1024) as (hi, lo)
  // blocks of 32 consecutive vectors (the preparation orders the vectors
  // along a Morton curve, so a block is spatially compact): FP32 box of sv32
  const float *blk_lo, *blk_hi;  // [d][nblk]
  int32_t nblk;
  double gamma, b;
  double sum_abs_alpha;
  float screen_r2;     // keep a term in the FP64 sum iff r^2 (FP32) <= screen_r2
  double drop_bound;   // sum_i |alpha_i| exp(-gamma * screen cut): bound on dropped terms
  double weak_limit;   // allowed error of the FP32 weak terms (2.5e-13 - drop_bound)
  double weak_rel;     // relative error bound of one FP32 weak term
  float weak_limit32, drop_bound32, weak_rel32;  // FP32 copies for the FP32 checks
  float smax;          // max |s_ik| over all support-vector coordinates
  // the mixed paths' root solve (|dt| <= 1e-6): its screen keeps the terms
  // with r^2 <= screen_r2_fast, dropping at most drop_bound32_fast (1e-12)
  float screen_r2_fast, drop_bound32_fast;
};

// ------------------------------------------------------------------------
// Batches: many independent traces advanced together by the same kernels.
// Every work item (frontier edge x mask, vertex, edge, cell) carries its
// trace through a prefix array over the slots.
// ------------------------------------------------------------------------
#define MF_MAX_SLOTS 1024
#define MF_TC_TILE 128  // vertices per tensor-core tile (the MMA's M)

struct MfSlot {  // one trace of a batch (device-resident descriptor)
  MfFrame F;
  MfRbfDev R;
  MfTraceBufs B;
  int32_t precision;
  double band;             // mixed precision: FP64 recheck band
  double root_tol;
  unsigned long long cap;  // frontier edges expanded per step
  uint32_t flags;          // MF_WANT_ROOTS | MF_WANT_CELLS
};

struct MfSlotState;
struct MfBatchPlan;

// Host launchers of the batched kernels.
void mf_b_launch_init(const MfSlot *slots, MfSlotState *st, int n, cudaStream_t s);
void mf_b_launch_expand(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n, bool edges,
                        int sms, cudaStream_t s);
void mf_b_launch_plan_eval(const MfSlot *slots, MfBatchPlan *P, int n, bool recheck, cudaStream_t s);
void mf_b_launch_advance(const MfSlot *slots, int n, cudaStream_t s);
void mf_b_launch_update(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n,
                        cudaGraphConditionalHandle h, int use_handle, cudaStream_t s);
// `only` (device, n int32, may be NULL): restrict roots / cells / CSR to the
// slots with a non-zero entry.
// dim > 0 restricts mode 0 (roots) to the slots of that dimension.
void mf_b_launch_plan_edges(const MfSlot *slots, MfBatchPlan *P, int n, int cells,
                            const int32_t *only, cudaStream_t s, int dim = 0);
void mf_b_launch_cells(const MfSlot *slots, MfBatchPlan *P, int n, const int32_t *only, int sms,
                       cudaStream_t s);
void mf_b_launch_cell_edges(const MfSlot *slots, MfBatchPlan *P, int n, bool fill,
                            const int32_t *only, int sms, cudaStream_t s);
// Vertex evaluation of every slot: FP64 or FP32 SIMT warps, the tensor-core
// tiles of MF_MIXED_BF16 slots (tc_chunk support vectors per MMA), the FP64
// recheck of the mixed slots, and the per-vertex root-screen lists.
void mf_b_launch_eval(const MfSlot *slots, MfBatchPlan *P, int n, bool any_mixed, int tc_chunk,
                      int sms, cudaStream_t s);
void mf_b_launch_eval_tc(const MfSlot *slots, const MfBatchPlan *P, int n, int n_chunk, int sms,
                         cudaStream_t st);
// dims: bit d set when some slot has dimension d (one exact-d launch each).
void mf_b_launch_roots(const MfSlot *slots, MfBatchPlan *P, int n, const int32_t *only,
                       uint32_t dims, int group, int sms, cudaStream_t s);

struct MfSlotState {  // breadth-first progress of one trace
  unsigned long long cursor;     // next frontier edge to expand
  unsigned long long level_end;  // end of the current level in the edge list
  unsigned long long chunk_n;    // edges expanded by the current step
  int32_t active, levels, err, pad;
};

struct MfBatchPlan {  // per-step work prefixes over the slots
  unsigned long long px[MF_MAX_SLOTS + 1];  // edges of this expansion chunk
  unsigned long long pv[MF_MAX_SLOTS + 1];  // vertices to evaluate
  unsigned long long pr[MF_MAX_SLOTS + 1];  // vertices to re-check in FP64
  unsigned long long pe[MF_MAX_SLOTS + 1];  // traced edges (roots, cells)
  unsigned long long pc[MF_MAX_SLOTS + 1];  // cells (CSR)
  unsigned long long pt[MF_MAX_SLOTS + 1];  // tensor-core tiles (MF_MIXED_BF16 slots)
  unsigned long long v0[MF_MAX_SLOTS], r0[MF_MAX_SLOTS];
  unsigned long long steps;  // steps run since the plan was cleared
  int32_t overrun;           // the step limit stopped the search
  int32_t budget;            // > 0: the graph loop pauses after this many steps
};
#define MF_MAX_STEPS (1ull << 22)  // bound on breadth-first steps of one batch

// Largest t in [0, n) with p[t] <= item (p non-decreasing, p[0] = 0).
__device__ __forceinline__ int mf_slot_of(const unsigned long long *p, int n,
                                          unsigned long long item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------------
// Lattice arithmetic with a fixed operation order (no contraction) so that a
// vertex's coordinates are bit-identical wherever they are computed.
// ------------------------------------------------------------------------
__device__ __forceinline__ void mf_vertex_x(const MfFrame &F, const int32_t *y, double *x) {
  long long s = 0;
#pragma unroll
  for (int i = 0; i < MF_MAXD; i++)
    if (i < F.d) s += y[i];
  const double cs = __dmul_rn(F.c, (double)s);
#pragma unroll
  for (int i = 0; i < MF_MAXD; i++)
    if (i < F.d) x[i] = __dadd_rn(__dmul_rn(F.lam, __dsub_rn((double)y[i], cs)), F.o[i]);
}

__device__ __forceinline__ bool mf_in_box(const MfFrame &F, const double *x) {
  bool in = true;
#pragma unroll
  for (int i = 0; i < MF_MAXD; i++)
    if (i < F.d) in = in && (x[i] >= F.lo[i]) && (x[i] <= F.hi[i]);
  return in;
}

// Is lattice vertex y inside the box?  Exactly the decision mf_in_box makes on
// mf_vertex_x(y): by integer table lookups when the frame has a table.
__device__ __forceinline__ bool mf_vertex_in(const MfFrame &F, const int32_t *y) {
  if (F.dom_tab) {
    int s = 0;
#pragma unroll
    for (int i = 0; i < MF_MAXD; i++)
      if (i < F.d) s += y[i];
    const unsigned row = (unsigned)(s - F.smin);
    if (row >= (unsigned)F.sspan) return false;
    const int2 *r = F.dom_tab + (size_t)row * F.d;
    bool in = true;
#pragma unroll
    for (int i = 0; i < MF_MAXD; i++)
      if (i < F.d) {
        const int2 b = r[i];
        in = in && y[i] >= b.x && y[i] <= b.y;
      }
    return in;
  }
  double x[MF_MAXD];
  mf_vertex_x(F, y, x);
  return mf_in_box(F, x);
}

// Vertex key (the packing described at MfFrame).  Unique over the vertices
// the kernels key: those within one lattice step of a point of the box.
__host__ __device__ __forceinline__ unsigned long long mf_vertex_key(const MfFrame &F,
                                                                     const int32_t *y) {
  // |s| < 2^30 on encodable vertices, so s, q and every digit fit 32 bits
  int s = 0;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int i = 0; i < MF_MAXD; i++)
    if (i < F.d) s += y[i];
  const int q = (int)(((long long)s * (long long)F.qc) >> 32);  // floor: arithmetic shift
  unsigned long long k = (unsigned long long)(uint32_t)(s - F.kmin_s) * F.sstride;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
  for (int i = 0; i < MF_MAXD - 1; i++)
    if (i < F.d - 1) k += (unsigned long long)(uint32_t)(y[i] - q - F.zmin[i]) * F.kstride[i];
  return k;
}

// Host: is y inside the packing's digit ranges (its key then unique)?
static inline bool mf_vertex_in_packing(const MfFrame &F, const int32_t *y) {
  long long s = 0;
  for (int i = 0; i < F.d; i++) s += y[i];
  if (s < F.kmin_s || s - F.kmin_s >= F.kspan_s) return false;
  const long long q = (s * (long long)F.qc) >> 32;
  for (int i = 0; i < F.d - 1; i++) {
    const long long z = (long long)y[i] - q - F.zmin[i];
    const long long next = i + 1 < F.d - 1 ? (long long)F.kstride[i + 1] : (long long)F.sstride;
    if (z < 0 || z >= next / (long long)F.kstride[i]) return false;
  }
  return true;
}

// Host: sets the key packing of a frame whose lattice and box are set; false
// when vertex or edge (vkey 2^d + mask) keys would not fit 64 bits (cells
// are written once each and need no key).  Every vertex the kernels key lies within one lattice step
// (|dy_i| <= 1) of a point p of the box; the packing covers three.  With
// u = (p - o) / lam in [A, B] and s' = sqrt(d+1) sum(u), such a vertex has
// y_i - c s within 2k of u_i (k steps, d c < 1), y_i - q(s) within [-e, 1 + e]
// of that, and s within d k of s': margins 8 and 9 on the digits, 3d + 2 on s.
static inline bool mf_frame_pack_keys(MfFrame *F) {
  const int d = F->d;
  F->qc = (uint32_t)std::llround(F->c * 4294967296.0);  // c < 1
  double sa = 0.0, sb = 0.0;
  long long zmin[MF_MAXD], zr[MF_MAXD];
  for (int i = 0; i < d; i++) {
    const double A = (F->lo[i] - F->o[i]) / F->lam, B = (F->hi[i] - F->o[i]) / F->lam;
    if (!(std::fabs(A) < 1e9 && std::fabs(B) < 1e9)) return false;
    zmin[i] = (long long)std::floor(A) - 8;
    zr[i] = (long long)std::ceil(B) + 9 - zmin[i] + 1;
    sa += A;
    sb += B;
  }
  const double r = std::sqrt((double)(d + 1));
  const long long s0 = (long long)std::floor(r * sa) - 3 * d - 2;
  const long long s1 = (long long)std::ceil(r * sb) + 3 * d + 2;
  if (s0 < -(1ll << 29) || s1 > (1ll << 29)) return false;  // s, q and digits fit int32
  F->kmin_s = (int32_t)s0;
  F->kspan_s = (int32_t)(s1 - s0 + 1);
  unsigned __int128 prod = 1;
  for (int i = 0; i < d - 1; i++) {
    F->zmin[i] = (int32_t)zmin[i];
    F->kstride[i] = (uint64_t)prod;
    prod *= (unsigned __int128)zr[i];
    if (prod > ((unsigned __int128)1 << 62)) return false;
  }
  F->sstride = (uint64_t)prod;
  prod *= (unsigned __int128)(s1 - s0 + 1);
  if (prod > ((unsigned __int128)1 << 62)) return false;
  const unsigned __int128 lim = ((unsigned __int128)1 << 64) - 2;
  return !((prod << d) > lim);
}

// Edge (y, p1) with p1 a non-empty mask over {0..d-1}: key = vidx * 2^d + p1.
__device__ __forceinline__ unsigned long long mf_edge_key(const MfFrame &F, const int32_t *y,
                                                          uint32_t mask) {
  return (mf_vertex_key(F, y) << F.d) | (unsigned long long)mask;
}

// v += e(M) for M a mask over {0..d-1}
__device__ __forceinline__ void mf_add_mask(int d, int32_t *v, uint32_t M, int sign) {
#pragma unroll
  for (int i = 0; i < MF_MAXD; i++)
    if (i < d && ((M >> i) & 1u)) v[i] += sign;
}

// Query type 1 (Sec. IV-A): locate the n-simplex holding x.  Same operation
// order as the inverse map y' = L^-1 (x - o) / lam; vertex = floor(y'); the walk
// order sorts the fractional parts descending, ties to the lower index.
__device__ __forceinline__ void mf_locate_point(const MfFrame &F, const double *x, int32_t *y,
                                                int *perm) {
  const int d = F.d;
  double s = 0.0;
  for (int j = 0; j < d; j++) s = __dadd_rn(s, __dsub_rn(x[j], F.o[j]));
  double fr[MF_MAXD];
  for (int i = 0; i < d; i++) {
    double u = __dadd_rn(__dsub_rn(x[i], F.o[i]), __dmul_rn(F.cinv, s));
    double yp = __ddiv_rn(u, F.lam);
    double fl = floor(yp);
    y[i] = (int32_t)fl;
    fr[i] = __dsub_rn(yp, fl);
    perm[i] = i;
  }
  for (int i = 1; i < d; i++) {
    int p = perm[i], j = i - 1;
    while (j >= 0 && fr[perm[j]] < fr[p]) { perm[j + 1] = perm[j]; j--; }
    perm[j + 1] = p;
  }
}

// ------------------------------------------------------------------------
// Open-addressing hash tables (linear probing, 64-bit keys, atomicCAS).
// ------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mf_hash64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Insert-if-absent.  Returns the slot; *won = true iff this call inserted.
// Returns ~0ull if the table is full (probe count exceeded its size).
template <int STRIDE = 1>
__device__ __forceinline__ uint64_t mf_table_insert(unsigned long long *keys, uint64_t mask,
                                                    unsigned long long key, bool *won) {
  uint64_t h = mf_hash64(key) & mask;
  for (uint64_t probe = 0; probe <= mask; probe++) {
    unsigned long long cur = keys[h * STRIDE];
    if (cur == key) { *won = false; return h; }
    if (cur == MF_EMPTY_KEY) {
      unsigned long long prev = atomicCAS(&keys[h * STRIDE], MF_EMPTY_KEY, key);
      if (prev == MF_EMPTY_KEY) { *won = true; return h; }
      if (prev == key) { *won = false; return h; }
    }
    h = (h + 1) & mask;
  }
  *won = false;
  return ~0ull;
}

// Lookup; returns the slot or ~0ull if absent.
template <int STRIDE = 1>
__device__ __forceinline__ uint64_t mf_table_find(const unsigned long long *keys, uint64_t mask,
                                                  unsigned long long key) {
  uint64_t h = mf_hash64(key) & mask;
  for (uint64_t probe = 0; probe <= mask; probe++) {
    unsigned long long cur = keys[h * STRIDE];
    if (cur == key) return h;
    if (cur == MF_EMPTY_KEY) return ~0ull;
    h = (h + 1) & mask;
  }
  return ~0ull;
}

// Value words of the interleaved vertex and edge tables.
__device__ __forceinline__ double &mf_vtab_f(const MfTraceBufs &B, uint64_t slot) {
  return reinterpret_cast<double *>(B.vtab_key)[2 * slot + 1];
}
__device__ __forceinline__ uint32_t &mf_etab_val(const MfTraceBufs &B, uint64_t slot) {
  return *reinterpret_cast<uint32_t *>(B.etab_key + 2 * slot + 1);
}

// Warp-aggregated list allocation: every calling lane with take = true gets
// a distinct index from *counter, with one atomic per group of lanes that
// share the counter (batched kernels mix traces in a warp).  Callable from
// divergent code: the group is the lanes active at the call.
__device__ __forceinline__ unsigned long long mf_warp_alloc(unsigned long long *counter, bool take) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, (unsigned long long)counter);
  const unsigned m = __ballot_sync(act, take) & peers;
  const int lane = threadIdx.x & 31;
  const int leader = m ? __ffs(m) - 1 : lane;
  unsigned long long base = 0;
  if (m && lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
  base = __shfl_sync(act, base, leader);
  return base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
}

// ------------------------------------------------------------------------
// Vertex and edge tables of a trace (the tracing and batch-triangulation
// kernels share them).
// ------------------------------------------------------------------------
// Inserts an in-domain vertex into the vertex table; first inserter appends it.
// Inserts vertex w if new (appending it to the vertex list); returns its
// table slot (~0: the table is full).
__device__ __forceinline__ uint64_t mf_visit_vertex(const MfFrame &F, const MfTraceBufs &B, const int32_t *w) {
  const unsigned long long key = mf_vertex_key(F, w);
  bool won;
  const uint64_t slot = mf_table_insert<2>(B.vtab_key, B.vtab_mask, key, &won);
  if (slot == ~0ull) atomicOr(&B.cnt->err_table_full, 1u);
  const bool take = slot != ~0ull && won;
  const unsigned long long idx = mf_warp_alloc(&B.cnt->n_vertices, take);
  if (!take) return slot;
  if (idx >= B.max_vertices) { atomicOr(&B.cnt->err_overflow, 1u); return slot; }
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++)
    if (k < F.d) B.vert_y[idx * F.d + k] = w[k];
  B.vert_slot[idx] = (uint32_t)slot;
  if (B.vtab_idx) B.vtab_idx[slot] = (uint32_t)idx;
  return slot;
}

__device__ __forceinline__ double mf_lookup_f(const MfFrame &F, const MfTraceBufs &B, const int32_t *w) {
  const uint64_t slot = mf_table_find<2>(B.vtab_key, B.vtab_mask, mf_vertex_key(F, w));
  if (slot == ~0ull) { atomicOr(&B.cnt->err_missing, 1u); return 0.0; }
  return mf_vtab_f(B, slot);
}

// Appends edge (y, mask) with end values (fa at y, fb at y + e(mask)) if new.
__device__ __forceinline__ void mf_emit_edge(const MfFrame &F, const MfTraceBufs &B, const int32_t *y,
                                          uint32_t mask, double fa, double fb) {
  const unsigned long long key = mf_edge_key(F, y, mask);
  bool won;
  const uint64_t slot = mf_table_insert<2>(B.etab_key, B.etab_mask, key, &won);
  if (slot == ~0ull) atomicOr(&B.cnt->err_table_full, 1u);
  const bool take = slot != ~0ull && won;
  const unsigned long long idx = mf_warp_alloc(&B.cnt->n_edges, take);
  if (!take) return;
  if (idx >= B.max_edges) { atomicOr(&B.cnt->err_overflow, 1u); return; }
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++)
    if (k < F.d) B.edge_y[idx * F.d + k] = y[k];
  B.edge_mask[idx] = mask;
  B.edge_f[2 * idx] = fa;
  B.edge_f[2 * idx + 1] = fb;
  mf_etab_val(B, slot) = (uint32_t)idx;
}

__device__ __forceinline__ unsigned long long mf_warp_sum_ull(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float mf_warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double mf_warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------------
// Host-side helpers shared by the translation units (defined in mf_api.cu).
// ------------------------------------------------------------------------
int mf_set_error(mf_ctx *ctx, int code, const char *fmt, ...);
int mf_cuda_check(mf_ctx *ctx, cudaError_t e, const char *what);
// Device arena of the context: returns a 256-byte aligned region of `bytes`
// from slot `slot` (each slot is a separately grown allocation), or NULL with
// the error set when the budget would be exceeded.
void *mf_ctx_buffer(mf_ctx *ctx, int slot, size_t bytes);
int mf_ctx_sm_count(mf_ctx *ctx);

// RBF preparation (mf_eval.cu): SoA FP32/FP64 copies in context buffers.
int mf_prepare_rbf(mf_ctx *ctx, const mf_rbf *rbf, MfRbfDev *out, cudaStream_t st);
size_t mf_rbf_prep_bytes(int d, int64_t n);
int mf_prepare_rbf_at(mf_ctx *ctx, const mf_rbf *rbf, char *base, MfRbfDev *out, cudaStream_t st);
// Squared radius of a vertex's root-screen list: the screen radius around
// any point of an edge leaving the vertex.  The longest edge is lam |L e(M)|
// with |L e(M)|^2 = k (1 - 2ck + c^2 k d) for |M| = k; the margins cover the
// FP32 distances of both screens.
// fast: for the mixed paths' root solve (screen_r2_fast).
static inline float mf_list_r2(const MfFrame &F, const MfRbfDev &R, bool fast = false) {
  double m2 = 0.0;
  for (int k = 1; k <= F.d; k++) {
    const double v = k * (1.0 - 2.0 * F.c * k + F.c * F.c * k * F.d);
    if (v > m2) m2 = v;
  }
  const double rs2 = fast ? (double)R.screen_r2_fast : (double)R.screen_r2;
  const double rl = std::sqrt(rs2) * 1.0001 + F.lam * std::sqrt(m2) + 1e-4;
  return (float)(rl * rl);
}
// Trace host helpers (mf_trace.cu).
int mf_build_frame(mf_ctx *ctx, int d, double lam, const mf_domain *dom, MfFrame *F);
void mf_exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch, cudaStream_t st);
uint64_t mf_next_pow2(uint64_t x);
void mf_launch_seeds(const MfFrame &F, const MfTraceBufs &B, const double *seeds, int64_t n,
                     bool vertices, cudaStream_t s);
// The crossing n-simplices of edges [0, n_edges) with their sign masks and
// CSR row lengths (in B.cell_off), and, once cell_off is scanned, the CSR
// fill of B.cell_idx (a missing edge sets err_missing).
void mf_launch_cells_enum(const MfFrame &F, const MfTraceBufs &B, uint64_t n_edges, cudaStream_t st);
void mf_launch_cells_fill(const MfFrame &F, const MfTraceBufs &B, uint64_t n_cells, cudaStream_t st);
// Launch choices picked by the autotuner (mf_autotune); the defaults serve
// untuned contexts and the allocation-free entry point.
struct MfTune {
  int roots_variant = 0;         // 0: no register cap (2 blocks/SM), 1: 3 blocks/SM
  int roots_bps = 4;             // root-solve blocks per SM in the grid
  int roots_group = 1;           // consecutive edges sharing one group screen (1 = none)
  int eval_bps = 8;              // FP64 vertex-evaluation blocks per SM
  int tc_chunk = 64;             // support vectors per tensor-core MMA: 64 or 128
  uint64_t frontier_chunk = 0;   // BFS chunk in edges; 0 = the caller's batch cap
};

// Evaluate f at vertex-list entries [begin, end) read from the device counter
// (FP64 path); writes f into each vertex's table slot.
void mf_launch_eval_vertices_f64(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                 const MfTune &T, int sms, cudaStream_t st);
void mf_launch_eval_vertices_mixed(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                   int precision, double band, const MfTune &T, int sms,
                                   cudaStream_t st);
// fast: the mixed paths' root accuracy (|dt| <= 1e-6 instead of 1e-9), with
// fewer terms in the FP64 step.
void mf_launch_roots_f64(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                         uint64_t n_edges, double tol, const MfTune &T, int sms, cudaStream_t st,
                         bool fast = false);
void mf_launch_eval_vertices_tc(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                double band, int n_chunk, int sms, cudaStream_t st);

// Context slots (each a separately grown device allocation).
enum {
  MF_SLOT_COUNTERS = 0,
  MF_SLOT_RBF = 1,
  MF_SLOT_TABLES = 2,
  MF_SLOT_EDGES = 3,
  MF_SLOT_VERTS = 4,
  MF_SLOT_CELLS = 5,
  MF_SLOT_SCAN = 6,
  MF_SLOT_MIXED = 7,
  MF_SLOT_CERT = 8,
  MF_SLOT_CELLIDX = 9,
  MF_SLOT_DOMTAB = 10,
  MF_SLOT_BATCH = 11,
  MF_SLOT_SERVER = 12,
  MF_SLOT_VLIST = 13,
  MF_SLOT_SUBDIV = 14,
  MF_SLOT_SORT = 15,
  MF_SLOT_DEFER = 16,
  MF_SLOT_ITEMS = 17,
  MF_NUM_SLOTS = 18
};

// ---------------------------------------------------------------------------
// Double-float arithmetic (a value as an unevaluated sum hi + lo of two
// floats; Dekker 1971, Knuth TAOCP vol. 2 4.2.2): the error-free transforms
// TwoSum and TwoProduct (by FMA) and the usual add / multiply built on them.
// They run on the FP32 pipe; on GB300 it issues about 70 times as many
// operations per clock as the FP64 pipe.
// ---------------------------------------------------------------------------
struct MfDf {
  float hi, lo;
};
// s + e == a + b exactly (any magnitudes)
__device__ __forceinline__ MfDf mf_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// s + e == a + b exactly when |a| >= |b| or a == 0
__device__ __forceinline__ MfDf mf_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
// p + e == a b exactly (barring underflow)
__device__ __forceinline__ MfDf mf_two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
// x + y, relative error below 2^-47 (|x| + |y|)
__device__ __forceinline__ MfDf mf_df_add(MfDf x, MfDf y) {
  const MfDf s = mf_two_sum(x.hi, y.hi);
  return mf_fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
// x y, relative error below 2^-46
__device__ __forceinline__ MfDf mf_df_mul(MfDf x, MfDf y) {
  const MfDf p = mf_two_prod(x.hi, y.hi);
  return mf_fast_two_sum(p.hi, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo)));
}

