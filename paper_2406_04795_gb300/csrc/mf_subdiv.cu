// mf_subdiv.cu -- batch triangulation (Sec. V-B, Figs. 5-6, Eqs. bc and
// local): trace the manifold at the coarse scale k * lambda, then subdivide
// every crossing n-simplex of that trace into the triangulation of scale
// lambda inside it, in batches of n-simplices, and keep the fine edges that
// cross f = 0.
//
// The subdivision of an n-simplex (z, pi) is the same for every one of them
// in local coordinates, so it is enumerated once on the host: the local
// vertices v' with k >= v'_0 >= v'_1 >= ... >= v'_{d-1} >= 0 (Eq. local, read
// as the closed simplex so that the edges on its faces are kept) and the
// local edges (v', M') whose other end v' + e(M') passes the same test.  The
// lattice vertex of v' in the n-simplex (z, pi) is
//   y = k z + sum_j v'_j e(pi_j)                       (Eq. bc, lattice units)
// and the local edge (v', M') is the edge (y, pi(M')).  Because the
// triangulation of scale k lambda is a coarsening of the one of scale lambda
// (same offset), these are edges of the fine triangulation.
//
// A batch runs three kernels over (n-simplex, template entry) items, a warp
// per n-simplex and its lanes over the template:
//   k_sub_vertices  inserts every in-box local vertex into the fine vertex
//                   table (edges on shared faces meet the same vertices, so
//                   f is evaluated once per vertex of the batch);
//   eval            f at the new vertices (FP64, or a mixed path with its
//                   FP64 recheck), the same launchers as mf_trace;
//   k_sub_edges     for every local edge with both vertices in the box and a
//                   sign change, inserts it into the fine edge table (an
//                   edge on a face shared by several n-simplices of the batch
//                   is kept once);
// then the root solve of mf_trace over the batch's edges.  Each batch starts
// from empty fine tables: its memory is bounded by the batch, and an edge on
// a face shared by n-simplices of different batches is reported by each of
// them (the paper's batches also hash within a batch only).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mf_internal.cuh"
#include "mf_ctx.h"

int mf_setup_buffers(mf_ctx *ctx, int d, uint64_t ME, uint64_t MV, uint64_t MC, bool mixed, int n_sv,
                     MfTraceBufs *B);
int mf_build_domain_table(mf_ctx *ctx, MfFrame *F, cudaStream_t st);
int mf_read_counters(mf_ctx *ctx, const MfTraceBufs &B, cudaStream_t st);

#define SUB_WARPS 8

// Lattice vertex of local vertex v' in n-simplex (z, pi): y = k z + sum_j v'_j e(pi_j).
__device__ __forceinline__ void sub_vertex(int d, int k, const int32_t *z, const int *pi,
                                           const uint8_t *v, int32_t *y) {
#pragma unroll
  for (int i = 0; i < MF_MAXD; i++) y[i] = i < d ? k * z[i] : 0;
  for (int j = 0; j < d; j++) y[pi[j]] += (int32_t)v[j];
}

__global__ void __launch_bounds__(SUB_WARPS * 32) k_sub_vertices(MfFrame F, MfTraceBufs B,
                                                                 const int32_t *cell_y,
                                                                 const uint8_t *cell_perm,
                                                                 uint64_t c0, uint64_t nc,
                                                                 const uint8_t *tv, int nv, int k) {
  const int d = F.d, lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * SUB_WARPS;
  for (uint64_t c = (uint64_t)blockIdx.x * SUB_WARPS + (threadIdx.x >> 5); c < nc; c += nwarps) {
    int32_t z[MF_MAXD];
    int pi[MF_MAXD];
#pragma unroll
    for (int i = 0; i < MF_MAXD; i++) {
      z[i] = i < d ? cell_y[(c0 + c) * d + i] : 0;
      pi[i] = i < d ? cell_perm[(c0 + c) * d + i] : 0;
    }
    for (int j = lane; j < nv; j += 32) {
      int32_t y[MF_MAXD];
      sub_vertex(d, k, z, pi, tv + (size_t)j * d, y);
      if (mf_vertex_in(F, y)) mf_visit_vertex(F, B, y);
    }
  }
}

__global__ void __launch_bounds__(SUB_WARPS * 32) k_sub_edges(MfFrame F, MfTraceBufs B,
                                                              const int32_t *cell_y,
                                                              const uint8_t *cell_perm, uint64_t c0,
                                                              uint64_t nc, const uint8_t *tv,
                                                              const uint32_t *te, int ne, int k) {
  const int d = F.d, lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * SUB_WARPS;
  for (uint64_t c = (uint64_t)blockIdx.x * SUB_WARPS + (threadIdx.x >> 5); c < nc; c += nwarps) {
    int32_t z[MF_MAXD];
    int pi[MF_MAXD];
#pragma unroll
    for (int i = 0; i < MF_MAXD; i++) {
      z[i] = i < d ? cell_y[(c0 + c) * d + i] : 0;
      pi[i] = i < d ? cell_perm[(c0 + c) * d + i] : 0;
    }
    for (int j = lane; j < ne; j += 32) {
      const uint32_t code = __ldg(te + j);
      const uint32_t ml = code & 0xFFu;
      int32_t y[MF_MAXD], y2[MF_MAXD];
      sub_vertex(d, k, z, pi, tv + (size_t)(code >> 8) * d, y);
      uint32_t M = 0;
      for (int q = 0; q < d; q++)
        if ((ml >> q) & 1u) M |= 1u << pi[q];
#pragma unroll
      for (int i = 0; i < MF_MAXD; i++) y2[i] = y[i] + (int32_t)((M >> i) & 1u);
      if (!mf_vertex_in(F, y) || !mf_vertex_in(F, y2)) continue;
      const double fa = mf_lookup_f(F, B, y), fb = mf_lookup_f(F, B, y2);
      if ((fa >= 0.0) == (fb >= 0.0)) continue;
      mf_emit_edge(F, B, y, M, fa, fb);
    }
  }
}

// Local triangulation of the subdivided reference n-simplex (host): vertices
// v' of Eq. local in lexicographic order, and the local edges (v', M') with
// both ends inside.
static void local_template(int d, int k, std::vector<uint8_t> &tv, std::vector<uint32_t> &te) {
  tv.clear();
  te.clear();
  std::vector<std::vector<int>> verts;
  std::vector<int> m(d, 0);
  long long total = 1;
  for (int i = 0; i < d; i++) total *= (k + 1);
  auto inside = [&](const std::vector<int> &v) {
    if (v[0] > k) return false;
    for (int i = 1; i < d; i++)
      if (v[i] > v[i - 1]) return false;
    return v[d - 1] >= 0;
  };
  for (long long code = 0; code < total; code++) {
    long long c = code;
    for (int i = d - 1; i >= 0; i--) {
      m[i] = (int)(c % (k + 1));
      c /= (k + 1);
    }
    if (inside(m)) verts.push_back(m);
  }
  for (size_t i = 0; i < verts.size(); i++) {
    for (int q = 0; q < d; q++) tv.push_back((uint8_t)verts[i][q]);
    for (uint32_t M = 1; M < (1u << d); M++) {
      std::vector<int> m2 = verts[i];
      for (int q = 0; q < d; q++) m2[q] += (M >> q) & 1u;
      if (inside(m2)) te.push_back(((uint32_t)i << 8) | M);
    }
  }
}

extern "C" int mf_subdiv_begin(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom,
                               const mf_trace_opts *opts, int32_t k, const double *seeds,
                               int64_t n_seeds, int64_t cells_per_batch, int64_t *n_coarse_cells,
                               void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  ctx->sub.valid = false;
  if (!rbf || !dom || !opts || !n_coarse_cells || k < 1 || k > 16 || cells_per_batch < 0 ||
      !(opts->lambda > 0.0) || !std::isfinite(opts->lambda) || rbf->d < 2 || rbf->d > MF_MAXD)
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_subdiv_begin: bad arguments");
  const int d = rbf->d;
  {
    // local vertices number C(k + d, d); their index must fit 24 bits
    double nv = 1.0;
    for (int i = 1; i <= d; i++) nv = nv * (k + i) / i;
    if (nv > (double)(1 << 23))
      return mf_set_error(ctx, MF_ERR_INVALID, "mf_subdiv_begin: k too large for d");
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  // 1. the coarse trace at k * lambda: its crossing n-simplices
  mf_trace_opts co = *opts;
  co.lambda = k * opts->lambda;
  co.flags = MF_WANT_CELLS;
  mf_trace_out out;
  memset(&out, 0, sizeof(out));
  int rc = mf_trace(ctx, rbf, dom, &co, seeds, n_seeds, &out, stream);
  if (rc) return rc;
  const MfTraceState &L = ctx->last;
  MfSubdivState &S = ctx->sub;
  S.n_cells = L.n_cells;
  S.coarse_levels = L.levels;
  S.dead_seeds = L.n_dead_seeds;
  S.R = L.R;  // prepared support vectors stay in their slot
  // 2. the shared local template
  std::vector<uint8_t> tv;
  std::vector<uint32_t> te;
  local_template(d, k, tv, te);
  S.nv = (int32_t)(tv.size() / d);
  S.ne = (int32_t)te.size();
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t nc = (size_t)S.n_cells;
  const size_t bytes = al(nc * d * 4 + 4) + al(nc * d + 4) + al(tv.size() + 4) + al(te.size() * 4 + 4);
  char *base = (char *)mf_ctx_buffer(ctx, MF_SLOT_SUBDIV, bytes);
  if (!base) return MF_ERR_OOM;
  char *p = base;
  int32_t *cy = (int32_t *)p;
  p += al(nc * d * 4 + 4);
  uint8_t *cp = (uint8_t *)p;
  p += al(nc * d + 4);
  uint8_t *dtv = (uint8_t *)p;
  p += al(tv.size() + 4);
  uint32_t *dte = (uint32_t *)p;
  if (nc) {
    cudaMemcpyAsync(cy, L.B.cell_y, nc * d * 4, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(cp, L.B.cell_perm, nc * d, cudaMemcpyDeviceToDevice, st);
  }
  cudaMemcpyAsync(dtv, tv.data(), tv.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dte, te.data(), te.size() * 4, cudaMemcpyHostToDevice, st);
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_subdiv_begin");
  if (rc) return rc;
  ctx->last.valid = false;  // the trace slots now serve the fine batches
  S.cell_y = cy;
  S.cell_perm = cp;
  S.tv = dtv;
  S.te = dte;
  // 3. the fine frame
  rc = mf_build_frame(ctx, d, opts->lambda, dom, &S.F);
  if (rc) return rc;
  rc = mf_build_domain_table(ctx, &S.F, st);
  if (rc) return rc;
  S.k = k;
  S.precision = opts->precision;
  S.flags = opts->flags & MF_ROOTS_FP64_EXACT ? (MF_WANT_ROOTS | MF_ROOTS_FP64_EXACT)
                                              : (opts->flags & MF_WANT_ROOTS);
  S.band = opts->recheck_band > 0 ? opts->recheck_band : 1e-3;
  S.tol = opts->root_tol > 0 ? opts->root_tol : 1e-12;
  S.ME = opts->max_edges > 0 ? (uint64_t)opts->max_edges : (1ull << 24);
  S.MV = opts->max_vertices > 0 ? (uint64_t)opts->max_vertices : S.ME;
  if (S.ME >= (1ull << 32) || S.MV >= (1ull << 32))
    return mf_set_error(ctx, MF_ERR_INVALID, "max_edges / max_vertices must be < 2^32");
  S.per_batch = cells_per_batch > 0 ? cells_per_batch : (S.n_cells > 0 ? S.n_cells : 1);
  S.next = 0;
  S.valid = true;
  *n_coarse_cells = S.n_cells;
  return MF_OK;
}

extern "C" int mf_subdiv_next(mf_ctx *ctx, mf_trace_out *out, int64_t *cells_left, void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  if (!out || !cells_left) return mf_set_error(ctx, MF_ERR_INVALID, "mf_subdiv_next: bad arguments");
  MfSubdivState &S = ctx->sub;
  if (!S.valid) return mf_set_error(ctx, MF_ERR_INVALID, "mf_subdiv_next: no subdivision in progress");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const MfFrame &F = S.F;
  const int d = F.d, sms = ctx->sms;
  const int64_t c0 = S.next, nb = std::min<int64_t>(S.per_batch, S.n_cells - S.next);
  out->n_edges = out->n_cells = out->n_cell_edges = out->n_vertices = out->n_near_zero = 0;
  out->n_recheck = out->n_boundary = out->root_evals = 0;
  out->levels = S.coarse_levels;
  out->n_dead_seeds = S.dead_seeds;
  *cells_left = S.n_cells - c0;
  if (nb <= 0) return MF_OK;
  const bool mixed = S.precision != MF_FP64;
  MfTraceBufs B;
  int rc = mf_setup_buffers(ctx, d, S.ME, S.MV, 1, mixed, S.R.n, &B);
  if (rc) return rc;
  if (B.vlist) B.list_r2 = mf_list_r2(F, S.R, mixed && !(S.flags & MF_ROOTS_FP64_EXACT));
  B.max_cells = 0;
  cudaMemsetAsync(B.cnt, 0, sizeof(MfCounters), st);
  cudaMemsetAsync(B.etab_key, 0xFF, (B.etab_mask + 1) * 16, st);
  cudaMemsetAsync(B.vtab_key, 0xFF, (B.vtab_mask + 1) * 16, st);
  const unsigned grid = (unsigned)std::min<int64_t>((nb + SUB_WARPS - 1) / SUB_WARPS, (int64_t)sms * 16);
  {
    MfProfScope ps(ctx, MF_PH_EXPAND_V, st, 1, nb);
    k_sub_vertices<<<grid, SUB_WARPS * 32, 0, st>>>(F, B, S.cell_y, S.cell_perm, (uint64_t)c0,
                                                    (uint64_t)nb, S.tv, S.nv, S.k);
  }
  {
    MfProfScope ps(ctx, MF_PH_EVAL, st, mixed ? (B.vlist ? 4 : 3) : 2);
    if (mixed) mf_launch_eval_vertices_mixed(F, S.R, B, S.precision, S.band, ctx->tune, sms, st);
    else mf_launch_eval_vertices_f64(F, S.R, B, ctx->tune, sms, st);
  }
  {
    MfProfScope ps(ctx, MF_PH_EXPAND_E, st, 1, nb);
    k_sub_edges<<<grid, SUB_WARPS * 32, 0, st>>>(F, B, S.cell_y, S.cell_perm, (uint64_t)c0,
                                                 (uint64_t)nb, S.tv, S.te, S.ne, S.k);
  }
  rc = mf_cuda_check(ctx, cudaGetLastError(), "subdivision kernels");
  if (rc) return rc;
  rc = mf_read_counters(ctx, B, st);
  if (rc) return rc;
  const uint64_t E = ctx->h_counters->n_edges;
  if (S.flags & MF_WANT_ROOTS) {
    MfProfScope ps(ctx, MF_PH_ROOTS, st, E > 0 ? 1 : 0, (int64_t)E);
    mf_launch_roots_f64(F, S.R, B, E, S.tol, ctx->tune, sms, st,
                        mixed && !(S.flags & MF_ROOTS_FP64_EXACT));
  }
  rc = mf_read_counters(ctx, B, st);
  if (rc) return rc;
  const MfCounters &h = *ctx->h_counters;
  out->n_edges = (int64_t)E;
  out->n_vertices = (int64_t)h.n_vertices;
  out->n_near_zero = (int64_t)h.n_near_zero;
  out->n_recheck = (int64_t)h.n_recheck;
  out->root_evals = (int64_t)h.root_evals;
  if (ctx->prof.on) {
    ctx->prof.stats.terms[MF_PH_EVAL] += (int64_t)h.eval_terms;
    ctx->prof.stats.terms[MF_PH_ROOTS] += (int64_t)h.root_terms;
    ctx->prof.stats.terms_weak[MF_PH_EVAL] += (int64_t)h.eval_terms_weak;
    ctx->prof.stats.terms_weak[MF_PH_ROOTS] += (int64_t)h.root_terms_weak;
  }
  if (out->cap_edges < out->n_edges && (out->edge_y || out->edge_mask || out->edge_f ||
                                        out->edge_t || out->points))
    return mf_set_error(ctx, MF_ERR_CAPACITY, "output buffers too small: need %lld edges",
                        (long long)E);
  {
    MfProfScope ps(ctx, MF_PH_COPY, st, 0);
    auto cp = [&](void *dst, const void *src, size_t bytes) {
      if (dst && bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
    };
    cp(out->edge_y, B.edge_y, E * d * 4);
    cp(out->edge_mask, B.edge_mask, E * 4);
    cp(out->edge_f, B.edge_f, E * 16);
    if (S.flags & MF_WANT_ROOTS) {
      cp(out->edge_t, B.edge_t, E * 8);
      cp(out->points, B.edge_pt, E * d * 8);
    }
    rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "subdivision copy");
  }
  mf_prof_collect(ctx);
  if (rc) return rc;
  S.next = c0 + nb;
  *cells_left = S.n_cells - S.next;
  return MF_OK;
}
