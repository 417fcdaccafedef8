// mf_batch.cu -- many independent traces in one launch (batched multi-trace).
//
// Every trace of a batch gets a slot: its frame, prepared support vectors,
// tables and lists, carved from one context arena.  The breadth-first search
// of all slots runs as ONE CUDA-graph launch: a conditional WHILE node whose
// body is one step of every active trace (expand vertices, evaluate f,
// expand edges, advance cursors); the last kernel of the body clears the
// loop condition once no trace is active.  Work items of all traces share
// each kernel: a trace id comes from a prefix over the slots, so uneven
// traces (different d, support vectors, lambda, precision) fill the GPU
// together.  Roots, cells and the CSR then run batched the same way.
#include <cmath>
#include <cstring>
#include <vector>

#include "mf_internal.cuh"
#include "mf_ctx.h"

bool mf_domain_table_host(MfFrame *F, std::vector<int2> &tab);

namespace {

struct Bump {
  size_t off = 0;
  size_t take(size_t bytes) {
    off = (off + 255) & ~(size_t)255;
    const size_t r = off;
    off += bytes;
    return r;
  }
};

struct TraceLayout {
  size_t rbf, dom, cnt, etab_key, vtab_key;
  size_t edge_y, edge_mask, edge_f, edge_t, edge_pt, vert_y, vert_slot, recheck;
  size_t cell_y, cell_perm, cell_sgn, cell_off, scan;
  size_t items, item_off;
  uint64_t IC;
  size_t vtab_idx, vlist_off, vlist_n, vlist;  // root-screen lists (0 bytes: none)
  uint64_t ME, MV, MC, TE, TV, VL;
  std::vector<int2> tab;
};

// One step of every active trace (captured into the graph's loop body).
void launch_step(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n, bool any_mixed,
                 int tc_chunk, int sms, cudaGraphConditionalHandle h, int use_handle,
                 cudaStream_t s) {
  mf_b_launch_expand(slots, st, P, n, false, sms, s);
  mf_b_launch_eval(slots, P, n, any_mixed, tc_chunk, sms, s);
  mf_b_launch_expand(slots, st, P, n, true, sms, s);
  mf_b_launch_update(slots, st, P, n, h, use_handle, s);
}

// Builds the search loop: a graph whose conditional WHILE node has one step of
// every slot as its body (k_b_update clears the condition when no slot is
// active or the plan's step budget is used up).  nullptr if unavailable.
cudaGraphExec_t build_loop(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n,
                           bool any_mixed, int tc_chunk, int sms) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  do {
    if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
    // the node-parameter union has no default constructor in C++: zeroed storage
    alignas(cudaGraphNodeParams) unsigned char storage[sizeof(cudaGraphNodeParams)];
    memset(storage, 0, sizeof(storage));
    cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(storage);
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p) != cudaSuccess) break;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) break;
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    launch_step(slots, st, P, n, any_mixed, tc_chunk, sms, h, 1, cs);
    cudaGraph_t captured = nullptr;
    if (cudaStreamEndCapture(cs, &captured) != cudaSuccess) break;
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
  } while (false);
  if (!exec) cudaGetLastError();
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  return exec;
}

// Runs the BFS of all slots as one launch of the search loop.  Returns false
// if the graph could not be built (the caller falls back to host steps).
bool run_graph(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n, bool any_mixed,
               int tc_chunk, int sms, cudaStream_t s) {
  cudaGraphExec_t exec = build_loop(slots, st, P, n, any_mixed, tc_chunk, sms);
  if (!exec) return false;
  bool ok = cudaGraphLaunch(exec, s) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) cudaGetLastError();
  cudaGraphExecDestroy(exec);
  return ok;
}

}  // namespace

// Frame, domain table and the byte layout of one trace's buffers (offsets
// taken from `bump`, relative to the base later given to mf_setup_trace).
int mf_layout_trace(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom, const mf_trace_opts *o,
                    MfSlot *S, TraceLayout *l, Bump *bump) {
  const mf_rbf &r = *rbf;
  if (r.d < 2 || r.d > MF_MAXD || r.n_sv < 1 || !(o->lambda > 0.0) || !std::isfinite(o->lambda) ||
      (o->precision != MF_FP64 && o->precision != MF_MIXED_FP32 && o->precision != MF_MIXED_BF16))
    return mf_set_error(ctx, MF_ERR_INVALID, "bad trace arguments");
  if (o->flags & MF_SORT_OUTPUT)
    return mf_set_error(ctx, MF_ERR_INVALID, "MF_SORT_OUTPUT is for mf_trace only");
  memset(S, 0, sizeof(*S));
  int rc = mf_build_frame(ctx, r.d, o->lambda, dom, &S->F);
  if (rc) return rc;
  if (!mf_domain_table_host(&S->F, l->tab)) l->tab.clear();
  const int d = r.d;
  l->ME = o->max_edges > 0 ? (uint64_t)o->max_edges : (1ull << 20);
  l->MV = o->max_vertices > 0 ? (uint64_t)o->max_vertices : l->ME;
  l->MC = o->max_cells > 0 ? (uint64_t)o->max_cells : 2 * l->ME;
  if (l->ME >= (1ull << 32) || l->MV >= (1ull << 32))
    return mf_set_error(ctx, MF_ERR_INVALID, "max_edges / max_vertices must be < 2^32");
  l->TE = mf_next_pow2(l->ME + l->ME / 3 + 1);
  l->TV = mf_next_pow2(l->MV + l->MV / 3 + 1);
  l->rbf = bump->take(mf_rbf_prep_bytes(d, r.n_sv));
  l->dom = bump->take(l->tab.size() * sizeof(int2) + 8);
  l->cnt = bump->take(sizeof(MfCounters));
  l->etab_key = bump->take(l->TE * 16);
  l->vtab_key = bump->take(l->TV * 16);
  l->edge_y = bump->take(l->ME * d * 4);
  l->edge_mask = bump->take(l->ME * 4);
  l->edge_f = bump->take(l->ME * 16);
  l->edge_t = bump->take(l->ME * 8);
  l->edge_pt = bump->take(l->ME * d * 8);
  // the expansion's vertex slots (16 items per edge on average; an edge
  // whose items do not fit looks its vertices up) and each edge's first item
  l->IC = l->ME * 16;
  l->items = bump->take(l->IC * 4 + 8);
  l->item_off = bump->take(l->ME * 8 + 8);
  l->vert_y = bump->take(l->MV * d * 4);
  l->vert_slot = bump->take(l->MV * 4);
  l->recheck = bump->take(l->MV * 4);
  const uint64_t mc = (o->flags & MF_WANT_CELLS) ? l->MC : 0;
  l->cell_y = bump->take(mc * d * 4 + 8);
  l->cell_perm = bump->take(mc * d + 8);
  l->cell_sgn = bump->take(mc * 4 + 8);
  l->cell_off = bump->take((mc + 1) * 8);
  l->scan = bump->take((mc / 4096 + 2) * 8);
  // root-screen lists: up to min(n_sv, 128) vectors per vertex on average;
  // vertices past the pool screen the vector blocks instead
  l->VL = (o->flags & MF_WANT_ROOTS) ? l->MV * (uint64_t)(r.n_sv < 128 ? r.n_sv : 128) : 0;
  l->vtab_idx = bump->take(l->VL ? l->TV * 4 : 8);
  l->vlist_off = bump->take(l->VL ? l->MV * 8 : 8);
  l->vlist_n = bump->take(l->VL ? l->MV * 4 : 8);
  l->vlist = bump->take(l->VL * 4 + 8);
  return MF_OK;
}

// Prepares the support vectors, uploads the domain table, points the slot's
// buffers into base + the layout's offsets, and clears counters and tables.
int mf_setup_trace(mf_ctx *ctx, const mf_rbf *rbf, const mf_trace_opts *o, char *base,
                   TraceLayout *l, MfSlot *S, cudaStream_t st) {
  int rc = mf_prepare_rbf_at(ctx, rbf, base + l->rbf, &S->R, st);
  if (rc) return rc;
  if (!l->tab.empty()) {
    rc = mf_cuda_check(ctx, cudaMemcpyAsync(base + l->dom, l->tab.data(), l->tab.size() * sizeof(int2),
                                            cudaMemcpyHostToDevice, st),
                       "domain table");
    if (rc) return rc;
    S->F.dom_tab = (const int2 *)(base + l->dom);
  }
  MfTraceBufs &B = S->B;
  B.cnt = (MfCounters *)(base + l->cnt);
  B.etab_key = (unsigned long long *)(base + l->etab_key);
  B.etab_mask = l->TE - 1;
  B.vtab_key = (unsigned long long *)(base + l->vtab_key);
  B.vtab_mask = l->TV - 1;
  B.edge_y = (int32_t *)(base + l->edge_y);
  B.edge_mask = (uint32_t *)(base + l->edge_mask);
  B.edge_f = (double *)(base + l->edge_f);
  B.edge_t = (double *)(base + l->edge_t);
  B.edge_pt = (double *)(base + l->edge_pt);
  B.max_edges = l->ME;
  B.item_slot = (uint32_t *)(base + l->items);
  B.edge_item_off = (unsigned long long *)(base + l->item_off);
  B.item_cap = l->IC;
  B.vert_y = (int32_t *)(base + l->vert_y);
  B.vert_slot = (uint32_t *)(base + l->vert_slot);
  B.recheck = (uint32_t *)(base + l->recheck);
  B.max_vertices = l->MV;
  B.cell_y = (int32_t *)(base + l->cell_y);
  B.cell_perm = (uint8_t *)(base + l->cell_perm);
  B.cell_sgn = (uint32_t *)(base + l->cell_sgn);
  B.cell_off = (int64_t *)(base + l->cell_off);
  B.max_cells = (o->flags & MF_WANT_CELLS) ? l->MC : 0;
  if (l->VL) {
    B.vtab_idx = (uint32_t *)(base + l->vtab_idx);
    B.vlist_off = (uint64_t *)(base + l->vlist_off);
    B.vlist_n = (uint32_t *)(base + l->vlist_n);
    B.vlist = (int32_t *)(base + l->vlist);
    B.vlist_cap = l->VL;
    B.list_r2 = mf_list_r2(S->F, S->R, o->precision != MF_FP64 && !(o->flags & MF_ROOTS_FP64_EXACT));
  } else {  // no per-vertex lists: the root screen scans the blocks
    B.vtab_idx = nullptr;
    B.vlist = nullptr;
    B.vlist_off = nullptr;
    B.vlist_n = nullptr;
    B.vlist_cap = 0;
    B.list_r2 = 0.f;
  }
  S->precision = o->precision;
  S->band = o->recheck_band > 0 ? o->recheck_band : 1e-3;
  S->root_tol = o->root_tol > 0 ? o->root_tol : 1e-12;
  S->cap = o->batch_cap_edges > 0 ? (uint64_t)o->batch_cap_edges : (1ull << 24);
  S->flags = o->flags;
  cudaMemsetAsync(B.cnt, 0, sizeof(MfCounters), st);
  cudaMemsetAsync(B.etab_key, 0xFF, l->TE * 16, st);
  cudaMemsetAsync(B.vtab_key, 0xFF, l->TV * 16, st);
  return MF_OK;
}

extern "C" int mf_trace_batch(mf_ctx *ctx, int32_t n, const mf_rbf *rbfs, const mf_domain *doms,
                              const mf_trace_opts *opts, const double *const *seeds,
                              const int64_t *n_seeds, mf_trace_out *outs, void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  if (n < 1 || n > MF_MAX_SLOTS || !rbfs || !doms || !opts || !seeds || !n_seeds || !outs)
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_trace_batch: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int sms = ctx->sms;
  // --- layout of every trace in one arena
  std::vector<TraceLayout> L(n);
  std::vector<MfSlot> slots(n);
  Bump bump;
  bool any_mixed = false;
  for (int t = 0; t < n; t++) {
    if (n_seeds[t] < 0 || (n_seeds[t] > 0 && !seeds[t]))
      return mf_set_error(ctx, MF_ERR_INVALID, "mf_trace_batch: bad seeds for trace %d", t);
    int rc = mf_layout_trace(ctx, &rbfs[t], &doms[t], &opts[t], &slots[t], &L[t], &bump);
    if (rc) return rc;
    if (opts[t].precision != MF_FP64) any_mixed = true;
  }
  const size_t off_slots = bump.take(sizeof(MfSlot) * n);
  const size_t off_state = bump.take(sizeof(MfSlotState) * n);
  const size_t off_plan = bump.take(sizeof(MfBatchPlan));
  char *arena = (char *)mf_ctx_buffer(ctx, MF_SLOT_BATCH, bump.off);
  if (!arena) return MF_ERR_OOM;
  MfSlot *d_slots = (MfSlot *)(arena + off_slots);
  MfSlotState *d_state = (MfSlotState *)(arena + off_state);
  MfBatchPlan *d_plan = (MfBatchPlan *)(arena + off_plan);
  cudaMemsetAsync(d_plan, 0, sizeof(MfBatchPlan), st);
  int rc;
  // --- per-trace preparation (support vectors, domain tables, tables)
  for (int t = 0; t < n; t++) {
    rc = mf_setup_trace(ctx, &rbfs[t], &opts[t], arena, &L[t], &slots[t], st);
    if (rc) return rc;
  }
  rc = mf_cuda_check(ctx, cudaMemcpyAsync(d_slots, slots.data(), sizeof(MfSlot) * n,
                                          cudaMemcpyHostToDevice, st),
                     "batch slots");
  if (rc) return rc;
  // --- locate edges (Fig. 3) of every trace; one batched evaluation
  {
    MfProfScope ps(ctx, MF_PH_SEEDS, st, 2 * n + 5);
    for (int t = 0; t < n; t++)
      if (n_seeds[t] > 0) mf_launch_seeds(slots[t].F, slots[t].B, seeds[t], n_seeds[t], true, st);
    mf_b_launch_eval(d_slots, d_plan, n, any_mixed, ctx->tune.tc_chunk, sms, st);
    for (int t = 0; t < n; t++)
      if (n_seeds[t] > 0) mf_launch_seeds(slots[t].F, slots[t].B, seeds[t], n_seeds[t], false, st);
    mf_b_launch_init(d_slots, d_state, n, st);
  }
  rc = mf_cuda_check(ctx, cudaGetLastError(), "batch seeds");
  if (rc) return rc;
  // --- search edges (Fig. 4) of all traces: one graph launch
  {
    MfProfScope ps(ctx, MF_PH_EXPAND_V, st, 1, n);
    if (!run_graph(d_slots, d_state, d_plan, n, any_mixed, ctx->tune.tc_chunk, sms, st)) {
      // host-driven steps (same kernels) when conditional graphs are unavailable
      std::vector<MfSlotState> hs(n);
      for (long it = 0; it < (1l << 24); it++) {
        cudaGraphConditionalHandle none = 0;
        launch_step(d_slots, d_state, d_plan, n, any_mixed, ctx->tune.tc_chunk, sms, none, 0, st);
        rc = mf_cuda_check(ctx, cudaMemcpyAsync(hs.data(), d_state, sizeof(MfSlotState) * n,
                                                cudaMemcpyDeviceToHost, st),
                           "batch state");
        if (rc) return rc;
        rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "batch step");
        if (rc) return rc;
        bool any = false;
        for (int t = 0; t < n; t++) any = any || hs[t].active;
        if (!any) break;
      }
    }
  }
  std::vector<MfSlotState> hs(n);
  rc = mf_cuda_check(ctx, cudaMemcpyAsync(hs.data(), d_state, sizeof(MfSlotState) * n,
                                          cudaMemcpyDeviceToHost, st),
                     "batch state");
  if (rc) return rc;
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "batch search");
  if (rc) return rc;
  for (int t = 0; t < n; t++)
    if (hs[t].err)
      return mf_set_error(ctx, MF_ERR_MAXEDGES, "trace %d exceeded its capacities or a table", t);
  // --- roots and cells of all traces
  {
    MfProfScope ps(ctx, MF_PH_ROOTS, st, 2);
    uint32_t dims = 0;
    for (int t = 0; t < n; t++) dims |= 1u << slots[t].F.d;
    mf_b_launch_roots(d_slots, d_plan, n, nullptr, dims, ctx->tune.roots_group, sms, st);
  }
  bool any_cells = false;
  for (int t = 0; t < n; t++) any_cells = any_cells || (opts[t].flags & MF_WANT_CELLS);
  std::vector<MfCounters> hc(n);
  std::vector<int64_t> n_cells(n, 0), n_ce(n, 0);
  if (any_cells) {
    {
      MfProfScope ps(ctx, MF_PH_CELLS, st, 2);
      mf_b_launch_cells(d_slots, d_plan, n, nullptr, sms, st);
    }
    for (int t = 0; t < n; t++)
      cudaMemcpyAsync(&hc[t], slots[t].B.cnt, sizeof(MfCounters), cudaMemcpyDeviceToHost, st);
    rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "batch cells");
    if (rc) return rc;
    for (int t = 0; t < n; t++) {
      if (hc[t].err_table_full || hc[t].err_overflow || hc[t].n_cells > slots[t].B.max_cells)
        return mf_set_error(ctx, MF_ERR_MAXEDGES, "trace %d: cells exceed capacity", t);
      n_cells[t] = (opts[t].flags & MF_WANT_CELLS) ? (int64_t)hc[t].n_cells : 0;
    }
    {
      MfProfScope ps(ctx, MF_PH_CSR, st, 2 + 3 * n);
      mf_b_launch_cell_edges(d_slots, d_plan, n, false, nullptr, sms, st);
      for (int t = 0; t < n; t++)
        if (n_cells[t] > 0)
          mf_exclusive_scan(slots[t].B.cell_off, slots[t].B.cell_off, n_cells[t],
                            (int64_t *)(arena + L[t].scan), st);
      for (int t = 0; t < n; t++)
        if (n_cells[t] > 0)
          cudaMemcpyAsync(&n_ce[t], slots[t].B.cell_off + n_cells[t], 8, cudaMemcpyDeviceToHost, st);
    }
    rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "batch CSR counts");
    if (rc) return rc;
    size_t total_ce = 0;
    std::vector<size_t> ce_off(n);
    for (int t = 0; t < n; t++) {
      ce_off[t] = total_ce;
      total_ce += ((size_t)n_ce[t] * 8 + 255) & ~(size_t)255;
    }
    char *idx = (char *)mf_ctx_buffer(ctx, MF_SLOT_CELLIDX, total_ce + 256);
    if (!idx) return MF_ERR_OOM;
    for (int t = 0; t < n; t++) slots[t].B.cell_idx = (int64_t *)(idx + ce_off[t]);
    rc = mf_cuda_check(ctx, cudaMemcpyAsync(d_slots, slots.data(), sizeof(MfSlot) * n,
                                            cudaMemcpyHostToDevice, st),
                       "batch slots");
    if (rc) return rc;
    {
      MfProfScope ps(ctx, MF_PH_CSR, st, 1);
      mf_b_launch_cell_edges(d_slots, d_plan, n, true, nullptr, sms, st);
    }
  }
  for (int t = 0; t < n; t++)
    cudaMemcpyAsync(&hc[t], slots[t].B.cnt, sizeof(MfCounters), cudaMemcpyDeviceToHost, st);
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "batch results");
  if (rc) return rc;
  // --- results into the callers' buffers
  int result = MF_OK;
  {
    MfProfScope ps(ctx, MF_PH_COPY, st, 0);
    for (int t = 0; t < n; t++) {
      const MfCounters &h = hc[t];
      const MfTraceBufs &B = slots[t].B;
      mf_trace_out &o = outs[t];
      const int d = rbfs[t].d;
      const size_t E = (size_t)(h.n_edges < B.max_edges ? h.n_edges : B.max_edges);
      o.n_edges = (int64_t)E;
      o.n_cells = n_cells[t];
      o.n_cell_edges = n_ce[t];
      o.n_vertices = (int64_t)h.n_vertices;
      o.n_near_zero = (int64_t)h.n_near_zero;
      o.n_recheck = (int64_t)h.n_recheck;
      o.n_boundary = (int64_t)h.n_boundary;
      o.n_dead_seeds = (int64_t)h.n_dead_seeds;
      o.levels = hs[t].levels;
      o.root_evals = (int64_t)h.root_evals;
      const bool small = o.cap_edges < o.n_edges ||
                         ((opts[t].flags & MF_WANT_CELLS) &&
                          (o.cap_cells < o.n_cells ||
                           (o.cell_edge_idx && o.cap_cell_edges < o.n_cell_edges)));
      if (small) {
        result = mf_set_error(ctx, MF_ERR_CAPACITY, "trace %d: output buffers too small", t);
        continue;
      }
      auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (dst && bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
      };
      cp(o.edge_y, B.edge_y, E * d * 4);
      cp(o.edge_mask, B.edge_mask, E * 4);
      cp(o.edge_f, B.edge_f, E * 16);
      if (opts[t].flags & MF_WANT_ROOTS) {
        cp(o.edge_t, B.edge_t, E * 8);
        cp(o.points, B.edge_pt, E * d * 8);
      }
      if (opts[t].flags & MF_WANT_CELLS) {
        const size_t C = (size_t)n_cells[t];
        cp(o.cell_y, B.cell_y, C * d * 4);
        cp(o.cell_perm, B.cell_perm, C * d);
        cp(o.cell_edge_off, B.cell_off, (C + 1) * 8);
        cp(o.cell_edge_idx, B.cell_idx, (size_t)n_ce[t] * 8);
      }
    }
  }
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "batch copy out");
  if (rc) return rc;
  mf_prof_collect(ctx);
  return result;
}

// ===========================================================================
// Proof server: continuous batching of tracing requests.
//
// The server owns an HBM arena (its budget) and up to max_slots slots.  A
// submitted request waits in a FIFO queue until a slot is free AND its
// buffers (sized from its capacities) fit a free range of the arena
// (first-fit with coalescing): that is the admission by HBM.  Every
// mf_server_step admits what fits, seeds the new traces, runs ONE
// breadth-first step of every running trace (a captured CUDA graph replayed
// each step), and finishes the traces whose search ended (roots, cells and
// CSR batched over just those slots).  A finished request keeps its slot and
// memory until mf_server_fetch copies its results out.
// ===========================================================================
#include <chrono>
#include <deque>
#include <map>
#include <unordered_map>

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing of freed ranges.
struct RangeAlloc {
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t size) { free_.clear(); free_[0] = size; }
  bool take(size_t bytes, size_t *off) {
    bytes = (bytes + 255) & ~(size_t)255;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void give(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Request {
  mf_rbf rbf;
  mf_domain dom;
  mf_trace_opts opts;
  const double *seeds = nullptr;
  int64_t n_seeds = 0;
  int state = 0;  // 0 queued, 1 running, 2 done, < 0 error code
  int slot = -1;
  size_t off = 0, bytes = 0, idx_off = 0, idx_bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  MfCounters cnt;
  int64_t n_cells = 0, n_ce = 0, levels = 0;
  MfSlot S;  // the descriptor of a finished trace: its results until fetched
  int64_t id = 0;
  bool wait_idx = false;  // cells counted, waiting for arena room for the CSR index
};

}  // namespace

struct mf_server {
  mf_ctx *ctx = nullptr;
  int max_slots = 0;
  char *arena = nullptr;
  size_t arena_bytes = 0, data_off = 0;
  RangeAlloc alloc;
  MfSlot *d_slots = nullptr;
  MfSlotState *d_state = nullptr;
  MfBatchPlan *d_plan = nullptr;
  int32_t *d_only = nullptr;
  std::vector<MfSlot> slots;
  std::vector<int64_t> slot_req;
  std::vector<MfSlotState> hstate;
  std::deque<int64_t> queue;
  std::deque<int64_t> finished;  // done or failed, not yet reported by mf_server_done
  std::unordered_map<int64_t, Request> reqs;
  int64_t next_id = 1;
  cudaGraphExec_t step_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  int tc_chunk = 64;  // tensor-core chunk width the step graph was built with
};

extern "C" int mf_server_create(mf_ctx *ctx, int32_t max_slots, size_t hbm_bytes, mf_server **out) {
  if (!ctx || !out || max_slots < 1 || max_slots > MF_MAX_SLOTS)
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_server_create: bad arguments");
  cudaSetDevice(ctx->device);
  mf_server *s = new mf_server();
  s->ctx = ctx;
  s->max_slots = max_slots;
  Bump b;
  const size_t o_slots = b.take(sizeof(MfSlot) * max_slots);
  const size_t o_state = b.take(sizeof(MfSlotState) * max_slots);
  const size_t o_plan = b.take(sizeof(MfBatchPlan));
  const size_t o_only = b.take(sizeof(int32_t) * max_slots);
  s->data_off = (b.off + 255) & ~(size_t)255;
  if (hbm_bytes <= s->data_off + (1 << 20)) {
    delete s;
    return mf_set_error(ctx, MF_ERR_OOM, "mf_server_create: budget too small");
  }
  s->arena = (char *)mf_ctx_buffer(ctx, MF_SLOT_SERVER, hbm_bytes);
  if (!s->arena) {
    delete s;
    return MF_ERR_OOM;
  }
  s->arena_bytes = hbm_bytes;
  s->d_slots = (MfSlot *)(s->arena + o_slots);
  s->d_state = (MfSlotState *)(s->arena + o_state);
  s->d_plan = (MfBatchPlan *)(s->arena + o_plan);
  s->d_only = (int32_t *)(s->arena + o_only);
  s->alloc.init(hbm_bytes - s->data_off);
  s->slots.assign(max_slots, MfSlot());
  memset(s->slots.data(), 0, sizeof(MfSlot) * max_slots);
  s->slot_req.assign(max_slots, -1);
  s->hstate.assign(max_slots, MfSlotState());
  cudaMemset(s->d_slots, 0, sizeof(MfSlot) * max_slots);
  cudaMemset(s->d_state, 0, sizeof(MfSlotState) * max_slots);
  // the search loop of every slot as one graph, replayed by each
  // mf_server_step for up to MF_SERVER_STEPS breadth-first steps
  s->step_exec = build_loop(s->d_slots, s->d_state, s->d_plan, max_slots, true,
                            ctx->tune.tc_chunk, ctx->sms);
  s->tc_chunk = ctx->tune.tc_chunk;
  cudaGetLastError();
  if (cudaDeviceSynchronize() != cudaSuccess) {
    mf_server_destroy(s);
    return mf_set_error(ctx, MF_ERR_CUDA, "mf_server_create failed");
  }
  *out = s;
  return MF_OK;
}

extern "C" void mf_server_destroy(mf_server *s) {
  if (!s) return;
  cudaSetDevice(s->ctx->device);
  cudaDeviceSynchronize();
  if (s->step_exec) cudaGraphExecDestroy(s->step_exec);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  delete s;
}

extern "C" int mf_server_submit(mf_server *s, const mf_rbf *rbf, const mf_domain *dom,
                                const mf_trace_opts *opts, const double *seeds, int64_t n_seeds,
                                int64_t *id) {
  if (!s || !rbf || !dom || !opts || !id || n_seeds < 0 || (n_seeds > 0 && !seeds))
    return mf_set_error(s ? s->ctx : nullptr, MF_ERR_INVALID, "mf_server_submit: bad arguments");
  Request r;
  r.rbf = *rbf;
  r.dom = *dom;
  r.opts = *opts;
  r.seeds = seeds;
  r.n_seeds = n_seeds;
  r.t_submit = now_s();
  memset(&r.cnt, 0, sizeof(r.cnt));
  *id = s->next_id++;
  r.id = *id;
  s->reqs[*id] = r;
  s->queue.push_back(*id);
  return MF_OK;
}

// A finished or failed trace gives its slot back at once: the descriptor is
// zeroed on the host and (stream-ordered) on the device, and every per-slot
// kernel skips empty descriptors.  Its memory stays taken until fetched.
static void free_slot(mf_server *s, Request &r, cudaStream_t st) {
  if (r.slot < 0) return;
  memset(&s->slots[r.slot], 0, sizeof(MfSlot));
  cudaMemsetAsync(s->d_slots + r.slot, 0, sizeof(MfSlot), st);
  cudaMemsetAsync(s->d_state + r.slot, 0, sizeof(MfSlotState), st);
  s->slot_req[r.slot] = -1;
  r.slot = -1;
}

static void free_memory(mf_server *s, Request &r) {
  if (r.bytes) s->alloc.give(r.off, r.bytes);
  if (r.idx_bytes) s->alloc.give(r.idx_off, r.idx_bytes);
  r.bytes = r.idx_bytes = 0;
}

static void fail(mf_server *s, Request &r, int code, cudaStream_t st) {
  r.state = code;
  free_slot(s, r, st);
  free_memory(s, r);
  s->finished.push_back(r.id);
}

extern "C" int mf_server_step(mf_server *s, void *stream, int32_t *n_running, int32_t *n_queued) {
  if (!s) return MF_ERR_INVALID;
  mf_ctx *ctx = s->ctx;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int n = s->max_slots, sms = ctx->sms;
  int rc;
  // --- finish traces that waited for room for their CSR index
  {
    std::vector<int32_t> only(n, 0);
    std::vector<int> ready;
    for (int t = 0; t < n; t++) {
      if (s->slot_req[t] < 0) continue;
      Request &r = s->reqs[s->slot_req[t]];
      if (!r.wait_idx) continue;
      size_t off;
      if (!s->alloc.take((size_t)r.n_ce * 8, &off)) continue;
      r.idx_off = off;
      r.idx_bytes = (size_t)r.n_ce * 8;
      s->slots[t].B.cell_idx = (int64_t *)(s->arena + s->data_off + off);
      cudaMemcpyAsync(s->d_slots + t, &s->slots[t], sizeof(MfSlot), cudaMemcpyHostToDevice, st);
      only[t] = 1;
      ready.push_back(t);
    }
    if (!ready.empty()) {
      cudaMemcpyAsync(s->d_only, only.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
      mf_b_launch_plan_edges(s->d_slots, s->d_plan, n, 1, s->d_only, st);
      mf_b_launch_cell_edges(s->d_slots, s->d_plan, n, true, s->d_only, sms, st);
      for (int t : ready)
        cudaMemcpyAsync(&s->reqs[s->slot_req[t]].cnt, s->slots[t].B.cnt, sizeof(MfCounters),
                        cudaMemcpyDeviceToHost, st);
      if ((rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "server CSR fill"))) return rc;
      const double tnow = now_s();
      for (int t : ready) {
        Request &r = s->reqs[s->slot_req[t]];
        r.wait_idx = false;
        r.levels = s->hstate[t].levels;
        r.state = 2;
        r.t_done = tnow;
        s->finished.push_back(r.id);
        r.S = s->slots[t];
        free_slot(s, r, st);
      }
    }
  }
  // --- admission: FIFO, while a slot is free and the request's buffers fit
  std::vector<int> fresh;
  while (!s->queue.empty()) {
    int t = -1;
    for (int k = 0; k < n; k++)
      if (s->slot_req[k] < 0) { t = k; break; }
    if (t < 0) break;
    const int64_t id = s->queue.front();
    Request &r = s->reqs[id];
    TraceLayout l;
    MfSlot S;
    Bump b;
    rc = mf_layout_trace(ctx, &r.rbf, &r.dom, &r.opts, &S, &l, &b);
    if (rc) {  // a malformed request fails alone
      r.state = rc;
      s->finished.push_back(id);
      s->queue.pop_front();
      continue;
    }
    size_t off;
    if (!s->alloc.take(b.off, &off)) {
      if (b.off > s->arena_bytes - s->data_off) {  // can never fit
        r.state = mf_set_error(ctx, MF_ERR_OOM, "request %lld exceeds the server budget", (long long)id);
        s->finished.push_back(id);
        s->queue.pop_front();
        continue;
      }
      break;  // wait for memory
    }
    rc = mf_setup_trace(ctx, &r.rbf, &r.opts, s->arena + s->data_off + off, &l, &S, st);
    if (rc) {
      s->alloc.give(off, b.off);
      r.state = rc;
      s->finished.push_back(id);
      s->queue.pop_front();
      continue;
    }
    r.off = off;
    r.bytes = b.off;
    r.slot = t;
    r.state = 1;
    r.t_admit = now_s();
    s->slots[t] = S;
    s->slot_req[t] = id;
    cudaMemcpyAsync(s->d_slots + t, &s->slots[t], sizeof(MfSlot), cudaMemcpyHostToDevice, st);
    fresh.push_back(t);
    s->queue.pop_front();
  }
  if (!fresh.empty()) {
    for (int t : fresh) {
      const Request &r = s->reqs[s->slot_req[t]];
      if (r.n_seeds > 0) mf_launch_seeds(s->slots[t].F, s->slots[t].B, r.seeds, r.n_seeds, true, st);
    }
    mf_b_launch_eval(s->d_slots, s->d_plan, n, true, s->tc_chunk, sms, st);
    for (int t : fresh) {
      const Request &r = s->reqs[s->slot_req[t]];
      if (r.n_seeds > 0) mf_launch_seeds(s->slots[t].F, s->slots[t].B, r.seeds, r.n_seeds, false, st);
      mf_b_launch_init(s->d_slots + t, s->d_state + t, 1, st);
    }
  }
  // --- one breadth-first step of every running trace
  bool running = false;
  for (int t = 0; t < n; t++)
    if (s->slot_req[t] >= 0 && s->reqs[s->slot_req[t]].state == 1) running = true;
  if (running) {
    // the step count restarts per call; the loop pauses after the budget
    static const int32_t budget = MF_SERVER_STEPS;
    cudaMemsetAsync(&s->d_plan->steps, 0, sizeof(unsigned long long), st);
    cudaMemcpyAsync(&s->d_plan->budget, &budget, sizeof(budget), cudaMemcpyHostToDevice, st);
    if (s->step_exec) {
      if ((rc = mf_cuda_check(ctx, cudaGraphLaunch(s->step_exec, st), "server step"))) return rc;
    } else {
      launch_step(s->d_slots, s->d_state, s->d_plan, n, true, s->tc_chunk, sms, 0, 0, st);
    }
  }
  rc = mf_cuda_check(ctx, cudaMemcpyAsync(s->hstate.data(), s->d_state, sizeof(MfSlotState) * n,
                                          cudaMemcpyDeviceToHost, st),
                     "server state");
  if (rc) return rc;
  if ((rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "server step"))) return rc;
  // --- finish the traces whose search ended: roots, cells, CSR
  std::vector<int32_t> only(n, 0);
  std::vector<int> fin;
  for (int t = 0; t < n; t++) {
    if (s->slot_req[t] < 0) continue;
    Request &r = s->reqs[s->slot_req[t]];
    if (r.state != 1 || s->hstate[t].active || r.wait_idx) continue;
    if (s->hstate[t].err) {
      fail(s, r, mf_set_error(ctx, MF_ERR_MAXEDGES, "request exceeded its capacities"), st);
      continue;
    }
    only[t] = 1;
    fin.push_back(t);
  }
  if (!fin.empty()) {
    cudaMemcpyAsync(s->d_only, only.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    uint32_t dims = 0;
    for (int t : fin) dims |= 1u << s->slots[t].F.d;
    mf_b_launch_roots(s->d_slots, s->d_plan, n, s->d_only, dims, ctx->tune.roots_group, sms, st);
    bool cells = false;
    for (int t : fin) cells = cells || (s->slots[t].flags & MF_WANT_CELLS);
    if (cells) {
      mf_b_launch_cells(s->d_slots, s->d_plan, n, s->d_only, sms, st);
      for (int t : fin)
        if (s->slot_req[t] >= 0)
          cudaMemcpyAsync(&s->reqs[s->slot_req[t]].cnt, s->slots[t].B.cnt, sizeof(MfCounters),
                          cudaMemcpyDeviceToHost, st);
      if ((rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "server cells"))) return rc;
      mf_b_launch_cell_edges(s->d_slots, s->d_plan, n, false, s->d_only, sms, st);
      for (int t : fin) {
        if (s->slot_req[t] < 0) continue;
        Request &r = s->reqs[s->slot_req[t]];
        r.n_cells = (s->slots[t].flags & MF_WANT_CELLS) ? (int64_t)r.cnt.n_cells : 0;
        if ((uint64_t)r.n_cells > s->slots[t].B.max_cells || r.cnt.err_overflow ||
            r.cnt.err_table_full) {
          r.n_cells = 0;
          fail(s, r, mf_set_error(ctx, MF_ERR_MAXEDGES, "request cells exceed capacity"), st);
          continue;
        }
        if (r.n_cells > 0) {
          // scan scratch lives after the cell offsets (layout: scan region)
          int64_t *scratch = s->slots[t].B.cell_off + s->slots[t].B.max_cells + 1;
          mf_exclusive_scan(s->slots[t].B.cell_off, s->slots[t].B.cell_off, r.n_cells,
                            (int64_t *)(((uintptr_t)scratch + 255) & ~(uintptr_t)255), st);
          cudaMemcpyAsync(&r.n_ce, s->slots[t].B.cell_off + r.n_cells, 8, cudaMemcpyDeviceToHost, st);
        }
      }
      if ((rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "server CSR counts"))) return rc;
      for (int t : fin) {
        if (s->slot_req[t] < 0) continue;
        Request &r = s->reqs[s->slot_req[t]];
        if (r.state != 1 || r.n_ce <= 0) continue;
        size_t off;
        if (!s->alloc.take((size_t)r.n_ce * 8, &off)) {
          if ((size_t)r.n_ce * 8 > s->arena_bytes - s->data_off) {
            fail(s, r, mf_set_error(ctx, MF_ERR_OOM, "server budget: no room for a cell index"), st);
          } else {  // room frees up as results are fetched: fill on a later step
            r.wait_idx = true;
            only[t] = 0;
          }
          continue;
        }
        r.idx_off = off;
        r.idx_bytes = (size_t)r.n_ce * 8;
        s->slots[t].B.cell_idx = (int64_t *)(s->arena + s->data_off + off);
        cudaMemcpyAsync(s->d_slots + t, &s->slots[t], sizeof(MfSlot), cudaMemcpyHostToDevice, st);
      }
      // the fill reuses the count pass's plan; slots now waiting are masked out
      cudaMemcpyAsync(s->d_only, only.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
      mf_b_launch_plan_edges(s->d_slots, s->d_plan, n, 1, s->d_only, st);
      mf_b_launch_cell_edges(s->d_slots, s->d_plan, n, true, s->d_only, sms, st);
    }
    for (int t : fin)
      if (s->slot_req[t] >= 0)
        cudaMemcpyAsync(&s->reqs[s->slot_req[t]].cnt, s->slots[t].B.cnt, sizeof(MfCounters),
                        cudaMemcpyDeviceToHost, st);
    if ((rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "server finish"))) return rc;
    const double tnow = now_s();
    for (int t : fin) {
      if (s->slot_req[t] < 0) continue;
      Request &r = s->reqs[s->slot_req[t]];
      if (r.state != 1 || r.wait_idx) continue;
      r.levels = s->hstate[t].levels;
      r.state = 2;
      r.t_done = tnow;
      s->finished.push_back(r.id);
      r.S = s->slots[t];
      free_slot(s, r, st);
    }
  }
  if (n_running) {
    int c = 0;
    for (int t = 0; t < n; t++)
      if (s->slot_req[t] >= 0 && s->reqs[s->slot_req[t]].state == 1) c++;
    *n_running = c;
  }
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  return MF_OK;
}

extern "C" int mf_server_done(mf_server *s, int64_t *ids, int32_t cap, int32_t *n) {
  if (!s || !n || cap < 0 || (cap > 0 && !ids)) return MF_ERR_INVALID;
  int32_t k = 0;
  while (k < cap && !s->finished.empty()) {
    ids[k++] = s->finished.front();
    s->finished.pop_front();
  }
  *n = k;
  return MF_OK;
}

extern "C" int mf_server_status(mf_server *s, int64_t id, int32_t *state, double *t_submit,
                                double *t_admit, double *t_done) {
  if (!s || !state) return MF_ERR_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return mf_set_error(s->ctx, MF_ERR_INVALID, "unknown request");
  *state = it->second.state;
  if (t_submit) *t_submit = it->second.t_submit;
  if (t_admit) *t_admit = it->second.t_admit;
  if (t_done) *t_done = it->second.t_done;
  return MF_OK;
}

// Releases the memory of request `it` (done or failed) and forgets it.  Its
// slot was given back when it finished.
static void release(mf_server *s, std::unordered_map<int64_t, Request>::iterator it, cudaStream_t st) {
  free_slot(s, it->second, st);
  free_memory(s, it->second);
  s->reqs.erase(it);
}

extern "C" int mf_server_fetch(mf_server *s, int64_t id, mf_trace_out *o, void *stream) {
  if (!s || !o) return MF_ERR_INVALID;
  mf_ctx *ctx = s->ctx;
  cudaSetDevice(ctx->device);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return mf_set_error(ctx, MF_ERR_INVALID, "unknown request");
  Request &r = it->second;
  if (r.state < 0) {
    const int code = r.state;
    release(s, it, (cudaStream_t)stream);
    return code;
  }
  if (r.state != 2) return mf_set_error(ctx, MF_ERR_INVALID, "request %lld is not done", (long long)id);
  cudaStream_t st = (cudaStream_t)stream;
  const MfTraceBufs &B = r.S.B;
  const MfCounters &h = r.cnt;
  const int d = r.rbf.d;
  const size_t E = (size_t)(h.n_edges < B.max_edges ? h.n_edges : B.max_edges);
  o->n_edges = (int64_t)E;
  o->n_cells = r.n_cells;
  o->n_cell_edges = r.n_ce;
  o->n_vertices = (int64_t)h.n_vertices;
  o->n_near_zero = (int64_t)h.n_near_zero;
  o->n_recheck = (int64_t)h.n_recheck;
  o->n_boundary = (int64_t)h.n_boundary;
  o->n_dead_seeds = (int64_t)h.n_dead_seeds;
  o->levels = r.levels;
  o->root_evals = (int64_t)h.root_evals;
  const bool cells = (r.opts.flags & MF_WANT_CELLS) != 0;
  if (o->cap_edges < o->n_edges ||
      (cells && (o->cap_cells < o->n_cells || (o->cell_edge_idx && o->cap_cell_edges < o->n_cell_edges))))
    return mf_set_error(ctx, MF_ERR_CAPACITY, "output buffers too small (request kept)");
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    if (dst && bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
  };
  cp(o->edge_y, B.edge_y, E * d * 4);
  cp(o->edge_mask, B.edge_mask, E * 4);
  cp(o->edge_f, B.edge_f, E * 16);
  if (r.opts.flags & MF_WANT_ROOTS) {
    cp(o->edge_t, B.edge_t, E * 8);
    cp(o->points, B.edge_pt, E * d * 8);
  }
  if (cells) {
    cp(o->cell_y, B.cell_y, (size_t)r.n_cells * d * 4);
    cp(o->cell_perm, B.cell_perm, (size_t)r.n_cells * d);
    cp(o->cell_edge_off, B.cell_off, ((size_t)r.n_cells + 1) * 8);
    cp(o->cell_edge_idx, B.cell_idx, (size_t)r.n_ce * 8);
  }
  const int rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "server fetch");
  if (rc) return rc;
  release(s, it, st);
  return MF_OK;
}

extern "C" int mf_server_wait(mf_server *s, int64_t id, double timeout_ms, void *stream,
                              int32_t *state) {
  if (!s || !state || !(timeout_ms >= 0.0)) return MF_ERR_INVALID;
  const double t_end = now_s() + timeout_ms * 1e-3;
  for (;;) {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return mf_set_error(s->ctx, MF_ERR_INVALID, "unknown request");
    *state = it->second.state;
    if (*state == 2 || *state < 0) return MF_OK;
    if (now_s() >= t_end)
      return mf_set_error(s->ctx, MF_ERR_TIMEOUT, "request %lld not done after %.1f ms",
                          (long long)id, timeout_ms);
    int32_t running = 0, queued = 0;
    const int rc = mf_server_step(s, stream, &running, &queued);
    if (rc) return rc;
  }
}
