// mf_tune.cu -- the autotuner: times launch variants of the hot kernels on a
// real trace of the caller's request and keeps the fastest in the context.
//
// Candidates:
//   BFS chunk (edges per expansion step): the batch cap, 2^20, 2^18;
//   root solve: register cap (2 or 3 blocks per SM) x grid (2, 4, 8 blocks
//     per SM) x group screen (1, 8, 16 edges), on the first 2^20 traced edges;
//   FP64 vertex evaluation: grid (4, 8, 16 blocks per SM), all vertices;
//   tensor-core evaluation (MF_MIXED_BF16): chunk width 64 or 128.
// Each kernel candidate is timed three times with CUDA events on the
// caller's stream (the first launch of a variant also loads it) and the
// minimum is kept.  Timed re-runs write the same roots; vertex re-evaluations
// go through a scratch copy of the counters.
#include <chrono>
#include <cstring>
#include <functional>

#include "mf_internal.cuh"
#include "mf_ctx.h"

namespace {

__global__ void k_tune_reset(MfCounters *c) {
  c->v_evaluated = 0;
  c->n_recheck = 0;
  c->n_recheck_done = 0;
  c->err_overflow = 0;
}

float time_ms(cudaStream_t st, const std::function<void()> &launch, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

void to_public(const MfTune &t, mf_tune *o) {
  o->roots_variant = t.roots_variant;
  o->roots_blocks_per_sm = t.roots_bps;
  o->eval_blocks_per_sm = t.eval_bps;
  o->tc_chunk = t.tc_chunk;
  o->frontier_chunk = (int64_t)t.frontier_chunk;
  o->roots_group = t.roots_group;
}

}  // namespace

extern "C" int mf_trace(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom,
                        const mf_trace_opts *opts, const double *seeds, int64_t n_seeds,
                        mf_trace_out *out, void *stream);

extern "C" int mf_ctx_set_tune(mf_ctx *ctx, const mf_tune *t) {
  if (!ctx) return MF_ERR_INVALID;
  MfTune n;
  if (t) {
    if ((t->roots_variant != 0 && t->roots_variant != 1) || t->roots_blocks_per_sm < 1 ||
        t->roots_blocks_per_sm > 32 || t->eval_blocks_per_sm < 1 || t->eval_blocks_per_sm > 32 ||
        (t->tc_chunk != 64 && t->tc_chunk != 128) || t->frontier_chunk < 0 ||
        t->roots_group < 1 || t->roots_group > 32)
      return mf_set_error(ctx, MF_ERR_INVALID, "mf_ctx_set_tune: value out of range");
    n.roots_variant = t->roots_variant;
    n.roots_bps = t->roots_blocks_per_sm;
    n.eval_bps = t->eval_blocks_per_sm;
    n.tc_chunk = t->tc_chunk;
    n.frontier_chunk = (uint64_t)t->frontier_chunk;
    n.roots_group = t->roots_group;
  }
  ctx->tune = n;
  return MF_OK;
}

extern "C" int mf_ctx_get_tune(mf_ctx *ctx, mf_tune *out) {
  if (!ctx || !out) return MF_ERR_INVALID;
  memset(out, 0, sizeof(*out));
  to_public(ctx->tune, out);
  return MF_OK;
}

extern "C" int mf_autotune(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom,
                           const mf_trace_opts *opts, const double *seeds, int64_t n_seeds,
                           mf_tune *out, void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  ctx->sub.valid = false;  // its slots are reused here
  if (!rbf || !dom || !opts || !out)
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_autotune: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  memset(out, 0, sizeof(*out));
  ctx->tune = MfTune();
  mf_trace_opts o = *opts;
  o.flags = 0;  // the breadth-first search only
  const uint64_t cap = o.batch_cap_edges > 0 ? (uint64_t)o.batch_cap_edges : (1ull << 24);
  int n_cand = 0;

  // 1. BFS chunk: one search per candidate (the last search leaves the state)
  const uint64_t chunks[3] = {0, 1ull << 20, 1ull << 18};
  double best_bfs = 1e300;
  uint64_t best_chunk = 0, last_run = 0;
  int rc = MF_OK;
  for (int i = 0; i < 3; i++) {
    if (i > 0 && chunks[i] >= cap) continue;
    ctx->tune.frontier_chunk = chunks[i];
    last_run = chunks[i];
    mf_trace_out to;
    memset(&to, 0, sizeof(to));
    const auto t0 = std::chrono::steady_clock::now();
    rc = mf_trace(ctx, rbf, dom, &o, seeds, n_seeds, &to, stream);
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (rc != MF_OK && rc != MF_ERR_CAPACITY) return rc;
    n_cand++;
    if (ms < best_bfs) {
      best_bfs = ms;
      best_chunk = chunks[i];
    }
  }
  ctx->tune.frontier_chunk = best_chunk;
  if (best_chunk != last_run) {
    // trace again with the chosen chunk, so that the kernels below are timed
    // on the lists in the order later calls produce
    mf_trace_out to;
    memset(&to, 0, sizeof(to));
    rc = mf_trace(ctx, rbf, dom, &o, seeds, n_seeds, &to, stream);
    if (rc != MF_OK && rc != MF_ERR_CAPACITY) return rc;
  }
  const MfTraceState L = ctx->last;
  ctx->last.valid = false;
  if (!L.valid) return mf_set_error(ctx, MF_ERR_INVALID, "mf_autotune: the trace left no state");
  const int sms = ctx->sms;

  // 2. root solve on the first 2^20 edges
  const uint64_t es = L.n_edges < (int64_t)(1 << 20) ? (uint64_t)L.n_edges : (1ull << 20);
  float best_roots = 1e30f;
  if (es > 0) {
    MfTune best = ctx->tune;
    const int bps[3] = {2, 4, 8}, groups[3] = {1, 8, 16};
    for (int v = 0; v < 2; v++)
      for (int g = 0; g < 3; g++)
        for (int q = 0; q < 3; q++) {
          MfTune t = ctx->tune;
          t.roots_variant = v;
          t.roots_bps = bps[g];
          t.roots_group = groups[q];
          const float ms = time_ms(
              st, [&]() {
                mf_launch_roots_f64(L.F, L.R, L.B, es, L.tol, t, sms, st,
                                    L.precision != MF_FP64 && !(L.flags & MF_ROOTS_FP64_EXACT));
              }, 3);
          n_cand++;
          if (ms < best_roots) {
            best_roots = ms;
            best = t;
          }
        }
    ctx->tune.roots_variant = best.roots_variant;
    ctx->tune.roots_bps = best.roots_bps;
    ctx->tune.roots_group = best.roots_group;
  }

  // 3. vertex evaluation of every traced vertex, through scratch counters
  float best_eval = 0.f;
  if (L.n_vertices > 0) {
    MfCounters *scratch = (MfCounters *)mf_ctx_buffer(ctx, MF_SLOT_SCAN, 4096);
    if (!scratch) return MF_ERR_OOM;
    MfTraceBufs Bt = L.B;
    Bt.cnt = scratch;
    auto reset = [&]() {
      cudaMemcpyAsync(scratch, L.B.cnt, sizeof(MfCounters), cudaMemcpyDeviceToDevice, st);
      k_tune_reset<<<1, 1, 0, st>>>(scratch);
    };
    best_eval = 1e30f;
    if (L.precision == MF_FP64) {
      const int bps[3] = {4, 8, 16};
      int pick = ctx->tune.eval_bps;
      for (int g = 0; g < 3; g++) {
        MfTune t = ctx->tune;
        t.eval_bps = bps[g];
        float ms = 1e30f;
        for (int r = 0; r < 3; r++) {
          reset();
          ms = fminf(ms, time_ms(st, [&]() { mf_launch_eval_vertices_f64(L.F, L.R, Bt, t, sms, st); },
                                 1));
        }
        n_cand++;
        if (ms < best_eval) {
          best_eval = ms;
          pick = bps[g];
        }
      }
      ctx->tune.eval_bps = pick;
    } else if (L.precision == MF_MIXED_BF16) {
      const int widths[2] = {64, 128};
      int pick = ctx->tune.tc_chunk;
      for (int g = 0; g < 2; g++) {
        float ms = 1e30f;
        for (int r = 0; r < 3; r++) {
          reset();
          ms = fminf(ms, time_ms(st, [&]() {
            mf_launch_eval_vertices_tc(L.F, L.R, Bt, L.band, widths[g], sms, st);
          }, 1));
        }
        n_cand++;
        if (ms < best_eval) {
          best_eval = ms;
          pick = widths[g];
        }
      }
      ctx->tune.tc_chunk = pick;
    } else {
      best_eval = 0.f;
    }
  }
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_autotune");
  if (rc) return rc;
  to_public(ctx->tune, out);
  out->ms_bfs = best_bfs;
  out->ms_roots = es > 0 ? best_roots : 0.0;
  out->ms_eval = best_eval;
  out->n_candidates = n_cand;
  return MF_OK;
}
