// mf_eval.cu -- evaluation of the learned manifold f(q) = sum_i alpha_i
// exp(-gamma |q - s_i|^2) + b (RBF-SVM decision function, Sec. IV-A), and the
// root solve along traced edges (the "iterative algorithm" of Sec. VI).
//
// FP64 path: one warp per point.  Each lane screens one support vector per
// step in FP32; the survivors (gamma r^2 <= T, T chosen on the host so that
// the dropped terms sum to <= 1e-13) are compacted into a per-warp queue and
// evaluated in FP64 by all 32 lanes at once, so FP64 work is spent only on
// terms that can change f above 1e-13.  GB300 issues few FP64 operations per
// clock, so this compaction is what bounds the FP64 path.
//
// Mixed FP32 SIMT path: one thread per two points, support vectors broadcast
// from shared memory, FP32 differences and ex2, and a per-point rigorous bound
// B on |f~ - f|; points with |f~| <= max(B, band) are re-evaluated in FP64.
#include <cmath>
#include <cstdio>

#include "mf_internal.cuh"
#include "mf_ctx.h"

#define FULL 0xffffffffu

// ---------------------------------------------------------------------------
// RBF preparation
// ---------------------------------------------------------------------------
struct MfRbfStats {
  double sum_abs_alpha;
  float max_abs_s;
  int bad;  // NaN / Inf in the inputs
};

__global__ void k_prepare_rbf(int d, int n, const double *sv, const double *alpha, float *sv32,
                              double *sv64, float *alpha32, MfRbfStats *st) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0;
  float m = 0.f;
  int bad = 0;
  if (j < n) {
    for (int k = 0; k < d; k++) {
      double s = sv[(int64_t)j * d + k];
      if (!isfinite(s)) bad = 1;
      sv64[(int64_t)k * n + j] = s;
      sv32[(int64_t)k * n + j] = (float)s;
      m = fmaxf(m, fabsf((float)s));
    }
    double al = alpha[j];
    if (!isfinite(al)) bad = 1;
    alpha32[j] = (float)al;
    a = fabs(al);
  }
  a = mf_warp_sum_d(a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
    bad |= __shfl_xor_sync(FULL, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&st->sum_abs_alpha, a);
    atomicMax((int *)&st->max_abs_s, __float_as_int(m));  // non-negative floats order as ints
    if (bad) atomicOr(&st->bad, 1);
  }
}

int mf_prepare_rbf(mf_ctx *ctx, const mf_rbf *rbf, MfRbfDev *out, cudaStream_t st) {
  if (!rbf || rbf->d < 2 || rbf->d > MF_MAXD || rbf->n_sv < 1 || rbf->n_sv > (1ll << 30) ||
      !rbf->sv || !rbf->alpha || !(rbf->gamma > 0.0) || !std::isfinite(rbf->gamma) ||
      !std::isfinite(rbf->b))
    return mf_set_error(ctx, MF_ERR_INVALID, "bad RBF parameters");
  const int d = rbf->d, n = (int)rbf->n_sv;
  size_t nb = (size_t)n;
  size_t bytes = nb * d * 4 + nb * d * 8 + nb * 4 + 1024;
  char *base = (char *)mf_ctx_buffer(ctx, MF_SLOT_RBF, bytes);
  if (!base) return MF_ERR_OOM;
  MfRbfStats *dst = (MfRbfStats *)base;
  double *sv64 = (double *)(base + 256);
  float *sv32 = (float *)(sv64 + nb * d);
  float *alpha32 = sv32 + nb * d;
  cudaMemsetAsync(dst, 0, sizeof(MfRbfStats), st);
  k_prepare_rbf<<<(n + 255) / 256, 256, 0, st>>>(d, n, rbf->sv, rbf->alpha, sv32, sv64, alpha32, dst);
  MfRbfStats h;
  int rc = mf_cuda_check(ctx, cudaMemcpyAsync(&h, dst, sizeof(h), cudaMemcpyDeviceToHost, st),
                         "prepare rbf");
  if (rc) return rc;
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "prepare rbf");
  if (rc) return rc;
  if (h.bad) return mf_set_error(ctx, MF_ERR_INVALID, "NaN or Inf in support vectors / alpha");
  out->d = d;
  out->n = n;
  out->sv32 = sv32;
  out->sv64 = sv64;
  out->alpha = rbf->alpha;
  out->alpha32 = alpha32;
  out->gamma = rbf->gamma;
  out->b = rbf->b;
  // Screen: drop terms with gamma r^2 > T where sum|alpha| e^-T <= 1e-13.
  double sa = h.sum_abs_alpha > 0 ? h.sum_abs_alpha : 1e-300;
  double T = std::log(sa / 1e-13);
  if (T < 30.0) T = 30.0;
  if (T > 740.0) T = 740.0;
  out->screen_r2 = (float)((T + 0.5) / rbf->gamma);
  out->drop_bound = sa * std::exp(-T);
  out->smax = h.max_abs_s;
  return MF_OK;
}

// ---------------------------------------------------------------------------
// FP64 warp evaluator with FP32 screening and lane compaction.
// ---------------------------------------------------------------------------
struct F64Acc {
  double f, g;
};

// One compacted batch: lane processes support vector `j` (or nothing if j<0).
template <bool GRAD>
__device__ __forceinline__ void f64_term(const MfRbfDev &R, const double *x, const double *dir,
                                         int j, F64Acc &acc) {
  if (j < 0) return;
  double r2 = 0.0, proj = 0.0;
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) {
    if (k < R.d) {
      double t = x[k] - R.sv64[(int64_t)k * R.n + j];
      r2 = fma(t, t, r2);
      if (GRAD) proj = fma(t, dir[k], proj);
    }
  }
  double e = R.alpha[j] * exp(-R.gamma * r2);
  acc.f += e;
  if (GRAD) acc.g = fma(e, proj, acc.g);
}

// All lanes pass the same x (FP64) and get f (and, with GRAD, g = grad f . dir).
// `terms` accumulates the number of terms evaluated in FP64.
template <bool GRAD>
__device__ F64Acc warp_f64(const MfRbfDev &R, const double *x, const double *dir, int *buf,
                           unsigned long long &terms) {
  const int lane = threadIdx.x & 31;
  float x32[MF_MAXD];
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) x32[k] = k < R.d ? (float)x[k] : 0.f;
  F64Acc acc = {0.0, 0.0};
  int nbuf = 0;
  const unsigned lt = (1u << lane) - 1u;
  for (int base = 0; base < R.n; base += 32) {
    const int j = base + lane;
    bool near = false;
    if (j < R.n) {
      float r2 = 0.f;
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++)
        if (k < R.d) {
          float t = x32[k] - R.sv32[(int64_t)k * R.n + j];
          r2 = fmaf(t, t, r2);
        }
      near = r2 <= R.screen_r2;
    }
    const unsigned m = __ballot_sync(FULL, near);
    if (near) buf[nbuf + __popc(m & lt)] = j;
    nbuf += __popc(m);
    terms += __popc(m);
    if (nbuf >= 32) {
      __syncwarp();
      const int jj = buf[lane];
      __syncwarp();
      if (lane < nbuf - 32) buf[lane] = buf[32 + lane];
      __syncwarp();
      nbuf -= 32;
      f64_term<GRAD>(R, x, dir, jj, acc);
    }
  }
  __syncwarp();
  const int jj = lane < nbuf ? buf[lane] : -1;
  __syncwarp();
  f64_term<GRAD>(R, x, dir, jj, acc);
  acc.f = mf_warp_sum_d(acc.f) + R.b;
  if (GRAD) acc.g = -2.0 * R.gamma * mf_warp_sum_d(acc.g);
  return acc;
}

#define EVAL_WARPS 8

// f at vertex-list entries [v_evaluated, n_vertices) (FP64).
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval_vertices_f64(MfFrame F, MfRbfDev R, MfTraceBufs B) {
  __shared__ int sbuf[EVAL_WARPS][64];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t begin = B.cnt->v_evaluated;
  uint64_t end = B.cnt->n_vertices;
  if (end > B.max_vertices) end = B.max_vertices;
  const uint64_t nw = (uint64_t)gridDim.x * EVAL_WARPS;
  unsigned long long terms = 0;
  for (uint64_t i = begin + (uint64_t)blockIdx.x * EVAL_WARPS + w; i < end; i += nw) {
    int32_t y[MF_MAXD];
    double x[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = k < F.d ? B.vert_y[i * F.d + k] : 0;
    mf_vertex_x(F, y, x);
    F64Acc a = warp_f64<false>(R, x, nullptr, sbuf[w], terms);
    if (lane == 0) {
      B.vtab_f[B.vert_slot[i]] = a.f;
      if (fabs(a.f) < 1e-12) atomicAdd(&B.cnt->n_near_zero, 1ull);
    }
  }
  if (lane == 0 && terms) atomicAdd(&B.cnt->eval_terms, terms);
}

// FP64 re-evaluation of the recheck queue [n_recheck_done, n_recheck).
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_recheck_vertices_f64(MfFrame F, MfRbfDev R, MfTraceBufs B) {
  __shared__ int sbuf[EVAL_WARPS][64];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t begin = B.cnt->n_recheck_done;
  uint64_t end = B.cnt->n_recheck;
  if (end > B.max_vertices) end = B.max_vertices;
  const uint64_t nw = (uint64_t)gridDim.x * EVAL_WARPS;
  unsigned long long terms = 0;
  for (uint64_t q = begin + (uint64_t)blockIdx.x * EVAL_WARPS + w; q < end; q += nw) {
    const uint32_t i = B.recheck[q];
    int32_t y[MF_MAXD];
    double x[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = k < F.d ? B.vert_y[(uint64_t)i * F.d + k] : 0;
    mf_vertex_x(F, y, x);
    F64Acc a = warp_f64<false>(R, x, nullptr, sbuf[w], terms);
    if (lane == 0) {
      B.vtab_f[B.vert_slot[i]] = a.f;
      if (fabs(a.f) < 1e-12) atomicAdd(&B.cnt->n_near_zero, 1ull);
    }
  }
  if (lane == 0 && terms) atomicAdd(&B.cnt->eval_terms, terms);
}

__global__ void k_advance_eval(MfCounters *c) {
  c->v_evaluated = c->n_vertices;
  c->n_recheck_done = c->n_recheck;
}

// ---------------------------------------------------------------------------
// Mixed FP32 SIMT evaluator: thread per MIX_VPT points, support vectors in
// shared memory tiles.  Per point it accumulates
//   acc = sum alpha_j e_j,  A = sum |alpha_j| e_j,  Q = sum |alpha_j| e_j r_j^2
// and bounds |f~ - f| <= A (gamma rho0 + eps_exp + (n/1 + 2) u) + Q gamma (d+2) u,
// where rho0 = d (2 D eta + eta^2) bounds the error of r^2 from rounding the
// coordinates to FP32 (eta = 2.01 u (|x|max + |s|max), D = |x|max + |s|max).
// ---------------------------------------------------------------------------
#define MIX_THREADS 128
#define MIX_VPT 2
#define MIX_TILE 256

struct MixOut {
  double f;
  double bound;
};

__device__ __forceinline__ void mix_tile_loop(const MfRbfDev &R, const float (*xs)[MF_MAXD],
                                              float *acc, float *A, float *Q, const float *s_sv,
                                              const float *s_al, int cnt, float g2) {
  for (int j = 0; j < cnt; j++) {
    float s[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) s[k] = k < R.d ? s_sv[k * MIX_TILE + j] : 0.f;
    const float al = s_al[j];
    const float aa = fabsf(al);
#pragma unroll
    for (int v = 0; v < MIX_VPT; v++) {
      float r2 = 0.f;
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++)
        if (k < R.d) {
          float t = xs[v][k] - s[k];
          r2 = fmaf(t, t, r2);
        }
      const float e = exp2f(-g2 * r2);
      acc[v] = fmaf(al, e, acc[v]);
      const float ae = aa * e;
      A[v] += ae;
      Q[v] = fmaf(ae, r2, Q[v]);
    }
  }
}

// Source of points: vertex list (lattice) or a plain [n][d] array.
template <bool VERTS>
__global__ void __launch_bounds__(MIX_THREADS) k_eval_mixed_f32(MfFrame F, MfRbfDev R, MfTraceBufs B,
                                                                const double *pts, int64_t npts,
                                                                double *fout, uint8_t *flag,
                                                                double band, float smax) {
  __shared__ float s_sv[MF_MAXD * MIX_TILE];
  __shared__ float s_al[MIX_TILE];
  const int d = R.d;
  uint64_t begin = 0, end = (uint64_t)npts;
  if (VERTS) {
    begin = B.cnt->v_evaluated;
    end = B.cnt->n_vertices;
    if (end > B.max_vertices) end = B.max_vertices;
  }
  const float g2 = (float)(R.gamma * 1.4426950408889634);
  const double u = 5.9604644775390625e-08;  // 2^-24
  const uint64_t per_block = (uint64_t)MIX_THREADS * MIX_VPT;
  for (uint64_t base = begin + (uint64_t)blockIdx.x * per_block; base < end;
       base += (uint64_t)gridDim.x * per_block) {
    float xs[MIX_VPT][MF_MAXD];
    double xmax[MIX_VPT];
    double fx[MIX_VPT];
    uint64_t idx[MIX_VPT];
#pragma unroll
    for (int v = 0; v < MIX_VPT; v++) {
      idx[v] = base + (uint64_t)v * MIX_THREADS + threadIdx.x;
      double x[MF_MAXD];
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++) x[k] = 0.0;
      if (idx[v] < end) {
        if (VERTS) {
          int32_t y[MF_MAXD];
#pragma unroll
          for (int k = 0; k < MF_MAXD; k++) y[k] = k < d ? B.vert_y[idx[v] * d + k] : 0;
          mf_vertex_x(F, y, x);
        } else {
#pragma unroll
          for (int k = 0; k < MF_MAXD; k++) x[k] = k < d ? pts[idx[v] * d + k] : 0.0;
        }
      }
      xmax[v] = 0.0;
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++) {
        xs[v][k] = (float)x[k];
        xmax[v] = fmax(xmax[v], fabs(x[k]));
      }
      fx[v] = 0.0;
    }
    float acc[MIX_VPT], A[MIX_VPT], Q[MIX_VPT];
#pragma unroll
    for (int v = 0; v < MIX_VPT; v++) acc[v] = A[v] = Q[v] = 0.f;
    for (int t0 = 0; t0 < R.n; t0 += MIX_TILE) {
      const int cnt = min(MIX_TILE, R.n - t0);
      __syncthreads();
      for (int i = threadIdx.x; i < cnt; i += MIX_THREADS) {
        for (int k = 0; k < d; k++) s_sv[k * MIX_TILE + i] = R.sv32[(int64_t)k * R.n + t0 + i];
        s_al[i] = R.alpha32[t0 + i];
      }
      __syncthreads();
      float part[MIX_VPT];
#pragma unroll
      for (int v = 0; v < MIX_VPT; v++) part[v] = 0.f;
      mix_tile_loop(R, xs, part, A, Q, s_sv, s_al, cnt, g2);
#pragma unroll
      for (int v = 0; v < MIX_VPT; v++) acc[v] += part[v];
    }
#pragma unroll
    for (int v = 0; v < MIX_VPT; v++) {
      if (idx[v] >= end) continue;
      // |r~^2 - r^2| <= sum_k eta (2 |t_k| + eta) <= 2 eta sqrt(d) r + d eta^2 per term, and
      // sum |alpha| e r <= sqrt(A Q) (Cauchy-Schwarz).
      const double D = xmax[v] + (double)smax;
      const double eta = 2.01 * u * D;
      const double Av = (double)A[v], Qv = (double)Q[v];
      const double coord = R.gamma * (2.0 * eta * sqrt((double)d) * sqrt(Av * Qv) + d * eta * eta * Av);
      const double eps_exp = 9.5367431640625e-07;  // 2^-20, above ex2.approx's error
      const double nsum = (double)MIX_TILE + (double)R.n / MIX_TILE + 2.0;  // blocked FP32 sums
      const double bound = (coord + Av * (eps_exp + (nsum + 2.0) * u) +
                            Qv * R.gamma * (d + 2) * u) * 1.02 + 1e-30;
      fx[v] = (double)acc[v] + R.b;
      const bool recheck = fabs(fx[v]) <= fmax(bound, band);
      if (VERTS) {
        const uint32_t slot = B.vert_slot[idx[v]];
        B.vtab_f[slot] = fx[v];
        if (recheck) {
          unsigned long long q = atomicAdd(&B.cnt->n_recheck, 1ull);
          if (q < B.max_vertices) B.recheck[q] = (uint32_t)idx[v];
          else atomicOr(&B.cnt->err_overflow, 1u);
        }
      } else {
        fout[idx[v]] = fx[v];
        flag[idx[v]] = recheck ? 1 : 0;
      }
    }
  }
}

// FP64 evaluation of flagged plain points (mf_eval mixed recheck), or of all
// points when flag == NULL.
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval_points_f64(MfRbfDev R, const double *pts, int64_t n,
                                                        double *fout, const uint8_t *flag,
                                                        unsigned long long *nre) {
  __shared__ int sbuf[EVAL_WARPS][64];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * EVAL_WARPS;
  for (int64_t i = (int64_t)blockIdx.x * EVAL_WARPS + w; i < n; i += nw) {
    if (flag && !flag[i]) continue;
    double x[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) x[k] = k < R.d ? pts[i * R.d + k] : 0.0;
    unsigned long long terms = 0;
    F64Acc a = warp_f64<false>(R, x, nullptr, sbuf[w], terms);
    if (lane == 0) {
      fout[i] = a.f;
      if (nre) atomicAdd(nre, 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// Root solve (FP64): safeguarded Newton on g(t) = f(x1 + t (x2 - x1)) with the
// analytic derivative g'(t) = -2 gamma sum alpha_i e_i (x - s_i).(x2 - x1),
// bracket [lo, hi] kept under the sign rule s = [f >= 0]; start from the
// linear interpolant of the end values.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_roots_f64(MfFrame F, MfRbfDev R, MfTraceBufs B, uint64_t n_edges,
                                                  double tol) {
  __shared__ int sbuf[EVAL_WARPS][64];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int d = F.d;
  const uint64_t nw = (uint64_t)gridDim.x * EVAL_WARPS;
  unsigned long long evals = 0, terms = 0;
  for (uint64_t e = (uint64_t)blockIdx.x * EVAL_WARPS + w; e < n_edges; e += nw) {
    int32_t y[MF_MAXD], y2[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = y2[k] = k < d ? B.edge_y[e * d + k] : 0;
    mf_add_mask(d, y2, B.edge_mask[e], 1);
    double x1[MF_MAXD], x2[MF_MAXD], dir[MF_MAXD], x[MF_MAXD];
    mf_vertex_x(F, y, x1);
    mf_vertex_x(F, y2, x2);
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) dir[k] = k < d ? __dsub_rn(x2[k], x1[k]) : 0.0;
    const double f0 = B.edge_f[2 * e], f1 = B.edge_f[2 * e + 1];
    const bool s1 = f0 >= 0.0;
    double lo = 0.0, hi = 1.0;
    double t = f0 / (f0 - f1);
    if (!(t > 0.0 && t < 1.0)) t = 0.5;
    for (int it = 0; it < 64; it++) {
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++) x[k] = k < d ? __dadd_rn(x1[k], __dmul_rn(t, dir[k])) : 0.0;
      F64Acc a = warp_f64<true>(R, x, dir, sbuf[w], terms);
      evals++;
      if (a.f == 0.0) break;
      if ((a.f >= 0.0) == s1) lo = t; else hi = t;
      double tn = t - a.f / a.g;
      if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
      const double step = fabs(tn - t);
      t = tn;
      if (step <= tol || hi - lo <= 9.094947017729282e-13) break;
    }
    if (lane == 0) {
      B.edge_t[e] = t;
      for (int k = 0; k < d; k++) B.edge_pt[e * d + k] = __dadd_rn(x1[k], __dmul_rn(t, dir[k]));
    }
  }
  if (lane == 0 && evals) {
    atomicAdd(&B.cnt->root_evals, evals);
    atomicAdd(&B.cnt->root_terms, terms);
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void mf_launch_eval_vertices_f64(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B, int sms,
                                 cudaStream_t st) {
  k_eval_vertices_f64<<<sms * 8, EVAL_WARPS * 32, 0, st>>>(F, R, B);
  k_advance_eval<<<1, 1, 0, st>>>(B.cnt);
}

void mf_launch_eval_vertices_mixed(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                   int precision, double band, int sms, cudaStream_t st) {
  (void)precision;
  k_eval_mixed_f32<true><<<sms * 4, MIX_THREADS, 0, st>>>(F, R, B, nullptr, 0, nullptr, nullptr,
                                                          band, R.smax);
  k_recheck_vertices_f64<<<sms * 8, EVAL_WARPS * 32, 0, st>>>(F, R, B);
  k_advance_eval<<<1, 1, 0, st>>>(B.cnt);
}

void mf_launch_roots_f64(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B, uint64_t n_edges,
                         double tol, int sms, cudaStream_t st) {
  if (n_edges == 0) return;
  k_roots_f64<<<sms * 8, EVAL_WARPS * 32, 0, st>>>(F, R, B, n_edges, tol);
}

extern "C" int mf_eval(mf_ctx *ctx, const mf_rbf *rbf, const double *q, int64_t n, int32_t precision,
                       double band, double *f_out, void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  if (n < 0 || (n > 0 && (!q || !f_out)) ||
      (precision != MF_FP64 && precision != MF_MIXED_FP32 && precision != MF_MIXED_BF16))
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_eval: bad arguments");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  MfRbfDev R;
  int rc = mf_prepare_rbf(ctx, rbf, &R, st);
  if (rc) return rc;
  if (n == 0) return MF_OK;
  const int sms = ctx->sms;
  if (precision == MF_FP64) {
    k_eval_points_f64<<<sms * 8, EVAL_WARPS * 32, 0, st>>>(R, q, n, f_out, nullptr, nullptr);
  } else {
    uint8_t *flag = (uint8_t *)mf_ctx_buffer(ctx, MF_SLOT_SCAN, (size_t)n + 256);
    if (!flag) return MF_ERR_OOM;
    MfFrame F;
    mf_frame_lattice(&F, R.d, 1.0, nullptr);
    MfTraceBufs B = {};
    k_eval_mixed_f32<false><<<sms * 4, MIX_THREADS, 0, st>>>(F, R, B, q, n, f_out, flag,
                                                             band > 0 ? band : 1e-3, R.smax);
    k_eval_points_f64<<<sms * 8, EVAL_WARPS * 32, 0, st>>>(R, q, n, f_out, flag, nullptr);
  }
  rc = mf_cuda_check(ctx, cudaGetLastError(), "mf_eval launch");
  if (rc) return rc;
  return mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_eval");
}
