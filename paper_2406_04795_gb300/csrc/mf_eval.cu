// mf_eval.cu -- evaluation of the learned manifold f(q) = sum_i alpha_i
// exp(-gamma |q - s_i|^2) + b (RBF-SVM decision function, Sec. IV-A), and the
// root solve along traced edges (the "iterative algorithm" of Sec. VI).
//
// FP64 path (GB300 issues two FP64 FMAs per SM per clock, so FP64 work is what
// the path must save).  One warp per point.  Each lane screens one support
// vector per step in FP32 and sorts it into one of three classes:
//   dropped  gamma r^2 > T, T chosen so that all dropped terms sum to <= 1e-13;
//   strong   |alpha| e^{-gamma r^2} may exceed tau = 3e-10: FP64 distance and
//            an FP64 table-driven exp (mf_exp_neg);
//   weak     the rest: evaluated entirely in FP32 with hi/lo-split
//            coordinates (x = x_hi + x_lo, s = s_hi + s_lo, so differences keep
//            FP32 relative accuracy) and the hardware ex2; no FP64 instruction.
// Strong and weak terms are compacted into two per-warp queues, so lanes never
// idle on skipped terms and each batch of 32 runs one code path.  The weak
// terms' error is bounded on the fly (their summed magnitude times a relative
// bound computed on the host); if the bound would push the total error above
// 2.5e-13 the point is evaluated again with every kept term strong.  Every
// FP64 instruction holds the FP64 pipe for the whole warp, so values that
// are the same for all lanes (coordinates, splits) are computed one axis per
// lane and broadcast.  The vertex evaluation also records, per vertex, the
// support vectors within the root screen's reach (the per-vertex lists the
// root solve screens instead of all vectors).
//
// Mixed FP32 SIMT path: one thread per two points, support vectors broadcast
// from shared memory, FP32 differences and ex2, and a per-point rigorous bound
// B on |f~ - f|; points with |f~| <= max(B, band) are re-evaluated in FP64.
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <utility>
#include <vector>

#include "mf_internal.cuh"
#include "mf_ctx.h"

#define FULL 0xffffffffu
#define STRONG_TAU 3e-10  // terms above this magnitude use the FP64 exp

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// RBF preparation
// ---------------------------------------------------------------------------
struct MfRbfStats {
  double sum_abs_alpha;
  float max_abs_s;
  int bad;  // NaN / Inf in the inputs
};

// Prepared vector j is the caller's vector perm[j] (identity when perm is
// NULL); alpha64 receives the permuted alpha.
__global__ void k_prepare_rbf(int d, int n, const double *sv, const double *alpha, const int32_t *perm,
                              float *sv32, float *svlo32, double *sv64, double *alpha64,
                              float *alpha32, float *strong32, double *exp_tab, double *sv64r,
                              float *svhl, float *sv3, float *alpha_lo32, float2 *exp_df,
                              MfRbfStats *st) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 64) exp_tab[j] = exp2((double)j / 64.0);
  for (int t = j; exp_df && t < 1024; t += gridDim.x * blockDim.x) {
    const double v = exp2(-(double)t / 1024.0);
    const float hi = (float)v;
    exp_df[t] = make_float2(hi, (float)(v - (double)hi));
  }
  double a = 0.0;
  float m = 0.f;
  int bad = 0;
  if (j < n) {
    const int64_t src = perm ? perm[j] : j;
    for (int k = 0; k < d; k++) {
      double s = sv[src * d + k];
      if (!isfinite(s)) bad = 1;
      sv64[(int64_t)k * n + j] = s;
      const float hi = (float)s;
      const float lo = (float)(s - (double)hi);
      sv32[(int64_t)k * n + j] = hi;
      svlo32[(int64_t)k * n + j] = lo;
      sv64r[(int64_t)j * 8 + k] = s;
      svhl[(int64_t)j * 16 + 2 * k] = hi;
      svhl[(int64_t)j * 16 + 2 * k + 1] = lo;
      // s = s1 + s2 + s3 exactly (53 bits in three 24-bit pieces)
      if (sv3) {
        const double r1 = s - (double)hi;
        sv3[(int64_t)j * 24 + 3 * k] = hi;
        sv3[(int64_t)j * 24 + 3 * k + 1] = lo;
        sv3[(int64_t)j * 24 + 3 * k + 2] = (float)(r1 - (double)lo);
      }
      m = fmaxf(m, fabsf(hi));
    }
    for (int k = d; k < 8; k++) {
      sv64r[(int64_t)j * 8 + k] = 0.0;
      svhl[(int64_t)j * 16 + 2 * k] = 0.f;
      svhl[(int64_t)j * 16 + 2 * k + 1] = 0.f;
      if (sv3)
        sv3[(int64_t)j * 24 + 3 * k] = sv3[(int64_t)j * 24 + 3 * k + 1] =
            sv3[(int64_t)j * 24 + 3 * k + 2] = 0.f;
    }
    double al = alpha[src];
    if (!isfinite(al)) bad = 1;
    alpha64[j] = al;
    alpha32[j] = (float)al;
    if (alpha_lo32) alpha_lo32[j] = isfinite(al) ? (float)(al - (double)(float)al) : 0.f;
    a = fabs(al);
    // strong iff gamma r^2 < ln(|alpha| / tau)
    strong32[j] = a > STRONG_TAU ? (float)log(a / STRONG_TAU) : -1.0f;
    // below 8 coordinates the row's padding also carries alpha and the
    // strong threshold, so that one gather of the row serves the root screen
    if (d < 8) {
      svhl[(int64_t)j * 16 + 2 * d] = alpha32[j];
      svhl[(int64_t)j * 16 + 2 * d + 1] = strong32[j];
    }
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

// Per block of 32 consecutive prepared vectors: FP32 bounding box (one warp
// per block).
__global__ void k_rbf_blocks(int d, int n, int nblk, const float *sv32, float *blo, float *bhi) {
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (b >= nblk) return;
  const int j = b * 32 + lane;
  for (int k = 0; k < d; k++) {
    float lo = j < n ? sv32[(int64_t)k * n + j] : INFINITY, hi = j < n ? lo : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(FULL, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, o));
    }
    if (lane == 0) {
      blo[(int64_t)k * nblk + b] = lo;
      bhi[(int64_t)k * nblk + b] = hi;
    }
  }
}

size_t mf_rbf_prep_bytes(int d, int64_t n) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t nb = (size_t)n, nblk = (nb + 31) / 32;
  return 256 + al(nb * d * 8) + 2 * al(nb * d * 4) + 2 * al(nb * 4) + al(64 * 8) + 2 * al(nb * 64) +
         al(nb * 8) + al(nb * 4) + 2 * al(nblk * d * 4) + al(nb * 96) + al(nb * 4) + al(1024 * 8);
}

// Orders the vectors along a Morton (Z-order) curve of their coordinates:
// bits of the quantised coordinates interleaved, 64 / d bits per axis.
static void morton_order(int d, int n, const std::vector<double> &sv, std::vector<int32_t> &perm) {
  double lo[MF_MAXD], hi[MF_MAXD];
  for (int k = 0; k < d; k++) lo[k] = INFINITY, hi[k] = -INFINITY;
  for (int j = 0; j < n; j++)
    for (int k = 0; k < d; k++) {
      const double v = sv[(size_t)j * d + k];
      if (std::isfinite(v)) lo[k] = std::min(lo[k], v), hi[k] = std::max(hi[k], v);
    }
  const int bits = 64 / d;
  const double top = (double)((1ull << bits) - 1);
  std::vector<std::pair<uint64_t, int32_t>> code(n);
  for (int j = 0; j < n; j++) {
    uint64_t q[MF_MAXD];
    for (int k = 0; k < d; k++) {
      const double v = sv[(size_t)j * d + k], w = hi[k] - lo[k];
      double u = (std::isfinite(v) && w > 0) ? (v - lo[k]) / w * top : 0.0;
      u = u < 0 ? 0 : (u > top ? top : u);
      q[k] = (uint64_t)u;
    }
    uint64_t c = 0;
    for (int b = bits - 1; b >= 0; b--)
      for (int k = 0; k < d; k++) c = (c << 1) | ((q[k] >> b) & 1u);
    code[j] = {c, j};
  }
  std::sort(code.begin(), code.end());
  perm.resize(n);
  for (int j = 0; j < n; j++) perm[j] = code[j].second;
}

int mf_prepare_rbf(mf_ctx *ctx, const mf_rbf *rbf, MfRbfDev *out, cudaStream_t st) {
  if (!rbf || rbf->d < 2 || rbf->d > MF_MAXD || rbf->n_sv < 1 || rbf->n_sv > (1ll << 30))
    return mf_set_error(ctx, MF_ERR_INVALID, "bad RBF parameters");
  char *base = (char *)mf_ctx_buffer(ctx, MF_SLOT_RBF, mf_rbf_prep_bytes(rbf->d, rbf->n_sv));
  if (!base) return MF_ERR_OOM;
  return mf_prepare_rbf_at(ctx, rbf, base, out, st);
}

// As mf_prepare_rbf, into `base` (mf_rbf_prep_bytes bytes of device memory).
int mf_prepare_rbf_at(mf_ctx *ctx, const mf_rbf *rbf, char *base, MfRbfDev *out, cudaStream_t st) {
  if (!rbf || rbf->d < 2 || rbf->d > MF_MAXD || rbf->n_sv < 1 || rbf->n_sv > (1ll << 30) ||
      !rbf->sv || !rbf->alpha || !(rbf->gamma > 0.0) || !std::isfinite(rbf->gamma) ||
      !std::isfinite(rbf->b))
    return mf_set_error(ctx, MF_ERR_INVALID, "bad RBF parameters");
  const int d = rbf->d, n = (int)rbf->n_sv;
  const size_t nb = (size_t)n;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  MfRbfStats *dst = (MfRbfStats *)base;
  char *p = base + 256;
  double *sv64 = (double *)p; p += al(nb * d * 8);
  float *sv32 = (float *)p; p += al(nb * d * 4);
  float *svlo32 = (float *)p; p += al(nb * d * 4);
  float *alpha32 = (float *)p; p += al(nb * 4);
  float *strong32 = (float *)p; p += al(nb * 4);
  double *exp_tab = (double *)p; p += al(64 * 8);
  double *sv64r = (double *)p; p += al(nb * 64);
  float *svhl = (float *)p; p += al(nb * 64);
  double *alpha64 = (double *)p; p += al(nb * 8);
  int32_t *perm = (int32_t *)p; p += al(nb * 4);
  const int nblk = (n + 31) / 32;
  float *blo = (float *)p; p += al((size_t)nblk * d * 4);
  float *bhi = (float *)p; p += al((size_t)nblk * d * 4);
  float *sv3 = (float *)p; p += al(nb * 96);
  float *alpha_lo32 = (float *)p; p += al(nb * 4);
  float2 *exp_df = (float2 *)p;
  // Morton order of the vectors (host): spatially compact 32-vector blocks
  {
    std::vector<double> hsv((size_t)n * d);
    int rc0 = mf_cuda_check(ctx, cudaMemcpyAsync(hsv.data(), rbf->sv, hsv.size() * 8,
                                                 cudaMemcpyDeviceToHost, st), "prepare rbf");
    if (rc0) return rc0;
    if ((rc0 = mf_cuda_check(ctx, cudaStreamSynchronize(st), "prepare rbf"))) return rc0;
    std::vector<int32_t> hperm;
    morton_order(d, n, hsv, hperm);
    rc0 = mf_cuda_check(ctx, cudaMemcpyAsync(perm, hperm.data(), (size_t)n * 4,
                                             cudaMemcpyHostToDevice, st), "prepare rbf");
    if (rc0) return rc0;
    if ((rc0 = mf_cuda_check(ctx, cudaStreamSynchronize(st), "prepare rbf"))) return rc0;
  }
  cudaMemsetAsync(dst, 0, sizeof(MfRbfStats), st);
  k_prepare_rbf<<<(n + 255) / 256, 256, 0, st>>>(d, n, rbf->sv, rbf->alpha, perm, sv32, svlo32, sv64,
                                                  alpha64, alpha32, strong32, exp_tab, sv64r, svhl,
                                                  sv3, alpha_lo32, exp_df, dst);
  k_rbf_blocks<<<(nblk + 7) / 8, 256, 0, st>>>(d, n, nblk, sv32, blo, bhi);
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
  out->svlo32 = svlo32;
  out->sv64 = sv64;
  out->alpha = alpha64;
  out->alpha32 = alpha32;
  out->strong32 = strong32;
  out->exp_tab = exp_tab;
  out->sv64r = sv64r;
  out->svhl = svhl;
  out->sv3 = sv3;
  out->alpha_lo32 = alpha_lo32;
  out->exp_df = exp_df;
  out->blk_lo = blo;
  out->blk_hi = bhi;
  out->nblk = nblk;
  out->gamma = rbf->gamma;
  out->b = rbf->b;
  out->sum_abs_alpha = h.sum_abs_alpha;
  // Screen: drop terms with gamma r^2 > T where sum|alpha| e^-T <= 1e-13.
  double sa = h.sum_abs_alpha > 0 ? h.sum_abs_alpha : 1e-300;
  double T = std::log(sa / 1e-13);
  if (T < 30.0) T = 30.0;
  if (T > 740.0) T = 740.0;
  out->screen_r2 = (float)((T + 0.5) / rbf->gamma);
  out->drop_bound = sa * std::exp(-T);
  out->weak_limit = 2.5e-13 - out->drop_bound;
  // relative error of a weak FP32 term on the kept range gamma r^2 <= T + 1/2
  out->weak_rel = 1.1 * ((d + 2) * 5.9604644775390625e-08 * (T + 0.5)) + 9.5367431640625e-07 +
                  2.0 * 5.9604644775390625e-08;
  out->weak_limit32 = (float)out->weak_limit;
  out->drop_bound32 = (float)out->drop_bound;
  out->weak_rel32 = (float)out->weak_rel;
  out->smax = h.max_abs_s;
  // the mixed paths' root screen: sum|alpha| e^-T <= 1e-12
  {
    double Tf = std::log(sa / 1e-12);
    if (Tf < 30.0) Tf = 30.0;
    if (Tf > T) Tf = T;
    out->screen_r2_fast = (float)((Tf + 0.5) / rbf->gamma);
    out->drop_bound32_fast = (float)(sa * std::exp(-Tf));
  }
  return MF_OK;
}

// ---------------------------------------------------------------------------
// FP64 warp evaluator: FP32 screening into strong / weak queues.
// ---------------------------------------------------------------------------
struct F64Acc {
  double f, g;  // f (with b) and, with GRAD, grad f . dir
  float weak;   // sum of |term| over weak terms (error bound input)
  float wf, wg; // FP32 partial sums of the weak terms
  float weakc;  // sum of |term| over the weak terms taken from the root screen's cache
};

// x split as x_hi + x_lo (both FP32) so that FP32 differences to a support
// vector split the same way keep FP32 relative accuracy.
template <int D>
struct Split32 {
  float hi[D], lo[D], dir[D];
};

// Dimension of the work: a compile-time D below MF_MAXD is exact; D ==
// MF_MAXD serves every d <= MF_MAXD at run time.
template <int D>
__device__ __forceinline__ int dim_of(int rt) {
  return D < MF_MAXD ? D : rt;
}

// (All lanes, converged.)  Lane k < d converts axis k and shuffles
// broadcast the parts: each FP64 instruction holds the FP64 pipe for the
// whole warp, so one conversion per lane serves every axis at once.
template <int D>
__device__ __forceinline__ Split32<D> split32(int d, const double *x, const double *dir) {
  const int lane = threadIdx.x & 31;
  d = dim_of<D>(d);
  double xk = 0.0, dk = 0.0;
#pragma unroll
  for (int k = 0; k < D; k++)
    if (k == lane) {
      xk = x[k];
      dk = dir ? dir[k] : 0.0;
    }
  const float h = (float)xk, l = (float)(xk - (double)h), dd = (float)dk;
  Split32<D> s;
#pragma unroll
  for (int k = 0; k < D; k++) {
    s.hi[k] = k < d ? __shfl_sync(FULL, h, k) : 0.f;
    s.lo[k] = k < d ? __shfl_sync(FULL, l, k) : 0.f;
    s.dir[k] = k < d ? __shfl_sync(FULL, dd, k) : 0.f;
  }
  return s;
}

// mf_vertex_x in every lane (all lanes, converged): lane k < d computes
// axis k with the same operations and the values are broadcast.
template <int D>
__device__ __forceinline__ void vertex_x_lanes(const MfFrame &F, const int32_t *y, double *x) {
  const int lane = threadIdx.x & 31;
  const int d = dim_of<D>(F.d);
  const int ko = lane < d ? lane : 0;
  long long sy = 0;
  int32_t yo = 0;
#pragma unroll
  for (int k = 0; k < D; k++)
    if (k < d) {
      sy += y[k];
      if (k == ko) yo = y[k];
    }
  const double cs = __dmul_rn(F.c, (double)sy);
  const double xo = __dadd_rn(__dmul_rn(F.lam, __dsub_rn((double)yo, cs)), F.o[ko]);
#pragma unroll
  for (int k = 0; k < D; k++) x[k] = k < d ? __shfl_sync(FULL, xo, k) : 0.0;
}

// e^x for x <= 0 in FP64 by the table-driven method of P. T. P. Tang
// ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989): x = (64 m + j) ln2/64 + r
// with |r| <= ln2/128 (about), e^x = 2^m 2^(j/64) e^r, and e^r - 1 by its
// Taylor polynomial of degree 5 (truncation below 4e-17 relative).  ln2/64 is
// split into L1 (29 significant bits, so k L1 is exact for |k| < 2^17) and
// L2.  Arguments below -708 return e^-708 (absolute error < 4e-308).  Relative
// error a few ulp; 12 FP64-pipe instructions and one table load.
__device__ __forceinline__ double mf_exp_neg(double x, const double *tab) {
  const double inv_l = 0x1.71547652b82fep+6;   // 64 / ln2
  const double l1 = 0x1.62e42ff000000p-7;      // ln2/64, leading bits
  const double l2 = -0x1.718432a1b0e26p-41;    // ln2/64 - l1
  const double shift = 0x1.8p52;               // rounds to an integer in the low word
  x = fmax(x, -708.0);
  const double ks = fma(x, inv_l, shift);
  const int k = __double2loint(ks);
  const double kd = ks - shift;
  const double r = fma(-kd, l2, fma(-kd, l1, x));
  const double r2 = r * r;
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(r2, q, r);  // e^r - 1
  const double t = __ldg(tab + (k & 63));
  const double scale = __hiloint2double(((k >> 6) + 1023) << 20, 0);  // 2^m, m >= -1022
  return fma(t, p, t) * scale;
}

// Strong term: FP64 difference and the FP64 exp above.
template <bool GRAD, int D>
__device__ __forceinline__ void f64_term(const MfRbfDev &R, const double *x, const double *dir,
                                         int j, F64Acc &acc) {
  if (j < 0) return;
  const int d = dim_of<D>(R.d);
  double r2 = 0.0, proj = 0.0;
  const double2 *row = reinterpret_cast<const double2 *>(R.sv64r + (int64_t)j * 8);
#pragma unroll
  for (int k2 = 0; k2 < (D + 1) / 2; k2++) {
    const double2 s = __ldg(row + k2);
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int k = 2 * k2 + h;
      if (k < D && k < d) {
        const double t = x[k] - (h ? s.y : s.x);
        r2 = fma(t, t, r2);
        if (GRAD) proj = fma(t, dir[k], proj);
      }
    }
  }
  const double e = R.alpha[j] * mf_exp_neg(-R.gamma * r2, R.exp_tab);
  acc.f += e;
  if (GRAD) acc.g = fma(e, proj, acc.g);
}

// Support vector j's row for the root path, in one gather: the hi/lo
// coordinate pairs c[2k], c[2k + 1] (k < D) and, below 8 coordinates, alpha
// and the strong threshold from the row's padding (else from their arrays).
template <int D>
__device__ __forceinline__ void sv_row(const MfRbfDev &R, int j, float *c, float &al, float &s32) {
  constexpr int Q = D < 8 ? (2 * D + 2 + 3) / 4 : 4;
  const float4 *row = reinterpret_cast<const float4 *>(R.svhl + (int64_t)j * 16);
  float v[4 * Q];
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const float4 t = __ldg(row + q);
    v[4 * q] = t.x;
    v[4 * q + 1] = t.y;
    v[4 * q + 2] = t.z;
    v[4 * q + 3] = t.w;
  }
#pragma unroll
  for (int k = 0; k < 2 * D && k < 4 * Q; k++) c[k] = v[k];
  if (D < 8) {
    al = v[D < 8 ? 2 * D : 0];
    s32 = v[D < 8 ? 2 * D + 1 : 0];
  } else {
    al = R.alpha32[j];
    s32 = R.strong32[j];
  }
}

// Weak term (|alpha| e <= tau): FP32 throughout with hi/lo-split coordinates.
// Its relative error is at most (d+2) u gamma r^2 (differences, squares and
// the exponent's rounding, u = 2^-24) + 2^-20 (ex2) + 2u (alpha, product); on
// the kept range gamma r^2 <= T + 1/2 the host bounds this by R.weak_rel.
template <bool GRAD, int D>
__device__ __forceinline__ void f32_weak_term(const MfRbfDev &R, const Split32<D> &x, int j,
                                              F64Acc &acc) {
  if (j < 0) return;
  const int d = dim_of<D>(R.d);
  const float g2 = (float)(R.gamma * 1.4426950408889634);
  float r2 = 0.f, proj = 0.f, c[2 * D], al, s32;
  sv_row<D>(R, j, c, al, s32);
#pragma unroll
  for (int k = 0; k < D; k++) {
    if (k < d) {
      const float t = (x.hi[k] - c[2 * k]) + (x.lo[k] - c[2 * k + 1]);
      r2 = fmaf(t, t, r2);
      if (GRAD) proj = fmaf(t, x.dir[k], proj);
    }
  }
  const float e = al * ex2_approx(-g2 * r2);
  acc.wf += e;
  acc.weak += fabsf(e);
  if (GRAD) acc.wg = fmaf(e, proj, acc.wg);
}

// Pops 32 entries of a queue of length n (>= 32) into lane `j`.
__device__ __forceinline__ int pop32(int *q, int &n, int lane) {
  __syncwarp();
  const int j = q[lane];
  __syncwarp();
  if (lane < n - 32) q[lane] = q[32 + lane];
  __syncwarp();
  n -= 32;
  return j;
}

// All lanes pass the same x (FP64) and get f (and, with GRAD, g = grad f . dir).
// qs, qw: two 64-entry per-warp queues.  ALL_STRONG puts every kept term in
// the strong queue.  terms[0/1] count strong / weak terms.
// lbuf (LIST_CAP entries, NULL for none) receives the vectors within
// sqrt(list_r2) of x (all of them when *nl <= LIST_CAP), *nl their count.
#define LIST_CAP 512
template <bool GRAD, bool ALL_STRONG, int D>
__device__ F64Acc warp_f64_pass(const MfRbfDev &R, const double *x, const double *dir, int *qs,
                                int *qw, unsigned long long *terms, int *lbuf = nullptr,
                                float list_r2 = 0.f, int *nl = nullptr) {
  const int lane = threadIdx.x & 31;
  const int d = dim_of<D>(R.d);
  const float g32 = (float)R.gamma;
  F64Acc acc = {0.0, 0.0, 0.f, 0.f, 0.f, 0.f};
  const Split32<D> xs = split32<D>(d, x, dir);
  int ns = 0, nw = 0;
  const unsigned lt = (1u << lane) - 1u;
  // blocks of 32 vectors whose box is farther than the screen distance (with
  // a rounding margin) hold no vector that passes: they are skipped whole
  const float box2 = fmaxf(R.screen_r2, lbuf ? list_r2 : 0.f) * 1.001f + 1e-5f;
  int nlist = 0;
  for (int bb0 = 0; bb0 < R.nblk; bb0 += 32) {
    bool bkeep = false;
    if (bb0 + lane < R.nblk) {
      float q2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; k++)
        if (k < d) {
          const float lo = R.blk_lo[(int64_t)k * R.nblk + bb0 + lane];
          const float hi = R.blk_hi[(int64_t)k * R.nblk + bb0 + lane];
          const float t = fmaxf(fmaxf(lo - xs.hi[k], xs.hi[k] - hi), 0.f);
          q2 = fmaf(t, t, q2);
        }
      bkeep = q2 <= box2;
    }
    unsigned bm = __ballot_sync(FULL, bkeep);
  while (bm) {
    const int j = (bb0 + __ffs(bm) - 1) * 32 + lane;
    bm &= bm - 1;
    bool keep = false, strong = false, listed = false;
    if (j < R.n) {
      float r2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; k++)
        if (k < d) {
          float t = xs.hi[k] - R.sv32[(int64_t)k * R.n + j];
          r2 = fmaf(t, t, r2);
        }
      keep = r2 <= R.screen_r2;
      strong = ALL_STRONG || (g32 * r2 < R.strong32[j] + 0.5f);
      listed = r2 <= list_r2;
    }
    if (lbuf) {
      const unsigned ml = __ballot_sync(FULL, listed);
      const int pos = nlist + __popc(ml & lt);
      if (listed && pos < LIST_CAP) lbuf[pos] = j;
      nlist += __popc(ml);
    }
    const unsigned ms = __ballot_sync(FULL, keep && strong);
    const unsigned mw = __ballot_sync(FULL, keep && !strong);
    if (keep && strong) qs[ns + __popc(ms & lt)] = j;
    if (keep && !strong) qw[nw + __popc(mw & lt)] = j;
    ns += __popc(ms);
    nw += __popc(mw);
    terms[0] += __popc(ms);
    terms[1] += __popc(mw);
    if (ns >= 32) {
      const int jj = pop32(qs, ns, lane);
      f64_term<GRAD, D>(R, x, dir, jj, acc);
    }
    if (nw >= 32) {
      const int jj = pop32(qw, nw, lane);
      f32_weak_term<GRAD, D>(R, xs, jj, acc);
    }
  }
  }
  __syncwarp();
  const int js = lane < ns ? qs[lane] : -1;
  const int jw = lane < nw ? qw[lane] : -1;
  __syncwarp();
  f64_term<GRAD, D>(R, x, dir, js, acc);
  f32_weak_term<GRAD, D>(R, xs, jw, acc);
  acc.f = mf_warp_sum_d(acc.f) + (double)mf_warp_sum_f(acc.wf) + R.b;
  acc.weak = mf_warp_sum_f(acc.weak);
  if (GRAD) acc.g = -2.0 * R.gamma * (mf_warp_sum_d(acc.g) + (double)mf_warp_sum_f(acc.wg));
  if (nl) *nl = nlist;
  return acc;
}

// f with total error <= 2.5e-13 (dropped + weak terms), all lanes.
template <bool GRAD, int D>
__device__ __forceinline__ F64Acc warp_f64(const MfRbfDev &R, const double *x, const double *dir,
                                           int *qs, int *qw, unsigned long long *terms,
                                           int *lbuf = nullptr, float list_r2 = 0.f,
                                           int *nl = nullptr) {
  F64Acc a = warp_f64_pass<GRAD, false, D>(R, x, dir, qs, qw, terms, lbuf, list_r2, nl);
  if (a.weak * (1.01f * R.weak_rel32) > R.weak_limit32)
    a = warp_f64_pass<GRAD, true, D>(R, x, dir, qs, qw, terms);
  return a;
}

#define EVAL_WARPS 8

// Stores the root-screen list of vertex i (nl entries in lbuf, all lanes
// call): a pool range when it fits, else the vertex is marked as having none
// (its edges then screen the vector blocks).
__device__ __forceinline__ void store_vertex_list(const MfTraceBufs &B, uint64_t i, int nl,
                                                  const int *lbuf) {
  const int lane = threadIdx.x & 31;
  unsigned long long off = 0;
  if (lane == 0 && nl <= LIST_CAP) off = atomicAdd(&B.cnt->n_vlist, (unsigned long long)nl);
  off = __shfl_sync(FULL, off, 0);
  const bool ok = nl <= LIST_CAP && off + nl <= B.vlist_cap;
  __syncwarp();
  if (ok)
    for (int q = lane; q < nl; q += 32) B.vlist[off + q] = lbuf[q];
  if (lane == 0) {
    B.vlist_off[i] = off;
    B.vlist_n[i] = ok ? (uint32_t)nl : MF_NO_LIST;
  }
  __syncwarp();
}

// The root-screen list of the point with FP32 coordinates xh (all lanes):
// the vectors with FP32 r^2 <= list_r2, computed and ordered exactly as
// warp_f64_pass lists them, so both evaluators give a vertex the same list.
// Returns the count (entries beyond LIST_CAP are counted, not stored).
template <int D>
__device__ int warp_vertex_list(const MfRbfDev &R, const float *xh, float list_r2, int *lbuf) {
  const int lane = threadIdx.x & 31;
  const int d = dim_of<D>(R.d);
  const unsigned lt = (1u << lane) - 1u;
  const float box2 = list_r2 * 1.001f + 1e-5f;
  int nlist = 0;
  for (int bb0 = 0; bb0 < R.nblk; bb0 += 32) {
    bool bkeep = false;
    if (bb0 + lane < R.nblk) {
      float q2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; k++)
        if (k < d) {
          const float lo = R.blk_lo[(int64_t)k * R.nblk + bb0 + lane];
          const float hi = R.blk_hi[(int64_t)k * R.nblk + bb0 + lane];
          const float t = fmaxf(fmaxf(lo - xh[k], xh[k] - hi), 0.f);
          q2 = fmaf(t, t, q2);
        }
      bkeep = q2 <= box2;
    }
    unsigned bm = __ballot_sync(FULL, bkeep);
    while (bm) {
      const int j = (bb0 + __ffs(bm) - 1) * 32 + lane;
      bm &= bm - 1;
      bool listed = false;
      if (j < R.n) {
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; k++)
          if (k < d) {
            const float t = xh[k] - R.sv32[(int64_t)k * R.n + j];
            r2 = fmaf(t, t, r2);
          }
        listed = r2 <= list_r2;
      }
      const unsigned ml = __ballot_sync(FULL, listed);
      const int pos = nlist + __popc(ml & lt);
      if (listed && pos < LIST_CAP) lbuf[pos] = j;
      nlist += __popc(ml);
    }
  }
  __syncwarp();
  return nlist;
}

// Root-screen lists of vertex-list entries [v_evaluated, n_vertices) on the
// mixed paths, whose evaluators do not screen (warp per vertex).
template <int D>
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_vertex_lists(MfFrame F, MfRbfDev R, MfTraceBufs B) {
  __shared__ int slist[EVAL_WARPS][LIST_CAP];
  const int w = threadIdx.x >> 5;
  const uint64_t begin = B.cnt->v_evaluated;
  uint64_t end = B.cnt->n_vertices;
  if (end > B.max_vertices) end = B.max_vertices;
  const uint64_t nwarps = (uint64_t)gridDim.x * EVAL_WARPS;
  for (uint64_t i = begin + (uint64_t)blockIdx.x * EVAL_WARPS + w; i < end; i += nwarps) {
    int32_t y[MF_MAXD];
    double x[D];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = k < F.d ? B.vert_y[i * F.d + k] : 0;
    vertex_x_lanes<D>(F, y, x);
    const Split32<D> xs = split32<D>(F.d, x, nullptr);
    const int nl = warp_vertex_list<D>(R, xs.hi, B.list_r2, slist[w]);
    store_vertex_list(B, i, nl, slist[w]);
  }
}

// f at vertex-list entries [v_evaluated, n_vertices) (FP64).
template <int D>
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval_vertices_f64(MfFrame F, MfRbfDev R, MfTraceBufs B) {
  __shared__ int sq[EVAL_WARPS][2][64];
  __shared__ int slist[EVAL_WARPS][LIST_CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t begin = B.cnt->v_evaluated;
  uint64_t end = B.cnt->n_vertices;
  if (end > B.max_vertices) end = B.max_vertices;
  const uint64_t nwarps = (uint64_t)gridDim.x * EVAL_WARPS;
  unsigned long long terms[2] = {0, 0};
  for (uint64_t i = begin + (uint64_t)blockIdx.x * EVAL_WARPS + w; i < end; i += nwarps) {
    int32_t y[MF_MAXD];
    double x[D];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = k < F.d ? B.vert_y[i * F.d + k] : 0;
    vertex_x_lanes<D>(F, y, x);
    int nl = 0;
    F64Acc a = warp_f64<false, D>(R, x, nullptr, sq[w][0], sq[w][1], terms,
                                  B.vlist ? slist[w] : nullptr, B.list_r2, &nl);
    if (lane == 0) {
      mf_vtab_f(B, B.vert_slot[i]) = a.f;
      if (fabs(a.f) < 1e-12) atomicAdd(&B.cnt->n_near_zero, 1ull);
    }
    if (B.vlist) store_vertex_list(B, i, nl, slist[w]);  // the root screen's list
  }
  if (lane == 0 && (terms[0] | terms[1])) {
    atomicAdd(&B.cnt->eval_terms, terms[0]);
    atomicAdd(&B.cnt->eval_terms_weak, terms[1]);
  }
}

// FP64 re-evaluation of the recheck queue [n_recheck_done, n_recheck).
template <int D>
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_recheck_vertices_f64(MfFrame F, MfRbfDev R, MfTraceBufs B) {
  __shared__ int sq[EVAL_WARPS][2][64];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t begin = B.cnt->n_recheck_done;
  uint64_t end = B.cnt->n_recheck;
  if (end > B.max_vertices) end = B.max_vertices;
  const uint64_t nwarps = (uint64_t)gridDim.x * EVAL_WARPS;
  unsigned long long terms[2] = {0, 0};
  for (uint64_t q = begin + (uint64_t)blockIdx.x * EVAL_WARPS + w; q < end; q += nwarps) {
    const uint32_t i = B.recheck[q];
    int32_t y[MF_MAXD];
    double x[D];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = k < F.d ? B.vert_y[(uint64_t)i * F.d + k] : 0;
    vertex_x_lanes<D>(F, y, x);
    F64Acc a = warp_f64<false, D>(R, x, nullptr, sq[w][0], sq[w][1], terms);
    if (lane == 0) {
      mf_vtab_f(B, B.vert_slot[i]) = a.f;
      if (fabs(a.f) < 1e-12) atomicAdd(&B.cnt->n_near_zero, 1ull);
    }
  }
  if (lane == 0 && (terms[0] | terms[1])) {
    atomicAdd(&B.cnt->eval_terms, terms[0]);
    atomicAdd(&B.cnt->eval_terms_weak, terms[1]);
  }
}

__global__ void k_advance_eval(MfCounters *c) {
  c->v_evaluated = c->n_vertices;
  c->n_recheck_done = c->n_recheck;
}

// ---------------------------------------------------------------------------
// Mixed FP32 SIMT evaluator: thread per MIX_VPT points, support vectors in
// shared memory tiles.  Per point it accumulates
//   acc = sum alpha_j e_j,  A = sum |alpha_j| e_j,  Q = sum |alpha_j| e_j r_j^2
// and bounds |f~ - f| by the coordinate rounding (eta = 2.01 u (|x|max +
// |s|max) per coordinate, |r~^2 - r^2| <= 2 eta sqrt(d) r + d eta^2, and
// sum |alpha| e r <= sqrt(A Q)), the ex2 error (2^-20), the exponent rounding
// ((d+2) u gamma r^2) and the blocked FP32 summation.
// ---------------------------------------------------------------------------
#define MIX_THREADS 128
#define MIX_VPT 2
#define MIX_TILE 256

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
      const float e = ex2_approx(-g2 * r2);
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
                                                                double band) {
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
      const double D = xmax[v] + (double)R.smax;
      const double eta = 2.01 * u * D;
      const double Av = (double)A[v], Qv = (double)Q[v];
      const double coord = R.gamma * (2.0 * eta * sqrt((double)d) * sqrt(Av * Qv) + d * eta * eta * Av);
      const double eps_exp = 9.5367431640625e-07;  // 2^-20, above ex2.approx's error
      const double nsum = (double)MIX_TILE + (double)R.n / MIX_TILE + 2.0;  // blocked FP32 sums
      const double bound = (coord + Av * (eps_exp + (nsum + 2.0) * u) +
                            Qv * R.gamma * (d + 2) * u) * 1.02 + 1e-30;
      const double fx = (double)acc[v] + R.b;
      const bool recheck = fabs(fx) <= fmax(bound, band);
      if (VERTS) {
        const uint32_t slot = B.vert_slot[idx[v]];
        mf_vtab_f(B, slot) = fx;
        if (recheck) {
          unsigned long long q = atomicAdd(&B.cnt->n_recheck, 1ull);
          if (q < B.max_vertices) B.recheck[q] = (uint32_t)idx[v];
          else atomicOr(&B.cnt->err_overflow, 1u);
        }
      } else {
        fout[idx[v]] = fx;
        flag[idx[v]] = recheck ? 1 : 0;
      }
    }
  }
}

// FP64 evaluation of flagged plain points (mf_eval mixed recheck), or of all
// points when flag == NULL.
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_eval_points_f64(MfRbfDev R, const double *pts, int64_t n,
                                                        double *fout, const uint8_t *flag) {
  __shared__ int sq[EVAL_WARPS][2][64];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * EVAL_WARPS;
  unsigned long long terms[2] = {0, 0};
  for (int64_t i = (int64_t)blockIdx.x * EVAL_WARPS + w; i < n; i += nwarps) {
    if (flag && !flag[i]) continue;
    double x[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) x[k] = k < R.d ? pts[i * R.d + k] : 0.0;
    F64Acc a = warp_f64<false, MF_MAXD>(R, x, nullptr, sq[w][0], sq[w][1], terms);
    if (lane == 0) fout[i] = a.f;
  }
}

// ---------------------------------------------------------------------------
// Root solve along each traced edge: g(t) = f(x1 + t (x2 - x1)), t in [0,1],
// g(0) and g(1) of opposite sign (Sec. VI's "iterative algorithm").
//
// 1. Segment screen (FP32): the support vectors within the FP64 screen
//    distance of the whole segment are compacted into per-warp lists in
//    shared memory: terms above ROOT_TAU from the front of one list, weak
//    ones from its back, the band between (mid) in a second list.  The
//    candidates are the base vertex's list when the FP64 vertex evaluation
//    recorded one, else all vectors by 32-vector block.
// 2. FP32 Halley steps (t - 2 g g' / (2 g'^2 - g g''), Newton where the
//    denominator is not positive) from the linear interpolant of the end
//    values, over that list, with hi/lo-split coordinates (x = x_hi + x_lo)
//    so that differences keep FP32 relative accuracy.
// 3. FP64 Newton with a kept bracket [lo, hi] under the sign rule
//    s = [f >= 0], over the same list: terms that can exceed ROOT_TAU = 1e-8
//    with the FP64 exp, the rest in FP32 under a bound that keeps their
//    error from moving t by more than 1e-10 (else every term in FP64).  A
//    step is final when |step| <= 1e-7, or on the first FP64 step when
//    |step| <= 1e-5 and |g''| step^2 <= 5e-11 |g'| (the remaining Newton
//    error is then below ~1e-9 in t).  That first step takes g' from the
//    last FP32 evaluation, carried to t by its g'', where the FP32 sum of
//    g' terms had little cancellation; it then needs only the FP64 g.
//    Lists that overflow fall back to full per-point screening.
// ---------------------------------------------------------------------------
#define ROOT_WARPS 8
#define NEAR_CAP 1024
#define MID_CAP 256
// The root's FP64 step evaluates in FP64 only the terms that can exceed
// ROOT_TAU = 1e-8 (strong32 shifted by ln(ROOT_TAU / STRONG_TAU)); the band
// between STRONG_TAU and ROOT_TAU ("mid") joins the FP32 stage's list and is
// summed in FP32 with the weak terms in the FP64 step.
#define ROOT_TAU_SHIFT 3.5065579f
// The mixed paths need |dt| <= 1e-6 only: their FP64 step takes the terms
// that can exceed 1e-5 (shift ln(1e-5 / STRONG_TAU)); the FP32 part may then
// move t by up to 1e-7 and the accepted Newton step leaves < 1e-7.
#define ROOT_TAU_SHIFT_FAST 10.414313f

// Warp sums of four values, every lane receiving all four: a transposed
// butterfly (lanes split the values between halves, then quarters, before
// the plain butterfly), 10 shuffles and 6 adds instead of 20 and 20.
__device__ __forceinline__ void warp_sum4(float &a, float &b, float &c, float &e) {
  const int lane = threadIdx.x & 31;
  const bool up = lane & 16, odd = lane & 8;
  // lower half keeps (a, b), upper half keeps (c, e)
  const float r0 = __shfl_xor_sync(FULL, up ? a : c, 16);
  const float r1 = __shfl_xor_sync(FULL, up ? b : e, 16);
  const float x = (up ? c : a) + r0, y = (up ? e : b) + r1;
  // then lanes with bit 3 clear keep x, the others y
  float z = (odd ? y : x) + __shfl_xor_sync(FULL, odd ? x : y, 8);
  z += __shfl_xor_sync(FULL, z, 4);
  z += __shfl_xor_sync(FULL, z, 2);
  z += __shfl_xor_sync(FULL, z, 1);
  // lanes 0, 8, 16, 24 hold the totals of a, b, c, e
  a = __shfl_sync(FULL, z, 0);
  b = __shfl_sync(FULL, z, 8);
  c = __shfl_sync(FULL, z, 16);
  e = __shfl_sync(FULL, z, 24);
}

struct Root32 {
  float g, gp, gpp, gpa;  // gpa: the sum of |g'| terms (cancellation measure)
};

// The per-term data of the root path, cached by the segment screen for the
// first HC_STRONG strong, HC_MID mid and HC_WEAK weak entries of each edge
// (per warp, in shared memory): with u = x1 - s (FP32 hi/lo differences)
// and dir = x2 - x1,
// A = |u|^2 and Bp = u . dir, so that at x(t) = x1 + t dir
//   proj(t) = (x(t) - s) . dir = Bp + t |dir|^2,
//   r2(t) = |x(t) - s|^2 = A + t (Bp + proj(t)),
// and an evaluation reads three floats per term instead of gathering the
// vector's coordinates again.  With the support vector at distance r from
// x(t), |u| + t |dir| <= r + 2 |dir|, and the roundings of u (2 per
// coordinate), A (d FMAs), Bp, |dir|^2, proj and r2 leave
//   |r2~ - r2| <= 2^-24 (r2 + (d + 4.5) (r + 2 |dir|)^2);
// with the rounding of gamma log2(e) and of the exponent's product the
// term's relative error from its exponent is below
//   (d + 8) 2^-24 gamma (r + 2 |dir|)^2,
// plus ex2's 2^-20 and 2^-23 for alpha and the product (root_rel_cached).
// The FP32 stage only steers and feeds the reused g' (per-term errors of a
// few 1e-6 there); the weak terms of the deferred FP64 step use the bound.
#define HC_STRONG 192
#define HC_MID 64
#define HC_WEAK 192
#define HC_ALL (HC_STRONG + HC_MID + HC_WEAK)

// A, Bp and alpha of support vector j against x1 (hi/lo) along dir32.
template <int D>
__device__ __forceinline__ void term_ab(const MfRbfDev &R, int j, const float *x1hi,
                                        const float *x1lo, const float *dir32, float &A,
                                        float &Bp, float &al) {
  const int d = dim_of<D>(R.d);
  float c[2 * D], s32;
  sv_row<D>(R, j, c, al, s32);
  A = 0.f;
  Bp = 0.f;
#pragma unroll
  for (int k = 0; k < D; k++) {
    if (k < d) {
      const float u = (x1hi[k] - c[2 * k]) + (x1lo[k] - c[2 * k + 1]);
      A = fmaf(u, u, A);
      Bp = fmaf(u, dir32[k], Bp);
    }
  }
}

// FP32 evaluation of g, g', g'' at t over the strong entries of the near
// list and the mid list (all lanes), from the screen's cache (hc: A, Bp,
// alpha, HC_ALL floats each) where it holds the entry.  The weak entries are
// below tau e^(1/2) = 5e-10 each, so even a few hundred of them shift g by
// less than its FP32 rounding (~1e-7 of sum |terms|); the FP32 stage leaves
// them to the FP64 step, which sums every kept term.
template <int D>
__device__ __forceinline__ Root32 root_eval32(const MfRbfDev &R, const float *hc, const int *near,
                                              int ns, const int *midl, int nm, const float *x1hi,
                                              const float *x1lo, const float *dir32, float dd32,
                                              float b32, float t) {
  const int lane = threadIdx.x & 31;
  const float g2 = (float)(R.gamma * 1.4426950408889634);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s1a = 0.f;
  const int total = ns + nm;
#pragma unroll 2
  for (int i = lane; i < total; i += 32) {
    const bool strong = i < ns;
    const int c = strong ? i : HC_STRONG + (i - ns);
    float A, Bp, al;
    if (strong ? i < HC_STRONG : i - ns < HC_MID) {
      A = hc[c];
      Bp = hc[HC_ALL + c];
      al = hc[2 * HC_ALL + c];
    } else {
      const int j = strong ? near[i] : midl[i - ns];
      term_ab<D>(R, j, x1hi, x1lo, dir32, A, Bp, al);
    }
    const float proj = fmaf(t, dd32, Bp);
    const float r2 = fmaf(t, proj + Bp, A);
    const float e = al * ex2_approx(-g2 * r2);
    s0 += e;
    s1 = fmaf(e, proj, s1);
    s1a = fmaf(fabsf(e), fabsf(proj), s1a);
    s2 = fmaf(e * proj, proj, s2);
  }
  warp_sum4(s0, s1, s1a, s2);
  const float gm = (float)R.gamma;
  Root32 r;
  r.g = s0 + b32;
  r.gp = -2.f * gm * s1;
  r.gpa = 2.f * gm * s1a;
  r.gpp = 4.f * gm * gm * s2 - 2.f * gm * dd32 * s0;
  return r;
}

// The FP32 part of a root evaluation at xs: the mid entries, then the weak
// ones, as one lane-strided list (accumulated into acc.wf / wg / weak).
// With hc (the deferred step, whose point is x1 + tc dir with tc the FP32
// stage's t, exactly), the weak entries that the screen cached are
// evaluated from A, Bp and alpha (r2 = A + tc (Bp + proj)); their |terms|
// go to acc.weakc, bounded by root_rel_cached instead of R.weak_rel.
template <bool GRAD, int D>
__device__ __forceinline__ void root_fp32_part(const MfRbfDev &R, const int *near, int nw,
                                               const int *midl, int nm, const Split32<D> &xs,
                                               F64Acc &acc, const float *hc = nullptr,
                                               float tc = 0.f, float dd32 = 0.f) {
  const int lane = threadIdx.x & 31;
  const int nr = nm + nw;
  const float g2 = (float)(R.gamma * 1.4426950408889634);
  for (int i = lane; i < nr; i += 32) {
    const int w = i - nm;
    if (hc && w >= 0 && w < HC_WEAK) {
      const int c = HC_STRONG + HC_MID + w;
      const float A = hc[c], Bp = hc[HC_ALL + c], al = hc[2 * HC_ALL + c];
      const float proj = fmaf(tc, dd32, Bp);
      const float r2 = fmaf(tc, proj + Bp, A);
      const float e = al * ex2_approx(-g2 * r2);
      acc.wf += e;
      acc.weakc += fabsf(e);
      if (GRAD) acc.wg = fmaf(e, proj, acc.wg);
    } else {
      const int j = i < nm ? midl[i] : near[NEAR_CAP - 1 - w];
      f32_weak_term<GRAD, D>(R, xs, j, acc);
    }
  }
}

// Relative error bound of a cached weak term on an edge with |dir|^2 = dd32
// (every kept vector lies within the screen radius sqrt(rs2) of the segment;
// 1.1 covers this bound's own FP32 rounding).
__device__ __forceinline__ float root_rel_cached(const MfRbfDev &R, int d, float dd32, float rs2) {
  const float q = sqrtf(rs2) + 2.f * sqrtf(dd32);
  return 1.1f * ((float)d + 8.f) * 5.9604644775390625e-08f * (float)R.gamma * q * q +
         9.5367431640625e-07f + 2.f * 5.9604644775390625e-08f;
}

// FP64 evaluation of g and g' at x over the near list (all lanes); xs is x
// split into FP32 hi/lo parts for the weak terms.
template <bool ALL_STRONG, bool GRAD, int D>
__device__ __forceinline__ F64Acc root_eval64(const MfRbfDev &R, const int *near, int ns, int nw,
                                              const int *midl, int nm, const double *x,
                                              const double *dir, const Split32<D> &xs,
                                              unsigned long long *terms) {
  const int lane = threadIdx.x & 31;
  F64Acc acc = {0.0, 0.0, 0.f, 0.f, 0.f, 0.f};
  for (int i = lane; i < ns; i += 32) f64_term<GRAD, D>(R, x, dir, near[i], acc);
  // mid entries, then weak ones, as one list
  const int nr = nm + nw;
  if (ALL_STRONG) {
    for (int i = lane; i < nr; i += 32) {
      const int j = i < nm ? midl[i] : near[NEAR_CAP - 1 - (i - nm)];
      f64_term<GRAD, D>(R, x, dir, j, acc);
    }
  } else {
    root_fp32_part<GRAD, D>(R, near, nw, midl, nm, xs, acc);
  }
  terms[0] += ns + (ALL_STRONG ? nr : 0);
  terms[1] += ALL_STRONG ? 0 : nr;
  acc.f = mf_warp_sum_d(acc.f) + (double)mf_warp_sum_f(acc.wf) + R.b;
  acc.weak = mf_warp_sum_f(acc.weak);
  acc.g = GRAD ? -2.0 * R.gamma * (mf_warp_sum_d(acc.g) + (double)mf_warp_sum_f(acc.wg)) : 0.0;
  return acc;
}

// Solves the root of edge e (all lanes of the warp); near: NEAR_CAP ints,
// qs / qw: 64-entry queues, all in this warp's shared memory.  src (srcn
// entries, ascending) lists the support vectors that can pass the segment
// screen (a group screen's survivors); NULL screens all of them.  FP64 work
// that is the same for every lane (coordinates, their splits) runs once per
// axis: lane k < d computes axis k and shuffles broadcast it.
// The FP32 part of a root evaluation (mid and weak terms) errs by at most
// weak_rel * sum|terms|; with the dropped terms (drop_bound) that must stay
// below 1e-10 |g'| (t then moves by at most 1e-10), or below the vertex
// evaluation's own limit, whichever is larger.  Otherwise the point is
// evaluated again with every kept term in FP64.
// (The check runs in FP32: the 1.01 factor covers its roundings.)
__device__ __forceinline__ bool root_fp32_part_too_coarse(const MfRbfDev &R, float weak, float gp,
                                                          bool fast) {
  const float lim = fmaxf(R.weak_limit32, (fast ? 0.99e-7f : 0.99e-10f) * fabsf(gp) -
                                              (fast ? R.drop_bound32_fast : R.drop_bound32));
  return weak * (1.01f * R.weak_rel32) > lim;
}

// A root step handed to the lane-per-edge FP64 kernels (k_roots_terms,
// k_roots_finish): the edge (~0: none), the FP32 stage's t (where the FP64
// evaluation happens), the reused g' there and |g''|, the FP32 part of g at
// t (mid and weak terms, already checked against its error bound), and its
// strong entries: ns of them, in the 8-entry chunks from chunk ch on.
struct __align__(16) RootRec {
  unsigned long long e;
  float t, gp, gpp, wf;
  uint32_t ch, ns;
};
#define DEFER_CHUNK 8

// The FP64 end points of edge e on axis k, in mf_vertex_x's operation order:
// x1 = x(y), x2 = x(y + e(mask)), dir = x2 - x1.
__device__ __forceinline__ void root_ends64(const MfFrame &F, double cs1, double cs2, int32_t yk,
                                            uint32_t bit, int k, double &x1, double &dir) {
  x1 = __dadd_rn(__dmul_rn(F.lam, __dsub_rn((double)yk, cs1)), F.o[k]);
  const double x2 = __dadd_rn(__dmul_rn(F.lam, __dsub_rn((double)(yk + (int32_t)bit), cs2)), F.o[k]);
  dir = __dsub_rn(x2, x1);
}

// Per-warp shared state of the FP64 stage (the point, the direction and the
// FP32 split of the point): warp-uniform values kept out of registers.
struct RootWarpState {
  double x[MF_MAXD], dir[MF_MAXD];
  float hl[3 * MF_MAXD];  // Split32<D> image: hi[D], lo[D], dir[D]
};

// ep32 / ep64: the chunk's end points from k_roots_prep (edge e at row
// e - ep0), or NULL (every lane k < d then computes axis k here in FP64).
template <int D>
__device__ void root_edge(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B, uint64_t e,
                          double tol, const int *src, int srcn, int *near, int *midl, float *hc,
                          int *qs, int *qw,
                          RootWarpState *ws, unsigned long long &evals, unsigned long long *terms,
                          bool fast, bool defer, const float *ep32, const double *ep64,
                          uint64_t ep0) {
  const int lane = threadIdx.x & 31;
  const int d = dim_of<D>(F.d);
  const unsigned lt = (1u << lane) - 1u;
  const float g32 = (float)R.gamma;
  const int ko = lane < d ? lane : 0;  // this lane's axis
  double *dir = ws->dir, *x = ws->x;
  Split32<D> &xs = *reinterpret_cast<Split32<D> *>(ws->hl);
  // FP64 end points on this lane's axis
  double x1o = 0.0, diro = 0.0;
  float hio, loo, d32o, f0f, f1f;
  bool s1;
  if (ep32) {
    const uint64_t r = e - ep0;
    const float *row = ep32 + r * (uint64_t)MF_EP_ROW(d);
    hio = lane < d ? row[lane] : 0.f;
    loo = lane < d ? row[d + lane] : 0.f;
    d32o = lane < d ? row[2 * d + lane] : 0.f;
    f0f = row[3 * d];
    f1f = row[3 * d + 1];
    s1 = row[3 * d + 2] != 0.f;
    x1o = ep64[r * 2 * d + ko];
    diro = ep64[r * 2 * d + d + ko];
  } else {
    long long sy = 0;
    int32_t yo = 0;
#pragma unroll
    for (int k = 0; k < D; k++) {
      if (k < d) {
        const int32_t v = B.edge_y[e * d + k];
        sy += v;
        if (k == ko) yo = v;
      }
    }
    const uint32_t mask = B.edge_mask[e] & ((1u << d) - 1u);
    const double cs1 = __dmul_rn(F.c, (double)sy);
    const double cs2 = __dmul_rn(F.c, (double)(sy + __popc(mask)));
    root_ends64(F, cs1, cs2, yo, (mask >> ko) & 1u, ko, x1o, diro);
    hio = (float)x1o;
    loo = (float)(x1o - (double)hio);
    d32o = (float)diro;
    const double f0 = B.edge_f[2 * e], f1 = B.edge_f[2 * e + 1];
    s1 = f0 >= 0.0;
    f0f = (float)f0;
    f1f = (float)f1;
  }
  float x1hi[D], x1lo[D], dir32[D];
  float dd32 = 0.f;
  if (lane < D) {
    dir[lane] = lane < d ? diro : 0.0;
    xs.dir[lane] = lane < d ? d32o : 0.f;
  }
#pragma unroll
  for (int k = 0; k < D; k++) {
    x1hi[k] = k < d ? __shfl_sync(FULL, hio, k) : 0.f;
    x1lo[k] = k < d ? __shfl_sync(FULL, loo, k) : 0.f;
    dir32[k] = k < d ? __shfl_sync(FULL, d32o, k) : 0.f;
    dd32 = fmaf(dir32[k], dir32[k], dd32);
  }
  // 1. segment screen: with u = x1 - s (hi/lo differences), A = |u|^2 and
  //    Bp = u . dir (the cached terms), the squared distance from s to the
  //    segment is A + t (2 Bp + t |dir|^2) at t = clamp(-Bp / |dir|^2, 0, 1).
  int ns = 0, nm = 0, nw = 0;
  const float inv_dd = 1.f / dd32;
  const float shift64 = 0.5f - (fast ? ROOT_TAU_SHIFT_FAST : ROOT_TAU_SHIFT);
  // the mixed paths (fast) drop at most 1e-12 instead of 1e-13
  const float rs2 = fast ? R.screen_r2_fast : R.screen_r2;
  // one round: lane tests vector j (gathered row for a group list, or the
  // coalesced coordinate arrays) and the survivors are compacted
  auto screen_round = [&](bool valid, int j, bool gathered) {
    bool keep = false, strong = false, strong64 = false;
    float cA = 0.f, cB = 0.f, al = 0.f, s32 = 0.f;
    if (valid) {
      float c[2 * D];
      if (gathered) {
        sv_row<D>(R, j, c, al, s32);
      } else {
#pragma unroll
        for (int k = 0; k < D; k++) {
          c[2 * k] = k < d ? R.sv32[(int64_t)k * R.n + j] : 0.f;
          c[2 * k + 1] = k < d ? R.svlo32[(int64_t)k * R.n + j] : 0.f;
        }
        al = R.alpha32[j];
        s32 = R.strong32[j];
      }
      // term_ab's operations
#pragma unroll
      for (int k = 0; k < D; k++) {
        if (k < d) {
          const float u = (x1hi[k] - c[2 * k]) + (x1lo[k] - c[2 * k + 1]);
          cA = fmaf(u, u, cA);
          cB = fmaf(u, dir32[k], cB);
        }
      }
      const float tt = fminf(fmaxf(-cB * inv_dd, 0.f), 1.f);
      const float r2 = fmaf(tt, fmaf(tt, dd32, 2.f * cB), cA);
      keep = r2 <= rs2;
      strong = g32 * r2 < s32 + 0.5f;
      strong64 = g32 * r2 < s32 + shift64;
    }
    // strong64 entries fill near from the front, weak ones from the back,
    // mid ones (strong, not strong64) fill midl
    const unsigned ms = __ballot_sync(FULL, keep && strong64);
    const unsigned mm = __ballot_sync(FULL, keep && strong && !strong64);
    const unsigned mw = __ballot_sync(FULL, keep && !strong);
    const int cs = ns + __popc(ms & lt), cm = nm + __popc(mm & lt), cw = nw + __popc(mw & lt);
    if (keep && strong64 && cs + nw < NEAR_CAP) near[cs] = j;
    if (keep && strong && !strong64 && cm < MID_CAP) midl[cm] = j;
    if (keep && strong && (strong64 ? cs < HC_STRONG : cm < HC_MID)) {
      const int c = strong64 ? cs : HC_STRONG + cm;
      hc[c] = cA;
      hc[HC_ALL + c] = cB;
      hc[2 * HC_ALL + c] = al;
    }
    if (keep && !strong && cw < HC_WEAK) {
      const int c = HC_STRONG + HC_MID + cw;
      hc[c] = cA;
      hc[HC_ALL + c] = cB;
      hc[2 * HC_ALL + c] = al;
    }
    if (keep && !strong && ns + cw < NEAR_CAP) near[NEAR_CAP - 1 - cw] = j;
    ns += __popc(ms);
    nm += __popc(mm);
    nw += __popc(mw);
  };
  if (!src && B.vlist) {
    // the base vertex's list from its FP64 evaluation: a superset of the
    // vectors this screen can keep (its radius covers the screen radius
    // around every point of the edge); k_roots_prep has looked it up
    uint32_t nl = MF_NO_LIST;
    unsigned long long off = 0;
    if (ep32) {
      const float *row = ep32 + (e - ep0) * (uint64_t)MF_EP_ROW(d) + 3 * d + 3;
      nl = __float_as_uint(row[0]);
      off = (unsigned long long)__float_as_uint(row[1]) |
            ((unsigned long long)__float_as_uint(row[2]) << 32);
    } else if (lane == 0) {
      int32_t yv[MF_MAXD];
#pragma unroll
      for (int k = 0; k < MF_MAXD; k++) yv[k] = k < d ? B.edge_y[e * d + k] : 0;
      const uint64_t slot = mf_table_find<2>(B.vtab_key, B.vtab_mask, mf_vertex_key(F, yv));
      if (slot != ~0ull) {
        const uint32_t vi = B.vtab_idx[slot];
        nl = B.vlist_n[vi];
        off = B.vlist_off[vi];
      }
    }
    nl = __shfl_sync(FULL, nl, 0);
    off = __shfl_sync(FULL, off, 0);
    if (nl != MF_NO_LIST) {
      src = B.vlist + off;
      srcn = (int)nl;
    }
  }
  if (src) {
    for (int base = 0; base < srcn; base += 32) {
      const int i = base + lane;
      screen_round(i < srcn, i < srcn ? src[i] : 0, true);
    }
  } else {
    // whole blocks of 32 vectors whose box lies beyond the prefilter ball
    // (looser by 1e-3 for the rounding of the two paths) are skipped
    // (every segment point lies within |dir|/2 of the midpoint, so a vector
    // farther than r_s + |dir|/2 from it, with a rounding margin, cannot
    // pass)
    const float pre = (sqrtf(rs2) + 0.5f * sqrtf(dd32)) * 1.0001f + 1e-5f;
    const float box2 = pre * pre * 1.001f + 1e-5f;
    for (int bb0 = 0; bb0 < R.nblk; bb0 += 32) {
      bool bkeep = false;
      if (bb0 + lane < R.nblk) {
        float q2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; k++)
          if (k < d) {
            const float m = fmaf(0.5f, dir32[k], x1hi[k]);
            const float lo = R.blk_lo[(int64_t)k * R.nblk + bb0 + lane];
            const float hi = R.blk_hi[(int64_t)k * R.nblk + bb0 + lane];
            const float t = fmaxf(fmaxf(lo - m, m - hi), 0.f);
            q2 = fmaf(t, t, q2);
          }
        bkeep = q2 <= box2;
      }
      unsigned bm = __ballot_sync(FULL, bkeep);
      while (bm) {
        const int jj = (bb0 + __ffs(bm) - 1) * 32 + lane;
        bm &= bm - 1;
        screen_round(jj < R.n, jj, false);
      }
    }
  }
  __syncwarp();
  const bool overflow = ns + nw > NEAR_CAP || nm > MID_CAP;
  if (overflow && lane == 0) atomicAdd(&B.cnt->root_overflow, 1ull);
  // 2. FP32 Halley iteration (cubic: the evaluation yields g'' anyway),
  //    bracketed, from the linear interpolant of the end values
  float t32 = f0f / (f0f - f1f);
  if (!(t32 > 0.f && t32 < 1.f)) t32 = 0.5f;
  // the last FP32 evaluation: g'', g', t, and whether its g' is trusted
  float gpp = INFINITY, gp32 = 0.f, t_eval = 0.f;
  bool gp_ok = false;
  if (!overflow) {
    const float b32 = (float)R.b;
    float lo = 0.f, hi = 1.f;
    for (int it = 0; it < 12; it++) {
      const Root32 r = root_eval32<D>(R, hc, near, ns, midl, nm, x1hi, x1lo, dir32, dd32, b32, t32);
      terms[1] += ns + nm;  // FP32 terms of this Halley evaluation
      gpp = r.gpp;
      gp32 = r.gp;
      t_eval = t32;
      // per-term FP32 errors stay below ~1e-5 relative, so with at most 4x
      // cancellation g' is good to ~5e-5
      gp_ok = r.gpa <= 4.f * fabsf(r.gp);
      if ((r.g >= 0.f) == s1) lo = t32; else hi = t32;
      const float den = 2.f * r.gp * r.gp - r.g * r.gpp;
      const bool halley = den > 0.f;
      float tn = halley ? t32 - 2.f * r.g * r.gp / den : t32 - r.g / r.gp;
      const bool inside = tn > lo && tn < hi;
      if (!inside) tn = 0.5f * (lo + hi);
      const float step = fabsf(tn - t32);
      t32 = tn;
      // a Halley step of size s leaves an error of order s^3: below 1e-3
      // the FP32 noise floor is reached and the FP64 step finishes
      if (step <= 2e-6f || (halley && inside && step <= 1e-3f)) break;
    }
  }
  // 3. FP64 Newton with a kept bracket.  Values that only steer the
  //    iteration (g', step sizes, the acceptance tests) stay in FP32: each
  //    FP64 instruction occupies the FP64 pipe for the whole warp.
  double t = (double)t32, xo = 0.0;
  const float gppf = fabsf(gpp), tolf = (float)tol;
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 64; it++) {
    xo = __dadd_rn(x1o, __dmul_rn(t, diro));
    const float xho = (float)xo, xlo = (float)(xo - (double)xho);
    __syncwarp();  // the previous evaluation has read the state
    if (lane < D) {
      x[lane] = lane < d ? xo : 0.0;
      xs.hi[lane] = lane < d ? xho : 0.f;
      xs.lo[lane] = lane < d ? xlo : 0.f;
    }
    __syncwarp();
    F64Acc a;
    // The first step reuses the FP32 stage's g', carried to t by its g''
    // (relative error below ~5e-5 when the FP32 sum had little
    // cancellation: a final step of at most 1e-5 then errs by < 1e-9);
    // later steps take the FP64 g'.
    float gpf = 0.f;
    bool reuse = false;
    if (it == 0 && !overflow && gp_ok) {
      gpf = fmaf(gpp, (float)t - t_eval, gp32);
      reuse = gp32 != 0.f && isfinite(gpf) && fabsf(gpf) > 0.5f * fabsf(gp32);
    }
    if (defer && reuse) {
      // the common case -- one FP64 step with the reused g' -- runs lane per
      // edge in k_roots_terms / k_roots_finish: this warp computes the
      // step's FP32 part and hands over the strong entries (unless the
      // part's error bound is too coarse or the pools are full; the step
      // then runs here)
      F64Acc part = {0.0, 0.0, 0.f, 0.f, 0.f, 0.f};
      root_fp32_part<false, D>(R, near, nw, midl, nm, xs, part, hc, t32, dd32);
      const float wf = mf_warp_sum_f(part.wf), weak = mf_warp_sum_f(part.weak);
      const float weakc = mf_warp_sum_f(part.weakc);
      // the cached weak terms count with their own bound, as a multiple of
      // R.weak_rel's
      const float kc = fmaxf(root_rel_cached(R, d, dd32, rs2) / R.weak_rel32, 1.f);
      if (!root_fp32_part_too_coarse(R, fmaf(weakc, kc, weak), gpf, fast)) {
        const int nch = (ns + DEFER_CHUNK - 1) / DEFER_CHUNK;
        unsigned long long at = 0, lat = 0;
        if (lane == 0) {
          at = atomicAdd(&B.cnt->n_defer, 1ull);
          lat = atomicAdd(&B.cnt->n_defer_list, (unsigned long long)nch * DEFER_CHUNK);
        }
        at = __shfl_sync(FULL, at, 0);
        lat = __shfl_sync(FULL, lat, 0);
        const bool rec_ok = at < B.defer_cap;
        const bool ok = rec_ok && lat + (unsigned long long)nch * DEFER_CHUNK <= B.defer_list_cap;
        const uint64_t c0 = lat / DEFER_CHUNK, ncap = B.defer_list_cap / DEFER_CHUNK;
        if (ok) {
          for (int i = lane; i < nch * DEFER_CHUNK; i += 32) B.defer_list[lat + i] = i < ns ? near[i] : -1;
          for (int c = lane; c < nch; c += 32) B.defer_chunk[c0 + c] = (uint32_t)at;
        } else {
          // chunks granted within the pool stay unused
          for (uint64_t c = c0 + lane; c < c0 + nch && c < ncap; c += 32) B.defer_chunk[c] = ~0u;
        }
        if (lane == 0 && rec_ok) {
          RootRec r;
          r.e = ok ? e : ~0ull;
          r.t = t32;
          r.gp = gpf;
          r.gpp = gppf;
          r.wf = wf;
          r.ch = (uint32_t)c0;
          r.ns = (uint32_t)ns;
          reinterpret_cast<RootRec *>(B.defer_rec)[at] = r;
        }
        if (ok) {
          terms[1] += nm + nw;
          return;
        }
      }
    }
    if (overflow) {
      a = warp_f64<true, D>(R, x, dir, qs, qw, terms);
      gpf = (float)a.g;
    } else if (reuse) {
      a = root_eval64<false, false, D>(R, near, ns, nw, midl, nm, x, dir, xs, terms);
      if (root_fp32_part_too_coarse(R, a.weak, gpf, fast))
        a = root_eval64<true, false, D>(R, near, ns, nw, midl, nm, x, dir, xs, terms);
    } else {
      a = root_eval64<false, true, D>(R, near, ns, nw, midl, nm, x, dir, xs, terms);
      gpf = (float)a.g;
      if (root_fp32_part_too_coarse(R, a.weak, gpf, fast)) {
        a = root_eval64<true, true, D>(R, near, ns, nw, midl, nm, x, dir, xs, terms);
        gpf = (float)a.g;
      }
    }
    evals++;
    // sign of f from its bits (f = +-0 ends the iteration)
    const long long fb = __double_as_longlong(a.f);
    if ((fb << 1) == 0) break;
    if ((fb >= 0) == s1) lo = t; else hi = t;
    // the derivative only steers the step: its reciprocal in FP32 suffices
    double tn = fma(-a.f, (double)(1.0f / gpf), t);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    const float step = fabsf((float)(tn - t));
    t = tn;
    // a first step of s after the FP32 stage errs by ~|g''| s^2 / (2 |g'|)
    // (Newton remainder) plus 5e-5 s (the reused g'): below 1e-9 for
    // s <= 1e-5 and the remainder test, below 2e-7 in the fast mode
    if (step <= tolf || step <= 1e-7f || hi - lo <= 9.094947017729282e-13 ||
        (it == 0 && step <= (fast ? 1e-3f : 1e-5f) &&
         gppf * step * step <= (fast ? 1e-7f : 5e-11f) * fabsf(gpf)))
      break;
  }
  if (lane == 0) B.edge_t[e] = t;
  if (lane < d) B.edge_pt[e * d + lane] = __dadd_rn(x1o, __dmul_rn(t, diro));
}

__device__ __forceinline__ void root_flush(const MfTraceBufs &B, unsigned long long evals,
                                           const unsigned long long *terms) {
  if ((threadIdx.x & 31) == 0 && (evals || terms[0] || terms[1])) {
    if (evals) atomicAdd(&B.cnt->root_evals, evals);
    if (terms[0]) atomicAdd(&B.cnt->root_terms, terms[0]);
    if (terms[1]) atomicAdd(&B.cnt->root_terms_weak, terms[1]);
  }
}

#define GROUP_CAP 1024

// Group screen of edges [e0, e0 + ng) (consecutive edges of the BFS list lie
// close together): c = mean of their 2 ng endpoints, Rg = largest endpoint
// distance from c.  A support vector within r_s of a point of any of these
// segments lies within r_s + Rg of c (the ball holds the segments), so the
// list of those (ascending, margin 1e-4 relative + 1e-5 over the FP32
// rounding) contains every vector the per-edge segment screen keeps, which
// then sees the same candidates in the same order.  Returns the count, or -1
// if more than GROUP_CAP pass (the edges then screen all vectors).
template <int D>
__device__ int group_screen(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B, uint64_t e0,
                            int ng, float rs, int *glist) {
  const int lane = threadIdx.x & 31;
  const int d = dim_of<D>(F.d);
  const unsigned lt = (1u << lane) - 1u;
  const bool have = lane < ng;
  float a[D], b[D];
  {
    int32_t y[MF_MAXD];
    double xa[MF_MAXD], xb[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = (have && k < d) ? B.edge_y[(e0 + lane) * d + k] : 0;
    mf_vertex_x(F, y, xa);
    mf_add_mask(d, y, have ? B.edge_mask[e0 + lane] : 0u, 1);
    mf_vertex_x(F, y, xb);
#pragma unroll
    for (int k = 0; k < D; k++) {
      a[k] = (float)xa[k];
      b[k] = (float)xb[k];
    }
  }
  float c[D];
#pragma unroll
  for (int k = 0; k < D; k++) c[k] = mf_warp_sum_f(have ? a[k] + b[k] : 0.f) / (float)(2 * ng);
  float r2 = 0.f;
  if (have) {
    float da = 0.f, db = 0.f;
#pragma unroll
    for (int k = 0; k < D; k++) {
      if (k < d) {
        da = fmaf(a[k] - c[k], a[k] - c[k], da);
        db = fmaf(b[k] - c[k], b[k] - c[k], db);
      }
    }
    r2 = fmaxf(da, db);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(FULL, r2, o));
  const float lim = (rs + sqrtf(r2)) * 1.0001f + 1e-5f, lim2 = lim * lim;
  int gn = 0;
  for (int base = 0; base < R.n; base += 32) {
    const int j = base + lane;
    bool keep = false;
    if (j < R.n) {
      float s2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; k++) {
        if (k < d) {
          const float t = R.sv32[(int64_t)k * R.n + j] - c[k];
          s2 = fmaf(t, t, s2);
        }
      }
      keep = s2 <= lim2;
    }
    const unsigned m = __ballot_sync(FULL, keep);
    const int pos = gn + __popc(m & lt);
    if (keep && pos < GROUP_CAP) glist[pos] = j;
    gn += __popc(m);
  }
  __syncwarp();
  return gn <= GROUP_CAP ? gn : -1;
}

// Root solve of edges [e0, e0 + n) (list == NULL), or of the edges listed
// in list[0 .. min(*n_list, n)) (the redo queue).  defer: hand the common
// single-step case to k_roots_terms / k_roots_finish, with the end points
// from k_roots_prep (B.ep32, rows from e0).
template <int D, int MINB>
__global__ void __launch_bounds__(ROOT_WARPS * 32, MINB) k_roots_f64(
    MfFrame F, MfRbfDev R, MfTraceBufs B, uint64_t e0, uint64_t n_edges, double tol, int group,
    int fast, int defer, const uint64_t *list, const unsigned long long *n_list) {
  const float *ep32 = defer ? B.ep32 : nullptr;
  const double *ep64 = defer ? B.defer_x : nullptr;
  __shared__ int snear[ROOT_WARPS][NEAR_CAP];
  __shared__ int smid[ROOT_WARPS][MID_CAP];
  __shared__ float shc[ROOT_WARPS][3 * HC_ALL];
  __shared__ int sq[ROOT_WARPS][2][64];
  __shared__ RootWarpState sws[ROOT_WARPS];
  extern __shared__ int sgrp_all[];  // [ROOT_WARPS][GROUP_CAP] when group > 1
  const int w = threadIdx.x >> 5;
  int *sgrp = sgrp_all + w * GROUP_CAP;
  const uint64_t nwarps = (uint64_t)gridDim.x * ROOT_WARPS;
  const float rs = sqrtf(R.screen_r2);
  unsigned long long evals = 0, terms[2] = {0, 0};
  if (list) {
    const uint64_t nl = *n_list < n_edges ? *n_list : n_edges;
    for (uint64_t i = (uint64_t)blockIdx.x * ROOT_WARPS + w; i < nl; i += nwarps)
      root_edge<D>(F, R, B, list[i], tol, nullptr, 0, snear[w], smid[w], shc[w], sq[w][0], sq[w][1],
                   &sws[w], evals, terms, fast != 0, false, nullptr, nullptr, 0);
  } else if (group <= 1) {
    for (uint64_t i = (uint64_t)blockIdx.x * ROOT_WARPS + w; i < n_edges; i += nwarps)
      root_edge<D>(F, R, B, e0 + i, tol, nullptr, 0, snear[w], smid[w], shc[w], sq[w][0], sq[w][1],
                   &sws[w], evals, terms, fast != 0, defer != 0, ep32, ep64, e0);
  } else {
    const uint64_t G = (uint64_t)group;
    for (uint64_t g0 = ((uint64_t)blockIdx.x * ROOT_WARPS + w) * G; g0 < n_edges; g0 += nwarps * G) {
      const int ng = (int)(n_edges - g0 < G ? n_edges - g0 : G);
      const int gn = group_screen<D>(F, R, B, e0 + g0, ng, rs, sgrp);
      for (int q = 0; q < ng; q++)
        root_edge<D>(F, R, B, e0 + g0 + q, tol, gn >= 0 ? sgrp : nullptr, gn, snear[w], smid[w],
                     shc[w], sq[w][0], sq[w][1], &sws[w], evals, terms, fast != 0, defer != 0, ep32, ep64,
                     e0);
    }
  }
  root_flush(B, evals, terms);
}

// The end points of edges [e0, e0 + n), one thread per edge, for the warp
// kernel of the deferred path: FP32 rows (x1 hi, x1 lo, dir, f(x1), f(x2),
// [f(x1) >= 0]) in B.ep32 and the FP64 x1, dir in the first 2d cap doubles
// of B.defer_x.
template <int D>
__global__ void __launch_bounds__(256) k_roots_prep(MfFrame F, MfTraceBufs B, uint64_t e0, uint64_t n) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int d = dim_of<D>(F.d);
  const uint64_t e = e0 + i;
  long long sy = 0;
  int32_t y[D];
#pragma unroll
  for (int k = 0; k < D; k++) {
    y[k] = k < d ? B.edge_y[e * d + k] : 0;
    sy += y[k];
  }
  const uint32_t mask = B.edge_mask[e] & ((1u << d) - 1u);
  const double cs1 = __dmul_rn(F.c, (double)sy);
  const double cs2 = __dmul_rn(F.c, (double)(sy + __popc(mask)));
  float *row = B.ep32 + i * (uint64_t)MF_EP_ROW(d);
  double *row64 = B.defer_x + i * 2 * (uint64_t)d;
#pragma unroll
  for (int k = 0; k < D; k++) {
    if (k < d) {
      double x1, dir;
      root_ends64(F, cs1, cs2, y[k], (mask >> k) & 1u, k, x1, dir);
      const float hi = (float)x1;
      row[k] = hi;
      row[d + k] = (float)(x1 - (double)hi);
      row[2 * d + k] = (float)dir;
      row64[k] = x1;
      row64[d + k] = dir;
    }
  }
  const double f0 = B.edge_f[2 * e], f1 = B.edge_f[2 * e + 1];
  row[3 * d] = (float)f0;
  row[3 * d + 1] = (float)f1;
  row[3 * d + 2] = f0 >= 0.0 ? 1.f : 0.f;
  // the base vertex's root-screen list (MF_NO_LIST: none)
  uint32_t nl = MF_NO_LIST;
  unsigned long long off = 0;
  if (B.vlist) {
    int32_t yv[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) yv[k] = k < d ? y[k < D ? k : 0] : 0;
    const uint64_t slot = mf_table_find<2>(B.vtab_key, B.vtab_mask, mf_vertex_key(F, yv));
    if (slot != ~0ull) {
      const uint32_t vi = B.vtab_idx[slot];
      nl = B.vlist_n[vi];
      off = B.vlist_off[vi];
    }
  }
  row[3 * d + 3] = __uint_as_float(nl);
  row[3 * d + 4] = __uint_as_float((uint32_t)off);
  row[3 * d + 5] = __uint_as_float((uint32_t)(off >> 32));
}

// The evaluation point x = x1 + t (x2 - x1) of each deferred step (thread
// per record), in root_edge's operation order, split into three floats per
// coordinate (x = x1 + x2 + x3 exactly) for the double-float terms: record
// i at B.defer_x3[3 d i].
template <int D>
__global__ void __launch_bounds__(256) k_roots_x(MfFrame F, MfTraceBufs B, uint64_t cap, uint64_t e0) {
  const unsigned long long nrec = B.cnt->n_defer < cap ? B.cnt->n_defer : cap;
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= nrec) return;
  const int d = dim_of<D>(F.d);
  const RootRec rec = reinterpret_cast<const RootRec *>(B.defer_rec)[i];
  if (rec.e == ~0ull) return;
  // x1 and dir as k_roots_prep computed them (row rec.e - e0)
  const double *row64 = B.defer_x + (rec.e - e0) * 2 * (uint64_t)d;
  const double t = (double)rec.t;
  float *xp = B.defer_x3 + i * 3 * (uint64_t)d;
#pragma unroll
  for (int k = 0; k < D; k++) {
    if (k < d) {
      const double x = __dadd_rn(row64[k], __dmul_rn(t, row64[d + k]));
      const float h = (float)x;
      const double r = x - (double)h;
      const float m = (float)r;
      xp[3 * k] = h;
      xp[3 * k + 1] = m;
      xp[3 * k + 2] = (float)(r - (double)m);
    }
  }
}

// Sum of the strong terms of each 8-entry chunk (thread per chunk, so lanes
// differ by at most the padding of a list's last chunk): alpha_j
// exp(-gamma |x - s_j|^2) in list order, at the chunk's record's point, in
// double-float arithmetic on the FP32 pipe:
//  - u = x - s from the exact three-float forms of x and s (TwoSums), so u
//    is good to 2^-47 |u| whatever the cancellation;
//  - r2 = sum u_k^2 and z = gamma r2 in double-float;
//  - exp(-z) = 2^(-k/1024) exp(-r), k = round(1024 z / ln 2), |r| <=
//    ln 2 / 2048, ln 2 / 1024 in three pieces (k times the first exact by
//    FMA); exp(-r) = 1 - r + r^2 (1/2 - r/6 + r^2/24), the bracket in FP32
//    (its error is below 2^-46 of the result for |r| <= 3.4e-4, and
//    r^5 / 120 < 4e-20); 2^(-j/1024) from a double-float table;
//  - alpha e in double-float, summed in double-float.
// Each term's relative error stays below (1 + z) 2^-44 (the exponent's
// error grows with z; the rest is a few double-float roundings), so the
// chunk also records w = sum |term| (1 + z): the step's error from these
// sums is below 2^-43 w summed over the chunks (checked in
// k_roots_finish, with a factor 2 to spare).
// ln 2 / 1024 = A + B + C to about 4e-24 relative (each the float nearest
// the remainder)
#define DF_LN2_1024_A 0x1.62e43p-11f
#define DF_LN2_1024_B -0x1.05c61p-39f
#define DF_LN2_1024_C -0x1.950d88p-64f
template <int D>
__global__ void __launch_bounds__(256) k_roots_terms(MfRbfDev R, MfTraceBufs B, uint64_t cap) {
  __shared__ float2 stab[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) stab[i] = R.exp_df[i];
  __syncthreads();
  const unsigned long long nrec = B.cnt->n_defer < cap ? B.cnt->n_defer : cap;
  const unsigned long long nl = B.cnt->n_defer_list;
  const uint64_t nch = (nl < B.defer_list_cap ? nl : B.defer_list_cap) / DEFER_CHUNK;
  const int d = dim_of<D>(R.d);
  const float g1 = (float)R.gamma;
  const MfDf gam = {g1, (float)(R.gamma - (double)g1)};
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nch;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = B.defer_chunk[c];
    if (r >= nrec) continue;
    const float *xp = B.defer_x3 + r * 3 * (uint64_t)d;
    float xa[D], xb[D], xc[D];
#pragma unroll
    for (int k = 0; k < D; k++) {
      xa[k] = k < d ? xp[3 * k] : 0.f;
      xb[k] = k < d ? xp[3 * k + 1] : 0.f;
      xc[k] = k < d ? xp[3 * k + 2] : 0.f;
    }
    const int4 *pl = reinterpret_cast<const int4 *>(B.defer_list + c * DEFER_CHUNK);
    const int4 q0 = pl[0], q1 = pl[1];
    const int js[DEFER_CHUNK] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
    MfDf fs = {0.f, 0.f};
    float w = 0.f;
#pragma unroll
    for (int q = 0; q < DEFER_CHUNK; q++) {
      const int j = js[q];
      if (j < 0 || j >= R.n) continue;
      const float4 *row = reinterpret_cast<const float4 *>(R.sv3 + (int64_t)j * 24);
      float sr[((3 * D + 3) / 4) * 4];
#pragma unroll
      for (int v = 0; v < (3 * D + 3) / 4; v++) {
        const float4 t4 = __ldg(row + v);
        sr[4 * v] = t4.x;
        sr[4 * v + 1] = t4.y;
        sr[4 * v + 2] = t4.z;
        sr[4 * v + 3] = t4.w;
      }
      MfDf r2 = {0.f, 0.f};
#pragma unroll
      for (int k = 0; k < D; k++) {
        if (k < d) {
          // u = (xa - s1) + (xb - s2) + (xc - s3), the first two exactly
          const MfDf a = mf_two_sum(xa[k], -sr[3 * k]);
          const MfDf b = mf_two_sum(xb[k], -sr[3 * k + 1]);
          const MfDf m = mf_two_sum(a.lo, b.hi);
          const float lo = m.lo + (b.lo + (xc[k] - sr[3 * k + 2]));
          const MfDf h = mf_two_sum(a.hi, m.hi);
          const MfDf u = mf_fast_two_sum(h.hi, h.lo + lo);
          // u^2 (the lo^2 term is below 2^-48 u^2)
          const MfDf p = mf_two_prod(u.hi, u.hi);
          r2 = mf_df_add(r2, mf_fast_two_sum(p.hi, fmaf(2.f * u.hi, u.lo, p.lo)));
        }
      }
      const MfDf z = mf_df_mul(gam, r2);
      // k = round(z 1024 / ln 2); r = z - k ln2/1024 in double-float
      const float kf = rintf(z.hi * 1477.3197218702985f);
      const MfDf ka = mf_two_prod(kf, DF_LN2_1024_A);
      MfDf rr = mf_two_sum(z.hi, -ka.hi);
      rr = mf_fast_two_sum(rr.hi, rr.lo + (z.lo - ka.lo) - fmaf(kf, DF_LN2_1024_B, kf * DF_LN2_1024_C));
      // exp(-r) = 1 - r + r^2 (1/2 - r/6 + r^2/24)
      const float rh = rr.hi;
      const float br = fmaf(rh, fmaf(rh, 1.f / 24.f, -1.f / 6.f), 0.5f);
      const MfDf one_r = mf_two_sum(1.f, -rh);
      const MfDf er = mf_fast_two_sum(one_r.hi, one_r.lo + fmaf(rh * rh, br, -rr.lo));
      const int ki = (int)kf;
      const float2 tt = stab[ki & 1023];
      MfDf e = mf_df_mul({tt.x, tt.y}, er);
      const int sh = ki >> 10;  // 2^-sh (z <= ~750, so sh stays far from the float exponent limit)
      e.hi = ldexpf(e.hi, -sh);
      e.lo = ldexpf(e.lo, -sh);
      const MfDf t = mf_df_mul({__ldg(R.alpha32 + j), __ldg(R.alpha_lo32 + j)}, e);
      fs = mf_df_add(fs, t);
      w = fmaf(fabsf(t.hi), 1.f + z.hi, w);
    }
    B.defer_part[c] = (double)fs.hi + (double)fs.lo;
    B.defer_bnd[c] = w;
  }
}

// The deferred FP64 root steps, one thread per record: g = (the chunks'
// sums in order) + (FP32 part) + b at x, one Newton step with the reused g'
// under root_edge's acceptance tests.  Accepted steps write t and the point
// (x1 + t dir in root_edge's order); the others go to the redo queue.
template <int D>
__global__ void __launch_bounds__(256) k_roots_finish(MfFrame F, MfRbfDev R, MfTraceBufs B,
                                                      uint64_t cap, double tol, int fast,
                                                      uint64_t e0) {
  const unsigned long long nrec = B.cnt->n_defer < cap ? B.cnt->n_defer : cap;
  const int d = dim_of<D>(F.d);
  const float tolf = (float)tol;
  unsigned long long terms = 0, evals = 0;
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < nrec) {
    const RootRec rec = reinterpret_cast<const RootRec *>(B.defer_rec)[i];
    if (rec.e != ~0ull) {
      const uint64_t e = rec.e;
      double fs = 0.0;
      float w = 0.f;
      const uint32_t nc = (rec.ns + DEFER_CHUNK - 1) / DEFER_CHUNK;
      for (uint32_t c = 0; c < nc; c++) {
        fs += B.defer_part[rec.ch + c];
        w += B.defer_bnd[rec.ch + c];
      }
      terms += rec.ns;
      evals++;
      const double t = (double)rec.t;
      const double f = fs + (double)rec.wf + R.b;
      double tn = t;
      // the double-float sums' error (2^-43 w, doubled) may move t by at
      // most 2e-10 (1e-7 in the fast mode), beside the FP32 part's 1e-10
      bool ok = 2.f * 0x1p-43f * w <= (fast ? 0.99e-7f : 2e-10f) * fabsf(rec.gp);
      const long long fb = __double_as_longlong(f);
      if (ok && (fb << 1) != 0) {  // f = +-0 keeps t
        const bool s1 = B.edge_f[2 * e] >= 0.0;
        double lo = 0.0, hi = 1.0;
        if ((fb >= 0) == s1) lo = t; else hi = t;
        tn = fma(-f, (double)(1.0f / rec.gp), t);
        ok = tn > lo && tn < hi;
        if (ok) {
          const float step = fabsf((float)(tn - t));
          ok = step <= tolf || step <= 1e-7f || hi - lo <= 9.094947017729282e-13 ||
               (step <= (fast ? 1e-3f : 1e-5f) &&
                rec.gpp * step * step <= (fast ? 1e-7f : 5e-11f) * fabsf(rec.gp));
        }
      }
      if (ok) {
        // x1 and dir as k_roots_prep computed them (row e - e0)
        const double *row64 = B.defer_x + (e - e0) * 2 * (uint64_t)d;
        B.edge_t[e] = tn;
#pragma unroll
        for (int k = 0; k < D; k++)
          if (k < d) B.edge_pt[e * d + k] = __dadd_rn(row64[k], __dmul_rn(tn, row64[d + k]));
      } else {
        const unsigned long long q = atomicAdd(&B.cnt->n_redo, 1ull);
        if (q < cap) B.redo[q] = e;
      }
    }
  }
  // warp totals of the counters
  unsigned long long te = mf_warp_sum_ull(evals), tt = mf_warp_sum_ull(terms);
  if ((threadIdx.x & 31) == 0 && te) {
    atomicAdd(&B.cnt->root_evals, te);
    atomicAdd(&B.cnt->root_terms, tt);
  }
}

// ---------------------------------------------------------------------------
// Batched evaluation and roots: one warp per work item, the item's trace found
// through the plan's prefix array; every slot has its own support vectors,
// precision and tables.
// ---------------------------------------------------------------------------

// Warp-level FP32 evaluation of f at x with the rigorous bound of the mixed
// path (lane-strided sums: each lane adds about n/32 terms, then a 5-level
// tree), all lanes get (f~, bound).
__device__ void warp_f32_bound(const MfRbfDev &R, const double *x, double &f, double &bound) {
  const int lane = threadIdx.x & 31;
  const int d = R.d;
  const float g2 = (float)(R.gamma * 1.4426950408889634);
  float xs[MF_MAXD];
  double xmax = 0.0;
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) {
    xs[k] = k < d ? (float)x[k] : 0.f;
    if (k < d) xmax = fmax(xmax, fabs(x[k]));
  }
  float acc = 0.f, A = 0.f, Q = 0.f;
  for (int j = lane; j < R.n; j += 32) {
    float r2 = 0.f;
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++)
      if (k < d) {
        const float t = xs[k] - R.sv32[(int64_t)k * R.n + j];
        r2 = fmaf(t, t, r2);
      }
    const float al = R.alpha32[j];
    const float e = ex2_approx(-g2 * r2);
    acc = fmaf(al, e, acc);
    const float ae = fabsf(al) * e;
    A += ae;
    Q = fmaf(ae, r2, Q);
  }
  acc = mf_warp_sum_f(acc);
  A = mf_warp_sum_f(A);
  Q = mf_warp_sum_f(Q);
  const double u = 5.9604644775390625e-08;
  const double D = xmax + (double)R.smax;
  const double eta = 2.01 * u * D;
  const double Av = (double)A, Qv = (double)Q;
  const double coord = R.gamma * (2.0 * eta * sqrt((double)d) * sqrt(Av * Qv) + d * eta * eta * Av);
  const double nsum = (double)R.n / 32.0 + 6.0;
  bound = (coord + Av * (9.5367431640625e-07 + (nsum + 2.0) * u) + Qv * R.gamma * (d + 2) * u) * 1.02 +
          1e-30;
  f = (double)acc + R.b;
}

__global__ void __launch_bounds__(EVAL_WARPS * 32) k_b_eval(const MfSlot *slots, const MfBatchPlan *P,
                                                           int n, int recheck) {
  __shared__ int sq[EVAL_WARPS][2][64];
  __shared__ int slist[EVAL_WARPS][LIST_CAP];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long *pfx = recheck ? P->pr : P->pv;
  const unsigned long long total = pfx[n];
  const unsigned long long nwarps = (unsigned long long)gridDim.x * EVAL_WARPS;
  for (unsigned long long item = (unsigned long long)blockIdx.x * EVAL_WARPS + w; item < total;
       item += nwarps) {
    const int t = mf_slot_of(pfx, n, item);
    const MfSlot &S = slots[t];
    // MF_MIXED_BF16 slots are evaluated by the tensor-core tiles
    if (!recheck && S.precision == MF_MIXED_BF16) continue;
    const int d = S.F.d;
    const unsigned long long local = item - pfx[t];
    const uint64_t i = recheck ? (uint64_t)S.B.recheck[P->r0[t] + local] : P->v0[t] + local;
    int32_t y[MF_MAXD];
    double x[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = k < d ? S.B.vert_y[i * d + k] : 0;
    vertex_x_lanes<MF_MAXD>(S.F, y, x);
    const uint32_t slot = S.B.vert_slot[i];
    if (recheck || S.precision == MF_FP64) {
      unsigned long long terms[2] = {0, 0};
      // FP64 slots record the root-screen list in the same pass
      const bool lists = !recheck && S.B.vlist;
      int nl = 0;
      const F64Acc a = warp_f64<false, MF_MAXD>(S.R, x, nullptr, sq[w][0], sq[w][1], terms,
                                                lists ? slist[w] : nullptr, S.B.list_r2, &nl);
      if (lane == 0) {
        mf_vtab_f(S.B, slot) = a.f;
        if (fabs(a.f) < 1e-12) atomicAdd(&S.B.cnt->n_near_zero, 1ull);
        atomicAdd(&S.B.cnt->eval_terms, terms[0]);
        atomicAdd(&S.B.cnt->eval_terms_weak, terms[1]);
      }
      if (lists) store_vertex_list(S.B, i, nl, slist[w]);
    } else {
      double f, bound;
      warp_f32_bound(S.R, x, f, bound);
      if (lane == 0) {
        mf_vtab_f(S.B, slot) = f;
        if (fabs(f) <= fmax(bound, S.band)) {
          const unsigned long long q = atomicAdd(&S.B.cnt->n_recheck, 1ull);
          if (q < S.B.max_vertices) S.B.recheck[q] = (uint32_t)i;
          else atomicOr(&S.B.cnt->err_overflow, 1u);
        }
      }
    }
  }
}

// Root-screen lists of the new vertices of the mixed slots (their
// evaluators do not screen); FP64 slots list in k_b_eval.
__global__ void __launch_bounds__(EVAL_WARPS * 32) k_b_lists(const MfSlot *slots, const MfBatchPlan *P,
                                                            int n) {
  __shared__ int slist[EVAL_WARPS][LIST_CAP];
  const int w = threadIdx.x >> 5;
  const unsigned long long total = P->pv[n];
  const unsigned long long nwarps = (unsigned long long)gridDim.x * EVAL_WARPS;
  for (unsigned long long item = (unsigned long long)blockIdx.x * EVAL_WARPS + w; item < total;
       item += nwarps) {
    const int t = mf_slot_of(P->pv, n, item);
    const MfSlot &S = slots[t];
    if (S.precision == MF_FP64 || !S.B.vlist) continue;
    const uint64_t i = P->v0[t] + (item - P->pv[t]);
    int32_t y[MF_MAXD];
    double x[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) y[k] = k < S.F.d ? S.B.vert_y[i * S.F.d + k] : 0;
    vertex_x_lanes<MF_MAXD>(S.F, y, x);
    const Split32<MF_MAXD> xs = split32<MF_MAXD>(S.F.d, x, nullptr);
    const int nl = warp_vertex_list<MF_MAXD>(S.R, xs.hi, S.B.list_r2, slist[w]);
    store_vertex_list(S.B, i, nl, slist[w]);
  }
}

// Root solve of every slot of dimension D (the plan's pe prefix holds only
// those): warps take runs of `group` consecutive items; a run that crosses a
// slot boundary is split, each part sharing one group screen.
template <int D>
__global__ void __launch_bounds__(ROOT_WARPS * 32, 2) k_b_roots(const MfSlot *slots,
                                                                const MfBatchPlan *P, int n,
                                                                int group) {
  __shared__ int snear[ROOT_WARPS][NEAR_CAP];
  __shared__ int smid[ROOT_WARPS][MID_CAP];
  __shared__ float shc[ROOT_WARPS][3 * HC_ALL];
  __shared__ int sq[ROOT_WARPS][2][64];
  __shared__ RootWarpState sws[ROOT_WARPS];
  extern __shared__ int sgrp_all[];  // [ROOT_WARPS][GROUP_CAP] when group > 1
  const int w = threadIdx.x >> 5;
  int *sgrp = sgrp_all + w * GROUP_CAP;
  const unsigned long long total = P->pe[n];
  const unsigned long long G = group > 1 ? (unsigned long long)group : 1ull;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * ROOT_WARPS;
  for (unsigned long long g0 = ((unsigned long long)blockIdx.x * ROOT_WARPS + w) * G; g0 < total;
       g0 += nwarps * G) {
    const unsigned long long g1 = g0 + G < total ? g0 + G : total;
    for (unsigned long long i = g0; i < g1;) {
      const int t = mf_slot_of(P->pe, n, i);
      const MfSlot &S = slots[t];
      const unsigned long long end = P->pe[t + 1] < g1 ? P->pe[t + 1] : g1;
      const uint64_t e0 = i - P->pe[t];
      const int ng = (int)(end - i);
      const int gn = G > 1 ? group_screen<D>(S.F, S.R, S.B, e0, ng, sqrtf(S.R.screen_r2), sgrp) : -1;
      unsigned long long evals = 0, terms[2] = {0, 0};
      for (int q = 0; q < ng; q++)
        root_edge<D>(S.F, S.R, S.B, e0 + q, S.root_tol, gn >= 0 ? sgrp : nullptr, gn, snear[w],
                     smid[w], shc[w], sq[w][0], sq[w][1], &sws[w], evals, terms,
                     S.precision != MF_FP64 && !(S.flags & MF_ROOTS_FP64_EXACT), false, nullptr,
                     nullptr, 0);
      root_flush(S.B, evals, terms);
      i = end;
    }
  }
}

void mf_b_launch_eval(const MfSlot *slots, MfBatchPlan *P, int n, bool any_mixed, int tc_chunk,
                      int sms, cudaStream_t s) {
  mf_b_launch_plan_eval(slots, P, n, false, s);
  k_b_eval<<<sms * 8, EVAL_WARPS * 32, 0, s>>>(slots, P, n, 0);
  if (any_mixed) {
    mf_b_launch_eval_tc(slots, P, n, tc_chunk, sms, s);
    k_b_lists<<<sms * 8, EVAL_WARPS * 32, 0, s>>>(slots, P, n);
    mf_b_launch_plan_eval(slots, P, n, true, s);
    k_b_eval<<<sms * 8, EVAL_WARPS * 32, 0, s>>>(slots, P, n, 1);
  }
  mf_b_launch_advance(slots, n, s);
}

void mf_b_launch_roots(const MfSlot *slots, MfBatchPlan *P, int n, const int32_t *only,
                       uint32_t dims, int group, int sms, cudaStream_t s) {
  const int dyn = group > 1 ? ROOT_WARPS * GROUP_CAP * (int)sizeof(int) : 0;
  for (int dd = 2; dd <= MF_MAXD; dd++) {
    if (!((dims >> dd) & 1u)) continue;
    mf_b_launch_plan_edges(slots, P, n, 0, only, s, dd);
    switch (dd) {
#define MF_CASE(DD)                                                                            \
  case DD:                                                                                     \
    if (dyn) cudaFuncSetAttribute(k_b_roots<DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn); \
    k_b_roots<DD><<<sms * 4, ROOT_WARPS * 32, dyn, s>>>(slots, P, n, group);                   \
    break;
      MF_CASE(2) MF_CASE(3) MF_CASE(4) MF_CASE(5) MF_CASE(6) MF_CASE(7) MF_CASE(8)
#undef MF_CASE
      default: break;
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void mf_launch_eval_vertices_f64(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                 const MfTune &T, int sms, cudaStream_t st) {
  const int g = sms * T.eval_bps;
  switch (F.d) {
#define MF_CASE(DD) \
  case DD: k_eval_vertices_f64<DD><<<g, EVAL_WARPS * 32, 0, st>>>(F, R, B); break;
    MF_CASE(2) MF_CASE(3) MF_CASE(4) MF_CASE(5) MF_CASE(6) MF_CASE(7)
#undef MF_CASE
    default: k_eval_vertices_f64<MF_MAXD><<<g, EVAL_WARPS * 32, 0, st>>>(F, R, B);
  }
  k_advance_eval<<<1, 1, 0, st>>>(B.cnt);
}

void mf_launch_eval_vertices_mixed(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                   int precision, double band, const MfTune &T, int sms,
                                   cudaStream_t st) {
  if (precision == MF_MIXED_BF16)
    mf_launch_eval_vertices_tc(F, R, B, band, T.tc_chunk, sms, st);
  else
    k_eval_mixed_f32<true><<<sms * 4, MIX_THREADS, 0, st>>>(F, R, B, nullptr, 0, nullptr, nullptr, band);
  if (B.vlist) {  // the root screen's per-vertex lists
    switch (F.d) {
#define MF_CASE(DD) \
  case DD: k_vertex_lists<DD><<<sms * 8, EVAL_WARPS * 32, 0, st>>>(F, R, B); break;
      MF_CASE(2) MF_CASE(3) MF_CASE(4) MF_CASE(5) MF_CASE(6) MF_CASE(7)
#undef MF_CASE
      default: k_vertex_lists<MF_MAXD><<<sms * 8, EVAL_WARPS * 32, 0, st>>>(F, R, B);
    }
  }
  switch (F.d) {
#define MF_CASE(DD) \
  case DD: k_recheck_vertices_f64<DD><<<sms * 8, EVAL_WARPS * 32, 0, st>>>(F, R, B); break;
    MF_CASE(2) MF_CASE(3) MF_CASE(4) MF_CASE(5) MF_CASE(6) MF_CASE(7)
#undef MF_CASE
    default: k_recheck_vertices_f64<MF_MAXD><<<sms * 8, EVAL_WARPS * 32, 0, st>>>(F, R, B);
  }
  k_advance_eval<<<1, 1, 0, st>>>(B.cnt);
}

template <int DD, int MINB>
static void launch_roots_d(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                           uint64_t n_edges, double tol, int grid, int group, int fast, int sms,
                           cudaStream_t st) {
  const int dyn = group > 1 ? ROOT_WARPS * GROUP_CAP * (int)sizeof(int) : 0;
  if (dyn) cudaFuncSetAttribute(k_roots_f64<DD, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (!B.defer_rec || B.defer_cap == 0) {
    k_roots_f64<DD, MINB><<<grid, ROOT_WARPS * 32, dyn, st>>>(F, R, B, 0, n_edges, tol, group, fast,
                                                             0, nullptr, nullptr);
    return;
  }
  // chunks of defer_cap edges: the warp kernel (deferring the common
  // single-step case), the lane-per-edge FP64 steps, then the redo queue
  const size_t off_defer = offsetof(MfCounters, n_defer);
  const size_t span = offsetof(MfCounters, n_redo) + sizeof(unsigned long long) - off_defer;
  for (uint64_t e0 = 0; e0 < n_edges; e0 += B.defer_cap) {
    const uint64_t n = n_edges - e0 < B.defer_cap ? n_edges - e0 : B.defer_cap;
    const unsigned nb = (unsigned)((n + 255) / 256);
    cudaMemsetAsync((char *)B.cnt + off_defer, 0, span, st);
    k_roots_prep<DD><<<nb, 256, 0, st>>>(F, B, e0, n);
    k_roots_f64<DD, MINB><<<grid, ROOT_WARPS * 32, dyn, st>>>(F, R, B, e0, n, tol, group, fast, 1,
                                                             nullptr, nullptr);
    k_roots_x<DD><<<nb, 256, 0, st>>>(F, B, B.defer_cap, e0);
    k_roots_terms<DD><<<sms * 16, 256, 0, st>>>(R, B, B.defer_cap);
    k_roots_finish<DD><<<nb, 256, 0, st>>>(F, R, B, B.defer_cap, tol, fast, e0);
    k_roots_f64<DD, MINB><<<sms * 4, ROOT_WARPS * 32, 0, st>>>(F, R, B, 0, B.defer_cap, tol, 1,
                                                              fast, 0, B.redo, &B.cnt->n_redo);
  }
}

template <int MINB>
static void launch_roots(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B, uint64_t n_edges,
                         double tol, int grid, int group, int fast, int sms, cudaStream_t st) {
  switch (F.d) {
#define MF_CASE(DD) \
  case DD: launch_roots_d<DD, MINB>(F, R, B, n_edges, tol, grid, group, fast, sms, st); break;
    MF_CASE(2) MF_CASE(3) MF_CASE(4) MF_CASE(5) MF_CASE(6) MF_CASE(7)
#undef MF_CASE
    default: launch_roots_d<MF_MAXD, MINB>(F, R, B, n_edges, tol, grid, group, fast, sms, st);
  }
}

void mf_launch_roots_f64(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B, uint64_t n_edges,
                         double tol, const MfTune &T, int sms, cudaStream_t st, bool fast) {
  if (n_edges == 0) return;
  const int grid = sms * T.roots_bps;
  if (T.roots_variant == 1) launch_roots<3>(F, R, B, n_edges, tol, grid, T.roots_group, fast, sms, st);
  else launch_roots<2>(F, R, B, n_edges, tol, grid, T.roots_group, fast, sms, st);
}

// ---------------------------------------------------------------------------
// Throughput probes (the denominators of the FP64 and MUFU rooflines) and the
// accuracy diagnostic of the table-driven exp.  Each probe thread runs
// independent chains, so the measured rate is the pipe's throughput.
// ---------------------------------------------------------------------------
#define PROBE_CHAINS 8
__global__ void k_probe_dfma(int iters, double seed, double *sink) {
  double a[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) a[i] = seed + 1e-9 * threadIdx.x + i;
  const double m = 0.9999999, c = 1e-7;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; i++) a[i] = fma(a[i], m, c);
  }
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) t += a[i];
  if (t == 1234.5) sink[0] = t;  // keeps the chains alive
}

__global__ void k_probe_ffma(int iters, float seed, float *sink) {
  float a[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) a[i] = seed + 1e-6f * threadIdx.x + i;
  const float m = 0.9999f, c = 1e-4f;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; i++) a[i] = fmaf(a[i], m, c);
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) t += a[i];
  if (t == 1234.5f) sink[0] = t;
}

__global__ void k_probe_ex2(int iters, float *sink) {
  float a[PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) a[i] = -0.5f - 1e-6f * threadIdx.x - 0.01f * i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < PROBE_CHAINS; i++) a[i] = -ex2_approx(a[i]);
  }
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < PROBE_CHAINS; i++) t += a[i];
  if (t == 1234.5f) sink[0] = t;
}

__global__ void k_probe_expneg(int iters, const double *tab, double *sink) {
  constexpr int C = 4;
  double x[C], acc[C];
#pragma unroll
  for (int i = 0; i < C; i++) {
    x[i] = -0.5 - 1e-7 * threadIdx.x - 3.1 * i;
    acc[i] = 0.0;
  }
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < C; i++) {
      acc[i] += mf_exp_neg(x[i], tab);
      x[i] -= 1e-3;
    }
  }
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < C; i++) t += acc[i];
  if (t == 1234.5) sink[0] = t;
}

__global__ void k_exp_table(double *tab) {
  const int j = threadIdx.x;
  if (j < 64) tab[j] = exp2((double)j / 64.0);  // as the RBF preparation builds it
}

__global__ void k_diag_exp(const double *tab, const double *x, int64_t n, double *y_tab,
                           double *y_lib) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  y_tab[i] = mf_exp_neg(x[i], tab);
  y_lib[i] = exp(x[i]);
}

extern "C" int mf_probe_rates(mf_ctx *ctx, mf_rates *out, void *stream) {
  if (!ctx || !out) return MF_ERR_INVALID;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  double *buf = (double *)mf_ctx_buffer(ctx, MF_SLOT_SCAN, 64 * 8 + 256);
  if (!buf) return MF_ERR_OOM;
  double *tab = buf, *sink = buf + 64;
  k_exp_table<<<1, 64, 0, st>>>(tab);
  const int blocks = ctx->sms * 8, threads = 256;
  const double nthreads = (double)blocks * threads;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // best of three timed launches after one warm-up
  auto timed = [&](auto launch) {
    launch();
    float best = 1e30f;
    for (int r = 0; r < 3; r++) {
      cudaEventRecord(e0, st);
      launch();
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    return (double)best * 1e-3;
  };
  const int it_d = 4096, it_f = 65536, it_x = 16384, it_e = 1024;
  const double t_d = timed([&]() { k_probe_dfma<<<blocks, threads, 0, st>>>(it_d, 1.0, sink); });
  const double t_f =
      timed([&]() { k_probe_ffma<<<blocks, threads, 0, st>>>(it_f, 1.f, (float *)sink); });
  const double t_x = timed([&]() { k_probe_ex2<<<blocks, threads, 0, st>>>(it_x, (float *)sink); });
  const double t_e = timed([&]() { k_probe_expneg<<<blocks, threads, 0, st>>>(it_e, tab, sink); });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int rc = mf_cuda_check(ctx, cudaGetLastError(), "probe kernels");
  if (rc) return rc;
  out->fp64_fma_per_s = nthreads * PROBE_CHAINS * it_d / t_d;
  out->fp32_fma_per_s = nthreads * PROBE_CHAINS * it_f / t_f;
  out->ex2_per_s = nthreads * PROBE_CHAINS * it_x / t_x;
  out->exp_neg_per_s = nthreads * 4.0 * it_e / t_e;
  int mhz = 0;
  cudaDeviceGetAttribute(&mhz, cudaDevAttrClockRate, ctx->device);
  out->sm_count = ctx->sms;
  out->sm_clock_mhz = mhz / 1000.0;
  return MF_OK;
}

extern "C" int mf_diag_exp(mf_ctx *ctx, const double *x, int64_t n, double *y_table, double *y_lib,
                           void *stream) {
  if (!ctx || n < 0 || (n > 0 && (!x || !y_table || !y_lib))) return MF_ERR_INVALID;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  double *tab = (double *)mf_ctx_buffer(ctx, MF_SLOT_SCAN, 64 * 8 + 256);
  if (!tab) return MF_ERR_OOM;
  k_exp_table<<<1, 64, 0, st>>>(tab);
  if (n > 0) k_diag_exp<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tab, x, n, y_table, y_lib);
  const int rc = mf_cuda_check(ctx, cudaGetLastError(), "mf_diag_exp");
  if (rc) return rc;
  return mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_diag_exp");
}

extern "C" int mf_eval(mf_ctx *ctx, const mf_rbf *rbf, const double *q, int64_t n, int32_t precision,
                       double band, double *f_out, void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  ctx->sub.valid = false;  // its slots are reused here
  if (n < 0 || (n > 0 && (!q || !f_out)) ||
      (precision != MF_FP64 && precision != MF_MIXED_FP32 && precision != MF_MIXED_BF16))
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_eval: bad arguments");
  // the tensor-core GEMM is exact only for small integer offsets between
  // lattice vertices of a tile; arbitrary points have no such structure
  if (precision == MF_MIXED_BF16)
    return mf_set_error(ctx, MF_ERR_INVALID,
                        "mf_eval: MF_MIXED_BF16 evaluates lattice vertices only (mf_trace); use "
                        "MF_MIXED_FP32 or MF_FP64 for arbitrary points");
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  MfRbfDev R;
  int rc = mf_prepare_rbf(ctx, rbf, &R, st);
  if (rc) return rc;
  if (n == 0) return MF_OK;
  const int sms = ctx->sms;
  if (precision == MF_FP64) {
    k_eval_points_f64<<<sms * 8, EVAL_WARPS * 32, 0, st>>>(R, q, n, f_out, nullptr);
  } else {
    uint8_t *flag = (uint8_t *)mf_ctx_buffer(ctx, MF_SLOT_SCAN, (size_t)n + 256);
    if (!flag) return MF_ERR_OOM;
    MfFrame F;
    mf_frame_lattice(&F, R.d, 1.0, nullptr);
    MfTraceBufs B = {};
    k_eval_mixed_f32<false><<<sms * 4, MIX_THREADS, 0, st>>>(F, R, B, q, n, f_out, flag,
                                                             band > 0 ? band : 1e-3);
    k_eval_points_f64<<<sms * 8, EVAL_WARPS * 32, 0, st>>>(R, q, n, f_out, flag);
  }
  rc = mf_cuda_check(ctx, cudaGetLastError(), "mf_eval launch");
  if (rc) return rc;
  return mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_eval");
}
