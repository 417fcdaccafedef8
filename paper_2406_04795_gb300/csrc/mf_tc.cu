// mf_tc.cu -- f at lattice vertices on the 5th-generation tensor cores
// (precision MF_MIXED_BF16): the RBF decision function of Sec. IV-A with its
// distance term computed as a GEMM.
//
// A CTA evaluates tiles of 128 vertices.  With y0 the tile's first vertex,
// q0 = x(y0), dy = y - y0 (small integers) and u_j = q0 - s_j,
//   |q - s_j|^2 = |u_j|^2 + dy . w_j + |lam L dy|^2,     w_j = 2 lam L u_j
// (L = I - c 11^T is symmetric).  Per chunk of 64 support vectors one
// tcgen05 MMA (M = 128, N = 64, K = 32, BF16 operands, FP32 accumulator in
// TMEM) computes D[v][j] = sum_k A[v][k] B[j][k] with
//   A[v] = [dy, dy, dy, 1, 1, 1, 0 ...]          exact in BF16 for |dy| <= 256
//   B[j] = [w_hi, w_mid, w_lo, c_hi, c_mid, c_lo, 0 ...],   c = |u_j|^2,
// where the three BF16 pieces of an FP32 value sum to it exactly, so D is an
// FP32-accumulated dot product of exact products.  B is built per tile from
// q0 (FP32 hi/lo differences, so u_j keeps FP32 relative accuracy).  The
// epilogue (thread = TMEM lane = vertex) forms e = 2^(-g2 (D + qq)) with the
// MUFU ex2, sums alpha e in FP32 and bounds |f~ - f| rigorously.  Vertices
// with |f~| <= max(bound, band), or with some |dy| > 256, are queued for the
// FP64 recheck (k_recheck_vertices_f64), so every sign decision is FP64-exact.
//
// Two chunk accumulators (2 x 64 TMEM columns) let the MMA of chunk c run
// while the epilogue drains chunk c - 1.  4 CTAs per SM share its 512 TMEM
// columns.
#include <cmath>
#include <cuda_bf16.h>

#include "mf_internal.cuh"
#include "mf_ctx.h"
#include "mf_tc_ptx.cuh"

#define TC_M MF_TC_TILE
#define TC_K 32
#define TC_DY_MAX 256
#define TC_WAIT_NS 2000000000ull  // bounded waits: 2 s

// Chunk width N (support vectors per MMA): 2 N TMEM columns per CTA, so
// 512 / (2 N) CTAs share an SM; the shared-memory request caps residency there.
template <int N>
struct TcCfg {
  static constexpr int kCols = 2 * N;
  static constexpr int kCtasPerSm = 512 / (2 * N);
  static constexpr int kSmemPerCta = (N == 64 ? 52 : 100) * 1024;
};

template <int N>
struct TcShared {
  alignas(128) unsigned char a[TC_M * TC_K * 2];
  alignas(128) unsigned char b[2][N * TC_K * 2];
  float alpha[2][N];
  uint64_t bar[2];
  uint32_t tmem;
  int timeout;
  int32_t y0[MF_MAXD];
  float q0hi[MF_MAXD], q0lo[MF_MAXD];
};

__device__ __forceinline__ float tc_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t tc_pack(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// Three BF16 pieces whose sum is x exactly (x FP32, no underflow).
__device__ __forceinline__ void tc_split3(float x, float &h, float &m, float &l) {
  h = __bfloat162float(__float2bfloat16_rn(x));
  const float r = x - h;
  m = __bfloat162float(__float2bfloat16_rn(r));
  l = r - m;
}

// Stores 32 FP32 values (exact in BF16) as row r of a K = 32 operand tile.
__device__ __forceinline__ void tc_store_row(unsigned char *tile, int r, const float (&v)[TC_K]) {
#pragma unroll
  for (int c = 0; c < TC_K / 8; c++) {
    uint4 q;
    q.x = tc_pack(v[8 * c + 0], v[8 * c + 1]);
    q.y = tc_pack(v[8 * c + 2], v[8 * c + 3]);
    q.z = tc_pack(v[8 * c + 4], v[8 * c + 5]);
    q.w = tc_pack(v[8 * c + 6], v[8 * c + 7]);
    *reinterpret_cast<uint4 *>(tile + mf_tc_off_k32(r, 8 * c)) = q;
  }
}

// mbarrier phases and outstanding commits of a CTA's two chunk accumulators;
// kept across tiles (the barriers live as long as the CTA).
struct TcPipe {
  uint32_t phase0 = 0, phase1 = 0;
  int pending0 = 0, pending1 = 0;  // commits issued and not yet waited for
};

// One tile: f at the vertices [v_first, v_end) (at most TC_M) of one trace's
// vertex list, every chunk of support vectors through the MMA; vertices the
// bound cannot decide go to the trace's FP64 recheck queue.  All threads of
// the CTA call it; returns false when a bounded wait gave up.
template <int D, int N>
__device__ __forceinline__ bool tc_tile(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                        double band, uint64_t v_first, uint64_t v_end,
                                        TcShared<N> &sh, uint32_t tmem, TcPipe &pp) {
  constexpr int TC_N = N;
  const int t = threadIdx.x, w = t >> 5;
  const uint32_t lane_base = (uint32_t)(32 * w) << 16;
  const uint32_t idesc = mf_tc_idesc_bf16(TC_M, TC_N);
  const float g2 = (float)(R.gamma * 1.4426950408889634);
  const float lam2 = (float)(2.0 * F.lam);
  const float c32 = (float)F.c;
  const int nchunks = (R.n + TC_N - 1) / TC_N;
  const uint64_t v = v_first + t;
  const bool valid = v < v_end;
  int32_t y[D];
#pragma unroll
  for (int k = 0; k < D; k++) y[k] = valid ? B.vert_y[v * D + k] : 0;
  if (t == 0) {
    int32_t ym[MF_MAXD];
    double q0[MF_MAXD];
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) ym[k] = k < D ? y[k] : 0;
    mf_vertex_x(F, ym, q0);
#pragma unroll
    for (int k = 0; k < D; k++) {
      sh.y0[k] = y[k];
      sh.q0hi[k] = (float)q0[k];
      sh.q0lo[k] = (float)(q0[k] - (double)sh.q0hi[k]);
    }
  }
  __syncthreads();
  // this vertex relative to the tile base
  int32_t dy[D];
  bool far = false;
  long long sdy = 0;
  double dyn2 = 0.0;
#pragma unroll
  for (int k = 0; k < D; k++) {
    dy[k] = valid ? y[k] - sh.y0[k] : 0;
    far = far || dy[k] > TC_DY_MAX || dy[k] < -TC_DY_MAX;
    sdy += dy[k];
    dyn2 += (double)dy[k] * (double)dy[k];
  }
  double qq = 0.0;
#pragma unroll
  for (int k = 0; k < D; k++) {
    const double l = (double)dy[k] - F.c * (double)sdy;
    qq = fma(l, l, qq);
  }
  qq *= F.lam * F.lam;
  {
    float row[TC_K];
#pragma unroll
    for (int c = 0; c < TC_K; c++) {
      float val = 0.f;
      if (c < 3 * D) val = far ? 0.f : (float)dy[c % D];
      else if (c < 3 * D + 3) val = 1.f;
      row[c] = val;
    }
    tc_store_row(sh.a, t, row);
  }
  const float kq = -g2 * (float)qq;
  float acc = 0.f, aab = 0.f, qa = 0.f;
  bool ok = true;

  for (int c = 0; c <= nchunks; c++) {
    const int buf = c & 1;
    if (c < nchunks) {
      if (t < TC_N) {
        // row t of chunk c: support vector j
        const int j = c * TC_N + t;
        float row[TC_K];
#pragma unroll
        for (int k = 0; k < TC_K; k++) row[k] = 0.f;
        float al = 0.f;
        if (j < R.n) {
          float u[D], su = 0.f, cc = 0.f;
#pragma unroll
          for (int k = 0; k < D; k++) {
            u[k] = (sh.q0hi[k] - R.sv32[(int64_t)k * R.n + j]) +
                   (sh.q0lo[k] - R.svlo32[(int64_t)k * R.n + j]);
            su += u[k];
            cc = fmaf(u[k], u[k], cc);
          }
          const float cs = c32 * su;
#pragma unroll
          for (int k = 0; k < D; k++) {
            float h, m, l;
            tc_split3(lam2 * (u[k] - cs), h, m, l);
            row[k] = h;
            row[D + k] = m;
            row[2 * D + k] = l;
          }
          float h, m, l;
          tc_split3(cc, h, m, l);
          row[3 * D] = h;
          row[3 * D + 1] = m;
          row[3 * D + 2] = l;
          al = R.alpha32[j];
        }
        tc_store_row(sh.b[buf], t, row);
        sh.alpha[buf][t] = al;
      }
      mf_fence_proxy_async_smem();
      mf_tc_fence_before();
      __syncthreads();
      if (t == 0) {
        mf_tc_fence_after();
        const uint32_t a0 = mf_smem_u32(sh.a), b0 = mf_smem_u32(sh.b[buf]);
        const uint32_t dcol = tmem + (uint32_t)(buf * TC_N);
        mf_tc_mma_bf16(dcol, mf_tc_desc(a0, 128, 512), mf_tc_desc(b0, 128, 512), idesc, 0u);
        mf_tc_mma_bf16(dcol, mf_tc_desc(a0 + 256, 128, 512), mf_tc_desc(b0 + 256, 128, 512), idesc,
                       1u);
        mf_tc_commit(&sh.bar[buf]);
      }
      if (buf) pp.pending1 = 1; else pp.pending0 = 1;
    }
    if (c > 0) {
      const int pb = buf ^ 1;  // chunk c - 1
      const bool got = mf_mbar_wait(&sh.bar[pb], pb ? pp.phase1 : pp.phase0, TC_WAIT_NS);
      if (pb) { pp.phase1 ^= 1u; pp.pending1 = 0; } else { pp.phase0 ^= 1u; pp.pending0 = 0; }
      if (!got) sh.timeout = 1;
      mf_tc_fence_after();
#pragma unroll
      for (int h = 0; h < TC_N / 32; h++) {
        float dv[32];
        mf_tmem_ld32(tmem + lane_base + (uint32_t)(pb * TC_N + 32 * h), dv);
        float part = 0.f;
#pragma unroll
        for (int i = 0; i < 32; i++) {
          const float arg = fmaf(dv[i], -g2, kq);
          const float term = sh.alpha[pb][32 * h + i] * tc_ex2(arg);
          part += term;
          aab += fabsf(term);
          qa = fmaf(fabsf(term), fabsf(arg), qa);
        }
        acc += part;
      }
      mf_tc_fence_before();
    }
    __syncthreads();
    if (sh.timeout) {
      ok = false;
      break;
    }
  }
  if (!ok) return false;

  if (valid) {
    // |f~ - f| bound (u = 2^-24): MMA accumulation and operand rounding
    // scale with |dy| |w| and |u|^2, which are bounded through r and qq
    // (|u| <= r + sqrt(qq)); exponent rounding through sum |t| |arg|; ex2,
    // products and the blocked FP32 sums through sum |t|.
    const double u = 5.9604644775390625e-08;
    const double A = (double)aab, Qa = (double)qa;
    const double Q = 1.01 * Qa / (double)g2 + 1e-300;  // sum |t| r^2
    const double a1 = 80.0 * 2.0 * F.lam * sqrt(dyn2);
    const double a2 = 72.0 + D;
    const double coord = R.gamma * u *
                         (a1 * sqrt(A * Q) + (a1 * sqrt(qq) + (2.0 * a2 + 1.0) * qq) * A + 2.0 * a2 * Q);
    const double expo = 3.0 * 0.6931471805599453 * u * Qa;
    const double other = (9.5367431640625e-07 + (34.0 + 2.0 * nchunks) * u) * A;
    const double bound = 1.05 * (coord + expo + other) + 1e-30 + R.sum_abs_alpha * 1.2e-38;
    const double fx = (double)acc + R.b;
    const uint32_t slot = B.vert_slot[v];
    mf_vtab_f(B, slot) = fx;
    if (far || fabs(fx) <= fmax(bound, band)) {
      const unsigned long long q = atomicAdd(&B.cnt->n_recheck, 1ull);
      if (q < B.max_vertices) B.recheck[q] = (uint32_t)v;
      else atomicOr(&B.cnt->err_overflow, 1u);
    }
  }
  __syncthreads();  // the next tile rewrites A and the tile base
  return true;
}

// TMEM columns and barriers of a CTA: allocated once, used by every tile.
template <int N>
__device__ __forceinline__ void tc_begin(TcShared<N> &sh) {
  const int t = threadIdx.x, w = t >> 5;
  if (w == 0) mf_tmem_alloc(&sh.tmem, TcCfg<N>::kCols);
  if (t == 0) {
    mf_mbar_init(&sh.bar[0], 1);
    mf_mbar_init(&sh.bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh.timeout = 0;
  }
  mf_tc_fence_before();
  __syncthreads();
  mf_tc_fence_after();
}

// After a wait gave up (ok false): flags it, gives in-flight MMAs a bounded
// chance to finish, then frees the columns.
template <int N>
__device__ __forceinline__ void tc_end(TcShared<N> &sh, TcPipe &pp, bool ok, MfCounters *cnt) {
  const int t = threadIdx.x, w = t >> 5;
  if (!ok) {
    if (t == 0) atomicOr(&cnt->err_timeout, 1u);
    if (pp.pending0) mf_mbar_wait(&sh.bar[0], pp.phase0, TC_WAIT_NS);
    if (pp.pending1) mf_mbar_wait(&sh.bar[1], pp.phase1, TC_WAIT_NS);
  }
  mf_tc_fence_before();
  __syncthreads();
  if (w == 0) {
    mf_tc_fence_after();
    mf_tmem_dealloc(sh.tmem, TcCfg<N>::kCols);
  }
}

template <int D, int N>
__global__ void __launch_bounds__(TC_M, TcCfg<N>::kCtasPerSm) k_eval_tc(MfFrame F, MfRbfDev R,
                                                                        MfTraceBufs B, double band) {
  __shared__ TcShared<N> sh;
  const uint64_t begin = B.cnt->v_evaluated;
  uint64_t end = B.cnt->n_vertices;
  if (end > B.max_vertices) end = B.max_vertices;
  if (begin >= end) return;
  const uint64_t ntiles = (end - begin + TC_M - 1) / TC_M;
  if (blockIdx.x >= ntiles) return;  // uniform per CTA, before any allocation
  tc_begin<N>(sh);
  TcPipe pp;
  bool ok = true;
  for (uint64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const uint64_t v0 = begin + tile * TC_M;
    ok = tc_tile<D, N>(F, R, B, band, v0, v0 + TC_M < end ? v0 + TC_M : end, sh, sh.tmem, pp);
  }
  tc_end<N>(sh, pp, ok, B.cnt);
}

// Batched form: the tiles of every MF_MIXED_BF16 slot of a batch (the plan's
// pt prefix; a tile never spans two traces), each with its trace's frame,
// support vectors and tables.
template <int N>
__global__ void __launch_bounds__(TC_M, TcCfg<N>::kCtasPerSm) k_b_eval_tc(const MfSlot *slots,
                                                                          const MfBatchPlan *P,
                                                                          int n) {
  __shared__ TcShared<N> sh;
  const unsigned long long ntiles = P->pt[n];
  if (blockIdx.x >= ntiles) return;  // uniform per CTA, before any allocation
  tc_begin<N>(sh);
  TcPipe pp;
  bool ok = true;
  MfCounters *last = nullptr;
  for (unsigned long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int s = mf_slot_of(P->pt, n, tile);
    const MfSlot &S = slots[s];
    last = S.B.cnt;
    const uint64_t end = P->v0[s] + (P->pv[s + 1] - P->pv[s]);
    const uint64_t v0 = P->v0[s] + (tile - P->pt[s]) * TC_M;
    const uint64_t v1 = v0 + TC_M < end ? v0 + TC_M : end;
    switch (S.F.d) {
#define MF_CASE(DD) \
  case DD: ok = tc_tile<DD, N>(S.F, S.R, S.B, S.band, v0, v1, sh, sh.tmem, pp); break;
      MF_CASE(2) MF_CASE(3) MF_CASE(4) MF_CASE(5) MF_CASE(6) MF_CASE(7) MF_CASE(8)
#undef MF_CASE
      default: break;
    }
  }
  tc_end<N>(sh, pp, ok, last);
}

// Vertex evaluation on the tensor cores with chunk width n_chunk (64 or
// 128 support vectors per MMA); the caller launches the FP64 recheck of the
// queued vertices afterwards.
template <int N>
static void launch_tc(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B, double band,
                      int sms, cudaStream_t st) {
  const size_t dyn = TcCfg<N>::kSmemPerCta - sizeof(TcShared<N>);
  const int grid = sms * TcCfg<N>::kCtasPerSm;
  switch (F.d) {
#define MF_CASE(DD)                                                                       \
  case DD:                                                                                \
    cudaFuncSetAttribute(k_eval_tc<DD, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                         (int)dyn);                                                       \
    k_eval_tc<DD, N><<<grid, TC_M, dyn, st>>>(F, R, B, band);                             \
    break;
    MF_CASE(2) MF_CASE(3) MF_CASE(4) MF_CASE(5) MF_CASE(6) MF_CASE(7) MF_CASE(8)
#undef MF_CASE
    default: break;
  }
}

void mf_launch_eval_vertices_tc(const MfFrame &F, const MfRbfDev &R, const MfTraceBufs &B,
                                double band, int n_chunk, int sms, cudaStream_t st) {
  if (n_chunk == 128) launch_tc<128>(F, R, B, band, sms, st);
  else launch_tc<64>(F, R, B, band, sms, st);
}

void mf_b_launch_eval_tc(const MfSlot *slots, const MfBatchPlan *P, int n, int n_chunk, int sms,
                         cudaStream_t st) {
  if (n_chunk == 128) {
    const size_t dyn = TcCfg<128>::kSmemPerCta - sizeof(TcShared<128>);
    cudaFuncSetAttribute(k_b_eval_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    k_b_eval_tc<128><<<sms * TcCfg<128>::kCtasPerSm, TC_M, dyn, st>>>(slots, P, n);
  } else {
    const size_t dyn = TcCfg<64>::kSmemPerCta - sizeof(TcShared<64>);
    cudaFuncSetAttribute(k_b_eval_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    k_b_eval_tc<64><<<sms * TcCfg<64>::kCtasPerSm, TC_M, dyn, st>>>(slots, P, n);
  }
}
