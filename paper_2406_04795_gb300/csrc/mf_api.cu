// mf_api.cu -- context lifetime, error reporting, the device arena, and the
// locate query (query type 1 of Sec. IV-A).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "mf_internal.cuh"
#include "mf_ctx.h"

extern "C" int mf_ctx_create(int device, size_t budget, mf_ctx **out) {
  if (!out) return MF_ERR_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return MF_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return MF_ERR_CUDA;
  mf_ctx *c = new mf_ctx();
  c->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return MF_ERR_CUDA; }
  c->sms = prop.multiProcessorCount;
  size_t freeb = 0, totalb = 0;
  if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) { delete c; return MF_ERR_CUDA; }
  c->budget = budget ? budget : (size_t)(0.9 * (double)freeb);
  if (cudaMallocHost((void **)&c->h_counters, sizeof(MfCounters)) != cudaSuccess) {
    delete c;
    return MF_ERR_CUDA;
  }
  *out = c;
  return MF_OK;
}

// ---------------------------------------------------------------------------
// Profiling
// ---------------------------------------------------------------------------
static cudaEvent_t prof_event(mf_ctx *c) {
  if (c->prof.used == c->prof.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->prof.pool.push_back(e);
  }
  return c->prof.pool[c->prof.used++];
}

MfProfScope::MfProfScope(mf_ctx *ctx, int ph, cudaStream_t s, int launches, int64_t units)
    : c(ctx), phase(ph), st(s) {
  if (!c || !c->prof.on) return;
  c->prof.stats.launches[ph] += launches;
  c->prof.stats.units[ph] += units;
  a = prof_event(c);
  b = prof_event(c);
  if (a) cudaEventRecord(a, st);
}

MfProfScope::~MfProfScope() {
  if (!c || !c->prof.on || !a || !b) return;
  cudaEventRecord(b, st);
  c->prof.pending.push_back({phase, {a, b}});
}

void mf_prof_collect(mf_ctx *c) {
  if (!c->prof.on) return;
  for (auto &p : c->prof.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.second.second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess)
      c->prof.stats.ms[p.first] += ms;
  }
  c->prof.pending.clear();
  c->prof.used = 0;
}

extern "C" int mf_ctx_set_profiling(mf_ctx *c, int enable) {
  if (!c) return MF_ERR_INVALID;
  cudaSetDevice(c->device);
  mf_prof_collect(c);
  c->prof.on = enable != 0;
  memset(&c->prof.stats, 0, sizeof(c->prof.stats));
  return MF_OK;
}

extern "C" int mf_ctx_get_stats(mf_ctx *c, mf_stats *out) {
  if (!c || !out) return MF_ERR_INVALID;
  cudaSetDevice(c->device);
  mf_prof_collect(c);
  *out = c->prof.stats;
  return MF_OK;
}

extern "C" void mf_ctx_destroy(mf_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (auto e : c->prof.pool) cudaEventDestroy(e);
  for (int s = 0; s < MF_NUM_SLOTS; s++)
    if (c->slot_ptr[s]) cudaFree(c->slot_ptr[s]);
  if (c->h_counters) cudaFreeHost(c->h_counters);
  delete c;
}

extern "C" const char *mf_last_error(mf_ctx *c) { return c ? c->err.c_str() : "null context"; }

extern "C" size_t mf_ctx_bytes(mf_ctx *c) { return c ? c->total : 0; }

int mf_set_error(mf_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int mf_cuda_check(mf_ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return MF_OK;
  return mf_set_error(c, MF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int mf_ctx_sm_count(mf_ctx *c) { return c->sms; }

void *mf_ctx_buffer(mf_ctx *c, int slot, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  if (c->slot_bytes[slot] >= bytes) return c->slot_ptr[slot];
  size_t others = c->total - c->slot_bytes[slot];
  if (others + bytes > c->budget) {
    mf_set_error(c, MF_ERR_OOM, "HBM budget: need %zu more bytes (budget %zu, held %zu)",
                 bytes - c->slot_bytes[slot], c->budget, c->total);
    return nullptr;
  }
  if (c->slot_ptr[slot]) {
    cudaDeviceSynchronize();
    cudaFree(c->slot_ptr[slot]);
    c->slot_ptr[slot] = nullptr;
    c->total -= c->slot_bytes[slot];
    c->slot_bytes[slot] = 0;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mf_set_error(c, MF_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return nullptr;
  }
  c->slot_ptr[slot] = p;
  c->slot_bytes[slot] = bytes;
  c->total += bytes;
  return p;
}

// ---------------------------------------------------------------------------
// Query type 1: locate the n-simplex holding a point.  Same operation order as
// the lattice map's inverse y' = L^-1 (x - o) / lam; vertex = floor(y'); the
// walk order sorts the fractional parts descending, ties to the lower index.
// ---------------------------------------------------------------------------
__global__ void k_locate(MfFrame F, const double *pts, int64_t n, int32_t *y_out, uint8_t *perm_out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int d = F.d;
  double x[MF_MAXD];
  for (int k = 0; k < d; k++) x[k] = pts[i * d + k];
  int32_t y[MF_MAXD];
  int perm[MF_MAXD];
  mf_locate_point(F, x, y, perm);
  for (int k = 0; k < d; k++) {
    y_out[i * d + k] = y[k];
    perm_out[i * d + k] = (uint8_t)perm[k];
  }
}

void mf_frame_lattice(MfFrame *F, int d, double lam, const double *o) {
  memset(F, 0, sizeof(*F));
  F->d = d;
  F->lam = lam;
  F->c = (1.0 - 1.0 / std::sqrt((double)(d + 1))) / (double)d;
  F->cinv = F->c * std::sqrt((double)(d + 1));
  for (int i = 0; i < d; i++) F->o[i] = o ? o[i] : 0.0;
}

extern "C" int mf_locate(mf_ctx *ctx, int32_t d, double lambda, const double *offset_host,
                         const double *points, int64_t n, int32_t *y_out, uint8_t *perm_out,
                         void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  if (d < 2 || d > MF_MAXD || !(lambda > 0.0) || n < 0 || (n > 0 && (!points || !y_out || !perm_out)))
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_locate: bad arguments");
  if (n == 0) return MF_OK;
  cudaSetDevice(ctx->device);
  MfFrame F;
  mf_frame_lattice(&F, d, lambda, offset_host);
  cudaStream_t st = (cudaStream_t)stream;
  k_locate<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(F, points, n, y_out, perm_out);
  int rc = mf_cuda_check(ctx, cudaGetLastError(), "mf_locate launch");
  if (rc) return rc;
  return mf_cuda_check(ctx, cudaStreamSynchronize(st), "mf_locate");
}
