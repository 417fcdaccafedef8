// mf_noalloc.cu -- mf_trace_noalloc: the tracing entry point for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator (which would be bypassed or starved),
// real-time loops that forbid allocation after start-up, and processes whose
// device memory is fully reserved by someone else.  This entry point performs
// the same trace as mf_trace (seeds, breadth-first search, roots, cells and
// their CSR) without allocating anything: all of its scratch -- hash tables,
// edge / vertex / cell lists, counters, the prepared support vectors -- lives
// in one file-scope device array of MF_NOALLOC_SCRATCH_BYTES bytes, which
// every GPU that loads the library holds until the process exits.  The caller
// still passes the inputs and the output buffers.
//
// Set-up: the first call on a device (with that device current) looks up the
// array's device address with cudaGetSymbolAddress; make that first call
// before any stream capture.  Every call on a device shares the one array and
// clears what must start empty (counters, hash tables); two calls that overlap
// on the GPU (different streams, threads) race on it and must not be issued.
#include <cmath>
#include <cstring>

#include "mf_internal.cuh"

#define MF_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_mf_noalloc_scratch[MF_NOALLOC_SCRATCH_BYTES];

// Kernels of the traced path (defined in mf_trace.cu / mf_eval.cu).
struct MfRbfStats {
  double sum_abs_alpha;
  float max_abs_s;
  int bad;
};
__global__ void k_prepare_rbf(int d, int n, const double *sv, const double *alpha, const int32_t *perm,
                              float *sv32, float *svlo32, double *sv64, double *alpha64,
                              float *alpha32, float *strong32, double *exp_tab, double *sv64r,
                              float *svhl, MfRbfStats *st);
__global__ void k_rbf_blocks(int d, int n, int nblk, const float *sv32, float *blo, float *bhi);
__global__ void k_seed_vertices(MfFrame F, MfTraceBufs B, const double *seeds, int64_t n);
__global__ void k_seed_edges(MfFrame F, MfTraceBufs B, const double *seeds, int64_t n);
__global__ void k_expand_vertices(MfFrame F, MfTraceBufs B, uint64_t e0, uint64_t n);
__global__ void k_expand_edges(MfFrame F, MfTraceBufs B, uint64_t e0, uint64_t n);
__global__ void k_cells_enum(MfFrame F, MfTraceBufs B, uint64_t n_edges);
__global__ void k_scan_tiles(const int64_t *in, int64_t *out, int64_t n, int64_t *tile_tot);
__global__ void k_scan_totals(int64_t *tile_tot, int64_t ntiles, int64_t *grand);
__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *tile_tot);

// Cell -> traced edges for this entry point: the (d+1)d/2 edges of each cell
// looked up in the edge table (count pass, then fill pass at the scanned
// offsets).  Same rule as mf_trace's CSR.
template <bool FILL>
__global__ void k_noalloc_cell_edges(MfFrame F, MfTraceBufs B, uint64_t n_cells,
                                     int64_t *cnt_or_off) {
  const int d = F.d;
  const uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  int32_t vi[MF_MAXD];
  int pi[MF_MAXD];
  for (int k = 0; k < MF_MAXD; k++) vi[k] = k < d ? B.cell_y[c * d + k] : 0;
  for (int k = 0; k < d; k++) pi[k] = B.cell_perm[c * d + k];
  const int64_t pos = FILL ? cnt_or_off[c] : 0;
  int64_t count = 0;
  for (int i = 0; i < d; i++) {
    int32_t vj[MF_MAXD];
    for (int k = 0; k < MF_MAXD; k++) vj[k] = vi[k];
    uint32_t mask = 0;
    for (int j = i + 1; j <= d; j++) {
      mask |= 1u << pi[j - 1];
      vj[pi[j - 1]] += 1;
      const uint64_t slot = mf_table_find<2>(B.etab_key, B.etab_mask, mf_edge_key(F, vi, mask));
      if (slot == ~0ull) continue;
      if (FILL) B.cell_idx[pos + count] = (int64_t)mf_etab_val(B, slot);
      count++;
    }
    vi[pi[i]] += 1;
  }
  if (!FILL) cnt_or_off[c] = count;
}

namespace {

const int64_t kScanTile = 512 * 8;

unsigned char *g_scratch_ptr[MF_NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device (set up once).
unsigned char *scratch_base(int dev) {
  if (dev < 0 || dev >= MF_NOALLOC_MAX_DEVICES) return nullptr;
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mf_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[dev] = (unsigned char *)p;
  }
  return g_scratch_ptr[dev];
}

struct Carver {
  unsigned char *base;
  size_t used = 0, cap;
  void *take(size_t bytes) {
    size_t a = (used + 255) & ~(size_t)255;
    if (a + bytes > cap) return nullptr;
    used = a + bytes;
    return base + a;
  }
};

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

int frame_for(int d, double lam, const mf_domain *dom, MfFrame *F) {
  memset(F, 0, sizeof(*F));
  F->d = d;
  F->lam = lam;
  F->c = (1.0 - 1.0 / std::sqrt((double)(d + 1))) / (double)d;
  F->cinv = F->c * std::sqrt((double)(d + 1));
  double slo = 0.0, shi = 0.0;
  for (int j = 0; j < d; j++) {
    if (!(dom->lo[j] <= dom->hi[j]) || !std::isfinite(dom->lo[j]) || !std::isfinite(dom->hi[j]) ||
        !std::isfinite(dom->offset[j]))
      return MF_ERR_INVALID;
    F->o[j] = dom->offset[j];
    F->lo[j] = dom->lo[j];
    F->hi[j] = dom->hi[j];
    slo += dom->lo[j] - dom->offset[j];
    shi += dom->hi[j] - dom->offset[j];
  }
  for (int i = 0; i < d; i++) {
    const double a = ((dom->lo[i] - dom->offset[i]) + F->cinv * slo) / lam;
    const double b = ((dom->hi[i] - dom->offset[i]) + F->cinv * shi) / lam;
    if (!(std::fabs(a) < 1e9 && std::fabs(b) < 1e9)) return MF_ERR_DOMAIN;
    const long long ymin = (long long)std::floor(a) - 3, ymax = (long long)std::ceil(b) + 3;
    F->ymin[i] = (int32_t)ymin;
    F->range[i] = (int32_t)(ymax - ymin + 1);
  }
  return mf_frame_pack_keys(F) ? MF_OK : MF_ERR_DOMAIN;
}

int sync_read(MfCounters *h, const MfCounters *d, cudaStream_t st) {
  if (cudaMemcpyAsync(h, d, sizeof(MfCounters), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return MF_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MF_ERR_CUDA;
  if (h->err_table_full || h->err_missing) return MF_ERR_DEVICE;
  if (h->err_timeout) return MF_ERR_TIMEOUT;
  if (h->err_overflow) return MF_ERR_MAXEDGES;
  return MF_OK;
}

}  // namespace

extern "C" int mf_trace_noalloc(const mf_rbf *rbf, const mf_domain *dom, const mf_trace_opts *opts,
                                const double *seeds, int64_t n_seeds, mf_trace_out *out,
                                void *stream) {
  if (!rbf || !dom || !opts || !out || n_seeds < 0 || (n_seeds > 0 && !seeds) || rbf->d < 2 ||
      rbf->d > MF_MAXD || rbf->n_sv < 1 || rbf->n_sv > (1ll << 30) || !rbf->sv || !rbf->alpha ||
      !(rbf->gamma > 0.0) || !std::isfinite(rbf->gamma) || !std::isfinite(rbf->b) ||
      !(opts->lambda > 0.0) || !std::isfinite(opts->lambda) ||
      (opts->precision != MF_FP64 && opts->precision != MF_MIXED_FP32 &&
       opts->precision != MF_MIXED_BF16))
    return MF_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MF_ERR_CUDA;
  unsigned char *base = scratch_base(dev);
  if (!base) return MF_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const int d = rbf->d, n = (int)rbf->n_sv;
  const bool mixed = opts->precision != MF_FP64;
  MfFrame F;
  int rc = frame_for(d, opts->lambda, dom, &F);
  if (rc) return rc;

  // Capacities: the caller's; a zero leaves the largest default that fits.
  const size_t nb = (size_t)n;
  uint64_t ME = 0, MV = 0, MC = 0, TE = 0, TV = 0, cell_edges = 0;
  size_t need = 0;
  for (uint64_t def = 1ull << 17;; def >>= 1) {
    ME = opts->max_edges > 0 ? (uint64_t)opts->max_edges : def;
    MV = opts->max_vertices > 0 ? (uint64_t)opts->max_vertices : ME;
    MC = opts->max_cells > 0 ? (uint64_t)opts->max_cells : 2 * ME;
    TE = pow2_at_least(ME + ME / 3 + 1);
    TV = pow2_at_least(MV + MV / 3 + 1);
    cell_edges = MC * (uint64_t)((d + 1) * d / 2);
    need = 256 * 38 + 64 * 8 + nb * 136 + ((nb + 31) / 32) * d * 8 + nb * d * 16 + nb * 8 + TE * 16 + TV * 16 + ME * (12 * d + 28) +
           MV * (4 * d + 8) + MC * (5 * d + 8) + 8 + cell_edges * 8 + (MC / kScanTile + 2) * 8;
    if (need <= MF_NOALLOC_SCRATCH_BYTES || def < 1024) break;
  }
  if (ME >= (1ull << 32) || MV >= (1ull << 32) || need > MF_NOALLOC_SCRATCH_BYTES)
    return MF_ERR_OOM;  // the request does not fit the fixed scratch array
  Carver cv{base, 0, MF_NOALLOC_SCRATCH_BYTES};
  MfCounters *cnt = (MfCounters *)cv.take(sizeof(MfCounters));
  MfRbfStats *stats = (MfRbfStats *)cv.take(sizeof(MfRbfStats));
  double *sv64 = (double *)cv.take(nb * d * 8);
  float *sv32 = (float *)cv.take(nb * d * 4);
  float *svlo32 = (float *)cv.take(nb * d * 4);
  float *alpha32 = (float *)cv.take(nb * 4);
  float *strong32 = (float *)cv.take(nb * 4);
  double *exp_tab = (double *)cv.take(64 * 8);
  double *sv64r = (double *)cv.take(nb * 64);
  float *svhl = (float *)cv.take(nb * 64);
  double *alpha64 = (double *)cv.take(nb * 8);
  const int nblk = (n + 31) / 32;
  float *blo = (float *)cv.take((size_t)nblk * d * 4);
  float *bhi = (float *)cv.take((size_t)nblk * d * 4);
  MfTraceBufs B;
  memset(&B, 0, sizeof(B));
  B.etab_key = (unsigned long long *)cv.take(TE * 16);
  B.vtab_key = (unsigned long long *)cv.take(TV * 16);
  B.etab_mask = TE - 1;
  B.vtab_mask = TV - 1;
  B.edge_y = (int32_t *)cv.take(ME * d * 4);
  B.edge_mask = (uint32_t *)cv.take(ME * 4);
  B.edge_f = (double *)cv.take(ME * 16);
  B.edge_t = (double *)cv.take(ME * 8);
  B.edge_pt = (double *)cv.take(ME * d * 8);
  B.max_edges = ME;
  B.vert_y = (int32_t *)cv.take(MV * d * 4);
  B.vert_slot = (uint32_t *)cv.take(MV * 4);
  B.recheck = (uint32_t *)cv.take(MV * 4);
  B.max_vertices = MV;
  B.cell_y = (int32_t *)cv.take(MC * d * 4);
  B.cell_perm = (uint8_t *)cv.take(MC * d);
  B.cell_off = (int64_t *)cv.take((MC + 1) * 8);
  B.cell_idx = (int64_t *)cv.take(cell_edges * 8);
  B.max_cells = MC;
  B.cnt = cnt;
  int64_t *scan_tmp = (int64_t *)cv.take((MC / kScanTile + 2) * 8);
  if (!scan_tmp) return MF_ERR_OOM;

  // Support vectors: the same preparation as mf_trace.
  cudaMemsetAsync(stats, 0, sizeof(MfRbfStats), st);
  // vectors in the caller's order (no host pass): the block screen still
  // holds, it just skips fewer blocks
  k_prepare_rbf<<<(n + 255) / 256, 256, 0, st>>>(d, n, rbf->sv, rbf->alpha, nullptr, sv32, svlo32,
                                                  sv64, alpha64, alpha32, strong32, exp_tab, sv64r,
                                                  svhl, stats);
  k_rbf_blocks<<<(nblk + 7) / 8, 256, 0, st>>>(d, n, nblk, sv32, blo, bhi);
  MfRbfStats hs;
  if (cudaMemcpyAsync(&hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MF_ERR_CUDA;
  if (hs.bad) return MF_ERR_INVALID;
  MfRbfDev R;
  R.d = d;
  R.n = n;
  R.sv32 = sv32;
  R.svlo32 = svlo32;
  R.sv64 = sv64;
  R.alpha = alpha64;
  R.alpha32 = alpha32;
  R.strong32 = strong32;
  R.exp_tab = exp_tab;
  R.sv64r = sv64r;
  R.svhl = svhl;
  R.blk_lo = blo;
  R.blk_hi = bhi;
  R.nblk = nblk;
  R.gamma = rbf->gamma;
  R.b = rbf->b;
  R.sum_abs_alpha = hs.sum_abs_alpha;
  const double sa = hs.sum_abs_alpha > 0 ? hs.sum_abs_alpha : 1e-300;
  double T = std::log(sa / 1e-13);
  T = T < 30.0 ? 30.0 : (T > 740.0 ? 740.0 : T);
  R.screen_r2 = (float)((T + 0.5) / rbf->gamma);
  R.drop_bound = sa * std::exp(-T);
  R.weak_limit = 2.5e-13 - R.drop_bound;
  R.weak_rel = 1.1 * ((d + 2) * 5.9604644775390625e-08 * (T + 0.5)) + 9.5367431640625e-07 +
               2.0 * 5.9604644775390625e-08;
  R.weak_limit32 = (float)R.weak_limit;
  R.drop_bound32 = (float)R.drop_bound;
  R.weak_rel32 = (float)R.weak_rel;
  R.smax = hs.max_abs_s;

  // Everything that must start empty.
  cudaMemsetAsync(cnt, 0, sizeof(MfCounters), st);
  cudaMemsetAsync(B.etab_key, 0xFF, TE * 16, st);
  cudaMemsetAsync(B.vtab_key, 0xFF, TV * 16, st);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MF_ERR_CUDA;
  const double band = opts->recheck_band > 0 ? opts->recheck_band : 1e-3;
  auto eval = [&]() {
    if (mixed) mf_launch_eval_vertices_mixed(F, R, B, opts->precision, band, MfTune(), sms, st);
    else mf_launch_eval_vertices_f64(F, R, B, MfTune(), sms, st);
  };
  MfCounters h;
  if (n_seeds > 0) {
    const unsigned g = (unsigned)((n_seeds + 127) / 128);
    k_seed_vertices<<<g, 128, 0, st>>>(F, B, seeds, n_seeds);
    eval();
    k_seed_edges<<<g, 128, 0, st>>>(F, B, seeds, n_seeds);
  }
  if (cudaGetLastError() != cudaSuccess) return MF_ERR_CUDA;
  if ((rc = sync_read(&h, cnt, st))) return rc;
  const uint64_t cap = opts->batch_cap_edges > 0 ? (uint64_t)opts->batch_cap_edges : (1ull << 24);
  uint64_t fs = 0, fe = h.n_edges;
  int64_t levels = fe > 0 ? 1 : 0;
  while (fe > fs) {
    for (uint64_t a = fs; a < fe; a += cap) {
      const uint64_t m = fe - a < cap ? fe - a : cap;
      const unsigned g = (unsigned)((m + 255) / 256);  // a warp per 32 edges, 8 per block
      k_expand_vertices<<<g, 256, 0, st>>>(F, B, a, m);
      eval();
      k_expand_edges<<<g, 256, 0, st>>>(F, B, a, m);
    }
    if (cudaGetLastError() != cudaSuccess) return MF_ERR_CUDA;
    if ((rc = sync_read(&h, cnt, st))) return rc;
    fs = fe;
    fe = h.n_edges;
    if (fe > fs) levels++;
  }
  const uint64_t E = fe;
  if (opts->flags & MF_WANT_ROOTS)
    mf_launch_roots_f64(F, R, B, E, opts->root_tol > 0 ? opts->root_tol : 1e-12, MfTune(), sms,
                        st);
  int64_t n_cells = 0, n_cell_edges = 0;
  if ((opts->flags & MF_WANT_CELLS) && E > 0) {
    k_cells_enum<<<(unsigned)((E * 32 + 255) / 256), 256, 0, st>>>(F, B, E);
    if ((rc = sync_read(&h, cnt, st))) return rc;
    n_cells = (int64_t)h.n_cells;
    const unsigned g = (unsigned)((n_cells + 255) / 256);
    k_noalloc_cell_edges<false><<<g, 256, 0, st>>>(F, B, (uint64_t)n_cells, B.cell_off);
    const int64_t ntiles = (n_cells + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<(unsigned)ntiles, 512, 0, st>>>(B.cell_off, B.cell_off, n_cells, scan_tmp);
    k_scan_totals<<<1, 512, 0, st>>>(scan_tmp, ntiles, B.cell_off + n_cells);
    k_scan_add<<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(B.cell_off, n_cells, scan_tmp);
    if (cudaMemcpyAsync(&n_cell_edges, B.cell_off + n_cells, 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return MF_ERR_CUDA;
    if ((uint64_t)n_cell_edges > cell_edges) return MF_ERR_MAXEDGES;
    k_noalloc_cell_edges<true><<<g, 256, 0, st>>>(F, B, (uint64_t)n_cells, B.cell_off);
  }
  if (cudaGetLastError() != cudaSuccess) return MF_ERR_CUDA;
  if ((rc = sync_read(&h, cnt, st))) return rc;

  out->n_edges = (int64_t)E;
  out->n_cells = n_cells;
  out->n_cell_edges = n_cell_edges;
  out->n_vertices = (int64_t)h.n_vertices;
  out->n_near_zero = (int64_t)h.n_near_zero;
  out->n_recheck = (int64_t)h.n_recheck;
  out->n_boundary = (int64_t)h.n_boundary;
  out->n_dead_seeds = (int64_t)h.n_dead_seeds;
  out->levels = levels;
  out->root_evals = (int64_t)h.root_evals;
  const bool want_cells = (opts->flags & MF_WANT_CELLS) != 0;
  if (out->cap_edges < out->n_edges || (want_cells && out->cap_cells < n_cells) ||
      (want_cells && out->cell_edge_idx && out->cap_cell_edges < n_cell_edges))
    return MF_ERR_CAPACITY;
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    if (dst && bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
  };
  cp(out->edge_y, B.edge_y, E * d * 4);
  cp(out->edge_mask, B.edge_mask, E * 4);
  cp(out->edge_f, B.edge_f, E * 16);
  if (opts->flags & MF_WANT_ROOTS) {
    cp(out->edge_t, B.edge_t, E * 8);
    cp(out->points, B.edge_pt, E * d * 8);
  }
  if (want_cells) {
    cp(out->cell_y, B.cell_y, (size_t)n_cells * d * 4);
    cp(out->cell_perm, B.cell_perm, (size_t)n_cells * d);
    cp(out->cell_edge_off, B.cell_off, ((size_t)n_cells + 1) * 8);
    cp(out->cell_edge_idx, B.cell_idx, (size_t)n_cell_edges * 8);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return MF_ERR_CUDA;
  return MF_OK;
}
