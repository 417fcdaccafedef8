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
// before any stream capture.  Under CUDA's lazy module loading the library's
// device code, and with it the array, is loaded on a device by the first call
// or the first launch of any of the library's kernels there: that is the
// moment the array's memory is taken, so make that first call at start-up,
// before the device memory is reserved elsewhere.  Every call on a device
// shares the one array and clears what must start empty (counters, hash
// tables); two calls that overlap on the GPU (different streams, threads)
// race on it and must not be issued.
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
                              float *svhl, float *sv3, float *alpha_lo32, float2 *exp_df,
                              MfRbfStats *st);
__global__ void k_rbf_blocks(int d, int n, int nblk, const float *sv32, float *blo, float *bhi);
__global__ void k_seed_vertices(MfFrame F, MfTraceBufs B, const double *seeds, int64_t n);
__global__ void k_seed_edges(MfFrame F, MfTraceBufs B, const double *seeds, int64_t n);
__global__ void k_expand_vertices(MfFrame F, MfTraceBufs B, uint64_t e0, uint64_t n);
__global__ void k_expand_edges(MfFrame F, MfTraceBufs B, uint64_t e0, uint64_t n);
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

// Sequential 256-byte aligned carving of the array.  A take that does not
// fit marks the carver failed (sticky); the same carve sequence run over a
// null base with no capacity measures the bytes a request needs, so the size
// check and the layout cannot diverge.
struct Carver {
  unsigned char *base;
  size_t used, cap;
  bool failed;
  void *take(size_t bytes) {
    const size_t a = (used + 255) & ~(size_t)255;
    used = a + bytes;
    if (used > cap) {
      failed = true;
      return nullptr;
    }
    return base ? base + a : nullptr;
  }
};

struct NoallocLayout {
  MfCounters *cnt;
  MfRbfStats *stats;
  double *sv64, *exp_tab, *sv64r, *alpha64;
  float *sv32, *svlo32, *alpha32, *strong32, *svhl, *blo, *bhi;
  int64_t *scan_tmp;
};

// Every region of one call, in order; B receives the trace buffers.
void carve(Carver &cv, int d, size_t nb, uint64_t ME, uint64_t MV, uint64_t MC, uint64_t TE,
           uint64_t TV, uint64_t cell_edges, NoallocLayout &L, MfTraceBufs &B) {
  L.cnt = (MfCounters *)cv.take(sizeof(MfCounters));
  L.stats = (MfRbfStats *)cv.take(sizeof(MfRbfStats));
  L.sv64 = (double *)cv.take(nb * d * 8);
  L.sv32 = (float *)cv.take(nb * d * 4);
  L.svlo32 = (float *)cv.take(nb * d * 4);
  L.alpha32 = (float *)cv.take(nb * 4);
  L.strong32 = (float *)cv.take(nb * 4);
  L.exp_tab = (double *)cv.take(64 * 8);
  L.sv64r = (double *)cv.take(nb * 64);
  L.svhl = (float *)cv.take(nb * 64);
  L.alpha64 = (double *)cv.take(nb * 8);
  const size_t nblk = (nb + 31) / 32;
  L.blo = (float *)cv.take(nblk * d * 4);
  L.bhi = (float *)cv.take(nblk * d * 4);
  B.etab_key = (unsigned long long *)cv.take(TE * 16);
  B.vtab_key = (unsigned long long *)cv.take(TV * 16);
  B.edge_y = (int32_t *)cv.take(ME * d * 4);
  B.edge_mask = (uint32_t *)cv.take(ME * 4);
  B.edge_f = (double *)cv.take(ME * 16);
  B.edge_t = (double *)cv.take(ME * 8);
  B.edge_pt = (double *)cv.take(ME * d * 8);
  B.vert_y = (int32_t *)cv.take(MV * d * 4);
  B.vert_slot = (uint32_t *)cv.take(MV * 4);
  B.recheck = (uint32_t *)cv.take(MV * 4);
  B.cell_y = (int32_t *)cv.take(MC * d * 4);
  B.cell_perm = (uint8_t *)cv.take(MC * d);
  B.cell_sgn = (uint32_t *)cv.take(MC * 4);
  B.cell_off = (int64_t *)cv.take((MC + 1) * 8);
  B.cell_idx = (int64_t *)cv.take(cell_edges * 8);
  L.scan_tmp = (int64_t *)cv.take((MC / kScanTile + 2) * 8);
}

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
       opts->precision != MF_MIXED_BF16) ||
      (opts->flags & MF_SORT_OUTPUT))
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
  NoallocLayout L;
  MfTraceBufs B;
  memset(&B, 0, sizeof(B));
  size_t need = 0;
  for (uint64_t def = 1ull << 17;; def >>= 1) {
    ME = opts->max_edges > 0 ? (uint64_t)opts->max_edges : def;
    MV = opts->max_vertices > 0 ? (uint64_t)opts->max_vertices : ME;
    MC = opts->max_cells > 0 ? (uint64_t)opts->max_cells : 2 * ME;
    TE = pow2_at_least(ME + ME / 3 + 1);
    TV = pow2_at_least(MV + MV / 3 + 1);
    cell_edges = MC * (uint64_t)((d + 1) * d / 2);
    Carver dry{nullptr, 0, ~(size_t)0, false};
    carve(dry, d, nb, ME, MV, MC, TE, TV, cell_edges, L, B);
    need = dry.used;
    if (need <= MF_NOALLOC_SCRATCH_BYTES || def < 1024) break;
  }
  if (ME >= (1ull << 32) || MV >= (1ull << 32) || need > MF_NOALLOC_SCRATCH_BYTES)
    return MF_ERR_OOM;  // the request does not fit the fixed scratch array
  Carver cv{base, 0, MF_NOALLOC_SCRATCH_BYTES, false};
  carve(cv, d, nb, ME, MV, MC, TE, TV, cell_edges, L, B);
  if (cv.failed) return MF_ERR_OOM;
  MfCounters *cnt = L.cnt;
  MfRbfStats *stats = L.stats;
  double *sv64 = L.sv64, *exp_tab = L.exp_tab, *sv64r = L.sv64r, *alpha64 = L.alpha64;
  float *sv32 = L.sv32, *svlo32 = L.svlo32, *alpha32 = L.alpha32, *strong32 = L.strong32;
  float *svhl = L.svhl, *blo = L.blo, *bhi = L.bhi;
  int64_t *scan_tmp = L.scan_tmp;
  const int nblk = (n + 31) / 32;
  B.etab_mask = TE - 1;
  B.vtab_mask = TV - 1;
  B.max_edges = ME;
  B.max_vertices = MV;
  B.max_cells = MC;
  B.cnt = cnt;

  // Support vectors: the same preparation as mf_trace.
  cudaMemsetAsync(stats, 0, sizeof(MfRbfStats), st);
  // vectors in the caller's order (no host pass): the block screen still
  // holds, it just skips fewer blocks
  k_prepare_rbf<<<(n + 255) / 256, 256, 0, st>>>(d, n, rbf->sv, rbf->alpha, nullptr, sv32, svlo32,
                                                  sv64, alpha64, alpha32, strong32, exp_tab, sv64r,
                                                  svhl, nullptr, nullptr, nullptr, stats);
  k_rbf_blocks<<<(nblk + 7) / 8, 256, 0, st>>>(d, n, nblk, sv32, blo, bhi);
  MfRbfStats hs;
  if (cudaMemcpyAsync(&hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return MF_ERR_CUDA;
  if (hs.bad) return MF_ERR_INVALID;
  MfRbfDev R = {};
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
  // the mixed paths' root screen: sum|alpha| e^-T <= 1e-12
  {
    double Tf = std::log(sa / 1e-12);
    if (Tf < 30.0) Tf = 30.0;
    if (Tf > T) Tf = T;
    R.screen_r2_fast = (float)((Tf + 0.5) / rbf->gamma);
    R.drop_bound32_fast = (float)(sa * std::exp(-Tf));
  }


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
                        st, mixed && !(opts->flags & MF_ROOTS_FP64_EXACT));
  int64_t n_cells = 0, n_cell_edges = 0;
  if ((opts->flags & MF_WANT_CELLS) && E > 0) {
    // mf_trace's cell rule: the enumeration writes each cell's sign mask and
    // CSR row length, the scan turns the lengths into offsets, the fill
    // looks up the cell's traced edges (a missing one is an error)
    mf_launch_cells_enum(F, B, E, st);
    if ((rc = sync_read(&h, cnt, st))) return rc;
    n_cells = (int64_t)h.n_cells;
    mf_exclusive_scan(B.cell_off, B.cell_off, n_cells, scan_tmp, st);
    if (cudaMemcpyAsync(&n_cell_edges, B.cell_off + n_cells, 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return MF_ERR_CUDA;
    if ((uint64_t)n_cell_edges > cell_edges) return MF_ERR_MAXEDGES;
    mf_launch_cells_fill(F, B, (uint64_t)n_cells, st);
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
