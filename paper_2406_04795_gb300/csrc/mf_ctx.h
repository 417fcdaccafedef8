// mf_ctx.h -- host-side layout of a library context (private).
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "mf_internal.cuh"

// The result of the last mf_trace on a context: its frame, buffers and counts.
struct MfTraceState {
  bool valid = false;
  MfFrame F;
  MfTraceBufs B;
  MfRbfDev R;
  int32_t precision = 0;
  double band = 0.0, tol = 0.0;
  int64_t n_edges = 0, n_cells = 0, n_cell_edges = 0, n_vertices = 0, n_near_zero = 0,
          n_recheck = 0, n_boundary = 0, n_dead_seeds = 0, levels = 0, root_evals = 0;
  uint32_t flags = 0;
  // MF_SORT_OUTPUT: the sorted orders (new -> old) and the edges' inverse,
  // in MF_SLOT_SORT, with a scan scratch for the CSR copy
  bool sorted = false;
  const uint32_t *perm_e = nullptr, *inv_e = nullptr, *perm_c = nullptr;
  int64_t *sort_scan = nullptr;
};

int mf_sort_trace(mf_ctx *ctx, MfTraceState &L, cudaStream_t st);
int mf_copy_out_sorted(mf_ctx *ctx, const MfTraceState &L, mf_trace_out *out, cudaStream_t st);

// Batch triangulation in progress (mf_subdiv_begin / mf_subdiv_next): the
// coarse trace's crossing n-simplices and the shared local template live in
// MF_SLOT_SUBDIV; each batch reuses the trace slots for its fine tables.
struct MfSubdivState {
  bool valid = false;
  MfFrame F;  // the fine frame (scale lambda) with its domain table
  MfRbfDev R;
  int32_t k = 0, precision = 0;
  uint32_t flags = 0;
  double band = 0.0, tol = 0.0;
  uint64_t ME = 0, MV = 0;
  int64_t n_cells = 0, next = 0, per_batch = 0, coarse_levels = 0, dead_seeds = 0;
  const int32_t *cell_y = nullptr;   // [n_cells][d] coarse cells (z)
  const uint8_t *cell_perm = nullptr;  // [n_cells][d] (pi)
  const uint8_t *tv = nullptr;       // [nv][d] local template vertices v'
  const uint32_t *te = nullptr;      // [ne] local edges: (vertex index << 8) | local mask
  int32_t nv = 0, ne = 0;
};

// Event pairs recorded around library launches while profiling is on.
struct MfProfiler {
  bool on = false;
  mf_stats stats = {};
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  size_t used = 0;
};

struct mf_ctx {
  int device = 0;
  int sms = 0;
  size_t budget = 0;
  size_t total = 0;
  std::string err;
  void *slot_ptr[MF_NUM_SLOTS] = {};
  size_t slot_bytes[MF_NUM_SLOTS] = {};
  MfCounters *h_counters = nullptr;  // pinned host mirror of the device counters
  MfTraceState last;
  MfSubdivState sub;
  MfProfiler prof;
  MfTune tune;
};

void mf_frame_lattice(MfFrame *F, int d, double lam, const double *o);

// Profiling scope: records an event pair around the launches issued between
// construction and destruction (no-op when profiling is off).
struct MfProfScope {
  mf_ctx *c;
  int phase;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  MfProfScope(mf_ctx *ctx, int ph, cudaStream_t s, int launches, int64_t units = 0);
  ~MfProfScope();
};
// Resolves pending event pairs into the stats (call after a stream sync).
void mf_prof_collect(mf_ctx *c);
