// mf_sort.cu -- the sorted output order of mf_trace (MF_SORT_OUTPUT): edges
// by their 64-bit edge key, cells by (vertex key of z, pi), and the cell ->
// edge CSR carried over to both new orders.
//
// The sort is a stable least-significant-digit radix sort of (key, payload)
// pairs with 8-bit digits; a first pass finds the bits where the keys
// differ, and only the bytes holding such bits are sorted.  Per pass, a
// block owns a tile of 4096 keys:
//   k_sort_hist     digit histogram of the tile (digit-major over the tiles,
//                   so one exclusive scan gives every (digit, tile) its
//                   output offset);
//   k_sort_scatter  each warp re-reads its contiguous 512-key part of the
//                   tile in order, ranks the keys of one digit among
//                   themselves with __match_any_sync and writes them after
//                   the keys of earlier warps and tiles: stable.
#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "mf_internal.cuh"
#include "mf_ctx.h"

#define SORT_THREADS 256
#define SORT_ITEMS 16
#define SORT_TILE (SORT_THREADS * SORT_ITEMS)
#define SORT_SEG (SORT_TILE / (SORT_THREADS / 32))  // keys per warp: 512

__global__ void k_sort_bits(const unsigned long long *keys, int64_t n, unsigned long long *and_or) {
  unsigned long long a = ~0ull, o = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    a &= keys[i];
    o |= keys[i];
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    a &= __shfl_xor_sync(0xffffffffu, a, s);
    o |= __shfl_xor_sync(0xffffffffu, o, s);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAnd(&and_or[0], a);
    atomicOr(&and_or[1], o);
  }
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_hist(const unsigned long long *keys, int64_t n,
                                                            int shift, int64_t *hist, int64_t nb) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = blockIdx.x * (int64_t)SORT_TILE;
#pragma unroll
  for (int i = 0; i < SORT_ITEMS; i++) {
    const int64_t k = base + i * SORT_THREADS + threadIdx.x;
    if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & 0xFFu], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(SORT_THREADS) k_sort_scatter(const unsigned long long *keys,
                                                               const uint32_t *vals, int64_t n,
                                                               int shift, const int64_t *offs,
                                                               int64_t nb,
                                                               unsigned long long *keys_out,
                                                               uint32_t *vals_out) {
  constexpr int W = SORT_THREADS / 32;
  __shared__ int64_t pos[W][256];
  __shared__ int cnt[W][256];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int i = threadIdx.x; i < W * 256; i += SORT_THREADS) cnt[i / 256][i % 256] = 0;
  __syncthreads();
  const int64_t seg = blockIdx.x * (int64_t)SORT_TILE + (int64_t)w * SORT_SEG;
  // 1. digit counts of this warp's part
  for (int c = 0; c < SORT_SEG; c += 32) {
    const int64_t k = seg + c + lane;
    const int dg = k < n ? (int)((keys[k] >> shift) & 0xFFu) : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, dg);
    if (dg < 256 && (peers & lt) == 0) cnt[w][dg] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // 2. where each warp's keys of each digit start
  {
    const int dg = threadIdx.x;  // SORT_THREADS == 256 digits
    int64_t run = offs[(int64_t)dg * nb + blockIdx.x];
    for (int q = 0; q < W; q++) {
      pos[q][dg] = run;
      run += cnt[q][dg];
    }
  }
  __syncthreads();
  // 3. the keys again, in order, to their places
  for (int c = 0; c < SORT_SEG; c += 32) {
    const int64_t k = seg + c + lane;
    const bool have = k < n;
    const unsigned long long key = have ? keys[k] : 0ull;
    const int dg = have ? (int)((key >> shift) & 0xFFu) : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, dg);
    if (have) {
      const int64_t at = pos[w][dg] + __popc(peers & lt);
      keys_out[at] = key;
      vals_out[at] = vals[k];
    }
    __syncwarp();
    if (have && (peers & lt) == 0) pos[w][dg] += __popc(peers);
    __syncwarp();
  }
}

// Stable sort of n (key, payload) pairs; the result is in keys / vals.
// tmp_k, tmp_v: n each; hist: 256 * ceil(n / SORT_TILE) + 1 int64; scan:
// scratch of mf_exclusive_scan for that many entries; ao: 2 words.
static int radix_sort(mf_ctx *ctx, unsigned long long *keys, uint32_t *vals,
                      unsigned long long *tmp_k, uint32_t *tmp_v, int64_t n, int64_t *hist,
                      int64_t *scan, unsigned long long *ao, cudaStream_t st) {
  if (n <= 1) return MF_OK;
  const unsigned long long init[2] = {~0ull, 0ull};
  unsigned long long h[2];
  cudaMemcpyAsync(ao, init, sizeof(init), cudaMemcpyHostToDevice, st);
  k_sort_bits<<<ctx->sms * 4, 256, 0, st>>>(keys, n, ao);
  cudaMemcpyAsync(h, ao, sizeof(h), cudaMemcpyDeviceToHost, st);
  int rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "sort bits");
  if (rc) return rc;
  const unsigned long long diff = h[0] ^ h[1];
  const int64_t nb = (n + SORT_TILE - 1) / SORT_TILE;
  unsigned long long *ka = keys, *kb = tmp_k;
  uint32_t *va = vals, *vb = tmp_v;
  for (int shift = 0; shift < 64; shift += 8) {
    if (!((diff >> shift) & 0xFFull)) continue;
    k_sort_hist<<<(unsigned)nb, SORT_THREADS, 0, st>>>(ka, n, shift, hist, nb);
    mf_exclusive_scan(hist, hist, 256 * nb, scan, st);
    k_sort_scatter<<<(unsigned)nb, SORT_THREADS, 0, st>>>(ka, va, n, shift, hist, nb, kb, vb);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, (size_t)n * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
  }
  return mf_cuda_check(ctx, cudaGetLastError(), "radix sort");
}

__global__ void k_edge_keys(MfFrame F, MfTraceBufs B, uint64_t n, unsigned long long *keys,
                            uint32_t *vals) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t y[MF_MAXD];
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) y[k] = k < F.d ? B.edge_y[i * F.d + k] : 0;
  keys[i] = mf_edge_key(F, y, B.edge_mask[i]);
  vals[i] = (uint32_t)i;
}

// cell keys: lo = pi as base-8 digits (pi_0 most significant), then hi =
// the vertex key of z for the cells in the order of the first sort
__global__ void k_cell_keys_lo(MfFrame F, MfTraceBufs B, uint64_t n, unsigned long long *keys,
                               uint32_t *vals) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long code = 0;
  for (int k = 0; k < F.d; k++) code = (code << 3) | B.cell_perm[i * F.d + k];
  keys[i] = code;
  vals[i] = (uint32_t)i;
}

__global__ void k_cell_keys_hi(MfFrame F, MfTraceBufs B, uint64_t n, const uint32_t *vals,
                               unsigned long long *keys) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t z[MF_MAXD];
  const uint64_t c = vals[i];
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) z[k] = k < F.d ? B.cell_y[c * F.d + k] : 0;
  keys[i] = mf_vertex_key(F, z);
}

__global__ void k_inverse(const uint32_t *perm, uint64_t n, uint32_t *inv) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) inv[perm[i]] = (uint32_t)i;
}

// Sorted copies into the caller's buffers.
__global__ void k_gather_edges(int d, MfTraceBufs B, const uint32_t *perm, uint64_t n, bool roots,
                               int32_t *ey, uint32_t *em, double *ef, double *et, double *ep) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t o = perm[i];
  for (int k = 0; k < d; k++) {
    if (ey) ey[i * d + k] = B.edge_y[o * d + k];
    if (ep && roots) ep[i * d + k] = B.edge_pt[o * d + k];
  }
  if (em) em[i] = B.edge_mask[o];
  if (ef) {
    ef[2 * i] = B.edge_f[2 * o];
    ef[2 * i + 1] = B.edge_f[2 * o + 1];
  }
  if (et && roots) et[i] = B.edge_t[o];
}

__global__ void k_gather_cells(int d, MfTraceBufs B, const uint32_t *perm, uint64_t n, int32_t *cy,
                               uint8_t *cp, int64_t *len) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t o = perm[i];
  for (int k = 0; k < d; k++) {
    if (cy) cy[i * d + k] = B.cell_y[o * d + k];
    if (cp) cp[i * d + k] = B.cell_perm[o * d + k];
  }
  if (len) len[i] = B.cell_off[o + 1] - B.cell_off[o];
}

__global__ void k_gather_csr(MfTraceBufs B, const uint32_t *perm, const uint32_t *inv_e, uint64_t n,
                             const int64_t *new_off, int64_t *idx) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t o = perm[i];
  const int64_t a = B.cell_off[o], b = B.cell_off[o + 1], at = new_off[i];
  for (int64_t j = a; j < b; j++) {
    const int64_t e = B.cell_idx[j];
    idx[at + (j - a)] = e >= 0 ? (int64_t)inv_e[e] : -1;
  }
}

// Computes the sorted orders of the trace in L (edge and cell permutations,
// new -> old, and the edges' inverse) into the context's sort slot.
int mf_sort_trace(mf_ctx *ctx, MfTraceState &L, cudaStream_t st) {
  const uint64_t E = (uint64_t)L.n_edges, C = (uint64_t)L.n_cells;
  if (E >= (1ull << 32) || C >= (1ull << 32))
    return mf_set_error(ctx, MF_ERR_INVALID, "sorted output needs fewer than 2^32 edges and cells");
  const uint64_t N = std::max<uint64_t>(std::max<uint64_t>(E, C), 2);
  const int64_t nb = (int64_t)((N + SORT_TILE - 1) / SORT_TILE);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t hist_n = (size_t)256 * nb + 1;
  const size_t bytes = al(E * 4 + 8) * 2 + al(C * 4 + 8) + al(N * 8) * 2 + al(N * 4) +
                       al(hist_n * 8) + al((hist_n / 4096 + 2) * 8) + 256;
  char *p = (char *)mf_ctx_buffer(ctx, MF_SLOT_SORT, bytes);
  if (!p) return MF_ERR_OOM;
  uint32_t *perm_e = (uint32_t *)p; p += al(E * 4 + 8);
  uint32_t *inv_e = (uint32_t *)p; p += al(E * 4 + 8);
  uint32_t *perm_c = (uint32_t *)p; p += al(C * 4 + 8);
  unsigned long long *keys = (unsigned long long *)p; p += al(N * 8);
  unsigned long long *tk = (unsigned long long *)p; p += al(N * 8);
  uint32_t *tv = (uint32_t *)p; p += al(N * 4);
  int64_t *hist = (int64_t *)p; p += al(hist_n * 8);
  int64_t *scan = (int64_t *)p; p += al((hist_n / 4096 + 2) * 8);
  unsigned long long *ao = (unsigned long long *)p;
  int rc;
  if (E) {
    k_edge_keys<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(L.F, L.B, E, keys, perm_e);
    if ((rc = radix_sort(ctx, keys, perm_e, tk, tv, (int64_t)E, hist, scan, ao, st))) return rc;
    k_inverse<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(perm_e, E, inv_e);
  }
  if (C) {
    k_cell_keys_lo<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(L.F, L.B, C, keys, perm_c);
    if ((rc = radix_sort(ctx, keys, perm_c, tk, tv, (int64_t)C, hist, scan, ao, st))) return rc;
    k_cell_keys_hi<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(L.F, L.B, C, perm_c, keys);
    if ((rc = radix_sort(ctx, keys, perm_c, tk, tv, (int64_t)C, hist, scan, ao, st))) return rc;
  }
  L.perm_e = perm_e;
  L.inv_e = inv_e;
  L.perm_c = perm_c;
  L.sort_scan = scan;
  return mf_cuda_check(ctx, cudaGetLastError(), "sorted output");
}

// The copy-out of mf_trace in the sorted order (the caller checked the
// capacities).
int mf_copy_out_sorted(mf_ctx *ctx, const MfTraceState &L, mf_trace_out *out, cudaStream_t st) {
  const int d = L.F.d;
  const uint64_t E = (uint64_t)L.n_edges, C = (uint64_t)L.n_cells;
  const bool roots = (L.flags & MF_WANT_ROOTS) != 0;
  if (E && (out->edge_y || out->edge_mask || out->edge_f || out->edge_t || out->points))
    k_gather_edges<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(
        d, L.B, L.perm_e, E, roots, out->edge_y, out->edge_mask, out->edge_f, out->edge_t,
        out->points);
  if ((L.flags & MF_WANT_CELLS) && (out->cell_y || out->cell_perm || out->cell_edge_off)) {
    if (C) {
      k_gather_cells<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(
          d, L.B, L.perm_c, C, out->cell_y, out->cell_perm, out->cell_edge_off);
      if (out->cell_edge_off) {
        mf_exclusive_scan(out->cell_edge_off, out->cell_edge_off, (int64_t)C, L.sort_scan, st);
        if (out->cell_edge_idx)
          k_gather_csr<<<(unsigned)((C + 255) / 256), 256, 0, st>>>(
              L.B, L.perm_c, L.inv_e, C, out->cell_edge_off, out->cell_edge_idx);
      }
    } else if (out->cell_edge_off) {
      cudaMemsetAsync(out->cell_edge_off, 0, 8, st);
    }
  }
  return mf_cuda_check(ctx, cudaGetLastError(), "sorted copy");
}
