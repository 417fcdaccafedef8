// mf_trace.cu -- manifold tracing over the Coxeter triangulation
// (Sec. IV-A, Figs. 3-4), the crossing n-simplices (Sec. IV-C), and the host
// driver of mf_trace.
//
// Device state of one trace (all resident in the context):
//   edge table   key(y, p1) -> index in the edge list     (dedup, Sec. IV-A)
//   vertex table key(y)     -> f(y)                        (each vertex evaluated once)
//   cell list    (z, pi), each n-coface written once by its canonical pair (Sec. IV-C)
//   edge list    insertion order; BFS level L is the contiguous range appended
//                while level L-1 was expanded, so the list is also the queue.
//
// One BFS level, per frontier chunk of <= batch_cap edges:
//   k_expand_vertices  warp per 32 edges, lane per coface item (the new
//                      vertex w of one 2-simplex coface, query type 3): w is
//                      inserted into the vertex table; first inserters append
//                      it to the vertex list.
//   eval               f at the newly appended vertices (FP64 or mixed).
//   k_expand_edges     same items: sign of f(w) decides which of the coface's
//                      two edges through w crosses (query type 4); insert it into
//                      the edge table; first inserters append it to the edge list.
#include <algorithm>
#include <cmath>
#include <vector>
#include <cstdio>
#include <cstring>

#include "mf_internal.cuh"
#include "mf_ctx.h"

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_y(const int32_t *src, int d, int32_t *y) {
#pragma unroll
  for (int k = 0; k < MF_MAXD; k++) y[k] = k < d ? src[k] : 0;
}

__device__ __forceinline__ bool vertex_in(const MfFrame &F, const int32_t *v) {
  return mf_vertex_in(F, v);
}

// ---------------------------------------------------------------------------
// Locate edges (Fig. 3): seed -> n-simplex (query type 1) -> its vertices.
// ---------------------------------------------------------------------------
__global__ void k_seed_vertices(MfFrame F, MfTraceBufs B, const double *seeds, int64_t n) {
  constexpr bool DEAD_COUNT = false;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int d = F.d;
  double x[MF_MAXD];
  bool finite = true;
  for (int k = 0; k < d; k++) {
    x[k] = seeds[s * d + k];
    finite = finite && isfinite(x[k]) && fabs(x[k]) < 1e12;
  }
  if (!finite) {  // a non-finite seed locates nothing; it counts as dead
    if (DEAD_COUNT) atomicAdd(&B.cnt->n_dead_seeds, 1ull);
    return;
  }
  int32_t v[MF_MAXD];
  int perm[MF_MAXD];
  mf_locate_point(F, x, v, perm);
  // f is needed at the vertices of the simplex's in-box edges: none when
  // fewer than two of its vertices lie in the box
  int n_in = 0;
  {
    int32_t u[MF_MAXD];
    for (int k = 0; k < MF_MAXD; k++) u[k] = v[k];
    for (int j = 0; j <= d; j++) {
      n_in += vertex_in(F, u) ? 1 : 0;
      if (j < d) u[perm[j]] += 1;
    }
  }
  if (n_in < 2) return;
  for (int j = 0; j <= d; j++) {
    if (vertex_in(F, v)) mf_visit_vertex(F, B, v);
    if (j < d) v[perm[j]] += 1;
  }
}

// The (d+1)d/2 edges of each seed's n-simplex (query type 2) that cross.
__global__ void k_seed_edges(MfFrame F, MfTraceBufs B, const double *seeds, int64_t n) {
  constexpr bool DEAD_COUNT = true;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int d = F.d;
  double x[MF_MAXD];
  bool finite = true;
  for (int k = 0; k < d; k++) {
    x[k] = seeds[s * d + k];
    finite = finite && isfinite(x[k]) && fabs(x[k]) < 1e12;
  }
  if (!finite) {  // a non-finite seed locates nothing; it counts as dead
    if (DEAD_COUNT) atomicAdd(&B.cnt->n_dead_seeds, 1ull);
    return;
  }
  int32_t y[MF_MAXD];
  int perm[MF_MAXD];
  mf_locate_point(F, x, y, perm);
  bool any = false;
  int32_t vi[MF_MAXD];
  load_y(y, d, vi);
  for (int i = 0; i < d; i++) {
    const bool in_i = vertex_in(F, vi);
    // f is known at a vertex only if it belongs to an in-box edge: looked up
    // when the first such edge appears
    double fi = 0.0;
    bool have_fi = false;
    uint32_t mask = 0;
    int32_t vj[MF_MAXD];
    load_y(vi, d, vj);
    for (int j = i + 1; j <= d; j++) {
      mask |= 1u << perm[j - 1];
      vj[perm[j - 1]] += 1;
      if (!in_i || !vertex_in(F, vj)) continue;
      if (!have_fi) {
        fi = mf_lookup_f(F, B, vi);
        have_fi = true;
      }
      const double fj = mf_lookup_f(F, B, vj);
      if ((fi >= 0.0) == (fj >= 0.0)) continue;
      any = true;
      mf_emit_edge(F, B, vi, mask, fi, fj);
    }
    vi[perm[i]] += 1;
  }
  if (!any) atomicAdd(&B.cnt->n_dead_seeds, 1ull);
}

// ---------------------------------------------------------------------------
// Search edges (Fig. 4).  For edge (y, S), S = p1, T = {0..d-1} \ S, the
// 2-simplex cofaces (query type 3, ordered two-set partitions of p1 and of
// p2 = T + {d}) are, for each non-empty mask M:
//   M a proper subset of S : triangle (y, (M, S\M, p2)),          new vertex y + e(M)
//   M a subset of T        : triangle (y, (S, M, rest)),          new vertex y + e(S) + e(M)
//                            triangle (y - e(M), (M, S, rest)),    new vertex y - e(M)
// Each new vertex is one work item: 2^|S| - 2 + 2 (2^|T| - 1) per edge.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t expand_item_count(uint32_t S, int d) {
  const int k = __popc(S);
  return (1u << k) - 2u + 2u * ((1u << (d - k)) - 1u);
}

// The v-th subset of `mask` in binary counting order: bit j of v selects the
// j-th lowest set bit of mask.
__device__ __forceinline__ uint32_t deposit_bits(uint32_t v, uint32_t mask) {
  uint32_t r = 0;
  for (uint32_t m = mask; m && v; m &= m - 1u, v >>= 1)
    if (v & 1u) r |= m & (0u - m);
  return r;
}

// Item r of edge (y, S): kind 0 -> vertex y + e(M), M the (r+1)-th subset of
// S (r < 2^|S| - 2, so M is proper and non-empty); otherwise with
// r' = r - (2^|S| - 2), M is the (r'/2 + 1)-th subset of T and kind 1 ->
// y + e(S) + e(M) (r' even), kind 2 -> y - e(M) (r' odd).
__device__ __forceinline__ uint32_t expand_item_decode(uint32_t S, int d, uint32_t r, int *kind) {
  const uint32_t nsub = (1u << __popc(S)) - 2u;
  if (r < nsub) {
    *kind = 0;
    return deposit_bits(r + 1u, S);
  }
  r -= nsub;
  *kind = 1 + (int)(r & 1u);
  return deposit_bits((r >> 1) + 1u, ~S & ((1u << d) - 1u));
}

// Visits the new vertex of one item; returns 1 if it lies outside the box.
// *slot: its table slot (~0u outside the box or with a full table).
__device__ __forceinline__ unsigned expand_vertices_item(const MfFrame &F, const MfTraceBufs &B,
                                                         uint64_t e, uint32_t S, int kind,
                                                         uint32_t M, uint32_t *slot = nullptr) {
  const int d = F.d;
  int32_t w[MF_MAXD];
  load_y(B.edge_y + e * d, d, w);
  if (kind == 0) mf_add_mask(d, w, M, 1);
  else if (kind == 1) mf_add_mask(d, w, S | M, 1);
  else mf_add_mask(d, w, M, -1);
  if (vertex_in(F, w)) {
    const uint64_t sl = mf_visit_vertex(F, B, w);
    if (slot) *slot = sl == ~0ull ? ~0u : (uint32_t)sl;
    return 0;
  }
  if (slot) *slot = ~0u;
  return 1;
}

// Under the sign rule s = [f >= 0] a crossing triangle has exactly two
// crossing edges (Sec. IV-A): the parent and the one joining the new vertex w
// to the parent end whose sign differs from s(w).
// slot: the new vertex's table slot recorded by k_expand_vertices (~0u:
// outside the box), or MF_SLOT_UNKNOWN to look it up.
#define MF_SLOT_UNKNOWN 0xfffffffeu
__device__ __forceinline__ void expand_edges_item(const MfFrame &F, const MfTraceBufs &B,
                                                  uint64_t e, uint32_t S, int kind, uint32_t M,
                                                  uint32_t slot = MF_SLOT_UNKNOWN) {
  const int d = F.d;
  int32_t y[MF_MAXD], w[MF_MAXD];
  load_y(B.edge_y + e * d, d, y);
  load_y(y, d, w);
  if (kind == 0) mf_add_mask(d, w, M, 1);
  else if (kind == 1) mf_add_mask(d, w, S | M, 1);
  else mf_add_mask(d, w, M, -1);
  double fw;
  if (slot == MF_SLOT_UNKNOWN) {
    if (!vertex_in(F, w)) return;
    fw = mf_lookup_f(F, B, w);
  } else {
    if (slot == ~0u) return;
    fw = mf_vtab_f(B, slot);
  }
  const double f0 = B.edge_f[2 * e], f1 = B.edge_f[2 * e + 1];
  const bool cross0 = (fw >= 0.0) != (f0 >= 0.0);
  if (kind == 0) {
    if (cross0) mf_emit_edge(F, B, y, M, f0, fw);
    else mf_emit_edge(F, B, w, S & ~M, fw, f1);
  } else if (kind == 1) {
    if (cross0) {
      mf_emit_edge(F, B, y, S | M, f0, fw);
    } else {
      mf_add_mask(d, y, S, 1);
      mf_emit_edge(F, B, y, M, f1, fw);
    }
  } else {
    if (cross0) mf_emit_edge(F, B, w, M, fw, f0);
    else mf_emit_edge(F, B, w, M | S, fw, f1);
  }
}

// Inclusive warp scan of the per-lane item counts into s_end[0..31]; returns
// the warp's total.  Item j then belongs to the first lane o with
// s_end[o] > j, as local item j - s_end[o - 1].
__device__ __forceinline__ uint32_t expand_warp_scan(uint32_t c, uint32_t *s_end) {
  const int lane = threadIdx.x & 31;
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  s_end[lane] = inc;
  __syncwarp();
  return __shfl_sync(0xffffffffu, inc, 31);
}

__device__ __forceinline__ int expand_owner(const uint32_t *s_end, uint32_t j, uint32_t *local) {
  int o = 0;
#pragma unroll
  for (int step = 16; step; step >>= 1)
    if (s_end[o + step - 1] <= j) o += step;
  *local = j - (o ? s_end[o - 1] : 0u);
  return o;
}

#define EXPAND_WARPS 8

// Warp per 32 consecutive edges of [e0, e0 + n), lane per coface item, so
// that no lane idles on masks that select no coface.
template <bool EDGES>
__device__ __forceinline__ void expand_warp(const MfFrame &F, const MfTraceBufs &B, uint64_t e0,
                                            uint64_t n) {
  __shared__ uint32_t s_end[EXPAND_WARPS][32], s_S[EXPAND_WARPS][32];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const uint64_t first = (blockIdx.x * (uint64_t)EXPAND_WARPS + wi) * 32;
  if (first >= n) return;  // whole warp
  const int d = F.d;
  uint32_t S = 0, c = 0;
  if (first + lane < n) {
    S = B.edge_mask[e0 + first + lane];
    c = S ? expand_item_count(S, d) : 0u;
  }
  s_S[wi][lane] = S;
  const uint32_t total = expand_warp_scan(c, s_end[wi]);
  // the warp's items in the chunk's slot record (see MfTraceBufs.item_slot)
  const uint64_t wg = blockIdx.x * (uint64_t)EXPAND_WARPS + wi;
  unsigned long long ib = ~0ull;
  if (B.item_slot) {
    if (EDGES) {
      ib = B.warp_base[wg];
    } else {
      if (lane == 0) {
        ib = atomicAdd(&B.cnt->n_items, (unsigned long long)total);
        if (ib + total > B.item_cap) ib = ~0ull;
        B.warp_base[wg] = ib;
      }
      ib = __shfl_sync(0xffffffffu, ib, 0);
      // each lane's edge: the first of its items
      if (B.edge_item_off && first + lane < n)
        B.edge_item_off[e0 + first + lane] =
            ib == ~0ull ? ~0ull : ib + (lane ? s_end[wi][lane - 1] : 0u);
    }
  }
  unsigned nb = 0;
  for (uint32_t j = lane; j < total; j += 32) {
    uint32_t r;
    const int o = expand_owner(s_end[wi], j, &r);
    const uint32_t So = s_S[wi][o];
    int kind;
    const uint32_t M = expand_item_decode(So, d, r, &kind);
    if (EDGES) {
      expand_edges_item(F, B, e0 + first + o, So, kind, M,
                        ib != ~0ull ? B.item_slot[ib + j] : MF_SLOT_UNKNOWN);
    } else {
      uint32_t sl;
      nb += expand_vertices_item(F, B, e0 + first + o, So, kind, M, &sl);
      if (ib != ~0ull) B.item_slot[ib + j] = sl;
    }
  }
  if (!EDGES) {
    nb = __reduce_add_sync(0xffffffffu, nb);
    if (lane == 0 && nb) atomicAdd(&B.cnt->n_boundary, (unsigned long long)nb);
  }
}

__global__ void __launch_bounds__(EXPAND_WARPS * 32) k_expand_vertices(MfFrame F, MfTraceBufs B,
                                                                       uint64_t e0, uint64_t n) {
  expand_warp<false>(F, B, e0, n);
}

__global__ void __launch_bounds__(EXPAND_WARPS * 32) k_expand_edges(MfFrame F, MfTraceBufs B,
                                                                    uint64_t e0, uint64_t n) {
  expand_warp<true>(F, B, e0, n);
}

// ---------------------------------------------------------------------------
// Cells (Sec. IV-C): the n-simplex cofaces of every traced edge (y, y+e(S)).
// A coface is an ordering sigma of p1 = S followed by an ordering of
// p2 = T u {d} (|p1|!|p2|! of them); the walk is then rotated so that d comes
// last: vertex z = y + sum_{i<pos(d)} e_sigma_i - 1, permutation pi.  In
// the cell's vertex order, position a = d - pos(d) holds y and a + |p1|
// holds y + e(S); positions a + m (0 < m < |p1|) hold y + e(sigma_0..m-1)
// and positions i < a hold y - e(sigma_{pos(d)+i+1..d}).
//
// A cell has several traced edges (every pair of in-domain vertices of
// opposite sign: they are connected through crossing triangles whose
// vertices are in the domain, which the search follows).  It is emitted once,
// by its canonical pair: the first such pair (i, j), i < j, in the order of
// its vertices z, z + e(pi_0), ...  That pair is (y, y + e(S)) exactly when
//   A: every vertex at a position i < a is outside the domain, and
//   B: every vertex at a + m, 0 < m < |p1|, is outside the domain or has y's
//      sign
// (an in-domain vertex before y would pair with y or y + e(S); one between
// them of the other sign would pair with y first).  A constrains only the
// elements after d (each suffix set of them, compressed to T, must index an
// out-of-domain c-vertex), B only the ordering of S (each proper prefix set).
// So the canonical cofaces are (orderings of S passing B) x (suffix
// sequences Q passing A) x (orderings of the rest of T before d), counted by
// chain counts over subsets and unranked directly: the edge enumerates only
// the cells it writes.  The vertex signs come from the edge's link table, so
// the cell needs no hash table, and its sign mask and CSR row length are
// known when it is written.
// ---------------------------------------------------------------------------
__constant__ uint32_t c_fact[13] = {1u, 1u, 2u, 6u, 24u, 120u, 720u, 5040u, 40320u, 362880u,
                                    3628800u, 39916800u, 479001600u};

// Link table of edge (y, S): every vertex of an n-coface of the edge is
// y + e(M) for M within S (a), y + e(S) + e(M) (b) or y - e(M) (c) for M
// within T = {0..d-1} \ S, indexed by M's bits compressed to S or T.
// Entry bit 0: in the vertex table (in the domain); bit 1: f >= 0.
#define LINK_MAX (1 << MF_MAXD)
struct CellLink {
  uint8_t a[LINK_MAX], b[LINK_MAX], c[LINK_MAX];
  uint16_t cnt[LINK_MAX];      // chains of p1 prefixes (subsets of S)
  uint16_t cc[LINK_MAX / 2];   // chains of suffix sets after d (subsets of T)
  uint32_t cum[LINK_MAX / 2 + 1];  // prefix sums of the p2 orderings per suffix set
};
#define CELL_WARPS 8

__device__ __forceinline__ void cells_enum_edge(const MfFrame &F, const MfTraceBufs &B, uint64_t e,
                                                int lane, CellLink &L);

__global__ void __launch_bounds__(CELL_WARPS * 32) k_cells_enum(MfFrame F, MfTraceBufs B,
                                                                uint64_t n_edges) {
  __shared__ CellLink sl[CELL_WARPS];
  const int lane = threadIdx.x & 31;
  const uint64_t e = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (e >= n_edges) return;
  cells_enum_edge(F, B, e, lane, sl[threadIdx.x >> 5]);
}

// The n-cofaces j = lane, lane + 32, ... of edge e (all lanes of the warp).
// Orderings and permutations are kept as 4-bit nibbles in 64-bit words, so
// the decode needs no indexed arrays (they would live in local memory).
__device__ __forceinline__ void cells_enum_edge(const MfFrame &F, const MfTraceBufs &B, uint64_t e,
                                                int lane, CellLink &L) {
  const int d = F.d;
  int32_t y[MF_MAXD];
  load_y(B.edge_y + e * d, d, y);
  const uint32_t S = B.edge_mask[e], T = ~S & ((1u << d) - 1u);
  const int n1 = __popc(S), n2 = d + 1 - n1;
  // the link table, one vertex lookup per entry
  const int na = 1 << n1, nb = 1 << (n2 - 1);
  // the edge's expand items and end values: the link table's vertices are
  // the edge's ends (a[0] = c[0] = y, a[na - 1] = b[0] = y + e(S)) and its
  // coface items (a[q]: item q - 1; b[r], c[r]: items na - 2 + 2 (r - 1)
  // and the one after), whose vertex slots the expansion recorded
  const unsigned long long ioff = B.edge_item_off ? B.edge_item_off[e] : ~0ull;
  const uint8_t c_y = B.edge_f[2 * e] >= 0.0 ? 3 : 1, c_ys = B.edge_f[2 * e + 1] >= 0.0 ? 3 : 1;
  __syncwarp();  // the previous edge's cofaces have read the table
  for (int q = lane; q < na + 2 * nb; q += 32) {
    uint8_t *dst;
    uint32_t M;
    int sgn = 1;
    long long ri;  // the item, -1: an end of the edge
    uint8_t code = 0;
    if (q < na) {
      M = deposit_bits((uint32_t)q, S);
      dst = &L.a[q];
      ri = (q == 0 || q == na - 1) ? -1 : q - 1;
      if (q == 0) code = c_y;
      else if (q == na - 1) code = c_ys;
    } else if (q < na + nb) {
      const uint32_t r = (uint32_t)(q - na);
      M = S | deposit_bits(r, T);
      dst = &L.b[r];
      ri = r == 0 ? -1 : (long long)(na - 2) + 2 * ((long long)r - 1);
      if (r == 0) code = c_ys;
    } else {
      const uint32_t r = (uint32_t)(q - na - nb);
      M = deposit_bits(r, T);
      sgn = -1;
      dst = &L.c[r];
      ri = r == 0 ? -1 : (long long)(na - 2) + 2 * ((long long)r - 1) + 1;
      if (r == 0) code = c_y;
    }
    if (ri >= 0) {
      if (ioff != ~0ull) {
        const uint32_t slot = B.item_slot[ioff + (unsigned long long)ri];
        code = slot == ~0u ? 0 : (mf_vtab_f(B, slot) >= 0.0 ? 3 : 1);
      } else {
        int32_t w[MF_MAXD];
        load_y(y, d, w);
        mf_add_mask(d, w, M, sgn);
        if (vertex_in(F, w)) {
          const uint64_t slot = mf_table_find<2>(B.vtab_key, B.vtab_mask, mf_vertex_key(F, w));
          if (slot != ~0ull) code = mf_vtab_f(B, slot) >= 0.0 ? 3 : 1;
        }
      }
    }
    *dst = code;
  }
  __syncwarp();
  uint64_t ls = 0, lt = 0;  // the elements of S and of T, ascending
  {
    int c1 = 0, c2 = 0;
    for (int i = 0; i < d; i++) {
      if ((S >> i) & 1u) ls |= (uint64_t)i << (4 * c1++);
      else lt |= (uint64_t)i << (4 * c2++);
    }
  }
  const int nt = n2 - 1, nc = 1 << nt;
  // chain counts by subset size: cnt[U] = orderings of U whose nonempty
  // prefix sets all pass B (U = S itself always passes); cc[W] = orderings
  // of W, built from its last element, whose suffix sets all pass A
  const uint32_t ys = (L.a[0] >> 1) & 1u;
  if (na <= 32 && nc <= 32) {
    // lane u holds cnt[u] and cc[u]; each level sums the lanes one bit below
    const uint32_t u = (uint32_t)lane;
    const uint32_t ca = u < (uint32_t)na ? L.a[u] : 0u;
    const bool oka = u < (uint32_t)na && (u == (uint32_t)(na - 1) || !(ca & 1u) || ((ca >> 1) & 1u) == ys);
    const bool okc = u < (uint32_t)nc && !(L.c[u] & 1u);
    uint32_t cv = u == 0 ? 1u : 0u, qv = u == 0 ? 1u : 0u;
    const int levels = n1 > nt ? n1 : nt;
    for (int lev = 1; lev <= levels; lev++) {
      uint32_t sa = 0, sc = 0;
#pragma unroll
      for (int b = 0; b < 5; b++) {
        const uint32_t va = __shfl_xor_sync(0xffffffffu, cv, 1 << b);
        const uint32_t vc = __shfl_xor_sync(0xffffffffu, qv, 1 << b);
        if ((u >> b) & 1u) {
          sa += va;
          sc += vc;
        }
      }
      if (__popc(u) == lev) {
        cv = oka ? sa : 0u;
        qv = okc ? sc : 0u;
      }
    }
    if (u < (uint32_t)na) L.cnt[u] = (uint16_t)cv;
    if (u < (uint32_t)nc) L.cc[u] = (uint16_t)qv;
    __syncwarp();
  } else
  for (int lev = 0; lev <= n1 || lev <= nt; lev++) {
    for (int u = lane; u < na; u += 32) {
      if (__popc(u) != lev) continue;
      uint32_t v = 1;
      if (u) {
        const uint32_t code = L.a[u];
        v = 0;
        if (u == na - 1 || !(code & 1u) || ((code >> 1) & 1u) == ys)
          for (uint32_t m = (uint32_t)u; m; m &= m - 1) v += L.cnt[u & ~(m & (0u - m))];
      }
      L.cnt[u] = (uint16_t)v;
    }
    for (int w = lane; w < nc; w += 32) {
      if (__popc(w) != lev) continue;
      uint32_t v = 1;
      if (w) {
        v = 0;
        if (!(L.c[w] & 1u))
          for (uint32_t m = (uint32_t)w; m; m &= m - 1) v += L.cc[w & ~(m & (0u - m))];
      }
      L.cc[w] = (uint16_t)v;
    }
    __syncwarp();
  }
  // cum[w]: p2 orderings whose suffix set (compressed) is below w: each set
  // W contributes cc[W] (|T| - |W|)! (the rest of T in any order before d)
  uint32_t run = 0;
  for (int base = 0; base < nc; base += 32) {
    const int w = base + lane;
    uint32_t inc = w < nc ? (uint32_t)L.cc[w] * c_fact[nt - __popc(w)] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (w < nc) L.cum[w + 1] = run + inc;
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (lane == 0) L.cum[0] = 0;
  __syncwarp();
  const uint32_t c1 = L.cnt[na - 1], total = c1 * run;
  if (total == 0) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&B.cnt->n_cells, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (uint32_t k = lane; k < total; k += 32) {
    const unsigned long long idx = base + k;
    if (idx >= B.max_cells) { atomicOr(&B.cnt->err_overflow, 1u); continue; }
    // unrank: k = k1 + c1 k2; the ordering of S from its last element back
    uint32_t k1 = k % c1, k2 = k / c1;
    uint64_t sig = 0;
    {
      uint32_t u = (uint32_t)(na - 1);
      for (int pos = n1 - 1; pos >= 0; pos--) {
        for (uint32_t m = u; m; m &= m - 1) {
          const uint32_t bit = m & (0u - m), c = L.cnt[u & ~bit];
          if (k1 < c) {
            sig |= ((ls >> (4 * (__ffs(bit) - 1))) & 15ull) << (4 * pos);
            u &= ~bit;
            break;
          }
          k1 -= c;
        }
      }
    }
    // the suffix set W: the first w with cum[w + 1] > k2
    int lo = 0, hi = nc - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (L.cum[mid + 1] > k2) hi = mid; else lo = mid + 1;
    }
    const uint32_t w = (uint32_t)lo, cw = L.cc[w];
    const uint32_t r2 = k2 - L.cum[w], kp = r2 / cw;
    uint32_t kq = r2 - kp * cw;
    const int nw = __popc(w), nP = nt - nw, p = n1 + nP;
    // the rest of T before d, ordering kp (Lehmer code)
    {
      uint64_t pool = 0;
      int np = 0;
      for (int b = 0; b < nt; b++)
        if (!((w >> b) & 1u)) pool |= ((lt >> (4 * b)) & 15ull) << (4 * np++);
      uint32_t r = kp;
      for (int i = 0; i < nP; i++) {
        const uint32_t f = c_fact[nP - 1 - i], q = r / f;
        r -= q * f;
        sig |= ((pool >> (4 * q)) & 15ull) << (4 * (n1 + i));
        const uint64_t low = q ? (pool & ((1ull << (4 * q)) - 1ull)) : 0ull;
        pool = low | ((pool >> (4 * (q + 1))) << (4 * q));
      }
    }
    sig |= (uint64_t)d << (4 * p);
    // Q after d: walking W back to the empty set gives q_1, q_2, ...
    {
      uint32_t ww = w;
      for (int pos = p + 1; pos <= d; pos++) {
        for (uint32_t m = ww; m; m &= m - 1) {
          const uint32_t bit = m & (0u - m), c = L.cc[ww & ~bit];
          if (kq < c) {
            sig |= ((lt >> (4 * (__ffs(bit) - 1))) & 15ull) << (4 * pos);
            ww &= ~bit;
            break;
          }
          kq -= c;
        }
      }
    }
    // vertex signs in the cell's order: y sits at position a = d - p and
    // y + e(S) at a + n1; positions a + m (m <= p) are y + e(sigma_0..m-1),
    // positions i < a are y - e(sigma_{p+i+1..d})
    const int a = d - p;
    uint32_t inm = 0, posm = 0, ia = 0, ib = 0, ic = 0;
    for (int m = 0; m <= p; m++) {
      if (m > 0) {
        const uint32_t v = (uint32_t)((sig >> (4 * (m - 1))) & 15ull);
        if (m - 1 < n1) ia |= 1u << __popc(S & ((1u << v) - 1u));
        else ib |= 1u << __popc(T & ((1u << v) - 1u));
      }
      const uint32_t code = m <= n1 ? L.a[ia] : L.b[ib];
      inm |= (code & 1u) << (a + m);
      posm |= ((code >> 1) & 1u) << (a + m);
    }
    for (int i = a - 1; i >= 0; i--) {
      const uint32_t v = (uint32_t)((sig >> (4 * (p + i + 1))) & 15ull);
      ic |= 1u << __popc(T & ((1u << v) - 1u));
      const uint32_t code = L.c[ic];
      inm |= (code & 1u) << i;
      posm |= ((code >> 1) & 1u) << i;
    }
    // the canonical pair, checked: the first position i with an in-domain
    // vertex of the other sign after it (a positive vertex below the highest
    // negative one, or the reverse), and the first such vertex after it,
    // must be a and a + n1
    const uint32_t P = inm & posm, N = inm & ~posm;
    const uint32_t belowN = N ? (1u << (31 - __clz(N))) - 1u : 0u;  // positions below N's top
    const uint32_t belowP = P ? (1u << (31 - __clz(P))) - 1u : 0u;
    const uint32_t cand = (P & belowN) | (N & belowP);
    const int ci = cand ? __ffs(cand) - 1 : -1;
    bool canon = false;
    if (ci == a) {
      const uint32_t other = (((P >> ci) & 1u) ? N : P) >> (ci + 1);
      canon = ci + __ffs(other) == a + n1;
    }
    if (!canon) atomicOr(&B.cnt->err_missing, 4u);
    // z = y + e(sigma_0..sigma_{p-1}) - 1; pi = sigma_{p+1..d}, sigma_{0..p-1}
    uint32_t inc = 0;
    for (int i = 0; i < p; i++) inc |= 1u << ((sig >> (4 * i)) & 15ull);
    const uint64_t hi4 = sig >> (4 * (p + 1)), lo4 = p ? (sig & ((1ull << (4 * p)) - 1ull)) : 0ull;
    const uint64_t pi = hi4 | (lo4 << (4 * (d - p)));
    for (int k2i = 0; k2i < d; k2i++) {
      B.cell_y[idx * d + k2i] = y[k2i] + (int32_t)((inc >> k2i) & 1u) - 1;
      B.cell_perm[idx * d + k2i] = (uint8_t)((pi >> (4 * k2i)) & 15ull);
    }
    // sign mask and CSR row length (paths without these arrays count later)
    if (B.cell_sgn) B.cell_sgn[idx] = inm | (posm << 16);
    if (B.cell_off) B.cell_off[idx] = (int64_t)__popc(P) * (int64_t)__popc(N);
  }
}

// Cell -> traced edges: the (d+1)d/2 edges of the cell (query type 2) found
// in the edge table.  FILL = false counts, FILL = true writes indices.
template <bool FILL>
__device__ __forceinline__ void cell_edges_item(const MfFrame &F, const MfTraceBufs &B, uint64_t c,
                                                int64_t *cnt_or_off);

template <bool FILL>
__global__ void k_cells_edges(MfFrame F, MfTraceBufs B, uint64_t n_cells, int64_t *cnt_or_off) {
  const uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  cell_edges_item<FILL>(F, B, c, cnt_or_off);
}

template <bool FILL>
__device__ __forceinline__ void cell_edges_item(const MfFrame &F, const MfTraceBufs &B, uint64_t c,
                                                int64_t *cnt_or_off) {
  // The cell's vertices v_0 = z, v_i = v_{i-1} + e(pi_{i-1}) (query type 5).
  // Each of them lies in the domain iff it is in the vertex table: the BFS
  // visits the third vertex of every 2-coface of a traced edge, and every
  // vertex of this cell shares a 2-coface with the traced edge that made it.
  // Inside one simplex all crossing edges between in-domain vertices are
  // linked through 2-cofaces, so the traced edges of the cell are exactly its
  // in-domain vertex pairs with different signs: the count pass needs only
  // the d+1 vertex signs, and the fill pass looks up only those pairs.
  const int d = F.d;
  int32_t vi[MF_MAXD];
  load_y(B.cell_y + c * d, d, vi);
  // the permutation as 4-bit nibbles (no indexed local array)
  uint64_t pw = 0;
  for (int k = 0; k < d; k++) pw |= (uint64_t)B.cell_perm[c * d + k] << (4 * k);
  uint32_t sg;
  if (!FILL) {
    uint32_t in = 0, pos = 0;
    int32_t w[MF_MAXD];
    load_y(vi, d, w);
    for (int i = 0; i <= d; i++) {
      if (i > 0) {
        const int p = (int)((pw >> (4 * (i - 1))) & 15ull);
#pragma unroll
        for (int k = 0; k < MF_MAXD; k++) w[k] += k == p ? 1 : 0;
      }
      const uint64_t slot = mf_table_find<2>(B.vtab_key, B.vtab_mask, mf_vertex_key(F, w));
      if (slot == ~0ull) continue;
      in |= 1u << i;
      if (mf_vtab_f(B, slot) >= 0.0) pos |= 1u << i;
    }
    sg = in | (pos << 16);
    B.cell_sgn[c] = sg;
    cnt_or_off[c] = (int64_t)__popc(in & pos) * (int64_t)__popc(in & ~pos);
    return;
  }
  sg = B.cell_sgn[c];
  const uint32_t in = sg & 0xFFFFu, pos = sg >> 16;
  int64_t at = cnt_or_off[c];
  for (int i = 0; i < d; i++) {
    uint32_t mask = 0;
    for (int j = i + 1; j <= d; j++) {
      mask |= 1u << (uint32_t)((pw >> (4 * (j - 1))) & 15ull);
      if (!((in >> i) & (in >> j) & 1u) || ((pos >> i) & 1u) == ((pos >> j) & 1u)) continue;
      const uint64_t slot = mf_table_find<2>(B.etab_key, B.etab_mask, mf_edge_key(F, vi, mask));
      if (slot == ~0ull) {
        atomicOr(&B.cnt->err_missing, 2u);
        B.cell_idx[at++] = -1;
        continue;
      }
      B.cell_idx[at++] = (int64_t)mf_etab_val(B, slot);
    }
    const int p = (int)((pw >> (4 * i)) & 15ull);
#pragma unroll
    for (int k = 0; k < MF_MAXD; k++) vi[k] += k == p ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// Batched kernels: all traces of a batch advance together.  Plan kernels run
// as one block of MF_MAX_SLOTS threads (thread t = slot t) and write work
// prefixes; work kernels are grid-stride loops over the prefix total, so a
// step can be captured once in a CUDA graph and replayed for any mix of
// active traces.
// ---------------------------------------------------------------------------
__device__ unsigned long long block_scan_u64(unsigned long long v, unsigned long long *total) {
  __shared__ unsigned long long wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    const unsigned long long t = lane < nw ? wsum[lane] : 0ull;
    unsigned long long s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) wsum[lane] = s - t;
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const unsigned long long r = x - v + wsum[w];
  __syncthreads();
  return r;
}

// After the seeds: every slot's first level is its seed edges.
__global__ void k_b_init(const MfSlot *slots, MfSlotState *st, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const MfCounters *c = slots[t].B.cnt;
  MfSlotState s;
  s.cursor = 0;
  s.level_end = c->n_edges < slots[t].B.max_edges ? c->n_edges : slots[t].B.max_edges;
  s.chunk_n = 0;
  s.err = (c->err_table_full || c->err_missing || c->err_overflow || c->err_timeout) ? 1 : 0;
  s.active = (s.level_end > 0 && !s.err) ? 1 : 0;
  s.levels = s.level_end > 0 ? 1 : 0;
  s.pad = 0;
  st[t] = s;
}

__global__ void k_b_plan_expand(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n) {
  __shared__ unsigned long long total;
  const int t = threadIdx.x;
  unsigned long long cnt = 0;
  if (t < n) {
    unsigned long long chunk = 0;
    if (st[t].active) {
      const unsigned long long left = st[t].level_end - st[t].cursor;
      chunk = left < slots[t].cap ? left : slots[t].cap;
    }
    st[t].chunk_n = chunk;
    cnt = chunk;
  }
  const unsigned long long ex = block_scan_u64(cnt, &total);
  if (t < n) P->px[t] = ex;
  if (t == 0) P->px[n] = total;
}

template <bool EDGES>
__global__ void __launch_bounds__(EXPAND_WARPS * 32) k_b_expand(const MfSlot *slots,
                                                                const MfSlotState *st,
                                                                const MfBatchPlan *P, int n) {
  __shared__ uint32_t s_end[EXPAND_WARPS][32], s_S[EXPAND_WARPS][32];
  __shared__ int s_t[EXPAND_WARPS][32];
  __shared__ unsigned long long s_e[EXPAND_WARPS][32], s_io[EXPAND_WARPS][32];
  const unsigned long long total = P->px[n];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * EXPAND_WARPS;
  for (unsigned long long g = blockIdx.x * (unsigned long long)EXPAND_WARPS + wi; g * 32 < total;
       g += nwarps) {
    const unsigned long long item = g * 32 + lane;
    uint32_t S = 0, c = 0;
    int t = 0;
    unsigned long long e = 0;
    if (item < total) {
      t = mf_slot_of(P->px, n, item);
      e = st[t].cursor + (item - P->px[t]);
      S = slots[t].B.edge_mask[e];
      c = S ? expand_item_count(S, slots[t].F.d) : 0u;
    }
    s_S[wi][lane] = S;
    s_t[wi][lane] = t;
    s_e[wi][lane] = e;
    // the edge's first item in its trace's slot record (see
    // MfTraceBufs.item_slot; per edge, as the warp's edges may belong to
    // several traces): taken by the vertices pass, read by the edges pass
    unsigned long long io = ~0ull;
    if (item < total && slots[t].B.item_slot) {
      const MfTraceBufs &TB = slots[t].B;
      if (EDGES) {
        io = TB.edge_item_off[e];
      } else {
        io = atomicAdd(&TB.cnt->n_items, (unsigned long long)c);
        if (io + c > TB.item_cap) io = ~0ull;
        TB.edge_item_off[e] = io;
      }
    }
    s_io[wi][lane] = io;
    const uint32_t nit = expand_warp_scan(c, s_end[wi]);
    for (uint32_t j = lane; j < nit; j += 32) {
      uint32_t r;
      const int o = expand_owner(s_end[wi], j, &r);
      const MfSlot &SL = slots[s_t[wi][o]];
      const uint32_t So = s_S[wi][o];
      const unsigned long long oo = s_io[wi][o];
      int kind;
      const uint32_t M = expand_item_decode(So, SL.F.d, r, &kind);
      if (EDGES) {
        expand_edges_item(SL.F, SL.B, s_e[wi][o], So, kind, M,
                          oo != ~0ull ? SL.B.item_slot[oo + r] : MF_SLOT_UNKNOWN);
      } else {
        uint32_t sl;
        if (expand_vertices_item(SL.F, SL.B, s_e[wi][o], So, kind, M, &sl))
          atomicAdd(&SL.B.cnt->n_boundary, 1ull);
        if (oo != ~0ull) SL.B.item_slot[oo + r] = sl;
      }
    }
    __syncwarp();  // the next group overwrites this warp's shared entries
  }
}

// Vertex-evaluation and FP64-recheck ranges of every slot, and the
// tensor-core tiles of the MF_MIXED_BF16 slots.
__global__ void k_b_plan_eval(const MfSlot *slots, MfBatchPlan *P, int n) {
  __shared__ unsigned long long total, ttotal;
  const int t = threadIdx.x;
  unsigned long long cv = 0, ct = 0;
  if (t < n && slots[t].B.cnt) {  // empty (zeroed) descriptors hold no trace
    const MfTraceBufs &B = slots[t].B;
    const unsigned long long v0 = B.cnt->v_evaluated;
    unsigned long long v1 = B.cnt->n_vertices;
    if (v1 > B.max_vertices) v1 = B.max_vertices;
    cv = v1 > v0 ? v1 - v0 : 0;
    if (slots[t].precision == MF_MIXED_BF16) ct = (cv + MF_TC_TILE - 1) / MF_TC_TILE;
    P->v0[t] = v0;
  }
  const unsigned long long ex = block_scan_u64(cv, &total);
  const unsigned long long et = block_scan_u64(ct, &ttotal);
  if (t < n) {
    P->pv[t] = ex;
    P->pt[t] = et;
  }
  if (t == 0) {
    P->pv[n] = total;
    P->pt[n] = ttotal;
  }
}

__global__ void k_b_plan_recheck(const MfSlot *slots, MfBatchPlan *P, int n) {
  __shared__ unsigned long long total;
  const int t = threadIdx.x;
  unsigned long long cr = 0;
  if (t < n && slots[t].B.cnt) {
    const MfTraceBufs &B = slots[t].B;
    const unsigned long long r0 = B.cnt->n_recheck_done;
    unsigned long long r1 = B.cnt->n_recheck;
    if (r1 > B.max_vertices) r1 = B.max_vertices;
    cr = r1 > r0 ? r1 - r0 : 0;
    P->r0[t] = r0;
  }
  const unsigned long long ex = block_scan_u64(cr, &total);
  if (t < n) P->pr[t] = ex;
  if (t == 0) P->pr[n] = total;
}

__global__ void k_b_advance(const MfSlot *slots, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n || !slots[t].B.cnt) return;
  MfCounters *c = slots[t].B.cnt;
  c->v_evaluated = c->n_vertices;
  c->n_recheck_done = c->n_recheck;
}

// End of a step: advance each slot's cursor; a finished level opens the next
// one if it appended edges, otherwise the slot is done.  Any slot still active
// keeps the enclosing graph loop running.
__global__ void k_b_update(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n,
                           cudaGraphConditionalHandle handle, int use_handle) {
  __shared__ int any, stop, pause;
  if (threadIdx.x == 0) {
    any = 0;
    // a hard bound on the number of steps: the loop ends even if a slot
    // never finished (reported as an overrun error)
    const unsigned long long s = ++P->steps;
    stop = s > MF_MAX_STEPS;
    if (stop) P->overrun = 1;
    // a step budget ends this launch of the loop; active slots stay active
    pause = P->budget > 0 && s >= (unsigned long long)P->budget;
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < n && st[t].active && stop) {
    st[t].active = 0;
    st[t].err = 1;
  } else if (t < n && st[t].active) {
    MfSlotState s = st[t];
    s.cursor += s.chunk_n;
    s.chunk_n = 0;
    if (s.cursor >= s.level_end) {
      const MfCounters *c = slots[t].B.cnt;
      const unsigned long long ne = c->n_edges;
      if (c->err_table_full || c->err_missing || c->err_overflow || c->err_timeout ||
          ne > slots[t].B.max_edges) {
        s.err = 1;
        s.active = 0;
      } else if (ne > s.level_end) {
        s.level_end = ne;
        s.levels++;
      } else {
        s.active = 0;
      }
    }
    st[t] = s;
    if (s.active) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(handle, (any && !pause) ? 1u : 0u);
}

// Traced-edge and cell prefixes.  mode 0: edges of slots that want roots;
// mode 1: cells of slots that want cells (into pc); mode 2: edges of slots
// that want cells.
__global__ void k_b_plan_edges(const MfSlot *slots, MfBatchPlan *P, int n, int mode,
                               const int32_t *only, int dim) {
  __shared__ unsigned long long total;
  const int t = threadIdx.x;
  unsigned long long c = 0;
  if (t < n && (!only || only[t]) && slots[t].B.cnt && (dim <= 0 || slots[t].F.d == dim)) {
    const MfTraceBufs &B = slots[t].B;
    const uint32_t want = mode == 0 ? MF_WANT_ROOTS : MF_WANT_CELLS;
    if (slots[t].flags & want) {
      if (mode == 1) c = B.cnt->n_cells < B.max_cells ? B.cnt->n_cells : B.max_cells;
      else c = B.cnt->n_edges < B.max_edges ? B.cnt->n_edges : B.max_edges;
    }
  }
  const unsigned long long ex = block_scan_u64(c, &total);
  unsigned long long *p = mode == 1 ? P->pc : P->pe;
  if (t < n) p[t] = ex;
  if (t == 0) p[n] = total;
}

__global__ void __launch_bounds__(CELL_WARPS * 32) k_b_cells_enum(const MfSlot *slots,
                                                                  const MfBatchPlan *P, int n) {
  __shared__ CellLink sl[CELL_WARPS];
  const unsigned long long total = P->pe[n];
  const int lane = threadIdx.x & 31;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long item = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
       item < total; item += nwarps) {
    const int t = mf_slot_of(P->pe, n, item);
    cells_enum_edge(slots[t].F, slots[t].B, item - P->pe[t], lane, sl[threadIdx.x >> 5]);
  }
}

template <bool FILL>
__global__ void k_b_cell_edges(const MfSlot *slots, const MfBatchPlan *P, int n) {
  const unsigned long long total = P->pc[n];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long item = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
       item < total; item += stride) {
    const int t = mf_slot_of(P->pc, n, item);
    cell_edges_item<FILL>(slots[t].F, slots[t].B, item - P->pc[t], slots[t].B.cell_off);
  }
}

// Host launchers of the batched kernels (used by the batch driver).
void mf_b_launch_init(const MfSlot *slots, MfSlotState *st, int n, cudaStream_t s) {
  k_b_init<<<(n + 255) / 256, 256, 0, s>>>(slots, st, n);
}
void mf_b_launch_expand(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n, bool edges,
                        int sms, cudaStream_t s) {
  if (!edges) {
    k_b_plan_expand<<<1, MF_MAX_SLOTS, 0, s>>>(slots, st, P, n);
    k_b_expand<false><<<sms * 8, EXPAND_WARPS * 32, 0, s>>>(slots, st, P, n);
  } else {
    k_b_expand<true><<<sms * 8, EXPAND_WARPS * 32, 0, s>>>(slots, st, P, n);
  }
}
void mf_b_launch_plan_eval(const MfSlot *slots, MfBatchPlan *P, int n, bool recheck, cudaStream_t s) {
  if (recheck) k_b_plan_recheck<<<1, MF_MAX_SLOTS, 0, s>>>(slots, P, n);
  else k_b_plan_eval<<<1, MF_MAX_SLOTS, 0, s>>>(slots, P, n);
}
void mf_b_launch_advance(const MfSlot *slots, int n, cudaStream_t s) {
  k_b_advance<<<(n + 255) / 256, 256, 0, s>>>(slots, n);
}
void mf_b_launch_update(const MfSlot *slots, MfSlotState *st, MfBatchPlan *P, int n,
                        cudaGraphConditionalHandle h, int use_handle, cudaStream_t s) {
  k_b_update<<<1, MF_MAX_SLOTS, 0, s>>>(slots, st, P, n, h, use_handle);
}
void mf_b_launch_plan_edges(const MfSlot *slots, MfBatchPlan *P, int n, int cells,
                            const int32_t *only, cudaStream_t s, int dim) {
  k_b_plan_edges<<<1, MF_MAX_SLOTS, 0, s>>>(slots, P, n, cells, only, dim);
}
void mf_b_launch_cells(const MfSlot *slots, MfBatchPlan *P, int n, const int32_t *only, int sms,
                       cudaStream_t s) {
  k_b_plan_edges<<<1, MF_MAX_SLOTS, 0, s>>>(slots, P, n, 2, only, 0);
  k_b_cells_enum<<<sms * 8, 256, 0, s>>>(slots, P, n);
}
void mf_b_launch_cell_edges(const MfSlot *slots, MfBatchPlan *P, int n, bool fill,
                            const int32_t *only, int sms, cudaStream_t s) {
  if (!fill) {
    // the cells' plan; their sign masks and row lengths were written by the
    // enumeration (cells_enum_edge), so no counting pass is needed
    k_b_plan_edges<<<1, MF_MAX_SLOTS, 0, s>>>(slots, P, n, 1, only, 0);
  } else {
    k_b_cell_edges<true><<<sms * 8, 256, 0, s>>>(slots, P, n);
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan of int64 counts (three passes): per-tile scans, a scan of the
// tile totals, and the tile offsets added back.  out[n] receives the total.
// ---------------------------------------------------------------------------
#define SCAN_THREADS 512
#define SCAN_PER_THREAD 8
#define SCAN_TILE (SCAN_THREADS * SCAN_PER_THREAD)

__device__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
  __shared__ int64_t warp_tot[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
    int64_t s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = s - t;
    if (lane == 31) *total = s;
  }
  __syncthreads();
  const int64_t r = x - v + warp_tot[w];
  __syncthreads();
  return r;
}

__global__ void k_scan_tiles(const int64_t *in, int64_t *out, int64_t n, int64_t *tile_tot) {
  __shared__ int64_t tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_PER_THREAD;
  int64_t v[SCAN_PER_THREAD], s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; i++) {
    v[i] = base + i < n ? in[base + i] : 0;
    s += v[i];
  }
  int64_t off = block_exclusive_scan(s, &tot);
#pragma unroll
  for (int i = 0; i < SCAN_PER_THREAD; i++) {
    if (base + i < n) out[base + i] = off;
    off += v[i];
  }
  if (threadIdx.x == 0) tile_tot[blockIdx.x] = tot;
}

__global__ void k_scan_totals(int64_t *tile_tot, int64_t ntiles, int64_t *grand) {
  __shared__ int64_t tot;
  int64_t carry = 0;
  for (int64_t b = 0; b < ntiles; b += SCAN_THREADS) {
    const int64_t i = b + threadIdx.x;
    const int64_t v = i < ntiles ? tile_tot[i] : 0;
    const int64_t ex = block_exclusive_scan(v, &tot);
    if (i < ntiles) tile_tot[i] = ex + carry;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *tile_tot) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_tot[i / SCAN_TILE];
}

// in and out may alias.  scratch: ceil(n / SCAN_TILE) + 1 int64.
static void exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch,
                           cudaStream_t st) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (ntiles == 0) {
    cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    return;
  }
  k_scan_tiles<<<(unsigned)ntiles, SCAN_THREADS, 0, st>>>(in, out, n, scratch);
  k_scan_totals<<<1, SCAN_THREADS, 0, st>>>(scratch, ntiles, out + n);
  k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, scratch);
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
static uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Builds the frame: lattice constants, the box, the bounding box of its
// lattice coordinates (the box under L^-1, margin 3; the domain table searches
// it) and the key packing.  Fails if keys do not fit 64 bits.
static int build_frame(mf_ctx *ctx, int d, double lam, const mf_domain *dom, MfFrame *F) {
  mf_frame_lattice(F, d, lam, dom->offset);
  double slo = 0.0, shi = 0.0;
  for (int j = 0; j < d; j++) {
    if (!(dom->lo[j] <= dom->hi[j]) || !std::isfinite(dom->lo[j]) || !std::isfinite(dom->hi[j]) ||
        !std::isfinite(dom->offset[j]))
      return mf_set_error(ctx, MF_ERR_INVALID, "bad domain on axis %d", j);
    F->lo[j] = dom->lo[j];
    F->hi[j] = dom->hi[j];
    slo += dom->lo[j] - dom->offset[j];
    shi += dom->hi[j] - dom->offset[j];
  }
  for (int i = 0; i < d; i++) {
    const double a = ((dom->lo[i] - dom->offset[i]) + F->cinv * slo) / lam;
    const double b = ((dom->hi[i] - dom->offset[i]) + F->cinv * shi) / lam;
    if (!(std::fabs(a) < 1e9 && std::fabs(b) < 1e9))
      return mf_set_error(ctx, MF_ERR_DOMAIN, "lattice range too large on axis %d", i);
    const long long ymin = (long long)std::floor(a) - 3, ymax = (long long)std::ceil(b) + 3;
    F->ymin[i] = (int32_t)ymin;
    F->range[i] = (int32_t)(ymax - ymin + 1);
  }
  if (!mf_frame_pack_keys(F))
    return mf_set_error(ctx, MF_ERR_DOMAIN,
                        "edge keys need more than 64 bits (domain too large for lambda)");
  return MF_OK;
}

// The exact domain table of the frame (see MfFrame::dom_tab): x_i(y, s) =
// lam * ((double)y_i - c * s) + o_i rises with y_i, so the in-box y_i form one
// interval per (s, i), found by binary search with the device's operation
// order (this translation unit's host code is compiled without contraction).
// Fills `tab` and sets F->smin / F->sspan; false if the table would be too
// large (the kernels then test the domain in FP64).
bool mf_domain_table_host(MfFrame *F, std::vector<int2> &tab) {
  const int d = F->d;
  long long smin = 0, smax = 0;
  for (int i = 0; i < d; i++) {
    smin += F->ymin[i];
    smax += (long long)F->ymin[i] + F->range[i] - 1;
  }
  const long long span = smax - smin + 1;
  F->dom_tab = nullptr;
  if (span <= 0 || span > (1ll << 22)) return false;
  tab.assign((size_t)span * d, int2());
  for (long long s = smin; s <= smax; s++) {
    const double cs = F->c * (double)s;
    for (int i = 0; i < d; i++) {
      auto xof = [&](long long y) {
        const volatile double u = (double)y - cs;
        const volatile double w = F->lam * u;
        return w + F->o[i];
      };
      const long long y0 = F->ymin[i], y1 = (long long)F->ymin[i] + F->range[i] - 1;
      // midpoints from a + (b - a) / 2 with b > a: never truncated onto an end,
      // so each search halves a non-empty interval (coordinates may be negative)
      long long a = y0, b = y1 + 1;  // first y with x >= lo
      while (a < b) {
        const long long m = a + (b - a) / 2;
        if (xof(m) >= F->lo[i]) b = m; else a = m + 1;
      }
      const long long first = a;
      a = y0 - 1;
      b = y1;  // last y with x <= hi
      while (a < b) {
        const long long m = a + (b - a + 1) / 2;
        if (xof(m) <= F->hi[i]) a = m; else b = m - 1;
      }
      const long long last = a;
      int2 v;
      if (first <= last) { v.x = (int)first; v.y = (int)last; }
      else { v.x = 1 << 30; v.y = -(1 << 30); }
      tab[(size_t)(s - smin) * d + i] = v;
    }
  }
  F->smin = (int32_t)smin;
  F->sspan = (int32_t)span;
  return true;
}

static int build_domain_table(mf_ctx *ctx, MfFrame *F, cudaStream_t st) {
  std::vector<int2> tab;
  if (!mf_domain_table_host(F, tab)) return MF_OK;  // FP64 test instead
  int2 *dev = (int2 *)mf_ctx_buffer(ctx, MF_SLOT_DOMTAB, tab.size() * sizeof(int2));
  if (!dev) return MF_ERR_OOM;
  int rc = mf_cuda_check(ctx, cudaMemcpyAsync(dev, tab.data(), tab.size() * sizeof(int2),
                                              cudaMemcpyHostToDevice, st),
                         "domain table");
  if (rc) return rc;
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "domain table");
  if (rc) return rc;
  F->dom_tab = dev;
  return MF_OK;
}

extern "C" int mf_domain_table(int32_t d, double lambda, const mf_domain *dom, int32_t *smin,
                               int32_t *span, int32_t *tab, int64_t cap) {
  if (d < 2 || d > MF_MAXD || !(lambda > 0.0) || !dom || !smin || !span) return MF_ERR_INVALID;
  MfFrame F;
  const int rc = build_frame(nullptr, d, lambda, dom, &F);
  if (rc) return rc;
  std::vector<int2> t;
  if (!mf_domain_table_host(&F, t)) return MF_ERR_DOMAIN;
  *smin = F.smin;
  *span = F.sspan;
  if (!tab) return MF_OK;
  if (cap < (int64_t)t.size() * 2) return MF_ERR_CAPACITY;
  for (size_t i = 0; i < t.size(); i++) {
    tab[2 * i] = t[i].x;
    tab[2 * i + 1] = t[i].y;
  }
  return MF_OK;
}

// Entry points for the batch driver (mf_batch.cu).
int mf_build_frame(mf_ctx *ctx, int d, double lam, const mf_domain *dom, MfFrame *F) {
  return build_frame(ctx, d, lam, dom, F);
}
void mf_exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch,
                       cudaStream_t st) {
  exclusive_scan(in, out, n, scratch, st);
}
uint64_t mf_next_pow2(uint64_t x) { return next_pow2(x); }
int mf_setup_buffers(mf_ctx *ctx, int d, uint64_t ME, uint64_t MV, uint64_t MC, bool mixed, int n_sv,
                     MfTraceBufs *B);
int mf_build_domain_table(mf_ctx *ctx, MfFrame *F, cudaStream_t st);
int mf_read_counters(mf_ctx *ctx, const MfTraceBufs &B, cudaStream_t st);
void mf_launch_cells_fill(const MfFrame &F, const MfTraceBufs &B, uint64_t n_cells, cudaStream_t st) {
  if (n_cells == 0) return;
  k_cells_edges<true><<<(unsigned)((n_cells + 255) / 256), 256, 0, st>>>(F, B, n_cells, B.cell_off);
}
void mf_launch_cells_enum(const MfFrame &F, const MfTraceBufs &B, uint64_t n_edges, cudaStream_t st) {
  if (n_edges == 0) return;
  k_cells_enum<<<(unsigned)((n_edges * 32 + 255) / 256), 256, 0, st>>>(F, B, n_edges);
}
void mf_launch_seeds(const MfFrame &F, const MfTraceBufs &B, const double *seeds, int64_t n,
                     bool vertices, cudaStream_t s) {
  const unsigned g = (unsigned)((n + 127) / 128);
  if (vertices) k_seed_vertices<<<g, 128, 0, s>>>(F, B, seeds, n);
  else k_seed_edges<<<g, 128, 0, s>>>(F, B, seeds, n);
}

static int read_counters(mf_ctx *ctx, const MfTraceBufs &B, cudaStream_t st) {
  int rc = mf_cuda_check(ctx, cudaMemcpyAsync(ctx->h_counters, B.cnt, sizeof(MfCounters),
                                              cudaMemcpyDeviceToHost, st),
                         "read counters");
  if (rc) return rc;
  rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "trace kernels");
  if (rc) return rc;
  const MfCounters &h = *ctx->h_counters;
  if (h.err_table_full)
    return mf_set_error(ctx, MF_ERR_DEVICE, "a resident hash table is full");
  if (h.err_missing & 4u)
    return mf_set_error(ctx, MF_ERR_DEVICE, "an enumerated cell failed its canonical-pair check");
  if (h.err_missing)
    return mf_set_error(ctx, MF_ERR_DEVICE, "vertex missing from the vertex table");
  if (h.err_timeout)
    return mf_set_error(ctx, MF_ERR_TIMEOUT, "a tensor-core wait gave up");
  if (h.err_overflow || h.n_edges > B.max_edges || h.n_vertices > B.max_vertices ||
      h.n_cells > B.max_cells)
    return mf_set_error(ctx, MF_ERR_MAXEDGES,
                        "traced set exceeds capacity (edges %llu/%llu, vertices %llu/%llu, "
                        "cells %llu/%llu)",
                        h.n_edges, (unsigned long long)B.max_edges, h.n_vertices,
                        (unsigned long long)B.max_vertices, h.n_cells,
                        (unsigned long long)B.max_cells);
  return MF_OK;
}

// Carves the trace's buffers from the context slots.
static int setup_buffers(mf_ctx *ctx, int d, uint64_t ME, uint64_t MV, uint64_t MC, bool mixed,
                         int n_sv, MfTraceBufs *B) {
  memset(B, 0, sizeof(*B));
  // load factor <= 3/4 at capacity
  const uint64_t TE = next_pow2(ME + ME / 3 + 1), TV = next_pow2(MV + MV / 3 + 1);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t tb = al(TE * 16) + al(TV * 16);
  char *t = (char *)mf_ctx_buffer(ctx, MF_SLOT_TABLES, tb);
  if (!t) return MF_ERR_OOM;
  B->etab_key = (unsigned long long *)t; t += al(TE * 16);
  B->vtab_key = (unsigned long long *)t; t += al(TV * 16);
  B->etab_mask = TE - 1;
  B->vtab_mask = TV - 1;
  size_t eb = al(ME * d * 4) + al(ME * 4) + al(ME * 16) + al(ME * 8) + al(ME * d * 8);
  char *e = (char *)mf_ctx_buffer(ctx, MF_SLOT_EDGES, eb);
  if (!e) return MF_ERR_OOM;
  B->edge_y = (int32_t *)e; e += al(ME * d * 4);
  B->edge_mask = (uint32_t *)e; e += al(ME * 4);
  B->edge_f = (double *)e; e += al(ME * 16);
  B->edge_t = (double *)e; e += al(ME * 8);
  B->edge_pt = (double *)e;
  B->max_edges = ME;
  size_t vb = al(MV * d * 4) + al(MV * 4) + (mixed ? al(MV * 4) : 0);
  char *v = (char *)mf_ctx_buffer(ctx, MF_SLOT_VERTS, vb);
  if (!v) return MF_ERR_OOM;
  B->vert_y = (int32_t *)v; v += al(MV * d * 4);
  B->vert_slot = (uint32_t *)v; v += al(MV * 4);
  B->recheck = mixed ? (uint32_t *)v : nullptr;
  B->max_vertices = MV;
  size_t cb = al(MC * d * 4) + al(MC * d) + al(MC * 4) + al((MC + 1) * 8);
  char *c = (char *)mf_ctx_buffer(ctx, MF_SLOT_CELLS, cb);
  if (!c) return MF_ERR_OOM;
  B->cell_y = (int32_t *)c; c += al(MC * d * 4);
  B->cell_perm = (uint8_t *)c; c += al(MC * d);
  B->cell_sgn = (uint32_t *)c; c += al(MC * 4);
  B->cell_off = (int64_t *)c;
  B->max_cells = MC;
  B->cnt = (MfCounters *)mf_ctx_buffer(ctx, MF_SLOT_COUNTERS, sizeof(MfCounters));
  if (!B->cnt) return MF_ERR_OOM;
  // deferred FP64 root steps: chunks of up to 4M edges, ~48 strong entries
  // each on average (when the budget allows; else every step runs in the
  // warp-per-edge kernel)
  {
    const uint64_t dc = std::min<uint64_t>(ME, 1ull << 22), dl = dc * 48;
    const size_t db = al(dc * 32) + al(dc * 8) + al(dl * 4) + al(dc * MF_EP_ROW(d) * 4) +
                      al(dc * 2 * d * 8) + al(dc * 3 * d * 4) + al(dl) + al(dl / 2) + al(dl / 2);
    std::string keep = ctx->err;
    char *q = (char *)mf_ctx_buffer(ctx, MF_SLOT_DEFER, db);
    if (q) {
      B->defer_rec = q; q += al(dc * 32);
      B->redo = (uint64_t *)q; q += al(dc * 8);
      B->defer_list = (int32_t *)q; q += al(dl * 4);
      B->ep32 = (float *)q; q += al(dc * MF_EP_ROW(d) * 4);
      B->defer_x = (double *)q; q += al(dc * 2 * d * 8);
      B->defer_x3 = (float *)q; q += al(dc * 3 * d * 4);
      B->defer_part = (double *)q; q += al(dl);  // dl / 8 doubles
      B->defer_bnd = (float *)q; q += al(dl / 2);  // dl / 8 floats
      B->defer_chunk = (uint32_t *)q;              // dl / 8 uint32
      B->defer_cap = dc;
      B->defer_list_cap = dl;
    } else {
      ctx->err = keep;
    }
  }
  // per-vertex lists for the root screen, when they fit the budget (else
  // the root screen scans the vector blocks)
  if (n_sv > 0) {
    const uint64_t per = (uint64_t)std::min(n_sv, 192);
    const uint64_t cap = MV * per;
    const size_t lb = al(TV * 4) + al(MV * 8) + al(MV * 4) + al(cap * 4);
    std::string keep = ctx->err;
    char *l = (char *)mf_ctx_buffer(ctx, MF_SLOT_VLIST, lb);
    if (l) {
      B->vtab_idx = (uint32_t *)l; l += al(TV * 4);
      B->vlist_off = (uint64_t *)l; l += al(MV * 8);
      B->vlist_n = (uint32_t *)l; l += al(MV * 4);
      B->vlist = (int32_t *)l;
      B->vlist_cap = cap;
    } else {
      ctx->err = keep;
    }
  }
  return MF_OK;
}

static int copy_out(mf_ctx *ctx, const MfTraceState &L, mf_trace_out *out, cudaStream_t st) {
  const int d = L.F.d;
  out->n_edges = L.n_edges;
  out->n_cells = L.n_cells;
  out->n_cell_edges = L.n_cell_edges;
  out->n_vertices = L.n_vertices;
  out->n_near_zero = L.n_near_zero;
  out->n_recheck = L.n_recheck;
  out->n_boundary = L.n_boundary;
  out->n_dead_seeds = L.n_dead_seeds;
  out->levels = L.levels;
  out->root_evals = L.root_evals;
  const MfTraceBufs &B = L.B;
  bool small = false;
  const size_t E = (size_t)L.n_edges;
  if (L.sorted) {
    // the sorted order: gathers instead of copies
    small = ((out->edge_y || out->edge_mask || out->edge_f || out->edge_t || out->points) &&
             out->cap_edges < L.n_edges) ||
            ((L.flags & MF_WANT_CELLS) && (out->cell_y || out->cell_perm || out->cell_edge_off) &&
             out->cap_cells < L.n_cells) ||
            ((L.flags & MF_WANT_CELLS) && out->cell_edge_idx && out->cap_cell_edges < L.n_cell_edges);
    if (small)
      return mf_set_error(ctx, MF_ERR_CAPACITY,
                          "output buffers too small: need %lld edges, %lld cells, %lld cell edges",
                          (long long)L.n_edges, (long long)L.n_cells, (long long)L.n_cell_edges);
    int rc = mf_copy_out_sorted(ctx, L, out, st);
    if (rc) return rc;
    return mf_cuda_check(ctx, cudaStreamSynchronize(st), "copy out");
  }
  auto cp = [&](void *dst, const void *src, size_t bytes) {
    if (dst && bytes) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
  };
  if (out->edge_y || out->edge_mask || out->edge_f || out->edge_t || out->points) {
    if (out->cap_edges < L.n_edges) small = true;
    else {
      cp(out->edge_y, B.edge_y, E * d * 4);
      cp(out->edge_mask, B.edge_mask, E * 4);
      cp(out->edge_f, B.edge_f, E * 16);
      if (L.flags & MF_WANT_ROOTS) {
        cp(out->edge_t, B.edge_t, E * 8);
        cp(out->points, B.edge_pt, E * d * 8);
      }
    }
  }
  if ((L.flags & MF_WANT_CELLS) && (out->cell_y || out->cell_perm || out->cell_edge_off)) {
    if (out->cap_cells < L.n_cells) small = true;
    else {
      const size_t C = (size_t)L.n_cells;
      cp(out->cell_y, B.cell_y, C * d * 4);
      cp(out->cell_perm, B.cell_perm, C * d);
      cp(out->cell_edge_off, B.cell_off, (C + 1) * 8);
    }
  }
  if ((L.flags & MF_WANT_CELLS) && out->cell_edge_idx) {
    if (out->cap_cell_edges < L.n_cell_edges) small = true;
    else cp(out->cell_edge_idx, B.cell_idx, (size_t)L.n_cell_edges * 8);
  }
  int rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "copy out");
  if (rc) return rc;
  if (small)
    return mf_set_error(ctx, MF_ERR_CAPACITY,
                        "output buffers too small: need %lld edges, %lld cells, %lld cell edges",
                        (long long)L.n_edges, (long long)L.n_cells, (long long)L.n_cell_edges);
  return MF_OK;
}

extern "C" int mf_trace(mf_ctx *ctx, const mf_rbf *rbf, const mf_domain *dom,
                        const mf_trace_opts *opts, const double *seeds, int64_t n_seeds,
                        mf_trace_out *out, void *stream) {
  if (!ctx) return MF_ERR_INVALID;
  ctx->last.valid = false;
  ctx->sub.valid = false;  // its slots are reused here
  if (!rbf || !dom || !opts || !out || n_seeds < 0 || (n_seeds > 0 && !seeds))
    return mf_set_error(ctx, MF_ERR_INVALID, "mf_trace: NULL argument");
  if (!(opts->lambda > 0.0) || !std::isfinite(opts->lambda))
    return mf_set_error(ctx, MF_ERR_INVALID, "lambda must be > 0");
  if (opts->precision != MF_FP64 && opts->precision != MF_MIXED_FP32 &&
      opts->precision != MF_MIXED_BF16)
    return mf_set_error(ctx, MF_ERR_INVALID, "unknown precision %d", opts->precision);
  cudaSetDevice(ctx->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int d = rbf->d;
  MfRbfDev R;
  int rc;
  {
    MfProfScope ps(ctx, MF_PH_PREPARE, st, 1, rbf ? rbf->n_sv : 0);
    rc = mf_prepare_rbf(ctx, rbf, &R, st);
  }
  if (rc) return rc;
  MfFrame F;
  rc = build_frame(ctx, d, opts->lambda, dom, &F);
  if (rc) return rc;
  rc = build_domain_table(ctx, &F, st);
  if (rc) return rc;
  const uint64_t ME = opts->max_edges > 0 ? (uint64_t)opts->max_edges : (1ull << 24);
  const uint64_t MV = opts->max_vertices > 0 ? (uint64_t)opts->max_vertices : ME;
  const uint64_t MC = opts->max_cells > 0 ? (uint64_t)opts->max_cells : 2 * ME;
  if (ME >= (1ull << 32) || MV >= (1ull << 32))
    return mf_set_error(ctx, MF_ERR_INVALID, "max_edges / max_vertices must be < 2^32");
  const bool mixed = opts->precision != MF_FP64;
  MfTraceBufs B;
  rc = setup_buffers(ctx, d, ME, MV, MC, mixed, (int)rbf->n_sv, &B);
  if (rc) return rc;
  // the root screen's lists: the mixed paths' radius when their roots are fast
  if (B.vlist)
    B.list_r2 = mf_list_r2(F, R, mixed && !(opts->flags & MF_ROOTS_FP64_EXACT));
  uint64_t cap = opts->batch_cap_edges > 0 ? (uint64_t)opts->batch_cap_edges : (1ull << 24);
  if (ctx->tune.frontier_chunk > 0 && ctx->tune.frontier_chunk < cap) cap = ctx->tune.frontier_chunk;
  // the expand items' vertex slots of the whole search: up to (2^d - 2)
  // items per edge (at most 2^31, halved while the budget refuses), the
  // first item of each edge and the bases of one chunk's warps
  {
    const uint64_t ce = std::min<uint64_t>(cap, ME);
    const uint64_t nw = (ce + 255) / 256 * EXPAND_WARPS + EXPAND_WARPS;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    std::string keep = ctx->err;
    for (uint64_t ic = std::min<uint64_t>(ME * ((1ull << d) - 2), 1ull << 31); ic >= (1ull << 20);
         ic >>= 1) {
      char *q = (char *)mf_ctx_buffer(ctx, MF_SLOT_ITEMS, al(ic * 4) + al(nw * 8) + al(ME * 8));
      if (q) {
        B.item_slot = (uint32_t *)q;
        B.warp_base = (unsigned long long *)(q + al(ic * 4));
        B.edge_item_off = (unsigned long long *)(q + al(ic * 4) + al(nw * 8));
        B.item_cap = ic;
        break;
      }
    }
    ctx->err = keep;
  }
  const double band = opts->recheck_band > 0 ? opts->recheck_band : 1e-3;
  const double tol = opts->root_tol > 0 ? opts->root_tol : 1e-12;
  const int sms = ctx->sms;

  cudaMemsetAsync(B.cnt, 0, sizeof(MfCounters), st);
  cudaMemsetAsync(B.etab_key, 0xFF, (B.etab_mask + 1) * 16, st);
  cudaMemsetAsync(B.vtab_key, 0xFF, (B.vtab_mask + 1) * 16, st);

  auto eval = [&]() {
    if (mixed) mf_launch_eval_vertices_mixed(F, R, B, opts->precision, band, ctx->tune, sms, st);
    else mf_launch_eval_vertices_f64(F, R, B, ctx->tune, sms, st);
  };

  // Locate edges (Fig. 3)
  if (n_seeds > 0) {
    const unsigned g = (unsigned)((n_seeds + 127) / 128);
    MfProfScope ps(ctx, MF_PH_SEEDS, st, mixed ? (B.vlist ? 6 : 5) : 4, n_seeds);
    k_seed_vertices<<<g, 128, 0, st>>>(F, B, seeds, n_seeds);
    eval();
    k_seed_edges<<<g, 128, 0, st>>>(F, B, seeds, n_seeds);
  }
  rc = mf_cuda_check(ctx, cudaGetLastError(), "seed kernels");
  if (rc) return rc;
  rc = read_counters(ctx, B, st);
  if (rc) return rc;

  // Search edges (Fig. 4): one level per pass, each in chunks of <= cap edges.
  uint64_t fs = 0, fe = ctx->h_counters->n_edges;
  int64_t levels = fe > 0 ? 1 : 0;
  while (fe > fs) {
    for (uint64_t a = fs; a < fe; a += cap) {
      const uint64_t n = std::min(cap, fe - a);
      const unsigned g = (unsigned)((n + EXPAND_WARPS * 32 - 1) / (EXPAND_WARPS * 32));
      {
        MfProfScope ps(ctx, MF_PH_EXPAND_V, st, 1, (int64_t)n);
        k_expand_vertices<<<g, EXPAND_WARPS * 32, 0, st>>>(F, B, a, n);
      }
      {
        MfProfScope ps(ctx, MF_PH_EVAL, st, mixed ? (B.vlist ? 4 : 3) : 2);
        eval();
      }
      {
        MfProfScope ps(ctx, MF_PH_EXPAND_E, st, 1, (int64_t)n);
        k_expand_edges<<<g, EXPAND_WARPS * 32, 0, st>>>(F, B, a, n);
      }
    }
    rc = mf_cuda_check(ctx, cudaGetLastError(), "BFS kernels");
    if (rc) return rc;
    rc = read_counters(ctx, B, st);
    if (rc) return rc;
    fs = fe;
    fe = ctx->h_counters->n_edges;
    if (fe > fs) levels++;
  }
  const uint64_t E = fe;

  // Roots (the iterative intersection solve of Sec. VI), FP64 Newton.
  if (opts->flags & MF_WANT_ROOTS) {
    MfProfScope ps(ctx, MF_PH_ROOTS, st, E > 0 ? 1 : 0, (int64_t)E);
    mf_launch_roots_f64(F, R, B, E, tol, ctx->tune, sms, st,
                        mixed && !(opts->flags & MF_ROOTS_FP64_EXACT));
  }

  // Cells (Sec. IV-C) and the cell -> edge CSR.
  int64_t n_cells = 0, n_cell_edges = 0;
  if ((opts->flags & MF_WANT_CELLS) && E > 0) {
    {
      MfProfScope ps(ctx, MF_PH_CELLS, st, 1, (int64_t)E);
      k_cells_enum<<<(unsigned)((E * 32 + 255) / 256), 256, 0, st>>>(F, B, E);
    }
    rc = mf_cuda_check(ctx, cudaGetLastError(), "cell kernels");
    if (rc) return rc;
    rc = read_counters(ctx, B, st);
    if (rc) return rc;
    n_cells = (int64_t)ctx->h_counters->n_cells;
    const unsigned g = (unsigned)((n_cells + 255) / 256);
    int64_t *scratch = (int64_t *)mf_ctx_buffer(ctx, MF_SLOT_SCAN,
                                                ((size_t)n_cells / SCAN_TILE + 2) * 8);
    if (!scratch) return MF_ERR_OOM;
    {
      // the enumeration wrote each cell's sign mask and CSR row length
      MfProfScope ps(ctx, MF_PH_CSR, st, 3, n_cells);
      exclusive_scan(B.cell_off, B.cell_off, n_cells, scratch, st);
    }
    rc = mf_cuda_check(ctx, cudaMemcpyAsync(&n_cell_edges, B.cell_off + n_cells, 8,
                                            cudaMemcpyDeviceToHost, st),
                       "cell totals");
    if (rc) return rc;
    rc = mf_cuda_check(ctx, cudaStreamSynchronize(st), "cell scan");
    if (rc) return rc;
    B.cell_idx = (int64_t *)mf_ctx_buffer(ctx, MF_SLOT_CELLIDX, (size_t)n_cell_edges * 8 + 256);
    if (!B.cell_idx) return MF_ERR_OOM;
    {
      MfProfScope ps(ctx, MF_PH_CSR, st, 1);
      k_cells_edges<true><<<g, 256, 0, st>>>(F, B, (uint64_t)n_cells, B.cell_off);
    }
  }
  rc = mf_cuda_check(ctx, cudaGetLastError(), "CSR kernels");
  if (rc) return rc;
  rc = read_counters(ctx, B, st);
  if (rc) return rc;

  MfTraceState &L = ctx->last;
  L.F = F;
  L.B = B;
  L.R = R;
  L.precision = opts->precision;
  L.band = band;
  L.tol = tol;
  L.flags = opts->flags;
  const MfCounters &h = *ctx->h_counters;
  L.n_edges = (int64_t)E;
  L.n_cells = n_cells;
  L.n_cell_edges = n_cell_edges;
  L.n_vertices = (int64_t)h.n_vertices;
  L.n_near_zero = (int64_t)h.n_near_zero;
  L.n_recheck = (int64_t)h.n_recheck;
  L.n_boundary = (int64_t)h.n_boundary;
  L.n_dead_seeds = (int64_t)h.n_dead_seeds;
  L.levels = levels;
  L.root_evals = (int64_t)h.root_evals;
  L.sorted = false;
  if (opts->flags & MF_SORT_OUTPUT) {
    MfProfScope ps(ctx, MF_PH_COPY, st, 0);
    rc = mf_sort_trace(ctx, L, st);
    if (rc) return rc;
    L.sorted = true;
  }
  L.valid = true;
  if (ctx->prof.on) {
    ctx->prof.stats.terms[MF_PH_EVAL] += (int64_t)h.eval_terms;
    ctx->prof.stats.terms[MF_PH_ROOTS] += (int64_t)h.root_terms;
    ctx->prof.stats.terms_weak[MF_PH_EVAL] += (int64_t)h.eval_terms_weak;
    ctx->prof.stats.terms_weak[MF_PH_ROOTS] += (int64_t)h.root_terms_weak;
    // the tensor-core evaluation computes every term of every vertex
    if (opts->precision == MF_MIXED_BF16)
      ctx->prof.stats.terms_weak[MF_PH_EVAL] += (int64_t)h.n_vertices * rbf->n_sv;
  }
  {
    MfProfScope ps(ctx, MF_PH_COPY, st, 0);
    rc = copy_out(ctx, L, out, st);
  }
  mf_prof_collect(ctx);
  return rc;
}

extern "C" int mf_trace_fetch(mf_ctx *ctx, mf_trace_out *out, void *stream) {
  if (!ctx || !out) return MF_ERR_INVALID;
  if (!ctx->last.valid) return mf_set_error(ctx, MF_ERR_INVALID, "no trace result to fetch");
  cudaSetDevice(ctx->device);
  return copy_out(ctx, ctx->last, out, (cudaStream_t)stream);
}

extern "C" int mf_vertex_keys(int32_t d, double lambda, const mf_domain *dom, const int32_t *y,
                              int64_t n, uint64_t *keys, uint8_t *in_range) {
  if (d < 2 || d > MF_MAXD || !(lambda > 0.0) || !dom || n < 0 || (n > 0 && (!y || !keys)))
    return MF_ERR_INVALID;
  MfFrame F;
  const int rc = build_frame(nullptr, d, lambda, dom, &F);
  if (rc) return rc;
  for (int64_t i = 0; i < n; i++) {
    keys[i] = mf_vertex_key(F, y + i * d);
    if (in_range) in_range[i] = mf_vertex_in_packing(F, y + i * d) ? 1 : 0;
  }
  return MF_OK;
}

// Host helpers shared with the batch triangulation (mf_subdiv.cu).
int mf_setup_buffers(mf_ctx *ctx, int d, uint64_t ME, uint64_t MV, uint64_t MC, bool mixed, int n_sv,
                     MfTraceBufs *B) {
  return setup_buffers(ctx, d, ME, MV, MC, mixed, n_sv, B);
}
int mf_build_domain_table(mf_ctx *ctx, MfFrame *F, cudaStream_t st) {
  return build_domain_table(ctx, F, st);
}
int mf_read_counters(mf_ctx *ctx, const MfTraceBufs &B, cudaStream_t st) {
  return read_counters(ctx, B, st);
}
