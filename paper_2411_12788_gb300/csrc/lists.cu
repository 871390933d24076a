// Tile lists by a sort of (item, tile row) pairs and counting placement:
// every tile's list of items in the depth order of Sec. 3.1, built without
// sorting the tile entries themselves.
//
// The items come depth-sorted (the preprocess's depth sort).  An item covers
// a band of tile rows [ty0, ty1] of its view and, in each row, one
// contiguous run of tile columns [a, b] (the row-interval form of its support,
// project.cuh row_tiles).  Two levels:
//
//   level 1  one (item, row) pair per band row, written in depth order with
//            the row's [a, b] packed above the global row id in a 32-bit key
//            (row | a << 12 | b << 22); a stable radix sort over the 12 row
//            bits groups the pairs by row and keeps each row's pairs in depth
//            order (the onesweep sort of sort.cu, which writes its output in
//            runs).
//   level 2  entries, grouped by tile inside each row: chunks of
//            kListPairsPerChunk consecutive pairs of one row count their
//            entries per tile column (a difference array over [a, b]); a
//            column scan over the row's chunks and an exclusive scan over all
//            tiles give every chunk its offset in each tile's list; each chunk
//            then places its entries in shared memory, grouped by column and
//            in pair order (ranks among 32 pairs from one coverage word per
//            column), and writes every column's run out contiguously.
//
// Every placement is a prefix count in the order of the input, so a tile's
// list holds its items in depth order (ties by item index, as the depth sort
// is stable): exactly the order of a stable sort of the entries by tile id.
// Traffic: 4 B of output per entry plus about 40 B per pair, against 44 B
// per entry for emitting every entry and sorting the entries by tile id
// (about 2.7 entries per pair at the training workloads).  Consistency checks:
// the pairs written equal the preprocess's count and the entries placed equal
// the scanned tile counts; a mismatch sets kStatusEntryMismatch.
#include "project.cuh"

namespace gs {

namespace {

constexpr int kL2Warps = 4;
constexpr int kStageCap = 2048;            // entries a chunk stages in shared memory
constexpr int kRowBits = 12;               // kListRowsMax == 1 << kRowBits
constexpr uint32_t kRowMask = (1u << kRowBits) - 1u;
static_assert(kListRowsMax <= (1 << kRowBits), "row ids must fit the key's row bits");
static_assert(kListTxMax <= 1023, "tile columns must fit the key's 10-bit fields");

__device__ __forceinline__ uint32_t pair_key(int row, int a, int b) {
  return (uint32_t)row | ((uint32_t)a << kRowBits) | ((uint32_t)b << (kRowBits + 10));
}
__device__ __forceinline__ int key_a(uint32_t k) { return (int)((k >> kRowBits) & 1023u); }
__device__ __forceinline__ int key_b(uint32_t k) { return (int)(k >> (kRowBits + 10)); }
// an empty row of a band (its support misses the image): a > b
constexpr uint32_t kEmptyAB = 1u << kRowBits;

// global tile row -> view (views are few: a linear search)
__device__ __forceinline__ int view_of_row(const ViewDev* views, int n_views, int row) {
  int v = 0;
  for (int k = 1; k < n_views; ++k)
    if (views[k].row_base <= row) v = k;
  return v;
}

// Inclusive scan over a warp (all lanes active).
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  return x;
}

// Lane owning element e of a group whose lanes hold runs [start_l, start_l +
// len_l) laid end to end in lane order: the last lane with len > 0 starting at
// or before e.  s_nz lists the lanes with len > 0 in order; e0 is the window's
// first element (every lane of the warp calls this together).  Always a lane
// of s_nz (lanes past the last element get the last run's lane).
__device__ __forceinline__ int run_owner(uint32_t start, uint32_t len, uint32_t e0, const uint8_t* s_nz) {
  const int lane = threadIdx.x & 31;
  const bool in_window = len > 0 && start >= e0 && start < e0 + 32;
  const uint32_t M = __reduce_or_sync(0xffffffffu, in_window ? 1u << (start - e0) : 0u);
  const uint32_t before = __popc(__ballot_sync(0xffffffffu, len > 0 && start < e0));
  const uint32_t idx = before + __popc(M & ((2u << lane) - 1u));
  return idx > 0 ? s_nz[idx - 1] : 0;
}

// ---- level 1: pairs in depth order -----------------------------------------
// A warp takes 32 consecutive positions of the depth order.  Their pairs are
// one contiguous run of the pair array (the preprocess scanned the band
// sizes), so the warp enumerates (item, row) pairs 32 at a time: each lane
// finds its pair's item (run_owner), evaluates that row's columns with
// row_tiles (the same arithmetic the preprocess counted with) and writes the
// pair at the run's start + its index: consecutive lanes, consecutive slots.
struct PairItem {
  BinParams b;
  uint32_t item;
  int ty0, row_base, tiles_x;
};
constexpr int kPairWarps = 8;

__global__ void __launch_bounds__(32 * kPairWarps) pairs_kernel(ListArgs A) {
  __shared__ PairItem s_it[kPairWarps][32];
  __shared__ uint8_t s_nz[kPairWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t k0 = ((int64_t)blockIdx.x * kPairWarps + warp) * 32;
  if (k0 >= A.n_items) return;                               // warp-uniform
  const int64_t k = k0 + lane;
  uint32_t nrows = 0;
  {
    PairItem d;
    d.item = 0;
    d.ty0 = d.row_base = d.tiles_x = 0;
    if (k < A.n_items) {
      uint32_t item = A.sorted_items[k];
      if (!GS_IN_RANGE(item, A.n_items, A.status)) item = 0;
      nrows = A.st.band_rows[item];
      if (nrows) {
        const ViewDev& V = A.views[item / A.n];
        const float4 a = A.st.xy_tau_z[item];
        const float4 b0 = A.st.bin[2 * item], b1 = A.st.bin[2 * item + 1];
        d.b.mx = a.x;
        d.b.my = a.y;
        d.b.tau = a.z;
        d.b.k = b0.x;
        d.b.sc = b0.y;
        d.b.isyy = b0.z;
        d.b.h = b0.w;
        d.b.rx = b1.x;
        d.b.ys = b1.y;
        d.item = item;
        d.ty0 = (int)(A.st.rect[item].x >> 16);
        d.row_base = V.row_base;
        d.tiles_x = V.tiles_x;
      }
    }
    s_it[warp][lane] = d;
  }
  const uint32_t nzmask = __ballot_sync(0xffffffffu, nrows > 0);
  if (!nzmask) return;                                       // warp-uniform
  if (nrows > 0) s_nz[warp][__popc(nzmask & ((1u << lane) - 1u))] = (uint8_t)lane;
  const uint32_t rs = warp_incl_scan(nrows);
  const uint32_t R = __shfl_sync(0xffffffffu, rs, 31);
  const uint32_t rstart = rs - nrows;
  const uint32_t base = A.pair_offsets[k0];                  // the warp's first pair
  __syncwarp();
  for (uint32_t u0 = 0; u0 < R; u0 += 32) {
    const int j = run_owner(rstart, nrows, u0, s_nz[warp]);
    const uint32_t u = u0 + lane;
    const uint32_t r = u - __shfl_sync(0xffffffffu, rstart, j);
    if (u < R) {
      const PairItem& d = s_it[warp][j];
      const int ty = d.ty0 + (int)r;
      int ta, tb;
      const uint32_t key = row_tiles(d.b, ty, d.tiles_x, &ta, &tb) ? pair_key(d.row_base + ty, ta, tb)
                                                                   : ((uint32_t)(d.row_base + ty) | kEmptyAB);
      const uint64_t pos = (uint64_t)base + u;
      if (pos < (uint64_t)A.n_pairs) {
        A.pkey[pos] = key;
        A.pval[pos] = d.item;
      } else {
        atomicOr(A.status, kStatusEntryMismatch);            // more pairs than the scan counted
      }
    }
  }
}

// [start, end) of every global row in the row-sorted pairs (binary search
// on the row bits of the keys, like the tile ranges of the radix path); the
// end goes to row_T and is made a length by rows_kernel.
__global__ void row_ranges_kernel(ListArgs A) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r > A.rows) return;
  int64_t lo = 0, hi = A.n_pairs;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((A.pkey[mid] & kRowMask) < (uint32_t)r) lo = mid + 1;
    else hi = mid;
  }
  if (r < A.rows) A.row_start[r] = (uint32_t)lo;
  if (r > 0) A.row_T[r - 1] = (uint32_t)lo;
}

// One block: row lengths, the second-level chunk table and counter offsets.
__global__ void __launch_bounds__(1024) rows_kernel(ListArgs A) {
  __shared__ uint32_t s_w[2][32];
  __shared__ unsigned long long s_carry[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 2) s_carry[threadIdx.x] = 0ull;
  __syncthreads();
  for (int base = 0; base < A.rows; base += 1024) {
    const int r = base + threadIdx.x;
    uint32_t nch = 0, ncnt = 0;
    if (r < A.rows) {
      const uint32_t t = A.row_T[r] - A.row_start[r];
      A.row_T[r] = t;
      nch = (t + kListPairsPerChunk - 1) / kListPairsPerChunk;
      ncnt = nch * (uint32_t)A.views[view_of_row(A.views, A.n_views, r)].tiles_x;
    }
    const uint32_t in[2] = {nch, ncnt};
    uint32_t x[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      x[q] = warp_incl_scan(in[q]);
      if (lane == 31) s_w[q][warp] = x[q];
    }
    __syncthreads();
    unsigned long long ex[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      unsigned long long add = s_carry[q];
      for (int w = 0; w < warp; ++w) add += s_w[q][w];
      ex[q] = add + x[q] - in[q];
    }
    if (r < A.rows) {
      A.c2_start[r] = (uint32_t)ex[0];
      A.cnt2_off[r] = (uint32_t)ex[1];
    }
    __syncthreads();
    if (threadIdx.x == 1023) {
#pragma unroll
      for (int q = 0; q < 2; ++q) s_carry[q] = ex[q] + in[q];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    A.c2_start[A.rows] = (uint32_t)s_carry[0];
    A.cnt2_off[A.rows] = (uint32_t)s_carry[1];
  }
}

// ---- level 2 ---------------------------------------------------------------
struct Chunk2 {
  int row, tx_n, tb;            // row, tiles across its view, global id of the row's first tile
  uint32_t j, p0, p1;           // chunk index in the row, its pairs [p0, p1)
  uint32_t cnt;                 // offset of its counters
};

// The second-level chunk c: its row by binary search in the chunk table.
__device__ __forceinline__ bool chunk2(const ListArgs& A, uint32_t c, Chunk2* k) {
  if (c >= A.c2_start[A.rows]) return false;
  int lo = 0, hi = A.rows - 1;                  // last row with c2_start <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.c2_start[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  k->row = lo;
  const ViewDev& V = A.views[view_of_row(A.views, A.n_views, lo)];
  k->tx_n = V.tiles_x;
  k->tb = V.tile_base + (lo - V.row_base) * V.tiles_x;
  k->j = c - A.c2_start[lo];
  const uint32_t rs = A.row_start[lo], re = A.row_start[lo] + A.row_T[lo];
  k->p0 = rs + k->j * (uint32_t)kListPairsPerChunk;
  k->p1 = min(k->p0 + (uint32_t)kListPairsPerChunk, re);
  k->cnt = A.cnt2_off[lo] + k->j * (uint32_t)k->tx_n;
  // pairs and counters stay inside their arrays even if the counts disagree
  // with the preprocess's (the disagreement itself is flagged by the totals)
  if (k->p1 > (uint32_t)A.n_pairs || (int64_t)k->cnt + k->tx_n > A.counts2_n) return false;
  return true;
}

// Entries per tile column of every second-level chunk (warp per chunk).
__global__ void __launch_bounds__(32 * kL2Warps) l2_count_kernel(ListArgs A) {
  extern __shared__ int s_dyn2[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* s_c = s_dyn2 + warp * (A.max_tx + 1);
  Chunk2 k;
  if (!chunk2(A, blockIdx.x * kL2Warps + warp, &k)) return;   // warp-uniform
  for (int t = lane; t <= k.tx_n; t += 32) s_c[t] = 0;
  __syncwarp();
  for (uint32_t p = k.p0 + lane; p < k.p1; p += 32) {
    const uint32_t key = A.pkey[p];
    const int a = key_a(key), b = key_b(key);
    if (a <= b) {
      atomicAdd(&s_c[a], 1);
      atomicAdd(&s_c[b + 1], -1);
    }
  }
  __syncwarp();
  int carry = 0;
  for (int t0 = 0; t0 < k.tx_n; t0 += 32) {
    const int t = t0 + lane;
    const int x = (int)warp_incl_scan(t < k.tx_n ? (uint32_t)s_c[t] : 0u) + carry;
    if (t < k.tx_n) A.counts2[k.cnt + t] = x;
    carry = __shfl_sync(0xffffffffu, x, 31);
  }
}

// Per row: exclusive scan of each column's counts over the row's chunks
// (into prefix2), and the tile totals.  One block per row.
__global__ void __launch_bounds__(128) l2_tile_kernel(ListArgs A) {
  const int r = blockIdx.x;
  const ViewDev& V = A.views[view_of_row(A.views, A.n_views, r)];
  const int tx_n = V.tiles_x;
  const uint32_t nch = A.c2_start[r + 1] - A.c2_start[r];
  const int tb = V.tile_base + (r - V.row_base) * tx_n;
  const int64_t off = A.cnt2_off[r];
  for (int t = threadIdx.x; t < tx_n; t += blockDim.x) {
    uint32_t run = 0;
    uint32_t j = 0;
    for (; j + 4 <= nch; j += 4) {               // four independent loads at a time
      const int64_t i = off + (int64_t)j * tx_n + t;
      const uint32_t c0 = (uint32_t)A.counts2[i], c1 = (uint32_t)A.counts2[i + tx_n],
                     c2 = (uint32_t)A.counts2[i + 2 * tx_n], c3 = (uint32_t)A.counts2[i + 3 * tx_n];
      A.prefix2[i] = run;
      A.prefix2[i + tx_n] = run + c0;
      A.prefix2[i + 2 * tx_n] = run + c0 + c1;
      A.prefix2[i + 3 * tx_n] = run + c0 + c1 + c2;
      run += c0 + c1 + c2 + c3;
    }
    for (; j < nch; ++j) {
      const int64_t i = off + (int64_t)j * tx_n + t;
      A.prefix2[i] = run;
      run += (uint32_t)A.counts2[i];
    }
    A.tile_count[tb + t] = run;
  }
}

// [start, end) of every tile; checks the entry total against the preprocess's.
__global__ void l2_ranges_kernel(ListArgs A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < A.total_tiles) A.ranges[t] = make_uint2(A.tile_start[t], A.tile_start[t] + A.tile_count[t]);
  if (t == 0 && *A.scan_total != (unsigned long long)A.n_entries) atomicOr(A.status, kStatusEntryMismatch);
}

// Places the entries of every second-level chunk (warp per chunk) in pair
// order and, inside a pair, in column order.  The entries of 32 consecutive
// pairs are taken 32 at a time (lane l the l-th, its pair found by
// run_owner); an entry's rank at its column is the number of lower lanes with
// the same column, read from a coverage word per column (bit l set by lane
// l); the column's lowest lane then advances the column's next slot and
// clears the word.  Entries go to shared memory, grouped by column, and are
// written out in runs of one column (consecutive addresses); a chunk with
// more than kStageCap entries writes them straight to their places instead.
__global__ void __launch_bounds__(32 * kL2Warps) l2_emit_kernel(ListArgs A) {
  extern __shared__ uint32_t s_dyn3[];
  __shared__ uint8_t s_nz[kL2Warps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = A.max_tx + 1;
  uint32_t* s_next = s_dyn3 + warp * (3 * w + kStageCap);   // next slot of each column (local or global)
  uint32_t* s_cov = s_next + w;                              // coverage words of the current group
  uint32_t* s_gd = s_cov + w;                                // global position minus local position
  uint32_t* s_stage = s_gd + w;                              // the chunk's entries, grouped by column
  Chunk2 k;
  if (!chunk2(A, blockIdx.x * kL2Warps + warp, &k)) return;   // warp-uniform
  uint32_t carry = 0;
  for (int t0 = 0; t0 < k.tx_n; t0 += 32) {
    const int t = t0 + lane;
    const uint32_t own = t < k.tx_n ? (uint32_t)A.counts2[k.cnt + t] : 0u;
    const uint32_t incl = warp_incl_scan(own) + carry;
    if (t < k.tx_n) {
      const uint32_t start = incl - own;
      s_next[t] = start;
      s_cov[t] = 0u;
      s_gd[t] = A.tile_start[k.tb + t] + A.prefix2[k.cnt + t] - start;
    }
    carry = __shfl_sync(0xffffffffu, incl, 31);
  }
  const uint32_t total = carry;
  const bool direct = total > (uint32_t)kStageCap;
  __syncwarp();
  if (direct)
    for (int t = lane; t < k.tx_n; t += 32) s_next[t] += s_gd[t];
  const uint32_t bit = 1u << lane, lt = bit - 1u;
  __syncwarp();
  for (uint32_t pb = k.p0; pb < k.p1; pb += 32) {
    const uint32_t p = pb + lane;
    uint32_t item = 0, a = 0, len = 0;
    if (p < k.p1) {
      const uint32_t key = A.pkey[p];
      const int ka = key_a(key), kb = key_b(key);
      if (ka <= kb) {
        item = A.pval[p];
        a = (uint32_t)ka;
        len = (uint32_t)(kb - ka + 1);
      }
    }
    const uint32_t nzmask = __ballot_sync(0xffffffffu, len > 0);
    if (len > 0) s_nz[warp][__popc(nzmask & lt)] = (uint8_t)lane;
    const uint32_t es = warp_incl_scan(len);
    const uint32_t T = __shfl_sync(0xffffffffu, es, 31);
    const uint32_t estart = es - len;
    __syncwarp();
    // the group's entries 32 at a time: entry e belongs to pair run_owner(e),
    // column a + (e - its start); a column's rank among the window's entries
    // comes from its coverage word (one bit per lane)
    for (uint32_t e0 = 0; e0 < T; e0 += 32) {
      const int j = run_owner(estart, len, e0, s_nz[warp]);
      const uint32_t e = e0 + lane;
      const bool valid = e < T;
      const uint32_t tx = __shfl_sync(0xffffffffu, a, j) + (e - __shfl_sync(0xffffffffu, estart, j));
      const uint32_t it = __shfl_sync(0xffffffffu, item, j);
      if (valid) atomicOr(&s_cov[tx], bit);
      __syncwarp();
      uint32_t cov = 0;
      if (valid) {
        cov = s_cov[tx];
        const uint32_t pos = s_next[tx] + (uint32_t)__popc(cov & lt);
        if (!direct) {
          if (pos < (uint32_t)kStageCap) s_stage[pos] = it;
        } else if (pos < (uint64_t)A.n_entries) {
          A.vals[pos] = it;
        } else {
          atomicOr(A.status, kStatusEntryMismatch);
        }
      }
      __syncwarp();
      if (valid && (cov & lt) == 0u) {          // the column's lowest lane in the window
        s_next[tx] += (uint32_t)__popc(cov);
        s_cov[tx] = 0u;
      }
      __syncwarp();
    }
  }
  if (direct) return;
  // s_next now holds each column's local end: the column of staged entry i is
  // the first whose end exceeds i
  for (uint32_t i = lane; i < total; i += 32) {
    int lo = 0, hi = k.tx_n - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_next[mid] > i) hi = mid;
      else lo = mid + 1;
    }
    const uint32_t pos = s_gd[lo] + i;
    if (pos < (uint64_t)A.n_entries) A.vals[pos] = s_stage[i];
    else atomicOr(A.status, kStatusEntryMismatch);
  }
}

}  // namespace

size_t list_pair_radix_bytes(int64_t pairs) { return radix_scratch_bytes(pairs, kRowBits); }

cudaError_t launch_lists(const ListArgs& a, cudaStream_t stream) {
  if (a.n_entries <= 0 || a.n_pairs <= 0) {
    // no entries: every range is empty
    if (a.total_tiles > 0) return cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * (size_t)a.total_tiles, stream);
    return cudaSuccess;
  }
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = once_per_device(attr_done, [] {
    cudaError_t r = cudaFuncSetAttribute(l2_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kL2Warps * (kListTxMax + 1) * 4);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(l2_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kL2Warps * (3 * (kListTxMax + 1) + kStageCap) * 4);
    return r;
  });
  if (e != cudaSuccess) return e;
  const size_t smem2 = (size_t)kL2Warps * (a.max_tx + 1) * 4;
  const size_t smem3 = (size_t)kL2Warps * (3 * (a.max_tx + 1) + kStageCap) * 4;
  // second-level chunks: at most one partial chunk per row
  const int64_t c2_max = a.n_pairs / kListPairsPerChunk + a.rows;
  const int l2_blocks = (int)((c2_max + kL2Warps - 1) / kL2Warps);
  GS_TIMED("lists_pairs", stream,
           (pairs_kernel<<<ceil_div(a.n_items, 32 * kPairWarps), 32 * kPairWarps, 0, stream>>>(a)));
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = radix_sort_pairs(a.pkey, a.pkey_alt, a.pval, a.pval_alt, a.n_pairs, kRowBits, a.pair_radix, a.status, stream,
                         "pairs");
  if (e != cudaSuccess) return e;
  GS_TIMED("lists_rows", stream, (row_ranges_kernel<<<ceil_div((int64_t)a.rows + 1, 256), 256, 0, stream>>>(a)));
  GS_TIMED("lists_rows", stream, (rows_kernel<<<1, 1024, 0, stream>>>(a)));
  GS_TIMED("lists_tile_count", stream, (l2_count_kernel<<<l2_blocks, 32 * kL2Warps, smem2, stream>>>(a)));
  GS_TIMED("lists_tile_scan", stream, (l2_tile_kernel<<<a.rows, 128, 0, stream>>>(a)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = gather_exclusive_scan(a.tile_count, nullptr, a.tile_start, a.total_tiles, a.scan_blocks, a.scan_total, stream);
  if (e != cudaSuccess) return e;
  GS_TIMED("lists_ranges", stream,
           (l2_ranges_kernel<<<ceil_div(a.total_tiles, 256), 256, 0, stream>>>(a)));
  GS_TIMED("lists_entries", stream, (l2_emit_kernel<<<l2_blocks, 32 * kL2Warps, smem3, stream>>>(a)));
  return cudaGetLastError();
}

}  // namespace gs
