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
//            in pair order (ranks among 32 entries from one coverage word per
//            column), and writes every column's run out contiguously.
//
// Every placement is a prefix count in the order of the input, so a tile's
// list holds its items in depth order (ties by item index, as the depth sort
// is stable): exactly the order of a stable sort of the entries by tile id.
// Traffic: 4 B of output per entry plus about 40 B per pair, against 44 B
// per entry for emitting every entry and sorting the entries by tile id
// (about 2.7 entries per pair at the training workloads).  The tile scan and
// the ranges pass also write the forward's launch order of the tiles,
// longest list first (tiles bucketed by the bit length of their list).
// Consistency checks:
// the pairs written equal the preprocess's count and the entries placed equal
// the scanned tile counts; a mismatch sets kStatusEntryMismatch.
#include "project.cuh"

namespace gs {

namespace {

constexpr int kL2Warps = 4;
constexpr int kL2EmitWarps = 4;
constexpr int kStageCap = 768;             // entries a second-level chunk stages in shared memory
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
constexpr int kPairWarps = 4;

__global__ void __launch_bounds__(32 * kPairWarps) pairs_kernel(ListArgs A) {
  // each lane's item record as three float4 (one 128-bit shared access each):
  // (mx, my, tau, k), (sc, 1/Syy, h, rx), (ys, item, ty0, row_base | tiles_x << 16)
  __shared__ float4 s_it[kPairWarps][3][32];
  __shared__ uint8_t s_nz[kPairWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t k0 = ((int64_t)blockIdx.x * kPairWarps + warp) * 32;
  if (k0 >= A.n_items) return;                               // warp-uniform
  const int64_t k = k0 + lane;
  uint32_t nrows = 0;
  if (k < A.n_items) {
    // band size from the scanned offsets (coalesced), so that only visible
    // items are gathered
    const uint32_t o0 = A.pair_offsets[k];
    const uint32_t o1 = k + 1 < A.n_items ? A.pair_offsets[k + 1] : (uint32_t)A.n_pairs;
    nrows = o1 - o0;
    if (nrows) {
      uint32_t item = A.sorted_items[k];
      if (!GS_IN_RANGE(item, A.n_items, A.status)) item = 0;
      const ViewDev& V = A.views[item / A.n];
      // one 32-byte record per item (the gathers follow the depth order)
      const float4 r0 = A.st.bin[2 * item], r1 = A.st.bin[2 * item + 1];
      const BinParams b = bin_decode(r0, r1);
      s_it[warp][0][lane] = make_float4(b.mx, b.my, b.tau, b.k);
      s_it[warp][1][lane] = make_float4(b.sc, b.isyy, b.h, b.rx);
      s_it[warp][2][lane] = make_float4(b.ys, __uint_as_float(item), r1.w,
                                        __uint_as_float((uint32_t)V.row_base | ((uint32_t)V.tiles_x << 16)));
    }
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
      const float4 q0 = s_it[warp][0][j], q1 = s_it[warp][1][j], q2 = s_it[warp][2][j];
      BinParams b;
      b.mx = q0.x;
      b.my = q0.y;
      b.tau = q0.z;
      b.k = q0.w;
      b.sc = q1.x;
      b.isyy = q1.y;
      b.h = q1.z;
      b.rx = q1.w;
      b.ys = q2.x;
      const uint32_t rb = __float_as_uint(q2.w);
      const int row_base = (int)(rb & 0xFFFFu), tiles_x = (int)(rb >> 16);
      const int ty = __float_as_int(q2.z) + (int)r;
      int ta, tb;
      const uint32_t key = row_tiles(b, ty, tiles_x, &ta, &tb) ? pair_key(row_base + ty, ta, tb)
                                                              : ((uint32_t)(row_base + ty) | kEmptyAB);
      const uint64_t pos = (uint64_t)base + u;
      if (pos < (uint64_t)A.n_pairs) {
        A.pkey[pos] = key;
        A.pval[pos] = __float_as_uint(q2.y);
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
  int tx_n, tb;                 // tiles across the row's view, global id of the row's first tile
  uint32_t p0, p1;              // the chunk's pairs [p0, p1)
  uint32_t cnt;                 // offset of its counters
};

// The table of second-level chunks: thread per chunk (its row by binary
// search in the chunk table), so that the chunk kernels read one record.
__global__ void chunk_table_kernel(ListArgs A) {
  const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.c2_start[A.rows]) return;
  int lo = 0, hi = A.rows - 1;                  // last row with c2_start <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.c2_start[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  const ViewDev& V = A.views[view_of_row(A.views, A.n_views, lo)];
  const uint32_t j = c - A.c2_start[lo];
  const uint32_t rs = A.row_start[lo], re = A.row_start[lo] + A.row_T[lo];
  const uint32_t p0 = rs + j * (uint32_t)kListPairsPerChunk;
  A.chunks[c] = make_int4(V.tiles_x, V.tile_base + (lo - V.row_base) * V.tiles_x, (int)p0,
                          (int)min(p0 + (uint32_t)kListPairsPerChunk, re));
  A.chunk_cnt[c] = A.cnt2_off[lo] + j * (uint32_t)V.tiles_x;
}

// The second-level chunk c from the table; false past the last chunk or if
// its pairs or counters would leave their arrays (counts that disagree with
// the preprocess's are flagged by the totals).
__device__ __forceinline__ bool chunk2(const ListArgs& A, uint32_t c, Chunk2* k) {
  if (c >= A.c2_start[A.rows]) return false;
  const int4 r = A.chunks[c];
  k->tx_n = r.x;
  k->tb = r.y;
  k->p0 = (uint32_t)r.z;
  k->p1 = (uint32_t)r.w;
  k->cnt = A.chunk_cnt[c];
  return k->p1 <= (uint32_t)A.n_pairs && (int64_t)k->cnt + k->tx_n <= A.counts2_n;
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

// The identity launch order (no entries).
__global__ void identity_order_kernel(uint32_t* order, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) order[t] = (uint32_t)t;
}

// Bucket of a tile's list length: its bit length (0 for an empty list).
__device__ __forceinline__ uint32_t tile_bucket(uint32_t len) { return len ? 32u - (uint32_t)__clz(len) : 0u; }

// Per row: exclusive scan of each column's counts over the row's chunks
// (into prefix2), and the tile totals.  Block per (row, 32 columns); its
// warps split the row's chunks, sum their share, and then scan it from the
// sums of the warps before them.
constexpr int kTileScanWarps = 8;

__global__ void __launch_bounds__(32 * kTileScanWarps) l2_tile_kernel(ListArgs A) {
  __shared__ uint32_t s_part[kTileScanWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r = blockIdx.x;
  const ViewDev& V = A.views[view_of_row(A.views, A.n_views, r)];
  const int tx_n = V.tiles_x;
  const int t = blockIdx.y * 32 + lane;
  if (blockIdx.y * 32 >= tx_n) return;                       // block-uniform
  const uint32_t nch = A.c2_start[r + 1] - A.c2_start[r];
  const int64_t off = A.cnt2_off[r];
  const uint32_t per = (nch + kTileScanWarps - 1) / kTileScanWarps;
  const uint32_t j0 = min(warp * per, nch), j1 = min(j0 + per, nch);
  uint32_t sum = 0;
  if (t < tx_n)
    for (uint32_t j = j0; j < j1; ++j) sum += (uint32_t)A.counts2[off + (int64_t)j * tx_n + t];
  s_part[warp][lane] = sum;
  __syncthreads();
  if (t >= tx_n) return;
  uint32_t run = 0;
  for (int w2 = 0; w2 < warp; ++w2) run += s_part[w2][lane];
  for (uint32_t j = j0; j < j1; ++j) {
    const int64_t i = off + (int64_t)j * tx_n + t;
    A.prefix2[i] = run;
    run += (uint32_t)A.counts2[i];
  }
  if (warp == kTileScanWarps - 1) {
    A.tile_count[V.tile_base + (r - V.row_base) * tx_n + t] = run;
    // the tile's length bucket for the render kernels' launch order
    // (warp-aggregated: one atomic per bucket present in the warp)
    const uint32_t b = tile_bucket(run);
    const uint32_t peers = __match_any_sync(__activemask(), b);
    if (lane == __ffs(peers) - 1) atomicAdd(&A.tile_hist[b], (uint32_t)__popc(peers));
  }
}

// [start, end) of every tile and the tiles' launch order; checks the entry
// total against the preprocess's.
__global__ void l2_ranges_kernel(ListArgs A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < A.total_tiles) {
    const uint32_t c = A.tile_count[t];
    A.ranges[t] = make_uint2(A.tile_start[t], A.tile_start[t] + c);
    // launch order, longest lists first: the tile goes after every tile of
    // a longer bucket, at its bucket's cursor (any order inside a bucket)
    const uint32_t b = tile_bucket(c);
    uint32_t off = 0;
    for (int k = kTileBuckets - 1; k > (int)b; --k) off += A.tile_hist[k];
    const uint32_t peers = __match_any_sync(__activemask(), b);
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&A.tile_hist[kTileBuckets + b], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    const uint32_t pos = off + base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    if (pos < (uint32_t)A.total_tiles) A.tile_order[pos] = (uint32_t)t;
    else atomicOr(A.status, kStatusEntryMismatch);
  }
  if (t == 0 && *A.scan_total != (unsigned long long)A.n_entries) atomicOr(A.status, kStatusEntryMismatch);
}

// Places the entries of every second-level chunk (warp per chunk) in pair
// order and, inside a pair, in column order.  The entries of 32 consecutive
// pairs are taken 32 at a time (lane l the l-th, its pair found by
// run_owner); an entry's rank at its column is the number of lower lanes with
// the same column, read from a coverage word per column (bit l set by lane
// l); the column's lowest lane then advances the column's next slot and
// clears the word.  The entries are staged in shared memory grouped by column
// (the chunk's own counts give each column's local start) and then written
// out column by column, each column's run to consecutive addresses of its
// tile's list, so that stores coalesce.  A chunk with more than kStageCap
// entries (very wide supports) writes its entries straight to their places.
__global__ void __launch_bounds__(32 * kL2EmitWarps) l2_emit_kernel(ListArgs A) {
  extern __shared__ uint32_t s_dyn3[];
  __shared__ uint8_t s_nz[kL2EmitWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w = A.max_tx + 1;
  uint32_t* s_next = s_dyn3 + warp * (2 * w + kStageCap + kStageCap / 2);   // next slot of each column
  uint32_t* s_cov = s_next + w;                              // coverage words of the current window
  uint32_t* s_stage = s_cov + w;                             // the chunk's entries, grouped by column
  uint16_t* s_tag = reinterpret_cast<uint16_t*>(s_stage + kStageCap);   // their columns
  Chunk2 k;
  if (!chunk2(A, blockIdx.x * kL2EmitWarps + warp, &k)) return;   // warp-uniform
  uint32_t carry = 0;
  for (int t0 = 0; t0 < k.tx_n; t0 += 32) {                 // local starts: scan of the chunk's counts
    const int t = t0 + lane;
    const uint32_t own = t < k.tx_n ? (uint32_t)A.counts2[k.cnt + t] : 0u;
    const uint32_t incl = warp_incl_scan(own) + carry;
    if (t < k.tx_n) {
      s_next[t] = incl - own;
      s_cov[t] = 0u;
    }
    carry = __shfl_sync(0xffffffffu, incl, 31);
  }
  const uint32_t total = carry;
  const bool direct = total > (uint32_t)kStageCap;
  __syncwarp();
  if (direct)
    for (int t = lane; t < k.tx_n; t += 32) s_next[t] = A.tile_start[k.tb + t] + A.prefix2[k.cnt + t];
  const uint32_t bit = 1u << lane, lt = bit - 1u;
  __syncwarp();
  // the pairs of the next group are loaded while the current one is placed
  uint32_t nkey = k.p0 + lane < k.p1 ? A.pkey[k.p0 + lane] : kEmptyAB;
  uint32_t nval = k.p0 + lane < k.p1 ? A.pval[k.p0 + lane] : 0u;
  for (uint32_t pb = k.p0; pb < k.p1; pb += 32) {
    const uint32_t key = nkey, val = nval;
    const uint32_t pn = pb + 32 + lane;
    nkey = pn < k.p1 ? A.pkey[pn] : kEmptyAB;
    nval = pn < k.p1 ? A.pval[pn] : 0u;
    uint32_t item = 0, a = 0, len = 0;
    {
      const int ka = key_a(key), kb = key_b(key);
      if (ka <= kb) {
        item = val;
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
          if (pos < (uint32_t)kStageCap) {
            s_stage[pos] = it;
            s_tag[pos] = (uint16_t)tx;
          }
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
  // write-out: the coverage words (all zero again) take each column's global
  // start minus its local start; staged entry i goes to that + i, so runs of
  // one column go to consecutive addresses
  {
    uint32_t carry2 = 0;
    for (int t0 = 0; t0 < k.tx_n; t0 += 32) {
      const int t = t0 + lane;
      const uint32_t own = t < k.tx_n ? (uint32_t)A.counts2[k.cnt + t] : 0u;
      const uint32_t incl = warp_incl_scan(own) + carry2;
      if (t < k.tx_n) s_cov[t] = A.tile_start[k.tb + t] + A.prefix2[k.cnt + t] - (incl - own);
      carry2 = __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncwarp();
  for (uint32_t i = lane; i < total; i += 32) {
    const uint32_t pos = s_cov[s_tag[i]] + i;
    if (pos < (uint64_t)A.n_entries) A.vals[pos] = s_stage[i];
    else atomicOr(A.status, kStatusEntryMismatch);
  }
}

}  // namespace

size_t list_pair_radix_bytes(int64_t pairs) { return radix_scratch_bytes(pairs, kRowBits); }

cudaError_t launch_lists(const ListArgs& a, cudaStream_t stream) {
  if (a.n_entries <= 0 || a.n_pairs <= 0) {
    // no entries: every range is empty, and the tiles launch in id order
    if (a.total_tiles <= 0) return cudaSuccess;
    cudaError_t e0 = cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * (size_t)a.total_tiles, stream);
    if (e0 != cudaSuccess) return e0;
    identity_order_kernel<<<ceil_div(a.total_tiles, 256), 256, 0, stream>>>(a.tile_order, a.total_tiles);
    return cudaGetLastError();
  }
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t e = once_per_device(attr_done, [] {
    cudaError_t r = cudaFuncSetAttribute(l2_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kL2Warps * (kListTxMax + 1) * 4);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(l2_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kL2EmitWarps * (2 * (kListTxMax + 1) + kStageCap + kStageCap / 2) * 4);
    return r;
  });
  if (e != cudaSuccess) return e;
  const size_t smem2 = (size_t)kL2Warps * (a.max_tx + 1) * 4;
  const size_t smem3 = (size_t)kL2EmitWarps * (2 * (a.max_tx + 1) + kStageCap + kStageCap / 2) * 4;
  // second-level chunks: at most one partial chunk per row
  const int64_t c2_max = a.n_pairs / kListPairsPerChunk + a.rows;
  const int l2_blocks = (int)((c2_max + kL2Warps - 1) / kL2Warps);
  GS_TIMED("lists_pairs", stream,
           (pairs_kernel<<<ceil_div(a.n_items, 32 * kPairWarps), 32 * kPairWarps, 0, stream>>>(a)));
  e = cudaGetLastError();
  // the sort covers the bits the row ids use: one 8- or 9-bit pass up to 512
  // rows; with one pass the sorted pairs stay in the alternate buffers
  int row_bits = 1;
  while ((1 << row_bits) < a.rows) ++row_bits;
  bool in_alt = false;
  if (e == cudaSuccess)
    e = radix_sort_pairs(a.pkey, a.pkey_alt, a.pval, a.pval_alt, a.n_pairs, row_bits, a.pair_radix, a.status, stream,
                         "pairs", &in_alt);
  if (e != cudaSuccess) return e;
  ListArgs L = a;
  if (in_alt) {
    std::swap(L.pkey, L.pkey_alt);
    std::swap(L.pval, L.pval_alt);
  }
  GS_TIMED("lists_rows", stream, (row_ranges_kernel<<<ceil_div((int64_t)a.rows + 1, 256), 256, 0, stream>>>(L)));
  GS_TIMED("lists_rows", stream, (rows_kernel<<<1, 1024, 0, stream>>>(L)));
  GS_TIMED("lists_rows", stream, (chunk_table_kernel<<<ceil_div(c2_max, 256), 256, 0, stream>>>(L)));
  GS_TIMED("lists_tile_count", stream, (l2_count_kernel<<<l2_blocks, 32 * kL2Warps, smem2, stream>>>(L)));
  e = cudaMemsetAsync(L.tile_hist, 0, 2 * kTileBuckets * sizeof(uint32_t), stream);
  if (e != cudaSuccess) return e;
  GS_TIMED("lists_tile_scan", stream,
           (l2_tile_kernel<<<dim3(a.rows, (a.max_tx + 31) / 32), 32 * kTileScanWarps, 0, stream>>>(L)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = gather_exclusive_scan(L.tile_count, nullptr, L.tile_start, L.total_tiles, L.scan_blocks, L.scan_total, stream,
                            L.status);
  if (e != cudaSuccess) return e;
  GS_TIMED("lists_ranges", stream,
           (l2_ranges_kernel<<<ceil_div(a.total_tiles, 256), 256, 0, stream>>>(L)));
  GS_TIMED("lists_entries", stream,
           (l2_emit_kernel<<<(int)((c2_max + kL2EmitWarps - 1) / kL2EmitWarps), 32 * kL2EmitWarps, smem3, stream>>>(
               L)));
  return cudaGetLastError();
}

}  // namespace gs
