// Tile binning: one (global tile id, item) entry per touched tile, emitted in
// the depth order of the items (Sec. 3.1), then tile ranges of the list
// sorted by tile id.  Also the L1 photometric loss of the training step.
//
// Duplication: the entries of each item of the depth order, its tile rows
// evaluated with the same interval form of the support as the counting pass
// in preprocess (identical arithmetic on the same stored parameters), written
// at its scanned offset, row-major.
#include "project.cuh"

namespace gs {

namespace {

constexpr int kDupThreads = 256;
constexpr int kDupWarps = kDupThreads / 32;

// Per-lane state of the item a lane loaded (the warp's 32 consecutive items
// of the depth order).
struct DupItem {
  BinParams b;
  uint32_t item, off, cnt;
  int ty0, tiles_x, tile_base;
};

// One warp per 32 consecutive items of the depth order.  Their entries form
// one contiguous run of the output, and every item's are its tile rows in
// order, so the warp enumerates (item, tile row) pairs 32 at a time: each
// lane evaluates one row's tile interval (the same row_tiles the preprocess
// counted with), a warp scan turns the row lengths into positions, and the
// lanes then write the 32 rows' entries together (entry e of the iteration
// is the e-th of one contiguous run, so the stores coalesce).  A lane finds
// the row of its entry (and the item of its row) without a search: the rows
// with entries have distinct, increasing starts, so the row holding e is the
// last one starting at or before e, counted with one ballot (starts before
// the window of 32) and one OR-reduction (one bit per start inside it).
// Every item's rows must add up to the count the preprocess stored; a
// mismatch sets kStatusEntryMismatch and nothing is written out of range.
__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(const ViewDev* __restrict__ views, int64_t n_items,
                                                                int64_t n, const uint32_t* __restrict__ sorted_items,
                                                                const uint32_t* __restrict__ offsets, ItemState st,
                                                                uint32_t* __restrict__ keys,
                                                                uint32_t* __restrict__ vals,
                                                                uint32_t* __restrict__ status) {
  __shared__ DupItem s_it[kDupWarps][32];
  __shared__ uint32_t s_rstart[kDupWarps][33];     // first row unit of each lane's item
  __shared__ uint32_t s_pre[kDupWarps][33];        // entries before each row of the iteration
  __shared__ uint32_t s_key0[kDupWarps][32];       // key of each row's first entry
  __shared__ uint32_t s_item[kDupWarps][32];       // item of each row
  __shared__ uint32_t s_out0[kDupWarps][32];       // output position of each row's first entry
  __shared__ uint32_t s_lim[kDupWarps][32];        // entries the row may write (its item's remaining count)
  __shared__ uint8_t s_nerow[kDupWarps][32];       // the lanes of the rows with entries, in order
  __shared__ uint8_t s_neitem[kDupWarps][32];      // the lanes of the items with rows, in order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t k = ((int64_t)blockIdx.x * kDupWarps + warp) * 32 + lane;
  if (((int64_t)blockIdx.x * kDupWarps + warp) * 32 >= n_items) return;     // warp-uniform

  // 1. this lane's item and its band of tile rows
  uint32_t nrows = 0;
  {
    DupItem d;
    d.item = 0;
    d.cnt = 0;
    d.off = 0;
    d.ty0 = 0;
    d.tiles_x = 0;
    d.tile_base = 0;
    if (k < n_items) {
      d.item = sorted_items[k];
      const bool known = GS_IN_RANGE(d.item, n_items, status);
      if (!known) d.item = 0;
      d.cnt = known ? st.tiles[d.item] : 0u;
      if (d.cnt) {
        d.off = offsets[k];
        d.b = bin_decode(st.bin[2 * d.item], st.bin[2 * d.item + 1]);
        const ViewDev& V = views[d.item / n];
        d.tiles_x = V.tiles_x;
        d.tile_base = V.tile_base;
        int ty1 = -1;
        if (tile_rows(d.b, V.tiles_y, &d.ty0, &ty1)) nrows = (uint32_t)(ty1 - d.ty0 + 1);
        else atomicOr(status, kStatusEntryMismatch);      // a counted item always has rows
      }
    }
    s_it[warp][lane] = d;
  }
  uint32_t rs = nrows;                                    // exclusive scan of the row counts
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, rs, o);
    if (lane >= o) rs += t;
  }
  const uint32_t R = __shfl_sync(0xffffffffu, rs, 31);
  s_rstart[warp][lane] = rs - nrows;
  if (lane == 31) s_rstart[warp][32] = R;
  const uint32_t rstart = rs - nrows;                     // this lane's item's first row unit
  const uint32_t has_rows = __ballot_sync(0xffffffffu, nrows > 0);
  if (nrows > 0) s_neitem[warp][__popc(has_rows & ((1u << lane) - 1u))] = (uint8_t)lane;
  __syncwarp();

  // 2. 32 rows at a time
  int carry_j = -1;                                       // item continuing from the last iteration
  uint32_t carry = 0;                                     // its entries in earlier iterations
  for (uint32_t u0 = 0; u0 < R; u0 += 32) {
    const uint32_t u = u0 + lane;
    const bool valid = u < R;
    int j = 32;                                           // owner item (lane index), 32 = none
    uint32_t c = 0, key0 = 0;
    // the item owning row u: the last item with rows whose first row is at or
    // before u (items before the window, plus one bit per start inside it)
    const bool in_window = nrows > 0 && rstart >= u0 && rstart < u0 + 32;
    const uint32_t M = __reduce_or_sync(0xffffffffu, in_window ? 1u << (rstart - u0) : 0u);
    const uint32_t before = __popc(__ballot_sync(0xffffffffu, nrows > 0 && rstart < u0));
    if (valid) {
      j = s_neitem[warp][before + __popc(M & ((2u << lane) - 1u)) - 1u];
      const DupItem& d = s_it[warp][j];
      const int ty = d.ty0 + (int)(u - s_rstart[warp][j]);
      int ta, tb;
      if (row_tiles(d.b, ty, d.tiles_x, &ta, &tb)) {
        c = (uint32_t)(tb - ta + 1);
        key0 = (uint32_t)(d.tile_base + ty * d.tiles_x + ta);
      }
    }
    // entries of the same item in earlier lanes of this iteration (segmented
    // inclusive scan; j is non-decreasing across the lanes)
    uint32_t seg = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, seg, o);
      const int jo = __shfl_up_sync(0xffffffffu, j, o);
      if (lane >= o && jo == j) seg += t;
    }
    const uint32_t in_item = seg - c + (j == carry_j ? carry : 0u);    // entries of the item before this row
    if (valid && u + 1 == s_rstart[warp][j + 1] && in_item + c != s_it[warp][j].cnt)
      atomicOr(status, kStatusEntryMismatch);            // the item's last row: the totals must agree
    // positions of the rows in the iteration's run
    uint32_t pre = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += t;
    }
    const uint32_t T = __shfl_sync(0xffffffffu, pre, 31);
    s_pre[warp][lane] = pre - c;
    if (lane == 31) s_pre[warp][32] = T;
    s_key0[warp][lane] = key0;
    s_item[warp][lane] = valid ? s_it[warp][j].item : 0u;
    // a row writes at its item's offset plus the item's earlier entries, and
    // never beyond the item's count (with counts that agree, consecutive rows
    // continue one run, so entry e lands at the run start + e)
    const uint32_t icnt = valid ? s_it[warp][j].cnt : 0u;
    s_out0[warp][lane] = valid ? s_it[warp][j].off + in_item : 0u;
    s_lim[warp][lane] = icnt > in_item ? icnt - in_item : 0u;
    const int next_j = __shfl_sync(0xffffffffu, j, 31);
    const uint32_t next_carry = __shfl_sync(0xffffffffu, in_item + c, 31);
    // the rows with entries, ranked: their starts are distinct and increasing
    const uint32_t start = pre - c;
    const uint32_t nonempty = __ballot_sync(0xffffffffu, c > 0);
    if (c > 0) s_nerow[warp][__popc(nonempty & ((1u << lane) - 1u))] = (uint8_t)lane;
    __syncwarp();
    for (uint32_t e0 = 0; e0 < T; e0 += 32) {
      // the row holding entry e = e0 + lane is the last row with entries that
      // starts at or before e: those starting before e0, plus those starting
      // in [e0, e] (one bit each in M)
      const bool in_window = c > 0 && start >= e0 && start < e0 + 32;
      const uint32_t M = __reduce_or_sync(0xffffffffu, in_window ? 1u << (start - e0) : 0u);
      const uint32_t before = __popc(__ballot_sync(0xffffffffu, c > 0 && start < e0));
      const uint32_t e = e0 + lane;
      if (e < T) {
        const int lo = s_nerow[warp][before + __popc(M & ((2u << lane) - 1u)) - 1u];
        const uint32_t d = e - s_pre[warp][lo];
        if (d < s_lim[warp][lo]) {
          const uint32_t at = s_out0[warp][lo] + d;
          if (GS_IN_RANGE(at, *st.n_entries, status)) {
            keys[at] = s_key0[warp][lo] + d;
            vals[at] = s_item[warp][lo];
          }
        }
      }
    }
    __syncwarp();
    carry_j = next_j;
    carry = next_carry;
  }
}

// [start, end) of every tile in the sorted key list by binary search: thread
// t finds the first entry with key >= t, which starts tile t and ends tile
// t - 1 (t = total_tiles closes the last tile).
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, int64_t n, uint2* __restrict__ ranges,
                              int total_tiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > total_tiles) return;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < (uint32_t)t) lo = mid + 1;
    else hi = mid;
  }
  if (t < total_tiles) ranges[t].x = (uint32_t)lo;
  if (t > 0) ranges[t - 1].y = (uint32_t)lo;
}

__global__ void l1_kernel(const float* __restrict__ img, const float* __restrict__ tgt, int64_t count,
                          float* __restrict__ loss, float* __restrict__ dL) {
  const float inv = 1.f / (float)count;
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[i] - tgt[i];
    acc += fabsf(d);
    dL[i] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ float s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.f;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) atomicAdd(loss, v * inv);
  }
}


}  // namespace

cudaError_t launch_duplicate(const ViewDev* views, int n_views, int64_t n_items, int64_t n,
                             const uint32_t* sorted_items, const uint32_t* offsets, const ItemState& st,
                             uint32_t* keys, uint32_t* vals, uint32_t* status, cudaStream_t stream) {
  (void)n_views;
  const int blocks = ceil_div(n_items, kDupThreads);
  if (blocks > 0)
    GS_TIMED("duplicate", stream,
             (duplicate_kernel<<<blocks, kDupThreads, 0, stream>>>(views, n_items, n, sorted_items, offsets, st,
                                                                    keys, vals, status)));
  return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t* keys, int64_t n_entries, uint2* ranges, int total_tiles,
                          cudaStream_t stream) {
  if (total_tiles > 0)
    GS_TIMED("ranges", stream,
             (ranges_kernel<<<ceil_div((int64_t)total_tiles + 1, 256), 256, 0, stream>>>(keys, n_entries, ranges,
                                                                                         total_tiles)));
  return cudaGetLastError();
}


cudaError_t launch_loss_l1(const float* image, const float* target, int64_t count, float* loss, float* dL,
                           cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), stream);
  if (e != cudaSuccess) return e;
  if (count > 0) {
    const int blocks = (int)std::min<int64_t>(ceil_div(count, 256), (int64_t)8 * device_sm_count());
    GS_TIMED("loss_l1", stream, (l1_kernel<<<blocks, 256, 0, stream>>>(image, target, count, loss, dL)));
  }
  return cudaGetLastError();
}

}  // namespace gs
