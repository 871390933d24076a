// Internal definitions shared by the rasterizer's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <utility>

#include "../../include/gs.h"

namespace gs {

constexpr int kTile = GS_TILE;
constexpr int kTilePixels = kTile * kTile;     // 256 threads per tile block
constexpr uint32_t kCulledKey = 0xFFFFFFFFu;   // depth key of a culled item

// Device status word bits (preprocess workspace).
constexpr uint32_t kStatusTimeout = 1u;        // a look-back spin ran out
constexpr uint32_t kStatusEntryMismatch = 2u;  // duplicate != counted tiles
constexpr uint32_t kStatusBounds = 4u;         // checked build: an index out of its array

// Index check of the checked build (GS_CHECKED): true when 0 <= i < n;
// otherwise it records kStatusBounds in *status and is false, so that the
// caller skips the access.  Without GS_CHECKED it is always true.
#ifdef GS_CHECKED
#define GS_IN_RANGE(i, n, status) \
  ((uint64_t)(i) < (uint64_t)(n) ? true : (atomicOr((status), ::gs::kStatusBounds), false))
#else
#define GS_IN_RANGE(i, n, status) true
#endif

// Per-view constants, uploaded into the preprocess workspace.
struct ViewDev {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float limx, limy;          // clamp * tan(half fov)
  float campos[3];           // camera centre -R^T t
  int32_t width, height, tiles_x, tiles_y;
  int32_t tile_base;
  int32_t row_base;          // first global tile row of the view (rows of all views concatenated)
  int64_t pixel_base;
};

// Per-item projected state, written by the preprocess kernel.
struct ItemState {
  float4* xy_tau_z;          // (mean2d.x, mean2d.y, tau, z)
  float4* conic_o;           // (A, B, C, opacity); q = A dx^2 + 2B dx dy + C dy^2
  float4* rgb;               // (r, g, b, support half-extents as two halves; see pack_extent)
  float4* depth_frame;       // 3 x float4 per item: rows of W = diag(1/s) (R Rq)^T, then e = W p_c
  uint2* rect;               // (tx0 | ty0 << 16, tx1 | ty1 << 16), inclusive bounding box
  float4* bin;               // 2 x float4 per item: the binning record of bin_decode (with the first band row)
  uint32_t* tiles;           // exact touched-tile count (0 = culled)
  uint32_t* depth_key;       // float bits of z, kCulledKey if culled
  uint32_t* depth_val;       // the item's own index: the depth sort's values
  uint32_t* status;          // device status word (kStatus* bits)
  const unsigned long long* n_entries;   // tile entries (sum of tiles)
  unsigned long long* entries_acc;       // the same word, summed by the preprocess with atomics
  uint32_t* band_rows;       // tile rows of the item's band (ty1 - ty0 + 1; 0 = culled)
};

// Offsets of the preprocess workspace regions (bytes), host-computed.
struct PreLayout {
  size_t views, status, n_entries;
  size_t xy_tau_z, conic_o, rgb, depth_frame, rect, bin, tiles, band_rows, depth_key;
  size_t sort_keys_alt, sort_vals, sort_vals_alt;   // depth sort buffers
  size_t sorted_items, offsets, pair_offsets;        // after the depth sort: scanned tiles / band sizes
  size_t scan_blocks;
  size_t radix_scratch;                              // histograms + look-back
  size_t grad2d;                                     // 2 x float4 per item, then 1 float per item
  size_t total;
};

// Sort workspace.  Two layouts: the counting-placement tile lists (lists.cu,
// `lists` true: vals, ranges and the lists' scratch) and the radix path
// (duplicate + onesweep sort by tile id: keys, alternates, radix scratch).
struct SortLayout {
  bool lists;
  size_t keys, keys_alt, vals, vals_alt, ranges, radix_scratch;
  size_t pkey, pkey_alt, pval, pval_alt, pair_radix, row_T, row_start, c2_start, cnt2_off, counts2, prefix2,
      tile_count, tile_start, scan_blocks, chunks, chunk_cnt, tile_order, tile_hist;
  int rows;
  int64_t counts2_n;
  size_t total;
};

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

__host__ __device__ inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---- bulk asynchronous copies (cp.async.bulk + mbarrier) --------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned) whose completion is counted on `bar`
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bounded wait for phase `phase` of `bar`; false if the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, long budget) {
  for (long it = 0; it < budget; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Runs `init` once per (device, slot): per-device state such as a kernel's
// dynamic shared-memory limit or a __constant__ table.  Thread-safe; a failed
// init is retried on the next call.
template <typename F>
cudaError_t once_per_device(std::atomic<uint64_t>& done, F&& init) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const uint64_t bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = init();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Streaming multiprocessors of the current device, queried once per device
// (api.cu); grid-stride launch shapes are sized in multiples of it.  1 if the
// query fails (every such launch is still correct, only narrower).
int device_sm_count();

// ---- onesweep radix sort sizing (sort.cu) ----------------------------------
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 512;
constexpr int kSortItemsPerThread = 15;
constexpr int kSortTile = kSortThreads * kSortItemsPerThread;   // keys per CTA tile

size_t radix_scratch_bytes(int64_t n, int bits);
// Stable LSD sort of (key, value) pairs over bits [0, bits) (higher key bits
// are carried along, not sorted): 8-bit passes and a narrow last one, or one
// 512-digit pass when bits is 9.  The result ends up in (keys, vals) (the alt
// buffers are scratch), except that with result_in_alt given an odd number
// of passes leaves it in the alt buffers and sets *result_in_alt instead of
// copying it back.  `status` receives kStatusTimeout if a look-back spin ran
// out.
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                             int64_t n, int bits, void* scratch, uint32_t* status,
                             cudaStream_t stream, const char* tag, bool* result_in_alt = nullptr);

// ---- exclusive scan of gathered counts (sort.cu) ---------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
size_t scan_block_bytes(int64_t n);
// Self-test of the sort's bounded look-back wait (scratch: 3 * 256 words).
cudaError_t lookback_timeout_probe(uint32_t* scratch, uint32_t* status, cudaStream_t stream);
// The same for the exclusive scan's look-back (scratch: 3 words of 8 bytes).
cudaError_t scan_timeout_probe(uint64_t* scratch, uint32_t* status, cudaStream_t stream);
// out[k] = sum_{j<k} counts[idx[j]] (idx == nullptr: counts[j]); *total = sum of
// all (device, 64-bit).  One pass with a decoupled look-back; block_scratch:
// scan_block_bytes(n), cleared by the call; a look-back wait that runs out
// records kStatusTimeout in *status (if given).
cudaError_t gather_exclusive_scan(const uint32_t* counts, const uint32_t* idx, uint32_t* out,
                                  int64_t n, uint64_t* block_scratch, unsigned long long* total,
                                  cudaStream_t stream, uint32_t* status = nullptr);

// ---- opt-in per-kernel timing (timing.cu) ----------------------------------
void timing_begin(const char* name, cudaStream_t stream);
void timing_end(cudaStream_t stream);
struct TimedLaunch {
  cudaStream_t s;
  TimedLaunch(const char* name, cudaStream_t st) : s(st) { timing_begin(name, st); }
  ~TimedLaunch() { timing_end(s); }
};
#define GS_TIMED(name, stream, launch) \
  do {                                 \
    ::gs::TimedLaunch _t(name, stream); \
    launch;                            \
  } while (0)

// ---- kernel launchers -------------------------------------------------------
cudaError_t launch_preprocess(const gs_scene& sc, const ViewDev* views, int n_views, const uint8_t* mask,
                              const gs_config& cfg, const ItemState& st, cudaStream_t stream);
cudaError_t launch_preprocess_backward(const gs_scene& sc, const ViewDev* views, int n_views, const gs_config& cfg,
                                       const uint32_t* tiles, const float4* grad2d, const float* grad2d_b,
                                       const gs_grads& gr, cudaStream_t stream);
cudaError_t launch_duplicate(const ViewDev* views, int n_views, int64_t n_items, int64_t n, const uint32_t* sorted_items,
                             const uint32_t* offsets, const ItemState& st, uint32_t* keys, uint32_t* vals,
                             uint32_t* status, cudaStream_t stream);
cudaError_t launch_ranges(const uint32_t* keys, int64_t n_entries, uint2* ranges, int total_tiles,
                          cudaStream_t stream);
// order: the tiles' launch order written by the tile-list builder (null: tile
// id order).  Only the forward takes it: the backward, whose cost follows the
// pixels' contribution counts more than the list lengths, gains no time from
// it and loses the L2 reuse of neighbouring tiles (its DRAM traffic rose from
// 590 to 959 MB per launch at 1M Gaussians over 8 views)
cudaError_t launch_render_fwd(const ViewDev* views, int n_views, int64_t n, int total_tiles, const uint2* ranges,
                              const uint32_t* vals, const uint32_t* order, const ItemState& st, const gs_config& cfg,
                              const gs_fwd_outputs& out, cudaStream_t stream);
cudaError_t launch_render_bwd(const ViewDev* views, int n_views, int64_t n, int total_tiles, const uint2* ranges,
                              const uint32_t* vals, const ItemState& st, const gs_config& cfg,
                              const float* dL_dimage, const float* image, const uint32_t* n_contrib,
                              float4* grad2d, float* grad2d_b, float* weight_sum, uint64_t* weight_sum_fixed,
                              cudaStream_t stream);
// ---- tile lists by counting placement (lists.cu) ----------------------------
constexpr int kListRowsMax = 4096;        // global tile rows (all views) the lists path handles
constexpr int kListTxMax = 1023;          // tiles per row
constexpr int kListPairsPerChunk = 256;   // (item, row) pairs per second-level chunk
constexpr uint32_t kListEmpty = 0xFFFFFFFFu;   // a pair whose row has no tile in the image
struct ListArgs {
  const ViewDev* views;     // device
  int n_views;
  int64_t n, n_items, n_entries, n_pairs;
  int rows, total_tiles, max_tx;
  int64_t counts2_n;        // second-level counters allocated
  const uint32_t* sorted_items;
  const uint32_t* pair_offsets;   // scanned band sizes in depth order (the preprocess's offsets array)
  ItemState st;
  uint32_t* vals;           // [n_entries] items in tile order (the output)
  uint2* ranges;            // [total_tiles] (the output)
  uint32_t *pkey, *pkey_alt, *pval, *pval_alt;   // pairs and the radix sort's alternates
  void* pair_radix;         // radix scratch for n_pairs keys over the row bits
  int32_t* counts2;         // per second-level chunk, entries per column
  uint32_t* prefix2;        // the same, exclusive over the row's chunks
  uint32_t *row_T, *row_start, *c2_start, *cnt2_off, *tile_count, *tile_start;
  int4* chunks;             // per second-level chunk: tiles across, first tile, pairs [p0, p1)
  uint32_t* chunk_cnt;      // per second-level chunk: offset of its counters
  uint64_t* scan_blocks;
  unsigned long long* scan_total;
  uint32_t* status;
  // launch order of the render kernels' tiles, longest list first (tiles
  // bucketed by the bit length of their list), and the buckets' counts and
  // cursors (kTileBuckets each, zeroed before the tile scan)
  uint32_t* tile_order;
  uint32_t* tile_hist;
};
constexpr int kTileBuckets = 33;    // bit lengths 0 .. 32 of a list length
size_t list_pair_radix_bytes(int64_t pairs);
cudaError_t launch_lists(const ListArgs& a, cudaStream_t stream);

cudaError_t launch_loss_l1(const float* image, const float* target, int64_t count, float* loss, float* dL,
                           cudaStream_t stream);

}  // namespace gs
