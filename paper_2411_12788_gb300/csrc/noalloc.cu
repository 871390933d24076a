// gs_bin_sort_noalloc: the binning and tile sort of gs_bin_sort (Sec. 3.1) for
// callers that cannot allocate device memory; the variant itself has no
// counterpart in the paper.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they render: a renderer embedded in a host that owns all GPU
// memory and hands out fixed buffers, code running where an allocation could
// block or fail mid-frame, or a caller that sized every buffer up front.  They
// can still allocate the outputs once, but not the sort's scratch, whose size
// depends on the number of tile entries.  This entry point takes that scratch
// from a file-scope device array of fixed size instead, so it needs no
// allocation at all.  The array's cost: every GPU that loads the library keeps
// GS_NOALLOC_SCRATCH_BYTES reserved until the process exits.
//
// Set-up: the array's device address is looked up once per device with
// cudaGetSymbolAddress (in host code the array's name is only a host-side
// stand-in, not a device address).  The first call on a device does this
// look-up, so that first call should be made before any stream capture.
//
// Every call shares the one array and leaves its contents behind: the parts
// that must start at zero (radix histograms, tile counters, look-back flags)
// are cleared by each call on its stream, and calls whose work overlaps on the
// GPU (different streams, or different host threads) race on the array.
#include <mutex>

#include "common.cuh"

namespace gs {

void preprocess_parts(const gs_plan* plan, void* pre_ws, const ViewDev** views, ItemState* st,
                      const uint32_t** sorted_items, uint32_t** offsets, uint32_t** status, uint64_t** scan_blocks,
                      unsigned long long** n_entries);

namespace {

constexpr int64_t kMaxEntries = GS_NOALLOC_MAX_ENTRIES;
constexpr size_t kAltBytes = (size_t)kMaxEntries * 4;          // one alternate buffer
constexpr size_t kRadixBytes =
    ((4 * kRadix + 4) * 4 + 255) / 256 * 256 +                   // histograms + counters
    (size_t)4 * ((kMaxEntries + kSortTile - 1) / kSortTile) * kRadix * 4;   // look-back, 4 passes
constexpr size_t kScratchBytes = 2 * kAltBytes + kRadixBytes;
static_assert(kScratchBytes <= GS_NOALLOC_SCRATCH_BYTES, "scratch array too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[GS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_bin_sort_noalloc(const gs_plan* plan, void* pre_ws, uint32_t* tile_ids, uint32_t* items,
                                         uint32_t* ranges, void* stream_) {
  if (!plan || plan->n_views < 1 || plan->n_views > GS_MAX_VIEWS || plan->n_entries < 0 || !pre_ws || !ranges)
    return GS_ERR_INVALID_ARG;
  if (plan->n_entries > 0 && (!tile_ids || !items)) return GS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(tile_ids) | reinterpret_cast<uintptr_t>(items)) & 15) return GS_ERR_INVALID_ARG;
  if (plan->n_entries > kMaxEntries) return GS_ERR_CAPACITY;
  if (plan->sort_bits < 1 || plan->sort_bits > 32) return GS_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return GS_ERR_CUDA;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  uint32_t* keys_alt = reinterpret_cast<uint32_t*>(base);
  uint32_t* vals_alt = reinterpret_cast<uint32_t*>(base + kAltBytes);
  void* radix = base + 2 * kAltBytes;

  const ViewDev* views;
  ItemState st;
  const uint32_t* sorted_items;
  uint32_t *offsets, *status;
  uint64_t* scan_blocks;
  unsigned long long* n_entries;
  preprocess_parts(plan, pre_ws, &views, &st, &sorted_items, &offsets, &status, &scan_blocks, &n_entries);
  cudaError_t e = cudaSuccess;
  if (plan->n_entries > 0) {
    // the entry offsets of the depth order (the preprocess may have scanned
    // the band sizes instead, for the tile-list builder of gs_bin_sort)
    e = gather_exclusive_scan(st.tiles, sorted_items, offsets, plan->n_items, scan_blocks, n_entries, stream,
                              status);
    if (e == cudaSuccess)
      e = launch_duplicate(views, plan->n_views, plan->n_items, plan->n, sorted_items, offsets, st, tile_ids, items,
                         status, stream);
    // radix_sort_pairs clears the histogram, counter and look-back region first
    if (e == cudaSuccess)
      e = radix_sort_pairs(tile_ids, keys_alt, items, vals_alt, plan->n_entries, plan->sort_bits, radix, status,
                           stream, "tile");
  }
  if (e == cudaSuccess)
    e = launch_ranges(tile_ids, plan->n_entries, reinterpret_cast<uint2*>(ranges), plan->total_tiles, stream);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
