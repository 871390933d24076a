// C ABI of the rasterizer: plans, workspace layouts, argument validation and
// the launch sequences of gs_preprocess / gs_bin_sort / gs_render_fwd /
// gs_render_bwd.  Every device buffer is the caller's; the only allocation is
// one pinned, mapped 16-byte host word per host thread (first use, kept for
// the process) through which gs_preprocess reads its status and entry count.
// The calls sequence the steps of the paper's rasterizer (projection and SH
// colour, binning and sort, Sec. 3.1; blending, Eq. 1; the outputs of Sec. 3.2,
// 3.3 and 4.1); the plans, layouts and checks here have no counterpart in it.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace gs {
namespace {

// The per-view constants, handed to a kernel by value (so the upload takes
// no copy engine, whose queue may hold other streams' large transfers).
struct ViewTable {
  ViewDev v[GS_MAX_VIEWS];
};
static_assert(sizeof(ViewTable) <= 32000, "kernel parameters are limited to 32764 bytes");

// Writes the plan's views into the workspace and clears the status words.
__global__ void set_views_kernel(const ViewTable t, int n_views, ViewDev* __restrict__ dst,
                                 uint32_t* __restrict__ status) {
  const int i = threadIdx.x;
  if (i < n_views) dst[i] = t.v[i];
  if (i < 8) status[i] = 0u;
}

// Copies the status word, the entry count and the pair count (24 bytes) into
// mapped host memory: the read-back then needs only the stream
// synchronisation.
__global__ void copy_head_kernel(const uint64_t* __restrict__ src, volatile uint64_t* dst) {
  if (threadIdx.x < 3) dst[threadIdx.x] = src[threadIdx.x];
}

// bits[v][g / 32] bit g % 32 = (mask[v * n + g] != 0); one ballot per 32
// Gaussians (blockIdx.y = view), padding bits zero.
__global__ void pack_mask_kernel(const uint8_t* __restrict__ mask, int64_t n, uint32_t* __restrict__ bits,
                                 int64_t words) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = blockIdx.y;
  const bool keep = g < n && mask[v * n + g] != 0;
  const uint32_t b = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0 && (g >> 5) < words) bits[v * words + (g >> 5)] = b;
}

struct HostHead {
  volatile uint64_t* host = nullptr;   // pinned, mapped
  uint64_t* dev = nullptr;             // its device address
};

// This host thread's head word pair, allocated on first use.
cudaError_t host_head(HostHead** out) {
  thread_local HostHead hh;
  if (!hh.host) {
    void* p = nullptr;
    cudaError_t e = cudaHostAlloc(&p, 32, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e != cudaSuccess) return e;
    void* dp = nullptr;
    e = cudaHostGetDevicePointer(&dp, p, 0);
    if (e != cudaSuccess) {
      cudaFreeHost(p);
      return e;
    }
    hh.host = static_cast<volatile uint64_t*>(p);
    hh.dev = static_cast<uint64_t*>(dp);
  }
  *out = &hh;
  return cudaSuccess;
}

PreLayout pre_layout(const gs_plan& p) {
  PreLayout L;
  const size_t m = (size_t)std::max<int64_t>(p.n_items, 1);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  L.views = take(sizeof(ViewDev) * GS_MAX_VIEWS);
  L.status = take(32);          // status word (u32), n_entries (u64) at +8, n_pairs (u64) at +16
  L.n_entries = L.status + 8;
  L.xy_tau_z = take(16 * m);
  L.conic_o = take(16 * m);
  L.rgb = take(16 * m);
  L.depth_frame = take(48 * m);
  L.rect = take(8 * m);
  L.bin = take(32 * m);
  L.tiles = take(4 * m);
  L.band_rows = take(4 * m);
  L.depth_key = take(4 * m);
  L.sort_keys_alt = take(4 * m);
  L.sort_vals = take(4 * m);
  L.sort_vals_alt = take(4 * m);
  L.sorted_items = L.sort_vals;
  L.offsets = take(4 * m);
  L.pair_offsets = take(4 * m);
  L.scan_blocks = take(scan_block_bytes((int64_t)m));
  L.radix_scratch = take(radix_scratch_bytes((int64_t)m, 32));
  L.grad2d = take(36 * m);       // 2 x float4 per item, then 1 float per item
  L.total = o;
  return L;
}

// Global tile rows of the plan and the widest view (tiles across).
void plan_rows(const gs_plan& p, int* rows, int* max_tx) {
  int64_t r = 0;
  int mx = 0;
  for (int v = 0; v < p.n_views; ++v) {
    r += ceil_div(p.cams[v].height, kTile);
    mx = std::max(mx, ceil_div(p.cams[v].width, kTile));
  }
  *rows = (int)std::min<int64_t>(r, INT32_MAX);
  *max_tx = mx;
}

// Whether gs_bin_sort builds the tile lists by the pair sort (lists.cu):
// the global tile rows and the tiles across every view fit the pair key.
bool lists_path(const gs_plan& p) {
  int rows = 0, max_tx = 0;
  plan_rows(p, &rows, &max_tx);
  return rows <= kListRowsMax && max_tx <= kListTxMax;
}

SortLayout sort_layout(const gs_plan& p) {
  SortLayout L;
  memset(&L, 0, sizeof(L));
  const size_t e = (size_t)std::max<int64_t>(p.n_entries, 1);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  int rows = 0, max_tx = 0;
  plan_rows(p, &rows, &max_tx);
  L.lists = lists_path(p);
  L.vals = take(4 * e);
  L.ranges = take(8 * (size_t)std::max(p.total_tiles, 1));
  if (L.lists) {
    const size_t np = (size_t)std::max<int32_t>(p.n_pairs, 1);
    L.rows = rows;
    L.counts2_n = (int64_t)((np + kListPairsPerChunk - 1) / kListPairsPerChunk) * max_tx + std::max(p.total_tiles, 1);
    L.pkey = take(4 * np);
    L.pkey_alt = take(4 * np);
    L.pval = take(4 * np);
    L.pval_alt = take(4 * np);
    L.pair_radix = take(list_pair_radix_bytes((int64_t)np));
    L.row_T = take(4 * ((size_t)rows + 1));
    L.row_start = take(4 * ((size_t)rows + 1));
    L.c2_start = take(4 * ((size_t)rows + 1));
    L.cnt2_off = take(4 * ((size_t)rows + 1));
    L.counts2 = take(4 * (size_t)L.counts2_n);
    L.prefix2 = take(4 * (size_t)L.counts2_n);
    L.tile_count = take(4 * (size_t)std::max(p.total_tiles, 1));
    L.tile_start = take(4 * (size_t)std::max(p.total_tiles, 1));
    L.scan_blocks = take(scan_block_bytes(std::max(p.total_tiles, 1)) + 8);
    const size_t c2 = np / kListPairsPerChunk + (size_t)rows + 1;   // second-level chunks, at most
    L.chunks = take(16 * c2);
    L.chunk_cnt = take(4 * c2);
    L.tile_order = take(4 * (size_t)std::max(p.total_tiles, 1));
    L.tile_hist = take(4 * 2 * (size_t)kTileBuckets);
  } else {
    L.keys = take(4 * e);
    L.keys_alt = take(4 * e);
    L.vals_alt = take(4 * e);
    L.radix_scratch = take(radix_scratch_bytes((int64_t)e, std::max(p.sort_bits, 1)));
  }
  L.total = o;
  return L;
}

template <class T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}
template <class T>
const T* at(const void* base, size_t off) {
  return reinterpret_cast<const T*>(static_cast<const char*>(base) + off);
}

ItemState item_state(void* ws, const PreLayout& L) {
  ItemState s;
  s.xy_tau_z = at<float4>(ws, L.xy_tau_z);
  s.conic_o = at<float4>(ws, L.conic_o);
  s.rgb = at<float4>(ws, L.rgb);
  s.depth_frame = at<float4>(ws, L.depth_frame);
  s.rect = at<uint2>(ws, L.rect);
  s.bin = at<float4>(ws, L.bin);
  s.tiles = at<uint32_t>(ws, L.tiles);
  s.depth_key = at<uint32_t>(ws, L.depth_key);
  s.depth_val = at<uint32_t>(ws, L.sort_vals);
  s.status = at<uint32_t>(ws, L.status);
  s.n_entries = at<unsigned long long>(ws, L.n_entries);
  s.entries_acc = at<unsigned long long>(ws, L.n_entries);
  s.band_rows = at<uint32_t>(ws, L.band_rows);
  return s;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

gs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

bool valid_config(const gs_config* c) {
  return c && c->znear > 0.f && c->lowpass >= 0.f && c->clamp > 0.f && c->alpha_max > 0.f &&
         c->alpha_max < 1.f && c->alpha_min > 0.f && c->alpha_min < c->alpha_max && c->t_min > 0.f &&
         c->t_min < 1.f;
}

bool valid_scene(const gs_plan* p, const gs_scene* s) {
  if (!s || !s->means || !s->scales || !s->rotations || !s->opacities || !s->sh) return s && p->n == 0 && s->n == 0;
  if (s->n != p->n) return false;
  if (s->sh_degree < 0 || s->sh_degree > GS_MAX_SH_DEGREE) return false;
  if (s->sh_coeffs < (s->sh_degree + 1) * (s->sh_degree + 1)) return false;
  if (!aligned(s->rotations, 16) || !aligned(s->means, 4) || !aligned(s->scales, 4) || !aligned(s->sh, 4))
    return false;
  return true;
}

bool valid_plan(const gs_plan* p) {
  return p && p->n >= 0 && p->n_views >= 1 && p->n_views <= GS_MAX_VIEWS && p->n_items == p->n * p->n_views;
}

}  // namespace

// Pointers into a preprocess workspace for another translation unit.
void preprocess_parts(const gs_plan* plan, void* pre_ws, const ViewDev** views, ItemState* st,
                      const uint32_t** sorted_items, uint32_t** offsets, uint32_t** status, uint64_t** scan_blocks,
                      unsigned long long** n_entries) {
  const PreLayout L = pre_layout(*plan);
  *views = at<ViewDev>(pre_ws, L.views);
  *st = item_state(pre_ws, L);
  *sorted_items = at<uint32_t>(pre_ws, L.sorted_items);
  *offsets = at<uint32_t>(pre_ws, L.offsets);
  *status = at<uint32_t>(pre_ws, L.status);
  *scan_blocks = at<uint64_t>(pre_ws, L.scan_blocks);
  *n_entries = at<unsigned long long>(pre_ws, L.n_entries);
}

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace gs

using namespace gs;

extern "C" {

void gs_config_default(gs_config* c) {
  if (!c) return;
  c->znear = 0.2f;
  c->lowpass = 0.3f;
  c->clamp = 1.3f;
  c->alpha_max = 0.99f;
  c->alpha_min = 1.0f / 255.0f;
  c->t_min = 1e-4f;
  c->bg[0] = c->bg[1] = c->bg[2] = 0.f;
  c->flags = 0u;
}

gs_status gs_plan_init(gs_plan* plan, int64_t n, const gs_camera* cams, int32_t n_views) {
  if (!plan || !cams || n < 0 || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
  memset(plan, 0, sizeof(*plan));
  plan->n = n;
  plan->n_views = n_views;
  plan->n_items = n * n_views;
  if (plan->n_items >= (int64_t)1 << 30) return GS_ERR_INVALID_ARG;   // radix sort counts are 30-bit
  int64_t tiles = 0, pixels = 0;
  for (int v = 0; v < n_views; ++v) {
    const gs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 65535 * kTile || c.height > 65535 * kTile) return GS_ERR_INVALID_ARG;
    if (!(c.fx > 0.f) || !(c.fy > 0.f)) return GS_ERR_INVALID_ARG;
    plan->cams[v] = c;
    plan->tile_base[v] = (int32_t)tiles;
    plan->pixel_base[v] = pixels;
    tiles += (int64_t)ceil_div(c.width, kTile) * ceil_div(c.height, kTile);
    pixels += (int64_t)c.width * c.height;
    if (tiles >= ((int64_t)1 << 31)) return GS_ERR_INVALID_ARG;
  }
  plan->tile_base[n_views] = (int32_t)tiles;
  plan->pixel_base[n_views] = pixels;
  plan->total_tiles = (int32_t)tiles;
  plan->total_pixels = pixels;
  int bits = 1;
  while (((int64_t)1 << bits) < tiles) ++bits;
  plan->sort_bits = bits;
  plan->n_entries = -1;
  return GS_OK;
}

size_t gs_preprocess_workspace_size(const gs_plan* plan) {
  if (!valid_plan(plan)) return 0;
  return pre_layout(*plan).total;
}

size_t gs_bin_sort_workspace_size(const gs_plan* plan) {
  if (!valid_plan(plan) || plan->n_entries < 0) return 0;
  return sort_layout(*plan).total;
}

gs_status gs_preprocess(gs_plan* plan, const gs_scene* scene, const gs_config* cfg, const uint8_t* mask,
                        void* pre_ws, size_t pre_ws_bytes, void* stream_) {
  if (!valid_plan(plan) || !valid_config(cfg) || !valid_scene(plan, scene)) return GS_ERR_INVALID_ARG;
  if (!pre_ws || !aligned(pre_ws, 256)) return GS_ERR_INVALID_ARG;
  if (mask && (cfg->flags & GS_FLAG_MASK_BITS) && !aligned(mask, 4)) return GS_ERR_INVALID_ARG;
  const PreLayout L = pre_layout(*plan);
  if (pre_ws_bytes < L.total) return GS_ERR_CAPACITY;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);

  ViewTable table;
  memset(&table, 0, sizeof(table));
  ViewDev* views = table.v;
  int32_t row_base = 0;
  for (int v = 0; v < plan->n_views; ++v) {
    const gs_camera& c = plan->cams[v];
    ViewDev& V = views[v];
    memcpy(V.R, c.R, sizeof(V.R));
    memcpy(V.t, c.t, sizeof(V.t));
    V.fx = c.fx;
    V.fy = c.fy;
    V.cx = c.cx;
    V.cy = c.cy;
    V.limx = cfg->clamp * (0.5f * (float)c.width / c.fx);
    V.limy = cfg->clamp * (0.5f * (float)c.height / c.fy);
    for (int k = 0; k < 3; ++k) V.campos[k] = -(c.R[k] * c.t[0] + c.R[3 + k] * c.t[1] + c.R[6 + k] * c.t[2]);
    V.width = c.width;
    V.height = c.height;
    V.tiles_x = ceil_div(c.width, kTile);
    V.tiles_y = ceil_div(c.height, kTile);
    V.tile_base = plan->tile_base[v];
    V.row_base = row_base;
    row_base += V.tiles_y;
    V.pixel_base = plan->pixel_base[v];
  }
  HostHead* head = nullptr;
  cudaError_t e = host_head(&head);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  GS_TIMED("preprocess_views", stream,
           (set_views_kernel<<<1, GS_MAX_VIEWS, 0, stream>>>(table, plan->n_views, at<ViewDev>(pre_ws, L.views),
                                                              at<uint32_t>(pre_ws, L.status))));
  e = cudaGetLastError();
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if (plan->n_items == 0) {
    plan->n_entries = 0;
    plan->n_pairs = 0;
    return cuda_status(cudaStreamSynchronize(stream));
  }
  const ItemState st = item_state(pre_ws, L);
  uint32_t* status = at<uint32_t>(pre_ws, L.status);
  e = launch_preprocess(*scene, at<ViewDev>(pre_ws, L.views), plan->n_views, mask, *cfg, st, stream);
  if (e == cudaSuccess)
    e = radix_sort_pairs(st.depth_key, at<uint32_t>(pre_ws, L.sort_keys_alt), at<uint32_t>(pre_ws, L.sort_vals),
                         at<uint32_t>(pre_ws, L.sort_vals_alt), plan->n_items, 32,
                         at<void>(pre_ws, L.radix_scratch), status, stream, "depth");
  // the tile-list builder needs the band sizes scanned in depth order (pair
  // offsets, total n_pairs; the entry total comes from the preprocess's
  // sums); the radix path the tile counts (entry offsets and total)
  if (e == cudaSuccess) {
    if (lists_path(*plan))
      e = gather_exclusive_scan(st.band_rows, at<uint32_t>(pre_ws, L.sorted_items), at<uint32_t>(pre_ws, L.pair_offsets),
                                plan->n_items, at<uint64_t>(pre_ws, L.scan_blocks),
                                at<unsigned long long>(pre_ws, L.status + 16), stream, status);
    else
      e = gather_exclusive_scan(st.tiles, at<uint32_t>(pre_ws, L.sorted_items), at<uint32_t>(pre_ws, L.offsets),
                                plan->n_items, at<uint64_t>(pre_ws, L.scan_blocks),
                                at<unsigned long long>(pre_ws, L.n_entries), stream, status);
  }
  if (e != cudaSuccess) return GS_ERR_CUDA;
  GS_TIMED("preprocess_readback", stream,
           (copy_head_kernel<<<1, 32, 0, stream>>>(at<uint64_t>(pre_ws, L.status), head->dev)));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const uint64_t h0 = head->host[0], h1 = head->host[1], h2 = head->host[2];
  const uint32_t st_word = (uint32_t)(h0 & 0xffffffffu);
  if (st_word & kStatusTimeout) return GS_ERR_TIMEOUT;
  if (h1 >= ((uint64_t)1 << 30)) return GS_ERR_CAPACITY;    // entries beyond the sort's range
  if (h2 >= ((uint64_t)1 << 31)) return GS_ERR_CAPACITY;    // pairs beyond the lists' 32-bit indices
  plan->n_entries = (int64_t)h1;
  plan->n_pairs = (int32_t)h2;
  return GS_OK;
}

gs_status gs_bin_sort(const gs_plan* plan, void* pre_ws, void* sort_ws, size_t sort_ws_bytes, void* stream_) {
  if (!valid_plan(plan) || plan->n_entries < 0 || !pre_ws || !sort_ws || !aligned(sort_ws, 256))
    return GS_ERR_INVALID_ARG;
  const PreLayout L = pre_layout(*plan);
  const SortLayout S = sort_layout(*plan);
  if (sort_ws_bytes < S.total) return GS_ERR_CAPACITY;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const ItemState st = item_state(pre_ws, L);
  uint32_t* status = at<uint32_t>(pre_ws, L.status);
  uint32_t* keys = at<uint32_t>(sort_ws, S.keys);
  uint32_t* vals = at<uint32_t>(sort_ws, S.vals);
  cudaError_t e = cudaSuccess;
  if (S.lists) {
    // tile lists by counting placement (lists.cu)
    ListArgs a;
    a.views = at<ViewDev>(pre_ws, L.views);
    a.n_views = plan->n_views;
    a.n = plan->n;
    a.n_items = plan->n_items;
    a.n_entries = plan->n_entries;
    a.n_pairs = plan->n_pairs;
    a.rows = S.rows;
    a.total_tiles = plan->total_tiles;
    int rows = 0, max_tx = 0;
    plan_rows(*plan, &rows, &max_tx);
    a.max_tx = max_tx;
    a.counts2_n = S.counts2_n;
    a.sorted_items = at<uint32_t>(pre_ws, L.sorted_items);
    a.pair_offsets = at<uint32_t>(pre_ws, L.pair_offsets);
    a.st = st;
    a.vals = vals;
    a.ranges = at<uint2>(sort_ws, S.ranges);
    a.pkey = at<uint32_t>(sort_ws, S.pkey);
    a.pkey_alt = at<uint32_t>(sort_ws, S.pkey_alt);
    a.pval = at<uint32_t>(sort_ws, S.pval);
    a.pval_alt = at<uint32_t>(sort_ws, S.pval_alt);
    a.pair_radix = at<void>(sort_ws, S.pair_radix);
    a.counts2 = at<int32_t>(sort_ws, S.counts2);
    a.prefix2 = at<uint32_t>(sort_ws, S.prefix2);
    a.row_T = at<uint32_t>(sort_ws, S.row_T);
    a.row_start = at<uint32_t>(sort_ws, S.row_start);
    a.c2_start = at<uint32_t>(sort_ws, S.c2_start);
    a.cnt2_off = at<uint32_t>(sort_ws, S.cnt2_off);
    a.tile_count = at<uint32_t>(sort_ws, S.tile_count);
    a.tile_start = at<uint32_t>(sort_ws, S.tile_start);
    a.scan_blocks = at<uint64_t>(sort_ws, S.scan_blocks);
    a.chunks = at<int4>(sort_ws, S.chunks);
    a.chunk_cnt = at<uint32_t>(sort_ws, S.chunk_cnt);
    a.scan_total = at<unsigned long long>(sort_ws, S.scan_blocks + scan_block_bytes(std::max(plan->total_tiles, 1)));
    a.status = status;
    a.tile_order = at<uint32_t>(sort_ws, S.tile_order);
    a.tile_hist = at<uint32_t>(sort_ws, S.tile_hist);
    return cuda_status(launch_lists(a, stream));
  }
  if (plan->n_entries > 0) {
    e = launch_duplicate(at<ViewDev>(pre_ws, L.views), plan->n_views, plan->n_items, plan->n,
                         at<uint32_t>(pre_ws, L.sorted_items), at<uint32_t>(pre_ws, L.offsets), st, keys, vals,
                         status, stream);
    if (e == cudaSuccess)
      e = radix_sort_pairs(keys, at<uint32_t>(sort_ws, S.keys_alt), vals, at<uint32_t>(sort_ws, S.vals_alt),
                           plan->n_entries, plan->sort_bits, at<void>(sort_ws, S.radix_scratch), status, stream,
                           "tile");
  }
  if (e == cudaSuccess) e = launch_ranges(keys, plan->n_entries, at<uint2>(sort_ws, S.ranges), plan->total_tiles, stream);
  return cuda_status(e);
}

gs_status gs_render_fwd(const gs_plan* plan, const gs_config* cfg, void* pre_ws, const void* sort_ws,
                        const gs_fwd_outputs* out, void* stream_) {
  if (!valid_plan(plan) || !valid_config(cfg) || plan->n_entries < 0 || !pre_ws || !sort_ws || !out)
    return GS_ERR_INVALID_ARG;
  if (!out->image || !out->final_T || !out->n_contrib) return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(out->weight_sum_fixed) & 7u) return GS_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const PreLayout L = pre_layout(*plan);
  const SortLayout S = sort_layout(*plan);
  cudaError_t e = cudaSuccess;
  if (cfg->flags & GS_FLAG_ZERO_ACCUM) {
    if (out->weight_sum) e = cudaMemsetAsync(out->weight_sum, 0, 4 * (size_t)plan->n_items, stream);
    if (e == cudaSuccess && out->max_area) e = cudaMemsetAsync(out->max_area, 0, 4 * (size_t)plan->n_items, stream);
    if (e == cudaSuccess && out->weight_sum_fixed)
      e = cudaMemsetAsync(out->weight_sum_fixed, 0, 8 * (size_t)plan->n_items, stream);
    if (e != cudaSuccess) return GS_ERR_CUDA;
  }
  e = launch_render_fwd(at<ViewDev>(pre_ws, L.views), plan->n_views, plan->n, plan->total_tiles,
                        at<uint2>(sort_ws, S.ranges), at<uint32_t>(sort_ws, S.vals),
                        S.lists ? at<uint32_t>(sort_ws, S.tile_order) : nullptr, item_state(pre_ws, L), *cfg,
                        *out, stream);
  return cuda_status(e);
}

gs_status gs_render_bwd(const gs_plan* plan, const gs_scene* scene, const gs_config* cfg, void* pre_ws,
                        const void* sort_ws, const float* dL_dimage, const float* image,
                        const uint32_t* n_contrib, const gs_grads* g, void* stream_) {
  if (!valid_plan(plan) || !valid_config(cfg) || !valid_scene(plan, scene) || plan->n_entries < 0 || !pre_ws ||
      !sort_ws || !dL_dimage || !image || !n_contrib || !g)
    return GS_ERR_INVALID_ARG;
  if (!g->d_means || !g->d_scales || !g->d_rotations || !g->d_opacities || !g->d_sh) return GS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(g->weight_sum_fixed) & 7u) return GS_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const PreLayout L = pre_layout(*plan);
  const SortLayout S = sort_layout(*plan);
  const int64_t n = plan->n;
  cudaError_t e = cudaMemsetAsync(at<char>(pre_ws, L.grad2d), 0, 36 * (size_t)plan->n_items, stream);
  // with GS_FLAG_ZERO_ACCUM the preprocess backward writes every attribute
  // gradient row (no read-modify-write); I_i is accumulated by atomics
  if (e == cudaSuccess && (cfg->flags & GS_FLAG_ZERO_ACCUM) && g->weight_sum)
    e = cudaMemsetAsync(g->weight_sum, 0, 4 * (size_t)plan->n_items, stream);
  if (e == cudaSuccess && (cfg->flags & GS_FLAG_ZERO_ACCUM) && g->weight_sum_fixed)
    e = cudaMemsetAsync(g->weight_sum_fixed, 0, 8 * (size_t)plan->n_items, stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const ItemState st = item_state(pre_ws, L);
  float4* grad2d = at<float4>(pre_ws, L.grad2d);
  float* grad2d_b = reinterpret_cast<float*>(grad2d + 2 * plan->n_items);
  e = launch_render_bwd(at<ViewDev>(pre_ws, L.views), plan->n_views, n, plan->total_tiles,
                        at<uint2>(sort_ws, S.ranges), at<uint32_t>(sort_ws, S.vals), st, *cfg, dL_dimage, image,
                        n_contrib, grad2d, grad2d_b, g->weight_sum, g->weight_sum_fixed, stream);
  if (e == cudaSuccess)
    e = launch_preprocess_backward(*scene, at<ViewDev>(pre_ws, L.views), plan->n_views, *cfg, st.tiles, grad2d,
                                   grad2d_b, *g, stream);
  return cuda_status(e);
}

gs_status gs_loss_l1(const float* image, const float* target, int64_t count, float* loss, float* dL_dimage,
                     void* stream) {
  if (!image || !target || !loss || !dL_dimage || count < 0) return GS_ERR_INVALID_ARG;
  return cuda_status(launch_loss_l1(image, target, count, loss, dL_dimage, static_cast<cudaStream_t>(stream)));
}

gs_status gs_pack_mask(const uint8_t* mask, int64_t n, int32_t n_views, uint32_t* bits, void* stream_) {
  if (n < 0 || n_views < 1 || n_views > 65535 || (n > 0 && (!mask || !bits || !aligned(bits, 4))))
    return GS_ERR_INVALID_ARG;
  if (n == 0) return GS_OK;
  const int64_t words = (n + 31) / 32;
  const int64_t blocks = (words * 32 + 255) / 256;
  if (blocks > 0x7fffffff) return GS_ERR_INVALID_ARG;
  pack_mask_kernel<<<dim3((unsigned)blocks, (unsigned)n_views), 256, 0, static_cast<cudaStream_t>(stream_)>>>(
      mask, n, bits, words);
  return cuda_status(cudaGetLastError());
}

gs_status gs_device_status(const gs_plan* plan, void* pre_ws, void* stream_) {
  if (!valid_plan(plan) || !pre_ws) return GS_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const PreLayout L = pre_layout(*plan);
  uint32_t word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, at<char>(pre_ws, L.status), 4, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(at<char>(pre_ws, L.status), 0, 4, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if (word & kStatusTimeout) return GS_ERR_TIMEOUT;
  if (word & (kStatusEntryMismatch | kStatusBounds)) return GS_ERR_DEVICE_CHECK;
  return GS_OK;
}

gs_status gs_selftest_wait_timeout(void* scratch, size_t scratch_bytes, void* stream_) {
  if (!scratch || scratch_bytes < GS_SELFTEST_SCRATCH_BYTES || (reinterpret_cast<uintptr_t>(scratch) & 15))
    return GS_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  // [0, 3 kRadix) words: the sort's probe; then one status word per probe;
  // from byte 3200: the scan's probe
  static_assert(3 * kRadix * 4 + 8 <= 3200 && 3200 + 3 * 8 <= GS_SELFTEST_SCRATCH_BYTES, "self-test scratch layout");
  uint32_t* words = static_cast<uint32_t*>(scratch);
  uint32_t* status = words + 3 * kRadix;
  uint64_t* scan_words = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + 3200);
  uint32_t word[2] = {0u, 0u};
  cudaError_t e = cudaMemsetAsync(status, 0, 8, stream);
  if (e == cudaSuccess) e = lookback_timeout_probe(words, status, stream);
  if (e == cudaSuccess) e = scan_timeout_probe(scan_words, status + 1, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(word, status, 8, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  return ((word[0] & kStatusTimeout) && (word[1] & kStatusTimeout)) ? GS_ERR_TIMEOUT : GS_OK;
}

gs_status gs_inspect_preprocess(const gs_plan* plan, const void* pre_ws, gs_preprocess_view* out) {
  if (!valid_plan(plan) || !pre_ws || !out) return GS_ERR_INVALID_ARG;
  const PreLayout L = pre_layout(*plan);
  out->xy_tau_z = at<float>(pre_ws, L.xy_tau_z);
  out->conic_o = at<float>(pre_ws, L.conic_o);
  out->rgb = at<float>(pre_ws, L.rgb);
  out->tiles = at<uint32_t>(pre_ws, L.tiles);
  out->rect = at<uint32_t>(pre_ws, L.rect);
  out->sorted_items = at<uint32_t>(pre_ws, L.sorted_items);
  out->offsets = at<uint32_t>(pre_ws, L.offsets);
  out->pair_offsets = at<uint32_t>(pre_ws, L.pair_offsets);
  return GS_OK;
}

gs_status gs_inspect_sort(const gs_plan* plan, const void* sort_ws, gs_sort_view* out) {
  if (!valid_plan(plan) || plan->n_entries < 0 || !sort_ws || !out) return GS_ERR_INVALID_ARG;
  const SortLayout S = sort_layout(*plan);
  out->tile_ids = S.lists ? nullptr : at<uint32_t>(sort_ws, S.keys);   // the lists path stores no tile ids
  out->items = at<uint32_t>(sort_ws, S.vals);
  out->ranges = at<uint32_t>(sort_ws, S.ranges);
  return GS_OK;
}

const char* gs_status_string(gs_status s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CAPACITY: return "workspace too small";
    case GS_ERR_CUDA: return "CUDA runtime error";
    case GS_ERR_TIMEOUT: return "device wait exceeded its budget";
    case GS_ERR_DEVICE_CHECK: return "device consistency check failed";
  }
  return "unknown status";
}

size_t gs_sizeof_plan(void) { return sizeof(gs_plan); }
size_t gs_sizeof_camera(void) { return sizeof(gs_camera); }
size_t gs_sizeof_config(void) { return sizeof(gs_config); }
size_t gs_sizeof_scene(void) { return sizeof(gs_scene); }

}  // extern "C"
