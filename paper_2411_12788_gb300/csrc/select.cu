// Selections of Gaussians from the rasterizer's per-Gaussian statistics.
//
// * Importance pruning (MSv2-D, Sec. 6.1): keep the k Gaussians with the
//   largest accumulated blending weight I_i (Sec. 3.2), ties to the lower
//   index, listed in ascending index order; and the gather of their rows into
//   a compact scene for the re-render.
// * Identification, per view (gs_identify): blur-split candidates G^blur
//   (S_i > theta_blur H W, Sec. 4.1), intersected Gaussians G^int (S_i > 0,
//   Sec. 4.3), visibility V_i (I_i above the keep-quantile threshold,
//   Sec. 5.2) and critical Gaussians G^crit (the i_max of pixels whose w_max
//   is above the keep-quantile threshold, Sec. 5.1).  A keep quantile q over
//   the M positive values keeps the ceil(q M) largest, ties to the lower
//   index (the same rule as the pruning); K is computed on the device.
//
// * Primitive sampling (Sec. 4.3): k Gaussians drawn without replacement
//   with probabilities proportional to I_i, by exponential clocks (the
//   method of Efraimidis and Spirakis): with E_i ~ Exp(1) supplied by the
//   caller, keep the k largest I_i / E_i.
// * Depth reinitialization (Sec. 4.2): k pixels of a view drawn uniformly
//   without replacement among those with a maximum contributor and a
//   positive d^mid (the k largest of the caller's uniform draws), their
//   depth reprojected to world points and coloured from the target image.
//
// * Aggressive clone (Sec. 5.1): each listed Gaussian becomes two at the same
//   centre with opacity 1 - sqrt(1 - o) and covariance scaled by
//   o^2 (2 o' - o'^2 / sqrt 2)^-2 (scales by its square root).
//
// Selection is an MSD radix select on the bit patterns of the (non-negative)
// values, which order like the values: four passes each histogram the next
// 8 bits of the keys that still match the prefix found so far, and a single
// block picks the bucket holding the k-th largest.  That yields the exact
// threshold key t, the number of keys above it and how many keys equal to t
// are still needed.  A scan then ranks the keys equal to t in index order,
// which settles every key: kept iff key > t, or key == t with tie rank below
// the number still needed.
#include "common.cuh"

namespace gs {

namespace {

constexpr int kSelThreads = 256;

struct SelectState {
  uint32_t prefix;     // bits of t found so far
  uint32_t mask;       // which bits of the prefix are set
  uint32_t k_rem;      // how many of the keys matching the prefix are still wanted
  uint32_t n_above;    // keys above the prefix's range (kept for sure)
};

__global__ void __launch_bounds__(kSelThreads) select_hist_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                                  int shift, const SelectState* __restrict__ st,
                                                                  uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t prefix = st->prefix, mask = st->mask;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    if ((k & mask) == prefix) atomicAdd(&sh[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

// One block: the bucket b holding the k_rem-th largest key among those that
// match the prefix; keys in higher buckets are kept, b joins the prefix.
__global__ void __launch_bounds__(256) select_pick_kernel(uint32_t* __restrict__ hist, int shift,
                                                          SelectState* __restrict__ st) {
  __shared__ uint32_t suffix[257];
  const int b = threadIdx.x;
  const uint32_t c = hist[b];
  suffix[b] = c;
  if (b == 0) suffix[256] = 0;
  __syncthreads();
  // inclusive suffix sums: suffix[b] = sum_{j >= b} hist[j]
  for (int off = 1; off < 256; off <<= 1) {
    const uint32_t t = b + off < 256 ? suffix[b + off] : 0u;
    __syncthreads();
    suffix[b] += t;
    __syncthreads();
  }
  const uint32_t k = st->k_rem;
  const uint32_t above = suffix[b] - c;          // keys in buckets > b
  __syncthreads();
  if (c > 0 && above < k && above + c >= k) {    // exactly one bucket satisfies this
    st->prefix |= (uint32_t)b << shift;
    st->mask |= 255u << shift;
    st->k_rem = k - above;
    st->n_above += above;
  }
  hist[b] = 0;
}

__global__ void tie_flags_kernel(const uint32_t* __restrict__ keys, int64_t n, const SelectState* __restrict__ st,
                                 uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = keys[i] == st->prefix ? 1u : 0u;
}

// keep[i] = key > t, or key == t among the first k_rem such keys
__global__ void keep_flags_kernel(const uint32_t* __restrict__ keys, int64_t n, const SelectState* __restrict__ st,
                                  const uint32_t* __restrict__ tie_rank, uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t k = keys[i], t = st->prefix;
  flag[i] = (st->k_rem > 0 && (k > t || (k == t && tie_rank[i] < st->k_rem))) ? 1u : 0u;
}

__global__ void scatter_kept_kernel(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos, int64_t n,
                                    uint32_t* __restrict__ keep_idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && flag[i]) keep_idx[pos[i]] = (uint32_t)i;
}

__global__ void iota_u32_kernel(uint32_t* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)i;
}

// dst row r <- src row idx[r] for a [*, width] float array (width floats per row)
__global__ void gather_rows_kernel(const float* __restrict__ src, const uint32_t* __restrict__ idx, int64_t k,
                                   int width, float* __restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * width) return;
  const int64_t r = t / width;
  const int c = (int)(t - r * width);
  dst[t] = src[(int64_t)idx[r] * width + c];
}

// keys > 0 (as unsigned bit patterns: non-negative floats other than +0)
__global__ void __launch_bounds__(256) count_positive_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                             uint32_t* __restrict__ count) {
  uint32_t c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += keys[i] != 0u ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// k = ceil(q M) for the M positive keys (q in [0, 1]); the product is formed
// in double, exact for M < 2^29.
__global__ void select_init_kernel(SelectState* st, const uint32_t* __restrict__ count, float q) {
  const uint32_t m = *count;
  uint32_t k = (uint32_t)ceil((double)q * (double)m);
  if (k > m) k = m;
  *st = SelectState{0u, 0u, k, 0u};
}

__device__ __forceinline__ bool select_kept(uint32_t key, const SelectState& st, uint32_t tie_rank) {
  return st.k_rem > 0 && (key > st.prefix || (key == st.prefix && tie_rank < st.k_rem));
}

// Identification flags that are elementwise in S_i: G^blur (S_i >= s_min of
// the item's view, s_min = floor(theta H W) + 1, i.e. S_i > theta H W) and
// G^int (S_i > 0).  Overwrites flags.
struct BlurThresholds {
  uint32_t s_min[GS_MAX_VIEWS];
};

__global__ void __launch_bounds__(256) identify_area_kernel(const uint32_t* __restrict__ max_area, int64_t n,
                                                            int n_views, BlurThresholds th, uint8_t* __restrict__ flags,
                                                            uint32_t* __restrict__ counts) {
  const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n_items = n * n_views;
  uint32_t f = 0;
  int v = 0;
  if (item < n_items) {
    v = (int)(item / n);
    const uint32_t s = max_area[item];
    f = (s >= th.s_min[v] ? GS_ID_BLUR : 0u) | (s > 0u ? GS_ID_INTERSECT : 0u);
    flags[item] = (uint8_t)f;
  }
  if (counts) {
    const int v0 = __shfl_sync(0xffffffffu, v, 0);
    if (__all_sync(0xffffffffu, v == v0)) {
      const uint32_t cb = __reduce_add_sync(0xffffffffu, (f & GS_ID_BLUR) ? 1u : 0u);
      const uint32_t ci = __reduce_add_sync(0xffffffffu, (f & GS_ID_INTERSECT) ? 1u : 0u);
      if ((threadIdx.x & 31) == 0) {
        if (cb) atomicAdd(&counts[4 * v0 + 0], cb);
        if (ci) atomicAdd(&counts[4 * v0 + 1], ci);
      }
    } else {
      if (f & GS_ID_BLUR) atomicAdd(&counts[4 * v + 0], 1u);
      if (f & GS_ID_INTERSECT) atomicAdd(&counts[4 * v + 1], 1u);
    }
  }
}

// V_i: the view's selection over I (keys of that view's items).
__global__ void __launch_bounds__(256) identify_visible_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                               const SelectState* __restrict__ st,
                                                               const uint32_t* __restrict__ tie_rank,
                                                               uint8_t* __restrict__ flags,
                                                               uint8_t* __restrict__ visible_mask,
                                                               uint32_t* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  if (i < n) {
    const SelectState s = *st;
    keep = select_kept(keys[i], s, tie_rank[i]);
    if (keep) flags[i] |= (uint8_t)GS_ID_VISIBLE;
    if (visible_mask) visible_mask[i] = keep ? 1 : 0;
  }
  if (count) {
    const uint32_t c = __reduce_add_sync(0xffffffffu, keep ? 1u : 0u);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
  }
}

// G^crit: the i_max of every kept pixel (the view's selection over w_max).
// flags is addressed in 32-bit words (4-byte aligned base) so that pixels
// sharing an i_max set the bit with one atomic OR; the first setter counts.
__global__ void __launch_bounds__(256) identify_critical_kernel(const uint32_t* __restrict__ wmax_keys,
                                                                const int32_t* __restrict__ imax, int64_t n_pix,
                                                                const SelectState* __restrict__ st,
                                                                const uint32_t* __restrict__ tie_rank,
                                                                int64_t item_base, uint8_t* __restrict__ flags,
                                                                uint32_t* __restrict__ count) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  const SelectState s = *st;
  if (!select_kept(wmax_keys[p], s, tie_rank[p])) return;
  const int32_t g = imax[p];
  if (g < 0) return;
  const int64_t item = item_base + g;
  uint32_t* word = reinterpret_cast<uint32_t*>(flags + (item & ~(int64_t)3));
  const uint32_t bit = GS_ID_CRITICAL << (8 * (int)(item & 3));
  const uint32_t old = atomicOr(word, bit);
  if (count && !(old & bit)) atomicAdd(count, 1u);
}

// key_i = I_i / E_i (IEEE division), 0 where I_i is 0
__global__ void sampling_keys_kernel(const float* __restrict__ importance, const float* __restrict__ expo, int64_t n,
                                     float* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = __fdiv_rn(importance[i], expo[i]);
}

// key = u for pixels with a maximum contributor and d^mid > 0, else 0
__global__ void depth_point_keys_kernel(const float* __restrict__ depth, const int32_t* __restrict__ imax,
                                        const float* __restrict__ u, int64_t n, float* __restrict__ keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) keys[i] = (imax[i] >= 0 && depth[i] > 0.f) ? u[i] : 0.f;
}

// K = min(k, #positive keys)
__global__ void select_init_count_kernel(SelectState* st, const uint32_t* __restrict__ count, int64_t k,
                                         uint32_t* __restrict__ k_out) {
  const uint32_t m = *count;
  const uint32_t kk = (uint32_t)((int64_t)m < k ? (int64_t)m : k);
  *st = SelectState{0u, 0u, kk, 0u};
  if (k_out) *k_out = kk;
}

// Reprojection of the kept pixels: p_c = d ((x + 0.5 - cx) / fx,
// (y + 0.5 - cy) / fy, 1), world point R^T (p_c - t); colour from the
// view's planar target image.
struct CamDev {
  float R[9], t[3], fx, fy, cx, cy;
  int width, height;
};

__global__ void depth_points_kernel(const uint32_t* __restrict__ idx, const uint32_t* __restrict__ k_dev,
                                    const float* __restrict__ depth, const float* __restrict__ image, CamDev cam,
                                    float* __restrict__ points, float* __restrict__ colours) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= (int64_t)*k_dev) return;
  const uint32_t p = idx[r];
  const int x = (int)(p % (uint32_t)cam.width), y = (int)(p / (uint32_t)cam.width);
  const float d = depth[p];
  const float cx = d * (((float)x + 0.5f - cam.cx) / cam.fx);
  const float cy = d * (((float)y + 0.5f - cam.cy) / cam.fy);
  const float a = cx - cam.t[0], b = cy - cam.t[1], c = d - cam.t[2];
  points[3 * r + 0] = cam.R[0] * a + cam.R[3] * b + cam.R[6] * c;
  points[3 * r + 1] = cam.R[1] * a + cam.R[4] * b + cam.R[7] * c;
  points[3 * r + 2] = cam.R[2] * a + cam.R[5] * b + cam.R[8] * c;
  const int64_t hw = (int64_t)cam.width * cam.height;
  colours[3 * r + 0] = image[p];
  colours[3 * r + 1] = image[hw + p];
  colours[3 * r + 2] = image[2 * hw + p];
}

struct SelectLayout {
  size_t state, hist, count, k_dev, flag, rank, pos, keys, scan_blocks, total_dev, total;
};

SelectLayout select_layout(int64_t n) {
  SelectLayout L;
  const size_t m = (size_t)(n > 0 ? n : 1);
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o = align_up(o + b);
    return at;
  };
  L.state = take(sizeof(SelectState));
  L.hist = take(256 * 4);
  L.count = take(4);
  L.k_dev = take(4);
  L.total_dev = take(8);
  L.flag = take(4 * m);
  L.rank = take(4 * m);
  L.pos = take(4 * m);
  L.keys = take(4 * m);
  L.scan_blocks = take(scan_block_bytes((int64_t)m));
  L.total = o;
  return L;
}

struct SelectBufs {
  SelectState* st;
  uint32_t* hist;
  uint32_t* count;
  uint32_t* k_dev;
  float* keys;
  uint32_t* flag;
  uint32_t* rank;
  uint32_t* pos;
  uint64_t* sb;
  unsigned long long* tot;
};

SelectBufs select_bufs(void* ws, const SelectLayout& L) {
  char* base = static_cast<char*>(ws);
  return SelectBufs{reinterpret_cast<SelectState*>(base + L.state), reinterpret_cast<uint32_t*>(base + L.hist),
                    reinterpret_cast<uint32_t*>(base + L.count),     reinterpret_cast<uint32_t*>(base + L.k_dev),
                    reinterpret_cast<float*>(base + L.keys),         reinterpret_cast<uint32_t*>(base + L.flag),
                    reinterpret_cast<uint32_t*>(base + L.rank),      reinterpret_cast<uint32_t*>(base + L.pos),
                    reinterpret_cast<uint64_t*>(base + L.scan_blocks),
                    reinterpret_cast<unsigned long long*>(base + L.total_dev)};
}

// With B.st initialised (k_rem set), finds the threshold key t and writes the
// tie ranks (exclusive count of earlier keys equal to t) to B.rank.
cudaError_t select_threshold(const uint32_t* keys, int64_t n, const SelectBufs& B, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(B.hist, 0, 256 * 4, stream);
  if (e != cudaSuccess) return e;
  const int blocks = ceil_div(n, 256);
  const int hb = std::min(blocks, 4 * device_sm_count());
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    GS_TIMED("select_hist", stream, (select_hist_kernel<<<hb, kSelThreads, 0, stream>>>(keys, n, shift, B.st, B.hist)));
    GS_TIMED("select_pick", stream, (select_pick_kernel<<<1, 256, 0, stream>>>(B.hist, shift, B.st)));
  }
  GS_TIMED("select_ties", stream, (tie_flags_kernel<<<blocks, 256, 0, stream>>>(keys, n, B.st, B.flag)));
  e = cudaGetLastError();
  if (e == cudaSuccess) e = gather_exclusive_scan(B.flag, nullptr, B.rank, n, B.sb, B.tot, stream);
  return e;
}

// keep_idx[0..K) <- the kept indices in ascending order (after select_threshold).
cudaError_t select_compact(const uint32_t* keys, int64_t n, const SelectBufs& B, uint32_t* keep_idx,
                           cudaStream_t stream) {
  const int blocks = ceil_div(n, 256);
  GS_TIMED("select_keep", stream, (keep_flags_kernel<<<blocks, 256, 0, stream>>>(keys, n, B.st, B.rank, B.flag)));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = gather_exclusive_scan(B.flag, nullptr, B.pos, n, B.sb, B.tot, stream);
  if (e == cudaSuccess)
    GS_TIMED("select_scatter", stream, (scatter_kept_kernel<<<blocks, 256, 0, stream>>>(B.flag, B.pos, n, keep_idx)));
  return cudaGetLastError();
}

// B.st <- K = min(k, #(keys > 0)), also written to B.k_dev.
cudaError_t select_init_count(const uint32_t* keys, int64_t n, int64_t k, const SelectBufs& B, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(B.count, 0, 4, stream);
  if (e != cudaSuccess) return e;
  GS_TIMED("select_count", stream,
           (count_positive_kernel<<<std::max(1, std::min(ceil_div(n, 256), 4 * device_sm_count())), 256, 0, stream>>>(keys, n,
                                                                                                        B.count)));
  GS_TIMED("select_init", stream, (select_init_count_kernel<<<1, 1, 0, stream>>>(B.st, B.count, k, B.k_dev)));
  return cudaGetLastError();
}

// B.st <- k = ceil(q * #(keys > 0)).
cudaError_t select_init_quantile(const uint32_t* keys, int64_t n, float q, const SelectBufs& B, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(B.count, 0, 4, stream);
  if (e != cudaSuccess) return e;
  GS_TIMED("select_count", stream,
           (count_positive_kernel<<<std::max(1, std::min(ceil_div(n, 256), 4 * device_sm_count())), 256, 0, stream>>>(keys, n,
                                                                                                        B.count)));
  GS_TIMED("select_init", stream, (select_init_kernel<<<1, 1, 0, stream>>>(B.st, B.count, q)));
  return cudaGetLastError();
}

}  // namespace

}  // namespace gs

using namespace gs;

extern "C" size_t gs_prune_workspace_size(int64_t n) { return n < 0 ? 0 : select_layout(n).total; }

extern "C" gs_status gs_prune_select(const float* importance, int64_t n, int64_t k, uint32_t* keep_idx, void* ws,
                                     size_t ws_bytes, void* stream_) {
  if (n < 0 || k < 0 || k > n || n >= ((int64_t)1 << 32) || (n > 0 && !importance) || (k > 0 && !keep_idx) || !ws ||
      (reinterpret_cast<uintptr_t>(ws) & 255))
    return GS_ERR_INVALID_ARG;
  const SelectLayout L = select_layout(n);
  if (ws_bytes < L.total) return GS_ERR_CAPACITY;
  if (k == 0) return GS_OK;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int blocks = ceil_div(n, 256);
  if (k == n) {
    GS_TIMED("prune_iota", stream, (iota_u32_kernel<<<blocks, 256, 0, stream>>>(keep_idx, n)));
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  }
  const uint32_t* keys = reinterpret_cast<const uint32_t*>(importance);
  const SelectBufs B = select_bufs(ws, L);
  SelectState init{0u, 0u, (uint32_t)k, 0u};
  cudaError_t e = cudaMemcpyAsync(B.st, &init, sizeof(init), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = select_threshold(keys, n, B, stream);
  if (e == cudaSuccess) {
    GS_TIMED("prune_flags", stream, (keep_flags_kernel<<<blocks, 256, 0, stream>>>(keys, n, B.st, B.rank, B.flag)));
    e = gather_exclusive_scan(B.flag, nullptr, B.pos, n, B.sb, B.tot, stream);
  }
  if (e == cudaSuccess)
    GS_TIMED("prune_scatter", stream, (scatter_kept_kernel<<<blocks, 256, 0, stream>>>(B.flag, B.pos, n, keep_idx)));
  e = cudaGetLastError();
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

static int64_t identify_elements(const gs_plan* plan) {
  int64_t m = plan->n;
  for (int v = 0; v < plan->n_views; ++v) m = std::max(m, plan->pixel_base[v + 1] - plan->pixel_base[v]);
  return m;
}

extern "C" size_t gs_identify_workspace_size(const gs_plan* plan) {
  if (!plan || plan->n < 0 || plan->n_views < 1 || plan->n_views > GS_MAX_VIEWS) return 0;
  return select_layout(identify_elements(plan)).total;
}

extern "C" void gs_config_identify_default(gs_config_identify* out) {
  if (!out) return;
  out->theta_blur = 2e-4f;
  out->keep_visible = 0.99f;
  out->keep_critical = 0.99f;
}

extern "C" gs_status gs_identify(const gs_plan* plan, const gs_config_identify* cfg, const float* weight_sum,
                                 const uint32_t* max_area, const int32_t* imax, const float* wmax, uint8_t* flags,
                                 uint8_t* visible_mask, uint32_t* counts, void* ws, size_t ws_bytes, void* stream_) {
  if (!plan || !cfg || plan->n < 0 || plan->n_views < 1 || plan->n_views > GS_MAX_VIEWS || !ws ||
      (reinterpret_cast<uintptr_t>(ws) & 255))
    return GS_ERR_INVALID_ARG;
  if (!(cfg->theta_blur >= 0.f) || !(cfg->keep_visible >= 0.f && cfg->keep_visible <= 1.f) ||
      !(cfg->keep_critical >= 0.f && cfg->keep_critical <= 1.f))
    return GS_ERR_INVALID_ARG;
  const int64_t n = plan->n, n_items = plan->n_items;
  if (n_items != n * plan->n_views || n_items >= ((int64_t)1 << 32)) return GS_ERR_INVALID_ARG;
  if (n_items > 0 && (!weight_sum || !max_area || !flags || (reinterpret_cast<uintptr_t>(flags) & 3)))
    return GS_ERR_INVALID_ARG;
  if (plan->total_pixels > 0 && (!imax || !wmax)) return GS_ERR_INVALID_ARG;
  const SelectLayout L = select_layout(identify_elements(plan));
  if (ws_bytes < L.total) return GS_ERR_CAPACITY;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  cudaError_t e = cudaSuccess;
  if (counts) e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * 4 * plan->n_views, stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  if (n == 0) return GS_OK;
  BlurThresholds th{};
  for (int v = 0; v < plan->n_views; ++v) {
    const double hw = (double)plan->cams[v].width * (double)plan->cams[v].height;
    th.s_min[v] = (uint32_t)std::min(floor((double)cfg->theta_blur * hw) + 1.0, 4294967295.0);
  }
  GS_TIMED("identify_area", stream,
           (identify_area_kernel<<<ceil_div(n_items, 256), 256, 0, stream>>>(max_area, n, plan->n_views, th, flags,
                                                                              counts)));
  e = cudaGetLastError();
  const SelectBufs B = select_bufs(ws, L);
  for (int v = 0; v < plan->n_views && e == cudaSuccess; ++v) {
    // V_i over the view's I
    const uint32_t* keys = reinterpret_cast<const uint32_t*>(weight_sum) + v * n;
    e = select_init_quantile(keys, n, cfg->keep_visible, B, stream);
    if (e == cudaSuccess) e = select_threshold(keys, n, B, stream);
    if (e != cudaSuccess) break;
    GS_TIMED("identify_visible", stream,
             (identify_visible_kernel<<<ceil_div(n, 256), 256, 0, stream>>>(
                 keys, n, B.st, B.rank, flags + v * n, visible_mask ? visible_mask + v * n : nullptr,
                 counts ? counts + 4 * v + 2 : nullptr)));
    e = cudaGetLastError();
    // G^crit over the view's w_max
    const int64_t p0 = plan->pixel_base[v], np = plan->pixel_base[v + 1] - p0;
    if (e != cudaSuccess || np == 0) continue;
    const uint32_t* wk = reinterpret_cast<const uint32_t*>(wmax) + p0;
    e = select_init_quantile(wk, np, cfg->keep_critical, B, stream);
    if (e == cudaSuccess) e = select_threshold(wk, np, B, stream);
    if (e != cudaSuccess) break;
    GS_TIMED("identify_critical", stream,
             (identify_critical_kernel<<<ceil_div(np, 256), 256, 0, stream>>>(
                 wk, imax + p0, np, B.st, B.rank, v * n, flags, counts ? counts + 4 * v + 3 : nullptr)));
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" gs_status gs_gather_scene(const gs_scene* src, const uint32_t* idx, int64_t k, const gs_scene_buf* dst,
                                     void* stream_) {
  if (!src || !dst || k < 0 || k > dst->n || (k > 0 && !idx)) return GS_ERR_INVALID_ARG;
  if (src->sh_coeffs != dst->sh_coeffs || !src->means || !dst->means || !src->scales || !dst->scales ||
      !src->rotations || !dst->rotations || !src->opacities || !dst->opacities || !src->sh || !dst->sh)
    return GS_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  if (k == 0) return GS_OK;
  struct Part {
    const float* s;
    float* d;
    int w;
  } parts[5] = {{src->means, dst->means, 3},
                {src->scales, dst->scales, 3},
                {src->rotations, dst->rotations, 4},
                {src->opacities, dst->opacities, 1},
                {src->sh, dst->sh, 3 * src->sh_coeffs}};
  for (const Part& p : parts) {
    const int64_t total = k * p.w;
    GS_TIMED("gather_scene", stream,
             (gather_rows_kernel<<<ceil_div(total, 256), 256, 0, stream>>>(p.s, idx, k, p.w, p.d)));
  }
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" size_t gs_sample_workspace_size(int64_t n) { return n < 0 ? 0 : select_layout(n).total; }

extern "C" gs_status gs_sample_gaussians(const float* importance, const float* expo, int64_t n, int64_t k,
                                         uint32_t* keep_idx, uint32_t* k_out, void* ws, size_t ws_bytes,
                                         void* stream_) {
  if (n < 0 || k < 0 || n >= ((int64_t)1 << 32) || (n > 0 && (!importance || !expo)) || (k > 0 && !keep_idx) ||
      !ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return GS_ERR_INVALID_ARG;
  const SelectLayout L = select_layout(n);
  if (ws_bytes < L.total) return GS_ERR_CAPACITY;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const SelectBufs B = select_bufs(ws, L);
  cudaError_t e = cudaSuccess;
  if (n == 0 || k == 0) {
    if (k_out) e = cudaMemsetAsync(k_out, 0, 4, stream);
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  }
  GS_TIMED("sample_keys", stream,
           (sampling_keys_kernel<<<ceil_div(n, 256), 256, 0, stream>>>(importance, expo, n, B.keys)));
  const uint32_t* keys = reinterpret_cast<const uint32_t*>(B.keys);
  e = select_init_count(keys, n, k, B, stream);
  if (e == cudaSuccess) e = select_threshold(keys, n, B, stream);
  if (e == cudaSuccess) e = select_compact(keys, n, B, keep_idx, stream);
  if (e == cudaSuccess && k_out) e = cudaMemcpyAsync(k_out, B.k_dev, 4, cudaMemcpyDeviceToDevice, stream);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

extern "C" size_t gs_depth_points_workspace_size(const gs_plan* plan) {
  if (!plan || plan->n_views < 1 || plan->n_views > GS_MAX_VIEWS) return 0;
  int64_t m = 1;
  for (int v = 0; v < plan->n_views; ++v) m = std::max(m, plan->pixel_base[v + 1] - plan->pixel_base[v]);
  return select_layout(m).total;
}

extern "C" gs_status gs_depth_points(const gs_plan* plan, int32_t view, const float* depth, const int32_t* imax,
                                     const float* target, const float* u, int64_t k, float* points, float* colours,
                                     uint32_t* pixel_idx, uint32_t* k_out, void* ws, size_t ws_bytes,
                                     void* stream_) {
  if (!plan || view < 0 || view >= plan->n_views || plan->n_views > GS_MAX_VIEWS || k < 0 || !ws ||
      (reinterpret_cast<uintptr_t>(ws) & 255))
    return GS_ERR_INVALID_ARG;
  const int64_t p0 = plan->pixel_base[view], np = plan->pixel_base[view + 1] - p0;
  if (np >= ((int64_t)1 << 32)) return GS_ERR_INVALID_ARG;
  if (np > 0 && (!depth || !imax || !target || !u)) return GS_ERR_INVALID_ARG;
  if (k > 0 && (!points || !colours || !pixel_idx)) return GS_ERR_INVALID_ARG;
  const SelectLayout L = select_layout(std::max<int64_t>(np, 1));
  if (ws_bytes < L.total) return GS_ERR_CAPACITY;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  cudaError_t e = cudaSuccess;
  if (np == 0 || k == 0) {
    if (k_out) e = cudaMemsetAsync(k_out, 0, 4, stream);
    return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  }
  const SelectBufs B = select_bufs(ws, L);
  GS_TIMED("depth_point_keys", stream,
           (depth_point_keys_kernel<<<ceil_div(np, 256), 256, 0, stream>>>(depth + p0, imax + p0, u, np, B.keys)));
  const uint32_t* keys = reinterpret_cast<const uint32_t*>(B.keys);
  e = select_init_count(keys, np, k, B, stream);
  if (e == cudaSuccess) e = select_threshold(keys, np, B, stream);
  if (e == cudaSuccess) e = select_compact(keys, np, B, pixel_idx, stream);
  if (e == cudaSuccess) {
    const gs_camera& c = plan->cams[view];
    CamDev cam;
    for (int i = 0; i < 9; ++i) cam.R[i] = c.R[i];
    for (int i = 0; i < 3; ++i) cam.t[i] = c.t[i];
    cam.fx = c.fx;
    cam.fy = c.fy;
    cam.cx = c.cx;
    cam.cy = c.cy;
    cam.width = c.width;
    cam.height = c.height;
    GS_TIMED("depth_points", stream,
             (depth_points_kernel<<<ceil_div(std::min<int64_t>(k, np), 256), 256, 0, stream>>>(
                 pixel_idx, B.k_dev, depth + p0, target, cam, points, colours)));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && k_out) e = cudaMemcpyAsync(k_out, B.k_dev, 4, cudaMemcpyDeviceToDevice, stream);
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

namespace gs {
namespace {

// Rows [0, n) of dst are src; row idx[r] and row n + r become the clone pair
// of Gaussian idx[r].
__global__ void clone_pairs_kernel(const float* __restrict__ src_op, const float* __restrict__ src_sc,
                                   const uint32_t* __restrict__ idx, int64_t n, int64_t k,
                                   float* __restrict__ dst_op, float* __restrict__ dst_sc) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  const int64_t i = idx[r];
  const float o = src_op[i];
  const float on = o / (1.f + sqrtf(1.f - o));                        // = 1 - sqrt(1 - o), no cancellation
  const float f = o / (2.f * on - on * on * 0.70710678118654752f);   // sqrt of the covariance factor
  dst_op[i] = on;
  dst_op[n + r] = on;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float s = src_sc[3 * i + c] * f;
    dst_sc[3 * i + c] = s;
    dst_sc[3 * (n + r) + c] = s;
  }
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_clone_gaussians(const gs_scene* src, const uint32_t* idx, int64_t k, const gs_scene_buf* dst,
                                        void* stream_) {
  if (!src || !dst || k < 0 || src->n < 0 || (k > 0 && !idx) || dst->n < src->n + k ||
      src->sh_coeffs != dst->sh_coeffs || !src->means || !dst->means || !src->scales || !dst->scales ||
      !src->rotations || !dst->rotations || !src->opacities || !dst->opacities || !src->sh || !dst->sh)
    return GS_ERR_INVALID_ARG;
  if (src->means == dst->means || src->scales == dst->scales || src->opacities == dst->opacities)
    return GS_ERR_INVALID_ARG;                      // out of place only
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  const int64_t n = src->n;
  struct Part {
    const float* s;
    float* d;
    int w;
  } parts[5] = {{src->means, dst->means, 3},
                {src->scales, dst->scales, 3},
                {src->rotations, dst->rotations, 4},
                {src->opacities, dst->opacities, 1},
                {src->sh, dst->sh, 3 * src->sh_coeffs}};
  cudaError_t e = cudaSuccess;
  for (const Part& p : parts) {
    if (n > 0 && e == cudaSuccess)
      e = cudaMemcpyAsync(p.d, p.s, (size_t)n * p.w * sizeof(float), cudaMemcpyDeviceToDevice, stream);
    // the clones' rows: the unchanged attributes of the source row
    if (k > 0 && e == cudaSuccess)
      GS_TIMED("clone_rows", stream, (gather_rows_kernel<<<ceil_div(k * p.w, 256), 256, 0, stream>>>(
                                          p.s, idx, k, p.w, p.d + (size_t)n * p.w)));
  }
  if (k > 0 && e == cudaSuccess)
    GS_TIMED("clone_pairs", stream, (clone_pairs_kernel<<<ceil_div(k, 256), 256, 0, stream>>>(
                                         src->opacities, src->scales, idx, n, k, dst->opacities, dst->scales)));
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
