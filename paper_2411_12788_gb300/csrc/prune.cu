// Importance-based pruning (MSv2-D, Sec. 6.1): keep the k Gaussians with the
// largest accumulated blending weight I_i (Sec. 3.2), ties to the lower
// index, listed in ascending index order; and the gather of their rows into
// a compact scene for the re-render.
//
// Selection is an MSD radix select on the bit patterns of the (non-negative)
// weights, which order like the values: four passes each histogram the next
// 8 bits of the keys that still match the prefix found so far, and a single
// block picks the bucket holding the k-th largest.  That yields the exact
// threshold key t, the number of keys above it and how many keys equal to t
// are still needed.  Two scans then compact in index order: the first ranks
// the keys equal to t, the second places every kept index.
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
  flag[i] = (k > t || (k == t && tie_rank[i] < st->k_rem)) ? 1u : 0u;
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

struct PruneLayout {
  size_t state, hist, flag, rank, pos, scan_blocks, total_dev, total;
};

PruneLayout prune_layout(int64_t n) {
  PruneLayout L;
  const size_t m = (size_t)(n > 0 ? n : 1);
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t at = o;
    o = align_up(o + b);
    return at;
  };
  L.state = take(sizeof(SelectState));
  L.hist = take(256 * 4);
  L.total_dev = take(8);
  L.flag = take(4 * m);
  L.rank = take(4 * m);
  L.pos = take(4 * m);
  L.scan_blocks = take(scan_block_bytes((int64_t)m));
  L.total = o;
  return L;
}

}  // namespace

}  // namespace gs

using namespace gs;

extern "C" size_t gs_prune_workspace_size(int64_t n) { return n < 0 ? 0 : prune_layout(n).total; }

extern "C" gs_status gs_prune_select(const float* importance, int64_t n, int64_t k, uint32_t* keep_idx, void* ws,
                                     size_t ws_bytes, void* stream_) {
  if (n < 0 || k < 0 || k > n || n >= ((int64_t)1 << 32) || (n > 0 && !importance) || (k > 0 && !keep_idx) || !ws ||
      (reinterpret_cast<uintptr_t>(ws) & 255))
    return GS_ERR_INVALID_ARG;
  const PruneLayout L = prune_layout(n);
  if (ws_bytes < L.total) return GS_ERR_CAPACITY;
  if (k == 0) return GS_OK;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  char* base = static_cast<char*>(ws);
  const int blocks = ceil_div(n, 256);
  cudaError_t e = cudaSuccess;
  if (k == n) {
    GS_TIMED("prune_iota", stream, (iota_u32_kernel<<<blocks, 256, 0, stream>>>(keep_idx, n)));
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  }
  const uint32_t* keys = reinterpret_cast<const uint32_t*>(importance);
  SelectState* st = reinterpret_cast<SelectState*>(base + L.state);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + L.hist);
  SelectState init{0u, 0u, (uint32_t)k, 0u};
  e = cudaMemcpyAsync(st, &init, sizeof(init), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, 256 * 4, stream);
  if (e != cudaSuccess) return GS_ERR_CUDA;
  const int hb = std::min(blocks, 4 * 152);
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    GS_TIMED("prune_select_hist", stream, (select_hist_kernel<<<hb, kSelThreads, 0, stream>>>(keys, n, shift, st, hist)));
    GS_TIMED("prune_select_pick", stream, (select_pick_kernel<<<1, 256, 0, stream>>>(hist, shift, st)));
  }
  uint32_t* flag = reinterpret_cast<uint32_t*>(base + L.flag);
  uint32_t* rank = reinterpret_cast<uint32_t*>(base + L.rank);
  uint32_t* pos = reinterpret_cast<uint32_t*>(base + L.pos);
  uint64_t* sb = reinterpret_cast<uint64_t*>(base + L.scan_blocks);
  unsigned long long* tot = reinterpret_cast<unsigned long long*>(base + L.total_dev);
  GS_TIMED("prune_flags", stream, (tie_flags_kernel<<<blocks, 256, 0, stream>>>(keys, n, st, flag)));
  e = gather_exclusive_scan(flag, nullptr, rank, n, sb, tot, stream);
  if (e == cudaSuccess) {
    GS_TIMED("prune_flags", stream, (keep_flags_kernel<<<blocks, 256, 0, stream>>>(keys, n, st, rank, flag)));
    e = gather_exclusive_scan(flag, nullptr, pos, n, sb, tot, stream);
  }
  if (e == cudaSuccess)
    GS_TIMED("prune_scatter", stream, (scatter_kept_kernel<<<blocks, 256, 0, stream>>>(flag, pos, n, keep_idx)));
  e = cudaGetLastError();
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
