// Tile binning: one (global tile id, item) entry per touched tile, emitted in
// the depth order of the items (Sec. 3.1), then tile ranges of the list
// sorted by tile id.  Also the L1 photometric loss of the training step.
//
// Duplication is warp-cooperative: a warp takes 32 consecutive items of the
// depth order, flattens their candidate rectangles into one index space and
// walks it 32 candidates at a time, so a Gaussian covering hundreds of tiles
// does not serialise its warp.  Each candidate is tested with the same exact
// tile predicate as the counting pass in preprocess (identical arithmetic),
// and its output slot is the item's scanned offset plus the number of hits
// of the same item before it (ballot + popc).
#include "project.cuh"

namespace gs {

namespace {

constexpr int kDupThreads = 256;

__device__ __forceinline__ uint32_t lanemask_lt_() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(const ViewDev* __restrict__ views, int64_t n_items,
                                                                int64_t n, const uint32_t* __restrict__ sorted_items,
                                                                const uint32_t* __restrict__ offsets, ItemState st,
                                                                uint32_t* __restrict__ keys,
                                                                uint32_t* __restrict__ vals,
                                                                uint32_t* __restrict__ status) {
  const int64_t k = (int64_t)blockIdx.x * kDupThreads + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t item = 0, cnt = 0, off = 0;
  if (k < n_items) {
    item = sorted_items[k];
    cnt = st.tiles[item];
  }
  float mx = 0.f, my = 0.f, tau = 0.f, A = 0.f, B = 0.f, C = 0.f;
  uint2 rect = make_uint2(0u, 0u);
  int area = 0, tbase = 0, tiles_x = 1;
  if (cnt > 0) {
    off = offsets[k];
    rect = st.rect[item];
    area = rect_area(rect);
    const float4 a = st.xy_tau_z[item];
    const float4 c = st.conic_o[item];
    mx = a.x;
    my = a.y;
    tau = a.z;
    A = c.x;
    B = c.y;
    C = c.z;
    const ViewDev& V = views[item / n];
    tbase = V.tile_base;
    tiles_x = V.tiles_x;
  }
  uint32_t total;
  const uint32_t excl = warp_exclusive_sum((uint32_t)area, &total);
  uint32_t written = 0;
  const uint32_t lt = lanemask_lt_();
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t c = base + lane;
    const int own = warp_owner(excl, min(c, total - 1));
    const float omx = __shfl_sync(0xffffffffu, mx, own), omy = __shfl_sync(0xffffffffu, my, own);
    const float oA = __shfl_sync(0xffffffffu, A, own), oB = __shfl_sync(0xffffffffu, B, own);
    const float oC = __shfl_sync(0xffffffffu, C, own), otau = __shfl_sync(0xffffffffu, tau, own);
    const uint32_t orx = __shfl_sync(0xffffffffu, rect.x, own), ory = __shfl_sync(0xffffffffu, rect.y, own);
    const uint32_t oex = __shfl_sync(0xffffffffu, excl, own);
    const uint32_t ooff = __shfl_sync(0xffffffffu, off, own);
    const uint32_t owr = __shfl_sync(0xffffffffu, written, own);
    const uint32_t ocnt = __shfl_sync(0xffffffffu, cnt, own);
    const uint32_t oitem = __shfl_sync(0xffffffffu, item, own);
    const int otb = __shfl_sync(0xffffffffu, tbase, own), otx = __shfl_sync(0xffffffffu, tiles_x, own);
    bool hit = false;
    int tx = 0, ty = 0;
    if (c < total) {
      const int tx0 = orx & 0xffff, ty0 = orx >> 16, nx = (int)(ory & 0xffff) - tx0 + 1;
      const int kk = (int)(c - oex);
      tx = tx0 + kk % nx;
      ty = ty0 + kk / nx;
      hit = tile_touched(omx, omy, oA, oB, oC, otau, tx, ty);
    }
    const uint32_t hits = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const int lo_own = (int)(oex > base ? oex - base : 0u);   // <= lane here
      const uint32_t below = hits & lt & ~((1u << lo_own) - 1u);
      const uint32_t r = owr + __popc(below);
      if (r < ocnt) {
        keys[ooff + r] = (uint32_t)(otb + ty * otx + tx);
        vals[ooff + r] = oitem;
      } else {
        atomicOr(status, kStatusEntryMismatch);
      }
    }
    const int lo = (int)min(max((int64_t)excl - (int64_t)base, (int64_t)0), (int64_t)32);
    const int hi = (int)min(max((int64_t)excl + area - (int64_t)base, (int64_t)0), (int64_t)32);
    if (hi > lo) {
      const uint32_t bits = (hi - lo == 32) ? 0xffffffffu : (((1u << (hi - lo)) - 1u) << lo);
      written += __popc(hits & bits);
    }
  }
  if (cnt > 0 && written != cnt) atomicOr(status, kStatusEntryMismatch);
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

__global__ void iota_kernel(uint32_t* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)i;
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

cudaError_t launch_iota(uint32_t* out, int64_t n, cudaStream_t stream) {
  if (n > 0) GS_TIMED("iota", stream, (iota_kernel<<<ceil_div(n, 256), 256, 0, stream>>>(out, n)));
  return cudaGetLastError();
}

cudaError_t launch_loss_l1(const float* image, const float* target, int64_t count, float* loss, float* dL,
                           cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), stream);
  if (e != cudaSuccess) return e;
  if (count > 0) {
    const int blocks = (int)std::min<int64_t>(ceil_div(count, 256), 152 * 8);
    GS_TIMED("loss_l1", stream, (l1_kernel<<<blocks, 256, 0, stream>>>(image, target, count, loss, dL)));
  }
  return cudaGetLastError();
}

}  // namespace gs
