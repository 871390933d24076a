// Tile binning: one (global tile id, item) entry per touched tile, emitted in
// the depth order of the items (Sec. 3.1), then tile ranges of the list
// sorted by tile id.  Also the L1 photometric loss of the training step.
//
// Duplication: one thread per item of the depth order walks the item's tile
// rows with the same interval form of the support as the counting pass in
// preprocess (identical arithmetic on the same stored parameters) and writes
// its entries at its scanned offset, row-major.
#include "project.cuh"

namespace gs {

namespace {

constexpr int kDupThreads = 256;

__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(const ViewDev* __restrict__ views, int64_t n_items,
                                                                int64_t n, const uint32_t* __restrict__ sorted_items,
                                                                const uint32_t* __restrict__ offsets, ItemState st,
                                                                uint32_t* __restrict__ keys,
                                                                uint32_t* __restrict__ vals,
                                                                uint32_t* __restrict__ status) {
  const int64_t k = (int64_t)blockIdx.x * kDupThreads + threadIdx.x;
  if (k >= n_items) return;
  const uint32_t item = sorted_items[k];
  const uint32_t cnt = st.tiles[item];
  if (cnt == 0) return;
  const uint32_t off = offsets[k];
  const float4 a = st.xy_tau_z[item];
  const float4 b0 = st.bin[2 * item], b1 = st.bin[2 * item + 1];
  BinParams b;
  b.mx = a.x;
  b.my = a.y;
  b.tau = a.z;
  b.k = b0.x;
  b.sc = b0.y;
  b.isyy = b0.z;
  b.h = b0.w;
  b.rx = b1.x;
  b.ys = b1.y;
  const ViewDev& V = views[item / n];
  // this item's entries are the contiguous run [off, off + cnt): write it as
  // scalars up to a 16-byte boundary, then in groups of four (uint4), then
  // the scalar tail
  const uint32_t head = min((4u - (off & 3u)) & 3u, cnt);
  const uint32_t groups_end = head + ((cnt - head) & ~3u);
  const uint4 vals4 = make_uint4(item, item, item, item);
  uint32_t buf[4];
  uint32_t written = 0;
  int ty0, ty1;
  if (tile_rows(b, V.tiles_y, &ty0, &ty1)) {
    for (int ty = ty0; ty <= ty1; ++ty) {
      int tx_a, tx_b;
      if (!row_tiles(b, ty, V.tiles_x, &tx_a, &tx_b)) continue;
      const uint32_t base = (uint32_t)(V.tile_base + ty * V.tiles_x);
      for (int tx = tx_a; tx <= tx_b; ++tx) {
        const uint32_t key = base + (uint32_t)tx;
        if (written < head || (written >= groups_end && written < cnt)) {
          keys[off + written] = key;
          vals[off + written] = item;
        } else if (written < groups_end) {
          const uint32_t g = (written - head) & 3u;
          buf[g] = key;
          if (g == 3u) {
            const uint32_t at = off + written - 3u;     // 4-aligned
            *reinterpret_cast<uint4*>(keys + at) = make_uint4(buf[0], buf[1], buf[2], buf[3]);
            *reinterpret_cast<uint4*>(vals + at) = vals4;
          }
        }
        ++written;
      }
    }
  }
  if (written != cnt) atomicOr(status, kStatusEntryMismatch);
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
