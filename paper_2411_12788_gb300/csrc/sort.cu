// Onesweep LSD radix sort of (uint32 key, uint32 value) pairs and a gathered
// exclusive scan.  Both order the rasterizer's work: the depth sort of
// (view, Gaussian) items and the stable sort of tile entries by tile id give
// every tile its list in the depth order of Sec. 3.1.
//
// Radix sort, 8-bit digit passes (the last one narrower when the bit count is
// not a multiple of 8), or a single 9-bit pass of 512 digits for a 9-bit sort
// (the tile-row sort of the list builder, whose rows usually fit 9 bits):
//   * one histogram kernel counts every pass's digits in a single read;
//   * each CTA of the pass kernel takes the next tile of 7680 keys (dynamic
//     tile id, so every predecessor tile is already running), ranks its keys
//     stably by digit inside each warp (the lanes sharing a digit found by
//     one ballot per digit bit, the running per-warp digit counts kept by
//     shared atomics whose results are collected after all rows), publishes
//     its per-digit counts, stages keys and values in shared memory in
//     output order, and only then looks back over its predecessors'
//     published counts (decoupled look-back) for its global offset per
//     digit, so that the predecessors have had longer to publish; the staged
//     keys are written out in runs of equal digits, which coalesce.
// The look-back spin is bounded: after kSpinLimit polls the CTA records
// kStatusTimeout in the status word and carries on (the result is then
// wrong, and the host reports GS_ERR_TIMEOUT), so a bug cannot hang the GPU.
#include "common.cuh"

namespace gs {

namespace {

constexpr uint32_t kFlagAggregate = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr int kMaxPasses = 4;
constexpr int kWarps = kSortThreads / 32;
static_assert(kSortThreads % kRadix == 0, "one digit per thread in the digit phases");
constexpr int kWarpKeys = kSortItemsPerThread * 32;
constexpr long kSpinLimit = 1L << 20;

struct RadixScratch {
  uint32_t* hist;      // [kMaxPasses][kRadix] counts, then exclusive offsets
  uint32_t* counters;  // [kMaxPasses] dynamic tile counters
  uint32_t* lookback;  // [kMaxPasses][tiles][kRadix]
};

__host__ __device__ inline int64_t sort_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

RadixScratch carve(void* base, int64_t n) {
  RadixScratch s;
  char* p = static_cast<char*>(base);
  s.hist = reinterpret_cast<uint32_t*>(p);
  s.counters = s.hist + kMaxPasses * kRadix;
  s.lookback = reinterpret_cast<uint32_t*>(p + align_up((kMaxPasses * kRadix + kMaxPasses) * 4));
  return s;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Digit mask of the pass starting at bit `shift` of a sort over bits [0, bits)
// with digits of rbits bits: the key bits above `bits` ride along unsorted.
__host__ __device__ inline uint32_t digit_mask(int bits, int shift, int rbits = kRadixBits) {
  return bits - shift >= rbits ? (1u << rbits) - 1u : (1u << (bits - shift)) - 1u;
}

// A sort over at most 9 bits takes one pass of 512 digits (the wide
// instance of the pass kernel) instead of an 8-bit pass and a narrow one.
constexpr int kWideBits = 9;
constexpr int kWideRadix = 1 << kWideBits;
__host__ __device__ inline bool wide_sort(int bits) { return bits == kWideBits; }

// Counts the digits of every pass in one read of the keys.  Each thread
// takes 8 consecutive keys and adds runs of equal digits with one shared
// atomic per run, which keeps nearly-sorted inputs (long runs of one high
// digit) from serialising on a single counter.
constexpr int kHistKeys = 8;

template <int kRBits>
__global__ void __launch_bounds__(256) radix_histogram_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                              int passes, int bits, uint32_t* __restrict__ hist) {
  constexpr int kR = 1 << kRBits;
  __shared__ uint32_t sh[kMaxPasses * kRadix];   // passes x kR counters (at most 1,024)
  for (int i = threadIdx.x; i < passes * kR; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * kHistKeys;
  for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kHistKeys; base < n; base += stride) {
    uint32_t k[kHistKeys];
    const int cnt = (int)((n - base < kHistKeys) ? (n - base) : (int64_t)kHistKeys);
    if (cnt == kHistKeys && (base & 3) == 0) {
      const uint4 a = *reinterpret_cast<const uint4*>(keys + base);
      const uint4 b = *reinterpret_cast<const uint4*>(keys + base + 4);
      k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w; k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < kHistKeys; ++j) k[j] = j < cnt ? keys[base + j] : 0u;
    }
    for (int p = 0; p < passes; ++p) {
      const int sh_p = p * kRBits;
      const uint32_t msk = digit_mask(bits, sh_p, kRBits);
      uint32_t cur = (k[0] >> sh_p) & msk, run = 1;
#pragma unroll
      for (int j = 1; j < kHistKeys; ++j) {
        if (j >= cnt) break;
        const uint32_t d = (k[j] >> sh_p) & msk;
        if (d == cur) {
          ++run;
        } else {
          atomicAdd(&sh[p * kR + cur], run);
          cur = d;
          run = 1;
        }
      }
      atomicAdd(&sh[p * kR + cur], run);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kR; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of each pass's kR digit counts (one block of kR threads per pass).
template <int kR>
__global__ void __launch_bounds__(kR) radix_scan_hist_kernel(uint32_t* hist) {
  __shared__ uint32_t s[kR];
  uint32_t* h = hist + blockIdx.x * kR;
  uint32_t v = h[threadIdx.x];
  s[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < kR; off <<= 1) {
    uint32_t t = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  h[threadIdx.x] = s[threadIdx.x] - v;
}

// Decoupled look-back for digit d of `tile`: the sum of the predecessors'
// counts for d, read 8 predecessors per round (the loads of a window are
// independent, so a round costs one L2 latency) back to the first published
// inclusive prefix.  A round that meets a predecessor with nothing published
// yet is repeated; after kSpinLimit such rounds the wait gives up, records
// kStatusTimeout and returns what it has (the sort result is then wrong and
// the host reports GS_ERR_TIMEOUT), so a missing publisher cannot hang the GPU.
template <int kR = kRadix>
__device__ __forceinline__ uint32_t lookback_exclusive(const uint32_t* lookback, int64_t tile, int d,
                                                       uint32_t* status) {
  uint32_t exclusive = 0;
  int64_t j = tile - 1;
  long spins = 0;
  constexpr int kWin = 8;
  while (j >= 0) {
    uint32_t st[kWin];
#pragma unroll
    for (int w = 0; w < kWin; ++w)
      st[w] = (j - w >= 0) ? *(const volatile uint32_t*)(lookback + (j - w) * kR + d) : (uint32_t)kFlagPrefix;
    uint32_t add = 0;
    int used = 0;
    bool found = false, stalled = false;
#pragma unroll
    for (int w = 0; w < kWin; ++w) {
      if (found || stalled) continue;
      const uint32_t flag = st[w] & ~kValueMask;
      if (flag == 0) {
        stalled = true;
        continue;
      }
      add += st[w] & kValueMask;
      ++used;
      if (flag == kFlagPrefix) found = true;
    }
    exclusive += add;
    j -= used;
    if (found) break;
    if (stalled && ++spins > kSpinLimit) {
      atomicOr(status, kStatusTimeout);
      break;
    }
  }
  return exclusive;
}

// Self-test of the bounded wait: one block looks back from tile 1 over a
// tile 0 that never publishes (its counts are zero), so every digit's wait
// runs out; out[d] receives what the wait returned.
__global__ void lookback_timeout_probe_kernel(const uint32_t* __restrict__ lookback, uint32_t* __restrict__ status,
                                              uint32_t* __restrict__ out) {
  out[threadIdx.x] = lookback_exclusive(lookback, 1, (int)threadIdx.x, status);
}

// Dynamic shared memory of the pass kernel: the CTA's keys (original order,
// then reused for the keys in output order), its values (original order) and
// its values in output order.
constexpr size_t kOnesweepDynSmem = 3 * (size_t)kSortTile * sizeof(uint32_t);
constexpr long kCopyWaitLimit = 1L << 22;

// kDigitBits: the widest digit the instance ranks (8, or 4 for the narrow
// last pass of a sort whose bit count is not a multiple of 8, or 9 for the
// single pass of a 9-bit sort); kR: the digits of the instance (256, or 512
// for the 9-bit pass).  With 512 digits every thread owns one digit, the
// per-warp digit counts (at most 480) are kept two to a word (16 bits each)
// so that the shared memory stays that of the 256-digit instance, and the
// output bases reuse the CTA offsets' array.
template <int kDigitBits, int kR>
__global__ void __launch_bounds__(kSortThreads, 1024 / kSortThreads) radix_onesweep_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n, int shift, uint32_t dmask,
    const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ counter,
    uint32_t* __restrict__ lookback, uint32_t* __restrict__ status) {
  static_assert(kR == kRadix || (kR == kWideRadix && kR == kSortThreads), "256 digits, or one digit per thread");
  static_assert((1 << kDigitBits) <= kR, "digits of the instance");
  constexpr bool kPacked = kR > kRadix;
  static_assert(!kPacked || kWarpKeys < 65536, "16-bit per-warp counts");
  constexpr int kHistWords = kPacked ? kR / 2 : kR;
  extern __shared__ __align__(16) uint32_t s_dyn[];
  uint32_t* s_keys = s_dyn;                       // keys: loaded, then in output order
  uint32_t* s_vin = s_dyn + kSortTile;            // values as loaded
  uint32_t* s_vals = s_dyn + 2 * kSortTile;       // values in output order
  __shared__ uint32_t s_warp_hist[kWarps][kHistWords];
  __shared__ uint32_t s_cta_start[kR];
  __shared__ uint32_t s_out_arr[kPacked ? 1 : kR];
  // output index of the CTA's first key of each digit, minus its start
  uint32_t* s_out_base = kPacked ? s_cta_start : s_out_arr;
  __shared__ uint32_t s_tile;
  __shared__ __align__(8) uint64_t s_bar;

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(counter, 1u);
    mbar_init(&s_bar, 1);
  }
  for (int i = tid; i < kWarps * kHistWords; i += kSortThreads) {
    (&s_warp_hist[0][0])[i] = 0;
  }
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t tile_start = tile * kSortTile;
  const int count = (int)((n - tile_start < kSortTile) ? (n - tile_start) : (int64_t)kSortTile);

  // 0. stage the tile's keys and values in shared memory: two bulk copies of
  //    the 16-byte-aligned part, plain loads for a ragged tail of < 4 keys
  const int bulk = count & ~3;
  if (tid == 0) {
    if (bulk > 0) {
      mbar_arrive_expect_tx(&s_bar, 2u * (uint32_t)bulk * 4u);
      bulk_copy_g2s(s_keys, keys_in + tile_start, (uint32_t)bulk * 4u, &s_bar);
      bulk_copy_g2s(s_vin, vals_in + tile_start, (uint32_t)bulk * 4u, &s_bar);
    }
  }
  if (tid < count - bulk) {
    s_keys[bulk + tid] = keys_in[tile_start + bulk + tid];
    s_vin[bulk + tid] = vals_in[tile_start + bulk + tid];
  }
  if (bulk > 0 && !mbar_wait(&s_bar, 0, kCopyWaitLimit)) {
    atomicOr(status, kStatusTimeout);
    mbar_wait(&s_bar, 0, kCopyWaitLimit);        // let the copy land before the CTA exits
  }
  __syncthreads();

  // 1. rank the keys stably by digit inside each warp (warp-striped: warp w
  //    owns keys [480 w, 480 w + 480) of the tile).  Per key row k the lanes
  //    sharing a digit are found with one ballot per digit bit; their lowest
  //    lane adds their number to the warp's running count of the digit with
  //    one shared atomic, whose old value (the count of that digit in rows
  //    before k) is only collected after the last row, so the rows do not
  //    wait on one another.  meta[k] = leader lane | (same-digit lanes below
  //    this one) << 5 | (leader only) old count << 10.
  uint32_t key[kSortItemsPerThread];
  uint32_t rank[kSortItemsPerThread];
  const uint32_t lt = lanemask_lt();
  const int warp_start = warp * kWarpKeys;
#pragma unroll
  for (int k = 0; k < kSortItemsPerThread; ++k) {
    const int i = warp_start + k * 32 + lane;
    key[k] = i < count ? s_keys[i] : 0u;
  }
  uint32_t* whist = s_warp_hist[warp];
#pragma unroll
  for (int k = 0; k < kSortItemsPerThread; ++k) {
    const int i = warp_start + k * 32 + lane;
    const bool valid = i < count;
    const uint32_t d = (key[k] >> shift) & dmask;
    // diff: the lanes whose digit differs from this lane's (or that hold no
    // key); a bit's ballot XOR this lane's bit replicated marks them
    uint32_t diff = ~__ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < kDigitBits; ++b) {      // digit bits past the pass's mask are zero
      const uint32_t bit = (d >> b) & 1u;
      diff |= __ballot_sync(0xffffffffu, bit) ^ (0u - bit);
    }
    const uint32_t peers = ~diff;
    const uint32_t leader = valid ? (uint32_t)(__ffs(peers) - 1) : (uint32_t)lane;
    uint32_t m = leader | ((uint32_t)__popc(peers & lt) << 5);
    if (valid && (uint32_t)lane == leader) {
      if constexpr (kPacked) {
        const uint32_t sh16 = (d & 1u) * 16u;
        m |= ((atomicAdd(&whist[d >> 1], (uint32_t)__popc(peers) << sh16) >> sh16) & 0xFFFFu) << 10;
      } else {
        m |= atomicAdd(&whist[d], (uint32_t)__popc(peers)) << 10;
      }
    }
    // orders this row's counter update before the next row's (the next
    // leader may be another lane)
    __syncwarp();
    rank[k] = m;
  }
#pragma unroll
  for (int k = 0; k < kSortItemsPerThread; ++k) {
    const uint32_t m = rank[k];
    rank[k] = (__shfl_sync(0xffffffffu, m, (int)(m & 31u)) >> 10) + ((m >> 5) & 31u);
  }
  __syncthreads();

  // 2. per digit (threads < kR, one digit each): offsets of each warp
  //    inside the CTA and the CTA's count, published for the successors
  const bool digit_thread = tid < kR;
  uint32_t cta_count = 0;
  if (digit_thread) {
    const int d = tid;
    for (int w = 0; w < kWarps; ++w) {
      if constexpr (kPacked) {
        // digits 2j and 2j + 1 share word j and are neighbouring lanes: both
        // read it, then the even lane writes both offsets
        const uint32_t word = s_warp_hist[w][d >> 1];
        const uint32_t c = (d & 1) ? (word >> 16) : (word & 0xFFFFu);
        const uint32_t odd = __shfl_xor_sync(0xffffffffu, cta_count, 1);
        __syncwarp();
        if (!(d & 1)) s_warp_hist[w][d >> 1] = cta_count | (odd << 16);
        cta_count += c;
      } else {
        uint32_t c = s_warp_hist[w][d];
        s_warp_hist[w][d] = cta_count;
        cta_count += c;
      }
    }
    // publish this tile's count (or its inclusive prefix for tile 0)
    uint32_t* mine = lookback + tile * kR + d;
    if (tile == 0) {
      __threadfence();
      *(volatile uint32_t*)mine = kFlagPrefix | cta_count;
    } else {
      *(volatile uint32_t*)mine = kFlagAggregate | cta_count;
    }
  }

  // 3. CTA-local exclusive scan over digits (for the shared-memory staging):
  //    warp-level inclusive scans, then across the digit warps
  uint32_t start = 0;
  {
    uint32_t v = cta_count;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += t;
    }
    __shared__ uint32_t s_warp_tot[kR / 32];
    if (digit_thread && lane == 31) s_warp_tot[warp] = v;
    __syncthreads();
    if (digit_thread) {
      uint32_t add = 0;
      for (int w = 0; w < warp; ++w) add += s_warp_tot[w];
      start = v - cta_count + add;
      s_cta_start[tid] = start;
    }
  }
  __syncthreads();

  // 4. stage keys and values in output order (needs only CTA-local offsets,
  //    so it runs before the look-back and gives the predecessors more time
  //    to publish their prefixes)
#pragma unroll
  for (int k = 0; k < kSortItemsPerThread; ++k) {
    const int i = warp_start + k * 32 + lane;
    if (i < count) {
      const uint32_t d = (key[k] >> shift) & dmask;
      const uint32_t woff = kPacked ? (s_warp_hist[warp][d >> 1] >> ((d & 1u) * 16u)) & 0xFFFFu : s_warp_hist[warp][d];
      const uint32_t pos = s_cta_start[d] + woff + rank[k];
      if (GS_IN_RANGE(pos, count, status)) {
        s_keys[pos] = key[k];
        s_vals[pos] = s_vin[i];
      }
    }
  }

  // 5. decoupled look-back for this digit, then this tile's inclusive prefix
  uint32_t exclusive = 0;
  if (digit_thread && tile > 0) {
    exclusive = lookback_exclusive<kR>(lookback, tile, tid, status);
    *(volatile uint32_t*)(lookback + tile * kR + tid) = kFlagPrefix | (exclusive + cta_count);
  }
  if constexpr (kPacked) __syncthreads();         // the staging above has read every s_cta_start
  if (digit_thread) s_out_base[tid] = digit_base[tid] + exclusive - start;
  __syncthreads();

  // 6. write out: runs of equal digits are contiguous in the output
  for (int i = tid; i < count; i += kSortThreads) {
    const uint32_t k = s_keys[i];
    const uint32_t d = (k >> shift) & dmask;
    const uint32_t out = s_out_base[d] + (uint32_t)i;
    if (GS_IN_RANGE(out, n, status)) {
      keys_out[out] = k;
      vals_out[out] = s_vals[i];
    }
  }
}

// ---- gathered exclusive scan ------------------------------------------------

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += t;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t add = 0, tot = 0;
  for (int w = 0; w < kScanThreads / 32; ++w) {
    if (w < warp) add += s_warp[w];
    tot += s_warp[w];
  }
  *total = tot;
  return x - v + add;
}

// Single-pass exclusive scan of the (gathered) counts with a decoupled
// look-back.  Each block takes the next tile of kScanTile counts (dynamic tile
// ids, so every predecessor of a tile is running or done), scans it, publishes
// its total, finds the total of all tiles before it from its predecessors'
// published words and publishes its own inclusive prefix.  A word holds the
// flag in its top two bits and the value below them, so a reader sees both
// together.  The resident tiles of the first wave finish their loads at about
// the same time, when only tile 0 has a prefix, so the look-back warp reads
// kScanWindow predecessors per step (kScanWindow / 32 per lane, nearest
// first): the walk back to tile 0 takes a few L2 round trips, not one per 32
// tiles.  The wait for an unpublished predecessor is bounded like the sort's:
// after kSpinLimit polls it records kStatusTimeout (when a status word is
// given) and carries on with what it has.
constexpr uint64_t kScanAggregate = 1ull << 62, kScanPrefix = 2ull << 62, kScanValueMask = (1ull << 62) - 1;
constexpr int kScanPerLane = 4, kScanWindow = 32 * kScanPerLane;
static_assert(kScanItems % 4 == 0, "a thread's counts are read as uint4");

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) { return *(const volatile uint64_t*)p; }
__device__ __forceinline__ void st_volatile_u64(uint64_t* p, uint64_t v) { *(volatile uint64_t*)p = v; }

// The sum of the published values of tiles [0, tile): read back from tile - 1
// to the nearest inclusive prefix, kScanWindow words per step (lane l holds
// the words at distances 4l .. 4l + 3).  Warp-uniform result.
__device__ uint64_t scan_lookback(const uint64_t* words, int tile, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  uint64_t excl = 0;
  int64_t j = tile - 1;
  long spins = 0;
  while (true) {
    uint64_t w[kScanPerLane];
#pragma unroll
    for (int u = 0; u < kScanPerLane; ++u) {
      const int64_t q = j - (lane * kScanPerLane + u);
      w[u] = q >= 0 ? ld_volatile_u64(&words[q]) : kScanPrefix;
    }
    // this lane's nearest prefix (kScanPerLane: none), any word before it unpublished, their sum
    int up = kScanPerLane;
    bool unready = false;
    uint64_t v = 0;
#pragma unroll
    for (int u = 0; u < kScanPerLane; ++u) {
      if (up == kScanPerLane) {
        const uint64_t flag = w[u] & ~kScanValueMask;
        unready |= flag == 0;
        v += w[u] & kScanValueMask;
        if (flag == kScanPrefix) up = u;
      }
    }
    const uint32_t prefix = __ballot_sync(0xffffffffu, up < kScanPerLane);
    const int first = prefix ? __ffs(prefix) - 1 : 31;      // lanes 0..first hold the words that count
    const uint32_t upto = first == 31 ? 0xffffffffu : ((2u << first) - 1u);
    if (__ballot_sync(0xffffffffu, unready) & upto) {
      if (++spins > kSpinLimit) {
        if (status && lane == 0) atomicOr(status, kStatusTimeout);
        return excl;
      }
      continue;                                              // the same window again
    }
    if (lane > first) v = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (prefix) return excl;
    j -= kScanWindow;
  }
}

// Self-test of the scan's bounded wait: one warp looks back from tile 1 over
// a tile 0 that never publishes; *out receives what the wait returned.
__global__ void scan_timeout_probe_kernel(const uint64_t* __restrict__ words, uint32_t* __restrict__ status,
                                          unsigned long long* __restrict__ out) {
  const uint64_t v = scan_lookback(words, 1, status);
  if (threadIdx.x == 0) *out = (unsigned long long)v;
}

__global__ void __launch_bounds__(kScanThreads, 2048 / kScanThreads) scan_onepass_kernel(const uint32_t* __restrict__ counts,
                                                                    const uint32_t* __restrict__ idx, int64_t n,
                                                                    uint64_t* __restrict__ words, int nb,
                                                                    uint32_t* __restrict__ out,
                                                                    unsigned long long* __restrict__ total,
                                                                    uint32_t* __restrict__ status) {
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_excl;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(reinterpret_cast<uint32_t*>(words + nb), 1u);
  __syncthreads();
  const int tile = (int)s_tile;
  // thread t owns the contiguous counts [t kScanItems, (t + 1) kScanItems) of the tile
  const int64_t base = (int64_t)tile * kScanTile + (int64_t)tid * kScanItems;
  uint32_t c[kScanItems];
  const uint32_t* src = idx ? idx : counts;
  if (base + kScanItems <= n && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
#pragma unroll
    for (int k = 0; k < kScanItems; k += 4) {
      const uint4 q = *reinterpret_cast<const uint4*>(src + base + k);
      c[k] = q.x, c[k + 1] = q.y, c[k + 2] = q.z, c[k + 3] = q.w;
    }
    if (idx) {
#pragma unroll
      for (int k = 0; k < kScanItems; ++k) c[k] = counts[c[k]];
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const int64_t i = base + k;
      c[k] = i < n ? counts[idx ? idx[i] : i] : 0u;
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) acc += c[k];
  uint32_t tot;
  const uint32_t pre = block_exclusive_scan(acc, s_warp, &tot);
  if (tid == 0) st_volatile_u64(&words[tile], (tile == 0 ? kScanPrefix : kScanAggregate) | (uint64_t)tot);
  if (tid < 32) {
    const uint64_t excl = tile > 0 ? scan_lookback(words, tile, status) : 0ull;
    if (tid == 0) {
      if (tile > 0) st_volatile_u64(&words[tile], kScanPrefix | ((excl + tot) & kScanValueMask));
      s_excl = excl;
      if (tile == nb - 1) *total = (unsigned long long)(excl + tot);
    }
  }
  __syncthreads();
  uint32_t run = (uint32_t)s_excl + pre;
  if (base + kScanItems <= n && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
#pragma unroll
    for (int k = 0; k < kScanItems; k += 4) {
      uint4 q;
      q.x = run, run += c[k];
      q.y = run, run += c[k + 1];
      q.z = run, run += c[k + 2];
      q.w = run, run += c[k + 3];
      *reinterpret_cast<uint4*>(out + base + k) = q;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const int64_t i = base + k;
      if (i < n) out[i] = run;
      run += c[k];
    }
  }
}

}  // namespace

size_t radix_scratch_bytes(int64_t n, int bits) {
  const int passes = (bits + kRadixBits - 1) / kRadixBits;
  // look-back words: passes x 256 per tile, or 512 for the one wide pass
  const size_t per_tile = wide_sort(bits) ? (size_t)kWideRadix : (size_t)passes * kRadix;
  return align_up((kMaxPasses * kRadix + kMaxPasses) * 4) + align_up(per_tile * (size_t)sort_tiles(n) * 4);
}

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                             int64_t n, int bits, void* scratch, uint32_t* status, cudaStream_t stream,
                             const char* tag, bool* result_in_alt) {
  if (result_in_alt) *result_in_alt = false;
  if (n <= 0 || bits <= 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(keys_alt) | reinterpret_cast<uintptr_t>(vals) |
       reinterpret_cast<uintptr_t>(vals_alt)) & 15)
    return cudaErrorMisalignedAddress;     // the bulk copies need 16-byte aligned rows
  static std::atomic<uint64_t> attr_done{0};
  cudaError_t ea = once_per_device(attr_done, [] {
    cudaError_t e = cudaFuncSetAttribute(radix_onesweep_kernel<8, kRadix>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOnesweepDynSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(radix_onesweep_kernel<4, kRadix>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kOnesweepDynSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(radix_onesweep_kernel<kWideBits, kWideRadix>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOnesweepDynSmem);
    return e;
  });
  if (ea != cudaSuccess) return ea;
  const bool wide = wide_sort(bits);
  const int rbits = wide ? kWideBits : kRadixBits, radix = 1 << rbits;
  const int passes = (bits + rbits - 1) / rbits;
  RadixScratch s = carve(scratch, n);
  const int64_t tiles = sort_tiles(n);
  cudaError_t e = cudaMemsetAsync(scratch, 0, radix_scratch_bytes(n, bits), stream);
  if (e != cudaSuccess) return e;
  // 8 blocks per SM keep more key loads in flight, but every block ends by
  // adding passes x 256 counters to the global histogram: sorts of 3 or 4
  // passes keep 4 blocks per SM
  int hist_blocks = (int)std::min<int64_t>((int64_t)(passes <= 2 ? 8 : 4) * device_sm_count(),
                                          (n + 256 * kHistKeys - 1) / (256 * kHistKeys));
  const bool depth = tag && tag[0] == 'd', pairs = tag && tag[0] == 'p';
  const char* hist_name = depth ? "depth_sort_histogram" : pairs ? "pair_sort_histogram" : "tile_sort_histogram";
  const char* scan_name = depth ? "depth_sort_scan_hist" : pairs ? "pair_sort_scan_hist" : "tile_sort_scan_hist";
  if (wide) {
    GS_TIMED(hist_name, stream,
             (radix_histogram_kernel<kWideBits><<<hist_blocks, 256, 0, stream>>>(keys, n, passes, bits, s.hist)));
    GS_TIMED(scan_name, stream, (radix_scan_hist_kernel<kWideRadix><<<passes, kWideRadix, 0, stream>>>(s.hist)));
  } else {
    GS_TIMED(hist_name, stream,
             (radix_histogram_kernel<kRadixBits><<<hist_blocks, 256, 0, stream>>>(keys, n, passes, bits, s.hist)));
    GS_TIMED(scan_name, stream, (radix_scan_hist_kernel<kRadix><<<passes, kRadix, 0, stream>>>(s.hist)));
  }
  uint32_t *kin = keys, *kout = keys_alt, *vin = vals, *vout = vals_alt;
  for (int p = 0; p < passes; ++p) {
    const uint32_t dmask = digit_mask(bits, p * rbits, rbits);
    // a pass of at most 4 digit bits ranks with 4 ballots per key instead of 8
    auto pass = wide ? radix_onesweep_kernel<kWideBits, kWideRadix>
                     : dmask < 16u ? radix_onesweep_kernel<4, kRadix> : radix_onesweep_kernel<8, kRadix>;
    GS_TIMED(depth ? "depth_sort_onesweep" : pairs ? "pair_sort_onesweep" : "tile_sort_onesweep", stream,
             (pass<<<(unsigned)tiles, kSortThreads, kOnesweepDynSmem, stream>>>(
                 kin, vin, kout, vout, n, p * rbits, dmask, s.hist + p * radix, s.counters + p,
                 s.lookback + (size_t)p * tiles * radix, status)));
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  cudaError_t el = cudaGetLastError();
  if (el != cudaSuccess) return el;
  if (kin != keys && result_in_alt) {   // odd number of passes: the caller takes the alt buffers
    *result_in_alt = true;
  } else if (kin != keys) {   // odd number of passes: the result sits in the alt buffers
    el = cudaMemcpyAsync(keys, kin, n * 4, cudaMemcpyDeviceToDevice, stream);
    if (el == cudaSuccess) el = cudaMemcpyAsync(vals, vin, n * 4, cudaMemcpyDeviceToDevice, stream);
  }
  return el;
}

cudaError_t lookback_timeout_probe(uint32_t* scratch, uint32_t* status, cudaStream_t stream) {
  // scratch: [2][kRadix] look-back words (tile 0 never published) + [kRadix] outputs
  cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * kRadix * sizeof(uint32_t), stream);
  if (e != cudaSuccess) return e;
  lookback_timeout_probe_kernel<<<1, kRadix, 0, stream>>>(scratch, status, scratch + 2 * kRadix);
  return cudaGetLastError();
}

cudaError_t scan_timeout_probe(uint64_t* scratch, uint32_t* status, cudaStream_t stream) {
  // scratch: [2] look-back words (tile 0 never published) + [1] output
  cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(uint64_t), stream);
  if (e != cudaSuccess) return e;
  scan_timeout_probe_kernel<<<1, 32, 0, stream>>>(scratch, status, reinterpret_cast<unsigned long long*>(scratch + 2));
  return cudaGetLastError();
}

// One look-back word per tile and the tile counter.
size_t scan_block_bytes(int64_t n) {
  return align_up(((size_t)ceil_div(std::max<int64_t>(n, 1), kScanTile) + 1) * 8);
}

cudaError_t gather_exclusive_scan(const uint32_t* counts, const uint32_t* idx, uint32_t* out, int64_t n,
                                  uint64_t* block_scratch, unsigned long long* total, cudaStream_t stream,
                                  uint32_t* status) {
  if (n <= 0) return cudaMemsetAsync(total, 0, 8, stream);
  const int nb = ceil_div(n, kScanTile);
  cudaError_t e = cudaMemsetAsync(block_scratch, 0, ((size_t)nb + 1) * 8, stream);
  if (e != cudaSuccess) return e;
  GS_TIMED("scan", stream,
           (scan_onepass_kernel<<<nb, kScanThreads, 0, stream>>>(counts, idx, n, block_scratch, nb, out, total,
                                                                 status)));
  return cudaGetLastError();
}

}  // namespace gs
