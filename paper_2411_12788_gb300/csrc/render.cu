// Per-tile front-to-back alpha blending (Eq. 1) and its derivative.
//
// One CTA per 16x16 tile (128 threads forward, 256 backward); each warp owns
// a 16x4 strip forward and an 8x4 block backward.  The tile's depth-ordered list is
// streamed through shared memory in batches of 256 entries, gathered by item
// id.  Per entry the batch holds its
// centre, colour, depth and the 2-D Gaussian in exponent form:
//   alpha_raw(x) = o exp(-q/2) = 2^e,  e = log2 o + a2 dx^2 + b2 dx dy + c2 dy^2
// with (a2, b2, c2) = -log2(e) (A/2, B, C/2) for the conic (A, B, C).  An entry
// takes part at a pixel iff e >= log2(alpha_min) (that is alpha >= alpha_min);
// then alpha = min(alpha_max, 2^e).  Forward and backward evaluate e with the
// same explicitly rounded operations, so they make identical decisions.
//
// Forward (one thread per two pixels of one row, sharing the row part of each
// entry's exponent): front-to-back blending with a per-pixel stop before
// T (1 - alpha) < t_min, the CTA leaving the list once all its pixels stopped.  Side outputs (what the paper's reorganisation reads):
// i_max = argmax_i w_i and w_max, the midpoint depth d^mid_{i_max} (Eq. 2,
// Sec. 4.1) evaluated once per pixel from the winner's ellipsoid frame, the
// blended depth sum_i w_i z_i, the per-Gaussian accumulated weight I_i
// (Sec. 3.2; each warp's weights are summed in 2^-24 fixed point by one
// redux.sync, then one shared add per warp and one global atomic per
// (tile, entry)) and the maximum-contribution area S_i (Sec. 4.1;
// warp-aggregated atomics).
//
// Backward: two entries per lane, a warp walking its pixels with lane scans
// for the transmittance and the colour in front, over the entries whose
// support box meets its 8x4 block (see render_bwd_kernel);
// gradients accumulate in registers, are combined across the CTA's warps in
// shared memory and added to the per-item buffer with one vector atomic per
// (tile, entry).  They are taken with respect to (centre, a2, b2, c2,
// log2 o, colour); the preprocess backward converts them to the conic and
// the opacity.
#include "project.cuh"

namespace gs {

namespace {

constexpr int kRenderThreads = kTilePixels;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

struct RenderParams {
  const ViewDev* views;
  int n_views;
  int64_t n;                    // Gaussians (item = view * n + gaussian)
  const uint2* ranges;          // [total_tiles]
  const uint32_t* vals;         // sorted entries -> item
  const float4* xy_tau_z;
  const float4* conic_o;
  const float4* rgb;
  const float4* depth_frame;
  float alpha_max, e_min, t_min;   // e_min = log2(alpha_min)
  float bg[3];
  uint32_t* status;             // device status word (the checked build's index checks)
  const unsigned long long* n_entries;
  // launch order of the tiles (block b renders tile order[b]: the longest
  // lists start first, so that the grid does not end on a few long tiles);
  // null for the identity (the backward)
  const uint32_t* order;
  int total_tiles;
};

// The item of list position idx, with the checked build's checks: a position
// past the entries or an item past the items records kStatusBounds and reads
// as item 0 (the results are then wrong, but no access leaves its array).
__device__ __forceinline__ uint32_t list_item(const RenderParams& P, uint64_t idx) {
  uint32_t item = GS_IN_RANGE(idx, *P.n_entries, P.status) ? P.vals[idx] : 0u;
  if (!GS_IN_RANGE(item, (uint64_t)P.n * (uint64_t)P.n_views, P.status)) item = 0u;
  return item;
}

struct FwdOut {
  float* image;
  float* final_T;
  uint32_t* n_contrib;
  int32_t* imax;
  float* wmax;
  float* depth;
  float* depth_blend;
  float* weight_sum;
  uint32_t* max_area;
  uint64_t* weight_sum_fixed;   // I_i in units of 2^-24 (integer sums: order-independent)
  float* depth_center;          // camera z of i_max's centre
  uint32_t* n_blended;          // entries blended per pixel
};

// Exponent form of an entry's 2-D Gaussian (identical in both kernels).
__device__ __forceinline__ float4 exponent_form(float4 co) {
  return make_float4(__fmul_rn(-0.5f * kLog2e, co.x), __fmul_rn(-kLog2e, co.y), __fmul_rn(-0.5f * kLog2e, co.z),
                     __log2f(co.w));
}

// e = (a2 dx + b2 dy) dx + (lo + c2 dy^2), explicitly rounded.  The second
// part and b2 dy depend only on the pixel row, so pixels of one row share
// them (expo_row); expo_pix finishes one pixel.
__device__ __forceinline__ float2 expo_row(float4 ex, float dy) {
  return make_float2(__fmaf_rn(__fmul_rn(ex.z, dy), dy, ex.w), __fmul_rn(ex.y, dy));
}
__device__ __forceinline__ float expo_pix(float4 ex, float2 row, float dx) {
  return __fmaf_rn(__fmaf_rn(ex.x, dx, row.y), dx, row.x);
}
__device__ __forceinline__ float expo(float4 ex, float dx, float dy) { return expo_pix(ex, expo_row(ex, dy), dx); }

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Blackwell's packed FP32 instructions: two independent IEEE operations in
// one instruction, each rounded exactly as its scalar form.  The backward
// keeps a lane's two entries in the two halves.
#define GS_PK3(op)                                                                                       \
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t" op            \
      " rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"                                                      \
      : "=f"(d.x), "=f"(d.y)                                                                             \
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y))
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) {
  float2 d;
  GS_PK3("mul.rn.f32x2");
  return d;
}
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) {
  float2 d;
  GS_PK3("add.rn.f32x2");
  return d;
}
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) {
  float2 d;
  GS_PK3("sub.rn.f32x2");
  return d;
}
#undef GS_PK3
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 pk_dup(float x) { return make_float2(x, x); }

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Inclusive lane scan of the affine maps x -> m x + f (applied front to back):
// (m1, f1) then (m2, f2) composes to (m1 m2, f1 + m1 f2).  After the scan lane
// l holds (prod_{k<=l} m_k, sum_{k<=l} f_k prod_{j<k} m_j): the transmittance
// product and the transmittance-weighted sum in one 5-step chain.
__device__ __forceinline__ void scan_affine(float& m, float& f) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1)
    asm("{\n\t.reg .f32 tm, tf;\n\t.reg .pred p;\n\t"
        "shfl.sync.up.b32 tm|p, %0, %2, 0, 0xffffffff;\n\t"
        "shfl.sync.up.b32 tf, %1, %2, 0, 0xffffffff;\n\t"
        "@p fma.rn.f32 %1, tm, %1, tf;\n\t"
        "@p mul.f32 %0, %0, tm;\n\t}"
        : "+f"(m), "+f"(f)
        : "r"(off));
}

__device__ __forceinline__ int find_view(const ViewDev* views, int n_views, int tile) {
  int v = 0;
  for (int k = 1; k < n_views; ++k)
    if (views[k].tile_base <= tile) v = k;
  return v;
}

// Pixel of thread `t` in the tile: warp t/32 owns the 8x4 block at
// ((w & 1) * 8, (w >> 1) * 4), lane l is pixel (l & 7, l >> 3) of it.
__device__ __forceinline__ void pixel_of(const ViewDev& V, int tile, int t, int* px, int* py) {
  const int local = tile - V.tile_base;
  const int tx = local % V.tiles_x, ty = local / V.tiles_x;
  const int warp = t >> 5, lane = t & 31;
  *px = tx * kTile + (warp & 1) * 8 + (lane & 7);
  *py = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
}

// Forward state of one pixel.
struct FwdPix {
  float fx, fy;                 // pixel centre
  float T, cr, cg, cb, dblend, wmax;
  int imax_pos;                 // list position of the argmax, -1 if none
  uint32_t last;                // one past the last blended position
  uint32_t nbl;                 // blended entries (counted when asked for)
  bool done;
};

__device__ __forceinline__ void fwd_pix_init(FwdPix& q, int px, int py, bool inside) {
  q.fx = (float)px + 0.5f;
  q.fy = (float)py + 0.5f;
  q.T = 1.f;
  q.cr = q.cg = q.cb = q.dblend = q.wmax = 0.f;
  q.imax_pos = -1;
  q.last = 0;
  q.nbl = 0;
  q.done = !inside;
}

// Blends the entry at list position `pos`, with exponent e at this pixel, into
// the pixel; returns its weight.  kDBlend: the blended depth is asked for.
template <bool kCount, bool kDBlend>
__device__ __forceinline__ float fwd_pix_blend(FwdPix& q, float e, const float4* s_rgbz, int j, int pos,
                                               float alpha_max, float e_min, float t_min) {
  if (q.done) return 0.f;
  if (e < e_min) return 0.f;
  const float alpha = fminf(alpha_max, ex2_approx(e));
  const float Tn = q.T * (1.f - alpha);
  if (Tn < t_min) {
    q.done = true;
    return 0.f;
  }
  const float w = alpha * q.T;
  const float4 c = s_rgbz[j];
  q.cr += w * c.x;
  q.cg += w * c.y;
  q.cb += w * c.z;
  if (kDBlend) q.dblend += w * c.w;
  if (w > q.wmax) {
    q.wmax = w;
    q.imax_pos = pos;
  }
  q.T = Tn;
  q.last = pos + 1;
  if (kCount) ++q.nbl;
  return w;
}

// Writes one pixel's outputs; S_i is added warp-aggregated by the caller.
__device__ __forceinline__ void fwd_pix_store(const FwdPix& q, const RenderParams& P, const FwdOut& O, const ViewDev& V,
                                              int view, int px, int py, int64_t imax_item) {
  const int64_t pix = V.pixel_base + (int64_t)py * V.width + px;
  const int64_t hw = (int64_t)V.width * V.height;
  float* img = O.image + 3 * V.pixel_base + (int64_t)py * V.width + px;
  img[0] = q.cr + q.T * P.bg[0];
  img[hw] = q.cg + q.T * P.bg[1];
  img[2 * hw] = q.cb + q.T * P.bg[2];
  O.final_T[pix] = q.T;
  O.n_contrib[pix] = q.last;
  if (O.n_blended) O.n_blended[pix] = q.nbl;
  if (O.imax) O.imax[pix] = imax_item >= 0 ? (int32_t)(imax_item - (int64_t)view * P.n) : -1;
  if (O.wmax) O.wmax[pix] = q.wmax;
  if (O.depth_blend) O.depth_blend[pix] = q.dblend;
  if (O.depth_center) O.depth_center[pix] = imax_item >= 0 ? P.xy_tau_z[imax_item].w : 0.f;
  if (O.depth) {
    float d = 0.f;
    if (imax_item >= 0) {
      // d^mid: ray r(t) = t (dx, dy, 1); in the ellipsoid's unit frame the ray
      // is t Wd - e, and the chord midpoint is t = (e . Wd) / (Wd . Wd)
      const float4* df = P.depth_frame + 3 * imax_item;
      const float4 r0 = df[0], r1 = df[1], r2 = df[2];
      const float rx = (q.fx - V.cx) / V.fx, ry = (q.fy - V.cy) / V.fy;
      const float w0 = r0.x * rx + r0.y * ry + r0.z;
      const float w1 = r1.x * rx + r1.y * ry + r1.z;
      const float w2 = r2.x * rx + r2.y * ry + r2.z;
      d = (r0.w * w0 + r1.w * w1 + r2.w * w2) / (w0 * w0 + w1 * w1 + w2 * w2);
    }
    O.depth[pix] = d;
  }
}

// S_i: pixels whose i_max is i (warp-aggregated).
__device__ __forceinline__ void add_max_area(uint32_t* max_area, bool has, int64_t imax_item, int lane) {
  const uint32_t m = __ballot_sync(0xffffffffu, has);
  if (has) {
    const uint32_t peers = __match_any_sync(m, (unsigned long long)imax_item);
    if (lane == __ffs(peers) - 1) atomicAdd(&max_area[imax_item], (uint32_t)__popc(peers));
  }
}

// Support box (x0, x1, y0, y1) of an entry from its centre and the packed
// half-extents (see pack_extent).
__device__ __forceinline__ float4 support_box(float mx, float my, float packed) {
  const float2 e = unpack_extent(packed);
  return make_float4(mx - e.x, mx + e.x, my - e.y, my + e.y);
}

// Whether the box meets the pixel-centre rectangle [x0, x0 + 7] x [y0, y0 + 3]
// of an 8x4 block.  The box contains every pixel whose exponent test can
// pass (see pack_extent), so an entry whose box misses a block was blended
// at none of its pixels.
__device__ __forceinline__ bool box_meets_block(float4 b, float x0, float y0) {
  return b.x <= x0 + 7.f && b.y >= x0 && b.z <= y0 + 3.f && b.w >= y0;
}

// Whether an entry can pass the exponent test at some pixel of the 8x4 block
// with pixel centres [x0, x0 + 7] x [y0, y0 + 3]: the maximum over that
// rectangle of the concave e(dx, dy) = lo + a2 dx^2 + b2 dx dy + c2 dy^2 (at
// the centre if it lies inside, else on an edge at the clamped vertex) is
// compared with e_min - margin.  The margin, 2^-18 (|lo| + |e_min| + S) with
// S = |a2| DX^2 + |b2| DX DY + |c2| DY^2 over the block's largest offsets, is
// 16 times a bound on the rounding error of the per-pixel FP32 exponent (four
// roundings of terms no larger than S), so a block that fails the test holds
// no pixel where the entry is blended.
__device__ __forceinline__ bool block_may_blend(float4 ex, float mx, float my, float x0, float y0, float e_min) {
  const float dx0 = x0 - mx, dx1 = (x0 + 7.f) - mx, dy0 = y0 - my, dy1 = (y0 + 3.f) - my;
  const float a2 = ex.x, b2 = ex.y, c2 = ex.z, lo = ex.w;
  float best;
  if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) {
    best = 0.f;
  } else {
    const float ia = -0.5f / a2, ic = -0.5f / c2;            // a2, c2 < 0
    best = -INFINITY;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const float dx = s2 ? dx1 : dx0;                         // vertical edge: best dy
      const float dy = fminf(fmaxf(b2 * dx * ic, dy0), dy1);
      best = fmaxf(best, fmaf(fmaf(a2, dx, b2 * dy), dx, c2 * dy * dy));
      const float ey = s2 ? dy1 : dy0;                         // horizontal edge: best dx
      const float ex2 = fminf(fmaxf(b2 * ey * ia, dx0), dx1);
      best = fmaxf(best, fmaf(fmaf(a2, ex2, b2 * ey), ex2, c2 * ey * ey));
    }
  }
  const float DX = fmaxf(fabsf(dx0), fabsf(dx1)), DY = fmaxf(fabsf(dy0), fabsf(dy1));
  const float S = fabsf(a2) * DX * DX + fabsf(b2) * DX * DY + fabsf(c2) * DY * DY;
  const float margin = 3.814697265625e-6f * (fabsf(lo) + fabsf(e_min) + S);   // 2^-18
  return lo + best >= e_min - margin;
}

// One thread per two pixels, (x, y) and (x + 8, y) (warp w < 4 owns the 16x4
// strip at rows 4w .. 4w + 3 of the tile), so the shared-memory reads of an
// entry, the row part of its exponent and the loop control serve both.
constexpr int kFwdThreads = kTilePixels / 2;

__device__ __forceinline__ void fwd_pixel_of(const ViewDev& V, int tile, int t, int* px, int* py) {
  const int local = tile - V.tile_base;
  const int tx = local % V.tiles_x, ty = local / V.tiles_x;
  const int warp = t >> 5, lane = t & 31;
  *px = tx * kTile + (lane & 7);
  *py = ty * kTile + warp * 4 + (lane >> 3);
}

// Blends a staged batch of nb entries into the thread's two pixels (same
// row, so they share the exponent's row part); the warp stops once all
// its pixels have (checked every 8 entries: a stopped pixel ignores the rest).
// The staged batch as consecutive entry pairs, so that one 128-bit load gives
// a quantity of both entries in an aligned register pair for the packed
// instructions: s_m[j/2] = (mx_j, mx_j+1, my_j, my_j+1), s_ab[j/2] = (a2, a2',
// b2, b2'), s_cl[j/2] = (c2, c2', log2 o, log2 o').
__device__ __forceinline__ void stage_pair_slot(float4* s_m, float4* s_ab, float4* s_cl, int k, float2 m, float4 ex) {
  float* fm = reinterpret_cast<float*>(s_m) + 4 * (k >> 1) + (k & 1);
  float* fab = reinterpret_cast<float*>(s_ab) + 4 * (k >> 1) + (k & 1);
  float* fcl = reinterpret_cast<float*>(s_cl) + 4 * (k >> 1) + (k & 1);
  fm[0] = m.x;
  fm[2] = m.y;
  fab[0] = ex.x;
  fab[2] = ex.y;
  fcl[0] = ex.z;
  fcl[2] = ex.w;
}

// Blends a staged batch of nb entries into the thread's two pixels (same
// row, so they share the exponent's row part); the warp stops once all
// its pixels have (checked every 8 entries: a stopped pixel ignores the rest).
// The exponents of two consecutive entries are evaluated together with the
// packed FP32x2 instructions (each half rounded exactly as expo_row/expo_pix,
// so the decisions equal the backward's); blending stays entry by entry.
template <bool kWantW, bool kCount, bool kDBlend>
__device__ __forceinline__ void fwd_batch(FwdPix& q0, FwdPix& q1, int nb, int pos0, const float4* s_m,
                                          const float4* s_ab, const float4* s_cl, const float4* s_rgbz,
                                          uint32_t* s_wsum, const RenderParams& P, int lane) {
  const float2 fy = pk_dup(q0.fy), fx0 = pk_dup(q0.fx), fx1 = pk_dup(q1.fx);
  for (int j0 = 0; j0 < nb; j0 += 8) {
    if (__all_sync(0xffffffffu, q0.done && q1.done)) break;
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      const int j = j0 + u;
      if (j >= nb) break;
      const float4 m4 = s_m[j >> 1], ab4 = s_ab[j >> 1], cl4 = s_cl[j >> 1];
      const float2 mx = make_float2(m4.x, m4.y), my = make_float2(m4.z, m4.w);
      const float2 dy = pk_sub(fy, my);
      const float2 rowx = pk_fma(pk_mul(make_float2(cl4.x, cl4.y), dy), dy, make_float2(cl4.z, cl4.w));
      const float2 rowy = pk_mul(make_float2(ab4.z, ab4.w), dy);
      const float2 a2 = make_float2(ab4.x, ab4.y);
      const float2 e0 = pk_fma(pk_fma(a2, pk_sub(fx0, mx), rowy), pk_sub(fx0, mx), rowx);
      const float2 e1 = pk_fma(pk_fma(a2, pk_sub(fx1, mx), rowy), pk_sub(fx1, mx), rowx);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (j + h >= nb) break;
        const float w0 = fwd_pix_blend<kCount, kDBlend>(q0, h ? e0.y : e0.x, s_rgbz, j + h, pos0 + j + h, P.alpha_max,
                                               P.e_min, P.t_min);
        const float w1 = fwd_pix_blend<kCount, kDBlend>(q1, h ? e1.y : e1.x, s_rgbz, j + h, pos0 + j + h, P.alpha_max,
                                               P.e_min, P.t_min);
        if (kWantW && __any_sync(0xffffffffu, w0 > 0.f || w1 > 0.f)) {
          const uint32_t s = __reduce_add_sync(0xffffffffu, __float2uint_rn(w0 * 16777216.f) +
                                                                __float2uint_rn(w1 * 16777216.f));
          if (lane == 0) atomicAdd(&s_wsum[j + h], s);
        }
      }
    }
  }
}

// 12 CTAs (48 warps) per SM: 40 registers and a few spilled words; at 1M
// Gaussians over 8 views 0.967 ms against 0.996 ms at the compiler's own 48
// registers (10 CTAs) and 1.051 ms at 32 (16 CTAs, heavier spills).
template <bool kWantW, bool kCount, bool kDBlend>
__global__ void __launch_bounds__(kFwdThreads, 12) render_fwd_kernel(RenderParams P, FwdOut O) {
  constexpr int kBatch = kTilePixels;
  __shared__ int s_view;
  __shared__ float4 s_m[kBatch / 2];     // entry pairs: centres
  __shared__ float4 s_ab[kBatch / 2];    // entry pairs: a2, b2
  __shared__ float4 s_cl[kBatch / 2];    // entry pairs: c2, log2 o
  __shared__ float4 s_rgbz[kBatch];
  __shared__ uint32_t s_item[kBatch];
  __shared__ uint32_t s_wsum[kBatch];    // 2^-24 fixed point

  const uint32_t tile_u = P.order ? P.order[blockIdx.x] : (uint32_t)blockIdx.x;
  if (tile_u >= (uint32_t)P.total_tiles) {        // an order that names no tile: record, touch nothing
    if (threadIdx.x == 0) atomicOr(P.status, kStatusBounds);
    return;
  }
  const int tile = (int)tile_u;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) s_view = find_view(P.views, P.n_views, tile);
  s_wsum[tid] = 0u;
  s_wsum[tid + kFwdThreads] = 0u;
  __syncthreads();
  const int view = s_view;
  const ViewDev& V = P.views[view];
  int px, py;
  fwd_pixel_of(V, tile, tid, &px, &py);
  const int px2 = px + kTile / 2;
  const bool in0 = px < V.width && py < V.height;
  const bool in1 = px2 < V.width && py < V.height;
  FwdPix q0, q1;
  fwd_pix_init(q0, px, py, in0);
  fwd_pix_init(q1, px2, py, in1);
  const uint2 range = P.ranges[tile];
  for (uint32_t bstart = range.x; bstart < range.y; bstart += kBatch) {
    if (__syncthreads_count(q0.done && q1.done) == kFwdThreads) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = tid + h * kFwdThreads;
      const uint32_t idx = bstart + k;
      if (idx < range.y) {
        const uint32_t item = list_item(P, idx);
        s_item[k] = item;
        const float4 a = P.xy_tau_z[item];
        stage_pair_slot(s_m, s_ab, s_cl, k, make_float2(a.x, a.y), exponent_form(P.conic_o[item]));
        const float4 c = P.rgb[item];
        s_rgbz[k] = make_float4(c.x, c.y, c.z, a.w);
      }
    }
    __syncthreads();
    const int nb = (int)min(range.y - bstart, (uint32_t)kBatch);
    const int pos0 = (int)(bstart - range.x);
    fwd_batch<kWantW, kCount, kDBlend>(q0, q1, nb, pos0, s_m, s_ab, s_cl, s_rgbz, s_wsum, P, lane);
    __syncthreads();
    if (kWantW) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = tid + h * kFwdThreads;
        if (k < nb) {
          const uint32_t s = s_wsum[k];
          if (s) {
            if (O.weight_sum) atomicAdd(&O.weight_sum[s_item[k]], (float)s * (1.f / 16777216.f));
            if (O.weight_sum_fixed)
              atomicAdd(reinterpret_cast<unsigned long long*>(O.weight_sum_fixed) + s_item[k], (unsigned long long)s);
          }
          s_wsum[k] = 0u;
        }
      }
    }
  }

  const int64_t item0 = q0.imax_pos >= 0 ? (int64_t)list_item(P, (uint64_t)range.x + q0.imax_pos) : -1;
  const int64_t item1 = q1.imax_pos >= 0 ? (int64_t)list_item(P, (uint64_t)range.x + q1.imax_pos) : -1;
  if (O.max_area) {
    add_max_area(O.max_area, in0 && item0 >= 0, item0, lane);
    add_max_area(O.max_area, in1 && item1 >= 0, item1, lane);
  }
  if (in0) fwd_pix_store(q0, P, O, V, view, px, py, item0);
  if (in1) fwd_pix_store(q1, P, O, V, view, px2, py, item1);
}

struct BwdIn {
  const float* dL_dimage;
  const float* image;           // forward output c(x) + T_final bg
  const uint32_t* n_contrib;
  float4* grad2d;               // 2 x float4 per item: (mx, my, a2, b2), (c2, log2 o, r, g)
  float* grad2d_b;              // 1 float per item: b
  float* weight_sum;            // optional: += I_i per item
  uint64_t* weight_sum_fixed;   // optional: += I_i per item in units of 2^-24
};

// Backward of Eq. 1, two entries per lane.  For pixel x with blended entries
// k (alpha_k, colour c_k, w_k = alpha_k T_k) and image I = sum w_k c_k + T bg:
//   dI/dc_l     = w_l
//   dI/dalpha_l = T_l c_l - (I - F_l) / (1 - alpha_l),  F_l = sum_{k<=l} w_k c_k
// so with g = dL/dI the only per-pixel quantities an entry needs are the
// exclusive product T_l of (1 - alpha) and the inclusive sum of
// w_k (c_k . g) over the entries in front of it.  After a batch is staged,
// each warp lists the batch entries whose support box meets its 8x4 block
// (an entry outside the box was blended at none of the block's pixels), then
// takes 64 consecutive listed entries at a time (lane l holds the 2l-th and
// (2l + 1)-th) and walks its 32 pixels; a list tail of at most 32, 16 or 8
// entries is walked 2, 4 or 8 pixels per step by lane segments (see
// bwd_walk_chunk).  Each lane composes the affine maps x -> (1 - a) x + a (c.g)
// of its two entries, one shuffle scan over the lanes gives both
// prefix quantities for the lane's first entry, and the second follows from
// the first in registers; the pixel's state is continued from chunk to chunk
// through shared memory.  Each lane sums its entries' gradients over the
// pixels in registers, so no per-entry reduction across pixels is needed.
// Entries at or after a pixel's n_contrib and entries with
// e < log2(alpha_min) do not take part, exactly as in the forward pass.  With
// alpha_raw = 2^e unclamped, dalpha/de = alpha ln 2.
struct BwdEntry {
  float mx, my;        // centre
  float4 ex;           // exponent form
  float3 col;
};

// A lane's sums over the pixels for its two entries (first entry in .x,
// second in .y), with de = dL/de / ln 2 (the factor is applied at the
// flush): de dx, de dy (the centre's gradient follows from them and the
// entry's a2, b2, c2), de dx^2, de dx dy, de dy^2 (d a2, b2, c2), de
// (d log2 o), w dL/dI (d colour).
struct BwdSums {
  float2 acc[9];
  float2 wsum;         // blending weight over the warp's pixels (I_i)
  uint32_t wfix_a, wfix_b;   // the same, each pixel's weight rounded to a multiple of 2^-24
};

__device__ __forceinline__ void bwd_entry_load(BwdEntry& E, bool valid, const float2* s_xy, const float4* s_ex,
                                               const float4* s_rgb, int idx) {
  const float2 m = valid ? s_xy[idx] : make_float2(0.f, 0.f);
  E.mx = m.x;
  E.my = m.y;
  // an invalid entry gets an exponent that never passes the e_min test
  E.ex = valid ? s_ex[idx] : make_float4(0.f, 0.f, 0.f, -1e30f);
  const float4 c = valid ? s_rgb[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
  E.col = make_float3(c.x, c.y, c.z);
}

// Adds one pixel's contribution to a lane's two entries' gradient sums, both
// halves at once: a = (alpha_A, alpha_B) is zero for an entry that does not
// take part at this pixel, and ad the same with zero also where the 0.99
// clamp holds (no alpha gradient there), so such an entry adds nothing.
template <bool kFix>
__device__ __forceinline__ void bwd_pair_accumulate(BwdSums& S, const float4& pg, float2 dx, float2 dy, float2 a,
                                                    float2 ad, float2 one_minus_a, float2 T, float2 F, float2 cg) {
  const float2 w = pk_mul(a, T);
  S.wsum = pk_add(S.wsum, w);
  if (kFix) {
    S.wfix_a += __float2uint_rn(w.x * 16777216.f);
    S.wfix_b += __float2uint_rn(w.y * 16777216.f);
  }
  S.acc[6] = pk_fma(w, pk_dup(pg.x), S.acc[6]);
  S.acc[7] = pk_fma(w, pk_dup(pg.y), S.acc[7]);
  S.acc[8] = pk_fma(w, pk_dup(pg.z), S.acc[8]);
  // dL/dalpha = T (c.g) - (I - F) / (1 - alpha)
  const float2 r = make_float2(rcp_approx(one_minus_a.x), rcp_approx(one_minus_a.y));
  const float2 dal = pk_fma(pk_sub(F, pk_dup(pg.w)), r, pk_mul(T, cg));
  const float2 de = pk_mul(dal, ad);                 // dL/de / ln 2
  const float2 dedx = pk_mul(de, dx), dedy = pk_mul(de, dy);
  S.acc[5] = pk_add(S.acc[5], de);                   // log2 o
  S.acc[2] = pk_fma(dedx, dx, S.acc[2]);             // a2
  S.acc[3] = pk_fma(dedx, dy, S.acc[3]);             // b2
  S.acc[4] = pk_fma(dedy, dy, S.acc[4]);             // c2
  S.acc[0] = pk_add(S.acc[0], dedx);                 // centre, via the flush
  S.acc[1] = pk_add(S.acc[1], dedy);
}

template <bool kFix>
__device__ __forceinline__ void bwd_entry_flush(const BwdEntry& E, const float* acc, float wsum, uint32_t wfix,
                                                float (*s_g)[kRenderThreads], float* s_wsum, uint32_t* s_wfix, int idx,
                                                bool want_w) {
  // d = pixel - centre, so de/dcentre = -(2 a2 dx + b2 dy, b2 dx + 2 c2 dy);
  // every exponent term carries the factor ln 2 left out per pixel
  float g[9];
  g[0] = -kLn2 * fmaf(2.f * E.ex.x, acc[0], E.ex.y * acc[1]);
  g[1] = -kLn2 * fmaf(E.ex.y, acc[0], 2.f * E.ex.z * acc[1]);
#pragma unroll
  for (int k = 2; k < 6; ++k) g[k] = kLn2 * acc[k];
#pragma unroll
  for (int k = 6; k < 9; ++k) g[k] = acc[k];
#pragma unroll
  for (int k = 0; k < 9; ++k)
    if (g[k] != 0.f) atomicAdd(&s_g[k][idx], g[k]);
  if (want_w && wsum != 0.f) atomicAdd(&s_wsum[idx], wsum);
  if (kFix && wfix) atomicAdd(&s_wfix[idx], wfix);
}

// The affine scan of scan_affine within segments of kL lanes (kL a power of
// two): lane l ends with the composition over the lanes of its segment up to
// and including l.  The shuffle's segment mask keeps sources in the segment.
template <int kL>
__device__ __forceinline__ void scan_affine_seg(float& m, float& f) {
  constexpr uint32_t kSegMask = (uint32_t)(32 - kL) << 8;
#pragma unroll
  for (int off = 1; off < kL; off <<= 1)
    asm("{\n\t.reg .f32 tm, tf;\n\t.reg .pred p;\n\t"
        "shfl.sync.up.b32 tm|p, %0, %2, %3, 0xffffffff;\n\t"
        "shfl.sync.up.b32 tf, %1, %2, %3, 0xffffffff;\n\t"
        "@p fma.rn.f32 %1, tm, %1, tf;\n\t"
        "@p mul.f32 %0, %0, tm;\n\t}"
        : "+f"(m), "+f"(f)
        : "r"(off), "n"(kSegMask));
}

// What a chunk walk reads and writes besides the list: the staged batch, the
// per-pixel state and the per-entry gradient sums in shared memory.
struct BwdShared {
  const float2* xy;
  const float4* ex;
  const float4* rgb;
  const float4* pg;
  float4* st;
  float (*g)[kRenderThreads];
  float* wsum;
  uint32_t* wfix;
};

// Walks one chunk of a warp's list over the warp's 8x4 block, kSeg pixels
// per step.  The warp splits into kSeg segments of kL = 32 / kSeg lanes; lane
// j of each segment holds list entries c + 2j and c + 2j + 1 (those before
// cnt), and segment s takes pixel s of each run of kSeg pixels of a row.  A
// chunk thus holds 64 / kSeg entries: a short list tail is walked with
// several pixels per step instead of idle lanes.  The lane scans run within a
// segment, and an entry's sums over the segments' pixels are added together
// before the flush.
template <bool kFix, int kSeg>
__device__ __forceinline__ void bwd_walk_chunk(const RenderParams& P, const BwdShared& M, const uint8_t* list, int c,
                                               int cnt, uint32_t bstart, uint32_t my_nc, int warp, int lane,
                                               float bxf, float byf, bool want_w) {
  constexpr int kL = 32 / kSeg;
  const int j = lane & (kL - 1), seg = lane / kL;
  __syncwarp();                                 // list stores; the state stores of the last chunk
  const int ta = c + 2 * j, tb = ta + 1;        // my entries in the list
  const bool va = ta < cnt, vb = tb < cnt;
  const int ia = va ? list[ta] : 0, ib = vb ? list[tb] : 0;
  BwdEntry A, Bn;
  bwd_entry_load(A, va, M.xy, M.ex, M.rgb, ia);
  bwd_entry_load(Bn, vb, M.xy, M.ex, M.rgb, ib);
  BwdSums S;
#pragma unroll
  for (int k = 0; k < 9; ++k) S.acc[k] = make_float2(0.f, 0.f);
  S.wsum = make_float2(0.f, 0.f);
  S.wfix_a = S.wfix_b = 0u;
  // the two entries side by side for the packed instructions
  const float2 mx2 = make_float2(A.mx, Bn.mx), my2 = make_float2(A.my, Bn.my);
  const float2 exx = make_float2(A.ex.x, Bn.ex.x), exy = make_float2(A.ex.y, Bn.ex.y);
  const float2 exz = make_float2(A.ex.z, Bn.ex.z), exw = make_float2(A.ex.w, Bn.ex.w);
  const float2 colx = make_float2(A.col.x, Bn.col.x), coly = make_float2(A.col.y, Bn.col.y);
  const float2 colz = make_float2(A.col.z, Bn.col.z);
  const uint32_t posa = bstart + ia, posb = bstart + ib;   // list positions
  // pixels of this warp still blending at the chunk's first entry
  const uint32_t pmask = __ballot_sync(0xffffffffu, my_nc > bstart + list[c]);
  // the block's 4 rows, 8 pixels each: the row part of each entry's
  // exponent is computed once per row
#pragma unroll 1
  for (int r = 0; r < 4; ++r) {
    if (!((pmask >> (8 * r)) & 0xffu)) continue;
    // pixel centre minus entry centre, rounded exactly as in the forward
    const float fy = byf + (float)r;
    const float2 dy = pk_sub(pk_dup(fy), my2);
    const float2 rowx = pk_fma(pk_mul(exz, dy), dy, exw), rowy = pk_mul(exy, dy);   // expo_row, both entries
#pragma unroll 4
    for (int cx0 = 0; cx0 < 8; cx0 += kSeg) {
      if (!((pmask >> (8 * r + cx0)) & ((1u << kSeg) - 1u))) continue;
      const int cx = cx0 + seg;
      const int pt = warp * 32 + 8 * r + cx;        // the pixel's thread id
      const float4 st = M.st[pt];
      const uint32_t nc = __float_as_uint(st.z);
      const float fx = bxf + (float)cx;
      const float2 dx = pk_sub(pk_dup(fx), mx2);
      const float2 e = pk_fma(pk_fma(exx, dx, rowy), dx, rowx);   // expo_pix, both entries
      const bool acta = posa < nc && e.x >= P.e_min;
      const bool actb = posb < nc && e.y >= P.e_min;
      if (!__any_sync(0xffffffffu, acta || actb)) continue;
      const float4 pg = M.pg[pt];
      const float arawa = ex2_approx(e.x), arawb = ex2_approx(e.y);
      const float2 a = make_float2(acta ? fminf(P.alpha_max, arawa) : 0.f, actb ? fminf(P.alpha_max, arawb) : 0.f);
      const float2 cg = pk_fma(colz, pk_dup(pg.z), pk_fma(coly, pk_dup(pg.y), pk_mul(colx, pk_dup(pg.x))));
      // the lane's two maps composed, then one scan over the segment's
      // lanes: the product of (1 - a) and sum a_k cg_k prod_{j<k} (1 - a_j)
      const float2 oma = pk_sub(make_float2(1.f, 1.f), a);
      const float2 fab = pk_mul(a, cg);
      float m = oma.x * oma.y, f = fmaf(oma.x, fab.y, fab.x);
      scan_affine_seg<kL>(m, f);
      float mex = __shfl_up_sync(0xffffffffu, m, 1, kL);   // exclusive over the segment's lanes
      float fex = __shfl_up_sync(0xffffffffu, f, 1, kL);
      if (j == 0) {
        mex = 1.f;
        fex = 0.f;
      }
      const float T0 = st.x, F0 = st.y;
      const float Ta = T0 * mex;                            // T in front of entry A
      const float Fa = fmaf(Ta, fab.x, fmaf(T0, fex, F0));   // sum_{k<=A} w_k cg_k
      const float Tb = Ta * oma.x;
      const float Fb = fmaf(Tb * a.y, cg.y, Fa);
      // the segment's last lane holds the chunk's totals: carry the pixel's
      // state forward
      __syncwarp();
      if (j == kL - 1) {
        float2* stp = reinterpret_cast<float2*>(&M.st[pt]);
        *stp = make_float2(T0 * m, fmaf(T0, f, F0));
      }
      // alpha gradient only where the 0.99 clamp is not active
      const float2 ad = make_float2(arawa <= P.alpha_max ? a.x : 0.f, arawb <= P.alpha_max ? a.y : 0.f);
      bwd_pair_accumulate<kFix>(S, pg, dx, dy, a, ad, oma, make_float2(Ta, Tb), make_float2(Fa, Fb), cg);
    }
  }
  if (kSeg > 1) {
    // the segments hold the same entries over different pixels
#pragma unroll
    for (int o = kL; o < 32; o <<= 1) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        S.acc[k].x += __shfl_xor_sync(0xffffffffu, S.acc[k].x, o);
        S.acc[k].y += __shfl_xor_sync(0xffffffffu, S.acc[k].y, o);
      }
      if (want_w) {
        S.wsum.x += __shfl_xor_sync(0xffffffffu, S.wsum.x, o);
        S.wsum.y += __shfl_xor_sync(0xffffffffu, S.wsum.y, o);
      }
      if (kFix) {
        S.wfix_a += __shfl_xor_sync(0xffffffffu, S.wfix_a, o);
        S.wfix_b += __shfl_xor_sync(0xffffffffu, S.wfix_b, o);
      }
    }
    if (seg != 0) return;
  }
  if (va) {
    const float acc[9] = {S.acc[0].x, S.acc[1].x, S.acc[2].x, S.acc[3].x, S.acc[4].x,
                          S.acc[5].x, S.acc[6].x, S.acc[7].x, S.acc[8].x};
    bwd_entry_flush<kFix>(A, acc, S.wsum.x, S.wfix_a, M.g, M.wsum, M.wfix, ia, want_w);
  }
  if (vb) {
    const float acc[9] = {S.acc[0].y, S.acc[1].y, S.acc[2].y, S.acc[3].y, S.acc[4].y,
                          S.acc[5].y, S.acc[6].y, S.acc[7].y, S.acc[8].y};
    bwd_entry_flush<kFix>(Bn, acc, S.wsum.y, S.wfix_b, M.g, M.wsum, M.wfix, ib, want_w);
  }
}

// 4 CTAs (32 warps) per SM: 64 registers with a few hundred bytes spilled,
// which the extra warps more than pay for (at 1M Gaussians over 8 views
// 2.547 ms against 2.655 ms at 3 CTAs and 80 registers; 5 CTAs at 48
// registers spill 748 bytes and take 3.64 ms).
template <bool kFix>
__global__ void __launch_bounds__(kRenderThreads, 4) render_bwd_kernel(RenderParams P, BwdIn B) {
  constexpr int kWarps = kRenderThreads / 32;
  __shared__ int s_view;
  __shared__ uint32_t s_max_nc;
  __shared__ float2 s_xy[kRenderThreads];
  __shared__ float4 s_ex[kRenderThreads];
  __shared__ float4 s_rgb[kRenderThreads];
  __shared__ float4 s_box[kRenderThreads];
  __shared__ uint32_t s_item[kRenderThreads];
  __shared__ float s_g[9][kRenderThreads];
  __shared__ float s_wsum[kRenderThreads];     // I_i of the batch's entries (optional output)
  __shared__ uint32_t s_wfix[kRenderThreads];  // the same in 2^-24 fixed point (optional output)
  __shared__ uint8_t s_list[kWarps][kRenderThreads];   // the batch entries each warp walks
  // per-pixel state, indexed by the pixel's thread id (warp w owns 32w..32w+31)
  __shared__ float4 s_pg[kRenderThreads];     // dL/dI (r, g, b) and I . dL/dI
  // transmittance before the next chunk, sum of w (c . g) so far, n_contrib
  __shared__ float4 s_st[kRenderThreads];
  __shared__ uint32_t s_warp_nc[kWarps];

  const uint32_t tile_u = P.order ? P.order[blockIdx.x] : (uint32_t)blockIdx.x;
  if (tile_u >= (uint32_t)P.total_tiles) {        // an order that names no tile: record, touch nothing
    if (threadIdx.x == 0) atomicOr(P.status, kStatusBounds);
    return;
  }
  const int tile = (int)tile_u;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_view = find_view(P.views, P.n_views, tile);
    s_max_nc = 0;
  }
  __syncthreads();
  const ViewDev& V = P.views[s_view];
  const uint2 range = P.ranges[tile];
  const bool want_w = B.weight_sum != nullptr;
  uint32_t my_nc = 0;
  {
    int px, py;
    pixel_of(V, tile, tid, &px, &py);
    const bool inside = px < V.width && py < V.height;
    float4 pg = make_float4(0.f, 0.f, 0.f, 0.f);
    if (inside) {
      const int64_t pix = V.pixel_base + (int64_t)py * V.width + px;
      const int64_t hw = (int64_t)V.width * V.height;
      const int64_t o3 = 3 * V.pixel_base + (int64_t)py * V.width + px;
      pg.x = B.dL_dimage[o3];
      pg.y = B.dL_dimage[o3 + hw];
      pg.z = B.dL_dimage[o3 + 2 * hw];
      pg.w = B.image[o3] * pg.x + B.image[o3 + hw] * pg.y + B.image[o3 + 2 * hw] * pg.z;
      my_nc = B.n_contrib[pix];
    }
    s_pg[tid] = pg;
    s_st[tid] = make_float4(1.f, 0.f, __uint_as_float(my_nc), 0.f);
    const uint32_t wm = __reduce_max_sync(0xffffffffu, my_nc);
    if (lane == 0) {
      s_warp_nc[warp] = wm;
      atomicMax(&s_max_nc, wm);
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) s_g[k][tid] = 0.f;
  s_wsum[tid] = 0.f;
  s_wfix[tid] = 0u;
  __syncthreads();
  const uint32_t max_nc = s_max_nc;
  const uint32_t warp_nc = s_warp_nc[warp];
  int bx, by;
  pixel_of(V, tile, warp * 32, &bx, &by);        // this warp's first pixel
  const float bxf = (float)bx + 0.5f, byf = (float)by + 0.5f;
  const uint32_t lt_mask = (1u << lane) - 1u;

  for (uint32_t bstart = 0; bstart < max_nc; bstart += kRenderThreads) {
    const int nb = (int)min(max_nc - bstart, (uint32_t)kRenderThreads);
    if (tid < nb) {
      const uint32_t item = list_item(P, (uint64_t)range.x + bstart + tid);
      s_item[tid] = item;
      const float4 a = P.xy_tau_z[item];
      s_xy[tid] = make_float2(a.x, a.y);
      s_ex[tid] = exponent_form(P.conic_o[item]);
      const float4 c = P.rgb[item];
      s_rgb[tid] = c;
      s_box[tid] = support_box(a.x, a.y, c.w);
    }
    __syncthreads();
    // the batch entries this warp walks: list position before the last
    // blended position of its pixels, support box meeting its 8x4 block and
    // the exponent able to pass the threshold in the block
    int cnt = 0;
    for (int k0 = 0; k0 < nb; k0 += 32) {
      const int k = k0 + lane;
      bool hit = k < nb && bstart + (uint32_t)k < warp_nc && box_meets_block(s_box[k], bxf, byf);
      if (hit) hit = block_may_blend(s_ex[k], s_xy[k].x, s_xy[k].y, bxf, byf, P.e_min);
      const uint32_t bal = __ballot_sync(0xffffffffu, hit);
      if (hit) s_list[warp][cnt + __popc(bal & lt_mask)] = (uint8_t)k;
      cnt += __popc(bal);
    }
    // chunks of 64 entries, one pixel per step; a tail of at most 32, 16 or
    // 8 entries is walked 2, 4 or 8 pixels per step
    const BwdShared M{s_xy, s_ex, s_rgb, s_pg, s_st, s_g, s_wsum, s_wfix};
    for (int c = 0; c < cnt;) {
      const int rest = cnt - c;
      if (rest > 32) {
        bwd_walk_chunk<kFix, 1>(P, M, s_list[warp], c, cnt, bstart, my_nc, warp, lane, bxf, byf, want_w);
        c += 64;
      } else if (rest > 16) {
        bwd_walk_chunk<kFix, 2>(P, M, s_list[warp], c, cnt, bstart, my_nc, warp, lane, bxf, byf, want_w);
        c += 32;
      } else if (rest > 8) {
        bwd_walk_chunk<kFix, 4>(P, M, s_list[warp], c, cnt, bstart, my_nc, warp, lane, bxf, byf, want_w);
        c += 16;
      } else {
        bwd_walk_chunk<kFix, 8>(P, M, s_list[warp], c, cnt, bstart, my_nc, warp, lane, bxf, byf, want_w);
        c += 8;
      }
    }
    __syncthreads();
    if (tid < nb) {
      const int64_t item = s_item[tid];
      float v[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        v[k] = s_g[k][tid];
        s_g[k][tid] = 0.f;
      }
      float4* dst = B.grad2d + 2 * item;
      if (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f)
        atomicAdd(dst, make_float4(v[0], v[1], v[2], v[3]));
      if (v[4] != 0.f || v[5] != 0.f || v[6] != 0.f || v[7] != 0.f)
        atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
      if (v[8] != 0.f) atomicAdd(&B.grad2d_b[item], v[8]);
      if (kFix) {
        const uint32_t wf = s_wfix[tid];
        s_wfix[tid] = 0u;
        if (wf) atomicAdd(reinterpret_cast<unsigned long long*>(B.weight_sum_fixed) + item, (unsigned long long)wf);
      }
      if (want_w) {
        const float ws = s_wsum[tid];
        s_wsum[tid] = 0.f;
        if (ws != 0.f) atomicAdd(&B.weight_sum[item], ws);
      }
    }
    __syncthreads();
  }
}

RenderParams make_params(const ViewDev* views, int n_views, int64_t n, const uint2* ranges, const uint32_t* vals,
                         const ItemState& st, const gs_config& cfg) {
  RenderParams P;
  P.views = views;
  P.n_views = n_views;
  P.n = n;
  P.ranges = ranges;
  P.vals = vals;
  P.xy_tau_z = st.xy_tau_z;
  P.conic_o = st.conic_o;
  P.rgb = st.rgb;
  P.depth_frame = st.depth_frame;
  P.status = st.status;
  P.n_entries = st.n_entries;
  P.order = nullptr;
  P.total_tiles = 0;
  P.alpha_max = cfg.alpha_max;
  P.e_min = (float)log2((double)cfg.alpha_min);
  P.t_min = cfg.t_min;
  P.bg[0] = cfg.bg[0];
  P.bg[1] = cfg.bg[1];
  P.bg[2] = cfg.bg[2];
  return P;
}

}  // namespace

cudaError_t launch_render_fwd(const ViewDev* views, int n_views, int64_t n, int total_tiles, const uint2* ranges,
                              const uint32_t* vals, const uint32_t* order, const ItemState& st, const gs_config& cfg,
                              const gs_fwd_outputs& out, cudaStream_t stream) {
  RenderParams P = make_params(views, n_views, n, ranges, vals, st, cfg);
  P.order = order;
  P.total_tiles = total_tiles;
  FwdOut O{out.image, out.final_T, out.n_contrib, out.imax, out.wmax, out.depth, out.depth_blend,
           out.weight_sum, out.max_area, out.weight_sum_fixed, out.depth_center, out.n_blended};
  if (total_tiles > 0) {
    // instances by the optional outputs: I_i collected here, blended-entry
    // counts, blended depth
    using Kernel = void (*)(RenderParams, FwdOut);
    static const Kernel kInstances[8] = {
        render_fwd_kernel<false, false, false>, render_fwd_kernel<false, false, true>,
        render_fwd_kernel<false, true, false>,  render_fwd_kernel<false, true, true>,
        render_fwd_kernel<true, false, false>,  render_fwd_kernel<true, false, true>,
        render_fwd_kernel<true, true, false>,   render_fwd_kernel<true, true, true>};
    const bool w = O.weight_sum || O.weight_sum_fixed;
    const Kernel k = kInstances[(w ? 4 : 0) | (O.n_blended ? 2 : 0) | (O.depth_blend ? 1 : 0)];
    GS_TIMED("render_fwd", stream, (k<<<total_tiles, kFwdThreads, 0, stream>>>(P, O)));
  }
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const ViewDev* views, int n_views, int64_t n, int total_tiles, const uint2* ranges,
                              const uint32_t* vals, const ItemState& st, const gs_config& cfg,
                              const float* dL_dimage, const float* image, const uint32_t* n_contrib,
                              float4* grad2d, float* grad2d_b, float* weight_sum, uint64_t* weight_sum_fixed,
                              cudaStream_t stream) {
  RenderParams P = make_params(views, n_views, n, ranges, vals, st, cfg);
  P.total_tiles = total_tiles;                   // tiles in id order (no launch order)
  BwdIn B{dL_dimage, image, n_contrib, grad2d, grad2d_b, weight_sum, weight_sum_fixed};
  if (total_tiles > 0) {
    if (weight_sum_fixed)
      GS_TIMED("render_bwd", stream, (render_bwd_kernel<true><<<total_tiles, kRenderThreads, 0, stream>>>(P, B)));
    else
      GS_TIMED("render_bwd", stream, (render_bwd_kernel<false><<<total_tiles, kRenderThreads, 0, stream>>>(P, B)));
  }
  return cudaGetLastError();
}

}  // namespace gs
