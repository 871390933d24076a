// Per-tile front-to-back alpha blending (Eq. 1) and its derivative.
//
// One CTA of 256 threads per 16x16 tile; each warp owns an 8x4 block of the
// tile.  The tile's depth-ordered list is streamed through shared memory in
// batches of 256 entries, gathered by item id.  Per entry the batch holds its
// centre, colour, depth and the 2-D Gaussian in exponent form:
//   alpha_raw(x) = o exp(-q/2) = 2^e,  e = log2 o + a2 dx^2 + b2 dx dy + c2 dy^2
// with (a2, b2, c2) = -log2(e) (A/2, B, C/2) for the conic (A, B, C).  An entry
// takes part at a pixel iff e >= log2(alpha_min) (that is alpha >= alpha_min);
// then alpha = min(alpha_max, 2^e).  Forward and backward evaluate e with the
// same explicitly rounded operations, so they make identical decisions.
//
// Forward (one thread per pixel): front-to-back blending with a per-pixel
// stop before T (1 - alpha) < t_min, the CTA leaving the list once all its
// pixels stopped.  Side outputs (what the paper's reorganisation reads):
// i_max = argmax_i w_i and w_max, the midpoint depth d^mid_{i_max} (Eq. 2,
// Sec. 4.1) evaluated once per pixel from the winner's ellipsoid frame, the
// blended depth sum_i w_i z_i, the per-Gaussian accumulated weight I_i
// (Sec. 3.2; each warp's weights are summed in 2^-24 fixed point by one
// redux.sync, then one shared add per warp and one global atomic per
// (tile, entry)) and the maximum-contribution area S_i (Sec. 4.1;
// warp-aggregated atomics).
//
// Backward: one lane per entry, a warp walking its pixels with lane scans
// for the transmittance and the colour in front (see render_bwd_kernel);
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
};

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
};

// Exponent form of an entry's 2-D Gaussian (identical in both kernels).
__device__ __forceinline__ float4 exponent_form(float4 co) {
  return make_float4(__fmul_rn(-0.5f * kLog2e, co.x), __fmul_rn(-kLog2e, co.y), __fmul_rn(-0.5f * kLog2e, co.z),
                     __log2f(co.w));
}

// e = lo + a2 dx^2 + b2 dx dy + c2 dy^2, explicitly rounded.
__device__ __forceinline__ float expo(float4 ex, float dx, float dy) {
  const float t = __fmaf_rn(ex.x, dx, __fmul_rn(ex.y, dy));
  const float u = __fmaf_rn(__fmul_rn(ex.z, dy), dy, ex.w);
  return __fmaf_rn(t, dx, u);
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

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

__global__ void __launch_bounds__(kRenderThreads) render_fwd_kernel(RenderParams P, FwdOut O) {
  __shared__ int s_view;
  __shared__ float2 s_xy[kRenderThreads];
  __shared__ float4 s_ex[kRenderThreads];
  __shared__ float4 s_rgbz[kRenderThreads];
  __shared__ uint32_t s_item[kRenderThreads];
  __shared__ uint32_t s_wsum[kRenderThreads];    // 2^-24 fixed point

  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) s_view = find_view(P.views, P.n_views, tile);
  s_wsum[tid] = 0u;
  __syncthreads();
  const ViewDev& V = P.views[s_view];
  int px, py;
  pixel_of(V, tile, tid, &px, &py);
  const bool inside = px < V.width && py < V.height;
  const float fxp = (float)px + 0.5f, fyp = (float)py + 0.5f;
  const uint2 range = P.ranges[tile];
  const bool want_w = O.weight_sum != nullptr;

  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dblend = 0.f, wmax = 0.f;
  int imax_pos = -1;
  uint32_t last = 0;
  bool done = !inside;

  for (uint32_t bstart = range.x; bstart < range.y; bstart += kRenderThreads) {
    if (__syncthreads_count(done) == kRenderThreads) break;
    const uint32_t idx = bstart + tid;
    if (idx < range.y) {
      const uint32_t item = P.vals[idx];
      s_item[tid] = item;
      const float4 a = P.xy_tau_z[item];
      s_xy[tid] = make_float2(a.x, a.y);
      s_ex[tid] = exponent_form(P.conic_o[item]);
      const float4 c = P.rgb[item];
      s_rgbz[tid] = make_float4(c.x, c.y, c.z, a.w);
    }
    __syncthreads();
    const int nb = (int)min(range.y - bstart, (uint32_t)kRenderThreads);
    for (int j = 0; j < nb; ++j) {
      if (__all_sync(0xffffffffu, done)) break;
      float w = 0.f;
      if (!done) {
        const float2 m = s_xy[j];
        const float e = expo(s_ex[j], fxp - m.x, fyp - m.y);
        if (e >= P.e_min) {
          const float alpha = fminf(P.alpha_max, ex2_approx(e));
          const float Tn = T * (1.f - alpha);
          if (Tn < P.t_min) {
            done = true;
          } else {
            w = alpha * T;
            const float4 c = s_rgbz[j];
            cr += w * c.x;
            cg += w * c.y;
            cb += w * c.z;
            dblend += w * c.w;
            if (w > wmax) {
              wmax = w;
              imax_pos = (int)(bstart - range.x) + j;
            }
            T = Tn;
            last = bstart - range.x + j + 1;
          }
        }
      }
      if (want_w && __any_sync(0xffffffffu, w > 0.f)) {
        const uint32_t s = __reduce_add_sync(0xffffffffu, __float2uint_rn(w * 16777216.f));
        if (lane == 0) atomicAdd(&s_wsum[j], s);
      }
    }
    __syncthreads();
    if (want_w && tid < nb) {
      const uint32_t s = s_wsum[tid];
      if (s) atomicAdd(&O.weight_sum[s_item[tid]], (float)s * (1.f / 16777216.f));
      s_wsum[tid] = 0u;
    }
  }

  const int64_t imax_item = imax_pos >= 0 ? (int64_t)P.vals[range.x + imax_pos] : -1;
  // S_i: pixels whose i_max is i (warp-aggregated)
  if (O.max_area) {
    const bool has = inside && imax_item >= 0;
    const uint32_t m = __ballot_sync(0xffffffffu, has);
    if (has) {
      const uint32_t peers = __match_any_sync(m, (unsigned long long)imax_item);
      if (lane == __ffs(peers) - 1) atomicAdd(&O.max_area[imax_item], (uint32_t)__popc(peers));
    }
  }
  if (!inside) return;
  const int64_t pix = V.pixel_base + (int64_t)py * V.width + px;
  const int64_t hw = (int64_t)V.width * V.height;
  float* img = O.image + 3 * V.pixel_base + (int64_t)py * V.width + px;
  img[0] = cr + T * P.bg[0];
  img[hw] = cg + T * P.bg[1];
  img[2 * hw] = cb + T * P.bg[2];
  O.final_T[pix] = T;
  O.n_contrib[pix] = last;
  if (O.imax) O.imax[pix] = imax_item >= 0 ? (int32_t)(imax_item - (int64_t)s_view * P.n) : -1;
  if (O.wmax) O.wmax[pix] = wmax;
  if (O.depth_blend) O.depth_blend[pix] = dblend;
  if (O.depth) {
    float d = 0.f;
    if (imax_item >= 0) {
      // d^mid: ray r(t) = t (dx, dy, 1); in the ellipsoid's unit frame the ray
      // is t Wd - e, and the chord midpoint is t = (e . Wd) / (Wd . Wd)
      const float4* df = P.depth_frame + 3 * imax_item;
      const float4 r0 = df[0], r1 = df[1], r2 = df[2];
      const float rx = (fxp - V.cx) / V.fx, ry = (fyp - V.cy) / V.fy;
      const float w0 = r0.x * rx + r0.y * ry + r0.z;
      const float w1 = r1.x * rx + r1.y * ry + r1.z;
      const float w2 = r2.x * rx + r2.y * ry + r2.z;
      d = (r0.w * w0 + r1.w * w1 + r2.w * w2) / (w0 * w0 + w1 * w1 + w2 * w2);
    }
    O.depth[pix] = d;
  }
}

struct BwdIn {
  const float* dL_dimage;
  const float* image;           // forward output c(x) + T_final bg
  const uint32_t* n_contrib;
  float4* grad2d;               // 3 x float4 per item
  float* weight_sum;            // optional: += I_i per item
};

// Backward of Eq. 1, one lane per entry.  For pixel x with blended entries
// k (alpha_k, colour c_k, w_k = alpha_k T_k) and image I = sum w_k c_k + T bg:
//   dI/dc_l     = w_l
//   dI/dalpha_l = T_l c_l - (I - F_l) / (1 - alpha_l),  F_l = sum_{k<=l} w_k c_k
// so with g = dL/dI the only per-pixel quantities a lane needs are the
// exclusive product T_l of (1 - alpha) and the inclusive sum of
// w_k (c_k . g) over the entries in front of it.  A warp takes 32 consecutive
// entries of the tile's list (one per lane) and walks its 32 pixels; both
// prefix quantities are 5-step shuffle scans across the lanes, continued from
// chunk to chunk through per-pixel state in shared memory.  Each lane sums
// its entry's gradients over the pixels in registers, so no per-entry
// reduction across pixels is needed.  Entries at or after a pixel's
// n_contrib and entries with e < log2(alpha_min) do not take part, exactly as
// in the forward pass.  With alpha_raw = 2^e unclamped, dalpha/de = alpha ln 2.
__global__ void __launch_bounds__(kRenderThreads) render_bwd_kernel(RenderParams P, BwdIn B) {
  constexpr int kWarps = kRenderThreads / 32;
  __shared__ int s_view;
  __shared__ uint32_t s_max_nc;
  __shared__ float2 s_xy[kRenderThreads];
  __shared__ float4 s_ex[kRenderThreads];
  __shared__ float4 s_rgb[kRenderThreads];
  __shared__ uint32_t s_item[kRenderThreads];
  __shared__ float s_g[9][kRenderThreads];
  __shared__ float s_wsum[kRenderThreads];     // I_i of the batch's entries (optional output)
  // per-pixel state, indexed by the pixel's thread id (warp w owns 32w..32w+31)
  __shared__ float4 s_pg[kRenderThreads];     // dL/dI (r, g, b) and I . dL/dI
  __shared__ float s_T[kRenderThreads];       // transmittance before the next chunk
  __shared__ float s_F[kRenderThreads];       // sum of w (c . g) so far
  __shared__ uint32_t s_nc[kRenderThreads];
  __shared__ uint32_t s_warp_nc[kWarps];

  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_view = find_view(P.views, P.n_views, tile);
    s_max_nc = 0;
  }
  __syncthreads();
  const ViewDev& V = P.views[s_view];
  const uint2 range = P.ranges[tile];
  {
    int px, py;
    pixel_of(V, tile, tid, &px, &py);
    const bool inside = px < V.width && py < V.height;
    float4 pg = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t nc = 0;
    if (inside) {
      const int64_t pix = V.pixel_base + (int64_t)py * V.width + px;
      const int64_t hw = (int64_t)V.width * V.height;
      const int64_t o3 = 3 * V.pixel_base + (int64_t)py * V.width + px;
      pg.x = B.dL_dimage[o3];
      pg.y = B.dL_dimage[o3 + hw];
      pg.z = B.dL_dimage[o3 + 2 * hw];
      pg.w = B.image[o3] * pg.x + B.image[o3 + hw] * pg.y + B.image[o3 + 2 * hw] * pg.z;
      nc = B.n_contrib[pix];
    }
    s_pg[tid] = pg;
    s_T[tid] = 1.f;
    s_F[tid] = 0.f;
    s_nc[tid] = nc;
    const uint32_t wm = __reduce_max_sync(0xffffffffu, nc);
    if (lane == 0) {
      s_warp_nc[warp] = wm;
      atomicMax(&s_max_nc, wm);
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) s_g[k][tid] = 0.f;
  s_wsum[tid] = 0.f;
  __syncthreads();
  const uint32_t max_nc = s_max_nc;
  const uint32_t warp_nc = s_warp_nc[warp];
  int bx, by;
  pixel_of(V, tile, warp * 32, &bx, &by);        // this warp's first pixel
  const float bxf = (float)bx + 0.5f, byf = (float)by + 0.5f;

  for (uint32_t bstart = 0; bstart < max_nc; bstart += kRenderThreads) {
    const int nb = (int)min(max_nc - bstart, (uint32_t)kRenderThreads);
    if (tid < nb) {
      const uint32_t item = P.vals[range.x + bstart + tid];
      s_item[tid] = item;
      const float4 a = P.xy_tau_z[item];
      s_xy[tid] = make_float2(a.x, a.y);
      s_ex[tid] = exponent_form(P.conic_o[item]);
      s_rgb[tid] = P.rgb[item];
    }
    __syncthreads();
    for (int c = 0; c < nb; c += 32) {
      const uint32_t c0 = bstart + c;
      if (c0 >= warp_nc) break;
      const int e_idx = c + lane;                   // my entry in the batch
      const bool valid = e_idx < nb;
      const float2 m = valid ? s_xy[e_idx] : make_float2(0.f, 0.f);
      // an invalid lane gets an exponent that never passes the e_min test
      const float4 ex = valid ? s_ex[e_idx] : make_float4(0.f, 0.f, 0.f, -1e30f);
      const float4 col = valid ? s_rgb[e_idx] : make_float4(0.f, 0.f, 0.f, 0.f);
      const uint32_t pos = c0 + lane;
      const float dx0 = bxf - m.x, dy0 = byf - m.y;
      float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float wsum = 0.f;                             // this entry's blending weight over the warp's pixels
      // pixels of this warp that are still blending at this chunk
      const uint32_t pmask = __ballot_sync(0xffffffffu, s_nc[warp * 32 + lane] > c0);
      const float a2x2 = 2.f * ex.x, c2x2 = 2.f * ex.z;
#pragma unroll
      for (int p = 0; p < 32; ++p) {
        if (!(pmask & (1u << p))) continue;
        const int pt = warp * 32 + p;                 // the pixel's thread id
        const uint32_t nc = s_nc[pt];
        const float dx = dx0 + (float)(p & 7), dy = dy0 + (float)(p >> 3);
        const float e = expo(ex, dx, dy);
        const bool act = pos < nc && e >= P.e_min;
        if (!__any_sync(0xffffffffu, act)) continue;
        const float T0 = s_T[pt];
        const float F0 = s_F[pt];
        const float4 pg = s_pg[pt];
        const float araw = ex2_approx(e);
        const float a = act ? fminf(P.alpha_max, araw) : 0.f;
        const float cg = col.x * pg.x + col.y * pg.y + col.z * pg.z;
        // one scan gives the product of (1 - a) and sum a_k cg_k prod_{j<k} (1 - a_j)
        float m = 1.f - a, f = a * cg;
        scan_affine(m, f);
        float mex = __shfl_up_sync(0xffffffffu, m, 1);     // exclusive product
        if (lane == 0) mex = 1.f;
        const float Tl = T0 * mex;
        const float w = a * Tl;
        const float Fl = fmaf(T0, f, F0);                  // sum_{k<=l} w_k cg_k
        // lane 31 holds the chunk's totals: carry the pixel's state forward
        __syncwarp();
        if (lane == 31) {
          s_T[pt] = T0 * m;
          s_F[pt] = Fl;
        }
        if (act) {
          wsum += w;
          acc[6] = fmaf(w, pg.x, acc[6]);
          acc[7] = fmaf(w, pg.y, acc[7]);
          acc[8] = fmaf(w, pg.z, acc[8]);
          if (araw <= P.alpha_max) {
            const float dal = fmaf(Tl, cg, -(pg.w - Fl) * rcp_approx(1.f - a));
            const float de = dal * a * kLn2;          // dL/de
            const float dedx = de * dx, dedy = de * dy;
            acc[5] += de;                             // d log2 o
            acc[2] = fmaf(dedx, dx, acc[2]);          // d a2
            acc[3] = fmaf(dedx, dy, acc[3]);          // d b2
            acc[4] = fmaf(dedy, dy, acc[4]);          // d c2
            // d = pixel - centre: de/dcentre = -(2 a2 dx + b2 dy, b2 dx + 2 c2 dy)
            acc[0] = fmaf(-a2x2, dedx, fmaf(-ex.y, dedy, acc[0]));
            acc[1] = fmaf(-ex.y, dedx, fmaf(-c2x2, dedy, acc[1]));
          }
        }
      }
      if (valid) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (acc[k] != 0.f) atomicAdd(&s_g[k][e_idx], acc[k]);
        if (B.weight_sum && wsum != 0.f) atomicAdd(&s_wsum[e_idx], wsum);
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
      float4* dst = B.grad2d + 3 * item;
      if (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f)
        atomicAdd(dst, make_float4(v[0], v[1], v[2], v[3]));
      if (v[4] != 0.f || v[5] != 0.f || v[6] != 0.f || v[7] != 0.f)
        atomicAdd(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
      if (v[8] != 0.f) atomicAdd(&dst[2].x, v[8]);
      if (B.weight_sum) {
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
                              const uint32_t* vals, const ItemState& st, const gs_config& cfg,
                              const gs_fwd_outputs& out, cudaStream_t stream) {
  RenderParams P = make_params(views, n_views, n, ranges, vals, st, cfg);
  FwdOut O{out.image, out.final_T, out.n_contrib, out.imax, out.wmax, out.depth, out.depth_blend,
           out.weight_sum, out.max_area};
  if (total_tiles > 0)
    GS_TIMED("render_fwd", stream, (render_fwd_kernel<<<total_tiles, kRenderThreads, 0, stream>>>(P, O)));
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const ViewDev* views, int n_views, int64_t n, int total_tiles, const uint2* ranges,
                              const uint32_t* vals, const ItemState& st, const gs_config& cfg,
                              const float* dL_dimage, const float* image, const uint32_t* n_contrib,
                              float4* grad2d, float* weight_sum, cudaStream_t stream) {
  RenderParams P = make_params(views, n_views, n, ranges, vals, st, cfg);
  BwdIn B{dL_dimage, image, n_contrib, grad2d, weight_sum};
  if (total_tiles > 0)
    GS_TIMED("render_bwd", stream, (render_bwd_kernel<<<total_tiles, kRenderThreads, 0, stream>>>(P, B)));
  return cudaGetLastError();
}

}  // namespace gs
