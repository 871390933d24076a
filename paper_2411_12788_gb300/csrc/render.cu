// Per-tile front-to-back alpha blending (Eq. 1) and its reverse replay.
//
// One CTA of 256 threads per 16x16 tile, one thread per pixel; each warp
// owns an 8x4 block of the tile so that a Gaussian's footprint touches few
// warps.  The tile's depth-ordered list is streamed through shared memory in
// batches of 256 entries ({centre, conic, opacity, colour, depth}, gathered
// by item id); a thread stops when its transmittance would drop below t_min
// and the CTA leaves the list once all its pixels have stopped.
//
// Forward side outputs (what the paper's reorganisation reads): i_max =
// argmax_i w_i with its weight, the midpoint depth d^mid_{i_max} (Eq. 2,
// Sec. 4.1) evaluated once per pixel from the winner's ellipsoid frame, the
// blended depth sum_i w_i z_i, the per-Gaussian accumulated weight I_i
// (Sec. 3.2; warp-reduced, then one shared-memory add per warp and one
// global atomic per (tile, entry)) and the maximum-contribution area S_i
// (Sec. 4.1; warp-aggregated atomics).
//
// Backward: one lane per entry, a warp walking its pixels front to back with
// lane scans for the transmittance and the colour in front (see the kernel),
// so each entry's nine gradients (centre 2, conic 3, opacity 1, colour 3)
// accumulate in registers; they are combined across the CTA's warps in
// shared memory and added to the per-item gradient buffer with one vector
// atomic per (tile, entry).
#include "project.cuh"

namespace gs {

namespace {

constexpr int kRenderThreads = kTilePixels;

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
  float alpha_max, alpha_min, t_min;
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

// alpha = min(alpha_max, o exp(-q/2)) with explicit rounding so that the
// forward and backward kernels make identical skip decisions.
__device__ __forceinline__ float splat_alpha(float4 co, float dx, float dy, float alpha_max, float* G_out,
                                             bool* clamped) {
  const float q = conic_q(co.x, co.y, co.z, dx, dy);
  const float G = __expf(__fmul_rn(-0.5f, q));
  const float a = __fmul_rn(co.w, G);
  *G_out = G;
  *clamped = a > alpha_max;
  return fminf(alpha_max, a);
}

__device__ __forceinline__ int find_view(const ViewDev* views, int n_views, int tile) {
  int v = 0;
  for (int k = 1; k < n_views; ++k)
    if (views[k].tile_base <= tile) v = k;
  return v;
}

__device__ __forceinline__ void pixel_of(const ViewDev& V, int tile, int* px, int* py) {
  const int local = tile - V.tile_base;
  const int tx = local % V.tiles_x, ty = local / V.tiles_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  *px = tx * kTile + (warp & 1) * 8 + (lane & 7);
  *py = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void __launch_bounds__(kRenderThreads) render_fwd_kernel(RenderParams P, FwdOut O) {
  __shared__ int s_view;
  __shared__ float2 s_xy[kRenderThreads];
  __shared__ float4 s_co[kRenderThreads];
  __shared__ float4 s_rgbz[kRenderThreads];
  __shared__ uint32_t s_item[kRenderThreads];
  __shared__ float s_wsum[kRenderThreads];

  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) s_view = find_view(P.views, P.n_views, tile);
  s_wsum[tid] = 0.f;
  __syncthreads();
  const ViewDev& V = P.views[s_view];
  int px, py;
  pixel_of(V, tile, &px, &py);
  const bool inside = px < V.width && py < V.height;
  const float fxp = (float)px + 0.5f, fyp = (float)py + 0.5f;
  const uint2 range = P.ranges[tile];
  const bool want_w = O.weight_sum != nullptr;

  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dblend = 0.f, wmax = 0.f;
  int64_t imax_item = -1;
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
      s_co[tid] = P.conic_o[item];
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
        const float4 co = s_co[j];
        float G;
        bool cl;
        const float alpha = splat_alpha(co, fxp - m.x, fyp - m.y, P.alpha_max, &G, &cl);
        if (alpha >= P.alpha_min) {
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
              imax_item = s_item[j];
            }
            T = Tn;
            last = bstart - range.x + j + 1;
          }
        }
      }
      if (want_w && __any_sync(0xffffffffu, w > 0.f)) {
        const float s = warp_sum(w);
        if (lane == 0) atomicAdd(&s_wsum[j], s);
      }
    }
    __syncthreads();
    if (want_w && tid < nb) {
      const float s = s_wsum[tid];
      if (s > 0.f) atomicAdd(&O.weight_sum[s_item[tid]], s);
      s_wsum[tid] = 0.f;
    }
  }

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
};

__device__ __forceinline__ void atomic_add_f4(float4* addr, float4 v) {
  atomicAdd(addr, v);
}

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
// its entry's nine gradients over the pixels in registers, so no per-entry
// reduction across pixels is needed.  Entries at or after a pixel's
// n_contrib and entries with alpha < alpha_min do not take part, exactly as
// in the forward pass.
__global__ void __launch_bounds__(kRenderThreads) render_bwd_kernel(RenderParams P, BwdIn B) {
  constexpr int kWarps = kRenderThreads / 32;
  __shared__ int s_view;
  __shared__ uint32_t s_max_nc;
  __shared__ float2 s_xy[kRenderThreads];
  __shared__ float4 s_co[kRenderThreads];
  __shared__ float4 s_rgb[kRenderThreads];
  __shared__ uint32_t s_item[kRenderThreads];
  __shared__ float s_g[9][kRenderThreads];
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
  // this thread's pixel: load its state
  {
    int px, py;
    pixel_of(V, tile, &px, &py);
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
  __syncthreads();
  const uint32_t max_nc = s_max_nc;
  const uint32_t warp_nc = s_warp_nc[warp];
  // pixel centres of this warp's 32 pixels (same layout as pixel_of)
  const int local = tile - V.tile_base;
  const float tx0 = (float)((local % V.tiles_x) * kTile) + (float)((warp & 1) * 8) + 0.5f;
  const float ty0 = (float)((local / V.tiles_x) * kTile) + (float)((warp >> 1) * 4) + 0.5f;

  for (uint32_t bstart = 0; bstart < max_nc; bstart += kRenderThreads) {
    const int nb = (int)min(max_nc - bstart, (uint32_t)kRenderThreads);
    if (tid < nb) {
      const uint32_t item = P.vals[range.x + bstart + tid];
      s_item[tid] = item;
      const float4 a = P.xy_tau_z[item];
      s_xy[tid] = make_float2(a.x, a.y);
      s_co[tid] = P.conic_o[item];
      s_rgb[tid] = P.rgb[item];
    }
    __syncthreads();
    for (int c = 0; c < nb; c += 32) {
      const uint32_t c0 = bstart + c;
      if (c0 >= warp_nc) break;
      const int e = c + lane;                         // my entry in the batch
      const bool valid = e < nb;
      const float2 m = valid ? s_xy[e] : make_float2(0.f, 0.f);
      const float4 co = valid ? s_co[e] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 col = valid ? s_rgb[e] : make_float4(0.f, 0.f, 0.f, 0.f);
      const uint32_t pos = c0 + lane;
      float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int p = 0; p < 32; ++p) {
        const int pt = warp * 32 + p;                 // the pixel's thread id
        const uint32_t nc = s_nc[pt];
        if (c0 >= nc) continue;                       // pixel stopped before this chunk
        const float dx = tx0 + (float)(p & 7) - m.x, dy = ty0 + (float)(p >> 3) - m.y;
        float G;
        bool clamped;
        const float alpha = splat_alpha(co, dx, dy, P.alpha_max, &G, &clamped);
        const bool act = valid && pos < nc && alpha >= P.alpha_min;
        if (!__any_sync(0xffffffffu, act)) continue;
        const float a = act ? alpha : 0.f;
        // exclusive product of (1 - a) over lanes, continued from s_T
        float prod = 1.f - a;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float t = __shfl_up_sync(0xffffffffu, prod, off);
          if (lane >= off) prod *= t;
        }
        float excl = __shfl_up_sync(0xffffffffu, prod, 1);
        if (lane == 0) excl = 1.f;
        const float T0 = s_T[pt];
        const float Tl = T0 * excl;
        const float w = a * Tl;
        const float4 pg = s_pg[pt];
        const float cg = col.x * pg.x + col.y * pg.y + col.z * pg.z;
        float fs = w * cg;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float t = __shfl_up_sync(0xffffffffu, fs, off);
          if (lane >= off) fs += t;
        }
        const float F0 = s_F[pt];
        const float total_prod = __shfl_sync(0xffffffffu, prod, 31);
        const float total_fs = __shfl_sync(0xffffffffu, fs, 31);
        __syncwarp();
        if (lane == 0) {
          s_T[pt] = T0 * total_prod;
          s_F[pt] = F0 + total_fs;
        }
        if (act) {
          acc[6] += w * pg.x;
          acc[7] += w * pg.y;
          acc[8] += w * pg.z;
          if (!clamped) {
            const float dal = Tl * cg - (pg.w - (F0 + fs)) / (1.f - a);
            acc[5] += G * dal;
            const float dq = -0.5f * G * co.w * dal;
            acc[2] += dq * dx * dx;
            acc[3] += dq * 2.f * dx * dy;
            acc[4] += dq * dy * dy;
            // d = pixel - centre, so dq/dcentre = -(2 A dx + 2 B dy, 2 B dx + 2 C dy)
            acc[0] -= dq * (2.f * co.x * dx + 2.f * co.y * dy);
            acc[1] -= dq * (2.f * co.y * dx + 2.f * co.z * dy);
          }
        }
      }
      if (valid) {
#pragma unroll
        for (int k = 0; k < 9; ++k)
          if (acc[k] != 0.f) atomicAdd(&s_g[k][e], acc[k]);
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
      if (v[0] != 0.f || v[1] != 0.f || v[2] != 0.f || v[3] != 0.f) atomic_add_f4(dst, make_float4(v[0], v[1], v[2], v[3]));
      if (v[4] != 0.f || v[5] != 0.f || v[6] != 0.f || v[7] != 0.f) atomic_add_f4(dst + 1, make_float4(v[4], v[5], v[6], v[7]));
      if (v[8] != 0.f) atomicAdd(&dst[2].x, v[8]);
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
  P.alpha_min = cfg.alpha_min;
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
  if (total_tiles > 0) GS_TIMED("render_fwd", stream, (render_fwd_kernel<<<total_tiles, kRenderThreads, 0, stream>>>(P, O)));
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const ViewDev* views, int n_views, int64_t n, int total_tiles, const uint2* ranges,
                              const uint32_t* vals, const ItemState& st, const gs_config& cfg,
                              const float* dL_dimage, const float* image, const uint32_t* n_contrib,
                              float4* grad2d, cudaStream_t stream) {
  RenderParams P = make_params(views, n_views, n, ranges, vals, st, cfg);
  BwdIn B{dL_dimage, image, n_contrib, grad2d};
  if (total_tiles > 0) GS_TIMED("render_bwd", stream, (render_bwd_kernel<<<total_tiles, kRenderThreads, 0, stream>>>(P, B)));
  return cudaGetLastError();
}

}  // namespace gs
