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
// Backward: per pixel, entries are replayed back to front from n_contrib,
// recovering T_k by division, and the nine per-entry gradients
// (centre 2, conic 3, opacity 1, colour 3) are reduced across the warp with
// shuffles before touching shared memory, then added to the per-item
// gradient buffer with one vector atomic per (tile, entry).
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
  const float* final_T;
  const uint32_t* n_contrib;
  float4* grad2d;               // 3 x float4 per item
};

__device__ __forceinline__ void atomic_add_f4(float4* addr, float4 v) {
  atomicAdd(addr, v);
}

__global__ void __launch_bounds__(kRenderThreads) render_bwd_kernel(RenderParams P, BwdIn B) {
  __shared__ int s_view;
  __shared__ uint32_t s_max_nc;
  __shared__ float2 s_xy[kRenderThreads];
  __shared__ float4 s_co[kRenderThreads];
  __shared__ float4 s_rgb[kRenderThreads];
  __shared__ uint32_t s_item[kRenderThreads];
  __shared__ float s_g[9][kRenderThreads];

  const int tile = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    s_view = find_view(P.views, P.n_views, tile);
    s_max_nc = 0;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) s_g[k][tid] = 0.f;
  __syncthreads();
  const ViewDev& V = P.views[s_view];
  int px, py;
  pixel_of(V, tile, &px, &py);
  const bool inside = px < V.width && py < V.height;
  const float fxp = (float)px + 0.5f, fyp = (float)py + 0.5f;
  const uint2 range = P.ranges[tile];

  float T = 1.f, Tfin = 1.f, dpix[3] = {0.f, 0.f, 0.f};
  uint32_t nc = 0;
  if (inside) {
    const int64_t pix = V.pixel_base + (int64_t)py * V.width + px;
    const int64_t hw = (int64_t)V.width * V.height;
    const float* g = B.dL_dimage + 3 * V.pixel_base + (int64_t)py * V.width + px;
    dpix[0] = g[0];
    dpix[1] = g[hw];
    dpix[2] = g[2 * hw];
    Tfin = B.final_T[pix];
    T = Tfin;
    nc = B.n_contrib[pix];
  }
  {
    const uint32_t wm = __reduce_max_sync(0xffffffffu, nc);
    if (lane == 0) atomicMax(&s_max_nc, wm);
  }
  __syncthreads();
  const uint32_t max_nc = s_max_nc;
  const float bg_dot = P.bg[0] * dpix[0] + P.bg[1] * dpix[1] + P.bg[2] * dpix[2];
  float acc[3] = {0.f, 0.f, 0.f}, last_alpha = 0.f, last_col[3] = {0.f, 0.f, 0.f};

  for (int bend = (int)max_nc; bend > 0; bend -= kRenderThreads) {
    const int bstart = max(bend - kRenderThreads, 0);
    const int nb = bend - bstart;
    __syncthreads();
    if (tid < nb) {
      const uint32_t item = P.vals[range.x + bstart + tid];
      s_item[tid] = item;
      const float4 a = P.xy_tau_z[item];
      s_xy[tid] = make_float2(a.x, a.y);
      s_co[tid] = P.conic_o[item];
      s_rgb[tid] = P.rgb[item];
    }
    __syncthreads();
    for (int jj = nb - 1; jj >= 0; --jj) {
      const uint32_t pos = (uint32_t)(bstart + jj);
      float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool act = false;
      if (pos < nc) {
        const float2 m = s_xy[jj];
        const float4 co = s_co[jj];
        const float dx = fxp - m.x, dy = fyp - m.y;
        float G;
        bool clamped;
        const float alpha = splat_alpha(co, dx, dy, P.alpha_max, &G, &clamped);
        if (alpha >= P.alpha_min) {
          act = true;
          const float one_m = 1.f - alpha;
          T = T / one_m;
          const float w = alpha * T;
          const float4 c = s_rgb[jj];
          g[6] = w * dpix[0];
          g[7] = w * dpix[1];
          g[8] = w * dpix[2];
          acc[0] = last_alpha * last_col[0] + (1.f - last_alpha) * acc[0];
          acc[1] = last_alpha * last_col[1] + (1.f - last_alpha) * acc[1];
          acc[2] = last_alpha * last_col[2] + (1.f - last_alpha) * acc[2];
          float dal = (c.x - acc[0]) * dpix[0] + (c.y - acc[1]) * dpix[1] + (c.z - acc[2]) * dpix[2];
          dal *= T;
          last_alpha = alpha;
          last_col[0] = c.x;
          last_col[1] = c.y;
          last_col[2] = c.z;
          dal += -Tfin / one_m * bg_dot;
          if (!clamped) {
            const float dG = co.w * dal;
            g[5] = G * dal;
            const float dq = -0.5f * G * dG;
            g[2] = dq * dx * dx;
            g[3] = dq * 2.f * dx * dy;
            g[4] = dq * dy * dy;
            // d = pixel - centre, so dq/dcentre = -(2 A dx + 2 B dy, 2 B dx + 2 C dy)
            g[0] = -dq * (2.f * co.x * dx + 2.f * co.y * dy);
            g[1] = -dq * (2.f * co.y * dx + 2.f * co.z * dy);
          }
        }
      }
      if (__any_sync(0xffffffffu, act)) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          const float s = warp_sum(g[k]);
          if (lane == 0 && s != 0.f) atomicAdd(&s_g[k][jj], s);
        }
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
                              const float* dL_dimage, const float* final_T, const uint32_t* n_contrib,
                              float4* grad2d, cudaStream_t stream) {
  RenderParams P = make_params(views, n_views, n, ranges, vals, st, cfg);
  BwdIn B{dL_dimage, final_T, n_contrib, grad2d};
  if (total_tiles > 0) GS_TIMED("render_bwd", stream, (render_bwd_kernel<<<total_tiles, kRenderThreads, 0, stream>>>(P, B)));
  return cudaGetLastError();
}

}  // namespace gs
