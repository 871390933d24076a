// Fused photometric loss of the training step: L = (1 - lambda) L1 +
// lambda (1 - SSIM), the 3DGS objective the paper trains with (Sec. 6.2),
// and its gradient with respect to the rendered image, in one pass.
//
// SSIM per channel with an 11x11 Gaussian window (sigma 1.5, weights
// normalised to sum 1) and zero padding, C1 = 0.01^2, C2 = 0.03^2:
//   mu_x = G*x, mu_y = G*y, E_xx = G*(x x), E_yy = G*(y y), E_xy = G*(x y)
//   S = (2 mu_x mu_y + C1)(2 (E_xy - mu_x mu_y) + C2)
//       / ((mu_x^2 + mu_y^2 + C1)(E_xx - mu_x^2 + E_yy - mu_y^2 + C2))
// SSIM is the mean of S over every pixel and channel of every view (the
// views' maps concatenated).  With a = dS/dmu_x, b = dS/dE_xx, c = dS/dE_xy
// (at fixed raw moments), the derivative of sum_q S_q with respect to x_p is
//   (G*a)(p) + 2 x_p (G*b)(p) + y_p (G*c)(p)
// (the window is symmetric; a, b, c are zero outside the image).
//
// One CTA per 32x32 output tile and channel, everything in shared memory:
// x, y with a 10-pixel halo (52x52), the horizontal pass of the five moments
// (52x42, six outputs per work item from registers), their vertical pass in
// place (each column in registers, 42x42), a, b, c on that 42x42
// region, and their two blur passes back to the 32x32 tile (four outputs per
// work item).  Each CTA writes its partial L1 and SSIM sums; a one-block
// kernel adds them in double.
#include "common.cuh"

namespace gs {

namespace {

constexpr int kT = 32;                 // output tile
constexpr int kR = 5;                  // window radius
constexpr int kW = 2 * kR + 1;         // window width
constexpr int kIn = kT + 4 * kR;       // 52: input rows/cols
constexpr int kMid = kT + 2 * kR;      // 42: moment region
constexpr int kSsimThreads = 256;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

__constant__ float c_win[kW];

struct SsimView {
  int64_t base;        // offset of the view's planar [3][H][W] image
  int width, height, tiles_x, tile_base;
};

struct SsimParams {
  SsimView views[GS_MAX_VIEWS];
  int n_views;
  const float* x;
  const float* y;
  float* grad;
  float* partial;      // [2 * blocks]: L1 sum, SSIM sum
  float w_l1, w_ssim;  // (1 - lambda) / count, lambda / count
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

struct SsimSmem {
  float in[2][kIn][kIn];           // x, y; later the horizontal blur of a, b, c
  float mom[5][kIn][kMid];         // horizontal moments, then (rows < 42) vertical
};

__global__ void __launch_bounds__(kSsimThreads) l1_ssim_kernel(SsimParams P) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  SsimSmem& S = *reinterpret_cast<SsimSmem*>(s_raw);
  const int tid = threadIdx.x;
  // which view and tile
  int v = 0;
  for (int k = 1; k < P.n_views; ++k)
    if (P.views[k].tile_base <= (int)blockIdx.x) v = k;
  const SsimView V = P.views[v];
  const int local = (int)blockIdx.x - V.tile_base;
  const int ox = (local % V.tiles_x) * kT, oy = (local / V.tiles_x) * kT;
  const int ch = blockIdx.y;
  const int64_t hw = (int64_t)V.width * V.height;
  const float* X = P.x + V.base + ch * hw;
  const float* Y = P.y + V.base + ch * hw;

  // 1. x, y over [ox - 10, ox + 42) x [oy - 10, oy + 42), zero outside
  for (int i = tid; i < kIn * kIn; i += kSsimThreads) {
    const int r = i / kIn, c = i - r * kIn;
    const int gx = ox - 2 * kR + c, gy = oy - 2 * kR + r;
    const bool in = gx >= 0 && gy >= 0 && gx < V.width && gy < V.height;
    const int64_t o = (int64_t)gy * V.width + gx;
    S.in[0][r][c] = in ? X[o] : 0.f;
    S.in[1][r][c] = in ? Y[o] : 0.f;
  }
  __syncthreads();

  // 2. horizontal pass of the five moments: rows 0..51, cols 0..41, six
  //    consecutive outputs per work item from 16 loaded values
  constexpr int kHG = 6;                                  // 42 = 7 x 6
  for (int i = tid; i < kIn * (kMid / kHG); i += kSsimThreads) {
    const int r = i / (kMid / kHG), c0 = (i - r * (kMid / kHG)) * kHG;
    float xv[kHG + kW - 1], yv[kHG + kW - 1];
#pragma unroll
    for (int t = 0; t < kHG + kW - 1; ++t) {
      xv[t] = S.in[0][r][c0 + t];
      yv[t] = S.in[1][r][c0 + t];
    }
#pragma unroll
    for (int o = 0; o < kHG; ++o) {
      float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
      for (int t = 0; t < kW; ++t) {
        const float w = c_win[t], a = xv[o + t], b = yv[o + t];
        const float wx = w * a, wy = w * b;
        mx += wx;
        my += wy;
        exx = fmaf(wx, a, exx);
        eyy = fmaf(wy, b, eyy);
        exy = fmaf(wx, b, exy);
      }
      S.mom[0][r][c0 + o] = mx;
      S.mom[1][r][c0 + o] = my;
      S.mom[2][r][c0 + o] = exx;
      S.mom[3][r][c0 + o] = eyy;
      S.mom[4][r][c0 + o] = exy;
    }
  }
  __syncthreads();

  // 3. vertical pass in place: thread (q, column) holds the column's 52
  //    values in registers and writes its 42 outputs back over the first
  //    rows (the loops are unrolled, so the window needs no moves)
  if (tid < 5 * kMid) {
    const int q = tid / kMid, c = tid - q * kMid;
    float col[kIn];
#pragma unroll
    for (int r = 0; r < kIn; ++r) col[r] = S.mom[q][r][c];
#pragma unroll
    for (int r = 0; r < kMid; ++r) {
      float acc = 0.f;
#pragma unroll
      for (int t = 0; t < kW; ++t) acc = fmaf(c_win[t], col[r + t], acc);
      S.mom[q][r][c] = acc;
    }
  }
  __syncthreads();

  // 4. S and its partials a, b, c on the 42x42 region (zero outside the
  //    image); the inner 32x32 adds to the SSIM sum.  a, b, c overwrite
  //    moments 0, 2, 4 of the same point.
  float ssim_sum = 0.f;
  for (int i = tid; i < kMid * kMid; i += kSsimThreads) {
    const int r = i / kMid, c = i - r * kMid;
    const int gx = ox - kR + c, gy = oy - kR + r;
    const bool in = gx >= 0 && gy >= 0 && gx < V.width && gy < V.height;
    const float mx = S.mom[0][r][c], my = S.mom[1][r][c];
    const float exx = S.mom[2][r][c], eyy = S.mom[3][r][c], exy = S.mom[4][r][c];
    const float ln = 2.f * mx * my + kC1, ld = mx * mx + my * my + kC1;
    const float cn = 2.f * (exy - mx * my) + kC2, cd = (exx - mx * mx) + (eyy - my * my) + kC2;
    const float iden = 1.f / (ld * cd);
    const float s = ln * cn * iden;
    float a = 0.f, b = 0.f, cc = 0.f;
    if (in) {
      a = 2.f * my * (cn - ln) * iden + 2.f * mx * s * (1.f / cd - 1.f / ld);
      b = -s / cd;
      cc = 2.f * ln * iden;
      if (r >= kR && r < kR + kT && c >= kR && c < kR + kT) ssim_sum += s;
    }
    S.mom[0][r][c] = a;
    S.mom[2][r][c] = b;
    S.mom[4][r][c] = cc;
  }
  __syncthreads();

  // 5. horizontal blur of a, b, c: rows 0..41, cols 0..31, into in[] (3 planes
  //    of 42x32 laid out in the 2x52x52 buffer), four outputs per work item
  constexpr int kBG = 4;
  float* hb = &S.in[0][0][0];
  for (int i = tid; i < kMid * (kT / kBG); i += kSsimThreads) {
    const int r = i / (kT / kBG), c0 = (i - r * (kT / kBG)) * kBG;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float* src = &S.mom[2 * q][r][c0];            // planes 0, 2, 4 hold a, b, c
      float v[kBG + kW - 1];
#pragma unroll
      for (int t = 0; t < kBG + kW - 1; ++t) v[t] = src[t];
#pragma unroll
      for (int o = 0; o < kBG; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < kW; ++t) acc = fmaf(c_win[t], v[o + t], acc);
        hb[(q * kMid + r) * kT + c0 + o] = acc;
      }
    }
  }
  __syncthreads();

  // 6. vertical blur and the gradient: four consecutive rows of one column per
  //    work item (32 columns x 8 row groups = the 256 threads)
  float l1_sum = 0.f;
  {
    constexpr int kVG = 4;
    const int c = tid % kT, r0 = (tid / kT) * kVG;
    float g[3][kVG];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      float v[kVG + kW - 1];
#pragma unroll
      for (int t = 0; t < kVG + kW - 1; ++t) v[t] = hb[(q * kMid + r0 + t) * kT + c];
#pragma unroll
      for (int o = 0; o < kVG; ++o) {
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < kW; ++t) acc = fmaf(c_win[t], v[o + t], acc);
        g[q][o] = acc;
      }
    }
#pragma unroll
    for (int o = 0; o < kVG; ++o) {
      const int gx = ox + c, gy = oy + r0 + o;
      if (gx >= V.width || gy >= V.height) continue;
      const int64_t off = (int64_t)gy * V.width + gx;
      const float xv = X[off], yv = Y[off];
      const float d = xv - yv;
      l1_sum += fabsf(d);
      const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
      const float dssim = g[0][o] + 2.f * xv * g[1][o] + yv * g[2][o];
      P.grad[V.base + ch * hw + off] = P.w_l1 * sgn - P.w_ssim * dssim;
    }
  }

  // partial sums of the CTA
  l1_sum = warp_sum(l1_sum);
  ssim_sum = warp_sum(ssim_sum);
  __shared__ float s_red[2][kSsimThreads / 32];
  if ((tid & 31) == 0) {
    s_red[0][tid >> 5] = l1_sum;
    s_red[1][tid >> 5] = ssim_sum;
  }
  __syncthreads();
  if (tid == 0) {
    float a = 0.f, b = 0.f;
    for (int w = 0; w < kSsimThreads / 32; ++w) {
      a += s_red[0][w];
      b += s_red[1][w];
    }
    const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    P.partial[2 * blk] = a;
    P.partial[2 * blk + 1] = b;
  }
}

// loss = (1 - lambda) L1 / count + lambda (1 - SSIM sum / count)
__global__ void __launch_bounds__(256) l1_ssim_finish_kernel(const float* __restrict__ partial, int blocks,
                                                             double inv_count, float lambda, float* loss,
                                                             float* l1_out, float* ssim_out) {
  __shared__ double s[2][256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < blocks; i += 256) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      s[0][threadIdx.x] += s[0][threadIdx.x + off];
      s[1][threadIdx.x] += s[1][threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double l1 = s[0][0] * inv_count, ss = s[1][0] * inv_count;
    *loss = (float)((1.0 - lambda) * l1 + lambda * (1.0 - ss));
    if (l1_out) *l1_out = (float)l1;
    if (ssim_out) *ssim_out = (float)ss;
  }
}

int ssim_blocks(const gs_plan* plan) {
  int t = 0;
  for (int v = 0; v < plan->n_views; ++v)
    t += ceil_div(plan->cams[v].width, kT) * ceil_div(plan->cams[v].height, kT);
  return t;
}

}  // namespace

}  // namespace gs

using namespace gs;

extern "C" size_t gs_loss_l1_ssim_workspace_size(const gs_plan* plan) {
  if (!plan || plan->n_views < 1 || plan->n_views > GS_MAX_VIEWS) return 0;
  return align_up((size_t)2 * 3 * std::max(1, ssim_blocks(plan)) * sizeof(float));
}

extern "C" gs_status gs_loss_l1_ssim(const gs_plan* plan, const float* image, const float* target, float lambda,
                                     float* loss, float* dL_dimage, float* l1_out, float* ssim_out, void* ws,
                                     size_t ws_bytes, void* stream_) {
  if (!plan || plan->n_views < 1 || plan->n_views > GS_MAX_VIEWS || !(lambda >= 0.f && lambda <= 1.f) || !loss ||
      !ws)
    return GS_ERR_INVALID_ARG;
  const int64_t count = 3 * plan->total_pixels;
  if (count > 0 && (!image || !target || !dL_dimage)) return GS_ERR_INVALID_ARG;
  if (ws_bytes < gs_loss_l1_ssim_workspace_size(plan)) return GS_ERR_CAPACITY;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  // the window and the shared-memory limit, once per device
  static std::atomic<uint64_t> init_done{0};
  const cudaError_t ei = once_per_device(init_done, [] {
    // normalised 11-tap Gaussian, sigma 1.5
    double g[kW], sum = 0.0;
    for (int t = 0; t < kW; ++t) {
      g[t] = exp(-(double)((t - kR) * (t - kR)) / (2.0 * 1.5 * 1.5));
      sum += g[t];
    }
    float gf[kW];
    for (int t = 0; t < kW; ++t) gf[t] = (float)(g[t] / sum);
    cudaError_t e = cudaMemcpyToSymbol(c_win, gf, sizeof(gf));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(l1_ssim_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SsimSmem));
    return e;
  });
  if (ei != cudaSuccess) return GS_ERR_CUDA;
  if (count == 0) return cudaMemsetAsync(loss, 0, 4, stream) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
  SsimParams P;
  int tb = 0;
  for (int v = 0; v < plan->n_views; ++v) {
    const gs_camera& c = plan->cams[v];
    P.views[v].base = 3 * plan->pixel_base[v];
    P.views[v].width = c.width;
    P.views[v].height = c.height;
    P.views[v].tiles_x = ceil_div(c.width, kT);
    P.views[v].tile_base = tb;
    tb += ceil_div(c.width, kT) * ceil_div(c.height, kT);
  }
  P.n_views = plan->n_views;
  P.x = image;
  P.y = target;
  P.grad = dL_dimage;
  P.partial = static_cast<float*>(ws);
  P.w_l1 = (float)((1.0 - lambda) / (double)count);
  P.w_ssim = (float)(lambda / (double)count);
  GS_TIMED("loss_l1_ssim", stream,
           (l1_ssim_kernel<<<dim3((unsigned)tb, 3), kSsimThreads, sizeof(SsimSmem), stream>>>(P)));
  GS_TIMED("loss_finish", stream,
           (l1_ssim_finish_kernel<<<1, 256, 0, stream>>>(P.partial, 3 * tb, 1.0 / (double)count, lambda, loss,
                                                          l1_out, ssim_out)));
  return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
