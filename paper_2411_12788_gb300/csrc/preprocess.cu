// Per-(view, Gaussian) projection (Sec. 3.1) and its backward pass.
//
// Forward, one thread per Gaussian, looping over the views so that the
// Gaussian's attributes (236 B at SH degree 3) are read from HBM once per
// batch: covariance Sigma = M M^T with M = R(q) diag(s), EWA projection
// cov2d = F F^T + lowpass I with F = J W M (2x3), conic = cov2d^{-1}, centre,
// SH colour in the viewing direction, the frame for the midpoint depth
// (Sec. 4.1) and the exact number of touched tiles, counted row by row with
// the interval form of the support (project.cuh, row_tiles).  det(cov2d) is
// taken from the Lagrange identity |F0|^2 |F1|^2 - (F0.F1)^2 = sum of the
// squared 2x2 minors of F, which does not cancel for thin Gaussians.
// SH rows are staged through shared memory with coalesced loads.  Both
// kernels are instantiated per SH degree so the coefficient loops unroll.
#include "project.cuh"

namespace gs {

namespace {

constexpr int kPreThreads = 64;
constexpr float kLog2eF = 1.4426950408889634f;
constexpr float kLn2F = 0.6931471805599453f;

struct PreParams {
  const float* means;
  const float* scales;
  const float* rots;
  const float* opac;
  const float* sh;
  int64_t n;
  int sh_coeffs;
  const ViewDev* views;
  int n_views;
  const uint8_t* mask;
  bool mask_bits;              // GS_FLAG_MASK_BITS: mask is [n_views][mask_words] 32-bit words
  int64_t mask_words;
  float znear, lowpass, alpha_min;
  ItemState st;
};

// A thread's SH row in shared memory: the first K coefficients (3 floats
// each) in an odd number of float4, so the row is read and written with
// 128-bit accesses and the 8 lanes of each quarter-warp phase of such an
// access fall on distinct banks.
template <int K>
__host__ __device__ constexpr int sh_row_floats() { return 4 * (((3 * K + 3) / 4) | 1); }

// Stage this block's SH rows into shared memory (row stride sh_row_floats).
template <int K, int THREADS>
__device__ __forceinline__ void stage_sh(const float* __restrict__ sh, int sh_coeffs, int64_t i0, int64_t n,
                                         float* s_sh) {
  constexpr int per = 3 * K, row = sh_row_floats<K>();
  const int64_t rows = (n - i0 < THREADS) ? (n - i0) : (int64_t)THREADS;
  if constexpr (per % 4 == 0) {
    // rows stored back to back at the degree's own width and 16-byte aligned:
    // 128-bit loads and stores (a float4 never straddles two rows)
    const float* base = sh + i0 * per;
    if (sh_coeffs == K && (reinterpret_cast<uintptr_t>(base) & 15u) == 0) {
      constexpr int q = per / 4;
      for (int f = threadIdx.x; f < rows * q; f += THREADS) {
        const int g = f / q, c4 = f - g * q;
        reinterpret_cast<float4*>(s_sh + g * row)[c4] = reinterpret_cast<const float4*>(base)[f];
      }
      return;
    }
  }
  for (int f = threadIdx.x; f < rows * per; f += THREADS) {
    const int g = f / per, c = f - g * per;
    s_sh[g * row + c] = sh[(i0 + g) * (int64_t)sh_coeffs * 3 + c];
  }
}

// acc[c] += sum_k Y_k sh[k][c] over a shared row (entry e = 3k + c), read a
// float4 at a time.
template <int K>
__device__ __forceinline__ void sh_dot_rows(const float* row, const float* Y, float* acc) {
#pragma unroll
  for (int j = 0; j < (3 * K + 3) / 4; ++j) {
    const float4 q = reinterpret_cast<const float4*>(row)[j];
    const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e = 4 * j + t;
      if (e < 3 * K) acc[e % 3] += Y[e / 3] * qv[t];
    }
  }
}

__device__ __forceinline__ void cull(const ItemState& st, int64_t item) {
  st.tiles[item] = 0u;
  st.band_rows[item] = 0u;
  st.depth_key[item] = kCulledKey;
  st.depth_val[item] = (uint32_t)item;
}

template <int DEG, bool THREE_SIGMA>
__global__ void __launch_bounds__(kPreThreads) preprocess_kernel(PreParams P) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int row = sh_row_floats<K>();
  __shared__ __align__(16) float s_sh[kPreThreads * row];
  const int64_t i0 = (int64_t)blockIdx.x * kPreThreads;
  const int64_t i = i0 + threadIdx.x;
  stage_sh<K, kPreThreads>(P.sh, P.sh_coeffs, i0, P.n, s_sh);
  __syncthreads();
  if (i >= P.n) return;

  const float3 p = make_float3(P.means[3 * i], P.means[3 * i + 1], P.means[3 * i + 2]);
  const float s0 = P.scales[3 * i], s1 = P.scales[3 * i + 1], s2 = P.scales[3 * i + 2];
  const float4 q = reinterpret_cast<const float4*>(P.rots)[i];
  const float qi = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  float Rq[9];
  quat_to_rot(q.x * qi, q.y * qi, q.z * qi, q.w * qi, Rq);
  const float o = P.opac[i];
  const float M[9] = {Rq[0] * s0, Rq[1] * s1, Rq[2] * s2, Rq[3] * s0, Rq[4] * s1, Rq[5] * s2,
                      Rq[6] * s0, Rq[7] * s1, Rq[8] * s2};
  const float tau = 2.f * logf(o / P.alpha_min);
  const float* shc = s_sh + threadIdx.x * row;     // coefficient k, channel c at [3k + c]
  const float lp = P.lowpass;
  uint32_t entries = 0;                            // touched tiles of this Gaussian's items

  for (int v = 0; v < P.n_views; ++v) {
    const ViewDev& V = P.views[v];
    const int64_t item = (int64_t)v * P.n + i;
    bool vis = tau > 0.f;
    if (vis && P.mask) {
      if (P.mask_bits)
        vis = (reinterpret_cast<const uint32_t*>(P.mask)[v * P.mask_words + (i >> 5)] >> (i & 31)) & 1u;
      else
        vis = P.mask[item] != 0;
    }
    if (!vis) {
      cull(P.st, item);
      continue;
    }
    const float3 pc = make_float3(V.R[0] * p.x + V.R[1] * p.y + V.R[2] * p.z + V.t[0],
                                  V.R[3] * p.x + V.R[4] * p.y + V.R[5] * p.z + V.t[1],
                                  V.R[6] * p.x + V.R[7] * p.y + V.R[8] * p.z + V.t[2]);
    if (!(pc.z > P.znear)) {
      cull(P.st, item);
      continue;
    }
    const float iz = 1.f / pc.z;
    const float txr = fminf(fmaxf(pc.x * iz, -V.limx), V.limx);
    const float tyr = fminf(fmaxf(pc.y * iz, -V.limy), V.limy);
    const float J00 = V.fx * iz, J02 = -V.fx * txr * iz;
    const float J11 = V.fy * iz, J12 = -V.fy * tyr * iz;
    float T0[3], T1[3], F0[3], F1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = J00 * V.R[k] + J02 * V.R[6 + k];
      T1[k] = J11 * V.R[3 + k] + J12 * V.R[6 + k];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      F0[k] = T0[0] * M[k] + T0[1] * M[3 + k] + T0[2] * M[6 + k];
      F1[k] = T1[0] * M[k] + T1[1] * M[3 + k] + T1[2] * M[6 + k];
    }
    const float f00 = F0[0] * F0[0] + F0[1] * F0[1] + F0[2] * F0[2];
    const float f11 = F1[0] * F1[0] + F1[1] * F1[1] + F1[2] * F1[2];
    const float f01 = F0[0] * F1[0] + F0[1] * F1[1] + F0[2] * F1[2];
    const float m01 = F0[0] * F1[1] - F0[1] * F1[0];
    const float m02 = F0[0] * F1[2] - F0[2] * F1[0];
    const float m12 = F0[1] * F1[2] - F0[2] * F1[1];
    const float cxx = f00 + lp, cyy = f11 + lp, cxy = f01;
    const float det = m01 * m01 + m02 * m02 + m12 * m12 + lp * (f00 + f11) + lp * lp;
    if (!(det > 0.f)) {
      cull(P.st, item);
      continue;
    }
    const float idet = 1.f / det;
    const float A = cyy * idet, B = -cxy * idet, C = cxx * idet;
    // support half-extents (exact support; they bound the culling boxes in both modes)
    const float h_sup = sqrtf(tau * cyy), rx_sup = sqrtf(tau * cxx);
    // largest eigenvalue of the 2-D covariance
    const auto eig_max = [&]() {
      const float hd = 0.5f * (cxx - cyy);
      return 0.5f * (cxx + cyy) + sqrtf(hd * hd + cxy * cxy);
    };
    float lmax = 0.f;
    const float mx = V.fx * pc.x * iz + V.cx, my = V.fy * pc.y * iz + V.cy;
    float sq_r = 0.f;
    if (THREE_SIGMA) {
      // the square of half-width r = ceil(3 sqrt(lambda_max))
      lmax = eig_max();
      sq_r = ceilf(3.f * sqrtf(lmax));
    }
    const BinParams b = THREE_SIGMA ? bin_params_square(mx, my, sq_r) : bin_params_exact(mx, my, tau, cxx, cyy, cxy, det);
    // exact tile count, row by row
    uint32_t count = 0;
    int ty0 = 0, ty1 = -1;
    if (tile_rows(b, V.tiles_y, &ty0, &ty1)) {
      for (int ty = ty0; ty <= ty1; ++ty) {
        int a, c;
        if (row_tiles(b, ty, V.tiles_x, &a, &c)) count += (uint32_t)(c - a + 1);
      }
    }
    // condition number of the 2-D covariance (for the culling boxes)
    if (!THREE_SIGMA) lmax = eig_max();
    const float kappa = lmax * lmax / det;
    P.st.tiles[item] = count;
    P.st.band_rows[item] = count ? (uint32_t)(ty1 - ty0 + 1) : 0u;
    P.st.depth_key[item] = count ? __float_as_uint(pc.z) : kCulledKey;
    P.st.depth_val[item] = (uint32_t)item;
    if (!count) continue;
    P.st.rect[item] = make_uint2((uint32_t)ty0 << 16, (uint32_t)(V.tiles_x - 1) | ((uint32_t)ty1 << 16));
    entries += count;
    P.st.xy_tau_z[item] = make_float4(b.mx, b.my, b.tau, pc.z);
    P.st.conic_o[item] = make_float4(A, B, C, o);
    // the binning record (see bin_decode) with the first band row
    P.st.bin[2 * item] = THREE_SIGMA ? make_float4(mx, my, 1.f, sq_r) : make_float4(mx, my, tau, cxx);
    P.st.bin[2 * item + 1] = THREE_SIGMA ? make_float4(0.f, 0.f, -1.f, __int_as_float(ty0))
                                         : make_float4(cyy, cxy, det, __int_as_float(ty0));

    // colour (Sec. 3.1): SH in the direction camera centre -> Gaussian
    float dx = p.x - V.campos[0], dy = p.y - V.campos[1], dz = p.z - V.campos[2];
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= il;
    dy *= il;
    dz *= il;
    float Y[16];
    sh_eval(DEG, dx, dy, dz, Y);
    float raw[3] = {0.5f, 0.5f, 0.5f};
    sh_dot_rows<K>(shc, Y, raw);
    P.st.rgb[item] = make_float4(fmaxf(raw[0], 0.f), fmaxf(raw[1], 0.f), fmaxf(raw[2], 0.f), 
                                 pack_extent(support_extent(rx_sup, cxx, kappa), support_extent(h_sup, cyy, kappa)));

    // midpoint-depth frame: W = diag(1/s) (R Rq)^T maps camera offsets to the
    // unit-sphere frame of the ellipsoid x^2/sx^2 + y^2/sy^2 + z^2/sz^2 = 1
    float RRq[9];
#pragma unroll
    for (int r3 = 0; r3 < 3; ++r3)
#pragma unroll
      for (int c3 = 0; c3 < 3; ++c3)
        RRq[r3 * 3 + c3] = V.R[r3 * 3] * Rq[c3] + V.R[r3 * 3 + 1] * Rq[3 + c3] + V.R[r3 * 3 + 2] * Rq[6 + c3];
    const float is[3] = {1.f / s0, 1.f / s1, 1.f / s2};
    float W[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      W[3 * k + 0] = RRq[0 * 3 + k] * is[k];
      W[3 * k + 1] = RRq[1 * 3 + k] * is[k];
      W[3 * k + 2] = RRq[2 * 3 + k] * is[k];
    }
    const float e0 = W[0] * pc.x + W[1] * pc.y + W[2] * pc.z;
    const float e1 = W[3] * pc.x + W[4] * pc.y + W[5] * pc.z;
    const float e2 = W[6] * pc.x + W[7] * pc.y + W[8] * pc.z;
    float4* df = P.st.depth_frame + 3 * item;
    df[0] = make_float4(W[0], W[1], W[2], e0);
    df[1] = make_float4(W[3], W[4], W[5], e1);
    df[2] = make_float4(W[6], W[7], W[8], e2);
  }
  // the entry total, summed per warp
  const uint32_t am = __activemask();
  const uint32_t we = __reduce_add_sync(am, entries);
  if ((int)(threadIdx.x & 31) == __ffs(am) - 1 && we) atomicAdd(P.st.entries_acc, (unsigned long long)we);
}

// ---- backward ------------------------------------------------------------

struct PreBwdParams {
  const float* means;
  const float* scales;
  const float* rots;
  const float* opac;
  const float* sh;
  int64_t n;
  int sh_coeffs;
  const ViewDev* views;
  int n_views;
  float lowpass;
  const uint32_t* tiles;
  const float4* grad2d;   // 2 x float4 per item: (mx, my, a2, b2), (c2, log2 o, r, g)
  const float* grad2d_b;  // 1 float per item: b
  float* d_means;
  float* d_scales;
  float* d_rots;
  float* d_opac;
  float* d_sh;
  float* d_mean2d_abs;
  bool overwrite;         // write the gradients (every row) instead of adding to them
};

constexpr int kPreBwdThreads = 32;

// One thread per Gaussian; its SH row and the row's gradient live in shared
// memory (per-thread rows, see sh_row_floats) rather than in registers: at
// degree 3 the kernel takes 128 registers and 26 KB of shared memory, 8 blocks
// per SM.
template <int DEG>
__global__ void __launch_bounds__(kPreBwdThreads) preprocess_backward_kernel(PreBwdParams P) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int row = sh_row_floats<K>();
  __shared__ __align__(16) float s_sh[kPreBwdThreads * row];
  __shared__ __align__(16) float s_dsh[kPreBwdThreads * row];
  const int64_t i0 = (int64_t)blockIdx.x * kPreBwdThreads;
  const int64_t i = i0 + threadIdx.x;
  stage_sh<K, kPreBwdThreads>(P.sh, P.sh_coeffs, i0, P.n, s_sh);
  for (int f = threadIdx.x; f < kPreBwdThreads * row; f += kPreBwdThreads) s_dsh[f] = 0.f;
  __syncthreads();
  const bool live = i < P.n;
  const float* shc = s_sh + threadIdx.x * row;      // coefficient k, channel c at [3k + c]
  float* dsh = s_dsh + threadIdx.x * row;
  float dp[3] = {0.f, 0.f, 0.f};
  float dSig[6] = {0, 0, 0, 0, 0, 0};       // symmetric dL/dSigma (00,01,02,11,12,22)
  float dop = 0.f, m2abs = 0.f;
  float Rq[9], M[9], sig[6], s[3] = {1.f, 1.f, 1.f};
  float qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f, qinv = 1.f, opac_i = 1.f;
  float3 p = make_float3(0.f, 0.f, 0.f);
  if (live) {
    p = make_float3(P.means[3 * i], P.means[3 * i + 1], P.means[3 * i + 2]);
    s[0] = P.scales[3 * i];
    s[1] = P.scales[3 * i + 1];
    s[2] = P.scales[3 * i + 2];
    const float4 q = reinterpret_cast<const float4*>(P.rots)[i];
    qinv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    qw = q.x * qinv;
    qx = q.y * qinv;
    qy = q.z * qinv;
    qz = q.w * qinv;
    opac_i = P.opac[i];
  }
  quat_to_rot(qw, qx, qy, qz, Rq);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
  sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];

  // The views in which this Gaussian has tiles, their counts loaded together;
  // the warp walks the union of its lanes' views in order (the view constants
  // stay warp-uniform), each lane's 2-D gradients loaded one view ahead.
  uint64_t vis = 0;
  if (live) {
#pragma unroll 8
    for (int v = 0; v < P.n_views; ++v) vis |= (uint64_t)(P.tiles[(int64_t)v * P.n + i] != 0u) << v;
  }
  uint64_t wvis = ((uint64_t)__reduce_or_sync(0xffffffffu, (uint32_t)(vis >> 32)) << 32) |
                  (uint64_t)__reduce_or_sync(0xffffffffu, (uint32_t)vis);
  const bool any = vis != 0;
  float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
  float n2 = 0.f;
  if (wvis) {
    const int v0 = __ffsll((long long)wvis) - 1;
    if ((vis >> v0) & 1u) {
      const int64_t item = (int64_t)v0 * P.n + i;
      n0 = P.grad2d[2 * item];
      n1 = P.grad2d[2 * item + 1];
      n2 = P.grad2d_b[item];
    }
  }
  while (wvis) {
    const int v = __ffsll((long long)wvis) - 1;
    wvis &= wvis - 1;
    const bool mine = (vis >> v) & 1u;
    const float4 g0 = n0, g1 = n1;
    const float g2 = n2;
    if (wvis) {
      const int vn = __ffsll((long long)wvis) - 1;
      if ((vis >> vn) & 1u) {
        const int64_t item = (int64_t)vn * P.n + i;
        n0 = P.grad2d[2 * item];
        n1 = P.grad2d[2 * item + 1];
        n2 = P.grad2d_b[item];
      }
    }
    if (!mine) continue;
    const ViewDev& V = P.views[v];
    // the render backward differentiates the exponent form
    // e = log2 o - log2(e) (A dx^2 / 2 + B dx dy + C dy^2 / 2): convert to (A, B, C, o)
    const float dmx = g0.x, dmy = g0.y;
    const float dA = -0.5f * kLog2eF * g0.z, dB = -kLog2eF * g0.w, dC = -0.5f * kLog2eF * g1.x;
    dop += g1.y / (opac_i * kLn2F);
    m2abs += sqrtf(dmx * dmx + dmy * dmy);
    const float drgb[3] = {g1.z, g1.w, g2};

    // recompute the forward quantities of this view
    const float px = V.R[0] * p.x + V.R[1] * p.y + V.R[2] * p.z + V.t[0];
    const float py = V.R[3] * p.x + V.R[4] * p.y + V.R[5] * p.z + V.t[1];
    const float pz = V.R[6] * p.x + V.R[7] * p.y + V.R[8] * p.z + V.t[2];
    const float iz = 1.f / pz;
    const float rx = px * iz, ry = py * iz;
    const float txr = fminf(fmaxf(rx, -V.limx), V.limx);
    const float tyr = fminf(fmaxf(ry, -V.limy), V.limy);
    const bool freex = rx > -V.limx && rx < V.limx;
    const bool freey = ry > -V.limy && ry < V.limy;
    const float J00 = V.fx * iz, J02 = -V.fx * txr * iz;
    const float J11 = V.fy * iz, J12 = -V.fy * tyr * iz;
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = J00 * V.R[k] + J02 * V.R[6 + k];
      T1[k] = J11 * V.R[3 + k] + J12 * V.R[6 + k];
    }
    const float ST0[3] = {sig[0] * T0[0] + sig[1] * T0[1] + sig[2] * T0[2],
                          sig[1] * T0[0] + sig[3] * T0[1] + sig[4] * T0[2],
                          sig[2] * T0[0] + sig[4] * T0[1] + sig[5] * T0[2]};
    const float ST1[3] = {sig[0] * T1[0] + sig[1] * T1[1] + sig[2] * T1[2],
                          sig[1] * T1[0] + sig[3] * T1[1] + sig[4] * T1[2],
                          sig[2] * T1[0] + sig[4] * T1[1] + sig[5] * T1[2]};
    const float a = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + P.lowpass;
    const float b = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
    const float c = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + P.lowpass;
    const float det = a * c - b * b;
    const float id2 = 1.f / (det * det);

    // conic (A, B, C) = (c, -b, a) / det  ->  cov2d (a, b, c)
    const float da = (-c * c * dA + b * c * dB - b * b * dC) * id2;
    const float dc = (-b * b * dA + a * b * dB - a * a * dC) * id2;
    const float db = (2.f * b * c * dA - (a * c + b * b) * dB + 2.f * a * b * dC) * id2;

    // cov2d = T Sigma T^T: dSigma += da T0T0^T + db (T0T1^T + T1T0^T)/2 + dc T1T1^T
    dSig[0] += da * T0[0] * T0[0] + db * T0[0] * T1[0] + dc * T1[0] * T1[0];
    dSig[1] += da * T0[0] * T0[1] + 0.5f * db * (T0[0] * T1[1] + T1[0] * T0[1]) + dc * T1[0] * T1[1];
    dSig[2] += da * T0[0] * T0[2] + 0.5f * db * (T0[0] * T1[2] + T1[0] * T0[2]) + dc * T1[0] * T1[2];
    dSig[3] += da * T0[1] * T0[1] + db * T0[1] * T1[1] + dc * T1[1] * T1[1];
    dSig[4] += da * T0[1] * T0[2] + 0.5f * db * (T0[1] * T1[2] + T1[1] * T0[2]) + dc * T1[1] * T1[2];
    dSig[5] += da * T0[2] * T0[2] + db * T0[2] * T1[2] + dc * T1[2] * T1[2];
    // dT0 = 2 da S T0 + db S T1, dT1 = db S T0 + 2 dc S T1
    float dT0[3], dT1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dT0[k] = 2.f * da * ST0[k] + db * ST1[k];
      dT1[k] = db * ST0[k] + 2.f * dc * ST1[k];
    }
    // T = J R
    const float dJ00 = dT0[0] * V.R[0] + dT0[1] * V.R[1] + dT0[2] * V.R[2];
    const float dJ02 = dT0[0] * V.R[6] + dT0[1] * V.R[7] + dT0[2] * V.R[8];
    const float dJ11 = dT1[0] * V.R[3] + dT1[1] * V.R[4] + dT1[2] * V.R[5];
    const float dJ12 = dT1[0] * V.R[6] + dT1[1] * V.R[7] + dT1[2] * V.R[8];
    const float iz2 = iz * iz;
    float dpc[3] = {0.f, 0.f, 0.f};
    // J00 = fx/z, J11 = fy/z, J02 = -fx txr/z, J12 = -fy tyr/z
    dpc[2] += -V.fx * iz2 * dJ00 - V.fy * iz2 * dJ11;
    dpc[2] += dJ02 * V.fx * txr * iz2 + dJ12 * V.fy * tyr * iz2;
    if (freex) {   // d txr/dx = 1/z, d txr/dz = -x/z^2
      dpc[0] += dJ02 * (-V.fx * iz) * iz;
      dpc[2] += dJ02 * (-V.fx * iz) * (-px * iz2);
    }
    if (freey) {
      dpc[1] += dJ12 * (-V.fy * iz) * iz;
      dpc[2] += dJ12 * (-V.fy * iz) * (-py * iz2);
    }
    // centre (fx x/z + cx, fy y/z + cy)
    dpc[0] += dmx * V.fx * iz;
    dpc[1] += dmy * V.fy * iz;
    dpc[2] += -dmx * V.fx * px * iz2 - dmy * V.fy * py * iz2;
    // p_c = R p + t
#pragma unroll
    for (int k = 0; k < 3; ++k) dp[k] += V.R[k] * dpc[0] + V.R[3 + k] * dpc[1] + V.R[6 + k] * dpc[2];

    // colour: rgb = max(0, sum sh Y(dir) + 0.5), dir = (p - campos)/|p - campos|
    const float dvx = p.x - V.campos[0], dvy = p.y - V.campos[1], dvz = p.z - V.campos[2];
    const float il = rsqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
    const float dx = dvx * il, dy = dvy * il, dz = dvz * il;
    float Y[16];
    sh_eval(DEG, dx, dy, dz, Y);
    float raw[3] = {0.5f, 0.5f, 0.5f};
    sh_dot_rows<K>(shc, Y, raw);
    const float dr[3] = {raw[0] >= 0.f ? drgb[0] : 0.f, raw[1] >= 0.f ? drgb[1] : 0.f,
                         raw[2] >= 0.f ? drgb[2] : 0.f};
    // dL/dsh[k][c] += Y_k dr_c and cdot_k = sum_c sh[k][c] dr_c, a float4 of
    // the row (entry e = 3k + c) at a time
    float cdot[16];
#pragma unroll
    for (int k = 0; k < K; ++k) cdot[k] = 0.f;
#pragma unroll
    for (int j = 0; j < (3 * K + 3) / 4; ++j) {
      const float4 q = reinterpret_cast<const float4*>(shc)[j];
      float4 d = reinterpret_cast<float4*>(dsh)[j];
      const float qv[4] = {q.x, q.y, q.z, q.w};
      float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = 4 * j + t;
        if (e < 3 * K) {
          dv[t] += Y[e / 3] * dr[e % 3];
          cdot[e / 3] += qv[t] * dr[e % 3];
        }
      }
      reinterpret_cast<float4*>(dsh)[j] = make_float4(dv[0], dv[1], dv[2], dv[3]);
    }
    if (DEG > 0) {
      float gdir[3] = {0.f, 0.f, 0.f};
      sh_grad_dot(DEG, dx, dy, dz, cdot, gdir);
      const float proj = gdir[0] * dx + gdir[1] * dy + gdir[2] * dz;
      dp[0] += (gdir[0] - proj * dx) * il;
      dp[1] += (gdir[1] - proj * dy) * il;
      dp[2] += (gdir[2] - proj * dz) * il;
    }
  }

  // SH gradients of the block's rows, coalesced: written whole (coefficients
  // beyond the degree get 0) or added
  __syncthreads();
  {
    constexpr int per = 3 * K;
    const int64_t rows = (P.n - i0 < kPreBwdThreads) ? (P.n - i0) : (int64_t)kPreBwdThreads;
    float* base = P.d_sh + i0 * per;
    const bool vec = per % 4 == 0 && P.sh_coeffs == K && (reinterpret_cast<uintptr_t>(base) & 15u) == 0;
    if (vec) {
      // rows back to back at the degree's own width: 128-bit accesses
      constexpr int q = per / 4 > 0 ? per / 4 : 1;
      for (int f = threadIdx.x; f < rows * q; f += kPreBwdThreads) {
        const int g = f / q, c4 = f - g * q;
        const float4 v = reinterpret_cast<const float4*>(s_dsh + g * row)[c4];
        float4* dst = reinterpret_cast<float4*>(base) + f;
        if (P.overwrite) {
          *dst = v;
        } else if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
          const float4 o = *dst;
          *dst = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
        }
      }
    } else if (P.overwrite) {
      const int full = 3 * P.sh_coeffs;
      for (int f = threadIdx.x; f < rows * full; f += kPreBwdThreads) {
        const int g = f / full, c = f - g * full;
        P.d_sh[(i0 + g) * (int64_t)full + c] = c < per ? s_dsh[g * row + c] : 0.f;
      }
    } else {
      for (int f = threadIdx.x; f < rows * per; f += kPreBwdThreads) {
        const int g = f / per, c = f - g * per;
        const float v = s_dsh[g * row + c];
        if (v != 0.f) P.d_sh[(i0 + g) * (int64_t)P.sh_coeffs * 3 + c] += v;
      }
    }
  }
  if (!live) return;
  if (!any) {
    if (P.overwrite) {     // not rendered in any view: zero gradients
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        P.d_means[3 * i + c] = 0.f;
        P.d_scales[3 * i + c] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) P.d_rots[4 * i + c] = 0.f;
      P.d_opac[i] = 0.f;
      if (P.d_mean2d_abs) P.d_mean2d_abs[i] = 0.f;
    }
    return;
  }

  // Sigma = M M^T, M = Rq diag(s): dM = 2 dSigma M
  const float G[9] = {dSig[0], dSig[1], dSig[2], dSig[1], dSig[3], dSig[4], dSig[2], dSig[4], dSig[5]};
  float dM[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      dM[3 * r + c] = 2.f * (G[3 * r] * M[c] + G[3 * r + 1] * M[3 + c] + G[3 * r + 2] * M[6 + c]);
  float ds[3], dR[9];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    ds[c] = dM[c] * Rq[c] + dM[3 + c] * Rq[3 + c] + dM[6 + c] * Rq[6 + c];
    dR[c] = dM[c] * s[c];
    dR[3 + c] = dM[3 + c] * s[c];
    dR[6 + c] = dM[6 + c] * s[c];
  }
  // rotation matrix of the unit quaternion -> (w, x, y, z)
  const float w = qw, x = qx, y = qy, z = qz;
  float dqw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
  float dqx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                     2.f * x * dR[8]);
  float dqy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                     2.f * y * dR[8]);
  float dqz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] +
                     x * dR[6] + y * dR[7]);
  // normalisation q_hat = q / |q|
  const float dotq = dqw * qw + dqx * qx + dqy * qy + dqz * qz;
  dqw = (dqw - dotq * qw) * qinv;
  dqx = (dqx - dotq * qx) * qinv;
  dqy = (dqy - dotq * qy) * qinv;
  dqz = (dqz - dotq * qz) * qinv;

  const float out[11] = {dp[0], dp[1], dp[2], ds[0], ds[1], ds[2], dqw, dqx, dqy, dqz, dop};
  float* const dst[11] = {P.d_means + 3 * i,     P.d_means + 3 * i + 1,  P.d_means + 3 * i + 2,
                          P.d_scales + 3 * i,    P.d_scales + 3 * i + 1, P.d_scales + 3 * i + 2,
                          P.d_rots + 4 * i,      P.d_rots + 4 * i + 1,   P.d_rots + 4 * i + 2,
                          P.d_rots + 4 * i + 3,  P.d_opac + i};
  if (P.overwrite) {
#pragma unroll
    for (int c = 0; c < 11; ++c) *dst[c] = out[c];
    if (P.d_mean2d_abs) P.d_mean2d_abs[i] = m2abs;
  } else {
#pragma unroll
    for (int c = 0; c < 11; ++c) *dst[c] += out[c];
    if (P.d_mean2d_abs) P.d_mean2d_abs[i] += m2abs;
  }
}

}  // namespace

cudaError_t launch_preprocess(const gs_scene& sc, const ViewDev* views, int n_views, const uint8_t* mask,
                              const gs_config& cfg, const ItemState& st, cudaStream_t stream) {
  PreParams P;
  P.means = sc.means;
  P.scales = sc.scales;
  P.rots = sc.rotations;
  P.opac = sc.opacities;
  P.sh = sc.sh;
  P.n = sc.n;
  P.sh_coeffs = sc.sh_coeffs;
  P.views = views;
  P.n_views = n_views;
  P.mask = mask;
  P.mask_bits = (cfg.flags & GS_FLAG_MASK_BITS) != 0;
  P.mask_words = (sc.n + 31) / 32;
  P.znear = cfg.znear;
  P.lowpass = cfg.lowpass;
  P.alpha_min = cfg.alpha_min;
  P.st = st;
  const int blocks = ceil_div(sc.n, kPreThreads);
  if (blocks == 0) return cudaSuccess;
  // the 3-sigma extent (GS_FLAG_EXTENT_3SIGMA) is a separate instance, so the
  // default path carries none of it
  const bool sq = (cfg.flags & GS_FLAG_EXTENT_3SIGMA) != 0;
  switch (sc.sh_degree * 2 + (sq ? 1 : 0)) {
#define GS_PRE(D, Q) \
    GS_TIMED("preprocess", stream, (preprocess_kernel<D, Q><<<blocks, kPreThreads, 0, stream>>>(P))); break
    case 0: GS_PRE(0, false);
    case 1: GS_PRE(0, true);
    case 2: GS_PRE(1, false);
    case 3: GS_PRE(1, true);
    case 4: GS_PRE(2, false);
    case 5: GS_PRE(2, true);
    case 7: GS_PRE(3, true);
    default: GS_PRE(3, false);
#undef GS_PRE
  }
  return cudaGetLastError();
}

cudaError_t launch_preprocess_backward(const gs_scene& sc, const ViewDev* views, int n_views, const gs_config& cfg,
                                       const uint32_t* tiles, const float4* grad2d, const float* grad2d_b,
                                       const gs_grads& gr, cudaStream_t stream) {
  PreBwdParams P;
  P.means = sc.means;
  P.scales = sc.scales;
  P.rots = sc.rotations;
  P.opac = sc.opacities;
  P.sh = sc.sh;
  P.n = sc.n;
  P.sh_coeffs = sc.sh_coeffs;
  P.views = views;
  P.n_views = n_views;
  P.lowpass = cfg.lowpass;
  P.tiles = tiles;
  P.grad2d = grad2d;
  P.grad2d_b = grad2d_b;
  P.d_means = gr.d_means;
  P.d_scales = gr.d_scales;
  P.d_rots = gr.d_rotations;
  P.d_opac = gr.d_opacities;
  P.d_sh = gr.d_sh;
  P.d_mean2d_abs = gr.d_mean2d_abs;
  P.overwrite = (cfg.flags & GS_FLAG_ZERO_ACCUM) != 0;
  const int blocks = ceil_div(sc.n, kPreBwdThreads);
  if (blocks == 0) return cudaSuccess;
  switch (sc.sh_degree) {
    case 0:
      GS_TIMED("preprocess_backward", stream, (preprocess_backward_kernel<0><<<blocks, kPreBwdThreads, 0, stream>>>(P)));
      break;
    case 1:
      GS_TIMED("preprocess_backward", stream, (preprocess_backward_kernel<1><<<blocks, kPreBwdThreads, 0, stream>>>(P)));
      break;
    case 2:
      GS_TIMED("preprocess_backward", stream, (preprocess_backward_kernel<2><<<blocks, kPreBwdThreads, 0, stream>>>(P)));
      break;
    default:
      GS_TIMED("preprocess_backward", stream, (preprocess_backward_kernel<3><<<blocks, kPreBwdThreads, 0, stream>>>(P)));
      break;
  }
  return cudaGetLastError();
}

}  // namespace gs
