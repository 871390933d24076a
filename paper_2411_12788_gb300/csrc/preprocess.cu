// Per-(view, Gaussian) projection (Sec. 3.1) and its backward pass.
//
// Forward, one thread per Gaussian, looping over the views so that the
// Gaussian's attributes (236 B at SH degree 3) are read from HBM once:
//   covariance Sigma = R(q) diag(s^2) R(q)^T, EWA projection
//   cov2d = J W Sigma W^T J^T + lowpass I, conic = cov2d^{-1}, centre, SH
//   colour in the viewing direction, the frame for the midpoint depth
//   (Sec. 4.1), the candidate tile rectangle and, warp-cooperatively, the
//   exact number of tiles whose pixel-centre rectangle meets the support
//   q <= 2 ln(o / alpha_min).
// SH rows are staged through shared memory with coalesced loads.
#include "project.cuh"

namespace gs {

namespace {

constexpr int kPreThreads = 128;
constexpr float kLog2eF = 1.4426950408889634f;
constexpr float kLn2F = 0.6931471805599453f;

struct PreParams {
  const float* means;
  const float* scales;
  const float* rots;
  const float* opac;
  const float* sh;
  int64_t n;
  int sh_degree, sh_coeffs;
  const ViewDev* views;
  int n_views;
  const uint8_t* mask;
  float znear, lowpass, alpha_min;
  ItemState st;
};

__global__ void __launch_bounds__(kPreThreads) preprocess_kernel(PreParams P) {
  extern __shared__ float s_sh[];                 // [kPreThreads][used*3 + 1]
  const int used = (P.sh_degree + 1) * (P.sh_degree + 1);
  const int row = used * 3 + 1;                   // odd stride: no bank conflicts
  const int64_t i0 = (int64_t)blockIdx.x * kPreThreads;
  const int64_t i = i0 + threadIdx.x;
  const bool live = i < P.n;
  const int lane = threadIdx.x & 31;

  // stage this block's SH rows (first `used` coefficients of each)
  {
    const int per = used * 3;
    const int64_t rows = (P.n - i0 < kPreThreads) ? (P.n - i0) : (int64_t)kPreThreads;
    for (int f = threadIdx.x; f < rows * per; f += kPreThreads) {
      int g = f / per, c = f - g * per;
      s_sh[g * row + c] = P.sh[(i0 + g) * (int64_t)P.sh_coeffs * 3 + c];
    }
  }
  __syncthreads();

  float3 p = make_float3(0.f, 0.f, 0.f);
  float sig[6] = {0, 0, 0, 0, 0, 0};                // Sigma_00,01,02,11,12,22
  float RRq[9];
  float s0 = 1.f, s1 = 1.f, s2 = 1.f, o = 0.f;
  float Rq[9];
  if (live) {
    p = make_float3(P.means[3 * i], P.means[3 * i + 1], P.means[3 * i + 2]);
    s0 = P.scales[3 * i];
    s1 = P.scales[3 * i + 1];
    s2 = P.scales[3 * i + 2];
    float4 q = reinterpret_cast<const float4*>(P.rots)[i];
    float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    quat_to_rot(q.x * inv, q.y * inv, q.z * inv, q.w * inv, Rq);
    o = P.opac[i];
    float M[9] = {Rq[0] * s0, Rq[1] * s1, Rq[2] * s2, Rq[3] * s0, Rq[4] * s1, Rq[5] * s2,
                  Rq[6] * s0, Rq[7] * s1, Rq[8] * s2};
    sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
  }
  const float tau = 2.f * logf(o / P.alpha_min);
  const float* my_sh = s_sh + threadIdx.x * row;

  for (int v = 0; v < P.n_views; ++v) {
    const ViewDev& V = P.views[v];
    const int64_t item = (int64_t)v * P.n + i;
    bool vis = live && tau > 0.f;
    if (vis && P.mask) vis = P.mask[item] != 0;
    float3 pc = make_float3(0.f, 0.f, 1.f);
    if (vis) {
      pc.x = V.R[0] * p.x + V.R[1] * p.y + V.R[2] * p.z + V.t[0];
      pc.y = V.R[3] * p.x + V.R[4] * p.y + V.R[5] * p.z + V.t[1];
      pc.z = V.R[6] * p.x + V.R[7] * p.y + V.R[8] * p.z + V.t[2];
      vis = pc.z > P.znear;
    }
    float mx = 0.f, my = 0.f, A = 0.f, B = 0.f, C = 0.f, cxx = 0.f, cyy = 0.f;
    if (vis) {
      const float iz = 1.f / pc.z;
      const float txr = fminf(fmaxf(pc.x * iz, -V.limx), V.limx);
      const float tyr = fminf(fmaxf(pc.y * iz, -V.limy), V.limy);
      const float J00 = V.fx * iz, J02 = -V.fx * txr * iz;
      const float J11 = V.fy * iz, J12 = -V.fy * tyr * iz;
      float T0[3], T1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        T0[k] = J00 * V.R[k] + J02 * V.R[6 + k];
        T1[k] = J11 * V.R[3 + k] + J12 * V.R[6 + k];
      }
      // S T0, S T1 with S = Sigma
      float ST0[3] = {sig[0] * T0[0] + sig[1] * T0[1] + sig[2] * T0[2],
                      sig[1] * T0[0] + sig[3] * T0[1] + sig[4] * T0[2],
                      sig[2] * T0[0] + sig[4] * T0[1] + sig[5] * T0[2]};
      float ST1[3] = {sig[0] * T1[0] + sig[1] * T1[1] + sig[2] * T1[2],
                      sig[1] * T1[0] + sig[3] * T1[1] + sig[4] * T1[2],
                      sig[2] * T1[0] + sig[4] * T1[1] + sig[5] * T1[2]};
      cxx = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + P.lowpass;
      const float cxy = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
      cyy = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + P.lowpass;
      const float det = cxx * cyy - cxy * cxy;
      vis = det > 0.f;
      if (vis) {
        const float idet = 1.f / det;
        A = cyy * idet;
        B = -cxy * idet;
        C = cxx * idet;
        mx = V.fx * pc.x * iz + V.cx;
        my = V.fy * pc.y * iz + V.cy;
      }
    }
    // candidate rectangle of tiles
    uint2 rect = make_uint2(0u, 0u);
    int area = 0;
    if (vis) {
      const float rx = sqrtf(tau * cxx), ry = sqrtf(tau * cyy);
      const float fx0 = fmaxf(ceilf((mx - rx - 15.5f) * (1.f / kTile)), 0.f);
      const float fx1 = fminf(floorf((mx + rx - 0.5f) * (1.f / kTile)), (float)(V.tiles_x - 1));
      const float fy0 = fmaxf(ceilf((my - ry - 15.5f) * (1.f / kTile)), 0.f);
      const float fy1 = fminf(floorf((my + ry - 0.5f) * (1.f / kTile)), (float)(V.tiles_y - 1));
      if (fx0 <= fx1 && fy0 <= fy1) {
        int tx0 = (int)fx0, tx1 = (int)fx1, ty0 = (int)fy0, ty1 = (int)fy1;
        rect = make_uint2((uint32_t)tx0 | ((uint32_t)ty0 << 16), (uint32_t)tx1 | ((uint32_t)ty1 << 16));
        area = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
      } else {
        vis = false;
      }
    }

    // exact tile count, warp-cooperatively over the warp's candidate tiles
    uint32_t total;
    const uint32_t excl = warp_exclusive_sum((uint32_t)area, &total);
    uint32_t my_count = 0;
    for (uint32_t base = 0; base < total; base += 32) {
      const uint32_t c = base + lane;
      const int own = warp_owner(excl, min(c, total - 1));
      const float omx = __shfl_sync(0xffffffffu, mx, own), omy = __shfl_sync(0xffffffffu, my, own);
      const float oA = __shfl_sync(0xffffffffu, A, own), oB = __shfl_sync(0xffffffffu, B, own);
      const float oC = __shfl_sync(0xffffffffu, C, own), otau = __shfl_sync(0xffffffffu, tau, own);
      const uint32_t orx = __shfl_sync(0xffffffffu, rect.x, own), ory = __shfl_sync(0xffffffffu, rect.y, own);
      const uint32_t oex = __shfl_sync(0xffffffffu, excl, own);
      bool hit = false;
      if (c < total) {
        const int tx0 = orx & 0xffff, ty0 = orx >> 16, nx = (int)(ory & 0xffff) - tx0 + 1;
        const int k = (int)(c - oex);
        hit = tile_touched(omx, omy, oA, oB, oC, otau, tx0 + k % nx, ty0 + k / nx);
      }
      const uint32_t hits = __ballot_sync(0xffffffffu, hit);
      // lanes of this chunk that belong to me: [lo, hi)
      const int lo = (int)min(max((int64_t)excl - (int64_t)base, (int64_t)0), (int64_t)32);
      const int hi = (int)min(max((int64_t)excl + area - (int64_t)base, (int64_t)0), (int64_t)32);
      if (hi > lo) {
        const uint32_t bits = (hi - lo == 32) ? 0xffffffffu : (((1u << (hi - lo)) - 1u) << lo);
        my_count += __popc(hits & bits);
      }
    }
    if (!live) continue;
    if (my_count == 0) vis = false;
    P.st.tiles[item] = vis ? my_count : 0u;
    P.st.depth_key[item] = vis ? __float_as_uint(pc.z) : kCulledKey;
    if (!vis) continue;
    P.st.rect[item] = rect;
    P.st.xy_tau_z[item] = make_float4(mx, my, tau, pc.z);
    P.st.conic_o[item] = make_float4(A, B, C, o);

    // colour (Sec. 3.1): SH in the direction camera centre -> Gaussian
    float dx = p.x - V.campos[0], dy = p.y - V.campos[1], dz = p.z - V.campos[2];
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= il;
    dy *= il;
    dz *= il;
    float Y[16];
    sh_eval(P.sh_degree, dx, dy, dz, Y);
    float r = 0.5f, g = 0.5f, b = 0.5f;
    for (int k = 0; k < used; ++k) {
      r += Y[k] * my_sh[3 * k];
      g += Y[k] * my_sh[3 * k + 1];
      b += Y[k] * my_sh[3 * k + 2];
    }
    P.st.rgb[item] = make_float4(fmaxf(r, 0.f), fmaxf(g, 0.f), fmaxf(b, 0.f), 0.f);

    // midpoint-depth frame: W = diag(1/s) (R Rq)^T maps camera offsets to the
    // unit-sphere frame of the ellipsoid x^2/sx^2 + y^2/sy^2 + z^2/sz^2 = 1
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
}

// ---- backward ------------------------------------------------------------

struct PreBwdParams {
  const float* means;
  const float* scales;
  const float* rots;
  const float* opac;
  const float* sh;
  int64_t n;
  int sh_degree, sh_coeffs;
  const ViewDev* views;
  int n_views;
  float lowpass;
  const uint32_t* tiles;
  const float4* grad2d;   // 3 x float4 per item: (mx, my, A, B), (C, o, r, g), (b, -, -, -)
  float* d_means;
  float* d_scales;
  float* d_rots;
  float* d_opac;
  float* d_sh;
  float* d_mean2d_abs;
};

__global__ void __launch_bounds__(kPreThreads) preprocess_backward_kernel(PreBwdParams P) {
  const int64_t i = (int64_t)blockIdx.x * kPreThreads + threadIdx.x;
  if (i >= P.n) return;
  const int used = (P.sh_degree + 1) * (P.sh_degree + 1);
  const float3 p = make_float3(P.means[3 * i], P.means[3 * i + 1], P.means[3 * i + 2]);
  const float s[3] = {P.scales[3 * i], P.scales[3 * i + 1], P.scales[3 * i + 2]};
  const float4 q = reinterpret_cast<const float4*>(P.rots)[i];
  const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  const float qinv = rsqrtf(qn2);
  const float qw = q.x * qinv, qx = q.y * qinv, qy = q.z * qinv, qz = q.w * qinv;
  float Rq[9];
  quat_to_rot(qw, qx, qy, qz, Rq);
  const float M[9] = {Rq[0] * s[0], Rq[1] * s[1], Rq[2] * s[2], Rq[3] * s[0], Rq[4] * s[1], Rq[5] * s[2],
                      Rq[6] * s[0], Rq[7] * s[1], Rq[8] * s[2]};
  const float sig[6] = {M[0] * M[0] + M[1] * M[1] + M[2] * M[2], M[0] * M[3] + M[1] * M[4] + M[2] * M[5],
                        M[0] * M[6] + M[1] * M[7] + M[2] * M[8], M[3] * M[3] + M[4] * M[4] + M[5] * M[5],
                        M[3] * M[6] + M[4] * M[7] + M[5] * M[8], M[6] * M[6] + M[7] * M[7] + M[8] * M[8]};
  const float* shrow = P.sh + i * (int64_t)P.sh_coeffs * 3;
  const float opac_i = P.opac[i];

  float dp[3] = {0.f, 0.f, 0.f};
  float dSig[6] = {0, 0, 0, 0, 0, 0};       // symmetric dL/dSigma (00,01,02,11,12,22)
  float dop = 0.f, m2abs = 0.f;
  float dsh[48];
  for (int k = 0; k < used * 3; ++k) dsh[k] = 0.f;
  bool any = false;

  for (int v = 0; v < P.n_views; ++v) {
    const int64_t item = (int64_t)v * P.n + i;
    if (P.tiles[item] == 0) continue;
    any = true;
    const ViewDev& V = P.views[v];
    const float4 g0 = P.grad2d[3 * item], g1 = P.grad2d[3 * item + 1], g2 = P.grad2d[3 * item + 2];
    // the render backward differentiates the exponent form
    // e = log2 o - log2(e) (A dx^2 / 2 + B dx dy + C dy^2 / 2): convert to (A, B, C, o)
    const float dmx = g0.x, dmy = g0.y;
    const float dA = -0.5f * kLog2eF * g0.z, dB = -kLog2eF * g0.w, dC = -0.5f * kLog2eF * g1.x;
    dop += g1.y / (opac_i * kLn2F);
    m2abs += sqrtf(dmx * dmx + dmy * dmy);
    const float drgb[3] = {g1.z, g1.w, g2.x};

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
    float dvx = p.x - V.campos[0], dvy = p.y - V.campos[1], dvz = p.z - V.campos[2];
    const float il = rsqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
    const float dx = dvx * il, dy = dvy * il, dz = dvz * il;
    float Y[16];
    sh_eval(P.sh_degree, dx, dy, dz, Y);
    float raw[3] = {0.5f, 0.5f, 0.5f};
    for (int k = 0; k < used; ++k) {
      raw[0] += Y[k] * shrow[3 * k];
      raw[1] += Y[k] * shrow[3 * k + 1];
      raw[2] += Y[k] * shrow[3 * k + 2];
    }
    const float dr[3] = {raw[0] >= 0.f ? drgb[0] : 0.f, raw[1] >= 0.f ? drgb[1] : 0.f,
                         raw[2] >= 0.f ? drgb[2] : 0.f};
    float cdot[16];
    for (int k = 0; k < used; ++k) {
      dsh[3 * k] += Y[k] * dr[0];
      dsh[3 * k + 1] += Y[k] * dr[1];
      dsh[3 * k + 2] += Y[k] * dr[2];
      cdot[k] = shrow[3 * k] * dr[0] + shrow[3 * k + 1] * dr[1] + shrow[3 * k + 2] * dr[2];
    }
    if (P.sh_degree > 0) {
      float gdir[3] = {0.f, 0.f, 0.f};
      sh_grad_dot(P.sh_degree, dx, dy, dz, cdot, gdir);
      const float proj = gdir[0] * dx + gdir[1] * dy + gdir[2] * dz;
      dp[0] += (gdir[0] - proj * dx) * il;
      dp[1] += (gdir[1] - proj * dy) * il;
      dp[2] += (gdir[2] - proj * dz) * il;
    }
  }
  if (!any) return;

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

  P.d_means[3 * i] += dp[0];
  P.d_means[3 * i + 1] += dp[1];
  P.d_means[3 * i + 2] += dp[2];
  P.d_scales[3 * i] += ds[0];
  P.d_scales[3 * i + 1] += ds[1];
  P.d_scales[3 * i + 2] += ds[2];
  P.d_rots[4 * i] += dqw;
  P.d_rots[4 * i + 1] += dqx;
  P.d_rots[4 * i + 2] += dqy;
  P.d_rots[4 * i + 3] += dqz;
  P.d_opac[i] += dop;
  float* dshrow = P.d_sh + i * (int64_t)P.sh_coeffs * 3;
  for (int k = 0; k < used * 3; ++k) dshrow[k] += dsh[k];
  if (P.d_mean2d_abs) P.d_mean2d_abs[i] += m2abs;
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
  P.sh_degree = sc.sh_degree;
  P.sh_coeffs = sc.sh_coeffs;
  P.views = views;
  P.n_views = n_views;
  P.mask = mask;
  P.znear = cfg.znear;
  P.lowpass = cfg.lowpass;
  P.alpha_min = cfg.alpha_min;
  P.st = st;
  const int used = (sc.sh_degree + 1) * (sc.sh_degree + 1);
  const size_t smem = (size_t)kPreThreads * (used * 3 + 1) * sizeof(float);
  const int blocks = ceil_div(sc.n, kPreThreads);
  if (blocks > 0) GS_TIMED("preprocess", stream, (preprocess_kernel<<<blocks, kPreThreads, smem, stream>>>(P)));
  return cudaGetLastError();
}

cudaError_t launch_preprocess_backward(const gs_scene& sc, const ViewDev* views, int n_views, const gs_config& cfg,
                                       const uint32_t* tiles, const float4* grad2d, const gs_grads& gr,
                                       cudaStream_t stream) {
  PreBwdParams P;
  P.means = sc.means;
  P.scales = sc.scales;
  P.rots = sc.rotations;
  P.opac = sc.opacities;
  P.sh = sc.sh;
  P.n = sc.n;
  P.sh_degree = sc.sh_degree;
  P.sh_coeffs = sc.sh_coeffs;
  P.views = views;
  P.n_views = n_views;
  P.lowpass = cfg.lowpass;
  P.tiles = tiles;
  P.grad2d = grad2d;
  P.d_means = gr.d_means;
  P.d_scales = gr.d_scales;
  P.d_rots = gr.d_rotations;
  P.d_opac = gr.d_opacities;
  P.d_sh = gr.d_sh;
  P.d_mean2d_abs = gr.d_mean2d_abs;
  const int blocks = ceil_div(sc.n, kPreThreads);
  if (blocks > 0)
    GS_TIMED("preprocess_backward", stream, (preprocess_backward_kernel<<<blocks, kPreThreads, 0, stream>>>(P)));
  return cudaGetLastError();
}

}  // namespace gs
