// Device helpers for the per-Gaussian projection (Sec. 3.1): quaternion
// rotation, real spherical harmonics up to degree 3 and the exact
// row-by-row tile coverage of a Gaussian's support.  Shared by the preprocess, binning and backward
// kernels so that every call site evaluates bit-identical arithmetic.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace gs {

// Rotation matrix of the unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// Real SH basis constants (Condon-Shortley phase, m = -l..l), written as the
// polynomial coefficients of Y_lm on the unit sphere:
//   band 0: 1/(2 sqrt(pi))
//   band 1: sqrt(3/(4 pi))                      * (-y, z, -x)
//   band 2: sqrt(15/pi)/2 xy, -sqrt(15/pi)/2 yz, sqrt(5/pi)/4 (2z^2-x^2-y^2),
//           -sqrt(15/pi)/2 xz, sqrt(15/pi)/4 (x^2-y^2)
//   band 3: -sqrt(35/(2pi))/4 y(3x^2-y^2), sqrt(105/pi)/2 xyz,
//           -sqrt(21/(2pi))/4 y(4z^2-x^2-y^2), sqrt(7/pi)/4 z(2z^2-3x^2-3y^2),
//           -sqrt(21/(2pi))/4 x(4z^2-x^2-y^2), sqrt(105/pi)/4 z(x^2-y^2),
//           -sqrt(35/(2pi))/4 x(x^2-3y^2)
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.4886025119029199f;
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kSH2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float kSH3a = 0.5900435899266435f;   // sqrt(35/(2pi))/4
constexpr float kSH3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float kSH3c = 0.4570457994644658f;   // sqrt(21/(2pi))/4
constexpr float kSH3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kSH3e = 1.445305721320277f;    // sqrt(105/pi)/4

// Y[k] for k < (degree+1)^2 at the unit direction (x, y, z).
__device__ __forceinline__ void sh_eval(int degree, float x, float y, float z, float* Y) {
  Y[0] = kSH0;
  if (degree < 1) return;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  if (degree < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSH2a * x * y;
  Y[5] = -kSH2a * y * z;
  Y[6] = kSH2b * (2.f * zz - xx - yy);
  Y[7] = -kSH2a * x * z;
  Y[8] = kSH2c * (xx - yy);
  if (degree < 3) return;
  Y[9] = -kSH3a * y * (3.f * xx - yy);
  Y[10] = kSH3b * x * y * z;
  Y[11] = -kSH3c * y * (4.f * zz - xx - yy);
  Y[12] = kSH3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kSH3c * x * (4.f * zz - xx - yy);
  Y[14] = kSH3e * z * (xx - yy);
  Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

// Accumulates sum_k c[k] * grad Y_k(x, y, z) (gradient of the polynomial
// forms above, x, y, z treated as independent) into g.
__device__ __forceinline__ void sh_grad_dot(int degree, float x, float y, float z, const float* c, float* g) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (degree >= 1) {
    gy += -kSH1 * c[1];
    gz += kSH1 * c[2];
    gx += -kSH1 * c[3];
  }
  if (degree >= 2) {
    gx += kSH2a * y * c[4];
    gy += kSH2a * x * c[4];
    gy += -kSH2a * z * c[5];
    gz += -kSH2a * y * c[5];
    gx += -2.f * kSH2b * x * c[6];
    gy += -2.f * kSH2b * y * c[6];
    gz += 4.f * kSH2b * z * c[6];
    gx += -kSH2a * z * c[7];
    gz += -kSH2a * x * c[7];
    gx += 2.f * kSH2c * x * c[8];
    gy += -2.f * kSH2c * y * c[8];
  }
  if (degree >= 3) {
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += -6.f * kSH3a * x * y * c[9];
    gy += -kSH3a * (3.f * xx - 3.f * yy) * c[9];
    gx += kSH3b * y * z * c[10];
    gy += kSH3b * x * z * c[10];
    gz += kSH3b * x * y * c[10];
    gx += 2.f * kSH3c * x * y * c[11];
    gy += -kSH3c * (4.f * zz - xx - 3.f * yy) * c[11];
    gz += -8.f * kSH3c * y * z * c[11];
    gx += -6.f * kSH3d * x * z * c[12];
    gy += -6.f * kSH3d * y * z * c[12];
    gz += kSH3d * (6.f * zz - 3.f * xx - 3.f * yy) * c[12];
    gx += -kSH3c * (4.f * zz - 3.f * xx - yy) * c[13];
    gy += 2.f * kSH3c * x * y * c[13];
    gz += -8.f * kSH3c * x * z * c[13];
    gx += 2.f * kSH3e * x * z * c[14];
    gy += -2.f * kSH3e * y * z * c[14];
    gz += kSH3e * (xx - yy) * c[14];
    gx += -kSH3a * (3.f * xx - 3.f * yy) * c[15];
    gy += 6.f * kSH3a * x * y * c[15];
  }
  g[0] += gx;
  g[1] += gy;
  g[2] += gz;
}

// Exact tile rows of the support q <= tau, one row of tiles at a time.
//
// With the 2-D covariance S = [[Sxx, Sxy], [Sxy, Syy]] (S = conic^-1), the
// support at height dy (offset from the centre) is the x-interval
//   k dy -+ sc sqrt(tau - dy^2 / Syy),  k = Sxy / Syy,  sc^2 = det(S) / Syy,
// the x | y decomposition of the Mahalanobis distance.  Over a band of rows
// dy in [lo, hi] the union of these intervals is [xa, xb]: the right end is
// concave in dy with its maximum rx = sqrt(tau Sxx) at dy = ys =
// Sxy sqrt(tau / Sxx) (the ellipse's rightmost point), the left end mirrors
// it at -ys.  Tile column tx of a tile row is touched iff its pixel-centre
// range [16 tx + 0.5, 16 tx + 15.5] meets [mx + xa, mx + xb]; that is the
// same set as "the minimum of q over the tile's pixel-centre rectangle is
// <= tau".  Counting (preprocess) and emitting (duplicate) call this with
// the same stored parameters and explicitly rounded arithmetic, so both
// produce the same tiles.
struct BinParams {
  float mx, my, tau;   // centre and support bound
  float k, sc, isyy;   // x | y decomposition
  float h, rx, ys;     // half-height sqrt(tau Syy), half-width, y of the rightmost point
};

// The row parameters of an exact support q(d) <= tau of the 2-D covariance
// (Sxx, Syy, Sxy) with determinant det: x | y decomposition x = k y +- sc
// sqrt(tau - y^2 / Syy), half-height sqrt(tau Syy), half-width sqrt(tau Sxx)
// reached at y = ys.  Explicitly rounded operations, so that every kernel
// that rebuilds them from the same inputs gets the same bits.
__device__ __forceinline__ BinParams bin_params_exact(float mx, float my, float tau, float sxx, float syy, float sxy,
                                                      float det) {
  BinParams b;
  b.mx = mx;
  b.my = my;
  b.tau = tau;
  b.k = __fdiv_rn(sxy, syy);
  b.sc = __fsqrt_rn(__fdiv_rn(det, syy));
  b.isyy = __frcp_rn(syy);
  b.h = __fsqrt_rn(__fmul_rn(tau, syy));
  b.rx = __fsqrt_rn(__fmul_rn(tau, sxx));
  b.ys = __fmul_rn(sxy, __fsqrt_rn(__fdiv_rn(tau, sxx)));
  return b;
}

// The square of half-width r: with tau = 1, no slope, no y-dependence and
// the extreme points out of reach, the row functions return the square's
// rows and columns.
__device__ __forceinline__ BinParams bin_params_square(float mx, float my, float r) {
  BinParams b;
  b.mx = mx;
  b.my = my;
  b.tau = 1.f;
  b.k = 0.f;
  b.sc = r;
  b.isyy = 0.f;
  b.h = r;
  b.rx = r;
  b.ys = INFINITY;
  return b;
}

// An item's binning record, two float4 written by the preprocess: the inputs
// of its row parameters, (mx, my, tau, Sxx), (Syy, Sxy, det, first band row)
// for an exact support (det > 0) or (mx, my, 1, r), (0, 0, -1, first band
// row) for a square of half-width r.  The consumers rebuild the parameters
// with the functions above, so one 32-byte read per item serves them.
__device__ __forceinline__ BinParams bin_decode(float4 r0, float4 r1) {
  return r1.z > 0.f ? bin_params_exact(r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z) : bin_params_square(r0.x, r0.y, r0.w);
}

__device__ __forceinline__ bool row_tiles(const BinParams& b, int ty, int tiles_x, int* tx_a, int* tx_b) {
  const float lo = __fsub_rn((float)(ty * kTile) + 0.5f, b.my);
  const float hi = __fadd_rn(lo, (float)(kTile - 1));
  const float a = fmaxf(lo, -b.h), c = fminf(hi, b.h);
  if (a > c) return false;
  const float ra = __fmul_rn(b.sc, __fsqrt_rn(fmaxf(__fmaf_rn(-__fmul_rn(a, a), b.isyy, b.tau), 0.f)));
  const float rc = __fmul_rn(b.sc, __fsqrt_rn(fmaxf(__fmaf_rn(-__fmul_rn(c, c), b.isyy, b.tau), 0.f)));
  const float xb = (b.ys >= a && b.ys <= c) ? b.rx : fmaxf(__fmaf_rn(b.k, a, ra), __fmaf_rn(b.k, c, rc));
  const float xa = (-b.ys >= a && -b.ys <= c) ? -b.rx : fminf(__fmaf_rn(b.k, a, -ra), __fmaf_rn(b.k, c, -rc));
  const float fa = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(b.mx, xa), (float)kTile - 0.5f), 1.f / kTile));
  const float fb = floorf(__fmul_rn(__fsub_rn(__fadd_rn(b.mx, xb), 0.5f), 1.f / kTile));
  const int ia = (int)fmaxf(fa, 0.f);
  const int ib = (int)fminf(fb, (float)(tiles_x - 1));
  *tx_a = ia;
  *tx_b = ib;
  return ia <= ib;
}

// Rows [ty0, ty1] of tiles whose pixel-centre band meets [my - h, my + h].
__device__ __forceinline__ bool tile_rows(const BinParams& b, int tiles_y, int* ty0, int* ty1) {
  const float f0 = ceilf(__fmul_rn(__fsub_rn(__fsub_rn(b.my, b.h), (float)kTile - 0.5f), 1.f / kTile));
  const float f1 = floorf(__fmul_rn(__fsub_rn(__fadd_rn(b.my, b.h), 0.5f), 1.f / kTile));
  *ty0 = (int)fmaxf(f0, 0.f);
  *ty1 = (int)fminf(f1, (float)(tiles_y - 1));
  return *ty0 <= *ty1;
}

// Support half-extents of an item for the backward kernel's per-block
// culling, packed as two halves in the colour's fourth component.
//
// The render kernels decide membership pixel by pixel with the FP32 exponent
// e = log2 o + a2 dx^2 + b2 dx dy + c2 dy^2 >= log2(alpha_min), whose rounding
// error is bounded by a few ulp times S = |A| dx^2 + 2|B||dx dy| + |C| dy^2,
// plus an absolute part from log2 o and the threshold.  For the 2-D
// covariance S2 with eigenvalues l_max >= l_min and kappa = l_max / l_min,
// S <= 4 kappa q, while outside the box [-f rx, f rx] (rx = sqrt(tau Sxx))
// q >= f^2 tau.  The relative error of q is at most about 3e-6 kappa (a few
// roundings of the evaluation and of the conic), so with f = 1.02 + 4e-6 kappa
// no pixel outside the box passes while f^2 (1 - 3e-6 kappa) > 1, which holds
// up to kappa = 2e5 (an axis ratio of about 450, where the FP32 exponent has
// lost most of its digits near the support edge anyway).  The term
// 2e-3 sqrt(Sxx) covers the absolute part (q error up to 4e-6) and 0.5 px more
// the rounding of the box ends.  The result is rounded up to half precision,
// so the box contains every pixel whose exponent test can pass.  Beyond
// kappa = 2e5 (or for a kappa that is not a finite number) the argument does
// not hold, and the extent is infinite: the box then meets every block and
// only the exact exponent test of the backward (block_may_blend) culls.
constexpr float kSupportKappaMax = 2e5f;

__device__ __forceinline__ float support_extent(float r, float s_diag, float kappa) {
  if (!(kappa <= kSupportKappaMax)) return INFINITY;
  return fmaf(fmaf(4e-6f, kappa, 1.02f), r, fmaf(2e-3f, sqrtf(s_diag), 0.5f));
}

__device__ __forceinline__ float pack_extent(float ex, float ey) {
  const __half2 h = __halves2half2(__float2half_ru(ex), __float2half_ru(ey));
  return __uint_as_float(*reinterpret_cast<const uint32_t*>(&h));
}

__device__ __forceinline__ float2 unpack_extent(float packed) {
  const uint32_t u = __float_as_uint(packed);
  return __half22float2(*reinterpret_cast<const __half2*>(&u));
}

}  // namespace gs
