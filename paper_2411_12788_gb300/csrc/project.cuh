// Device helpers for the per-Gaussian projection (Sec. 3.1): quaternion
// rotation, real spherical harmonics up to degree 3 and the exact
// tile-touch predicate.  Shared by the preprocess, binning and backward
// kernels so that every call site evaluates bit-identical arithmetic.
#pragma once

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

// q(d) = A dx^2 + 2 B dx dy + C dy^2 with explicitly rounded operations, so
// that every call site (counting, emitting) decides identically.
__device__ __forceinline__ float conic_q(float A, float B, float C, float dx, float dy) {
  float t = __fmul_rn(__fmul_rn(C, dy), dy);
  t = __fmaf_rn(__fmul_rn(__fmul_rn(2.f, B), dx), dy, t);
  return __fmaf_rn(__fmul_rn(A, dx), dx, t);
}

// Tile (tx, ty) is touched iff the minimum of q over its pixel-centre
// rectangle [16tx+0.5, 16tx+15.5] x [16ty+0.5, 16ty+15.5] is <= tau.  The
// minimum of the convex quadratic is 0 if the centre is inside; otherwise it
// lies on an edge, where q is a 1-D quadratic minimised at its clamped vertex.
__device__ __forceinline__ bool tile_touched(float mx, float my, float A, float B, float C, float tau, int tx,
                                             int ty) {
  const float x0 = (float)(tx * kTile) + 0.5f, x1 = x0 + (float)(kTile - 1);
  const float y0 = (float)(ty * kTile) + 0.5f, y1 = y0 + (float)(kTile - 1);
  if (mx >= x0 && mx <= x1 && my >= y0 && my <= y1) return true;
  const float lox = __fsub_rn(x0, mx), hix = __fsub_rn(x1, mx);
  const float loy = __fsub_rn(y0, my), hiy = __fsub_rn(y1, my);
  float best = INFINITY;
  // vertical edges (dx fixed): vertex at dy = -B dx / C
  {
    float dy = fminf(fmaxf(__fdiv_rn(-__fmul_rn(B, lox), C), loy), hiy);
    best = fminf(best, conic_q(A, B, C, lox, dy));
    dy = fminf(fmaxf(__fdiv_rn(-__fmul_rn(B, hix), C), loy), hiy);
    best = fminf(best, conic_q(A, B, C, hix, dy));
  }
  // horizontal edges (dy fixed): vertex at dx = -B dy / A
  {
    float dx = fminf(fmaxf(__fdiv_rn(-__fmul_rn(B, loy), A), lox), hix);
    best = fminf(best, conic_q(A, B, C, dx, loy));
    dx = fminf(fmaxf(__fdiv_rn(-__fmul_rn(B, hiy), A), lox), hix);
    best = fminf(best, conic_q(A, B, C, dx, hiy));
  }
  return best <= tau;
}

// Candidate-tile rectangle packed as (tx0 | ty0 << 16, tx1 | ty1 << 16).
__device__ __forceinline__ int rect_area(uint2 r) {
  int tx0 = r.x & 0xffff, ty0 = r.x >> 16, tx1 = r.y & 0xffff, ty1 = r.y >> 16;
  return (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
}

// Per-lane owner search for warp-cooperative tile enumeration: the lane
// `owner` with excl[owner] <= c < excl[owner] + area[owner], given each
// lane's exclusive prefix `excl` of the candidate counts.
__device__ __forceinline__ int warp_owner(uint32_t excl, uint32_t c) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    int cand = lo + step;
    uint32_t e = __shfl_sync(0xffffffffu, excl, cand & 31);
    if (cand < 32 && e <= c) lo = cand;
  }
  return lo;
}

__device__ __forceinline__ uint32_t warp_exclusive_sum(uint32_t v, uint32_t* total) {
  const int lane = threadIdx.x & 31;
  uint32_t x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += t;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

}  // namespace gs
