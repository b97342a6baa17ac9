// Device helpers of the reverse-mode kernels (k_adjoint.cu, k_adj_mdf.cu):
// warp maxima of the fixed-point bounds, 64-bit fixed-point terms, and the
// Peskin stencil with its derivative.
#pragma once

#include "mc_internal.cuh"

namespace mc {

// The largest |v| of the warp's lanes into *slot (float bits; non-negative
// floats order like their bit patterns).
__device__ __forceinline__ void warp_max_abs(unsigned* slot, float v) {
  v = fabsf(v);
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.0f) atomicMax(slot, __float_as_uint(v));
}

// A 64-bit fixed-point term (two's complement in the unsigned accumulator).
__device__ __forceinline__ unsigned long long fx64(float v) { return (unsigned long long)__float2ll_rn(v); }
__device__ __forceinline__ float fx64_value(unsigned long long q, float inv) { return (float)(long long)q * inv; }

// Peskin weights and their derivatives with respect to the bead coordinate:
// with s = sqrt(1 + 4a - 4a^2), s' = (2 - 4a)/s.
__device__ __forceinline__ void peskin4_d(float a, float w[4], float dw[4]) {
  const float s = sqrtf(fmaf(-4.0f * a, a, fmaf(4.0f, a, 1.0f)));
  const float ds = (2.0f - 4.0f * a) / s;
  const float p = 3.0f - 2.0f * a, q = 1.0f + 2.0f * a;
  w[0] = (p - s) * 0.125f;
  w[1] = (p + s) * 0.125f;
  w[2] = (q + s) * 0.125f;
  w[3] = (q - s) * 0.125f;
  dw[0] = (-2.0f - ds) * 0.125f;
  dw[1] = (-2.0f + ds) * 0.125f;
  dw[2] = (2.0f + ds) * 0.125f;
  dw[3] = (2.0f - ds) * 0.125f;
}

struct Stencil {
  float wx[4], wy[4], dx[4], dy[4];
  int ix[4], iy[4];   // wrapped column / row-start indices
};

// The stencil of the two-layer point X + d n of bead p (the forward's
// layer_cell: cell and fraction of the shifted point).
__device__ __forceinline__ Stencil make_layer_stencil(const float4& p, float2 n, float d, int W, int H) {
  int cx, cy;
  float fx, fy;
  layer_cell(p, n, d, W, H, cx, cy, fx, fy);
  Stencil s;
  peskin4_d(fx, s.wx, s.dx);
  peskin4_d(fy, s.wy, s.dy);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    s.ix[a] = wrap_once(cx - 1 + a, W);
    s.iy[a] = wrap_once(cy - 1 + a, H) * W;
  }
  return s;
}

__device__ __forceinline__ Stencil make_stencil(const float4& p, int W, int H) {
  Stencil s;
  peskin4_d(p.x, s.wx, s.dx);
  peskin4_d(p.y, s.wy, s.dy);
  const int cx = cell_x(p), cy = cell_y(p);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    s.ix[a] = wrap_once(cx - 1 + a, W);
    s.iy[a] = wrap_once(cy - 1 + a, H) * W;
  }
  return s;
}

}  // namespace mc
