// Per-Gaussian kernels of the FE-4DGS pass (one thread per Gaussian):
//   hexplane_split: HexPlane sample of the FST deformation query (Sec. 3.2,
//              Eq. 5-6), written as three BF16 terms for the MLP (Eq. 4),
//              which runs on the tensor cores (deform_mlp.cu);
//   gauss_fwd: the offsets applied, EWA projection (Sec. 3.3), SH colour
//              (Sec. 3.1), tile rect and depth key.  Writes the 48-byte
//              render record.
//   gauss_bwd: fixed-order sum of the per-(tile, Gaussian) partials, then
//              the reverse of projection, colour, activations and the
//              deformation query back to the canonical parameters (the MLP
//              reverse, from the forward's unit masks, on the tensor cores:
//              deform_mlp.cu).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace fe {

namespace {

// Real SH with the Condon-Shortley phase, normalisation
// K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), as polynomials of the unit
// direction.  Constants: 1/(2 sqrt(pi)); sqrt(3/(4 pi)); sqrt(15/(4 pi)),
// sqrt(5/(16 pi)), sqrt(15/(16 pi)); sqrt(35/(32 pi)), sqrt(105/(4 pi)),
// sqrt(21/(32 pi)), sqrt(7/(16 pi)), sqrt(105/(16 pi)).
constexpr float kY0 = 0.282094792f;
constexpr float kY1 = 0.488602512f;
constexpr float kY2a = 1.09254843f, kY2b = 0.315391565f, kY2c = 0.546274215f;
constexpr float kY3a = 0.59004359f, kY3b = 2.89061144f, kY3c = 0.457045799f, kY3d = 0.373176333f,
                kY3e = 1.44530572f;

__device__ __forceinline__ void sh_basis(const float d[3], float Y[16]) {
  const float x = d[0], y = d[1], z = d[2];
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = kY0;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// ddir = sum_k w[k] * grad Y_k (gradient of the polynomial extension).
__device__ __forceinline__ void sh_basis_vjp(const float d[3], const float w[16], float g[3]) {
  const float x = d[0], y = d[1], z = d[2];
  const float xx = x * x, yy = y * y, zz = z * z;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  gy += w[1] * -kY1;
  gz += w[2] * kY1;
  gx += w[3] * -kY1;
  gx += w[4] * kY2a * y;  gy += w[4] * kY2a * x;
  gy += w[5] * -kY2a * z; gz += w[5] * -kY2a * y;
  gx += w[6] * -2.f * kY2b * x; gy += w[6] * -2.f * kY2b * y; gz += w[6] * 4.f * kY2b * z;
  gx += w[7] * -kY2a * z; gz += w[7] * -kY2a * x;
  gx += w[8] * 2.f * kY2c * x; gy += w[8] * -2.f * kY2c * y;
  gx += w[9] * -6.f * kY3a * x * y; gy += w[9] * -kY3a * (3.f * xx - 3.f * yy);
  gx += w[10] * kY3b * y * z; gy += w[10] * kY3b * x * z; gz += w[10] * kY3b * x * y;
  gx += w[11] * 2.f * kY3c * x * y; gy += w[11] * -kY3c * (4.f * zz - xx - 3.f * yy); gz += w[11] * -8.f * kY3c * y * z;
  gx += w[12] * -6.f * kY3d * x * z; gy += w[12] * -6.f * kY3d * y * z;
  gz += w[12] * kY3d * (6.f * zz - 3.f * xx - 3.f * yy);
  gx += w[13] * -kY3c * (4.f * zz - 3.f * xx - yy); gy += w[13] * 2.f * kY3c * x * y; gz += w[13] * -8.f * kY3c * x * z;
  gx += w[14] * 2.f * kY3e * x * z; gy += w[14] * -2.f * kY3e * y * z; gz += w[14] * kY3e * (xx - yy);
  gx += w[15] * -kY3a * (3.f * xx - 3.f * yy); gy += w[15] * 6.f * kY3a * x * y;
  g[0] = gx; g[1] = gy; g[2] = gz;
}

__device__ __forceinline__ void load_sh(const void* sh, int bf16, int g, float c[48]) {
  if (bf16) {
    const uint4* p = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(sh) + (size_t)g * 48);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const uint4 q = __ldg(p + i);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        c[8 * i + 2 * j] = __uint_as_float(w[j] << 16);
        c[8 * i + 2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
      }
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(static_cast<const float*>(sh) + (size_t)g * 48);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float4 q = __ldg(p + i);
      c[4 * i] = q.x; c[4 * i + 1] = q.y; c[4 * i + 2] = q.z; c[4 * i + 3] = q.w;
    }
  }
}

// ---------------------------------------------------------------------------
// Deformation query
// ---------------------------------------------------------------------------
// Plane k samples coordinates (pair_a(k), pair_b(k)) of (x, y, z, t):
// xy, xz, yz, xt, yt, zt.  Compile-time so register arrays stay in registers.
__host__ __device__ constexpr int pair_a(int k) { return k < 2 ? 0 : (k == 2 ? 1 : k - 3); }
__host__ __device__ constexpr int pair_b(int k) { return k == 0 ? 1 : (k < 3 ? 2 : 3); }

struct GridPos {
  int i0, j0;
  float f0, f1;
  bool c0, c1;  // clamped at the border (zero derivative)
};

__device__ __forceinline__ void grid_coords(const GaussArgs& a, const float mu[3], float coord[4]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) coord[k] = (mu[k] - a.bmin[k]) * a.bscale[k] - 1.0f;
  coord[3] = 2.0f * a.t - 1.0f;
}

__device__ __forceinline__ GridPos grid_pos(const GaussArgs& a, float ca, float cb) {
  GridPos p;
  const float hi = (float)(a.R - 1);
  float g0 = (ca + 1.0f) * 0.5f * hi, g1 = (cb + 1.0f) * 0.5f * hi;
  p.c0 = !(g0 >= 0.0f && g0 <= hi);
  p.c1 = !(g1 >= 0.0f && g1 <= hi);
  g0 = fminf(fmaxf(g0, 0.0f), hi);
  g1 = fminf(fmaxf(g1, 0.0f), hi);
  p.i0 = min((int)floorf(g0), a.R - 2);
  p.j0 = min((int)floorf(g1), a.R - 2);
  p.f0 = g0 - (float)p.i0;
  p.f1 = g1 - (float)p.j0;
  return p;
}

// f[c] = prod over the six planes of the bilinear sample (channels-last texels).
template <int C>
__device__ __forceinline__ void hexplane_sample(const GaussArgs& a, const float mu[3], float f[C]) {
  float coord[4];
  grid_coords(a, mu, coord);
#pragma unroll
  for (int c = 0; c < C; ++c) f[c] = 1.0f;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const GridPos gp = grid_pos(a, coord[pair_a(k)], coord[pair_b(k)]);
    const float w00 = (1.f - gp.f0) * (1.f - gp.f1), w10 = gp.f0 * (1.f - gp.f1);
    const float w01 = (1.f - gp.f0) * gp.f1, w11 = gp.f0 * gp.f1;
    const float4* p00 = reinterpret_cast<const float4*>(a.planes + ((size_t)(k * a.R + gp.i0) * a.R + gp.j0) * C);
    const float4* p01 = p00 + C / 4;
    const float4* p10 = p00 + (size_t)a.R * C / 4;
    const float4* p11 = p10 + C / 4;
#pragma unroll
    for (int c4 = 0; c4 < C / 4; ++c4) {
      const float4 x00 = __ldg(p00 + c4), x01 = __ldg(p01 + c4), x10 = __ldg(p10 + c4), x11 = __ldg(p11 + c4);
      f[4 * c4 + 0] *= w00 * x00.x + w10 * x10.x + w01 * x01.x + w11 * x11.x;
      f[4 * c4 + 1] *= w00 * x00.y + w10 * x10.y + w01 * x01.y + w11 * x11.y;
      f[4 * c4 + 2] *= w00 * x00.z + w10 * x10.z + w01 * x01.z + w11 * x11.z;
      f[4 * c4 + 3] *= w00 * x00.w + w10 * x10.w + w01 * x01.w + w11 * x11.w;
    }
  }
}

// Warp-cooperative HexPlane sample.  For each active Gaussian j of the warp
// in turn, lane c handles channel c (and c+32 when C = 64): its texel loads
// for a fixed j are one coalesced line per texel instead of 32 scattered
// lines per load instruction.  The products are transposed through the
// warp's shared slice sfw[32][C+1] into each Gaussian's own thread.
struct PlaneParams {
  uint32_t base[6];   // float offset of texel (i0, j0) of each plane
  float w[6][4];      // bilinear weights w00 w10 w01 w11
};

template <int C>
__device__ __forceinline__ PlaneParams plane_params(const GaussArgs& a, const float mu[3]) {
  PlaneParams pp;
  float coord[4];
  grid_coords(a, mu, coord);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const GridPos gp = grid_pos(a, coord[pair_a(k)], coord[pair_b(k)]);
    pp.base[k] = (uint32_t)(((k * a.R + gp.i0) * a.R + gp.j0) * C);
    pp.w[k][0] = (1.f - gp.f0) * (1.f - gp.f1);
    pp.w[k][1] = gp.f0 * (1.f - gp.f1);
    pp.w[k][2] = (1.f - gp.f0) * gp.f1;
    pp.w[k][3] = gp.f0 * gp.f1;
  }
  return pp;
}

template <int C>
__device__ __forceinline__ void hexplane_sample_warp(const GaussArgs& a, const float mu[3], bool active, float* sfw,
                                                     float f[C]) {
  constexpr int CPL = C / 32;
  const int lane = threadIdx.x & 31;
  PlaneParams pp{};
  if (active) pp = plane_params<C>(a, mu);
  const unsigned act = __ballot_sync(0xFFFFFFFFu, active);
  const size_t RC = (size_t)a.R * C;
  for (int j = 0; j < 32; ++j) {
    if (!((act >> j) & 1u)) continue;
    float prod[CPL];
#pragma unroll
    for (int q = 0; q < CPL; ++q) prod[q] = 1.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const uint32_t bj = __shfl_sync(0xFFFFFFFFu, pp.base[k], j);
      const float w00 = __shfl_sync(0xFFFFFFFFu, pp.w[k][0], j), w10 = __shfl_sync(0xFFFFFFFFu, pp.w[k][1], j);
      const float w01 = __shfl_sync(0xFFFFFFFFu, pp.w[k][2], j), w11 = __shfl_sync(0xFFFFFFFFu, pp.w[k][3], j);
      const float* p00 = a.planes + bj;
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const int c = lane + 32 * q;
        const float x00 = __ldg(p00 + c), x01 = __ldg(p00 + C + c), x10 = __ldg(p00 + RC + c),
                    x11 = __ldg(p00 + RC + C + c);
        prod[q] *= w00 * x00 + w10 * x10 + w01 * x01 + w11 * x11;
      }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) sfw[j * (C + 1) + lane + 32 * q] = prod[q];
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int c = 0; c < C; ++c) f[c] = sfw[lane * (C + 1) + c];
  }
  __syncwarp();
}

// dmu from df (thread-private slice of shared memory, C floats) through the
// six bilinear samples and their product.
template <int C>
__device__ __forceinline__ void hexplane_backward(const GaussArgs& a, const float mu[3], const float* df, float dmu[3]) {
  float coord[4];
  grid_coords(a, mu, coord);
  GridPos gp[6];
  float w[6][4];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    gp[k] = grid_pos(a, coord[pair_a(k)], coord[pair_b(k)]);
    w[k][0] = (1.f - gp[k].f0) * (1.f - gp[k].f1);
    w[k][1] = gp[k].f0 * (1.f - gp[k].f1);
    w[k][2] = (1.f - gp[k].f0) * gp[k].f1;
    w[k][3] = gp[k].f0 * gp[k].f1;
  }
  float dg[6][2];
#pragma unroll
  for (int k = 0; k < 6; ++k) dg[k][0] = dg[k][1] = 0.0f;
  // Four channels at a time: samples of all planes, then the product of the
  // other five by prefix/suffix products (no division).
#pragma unroll 1
  for (int c4 = 0; c4 < C / 4; ++c4) {
    const float4 dfv = *reinterpret_cast<const float4*>(df + 4 * c4);
    const float dfc[4] = {dfv.x, dfv.y, dfv.z, dfv.w};
    float sv[6][4], d0[6][4], d1[6][4];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4* p00 = reinterpret_cast<const float4*>(a.planes + ((size_t)(k * a.R + gp[k].i0) * a.R + gp[k].j0) * C) + c4;
      const float4 x00 = __ldg(p00), x01 = __ldg(p00 + C / 4), x10 = __ldg(p00 + (size_t)a.R * C / 4),
                   x11 = __ldg(p00 + (size_t)a.R * C / 4 + C / 4);
      const float e00[4] = {x00.x, x00.y, x00.z, x00.w}, e01[4] = {x01.x, x01.y, x01.z, x01.w};
      const float e10[4] = {x10.x, x10.y, x10.z, x10.w}, e11[4] = {x11.x, x11.y, x11.z, x11.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        sv[k][j] = w[k][0] * e00[j] + w[k][1] * e10[j] + w[k][2] * e01[j] + w[k][3] * e11[j];
        d0[k][j] = (1.f - gp[k].f1) * (e10[j] - e00[j]) + gp[k].f1 * (e11[j] - e01[j]);
        d1[k][j] = (1.f - gp[k].f0) * (e01[j] - e00[j]) + gp[k].f0 * (e11[j] - e10[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float pre[6], suf = 1.0f;
      pre[0] = 1.0f;
#pragma unroll
      for (int k = 1; k < 6; ++k) pre[k] = pre[k - 1] * sv[k - 1][j];
#pragma unroll
      for (int k = 5; k >= 0; --k) {
        const float ds = dfc[j] * pre[k] * suf;
        dg[k][0] = fmaf(ds, d0[k][j], dg[k][0]);
        dg[k][1] = fmaf(ds, d1[k][j], dg[k][1]);
        suf *= sv[k][j];
      }
    }
  }
  float dcoord[4] = {0.f, 0.f, 0.f, 0.f};
  const float half = 0.5f * (float)(a.R - 1);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    if (!gp[k].c0) dcoord[pair_a(k)] += dg[k][0] * half;
    if (!gp[k].c1) dcoord[pair_b(k)] += dg[k][1] * half;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) dmu[i] = dcoord[i] * a.bscale[i];
}

// Warp-cooperative reverse of the HexPlane sample: for each active Gaussian
// j of the warp, lane c takes channel c of its six planes (coalesced texel
// loads), forms d f_c / d(grid position) by prefix/suffix products, weights
// it by df_j[c] (thread j's slice of dfs), and the warp reduces the twelve
// (plane, axis) sums.  Returns dmu of this thread's own Gaussian.
template <int C>
__device__ __forceinline__ void hexplane_backward_warp(const GaussArgs& a, const float mu[3], bool active,
                                                       const float* dfs, float* sred, float dmu[3]) {
  constexpr int CPL = C / 32;
  const int lane = threadIdx.x & 31;
  PlaneParams pp{};
  float fr[6][2];
  bool clamp[6][2];
#pragma unroll
  for (int k = 0; k < 6; ++k) { fr[k][0] = fr[k][1] = 0.f; clamp[k][0] = clamp[k][1] = true; }
  if (active) {
    float coord[4];
    grid_coords(a, mu, coord);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const GridPos gp = grid_pos(a, coord[pair_a(k)], coord[pair_b(k)]);
      pp.base[k] = (uint32_t)(((k * a.R + gp.i0) * a.R + gp.j0) * C);
      fr[k][0] = gp.f0;
      fr[k][1] = gp.f1;
      clamp[k][0] = gp.c0;
      clamp[k][1] = gp.c1;
      pp.w[k][0] = (1.f - gp.f0) * (1.f - gp.f1);
      pp.w[k][1] = gp.f0 * (1.f - gp.f1);
      pp.w[k][2] = (1.f - gp.f0) * gp.f1;
      pp.w[k][3] = gp.f0 * gp.f1;
    }
  }
  const unsigned act = __ballot_sync(0xFFFFFFFFu, active);
  const size_t RC = (size_t)a.R * C;
  for (int j = 0; j < 32; ++j) {
    if (!((act >> j) & 1u)) continue;
    float v[16];  // dg[k][0], dg[k][1] for k < 6 (lane-partial), 4 pad
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = 0.0f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = lane + 32 * q;
      float sv[6], d0[6], d1[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const uint32_t bj = __shfl_sync(0xFFFFFFFFu, pp.base[k], j);
        const float f0 = __shfl_sync(0xFFFFFFFFu, fr[k][0], j), f1 = __shfl_sync(0xFFFFFFFFu, fr[k][1], j);
        const float* p00 = a.planes + bj;
        const float x00 = __ldg(p00 + c), x01 = __ldg(p00 + C + c), x10 = __ldg(p00 + RC + c),
                    x11 = __ldg(p00 + RC + C + c);
        sv[k] = (1.f - f0) * (1.f - f1) * x00 + f0 * (1.f - f1) * x10 + (1.f - f0) * f1 * x01 + f0 * f1 * x11;
        d0[k] = (1.f - f1) * (x10 - x00) + f1 * (x11 - x01);
        d1[k] = (1.f - f0) * (x01 - x00) + f0 * (x11 - x10);
      }
      const float dfc = dfs[j * C + c];
      float pre[6], suf = 1.0f;
      pre[0] = 1.0f;
#pragma unroll
      for (int k = 1; k < 6; ++k) pre[k] = pre[k - 1] * sv[k - 1];
#pragma unroll
      for (int k = 5; k >= 0; --k) {
        const float ds = dfc * pre[k] * suf;
        v[2 * k] = fmaf(ds, d0[k], v[2 * k]);
        v[2 * k + 1] = fmaf(ds, d1[k], v[2 * k + 1]);
        suf *= sv[k];
      }
    }
    // Reduce-scatter of v[0..15] over the warp: lane 2m ends with index m.
    const int b16 = (lane >> 4) & 1, b8 = (lane >> 3) & 1, b4 = (lane >> 2) & 1, b2 = (lane >> 1) & 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float send = b16 ? v[i] : v[i + 8], keep = b16 ? v[i + 8] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float send = b8 ? v[i] : v[i + 4], keep = b8 ? v[i + 4] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float send = b4 ? v[i] : v[i + 2], keep = b4 ? v[i + 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 4);
    }
    {
      const float send = b2 ? v[0] : v[1], keep = b2 ? v[1] : v[0];
      v[0] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, 2);
    }
    v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], 1);
    const int m = b2 + 2 * b4 + 4 * b8 + 8 * b16;
    if ((lane & 1) == 0 && m < 12) sred[j * 12 + m] = v[0];
  }
  __syncwarp();
  dmu[0] = dmu[1] = dmu[2] = 0.0f;
  if (active) {
    float dcoord[4] = {0.f, 0.f, 0.f, 0.f};
    const float half = 0.5f * (float)(a.R - 1);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (!clamp[k][0]) dcoord[pair_a(k)] += sred[lane * 12 + 2 * k] * half;
      if (!clamp[k][1]) dcoord[pair_b(k)] += sred[lane * 12 + 2 * k + 1] * half;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) dmu[i] = dcoord[i] * a.bscale[i];
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Projection state of one deformed Gaussian.
// ---------------------------------------------------------------------------
struct Proj {
  float mu[3];
  float qt[4], qinv, q[4];
  float s[3];
  float o;
  float R[9], M[9];
  float S00, S01, S02, S11, S12, S22;  // 3D covariance (symmetric)
  float p[3];
  float tx, ty, txc, tyc;
  bool clx, cly;
  float J00, J02, J11, J12;
  float T[6];
  float a, b, c, det;   // dilated 2D covariance [[a,b],[b,c]], its determinant
  float ca, cb, cc;     // conic
  float u, v;
  float dir[3], dinv;
  float Y[16];
  float rgb_raw[3];
  int radius;
  bool visible;
  bool finite;
};

__device__ __forceinline__ void project(const GaussArgs& a, int g, const float delta[kHeads], const float sh[48],
                                        Proj& s) {
  const float m0 = a.means[3 * g], m1 = a.means[3 * g + 1], m2 = a.means[3 * g + 2];
  const float4 q4 = __ldg(reinterpret_cast<const float4*>(a.quats) + g);
  const float l0 = a.log_scales[3 * g], l1 = a.log_scales[3 * g + 1], l2 = a.log_scales[3 * g + 2];
  const float lg = a.logits[g];
  s.finite = isfinite(m0) && isfinite(m1) && isfinite(m2) && isfinite(q4.x) && isfinite(q4.y) && isfinite(q4.z) &&
             isfinite(q4.w) && isfinite(l0) && isfinite(l1) && isfinite(l2) && isfinite(lg);
  // Eq. 6 reading: mu + d_mu, normalise(q + d_q), log s + d_s, logit + d_o.
  s.mu[0] = m0 + delta[0];
  s.mu[1] = m1 + delta[1];
  s.mu[2] = m2 + delta[2];
  s.qt[0] = q4.x + delta[3];
  s.qt[1] = q4.y + delta[4];
  s.qt[2] = q4.z + delta[5];
  s.qt[3] = q4.w + delta[6];
  s.qinv = rsqrtf(s.qt[0] * s.qt[0] + s.qt[1] * s.qt[1] + s.qt[2] * s.qt[2] + s.qt[3] * s.qt[3]);
#pragma unroll
  for (int i = 0; i < 4; ++i) s.q[i] = s.qt[i] * s.qinv;
  s.s[0] = expf(l0 + delta[7]);
  s.s[1] = expf(l1 + delta[8]);
  s.s[2] = expf(l2 + delta[9]);
  s.o = 1.0f / (1.0f + expf(-(lg + delta[10])));
  // Eq. 2: Sigma = R S S^T R^T.
  const float w = s.q[0], x = s.q[1], y = s.q[2], z = s.q[3];
  s.R[0] = 1.f - 2.f * (y * y + z * z); s.R[1] = 2.f * (x * y - w * z);       s.R[2] = 2.f * (x * z + w * y);
  s.R[3] = 2.f * (x * y + w * z);       s.R[4] = 1.f - 2.f * (x * x + z * z); s.R[5] = 2.f * (y * z - w * x);
  s.R[6] = 2.f * (x * z - w * y);       s.R[7] = 2.f * (y * z + w * x);       s.R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s.M[3 * i + j] = s.R[3 * i + j] * s.s[j];
  s.S00 = s.M[0] * s.M[0] + s.M[1] * s.M[1] + s.M[2] * s.M[2];
  s.S01 = s.M[0] * s.M[3] + s.M[1] * s.M[4] + s.M[2] * s.M[5];
  s.S02 = s.M[0] * s.M[6] + s.M[1] * s.M[7] + s.M[2] * s.M[8];
  s.S11 = s.M[3] * s.M[3] + s.M[4] * s.M[4] + s.M[5] * s.M[5];
  s.S12 = s.M[3] * s.M[6] + s.M[4] * s.M[7] + s.M[5] * s.M[8];
  s.S22 = s.M[6] * s.M[6] + s.M[7] * s.M[7] + s.M[8] * s.M[8];
  const float* V = a.V;
#pragma unroll
  for (int i = 0; i < 3; ++i) s.p[i] = V[4 * i] * s.mu[0] + V[4 * i + 1] * s.mu[1] + V[4 * i + 2] * s.mu[2] + V[4 * i + 3];
  // View direction for colour.
  const float dx = s.mu[0] - a.campos[0], dy = s.mu[1] - a.campos[1], dz = s.mu[2] - a.campos[2];
  s.dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
  s.dir[0] = dx * s.dinv; s.dir[1] = dy * s.dinv; s.dir[2] = dz * s.dinv;
  sh_basis(s.dir, s.Y);
  const int nb = (a.sh_degree + 1) * (a.sh_degree + 1);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < nb) acc = fmaf(sh[3 * k + ch], s.Y[k], acc);
    s.rgb_raw[ch] = acc;
  }
  s.visible = false;
  s.radius = 0;
  const float zc = s.p[2];
  if (!s.finite || !(zc > a.znear)) return;
  // EWA (Sec. 3.3): Jacobian of the pinhole projection at the centre, with
  // x/z, y/z clamped to 1.3x the half field of view.
  s.tx = s.p[0] / zc;
  s.ty = s.p[1] / zc;
  s.clx = !(s.tx >= -a.limx && s.tx <= a.limx);
  s.cly = !(s.ty >= -a.limy && s.ty <= a.limy);
  s.txc = fminf(fmaxf(s.tx, -a.limx), a.limx);
  s.tyc = fminf(fmaxf(s.ty, -a.limy), a.limy);
  const float iz = 1.0f / zc;
  s.J00 = a.fx * iz;
  s.J02 = -a.fx * s.txc * iz;
  s.J11 = a.fy * iz;
  s.J12 = -a.fy * s.tyc * iz;
  // T = J W (2x3).
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    s.T[j] = s.J00 * V[j] + s.J02 * V[8 + j];
    s.T[3 + j] = s.J11 * V[4 + j] + s.J12 * V[8 + j];
  }
  // Sigma' = T Sigma T^T.
  float u0[3], u1[3];
  u0[0] = s.S00 * s.T[0] + s.S01 * s.T[1] + s.S02 * s.T[2];
  u0[1] = s.S01 * s.T[0] + s.S11 * s.T[1] + s.S12 * s.T[2];
  u0[2] = s.S02 * s.T[0] + s.S12 * s.T[1] + s.S22 * s.T[2];
  u1[0] = s.S00 * s.T[3] + s.S01 * s.T[4] + s.S02 * s.T[5];
  u1[1] = s.S01 * s.T[3] + s.S11 * s.T[4] + s.S12 * s.T[5];
  u1[2] = s.S02 * s.T[3] + s.S12 * s.T[4] + s.S22 * s.T[5];
  s.a = s.T[0] * u0[0] + s.T[1] * u0[1] + s.T[2] * u0[2] + kDilation;
  s.b = s.T[3] * u0[0] + s.T[4] * u0[1] + s.T[5] * u0[2];
  s.c = s.T[3] * u1[0] + s.T[4] * u1[1] + s.T[5] * u1[2] + kDilation;
  // Compensated determinant a*c - b*b (Kahan's FMA scheme for a 2x2
  // determinant): the rounding error of b*b is recovered exactly by an FMA.
  const float bb = s.b * s.b;
  const float err = fmaf(-s.b, s.b, bb);
  const float ac = fmaf(s.a, s.c, -bb);
  s.det = ac + err;
  if (!(s.det > 0.0f)) return;
  const float idet = 1.0f / s.det;
  s.ca = s.c * idet;
  s.cb = -s.b * idet;
  s.cc = s.a * idet;
  const float mid = 0.5f * (s.a + s.c);
  const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - s.det));
  s.radius = (int)ceilf(3.0f * sqrtf(lam));
  s.u = a.fx * s.tx + a.cx;
  s.v = a.fy * s.ty + a.cy;
  s.visible = isfinite(s.u) && isfinite(s.v);
}

}  // namespace

// ---------------------------------------------------------------------------
// HexPlane feature of every Gaussian for the tensor-core MLP: f (Eq. 4-6)
// split into three BF16 terms f = hi + mid + lo, each the BF16 rounding of
// what the previous terms leave, written as three [P][C] arrays (term t at
// fsplit + t P C).
template <int C>
__global__ void __launch_bounds__(kThreads) hexplane_split_kernel(const GaussArgs a) {
  extern __shared__ __align__(16) float s_slices[];
  float* sfw = s_slices + (threadIdx.x >> 5) * 32 * (C + 1);  // this warp's transpose slice
  const int g = blockIdx.x * kThreads + threadIdx.x;
  const bool active = g < a.P;
  float mu[3] = {0.f, 0.f, 0.f};
  if (active) { mu[0] = a.means[3 * g]; mu[1] = a.means[3 * g + 1]; mu[2] = a.means[3 * g + 2]; }
  float f[C];
  hexplane_sample_warp<C>(a, mu, active, sfw, f);
  if (!active) return;
  auto pack = [](float x, float y) -> uint32_t {
    const __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<const uint32_t*>(&v);
  };
  const size_t term = (size_t)a.P * C;
  uint4* hi = reinterpret_cast<uint4*>(a.fsplit + (size_t)g * C);
  uint4* mid = reinterpret_cast<uint4*>(a.fsplit + term + (size_t)g * C);
  uint4* lo = reinterpret_cast<uint4*>(a.fsplit + 2 * term + (size_t)g * C);
#pragma unroll
  for (int c8 = 0; c8 < C / 8; ++c8) {
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float x = f[8 * c8 + 2 * i], y = f[8 * c8 + 2 * i + 1];
      h[i] = pack(x, y);
      x -= __uint_as_float(h[i] << 16);
      y -= __uint_as_float(h[i] & 0xFFFF0000u);
      m[i] = pack(x, y);
      x -= __uint_as_float(m[i] << 16);
      y -= __uint_as_float(m[i] & 0xFFFF0000u);
      l[i] = pack(x, y);
    }
    hi[c8] = make_uint4(h[0], h[1], h[2], h[3]);
    mid[c8] = make_uint4(m[0], m[1], m[2], m[3]);
    lo[c8] = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// Deformation offsets of Gaussian g (zero for a static scene): the MLP's
// output in dstate, plus the optional positional noise, which is stored
// back so that the reverse pass sees the offsets that were applied.
__device__ __forceinline__ void deform_delta(const GaussArgs& a, int g, float delta[kHeads]) {
#pragma unroll
  for (int k = 0; k < kHeads; ++k) delta[k] = 0.0f;
  if (!a.has_deform) return;  // uniform over the launch
  float4* d = reinterpret_cast<float4*>(a.dstate + (size_t)g * kDStride);
  const float4 q0 = d[0], q1 = d[1], q2 = d[2];
  delta[0] = q0.x; delta[1] = q0.y; delta[2] = q0.z; delta[3] = q0.w; delta[4] = q1.x; delta[5] = q1.y;
  delta[6] = q1.z; delta[7] = q1.w; delta[8] = q2.x; delta[9] = q2.y; delta[10] = q2.z;
  if (a.noise) {
    const float nt = a.noise_scale * a.t;
#pragma unroll
    for (int k = 0; k < 3; ++k) delta[k] = fmaf(nt, a.noise[3 * g + k], delta[k]);
    d[0] = make_float4(delta[0], delta[1], delta[2], delta[3]);
  }
}

__global__ void __launch_bounds__(kThreads, 2) gauss_fwd_kernel(const GaussArgs a) {
  const int g = blockIdx.x * kThreads + threadIdx.x;
  bool vis = false;
  if (g < a.P) {
    float delta[kHeads];
    deform_delta(a, g, delta);
    float sh[48];
    load_sh(a.sh, a.sh_bf16, g, sh);
    Proj s;
    project(a, g, delta, sh, s);
    if (!s.finite) set_err(a.err, kErrNonFinite);
    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    ushort4 rect = make_ushort4(1, 1, 0, 0);
    uint32_t touched = 0, key = 0xFFFFFFFFu;
    if (s.visible) {
      int x0, y0, x1, y1;
      if (pixel_rect(s.u, s.v, s.radius, a.W, a.H, x0, y0, x1, y1)) {
        // On screen: its record is written.  Its tiles are those of the
        // pixel rect cut to the blend box (the pixels whose centres lie
        // within the box's half-widths of the centre): outside it the
        // Gaussian blends nowhere, so the lists lose only entries that no
        // pixel would blend.
        const float box = blend_box(0.5f * kLog2e * s.ca, kLog2e * s.cb, 0.5f * kLog2e * s.cc, s.o);
        const uint32_t hb = __float_as_uint(box);
        const __half2 h2 = *reinterpret_cast<const __half2*>(&hb);
        const float hx = __low2float(h2), hy = __high2float(h2);
        bool blends = hx >= 0.0f;
        if (blends && hx < 1e30f) {
          x0 = max(x0, (int)ceilf(s.u - hx - 0.5f));
          x1 = min(x1, (int)floorf(s.u + hx - 0.5f));
        }
        if (blends && hy < 1e30f) {
          y0 = max(y0, (int)ceilf(s.v - hy - 0.5f));
          y1 = min(y1, (int)floorf(s.v + hy - 0.5f));
        }
        blends = blends && x0 <= x1 && y0 <= y1;
        if (blends) {
          const int tx0 = x0 / a.tw, tx1 = x1 / a.tw, ty0 = y0 / a.th, ty1 = y1 / a.th;
          rect = make_ushort4(tx0, ty0, tx1, ty1);
          touched = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        }
        key = __float_as_uint(s.p[2]);
        vis = true;
        r0 = make_float4(s.u, s.v, -0.5f * kLog2e * s.ca, -kLog2e * s.cb);
        r1 = make_float4(-0.5f * kLog2e * s.cc, s.o, s.p[2], fmaxf(s.rgb_raw[0], 0.0f));
        r2 = make_float4(fmaxf(s.rgb_raw[1], 0.0f), fmaxf(s.rgb_raw[2], 0.0f), (float)s.radius, box);
      }
    }
    float4* rec = a.rec + 3 * (size_t)g;
    rec[0] = r0; rec[1] = r1; rec[2] = r2;
    a.rect[g] = rect;
    a.touched[g] = touched;
    a.dkey[g] = key;
  }
  const unsigned vote = __ballot_sync(0xFFFFFFFFu, vis);
  if ((threadIdx.x & 31) == 0 && vote) atomicAdd(a.num_visible, (uint32_t)__popc(vote));
}

// ---------------------------------------------------------------------------
// Sum of each Gaussian's partial rows, writing d_feat[g] and the ten scalar
// sums to psum[g].  The entries of consecutive depth ranks occupy
// consecutive emission ranges, so one warp takes ranks_per_warp(D) consecutive
// ranks: one coalesced load of their ranges, one of the bitmask words of
// the whole range (read back by shuffle), then the written rows streamed RG
// at a time (all RG rows' loads in flight before any is added), lane c
// adding column c (and c + 32, ...).  Each Gaussian's rows are added one
// after another in increasing emission order: a fixed order, so the result
// is bitwise reproducible.
// Ranks per warp: 8 for rows of at most 64 floats (D <= 52), else 4
// (measured best at D = 32 and D = 128).
__host__ __device__ constexpr int ranks_per_warp(int D) { return (partial_stride(D) + 31) / 32 <= 2 ? 8 : 4; }

template <int D>
__global__ void __launch_bounds__(kThreads, 3) partial_reduce_kernel(const GaussBwdArgs b, int P) {
  constexpr int NP = partial_stride(D);
  constexpr int NQ = (NP + 31) / 32;  // columns per lane
  constexpr int RG = NQ <= 2 ? 16 : (NQ <= 4 ? 8 : 4);  // rows in flight
  const int lane = threadIdx.x & 31;
  constexpr int GPW = ranks_per_warp(D);
  const int64_t r0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * GPW;
  if (r0 >= P) return;
  const int nvalid = (int)min((int64_t)GPW, (int64_t)P - r0);
  const uint64_t cap = (uint64_t)b.cap;
  // Lane j < nvalid: the Gaussian of rank r0 + j and the end of its range.
  const bool mine = lane < nvalid;
  const uint32_t gid = mine ? b.order[r0 + lane] : 0u;
  const uint32_t ebeg = mine ? (uint32_t)min((uint64_t)b.offs[r0 + lane], cap) : 0u;
  const uint32_t eend = mine ? (uint32_t)min((uint64_t)b.offs[r0 + lane + 1], cap) : 0u;
  const uint32_t E0 = __shfl_sync(0xFFFFFFFFu, ebeg, 0);
  const uint32_t E1 = __shfl_sync(0xFFFFFFFFu, eend, nvalid - 1);
  // Bitmask words of the range: word wbase + l in lane l (the rest, for a
  // range of more than 32 words, read when reached).
  const uint32_t wbase = E0 >> 5;
  const uint32_t wlast = E0 < E1 ? (E1 - 1) >> 5 : wbase;
  const uint32_t wl = (E0 < E1 && wbase + (uint32_t)lane <= wlast) ? __ldg(b.pflags + wbase + lane) : 0u;
  auto word = [&](uint32_t w) -> uint32_t {
    const uint32_t k = w - wbase;
    const uint32_t v = __shfl_sync(0xFFFFFFFFu, wl, (int)(k & 31u));
    return k < 32u ? v : __ldg(b.pflags + w);
  };
  float acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0f;
  int j = 0;  // Gaussian (lane) whose rows are being added
  uint32_t jend = __shfl_sync(0xFFFFFFFFu, eend, 0);
  // Writes Gaussian j's sums and moves to the next one.
  auto flush = [&]() {
    const uint32_t g = __shfl_sync(0xFFFFFFFFu, gid, j);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int col = lane + 32 * q;
      if (col < D) {
        float* o = b.d_feat + (size_t)g * D + col;
        *o = b.accumulate ? *o + acc[q] : acc[q];
      } else if (col < NP) {
        b.psum[(size_t)g * 12 + (col - D)] = acc[q];
      }
      acc[q] = 0.0f;
    }
    ++j;
    jend = __shfl_sync(0xFFFFFFFFu, eend, j < nvalid ? j : nvalid - 1);
  };
  // Word w of the bitmask, m its bits not yet taken.
  uint32_t w = wbase;
  uint32_t m = E0 < E1 ? word(w) & (~0u << (E0 & 31u)) : 0u;
  bool done = E0 >= E1;
  while (!done) {
    // The next RG written rows (warp-uniform; slot u holds one if has[u]).
    uint32_t idx[RG];
    bool has[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      while (!done && m == 0u) {
        ++w;
        if (w > wlast) done = true;
        else m = word(w);
      }
      const uint32_t e = (w << 5) + (uint32_t)(__ffs(m) - 1);
      has[u] = !done && e < E1;
      if (!done && e >= E1) done = true;
      idx[u] = has[u] ? e : 0u;
      if (has[u]) m &= m - 1u;
    }
    float x[RG][NQ];
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      const float* row = b.partials + (size_t)idx[u] * NP;
#pragma unroll
      for (int q = 0; q < NQ; ++q) x[u][q] = (has[u] && lane + 32 * q < NP) ? __ldg(row + lane + 32 * q) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      if (has[u]) {
        while (idx[u] >= jend) flush();  // rows belong to the Gaussians in order
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] += x[u][q];
      }
    }
  }
  while (j < nvalid) flush();  // the last Gaussian with rows, and any after it without
}

// ---------------------------------------------------------------------------
// Reverse of projection and colour, per Gaussian: sums the partial rows,
// recomputes the projection from the stored deformation offsets and writes
// the gradients of the deformed parameters, which are also the canonical
// gradients of log-scale, quaternion, opacity logit and SH; the mean's
// path through the HexPlane grid is added by gauss_bwd_deform_kernel from
// dd = d L / d delta stored per Gaussian.
__global__ void __launch_bounds__(kThreads, 2) gauss_bwd_proj_kernel(const GaussArgs a, const GaussBwdArgs b) {
  const int g = blockIdx.x * kThreads + threadIdx.x;
  if (g >= a.P) return;
  float acc[kPartialScalars + 2];
  {
    const float4* ps = reinterpret_cast<const float4*>(b.psum + (size_t)g * 12);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 v = ps[k];
      acc[4 * k] = v.x; acc[4 * k + 1] = v.y; acc[4 * k + 2] = v.z; acc[4 * k + 3] = v.w;
    }
  }
  const uint32_t nt = b.touched[g];
  float delta[kHeads];
  if (a.has_deform) {
    const float4* d = reinterpret_cast<const float4*>(a.dstate + (size_t)g * kDStride);
    const float4 d0 = d[0], d1 = d[1], d2 = d[2];
    delta[0] = d0.x; delta[1] = d0.y; delta[2] = d0.z; delta[3] = d0.w;
    delta[4] = d1.x; delta[5] = d1.y; delta[6] = d1.z; delta[7] = d1.w;
    delta[8] = d2.x; delta[9] = d2.y; delta[10] = d2.z;
  } else {
#pragma unroll
    for (int k = 0; k < kHeads; ++k) delta[k] = 0.0f;
  }
  float sh[48];
  load_sh(a.sh, a.sh_bf16, g, sh);
  Proj s;
  project(a, g, delta, sh, s);
  const float du = acc[0], dv = acc[1];
  // Scaled conic back to (a, b, c) of the conic: A = -0.5 log2e a, B = -log2e b.
  const float dca = -0.5f * kLog2e * acc[2], dcb = -kLog2e * acc[3], dcc = -0.5f * kLog2e * acc[4];
  const float dop = acc[5];
  const float drgb[3] = {acc[6], acc[7], acc[8]};
  const float ddepth = acc[9];
  float dmu[3] = {0.f, 0.f, 0.f};
  // Colour (clamp at 0 passes the gradient where raw >= 0).
  {
    float gch[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) gch[ch] = s.rgb_raw[ch] >= 0.0f ? drgb[ch] : 0.0f;
    const int nb = (a.sh_degree + 1) * (a.sh_degree + 1);
    float wk[16];
    float* dsh = b.d_sh + (size_t)g * 48;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      wk[k] = k < nb ? gch[0] * sh[3 * k] + gch[1] * sh[3 * k + 1] + gch[2] * sh[3 * k + 2] : 0.0f;
#pragma unroll
    for (int k4 = 0; k4 < 12; ++k4) {
      float v4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int idx = 4 * k4 + j, k = idx / 3, ch = idx % 3;
        v4[j] = k < nb ? gch[ch] * s.Y[k] : 0.0f;
      }
      float4 o4 = make_float4(v4[0], v4[1], v4[2], v4[3]);
      if (b.accumulate) {
        const float4 old = reinterpret_cast<const float4*>(dsh)[k4];
        o4 = make_float4(old.x + o4.x, old.y + o4.y, old.z + o4.z, old.w + o4.w);
      }
      reinterpret_cast<float4*>(dsh)[k4] = o4;
    }
    float gd[3];
    sh_basis_vjp(s.dir, wk, gd);
    const float dd = gd[0] * s.dir[0] + gd[1] * s.dir[1] + gd[2] * s.dir[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) dmu[i] += (gd[i] - s.dir[i] * dd) * s.dinv;
  }
  const float dlogit = dop * s.o * (1.0f - s.o);
  float dlogs[3] = {0.f, 0.f, 0.f};
  float dqt[4] = {0.f, 0.f, 0.f, 0.f};
  const bool active = s.visible && nt > 0;
  if (active) {
    const float* V = a.V;
    const float zc = s.p[2], iz = 1.0f / zc;
    // Conic M = inverse of [[a,b],[b,c]]: Gs = -M Gm M with Gm = [[da, db/2],[db/2, dc]].
    const float M00 = s.ca, M01 = s.cb, M11 = s.cc;
    const float G00 = dca, G01 = 0.5f * dcb, G11 = dcc;
    const float A00 = M00 * G00 + M01 * G01, A01 = M00 * G01 + M01 * G11;
    const float A10 = M01 * G00 + M11 * G01, A11 = M01 * G01 + M11 * G11;
    const float Gs00 = -(A00 * M00 + A01 * M01);
    const float Gs01 = -(A00 * M01 + A01 * M11);
    const float Gs11 = -(A10 * M01 + A11 * M11);
    // dSigma = T^T Gs T (symmetric), dT = 2 Gs T Sigma.
    const float* T = s.T;
    float GT[6];  // Gs T
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      GT[j] = Gs00 * T[j] + Gs01 * T[3 + j];
      GT[3 + j] = Gs01 * T[j] + Gs11 * T[3 + j];
    }
    float dS[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) dS[3 * i + j] = T[i] * GT[j] + T[3 + i] * GT[3 + j];
    const float Sg[9] = {s.S00, s.S01, s.S02, s.S01, s.S11, s.S12, s.S02, s.S12, s.S22};
    float dT[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dT[3 * r + j] = 2.0f * (GT[3 * r] * Sg[j] + GT[3 * r + 1] * Sg[3 + j] + GT[3 * r + 2] * Sg[6 + j]);
    // T = J W: dJ = dT W^T (only the non-zero entries of J).
    const float dJ00 = dT[0] * V[0] + dT[1] * V[1] + dT[2] * V[2];
    const float dJ02 = dT[0] * V[8] + dT[1] * V[9] + dT[2] * V[10];
    const float dJ11 = dT[3] * V[4] + dT[4] * V[5] + dT[5] * V[6];
    const float dJ12 = dT[3] * V[8] + dT[4] * V[9] + dT[5] * V[10];
    float dp0 = 0.f, dp1 = 0.f, dp2 = 0.f;
    dp2 += -a.fx * iz * iz * dJ00 - a.fy * iz * iz * dJ11;
    dp2 += a.fx * s.txc * iz * iz * dJ02 + a.fy * s.tyc * iz * iz * dJ12;
    float dtx = s.clx ? 0.0f : -a.fx * iz * dJ02;
    float dty = s.cly ? 0.0f : -a.fy * iz * dJ12;
    dtx += a.fx * du;
    dty += a.fy * dv;
    dp0 += dtx * iz;
    dp1 += dty * iz;
    dp2 += -(s.p[0] * dtx + s.p[1] * dty) * iz * iz;
    dp2 += ddepth;
#pragma unroll
    for (int i = 0; i < 3; ++i) dmu[i] += V[i] * dp0 + V[4 + i] * dp1 + V[8 + i] * dp2;
    // Sigma = M M^T, M = R diag(s): dM = (dS + dS^T) M.
    float dM[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dM[3 * i + j] = (dS[3 * i] + dS[i]) * s.M[j] + (dS[3 * i + 1] + dS[3 + i]) * s.M[3 + j] +
                        (dS[3 * i + 2] + dS[6 + i]) * s.M[6 + j];
    float dR[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) dR[3 * i + j] = dM[3 * i + j] * s.s[j];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      dlogs[j] = (dM[j] * s.R[j] + dM[3 + j] * s.R[3 + j] + dM[6 + j] * s.R[6 + j]) * s.s[j];
    const float w = s.q[0], x = s.q[1], y = s.q[2], z = s.q[3];
    float dq[4];
    dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] -
                   2.f * x * dR[8]);
    dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] -
                   2.f * y * dR[8]);
    dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] +
                   y * dR[7]);
    const float qd = dq[0] * s.q[0] + dq[1] * s.q[1] + dq[2] * s.q[2] + dq[3] * s.q[3];
#pragma unroll
    for (int i = 0; i < 4; ++i) dqt[i] = (dq[i] - s.q[i] * qd) * s.qinv;
  }
  if (b.accumulate) {
    // With a deformation field the reverse pass through the grid adds this
    // view's whole mean gradient (dmu + grid term) in one addition.
    const bool defer_mu = a.has_deform && active;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (!defer_mu) b.d_means[3 * g + i] += dmu[i];
      b.d_log_scales[3 * g + i] += dlogs[i];
    }
    const float4 oq = reinterpret_cast<const float4*>(b.d_quats)[g];
    reinterpret_cast<float4*>(b.d_quats)[g] = make_float4(oq.x + dqt[0], oq.y + dqt[1], oq.z + dqt[2], oq.w + dqt[3]);
    b.d_logits[g] += dlogit;
  } else {
    b.d_means[3 * g] = dmu[0];
    b.d_means[3 * g + 1] = dmu[1];
    b.d_means[3 * g + 2] = dmu[2];
    b.d_log_scales[3 * g] = dlogs[0];
    b.d_log_scales[3 * g + 1] = dlogs[1];
    b.d_log_scales[3 * g + 2] = dlogs[2];
    reinterpret_cast<float4*>(b.d_quats)[g] = make_float4(dqt[0], dqt[1], dqt[2], dqt[3]);
    b.d_logits[g] = dlogit;
  }
  if (a.has_deform) {
    // dd = dL/d delta: d_mu, d_q (pre-normalisation), d_log_s, d_logit; [11] = active flag.
    float4* o = reinterpret_cast<float4*>(b.ddstate + (size_t)g * 12);
    o[0] = make_float4(dmu[0], dmu[1], dmu[2], dqt[0]);
    o[1] = make_float4(dqt[1], dqt[2], dqt[3], dlogs[0]);
    o[2] = make_float4(dlogs[1], dlogs[2], dlogit, active ? 1.0f : 0.0f);
  }
}

// ---------------------------------------------------------------------------
// Mean gradient through the deformation: MLP reverse from the stored
// HexPlane feature, then the six bilinear samples (Sec. 3.2, Eq. 4-6).
template <int C>
__global__ void __launch_bounds__(kThreads, 2) gauss_bwd_deform_kernel(const GaussArgs a, const GaussBwdArgs b,
                                                                     const float* __restrict__ df_all) {
  extern __shared__ __align__(16) float sw[];
  float* s_df = sw;                                                  // [kThreads][C]
  float* s_red = s_df + (size_t)kThreads * C + (threadIdx.x >> 5) * 32 * 12;  // this warp's [32][12]
  const int g = blockIdx.x * kThreads + threadIdx.x;
  bool active = false;
  float dd[kHeads];
  if (g < a.P) {
    const float4* dd4 = reinterpret_cast<const float4*>(b.ddstate + (size_t)g * 12);
    const float4 q0 = dd4[0], q1 = dd4[1], q2 = dd4[2];
    active = q2.w != 0.0f;
    dd[0] = q0.x; dd[1] = q0.y; dd[2] = q0.z;
  }
  if (!__any_sync(0xFFFFFFFFu, active)) return;  // whole warp idle
  // dL/df of this Gaussian: the MLP reverse on the tensor cores wrote it.
  float* my_df = s_df + (size_t)threadIdx.x * C;
  if (active) {
    const float4* src = reinterpret_cast<const float4*>(df_all + (size_t)g * C);
#pragma unroll
    for (int c4 = 0; c4 < C / 4; ++c4) reinterpret_cast<float4*>(my_df)[c4] = src[c4];
  }
  __syncwarp();
  float mu0[3] = {0.f, 0.f, 0.f};
  if (active) { mu0[0] = a.means[3 * g]; mu0[1] = a.means[3 * g + 1]; mu0[2] = a.means[3 * g + 2]; }
  float dg[3];
  hexplane_backward_warp<C>(a, mu0, active, s_df + (size_t)(threadIdx.x & ~31) * C, s_red, dg);
  if (active) {
    if (b.accumulate) {
      // This view's mean gradient (projection part + grid part), added once.
#pragma unroll
      for (int i = 0; i < 3; ++i) b.d_means[3 * g + i] += dd[i] + dg[i];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) b.d_means[3 * g + i] += dg[i];
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int C>
static cudaError_t launch_split_t(const GaussArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)8 * 32 * (C + 1) * sizeof(float);  // 66.5 KB at C = 64
  auto k = hexplane_split_kernel<C>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<ceil_div(a.P, kThreads), kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// Deformed scenes: HexPlane features (split), the MLP on the tensor cores,
// then the projection; static scenes: the projection alone.
cudaError_t launch_gauss_fwd(const GaussArgs& a, cudaStream_t st) {
  if (a.P <= 0) return cudaSuccess;
  if (a.has_deform) {
    cudaError_t e = a.C == 32 ? launch_split_t<32>(a, st) : (a.C == 64 ? launch_split_t<64>(a, st) : cudaErrorInvalidValue);
    if (e != cudaSuccess) return e;
    if ((e = launch_deform_mlp(a, st)) != cudaSuccess) return e;
  }
  gauss_fwd_kernel<<<ceil_div(a.P, kThreads), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// The MLP reverse on the tensor cores writes dL/df into the region of the
// split features (free once the forward's MLP has read them), then the
// HexPlane reverse takes it from there.
template <int C>
static cudaError_t launch_bwd_deform_t(const GaussArgs& a, const GaussBwdArgs& b, cudaStream_t st) {
  float* df = reinterpret_cast<float*>(a.fsplit);
  cudaError_t e = launch_deform_mlp_bwd(a, b, df, st);
  if (e != cudaSuccess) return e;
  const size_t smem = ((size_t)kThreads * C + (size_t)8 * 32 * 12) * sizeof(float);
  auto k = gauss_bwd_deform_kernel<C>;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  k<<<ceil_div(a.P, kThreads), kThreads, smem, st>>>(a, b, df);
  return cudaGetLastError();
}

cudaError_t launch_gauss_bwd(const GaussArgs& a, const GaussBwdArgs& b, cudaStream_t st, cudaEvent_t mid) {
  if (a.P <= 0) return mid ? cudaEventRecord(mid, st) : cudaSuccess;
  const int gpw = ranks_per_warp(b.D);
  const int64_t nthreads = ((int64_t)a.P + gpw - 1) / gpw * 32;  // a warp per gpw depth ranks
  const int nblk = (int)((nthreads + kThreads - 1) / kThreads);
  switch (b.D) {
    case 16: partial_reduce_kernel<16><<<nblk, kThreads, 0, st>>>(b, a.P); break;
    case 32: partial_reduce_kernel<32><<<nblk, kThreads, 0, st>>>(b, a.P); break;
    case 64: partial_reduce_kernel<64><<<nblk, kThreads, 0, st>>>(b, a.P); break;
    case 128: partial_reduce_kernel<128><<<nblk, kThreads, 0, st>>>(b, a.P); break;
    case 256: partial_reduce_kernel<256><<<nblk, kThreads, 0, st>>>(b, a.P); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mid && (e = cudaEventRecord(mid, st)) != cudaSuccess) return e;
  gauss_bwd_proj_kernel<<<ceil_div(a.P, kThreads), kThreads, 0, st>>>(a, b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (!a.has_deform) return cudaSuccess;
  if (a.C == 32) return launch_bwd_deform_t<32>(a, b, st);
  if (a.C == 64) return launch_bwd_deform_t<64>(a, b, st);
  return cudaErrorInvalidValue;
}

}  // namespace fe
