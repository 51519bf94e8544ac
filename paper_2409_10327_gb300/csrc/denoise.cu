// Spatial SVGF denoiser (Schied et al. 2017 with its temporal parts removed,
// as the paper applies it to its raw Monte Carlo frames, Sec. 4.1; the depth
// gradient comes from the depth map offset by one pixel, supplementary
// "Rendering Details").  One thread per pixel:
//   svgf_variance_kernel: luminance variance from 7 x 7 depth/normal-weighted
//     moments (no history to estimate it from);
//   svgf_atrous_kernel:   one a-trous pass of the 5 x 5 B3 spline at step
//     2^i with depth, normal and variance-scaled luminance edge-stopping;
//     colour and variance travel together as float4 (rgb, Var).
// The image (16 B of colour, 4 B of depth and 16 B of normal per pixel) is a
// few MB at 800 x 800 and stays in L2 across the passes; taps go through the
// read-only cache.
#include "device_common.cuh"

namespace rtk {
namespace {

constexpr float kEps = 1e-10f;

__device__ __forceinline__ float luminance(float4 c) { return 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z; }

// forward differences of the depth map, backward at the last column / row
__device__ __forceinline__ float2 depth_gradient(const float* __restrict__ z, int W, int H, int x, int y) {
  const float zc = __ldg(z + y * W + x);
  float gx = 0.f, gy = 0.f;
  if (W > 1) gx = x + 1 < W ? __ldg(z + y * W + x + 1) - zc : zc - __ldg(z + y * W + x - 1);
  if (H > 1) gy = y + 1 < H ? __ldg(z + (y + 1) * W + x) - zc : zc - __ldg(z + (y - 1) * W + x);
  return make_float2(gx, gy);
}

__device__ __forceinline__ float geom_weight(float zp, float zq, float2 gz, float sx, float sy, f3 np_, f3 nq,
                                             float sigma_z, float sigma_n) {
  const float wz = expf(-fabsf(zp - zq) / (sigma_z * fabsf(gz.x * sx + gz.y * sy) + kEps));
  const float wn = powf(fmaxf(0.0f, dot(np_, nq)), sigma_n);
  return wz * wn;
}

__global__ void svgf_variance_kernel(int W, int H, const float4* __restrict__ rad, const float* __restrict__ z,
                                     const float4* __restrict__ nrm, float sigma_z, float sigma_n,
                                     float4* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  const int p = y * W + x;
  const float zp = __ldg(z + p);
  const f3 np_ = xyz(__ldg(nrm + p));
  const float2 gz = depth_gradient(z, W, H, x, y);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int dy = -3; dy <= 3; ++dy) {
    const int qy = y + dy;
    if (qy < 0 || qy >= H) continue;
    for (int dx = -3; dx <= 3; ++dx) {
      const int qx = x + dx;
      if (qx < 0 || qx >= W) continue;
      const int q = qy * W + qx;
      const float w = geom_weight(zp, __ldg(z + q), gz, (float)dx, (float)dy, np_, xyz(__ldg(nrm + q)), sigma_z,
                                  sigma_n);
      const float l = luminance(__ldg(rad + q));
      s0 += w;
      s1 += w * l;
      s2 += w * l * l;
    }
  }
  const float m1 = s1 / s0, m2 = s2 / s0;
  const float4 c = __ldg(rad + p);
  out[p] = make_float4(c.x, c.y, c.z, fmaxf(0.0f, m2 - m1 * m1));
}

__global__ void svgf_atrous_kernel(int W, int H, int step, const float4* __restrict__ in, const float* __restrict__ z,
                                   const float4* __restrict__ nrm, float sigma_z, float sigma_n, float sigma_l,
                                   float4* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= W || y >= H) return;
  const int p = y * W + x;
  // 3 x 3 Gaussian of the variance, out-of-image taps skipped
  float gs = 0.f, gw = 0.f;
  for (int dy = -1; dy <= 1; ++dy) {
    const int qy = y + dy;
    if (qy < 0 || qy >= H) continue;
    for (int dx = -1; dx <= 1; ++dx) {
      const int qx = x + dx;
      if (qx < 0 || qx >= W) continue;
      const float w = (dx == 0 ? 2.f : 1.f) * (dy == 0 ? 2.f : 1.f);
      gs += w * __ldg(in + qy * W + qx).w;
      gw += w;
    }
  }
  const float den_l = sigma_l * sqrtf(fmaxf(gs / gw, 0.0f)) + kEps;
  const float4 cp = __ldg(in + p);
  const float lp = luminance(cp);
  const float zp = __ldg(z + p);
  const f3 np_ = xyz(__ldg(nrm + p));
  const float2 gz = depth_gradient(z, W, H, x, y);
  const float h1[5] = {1.f / 16.f, 1.f / 4.f, 3.f / 8.f, 1.f / 4.f, 1.f / 16.f};
  float ws = 0.f, ax = 0.f, ay = 0.f, az = 0.f, av = 0.f;
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy) {
    const int qy = y + step * dy;
    if (qy < 0 || qy >= H) continue;
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      const int qx = x + step * dx;
      if (qx < 0 || qx >= W) continue;
      const int q = qy * W + qx;
      const float4 cq = __ldg(in + q);
      float w = h1[dy + 2] * h1[dx + 2];
      w *= geom_weight(zp, __ldg(z + q), gz, (float)(step * dx), (float)(step * dy), np_, xyz(__ldg(nrm + q)),
                       sigma_z, sigma_n);
      w *= expf(-fabsf(lp - luminance(cq)) / den_l);
      ws += w;
      ax += w * cq.x;
      ay += w * cq.y;
      az += w * cq.z;
      av += w * w * cq.w;
    }
  }
  const float inv = 1.0f / ws;
  out[p] = make_float4(ax * inv, ay * inv, az * inv, av * inv * inv);
}

}  // namespace

cudaError_t launch_denoise(int W, int H, const float4* rad, const float* z, const float4* nrm, int iterations,
                           float sigma_z, float sigma_n, float sigma_l, float4* work, float4* out, cudaStream_t s) {
  const dim3 block(16, 16);
  const dim3 grid((W + 15) / 16, (H + 15) / 16);
  // the last pass writes `out`: start in `out` for an even pass count, in `work` for an odd one
  float4* a = (iterations % 2 == 0) ? out : work;
  float4* b = (iterations % 2 == 0) ? work : out;
  svgf_variance_kernel<<<grid, block, 0, s>>>(W, H, rad, z, nrm, sigma_z, sigma_n, a);
  cudaError_t e = cudaGetLastError();
  for (int i = 0; i < iterations && e == cudaSuccess; ++i) {
    svgf_atrous_kernel<<<grid, block, 0, s>>>(W, H, 1 << i, a, z, nrm, sigma_z, sigma_n, sigma_l, b);
    e = cudaGetLastError();
    float4* t = a;
    a = b;
    b = t;
  }
  return e;
}

}  // namespace rtk
