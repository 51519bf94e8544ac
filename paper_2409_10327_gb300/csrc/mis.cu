// Texel distribution of the bound environment map for the light strategy of
// the MIS primary sampler (Sec. 4.1): luminance 0.2126 R + 0.7152 G +
// 0.0722 B, negative parts clipped, plus 1e-6; conditional CDFs along each
// row and a marginal CDF over rows.  The inversion of these CDFs decides
// integers, so they are built in float32 with every product and sum
// rounded on its own (no contraction), running sums in index order, one
// correctly rounded division by the total, and the last entry set to 1.
// Cutpoint tables over each CDF then start the sampler's bisection close to
// its answer.
#include "mis.cuh"

namespace rtk {
namespace {

__global__ void env_cdf_rows_kernel(const float4* __restrict__ env, int H, int W, float* __restrict__ cdf_m,
                                    float* __restrict__ cdf_c) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= H) return;
  float* row = cdf_c + (size_t)r * (W + 1);
  float s = 0.0f;
  row[0] = 0.0f;
  for (int c = 0; c < W; ++c) {
    const float4 e = env[(size_t)r * W + c];
    float lum = __fadd_rn(__fadd_rn(__fmul_rn(e.x, 0.2126f), __fmul_rn(e.y, 0.7152f)), __fmul_rn(e.z, 0.0722f));
    lum = __fadd_rn(fmaxf(lum, 0.0f), 1e-6f);
    s = __fadd_rn(s, lum);
    row[c + 1] = s;
  }
  for (int c = 1; c < W; ++c) row[c] = __fdiv_rn(row[c], s);
  row[W] = 1.0f;
  cdf_m[r + 1] = s;   // the row total, turned into the marginal CDF below
}

__global__ void env_cdf_marginal_kernel(int H, float* __restrict__ cdf_m) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  cdf_m[0] = 0.0f;
  float s = 0.0f;
  for (int r = 1; r <= H; ++r) {
    s = __fadd_rn(s, cdf_m[r]);
    cdf_m[r] = s;
  }
  for (int r = 1; r < H; ++r) cdf_m[r] = __fdiv_rn(cdf_m[r], s);
  cdf_m[H] = 1.0f;
}

// Cutpoint tables: entry j of a CDF's table is the bisection's answer for
// u = j / 2^shift (exact in float32); thread per entry, the marginal's
// table in row -1.
__global__ void env_guide_kernel(int H, int W, const float* __restrict__ cdf_m, const float* __restrict__ cdf_c,
                                 int* __restrict__ guide_m, int gm_shift, int* __restrict__ guide_c, int gc_shift) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long Gm = 1LL << gm_shift, Gc = 1LL << gc_shift;
  if (k < Gm) {
    guide_m[k] = cdf_find(cdf_m, H, (float)k * (1.0f / (float)Gm));
    return;
  }
  const long long e = k - Gm;
  if (e >= (long long)H * Gc) return;
  const long long r = e >> gc_shift, j = e & (Gc - 1);
  guide_c[e] = cdf_find(cdf_c + r * (W + 1), W, (float)j * (1.0f / (float)Gc));
}

}  // namespace

cudaError_t launch_env_cdf(const float4* env, int H, int W, float* cdf_m, float* cdf_c, int* guide_m, int gm_shift,
                           int* guide_c, int gc_shift, cudaStream_t s) {
  env_cdf_rows_kernel<<<(H + 127) / 128, 128, 0, s>>>(env, H, W, cdf_m, cdf_c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  env_cdf_marginal_kernel<<<1, 32, 0, s>>>(H, cdf_m);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (1LL << gm_shift) + (long long)H * (1LL << gc_shift);
  env_guide_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(H, W, cdf_m, cdf_c, guide_m, gm_shift, guide_c,
                                                               gc_shift);
  return cudaGetLastError();
}

}  // namespace rtk
