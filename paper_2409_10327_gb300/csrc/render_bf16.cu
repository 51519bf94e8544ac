// BF16 weight image, the consecutive-sample and hard-visibility instantiations
// of the fused BF16 kernel (render_bf16_kernel.cuh) and the light dispatch of
// rt_render_frame / rt_render_frame_multi on RT_BF16.
#include <cuda_bf16.h>

#include "render_bf16_kernel.cuh"

namespace rtk {

// ---- BF16 weight image (runs after the FP32 repack on the same stream) -----
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// I's layer-1 weight of output n and input column k of the A tile [f | PE | 1 | 1 | 0]
// (the bias columns excluded), from the FP32 image.
__device__ __forceinline__ float irt_w1(const float* __restrict__ wp, int n, int k) {
  if (k < 32) return wp[OFF_IW1F + k * 64 + n];
  if (k < kBiasCol) return wp[OFF_IW1P + (k - 32) * 64 + n];
  return 0.0f;
}

// One thread per bf16 element of the image.
__global__ void repack_bf16_kernel(const float* __restrict__ wp, uint8_t* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= WBF16_BYTES / 2) return;
  const int byte = 2 * e;
  __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
  if (byte < OFFB_IB2 || byte >= OFFB_IW1L) {
    // one of the six 64 x 64 swizzled matrices: invert swz128
    const int tile = byte < OFFB_IB2 ? byte / 8192 : 4 + (byte - OFFB_IW1L) / 8192;
    const int o = byte % 8192;
    const int n = (o / 1024) * 8 + (o % 1024) / 128;
    const int chunk = ((o % 128) / 16) ^ (n & 7);
    const int k = chunk * 8 + (o % 16) / 2;
    float f = 0.0f;
    if (tile == 0 || tile == 4) {                       // I layer 1: [f | PE | 1 | 1 | 0]
      f = irt_w1(wp, n, k);
    } else if (tile == 1 || tile == 5) {
      f = wp[OFF_IW2 + k * 64 + n];
    } else if (tile == 2) {                             // B layer 1: [f | 0 | b1]
      if (k < 32) f = wp[OFF_BW1 + k * 64 + n];
    } else {
      f = wp[OFF_BW2 + k * 64 + n];
    }
    v = __float2bfloat16_rn(f);
    if (tile >= 4) {                                    // the rounding residual of the hi tile
      __nv_bfloat16 hi, lo;
      split_bf16(f, hi, lo);
      v = lo;
    }
    if (tile == 0 || tile == 2) {
      const float b = tile == 0 ? wp[OFF_IB1 + n] : wp[OFF_BB1 + n];
      __nv_bfloat16 hi, lo;
      split_bf16(b, hi, lo);
      if (k == kBiasCol) v = hi;
      if (k == kBiasCol + 1) v = lo;
    }
  } else if (byte < OFFB_ONES) {
    // layer-2 bias tiles: row n = 8 x hi/8, 8 x lo/8 (exact scalings by 1/8)
    const int tile = (byte - OFFB_IB2) / 2048, o = (byte - OFFB_IB2) % 2048;
    const int n = o / 32, k = (o % 32) / 2;
    const float b = tile == 0 ? wp[OFF_IB2 + n] : wp[OFF_BB2 + n];
    __nv_bfloat16 hi, lo;
    split_bf16(b, hi, lo);
    v = __float2bfloat16_rn(0.125f * __bfloat162float(k < 8 ? hi : lo));
  } else {
    v = __float2bfloat16_rn(1.0f);                      // the all-ones tile
  }
  *reinterpret_cast<__nv_bfloat16*>(out + byte) = v;
}

cudaError_t launch_repack_bf16(const float* wpack, uint8_t* wbf16, cudaStream_t s) {
  repack_bf16_kernel<<<(WBF16_BYTES / 2 + 255) / 256, 256, 0, s>>>(wpack, wbf16);
  return cudaGetLastError();
}


cudaError_t prepare_render_bf16() {
  cudaError_t e = prepare_wg<2, false, false>();
  e = e != cudaSuccess ? e : prepare_wg<3, false, false>();
  e = e != cudaSuccess ? e : prepare_wg<4, false, false>();
  e = e != cudaSuccess ? e : prepare_wg<4, true, false>();
  e = e != cudaSuccess ? e : prepare_render_bf16_chunked();
  return e;
}

// E lights in launches of up to `max_nl` (1, 2, 4 or 8) lights each; light e
// reads envs + e * env_h * env_w and writes out + e * P.  Every launch
// recomputes the geometry, so fewer, wider launches share more work.  Hard
// visibility always runs 4 warpgroups per CTA.
cudaError_t launch_render_bf16_lights(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P,
                                      long long offset, const float4* envs, int E, float4* out, int num_sms,
                                      int max_nl, int wg, cudaStream_t s) {
  const long long hw = (long long)m.env_h * m.env_w;
  for (int e0 = 0; e0 < E;) {
    int nl = 1;
    while (nl * 2 <= max_nl && nl * 2 <= E - e0) nl *= 2;
    ModelDesc mm = m;
    mm.env = envs + e0 * hw;
    const float4* ee = envs + e0 * hw;
    float4* oo = out + (long long)e0 * P;
    const bool chunk = !m.hard && (m.dpt == 32 || m.dpt == 64) && m.N % m.dpt == 0 && m.N > m.dpt;
    const cudaError_t err =
        chunk       ? launch_render_bf16_chunked(nl, wg, mm, hp, gb, P, offset, ee, oo, num_sms, s)
        : m.hard    ? launch_lights<4, true, false>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s)
        : wg == 2   ? launch_lights<2, false, false>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s)
        : wg == 3   ? launch_lights<3, false, false>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s)
                    : launch_lights<4, false, false>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s);
    if (err != cudaSuccess) return err;
    e0 += nl;
  }
  return cudaSuccess;
}

}  // namespace rtk
