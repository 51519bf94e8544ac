// Warp-level FP32 GEMM primitives shared by the FP32 forward and backward
// kernels.  A warp multiplies a 32-row activation block by a K x 64 weight
// matrix held in shared memory.  Activations are stored k-major ("column"
// k holds the 32 rows contiguously) with a 4-float pad after every 8 columns:
// element (k, row) is at aidx(k, row).  Each lane owns an 8-row x 8-column
// output tile (rows 8rg..8rg+7, columns ocol(cg, 0..7)).
#pragma once

#include "device_common.cuh"

namespace rtk {

constexpr int kActStride = 64 * 32 + 8 * 4;      // one 64-column activation buffer (floats)
constexpr int kActStride32 = 32 * 32 + 4 * 4;    // one 32-column activation buffer (floats)

// element (k, row) of an activation buffer
__device__ __forceinline__ int aidx(int k, int row) { return k * 32 + (k >> 3) * 4 + row; }

// Column owned by output slot c (0..7) of lane group cg: slots 0-3 are
// columns 4cg..4cg+3 and slots 4-7 are 32+4cg..32+4cg+3, so that each of the
// two float4 weight reads of a k step covers one contiguous 128-byte row span
// (one shared-memory wavefront).
__device__ __forceinline__ int ocol(int cg, int c) { return (c < 4 ? 0 : 28) + cg * 4 + c; }

// acc[r][c] += sum_k act(k, 8rg + r) * W[k][ocol(cg, c)]
template <int K>
__device__ __forceinline__ void warp_gemm(const float* __restrict__ act, const float* __restrict__ W,
                                          float (&acc)[8][8], int rg, int cg) {
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float* ap = act + aidx(k, rg * 8);
    const float4 a0 = *reinterpret_cast<const float4*>(ap);
    const float4 a1 = *reinterpret_cast<const float4*>(ap + 4);
    const float* wp = W + k * 64 + cg * 4;
    const float4 w0 = *reinterpret_cast<const float4*>(wp);
    const float4 w1 = *reinterpret_cast<const float4*>(wp + 32);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], wv[c], acc[r][c]);
  }
}

__device__ __forceinline__ void zero(float (&acc)[8][8]) {
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.0f;
}

// out(col, row) = relu(acc + bias[col])
__device__ __forceinline__ void store_relu_colbias(float* __restrict__ out, const float (&acc)[8][8],
                                                   const float* __restrict__ bias, int rg, int cg) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int col = ocol(cg, c);
    const float b = bias[col];
    float* o = out + aidx(col, rg * 8);
    *reinterpret_cast<float4*>(o) = make_float4(fmaxf(acc[0][c] + b, 0.f), fmaxf(acc[1][c] + b, 0.f),
                                                fmaxf(acc[2][c] + b, 0.f), fmaxf(acc[3][c] + b, 0.f));
    *reinterpret_cast<float4*>(o + 4) = make_float4(fmaxf(acc[4][c] + b, 0.f), fmaxf(acc[5][c] + b, 0.f),
                                                    fmaxf(acc[6][c] + b, 0.f), fmaxf(acc[7][c] + b, 0.f));
  }
}

// out(col, row) = relu(acc + bias[r][c]) (per-row bias held in registers)
__device__ __forceinline__ void store_relu_tilebias(float* __restrict__ out, const float (&acc)[8][8],
                                                    const float (&bias)[8][8], int rg, int cg) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int col = ocol(cg, c);
    float* o = out + aidx(col, rg * 8);
    *reinterpret_cast<float4*>(o) =
        make_float4(fmaxf(acc[0][c] + bias[0][c], 0.f), fmaxf(acc[1][c] + bias[1][c], 0.f),
                    fmaxf(acc[2][c] + bias[2][c], 0.f), fmaxf(acc[3][c] + bias[3][c], 0.f));
    *reinterpret_cast<float4*>(o + 4) =
        make_float4(fmaxf(acc[4][c] + bias[4][c], 0.f), fmaxf(acc[5][c] + bias[5][c], 0.f),
                    fmaxf(acc[6][c] + bias[6][c], 0.f), fmaxf(acc[7][c] + bias[7][c], 0.f));
  }
}

// layer 1 over a runtime K (multiple of 8, <= 32)
__device__ __forceinline__ void warp_gemm_k(const float* act, const float* W, float (&acc)[8][8], int K, int rg,
                                            int cg) {
  if (K == 8) warp_gemm<8>(act, W, acc, rg, cg);
  else if (K == 16) warp_gemm<16>(act, W, acc, rg, cg);
  else if (K == 24) warp_gemm<24>(act, W, acc, rg, cg);
  else warp_gemm<32>(act, W, acc, rg, cg);
}

// write PE(w) of this lane's row and zero rows 27..31
__device__ __forceinline__ void store_pe(float* act, f3 w, int lane) {
  positional_encoding(w, [&](int k, float v) { act[aidx(k, lane)] = v; });
#pragma unroll
  for (int k = kPE; k < kPEPad; ++k) act[aidx(k, lane)] = 0.0f;
}

// I's output layer for this lane's row: z = b3 + h2 . W3  (2 outputs)
__device__ __forceinline__ float2 irt_head(const float* act, const float* sw, int lane) {
  float z0 = sw[OFF_IB3], z1 = sw[OFF_IB3 + 1];
#pragma unroll 8
  for (int k = 0; k < kHidden; ++k) {
    const float h = act[aidx(k, lane)];
    const float2 w = *reinterpret_cast<const float2*>(sw + OFF_IW3 + 2 * k);
    z0 = fmaf(h, w.x, z0);
    z1 = fmaf(h, w.y, z1);
  }
  return make_float2(z0, z1);
}


}  // namespace rtk
