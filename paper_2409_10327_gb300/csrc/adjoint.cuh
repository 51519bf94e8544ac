// Shared pieces of the hand-written FP32 adjoints (rt_backward, rt_distill_backward):
// the per-CTA weight-gradient accumulator of I in shared memory (I runs 1 + M
// times per row chunk; B, which runs once, adds its gradients straight into
// the caller's blob with global atomics: BlobB gives its offsets), the warp-level
// adjoints of the MLP layers (one row per lane, activations in the k-major
// layout of warp_gemm.cuh) and of the trilinear hash encode, and the flush
// of the accumulator into the caller's gradient blobs.
#pragma once

#include "warp_gemm.cuh"

namespace rtk {

// I's gradient accumulator in shared memory (floats; rows padded to K + 1)
constexpr int LD_I1 = 60;                  // >= L*F + 27 + 1
constexpr int LD_2 = 65;
constexpr int GI_W1 = 0, GI_B1 = GI_W1 + 64 * LD_I1, GI_W2 = GI_B1 + 64, GI_B2 = GI_W2 + 64 * LD_2;
constexpr int GI_W3 = GI_B2 + 64, GI_B3 = GI_W3 + 2 * LD_2;
constexpr int G_FLOATS = (GI_B3 + 2 + 3) / 4 * 4;

// B's gradient blob (canonical layout of rt_param_count: W1 [64][lf], b1, W2 [64][64], b2, W3 [7][64], b3)
struct BlobB {
  float* g;
  int lf;
  __device__ __forceinline__ float* w1() const { return g; }
  __device__ __forceinline__ float* b1() const { return g + 64 * lf; }
  __device__ __forceinline__ float* w2() const { return g + 64 * lf + 64; }
  __device__ __forceinline__ float* b2() const { return g + 64 * lf + 64 + 4096; }
  __device__ __forceinline__ float* w3() const { return g + 64 * lf + 128 + 4096; }
  __device__ __forceinline__ float* b3() const { return g + 64 * lf + 128 + 4096 + 448; }
};
// DZ2(c, row) = (sum_o dz[o][row] W3[c][o]) * [H2(c, row) > 0]   (thread per row)
template <int NOUT, int LDW>
__device__ __forceinline__ void bwd_head(const float* H2, const float* dz, const float* W3, float* DZ2, int lane) {
  float g[NOUT];
#pragma unroll
  for (int o = 0; o < NOUT; ++o) g[o] = dz[o * 32 + lane];
#pragma unroll 8
  for (int c = 0; c < 64; ++c) {
    float s = 0.0f;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) s = fmaf(g[o], W3[c * LDW + o], s);
    DZ2[aidx(c, lane)] = H2[aidx(c, lane)] > 0.0f ? s : 0.0f;
  }
}

// dW3[o][k] += sum_rows H2(k, row) dz[o][row]; db3[o] += sum_rows dz[o][row]
template <int NOUT>
__device__ __forceinline__ void bwd_w3(const float* H2, const float* dz, float* gW3, float* gb3, int lane,
                                       int ld = LD_2) {
#pragma unroll 1   // rolled: unrolled, the two passes' global atomics keep too many registers live
  for (int kk = 0; kk < 2; ++kk) {
    const int k = 2 * lane + kk;
    float acc[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; ++o) acc[o] = 0.0f;
    for (int r = 0; r < 32; ++r) {
      const float h = H2[aidx(k, r)];
#pragma unroll
      for (int o = 0; o < NOUT; ++o) acc[o] = fmaf(h, dz[o * 32 + r], acc[o]);
    }
#pragma unroll
    for (int o = 0; o < NOUT; ++o) atomicAdd(gW3 + o * ld + k, acc[o]);
  }
  if (lane < NOUT) {
    float s = 0.0f;
    for (int r = 0; r < 32; ++r) s += dz[lane * 32 + r];
    atomicAdd(gb3 + lane, s);
  }
}

// dW[c][koff + k] += sum_rows A(k, row) D(c, row) for k < K, c in {2 lane, 2 lane + 1};
// if gb != nullptr also db[c] += sum_rows D(c, row)
__device__ __forceinline__ void bwd_weights(const float* A, int K, const float* D, float* gW, int ld, int koff,
                                            float* gb, int lane) {
#pragma unroll
  for (int cc = 0; cc < 2; ++cc) {
    const int c = 2 * lane + cc;
    float d[32];
#pragma unroll
    for (int r = 0; r < 32; r += 4) {
      const float4 v = *reinterpret_cast<const float4*>(D + aidx(c, r));
      d[r] = v.x;
      d[r + 1] = v.y;
      d[r + 2] = v.z;
      d[r + 3] = v.w;
    }
    if (gb != nullptr) {
      float s = 0.0f;
#pragma unroll
      for (int r = 0; r < 32; ++r) s += d[r];
      atomicAdd(gb + c, s);
    }
    for (int k = 0; k < K; ++k) {
      float s = 0.0f;
#pragma unroll
      for (int r = 0; r < 32; r += 4) {
        const float4 a = *reinterpret_cast<const float4*>(A + aidx(k, r));
        s = fmaf(a.x, d[r], s);
        s = fmaf(a.y, d[r + 1], s);
        s = fmaf(a.z, d[r + 2], s);
        s = fmaf(a.w, d[r + 3], s);
      }
      atomicAdd(gW + c * ld + koff + k, s);
    }
  }
}

// OUT(k, row) = (sum_c D(c, row) W[k][c]) * [MASK(k, row) > 0] for k < 64 (thread per row);
// W is a [64][64] shared matrix stored [k][c]
__device__ __forceinline__ void bwd_hidden(const float* D, const float* W, const float* MASK, float* OUT, int lane) {
  float d[64];
#pragma unroll
  for (int c = 0; c < 64; ++c) d[c] = D[aidx(c, lane)];
  for (int k = 0; k < 64; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 64; c += 4) {
      const float4 w = *reinterpret_cast<const float4*>(W + k * 64 + c);
      s = fmaf(d[c], w.x, s);
      s = fmaf(d[c + 1], w.y, s);
      s = fmaf(d[c + 2], w.z, s);
      s = fmaf(d[c + 3], w.w, s);
    }
    OUT[aidx(k, lane)] = MASK[aidx(k, lane)] > 0.0f ? s : 0.0f;
  }
}

// din[k] += sum_c D(c, row) W[k][c] for k < K (thread per row)
__device__ __forceinline__ void bwd_input(const float* D, const float* W, int K, float (&din)[32], int lane) {
  float d[64];
#pragma unroll
  for (int c = 0; c < 64; ++c) d[c] = D[aidx(c, lane)];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < K) {
      float s = 0.0f;
#pragma unroll
      for (int c = 0; c < 64; c += 4) {
        const float4 w = *reinterpret_cast<const float4*>(W + k * 64 + c);
        s = fmaf(d[c], w.x, s);
        s = fmaf(d[c + 1], w.y, s);
        s = fmaf(d[c + 2], w.z, s);
        s = fmaf(d[c + 3], w.w, s);
      }
      din[k] += s;
    }
  }
}

// trilinear encode adjoint at point x for one level: table gradient scatter
// and (optionally) dLoss/dx
__device__ __forceinline__ void encode_level_bwd(const GridDesc& g, int l, f3 x, float df0, float df1,
                                                 float* __restrict__ g_table, f3* dx) {
  const int res = g.res[l];
  uint32_t ix, iy, iz;
  float wx, wy, wz;
  grid_cell_exact(x.x, res, ix, wx);
  grid_cell_exact(x.y, res, iy, wy);
  grid_cell_exact(x.z, res, iz, wz);
  const size_t base = (size_t)l << g.log2T;
  const int dense = g.dense[l];
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
    const uint32_t row = corner_row(ix + ox, iy + oy, iz + oz, res, dense, g.mask);
    const float ax = ox ? wx : 1.0f - wx, ay = oy ? wy : 1.0f - wy, az = oz ? wz : 1.0f - wz;
    const float w = ax * ay * az;
    atomicAdd(reinterpret_cast<float2*>(g_table) + base + row, make_float2(w * df0, w * df1));
    if (dx != nullptr) {
      const float2 e = table_entry(g, base + row);
      const float de = e.x * df0 + e.y * df1;
      gx += de * (ox ? 1.0f : -1.0f) * ay * az;
      gy += de * (oy ? 1.0f : -1.0f) * ax * az;
      gz += de * (oz ? 1.0f : -1.0f) * ax * ay;
    }
  }
  if (dx != nullptr) {
    // dg/dx = N_l / 2 inside the box, 0 on a clamped axis
    const float s = 0.5f * (float)res;
    const float ux = x.x * 0.5f + 0.5f, uy = x.y * 0.5f + 0.5f, uz = x.z * 0.5f + 0.5f;
    dx->x += (ux >= 0.0f && ux <= 1.0f) ? gx * s : 0.0f;
    dx->y += (uy >= 0.0f && uy <= 1.0f) ? gy * s : 0.0f;
    dx->z += (uz >= 0.0f && uz <= 1.0f) ? gz * s : 0.0f;
  }
}

// The same adjoint for the lanes `act` of a warp that all process level l,
// each at its own point (the secondary points x' of a chunk's directions, or
// the points of a B tile).  Lanes whose corner c falls on the same table row
// (common on the coarse levels, where a pixel's directions share cells) are
// summed inside the warp by a shuffle tree over their ranks among that row's
// lanes, so the sum has a fixed order, and the row receives one float2
// reduction instead of one per lane.  Where no row repeats (the usual case on
// the fine hashed levels) every lane adds its own contribution.
__device__ __forceinline__ void encode_level_bwd_warp(const GridDesc& g, int l, f3 x, float df0, float df1,
                                                      float* __restrict__ g_table, f3* dx, unsigned act) {
  const int res = g.res[l];
  const unsigned lane = threadIdx.x & 31u;
  uint32_t ix, iy, iz;
  float wx, wy, wz;
  grid_cell_exact(x.x, res, ix, wx);
  grid_cell_exact(x.y, res, iy, wy);
  grid_cell_exact(x.z, res, iz, wz);
  const size_t base = (size_t)l << g.log2T;
  const int dense = g.dense[l];
  float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
    const uint32_t row = corner_row(ix + ox, iy + oy, iz + oz, res, dense, g.mask);
    const float ax = ox ? wx : 1.0f - wx, ay = oy ? wy : 1.0f - wy, az = oz ? wz : 1.0f - wz;
    const float w = ax * ay * az;
    float v0 = w * df0, v1 = w * df1;
    const unsigned grp = __match_any_sync(act, row);
    bool lead = true;
    if (__any_sync(act, grp != (1u << lane))) {
      const unsigned rank = __popc(grp & ((1u << lane) - 1u));
#pragma unroll
      for (unsigned s = 1; s < 32; s <<= 1) {
        const unsigned src = __fns(grp, lane, (int)s + 1);   // the lane s places after this one in its row
        const bool take = (rank % (2 * s)) == 0 && src < 32u;
        const float o0 = __shfl_sync(act, v0, take ? src : lane);
        const float o1 = __shfl_sync(act, v1, take ? src : lane);
        if (take) {
          v0 += o0;
          v1 += o1;
        }
      }
      lead = rank == 0;
    }
    if (lead) atomicAdd(reinterpret_cast<float2*>(g_table) + base + row, make_float2(v0, v1));
    if (dx != nullptr) {
      const float2 e = table_entry(g, base + row);
      const float de = e.x * df0 + e.y * df1;
      gx += de * (ox ? 1.0f : -1.0f) * ay * az;
      gy += de * (oy ? 1.0f : -1.0f) * ax * az;
      gz += de * (oz ? 1.0f : -1.0f) * ax * ay;
    }
  }
  if (dx != nullptr) {
    const float s = 0.5f * (float)res;
    const float ux = x.x * 0.5f + 0.5f, uy = x.y * 0.5f + 0.5f, uz = x.z * 0.5f + 0.5f;
    dx->x += (ux >= 0.0f && ux <= 1.0f) ? gx * s : 0.0f;
    dx->y += (uy >= 0.0f && uy <= 1.0f) ? gy * s : 0.0f;
    dx->z += (uz >= 0.0f && uz <= 1.0f) ? gz * s : 0.0f;
  }
}

// Add the CTA's accumulated gradients of I into the caller's blob (canonical
// layout of rt_param_count); called by all threads after a barrier.
__device__ __forceinline__ void flush_irt_grads(const float* sg, int lf, float* __restrict__ g_irt, int nthreads) {
  const int in_i = lf + kPE;
  const int iW1 = 0, iB1 = 64 * in_i, iW2 = iB1 + 64, iB2 = iW2 + 4096, iW3 = iB2 + 64, iB3 = iW3 + 128;
  for (int e = threadIdx.x; e < 64 * in_i; e += nthreads) atomicAdd(g_irt + iW1 + e, sg[GI_W1 + (e / in_i) * LD_I1 + e % in_i]);
  for (int e = threadIdx.x; e < 64; e += nthreads) {
    atomicAdd(g_irt + iB1 + e, sg[GI_B1 + e]);
    atomicAdd(g_irt + iB2 + e, sg[GI_B2 + e]);
  }
  for (int e = threadIdx.x; e < 4096; e += nthreads) atomicAdd(g_irt + iW2 + e, sg[GI_W2 + (e / 64) * LD_2 + e % 64]);
  for (int e = threadIdx.x; e < 128; e += nthreads) atomicAdd(g_irt + iW3 + e, sg[GI_W3 + (e / 64) * LD_2 + e % 64]);
  for (int e = threadIdx.x; e < 2; e += nthreads) atomicAdd(g_irt + iB3 + e, sg[GI_B3 + e]);
}

}  // namespace rtk
