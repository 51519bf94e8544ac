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

// Bitonic sort of one 32-bit key per lane across the warp, ascending with the
// lane index.  All 32 lanes take part.
__device__ __forceinline__ uint32_t warp_sort_u32(uint32_t key) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint32_t other = __shfl_xor_sync(0xffffffffu, key, j);
      const bool up = (lane & (unsigned)k) == 0u;     // this k-block is sorted ascending
      const bool lower = (lane & (unsigned)j) == 0u;  // this lane is the lower position of its pair
      key = (lower == up) ? min(key, other) : max(key, other);
    }
  }
  return key;
}
// An integer of up to 10 bits spread to every third bit (the Morton interleave of one axis).
__device__ __forceinline__ uint32_t morton_spread(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
// The cell of coordinate u in [-1, 1] on a 256-cell axis (clamped).
__device__ __forceinline__ uint32_t morton_cell8(float u) {
  const float q = fminf(fmaxf((u * 0.5f + 0.5f) * 256.0f, 0.0f), 255.0f);
  return (uint32_t)q;
}

// The encode adjoint at the warp's 32 points (one per lane; `valid` marks the
// real ones): for every level, the table
// gradient of the 8 corners of each point's cell and dLoss/dx.  df holds the
// lane's dLoss/df as FP32 bits, features (2l, 2l + 1) of level l.
// Segmented scatter: the warp's points are first put in Morton order of their
// position (8 bits per axis) by a bitonic sort across the lanes, so that points
// that share a table row on a level sit, for the most part, in consecutive
// lanes.  Each run of consecutive lanes on one row is summed by a shuffle tree
// bounded by the run (a fixed order of additions) and reaches the table as one
// float2 reduction; a row whose points are not consecutive receives one
// reduction per run.  Levels without runs cost one ballot per corner over the
// plain scatter.  With WANT_DX, returns dLoss/dx of this lane's own point, and
// scratch is 512 bytes of the warp's shared memory (the points' dx on their way
// back); without it, returns zero and scratch is unused (may be null).
template <bool WANT_DX = true>
__device__ __forceinline__ f3 encode_bwd_sorted(const GridDesc& g, f3 x, const uint32_t (&df)[32], bool valid,
                                                float* __restrict__ g_table, float4* scratch) {
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t code = (morton_spread(morton_cell8(x.x)) << 2) | (morton_spread(morton_cell8(x.y)) << 1) |
                        morton_spread(morton_cell8(x.z));   // 24 bits
  // key: invalid flag, Morton code, lane (unique, so the sort is a permutation of the lanes)
  const uint32_t key = warp_sort_u32((valid ? 0u : 0x80000000u) | (code << 5) | lane);
  const int src = (int)(key & 31u);
  const int nv = __popc(__ballot_sync(0xffffffffu, valid));
  const bool live = (int)lane < nv;   // the valid points come first in the sorted order
  const f3 xs = mk(__shfl_sync(0xffffffffu, x.x, src), __shfl_sync(0xffffffffu, x.y, src),
                   __shfl_sync(0xffffffffu, x.z, src));
  uint32_t d[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) d[k] = __shfl_sync(0xffffffffu, df[k], src);

  f3 dx = mk(0.f, 0.f, 0.f);
#pragma unroll 1
  for (int l = 0; l < g.levels; ++l) {
    float df0 = 0.f, df1 = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k == l) {
        df0 = __uint_as_float(d[2 * k]);
        df1 = __uint_as_float(d[2 * k + 1]);
      }
    const int res = g.res[l];
    uint32_t ix, iy, iz;
    float wx, wy, wz;
    grid_cell_exact(xs.x, res, ix, wx);
    grid_cell_exact(xs.y, res, iy, wy);
    grid_cell_exact(xs.z, res, iz, wz);
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
      const uint32_t prev = __shfl_up_sync(0xffffffffu, row, 1);
      const bool head = lane == 0u || prev != row || !live;
      const unsigned heads = __ballot_sync(0xffffffffu, head);
      if (heads != 0xffffffffu) {
        // this lane's run is [lane, end): end is the next head (32 if none)
        const unsigned rest = heads & ~((2u << lane) - 1u);
        const unsigned end = rest ? (unsigned)(__ffs(rest) - 1) : 32u;
        const unsigned span = __reduce_max_sync(0xffffffffu, head ? end - lane : 0u);
        for (unsigned s = 1; s < span; s <<= 1) {
          const float o0 = __shfl_down_sync(0xffffffffu, v0, s);
          const float o1 = __shfl_down_sync(0xffffffffu, v1, s);
          if (lane + s < end) {
            v0 += o0;
            v1 += o1;
          }
        }
      }
      if (head && live) atomicAdd(reinterpret_cast<float2*>(g_table) + base + row, make_float2(v0, v1));
      if (WANT_DX && live) {
        const float2 e = table_entry(g, base + row);
        const float de = e.x * df0 + e.y * df1;
        gx += de * (ox ? 1.0f : -1.0f) * ay * az;
        gy += de * (oy ? 1.0f : -1.0f) * ax * az;
        gz += de * (oz ? 1.0f : -1.0f) * ax * ay;
      }
    }
    if (WANT_DX) {
      // dg/dx = N_l / 2 inside the box, 0 on a clamped axis
      const float s = 0.5f * (float)res;
      const float ux = xs.x * 0.5f + 0.5f, uy = xs.y * 0.5f + 0.5f, uz = xs.z * 0.5f + 0.5f;
      dx.x += (ux >= 0.0f && ux <= 1.0f) ? gx * s : 0.0f;
      dx.y += (uy >= 0.0f && uy <= 1.0f) ? gy * s : 0.0f;
      dx.z += (uz >= 0.0f && uz <= 1.0f) ? gz * s : 0.0f;
    }
  }
  if (!WANT_DX) return dx;
  // back to the lane that owns the point
  scratch[src] = make_float4(dx.x, dx.y, dx.z, 0.0f);
  __syncwarp();
  const float4 r = scratch[lane];
  __syncwarp();
  return mk(r.x, r.y, r.z);
}

// s = D F Vis of the simplified Disney model and its derivatives with respect
// to the roughness r and the normal n (w_i, w_o fixed).  The n-derivative is
// the textbook one (n.h, n.w_i, n.w_o as independent inputs); the component
// along n is irrelevant because the decoder's normal is normalised.
__device__ __forceinline__ float spec_with_grad(float rough, f3 n, f3 wi, f3 wo, float f0, float& ds_dr, f3& ds_dn) {
  const float alpha = rough * rough;
  const float a2 = alpha * alpha;
  const float ndl = dot(n, wi), ndv = dot(n, wo);
  const float nol = fmaxf(ndl, 0.0f), nov = fmaxf(ndv, 1e-4f);
  const f3 hv = wi + wo;
  const float hl2 = dot(hv, hv);
  f3 h = mk(0.f, 0.f, 0.f);
  float ndh = 0.0f, voh = 0.0f, q = 1.0f;
  if (hl2 > 1e-20f) {
    const float inv = rsqrtf(hl2);
    h = hv * inv;
    ndh = dot(n, h);
    voh = 0.5f * hl2 * inv;
    if (ndh > 0.0f) {
      const f3 c = cross(n, h);
      q = dot(c, c) + ndh * ndh * a2;     // = (n.h)^2 (a2 - 1) + 1 on the unit sphere
    }
  }
  const float noh = fmaxf(ndh, 0.0f);
  const float D = a2 / (kPi * q * q);
  const float om = 1.0f - voh;
  const float om2 = om * om;
  const float F = f0 + (1.0f - f0) * (om2 * om2 * om);
  const float A = sqrtf(nov * nov * (1.0f - a2) + a2);
  const float B = sqrtf(nol * nol * (1.0f - a2) + a2);
  const float den = nol * A + nov * B;
  const float vis = 0.5f / den;
  const float dD_da2 = 1.0f / (kPi * q * q) - 2.0f * a2 * noh * noh / (kPi * q * q * q);
  const float dD_dnoh = -4.0f * a2 * noh * (a2 - 1.0f) / (kPi * q * q * q);
  const float dvis_dden = -0.5f / (den * den);
  const float dden_da2 = nol * (1.0f - nov * nov) / (2.0f * A) + nov * (1.0f - nol * nol) / (2.0f * B);
  const float dden_dnol = A + nov * nol * (1.0f - a2) / B;
  const float dden_dnov = nol * nov * (1.0f - a2) / A + B;
  const float ds_da2 = F * (dD_da2 * vis + D * dvis_dden * dden_da2);
  ds_dr = ds_da2 * 4.0f * rough * rough * rough;
  const float g_nol = ndl > 0.0f ? F * D * dvis_dden * dden_dnol : 0.0f;
  const float g_nov = ndv > 1e-4f ? F * D * dvis_dden * dden_dnov : 0.0f;
  const float g_noh = ndh > 0.0f ? F * vis * dD_dnoh : 0.0f;
  ds_dn = wi * g_nol + wo * g_nov + h * g_noh;
  return D * F * vis;
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
