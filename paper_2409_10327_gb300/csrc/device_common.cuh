// Device functions shared by the renderer's kernels: counter-based RNG,
// cosine-lobe directions, hash-grid cells, environment lookup, BRDF and the
// positional encoding.  Each follows the definition stated in include/rt.h.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "rt_internal.h"

namespace rtk {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;

struct f3 {
  float x, y, z;
};
__device__ __forceinline__ f3 mk(float x, float y, float z) { return f3{x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return mk(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ f3 operator*(f3 a, f3 b) { return mk(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ f3 neg(f3 a) { return mk(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ f3 xyz(float4 v) { return mk(v.x, v.y, v.z); }

// ---- SplitMix64 (Steele, Lea & Flood 2014): output k of the stream at state `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// Top 24 bits scaled by 2^-24: exact in float.
__device__ __forceinline__ float uniform24(uint64_t r) {
  return (float)(uint32_t)(r >> 40) * 5.9604644775390625e-8f;
}

// Cosine-weighted direction about unit n for counter `ctr`:
// normalize(n + s), s uniform on the sphere (density of the result ~ w.n).
__device__ __forceinline__ f3 cosine_direction(f3 n, uint64_t seed, uint64_t ctr) {
  const float u1 = uniform24(splitmix64(seed, 2 * ctr + 1));
  const float u2 = uniform24(splitmix64(seed, 2 * ctr + 2));
  const float z = 1.0f - 2.0f * u1;
  const float rho = 2.0f * sqrtf(u1 * (1.0f - u1));
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  const f3 d = mk(n.x + rho * cp, n.y + rho * sp, n.z + z);
  const float l2 = dot(d, d);
  if (l2 > 1e-20f) return d * rsqrtf(l2);
  return n;
}

// ---- hash grid ------------------------------------------------------------
// Cell origin and fraction along one axis: u = x*0.5 + 0.5 clamped, g = u*N,
// each rounded to float32 without contraction so the cell is reproducible.
__device__ __forceinline__ void grid_cell(float x, int res, uint32_t& i0, float& w) {
  float u = __fadd_rn(__fmul_rn(x, 0.5f), 0.5f);
  u = fminf(fmaxf(u, 0.0f), 1.0f);
  const float g = __fmul_rn(u, (float)res);
  int i = (int)floorf(g);
  i = min(i, res - 1);
  i0 = (uint32_t)i;
  w = __fsub_rn(g, (float)i);   // exact
}

// The same cell (decided from the float32 u and g above, so indices stay
// reproducible) with the fraction taken from the exact grid coordinate: u =
// x/2 + 1/2 and g = u N are carried as float32 values plus their rounding
// residuals (Fast2Sum for the sum, an FMA for the product), so w = g - i0 is
// accurate to the rounding of w itself instead of to the rounding of g
// (N 2^-24 of a cell, about 1.2e-4 on a 2048 level).  Where the float32 g
// rounded across a cell face, w lies that hair outside [0, 1]; the trilinear
// interpolant is continuous across the face, so the feature is unaffected.
__device__ __forceinline__ void grid_cell_exact(float x, int res, uint32_t& i0, float& w) {
  const float h = __fmul_rn(x, 0.5f);                       // exact
  float u = __fadd_rn(h, 0.5f);
  float ul = __fadd_rn(__fsub_rn(0.5f, u), h);              // u + ul = h + 1/2 exactly when |h| <= 1/2
  if (u > 1.0f || (u == 1.0f && ul >= 0.0f)) {              // clamp the exact value to [0, 1]
    u = 1.0f;
    ul = 0.0f;
  }
  if (u < 0.0f || (u == 0.0f && ul <= 0.0f)) {
    u = 0.0f;
    ul = 0.0f;
  }
  const float rf = (float)res;
  const float g = __fmul_rn(u, rf);                         // the float32 g of grid_cell
  int i = (int)floorf(g);
  i = min(i, res - 1);
  i0 = (uint32_t)i;
  const float g_lo = __fmaf_rn(ul, rf, __fmaf_rn(u, rf, -g));   // (u + ul) N - g
  w = __fadd_rn(__fsub_rn(g, (float)i), g_lo);
}

__device__ __forceinline__ uint32_t corner_row(uint32_t ix, uint32_t iy, uint32_t iz, int res, int dense,
                                               uint32_t mask) {
  if (dense) {
    const uint32_t n1 = (uint32_t)res + 1u;
    return ix + n1 * (iy + n1 * iz);
  }
  return ((ix * 1u) ^ (iy * 2654435761u) ^ (iz * 805459861u)) & mask;
}

__device__ __forceinline__ float2 table_entry(const GridDesc& g, size_t row) {
  if (g.half) {
    const __half2 h = __ldg(reinterpret_cast<const __half2*>(g.table) + row);
    return __half22float2(h);
  }
  return __ldg(reinterpret_cast<const float2*>(g.table) + row);
}

// Trilinear feature of level l at x.  Corner c has offsets (c&1, c>>1&1, c>>2&1).
__device__ __forceinline__ float2 encode_level(const GridDesc& g, int l, f3 x) {
  const int res = g.res[l];
  uint32_t ix, iy, iz;
  float wx, wy, wz;
  grid_cell(x.x, res, ix, wx);
  grid_cell(x.y, res, iy, wy);
  grid_cell(x.z, res, iz, wz);
  const size_t base = (size_t)l << g.log2T;
  const int dense = g.dense[l];
  float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t row = corner_row(ix + (c & 1), iy + ((c >> 1) & 1), iz + ((c >> 2) & 1), res, dense, g.mask);
    const float w = ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
    const float2 v = table_entry(g, base + row);
    f0 = fmaf(w, v.x, f0);
    f1 = fmaf(w, v.y, f1);
  }
  return make_float2(f0, f1);
}

// encode_level with the exact fractions of grid_cell_exact (the FP32 fused kernels).
__device__ __forceinline__ float2 encode_level_exact(const GridDesc& g, int l, f3 x) {
  const int res = g.res[l];
  uint32_t ix, iy, iz;
  float wx, wy, wz;
  grid_cell_exact(x.x, res, ix, wx);
  grid_cell_exact(x.y, res, iy, wy);
  grid_cell_exact(x.z, res, iz, wz);
  const size_t base = (size_t)l << g.log2T;
  const int dense = g.dense[l];
  float f0 = 0.0f, f1 = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t row = corner_row(ix + (c & 1), iy + ((c >> 1) & 1), iz + ((c >> 2) & 1), res, dense, g.mask);
    const float w = ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
    const float2 v = table_entry(g, base + row);
    f0 = fmaf(w, v.x, f0);
    f1 = fmaf(w, v.y, f1);
  }
  return make_float2(f0, f1);
}

// ---- positional encoding: [w, sin(2^k pi w), cos(2^k pi w)], k = 0..3 ------
// k = 0 by sincospif (exact argument), k > 0 by the double-angle identities.
template <typename Store>
__device__ __forceinline__ void positional_encoding(f3 w, Store st) {
  st(0, w.x);
  st(1, w.y);
  st(2, w.z);
  float s[3], c[3];
  sincospif(w.x, &s[0], &c[0]);
  sincospif(w.y, &s[1], &c[1]);
  sincospif(w.z, &s[2], &c[2]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      st(3 + 6 * k + d, s[d]);
      st(6 + 6 * k + d, c[d]);
    }
    if (k < 3) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const float s2 = 2.0f * s[d] * c[d];
        const float c2 = (c[d] - s[d]) * (c[d] + s[d]);
        s[d] = s2;
        c[d] = c2;
      }
    }
  }
}

// ---- environment map (equirectangular, bilinear, wrap in s, clamp in q) ---
__device__ __forceinline__ f3 env_lookup(const float4* __restrict__ env, int H, int W, f3 w) {
  const float phi = atan2f(w.y, w.x);
  const float theta = atan2f(sqrtf(w.x * w.x + w.y * w.y), w.z);   // = acos(w.z), well conditioned
  const float s = (phi + kPi) * ((float)W * (0.5f * kInvPi)) - 0.5f;
  const float q = theta * ((float)H * kInvPi) - 0.5f;
  const float s0f = floorf(s), q0f = floorf(q);
  const float fs = s - s0f, fq = q - q0f;
  int c0 = (int)s0f % W;
  if (c0 < 0) c0 += W;
  const int c1 = (c0 + 1 == W) ? 0 : c0 + 1;
  const int q0 = (int)q0f;
  const int r0 = min(max(q0, 0), H - 1);
  const int r1 = min(max(q0 + 1, 0), H - 1);
  const float4 e00 = __ldg(env + r0 * W + c0), e01 = __ldg(env + r0 * W + c1);
  const float4 e10 = __ldg(env + r1 * W + c0), e11 = __ldg(env + r1 * W + c1);
  const float a = 1.0f - fs, b = 1.0f - fq;
  return mk(b * (a * e00.x + fs * e01.x) + fq * (a * e10.x + fs * e11.x),
            b * (a * e00.y + fs * e01.y) + fq * (a * e10.y + fs * e11.y),
            b * (a * e00.z + fs * e01.z) + fq * (a * e10.z + fs * e11.z));
}

// ---- simplified Disney BRDF ----------------------------------------------
// f_r = a/pi + D F Vis; D is evaluated with 1 - (n.h)^2 = |n x h|^2 so that it
// stays accurate in float32 at low roughness near n.h = 1.
__device__ __forceinline__ float spec_term(float rough, f3 n, f3 wi, f3 wo, float f0) {
  const float alpha = rough * rough;
  const float a2 = alpha * alpha;
  const float nol = fmaxf(dot(n, wi), 0.0f);
  const float nov = fmaxf(dot(n, wo), 1e-4f);
  const f3 hv = wi + wo;
  const float hl2 = dot(hv, hv);
  float dd = 1.0f, voh = 0.0f;
  if (hl2 > 1e-20f) {
    const float inv = rsqrtf(hl2);
    const f3 h = hv * inv;
    const float noh = dot(n, h);
    voh = 0.5f * hl2 * inv;
    if (noh > 0.0f) {
      const f3 c = cross(n, h);
      dd = dot(c, c) + noh * noh * a2;
    }
  }
  const float D = a2 / (kPi * dd * dd);
  const float om = 1.0f - voh;
  const float om2 = om * om;
  const float F = f0 + (1.0f - f0) * (om2 * om2 * om);
  const float vis = 0.5f / (nol * sqrtf(nov * nov * (1.0f - a2) + a2) + nov * sqrtf(nol * nol * (1.0f - a2) + a2));
  return D * F * vis;
}

__device__ __forceinline__ f3 brdf_eval(f3 albedo, float rough, f3 n, f3 wi, f3 wo, float f0, int lambert) {
  const f3 d = albedo * kInvPi;
  if (lambert) return d;
  const float s = spec_term(rough, n, wi, wo, f0);
  return mk(d.x + s, d.y + s, d.z + s);
}

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }
__device__ __forceinline__ float softplusf_(float z) { return z > 15.0f ? z : log1pf(expf(z)); }
// Visibility from I's logit z0: soft sigmoid(z0) (Eq. 2 as a blend), or the
// hit test of the paper's inference, 1 when sigmoid(z0) > 0.5, i.e. z0 > 0
// (Sec. 3.2 overview).  A forced value (>= 0) replaces the network's; in hard
// mode it counts as 1 above 0.5.
__device__ __forceinline__ float visibility_from_logit(float z0, float forced, int hard) {
  if (forced >= 0.0f) return hard ? (forced > 0.5f ? 1.0f : 0.0f) : forced;
  return hard ? (z0 > 0.0f ? 1.0f : 0.0f) : sigmoidf_(z0);
}

__device__ __forceinline__ float depth_from_logit(float z, float near_t, float far_t) {
  return near_t + (far_t - near_t) * fminf(softplusf_(z), 1.0f);
}

// RNG counters: slot c of secondary sample q.
__device__ __forceinline__ uint64_t dir_counter(uint64_t q, int M, int slot) {
  return q * (uint64_t)(M + 1) + (uint64_t)slot;
}

}  // namespace rtk
