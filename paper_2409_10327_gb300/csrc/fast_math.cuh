// Reduced-precision device functions for the BF16 path.  The MLP operands of
// that path are rounded to bf16 (8-bit significand), so the sampler, the
// positional encoding and the environment lookup may use the MUFU
// approximations (about 1e-6 absolute error here) without changing its
// accuracy; the FP32 path keeps the correctly rounded library functions.
#pragma once

#include "device_common.cuh"

namespace rtk {

__device__ __forceinline__ float sigmoid_fast(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float softplus_fast(float z) { return z > 15.0f ? z : __logf(1.0f + __expf(z)); }
__device__ __forceinline__ float depth_fast(float z, float near_t, float far_t) {
  return near_t + (far_t - near_t) * fminf(softplus_fast(z), 1.0f);
}

// atan(a) for 0 <= a <= 1 by the polynomial of Abramowitz & Stegun 4.4.49
// (|error| <= 2e-8), then atan2 by octant reduction.
__device__ __forceinline__ float atan01(float a) {
  const float x2 = a * a;
  float p = 0.0028662257f;
  p = fmaf(p, x2, -0.0161657367f);
  p = fmaf(p, x2, 0.0429096138f);
  p = fmaf(p, x2, -0.0752896400f);
  p = fmaf(p, x2, 0.1065626393f);
  p = fmaf(p, x2, -0.1420889944f);
  p = fmaf(p, x2, 0.1999355085f);
  p = fmaf(p, x2, -0.3333314528f);
  return fmaf(p * x2, a, a);
}
__device__ __forceinline__ float atan2_fast(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  float r = mx > 0.0f ? atan01(__fdividef(mn, mx)) : 0.0f;
  if (ay > ax) r = 1.57079632679489662f - r;
  if (x < 0.0f) r = kPi - r;
  return copysignf(r, y);
}

// Cosine-weighted direction (same definition and counters as cosine_direction).
__device__ __forceinline__ f3 cosine_direction_fast(f3 n, uint64_t seed, uint64_t ctr) {
  const float u1 = uniform24(splitmix64(seed, 2 * ctr + 1));
  const float u2 = uniform24(splitmix64(seed, 2 * ctr + 2));
  const float z = 1.0f - 2.0f * u1;
  const float rho = 2.0f * sqrtf(u1 * (1.0f - u1));
  float sp, cp;
  __sincosf(2.0f * kPi * u2, &sp, &cp);
  const f3 d = mk(n.x + rho * cp, n.y + rho * sp, n.z + z);
  const float l2 = dot(d, d);
  if (l2 > 1e-20f) return d * rsqrtf(l2);
  return n;
}

// PE(w) with k = 0 from __sincosf(pi w) (|pi w| <= pi) and k > 0 by double angles.
template <typename Store>
__device__ __forceinline__ void positional_encoding_fast(f3 w, Store st) {
  st(0, w.x);
  st(1, w.y);
  st(2, w.z);
  float s[3], c[3];
  __sincosf(kPi * w.x, &s[0], &c[0]);
  __sincosf(kPi * w.y, &s[1], &c[1]);
  __sincosf(kPi * w.z, &s[2], &c[2]);
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

// Equirectangular lookup (same texel convention as env_lookup).
__device__ __forceinline__ f3 env_lookup_fast(const float4* __restrict__ env, int H, int W, f3 w) {
  const float phi = atan2_fast(w.y, w.x);
  const float theta = atan2_fast(sqrtf(w.x * w.x + w.y * w.y), w.z);
  const float s = (phi + kPi) * ((float)W * (0.5f * kInvPi)) - 0.5f;
  const float q = theta * ((float)H * kInvPi) - 0.5f;
  const float s0f = floorf(s), q0f = floorf(q);
  const float fs = s - s0f, fq = q - q0f;
  int c0 = (int)s0f;
  c0 = c0 < 0 ? c0 + W : (c0 >= W ? c0 - W : c0);
  c0 = min(max(c0, 0), W - 1);
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

// The same lookup split in two: the texel taps and weights of a direction
// (the arctangents), computed once, then the fetch from one map, so that a
// direction can be shaded against several environment maps of one size.
struct EnvTap {
  int o00, o01, o10, o11;   // texel offsets (row * W + column)
  float fs, fq;             // bilinear weights along s and q
};
__device__ __forceinline__ EnvTap env_tap_fast(int H, int W, f3 w) {
  const float phi = atan2_fast(w.y, w.x);
  const float theta = atan2_fast(sqrtf(w.x * w.x + w.y * w.y), w.z);
  const float s = (phi + kPi) * ((float)W * (0.5f * kInvPi)) - 0.5f;
  const float q = theta * ((float)H * kInvPi) - 0.5f;
  const float s0f = floorf(s), q0f = floorf(q);
  EnvTap t;
  t.fs = s - s0f;
  t.fq = q - q0f;
  int c0 = (int)s0f;
  c0 = c0 < 0 ? c0 + W : (c0 >= W ? c0 - W : c0);
  c0 = min(max(c0, 0), W - 1);
  const int c1 = (c0 + 1 == W) ? 0 : c0 + 1;
  const int q0 = (int)q0f;
  const int r0 = min(max(q0, 0), H - 1);
  const int r1 = min(max(q0 + 1, 0), H - 1);
  t.o00 = r0 * W + c0;
  t.o01 = r0 * W + c1;
  t.o10 = r1 * W + c0;
  t.o11 = r1 * W + c1;
  return t;
}
__device__ __forceinline__ f3 env_fetch(const float4* __restrict__ env, const EnvTap& t) {
  const float4 e00 = __ldg(env + t.o00), e01 = __ldg(env + t.o01);
  const float4 e10 = __ldg(env + t.o10), e11 = __ldg(env + t.o11);
  const float a = 1.0f - t.fs, b = 1.0f - t.fq;
  return mk(b * (a * e00.x + t.fs * e01.x) + t.fq * (a * e10.x + t.fs * e11.x),
            b * (a * e00.y + t.fs * e01.y) + t.fq * (a * e10.y + t.fs * e11.y),
            b * (a * e00.z + t.fs * e01.z) + t.fq * (a * e10.z + t.fs * e11.z));
}

__device__ __forceinline__ f3 brdf_eval_fast(f3 albedo, float rough, f3 n, f3 wi, f3 wo, float f0, int lambert) {
  const f3 d = albedo * kInvPi;
  if (lambert) return d;
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
  const float om = 1.0f - voh;
  const float om2 = om * om;
  const float F = f0 + (1.0f - f0) * (om2 * om2 * om);
  const float den = nol * sqrtf(nov * nov * (1.0f - a2) + a2) + nov * sqrtf(nol * nol * (1.0f - a2) + a2);
  const float s = __fdividef(a2 * F * 0.5f, kPi * dd * dd * den);
  return mk(d.x + s, d.y + s, d.z + s);
}

}  // namespace rtk
