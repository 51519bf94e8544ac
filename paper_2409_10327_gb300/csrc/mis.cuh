// Multiple importance sampling of the primary directions (Sec. 4.1): a
// light-importance and a GGX visible-normal strategy, alternating over the
// N directions of a point (light for even i, GGX for odd i; a point seen
// from below, n . w_o <= 1e-4, uses light samples only), combined with the
// balance heuristic.  Each direction's Eq. 1 weight relative to cosine
// sampling, (n . w)+ / (n_L p_L(w) + n_G p_G(w)) * N / pi, rides on its BRDF
// (mis_weighted_brdf).
//   light: texel (r, c) by inverting the float32 CDFs of the bound
//     environment map (built by env_cdf kernels in the same order as their
//     float32 reference), then a point uniform in (phi, theta) inside the
//     texel: p_L = p_texel / (dphi dtheta sin(theta));
//   GGX: Heitz's visible-normal sampler (alpha = r^2) in Duff et al.'s frame
//     about n, reflected: p_G = G1(w_o) D(h) / (4 n . w_o).
#pragma once

#include "device_common.cuh"

namespace rtk {

constexpr float kMisNovMin = 1e-4f;

// largest k in [0, n - 1] with cdf[k] <= u, for cdf[0] = 0 <= u < cdf[n] = 1
__device__ __forceinline__ int cdf_find(const float* __restrict__ cdf, int n, float u) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(cdf + mid) <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

// cdf_find with a cutpoint table (Chen & Asau's guide table): guide[j] =
// cdf_find(cdf, n, j / G) for G = 2^gshift.  For u in [j, j + 1) / G the
// answer lies in [guide[j], guide[j + 1]] because the CDF does not decrease,
// so the bisection over that range returns the same index as over [0, n).
__device__ __forceinline__ int cdf_find_guided(const float* __restrict__ cdf, int n, float u,
                                               const int* __restrict__ guide, int gshift) {
  const int G = 1 << gshift;
  const int j = min((int)(u * (float)G), G - 1);   // exact: G is a power of two
  int lo = __ldg(guide + j);
  int hi = j + 1 < G ? min(__ldg(guide + j + 1) + 1, n) : n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(cdf + mid) <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ f3 mis_light_direction(const ModelDesc& m, float u1, float u2) {
  const int H = m.env_h, W = m.env_w;
  const int r = cdf_find_guided(m.cdf_m, H, u1, m.guide_m, m.gm_shift);
  const float m0 = __ldg(m.cdf_m + r), m1 = __ldg(m.cdf_m + r + 1);
  const float ur = (u1 - m0) / (m1 - m0);
  const float* row = m.cdf_c + (size_t)r * (W + 1);
  const int c = cdf_find_guided(row, W, u2, m.guide_c + ((size_t)r << m.gc_shift), m.gc_shift);
  const float c0 = __ldg(row + c), c1 = __ldg(row + c + 1);
  const float uc = (u2 - c0) / (c1 - c0);
  const float theta = kPi * ((float)r + ur) / (float)H;
  const float phi = 2.0f * kPi * ((float)c + uc) / (float)W - kPi;
  float st, ct, sp, cp;
  sincosf(theta, &st, &ct);
  sincosf(phi, &sp, &cp);
  return mk(st * cp, st * sp, ct);
}

__device__ __forceinline__ float mis_pdf_light(const ModelDesc& m, f3 w) {
  const int H = m.env_h, W = m.env_w;
  const float rho = sqrtf(w.x * w.x + w.y * w.y);
  const float theta = atan2f(rho, w.z);
  const float phi = atan2f(w.y, w.x);
  const int r = min(max((int)floorf(theta * ((float)H / kPi)), 0), H - 1);
  const int c = min(max((int)floorf((phi + kPi) * ((float)W / (2.0f * kPi))), 0), W - 1);
  const float* row = m.cdf_c + (size_t)r * (W + 1);
  const float pt = (__ldg(m.cdf_m + r + 1) - __ldg(m.cdf_m + r)) * (__ldg(row + c + 1) - __ldg(row + c));
  return pt / ((2.0f * kPi / (float)W) * (kPi / (float)H) * rho);
}

// orthonormal (t, b) completing the unit normal n (Duff et al. 2017)
__device__ __forceinline__ void mis_frame(f3 n, f3& t, f3& b) {
  const float sign = n.z >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (sign + n.z);
  const float bb = n.x * n.y * a;
  t = mk(1.0f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
  b = mk(bb, sign + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ f3 mis_ggx_direction(f3 n, f3 wo, float alpha, float u1, float u2) {
  f3 t, b;
  mis_frame(n, t, b);
  const f3 v = mk(dot(wo, t), dot(wo, b), dot(wo, n));
  f3 vh = mk(alpha * v.x, alpha * v.y, v.z);
  vh = vh * rsqrtf(dot(vh, vh));
  const float lensq = vh.x * vh.x + vh.y * vh.y;
  f3 t1 = mk(1.0f, 0.0f, 0.0f);
  if (lensq > 0.0f) {
    const float inv = rsqrtf(lensq);
    t1 = mk(-vh.y * inv, vh.x * inv, 0.0f);
  }
  const f3 t2 = cross(vh, t1);
  const float rr = sqrtf(u1);
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  const float p1 = rr * cp;
  float p2 = rr * sp;
  const float s = 0.5f * (1.0f + vh.z);
  p2 = (1.0f - s) * sqrtf(1.0f - p1 * p1) + s * p2;
  const f3 nh = t1 * p1 + t2 * p2 + vh * sqrtf(fmaxf(1.0f - p1 * p1 - p2 * p2, 0.0f));
  f3 ne = mk(alpha * nh.x, alpha * nh.y, fmaxf(nh.z, 0.0f));
  ne = ne * rsqrtf(dot(ne, ne));
  const f3 h = t * ne.x + b * ne.y + n * ne.z;
  return h * (2.0f * dot(wo, h)) - wo;
}

__device__ __forceinline__ float mis_pdf_ggx(f3 w, f3 n, f3 wo, float alpha) {
  const float nov = dot(n, wo);
  const f3 hv = w + wo;
  const float hl2 = dot(hv, hv);
  if (!(nov > kMisNovMin) || !(hl2 > 0.0f)) return 0.0f;
  const f3 h = hv * rsqrtf(hl2);
  const float noh = dot(n, h), voh = dot(wo, h);
  if (!(noh > 0.0f) || !(voh > 0.0f)) return 0.0f;
  const float a2 = alpha * alpha;
  const f3 c = cross(n, h);
  const float dd = dot(c, c) + noh * noh * a2;
  const float d = a2 / (kPi * dd * dd);
  const float g1 = 2.0f * nov / (nov + sqrtf(a2 + (1.0f - a2) * nov * nov));
  return g1 * d / (4.0f * nov);
}

// f_r(w, w_o) (n . w)+ / (n_L p_L(w) + n_G p_G(w)) * N / pi, the MIS-weighted
// BRDF of a primary direction.  The GGX term D(h) is evaluated once and
// shared by the specular lobe and p_G: a GGX sample in a sharp lobe weighs
// ~ D / D, and two separately rounded D's would not cancel.
__device__ __forceinline__ f3 mis_weighted_brdf(const ModelDesc& m, f3 albedo, float rough, f3 n, f3 wo, f3 w) {
  const float alpha = rough * rough;
  const float a2 = alpha * alpha;
  const float ndl = dot(n, w), ndv = dot(n, wo);
  const float nol = fmaxf(ndl, 0.0f);
  const f3 hv = w + wo;
  const float hl2 = dot(hv, hv);
  float dd = 1.0f, noh = 0.0f, voh = 0.0f;
  if (hl2 > 1e-20f) {
    const float inv = rsqrtf(hl2);
    const f3 h = hv * inv;
    noh = dot(n, h);
    voh = dot(wo, h);
    if (noh > 0.0f) {
      const f3 c = cross(n, h);
      dd = dot(c, c) + noh * noh * a2;
    }
  }
  const float D = a2 / (kPi * dd * dd);
  f3 fr = albedo * kInvPi;
  if (!m.lambert) {
    const float nov = fmaxf(ndv, 1e-4f);
    const float om = 1.0f - fmaxf(voh, 0.0f);
    const float om2 = om * om;
    const float F = m.f0 + (1.0f - m.f0) * (om2 * om2 * om);
    const float den = nol * sqrtf(nov * nov * (1.0f - a2) + a2) + nov * sqrtf(nol * nol * (1.0f - a2) + a2);
    const float spec = D * F * (0.5f / den);
    fr = mk(fr.x + spec, fr.y + spec, fr.z + spec);
  }
  const int N = m.N;
  const bool ggx = ndv > kMisNovMin;
  const float ng = ggx ? (float)(N / 2) : 0.0f;
  float pdf = ((float)N - ng) * mis_pdf_light(m, w);
  if (ggx && noh > 0.0f && voh > 0.0f && hl2 > 0.0f) {
    const float g1 = 2.0f * ndv / (ndv + sqrtf(a2 + (1.0f - a2) * ndv * ndv));
    pdf += ng * (g1 * D / (4.0f * ndv));
  }
  return fr * (nol / pdf * ((float)N / kPi));
}

// Direction of sample i (counter ctr) of a point with normal n, view wo and roughness rough.
__device__ __forceinline__ f3 mis_direction(const ModelDesc& m, f3 n, f3 wo, float rough, int i, uint64_t ctr) {
  const float u1 = uniform24(splitmix64(m.seed, 2 * ctr + 1));
  const float u2 = uniform24(splitmix64(m.seed, 2 * ctr + 2));
  if ((i & 1) && dot(n, wo) > kMisNovMin) return mis_ggx_direction(n, wo, rough * rough, u1, u2);
  return mis_light_direction(m, u1, u2);
}

}  // namespace rtk
