// Stand-alone stage kernels: weight repacking, stage (a) encode, stage (b)
// decode, stage (c) trace, the direction sampler and stage (e) shading at one
// level.  They compute exactly what the fused kernel computes per sample and
// give each stage its own parity check; one thread per output item, except
// the trace, which also serves the teacher of the distillation step (a point
// with K directions) and runs as 32-row warp GEMMs.
#include "warp_gemm.cuh"

namespace rtk {

// ---- weight repacking ------------------------------------------------------
// Canonical blob (per MLP): W1 [64][in], b1 [64], W2 [64][64], b2 [64],
// W3 [out][64], b3 [out].  Output: the transposed image of rt_internal.h.
__global__ void repack_kernel(const float* __restrict__ bw, const float* __restrict__ iw, int lf,
                              float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= WPACK_FLOATS) return;
  const int in_i = lf + kPE;
  // I blob offsets
  const int iW1 = 0, iB1 = iW1 + 64 * in_i, iW2 = iB1 + 64, iB2 = iW2 + 64 * 64, iW3 = iB2 + 64, iB3 = iW3 + 2 * 64;
  // B blob offsets
  const int bW1 = 0, bB1 = bW1 + 64 * lf, bW2 = bB1 + 64, bB2 = bW2 + 64 * 64, bW3 = bB2 + 64, bB3 = bW3 + 7 * 64;
  float v = 0.0f;
  if (e < OFF_IW1P) {                         // I W1, feature rows [k][c]
    const int k = (e - OFF_IW1F) / 64, c = (e - OFF_IW1F) % 64;
    if (k < lf) v = iw[iW1 + c * in_i + k];
  } else if (e < OFF_IB1) {                   // I W1, PE rows
    const int k = (e - OFF_IW1P) / 64, c = (e - OFF_IW1P) % 64;
    if (k < kPE) v = iw[iW1 + c * in_i + lf + k];
  } else if (e < OFF_IW2) {
    v = iw[iB1 + (e - OFF_IB1)];
  } else if (e < OFF_IB2) {
    const int k = (e - OFF_IW2) / 64, c = (e - OFF_IW2) % 64;
    v = iw[iW2 + c * 64 + k];
  } else if (e < OFF_IW3) {
    v = iw[iB2 + (e - OFF_IB2)];
  } else if (e < OFF_IB3) {
    const int k = (e - OFF_IW3) / 2, c = (e - OFF_IW3) % 2;
    v = iw[iW3 + c * 64 + k];
  } else if (e < OFF_BW1) {
    const int c = e - OFF_IB3;
    if (c < 2) v = iw[iB3 + c];
  } else if (e < OFF_BB1) {
    const int k = (e - OFF_BW1) / 64, c = (e - OFF_BW1) % 64;
    if (k < lf) v = bw[bW1 + c * lf + k];
  } else if (e < OFF_BW2) {
    v = bw[bB1 + (e - OFF_BB1)];
  } else if (e < OFF_BB2) {
    const int k = (e - OFF_BW2) / 64, c = (e - OFF_BW2) % 64;
    v = bw[bW2 + c * 64 + k];
  } else if (e < OFF_BW3) {
    v = bw[bB2 + (e - OFF_BB2)];
  } else if (e < OFF_BB3) {
    const int k = (e - OFF_BW3) / 8, c = (e - OFF_BW3) % 8;
    if (c < 7) v = bw[bW3 + c * 64 + k];
  } else {
    const int c = e - OFF_BB3;
    if (c < 7) v = bw[bB3 + c];
  }
  out[e] = v;
}

cudaError_t launch_repack(const float* brdf_w, const float* irt_w, int lf, float* wpack, cudaStream_t s) {
  repack_kernel<<<(WPACK_FLOATS + 255) / 256, 256, 0, s>>>(brdf_w, irt_w, lf, wpack);
  return cudaGetLastError();
}

// ---- per-thread MLP helpers (weights read through the read-only cache) -----
// h1 = relu(b1 + in_a . W1a + in_b . W1b), h2 = relu(b2 + h1 . W2), both [64].
__device__ __forceinline__ void hidden_layers(const float* __restrict__ wp, int offW1a, const float* in_a, int ka,
                                              int offW1b, const float* in_b, int kb, int offB1, int offW2,
                                              int offB2, float (&h2)[kHidden]) {
  float h1[kHidden];
#pragma unroll
  for (int c = 0; c < kHidden; ++c) h1[c] = __ldg(wp + offB1 + c);
  for (int k = 0; k < ka; ++k) {
    const float a = in_a[k];
#pragma unroll
    for (int c = 0; c < kHidden; ++c) h1[c] = fmaf(a, __ldg(wp + offW1a + k * 64 + c), h1[c]);
  }
  for (int k = 0; k < kb; ++k) {
    const float a = in_b[k];
#pragma unroll
    for (int c = 0; c < kHidden; ++c) h1[c] = fmaf(a, __ldg(wp + offW1b + k * 64 + c), h1[c]);
  }
#pragma unroll
  for (int c = 0; c < kHidden; ++c) {
    h1[c] = fmaxf(h1[c], 0.0f);
    h2[c] = __ldg(wp + offB2 + c);
  }
#pragma unroll 4
  for (int k = 0; k < kHidden; ++k) {
    const float a = h1[k];
#pragma unroll
    for (int c = 0; c < kHidden; ++c) h2[c] = fmaf(a, __ldg(wp + offW2 + k * 64 + c), h2[c]);
  }
#pragma unroll
  for (int c = 0; c < kHidden; ++c) h2[c] = fmaxf(h2[c], 0.0f);
}

// ---- stage (a) -------------------------------------------------------------
__global__ void encode_kernel(GridDesc g, const float4* __restrict__ pos, int P, float* __restrict__ feat,
                              uint32_t* __restrict__ idx, float* __restrict__ wout) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const f3 x = xyz(pos[p]);
  const int lf = 2 * g.levels;
  for (int l = 0; l < g.levels; ++l) {
    const float2 f = encode_level(g, l, x);
    feat[(size_t)p * lf + 2 * l] = f.x;
    feat[(size_t)p * lf + 2 * l + 1] = f.y;
    if (idx != nullptr || wout != nullptr) {
      const int res = g.res[l];
      uint32_t ix, iy, iz;
      float wx, wy, wz;
      grid_cell(x.x, res, ix, wx);
      grid_cell(x.y, res, iy, wy);
      grid_cell(x.z, res, iz, wz);
      for (int c = 0; c < 8; ++c) {
        const size_t o = ((size_t)p * g.levels + l) * 8 + c;
        if (idx) idx[o] = corner_row(ix + (c & 1), iy + ((c >> 1) & 1), iz + ((c >> 2) & 1), res, g.dense[l], g.mask);
        if (wout) wout[o] = ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
      }
    }
  }
}

cudaError_t launch_encode(const ModelDesc& m, const float4* pos, int P, float* feat, uint32_t* idx, float* w,
                          cudaStream_t s) {
  encode_kernel<<<(P + 127) / 128, 128, 0, s>>>(m.grid, pos, P, feat, idx, w);
  return cudaGetLastError();
}

// ---- stage (b) -------------------------------------------------------------
__global__ void decode_kernel(ModelDesc m, const float* __restrict__ feat, int P, float* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float f[32];
  for (int k = 0; k < m.lf; ++k) f[k] = feat[(size_t)p * m.lf + k];
  float h2[kHidden];
  hidden_layers(m.wpack, OFF_BW1, f, m.lf, 0, nullptr, 0, OFF_BB1, OFF_BW2, OFF_BB2, h2);
  float y[8];
#pragma unroll
  for (int o = 0; o < 7; ++o) {
    float acc = __ldg(m.wpack + OFF_BB3 + o);
#pragma unroll
    for (int k = 0; k < kHidden; ++k) acc = fmaf(h2[k], __ldg(m.wpack + OFF_BW3 + k * 8 + o), acc);
    y[o] = acc;
  }
  const float inv = rsqrtf(fmaxf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2], 1e-24f));
  float4* o4 = reinterpret_cast<float4*>(out + (size_t)p * 8);
  o4[0] = make_float4(y[0] * inv, y[1] * inv, y[2] * inv, sigmoidf_(y[3]));
  o4[1] = make_float4(sigmoidf_(y[4]), sigmoidf_(y[5]), 0.09f + 0.91f * sigmoidf_(y[6]), 0.0f);
}

cudaError_t launch_decode(const ModelDesc& m, const float* feat, int P, float* brdf, cudaStream_t s) {
  decode_kernel<<<(P + 127) / 128, 128, 0, s>>>(m, feat, P, brdf);
  return cudaGetLastError();
}

// ---- stage (c) -------------------------------------------------------------
// A warp takes one point's directions 32 at a time (lane = direction): the
// point's layer-1 feature part b1 + W1f f once, then the PE part, layer 2 and
// the head as in the FP32 frame kernel.  The PE lives in the layer-2 buffer
// until layer 1 has read it.
constexpr int kTW = 8;                                    // warps per CTA
constexpr int kTWFloats = 2 * kActStride + 96;            // H1, PE/H2, f (32), b1 + W1f f (64)
constexpr size_t kTSmem = (size_t)(WPACK_FLOATS + kTW * kTWFloats) * sizeof(float);
static_assert(kTSmem <= 232448, "one CTA per SM");

__global__ void __launch_bounds__(kTW * 32, 1)
trace_kernel(ModelDesc m, const float* __restrict__ feat, const float4* __restrict__ dirs, int P, int K,
             float* __restrict__ vis, float* __restrict__ depth) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  for (int i = threadIdx.x; i < WPACK_FLOATS / 4; i += kTW * 32)
    smem4[i] = __ldg(reinterpret_cast<const float4*>(m.wpack) + i);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = lane >> 3, cg = lane & 7;
  float* H1 = sw + WPACK_FLOATS + warp * kTWFloats;
  float* H2 = H1 + kActStride;
  float* fP = H2 + kActStride;
  float* aP = fP + 32;
  const int nch = (K + 31) / 32;
  const long long units = (long long)P * nch;
  long long cur = -1;
  for (long long u = (long long)blockIdx.x * kTW + warp; u < units; u += (long long)gridDim.x * kTW) {
    const long long p = u / nch;
    const int k = (int)(u - p * nch) * 32 + lane;
    if (p != cur) {
      __syncwarp();
      fP[lane] = lane < m.lf ? feat[p * m.lf + lane] : 0.0f;
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        float acc = sw[OFF_IB1 + c];
        for (int j = 0; j < m.lfp; ++j) acc = fmaf(fP[j], sw[OFF_IW1F + j * 64 + c], acc);
        aP[c] = acc;
      }
      cur = p;
    }
    const bool valid = k < K;
    const long long e = p * K + k;
    const f3 w = valid ? xyz(dirs[e]) : mk(0.f, 0.f, 1.f);
    float acc[8][8];
    store_pe(H2, w, lane);
    __syncwarp();
    zero(acc);
    warp_gemm<kPEPad>(H2, sw + OFF_IW1P, acc, rg, cg);
    store_relu_colbias(H1, acc, aP, rg, cg);
    __syncwarp();
    zero(acc);
    warp_gemm<kHidden>(H1, sw + OFF_IW2, acc, rg, cg);
    store_relu_colbias(H2, acc, sw + OFF_IB2, rg, cg);
    __syncwarp();
    const float2 z = irt_head(H2, sw, lane);
    if (valid) {
      vis[e] = sigmoidf_(z.x);
      depth[e] = depth_from_logit(z.y, m.near_t, m.far_t);
    }
    __syncwarp();
  }
}

cudaError_t launch_trace(const ModelDesc& m, const float* feat, const float4* dirs, int P, int K, float* vis,
                         float* depth, int num_sms, cudaStream_t s) {
  const long long units = (long long)P * ((K + 31) / 32);
  const long long need = (units + kTW - 1) / kTW;
  const int grid = (int)(need < num_sms ? need : num_sms);
  trace_kernel<<<grid, kTW * 32, kTSmem, s>>>(m, feat, dirs, P, K, vis, depth);
  return cudaGetLastError();
}

// ---- direction sampler -----------------------------------------------------
__global__ void sample_kernel(ModelDesc m, const float4* __restrict__ normal, long long PK, int K, int level,
                              long long offset, float4* __restrict__ dirs) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= PK) return;
  const long long p = e / K;
  const int k = (int)(e % K);
  uint64_t ctr;
  if (level == 0) {
    const uint64_t q = (uint64_t)(offset + p) * (uint64_t)m.N + (uint64_t)k;
    ctr = dir_counter(q, m.M, 0);
  } else {
    ctr = dir_counter((uint64_t)(offset + p), m.M, 1 + k);
  }
  const f3 w = cosine_direction(xyz(normal[p]), m.seed, ctr);
  dirs[e] = make_float4(w.x, w.y, w.z, 0.0f);
}

cudaError_t launch_sample(const ModelDesc& m, const float4* normal, int P, int level, long long offset,
                          float4* dirs, cudaStream_t s) {
  const int K = level == 0 ? m.N : m.M;
  const long long PK = (long long)P * K;
  sample_kernel<<<(unsigned)((PK + 127) / 128), 128, 0, s>>>(m, normal, PK, K, level, offset, dirs);
  return cudaGetLastError();
}

// ---- stage (e) at one level ------------------------------------------------
__global__ void shade_kernel(ModelDesc m, rt_gbuffer pts, int P, int level, long long offset,
                             const float* __restrict__ vis, const float4* __restrict__ lin, float4* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const f3 n = xyz(reinterpret_cast<const float4*>(pts.normal)[p]);
  const f3 wo = xyz(reinterpret_cast<const float4*>(pts.view)[p]);
  const float4 ar = reinterpret_cast<const float4*>(pts.albedo_rough)[p];
  const f3 alb = xyz(ar);
  const int K = level == 0 ? m.N : m.M;
  f3 acc = mk(0.f, 0.f, 0.f);
  for (int k = 0; k < K; ++k) {
    uint64_t ctr;
    if (level == 0) ctr = dir_counter((uint64_t)(offset + p) * (uint64_t)m.N + (uint64_t)k, m.M, 0);
    else ctr = dir_counter((uint64_t)(offset + p), m.M, 1 + k);
    const f3 w = cosine_direction(n, m.seed, ctr);
    const float v = vis[(size_t)p * K + k];
    f3 li = env_lookup(m.env, m.env_h, m.env_w, w) * v;
    if (lin != nullptr) li = li + xyz(lin[(size_t)p * K + k]) * (1.0f - v);
    acc = acc + li * brdf_eval(alb, ar.w, n, w, wo, m.f0, m.lambert);
  }
  const float sc = kPi / (float)K;
  out[p] = make_float4(acc.x * sc, acc.y * sc, acc.z * sc, 0.0f);
}

cudaError_t launch_shade(const ModelDesc& m, const rt_gbuffer& pts, int P, int level, long long offset,
                         const float* vis, const float4* lin, float4* out, cudaStream_t s) {
  shade_kernel<<<(P + 127) / 128, 128, 0, s>>>(m, pts, P, level, offset, vis, lin, out);
  return cudaGetLastError();
}

cudaError_t prepare_render_fp32();
cudaError_t prepare_render_bf16();
cudaError_t prepare_backward_fp32();

cudaError_t prepare_kernels() {
  cudaError_t e = prepare_render_fp32();
  if (e == cudaSuccess) e = prepare_render_bf16();
  if (e == cudaSuccess) e = prepare_backward_fp32();
  if (e == cudaSuccess) e = prepare_backward_bf16();
  if (e == cudaSuccess) e = prepare_distill();
  if (e == cudaSuccess) e = cudaFuncSetAttribute(trace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
  return e;
}

}  // namespace rtk
