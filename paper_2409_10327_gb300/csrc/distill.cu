// Per-head distillation of the hash renderer (Sec. 3.3 "Training Procedure";
// supplementary "Training Details"): the stratified whole-sphere directions
// (rt_distill_dirs), the FP32 adjoint of the per-head loss
// (rt_distill_backward) and the Adam update (rt_adam_step).
//
// Loss, for P points x with normals n and K directions each:
//   L1 over B's (n', a', r') against the teacher's, averaged over points and
//   the 7 components; BCE of sigmoid(z0) against the teacher's visibility
//   binarised at 0.5 and L1 of min(softplus(z1), 1) against the teacher's
//   normalised depth, each averaged over the point's front-facing directions
//   (w . n > 0) and then over points.
//
// Work, in two phases of one persistent launch.  I phase: a unit is one
// point and up to 128 of its directions; the warp encodes f = H(x), counts
// the point's front-facing directions and walks the unit's directions 32 at
// a time (lane = direction): I forward, the head gradients, I's adjoint with
// the layer-1 f part shared by the rows; then it scatters the unit's share of
// dLoss/df into the table (the encode adjoint is linear in it).  Splitting a
// point's directions over units spreads a small batch (2048 points) over
// every SM.  B phase: a warp takes 32 points as one 32-row tile (lane =
// point), runs B, back-propagates the L1 of the BRDF heads and scatters the
// B part of dLoss/df.  I's weight gradients go to the CTA's shared
// accumulator and then to the caller's blob, B's straight to the caller's
// blob (adjoint.cuh).
#include "adjoint.cuh"

namespace rtk {

namespace {

constexpr int kDW = 6;                      // warps per CTA (shared memory holds one CTA of 6 warps)
constexpr int kUnitDirs = 128;              // directions of one point per I-phase work unit
constexpr int kDT = 32 * kDW;
// per-warp buffers (floats)
constexpr int DB_F = 0;                                    // f of the warp's 32 points [32 cols]
constexpr int DB_H1 = DB_F + kActStride32;                 // layer-1 activations, then dZ1 (in place) [64 cols]
// PE of the current directions [32 cols] for layer 1, then layer-2 activations and dZ2 (in place)
// [64 cols]; the PE is written again for the PE part of dW1 once dZ2 is consumed
constexpr int DB_H2 = DB_H1 + kActStride;
constexpr int DB_DZ = DB_H2 + kActStride;                 // output gradients [8][32]
constexpr int DB_FP = DB_DZ + 8 * 32;                      // f of the current point [32]
constexpr int DB_AP = DB_FP + 32;                          // b1 + W1f f of the current point [64]
constexpr int DB_DFP = DB_AP + 64;                         // dLoss/df of the current point, I part [32]
constexpr int DB_FLOATS = DB_DFP + 32;
constexpr size_t kDSmem = (size_t)(WPACK_FLOATS + G_FLOATS + kDW * DB_FLOATS) * sizeof(float);
static_assert(kDSmem <= 232448, "one CTA per SM");
static_assert(DB_H1 % 4 == 0 && DB_H2 % 4 == 0 && DB_DZ % 4 == 0 &&
                  DB_FLOATS % 4 == 0,
              "float4 alignment");

__device__ __forceinline__ float sgnf(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

__global__ void distill_dirs_kernel(long long PK, int K, int S, long long ray_offset, uint64_t seed,
                                    float4* __restrict__ dirs) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= PK) return;
  const long long p = e / K;
  const int k = (int)(e - p * K);
  const uint64_t ctr = (uint64_t)(ray_offset + p) * (uint64_t)K + (uint64_t)k;
  const float xi1 = uniform24(splitmix64(seed, 2 * ctr + 1));
  const float xi2 = uniform24(splitmix64(seed, 2 * ctr + 2));
  const float u1 = ((float)(k / S) + xi1) / (float)S;
  const float u2 = ((float)(k % S) + xi2) / (float)S;
  const float z = 1.0f - 2.0f * u1;
  const float rho = 2.0f * sqrtf(fmaxf(u1 * (1.0f - u1), 0.0f));
  float sp, cp;
  sincospif(2.0f * u2, &sp, &cp);
  dirs[e] = make_float4(rho * cp, rho * sp, z, 0.0f);
}

__global__ void __launch_bounds__(kDT, 1)
distill_fp32_kernel(ModelDesc m, const float4* __restrict__ pos4, const float4* __restrict__ nrm4, int P, int K,
                    const float4* __restrict__ dirs, const float* __restrict__ brdf_t, const float* __restrict__ vis_t,
                    const float* __restrict__ depth_t, float* __restrict__ loss, float* __restrict__ g_table,
                    float* __restrict__ g_brdf, float* __restrict__ g_irt) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  float* sg = sw + WPACK_FLOATS;
  for (int i = threadIdx.x; i < WPACK_FLOATS / 4; i += kDT)
    smem4[i] = __ldg(reinterpret_cast<const float4*>(m.wpack) + i);
  for (int i = threadIdx.x; i < G_FLOATS; i += kDT) sg[i] = 0.0f;
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = lane >> 3, cg = lane & 7;
  float* wb = sg + G_FLOATS + warp * DB_FLOATS;
  float* F = wb + DB_F;
  float* PEb = wb + DB_H2;   // shares H2's buffer (see DB_H2)
  float* H1 = wb + DB_H1;
  float* H2 = wb + DB_H2;
  float* DZ = wb + DB_DZ;
  float* fP = wb + DB_FP;
  float* aP = wb + DB_AP;
  float* dfP = wb + DB_DFP;
  const int lf = m.lf, lfp = m.lfp, levels = m.grid.levels;
  const BlobB gB{g_brdf, lf};
  const float invR = 1.0f / (float)P;
  const float inv_range = 1.0f / (m.far_t - m.near_t);
  float l_brdf = 0.0f, l_bce = 0.0f, l_depth = 0.0f;

  // ---- I phase: units of (point, up to kUnitDirs of its directions), lane = direction
  const int nch = (K + kUnitDirs - 1) / kUnitDirs;
  const long long units = (long long)P * nch;
  for (long long u = (long long)blockIdx.x * kDW + warp; u < units; u += (long long)gridDim.x * kDW) {
    {
      const int p = (int)(u / nch);
      const int kb = (int)(u - (long long)p * nch) * kUnitDirs;
      const int ke = min(K, kb + kUnitDirs);
      const f3 x = xyz(pos4[p]);
      const f3 n = xyz(nrm4[p]);
      {
        const int l = lane >> 1;
        float2 part = make_float2(0.f, 0.f);
        if (l < levels) {
          const float2 f = encode_level_exact(m.grid, l, x);
          part = (lane & 1) ? make_float2(0.f, 0.f) : f;
        }
        if ((lane & 1) == 0) {
          fP[lane] = part.x;
          fP[lane + 1] = part.y;
        }
        dfP[lane] = 0.0f;
      }
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        float acc = sw[OFF_IB1 + c];
        for (int k = 0; k < lfp; ++k) acc = fmaf(fP[k], sw[OFF_IW1F + k * 64 + c], acc);
        aP[c] = acc;
      }
      int cnt = 0;
      for (int k0 = 0; k0 < K; k0 += 32) {
        const int k = k0 + lane;
        const bool ff = k < K && dot(xyz(dirs[(size_t)p * K + k]), n) > 0.0f;
        cnt += __popc(__ballot_sync(0xffffffffu, ff));
      }
      const float wI = cnt > 0 ? invR / (float)cnt : 0.0f;
      __syncwarp();
      for (int k0 = kb; k0 < ke; k0 += 32) {
        const int k = k0 + lane;
        const bool valid = k < ke;
        const f3 w = valid ? xyz(dirs[(size_t)p * K + k]) : n;
        const bool ff = valid && dot(w, n) > 0.0f;
        float acc[8][8];
        store_pe(PEb, w, lane);
        __syncwarp();
        zero(acc);
        warp_gemm<kPEPad>(PEb, sw + OFF_IW1P, acc, rg, cg);
        store_relu_colbias(H1, acc, aP, rg, cg);
        __syncwarp();
        zero(acc);
        warp_gemm<kHidden>(H1, sw + OFF_IW2, acc, rg, cg);
        store_relu_colbias(H2, acc, sw + OFF_IB2, rg, cg);
        __syncwarp();
        const float2 z = irt_head(H2, sw, lane);
        float dz0 = 0.0f, dz1 = 0.0f;
        if (ff) {
          const size_t e = (size_t)p * K + k;
          const float vt = vis_t[e] > 0.5f ? 1.0f : 0.0f;
          const float dt = (depth_t[e] - m.near_t) * inv_range;
          l_bce += wI * (fmaxf(z.x, 0.0f) - z.x * vt + log1pf(expf(-fabsf(z.x))));
          dz0 = wI * (sigmoidf_(z.x) - vt);
          const float sp = softplusf_(z.y);
          const float d = fminf(sp, 1.0f) - dt;
          l_depth += wI * fabsf(d);
          dz1 = sp < 1.0f ? wI * sgnf(d) * sigmoidf_(z.y) : 0.0f;
        }
        DZ[lane] = dz0;
        DZ[32 + lane] = dz1;
        __syncwarp();
        bwd_w3<2>(H2, DZ, sg + GI_W3, sg + GI_B3, lane);
        __syncwarp();
        bwd_head<2, 2>(H2, DZ, sw + OFF_IW3, H2, lane);   // dZ2 over H2, in place
        __syncwarp();
        bwd_weights(H1, 64, H2, sg + GI_W2, LD_2, 0, sg + GI_B2, lane);
        __syncwarp();
        bwd_hidden(H2, sw + OFF_IW2, H1, H1, lane);   // dZ1 over H1, in place
        __syncwarp();
        store_pe(PEb, w, lane);   // again, over the consumed dZ2
        __syncwarp();
        bwd_weights(PEb, kPE, H1, sg + GI_W1, LD_I1, lf, sg + GI_B1, lane);
        // the f part of layer 1 is shared by the rows: dW1f[c][k] += f[k] colsum(dZ1)[c],
        // dLoss/df[k] += sum_c colsum(dZ1)[c] W1f[k][c]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = lane + 32 * h;
          float cs = 0.0f;
          for (int r = 0; r < 32; ++r) cs += H1[aidx(c, r)];
          DZ[c] = cs;   // scratch: column sums of dZ1 (the output gradients are consumed)
        }
        __syncwarp();
        for (int kk = 0; kk < lf; ++kk) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            atomicAdd(sg + GI_W1 + c * LD_I1 + kk, fP[kk] * DZ[c]);
          }
        }
        if (lane < lf) {
          float s = 0.0f;
          for (int c = 0; c < 64; ++c) s = fmaf(DZ[c], sw[OFF_IW1F + lane * 64 + c], s);
          dfP[lane] += s;
        }
        __syncwarp();
      }
      {
        // the unit's share of dLoss/df (the encode adjoint is linear in it)
        const int l = lane >> 1;
        if ((lane & 1) == 0 && l < levels)
          encode_level_bwd(m.grid, l, x, dfP[lane], dfP[lane + 1], g_table, nullptr);
      }
      __syncwarp();
    }
  }

  // ---- B phase: groups of 32 points as one 32-row tile (lane = point)
  for (int g0 = (blockIdx.x * kDW + warp) * 32; g0 < P; g0 += gridDim.x * kDW * 32) {
    const int p = g0 + lane;
    const bool vp = p < P;
    {
      const f3 x = vp ? xyz(pos4[p]) : mk(0.f, 0.f, 0.f);
#pragma unroll 1
      for (int l = 0; l < kMaxLevels; ++l) {
        const float2 f = (vp && l < levels) ? encode_level_exact(m.grid, l, x) : make_float2(0.f, 0.f);
        F[aidx(2 * l, lane)] = f.x;
        F[aidx(2 * l + 1, lane)] = f.y;
      }
    }
    __syncwarp();
    float acc[8][8];
    zero(acc);
    warp_gemm_k(F, sw + OFF_BW1, acc, lfp, rg, cg);
    store_relu_colbias(H1, acc, sw + OFF_BB1, rg, cg);
    __syncwarp();
    zero(acc);
    warp_gemm<kHidden>(H1, sw + OFF_BW2, acc, rg, cg);
    store_relu_colbias(H2, acc, sw + OFF_BB2, rg, cg);
    __syncwarp();
    float y[7];
#pragma unroll
    for (int o = 0; o < 7; ++o) y[o] = sw[OFF_BB3 + o];
    for (int k = 0; k < kHidden; ++k) {
      const float hk = H2[aidx(k, lane)];
#pragma unroll
      for (int o = 0; o < 7; ++o) y[o] = fmaf(hk, sw[OFF_BW3 + 8 * k + o], y[o]);
    }
    const float nlen = sqrtf(fmaxf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2], 1e-24f));
    const f3 n2 = mk(y[0] / nlen, y[1] / nlen, y[2] / nlen);
    const f3 a2 = mk(sigmoidf_(y[3]), sigmoidf_(y[4]), sigmoidf_(y[5]));
    const float s6 = sigmoidf_(y[6]);
    const float r2 = 0.09f + 0.91f * s6;
    float dy[7];
    {
      const float wB = vp ? invR / 7.0f : 0.0f;
      float t[7];
#pragma unroll
      for (int o = 0; o < 7; ++o) t[o] = vp ? brdf_t[(size_t)p * 8 + o] : 0.0f;
      const float out[7] = {n2.x, n2.y, n2.z, a2.x, a2.y, a2.z, r2};
      float g[7];
#pragma unroll
      for (int o = 0; o < 7; ++o) {
        l_brdf += wB * fabsf(out[o] - t[o]);
        g[o] = wB * sgnf(out[o] - t[o]);
      }
      const f3 dn = mk(g[0], g[1], g[2]);
      const float dnn = dot(n2, dn);
      dy[0] = (dn.x - n2.x * dnn) / nlen;
      dy[1] = (dn.y - n2.y * dnn) / nlen;
      dy[2] = (dn.z - n2.z * dnn) / nlen;
      dy[3] = g[3] * a2.x * (1.0f - a2.x);
      dy[4] = g[4] * a2.y * (1.0f - a2.y);
      dy[5] = g[5] * a2.z * (1.0f - a2.z);
      dy[6] = g[6] * 0.91f * s6 * (1.0f - s6);
    }
#pragma unroll
    for (int o = 0; o < 7; ++o) DZ[o * 32 + lane] = dy[o];
    __syncwarp();
    bwd_w3<7>(H2, DZ, gB.w3(), gB.b3(), lane, 64);
    __syncwarp();
    bwd_head<7, 8>(H2, DZ, sw + OFF_BW3, H2, lane);   // dZ2 over H2, in place
    __syncwarp();
    bwd_weights(H1, 64, H2, gB.w2(), 64, 0, gB.b2(), lane);
    __syncwarp();
    bwd_hidden(H2, sw + OFF_BW2, H1, H1, lane);   // dZ1 over H1, in place
    __syncwarp();
    bwd_weights(F, lf, H1, gB.w1(), lf, 0, gB.b1(), lane);
    float dF[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) dF[k] = 0.0f;
    bwd_input(H1, sw + OFF_BW1, lf, dF, lane);
    {
      // segmented scatter over the warp's points (Morton order, runs of equal rows summed first)
      uint32_t dbits[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) dbits[k] = __float_as_uint(dF[k]);
      const f3 x = vp ? xyz(pos4[p]) : mk(0.f, 0.f, 0.f);
      (void)encode_bwd_sorted<false>(m.grid, x, dbits, vp, g_table, nullptr);
    }
    __syncwarp();
  }

  // ---- loss terms (one atomic per warp) and the weight gradients
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l_brdf += __shfl_xor_sync(0xffffffffu, l_brdf, o);
    l_bce += __shfl_xor_sync(0xffffffffu, l_bce, o);
    l_depth += __shfl_xor_sync(0xffffffffu, l_depth, o);
  }
  if (lane == 0 && loss != nullptr) {
    atomicAdd(loss + 0, l_brdf);
    atomicAdd(loss + 1, l_bce);
    atomicAdd(loss + 2, l_depth);
  }
  __syncthreads();
  flush_irt_grads(sg, m.lf, g_irt, kDT);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, long long n, float lr, float b1, float b2, float eps, float wd,
                            float bc1, float bc2) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gg = g[e] + wd * p[e];
    const float a = b1 * m1[e] + (1.0f - b1) * gg;
    const float b = b2 * m2[e] + (1.0f - b2) * gg * gg;
    m1[e] = a;
    m2[e] = b;
    p[e] -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
  }
}

}  // namespace

cudaError_t prepare_distill() {
  return cudaFuncSetAttribute(distill_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDSmem);
}

cudaError_t launch_distill_dirs(int P, int K, long long ray_offset, uint64_t seed, float4* dirs, cudaStream_t s) {
  int S = 1;
  while ((S + 1) * (S + 1) <= K) ++S;
  const long long PK = (long long)P * K;
  distill_dirs_kernel<<<(unsigned)((PK + 255) / 256), 256, 0, s>>>(PK, K, S, ray_offset, seed, dirs);
  return cudaGetLastError();
}

cudaError_t launch_distill_fp32(const ModelDesc& m, const float4* pos, const float4* nrm, int P, int K,
                                const float4* dirs, const float* brdf_t, const float* vis_t, const float* depth_t,
                                float* loss, float* g_table, float* g_brdf, float* g_irt, int num_sms, cudaStream_t s) {
  const long long units = (long long)P * ((K + kUnitDirs - 1) / kUnitDirs);
  const long long groups = (P + 31) / 32;
  const long long need = ((units > groups ? units : groups) + kDW - 1) / kDW;
  const int grid = (int)(need < num_sms ? need : num_sms);
  distill_fp32_kernel<<<grid, kDT, kDSmem, s>>>(m, pos, nrm, P, K, dirs, brdf_t, vis_t, depth_t, loss, g_table,
                                                g_brdf, g_irt);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, long long n, float lr, float b1, float b2,
                        float eps, float wd, float bc1, float bc2, int num_sms, cudaStream_t s) {
  const long long blocks = (n + 255) / 256;
  const int grid = (int)(blocks < 8LL * num_sms ? blocks : 8LL * num_sms);
  adam_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(p, g, m1, m2, n, lr, b1, b2, eps, wd, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace rtk
