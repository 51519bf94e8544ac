// Hand-written adjoint of the fused renderer (rt_backward).
//
// The loss is any function of the radiance; the caller supplies dLoss/dL per
// pixel.  Gradients flow to the hash table (both encodes) and to every weight
// and bias of B and I.  Sampled directions are constants of the estimator.
// Activations are recomputed, never stored in global memory.
//
// Work unit: as in the FP32 forward, one warp owns one primary point and its
// directions 32 at a time (lane = direction i).  For every chunk the warp
//   1. recomputes I(f, w_i), the bounce, f' = H(x') and B(f'),
//   2. runs each secondary I(f', w'_j) forward and immediately backward
//      (dv'_j and dfr2_j only need dLo2 = (1 - v) dL_i, which is known),
//      collecting dLoss/df' and dLoss/d(a', r', n'),
//   3. back-propagates B (recomputed), then the encode at x': table
//      gradients by float2 atomics and dLoss/dx' through the trilinear
//      weights (zero on a clamped axis),
//   4. turns dx' into dt = dx' . w_i and dz1 through min(softplus, 1), adds
//      dz0 from dv = dL_i . (Lenv(w_i) - L'_o,i), and back-propagates the
//      primary I (recomputed) into its weights and into dLoss/df.
// After the pixel's last chunk the primary encode scatters dLoss/df into the
// table.  Weight gradients of each chunk are small warp GEMMs.  I's (1 + M
// evaluations per chunk) are added to a per-CTA shared-memory accumulator
// (padded rows, shared atomics) that the CTA adds to the caller's blob once at
// the end; B's (one evaluation per chunk) go to the caller's blob directly.
// With MIS primary directions (Sec. 4.1) each draw and its weight are
// constants too; only w_i and its Eq. 1 factor change.
#include "adjoint.cuh"
#include "mis.cuh"

namespace rtk {

namespace {

constexpr int kBW = 6;                     // warps per CTA
constexpr int kBT = 32 * kBW;
// per-warp buffers (floats)
constexpr int WB_F2 = 0;                                   // f' of the chunk's rows  [32 cols]
constexpr int WB_H1 = WB_F2 + kActStride32;                 // layer-1 activations, then dZ1 (in place) [64 cols]
// PE of the current direction [32 cols] for layer 1, then layer-2 activations and dZ2 (in place)
// [64 cols]; the PE is written again for the PE part of dW1 once dZ2 is consumed
constexpr int WB_H2 = WB_H1 + kActStride;
constexpr int WB_DZ = WB_H2 + kActStride;                  // output gradients [8][32]
constexpr int WB_FP = WB_DZ + 8 * 32;                       // primary feature f [32]
constexpr int WB_AP = WB_FP + 32;                           // primary b1 + W1f f [64]
constexpr int WB_DFP = WB_AP + 64;                          // dLoss/df of the pixel [32]
constexpr int WB_FLOATS = WB_DFP + 32;
constexpr size_t kBSmem = (size_t)(WPACK_FLOATS + G_FLOATS + kBW * WB_FLOATS) * sizeof(float);
static_assert(LD_I1 >= 32 + 27 + 1, "gradient rows");
static_assert(kBSmem <= 232448, "one CTA per SM");
static_assert(WB_F2 % 4 == 0 && WB_H1 % 4 == 0 && WB_H2 % 4 == 0 &&
                  WB_DZ % 4 == 0 && WB_FLOATS % 4 == 0 && G_FLOATS % 4 == 0,
              "float4 alignment");

// ---- warp-level pieces of an MLP backward -----------------------------------

__global__ void __launch_bounds__(kBT, 1)
backward_fp32_kernel(ModelDesc m, rt_gbuffer gb, int P, long long pixel_offset, const float4* __restrict__ dL,
                     float* __restrict__ g_table, float* __restrict__ g_brdf, float* __restrict__ g_irt) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  float* sg = sw + WPACK_FLOATS;
  for (int i = threadIdx.x; i < WPACK_FLOATS / 4; i += kBT)
    smem4[i] = __ldg(reinterpret_cast<const float4*>(m.wpack) + i);
  for (int i = threadIdx.x; i < G_FLOATS; i += kBT) sg[i] = 0.0f;
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = lane >> 3, cg = lane & 7;
  float* wb = sg + G_FLOATS + warp * WB_FLOATS;
  float* F2 = wb + WB_F2;
  float* PEb = wb + WB_H2;   // shares H2's buffer (see WB_H2)
  float* H1 = wb + WB_H1;
  float* H2 = wb + WB_H2;
  float* DZ = wb + WB_DZ;
  float* fP = wb + WB_FP;
  float* aP = wb + WB_AP;
  float* dfP = wb + WB_DFP;
  const int N = m.N, M = m.M, lf = m.lf, lfp = m.lfp;
  const bool disney = !m.lambert;
  const BlobB gB{g_brdf, lf};
  const float4* pos4 = reinterpret_cast<const float4*>(gb.pos);
  const float4* nrm4 = reinterpret_cast<const float4*>(gb.normal);
  const float4* view4 = reinterpret_cast<const float4*>(gb.view);
  const float4* ar4 = reinterpret_cast<const float4*>(gb.albedo_rough);

  for (int pix = blockIdx.x * kBW + warp; pix < P; pix += gridDim.x * kBW) {
    const f3 x = xyz(pos4[pix]);
    const f3 n = xyz(nrm4[pix]);
    const f3 wo = xyz(view4[pix]);
    const float4 ar = ar4[pix];
    const f3 G = xyz(dL[pix]);

    // primary feature and I's layer-1 bias for the point (as in the forward)
    {
      const int l = lane >> 1;
      float2 part = make_float2(0.f, 0.f);
      if (l < m.grid.levels) {
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
    __syncwarp();

    for (int i0 = 0; i0 < N; i0 += 32) {
      const int i = i0 + lane;
      const bool valid = i < N;
      const uint64_t q = (uint64_t)(pixel_offset + pix) * (uint64_t)N + (uint64_t)i;
      // the primary direction and its Eq. 1 factor are constants of the estimator (MIS included)
      const f3 wi = m.mis ? mis_direction(m, n, wo, ar.w, i, dir_counter(q, M, 0))
                          : cosine_direction(n, m.seed, dir_counter(q, M, 0));
      float acc[8][8];

      // ---- forward of I(f, w_i)
      store_pe(PEb, wi, lane);
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
      const float v = m.force_vis >= 0.f ? m.force_vis : sigmoidf_(z.x);
      const float sp = softplusf_(z.y);
      const float t = m.near_t + (m.far_t - m.near_t) * fminf(sp, 1.0f);
      const f3 x2 = x + wi * t;

      // ---- f' = H(x') into F2, then B(f')
      __syncwarp();
      for (int l = 0; l < m.grid.levels; ++l) {
        const float2 f = encode_level_exact(m.grid, l, x2);
        F2[aidx(2 * l, lane)] = f.x;
        F2[aidx(2 * l + 1, lane)] = f.y;
      }
      for (int k = lf; k < 32; ++k) F2[aidx(k, lane)] = 0.0f;
      __syncwarp();
      zero(acc);
      warp_gemm_k(F2, sw + OFF_BW1, acc, lfp, rg, cg);
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
      const f3 wo2 = neg(wi);

      // ---- primary shading factors and the incoming-radiance gradient
      const f3 e1 = env_lookup(m.env, m.env_h, m.env_w, wi);
      const f3 fr1 = m.mis ? mis_weighted_brdf(m, xyz(ar), ar.w, n, wo, wi)
                           : brdf_eval(xyz(ar), ar.w, n, wi, wo, m.f0, m.lambert);
      const float sN = kPi / (float)N, sM = kPi / (float)M;
      const f3 dli = valid ? (G * fr1) * sN : mk(0.f, 0.f, 0.f);
      const f3 dlo2 = dli * (1.0f - v);

      // ---- secondary directions: forward and backward of I(f', w'_j)
      float dF2[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) dF2[k] = 0.0f;
      f3 lo2 = mk(0.f, 0.f, 0.f), da2 = mk(0.f, 0.f, 0.f), dn2 = mk(0.f, 0.f, 0.f);
      float dr2 = 0.0f;
      for (int j = 0; j < M; ++j) {
        const f3 wj = cosine_direction(n2, m.seed, dir_counter(q, M, 1 + j));
        __syncwarp();
        store_pe(PEb, wj, lane);
        __syncwarp();
        zero(acc);
        warp_gemm_k(F2, sw + OFF_IW1F, acc, lfp, rg, cg);
        warp_gemm<kPEPad>(PEb, sw + OFF_IW1P, acc, rg, cg);
        store_relu_colbias(H1, acc, sw + OFF_IB1, rg, cg);
        __syncwarp();
        zero(acc);
        warp_gemm<kHidden>(H1, sw + OFF_IW2, acc, rg, cg);
        store_relu_colbias(H2, acc, sw + OFF_IB2, rg, cg);
        __syncwarp();
        const float z0 = irt_head(H2, sw, lane).x;
        const float v2 = m.force_vis2 >= 0.f ? m.force_vis2 : sigmoidf_(z0);
        const f3 le = env_lookup(m.env, m.env_h, m.env_w, wj);
        float ds_dr = 0.0f;
        f3 ds_dn = mk(0.f, 0.f, 0.f);
        const float s = disney ? spec_with_grad(r2, n2, wj, wo2, m.f0, ds_dr, ds_dn) : 0.0f;
        const f3 fr2 = mk(a2.x * kInvPi + s, a2.y * kInvPi + s, a2.z * kInvPi + s);
        const f3 ef = le * fr2;
        lo2 = lo2 + ef * v2;
        // Eq. 1 at x': dLo2 -> dv'_j, d fr2
        const float dv2 = sM * dot(dlo2, ef);
        const f3 dfr = (dlo2 * le) * (sM * v2);
        da2 = da2 + dfr * kInvPi;
        if (disney) {
          const float dsum = dfr.x + dfr.y + dfr.z;
          dr2 += dsum * ds_dr;
          dn2 = dn2 + ds_dn * dsum;
        }
        const float dz0 = m.force_vis2 >= 0.f ? 0.0f : dv2 * v2 * (1.0f - v2);
        DZ[lane] = dz0;
        __syncwarp();
        // I backward: head, W3, W2, hidden, W1 (f' and PE parts), input f'
        bwd_w3<1>(H2, DZ, sg + GI_W3, sg + GI_B3, lane);
        __syncwarp();
        bwd_head<1, 2>(H2, DZ, sw + OFF_IW3, H2, lane);   // dZ2 over H2, in place
        __syncwarp();
        bwd_weights(H1, 64, H2, sg + GI_W2, LD_2, 0, sg + GI_B2, lane);
        __syncwarp();
        bwd_hidden(H2, sw + OFF_IW2, H1, H1, lane);   // dZ1 over H1, in place
        __syncwarp();
        store_pe(PEb, cosine_direction(n2, m.seed, dir_counter(q, M, 1 + j)), lane);   // again, over dZ2
        bwd_weights(F2, lf, H1, sg + GI_W1, LD_I1, 0, sg + GI_B1, lane);
        __syncwarp();
        bwd_weights(PEb, kPE, H1, sg + GI_W1, LD_I1, lf, nullptr, lane);
        bwd_input(H1, sw + OFF_IW1F, lf, dF2, lane);
      }
      lo2 = lo2 * sM;
      const float dv = dot(dli, e1 - lo2);

      // ---- B backward (forward recomputed)
      float dy[7];
      {
        const float dnn = dot(n2, dn2);
        dy[0] = (dn2.x - n2.x * dnn) / nlen;
        dy[1] = (dn2.y - n2.y * dnn) / nlen;
        dy[2] = (dn2.z - n2.z * dnn) / nlen;
        dy[3] = da2.x * a2.x * (1.0f - a2.x);
        dy[4] = da2.y * a2.y * (1.0f - a2.y);
        dy[5] = da2.z * a2.z * (1.0f - a2.z);
        dy[6] = dr2 * 0.91f * s6 * (1.0f - s6);
      }
      __syncwarp();
      zero(acc);
      warp_gemm_k(F2, sw + OFF_BW1, acc, lfp, rg, cg);
      store_relu_colbias(H1, acc, sw + OFF_BB1, rg, cg);
      __syncwarp();
      zero(acc);
      warp_gemm<kHidden>(H1, sw + OFF_BW2, acc, rg, cg);
      store_relu_colbias(H2, acc, sw + OFF_BB2, rg, cg);
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
      bwd_weights(F2, lf, H1, gB.w1(), lf, 0, gB.b1(), lane);
      bwd_input(H1, sw + OFF_BW1, lf, dF2, lane);

      // ---- encode adjoint at x': table gradients (segmented scatter over the warp's points in Morton
      // order) and dLoss/dx'; H2's buffer, free until the next store_pe, carries dx' back to its lane
      uint32_t dbits[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) dbits[k] = __float_as_uint(dF2[k]);
      const f3 dx2 = encode_bwd_sorted(m.grid, x2, dbits, valid, g_table, reinterpret_cast<float4*>(H2));
      const float dt = dot(dx2, wi);
      const float dz1 = (sp <= 1.0f) ? dt * (m.far_t - m.near_t) * sigmoidf_(z.y) : 0.0f;
      const float dz0p = (m.force_vis >= 0.f || !valid) ? 0.0f : dv * v * (1.0f - v);

      // ---- primary I backward (forward recomputed)
      __syncwarp();
      store_pe(PEb, wi, lane);
      __syncwarp();
      zero(acc);
      warp_gemm<kPEPad>(PEb, sw + OFF_IW1P, acc, rg, cg);
      store_relu_colbias(H1, acc, aP, rg, cg);
      __syncwarp();
      zero(acc);
      warp_gemm<kHidden>(H1, sw + OFF_IW2, acc, rg, cg);
      store_relu_colbias(H2, acc, sw + OFF_IB2, rg, cg);
      DZ[lane] = dz0p;
      DZ[32 + lane] = valid ? dz1 : 0.0f;
      __syncwarp();
      bwd_w3<2>(H2, DZ, sg + GI_W3, sg + GI_B3, lane);
      __syncwarp();
      bwd_head<2, 2>(H2, DZ, sw + OFF_IW3, H2, lane);   // dZ2 over H2, in place
      __syncwarp();
      bwd_weights(H1, 64, H2, sg + GI_W2, LD_2, 0, sg + GI_B2, lane);
      __syncwarp();
      bwd_hidden(H2, sw + OFF_IW2, H1, H1, lane);   // dZ1 over H1, in place
      __syncwarp();
      store_pe(PEb, wi, lane);   // again, over the consumed dZ2
      __syncwarp();
      bwd_weights(PEb, kPE, H1, sg + GI_W1, LD_I1, lf, sg + GI_B1, lane);
      // the f part of layer 1 is shared by the chunk's rows: dW1f[c][k] += f[k] colsum(dZ1)[c]
      // and dLoss/df[k] += sum_c colsum(dZ1)[c] W1f[k][c]
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        float cs = 0.0f;
        for (int r = 0; r < 32; ++r) cs += H1[aidx(c, r)];
        DZ[c] = cs;   // scratch: column sums of dZ1 (the output gradients are consumed)
      }
      __syncwarp();
      for (int k = 0; k < lf; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = lane + 32 * h;
          atomicAdd(sg + GI_W1 + c * LD_I1 + k, fP[k] * DZ[c]);
        }
      }
      if (lane < lf) {
        float s = 0.0f;
        for (int c = 0; c < 64; ++c) s = fmaf(DZ[c], sw[OFF_IW1F + lane * 64 + c], s);
        dfP[lane] += s;
      }
      __syncwarp();
    }

    // ---- primary encode adjoint: table gradients at x
    {
      const int l = lane >> 1;
      if ((lane & 1) == 0 && l < m.grid.levels) encode_level_bwd(m.grid, l, x, dfP[lane], dfP[lane + 1], g_table, nullptr);
    }
    __syncwarp();
  }

  // ---- flush the CTA's weight gradients into the caller's blobs (canonical layouts)
  __syncthreads();
  flush_irt_grads(sg, m.lf, g_irt, kBT);
}

}  // namespace

cudaError_t prepare_backward_fp32() {
  return cudaFuncSetAttribute(backward_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmem);
}

cudaError_t launch_backward_fp32(const ModelDesc& m, const rt_gbuffer& gb, int P, long long offset, const float4* dL,
                                 float* g_table, float* g_brdf, float* g_irt, int num_sms, cudaStream_t s) {
  const int need = (P + kBW - 1) / kBW;
  const int grid = need < num_sms ? need : num_sms;
  backward_fp32_kernel<<<grid, kBT, kBSmem, s>>>(m, gb, P, offset, dL, g_table, g_brdf, g_irt);
  return cudaGetLastError();
}

}  // namespace rtk
