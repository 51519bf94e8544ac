// Fused FP32 hot path: stages (a)-(e) of the hash renderer in one persistent
// kernel (rt_render_frame with precision RT_FP32).
//
// Work unit: one warp owns one primary point at a time and walks its N
// directions in chunks of 32, one direction per lane.  The MLP layers of the
// chunk are 32 x 64 x K products computed by a register-tiled SIMT GEMM
// (each lane owns an 8-row x 8-column output tile; weights live in shared
// memory for the whole kernel).  Activations pass between layers through a
// per-warp shared buffer laid out k-major with a 4-float pad every 8 rows, so
// the GEMM operand reads are broadcasts and the epilogue stores are free of
// bank conflicts.  The per-point reductions over directions are warp
// shuffles; nothing but the radiance is written to global memory.
#include "mis.cuh"
#include "warp_gemm.cuh"

namespace rtk {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kWarpFloats = 2 * kActStride + 96;  // two buffers + primary feature (32) + primary bias (64)
constexpr size_t kSmemBytes = (size_t)(WPACK_FLOATS + kWarps * kWarpFloats) * sizeof(float);

__global__ void __launch_bounds__(kThreads, 1)
render_fp32_kernel(ModelDesc m, rt_gbuffer gb, int P, long long pixel_offset, float4* __restrict__ out) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  for (int i = threadIdx.x; i < WPACK_FLOATS / 4; i += kThreads)
    smem4[i] = __ldg(reinterpret_cast<const float4*>(m.wpack) + i);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rg = lane >> 3, cg = lane & 7;
  float* actA = sw + WPACK_FLOATS + warp * kWarpFloats;
  float* actB = actA + kActStride;
  float* fP = actB + kActStride;   // primary feature, 32 floats
  float* aP = fP + 32;             // primary layer-1 bias b1 + W1f f, 64 floats
  const int N = m.N, M = m.M, lfp = m.lfp;
  const float4* pos4 = reinterpret_cast<const float4*>(gb.pos);
  const float4* nrm4 = reinterpret_cast<const float4*>(gb.normal);
  const float4* view4 = reinterpret_cast<const float4*>(gb.view);
  const float4* ar4 = reinterpret_cast<const float4*>(gb.albedo_rough);

  for (int pix = blockIdx.x * kWarps + warp; pix < P; pix += gridDim.x * kWarps) {
    const f3 x = xyz(pos4[pix]);
    const f3 n = xyz(nrm4[pix]);
    const f3 wo = xyz(view4[pix]);
    const float4 ar = ar4[pix];
    const f3 alb = xyz(ar);

    // (a) primary feature: lane 2l and 2l+1 each gather 4 corners of level l
    {
      const int l = lane >> 1;
      float2 part = make_float2(0.f, 0.f);
      if (l < m.grid.levels) {
        const int res = m.grid.res[l];
        uint32_t ix, iy, iz;
        float wx, wy, wz;
        grid_cell_exact(x.x, res, ix, wx);
        grid_cell_exact(x.y, res, iy, wy);
        grid_cell_exact(x.z, res, iz, wz);
        const size_t base = (size_t)l << m.grid.log2T;
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c = (lane & 1) * 4 + cc;
          const uint32_t row = corner_row(ix + (c & 1), iy + ((c >> 1) & 1), iz + ((c >> 2) & 1), res,
                                          m.grid.dense[l], m.grid.mask);
          const float w = ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
          const float2 v = table_entry(m.grid, base + row);
          part.x = fmaf(w, v.x, part.x);
          part.y = fmaf(w, v.y, part.y);
        }
      }
      part.x += __shfl_xor_sync(0xffffffffu, part.x, 1);
      part.y += __shfl_xor_sync(0xffffffffu, part.y, 1);
      if ((lane & 1) == 0) {
        fP[lane] = part.x;
        fP[lane + 1] = part.y;
      }
    }
    __syncwarp();
    // primary layer-1 bias of I: b1 + W1f . f (shared by all N directions)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      float acc = sw[OFF_IB1 + c];
      for (int k = 0; k < lfp; ++k) acc = fmaf(fP[k], sw[OFF_IW1F + k * 64 + c], acc);
      aP[c] = acc;
    }
    __syncwarp();

    f3 sum = mk(0.f, 0.f, 0.f);
    for (int i0 = 0; i0 < N; i0 += 32) {
      const int i = i0 + lane;
      const uint64_t q = (uint64_t)(pixel_offset + pix) * (uint64_t)N + (uint64_t)i;
      // primary direction (MIS: its Eq. 1 weight relative to cosine sampling rides on the BRDF below)
      const f3 wi = m.mis ? mis_direction(m, n, wo, ar.w, i, dir_counter(q, M, 0))
                          : cosine_direction(n, m.seed, dir_counter(q, M, 0));

      // (c) I(f, w_i)
      float acc[8][8];
      store_pe(actA, wi, lane);
      __syncwarp();
      zero(acc);
      warp_gemm<kPEPad>(actA, sw + OFF_IW1P, acc, rg, cg);
      store_relu_colbias(actB, acc, aP, rg, cg);
      __syncwarp();
      zero(acc);
      warp_gemm<kHidden>(actB, sw + OFF_IW2, acc, rg, cg);
      store_relu_colbias(actA, acc, sw + OFF_IB2, rg, cg);
      __syncwarp();
      const float2 z = irt_head(actA, sw, lane);
      const float v = visibility_from_logit(z.x, m.force_vis, m.hard);
      const float t = depth_from_logit(z.y, m.near_t, m.far_t);

      // (d) bounce: x' = x + t w_i, f' = H(x')
      const f3 x2 = x + wi * t;
      __syncwarp();
      for (int l = 0; l < m.grid.levels; ++l) {
        const float2 f = encode_level_exact(m.grid, l, x2);
        actA[aidx(2 * l, lane)] = f.x;
        actA[aidx(2 * l + 1, lane)] = f.y;
      }
      for (int k = m.lf; k < lfp; ++k) actA[aidx(k, lane)] = 0.0f;
      __syncwarp();

      // (b) B(f') layer 1, and I's layer-1 bias for the secondary point
      zero(acc);
      warp_gemm_k(actA, sw + OFF_BW1, acc, lfp, rg, cg);
      store_relu_colbias(actB, acc, sw + OFF_BB1, rg, cg);
      float a2b[8][8];
      zero(a2b);
      warp_gemm_k(actA, sw + OFF_IW1F, a2b, lfp, rg, cg);
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) a2b[r][c] += sw[OFF_IB1 + ocol(cg, c)];
      __syncwarp();
      zero(acc);
      warp_gemm<kHidden>(actB, sw + OFF_BW2, acc, rg, cg);
      store_relu_colbias(actA, acc, sw + OFF_BB2, rg, cg);
      __syncwarp();
      float y[7];
#pragma unroll
      for (int o = 0; o < 7; ++o) y[o] = sw[OFF_BB3 + o];
#pragma unroll 4
      for (int k = 0; k < kHidden; ++k) {
        const float h = actA[aidx(k, lane)];
        const float4 w0 = *reinterpret_cast<const float4*>(sw + OFF_BW3 + 8 * k);
        const float4 w1 = *reinterpret_cast<const float4*>(sw + OFF_BW3 + 8 * k + 4);
        y[0] = fmaf(h, w0.x, y[0]);
        y[1] = fmaf(h, w0.y, y[1]);
        y[2] = fmaf(h, w0.z, y[2]);
        y[3] = fmaf(h, w0.w, y[3]);
        y[4] = fmaf(h, w1.x, y[4]);
        y[5] = fmaf(h, w1.y, y[5]);
        y[6] = fmaf(h, w1.z, y[6]);
      }
      const float ninv = rsqrtf(fmaxf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2], 1e-24f));
      const f3 n2 = mk(y[0] * ninv, y[1] * ninv, y[2] * ninv);
      const f3 a2 = mk(sigmoidf_(y[3]), sigmoidf_(y[4]), sigmoidf_(y[5]));
      const float r2 = 0.09f + 0.91f * sigmoidf_(y[6]);
      const f3 wo2 = neg(wi);

      // (c) + (e) at x': M directions about n'
      f3 lo2 = mk(0.f, 0.f, 0.f);
      for (int j = 0; j < M; ++j) {
        const f3 wj = cosine_direction(n2, m.seed, dir_counter(q, M, 1 + j));
        __syncwarp();
        store_pe(actA, wj, lane);
        __syncwarp();
        zero(acc);
        warp_gemm<kPEPad>(actA, sw + OFF_IW1P, acc, rg, cg);
        store_relu_tilebias(actB, acc, a2b, rg, cg);
        __syncwarp();
        zero(acc);
        warp_gemm<kHidden>(actB, sw + OFF_IW2, acc, rg, cg);
        store_relu_colbias(actA, acc, sw + OFF_IB2, rg, cg);
        __syncwarp();
        const float z0 = irt_head(actA, sw, lane).x;
        const float v2 = visibility_from_logit(z0, m.force_vis2, m.hard);
        const f3 le = env_lookup(m.env, m.env_h, m.env_w, wj);
        const f3 fr = brdf_eval(a2, r2, n2, wj, wo2, m.f0, m.lambert);
        lo2 = lo2 + (le * fr) * v2;
      }
      lo2 = lo2 * (kPi / (float)M);

      // Eq. 2 then the primary term of Eq. 1
      const f3 li = env_lookup(m.env, m.env_h, m.env_w, wi) * v + lo2 * (1.0f - v);
      const f3 c = li * (m.mis ? mis_weighted_brdf(m, alb, ar.w, n, wo, wi)
                               : brdf_eval(alb, ar.w, n, wi, wo, m.f0, m.lambert));
      if (i < N) sum = sum + c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
      sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
      sum.z += __shfl_xor_sync(0xffffffffu, sum.z, o);
    }
    if (lane == 0) {
      const float sc = kPi / (float)N;
      out[pix] = make_float4(sum.x * sc, sum.y * sc, sum.z * sc, 0.0f);
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t prepare_render_fp32() {
  return cudaFuncSetAttribute(render_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

cudaError_t launch_render_fp32(const ModelDesc& m, const rt_gbuffer& gb, int P, long long offset, float4* out,
                               int num_sms, cudaStream_t s) {
  const int need = (P + kWarps - 1) / kWarps;
  const int grid = need < num_sms ? need : num_sms;
  render_fp32_kernel<<<grid, kThreads, kSmemBytes, s>>>(m, gb, P, offset, out);
  return cudaGetLastError();
}

}  // namespace rtk
