// tcgen05 building blocks shared by the BF16 tensor-core kernels (the fused
// render and its adjoint): instruction and shared-memory descriptors, MMA
// issue and commit, tensor-memory loads and stores, bf16 packing, the MLP
// layer chains and epilogues of the forward, and the hash encodes that write
// their features straight into a tile's A operand.
//
// Conventions: a warpgroup owns 128 TMEM lanes (thread t of the warpgroup =
// lane t = row t of the tile).  Column c of an A operand in TMEM holds the
// bf16 pair (2c, 2c + 1) of the row.  Weight tiles in shared memory are
// K-major with the 128-byte swizzle (element (n, k) at swz128(n, k)).
#pragma once

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "fast_math.cuh"

namespace rtk {

constexpr int kPixSlots = 34;                // pixels touched by one 128-row tile when N >= 4
constexpr int kFpixLo = kPixSlots * 64;      // offset of the lo parts in a tile's primary-feature slots

constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdescN64 = idesc_bf16(128, 64);

// K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// K-major, 32-byte swizzle, 8-row groups 256 bytes apart (the K = 16 bias tiles).
__device__ __forceinline__ uint64_t sdesc32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// The same with the A operand in tensor memory (rows in lanes, K-major bf16 pairs).
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warpgroup barrier (named barrier 1 + wg) that also ORs a flag across the group.
__device__ __forceinline__ int wg_sync_or(int wg, int v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.or.pred q, %2, 128, p;\n"
      " selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v), "r"(wg + 1)
      : "memory");
  return r;
}
__device__ __forceinline__ void wg_sync(int wg) { asm volatile("bar.sync %0, 128;" ::"r"(wg + 1) : "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// The two bf16 halves of a packed pair as floats (element 2c in the low half).
__device__ __forceinline__ float bf16_lo_half(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi_half(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }
// The bf16 pair of the rounding residuals (a - bf16(a), b - bf16(b)) of a packed pair hi = bf16x2(a, b).
__device__ __forceinline__ uint32_t pack_residual(float a, float b, uint32_t hi) {
  return pack_bf16(a - bf16_lo_half(hi), b - bf16_hi_half(hi));
}

// D <- X . W1^T (k-steps 0..3 of the layer-1 input in TMEM)
__device__ __forceinline__ void mma_layer1(uint32_t d, uint32_t x_t, uint32_t w_s) {
#pragma unroll
  for (int k = 0; k < 4; ++k) mma_bf16_ts(d, x_t + 8 * k, sdesc(w_s + 32 * k), kIdescN64, k > 0 ? 1u : 0u);
}
// layer 2: D <- H . W2^T + ones . Bias2^T
__device__ __forceinline__ void mma_layer2(uint32_t d, uint32_t h_t, uint32_t w_s, uint32_t ones_s, uint32_t bias_s) {
#pragma unroll
  for (int k = 0; k < 4; ++k) mma_bf16_ts(d, h_t + 8 * k, sdesc(w_s + 32 * k), kIdescN64, k > 0 ? 1u : 0u);
  mma_bf16(d, sdesc32(ones_s), sdesc32(bias_s), kIdescN64, 1u);
}
// B's layer 1: f' (k-steps 0, 1) and the bias columns (k-step 3; B's weights are zero on the PE columns)
__device__ __forceinline__ void mma_brdf_layer1(uint32_t d, uint32_t x_t, uint32_t w_s) {
  mma_bf16_ts(d, x_t, sdesc(w_s), kIdescN64, 0u);
  mma_bf16_ts(d, x_t + 8, sdesc(w_s + 32), kIdescN64, 1u);
  mma_bf16_ts(d, x_t + 24, sdesc(w_s + 96), kIdescN64, 1u);
}

// The primary evaluation of I in split precision.  Every operand is a bf16
// hi part plus a bf16 lo part (its rounding residual): A = Ah + Al, W = Wh +
// Wl, and A W ~ Ah Wh + Al Wh + Ah Wl in FP32, which carries about 16
// significant bits instead of bf16's 8.  The lo operands take the H columns
// during layer 1 (and X / H hold the hi / lo parts of the hidden layer during
// layer 2), so the warpgroup's 128 TMEM columns suffice.
// Layer 1: D <- Xh W1h + Xl W1h + Xh W1l (the bias rides on Xh's ones columns).
__device__ __forceinline__ void mma_layer1_split(uint32_t d, uint32_t xh_t, uint32_t xl_t, uint32_t w_s,
                                                 uint32_t wl_s) {
#pragma unroll
  for (int k = 0; k < 4; ++k) mma_bf16_ts(d, xh_t + 8 * k, sdesc(w_s + 32 * k), kIdescN64, k > 0 ? 1u : 0u);
#pragma unroll
  for (int k = 0; k < 4; ++k) mma_bf16_ts(d, xl_t + 8 * k, sdesc(w_s + 32 * k), kIdescN64, 1u);
#pragma unroll
  for (int k = 0; k < 4; ++k) mma_bf16_ts(d, xh_t + 8 * k, sdesc(wl_s + 32 * k), kIdescN64, 1u);
}
// Layer 2: D <- Hh W2h + Hl W2h + Hh W2l + ones . Bias2
__device__ __forceinline__ void mma_layer2_split(uint32_t d, uint32_t hh_t, uint32_t hl_t, uint32_t w_s,
                                                 uint32_t wl_s, uint32_t ones_s, uint32_t bias_s) {
  mma_layer1_split(d, hh_t, hl_t, w_s, wl_s);
  mma_bf16(d, sdesc32(ones_s), sdesc32(bias_s), kIdescN64, 1u);
}
// Split hidden epilogue: Hh = bf16(relu(D)), Hl = bf16(relu(D) - Hh), 16 columns at a time.
__device__ __forceinline__ void epilogue_hidden_split(uint32_t d_taddr, uint32_t hh_taddr, uint32_t hl_taddr) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t r[16];
    tmem_ld16(d_taddr + 16 * q, r);
    tmem_ld_wait();
    uint32_t qh[8], ql[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float a = fmaxf(__uint_as_float(r[2 * e]), 0.0f), b = fmaxf(__uint_as_float(r[2 * e + 1]), 0.0f);
      qh[e] = pack_bf16(a, b);
      ql[e] = pack_residual(a, b, qh[e]);
    }
    tmem_st8(hh_taddr + 8 * q, qh);
    tmem_st8(hl_taddr + 8 * q, ql);
  }
}

// hidden epilogue: H[row] = bf16(relu(D[row][0:64])) (the bias is already in D)
__device__ __forceinline__ void epilogue_hidden(uint32_t d_taddr, uint32_t h_taddr) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t r[32];
    tmem_ld32(d_taddr + 32 * h, r);
    tmem_ld_wait();
    uint32_t q[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) q[e] = pack_relu_bf16(__uint_as_float(r[2 * e]), __uint_as_float(r[2 * e + 1]));
    tmem_st16(h_taddr + 16 * h, q);
  }
}

// Output layer in FP32 with packed FMAs: z[o] = b3[o] + sum_k relu(D[row][k]) W3[k][o]
template <int NOUT, int LDW>
__device__ __forceinline__ void head_fp32(uint32_t taddr, const float* W3, const float* b3, float (&z)[NOUT]) {
  constexpr int NP = (NOUT + 1) / 2;
  float2 acc[NP];
#pragma unroll
  for (int o = 0; o < NP; ++o) acc[o] = make_float2(b3[2 * o], 2 * o + 1 < NOUT ? b3[2 * o + 1] : 0.0f);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t r[32];
    tmem_ld32(taddr + 32 * h, r);
    tmem_ld_wait();
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float a = fmaxf(__uint_as_float(r[k]), 0.0f);
      const float2 aa = make_float2(a, a);
#pragma unroll
      for (int o = 0; o < NP; ++o)
        acc[o] = __ffma2_rn(aa, *reinterpret_cast<const float2*>(&W3[(32 * h + k) * LDW + 2 * o]), acc[o]);
    }
  }
#pragma unroll
  for (int o = 0; o < NOUT; ++o) z[o] = (o & 1) ? acc[o / 2].y : acc[o / 2].x;
}

// One output (I's visibility logit): pairs of hidden units per packed FMA.
__device__ __forceinline__ float head_vis(uint32_t taddr, const float* w, float b) {
  float2 acc = make_float2(b, 0.0f);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t r[32];
    tmem_ld32(taddr + 32 * h, r);
    tmem_ld_wait();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 a = make_float2(fmaxf(__uint_as_float(r[2 * k]), 0.0f), fmaxf(__uint_as_float(r[2 * k + 1]), 0.0f));
      acc = __ffma2_rn(a, *reinterpret_cast<const float2*>(&w[32 * h + 2 * k]), acc);
    }
  }
  return acc.x + acc.y;
}


// f' = H(x') as 16 bf16 pairs written to X columns 0..15 (zero beyond L
// levels), from an FP16 table.  The loop over groups of four levels stays
// rolled (the unrolled sixteen levels cost more in instruction fetch than
// they save); within a group each level's gathers are issued and consumed
// before the next level's: more gathers in flight per thread only add L1
// pressure (two levels at a time measured 3 % slower, four 8 % slower).  The
// two x-neighbour corners of a cell share one 8-byte load when their rows
// form an aligned pair (rows r and r ^ 1: a hashed level with even i, or a
// dense level with an even row), which removes about a quarter of the
// gathers.  (Aligned 16-byte loads, which pair the corners three times in
// four, measured 5 % slower.)
// With JAC, also the interpolation's derivative along each axis, per level: for
// features (f0, f1) of level l, d f / d w_a (w_a the cell fraction on axis a),
// halved and stored as a half2 in jac[(3 l + a) * 128 + row] (column-major over
// the tile's 128 rows; halved so that it always fits half precision when the
// table is FP16).  The adjoint's dLoss/dx' then needs no second gather.
template <bool JAC = false>
__device__ __forceinline__ void encode_point_tmem(const GridDesc& g, f3 x, uint32_t x_taddr, uint32_t* jac = nullptr,
                                                  int row = 0) {
#pragma unroll 1
  for (int it = 0; it < kMaxLevels / 4; ++it) {
    uint32_t fq[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int l = 4 * it + b;
      float f0 = 0.f, f1 = 0.f;
      if (l < g.levels) {
        const int res = g.res[l];
        uint32_t ix, iy, iz;
        float w[3];
        grid_cell(x.x, res, ix, w[0]);
        grid_cell(x.y, res, iy, w[1]);
        grid_cell(x.z, res, iz, w[2]);
        const uint32_t* tab = reinterpret_cast<const uint32_t*>(g.table) + ((size_t)l << g.log2T);
        const int dn = g.dense[l];
        uint32_t v[8];
#pragma unroll
        for (int yz = 0; yz < 4; ++yz) {
          const uint32_t r0 = corner_row(ix, iy + (yz & 1), iz + (yz >> 1), res, dn, g.mask);
          const uint32_t r1 = corner_row(ix + 1, iy + (yz & 1), iz + (yz >> 1), res, dn, g.mask);
          const uint2 pr = __ldg(reinterpret_cast<const uint2*>(tab + (r0 & ~1u)));
          const bool odd = r0 & 1u;
          v[2 * yz] = odd ? pr.y : pr.x;
          v[2 * yz + 1] = ((r0 ^ r1) == 1u) ? (odd ? pr.x : pr.y) : __ldg(tab + r1);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          // v[2*yz + dx] holds corner (dx, yz & 1, yz >> 1)
          const int dx = c & 1, yz = c >> 1;
          const float wt = (dx ? w[0] : 1.0f - w[0]) * ((yz & 1) ? w[1] : 1.0f - w[1]) *
                           ((yz & 2) ? w[2] : 1.0f - w[2]);
          const float2 e = __half22float2(*reinterpret_cast<const __half2*>(&v[c]));
          f0 = fmaf(wt, e.x, f0);
          f1 = fmaf(wt, e.y, f1);
        }
        if constexpr (JAC) {
          float2 j[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;   // corner c = v[c] (x fastest)
            const float2 e = __half22float2(*reinterpret_cast<const __half2*>(&v[c]));
            const float ax = cx ? w[0] : 1.0f - w[0], ay = cy ? w[1] : 1.0f - w[1], az = cz ? w[2] : 1.0f - w[2];
            const float gx = (cx ? 0.5f : -0.5f) * ay * az, gy = (cy ? 0.5f : -0.5f) * ax * az,
                        gz = (cz ? 0.5f : -0.5f) * ax * ay;
            j[0] = make_float2(fmaf(gx, e.x, j[0].x), fmaf(gx, e.y, j[0].y));
            j[1] = make_float2(fmaf(gy, e.x, j[1].x), fmaf(gy, e.y, j[1].y));
            j[2] = make_float2(fmaf(gz, e.x, j[2].x), fmaf(gz, e.y, j[2].y));
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const __half2 h = __floats2half2_rn(j[a].x, j[a].y);
            jac[(3 * l + a) * 128 + row] = *reinterpret_cast<const uint32_t*>(&h);
          }
        }
      }
      fq[b] = pack_bf16(f0, f1);
    }
    tmem_st4(x_taddr + 4 * it, fq[0], fq[1], fq[2], fq[3]);
  }
}

// PE(w) as bf16 into X columns 16..31: 27 values, then the two 1.0 columns
// that carry layer 1's bias, then zeros
__device__ __forceinline__ void store_pe_tmem(uint32_t x_taddr, f3 w) {
  float pe[32];
  positional_encoding_fast(w, [&](int k, float v) { pe[k] = v; });
#pragma unroll
  for (int k = kPE; k < 32; ++k) pe[k] = (k == kBiasCol - 32 || k == kBiasCol - 31) ? 1.0f : 0.0f;
  uint32_t q[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) q[e] = pack_bf16(pe[2 * e], pe[2 * e + 1]);
  tmem_st16(x_taddr + 16, q);
}

// X columns 24..31 (elements 48..63) as B's layer 1 reads them: zero but for
// the two 1.0 columns that carry its bias.  The split primary evaluation of I
// leaves the hidden layer's hi parts there, so this is rewritten before B.
__device__ __forceinline__ void store_bias_cols_tmem(uint32_t x_taddr) {
  uint32_t q[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = 48 + 2 * e;   // elements k, k + 1 of the layer-1 input
    q[e] = pack_bf16((k == kBiasCol || k == kBiasCol + 1) ? 1.0f : 0.0f,
                     (k + 1 == kBiasCol || k + 1 == kBiasCol + 1) ? 1.0f : 0.0f);
  }
  tmem_st8(x_taddr + 24, q);
}

// The split layer-1 input of the primary evaluation of I: [f | PE(w) | 1 | 1 | 0]
// as bf16 hi parts into X (xh_taddr) and lo parts into H (xl_taddr).  f's hi
// and lo parts come from the tile's feature slots; PE(w) is split here (the
// ones and zeros have no residual).
__device__ __forceinline__ void store_primary_split(const uint8_t* fpix, int slot, uint32_t xh_taddr,
                                                    uint32_t xl_taddr, f3 w) {
#pragma unroll
  for (int part = 0; part < 2; ++part) {
    const uint4* src = reinterpret_cast<const uint4*>(fpix + part * kFpixLo + slot * 64);
    uint32_t fr[16];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 v = src[c];
      fr[4 * c] = v.x;
      fr[4 * c + 1] = v.y;
      fr[4 * c + 2] = v.z;
      fr[4 * c + 3] = v.w;
    }
    tmem_st16(part ? xl_taddr : xh_taddr, fr);
  }
  float pe[32];
  positional_encoding_fast(w, [&](int k, float v) { pe[k] = v; });
#pragma unroll
  for (int k = kPE; k < 32; ++k) pe[k] = (k == kBiasCol - 32 || k == kBiasCol - 31) ? 1.0f : 0.0f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t qh[8], ql[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float a = pe[16 * h + 2 * e], b = pe[16 * h + 2 * e + 1];
      qh[e] = pack_bf16(a, b);
      ql[e] = pack_residual(a, b, qh[e]);
    }
    tmem_st8(xh_taddr + 16 + 8 * h, qh);
    tmem_st8(xl_taddr + 16 + 8 * h, ql);
  }
}

// (a) f = H(x) of a tile's npix pixels into fpix [npix][32] bf16, 32
// threads per pixel (two per level, four corners each), four pixels per pass.
__device__ __forceinline__ void gather_primary_features(const GridDesc& g, const float4* __restrict__ pos4,
                                                        long long p_first, int npix, int warp, int lane,
                                                        uint8_t* fpix) {
  for (int s0 = 0; s0 < npix; s0 += 4) {
    const int slot = s0 + warp;
    float2 part = make_float2(0.f, 0.f);
    const int l = lane >> 1;
    if (slot < npix && l < g.levels) {
      const f3 xs = xyz(pos4[p_first + slot]);
      const int res = g.res[l];
      uint32_t ix, iy, iz;
      float wx, wy, wz;
      grid_cell_exact(xs.x, res, ix, wx);   // f feeds the split-precision primary evaluation of I
      grid_cell_exact(xs.y, res, iy, wy);
      grid_cell_exact(xs.z, res, iz, wz);
      const size_t base = (size_t)l << g.log2T;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = (lane & 1) * 4 + cc;
        const uint32_t row = corner_row(ix + (c & 1), iy + ((c >> 1) & 1), iz + ((c >> 2) & 1), res, g.dense[l],
                                        g.mask);
        const float w = ((c & 1) ? wx : 1.0f - wx) * ((c & 2) ? wy : 1.0f - wy) * ((c & 4) ? wz : 1.0f - wz);
        const float2 v = table_entry(g, base + row);
        part.x = fmaf(w, v.x, part.x);
        part.y = fmaf(w, v.y, part.y);
      }
    }
    part.x += __shfl_xor_sync(0xffffffffu, part.x, 1);
    part.y += __shfl_xor_sync(0xffffffffu, part.y, 1);
    if (slot < npix && (lane & 1) == 0) {
      // hi parts for every use of f, lo parts (rounding residuals) for the split primary evaluation of I
      const uint32_t hi = pack_bf16(part.x, part.y);
      *reinterpret_cast<uint32_t*>(fpix + slot * 64 + 2 * lane) = hi;
      *reinterpret_cast<uint32_t*>(fpix + kFpixLo + slot * 64 + 2 * lane) = pack_residual(part.x, part.y, hi);
    }
  }
}


}  // namespace rtk
