// Fused BF16 tensor-core hot path: stages (a)-(e) of the hash renderer in one
// persistent kernel (rt_render_frame with precision RT_BF16).
//
// Layout of the work.  A CTA holds WG independent warpgroups.  Each
// warpgroup owns a contiguous range of primary points and walks its
// secondary samples (point p, direction i) in tiles of 128 consecutive
// samples: thread t of the warpgroup owns row t of the tile, which is also
// TMEM lane t of the warpgroup's columns.  Every 64-wide MLP layer of the
// tile is one chain of tcgen05.mma (M = 128, N = 64, K = 16 per instruction)
// issued by one thread.  The A operand (the layer input, bf16) lives in
// tensor memory next to the FP32 accumulator: threads write their rows with
// tcgen05.st and the MMA reads them from TMEM, so activations never pass
// through shared memory; the B operand (weights, bf16) sits in 128-byte-
// swizzled shared memory, loaded once per CTA.  Layer biases ride on the
// MMAs (a ones column in the layer-1 input, a ones tile times a bias tile
// for layer 2), so the epilogue only applies ReLU, rounds to bf16 and
// writes the next A operand.  Hash interpolation, depth, shading and all
// sums stay in FP32; the table is read as FP16.
//
// Per tile: I on [f, PE(w_i)], the bounce and f' = H(x'), B on f', then for
// each of the M secondary directions I on [f', PE(w'_j)] with f' kept in the
// A operand, then Eq. 1 / Eq. 2 and a deterministic segmented reduction of
// the rows into their pixels.  The narrow output layer (2 or 7 outputs)
// runs in FP32 on the CUDA cores straight from the FP32 layer-2
// accumulator, which saves a round trip per MLP and keeps t and n' free of
// one bf16 rounding.
//
// Every wait on an mbarrier is bounded (2 s of %globaltimer); on expiry the
// warpgroup records kStatusTimeout in the status word and stops.
#include <cuda_bf16.h>

#include "device_common.cuh"
#include "fast_math.cuh"
#include "mbarrier.cuh"
#include "mis.cuh"

namespace rtk {

// ---- BF16 weight image (runs after the FP32 repack on the same stream) -----
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// I's layer-1 weight of output n and input column k of the A tile [f | PE | 1 | 1 | 0]
// (the bias columns excluded), from the FP32 image.
__device__ __forceinline__ float irt_w1(const float* __restrict__ wp, int n, int k) {
  if (k < 32) return wp[OFF_IW1F + k * 64 + n];
  if (k < kBiasCol) return wp[OFF_IW1P + (k - 32) * 64 + n];
  return 0.0f;
}

// One thread per bf16 element of the image.
__global__ void repack_bf16_kernel(const float* __restrict__ wp, uint8_t* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= WBF16_BYTES / 2) return;
  const int byte = 2 * e;
  __nv_bfloat16 v = __float2bfloat16_rn(0.0f);
  if (byte < OFFB_IB2 || byte >= OFFB_IW1L) {
    // one of the six 64 x 64 swizzled matrices: invert swz128
    const int tile = byte < OFFB_IB2 ? byte / 8192 : 4 + (byte - OFFB_IW1L) / 8192;
    const int o = byte % 8192;
    const int n = (o / 1024) * 8 + (o % 1024) / 128;
    const int chunk = ((o % 128) / 16) ^ (n & 7);
    const int k = chunk * 8 + (o % 16) / 2;
    float f = 0.0f;
    if (tile == 0 || tile == 4) {                       // I layer 1: [f | PE | 1 | 1 | 0]
      f = irt_w1(wp, n, k);
    } else if (tile == 1 || tile == 5) {
      f = wp[OFF_IW2 + k * 64 + n];
    } else if (tile == 2) {                             // B layer 1: [f | 0 | b1]
      if (k < 32) f = wp[OFF_BW1 + k * 64 + n];
    } else {
      f = wp[OFF_BW2 + k * 64 + n];
    }
    v = __float2bfloat16_rn(f);
    if (tile >= 4) {                                    // the rounding residual of the hi tile
      __nv_bfloat16 hi, lo;
      split_bf16(f, hi, lo);
      v = lo;
    }
    if (tile == 0 || tile == 2) {
      const float b = tile == 0 ? wp[OFF_IB1 + n] : wp[OFF_BB1 + n];
      __nv_bfloat16 hi, lo;
      split_bf16(b, hi, lo);
      if (k == kBiasCol) v = hi;
      if (k == kBiasCol + 1) v = lo;
    }
  } else if (byte < OFFB_ONES) {
    // layer-2 bias tiles: row n = 8 x hi/8, 8 x lo/8 (exact scalings by 1/8)
    const int tile = (byte - OFFB_IB2) / 2048, o = (byte - OFFB_IB2) % 2048;
    const int n = o / 32, k = (o % 32) / 2;
    const float b = tile == 0 ? wp[OFF_IB2 + n] : wp[OFF_BB2 + n];
    __nv_bfloat16 hi, lo;
    split_bf16(b, hi, lo);
    v = __float2bfloat16_rn(0.125f * __bfloat162float(k < 8 ? hi : lo));
  } else {
    v = __float2bfloat16_rn(1.0f);                      // the all-ones tile
  }
  *reinterpret_cast<__nv_bfloat16*>(out + byte) = v;
}

cudaError_t launch_repack_bf16(const float* wpack, uint8_t* wbf16, cudaStream_t s) {
  repack_bf16_kernel<<<(WBF16_BYTES / 2 + 255) / 256, 256, 0, s>>>(wpack, wbf16);
  return cudaGetLastError();
}

namespace {

// Kernel variants: NL lights per launch (1, 2, 4, 8) and WG warpgroups per
// CTA: 2 (two CTAs per SM) or 3 and 4 (one CTA per SM, one shared copy of the
// weights).  Shared memory holds only the weights and a small block per
// warpgroup, and the carveout is kept to that, so most of the SM's 256 KB
// serves as L1 for the environment maps and the coarse hash levels.
//
// TMEM columns of a warpgroup (128 from column 128 * wg):
//   D [0, 64)    FP32 accumulator, shared by layer 1 and layer 2
//   X [64, 96)   layer-1 input: [f or f' (32 bf16) | PE(w) (27) | 1 | 1 | 0 ...]
//   H [96, 128)  layer-2 input: bf16(ReLU(layer 1))
// Column c of X or H holds the bf16 pair (2c, 2c + 1) of the row.
constexpr int TM_D = 0, TM_X = 64, TM_H = 96;
constexpr int kPixSlots = 34;                // pixels touched by one tile when N >= 4
// shared-memory layout (offsets from a 1024-aligned base)
constexpr int SM_W = 0;
constexpr int WG_FPIX = 0;                   // primary features, bf16 hi parts [34][32]; reused as red[128] float4
constexpr int WG_FPIX_LO = kPixSlots * 64;   // their bf16 lo parts [34][32]
constexpr int WG_MISC = 2 * kPixSlots * 64;  // mbarrier (8), then carry[NL] float4 from +16
constexpr int WG_BYTES = WG_MISC + 256;
// hard visibility: a ring of 256 queued shadow rows, the row keys of a tile and per-warp counts
constexpr int WG_QA = WG_BYTES;              // float4 (w_i, t) [256]
constexpr int WG_QB = WG_QA + 256 * 16;      // int2 (pixel, i) [256]
constexpr int WG_KEYS = WG_QB + 256 * 8;     // int [128]
constexpr int WG_CNT = WG_KEYS + 128 * 4;    // int [4]
constexpr int WG_BYTES_HARD = WG_CNT + 128;
constexpr int SM_WG = WBF16_BYTES;
static_assert(WG_MISC + 16 + 8 * 16 <= WG_BYTES, "warpgroup block overflow");
static_assert(WG_CNT + 16 <= WG_BYTES_HARD, "warpgroup block overflow (hard visibility)");
static_assert(128 * 16 <= 2 * kPixSlots * 64 && WG_MISC % 16 == 0 && WG_BYTES_HARD % 16 == 0, "pixel slots");

template <int WG, bool HARD = false>
struct Layout {
  static constexpr int kThreads = 128 * WG;
  static constexpr int kTmemCols = WG <= 2 ? 128 * WG : 512;   // allocations are powers of two
  static constexpr int kWgBytes = HARD ? WG_BYTES_HARD : WG_BYTES;
  static constexpr int kTmemSlot = SM_WG + WG * kWgBytes;
  static constexpr size_t kSmem = kTmemSlot + 16 + 1024;
  static constexpr int kMinBlocks = WG <= 2 ? 2 : 1;
  // smallest carveout (percent of the 228 KB maximum) that holds kMinBlocks CTAs
  static constexpr int kCarveout = (int)((kMinBlocks * (kSmem + 1024) * 100 + 233471) / 233472);
};

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
__device__ __forceinline__ void encode_point_tmem(const GridDesc& g, f3 x, uint32_t x_taddr) {
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
    const uint4* src = reinterpret_cast<const uint4*>(fpix + part * WG_FPIX_LO + slot * 64);
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
      *reinterpret_cast<uint32_t*>(fpix + WG_FPIX_LO + slot * 64 + 2 * lane) = pack_residual(part.x, part.y, hi);
    }
  }
}

template <int NL, int WG, bool HARD>
__global__ void __launch_bounds__(Layout<WG, HARD>::kThreads, Layout<WG, HARD>::kMinBlocks)
render_bf16_kernel(const __grid_constant__ ModelDesc m, const __grid_constant__ HeadParams hp, rt_gbuffer gb, int P,
                   long long pixel_offset, const float4* __restrict__ envs, float4* __restrict__ out) {
  using L = Layout<WG, HARD>;
  constexpr int kThreadsB = L::kThreads;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int wg = tid >> 7, t = tid & 127, warp = t >> 5, lane = t & 31;
  uint8_t* Wsm = sm + SM_W;
  uint8_t* wgb = sm + SM_WG + wg * L::kWgBytes;
  uint8_t* fpix = wgb + WG_FPIX;
  float4* red = reinterpret_cast<float4*>(wgb + WG_FPIX);
  uint64_t* bar = reinterpret_cast<uint64_t*>(wgb + WG_MISC);
  float4* carry_s = reinterpret_cast<float4*>(wgb + WG_MISC + 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::kTmemSlot);

  // ---- CTA set-up: weights into shared memory, TMEM, barriers
  for (int i = tid; i < WBF16_BYTES / 16; i += kThreadsB)
    reinterpret_cast<uint4*>(Wsm)[i] = __ldg(reinterpret_cast<const uint4*>(m.wbf16) + i);
  if (t == 0) {
    mbar_init(smem_u32(bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();   // the weight tiles are read by the async proxy
  if (warp == 0 && wg == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(L::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + (uint32_t)(128 * wg);
  const uint32_t D_t = tmem + TM_D, X_t = tmem + TM_X, H_t = tmem + TM_H;   // MMA operands (lane 0)
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;                    // this warp's 32 lanes
  const uint32_t D_w = D_t + lane_off, X_w = X_t + lane_off, H_w = H_t + lane_off;
  const uint32_t bar_a = smem_u32(bar);
  const uint32_t W_s = smem_u32(Wsm);

  const int N = m.N, M = m.M;
  const int env_hw = m.env_h * m.env_w;
  const float4* pos4 = reinterpret_cast<const float4*>(gb.pos);
  const float4* nrm4 = reinterpret_cast<const float4*>(gb.normal);
  const float4* view4 = reinterpret_cast<const float4*>(gb.view);
  const float4* ar4 = reinterpret_cast<const float4*>(gb.albedo_rough);

  const long long workers = (long long)gridDim.x * WG;
  const long long worker = (long long)blockIdx.x * WG + wg;
  const long long p0 = (long long)P * worker / workers, p1 = (long long)P * (worker + 1) / workers;
  const long long s_end = p1 * N;
  uint32_t phase = 0;
  int abort = 0;
  if (t < NL) carry_s[t] = make_float4(0.f, 0.f, 0.f, 0.f);

  // One MMA round trip: barrier with an abort vote, issue by thread 0,
  // commit, bounded wait.  A wait that gives up only raises `abort`; the
  // vote at the next round trip then stops all 128 threads together, so the
  // warpgroup never splits across barriers.
  uint32_t pending_phase = 0;
  auto run_mma = [&](auto issue) -> bool {
    tmem_st_wait();   // this thread's rows of the A operand have landed in TMEM
    tc_fence_before();
    abort = wg_sync_or(wg, abort);
    if (abort) return false;
    if (t == 0) {
      tc_fence_after();
      issue();
      mma_commit(bar_a);
    }
    if (!mbar_wait(bar_a, phase)) {
      if (!abort && t == 0) atomicOr(m.status, kStatusTimeout | 1u);
      abort = 1;
      pending_phase = phase;
    }
    phase ^= 1u;
    tc_fence_after();
    return true;
  };

  if constexpr (HARD) {
    // Hard visibility (Sec. 3.2 overview): a primary tile adds the direct term
    // of its visible rows and queues its shadow rows (w_i, t, pixel, i) in a
    // ring in shared memory; every 128 queued rows make one secondary tile
    // (x' encode, B, the M secondary I evaluations, Eq. 1 at x').  Pixel sums
    // are added into `out` by one thread per pixel and tile, in program
    // order, and scaled by pi/N at the end; the warpgroup owns its pixels.
    float4* qa = reinterpret_cast<float4*>(wgb + WG_QA);
    int2* qb = reinterpret_cast<int2*>(wgb + WG_QB);
    int* keys = reinterpret_cast<int*>(wgb + WG_KEYS);
    int* wcnt = reinterpret_cast<int*>(wgb + WG_CNT);
    for (long long p = p0 + t; p < p1; p += 128)
#pragma unroll
      for (int e = 0; e < NL; ++e) __stcg(out + (long long)e * P + p, make_float4(0.f, 0.f, 0.f, 0.f));
    uint32_t qhead = 0, qtail = 0;
    bool ok = true;

    // out[e][key] += sum of c[e] over the rows with that key; rows come in key
    // order, key < 0 marks an idle row.  One thread per key does the update.
    auto add_rows = [&](int key, const f3 (&c)[NL]) {
      const int prev = __shfl_up_sync(0xffffffffu, key, 1);
      const bool head = lane == 0 || prev != key;
      wg_sync(wg);   // earlier readers of keys / red are done; the zeroing above is ordered
      keys[t] = key;
#pragma unroll
      for (int e = 0; e < NL; ++e) {
        f3 ce = key >= 0 ? c[e] : mk(0.f, 0.f, 0.f);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float ox = __shfl_down_sync(0xffffffffu, ce.x, off);
          const float oy = __shfl_down_sync(0xffffffffu, ce.y, off);
          const float oz = __shfl_down_sync(0xffffffffu, ce.z, off);
          const int k2 = __shfl_down_sync(0xffffffffu, key, off);
          if (lane + off < 32 && k2 == key) ce = mk(ce.x + ox, ce.y + oy, ce.z + oz);
        }
        if (e > 0) wg_sync(wg);   // the previous light's sums are read
        red[t] = head ? make_float4(ce.x, ce.y, ce.z, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        wg_sync(wg);
        if (key >= 0 && (t == 0 || keys[t - 1] != key)) {
          float4 sum = red[t];
          for (int r = ((t >> 5) + 1) << 5; r < 128 && keys[r] == key; r += 32) {
            const float4 h = red[r];
            sum = make_float4(sum.x + h.x, sum.y + h.y, sum.z + h.z, 0.f);
          }
          float4* o = out + (long long)e * P + key;
          const float4 cur = __ldcg(o);
          __stcg(o, make_float4(cur.x + sum.x, cur.y + sum.y, cur.z + sum.z, 0.f));
        }
      }
      wg_sync(wg);   // red (the primary-feature area) and keys are free again
    };

    // One secondary tile over the queued rows [qhead, qhead + nvalid).
    auto secondary = [&](int nvalid) -> bool {
      const bool valid = t < nvalid;
      const uint32_t slot = (qhead + (uint32_t)(valid ? t : 0)) & 255u;
      const float4 qw = qa[slot];
      const int2 pi = qb[slot];
      const long long p = pi.x;
      const f3 wi = mk(qw.x, qw.y, qw.z);
      const f3 x = xyz(pos4[p]);
      const f3 n = xyz(nrm4[p]);
      const f3 wo = xyz(view4[p]);
      const float4 ar = ar4[p];
      const uint64_t q = (uint64_t)(pixel_offset + p) * (uint64_t)N + (uint64_t)pi.y;
      // MIS: the direction's Eq. 1 weight relative to cosine sampling rides on fr1
      const f3 fr1 = m.mis ? mis_weighted_brdf(m, xyz(ar), ar.w, n, wo, wi)
                           : brdf_eval_fast(xyz(ar), ar.w, n, wi, wo, m.f0, m.lambert);
      // (d) x' = x + t w_i and f' = H(x'); (b) B(f')
      encode_point_tmem(m.grid, x + wi * qw.w, X_w);
      store_bias_cols_tmem(X_w);
      if (!run_mma([&] { mma_brdf_layer1(D_t, X_t, W_s + OFFB_BW1); })) return false;
      epilogue_hidden(D_w, H_w);
      if (!run_mma([&] { mma_layer2(D_t, H_t, W_s + OFFB_BW2, W_s + OFFB_ONES, W_s + OFFB_BB2); })) return false;
      f3 n2, a2;
      float r2;
      {
        float y[7];
        head_fp32<7, 8>(D_w, &hp.bw3[0][0], hp.bb3, y);
        const float ninv = rsqrtf(fmaxf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2], 1e-24f));
        n2 = mk(y[0] * ninv, y[1] * ninv, y[2] * ninv);
        a2 = mk(sigmoid_fast(y[3]), sigmoid_fast(y[4]), sigmoid_fast(y[5]));
        r2 = 0.09f + 0.91f * sigmoid_fast(y[6]);
      }
      const f3 wo2 = neg(wi);
      const float wsec = kPi / (float)M;   // a shadow row: 1 - v = 1
      f3 c[NL];
#pragma unroll
      for (int e = 0; e < NL; ++e) c[e] = mk(0.f, 0.f, 0.f);
      // (c) + (e) at x': only visible secondary directions count
      for (int j = 0; j < M; ++j) {
        const f3 wj = cosine_direction_fast(n2, m.seed, dir_counter(q, M, 1 + j));
        const EnvTap tapj = env_tap_fast(m.env_h, m.env_w, wj);
        const f3 frw = fr1 * brdf_eval_fast(a2, r2, n2, wj, wo2, m.f0, m.lambert);
        f3 lej = mk(0.f, 0.f, 0.f);
        if (NL == 1) lej = env_fetch(envs, tapj);
        store_pe_tmem(X_w, wj);
        if (!run_mma([&] { mma_layer1(D_t, X_t, W_s + OFFB_IW1); })) return false;
        epilogue_hidden(D_w, H_w);
        if (!run_mma([&] { mma_layer2(D_t, H_t, W_s + OFFB_IW2, W_s + OFFB_ONES, W_s + OFFB_IB2); })) return false;
        const float v2 = visibility_from_logit(head_vis(D_w, hp.iw3v, hp.ib3[0]), m.force_vis2, 1);
        const f3 wj3 = frw * (wsec * v2);
        if (NL == 1) {
          c[0] = c[0] + wj3 * lej;
        } else {
#pragma unroll
          for (int e = 0; e < NL; ++e) c[e] = c[e] + wj3 * env_fetch(envs + e * env_hw, tapj);
        }
      }
      add_rows(valid ? (int)p : -1, c);
      return true;
    };

    for (long long sbase = p0 * N; ok && sbase < s_end; sbase += 128) {
      const long long p_first = sbase / N;
      const int off0 = (int)(sbase - p_first * N);
      const int nvalid = (int)min(128LL, s_end - sbase);
      const int npix = (int)((sbase + nvalid - 1) / N - p_first) + 1;
      const bool valid = t < nvalid;
      const int local = off0 + (valid ? t : nvalid - 1);
      const int ps = local / N;
      const int i = local - ps * N;
      const long long p = p_first + ps;

      // (a) primary features of the tile's pixels
      gather_primary_features(m.grid, pos4, p_first, npix, warp, lane, fpix);
      wg_sync(wg);

      const f3 x = xyz(pos4[p]);
      const f3 n = xyz(nrm4[p]);
      const f3 wo = xyz(view4[p]);
      const float4 ar = ar4[p];
      const uint64_t q = (uint64_t)(pixel_offset + p) * (uint64_t)N + (uint64_t)i;
      const f3 wi = m.mis ? mis_direction(m, n, wo, ar.w, i, dir_counter(q, M, 0))
                          : cosine_direction_fast(n, m.seed, dir_counter(q, M, 0));
      const EnvTap tap1 = env_tap_fast(m.env_h, m.env_w, wi);
      // MIS: the direction's Eq. 1 weight relative to cosine sampling rides on fr1
      const f3 fr1 = m.mis ? mis_weighted_brdf(m, xyz(ar), ar.w, n, wo, wi)
                           : brdf_eval_fast(xyz(ar), ar.w, n, wi, wo, m.f0, m.lambert);
      store_primary_split(fpix, ps, X_w, H_w, wi);

      // (c) I(f, w_i) in split precision: the hit test and the depth
      if (!run_mma([&] { mma_layer1_split(D_t, X_t, H_t, W_s + OFFB_IW1, W_s + OFFB_IW1L); })) { ok = false; break; }
      epilogue_hidden_split(D_w, X_w, H_w);
      if (!run_mma([&] {
            mma_layer2_split(D_t, X_t, H_t, W_s + OFFB_IW2, W_s + OFFB_IW2L, W_s + OFFB_ONES, W_s + OFFB_IB2);
          })) {
        ok = false;
        break;
      }
      float vis, tdep;
      {
        float z[2];
        head_fp32<2, 2>(D_w, &hp.iw3[0][0], hp.ib3, z);
        vis = visibility_from_logit(z[0], m.force_vis, 1);
        tdep = depth_fast(z[1], m.near_t, m.far_t);
      }
      // visible rows: the direct term of Eq. 2
      {
        f3 c[NL];
        const f3 w0 = fr1 * vis;
#pragma unroll
        for (int e = 0; e < NL; ++e) c[e] = w0 * env_fetch(envs + e * env_hw, tap1);
        add_rows(valid ? (int)p : -1, c);
      }
      // shadow rows join the queue in row order
      const bool shadow = valid && vis == 0.0f;
      const unsigned bal = __ballot_sync(0xffffffffu, shadow);
      if (lane == 0) wcnt[warp] = __popc(bal);
      wg_sync(wg);
      int before = 0, total = 0;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int cw = wcnt[w];
        before += w < warp ? cw : 0;
        total += cw;
      }
      if (shadow) {
        const uint32_t slot = (qtail + (uint32_t)(before + __popc(bal & ((1u << lane) - 1u)))) & 255u;
        qa[slot] = make_float4(wi.x, wi.y, wi.z, tdep);
        qb[slot] = make_int2((int)p, i);
      }
      qtail += (uint32_t)total;
      wg_sync(wg);   // the new entries are visible; wcnt is free
      while (ok && qtail - qhead >= 128u) {
        ok = secondary(128);
        qhead += 128u;
      }
    }
    if (ok && qtail != qhead) {
      ok = secondary((int)(qtail - qhead));
      qhead = qtail;
    }
    wg_sync(wg);
    if (ok) {
      const float sc = kPi / (float)N;
      for (long long p = p0 + t; p < p1; p += 128)
#pragma unroll
        for (int e = 0; e < NL; ++e) {
          float4* o = out + (long long)e * P + p;
          const float4 v = __ldcg(o);
          __stcg(o, make_float4(v.x * sc, v.y * sc, v.z * sc, 0.f));
        }
    }
  } else {
    for (long long sbase = p0 * N; sbase < s_end; sbase += 128) {
      const long long p_first = sbase / N;
      const int off0 = (int)(sbase - p_first * N);
      const int nvalid = (int)min(128LL, s_end - sbase);
      const int npix = (int)((sbase + nvalid - 1) / N - p_first) + 1;
      const bool valid = t < nvalid;
      const int local = off0 + (valid ? t : nvalid - 1);
      const int ps = local / N;
      const int i = local - ps * N;
      const long long p = p_first + ps;

      // (a) primary features of the tile's pixels
      gather_primary_features(m.grid, pos4, p_first, npix, warp, lane, fpix);
      wg_sync(wg);

      const f3 x = xyz(pos4[p]);
      const f3 n = xyz(nrm4[p]);
      const f3 wo = xyz(view4[p]);
      const float4 ar = ar4[p];
      const uint64_t q = (uint64_t)(pixel_offset + p) * (uint64_t)N + (uint64_t)i;
      const f3 wi = m.mis ? mis_direction(m, n, wo, ar.w, i, dir_counter(q, M, 0))
                          : cosine_direction_fast(n, m.seed, dir_counter(q, M, 0));
      // Eq. 1 factors of the primary direction, fetched before the MMAs so the
      // env-map loads overlap them
      const EnvTap tap1 = env_tap_fast(m.env_h, m.env_w, wi);
      // MIS: the direction's Eq. 1 weight relative to cosine sampling rides on fr1
      const f3 fr1 = m.mis ? mis_weighted_brdf(m, xyz(ar), ar.w, n, wo, wi)
                           : brdf_eval_fast(xyz(ar), ar.w, n, wi, wo, m.f0, m.lambert);
      f3 le1 = mk(0.f, 0.f, 0.f);
      if (NL == 1) le1 = env_fetch(envs, tap1);
      store_primary_split(fpix, ps, X_w, H_w, wi);

      // (c) I(f, w_i) in split precision: it alone sets t, and so x'
      if (!run_mma([&] { mma_layer1_split(D_t, X_t, H_t, W_s + OFFB_IW1, W_s + OFFB_IW1L); })) break;
      epilogue_hidden_split(D_w, X_w, H_w);
      if (!run_mma([&] {
            mma_layer2_split(D_t, X_t, H_t, W_s + OFFB_IW2, W_s + OFFB_IW2L, W_s + OFFB_ONES, W_s + OFFB_IB2);
          }))
        break;
      float v, tdep;
      {
        float z[2];
        head_fp32<2, 2>(D_w, &hp.iw3[0][0], hp.ib3, z);
        v = m.force_vis >= 0.f ? m.force_vis : sigmoid_fast(z[0]);
        tdep = depth_fast(z[1], m.near_t, m.far_t);
      }
      // Radiance is linear in the environment map: each light's contribution of
      // this row is fr1 (v Lenv(w_i) + (1 - v) (pi/M) sum_j v'_j fr2_j Lenv(w'_j)).
      f3 c[NL];
      {
        const f3 w0 = fr1 * v;
        if (NL == 1) {
          c[0] = w0 * le1;
        } else {
  #pragma unroll
          for (int e = 0; e < NL; ++e) c[e] = w0 * env_fetch(envs + e * env_hw, tap1);
        }
      }

      // (d) bounce: x' = x + t w_i; f' = H(x') into X columns 0..15
      encode_point_tmem(m.grid, x + wi * tdep, X_w);
      store_bias_cols_tmem(X_w);

      // (b) B(f')
      if (!run_mma([&] { mma_brdf_layer1(D_t, X_t, W_s + OFFB_BW1); })) break;
      epilogue_hidden(D_w, H_w);
      if (!run_mma([&] { mma_layer2(D_t, H_t, W_s + OFFB_BW2, W_s + OFFB_ONES, W_s + OFFB_BB2); })) break;
      f3 n2, a2;
      float r2;
      {
        float y[7];
        head_fp32<7, 8>(D_w, &hp.bw3[0][0], hp.bb3, y);
        const float ninv = rsqrtf(fmaxf(y[0] * y[0] + y[1] * y[1] + y[2] * y[2], 1e-24f));
        n2 = mk(y[0] * ninv, y[1] * ninv, y[2] * ninv);
        a2 = mk(sigmoid_fast(y[3]), sigmoid_fast(y[4]), sigmoid_fast(y[5]));
        r2 = 0.09f + 0.91f * sigmoid_fast(y[6]);
      }
      const f3 wo2 = neg(wi);
      const float wsec = (1.0f - v) * (kPi / (float)M);

      // (c) + (e) at x': M directions about n'
      bool ok = true;
      for (int j = 0; j < M && ok; ++j) {
        const f3 wj = cosine_direction_fast(n2, m.seed, dir_counter(q, M, 1 + j));
        const EnvTap tapj = env_tap_fast(m.env_h, m.env_w, wj);
        const f3 frw = fr1 * brdf_eval_fast(a2, r2, n2, wj, wo2, m.f0, m.lambert);
        f3 lej = mk(0.f, 0.f, 0.f);
        if (NL == 1) lej = env_fetch(envs, tapj);
        store_pe_tmem(X_w, wj);
        ok = run_mma([&] { mma_layer1(D_t, X_t, W_s + OFFB_IW1); });
        if (!ok) break;
        epilogue_hidden(D_w, H_w);
        ok = run_mma([&] { mma_layer2(D_t, H_t, W_s + OFFB_IW2, W_s + OFFB_ONES, W_s + OFFB_IB2); });
        if (!ok) break;
        const float v2 = m.force_vis2 >= 0.f ? m.force_vis2 : sigmoid_fast(head_vis(D_w, hp.iw3v, hp.ib3[0]));
        const f3 wj3 = frw * (wsec * v2);
        if (NL == 1) {
          c[0] = c[0] + wj3 * lej;
        } else {
  #pragma unroll
          for (int e = 0; e < NL; ++e) c[e] = c[e] + wj3 * env_fetch(envs + e * env_hw, tapj);
        }
      }
      if (!ok) break;

      // deterministic segmented reduction of the tile's rows into their pixels,
      // one light at a time
      const int key = valid ? ps : -1;
      const int prev = __shfl_up_sync(0xffffffffu, key, 1);
      const bool head = lane == 0 || prev != key;
  #pragma unroll
      for (int e = 0; e < NL; ++e) {
        f3 ce = valid ? c[e] : mk(0.f, 0.f, 0.f);
  #pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const float ox = __shfl_down_sync(0xffffffffu, ce.x, off);
          const float oy = __shfl_down_sync(0xffffffffu, ce.y, off);
          const float oz = __shfl_down_sync(0xffffffffu, ce.z, off);
          const int ok2 = __shfl_down_sync(0xffffffffu, key, off);
          if (lane + off < 32 && ok2 == key) ce = mk(ce.x + ox, ce.y + oy, ce.z + oz);
        }
        wg_sync(wg);   // fpix reads (first light) or the previous light's sums are done
        red[t] = head ? make_float4(ce.x, ce.y, ce.z, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        wg_sync(wg);
        if (t < npix) {
          const int ra = max(0, t * N - off0);
          const int rb = min(nvalid, (t + 1) * N - off0);
          f3 sum = mk(0.f, 0.f, 0.f);
          if (t == 0) {
            const float4 cs = carry_s[e];
            sum = mk(cs.x, cs.y, cs.z);
          }
          for (int r = ra; r < rb; r = ((r >> 5) + 1) << 5) {
            const float4 h = red[r];
            sum = mk(sum.x + h.x, sum.y + h.y, sum.z + h.z);
          }
          const bool complete = (p_first + t + 1) * N <= sbase + nvalid;
          if (complete) {
            const float sc = kPi / (float)N;
            out[(long long)e * P + p_first + t] = make_float4(sum.x * sc, sum.y * sc, sum.z * sc, 0.0f);
          }
          if (t == npix - 1)
            carry_s[e] = complete ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(sum.x, sum.y, sum.z, 0.f);
        }
      }
      wg_sync(wg);
    }

  }

  // ---- teardown: drain, then free TMEM
  abort = wg_sync_or(wg, abort);
  if (abort && t == 0) (void)mbar_wait(bar_a, pending_phase);   // let an MMA still in flight finish
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0 && wg == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(L::kTmemCols)
                 : "memory");
}

template <int NL, int WG, bool HARD>
cudaError_t prepare_variant() {
  using L = Layout<WG, HARD>;
  cudaError_t e = cudaFuncSetAttribute(render_bf16_kernel<NL, WG, HARD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L::kSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(render_bf16_kernel<NL, WG, HARD>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              L::kCarveout);
}

template <int NL, int WG, bool HARD>
cudaError_t launch_variant(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P, long long offset,
                           const float4* envs, float4* out, int num_sms, cudaStream_t s) {
  using L = Layout<WG, HARD>;
  const long long per_sm = L::kMinBlocks;
  const long long want = ((long long)P + WG - 1) / WG;
  const int grid = (int)(want < per_sm * num_sms ? want : per_sm * num_sms);
  render_bf16_kernel<NL, WG, HARD><<<grid, L::kThreads, L::kSmem, s>>>(m, hp, gb, P, offset, envs, out);
  return cudaGetLastError();
}

template <int WG, bool HARD>
cudaError_t launch_lights(int nl, const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P,
                          long long offset, const float4* envs, float4* out, int num_sms, cudaStream_t s) {
  switch (nl) {
    case 8: return launch_variant<8, WG, HARD>(m, hp, gb, P, offset, envs, out, num_sms, s);
    case 4: return launch_variant<4, WG, HARD>(m, hp, gb, P, offset, envs, out, num_sms, s);
    case 2: return launch_variant<2, WG, HARD>(m, hp, gb, P, offset, envs, out, num_sms, s);
    default: return launch_variant<1, WG, HARD>(m, hp, gb, P, offset, envs, out, num_sms, s);
  }
}

template <int WG, bool HARD>
cudaError_t prepare_wg() {
  cudaError_t e = prepare_variant<1, WG, HARD>();
  e = e != cudaSuccess ? e : prepare_variant<2, WG, HARD>();
  e = e != cudaSuccess ? e : prepare_variant<4, WG, HARD>();
  e = e != cudaSuccess ? e : prepare_variant<8, WG, HARD>();
  return e;
}

}  // namespace

cudaError_t prepare_render_bf16() {
  cudaError_t e = prepare_wg<2, false>();
  e = e != cudaSuccess ? e : prepare_wg<3, false>();
  e = e != cudaSuccess ? e : prepare_wg<4, false>();
  e = e != cudaSuccess ? e : prepare_wg<4, true>();
  return e;
}

// E lights in launches of up to `max_nl` (1, 2, 4 or 8) lights each; light e
// reads envs + e * env_h * env_w and writes out + e * P.  Every launch
// recomputes the geometry, so fewer, wider launches share more work.  Hard
// visibility always runs 4 warpgroups per CTA.
cudaError_t launch_render_bf16_lights(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P,
                                      long long offset, const float4* envs, int E, float4* out, int num_sms,
                                      int max_nl, int wg, cudaStream_t s) {
  const long long hw = (long long)m.env_h * m.env_w;
  for (int e0 = 0; e0 < E;) {
    int nl = 1;
    while (nl * 2 <= max_nl && nl * 2 <= E - e0) nl *= 2;
    ModelDesc mm = m;
    mm.env = envs + e0 * hw;
    const float4* ee = envs + e0 * hw;
    float4* oo = out + (long long)e0 * P;
    const cudaError_t err = m.hard    ? launch_lights<4, true>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s)
                            : wg == 2 ? launch_lights<2, false>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s)
                            : wg == 3 ? launch_lights<3, false>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s)
                                      : launch_lights<4, false>(nl, mm, hp, gb, P, offset, ee, oo, num_sms, s);
    if (err != cudaSuccess) return err;
    e0 += nl;
  }
  return cudaSuccess;
}

cudaError_t launch_render_bf16(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P,
                               long long offset, float4* out, int num_sms, cudaStream_t s) {
  return m.hard ? launch_variant<1, 4, true>(m, hp, gb, P, offset, m.env, out, num_sms, s)
                : launch_variant<1, 4, false>(m, hp, gb, P, offset, m.env, out, num_sms, s);
}

}  // namespace rtk
