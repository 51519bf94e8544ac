// Hand-written adjoint of the BF16 tensor-core renderer: rt_backward on a
// context with precision RT_BF16 (FP16 table, BF16 MLP operands, FP32
// accumulation).  For an upstream gradient dLoss/dL per pixel it accumulates
// dLoss/dtable (FP32, [L][T][F]) and dLoss/d(every weight and bias of B and
// I).  Sampled directions are constants of the estimator (Sec. 3.3
// distillation differentiates through the renderer; the sampling is not a
// parameter).  Activations are recomputed, never stored in global memory.
//
// Work unit: as in the BF16 forward, a warpgroup walks 128-row tiles of
// secondary samples (pixel p, direction i); thread t owns row t, TMEM lane t.
// Per tile it
//   1. recomputes I(f, w_i) in split precision (as the forward does: it sets
//      t and x'), f' = H(x') and B(f');
//   2. runs each secondary I(f', w'_j) forward, then its backward at once
//      (dv'_j and dfr2_j need only dLo2 = (1 - v) dL_i, which is known):
//      the output layer's gradient dZ3, then dZ2 = (dZ3 W3) . [pre2 > 0],
//      dH1 = dZ2 W2, dZ1 = dH1 . [H1 > 0] and df' += dZ1 W1f on the tensor
//      cores (dZ in TMEM as the A operand, the forward's weight tiles read
//      MN-major as W^T), and the weight gradients dW = dZ^T Xin as M = 64 MMAs whose
//      K dimension is the tile's 128 rows (dZ and the layer input staged in
//      shared memory, MN-major); the bias gradients db1 and db2 are dZ^T 1
//      against an all-ones tile, dW3 is relu(pre2)^T dZ3 and db3 a warp sum;
//   3. recomputes B and back-propagates it (dLoss/d(a', r', n') from step 2)
//      the same way into df';
//   4. scatters df' into the table at x' (the warp's points in Morton order,
//      runs of equal rows summed before one float2 reduction each), takes
//      dLoss/dx' from the interpolation derivative that step 1's encode of
//      x' cached in shared memory, turns it into dt and dz1, and back-
//      propagates the primary I (recomputed in split precision, back-
//      propagated in bf16) into its weights and into df;
//   5. sums df over the rows of each pixel of the tile and scatters it into
//      the table at x (the encode adjoint is linear, so a pixel split over
//      tiles scatters each part).
// Each weight-gradient MMA writes a scratch block in tensor memory (M = 64:
// the warp's 16 rows in lanes 0..15), which each warp transposes through its
// own slice of a staging tile (free once the MMAs that read it completed) and
// adds to the caller's blob with coalesced global reductions (float4 where the
// blobs are 16-byte aligned).  Every mbarrier wait is bounded; on expiry the
// warpgroup records kStatusTimeout | 2 and stops.
#include "adjoint.cuh"
#include "mbarrier.cuh"
#include "mis.cuh"
#include "tc_common.cuh"

namespace rtk {

namespace {

constexpr int kBWG = 2;                        // warpgroups per CTA (256 TMEM columns each)
constexpr int kBThreads = 128 * kBWG;
// TMEM columns of a warpgroup (from column 256 * wg)
constexpr int BT_D = 0;      // FP32 accumulator: forward layers, then dH = dZ W^T
constexpr int BT_X = 64;     // layer-1 input (bf16 pairs); the split primary's hi operands
constexpr int BT_H = 96;     // layer-2 input; the split primary's lo operands; dZ as an A operand
constexpr int BT_G = 128;    // weight-gradient scratch, M = 64 (dW row m in lane 32 (m / 16) + m % 16): 80 columns
constexpr int BT_F = 224;    // dLoss/df' (then df at the primary point) of the row, FP32 [32]
constexpr int kBTmemCols = 512;
// shared memory (from a 1024-aligned base)
constexpr int BS_W = 0;                               // the forward's BF16 weight image
constexpr int BS_WGB = ((WBF16_BYTES + 1023) / 1024) * 1024;
// per warpgroup: the MN-major staging tiles of the weight-gradient MMAs, the tile's primary features
// (hi / lo, then the per-pixel df sums) and the mbarrier
constexpr int WB_SA = 0;                              // [128 rows][64] bf16: dZ2 or dZ1 of the rows (A = dZ^T)
constexpr int WB_SB = 16384;                          // [128 rows][64] bf16: the layer input (B = Xin^T)
constexpr int WB_SC = 32768;                          // [128 rows][64] bf16: relu(pre2), for dW3^T = relu(pre2)^T dZ3
constexpr int WB_SD = 49152;                          // [128 rows][16] bf16 (32-byte swizzle): dZ3, zero-padded
constexpr int WB_FPIX = 53248;                        // kPixSlots x 64 B hi, then lo; later float [kPixSlots][32]
constexpr int WB_BAR = WB_FPIX + 2 * kFpixLo;
constexpr int WB_JAC = ((WB_BAR + 16 + 127) / 128) * 128;   // uint32 (half2) [3 L][128 rows]: d f' / d w at x'
constexpr int WB_BYTES = ((WB_JAC + 3 * kMaxLevels * 128 * 4 + 1023) / 1024) * 1024;
constexpr int BS_TSLOT = BS_WGB + kBWG * WB_BYTES;
constexpr size_t kBSmem16 = (size_t)BS_TSLOT + 16 + 1024;
static_assert(kPixSlots * 32 * 4 <= 2 * kFpixLo, "per-pixel df sums fit the feature slots");
static_assert(kBSmem16 <= 232448, "one CTA per SM");

// MN-major operand, 128-byte swizzle: K rows of 128 bytes (64 M/N elements), 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(1024u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// MN-major operand, 32-byte swizzle: K rows of 32 bytes (16 elements), 8-row groups 256 bytes apart
// (the all-ones tile, whose layout does not change its values).
__device__ __forceinline__ uint64_t sdesc_mn32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(256u >> 4) << 16;
  d |= (uint64_t)(256u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;
  return d;
}
constexpr uint32_t idesc_mn(int M, int N) { return idesc_bf16(M, N) | (1u << 15) | (1u << 16); }
constexpr uint32_t kIdescDW = idesc_mn(64, 64);
constexpr uint32_t kIdescDB = idesc_mn(64, 16);
// A in tensor memory, B MN-major: a forward weight tile [out rows][in, contiguous] read as W^T
constexpr uint32_t kIdescT64 = idesc_bf16(128, 64) | (1u << 16);
constexpr uint32_t kIdescT32 = idesc_bf16(128, 32) | (1u << 16);

// Chunk k (8 bf16, 4 packed pairs) of row `row` of an MN-major 128-byte-swizzled staging tile
// ([128 rows][64] bf16, the rows of an 8-row group 128 bytes apart, groups 1024 bytes apart).
__device__ __forceinline__ void stage_chunk(uint8_t* tile, int row, int k, uint32_t a, uint32_t b, uint32_t c,
                                            uint32_t d) {
  *reinterpret_cast<uint4*>(tile + (row >> 3) * 1024 + (row & 7) * 128 + ((k ^ (row & 7)) << 4)) =
      make_uint4(a, b, c, d);
}

// Row `row` of the 32-byte-swizzled MN-major tile SD: 8 bf16 (4 packed pairs) written into both 16-byte
// halves of the row, so that the swizzle's exchange of the halves leaves the row's values in place.
__device__ __forceinline__ void stage_row16(uint8_t* tile, int row, const uint32_t (&v)[4]) {
  uint8_t* base = tile + (row >> 3) * 256 + (row & 7) * 32;
  const uint4 q = make_uint4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<uint4*>(base) = q;
  *reinterpret_cast<uint4*>(base + 16) = q;
}

// The warp's 16 rows of a 64-column weight-gradient block in tensor memory (M = 64: row 16 warp + i in
// lane i < 16) into the warp's 4 KB slice of a staging tile, row r's 16-byte chunk k at
// r * 256 + ((k ^ r) << 4), so that writes by row and reads by column are free of bank conflicts.
__device__ __forceinline__ void block_to_slice(uint32_t g_w, uint8_t* slice, int lane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t r[32];
    tmem_ld32(g_w + 32 * h, r);
    tmem_ld_wait();
    if (lane < 16) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        *reinterpret_cast<uint4*>(slice + lane * 256 + (((8 * h + k) ^ lane) << 4)) =
            make_uint4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
    }
  }
  __syncwarp();
}
__device__ __forceinline__ float slice_at(const uint8_t* slice, int r, int c) {
  return *reinterpret_cast<const float*>(slice + r * 256 + (((c >> 2) ^ r) << 4) + 4 * (c & 3));
}
// dst[r * 64 + c] += slice[r][c] over the slice's 16 x 64 values, dst 16-byte aligned: float4 reductions,
// two rows per instruction.
__device__ __forceinline__ void slice_add_v4(const uint8_t* slice, float* dst, int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = 2 * i + (lane >> 4), k = lane & 15;
    const float4 v = *reinterpret_cast<const float4*>(slice + r * 256 + ((k ^ r) << 4));
    atomicAdd(reinterpret_cast<float4*>(dst + r * 64 + 4 * k), v);
  }
}
// dst[r * ld + map(c)] += slice[r][c] where map(c) >= 0: scalar reductions, 32 columns of a row per instruction.
template <class Map>
__device__ __forceinline__ void slice_add_mapped(const uint8_t* slice, float* dst, int ld, Map map, int lane) {
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    const int r = i >> 1, c = 32 * (i & 1) + lane;
    const int col = map(c);
    if (col >= 0) atomicAdd(dst + r * ld + col, slice_at(slice, r, c));
  }
}

// dW (+ db) of one layer over the tile: G[0:64) <- A^T B over the 128 rows, G[64:80) <- A^T ones.
__device__ __forceinline__ void mma_weight_grad(uint32_t g, uint32_t sa, uint32_t sb, uint32_t ones) {
#pragma unroll
  for (int k = 0; k < 8; ++k) mma_bf16(g, sdesc_mn(sa + 2048 * k), sdesc_mn(sb + 2048 * k), kIdescDW, k > 0 ? 1u : 0u);
#pragma unroll
  for (int k = 0; k < 8; ++k) mma_bf16(g + 64, sdesc_mn(sa + 2048 * k), sdesc_mn32(ones + 512 * k), kIdescDB, k > 0 ? 1u : 0u);
}
// dW3^T over the tile: G[80:96) <- relu(pre2)^T dZ3 (rows = hidden units, columns = outputs)
__device__ __forceinline__ void mma_w3_grad(uint32_t g, uint32_t sc, uint32_t sd) {
#pragma unroll
  for (int k = 0; k < 8; ++k) mma_bf16(g + 80, sdesc_mn(sc + 2048 * k), sdesc_mn32(sd + 512 * k), kIdescDB, k > 0 ? 1u : 0u);
}
// D <- Z . W^T: Z (the rows' dZ, bf16) in tensor memory, W the forward's weight tile [out][in]
// (K-major for the forward) read MN-major, i.e. as W^T [in][out]; N = 64 (all inputs) or 32 (f)
__device__ __forceinline__ void mma_input_grad(uint32_t d, uint32_t z_t, uint32_t w_s, uint32_t idesc, uint32_t acc0) {
#pragma unroll
  for (int k = 0; k < 4; ++k) mma_bf16_ts(d, z_t + 8 * k, sdesc_mn(w_s + 2048 * k), idesc, (k > 0 || acc0) ? 1u : 0u);
}

// The primary evaluation's layer-1 input [f | PE(w) | 1 | 1 | 0] as bf16 hi parts into X (the
// operand of its weight gradient; the split forward's hi parts).
__device__ __forceinline__ void store_primary_hi(const uint8_t* fpix, int slot, uint32_t x_taddr, f3 w) {
  const uint4* src = reinterpret_cast<const uint4*>(fpix + slot * 64);
  uint32_t fr[16];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const uint4 v = src[c];
    fr[4 * c] = v.x;
    fr[4 * c + 1] = v.y;
    fr[4 * c + 2] = v.z;
    fr[4 * c + 3] = v.w;
  }
  tmem_st16(x_taddr, fr);
  store_pe_tmem(x_taddr, w);
}


}  // namespace

namespace {

template <int DUMMY>
__global__ void __launch_bounds__(kBThreads, 1)
backward_bf16_kernel(const __grid_constant__ ModelDesc m, const __grid_constant__ HeadParams hp, rt_gbuffer gb, int P,
                     long long pixel_offset, const float4* __restrict__ dL, float* __restrict__ g_table,
                     float* __restrict__ g_brdf, float* __restrict__ g_irt) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x;
  const int wg = tid >> 7, t = tid & 127, warp = t >> 5, lane = t & 31;
  uint8_t* Wsm = sm + BS_W;
  uint8_t* wgb = sm + BS_WGB + wg * WB_BYTES;
  uint8_t* SA = wgb + WB_SA;
  uint8_t* SB = wgb + WB_SB;
  uint8_t* fpix = wgb + WB_FPIX;
  float* dfs = reinterpret_cast<float*>(wgb + WB_FPIX);   // [kPixSlots][32] after the features are consumed
  uint64_t* bar = reinterpret_cast<uint64_t*>(wgb + WB_BAR);
  uint32_t* jac = reinterpret_cast<uint32_t*>(wgb + WB_JAC);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + BS_TSLOT);

  // ---- CTA set-up: weights (the forward's image), TMEM, barriers
  for (int i = tid; i < WBF16_BYTES / 16; i += kBThreads)
    reinterpret_cast<uint4*>(Wsm)[i] = __ldg(reinterpret_cast<const uint4*>(m.wbf16) + i);
  if (t == 0) {
    mbar_init(smem_u32(bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kBTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot + (uint32_t)(256 * wg);
  const uint32_t D_t = tmem + BT_D, X_t = tmem + BT_X, H_t = tmem + BT_H, G_t = tmem + BT_G, F_t = tmem + BT_F;
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
  const uint32_t D_w = D_t + lane_off, X_w = X_t + lane_off, H_w = H_t + lane_off, G_w = G_t + lane_off,
                 F_w = F_t + lane_off;
  const uint32_t bar_a = smem_u32(bar);
  uint8_t* SC = wgb + WB_SC;
  uint8_t* SD = wgb + WB_SD;
  const uint32_t W_s = smem_u32(Wsm), SA_s = smem_u32(SA), SB_s = smem_u32(SB), SC_s = smem_u32(SC),
                 SD_s = smem_u32(SD);
  const uint32_t ONES_s = W_s + OFFB_ONES;

  const int N = m.N, M = m.M, lf = m.lf;
  const int in_i = lf + kPE;
  const bool disney = !m.lambert;
  const BlobB gB{g_brdf, lf};
  const float4* pos4 = reinterpret_cast<const float4*>(gb.pos);
  const float4* nrm4 = reinterpret_cast<const float4*>(gb.normal);
  const float4* view4 = reinterpret_cast<const float4*>(gb.view);
  const float4* ar4 = reinterpret_cast<const float4*>(gb.albedo_rough);

  const long long workers = (long long)gridDim.x * kBWG;
  const long long worker = (long long)blockIdx.x * kBWG + wg;
  const long long p0 = (long long)P * worker / workers, p1 = (long long)P * (worker + 1) / workers;
  const long long s_end = p1 * N;
  uint32_t phase = 0, pending_phase = 0;
  int abort = 0;

  // One MMA round trip (as in the forward): the rows' TMEM stores and staging-tile stores are made
  // visible to the tensor core, the warpgroup votes on `abort`, thread 0 issues and commits, and every
  // thread waits on the mbarrier with a bound.
  auto run_mma = [&](auto issue) -> bool {
    tmem_st_wait();
    fence_async_smem();
    tc_fence_before();
    abort = wg_sync_or(wg, abort);
    if (abort) return false;
    if (t == 0) {
      tc_fence_after();
      issue();
      mma_commit(bar_a);
    }
    if (!mbar_wait(bar_a, phase)) {
      if (!abort && t == 0) atomicOr(m.status, kStatusTimeout | 2u);
      abort = 1;
      pending_phase = phase;
    }
    phase ^= 1u;
    tc_fence_after();
    return true;
  };

  // layer-1 input column (f features, then the PE, then the two ones columns) -> blob column
  auto map_w1 = [lf](int c) { return c < lf ? c : (c >= 32 && c < 32 + kPE ? lf + (c - 32) : -1); };
  auto map_w1b = [lf](int c) { return c < lf ? c : -1; };
  auto w3_i = [&](int k, int o) { return hp.iw3[k][o]; };
  auto w3_b = [&](int k, int o) { return hp.bw3[k][o]; };
  // the weight-gradient blocks go out as float4 reductions where both blobs are 16-byte aligned
  const bool v4ok = ((reinterpret_cast<uintptr_t>(g_irt) | reinterpret_cast<uintptr_t>(g_brdf)) & 15u) == 0u;
  uint8_t* slice = SA + 4096 * warp;   // the warp's staged rows (32 warp .. 32 warp + 31) of SA
  // canonical blob of I: W1 [64][in_i], b1, W2, b2, W3 [2][64], b3
  float* const iW1 = g_irt;
  float* const iB1 = iW1 + 64 * in_i;
  float* const iW2 = iB1 + 64;
  float* const iB2 = iW2 + 4096;
  float* const iW3 = iB2 + 64;
  float* const iB3 = iW3 + 128;

  // Backward of one MLP evaluation of the tile from its output gradient dz3 (a float array of the net's
  // outputs; w3(k, o) the output layer's weight from hidden unit k to output o), with pre2 (the layer-2
  // accumulator) in D, H1 in the H columns and the layer-1 input in the X columns.
  //   round trip 1: dZ2 = (dZ3 W3) . [pre2 > 0] (in H as the A operand, and in SA), H1 in SB,
  //     relu(pre2) in SC, dZ3 in SD: dH1 = dZ2 W2 into D; dW2 and db2 (A^T ones) into G[0:80),
  //     dW3^T into G[80:96);
  //   round trip 2: dZ1 = dH1 . [H1 > 0] (H and SA), the layer-1 input in SB: df += dZ1 W1f into F,
  //     dW1 and db1 into G.
  // Each weight-gradient block goes to the caller's blob through the warp's slice of SA (global
  // reductions); db3 by warp reductions.  w1s / w2s are the forward's weight tiles, read as W^T.
  auto layer_backward = [&](const auto& dz3, auto w3, uint32_t w2s, uint32_t w1s, bool acc_f, float* gw3,
                            float* gb3, float* gw2, float* gb2, float* gw1, float* gb1, int ldw1, auto map1) -> bool {
    constexpr int nout = (int)(sizeof(dz3) / sizeof(float));
    uint32_t mlo = 0, mhi = 0;   // the ReLU mask of layer 1, one bit per hidden unit
    // H1 (layer 2's input) into SB, and its mask (H1 = bf16(relu(.)) is positive or zero)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t r[16];
      tmem_ld16(H_w + 16 * h, r);
      tmem_ld_wait();
#pragma unroll
      for (int k = 0; k < 4; ++k) stage_chunk(SB, t, 4 * h + k, r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
      uint32_t bits = 0;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        bits |= (((r[c] & 0xFFFFu) != 0u ? 1u : 0u) | ((r[c] >> 16) != 0u ? 2u : 0u)) << (2 * c);
      if (h == 0) mlo = bits;
      else mhi = bits;
    }
    // dZ2 into SA and H, relu(pre2) into SC, 32 hidden units at a time
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t r[32];
      tmem_ld32(D_w + 32 * h, r);
      tmem_ld_wait();
      uint32_t a[16], h2[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float z[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int k = 32 * h + 2 * c + u;
          float acc = 0.0f;
#pragma unroll
          for (int o = 0; o < nout; ++o) acc = fmaf(dz3[o], w3(k, o), acc);
          z[u] = __uint_as_float(r[2 * c + u]) > 0.0f ? acc : 0.0f;
        }
        a[c] = pack_bf16(z[0], z[1]);
        h2[c] = pack_relu_bf16(__uint_as_float(r[2 * c]), __uint_as_float(r[2 * c + 1]));
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        stage_chunk(SA, t, 4 * h + k, a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        stage_chunk(SC, t, 4 * h + k, h2[4 * k], h2[4 * k + 1], h2[4 * k + 2], h2[4 * k + 3]);
      }
      tmem_st16(H_w + 16 * h, a);
    }
    {
      uint32_t d3[4];
#pragma unroll
      for (int c = 0; c < 4; ++c)
        d3[c] = pack_bf16(2 * c < nout ? dz3[2 * c < nout ? 2 * c : 0] : 0.0f,
                          2 * c + 1 < nout ? dz3[2 * c + 1 < nout ? 2 * c + 1 : 0] : 0.0f);
      stage_row16(SD, t, d3);
    }
    // db3: the column sums of dZ3, one warp reduction per output
#pragma unroll
    for (int o = 0; o < nout; ++o) {
      float v = dz3[o];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) atomicAdd(gb3 + o, v);
    }
    if (!run_mma([&] {
          mma_input_grad(D_t, H_t, w2s, kIdescT64, 0u);
          mma_weight_grad(G_t, SA_s, SB_s, ONES_s);
          mma_w3_grad(G_t, SC_s, SD_s);
        }))
      return false;
    const int grow = 16 * warp + lane;   // the G row of lanes 0..15
    block_to_slice(G_w, slice, lane);
    if (v4ok) slice_add_v4(slice, gw2 + 16 * warp * 64, lane);
    else slice_add_mapped(slice, gw2 + 16 * warp * 64, 64, [](int c) { return c; }, lane);
    {
      uint32_t r[32];
      tmem_ld32(G_w + 64, r);   // column 64 (db2) and columns 80.. (dW3^T)
      tmem_ld_wait();
      if (lane < 16) {
        atomicAdd(gb2 + grow, __uint_as_float(r[0]));
#pragma unroll
        for (int o = 0; o < nout; ++o) atomicAdd(gw3 + o * 64 + grow, __uint_as_float(r[16 + o]));
      }
    }
    __syncwarp();   // the slice is read before the rows are staged again
    // dZ1 into SA and H, the layer-1 input into SB
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t r[32];
      tmem_ld32(D_w + 32 * h, r);
      tmem_ld_wait();
      const uint32_t mk = h ? mhi : mlo;
      uint32_t a[16];
#pragma unroll
      for (int c = 0; c < 16; ++c)
        a[c] = pack_bf16(((mk >> (2 * c)) & 1u) ? __uint_as_float(r[2 * c]) : 0.0f,
                         ((mk >> (2 * c)) & 2u) ? __uint_as_float(r[2 * c + 1]) : 0.0f);
#pragma unroll
      for (int k = 0; k < 4; ++k) stage_chunk(SA, t, 4 * h + k, a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
      tmem_st16(H_w + 16 * h, a);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t r[16];
      tmem_ld16(X_w + 16 * h, r);
      tmem_ld_wait();
#pragma unroll
      for (int k = 0; k < 4; ++k) stage_chunk(SB, t, 4 * h + k, r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
    }
    if (!run_mma([&] {
          mma_input_grad(F_t, H_t, w1s, kIdescT32, acc_f ? 1u : 0u);
          mma_weight_grad(G_t, SA_s, SB_s, ONES_s);
        }))
      return false;
    // dW1 (the ones columns of the input are not mapped; db1 is column 64)
    block_to_slice(G_w, slice, lane);
    slice_add_mapped(slice, gw1 + 16 * warp * ldw1, ldw1, map1, lane);
    {
      uint32_t b[1];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(b[0]) : "r"(G_w + 64));
      tmem_ld_wait();
      if (lane < 16) atomicAdd(gb1 + grow, __uint_as_float(b[0]));
    }
    __syncwarp();
    return true;
  };

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

    // (a) primary features of the tile's pixels (hi / lo)
    gather_primary_features(m.grid, pos4, p_first, npix, warp, lane, fpix);
    wg_sync(wg);

    const f3 x = xyz(pos4[p]);
    const f3 n = xyz(nrm4[p]);
    const f3 wo = xyz(view4[p]);
    const float4 ar = ar4[p];
    const f3 Gp = valid ? xyz(dL[p]) : mk(0.f, 0.f, 0.f);
    const uint64_t q = (uint64_t)(pixel_offset + p) * (uint64_t)N + (uint64_t)i;
    const f3 wi = m.mis ? mis_direction(m, n, wo, ar.w, i, dir_counter(q, M, 0))
                        : cosine_direction_fast(n, m.seed, dir_counter(q, M, 0));
    const EnvTap tap1 = env_tap_fast(m.env_h, m.env_w, wi);
    const f3 fr1 = m.mis ? mis_weighted_brdf(m, xyz(ar), ar.w, n, wo, wi)
                         : brdf_eval_fast(xyz(ar), ar.w, n, wi, wo, m.f0, m.lambert);
    const f3 le1 = env_fetch(m.env, tap1);

    // (c) I(f, w_i) in split precision, as the forward: v and t
    store_primary_split(fpix, ps, X_w, H_w, wi);
    if (!run_mma([&] { mma_layer1_split(D_t, X_t, H_t, W_s + OFFB_IW1, W_s + OFFB_IW1L); })) break;
    epilogue_hidden_split(D_w, X_w, H_w);
    if (!run_mma([&] {
          mma_layer2_split(D_t, X_t, H_t, W_s + OFFB_IW2, W_s + OFFB_IW2L, W_s + OFFB_ONES, W_s + OFFB_IB2);
        }))
      break;
    float z0p, z1p;
    {
      float z[2];
      head_fp32<2, 2>(D_w, &hp.iw3[0][0], hp.ib3, z);
      z0p = z[0];
      z1p = z[1];
    }
    const float v = m.force_vis >= 0.f ? m.force_vis : sigmoid_fast(z0p);
    const float sp = softplus_fast(z1p);
    const float tdep = m.near_t + (m.far_t - m.near_t) * fminf(sp, 1.0f);
    const f3 x2 = x + wi * tdep;

    // (d) f' = H(x') into X, with its derivative along the cell fractions for dLoss/dx'; (b) B(f')
    encode_point_tmem<true>(m.grid, x2, X_w, jac, t);
    store_bias_cols_tmem(X_w);
    if (!run_mma([&] { mma_brdf_layer1(D_t, X_t, W_s + OFFB_BW1); })) break;
    epilogue_hidden(D_w, H_w);
    if (!run_mma([&] { mma_layer2(D_t, H_t, W_s + OFFB_BW2, W_s + OFFB_ONES, W_s + OFFB_BB2); })) break;
    float yB[7];
    head_fp32<7, 8>(D_w, &hp.bw3[0][0], hp.bb3, yB);
    const float nlen = sqrtf(fmaxf(yB[0] * yB[0] + yB[1] * yB[1] + yB[2] * yB[2], 1e-24f));
    const f3 n2 = mk(yB[0] / nlen, yB[1] / nlen, yB[2] / nlen);
    const f3 a2 = mk(sigmoid_fast(yB[3]), sigmoid_fast(yB[4]), sigmoid_fast(yB[5]));
    const float s6 = sigmoid_fast(yB[6]);
    const float r2 = 0.09f + 0.91f * s6;
    const f3 wo2 = neg(wi);

    // (e) Eq. 2 / Eq. 1 adjoint of the row: dL_i and dLo2
    const float sN = kPi / (float)N, sM = kPi / (float)M;
    const f3 dli = (Gp * fr1) * sN;
    const f3 dlo2 = dli * (1.0f - v);

    // secondary directions: forward, then backward, of I(f', w'_j)
    f3 lo2 = mk(0.f, 0.f, 0.f), da2 = mk(0.f, 0.f, 0.f), dn2 = mk(0.f, 0.f, 0.f);
    float dr2 = 0.0f;
    bool ok = true;
    for (int j = 0; j < M && ok; ++j) {
      const f3 wj = cosine_direction_fast(n2, m.seed, dir_counter(q, M, 1 + j));
      const EnvTap tapj = env_tap_fast(m.env_h, m.env_w, wj);
      const f3 le = env_fetch(m.env, tapj);
      float ds_dr = 0.0f;
      f3 ds_dn = mk(0.f, 0.f, 0.f);
      const float s = disney ? spec_with_grad(r2, n2, wj, wo2, m.f0, ds_dr, ds_dn) : 0.0f;
      const f3 fr2 = mk(a2.x * kInvPi + s, a2.y * kInvPi + s, a2.z * kInvPi + s);
      const f3 ef = le * fr2;
      store_pe_tmem(X_w, wj);
      ok = run_mma([&] { mma_layer1(D_t, X_t, W_s + OFFB_IW1); });
      if (!ok) break;
      epilogue_hidden(D_w, H_w);
      ok = run_mma([&] { mma_layer2(D_t, H_t, W_s + OFFB_IW2, W_s + OFFB_ONES, W_s + OFFB_IB2); });
      if (!ok) break;
      const float z0 = head_vis(D_w, hp.iw3v, hp.ib3[0]);
      const float v2 = m.force_vis2 >= 0.f ? m.force_vis2 : sigmoid_fast(z0);
      lo2 = lo2 + ef * v2;
      const float dv2 = sM * dot(dlo2, ef);
      const f3 dfr = (dlo2 * le) * (sM * v2);
      da2 = da2 + dfr * kInvPi;
      if (disney) {
        const float dsum = dfr.x + dfr.y + dfr.z;
        dr2 += dsum * ds_dr;
        dn2 = dn2 + ds_dn * dsum;
      }
      const float dz3[1] = {m.force_vis2 >= 0.f ? 0.0f : dv2 * v2 * (1.0f - v2)};
      ok = layer_backward(dz3, w3_i, W_s + OFFB_IW2, W_s + OFFB_IW1, j > 0, iW3, iB3, iW2, iB2, iW1, iB1, in_i, map_w1);
    }
    if (!ok) break;
    lo2 = lo2 * sM;
    const float dv = dot(dli, le1 - lo2);

    // B backward (forward recomputed: the secondary loop overwrote D and H)
    store_bias_cols_tmem(X_w);
    if (!run_mma([&] { mma_brdf_layer1(D_t, X_t, W_s + OFFB_BW1); })) break;
    epilogue_hidden(D_w, H_w);
    if (!run_mma([&] { mma_layer2(D_t, H_t, W_s + OFFB_BW2, W_s + OFFB_ONES, W_s + OFFB_BB2); })) break;
    {
      float dy[7];
      const float dnn = dot(n2, dn2);
      dy[0] = (dn2.x - n2.x * dnn) / nlen;
      dy[1] = (dn2.y - n2.y * dnn) / nlen;
      dy[2] = (dn2.z - n2.z * dnn) / nlen;
      dy[3] = da2.x * a2.x * (1.0f - a2.x);
      dy[4] = da2.y * a2.y * (1.0f - a2.y);
      dy[5] = da2.z * a2.z * (1.0f - a2.z);
      dy[6] = dr2 * 0.91f * s6 * (1.0f - s6);
      if (!layer_backward(dy, w3_b, W_s + OFFB_BW2, W_s + OFFB_BW1, M > 0, gB.w3(), gB.b3(), gB.w2(), gB.b2(), gB.w1(),
                          gB.b1(), lf, map_w1b))
        break;
    }

    // encode adjoint at x': table gradients (segmented scatter over the warp's points in Morton order),
    // and dLoss/dx' = sum over levels of (N_l / 2) (d f'_l / d w) . dLoss/df'_l from the cached derivative
    f3 dx2 = mk(0.f, 0.f, 0.f);
    {
      uint32_t r[32];
      tmem_ld32(F_w, r);
      tmem_ld_wait();
      (void)encode_bwd_sorted<false>(m.grid, x2, r, valid, g_table, nullptr);
      if (valid) {
#pragma unroll 1
        for (int l = 0; l < m.grid.levels; ++l) {
          float d0 = 0.f, d1 = 0.f;
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (k == l) {
              d0 = __uint_as_float(r[2 * k]);
              d1 = __uint_as_float(r[2 * k + 1]);
            }
          const float s = (float)m.grid.res[l];   // N_l / 2 times the halving of the stored derivative
          float g3[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const uint32_t wv = jac[(3 * l + a) * 128 + t];
            const float2 j = __half22float2(*reinterpret_cast<const __half2*>(&wv));
            g3[a] = s * fmaf(j.x, d0, j.y * d1);
          }
          dx2 = mk(dx2.x + g3[0], dx2.y + g3[1], dx2.z + g3[2]);
        }
        // dg/dx = N_l / 2 inside the box, 0 on a clamped axis
        const float ux = x2.x * 0.5f + 0.5f, uy = x2.y * 0.5f + 0.5f, uz = x2.z * 0.5f + 0.5f;
        dx2 = mk((ux >= 0.0f && ux <= 1.0f) ? dx2.x : 0.0f, (uy >= 0.0f && uy <= 1.0f) ? dx2.y : 0.0f,
                 (uz >= 0.0f && uz <= 1.0f) ? dx2.z : 0.0f);
      }
    }
    const float dt = dot(dx2, wi);
    float dzp[2];
    dzp[0] = (m.force_vis >= 0.f || !valid) ? 0.0f : dv * v * (1.0f - v);
    dzp[1] = (sp <= 1.0f && valid) ? dt * (m.far_t - m.near_t) * sigmoid_fast(z1p) : 0.0f;

    // primary I backward: forward recomputed in split precision, back-propagated in bf16 (layer-1
    // input and hidden layer taken as their hi parts)
    store_primary_split(fpix, ps, X_w, H_w, wi);
    if (!run_mma([&] { mma_layer1_split(D_t, X_t, H_t, W_s + OFFB_IW1, W_s + OFFB_IW1L); })) break;
    epilogue_hidden_split(D_w, H_w, X_w);   // hi parts into H (layer 2's input as layer_backward reads it), lo into X
    if (!run_mma([&] {
          mma_layer2_split(D_t, H_t, X_t, W_s + OFFB_IW2, W_s + OFFB_IW2L, W_s + OFFB_ONES, W_s + OFFB_IB2);
        }))
      break;
    store_primary_hi(fpix, ps, X_w, wi);   // the layer-1 input's hi parts back into X
    {
      // as layer_backward, with the primary point's df accumulated into F afresh
      if (!layer_backward(dzp, w3_i, W_s + OFFB_IW2, W_s + OFFB_IW1, false, iW3, iB3, iW2, iB2, iW1, iB1, in_i, map_w1))
        break;
    }

    // primary encode adjoint: df summed over the tile's rows of each pixel, then scattered at x
    {
      uint32_t r[32];
      tmem_ld32(F_w, r);
      tmem_ld_wait();
      wg_sync(wg);   // the feature slots are no longer read
      for (int e = t; e < npix * 32; e += 128) dfs[e] = 0.0f;
      wg_sync(wg);
      // rows of a warp that share a pixel are summed by a segmented shuffle reduction first
      const int key = valid ? ps : -1;
      const int prev = __shfl_up_sync(0xffffffffu, key, 1);
      const bool head = lane == 0 || prev != key;
      uint32_t same = 0;   // bit s: the row 2^s lanes down belongs to the same pixel
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        const int k2 = __shfl_down_sync(0xffffffffu, key, 1 << s);
        if (lane + (1 << s) < 32 && k2 == key) same |= 1u << s;
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        float val = valid ? __uint_as_float(r[k]) : 0.0f;
#pragma unroll
        for (int s = 0; s < 5; ++s) {
          const float o = __shfl_down_sync(0xffffffffu, val, 1 << s);
          if (same & (1u << s)) val += o;
        }
        if (head && key >= 0 && k < lf) atomicAdd(dfs + key * 32 + k, val);
      }
      wg_sync(wg);
      for (int e = t; e < npix * 16; e += 128) {
        const int slot = e >> 4, l = e & 15;
        if (l < m.grid.levels)
          encode_level_bwd(m.grid, l, xyz(pos4[p_first + slot]), dfs[slot * 32 + 2 * l], dfs[slot * 32 + 2 * l + 1],
                           g_table, nullptr);
      }
      wg_sync(wg);   // the slots are free for the next tile's features
    }
  }

  // ---- teardown: drain, free TMEM
  abort = wg_sync_or(wg, abort);
  if (abort && t == 0) (void)mbar_wait(bar_a, pending_phase);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(kBTmemCols) : "memory");
}

}  // namespace

cudaError_t prepare_backward_bf16() {
  cudaError_t e = cudaFuncSetAttribute(backward_bf16_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kBSmem16);
  return e;
}

cudaError_t launch_backward_bf16(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P, long long offset,
                                 const float4* dL, float* g_table, float* g_brdf, float* g_irt, int num_sms,
                                 cudaStream_t s) {
  const long long want = ((long long)P + kBWG - 1) / kBWG;
  const int grid = (int)(want < num_sms ? want : num_sms);
  backward_bf16_kernel<0><<<grid, kBThreads, kBSmem16, s>>>(m, hp, gb, P, offset, dL, g_table, g_brdf, g_irt);
  return cudaGetLastError();
}

}  // namespace rtk
