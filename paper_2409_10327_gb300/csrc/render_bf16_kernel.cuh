// Fused BF16 tensor-core hot path: stages (a)-(e) of the hash renderer in one
// persistent kernel (rt_render_frame with precision RT_BF16).  The kernel
// template and its launch helpers; render_bf16.cu instantiates the
// consecutive-sample and hard-visibility variants, render_bf16_chunked.cu
// the direction-chunk tile shapes (rt_set_tile_shape).
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
#pragma once

#include <cuda_bf16.h>

#include "device_common.cuh"
#include "fast_math.cuh"
#include "mbarrier.cuh"
#include "mis.cuh"
#include "tc_common.cuh"

namespace rtk {

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
// shared-memory layout (offsets from a 1024-aligned base)
constexpr int SM_W = 0;
constexpr int WG_FPIX = 0;                   // primary features, bf16 hi parts [34][32]; reused as red[128] float4
constexpr int WG_FPIX_LO = kFpixLo;          // their bf16 lo parts [34][32]
constexpr int WG_MISC = 2 * kPixSlots * 64;  // mbarrier (8), then carry[kCarrySlots][NL] float4 from +16
constexpr int kCarrySlots = 4;               // pixels of a tile that carry partial sums to the next tile
constexpr int WG_BYTES = WG_MISC + 16 + kCarrySlots * 8 * 16;
// hard visibility: a ring of 256 queued shadow rows, the row keys of a tile and per-warp counts
constexpr int WG_QA = WG_BYTES;              // float4 (w_i, t) [256]
constexpr int WG_QB = WG_QA + 256 * 16;      // int2 (pixel, i) [256]
constexpr int WG_KEYS = WG_QB + 256 * 8;     // int [128]
constexpr int WG_CNT = WG_KEYS + 128 * 4;    // int [4]
constexpr int WG_BYTES_HARD = WG_CNT + 128;
constexpr int SM_WG = WBF16_BYTES;
static_assert(WG_MISC + 16 + kCarrySlots * 8 * 16 <= WG_BYTES, "warpgroup block overflow");
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

template <int NL, int WG, bool HARD, bool CHUNK>
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
  if (t < kCarrySlots * NL) carry_s[t] = make_float4(0.f, 0.f, 0.f, 0.f);

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
    // Tile order.  dpt = 0: tiles of 128 consecutive samples (pixel-major); a
    // pixel may start in one tile and end in the next.  dpt = 32 or 64 (the
    // tile shape of rt_set_tile_shape, N a multiple of it): a tile is
    // 128 / dpt pixels x dpt directions, and the warpgroup walks the N / dpt
    // direction chunks of a pixel group before the next group, each pixel's
    // sum carried across its chunks.  Every (pixel, direction) row computes
    // the same values in either order, and for N a multiple of 32 the sums are
    // added in the same order, so the two orders give the same bits.
    // (the chunked order is compiled only into the CHUNK instantiations: in the others dpt is the
    // constant 0, which keeps the consecutive order's code as tight as without the option)
    const int dpt = CHUNK && (m.dpt == 32 || m.dpt == 64) && N % m.dpt == 0 && N > m.dpt ? m.dpt : 0;
    const int gpix = dpt ? 128 / dpt : 0;
    const int nchunk = dpt ? N / dpt : 1;
    const long long ntiles = dpt ? (p1 - p0 + gpix - 1) / gpix * nchunk : (s_end - p0 * N + 127) / 128;
    for (long long tile = 0; tile < ntiles; ++tile) {
      long long p_first, sbase = 0;
      int off0 = 0, nvalid, npix, chunk = 0;
      if (dpt) {
        chunk = (int)(tile % nchunk);
        p_first = p0 + tile / nchunk * gpix;
        npix = (int)min((long long)gpix, p1 - p_first);
        nvalid = npix * dpt;
      } else {
        sbase = p0 * N + 128 * tile;
        p_first = sbase / N;
        off0 = (int)(sbase - p_first * N);
        nvalid = (int)min(128LL, s_end - sbase);
        npix = (int)((sbase + nvalid - 1) / N - p_first) + 1;
      }
      const bool valid = t < nvalid;
      const int row = valid ? t : nvalid - 1;
      int ps, i;
      if (dpt) {
        ps = row / dpt;
        i = chunk * dpt + (row - ps * dpt);
      } else {
        const int local = off0 + row;
        ps = local / N;
        i = local - ps * N;
      }
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
        // pixel slot t's partial sum from the previous tile (read before the barrier that orders it
        // against this tile's carry writes): slot 0 in the consecutive order, every slot between chunks
        f3 sum = mk(0.f, 0.f, 0.f);
        if (t < npix && (dpt ? chunk > 0 : t == 0)) {
          const float4 cs = carry_s[(dpt ? t : 0) * NL + e];
          sum = mk(cs.x, cs.y, cs.z);
        }
        wg_sync(wg);   // fpix reads (first light) or the previous light's sums are done
        red[t] = head ? make_float4(ce.x, ce.y, ce.z, 1.f) : make_float4(0.f, 0.f, 0.f, 0.f);
        wg_sync(wg);
        if (t < npix) {
          const int ra = dpt ? t * dpt : max(0, t * N - off0);
          const int rb = dpt ? ra + dpt : min(nvalid, (t + 1) * N - off0);
          for (int r = ra; r < rb; r = ((r >> 5) + 1) << 5) {
            const float4 h = red[r];
            sum = mk(sum.x + h.x, sum.y + h.y, sum.z + h.z);
          }
          const bool complete = dpt ? chunk == nchunk - 1 : (p_first + t + 1) * N <= sbase + nvalid;
          if (complete) {
            const float sc = kPi / (float)N;
            out[(long long)e * P + p_first + t] = make_float4(sum.x * sc, sum.y * sc, sum.z * sc, 0.0f);
          }
          if (dpt) {
            if (!complete) carry_s[t * NL + e] = make_float4(sum.x, sum.y, sum.z, 0.f);
          } else if (t == npix - 1) {
            carry_s[e] = complete ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(sum.x, sum.y, sum.z, 0.f);
          }
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

template <int NL, int WG, bool HARD, bool CHUNK>
cudaError_t prepare_variant() {
  using L = Layout<WG, HARD>;
  cudaError_t e = cudaFuncSetAttribute(render_bf16_kernel<NL, WG, HARD, CHUNK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L::kSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(render_bf16_kernel<NL, WG, HARD, CHUNK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              L::kCarveout);
}

template <int NL, int WG, bool HARD, bool CHUNK>
cudaError_t launch_variant(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P, long long offset,
                           const float4* envs, float4* out, int num_sms, cudaStream_t s) {
  using L = Layout<WG, HARD>;
  const long long per_sm = L::kMinBlocks;
  const long long want = ((long long)P + WG - 1) / WG;
  const int grid = (int)(want < per_sm * num_sms ? want : per_sm * num_sms);
  render_bf16_kernel<NL, WG, HARD, CHUNK><<<grid, L::kThreads, L::kSmem, s>>>(m, hp, gb, P, offset, envs, out);
  return cudaGetLastError();
}

template <int WG, bool HARD, bool CHUNK>
cudaError_t launch_lights(int nl, const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P,
                          long long offset, const float4* envs, float4* out, int num_sms, cudaStream_t s) {
  switch (nl) {
    case 8: return launch_variant<8, WG, HARD, CHUNK>(m, hp, gb, P, offset, envs, out, num_sms, s);
    case 4: return launch_variant<4, WG, HARD, CHUNK>(m, hp, gb, P, offset, envs, out, num_sms, s);
    case 2: return launch_variant<2, WG, HARD, CHUNK>(m, hp, gb, P, offset, envs, out, num_sms, s);
    default: return launch_variant<1, WG, HARD, CHUNK>(m, hp, gb, P, offset, envs, out, num_sms, s);
  }
}

template <int WG, bool HARD, bool CHUNK>
cudaError_t prepare_wg() {
  cudaError_t e = prepare_variant<1, WG, HARD, CHUNK>();
  e = e != cudaSuccess ? e : prepare_variant<2, WG, HARD, CHUNK>();
  e = e != cudaSuccess ? e : prepare_variant<4, WG, HARD, CHUNK>();
  e = e != cudaSuccess ? e : prepare_variant<8, WG, HARD, CHUNK>();
  return e;
}

}  // namespace

}  // namespace rtk
