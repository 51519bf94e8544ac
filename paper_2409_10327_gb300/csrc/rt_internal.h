// Internal types shared by the host API and the kernels of the GB300 renderer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rt.h"

namespace rtk {

constexpr int kMaxLevels = 16;
constexpr int kHidden = 64;     // width of both MLPs (Sec. 4.1)
constexpr int kPE = 27;         // [w, sin(2^k pi w), cos(2^k pi w)], k = 0..3
constexpr int kPEPad = 32;
constexpr int kBrdfOut = 7;     // [n(3), a(3), r]
constexpr int kIrtOut = 2;      // [visibility logit, depth logit]

// Packed FP32 weight image (floats).  Weights are stored transposed,
// [in][out] with out = 64 contiguous, so that one k step of a warp GEMM
// reads a 64-wide row.  Rows beyond the true fan-in are zero.  The image is
// copied verbatim into shared memory by the fused kernels.
constexpr int OFF_IW1F = 0;                      // I, layer 1, feature rows   [32][64]
constexpr int OFF_IW1P = OFF_IW1F + 32 * 64;     // I, layer 1, PE rows        [32][64]
constexpr int OFF_IB1 = OFF_IW1P + 32 * 64;      // [64]
constexpr int OFF_IW2 = OFF_IB1 + 64;            // [64][64]
constexpr int OFF_IB2 = OFF_IW2 + 64 * 64;       // [64]
constexpr int OFF_IW3 = OFF_IB2 + 64;            // [64][2]
constexpr int OFF_IB3 = OFF_IW3 + 64 * 2;        // [2] + 2 pad
constexpr int OFF_BW1 = OFF_IB3 + 4;             // B, layer 1                 [32][64]
constexpr int OFF_BB1 = OFF_BW1 + 32 * 64;       // [64]
constexpr int OFF_BW2 = OFF_BB1 + 64;            // [64][64]
constexpr int OFF_BB2 = OFF_BW2 + 64 * 64;       // [64]
constexpr int OFF_BW3 = OFF_BB2 + 64;            // [64][8] (7 + pad)
constexpr int OFF_BB3 = OFF_BW3 + 64 * 8;        // [8]
constexpr int WPACK_FLOATS = OFF_BB3 + 8;
static_assert(OFF_BW1 % 4 == 0 && OFF_BW3 % 4 == 0 && WPACK_FLOATS % 4 == 0, "float4 alignment");

// BF16 weight image for the tensor-core path (bytes).  The 64 x 64 matrices
// are stored as [N rows = outputs][K = 64 inputs] bf16, K-major, in the
// 128-byte swizzle of tcgen05 shared-memory descriptors: element (n, k) of a
// tile lives at (n/8)*1024 + (n%8)*128 + (((2k)/16) ^ (n%8))*16 + (2k)%16.
// Layer-1 biases ride in the A tile: its columns 59 and 60 hold 1.0, and
// columns 59/60 of I's and B's layer-1 tiles hold the bf16 hi/lo split of b1
// (B's layer 1 reads K-steps 0, 1 and 3).  Layer-2 biases come from one more
// K = 16 MMA of a constant all-ones tile [128 x 16] against a bias tile
// [64 x 16] whose row n holds 8 x hi/8 and 8 x lo/8 of b2[n] (both tiles in
// the 32-byte swizzle, 32-byte rows, 8-row groups 256 bytes apart; a row's
// sum does not depend on how the swizzle permutes its two 16-byte halves).
// I layer 1 takes [f (32, zero beyond L*F) | PE (27) | 1 | 1 | 0 (3)].
// The primary evaluation of I runs in split precision: each operand is the
// sum of a bf16 hi part and a bf16 lo part (the rounding residual), and the
// product is hi.hi + lo.hi + hi.lo; the last two tiles hold the lo parts of
// I's layer-1 and layer-2 weights (zero in the bias columns).
constexpr int OFFB_IW1 = 0;        // 64 x 64
constexpr int OFFB_IW2 = 8192;     // 64 x 64
constexpr int OFFB_BW1 = 16384;    // 64 x 64 (k < L*F, and the bias columns)
constexpr int OFFB_BW2 = 24576;    // 64 x 64
constexpr int OFFB_IB2 = 32768;    // 64 x 16, 32-byte swizzle
constexpr int OFFB_BB2 = 34816;    // 64 x 16, 32-byte swizzle
constexpr int OFFB_ONES = 36864;   // 128 x 16 of 1.0, 32-byte swizzle
constexpr int OFFB_IW1L = 40960;   // 64 x 64, lo parts of I's layer 1 (f and PE columns)
constexpr int OFFB_IW2L = 49152;   // 64 x 64, lo parts of I's layer 2
constexpr int WBF16_BYTES = 57344;
constexpr int kBiasCol = 59;       // A-tile / layer-1 columns carrying b1 (hi at 59, lo at 60)

__host__ __device__ constexpr int swz128(int n, int k) {
  return (n >> 3) * 1024 + (n & 7) * 128 + ((((2 * k) >> 4) ^ (n & 7)) << 4) + ((2 * k) & 15);
}

// Hash-grid description passed by value to kernels.
struct GridDesc {
  int levels;
  int log2T;
  uint32_t mask;               // T - 1
  int half;                    // 1: table entries are 2 x IEEE half
  const void* table;           // [L][T][2]
  int res[kMaxLevels];
  int dense[kMaxLevels];
};

// Everything the stage kernels and the fused kernels read besides the G-buffer.
struct ModelDesc {
  GridDesc grid;
  const float* wpack;          // WPACK_FLOATS, device
  const uint8_t* wbf16;        // WBF16_BYTES, device
  uint32_t* status;            // device status word (timeouts, bounds)
  const float4* env;           // [env_h][env_w]
  int env_h, env_w;
  int lf;                      // L * F
  int lfp;                     // lf rounded up to a multiple of 8
  int N, M;
  float near_t, far_t, f0;
  float force_vis, force_vis2;
  int hard;                    // 1: hard visibility (RT_VIS_HARD)
  int mis;                     // 1: MIS primary directions (RT_SAMPLE_MIS)
  const float* cdf_m;          // [env_h + 1] marginal CDF of the bound map's texel distribution
  const float* cdf_c;          // [env_h][env_w + 1] conditional CDFs
  const int* guide_m;          // [1 << gm_shift] cutpoints of cdf_m: the search's start for u in [j, j + 1) / 2^gm_shift
  const int* guide_c;          // [env_h][1 << gc_shift] cutpoints of each conditional CDF
  int gm_shift, gc_shift;
  int lambert;
  int dpt;                     // BF16 soft-visibility tile shape: directions of a pixel per 128-row tile (32, 64;
                               // anything else: tiles of 128 consecutive samples)
  uint64_t seed;
};

// FP32 biases and output layers of both MLPs, passed to the BF16 kernel by
// value as a kernel parameter (constant bank) so that its epilogues read them
// without shared-memory traffic.  Filled on the host by rt_set_params.  The
// output layers are read as float2 pairs, hence the 8-byte alignment.
struct alignas(16) HeadParams {
  float ib3[2], bb3[8];
  float iw3[64][2];             // I's output layer, [hidden][output]
  float bw3[64][8];             // B's output layer, [hidden][output] (column 7 zero)
  float iw3v[64];               // I's visibility row, contiguous
};
static_assert(offsetof(HeadParams, iw3) % 8 == 0 && offsetof(HeadParams, bw3) % 8 == 0 &&
                  offsetof(HeadParams, iw3v) % 8 == 0,
              "float2 reads of the output layers");

// Launch helpers implemented in the .cu files.
// One-time per-device kernel attributes (large dynamic shared memory); called by rt_create.
cudaError_t prepare_kernels();
cudaError_t launch_repack(const float* brdf_w, const float* irt_w, int lf, float* wpack, cudaStream_t s);
cudaError_t launch_encode(const ModelDesc& m, const float4* pos, int P, float* feat, uint32_t* idx,
                          float* w, cudaStream_t s);
cudaError_t launch_decode(const ModelDesc& m, const float* feat, int P, float* brdf, cudaStream_t s);
cudaError_t launch_trace(const ModelDesc& m, const float* feat, const float4* dirs, int P, int K,
                         float* vis, float* depth, int num_sms, cudaStream_t s);
cudaError_t launch_sample(const ModelDesc& m, const float4* normal, int P, int level, long long offset,
                          float4* dirs, cudaStream_t s);
cudaError_t launch_shade(const ModelDesc& m, const rt_gbuffer& pts, int P, int level, long long offset,
                         const float* vis, const float4* lin, float4* out, cudaStream_t s);
cudaError_t launch_repack_bf16(const float* wpack, uint8_t* wbf16, cudaStream_t s);
// the direction-chunk tile shapes (m.dpt 32 / 64), soft visibility, one launch of nl lights
cudaError_t prepare_render_bf16_chunked();
cudaError_t launch_render_bf16_chunked(int nl, int wg, const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb,
                                       int P, long long offset, const float4* envs, float4* out, int num_sms,
                                       cudaStream_t s);
cudaError_t launch_render_bf16_lights(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P,
                                      long long offset, const float4* envs, int E, float4* out, int num_sms,
                                      int max_nl, int wg, cudaStream_t s);
// Status-word codes: (kStatusTimeout | where) after a bounded wait gave up.
constexpr uint32_t kStatusTimeout = 1u << 28;
constexpr uint32_t kWhereSelftest = 0xFu;   // the wait of rt_selftest_wait
cudaError_t launch_wait_never(uint32_t* status, uint64_t limit_ns, cudaStream_t s);
cudaError_t launch_render_fp32(const ModelDesc& m, const rt_gbuffer& gb, int P, long long offset,
                               float4* out, int num_sms, cudaStream_t s);
cudaError_t prepare_distill();
cudaError_t launch_distill_dirs(int P, int K, long long ray_offset, uint64_t seed, float4* dirs, cudaStream_t s);
cudaError_t launch_distill_fp32(const ModelDesc& m, const float4* pos, const float4* nrm, int P, int K,
                                const float4* dirs, const float* brdf_t, const float* vis_t, const float* depth_t,
                                float* loss, float* g_table, float* g_brdf, float* g_irt, int num_sms, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m1, float* m2, long long n, float lr, float b1, float b2,
                        float eps, float wd, float bc1, float bc2, int num_sms, cudaStream_t s);
cudaError_t launch_env_cdf(const float4* env, int H, int W, float* cdf_m, float* cdf_c, int* guide_m, int gm_shift,
                           int* guide_c, int gc_shift, cudaStream_t s);
// smallest s with 2^s >= n (n >= 1): the cutpoint tables have 2^s entries
inline int guide_shift(int n) {
  int s = 0;
  while ((1 << s) < n) ++s;
  return s;
}
cudaError_t launch_denoise(int W, int H, const float4* rad, const float* z, const float4* nrm, int iterations,
                           float sigma_z, float sigma_n, float sigma_l, float4* work, float4* out, cudaStream_t s);
cudaError_t prepare_backward_bf16();
cudaError_t launch_backward_bf16(const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb, int P, long long offset,
                                 const float4* dL, float* g_table, float* g_brdf, float* g_irt, int num_sms,
                                 cudaStream_t s);
cudaError_t launch_backward_fp32(const ModelDesc& m, const rt_gbuffer& gb, int P, long long offset,
                                 const float4* dL, float* g_table, float* g_brdf, float* g_irt, int num_sms,
                                 cudaStream_t s);

}  // namespace rtk
