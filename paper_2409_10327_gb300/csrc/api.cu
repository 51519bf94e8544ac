// Host side of the C ABI declared in include/rt.h: validation, the context,
// and the launches.  No entry point allocates except rt_create.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <atomic>
#include <new>

#include "rt_internal.h"

using namespace rtk;

struct rt_ctx {
  rt_config cfg;
  int device;
  int num_sms;
  int res[kMaxLevels];
  int dense[kMaxLevels];
  float* wpack;        // WPACK_FLOATS
  uint8_t* wbf16;      // WBF16_BYTES
  uint32_t* status;    // device status word
  float* cdf;          // MIS texel CDFs: marginal [env_h + 1], then conditional [env_h][env_w + 1],
                       // then the int cutpoint tables [2^gm_shift] and [env_h][2^gc_shift]
  const void* table;
  const float* env;
  HeadParams head;     // host copy of the FP32 output layers (BF16 kernel parameter)
  bool ready;
  int tuned_nl;        // lights per launch of the BF16 kernel (rt_tune), default 8
  int tuned_wg;        // warpgroups per CTA of the BF16 kernel (rt_tune), default 4
  int tuned_dpt;       // directions of a pixel per 128-row tile of the BF16 kernel (rt_tune), default 128
};

namespace {

constexpr int64_t kMaxP = 2147483647LL;

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int level_res(const rt_config* c, int l) {
  if (c->levels == 1) return c->base_res;
  const double b = std::exp((std::log((double)c->max_res) - std::log((double)c->base_res)) / (c->levels - 1));
  return (int)std::floor((double)c->base_res * std::pow(b, (double)l) + 1e-9);
}

bool level_dense(const rt_config* c, int res) {
  if (!c->dense_coarse) return false;
  const double n1 = (double)res + 1.0;
  return n1 * n1 * n1 <= (double)(1LL << c->log2_T);
}

int64_t cdf_floats(const rt_config& c) { return (int64_t)(c.env_h + 1) + (int64_t)c.env_h * (c.env_w + 1); }
int64_t cdf_words(const rt_config& c) {
  return cdf_floats(c) + (1LL << guide_shift(c.env_h)) + (int64_t)c.env_h * (1LL << guide_shift(c.env_w));
}
int* guide_m_of(float* cdf, const rt_config& c) { return reinterpret_cast<int*>(cdf + cdf_floats(c)); }
int* guide_c_of(float* cdf, const rt_config& c) { return guide_m_of(cdf, c) + (1 << guide_shift(c.env_h)); }

ModelDesc model_desc(const rt_ctx* ctx) {
  ModelDesc m{};
  const rt_config& c = ctx->cfg;
  m.grid.levels = c.levels;
  m.grid.log2T = c.log2_T;
  m.grid.mask = (uint32_t)((1ULL << c.log2_T) - 1ULL);
  m.grid.half = c.precision == RT_BF16 ? 1 : 0;
  m.grid.table = ctx->table;
  for (int l = 0; l < kMaxLevels; ++l) {
    m.grid.res[l] = l < c.levels ? ctx->res[l] : 1;
    m.grid.dense[l] = l < c.levels ? ctx->dense[l] : 0;
  }
  m.wpack = ctx->wpack;
  m.wbf16 = ctx->wbf16;
  m.status = ctx->status;
  m.env = reinterpret_cast<const float4*>(ctx->env);
  m.env_h = c.env_h;
  m.env_w = c.env_w;
  m.lf = c.levels * c.feat_dim;
  m.lfp = (m.lf + 7) / 8 * 8;
  m.N = c.n_dirs;
  m.M = c.m_dirs;
  m.near_t = c.near_t;
  m.far_t = c.far_t;
  m.f0 = c.f0;
  m.force_vis = c.force_vis;
  m.force_vis2 = c.force_vis2;
  m.hard = c.visibility == RT_VIS_HARD ? 1 : 0;
  m.mis = c.sampling == RT_SAMPLE_MIS ? 1 : 0;
  m.cdf_m = ctx->cdf;
  m.cdf_c = ctx->cdf + (c.env_h + 1);
  m.guide_m = guide_m_of(ctx->cdf, c);
  m.guide_c = guide_c_of(ctx->cdf, c);
  m.gm_shift = guide_shift(c.env_h);
  m.gc_shift = guide_shift(c.env_w);
  m.lambert = c.brdf_mode == RT_LAMBERT;
  m.dpt = ctx->tuned_dpt;
  m.seed = c.dir_seed;
  return m;
}

rt_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RT_OK : RT_ERR_CUDA; }

// Host-side fault injection (rt_debug_fail_alloc): the number of workspace
// allocations still to go before one fails; 0 = armed for none.
std::atomic<int> g_fail_alloc{0};

// cudaMalloc of rt_create's workspace, failing on request as if the device
// were out of memory.
cudaError_t ws_malloc(void** p, size_t bytes) {
  int n = g_fail_alloc.load();
  while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

rt_status check_ctx(const rt_ctx* ctx) {
  if (ctx == nullptr) return RT_ERR_INVALID_ARG;
  if (!ctx->ready) return RT_ERR_NOT_READY;
  return RT_OK;
}

bool check_plane(const float* p) { return p != nullptr && aligned(p, 16); }

bool check_gbuffer(const rt_gbuffer* gb) {
  return gb != nullptr && check_plane(gb->pos) && check_plane(gb->normal) && check_plane(gb->view) &&
         check_plane(gb->albedo_rough);
}

}  // namespace

extern "C" {

const char* rt_status_str(rt_status s) {
  switch (s) {
    case RT_OK: return "RT_OK";
    case RT_ERR_INVALID_ARG: return "RT_ERR_INVALID_ARG";
    case RT_ERR_UNSUPPORTED: return "RT_ERR_UNSUPPORTED";
    case RT_ERR_OOM: return "RT_ERR_OOM";
    case RT_ERR_CUDA: return "RT_ERR_CUDA";
    case RT_ERR_TIMEOUT: return "RT_ERR_TIMEOUT";
    case RT_ERR_BOUNDS: return "RT_ERR_BOUNDS";
    case RT_ERR_NOT_READY: return "RT_ERR_NOT_READY";
  }
  return "RT_ERR_UNKNOWN";
}

rt_status rt_config_default(rt_config* c) {
  if (c == nullptr) return RT_ERR_INVALID_ARG;
  c->levels = 16;
  c->feat_dim = 2;
  c->log2_T = 19;
  c->base_res = 16;
  c->max_res = 2048;
  c->dense_coarse = 1;
  c->precision = RT_FP32;
  c->n_dirs = 128;
  c->m_dirs = 8;
  c->brdf_mode = RT_DISNEY;
  c->near_t = 0.05f;
  c->far_t = 1.5f;
  c->f0 = 0.04f;
  c->force_vis = -1.0f;
  c->force_vis2 = -1.0f;
  c->visibility = RT_VIS_SOFT;
  c->sampling = RT_SAMPLE_COSINE;
  c->env_h = 64;
  c->env_w = 128;
  c->dir_seed = 0x5EED;
  return RT_OK;
}

rt_status rt_config_validate(const rt_config* c) {
  if (c == nullptr) return RT_ERR_INVALID_ARG;
  const bool ok = c->levels >= 1 && c->levels <= kMaxLevels && c->feat_dim == 2 && c->log2_T >= 8 &&
                  c->log2_T <= 24 && c->base_res >= 2 && c->max_res >= c->base_res && c->max_res <= (1 << 20) &&
                  (c->dense_coarse == 0 || c->dense_coarse == 1) &&
                  (c->precision == RT_FP32 || c->precision == RT_BF16) && c->n_dirs >= 1 && c->n_dirs <= 4096 &&
                  c->m_dirs >= 1 && c->m_dirs <= 64 && (c->brdf_mode == RT_DISNEY || c->brdf_mode == RT_LAMBERT) &&
                  std::isfinite(c->near_t) && std::isfinite(c->far_t) && c->near_t >= 0.0f &&
                  c->far_t > c->near_t && std::isfinite(c->f0) && c->f0 >= 0.0f && c->f0 <= 1.0f &&
                  !std::isnan(c->force_vis) && c->force_vis <= 1.0f && !std::isnan(c->force_vis2) &&
                  c->force_vis2 <= 1.0f && (c->visibility == RT_VIS_SOFT || c->visibility == RT_VIS_HARD) &&
                  (c->sampling == RT_SAMPLE_COSINE || c->sampling == RT_SAMPLE_MIS) &&
                  c->env_h >= 1 && c->env_h <= 8192 && c->env_w >= 1 &&
                  c->env_w <= 8192;
  return ok ? RT_OK : RT_ERR_INVALID_ARG;
}

int32_t rt_level_resolution(const rt_config* c, int32_t level) {
  if (rt_config_validate(c) != RT_OK || level < 0 || level >= c->levels) return -1;
  return level_res(c, level);
}

int32_t rt_level_is_dense(const rt_config* c, int32_t level) {
  if (rt_config_validate(c) != RT_OK || level < 0 || level >= c->levels) return -1;
  return level_dense(c, level_res(c, level)) ? 1 : 0;
}

int64_t rt_param_count(const rt_config* c, int32_t which) {
  if (rt_config_validate(c) != RT_OK) return -1;
  const int64_t lf = (int64_t)c->levels * c->feat_dim;
  auto mlp = [](int64_t in, int64_t out) { return in * 64 + 64 + 64 * 64 + 64 + 64 * out + out; };
  switch (which) {
    case 0: return (int64_t)c->levels * (1LL << c->log2_T) * c->feat_dim;
    case 1: return mlp(lf, kBrdfOut);
    case 2: return mlp(lf + kPE, kIrtOut);
  }
  return -1;
}

int64_t rt_workspace_bytes(const rt_config* c) {
  if (rt_config_validate(c) != RT_OK) return -1;
  return (int64_t)WPACK_FLOATS * 4 + WBF16_BYTES + 256 + cdf_words(*c) * 4;
}

rt_status rt_create(const rt_config* cfg, rt_ctx** out) {
  // (the MIS texel CDFs are allocated with the rest of the workspace, whatever the sampling mode)
  if (out == nullptr) return RT_ERR_INVALID_ARG;
  *out = nullptr;
  if (rt_config_validate(cfg) != RT_OK) return RT_ERR_INVALID_ARG;
  rt_ctx* ctx = new (std::nothrow) rt_ctx{};
  if (ctx == nullptr) return RT_ERR_OOM;
  ctx->cfg = *cfg;
  ctx->tuned_nl = 8;
  ctx->tuned_wg = 4;
  ctx->tuned_dpt = 128;
  for (int l = 0; l < cfg->levels; ++l) {
    ctx->res[l] = level_res(cfg, l);
    ctx->dense[l] = level_dense(cfg, ctx->res[l]) ? 1 : 0;
  }
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    delete ctx;
    return RT_ERR_CUDA;
  }
  if (ws_malloc((void**)&ctx->wpack, (size_t)WPACK_FLOATS * 4) != cudaSuccess) {
    delete ctx;
    return RT_ERR_OOM;
  }
  if (ws_malloc((void**)&ctx->wbf16, (size_t)WBF16_BYTES) != cudaSuccess) {
    cudaFree(ctx->wpack);
    delete ctx;
    return RT_ERR_OOM;
  }
  if (ws_malloc((void**)&ctx->status, 256) != cudaSuccess || cudaMemset(ctx->status, 0, 256) != cudaSuccess) {
    cudaFree(ctx->wpack);
    cudaFree(ctx->wbf16);
    delete ctx;
    return RT_ERR_OOM;
  }
  if (ws_malloc((void**)&ctx->cdf, (size_t)cdf_words(*cfg) * 4) != cudaSuccess) {
    cudaFree(ctx->wpack);
    cudaFree(ctx->wbf16);
    cudaFree(ctx->status);
    delete ctx;
    return RT_ERR_OOM;
  }
  cudaError_t e = rtk::prepare_kernels();
  if (e != cudaSuccess) {
    cudaFree(ctx->wpack);
    cudaFree(ctx->wbf16);
    cudaFree(ctx->status);
    cudaFree(ctx->cdf);
    delete ctx;
    return RT_ERR_CUDA;
  }
  *out = ctx;
  return RT_OK;
}

rt_status rt_destroy(rt_ctx* ctx) {
  if (ctx == nullptr) return RT_OK;
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(ctx->wpack);
  cudaFree(ctx->wbf16);
  cudaFree(ctx->status);
  cudaFree(ctx->cdf);
  delete ctx;
  return cuda_status(e);
}

rt_status rt_set_params(rt_ctx* ctx, const void* table, const float* brdf_w, const float* irt_w, const float* env,
                        void* stream) {
  if (ctx == nullptr || table == nullptr || brdf_w == nullptr || irt_w == nullptr || env == nullptr)
    return RT_ERR_INVALID_ARG;
  const uintptr_t ta = 8;   // the BF16 kernel reads pairs of FP16 entries as one 8-byte load
  if (!aligned(table, ta) || !aligned(brdf_w, 4) || !aligned(irt_w, 4) || !aligned(env, 16))
    return RT_ERR_INVALID_ARG;
  ctx->table = table;
  ctx->env = env;
  const int lf = ctx->cfg.levels * ctx->cfg.feat_dim;
  cudaStream_t s = (cudaStream_t)stream;
  rt_status st = cuda_status(launch_repack(brdf_w, irt_w, lf, ctx->wpack, s));
  if (st == RT_OK)
    st = cuda_status(launch_env_cdf(reinterpret_cast<const float4*>(env), ctx->cfg.env_h, ctx->cfg.env_w, ctx->cdf,
                                    ctx->cdf + (ctx->cfg.env_h + 1), guide_m_of(ctx->cdf, ctx->cfg),
                                    guide_shift(ctx->cfg.env_h), guide_c_of(ctx->cdf, ctx->cfg),
                                    guide_shift(ctx->cfg.env_w), s));
  if (st == RT_OK) st = cuda_status(launch_repack_bf16(ctx->wpack, ctx->wbf16, s));
  if (st != RT_OK) return st;
  // host copy of the output layers for the BF16 kernel's parameters
  static thread_local float host[WPACK_FLOATS];
  if (cudaMemcpyAsync(host, ctx->wpack, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RT_ERR_CUDA;
  HeadParams& h = ctx->head;
  for (int i = 0; i < 64; ++i) {
    h.iw3[i][0] = host[OFF_IW3 + 2 * i];
    h.iw3[i][1] = host[OFF_IW3 + 2 * i + 1];
    h.iw3v[i] = host[OFF_IW3 + 2 * i];
    for (int o = 0; o < 8; ++o) h.bw3[i][o] = host[OFF_BW3 + 8 * i + o];
  }
  h.ib3[0] = host[OFF_IB3];
  h.ib3[1] = host[OFF_IB3 + 1];
  for (int o = 0; o < 8; ++o) h.bb3[o] = host[OFF_BB3 + o];
  ctx->ready = true;
  return RT_OK;
}

rt_status rt_selftest_wait(rt_ctx* ctx, int64_t limit_ns, void* stream) {
  if (ctx == nullptr) return RT_ERR_INVALID_ARG;
  const int64_t lim = limit_ns < 1000000 ? 1000000 : (limit_ns > 2000000000 ? 2000000000 : limit_ns);
  return cuda_status(launch_wait_never(ctx->status, (uint64_t)lim, (cudaStream_t)stream));
}

rt_status rt_debug_fail_alloc(int32_t n) {
  if (n < 0) return RT_ERR_INVALID_ARG;
  g_fail_alloc.store(n);
  return RT_OK;
}

rt_status rt_check(rt_ctx* ctx, uint32_t* word, void* stream) {
  if (ctx == nullptr || word == nullptr) return RT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h = 0;
  if (cudaMemcpyAsync(&h, ctx->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return RT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RT_ERR_CUDA;
  if (cudaMemsetAsync(ctx->status, 0, 4, s) != cudaSuccess) return RT_ERR_CUDA;
  *word = h;
  if (h == 0) return RT_OK;
  return (h >> 28) == 1 ? RT_ERR_TIMEOUT : RT_ERR_BOUNDS;
}

rt_status rt_encode(rt_ctx* ctx, const float* pos, int64_t P, float* feat, uint32_t* idx, float* w, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP) return RT_ERR_INVALID_ARG;
  if (P == 0) return RT_OK;
  if (!check_plane(pos) || feat == nullptr || !aligned(feat, 4) || (idx != nullptr && !aligned(idx, 4)) ||
      (w != nullptr && !aligned(w, 4)))
    return RT_ERR_INVALID_ARG;
  return cuda_status(launch_encode(model_desc(ctx), reinterpret_cast<const float4*>(pos), (int)P, feat, idx, w,
                                   (cudaStream_t)stream));
}

rt_status rt_decode(rt_ctx* ctx, const float* feat, int64_t P, float* brdf, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP) return RT_ERR_INVALID_ARG;
  if (P == 0) return RT_OK;
  if (feat == nullptr || !aligned(feat, 4) || brdf == nullptr || !aligned(brdf, 16)) return RT_ERR_INVALID_ARG;
  return cuda_status(launch_decode(model_desc(ctx), feat, (int)P, brdf, (cudaStream_t)stream));
}

rt_status rt_trace(rt_ctx* ctx, const float* feat, const float* dirs, int64_t P, int32_t K, float* vis,
                   float* depth, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP || K < 1 || K > 4096) return RT_ERR_INVALID_ARG;
  if (P == 0) return RT_OK;
  if (feat == nullptr || !aligned(feat, 4) || !check_plane(dirs) || vis == nullptr || !aligned(vis, 4) ||
      depth == nullptr || !aligned(depth, 4))
    return RT_ERR_INVALID_ARG;
  return cuda_status(launch_trace(model_desc(ctx), feat, reinterpret_cast<const float4*>(dirs), (int)P, K, vis,
                                  depth, ctx->num_sms, (cudaStream_t)stream));
}

rt_status rt_sample(rt_ctx* ctx, const float* normal, int64_t P, int32_t level, int64_t index_offset, float* dirs,
                    void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP || (level != 0 && level != 1) || index_offset < 0) return RT_ERR_INVALID_ARG;
  if (level == 0 && ctx->cfg.sampling == RT_SAMPLE_MIS) return RT_ERR_UNSUPPORTED;
  if (P == 0) return RT_OK;
  if (!check_plane(normal) || !check_plane(dirs)) return RT_ERR_INVALID_ARG;
  return cuda_status(launch_sample(model_desc(ctx), reinterpret_cast<const float4*>(normal), (int)P, level,
                                   index_offset, reinterpret_cast<float4*>(dirs), (cudaStream_t)stream));
}

rt_status rt_shade(rt_ctx* ctx, const rt_gbuffer* pts, int64_t P, int32_t level, int64_t index_offset,
                   const float* vis, const float* lin, float* out, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP || (level != 0 && level != 1) || index_offset < 0) return RT_ERR_INVALID_ARG;
  if (level == 0 && ctx->cfg.sampling == RT_SAMPLE_MIS) return RT_ERR_UNSUPPORTED;
  if (P == 0) return RT_OK;
  if (pts == nullptr || !check_plane(pts->normal) || !check_plane(pts->view) || !check_plane(pts->albedo_rough) ||
      vis == nullptr || !aligned(vis, 4) || (lin != nullptr && (level == 1 || !aligned(lin, 16))) ||
      !check_plane(out))
    return RT_ERR_INVALID_ARG;
  return cuda_status(launch_shade(model_desc(ctx), *pts, (int)P, level, index_offset, vis,
                                  reinterpret_cast<const float4*>(lin), reinterpret_cast<float4*>(out),
                                  (cudaStream_t)stream));
}

rt_status rt_render_frame(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset, float* radiance,
                          void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP || pixel_offset < 0) return RT_ERR_INVALID_ARG;
  if (P == 0) return RT_OK;
  if (!check_gbuffer(gb) || !check_plane(radiance)) return RT_ERR_INVALID_ARG;
  const ModelDesc m = model_desc(ctx);
  if (ctx->cfg.precision == RT_FP32)
    return cuda_status(launch_render_fp32(m, *gb, (int)P, pixel_offset, reinterpret_cast<float4*>(radiance),
                                          ctx->num_sms, (cudaStream_t)stream));
  if (ctx->cfg.n_dirs < 4) return RT_ERR_UNSUPPORTED;   // the BF16 tile holds at most 33 pixels
  return cuda_status(launch_render_bf16_lights(m, ctx->head, *gb, (int)P, pixel_offset, m.env, 1,
                                               reinterpret_cast<float4*>(radiance), ctx->num_sms, 1, ctx->tuned_wg,
                                               (cudaStream_t)stream));
}

rt_status rt_render_frame_multi(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset,
                                const float* envs, int32_t E, float* radiance, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP || pixel_offset < 0 || E < 0 || E > 1024 || P * (int64_t)E > (int64_t)1 << 40)
    return RT_ERR_INVALID_ARG;
  if (P == 0 || E == 0) return RT_OK;
  if (!check_gbuffer(gb) || !check_plane(envs) || !check_plane(radiance)) return RT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const ModelDesc m = model_desc(ctx);
  const float4* env4 = reinterpret_cast<const float4*>(envs);
  float4* out4 = reinterpret_cast<float4*>(radiance);
  if (ctx->cfg.precision == RT_BF16) {
    if (ctx->cfg.n_dirs < 4) return RT_ERR_UNSUPPORTED;
    return cuda_status(launch_render_bf16_lights(m, ctx->head, *gb, (int)P, pixel_offset, env4, E, out4,
                                                 ctx->num_sms, ctx->tuned_nl, ctx->tuned_wg, s));
  }
  // FP32: one full pass per light
  const int64_t hw = (int64_t)ctx->cfg.env_h * ctx->cfg.env_w;
  for (int e = 0; e < E; ++e) {
    ModelDesc me = m;
    me.env = env4 + e * hw;
    st = cuda_status(launch_render_fp32(me, *gb, (int)P, pixel_offset, out4 + e * P, ctx->num_sms, s));
    if (st != RT_OK) return st;
  }
  return RT_OK;
}

rt_status rt_tune(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset, const float* envs, int32_t E,
                  float* radiance, void* stream, float* best_ms) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P <= 0 || P > kMaxP || E <= 0 || E > 1024 || pixel_offset < 0 || !check_gbuffer(gb) || !check_plane(envs) ||
      !check_plane(radiance))
    return RT_ERR_INVALID_ARG;
  if (ctx->cfg.precision != RT_BF16) {
    if (best_ms) *best_ms = -1.0f;
    return RT_OK;   // the FP32 path has a single launch shape
  }
  if (ctx->cfg.n_dirs < 4) return RT_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RT_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RT_ERR_CUDA;
  }
  ModelDesc m = model_desc(ctx);
  const float4* env4 = reinterpret_cast<const float4*>(envs);
  float4* out4 = reinterpret_cast<float4*>(radiance);
  float best = 3.0e38f;
  int best_nl = ctx->tuned_nl, best_wg = ctx->tuned_wg, best_dpt = ctx->tuned_dpt;
  st = RT_OK;
  const int N = ctx->cfg.n_dirs;
  for (int dpt = 128; dpt >= 32 && st == RT_OK; dpt /= 2) {
    // a tile of 128 / dpt pixels x dpt directions; other shapes repeat the consecutive order
    if (dpt < 128 && (ctx->cfg.visibility == RT_VIS_HARD || N % dpt != 0 || N <= dpt)) continue;
    m.dpt = dpt;
    for (int wg = ctx->cfg.visibility == RT_VIS_HARD ? 4 : 2; wg <= 4 && st == RT_OK; ++wg) {
      for (int nl = 1; nl <= 8 && st == RT_OK; nl *= 2) {
        if (nl > 1 && nl / 2 >= E) break;   // wider launches than E lights repeat the previous shape
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && st == RT_OK; ++rep) {   // rep 0 warms up
          if (cudaEventRecord(e0, s) != cudaSuccess ||
              launch_render_bf16_lights(m, ctx->head, *gb, (int)P, pixel_offset, env4, E, out4, ctx->num_sms, nl,
                                        wg, s) != cudaSuccess ||
              cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = RT_ERR_CUDA;
        }
        if (st == RT_OK && ms < best) {
          best = ms;
          best_nl = nl;
          best_wg = wg;
          best_dpt = dpt;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RT_OK) return st;
  ctx->tuned_nl = best_nl;
  ctx->tuned_wg = best_wg;
  ctx->tuned_dpt = best_dpt;
  if (best_ms) *best_ms = best;
  return RT_OK;
}

rt_status rt_tuned_shape(const rt_ctx* ctx, int32_t* lights_per_launch, int32_t* warpgroups) {
  if (ctx == nullptr || lights_per_launch == nullptr || warpgroups == nullptr) return RT_ERR_INVALID_ARG;
  *lights_per_launch = ctx->tuned_nl;
  *warpgroups = ctx->tuned_wg;
  return RT_OK;
}

rt_status rt_set_launch_shape(rt_ctx* ctx, int32_t lights_per_launch, int32_t warpgroups) {
  if (ctx == nullptr) return RT_ERR_INVALID_ARG;
  const int nl = lights_per_launch;
  if (!(nl == 1 || nl == 2 || nl == 4 || nl == 8) || warpgroups < 2 || warpgroups > 4) return RT_ERR_INVALID_ARG;
  ctx->tuned_nl = nl;
  ctx->tuned_wg = warpgroups;
  return RT_OK;
}

rt_status rt_tuned_tile_shape(const rt_ctx* ctx, int32_t* dirs_per_tile) {
  if (ctx == nullptr || dirs_per_tile == nullptr) return RT_ERR_INVALID_ARG;
  *dirs_per_tile = ctx->tuned_dpt;
  return RT_OK;
}

rt_status rt_set_tile_shape(rt_ctx* ctx, int32_t dirs_per_tile) {
  if (ctx == nullptr || !(dirs_per_tile == 32 || dirs_per_tile == 64 || dirs_per_tile == 128))
    return RT_ERR_INVALID_ARG;
  ctx->tuned_dpt = dirs_per_tile;
  return RT_OK;
}

rt_status rt_backward(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset, const float* d_radiance,
                      float* g_table, float* g_brdf, float* g_irt, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || P > kMaxP || pixel_offset < 0) return RT_ERR_INVALID_ARG;
  if (ctx->cfg.visibility == RT_VIS_HARD) return RT_ERR_UNSUPPORTED;
  if (P == 0) return RT_OK;
  if (!check_gbuffer(gb) || !check_plane(d_radiance) || g_table == nullptr || !aligned(g_table, 8) ||
      g_brdf == nullptr || !aligned(g_brdf, 4) || g_irt == nullptr || !aligned(g_irt, 4))
    return RT_ERR_INVALID_ARG;
  if (ctx->cfg.precision == RT_BF16) {
    if (ctx->cfg.n_dirs < 4) return RT_ERR_UNSUPPORTED;   // as the BF16 render: a tile spans at most 34 pixels
    return cuda_status(launch_backward_bf16(model_desc(ctx), ctx->head, *gb, (int)P, pixel_offset,
                                            reinterpret_cast<const float4*>(d_radiance), g_table, g_brdf, g_irt,
                                            ctx->num_sms, (cudaStream_t)stream));
  }
  return cuda_status(launch_backward_fp32(model_desc(ctx), *gb, (int)P, pixel_offset,
                                          reinterpret_cast<const float4*>(d_radiance), g_table, g_brdf, g_irt,
                                          ctx->num_sms, (cudaStream_t)stream));
}

}  // extern "C"

rt_status rt_denoise(int32_t width, int32_t height, const float* radiance, const float* depth, const float* normal,
                     int32_t iterations, float sigma_z, float sigma_n, float sigma_l, float* work, float* out,
                     void* stream) {
  if (width < 1 || height < 1 || (int64_t)width * height > kMaxP || iterations < 0 || iterations > 12)
    return RT_ERR_INVALID_ARG;
  if (!std::isfinite(sigma_z) || !std::isfinite(sigma_n) || !std::isfinite(sigma_l) || !(sigma_z > 0.0f) ||
      !(sigma_l > 0.0f) || !(sigma_n >= 0.0f))
    return RT_ERR_INVALID_ARG;
  if (!check_plane(radiance) || depth == nullptr || !aligned(depth, 4) || !check_plane(normal) ||
      !check_plane(work) || !check_plane(out))
    return RT_ERR_INVALID_ARG;
  const int64_t bytes = (int64_t)width * height * 16;
  auto overlap = [&](const float* a, const float* b) {
    const char* x = reinterpret_cast<const char*>(a);
    const char* y = reinterpret_cast<const char*>(b);
    return x < y + bytes && y < x + bytes;
  };
  if (overlap(radiance, work) || overlap(radiance, out) || overlap(work, out)) return RT_ERR_INVALID_ARG;
  return cuda_status(launch_denoise(width, height, reinterpret_cast<const float4*>(radiance), depth,
                                    reinterpret_cast<const float4*>(normal), iterations, sigma_z, sigma_n, sigma_l,
                                    reinterpret_cast<float4*>(work), reinterpret_cast<float4*>(out),
                                    (cudaStream_t)stream));
}

rt_status rt_distill_dirs(rt_ctx* ctx, int64_t P, int32_t K, int64_t ray_offset, float* dirs, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  int32_t S = 1;
  while ((S + 1) * (S + 1) <= K) ++S;
  if (P < 0 || K < 1 || K > 65536 || S * S != K || P * (int64_t)K > kMaxP || ray_offset < 0)
    return RT_ERR_INVALID_ARG;
  if (P == 0) return RT_OK;
  if (!check_plane(dirs)) return RT_ERR_INVALID_ARG;
  return cuda_status(launch_distill_dirs((int)P, K, ray_offset, ctx->cfg.dir_seed, reinterpret_cast<float4*>(dirs),
                                         (cudaStream_t)stream));
}

rt_status rt_distill_backward(rt_ctx* ctx, const float* pos, const float* normal, int64_t P, int32_t K,
                              const float* dirs, const float* brdf_t, const float* vis_t, const float* depth_t,
                              float* loss, float* g_table, float* g_brdf, float* g_irt, void* stream) {
  rt_status st = check_ctx(ctx);
  if (st != RT_OK) return st;
  if (P < 0 || K < 1 || K > 65536 || P * (int64_t)K > kMaxP) return RT_ERR_INVALID_ARG;
  if (ctx->cfg.precision != RT_FP32) return RT_ERR_UNSUPPORTED;
  if (P == 0) return RT_OK;
  if (!check_plane(pos) || !check_plane(normal) || !check_plane(dirs) || brdf_t == nullptr || !aligned(brdf_t, 4) ||
      vis_t == nullptr || !aligned(vis_t, 4) || depth_t == nullptr || !aligned(depth_t, 4) ||
      (loss != nullptr && !aligned(loss, 4)) || g_table == nullptr || !aligned(g_table, 8) || g_brdf == nullptr ||
      !aligned(g_brdf, 4) || g_irt == nullptr || !aligned(g_irt, 4))
    return RT_ERR_INVALID_ARG;
  return cuda_status(launch_distill_fp32(model_desc(ctx), reinterpret_cast<const float4*>(pos),
                                         reinterpret_cast<const float4*>(normal), (int)P, K,
                                         reinterpret_cast<const float4*>(dirs), brdf_t, vis_t, depth_t, loss, g_table,
                                         g_brdf, g_irt, ctx->num_sms, (cudaStream_t)stream));
}

rt_status rt_adam_step(float* param, const float* grad, float* m1, float* m2, int64_t n, float lr, float beta1,
                       float beta2, float eps, float weight_decay, int32_t step, void* stream) {
  if (n < 0 || step < 1 || !std::isfinite(lr) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
      !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f) || !std::isfinite(weight_decay))
    return RT_ERR_INVALID_ARG;
  if (n == 0) return RT_OK;
  if (param == nullptr || grad == nullptr || m1 == nullptr || m2 == nullptr || !aligned(param, 4) ||
      !aligned(grad, 4) || !aligned(m1, 4) || !aligned(m2, 4))
    return RT_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RT_ERR_CUDA;
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
  return cuda_status(launch_adam(param, grad, m1, m2, n, lr, beta1, beta2, eps, weight_decay, bc1, bc2, sms,
                                 (cudaStream_t)stream));
}
