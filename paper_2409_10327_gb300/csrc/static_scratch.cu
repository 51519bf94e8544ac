// rt_render_frame_static: the FP32 fused render without a context and without
// any device allocation.
//
// Some callers cannot call cudaMalloc: a host application whose memory
// manager owns every device allocation (a pool or arena that forbids direct
// cudaMalloc/cudaFree), or a real-time frame loop with a fixed device memory
// budget where an allocation, and the device synchronisation cudaFree
// implies, is not allowed.  rt_create allocates the packed-weight workspace
// of the fused kernel; this entry point keeps that workspace in a file-scope
// __device__ array instead, so the caller only passes its own inputs and
// output.  Every GPU that loads this library holds the array (61 KB) until
// the process exits.
#include <mutex>

#include "rt_internal.h"

namespace rtk {

// The packed FP32 weight image of rt_internal.h, shared by every call.
static __device__ __align__(256) float g_static_wpack[WPACK_FLOATS];

cudaError_t prepare_render_fp32();

namespace {

constexpr int kMaxDevices = 64;

struct DeviceSlot {
  bool ready = false;
  float* wpack = nullptr;   // device address of g_static_wpack on this device
  int num_sms = 0;
};

std::mutex g_mutex;
DeviceSlot g_slots[kMaxDevices];

// Once per device, with that device current: the array's device address (the
// host-side symbol is not a device address), the SM count and the kernel's
// shared-memory attribute.  Every call looks the address up again (a host-side
// lookup that allocates nothing): if the device's context was reset since the
// set-up (cudaDeviceReset), the array lives at a new address in the new
// context and the kernel attribute is gone, so the set-up is redone instead of
// launching through a stale pointer.
rt_status device_slot(DeviceSlot** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return RT_ERR_CUDA;
  if (dev >= kMaxDevices) return RT_ERR_UNSUPPORTED;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_wpack) != cudaSuccess || p == nullptr) return RT_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceSlot& s = g_slots[dev];
  if (!s.ready || s.wpack != static_cast<float*>(p)) {
    s.ready = false;
    if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RT_ERR_CUDA;
    if (prepare_render_fp32() != cudaSuccess) return RT_ERR_CUDA;
    s.wpack = static_cast<float*>(p);
    s.ready = true;
  }
  *out = &s;
  return RT_OK;
}

bool aligned_to(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

}  // namespace rtk

using namespace rtk;

extern "C" rt_status rt_render_frame_static(const rt_config* cfg, const void* table, const float* brdf_w,
                                            const float* irt_w, const float* env, const rt_gbuffer* gb, int64_t P,
                                            int64_t pixel_offset, float* radiance, void* stream) {
  if (rt_config_validate(cfg) != RT_OK) return RT_ERR_INVALID_ARG;
  if (cfg->precision != RT_FP32 || cfg->sampling == RT_SAMPLE_MIS) return RT_ERR_UNSUPPORTED;
  // The static array holds exactly one packed image: 2 x L features per point
  // must fit its 32 feature rows (always true for a valid config, L <= 16).
  if (cfg->levels * cfg->feat_dim > 32) return RT_ERR_INVALID_ARG;
  if (P < 0 || P > 2147483647LL || pixel_offset < 0) return RT_ERR_INVALID_ARG;
  if (P == 0) return RT_OK;
  if (table == nullptr || !aligned_to(table, 8) || brdf_w == nullptr || irt_w == nullptr || env == nullptr ||
      !aligned_to(env, 16) || gb == nullptr || radiance == nullptr || !aligned_to(radiance, 16) ||
      gb->pos == nullptr || gb->normal == nullptr || gb->view == nullptr || gb->albedo_rough == nullptr ||
      !aligned_to(gb->pos, 16) || !aligned_to(gb->normal, 16) || !aligned_to(gb->view, 16) ||
      !aligned_to(gb->albedo_rough, 16))
    return RT_ERR_INVALID_ARG;

  DeviceSlot* slot = nullptr;
  const rt_status st = device_slot(&slot);
  if (st != RT_OK) return st;

  ModelDesc m{};
  m.grid.levels = cfg->levels;
  m.grid.log2T = cfg->log2_T;
  m.grid.mask = (uint32_t)((1ULL << cfg->log2_T) - 1ULL);
  m.grid.half = 0;
  m.grid.table = table;
  for (int l = 0; l < kMaxLevels; ++l) {
    m.grid.res[l] = l < cfg->levels ? rt_level_resolution(cfg, l) : 1;
    m.grid.dense[l] = l < cfg->levels ? rt_level_is_dense(cfg, l) : 0;
  }
  m.wpack = slot->wpack;
  m.env = reinterpret_cast<const float4*>(env);
  m.env_h = cfg->env_h;
  m.env_w = cfg->env_w;
  m.lf = cfg->levels * cfg->feat_dim;
  m.lfp = (m.lf + 7) / 8 * 8;
  m.N = cfg->n_dirs;
  m.M = cfg->m_dirs;
  m.near_t = cfg->near_t;
  m.far_t = cfg->far_t;
  m.f0 = cfg->f0;
  m.force_vis = cfg->force_vis;
  m.force_vis2 = cfg->force_vis2;
  m.hard = cfg->visibility == RT_VIS_HARD ? 1 : 0;
  m.mis = 0;   // MIS needs the texel CDFs of a context: rejected above
  m.lambert = cfg->brdf_mode == RT_LAMBERT;
  m.seed = cfg->dir_seed;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The repack overwrites the whole image, so nothing needs clearing first.
  if (launch_repack(brdf_w, irt_w, m.lf, slot->wpack, s) != cudaSuccess) return RT_ERR_CUDA;
  if (launch_render_fp32(m, *gb, (int)P, pixel_offset, reinterpret_cast<float4*>(radiance), slot->num_sms, s) !=
      cudaSuccess)
    return RT_ERR_CUDA;
  return RT_OK;
}
