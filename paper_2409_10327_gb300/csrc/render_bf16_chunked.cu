// The direction-chunk tile shapes of the fused BF16 kernel (rt_set_tile_shape
// with 32 or 64 directions per tile, soft visibility): a second translation
// unit so that these instantiations compile beside the consecutive-sample ones.
#include "render_bf16_kernel.cuh"

namespace rtk {

cudaError_t prepare_render_bf16_chunked() {
  cudaError_t e = prepare_wg<2, false, true>();
  e = e != cudaSuccess ? e : prepare_wg<3, false, true>();
  e = e != cudaSuccess ? e : prepare_wg<4, false, true>();
  return e;
}

cudaError_t launch_render_bf16_chunked(int nl, int wg, const ModelDesc& m, const HeadParams& hp, const rt_gbuffer& gb,
                                       int P, long long offset, const float4* envs, float4* out, int num_sms,
                                       cudaStream_t s) {
  return wg == 2 ? launch_lights<2, false, true>(nl, m, hp, gb, P, offset, envs, out, num_sms, s)
       : wg == 3 ? launch_lights<3, false, true>(nl, m, hp, gb, P, offset, envs, out, num_sms, s)
                 : launch_lights<4, false, true>(nl, m, hp, gb, P, offset, envs, out, num_sms, s);
}

}  // namespace rtk
