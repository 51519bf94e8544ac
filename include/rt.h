/*
 * rt.h -- C ABI of the GB300 hash-grid secondary-ray renderer.
 *
 * The renderer is the "hash grid-based renderer" of Baking Relightable NeRF
 * for Real-time Direct/Indirect Illumination Rendering (arXiv 2409.10327):
 * for every primary surface point x (a G-buffer texel produced upstream)
 *
 *   (a) f = H(x)                       multi-resolution hash encoding  (Sec. 3.2)
 *   (c) v_i, t_i = I(f, w_i)           implicit ray tracer MLP          (Sec. 3.2)
 *   (d) x'_i = x + t_i w_i, f'_i = H(x'_i)                              (Sec. 3.1)
 *   (b) a'_i, r'_i, n'_i = B(f'_i)     BRDF decoder MLP                 (Sec. 3.2, 3.3)
 *   (c) v'_ij = I(f'_i, w'_ij)         M directions per secondary point (suppl. "Rendering Details")
 *   (e) L'_o,i = (pi/M) sum_j v'_ij Lenv(w'_ij) f_r(a'_i, r'_i, n'_i; w'_ij, -w_i)    (Eq. 1 at x')
 *       L(x, w_i) = v_i Lenv(w_i) + (1 - v_i) L'_o,i                                (Eq. 2)
 *       L(x, w_o) = (pi/N) sum_i L(x, w_i) f_r(a, r, n; w_i, w_o)                   (Eq. 1)
 *
 * with cosine-weighted directions (so (w.n)/p(w) = pi), soft visibility,
 * the simplified Disney BRDF (GGX D with alpha = r^2, Schlick F with F0,
 * height-correlated Smith visibility; Sec. 4.1, Sec. 4.2, Sec. 5) and an
 * equirectangular environment map with bilinear texel interpolation (Sec. 2.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers owned by the caller, unless a
 *    comment says "host".  The library keeps the table and env pointers given
 *    to rt_set_params by reference: they must stay valid and unchanged while
 *    calls that read them are in flight.
 *  - float4 planes ([P][4] floats) must be 16-byte aligned; other arrays
 *    4-byte aligned.  Misaligned or NULL required pointers return
 *    RT_ERR_INVALID_ARG before anything is launched.
 *  - Every compute call is asynchronous on the caller's stream (`stream` is a
 *    cudaStream_t passed as void*; NULL = the legacy default stream), performs
 *    no allocation and no host synchronisation.  Launch failures return
 *    RT_ERR_CUDA; asynchronous device faults surface from a later CUDA call.
 *  - P = 0 is valid and launches nothing.  P is limited to 2^31 - 1.
 *  - Random directions come from SplitMix64 (Steele, Lea & Flood 2014):
 *    output k >= 1 of the generator started at state = dir_seed.  Slot c of
 *    secondary sample q (q = pixel * N + i) has counter q*(M+1) + c; slot 0 is
 *    the primary direction w_i, slot 1 + j the j-th direction at x'_i;
 *    counter k draws outputs 2k+1 and 2k+2 for (u1, u2) = top 24 bits * 2^-24.
 *    The direction is normalize(n + s), s = (2 sqrt(u1(1-u1)) cos 2pi u2,
 *    2 sqrt(u1(1-u1)) sin 2pi u2, 1 - 2 u1) uniform on the sphere.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rt_status {
  RT_OK = 0,
  RT_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or config field */
  RT_ERR_UNSUPPORTED = 2,   /* valid request this build does not implement */
  RT_ERR_OOM = 3,           /* rt_create could not allocate its workspace */
  RT_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed */
  RT_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out (status word) */
  RT_ERR_BOUNDS = 6,        /* a device-side bounds check fired (status word) */
  RT_ERR_NOT_READY = 7      /* rt_set_params has not been called */
} rt_status;

enum { RT_FP32 = 0, RT_BF16 = 1 };        /* precision                          */
enum { RT_DISNEY = 0, RT_LAMBERT = 1 };   /* brdf_mode                          */
enum { RT_VIS_SOFT = 0, RT_VIS_HARD = 1 }; /* visibility                         */
enum { RT_SAMPLE_COSINE = 0, RT_SAMPLE_MIS = 1 }; /* sampling                    */

/* Sizes and constants of one renderer instance.  Defaults: rt_config_default. */
typedef struct rt_config {
  int32_t levels;        /* L, 1..16 hash levels (paper: 14)                     */
  int32_t feat_dim;      /* F, features per entry; must be 2 (paper: 2)          */
  int32_t log2_T;        /* T = 2^log2_T entries per level, 8..24 (paper: 17)    */
  int32_t base_res;      /* N_min >= 2                                          */
  int32_t max_res;       /* N_max >= N_min, <= 2^20                             */
  int32_t dense_coarse;  /* 1: levels with (N_l+1)^3 <= T are indexed densely   */
  int32_t precision;     /* RT_FP32: float table, FP32 MLPs.
                            RT_BF16: half table, BF16 MLP operands, FP32 accum  */
  int32_t n_dirs;        /* N, directions per primary point, 1..4096           */
  int32_t m_dirs;        /* M, directions per secondary point, 1..64 (paper: 8) */
  int32_t brdf_mode;     /* RT_DISNEY or RT_LAMBERT (diffuse lobe only)         */
  float near_t, far_t;   /* depth range of I (paper: 0.05, 1.5)                 */
  float f0;              /* Schlick F0 (paper: 0.04)                            */
  float force_vis;       /* < 0: v from I; else v := force_vis  (0..1)          */
  float force_vis2;      /* < 0: v' from I; else v' := force_vis2 (0..1)        */
  int32_t visibility;    /* RT_VIS_SOFT: Eq. 2 with v = sigmoid(z0), every
                            direction bounces with weight 1 - v (differentiable).
                            RT_VIS_HARD: the paper's inference (Sec. 3.2
                            overview): v, v' = 1 when sigmoid(z0) > 0.5, else 0
                            (a forced value counts as 1 above 0.5); only shadow
                            directions bounce and only visible secondary
                            directions count.  Render calls only.              */
  int32_t sampling;      /* primary directions.  RT_SAMPLE_COSINE: cosine-weighted
                            (header conventions).  RT_SAMPLE_MIS (Sec. 4.1):
                            sample i is a light-importance draw for even i and a
                            GGX visible-normal draw (Heitz 2018, alpha = r^2) for
                            odd i (all light draws when n.w_o <= 1e-4), combined
                            with the balance heuristic: each direction weighs
                            f_r (n.w)+ L / (n_L p_L + n_G p_G).  The light draw
                            inverts float32 CDFs of the map bound by rt_set_params
                            (texel probability ~ max(0, luminance) + 1e-6, point
                            uniform in (phi, theta) inside the texel) with (u1,
                            u2).  Secondary directions stay cosine-weighted.
                            Render calls (rt_render_frame[_multi], rt_tune) and
                            rt_backward, where the draws and their weights are
                            constants of the estimator; rt_sample / rt_shade at
                            level 0 and rt_render_frame_static return
                            RT_ERR_UNSUPPORTED.
                            Multi-light renders draw from the bound map's
                            distribution for every light (unbiased for each). */
  int32_t env_h, env_w;  /* environment map size, each 1..8192                  */
  uint64_t dir_seed;     /* SplitMix64 starting state of the direction sampler  */
} rt_config;

/* Four [P][4] float planes describing primary surface points (device). */
typedef struct rt_gbuffer {
  const float* pos;           /* x.xyz, .w ignored                               */
  const float* normal;        /* unit n.xyz                                      */
  const float* view;          /* unit w_o.xyz, pointing away from the surface     */
  const float* albedo_rough;  /* albedo rgb in .xyz, roughness in .w              */
} rt_gbuffer;

typedef struct rt_ctx rt_ctx;

/* ---- host-only helpers (no GPU needed) --------------------------------- */

/* Status name, e.g. "RT_ERR_INVALID_ARG".  Never NULL. */
const char* rt_status_str(rt_status s);

/* Fill *cfg with the 800x800 workload's defaults (L=16, T=2^19, 16..2048,
 * N=128, M=8, FP32, Disney, near 0.05, far 1.5, F0 0.04, env 64x128). */
rt_status rt_config_default(rt_config* cfg);

/* RT_OK if every field is in range, else RT_ERR_INVALID_ARG. */
rt_status rt_config_validate(const rt_config* cfg);

/* Level resolution N_l = floor(N_min b^l), b = exp((ln N_max - ln N_min)/(L-1))
 * (Instant-NGP's ladder, referenced in Sec. 3.2), computed in double with a
 * 1e-9 guard; -1 for an invalid config or level. */
int32_t rt_level_resolution(const rt_config* cfg, int32_t level);

/* 1 if level l is indexed densely, 0 if hashed, -1 if invalid. */
int32_t rt_level_is_dense(const rt_config* cfg, int32_t level);

/* Float counts of the parameter blobs: which = 0 table (L*T*F entries),
 * 1 BRDF decoder B, 2 implicit ray tracer I; -1 if invalid.
 * MLP blob layout (both): W1 [64][in], b1 [64], W2 [64][64], b2 [64],
 * W3 [out][64], b3 [out]; row-major, weights as (out, in).  B: in = L*F,
 * out = 7 ([n(3), a(3), r]).  I: in = L*F + 27 ([f, PE(w)] with
 * PE(w) = [w, sin(2^k pi w), cos(2^k pi w)] for k = 0..3), out = 2. */
int64_t rt_param_count(const rt_config* cfg, int32_t which);

/* Bytes of device memory that rt_create allocates for this config. */
int64_t rt_workspace_bytes(const rt_config* cfg);

/* ---- context ------------------------------------------------------------ */

/* Validate cfg and allocate the context's workspace on the current device
 * (packed weights, status word).  *out stays NULL on failure. */
rt_status rt_create(const rt_config* cfg, rt_ctx** out);

/* Free the workspace; synchronises the device first.  NULL is a no-op. */
rt_status rt_destroy(rt_ctx* ctx);

/* Bind the model: table [L][T][F] (float for RT_FP32, IEEE half for RT_BF16;
 * kept by reference), B and I blobs (float, layout of rt_param_count; copied
 * and repacked on `stream` into the context) and env [env_h][env_w][4] float
 * (rgb + ignored lane; kept by reference).  The table must be 8-byte
 * aligned.  Also builds the MIS texel CDFs of env (RT_SAMPLE_MIS) from its
 * values at this call.  Call again after the weights or the map change.  Synchronises `stream`: the
 * FP32 biases and output layers are copied to the host once here, because
 * the BF16 kernel takes them as launch parameters. */
rt_status rt_set_params(rt_ctx* ctx, const void* table, const float* brdf_w, const float* irt_w,
                        const float* env, void* stream);

/* Read (and clear) the device status word written by bounded waits and
 * bounds checks; synchronises `stream`.  *word = 0 when nothing fired. */
rt_status rt_check(rt_ctx* ctx, uint32_t* word, void* stream);

/* ---- stages ------------------------------------------------------------- */

/* Stage (a), f = H(x) (Sec. 3.2).  pos [P][4]; feat [P][L*F] (float, level-
 * major, F inner).  Optional idx [P][L][8] (uint32 table row within the
 * level) and w [P][L][8] (trilinear weight), corner c at offset
 * (c&1, c>>1&1, c>>2&1).  The grid coordinate is u = x*0.5 + 0.5 clamped to
 * [0,1], g = u * N_l, each rounded to float32 (no contraction), cell
 * i0 = min(floor(g), N_l - 1), w = g - i0: indices are bit-exact
 * reproducible.  Dense rows: i + j(N+1) + k(N+1)^2; hashed rows:
 * (i ^ j*2654435761 ^ k*805459861) mod T in uint32 arithmetic. */
rt_status rt_encode(rt_ctx* ctx, const float* pos, int64_t P, float* feat, uint32_t* idx, float* w,
                    void* stream);

/* Stage (b), a, r, n = B(f) (Sec. 3.2, Sec. 3.3).  feat [P][L*F] float;
 * brdf [P][8] = (n.xyz normalised, a.rgb = sigmoid, r = 0.09 + 0.91 sigmoid, 0). */
rt_status rt_decode(rt_ctx* ctx, const float* feat, int64_t P, float* brdf, void* stream);

/* Stage (c), v, t = I(f, w) (Sec. 3.2).  feat [P][L*F]; dirs [P][K][4] unit
 * directions; vis [P][K] = sigmoid(z0); depth [P][K] = near + (far - near) *
 * min(softplus(z1), 1).  K in 1..4096. */
rt_status rt_trace(rt_ctx* ctx, const float* feat, const float* dirs, int64_t P, int32_t K,
                   float* vis, float* depth, void* stream);

/* Direction sampler (header conventions).  level 0: K = N directions about
 * normal[p] for primary point p, sample ids (index_offset + p)*N + i, slot 0.
 * level 1: K = M directions about normal[q] for secondary sample
 * q' = index_offset + q, slots 1..M.  normal [P][4]; dirs [P][K][4]. */
rt_status rt_sample(rt_ctx* ctx, const float* normal, int64_t P, int32_t level, int64_t index_offset,
                    float* dirs, void* stream);

/* Stage (e) at one level, directions regenerated as in rt_sample.
 * level 0 (Eq. 1 + Eq. 2): out[p] = (pi/N) sum_i (vis[p][i] Lenv(w_i) +
 *   (1 - vis[p][i]) lin[p][i]) f_r(pts[p]; w_i, view[p]); lin [P][N][4] may be
 *   NULL (treated as 0).
 * level 1 (Eq. 1 at x'): out[q] = (pi/M) sum_j vis[q][j] Lenv(w'_j) f_r(pts[q]; w'_j, view[q]);
 *   lin must be NULL.  view[q] is -w_i for a secondary point.
 * out [P][4] float (rgb, 0).  force_vis / force_vis2 are NOT applied here. */
rt_status rt_shade(rt_ctx* ctx, const rt_gbuffer* pts, int64_t P, int32_t level, int64_t index_offset,
                   const float* vis, const float* lin, float* out, void* stream);

/* ---- the fused hot path -------------------------------------------------- */

/* Stages (a)-(e) fused in one persistent kernel: radiance [P][4] (rgb, 0) of
 * the P G-buffer points; point p uses RNG pixel id pixel_offset + p, so a
 * frame rendered in shards equals the frame rendered at once.
 * With cfg.visibility = RT_VIS_HARD the BF16 path does the secondary work
 * (x' encode, B, the M secondary I evaluations, Eq. 1 at x') only for shadow
 * directions: each warpgroup queues its shadow rows in shared memory and
 * runs them in full 128-row tiles, adding every tile's pixel sums into
 * radiance in a fixed order (deterministic for a given launch shape; a
 * sharded frame agrees with the whole frame up to float rounding).  It
 * always runs 4 warpgroups per CTA.  The FP32 path takes the same decisions
 * without compaction. */
rt_status rt_render_frame(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset,
                          float* radiance, void* stream);

/* Batched lights for serving: the P points lit by E environment maps of the
 * bound size, envs [E][env_h][env_w][4] float (contiguous, 16-byte aligned);
 * radiance [E][P][4], light e at radiance + 4 e P.  Radiance is linear in
 * the map and the RNG ignores the light, so the BF16 path renders several
 * lights per launch on one shared geometry pass (hash encodes, both MLPs,
 * bounce): each row contributes fr1 (v Lenv(w_i) + (1 - v) (pi/M) sum_j v'_j
 * fr2_j Lenv(w'_j)) to every light.  Lights per launch (1, 2, 4, 8) and
 * warpgroups per CTA (2: two CTAs per SM; 3 or 4: one CTA per SM) follow the
 * context's launch shape (rt_tune / rt_set_launch_shape; default 8 and 4),
 * which rt_render_frame (one light) also uses.  The FP32 path renders one light
 * per pass.  Equal, light by light, to rt_render_frame with that map bound.
 * E in 0..1024.  No allocation, no synchronisation: capturable. */
rt_status rt_render_frame_multi(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset,
                                const float* envs, int32_t E, float* radiance, void* stream);

/* Autotuner of rt_render_frame_multi's launch shape: times every shape (tile
 * shape 128/64/32 directions per tile, see rt_set_tile_shape; lights per launch
 * 1/2/4/8 up to E; warpgroups per CTA 2/3/4) once after a warm-up on this
 * workload, writing radiance as rt_render_frame_multi does, keeps the fastest
 * in the context and returns its time in *best_ms (may be NULL; -1 for the
 * FP32 path, which has one shape).  Tile shapes that do not divide n_dirs, or
 * RT_VIS_HARD, are skipped.  Synchronises `stream`. */
rt_status rt_tune(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset, const float* envs, int32_t E,
                  float* radiance, void* stream, float* best_ms);

/* Read or force the BF16 launch shape (lights_per_launch in {1,2,4,8},
 * warpgroups in {2,3,4}; anything else is RT_ERR_INVALID_ARG).  RT_VIS_HARD
 * renders ignore the warpgroups part (always 4). */
rt_status rt_tuned_shape(const rt_ctx* ctx, int32_t* lights_per_launch, int32_t* warpgroups);
rt_status rt_set_launch_shape(rt_ctx* ctx, int32_t lights_per_launch, int32_t warpgroups);

/* Read or force the BF16 tile shape (soft visibility): dirs_per_tile = 128
 * walks the samples (pixel, direction) in tiles of 128 consecutive samples;
 * 64 or 32, with n_dirs a larger multiple of it, makes each 128-row tile
 * 128 / dirs_per_tile pixels x dirs_per_tile directions, the warpgroup
 * finishing a pixel group's direction chunks before the next group (Sec. 3.2:
 * the per-point work over directions).  Every row computes the same values in
 * either order and, for n_dirs a multiple of 32, the pixel sums are added in
 * the same order, so the radiance bits do not depend on the shape.  Other
 * values: RT_ERR_INVALID_ARG.  Default 128; rt_tune may change it. */
rt_status rt_tuned_tile_shape(const rt_ctx* ctx, int32_t* dirs_per_tile);
rt_status rt_set_tile_shape(rt_ctx* ctx, int32_t dirs_per_tile);

/* Adjoint of rt_render_frame for an upstream gradient d_radiance [P][4]
 * (lane 3 ignored): ACCUMULATES dLoss/dtable into g_table [L][T][F] float and
 * dLoss/dweights into g_brdf / g_irt (float, blob layouts).  Sampled
 * directions are constants of the estimator.  The caller zeroes the
 * gradient buffers.  RT_VIS_HARD is not differentiable: RT_ERR_UNSUPPORTED.
 * On an RT_FP32 context the adjoint runs in FP32 on the CUDA cores.  On an
 * RT_BF16 context it differentiates the BF16 render as computed (FP16 table,
 * the primary evaluation of I in split precision) with tensor-core MMAs: the
 * forward is recomputed, input gradients dZ W^T and weight gradients dZ^T X
 * run in bf16 with FP32 accumulation, table and weight gradients are summed
 * in FP32; n_dirs < 4 gives RT_ERR_UNSUPPORTED, as for the BF16 render.
 * Table gradients arrive by float reductions whose order across warps
 * varies, so repeated calls agree to rounding, not bit for bit. */
rt_status rt_backward(rt_ctx* ctx, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset,
                      const float* d_radiance, float* g_table, float* g_brdf, float* g_irt,
                      void* stream);

/* ---- rendering without any device allocation ---------------------------- */

/* rt_render_frame for callers that cannot allocate device memory: a host
 * whose memory manager owns every device allocation (pools or arenas that
 * forbid direct cudaMalloc), or a frame loop with a fixed device-memory
 * budget where an allocation, or the synchronisation a free implies, is not
 * allowed.  The paper has no counterpart: this is a deployment variant of the
 * fused FP32 kernel.  It needs no context: cfg describes the renderer and
 * the model arrays are passed directly, in the layouts of rt_set_params
 * (float table [L][T][F], 8-byte aligned; FP32 B and I blobs; env
 * [env_h][env_w][4]).  The packed weight image that rt_create would allocate
 * lives instead in one file-scope device array of 15,244 floats (61 KB), which
 * every GPU that loads the library keeps until the process exits; it is
 * rewritten in full by every call, so it needs no clearing.
 *  - precision must be RT_FP32 (else RT_ERR_UNSUPPORTED); L*F must fit the
 *    array's 32 feature rows (else RT_ERR_INVALID_ARG; every valid config does);
 *  - sampling = RT_SAMPLE_MIS returns RT_ERR_UNSUPPORTED: MIS draws from the
 *    texel CDFs of a bound map, which live in a context's workspace;
 *  - hard visibility (RT_VIS_HARD) and any pixel_offset >= 0 are accepted, as
 *    in rt_render_frame's FP32 path;
 *  - the first call on a device finds the array's device address
 *    (cudaGetSymbolAddress) and sets the kernel's shared-memory limit, with
 *    that device current; make that first call before any stream capture.
 *    Later calls look the address up again and redo that set-up if it moved
 *    (the device's context was reset in between);
 *  - all calls on a device share the array: calls whose work overlaps on the
 *    GPU (different streams, or different models in flight) race; serialise
 *    them on one stream;
 *  - no cudaMalloc, cudaFree or allocating library routine is called.
 * Results equal rt_render_frame's for the same inputs. */
rt_status rt_render_frame_static(const rt_config* cfg, const void* table, const float* brdf_w, const float* irt_w,
                                 const float* env, const rt_gbuffer* gb, int64_t P, int64_t pixel_offset,
                                 float* radiance, void* stream);

/* ---- fault-path self-tests ------------------------------------------------
 * The paper has no counterpart: these two calls let a test drive the
 * library's own failure handling without faulting or hanging a GPU. */

/* Run the device-side timeout path of the tensor-core kernels: one warp
 * waits, with their bounded mbarrier wait but a limit of limit_ns (clamped
 * to 1 ms .. 2 s), on an mbarrier that nothing arrives on, then records a
 * timeout in ctx's status word and returns; the context stays usable.  The
 * following rt_check returns RT_ERR_TIMEOUT with word = (1 << 28) | 0xF.
 * Needs a context (rt_set_params not required); asynchronous on `stream`. */
rt_status rt_selftest_wait(rt_ctx* ctx, int64_t limit_ns, void* stream);

/* Host-side fault injection for rt_create: the n-th device allocation that
 * rt_create makes from now on fails as if cudaMalloc had reported an
 * out-of-memory error (n >= 1; n = 0 disarms; n < 0 is RT_ERR_INVALID_ARG).
 * It fires once.  rt_create then frees what it had allocated and returns
 * RT_ERR_OOM with *out left NULL.  Process-wide: not for concurrent use. */
rt_status rt_debug_fail_alloc(int32_t n);

/* ---- roofline probes (measurement) ----------------------------------------
 * The paper has no counterpart: these kernels measure the two ceilings the
 * renderer's kernels are reported against that a stream copy and a library
 * GEMM do not give.  Time them with events on `stream`; they read nothing
 * but their arguments and write only `sink`. */

/* Random gathers from an L2-resident table: blocks x 512 threads, each
 * issuing iters x 8 independent loads of bytes_per_load (4 or 8) bytes at
 * rows hash(thread, k) mod rows of `table` (device, rows entries of
 * bytes_per_load bytes; rows a power of two <= 2^31; aligned to
 * bytes_per_load).  sink [blocks * 512] uint32 (device).  Loads per launch:
 * blocks * 512 * iters * 8, each one 32-byte L2 sector request. */
rt_status rt_probe_gather(const void* table, int64_t rows, int32_t bytes_per_load, int32_t iters, int32_t blocks,
                          uint32_t* sink, void* stream);

/* FP32 FMA throughput: blocks x 512 threads, each running 8 independent
 * chains of iters x 16 fmaf.  FLOP per launch: blocks * 512 * iters * 256.
 * sink [blocks * 512] float (device). */
rt_status rt_probe_ffma(int32_t iters, int32_t blocks, float* sink, void* stream);

/* ---- per-head distillation (Sec. 3.3, supplementary "Training Details") -- */

/* K stratified directions on the whole sphere for each of P points: K = S^2
 * cells of the unit square, direction k of point p from cell (k / S, k % S)
 * plus the uniforms of counter (ray_offset + p) * K + k (header
 * conventions' SplitMix64, seed cfg.dir_seed), mapped by z = 1 - 2 u1,
 * azimuth 2 pi u2.  dirs [P][K][4] float (xyz, 0), device, 16-byte aligned.
 * K must be a perfect square (1..65536); P * K < 2^31. */
rt_status rt_distill_dirs(rt_ctx* ctx, int64_t P, int32_t K, int64_t ray_offset, float* dirs, void* stream);

/* ACCUMULATES the gradient of the per-head distillation loss of the student
 * ctx (RT_FP32 only, else RT_ERR_UNSUPPORTED) into g_table [L][T][F],
 * g_brdf and g_irt (float, blob layouts; the caller zeroes them), and adds
 * the three loss terms to loss[0..2] (float, may be NULL):
 *   loss[0] = mean over points and the 7 components of |B's (n', a', r') -
 *             brdf_t| (L1 after n/|n|, sigmoid and 0.09 + 0.91 sigmoid);
 *   loss[1] = mean over points of the mean over the point's front-facing
 *             directions (w . n > 0) of BCE(sigmoid(z0), v_t), v_t =
 *             1 when vis_t > 0.5 (the teacher's visibility binarised);
 *   loss[2] = the same mean of |min(softplus(z1), 1) - (depth_t - near) /
 *             (far - near)| (min-max normalised depth).
 * pos, normal [P][4] (xyz used), dirs [P][K][4] (rt_distill_dirs); brdf_t
 * [P][8] (n', a', r', pad: a teacher's rt_decode), vis_t, depth_t [P][K]
 * (a teacher's rt_trace on dirs).  Sampled directions are constants. */
rt_status rt_distill_backward(rt_ctx* ctx, const float* pos, const float* normal, int64_t P, int32_t K,
                              const float* dirs, const float* brdf_t, const float* vis_t, const float* depth_t,
                              float* loss, float* g_table, float* g_brdf, float* g_irt, void* stream);

/* One Adam step in place over n floats (device): g' = grad + weight_decay *
 * param (L2 form), m1 = beta1 m1 + (1 - beta1) g', m2 = beta2 m2 + (1 -
 * beta2) g'^2, param -= lr (m1 / (1 - beta1^step)) / (sqrt(m2 / (1 -
 * beta2^step)) + eps).  step >= 1.  Needs no context. */
rt_status rt_adam_step(float* param, const float* grad, float* m1, float* m2, int64_t n, float lr, float beta1,
                       float beta2, float eps, float weight_decay, int32_t step, void* stream);

/* ---- denoising --------------------------------------------------------- */

/* Spatial SVGF (Schied et al. 2017) with its temporal parts removed, as the
 * paper applies it to the raw Monte Carlo frame (Sec. 4.1).  Needs no
 * context.  For the width x height image (pixel p = y * width + x):
 *   radiance [P][4] float (rgb used), depth [P] float, normal [P][4] float
 *   (unit xyz used), all device, float4 planes 16-byte aligned;
 *   work [P][4] float scratch, out [P][4] float: denoised rgb and the
 *   filtered luminance variance in lane 3.  radiance, work and out must not
 *   overlap.
 * First the luminance variance from 7 x 7 moments weighted by
 *   w_z = exp(-|z(p) - z(q)| / (sigma_z |grad z(p) . (q - p)| + 1e-10)) and
 *   w_n = max(0, n(p) . n(q))^sigma_n, grad z by one-pixel forward
 *   differences of the depth map (backward at the last column / row; the
 *   paper's "offset" depth gradient, supplementary "Rendering Details");
 * then `iterations` a-trous passes (step 2^i, 5 x 5 taps of the B3 spline
 *   [1, 4, 6, 4, 1] / 16 in each axis) with weights h w_z w_n w_l,
 *   w_l = exp(-|l(p) - l(q)| / (sigma_l sqrt(g(p)) + 1e-10)), l the
 *   luminance (0.2126, 0.7152, 0.0722) and g the 3 x 3 Gaussian of the
 *   variance: c' = sum w c / sum w, Var' = sum w^2 Var / (sum w)^2.  Taps
 *   outside the image are skipped.  SVGF's defaults: iterations 5,
 *   sigma_z 1, sigma_n 128, sigma_l 4.
 * width, height >= 1 with width * height < 2^31; iterations 0..12; sigmas
 * finite, sigma_z, sigma_l > 0, sigma_n >= 0; else RT_ERR_INVALID_ARG.
 * 1 + iterations launches on `stream`; no allocation. */
rt_status rt_denoise(int32_t width, int32_t height, const float* radiance, const float* depth, const float* normal,
                     int32_t iterations, float sigma_z, float sigma_n, float sigma_l, float* work, float* out,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_GB300_H */
