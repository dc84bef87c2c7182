/*
 * prdpt.h -- C ABI of the GB300 (sm_103a) plateau-reduced gradient library.
 *
 * The library computes the plateau-reduced gradient of Fischer & Ritschel,
 * "Plateau-reduced Differentiable Path Tracing": the image loss L of a path-traced
 * scene is convolved with a Gaussian kernel over the scene parameters theta
 * (Eq. 6), and the gradient of the smoothed loss is estimated by perturbing
 * theta, path-tracing the perturbed scenes and weighting each render's loss by the
 * kernel gradient over the sampling density (Eq. 10, Eq. 11, Algorithm 1). The
 * renderer is treated as a black box; only its forward image is needed.
 *
 * Conventions for every entry point:
 *  - Every call returns a prdpt_status; 0 is success. No exception crosses the ABI.
 *    On failure prdpt_last_error() returns a message owned by the library, valid
 *    until the next call on the same context from the same thread.
 *  - Pointers named *_dev are device pointers owned by the caller (for instance
 *    torch tensor storage); *_host pointers are host memory owned by the caller.
 *    The library never frees caller memory and never keeps caller pointers after
 *    a call returns, except where a call says so.
 *  - Host threads: calls on one context may come from several threads. Each call
 *    holds the context while it checks its arguments and enqueues its work (and, for a
 *    synchronous call, until it returns), so calls from different threads run one
 *    after another on the host; their GPU work overlaps as the stream rules below allow.
 *  - Calls taking `stream` (a cudaStream_t, NULL = legacy default stream) only
 *    enqueue work and return; their device-side results are ready when the stream
 *    reaches that point. Calls without a stream are synchronous.
 *  - Order on the GPU: prdpt_render_batch, prdpt_sample_perturbations,
 *    prdpt_smoothed_grad(_host), prdpt_step_host and prdpt_step_batch use the context's shared scratch
 *    buffers and work counters, so such calls on one context must execute in order
 *    (one stream, or streams ordered by events). A resident job has buffers of its
 *    own: different jobs may step (prdpt_step) concurrently on different streams,
 *    while the steps of one job must be ordered.
 *  - Images are row-major [H][W] of float4 (R, G, B, pad); pixel (0,0) is the top
 *    left; the pad channel is written as 0 and ignored on input.
 *  - Random numbers: Philox4x32-10 with key = 64-bit seed; counter words
 *    (c0, c1, c2, c3). Perturbation draws use (pair or draw index, block, step,
 *    1 << 28); path samples use (pixel y*W+x, sample | vertex << 16 | slot << 24,
 *    step, tag << 28 | render field). The four uniforms of slot 0 are the light point
 *    (u, v) of next-event estimation and the BSDF sample (u1, u2); slot 1 holds the
 *    light choice, the Russian-roulette uniform and the dielectric's reflect-or-refract
 *    uniform (its fourth word is unused); slot 2 (vertex 0 only) is the pixel jitter
 *    (x, y). Uniforms are ((word >> 9) * 2 + 1) / 2^24.
 *  - Limits: at most PRDPT_MAX_PRIMS primitives, PRDPT_MAX_MATS materials,
 *    PRDPT_MAX_LIGHTS emitters, PRDPT_MAX_D parameters and PRDPT_MAX_PAIRS
 *    antithetic pairs per call. Width and height at most 8192, spp at most 65535,
 *    depth at most 64.
 */
#ifndef PRDPT_H
#define PRDPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct prdpt_ctx prdpt_ctx;
typedef int32_t prdpt_status;

#define PRDPT_OK 0
#define PRDPT_E_INVALID_ARG 1   /* an argument is out of range or inconsistent */
#define PRDPT_E_OUT_OF_BUDGET 2 /* the allocation would exceed the context's HBM budget */
#define PRDPT_E_CUDA 3          /* a CUDA runtime call failed */
#define PRDPT_E_TIMEOUT 4       /* a bounded device-side wait expired */
#define PRDPT_E_NOT_READY 5     /* the result is not available yet */
#define PRDPT_E_NOT_FOUND 6     /* unknown scene or job handle */
#define PRDPT_E_DEVICE 7        /* a kernel reported an error through the status word */

#define PRDPT_MAX_PRIMS 32
#define PRDPT_MAX_MATS 32
#define PRDPT_MAX_LIGHTS 8
#define PRDPT_MAX_D 64
#define PRDPT_MAX_PAIRS 256

/* primitive, material, binding and sampler kinds */
#define PRDPT_PRIM_SPHERE 0
#define PRDPT_PRIM_QUAD 1
#define PRDPT_PRIM_BOX 2
#define PRDPT_MAT_DIFFUSE 0
#define PRDPT_MAT_MIRROR 1
#define PRDPT_MAT_DIELECTRIC 2
#define PRDPT_BIND_PRIM_POS 0     /* theta_d sets primitive `index`'s centre component */
#define PRDPT_BIND_SPHERE_RADIUS 1 /* theta_d sets sphere `index`'s radius (absolute value) */
#define PRDPT_BIND_MAT_ALBEDO 2   /* theta_d sets material `index`'s albedo channel, clamped to [0,1] */
#define PRDPT_BIND_MAT_EMISSION 3 /* theta_d sets material `index`'s emission channel, clamped to >= 0 */
#define PRDPT_SAMPLER_RADIAL 0    /* q ~ |grad kappa| as a vector norm; exact 1-D sampler of the paper */
#define PRDPT_SAMPLER_PERDIM 1    /* literal per-dimension two-sided inverse CDF */
#define PRDPT_SAMPLER_GAUSS 2     /* tau ~ N(0, sigma^2): no importance sampling ("noIS") */

/* Scene in host memory; copied by prdpt_scene_upload.
 *  prim_geom: [n_prims][9] floats; sphere: centre(3), radius; quad: centre(3),
 *    edge u(3), edge v(3) (orthogonal; one-sided emitters radiate along
 *    normalize(u x v)); box: centre(3), half size(3).
 *  mat_param: [n_mats][8] floats: albedo(3), emission(3), ior, unused.
 *  camera: eye(3), look-at(3), up(3), vertical field of view in degrees.
 *  background: constant radiance of rays that leave the scene. */
typedef struct {
    int32_t n_prims, n_mats;
    const int32_t* prim_type;
    const int32_t* prim_mat;
    const float* prim_geom;
    const int32_t* mat_type;
    const float* mat_param;
    const float* camera;
    const float* background;
} prdpt_scene_desc;

/* theta_d -> scene field. `component` is 0..2 (x/y/z or R/G/B); unused for radius. */
typedef struct {
    int32_t kind, index, component;
} prdpt_param_binding;

/* Forward rendering options (Eq. 3: `spp` Monte-Carlo paths per pixel). */
typedef struct {
    int32_t width, height, spp, depth;
    int32_t rr_start;          /* 0-based vertex index from which Russian roulette applies; -1 = never */
    uint64_t seed;
    uint32_t step, tag;        /* Philox counter word 2 and stream tag (2 = path, 3 = target) */
    int32_t crn;               /* 1: every render uses path field 0; 0: render i uses field i */
    int32_t block_pixels;      /* pixels per warp work item (8, 16 or 32); 0 = automatic */
    int32_t ctas_per_sm;       /* resident render CTAs per SM, counted as 256-thread CTAs (kernels with
                                  smaller CTAs keep proportionally more; capped at the occupancy
                                  limit); 0 = occupancy limit */
} prdpt_render_opts;

/* Gradient-estimator options (Eq. 10 / Eq. 9, Algorithm 1). R = 2 * pairs renders. */
typedef struct {
    int32_t pairs;             /* P antithetic pairs (Algorithm 1's N = 2P) */
    int32_t width, height, spp, depth, rr_start;
    int32_t sampler;           /* PRDPT_SAMPLER_* */
    int32_t antithetic;        /* 1: renders 2p, 2p+1 use +tau_p, -tau_p; 0: 2P independent draws */
    int32_t crn;               /* 1: all renders share path samples (field 0); 0: render r uses field r+1 */
    uint64_t seed;
    uint32_t step;             /* optimiser step: Philox counter word 2 of every draw */
    int32_t block_pixels;      /* pixels per warp work item (8, 16 or 32); 0 = automatic */
    int32_t ctas_per_sm;       /* resident render CTAs per SM, counted as 256-thread CTAs (kernels with
                                  smaller CTAs keep proportionally more; capped at the occupancy
                                  limit); 0 = occupancy limit */
    int32_t no_path_sharing;   /* 0: with crn = 1, trace paths that no perturbation can touch once for
                                  all renders (geometry-only perturbations), or, when every emitter is
                                  perturbed and only positions and radii are bound (at most 64
                                  renders, Eq. 10, no texture), trace each path once with each
                                  render's own next-event estimates (emitter sharing); same result,
                                  bit for bit; 1: trace every render */
    int32_t estimator;         /* PRDPT_ESTIMATOR_*: 0 = Eq. 10 (kernel-gradient weights times render
                                  losses); 1 = Eq. 9 (mean over the renders of each render's pathwise
                                  loss gradient: requires sampler = GAUSS, every binding an albedo or
                                  emission one, D <= 8; no path sharing; single-job steps only) */
    int32_t pair_begin;        /* first pair of a shard of a larger estimate (0 normally): this call
                                  computes pairs [pair_begin, pair_begin + pairs) with their global
                                  draw indices (and, with crn = 0, global path-stream fields), and
                                  returns their mean; shards combine as g = sum_s (P_s / P) g_s */
    int32_t render_groups;     /* renders traced side by side in one warp when paths are not shared
                                  (each lane one render of the same path sample; same result, bit for
                                  bit): 0 = automatic (the largest of 32, 16, 8, 4, 2 that divides 2P
                                  and whose per-render records fit), -1 = off (one render per work
                                  item), or 2, 4, 8, 16, 32. Used with crn = 1, the Eq. 10 estimator
                                  and no texture or emission bindings; ignored otherwise, and when
                                  emitter sharing applies (see no_path_sharing) */
} prdpt_grad_opts;
#define PRDPT_ESTIMATOR_KERNEL_GRADIENT 0 /* Eq. 10: sum_r w_r L_r */
#define PRDPT_ESTIMATOR_PATHWISE 1        /* Eq. 9: mean_r dL/dtheta (theta + tau_r) */

/* A resident optimisation job: scene parameters, Adam state and target stay on
 * the device between steps (Adam, Sec. 3.4; bandwidth schedule, Sec. 3.3). */
typedef struct {
    prdpt_grad_opts grad;      /* grad.step is the first step index */
    const float* theta0_host;  /* [D] initial parameters */
    const float* sigma0_host;  /* [D] kernel bandwidth */
    const float* target_host;  /* [H][W][4] target image */
    float lr, beta1, beta2, eps;
    float sigma_min;           /* lower end of the linear bandwidth decay */
    int32_t anneal;            /* 1: sigma constant for total_steps/2 steps, then linear to sigma_min */
    int32_t total_steps;       /* schedule length (used only when anneal = 1) */
} prdpt_job_desc;

/* Create a context on CUDA device `device`. hbm_budget_bytes bounds the device
 * memory the context may allocate (0 = no bound). */
prdpt_status prdpt_create(prdpt_ctx** out, int32_t device, uint64_t hbm_budget_bytes);

/* Destroy a context and free all library-owned device memory. Synchronises the device. */
prdpt_status prdpt_destroy(prdpt_ctx* ctx);

/* Message describing the last failure on this context (never NULL). */
const char* prdpt_last_error(prdpt_ctx* ctx);

/* Copy a scene and its parameter bindings (the map theta -> scene, Eq. 1's
 * f(x, theta)) into device memory. D = number of bindings (1..PRDPT_MAX_D).
 * Synchronous. Emissive boxes are rejected. */
prdpt_status prdpt_scene_upload(prdpt_ctx* ctx, const prdpt_scene_desc* scene, const prdpt_param_binding* binds,
                                int32_t D, int32_t* scene_id_out);

/* Free a scene. Jobs using it must have been released (each job keeps its own copy of
 * the scene). Does not wait for the device: the scene's block is reused once the last
 * stateless call that read it has completed. */
prdpt_status prdpt_scene_release(prdpt_ctx* ctx, int32_t scene_id);

/* Render n scenes at parameter vectors thetas_dev [n][D] (Eq. 3 per pixel):
 * images_dev [n][H][W][4]. Render i uses path field (crn ? 0 : i). */
prdpt_status prdpt_render_batch(prdpt_ctx* ctx, int32_t scene_id, const float* thetas_dev, int32_t n,
                                const prdpt_render_opts* opts, float* images_dev, void* stream);

/* The perturbations and weights a gradient call with the same options draws
 * (Sec. 3.2, Eq. 11): tau_dev [2P][D] (tau of render r; antithetic renders are
 * negated) and w_dev [2P][D] (d kappa / q of render r). sigma_dev [D]. */
prdpt_status prdpt_sample_perturbations(prdpt_ctx* ctx, int32_t D, const float* sigma_dev,
                                        const prdpt_grad_opts* opts, float* tau_dev, float* w_dev, void* stream);

/* One plateau-reduced gradient (Eq. 10): grad_dev[d] = (1/2P) sum_p w_pd (L_2p - L_2p+1)
 * with L_r the image MSE (1/3HW) sum (I_r - T)^2 of render r at theta + tau_r.
 * theta_dev, sigma_dev: [D]; target_dev: [H][W][4]; grad_dev: [D];
 * losses_dev: [2P] or NULL. The perturbed images never reach device memory:
 * each render's loss is reduced inside the render kernel. */
prdpt_status prdpt_smoothed_grad(prdpt_ctx* ctx, int32_t scene_id, const float* theta_dev, const float* sigma_dev,
                                 const prdpt_grad_opts* opts, const float* target_dev, float* grad_dev,
                                 float* losses_dev, void* stream);

/* The same gradient with host buffers, for callers whose inputs and results live in host
 * memory: copies theta_host [D], sigma_host [D] and target_host [H][W][4] into the
 * context's scratch on `stream`, computes the gradient as prdpt_smoothed_grad, copies
 * grad_host [D] and losses_host [2P] (NULL allowed) back, and returns when the stream has
 * reached that point (synchronous). theta and sigma travel through a page-locked staging
 * buffer of the context; a page-locked target is copied by direct DMA, a pageable one is
 * staged by the CUDA runtime. Holds the context for the whole call (concurrent calls on
 * one context from several host threads run one after another) and shares its scratch
 * (see the ordering rules above). */
prdpt_status prdpt_smoothed_grad_host(prdpt_ctx* ctx, int32_t scene_id, const float* theta_host,
                                      const float* sigma_host, const prdpt_grad_opts* opts, const float* target_host,
                                      float* grad_host, float* losses_host, void* stream);

/* A whole optimisation step with host buffers: the gradient as prdpt_smoothed_grad_host
 * at theta_host, then one Adam update (as prdpt_adam_step, step t >= 1, lr, beta1, beta2,
 * eps) of theta_host, m_host and v_host [D], which are read and written back in place.
 * The update runs in the gradient's last kernel on the device, with the same arithmetic
 * as prdpt_adam_step. grad_host [D] and losses_host [2P] receive the step's gradient and
 * losses (either may be NULL). Synchronous; shares the context's scratch like
 * prdpt_smoothed_grad_host. */
prdpt_status prdpt_step_host(prdpt_ctx* ctx, int32_t scene_id, float* theta_host, float* m_host, float* v_host,
                             int32_t t, float lr, float beta1, float beta2, float eps, const float* sigma_host,
                             const prdpt_grad_opts* opts, const float* target_host, float* grad_host,
                             float* losses_host, void* stream);

/* One Adam update (Sec. 3.4; PyTorch's formula, FP32 arithmetic as its FP32 Adam; t is
 * the 1-based step) of D parameters in place: theta_dev, m_dev, v_dev [D], grad_dev [D]. */
prdpt_status prdpt_adam_step(prdpt_ctx* ctx, int32_t D, float* theta_dev, float* m_dev, float* v_dev,
                             const float* grad_dev, int32_t t, float lr, float beta1, float beta2, float eps,
                             void* stream);

/* Create a resident job on a scene: copies theta0, sigma0, the target (target_host may be
 * NULL: then the target starts at zero and is rendered on the device by
 * prdpt_job_render_target) and the scene into a block of the context's arena (see
 * prdpt_job_release): chunks of 256 MB are reserved from the device while the HBM budget
 * leaves room for four, else exactly what a block needs, and charged to the budget whole.
 * Synchronous, but the uploads run on a stream of the context's own that waits for no
 * other work on the device. */
prdpt_status prdpt_job_create(prdpt_ctx* ctx, int32_t scene_id, const prdpt_job_desc* desc, int32_t* job_out);

/* One optimisation step of a resident job, all on the device: draw perturbations,
 * render and reduce losses, form the gradient, apply Adam, advance the step and
 * the bandwidth schedule. No host synchronisation; capturable in a CUDA graph
 * once the context has run one step with the same shape. */
prdpt_status prdpt_step(prdpt_ctx* ctx, int32_t job_id, void* stream);

/* One step of each of n resident jobs, packed into one sampler launch and one
 * persistent render launch (the jobs' renders share the GPU). Each job's result
 * is identical to what prdpt_step would give it alone. */
prdpt_status prdpt_step_batch(prdpt_ctx* ctx, const int32_t* job_ids, int32_t n, void* stream);

/* Copy a job's current parameters [D], last gradient [D], last per-render losses
 * [2P] and completed-step count to the host (any pointer may be NULL). Waits for the
 * job's last enqueued work only (after a step enqueued inside a CUDA-graph capture: for
 * the whole device) and checks the device status word. */
prdpt_status prdpt_job_read(prdpt_ctx* ctx, int32_t job_id, float* theta_host, float* grad_host,
                            float* losses_host, int32_t* steps_host);

/* Release a job. Does not wait for the device: the job's block returns to the context's
 * arena (device memory the context reserves in chunks and carves into job and scene
 * blocks) once the job's last enqueued work has completed, and is carved again by later
 * prdpt_job_create and prdpt_scene_upload calls. The arena's chunks are returned to the
 * device by prdpt_destroy. A job stepped inside a CUDA-graph capture waits for the device
 * here (replays are not tracked); such a graph must not be replayed after the release. */
prdpt_status prdpt_job_release(prdpt_ctx* ctx, int32_t job_id);

/* Render the target image of a job (Sec. 4.1: the target is a render at the reference
 * parameters) straight into its device buffer: one render at theta_ref_dev [D] (device
 * memory; for a texture scene the texture itself) on random stream TARGET (tag 3), step
 * 0, common path field 0, with the job's image size, spp, depth, Russian roulette and
 * seed -- the same image as prdpt_render_batch with those options. Enqueued on `stream`;
 * the job's steps must come after it in stream order. No host round trip. */
prdpt_status prdpt_job_render_target(prdpt_ctx* ctx, int32_t job_id, const float* theta_ref_dev, void* stream);

/* Philox4x32-10 words for counters (c0_base + i, c1, c2, c3), key = seed:
 * words_dev [n][4]. Exposed so that the random streams can be checked bit for bit. */
prdpt_status prdpt_philox_words(prdpt_ctx* ctx, uint64_t seed, uint32_t c0_base, uint32_t c1, uint32_t c2,
                                uint32_t c3, int32_t n, uint32_t* words_dev, void* stream);

/* Work counters of the render kernel (the algorithmic work of Eq. 3's path
 * samples), accumulated while enabled: [0] ray-sphere tests, [1] ray-quad tests,
 * [2] ray-box tests, [3] camera paths, [4] surface vertices, [5] shadow rays,
 * [6] closest-hit rays, [7] unused. enable=1 zeroes them and makes later render
 * launches use the counting kernel variant; enable=0 returns to the uncounted
 * variant. prdpt_counters_read copies them to counts_host[8] (synchronous). */
prdpt_status prdpt_counters_enable(prdpt_ctx* ctx, int32_t enable);
prdpt_status prdpt_counters_read(prdpt_ctx* ctx, uint64_t* counts_host);

/* CUDA-event timing of the render kernel: while enabled, every render launch is
 * bracketed by two events recorded on its own stream. prdpt_kernel_timing_read
 * waits for the recorded launches and returns their summed duration (ms) and
 * count, then forgets them. Not for use inside CUDA-graph capture. */
prdpt_status prdpt_kernel_timing_enable(prdpt_ctx* ctx, int32_t enable);
prdpt_status prdpt_kernel_timing_read(prdpt_ctx* ctx, double* total_ms, int64_t* launches);

/* Device memory the context currently holds (its arena's chunks, free space included,
 * and the scratch of the stateless calls), in bytes. */
prdpt_status prdpt_memory_used(prdpt_ctx* ctx, uint64_t* bytes_out);

/* FP32 issue-rate probe (a measurement utility; the paper has no counterpart): one
 * full-occupancy launch on every SM in which each thread runs independent fused
 * multiply-add chains for `iters` iterations (16 flop per thread per iteration), timed
 * with CUDA events after a short warm-up launch on a stream of its own. Writes the
 * achieved FP32 TFLOP/s, the denominator of the render kernels' roofline, and the
 * launch's duration in ms (ms_out may be NULL). Synchronous; allocates and frees a
 * small device buffer. */
prdpt_status prdpt_fp32_peak_probe(prdpt_ctx* ctx, int32_t iters, double* tflops_out, double* ms_out);

/* Synchronise `stream` and check the context's device status word. */
prdpt_status prdpt_sync(prdpt_ctx* ctx, void* stream);

/* The same plateau-reduced gradient as prdpt_smoothed_grad, for callers that cannot
 * allocate device memory -- for example a process whose device memory belongs to
 * another allocator (a framework's caching allocator, a fixed arena of a serving
 * runtime), or code that may not grow its footprint or create a context after
 * start-up. It takes no context and allocates nothing: the scene comes from host
 * memory (`scene`, `binds`, D as for prdpt_scene_upload, checked by the same rules;
 * no texture bindings), theta_dev, sigma_dev, target_dev, grad_dev and losses_dev (NULL
 * allowed) are the caller's device buffers exactly as for prdpt_smoothed_grad, and
 * every intermediate buffer lives in one fixed 6 MiB __device__ array that each GPU
 * loading the library holds until the process exits. The call enqueues three kernels
 * and one memset on `stream` and returns; the scene is passed as a kernel parameter,
 * so no host buffer needs to outlive the call. With the same block_pixels it gives the
 * same losses and gradient as prdpt_smoothed_grad, bit for bit; block_pixels = 0 means
 * 32-pixel blocks here.
 * Limits: 1..32 antithetic pairs, pair_begin 0..2^26, and 2P x (image blocks) x 8 bytes
 * of loss partials within the 6 MiB (512 x 512 with 32-pixel blocks fits 32 pairs);
 * larger requests return PRDPT_E_OUT_OF_BUDGET with a message, before any launch. All
 * calls share that array and each call overwrites what the last one left: calls that
 * overlap on the GPU (different streams, no ordering) race and must not be issued.
 * Calls from several host threads enqueue one after another (a lock per device), so
 * calls on one stream are ordered. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and the device's SM count. Errors are written
 * to err (err_len bytes, may be NULL); there is no context to query, and the kernels'
 * device status word is not reported (the host checks above leave the kernels nothing
 * to refuse). Only
 * opts->estimator = PRDPT_ESTIMATOR_KERNEL_GRADIENT. The paper has no counterpart to
 * this entry point. */
prdpt_status prdpt_smoothed_grad_static(const prdpt_scene_desc* scene, const prdpt_param_binding* binds, int32_t D,
                                        const float* theta_dev, const float* sigma_dev, const prdpt_grad_opts* opts,
                                        const float* target_dev, float* grad_dev, float* losses_dev, void* stream,
                                        char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* PRDPT_H */
