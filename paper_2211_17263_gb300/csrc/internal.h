// internal.h -- device-side data layout shared by the kernels and the C ABI host code.
//
// Memory layout in HBM (all library-owned except where noted):
//   BaseScene   one per uploaded scene: primitives in natural order, materials,
//               parameter bindings and the host-computed camera basis (~3.6 KB).
//   InstScene   one per render of a launch: the scene instantiated at theta +- tau
//               (Eq. 10's P(theta - tau_i)), primitives grouped by type, derived
//               constants precomputed (quad normals, reciprocal edge lengths, box
//               corners, light areas) and the render's random-stream words. Each
//               render CTA copies it into shared memory (~3.4 KB).
//   partials    [R][blocks] FP64 sums of squared pixel errors, one per warp work item.
//               k_finalize reduces them per render in a fixed order.
//   weights     [R][D] FP32 estimator weights d kappa / q of each render.
//   per job     theta, Adam m and v, sigma0, gradient, losses, step counter, target.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace prdpt {

constexpr int kMaxPrims = 32;
constexpr int kMaxMats = 32;
constexpr int kMaxLights = 8;
constexpr int kMaxD = 64;
constexpr int kMaxPairs = 256;
constexpr int kMaxRenders = 2 * kMaxPairs;
constexpr int kBlock = 256;      // render CTA size
constexpr int kInstBlock = 64;   // instantiation CTA size (one thread per parameter)
constexpr float kEps = 1e-4f;    // ray t_min and surface offset (scene units)
constexpr int kMaxVariant = 4;   // path sharing: perturbed primitives
constexpr int kMaxShareSpp = 64; // path sharing: samples per pixel (6 bits of a path code)
constexpr int kSeg = 4;          // path sharing: touching segments kept per path
constexpr int kMaxDiff = 8;      // pathwise estimator (Eq. 9): differentiated parameters

constexpr unsigned kTagPerturb = 1u;
constexpr unsigned kTagPath = 2u;
constexpr unsigned kTagTarget = 3u;

enum : int { kSphere = 0, kQuad = 1, kBox = 2 };
enum : int { kDiffuse = 0, kMirror = 1, kDielectric = 2 };
enum : int { kBindPos = 0, kBindRadius = 1, kBindAlbedo = 2, kBindEmission = 3, kBindTexture = 4 };
constexpr int kMaxTexRes = 1024;  // texture parameters: up to 3 x 1024^2
enum : int { kRadial = 0, kPerDim = 1, kGauss = 2 };

// Device status word bits.
enum : int { kStatusBadItem = 1, kStatusBadScene = 2 };

struct BaseScene {
    int n_prims, n_mats, n_sph, n_quad, n_box, D;
    int prim_type[kMaxPrims], prim_mat[kMaxPrims], prim_slot[kMaxPrims];
    float prim_geom[kMaxPrims][9];
    int mat_type[kMaxMats];
    float mat_param[kMaxMats][8];
    int bind_kind[kMaxD], bind_index[kMaxD], bind_comp[kMaxD];
    float eye[3], fwd[3], right[3], up[3], tan_half;
    float bg[3];
    int tex_mat, tex_res;  // texture binding: material tex_mat's albedo on quads, tex_res^2 RGB texels; -1: none
};

// Primitive records (4 x float4, grouped: spheres, quads, boxes):
//   sphere: [0] centre, radius   [1] r^2, 1/r, mat (int bits), prim (int bits)
//   quad:   [0] centre, mat      [1] unit normal, prim   [2] u, 1/(u.u)   [3] v, 1/(v.v)
//   box:    [0] min corner, mat  [1] max corner, prim
// Materials (2 x float4): [0] albedo, type (int bits)  [1] emission, ior.
// Lights: int4 (kind, record slot, prim, mat) and the emitter's area.
struct __align__(16) InstScene {
    int n_sph, n_quad, n_box, n_lights;
    unsigned seed_lo, seed_hi, step, c3;  // path stream: key and counter words 2, 3
    float4 eye;    // xyz, tan(vfov/2)
    float4 fwd;    // xyz, aspect W/H
    float4 right;  // xyz, 0
    float4 up;     // xyz, 0
    float4 bg;     // background radiance, 0
    int4 light[kMaxLights];
    float light_area[kMaxLights];
    float dclamp[kMaxDiff];  // pathwise estimator: derivative of each parameter's clamp (1 or 0)
    const float* tex;        // this render's texture [tex_res][tex_res][3] (texture scenes), or null
    int tex_mat, tex_res;    // material whose quads are textured (-1: none), resolution
    float4 mat[kMaxMats][2];
    float4 prim[kMaxPrims][4];
};
static_assert(sizeof(InstScene) % 16 == 0, "InstScene must be float4-copyable");

// Per-job description of one instantiation launch (sampler + scene binding).
struct InstJob {
    const BaseScene* base;
    InstScene* scenes;        // [R] out
    const float* theta;       // grad mode: [D] centre; render mode: [R][D] parameter vectors
    const float* sigma;       // grad mode: [D] bandwidth (sigma0 when annealing)
    float* tau_out;           // [R][D] or null
    float* w_out;             // [R][D] or null
    const int* step_dev;      // resident job: device step counter (added to `step`), else null
    unsigned long long seed;
    unsigned step, tag;
    int R, D, W, H, sampler, antithetic, crn, render_mode;
    int anneal, total_steps;
    float sigma_min, c_radial;  // c_radial = sqrt(2) Gamma((D+1)/2) / Gamma(D/2)
    int block_begin;          // first CTA index of this job in a packed launch
    int pair_begin;           // the job's first antithetic pair of a sharded estimate (draw/render offset)
    int diff;                 // pathwise estimator: write each render's clamp derivatives
    int hd;                   // high-dimensional parameters: draws made by k_perturb_hd, skip a1 here
    const float* tex_all;     // texture scenes: [R][tex_D] per-render textures, or null
    int tex_D;
    unsigned* share_reset;    // [4] path-sharing counters of the job, zeroed by its first CTA, or null
    // path sharing: bounds of each perturbed primitive in each render, [R][kMaxVariant][2]
    // (min, max corner, inflated), written by the render's CTA; null when not sharing
    float4* var_box;
    unsigned* aff_cursor;     // [R] per-render cursors of the per-render pass, zeroed by the render's CTA
    unsigned* aff_flags;      // [R][flag_words] pixels with corrections per render, zeroed by the render's CTA
    int flag_words;
    int n_var;
    int var_prim[kMaxVariant];  // the perturbed primitives (natural order indices)
};

// Per-job description of one render launch. The image is cut into blocks of
// bw x bh <= 32 pixels; one warp renders one (render, block) work item.
struct TraceJob {
    const InstScene* scenes;  // [R]
    const float4* target;     // [H][W] (gradient mode) or null
    float4* images;           // [R][H][W] (render mode) or null
    double* partials;         // [R][tiles] sums of squared pixel errors per block
    unsigned* done;           // renders finalised (reset by the CTA that completes the job)
    double* losses;           // [R] L_r
    const float* w;           // [R][D]
    float* grad_out;          // [D] or null
    float* loss_out;          // [R] or null
    float* theta;             // Adam state (null: no optimiser step)
    float* m;
    float* v;
    int* step_dev;
    float lr, b1, b2, eps;
    int W, H, spp, depth, rr_start, R, D, antithetic;
    int bw, bh, tiles_x, tiles;
    int n_prims, n_mats;      // used primitive and material records (staging size)
    int item_begin;           // first work item of this job in a packed launch
    int fin_begin;            // first finalisation CTA of this job in a packed launch
    // Path sharing across renders (common random numbers, geometry-only bindings): a work
    // item is one pixel block of all R renders. share = 0 disables it.
    int share;
    unsigned long long* share_acc;   // [tiles][3][32] shared radiance of blocks with affected paths
    unsigned long long* acc_aff;     // [R][H*W][3] per-render radiance corrections of recorded paths, 2^-32
                                     // fixed point modulo 2^64 (kept zero between steps)
    // recorded paths (a ray touched a union box of the perturbed primitives): [H*W*spp] capacity
    unsigned* aff_codes;      // (pixel << 6) | sample
    unsigned* aff_segw;       // segment word: where its touching segments are kept, or "every render"
    float* aff_lsh;           // [3] radiance of the path in the shared pass
    float4* seg_pool;         // [seg_cap][2] touching segments (o, tmax), (d, 0), kSeg slots per path
    float4* seg_state;        // [seg_cap / kSeg][4] path state where a path's renders part (see note_touch)
    unsigned seg_cap;
    const float4* var_box;    // [R][kMaxVariant][2] per-render bounds of the perturbed primitives
    unsigned* aff_cursor;     // [R] next list entry of each render in the per-render pass
    // [R][flag_words] bit p of render r: the per-render pass added a correction to pixel p of
    // render r (the epilogue reads and clears only those pixels' corrections)
    unsigned* aff_flags;
    int flag_words;
    int* aff_tiles;           // [tiles] blocks with affected paths (appended by the shared pass)
    unsigned* share_ctl;      // [0] listed blocks, [1] recorded paths, [2] segment slots claimed,
                              // [3] spare; zeroed by the instantiation launch
    // Pathwise estimator (Eq. 9): diff_n parameters, all albedo (kind 2) or emission (kind 3)
    // of material diff_mat, channel diff_comp; each block writes its partial sums of
    // (I - T) dI/dtheta_k to gpartials [R][tiles][diff_n]; k_finalize reduces them per render
    // into rgrads [R][kMaxDiff] and forms the mean over renders.
    int hd;                   // high-dimensional parameters: gradient and Adam by k_grad_adam_hd
    int diff, diff_n;
    int diff_mat[kMaxDiff], diff_comp[kMaxDiff], diff_kind[kMaxDiff];
    double* gpartials;
    double* rgrads;
    int n_var;                // perturbed primitives (<= kMaxVariant)
    int var_slot[kMaxVariant];  // their record slots
    unsigned var_prims;       // record-slot bitmask of perturbed primitives
    unsigned var_mats;        // bitmask of materials whose parameters are bound
    // Render-group mode (k_trace_group): gsize renders per work item (0: per-render items);
    // each render's row of the per-warp table holds gstride float4 (its records of the
    // n_var perturbed primitives, the albedo rows of the bound materials, and its emitter
    // areas when a radius binding can change them)
    int gsize, gstride;
    // Emitter-sharing mode (k_trace_emit): 1 when the job's paths are traced once for all its
    // renders, each render adding its own next-event estimates (gstride as above; items are
    // pixel blocks of all renders)
    int emit;
};
struct TraceLaunch {
    TraceJob job0;            // used when jobs == null (single job, passed by value)
    const TraceJob* jobs;     // packed launch: [njobs] in device memory
    int njobs, total_items;
    int share;                // 1: every job of the launch shares paths (selects the kernel variant)
    int diff_nd;              // pathwise estimator: tangent slots of the kernel variant (0, 4 or 8)
    int group;                // 1: every job of the launch runs in render-group mode (k_trace_group),
                              // 2: in emitter-sharing mode (k_trace_emit)
    int fin_total;            // packed launch: finalisation CTAs (sum of R over jobs)
    unsigned* queue;          // work-queue head, zeroed by the instantiation launch
    unsigned long long* counters;  // [8] or null (null: the uncounted kernel variant runs)
    int* status;
};

struct InstLaunch {
    InstJob job0;
    const InstJob* jobs;
    int njobs, total_blocks;
    unsigned* queue_reset;    // zeroed by CTA 0
    unsigned* queue_reset2;   // zeroed by CTA 0 (second queue of a packed launch), or null
    unsigned* queue_reset3;   // zeroed by CTA 0 (third queue of a packed launch), or null
    unsigned* queue_reset4;   // zeroed by CTA 0 (fourth queue of a packed launch), or null
};

// High-dimensional parameter draws (texture scenes, D > kMaxD): norms per draw, then
// per (render, parameter) perturbation, weight and perturbed parameter.
constexpr int kNormSplitMax = 64;  // radial sampler: CTAs per draw for the norms of D > kMaxD normals

// One draw of the radial sampler in D > kMaxD dimensions: v = (|z|, radius) and the
// partial sums (|z|^2, radius^2) of its CTAs; ctr counts the parts done and is reset to 0
// by the CTA that combines them (so it is zero between launches).
struct HdNorm {
    float2 v;
    unsigned ctr, pad;
    double2 part[kNormSplitMax];
};

struct HdDraws {
    int D, R, sampler, antithetic;
    int draw_begin;           // global index of draw 0 (sharded estimates)
    unsigned long long seed;
    unsigned step;
    const int* step_dev;      // resident job: device step counter added to `step`, else null
    const float* theta;       // [D] centre
    const float* sigma;       // [D] bandwidth (sigma0 when annealing)
    int anneal, total_steps;
    float sigma_min, c_radial;
    HdNorm* norms;            // [draws] the radial sampler's norms (counters zero on entry)
    int norm_split;           // CTAs per draw in k_hd_norms (1..kNormSplitMax)
    float* theta_out;         // [R][D] theta + tau (per-render texture), or null
    float* tau_out;           // [R][D] or null
    float* w_out;             // [R][D] or null
};
// The gradient of Eq. 10 over D > kMaxD parameters (g = W^T dL / 2P) and Adam.
struct HdGrad {
    int D, R, antithetic;
    const float* w;           // [R][D]
    const double* losses;     // [R]
    float* grad_out;          // [D] or null
    float *theta, *m, *v;     // Adam state, or null (no optimiser step)
    const int* step_dev;      // incremented by k_finalize before this kernel runs: Adam's 1-based t
    float lr, b1, b2, eps;
};

// Launchers (kernels.cu). All enqueue on `stream` and return the launch error.
cudaError_t launch_hd_draws(const HdDraws& H, cudaStream_t stream);
cudaError_t launch_hd_grad(const HdGrad& G, cudaStream_t stream);
cudaError_t launch_instantiate(const InstLaunch& L, cudaStream_t stream);
cudaError_t launch_trace(const TraceLaunch& L, bool render_mode, int grid, cudaStream_t stream);
// Second and third passes of a path-sharing job: the affected paths per render, then the
// per-render errors of the blocks that had affected paths.
cudaError_t launch_trace_affected(const TraceLaunch& L, int grid, cudaStream_t stream);
cudaError_t launch_shared_epilogue(const TraceLaunch& L, int grid, cudaStream_t stream);
// Per-render losses, gradient and Adam: one CTA per render of every job in the launch.
cudaError_t launch_finalize(const TraceLaunch& L, int n_renders, cudaStream_t stream);
cudaError_t launch_adam(int D, float* theta, float* m, float* v, const float* g, int t, float lr, float b1,
                        float b2, float eps, cudaStream_t stream);
// FP32 FMA throughput probe: `blocks` CTAs of kBlock threads, each thread 2 x kFfmaChains
// x iters flop; out holds blocks x kBlock floats.
cudaError_t launch_ffma_probe(float* out, int blocks, int iters, cudaStream_t stream);
int ffma_probe_flops_per_thread_iter();
cudaError_t launch_philox(unsigned long long seed, unsigned c0, unsigned c1, unsigned c2, unsigned c3, int n,
                          uint32_t* out, cudaStream_t stream);
// Resident CTAs per SM of the render kernel; the pathwise-estimator variant runs CTAs of
// kDiffBlock threads.
int trace_blocks_per_sm(bool render_mode);
int trace_group_blocks_per_sm();
int trace_emit_blocks_per_sm();
constexpr int kGroupBlock = 128;    // render-group CTAs: 4 warps (their per-warp tables fit 48 KB)
constexpr int kGroupPrims = 16;     // render-group mode: at most 16 primitives ...
constexpr int kGroupMats = 16;      // ... and 16 materials (the staged copy is smaller)
constexpr int kGroupTabRows = 192;  // float4 of a warp's per-render record table (render-group mode)
constexpr int kEmitTabRows = 256;   // float4 of a CTA's per-render record table (emitter-sharing mode)
constexpr int kDiffBlock = 128;
int trace_diff_blocks_per_sm();

// Pixel block of one warp work item for 8, 16 or 32 pixels.
inline void block_shape(int pixels, int* bw, int* bh) {
    *bw = (pixels >= 16) ? 8 : 4;
    *bh = pixels / *bw;
}

}  // namespace prdpt
