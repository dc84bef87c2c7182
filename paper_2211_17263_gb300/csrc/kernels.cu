// kernels.cu -- sm_103a kernels of the plateau-reduced gradient estimator.
//
//   k_instantiate   one CTA per render: Philox draws -> perturbation tau and weight
//                   w (Sec. 3.2, Eq. 11, Algorithm 1), theta +- tau bound into the
//                   scene (Eq. 10's P(theta - tau_i)), derived constants precomputed;
//                   the scene is built in shared memory and written out in one copy.
//   k_trace         persistent render kernel. Each warp pulls (render, pixel block)
//                   work items from a queue, stages the render's scene in its own
//                   shared-memory slot, and traces the block's pixels x samples as a
//                   pool of path tasks: a lane whose path ends takes the next task
//                   at once (ballot + popc), so live paths stay packed in the warp.
//                   Radiance is accumulated per pixel in 2^-32 fixed point (integer
//                   adds are order-independent, so results do not depend on which
//                   lane traced which path). Each pixel's error against the target is
//                   formed exactly in integers, squared in FP32, and summed per block
//                   in FP64 -- the perturbed image never reaches HBM. Variants: path
//                   sharing (a block of all renders traced once in the scene without
//                   the perturbed primitives, recording the paths that may differ) and
//                   the pathwise estimator (Eq. 9, forward-mode tangents).
//   k_trace_affected  path sharing, per-render pass: each render traces again the
//                   recorded paths that may meet its own primitives, resuming where
//                   the renders part, and adds its radiance minus the shared one.
//   k_shared_epilogue path sharing: the blocks with recorded paths, all renders.
//   k_finalize      one CTA per render: L_r from the block partials (fixed order); the
//                   CTA completing a job's last render forms the gradient of Eq. 10
//                   (or the mean of Eq. 9's pathwise gradients) and applies Adam.
//   k_hd_norms, k_hd_perturb, k_hd_grad  high-dimensional parameters (texture scenes):
//                   D-dimensional draws and the gradient W^T dL with Adam.
//   k_adam          standalone Adam update.
//   k_philox        raw Philox words (for bit-exact checks of the random streams).
//   k_ffma_probe    FMA-chain throughput probe (the FP32 peak of the roofline).
//
// FP32 throughout the path tracer; every floating-point reduction is in a fixed order
// and every per-pixel sum is an integer sum, so results are deterministic and
// independent of the launch shape and of other jobs sharing the launch.
#include <cstddef>
#include <cstdint>

#include "internal.h"

namespace prdpt {

constexpr unsigned kFull = 0xffffffffu;  // all lanes of a warp

// Programmatic dependent launch: the kernels of a step are launched so that the next one
// may be scheduled while the previous one drains. Each kernel reads only host-written data
// (job descriptors, the base scene) before pdl_enter, which waits until every kernel
// before it in the stream has completed and its writes are visible (a no-op for a launch
// without the attribute), then lets the next kernel be scheduled.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 xyz(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalized(float3 a) { return a * rsqrtf(dot3(a, a)); }
__device__ __forceinline__ float maxc(float3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }
// Approximate reciprocal (MUFU.RCP, 1 ulp); +-0 gives +-inf as the slab test needs.
__device__ __forceinline__ float3 rcp3(float3 d) {
    return f3(__fdividef(1.0f, d.x), __fdividef(1.0f, d.y), __fdividef(1.0f, d.z));
}
__device__ __forceinline__ int as_int(float f) { return __float_as_int(f); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and the open-interval uniform
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, unsigned k0, unsigned k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same generator kept out of line: one copy of its code instead of one per call site,
// for the kernels whose code outgrows the instruction cache (emitter sharing, render groups;
// measured: caustic step 7.16 -> 6.72 ms).
__device__ __noinline__ uint4 philox_ool(uint4 c, unsigned k0, unsigned k1) { return philox(c, k0, k1); }

// ((x >> 9) * 2 + 1) / 2^24: exact in FP32, never 0, 1 or 1/2.
__device__ __forceinline__ float u01(unsigned x) { return __uint2float_rn((x >> 9) * 2u + 1u) * 0x1p-24f; }

// ---------------------------------------------------------------------------
// Perturbation sampler (Sec. 3.2; Eq. 11 positivized; supplemental inverse CDF)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int sampler_uniforms(int mode, int D) {
    if (mode == kRadial) {
        if (D == 1) return 2;
        const int n_exp = (D + 1) / 2, extra = (D % 2 == 0);
        return n_exp + 2 * ((D + extra + 1) / 2);
    }
    if (mode == kPerDim) return D;
    return 2 * ((D + 1) / 2);
}

// Box-Muller normal number j of the pairs starting at uniform index `base`.
__device__ __forceinline__ float bm_normal(const float* u, int base, int j) {
    const float a = u[base + 2 * (j / 2)], b = u[base + 2 * (j / 2) + 1];
    const float rad = sqrtf(-2.0f * logf(a));
    float s, c;
    sincospif(2.0f * b, &s, &c);
    return rad * ((j & 1) ? s : c);
}

// Bandwidth at step t: constant, or the warm-started linear decay (Sec. 3.3).
__device__ __forceinline__ float sigma_sched(const float* sigma, int anneal, int total_steps, float sigma_min, int d,
                                             int t) {
    const float s0 = sigma[d];
    if (!anneal) return s0;
    const int w = total_steps / 2;
    if (t < w || total_steps - w <= 0) return s0;
    float frac = float(t - w) / float(total_steps - w);
    frac = fminf(frac, 1.0f);
    return s0 - frac * (s0 - sigma_min);
}
__device__ __forceinline__ float sigma_at(const InstJob& J, int d, int t) {
    return sigma_sched(J.sigma, J.anneal, J.total_steps, J.sigma_min, d, t);
}

// Axis-aligned bounds of a primitive record, inflated by 1e-3 scene units plus 1e-5
// relative, so that a slab test against them is conservative for the exact FP32
// intersection tests of the primitive (path sharing).
__device__ __forceinline__ void prim_bounds(const float4* P, int type, float3& lo, float3& hi) {
    if (type == kSphere) {
        const float4 c = P[0];
        const float rad = fabsf(c.w);
        lo = f3(c.x - rad, c.y - rad, c.z - rad);
        hi = f3(c.x + rad, c.y + rad, c.z + rad);
    } else if (type == kQuad) {
        const float3 c = xyz(P[0]), u = xyz(P[2]), v = xyz(P[3]);
        const float3 e = f3(0.5f * (fabsf(u.x) + fabsf(v.x)), 0.5f * (fabsf(u.y) + fabsf(v.y)),
                            0.5f * (fabsf(u.z) + fabsf(v.z)));
        lo = c - e;
        hi = c + e;
    } else {
        lo = xyz(P[0]);
        hi = xyz(P[1]);
    }
    const float3 m = f3(1e-3f + 1e-5f * fmaxf(fabsf(lo.x), fabsf(hi.x)), 1e-3f + 1e-5f * fmaxf(fabsf(lo.y), fabsf(hi.y)),
                        1e-3f + 1e-5f * fmaxf(fabsf(lo.z), fabsf(hi.z)));
    lo = lo - m;
    hi = hi + m;
}

// ---------------------------------------------------------------------------
// k_instantiate: one CTA (kInstBlock threads) per render
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kInstBlock) k_instantiate(const InstLaunch L) {
    __shared__ float s_u[4 * 32];
    __shared__ float s_red[kInstBlock];
    __shared__ float s_theta[kMaxD];
    __shared__ float s_scalar[2];
    __shared__ int s_job;
    __shared__ __align__(16) BaseScene s_base;  // the job's base scene, staged once (int4 stores)
    __shared__ InstScene s_inst;  // render r's scene, built here and written out in one copy

    const int tid = threadIdx.x;
    // Before waiting on the previous kernel: only data the host wrote (job descriptors, the
    // base scene). Parameters, step counters and work counters come after the wait.
    if (tid == 0) {
        int j = 0;
        if (L.jobs) {
            int lo = 0, hi = L.njobs - 1;  // last job with block_begin <= blockIdx.x
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (L.jobs[mid].block_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
            }
            j = lo;
        }
        s_job = j;
    }
    __syncthreads();
    const InstJob& J = L.jobs ? L.jobs[s_job] : L.job0;
    const int r = blockIdx.x - J.block_begin;
    const int D = J.D;
    {  // stage the base scene: all loads in flight at once, then the shared-memory stores
        constexpr int n16 = int(sizeof(BaseScene) / 16), n4 = int(sizeof(BaseScene) / 4);
        constexpr int kPer = (n16 + kInstBlock - 1) / kInstBlock;
        if (J.base && (reinterpret_cast<size_t>(J.base) & 15) == 0) {
            const int4* src = reinterpret_cast<const int4*>(J.base);
            int4* dst = reinterpret_cast<int4*>(&s_base);
            int4 v[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q)
                if (tid + q * kInstBlock < n16) v[q] = __ldg(src + tid + q * kInstBlock);
#pragma unroll
            for (int q = 0; q < kPer; ++q)
                if (tid + q * kInstBlock < n16) dst[tid + q * kInstBlock] = v[q];
            for (int i = 4 * n16 + tid; i < n4; i += kInstBlock)
                reinterpret_cast<int*>(&s_base)[i] = __ldg(reinterpret_cast<const int*>(J.base) + i);
        } else if (J.base) {
            for (int i = tid; i < n4; i += kInstBlock)
                reinterpret_cast<int*>(&s_base)[i] = __ldg(reinterpret_cast<const int*>(J.base) + i);
        }
    }
    pdl_enter();
    if (blockIdx.x == 0 && tid == 0) {
        if (L.queue_reset) *L.queue_reset = 0u;
        if (L.queue_reset2) *L.queue_reset2 = 0u;
        if (L.queue_reset3) *L.queue_reset3 = 0u;
        if (L.queue_reset4) *L.queue_reset4 = 0u;
    }
    if (r == 0 && tid == 0 && J.share_reset)
        for (int i = 0; i < 4; ++i) J.share_reset[i] = 0u;
    if (tid == 0 && J.aff_cursor) J.aff_cursor[r] = 0u;
    if (J.aff_flags)  // this render's corrected-block bits, read by the last step's epilogue
        for (int i = tid; i < J.flag_words; i += kInstBlock) J.aff_flags[size_t(r) * J.flag_words + i] = 0u;
    const unsigned step = J.step + (J.step_dev ? (unsigned)*J.step_dev : 0u);
    const float theta_d = (tid < D && J.theta) ? J.theta[(J.render_mode ? r * D : 0) + tid] : 0.0f;
    __syncthreads();

    // ---- a1: perturbation and weight of render r --------------------------------
    // (texture scenes: the draws are made by the high-dimensional kernels, k_hd_*)
    const bool texscene = J.base && s_base.tex_mat >= 0;
    if (texscene) {
    } else if (J.render_mode) {
        if (tid < D) s_theta[tid] = theta_d;
    } else {
        const bool anti = J.antithetic && (r & 1);
        const unsigned index = (J.antithetic ? unsigned(r >> 1) : unsigned(r)) +
                               unsigned(J.antithetic ? J.pair_begin : 2 * J.pair_begin);
        const int nu = sampler_uniforms(J.sampler, D);
        const int nblk = (nu + 3) / 4;
        if (tid < nblk) {
            const uint4 w = philox(make_uint4(index, tid, step, kTagPerturb << 28), unsigned(J.seed),
                                   unsigned(J.seed >> 32));
            s_u[4 * tid + 0] = u01(w.x);
            s_u[4 * tid + 1] = u01(w.y);
            s_u[4 * tid + 2] = u01(w.z);
            s_u[4 * tid + 3] = u01(w.w);
        }
        __syncthreads();
        float tt = 0.0f, wt = 0.0f;  // unit-bandwidth tau~_d and w~_d of this thread's d
        if (J.sampler == kRadial && D == 1) {
            if (tid == 0) {
                const float rho = sqrtf(-2.0f * logf(s_u[0]));
                const float sg = (s_u[1] < 0.5f) ? -1.0f : 1.0f;
                tt = sg * rho;
                wt = sg * J.c_radial;
            }
        } else if (J.sampler == kRadial) {
            const int n_exp = (D + 1) / 2, extra = (D % 2 == 0);
            const float z = (tid < D) ? bm_normal(s_u, n_exp, tid) : 0.0f;
            // squared direction norm and chi^2_{D+1} radius, summed in a fixed order
            s_red[tid] = z * z;
            __syncthreads();
            if (tid == 0) {
                float zn = 0.0f;
                for (int d = 0; d < D; ++d) zn += s_red[d];
                float r2 = 0.0f;
                for (int j = 0; j < n_exp; ++j) r2 += -2.0f * logf(s_u[j]);
                if (extra) {  // one more degree of freedom when D + 1 is odd: normal number D
                    const float ze = bm_normal(s_u, n_exp, D);
                    r2 += ze * ze;
                }
                s_scalar[0] = sqrtf(zn);
                s_scalar[1] = r2;
            }
            __syncthreads();
            if (tid < D) {
                const float dir = z / s_scalar[0];
                tt = sqrtf(s_scalar[1]) * dir;
                wt = J.c_radial * dir;
            }
        } else if (J.sampler == kPerDim) {
            if (tid < D) {
                const float xi = s_u[tid];
                const float c1 = 0.7978845608028654f;  // sqrt(2/pi)
                if (xi < 0.5f) {
                    tt = -sqrtf(-2.0f * logf(2.0f * xi));
                    wt = -c1;
                } else {
                    tt = sqrtf(-2.0f * logf(2.0f * (1.0f - xi)));
                    wt = c1;
                }
            }
        } else {
            if (tid < D) {
                tt = bm_normal(s_u, 0, tid);
                wt = tt;
            }
        }
        if (tid < D) {
            const float sg = sigma_at(J, tid, (int)step);
            float tau = sg * tt;
            float w = wt / sg;
            if (anti) {
                tau = -tau;
                w = -w;
            }
            s_theta[tid] = theta_d + tau;  // FP32 sum: the parameters this render gets
            if (J.tau_out) J.tau_out[r * D + tid] = tau;
            if (J.w_out) J.w_out[r * D + tid] = w;
        }
    }
    __syncthreads();
    if (!J.scenes) return;  // draws only

    // ---- a2: bind theta_r into the scene -----------------------------------------
    const BaseScene& B = s_base;
    InstScene& S = s_inst;
    if (tid < kMaxDiff) {  // pathwise estimator: derivative of each parameter's clamp
        float dc = 0.0f;
        if (J.diff && !texscene && tid < D) {
            const float t = s_theta[tid];
            dc = B.bind_kind[tid] == kBindAlbedo ? ((t >= 0.0f && t <= 1.0f) ? 1.0f : 0.0f) : (t >= 0.0f ? 1.0f : 0.0f);
        }
        S.dclamp[tid] = dc;
    }
    if (tid < B.n_prims) {
        const int i = tid;
        const int type = B.prim_type[i], mat = B.prim_mat[i], slot = B.prim_slot[i];
        float g[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) g[q] = B.prim_geom[i][q];
        for (int d = 0; d < (texscene ? 0 : D); ++d) {
            if (B.bind_index[d] != i) continue;
            if (B.bind_kind[d] == kBindPos) g[B.bind_comp[d]] = s_theta[d];
            if (B.bind_kind[d] == kBindRadius && type == kSphere) g[3] = fabsf(s_theta[d]);
        }
        float4* P = S.prim[slot];
        const float3 c = f3(g[0], g[1], g[2]);
        if (type == kSphere) {
            P[0] = make_float4(c.x, c.y, c.z, g[3]);
            P[1] = make_float4(g[3] * g[3], 1.0f / g[3], __int_as_float(mat), __int_as_float(i));
        } else if (type == kQuad) {
            const float3 u = f3(g[3], g[4], g[5]), v = f3(g[6], g[7], g[8]);
            const float3 n = normalized(cross3(u, v));
            P[0] = make_float4(c.x, c.y, c.z, __int_as_float(mat));
            P[1] = make_float4(n.x, n.y, n.z, __int_as_float(i));
            P[2] = make_float4(u.x, u.y, u.z, 1.0f / dot3(u, u));
            P[3] = make_float4(v.x, v.y, v.z, 1.0f / dot3(v, v));
        } else {
            P[0] = make_float4(g[0] - g[3], g[1] - g[4], g[2] - g[5], __int_as_float(mat));
            P[1] = make_float4(g[0] + g[3], g[1] + g[4], g[2] + g[5], __int_as_float(i));
        }
    }
    if (tid < B.n_mats) {
        const int i = tid;
        float p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) p[q] = B.mat_param[i][q];
        for (int d = 0; d < (texscene ? 0 : D); ++d) {
            if (B.bind_index[d] != i) continue;
            if (B.bind_kind[d] == kBindAlbedo) p[B.bind_comp[d]] = s_theta[d];
            if (B.bind_kind[d] == kBindEmission) p[3 + B.bind_comp[d]] = s_theta[d];
        }
        for (int q = 0; q < 3; ++q) p[q] = fminf(fmaxf(p[q], 0.0f), 1.0f);
        for (int q = 3; q < 6; ++q) p[q] = fmaxf(p[q], 0.0f);
        S.mat[i][0] = make_float4(p[0], p[1], p[2], __int_as_float(B.mat_type[i]));
        S.mat[i][1] = make_float4(p[3], p[4], p[5], p[6]);
    }
    __syncthreads();
    if (J.var_box && tid < J.n_var) {  // path sharing: this render's bounds of a perturbed primitive
        const int i = J.var_prim[tid];
        float3 lo, hi;
        prim_bounds(S.prim[B.prim_slot[i]], B.prim_type[i], lo, hi);
        J.var_box[(size_t(r) * kMaxVariant + tid) * 2 + 0] = make_float4(lo.x, lo.y, lo.z, 0.0f);
        J.var_box[(size_t(r) * kMaxVariant + tid) * 2 + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
    }
    if (tid == 0) {
        S.tex = texscene ? J.tex_all + size_t(r) * size_t(J.tex_D) : nullptr;
        S.tex_mat = texscene ? B.tex_mat : -1;
        S.tex_res = texscene ? B.tex_res : 0;
        S.n_sph = B.n_sph;
        S.n_quad = B.n_quad;
        S.n_box = B.n_box;
        const unsigned field =
            J.render_mode ? (J.crn ? 0u : unsigned(r)) : (J.crn ? 0u : unsigned(r + 1 + 2 * J.pair_begin));
        S.seed_lo = unsigned(J.seed);
        S.seed_hi = unsigned(J.seed >> 32);
        S.step = step;
        S.c3 = (J.tag << 28) | (field & 0x0fffffffu);
        S.eye = make_float4(B.eye[0], B.eye[1], B.eye[2], B.tan_half);
        S.fwd = make_float4(B.fwd[0], B.fwd[1], B.fwd[2], float(J.W) / float(J.H));
        S.right = make_float4(B.right[0], B.right[1], B.right[2], 0.0f);
        S.up = make_float4(B.up[0], B.up[1], B.up[2], 0.0f);
        S.bg = make_float4(B.bg[0], B.bg[1], B.bg[2], 0.0f);
        int nl = 0;
        for (int i = 0; i < B.n_prims && nl < kMaxLights; ++i) {  // emitters, in primitive order
            const int mat = B.prim_mat[i];
            const float4 e = S.mat[mat][1];
            if (!(e.x > 0.0f || e.y > 0.0f || e.z > 0.0f) || B.prim_type[i] == kBox) continue;
            const int slot = B.prim_slot[i];
            float area;
            if (B.prim_type[i] == kQuad) {
                const float3 u = xyz(S.prim[slot][2]), v = xyz(S.prim[slot][3]);
                const float3 cr = cross3(u, v);
                area = sqrtf(dot3(cr, cr));
            } else {
                const float rad = S.prim[slot][0].w;
                area = 4.0f * 3.14159265358979f * rad * rad;
            }
            S.light[nl] = make_int4(B.prim_type[i], slot, i, mat);
            S.light_area[nl] = area;
            ++nl;
        }
        S.n_lights = nl;
    }
    __syncthreads();
    {  // write out what the render kernels stage: header, used materials, used primitives
        const float4* src = reinterpret_cast<const float4*>(&s_inst);
        float4* dst = reinterpret_cast<float4*>(J.scenes + r);
        constexpr int kHead = int(offsetof(InstScene, mat) / 16);
        constexpr int kPrim = int(offsetof(InstScene, prim) / 16);
        const int nm = 2 * B.n_mats, np = 4 * B.n_prims;
        for (int i = tid; i < kHead + nm + np; i += kInstBlock) {
            const int o = (i < kHead + nm) ? i : kPrim + (i - kHead - nm);
            dst[o] = src[o];
        }
    }
}

// ---------------------------------------------------------------------------
// Ray casting against the shared-memory scene (brute force over <= 32 primitives)
// ---------------------------------------------------------------------------
// Work counters (only counted when the launch asks for them): primitive tests by
// type, camera paths, surface vertices, shadow rays, closest-hit rays.
constexpr int kNumCounters = 8;
struct Counters {
    unsigned sph, quad, box, paths, vertices, shadow, rays, pad;
};

// The intersection tests read a primitive record through P[j]: a pointer to its four float4,
// or a strided view of a per-render table (SRec).
template <class Rec>
__device__ __forceinline__ float sphere_t(const Rec& P, float3 o, float3 d) {
    const float4 a = P[0];
    const float r2 = P[1].x;
    const float3 oc = o - xyz(a);
    const float b = dot3(oc, d);
    const float3 l = oc - d * b;  // centre offset from the ray line: better conditioned than b^2 - c
    const float disc = r2 - dot3(l, l);
    if (!(disc > 0.0f)) return INFINITY;  // tangent rays (disc == 0) count as misses
    const float sq = disc * rsqrtf(disc);
    float t = -b - sq;
    if (t <= kEps) t = -b + sq;
    return (t > kEps) ? t : INFINITY;
}

template <class Rec>
__device__ __forceinline__ float quad_t(const Rec& P, float3 o, float3 d) {
    const float4 a = P[0], nb = P[1], uu = P[2], vv = P[3];
    const float3 n = xyz(nb);
    const float den = dot3(n, d);
    if (fabsf(den) < 1e-12f) return INFINITY;
    const float3 co = xyz(a) - o;
    const float t = __fdividef(dot3(n, co), den);
    if (!(t > kEps)) return INFINITY;
    const float3 q = d * t - co;  // hit point relative to the centre
    const float pa = dot3(q, xyz(uu)) * uu.w, pb = dot3(q, xyz(vv)) * vv.w;
    return (fabsf(pa) <= 0.5f && fabsf(pb) <= 0.5f) ? t : INFINITY;
}

// Slab test; returns the nearest t > eps (entering, or leaving from inside).
template <class Rec>
__device__ __forceinline__ float box_t(const Rec& P, float3 o, float3 inv) {
    const float3 lo = xyz(P[0]), hi = xyz(P[1]);
    const float tx0 = (lo.x - o.x) * inv.x, tx1 = (hi.x - o.x) * inv.x;
    const float ty0 = (lo.y - o.y) * inv.y, ty1 = (hi.y - o.y) * inv.y;
    const float tz0 = (lo.z - o.z) * inv.z, tz1 = (hi.z - o.z) * inv.z;
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fminf(tz0, tz1));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    if (tn > tf) return INFINITY;
    if (tn > kEps) return tn;
    return (tf > kEps) ? tf : INFINITY;
}

// Outward normal of box record P at the hit found by box_t.
template <class Rec>
__device__ __forceinline__ float3 box_normal(const Rec& P, float3 o, float3 d, float3 inv) {
    const float3 lo = xyz(P[0]), hi = xyz(P[1]);
    float tn[3], tf[3];
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z}, ii[3] = {inv.x, inv.y, inv.z};
    const float l3[3] = {lo.x, lo.y, lo.z}, h3[3] = {hi.x, hi.y, hi.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t0 = (l3[a] - oo[a]) * ii[a], t1 = (h3[a] - oo[a]) * ii[a];
        tn[a] = fminf(t0, t1);
        tf[a] = fmaxf(t0, t1);
    }
    int an = 0, af = 0;
    float bn = tn[0], bf = tf[0];
#pragma unroll
    for (int a = 1; a < 3; ++a) {
        if (tn[a] > bn) { bn = tn[a]; an = a; }
        if (tf[a] < bf) { bf = tf[a]; af = a; }
    }
    const bool entering = bn > kEps;
    const int axis = entering ? an : af;
    const float s = (dd[axis] > 0.0f ? 1.0f : -1.0f) * (entering ? -1.0f : 1.0f);
    return f3(axis == 0 ? s : 0.0f, axis == 1 ? s : 0.0f, axis == 2 ? s : 0.0f);
}

struct Hit {
    float t;
    int slot;   // record slot, -1 = miss
    int type;
};

// Closest hit over all primitives, grouped by type. With kSkip, primitives whose
// record slot is set in `skip` are left out (the perturbed ones, in shared mode).
template <bool kCount, bool kSkip, class Scn>
__device__ __forceinline__ Hit closest_hit(const Scn& S, float3 o, float3 d, Counters& cnt, unsigned skip) {
    Hit h{INFINITY, -1, 0};
    const int ns = S.n_sph, nq = S.n_quad, nb = S.n_box;
    if (kCount) {
        const unsigned sk = kSkip ? skip : 0u;
        cnt.sph += ns - __popc(sk & ((1u << ns) - 1u));
        cnt.quad += nq - __popc((sk >> ns) & ((1u << nq) - 1u));
        cnt.box += nb - __popc((sk >> (ns + nq)) & ((1u << nb) - 1u));
        ++cnt.rays;
    }
    for (int i = 0; i < ns; ++i) {
        if (kSkip && ((skip >> i) & 1u)) continue;
        const float t = sphere_t(S.prim[i], o, d);
        if (t < h.t) { h.t = t; h.slot = i; h.type = kSphere; }
    }
    for (int i = ns; i < ns + nq; ++i) {
        if (kSkip && ((skip >> i) & 1u)) continue;
        const float t = quad_t(S.prim[i], o, d);
        if (t < h.t) { h.t = t; h.slot = i; h.type = kQuad; }
    }
    if (nb) {
        const float3 inv = rcp3(d);
        for (int i = ns + nq; i < ns + nq + nb; ++i) {
            if (kSkip && ((skip >> i) & 1u)) continue;
            const float t = box_t(S.prim[i], o, inv);
            if (t < h.t) { h.t = t; h.slot = i; h.type = kBox; }
        }
    }
    return h;
}

// Is anything but primitive slot `light` (and, with kSkip, the slots in `skip`) hit
// closer than dist?
template <bool kCount, bool kSkip, class Scn>
__device__ __forceinline__ bool occluded(const Scn& S, float3 o, float3 d, float dist, int light,
                                         Counters& cnt, unsigned skip) {
    const int ns = S.n_sph, nq = S.n_quad, nb = S.n_box;
    if (kCount) ++cnt.shadow;
    for (int i = 0; i < ns; ++i) {
        if (i == light || (kSkip && ((skip >> i) & 1u))) continue;
        if (kCount) ++cnt.sph;
        if (sphere_t(S.prim[i], o, d) < dist) return true;
    }
    for (int i = ns; i < ns + nq; ++i) {
        if (i == light || (kSkip && ((skip >> i) & 1u))) continue;
        if (kCount) ++cnt.quad;
        if (quad_t(S.prim[i], o, d) < dist) return true;
    }
    if (nb) {
        const float3 inv = rcp3(d);
        for (int i = ns + nq; i < ns + nq + nb; ++i) {
            if (i == light || (kSkip && ((skip >> i) & 1u))) continue;
            if (kCount) ++cnt.box;
            if (box_t(S.prim[i], o, inv) < dist) return true;
        }
    }
    return false;
}

// Render-group mode: the lanes of a warp trace the same path samples for up to 32
// renders of a job at once (with common random numbers the renders' paths agree until a
// perturbed primitive intervenes, so the lanes stay coherent). The invariant part of the
// scene is the warp's staged InstScene; each lane reads what differs between renders from
// its row of a per-warp table:
//   [4 k .. 4 k + 3]   record of the k-th perturbed primitive (in record-slot order)
//   [4 n + j]          albedo row (albedo, type) of the j-th bound material (only albedos
//                      are bound in this mode; the emission row is the staged scene's)
//   [4 n + m .. + 1]   the render's emitter areas (8 floats), only when a radius binding
//                      can change an emitter's area (m = bound materials)
// A record in a per-render table kept field-major (field j of every render contiguous), so
// that lanes reading their own renders' fields load consecutive float4 without bank
// conflicts: field j at p[j * s].
struct SRec {
    const float4* p;
    int s;
    __device__ __forceinline__ float4 operator[](int j) const { return p[j * s]; }
};

struct GroupLane {
    const float4* rec;  // this lane's row: field q at rec[q * rs]
    unsigned prims;     // record-slot mask of the perturbed primitives
    unsigned mats;      // mask of the bound materials
    int n_var;          // perturbed primitives
    int areas;          // 1: the row holds the emitter areas
    const uint4* rng;   // the sample group's Philox blocks: [0] jitter, [1 + 2 b + k] vertex b, slot k
    int bpre;           // vertices b < bpre have their blocks in `rng`
    int rs;             // float4 between consecutive fields of a row (the table's render count)
};

// Record of primitive slot `slot`: the lane's own for a perturbed primitive, else the
// staged scene's.
template <bool kGroup, class Scn>
__device__ __forceinline__ auto prim_rec(const Scn& S, int slot, const GroupLane* g) {
    if constexpr (kGroup) {
        if ((g->prims >> slot) & 1u) return SRec{g->rec + 4 * __popc(g->prims & ((1u << slot) - 1u)) * g->rs, g->rs};
        return SRec{S.prim[slot], 1};
    } else {
        return static_cast<const float4*>(S.prim[slot]);
    }
}

// Albedo row (albedo, type) of material m: the lane's own for a bound material.
template <bool kGroup, class Scn>
__device__ __forceinline__ float4 mat_albedo(const Scn& S, int m, const GroupLane* g) {
    if constexpr (kGroup) {
        if ((g->mats >> m) & 1u) return g->rec[(4 * g->n_var + __popc(g->mats & ((1u << m) - 1u))) * g->rs];
    }
    return S.mat[m][0];
}

template <bool kGroup, class Scn>
__device__ __forceinline__ float light_area(const Scn& S, int li, const GroupLane* g) {
    if constexpr (kGroup) {
        if (g->areas)
            return reinterpret_cast<const float*>(g->rec + (4 * g->n_var + __popc(g->mats) + (li >> 2)) * g->rs)[li & 3];
    }
    return S.light_area[li];
}

// The lane's perturbed primitives against a ray: closer hits replace h (the staged scene's
// closest hit over the other primitives).
template <bool kCount, class Scn>
__device__ __forceinline__ void group_hit(const Scn& S, const GroupLane& g, float3 o, float3 d, Hit& h,
                                          Counters& cnt) {
    unsigned m = g.prims;
    for (int k = 0; m; ++k) {
        const int slot = __ffs(m) - 1;
        m &= m - 1u;
        const SRec P{g.rec + 4 * k * g.rs, g.rs};
        float t;
        int type;
        if (slot < S.n_sph) {
            t = sphere_t(P, o, d);
            type = kSphere;
            if (kCount) ++cnt.sph;
        } else if (slot < S.n_sph + S.n_quad) {
            t = quad_t(P, o, d);
            type = kQuad;
            if (kCount) ++cnt.quad;
        } else {
            t = box_t(P, o, rcp3(d));
            type = kBox;
            if (kCount) ++cnt.box;
        }
        if (t < h.t) { h.t = t; h.slot = slot; h.type = type; }
    }
}

// Is one of the lane's perturbed primitives other than slot `light` hit closer than dist?
template <bool kCount, class Scn>
__device__ __forceinline__ bool group_occluded(const Scn& S, const GroupLane& g, float3 o, float3 d, float dist,
                                               int light, Counters& cnt) {
    unsigned m = g.prims;
    for (int k = 0; m; ++k) {
        const int slot = __ffs(m) - 1;
        m &= m - 1u;
        if (slot == light) continue;
        const SRec P{g.rec + 4 * k * g.rs, g.rs};
        float t;
        if (slot < S.n_sph) {
            t = sphere_t(P, o, d);
            if (kCount) ++cnt.sph;
        } else if (slot < S.n_sph + S.n_quad) {
            t = quad_t(P, o, d);
            if (kCount) ++cnt.quad;
        } else {
            t = box_t(P, o, rcp3(d));
            if (kCount) ++cnt.box;
        }
        if (t < dist) return true;
    }
    return false;
}

// Union over the job's R renders of the perturbed primitives' bounds (shared mode; each
// render's bounds are inflated so that a slab test is conservative against the exact
// intersection tests), and the pool that keeps the segments touching them.
// One live path sample (Eq. 1's integrand along one path; Eq. 3 averages them).
struct Path {
    float3 o, d, beta, L;
    unsigned pixel;  // y * W + x
    int s, b;        // sample index, vertex index
    int slot;        // pixel slot inside the warp's block (per-render pass: the path's record)
    bool specular;   // emission counts: camera rays and rays after specular bounces
    unsigned seg;    // shared pass: touching-segment word (see note_touch)
};

struct VarBoxes {
    float4 lo[kMaxVariant], hi[kMaxVariant];  // union over renders
    float4* seg_pool;                         // touching segments, kSeg slots per path
    float4* seg_state;                        // 4 per path group: where the path's renders part
    unsigned* seg_ctr;                        // slots claimed
    unsigned seg_cap;                         // slots available
    int n;
    unsigned skip, mats;
};

// Does the segment o + t inv^-1, 0 <= t <= tm, touch the box [lo, hi]?
__device__ __forceinline__ bool slab_touch(float3 lo, float3 hi, float3 o, float3 inv, float tm) {
    const float tx0 = (lo.x - o.x) * inv.x, tx1 = (hi.x - o.x) * inv.x;
    const float ty0 = (lo.y - o.y) * inv.y, ty1 = (hi.y - o.y) * inv.y;
    const float tz0 = (lo.z - o.z) * inv.z, tz1 = (hi.z - o.z) * inv.z;
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tm));
    return tn <= tf;
}

// Touching segments of a shared-pass path. A path that touches a union box of the
// perturbed primitives claims a group g of kSeg segment slots and keeps, besides the
// segments, its state at the start of the vertex of the first touch: up to there none of
// its rays can meet a render's own primitive, so every render's path agrees with the
// shared one and the per-render pass resumes from that state instead of the camera.
// A path's segment word p.seg is
//   0                          no ray touched a union box;
//   (g + 1) << 3 | count       count <= kSeg touching segments (o, tmax), (d, 0) in slots
//                              kSeg g ..; a render traces the path again only if one of them
//                              touches that render's own bounds;
//   kSegAll | (g + 1) << 3     every render traces the path again from state g (a bound
//                              material was hit, or more than kSeg segments touched);
//   kSegFull                   every render traces the path again from the camera (the pool
//                              ran out before the first touch).
// State g: (o, d.x), (d.y, d.z, beta.x, beta.y), (beta.z, L), (vertex b, emission flag).
// A first touch by a shadow ray is kept as the vertex's state after its emission was
// added (o and d from the stash below), with the emission flag cleared so that the
// resumed vertex does not add it again.
constexpr unsigned kSegAll = 0x80000000u, kSegFull = 0xffffffffu;

// Ray (o, d) of each shared-pass thread's current vertex, kept while its path has not
// touched (a shadow ray's first touch records the vertex's state).
__shared__ float s_stash[6][kBlock];

template <bool kNee>
__device__ __forceinline__ unsigned open_group(const VarBoxes& V, const Path& p) {
    const unsigned base = atomicAdd(V.seg_ctr, unsigned(kSeg));
    if (base + unsigned(kSeg) > V.seg_cap) return kSegFull;
    const unsigned g = base / unsigned(kSeg);
    float3 o = p.o, d = p.d;
    if (kNee) {
        const int t = threadIdx.x;
        o = f3(s_stash[0][t], s_stash[1][t], s_stash[2][t]);
        d = f3(s_stash[3][t], s_stash[4][t], s_stash[5][t]);
    }
    float4* st = V.seg_state + 4 * size_t(g);
    st[0] = make_float4(o.x, o.y, o.z, d.x);
    st[1] = make_float4(d.y, d.z, p.beta.x, p.beta.y);
    st[2] = make_float4(p.beta.z, p.L.x, p.L.y, p.L.z);
    st[3] = make_float4(__int_as_float(p.b), __int_as_float((!kNee && p.specular) ? 1 : 0), 0.0f, 0.0f);
    return (g + 1u) << 3;
}

// Test the segment o + t d, 0 <= t <= tmax, of path p against the union boxes and keep it
// if it touches (kNee: a shadow ray). The caller returns kAffected once kSegAll is set.
template <bool kCount, bool kNee>
__device__ __forceinline__ void note_touch(const VarBoxes& V, float3 o, float3 d, float tmax, Path& p,
                                           Counters& cnt) {
    const float3 inv = rcp3(d);
    const float tm = tmax * 1.0001f + 1e-3f;
    bool hit = false;
    for (int k = 0; k < V.n; ++k) hit = hit || slab_touch(xyz(V.lo[k]), xyz(V.hi[k]), o, inv, tm);
    if (kCount) cnt.box += V.n;
    if (!hit) return;
    unsigned seg = p.seg;
    if (seg == 0u) {
        seg = open_group<kNee>(V, p);
        if (seg == kSegFull) {
            p.seg = kSegFull;
            return;
        }
    } else if ((seg & 7u) == unsigned(kSeg)) {
        p.seg = seg | kSegAll;
        return;
    }
    const size_t slot = size_t((seg >> 3) - 1u) * kSeg + (seg & 7u);
    V.seg_pool[2 * slot + 0] = make_float4(o.x, o.y, o.z, tmax);
    V.seg_pool[2 * slot + 1] = make_float4(d.x, d.y, d.z, 0.0f);
    p.seg = seg + 1u;
}

template <bool kOol = false, class Scn>
__device__ __forceinline__ uint4 path_words(const Scn& S, unsigned pixel, int s, int b, int slot) {
    const unsigned c1 = unsigned(s) | (unsigned(b) << 16) | (unsigned(slot) << 24);
    if constexpr (kOol) return philox_ool(make_uint4(pixel, c1, S.step, S.c3), S.seed_lo, S.seed_hi);
    return philox(make_uint4(pixel, c1, S.step, S.c3), S.seed_lo, S.seed_hi);
}

// Block `slot` of the path's current vertex: from the render group's table while the
// vertex is within it (the same words, drawn ahead by the group's lanes), else drawn here.
template <bool kGroup, bool kOol = false, class Scn>
__device__ __forceinline__ uint4 vertex_words(const Scn& S, const Path& p, int slot, const GroupLane* gl) {
    if constexpr (kGroup) {
        if (p.b < gl->bpre) return gl->rng[1 + 2 * p.b + slot];
    }
    return path_words<kOol>(S, p.pixel, p.s, p.b, slot);
}

// Orthonormal basis around unit n (Duff et al. 2017).
__device__ __forceinline__ void onb(float3 n, float3& t1, float3& t2) {
    const float sg = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = __fdividef(-1.0f, sg + n.z);
    const float b = n.x * n.y * a;
    t1 = f3(1.0f + sg * n.x * n.x * a, sg * b, -sg * n.x);
    t2 = f3(b, sg + n.y * n.y * a, -n.y);
}

// Albedo of a textured quad at hit point pt: texel (floor(s T), floor(t T)) with
// s = (pt - c).u / |u|^2 + 1/2, t = (pt - c).v / |v|^2 + 1/2 (each clamped to [0, T-1]) of
// the render's texture [T][T][3]; channels clamped to [0, 1].
template <class Scn, class Rec>
__device__ __forceinline__ float3 tex_albedo(const Scn& S, const Rec& P, float3 pt) {
    const float4 c = P[0], u = P[2], v = P[3];
    const float3 l = pt - xyz(c);
    const float s = fmaf(dot3(l, xyz(u)), u.w, 0.5f), t = fmaf(dot3(l, xyz(v)), v.w, 0.5f);
    const int T = S.tex_res;
    const int tx = min(max(int(floorf(s * float(T))), 0), T - 1);
    const int ty = min(max(int(floorf(t * float(T))), 0), T - 1);
    const float* q = S.tex + (size_t(ty) * T + tx) * 3;
    return f3(fminf(fmaxf(__ldg(q), 0.0f), 1.0f), fminf(fmaxf(__ldg(q + 1), 0.0f), 1.0f),
              fminf(fmaxf(__ldg(q + 2), 0.0f), 1.0f));
}

// Camera ray of sample s through pixel (x, y): pinhole, box-filtered jitter (slot 2). The
// jitter block is drawn here unless the caller passes it (`pre`).
template <bool kOol = false, class Scn>
__device__ __forceinline__ void start_path(const Scn& S, int W, int H, int x, int y, int s, int slot,
                                           Path& p, const uint4* pre = nullptr) {
    p.pixel = unsigned(y * W + x);
    const uint4 jw = pre ? *pre : path_words<kOol>(S, p.pixel, s, 0, 2);
    const float th = S.eye.w, aspect = S.fwd.w;
    const float sx = (float(2 * x - W) + 2.0f * u01(jw.x)) * __fdividef(aspect * th, float(W));
    const float sy = (float(H - 2 * y) - 2.0f * u01(jw.y)) * __fdividef(th, float(H));
    p.o = xyz(S.eye);
    p.d = normalized(xyz(S.fwd) + xyz(S.right) * sx + xyz(S.up) * sy);
    p.L = f3(0.f, 0.f, 0.f);
    p.beta = f3(1.f, 1.f, 1.f);
    p.s = s;
    p.b = 0;
    p.slot = slot;
    p.specular = true;
}

// One surface interaction of a path: unidirectional path tracing with next-event
// estimation on diffuse vertices. Returns kEnded when the path has ended.
// Random slots of vertex b: slot 0 = (light point u, v, BSDF u1, u2); slot 1 =
// (light choice, Russian roulette, dielectric choice), drawn only when needed.
//
// With kShared (path sharing across renders), the scene is the invariant part only. A
// render whose perturbed primitives no ray segment of the path can meet traces exactly
// this path, because all renders share its random numbers. Segments that touch a union
// box are kept (note_touch) for the per-render pass, which traces the path again in the
// renders whose own bounds a kept segment touches. A path that hits a material whose
// parameters are bound, or that every render must trace again, returns kAffected.
constexpr int kLive = 0, kEnded = 1, kAffected = 2;

// Forward-mode tangents of one path for the pathwise estimator (Eq. 9): dL[k] is the
// derivative of radiance channel c_k with respect to parameter k (an albedo or emission of
// material m_k), dB[k] that of the throughput's channel c_k. The path's discrete choices
// are held fixed and the Russian-roulette probability is a constant of the derivative,
// which keeps the derivative estimate unbiased as it keeps the radiance unbiased.
template <int kND>
struct Tangents {
    float dB[kND > 0 ? kND : 1], dL[kND > 0 ? kND : 1];
};

__device__ __forceinline__ float comp3(float3 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

template <int kND>
__device__ __forceinline__ void tan_reset(Tangents<kND>& t) {
#pragma unroll
    for (int k = 0; k < kND; ++k) t.dB[k] = t.dL[k] = 0.0f;
}

// L += beta * E (background or emitter seen on a camera or specular ray); E may be bound.
template <int kND, class Scn>
__device__ __forceinline__ void tan_emit(Tangents<kND>& t, const TraceJob& J, const Scn& S, float3 beta,
                                         float3 E, int mat) {
#pragma unroll
    for (int k = 0; k < kND; ++k) {
        if (k >= J.diff_n) break;
        const int c = J.diff_comp[k];
        float d = t.dB[k] * comp3(E, c);
        if (J.diff_kind[k] == kBindEmission && J.diff_mat[k] == mat) d = fmaf(comp3(beta, c), S.dclamp[k], d);
        t.dL[k] += d;
    }
}

// L += beta * albedo * Le * g (next-event estimation at a vertex of material mat).
template <int kND, class Scn>
__device__ __forceinline__ void tan_nee(Tangents<kND>& t, const TraceJob& J, const Scn& S, float3 beta,
                                        float3 albedo, int mat, float3 Le, int lmat, float g) {
#pragma unroll
    for (int k = 0; k < kND; ++k) {
        if (k >= J.diff_n) break;
        const int c = J.diff_comp[k];
        const float bc = comp3(beta, c), rc = comp3(albedo, c), ec = comp3(Le, c);
        float d = t.dB[k] * rc * ec;
        if (J.diff_kind[k] == kBindAlbedo && J.diff_mat[k] == mat) d = fmaf(bc * S.dclamp[k], ec, d);
        if (J.diff_kind[k] == kBindEmission && J.diff_mat[k] == lmat) d = fmaf(bc * rc, S.dclamp[k], d);
        t.dL[k] = fmaf(d, g, t.dL[k]);
    }
}

// beta <- beta * albedo (scattering at a vertex of material mat); beta is the old value.
template <int kND, class Scn>
__device__ __forceinline__ void tan_scatter(Tangents<kND>& t, const TraceJob& J, const Scn& S, float3 beta,
                                            float3 albedo, int mat) {
#pragma unroll
    for (int k = 0; k < kND; ++k) {
        if (k >= J.diff_n) break;
        const int c = J.diff_comp[k];
        float d = t.dB[k] * comp3(albedo, c);
        if (J.diff_kind[k] == kBindAlbedo && J.diff_mat[k] == mat) d = fmaf(comp3(beta, c), S.dclamp[k], d);
        t.dB[k] = d;
    }
}

template <int kND>
__device__ __forceinline__ void tan_rr(Tangents<kND>& t, float inv_q) {
#pragma unroll
    for (int k = 0; k < kND; ++k) t.dB[k] *= inv_q;
}

// Next-event estimation at a diffuse vertex po with shading normal ns: emitter li chosen by
// slot 1's first word wl, a uniform point on it from slot 0's first two words (wx, wy).
// True, with the geometry term g (cosines over squared distance, times the emitter's area
// and count over pi) and the emitter's material, when the point is visible from po.
// Emitter of a next-event estimate: floor(u n) of slot 1's first word, exactly.
template <class Scn>
__device__ __forceinline__ int nee_light(const Scn& S, unsigned wl) {
    const int li = int((((wl >> 9) * 2u + 1u) * unsigned(S.n_lights)) >> 24);
    return min(li, S.n_lights - 1);
}

// Is one of the primitives whose record slots are set in `cand` hit closer than dist?
template <bool kCount, class Scn>
__device__ __forceinline__ bool occluded_set(const Scn& S, float3 o, float3 d, float dist, unsigned cand,
                                             Counters& cnt) {
    if (kCount) ++cnt.shadow;
    const int ns = S.n_sph, nsq = S.n_sph + S.n_quad;
    while (cand) {
        const int i = __ffs(cand) - 1;
        cand &= cand - 1u;
        float t;
        if (i < ns) {
            if (kCount) ++cnt.sph;
            t = sphere_t(S.prim[i], o, d);
        } else if (i < nsq) {
            if (kCount) ++cnt.quad;
            t = quad_t(S.prim[i], o, d);
        } else {
            if (kCount) ++cnt.box;
            t = box_t(S.prim[i], o, rcp3(d));
        }
        if (t < dist) return true;
    }
    return false;
}

// The estimate toward emitter li at the point (lu, lv) of its parameterisation (see
// nee_visible).
template <bool kCount, bool kShared, bool kGroup, class Scn>
__device__ __forceinline__ bool nee_to(const Scn& S, float3 po, float3 ns, float lu, float lv, int li, Counters& cnt,
                                       unsigned skip, const GroupLane* gl, float3& wi, float& dist, float& g,
                                       int& lmat) {
    const int4 lt = S.light[li];
    const auto LP = prim_rec<kGroup>(S, lt.y, gl);
    float3 yl, ny;
    if (lt.x == kQuad) {
        const float3 uu = xyz(LP[2]), vv = xyz(LP[3]);
        yl = xyz(LP[0]) + uu * (lu - 0.5f) + vv * (lv - 0.5f);
        ny = xyz(LP[1]);
    } else {
        const float z = 1.0f - 2.0f * lu;
        const float rr2 = fmaxf(0.0f, 1.0f - z * z);
        const float rr_ = rr2 * rsqrtf(fmaxf(rr2, 1e-30f));
        float sp, cp;
        sincospif(2.0f * lv, &sp, &cp);
        ny = f3(rr_ * cp, rr_ * sp, z);
        yl = xyz(LP[0]) + ny * LP[0].w;
    }
    const float3 dv = yl - po;
    const float dist2 = dot3(dv, dv);
    const float inv_dist = rsqrtf(dist2);
    wi = dv * inv_dist;
    const float cx = dot3(ns, wi), cl = -dot3(ny, wi);
    if (!(cx > 0.0f && cl > 0.0f)) return false;
    dist = dist2 * inv_dist;
    bool blocked;
    if constexpr (kGroup) {  // skip: invariant primitives known not to meet the shadow ray
        const int np = S.n_sph + S.n_quad + S.n_box;
        const unsigned all = np >= 32 ? 0xffffffffu : (1u << np) - 1u;
        blocked = occluded_set<kCount>(S, po, wi, dist, all & ~(gl->prims | skip | (1u << lt.y)), cnt) ||
                  group_occluded<kCount>(S, *gl, po, wi, dist, lt.y, cnt);
    } else {
        blocked = occluded<kCount, kShared>(S, po, wi, dist, lt.y, cnt, skip);
    }
    if (blocked) return false;
    g = cx * cl * (inv_dist * inv_dist) * light_area<kGroup>(S, li, gl) * float(S.n_lights) * 0.3183098861837907f;
    lmat = lt.w;
    return true;
}

template <bool kCount, bool kShared, bool kGroup, class Scn>
__device__ __forceinline__ bool nee_visible(const Scn& S, float3 po, float3 ns, unsigned wx, unsigned wy, unsigned wl,
                                            Counters& cnt, unsigned skip, const GroupLane* gl, float3& wi,
                                            float& dist, float& g, int& lmat) {
    return nee_to<kCount, kShared, kGroup>(S, po, ns, u01(wx), u01(wy), nee_light(S, wl), cnt, skip, gl, wi, dist, g,
                                          lmat);
}

// The radiance terms of a path: L + ba Le g (next-event estimation, ba = beta * albedo) and
// L + beta bg (a ray that leaves the scene).
__device__ __forceinline__ float3 nee_add(float3 L, float3 ba, float3 Le, float g) { return L + ba * Le * g; }
__device__ __forceinline__ float3 bg_add(float3 L, float3 beta, float3 bg) { return L + beta * bg; }

// Emitter-sharing mode (k_trace_emit): a path is traced once in the invariant scene for all
// renders; its diffuse vertices are kept (up to kEmitCap) so that each render evaluates its
// own next-event estimate there, and a path whose ray could meet a perturbed primitive (its
// segment touches their union bounds) stops so that each render traces it on from there.
#ifndef PRDPT_EMIT_CAP
#define PRDPT_EMIT_CAP 2
#endif
constexpr int kEmitCap = PRDPT_EMIT_CAP;  // diffuse vertices kept per path
constexpr int kEmitFields = 13;  // po, ns, beta * albedo, the emitter point (lu, lv), emitter li, cull mask
struct EmitLane {
    const float4* ulo;  // union over the renders of each perturbed primitive's bounds
    const float4* uhi;
    int n_var;
    unsigned skip;      // record slots of the perturbed primitives
    float* ent;         // the warp's kept vertices: ent[(k * kEmitFields + field) * 32 + lane]
    int lane;
    int n;              // vertices kept by this lane's path
    bool miss;          // the path ended by leaving the scene
};

// Invariant primitives that no render's shadow ray from po to its emitter li can meet, as a
// record-slot mask: every such ray lies
// in the cone from po over the emitter's union bounds (centre b, half-diagonal rb: the ray
// to a point y deviates from the axis po -> b by at most t rb at parameter t). A primitive
// is left out when its bounding sphere (a sphere itself; a quad's or box's enclosing one)
// keeps clear of that cone, or when a quad's plane has po and the whole union box strictly
// on one side. The margins exceed the FP32 rounding of the intersection tests, so leaving
// these primitives out never changes a shadow ray's outcome.
template <class Scn>
__device__ __forceinline__ unsigned shadow_cull(const Scn& S, const EmitLane& E, float3 po, int li) {
    const int slot = S.light[li].y;
    if (!((E.skip >> slot) & 1u)) return 0u;
    const int k = __popc(E.skip & ((1u << slot) - 1u));
    const float3 lo = xyz(E.ulo[k]), hi = xyz(E.uhi[k]);
    const float3 bc = (lo + hi) * 0.5f, bh = (hi - lo) * 0.5f;
    const float rb = sqrtf(dot3(bh, bh));
    const float3 v = bc - po;
    const float vv = dot3(v, v), lv = sqrtf(vv);
    unsigned m = 0u;
    const int ns = S.n_sph, nq = S.n_quad, np = ns + nq + S.n_box;
    for (int i = 0; i < np; ++i) {
        if ((E.skip >> i) & 1u) continue;
        const float4* P = S.prim[i];
        float3 c;
        float rad;
        if (i < ns) {
            c = xyz(P[0]);
            rad = fabsf(P[0].w);
        } else if (i < ns + nq) {
            c = xyz(P[0]);
            const float3 n = xyz(P[1]), pc = po - c;
            const float mg = (1e-5f + 2e-6f * sqrtf(dot3(pc, pc))) * sqrtf(dot3(n, n));
            const float sp = dot3(pc, n), sb = dot3(bc - c, n);
            const float eb = fabsf(n.x) * bh.x + fabsf(n.y) * bh.y + fabsf(n.z) * bh.z;
            if ((sp > mg && sb - eb > mg) || (sp < -mg && sb + eb < -mg)) {
                m |= 1u << i;
                continue;
            }
            const float3 u = xyz(P[2]), w = xyz(P[3]);
            rad = 0.5f * (sqrtf(dot3(u, u)) + sqrtf(dot3(w, w)));
        } else {
            const float3 a = xyz(P[0]), b = xyz(P[1]);
            c = (a + b) * 0.5f;
            const float3 e = (b - a) * 0.5f;
            rad = sqrtf(dot3(e, e));
        }
        const float R = rad + 1e-3f + 1e-5f * (fabsf(c.x) + fabsf(c.y) + fabsf(c.z));
        const float3 w = c - po;
        const float t0 = vv > 0.0f ? dot3(w, v) / vv : 0.0f;
        const float tc = fminf(fmaxf(t0, 0.0f), 1.0f);
        const float3 q = w - v * tc;
        const float dc = sqrtf(dot3(q, q));
        const float thi = lv > 0.0f ? fminf(1.0f, t0 + (R + rb) / lv) : 1.0f;
        if (dc > R + fmaxf(thi, 0.0f) * rb) m |= 1u << i;
    }
    return m;
}

// Does the segment o + t d, 0 <= t <= tmax, touch a union box of the perturbed primitives?
template <bool kCount>
__device__ __forceinline__ bool emit_touch(const EmitLane& E, float3 o, float3 d, float tmax, Counters& cnt) {
    const float3 inv = rcp3(d);
    const float tm = tmax * 1.0001f + 1e-3f;
    bool hit = false;
    for (int k = 0; k < E.n_var; ++k) hit = hit || slab_touch(xyz(E.ulo[k]), xyz(E.uhi[k]), o, inv, tm);
    if (kCount) cnt.box += E.n_var;
    return hit;
}

template <bool kCount, bool kShared, int kND = 0, bool kGroup = false, bool kEmit = false, class Scn>
__device__ __forceinline__ int advance(const Scn& S, int depth, int rr_start, Path& p, Counters& cnt,
                                       const VarBoxes* V = nullptr, Tangents<kND>* tn = nullptr,
                                       const TraceJob* Jd = nullptr, const GroupLane* gl = nullptr,
                                       EmitLane* el = nullptr) {
    if (kShared && p.seg == 0u) {
        const int t = threadIdx.x;
        s_stash[0][t] = p.o.x;
        s_stash[1][t] = p.o.y;
        s_stash[2][t] = p.o.z;
        s_stash[3][t] = p.d.x;
        s_stash[4][t] = p.d.y;
        s_stash[5][t] = p.d.z;
    }
    Hit h;
    if constexpr (kEmit) {  // the invariant scene; a ray that could meet a perturbed primitive stops here
        h = closest_hit<kCount, true>(S, p.o, p.d, cnt, el->skip);
        if (emit_touch<kCount>(*el, p.o, p.d, h.slot < 0 ? 3.0e38f : h.t, cnt)) return kAffected;
    } else if constexpr (kGroup) {  // the staged scene without the perturbed primitives, then the lane's own
        h = closest_hit<kCount, true>(S, p.o, p.d, cnt, gl->prims);
        group_hit<kCount>(S, *gl, p.o, p.d, h, cnt);
    } else {
        h = closest_hit<kCount, kShared>(S, p.o, p.d, cnt, kShared ? V->skip : 0u);
    }
    if (kShared) {
        note_touch<kCount, false>(*V, p.o, p.d, h.slot < 0 ? 3.0e38f : h.t, p, cnt);
        if (p.seg & kSegAll) return kAffected;
    }
    if (h.slot < 0) {
        if constexpr (kEmit) {
            el->miss = true;  // the background term is added per render, after its vertex terms
            return kEnded;
        }
        if (kND > 0) tan_emit(*tn, *Jd, S, p.beta, xyz(S.bg), -1);
        p.L = bg_add(p.L, p.beta, xyz(S.bg));
        return kEnded;
    }
    if (kCount) ++cnt.vertices;
    const float3 pt = p.o + p.d * h.t;
    const auto P = prim_rec<kGroup>(S, h.slot, gl);
    float3 ng;
    int mat;
    if (h.type == kSphere) {
        const float4 a = P[0];
        ng = (pt - xyz(a)) * P[1].y;
        mat = as_int(P[1].z);
    } else if (h.type == kQuad) {
        ng = xyz(P[1]);
        mat = as_int(P[0].w);
    } else {
        ng = box_normal(P, p.o, p.d, rcp3(p.d));
        mat = as_int(P[0].w);
    }
    if (kShared && ((V->mats >> mat) & 1u)) {  // every render from here (state: this vertex)
        p.seg = (p.seg == 0u ? open_group<false>(*V, p) : p.seg) | kSegAll;
        return kAffected;
    }
    const float4 m0 = mat_albedo<kGroup>(S, mat, gl), m1 = S.mat[mat][1];
    const int mtype = as_int(m0.w);
    const float3 emission = xyz(m1);
    float3 albedo = xyz(m0);
    if (mat == S.tex_mat && h.type == kQuad) albedo = tex_albedo(S, P, pt);
    if (p.specular && (emission.x > 0.f || emission.y > 0.f || emission.z > 0.f) && dot3(p.d, ng) < 0.0f) {
        if constexpr (kEmit) return kAffected;  // an invariant emitter: not in this mode's jobs
        if (kND > 0) tan_emit(*tn, *Jd, S, p.beta, emission, mat);
        p.L = p.L + p.beta * emission;
    }
    const bool last = (p.b + 1 >= depth);
    const bool rr = !last && rr_start >= 0 && p.b >= rr_start;
    uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
    if (mtype == kDiffuse) {
        const float3 ns = dot3(ng, p.d) < 0.0f ? ng : ng * -1.0f;
        const float3 po = pt + ns * kEps;
        const uint4 w0 = vertex_words<kGroup, kGroup || kEmit>(S, p, 0, gl);
        if (S.n_lights > 1 || rr) w1 = vertex_words<kGroup, kGroup || kEmit>(S, p, 1, gl);
        if (S.n_lights > 0) {  // next-event estimation: one emitter, uniform area sample
            if constexpr (kEmit) {  // kept for the renders' own estimates (the renders' emitters differ)
                if (el->n == kEmitCap) return kAffected;
                float* e = el->ent + el->n * kEmitFields * 32 + el->lane;
                const float3 ba = p.beta * albedo;
                e[0] = po.x; e[32] = po.y; e[64] = po.z;
                e[96] = ns.x; e[128] = ns.y; e[160] = ns.z;
                e[192] = ba.x; e[224] = ba.y; e[256] = ba.z;
                const int li = nee_light(S, w1.x);
                e[288] = u01(w0.x); e[320] = u01(w0.y); e[352] = __int_as_float(li);
                e[384] = __uint_as_float(shadow_cull(S, *el, po, li));
                ++el->n;
            } else {
                float3 wi;
                float dist, g;
                int lmat;
                if (nee_visible<kCount, kShared, kGroup>(S, po, ns, w0.x, w0.y, w1.x, cnt, kShared ? V->skip : 0u, gl,
                                                         wi, dist, g, lmat)) {
                    if (kShared) {
                        note_touch<kCount, true>(*V, po, wi, dist, p, cnt);
                        if (p.seg & kSegAll) return kAffected;
                    }
                    const float3 Le = xyz(S.mat[lmat][1]);
                    if (kND > 0) tan_nee(*tn, *Jd, S, p.beta, albedo, mat, Le, lmat, g);
                    p.L = nee_add(p.L, p.beta * albedo, Le, g);
                }
            }
        }
        if (last) return kEnded;
        const float u1 = u01(w0.z), u2 = u01(w0.w);
        const float rad = u1 * rsqrtf(u1);
        float sp, cp;
        sincospif(2.0f * u2, &sp, &cp);
        float3 t1, t2;
        onb(ns, t1, t2);
        const float cz2 = fmaxf(0.0f, 1.0f - u1);
        const float3 wo = t1 * (rad * cp) + t2 * (rad * sp) + ns * (cz2 * rsqrtf(fmaxf(cz2, 1e-30f)));
        if (kND > 0) tan_scatter(*tn, *Jd, S, p.beta, albedo, mat);
        p.beta = p.beta * albedo;
        p.o = po;
        p.d = normalized(wo);
        p.specular = false;
    } else if (mtype == kMirror) {
        if (last) return kEnded;
        if (rr) w1 = vertex_words<kGroup, kGroup || kEmit>(S, p, 1, gl);
        const float3 ns = dot3(ng, p.d) < 0.0f ? ng : ng * -1.0f;
        p.d = normalized(p.d - ns * (2.0f * dot3(p.d, ns)));
        p.o = pt + ns * kEps;
        if (kND > 0) tan_scatter(*tn, *Jd, S, p.beta, albedo, mat);
        p.beta = p.beta * albedo;
        p.specular = true;
    } else {  // smooth dielectric: exact unpolarised Fresnel, reflect or refract
        if (last) return kEnded;
        w1 = vertex_words<kGroup, kGroup || kEmit>(S, p, 1, gl);
        float ci = -dot3(p.d, ng);
        float eta;
        float3 n;
        if (ci > 0.0f) {
            eta = __fdividef(1.0f, m1.w);
            n = ng;
        } else {
            eta = m1.w;
            n = ng * -1.0f;
            ci = -ci;
        }
        const float s2t = eta * eta * (1.0f - ci * ci);
        float F, ct = 0.0f;
        if (s2t >= 1.0f) {
            F = 1.0f;
        } else {
            ct = sqrtf(1.0f - s2t);
            const float rs = __fdividef(eta * ci - ct, eta * ci + ct);
            const float rp = __fdividef(ci - eta * ct, ci + eta * ct);
            F = 0.5f * (rs * rs + rp * rp);
        }
        if (u01(w1.z) < F) {
            p.d = normalized(p.d + n * (2.0f * ci));
            p.o = pt + n * kEps;
        } else {
            p.d = normalized(p.d * eta + n * (eta * ci - ct));
            p.o = pt - n * kEps;
        }
        if (kND > 0) tan_scatter(*tn, *Jd, S, p.beta, albedo, mat);
        p.beta = p.beta * albedo;
        p.specular = true;
    }
    if (maxc(p.beta) <= 0.0f) return kEnded;
    if (rr) {  // Russian roulette on slot 1's second uniform
        const float q = fminf(0.95f, maxc(p.beta));
        if (u01(w1.y) >= q) return kEnded;
        const float inv_q = __fdividef(1.0f, q);
        if (kND > 0) tan_rr(*tn, inv_q);
        p.beta = p.beta * inv_q;
    }
    ++p.b;
    return kLive;
}

// ---------------------------------------------------------------------------
// k_trace: persistent render + fused loss/gradient/Adam epilogue
// ---------------------------------------------------------------------------
constexpr int kWarps = kBlock / 32;
#ifndef PRDPT_TRACE_MIN_BLOCKS
#define PRDPT_TRACE_MIN_BLOCKS 3  // <= 85 registers: 24 resident warps per SM
#endif
constexpr int kTraceMinBlocks = PRDPT_TRACE_MIN_BLOCKS;
constexpr int kDiffMinBlocks = 5;  // pathwise-estimator CTAs of kDiffBlock threads: <= 102 registers
constexpr float kFix = 4294967296.0f;  // 2^32: fixed-point scale of the radiance accumulators

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned warp_sum_u(unsigned v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// n / d for d >= 1 given m = ceil(2^32 / d) (m wraps to 0 for d = 1).
__device__ __forceinline__ int div_magic(int n, int d, unsigned m) {
    return d == 1 ? n : int(__umulhi(unsigned(n), m));
}

// Radiance to fixed point (2^-32 units): integer sums are exact and independent of
// the order in which the warp's lanes finish their paths. The conversion is done
// on the significand bits (a float -> int64 conversion would run on the FP64 pipe):
// v * 2^32 = m * 2^(e + 9) for v = m * 2^(e - 23); values below 2^-9 are truncated.
__device__ __forceinline__ unsigned long long to_fixed(float v) {
    v = fminf(fmaxf(v, 0.0f), 2.0e9f);  // NaN -> 0
    const unsigned bits = __float_as_uint(v);
    const int e = int(bits >> 23) - 127;
    if (e < -32) return 0ull;
    const unsigned long long m = (bits & 0x7fffffu) | 0x800000u;
    const int sh = e + 9;
    return sh >= 0 ? (m << sh) : (m >> (-sh));
}

// Signed value to 2^-32 fixed point as a two's-complement 64-bit word (tangent sums).
__device__ __forceinline__ unsigned long long to_fixed_signed(float v) {
    return v >= 0.0f ? to_fixed(v) : 0ull - to_fixed(-v);
}

// Two's-complement 64-bit integer to float (magnitude split into 32-bit halves, so no
// 64-bit conversion instruction is needed); relative rounding error below 2^-23.
__device__ __forceinline__ float signed_word_to_float(long long D) {
    const unsigned long long m = D < 0 ? (unsigned long long)(-D) : (unsigned long long)D;
    const float f = fmaf(float(unsigned(m >> 32)), 4294967296.0f, float(unsigned(m)));
    return D < 0 ? -f : f;
}

// Squared error of one pixel against the target, summed over RGB (a4). The pixel's sums
// are 2^-32 fixed point over spp samples; acc - T * spp * 2^32 is formed exactly in 64-bit
// integers (T truncated to 2^-32), so the difference suffers no cancellation, and is then
// scaled to the mean and squared in FP32. Only the sums over pixels are FP64.
__device__ __forceinline__ float fixed_diff(unsigned long long a, float t, unsigned spp, float inv) {
    return signed_word_to_float((long long)(a - to_fixed(t) * (unsigned long long)spp)) * inv;
}

__device__ __forceinline__ double pixel_sq_error(unsigned long long ax, unsigned long long ay, unsigned long long az,
                                                 float4 T, unsigned spp, float inv) {
    const float dx = fixed_diff(ax, T.x, spp, inv), dy = fixed_diff(ay, T.y, spp, inv),
                dz = fixed_diff(az, T.z, spp, inv);
    return double(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
}

// 1 / (spp * 2^32): scale of a pixel's fixed-point sum to its mean.
__device__ __forceinline__ float mean_scale(int spp) { return 1.0f / (float(spp) * 4294967296.0f); }

// Per-warp shared-memory workspace of the render kernel.
struct WarpSmem {
    InstScene scene;                  // the render being traced (render 0 in shared phase A)
    TraceJob job;
    unsigned long long acc[3][32];    // radiance of the block's pixels, 2^-32 fixed point
    unsigned recorded;                // shared mode: the block has recorded paths
    VarBoxes vb;                      // shared mode: bounds of the perturbed primitives

};

// Copy render r's scene (header, used materials, used primitives) into a warp's slot.
__device__ __forceinline__ void stage_scene(InstScene& S, const TraceJob& J, int r, int lane) {
    const float4* src = reinterpret_cast<const float4*>(J.scenes + r);
    float4* dst = reinterpret_cast<float4*>(&S);
    constexpr int kHead = int(offsetof(InstScene, mat) / 16);
    constexpr int kPrim = int(offsetof(InstScene, prim) / 16);
    const int nm = 2 * J.n_mats, np = 4 * J.n_prims;
    for (int i = lane; i < kHead + nm + np; i += 32) {
        const int o = (i < kHead + nm) ? i : kPrim + (i - kHead - nm);
        dst[o] = __ldg(src + o);
    }
    __syncwarp();
}

// Union over the job's R renders of each perturbed primitive's bounds (shared mode).
__device__ void build_var_boxes(WarpSmem& W, const TraceJob& J, int lane) {
    for (int k = 0; k < J.n_var; ++k) {
        float3 lo = f3(INFINITY, INFINITY, INFINITY), hi = f3(-INFINITY, -INFINITY, -INFINITY);
        for (int r = lane; r < J.R; r += 32) {
            const float4* b = J.var_box + (size_t(r) * kMaxVariant + k) * 2;
            const float3 a = xyz(__ldg(b)), c = xyz(__ldg(b + 1));
            lo = f3(fminf(lo.x, a.x), fminf(lo.y, a.y), fminf(lo.z, a.z));
            hi = f3(fmaxf(hi.x, c.x), fmaxf(hi.y, c.y), fmaxf(hi.z, c.z));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo.x = fminf(lo.x, __shfl_xor_sync(kFull, lo.x, o));
            lo.y = fminf(lo.y, __shfl_xor_sync(kFull, lo.y, o));
            lo.z = fminf(lo.z, __shfl_xor_sync(kFull, lo.z, o));
            hi.x = fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, o));
            hi.y = fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, o));
            hi.z = fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, o));
        }
        if (lane == 0) {
            W.vb.lo[k] = make_float4(lo.x, lo.y, lo.z, 0.f);
            W.vb.hi[k] = make_float4(hi.x, hi.y, hi.z, 0.f);
        }
    }
    if (lane == 0) {
        W.vb.seg_pool = J.seg_pool;
        W.vb.seg_state = J.seg_state;
        W.vb.seg_ctr = J.share_ctl + 2;
        W.vb.seg_cap = J.seg_cap;
        W.vb.n = J.n_var;
        W.vb.skip = J.var_prims;
        W.vb.mats = J.var_mats;
    }
    __syncwarp();
}

// a += v modulo 2^64 on a shared-memory word, as two native 32-bit atomics: the low
// word's carry (seen from the value it held before the add) goes into the high word.
// Concurrent adds give the exact sum whatever their order; the word is read only after
// every add has completed.
__device__ __forceinline__ void smem_add_u64(unsigned long long* a, unsigned long long v) {
    unsigned* w = reinterpret_cast<unsigned*>(a);  // little-endian: w[0] low, w[1] high
    const unsigned lo = unsigned(v), old = atomicAdd(w, lo);
    atomicAdd(w + 1, unsigned(v >> 32) + (old + lo < old ? 1u : 0u));
}

// k-th (0-based) set bit of m.
__device__ __forceinline__ int nth_set_bit(unsigned long long m, int k) {
    int pos = 0;
    unsigned x = unsigned(m);
    const int c = __popc(x);
    if (k >= c) {
        k -= c;
        x = unsigned(m >> 32);
        pos = 32;
    }
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int cw = __popc(x & ((1u << w) - 1u));
        if (k >= cw) {
            k -= cw;
            x >>= w;
            pos += w;
        }
    }
    return pos;
}

// Trace `ntasks` path tasks with the warp as a pool: each lane holds one live path and,
// when it ends, takes the next task (ballot + popc). decode(task, slot, sample) maps a
// task to its pixel slot and sample; every lane calls it (it may use warp shuffles).
// Ended paths add their radiance to acc[.][slot]. In shared mode a path that touched a
// perturbed primitive's union box is also recorded -- its code, segment word and
// shared-pass radiance -- in the job's list, and *recorded is set.
template <bool kCount, bool kShared, class Decode, int kND = 0, class Scn>
__device__ __forceinline__ void run_pool(const Scn& S, const TraceJob& J, int ntasks, int x0, int y0, int vw,
                                         unsigned magic_w, Decode decode, unsigned long long (&acc)[3][32],
                                         unsigned* recorded, const VarBoxes* V, Counters& cnt, int lane,
                                         unsigned long long (*dacc)[32] = nullptr) {
    const unsigned lt_mask = (1u << lane) - 1u;
    Path p;
    Tangents<kND> tn;
    bool alive = false, ended = true;  // every lane takes its first task at the first refill
    int next = 0, slot, smp;
    for (;;) {
        // lanes whose path ended take the next tasks, in lane order (one code site for the
        // first tasks and the later ones)
        const unsigned need = __ballot_sync(kFull, ended);
        const int mine = next + __popc(need & lt_mask);
        decode((ended && mine < ntasks) ? mine : 0, slot, smp);
        if (ended) {
            alive = mine < ntasks;
            if (alive) {
                const int row = div_magic(slot, vw, magic_w);
                start_path(S, J.W, J.H, x0 + slot - row * vw, y0 + row, smp, slot, p);
                if (kShared) p.seg = 0u;
                if (kND > 0) tan_reset(tn);
                if (kCount) ++cnt.paths;
            }
        }
        next += __popc(need);
        if (!__any_sync(kFull, alive)) break;
        int st = kLive;
        if (alive) st = advance<kCount, kShared, kND>(S, J.depth, J.rr_start, p, cnt, V, &tn, &J);
        ended = alive && st != kLive;
        // every ended path counts in the shared radiance; the per-render pass later adds,
        // for each render in a recorded path's mask, its own radiance minus this value
        if (ended) {
            smem_add_u64(&acc[0][p.slot], to_fixed(p.L.x));
            smem_add_u64(&acc[1][p.slot], to_fixed(p.L.y));
            smem_add_u64(&acc[2][p.slot], to_fixed(p.L.z));
#pragma unroll
            for (int k = 0; k < kND; ++k)  // tangents: signed fixed point, exact and order-free
                if (k < J.diff_n) smem_add_u64(&dacc[k][p.slot], to_fixed_signed(tn.dL[k]));
        }
        if (kShared) {  // record the paths some render must trace itself
            const bool rec = ended && p.seg != 0u;
            const unsigned am = __ballot_sync(kFull, rec);
            if (am) {
                unsigned base = 0;
                if (lane == __ffs(am) - 1) base = atomicAdd(J.share_ctl + 1, unsigned(__popc(am)));
                base = __shfl_sync(kFull, base, __ffs(am) - 1);
                if (rec) {
                    const unsigned e = base + __popc(am & lt_mask);
                    J.aff_codes[e] = (p.pixel << 6) | unsigned(p.s);
                    J.aff_segw[e] = p.seg;
                    J.aff_lsh[3 * size_t(e) + 0] = p.L.x;
                    J.aff_lsh[3 * size_t(e) + 1] = p.L.y;
                    J.aff_lsh[3 * size_t(e) + 2] = p.L.z;
                }
                if (lane == 0) *recorded = 1u;
            }
        }
    }
    __syncwarp();
}

// Pixel means of render r's block, then either the image (render mode) or the squared
// error and the block partial.
template <bool kRender>
__device__ __forceinline__ void block_epilogue(const TraceJob& J, int r, int t, const WarpSmem& W, int x0, int y0,
                                               int vw, int npx, int lane) {
    double e = 0.0;
    const int px = x0 + lane % vw, py = y0 + lane / vw;
    if (lane < npx && px < J.W && py < J.H) {
        const unsigned long long ax = W.acc[0][lane], ay = W.acc[1][lane], az = W.acc[2][lane];
        if (kRender) {
            const double inv = 1.0 / (double(J.spp) * double(kFix));
            J.images[(size_t(r) * J.H + py) * J.W + px] =
                make_float4(float(double(ax) * inv), float(double(ay) * inv), float(double(az) * inv), 0.0f);
        } else {
            e = pixel_sq_error(ax, ay, az, __ldg(J.target + size_t(py) * J.W + px), unsigned(J.spp),
                               mean_scale(J.spp));
        }
    }
    if (!kRender) {
        e = warp_sum_d(e);
        if (lane == 0) J.partials[size_t(r) * J.tiles + t] = e;  // a5: one partial per block
    }
    __syncwarp();
}

// The same squared error for all R renders of a block whose paths are all shared.
__device__ __forceinline__ void shared_block_epilogue(const TraceJob& J, int t, const WarpSmem& W, int x0, int y0,
                                                      int vw, int npx, int lane) {
    double e = 0.0;
    const int px = x0 + lane % vw, py = y0 + lane / vw;
    if (lane < npx && px < J.W && py < J.H) {
        e = pixel_sq_error(W.acc[0][lane], W.acc[1][lane], W.acc[2][lane], __ldg(J.target + size_t(py) * J.W + px),
                           unsigned(J.spp), mean_scale(J.spp));
    }
    e = warp_sum_d(e);
    for (int r = lane; r < J.R; r += 32) J.partials[size_t(r) * J.tiles + t] = e;
    __syncwarp();
}

// Pathwise estimator (Eq. 9): the block's loss partial as in block_epilogue, and for each
// parameter k the partial sum over its pixels of (I - T)_c dI_c/dtheta_k (c = c_k), where
// dI is the tangent sum divided by spp; the 2 / (3HW) factor is applied in k_finalize.
template <int kND>
__device__ __forceinline__ void diff_epilogue(const TraceJob& J, int r, int t, const unsigned long long (&acc)[3][32],
                                              const unsigned long long (*dacc)[32], int x0, int y0, int vw, int npx,
                                              int lane) {
    const int px = x0 + lane % vw, py = y0 + lane / vw;
    const bool ok = lane < npx && px < J.W && py < J.H;
    const float inv = mean_scale(J.spp);
    float3 res = f3(0.f, 0.f, 0.f);
    double e = 0.0;
    if (ok) {
        const float4 T = __ldg(J.target + size_t(py) * J.W + px);
        res = f3(fixed_diff(acc[0][lane], T.x, unsigned(J.spp), inv), fixed_diff(acc[1][lane], T.y, unsigned(J.spp), inv),
                 fixed_diff(acc[2][lane], T.z, unsigned(J.spp), inv));
        e = double(fmaf(res.x, res.x, fmaf(res.y, res.y, res.z * res.z)));
    }
    e = warp_sum_d(e);
    if (lane == 0) J.partials[size_t(r) * J.tiles + t] = e;
#pragma unroll
    for (int k = 0; k < kND; ++k) {
        if (k >= J.diff_n) break;
        double g = 0.0;
        if (ok) g = double(comp3(res, J.diff_comp[k]) * (signed_word_to_float((long long)dacc[k][lane]) * inv));
        g = warp_sum_d(g);
        if (lane == 0) J.gpartials[(size_t(r) * J.tiles + t) * J.diff_n + k] = g;
    }
    __syncwarp();
}

// kShare: every item is a pixel block of all renders of a path-sharing job (single-job
// launches only); otherwise every item is one render's block and job.share is ignored.
// kND > 0: the pathwise estimator (Eq. 9) with tangents of up to kND parameters, in CTAs
// of kDiffBlock threads (room for the per-pixel tangent sums in shared memory).
template <bool kRender, bool kCount, bool kShare, int kND>
__global__ void __launch_bounds__(kND > 0 ? kDiffBlock : kBlock, kND > 0 ? kDiffMinBlocks : kTraceMinBlocks)
    k_trace(const __grid_constant__ TraceLaunch L) {
    constexpr int kW = (kND > 0 ? kDiffBlock : kBlock) / 32;
    __shared__ WarpSmem s_warp[kW];
    __shared__ unsigned long long s_dacc[kND > 0 ? kW : 1][kND > 0 ? kND : 1][32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem& W = s_warp[warp];
    const TraceJob& J = W.job;
    int cur_job = -1, cur_r = -1;
    Counters cnt{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (!L.jobs) {  // a single job's descriptor is host data: copied before the wait
        const unsigned* src = reinterpret_cast<const unsigned*>(&L.job0);
        unsigned* dst = reinterpret_cast<unsigned*>(&W.job);
        for (int i = lane; i < int(sizeof(TraceJob) / 4); i += 32) dst[i] = src[i];
        __syncwarp();
    }
    pdl_enter();
    if (!L.jobs) {
        if (kShare) build_var_boxes(W, J, lane);  // the renders' bounds: written by k_instantiate
        cur_job = 0;
    }

    for (;;) {
        // ---- pop one work item for this warp --------------------------------------
        unsigned item = 0;
        int j = 0;
        if (lane == 0) {
            item = atomicAdd(L.queue, 1u);
            if (item < unsigned(L.total_items) && L.jobs) {
                int lo = 0, hi = L.njobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (L.jobs[mid].item_begin <= int(item)) lo = mid; else hi = mid - 1;
                }
                j = lo;
            }
        }
        item = __shfl_sync(kFull, item, 0);
        if (item >= unsigned(L.total_items)) break;
        j = __shfl_sync(kFull, j, 0);
        if (j != cur_job) {
            const unsigned* src = reinterpret_cast<const unsigned*>(L.jobs ? L.jobs + j : &L.job0);
            unsigned* dst = reinterpret_cast<unsigned*>(&W.job);
            for (int i = lane; i < int(sizeof(TraceJob) / 4); i += 32) dst[i] = src[i];
            __syncwarp();
            if (kShare) build_var_boxes(W, J, lane);
            cur_job = j;
            cur_r = -1;
        }
        const int li = int(item) - J.item_begin;
        const int r = kShare ? 0 : li % J.R;  // render-interleaved: neighbouring items share pixels
        const int t = kShare ? li : li / J.R;
        if (r >= J.R || t >= J.tiles) {
            if (lane == 0) atomicOr(L.status, kStatusBadItem);
            break;
        }
        if (r != cur_r) {  // a2 -> shared memory
            stage_scene(W.scene, J, r, lane);
            cur_r = r;
        }

        // ---- block geometry and task decoding ------------------------------------------
        const int x0 = (t % J.tiles_x) * J.bw, y0 = (t / J.tiles_x) * J.bh;
        const int vw = min(J.bw, J.W - x0), vh = min(J.bh, J.H - y0);
        const int npx = vw * vh, ntasks = npx * J.spp;
        // task -> (pixel slot, sample) by multiply-high with m = ceil(2^32 / d): exact for
        // n < 2^32 / d (here n < 2^21, d <= 32); d = 1 has no 32-bit m and is special-cased
        const unsigned magic = 0xffffffffu / unsigned(npx) + 1u, magic_w = 0xffffffffu / unsigned(vw) + 1u;
        auto dense = [&](int task, int& slot, int& smp) {
            smp = div_magic(task, npx, magic);
            slot = task - smp * npx;
        };
        W.acc[0][lane] = 0ull;
        W.acc[1][lane] = 0ull;
        W.acc[2][lane] = 0ull;
        __syncwarp();

        if (!kShare && kND > 0) {
            // ---- pathwise estimator: radiance and tangents of every pixel x sample ----------
#pragma unroll
            for (int k = 0; k < (kND > 0 ? kND : 1); ++k) s_dacc[warp][k][lane] = 0ull;
            __syncwarp();
            run_pool<kCount, false, decltype(dense), kND>(W.scene, J, ntasks, x0, y0, vw, magic_w, dense, W.acc,
                                                          nullptr, nullptr, cnt, lane, s_dacc[warp]);
            diff_epilogue<kND>(J, r, t, W.acc, s_dacc[warp], x0, y0, vw, npx, lane);
            continue;
        }
        if (!kShare) {
            // ---- a3: every pixel x sample of this render ----------------------------------
            run_pool<kCount, false>(W.scene, J, ntasks, x0, y0, vw, magic_w, dense, W.acc, nullptr, nullptr, cnt,
                                    lane);
            block_epilogue<kRender>(J, r, t, W, x0, y0, vw, npx, lane);  // a4/a5
            continue;
        }

        // ---- shared pass: every path once in the invariant scene ---------------------------
        if (lane == 0) W.recorded = 0u;
        __syncwarp();
        run_pool<kCount, true>(W.scene, J, ntasks, x0, y0, vw, magic_w, dense, W.acc, &W.recorded, &W.vb, cnt, lane);
        if (W.recorded == 0u) {  // every path is shared by all renders
            shared_block_epilogue(J, t, W, x0, y0, vw, npx, lane);
            continue;
        }
        // some paths differ between renders: keep the shared radiance for the epilogue pass
        // and list the block; its affected paths are already in the job's list
        unsigned long long* dst = J.share_acc + size_t(t) * 96;
        dst[lane] = W.acc[0][lane];
        dst[32 + lane] = W.acc[1][lane];
        dst[64 + lane] = W.acc[2][lane];
        if (lane == 0) J.aff_tiles[atomicAdd(J.share_ctl + 0, 1u)] = t;
        __syncwarp();
    }
    if (kCount) {
        const unsigned v[kNumCounters] = {warp_sum_u(cnt.sph), warp_sum_u(cnt.quad), warp_sum_u(cnt.box),
                                          warp_sum_u(cnt.paths), warp_sum_u(cnt.vertices), warp_sum_u(cnt.shadow),
                                          warp_sum_u(cnt.rays), 0u};
        if (lane == 0)
            for (int i = 0; i < kNumCounters; ++i) atomicAdd(L.counters + i, (unsigned long long)v[i]);
    }
}

// ---------------------------------------------------------------------------
// k_trace_group: render-group variant of the per-render kernel (a3-a5)
// ---------------------------------------------------------------------------
// A work item is (pixel block t, render group g): G = J.gsize consecutive renders of a
// job (G divides R; 32 / G lanes per render). Lane l traces render g G + (l mod G), and
// the 32 / G lanes of one render take the samples s = l / G, l / G + 32 / G, ... of the
// current pixel: all lanes follow one pixel, so with common random numbers the renders'
// paths agree until a perturbed primitive intervenes and the warp stays coherent. The
// block's pixels are taken in bit-reversed slot order and their squared errors summed
// pairwise in that order, which is the shuffle tree of the per-render kernel's epilogue:
// with the same block shape, the same integer pixel sums and the same FP32 path
// arithmetic, every partial is bit-identical to the per-render kernel's.
constexpr int kGroupTab = kGroupTabRows;  // float4 per warp for the group's per-render records
static_assert(offsetof(InstScene, light_area) % 16 == 0, "emitter areas are copied as two float4");

// The render-group kernel's staged scene: the fields of InstScene with arrays for at most
// kGroupPrims primitives and kGroupMats materials (the per-warp copy is then 1.9 KB instead
// of 3.4 KB, so more warps fit an SM). Its header is laid out as InstScene's.
struct __align__(16) GroupScene {
    int n_sph, n_quad, n_box, n_lights;
    unsigned seed_lo, seed_hi, step, c3;
    float4 eye, fwd, right, up, bg;
    int4 light[kMaxLights];
    float light_area[kMaxLights];
    float dclamp[kMaxDiff];
    const float* tex;
    int tex_mat, tex_res;
    float4 mat[kGroupMats][2];
    float4 prim[kGroupPrims][4];
};
static_assert(offsetof(GroupScene, light) == offsetof(InstScene, light) &&
                  offsetof(GroupScene, light_area) == offsetof(InstScene, light_area) &&
                  offsetof(GroupScene, tex) == offsetof(InstScene, tex) &&
                  offsetof(GroupScene, mat) == offsetof(InstScene, mat),
              "GroupScene's header must be laid out as InstScene's");

// Copy render r's scene (header, used materials, used primitives) into a warp's GroupScene
// (the job has at most kGroupPrims primitives and kGroupMats materials).
__device__ __forceinline__ void stage_group_scene(GroupScene& S, const TraceJob& J, int r, int lane) {
    const float4* src = reinterpret_cast<const float4*>(J.scenes + r);
    float4* dst = reinterpret_cast<float4*>(&S);
    constexpr int kHead = int(offsetof(InstScene, mat) / 16);
    constexpr int kPrimSrc = int(offsetof(InstScene, prim) / 16);
    constexpr int kPrimDst = int(offsetof(GroupScene, prim) / 16);
    const int nm = 2 * J.n_mats, np = 4 * J.n_prims;
    for (int i = lane; i < kHead + nm + np; i += 32) {
        const bool is_prim = i >= kHead + nm;
        const int o = is_prim ? i - kHead - nm : i;
        dst[is_prim ? kPrimDst + o : o] = __ldg(src + (is_prim ? kPrimSrc + o : o));
    }
    __syncwarp();
}

struct GroupSmem {
    GroupScene scene;  // the invariant part (render g G's records of the other primitives)
    TraceJob job;
    float4 tab[kGroupTab];
    double pair[5][32];  // each lane's pairwise-sum stack (touched once per pixel)
    unsigned long long acc[3][32];  // each lane's radiance sums of the current pixel, 2^-32 fixed point
    uint4 rng[32];  // each sample group's Philox blocks of its current path (G per group)
};

#ifndef PRDPT_GROUP_MIN_BLOCKS
#define PRDPT_GROUP_MIN_BLOCKS 6  // 128-thread CTAs, <= 85 registers: 24 resident warps per SM
#endif
constexpr int kGroupMinBlocks = PRDPT_GROUP_MIN_BLOCKS;

__device__ __forceinline__ int brev5(int q) { return int(__brev(unsigned(q)) >> 27); }

// Pairwise sum over 32 values pushed in order: level l of the stack (s[l][lane]) holds a
// completed subtree of 2^l values; value q merges with levels 0, 1, ... while bit l of q is
// set. After the 32nd push the result is the total, summed as ((v0 + v1) + (v2 + v3)) + ...
__device__ __forceinline__ double pairwise_push(int q, double v, double (*s)[32], int lane) {
    int l = 0;
    for (; (q >> l) & 1; ++l) v = s[l][lane] + v;
    if (l < 5) s[l][lane] = v;
    return v;
}

template <bool kCount>
__global__ void __launch_bounds__(kGroupBlock, kGroupMinBlocks) k_trace_group(const __grid_constant__ TraceLaunch L) {
    __shared__ GroupSmem s_grp[kGroupBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    GroupSmem& W = s_grp[warp];
    const TraceJob& J = W.job;
    int cur_job = -1, cur_item_g = -1;
    Counters cnt{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (!L.jobs) {  // a single job's descriptor is host data: copied before the wait
        const unsigned* src = reinterpret_cast<const unsigned*>(&L.job0);
        unsigned* dst = reinterpret_cast<unsigned*>(&W.job);
        for (int i = lane; i < int(sizeof(TraceJob) / 4); i += 32) dst[i] = src[i];
        __syncwarp();
        cur_job = 0;
    }
    pdl_enter();
    for (;;) {
        unsigned item = 0;
        int j = 0;
        if (lane == 0) {
            item = atomicAdd(L.queue, 1u);
            if (item < unsigned(L.total_items) && L.jobs) {
                int lo = 0, hi = L.njobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (L.jobs[mid].item_begin <= int(item)) lo = mid; else hi = mid - 1;
                }
                j = lo;
            }
        }
        item = __shfl_sync(kFull, item, 0);
        if (item >= unsigned(L.total_items)) break;
        j = __shfl_sync(kFull, j, 0);
        if (j != cur_job) {
            const unsigned* src = reinterpret_cast<const unsigned*>(L.jobs ? L.jobs + j : &L.job0);
            unsigned* dst = reinterpret_cast<unsigned*>(&W.job);
            for (int i = lane; i < int(sizeof(TraceJob) / 4); i += 32) dst[i] = src[i];
            __syncwarp();
            cur_job = j;
            cur_item_g = -1;
        }
        const int G = J.gsize, ngr = J.R / G, stride = J.gstride;
        const int li = int(item) - J.item_begin;
        const int g = li % ngr, t = li / ngr;  // group-interleaved: neighbouring items share pixels
        if (G < 1 || G > 32 || (32 % G) != 0 || t >= J.tiles || G * stride > kGroupTab || J.n_prims > kGroupPrims ||
            J.n_mats > kGroupMats) {
            if (lane == 0) atomicOr(L.status, kStatusBadItem);
            break;
        }
        if (g != cur_item_g) {  // stage render g G's scene and the group's per-render records
            stage_group_scene(W.scene, J, g * G, lane);
            const int n = J.n_var, nm = __popc(J.var_mats);
            for (int i = lane; i < G * stride; i += 32) {
                const int gi = i / stride, q = i - gi * stride;
                const InstScene& R = J.scenes[g * G + gi];
                float4 v;
                if (q < 4 * n) {  // record of the (q / 4)-th perturbed primitive
                    const int slot = nth_set_bit(J.var_prims, q >> 2);
                    v = __ldg(&R.prim[slot][q & 3]);
                } else if (q < 4 * n + nm) {  // albedo row of a bound material
                    v = __ldg(&R.mat[nth_set_bit(J.var_mats, q - 4 * n)][0]);
                } else {  // emitter areas
                    v = __ldg(reinterpret_cast<const float4*>(R.light_area) + (q - 4 * n - nm));
                }
                W.tab[q * G + gi] = v;  // field-major: the lanes' loads of one field are contiguous
            }
            __syncwarp();
            cur_item_g = g;
        }
        const int gi = lane % G, ks = lane / G, nsg = 32 / G;  // render in group, sample group, groups
        // Under common random numbers the G renders of a path sample draw the same Philox
        // blocks, so the group's lanes draw them ahead, one block each: the jitter and
        // slots 0 and 1 of vertices b < bpre.
        const int bpre = (G - 1) >> 1;
        const GroupLane gl{W.tab + gi, J.var_prims, J.var_mats, J.n_var,
                           stride > 4 * J.n_var + __popc(J.var_mats) ? 1 : 0, W.rng + ks * G, bpre, G};
        const unsigned gmask = G == 32 ? kFull : ((1u << G) - 1u) << (ks * G);
        const int x0 = (t % J.tiles_x) * J.bw, y0 = (t / J.tiles_x) * J.bh;
        const int vw = min(J.bw, J.W - x0), vh = min(J.bh, J.H - y0);
        const int npx = vw * vh;
        const unsigned magic_w = 0xffffffffu / unsigned(vw) + 1u;
        const float inv = mean_scale(J.spp);
        double part = 0.0;
        for (int q = 0; q < 32; ++q) {
            const int slot = brev5(q);  // pixels in bit-reversed slot order (see above)
            double e = 0.0;
            if (slot < npx) {
                const int row = div_magic(slot, vw, magic_w);
                const int px = x0 + slot - row * vw, py = y0 + row;
                W.acc[0][lane] = 0ull;
                W.acc[1][lane] = 0ull;
                W.acc[2][lane] = 0ull;
                for (int smp = ks; smp < J.spp; smp += nsg) {
                    __syncwarp(gmask);  // the group's lanes are done with the previous path's blocks
                    if (gi == 0 || gi <= 2 * bpre)
                        W.rng[lane] = path_words(W.scene, unsigned(py * J.W + px), smp, gi == 0 ? 0 : (gi - 1) >> 1,
                                                 gi == 0 ? 2 : (gi - 1) & 1);
                    __syncwarp(gmask);
                    Path p;
                    start_path(W.scene, J.W, J.H, px, py, smp, slot, p, gl.rng);
                    if (kCount) ++cnt.paths;
                    while (advance<kCount, false, 0, true>(W.scene, J.depth, J.rr_start, p, cnt, nullptr, nullptr,
                                                          nullptr, &gl) == kLive) {
                    }
                    W.acc[0][lane] += to_fixed(p.L.x);
                    W.acc[1][lane] += to_fixed(p.L.y);
                    W.acc[2][lane] += to_fixed(p.L.z);
                }
                unsigned long long a0 = W.acc[0][lane], a1 = W.acc[1][lane], a2 = W.acc[2][lane];
                for (int o = G; o < 32; o <<= 1) {  // the render's other sample groups
                    a0 += __shfl_xor_sync(kFull, a0, o);
                    a1 += __shfl_xor_sync(kFull, a1, o);
                    a2 += __shfl_xor_sync(kFull, a2, o);
                }
                e = pixel_sq_error(a0, a1, a2, __ldg(J.target + size_t(py) * J.W + px), unsigned(J.spp), inv);
            }
            part = pairwise_push(q, e, W.pair, lane);
        }
        if (ks == 0) J.partials[size_t(g * G + gi) * J.tiles + t] = part;  // a5: one partial per block
        __syncwarp();
    }
    if (kCount) {
        const unsigned v[kNumCounters] = {warp_sum_u(cnt.sph), warp_sum_u(cnt.quad), warp_sum_u(cnt.box),
                                          warp_sum_u(cnt.paths), warp_sum_u(cnt.vertices), warp_sum_u(cnt.shadow),
                                          warp_sum_u(cnt.rays), 0u};
        if (lane == 0)
            for (int i = 0; i < kNumCounters; ++i) atomicAdd(L.counters + i, (unsigned long long)v[i]);
    }
}

// ---------------------------------------------------------------------------
// k_trace_emit: emitter-sharing variant of the per-render kernel (a3-a5)
// ---------------------------------------------------------------------------
// For a job whose perturbed primitives include every emitter and whose materials are not
// bound (e.g. a moving light): under common random numbers the renders' paths agree until
// one of their rays could meet a perturbed primitive, and differ before that only in the
// next-event estimates. A work item is one pixel block of all R <= 64 renders, taken by a
// CTA of kEmitWarps warps; warp w takes the pixel slots of positions q = 8w .. 8w + 7 of
// the bit-reversed order. For each pixel, 32 samples at a time:
//   phase A  lane = sample: the path is traced once in the invariant scene, keeping its
//            diffuse vertices (EmitLane) and its end: left the scene (the background term),
//            ended, or stopped where a ray could meet a perturbed primitive;
//   phase B  lane = render (lane and lane + 32; with R <= 16, render lane mod G of sample
//            group lane / G, G the power of two >= R): for each sample that adds anything,
//            the render's own next-event estimates at the kept vertices (occlusion tested
//            against the primitives the vertex's cull mask leaves), then the background term
//            or, for a stopped path, the rest of the path traced in the render's scene (as in
//            k_trace_group).
// Each render's radiance is the same sum, term by term and in the same order, as tracing
// the path in that render alone, so with the same block shape every partial is
// bit-identical to the per-render kernel's; the warps' subtrees of the pairwise pixel sum
// are combined as that sum's top two levels.
constexpr int kEmitWarps = kGroupBlock / 32;
constexpr int kEmitTab = kEmitTabRows;
static_assert(32 % kEmitWarps == 0, "each warp takes 32 / kEmitWarps pixel slots");
constexpr int kEmitSlots = 32 / kEmitWarps;
static_assert(kEmitSlots == 8, "the warps' subtrees are the pairwise sum's levels 0-2");

struct EmitWarp {
    float ent[kEmitCap * kEmitFields * 32];  // kept vertices of the warp's 32 paths
    float st[10][32];                        // end state: o, d, beta, vertex b (bits)
    int n[32];                               // vertices kept
    int kind[32];                            // 0 ended, 1 left the scene, 2 stopped (specular flag: 4)
    double pair[2][3][32];                   // pairwise-sum stacks of the lane's two renders
};
struct EmitSmem {
    GroupScene scene;  // the invariant part (render 0's records of the other primitives)
    TraceJob job;
    float4 tab[kEmitTab];  // per-render rows (as k_trace_group's), R x gstride
    float4 ulo[kMaxVariant], uhi[kMaxVariant];
    double sub[kEmitWarps][64];
    EmitWarp w[kEmitWarps];
    unsigned item;
    int job_index;
};

// The rest of a stopped path in one render's scene (as k_trace_group traces it).
template <bool kCount>
__device__ __forceinline__ float3 emit_continue(const GroupScene& S, int depth, int rr_start, const GroupLane& gl,
                                                Path p, Counters& cnt) {
    while (advance<kCount, false, 0, true>(S, depth, rr_start, p, cnt, nullptr, nullptr, nullptr, &gl) == kLive) {
    }
    return p.L;
}

#ifndef PRDPT_EMIT_MIN_BLOCKS
#define PRDPT_EMIT_MIN_BLOCKS 5  // <= 102 registers: 20 resident warps per SM
#endif
constexpr int kEmitMinBlocks = PRDPT_EMIT_MIN_BLOCKS;

template <bool kCount>
__global__ void __launch_bounds__(kGroupBlock, kEmitMinBlocks) k_trace_emit(const __grid_constant__ TraceLaunch L) {
    __shared__ EmitSmem E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    EmitWarp& Wp = E.w[warp];
    const TraceJob& J = E.job;
    int cur_job = -1;
    Counters cnt{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    if (!L.jobs) {  // a single job's descriptor is host data: copied before the wait
        const unsigned* src = reinterpret_cast<const unsigned*>(&L.job0);
        unsigned* dst = reinterpret_cast<unsigned*>(&E.job);
        for (int i = threadIdx.x; i < int(sizeof(TraceJob) / 4); i += kGroupBlock) dst[i] = src[i];
    }
    __syncthreads();
    pdl_enter();
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned item = atomicAdd(L.queue, 1u);
            int j = 0;
            if (item < unsigned(L.total_items) && L.jobs) {
                int lo = 0, hi = L.njobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (L.jobs[mid].item_begin <= int(item)) lo = mid; else hi = mid - 1;
                }
                j = lo;
            }
            E.item = item;
            E.job_index = j;
        }
        __syncthreads();
        const unsigned item = E.item;
        const int j = E.job_index;
        if (item >= unsigned(L.total_items)) break;
        if (j != cur_job) {  // stage the job, its invariant scene, per-render rows and union bounds
            if (L.jobs) {
                const unsigned* src = reinterpret_cast<const unsigned*>(L.jobs + j);
                unsigned* dst = reinterpret_cast<unsigned*>(&E.job);
                for (int i = threadIdx.x; i < int(sizeof(TraceJob) / 4); i += kGroupBlock) dst[i] = src[i];
                __syncthreads();
            }
            if (J.R < 1 || J.R > 64 || J.R * J.gstride > kEmitTab || J.gstride < 4 * J.n_var || J.n_var < 1 ||
                J.n_var > kMaxVariant || J.n_prims > kGroupPrims || J.n_mats > kGroupMats) {
                if (threadIdx.x == 0) atomicOr(L.status, kStatusBadItem);
                break;
            }
            if (warp == 0) stage_group_scene(E.scene, J, 0, lane);
            const int stride = J.gstride, n = J.n_var;
            for (int i = threadIdx.x; i < J.R * stride; i += kGroupBlock) {
                const int r = i / stride, q = i - r * stride;
                const InstScene& R = J.scenes[r];
                float4 v;
                if (q < 4 * n) v = __ldg(&R.prim[nth_set_bit(J.var_prims, q >> 2)][q & 3]);
                else v = __ldg(reinterpret_cast<const float4*>(R.light_area) + (q - 4 * n));  // emitter areas
                E.tab[q * J.R + r] = v;  // field-major, as k_trace_group's table
            }
            __syncthreads();
            if (warp == 0) {
                for (int k = 0; k < n; ++k) {
                    const int slot = nth_set_bit(J.var_prims, k);
                    const int type = slot < E.scene.n_sph ? kSphere : (slot < E.scene.n_sph + E.scene.n_quad ? kQuad : kBox);
                    float3 lo = f3(INFINITY, INFINITY, INFINITY), hi = f3(-INFINITY, -INFINITY, -INFINITY);
                    for (int r = lane; r < J.R; r += 32) {
                        float3 a, c;
                        const float4 rec[4] = {E.tab[(4 * k) * J.R + r], E.tab[(4 * k + 1) * J.R + r],
                                               E.tab[(4 * k + 2) * J.R + r], E.tab[(4 * k + 3) * J.R + r]};
                        prim_bounds(rec, type, a, c);
                        lo = f3(fminf(lo.x, a.x), fminf(lo.y, a.y), fminf(lo.z, a.z));
                        hi = f3(fmaxf(hi.x, c.x), fmaxf(hi.y, c.y), fmaxf(hi.z, c.z));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        lo.x = fminf(lo.x, __shfl_xor_sync(kFull, lo.x, o));
                        lo.y = fminf(lo.y, __shfl_xor_sync(kFull, lo.y, o));
                        lo.z = fminf(lo.z, __shfl_xor_sync(kFull, lo.z, o));
                        hi.x = fmaxf(hi.x, __shfl_xor_sync(kFull, hi.x, o));
                        hi.y = fmaxf(hi.y, __shfl_xor_sync(kFull, hi.y, o));
                        hi.z = fmaxf(hi.z, __shfl_xor_sync(kFull, hi.z, o));
                    }
                    if (lane == 0) {
                        E.ulo[k] = make_float4(lo.x, lo.y, lo.z, 0.f);
                        E.uhi[k] = make_float4(hi.x, hi.y, hi.z, 0.f);
                    }
                }
            }
            __syncthreads();
            cur_job = j;
        }
        const int t = int(item) - J.item_begin;
        if (t < 0 || t >= J.tiles) {
            if (threadIdx.x == 0) atomicOr(L.status, kStatusBadItem);
            break;
        }
        const int R = J.R, nh = R > 32 ? 2 : 1, stride = J.gstride;
        // phase B lanes: render gi = lane mod G of sample group ks = lane / G (G the power of
        // two >= R, at most 32): with few renders a warp takes 32 / G samples at a time
        const int G = R >= 32 ? 32 : (R <= 1 ? 1 : 1 << (32 - __clz(R - 1)));
        const int nsg = 32 / G, gi = lane % G, ks = lane / G;
        const int areas = stride > 4 * J.n_var ? 1 : 0;
        const int x0 = (t % J.tiles_x) * J.bw, y0 = (t / J.tiles_x) * J.bh;
        const int vw = min(J.bw, J.W - x0), vh = min(J.bh, J.H - y0);
        const int npx = vw * vh;
        const unsigned magic_w = 0xffffffffu / unsigned(vw) + 1u;
        const float inv = mean_scale(J.spp);
        EmitLane el{E.ulo, E.uhi, J.n_var, J.var_prims, Wp.ent, lane, 0, false};
        const bool bg_nonzero = E.scene.bg.x != 0.0f || E.scene.bg.y != 0.0f || E.scene.bg.z != 0.0f;
        double sub[2] = {0.0, 0.0};
        // The loops below stay rolled: unrolled copies of the tracer overflow the instruction
        // cache (measured on the caustic step: 13.1 ms unrolled, 11.0 ms rolled).
#pragma unroll 1
        for (int qq = 0; qq < kEmitSlots; ++qq) {
            const int slot = brev5(warp * kEmitSlots + qq);  // pixels in bit-reversed slot order
            double e[2] = {0.0, 0.0};
            if (slot < npx) {
                const int row = div_magic(slot, vw, magic_w);
                const int px = x0 + slot - row * vw, py = y0 + row;
                unsigned long long acc[2][3] = {{0ull, 0ull, 0ull}, {0ull, 0ull, 0ull}};
                for (int s0 = 0; s0 < J.spp; s0 += 32) {
                    // ---- phase A: one path per lane, traced once for all renders ----------
                    __syncwarp();  // phase B of the previous samples is done with the table
                    bool work = false;  // does the sample add anything to a render?
                    if (s0 + lane < J.spp) {
                        Path p;
                        start_path<true>(E.scene, J.W, J.H, px, py, s0 + lane, slot, p);
                        if (kCount) ++cnt.paths;
                        el.n = 0;
                        el.miss = false;
                        int res;
                        while ((res = advance<kCount, false, 0, false, true>(E.scene, J.depth, J.rr_start, p, cnt,
                                                                             nullptr, nullptr, nullptr, nullptr,
                                                                             &el)) == kLive) {
                        }
                        Wp.n[lane] = el.n;
                        Wp.kind[lane] = (res == kAffected ? 2 : (el.miss ? 1 : 0)) | (p.specular ? 4 : 0);
                        Wp.st[0][lane] = p.o.x;
                        Wp.st[1][lane] = p.o.y;
                        Wp.st[2][lane] = p.o.z;
                        Wp.st[3][lane] = p.d.x;
                        Wp.st[4][lane] = p.d.y;
                        Wp.st[5][lane] = p.d.z;
                        Wp.st[6][lane] = p.beta.x;
                        Wp.st[7][lane] = p.beta.y;
                        Wp.st[8][lane] = p.beta.z;
                        Wp.st[9][lane] = __int_as_float(p.b);
                        work = el.n > 0 || res == kAffected || (el.miss && bg_nonzero);
                    }
                    // ---- phase B: each render's terms of each sample, in sample order -----
                    // (samples that add nothing to any render -- no kept vertex, not stopped,
                    // no background term -- are passed over: their sums would add zero)
                    __syncwarp();
                    unsigned todo = __ballot_sync(kFull, work);
#pragma unroll 1
                    while (todo) {
                        int jj = -1;  // sample group ks takes the ks-th of the next nsg samples
                        for (int i = 0; i < nsg && todo; ++i) {
                            if (i == ks) jj = __ffs(todo) - 1;
                            todo &= todo - 1u;
                        }
                        if (jj < 0) continue;
                        const int nk = Wp.n[jj], kind = Wp.kind[jj];
#pragma unroll 1
                        for (int h = 0; h < nh; ++h) {
                            const int r = gi + 32 * h;
                            if (r >= R) continue;
                            const GroupLane gl{E.tab + r, J.var_prims, 0u, J.n_var, areas, nullptr, 0, R};
                            float3 Lr = f3(0.f, 0.f, 0.f);
#pragma unroll 1
                            for (int k = 0; k < nk; ++k) {
                                const float* en = Wp.ent + k * kEmitFields * 32 + jj;
                                const float3 po = f3(en[0], en[32], en[64]), nsv = f3(en[96], en[128], en[160]);
                                float3 wi;
                                float dist, g;
                                int lmat;
                                if (nee_to<kCount, false, true>(E.scene, po, nsv, en[288], en[320],
                                                                __float_as_int(en[352]), cnt, __float_as_uint(en[384]),
                                                                &gl, wi, dist, g, lmat))
                                    Lr = nee_add(Lr, f3(en[192], en[224], en[256]), xyz(E.scene.mat[lmat][1]), g);
                            }
                            const float3 beta = f3(Wp.st[6][jj], Wp.st[7][jj], Wp.st[8][jj]);
                            if ((kind & 3) == 1) {
                                Lr = bg_add(Lr, beta, xyz(E.scene.bg));
                            } else if ((kind & 3) == 2) {  // the rest of the path in render r's scene
                                Path p;
                                p.o = f3(Wp.st[0][jj], Wp.st[1][jj], Wp.st[2][jj]);
                                p.d = f3(Wp.st[3][jj], Wp.st[4][jj], Wp.st[5][jj]);
                                p.beta = beta;
                                p.L = Lr;
                                p.pixel = unsigned(py * J.W + px);
                                p.s = s0 + jj;
                                p.b = __float_as_int(Wp.st[9][jj]);
                                p.slot = slot;
                                p.specular = (kind & 4) != 0;
                                p.seg = 0u;
                                Lr = emit_continue<kCount>(E.scene, J.depth, J.rr_start, gl, p, cnt);
                            }
                            if (Lr.x != 0.0f || Lr.y != 0.0f || Lr.z != 0.0f) {
                                acc[h][0] += to_fixed(Lr.x);
                                acc[h][1] += to_fixed(Lr.y);
                                acc[h][2] += to_fixed(Lr.z);
                            }
                        }
                    }
                }
                for (int o = G; o < 32; o <<= 1) {  // the render's other sample groups
                    acc[0][0] += __shfl_xor_sync(kFull, acc[0][0], o);
                    acc[0][1] += __shfl_xor_sync(kFull, acc[0][1], o);
                    acc[0][2] += __shfl_xor_sync(kFull, acc[0][2], o);
                }
                const float4 T = __ldg(J.target + size_t(py) * J.W + px);
                for (int h = 0; h < nh; ++h)
                    e[h] = pixel_sq_error(acc[h][0], acc[h][1], acc[h][2], T, unsigned(J.spp), inv);
            }
            for (int h = 0; h < 2; ++h) {  // levels 0-2 of the pairwise sum over this warp's slots
                double v = e[h];
                int l = 0;
                for (; (qq >> l) & 1; ++l) v = Wp.pair[h][l][lane] + v;
                if (l < 3) Wp.pair[h][l][lane] = v;
                else sub[h] = v;
            }
        }
        for (int h = 0; h < nh; ++h)
            if (ks == 0 && gi + 32 * h < R) E.sub[warp][gi + 32 * h] = sub[h];
        __syncthreads();
        for (int r = threadIdx.x; r < R; r += kGroupBlock)  // a5: levels 3 and 4
            J.partials[size_t(r) * J.tiles + t] = (E.sub[0][r] + E.sub[1][r]) + (E.sub[2][r] + E.sub[3][r]);
        __syncthreads();
    }
    if (kCount) {
        const unsigned v[kNumCounters] = {warp_sum_u(cnt.sph), warp_sum_u(cnt.quad), warp_sum_u(cnt.box),
                                          warp_sum_u(cnt.paths), warp_sum_u(cnt.vertices), warp_sum_u(cnt.shadow),
                                          warp_sum_u(cnt.rays), 0u};
        if (lane == 0)
            for (int i = 0; i < kNumCounters; ++i) atomicAdd(L.counters + i, (unsigned long long)v[i]);
    }
}

// Per-render pass of a path-sharing job: render r traces again each recorded path one of
// whose kept segments touches render r's bounds of a perturbed primitive, and adds its radiance minus the shared-pass radiance (2^-32 fixed point,
// modulo 2^64) to the render's image-sized buffer with global atomic adds -- integer
// sums, so the order does not matter and the block sums equal those of tracing every
// path in every render.
// Work distribution: warp g starts on render g mod R and streams that render's paths.
// Batches of 32 list entries are claimed from the render's cursor, the entries that
// render r must trace are compacted into a per-warp ring, and a lane whose path ends takes the
// next ring entry at once, so the warp's pool only drains when the render's list is
// used up; the warp then moves on to the next render with entries left.
constexpr int kAffRing = 64;  // ring entries per warp (the ring never holds more than 63)

template <bool kCount>
__global__ void __launch_bounds__(kBlock, kTraceMinBlocks) k_trace_affected(const __grid_constant__ TraceLaunch L) {
    __shared__ InstScene s_scene[kWarps];
    __shared__ TraceJob s_job[kWarps];
    __shared__ unsigned s_ring[kWarps][kAffRing];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    InstScene& S = s_scene[warp];
    TraceJob& J = s_job[warp];
    unsigned* ring = s_ring[warp];
    const int gwarp = int(blockIdx.x) * kWarps + warp;
    Counters cnt{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    const int njobs = L.jobs ? L.njobs : 1;
    for (int jb = 0; jb < njobs; ++jb) {  // the jobs of a packed launch one after another
    {  // job descriptors are host data: the first is copied before the wait on the previous kernel
        const unsigned* src = reinterpret_cast<const unsigned*>(L.jobs ? L.jobs + jb : &L.job0);
        unsigned* dst = reinterpret_cast<unsigned*>(&J);
        for (int i = lane; i < int(sizeof(TraceJob) / 4); i += 32) dst[i] = src[i];
        __syncwarp();
        if (jb == 0) pdl_enter();
    }
    const bool job_shares = J.share != 0;
    __syncwarp();  // every lane has read the descriptor before the next copy may overwrite it
    if (!job_shares) continue;
    const unsigned n_codes = __ldcg(J.share_ctl + 1);
    const unsigned magic_W = 0xffffffffu / unsigned(J.W) + 1u;
    for (int k = 0; k < J.R; ++k) {
        {  // the next render, in the order gwarp + k, ..., with entries left: 32 cursors at a time
            const bool left = k + lane < J.R && __ldcg(J.aff_cursor + (gwarp + k + lane) % J.R) < n_codes;
            const unsigned m = __ballot_sync(kFull, left);
            if (!m) {
                k += 31;
                continue;
            }
            k += __ffs(m) - 1;
        }
        const int r = (gwarp + k) % J.R;
        unsigned* cursor = J.aff_cursor + r;
        {  // stage render r's scene
            const float4* src = reinterpret_cast<const float4*>(J.scenes + r);
            float4* dst = reinterpret_cast<float4*>(&S);
            constexpr int kHead = int(offsetof(InstScene, mat) / 16);
            constexpr int kPrim = int(offsetof(InstScene, prim) / 16);
            const int nm = 2 * J.n_mats, np = 4 * J.n_prims;
            for (int i = lane; i < kHead + nm + np; i += 32) {
                const int o = (i < kHead + nm) ? i : kPrim + (i - kHead - nm);
                dst[o] = __ldg(src + o);
            }
            __syncwarp();
        }
        unsigned long long* acc = J.acc_aff + size_t(r) * J.W * J.H * 3;
        unsigned head = 0, tail = 0;  // ring positions, the same in every lane
        bool src_done = false, alive = false;
        Path p;
        for (;;) {
            while (!src_done && tail - head < 32u) {  // claim 32 entries, keep render r's
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(cursor, 32u);
                base = __shfl_sync(kFull, base, 0);
                if (base >= n_codes) {
                    src_done = true;
                    break;
                }
                const unsigned e = base + unsigned(lane);
                bool need = false;
                if (e < n_codes) {  // does a kept segment of the path touch render r's bounds?
                    const unsigned sw = __ldcg(J.aff_segw + e);
                    need = (sw & kSegAll) != 0u;
                    const unsigned s0 = ((sw >> 3) - 1u) * unsigned(kSeg), ns = need ? 0u : (sw & 7u);
                    for (unsigned q = 0; q < ns && !need; ++q) {
                        const float4 A = __ldcg(J.seg_pool + 2 * size_t(s0 + q));
                        const float4 B = __ldcg(J.seg_pool + 2 * size_t(s0 + q) + 1);
                        const float3 o = xyz(A), inv = rcp3(xyz(B));
                        const float tm = A.w * 1.0001f + 1e-3f;
                        for (int k = 0; k < J.n_var && !need; ++k) {
                            const float4* bx = J.var_box + (size_t(r) * kMaxVariant + k) * 2;
                            need = slab_touch(xyz(__ldg(bx)), xyz(__ldg(bx + 1)), o, inv, tm);
                        }
                    }
                }
                const unsigned nb = __ballot_sync(kFull, need);
                if (need) ring[(tail + __popc(nb & lt_mask)) % kAffRing] = e;
                tail += unsigned(__popc(nb));
            }
            __syncwarp();
            const unsigned fr = __ballot_sync(kFull, !alive);  // lanes free for a new path
            const unsigned avail = tail - head, rank = unsigned(__popc(fr & lt_mask));
            if (!alive && rank < avail) {
                const unsigned e = ring[(head + rank) % kAffRing];
                const unsigned code = __ldcg(J.aff_codes + e), sw = __ldcg(J.aff_segw + e);
                const int pixel = int(code >> 6), smp = int(code & 63u);
                if (sw == kSegFull) {
                    const int y = div_magic(pixel, J.W, magic_W);
                    start_path(S, J.W, J.H, pixel - y * J.W, y, smp, int(e), p);
                } else {  // resume where the path's renders part
                    const float4* st = J.seg_state + 4 * size_t(((sw & ~kSegAll) >> 3) - 1u);
                    const float4 a = __ldcg(st), b = __ldcg(st + 1), c = __ldcg(st + 2), q = __ldcg(st + 3);
                    p.o = f3(a.x, a.y, a.z);
                    p.d = f3(a.w, b.x, b.y);
                    p.beta = f3(b.z, b.w, c.x);
                    p.L = f3(c.y, c.z, c.w);
                    p.b = __float_as_int(q.x);
                    p.specular = __float_as_int(q.y) != 0;
                    p.pixel = unsigned(pixel);
                    p.s = smp;
                    p.slot = int(e);
                }
                if (kCount) ++cnt.paths;
                alive = true;
            }
            head += min(avail, unsigned(__popc(fr)));
            __syncwarp();
            if (!__any_sync(kFull, alive)) break;  // ring empty and the render's list used up
            int st = kLive;
            if (alive) st = advance<kCount, false>(S, J.depth, J.rr_start, p, cnt);
            if (alive && st != kLive) {
                unsigned long long* a = acc + size_t(p.pixel) * 3;
                const float* ls = J.aff_lsh + 3 * size_t(p.slot);
                const unsigned long long dx = to_fixed(p.L.x) - to_fixed(__ldcg(ls + 0));
                const unsigned long long dy = to_fixed(p.L.y) - to_fixed(__ldcg(ls + 1));
                const unsigned long long dz = to_fixed(p.L.z) - to_fixed(__ldcg(ls + 2));
                if (dx) atomicAdd(a + 0, dx);
                if (dy) atomicAdd(a + 1, dy);
                if (dz) atomicAdd(a + 2, dz);
                if (dx | dy | dz) {  // mark the pixel as corrected in render r
                    unsigned* fw = J.aff_flags + size_t(r) * J.flag_words + (p.pixel >> 5);
                    const unsigned bit = 1u << (p.pixel & 31u);
                    if (!(__ldcg(fw) & bit)) atomicOr(fw, bit);
                }
                alive = false;
            }
        }
        __syncwarp();
    }
    }
    if (kCount) {
        const unsigned v[kNumCounters] = {warp_sum_u(cnt.sph), warp_sum_u(cnt.quad), warp_sum_u(cnt.box),
                                          warp_sum_u(cnt.paths), warp_sum_u(cnt.vertices), warp_sum_u(cnt.shadow),
                                          warp_sum_u(cnt.rays), 0u};
        if (lane == 0)
            for (int i = 0; i < kNumCounters; ++i) atomicAdd(L.counters + i, (unsigned long long)v[i]);
    }
}

// Epilogue pass of a path-sharing job: one item per listed block, all renders. Lanes form
// segments of `pw` lanes (one render each, one pixel per lane); a segment's error sum uses
// the same shuffle tree as a full warp whose other lanes hold zeros, so the partial is
// bit-identical to the per-render path. Clears the affected radiance it read, so the
// buffers are zero for the next step.
__global__ void __launch_bounds__(kBlock) k_shared_epilogue(const __grid_constant__ TraceLaunch L) {
    __shared__ TraceJob s_job[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    TraceJob& J = s_job[warp];
    const int njobs = L.jobs ? L.njobs : 1;
    for (int jb = 0; jb < njobs; ++jb) {  // the jobs of a packed launch one after another
    {  // job descriptors are host data: the first is copied before the wait on the previous kernel
        const unsigned* src = reinterpret_cast<const unsigned*>(L.jobs ? L.jobs + jb : &L.job0);
        unsigned* dst = reinterpret_cast<unsigned*>(&J);
        for (int i = lane; i < int(sizeof(TraceJob) / 4); i += 32) dst[i] = src[i];
        __syncwarp();
        if (jb == 0) pdl_enter();
    }
    const bool job_shares = J.share != 0;
    __syncwarp();  // every lane has read the descriptor before the next copy may overwrite it
    if (!job_shares) continue;
    const unsigned n_items = __ldcg(J.share_ctl + 0);
    const float inv = mean_scale(J.spp);
    const unsigned gw = blockIdx.x * kWarps + unsigned(warp), nw = gridDim.x * kWarps;
    for (unsigned item = gw; item < n_items; item += nw) {  // listed blocks cost alike: a static split
        const int t = __ldcg(J.aff_tiles + item);
        if (t < 0 || t >= J.tiles) {
            if (lane == 0) atomicOr(L.status, kStatusBadItem);
            break;
        }
        const int x0 = (t % J.tiles_x) * J.bw, y0 = (t / J.tiles_x) * J.bh;
        const int vw = min(J.bw, J.W - x0), vh = min(J.bh, J.H - y0);
        const int npx = vw * vh;
        const int pw = npx <= 8 ? 8 : (npx <= 16 ? 16 : 32);  // lanes per render segment
        const int G = 32 / pw, sub = lane / pw, pl = lane % pw;
        const int px = x0 + pl % vw, py = y0 + pl / vw;
        const bool pix_ok = pl < npx && px < J.W && py < J.H;
        const unsigned long long* sh = J.share_acc + size_t(t) * 96;
        const unsigned long long s0 = pix_ok ? __ldcg(sh + pl) : 0ull, s1 = pix_ok ? __ldcg(sh + 32 + pl) : 0ull,
                                 s2 = pix_ok ? __ldcg(sh + 64 + pl) : 0ull;
        const float4 T = pix_ok ? __ldg(J.target + size_t(py) * J.W + px) : make_float4(0.f, 0.f, 0.f, 0.f);
        const size_t plane = size_t(J.W) * J.H * 3, pix3 = (size_t(py) * J.W + px) * 3;
        const unsigned pixel = pix_ok ? unsigned(py * J.W + px) : 0u, pbit = 1u << (pixel & 31u);
        constexpr int kBatch = 4;  // rounds whose loads are issued before any store
        for (int rb = 0; rb < J.R; rb += kBatch * G) {
            unsigned long long a[kBatch][3];
            bool corr[kBatch];  // render r corrected this pixel: read (and clear) its correction
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                const int r = rb + q * G + sub;
                corr[q] = pix_ok && r < J.R &&
                          (__ldcg(J.aff_flags + size_t(r) * J.flag_words + (pixel >> 5)) & pbit) != 0u;
                const bool ok = corr[q];
                const unsigned long long* af = J.acc_aff + size_t(ok ? r : 0) * plane + (ok ? pix3 : 0);
                a[q][0] = ok ? __ldcg(af + 0) : 0ull;
                a[q][1] = ok ? __ldcg(af + 1) : 0ull;
                a[q][2] = ok ? __ldcg(af + 2) : 0ull;
            }
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                const int r = rb + q * G + sub;
                double e = 0.0;
                if (pix_ok && r < J.R) {
                    if (corr[q]) {
                        unsigned long long* af = J.acc_aff + size_t(r) * plane + pix3;
                        af[0] = 0ull;
                        af[1] = 0ull;
                        af[2] = 0ull;
                    }
                    e = pixel_sq_error(s0 + a[q][0], s1 + a[q][1], s2 + a[q][2], T, unsigned(J.spp), inv);
                }
                for (int o = pw / 2; o > 0; o >>= 1) e += __shfl_xor_sync(kFull, e, o);
                if (pl == 0 && r < J.R) J.partials[size_t(r) * J.tiles + t] = e;
            }
        }
        __syncwarp();
    }
    }
}

// One Adam update (Sec. 3.4: Adam with PyTorch's default betas and eps) of one parameter
// in FP32, as PyTorch's FP32 Adam. The bias corrections 1 - beta^t are formed as
// -expm1(t log1p(beta - 1)), which keeps their relative accuracy while beta^t is near 1.
__device__ __forceinline__ void adam_update(float& th, float& m, float& v, float g, int t, float lr, float b1,
                                            float b2, float eps) {
    m = fmaf(b1, m, (1.0f - b1) * g);
    v = fmaf(b2, v, (1.0f - b2) * g * g);
    const float bc1 = -expm1f(float(t) * log1pf(b1 - 1.0f));
    const float bc2 = -expm1f(float(t) * log1pf(b2 - 1.0f));
    th -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

// ---------------------------------------------------------------------------
// k_finalize: a5 (per-render loss), a6 (gradient, Eq. 10), a7 (Adam)
// ---------------------------------------------------------------------------
// One 256-thread CTA per render of every job in the launch: L_r = (1/3HW) sum of the
// render's block partials in a fixed order (strided per thread into eight accumulators, a
// warp shuffle tree, then the eight warp sums in order). The CTA that completes a job's
// last render forms the gradient in FP64 (one warp per parameter) and applies Adam.
__global__ void __launch_bounds__(kBlock) k_finalize(const __grid_constant__ TraceLaunch L) {
    __shared__ double s_red[kBlock / 32];
    __shared__ int s_job, s_last;
    const int tid = threadIdx.x;
    if (tid == 0) {
        int j = 0;
        if (L.jobs) {
            int lo = 0, hi = L.njobs - 1;  // last job with fin_begin <= blockIdx.x
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (L.jobs[mid].fin_begin <= int(blockIdx.x)) lo = mid; else hi = mid - 1;
            }
            j = lo;
        }
        s_job = j;
    }
    __syncthreads();
    pdl_enter();  // the job lookup above reads host data only
    const TraceJob& J = L.jobs ? L.jobs[s_job] : L.job0;
    const int r = int(blockIdx.x) - J.fin_begin;
    // fixed-order sum of src[i * stride], i < n: strided per thread into eight
    // accumulators, a warp shuffle tree, then the eight warp sums in order (thread 0)
    auto reduce = [&](const double* src, int n, int stride) -> double {
        double a[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) a[q] = 0.0;
        int i = tid;
        for (; i + 31 * kBlock < n; i += 32 * kBlock) {  // 32 loads in flight, then the same adds
            double v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = __ldcg(src + size_t(i + q * kBlock) * stride);
#pragma unroll
            for (int q = 0; q < 32; ++q) a[q & 7] += v[q];
        }
        for (; i + 7 * kBlock < n; i += 8 * kBlock) {
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] += __ldcg(src + size_t(i + q * kBlock) * stride);
        }
        for (; i < n; i += kBlock) a[0] += __ldcg(src + size_t(i) * stride);
        double v = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        v = warp_sum_d(v);
        if ((tid & 31) == 0) s_red[tid >> 5] = v;
        __syncthreads();
        double sum = 0.0;
        if (tid == 0)
            for (int w = 0; w < kBlock / 32; ++w) sum += s_red[w];
        __syncthreads();
        return sum;
    };
    const double lsum = reduce(J.partials + size_t(r) * J.tiles, J.tiles, 1);
    if (tid == 0) {
        const double Lr = lsum / (3.0 * double(J.W) * double(J.H));
        J.losses[r] = Lr;
        if (J.loss_out) J.loss_out[r] = float(Lr);
    }
    if (J.diff)  // pathwise estimator: render r's loss gradient (without the 2 / 3HW factor)
        for (int k = 0; k < J.diff_n; ++k) {
            const double gsum = reduce(J.gpartials + size_t(r) * J.tiles * J.diff_n + k, J.tiles, J.diff_n);
            if (tid == 0) J.rgrads[size_t(r) * kMaxDiff + k] = gsum;
        }
    if (tid == 0) {
        __threadfence();
        s_last = (atomicAdd(J.done, 1u) == unsigned(J.R - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // a6: one warp per parameter, lanes over pairs (fixed order), FP64; a7: Adam in FP32
    const int t = J.step_dev ? __ldcg(J.step_dev) : 0;
    const int warp = tid >> 5, lane = tid & 31;
    for (int d = warp; d < (J.hd ? 0 : J.D); d += kBlock / 32) {  // hd: k_hd_grad
        double g = 0.0;
        if (J.diff) {  // Eq. 9: mean over renders of the pathwise loss gradients
            for (int q = lane; q < J.R; q += 32) g += __ldcg(J.rgrads + size_t(q) * kMaxDiff + d);
            g = warp_sum_d(g) * (2.0 / (3.0 * double(J.W) * double(J.H))) / double(J.R);
        } else if (J.antithetic) {
            const int P = J.R / 2;
            for (int p = lane; p < P; p += 32)
                g += double(J.w[size_t(2 * p) * J.D + d]) * (__ldcg(J.losses + 2 * p) - __ldcg(J.losses + 2 * p + 1));
            g = warp_sum_d(g) / double(2 * P);
        } else {
            for (int q = lane; q < J.R; q += 32) g += double(J.w[size_t(q) * J.D + d]) * __ldcg(J.losses + q);
            g = warp_sum_d(g) / double(J.R);
        }
        if (lane == 0) {
            const float gf = float(g);
            if (J.grad_out) J.grad_out[d] = gf;
            if (J.theta) adam_update(J.theta[d], J.m[d], J.v[d], gf, t + 1, J.lr, J.b1, J.b2, J.eps);
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (J.step_dev) *J.step_dev = t + 1;
        *J.done = 0u;  // ready for the next launch
    }
}

// ---------------------------------------------------------------------------
// standalone Adam and raw Philox
// ---------------------------------------------------------------------------
__global__ void k_adam(int D, float* theta, float* m, float* v, const float* g, int t, float lr, float b1, float b2,
                       float eps) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    adam_update(theta[d], m[d], v[d], g[d], t, lr, b1, b2, eps);
}

__global__ void k_philox(unsigned long long seed, unsigned c0, unsigned c1, unsigned c2, unsigned c3, int n,
                         uint4* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = philox(make_uint4(c0 + unsigned(i), c1, c2, c3), unsigned(seed), unsigned(seed >> 32));
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// Launch with the programmatic-stream-serialisation attribute (see pdl_enter).
template <typename... Args>
static cudaError_t launch_pdl(void (*kernel)(Args...), int grid, int block, cudaStream_t stream, const Args&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(unsigned(block));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_instantiate(const InstLaunch& L, cudaStream_t stream) {
    if (L.total_blocks <= 0) return cudaSuccess;
    return launch_pdl(k_instantiate, L.total_blocks, kInstBlock, stream, L);
}

int trace_diff_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<false, false, false, 8>, kDiffBlock, 0);
    return n > 0 ? n : 1;
}

int trace_blocks_per_sm(bool render_mode) {
    int n = 0;
    if (render_mode)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<true, false, false, 0>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<false, false, false, 0>, kBlock, 0);
    return n > 0 ? n : 1;
}

int trace_group_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_group<false>, kGroupBlock, 0);
    return n > 0 ? n : 1;
}

int trace_emit_blocks_per_sm() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace_emit<false>, kGroupBlock, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_trace(const TraceLaunch& L, bool render_mode, int grid, cudaStream_t stream) {
    if (L.total_items <= 0) return cudaSuccess;
    const bool count = L.counters != nullptr;
    if (L.group == 2 && !render_mode)
        return launch_pdl(count ? k_trace_emit<true> : k_trace_emit<false>, grid, kGroupBlock, stream, L);
    if (L.group && !render_mode)
        return launch_pdl(count ? k_trace_group<true> : k_trace_group<false>, grid, kGroupBlock, stream, L);
    const bool share = !render_mode && L.share;
    if (render_mode) return launch_pdl(count ? k_trace<true, true, false, 0> : k_trace<true, false, false, 0>, grid, kBlock,
                                       stream, L);
    if (share) return launch_pdl(count ? k_trace<false, true, true, 0> : k_trace<false, false, true, 0>, grid, kBlock,
                                 stream, L);
    if (L.diff_nd == 4)
        return launch_pdl(count ? k_trace<false, true, false, 4> : k_trace<false, false, false, 4>, grid, kDiffBlock,
                          stream, L);
    if (L.diff_nd == 6)
        return launch_pdl(count ? k_trace<false, true, false, 6> : k_trace<false, false, false, 6>, grid, kDiffBlock,
                          stream, L);
    if (L.diff_nd == 8)
        return launch_pdl(count ? k_trace<false, true, false, 8> : k_trace<false, false, false, 8>, grid, kDiffBlock,
                          stream, L);
    return launch_pdl(count ? k_trace<false, true, false, 0> : k_trace<false, false, false, 0>, grid, kBlock, stream, L);
}

cudaError_t launch_trace_affected(const TraceLaunch& L, int grid, cudaStream_t stream) {
    return launch_pdl(L.counters ? k_trace_affected<true> : k_trace_affected<false>, grid, kBlock, stream, L);
}

cudaError_t launch_shared_epilogue(const TraceLaunch& L, int grid, cudaStream_t stream) {
    return launch_pdl(k_shared_epilogue, grid, kBlock, stream, L);
}

cudaError_t launch_finalize(const TraceLaunch& L, int n_renders, cudaStream_t stream) {
    if (n_renders <= 0) return cudaSuccess;
    return launch_pdl(k_finalize, n_renders, kBlock, stream, L);
}

cudaError_t launch_adam(int D, float* theta, float* m, float* v, const float* g, int t, float lr, float b1,
                        float b2, float eps, cudaStream_t stream) {
    k_adam<<<(D + 63) / 64, 64, 0, stream>>>(D, theta, m, v, g, t, lr, b1, b2, eps);
    return cudaGetLastError();
}

cudaError_t launch_philox(unsigned long long seed, unsigned c0, unsigned c1, unsigned c2, unsigned c3, int n,
                          uint32_t* out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_philox<<<(n + 255) / 256, 256, 0, stream>>>(seed, c0, c1, c2, c3, n, reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// High-dimensional parameters (texture scenes): a1 and a6/a7 over D > kMaxD
// ---------------------------------------------------------------------------
// Uniform number k of draw `index` (stream PERTURB): word k mod 4 of Philox block k / 4,
// the same counter layout as the small-D sampler of k_instantiate.
__device__ __forceinline__ float perturb_uniform(const HdDraws& H, unsigned index, unsigned step, int k) {
    const uint4 w = philox(make_uint4(index, unsigned(k >> 2), step, kTagPerturb << 28), unsigned(H.seed),
                           unsigned(H.seed >> 32));
    const unsigned x = (k & 3) == 0 ? w.x : ((k & 3) == 1 ? w.y : ((k & 3) == 2 ? w.z : w.w));
    return u01(x);
}

// Uniforms k and k + 1 of a draw (one Philox block unless k is a block's last word).
__device__ __forceinline__ float2 perturb_uniform_pair(const HdDraws& H, unsigned index, unsigned step, int k) {
    const uint4 w = philox(make_uint4(index, unsigned(k >> 2), step, kTagPerturb << 28), unsigned(H.seed),
                           unsigned(H.seed >> 32));
    const int q = k & 3;
    const unsigned xa = q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
    unsigned xb;
    if (q < 3) {
        xb = q == 0 ? w.y : (q == 1 ? w.z : w.w);
    } else {
        xb = philox(make_uint4(index, unsigned(k >> 2) + 1u, step, kTagPerturb << 28), unsigned(H.seed),
                    unsigned(H.seed >> 32)).x;
    }
    return make_float2(u01(xa), u01(xb));
}

// Box-Muller normals 2m and 2m + 1 of a draw whose pairs start at uniform `base` (as
// bm_normal): (cos, sin) parts.
__device__ __forceinline__ float2 hd_normal_pair(const HdDraws& H, unsigned index, unsigned step, int base, int m) {
    const float2 ab = perturb_uniform_pair(H, index, step, base + 2 * m);
    const float rad = sqrtf(-2.0f * logf(ab.x));
    float sn, cs;
    sincospif(2.0f * ab.y, &sn, &cs);
    return make_float2(rad * cs, rad * sn);
}

__device__ __forceinline__ unsigned hd_step(const HdDraws& H) {
    return H.step + (H.step_dev ? unsigned(*H.step_dev) : 0u);
}

// Radial sampler (Sec. 3.2, reading R1) in D dimensions: the norm of the D Box-Muller
// normals and the chi_{D+1} radius (sum of (D+1)/2 exponentials, plus one more squared
// normal when D is even). Each draw's terms are split into norm_split contiguous parts,
// one CTA each, summed in FP64 in a fixed order; the CTA that finishes a draw's last part
// adds the parts in order.
__global__ void __launch_bounds__(kBlock) k_hd_norms(const HdDraws H) {
    __shared__ double s_z[kBlock / 32], s_r[kBlock / 32];
    __shared__ int s_last;
    const int split = H.norm_split, part = int(blockIdx.x) % split;
    const unsigned local = blockIdx.x / unsigned(split);
    pdl_enter();
    const unsigned index = local + unsigned(H.draw_begin), step = hd_step(H);
    const int D = H.D, n_exp = (D + 1) / 2, nz = D + (D % 2 == 0 ? 1 : 0), npair = (nz + 1) / 2;
    const int m0 = int((long long)npair * part / split), m1 = int((long long)npair * (part + 1) / split);
    const int e0 = int((long long)n_exp * part / split), e1 = int((long long)n_exp * (part + 1) / split);
    double zs = 0.0, rs = 0.0;
    for (int m = m0 + int(threadIdx.x); m < m1; m += kBlock) {  // normals 2m and 2m + 1
        const float2 z = hd_normal_pair(H, index, step, n_exp, m);
        const float q0 = z.x * z.x, q1 = z.y * z.y;
        if (2 * m < D) zs += double(q0); else rs += double(q0);
        if (2 * m + 1 < D) zs += double(q1); else if (2 * m + 1 < nz) rs += double(q1);
    }
    for (int j = e0 + int(threadIdx.x); j < e1; j += kBlock)
        rs += double(-2.0f * logf(perturb_uniform(H, index, step, j)));
    zs = warp_sum_d(zs);
    rs = warp_sum_d(rs);
    if ((threadIdx.x & 31) == 0) {
        s_z[threadIdx.x >> 5] = zs;
        s_r[threadIdx.x >> 5] = rs;
    }
    __syncthreads();
    HdNorm& N = H.norms[local];
    if (threadIdx.x == 0) {
        double z = 0.0, r = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) {
            z += s_z[w];
            r += s_r[w];
        }
        N.part[part] = make_double2(z, r);
        __threadfence();
        s_last = atomicAdd(&N.ctr, 1u) == unsigned(split - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double z = 0.0, r = 0.0;
        for (int q = 0; q < split; ++q) {
            const double2 v = __ldcg(&N.part[q]);
            z += v.x;
            r += v.y;
        }
        N.v = make_float2(float(sqrt(z)), float(sqrt(r)));
        N.ctr = 0u;  // ready for the next launch
    }
}

// One thread per (render, pair of parameters 2m, 2m + 1): tau, w and theta + tau of every
// sampler (as the small-D sampler, per dimension), antithetic renders negated. A pair of
// Box-Muller normals comes from one pair of uniforms, so a thread forms both.
__global__ void __launch_bounds__(kBlock) k_hd_perturb(const HdDraws H) {
    pdl_enter();
    const size_t half = (size_t(H.D) + 1) / 2;
    const size_t i = size_t(blockIdx.x) * kBlock + threadIdx.x;
    if (i >= size_t(H.R) * half) return;
    const int r = int(i / half), m = int(i - size_t(r) * half);
    const bool anti = H.antithetic && (r & 1);
    const unsigned local = H.antithetic ? unsigned(r >> 1) : unsigned(r), step = hd_step(H);
    const unsigned index = local + unsigned(H.draw_begin);
    float tt[2], wt[2];
    if (H.sampler == kRadial) {
        const float2 z = hd_normal_pair(H, index, step, (H.D + 1) / 2, m);
        const float2 nr = H.norms[local].v;
        const float dir0 = z.x / nr.x, dir1 = z.y / nr.x;
        tt[0] = nr.y * dir0;
        wt[0] = H.c_radial * dir0;
        tt[1] = nr.y * dir1;
        wt[1] = H.c_radial * dir1;
    } else if (H.sampler == kPerDim) {
        const float2 xi2 = perturb_uniform_pair(H, index, step, 2 * m);
        const float c1 = 0.7978845608028654f;  // sqrt(2/pi)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float xi = k == 0 ? xi2.x : xi2.y;
            if (xi < 0.5f) {
                tt[k] = -sqrtf(-2.0f * logf(2.0f * xi));
                wt[k] = -c1;
            } else {
                tt[k] = sqrtf(-2.0f * logf(2.0f * (1.0f - xi)));
                wt[k] = c1;
            }
        }
    } else {
        const float2 z = hd_normal_pair(H, index, step, 0, m);
        tt[0] = wt[0] = z.x;
        tt[1] = wt[1] = z.y;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int d = 2 * m + k;
        if (d >= H.D) break;
        const float sg = sigma_sched(H.sigma, H.anneal, H.total_steps, H.sigma_min, d, int(step));
        float tau = sg * tt[k], w = wt[k] / sg;
        if (anti) {
            tau = -tau;
            w = -w;
        }
        const size_t o = size_t(r) * size_t(H.D) + size_t(d);
        if (H.theta_out) H.theta_out[o] = H.theta[d] + tau;  // FP32 sum: the parameters this render gets
        if (H.tau_out) H.tau_out[o] = tau;
        if (H.w_out) H.w_out[o] = w;
    }
}

// a6 + a7 over D parameters: g_d = (1/2P) sum_p w_{2p,d} (L_2p - L_2p+1) (a skinny GEMV,
// W^T dL, fixed order over p in FP64), then Adam with t = the already advanced step.
__global__ void __launch_bounds__(kBlock) k_hd_grad(const HdGrad G) {
    pdl_enter();
    const int d = int(blockIdx.x) * kBlock + int(threadIdx.x);
    if (d >= G.D) return;
    double g = 0.0;
    if (G.antithetic) {
        const int P = G.R / 2;
        for (int p = 0; p < P; ++p)
            g += double(G.w[size_t(2 * p) * G.D + d]) * (__ldcg(G.losses + 2 * p) - __ldcg(G.losses + 2 * p + 1));
        g /= double(2 * P);
    } else {
        for (int q = 0; q < G.R; ++q) g += double(G.w[size_t(q) * G.D + d]) * __ldcg(G.losses + q);
        g /= double(G.R);
    }
    const float gf = float(g);
    if (G.grad_out) G.grad_out[d] = gf;
    if (G.theta) adam_update(G.theta[d], G.m[d], G.v[d], gf, __ldcg(G.step_dev), G.lr, G.b1, G.b2, G.eps);
}

cudaError_t launch_hd_draws(const HdDraws& H, cudaStream_t stream) {
    if (H.D <= 0 || H.R <= 0) return cudaSuccess;
    if (H.sampler == kRadial) {
        if (H.norm_split < 1 || H.norm_split > kNormSplitMax) return cudaErrorInvalidValue;
        const cudaError_t e = launch_pdl(k_hd_norms, (H.antithetic ? H.R / 2 : H.R) * H.norm_split, kBlock, stream, H);
        if (e != cudaSuccess) return e;
    }
    const size_t n = size_t(H.R) * ((size_t(H.D) + 1) / 2);  // one thread per (render, parameter pair)
    return launch_pdl(k_hd_perturb, int((n + kBlock - 1) / kBlock), kBlock, stream, H);
}

cudaError_t launch_hd_grad(const HdGrad& G, cudaStream_t stream) {
    if (G.D <= 0) return cudaSuccess;
    return launch_pdl(k_hd_grad, (G.D + kBlock - 1) / kBlock, kBlock, stream, G);
}

// ---------------------------------------------------------------------------
// FP32 issue-rate probe: the denominator of the render kernels' roofline
// ---------------------------------------------------------------------------
// Every thread runs kFfmaChains independent fused multiply-add chains, so each warp
// always has an FMA ready; a full-occupancy grid then issues FFMA on every FP32 lane
// of every SM each cycle, up to the loop's few integer instructions.
constexpr int kFfmaChains = 8;

__global__ void __launch_bounds__(kBlock) k_ffma_probe(float* out, int iters, float b, float c) {
    float a[kFfmaChains];
#pragma unroll
    for (int i = 0; i < kFfmaChains; ++i) a[i] = float(threadIdx.x) * 1e-7f + float(i);
    for (int k = 0; k < iters; ++k) {
#pragma unroll 16
        for (int i = 0; i < kFfmaChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kFfmaChains; ++i) s += a[i];
    out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

int ffma_probe_flops_per_thread_iter() { return 2 * kFfmaChains; }

cudaError_t launch_ffma_probe(float* out, int blocks, int iters, cudaStream_t stream) {
    if (blocks <= 0 || iters <= 0) return cudaErrorInvalidValue;
    k_ffma_probe<<<blocks, kBlock, 0, stream>>>(out, iters, 0.9999999f, 1e-7f);
    return cudaGetLastError();
}

}  // namespace prdpt
