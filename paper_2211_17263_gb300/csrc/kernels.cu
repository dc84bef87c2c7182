// kernels.cu -- sm_103a kernels of the plateau-reduced gradient estimator.
//
//   k_instantiate   one CTA per render: Philox draws -> perturbation tau and weight
//                   w (Sec. 3.2, Eq. 11, Algorithm 1), theta +- tau bound into the
//                   scene (Eq. 10's P(theta - tau_i)), derived constants precomputed.
//   k_trace         persistent render kernel: CTAs pull (render, tile) items from a
//                   work queue, stage the render's scene in shared memory, path-trace
//                   every pixel of the tile (Eq. 1 / Eq. 3), and reduce the squared
//                   pixel errors against the target to one tile partial (the image
//                   never reaches HBM). The CTA that completes a job's last tile
//                   forms L_r, the gradient of Eq. 10 and the Adam step.
//   k_adam          standalone Adam update.
//   k_philox        raw Philox words (for bit-exact checks of the random streams).
//
// FP32 throughout the tracer; loss partials are FP32 per tile and summed in FP64
// in a fixed order, so every result is deterministic and independent of which CTA
// processed which tile.
#include <cstdint>

#include "internal.h"

namespace prdpt {

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
__device__ __forceinline__ float sigma_at(const InstJob& J, int d, int t) {
    const float s0 = J.sigma[d];
    if (!J.anneal) return s0;
    const int w = J.total_steps / 2;
    if (t < w || J.total_steps - w <= 0) return s0;
    float frac = float(t - w) / float(J.total_steps - w);
    frac = fminf(frac, 1.0f);
    return s0 - frac * (s0 - J.sigma_min);
}

// ---------------------------------------------------------------------------
// k_instantiate: one CTA (kInstBlock threads) per render
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kInstBlock) k_instantiate(const InstLaunch L) {
    __shared__ float s_u[4 * 32];
    __shared__ float s_red[kInstBlock];
    __shared__ float s_theta[kMaxD];
    __shared__ float s_w[kMaxD];
    __shared__ float s_scalar[2];
    __shared__ int s_job;

    const int tid = threadIdx.x;
    if (blockIdx.x == 0 && tid == 0 && L.queue_reset) *L.queue_reset = 0u;
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
    const unsigned step = J.step + (J.step_dev ? (unsigned)*J.step_dev : 0u);

    // ---- a1: perturbation and weight of render r --------------------------------
    if (J.render_mode) {
        if (tid < D) {
            s_theta[tid] = J.theta[r * D + tid];
            s_w[tid] = 0.0f;
        }
    } else {
        const bool anti = J.antithetic && (r & 1);
        const unsigned index = J.antithetic ? unsigned(r >> 1) : unsigned(r);
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
            s_theta[tid] = J.theta[tid] + tau;  // FP32 sum: the parameters this render gets
            s_w[tid] = w;
            if (J.tau_out) J.tau_out[r * D + tid] = tau;
            if (J.w_out) J.w_out[r * D + tid] = w;
        }
    }
    __syncthreads();
    if (!J.scenes) return;  // draws only

    // ---- a2: bind theta_r into the scene -----------------------------------------
    const BaseScene& B = *J.base;
    InstScene& S = J.scenes[r];
    if (tid < B.n_prims) {
        const int i = tid;
        const int type = B.prim_type[i], mat = B.prim_mat[i], slot = B.prim_slot[i];
        float g[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) g[q] = B.prim_geom[i][q];
        for (int d = 0; d < D; ++d) {
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
        for (int d = 0; d < D; ++d) {
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
    if (tid == 0) {
        S.n_sph = B.n_sph;
        S.n_quad = B.n_quad;
        S.n_box = B.n_box;
        const unsigned field = J.render_mode ? (J.crn ? 0u : unsigned(r)) : (J.crn ? 0u : unsigned(r + 1));
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

__device__ __forceinline__ float sphere_t(const InstScene& S, int i, float3 o, float3 d) {
    const float4 a = S.prim[i][0];
    const float r2 = S.prim[i][1].x;
    const float3 oc = o - xyz(a);
    const float b = dot3(oc, d);
    const float3 l = oc - d * b;  // centre offset from the ray line: better conditioned than b^2 - c
    const float disc = r2 - dot3(l, l);
    if (disc < 0.0f) return INFINITY;
    const float sq = sqrtf(disc);
    float t = -b - sq;
    if (t <= kEps) t = -b + sq;
    return (t > kEps) ? t : INFINITY;
}

__device__ __forceinline__ float quad_t(const InstScene& S, int i, float3 o, float3 d) {
    const float4 a = S.prim[i][0], nb = S.prim[i][1], uu = S.prim[i][2], vv = S.prim[i][3];
    const float3 n = xyz(nb);
    const float den = dot3(n, d);
    if (fabsf(den) < 1e-12f) return INFINITY;
    const float3 co = xyz(a) - o;
    const float t = dot3(n, co) / den;
    if (!(t > kEps)) return INFINITY;
    const float3 q = d * t - co;  // hit point relative to the centre
    const float pa = dot3(q, xyz(uu)) * uu.w, pb = dot3(q, xyz(vv)) * vv.w;
    return (fabsf(pa) <= 0.5f && fabsf(pb) <= 0.5f) ? t : INFINITY;
}

// Slab test; returns the nearest t > eps (entering, or leaving from inside).
__device__ __forceinline__ float box_t(const InstScene& S, int i, float3 o, float3 inv) {
    const float3 lo = xyz(S.prim[i][0]), hi = xyz(S.prim[i][1]);
    const float tx0 = (lo.x - o.x) * inv.x, tx1 = (hi.x - o.x) * inv.x;
    const float ty0 = (lo.y - o.y) * inv.y, ty1 = (hi.y - o.y) * inv.y;
    const float tz0 = (lo.z - o.z) * inv.z, tz1 = (hi.z - o.z) * inv.z;
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fminf(tz0, tz1));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    if (tn > tf) return INFINITY;
    if (tn > kEps) return tn;
    return (tf > kEps) ? tf : INFINITY;
}

// Outward normal of box i at the hit found by box_t.
__device__ __forceinline__ float3 box_normal(const InstScene& S, int i, float3 o, float3 d, float3 inv) {
    const float3 lo = xyz(S.prim[i][0]), hi = xyz(S.prim[i][1]);
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

template <bool kCount>
__device__ __forceinline__ Hit closest_hit(const InstScene& S, float3 o, float3 d, Counters& cnt) {
    Hit h{INFINITY, -1, 0};
    const int ns = S.n_sph, nq = S.n_quad, nb = S.n_box;
    if (kCount) {
        cnt.sph += ns;
        cnt.quad += nq;
        cnt.box += nb;
        ++cnt.rays;
    }
    for (int i = 0; i < ns; ++i) {
        const float t = sphere_t(S, i, o, d);
        if (t < h.t) { h.t = t; h.slot = i; h.type = kSphere; }
    }
    for (int i = ns; i < ns + nq; ++i) {
        const float t = quad_t(S, i, o, d);
        if (t < h.t) { h.t = t; h.slot = i; h.type = kQuad; }
    }
    if (nb) {
        const float3 inv = f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
        for (int i = ns + nq; i < ns + nq + nb; ++i) {
            const float t = box_t(S, i, o, inv);
            if (t < h.t) { h.t = t; h.slot = i; h.type = kBox; }
        }
    }
    return h;
}

// Is anything but primitive slot `skip` hit closer than dist?
template <bool kCount>
__device__ __forceinline__ bool occluded(const InstScene& S, float3 o, float3 d, float dist, int skip, Counters& cnt) {
    const int ns = S.n_sph, nq = S.n_quad, nb = S.n_box;
    if (kCount) ++cnt.shadow;
    for (int i = 0; i < ns; ++i) {
        if (i == skip) continue;
        if (kCount) ++cnt.sph;
        if (sphere_t(S, i, o, d) < dist) return true;
    }
    for (int i = ns; i < ns + nq; ++i) {
        if (i == skip) continue;
        if (kCount) ++cnt.quad;
        if (quad_t(S, i, o, d) < dist) return true;
    }
    if (nb) {
        const float3 inv = f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
        for (int i = ns + nq; i < ns + nq + nb; ++i) {
            if (i == skip) continue;
            if (kCount) ++cnt.box;
            if (box_t(S, i, o, inv) < dist) return true;
        }
    }
    return false;
}

__device__ __forceinline__ float4 path_uniforms(const InstScene& S, unsigned pixel, int s, int b, int slot,
                                                uint4* words = nullptr) {
    const unsigned c1 = unsigned(s) | (unsigned(b) << 16) | (unsigned(slot) << 24);
    const uint4 w = philox(make_uint4(pixel, c1, S.step, S.c3), S.seed_lo, S.seed_hi);
    if (words) *words = w;
    return make_float4(u01(w.x), u01(w.y), u01(w.z), u01(w.w));
}

// Orthonormal basis around unit n (Duff et al. 2017).
__device__ __forceinline__ void onb(float3 n, float3& t1, float3& t2) {
    const float sg = n.z >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + n.z);
    const float b = n.x * n.y * a;
    t1 = f3(1.0f + sg * n.x * n.x * a, sg * b, -sg * n.x);
    t2 = f3(b, sg + n.y * n.y * a, -n.y);
}

// Radiance of one path sample through pixel (x, y): unidirectional path tracing
// with next-event estimation on diffuse vertices (the Monte-Carlo estimate of
// Eq. 1 whose pixel average is Eq. 3).
template <bool kCount>
__device__ float3 trace_path(const InstScene& S, int W, int H, int depth, int rr_start, int x, int y, int s,
                             Counters& cnt) {
    const unsigned pixel = unsigned(y * W + x);
    const float4 jit = path_uniforms(S, pixel, s, 0, 2);
    const float th = S.eye.w, aspect = S.fwd.w;
    const float sx = (float(2 * x - W) + 2.0f * jit.x) * (aspect * th / float(W));
    const float sy = (float(H - 2 * y) - 2.0f * jit.y) * (th / float(H));
    float3 o = xyz(S.eye);
    float3 d = normalized(xyz(S.fwd) + xyz(S.right) * sx + xyz(S.up) * sy);
    float3 L = f3(0.f, 0.f, 0.f), beta = f3(1.f, 1.f, 1.f);
    bool specular = true;
    if (kCount) ++cnt.paths;
    for (int b = 0; b < depth; ++b) {
        const Hit h = closest_hit<kCount>(S, o, d, cnt);
        if (h.slot < 0) {
            L = L + beta * xyz(S.bg);
            break;
        }
        if (kCount) ++cnt.vertices;
        const float3 p = o + d * h.t;
        float3 ng;
        int mat;
        if (h.type == kSphere) {
            const float4 a = S.prim[h.slot][0];
            ng = (p - xyz(a)) * S.prim[h.slot][1].y;
            mat = as_int(S.prim[h.slot][1].z);
        } else if (h.type == kQuad) {
            ng = xyz(S.prim[h.slot][1]);
            mat = as_int(S.prim[h.slot][0].w);
        } else {
            ng = box_normal(S, h.slot, o, d, f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z));
            mat = as_int(S.prim[h.slot][0].w);
        }
        const float4 m0 = S.mat[mat][0], m1 = S.mat[mat][1];
        const int mtype = as_int(m0.w);
        const float3 albedo = xyz(m0), emission = xyz(m1);
        if (specular && (emission.x > 0.f || emission.y > 0.f || emission.z > 0.f) && dot3(d, ng) < 0.0f)
            L = L + beta * emission;
        const bool last = (b + 1 >= depth);
        float4 u;
        if (mtype == kDiffuse) {
            const float3 ns = dot3(ng, d) < 0.0f ? ng : ng * -1.0f;
            const float3 po = p + ns * kEps;
            if (S.n_lights > 0) {  // next-event estimation: one emitter, uniform area sample
                uint4 words;
                const float4 lu = path_uniforms(S, pixel, s, b, 1, &words);
                int li = int((((words.z >> 9) * 2u + 1u) * unsigned(S.n_lights)) >> 24);  // floor(u * n) exactly
                li = min(li, S.n_lights - 1);
                const int4 lt = S.light[li];
                float3 yl, ny;
                if (lt.x == kQuad) {
                    const float3 uu = xyz(S.prim[lt.y][2]), vv = xyz(S.prim[lt.y][3]);
                    yl = xyz(S.prim[lt.y][0]) + uu * (lu.x - 0.5f) + vv * (lu.y - 0.5f);
                    ny = xyz(S.prim[lt.y][1]);
                } else {
                    const float z = 1.0f - 2.0f * lu.x;
                    const float rr = sqrtf(fmaxf(0.0f, 1.0f - z * z));
                    float sp, cp;
                    sincospif(2.0f * lu.y, &sp, &cp);
                    ny = f3(rr * cp, rr * sp, z);
                    yl = xyz(S.prim[lt.y][0]) + ny * S.prim[lt.y][0].w;
                }
                const float3 dv = yl - po;
                const float dist2 = dot3(dv, dv);
                const float inv_dist = rsqrtf(dist2);
                const float3 wi = dv * inv_dist;
                const float cx = dot3(ns, wi), cl = -dot3(ny, wi);
                if (cx > 0.0f && cl > 0.0f) {
                    if (!occluded<kCount>(S, po, wi, dist2 * inv_dist, lt.y, cnt)) {
                        const float g = cx * cl / dist2 * S.light_area[li] * float(S.n_lights) * 0.3183098861837907f;
                        L = L + beta * albedo * xyz(S.mat[lt.w][1]) * g;
                    }
                }
            }
            if (last) break;
            u = path_uniforms(S, pixel, s, b, 0);
            const float rad = sqrtf(u.x);
            float sp, cp;
            sincospif(2.0f * u.y, &sp, &cp);
            float3 t1, t2;
            onb(ns, t1, t2);
            const float3 wo = t1 * (rad * cp) + t2 * (rad * sp) + ns * sqrtf(fmaxf(0.0f, 1.0f - u.x));
            beta = beta * albedo;
            o = po;
            d = normalized(wo);
            specular = false;
        } else if (mtype == kMirror) {
            if (last) break;
            u = path_uniforms(S, pixel, s, b, 0);
            const float3 ns = dot3(ng, d) < 0.0f ? ng : ng * -1.0f;
            d = normalized(d - ns * (2.0f * dot3(d, ns)));
            o = p + ns * kEps;
            beta = beta * albedo;
            specular = true;
        } else {  // smooth dielectric: exact unpolarised Fresnel, reflect or refract
            if (last) break;
            u = path_uniforms(S, pixel, s, b, 0);
            float ci = -dot3(d, ng);
            float eta;
            float3 n;
            if (ci > 0.0f) {
                eta = 1.0f / m1.w;
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
                const float rs = (eta * ci - ct) / (eta * ci + ct);
                const float rp = (ci - eta * ct) / (ci + eta * ct);
                F = 0.5f * (rs * rs + rp * rp);
            }
            if (u.z < F) {
                d = normalized(d + n * (2.0f * ci));
                o = p + n * kEps;
            } else {
                d = normalized(d * eta + n * (eta * ci - ct));
                o = p - n * kEps;
            }
            beta = beta * albedo;
            specular = true;
        }
        if (maxc(beta) <= 0.0f) break;
        if (rr_start >= 0 && b >= rr_start) {  // Russian roulette on slot 0's fourth uniform
            const float q = fminf(0.95f, maxc(beta));
            if (u.w >= q) break;
            beta = beta * (1.0f / q);
        }
    }
    return L;
}

// ---------------------------------------------------------------------------
// k_trace: persistent render + fused loss/gradient/Adam epilogue
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned warp_sum_u(unsigned v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Loss of every render, the gradient of Eq. 10 and (for a resident job) the Adam
// step. Run by the one CTA that finished the job's last tile.
__device__ void finalize_job(const TraceJob& J, double* s_L) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double norm = 1.0 / (3.0 * double(J.W) * double(J.H));
    for (int r = warp; r < J.R; r += kBlock / 32) {
        double acc = 0.0;
        for (int i = lane; i < J.tiles; i += 32) acc += double(__ldcg(J.partials + size_t(r) * J.tiles + i));
        acc = warp_sum_d(acc);
        if (lane == 0) s_L[r] = acc * norm;
    }
    __syncthreads();
    if (J.loss_out)
        for (int r = tid; r < J.R; r += kBlock) J.loss_out[r] = float(s_L[r]);
    int t = 0;
    if (J.step_dev) t = *J.step_dev;
    __syncthreads();
    if (tid < J.D) {
        const int d = tid;
        double g = 0.0;
        if (J.antithetic) {
            const int P = J.R / 2;
            for (int p = 0; p < P; ++p) g += double(J.w[size_t(2 * p) * J.D + d]) * (s_L[2 * p] - s_L[2 * p + 1]);
            g /= double(2 * P);
        } else {
            for (int r = 0; r < J.R; ++r) g += double(J.w[size_t(r) * J.D + d]) * s_L[r];
            g /= double(J.R);
        }
        const float gf = float(g);
        if (J.grad_out) J.grad_out[d] = gf;
        if (J.theta) {  // Adam (Kingma & Ba), state in FP32, arithmetic in FP64
            const int tt = t + 1;
            const double m = double(J.b1) * J.m[d] + (1.0 - double(J.b1)) * double(gf);
            const double v = double(J.b2) * J.v[d] + (1.0 - double(J.b2)) * double(gf) * double(gf);
            const double mh = m / (1.0 - pow(double(J.b1), tt));
            const double vh = v / (1.0 - pow(double(J.b2), tt));
            J.m[d] = float(m);
            J.v[d] = float(v);
            J.theta[d] = float(double(J.theta[d]) - double(J.lr) * mh / (sqrt(vh) + double(J.eps)));
        }
    }
    if (tid == 0) {
        if (J.step_dev) *J.step_dev = t + 1;
        *J.done = 0u;  // ready for the next launch
    }
}

template <bool kRender, bool kCount>
__global__ void __launch_bounds__(kBlock) k_trace(const TraceLaunch L) {
    __shared__ InstScene s_scene;
    __shared__ TraceJob s_job;
    __shared__ float s_acc[3][kBlock];
    __shared__ float s_red[kBlock / 32];
    __shared__ double s_L[kMaxRenders];
    __shared__ int s_item, s_jobi, s_last;
    __shared__ unsigned s_cnt[kNumCounters][kBlock / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int cur_job = -1, cur_r = -1;
    Counters cnt{0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};

    for (;;) {
        if (tid == 0) {
            const int item = int(atomicAdd(L.queue, 1u));
            s_item = item;
            int j = 0;
            if (item < L.total_items && L.jobs) {
                int lo = 0, hi = L.njobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (L.jobs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
                }
                j = lo;
            }
            s_jobi = j;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= L.total_items) break;
        const int j = s_jobi;
        if (j != cur_job) {
            if (tid == 0) s_job = L.jobs ? L.jobs[j] : L.job0;
            __syncthreads();
        }
        const TraceJob& J = s_job;
        const int li = item - J.item_begin;
        const int r = li % J.R, t = li / J.R;  // tile-major: consecutive items share pixels
        if (r >= J.R || t >= J.tiles) {
            if (tid == 0) atomicOr(L.status, kStatusBadItem);
            break;
        }
        if (j != cur_job || r != cur_r) {  // stage the render's scene in shared memory
            const float4* src = reinterpret_cast<const float4*>(J.scenes + r);
            float4* dst = reinterpret_cast<float4*>(&s_scene);
            for (int i = tid; i < int(sizeof(InstScene) / 16); i += kBlock) dst[i] = __ldg(src + i);
            cur_job = j;
            cur_r = r;
            __syncthreads();
        }
        // tile geometry: k threads per pixel, warps cover 8x4 pixel blocks
        int TW, TH;
        tile_shape(J.k, &TW, &TH);
        const int npix = kBlock / J.k;
        const int q = tid % npix, c = tid / npix;
        const int g = q >> 5, ql = q & 31;
        const int gx = g % (TW / 8), gy = g / (TW / 8);
        const int px = (t % J.tiles_x) * TW + gx * 8 + (ql & 7);
        const int py = (t / J.tiles_x) * TH + gy * 4 + (ql >> 3);
        const bool inside = px < J.W && py < J.H;

        float3 rad = f3(0.f, 0.f, 0.f);
        if (inside)
            for (int s = c; s < J.spp; s += J.k)
                rad = rad + trace_path<kCount>(s_scene, J.W, J.H, J.depth, J.rr_start, px, py, s, cnt);
        if (J.k > 1) {  // combine the k sample chunks of each pixel in chunk order
            s_acc[0][tid] = rad.x;
            s_acc[1][tid] = rad.y;
            s_acc[2][tid] = rad.z;
            __syncthreads();
            if (c == 0) {
                for (int cc = 1; cc < J.k; ++cc) {
                    rad.x += s_acc[0][q + cc * npix];
                    rad.y += s_acc[1][q + cc * npix];
                    rad.z += s_acc[2][q + cc * npix];
                }
            }
        }
        const float inv_spp = 1.0f / float(J.spp);
        const float3 I = rad * inv_spp;
        if (kRender) {
            if (c == 0 && inside)
                J.images[(size_t(r) * J.H + py) * J.W + px] = make_float4(I.x, I.y, I.z, 0.0f);
            __syncthreads();
        } else {
            float e = 0.0f;
            if (c == 0 && inside) {  // a4: squared error of the pixel mean against the target
                const float4 T = __ldg(J.target + size_t(py) * J.W + px);
                const float ex = I.x - T.x, ey = I.y - T.y, ez = I.z - T.z;
                e = ex * ex + ey * ey + ez * ez;
            }
            e = warp_sum(e);  // a5: warp shuffle, then CTA, then one partial per tile
            if (lane == 0) s_red[warp] = e;
            __syncthreads();
            if (tid == 0) {
                float tot = 0.0f;
                for (int w = 0; w < kBlock / 32; ++w) tot += s_red[w];
                J.partials[size_t(r) * J.tiles + t] = tot;
                __threadfence();
                const unsigned prev = atomicAdd(J.done, 1u);
                s_last = (prev == unsigned(J.R * J.tiles - 1));
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                finalize_job(J, s_L);
                __syncthreads();
            }
        }
    }
    if (kCount) {
        const unsigned v[kNumCounters] = {warp_sum_u(cnt.sph), warp_sum_u(cnt.quad), warp_sum_u(cnt.box),
                                          warp_sum_u(cnt.paths), warp_sum_u(cnt.vertices), warp_sum_u(cnt.shadow),
                                          warp_sum_u(cnt.rays), 0u};
        if (lane == 0)
            for (int i = 0; i < kNumCounters; ++i) s_cnt[i][warp] = v[i];
        __syncthreads();
        if (tid < kNumCounters) {
            unsigned long long tot = 0;
            for (int w = 0; w < kBlock / 32; ++w) tot += s_cnt[tid][w];
            atomicAdd(L.counters + tid, tot);
        }
    }
}

// ---------------------------------------------------------------------------
// standalone Adam and raw Philox
// ---------------------------------------------------------------------------
__global__ void k_adam(int D, float* theta, float* m, float* v, const float* g, int t, float lr, float b1, float b2,
                       float eps) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    const double gd = g[d];
    const double mm = double(b1) * m[d] + (1.0 - double(b1)) * gd;
    const double vv = double(b2) * v[d] + (1.0 - double(b2)) * gd * gd;
    const double mh = mm / (1.0 - pow(double(b1), t));
    const double vh = vv / (1.0 - pow(double(b2), t));
    m[d] = float(mm);
    v[d] = float(vv);
    theta[d] = float(double(theta[d]) - double(lr) * mh / (sqrt(vh) + double(eps)));
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
cudaError_t launch_instantiate(const InstLaunch& L, cudaStream_t stream) {
    if (L.total_blocks <= 0) return cudaSuccess;
    k_instantiate<<<L.total_blocks, kInstBlock, 0, stream>>>(L);
    return cudaGetLastError();
}

int trace_blocks_per_sm(bool render_mode) {
    int n = 0;
    if (render_mode)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<true, false>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<false, false>, kBlock, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_trace(const TraceLaunch& L, bool render_mode, int grid, cudaStream_t stream) {
    if (L.total_items <= 0) return cudaSuccess;
    const bool count = L.counters != nullptr;
    if (render_mode && count)
        k_trace<true, true><<<grid, kBlock, 0, stream>>>(L);
    else if (render_mode)
        k_trace<true, false><<<grid, kBlock, 0, stream>>>(L);
    else if (count)
        k_trace<false, true><<<grid, kBlock, 0, stream>>>(L);
    else
        k_trace<false, false><<<grid, kBlock, 0, stream>>>(L);
    return cudaGetLastError();
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

}  // namespace prdpt
