/*
 * prdpt_oracle.c -- plain FP64 CPU oracle of the plateau-reduced gradient
 * estimator (Fischer & Ritschel, "Plateau-reduced Differentiable Path Tracing").
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The CUDA product path never calls
 * it and shares no code, header, table or helper with it; the two consume only
 * the seeded scene data of the `workloads` package.
 *
 * Everything is written for a reader checking it against the paper by eye:
 * no blocking, no fusion, double precision throughout, one function per step.
 *
 *   Philox4x32-10 ............ Salmon, Moraes, Dror, Shaw (SC'11), "Parallel random
 *                              numbers: as easy as 1, 2, 3" -- the uniform(0,1)
 *                              draws of Algorithm 1.
 *   perturbation sampler ..... Sec. 3.2 (variance reduction): importance sampling of
 *                              the positivized kernel gradient |d kappa/d theta|
 *                              (Eq. 11), inverse CDF (supplemental derivation),
 *                              antithetic pairs; the D>1 reading is radial (see
 *                              orc_sample_unit).
 *   forward model P(theta) ... Eq. 1 / Eq. 3: a Monte-Carlo path tracer.
 *   loss ..................... image MSE (Sec. 4.1, metrics).
 *   gradient ................. Eq. 10 with the antithetic pairing of Algorithm 1.
 *   Adam ..................... the optimiser of Sec. 3.4 (Kingma & Ba 2015).
 *
 * Parity pins: Philox against curand's host generator and published known
 * answers; sampler against its closed-form distribution; estimator against
 * closed-form smoothed gradients; tracer against the white furnace and analytic
 * irradiance; the smooth dielectric against the textbook Fresnel equations and
 * Snell's law; Russian roulette against the furnace mean and the unrouletted image;
 * Adam against torch.optim.Adam. All pins live in tests/.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_MAX_PRIMS 64
#define ORC_MAX_MATS 64
#define ORC_MAX_LIGHTS 16
#define ORC_MAX_D 64
#define ORC_EPS 1e-4 /* ray t_min and surface offset, in scene units */

/* random-stream tags (high nibble of counter word 3) */
#define TAG_PERTURB 1u
#define TAG_PATH 2u
#define TAG_TARGET 3u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011).                                       */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key increments */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Open-interval uniform: the top 23 bits of a word, as the odd multiple
 * (2k+1)/2^24. Never 0, never 1, never exactly 1/2. */
double orc_u01(uint32_t x) { return (double)((x >> 9) * 2u + 1u) * (1.0 / 16777216.0); }

/* Four uniforms of one Philox block. */
static void uniforms4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double u[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(w[i]);
}

/* Bulk Philox words for the known-answer and bit-exactness tests. */
void orc_philox_fill(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t c0_base, int n, uint32_t* out) {
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    for (int i = 0; i < n; ++i) {
        uint32_t ctr[4] = {c0_base + (uint32_t)i, c1, c2, c3};
        orc_philox4x32_10(ctr, key, out + 4 * i);
    }
}

/* ------------------------------------------------------------------------ */
/* Perturbation sampler (Sec. 3.2; Eq. 11; supplemental ICDF derivation).    */
/* ------------------------------------------------------------------------ */
/* Number of uniforms one unit-bandwidth draw consumes. */
int orc_sampler_uniforms(int mode, int D) {
    if (mode == 0) { /* radial */
        if (D == 1) return 2;
        int n_exp = (D + 1) / 2;
        int extra = (D % 2 == 0) ? 1 : 0;
        return n_exp + 2 * ((D + extra + 1) / 2);
    }
    if (mode == 1) return D;               /* per-dimension */
    return 2 * ((D + 1) / 2);              /* Gaussian (no importance sampling) */
}

/* sqrt(2) * Gamma((D+1)/2) / Gamma(D/2): the mean norm of a D-dim standard normal,
 * i.e. the normaliser of q(tau) ~ |tau| kappa(tau) for unit sigma. */
double orc_radial_constant(int D) { return sqrt(2.0) * exp(lgamma(0.5 * (D + 1)) - lgamma(0.5 * D)); }

/*
 * One unit-bandwidth draw tau~ and its estimator weight w~ from uniforms u[].
 * The weight is d kappa / q, so the smoothed gradient is E_q[w L(theta+tau)]
 * (with sigma: tau = sigma*tau~, w = w~/sigma, per dimension).
 *
 * mode 0 (radial): q(tau) proportional to |grad kappa(tau)| = |tau| kappa(tau)/sigma^2,
 *   the positivized gradient of Eq. 11 taken as a vector norm. Its radius is
 *   chi-distributed with D+1 degrees of freedom and its direction is uniform;
 *   w = c_D * direction with c_D = E|tau~|. For D=1 this is exactly the paper's
 *   1-D sampler: radius sqrt(-2 log xi) (Algorithm 1), a random sign, weight
 *   sqrt(2/pi) (the half-space normalisation of the supplemental).
 * mode 1 (per-dimension): each dimension independently from the two-sided
 *   1-D density |tau| exp(-tau^2/2)/2 by its inverse CDF (supplemental, with the
 *   signs corrected so the CDF is increasing), weight sign * sqrt(2/pi).
 * mode 2 (Gaussian, the "noIS" ablation): tau~ standard normal, w~ = tau~.
 */
void orc_sample_unit(int mode, int D, const double* u, double* tau, double* w) {
    if (mode == 0) {
        double c = orc_radial_constant(D);
        if (D == 1) {
            double r = sqrt(-2.0 * log(u[0]));
            double s = (u[1] < 0.5) ? -1.0 : 1.0;
            tau[0] = s * r;
            w[0] = s * c;
            return;
        }
        int n_exp = (D + 1) / 2;
        int extra = (D % 2 == 0) ? 1 : 0;
        double r2 = 0.0;
        for (int j = 0; j < n_exp; ++j) r2 += -2.0 * log(u[j]); /* chi^2 with 2 dof each */
        int nz = D + extra;
        double* z = (double*)malloc(sizeof(double) * (size_t)(nz + 1));
        for (int m = 0; 2 * m < nz; ++m) { /* Box-Muller pairs */
            double a = u[n_exp + 2 * m], b = u[n_exp + 2 * m + 1];
            double rad = sqrt(-2.0 * log(a));
            z[2 * m] = rad * cos(2.0 * M_PI * b);
            z[2 * m + 1] = rad * sin(2.0 * M_PI * b);
        }
        if (extra) r2 += z[D] * z[D]; /* one more degree of freedom when D+1 is odd */
        double zn = 0.0;
        for (int d = 0; d < D; ++d) zn += z[d] * z[d];
        zn = sqrt(zn);
        double r = sqrt(r2);
        for (int d = 0; d < D; ++d) {
            double dir = z[d] / zn;
            tau[d] = r * dir;
            w[d] = c * dir;
        }
        free(z);
        return;
    }
    if (mode == 1) {
        double c = sqrt(2.0 / M_PI);
        for (int d = 0; d < D; ++d) {
            double xi = u[d];
            if (xi < 0.5) {
                tau[d] = -sqrt(-2.0 * log(2.0 * xi));
                w[d] = -c;
            } else {
                tau[d] = sqrt(-2.0 * log(2.0 * (1.0 - xi)));
                w[d] = c;
            }
        }
        return;
    }
    for (int m = 0; 2 * m < D; ++m) {
        double a = u[2 * m], b = u[2 * m + 1];
        double rad = sqrt(-2.0 * log(a));
        double z0 = rad * cos(2.0 * M_PI * b), z1 = rad * sin(2.0 * M_PI * b);
        tau[2 * m] = z0;
        w[2 * m] = z0;
        if (2 * m + 1 < D) {
            tau[2 * m + 1] = z1;
            w[2 * m + 1] = z1;
        }
    }
}

/* Draw number `index` of step `step`: uniforms from stream PERTURB, counter
 * (index, block, step, tag), then scale by sigma. tau is returned both in FP64
 * and rounded to FP32 (the value the renderer is given). */
void orc_sample(int mode, int D, const float* sigma, uint64_t seed, uint32_t step, uint32_t index,
                double* tau, float* tau_f32, double* w) {
    int nu = orc_sampler_uniforms(mode, D);
    double* u = (double*)malloc(sizeof(double) * (size_t)(4 * (nu / 4 + 1)));
    double* tt = (double*)malloc(sizeof(double) * (size_t)D * 2);
    double* wt = tt + D;
    for (int k = 0; 4 * k < nu; ++k) uniforms4(seed, index, (uint32_t)k, step, TAG_PERTURB << 28, u + 4 * k);
    orc_sample_unit(mode, D, u, tt, wt);
    for (int d = 0; d < D; ++d) {
        tau[d] = (double)sigma[d] * tt[d];
        tau_f32[d] = (float)tau[d];
        w[d] = wt[d] / (double)sigma[d];
    }
    free(u);
    free(tt);
}

/* ------------------------------------------------------------------------ */
/* Scene description and instantiation at parameters theta.                  */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;
static v3 V(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 mul(v3 a, double s) { return V(a.x * s, a.y * s, a.z * s); }
static v3 hmul(v3 a, v3 b) { return V(a.x * b.x, a.y * b.y, a.z * b.z); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) { return V(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static v3 normalize(v3 a) { return mul(a, 1.0 / sqrt(dot(a, a))); }
static double comp(v3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static double maxc(v3 a) { return fmax(a.x, fmax(a.y, a.z)); }

enum { P_SPHERE = 0, P_QUAD = 1, P_BOX = 2 };
enum { M_DIFFUSE = 0, M_MIRROR = 1, M_DIELECTRIC = 2 };

typedef struct {
    int type, mat;
    v3 c;        /* centre */
    double r;    /* sphere radius */
    v3 u, v;     /* quad edges */
    v3 h;        /* box half size */
} orc_prim;

typedef struct {
    int type;
    v3 albedo, emission;
    double ior;
} orc_mat;

typedef struct {
    int n_prims, n_mats, n_lights;
    orc_prim prim[ORC_MAX_PRIMS];
    orc_mat mat[ORC_MAX_MATS];
    int light[ORC_MAX_LIGHTS];
    v3 eye, look, up;
    double vfov_deg;
    v3 background;
    /* texture: the albedo of material tex_mat on quads is looked up in tex, tex_res x
     * tex_res texels of RGB (row-major [t][s][3], texel (0,0) at the quad corner
     * c - u/2 - v/2), clamped to [0,1] at lookup; tex_mat = -1: none */
    int tex_mat, tex_res;
    const float* tex;
} orc_scene;

/* Flat scene arrays exactly as the workloads package lays them out. */
typedef struct {
    int n_prims, n_mats;
    const int32_t* prim_type;
    const int32_t* prim_mat;
    const float* prim_geom;  /* [n_prims][9] */
    const int32_t* mat_type;
    const float* mat_param;  /* [n_mats][8] */
    const float* camera;     /* [10] */
    const float* background; /* [3] */
} orc_scene_arrays;

static int is_emissive(const orc_mat* m) { return m->emission.x > 0 || m->emission.y > 0 || m->emission.z > 0; }

/* Build the scene at parameters theta (FP32 values, as the renderer receives them).
 * A binding (kind, index, component) sets one field to theta_d: 0 primitive centre,
 * 1 sphere radius, 2 material albedo (clamped to [0,1]), 3 material emission
 * (clamped to >= 0). Returns 0 on success. */
int orc_instantiate(const orc_scene_arrays* a, const int32_t* binds, int D, const float* theta, orc_scene* s) {
    int texture = D > 0 && binds && binds[0] == 4;
    if (a->n_prims > ORC_MAX_PRIMS || a->n_mats > ORC_MAX_MATS || (!texture && D > ORC_MAX_D)) return 1;
    memset(s, 0, sizeof(*s));
    s->tex_mat = -1;
    s->n_prims = a->n_prims;
    s->n_mats = a->n_mats;
    for (int i = 0; i < a->n_prims; ++i) {
        const float* g = a->prim_geom + 9 * i;
        orc_prim* p = &s->prim[i];
        p->type = a->prim_type[i];
        p->mat = a->prim_mat[i];
        p->c = V(g[0], g[1], g[2]);
        if (p->type == P_SPHERE) p->r = g[3];
        if (p->type == P_QUAD) { p->u = V(g[3], g[4], g[5]); p->v = V(g[6], g[7], g[8]); }
        if (p->type == P_BOX) p->h = V(g[3], g[4], g[5]);
    }
    for (int i = 0; i < a->n_mats; ++i) {
        const float* q = a->mat_param + 8 * i;
        s->mat[i].type = a->mat_type[i];
        s->mat[i].albedo = V(q[0], q[1], q[2]);
        s->mat[i].emission = V(q[3], q[4], q[5]);
        s->mat[i].ior = q[6];
    }
    if (texture) { /* kind 4: one binding row (4, material, resolution) for all 3 res^2 parameters */
        int idx = binds[1], res = binds[2];
        if (idx < 0 || idx >= s->n_mats || res < 1 || D != 3 * res * res) return 2;
        s->tex_mat = idx;
        s->tex_res = res;
        s->tex = theta;
        D = 0;
    }
    for (int d = 0; d < D; ++d) {
        int kind = binds[3 * d], idx = binds[3 * d + 1], c = binds[3 * d + 2];
        double t = (double)theta[d];
        if (kind == 0) {
            if (idx < 0 || idx >= s->n_prims || c < 0 || c > 2) return 2;
            if (c == 0) s->prim[idx].c.x = t;
            if (c == 1) s->prim[idx].c.y = t;
            if (c == 2) s->prim[idx].c.z = t;
        } else if (kind == 1) {
            if (idx < 0 || idx >= s->n_prims || s->prim[idx].type != P_SPHERE) return 2;
            s->prim[idx].r = fabs(t);
        } else if (kind == 2 || kind == 3) {
            if (idx < 0 || idx >= s->n_mats || c < 0 || c > 2) return 2;
            v3* f = (kind == 2) ? &s->mat[idx].albedo : &s->mat[idx].emission;
            if (c == 0) f->x = t;
            if (c == 1) f->y = t;
            if (c == 2) f->z = t;
        } else {
            return 2;
        }
    }
    for (int i = 0; i < s->n_mats; ++i) { /* albedo in [0,1], emission >= 0 */
        v3* al = &s->mat[i].albedo;
        al->x = fmin(fmax(al->x, 0.0), 1.0);
        al->y = fmin(fmax(al->y, 0.0), 1.0);
        al->z = fmin(fmax(al->z, 0.0), 1.0);
        v3* em = &s->mat[i].emission;
        em->x = fmax(em->x, 0.0);
        em->y = fmax(em->y, 0.0);
        em->z = fmax(em->z, 0.0);
    }
    s->n_lights = 0;
    for (int i = 0; i < s->n_prims; ++i) {
        if (!is_emissive(&s->mat[s->prim[i].mat])) continue;
        if (s->prim[i].type == P_BOX) return 3; /* emissive boxes are not supported */
        if (s->n_lights == ORC_MAX_LIGHTS) return 3;
        s->light[s->n_lights++] = i;
    }
    s->eye = V(a->camera[0], a->camera[1], a->camera[2]);
    s->look = V(a->camera[3], a->camera[4], a->camera[5]);
    s->up = V(a->camera[6], a->camera[7], a->camera[8]);
    s->vfov_deg = a->camera[9];
    s->background = V(a->background[0], a->background[1], a->background[2]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ray-primitive intersection (textbook geometry, FP64).                     */
/* Each returns the nearest t > ORC_EPS, or INFINITY, and the outward        */
/* geometric normal at the hit.                                              */
/* ------------------------------------------------------------------------ */
static double hit_sphere(const orc_prim* p, v3 o, v3 d, v3* n) {
    v3 oc = sub(o, p->c);
    double b = dot(oc, d);
    v3 l = sub(oc, mul(d, b));           /* offset of the centre from the ray line */
    double disc = p->r * p->r - dot(l, l);
    if (disc < 0.0) return INFINITY;
    double sq = sqrt(disc);
    double t = -b - sq;
    if (t <= ORC_EPS) t = -b + sq;
    if (t <= ORC_EPS) return INFINITY;
    *n = mul(sub(add(o, mul(d, t)), p->c), 1.0 / p->r);
    return t;
}

static double hit_quad(const orc_prim* p, v3 o, v3 d, v3* n) {
    v3 nn = normalize(cross(p->u, p->v));
    double den = dot(nn, d);
    if (fabs(den) < 1e-12) return INFINITY;
    double t = dot(nn, sub(p->c, o)) / den;
    if (t <= ORC_EPS) return INFINITY;
    v3 q = sub(add(o, mul(d, t)), p->c);
    double a = dot(q, p->u) / dot(p->u, p->u);
    double b = dot(q, p->v) / dot(p->v, p->v);
    if (fabs(a) > 0.5 || fabs(b) > 0.5) return INFINITY;
    *n = nn;
    return t;
}

static double hit_box(const orc_prim* p, v3 o, v3 d, v3* n) {
    double tn = -INFINITY, tf = INFINITY;
    int an = -1, af = -1;
    for (int i = 0; i < 3; ++i) {
        double oi = comp(o, i), di = comp(d, i);
        double lo = comp(p->c, i) - comp(p->h, i), hi = comp(p->c, i) + comp(p->h, i);
        if (di == 0.0) {
            if (oi < lo || oi > hi) return INFINITY;
            continue;
        }
        double t0 = (lo - oi) / di, t1 = (hi - oi) / di;
        if (t0 > t1) { double tmp = t0; t0 = t1; t1 = tmp; }
        if (t0 > tn) { tn = t0; an = i; }
        if (t1 < tf) { tf = t1; af = i; }
    }
    if (tn > tf) return INFINITY;
    double t;
    int axis;
    double sgn;
    if (tn > ORC_EPS) {
        t = tn; axis = an; sgn = -1.0;  /* entering: normal opposes the ray */
    } else if (tf > ORC_EPS) {
        t = tf; axis = af; sgn = 1.0;   /* leaving from inside */
    } else {
        return INFINITY;
    }
    double dc = comp(d, axis);
    double s = (dc > 0.0 ? 1.0 : -1.0) * sgn;
    *n = V(axis == 0 ? s : 0.0, axis == 1 ? s : 0.0, axis == 2 ? s : 0.0);
    return t;
}

static double hit_prim(const orc_prim* p, v3 o, v3 d, v3* n) {
    if (p->type == P_SPHERE) return hit_sphere(p, o, d, n);
    if (p->type == P_QUAD) return hit_quad(p, o, d, n);
    return hit_box(p, o, d, n);
}

/* Closest hit over all primitives in index order (brute force). */
static int closest_hit(const orc_scene* s, v3 o, v3 d, double* t_out, v3* n_out) {
    int best = -1;
    double bt = INFINITY;
    v3 bn = V(0, 0, 0);
    for (int i = 0; i < s->n_prims; ++i) {
        v3 n;
        double t = hit_prim(&s->prim[i], o, d, &n);
        if (t < bt) { bt = t; best = i; bn = n; }
    }
    *t_out = bt;
    *n_out = bn;
    return best;
}

/* Shadow ray: is anything except primitive `skip` hit closer than dist? */
static int occluded(const orc_scene* s, v3 o, v3 d, double dist, int skip) {
    for (int i = 0; i < s->n_prims; ++i) {
        if (i == skip) continue;
        v3 n;
        if (hit_prim(&s->prim[i], o, d, &n) < dist) return 1;
    }
    return 0;
}

/* Test hook: one primitive, one ray. */
double orc_intersect(const orc_scene_arrays* a, int prim, const double* o, const double* d, double* n_out) {
    orc_scene s;
    if (orc_instantiate(a, NULL, 0, NULL, &s)) return NAN;
    v3 n = V(0, 0, 0);
    double t = hit_prim(&s.prim[prim], V(o[0], o[1], o[2]), V(d[0], d[1], d[2]), &n);
    n_out[0] = n.x; n_out[1] = n.y; n_out[2] = n.z;
    return t;
}

/* ------------------------------------------------------------------------ */
/* Path tracer: the Monte-Carlo pixel estimate of Eq. 3 for Eq. 1.           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int width, height, spp, depth, rr_start;
    uint64_t seed;
    uint32_t step, tag, render_field;
} orc_trace_opts;

/* Orthonormal basis around unit n (Duff et al. 2017). */
static void onb(v3 n, v3* t1, v3* t2) {
    double sgn = n.z >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sgn + n.z);
    double b = n.x * n.y * a;
    *t1 = V(1.0 + sgn * n.x * n.x * a, sgn * b, -sgn * n.x);
    *t2 = V(b, sgn + n.y * n.y * a, -n.y);
}

/* Uniforms for (pixel, sample, vertex, slot) of one render's path stream.
 * slot 0: light-point u1, u2, BSDF u1, u2
 * slot 1: light choice, Russian roulette, dielectric choice, unused
 * slot 2: pixel jitter x, y (vertex 0 only) */
static void path_uniforms(const orc_trace_opts* o, uint32_t pixel, int s, int b, int slot, double u[4]) {
    uint32_t c1 = (uint32_t)s | ((uint32_t)b << 16) | ((uint32_t)slot << 24);
    uint32_t c3 = (o->tag << 28) | (o->render_field & 0x0fffffffu);
    uniforms4(o->seed, pixel, c1, o->step, c3, u);
}

/* Fresnel reflectance of an unpolarised wave at a smooth dielectric interface (the
 * textbook Fresnel equations in their cosine form): ci = cos(incidence) > 0, eta =
 * n_incident / n_transmitted. Returns F = (r_s^2 + r_p^2) / 2 with the amplitude
 * ratios r_s, r_p and the cosine of the refraction angle ct; F = 1 (and r_s, r_p, ct
 * = 1, 1, 0) under total internal reflection, when Snell's law has no solution. */
static double fresnel_dielectric(double ci, double eta, double* rs_out, double* rp_out, double* ct_out) {
    double s2t = eta * eta * (1.0 - ci * ci); /* sin^2 of the refraction angle (Snell) */
    if (s2t >= 1.0) {
        *rs_out = 1.0;
        *rp_out = 1.0;
        *ct_out = 0.0;
        return 1.0;
    }
    double ct = sqrt(1.0 - s2t);
    double rs = (eta * ci - ct) / (eta * ci + ct);
    double rp = (ci - eta * ct) / (ci + eta * ct);
    *rs_out = rs;
    *rp_out = rp;
    *ct_out = ct;
    return 0.5 * (rs * rs + rp * rp);
}

/* Scattering at a smooth dielectric of index `ior` (outside index 1): the ray
 * direction dir meets a surface with outward geometric normal ng at point p. With
 * probability F (uniform u < F) the ray is reflected, otherwise refracted by Snell's
 * law; the new origin is offset by ORC_EPS to the side the new ray leaves into.
 * fr receives F and the amplitude ratios r_s, r_p. Returns 1 for a reflection, 0 for
 * a refraction. */
static int dielectric_event(v3 dir, v3 ng, double ior, double u, v3 p, v3* dir_out, v3* org_out, double fr[3]) {
    double ci = -dot(dir, ng);
    double eta;
    v3 n; /* normal on the incident side */
    if (ci > 0.0) { eta = 1.0 / ior; n = ng; }
    else { eta = ior; n = mul(ng, -1.0); ci = -ci; }
    double rs, rp, ct;
    double F = fresnel_dielectric(ci, eta, &rs, &rp, &ct);
    fr[0] = F;
    fr[1] = rs;
    fr[2] = rp;
    if (u < F) {
        *dir_out = normalize(add(dir, mul(n, 2.0 * ci)));
        *org_out = add(p, mul(n, ORC_EPS));
        return 1;
    }
    *dir_out = normalize(add(mul(dir, eta), mul(n, eta * ci - ct)));
    *org_out = sub(p, mul(n, ORC_EPS));
    return 0;
}

/* Test hook: the dielectric event of the tracer for one ray (dir unit, ng the outward
 * unit normal, p the hit point). Writes the new direction and origin, and F, r_s, r_p
 * of the incidence; returns 1 for a reflection. */
int orc_dielectric(const double* dir, const double* ng, double ior, double u, const double* p, double* dir_out,
                   double* org_out, double* fresnel_out) {
    v3 nd, no;
    int refl = dielectric_event(V(dir[0], dir[1], dir[2]), V(ng[0], ng[1], ng[2]), ior, u, V(p[0], p[1], p[2]), &nd,
                                &no, fresnel_out);
    dir_out[0] = nd.x; dir_out[1] = nd.y; dir_out[2] = nd.z;
    org_out[0] = no.x; org_out[1] = no.y; org_out[2] = no.z;
    return refl;
}

/* Forward-mode tangents of a path sample for Eq. 9's pathwise derivative dP/dtheta with
 * respect to n bound material parameters: kind 2 (albedo) or 3 (emission) of material
 * mat, colour channel c; dclamp is the derivative of the clamp applied at instantiation
 * (1 inside the valid range, 0 where the value was clamped). The discrete choices of the
 * path (light choice, Fresnel choice, Russian-roulette survival) are held fixed, and the
 * Russian-roulette probability is a constant of the derivative: dividing by it keeps the
 * derivative estimate unbiased, as it keeps the radiance estimate unbiased. */
typedef struct {
    int n;
    int kind[ORC_MAX_D], mat[ORC_MAX_D], c[ORC_MAX_D];
    double dclamp[ORC_MAX_D];
} orc_tangent_spec;

/* Albedo of a textured quad at hit point p: texel (floor(s T), floor(t T)) with
 * s = (p - c).u / |u|^2 + 1/2, t = (p - c).v / |v|^2 + 1/2, each clamped to [0, T-1];
 * channels clamped to [0,1]. */
static v3 tex_albedo(const orc_scene* sc, const orc_prim* pr, v3 p) {
    v3 l = sub(p, pr->c);
    double s = dot(l, pr->u) / dot(pr->u, pr->u) + 0.5, t = dot(l, pr->v) / dot(pr->v, pr->v) + 0.5;
    int T = sc->tex_res;
    int tx = (int)floor(s * T), ty = (int)floor(t * T);
    tx = tx < 0 ? 0 : (tx > T - 1 ? T - 1 : tx);
    ty = ty < 0 ? 0 : (ty > T - 1 ? T - 1 : ty);
    const float* q = sc->tex + ((size_t)ty * T + tx) * 3;
    return V(fmin(fmax(q[0], 0.0), 1.0), fmin(fmax(q[1], 0.0), 1.0), fmin(fmax(q[2], 0.0), 1.0));
}

/* beta <- beta * albedo (material mat): product rule on each tangent's channel. */
static void scatter_tangents(const orc_tangent_spec* ts, double* dB, v3 beta, v3 albedo, int mat) {
    if (!ts) return;
    for (int k = 0; k < ts->n; ++k) {
        int c = ts->c[k];
        double d = dB[k] * comp(albedo, c);
        if (ts->kind[k] == 2 && ts->mat[k] == mat) d += comp(beta, c) * ts->dclamp[k];
        dB[k] = d;
    }
}

/* Radiance of one path sample through pixel (x, y); with ts, also the derivative of
 * channel ts->c[k] of the radiance with respect to each parameter k, in dL[k]. */
static v3 trace_path_t(const orc_scene* sc, const orc_trace_opts* o, int x, int y, int s,
                       const orc_tangent_spec* ts, double* dL) {
    uint32_t pixel = (uint32_t)(y * o->width + x);
    double u[4];
    int nt = ts ? ts->n : 0;
    double dB[ORC_MAX_D]; /* d(beta channel c_k) / d theta_k */
    for (int k = 0; k < nt; ++k) { dB[k] = 0.0; dL[k] = 0.0; }

    /* pinhole camera, box-filtered jitter inside the pixel */
    v3 f = normalize(sub(sc->look, sc->eye));
    v3 r = normalize(cross(f, sc->up));
    v3 up = cross(r, f);
    double th = tan(0.5 * sc->vfov_deg * M_PI / 180.0);
    double aspect = (double)o->width / (double)o->height;
    path_uniforms(o, pixel, s, 0, 2, u);
    double sx = (2.0 * (x + u[0]) / o->width - 1.0) * aspect * th;
    double sy = (1.0 - 2.0 * (y + u[1]) / o->height) * th;
    v3 org = sc->eye;
    v3 dir = normalize(add(f, add(mul(r, sx), mul(up, sy))));

    v3 L = V(0, 0, 0), beta = V(1, 1, 1);
    int specular = 1; /* emission is counted on camera rays and after specular bounces */
    double u1[4];     /* slot 1 of the current vertex */
    for (int b = 0; b < o->depth; ++b) {
        double t;
        v3 ng;
        int hit = closest_hit(sc, org, dir, &t, &ng);
        if (hit < 0) {
            L = add(L, hmul(beta, sc->background));
            for (int k = 0; k < nt; ++k) dL[k] += dB[k] * comp(sc->background, ts->c[k]);
            break;
        }
        const orc_prim* pr = &sc->prim[hit];
        const orc_mat* m = &sc->mat[pr->mat];
        v3 p = add(org, mul(dir, t));
        v3 albedo = m->albedo;
        if (pr->mat == sc->tex_mat && pr->type == P_QUAD) albedo = tex_albedo(sc, pr, p);
        if (specular && is_emissive(m) && dot(dir, ng) < 0.0) {
            L = add(L, hmul(beta, m->emission));
            for (int k = 0; k < nt; ++k) {
                int c = ts->c[k];
                dL[k] += dB[k] * comp(m->emission, c);
                if (ts->kind[k] == 3 && ts->mat[k] == pr->mat) dL[k] += comp(beta, c) * ts->dclamp[k];
            }
        }
        int last = (b + 1 >= o->depth);
        path_uniforms(o, pixel, s, b, 0, u);
        path_uniforms(o, pixel, s, b, 1, u1);

        if (m->type == M_DIFFUSE) {
            v3 ns = dot(ng, dir) < 0.0 ? ng : mul(ng, -1.0);
            v3 po = add(p, mul(ns, ORC_EPS));
            if (sc->n_lights > 0) { /* next-event estimation: one light, uniform area sample */
                int li = (int)floor(u1[0] * sc->n_lights);
                if (li > sc->n_lights - 1) li = sc->n_lights - 1;
                const orc_prim* lp = &sc->prim[sc->light[li]];
                v3 y, ny;
                double area;
                if (lp->type == P_QUAD) {
                    y = add(lp->c, add(mul(lp->u, u[0] - 0.5), mul(lp->v, u[1] - 0.5)));
                    v3 cr = cross(lp->u, lp->v);
                    ny = normalize(cr);
                    area = sqrt(dot(cr, cr));
                } else {
                    double z = 1.0 - 2.0 * u[0];
                    double rr = sqrt(fmax(0.0, 1.0 - z * z));
                    double phi = 2.0 * M_PI * u[1];
                    ny = V(rr * cos(phi), rr * sin(phi), z);
                    y = add(lp->c, mul(ny, lp->r));
                    area = 4.0 * M_PI * lp->r * lp->r;
                }
                v3 dv = sub(y, po);
                double dist2 = dot(dv, dv);
                double dist = sqrt(dist2);
                v3 wi = mul(dv, 1.0 / dist);
                double cx = dot(ns, wi), cl = -dot(ny, wi);
                if (cx > 0.0 && cl > 0.0 && !occluded(sc, po, wi, dist, sc->light[li])) {
                    double g = cx * cl / dist2 * area * sc->n_lights / M_PI;
                    v3 le = sc->mat[lp->mat].emission;
                    L = add(L, mul(hmul(hmul(beta, albedo), le), g));
                    for (int k = 0; k < nt; ++k) { /* product rule on beta * albedo * Le */
                        int c = ts->c[k];
                        double bc = comp(beta, c), rc = comp(albedo, c), ec = comp(le, c);
                        double d = dB[k] * rc * ec;
                        if (ts->kind[k] == 2 && ts->mat[k] == pr->mat) d += bc * ts->dclamp[k] * ec;
                        if (ts->kind[k] == 3 && ts->mat[k] == lp->mat) d += bc * rc * ts->dclamp[k];
                        dL[k] += d * g;
                    }
                }
            }
            if (last) break;
            double rad = sqrt(u[2]), phi = 2.0 * M_PI * u[3];
            v3 t1, t2;
            onb(ns, &t1, &t2);
            v3 wo = add(add(mul(t1, rad * cos(phi)), mul(t2, rad * sin(phi))), mul(ns, sqrt(fmax(0.0, 1.0 - u[2]))));
            scatter_tangents(ts, dB, beta, albedo, pr->mat);
            beta = hmul(beta, albedo);
            org = po;
            dir = normalize(wo);
            specular = 0;
        } else if (m->type == M_MIRROR) {
            if (last) break;
            v3 ns = dot(ng, dir) < 0.0 ? ng : mul(ng, -1.0);
            dir = normalize(sub(dir, mul(ns, 2.0 * dot(dir, ns))));
            org = add(p, mul(ns, ORC_EPS));
            scatter_tangents(ts, dB, beta, albedo, pr->mat);
            beta = hmul(beta, albedo);
            specular = 1;
        } else { /* smooth dielectric: exact unpolarised Fresnel, reflect or refract */
            if (last) break;
            double fr[3];
            v3 nd, no;
            dielectric_event(dir, ng, m->ior, u1[2], p, &nd, &no, fr);
            dir = nd;
            org = no;
            scatter_tangents(ts, dB, beta, albedo, pr->mat);
            beta = hmul(beta, albedo);
            specular = 1;
        }
        if (maxc(beta) <= 0.0) break; /* nothing more can be added */
        if (o->rr_start >= 0 && b >= o->rr_start) { /* Russian roulette (slot 1, second uniform) */
            double q = fmin(0.95, maxc(beta));
            if (u1[1] >= q) break;
            beta = mul(beta, 1.0 / q);
            for (int k = 0; k < nt; ++k) dB[k] /= q;
        }
    }
    return L;
}

static v3 trace_path(const orc_scene* sc, const orc_trace_opts* o, int x, int y, int s) {
    return trace_path_t(sc, o, x, y, s, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Rendering many scenes (threads over image rows; results are independent  */
/* of the thread count).                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_scene* scenes;
    const orc_trace_opts* opts; /* one per scene */
    double* images;             /* [n][H][W][3] */
    int n, width, height;
    int next_row;
    pthread_mutex_t lock;
    const orc_tangent_spec* ts; /* one per scene, or NULL */
    double* dimages;            /* [n][H][W][ts->n] pixel-mean tangents, or NULL */
} render_job;

static void* render_worker(void* arg) {
    render_job* j = (render_job*)arg;
    for (;;) {
        pthread_mutex_lock(&j->lock);
        int row = j->next_row++;
        pthread_mutex_unlock(&j->lock);
        if (row >= j->n * j->height) break;
        int i = row / j->height, y = row % j->height;
        const orc_trace_opts* o = &j->opts[i];
        const orc_tangent_spec* ts = j->ts ? &j->ts[i] : NULL;
        int nt = ts ? ts->n : 0;
        for (int x = 0; x < j->width; ++x) {
            v3 acc = V(0, 0, 0);
            double dacc[ORC_MAX_D], dl[ORC_MAX_D];
            for (int k = 0; k < nt; ++k) dacc[k] = 0.0;
            for (int s = 0; s < o->spp; ++s) {
                acc = add(acc, trace_path_t(&j->scenes[i], o, x, y, s, ts, dl));
                for (int k = 0; k < nt; ++k) dacc[k] += dl[k];
            }
            acc = mul(acc, 1.0 / o->spp);
            size_t pix = ((size_t)i * j->height + y) * j->width + x;
            double* px = j->images + pix * 3;
            px[0] = acc.x; px[1] = acc.y; px[2] = acc.z;
            for (int k = 0; k < nt; ++k) j->dimages[pix * nt + k] = dacc[k] / o->spp;
        }
    }
    return NULL;
}

static int resolve_threads(int nthreads) {
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void render_scenes_t(const orc_scene* scenes, const orc_trace_opts* opts, int n, double* images,
                            const orc_tangent_spec* ts, double* dimages, int nthreads) {
    render_job j;
    j.scenes = scenes; j.opts = opts; j.images = images; j.n = n;
    j.ts = ts; j.dimages = dimages;
    j.width = opts[0].width; j.height = opts[0].height; j.next_row = 0;
    pthread_mutex_init(&j.lock, NULL);
    int nt = resolve_threads(nthreads);
    if (nt > 256) nt = 256;
    pthread_t th[256];
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, render_worker, &j);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j.lock);
}

static void render_scenes(const orc_scene* scenes, const orc_trace_opts* opts, int n, double* images, int nthreads) {
    render_scenes_t(scenes, opts, n, images, NULL, NULL, nthreads);
}

/* Render n scenes at parameter vectors thetas[n][D]; render i uses the path
 * stream field (crn ? 0 : i). images: [n][H][W][3] doubles. */
int orc_render(const orc_scene_arrays* a, const int32_t* binds, int D, const float* thetas, int n,
               int width, int height, int spp, int depth, int rr_start, uint64_t seed, uint32_t step,
               uint32_t tag, int crn, double* images, int nthreads) {
    orc_scene* sc = (orc_scene*)malloc(sizeof(orc_scene) * (size_t)n);
    orc_trace_opts* op = (orc_trace_opts*)malloc(sizeof(orc_trace_opts) * (size_t)n);
    if (!sc || !op) { free(sc); free(op); return 9; }
    for (int i = 0; i < n; ++i) {
        int rc = orc_instantiate(a, binds, D, thetas + (size_t)i * D, &sc[i]);
        if (rc) { free(sc); free(op); return rc; }
        orc_trace_opts o = {width, height, spp, depth, rr_start, seed, step, tag, crn ? 0u : (uint32_t)i};
        op[i] = o;
    }
    render_scenes(sc, op, n, images, nthreads);
    free(sc);
    free(op);
    return 0;
}

/* Render only selected pixels (for full-size spot checks). pix: [m] linear
 * indices y*W+x into render `ri` of the list; out: [m][3]. */
int orc_render_pixels(const orc_scene_arrays* a, const int32_t* binds, int D, const float* theta, int render_field,
                      int width, int height, int spp, int depth, int rr_start, uint64_t seed, uint32_t step,
                      uint32_t tag, const int32_t* pix, int m, double* out) {
    orc_scene sc;
    int rc = orc_instantiate(a, binds, D, theta, &sc);
    if (rc) return rc;
    orc_trace_opts o = {width, height, spp, depth, rr_start, seed, step, tag, (uint32_t)render_field};
    for (int k = 0; k < m; ++k) {
        int x = pix[k] % width, y = pix[k] / width;
        v3 acc = V(0, 0, 0);
        for (int s = 0; s < spp; ++s) acc = add(acc, trace_path(&sc, &o, x, y, s));
        acc = mul(acc, 1.0 / spp);
        out[3 * k] = acc.x; out[3 * k + 1] = acc.y; out[3 * k + 2] = acc.z;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Loss and the smoothed gradient (Eq. 10 with antithetic pairs).            */
/* ------------------------------------------------------------------------ */
/* Image MSE over RGB: (1/3HW) sum (I - T)^2; target is [H][W][4] (RGB + pad). */
double orc_mse(const double* image, const float* target, int width, int height) {
    double acc = 0.0;
    for (int i = 0; i < width * height; ++i)
        for (int c = 0; c < 3; ++c) {
            double e = image[3 * i + c] - (double)target[4 * i + c];
            acc += e * e;
        }
    return acc / (3.0 * width * height);
}

/*
 * Eq. 10 with the antithetic pairs of Algorithm 1, for any loss L(theta).
 * antithetic=1: P pairs; pair p draws (tau_p, w_p) with counter index p, evaluates
 *   theta+tau_p (evaluation 2p) and theta-tau_p (evaluation 2p+1), and
 *   g = (1/2P) sum_p w_p (L_2p - L_2p+1).
 * antithetic=0: R = 2P independent draws (counter index r), g = (1/R) sum_r w_r L_r.
 * pair_begin: the first pair of a shard of a larger estimate: draw indices and the
 *   render numbers handed to the loss are global (pair_begin + p, 2 pair_begin + r).
 * The perturbed parameters are FP32 sums theta + tau_f32 (what a renderer gets).
 * Outputs: grad[D], losses[2P], taus[2P][D] (FP32), weights[2P][D].
 */
typedef double (*orc_loss_cb)(const float* theta_r, int D, int r, void* user);

int orc_estimate(int mode, int antithetic, int D, const float* theta, const float* sigma, int pairs, int pair_begin,
                 uint64_t seed, uint32_t step, orc_loss_cb loss, void* user, double* grad, double* losses,
                 float* taus, double* weights) {
    int R = 2 * pairs;
    if (D < 1 || pairs < 1) return 1;
    double* tau = (double*)malloc(sizeof(double) * (size_t)D * 2);
    float* tf = (float*)malloc(sizeof(float) * (size_t)D * 2);
    if (!tau || !tf) { free(tau); free(tf); return 9; }
    double* w = tau + D;
    float* th = tf + D;
    for (int r = 0; r < R; ++r) {
        int anti = antithetic && (r % 2 == 1);
        uint32_t index = (antithetic ? (uint32_t)(r / 2) : (uint32_t)r) +
                         (uint32_t)(antithetic ? pair_begin : 2 * pair_begin);
        orc_sample(mode, D, sigma, seed, step, index, tau, tf, w);
        for (int d = 0; d < D; ++d) {
            float t = anti ? -tf[d] : tf[d];
            th[d] = theta[d] + t; /* FP32 sum */
            taus[(size_t)r * D + d] = t;
            weights[(size_t)r * D + d] = anti ? -w[d] : w[d];
        }
        losses[r] = loss(th, D, 2 * pair_begin + r, user);
        if (isnan(losses[r])) { free(tau); free(tf); return 4; }
    }
    free(tau);
    free(tf);
    for (int d = 0; d < D; ++d) {
        double g = 0.0;
        if (antithetic) {
            for (int p = 0; p < pairs; ++p) g += weights[(size_t)(2 * p) * D + d] * (losses[2 * p] - losses[2 * p + 1]);
            grad[d] = g / (2.0 * pairs);
        } else {
            for (int r = 0; r < R; ++r) g += weights[(size_t)r * D + d] * losses[r];
            grad[d] = g / R;
        }
    }
    return 0;
}

/* Loss of one perturbed render: instantiate, path-trace, image MSE. */
typedef struct {
    const orc_scene_arrays* a;
    const int32_t* binds;
    const float* target;
    int width, height, spp, depth, rr_start, crn, nthreads;
    uint64_t seed;
    uint32_t step;
    double* image; /* [H][W][3] scratch */
} render_loss_ctx;

static double render_loss(const float* theta_r, int D, int r, void* user) {
    render_loss_ctx* c = (render_loss_ctx*)user;
    orc_scene sc;
    if (orc_instantiate(c->a, c->binds, D, theta_r, &sc)) return NAN;
    orc_trace_opts o = {c->width, c->height, c->spp, c->depth, c->rr_start, c->seed, c->step, TAG_PATH,
                        c->crn ? 0u : (uint32_t)(r + 1)};
    render_scenes(&sc, &o, 1, c->image, c->nthreads);
    return orc_mse(c->image, c->target, c->width, c->height);
}

/* The plateau-reduced gradient of the image loss of a scene (path streams:
 * render r uses field (crn ? 0 : r + 1)). */
int orc_smoothed_grad(const orc_scene_arrays* a, const int32_t* binds, int D, const float* theta,
                      const float* sigma, int pairs, int pair_begin, int mode, int antithetic, int crn, int width,
                      int height, int spp, int depth, int rr_start, uint64_t seed, uint32_t step,
                      const float* target, double* grad, double* losses, float* taus, double* weights,
                      int nthreads) {
    render_loss_ctx c = {a, binds, target, width, height, spp, depth, rr_start, crn, nthreads, seed, step, NULL};
    c.image = (double*)malloc(sizeof(double) * (size_t)width * height * 3);
    if (!c.image) return 9;
    int rc = orc_estimate(mode, antithetic, D, theta, sigma, pairs, pair_begin, seed, step, render_loss, &c, grad,
                          losses, taus, weights);
    free(c.image);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* The kappa-dP estimator (Eq. 9) for albedo and emission parameters.       */
/* ------------------------------------------------------------------------ */
/* Tangent spec of all D bindings at parameters theta; every binding must be an albedo
 * or emission one. Returns 0 on success. */
static int tangent_spec(const int32_t* binds, int D, const float* theta, orc_tangent_spec* ts) {
    if (D < 1 || D > ORC_MAX_D) return 1;
    ts->n = D;
    for (int d = 0; d < D; ++d) {
        int kind = binds[3 * d], idx = binds[3 * d + 1], c = binds[3 * d + 2];
        if (kind != 2 && kind != 3) return 5;
        double t = (double)theta[d];
        ts->kind[d] = kind;
        ts->mat[d] = idx;
        ts->c[d] = c;
        ts->dclamp[d] = (kind == 2) ? ((t >= 0.0 && t <= 1.0) ? 1.0 : 0.0) : (t >= 0.0 ? 1.0 : 0.0);
    }
    return 0;
}

/* One render at theta (path stream field `render_field`) with its pathwise tangents:
 * image [H][W][3] pixel means and dimage [H][W][D], the derivative of the pixel mean's
 * channel c_d with respect to theta_d. */
int orc_render_tangent(const orc_scene_arrays* a, const int32_t* binds, int D, const float* theta, int render_field,
                       int width, int height, int spp, int depth, int rr_start, uint64_t seed, uint32_t step,
                       uint32_t tag, double* image, double* dimage, int nthreads) {
    orc_scene sc;
    orc_tangent_spec ts;
    int rc = orc_instantiate(a, binds, D, theta, &sc);
    if (rc) return rc;
    rc = tangent_spec(binds, D, theta, &ts);
    if (rc) return rc;
    orc_trace_opts o = {width, height, spp, depth, rr_start, seed, step, tag, (uint32_t)render_field};
    render_scenes_t(&sc, &o, 1, image, &ts, dimage, nthreads);
    return 0;
}

/* Gradient of the image loss (1/3HW) sum (I - T)^2 from a render and its tangents:
 * dL/dtheta_d = (2/3HW) sum_px (I_c - T_c) dI_c/dtheta_d with c = c_d. */
static void loss_gradient(const double* image, const double* dimage, const float* target, const int32_t* binds,
                          int D, int width, int height, double* g) {
    for (int d = 0; d < D; ++d) g[d] = 0.0;
    for (int i = 0; i < width * height; ++i)
        for (int d = 0; d < D; ++d) {
            int c = binds[3 * d + 2];
            g[d] += (image[3 * i + c] - (double)target[4 * i + c]) * dimage[(size_t)i * D + d];
        }
    for (int d = 0; d < D; ++d) g[d] *= 2.0 / (3.0 * width * height);
}

/*
 * Eq. 9 with the Gaussian kernel sampled exactly (tau ~ N(0, sigma^2), so the kernel
 * weight over the sampling density is 1): g = (1/R) sum_r dL/dtheta (theta + tau_r), the
 * mean over the R = 2P renders of each render's pathwise loss gradient. Draws and pairing
 * are those of the gauss sampler of orc_smoothed_grad (antithetic: tau_p, -tau_p); render
 * r uses path-stream field (crn ? 0 : r + 1). Outputs grad[D], losses[2P], taus[2P][D]
 * (FP32) and the per-render gradients rgrads[2P][D].
 */
int orc_kdp_grad(const orc_scene_arrays* a, const int32_t* binds, int D, const float* theta, const float* sigma,
                 int pairs, int pair_begin, int antithetic, int crn, int width, int height, int spp, int depth,
                 int rr_start,
                 uint64_t seed, uint32_t step, const float* target, double* grad, double* losses, float* taus,
                 double* rgrads, int nthreads) {
    const int mode = 2; /* Gaussian draws */
    int R = 2 * pairs;
    if (D < 1 || D > ORC_MAX_D || pairs < 1) return 1;
    double* image = (double*)malloc(sizeof(double) * (size_t)width * height * 3);
    double* dimage = (double*)malloc(sizeof(double) * (size_t)width * height * D);
    if (!image || !dimage) { free(image); free(dimage); return 9; }
    for (int d = 0; d < D; ++d) grad[d] = 0.0;
    int rc = 0;
    for (int r = 0; r < R && !rc; ++r) {
        double tau[ORC_MAX_D], w[ORC_MAX_D];
        float tf[ORC_MAX_D], th[ORC_MAX_D];
        int anti = antithetic && (r % 2 == 1);
        uint32_t index = (antithetic ? (uint32_t)(r / 2) : (uint32_t)r) +
                         (uint32_t)(antithetic ? pair_begin : 2 * pair_begin);
        orc_sample(mode, D, sigma, seed, step, index, tau, tf, w);
        for (int d = 0; d < D; ++d) {
            float t = anti ? -tf[d] : tf[d];
            th[d] = theta[d] + t; /* FP32 sum */
            taus[(size_t)r * D + d] = t;
        }
        rc = orc_render_tangent(a, binds, D, th, crn ? 0 : 2 * pair_begin + r + 1, width, height, spp, depth, rr_start,
                                seed, step,
                                TAG_PATH, image, dimage, nthreads);
        if (rc) break;
        losses[r] = orc_mse(image, target, width, height);
        loss_gradient(image, dimage, target, binds, D, width, height, rgrads + (size_t)r * D);
        for (int d = 0; d < D; ++d) grad[d] += rgrads[(size_t)r * D + d];
    }
    for (int d = 0; d < D; ++d) grad[d] /= R;
    free(image);
    free(dimage);
    return rc;
}

/* Batched unit-bandwidth draws from explicit uniforms u[n][nu] (quadrature pins). */
void orc_sample_unit_batch(int mode, int D, int n, const double* u, double* tau, double* w) {
    int nu = orc_sampler_uniforms(mode, D);
    for (int i = 0; i < n; ++i) orc_sample_unit(mode, D, u + (size_t)i * nu, tau + (size_t)i * D, w + (size_t)i * D);
}

/* ------------------------------------------------------------------------ */
/* Adam (Kingma & Ba 2015), PyTorch's defaults, one step t (1-based).        */
/* ------------------------------------------------------------------------ */
void orc_adam(int D, double* theta, double* m, double* v, const double* g, int t, double lr, double b1, double b2,
              double eps) {
    for (int d = 0; d < D; ++d) {
        m[d] = b1 * m[d] + (1.0 - b1) * g[d];
        v[d] = b2 * v[d] + (1.0 - b2) * g[d] * g[d];
        double mh = m[d] / (1.0 - pow(b1, t));
        double vh = v[d] / (1.0 - pow(b2, t));
        theta[d] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Bandwidth schedule (Sec. 3.3 with the supplemental's warm start): constant
 * sigma0 for the first half of the run, then linear decay to sigma_min at the
 * last step. */
double orc_sigma_schedule(double sigma0, double sigma_min, int t, int total) {
    int w = total / 2;
    if (t < w || total - w <= 0) return sigma0;
    double frac = (double)(t - w) / (double)(total - w);
    if (frac > 1.0) frac = 1.0;
    return sigma0 - frac * (sigma0 - sigma_min);
}
