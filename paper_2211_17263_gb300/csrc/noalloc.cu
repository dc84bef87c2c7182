// noalloc.cu -- prdpt_smoothed_grad_static: the plateau-reduced gradient for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned by
// another allocator (a framework's caching allocator, a fixed arena handed out by a
// serving runtime), code that must not grow its footprint after start-up, or callers
// that may not create a library context (prdpt_create allocates its control block).
// This entry point needs neither a context nor any allocation: every buffer the
// launch needs besides the caller's inputs and outputs lives in one file-scope
// __device__ array of fixed size, which every GPU that loads the library holds until
// the process exits.
//
// Host code never dereferences that array: its name in host code is only a stand-in.
// The device address is obtained once per device with cudaGetSymbolAddress (with that
// device current) and passed to the kernels like any other pointer.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/prdpt.h"
#include "internal.h"

using namespace prdpt;

namespace {

constexpr size_t kStaticScratchBytes = size_t(6) << 20;  // 6 MiB per device
constexpr int kStaticMaxRenders = 64;                    // at most 32 antithetic pairs
constexpr int kMaxDevices = 64;

// The shared scratch of every call on a device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_static_scratch
    int sms = 0, occ = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

prdpt_status report(char* err, size_t err_len, prdpt_status code, const char* msg) {
    if (err && err_len > 0) {
        std::snprintf(err, err_len, "%s", msg);
    }
    return code;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Scene validation and host-side precomputation, as for an uploaded scene.
bool build_base_scene(const prdpt_scene_desc* sd, const prdpt_param_binding* binds, int D, BaseScene* B,
                      const char** why) {
    *why = nullptr;
    if (sd->n_prims < 1 || sd->n_prims > kMaxPrims) return *why = "n_prims must be in 1..32", false;
    if (sd->n_mats < 1 || sd->n_mats > kMaxMats) return *why = "n_mats must be in 1..32", false;
    if (D < 1 || D > kMaxD) return *why = "D must be in 1..64", false;
    if (!sd->prim_type || !sd->prim_mat || !sd->prim_geom || !sd->mat_type || !sd->mat_param || !sd->camera ||
        !sd->background)
        return *why = "scene array is NULL", false;
    std::memset(B, 0, sizeof(*B));
    B->tex_mat = -1;  // no texture parameters in this entry point
    B->n_prims = sd->n_prims;
    B->n_mats = sd->n_mats;
    B->D = D;
    bool emission_bound[kMaxMats] = {};
    for (int i = 0; i < sd->n_mats; ++i) {
        if (sd->mat_type[i] < 0 || sd->mat_type[i] > 2) return *why = "bad material type", false;
        B->mat_type[i] = sd->mat_type[i];
        for (int q = 0; q < 8; ++q) B->mat_param[i][q] = sd->mat_param[8 * i + q];
    }
    for (int d = 0; d < D; ++d) {
        const int k = binds[d].kind, idx = binds[d].index, comp = binds[d].component;
        if (k == kBindPos || k == kBindRadius) {
            if (idx < 0 || idx >= sd->n_prims) return *why = "binding: primitive index out of range", false;
            if (k == kBindRadius && sd->prim_type[idx] != kSphere) return *why = "binding: radius of a non-sphere", false;
        } else if (k == kBindAlbedo || k == kBindEmission) {
            if (idx < 0 || idx >= sd->n_mats) return *why = "binding: material index out of range", false;
            if (k == kBindEmission) emission_bound[idx] = true;
        } else {
            return *why = "binding: unknown kind", false;
        }
        if (k != kBindRadius && (comp < 0 || comp > 2)) return *why = "binding: component must be 0..2", false;
        B->bind_kind[d] = k;
        B->bind_index[d] = idx;
        B->bind_comp[d] = (k == kBindRadius) ? 0 : comp;
    }
    int lights = 0;
    for (int i = 0; i < sd->n_prims; ++i) {
        const int t = sd->prim_type[i], m = sd->prim_mat[i];
        if (t < 0 || t > 2) return *why = "bad primitive type", false;
        if (m < 0 || m >= sd->n_mats) return *why = "primitive material out of range", false;
        const float* mp = &sd->mat_param[8 * m];
        const bool can_emit = mp[3] > 0.f || mp[4] > 0.f || mp[5] > 0.f || emission_bound[m];
        if (t == kBox && can_emit) return *why = "emissive boxes are not supported", false;
        lights += can_emit ? 1 : 0;
        B->prim_type[i] = t;
        B->prim_mat[i] = m;
        for (int q = 0; q < 9; ++q) B->prim_geom[i][q] = sd->prim_geom[9 * i + q];
        B->n_sph += (t == kSphere);
        B->n_quad += (t == kQuad);
        B->n_box += (t == kBox);
    }
    if (lights > kMaxLights) return *why = "more than 8 emitters", false;
    int next[3] = {0, B->n_sph, B->n_sph + B->n_quad};
    for (int i = 0; i < sd->n_prims; ++i) B->prim_slot[i] = next[B->prim_type[i]]++;
    double eye[3], look[3], up[3];
    for (int q = 0; q < 3; ++q) {
        eye[q] = sd->camera[q];
        look[q] = sd->camera[3 + q];
        up[q] = sd->camera[6 + q];
    }
    double f[3] = {look[0] - eye[0], look[1] - eye[1], look[2] - eye[2]};
    const double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fn > 0)) return *why = "camera eye equals look-at", false;
    for (double& x : f) x /= fn;
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rn > 0)) return *why = "camera up is parallel to the view direction", false;
    for (double& x : r) x /= rn;
    const double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    for (int q = 0; q < 3; ++q) {
        B->eye[q] = float(eye[q]);
        B->fwd[q] = float(f[q]);
        B->right[q] = float(r[q]);
        B->up[q] = float(u[q]);
        B->bg[q] = sd->background[q];
    }
    const double vfov = sd->camera[9];
    if (!(vfov > 0 && vfov < 180)) return *why = "field of view must be in (0, 180) degrees", false;
    B->tan_half = float(std::tan(0.5 * vfov * M_PI / 180.0));
    return true;
}

}  // namespace

extern "C" prdpt_status prdpt_smoothed_grad_static(const prdpt_scene_desc* scene, const prdpt_param_binding* binds,
                                                   int32_t D, const float* theta_dev, const float* sigma_dev,
                                                   const prdpt_grad_opts* o, const float* target_dev,
                                                   float* grad_dev, float* losses_dev, void* stream, char* err,
                                                   size_t err_len) {
    if (!scene || !binds || !o || !theta_dev || !sigma_dev || !target_dev || !grad_dev)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "NULL argument");
    if (o->pairs < 1 || 2 * o->pairs > kStaticMaxRenders)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "pairs must be in 1..32 for the allocation-free call");
    if (o->sampler < 0 || o->sampler > 2) return report(err, err_len, PRDPT_E_INVALID_ARG, "unknown sampler");
    if (o->estimator != PRDPT_ESTIMATOR_KERNEL_GRADIENT)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "the allocation-free call computes Eq. 10 only");
    if (o->width < 1 || o->height < 1 || o->width > 8192 || o->height > 8192)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "width/height must be in 1..8192");
    if (o->spp < 1 || o->spp > 65535) return report(err, err_len, PRDPT_E_INVALID_ARG, "spp must be in 1..65535");
    if (o->depth < 1 || o->depth > 64) return report(err, err_len, PRDPT_E_INVALID_ARG, "depth must be in 1..64");
    if (o->rr_start < -1 || o->rr_start > 64)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "rr_start must be -1 or 0..64");
    BaseScene B;
    const char* why = nullptr;
    if (!build_base_scene(scene, binds, D, &B, &why)) return report(err, err_len, PRDPT_E_INVALID_ARG, why);

    const int R = 2 * o->pairs;
    int px = o->block_pixels;
    if (px != 8 && px != 16 && px != 32) px = 32;
    int bw, bh;
    block_shape(px, &bw, &bh);
    const int tiles_x = (o->width + bw - 1) / bw;
    const int tiles = tiles_x * ((o->height + bh - 1) / bh);

    // layout of the static scratch
    const size_t off_base = 0;
    const size_t off_ctl = align256(off_base + sizeof(BaseScene));  // [0] queue, [1] done, [2] status
    const size_t off_rdone = align256(off_ctl + 64);
    const size_t off_loss = align256(off_rdone + sizeof(unsigned) * R);
    const size_t off_w = align256(off_loss + sizeof(double) * R);
    const size_t off_scn = align256(off_w + sizeof(float) * R * D);
    const size_t off_part = align256(off_scn + sizeof(InstScene) * R);
    const size_t need = off_part + sizeof(double) * size_t(R) * size_t(tiles);
    if (need > kStaticScratchBytes) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "needs %zu bytes of scratch, the allocation-free call has %zu", need,
                      kStaticScratchBytes);
        return report(err, err_len, PRDPT_E_OUT_OF_BUDGET, msg);
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report(err, err_len, PRDPT_E_CUDA, "cudaGetDevice failed");
    DeviceSetup setup;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        DeviceSetup& s = g_setup[dev];
        if (!s.ready) {  // once per device, with that device current
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));
            s.scratch = static_cast<unsigned char*>(p);
            s.sms = sms;
            s.occ = trace_blocks_per_sm(false);
            s.ready = true;
        }
        setup = s;
    }
    unsigned char* base = setup.scratch;
    BaseScene* d_base = reinterpret_cast<BaseScene*>(base + off_base);
    unsigned* ctl = reinterpret_cast<unsigned*>(base + off_ctl);
    unsigned* rdone = reinterpret_cast<unsigned*>(base + off_rdone);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    cudaError_t e = cudaMemcpyAsync(d_base, &B, sizeof(BaseScene), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, 64, st);  // queue, done counter, status start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(rdone, 0, sizeof(unsigned) * R, st);
    if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));

    InstLaunch IL{};
    InstJob& I = IL.job0;
    I.base = d_base;
    I.scenes = reinterpret_cast<InstScene*>(base + off_scn);
    I.theta = theta_dev;
    I.sigma = sigma_dev;
    I.w_out = reinterpret_cast<float*>(base + off_w);
    I.seed = o->seed;
    I.step = o->step;
    I.tag = kTagPath;
    I.R = R;
    I.D = D;
    I.W = o->width;
    I.H = o->height;
    I.sampler = o->sampler;
    I.antithetic = o->antithetic ? 1 : 0;
    I.crn = o->crn ? 1 : 0;
    I.pair_begin = o->pair_begin;
    I.c_radial = float(std::sqrt(2.0) * std::exp(std::lgamma(0.5 * (D + 1)) - std::lgamma(0.5 * D)));
    IL.total_blocks = R;
    IL.queue_reset = ctl + 0;
    e = launch_instantiate(IL, st);
    if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));

    TraceLaunch TL{};
    TraceJob& J = TL.job0;
    J.scenes = I.scenes;
    J.target = reinterpret_cast<const float4*>(target_dev);
    J.partials = reinterpret_cast<double*>(base + off_part);
    J.done = ctl + 1;
    J.losses = reinterpret_cast<double*>(base + off_loss);
    J.w = I.w_out;
    J.grad_out = grad_dev;
    J.loss_out = losses_dev;
    J.W = o->width;
    J.H = o->height;
    J.spp = o->spp;
    J.depth = o->depth;
    J.rr_start = o->rr_start;
    J.R = R;
    J.D = D;
    J.antithetic = I.antithetic;
    J.bw = bw;
    J.bh = bh;
    J.tiles_x = tiles_x;
    J.tiles = tiles;
    J.n_prims = B.n_prims;
    J.n_mats = B.n_mats;
    TL.total_items = R * tiles;
    TL.queue = ctl + 0;
    TL.status = reinterpret_cast<int*>(ctl + 2);
    const int per_sm = (o->ctas_per_sm > 0 && o->ctas_per_sm < setup.occ) ? o->ctas_per_sm : setup.occ;
    const int cap = setup.sms * per_sm;
    const int want = (TL.total_items + kBlock / 32 - 1) / (kBlock / 32);
    e = launch_trace(TL, false, want < cap ? want : cap, st);
    if (e == cudaSuccess) e = launch_finalize(TL, R, st);
    if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));
    return PRDPT_OK;
}
