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
// device current) and passed to the kernels like any other pointer. The call enqueues
// kernels and one memset only: the scene travels as a kernel parameter and is written
// into the array by the first kernel, so no host buffer has to outlive the call.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/prdpt.h"
#include "internal.h"
#include "scene_host.h"

using namespace prdpt;

namespace {

constexpr size_t kStaticScratchBytes = size_t(6) << 20;  // 6 MiB per device
constexpr int kStaticMaxPairs = 32;                      // 64 renders
constexpr int kMaxDevices = 64;
constexpr int kCtlWords = 16;                            // [0] queue, [1] done counter, [2] status, rest spare

// The shared scratch of every call on a device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_static_scratch
    int sms = 0, occ = 0;
};

// One lock per device: held from the set-up through the last launch of a call, so calls
// from several host threads enqueue one after another (their scratch use then follows
// the streams' order; calls on different, unordered streams still race on the GPU).
std::mutex g_mu[kMaxDevices];
DeviceSetup g_setup[kMaxDevices];

prdpt_status report(char* err, size_t err_len, prdpt_status code, const char* msg) {
    if (err && err_len > 0) std::snprintf(err, err_len, "%s", msg);
    return code;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static_assert(sizeof(BaseScene) % 4 == 0 && sizeof(BaseScene) + sizeof(void*) <= 4096,
              "the base scene must fit a kernel's parameter space");

// Writes the call's base scene (a kernel parameter: host data that needs no copy) into the
// scratch.
__global__ void __launch_bounds__(256) k_static_scene(const BaseScene B, BaseScene* dst) {
    const unsigned* src = reinterpret_cast<const unsigned*>(&B);
    unsigned* out = reinterpret_cast<unsigned*>(dst);
    for (int i = threadIdx.x; i < int(sizeof(BaseScene) / 4); i += blockDim.x) out[i] = src[i];
}

}  // namespace

extern "C" prdpt_status prdpt_smoothed_grad_static(const prdpt_scene_desc* scene, const prdpt_param_binding* binds,
                                                   int32_t D, const float* theta_dev, const float* sigma_dev,
                                                   const prdpt_grad_opts* o, const float* target_dev,
                                                   float* grad_dev, float* losses_dev, void* stream, char* err,
                                                   size_t err_len) {
    if (!scene || !binds || !o || !theta_dev || !sigma_dev || !target_dev || !grad_dev)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "NULL argument");
    if (o->pairs < 1 || o->pairs > kStaticMaxPairs)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "pairs must be in 1..32 for the allocation-free call");
    if (o->pair_begin < 0 || o->pair_begin > (1 << 26))
        return report(err, err_len, PRDPT_E_INVALID_ARG, "pair_begin must be in 0..2^26");
    if (o->sampler < 0 || o->sampler > 2) return report(err, err_len, PRDPT_E_INVALID_ARG, "unknown sampler");
    if (o->estimator != PRDPT_ESTIMATOR_KERNEL_GRADIENT)
        return report(err, err_len, PRDPT_E_INVALID_ARG,
                      "the allocation-free call takes estimator = PRDPT_ESTIMATOR_KERNEL_GRADIENT only");
    if (o->width < 1 || o->height < 1 || o->width > 8192 || o->height > 8192)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "width/height must be in 1..8192");
    if (o->spp < 1 || o->spp > 65535) return report(err, err_len, PRDPT_E_INVALID_ARG, "spp must be in 1..65535");
    if (o->depth < 1 || o->depth > 64) return report(err, err_len, PRDPT_E_INVALID_ARG, "depth must be in 1..64");
    if (o->rr_start < -1 || o->rr_start > 64)
        return report(err, err_len, PRDPT_E_INVALID_ARG, "rr_start must be -1 or 0..64");
    BaseScene B;
    if (const char* why = build_base_scene(scene, binds, D, false, &B))
        return report(err, err_len, PRDPT_E_INVALID_ARG, why);

    const int R = 2 * o->pairs;
    int px = o->block_pixels;
    if (px != 8 && px != 16 && px != 32) px = 32;
    int bw, bh;
    block_shape(px, &bw, &bh);
    const int tiles_x = (o->width + bw - 1) / bw;
    const int tiles = tiles_x * ((o->height + bh - 1) / bh);

    // layout of the static scratch
    const size_t off_base = 0;
    const size_t off_ctl = align256(off_base + sizeof(BaseScene));
    const size_t off_loss = align256(off_ctl + sizeof(unsigned) * kCtlWords);
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
    std::lock_guard<std::mutex> lk(g_mu[dev]);
    DeviceSetup& setup = g_setup[dev];
    if (!setup.ready) {  // once per device, with that device current
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));
        setup.scratch = static_cast<unsigned char*>(p);
        setup.sms = sms;
        setup.occ = trace_blocks_per_sm(false);
        setup.ready = true;
    }
    unsigned char* base = setup.scratch;
    BaseScene* d_base = reinterpret_cast<BaseScene*>(base + off_base);
    unsigned* ctl = reinterpret_cast<unsigned*>(base + off_ctl);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // The sampler kernel reads the base scene before it waits on the kernel ahead of it
    // (programmatic dependent launch); the memset between them makes it wait for the
    // scene write in plain stream order.
    k_static_scene<<<1, 256, 0, st>>>(B, d_base);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(unsigned) * kCtlWords, st);  // queue, done, status
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
    TL.status = reinterpret_cast<int*>(ctl + 2);  // written by the kernels, not reported by this call
    const int per_sm = (o->ctas_per_sm > 0 && o->ctas_per_sm < setup.occ) ? o->ctas_per_sm : setup.occ;
    const int cap = setup.sms * per_sm;
    const int want = (TL.total_items + kBlock / 32 - 1) / (kBlock / 32);
    e = launch_trace(TL, false, want < cap ? want : cap, st);
    if (e == cudaSuccess) e = launch_finalize(TL, R, st);
    if (e != cudaSuccess) return report(err, err_len, PRDPT_E_CUDA, cudaGetErrorString(e));
    return PRDPT_OK;
}
