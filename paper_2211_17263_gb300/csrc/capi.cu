// capi.cu -- host implementation of the C ABI declared in include/prdpt.h.
//
// Owns the context (device, HBM budget, scenes, resident jobs, scratch buffers for
// the stateless calls, descriptor arrays for packed launches) and turns each call
// into at most two kernel launches: k_instantiate (sampler + scene binding) and
// k_trace (persistent render with the fused loss / gradient / Adam epilogue).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/prdpt.h"
#include "internal.h"
#include "scene_host.h"

using namespace prdpt;

namespace {

thread_local std::string g_err = "no error";

prdpt_status fail(prdpt_status code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define PRDPT_CUDA(call)                                                                          \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(PRDPT_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

struct Scene {
    BaseScene host;
    BaseScene* dev = nullptr;
    int D = 0;
    int jobs = 0;
    cudaEvent_t use = nullptr;  // recorded after each stateless call that reads `dev`
    bool used = false;
    bool captured = false;      // read by work captured into a CUDA graph (no event to wait on)
};

struct Job {
    void* base = nullptr;  // the job's one device allocation
    BaseScene* scene_copy = nullptr;  // the job's own copy of its scene (in `base`)
    cudaEvent_t last = nullptr;       // recorded after each enqueue of the job's work
    bool used = false;
    bool captured = false;            // stepped inside a CUDA-graph capture: replays are not tracked
    int scene = -1;
    int D = 0, R = 0, tiles = 0, ctas_per_sm = 0;
    size_t bytes = 0;
    // device buffers
    float *theta = nullptr, *m = nullptr, *v = nullptr, *sigma0 = nullptr, *grad = nullptr, *losses = nullptr;
    float* w = nullptr;
    bool tex = false;              // texture scene: D > kMaxD parameters
    float* tex_all = nullptr;      // [R][D] per-render textures
    HdNorm* norms = nullptr;       // [R] radial-sampler norms
    unsigned long long* share = nullptr;
    unsigned long long* accaff = nullptr;
    void* afflist = nullptr;
    float4* varbox = nullptr;
    unsigned* cursor = nullptr;
    int* aff = nullptr;
    unsigned* flags = nullptr;     // path sharing: [R][(pixels + 31) / 32] corrected-pixel bits
    double *partials = nullptr, *losses_d = nullptr;
    unsigned* rdone = nullptr;
    int* step = nullptr;
    unsigned *done = nullptr, *queue = nullptr, *share_ctl = nullptr;
    InstScene* scenes = nullptr;
    float4* target = nullptr;
    InstJob inst{};
    TraceJob trace{};
};

}  // namespace

struct prdpt_ctx {
    int device = 0;
    int sms = 0;
    int occ_grad = 1, occ_render = 1, occ_diff = 1, occ_group = 1, occ_emit = 1;
    uint64_t budget = 0, used = 0;
    std::map<void*, size_t> allocs;
    std::vector<Scene*> scenes;
    std::vector<Job*> jobs;
    // control block: [0] status, [1..4] unused, then counters, queues
    int* status = nullptr;
    unsigned long long* counters = nullptr;
    bool counting = false;
    // scratch of the stateless calls (grown on demand)
    InstScene* s_scenes = nullptr;
    size_t s_scenes_n = 0;
    float* s_w = nullptr;
    size_t s_w_n = 0;
    float* s_host_io = nullptr;   // host-buffer calls: target, theta, sigma, m, v, grad, losses
    size_t s_host_io_n = 0;
    float* h_stage = nullptr;     // host-buffer calls: page-locked staging of the small vectors
    size_t h_stage_n = 0;
    double* s_partials = nullptr;
    size_t s_partials_n = 0;
    double* s_losses = nullptr;
    size_t s_losses_n = 0;
    unsigned* s_ctl = nullptr;    // [0] queue, [1] done counter, [2..3], [8], [9] batch queues, [4..7] sharing
                                  // counters, [8] third batch queue (16 words)
    unsigned long long* s_share = nullptr;  // path sharing: [tiles][96] shared radiance
    size_t s_share_n = 0;
    int* s_aff = nullptr;         // path sharing: list of blocks with affected paths
    size_t s_aff_n = 0;
    unsigned long long* s_accaff = nullptr;  // path sharing: [R][H*W][3] affected radiance (kept zero)
    size_t s_accaff_n = 0;
    unsigned char* s_afflist = nullptr;  // path sharing: recorded paths (masks, codes, radiance)
    size_t s_afflist_n = 0;
    float4* s_varbox = nullptr;   // path sharing: [R][kMaxVariant][2] per-render bounds
    size_t s_varbox_n = 0;
    unsigned* s_cursor = nullptr; // path sharing: [R] per-render cursors
    size_t s_cursor_n = 0;
    unsigned* s_flags = nullptr;  // path sharing: [R][(pixels + 31) / 32] corrected-pixel bits
    size_t s_flags_n = 0;
    float* s_tex = nullptr;       // texture scenes: [R][D] per-render textures
    size_t s_tex_n = 0;
    HdNorm* s_norms = nullptr;    // texture scenes: [draws] radial-sampler norms (counters kept zero)
    size_t s_norms_n = 0;
    double* s_gpart = nullptr;    // pathwise estimator: [R][tiles][D] gradient partials
    size_t s_gpart_n = 0;
    double* s_rgrads = nullptr;   // pathwise estimator: [R][kMaxDiff] per-render gradients
    size_t s_rgrads_n = 0;
    // packed launches
    std::vector<int> batch_ids;
    InstJob* d_inst = nullptr;
    TraceJob* d_trace = nullptr;
    size_t batch_cap = 0;
    int batch_blocks = 0;
    // the packed arrays hold the path-sharing jobs, then the render-group jobs, then the
    // per-render ones: jobs and work items of each kind (one render launch per kind)
    int batch_jobs[4] = {0, 0, 0, 0}, batch_items[4] = {0, 0, 0, 0};
    // optional CUDA-event timing of the render kernel, recorded on its launch stream
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
    // page-locked staging of the packed-step descriptors, two slots used in turn; each
    // slot's event marks the end of its last upload
    unsigned char* h_desc[2] = {nullptr, nullptr};
    size_t h_desc_n = 0;
    cudaEvent_t h_desc_ev[2] = {nullptr, nullptr};
    int desc_slot = 0;
    // Device memory of jobs and scenes: chunks reserved from the device (within the budget)
    // and carved into blocks first-fit. A released block returns to its chunk's free ranges
    // once the event recorded after its last use has completed. Reserving and returning
    // device memory can wait for the device, so after warm-up, admitting and releasing jobs
    // calls neither cudaMalloc nor cudaFree.
    struct Chunk {
        char* base;
        size_t bytes;
        std::map<size_t, size_t> free;  // offset -> length, coalesced
    };
    struct Block {
        int chunk;
        size_t off, len;
    };
    struct Pending {
        void* p;
        cudaEvent_t ready;  // null: idle already
    };
    std::vector<Chunk> chunks;
    std::map<void*, Block> blocks;       // blocks in use or pending
    std::vector<Pending> pending;        // released, last use possibly still in flight
    std::vector<cudaEvent_t> ev_pool;    // unrecorded events for jobs and scenes
    cudaStream_t io = nullptr;  // non-blocking stream of the synchronous uploads and reads
    // Page-locked zeros: device memory that must start at zero is cleared by copies from
    // here (copy engines), not by memset kernels, which would queue behind the persistent
    // render kernels that fill every SM, so that creating a job never waits for a step.
    unsigned char* h_zero = nullptr;
    std::mutex mu;
};

namespace {

prdpt_status dev_alloc(prdpt_ctx* c, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->budget && c->used + bytes > c->budget)
        return fail(PRDPT_E_OUT_OF_BUDGET, "allocation of " + std::to_string(bytes) + " bytes exceeds the HBM budget (" +
                                               std::to_string(c->used) + " of " + std::to_string(c->budget) + " used)");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();  // an out-of-memory result is not sticky: keep it from later launch checks
        return fail(PRDPT_E_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs[*p] = bytes;
    c->used += bytes;
    return PRDPT_OK;
}

// Free an allocation made by dev_alloc (other pointers are not the context's to free).
void dev_free(prdpt_ctx* c, void* p) {
    if (!p) return;
    auto it = c->allocs.find(p);
    if (it == c->allocs.end()) return;
    c->used -= it->second;
    c->allocs.erase(it);
    cudaFree(p);
}

constexpr size_t kZeroBytes = size_t(4) << 20;

// Clear `bytes` at dst on `st` with copies from the context's page-locked zeros.
cudaError_t zero_async(prdpt_ctx* c, void* dst, size_t bytes, cudaStream_t st) {
    if (!c->h_zero) {
        void* h = nullptr;
        cudaError_t e = cudaHostAlloc(&h, kZeroBytes, cudaHostAllocDefault);
        if (e != cudaSuccess) return e;
        std::memset(h, 0, kZeroBytes);
        c->h_zero = static_cast<unsigned char*>(h);
    }
    char* d = static_cast<char*>(dst);
    for (size_t off = 0; off < bytes; off += kZeroBytes) {
        const cudaError_t e = cudaMemcpyAsync(d + off, c->h_zero, std::min(kZeroBytes, bytes - off),
                                              cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
prdpt_status grow(prdpt_ctx* c, T** p, size_t* cap, size_t n) {
    if (*cap >= n) return PRDPT_OK;
    dev_free(c, *p);
    *p = nullptr;
    *cap = 0;
    prdpt_status st = dev_alloc(c, reinterpret_cast<void**>(p), n * sizeof(T));
    if (st) return st;
    *cap = n;
    return PRDPT_OK;
}

// Is `st` capturing a CUDA graph? An event recorded there marks nothing at replay time,
// so work enqueued during a capture is not tracked by events (conservatively true when
// the query itself fails).
bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Mark the end of a job's (or scene's) enqueued work on `st`.
cudaError_t mark_use(cudaEvent_t ev, bool* used, bool* captured, cudaStream_t st) {
    if (capturing(st)) {
        *captured = true;
        return cudaSuccess;
    }
    *used = true;
    return cudaEventRecord(ev, st);
}

cudaEvent_t take_event(prdpt_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

// Has the work before `e` completed? (A not-ready query leaves no error behind.)
bool event_done(cudaEvent_t e) {
    if (!e) return true;
    const cudaError_t q = cudaEventQuery(e);
    if (q == cudaErrorNotReady) {
        cudaGetLastError();
        return false;
    }
    return true;
}

constexpr size_t kChunkBytes = size_t(256) << 20;

// Return a block's range to its chunk, merging it with free neighbours.
void arena_free(prdpt_ctx* c, void* p) {
    auto it = c->blocks.find(p);
    if (it == c->blocks.end()) return;
    const prdpt_ctx::Block b = it->second;
    c->blocks.erase(it);
    auto& fr = c->chunks[b.chunk].free;
    size_t off = b.off, len = b.len;
    auto nx = fr.lower_bound(off);
    if (nx != fr.begin()) {
        auto pv = std::prev(nx);
        if (pv->first + pv->second == off) {
            off = pv->first;
            len += pv->second;
            fr.erase(pv);
        }
    }
    if (nx != fr.end() && off + len == nx->first) {
        len += nx->second;
        fr.erase(nx);
    }
    fr[off] = len;
}

// Free the released blocks whose last use has completed (all of them with `wait`).
void arena_collect(prdpt_ctx* c, bool wait) {
    std::vector<prdpt_ctx::Pending> keep;
    for (auto& q : c->pending) {
        if (wait && q.ready) cudaEventSynchronize(q.ready);
        if (event_done(q.ready)) {
            if (q.ready) c->ev_pool.push_back(q.ready);
            arena_free(c, q.p);
        } else {
            keep.push_back(q);
        }
    }
    c->pending.swap(keep);
}

// First fit over the chunks' free ranges.
void* arena_take(prdpt_ctx* c, size_t bytes) {
    for (int k = 0; k < (int)c->chunks.size(); ++k) {
        auto& fr = c->chunks[k].free;
        for (auto it = fr.begin(); it != fr.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rest = it->second - bytes;
            fr.erase(it);
            if (rest) fr[off + bytes] = rest;
            void* p = c->chunks[k].base + off;
            c->blocks[p] = {k, off, bytes};
            return p;
        }
    }
    return nullptr;
}

// Return the chunks that hold no block to the device (their slots stay, empty, so that the
// blocks' chunk indices keep their meaning).
bool arena_trim(prdpt_ctx* c) {
    bool any = false;
    for (auto& ch : c->chunks) {
        if (!ch.base || ch.free.size() != 1 || ch.free.begin()->first != 0 || ch.free.begin()->second != ch.bytes)
            continue;
        dev_free(c, ch.base);
        ch.base = nullptr;
        ch.bytes = 0;
        ch.free.clear();
        any = true;
    }
    return any;
}

// A job or scene block from the arena. A new chunk is reserved when no free range fits: 256
// MB while the budget leaves room for four, else exactly the request. If the budget or the
// device refuses, the blocks still in flight are waited for and the search repeated, and
// then the empty chunks are returned and an exact chunk is tried once more.
prdpt_status block_alloc(prdpt_ctx* c, void** p, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    arena_collect(c, false);
    if ((*p = arena_take(c, bytes))) return PRDPT_OK;
    const bool roomy = !c->budget || (c->budget > c->used && c->budget - c->used >= 4 * kChunkBytes);
    size_t chunk = roomy ? std::max(bytes, kChunkBytes) : bytes;
    void* base = nullptr;
    prdpt_status st = dev_alloc(c, &base, chunk);
    if (st != PRDPT_OK && !c->pending.empty()) {
        arena_collect(c, true);
        if ((*p = arena_take(c, bytes))) {
            g_err = "no error";
            return PRDPT_OK;
        }
        st = dev_alloc(c, &base, chunk);
    }
    if (st != PRDPT_OK && (arena_trim(c) || chunk != bytes)) {
        chunk = bytes;
        st = dev_alloc(c, &base, chunk);
    }
    if (st != PRDPT_OK) return st;
    g_err = "no error";
    int k = 0;
    while (k < (int)c->chunks.size() && c->chunks[k].base) ++k;
    if (k == (int)c->chunks.size()) c->chunks.push_back({});
    c->chunks[k] = prdpt_ctx::Chunk{static_cast<char*>(base), chunk, {}};
    c->chunks[k].free[0] = chunk;
    *p = arena_take(c, bytes);
    return PRDPT_OK;
}

// Release a block; `ready` (owned by the arena from now on, may be null) completes when the
// block's last use has.
void block_release(prdpt_ctx* c, void* p, cudaEvent_t ready) {
    if (!c->blocks.count(p)) return;
    c->pending.push_back({p, ready});
}

bool is_emissive(const float* mp) { return mp[3] > 0.f || mp[4] > 0.f || mp[5] > 0.f; }

double radial_constant(int D) { return std::sqrt(2.0) * std::exp(std::lgamma(0.5 * (D + 1)) - std::lgamma(0.5 * D)); }

prdpt_status check_common(int W, int H, int spp, int depth, int rr_start) {
    if (W < 1 || H < 1 || W > 8192 || H > 8192) return fail(PRDPT_E_INVALID_ARG, "width/height must be in 1..8192");
    if (spp < 1 || spp > 65535) return fail(PRDPT_E_INVALID_ARG, "spp must be in 1..65535");
    if (depth < 1 || depth > 64) return fail(PRDPT_E_INVALID_ARG, "depth must be in 1..64");
    if (rr_start < -1 || rr_start > 64) return fail(PRDPT_E_INVALID_ARG, "rr_start must be -1 or 0..64");
    return PRDPT_OK;
}

Scene* get_scene(prdpt_ctx* c, int id) {
    if (id < 0 || id >= (int)c->scenes.size()) return nullptr;
    return c->scenes[id];
}

Job* get_job(prdpt_ctx* c, int id) {
    if (id < 0 || id >= (int)c->jobs.size()) return nullptr;
    return c->jobs[id];
}

// Pixels per warp work item: the largest of 32, 16, 8 that still gives every
// resident warp at least two items (small jobs use small blocks to fill the GPU).
int choose_block(prdpt_ctx* c, int requested, int R, int W, int H, bool render) {
    if (requested == 8 || requested == 16 || requested == 32) return requested;
    const long long warps = (long long)c->sms * (render ? c->occ_render : c->occ_grad) * (kBlock / 32);
    for (int px : {32, 16}) {
        int bw, bh;
        block_shape(px, &bw, &bh);
        const long long items = (long long)R * ((W + bw - 1) / bw) * ((H + bh - 1) / bh);
        if (items >= 2 * warps) return px;
    }
    return 8;
}

// The render kernels number their work items (render x pixel block) with 32-bit integers.
prdpt_status check_items(long long items) {
    if (items > 0x7fffffffLL)
        return fail(PRDPT_E_INVALID_ARG, "more than 2^31 - 1 work items (renders x pixel blocks): use larger "
                                         "blocks, fewer renders or a smaller image");
    return PRDPT_OK;
}

void tiles_for(int pixels, int W, int H, int* bw, int* bh, int* tiles_x, int* tiles) {
    block_shape(pixels, bw, bh);
    *tiles_x = (W + *bw - 1) / *bw;
    *tiles = *tiles_x * ((H + *bh - 1) / *bh);
}

// Zero-initialised device array that grows on demand (kernels leave it zeroed).
template <typename T>
prdpt_status grow_zeroed(prdpt_ctx* c, T** p, size_t* cap, size_t n) {
    if (*cap >= n) return PRDPT_OK;
    if (prdpt_status st = grow(c, p, cap, n)) return st;
    if (cudaMemset(*p, 0, n * sizeof(T)) != cudaSuccess) return fail(PRDPT_E_CUDA, "cudaMemset failed");
    return PRDPT_OK;
}

int grid_for(prdpt_ctx* c, int items, bool render, int ctas_per_sm) {
    const int occ = render ? c->occ_render : c->occ_grad;
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    const int cap = c->sms * per_sm;
    const int need = (items + kBlock / 32 - 1) / (kBlock / 32);
    return need < cap ? need : cap;
}

// Persistent grid of the pathwise-estimator render kernel (CTAs of kDiffBlock threads).
int grid_for_diff(prdpt_ctx* c, int items, int ctas_per_sm) {
    // ctas_per_sm counts 256-thread CTAs, as for the other render kernels
    const int want = ctas_per_sm * (kBlock / kDiffBlock);
    const int per_sm = (want > 0 && want < c->occ_diff) ? want : c->occ_diff;
    const int cap = c->sms * per_sm;
    const int need = (items + kDiffBlock / 32 - 1) / (kDiffBlock / 32);
    return need < cap ? need : cap;
}

// Persistent grid of the render-group kernel (CTAs of kGroupBlock threads; ctas_per_sm counts
// 256-thread CTAs, so it allows twice as many of these).
int grid_for_group(prdpt_ctx* c, int items, int ctas_per_sm) {
    const int per_sm = (ctas_per_sm > 0 && 2 * ctas_per_sm < c->occ_group) ? 2 * ctas_per_sm : c->occ_group;
    const int cap = c->sms * per_sm;
    const int need = (items + kGroupBlock / 32 - 1) / (kGroupBlock / 32);
    return need < cap ? need : cap;
}

// Persistent grid of the emitter-sharing kernel: one work item per CTA of kGroupBlock threads
// (ctas_per_sm counts 256-thread CTAs, as above).
int grid_for_emit(prdpt_ctx* c, int items, int ctas_per_sm) {
    const int per_sm = (ctas_per_sm > 0 && 2 * ctas_per_sm < c->occ_emit) ? 2 * ctas_per_sm : c->occ_emit;
    const int cap = c->sms * per_sm;
    return items < cap ? items : cap;
}

// Work items of a gradient job's render launch: pixel blocks (path sharing, emitter sharing),
// (block, group of gsize renders) (render-group mode) or (render, block).
long long job_items(const TraceJob& J) {
    if (J.share || J.emit) return J.tiles;
    if (J.gsize > 0) return (long long)J.tiles * (J.R / J.gsize);
    return (long long)J.R * J.tiles;
}

// Launch the render kernel(s), bracketed by events on their stream when timing is on.
// Ls[0..nL): render-kernel launches (a packed step has one for its path-sharing jobs and
// one for the rest); a launch with share = 1 is followed by the affected-path and block
// epilogue passes over its jobs. fin (null when rendering only) covers every render of
// every job for the per-render losses, gradient and Adam.
cudaError_t timed_trace(prdpt_ctx* c, const TraceLaunch* Ls, int nL, const TraceLaunch* fin, bool render,
                        cudaStream_t stream, int ctas_per_sm) {
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (c->timing) {
        if (!c->ev_free.empty()) {
            ev = c->ev_free.back();
            c->ev_free.pop_back();
        } else {
            cudaError_t e = cudaEventCreate(&ev.first);
            if (e == cudaSuccess) e = cudaEventCreate(&ev.second);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaEventRecord(ev.first, stream);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nL; ++i) {
        const int grid = Ls[i].diff_nd ? grid_for_diff(c, Ls[i].total_items, ctas_per_sm)
                         : (Ls[i].group == 2 && !render) ? grid_for_emit(c, Ls[i].total_items, ctas_per_sm)
                         : (Ls[i].group && !render) ? grid_for_group(c, Ls[i].total_items, ctas_per_sm)
                                                    : grid_for(c, Ls[i].total_items, render, ctas_per_sm);
        e = launch_trace(Ls[i], render, grid, stream);
        if (e != cudaSuccess) return e;
    }
    for (int i = 0; i < nL && !render; ++i) {
        if (!Ls[i].share) continue;  // affected paths per render, then their blocks' errors
        e = launch_trace_affected(Ls[i], grid_for(c, 1 << 30, false, ctas_per_sm), stream);
        if (e != cudaSuccess) return e;
        e = launch_shared_epilogue(Ls[i], grid_for(c, 1 << 30, false, 0), stream);
        if (e != cudaSuccess) return e;
    }
    if (fin) {  // per-render losses, gradient, Adam
        e = launch_finalize(*fin, fin->jobs ? fin->fin_total : fin->job0.R, stream);
        if (e != cudaSuccess) return e;
    }
    if (c->timing) {
        e = cudaEventRecord(ev.second, stream);
        if (e != cudaSuccess) return e;
        c->ev_used.push_back(ev);
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char* prdpt_last_error(prdpt_ctx*) { return g_err.c_str(); }

prdpt_status prdpt_create(prdpt_ctx** out, int32_t device, uint64_t hbm_budget_bytes) {
    if (!out) return fail(PRDPT_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    PRDPT_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(PRDPT_E_INVALID_ARG, "no such CUDA device");
    PRDPT_CUDA(cudaSetDevice(device));
    prdpt_ctx* c = new prdpt_ctx();
    c->device = device;
    c->budget = hbm_budget_bytes;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        return fail(PRDPT_E_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
    }
    c->sms = prop.multiProcessorCount;
    c->occ_grad = trace_blocks_per_sm(false);
    c->occ_render = trace_blocks_per_sm(true);
    c->occ_diff = trace_diff_blocks_per_sm();
    c->occ_group = trace_group_blocks_per_sm();
    c->occ_emit = trace_emit_blocks_per_sm();
    e = cudaStreamCreateWithFlags(&c->io, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return fail(PRDPT_E_CUDA, std::string("cudaStreamCreateWithFlags: ") + cudaGetErrorString(e));
    }
    void* p = nullptr;
    prdpt_status st = dev_alloc(c, &p, 128);  // status word, then 8 counters
    if (st) {
        cudaStreamDestroy(c->io);
        delete c;
        return st;
    }
    c->status = static_cast<int*>(p);
    c->counters = reinterpret_cast<unsigned long long*>(static_cast<char*>(p) + 16);
    st = dev_alloc(c, &p, 64);
    if (st) {
        prdpt_destroy(c);
        return st;
    }
    c->s_ctl = static_cast<unsigned*>(p);
    if (cudaMemset(c->status, 0, 128) != cudaSuccess || cudaMemset(c->s_ctl, 0, 64) != cudaSuccess) {
        prdpt_destroy(c);
        return fail(PRDPT_E_CUDA, "cudaMemset of the control block failed");
    }
    *out = c;
    return PRDPT_OK;
}

prdpt_status prdpt_destroy(prdpt_ctx* c) {
    if (!c) return PRDPT_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& kv : c->allocs) cudaFree(kv.first);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->h_zero) cudaFreeHost(c->h_zero);
    for (int k = 0; k < 2; ++k) {
        if (c->h_desc[k]) cudaFreeHost(c->h_desc[k]);
        if (c->h_desc_ev[k]) cudaEventDestroy(c->h_desc_ev[k]);
    }
    for (auto& ev : c->ev_used) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    for (auto& ev : c->ev_free) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    for (auto& q : c->pending)
        if (q.ready) cudaEventDestroy(q.ready);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (Scene* s : c->scenes)
        if (s) {
            if (s->use) cudaEventDestroy(s->use);
            delete s;
        }
    for (Job* j : c->jobs)
        if (j) {
            if (j->last) cudaEventDestroy(j->last);
            delete j;
        }
    if (c->io) cudaStreamDestroy(c->io);
    delete c;
    return PRDPT_OK;
}

prdpt_status prdpt_scene_upload(prdpt_ctx* c, const prdpt_scene_desc* sd, const prdpt_param_binding* binds,
                                int32_t D, int32_t* scene_id_out) {
    if (!c || !sd || !binds || !scene_id_out) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    BaseScene B;
    if (const char* why = build_base_scene(sd, binds, D, true, &B)) return fail(PRDPT_E_INVALID_ARG, why);

    Scene* s = new Scene();
    s->host = B;
    s->D = D;
    void* p = nullptr;
    prdpt_status st = block_alloc(c, &p, sizeof(BaseScene));
    if (st) {
        delete s;
        return st;
    }
    s->dev = static_cast<BaseScene*>(p);
    s->use = take_event(c);
    // on the context's own stream: the copy waits for no other work on the device
    cudaError_t e = s->use ? cudaMemcpyAsync(s->dev, &s->host, sizeof(BaseScene), cudaMemcpyHostToDevice, c->io)
                           : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->io);
    if (e != cudaSuccess) {
        block_release(c, s->dev, nullptr);
        if (s->use) c->ev_pool.push_back(s->use);
        delete s;
        return fail(PRDPT_E_CUDA, std::string("scene upload: ") + cudaGetErrorString(e));
    }
    c->scenes.push_back(s);
    *scene_id_out = (int)c->scenes.size() - 1;
    return PRDPT_OK;
}

prdpt_status prdpt_scene_release(prdpt_ctx* c, int32_t scene_id) {
    if (!c) return fail(PRDPT_E_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    Scene* s = get_scene(c, scene_id);
    if (!s) return fail(PRDPT_E_NOT_FOUND, "unknown scene");
    if (s->jobs) return fail(PRDPT_E_INVALID_ARG, "scene still has jobs");
    // jobs read their own copy of the scene; only the stateless calls read this block, and
    // it is reused only after the last of them has completed
    if (s->captured) PRDPT_CUDA(cudaDeviceSynchronize());
    const bool track = s->used && !s->captured;
    block_release(c, s->dev, track ? s->use : nullptr);
    if (!track) c->ev_pool.push_back(s->use);
    delete s;
    c->scenes[scene_id] = nullptr;
    return PRDPT_OK;
}

// Path sharing across renders is exact when all renders share their path samples (crn)
// and emitters stay fixed: at most kMaxVariant primitives move (bound materials other
// than emitters' are allowed: a path that meets one is traced again by every render), and
// a recorded path's sample index fits the 6 bits of its code (spp <= kMaxShareSpp).
// Recorded-path list of a path-sharing job with room for n paths: codes and segment
// words (u32) and shared-pass radiance (3 floats), then the touching-segment pool
// (2 float4 per slot, kSeg slots and one path state for one path in 8, at least 4096
// paths; a path that finds the pool full is traced again by every render from the camera).
static size_t seg_slots(size_t n) {
    const size_t paths = n / 8 > 4096 ? n / 8 : 4096;
    return paths * kSeg;
}

// recorded-path list of n paths: codes, segment words, shared radiance, the segment pool
// (2 float4 per slot) and the path states (4 float4 per group of kSeg slots)
static size_t afflist_bytes(size_t n) {
    return 2 * ((sizeof(unsigned) * n + 255) & ~size_t(255)) + ((sizeof(float) * 3 * n + 255) & ~size_t(255)) +
           sizeof(float4) * 2 * seg_slots(n) + sizeof(float4) * 4 * (seg_slots(n) / kSeg);
}

static void afflist_carve(TraceJob& J, void* base, size_t n) {
    char* b = static_cast<char*>(base);
    J.aff_codes = reinterpret_cast<unsigned*>(b);
    b += (sizeof(unsigned) * n + 255) & ~size_t(255);
    J.aff_segw = reinterpret_cast<unsigned*>(b);
    b += (sizeof(unsigned) * n + 255) & ~size_t(255);
    J.aff_lsh = reinterpret_cast<float*>(b);
    b += (sizeof(float) * 3 * n + 255) & ~size_t(255);
    J.seg_pool = reinterpret_cast<float4*>(b);
    b += sizeof(float4) * 2 * seg_slots(n);
    J.seg_state = reinterpret_cast<float4*>(b);
    J.seg_cap = unsigned(seg_slots(n));
}

// Decide whether a gradient job shares paths across its renders and, if so, record its
// perturbed primitives in J (and in I, whose launch writes their per-render bounds).
static void fill_share(TraceJob& J, const BaseScene& B, const prdpt_grad_opts* o, InstJob* I = nullptr) {
    J.share = 0;
    J.n_var = 0;
    J.var_prims = 0u;
    J.var_mats = 0u;
    if (I) {
        I->n_var = 0;
        I->var_box = nullptr;
    }
    if (o->no_path_sharing || !o->crn || o->spp > kMaxShareSpp || o->estimator != PRDPT_ESTIMATOR_KERNEL_GRADIENT ||
        B.tex_mat >= 0)  // a texture changes every path that meets it
        return;
    // per-render radiance buffers (24 bytes per render and pixel) and the recorded-path
    // list (20 bytes per path plus the segment pool) each within 512 MB
    const double pix = double(o->width) * double(o->height);
    if (24.0 * 2.0 * o->pairs * pix > double(size_t(512) << 20)) return;
    if (double(afflist_bytes(size_t(pix) * o->spp)) > double(size_t(512) << 20)) return;
    bool var_prim[kMaxPrims] = {};
    for (int d = 0; d < B.D; ++d) {
        const int k = B.bind_kind[d], idx = B.bind_index[d];
        if (k == kBindEmission) return;
        if (k == kBindAlbedo) J.var_mats |= 1u << idx;
        if (k == kBindPos || k == kBindRadius) var_prim[idx] = true;
    }
    int prims[kMaxVariant];
    for (int i = 0; i < B.n_prims; ++i) {
        const float* mp = B.mat_param[B.prim_mat[i]];
        const bool emitter = mp[3] > 0.f || mp[4] > 0.f || mp[5] > 0.f;
        if (emitter && (var_prim[i] || ((J.var_mats >> B.prim_mat[i]) & 1u))) return;
        if (!var_prim[i]) continue;
        if (J.n_var == kMaxVariant) return;
        prims[J.n_var] = i;
        J.var_slot[J.n_var++] = B.prim_slot[i];
        J.var_prims |= 1u << B.prim_slot[i];
    }
    J.share = 1;
    if (I) {
        I->n_var = J.n_var;
        for (int k = 0; k < J.n_var; ++k) I->var_prim[k] = prims[k];
    }
}

// Render-group mode for a gradient job that does not share paths (see render_groups in
// prdpt.h): the perturbed primitives (position and radius bindings, emitters included) and
// the bound materials (albedo bindings) become per-render records of each lane; gsize
// renders of one path sample are traced side by side. Needs common random numbers (the
// renders' paths then agree until a perturbed primitive intervenes), the Eq. 10 estimator,
// no texture and no emission bindings (those change which primitives emit).
static void fill_group(TraceJob& J, const BaseScene& B, const prdpt_grad_opts* o) {
    J.gsize = 0;
    J.gstride = 0;
    J.emit = 0;
    if (J.share || o->render_groups < 0 || !o->crn || o->estimator != PRDPT_ESTIMATOR_KERNEL_GRADIENT ||
        B.tex_mat >= 0 || B.n_prims > kGroupPrims || B.n_mats > kGroupMats)
        return;
    unsigned prims = 0u, mats = 0u;
    bool radius = false;
    for (int d = 0; d < B.D; ++d) {
        const int k = B.bind_kind[d], idx = B.bind_index[d];
        if (k == kBindEmission) return;
        if (k == kBindAlbedo) mats |= 1u << idx;
        if (k == kBindPos || k == kBindRadius) prims |= 1u << B.prim_slot[idx];
        radius = radius || k == kBindRadius;
    }
    const int n = __builtin_popcount(prims), nm = __builtin_popcount(mats);
    if (n > kMaxVariant) return;
    // per render: the perturbed primitives' records (4 float4 each), the bound materials'
    // albedo rows, and the 8 emitter areas when a radius binding can change one
    const int stride = 4 * n + nm + (radius ? 2 : 0);
    if (stride == 0) return;
    const int R = J.R;
    // Emitter sharing (k_trace_emit): every emitter perturbed, no bound material, at most 64
    // renders; paths are traced once for all renders (path sharing's switch turns it off)
    bool emitters_perturbed = n > 0 && mats == 0u && R >= 1 && R <= 64 && R * stride <= kEmitTabRows;
    for (int i = 0; i < B.n_prims && emitters_perturbed; ++i)
        if (is_emissive(B.mat_param[B.prim_mat[i]]) && !((prims >> B.prim_slot[i]) & 1u)) emitters_perturbed = false;
    if (emitters_perturbed && !o->no_path_sharing) {
        J.emit = 1;
        J.gstride = stride;
        J.n_var = n;
        J.var_prims = prims;
        J.var_mats = 0u;
        return;
    }
    int G = 0;
    if (o->render_groups > 0) {
        const int g = o->render_groups;
        if ((g & (g - 1)) == 0 && g >= 2 && g <= 32 && R % g == 0 && g * stride <= kGroupTabRows) G = g;
    } else {
        for (int g = 32; g >= 2; g >>= 1)
            if (R % g == 0 && g * stride <= kGroupTabRows) {
                G = g;
                break;
            }
    }
    if (!G) return;
    J.gsize = G;
    J.gstride = stride;
    J.n_var = n;
    J.var_prims = prims;
    J.var_mats = mats;
}

static void fill_inst_common(InstJob& J, const Scene* s, int R, int D, int W, int H) {
    std::memset(&J, 0, sizeof(J));
    J.base = s->dev;
    J.R = R;
    J.D = D;
    J.W = W;
    J.H = H;
    J.c_radial = float(radial_constant(D));
}

prdpt_status prdpt_render_batch(prdpt_ctx* c, int32_t scene_id, const float* thetas_dev, int32_t n,
                                const prdpt_render_opts* o, float* images_dev, void* stream) {
    if (!c || !o || !thetas_dev || !images_dev) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    Scene* s = get_scene(c, scene_id);
    if (!s) return fail(PRDPT_E_NOT_FOUND, "unknown scene");
    if (n < 1 || n > kMaxRenders) return fail(PRDPT_E_INVALID_ARG, "n must be in 1..512");
    if (prdpt_status st = check_common(o->width, o->height, o->spp, o->depth, o->rr_start)) return st;
    if (o->tag > 15) return fail(PRDPT_E_INVALID_ARG, "tag must be in 0..15");
    PRDPT_CUDA(cudaSetDevice(c->device));
    if (prdpt_status st = grow(c, &c->s_scenes, &c->s_scenes_n, (size_t)n)) return st;
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    InstLaunch IL{};
    fill_inst_common(IL.job0, s, n, s->D, o->width, o->height);
    IL.job0.scenes = c->s_scenes;
    IL.job0.theta = thetas_dev;
    IL.job0.seed = o->seed;
    IL.job0.step = o->step;
    IL.job0.tag = o->tag;
    IL.job0.crn = o->crn;
    IL.job0.render_mode = 1;
    if (s->host.tex_mat >= 0) {  // texture scenes: thetas [n][D] are the textures themselves
        IL.job0.hd = 1;
        IL.job0.tex_all = thetas_dev;
        IL.job0.tex_D = s->D;
    }
    IL.total_blocks = n;
    IL.queue_reset = c->s_ctl + 0;
    PRDPT_CUDA(launch_instantiate(IL, st_));
    const int px = choose_block(c, o->block_pixels, n, o->width, o->height, true);
    TraceLaunch TL{};
    TraceJob& J = TL.job0;
    J.scenes = c->s_scenes;
    J.images = reinterpret_cast<float4*>(images_dev);
    J.W = o->width;
    J.H = o->height;
    J.spp = o->spp;
    J.depth = o->depth;
    J.rr_start = o->rr_start;
    J.R = n;
    J.D = s->D;
    J.n_prims = s->host.n_prims;
    J.n_mats = s->host.n_mats;
    tiles_for(px, o->width, o->height, &J.bw, &J.bh, &J.tiles_x, &J.tiles);
    if (prdpt_status st = check_items((long long)n * J.tiles)) return st;
    TL.total_items = n * J.tiles;
    TL.queue = c->s_ctl + 0;
    TL.counters = c->counting ? c->counters : nullptr;
    TL.status = c->status;
    PRDPT_CUDA(timed_trace(c, &TL, 1, nullptr, true, st_, o->ctas_per_sm));
    PRDPT_CUDA(mark_use(s->use, &s->used, &s->captured, st_));  // the scene block is in use until here
    return PRDPT_OK;
}

// CTAs per draw of the radial sampler's norms in D dimensions: about 2048 terms each.
static int hd_norm_split(int D) {
    const long long terms = (long long)D + 1 + (D + 1) / 2;
    const long long n = (terms + 2047) / 2048;
    return int(n < 1 ? 1 : (n > kNormSplitMax ? kNormSplitMax : n));
}

// Draws of a texture scene (D > kMaxD parameters) by the high-dimensional kernels.
static HdDraws hd_draws(const Scene* s, const prdpt_grad_opts* o, const float* theta, const float* sigma,
                        HdNorm* norms, float* theta_out, float* w_out) {
    HdDraws H{};
    H.D = s->D;
    H.R = 2 * o->pairs;
    H.sampler = o->sampler;
    H.antithetic = o->antithetic ? 1 : 0;
    H.draw_begin = o->antithetic ? o->pair_begin : 2 * o->pair_begin;
    H.seed = o->seed;
    H.step = o->step;
    H.theta = theta;
    H.sigma = sigma;
    H.c_radial = float(radial_constant(s->D));
    H.norms = norms;
    H.norm_split = hd_norm_split(s->D);
    H.theta_out = theta_out;
    H.w_out = w_out;
    return H;
}

static prdpt_status check_grad_opts(const prdpt_grad_opts* o) {
    if (o->pairs < 1 || o->pairs > kMaxPairs) return fail(PRDPT_E_INVALID_ARG, "pairs must be in 1..256");
    if (o->sampler < 0 || o->sampler > 2) return fail(PRDPT_E_INVALID_ARG, "unknown sampler");
    if (o->estimator != PRDPT_ESTIMATOR_KERNEL_GRADIENT && o->estimator != PRDPT_ESTIMATOR_PATHWISE)
        return fail(PRDPT_E_INVALID_ARG, "unknown estimator");
    if (o->pair_begin < 0 || o->pair_begin > (1 << 26)) return fail(PRDPT_E_INVALID_ARG, "pair_begin must be in 0..2^26");
    if (o->estimator == PRDPT_ESTIMATOR_PATHWISE && o->sampler != PRDPT_SAMPLER_GAUSS)
        return fail(PRDPT_E_INVALID_ARG, "the pathwise estimator (Eq. 9) samples the Gaussian kernel: sampler must be GAUSS");
    return check_common(o->width, o->height, o->spp, o->depth, o->rr_start);
}

// Pathwise estimator (Eq. 9): every binding must be an albedo or emission one (their
// tangents are exact pathwise derivatives; geometry would need boundary terms).
static prdpt_status fill_diff(TraceJob& J, const BaseScene& B, const prdpt_grad_opts* o) {
    J.diff = 0;
    J.diff_n = 0;
    if (o->estimator != PRDPT_ESTIMATOR_PATHWISE) return PRDPT_OK;
    if (B.tex_mat >= 0) return fail(PRDPT_E_INVALID_ARG, "the pathwise estimator does not take texture parameters");
    if (B.D > kMaxDiff) return fail(PRDPT_E_INVALID_ARG, "the pathwise estimator takes at most 8 parameters");
    for (int d = 0; d < B.D; ++d) {
        const int kind = B.bind_kind[d];
        if (kind != kBindAlbedo && kind != kBindEmission)
            return fail(PRDPT_E_INVALID_ARG, "the pathwise estimator differentiates albedo and emission bindings only");
        J.diff_mat[d] = B.bind_index[d];
        J.diff_comp[d] = B.bind_comp[d];
        J.diff_kind[d] = kind;
    }
    J.diff = 1;
    J.diff_n = B.D;
    return PRDPT_OK;
}

// tangent slots of the pathwise render kernel: the smallest of 4, 6, 8 that holds every parameter
static int diff_slots(const TraceJob& J) { return J.diff ? (J.diff_n <= 4 ? 4 : (J.diff_n <= 6 ? 6 : 8)) : 0; }

static void fill_inst_grad(InstJob& J, const Scene* s, const prdpt_grad_opts* o) {
    fill_inst_common(J, s, 2 * o->pairs, s->D, o->width, o->height);
    J.diff = o->estimator == PRDPT_ESTIMATOR_PATHWISE ? 1 : 0;
    J.pair_begin = o->pair_begin;
    J.seed = o->seed;
    J.step = o->step;
    J.tag = kTagPath;
    J.sampler = o->sampler;
    J.antithetic = o->antithetic ? 1 : 0;
    J.crn = o->crn ? 1 : 0;
    J.render_mode = 0;
}

prdpt_status prdpt_sample_perturbations(prdpt_ctx* c, int32_t D, const float* sigma_dev, const prdpt_grad_opts* o,
                                        float* tau_dev, float* w_dev, void* stream) {
    if (!c || !o || !sigma_dev || !tau_dev || !w_dev) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    if (D < 1 || D > 3 * kMaxTexRes * kMaxTexRes) return fail(PRDPT_E_INVALID_ARG, "D must be in 1..3 * 1024^2");
    if (o->pairs < 1 || o->pairs > kMaxPairs) return fail(PRDPT_E_INVALID_ARG, "pairs must be in 1..256");
    if (o->sampler < 0 || o->sampler > 2) return fail(PRDPT_E_INVALID_ARG, "unknown sampler");
    std::lock_guard<std::mutex> lk(c->mu);
    PRDPT_CUDA(cudaSetDevice(c->device));
    if (D > kMaxD) {  // the high-dimensional kernels
        if (prdpt_status st = grow_zeroed(c, &c->s_norms, &c->s_norms_n, (size_t)2 * o->pairs)) return st;
        HdDraws H{};
        H.D = D;
        H.R = 2 * o->pairs;
        H.sampler = o->sampler;
        H.antithetic = o->antithetic ? 1 : 0;
        H.draw_begin = o->antithetic ? o->pair_begin : 2 * o->pair_begin;
        H.seed = o->seed;
        H.step = o->step;
        H.sigma = sigma_dev;
        H.c_radial = float(radial_constant(D));
        H.norms = c->s_norms;
        H.norm_split = hd_norm_split(D);
        H.tau_out = tau_dev;
        H.w_out = w_dev;
        PRDPT_CUDA(launch_hd_draws(H, static_cast<cudaStream_t>(stream)));
        return PRDPT_OK;
    }
    // reuse the theta slot for a zero vector: the draws do not depend on theta
    if (prdpt_status st = grow(c, &c->s_w, &c->s_w_n, (size_t)kMaxD)) return st;
    PRDPT_CUDA(cudaMemsetAsync(c->s_w, 0, sizeof(float) * D, static_cast<cudaStream_t>(stream)));
    InstLaunch IL{};
    std::memset(&IL.job0, 0, sizeof(InstJob));
    IL.job0.R = 2 * o->pairs;
    IL.job0.D = D;
    IL.job0.W = 1;
    IL.job0.H = 1;
    IL.job0.c_radial = float(radial_constant(D));
    IL.job0.theta = c->s_w;
    IL.job0.sigma = sigma_dev;
    IL.job0.tau_out = tau_dev;
    IL.job0.w_out = w_dev;
    IL.job0.seed = o->seed;
    IL.job0.step = o->step;
    IL.job0.sampler = o->sampler;
    IL.job0.antithetic = o->antithetic ? 1 : 0;
    IL.job0.pair_begin = o->pair_begin;
    IL.total_blocks = 2 * o->pairs;  // scenes == null: draws only, no scene binding
    PRDPT_CUDA(launch_instantiate(IL, static_cast<cudaStream_t>(stream)));
    return PRDPT_OK;
}

}  // extern "C"

namespace {

// prdpt_smoothed_grad with the context's mutex held by the caller.
// Adam state on the device for a call that also takes the optimiser step: the last CTA of
// k_finalize (k_hd_grad for texture scenes) updates theta, m, v; *step holds t - 1 and is
// advanced to t on the device.
struct AdamDev {
    float *theta, *m, *v;
    int* step;
    float lr, b1, b2, eps;
};

prdpt_status smoothed_grad_locked(prdpt_ctx* c, int32_t scene_id, const float* theta_dev, const float* sigma_dev,
                                  const prdpt_grad_opts* o, const float* target_dev, float* grad_dev,
                                  float* losses_dev, void* stream, const AdamDev* adam = nullptr) {
    Scene* s = get_scene(c, scene_id);
    if (!s) return fail(PRDPT_E_NOT_FOUND, "unknown scene");
    if (prdpt_status st = check_grad_opts(o)) return st;
    PRDPT_CUDA(cudaSetDevice(c->device));
    const int R = 2 * o->pairs, D = s->D;
    TraceJob probe{};
    if (prdpt_status st = fill_diff(probe, s->host, o)) return st;
    probe.R = R;
    fill_share(probe, s->host, o);  // path or emitter sharing: items are blocks, not (render, block)
    fill_group(probe, s->host, o);
    const bool per_block = probe.share || probe.emit;
    const int px = choose_block(c, o->block_pixels, per_block ? 1 : R, o->width, o->height, false);
    int bw, bh, tiles_x, tiles;
    tiles_for(px, o->width, o->height, &bw, &bh, &tiles_x, &tiles);
    if (prdpt_status st = check_items(per_block ? (long long)tiles : (long long)R * tiles)) return st;
    if (probe.share) {
        const size_t pix = (size_t)o->width * o->height;
        if (prdpt_status st = grow(c, &c->s_share, &c->s_share_n, (size_t)tiles * 96)) return st;
        if (prdpt_status st = grow(c, &c->s_aff, &c->s_aff_n, (size_t)tiles)) return st;
        if (prdpt_status st = grow_zeroed(c, &c->s_accaff, &c->s_accaff_n, (size_t)R * pix * 3)) return st;
        if (prdpt_status st = grow(c, &c->s_afflist, &c->s_afflist_n, afflist_bytes(pix * o->spp))) return st;
        if (prdpt_status st = grow(c, &c->s_varbox, &c->s_varbox_n, (size_t)R * kMaxVariant * 2)) return st;
        if (prdpt_status st = grow(c, &c->s_cursor, &c->s_cursor_n, (size_t)R)) return st;
        if (prdpt_status st = grow(c, &c->s_flags, &c->s_flags_n, (size_t)R * ((pix + 31) / 32))) return st;
    }
    if (prdpt_status st = grow(c, &c->s_scenes, &c->s_scenes_n, (size_t)R)) return st;
    if (prdpt_status st = grow(c, &c->s_w, &c->s_w_n, (size_t)R * D > (size_t)kMaxD ? (size_t)R * D : (size_t)kMaxD))
        return st;
    if (prdpt_status st = grow(c, &c->s_partials, &c->s_partials_n, (size_t)R * tiles)) return st;
    if (prdpt_status st = grow(c, &c->s_losses, &c->s_losses_n, (size_t)R)) return st;
    if (probe.diff) {
        if (prdpt_status st = grow(c, &c->s_gpart, &c->s_gpart_n, (size_t)R * tiles * D)) return st;
        if (prdpt_status st = grow(c, &c->s_rgrads, &c->s_rgrads_n, (size_t)R * kMaxDiff)) return st;
    }
    const bool tex = s->host.tex_mat >= 0;
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    if (tex) {  // a1 over the texture's D parameters: per-render textures and weights
        if (prdpt_status st = grow(c, &c->s_tex, &c->s_tex_n, (size_t)R * D)) return st;
        if (prdpt_status st = grow_zeroed(c, &c->s_norms, &c->s_norms_n, (size_t)R)) return st;
        PRDPT_CUDA(launch_hd_draws(hd_draws(s, o, theta_dev, sigma_dev, c->s_norms, c->s_tex, c->s_w), st_));
    }
    InstLaunch IL{};
    fill_inst_grad(IL.job0, s, o);
    IL.job0.scenes = c->s_scenes;
    IL.job0.theta = theta_dev;
    IL.job0.sigma = sigma_dev;
    IL.job0.w_out = c->s_w;
    IL.job0.hd = tex ? 1 : 0;
    IL.job0.tex_all = tex ? c->s_tex : nullptr;
    IL.job0.tex_D = D;
    IL.total_blocks = R;
    IL.queue_reset = c->s_ctl + 0;
    IL.job0.share_reset = probe.share ? c->s_ctl + 4 : nullptr;
    fill_share(probe, s->host, o, &IL.job0);
    if (probe.share) {
        IL.job0.var_box = c->s_varbox;
        IL.job0.aff_cursor = c->s_cursor;
        IL.job0.aff_flags = c->s_flags;
        IL.job0.flag_words = int(((size_t)o->width * o->height + 31) / 32);
    }
    PRDPT_CUDA(launch_instantiate(IL, st_));
    TraceLaunch TL{};
    TraceJob& J = TL.job0;
    J.scenes = c->s_scenes;
    J.target = reinterpret_cast<const float4*>(target_dev);
    J.partials = c->s_partials;
    J.done = c->s_ctl + 1;
    J.losses = c->s_losses;
    J.w = c->s_w;
    J.grad_out = grad_dev;
    J.loss_out = losses_dev;
    J.W = o->width;
    J.H = o->height;
    J.spp = o->spp;
    J.depth = o->depth;
    J.rr_start = o->rr_start;
    J.R = R;
    J.D = D;
    J.antithetic = o->antithetic ? 1 : 0;
    J.bw = bw;
    J.bh = bh;
    J.tiles_x = tiles_x;
    J.tiles = tiles;
    J.n_prims = s->host.n_prims;
    J.n_mats = s->host.n_mats;
    fill_share(J, s->host, o);
    fill_group(J, s->host, o);
    if (J.share) {
        J.share_acc = c->s_share;
        J.acc_aff = c->s_accaff;
        afflist_carve(J, c->s_afflist, (size_t)o->width * o->height * o->spp);
        J.var_box = c->s_varbox;
        J.aff_cursor = c->s_cursor;
        J.aff_flags = c->s_flags;
        J.flag_words = int(((size_t)o->width * o->height + 31) / 32);
        J.aff_tiles = c->s_aff;
        J.share_ctl = c->s_ctl + 4;
    }
    fill_diff(J, s->host, o);
    if (J.diff) {
        J.gpartials = c->s_gpart;
        J.rgrads = c->s_rgrads;
    }
    J.hd = tex ? 1 : 0;
    if (adam) {
        J.theta = adam->theta;
        J.m = adam->m;
        J.v = adam->v;
        J.step_dev = adam->step;
        J.lr = adam->lr;
        J.b1 = adam->b1;
        J.b2 = adam->b2;
        J.eps = adam->eps;
    }
    TL.diff_nd = diff_slots(J);
    TL.total_items = int(job_items(J));
    TL.share = J.share;
    TL.group = J.emit ? 2 : (J.gsize > 0 ? 1 : 0);
    TL.queue = c->s_ctl + 0;
    TL.counters = c->counting ? c->counters : nullptr;
    TL.status = c->status;
    PRDPT_CUDA(timed_trace(c, &TL, 1, &TL, false, st_, o->ctas_per_sm));
    if (tex) {  // a6: g = W^T dL / 2P over the texture's parameters
        HdGrad G{};
        G.D = D;
        G.R = R;
        G.antithetic = o->antithetic ? 1 : 0;
        G.w = c->s_w;
        G.losses = c->s_losses;
        G.grad_out = grad_dev;
        if (adam) {
            G.theta = adam->theta;
            G.m = adam->m;
            G.v = adam->v;
            G.step_dev = adam->step;
            G.lr = adam->lr;
            G.b1 = adam->b1;
            G.b2 = adam->b2;
            G.eps = adam->eps;
        }
        PRDPT_CUDA(launch_hd_grad(G, st_));
    }
    PRDPT_CUDA(mark_use(s->use, &s->used, &s->captured, st_));  // the scene block is in use until here
    return PRDPT_OK;
}

}  // namespace

extern "C" {

prdpt_status prdpt_smoothed_grad(prdpt_ctx* c, int32_t scene_id, const float* theta_dev, const float* sigma_dev,
                                 const prdpt_grad_opts* o, const float* target_dev, float* grad_dev,
                                 float* losses_dev, void* stream) {
    if (!c || !o || !theta_dev || !sigma_dev || !target_dev || !grad_dev)
        return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    return smoothed_grad_locked(c, scene_id, theta_dev, sigma_dev, o, target_dev, grad_dev, losses_dev, stream);
}

}  // extern "C"

namespace {

struct HostAdam {  // prdpt_step_host: Adam state in host memory, updated in place
    float *theta, *m, *v;
    int t;
    float lr, b1, b2, eps;
};

// The gradient with host buffers, and with `adam` one Adam update of theta, m, v, taken by
// the gradient's last kernel. The small vectors go through a page-locked staging buffer (one
// upload, one download of what the caller gets back); the target is copied straight from
// the caller's buffer.
prdpt_status host_buffer_call(prdpt_ctx* c, int32_t scene_id, const float* theta_host, const float* sigma_host,
                              const prdpt_grad_opts* o, const float* target_host, float* grad_host,
                              float* losses_host, void* stream, const HostAdam* adam) {
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    float *target_d, *io_d, *stage;
    size_t D, R, small;
    std::lock_guard<std::mutex> lk(c->mu);  // the whole call: the scratch and staging are per context
    {
        Scene* s = get_scene(c, scene_id);
        if (!s) return fail(PRDPT_E_NOT_FOUND, "unknown scene");
        if (prdpt_status st = check_grad_opts(o)) return st;
        PRDPT_CUDA(cudaSetDevice(c->device));
        D = size_t(s->D);
        R = 2 * size_t(o->pairs);
        const size_t pix4 = 4 * size_t(o->width) * size_t(o->height);
        small = 5 * D + 1 + R;
        // device: [target (16-byte aligned for float4 loads) | sigma | step | theta | m | v | grad | losses],
        // the staging buffer mirrors everything after the target
        if (prdpt_status st = grow(c, &c->s_host_io, &c->s_host_io_n, pix4 + small)) return st;
        if (c->h_stage_n < small) {  // the previous call has synchronised: the old buffer is idle
            if (c->h_stage) cudaFreeHost(c->h_stage);
            c->h_stage = nullptr;
            c->h_stage_n = 0;
            void* p = nullptr;
            PRDPT_CUDA(cudaHostAlloc(&p, sizeof(float) * small, cudaHostAllocDefault));
            c->h_stage = static_cast<float*>(p);
            c->h_stage_n = small;
        }
        stage = c->h_stage;
        target_d = c->s_host_io;
        io_d = target_d + pix4;
        const int32_t step0 = adam ? adam->t - 1 : 0;
        std::memcpy(stage, sigma_host, sizeof(float) * D);
        std::memcpy(stage + D, &step0, sizeof(step0));
        std::memcpy(stage + D + 1, theta_host, sizeof(float) * D);
        if (adam) {
            std::memcpy(stage + 2 * D + 1, adam->m, sizeof(float) * D);
            std::memcpy(stage + 3 * D + 1, adam->v, sizeof(float) * D);
        }
        PRDPT_CUDA(cudaMemcpyAsync(io_d, stage, sizeof(float) * ((adam ? 4 : 2) * D + 1), cudaMemcpyHostToDevice, st_));
        PRDPT_CUDA(cudaMemcpyAsync(target_d, target_host, sizeof(float) * pix4, cudaMemcpyHostToDevice, st_));
    }
    float *sigma_d = io_d, *theta_d = io_d + D + 1, *grad_d = io_d + 4 * D + 1;
    AdamDev ad{};
    if (adam)
        ad = AdamDev{theta_d, io_d + 2 * D + 1, io_d + 3 * D + 1, reinterpret_cast<int*>(io_d + D),
                     adam->lr, adam->b1, adam->b2, adam->eps};
    if (prdpt_status st = smoothed_grad_locked(c, scene_id, theta_d, sigma_d, o, target_d, grad_d, grad_d + D, stream,
                                               adam ? &ad : nullptr))
        return st;
    // one download: [theta | m | v | grad | losses] after an optimiser step, else [grad | losses]
    const size_t first = adam ? D + 1 : 4 * D + 1;
    PRDPT_CUDA(cudaMemcpyAsync(stage + first, io_d + first, sizeof(float) * (small - first), cudaMemcpyDeviceToHost,
                               st_));
    PRDPT_CUDA(cudaStreamSynchronize(st_));
    if (adam) {
        std::memcpy(adam->theta, stage + D + 1, sizeof(float) * D);
        std::memcpy(adam->m, stage + 2 * D + 1, sizeof(float) * D);
        std::memcpy(adam->v, stage + 3 * D + 1, sizeof(float) * D);
    }
    if (grad_host) std::memcpy(grad_host, stage + 4 * D + 1, sizeof(float) * D);
    if (losses_host) std::memcpy(losses_host, stage + 5 * D + 1, sizeof(float) * R);
    return PRDPT_OK;
}

}  // namespace

extern "C" {

prdpt_status prdpt_smoothed_grad_host(prdpt_ctx* c, int32_t scene_id, const float* theta_host,
                                      const float* sigma_host, const prdpt_grad_opts* o, const float* target_host,
                                      float* grad_host, float* losses_host, void* stream) {
    if (!c || !o || !theta_host || !sigma_host || !target_host || !grad_host)
        return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    return host_buffer_call(c, scene_id, theta_host, sigma_host, o, target_host, grad_host, losses_host, stream,
                            nullptr);
}

prdpt_status prdpt_step_host(prdpt_ctx* c, int32_t scene_id, float* theta_host, float* m_host, float* v_host,
                             int32_t t, float lr, float beta1, float beta2, float eps, const float* sigma_host,
                             const prdpt_grad_opts* o, const float* target_host, float* grad_host,
                             float* losses_host, void* stream) {
    if (!c || !o || !theta_host || !m_host || !v_host || !sigma_host || !target_host)
        return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    if (t < 1) return fail(PRDPT_E_INVALID_ARG, "t must be >= 1");
    const HostAdam adam{theta_host, m_host, v_host, t, lr, beta1, beta2, eps};
    return host_buffer_call(c, scene_id, theta_host, sigma_host, o, target_host, grad_host, losses_host, stream,
                            &adam);
}

prdpt_status prdpt_adam_step(prdpt_ctx* c, int32_t D, float* theta_dev, float* m_dev, float* v_dev,
                             const float* grad_dev, int32_t t, float lr, float beta1, float beta2, float eps,
                             void* stream) {
    if (!c || !theta_dev || !m_dev || !v_dev || !grad_dev) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    if (D < 1 || t < 1) return fail(PRDPT_E_INVALID_ARG, "D and t must be >= 1");
    PRDPT_CUDA(cudaSetDevice(c->device));
    PRDPT_CUDA(launch_adam(D, theta_dev, m_dev, v_dev, grad_dev, t, lr, beta1, beta2, eps,
                           static_cast<cudaStream_t>(stream)));
    return PRDPT_OK;
}

prdpt_status prdpt_job_create(prdpt_ctx* c, int32_t scene_id, const prdpt_job_desc* d, int32_t* job_out) {
    if (!c || !d || !job_out || !d->theta0_host || !d->sigma0_host)
        return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    Scene* s = get_scene(c, scene_id);
    if (!s) return fail(PRDPT_E_NOT_FOUND, "unknown scene");
    const prdpt_grad_opts* o = &d->grad;
    if (prdpt_status st = check_grad_opts(o)) return st;
    PRDPT_CUDA(cudaSetDevice(c->device));
    TraceJob probe{};
    if (prdpt_status st = fill_diff(probe, s->host, o)) return st;
    probe.R = 2 * o->pairs;
    fill_share(probe, s->host, o);
    fill_group(probe, s->host, o);
    Job* j = new Job();
    j->scene = scene_id;
    j->D = s->D;
    j->R = 2 * o->pairs;
    const int D = j->D, R = j->R, W = o->width, H = o->height;
    const bool per_block = probe.share || probe.emit;
    const int px = choose_block(c, o->block_pixels, per_block ? 1 : R, W, H, false);
    int bw, bh, tiles_x, tiles;
    tiles_for(px, W, H, &bw, &bh, &tiles_x, &tiles);
    if (prdpt_status st = check_items(per_block ? (long long)tiles : (long long)R * tiles)) {
        delete j;
        return st;
    }
    j->tiles = tiles;
    j->ctas_per_sm = o->ctas_per_sm;
    // one device block per job: small state first (zeroed), then w, partials, scenes, target
    const size_t small = 6 * sizeof(float) * kMaxD + sizeof(float) * kMaxRenders + sizeof(double) * kMaxRenders +
                         sizeof(unsigned) * kMaxRenders + 64;
    const size_t off_w = (small + 255) & ~size_t(255);
    const size_t off_p = (off_w + sizeof(float) * R * D + 255) & ~size_t(255);
    const size_t off_s = (off_p + sizeof(double) * R * tiles + 255) & ~size_t(255);
    const size_t off_t = (off_s + sizeof(InstScene) * R + 255) & ~size_t(255);
    const size_t pix = (size_t)W * H;
    const size_t off_sh = (off_t + sizeof(float4) * pix + 255) & ~size_t(255);
    const size_t off_aa = (off_sh + (probe.share ? sizeof(unsigned long long) * 96 * (size_t)tiles : 0) + 255) &
                          ~size_t(255);
    const size_t off_cd = (off_aa + (probe.share ? sizeof(unsigned long long) * 3 * (size_t)R * pix : 0) + 255) &
                          ~size_t(255);
    const size_t off_vb = (off_cd + (probe.share ? afflist_bytes(pix * o->spp) : 0) + 255) & ~size_t(255);
    const size_t off_cu = (off_vb + (probe.share ? sizeof(float4) * 2 * kMaxVariant * (size_t)R : 0) + 255) &
                          ~size_t(255);
    const size_t off_af = (off_cu + (probe.share ? sizeof(unsigned) * (size_t)R : 0) + 255) & ~size_t(255);
    const size_t off_fl = (off_af + (probe.share ? sizeof(int) * (size_t)tiles : 0) + 255) & ~size_t(255);
    const int flag_words = int(((size_t)W * H + 31) / 32);
    const size_t off_gp =
        (off_fl + (probe.share ? sizeof(unsigned) * (size_t)R * flag_words : 0) + 255) & ~size_t(255);
    const size_t off_rg = (off_gp + (probe.diff ? sizeof(double) * (size_t)R * tiles * D : 0) + 255) & ~size_t(255);
    // texture scenes: theta, m, v, sigma0, grad of D entries; per-render textures; norms
    const bool tex = s->host.tex_mat >= 0;
    const size_t off_hs = (off_rg + (probe.diff ? sizeof(double) * (size_t)R * kMaxDiff : 0) + 255) & ~size_t(255);
    const size_t off_tx = (off_hs + (tex ? sizeof(float) * 5 * (size_t)D : 0) + 255) & ~size_t(255);
    const size_t off_nr = (off_tx + (tex ? sizeof(float) * (size_t)R * D : 0) + 255) & ~size_t(255);
    const size_t off_bs = (off_nr + (tex ? sizeof(HdNorm) * (size_t)R : 0) + 255) & ~size_t(255);
    const size_t total = off_bs + sizeof(BaseScene);  // the job's own copy of its scene
    void* base = nullptr;
    if (prdpt_status st = block_alloc(c, &base, total)) {
        delete j;
        return st;
    }
    j->last = take_event(c);
    if (!j->last) {
        block_release(c, base, nullptr);
        delete j;
        return fail(PRDPT_E_CUDA, "cudaEventCreate failed");
    }
    j->bytes = total;
    j->base = base;
    char* b = static_cast<char*>(base);
    j->theta = reinterpret_cast<float*>(b);
    j->m = j->theta + kMaxD;
    j->v = j->m + kMaxD;
    j->sigma0 = j->v + kMaxD;
    j->grad = j->sigma0 + kMaxD;
    j->losses = j->grad + kMaxD;
    j->losses_d = reinterpret_cast<double*>(j->losses + kMaxRenders);
    j->rdone = reinterpret_cast<unsigned*>(j->losses_d + kMaxRenders);
    j->step = reinterpret_cast<int*>(j->rdone + kMaxRenders);
    j->done = reinterpret_cast<unsigned*>(j->step + 1);
    j->queue = j->done + 1;
    unsigned* share_ctl = j->queue + 1;  // path-sharing counters: listed blocks, paths, segment slots, spare
    j->w = reinterpret_cast<float*>(b + off_w);
    j->partials = reinterpret_cast<double*>(b + off_p);
    j->scenes = reinterpret_cast<InstScene*>(b + off_s);
    j->target = reinterpret_cast<float4*>(b + off_t);
    if (probe.share) {
        j->share = reinterpret_cast<unsigned long long*>(b + off_sh);
        j->accaff = reinterpret_cast<unsigned long long*>(b + off_aa);
        j->afflist = b + off_cd;
        j->varbox = reinterpret_cast<float4*>(b + off_vb);
        j->cursor = reinterpret_cast<unsigned*>(b + off_cu);
        j->aff = reinterpret_cast<int*>(b + off_af);
        j->flags = reinterpret_cast<unsigned*>(b + off_fl);
    }
    j->tex = tex;
    j->scene_copy = reinterpret_cast<BaseScene*>(b + off_bs);
    // uploads on the context's own stream (they wait for no other work on the device); the
    // block may be a reused one, so everything that must start at zero is cleared here
    cudaStream_t io = c->io;
    cudaError_t e = zero_async(c, base, off_w, io);
    if (tex) {
        j->theta = reinterpret_cast<float*>(b + off_hs);
        j->m = j->theta + D;
        j->v = j->m + D;
        j->sigma0 = j->v + D;
        j->grad = j->sigma0 + D;
        j->tex_all = reinterpret_cast<float*>(b + off_tx);
        j->norms = reinterpret_cast<HdNorm*>(b + off_nr);
        if (e == cudaSuccess) e = zero_async(c, j->theta, sizeof(float) * 5 * (size_t)D, io);
        if (e == cudaSuccess) e = zero_async(c, j->norms, sizeof(HdNorm) * (size_t)R, io);  // part counters
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->scene_copy, &s->host, sizeof(BaseScene), cudaMemcpyHostToDevice, io);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->theta, d->theta0_host, sizeof(float) * D, cudaMemcpyHostToDevice, io);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->sigma0, d->sigma0_host, sizeof(float) * D, cudaMemcpyHostToDevice, io);
    if (e == cudaSuccess) {
        if (d->target_host)
            e = cudaMemcpyAsync(j->target, d->target_host, sizeof(float4) * (size_t)W * H, cudaMemcpyHostToDevice, io);
        else  // rendered later on the device (prdpt_job_render_target)
            e = zero_async(c, j->target, sizeof(float4) * (size_t)W * H, io);
    }
    if (e == cudaSuccess && probe.share)
        e = zero_async(c, j->accaff, sizeof(unsigned long long) * 3 * (size_t)R * pix, io);
    if (e == cudaSuccess) e = cudaStreamSynchronize(io);
    if (e != cudaSuccess) {
        c->ev_pool.push_back(j->last);
        block_release(c, base, nullptr);
        delete j;
        return fail(PRDPT_E_CUDA, std::string("job upload: ") + cudaGetErrorString(e));
    }
    InstJob& I = j->inst;
    fill_inst_grad(I, s, o);
    I.base = j->scene_copy;
    I.scenes = j->scenes;
    I.theta = j->theta;
    I.sigma = j->sigma0;
    I.w_out = j->w;
    I.step_dev = j->step;
    I.anneal = d->anneal ? 1 : 0;
    I.total_steps = d->total_steps;
    I.sigma_min = d->sigma_min;
    I.hd = tex ? 1 : 0;
    I.tex_all = j->tex_all;
    I.tex_D = D;
    TraceJob& T = j->trace;
    std::memset(&T, 0, sizeof(T));
    T.hd = tex ? 1 : 0;
    T.scenes = j->scenes;
    T.target = j->target;
    T.partials = j->partials;
    T.done = j->done;
    T.losses = j->losses_d;
    T.w = j->w;
    T.grad_out = j->grad;
    T.loss_out = j->losses;
    T.theta = j->theta;
    T.m = j->m;
    T.v = j->v;
    T.step_dev = j->step;
    T.lr = d->lr;
    T.b1 = d->beta1;
    T.b2 = d->beta2;
    T.eps = d->eps;
    T.W = W;
    T.H = H;
    T.spp = o->spp;
    T.depth = o->depth;
    T.rr_start = o->rr_start;
    T.R = R;
    T.D = D;
    T.antithetic = o->antithetic ? 1 : 0;
    T.bw = bw;
    T.bh = bh;
    T.tiles_x = tiles_x;
    T.tiles = tiles;
    T.n_prims = s->host.n_prims;
    T.n_mats = s->host.n_mats;
    fill_diff(T, s->host, o);
    if (T.diff) {
        T.gpartials = reinterpret_cast<double*>(b + off_gp);
        T.rgrads = reinterpret_cast<double*>(b + off_rg);
    }
    fill_share(T, s->host, o, &I);
    fill_group(T, s->host, o);
    if (T.share) {
        T.share_acc = j->share;
        T.acc_aff = j->accaff;
        afflist_carve(T, j->afflist, pix * o->spp);
        T.var_box = j->varbox;
        I.var_box = j->varbox;
        T.aff_cursor = j->cursor;
        I.aff_cursor = j->cursor;
        T.aff_flags = j->flags;
        I.aff_flags = j->flags;
        T.flag_words = flag_words;
        I.flag_words = flag_words;
        T.aff_tiles = j->aff;
        T.share_ctl = share_ctl;
        j->share_ctl = share_ctl;
        I.share_reset = share_ctl;
    }
    s->jobs++;
    c->jobs.push_back(j);
    *job_out = (int)c->jobs.size() - 1;
    return PRDPT_OK;
}

// Draws of a texture job's step by the high-dimensional kernels (from its sampler setup).
static HdDraws job_hd_draws(const Job* j) {
    const InstJob& I = j->inst;
    HdDraws H{};
    H.D = j->D;
    H.R = j->R;
    H.sampler = I.sampler;
    H.antithetic = I.antithetic;
    H.draw_begin = I.antithetic ? I.pair_begin : 2 * I.pair_begin;
    H.seed = I.seed;
    H.step = I.step;
    H.step_dev = j->step;
    H.theta = j->theta;
    H.sigma = j->sigma0;
    H.anneal = I.anneal;
    H.total_steps = I.total_steps;
    H.sigma_min = I.sigma_min;
    H.c_radial = I.c_radial;
    H.norms = j->norms;
    H.norm_split = hd_norm_split(j->D);
    H.theta_out = j->tex_all;
    H.w_out = j->w;
    return H;
}

static HdGrad job_hd_grad(const Job* j) {
    const TraceJob& T = j->trace;
    HdGrad G{};
    G.D = j->D;
    G.R = j->R;
    G.antithetic = T.antithetic;
    G.w = j->w;
    G.losses = j->losses_d;
    G.grad_out = j->grad;
    G.theta = j->theta;
    G.m = j->m;
    G.v = j->v;
    G.step_dev = j->step;
    G.lr = T.lr;
    G.b1 = T.b1;
    G.b2 = T.b2;
    G.eps = T.eps;
    return G;
}

prdpt_status prdpt_step(prdpt_ctx* c, int32_t job_id, void* stream) {
    if (!c) return fail(PRDPT_E_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);  // the job table, counters and timing events (enqueue only)
    Job* j = get_job(c, job_id);
    if (!j) return fail(PRDPT_E_NOT_FOUND, "unknown job");
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    if (j->tex) PRDPT_CUDA(launch_hd_draws(job_hd_draws(j), st_));  // a1 over the texture
    InstLaunch IL{};
    IL.job0 = j->inst;
    IL.total_blocks = j->R;
    IL.queue_reset = j->queue;
    PRDPT_CUDA(launch_instantiate(IL, st_));
    TraceLaunch TL{};
    TL.job0 = j->trace;
    TL.total_items = int(job_items(j->trace));
    TL.share = j->trace.share;
    TL.group = j->trace.emit ? 2 : (j->trace.gsize > 0 ? 1 : 0);
    TL.diff_nd = diff_slots(j->trace);
    TL.queue = j->queue;
    TL.counters = c->counting ? c->counters : nullptr;
    TL.status = c->status;
    PRDPT_CUDA(timed_trace(c, &TL, 1, &TL, false, st_, j->ctas_per_sm));
    if (j->tex) PRDPT_CUDA(launch_hd_grad(job_hd_grad(j), st_));  // a6 + a7 over the texture
    PRDPT_CUDA(mark_use(j->last, &j->used, &j->captured, st_));  // the job's buffers are in use until here
    return PRDPT_OK;
}

prdpt_status prdpt_step_batch(prdpt_ctx* c, const int32_t* job_ids, int32_t n, void* stream) {
    if (!c || !job_ids || n < 1) return fail(PRDPT_E_INVALID_ARG, "bad job list");
    std::lock_guard<std::mutex> lk(c->mu);
    std::vector<int> ids(job_ids, job_ids + n);
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    if (ids != c->batch_ids && capturing(st_))
        return fail(PRDPT_E_INVALID_ARG, "a packed step captured into a CUDA graph must step the same jobs as the "
                                         "previous packed step: run it once outside the capture first");
    if (ids != c->batch_ids) {
        // path-sharing jobs first (one render-kernel launch with items = pixel blocks), then
        // the rest (items = (render, block)); the order of the jobs does not change results
        std::vector<Job*> order;
        for (int i = 0; i < n; ++i) {
            Job* j = get_job(c, ids[i]);
            if (!j) return fail(PRDPT_E_NOT_FOUND, "unknown job in batch");
            for (int q = 0; q < i; ++q)
                if (ids[q] == ids[i]) return fail(PRDPT_E_INVALID_ARG, "a job appears twice in a batch");
            if (j->trace.diff) return fail(PRDPT_E_INVALID_ARG, "pathwise-estimator jobs step alone (prdpt_step)");
            if (j->tex) return fail(PRDPT_E_INVALID_ARG, "texture jobs step alone (prdpt_step)");
        }
        auto kind = [](const Job* j) {
            return j->trace.share ? 0 : (j->trace.gsize > 0 ? 1 : (j->trace.emit ? 3 : 2));
        };
        for (int pass = 0; pass < 4; ++pass)
            for (int i = 0; i < n; ++i) {
                Job* j = get_job(c, ids[i]);
                if (kind(j) == pass) order.push_back(j);
            }
        std::vector<InstJob> inst(n);
        std::vector<TraceJob> trace(n);
        int blocks = 0, jobs_of[4] = {0, 0, 0, 0}, items_of[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            Job* j = order[i];
            const int kd = kind(j);
            inst[i] = j->inst;
            inst[i].block_begin = blocks;
            blocks += j->R;
            trace[i] = j->trace;
            trace[i].item_begin = items_of[kd];  // items are numbered per launch
            trace[i].fin_begin = blocks - j->R;  // same prefix as the sampler CTAs
            const long long it = job_items(j->trace);
            if (prdpt_status st = check_items((long long)items_of[kd] + it)) return st;
            items_of[kd] += int(it);
            jobs_of[kd]++;
        }
        if ((size_t)n > c->batch_cap) {  // room for at least 64 jobs, doubling (rarely grows)
            const size_t cap = std::max<size_t>(std::max<size_t>(64, 2 * c->batch_cap), (size_t)n);
            PRDPT_CUDA(cudaStreamSynchronize(st_));  // the old arrays may still be in use
            dev_free(c, c->d_inst);
            dev_free(c, c->d_trace);
            c->d_inst = nullptr;
            c->d_trace = nullptr;
            c->batch_cap = 0;
            void* p = nullptr;
            if (prdpt_status st = dev_alloc(c, &p, sizeof(InstJob) * cap)) return st;
            c->d_inst = static_cast<InstJob*>(p);
            if (prdpt_status st = dev_alloc(c, &p, sizeof(TraceJob) * cap)) return st;
            c->d_trace = static_cast<TraceJob*>(p);
            c->batch_cap = cap;
        }
        // Uploaded in stream order (a previous packed step on this stream may still be
        // reading the arrays) from one of two page-locked staging slots, so the call does not
        // wait for the stream: the slot is rewritten only once its previous upload has run.
        const size_t bytes = sizeof(InstJob) * n + sizeof(TraceJob) * n;
        const int k = c->desc_slot;
        c->desc_slot ^= 1;
        if (c->h_desc_ev[k]) PRDPT_CUDA(cudaEventSynchronize(c->h_desc_ev[k]));
        else PRDPT_CUDA(cudaEventCreateWithFlags(&c->h_desc_ev[k], cudaEventDisableTiming));
        if (bytes > c->h_desc_n) {
            const size_t want = std::max<size_t>(bytes, 2 * c->h_desc_n);
            for (int q = 0; q < 2; ++q) {
                if (c->h_desc_ev[q]) PRDPT_CUDA(cudaEventSynchronize(c->h_desc_ev[q]));
                if (c->h_desc[q]) cudaFreeHost(c->h_desc[q]);
                c->h_desc[q] = nullptr;
            }
            c->h_desc_n = 0;
            for (int q = 0; q < 2; ++q) {
                void* h = nullptr;
                PRDPT_CUDA(cudaHostAlloc(&h, want, cudaHostAllocDefault));
                c->h_desc[q] = static_cast<unsigned char*>(h);
            }
            c->h_desc_n = want;
        }
        std::memcpy(c->h_desc[k], inst.data(), sizeof(InstJob) * n);
        std::memcpy(c->h_desc[k] + sizeof(InstJob) * n, trace.data(), sizeof(TraceJob) * n);
        PRDPT_CUDA(cudaMemcpyAsync(c->d_inst, c->h_desc[k], sizeof(InstJob) * n, cudaMemcpyHostToDevice, st_));
        PRDPT_CUDA(cudaMemcpyAsync(c->d_trace, c->h_desc[k] + sizeof(InstJob) * n, sizeof(TraceJob) * n,
                                   cudaMemcpyHostToDevice, st_));
        PRDPT_CUDA(cudaEventRecord(c->h_desc_ev[k], st_));
        c->batch_ids = ids;
        c->batch_blocks = blocks;
        for (int q = 0; q < 4; ++q) {
            c->batch_jobs[q] = jobs_of[q];
            c->batch_items[q] = items_of[q];
        }
    }
    InstLaunch IL{};
    IL.jobs = c->d_inst;
    IL.njobs = n;
    IL.total_blocks = c->batch_blocks;
    IL.queue_reset = c->s_ctl + 2;
    IL.queue_reset2 = c->s_ctl + 3;
    IL.queue_reset3 = c->s_ctl + 8;
    IL.queue_reset4 = c->s_ctl + 9;
    PRDPT_CUDA(launch_instantiate(IL, st_));
    TraceLaunch TL[4] = {};
    int nL = 0, first = 0;
    unsigned* queues[4] = {c->s_ctl + 2, c->s_ctl + 3, c->s_ctl + 8, c->s_ctl + 9};
    for (int kd = 0; kd < 4; ++kd) {  // path-sharing, render-group, per-render, emitter-sharing jobs
        if (c->batch_jobs[kd] > 0) {
            TraceLaunch& T = TL[nL++];
            T.jobs = c->d_trace + first;
            T.njobs = c->batch_jobs[kd];
            T.total_items = c->batch_items[kd];
            T.share = kd == 0 ? 1 : 0;
            T.group = kd == 1 ? 1 : (kd == 3 ? 2 : 0);
            T.queue = queues[kd];
        }
        first += c->batch_jobs[kd];
    }
    for (int i = 0; i < nL; ++i) {
        TL[i].counters = c->counting ? c->counters : nullptr;
        TL[i].status = c->status;
    }
    TraceLaunch FL{};
    FL.jobs = c->d_trace;
    FL.njobs = n;
    FL.fin_total = c->batch_blocks;
    FL.status = c->status;
    PRDPT_CUDA(timed_trace(c, TL, nL, &FL, false, st_, 0));
    for (int i = 0; i < n; ++i) {  // every job's buffers are in use until here
        Job* j = get_job(c, ids[i]);
        PRDPT_CUDA(mark_use(j->last, &j->used, &j->captured, st_));
    }
    return PRDPT_OK;
}

// The context's device status word, read on the context's own stream.
static prdpt_status check_status(prdpt_ctx* c) {
    int st = 0;
    PRDPT_CUDA(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->io));
    PRDPT_CUDA(cudaStreamSynchronize(c->io));
    if (st) return fail(PRDPT_E_DEVICE, "device status word " + std::to_string(st));
    return PRDPT_OK;
}

prdpt_status prdpt_job_read(prdpt_ctx* c, int32_t job_id, float* theta_host, float* grad_host, float* losses_host,
                            int32_t* steps_host) {
    if (!c) return fail(PRDPT_E_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);  // the job may not be released while it is read
    Job* j = get_job(c, job_id);
    if (!j) return fail(PRDPT_E_NOT_FOUND, "unknown job");
    PRDPT_CUDA(cudaSetDevice(c->device));
    if (j->captured) PRDPT_CUDA(cudaDeviceSynchronize());  // graph replays are not tracked
    else if (j->used) PRDPT_CUDA(cudaEventSynchronize(j->last));  // the job's last enqueued work only
    if (prdpt_status st = check_status(c)) return st;
    cudaStream_t io = c->io;
    if (theta_host) PRDPT_CUDA(cudaMemcpyAsync(theta_host, j->theta, sizeof(float) * j->D, cudaMemcpyDeviceToHost, io));
    if (grad_host) PRDPT_CUDA(cudaMemcpyAsync(grad_host, j->grad, sizeof(float) * j->D, cudaMemcpyDeviceToHost, io));
    if (losses_host)
        PRDPT_CUDA(cudaMemcpyAsync(losses_host, j->losses, sizeof(float) * j->R, cudaMemcpyDeviceToHost, io));
    if (steps_host) PRDPT_CUDA(cudaMemcpyAsync(steps_host, j->step, sizeof(int), cudaMemcpyDeviceToHost, io));
    PRDPT_CUDA(cudaStreamSynchronize(io));
    return PRDPT_OK;
}

prdpt_status prdpt_job_release(prdpt_ctx* c, int32_t job_id) {
    if (!c) return fail(PRDPT_E_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    Job* j = get_job(c, job_id);
    if (!j) return fail(PRDPT_E_NOT_FOUND, "unknown job");
    // no synchronisation: the block is kept and reused once the job's last work has
    // completed (after a graph capture that work is not tracked: wait for the device)
    if (j->captured) PRDPT_CUDA(cudaDeviceSynchronize());
    const bool track = j->used && !j->captured;
    block_release(c, j->base, track ? j->last : nullptr);
    if (!track) c->ev_pool.push_back(j->last);
    Scene* s = get_scene(c, j->scene);
    if (s) s->jobs--;
    for (int q : c->batch_ids)
        if (q == job_id) {
            c->batch_ids.clear();
            break;
        }
    delete j;
    c->jobs[job_id] = nullptr;
    return PRDPT_OK;
}

prdpt_status prdpt_job_render_target(prdpt_ctx* c, int32_t job_id, const float* theta_ref_dev, void* stream) {
    if (!c || !theta_ref_dev) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    Job* j = get_job(c, job_id);
    if (!j) return fail(PRDPT_E_NOT_FOUND, "unknown job");
    PRDPT_CUDA(cudaSetDevice(c->device));
    cudaStream_t st_ = static_cast<cudaStream_t>(stream);
    const TraceJob& T = j->trace;
    // one render at theta_ref on stream TARGET, step 0, common path field 0, with the job's
    // image size, spp, depth and Russian roulette, built in the job's own scene slot 0
    InstLaunch IL{};
    std::memset(&IL.job0, 0, sizeof(InstJob));
    IL.job0.base = j->scene_copy;
    IL.job0.scenes = j->scenes;
    IL.job0.theta = theta_ref_dev;
    IL.job0.seed = j->inst.seed;
    IL.job0.step = 0;
    IL.job0.tag = kTagTarget;
    IL.job0.crn = 1;
    IL.job0.render_mode = 1;
    IL.job0.R = 1;
    IL.job0.D = j->D;
    IL.job0.W = T.W;
    IL.job0.H = T.H;
    IL.job0.c_radial = j->inst.c_radial;
    if (j->tex) {  // texture scenes: theta_ref [D] is the texture itself
        IL.job0.hd = 1;
        IL.job0.tex_all = theta_ref_dev;
        IL.job0.tex_D = j->D;
    }
    IL.total_blocks = 1;
    IL.queue_reset = j->queue;
    PRDPT_CUDA(launch_instantiate(IL, st_));
    TraceLaunch TL{};
    TraceJob& J = TL.job0;
    J.scenes = j->scenes;
    J.images = j->target;
    J.W = T.W;
    J.H = T.H;
    J.spp = T.spp;
    J.depth = T.depth;
    J.rr_start = T.rr_start;
    J.R = 1;
    J.D = j->D;
    J.n_prims = T.n_prims;
    J.n_mats = T.n_mats;
    const int px = choose_block(c, 0, 1, T.W, T.H, true);
    tiles_for(px, T.W, T.H, &J.bw, &J.bh, &J.tiles_x, &J.tiles);
    TL.total_items = J.tiles;
    TL.queue = j->queue;
    TL.status = c->status;
    PRDPT_CUDA(launch_trace(TL, true, grid_for(c, TL.total_items, true, 0), st_));
    PRDPT_CUDA(mark_use(j->last, &j->used, &j->captured, st_));
    return PRDPT_OK;
}

prdpt_status prdpt_philox_words(prdpt_ctx* c, uint64_t seed, uint32_t c0_base, uint32_t c1, uint32_t c2, uint32_t c3,
                                int32_t n, uint32_t* words_dev, void* stream) {
    if (!c || !words_dev || n < 0) return fail(PRDPT_E_INVALID_ARG, "bad argument");
    PRDPT_CUDA(cudaSetDevice(c->device));
    PRDPT_CUDA(launch_philox(seed, c0_base, c1, c2, c3, n, words_dev, static_cast<cudaStream_t>(stream)));
    return PRDPT_OK;
}

prdpt_status prdpt_counters_enable(prdpt_ctx* c, int32_t enable) {
    if (!c) return fail(PRDPT_E_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    PRDPT_CUDA(cudaSetDevice(c->device));
    if (enable) PRDPT_CUDA(cudaMemset(c->counters, 0, 8 * sizeof(unsigned long long)));
    c->counting = enable != 0;
    return PRDPT_OK;
}

prdpt_status prdpt_counters_read(prdpt_ctx* c, uint64_t* counts_host) {
    if (!c || !counts_host) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    PRDPT_CUDA(cudaSetDevice(c->device));
    PRDPT_CUDA(cudaDeviceSynchronize());
    PRDPT_CUDA(cudaMemcpy(counts_host, c->counters, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return PRDPT_OK;
}

prdpt_status prdpt_kernel_timing_enable(prdpt_ctx* c, int32_t enable) {
    if (!c) return fail(PRDPT_E_INVALID_ARG, "NULL context");
    std::lock_guard<std::mutex> lk(c->mu);
    c->timing = enable != 0;
    for (auto& ev : c->ev_used) c->ev_free.push_back(ev);
    c->ev_used.clear();
    return PRDPT_OK;
}

prdpt_status prdpt_kernel_timing_read(prdpt_ctx* c, double* total_ms, int64_t* launches) {
    if (!c || !total_ms || !launches) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    PRDPT_CUDA(cudaSetDevice(c->device));
    double tot = 0.0;
    for (auto& ev : c->ev_used) {
        PRDPT_CUDA(cudaEventSynchronize(ev.second));
        float ms = 0.f;
        PRDPT_CUDA(cudaEventElapsedTime(&ms, ev.first, ev.second));
        tot += ms;
    }
    *total_ms = tot;
    *launches = (int64_t)c->ev_used.size();
    for (auto& ev : c->ev_used) c->ev_free.push_back(ev);
    c->ev_used.clear();
    return PRDPT_OK;
}

prdpt_status prdpt_memory_used(prdpt_ctx* c, uint64_t* bytes_out) {
    if (!c || !bytes_out) return fail(PRDPT_E_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(c->mu);
    *bytes_out = c->used;
    return PRDPT_OK;
}

prdpt_status prdpt_fp32_peak_probe(prdpt_ctx* c, int32_t iters, double* tflops_out, double* ms_out) {
    if (!c || !tflops_out || iters < 1) return fail(PRDPT_E_INVALID_ARG, "bad argument");
    std::lock_guard<std::mutex> lk(c->mu);
    PRDPT_CUDA(cudaSetDevice(c->device));
    int per_sm = 0;
    PRDPT_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, c->device));
    const int blocks = c->sms * (per_sm / kBlock > 0 ? per_sm / kBlock : 1);
    void* out = nullptr;
    if (prdpt_status st = dev_alloc(c, &out, sizeof(float) * (size_t)blocks * kBlock)) return st;
    cudaStream_t st_ = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t e = cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_ffma_probe(static_cast<float*>(out), blocks, iters / 8 + 1, st_);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st_);
    if (e == cudaSuccess) e = launch_ffma_probe(static_cast<float*>(out), blocks, iters, st_);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st_);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st_) cudaStreamDestroy(st_);
    dev_free(c, out);
    if (e != cudaSuccess) return fail(PRDPT_E_CUDA, std::string("fp32 peak probe: ") + cudaGetErrorString(e));
    const double flops = double(blocks) * kBlock * double(iters) * ffma_probe_flops_per_thread_iter();
    *tflops_out = flops / (double(ms) * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return PRDPT_OK;
}

prdpt_status prdpt_sync(prdpt_ctx* c, void* stream) {
    if (!c) return fail(PRDPT_E_INVALID_ARG, "NULL context");
    PRDPT_CUDA(cudaSetDevice(c->device));
    PRDPT_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return check_status(c);
}

}  // extern "C"
