// Host runtime of the C ABI declared in include/tilt.h: context, device-memory pool,
// admission, grouped launches, completion tracking.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <fstream>
#include <map>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tilt.h"
#include "tilt_launch.h"

using namespace tilt;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(TILT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

// First-fit allocator over [0, size) with coalescing free blocks.
class Pool {
public:
    void init(size_t size) { free_.clear(); free_[0] = size; size_ = size; used_ = 0; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = align_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

struct Layout {   // byte offsets inside one problem's workspace
    size_t dhat, j, a, e, y, p, mp, zg, bg, vg, tg, img, cay, order, total;
    bool has_cay;
    int smem_svd, minb, jsched, tc_nbuf;
    size_t smem;
};

struct Request {   // one problem as submitted
    const float* img;
    int H, W;
    size_t ld;
    int is_dev;
    int m, n, p;
    double tau0[8];
    Params prm;
    std::vector<float> host_copy;   // owned copy while waiting for admission
};

struct Ticket {
    int slot = -1;               // -1: waiting for admission
    size_t ws_off = 0, ws_bytes = 0;
    Layout lay{};
    int m = 0, n = 0, p = 0;
    double t_submit = 0, t_done = 0;
    int batch = -1;              // owning grouped launch (order-array lifetime)
    int klass = -1;              // its occupancy class in that launch
    Request req;
    bool reaped = false;         // finished; result and planes moved to host, device memory released
    Result res{};
    std::vector<float> A_host, E_host;   // row-major m x n, filled when reaped
};

struct Batch {
    size_t off = 0, bytes = 0;
    int live = 0;
};

}  // namespace

namespace tilt {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace tilt

struct tilt_ctx {
    int device = 0;
    int max_live = 0;
    size_t max_smem = 0;
    cudaStream_t streams[6] = {};   // two sets of three (one per launch class), alternating by batch
    cudaStream_t copy_stream = nullptr;
    bool own_streams = true;        // false: streams[] and copy_stream are the caller's stream
    int next_stream = 0;
    char* pool_base = nullptr;
    Pool pool;
    Problem* probs = nullptr;       // host-mapped
    Problem* probs_dev = nullptr;
    Result* res = nullptr;
    Result* res_dev = nullptr;
    int* done = nullptr;
    int* done_dev = nullptr;
    std::vector<int> free_slots;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::deque<uint64_t> waiting;   // admitted in FIFO order when memory frees up
    std::unordered_map<int, Batch> batches;
    int next_batch = 0;
    uint64_t next_ticket = 1;
    uint64_t launches = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    float* stage = nullptr;         // pinned host staging for plane reads (grows on demand)
    size_t stage_floats = 0;
    StepOut* step_out = nullptr;    // host-mapped
    StepOut* step_out_dev = nullptr;
    cudaEvent_t ev[6] = {};         // start/end events of the last grouped launches (3 classes)
    cudaEvent_t ev_copy[3] = {};    // end of the image uploads of a grouped submission, per stream
    cudaEvent_t ev_rasl[2] = {};    // start/end of the last RASL launch
    int ev_used = 0;
    // persistent workers serving single submissions
    int num_sms = 0;
    int* q_ring = nullptr;          // host-mapped ring of slot indices
    int* q_ring_dev = nullptr;
    int* q_ctl = nullptr;           // host-mapped: [0] tail, [1] stop, [2] cancel
    int* q_ctl_dev = nullptr;
    int* q_head_dev = nullptr;      // device memory
    int published = 0;
    cudaStream_t worker_stream = nullptr;
    cudaEvent_t worker_done = nullptr;
    bool workers_launched = false;
    // autotuned Jacobi group width per size bucket ((R+15)/16, (C+15)/16)
    std::map<std::pair<int, int>, int> tune;
    int force_js = 0;               // non-zero while the autotuner times a candidate schedule
    std::string tune_path;
    int last_cayley = 0;            // accepted Algorithm-2 steps of the last tilt_inner call
};

namespace {

Params to_params(const tilt_params* p) {
    tilt_params d;
    tilt_default_params(&d);
    if (!p) p = &d;
    Params q;
    q.lam = p->lambda;
    q.eps1 = p->eps1;
    q.eps2 = p->eps2;
    q.rho0 = p->rho0;
    q.mu0 = p->mu0;
    q.mu_max = p->mu_max;
    q.eps_svd = p->eps_svd;
    q.outer_tol = p->outer_tol;
    q.max_inner = p->max_inner;
    q.max_outer = p->max_outer;
    q.svd_ws = p->svd_ws;
    return q;
}

bool params_ok(const Params& q) {
    return q.eps1 >= 0 && q.eps2 >= 0 && q.rho0 >= 1.0 && q.mu_max > 0 && q.max_inner >= 1 && q.max_outer >= 1 &&
           q.outer_tol >= 0 && std::isfinite(q.lam) && std::isfinite(q.mu0) && (q.svd_ws == 0 || q.svd_ws == 1);
}

std::pair<int, int> size_bucket(int R, int C) { return {(R + 15) / 16, (C + 15) / 16}; }

// Jacobi schedule for an R x C problem: the autotuned one for its size bucket, else the
// default schedule (block-cyclic ordering).
int jsched_for(const tilt_ctx* ctx, int R, int C) {
    if (ctx->force_js) return ctx->force_js;
    auto it = ctx->tune.find(size_bucket(R, C));
    return it != ctx->tune.end() ? it->second : default_schedule(R, C);
}

bool jsched_valid(int js) {
    const int w = jsched_width(js), o = jsched_order(js);
    return (w == 4 || w == 8 || w == 16) && (o == 0 || o == 1);
}

Layout plan(const tilt_ctx* ctx, int m, int n, int p, int H, int W, bool copy_img, bool cayley) {
    Layout L{};
    const Dims d = make_dims(m, n, p);
    const size_t S = (size_t)d.S * sizeof(float);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += align_up(bytes); return r; };
    L.dhat = take(S);
    L.j = take(S * p);
    L.a = take(S);
    L.e = take(S);
    L.y = take(S);
    L.p = take(S);
    L.mp = take(S);
    L.zg = take((size_t)d.C * d.Cp * sizeof(float));
    // SVD buffers in shared memory as far as they fit next to the stage buffers of the
    // tensor-core products (two buffers where they fit, else one), B first (every dot
    // product reads it), then V, then T (bit 0 B, bit 1 V, bit 2 T); the others in the
    // workspace
    const size_t head = smem_head_bytes();
    const size_t nb = (size_t)d.ldb * d.Cp * sizeof(float), nv = (size_t)d.ldv * d.Cp * sizeof(float);
    const bool tc = use_tc_products(d);
    const size_t st1 = tc ? tc_stage_for(d, 1) : 0, st2 = tc ? tc_stage_for(d, 2) : 0;
    const int places[4] = {7, 3, 1, 0};
    int place = 0, nbuf = 1;
    for (int pi = 0; pi < 4; ++pi) {
        const int pl = places[pi];
        const size_t svd = ((pl & 1) ? nb : 0) + ((pl & 2) ? nv : 0) + ((pl & 4) ? nb : 0);
        if (head + svd + st2 <= ctx->max_smem) { place = pl; nbuf = 2; break; }
        if (head + svd + st1 <= ctx->max_smem) { place = pl; nbuf = 1; break; }
    }
    const size_t svd_bytes = ((place & 1) ? nb : 0) + ((place & 2) ? nv : 0) + ((place & 4) ? nb : 0);
    // the 2-CTA kernel keeps R <= 96 columns in registers and needs <= 100 KB of shared
    // memory per CTA: one stage buffer when two would not fit
    const size_t lim2 = (size_t)100 * 1024;
    L.minb = 1;
    if (place == 7 && d.ldb <= 96) {
        if (head + svd_bytes + st2 <= lim2) { L.minb = 2; nbuf = 2; }
        else if (head + svd_bytes + st1 <= lim2) { L.minb = 2; nbuf = 1; }
    }
    L.smem_svd = place;
    L.tc_nbuf = tc ? nbuf : 0;
    L.smem = head + svd_bytes + (nbuf == 2 ? st2 : st1);
    L.bg = (place & 1) ? 0 : take(nb);
    L.vg = (place & 2) ? 0 : take(nv);
    L.tg = (place & 4) ? 0 : take(nb);
    L.jsched = jsched_for(ctx, d.R, d.C);
    if (place == 0) {
        // B and V in device memory: staged sweeps, their column blocks sharing the stage region
        // with the tensor-core products (the two are never in use at once)
        const int bw = staged_block(d, ctx->max_smem - head);
        if (bw > 0) {
            L.jsched = bw | JSCHED_STAGED;
            L.smem = head + std::max(L.smem - head, jacobi_stage_bytes(d, bw));
        }
    }
    // the C x C SVT coefficients too, where they fit without changing the occupancy class
    // (bit 3); else they stay in the workspace
    {
        const size_t nz = (size_t)d.C * d.Cp * sizeof(float);
        const size_t lim = L.minb == 2 ? lim2 : ctx->max_smem;
        if (place && L.smem + nz <= lim) {
            L.smem_svd |= 8;
            L.smem += nz;
        }
    }
    L.img = copy_img ? take((size_t)H * W * sizeof(float)) : 0;
    L.cay = cayley ? take(cayley_floats(d) * sizeof(float)) : 0;
    L.has_cay = cayley;
    L.order = take(sizeof(int));
    L.total = o;
    return L;
}

int validate(int H, int W, size_t ld, int m, int n, int type, const float* img) {
    if (!img) return fail(TILT_E_INVAL, "null image");
    if (H < 2 || W < 2) return fail(TILT_E_INVAL, "image must be at least 2 x 2 (got %d x %d)", H, W);
    if (ld < (size_t)W) return fail(TILT_E_INVAL, "ld_elems %zu < W %d", ld, W);
    if (m < 2 || n < 2 || m > MAX_SIDE || n > MAX_SIDE)
        return fail(TILT_E_INVAL, "window %d x %d outside 2..%d", m, n, MAX_SIDE);
    if (type != TILT_AFFINE && type != TILT_PROJECTIVE) return fail(TILT_E_INVAL, "bad transform type %d", type);
    return TILT_OK;
}

// Fill the descriptor of an admitted ticket and upload its image (host case).
int prepare(tilt_ctx* ctx, Ticket& t, cudaStream_t st) {
    char* base = ctx->pool_base + t.ws_off;
    Problem& pr = ctx->probs[t.slot];
    const Request& rq = t.req;
    const Layout& L = t.lay;
    memset(&pr, 0, sizeof pr);
    if (rq.is_dev) {
        pr.img = rq.img;
        pr.ld = (long long)rq.ld;
    } else {
        float* dimg = reinterpret_cast<float*>(base + L.img);
        const float* src = rq.host_copy.empty() ? rq.img : rq.host_copy.data();
        const size_t lds = rq.host_copy.empty() ? rq.ld : (size_t)rq.W;
        CUDA_TRY(cudaMemcpy2DAsync(dimg, rq.W * sizeof(float), src, lds * sizeof(float), rq.W * sizeof(float), rq.H,
                                   cudaMemcpyHostToDevice, st));
        pr.img = dimg;
        pr.ld = rq.W;
    }
    pr.H = rq.H;
    pr.W = rq.W;
    pr.m = rq.m;
    pr.n = rq.n;
    pr.p = rq.p;
    pr.ttype = rq.p;
    for (int k = 0; k < 8; ++k) pr.tau[k] = k < rq.p ? rq.tau0[k] : 0.0;
    pr.prm = rq.prm;
    pr.pl.Dhat = reinterpret_cast<float*>(base + L.dhat);
    pr.pl.J = reinterpret_cast<float*>(base + L.j);
    pr.pl.A = reinterpret_cast<float*>(base + L.a);
    pr.pl.E = reinterpret_cast<float*>(base + L.e);
    pr.pl.Y = reinterpret_cast<float*>(base + L.y);
    pr.pl.P = reinterpret_cast<float*>(base + L.p);
    pr.pl.Mp = reinterpret_cast<float*>(base + L.mp);
    pr.pl.Zg = reinterpret_cast<float*>(base + L.zg);
    pr.pl.Bg = (L.smem_svd & 1) ? nullptr : reinterpret_cast<float*>(base + L.bg);
    pr.pl.Vg = (L.smem_svd & 2) ? nullptr : reinterpret_cast<float*>(base + L.vg);
    pr.pl.Tg = (L.smem_svd & 4) ? nullptr : reinterpret_cast<float*>(base + L.tg);
    pr.pl.Cay = L.has_cay ? reinterpret_cast<float*>(base + L.cay) : nullptr;
    pr.smem_svd = L.smem_svd;
    pr.tc_nbuf = L.tc_nbuf;
    pr.jsched = L.jsched;
    pr.res = ctx->res_dev + t.slot;
    pr.done = ctx->done_dev + t.slot;
    pr.cancel = ctx->q_ctl_dev + 2;
    ctx->done[t.slot] = 0;
    return TILT_OK;
}

void release_ticket(tilt_ctx* ctx, uint64_t id) {
    auto it = ctx->tickets.find(id);
    if (it == ctx->tickets.end()) return;
    Ticket& t = it->second;
    if (t.slot >= 0) {                    // (-1: never admitted, -2: already reaped)
        ctx->pool.release(t.ws_off, t.ws_bytes);
        ctx->free_slots.push_back(t.slot);
    }
    if (t.batch >= 0) {
        auto b = ctx->batches.find(t.batch);
        if (b != ctx->batches.end() && --b->second.live == 0) {
            ctx->pool.release(b->second.off, b->second.bytes);
            ctx->batches.erase(b);
        }
    }
    ctx->tickets.erase(it);
}

int fetch_planes(tilt_ctx* ctx, const float* devA, const float* devE, int m, int n, float* A, float* E);

// Move every finished problem's result and planes to host memory and release its device
// memory and slot, so that waiting requests can be admitted whatever order the caller
// polls in.
int reap_finished(tilt_ctx* ctx) {
    for (auto& kv : ctx->tickets) {
        Ticket& t = kv.second;
        if (t.slot < 0 || t.reaped) continue;
        if (!reinterpret_cast<volatile int*>(ctx->done)[t.slot]) continue;
        std::atomic_thread_fence(std::memory_order_acquire);
        if (t.t_done == 0) t.t_done = now_ms();
        t.res = ctx->res[t.slot];
        t.A_host.resize((size_t)t.m * t.n);
        t.E_host.resize((size_t)t.m * t.n);
        int rc = fetch_planes(ctx, ctx->probs[t.slot].pl.A, ctx->probs[t.slot].pl.E, t.m, t.n, t.A_host.data(),
                              t.E_host.data());
        if (rc) return rc;
        ctx->pool.release(t.ws_off, t.ws_bytes);
        ctx->free_slots.push_back(t.slot);
        t.slot = -2;     // finished and reaped
        t.reaped = true;
    }
    return TILT_OK;
}

constexpr int WORKER_IDLE_SPINS = 25000;   // about 50 ms of empty polls before a worker exits

bool workers_running(tilt_ctx* ctx) {
    return ctx->workers_launched && cudaEventQuery(ctx->worker_done) == cudaErrorNotReady;
}

// (Re)launch the persistent workers when none is running.
int ensure_workers(tilt_ctx* ctx) {
    if (workers_running(ctx)) return TILT_OK;
    reinterpret_cast<volatile int*>(ctx->q_ctl)[1] = 0;
    WorkQueue q;
    q.ring = ctx->q_ring_dev;
    q.cap = ctx->max_live;
    q.tail = ctx->q_ctl_dev;
    q.stop = ctx->q_ctl_dev + 1;
    q.cancel = ctx->q_ctl_dev + 2;
    q.head = ctx->q_head_dev;
    q.idle_spins = WORKER_IDLE_SPINS;
    CUDA_TRY(launch_workers(ctx->probs_dev, q, ctx->num_sms, ctx->max_smem, ctx->worker_stream));
    CUDA_TRY(cudaEventRecord(ctx->worker_done, ctx->worker_stream));
    ctx->workers_launched = true;
    ctx->launches++;
    return TILT_OK;
}

// Hand an admitted ticket to the workers: its image is on the device and its descriptor
// written before the slot is published (release order), then make sure workers run.
int publish(tilt_ctx* ctx, Ticket& t) {
    int rc = prepare(ctx, t, ctx->copy_stream);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(ctx->copy_stream));
    ctx->q_ring[ctx->published % ctx->max_live] = t.slot;
    std::atomic_thread_fence(std::memory_order_release);
    reinterpret_cast<volatile int*>(ctx->q_ctl)[0] = ++ctx->published;
    return ensure_workers(ctx);
}

// Admit as many waiting requests as fit, each as its own launch.
int admit_waiting(tilt_ctx* ctx) {
    if (!ctx->waiting.empty()) {
        int rc = reap_finished(ctx);
        if (rc) return rc;
    }
    while (!ctx->waiting.empty() && !ctx->free_slots.empty()) {
        const uint64_t id = ctx->waiting.front();
        auto it = ctx->tickets.find(id);
        if (it == ctx->tickets.end()) { ctx->waiting.pop_front(); continue; }
        Ticket& t = it->second;
        size_t off;
        if (!ctx->pool.alloc(t.ws_bytes, &off)) break;
        ctx->waiting.pop_front();
        t.ws_off = off;
        t.slot = ctx->free_slots.back();
        ctx->free_slots.pop_back();
        int rc = publish(ctx, t);
        if (rc) return rc;
        t.req.host_copy.clear();
        t.req.host_copy.shrink_to_fit();
    }
    return TILT_OK;
}

// Grouped-launch class of a problem: 0 two CTAs per SM (all SVD buffers in shared memory),
// 1 one CTA per SM (shared memory as far as it holds them, SIMT products), 2 one CTA per SM
// with the tensor-core products (short side >= TC_MIN_C) or with no SVD buffer in shared
// memory.
int launch_class_of(const Layout& L) {
    if (L.tc_nbuf > 0 || !L.smem_svd || L.has_cay) return 2;
    return L.minb == 2 ? 0 : 1;
}

void fill_result(const Result& r, const Ticket& t, tilt_result* out) {
    memset(out, 0, sizeof *out);
    out->status = r.status;
    out->p = r.p;
    for (int k = 0; k < 8; ++k) out->tau[k] = r.tau[k];
    out->objective = r.objective;
    out->lambda = r.lambda;
    out->rank_A = r.rank_A;
    out->outer_iters = r.outer_iters;
    out->inner_iters = r.inner_iters;
    out->svd_sweeps = r.svd_sweeps;
    out->svd_warm = r.svd_warm;
    out->oob_pixels = r.oob_pixels;
    out->kkt_residual = r.kkt_residual;
    out->latency_ms = (float)(t.t_done - t.t_submit);
    out->phase_cycles[0] = r.cyc_warp;
    out->phase_cycles[1] = r.cyc_svd;
    out->phase_cycles[2] = r.cyc_recon;
    out->phase_cycles[3] = r.cyc_elem;
    out->phase_cycles[4] = r.cyc_other;
    out->launch_class = t.batch < 0 ? -1 : t.klass;
    out->svd_reorth = r.svd_reorth;
    out->svd_cayley = r.svd_cayley;
}

// Copy the device planes A and E (long-side-contiguous) to host m x n row-major arrays (either
// may be NULL): both copies go through one pinned staging buffer and one synchronisation.
int fetch_planes(tilt_ctx* ctx, const float* devA, const float* devE, int m, int n, float* A, float* E) {
    const Dims d = make_dims(m, n, 0);
    const size_t S = (size_t)d.S;
    if (ctx->stage_floats < 2 * S) {
        if (ctx->stage) CUDA_TRY(cudaFreeHost(ctx->stage));
        ctx->stage = nullptr;
        ctx->stage_floats = 0;
        CUDA_TRY(cudaHostAlloc(&ctx->stage, sizeof(float) * 2 * S, cudaHostAllocDefault));
        ctx->stage_floats = 2 * S;
    }
    if (A) CUDA_TRY(cudaMemcpyAsync(ctx->stage, devA, sizeof(float) * S, cudaMemcpyDeviceToHost, ctx->copy_stream));
    if (E) CUDA_TRY(cudaMemcpyAsync(ctx->stage + S, devE, sizeof(float) * S, cudaMemcpyDeviceToHost, ctx->copy_stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->copy_stream));
    for (int h = 0; h < 2; ++h) {
        float* host = h ? E : A;
        if (!host) continue;
        const float* tmp = ctx->stage + (h ? S : 0);
        if (d.colmajor) {
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < m; ++i) host[(size_t)i * n + j] = tmp[(size_t)j * m + i];
        } else {
            memcpy(host, tmp, sizeof(float) * S);
        }
    }
    return TILT_OK;
}

int ensure_scratch(tilt_ctx* ctx, size_t bytes) {
    if (ctx->scratch_bytes >= bytes) return TILT_OK;
    CUDA_TRY(cudaSetDevice(ctx->device));
    if (ctx->scratch) {
        CUDA_TRY(cudaStreamSynchronize(ctx->streams[0]));
        CUDA_TRY(cudaFree(ctx->scratch));
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    CUDA_TRY(cudaMalloc(&ctx->scratch, bytes));
    ctx->scratch_bytes = bytes;
    return TILT_OK;
}

// Jacobi schedule and dynamic shared memory of a step entry point: the SVD buffers in shared
// memory when svd + head fits (default round-robin schedule), else in device memory with
// staged sweeps, whose blocks share the stage region with the tensor-core products.
void step_plan(const tilt_ctx* ctx, const Dims& d, size_t svd, size_t head_tc, int* smem_svd, int* jsched,
               size_t* smem) {
    const size_t head = smem_head_bytes();
    *smem_svd = (svd + head_tc <= ctx->max_smem) ? 1 : 0;
    *jsched = default_group_width(d.R, d.C);
    *smem = *smem_svd ? svd + head_tc : head_tc;
    if (!*smem_svd) {
        const int bw = staged_block(d, ctx->max_smem - head);
        if (bw > 0) {
            *jsched = bw | JSCHED_STAGED;
            *smem = head + std::max(head_tc - head, jacobi_stage_bytes(d, bw));
        }
    }
}

int run_step(tilt_ctx* ctx) {
    ctx->launches++;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(ctx->streams[0]));
    return TILT_OK;
}

}  // namespace

extern "C" {

void tilt_default_params(tilt_params* p) {
    if (!p) return;
    p->lambda = -1.0;
    p->eps1 = 1e-5;
    p->eps2 = 0.1;
    p->rho0 = 1.5;
    p->mu0 = -1.0;
    p->mu_max = 1e10;
    p->eps_svd = -1.0;      // the Jacobi warm start is exact: use it whenever V is valid
    p->max_inner = 500;
    p->max_outer = 10;
    p->outer_tol = 1e-2;
    p->svd_ws = 0;
}

const char* tilt_last_error(tilt_ctx*) { return g_err.c_str(); }

uint64_t tilt_kernel_launches(tilt_ctx* ctx) { return ctx ? ctx->launches : 0; }

int tilt_create(const tilt_config* cfg, tilt_ctx** out) {
    if (!cfg || !out) return fail(TILT_E_INVAL, "null argument");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (cfg->device < 0 || cfg->device >= ndev) return fail(TILT_E_INVAL, "device %d of %d", cfg->device, ndev);
    CUDA_TRY(cudaSetDevice(cfg->device));
    tilt_ctx* ctx = new tilt_ctx();
    ctx->device = cfg->device;
    ctx->max_live = cfg->max_live > 0 ? cfg->max_live : 65536;
    int optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cfg->device));
    ctx->max_smem = (size_t)optin - 2048;    // static shared memory of the solver kernel
    CUDA_TRY(configure_kernels(ctx->max_smem));
    CUDA_TRY(configure_rasl_kernels(ctx->max_smem));
    if (cfg->cuda_stream) {
        // the caller's stream carries every grouped launch, copy and step of this context
        ctx->own_streams = false;
        for (auto& s : ctx->streams) s = reinterpret_cast<cudaStream_t>(cfg->cuda_stream);
        ctx->copy_stream = reinterpret_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
        for (auto& s : ctx->streams) CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    }
    size_t freeb = 0, totalb = 0;
    CUDA_TRY(cudaMemGetInfo(&freeb, &totalb));
    size_t budget = cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : freeb / 4;
    budget = std::min<size_t>(budget, freeb > (size_t(1) << 30) ? freeb - (size_t(1) << 30) : freeb / 2);
    budget &= ~(ALIGN - 1);
    CUDA_TRY(cudaMalloc(&ctx->pool_base, budget));
    ctx->pool.init(budget);
    const size_t ns = (size_t)ctx->max_live;
    CUDA_TRY(cudaHostAlloc(&ctx->probs, ns * sizeof(Problem), cudaHostAllocMapped));
    CUDA_TRY(cudaHostAlloc(&ctx->res, ns * sizeof(Result), cudaHostAllocMapped));
    CUDA_TRY(cudaHostAlloc(&ctx->done, ns * sizeof(int), cudaHostAllocMapped));
    CUDA_TRY(cudaHostAlloc(&ctx->step_out, sizeof(StepOut), cudaHostAllocMapped));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&ctx->probs_dev, ctx->probs, 0));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&ctx->res_dev, ctx->res, 0));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&ctx->done_dev, ctx->done, 0));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&ctx->step_out_dev, ctx->step_out, 0));
    for (auto& e : ctx->ev) CUDA_TRY(cudaEventCreate(&e));
    for (auto& e : ctx->ev_copy) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (auto& e : ctx->ev_rasl) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, cfg->device));
    CUDA_TRY(cudaHostAlloc(&ctx->q_ring, ns * sizeof(int), cudaHostAllocMapped));
    CUDA_TRY(cudaHostAlloc(&ctx->q_ctl, 4 * sizeof(int), cudaHostAllocMapped));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&ctx->q_ring_dev, ctx->q_ring, 0));
    CUDA_TRY(cudaHostGetDevicePointer((void**)&ctx->q_ctl_dev, ctx->q_ctl, 0));
    ctx->q_ctl[0] = ctx->q_ctl[1] = ctx->q_ctl[2] = ctx->q_ctl[3] = 0;
    if (cfg->autotune_cache) {
        ctx->tune_path = cfg->autotune_cache;
        std::ifstream f(ctx->tune_path);
        int rb, cb, js;
        while (f >> rb >> cb >> js)
            if (jsched_valid(js)) ctx->tune[{rb, cb}] = js;
    }
    CUDA_TRY(cudaMalloc(&ctx->q_head_dev, sizeof(int)));
    CUDA_TRY(cudaMemset(ctx->q_head_dev, 0, sizeof(int)));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->worker_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&ctx->worker_done, cudaEventDisableTiming));
    memset(ctx->done, 0, ns * sizeof(int));
    ctx->free_slots.reserve(ns);
    for (int s = (int)ns - 1; s >= 0; --s) ctx->free_slots.push_back(s);
    *out = ctx;
    return TILT_OK;
}

int tilt_submit(tilt_ctx* ctx, const float* img, int H, int W, size_t ld_elems, int is_device_ptr, int m, int n,
                const double* tau0, tilt_transform type, const tilt_params* params, uint64_t* ticket_out) {
    if (!ctx || !tau0 || !ticket_out) return fail(TILT_E_INVAL, "null argument");
    int rc = validate(H, W, ld_elems, m, n, (int)type, img);
    if (rc) return rc;
    Ticket t;
    t.req.img = img;
    t.req.H = H;
    t.req.W = W;
    t.req.ld = ld_elems;
    t.req.is_dev = is_device_ptr ? 1 : 0;
    t.req.m = m;
    t.req.n = n;
    t.req.p = (int)type;
    for (int k = 0; k < 8; ++k) t.req.tau0[k] = k < (int)type ? tau0[k] : 0.0;
    for (int k = 0; k < (int)type; ++k)
        if (!std::isfinite(tau0[k])) return fail(TILT_E_INVAL, "non-finite tau0");
    t.req.prm = to_params(params);
    if (!params_ok(t.req.prm)) return fail(TILT_E_INVAL, "parameters out of range");
    t.lay = plan(ctx, m, n, (int)type, H, W, !is_device_ptr, t.req.prm.svd_ws == 1);
    t.ws_bytes = t.lay.total;
    if (t.ws_bytes > ctx->pool.size())
        return fail(TILT_E_NOMEM, "problem needs %zu bytes, budget is %zu", t.ws_bytes, ctx->pool.size());
    if ((int)ctx->tickets.size() >= ctx->max_live * 4) return fail(TILT_E_BUSY, "too many outstanding tickets");
    t.m = m;
    t.n = n;
    t.p = (int)type;
    t.t_submit = now_ms();
    const uint64_t id = ctx->next_ticket++;
    size_t off;
    const bool fits = ctx->waiting.empty() && !ctx->free_slots.empty() && ctx->pool.alloc(t.ws_bytes, &off);
    if (!fits) {
        if (!is_device_ptr) {   // keep a private copy: the caller may reuse img at once
            t.req.host_copy.resize((size_t)H * W);
            for (int y = 0; y < H; ++y) memcpy(&t.req.host_copy[(size_t)y * W], img + (size_t)y * ld_elems, sizeof(float) * W);
        }
        ctx->tickets.emplace(id, std::move(t));
        ctx->waiting.push_back(id);
        *ticket_out = id;
        return TILT_OK;
    }
    t.ws_off = off;
    t.slot = ctx->free_slots.back();
    ctx->free_slots.pop_back();
    auto& tk = ctx->tickets.emplace(id, std::move(t)).first->second;
    rc = publish(ctx, tk);
    if (rc) { release_ticket(ctx, id); return rc; }
    *ticket_out = id;
    return TILT_OK;
}

int tilt_submit_batch(tilt_ctx* ctx, int count, const tilt_problem* probs, int is_device_ptr, const tilt_params* params,
                      uint64_t* tickets_out) {
    if (!ctx || count < 0 || (count && (!probs || !tickets_out))) return fail(TILT_E_INVAL, "bad arguments");
    if (count == 0) return TILT_OK;
    const Params prm = to_params(params);
    if (!params_ok(prm)) return fail(TILT_E_INVAL, "parameters out of range");
    if ((int)ctx->free_slots.size() < count) return fail(TILT_E_BUSY, "%d free slots, %d problems", (int)ctx->free_slots.size(), count);
    std::vector<Ticket> ts((size_t)count);
    size_t total = 0;
    for (int q = 0; q < count; ++q) {
        const tilt_problem& pb = probs[q];
        int rc = validate(pb.H, pb.W, pb.ld_elems, pb.m, pb.n, pb.type, pb.img);
        if (rc) return fail(rc, "problem %d: %s", q, g_err.c_str());
        Ticket& t = ts[q];
        t.req.img = pb.img;
        t.req.H = pb.H;
        t.req.W = pb.W;
        t.req.ld = pb.ld_elems;
        t.req.is_dev = is_device_ptr ? 1 : 0;
        t.req.m = pb.m;
        t.req.n = pb.n;
        t.req.p = pb.type;
        for (int k = 0; k < 8; ++k) t.req.tau0[k] = k < pb.type ? pb.tau0[k] : 0.0;
        t.req.prm = prm;
        t.lay = plan(ctx, pb.m, pb.n, pb.type, pb.H, pb.W, !is_device_ptr, prm.svd_ws == 1);
        t.ws_bytes = t.lay.total;
        t.m = pb.m;
        t.n = pb.n;
        t.p = pb.type;
        if (t.ws_bytes > ctx->pool.size()) return fail(TILT_E_NOMEM, "problem %d needs %zu bytes", q, t.ws_bytes);
        total += align_up(t.ws_bytes);
    }
    // grouped launches: one per occupancy class, largest problems first
    std::vector<int> idx(count);
    for (int q = 0; q < count; ++q) idx[q] = q;
    std::vector<int> klass(count);
    for (int q = 0; q < count; ++q) klass[q] = launch_class_of(ts[q].lay);
    // a batch that does not fill the SMs gains nothing from two CTAs per SM: give every problem
    // the 128-register kernel (no spills, longer register-resident columns).  Not for the
    // autotuner's timing batches, which must run each bucket in the kernel it will use.
    if (count <= ctx->num_sms && !ctx->force_js)
        for (int q = 0; q < count; ++q)
            if (klass[q] == 0) klass[q] = 1;
    auto cls = [&](int q) { return klass[q]; };
    auto cost = [&](int q) {
        const Dims d = make_dims(ts[q].m, ts[q].n, ts[q].p);
        return (double)d.R * d.C * d.C;
    };
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        if (cls(a) != cls(b)) return cls(a) < cls(b);
        return cost(a) > cost(b);
    });
    const size_t order_bytes = align_up(sizeof(int) * count);
    size_t boff;
    if (!ctx->pool.alloc(order_bytes, &boff)) return fail(TILT_E_BUSY, "device memory for the batch order is in use");
    std::vector<size_t> offs(count);
    int got = 0;
    for (; got < count; ++got) {
        if (!ctx->pool.alloc(ts[got].ws_bytes, &offs[got])) break;
    }
    if (got < count) {
        for (int q = 0; q < got; ++q) ctx->pool.release(offs[q], ts[q].ws_bytes);
        ctx->pool.release(boff, order_bytes);
        return fail(TILT_E_BUSY, "batch needs %zu bytes; %zu of %zu in use", total, ctx->pool.used(), ctx->pool.size());
    }
    const int bid = ctx->next_batch++;
    ctx->batches[bid] = Batch{boff, order_bytes, count};
    const double t0 = now_ms();
    std::vector<uint64_t> ids(count);
    std::vector<int> order(count);
    for (int q = 0; q < count; ++q) {
        Ticket& t = ts[q];
        t.ws_off = offs[q];
        t.slot = ctx->free_slots.back();
        ctx->free_slots.pop_back();
        t.batch = bid;
        t.klass = klass[q];
        t.t_submit = t0;
        ids[q] = ctx->next_ticket++;
    }
    // consecutive batches take alternate stream sets, so that a batch's launches start on the
    // SMs the previous batch frees while its longest solves still run
    const int sset = 3 * (bid & 1);
    cudaStream_t st[3] = {ctx->streams[sset], ctx->streams[sset + 1], ctx->streams[sset + 2]};
    for (int q = 0; q < count; ++q) {
        Ticket& t = ctx->tickets.emplace(ids[q], std::move(ts[q])).first->second;
        int rc = prepare(ctx, t, st[cls(q)]);
        if (rc) return rc;
        order[q] = t.slot;
        tickets_out[q] = ids[q];
    }
    // host images: mark the end of the uploads on each stream; the call waits for them (not
    // for the solves) before returning, so the caller may reuse its buffers at once even
    // when they are pinned (the CUDA runtime stages pageable sources before it returns)
    if (!is_device_ptr)
        for (int c = 0; c < 3; ++c) CUDA_TRY(cudaEventRecord(ctx->ev_copy[c], st[c]));
    std::vector<int> ord_slots(count);
    for (int q = 0; q < count; ++q) ord_slots[q] = order[idx[q]];
    int* ord_dev = reinterpret_cast<int*>(ctx->pool_base + boff);
    // the order array is copied once (pageable source: staged before the call returns)
    CUDA_TRY(cudaMemcpyAsync(ord_dev, ord_slots.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st[0]));
    CUDA_TRY(cudaStreamSynchronize(st[0]));
    int start = 0, nev = 0;
    while (start < count) {
        const int c = cls(idx[start]);
        int end = start;
        size_t smem = 0;
        while (end < count && cls(idx[end]) == c) {
            smem = std::max(smem, ctx->tickets[ids[idx[end]]].lay.smem);
            ++end;
        }
        const int minb = (c == 0) ? 2 : 1;
        if (nev < 3) CUDA_TRY(cudaEventRecord(ctx->ev[2 * nev], st[c]));
        CUDA_TRY(launch_solver(ctx->probs_dev, ord_dev + start, end - start, minb, c == 2, smem, st[c]));
        if (nev < 3) { CUDA_TRY(cudaEventRecord(ctx->ev[2 * nev + 1], st[c])); ++nev; }
        ctx->launches++;
        start = end;
    }
    ctx->ev_used = nev;
    if (!is_device_ptr)
        for (int c = 0; c < 3; ++c) CUDA_TRY(cudaEventSynchronize(ctx->ev_copy[c]));
    return TILT_OK;
}

int tilt_batch_kernel_ms(tilt_ctx* ctx, float* ms_out, int cap) {
    if (!ctx || (cap > 0 && !ms_out)) return fail(TILT_E_INVAL, "bad arguments");
    const double t_end = now_ms() + 600000.0;
    int n = 0;
    for (int q = 0; q < ctx->ev_used && n < cap; ++q) {
        while (cudaEventQuery(ctx->ev[2 * q + 1]) == cudaErrorNotReady) {
            if (now_ms() > t_end) return fail(TILT_E_TIMEOUT, "grouped launch still running");
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev[2 * q], ctx->ev[2 * q + 1]));
        ms_out[n++] = ms;
    }
    return n;
}

int tilt_poll(tilt_ctx* ctx, uint64_t ticket, tilt_result* out, float* A_out, float* E_out) {
    if (!ctx) return fail(TILT_E_INVAL, "null context");
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(TILT_E_NOTFOUND, "ticket %llu", (unsigned long long)ticket);
    Ticket& t = it->second;
    if (t.reaped) {
        if (A_out) memcpy(A_out, t.A_host.data(), sizeof(float) * t.A_host.size());
        if (E_out) memcpy(E_out, t.E_host.data(), sizeof(float) * t.E_host.size());
        if (out) fill_result(t.res, t, out);
        release_ticket(ctx, ticket);
        return admit_waiting(ctx);
    }
    if (t.slot < 0) {
        int rc = admit_waiting(ctx);
        if (rc) return rc;
        return TILT_PENDING;
    }
    if (!reinterpret_cast<volatile int*>(ctx->done)[t.slot]) {
        cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) return fail(TILT_E_CUDA, "CUDA error while waiting: %s", cudaGetErrorString(e));
        // a worker only exits when the queue looked empty; if all have exited while this
        // queued problem is unfinished, it was published after their last look
        if (t.batch < 0 && ctx->workers_launched && !workers_running(ctx) &&
            !reinterpret_cast<volatile int*>(ctx->done)[t.slot]) {
            int rc = ensure_workers(ctx);
            if (rc) return rc;
        }
        return TILT_PENDING;
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    if (t.t_done == 0) t.t_done = now_ms();
    const Result r = ctx->res[t.slot];
    if (A_out || E_out) {
        int rc = fetch_planes(ctx, ctx->probs[t.slot].pl.A, ctx->probs[t.slot].pl.E, t.m, t.n, A_out, E_out);
        if (rc) return rc;
    }
    if (out) fill_result(r, t, out);
    release_ticket(ctx, ticket);
    return admit_waiting(ctx);
}

int tilt_best_of(const tilt_result* results, int n_groups, int starts, int* best_out) {
    if (!results || !best_out || n_groups < 0 || starts < 1) return fail(TILT_E_INVAL, "bad arguments");
    for (int g = 0; g < n_groups; ++g) {
        int best = -1;
        double bo = 0.0;
        for (int s = 0; s < starts; ++s) {
            const tilt_result& r = results[(size_t)g * starts + s];
            if (r.status < 0 || !std::isfinite(r.objective)) continue;
            if (best < 0 || r.objective < bo) {
                best = s;
                bo = r.objective;
            }
        }
        best_out[g] = best;
    }
    return TILT_OK;
}

int tilt_autotune(tilt_ctx* ctx, const int* shapes, int count, tilt_transform type, int* chosen_out) {
    if (!ctx || (count && !shapes) || count < 0) return fail(TILT_E_INVAL, "bad arguments");
    if (type != TILT_AFFINE && type != TILT_PROJECTIVE) return fail(TILT_E_INVAL, "bad type");
    CUDA_TRY(cudaSetDevice(ctx->device));
    bool changed = false;
    for (int s = 0; s < count; ++s) {
        const int m = shapes[2 * s], n = shapes[2 * s + 1];
        if (m < 2 || n < 2 || m > MAX_SIDE || n > MAX_SIDE) return fail(TILT_E_INVAL, "shape %d x %d", m, n);
        const Dims d = make_dims(m, n, (int)type);
        const auto key = size_bucket(d.R, d.C);
        if (!ctx->tune.count(key)) {
            // a smooth synthetic texture with noise, rotated slightly: one outer step of 30
            // inner iterations on one problem per SM for every candidate schedule
            const int H = m + 16, W = n + 16;
            std::vector<float> img((size_t)H * W);
            uint32_t st = 12345u;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    st = st * 1664525u + 1013904223u;
                    img[(size_t)y * W + x] = 0.5f + 0.3f * std::sin(0.37f * x) * std::cos(0.23f * y) +
                                             0.05f * ((st >> 8) * (1.0f / 16777216.0f) - 0.5f);
                }
            float* dimg = nullptr;
            CUDA_TRY(cudaMalloc(&dimg, img.size() * sizeof(float)));
            CUDA_TRY(cudaMemcpy(dimg, img.data(), img.size() * sizeof(float), cudaMemcpyHostToDevice));
            const int K = ctx->num_sms;
            std::vector<tilt_problem> probs((size_t)K);
            for (auto& pb : probs) {
                memset(&pb, 0, sizeof pb);
                pb.img = dimg;
                pb.H = H;
                pb.W = W;
                pb.ld_elems = W;
                pb.m = m;
                pb.n = n;
                pb.type = (int)type;
                const double th = 0.05;
                pb.tau0[0] = std::cos(th); pb.tau0[1] = -std::sin(th); pb.tau0[2] = 0.5 * (W - 1);
                pb.tau0[3] = std::sin(th); pb.tau0[4] = std::cos(th); pb.tau0[5] = 0.5 * (H - 1);
            }
            tilt_params prm;
            tilt_default_params(&prm);
            prm.max_outer = 1;
            prm.max_inner = 30;      // long enough that warm-started SVDs dominate, as in real solves
            prm.eps1 = 0.0;
            int best = default_schedule(d.R, d.C);
            float best_ms = 1e30f;
            const int widths[3] = {4, 8, 16};
            float cand_ms[6];
            for (float& v : cand_ms) v = 1e30f;
            // two passes over the candidates, each keeping its faster run (launch-to-launch noise
            // is a few per cent, about the gap between neighbouring schedules)
            for (int c12 = 0; c12 < 12; ++c12) {
                const int c = c12 % 6;
                const int gw = widths[c % 3], js = gw | (c >= 3 ? JSCHED_BLOCK : 0);
                if ((d.C + 1) / 2 > 8 * (NT / gw)) continue;    // more than 8 pairs per group per round
                ctx->force_js = js;
                std::vector<uint64_t> tk((size_t)K);
                int rc = tilt_submit_batch(ctx, K, probs.data(), 1, &prm, tk.data());
                ctx->force_js = 0;
                if (rc) { cudaFree(dimg); return rc; }
                float ms[3];
                const int nl = tilt_batch_kernel_ms(ctx, ms, 3);
                for (uint64_t t : tk) {
                    rc = tilt_wait(ctx, t, 600000, nullptr, nullptr, nullptr);
                    if (rc) { cudaFree(dimg); return rc; }
                }
                if (nl <= 0) { cudaFree(dimg); return nl < 0 ? nl : fail(TILT_E_CUDA, "no timing"); }
                float tot = 0.f;
                for (int q = 0; q < nl; ++q) tot = std::max(tot, ms[q]);
                cand_ms[c] = std::min(cand_ms[c], tot);
                if (c12 >= 6 && cand_ms[c] < best_ms) { best_ms = cand_ms[c]; best = js; }
            }
            CUDA_TRY(cudaFree(dimg));
            ctx->tune[key] = best;
            changed = true;
        }
        if (chosen_out) chosen_out[s] = ctx->tune[key];
    }
    if (changed && !ctx->tune_path.empty()) {
        std::ofstream f(ctx->tune_path, std::ios::trunc);
        for (const auto& kv : ctx->tune) f << kv.first.first << ' ' << kv.first.second << ' ' << kv.second << '\n';
    }
    return TILT_OK;
}

int tilt_wait(tilt_ctx* ctx, uint64_t ticket, int timeout_ms, tilt_result* out, float* A_out, float* E_out) {
    const double t_end = now_ms() + (timeout_ms < 0 ? 60000.0 : (double)timeout_ms);
    for (;;) {
        int rc = tilt_poll(ctx, ticket, out, A_out, E_out);
        if (rc != TILT_PENDING) return rc;
        if (now_ms() > t_end) return fail(TILT_E_TIMEOUT, "ticket %llu still running", (unsigned long long)ticket);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int tilt_destroy(tilt_ctx* ctx) {
    if (!ctx) return TILT_OK;
    cudaSetDevice(ctx->device);
    // running solves stop after their current inner iteration (status -4), queued ones are
    // retired unsolved, and the workers exit
    reinterpret_cast<volatile int*>(ctx->q_ctl)[2] = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    reinterpret_cast<volatile int*>(ctx->q_ctl)[1] = 1;
    const double t_end = now_ms() + 120000.0;
    for (;;) {
        bool busy = false;
        for (auto s : ctx->streams) busy = busy || cudaStreamQuery(s) == cudaErrorNotReady;
        busy = busy || cudaStreamQuery(ctx->copy_stream) == cudaErrorNotReady;
        busy = busy || cudaStreamQuery(ctx->worker_stream) == cudaErrorNotReady;
        if (!busy) break;
        if (now_ms() > t_end) return fail(TILT_E_TIMEOUT, "work still running after 120 s; context leaked");
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    if (ctx->own_streams) {
        for (auto s : ctx->streams) cudaStreamDestroy(s);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (auto e : ctx->ev) cudaEventDestroy(e);
    for (auto e : ctx->ev_copy) cudaEventDestroy(e);
    for (auto e : ctx->ev_rasl) cudaEventDestroy(e);
    cudaEventDestroy(ctx->worker_done);
    cudaStreamDestroy(ctx->worker_stream);
    cudaFree(ctx->q_head_dev);
    cudaFreeHost(ctx->q_ring);
    cudaFreeHost(ctx->q_ctl);
    cudaFree(ctx->pool_base);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->stage) cudaFreeHost(ctx->stage);
    cudaFreeHost(ctx->probs);
    cudaFreeHost(ctx->res);
    cudaFreeHost(ctx->done);
    cudaFreeHost(ctx->step_out);
    delete ctx;
    return TILT_OK;
}

// ------------------------------------------------------------------------------ step entry points
int tilt_warp_jacobian(tilt_ctx* ctx, const float* img_dev, int H, int W, size_t ld, int m, int n, const double* tau,
                       tilt_transform type, float* Dhat_dev, float* J_dev, double* norm_out, int* oob_out) {
    if (!ctx || !tau || !Dhat_dev || !J_dev) return fail(TILT_E_INVAL, "null argument");
    int rc = validate(H, W, ld, m, n, (int)type, img_dev);
    if (rc) return rc;
    WarpArgs a{};
    a.img = img_dev;
    a.ld = (long long)ld;
    a.H = H; a.W = W; a.m = m; a.n = n; a.ttype = (int)type;
    for (int k = 0; k < PMAX; ++k) a.tau[k] = k < (int)type ? tau[k] : 0.0;
    a.Dhat = Dhat_dev;
    a.J = J_dev;
    a.out = ctx->step_out_dev;
    CUDA_TRY(launch_warp_step(a, ctx->streams[0]));
    rc = run_step(ctx);
    if (rc) return rc;
    if (norm_out) *norm_out = ctx->step_out->norm;
    if (oob_out) *oob_out = ctx->step_out->oob;
    return TILT_OK;
}

int tilt_gram(tilt_ctx* ctx, const float* J_dev, int m, int n, const double* tau, tilt_transform type, double* Q_out,
              double* G_out, double* Ginv_out) {
    if (!ctx || !tau || !J_dev) return fail(TILT_E_INVAL, "null argument");
    if (m < 2 || n < 2 || m > MAX_SIDE || n > MAX_SIDE) return fail(TILT_E_INVAL, "window %d x %d", m, n);
    if (type != TILT_AFFINE && type != TILT_PROJECTIVE) return fail(TILT_E_INVAL, "bad type");
    int rc = ensure_scratch(ctx, sizeof(float) * (size_t)m * n);
    if (rc) return rc;
    CUDA_TRY(cudaMemsetAsync(ctx->scratch, 0, sizeof(float) * (size_t)m * n, ctx->streams[0]));
    GramArgs a{};
    a.J = J_dev;
    a.Dhat = reinterpret_cast<const float*>(ctx->scratch);
    a.m = m; a.n = n; a.ttype = (int)type;
    for (int k = 0; k < PMAX; ++k) a.tau[k] = k < (int)type ? tau[k] : 0.0;
    a.out = ctx->step_out_dev;
    CUDA_TRY(launch_gram_step(a, ctx->streams[0]));
    rc = run_step(ctx);
    if (rc) return rc;
    const int p = (int)type;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < p; ++c)
            if (Q_out) Q_out[r * p + c] = ctx->step_out->Q[r * PMAX + c];
    for (int r = 0; r < p; ++r)
        for (int c = 0; c < p; ++c) {
            if (G_out) G_out[r * p + c] = ctx->step_out->G[r * PMAX + c];
            if (Ginv_out) Ginv_out[r * p + c] = ctx->step_out->Gi[r * PMAX + c];
        }
    if (ctx->step_out->status) return fail(TILT_E_INVAL, "J^T J + Q^T Q is singular");
    return TILT_OK;
}

static int svt_call(tilt_ctx* ctx, const float* M_dev, int m, int n, float eps, float* V_dev, float* A_dev,
                    float* sigma_out, int* sweeps_out, int* reorth_out);

int tilt_svt(tilt_ctx* ctx, const float* M_dev, int m, int n, float eps, float* A_dev, float* sigma_out, int* sweeps_out) {
    return svt_call(ctx, M_dev, m, n, eps, nullptr, A_dev, sigma_out, sweeps_out, nullptr);
}

int tilt_svt_warm(tilt_ctx* ctx, const float* M_dev, int m, int n, float eps, float* V_dev, float* A_dev,
                  float* sigma_out, int* sweeps_out, int* reorth_out) {
    if (!V_dev) return fail(TILT_E_INVAL, "null V");
    return svt_call(ctx, M_dev, m, n, eps, V_dev, A_dev, sigma_out, sweeps_out, reorth_out);
}

static int svt_call(tilt_ctx* ctx, const float* M_dev, int m, int n, float eps, float* V_dev, float* A_dev,
                    float* sigma_out, int* sweeps_out, int* reorth_out) {
    if (!ctx || !M_dev || !A_dev) return fail(TILT_E_INVAL, "null argument");
    if (m < 1 || n < 1 || m > MAX_SIDE || n > MAX_SIDE) return fail(TILT_E_INVAL, "matrix %d x %d", m, n);
    if (!(eps >= 0.f)) return fail(TILT_E_INVAL, "eps must be >= 0");
    const Dims d = make_dims(m, n, 0);
    const size_t svd = svd_smem_bytes(d), head = smem_head_bytes() + (use_tc_products(d) ? tc_stage_for(d, 1) : 0);
    SvtArgs a{};
    a.M = M_dev;
    a.A = A_dev;
    a.m = m; a.n = n; a.eps = eps;
    size_t smem = 0;
    step_plan(ctx, d, svd, head, &a.smem_svd, &a.jsched, &smem);
    const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
    const size_t nz = (size_t)d.C * d.Cp;
    const size_t need = sizeof(float) * ((a.smem_svd ? 0 : (2 * nb + nv)) + MAX_SIDE + ((nz + 63) & ~(size_t)63));
    int rc = ensure_scratch(ctx, need);
    if (rc) return rc;
    float* s = reinterpret_cast<float*>(ctx->scratch);
    a.sigma = s;
    a.Zg = s + MAX_SIDE;
    if (!a.smem_svd) {
        a.Bg = a.Zg + ((nz + 63) & ~(size_t)63);
        a.Vg = a.Bg + nb;
        a.Tg = a.Vg + nv;
    }
    a.out = ctx->step_out_dev;
    a.Vio = V_dev;
    CUDA_TRY(launch_svt_step(a, smem, ctx->streams[0]));
    rc = run_step(ctx);
    if (rc) return rc;
    if (ctx->step_out->status == -5) return fail(TILT_E_TIMEOUT, "a tensor-core product did not complete");
    if (sigma_out) CUDA_TRY(cudaMemcpy(sigma_out, a.sigma, sizeof(float) * d.C, cudaMemcpyDeviceToHost));
    if (sweeps_out) *sweeps_out = ctx->step_out->sweeps;
    if (reorth_out) *reorth_out = ctx->step_out->reorth;
    return TILT_OK;
}

int tilt_inner(tilt_ctx* ctx, const float* Dhat_dev, const float* J_dev, int m, int n, const double* tau, tilt_transform type,
               const tilt_params* params, double mu0, float* A_dev, float* E_dev, float* Y_dev, int* iters_out,
               double* dtau_out, double* c1_out, double* c2_out, double* mu_out) {
    if (!ctx || !Dhat_dev || !J_dev || !A_dev || !E_dev || !Y_dev) return fail(TILT_E_INVAL, "null argument");
    if (m < 2 || n < 2 || m > MAX_SIDE || n > MAX_SIDE) return fail(TILT_E_INVAL, "window %d x %d", m, n);
    if (type != TILT_AFFINE && type != TILT_PROJECTIVE) return fail(TILT_E_INVAL, "bad type");
    InnerArgs a{};
    a.prm = to_params(params);
    if (!params_ok(a.prm)) return fail(TILT_E_INVAL, "parameters out of range");
    const Dims d = make_dims(m, n, (int)type);
    const size_t svd = svd_smem_bytes(d), head = smem_head_bytes() + (use_tc_products(d) ? tc_stage_for(d, 1) : 0);
    size_t smem = 0;
    step_plan(ctx, d, svd, head, &a.smem_svd, &a.jsched, &smem);
    const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
    const size_t S4 = ((size_t)d.S + 63) & ~(size_t)63, nz = ((size_t)d.C * d.Cp + 63) & ~(size_t)63;
    const size_t ncay = a.prm.svd_ws == 1 ? ((cayley_floats(d) + 63) & ~(size_t)63) : 0;
    const size_t need = sizeof(float) * (S4 + nz + ncay + (a.smem_svd ? 0 : (2 * nb + nv)));
    int rc = ensure_scratch(ctx, need);
    if (rc) return rc;
    float* s = reinterpret_cast<float*>(ctx->scratch);
    a.Mp = s;
    a.Zg = a.Mp + S4;
    a.Cay = ncay ? a.Zg + nz : nullptr;
    if (!a.smem_svd) {
        a.Bg = a.Zg + nz + ncay;
        a.Vg = a.Bg + nb;
        a.Tg = a.Vg + nv;
    }
    a.Dhat = Dhat_dev;
    a.J = J_dev;
    a.A = A_dev;
    a.E = E_dev;
    a.Y = Y_dev;
    a.m = m; a.n = n; a.ttype = (int)type;
    a.use_q = tau ? 1 : 0;
    for (int k = 0; k < PMAX; ++k) a.tau[k] = (tau && k < (int)type) ? tau[k] : 0.0;
    a.mu0 = mu0;
    a.out = ctx->step_out_dev;
    CUDA_TRY(launch_inner_step(a, smem, ctx->streams[0]));
    rc = run_step(ctx);
    if (rc) return rc;
    const StepOut& o = *ctx->step_out;
    if (o.status == -2) return fail(TILT_E_INVAL, "J^T J + Q^T Q is singular");
    if (o.status == -5) return fail(TILT_E_TIMEOUT, "a tensor-core product did not complete");
    if (iters_out) *iters_out = o.iters;
    if (dtau_out)
        for (int k = 0; k < (int)type; ++k) dtau_out[k] = o.dtau[k];
    ctx->last_cayley = o.accepted;
    if (c1_out) *c1_out = o.c1;
    if (c2_out) *c2_out = o.c2;
    if (mu_out) *mu_out = o.mu;
    return TILT_OK;
}

int tilt_step_counters(tilt_ctx* ctx, int* sweeps_out, int* cayley_steps_out) {
    if (!ctx) return fail(TILT_E_INVAL, "null context");
    if (sweeps_out) *sweeps_out = ctx->step_out->sweeps;
    if (cayley_steps_out) *cayley_steps_out = ctx->last_cayley;
    return TILT_OK;
}

int tilt_svd_cayley(tilt_ctx* ctx, const float* M_dev, int m, int n, float* U_dev, float* S_dev, float* V_dev,
                    double* f1_out, double* f2_out, double* t_out, int* accepted_out) {
    if (!ctx || !M_dev || !U_dev || !S_dev || !V_dev) return fail(TILT_E_INVAL, "null argument");
    if (m < 1 || n < 1 || m > MAX_SIDE || n > MAX_SIDE) return fail(TILT_E_INVAL, "matrix %d x %d", m, n);
    const Dims d = make_dims(m, n, 0);
    const size_t need = sizeof(float) * (cayley_floats(d) + (size_t)d.ldb * d.Cp + (size_t)d.ldv * d.Cp);
    int rc = ensure_scratch(ctx, need);
    if (rc) return rc;
    CayArgs a{};
    a.M = M_dev;
    a.U = U_dev;
    a.S = S_dev;
    a.V = V_dev;
    a.work = reinterpret_cast<float*>(ctx->scratch);
    a.m = m;
    a.n = n;
    a.out = ctx->step_out_dev;
    CUDA_TRY(launch_cayley_step(a, ctx->streams[0]));
    rc = run_step(ctx);
    if (rc) return rc;
    const StepOut& o = *ctx->step_out;
    if (f1_out) *f1_out = o.cay[0];
    if (f2_out) *f2_out = o.cay[1];
    if (t_out) *t_out = o.cay[2];
    if (accepted_out) *accepted_out = o.accepted;
    return TILT_OK;
}

int tilt_inner_adm(tilt_ctx* ctx, const float* D_dev, const float* J_dev, int m, int n, int p,
                   const tilt_params* params, double mu0, float* A_dev, float* E_dev, float* Y_dev, int* iters_out,
                   double* dtau_out, double* residual_out, int* sweeps_out) {
    if (!ctx || !D_dev || (p > 0 && !J_dev) || !A_dev || !E_dev || !Y_dev) return fail(TILT_E_INVAL, "null argument");
    if (m < 2 || n < 2 || m > MAX_SIDE || n > MAX_SIDE) return fail(TILT_E_INVAL, "window %d x %d", m, n);
    if (p < 0 || p > PMAX) return fail(TILT_E_INVAL, "p = %d outside 0..%d", p, PMAX);
    const Params prm = to_params(params);
    if (!(prm.rho0 > 1.0) || !(prm.eps1 > 0.0) || prm.max_inner < 1 || !std::isfinite(prm.lam) || !std::isfinite(mu0))
        return fail(TILT_E_INVAL, "ADM parameters out of range (rho0 > 1, eps1 > 0, max_inner >= 1)");
    const Dims d = make_dims(m, n, p);
    const size_t svd = svd_smem_bytes(d), head = smem_head_bytes() + (use_tc_products(d) ? tc_stage_for(d, 1) : 0);
    AdmArgs a{};
    size_t smem = 0;
    step_plan(ctx, d, svd, head, &a.smem_svd, &a.jsched, &smem);
    const size_t nb = (size_t)d.ldb * d.Cp, nv = (size_t)d.ldv * d.Cp;
    const size_t nz = ((size_t)d.C * d.Cp + 63) & ~(size_t)63;
    const size_t need = sizeof(float) * (nz + (a.smem_svd ? 0 : (2 * nb + nv)));
    int rc = ensure_scratch(ctx, need);
    if (rc) return rc;
    float* s = reinterpret_cast<float*>(ctx->scratch);
    a.Zg = s;
    if (!a.smem_svd) {
        a.Bg = a.Zg + nz;
        a.Vg = a.Bg + nb;
        a.Tg = a.Vg + nv;
    }
    a.D = D_dev;
    a.J = J_dev;
    a.A = A_dev;
    a.E = E_dev;
    a.Y = Y_dev;
    a.m = m; a.n = n; a.p = p;
    a.lam = prm.lam > 0.0 ? prm.lam : 1.0 / std::sqrt((double)std::max(m, n));
    a.tol = prm.eps1;
    a.rho = prm.rho0;
    a.mu0 = mu0;
    a.max_iter = prm.max_inner;
    a.out = ctx->step_out_dev;
    CUDA_TRY(launch_adm_step(a, smem, ctx->streams[0]));
    rc = run_step(ctx);
    if (rc) return rc;
    const StepOut& o = *ctx->step_out;
    if (o.status == -2) return fail(TILT_E_INVAL, "J^T J is singular");
    if (o.status == -5) return fail(TILT_E_TIMEOUT, "a tensor-core product did not complete");
    if (iters_out) *iters_out = o.iters;
    if (sweeps_out) *sweeps_out = o.sweeps;
    if (dtau_out)
        for (int k = 0; k < p; ++k) dtau_out[k] = o.dtau[k];
    if (residual_out) *residual_out = o.c1;
    return TILT_OK;
}

// ------------------------------------------------------------------------------ RASL
int tilt_rasl(tilt_ctx* ctx, int count, int nimg, const float* imgs, int is_device_ptr, int H, int W, int m, int n,
              tilt_transform type, const double* tau0, const tilt_params* params, double* tau_out, float* A_out,
              float* E_out, float* D_out, tilt_rasl_result* results, float* kernel_ms_out) {
    if (!ctx || (count > 0 && (!imgs || !tau0 || !tau_out || !results))) return fail(TILT_E_INVAL, "null argument");
    if (count < 0) return fail(TILT_E_INVAL, "count = %d", count);
    if (count == 0) {
        if (kernel_ms_out) *kernel_ms_out = 0.f;
        return TILT_OK;
    }
    if (type != TILT_AFFINE && type != TILT_PROJECTIVE) return fail(TILT_E_INVAL, "transform type %d", (int)type);
    if (nimg < 2 || nimg > RASL_NMAX) return fail(TILT_E_INVAL, "%d images per set (2 .. %d)", nimg, RASL_NMAX);
    if (m < 2 || n < 2 || H < 2 || W < 2) return fail(TILT_E_INVAL, "window %d x %d, images %d x %d", m, n, H, W);
    if ((long long)m * n < nimg) return fail(TILT_E_INVAL, "window of %d pixels for %d images", m * n, nimg);
    const Params prm = to_params(params);
    if (!params_ok(prm) || prm.svd_ws != 0) return fail(TILT_E_INVAL, "parameters out of range");
    const int p = (int)type;
    for (size_t k = 0; k < (size_t)count * nimg * p; ++k)
        if (!std::isfinite(tau0[k])) return fail(TILT_E_INVAL, "non-finite tau0");
    CUDA_TRY(cudaSetDevice(ctx->device));
    const Dims d = make_dims(m * n, nimg, p);
    Layout L = plan(ctx, m * n, nimg, p, 0, 0, false, false);
    if (jsched_order(L.jsched) != 2 && !ctx->force_js && !ctx->tune.count(size_bucket(d.R, d.C)))
        L.jsched = rasl_schedule(d.R, d.C);
    // tall data matrices whose M fits in shared memory with V, B_c and the small buffers take
    // the SVT's QR path (svt_tall_qr); its buffers are carved by the kernel, not by plan()
    const size_t tall_smem = smem_head_bytes() + sizeof(float) * ((size_t)d.ldv * d.Cp + (size_t)d.ldb * d.Cp +
                                                                  (size_t)d.C * d.Cp + tall_small_floats(d));
    const bool tall = tall_qr_ok(d) && tall_smem <= ctx->max_smem;
    if (tall) {
        L.smem = tall_smem;
        if (jsched_order(L.jsched) == 2) L.jsched = rasl_schedule(d.R, d.C);
    }
    const size_t img_floats = (size_t)nimg * H * W;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += align_up(bytes); return r; };
    const size_t per_set = align_up(L.total) + align_up((size_t)nimg * RASL_COLW * sizeof(double));
    const size_t sets = take(per_set * count);
    const size_t taus = take((size_t)count * nimg * p * sizeof(double));
    const size_t probs = take((size_t)count * sizeof(RaslProblem));
    const size_t resd = take((size_t)count * sizeof(RaslResult));
    const size_t imgd = is_device_ptr ? 0 : take((size_t)count * img_floats * sizeof(float));
    int rc = ensure_scratch(ctx, o);
    if (rc) return rc;
    char* base = static_cast<char*>(ctx->scratch);
    cudaStream_t st = ctx->streams[0];
    const float* imgs_dev = imgs;
    if (!is_device_ptr) {
        CUDA_TRY(cudaMemcpyAsync(base + imgd, imgs, (size_t)count * img_floats * sizeof(float), cudaMemcpyHostToDevice, st));
        imgs_dev = reinterpret_cast<const float*>(base + imgd);
    }
    CUDA_TRY(cudaMemcpyAsync(base + taus, tau0, (size_t)count * nimg * p * sizeof(double), cudaMemcpyHostToDevice, st));
    std::vector<RaslProblem> hp(count);
    for (int s = 0; s < count; ++s) {
        char* b = base + sets + per_set * s;
        RaslProblem& q = hp[s];
        q.imgs = imgs_dev + img_floats * s;
        q.img_stride = (long long)H * W;
        q.ld = W;
        q.H = H; q.W = W;
        q.nimg = nimg; q.m = m; q.n = n; q.p = p; q.ttype = p;
        q.prm = prm;
        q.pl.Dhat = reinterpret_cast<float*>(b + L.dhat);
        q.pl.J = reinterpret_cast<float*>(b + L.j);
        q.pl.A = reinterpret_cast<float*>(b + L.a);
        q.pl.E = reinterpret_cast<float*>(b + L.e);
        q.pl.Y = reinterpret_cast<float*>(b + L.y);
        q.pl.P = reinterpret_cast<float*>(b + L.p);
        q.pl.Mp = reinterpret_cast<float*>(b + L.mp);
        q.pl.Zg = reinterpret_cast<float*>(b + L.zg);
        q.pl.Bg = (L.smem_svd & 1) ? nullptr : reinterpret_cast<float*>(b + L.bg);
        q.pl.Vg = (L.smem_svd & 2) ? nullptr : reinterpret_cast<float*>(b + L.vg);
        q.pl.Tg = (L.smem_svd & 4) ? nullptr : reinterpret_cast<float*>(b + L.tg);
        q.pl.Cay = nullptr;
        q.col = reinterpret_cast<double*>(b + align_up(L.total));
        q.tau = reinterpret_cast<double*>(base + taus) + (size_t)s * nimg * p;
        q.smem_svd = L.smem_svd;
        q.jsched = L.jsched;
        q.tall = tall ? 1 : 0;
        q.res = reinterpret_cast<RaslResult*>(base + resd) + s;
    }
    CUDA_TRY(cudaMemcpyAsync(base + probs, hp.data(), (size_t)count * sizeof(RaslProblem), cudaMemcpyHostToDevice, st));
    const bool tcp = jsched_order(L.jsched) == 2;
    CUDA_TRY(cudaEventRecord(ctx->ev_rasl[0], st));
    CUDA_TRY(launch_rasl(reinterpret_cast<RaslProblem*>(base + probs), count, tcp, L.smem, st));
    CUDA_TRY(cudaEventRecord(ctx->ev_rasl[1], st));
    ctx->launches++;
    std::vector<RaslResult> hr(count);
    CUDA_TRY(cudaMemcpyAsync(hr.data(), base + resd, (size_t)count * sizeof(RaslResult), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(tau_out, base + taus, (size_t)count * nimg * p * sizeof(double), cudaMemcpyDeviceToHost, st));
    const size_t plane = (size_t)d.S * sizeof(float);
    for (int s = 0; s < count; ++s) {
        const RaslProblem& q = hp[s];
        if (A_out) CUDA_TRY(cudaMemcpyAsync(A_out + (size_t)d.S * s, q.pl.A, plane, cudaMemcpyDeviceToHost, st));
        if (E_out) CUDA_TRY(cudaMemcpyAsync(E_out + (size_t)d.S * s, q.pl.E, plane, cudaMemcpyDeviceToHost, st));
        if (D_out) CUDA_TRY(cudaMemcpyAsync(D_out + (size_t)d.S * s, q.pl.Dhat, plane, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    if (kernel_ms_out) CUDA_TRY(cudaEventElapsedTime(kernel_ms_out, ctx->ev_rasl[0], ctx->ev_rasl[1]));
    for (int s = 0; s < count; ++s) {
        const RaslResult& r = hr[s];
        tilt_rasl_result& out = results[s];
        out.status = r.status;
        out.outer_iters = r.outer_iters;
        out.inner_iters = r.inner_iters;
        out.svd_sweeps = r.svd_sweeps;
        out.svd_warm = r.svd_warm;
        out.svd_reorth = r.svd_reorth;
        out.rank = r.rank_A;
        out.oob_pixels = r.oob_pixels;
        out.svt_qr = r.svt_qr;
        out.objective = r.objective;
        out.lambda = r.lambda;
        out.kkt_residual = r.kkt_residual;
        out.cycles[0] = r.cyc_warp;
        out.cycles[1] = r.cyc_svd;
        out.cycles[2] = r.cyc_recon;
        out.cycles[3] = r.cyc_elem;
        out.cycles[4] = r.cyc_other;
    }
    return TILT_OK;
}

}  // extern "C"
