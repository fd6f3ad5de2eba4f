// CG server with continuous batching on one GPU.
//
// Requests (a mesh description, solver options and a right-hand-side seed)
// are queued by hb_server_submit. A builder thread takes them, first come
// first served, into free slots while the device-memory budget allows and
// builds each one's mesh and vectors on its own stream (stream-ordered
// allocations: nothing waits for the solves running meanwhile). A worker
// thread keeps every resident solve going on the slot's own stream: one
// launch of the slot's CUDA graph, captured when the server is created, runs
// one round, and the worker launches the slot's next round as soon as its
// last one has finished, so solves of different sizes advance at their own
// pace and share the GPU. A round is the FP32-inner / FP64 defect-correction
// scheme of hb_cg_solve written as per-slot device state:
//   - if the slot's inner CG has stopped: x += ||r|| d (FP64);
//   - if the slot needs an outer step: r = b - A x in FP64, stop when
//     ||r|| <= rtol ||b||, else start an inner CG on A d = r / ||r|| in FP32;
//   - k inner CG iterations (Algorithm 1 in FP32, dots accumulated to FP64
//     accuracy).
// Every kernel of a slot reads the slot's descriptor and state from device
// memory and returns at once when the slot is empty or has nothing to do, so
// a slot's graph serves whichever request the slot holds. Finished solves are
// retired with stream-ordered frees on the slot's stream.
// Each slot's kernels run on fixed grids with per-slot reductions, so a
// request's result does not depend on which other requests share the GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hb_serve.h"
#include "hb_vec.cuh"

using namespace hb;

// ---------------------------------------------------------------- kernels

// Ends a stopped inner CG: the slot goes back to the outer step.
__global__ void serve_transition_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    if (threadIdx.x != 0 || !D->active) return;
    if (S->phase == HB_SLOT_INNER && S->inner.run == 0) {
        S->inner_total += S->inner.it;
        if (S->inner.status == HB_ERR_BREAKDOWN && S->inner.it == 0) {
            S->status = HB_ERR_BREAKDOWN;
            S->phase = HB_SLOT_DONE;
        } else {
            S->phase = HB_SLOT_OUTER;
            S->x_pending = S->inner.it > 0 ? 1 : 0;
        }
    }
}

// x += ||r|| d32 after an inner solve.
__global__ void __launch_bounds__(HB_SERVE_THREADS) serve_xupdate_kernel(const hb_slot_desc *D, const hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (!d.active || S->phase != HB_SLOT_OUTER || !S->x_pending) return;
    update_x_body(d.x, d.d32, d.n_global, &S->outer);
}

// Surface gather of the FP64 outer product A x (no dot).
__global__ void __launch_bounds__(HB_SERVE_THREADS) serve_asm64_kernel(const hb_slot_desc *D, const hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (!d.active || S->phase != HB_SLOT_OUTER) return;
    if (d.screen)
        assemble_surf_body<double, 1, HB_DOT_NONE>((const double *)d.ysurf, d.srow_g, d.srowptr, d.scols, d.x,
                                                   d.mdiag, d.lambda, d.Ap, d.nsr, nullptr, 0, d.partials,
                                                   d.counters, nullptr);
    else
        assemble_surf_body<double, 0, HB_DOT_NONE>((const double *)d.ysurf, d.srow_g, d.srowptr, d.scols, d.x,
                                                   d.mdiag, d.lambda, d.Ap, d.nsr, nullptr, 0, d.partials,
                                                   d.counters, nullptr);
}

// r = b - A x, r.r and b.b into the outer state.
__global__ void __launch_bounds__(HB_SERVE_THREADS) serve_residual_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (!d.active || S->phase != HB_SLOT_OUTER) return;
    residual_body(d.b, d.Ap, d.r, d.n_global, d.partials, d.counters + 2, &S->outer);
}

// Outer decision: converged, out of budget, or start another inner solve.
__global__ void serve_decide_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (threadIdx.x != 0 || !d.active || S->phase != HB_SLOT_OUTER) return;
    S->x_pending = 0;
    const double rr = S->outer.rr, bb = S->outer.bb;
    if (!isfinite(rr)) {
        S->status = HB_ERR_BREAKDOWN;
        S->phase = HB_SLOT_DONE;
    } else if (bb == 0.0 || rr <= d.rtol * d.rtol * bb) {
        S->status = HB_OK;
        S->phase = HB_SLOT_DONE;
    } else if (S->outer_it >= d.max_outer || S->inner_total >= d.max_it) {
        S->status = HB_ERR_NOT_CONVERGED;
        S->phase = HB_SLOT_DONE;
    }
}

__global__ void __launch_bounds__(HB_SERVE_THREADS) serve_inner_init_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (!d.active || S->phase != HB_SLOT_OUTER) return;
    inner_init_body(d.r, d.r32, d.p32, d.d32, nullptr, d.n_global, d.inner_rtol, d.max_it - S->inner_total, d.partials,
                    d.counters + 2, &S->outer, &S->inner);
}

__global__ void serve_begin_inner_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    if (threadIdx.x != 0 || !D->active || S->phase != HB_SLOT_OUTER) return;
    S->phase = HB_SLOT_INNER;
    S->outer_it += 1;
}

// Inner CG iteration, after the element kernel: surface gather with p.Ap.
__global__ void __launch_bounds__(HB_SERVE_THREADS) serve_asm32_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (!d.active) return;
    if (d.screen)
        assemble_surf_body<float, 1, HB_DOT_CG_PAP>((const float *)d.ysurf, d.srow_g, d.srowptr, d.scols, d.p32,
                                                    d.mdiag32, d.lambda, d.Ap32, d.nsr, d.ax_partials,
                                                    HB_SERVE_AXP, d.partials, d.counters, &S->inner);
    else
        assemble_surf_body<float, 0, HB_DOT_CG_PAP>((const float *)d.ysurf, d.srow_g, d.srowptr, d.scols, d.p32,
                                                    d.mdiag32, d.lambda, d.Ap32, d.nsr, d.ax_partials,
                                                    HB_SERVE_AXP, d.partials, d.counters, &S->inner);
}

__global__ void __launch_bounds__(HB_SERVE_THREADS) serve_update_r_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (!d.active) return;
    cg_update_r_body<float, false>(d.r32, d.Ap32, nullptr, nullptr, d.n_global, d.partials, d.counters + 2,
                                   &S->inner);
}

__global__ void __launch_bounds__(HB_SERVE_THREADS) serve_update_xp_kernel(const hb_slot_desc *D, hb_slot_state *S)
{
    const hb_slot_desc &d = *D;
    if (!d.active) return;
    cg_update_xp_body<float>(d.d32, d.p32, d.r32, d.n_global, d.counters + 3, &S->inner);
}


// ---------------------------------------------------------------- host side

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct request {
    int64_t ticket;
    hb_mesh_desc desc;
    hb_cg_opts opts;
    uint64_t seed;
    int keep_x;
    double t_submit;
    double t_build0 = 0, t_build1 = 0;  // the build's start and end
    size_t est;
};

struct finished {
    hb_cg_result res;
    double latency_ms;
    int64_t n_global;
    std::vector<double> x;
    std::string msg;  // why it failed, when it did
};

// FREE -> BUILDING (builder, lock released) -> BUILT -> RUNNING (worker) -> FREE
enum slot_phase { SL_FREE = 0, SL_BUILDING, SL_BUILT, SL_RUNNING };

struct slot {
    int phase = SL_FREE;
    bool inflight = false;  // a round of the slot is on its stream
    cudaStream_t stream = nullptr;  // the slot's stream for this request (by its size)
    bool small = false;             // at most kSmallNodes local nodes
    double t_held = 0;              // > 0: a large solve's next round held back since then
    bool resolved = false;          // BUILDING: the failure path already answered its ticket
    hb_mesh *mesh = nullptr;
    void *mem = nullptr;  // vectors and per-slot workspace
    size_t bytes = 0;
    request req{};
};

}  // namespace

// Builder threads, each with its own stream; requests with at most
// kSmallNodes local nodes run on their slot's higher-priority stream.
constexpr int kBuilders = 2;
constexpr int64_t kSmallNodes = 4 << 20;
// Shortest job first, bounded: while a small request has a round in flight,
// a large one's next round waits, at most kHoldS seconds.
constexpr double kHoldS = 2e-3;

struct hb_server {
    int device = 0;
    cudaStream_t s_adm[kBuilders] = {};  // the builders' streams (highest priority)
    // per slot: rounds, publication and retirement on the low-priority stream
    // (large requests) or the middle-priority one (small requests)
    std::vector<cudaStream_t> streams, streams_hi;
    std::vector<cudaEvent_t> events;    // per slot: end of its last round
    std::vector<cudaGraph_t> graphs;    // per slot: one round
    std::vector<cudaGraphExec_t> execs;
    int cap = 0, k = 0;
    size_t budget = 0, used = 0;
    hb_slot_desc *d_desc = nullptr;
    hb_slot_state *d_state = nullptr;
    hb_slot_state *h_state = nullptr;  // pinned: each slot's state after its last round
    std::vector<hb_slot_desc> h_desc;  // the host's record of each slot's descriptor
    // pinned sources of the copies the worker issues (pageable sources would
    // stage through buffers the builders' copies share): per slot the
    // descriptor and initial state to publish, and one idle descriptor
    hb_slot_desc *pin_desc = nullptr;
    hb_slot_state *pin_init = nullptr;
    hb_slot_desc *pin_idle = nullptr;
    std::vector<slot> slots;
    std::deque<request> pending;
    std::map<int64_t, finished> done;
    std::thread worker, builders[kBuilders];
    std::mutex mu;
    std::condition_variable cv;        // worker: a slot was built, or stop
    std::condition_variable cv_build;  // builder: a request queued, a slot or memory freed, or stop
    bool stop = false;
    bool inject_round_error = false;  // test hook: the next launch reports a failed CUDA call
    int inflight = 0;
    int small_inflight = 0;
    double t_busy = 0;  // when the number of rounds in flight last left zero
    int64_t next_ticket = 1;
    hb_server_stats_t stats{};
    char err[256] = {0};
};

// Device bytes a request will hold once admitted (mesh + vectors + workspace).
static size_t estimate_bytes(const hb_mesh_desc &d)
{
    const int n = d.N + 1;
    const size_t E = (size_t)d.ex * d.ey * d.ez;
    const size_t NL = E * n * n * n;
    const size_t NG = (size_t)(d.N * d.ex + 1) * (d.N * d.ey + 1) * (d.N * d.ez + 1);
    // l2g 4, geo 56 + 28, surface store 8, CSRs <= 4 + 4 + 4 per local node;
    // per DOF: row pointers, mass diagonals 12, FP64 b x r Ap 32, FP32 r p Ap d 16
    return NL * (4 + 56 + 28 + 8 + 12) + NG * (4 + 12 + 4 + 32 + 16) + (4 << 20);
}

static size_t vec_stride(int64_t n) { return (size_t)((n + 63) / 64 * 64); }

// Captures one round of slot i on the slot's stream.
static hb_status capture_slot_graph(hb_server *S, int i)
{
    cudaStream_t s = S->streams[i];
    const hb_slot_desc *D = S->d_desc + i;
    hb_slot_state *T = S->d_state + i;
    HB_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    hb_status st = HB_OK;
    serve_transition_kernel<<<1, 32, 0, s>>>(D, T);
    serve_xupdate_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
    st = hb_serve_launch_ax_f64(D, T, s);
    if (st == HB_OK) {
        serve_asm64_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_residual_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_decide_kernel<<<1, 32, 0, s>>>(D, T);
        serve_inner_init_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_begin_inner_kernel<<<1, 32, 0, s>>>(D, T);
    }
    for (int it = 0; it < S->k && st == HB_OK; it++) {
        if ((st = hb_serve_launch_ax_f32(D, T, s)) != HB_OK) break;
        serve_asm32_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_update_r_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_update_xp_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
    }
    cudaError_t e = cudaGetLastError();
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e2;
    S->graphs[i] = g;
    if (e == cudaSuccess && st == HB_OK) e = cudaGraphInstantiate(&S->execs[i], g, 0);
    if (st != HB_OK) return st;
    if (e != cudaSuccess) {
        hb_set_error("round graph: %s", cudaGetErrorString(e));
        return HB_ERR_CUDA;
    }
    return HB_OK;
}
// Builds the slot's mesh, vectors and right-hand side on the builder's stream
// (called without the lock; the slot is BUILDING, which the worker leaves
// alone). On return the arrays are ready for any stream.
static hb_status admit(hb_server *S, int si, const request &rq, cudaStream_t sa)
{
    slot &sl = S->slots[si];
    hb_mesh_desc md = rq.desc;
    md.keep_fp32_copy = 1;
    hb_mesh *m = nullptr;
    hb_status st = hb_mesh_create(&md, sa, &m);
    if (st != HB_OK) return st;
    const int64_t n = m->n_global;
    const size_t ns = vec_stride(n);
    const size_t bytes = ns * (4 * sizeof(double) + 4 * sizeof(float)) +
                         sizeof(double) * (HB_RED_MAXV * HB_RED_BLOCKS + HB_SERVE_AXP) + 64 * sizeof(unsigned);
    void *mem = nullptr;
    cudaError_t e = hb_dev_alloc(&mem, bytes, sa);
    if (e != cudaSuccess) {
        hb_mesh_release(m, sa);
        hb_set_error("slot vectors: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
    }
    double *b = (double *)mem, *x = b + ns, *r = x + ns, *Ap = r + ns;
    float *r32 = (float *)(Ap + ns), *p32 = r32 + ns, *Ap32 = p32 + ns, *d32 = Ap32 + ns;
    double *partials = (double *)(d32 + ns);
    double *axp = partials + HB_RED_MAXV * HB_RED_BLOCKS;
    unsigned *ctr = (unsigned *)(axp + HB_SERVE_AXP);
    hb_slot_desc d{};
    d.active = 1;
    d.N = m->N;
    d.screen = rq.opts.screen;
    d.max_it = rq.opts.max_it;
    d.max_outer = rq.opts.max_outer > 0 ? rq.opts.max_outer : 30;
    d.E = m->E;
    d.n_local = m->n_local;
    d.n_global = n;
    d.nsr = m->nsr;
    d.l2g = m->l2g;
    d.srow_g = m->srow_g;
    d.srowptr = m->srowptr;
    d.scols = m->scols;
    d.geo = m->geo;
    d.geo32 = m->geo32;
    d.mdiag = m->mdiag;
    d.mdiag32 = m->mdiag32;
    d.ysurf = m->yL;
    d.b = b;
    d.x = x;
    d.r = r;
    d.Ap = Ap;
    d.r32 = r32;
    d.p32 = p32;
    d.Ap32 = Ap32;
    d.d32 = d32;
    d.lambda = rq.opts.lambda;
    d.rtol = rq.opts.rtol;
    d.inner_rtol = rq.opts.inner_rtol > 0 ? rq.opts.inner_rtol : 1e-4;
    d.partials = partials;
    d.ax_partials = axp;
    d.counters = ctr;
    hb_slot_state ss{};
    ss.phase = HB_SLOT_OUTER;
    ss.status = HB_OK;
    e = cudaMemsetAsync(x, 0, sizeof(double) * ns, sa);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, 64 * sizeof(unsigned), sa);
    if (e == cudaSuccess) e = cudaMemsetAsync(axp, 0, HB_SERVE_AXP * sizeof(double), sa);
    if (e == cudaSuccess) st = hb_fill_rhs(m, 0, rq.seed, 0.0, b, sa);
    // built: the slot's stream may use it from now on
    if (e == cudaSuccess && st == HB_OK) e = cudaStreamSynchronize(sa);
    if (e != cudaSuccess || st != HB_OK) {
        cudaStreamSynchronize(sa);
        hb_dev_free(mem, sa);
        hb_mesh_release(m, sa);
        if (st == HB_OK) {
            hb_set_error("admission: %s", cudaGetErrorString(e));
            st = HB_ERR_CUDA;
        }
        return st;
    }
    sl.mesh = m;
    sl.mem = mem;
    sl.bytes = m->device_bytes + bytes;
    S->pin_init[si] = ss;
    S->pin_desc[si] = d;
    sl.small = m->n_local <= kSmallNodes;
    sl.stream = sl.small ? S->streams_hi[si] : S->streams[si];
    S->h_desc[si] = d;  // published by the worker
    return HB_OK;
}


// Reads a finished slot's results and frees it in stream order on the slot's
// stream (its round has completed; the lock is held).
static void retire(hb_server *S, int si, finished &f)
{
    slot &sl = S->slots[si];
    cudaStream_t s = sl.stream;
    const hb_slot_state &st = S->h_state[si];
    f.res.iters = st.inner_total;
    f.res.outer_iters = st.outer_it;
    f.res.rel_res = st.outer.bb > 0 ? std::sqrt(st.outer.rr / st.outer.bb) : 0.0;
    f.res.status = (hb_status)st.status;
    f.n_global = sl.mesh->n_global;
    if (sl.req.keep_x) {
        f.x.resize((size_t)f.n_global);
        cudaMemcpyAsync(f.x.data(), S->h_desc[si].x, sizeof(double) * f.n_global, cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
    }
    S->h_desc[si].active = 0;
    cudaMemcpyAsync(S->d_desc + si, S->pin_idle, sizeof(hb_slot_desc), cudaMemcpyHostToDevice, s);
    hb_dev_free(sl.mem, s);
    hb_mesh_release(sl.mesh, s);
    // the slot's next request may run on its other stream: it publishes after this
    cudaEventRecord(S->events[si], s);
    S->used -= std::min(S->used, sl.bytes);
    sl = slot{};
}

// Frees a built or running slot without reading its results (the failure
// path and the server's destruction): waits for the device first.
static void release_slot(hb_server *S, int si)
{
    slot &sl = S->slots[si];
    cudaStream_t s = sl.stream ? sl.stream : S->streams[si];
    cudaDeviceSynchronize();
    hb_dev_free(sl.mem, s);
    hb_mesh_release(sl.mesh, s);
    S->used -= std::min(S->used, sl.bytes);
    S->h_desc[si].active = 0;
    sl = slot{};
}

// After a failed round the server stops: every request in a slot or in the
// queue fails, so each ticket resolves; built and resident requests release
// their memory here, the one being built when the builder is done with it.
static void fail_server(hb_server *S, cudaError_t e, bool injected)
{
    snprintf(S->err, sizeof S->err, "round%s: %s", injected ? " (injected)" : "", cudaGetErrorString(e));
    for (int i = 0; i < S->cap; i++) {
        const int ph = S->slots[i].phase;
        if (ph == SL_FREE) continue;
        finished f{};
        f.res.status = HB_ERR_CUDA;
        f.latency_ms = f.res.time_ms = (now_s() - S->slots[i].req.t_submit) * 1e3;
        S->done[S->slots[i].req.ticket] = std::move(f);
        if (ph != SL_BUILDING) release_slot(S, i);
        else S->slots[i].resolved = true;  // the builder frees what it is building
    }
    for (const request &rq : S->pending) {
        finished f{};
        f.res.status = HB_ERR_CUDA;
        f.latency_ms = f.res.time_ms = (now_s() - rq.t_submit) * 1e3;
        S->done[rq.ticket] = std::move(f);
    }
    S->pending.clear();
    S->inflight = 0;
    S->small_inflight = 0;
    int active = 0;
    for (auto &sl : S->slots) active += sl.phase != SL_FREE ? 1 : 0;
    S->stats.active = active;
    S->stats.pending = 0;
    S->stats.mem_used = S->used;
    S->stop = true;
    S->cv.notify_all();
    S->cv_build.notify_all();
}

// Launches slot i's next round and the read-back of its state.
static cudaError_t launch_round(hb_server *S, int i, bool *injected)
{
    *injected = S->inject_round_error;
    S->inject_round_error = false;
    cudaStream_t s = S->slots[i].stream;
    cudaError_t e = *injected ? cudaErrorLaunchFailure : cudaGraphLaunch(S->execs[i], s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->h_state + i, S->d_state + i, sizeof(hb_slot_state), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(S->events[i], s);
    if (e == cudaSuccess) {
        if (S->inflight++ == 0) S->t_busy = now_s();
        if (S->slots[i].small) S->small_inflight++;
        S->slots[i].inflight = true;
        S->slots[i].t_held = 0;
    }
    return e;
}

static void round_ended(hb_server *S, int i)
{
    S->slots[i].inflight = false;
    if (S->slots[i].small) S->small_inflight--;
    S->stats.rounds++;
    if (--S->inflight == 0) S->stats.round_s += now_s() - S->t_busy;
}

// Keeps every resident solve going: a slot whose round has finished is
// retired (solve done) or relaunched at once; built slots are published on
// their stream and started. Polls the slots' events while rounds run.
static void worker_loop(hb_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    double t_act = now_s();
    while (!S->stop) {
        bool acted = false;
        cudaError_t e = cudaSuccess;
        bool injected = false;
        for (int i = 0; i < S->cap && e == cudaSuccess; i++) {
            slot &sl = S->slots[i];
            if (sl.phase == SL_BUILT) {
                // publish: descriptor and initial state, then the first round
                // (after the slot's last retirement, which may sit on its other stream)
                cudaStream_t s = sl.stream;
                e = cudaStreamWaitEvent(s, S->events[i], 0);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(S->d_desc + i, S->pin_desc + i, sizeof(hb_slot_desc), cudaMemcpyHostToDevice, s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(S->d_state + i, S->pin_init + i, sizeof(hb_slot_state), cudaMemcpyHostToDevice,
                                        s);
                sl.phase = SL_RUNNING;
                if (e == cudaSuccess) e = launch_round(S, i, &injected);
                acted = true;
                continue;
            }
            if (sl.t_held > 0) {
                // a held large round goes once no small round is in flight
                if (S->small_inflight == 0 || now_s() - sl.t_held > kHoldS) {
                    e = launch_round(S, i, &injected);
                    acted = true;
                }
                continue;
            }
            if (!sl.inflight) continue;
            const cudaError_t q = cudaEventQuery(S->events[i]);
            if (q == cudaErrorNotReady) continue;
            round_ended(S, i);
            acted = true;
            if (q != cudaSuccess) {
                e = q;
                break;
            }
            if (S->h_state[i].phase == HB_SLOT_DONE) {
                const double tt = now_s();
                finished f{};
                const request rq = sl.req;
                retire(S, i, f);
                const double t_done = now_s();
                const int64_t ticket = rq.ticket;
                const double t_sub = rq.t_submit;
                S->stats.queue_s += rq.t_build0 - rq.t_submit;
                S->stats.build_s += rq.t_build1 - rq.t_build0;
                S->stats.run_s += t_done - rq.t_build1;
                f.latency_ms = (t_done - t_sub) * 1e3;
                f.res.time_ms = f.latency_ms;
                S->done[ticket] = std::move(f);
                S->stats.completed++;
                S->stats.retire_s += now_s() - tt;
                S->cv_build.notify_all();
            } else if (!sl.small && S->small_inflight > 0) {
                sl.t_held = now_s();
            } else {
                e = launch_round(S, i, &injected);
            }
        }
        if (e != cudaSuccess) {
            fail_server(S, e, injected);
            break;
        }
        int active = 0;
        for (auto &sl : S->slots) active += sl.phase != SL_FREE ? 1 : 0;
        S->stats.active = active;
        S->stats.pending = (int)S->pending.size();
        S->stats.mem_used = S->used;
        const double t = now_s();
        if (acted) {
            t_act = t;
            continue;
        }
        if (S->inflight == 0) {
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        } else {
            // poll: spin for 0.2 ms after the last launch or retirement (short
            // rounds end within it), then sleep between polls
            lk.unlock();
            if (t - t_act < 2e-4) std::this_thread::yield();
            else std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
    // rounds still on the slots' streams finish before the server is torn down
    for (int i = 0; i < S->cap; i++)
        if (S->slots[i].inflight) {
            lk.unlock();
            cudaEventSynchronize(S->events[i]);
            lk.lock();
            round_ended(S, i);
        }
}

// Takes queued requests, first come first served, into free slots while the
// budget allows and builds them on its own stream (the lock released meanwhile).
static void builder_loop(hb_server *S, int b)
{
    cudaSetDevice(S->device);
    cudaStream_t sa = S->s_adm[b];
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        if (!S->pending.empty() && S->pending.front().est > S->budget) {  // can never fit
            const request rq = S->pending.front();
            S->pending.pop_front();
            finished f{};
            f.res.status = HB_ERR_NOMEM;
            f.latency_ms = (now_s() - rq.t_submit) * 1e3;
            S->done[rq.ticket] = std::move(f);
            S->stats.rejected++;
            continue;
        }
        int si = -1;
        for (int i = 0; i < S->cap; i++)
            if (S->slots[i].phase == SL_FREE) { si = i; break; }
        if (S->pending.empty() || si < 0 || S->used + S->pending.front().est > S->budget) {
            S->cv_build.wait_for(lk, std::chrono::milliseconds(5));
            continue;
        }
        request rq = S->pending.front();
        S->pending.pop_front();
        S->used += rq.est;
        const double ta = now_s();
        rq.t_build0 = ta;
        S->slots[si].phase = SL_BUILDING;
        S->slots[si].req = rq;  // the failure path answers this ticket while it is built
        lk.unlock();
        const hb_status st = admit(S, si, rq, sa);
        const double tb = now_s();
        lk.lock();
        S->slots[si].req.t_build1 = tb;
        S->stats.admit_s += tb - ta;
        S->used -= rq.est;
        finished f{};
        if (S->slots[si].resolved) {
            // the server failed meanwhile and has resolved the ticket
            if (st == HB_OK) {
                S->used += S->slots[si].bytes;
                release_slot(S, si);
            } else {
                S->slots[si] = slot{};
            }
            int active = 0;
            for (auto &sl : S->slots) active += sl.phase != SL_FREE ? 1 : 0;
            S->stats.active = active;
            S->stats.mem_used = S->used;
            continue;
        }
        if (st != HB_OK) {
            S->slots[si] = slot{};
            f.res.status = st;
            f.msg = hb_last_error();
            S->stats.rejected++;
        } else if (S->stop) {
            // the server stopped meanwhile: the request fails, its memory goes
            S->used += S->slots[si].bytes;
            release_slot(S, si);
            f.res.status = HB_ERR_CUDA;
            int active = 0;
            for (auto &sl : S->slots) active += sl.phase != SL_FREE ? 1 : 0;
            S->stats.active = active;
            S->stats.mem_used = S->used;
        } else {
            S->used += S->slots[si].bytes;
            S->stats.admitted++;
            S->slots[si].phase = SL_BUILT;
            S->cv.notify_all();
            continue;
        }
        f.latency_ms = f.res.time_ms = (now_s() - rq.t_submit) * 1e3;
        S->done[rq.ticket] = std::move(f);
    }
}

// ---------------------------------------------------------------- C ABI

extern "C" hb_status hb_server_create(const hb_server_opts *o, hb_server **out)
{
    hb_clear_error();
    if (!o || !out) { hb_set_error("null argument"); return HB_ERR_ARG; }
    *out = nullptr;
    if (o->max_slots < 1 || o->max_slots > 256 || o->iters_per_launch < 1 || o->iters_per_launch > 256) {
        hb_set_error("max_slots must be 1..256 and iters_per_launch 1..256");
        return HB_ERR_ARG;
    }
    hb_status st = hb_ensure_device_tables();
    if (st != HB_OK) return st;
    hb_server *S = new hb_server();
    HB_TRY_CUDA(cudaGetDevice(&S->device));
    S->cap = o->max_slots;
    S->k = o->iters_per_launch;
    S->budget = o->mem_budget_bytes;
    S->slots.resize(S->cap);
    S->h_desc.resize(S->cap);
    S->streams.assign(S->cap, nullptr);
    S->events.assign(S->cap, nullptr);
    S->graphs.assign(S->cap, nullptr);
    S->execs.assign(S->cap, nullptr);
    S->streams_hi.assign(S->cap, nullptr);
    // priorities: builders highest, small requests' rounds next, large ones lowest
    int p_least = 0, p_greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&p_least, &p_greatest);
    const int p_mid = p_greatest < p_least ? p_greatest + 1 : p_greatest;
    for (int b = 0; b < kBuilders && e == cudaSuccess; b++)
        e = cudaStreamCreateWithPriority(&S->s_adm[b], cudaStreamNonBlocking, p_greatest);
    for (int i = 0; i < S->cap && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithPriority(&S->streams[i], cudaStreamNonBlocking, p_least);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S->streams_hi[i], cudaStreamNonBlocking, p_mid);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->events[i], cudaEventDisableTiming);
    }
    // resident requests come and go: keep up to 32 GiB of their freed memory
    // for reuse (more lets cached blocks crowd out new requests)
    if (e == cudaSuccess) e = hb_dev_keep(std::max<uint64_t>(std::min<uint64_t>(S->budget, 32ull << 30),
                                                            hb_dev_keep_default()));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_desc, sizeof(hb_slot_desc) * S->cap);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_state, sizeof(hb_slot_state) * S->cap);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->h_state, sizeof(hb_slot_state) * S->cap);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->pin_desc, sizeof(hb_slot_desc) * S->cap);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->pin_init, sizeof(hb_slot_state) * S->cap);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->pin_idle, sizeof(hb_slot_desc));
    if (e == cudaSuccess) memset(S->pin_idle, 0, sizeof(hb_slot_desc));
    if (e == cudaSuccess) e = cudaMemset(S->d_desc, 0, sizeof(hb_slot_desc) * S->cap);
    if (e == cudaSuccess) e = cudaMemset(S->d_state, 0, sizeof(hb_slot_state) * S->cap);
    if (e != cudaSuccess) {
        hb_set_error("server: %s", cudaGetErrorString(e));
        hb_server_destroy(S);
        return e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
    }
    memset(S->h_state, 0, sizeof(hb_slot_state) * S->cap);
    for (int i = 0; i < S->cap; i++)
        if ((st = capture_slot_graph(S, i)) != HB_OK) {
            hb_server_destroy(S);
            return st;
        }
    S->worker = std::thread(worker_loop, S);
    for (int b = 0; b < kBuilders; b++) S->builders[b] = std::thread(builder_loop, S, b);
    *out = S;
    return HB_OK;
}

extern "C" hb_status hb_server_submit(hb_server *S, const hb_mesh_desc *d, const hb_cg_opts *o, uint64_t rhs_seed,
                                      int keep_x, int64_t *ticket)
{
    hb_clear_error();
    if (!S || !d || !o || !ticket) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (d->N < 1 || d->N > HB_SERVE_MAX_N) { hb_set_error("server accepts N = 1..%d", HB_SERVE_MAX_N); return HB_ERR_ARG; }
    if (d->ex < 1 || d->ey < 1 || d->ez < 1 || !(d->perturb >= 0.0 && d->perturb < 0.5)) {
        hb_set_error("bad mesh description");
        return HB_ERR_ARG;
    }
    if (o->prec != HB_MIXED) { hb_set_error("the server runs HB_MIXED solves"); return HB_ERR_ARG; }
    if (o->precond != 0) { hb_set_error("the server runs unpreconditioned solves (precond = 0)"); return HB_ERR_ARG; }
    if (o->screen != HB_SCREEN_IDENTITY && o->screen != HB_SCREEN_MASS) { hb_set_error("bad screen"); return HB_ERR_ARG; }
    if (!(o->rtol > 0.0) || o->max_it < 1) { hb_set_error("the server needs rtol > 0 and max_it >= 1"); return HB_ERR_ARG; }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) { hb_set_error("server stopped: %s", S->err); return HB_ERR_CUDA; }
    request rq{};
    rq.ticket = S->next_ticket++;
    rq.desc = *d;
    rq.opts = *o;
    rq.seed = rhs_seed;
    rq.keep_x = keep_x;
    rq.t_submit = now_s();
    rq.est = estimate_bytes(*d);
    S->pending.push_back(rq);
    S->stats.submitted++;
    *ticket = rq.ticket;
    S->cv_build.notify_all();
    return HB_OK;
}

extern "C" hb_status hb_server_poll(hb_server *S, int64_t ticket, hb_cg_result *res, int64_t *n_global,
                                    double *x_host)
{
    hb_clear_error();
    if (!S) { hb_set_error("null server"); return HB_ERR_ARG; }
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        if (ticket >= 1 && ticket < S->next_ticket) {
            // a stopped server runs nothing more: report its error, not "busy"
            if (S->stop) { hb_set_error("server stopped: %s", S->err); return HB_ERR_CUDA; }
            return HB_ERR_BUSY;  // queued or running
        }
        hb_set_error("unknown ticket %lld", (long long)ticket);
        return HB_ERR_NOT_FOUND;
    }
    if (res) *res = it->second.res;
    if (n_global) *n_global = it->second.n_global;
    if (x_host && !it->second.x.empty())
        memcpy(x_host, it->second.x.data(), sizeof(double) * it->second.x.size());
    // a request that failed leaves its reason in hb_last_error
    if (!it->second.msg.empty()) hb_set_error("%s", it->second.msg.c_str());
    S->done.erase(it);
    return HB_OK;
}

extern "C" hb_status hb_server_inject_round_error(hb_server *S)
{
    hb_clear_error();
    if (!S) { hb_set_error("null server"); return HB_ERR_ARG; }
    std::lock_guard<std::mutex> lk(S->mu);
    S->inject_round_error = true;
    S->cv.notify_all();
    return HB_OK;
}

extern "C" hb_status hb_server_stats(hb_server *S, hb_server_stats_t *out)
{
    if (!S || !out) { hb_set_error("null argument"); return HB_ERR_ARG; }
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return HB_OK;
}

extern "C" hb_status hb_server_destroy(hb_server *S)
{
    if (!S) return HB_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->pending.clear();
        S->cv.notify_all();
        S->cv_build.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto &t : S->builders)
        if (t.joinable()) t.join();
    hb_device_guard dg(S->device);
    cudaDeviceSynchronize();
    for (int i = 0; i < S->cap; i++)
        if (S->slots[i].phase != SL_FREE) {
            cudaStream_t s = S->slots[i].stream ? S->slots[i].stream : S->streams[i];
            hb_dev_free(S->slots[i].mem, s);
            hb_mesh_release(S->slots[i].mesh, s);
        }
    cudaDeviceSynchronize();
    hb_dev_keep(hb_dev_keep_default());
    hb_dev_trim();
    for (auto x : S->execs)
        if (x) cudaGraphExecDestroy(x);
    for (auto g : S->graphs)
        if (g) cudaGraphDestroy(g);
    cudaFree(S->d_desc);
    cudaFree(S->d_state);
    if (S->h_state) cudaFreeHost(S->h_state);
    if (S->pin_desc) cudaFreeHost(S->pin_desc);
    if (S->pin_init) cudaFreeHost(S->pin_init);
    if (S->pin_idle) cudaFreeHost(S->pin_idle);
    for (auto s : S->streams)
        if (s) cudaStreamDestroy(s);
    for (auto ev : S->events)
        if (ev) cudaEventDestroy(ev);
    for (auto s : S->streams_hi)
        if (s) cudaStreamDestroy(s);
    for (auto s : S->s_adm)
        if (s) cudaStreamDestroy(s);
    delete S;
    return HB_OK;
}
