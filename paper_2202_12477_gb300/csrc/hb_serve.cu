// CG server with continuous batching on one GPU.
//
// Requests (a mesh description, solver options and a right-hand-side seed)
// are queued by hb_server_submit. A worker thread admits them into slots
// while slots and the device-memory budget allow, keeps each solve's mesh and
// vectors resident, and advances all resident solves together: one launch of
// a CUDA graph, captured when the server is created, runs one round for the
// slot positions it covers (graphs over the first 4, 8, 16, ... positions;
// a round takes the smallest covering every busy slot, and admission fills
// the lowest free position). A round is the FP32-inner / FP64 defect-correction
// scheme of hb_cg_solve written as per-slot device state:
//   - if the slot's inner CG has stopped: x += ||r|| d (FP64);
//   - if the slot needs an outer step: r = b - A x in FP64, stop when
//     ||r|| <= rtol ||b||, else start an inner CG on A d = r / ||r|| in FP32;
//   - k inner CG iterations (Algorithm 1 in FP32, dots accumulated to FP64
//     accuracy).
// Every kernel of a slot reads the slot's descriptor and state from device
// memory and returns at once when the slot is empty or has nothing to do, so
// the same graph serves whatever set of requests is resident. While a round
// runs the worker builds queued requests on a second stream (stream-ordered
// allocations: nothing waits for the round); between rounds it retires
// finished solves and publishes the built ones.
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
    size_t est;
};

struct finished {
    hb_cg_result res;
    double latency_ms;
    int64_t n_global;
    std::vector<double> x;
};

struct slot {
    bool busy = false;       // reserved: being built, built, or resident
    bool published = false;  // its descriptor is active on the device
    hb_mesh *mesh = nullptr;
    void *mem = nullptr;  // vectors and per-slot workspace
    size_t bytes = 0;
    request req{};
    hb_slot_state init{};  // the state published with the descriptor
    double t_admit = 0;
};

}  // namespace

struct hb_server {
    int device = 0;
    cudaStream_t s_main = nullptr;  // rounds, publication and retirement
    cudaStream_t s_adm = nullptr;   // building admitted requests beside the rounds
    cudaEvent_t ev_round = nullptr;
    int cap = 0, k = 0;
    size_t budget = 0, used = 0;
    hb_slot_desc *d_desc = nullptr;
    hb_slot_state *d_state = nullptr;
    hb_slot_state *h_state = nullptr;  // pinned
    std::vector<hb_slot_desc> h_desc;
    // round graphs over the first 4, 8, 16, ... slot positions (the last one
    // over all of them): a round runs the smallest that covers every busy
    // slot, and admission fills the lowest free position, so at low load the
    // launches of idle slot positions are not paid
    std::vector<int> graph_slots;
    std::vector<cudaGraph_t> graphs;
    std::vector<cudaGraphExec_t> execs;
    std::vector<slot> slots;
    std::deque<request> pending;
    std::map<int64_t, finished> done;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    bool inject_round_error = false;  // test hook: the next round reports a failed CUDA call
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

// Captures the round over the first `nslots` slot positions.
static hb_status capture_round_graph(hb_server *S, int nslots, cudaGraph_t *graph_out, cudaGraphExec_t *exec_out)
{
    // fork one branch per slot position from s_main, join them at the end
    std::vector<cudaStream_t> br(nslots);
    std::vector<cudaEvent_t> ev(nslots + 1);
    hb_status st = HB_OK;
    for (int i = 0; i < nslots; i++) HB_TRY_CUDA(cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking));
    for (int i = 0; i <= nslots; i++) HB_TRY_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
    HB_TRY_CUDA(cudaStreamBeginCapture(S->s_main, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(ev[nslots], S->s_main);
    for (int i = 0; i < nslots && e == cudaSuccess && st == HB_OK; i++) {
        cudaStream_t s = br[i];
        const hb_slot_desc *D = S->d_desc + i;
        hb_slot_state *T = S->d_state + i;
        if ((e = cudaStreamWaitEvent(s, ev[nslots], 0)) != cudaSuccess) break;
        serve_transition_kernel<<<1, 32, 0, s>>>(D, T);
        serve_xupdate_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        if ((st = hb_serve_launch_ax_f64(D, T, s)) != HB_OK) break;
        serve_asm64_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_residual_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_decide_kernel<<<1, 32, 0, s>>>(D, T);
        serve_inner_init_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        serve_begin_inner_kernel<<<1, 32, 0, s>>>(D, T);
        for (int it = 0; it < S->k && st == HB_OK; it++) {
            if ((st = hb_serve_launch_ax_f32(D, T, s)) != HB_OK) break;
            serve_asm32_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
            serve_update_r_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
            serve_update_xp_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, 0, s>>>(D, T);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventRecord(ev[i], s)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(S->s_main, ev[i], 0)) != cudaSuccess) break;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(S->s_main, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && st == HB_OK) e = cudaGraphInstantiate(exec_out, g, 0);
    *graph_out = g;
    for (auto s : br) cudaStreamDestroy(s);
    for (auto x : ev) cudaEventDestroy(x);
    if (st != HB_OK) return st;
    if (e != cudaSuccess) {
        hb_set_error("round graph: %s", cudaGetErrorString(e));
        return HB_ERR_CUDA;
    }
    return HB_OK;
}

// Creates the slot's mesh and vectors and publishes its descriptor and state.
static hb_status admit(hb_server *S, int si, const request &rq)
{
    slot &sl = S->slots[si];
    hb_mesh_desc md = rq.desc;
    md.keep_fp32_copy = 1;
    hb_mesh *m = nullptr;
    hb_status st = hb_mesh_create(&md, S->s_adm, &m);
    if (st != HB_OK) return st;
    const int64_t n = m->n_global;
    const size_t ns = vec_stride(n);
    const size_t bytes = ns * (4 * sizeof(double) + 4 * sizeof(float)) +
                         sizeof(double) * (HB_RED_MAXV * HB_RED_BLOCKS + HB_SERVE_AXP) + 64 * sizeof(unsigned);
    void *mem = nullptr;
    cudaError_t e = hb_dev_alloc(&mem, bytes, S->s_adm);
    if (e != cudaSuccess) {
        hb_mesh_release(m, S->s_adm);
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
    e = cudaMemsetAsync(x, 0, sizeof(double) * ns, S->s_adm);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, 64 * sizeof(unsigned), S->s_adm);
    if (e == cudaSuccess) e = cudaMemsetAsync(axp, 0, HB_SERVE_AXP * sizeof(double), S->s_adm);
    if (e == cudaSuccess) st = hb_fill_rhs(m, 0, rq.seed, 0.0, b, S->s_adm);
    // built: the round stream may use it from now on (published between rounds)
    if (e == cudaSuccess && st == HB_OK) e = cudaStreamSynchronize(S->s_adm);
    if (e != cudaSuccess || st != HB_OK) {
        cudaStreamSynchronize(S->s_adm);
        hb_dev_free(mem, S->s_adm);
        hb_mesh_release(m, S->s_adm);
        if (st == HB_OK) {
            hb_set_error("admission: %s", cudaGetErrorString(e));
            st = HB_ERR_CUDA;
        }
        return st;
    }
    sl.mesh = m;
    sl.mem = mem;
    sl.bytes = m->device_bytes + bytes;
    sl.req = rq;
    sl.init = ss;
    sl.t_admit = now_s();
    S->h_desc[si] = d;  // published by the worker between rounds
    return HB_OK;
}

static void retire(hb_server *S, int si, finished &f)
{
    slot &sl = S->slots[si];
    const hb_slot_state &st = S->h_state[si];
    f.res.iters = st.inner_total;
    f.res.outer_iters = st.outer_it;
    f.res.rel_res = st.outer.bb > 0 ? std::sqrt(st.outer.rr / st.outer.bb) : 0.0;
    f.res.status = (hb_status)st.status;
    f.n_global = sl.mesh->n_global;
    if (sl.req.keep_x) {
        f.x.resize((size_t)f.n_global);
        cudaMemcpy(f.x.data(), S->h_desc[si].x, sizeof(double) * f.n_global, cudaMemcpyDeviceToHost);
    }
    // the slot goes idle before the next round; its memory is freed after
    // that copy in stream order (no host wait)
    S->h_desc[si].active = 0;
    cudaMemcpyAsync(S->d_desc + si, &S->h_desc[si], sizeof(hb_slot_desc), cudaMemcpyHostToDevice, S->s_main);
    hb_dev_free(sl.mem, S->s_main);
    hb_mesh_release(sl.mesh, S->s_main);
    S->used -= std::min(S->used, sl.bytes);
    sl = slot{};
}

// Frees a resident slot's vectors and mesh without reading its results (the
// failure path: the round that should have advanced it did not complete).
static void release_slot(hb_server *S, int si)
{
    slot &sl = S->slots[si];
    cudaDeviceSynchronize();
    hb_dev_free(sl.mem, S->s_main);
    hb_mesh_release(sl.mesh, S->s_main);
    S->used -= std::min(S->used, sl.bytes);
    S->h_desc[si].active = 0;
    sl = slot{};
}

// The server stops after a failed round: every resident request fails and
// releases its memory, every queued one fails too, so each ticket resolves.
static void fail_server(hb_server *S, cudaError_t e, bool injected)
{
    snprintf(S->err, sizeof S->err, "round%s: %s", injected ? " (injected)" : "", cudaGetErrorString(e));
    for (int i = 0; i < S->cap; i++)
        if (S->slots[i].busy) {
            finished f{};
            f.res.status = HB_ERR_CUDA;
            f.latency_ms = f.res.time_ms = (now_s() - S->slots[i].req.t_submit) * 1e3;
            S->done[S->slots[i].req.ticket] = std::move(f);
            release_slot(S, i);
        }
    for (const request &rq : S->pending) {
        finished f{};
        f.res.status = HB_ERR_CUDA;
        f.latency_ms = f.res.time_ms = (now_s() - rq.t_submit) * 1e3;
        S->done[rq.ticket] = std::move(f);
    }
    S->pending.clear();
    S->stats.active = 0;
    S->stats.pending = 0;
    S->stats.mem_used = S->used;
    S->stop = true;
    S->cv.notify_all();
}

// Takes the next queued request into the lowest free slot and builds it on the
// admission stream (the lock is released meanwhile). Returns false when
// nothing could be admitted (queue empty, no free slot, or over budget).
static bool admit_one(hb_server *S, std::unique_lock<std::mutex> &lk)
{
    for (;;) {
        if (S->pending.empty()) return false;
        request rq = S->pending.front();
        if (rq.est > S->budget) {  // can never fit
            S->pending.pop_front();
            finished f{};
            f.res.status = HB_ERR_NOMEM;
            f.latency_ms = (now_s() - rq.t_submit) * 1e3;
            S->done[rq.ticket] = std::move(f);
            S->stats.rejected++;
            S->cv.notify_all();
            continue;
        }
        int si = -1;
        for (int i = 0; i < S->cap; i++)
            if (!S->slots[i].busy) { si = i; break; }
        if (si < 0 || S->used + rq.est > S->budget) return false;
        S->pending.pop_front();
        S->used += rq.est;
        S->slots[si].busy = true;  // reserved while it is built
        lk.unlock();
        const double ta = now_s();
        hb_status st = admit(S, si, rq);
        const double tb = now_s();
        lk.lock();
        S->stats.admit_s += tb - ta;
        S->used -= rq.est;
        if (st != HB_OK) {
            S->slots[si] = slot{};
            finished f{};
            f.res.status = st;
            f.latency_ms = (now_s() - rq.t_submit) * 1e3;
            S->done[rq.ticket] = std::move(f);
            S->stats.rejected++;
            S->cv.notify_all();
        } else {
            S->used += S->slots[si].bytes;
            S->stats.admitted++;
        }
        return true;
    }
}

// One round advances every published solve; while it runs the worker builds
// queued requests on the admission stream, one at a time, and goes back to the
// round as soon as it has finished. Between rounds: retire the finished solves
// (stream-ordered frees), publish the built ones, launch the next round.
static void worker_loop(hb_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    bool inflight = false;
    double t_launch = 0;
    for (;;) {
        if (S->stop) break;
        // publish what was built (no round in flight here)
        if (!inflight) {
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < S->cap && e == cudaSuccess; i++) {
                slot &sl = S->slots[i];
                if (!sl.busy || sl.published || !sl.mesh) continue;
                e = cudaMemcpyAsync(S->d_desc + i, &S->h_desc[i], sizeof(hb_slot_desc), cudaMemcpyHostToDevice,
                                    S->s_main);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(S->d_state + i, &sl.init, sizeof(hb_slot_state), cudaMemcpyHostToDevice,
                                        S->s_main);
                sl.published = true;
            }
            if (e != cudaSuccess) {
                fail_server(S, e, false);
                break;
            }
        }
        int active = 0, top = 0;
        for (int i = 0; i < S->cap; i++)
            if (S->slots[i].busy) {
                active++;
                if (S->slots[i].published) top = i + 1;
            }
        S->stats.active = active;
        S->stats.pending = (int)S->pending.size();
        S->stats.mem_used = S->used;
        // launch a round over the smallest graph that covers every published slot
        if (!inflight && top > 0) {
            const bool fail_round = S->inject_round_error;
            S->inject_round_error = false;
            size_t gi = 0;
            while (gi + 1 < S->execs.size() && S->graph_slots[gi] < top) gi++;
            t_launch = now_s();
            cudaError_t e = fail_round ? cudaErrorLaunchFailure : cudaGraphLaunch(S->execs[gi], S->s_main);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(S->h_state, S->d_state, sizeof(hb_slot_state) * S->cap, cudaMemcpyDeviceToHost,
                                    S->s_main);
            if (e == cudaSuccess) e = cudaEventRecord(S->ev_round, S->s_main);
            if (e != cudaSuccess) {
                fail_server(S, e, fail_round);
                break;
            }
            inflight = true;
        }
        // build queued requests while the round runs
        const bool admitted = admit_one(S, lk);
        if (S->stop) break;
        if (inflight) {
            const cudaError_t q = cudaEventQuery(S->ev_round);
            if (q == cudaErrorNotReady && admitted) continue;  // more to build meanwhile
            lk.unlock();
            const cudaError_t e = cudaEventSynchronize(S->ev_round);
            const double t_done = now_s();
            lk.lock();
            inflight = false;
            S->stats.rounds++;
            S->stats.round_s += t_done - t_launch;
            if (e != cudaSuccess) {
                fail_server(S, e, false);
                break;
            }
            const double tt = now_s();
            for (int i = 0; i < S->cap; i++) {
                if (!S->slots[i].published || S->h_state[i].phase != HB_SLOT_DONE) continue;
                finished f{};
                const int64_t ticket = S->slots[i].req.ticket;
                const double t_sub = S->slots[i].req.t_submit;
                retire(S, i, f);
                f.latency_ms = (now_s() - t_sub) * 1e3;
                f.res.time_ms = f.latency_ms;
                S->done[ticket] = std::move(f);
                S->stats.completed++;
            }
            S->stats.retire_s += now_s() - tt;
            S->cv.notify_all();
            continue;
        }
        if (!admitted && top == 0) S->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
    if (inflight) {
        lk.unlock();
        cudaEventSynchronize(S->ev_round);
        lk.lock();
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
    cudaError_t e = cudaStreamCreateWithFlags(&S->s_main, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->s_adm, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_round, cudaEventDisableTiming);
    // resident requests come and go: keep their freed memory for reuse
    if (e == cudaSuccess) e = hb_dev_keep(std::max<uint64_t>(S->budget, hb_dev_keep_default()));
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_desc, sizeof(hb_slot_desc) * S->cap);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->d_state, sizeof(hb_slot_state) * S->cap);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&S->h_state, sizeof(hb_slot_state) * S->cap);
    if (e == cudaSuccess) e = cudaMemset(S->d_desc, 0, sizeof(hb_slot_desc) * S->cap);
    if (e == cudaSuccess) e = cudaMemset(S->d_state, 0, sizeof(hb_slot_state) * S->cap);
    if (e != cudaSuccess) {
        hb_set_error("server: %s", cudaGetErrorString(e));
        hb_server_destroy(S);
        return e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
    }
    memset(S->h_state, 0, sizeof(hb_slot_state) * S->cap);
    for (int ns = 4;; ns *= 2) {
        const int take = ns < S->cap ? ns : S->cap;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        st = capture_round_graph(S, take, &g, &x);
        if (g) S->graphs.push_back(g);
        if (st != HB_OK) {
            hb_server_destroy(S);
            return st;
        }
        S->graph_slots.push_back(take);
        S->execs.push_back(x);
        if (take == S->cap) break;
    }
    S->worker = std::thread(worker_loop, S);
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
    S->cv.notify_all();
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
    }
    if (S->worker.joinable()) S->worker.join();
    hb_device_guard dg(S->device);
    cudaDeviceSynchronize();
    for (int i = 0; i < S->cap; i++)
        if (S->slots[i].busy) {
            hb_dev_free(S->slots[i].mem, S->s_main);
            hb_mesh_release(S->slots[i].mesh, S->s_main);
        }
    if (S->s_main) cudaStreamSynchronize(S->s_main);
    hb_dev_keep(hb_dev_keep_default());
    hb_dev_trim();
    for (auto x : S->execs)
        if (x) cudaGraphExecDestroy(x);
    for (auto g : S->graphs)
        if (g) cudaGraphDestroy(g);
    cudaFree(S->d_desc);
    cudaFree(S->d_state);
    if (S->h_state) cudaFreeHost(S->h_state);
    if (S->s_main) cudaStreamDestroy(S->s_main);
    if (S->s_adm) cudaStreamDestroy(S->s_adm);
    if (S->ev_round) cudaEventDestroy(S->ev_round);
    delete S;
    return HB_OK;
}
