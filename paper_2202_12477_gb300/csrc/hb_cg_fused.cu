// Fused CG for small meshes: every iteration of Algorithm 1 inside one
// cooperative kernel. On a mesh of a few dozen elements the element kernel
// itself needs a few microseconds of FP64 work, and launching the four
// kernels of an iteration costs more than that; here the phases of an
// iteration are separated by grid-wide barriers instead of launches:
//   A p (one element per block, its three line directions at once)
//   | Z^T on surface DOFs, p.Ap block partials
//   | every block sums the partials in index order -> alpha; r -= alpha Ap,
//     r.r block partials
//   | every block sums them -> beta, stopping test; x += alpha p, p = r + beta p
// Every block computes alpha and beta itself from the same partials in the
// same order, so all blocks take the same decisions (no broadcast needed).
// The barriers are bounded: a block that waits more than about a second
// records bit 1 in the mesh's error word and every block then leaves the
// iteration loop (the host reports HB_ERR_TIMEOUT).
#include "hb_internal.h"
#define HB_AX2_T double
#include "hb_ax2.cuh"
#include "hb_vec.cuh"

namespace {

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch (every block resident at once)
// on one counter word: block 0 adds 2^31 - (nb - 1) and every other block 1,
// so the counter's top bit flips exactly when the last of the nb blocks has
// arrived, once per barrier, with no reset. Thread 0 of each block arrives
// after a fence (its block's writes are then visible to the others) and
// polls until the top bit differs from the one its own atomic saw, for at
// most hb2::kWaitNs of wall time. Returns true in every thread of the block
// if this block gave up (the caller must then stop: the blocks still waiting
// give up in turn, so the launch ends).
__device__ bool grid_barrier(unsigned *bar, unsigned nb, unsigned *err)
{
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        int fail = 0;
        const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nb - 1u) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(bar, add);
        if (((old ^ ld_acquire(bar)) & 0x80000000u) == 0) {
            const unsigned long long t0 = hb2::wall_ns();
            while (((old ^ ld_acquire(bar)) & 0x80000000u) == 0) {
                if (hb2::wall_ns() - t0 > hb2::kWaitNs) {
                    atomicOr(err, 2u);
                    fail = 1;
                    break;
                }
            }
        }
        __threadfence();
        s_fail = fail;
    }
    __syncthreads();
    return s_fail != 0;
}

struct fused_args {
    const int32_t *l2g;
    const double *geo;
    const int32_t *srow_g, *srowptr, *scols;
    const double *mdiag;
    double *ysurf;
    double *x, *r, *p, *Ap;
    int64_t E, n_global, nsr;
    double lambda;
    int screen;
    double *part_a, *part_b;  // [gridDim.x] block partials (two, alternating)
    hb_cg_state *st;          // in: rr, tol2, max_it, run; out: final state
    unsigned *bar;            // grid barrier counter (zero at launch)
    unsigned *err;            // error word (bit 1: a barrier wait gave up)
};

// Block size for degree N: the three thread groups of pencil_element3, at
// least 256 threads for the vector phases.
template <int N>
constexpr int fused_threads()
{
    constexpr int t = 3 * (N + 1) * (N + 1);
    return t < 256 ? 256 : (t + 31) / 32 * 32;
}

__device__ __forceinline__ double sum_partials(const double *p, int nb)
{
    // every block adds the same values in the same order: thread t takes
    // partials t, t + blockDim, ..., then a fixed shuffle tree (a serial sum
    // by one thread waits on one L2 round trip per partial)
    __shared__ double s_w[32];
    __shared__ double s_tot;
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(p + b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) s_w[wid] = t;
    __syncthreads();
    if (wid == 0) {
        double u = lane < nw ? s_w[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
        if (lane == 0) s_tot = u;
    }
    __syncthreads();
    const double v = s_tot;
    __syncthreads();
    return v;
}

template <int N>
__global__ void __launch_bounds__(fused_threads<N>()) cg_fused_kernel(const fused_args F)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double *sm = reinterpret_cast<double *>(smem_raw);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
    const int nb = (int)gridDim.x;

    double rr = F.st->rr;
    const double tol2 = F.st->tol2;
    const int max_it = F.st->max_it;
    int run = F.st->run;
    int it = 0;
    int status = HB_OK;
    double alpha = 0.0, beta = 0.0, pAp = 0.0;

    hb2::pencil_args A{F.p, F.l2g, F.geo, F.ysurf, F.Ap, F.E, nullptr, F.lambda, F.screen, nullptr};
    // one element per block, its three line directions contracted at once
    // (pencil_element3): on a small mesh the element's latency sets the time;
    // the other threads of the block join the vector phases
    const int64_t ngroups = F.E;

    while (run) {
        // A p: element kernel (interior DOFs finished, surface values to ysurf)
        hbacc::dot_acc<double> acc;
        for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x)
            hb2::pencil_element3<N, hb2::GM_L2G_CG>(A, g, sm, acc);
        if (grid_barrier(F.bar, nb, F.err)) {
            status = HB_ERR_TIMEOUT;
            break;
        }
        // Z^T on the surface DOFs
        // (data written by other blocks in this launch is read through L2)
        for (int64_t rI = gtid; rI < F.nsr; rI += gthreads) {
            const int g = F.srow_g[rI];
            double t = 0.0;
            for (int q = F.srowptr[rI]; q < F.srowptr[rI + 1]; q++) t += __ldcg(F.ysurf + F.scols[q]);
            const double xv = __ldcg(F.p + g);
            t += F.screen ? F.lambda * (F.mdiag[g] * xv) : F.lambda * xv;
            F.Ap[g] = t;
            acc.add(xv, t);
        }
        {
            const double v = hbacc::block_sum(acc.value());
            if (threadIdx.x == 0) F.part_a[blockIdx.x] = v;
        }
        if (grid_barrier(F.bar, nb, F.err)) {
            status = HB_ERR_TIMEOUT;
            break;
        }
        pAp = sum_partials(F.part_a, nb);
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            status = HB_ERR_BREAKDOWN;
            break;  // every block takes the same branch
        }
        alpha = rr / pAp;
        // r -= alpha Ap and r.r
        hbacc::dot_acc<double> racc;
        for (int64_t i = gtid; i < F.n_global; i += gthreads) {
            const double ri = F.r[i] - alpha * __ldcg(F.Ap + i);
            F.r[i] = ri;
            racc.add(ri, ri);
        }
        {
            const double v = hbacc::block_sum(racc.value());
            if (threadIdx.x == 0) F.part_b[blockIdx.x] = v;
        }
        if (grid_barrier(F.bar, nb, F.err)) {
            status = HB_ERR_TIMEOUT;
            break;
        }
        const double rr_new = sum_partials(F.part_b, nb);
        beta = rr_new / rr;
        rr = rr_new;
        it++;
        run = (it < max_it && rr_new > tol2) ? 1 : 0;
        // x += alpha p with the old p, then p = r + beta p
        for (int64_t i = gtid; i < F.n_global; i += gthreads) {
            const double pi = __ldcg(F.p + i);
            F.x[i] += alpha * pi;
            F.p[i] = F.r[i] + beta * pi;
        }
        if (grid_barrier(F.bar, nb, F.err)) {
            status = HB_ERR_TIMEOUT;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hb_cg_state *st = F.st;
        st->it += it;
        st->rr = rr;
        st->res2 = rr;
        st->pAp = pAp;
        st->alpha = alpha;
        st->beta = beta;
        st->run = 0;
        st->next_run = 0;
        if (status != HB_OK) st->status = status;
    }
}

template <int N>
hb_status launch_fused(const fused_args &F, int blocks_cap, cudaStream_t s, bool probe_only, int *grid_out)
{
    constexpr int threads = fused_threads<N>();
    const size_t smem = sizeof(double) * 4 * (size_t)hb2::pad<N>::size;
    auto kern = cg_fused_kernel<N>;
    static int attr_set[32] = {0};
    int dev = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 32 && !attr_set[dev]) {
        HB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev] = 1;
    }
    int per_sm = 0, sms = 0;
    HB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    HB_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t ngroups = F.E;
    int64_t grid = (int64_t)per_sm * sms;  // every block resident at once (cooperative launch)
    if (grid > ngroups) grid = ngroups;
    if (grid > blocks_cap) grid = blocks_cap;
    if (grid < 1) grid = 1;
    if (grid_out) *grid_out = (int)grid;
    if (probe_only) return per_sm > 0 ? HB_OK : HB_ERR_ARG;
    void *args[] = {(void *)&F};
    hb_prof_scope prof("cg_fused", s);
    HB_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)grid), dim3(threads), args, smem, s));
    return HB_OK;
}

// Self-test of the bounded barrier: it waits for one block more than were
// launched, so every block gives up and sets bit 1 of *err.
__global__ void barrier_timeout_kernel(unsigned *bar, unsigned *err) { grid_barrier(bar, gridDim.x + 1, err); }

}  // namespace

hb_status hb_selftest_barrier_timeout(unsigned *bar, unsigned *err, cudaStream_t s)
{
    void *args[] = {(void *)&bar, (void *)&err};
    HB_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)barrier_timeout_kernel, dim3(2), dim3(32), args, 0, s));
    return HB_OK;
}

// This unit's copy of the derivative tables (every unit that includes the
// element kernel has its own constant bank).
hb_status hb_cg_fused_upload(const double *D_all) { return hb2::upload_tables(D_all); }

// Number of element groups a fused solve can keep resident at once for
// degree N (0 if the kernel cannot be launched cooperatively).
int hb_cg_fused_capacity(int N)
{
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    fused_args F{};
    F.E = 1 << 30;
    int grid = 0;
    hb_status st;
    switch (N) {
#define HB_CASE(NN) \
    case NN: st = launch_fused<NN>(F, 1 << 30, nullptr, true, &grid); break;
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: return 0;
    }
    return st == HB_OK ? grid : 0;
}

// max_it iterations (or until the state's tolerance) of Algorithm 1 on
// (x, r, p, Ap) in one cooperative launch; the state must hold rr, tol2,
// max_it and run as cg_init leaves them.
hb_status hb_cg_fused_run(const hb_mesh *m, int screen, double lambda, double *x, double *r, double *p, double *Ap,
                          hb_cg_state *st, cudaStream_t s)
{
    fused_args F{};
    F.l2g = m->l2g;
    F.geo = m->geo;
    F.srow_g = m->srow_g;
    F.srowptr = m->srowptr;
    F.scols = m->scols;
    F.mdiag = m->mdiag;
    F.ysurf = (double *)m->yL;
    F.x = x;
    F.r = r;
    F.p = p;
    F.Ap = Ap;
    F.E = m->E;
    F.n_global = m->n_global;
    F.nsr = m->nsr;
    F.lambda = lambda;
    F.screen = screen;
    F.part_a = m->partials;
    F.part_b = m->partials + HB_RED_BLOCKS;
    F.st = st;
    F.bar = m->counters + 4;
    F.err = m->counters + 7;
    HB_TRY_CUDA(cudaMemsetAsync(F.bar, 0, sizeof(unsigned), s));
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return launch_fused<NN>(F, HB_RED_BLOCKS, s, false, nullptr);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}
