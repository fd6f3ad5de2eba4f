// Instantiations of the element-local operator for T = float, N = 1..15.
#include "hb_ax.cuh"
#define HB_AX2_T float
#define HB_AX2_WS 1
#include "hb_ax2.cuh"

hb_status hb_launch_ax_local_f32(const hb_mesh *m, const float *x, float *yL, const int *run, cudaStream_t s)
{
    const float *Dg = hb_dev_D32(m->N);
    if (!m->geo32) { hb_set_error("mesh has no float geometric factors"); return HB_ERR_ARG; }
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return hb::launch_ax_local<NN, float>(x, m->l2g, m->geo32, yL, m->E, Dg, run, s);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}

hb_status hb_ax2_upload_f32(const double *D_all) { return hb2::upload_tables(D_all); }

namespace hb2 {
namespace {
// Self-test of the staged pipeline's bounded wait: an mbarrier that nothing
// arrives at, so every thread's wait gives up and sets bit 0 of *err.
__global__ void mbar_timeout_kernel(unsigned *err)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    mbar_wait(&bar, 0, err);
}
}  // namespace
}  // namespace hb2

hb_status hb_selftest_mbar_timeout(unsigned *err, cudaStream_t s)
{
    hb2::mbar_timeout_kernel<<<1, 32, 0, s>>>(err);
    HB_CHECK_LAUNCH();
    return HB_OK;
}

// Pencil variant with the interior/surface split: eo selects the even-odd
// split, eb_mult = 2 doubles the elements per block (N <= 10). Interior DOFs
// are finished here (y, lambda term, partial of x.y); surface values go to
// ysurf for the surface gather.
hb_status hb_launch_ax2_f32(const hb_mesh *m, const float *x, float *ysurf, float *y, double lambda, int screen,
                            double *partials, const int *run, int eo, int eb_mult, cudaStream_t s,
                            int64_t *nblocks)
{
    if (!m->geo32) { hb_set_error("mesh has no float geometric factors"); return HB_ERR_ARG; }
    hb2::pencil_args A{x, m->l2g, m->geo32, ysurf, y, m->E, run, (float)lambda, screen, partials, nullptr,
                       m->counters + 7, (eb_mult & 8) ? m->spos : nullptr};
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return eo ? hb2::launch<NN, true>(A, eb_mult, s, nblocks) : hb2::launch<NN, false>(A, eb_mult, s, nblocks);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}


// ---------------------------------------------------------------- serving

#include "hb_serve.h"

namespace hb2 {
namespace {

template <int N, int TH = HB_SERVE_THREADS>
__host__ __device__ constexpr int serve_eb() { return TH / ((N + 1) * (N + 1)); }

template <int N, int TH = HB_SERVE_THREADS>
__host__ __device__ constexpr size_t serve_smem_of() { return sizeof(T) * 4 * serve_eb<N, TH>() * pad<N>::size; }

constexpr size_t serve_smem_max()
{
    size_t m = 0;
    m = serve_smem_of<1>() > m ? serve_smem_of<1>() : m;
    m = serve_smem_of<2>() > m ? serve_smem_of<2>() : m;
    m = serve_smem_of<3>() > m ? serve_smem_of<3>() : m;
    m = serve_smem_of<4>() > m ? serve_smem_of<4>() : m;
    m = serve_smem_of<5>() > m ? serve_smem_of<5>() : m;
    m = serve_smem_of<6>() > m ? serve_smem_of<6>() : m;
    m = serve_smem_of<7>() > m ? serve_smem_of<7>() : m;
    m = serve_smem_of<8>() > m ? serve_smem_of<8>() : m;
    m = serve_smem_of<9>() > m ? serve_smem_of<9>() : m;
    m = serve_smem_of<10>() > m ? serve_smem_of<10>() : m;
    m = serve_smem_of<11>() > m ? serve_smem_of<11>() : m;
    return m;
}

template <int N, int TH>
__device__ __forceinline__ void serve_groups(const pencil_args &A, T *sm, hbacc::dot_acc<S> &acc)
{
    constexpr int EB = serve_eb<N, TH>();
    const int64_t ngroups = (A.E + EB - 1) / EB;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x)
        pencil_group<N, true, EB, GM_L2G, false, false, true>(A, g, sm, acc);
}

// Degree dispatch over [NN, HI] (only these degrees are instantiated).
template <int NN, int HI, int TH>
__device__ __forceinline__ void serve_dispatch(int N, const pencil_args &A, T *sm, hbacc::dot_acc<S> &acc)
{
    if (N == NN) serve_groups<NN, TH>(A, sm, acc);
    else if constexpr (NN < HI) serve_dispatch<NN + 1, HI, TH>(N, A, sm, acc);
}

template <int LO, int HI, int TH>
constexpr size_t serve_smem_range()
{
    if constexpr (LO == HI) return serve_smem_of<LO, TH>();
    else return serve_smem_of<LO, TH>() > serve_smem_range<LO + 1, HI, TH>() ? serve_smem_of<LO, TH>()
                                                                            : serve_smem_range<LO + 1, HI, TH>();
}

// One slot's FP32 element kernel for the degrees [LO, HI] on TH-thread
// blocks (the slot's degree is read from its descriptor; a kernel whose range
// does not hold it returns at once). Degree classes with their own register
// budgets and block sizes keep the small degrees at four resident blocks per
// SM and give N = 11 blocks of exactly one element (144 threads); one kernel
// for every degree took the register count of the largest and ran one block
// per SM. Each block walks element groups grid-stride and writes one partial
// of p.Ap.
template <int LO, int HI, int MINB, int TH>
__global__ void __launch_bounds__(TH, MINB)
    serve_ax_kernel(const hb_slot_desc *__restrict__ D, const hb_slot_state *__restrict__ St)
{
    const hb_slot_desc &d = *D;
    if (!d.active || St->inner.run == 0 || d.N < LO || d.N > HI) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    pencil_args A{(const T *)d.p32, d.l2g, d.geo32, (T *)d.ysurf, (T *)d.Ap32, d.E, nullptr, (T)d.lambda,
                  d.screen, d.ax_partials};
    hbacc::dot_acc<S> acc;
    serve_dispatch<LO, HI, TH>(d.N, A, sm, acc);
    const double v = hbacc::block_sum(acc.value());
    if (threadIdx.x == 0) A.partials[blockIdx.x] = v;
}

template <int LO, int HI, int MINB, int TH>
hb_status serve_launch_class(const hb_slot_desc *d, const hb_slot_state *st, cudaStream_t s)
{
    static int attr_set[32] = {0};
    static int grid_of[32] = {0};
    int dev = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    const size_t smem = serve_smem_range<LO, HI, TH>();
    auto kern = serve_ax_kernel<LO, HI, MINB, TH>;
    if (dev < 0 || dev >= 32) dev = 0;
    if (!attr_set[dev]) {
        HB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int sms = 0;
        HB_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        grid_of[dev] = MINB * sms < HB_SERVE_AXP ? MINB * sms : HB_SERVE_AXP;
        attr_set[dev] = 1;
    }
    hb_count_launch();
    kern<<<grid_of[dev], TH, smem, s>>>(d, st);
    HB_CHECK_LAUNCH();
    return HB_OK;
}

}  // namespace
}  // namespace hb2

size_t hb_serve_ax_smem_f32() { return hb2::serve_smem_max(); }

// Every degree class is launched; those that do not hold the slot's degree
// return at once (the round graph is captured before slots are filled).
static_assert(HB_SERVE_MAX_N == 11, "the serving degree classes cover N = 1..11");
hb_status hb_serve_launch_ax_f32(const hb_slot_desc *d, const hb_slot_state *st, cudaStream_t s)
{
    hb_status r = hb2::serve_launch_class<1, 7, 4, 256>(d, st, s);
    if (r != HB_OK) return r;
    r = hb2::serve_launch_class<8, 10, 2, 256>(d, st, s);
    if (r != HB_OK) return r;
    return hb2::serve_launch_class<11, 11, 3, 144>(d, st, s);
}
