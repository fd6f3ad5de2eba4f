// Instantiations of the element-local operator for T = double, N = 1..15.
#include "hb_ax.cuh"
#define HB_AX2_T double
#include "hb_ax2.cuh"

hb_status hb_launch_ax_local_f64(const hb_mesh *m, const double *x, double *yL, const int *run, cudaStream_t s)
{
    const double *Dg = hb_dev_D64(m->N);
    if (!m->geo) { hb_set_error("mesh has no double geometric factors"); return HB_ERR_ARG; }
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return hb::launch_ax_local<NN, double>(x, m->l2g, m->geo, yL, m->E, Dg, run, s);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}

hb_status hb_ax2_upload_f64(const double *D_all) { return hb2::upload_tables(D_all); }

// Pencil variant with the interior/surface split: eo selects the even-odd
// split, eb_mult = 2 doubles the elements per block (N <= 10). Interior DOFs
// are finished here (y, lambda term, partial of x.y); surface values go to
// ysurf for the surface gather.
hb_status hb_launch_ax2_f64(const hb_mesh *m, const double *x, double *ysurf, double *y, double lambda, int screen,
                            double *partials, const int *run, int eo, int eb_mult, cudaStream_t s,
                            int64_t *nblocks)
{
    if (!m->geo) { hb_set_error("mesh has no double geometric factors"); return HB_ERR_ARG; }
    hb2::pencil_args A{x, m->l2g, m->geo, ysurf, y, m->E, run, (double)lambda, screen, partials, nullptr, nullptr,
                       (eb_mult & 8) ? m->spos : nullptr};
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return eo ? hb2::launch<NN, true>(A, eb_mult, s, nblocks) : hb2::launch<NN, false>(A, eb_mult, s, nblocks);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}

// Pencil kernel (even-odd, base block shape) on a contiguous range of E
// elements given by its own arrays (l2g, geo and ysurf start at the range's
// first element); l2g entries <= -2 read halo values. Used by the partitioned
// operator; eo and eb_mult are accepted for symmetry and not used.
hb_status hb_launch_ax2_f64_range(int N, int64_t E, const double *x, const double *halo, const int32_t *l2g,
                                  const double *geo, double *ysurf, double *y, double lambda, int screen,
                                  const int *run, int eo, int eb_mult, cudaStream_t s)
{
    (void)eo;
    (void)eb_mult;
    hb2::pencil_args A{x, l2g, geo, ysurf, y, E, run, lambda, screen, nullptr, halo};
    switch (N) {
#define HB_CASE(NN) \
    case NN: return hb2::launch<NN, true, hb2::GM_HALO>(A, 1, s, nullptr);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", N); return HB_ERR_ARG;
    }
}

// Pencil kernel (even-odd, base block shape) on scattered vectors (x_L, y_L
// of length n_local, no l2g): interior nodes of every element get
// y_L = (S_L x_L) + lambda term, surface nodes go to ysurf for the
// gather-scatter; eo and eb_mult are accepted for symmetry and not used.
hb_status hb_launch_ax2_f64_scat(const hb_mesh *m, const double *xL, double *ysurf, double *yL, double lambda,
                                 int screen, const int *run, int eo, int eb_mult, cudaStream_t s)
{
    if (!m->geo) { hb_set_error("mesh has no double geometric factors"); return HB_ERR_ARG; }
    (void)eo;
    (void)eb_mult;
    hb2::pencil_args A{xL, nullptr, m->geo, ysurf, yL, m->E, run, lambda, screen, nullptr, nullptr};
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return hb2::launch<NN, true, hb2::GM_SCAT>(A, 1, s, nullptr);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}

int hb_surf_count(int N) { return 2 * (N + 1) * (N + 1) + 4 * N * (N - 1); }

// ---------------------------------------------------------------- serving

#include "hb_serve.h"

namespace hb2 {
namespace {

template <int N>
__host__ __device__ constexpr int serve_eb() { return HB_SERVE_THREADS / ((N + 1) * (N + 1)); }

template <int N>
__host__ __device__ constexpr size_t serve_smem_of() { return sizeof(T) * 4 * serve_eb<N>() * pad<N>::size; }

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

template <int N>
__device__ __forceinline__ void serve_groups(const pencil_args &A, T *sm, hbacc::dot_acc<S> &acc)
{
    constexpr int EB = serve_eb<N>();
    const int64_t ngroups = (A.E + EB - 1) / EB;
    for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x) pencil_group<N, true, EB>(A, g, sm, acc);
}

// One slot's element kernel on a fixed grid: the degree is read from the
// slot descriptor, each block walks element groups grid-stride.
__global__ void __launch_bounds__(HB_SERVE_THREADS, 1)
    serve_ax_kernel(const hb_slot_desc *__restrict__ D, const hb_slot_state *__restrict__ St)
{
    const hb_slot_desc &d = *D;
    if (!d.active || St->phase != HB_SLOT_OUTER) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    pencil_args A{(const T *)d.x, d.l2g, d.geo, (T *)d.ysurf, (T *)d.Ap, d.E, nullptr, (T)d.lambda,
                  d.screen, nullptr};
    hbacc::dot_acc<S> acc;
    switch (d.N) {
    case 1: serve_groups<1>(A, sm, acc); break;
    case 2: serve_groups<2>(A, sm, acc); break;
    case 3: serve_groups<3>(A, sm, acc); break;
    case 4: serve_groups<4>(A, sm, acc); break;
    case 5: serve_groups<5>(A, sm, acc); break;
    case 6: serve_groups<6>(A, sm, acc); break;
    case 7: serve_groups<7>(A, sm, acc); break;
    case 8: serve_groups<8>(A, sm, acc); break;
    case 9: serve_groups<9>(A, sm, acc); break;
    case 10: serve_groups<10>(A, sm, acc); break;
    case 11: serve_groups<11>(A, sm, acc); break;
    default: break;
    }
    if (A.partials) {
        const double v = hbacc::block_sum(acc.value());
        if (threadIdx.x == 0) A.partials[blockIdx.x] = v;
    }
}

}  // namespace
}  // namespace hb2

size_t hb_serve_ax_smem_f64() { return hb2::serve_smem_max(); }

hb_status hb_serve_launch_ax_f64(const hb_slot_desc *d, const hb_slot_state *st, cudaStream_t s)
{
    static int attr_set[32] = {0};
    int dev = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    const size_t smem = hb2::serve_smem_max();
    if (dev >= 0 && dev < 32 && !attr_set[dev]) {
        HB_TRY_CUDA(cudaFuncSetAttribute(hb2::serve_ax_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        attr_set[dev] = 1;
    }
    hb_count_launch();
    hb2::serve_ax_kernel<<<HB_SERVE_GRID, HB_SERVE_THREADS, smem, s>>>(d, st);
    HB_CHECK_LAUNCH();
    return HB_OK;
}
