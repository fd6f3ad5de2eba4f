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
    hb2::pencil_args A{x, m->l2g, m->geo, ysurf, y, m->E, run, (double)lambda, screen, partials};
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return eo ? hb2::launch<NN, true>(A, eb_mult, s, nblocks) : hb2::launch<NN, false>(A, eb_mult, s, nblocks);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}

int hb_surf_count(int N) { return 2 * (N + 1) * (N + 1) + 4 * N * (N - 1); }
