// Instantiations of the element-local operator for T = float, N = 1..15.
#include "hb_ax.cuh"
#define HB_AX2_T float
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

// Pencil variant with the interior/surface split: eo selects the even-odd
// split, eb_mult = 2 doubles the elements per block (N <= 10). Interior DOFs
// are finished here (y, lambda term, partial of x.y); surface values go to
// ysurf for the surface gather.
hb_status hb_launch_ax2_f32(const hb_mesh *m, const float *x, float *ysurf, float *y, double lambda, int screen,
                            double *partials, const int *run, int eo, int eb_mult, cudaStream_t s,
                            int64_t *nblocks)
{
    if (!m->geo32) { hb_set_error("mesh has no float geometric factors"); return HB_ERR_ARG; }
    hb2::pencil_args A{x, m->l2g, m->geo32, ysurf, y, m->E, run, (float)lambda, screen, partials};
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return eo ? hb2::launch<NN, true>(A, eb_mult, s, nblocks) : hb2::launch<NN, false>(A, eb_mult, s, nblocks);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}

