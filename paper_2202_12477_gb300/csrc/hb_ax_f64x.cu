// Element kernel on FP64 data in double-float arithmetic (HB_F64X): x, the
// geometric factors and the results are FP64 in memory; each value is split
// exactly into a float pair on load and every contraction runs as
// error-free FP32 operations (about 47 significant bits), on the FP32 pipes.
#define HB_AX2_T df
#define HB_AX2_S double
#include "hb_ax2.cuh"

hb_status hb_ax2_upload_f64x(const double *D_all) { return hb2::upload_tables(D_all); }

hb_status hb_launch_ax2_f64x(const hb_mesh *m, const double *x, double *ysurf, double *y, double lambda, int screen,
                             double *partials, const int *run, int eb_mode, cudaStream_t s, int64_t *nblocks)
{
    if (!m->geo) { hb_set_error("mesh has no FP64 geometric factors"); return HB_ERR_ARG; }
    hb2::pencil_args A{x, m->l2g, m->geo, ysurf, y, m->E, run, lambda, screen, partials, nullptr, nullptr,
                       (eb_mode & 8) ? m->spos : nullptr};
    switch (m->N) {
#define HB_CASE(NN) \
    case NN: return hb2::launch<NN, true>(A, eb_mode, s, nblocks);
        HB_CASE(1) HB_CASE(2) HB_CASE(3) HB_CASE(4) HB_CASE(5) HB_CASE(6) HB_CASE(7) HB_CASE(8)
        HB_CASE(9) HB_CASE(10) HB_CASE(11) HB_CASE(12) HB_CASE(13) HB_CASE(14) HB_CASE(15)
#undef HB_CASE
    default: hb_set_error("unsupported N=%d", m->N); return HB_ERR_ARG;
    }
}
