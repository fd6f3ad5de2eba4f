// Instantiations of the element-local operator for T = float, N = 1..15.
#include "hb_ax.cuh"

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
