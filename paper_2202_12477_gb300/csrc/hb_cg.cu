// Assembly Z^T, dot products and conjugate gradients (hipBone, arXiv
// 2202.12477: Eq. poisson, Sec. 3.2 for the gather, Sec. 3.5 and Algorithm 1
// for CG).
//
// Every reduction runs on a fixed grid (a function of the vector length only);
// each block reduces its grid-stride share with warp shuffles, stores one
// partial, and the block that finishes last adds the partials in index order.
// Results are therefore bitwise reproducible and need no atomics on data.
//
// The CG scalars of Algorithm 1 (r.r, p.Ap, alpha, beta, the iteration count)
// stay in device memory: p.Ap is reduced inside the assembly kernel that
// produces Ap, r.r inside the kernel that updates r, and the kernels of a
// finished solve return at once, so iterations are enqueued in runs without
// host round trips.
#include <cmath>
#include <mutex>

#include "hb_internal.h"
#include "hb_vec.cuh"

namespace hb {

static inline int red_grid(int64_t n)
{
    int64_t g = (n + HB_RED_THREADS * 4 - 1) / (HB_RED_THREADS * 4);
    if (g > HB_RED_BLOCKS) g = HB_RED_BLOCKS;
    return (int)(g < 1 ? 1 : g);
}


// ---------------------------------------------------------------- kernels

template <typename T, int SCREEN, int DOT>
__global__ void __launch_bounds__(HB_RED_THREADS)
    assemble_kernel(const T *__restrict__ yL, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ cols,
                    const T *__restrict__ x, const T *__restrict__ mdiag, double lambda, T *__restrict__ y,
                    int64_t ng, double *partials, unsigned *counter, hb_cg_state *st)
{
    assemble_body<T, SCREEN, DOT>(yL, rowptr, cols, x, mdiag, lambda, y, ng, partials, counter, st);
}

template <typename T, int SCREEN, int DOT, bool CONTIG>
__global__ void __launch_bounds__(HB_RED_THREADS)
    assemble_surf_kernel(const T *__restrict__ ys, const int32_t *__restrict__ srow_g,
                         const int32_t *__restrict__ rowptr, const int32_t *__restrict__ cols,
                         const T *__restrict__ x, const T *__restrict__ mdiag, double lambda, T *__restrict__ y,
                         int64_t nrows, const double *__restrict__ ax_partials, int64_t n_axp, double *partials,
                         unsigned *counter, hb_cg_state *st)
{
    assemble_surf_body<T, SCREEN, DOT, CONTIG>(ys, srow_g, rowptr, cols, x, mdiag, lambda, y, nrows, ax_partials,
                                               n_axp, partials, counter, st);
}

template <typename T, int SCREEN, int DOT>
__global__ void __launch_bounds__(HB_RED_THREADS)
    assemble_grid_kernel(const T *__restrict__ yL, const lattice_t L, const T *__restrict__ x,
                         const T *__restrict__ mdiag, double lambda, T *__restrict__ y, double *partials,
                         unsigned *counter, hb_cg_state *st)
{
    assemble_grid_body<T, SCREEN, DOT>(yL, L, x, mdiag, lambda, y, partials, counter, st);
}

template <typename T>
__global__ void __launch_bounds__(HB_RED_THREADS)
    dot_kernel(const T *__restrict__ a, const T *__restrict__ b, int64_t n, double *out, double *partials,
               unsigned *counter)
{
    dot_body<T>(a, b, n, out, partials, counter);
}

__global__ void __launch_bounds__(HB_RED_THREADS)
    cg_init_kernel(const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ r,
                   double *__restrict__ p, const double *__restrict__ inv_d, int64_t n, double rtol, int max_it,
                   double *partials, unsigned *counter, hb_cg_state *st)
{
    cg_init_body(b, Ax, r, p, inv_d, n, rtol, max_it, partials, counter, st);
}

template <typename T, bool PREC>
__global__ void __launch_bounds__(HB_RED_THREADS)
    cg_update_r_kernel(T *__restrict__ r, const T *__restrict__ Ap, T *__restrict__ z, const T *__restrict__ inv_d,
                       int64_t n, double *partials, unsigned *counter, hb_cg_state *st)
{
    cg_update_r_body<T, PREC>(r, Ap, z, inv_d, n, partials, counter, st);
}

template <typename T>
__global__ void __launch_bounds__(HB_RED_THREADS)
    cg_update_xp_kernel(T *__restrict__ x, T *__restrict__ p, const T *__restrict__ r, int64_t n, unsigned *counter,
                        hb_cg_state *st)
{
    cg_update_xp_body<T>(x, p, r, n, counter, st);
}

__global__ void __launch_bounds__(HB_RED_THREADS)
    cg_restart_kernel(const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ r,
                      double *__restrict__ p, double *__restrict__ z, const double *__restrict__ inv_d, int64_t n,
                      double *partials, unsigned *counter, hb_cg_state *st)
{
    cg_restart_body(b, Ax, r, p, z, inv_d, n, partials, counter, st);
}

__global__ void __launch_bounds__(HB_RED_THREADS)
    residual_kernel(const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ r, int64_t n,
                    double *partials, unsigned *counter, hb_cg_state *st)
{
    residual_body(b, Ax, r, n, partials, counter, st);
}

__global__ void __launch_bounds__(HB_RED_THREADS)
    inner_init_kernel(const double *__restrict__ r, float *__restrict__ r32, float *__restrict__ p32,
                      float *__restrict__ d32, const float *__restrict__ inv_d, int64_t n, double rtol_in,
                      int max_it, double *partials, unsigned *counter, const hb_cg_state *outer, hb_cg_state *st)
{
    inner_init_body(r, r32, p32, d32, inv_d, n, rtol_in, max_it, partials, counter, outer, st);
}

__global__ void update_x_kernel(double *__restrict__ x, const float *__restrict__ d32, int64_t n,
                                const hb_cg_state *outer)
{
    update_x_body(x, d32, n, outer);
}

template <typename T>
hb_status launch_assemble(const hb_mesh *m, const T *yL, const T *x, T *y, const T *mdiag, int screen,
                          double lambda, hb_cg_state *st, int dot_mode, cudaStream_t s)
{
    const int64_t ng = m->n_global;
    if (ng == 0) return HB_OK;
    const int grid = red_grid(ng);
    unsigned *ctr = m->counters + 0;
    hb_prof_scope prof("assemble", s);
#define HB_ASM(SC, DM)                                                                                   \
    assemble_kernel<T, SC, DM><<<grid, HB_RED_THREADS, 0, s>>>(yL, m->rowptr, m->cols, x, mdiag, lambda, \
                                                               y, ng, m->partials, ctr, st)
    if (screen == 0) {
        if (dot_mode == HB_DOT_NONE) HB_ASM(0, HB_DOT_NONE);
        else if (dot_mode == HB_DOT_TO_TMP) HB_ASM(0, HB_DOT_TO_TMP);
        else HB_ASM(0, HB_DOT_CG_PAP);
    } else {
        if (dot_mode == HB_DOT_NONE) HB_ASM(1, HB_DOT_NONE);
        else if (dot_mode == HB_DOT_TO_TMP) HB_ASM(1, HB_DOT_TO_TMP);
        else HB_ASM(1, HB_DOT_CG_PAP);
    }
#undef HB_ASM
    HB_CHECK_LAUNCH();
    return HB_OK;
}

// contig: the element kernel wrote the surface values at their CSR positions.
template <typename T>
hb_status launch_assemble_surf(const hb_mesh *m, const T *ys, const T *x, T *y, const T *mdiag, int screen,
                               double lambda, int64_t n_axp, hb_cg_state *st, int dot_mode, cudaStream_t s,
                               bool contig = false)
{
    const int64_t nr = m->nsr;
    const int grid = red_grid(nr > 0 ? nr : 1);
    unsigned *ctr = m->counters + 0;
    hb_prof_scope prof("assemble", s);
#define HB_ASM(SC, DM)                                                                                          \
    (contig ? assemble_surf_kernel<T, SC, DM, true><<<grid, HB_RED_THREADS, 0, s>>>(                           \
                  ys, m->srow_g, m->srowptr, nullptr, x, mdiag, lambda, y, nr, m->ax_partials, n_axp,          \
                  m->partials, ctr, st)                                                                         \
            : assemble_surf_kernel<T, SC, DM, false><<<grid, HB_RED_THREADS, 0, s>>>(                          \
                  ys, m->srow_g, m->srowptr, m->scols, x, mdiag, lambda, y, nr, m->ax_partials, n_axp,         \
                  m->partials, ctr, st))
    if (screen == 0) {
        if (dot_mode == HB_DOT_NONE) HB_ASM(0, HB_DOT_NONE);
        else if (dot_mode == HB_DOT_TO_TMP) HB_ASM(0, HB_DOT_TO_TMP);
        else HB_ASM(0, HB_DOT_CG_PAP);
    } else {
        if (dot_mode == HB_DOT_NONE) HB_ASM(1, HB_DOT_NONE);
        else if (dot_mode == HB_DOT_TO_TMP) HB_ASM(1, HB_DOT_TO_TMP);
        else HB_ASM(1, HB_DOT_CG_PAP);
    }
#undef HB_ASM
    HB_CHECK_LAUNCH();
    return HB_OK;
}

// The mesh's box as a lattice (DOF numbering of the node map: unmasked
// lattice points, first coordinate fastest).
static lattice_t mesh_lattice(const hb_mesh *m)
{
    const hb_mesh_desc &d = m->desc;
    lattice_t L;
    L.N = m->N;
    L.Ex = d.ex;
    L.Ey = d.ey;
    L.Ez = d.ez;
    const unsigned f = d.dirichlet_faces;
    L.x0 = (f & 1u) ? 1 : 0;
    L.y0 = (f & 4u) ? 1 : 0;
    L.z0 = (f & 16u) ? 1 : 0;
    L.NXu = m->N * d.ex + 1 - L.x0 - ((f & 2u) ? 1 : 0);
    L.NYu = m->N * d.ey + 1 - L.y0 - ((f & 8u) ? 1 : 0);
    L.NZu = m->N * d.ez + 1 - L.z0 - ((f & 32u) ? 1 : 0);
    return L;
}

// Z^T on every DOF by lattice arithmetic from the element-major local values.
template <typename T>
hb_status launch_assemble_grid(const hb_mesh *m, const T *yL, const T *x, T *y, const T *mdiag, int screen,
                               double lambda, hb_cg_state *st, int dot_mode, cudaStream_t s)
{
    const lattice_t L = mesh_lattice(m);
    const int grid = red_grid(m->n_global);
    unsigned *ctr = m->counters + 0;
    hb_prof_scope prof("assemble", s);
#define HB_ASM(SC, DM) \
    assemble_grid_kernel<T, SC, DM><<<grid, HB_RED_THREADS, 0, s>>>(yL, L, x, mdiag, lambda, y, m->partials, ctr, st)
    if (screen == 0) {
        if (dot_mode == HB_DOT_NONE) HB_ASM(0, HB_DOT_NONE);
        else if (dot_mode == HB_DOT_TO_TMP) HB_ASM(0, HB_DOT_TO_TMP);
        else HB_ASM(0, HB_DOT_CG_PAP);
    } else {
        if (dot_mode == HB_DOT_NONE) HB_ASM(1, HB_DOT_NONE);
        else if (dot_mode == HB_DOT_TO_TMP) HB_ASM(1, HB_DOT_TO_TMP);
        else HB_ASM(1, HB_DOT_CG_PAP);
    }
#undef HB_ASM
    HB_CHECK_LAUNCH();
    return HB_OK;
}

}  // namespace hb

using namespace hb;

// ---------------------------------------------------------------- internal entry points

hb_status hb_launch_assemble_f64(const hb_mesh *m, const double *yL, const double *x, double *y, int screen,
                                 double lambda, hb_cg_state *st, int dot_mode, cudaStream_t s)
{
    return launch_assemble<double>(m, yL, x, y, m->mdiag, screen, lambda, st, dot_mode, s);
}

hb_status hb_launch_assemble_f32(const hb_mesh *m, const float *yL, const float *x, float *y, int screen,
                                 double lambda, hb_cg_state *st, int dot_mode, cudaStream_t s)
{
    if (!m->mdiag32) { hb_set_error("mesh has no FP32 data (keep_fp32_copy = 0)"); return HB_ERR_ARG; }
    return launch_assemble<float>(m, yL, x, y, m->mdiag32, screen, lambda, st, dot_mode, s);
}

// A x: the element kernel, then Z^T. Pencil variants finish element-interior
// DOFs in the element kernel and gather only surface DOFs; variant 0 writes
// every local node and gathers all DOFs.
hb_status hb_apply_A_impl(const hb_mesh *m, hb_precision prec, int screen, double lambda, const void *x, void *y,
                          hb_cg_state *st, int dot_mode, cudaStream_t s)
{
    const int *run = (dot_mode == HB_DOT_CG_PAP && st) ? &st->run : nullptr;
    if (prec != HB_F64 && prec != HB_F32 && prec != HB_F64X) {
        hb_set_error("precision %d not valid for the operator", (int)prec);
        return HB_ERR_ARG;
    }
    if (prec == HB_F64X) {
        // double-float element kernel (pencil, even-odd) in its own variant's block shape
        const int v64 = m->variant[2];
        const int ebm = hb_variant_eb_mode(v64);
        if ((ebm & 8) && !m->spos) { hb_set_error("surface positions missing for variant %d", v64); return HB_ERR_ARG; }
        const bool grid = (ebm & 16) != 0;
        double *partials = (dot_mode != HB_DOT_NONE && !grid) ? m->ax_partials : nullptr;
        int64_t nblk = 0;
        hb_status r = hb_launch_ax2_f64x(m, (const double *)x, (double *)m->yL, (double *)y, lambda, screen,
                                         partials, run, ebm, s, &nblk);
        if (r != HB_OK) return r;
        if (grid)
            return launch_assemble_grid<double>(m, (const double *)m->yL, (const double *)x, (double *)y, m->mdiag,
                                                screen, lambda, st, dot_mode, s);
        return launch_assemble_surf<double>(m, (const double *)m->yL, (const double *)x, (double *)y, m->mdiag,
                                            screen, lambda, partials ? nblk : 0, st, dot_mode, s, (ebm & 8) != 0);
    }
    const int v = m->variant[hb_variant_slot(prec)];
    if (v & HB_VAR_TC) {
        if (prec != HB_F64) { hb_set_error("the tensor-core element kernel is FP64 only"); return HB_ERR_ARG; }
        const bool csr = (v & HB_VAR_CSR) != 0;
        if (csr && !m->spos) { hb_set_error("surface positions missing for variant %d", v); return HB_ERR_ARG; }
        double *partials = dot_mode != HB_DOT_NONE ? m->ax_partials : nullptr;
        int64_t nblk = 0;
        hb_status r = hb_launch_ax_tc_f64(m, (const double *)x, (double *)m->yL, (double *)y, lambda, screen,
                                          partials, run, csr, s, &nblk);
        if (r != HB_OK) return r;
        return launch_assemble_surf<double>(m, (const double *)m->yL, (const double *)x, (double *)y, m->mdiag,
                                            screen, lambda, partials ? nblk : 0, st, dot_mode, s, csr);
    }
    const int eo = (v & HB_VAR_EO) ? 1 : 0, ebm = hb_variant_eb_mode(v);
    if ((ebm & 8) && !m->spos) { hb_set_error("surface positions missing for variant %d", v); return HB_ERR_ARG; }
    hb_status r;
    if (!(v & HB_VAR_PENCIL)) {
        if (prec == HB_F64) {
            r = hb_launch_ax_local_f64(m, (const double *)x, (double *)m->yL, run, s);
            if (r != HB_OK) return r;
            return hb_launch_assemble_f64(m, (const double *)m->yL, (const double *)x, (double *)y, screen, lambda,
                                          st, dot_mode, s);
        }
        r = hb_launch_ax_local_f32(m, (const float *)x, (float *)m->yL, run, s);
        if (r != HB_OK) return r;
        return hb_launch_assemble_f32(m, (const float *)m->yL, (const float *)x, (float *)y, screen, lambda, st,
                                      dot_mode, s);
    }
    const bool grid = (ebm & 16) != 0;
    double *partials = (dot_mode != HB_DOT_NONE && !grid) ? m->ax_partials : nullptr;
    int64_t nblk = 0;
    if (prec == HB_F64) {
        r = hb_launch_ax2_f64(m, (const double *)x, (double *)m->yL, (double *)y, lambda, screen, partials, run, eo,
                              ebm, s, &nblk);
        if (r != HB_OK) return r;
        if (grid)
            return launch_assemble_grid<double>(m, (const double *)m->yL, (const double *)x, (double *)y, m->mdiag,
                                                screen, lambda, st, dot_mode, s);
        return launch_assemble_surf<double>(m, (const double *)m->yL, (const double *)x, (double *)y, m->mdiag,
                                            screen, lambda, partials ? nblk : 0, st, dot_mode, s, (ebm & 8) != 0);
    }
    if (!m->mdiag32) { hb_set_error("mesh has no FP32 data (keep_fp32_copy = 0)"); return HB_ERR_ARG; }
    r = hb_launch_ax2_f32(m, (const float *)x, (float *)m->yL, (float *)y, lambda, screen, partials, run, eo, ebm, s,
                          &nblk);
    if (r != HB_OK) return r;
    if (grid)
        return launch_assemble_grid<float>(m, (const float *)m->yL, (const float *)x, (float *)y, m->mdiag32, screen,
                                           lambda, st, dot_mode, s);
    return launch_assemble_surf<float>(m, (const float *)m->yL, (const float *)x, (float *)y, m->mdiag32, screen,
                                       lambda, partials ? nblk : 0, st, dot_mode, s, (ebm & 8) != 0);
}

hb_status hb_launch_dot_f64(const hb_mesh *m, const double *a, const double *b, int64_t n, double *out,
                            cudaStream_t s)
{
    hb_prof_scope prof("dot", s);
    dot_kernel<double><<<red_grid(n), HB_RED_THREADS, 0, s>>>(a, b, n, out, m->partials, m->counters + 1);
    HB_CHECK_LAUNCH();
    return HB_OK;
}

hb_status hb_launch_dot_f32(const hb_mesh *m, const float *a, const float *b, int64_t n, double *out,
                            cudaStream_t s)
{
    hb_prof_scope prof("dot", s);
    dot_kernel<float><<<red_grid(n), HB_RED_THREADS, 0, s>>>(a, b, n, out, m->partials, m->counters + 1);
    HB_CHECK_LAUNCH();
    return HB_OK;
}

// ---------------------------------------------------------------- C ABI

static bool valid_screen(int s) { return s == HB_SCREEN_IDENTITY || s == HB_SCREEN_MASS; }

extern "C" hb_status hb_set_kernel_variant(hb_mesh *m, hb_precision prec, int variant)
{
    hb_clear_error();
    if (!m) { hb_set_error("null mesh"); return HB_ERR_ARG; }
    const int slot = hb_variant_slot(prec);
    if (slot < 0) { hb_set_error("variant precision must be HB_F64, HB_F32 or HB_F64X"); return HB_ERR_ARG; }
    if (!hb_valid_variant(variant) || (prec == HB_F64X && !hb_valid_variant_f64x(variant))) {
        hb_set_error("invalid kernel variant %d for precision %d", variant, (int)prec);
        return HB_ERR_ARG;
    }
    if ((variant & HB_VAR_TC) && (prec != HB_F64 || m->N != 7)) {
        hb_set_error("the tensor-core element kernel (variant %d) is built for HB_F64 at N = 7", HB_VAR_TC);
        return HB_ERR_ARG;
    }
    if (variant & HB_VAR_CSR) {
        hb_device_guard dg(m->device);
        hb_status st = hb_mesh_ensure_spos(m, nullptr);
        if (st != HB_OK) return st;
    }
    m->variant[slot] = variant;
    return HB_OK;
}

extern "C" hb_status hb_get_kernel_variant(const hb_mesh *m, hb_precision prec, int *variant)
{
    if (!m || !variant) { hb_set_error("null argument"); return HB_ERR_ARG; }
    const int slot = hb_variant_slot(prec);
    if (slot < 0) { hb_set_error("variant precision must be HB_F64, HB_F32 or HB_F64X"); return HB_ERR_ARG; }
    *variant = m->variant[slot];
    return HB_OK;
}

extern "C" hb_status hb_apply_A(const hb_mesh *m, hb_precision prec, hb_screen screen, double lambda,
                                const void *x, void *y, void *stream)
{
    hb_clear_error();
    if (!m || (!x && m->n_global) || (!y && m->n_global)) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!valid_screen(screen)) { hb_set_error("bad screen mode %d", (int)screen); return HB_ERR_ARG; }
    if (prec != HB_F64 && prec != HB_F32 && prec != HB_F64X) {
        hb_set_error("hb_apply_A takes HB_F64, HB_F32 or HB_F64X");
        return HB_ERR_ARG;
    }
    if (m->n_global == 0) return HB_OK;
    const size_t esz = prec == HB_F32 ? 4 : 8;
    const char *xa = (const char *)x, *ya = (const char *)y;
    if (xa < ya + esz * m->n_global && ya < xa + esz * m->n_global) { hb_set_error("x and y overlap"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    return hb_apply_A_impl(m, prec, screen, lambda, x, y, nullptr, HB_DOT_NONE, (cudaStream_t)stream);
}

extern "C" hb_status hb_dot(const hb_mesh *m, hb_precision prec, const void *a, const void *b, double *out_dev,
                            double *out_host, void *stream)
{
    hb_clear_error();
    if (!m || ((!a || !b) && m->n_global)) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (prec != HB_F64 && prec != HB_F32) { hb_set_error("hb_dot takes HB_F64 or HB_F32"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    double *dst = out_dev ? out_dev : &m->state[1].dot_tmp;
    if (m->n_global == 0) {
        HB_TRY_CUDA(cudaMemsetAsync(dst, 0, sizeof(double), s));
    } else {
        hb_status r = prec == HB_F64
                          ? hb_launch_dot_f64(m, (const double *)a, (const double *)b, m->n_global, dst, s)
                          : hb_launch_dot_f32(m, (const float *)a, (const float *)b, m->n_global, dst, s);
        if (r != HB_OK) return r;
    }
    if (out_host) {
        HB_TRY_CUDA(cudaMemcpyAsync(out_host, dst, sizeof(double), cudaMemcpyDeviceToHost, s));
        HB_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return HB_OK;
}

// Error word the kernels set when a bounded wait gave up (bit 0: a
// staged-pipeline wait, bit 1: a fused-CG grid barrier); read and cleared at
// the solvers' sync points.
static hb_status check_dev_err(hb_mesh *m, cudaStream_t s)
{
    unsigned v = 0;
    HB_TRY_CUDA(cudaMemcpyAsync(&v, m->counters + 7, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    if (v) {
        HB_TRY_CUDA(cudaMemsetAsync(m->counters + 7, 0, sizeof(unsigned), s));
        hb_set_error("a kernel gave up waiting (%s)", (v & 2u) ? "fused CG grid barrier" : "staged data");
        return HB_ERR_TIMEOUT;
    }
    return HB_OK;
}

// ---------------------------------------------------------------- autotuner

extern "C" hb_status hb_autotune(hb_mesh *m, hb_precision prec, hb_screen screen, double lambda, int reps,
                                 int *best_variant, double *ms_per_variant, void *stream)
{
    hb_clear_error();
    if (!m) { hb_set_error("null mesh"); return HB_ERR_ARG; }
    if (hb_variant_slot(prec) < 0) { hb_set_error("hb_autotune takes HB_F64, HB_F32 or HB_F64X"); return HB_ERR_ARG; }
    if (prec == HB_F32 && !m->geo32) { hb_set_error("HB_F32 needs keep_fp32_copy"); return HB_ERR_ARG; }
    if (!valid_screen(screen)) { hb_set_error("bad screen mode"); return HB_ERR_ARG; }
    if (reps < 1) reps = 1;
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int pi = hb_variant_slot(prec);
    const int64_t n = m->n_global;
    const size_t esz = prec == HB_F32 ? 4 : 8;
    if (n == 0) {
        if (best_variant) *best_variant = m->variant[pi];
        return HB_OK;
    }
    void *x = nullptr, *y = nullptr;
    HB_TRY_CUDA(cudaMalloc(&x, esz * n));
    cudaError_t e = cudaMalloc(&y, esz * n);
    if (e == cudaSuccess) e = cudaMemsetAsync(x, 0, esz * n, s);
    if (e != cudaSuccess) {
        cudaFree(x);
        cudaFree(y);
        hb_set_error("autotune scratch: %s", cudaGetErrorString(e));
        return HB_ERR_NOMEM;
    }
    const int candidates[] = {0, HB_VAR_PENCIL, HB_VAR_PENCIL | HB_VAR_EO, HB_VAR_PENCIL | HB_VAR_EB2,
                              HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_EB2, HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_ONE,
                              HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_TMA, HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_WS,
                              HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_CSR,
                              HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_ONE | HB_VAR_CSR,
                              HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_GRID,
                              HB_VAR_PENCIL | HB_VAR_EO | HB_VAR_ONE | HB_VAR_GRID, HB_VAR_TC,
                              HB_VAR_TC | HB_VAR_CSR};
    {
        hb_status sp = hb_mesh_ensure_spos(m, s);
        if (sp != HB_OK) {
            cudaFree(x);
            cudaFree(y);
            return sp;
        }
    }
    const int saved = m->variant[pi];
    int best = saved;
    float best_ms = 1e30f;
    hb_status st = HB_OK;
    // each application also reduces x.y, as every CG iteration does (p.Ap):
    // variants differ in where that work runs (element kernel or gather)
    hb_cg_state *tmp = m->state + 1;
    for (int c : candidates) {
        if ((c & HB_VAR_TC) && (prec != HB_F64 || m->N != 7)) continue;
        if (prec == HB_F64X && !hb_valid_variant_f64x(c)) continue;
        m->variant[pi] = c;
        // one untimed application (first launch, attribute setup), then `reps` timed ones
        st = hb_apply_A_impl(m, prec, screen, lambda, x, y, tmp, HB_DOT_TO_TMP, s);
        if (st != HB_OK) break;
        if ((e = cudaEventRecord(m->ev0, s)) != cudaSuccess) break;
        for (int r = 0; r < reps && st == HB_OK; r++)
            st = hb_apply_A_impl(m, prec, screen, lambda, x, y, tmp, HB_DOT_TO_TMP, s);
        if (st != HB_OK) break;
        if ((e = cudaEventRecord(m->ev1, s)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(m->ev1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, m->ev0, m->ev1)) != cudaSuccess) break;
        ms /= reps;
        if (ms_per_variant) ms_per_variant[c] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaFree(x);
    cudaFree(y);
    if (st == HB_OK && e != cudaSuccess) {
        hb_set_error("autotune: %s", cudaGetErrorString(e));
        st = HB_ERR_CUDA;
    }
    if (st == HB_OK) st = check_dev_err(m, s);
    m->variant[pi] = st == HB_OK ? best : saved;
    if (best_variant) *best_variant = m->variant[pi];
    // the surface positions were built for the timing; keep them only if used
    if (m->spos && !((m->variant[0] | m->variant[1] | m->variant[2]) & HB_VAR_CSR)) {
        cudaStreamSynchronize(s);
        hb_mesh_drop_graphs(m);
        cudaFree(m->spos);
        m->spos = nullptr;
        m->device_bytes -= sizeof(int32_t) * (size_t)(m->E * (int64_t)hb_surf_count(m->N));
    }
    return st;
}

// Workspace vectors for the solvers, grown on demand (FP64 r, p, Ap; FP32 r, p,
// Ap, d), each starting on a 256-byte boundary.
static inline int64_t cg_stride(int64_t n) { return (n + 63) / 64 * 64; }
// Workspace vectors for the solvers, grown on demand (FP64 r, p, Ap; FP32 r, p, Ap, d).
static hb_status cg_workspace(hb_mesh *m)
{
    const size_t need = (size_t)cg_stride(m->n_global) * (4 * sizeof(double) + 5 * sizeof(float)) + 256;
    if (m->cg_vec_bytes >= need) return HB_OK;
    if (m->cg_vec) cudaFree(m->cg_vec);
    m->cg_vec = nullptr;
    m->cg_vec_bytes = 0;
    HB_TRY_CUDA(cudaMalloc(&m->cg_vec, need));
    m->cg_vec_bytes = need;
    return HB_OK;
}

// Enqueues `count` iterations of Algorithm 1 on the vectors (x, r, p, Ap);
// with inv_d (the Jacobi preconditioner) z = M^-1 r is kept in z.
template <typename T>
static hb_status cg_iterations(const hb_mesh *m, hb_precision prec, int screen, double lambda, T *x, T *r, T *p,
                               T *Ap, T *z, const T *inv_d, hb_cg_state *st, int count, cudaStream_t s)
{
    const int64_t n = m->n_global;
    const int grid = red_grid(n);
    for (int it = 0; it < count; it++) {
        hb_status rs = hb_apply_A_impl(m, prec, screen, lambda, p, Ap, st, HB_DOT_CG_PAP, s);
        if (rs != HB_OK) return rs;
        {
            hb_prof_scope prof("cg_update_r", s);
            if (inv_d)
                cg_update_r_kernel<T, true><<<grid, HB_RED_THREADS, 0, s>>>(r, Ap, z, inv_d, n, m->partials,
                                                                            m->counters + 2, st);
            else
                cg_update_r_kernel<T, false><<<grid, HB_RED_THREADS, 0, s>>>(r, Ap, nullptr, nullptr, n, m->partials,
                                                                             m->counters + 2, st);
            HB_CHECK_LAUNCH();
        }
        {
            hb_prof_scope prof("cg_update_xp", s);
            cg_update_xp_kernel<T><<<grid, HB_RED_THREADS, 0, s>>>(x, p, inv_d ? z : r, n, m->counters + 3, st);
            HB_CHECK_LAUNCH();
        }
    }
    return HB_OK;
}

// A run of `count` iterations as a CUDA graph, captured on the mesh's own
// stream the first time a (vectors, state, precision, screening, lambda,
// count, kernel variant) combination is seen and replayed while it stays the
// same; ordered after and before the caller's stream with events. Used unless
// per-kernel timing is on (its event pairs are not captured).
template <typename T>
static hb_status cg_iterations_graph(const hb_mesh *mc, hb_precision prec, int screen, double lambda, T *x, T *r,
                                     T *p, T *Ap, T *z, const T *inv_d, hb_cg_state *st, int count, cudaStream_t s)
{
    hb_mesh *m = const_cast<hb_mesh *>(mc);
    const int gi = prec == HB_F32 ? 1 : 0;
    hb_mesh::cg_graph &G = m->graphs[gi];
    const int variant = m->variant[hb_variant_slot(prec)];
    if (!m->cg_stream) {
        HB_TRY_CUDA(cudaStreamCreateWithFlags(&m->cg_stream, cudaStreamNonBlocking));
        HB_TRY_CUDA(cudaEventCreateWithFlags(&m->cg_ev[0], cudaEventDisableTiming));
        HB_TRY_CUDA(cudaEventCreateWithFlags(&m->cg_ev[1], cudaEventDisableTiming));
    }
    const bool hit = G.exec && G.x == x && G.r == r && G.p == p && G.Ap == Ap && G.z == z && G.inv_d == inv_d &&
                     G.st == st && G.prec == prec &&
                     G.screen == screen && G.count == count && G.variant == variant && G.lambda == lambda;
    if (!hit) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
        const unsigned long long before = hb_kernel_launches();
        HB_TRY_CUDA(cudaStreamBeginCapture(m->cg_stream, cudaStreamCaptureModeThreadLocal));
        hb_status rs = cg_iterations<T>(m, prec, screen, lambda, x, r, p, Ap, z, inv_d, st, count, m->cg_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(m->cg_stream, &g);
        if (rs != HB_OK) {
            if (g) cudaGraphDestroy(g);
            return rs;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            hb_set_error("CG graph: %s", cudaGetErrorString(e));
            return HB_ERR_CUDA;
        }
        G.launches = hb_kernel_launches() - before;
        G.x = x; G.r = r; G.p = p; G.Ap = Ap; G.z = z; G.inv_d = inv_d; G.st = st;
        G.prec = prec; G.screen = screen; G.count = count; G.variant = variant; G.lambda = lambda;
        // the captured launches were counted once at capture, for this first replay
    } else {
        hb_count_launches(G.launches);
    }
    HB_TRY_CUDA(cudaEventRecord(m->cg_ev[0], s));
    HB_TRY_CUDA(cudaStreamWaitEvent(m->cg_stream, m->cg_ev[0], 0));
    HB_TRY_CUDA(cudaGraphLaunch(G.exec, m->cg_stream));
    HB_TRY_CUDA(cudaEventRecord(m->cg_ev[1], m->cg_stream));
    HB_TRY_CUDA(cudaStreamWaitEvent(s, m->cg_ev[1], 0));
    return HB_OK;
}

// Runs iterations until the device state says stop; returns the final state.
template <typename T>
static hb_status cg_drive(const hb_mesh *m, hb_precision prec, int screen, double lambda, T *x, T *r, T *p, T *Ap,
                          T *z, const T *inv_d, hb_cg_state *st, int max_it, cudaStream_t s, hb_cg_state *out)
{
    int done = 0;
    const int chunk_first = 25;
    HB_TRY_CUDA(cudaMemcpyAsync(m->state_host, st, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    while (m->state_host->run && done < max_it) {
        int count = max_it - done;
        if (count > chunk_first && m->state_host->tol2 > 0.0) count = chunk_first;
        hb_status rs = hb_profiling_on()
                           ? cg_iterations<T>(m, prec, screen, lambda, x, r, p, Ap, z, inv_d, st, count, s)
                           : cg_iterations_graph<T>(m, prec, screen, lambda, x, r, p, Ap, z, inv_d, st, count, s);
        if (rs != HB_OK) return rs;
        done += count;
        HB_TRY_CUDA(cudaMemcpyAsync(m->state_host, st, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
        HB_TRY_CUDA(cudaStreamSynchronize(s));
    }
    *out = *m->state_host;
    return HB_OK;
}

// The true residual of the iterate x: r = b - A x with the FP64 operator
// (whatever precision the iterations ran in), z = M^-1 r, p = z, r.z and r.r
// into the state, which keeps the iteration count; run is set again while the
// true residual is above the tolerance and iterations remain (a restart of
// Algorithm 1 from x). Synchronises s; returns the state in *out.
static hb_status cg_true_residual(const hb_mesh *m, const hb_cg_opts *o, const double *b, const double *x, double *r,
                                  double *p, double *Ap, double *z, const double *inv_d, hb_cg_state *st,
                                  cudaStream_t s, hb_cg_state *out)
{
    const int64_t n = m->n_global;
    hb_status rs = hb_apply_A_impl(m, HB_F64, o->screen, o->lambda, x, Ap, nullptr, HB_DOT_NONE, s);
    if (rs != HB_OK) return rs;
    hb_count_launch();
    cg_restart_kernel<<<red_grid(n), HB_RED_THREADS, 0, s>>>(b, Ap, r, p, z, inv_d, n, m->partials,
                                                              m->counters + 2, st);
    HB_CHECK_LAUNCH();
    HB_TRY_CUDA(cudaMemcpyAsync(m->state_host, st, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    *out = *m->state_host;
    return HB_OK;
}

// Fused CG: FP64 without a preconditioner, when every element of the mesh
// fits in one cooperative launch (one per block; mode 0: and the mesh is
// small enough that latency sets the time, at most 300 elements, where it
// measured faster than the launched kernels; mode 2: whenever it fits).
static bool use_fused_cg(const hb_mesh *m, const hb_cg_opts *o)
{
    if (o->prec != HB_F64 || o->precond || m->fused_mode == 1) return false;
    const int64_t groups = m->E;  // one element per block
    const int cap = hb_cg_fused_capacity(m->N);
    if (cap <= 0 || groups > cap) return false;
    return m->fused_mode == 2 || groups <= 300;
}

extern "C" hb_status hb_cg_solve(const hb_mesh *mc, const hb_cg_opts *o, const double *b, double *x,
                                 hb_cg_result *res, void *stream)
{
    hb_clear_error();
    hb_mesh *m = const_cast<hb_mesh *>(mc);
    if (!m || !o || ((!b || !x) && m->n_global)) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!valid_screen(o->screen)) { hb_set_error("bad screen mode"); return HB_ERR_ARG; }
    if (o->prec != HB_F64 && o->prec != HB_MIXED && o->prec != HB_F64X) {
        hb_set_error("hb_cg_solve takes HB_F64, HB_F64X or HB_MIXED");
        return HB_ERR_ARG;
    }
    if (o->max_it < 0 || !(o->rtol >= 0.0)) { hb_set_error("bad max_it or rtol"); return HB_ERR_ARG; }
    if (o->precond != 0 && o->precond != 1) { hb_set_error("precond must be 0 or 1"); return HB_ERR_ARG; }
    if (o->prec == HB_MIXED && (!m->geo32 || !m->mdiag32)) { hb_set_error("HB_MIXED needs keep_fp32_copy"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    hb_cg_result R{};
    R.status = HB_OK;
    const int64_t n = m->n_global;
    if (n == 0) {
        if (res) *res = R;
        return HB_OK;
    }
    hb_status rs = cg_workspace(m);
    if (rs != HB_OK) return rs;
    const int64_t ns = cg_stride(n);
    double *r = (double *)m->cg_vec, *p = r + ns, *Ap = p + ns, *z = Ap + ns;
    float *r32 = (float *)(z + ns), *p32 = r32 + ns, *Ap32 = p32 + ns, *d32 = Ap32 + ns, *z32 = d32 + ns;
    if (o->precond) {
        rs = hb_mesh_inv_diag(m, o->screen, o->lambda, s);
        if (rs != HB_OK) return rs;
    }
    const double *inv_d = o->precond ? m->inv_diag : nullptr;
    const float *inv_d32 = o->precond ? m->inv_diag32 : nullptr;
    const int grid = red_grid(n);
    hb_cg_state *st = m->state, *st_in = m->state + 1;
    HB_TRY_CUDA(cudaEventRecord(m->ev0, s));
    hb_cg_state fin{};
    if (o->prec == HB_F64 || o->prec == HB_F64X) {
        // r0 = b - A x0, p = r0 (the start of Algorithm 1)
        rs = hb_apply_A_impl(m, o->prec, o->screen, o->lambda, x, Ap, nullptr, HB_DOT_NONE, s);
        if (rs != HB_OK) return rs;
        hb_count_launch();
        cg_init_kernel<<<grid, HB_RED_THREADS, 0, s>>>(b, Ap, r, p, inv_d, n, o->rtol, o->max_it, m->partials,
                                                       m->counters + 2, st);
        HB_CHECK_LAUNCH();
        if (use_fused_cg(m, o)) {
            rs = hb_cg_fused_run(m, o->screen, o->lambda, x, r, p, Ap, st, s);
            if (rs != HB_OK) return rs;
            HB_TRY_CUDA(cudaMemcpyAsync(m->state_host, st, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
            HB_TRY_CUDA(cudaStreamSynchronize(s));
            fin = *m->state_host;
        } else {
            rs = cg_drive<double>(m, o->prec, o->screen, o->lambda, x, r, p, Ap, z, inv_d, st, o->max_it, s, &fin);
            if (rs != HB_OK) return rs;
        }
        // With a tolerance, the stop is decided on the true residual b - A x
        // (FP64 operator): where the recursive residual met it and the true
        // one does not, Algorithm 1 restarts from x with the true residual
        // (each pass adds at least one iteration, up to max_it). A restart
        // that does not lower the true residual by a tenth of its norm ends
        // the solve (HB_ERR_NOT_CONVERGED): the operator's rounding floor is
        // then above the tolerance.
        if (o->rtol > 0.0) {
            double prev = -1.0;
            while (fin.status == HB_OK) {
                rs = cg_true_residual(m, o, b, x, r, p, Ap, z, inv_d, st, s, &fin);
                if (rs != HB_OK) return rs;
                if (!fin.run) break;
                if (prev >= 0.0 && fin.res2 > 0.81 * prev) break;
                prev = fin.res2;
                rs = cg_drive<double>(m, o->prec, o->screen, o->lambda, x, r, p, Ap, z, inv_d, st,
                                      o->max_it - fin.it, s, &fin);
                if (rs != HB_OK) return rs;
            }
        }
        R.iters = fin.it;
        R.rel_res = fin.bb > 0.0 ? sqrt(fin.res2 / fin.bb) : 0.0;
        if (fin.status == HB_ERR_BREAKDOWN) R.status = HB_ERR_BREAKDOWN;
        else if (o->rtol > 0.0 && fin.res2 > fin.tol2) R.status = HB_ERR_NOT_CONVERGED;
    } else {
        const double rtol_in = o->inner_rtol > 0.0 ? o->inner_rtol : 1e-4;
        const int max_outer = o->max_outer > 0 ? o->max_outer : 30;
        int used = 0, outer = 0;
        double rel = 0.0;
        for (;;) {
            rs = hb_apply_A_impl(m, HB_F64, o->screen, o->lambda, x, Ap, nullptr, HB_DOT_NONE, s);
            if (rs != HB_OK) return rs;
            hb_count_launch();
            residual_kernel<<<grid, HB_RED_THREADS, 0, s>>>(b, Ap, r, n, m->partials, m->counters + 2, st);
            HB_CHECK_LAUNCH();
            HB_TRY_CUDA(cudaMemcpyAsync(m->state_host, st, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
            HB_TRY_CUDA(cudaStreamSynchronize(s));
            const double rr = m->state_host->rr, bb = m->state_host->bb;
            // a non-finite b or residual (bb NaN would make rel 0 below) is a breakdown
            if (!std::isfinite(rr) || !std::isfinite(bb)) { R.status = HB_ERR_BREAKDOWN; rel = rr; break; }
            rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
            if (!std::isfinite(rel)) { R.status = HB_ERR_BREAKDOWN; break; }
            if (bb == 0.0 || rr <= o->rtol * o->rtol * bb) break;
            if (outer >= max_outer || used >= o->max_it) { R.status = HB_ERR_NOT_CONVERGED; break; }
            hb_count_launch();
            inner_init_kernel<<<grid, HB_RED_THREADS, 0, s>>>(r, r32, p32, d32, inv_d32, n, rtol_in,
                                                              o->max_it - used, m->partials, m->counters + 2, st,
                                                              st_in);
            HB_CHECK_LAUNCH();
            rs = cg_drive<float>(m, HB_F32, o->screen, o->lambda, d32, r32, p32, Ap32, z32, inv_d32, st_in,
                                 o->max_it - used, s, &fin);
            if (rs != HB_OK) return rs;
            used += fin.it;
            outer++;
            if (fin.status == HB_ERR_BREAKDOWN && fin.it == 0) { R.status = HB_ERR_BREAKDOWN; break; }
            hb_count_launch();
            update_x_kernel<<<grid, HB_RED_THREADS, 0, s>>>(x, d32, n, st);
            HB_CHECK_LAUNCH();
        }
        R.iters = used;
        R.outer_iters = outer;
        R.rel_res = rel;
    }
    HB_TRY_CUDA(cudaEventRecord(m->ev1, s));
    HB_TRY_CUDA(cudaEventSynchronize(m->ev1));
    float ms = 0.f;
    HB_TRY_CUDA(cudaEventElapsedTime(&ms, m->ev0, m->ev1));
    R.time_ms = ms;
    {
        const hb_status de = check_dev_err(m, s);
        if (de != HB_OK) R.status = de;
    }
    if (res) *res = R;
    return R.status;
}

extern "C" hb_status hb_set_cg_fused(hb_mesh *m, int mode)
{
    hb_clear_error();
    if (!m) { hb_set_error("null mesh"); return HB_ERR_ARG; }
    if (mode < 0 || mode > 2) { hb_set_error("fused mode must be 0, 1 or 2"); return HB_ERR_ARG; }
    m->fused_mode = mode;
    return HB_OK;
}

// ---------------------------------------------------------------- stepwise solve

extern "C" hb_status hb_cg_begin(hb_mesh *m, const hb_cg_opts *o, const double *b, double *x, void *stream)
{
    hb_clear_error();
    if (!m || !o || ((!b || !x) && m->n_global)) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!valid_screen(o->screen)) { hb_set_error("bad screen mode"); return HB_ERR_ARG; }
    if (o->prec != HB_F64 && o->prec != HB_F64X) { hb_set_error("hb_cg_begin takes HB_F64 or HB_F64X"); return HB_ERR_ARG; }
    if (o->max_it < 0 || !(o->rtol >= 0.0)) { hb_set_error("bad max_it or rtol"); return HB_ERR_ARG; }
    if (o->precond != 0 && o->precond != 1) { hb_set_error("precond must be 0 or 1"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    m->step.active = 0;
    const int64_t n = m->n_global;
    hb_status rs = cg_workspace(m);
    if (rs != HB_OK) return rs;
    if (o->precond) {
        rs = hb_mesh_inv_diag(m, o->screen, o->lambda, s);
        if (rs != HB_OK) return rs;
    }
    if (n > 0) {
        const int64_t ns = cg_stride(n);
        double *r = (double *)m->cg_vec, *p = r + ns, *Ap = p + ns;
        rs = hb_apply_A_impl(m, o->prec, o->screen, o->lambda, x, Ap, nullptr, HB_DOT_NONE, s);
        if (rs != HB_OK) return rs;
        hb_count_launch();
        cg_init_kernel<<<red_grid(n), HB_RED_THREADS, 0, s>>>(b, Ap, r, p, o->precond ? m->inv_diag : nullptr, n,
                                                              o->rtol, o->max_it, m->partials, m->counters + 2,
                                                              m->state);
        HB_CHECK_LAUNCH();
    }
    m->step.active = 1;
    m->step.o = *o;
    m->step.b = b;
    m->step.x = x;
    m->step.done = 0;
    return HB_OK;
}

extern "C" hb_status hb_cg_iterate(hb_mesh *m, int count, void *stream)
{
    hb_clear_error();
    if (!m) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!m->step.active) { hb_set_error("no stepwise solve begun on this mesh"); return HB_ERR_ARG; }
    if (count < 0) { hb_set_error("count < 0"); return HB_ERR_ARG; }
    const hb_cg_opts &o = m->step.o;
    count = std::min(count, o.max_it - m->step.done);
    if (count <= 0 || m->n_global == 0) return HB_OK;
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t ns = cg_stride(m->n_global);
    double *r = (double *)m->cg_vec, *p = r + ns, *Ap = p + ns, *z = Ap + ns;
    const double *inv_d = o.precond ? m->inv_diag : nullptr;
    double *x = m->step.x;
    hb_status rs = hb_profiling_on()
                       ? cg_iterations<double>(m, o.prec, o.screen, o.lambda, x, r, p, Ap, z, inv_d, m->state, count,
                                               s)
                       : cg_iterations_graph<double>(m, o.prec, o.screen, o.lambda, x, r, p, Ap, z, inv_d, m->state,
                                                     count, s);
    if (rs != HB_OK) return rs;
    m->step.done += count;
    return HB_OK;
}

extern "C" hb_status hb_cg_finish(hb_mesh *m, hb_cg_result *res, void *stream)
{
    hb_clear_error();
    if (!m) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!m->step.active) { hb_set_error("no stepwise solve begun on this mesh"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    m->step.active = 0;
    hb_cg_result R{};
    R.status = HB_OK;
    if (m->n_global > 0) {
        HB_TRY_CUDA(cudaMemcpyAsync(m->state_host, m->state, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
        HB_TRY_CUDA(cudaStreamSynchronize(s));
        hb_cg_state fin = *m->state_host;
        const hb_cg_opts &o = m->step.o;
        if (o.rtol > 0.0 && fin.status == HB_OK) {
            // report the true residual b - A x (no restart: the iterations are over)
            const int64_t ns = cg_stride(m->n_global);
            double *r = (double *)m->cg_vec, *p = r + ns, *Ap = p + ns, *z = Ap + ns;
            hb_status rs = cg_true_residual(m, &o, m->step.b, m->step.x, r, p, Ap, z,
                                            o.precond ? m->inv_diag : nullptr, m->state, s, &fin);
            if (rs != HB_OK) return rs;
        }
        R.iters = fin.it;
        R.rel_res = fin.bb > 0.0 ? sqrt(fin.res2 / fin.bb) : 0.0;
        if (fin.status == HB_ERR_BREAKDOWN) R.status = HB_ERR_BREAKDOWN;
        else if (o.rtol > 0.0 && fin.res2 > fin.tol2) R.status = HB_ERR_NOT_CONVERGED;
        const hb_status de = check_dev_err(m, s);
        if (de != HB_OK) R.status = de;
    }
    if (res) *res = R;
    return R.status;
}

// ---------------------------------------------------------------- dot without any allocation
//
// hb_dot needs a mesh, and a mesh holds device memory the library allocated.
// hb_dot_noalloc serves callers that may not allocate device memory at all:
// for instance an application whose own allocator has reserved the whole
// device (a caching allocator, or a serving loop that admits work against a
// fixed memory budget), where a cudaMalloc would fail or break the budget,
// or a latency-critical loop that cannot afford the device-wide
// synchronisation cudaMalloc and cudaFree can cause. Its scratch (one
// partial sum per block, the arrival counter and a result slot) lives in the
// file-scope array below, which every GPU that loads this library holds
// until the process exits.
#define HB_DOT_NOALLOC_BLOCKS 16384  // partial sums: 128 KB per device
#define HB_DOT_NOALLOC_MAX_N ((int64_t)HB_DOT_NOALLOC_BLOCKS * HB_RED_THREADS * 4)

static __device__ __align__(256) double g_dot_noalloc_scratch[HB_DOT_NOALLOC_BLOCKS + 32];

static std::mutex g_dot_noalloc_mu;
static double *g_dot_noalloc_ptr[64];  // device address of the array, per device

// Device address of the scratch array on the current device. Taken once per
// device, with that device current; host code must not use the array's name
// as a device pointer.
static hb_status dot_noalloc_scratch(double **out)
{
    int dev = -1;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { hb_set_error("hb_dot_noalloc: device index %d not supported", dev); return HB_ERR_ARG; }
    std::lock_guard<std::mutex> lk(g_dot_noalloc_mu);
    if (!g_dot_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dot_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            hb_set_error("hb_dot_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return HB_ERR_CUDA;
        }
        g_dot_noalloc_ptr[dev] = (double *)p;
    }
    *out = g_dot_noalloc_ptr[dev];
    return HB_OK;
}

extern "C" hb_status hb_dot_noalloc(hb_precision prec, const void *a, const void *b, int64_t n, double *out_dev,
                                    double *out_host, void *stream)
{
    hb_clear_error();
    if (n < 0) { hb_set_error("hb_dot_noalloc: n = %lld is negative", (long long)n); return HB_ERR_ARG; }
    if (n > HB_DOT_NOALLOC_MAX_N) {
        hb_set_error("hb_dot_noalloc: n = %lld exceeds the maximum of %lld elements its static scratch serves",
                     (long long)n, (long long)HB_DOT_NOALLOC_MAX_N);
        return HB_ERR_ARG;
    }
    if (n > 0 && (!a || !b)) { hb_set_error("hb_dot_noalloc: null vector"); return HB_ERR_ARG; }
    if (prec != HB_F64 && prec != HB_F32) { hb_set_error("hb_dot_noalloc takes HB_F64 or HB_F32"); return HB_ERR_ARG; }
    double *scratch = nullptr;
    hb_status st = dot_noalloc_scratch(&scratch);
    if (st != HB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + HB_DOT_NOALLOC_BLOCKS);
    double *result = out_dev ? out_dev : scratch + HB_DOT_NOALLOC_BLOCKS + 16;
    // the array keeps the previous call's contents: the arrival counter must start at zero
    HB_TRY_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
    if (n == 0) {
        HB_TRY_CUDA(cudaMemsetAsync(result, 0, sizeof(double), s));
    } else {
        // one block per 1024 elements: the same grid as hb_dot up to 1216 blocks
        const int blocks = (int)((n + HB_RED_THREADS * 4 - 1) / (HB_RED_THREADS * 4));
        hb_count_launch();
        if (prec == HB_F64)
            dot_kernel<double><<<blocks, HB_RED_THREADS, 0, s>>>((const double *)a, (const double *)b, n, result,
                                                                 scratch, counter);
        else
            dot_kernel<float><<<blocks, HB_RED_THREADS, 0, s>>>((const float *)a, (const float *)b, n, result,
                                                                scratch, counter);
        HB_CHECK_LAUNCH();
    }
    if (out_host) {
        HB_TRY_CUDA(cudaMemcpyAsync(out_host, result, sizeof(double), cudaMemcpyDeviceToHost, s));
        HB_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return HB_OK;
}
