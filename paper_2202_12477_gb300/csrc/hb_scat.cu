// Scattered (NekBone) storage of the DOF vectors, hipBone Sec. 2 and Sec. 3.1:
// vectors hold x_L = Z x_G (n_local entries), the operator is
// b_L = (Z Z^T S_L + lambda I) x_L and inner products are weighted by the
// inverse multiplicity. Kept beside the assembled path to measure what the
// paper's switch to assembled storage saves on GB300.
//
// Per application: the pencil element kernel on x_L (no l2g gather) finishes
// element-interior nodes (one copy each) and writes surface nodes to ysurf;
// the gather-scatter kernel sums each surface DOF's copies in element order,
// adds the screening term and writes the sum to every copy, and zeroes the
// masked (Dirichlet) nodes.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hb_internal.h"
#include "hb_vec.cuh"

struct hb_scat {
    const hb_mesh *m = nullptr;
    int device = 0;
    int64_t n_local = 0, n_masked = 0;
    double *w = nullptr;         // [n_local] 1 / multiplicity, 0 at masked nodes
    int32_t *sloc = nullptr;     // [nnz_s] local index of each surface copy (mesh surface CSR order)
    int32_t *masked = nullptr;   // [n_masked] local indices of masked nodes
    double *ysurf = nullptr;     // [E][surface nodes]
    double *partials = nullptr;
    unsigned *counters = nullptr;
    hb_cg_state *state = nullptr, *state_host = nullptr;
    double *cg_vec = nullptr;
    size_t cg_vec_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

using hb::dot_acc;

const int kThreads = 256;

inline unsigned grid_for(int64_t n)
{
    const int64_t b = (n + kThreads - 1) / kThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

inline int red_grid(int64_t n)
{
    const int64_t b = (n + HB_RED_THREADS - 1) / HB_RED_THREADS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, HB_RED_BLOCKS));
}

__global__ void k_weights(const int32_t *__restrict__ l2g, const int32_t *__restrict__ rowptr, int64_t n,
                          double *__restrict__ w)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = l2g[q];
        w[q] = g < 0 ? 0.0 : 1.0 / (double)(rowptr[g + 1] - rowptr[g]);
    }
}

__global__ void k_sloc(const int32_t *__restrict__ scols, int64_t nnz, int NS, int n3,
                       const int32_t *__restrict__ node_of, int32_t *__restrict__ sloc)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = scols[q];
        const int32_t e = c / NS;
        sloc[q] = e * n3 + node_of[c - e * NS];
    }
}

__global__ void k_scatter(const int32_t *__restrict__ l2g, const double *__restrict__ xG, int64_t n,
                          double *__restrict__ xL)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = l2g[q];
        xL[q] = g < 0 ? 0.0 : xG[g];
    }
}

// Z Z^T on the surface DOFs: y_L at every copy of g = sum of the copies'
// element results (element order) + lambda (x_g | M_gg x_g); items past the
// rows zero the masked nodes.
template <int SCREEN>
__global__ void __launch_bounds__(kThreads) k_gather_scatter(const double *__restrict__ ys,
                                                             const int32_t *__restrict__ row_g,
                                                             const int32_t *__restrict__ rowptr,
                                                             const int32_t *__restrict__ cols,
                                                             const int32_t *__restrict__ sloc,
                                                             const double *__restrict__ xL,
                                                             const double *__restrict__ mdiag, double lambda,
                                                             double *__restrict__ yL, int64_t nrows,
                                                             const int32_t *__restrict__ masked, int64_t n_masked,
                                                             const int *run)
{
    if (run && *run == 0) return;
    const int64_t total = nrows + n_masked;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (r >= nrows) {
            yL[masked[r - nrows]] = 0.0;
            continue;
        }
        const int a = rowptr[r], z = rowptr[r + 1];
        double t = 0.0;
        for (int p = a; p < z; p++) t += __ldcs(ys + cols[p]);
        const double xv = xL[sloc[a]];
        t += SCREEN ? lambda * (mdiag[row_g[r]] * xv) : lambda * xv;
        for (int p = a; p < z; p++) yL[sloc[p]] = t;
    }
}

__global__ void __launch_bounds__(HB_RED_THREADS) k_wdot(const double *__restrict__ a, const double *__restrict__ b,
                                                          const double *__restrict__ w, int64_t n, double *out,
                                                          double *partials, unsigned *counter)
{
    dot_acc<double> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc.add(w[i] * a[i], b[i]);
    double v[1] = {acc.value()}, tot[1];
    if (hb::grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) *out = tot[0];
}

// r = b - A x, p = r, weighted r.r and b.b; state for Algorithm 1.
__global__ void __launch_bounds__(HB_RED_THREADS) k_w_init(const double *__restrict__ b,
                                                            const double *__restrict__ Ax, double *__restrict__ r,
                                                            double *__restrict__ p, const double *__restrict__ w,
                                                            int64_t n, double rtol, int max_it, double *partials,
                                                            unsigned *counter, hb_cg_state *st)
{
    dot_acc<double> rr, bb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i], ri = bi - Ax[i], wi = w[i];
        r[i] = ri;
        p[i] = ri;
        rr.add(wi * ri, ri);
        bb.add(wi * bi, bi);
    }
    double v[2] = {rr.value(), bb.value()}, tot[2];
    if (hb::grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->res2 = tot[0];
        st->bb = tot[1];
        st->tol2 = rtol * rtol * tot[1];
        st->it = 0;
        st->max_it = max_it;
        st->alpha = st->beta = st->pAp = 0.0;
        // a non-finite b (or A x0) is reported as a breakdown, not a NaN residual
        const bool finite = isfinite(tot[0]) && isfinite(tot[1]);
        st->status = finite ? HB_OK : HB_ERR_BREAKDOWN;
        st->run = (finite && max_it > 0 && tot[0] > st->tol2) ? 1 : 0;
        st->next_run = st->run;
    }
}

// Restart (the one-mesh solver's rule with weighted dots): the true residual
// r = b - A x, p = r, its weighted r.r into the state (the iteration count
// stays); run again while it is above the tolerance.
__global__ void __launch_bounds__(HB_RED_THREADS) k_w_restart(const double *__restrict__ b,
                                                               const double *__restrict__ Ax, double *__restrict__ r,
                                                               double *__restrict__ p, const double *__restrict__ w,
                                                               int64_t n, double *partials, unsigned *counter,
                                                               hb_cg_state *st)
{
    dot_acc<double> rr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - Ax[i];
        r[i] = ri;
        p[i] = ri;
        rr.add(w[i] * ri, ri);
    }
    double v[1] = {rr.value()}, tot[1];
    if (hb::grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->res2 = tot[0];
        st->alpha = st->beta = st->pAp = 0.0;
        const bool finite = isfinite(tot[0]);
        if (!finite) st->status = HB_ERR_BREAKDOWN;
        st->run = (finite && st->status == HB_OK && st->it < st->max_it && tot[0] > st->tol2) ? 1 : 0;
        st->next_run = st->run;
    }
}

// Weighted p.Ap, alpha and the breakdown test.
__global__ void __launch_bounds__(HB_RED_THREADS) k_w_pap(const double *__restrict__ p, const double *__restrict__ Ap,
                                                           const double *__restrict__ w, int64_t n, double *partials,
                                                           unsigned *counter, hb_cg_state *st)
{
    if (st->run == 0) return;
    dot_acc<double> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc.add(w[i] * p[i], Ap[i]);
    double v[1] = {acc.value()}, tot[1];
    if (hb::grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        const double pAp = tot[0];
        st->pAp = pAp;
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            st->status = HB_ERR_BREAKDOWN;
            st->run = 0;
        } else {
            st->alpha = st->rr / pAp;
        }
    }
}

// r -= alpha Ap with the weighted new r.r, beta and the stopping test.
__global__ void __launch_bounds__(HB_RED_THREADS) k_w_update_r(double *__restrict__ r, const double *__restrict__ Ap,
                                                                const double *__restrict__ w, int64_t n,
                                                                double *partials, unsigned *counter, hb_cg_state *st)
{
    if (st->run == 0) return;
    const double alpha = st->alpha;
    dot_acc<double> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = r[i] - alpha * __ldcs(Ap + i);
        r[i] = ri;
        acc.add(w[i] * ri, ri);
    }
    double v[1] = {acc.value()}, tot[1];
    if (hb::grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        st->rr_new = tot[0];
        st->beta = tot[0] / st->rr;
        st->rr = tot[0];
        st->res2 = tot[0];
        st->it += 1;
        st->next_run = (st->it < st->max_it && tot[0] > st->tol2) ? 1 : 0;
    }
}

__global__ void __launch_bounds__(HB_RED_THREADS) k_update_xp(double *x, double *p, const double *r, int64_t n,
                                                               unsigned *counter, hb_cg_state *st)
{
    hb::cg_update_xp_body<double>(x, p, r, n, counter, st);
}

void free_scat(hb_scat *S)
{
    if (!S) return;
    for (void *a : {(void *)S->w, (void *)S->sloc, (void *)S->masked, (void *)S->ysurf, (void *)S->partials,
                    (void *)S->counters, (void *)S->state, (void *)S->cg_vec})
        if (a) cudaFree(a);
    if (S->state_host) cudaFreeHost(S->state_host);
    if (S->ev0) cudaEventDestroy(S->ev0);
    if (S->ev1) cudaEventDestroy(S->ev1);
    delete S;
}

hb_status build(hb_scat *S, cudaStream_t s)
{
    const hb_mesh *m = S->m;
    const int N = m->N, n = N + 1, n3 = n * n * n, NS = hb_surf_count(N);
    const int64_t nl = m->n_local;
    S->n_local = nl;
    // masked nodes (host scan of l2g, once)
    std::vector<int32_t> l2g((size_t)nl), masked;
    HB_TRY_CUDA(cudaMemcpyAsync(l2g.data(), m->l2g, (size_t)nl * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    for (int64_t q = 0; q < nl; q++)
        if (l2g[q] < 0) masked.push_back((int32_t)q);
    S->n_masked = (int64_t)masked.size();
    // surface index -> node index within the element
    std::vector<int32_t> node_of(NS, -1);
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                const int sp = hb_surf_pos(N, i, j, k);
                if (sp >= 0) node_of[sp] = (k * n + j) * n + i;
            }
    for (int v : node_of)
        if (v < 0) { hb_set_error("surface map incomplete"); return HB_ERR_ARG; }
    int32_t *d_node_of = nullptr;
    HB_TRY_CUDA(cudaMalloc((void **)&d_node_of, NS * sizeof(int32_t)));
    cudaError_t ce = cudaMemcpy(d_node_of, node_of.data(), NS * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) { cudaFree(d_node_of); HB_TRY_CUDA(ce); }
    HB_TRY_CUDA(cudaMalloc((void **)&S->w, (size_t)std::max<int64_t>(nl, 1) * sizeof(double)));
    HB_TRY_CUDA(cudaMalloc((void **)&S->sloc, (size_t)std::max<int64_t>(m->nnz_s, 1) * sizeof(int32_t)));
    HB_TRY_CUDA(cudaMalloc((void **)&S->masked, (size_t)std::max<int64_t>(S->n_masked, 1) * sizeof(int32_t)));
    HB_TRY_CUDA(cudaMalloc((void **)&S->ysurf, (size_t)std::max<int64_t>(m->E * NS, 1) * sizeof(double)));
    HB_TRY_CUDA(cudaMalloc((void **)&S->partials, HB_RED_MAXV * HB_RED_BLOCKS * sizeof(double)));
    HB_TRY_CUDA(cudaMalloc((void **)&S->counters, 8 * sizeof(unsigned)));
    HB_TRY_CUDA(cudaMalloc((void **)&S->state, 2 * sizeof(hb_cg_state)));
    HB_TRY_CUDA(cudaMallocHost((void **)&S->state_host, sizeof(hb_cg_state)));
    HB_TRY_CUDA(cudaMemsetAsync(S->counters, 0, 8 * sizeof(unsigned), s));
    if (!masked.empty())
        HB_TRY_CUDA(cudaMemcpyAsync(S->masked, masked.data(), masked.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
    if (nl > 0) {
        hb_count_launch();
        k_weights<<<grid_for(nl), kThreads, 0, s>>>(m->l2g, m->rowptr, nl, S->w);
        HB_CHECK_LAUNCH();
    }
    if (m->nnz_s > 0) {
        hb_count_launch();
        k_sloc<<<grid_for(m->nnz_s), kThreads, 0, s>>>(m->scols, m->nnz_s, NS, n3, d_node_of, S->sloc);
        HB_CHECK_LAUNCH();
    }
    HB_TRY_CUDA(cudaEventCreate(&S->ev0));
    HB_TRY_CUDA(cudaEventCreate(&S->ev1));
    ce = cudaStreamSynchronize(s);
    cudaFree(d_node_of);
    HB_TRY_CUDA(ce);
    return HB_OK;
}

hb_status scat_apply(const hb_scat *S, int screen, double lambda, const double *xL, double *yL, const int *run,
                     cudaStream_t s)
{
    const hb_mesh *m = S->m;
    const int v = m->variant[0];
    const int eo = (v & HB_VAR_PENCIL) ? ((v & HB_VAR_EO) ? 1 : 0) : 1;
    const int ebm = (v & HB_VAR_PENCIL) ? ((v & HB_VAR_ONE) ? 0 : ((v & HB_VAR_EB2) ? 2 : 1)) : 1;
    hb_status st = hb_launch_ax2_f64_scat(m, xL, S->ysurf, yL, lambda, screen, run, eo, ebm, s);
    if (st != HB_OK) return st;
    const int64_t total = m->nsr + S->n_masked;
    if (total == 0) return HB_OK;
    hb_prof_scope prof("gather_scatter", s);
    if (screen)
        k_gather_scatter<1><<<grid_for(total), kThreads, 0, s>>>(S->ysurf, m->srow_g, m->srowptr, m->scols, S->sloc,
                                                                 xL, m->mdiag, lambda, yL, m->nsr, S->masked,
                                                                 S->n_masked, run);
    else
        k_gather_scatter<0><<<grid_for(total), kThreads, 0, s>>>(S->ysurf, m->srow_g, m->srowptr, m->scols, S->sloc,
                                                                 xL, m->mdiag, lambda, yL, m->nsr, S->masked,
                                                                 S->n_masked, run);
    HB_CHECK_LAUNCH();
    return HB_OK;
}

bool valid_screen(int s) { return s == HB_SCREEN_IDENTITY || s == HB_SCREEN_MASS; }

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" hb_status hb_scat_create(const hb_mesh *mesh, void *stream, hb_scat **out)
{
    hb_clear_error();
    if (!mesh || !out) { hb_set_error("null argument"); return HB_ERR_ARG; }
    *out = nullptr;
    hb_device_guard dg(mesh->device);
    if (!dg.ok) { hb_set_error("cannot select device %d", mesh->device); return HB_ERR_CUDA; }
    hb_scat *S = new hb_scat();
    S->m = mesh;
    S->device = mesh->device;
    hb_status st = build(S, (cudaStream_t)stream);
    if (st != HB_OK) {
        free_scat(S);
        return st;
    }
    *out = S;
    return HB_OK;
}

extern "C" hb_status hb_scat_destroy(hb_scat *sc)
{
    hb_clear_error();
    if (!sc) return HB_OK;
    hb_device_guard dg(sc->device);
    cudaDeviceSynchronize();
    free_scat(sc);
    return HB_OK;
}

extern "C" hb_status hb_scat_scatter(const hb_scat *sc, const double *xG, double *xL, void *stream)
{
    hb_clear_error();
    if (!sc || !xL || (!xG && sc->m->n_global > 0)) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (sc->n_local == 0) return HB_OK;
    hb_device_guard dg(sc->device);
    cudaStream_t s = (cudaStream_t)stream;
    hb_prof_scope prof("scatter", s);
    k_scatter<<<grid_for(sc->n_local), kThreads, 0, s>>>(sc->m->l2g, xG, sc->n_local, xL);
    HB_CHECK_LAUNCH();
    return HB_OK;
}

extern "C" hb_status hb_scat_apply_A(const hb_scat *sc, hb_screen screen, double lambda, const double *xL, double *yL,
                                     void *stream)
{
    hb_clear_error();
    if (!sc || !xL || !yL) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!valid_screen(screen)) { hb_set_error("invalid screen %d", (int)screen); return HB_ERR_ARG; }
    if (xL == yL) { hb_set_error("x and y must not overlap"); return HB_ERR_ARG; }
    if (sc->n_local == 0) return HB_OK;
    hb_device_guard dg(sc->device);
    return scat_apply(sc, screen, lambda, xL, yL, nullptr, (cudaStream_t)stream);
}

extern "C" hb_status hb_scat_dot(const hb_scat *sc, const double *aL, const double *bL, double *out_host, void *stream)
{
    hb_clear_error();
    if (!sc || !aL || !bL || !out_host) { hb_set_error("null argument"); return HB_ERR_ARG; }
    hb_device_guard dg(sc->device);
    hb_scat *S = const_cast<hb_scat *>(sc);
    cudaStream_t s = (cudaStream_t)stream;
    double *out = &S->state[1].dot_tmp;
    {
        hb_prof_scope prof("wdot", s);
        k_wdot<<<red_grid(S->n_local), HB_RED_THREADS, 0, s>>>(aL, bL, S->w, S->n_local, out, S->partials,
                                                               S->counters + 1);
        HB_CHECK_LAUNCH();
    }
    HB_TRY_CUDA(cudaMemcpyAsync(out_host, out, sizeof(double), cudaMemcpyDeviceToHost, s));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    return HB_OK;
}

extern "C" hb_status hb_scat_cg_solve(const hb_scat *sc, const hb_cg_opts *o, const double *b, double *x,
                                      hb_cg_result *res, void *stream)
{
    hb_clear_error();
    hb_cg_result R{};
    R.status = HB_OK;
    if (res) *res = R;
    if (!sc || !o || !b || !x) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (o->prec != HB_F64) { hb_set_error("hb_scat_cg_solve takes HB_F64"); return HB_ERR_ARG; }
    if (o->precond != 0) { hb_set_error("hb_scat_cg_solve has no preconditioner"); return HB_ERR_ARG; }
    if (!valid_screen(o->screen) || o->max_it < 0 || !(o->rtol >= 0.0)) {
        hb_set_error("invalid options");
        return HB_ERR_ARG;
    }
    hb_device_guard dg(sc->device);
    hb_scat *S = const_cast<hb_scat *>(sc);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = S->n_local;
    if (n == 0) return HB_OK;
    const int64_t stride = (n + 63) / 64 * 64;
    const size_t need = (size_t)stride * 3 * sizeof(double);
    if (S->cg_vec_bytes < need) {
        if (S->cg_vec) cudaFree(S->cg_vec);
        S->cg_vec = nullptr;
        S->cg_vec_bytes = 0;
        HB_TRY_CUDA(cudaMalloc((void **)&S->cg_vec, need));
        S->cg_vec_bytes = need;
    }
    double *r = S->cg_vec, *p = r + stride, *Ap = p + stride;
    hb_cg_state *st = S->state;
    const int grid = red_grid(n);
    HB_TRY_CUDA(cudaEventRecord(S->ev0, s));
    hb_status rs = scat_apply(S, o->screen, o->lambda, x, Ap, nullptr, s);
    if (rs != HB_OK) return rs;
    hb_count_launch();
    k_w_init<<<grid, HB_RED_THREADS, 0, s>>>(b, Ap, r, p, S->w, n, o->rtol, o->max_it, S->partials, S->counters + 2,
                                             st);
    HB_CHECK_LAUNCH();
    // with a tolerance, a stop of the recursive residual is checked on the
    // true one (a restart from x, as in hb_cg_solve)
    int chunk = 16;
    bool checked = false;
    double prev = -1.0;
    hb_cg_state fin{};
    for (;;) {
        HB_TRY_CUDA(cudaMemcpyAsync(S->state_host, st, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
        HB_TRY_CUDA(cudaStreamSynchronize(s));
        fin = *S->state_host;
        if (!fin.run || fin.it >= o->max_it) {
            if (o->rtol > 0.0 && fin.status == HB_OK && !checked) {
                if ((rs = scat_apply(S, o->screen, o->lambda, x, Ap, nullptr, s)) != HB_OK) return rs;
                hb_count_launch();
                k_w_restart<<<grid, HB_RED_THREADS, 0, s>>>(b, Ap, r, p, S->w, n, S->partials, S->counters + 2,
                                                            st);
                HB_CHECK_LAUNCH();
                checked = true;
                continue;
            }
            break;
        }
        if (checked) {
            if (prev >= 0.0 && fin.res2 > 0.81 * prev) break;  // no progress: the rounding floor
            prev = fin.res2;
        }
        checked = false;
        const int cnt = std::min(chunk, o->max_it - fin.it);
        for (int it = 0; it < cnt; it++) {
            if ((rs = scat_apply(S, o->screen, o->lambda, p, Ap, &st->run, s)) != HB_OK) return rs;
            {
                hb_prof_scope prof("wdot_pap", s);
                k_w_pap<<<grid, HB_RED_THREADS, 0, s>>>(p, Ap, S->w, n, S->partials, S->counters + 1, st);
                HB_CHECK_LAUNCH();
            }
            {
                hb_prof_scope prof("cg_update_r", s);
                k_w_update_r<<<grid, HB_RED_THREADS, 0, s>>>(r, Ap, S->w, n, S->partials, S->counters + 2, st);
                HB_CHECK_LAUNCH();
            }
            {
                hb_prof_scope prof("cg_update_xp", s);
                k_update_xp<<<grid, HB_RED_THREADS, 0, s>>>(x, p, r, n, S->counters + 3, st);
                HB_CHECK_LAUNCH();
            }
        }
        chunk = std::min(chunk * 2, 256);
    }
    HB_TRY_CUDA(cudaEventRecord(S->ev1, s));
    HB_TRY_CUDA(cudaEventSynchronize(S->ev1));
    float ms = 0.f;
    HB_TRY_CUDA(cudaEventElapsedTime(&ms, S->ev0, S->ev1));
    R.iters = fin.it;
    R.rel_res = fin.bb > 0.0 ? std::sqrt(fin.res2 / fin.bb) : 0.0;
    R.time_ms = ms;
    if (fin.status == HB_ERR_BREAKDOWN) R.status = HB_ERR_BREAKDOWN;
    else if (o->rtol > 0.0 && fin.res2 > fin.tol2) R.status = HB_ERR_NOT_CONVERGED;
    if (res) *res = R;
    return R.status;
}
