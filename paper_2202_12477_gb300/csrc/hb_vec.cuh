// Device-side bodies of the reduction, assembly and CG vector kernels,
// shared by the solver kernels (one mesh) and the serving kernels (one slot
// descriptor per solve). All reductions run on a fixed grid and combine
// their block partials in index order, so results are bitwise reproducible.
#pragma once

#include "hb_acc.cuh"
#include "hb_internal.h"

namespace hb {

using hbacc::dot_acc;

// ---------------------------------------------------------------- grid reduction

// Sums NV values over the grid in a fixed order. Returns true in the block that
// arrives last (in all of its threads), with tot[] holding the grid totals.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double *partials, unsigned *counter, double (&tot)[NV])
{
    static_assert(NV >= 1 && NV <= HB_RED_MAXV, "partials buffers hold HB_RED_MAXV rows");
    __shared__ double sh[NV][32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double a = v[q];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[q][wid] = a;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double a = lane < nw ? sh[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) partials[q * HB_RED_BLOCKS + blockIdx.x] = a;
        }
        if (lane == 0) {
            __threadfence();
            unsigned t = atomicAdd(counter, 1u);
            s_last = (t == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double a = 0.0;
        for (int p = threadIdx.x; p < (int)gridDim.x; p += blockDim.x) a += __ldcg(&partials[q * HB_RED_BLOCKS + p]);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        __syncthreads();
        if (lane == 0) sh[q][wid] = a;
        __syncthreads();
        if (wid == 0) {
            double b = lane < nw ? sh[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(0xffffffffu, b, o);
            if (lane == 0) sh[q][0] = b;
        }
        __syncthreads();
        tot[q] = sh[q][0];
    }
    if (threadIdx.x == 0) *counter = 0;
    return true;
}

// ---------------------------------------------------------------- assembly

// y_g = sum_{p in row g} y_L[cols[p]] + lambda (x_g | M_gg x_g); optional x.y.
template <typename T, int SCREEN, int DOT>
__device__ __forceinline__ void assemble_body(const T *__restrict__ yL, const int32_t *__restrict__ rowptr,
                    const int32_t *__restrict__ cols, const T *__restrict__ x, const T *__restrict__ mdiag,
                    double lambda, T *__restrict__ y, int64_t ng, double *partials, unsigned *counter,
                    hb_cg_state *st)
{
    if (DOT == HB_DOT_CG_PAP && st->run == 0) return;
    const T lam = (T)lambda;
    dot_acc<T> acc;
    // four independent rows per pass (see assemble_surf_body)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g0 < ng; g0 += 4 * stride) {
        int a[4], z[4], c0[4], c1[4];
        T xv[4], s[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t g = g0 + u * stride;
            a[u] = g < ng ? __ldg(rowptr + g) : 0;
            z[u] = g < ng ? __ldg(rowptr + g + 1) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t g = g0 + u * stride;
            c0[u] = a[u] < z[u] ? __ldcs(cols + a[u]) : -1;
            c1[u] = a[u] + 1 < z[u] ? __ldcs(cols + a[u] + 1) : -1;
            xv[u] = g < ng ? x[g] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const T v0 = c0[u] >= 0 ? __ldcs(yL + c0[u]) : T(0);
            const T v1 = c1[u] >= 0 ? __ldcs(yL + c1[u]) : T(0);
            s[u] = v0 + v1;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t g = g0 + u * stride;
            if (g >= ng) continue;
            T t = s[u];
            for (int p = a[u] + 2; p < z[u]; p++) t += __ldcs(yL + __ldcs(cols + p));
            t += SCREEN ? lam * (mdiag[g] * xv[u]) : lam * xv[u];
            y[g] = t;
            if (DOT) acc.add(xv[u], t);
        }
    }
    if (DOT) {
        double v[1] = {acc.value()}, tot[1];
        if (grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) {
            if (DOT == HB_DOT_CG_PAP) {
                const double pAp = tot[0];
                st->pAp = pAp;
                if (!(pAp > 0.0) || !isfinite(pAp)) {
                    st->status = HB_ERR_BREAKDOWN;
                    st->run = 0;
                } else {
                    st->alpha = st->rr / pAp;
                }
            } else {
                st->dot_tmp = tot[0];
            }
        }
    }
}

// ---------------------------------------------------------------- surface assembly

// Z^T on the DOFs that have a copy on an element surface: y_g = sum over the
// copies of ysurf (ascending: element order) + lambda (x_g | M_gg x_g).
// With a dot mode, x.y over these rows plus the element kernel's per-block
// partials (interior DOFs) is reduced on the fixed grid.
// CONTIG: the copies of row r are ys[rowptr[r] .. rowptr[r+1]) (the element
// kernel wrote them at their CSR positions); cols is not read.
template <typename T, int SCREEN, int DOT, bool CONTIG = false>
__device__ __forceinline__ void assemble_surf_body(const T *__restrict__ ys, const int32_t *__restrict__ srow_g,
                         const int32_t *__restrict__ rowptr, const int32_t *__restrict__ cols,
                         const T *__restrict__ x, const T *__restrict__ mdiag, double lambda, T *__restrict__ y,
                         int64_t nrows, const double *__restrict__ ax_partials, int64_t n_axp, double *partials,
                         unsigned *counter, hb_cg_state *st)
{
    if (DOT == HB_DOT_CG_PAP && st->run == 0) return;
    const T lam = (T)lambda;
    dot_acc<T> acc;
    // four independent rows per pass keep several dependent load chains
    // (row pointer -> column -> value) in flight per thread
    constexpr int U4 = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r0 < nrows; r0 += U4 * stride) {
        int g[U4], a[U4], z[U4], c0[U4], c1[U4];
        T xv[U4], s[U4];
#pragma unroll
        for (int u = 0; u < U4; u++) {
            const int64_t r = r0 + u * stride;
            const bool ok = r < nrows;
            g[u] = ok ? __ldg(srow_g + r) : -1;
            a[u] = ok ? __ldg(rowptr + r) : 0;
            z[u] = ok ? __ldg(rowptr + r + 1) : 0;
        }
#pragma unroll
        for (int u = 0; u < U4; u++) {
            if constexpr (CONTIG) {
                c0[u] = a[u] < z[u] ? a[u] : -1;
                c1[u] = a[u] + 1 < z[u] ? a[u] + 1 : -1;
            } else {
                c0[u] = a[u] < z[u] ? __ldcs(cols + a[u]) : -1;
                c1[u] = a[u] + 1 < z[u] ? __ldcs(cols + a[u] + 1) : -1;
            }
            xv[u] = g[u] >= 0 ? x[g[u]] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U4; u++) {
            T v0 = c0[u] >= 0 ? __ldcs(ys + c0[u]) : T(0);
            T v1 = c1[u] >= 0 ? __ldcs(ys + c1[u]) : T(0);
            s[u] = v0 + v1;
        }
#pragma unroll
        for (int u = 0; u < U4; u++) {
            if (g[u] < 0) continue;
            T t = s[u];
            for (int p = a[u] + 2; p < z[u]; p++) t += __ldcs(ys + (CONTIG ? p : __ldcs(cols + p)));
            t += SCREEN ? lam * (mdiag[g[u]] * xv[u]) : lam * xv[u];
            y[g[u]] = t;
            if (DOT) acc.add(xv[u], t);
        }
    }
    if (DOT) {
        double v = acc.value();
        for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_axp;
             q += (int64_t)gridDim.x * blockDim.x)
            v += ax_partials[q];
        double vv[1] = {v}, tot[1];
        if (grid_sum<1>(vv, partials, counter, tot) && threadIdx.x == 0) {
            if (DOT == HB_DOT_CG_PAP) {
                const double pAp = tot[0];
                st->pAp = pAp;
                if (!(pAp > 0.0) || !isfinite(pAp)) {
                    st->status = HB_ERR_BREAKDOWN;
                    st->run = 0;
                } else {
                    st->alpha = st->rr / pAp;
                }
            } else {
                st->dot_tmp = tot[0];
            }
        }
    }
}

// ---------------------------------------------------------------- lattice assembly

// The box's lattice, for Z^T by index arithmetic: lattice point (I, J, K),
// 0 <= I <= N Ex, is node (I - N ex, ...) of element (ex, ey, ez); DOFs are
// the unmasked points, numbered (I - x0) + NXu ((J - y0) + NYu (K - z0))
// with x0 = 1 if the x = 0 face is Dirichlet (and so on).
struct lattice_t {
    int N, Ex, Ey, Ez;
    int x0, y0, z0;
    int NXu, NYu, NZu;
};

// The elements along one axis that hold lattice coordinate I (ascending) and
// I's local index in each: one inside an element, two on a shared face.
__device__ __forceinline__ int lattice_axis(int I, int N, int Eax, int (&ec)[2], int (&lc)[2])
{
    const int q = I / N, r = I - q * N;
    if (r != 0) { ec[0] = q; lc[0] = r; return 1; }
    if (q == 0) { ec[0] = 0; lc[0] = 0; return 1; }
    if (q == Eax) { ec[0] = Eax - 1; lc[0] = N; return 1; }
    ec[0] = q - 1; lc[0] = N;
    ec[1] = q; lc[1] = 0;
    return 2;
}

// Z^T on every DOF from the element-major local values yL[e][k][j][i]: y_g =
// the copies of DOF g summed in ascending element order (the association of
// the CSR gathers: (c0 + c1) + c2 + ..., a lone copy plus zero) + lambda
// (x_g | M_gg x_g). Lanes along I, so x, y and the runs of each element row
// of yL are read and written coalesced. With a dot mode, x.y over all DOFs is
// reduced on the fixed grid.
template <typename T, int SCREEN, int DOT>
__device__ __forceinline__ void assemble_grid_body(const T *__restrict__ yL, const lattice_t L, const T *__restrict__ x,
                                                   const T *__restrict__ mdiag, double lambda, T *__restrict__ y,
                                                   double *partials, unsigned *counter, hb_cg_state *st)
{
    if (DOT == HB_DOT_CG_PAP && st->run == 0) return;
    const T lam = (T)lambda;
    dot_acc<T> acc;
    const int n = L.N + 1;
    const int64_t n3 = (int64_t)n * n * n;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nrows = (int64_t)L.NYu * L.NZu;
    // one warp per lattice row (J, K), lanes along I
    for (int64_t row = warp; row < nrows; row += nwarps) {
        const int Ju = (int)(row % L.NYu), Ku = (int)(row / L.NYu);
        int eyc[2], jc[2], ezc[2], kc[2];
        const int ny = lattice_axis(L.y0 + Ju, L.N, L.Ey, eyc, jc);
        const int nz = lattice_axis(L.z0 + Ku, L.N, L.Ez, ezc, kc);
        const T *__restrict__ xr = x + row * L.NXu;
        T *__restrict__ yr = y + row * L.NXu;
        for (int Iu = lane; Iu < L.NXu; Iu += 32) {
            int exc[2], ic[2];
            const int nx = lattice_axis(L.x0 + Iu, L.N, L.Ex, exc, ic);
            T t = T(0);
            int cnt = 0;
            for (int cz = 0; cz < nz; cz++)
                for (int cy = 0; cy < ny; cy++) {
                    const int64_t base = ((int64_t)eyc[cy] + (int64_t)L.Ey * ezc[cz]) * L.Ex;
                    const int64_t off = ((int64_t)kc[cz] * n + jc[cy]) * n;
                    for (int cx = 0; cx < nx; cx++) {
                        const T v = __ldcs(yL + (base + exc[cx]) * n3 + off + ic[cx]);
                        t = cnt == 0 ? v : t + v;
                        cnt++;
                    }
                }
            if (cnt == 1) t = t + T(0);
            const T xv = xr[Iu];
            t += SCREEN ? lam * (mdiag[row * L.NXu + Iu] * xv) : lam * xv;
            yr[Iu] = t;
            if (DOT) acc.add(xv, t);
        }
    }
    if (DOT) {
        double vv[1] = {acc.value()}, tot[1];
        if (grid_sum<1>(vv, partials, counter, tot) && threadIdx.x == 0) {
            if (DOT == HB_DOT_CG_PAP) {
                const double pAp = tot[0];
                st->pAp = pAp;
                if (!(pAp > 0.0) || !isfinite(pAp)) {
                    st->status = HB_ERR_BREAKDOWN;
                    st->run = 0;
                } else {
                    st->alpha = st->rr / pAp;
                }
            } else {
                st->dot_tmp = tot[0];
            }
        }
    }
}

// ---------------------------------------------------------------- dot

template <typename T>
__device__ __forceinline__ void dot_body(const T *__restrict__ a, const T *__restrict__ b, int64_t n, double *out, double *partials,
               unsigned *counter)
{
    dot_acc<T> acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        T av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + u * stride;
            av[u] = i < n ? a[i] : T(0);
            bv[u] = i < n ? b[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (i0 + u * stride < n) acc.add(av[u], bv[u]);
    }
    double v[1] = {acc.value()}, tot[1];
    if (grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) *out = tot[0];
}

// ---------------------------------------------------------------- CG kernels

// r = b - Ax; z = M^-1 r (M = diag(A) when inv_d is given, else z = r);
// p = z; r.z, r.r and b.b; state set up for Algorithm 1 (preconditioned).
__device__ __forceinline__ void cg_init_body(const double *__restrict__ b, const double *__restrict__ Ax,
                                             double *__restrict__ r, double *__restrict__ p,
                                             const double *__restrict__ inv_d, int64_t n, double rtol, int max_it,
                                             double *partials, unsigned *counter, hb_cg_state *st)
{
    dot_acc<double> rz, rr, bb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i];
        const double ri = bi - Ax[i];
        const double zi = inv_d ? ri * inv_d[i] : ri;
        r[i] = ri;
        p[i] = zi;
        rz.add(ri, zi);
        rr.add(ri, ri);
        bb.add(bi, bi);
    }
    double v[3] = {rz.value(), rr.value(), bb.value()}, tot[3];
    if (grid_sum<3>(v, partials, counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->res2 = tot[1];
        st->bb = tot[2];
        st->tol2 = rtol * rtol * tot[2];
        st->it = 0;
        st->max_it = max_it;
        st->alpha = st->beta = st->pAp = 0.0;
        // a non-finite b (or A x0) would stop the loop at once with a NaN
        // residual: report it as a breakdown instead
        const bool finite = isfinite(tot[0]) && isfinite(tot[1]) && isfinite(tot[2]);
        st->status = finite ? HB_OK : HB_ERR_BREAKDOWN;
        st->run = (finite && max_it > 0 && tot[1] > st->tol2) ? 1 : 0;
        st->next_run = st->run;
    }
}

// Restart for the stopping test of Algorithm 1. The recursive residual
// r_{j+1} = r_j - alpha A p_j drifts from b - A x_{j+1} by rounding; a solve
// whose recursive residual meets the tolerance therefore checks the true one:
// r = b - Ax recomputed in FP64 (Ax from the caller's x), z = M^-1 r, and
// Algorithm 1 starts again from x with p = z (new r.z, r.r; the iteration
// count stays). Keeping the old p with the new r instead was measured to
// stall and break down on ill-conditioned meshes. The solve runs on while
// the true residual is above the tolerance and iterations remain; a
// non-finite residual is a breakdown.
__device__ __forceinline__ void cg_restart_body(const double *__restrict__ b, const double *__restrict__ Ax,
                                                double *__restrict__ r, double *__restrict__ p, double *__restrict__ z,
                                                const double *__restrict__ inv_d, int64_t n, double *partials,
                                                unsigned *counter, hb_cg_state *st)
{
    dot_acc<double> rz, rr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - Ax[i];
        r[i] = ri;
        const double zi = inv_d ? ri * inv_d[i] : ri;
        if (inv_d) z[i] = zi;
        p[i] = zi;
        rz.add(ri, zi);
        rr.add(ri, ri);
    }
    double v[2] = {rz.value(), rr.value()}, tot[2];
    if (grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->res2 = tot[1];
        st->alpha = st->beta = st->pAp = 0.0;
        const bool finite = isfinite(tot[0]) && isfinite(tot[1]);
        if (!finite) st->status = HB_ERR_BREAKDOWN;
        st->run = (finite && st->status == HB_OK && st->it < st->max_it && tot[1] > st->tol2) ? 1 : 0;
        st->next_run = st->run;
    }
}

// Algorithm 1: r -= alpha Ap and the new r.r. With the
// preconditioner (PREC) also z = M^-1 r, the new r.z (for beta) and r.r (for
// the stopping test); without it r.r serves both.
template <typename T, bool PREC>
__device__ __forceinline__ void cg_update_r_body(T *__restrict__ r, const T *__restrict__ Ap, T *__restrict__ z,
                                                 const T *__restrict__ inv_d, int64_t n, double *partials,
                                                 unsigned *counter, hb_cg_state *st)
{
    if (st->run == 0) return;
    const T alpha = (T)st->alpha;
    dot_acc<T> acc, acc2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        T rv[4], av[4], dv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + u * stride;
            rv[u] = i < n ? r[i] : T(0);
            av[u] = i < n ? __ldcs(Ap + i) : T(0);
            if (PREC) dv[u] = i < n ? inv_d[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                const T ri = rv[u] - alpha * av[u];
                r[i] = ri;
                if (PREC) {
                    const T zi = ri * dv[u];
                    z[i] = zi;
                    acc.add(ri, zi);
                    acc2.add(ri, ri);
                } else {
                    acc.add(ri, ri);
                }
            }
        }
    }
    if (PREC) {
        double v[2] = {acc.value(), acc2.value()}, tot[2];
        if (grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0) {
            st->rr_new = tot[0];
            st->beta = tot[0] / st->rr;
            st->rr = tot[0];
            st->res2 = tot[1];
            st->it += 1;
            st->next_run = (st->it < st->max_it && tot[1] > st->tol2) ? 1 : 0;
        }
    } else {
        double v[1] = {acc.value()}, tot[1];
        if (grid_sum<1>(v, partials, counter, tot) && threadIdx.x == 0) {
            st->rr_new = tot[0];
            st->beta = tot[0] / st->rr;
            st->rr = tot[0];
            st->res2 = tot[0];
            st->it += 1;
            st->next_run = (st->it < st->max_it && tot[0] > st->tol2) ? 1 : 0;
        }
    }
}

// Algorithm 1: x += alpha p with the old p, then p = r + beta p.
// The block that finishes last ends the iteration: run <- next_run.
template <typename T>
__device__ __forceinline__ void cg_update_xp_body(T *__restrict__ x, T *__restrict__ p, const T *__restrict__ r, int64_t n,
                        unsigned *counter, hb_cg_state *st)
{
    __shared__ int s_last;
    if (st->run == 0) return;
    const T alpha = (T)st->alpha, beta = (T)st->beta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += 4 * stride) {
        T pv[4], xv[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + u * stride;
            pv[u] = i < n ? p[i] : T(0);
            xv[u] = i < n ? x[i] : T(0);
            rv[u] = i < n ? r[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                x[i] = xv[u] + alpha * pv[u];
                p[i] = rv[u] + beta * pv[u];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
        if (s_last) {
            *counter = 0;
            st->run = st->next_run;
        }
    }
}

// ---------------------------------------------------------------- mixed precision

// Outer residual: r = b - A x (FP64) with r.r and b.b into the outer state.
__device__ __forceinline__ void residual_body(const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ r,
                    int64_t n, double *partials, unsigned *counter, hb_cg_state *st)
{
    dot_acc<double> rr, bb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i];
        const double ri = bi - Ax[i];
        r[i] = ri;
        rr.add(ri, ri);
        bb.add(bi, bi);
    }
    double v[2] = {rr.value(), bb.value()}, tot[2];
    if (grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->bb = tot[1];
    }
}

// Inner start: r32 = r / ||r|| (so the inner system is well scaled in FP32),
// z32 = M^-1 r32 when inv_d is given, p32 = z32, d32 = 0; inner state for
// A d = r32 with relative target rtol_in.
__device__ __forceinline__ void inner_init_body(const double *__restrict__ r, float *__restrict__ r32,
                                                float *__restrict__ p32, float *__restrict__ d32,
                                                const float *__restrict__ inv_d, int64_t n, double rtol_in,
                                                int max_it, double *partials, unsigned *counter,
                                                const hb_cg_state *outer, hb_cg_state *st)
{
    const double scale = 1.0 / sqrt(outer->rr);
    dot_acc<float> rz, rr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = (float)(r[i] * scale);
        const float zi = inv_d ? v * inv_d[i] : v;
        r32[i] = v;
        p32[i] = zi;
        d32[i] = 0.0f;
        rz.add(v, zi);
        rr.add(v, v);
    }
    double v[2] = {rz.value(), rr.value()}, tot[2];
    if (grid_sum<2>(v, partials, counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->res2 = tot[1];
        st->bb = tot[1];
        st->tol2 = rtol_in * rtol_in * tot[1];
        st->it = 0;
        st->max_it = max_it;
        st->status = HB_OK;
        st->alpha = st->beta = st->pAp = 0.0;
        st->run = (max_it > 0 && tot[1] > st->tol2) ? 1 : 0;
        st->next_run = st->run;
    }
}

// x += ||r|| d32 (FP64 solution update).
__device__ __forceinline__ void update_x_body(double *__restrict__ x, const float *__restrict__ d32, int64_t n,
                                const hb_cg_state *outer)
{
    const double s = sqrt(outer->rr);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += s * (double)d32[i];
}


}  // namespace hb
