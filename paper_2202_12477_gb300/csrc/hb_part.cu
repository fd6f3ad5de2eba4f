// Partitioned operator: the split application of A of hipBone Sec. 3.3
// ("Overlapping halo and gather communication"), with the ranks of a
// distributed run emulated on one GPU. Each virtual rank owns a box of
// elements, its own element data, CUDA streams and exchange buffers in device
// memory; the point-to-point messages of the distributed code become
// device-to-device copies between those buffers, ordered by events, so the
// per-rank kernel sequence and its overlap with the exchanges are the ones a
// multi-GPU run would have.
//
// Per rank and operator application (Sec. 3.3 and its operator timeline):
//   pack    sendbuf = the owned x values that other ranks hold as halo
//   K1      element kernel on the first half of the interior elements
//           || halo exchange: sendbuf segments -> the receivers' halo buffers
//   Kh      element kernel on the halo elements (reads the halo buffer)
//   hgath   sums at halo nodes over this rank's copies -> gather send buffer
//   K2      element kernel on the other half of the interior elements
//   lgath   Z^T on the rank's other surface DOFs
//           || gather exchange: partial sums at halo nodes -> their owners
//   final   owned halo DOFs: own partial + received partials (rank order)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hb_internal.h"
#include "hb_vec.cuh"

namespace {

using hb::dot_acc;

struct part_rank {
    int64_t off = 0, n_owned = 0, n_halo = 0, n_send = 0, n_oshared = 0;
    int64_t e_int1 = 0, e_halo = 0, e_int2 = 0;
    int32_t *l2g = nullptr;    // [E_p][n^3] local codes: >= 0 partition id, -1 masked, <= -2 halo
    double *geo = nullptr;     // [E_p][n][7][n^2]
    double *ysurf = nullptr;   // [E_p][surface nodes]
    double *halo = nullptr;    // [n_halo]
    double *sendbuf = nullptr; // [n_send]
    int32_t *send_idx = nullptr;     // [n_send] partition ids of the values sent
    std::vector<int64_t> send_off;   // [P+1] send segments by destination
    std::vector<int64_t> recv_off;   // [P+1] halo segments by source (owner)
    // halo-node rows: [0, n_halo) in halo order (-> gather send buffer), then
    // [n_halo, n_halo + n_oshared) the owned halo DOFs (-> own partials)
    int32_t *hrowptr = nullptr, *hcols = nullptr;
    double *hbuf = nullptr;
    // rank-local surface rows (owned DOFs no other rank holds)
    int64_t nlr = 0;
    int32_t *lrow_g = nullptr, *lrowptr = nullptr, *lcols = nullptr;
    // owned halo DOFs: partition id and the positions of their partials in grecv
    int32_t *frow_g = nullptr, *frowptr = nullptr, *fcols = nullptr;
    double *grecv = nullptr;   // [n_send] partial sums received, laid out like sendbuf
    cudaStream_t s = nullptr, sc = nullptr;
    cudaEvent_t ev_pack = nullptr, ev_hin = nullptr, ev_gpk = nullptr, ev_grecv = nullptr, ev_done = nullptr;
};

}  // namespace

struct hb_part {
    const hb_mesh *m = nullptr;
    int device = 0;
    int P = 0, px = 0, py = 0, pz = 0;
    uint64_t seed = 0;
    int N = 0, n = 0, NS = 0;
    int64_t n_global = 0, n_shared = 0, exchange_values = 0;
    std::vector<int32_t> perm;  // host copy: partition id -> lexicographic id
    double *mdiag = nullptr;    // [n_global] lumped mass in partition order
    std::vector<part_rank> R;
    cudaEvent_t ev_start = nullptr;
    // CG workspace and reductions
    double *partials = nullptr;
    unsigned *counters = nullptr;
    hb_cg_state *state = nullptr, *state_host = nullptr;
    double *cg_vec = nullptr;
    size_t cg_vec_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void *> allocs;  // every device allocation, freed by destroy
};

namespace {

const int kThreads = 256;

inline unsigned grid_for(int64_t n)
{
    const int64_t b = (n + kThreads - 1) / kThreads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// ---------------------------------------------------------------- kernels

__global__ void k_pack(const double *__restrict__ x, const int32_t *__restrict__ idx, int64_t n,
                       double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[idx[i]];
}

// out[r] = sum of ys over the row's copies (ascending: local element order).
__global__ void k_rowsum(const double *__restrict__ ys, const int32_t *__restrict__ rowptr,
                         const int32_t *__restrict__ cols, int64_t nrows, double *__restrict__ out)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int p = rowptr[r]; p < rowptr[r + 1]; p++) t += ys[cols[p]];
        out[r] = t;
    }
}

// Owned halo DOFs: y_g = own partial + received partials (rank order) + lambda term.
template <int SCREEN>
__global__ void k_final(const double *__restrict__ own, const double *__restrict__ grecv,
                        const int32_t *__restrict__ row_g, const int32_t *__restrict__ rowptr,
                        const int32_t *__restrict__ cols, int64_t nrows, const double *__restrict__ x,
                        const double *__restrict__ mdiag, double lambda, double *__restrict__ y)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        double t = own[r];
        for (int p = rowptr[r]; p < rowptr[r + 1]; p++) t += grecv[cols[p]];
        const int g = row_g[r];
        t += SCREEN ? lambda * (mdiag[g] * x[g]) : lambda * x[g];
        y[g] = t;
    }
}

template <int SCREEN>
__global__ void __launch_bounds__(HB_RED_THREADS) k_local_gather(const double *ys, const int32_t *row_g,
                                                                  const int32_t *rowptr, const int32_t *cols,
                                                                  const double *x, const double *mdiag,
                                                                  double lambda, double *y, int64_t nrows)
{
    hb::assemble_surf_body<double, SCREEN, HB_DOT_NONE>(ys, row_g, rowptr, cols, x, mdiag, lambda, y, nrows,
                                                        nullptr, 0, nullptr, nullptr, nullptr);
}

__global__ void k_permute(const double *__restrict__ src, const int32_t *__restrict__ perm, int64_t n,
                          double *__restrict__ dst)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

// geo rows of the listed elements, in list order
__global__ void k_gather_geo(const double *__restrict__ geo, const int32_t *__restrict__ elems, int64_t ne,
                             int64_t per, double *__restrict__ out)
{
    const int64_t total = ne * per;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t el = q / per, w = q - el * per;
        out[q] = geo[(int64_t)elems[el] * per + w];
    }
}

// CG on the partitioned operator: p.Ap with alpha and the breakdown test
// (Algorithm 1: alpha = r.r / p.Ap), the other vector kernels as in the one-mesh solver.
__global__ void __launch_bounds__(HB_RED_THREADS) k_pap(const double *p, const double *Ap, int64_t n,
                                                         double *partials, unsigned *counter, hb_cg_state *st)
{
    if (st->run == 0) return;
    dot_acc<double> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc.add(p[i], Ap[i]);
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

__global__ void __launch_bounds__(HB_RED_THREADS) k_cg_init(const double *b, const double *Ax, double *r, double *p,
                                                             int64_t n, double rtol, int max_it, double *partials,
                                                             unsigned *counter, hb_cg_state *st)
{
    hb::cg_init_body(b, Ax, r, p, nullptr, n, rtol, max_it, partials, counter, st);
}

__global__ void __launch_bounds__(HB_RED_THREADS) k_cg_restart(const double *b, const double *Ax, double *r,
                                                                double *p, int64_t n, double *partials,
                                                                unsigned *counter, hb_cg_state *st)
{
    hb::cg_restart_body(b, Ax, r, p, nullptr, nullptr, n, partials, counter, st);
}

__global__ void __launch_bounds__(HB_RED_THREADS) k_cg_update_r(double *r, const double *Ap, int64_t n,
                                                                 double *partials, unsigned *counter,
                                                                 hb_cg_state *st)
{
    hb::cg_update_r_body<double, false>(r, Ap, nullptr, nullptr, n, partials, counter, st);
}

__global__ void __launch_bounds__(HB_RED_THREADS) k_cg_update_xp(double *x, double *p, const double *r, int64_t n,
                                                                  unsigned *counter, hb_cg_state *st)
{
    hb::cg_update_xp_body<double>(x, p, r, n, counter, st);
}

inline int red_grid(int64_t n)
{
    const int64_t b = (n + HB_RED_THREADS - 1) / HB_RED_THREADS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, HB_RED_BLOCKS));
}

// ---------------------------------------------------------------- host helpers

template <typename T>
hb_status upload(hb_part *P, const std::vector<T> &h, T **d)
{
    *d = nullptr;
    if (h.empty()) return HB_OK;
    HB_TRY_CUDA(cudaMalloc((void **)d, h.size() * sizeof(T)));
    P->allocs.push_back(*d);
    HB_TRY_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return HB_OK;
}

template <typename T>
hb_status alloc(hb_part *P, size_t count, T **d)
{
    *d = nullptr;
    if (count == 0) return HB_OK;
    HB_TRY_CUDA(cudaMalloc((void **)d, count * sizeof(T)));
    P->allocs.push_back(*d);
    return HB_OK;
}

}  // namespace

// Surface position of node (i,j,k) in its element's surface block (the order
// the pencil kernel writes: k = 0 face, k = N face, then per slab k = 1..N-1
// the ring j = 0 row, j = N row, then i = 0 / i = N for j = 1..N-1); -1 for an
// element-interior node.
int hb_surf_pos(int N, int i, int j, int k)
{
    const int n = N + 1, n2 = n * n;
    if (k == 0) return j * n + i;
    if (k == N) return n2 + j * n + i;
    const bool ring = i == 0 || i == N || j == 0 || j == N;
    if (!ring) return -1;
    const int r = j == 0 ? i : (j == N ? N + 1 + i : 2 * (N + 1) + 2 * (j - 1) + (i == N ? 1 : 0));
    return 2 * n2 + (k - 1) * 4 * N + r;
}

namespace {

// CSR from (row, col) pairs: rows 0..nrows-1, columns ascending per row.
void build_csr(int64_t nrows, std::vector<std::pair<int32_t, int32_t>> &rc, std::vector<int32_t> &rowptr,
               std::vector<int32_t> &cols)
{
    std::sort(rc.begin(), rc.end());
    rowptr.assign(nrows + 1, 0);
    cols.resize(rc.size());
    for (size_t q = 0; q < rc.size(); q++) {
        rowptr[rc[q].first + 1]++;
        cols[q] = rc[q].second;
    }
    for (int64_t r = 0; r < nrows; r++) rowptr[r + 1] += rowptr[r];
}

void free_part(hb_part *P)
{
    if (!P) return;
    for (auto &r : P->R) {
        if (r.s) cudaStreamDestroy(r.s);
        if (r.sc) cudaStreamDestroy(r.sc);
        for (cudaEvent_t e : {r.ev_pack, r.ev_hin, r.ev_gpk, r.ev_grecv, r.ev_done})
            if (e) cudaEventDestroy(e);
    }
    for (cudaEvent_t e : {P->ev_start, P->ev0, P->ev1})
        if (e) cudaEventDestroy(e);
    for (void *a : P->allocs) cudaFree(a);
    if (P->state_host) cudaFreeHost(P->state_host);
    delete P;
}

// Host plan of one rank: everything build() uploads.
struct rank_plan {
    int64_t off = 0, n_owned = 0, n_halo = 0, n_send = 0, n_oshared = 0, nlr = 0;
    int64_t e_int1 = 0, e_halo = 0, e_int2 = 0;
    std::vector<int32_t> order;  // global element ids in local order
    std::vector<int32_t> lc;     // local codes of the rank's elements
    std::vector<int32_t> send;   // partition ids sent, by destination
    std::vector<int64_t> send_off, recv_off;
    std::vector<int32_t> hrowptr, hcols, lrows, lrowptr, lcols, oshared, frowptr, fcols;
};

struct part_plan {
    int64_t n_shared = 0, exchange_values = 0;
    std::vector<int32_t> perm;  // partition id -> lexicographic id
    std::vector<rank_plan> R;
};

// Plans the partition of a box mesh from its host node map (no device work):
// element ranks, DOF owners, partition order, per-rank element order, local
// codes, halo lists, send lists and the three CSRs; then checks that every
// index the kernels and copies will follow stays inside its buffer.
hb_status plan_partition(const int32_t *l2g, int Ex, int Ey, int Ez, int N, int64_t NG, int px, int py, int pz,
                         uint64_t seed, part_plan &PL)
{
    const int n = N + 1, n3 = n * n * n, NS = hb_surf_count(N);
    const int64_t E = (int64_t)Ex * Ey * Ez;
    const int Pn = px * py * pz;

    // rank of every element: block (ex * px / Ex, ...) of the element box
    std::vector<int8_t> erank((size_t)E);
    for (int64_t e = 0; e < E; e++) {
        const int64_t ex = e % Ex, ey = (e / Ex) % Ey, ez = e / ((int64_t)Ex * Ey);
        const int rx = (int)(ex * px / Ex), ry = (int)(ey * py / Ey), rz = (int)(ez * pz / Ez);
        erank[e] = (int8_t)(rx + px * (ry + py * rz));
    }
    // ranks holding each DOF, then its owner (one of them, uniformly at random)
    std::vector<uint64_t> held((size_t)NG, 0);
    for (int64_t e = 0; e < E; e++) {
        const uint64_t bit = 1ull << erank[e];
        const int32_t *lg = &l2g[(size_t)e * n3];
        for (int q = 0; q < n3; q++) {
            if (lg[q] >= NG) { hb_set_error("node map entry %d out of range", lg[q]); return HB_ERR_ARG; }
            if (lg[q] >= 0) held[lg[q]] |= bit;
        }
    }
    std::vector<int8_t> owner((size_t)NG);
    std::vector<int64_t> cnt(Pn, 0);
    int64_t n_shared = 0;
    for (int64_t g = 0; g < NG; g++) {
        const uint64_t h = held[g];
        if (!h) { hb_set_error("DOF %lld held by no element", (long long)g); return HB_ERR_ARG; }
        const int c = __builtin_popcountll(h);
        int pick = 0;
        if (c > 1) {
            n_shared++;
            pick = (int)(hb_u01(seed, 3, (uint64_t)g) * c);
            if (pick >= c) pick = c - 1;
        }
        uint64_t hh = h;
        for (int t = 0; t < pick; t++) hh &= hh - 1;  // drop the lowest set bits
        owner[g] = (int8_t)__builtin_ctzll(hh);
        cnt[owner[g]]++;
    }
    PL.n_shared = n_shared;
    // partition order: by owner, then lexicographic
    std::vector<int64_t> off(Pn + 1, 0);
    for (int p = 0; p < Pn; p++) off[p + 1] = off[p] + cnt[p];
    std::vector<int32_t> newid((size_t)NG);
    PL.perm.assign((size_t)NG, 0);
    {
        std::vector<int64_t> next(off.begin(), off.end() - 1);
        for (int64_t g = 0; g < NG; g++) {
            const int64_t id = next[owner[g]]++;
            newid[g] = (int32_t)id;
            PL.perm[id] = (int32_t)g;
        }
    }
    PL.R.assign(Pn, rank_plan());
    // elements per rank, halo elements (holding a shared DOF) apart
    {
        std::vector<std::vector<int32_t>> inter(Pn), halo(Pn);
        for (int64_t e = 0; e < E; e++) {
            const int32_t *lg = &l2g[(size_t)e * n3];
            bool h = false;
            for (int q = 0; q < n3 && !h; q++) h = lg[q] >= 0 && __builtin_popcountll(held[lg[q]]) > 1;
            (h ? halo : inter)[erank[e]].push_back((int32_t)e);
        }
        for (int p = 0; p < Pn; p++) {
            rank_plan &R = PL.R[p];
            const size_t half = inter[p].size() / 2;
            R.e_int1 = (int64_t)half;
            R.e_halo = (int64_t)halo[p].size();
            R.e_int2 = (int64_t)(inter[p].size() - half);
            R.order.insert(R.order.end(), inter[p].begin(), inter[p].begin() + half);
            R.order.insert(R.order.end(), halo[p].begin(), halo[p].end());
            R.order.insert(R.order.end(), inter[p].begin() + half, inter[p].end());
        }
    }
    // halo DOFs of each rank, in partition order (so grouped by owner)
    std::vector<std::vector<int32_t>> halo_ids(Pn);  // partition ids
    for (int p = 0; p < Pn; p++) {
        std::vector<int32_t> &H = halo_ids[p];
        for (int32_t e : PL.R[p].order) {
            const int32_t *lg = &l2g[(size_t)e * n3];
            for (int q = 0; q < n3; q++)
                if (lg[q] >= 0 && owner[lg[q]] != p) H.push_back(newid[lg[q]]);
        }
        std::sort(H.begin(), H.end());
        H.erase(std::unique(H.begin(), H.end()), H.end());
    }
    auto owner_of_id = [&](int32_t id) {
        return (int)(std::upper_bound(off.begin(), off.end(), (int64_t)id) - off.begin()) - 1;
    };
    std::vector<int32_t> slot((size_t)NG, -1);  // scratch: partition id -> row index
    int64_t exch = 0;
    for (int p = 0; p < Pn; p++) {
        rank_plan &R = PL.R[p];
        R.off = off[p];
        R.n_owned = cnt[p];
        R.n_halo = (int64_t)halo_ids[p].size();
        exch += R.n_halo;
        // halo segments by owner
        R.recv_off.assign(Pn + 1, 0);
        for (int32_t id : halo_ids[p]) R.recv_off[owner_of_id(id) + 1]++;
        for (int q = 0; q < Pn; q++) R.recv_off[q + 1] += R.recv_off[q];
    }
    PL.exchange_values = exch;
    for (int p = 0; p < Pn; p++) {
        rank_plan &R = PL.R[p];
        // send list: for each destination q, q's halo segment owned by p
        R.send_off.assign(Pn + 1, 0);
        for (int q = 0; q < Pn; q++) {
            const rank_plan &Q = PL.R[q];
            for (int64_t t = Q.recv_off[p]; t < Q.recv_off[p + 1]; t++) R.send.push_back(halo_ids[q][t]);
            R.send_off[q + 1] = (int64_t)R.send.size();
        }
        R.n_send = (int64_t)R.send.size();
        // owned halo DOFs (shared, owned by p), ascending
        R.oshared.assign(R.send.begin(), R.send.end());
        std::sort(R.oshared.begin(), R.oshared.end());
        R.oshared.erase(std::unique(R.oshared.begin(), R.oshared.end()), R.oshared.end());
        R.n_oshared = (int64_t)R.oshared.size();
        // local codes of the rank's elements
        for (int64_t t = 0; t < R.n_halo; t++) slot[halo_ids[p][t]] = (int32_t)t;
        const int64_t Ep = (int64_t)R.order.size();
        R.lc.assign((size_t)Ep * n3, 0);
        for (int64_t el = 0; el < Ep; el++) {
            const int32_t *lg = &l2g[(size_t)R.order[el] * n3];
            int32_t *o = &R.lc[(size_t)el * n3];
            for (int q = 0; q < n3; q++) {
                const int32_t g = lg[q];
                o[q] = g < 0 ? -1 : (owner[g] == p ? newid[g] : -2 - slot[newid[g]]);
            }
        }
        for (int64_t t = 0; t < R.n_halo; t++) slot[halo_ids[p][t]] = -1;
        // surface rows: halo rows (halo order, then owned halo DOFs) and local rows
        for (int64_t t = 0; t < R.n_oshared; t++) slot[R.oshared[t]] = (int32_t)(R.n_halo + t);
        std::vector<std::pair<int32_t, int32_t>> hrc, lrc;
        for (int64_t el = 0; el < Ep; el++)
            for (int k = 0; k < n; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++) {
                        const int sp = hb_surf_pos(N, i, j, k);
                        if (sp < 0) continue;
                        const int32_t c = R.lc[(size_t)el * n3 + (k * n + j) * n + i];
                        if (c == -1) continue;
                        const int32_t col = (int32_t)(el * NS + sp);
                        if (c <= -2) hrc.push_back({-2 - c, col});
                        else if (slot[c] >= 0) hrc.push_back({slot[c], col});
                        else lrc.push_back({c, col});
                    }
        // local rows: compact the partition ids
        for (auto &pr : lrc) R.lrows.push_back(pr.first);
        std::sort(R.lrows.begin(), R.lrows.end());
        R.lrows.erase(std::unique(R.lrows.begin(), R.lrows.end()), R.lrows.end());
        for (auto &pr : lrc)
            pr.first = (int32_t)(std::lower_bound(R.lrows.begin(), R.lrows.end(), pr.first) - R.lrows.begin());
        R.nlr = (int64_t)R.lrows.size();
        build_csr(R.n_halo + R.n_oshared, hrc, R.hrowptr, R.hcols);
        build_csr(R.nlr, lrc, R.lrowptr, R.lcols);
        for (int64_t t = 0; t < R.n_oshared; t++) slot[R.oshared[t]] = -1;
        // finalize rows: owned halo DOF -> its positions in the send list (= grecv)
        std::vector<std::pair<int32_t, int32_t>> frc;
        for (int64_t t = 0; t < R.n_oshared; t++) slot[R.oshared[t]] = (int32_t)t;
        for (int64_t q = 0; q < R.n_send; q++) frc.push_back({slot[R.send[q]], (int32_t)q});
        for (int64_t t = 0; t < R.n_oshared; t++) slot[R.oshared[t]] = -1;
        build_csr(R.n_oshared, frc, R.frowptr, R.fcols);

        // every index the kernels and copies will follow stays inside its buffer
        const int64_t lo = off[p], hi = off[p] + cnt[p], nsurf = Ep * NS;
        bool ok = true;
        for (int32_t c : R.lc) ok = ok && (c == -1 || (c >= lo && c < hi) || (c <= -2 && -2 - (int64_t)c < R.n_halo));
        // element-interior nodes are written to y directly: they must be owned
        for (int64_t el = 0; el < Ep && ok; el++)
            for (int k = 1; k < N; k++)
                for (int j = 1; j < N; j++)
                    for (int i = 1; i < N; i++) ok = ok && R.lc[(size_t)el * n3 + (k * n + j) * n + i] >= lo;
        for (int32_t c : R.send) ok = ok && c >= lo && c < hi;
        for (int32_t c : R.lrows) ok = ok && c >= lo && c < hi;
        for (int32_t c : R.oshared) ok = ok && c >= lo && c < hi;
        for (int32_t c : R.hcols) ok = ok && c >= 0 && c < nsurf;
        for (int32_t c : R.lcols) ok = ok && c >= 0 && c < nsurf;
        for (int32_t c : R.fcols) ok = ok && c >= 0 && c < R.n_send;
        ok = ok && (int64_t)R.hrowptr.back() == (int64_t)R.hcols.size() &&
             (int64_t)R.lrowptr.back() == (int64_t)R.lcols.size() && (int64_t)R.frowptr.back() == (int64_t)R.fcols.size();
        for (int64_t t = 0; t < R.n_oshared && ok; t++) ok = R.frowptr[t + 1] > R.frowptr[t];  // sent to someone
        for (int q = 0; q < Pn && ok; q++)
            ok = PL.R[q].recv_off[p + 1] - PL.R[q].recv_off[p] == R.send_off[q + 1] - R.send_off[q];
        if (!ok) {
            hb_set_error("partition of rank %d is inconsistent", p);
            return HB_ERR_ARG;
        }
    }
    return HB_OK;
}

hb_status build(hb_part *P, cudaStream_t s)
{
    const hb_mesh *m = P->m;
    const int N = m->N, n = N + 1, n3 = n * n * n;
    const int64_t E = m->E, NG = m->n_global;
    const int Pn = P->P;
    P->N = N;
    P->n = n;
    P->NS = hb_surf_count(N);
    P->n_global = NG;

    std::vector<int32_t> l2g((size_t)E * n3);
    HB_TRY_CUDA(cudaMemcpyAsync(l2g.data(), m->l2g, l2g.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    part_plan PL;
    hb_status st = plan_partition(l2g.data(), m->desc.ex, m->desc.ey, m->desc.ez, N, NG, P->px, P->py, P->pz,
                                  P->seed, PL);
    if (st != HB_OK) return st;
    P->n_shared = PL.n_shared;
    P->exchange_values = PL.exchange_values;
    P->perm = PL.perm;
    P->R.resize(Pn);
    for (int p = 0; p < Pn; p++) {
        const rank_plan &Q = PL.R[p];
        part_rank &R = P->R[p];
        R.off = Q.off;
        R.n_owned = Q.n_owned;
        R.n_halo = Q.n_halo;
        R.n_send = Q.n_send;
        R.n_oshared = Q.n_oshared;
        R.nlr = Q.nlr;
        R.e_int1 = Q.e_int1;
        R.e_halo = Q.e_halo;
        R.e_int2 = Q.e_int2;
        R.send_off = Q.send_off;
        R.recv_off = Q.recv_off;
        const int64_t Ep = (int64_t)Q.order.size();
        if ((st = upload(P, Q.lc, &R.l2g)) != HB_OK) return st;
        if ((st = upload(P, Q.send, &R.send_idx)) != HB_OK) return st;
        if ((st = upload(P, Q.hrowptr, &R.hrowptr)) != HB_OK) return st;
        if ((st = upload(P, Q.hcols, &R.hcols)) != HB_OK) return st;
        if ((st = upload(P, Q.lrows, &R.lrow_g)) != HB_OK) return st;
        if ((st = upload(P, Q.lrowptr, &R.lrowptr)) != HB_OK) return st;
        if ((st = upload(P, Q.lcols, &R.lcols)) != HB_OK) return st;
        if ((st = upload(P, Q.oshared, &R.frow_g)) != HB_OK) return st;
        if ((st = upload(P, Q.frowptr, &R.frowptr)) != HB_OK) return st;
        if ((st = upload(P, Q.fcols, &R.fcols)) != HB_OK) return st;
        if ((st = alloc(P, (size_t)Ep * 7 * n3, &R.geo)) != HB_OK) return st;
        if ((st = alloc(P, (size_t)Ep * P->NS, &R.ysurf)) != HB_OK) return st;
        if ((st = alloc(P, (size_t)R.n_halo, &R.halo)) != HB_OK) return st;
        if ((st = alloc(P, (size_t)R.n_send, &R.sendbuf)) != HB_OK) return st;
        if ((st = alloc(P, (size_t)(R.n_halo + R.n_oshared), &R.hbuf)) != HB_OK) return st;
        if ((st = alloc(P, (size_t)R.n_send, &R.grecv)) != HB_OK) return st;
        if (Ep > 0) {
            int32_t *d_el = nullptr;
            if ((st = upload(P, Q.order, &d_el)) != HB_OK) return st;
            hb_count_launch();
            k_gather_geo<<<grid_for(Ep * 7 * n3), kThreads, 0, s>>>(m->geo, d_el, Ep, (int64_t)7 * n3, R.geo);
            HB_CHECK_LAUNCH();
        }
        HB_TRY_CUDA(cudaStreamCreateWithFlags(&R.s, cudaStreamNonBlocking));
        HB_TRY_CUDA(cudaStreamCreateWithFlags(&R.sc, cudaStreamNonBlocking));
        for (cudaEvent_t *e : {&R.ev_pack, &R.ev_hin, &R.ev_gpk, &R.ev_grecv, &R.ev_done})
            HB_TRY_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    // lumped mass in partition order
    {
        int32_t *d_perm = nullptr;
        if ((st = upload(P, P->perm, &d_perm)) != HB_OK) return st;
        if ((st = alloc(P, (size_t)NG, &P->mdiag)) != HB_OK) return st;
        if (NG > 0) {
            hb_count_launch();
            k_permute<<<grid_for(NG), kThreads, 0, s>>>(m->mdiag, d_perm, NG, P->mdiag);
            HB_CHECK_LAUNCH();
        }
    }
    HB_TRY_CUDA(cudaEventCreateWithFlags(&P->ev_start, cudaEventDisableTiming));
    HB_TRY_CUDA(cudaEventCreate(&P->ev0));
    HB_TRY_CUDA(cudaEventCreate(&P->ev1));
    if ((st = alloc(P, (size_t)HB_RED_MAXV * HB_RED_BLOCKS, &P->partials)) != HB_OK) return st;
    if ((st = alloc(P, 8, &P->counters)) != HB_OK) return st;
    if ((st = alloc(P, 2, &P->state)) != HB_OK) return st;
    HB_TRY_CUDA(cudaMemsetAsync(P->counters, 0, 8 * sizeof(unsigned), s));
    HB_TRY_CUDA(cudaMallocHost((void **)&P->state_host, sizeof(hb_cg_state)));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    return HB_OK;
}

// The element kernel on local elements [e0, e0 + count) of rank R.
hb_status rank_elements(const hb_part *P, const part_rank &R, int64_t e0, int64_t count, const double *x, double *y,
                        int screen, double lambda, const int *run, int eo, int ebm)
{
    if (count <= 0) return HB_OK;
    const int64_t n3 = (int64_t)P->n * P->n * P->n;
    return hb_launch_ax2_f64_range(P->N, count, x, R.halo, R.l2g + e0 * n3, R.geo + e0 * 7 * n3,
                                   R.ysurf + e0 * P->NS, y, lambda, screen, run, eo, ebm, R.s);
}

// Every rank's halo buffer from x: pack on the owners' streams, copies on the
// receivers' exchange streams (recorded into ev_pack / ev_hin).
hb_status enqueue_pack(const hb_part *P, const double *x)
{
    for (const part_rank &R : P->R) {
        if (R.n_send > 0) {
            hb_prof_scope prof("part_pack", R.s);
            k_pack<<<grid_for(R.n_send), kThreads, 0, R.s>>>(x, R.send_idx, R.n_send, R.sendbuf);
            HB_CHECK_LAUNCH();
        }
        HB_TRY_CUDA(cudaEventRecord(R.ev_pack, R.s));
    }
    return HB_OK;
}

hb_status enqueue_halo_copies(const hb_part *P)
{
    for (int q = 0; q < P->P; q++) {
        const part_rank &Q = P->R[q];
        for (int p = 0; p < P->P; p++) {
            const int64_t len = Q.recv_off[p + 1] - Q.recv_off[p];
            if (len == 0) continue;
            const part_rank &Rp = P->R[p];
            HB_TRY_CUDA(cudaStreamWaitEvent(Q.sc, Rp.ev_pack, 0));
            HB_TRY_CUDA(cudaMemcpyAsync(Q.halo + Q.recv_off[p], Rp.sendbuf + Rp.send_off[q], len * sizeof(double),
                                        cudaMemcpyDeviceToDevice, Q.sc));
        }
        HB_TRY_CUDA(cudaEventRecord(Q.ev_hin, Q.sc));
    }
    return HB_OK;
}

hb_status fork(const hb_part *P, cudaStream_t s)
{
    HB_TRY_CUDA(cudaEventRecord(P->ev_start, s));
    for (const part_rank &R : P->R) {
        HB_TRY_CUDA(cudaStreamWaitEvent(R.s, P->ev_start, 0));
        HB_TRY_CUDA(cudaStreamWaitEvent(R.sc, P->ev_start, 0));
    }
    return HB_OK;
}

hb_status join(const hb_part *P, cudaStream_t s)
{
    for (const part_rank &R : P->R) {
        HB_TRY_CUDA(cudaEventRecord(R.ev_done, R.s));
        HB_TRY_CUDA(cudaStreamWaitEvent(s, R.ev_done, 0));
        HB_TRY_CUDA(cudaEventRecord(R.ev_done, R.sc));
        HB_TRY_CUDA(cudaStreamWaitEvent(s, R.ev_done, 0));
    }
    return HB_OK;
}

hb_status part_apply(const hb_part *P, int screen, double lambda, const double *x, double *y, const int *run,
                     cudaStream_t s)
{
    const int v = P->m->variant[0];
    const int eo = (v & HB_VAR_PENCIL) ? ((v & HB_VAR_EO) ? 1 : 0) : 1;
    const int ebm = (v & HB_VAR_PENCIL) ? ((v & HB_VAR_ONE) ? 0 : ((v & HB_VAR_EB2) ? 2 : 1)) : 1;
    hb_status st;
    if ((st = fork(P, s)) != HB_OK) return st;
    if ((st = enqueue_pack(P, x)) != HB_OK) return st;
    // first half of the interior elements, while the halo values travel
    for (const part_rank &R : P->R)
        if ((st = rank_elements(P, R, 0, R.e_int1, x, y, screen, lambda, run, eo, ebm)) != HB_OK) return st;
    if ((st = enqueue_halo_copies(P)) != HB_OK) return st;
    // halo elements, their halo-node sums, then the other interior half and
    // the rank-local gather while the partial sums travel
    for (const part_rank &R : P->R) {
        HB_TRY_CUDA(cudaStreamWaitEvent(R.s, R.ev_hin, 0));
        if ((st = rank_elements(P, R, R.e_int1, R.e_halo, x, y, screen, lambda, run, eo, ebm)) != HB_OK) return st;
        const int64_t nh = R.n_halo + R.n_oshared;
        if (nh > 0) {
            hb_prof_scope prof("part_halo_gather", R.s);
            k_rowsum<<<grid_for(nh), kThreads, 0, R.s>>>(R.ysurf, R.hrowptr, R.hcols, nh, R.hbuf);
            HB_CHECK_LAUNCH();
        }
        HB_TRY_CUDA(cudaEventRecord(R.ev_gpk, R.s));
        if ((st = rank_elements(P, R, R.e_int1 + R.e_halo, R.e_int2, x, y, screen, lambda, run, eo, ebm)) != HB_OK)
            return st;
        if (R.nlr > 0) {
            hb_prof_scope prof("part_local_gather", R.s);
            const int grid = red_grid(R.nlr);
            if (screen)
                k_local_gather<1><<<grid, HB_RED_THREADS, 0, R.s>>>(R.ysurf, R.lrow_g, R.lrowptr, R.lcols, x,
                                                                   P->mdiag, lambda, y, R.nlr);
            else
                k_local_gather<0><<<grid, HB_RED_THREADS, 0, R.s>>>(R.ysurf, R.lrow_g, R.lrowptr, R.lcols, x,
                                                                   P->mdiag, lambda, y, R.nlr);
            HB_CHECK_LAUNCH();
        }
    }
    // gather exchange: p's partials at q's DOFs -> q's grecv (laid out like q's send list)
    for (int q = 0; q < P->P; q++) {
        const part_rank &Q = P->R[q];
        for (int p = 0; p < P->P; p++) {
            const int64_t len = Q.send_off[p + 1] - Q.send_off[p];
            if (len == 0) continue;
            const part_rank &Rp = P->R[p];
            HB_TRY_CUDA(cudaStreamWaitEvent(Q.sc, Rp.ev_gpk, 0));
            HB_TRY_CUDA(cudaMemcpyAsync(Q.grecv + Q.send_off[p], Rp.hbuf + Rp.recv_off[q], len * sizeof(double),
                                        cudaMemcpyDeviceToDevice, Q.sc));
        }
        HB_TRY_CUDA(cudaEventRecord(Q.ev_grecv, Q.sc));
    }
    for (const part_rank &R : P->R) {
        HB_TRY_CUDA(cudaStreamWaitEvent(R.s, R.ev_grecv, 0));
        if (R.n_oshared > 0) {
            hb_prof_scope prof("part_final", R.s);
            if (screen)
                k_final<1><<<grid_for(R.n_oshared), kThreads, 0, R.s>>>(R.hbuf + R.n_halo, R.grecv, R.frow_g,
                                                                         R.frowptr, R.fcols, R.n_oshared, x,
                                                                         P->mdiag, lambda, y);
            else
                k_final<0><<<grid_for(R.n_oshared), kThreads, 0, R.s>>>(R.hbuf + R.n_halo, R.grecv, R.frow_g,
                                                                         R.frowptr, R.fcols, R.n_oshared, x,
                                                                         P->mdiag, lambda, y);
            HB_CHECK_LAUNCH();
        }
    }
    return join(P, s);
}

bool valid_screen(int s) { return s == HB_SCREEN_IDENTITY || s == HB_SCREEN_MASS; }

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" hb_status hb_part_create(const hb_mesh *mesh, int px, int py, int pz, uint64_t seed, void *stream,
                                    hb_part **out)
{
    hb_clear_error();
    if (!mesh || !out) { hb_set_error("null argument"); return HB_ERR_ARG; }
    *out = nullptr;
    if (px < 1 || py < 1 || pz < 1 || px > mesh->desc.ex || py > mesh->desc.ey || pz > mesh->desc.ez) {
        hb_set_error("rank grid %dx%dx%d does not fit %dx%dx%d elements", px, py, pz, mesh->desc.ex, mesh->desc.ey,
                     mesh->desc.ez);
        return HB_ERR_ARG;
    }
    if (px * py * pz > 64) { hb_set_error("at most 64 ranks"); return HB_ERR_ARG; }
    hb_device_guard dg(mesh->device);
    if (!dg.ok) { hb_set_error("cannot select device %d", mesh->device); return HB_ERR_CUDA; }
    hb_part *P = new hb_part();
    P->m = mesh;
    P->device = mesh->device;
    P->px = px;
    P->py = py;
    P->pz = pz;
    P->P = px * py * pz;
    P->seed = seed;
    hb_status st = build(P, (cudaStream_t)stream);
    if (st != HB_OK) {
        free_part(P);
        return st;
    }
    *out = P;
    return HB_OK;
}

extern "C" hb_status hb_part_plan(const int32_t *l2g_host, int ex, int ey, int ez, int N, int64_t n_global,
                                  int px, int py, int pz, uint64_t seed, int32_t *perm_host, int64_t *counts_host)
{
    hb_clear_error();
    if (!l2g_host || !perm_host || !counts_host) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (ex < 1 || ey < 1 || ez < 1 || N < 1 || N > HB_MAX_N || n_global < 0) { hb_set_error("bad mesh sizes"); return HB_ERR_ARG; }
    if (px < 1 || py < 1 || pz < 1 || px > ex || py > ey || pz > ez || px * py * pz > 64) {
        hb_set_error("rank grid %dx%dx%d does not fit %dx%dx%d elements (at most 64 ranks)", px, py, pz, ex, ey, ez);
        return HB_ERR_ARG;
    }
    part_plan PL;
    hb_status st = plan_partition(l2g_host, ex, ey, ez, N, n_global, px, py, pz, seed, PL);
    if (st != HB_OK) return st;
    if (!PL.perm.empty()) std::memcpy(perm_host, PL.perm.data(), PL.perm.size() * sizeof(int32_t));
    const int Pn = px * py * pz;
    counts_host[0] = PL.n_shared;
    counts_host[1] = PL.exchange_values;
    for (int p = 0; p < Pn; p++) {
        const rank_plan &R = PL.R[p];
        int64_t *c = counts_host + 2 + 8 * p;
        c[0] = R.n_owned;
        c[1] = R.off;
        c[2] = R.n_halo;
        c[3] = R.n_send;
        c[4] = R.e_int1;
        c[5] = R.e_halo;
        c[6] = R.e_int2;
        c[7] = R.n_oshared;
    }
    return HB_OK;
}

extern "C" hb_status hb_part_destroy(hb_part *part)
{
    hb_clear_error();
    if (!part) return HB_OK;
    hb_device_guard dg(part->device);
    for (const part_rank &R : part->R) {
        if (R.s) cudaStreamSynchronize(R.s);
        if (R.sc) cudaStreamSynchronize(R.sc);
    }
    free_part(part);
    return HB_OK;
}

extern "C" hb_status hb_part_info(const hb_part *part, hb_part_info_t *out)
{
    hb_clear_error();
    if (!part || !out) { hb_set_error("null argument"); return HB_ERR_ARG; }
    out->n_ranks = part->P;
    out->n_global = part->n_global;
    out->n_shared = part->n_shared;
    out->exchange_values = part->exchange_values;
    return HB_OK;
}

extern "C" hb_status hb_part_rank_info(const hb_part *part, int rank, hb_part_rank_info_t *out)
{
    hb_clear_error();
    if (!part || !out) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (rank < 0 || rank >= part->P) { hb_set_error("rank %d out of range", rank); return HB_ERR_ARG; }
    const part_rank &R = part->R[rank];
    out->n_owned = R.n_owned;
    out->offset = R.off;
    out->n_halo = R.n_halo;
    out->n_send = R.n_send;
    out->n_elem_interior1 = R.e_int1;
    out->n_elem_halo = R.e_halo;
    out->n_elem_interior2 = R.e_int2;
    return HB_OK;
}

extern "C" hb_status hb_part_copy_perm(const hb_part *part, int32_t *perm_host)
{
    hb_clear_error();
    if (!part || !perm_host) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!part->perm.empty()) std::memcpy(perm_host, part->perm.data(), part->perm.size() * sizeof(int32_t));
    return HB_OK;
}

extern "C" hb_status hb_part_apply_A(const hb_part *part, hb_screen screen, double lambda, const double *x,
                                     double *y, void *stream)
{
    hb_clear_error();
    if (!part || !x || !y) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (!valid_screen(screen)) { hb_set_error("invalid screen %d", (int)screen); return HB_ERR_ARG; }
    if (x == y) { hb_set_error("x and y must not overlap"); return HB_ERR_ARG; }
    if (part->n_global == 0) return HB_OK;
    hb_device_guard dg(part->device);
    return part_apply(part, screen, lambda, x, y, nullptr, (cudaStream_t)stream);
}

extern "C" hb_status hb_part_halo_exchange(const hb_part *part, const double *x, int rank, double *halo_host,
                                           void *stream)
{
    hb_clear_error();
    if (!part || !x) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (halo_host && (rank < 0 || rank >= part->P)) { hb_set_error("rank %d out of range", rank); return HB_ERR_ARG; }
    hb_device_guard dg(part->device);
    cudaStream_t s = (cudaStream_t)stream;
    hb_status st;
    if ((st = fork(part, s)) != HB_OK) return st;
    if ((st = enqueue_pack(part, x)) != HB_OK) return st;
    if ((st = enqueue_halo_copies(part)) != HB_OK) return st;
    if ((st = join(part, s)) != HB_OK) return st;
    if (halo_host) {
        const part_rank &R = part->R[rank];
        if (R.n_halo > 0)
            HB_TRY_CUDA(cudaMemcpyAsync(halo_host, R.halo, R.n_halo * sizeof(double), cudaMemcpyDeviceToHost, s));
        HB_TRY_CUDA(cudaStreamSynchronize(s));
    }
    return HB_OK;
}

extern "C" hb_status hb_part_cg_solve(const hb_part *part, const hb_cg_opts *o, const double *b, double *x,
                                      hb_cg_result *res, void *stream)
{
    hb_clear_error();
    hb_cg_result R{};
    R.status = HB_OK;
    if (res) *res = R;
    if (!part || !o || !b || !x) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (o->prec != HB_F64) { hb_set_error("hb_part_cg_solve takes HB_F64"); return HB_ERR_ARG; }
    if (o->precond != 0) { hb_set_error("hb_part_cg_solve has no preconditioner"); return HB_ERR_ARG; }
    if (!valid_screen(o->screen) || o->max_it < 0 || !(o->rtol >= 0.0)) {
        hb_set_error("invalid options");
        return HB_ERR_ARG;
    }
    hb_device_guard dg(part->device);
    hb_part *P = const_cast<hb_part *>(part);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = P->n_global;
    if (n == 0) {
        if (res) *res = R;
        return HB_OK;
    }
    const int64_t stride = (n + 63) / 64 * 64;
    const size_t need = (size_t)stride * 3 * sizeof(double);
    if (P->cg_vec_bytes < need) {
        if (P->cg_vec) {
            cudaFree(P->cg_vec);
            P->allocs.erase(std::find(P->allocs.begin(), P->allocs.end(), (void *)P->cg_vec));
        }
        P->cg_vec = nullptr;
        P->cg_vec_bytes = 0;
        HB_TRY_CUDA(cudaMalloc((void **)&P->cg_vec, need));
        P->allocs.push_back(P->cg_vec);
        P->cg_vec_bytes = need;
    }
    double *r = P->cg_vec, *p = r + stride, *Ap = p + stride;
    hb_cg_state *st = P->state;
    const int grid = red_grid(n);
    HB_TRY_CUDA(cudaEventRecord(P->ev0, s));
    hb_status rs = part_apply(P, o->screen, o->lambda, x, Ap, nullptr, s);
    if (rs != HB_OK) return rs;
    hb_count_launch();
    k_cg_init<<<grid, HB_RED_THREADS, 0, s>>>(b, Ap, r, p, n, o->rtol, o->max_it, P->partials, P->counters + 2, st);
    HB_CHECK_LAUNCH();
    // iterations in chunks; kernels of a finished solve return at once. With a
    // tolerance, a stop of the recursive residual is checked on the true one
    // (b - A x; Algorithm 1 restarts from x while it is above rtol and each
    // restart lowers it by a tenth at least).
    int chunk = 16;
    bool checked = false;
    double prev = -1.0;
    hb_cg_state fin{};
    for (;;) {
        HB_TRY_CUDA(cudaMemcpyAsync(P->state_host, st, sizeof(hb_cg_state), cudaMemcpyDeviceToHost, s));
        HB_TRY_CUDA(cudaStreamSynchronize(s));
        fin = *P->state_host;
        if (!fin.run || fin.it >= o->max_it) {
            if (o->rtol > 0.0 && fin.status == HB_OK && !checked) {
                if ((rs = part_apply(P, o->screen, o->lambda, x, Ap, nullptr, s)) != HB_OK) return rs;
                hb_count_launch();
                k_cg_restart<<<grid, HB_RED_THREADS, 0, s>>>(b, Ap, r, p, n, P->partials, P->counters + 2, st);
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
            if ((rs = part_apply(P, o->screen, o->lambda, p, Ap, &st->run, s)) != HB_OK) return rs;
            {
                hb_prof_scope prof("part_pap", s);
                k_pap<<<grid, HB_RED_THREADS, 0, s>>>(p, Ap, n, P->partials, P->counters + 1, st);
                HB_CHECK_LAUNCH();
            }
            {
                hb_prof_scope prof("cg_update_r", s);
                k_cg_update_r<<<grid, HB_RED_THREADS, 0, s>>>(r, Ap, n, P->partials, P->counters + 2, st);
                HB_CHECK_LAUNCH();
            }
            {
                hb_prof_scope prof("cg_update_xp", s);
                k_cg_update_xp<<<grid, HB_RED_THREADS, 0, s>>>(x, p, r, n, P->counters + 3, st);
                HB_CHECK_LAUNCH();
            }
        }
        chunk = std::min(chunk * 2, 256);
    }
    HB_TRY_CUDA(cudaEventRecord(P->ev1, s));
    HB_TRY_CUDA(cudaEventSynchronize(P->ev1));
    float ms = 0.f;
    HB_TRY_CUDA(cudaEventElapsedTime(&ms, P->ev0, P->ev1));
    R.iters = fin.it;
    R.rel_res = fin.bb > 0.0 ? std::sqrt(fin.res2 / fin.bb) : 0.0;
    R.time_ms = ms;
    if (fin.status == HB_ERR_BREAKDOWN) R.status = HB_ERR_BREAKDOWN;
    else if (o->rtol > 0.0 && fin.res2 > fin.tol2) R.status = HB_ERR_NOT_CONVERGED;
    if (res) *res = R;
    return R.status;
}
