// Mesh setup on the device: reference element, node map, Z^T as CSR and the
// geometric factors (hipBone, arXiv 2202.12477, Sec. 2 and Sec. 3.2).
//
// Routes chosen here on purpose differ from the textbook closed forms:
//   - GLL nodes by Newton's method on q(x) = (1-x^2) P_N'(x) written as
//     N (P_{N-1}(x) - x P_N(x)), with q'(x) = -N(N+1) P_N(x);
//   - the derivative matrix from barycentric weights, diagonal by negative sums;
//   - the Jacobian by applying that derivative matrix to the nodal coordinates
//     (exact, since a trilinear map is a polynomial of degree 1 <= N per axis).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "hb_internal.h"

// ---------------------------------------------------------------- errors

static thread_local char g_err[512];

void hb_set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}
void hb_clear_error() { g_err[0] = 0; }

extern "C" const char *hb_last_error(void) { return g_err; }

// ---------------------------------------------------------------- random numbers

__host__ __device__ static inline uint64_t hb_splitmix64(uint64_t state)
{
    uint64_t z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ static inline double hb_u01_impl(uint64_t seed, uint64_t stream, uint64_t idx)
{
    uint64_t s = (seed ^ (stream * 0x9E3779B97F4A7C15ull)) + idx;
    return (double)(hb_splitmix64(s) >> 11) * 0x1.0p-53;
}

extern "C" double hb_u01(uint64_t seed, uint64_t stream, uint64_t idx)
{
    return hb_u01_impl(seed, stream, idx);
}

// ---------------------------------------------------------------- reference element

static void legendre_pair(int N, double x, double *PN, double *PNm1)
{
    double a = 1.0, b = x;  // P_0, P_1
    if (N == 1) { *PN = b; *PNm1 = a; return; }
    for (int k = 2; k <= N; k++) {
        double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    *PN = b;
    *PNm1 = a;
}

void hb_reference_element(int N, double *xi, double *w, double *D)
{
    const int n = N + 1;
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int i = 1; i < N; i++) {
        double x = -std::cos(M_PI * i / N);
        for (int it = 0; it < 200; it++) {
            double P, Pm;
            legendre_pair(N, x, &P, &Pm);
            // q = N (P_{N-1} - x P_N), q' = -N (N+1) P_N  =>  dx = -q / q'
            double dx = (Pm - x * P) / ((N + 1) * P);
            x += dx;
            if (std::fabs(dx) <= 1e-17) break;
        }
        xi[i] = x;
    }
    for (int i = 0; i < n / 2; i++) {  // symmetric node set
        double a = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -a;
        xi[N - i] = a;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int i = 0; i < n; i++) {
        double P, Pm;
        legendre_pair(N, xi[i], &P, &Pm);
        w[i] = 2.0 / (N * (N + 1.0) * P * P);
    }
    // barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k)
    std::vector<double> lam(n);
    for (int j = 0; j < n; j++) {
        double p = 1.0;
        for (int k = 0; k < n; k++)
            if (k != j) p *= (xi[j] - xi[k]);
        lam[j] = 1.0 / p;
    }
    for (int i = 0; i < n; i++) {
        double diag = 0.0;
        for (int j = 0; j < n; j++) {
            if (i == j) continue;
            double v = (lam[j] / lam[i]) / (xi[i] - xi[j]);
            D[i * n + j] = v;
            diag -= v;
        }
        D[i * n + i] = diag;
    }
    // D is centro-antisymmetric; make the computed matrix exactly so
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            int ii = N - i, jj = N - j;
            if (i * n + j < ii * n + jj) {
                double a = 0.5 * (D[i * n + j] - D[ii * n + jj]);
                D[i * n + j] = a;
                D[ii * n + jj] = -a;
            } else if (i == ii && j == jj) {
                D[i * n + j] = 0.0;
            }
        }
}

// ---------------------------------------------------------------- device tables

static int d_offset(int N)
{
    int o = 0;
    for (int M = 1; M < N; M++) o += (M + 1) * (M + 1);
    return o;
}
static const int kTableSize = 1496;  // sum_{N=1..15} (N+1)^2 = 1495

__device__ double g_D64[kTableSize];
__device__ float g_D32[kTableSize];
__device__ double g_xi64[16 * 16];   // [N][i]
__device__ double g_w64[16 * 16];

static std::mutex g_table_mu;
static unsigned g_table_done = 0;  // bit per device (devices 0..31)
static double *g_dev_D64[32];
static float *g_dev_D32[32];

hb_status hb_ensure_device_tables()
{
    int dev = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 32) { hb_set_error("device index %d unsupported", dev); return HB_ERR_ARG; }
    std::lock_guard<std::mutex> lk(g_table_mu);
    if (g_table_done & (1u << dev)) return HB_OK;
    std::vector<double> D64(kTableSize, 0.0), xi(256, 0.0), w(256, 0.0);
    std::vector<float> D32(kTableSize, 0.0f);
    for (int N = 1; N <= HB_MAX_N; N++) {
        int n = N + 1;
        std::vector<double> x(n), ww(n), D(n * n);
        hb_reference_element(N, x.data(), ww.data(), D.data());
        for (int q = 0; q < n * n; q++) {
            D64[d_offset(N) + q] = D[q];
            D32[d_offset(N) + q] = (float)D[q];
        }
        for (int i = 0; i < n; i++) { xi[N * 16 + i] = x[i]; w[N * 16 + i] = ww[i]; }
    }
    { hb_status st2 = hb_ax2_upload_f64(D64.data()); if (st2 != HB_OK) return st2; }
    { hb_status st2 = hb_ax2_upload_f32(D64.data()); if (st2 != HB_OK) return st2; }
    { hb_status st2 = hb_ax2_upload_f64x(D64.data()); if (st2 != HB_OK) return st2; }
    { hb_status st2 = hb_cg_fused_upload(D64.data()); if (st2 != HB_OK) return st2; }
    { hb_status st2 = hb_tc_upload(); if (st2 != HB_OK) return st2; }
    HB_TRY_CUDA(cudaMemcpyToSymbol(g_D64, D64.data(), sizeof(double) * kTableSize));
    HB_TRY_CUDA(cudaMemcpyToSymbol(g_D32, D32.data(), sizeof(float) * kTableSize));
    HB_TRY_CUDA(cudaMemcpyToSymbol(g_xi64, xi.data(), sizeof(double) * 256));
    HB_TRY_CUDA(cudaMemcpyToSymbol(g_w64, w.data(), sizeof(double) * 256));
    void *p64 = nullptr, *p32 = nullptr;
    HB_TRY_CUDA(cudaGetSymbolAddress(&p64, g_D64));
    HB_TRY_CUDA(cudaGetSymbolAddress(&p32, g_D32));
    g_dev_D64[dev] = (double *)p64;
    g_dev_D32[dev] = (float *)p32;
    g_table_done |= 1u << dev;
    return HB_OK;
}

const double *hb_dev_D64(int N)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return g_dev_D64[dev] + d_offset(N);
}
const float *hb_dev_D32(int N)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return g_dev_D32[dev] + d_offset(N);
}

// ---------------------------------------------------------------- setup kernels

static int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}


struct box_t {
    int Ex, Ey, Ez, N;
    unsigned faces;
};

// Node map: lexicographic ids over unmasked lattice nodes, by closed form.
__global__ void k_l2g(box_t b, int64_t n_local, int32_t *l2g)
{
    const int n = b.N + 1;
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t NX = (int64_t)b.N * b.Ex + 1, NY = (int64_t)b.N * b.Ey + 1, NZ = (int64_t)b.N * b.Ez + 1;
    const int x0 = b.faces & 1u ? 1 : 0, x1 = b.faces & 2u ? 1 : 0;
    const int y0 = b.faces & 4u ? 1 : 0, y1 = b.faces & 8u ? 1 : 0;
    const int z0 = b.faces & 16u ? 1 : 0, z1 = b.faces & 32u ? 1 : 0;
    const int64_t NXu = NX - x0 - x1, NYu = NY - y0 - y1;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_local;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t e = q / n3;
        int node = (int)(q - e * n3);
        int i = node % n, j = (node / n) % n, k = node / (n * n);
        int64_t ex = e % b.Ex, ey = (e / b.Ex) % b.Ey, ez = e / ((int64_t)b.Ex * b.Ey);
        int64_t I = b.N * ex + i, J = b.N * ey + j, K = b.N * ez + k;
        bool masked = (x0 && I == 0) || (x1 && I == NX - 1) || (y0 && J == 0) || (y1 && J == NY - 1) ||
                      (z0 && K == 0) || (z1 && K == NZ - 1);
        l2g[q] = masked ? -1 : (int32_t)((I - x0) + NXu * ((J - y0) + NYu * (K - z0)));
    }
}

__device__ inline void vertex_pos(const box_t &b, double rho, uint64_t seed, int a, int bb, int c,
                                  double X[3])
{
    X[0] = (double)a / b.Ex;
    X[1] = (double)bb / b.Ey;
    X[2] = (double)c / b.Ez;
    if (a > 0 && a < b.Ex && bb > 0 && bb < b.Ey && c > 0 && c < b.Ez) {
        const double h[3] = {1.0 / b.Ex, 1.0 / b.Ey, 1.0 / b.Ez};
        uint64_t v = ((uint64_t)c * (b.Ey + 1) + bb) * (b.Ex + 1) + a;
        for (int ax = 0; ax < 3; ax++) {
            double u = hb_u01_impl(seed, 1, 3 * v + ax);
            X[ax] += (2.0 * u - 1.0) * rho * h[ax];
        }
    }
}

// Geometric factors, one element per block. The element map is trilinear in
// its 8 vertices, x(r, s, t) = sum_{a,b,c} V_abc phi_a(r) phi_b(s) phi_c(t)
// with phi_0 = (1 - r) / 2, phi_1 = (1 + r) / 2, so its Jacobian column along
// one reference direction is bilinear in the other two coordinates:
//   dx/dr = sum_{b,c} (V_1bc - V_0bc) / 2 phi_b(s) phi_c(t)
// (and likewise for s and t). Each column is formed once per line of nodes
// (3 n^2 lines per element, not n^3 nodes) and shared through shared memory;
// per node, with the adjugate rows a_l (a_r = j_s x j_t, a_s = j_t x j_r,
// a_t = j_r x j_s) and det J = j_r . a_r,
//   G_lm = w_ijk det J (J^-1 J^-T)_lm = (w_ijk / det J) a_l . a_m,
// the six factors of Sec. 2 and the weighted Jacobian w_ijk det J.
__global__ void k_geometry(box_t b, double rho, uint64_t seed, int64_t E, double *geo, float *geo32,
                           double *detmin_blk)
{
    extern __shared__ double smem[];
    const int N = b.N, n = N + 1, n2 = n * n, n3 = n2 * n;
    double *col = smem;  // [direction l][axis][line (u + n v)]: column l of J on the line
    __shared__ double V[8][3];
    __shared__ double dV[3][4][3];  // [direction][pair (p + 2 q)][axis]: halved edge differences
    __shared__ double red[32];
    const double *xi = g_xi64 + N * 16, *w = g_w64 + N * 16;
    double dmin = INFINITY;
    for (int64_t e = blockIdx.x; e < E; e += gridDim.x) {
        const int ex = (int)(e % b.Ex), ey = (int)((e / b.Ex) % b.Ey), ez = (int)(e / ((int64_t)b.Ex * b.Ey));
        __syncthreads();  // the previous element's columns are consumed
        if (threadIdx.x < 8) {
            const int a = threadIdx.x & 1, bb = (threadIdx.x >> 1) & 1, c = threadIdx.x >> 2;
            vertex_pos(b, rho, seed, ex + a, ey + bb, ez + c, V[threadIdx.x]);
        }
        __syncthreads();
        if (threadIdx.x < 36) {
            // vertex (a, bb, c) at (c * 2 + bb) * 2 + a. Direction l steps a (r),
            // bb (s) or c (t); p and q are the vertex sides of the line's first
            // and second coordinate: (bb, c) for r, (a, c) for s, (a, bb) for t
            const int l = threadIdx.x / 12, pq = (threadIdx.x / 3) % 4, ax = threadIdx.x % 3;
            const int p = pq & 1, q = pq >> 1;
            const int v0 = l == 0 ? (q * 2 + p) * 2 : (l == 1 ? q * 4 + p : q * 2 + p);
            const int step = 1 << l;
            dV[l][pq][ax] = 0.5 * (V[v0 + step][ax] - V[v0][ax]);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 3 * n2; t += blockDim.x) {
            const int l = t / n2, line = t % n2, u = line % n, v = line / n;
            // the two coordinates of the line: (s, t) for l = r, (r, t) for l = s, (r, s) for l = t
            const double fu0 = 0.5 - 0.5 * xi[u], fu1 = 0.5 + 0.5 * xi[u];
            const double fv0 = 0.5 - 0.5 * xi[v], fv1 = 0.5 + 0.5 * xi[v];
            for (int ax = 0; ax < 3; ax++) {
                // pair (p, q): p the first line coordinate's vertex side, q the second's
                const double c0 = fma(dV[l][1][ax], fu1, dV[l][0][ax] * fu0);
                const double c1 = fma(dV[l][3][ax], fu1, dV[l][2][ax] * fu0);
                col[(l * 3 + ax) * n2 + line] = fma(c1, fv1, c0 * fv0);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            const int i = q % n, j = (q / n) % n, k = q / n2;
            double jr[3], js[3], jt[3];
            for (int ax = 0; ax < 3; ax++) {
                jr[ax] = col[(0 * 3 + ax) * n2 + j + n * k];
                js[ax] = col[(1 * 3 + ax) * n2 + i + n * k];
                jt[ax] = col[(2 * 3 + ax) * n2 + i + n * j];
            }
            double ar[3], as[3], at[3];
            ar[0] = fma(js[1], jt[2], -js[2] * jt[1]);
            ar[1] = fma(js[2], jt[0], -js[0] * jt[2]);
            ar[2] = fma(js[0], jt[1], -js[1] * jt[0]);
            as[0] = fma(jt[1], jr[2], -jt[2] * jr[1]);
            as[1] = fma(jt[2], jr[0], -jt[0] * jr[2]);
            as[2] = fma(jt[0], jr[1], -jt[1] * jr[0]);
            at[0] = fma(jr[1], js[2], -jr[2] * js[1]);
            at[1] = fma(jr[2], js[0], -jr[0] * js[2]);
            at[2] = fma(jr[0], js[1], -jr[1] * js[0]);
            const double det = fma(jr[2], ar[2], fma(jr[1], ar[1], jr[0] * ar[0]));
            const double wq = w[i] * w[j] * w[k];
            const double sc = wq / det;
            double g[7];
            g[0] = sc * fma(ar[2], ar[2], fma(ar[1], ar[1], ar[0] * ar[0]));
            g[1] = sc * fma(ar[2], as[2], fma(ar[1], as[1], ar[0] * as[0]));
            g[2] = sc * fma(ar[2], at[2], fma(ar[1], at[1], ar[0] * at[0]));
            g[3] = sc * fma(as[2], as[2], fma(as[1], as[1], as[0] * as[0]));
            g[4] = sc * fma(as[2], at[2], fma(as[1], at[1], as[0] * at[0]));
            g[5] = sc * fma(at[2], at[2], fma(at[1], at[1], at[0] * at[0]));
            g[6] = wq * det;
            const int64_t base = ((e * n + k) * 7) * (int64_t)n2 + j * n + i;
            for (int c = 0; c < 7; c++) {
                geo[base + (int64_t)c * n2] = g[c];
                if (geo32) geo32[base + (int64_t)c * n2] = (float)g[c];
            }
            dmin = fmin(dmin, det);
        }
    }
    // block minimum of det J
    for (int o = 16; o > 0; o >>= 1) dmin = fmin(dmin, __shfl_down_sync(0xffffffffu, dmin, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dmin;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = red[0];
        for (int q = 1; q < (int)(blockDim.x + 31) / 32; q++) m = fmin(m, red[q]);
        detmin_blk[blockIdx.x] = m;
    }
}

__global__ void k_count(const int32_t *l2g, int64_t n_local, int32_t *cnt)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_local;
         q += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = l2g[q];
        if (g >= 0) atomicAdd(&cnt[g], 1);
    }
}

// Exclusive scan in three passes over chunks of 1024 entries.
__global__ void k_scan_chunks(const int32_t *in, int64_t n, int32_t *out, int64_t *chunk_sum)
{
    __shared__ int64_t s[1024];
    int64_t base = (int64_t)blockIdx.x * 1024;
    int t = threadIdx.x;
    int64_t v = base + t < n ? in[base + t] : 0;
    s[t] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int64_t a = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += a;
        __syncthreads();
    }
    if (base + t < n) out[base + t] = (int32_t)(s[t] - v);
    if (t == 1023) chunk_sum[blockIdx.x] = s[t];
}

// Exclusive scan of the chunk sums in place (chunk_sum[nchunks] = the total):
// one block of 1024 threads walks the sums in tiles of 1024, a warp-shuffle
// scan per tile plus the running carry. Launch with 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t *chunk_sum, int64_t nchunks)
{
    __shared__ int64_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int64_t carry = 0;
    for (int64_t base = 0; base < nchunks; base += 1024) {
        const int64_t c = base + t;
        const int64_t v = c < nchunks ? chunk_sum[c] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t z = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            wsum[lane] = z;
        }
        __syncthreads();
        const int64_t incl = x + (w > 0 ? wsum[w - 1] : 0);
        if (c < nchunks) chunk_sum[c] = carry + incl - v;
        carry += wsum[31];
        __syncthreads();  // wsum is rewritten by the next tile
    }
    if (t == 0) chunk_sum[nchunks] = carry;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int64_t *chunk_sum)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (int32_t)(out[q] + chunk_sum[q / 1024]);
}

__global__ void k_fill(const int32_t *l2g, int64_t n_local, const int32_t *rowptr, int32_t *cursor,
                       int32_t *cols)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_local;
         q += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = l2g[q];
        if (g >= 0) {
            int slot = atomicAdd(&cursor[g], 1);
            cols[rowptr[g] + slot] = (int32_t)q;
        }
    }
}

// Sort every row ascending (rows are short) and sum the mass diagonal in that order.
__global__ void k_sort_rows(const int32_t *rowptr, int32_t *cols, int64_t ng, const double *geo, int n,
                            double *mdiag, float *mdiag32)
{
    const int n2 = n * n, n3 = n2 * n;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x) {
        int a = rowptr[g], z = rowptr[g + 1];
        for (int p = a + 1; p < z; p++) {
            int32_t v = cols[p];
            int q = p - 1;
            while (q >= a && cols[q] > v) { cols[q + 1] = cols[q]; q--; }
            cols[q + 1] = v;
        }
        double m = 0.0;
        for (int p = a; p < z; p++) {
            int64_t lq = cols[p];
            int64_t e = lq / n3;
            int node = (int)(lq - e * n3);
            int k = node / n2, ij = node - k * n2;
            m += geo[((e * n + k) * 7 + 6) * (int64_t)n2 + ij];
        }
        mdiag[g] = m;
        if (mdiag32) mdiag32[g] = (float)m;
    }
}

// *out = min of v[0..n): one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_min_reduce(const double *v, int n, double *out)
{
    __shared__ double wm[32];
    double m = INFINITY;
    for (int q = threadIdx.x; q < n; q += blockDim.x) m = fmin(m, v[q]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (int)(blockDim.x >> 5) ? wm[threadIdx.x] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *out = m;
    }
}

// ---------------------------------------------------------------- surface CSR

__device__ __forceinline__ bool on_surface(int i, int j, int k, int N)
{
    return i == 0 || i == N || j == 0 || j == N || k == 0 || k == N;
}

// Same order as the element kernels: k = 0 face, k = N face, then the ring
// of 4N nodes of each slab k = 1..N-1.
__device__ __forceinline__ int surf_index(int i, int j, int k, int N)
{
    const int n = N + 1, n2 = n * n;
    if (k == 0) return j * n + i;
    if (k == N) return n2 + j * n + i;
    const int r = j == 0 ? i : (j == N ? n + i : 2 * n + 2 * (j - 1) + (i == N ? 1 : 0));
    return 2 * n2 + (k - 1) * 4 * N + r;
}

__global__ void k_surf_count(const int32_t *l2g, int64_t n_local, int N, int32_t *cnt)
{
    const int n = N + 1;
    const int64_t n3 = (int64_t)n * n * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_local;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = l2g[q];
        if (g < 0) continue;
        const int node = (int)(q % n3);
        const int i = node % n, j = (node / n) % n, k = node / (n * n);
        if (on_surface(i, j, k, N)) atomicAdd(&cnt[g], 1);
    }
}

__global__ void k_flag(const int32_t *cnt, int64_t ng, int32_t *flag)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
        flag[g] = cnt[g] > 0 ? 1 : 0;
}

__global__ void k_compact_rows(const int32_t *cnt, const int32_t *srow_of, int64_t ng, int32_t *srow_g,
                               int32_t *scnt)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x)
        if (cnt[g] > 0) {
            srow_g[srow_of[g]] = (int32_t)g;
            scnt[srow_of[g]] = cnt[g];
        }
}

__global__ void k_surf_fill(const int32_t *l2g, int64_t n_local, int N, const int32_t *srow_of,
                            const int32_t *srowptr, int32_t *cursor, int32_t *scols)
{
    const int n = N + 1;
    const int64_t n3 = (int64_t)n * n * n;
    const int NS = 2 * n * n + 4 * N * (N - 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_local;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = l2g[q];
        if (g < 0) continue;
        const int64_t e = q / n3;
        const int node = (int)(q - e * n3);
        const int i = node % n, j = (node / n) % n, k = node / (n * n);
        if (!on_surface(i, j, k, N)) continue;
        const int r = srow_of[g];
        const int slot = atomicAdd(&cursor[r], 1);
        scols[srowptr[r] + slot] = (int32_t)(e * NS + surf_index(i, j, k, N));
    }
}

__global__ void k_sort_surf_rows(const int32_t *rowptr, int32_t *cols, int64_t nrows)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        const int a = rowptr[r], z = rowptr[r + 1];
        for (int p = a + 1; p < z; p++) {
            const int32_t v = cols[p];
            int q = p - 1;
            while (q >= a && cols[q] > v) { cols[q + 1] = cols[q]; q--; }
            cols[q + 1] = v;
        }
    }
}

// Exclusive scan of n int32 values (out may equal in); returns the total.
static hb_status scan_exclusive(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s, int64_t *total)
{
    const int64_t nchunks = (n + 1023) / 1024;
    int64_t *sums = nullptr;
    HB_TRY_CUDA(hb_dev_alloc((void **)&sums, sizeof(int64_t) * (nchunks + 1), s));
    hb_count_launch();
    k_scan_chunks<<<(unsigned)nchunks, 1024, 0, s>>>(in, n, out, sums);
    hb_count_launch();
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nchunks);
    hb_count_launch();
    k_scan_add<<<grid_for(n, 256), 256, 0, s>>>(out, n, sums);
    cudaError_t e = cudaGetLastError();
    int64_t tot = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, sums + nchunks, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    hb_dev_free(sums, s);
    if (e != cudaSuccess) {
        hb_set_error("scan: %s", cudaGetErrorString(e));
        return HB_ERR_CUDA;
    }
    *total = tot;
    return HB_OK;
}

// Builds srow_g, srowptr, scols of the mesh (after l2g exists).
static hb_status build_surface_csr(hb_mesh *m, cudaStream_t s)
{
    const int64_t ng = m->n_global, nl = m->n_local;
    int32_t *cnt = nullptr, *srow_of = nullptr, *scnt = nullptr;
    hb_status st = HB_OK;
    int64_t nsr = 0, nnz = 0;
    auto fail = [&](cudaError_t e) {
        hb_set_error("surface CSR: %s", cudaGetErrorString(e));
        st = e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
    };
    cudaError_t e = hb_dev_alloc((void **)&cnt, sizeof(int32_t) * (ng + 1), s);
    if (e == cudaSuccess) e = hb_dev_alloc((void **)&srow_of, sizeof(int32_t) * (ng + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (ng + 1), s);
    if (e != cudaSuccess) { fail(e); goto done; }
    hb_count_launch();
    k_surf_count<<<grid_for(nl, 256), 256, 0, s>>>(m->l2g, nl, m->N, cnt);
    hb_count_launch();
    k_flag<<<grid_for(ng + 1, 256), 256, 0, s>>>(cnt, ng + 1, srow_of);
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e); goto done; }
    if ((st = scan_exclusive(srow_of, srow_of, ng + 1, s, &nsr)) != HB_OK) goto done;
    m->nsr = nsr;
    e = hb_dev_alloc((void **)&m->srow_g, sizeof(int32_t) * (nsr + 1), s);
    if (e == cudaSuccess) e = hb_dev_alloc((void **)&m->srowptr, sizeof(int32_t) * (nsr + 1), s);
    if (e == cudaSuccess) e = hb_dev_alloc((void **)&scnt, sizeof(int32_t) * (nsr + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(scnt, 0, sizeof(int32_t) * (nsr + 1), s);
    if (e != cudaSuccess) { fail(e); goto done; }
    hb_count_launch();
    k_compact_rows<<<grid_for(ng, 256), 256, 0, s>>>(cnt, srow_of, ng, m->srow_g, scnt);
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e); goto done; }
    if ((st = scan_exclusive(scnt, m->srowptr, nsr + 1, s, &nnz)) != HB_OK) goto done;
    m->nnz_s = nnz;
    e = hb_dev_alloc((void **)&m->scols, sizeof(int32_t) * (nnz > 0 ? nnz : 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(scnt, 0, sizeof(int32_t) * (nsr + 1), s);
    if (e != cudaSuccess) { fail(e); goto done; }
    hb_count_launch();
    k_surf_fill<<<grid_for(nl, 256), 256, 0, s>>>(m->l2g, nl, m->N, srow_of, m->srowptr, scnt, m->scols);
    hb_count_launch();
    k_sort_surf_rows<<<grid_for(nsr, 256), 256, 0, s>>>(m->srowptr, m->scols, nsr);
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e); goto done; }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e); goto done; }
    m->device_bytes += sizeof(int32_t) * (2 * (nsr + 1) + nnz);
done:
    hb_dev_free(cnt, s);
    hb_dev_free(srow_of, s);
    hb_dev_free(scnt, s);
    return st;
}

__global__ void k_spos(const int32_t *__restrict__ scols, int64_t nnz, int32_t *__restrict__ spos)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
        spos[scols[q]] = (int32_t)q;
}

// CSR position of every surface copy (the inverse of scols), -1 for masked
// surface nodes; built the first time a variant that writes it is chosen.
hb_status hb_mesh_ensure_spos(hb_mesh *m, cudaStream_t s)
{
    if (m->spos) return HB_OK;
    const int64_t total = m->E * (int64_t)hb_surf_count(m->N);
    int32_t *p = nullptr;
    HB_TRY_CUDA(cudaMalloc((void **)&p, sizeof(int32_t) * (total > 0 ? total : 1)));
    cudaError_t e = cudaMemsetAsync(p, 0xFF, sizeof(int32_t) * (total > 0 ? total : 1), s);
    if (e == cudaSuccess && m->nnz_s > 0) {
        hb_count_launch();
        k_spos<<<grid_for(m->nnz_s, 256), 256, 0, s>>>(m->scols, m->nnz_s, p);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(p);
        hb_set_error("surface positions: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
    }
    hb_mesh_drop_graphs(m);  // captured runs hold the array pointer of the time
    m->spos = p;
    m->device_bytes += sizeof(int32_t) * (size_t)total;
    return HB_OK;
}

void hb_mesh_drop_graphs(hb_mesh *m)
{
    for (auto &g : m->graphs)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
}

// ---------------------------------------------------------------- mesh lifetime


// Frees everything the mesh holds. The arrays allocated while it was built
// are stream-ordered (freed on s); the ones grown later by the solvers and the
// autotuner (cg_vec, spos, inv_diag) are plain allocations.
static void mesh_free(hb_mesh *m, cudaStream_t s)
{
    hb_dev_free(m->l2g, s);
    hb_dev_free(m->geo, s);
    hb_dev_free(m->geo32, s);
    hb_dev_free(m->rowptr, s);
    hb_dev_free(m->cols, s);
    hb_dev_free(m->mdiag, s);
    hb_dev_free(m->mdiag32, s);
    hb_dev_free(m->yL, s);
    hb_dev_free(m->partials, s);
    hb_dev_free(m->counters, s);
    hb_dev_free(m->state, s);
    hb_dev_free(m->srow_g, s);
    hb_dev_free(m->srowptr, s);
    hb_dev_free(m->scols, s);
    hb_dev_free(m->ax_partials, s);
    // (a plain cudaFree may wait for the device: only for arrays that exist)
    if (m->cg_vec) cudaFree(m->cg_vec);
    if (m->spos) cudaFree(m->spos);
    if (m->inv_diag) cudaFree(m->inv_diag);
    if (m->inv_diag32) cudaFree(m->inv_diag32);
    for (auto &g : m->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (m->cg_stream) cudaStreamDestroy(m->cg_stream);
    if (m->cg_ev[0]) cudaEventDestroy(m->cg_ev[0]);
    if (m->cg_ev[1]) cudaEventDestroy(m->cg_ev[1]);
    hb_pinned_put(m->state_host);
    if (m->ev0) cudaEventDestroy(m->ev0);
    if (m->ev1) cudaEventDestroy(m->ev1);
    delete m;
}

extern "C" hb_status hb_mesh_destroy(hb_mesh *m)
{
    if (!m) return HB_OK;
    hb_device_guard dg(m->device);
    // work on any stream may still read the arrays: wait for the device, as a
    // plain cudaFree would
    cudaDeviceSynchronize();
    mesh_free(m, nullptr);
    return HB_OK;
}

void hb_mesh_release(hb_mesh *m, cudaStream_t s)
{
    if (!m) return;
    hb_device_guard dg(m->device);
    mesh_free(m, s);
}

#define HB_TRY_MESH(call)                                                        \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            hb_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,              \
                         cudaGetErrorString(e_));                                \
            hb_mesh_destroy(m);                                                  \
            hb_dev_free(tmp_cnt, s);                                             \
            hb_dev_free(tmp_sum, s);                                             \
            hb_dev_free(tmp_det, s);                                             \
            return e_ == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA; \
        }                                                                        \
    } while (0)

extern "C" hb_status hb_mesh_create(const hb_mesh_desc *d, void *stream, hb_mesh **out)
{
    hb_clear_error();
    if (!d || !out) { hb_set_error("null argument"); return HB_ERR_ARG; }
    *out = nullptr;
    if (d->N < 1 || d->N > HB_MAX_N) { hb_set_error("N=%d outside 1..%d", d->N, HB_MAX_N); return HB_ERR_ARG; }
    if (d->ex < 1 || d->ey < 1 || d->ez < 1) { hb_set_error("element counts must be >= 1"); return HB_ERR_ARG; }
    if (!(d->perturb >= 0.0 && d->perturb < 0.5)) { hb_set_error("perturb must be in [0, 0.5)"); return HB_ERR_ARG; }
    if (d->dirichlet_faces > 0x3Fu) { hb_set_error("dirichlet_faces has bits above 0x3F"); return HB_ERR_ARG; }
    const int N = d->N, n = N + 1;
    const int64_t E = (int64_t)d->ex * d->ey * d->ez;
    const int64_t n_local = E * n * n * n;
    if (n_local > 2147483647LL) { hb_set_error("n_local=%lld exceeds 2^31-1", (long long)n_local); return HB_ERR_ARG; }
    hb_status st = hb_ensure_device_tables();
    if (st != HB_OK) return st;

    cudaStream_t s = (cudaStream_t)stream;
    hb_mesh *m = new hb_mesh();
    memset((void *)m, 0, sizeof(hb_mesh));
    int32_t *tmp_cnt = nullptr;
    int64_t *tmp_sum = nullptr;
    double *tmp_det = nullptr;
    HB_TRY_MESH(cudaGetDevice(&m->device));
    m->desc = *d;
    m->variant[0] = HB_VAR_PENCIL | HB_VAR_EO;
    m->variant[1] = HB_VAR_PENCIL | HB_VAR_EO;
    m->variant[2] = HB_VAR_PENCIL | HB_VAR_EO;
    m->N = N;
    m->n = n;
    m->E = E;
    m->n_local = n_local;
    // global count by closed form, checked against the CSR below
    const int64_t NX = (int64_t)N * d->ex + 1, NY = (int64_t)N * d->ey + 1, NZ = (int64_t)N * d->ez + 1;
    const unsigned f = d->dirichlet_faces;
    const int64_t NXu = NX - (f & 1u ? 1 : 0) - (f & 2u ? 1 : 0);
    const int64_t NYu = NY - (f & 4u ? 1 : 0) - (f & 8u ? 1 : 0);
    const int64_t NZu = NZ - (f & 16u ? 1 : 0) - (f & 32u ? 1 : 0);
    m->n_global = (NXu > 0 && NYu > 0 && NZu > 0) ? NXu * NYu * NZu : 0;
    const int64_t ng = m->n_global;

    size_t bytes = 0;
    auto alloc = [&](void **p, size_t b) {
        bytes += b;
        return hb_dev_alloc(p, b, s);
    };
    HB_TRY_MESH(alloc((void **)&m->l2g, sizeof(int32_t) * n_local));
    HB_TRY_MESH(alloc((void **)&m->geo, sizeof(double) * 7 * n_local));
    if (d->keep_fp32_copy) HB_TRY_MESH(alloc((void **)&m->geo32, sizeof(float) * 7 * n_local));
    HB_TRY_MESH(alloc((void **)&m->rowptr, sizeof(int32_t) * (ng + 1)));
    HB_TRY_MESH(alloc((void **)&m->mdiag, sizeof(double) * (ng + 1)));
    if (d->keep_fp32_copy) HB_TRY_MESH(alloc((void **)&m->mdiag32, sizeof(float) * (ng + 1)));
    HB_TRY_MESH(alloc((void **)&m->yL, sizeof(double) * n_local));
    HB_TRY_MESH(alloc((void **)&m->partials, sizeof(double) * HB_RED_MAXV * HB_RED_BLOCKS));
    HB_TRY_MESH(alloc((void **)&m->counters, sizeof(unsigned) * 8));
    HB_TRY_MESH(alloc((void **)&m->state, sizeof(hb_cg_state) * 4));
    HB_TRY_MESH(hb_pinned_get((void **)&m->state_host, sizeof(hb_cg_state)));
    HB_TRY_MESH(cudaEventCreate(&m->ev0));
    HB_TRY_MESH(cudaEventCreate(&m->ev1));
    HB_TRY_MESH(cudaMemsetAsync(m->counters, 0, sizeof(unsigned) * 8, s));
    HB_TRY_MESH(cudaMemsetAsync(m->state, 0, sizeof(hb_cg_state) * 4, s));

    box_t b{d->ex, d->ey, d->ez, N, d->dirichlet_faces};
    hb_count_launch();
    k_l2g<<<grid_for(n_local, 256), 256, 0, s>>>(b, n_local, m->l2g);
    HB_TRY_MESH(cudaGetLastError());

    // geometry: one element per block
    // at least 64 threads: 36 of them form the edge differences
    int gthreads = n * n * n < 256 ? std::max(64, ((n * n * n + 31) / 32) * 32) : 256;
    int gblocks = (int)(E < 152 * 64 ? E : 152 * 64);
    // 18.4 KB at N = 15: under the default limit, so no per-call attribute
    // (a per-degree value would race between threads building meshes)
    size_t gsmem = sizeof(double) * 9 * n * n;
    HB_TRY_MESH(hb_dev_alloc((void **)&tmp_det, sizeof(double) * (gblocks + 1), s));
    hb_count_launch();
    k_geometry<<<gblocks, gthreads, gsmem, s>>>(b, d->perturb, d->seed, E, m->geo, m->geo32, tmp_det);
    HB_TRY_MESH(cudaGetLastError());
    hb_count_launch();
    k_min_reduce<<<1, 1024, 0, s>>>(tmp_det, gblocks, tmp_det + gblocks);
    HB_TRY_MESH(cudaGetLastError());

    // CSR of Z^T: count, scan, fill, sort rows
    HB_TRY_MESH(hb_dev_alloc((void **)&tmp_cnt, sizeof(int32_t) * (ng + 1), s));
    HB_TRY_MESH(cudaMemsetAsync(tmp_cnt, 0, sizeof(int32_t) * (ng + 1), s));
    hb_count_launch();
    k_count<<<grid_for(n_local, 256), 256, 0, s>>>(m->l2g, n_local, tmp_cnt);
    HB_TRY_MESH(cudaGetLastError());
    const int64_t nchunks = (ng + 1 + 1023) / 1024;
    HB_TRY_MESH(hb_dev_alloc((void **)&tmp_sum, sizeof(int64_t) * (nchunks + 1), s));
    hb_count_launch();
    k_scan_chunks<<<(unsigned)nchunks, 1024, 0, s>>>(tmp_cnt, ng + 1, m->rowptr, tmp_sum);
    HB_TRY_MESH(cudaGetLastError());
    hb_count_launch();
    k_scan_sums<<<1, 1024, 0, s>>>(tmp_sum, nchunks);
    HB_TRY_MESH(cudaGetLastError());
    hb_count_launch();
    k_scan_add<<<grid_for(ng + 1, 256), 256, 0, s>>>(m->rowptr, ng + 1, tmp_sum);
    HB_TRY_MESH(cudaGetLastError());
    int32_t nnz32 = 0;
    HB_TRY_MESH(cudaMemcpyAsync(&nnz32, m->rowptr + ng, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    double detmin = 0.0;
    HB_TRY_MESH(cudaMemcpyAsync(&detmin, tmp_det + gblocks, sizeof(double), cudaMemcpyDeviceToHost, s));
    HB_TRY_MESH(cudaStreamSynchronize(s));
    m->nnz = nnz32;
    m->min_detJ = detmin;
    HB_TRY_MESH(alloc((void **)&m->cols, sizeof(int32_t) * (m->nnz > 0 ? m->nnz : 1)));
    HB_TRY_MESH(cudaMemsetAsync(tmp_cnt, 0, sizeof(int32_t) * (ng + 1), s));
    hb_count_launch();
    k_fill<<<grid_for(n_local, 256), 256, 0, s>>>(m->l2g, n_local, m->rowptr, tmp_cnt, m->cols);
    HB_TRY_MESH(cudaGetLastError());
    hb_count_launch();
    k_sort_rows<<<grid_for(ng, 256), 256, 0, s>>>(m->rowptr, m->cols, ng, m->geo, n, m->mdiag, m->mdiag32);
    HB_TRY_MESH(cudaGetLastError());
    HB_TRY_MESH(cudaStreamSynchronize(s));
    hb_dev_free(tmp_cnt, s);
    hb_dev_free(tmp_sum, s);
    hb_dev_free(tmp_det, s);
    tmp_cnt = nullptr;
    tmp_sum = nullptr;
    tmp_det = nullptr;
    m->device_bytes = bytes;
    {
        hb_status sst = build_surface_csr(m, s);
        if (sst != HB_OK) { hb_mesh_destroy(m); return sst; }
        // one partial per element-kernel block (at most one block per element)
        // one partial per element-kernel block: at most one block per element
        m->n_ax_partials = E + 1;
        cudaError_t ae = hb_dev_alloc((void **)&m->ax_partials, sizeof(double) * m->n_ax_partials, s);
        if (ae != cudaSuccess) {
            hb_set_error("ax partials: %s", cudaGetErrorString(ae));
            hb_mesh_destroy(m);
            return ae == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
        }
        m->device_bytes += sizeof(double) * m->n_ax_partials;
    }
    if (!(m->min_detJ > 0.0)) {
        hb_set_error("non-positive Jacobian determinant (min det J = %g)", m->min_detJ);
        hb_mesh_destroy(m);
        return HB_ERR_GEOMETRY;
    }
    // every stream-ordered array is ready for any stream once s has drained
    {
        const cudaError_t se = cudaStreamSynchronize(s);
        if (se != cudaSuccess) {
            hb_set_error("mesh set-up: %s", cudaGetErrorString(se));
            hb_mesh_destroy(m);
            return HB_ERR_CUDA;
        }
    }
    *out = m;
    return HB_OK;
}

extern "C" hb_status hb_mesh_info(const hb_mesh *m, hb_mesh_info_t *o)
{
    if (!m || !o) { hb_set_error("null argument"); return HB_ERR_ARG; }
    o->n_local = m->n_local;
    o->n_global = m->n_global;
    o->n_elem = m->E;
    o->nnz = m->nnz;
    o->N = m->N;
    o->l2g = m->l2g;
    o->geo = m->geo;
    o->geo32 = m->geo32;
    o->csr_rowptr = m->rowptr;
    o->csr_cols = m->cols;
    o->min_detJ = m->min_detJ;
    o->device_bytes = m->device_bytes;
    return HB_OK;
}

extern "C" hb_status hb_mesh_copy_l2g(const hb_mesh *m, int32_t *host)
{
    if (!m || !host) { hb_set_error("null argument"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    HB_TRY_CUDA(cudaMemcpy(host, m->l2g, sizeof(int32_t) * m->n_local, cudaMemcpyDeviceToHost));
    return HB_OK;
}

extern "C" hb_status hb_mesh_copy_geo(const hb_mesh *m, double *host)
{
    if (!m || !host) { hb_set_error("null argument"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    HB_TRY_CUDA(cudaMemcpy(host, m->geo, sizeof(double) * 7 * m->n_local, cudaMemcpyDeviceToHost));
    return HB_OK;
}

// ---------------------------------------------------------------- Jacobi preconditioner

// Diagonal of the element matrix Dbold^T G^e Dbold at every local node:
//   sum_m D[m][i]^2 G_rr(m,j,k) + sum_m D[m][j]^2 G_ss(i,m,k) + sum_m D[m][k]^2 G_tt(i,j,m)
//   + 2 D_ii D_jj G_rs + 2 D_ii D_kk G_rt + 2 D_jj D_kk G_st.
__global__ void k_elem_diag(const double *__restrict__ geo, const double *__restrict__ D, int N, int64_t n_local,
                            double *__restrict__ out)
{
    const int n = N + 1, n2 = n * n;
    const int64_t n3 = (int64_t)n2 * n;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_local;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / n3;
        const int node = (int)(q - e * n3);
        const int i = node % n, j = (node / n) % n, k = node / n2;
        auto G = [&](int c, int ii, int jj, int kk) { return geo[((e * n + kk) * 7 + c) * (int64_t)n2 + jj * n + ii]; };
        double a = 0.0;
        for (int p = 0; p < n; p++) {
            a += D[p * n + i] * D[p * n + i] * G(0, p, j, k);
            a += D[p * n + j] * D[p * n + j] * G(3, i, p, k);
            a += D[p * n + k] * D[p * n + k] * G(5, i, j, p);
        }
        a += 2.0 * D[i * n + i] * D[j * n + j] * G(1, i, j, k);
        a += 2.0 * D[i * n + i] * D[k * n + k] * G(2, i, j, k);
        a += 2.0 * D[j * n + j] * D[k * n + k] * G(4, i, j, k);
        out[q] = a;
    }
}

// diag(A)_g = sum of the copies (CSR order = element order) + screening; stores 1/diag.
__global__ void k_diag_assemble(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ cols,
                                const double *__restrict__ dl, const double *__restrict__ mdiag, int screen,
                                double lambda, int64_t ng, double *__restrict__ inv64, float *__restrict__ inv32)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng; g += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int p = rowptr[g]; p < rowptr[g + 1]; p++) s += dl[cols[p]];
        s += screen ? lambda * mdiag[g] : lambda;
        const double inv = 1.0 / s;
        inv64[g] = inv;
        inv32[g] = (float)inv;
    }
}

hb_status hb_mesh_inv_diag(hb_mesh *m, int screen, double lambda, cudaStream_t s)
{
    if (m->diag_valid && m->diag_screen == screen && m->diag_lambda == lambda) return HB_OK;
    const int64_t ng = m->n_global;
    if (!m->inv_diag) {
        HB_TRY_CUDA(cudaMalloc((void **)&m->inv_diag, sizeof(double) * (ng + 1)));
        HB_TRY_CUDA(cudaMalloc((void **)&m->inv_diag32, sizeof(float) * (ng + 1)));
        m->device_bytes += 12 * (size_t)(ng + 1);
    }
    hb_count_launch();
    k_elem_diag<<<grid_for(m->n_local, 256), 256, 0, s>>>(m->geo, hb_dev_D64(m->N), m->N, m->n_local,
                                                         (double *)m->yL);
    HB_CHECK_LAUNCH();
    hb_count_launch();
    k_diag_assemble<<<grid_for(ng, 256), 256, 0, s>>>(m->rowptr, m->cols, (const double *)m->yL, m->mdiag, screen,
                                                     lambda, ng, m->inv_diag, m->inv_diag32);
    HB_CHECK_LAUNCH();
    m->diag_valid = 1;
    m->diag_screen = screen;
    m->diag_lambda = lambda;
    return HB_OK;
}

extern "C" hb_status hb_diag_A(hb_mesh *m, hb_screen screen, double lambda, double *host_diag, void *stream)
{
    hb_clear_error();
    if (!m || (!host_diag && m->n_global)) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (screen != HB_SCREEN_IDENTITY && screen != HB_SCREEN_MASS) { hb_set_error("bad screen"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (m->n_global == 0) return HB_OK;
    hb_status st = hb_mesh_inv_diag(m, screen, lambda, s);
    if (st != HB_OK) return st;
    std::vector<double> inv((size_t)m->n_global);
    HB_TRY_CUDA(cudaMemcpyAsync(inv.data(), m->inv_diag, sizeof(double) * m->n_global, cudaMemcpyDeviceToHost, s));
    HB_TRY_CUDA(cudaStreamSynchronize(s));
    for (int64_t g = 0; g < m->n_global; g++) host_diag[g] = 1.0 / inv[(size_t)g];
    return HB_OK;
}

// ---------------------------------------------------------------- right-hand sides

__global__ void k_rhs_uniform(const int32_t *l2g, box_t b, int64_t n_local, uint64_t seed, double *out)
{
    const int n = b.N + 1;
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t NX = (int64_t)b.N * b.Ex + 1, NY = (int64_t)b.N * b.Ey + 1;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n_local;
         q += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = l2g[q];
        if (g < 0) continue;
        int64_t e = q / n3;
        int node = (int)(q - e * n3);
        int i = node % n, j = (node / n) % n, k = node / (n * n);
        int64_t ex = e % b.Ex, ey = (e / b.Ex) % b.Ey, ez = e / ((int64_t)b.Ex * b.Ey);
        int64_t lat = (b.N * ex + i) + NX * ((b.N * ey + j) + NY * (b.N * ez + k));
        out[g] = 2.0 * hb_u01_impl(seed, 2, (uint64_t)lat) - 1.0;  // same value from every copy
    }
}

// Manufactured load: one thread per global DOF sums Jw f over its copies
// (CSR order), with the physical position recomputed from the element map.
__global__ void k_rhs_manufactured(const int32_t *rowptr, const int32_t *cols, int64_t ng, box_t b,
                                   double rho, uint64_t seed, const double *geo, double lambda, double *out)
{
    const int N = b.N, n = N + 1, n2 = n * n;
    const int64_t n3 = (int64_t)n2 * n;
    const double *xi = g_xi64 + N * 16;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < ng;
         g += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int p = rowptr[g]; p < rowptr[g + 1]; p++) {
            int64_t lq = cols[p];
            int64_t e = lq / n3;
            int node = (int)(lq - e * n3);
            int i = node % n, j = (node / n) % n, k = node / n2;
            int ex = (int)(e % b.Ex), ey = (int)((e / b.Ex) % b.Ey), ez = (int)(e / ((int64_t)b.Ex * b.Ey));
            double r = xi[i], s = xi[j], t = xi[k];
            double fr[2] = {0.5 * (1 - r), 0.5 * (1 + r)};
            double fs[2] = {0.5 * (1 - s), 0.5 * (1 + s)};
            double ft[2] = {0.5 * (1 - t), 0.5 * (1 + t)};
            double X[3] = {0, 0, 0};
            for (int c = 0; c < 2; c++)
                for (int bb = 0; bb < 2; bb++)
                    for (int a = 0; a < 2; a++) {
                        double V[3];
                        vertex_pos(b, rho, seed, ex + a, ey + bb, ez + c, V);
                        double wgt = fr[a] * fs[bb] * ft[c];
                        for (int ax = 0; ax < 3; ax++) X[ax] += V[ax] * wgt;
                    }
            double f = (3.0 * M_PI * M_PI + lambda) * sin(M_PI * X[0]) * sin(M_PI * X[1]) * sin(M_PI * X[2]);
            acc += geo[((e * n + k) * 7 + 6) * (int64_t)n2 + j * n + i] * f;
        }
        out[g] = acc;
    }
}

extern "C" hb_status hb_fill_rhs(const hb_mesh *m, int kind, uint64_t seed, double lambda, double *bvec,
                                 void *stream)
{
    hb_clear_error();
    if (!m || !bvec) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (kind != 0 && kind != 1) { hb_set_error("kind must be 0 or 1"); return HB_ERR_ARG; }
    hb_device_guard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    box_t b{m->desc.ex, m->desc.ey, m->desc.ez, m->N, m->desc.dirichlet_faces};
    if (m->n_global == 0) return HB_OK;
    if (kind == 0) {
        hb_count_launch();
        k_rhs_uniform<<<grid_for(m->n_local, 256), 256, 0, s>>>(m->l2g, b, m->n_local, seed, bvec);
    } else {
        hb_count_launch();
        k_rhs_manufactured<<<grid_for(m->n_global, 128), 128, 0, s>>>(
            m->rowptr, m->cols, m->n_global, b, m->desc.perturb, m->desc.seed, m->geo, lambda, bvec);
    }
    HB_CHECK_LAUNCH();
    return HB_OK;
}
