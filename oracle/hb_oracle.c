/*
 * hb_oracle.c -- plain, slow FP64 CPU oracle for the hipBone hot path.
 *
 * TEST INFRASTRUCTURE. This is the independent reference the CUDA library is
 * checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may build, load or call it; the product path never does.
 * It shares no code, header, table or constant generator with the CUDA
 * library: GLL points, the derivative matrix, the mesh, the numbering, the
 * geometric factors and the random numbers are all computed here on their own.
 *
 * What it computes (hipBone, arXiv 2202.12477):
 *   - Sec. 2, Eq. (poisson):   A = S + lambda I
 *   - Sec. 2, Eq. (stiffness): S = Z^T S_L Z, S_L^e = Dbold^T G^e Dbold with
 *     Dbold = [D(x)I(x)I; I(x)D(x)I; I(x)I(x)D] and G^e the symmetric 3x3 block
 *     of diagonal metric factors combined with GLL weights.
 *   - Algorithm 1: unpreconditioned conjugate gradients.
 * Textbook pieces the paper cites (Canuto et al.; Deville, Fischer & Mund):
 *   - GLL nodes: +-1 and the roots of P_N'; weights 2 / (N(N+1) P_N(xi)^2).
 *   - D_ij = l_j'(xi_i) in the closed Legendre form.
 *   - G_ab = w_i w_j w_k detJ sum_c (J^-1)_ac (J^-1)_bc for the trilinear map.
 * Readings where the paper is silent (all listed with the design notes):
 *   - the box is [0,1]^3 split into Ex x Ey x Ez hexahedra; vertices strictly
 *     inside the box move by U[-rho h, rho h] per axis; maps are trilinear;
 *   - Dirichlet nodes are left out of the global numbering; global ids are
 *     lexicographic over the remaining lattice nodes, I fastest;
 *   - the lambda W term: W Z x summed by Z^T gives lambda x once per DOF
 *     (identity screening); mass screening adds lambda Z^T (Jw . Z x);
 *   - CG starts from the caller's x, stops when ||r|| <= rtol ||b|| or after
 *     max_it iterations (rtol = 0 runs exactly max_it iterations).
 * Random numbers: u01(seed, stream, idx) = (splitmix64(seed ^ (stream * G)
 * + idx) >> 11) * 2^-53 with G = 0x9E3779B97F4A7C15 and the published
 * SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
 *
 * Built with -ffp-contract=off: no fused multiply-adds are formed, every
 * product and sum rounds on its own, in the order written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Random numbers                                                      */
/* ------------------------------------------------------------------ */

/* SplitMix64 output for the state value s (the generator adds the golden
 * gamma to its state and then mixes; this is that step for one state). */
static uint64_t splitmix64_at(uint64_t s)
{
    uint64_t z = s + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t s) { return splitmix64_at(s); }

double or_u01(uint64_t seed, uint64_t stream, uint64_t idx)
{
    uint64_t s = (seed ^ (stream * 0x9E3779B97F4A7C15ULL)) + idx;
    return (double)(splitmix64_at(s) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------ */
/* GLL nodes, weights and the 1-D derivative matrix                    */
/* ------------------------------------------------------------------ */

/* Legendre P_N(x) and P_N'(x) by the three-term recurrence
 * k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}, and P_k' = P_{k-2}' + (2k-1) P_{k-1}. */
static void legendre(int N, double x, double *P, double *dP)
{
    double p_km2 = 1.0, p_km1 = x;      /* P_0, P_1 */
    double d_km2 = 0.0, d_km1 = 1.0;    /* P_0', P_1' */
    if (N == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int k = 2; k <= N; k++) {
        double p_k = ((2.0 * k - 1.0) * x * p_km1 - (k - 1.0) * p_km2) / k;
        double d_k = d_km2 + (2.0 * k - 1.0) * p_km1;
        p_km2 = p_km1; p_km1 = p_k;
        d_km2 = d_km1; d_km1 = d_k;
    }
    *P = p_km1;
    *dP = d_km1;
}

/* GLL nodes xi[0..N] (ascending) and weights w[0..N]. Interior nodes are the
 * roots of P_N', found by Newton's method from the Chebyshev-Gauss-Lobatto
 * points; P_N'' comes from Legendre's equation
 * (1-x^2) P'' = 2x P' - N(N+1) P. Returns 0 on success. */
int or_gll(int N, double *xi, double *w)
{
    if (N < 1) return 1;
    const double pi = 3.14159265358979323846;
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int i = 1; i < N; i++) {
        double x = -cos(pi * i / N);
        for (int it = 0; it < 100; it++) {
            double P, dP;
            legendre(N, x, &P, &dP);
            double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
            double dx = dP / d2P;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        xi[i] = x;
    }
    /* The node set is symmetric about 0; make the computed set exactly so. */
    for (int i = 0; i < (N + 1) / 2; i++) {
        double a = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -a;
        xi[N - i] = a;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int i = 0; i <= N; i++) {
        double P, dP;
        legendre(N, xi[i], &P, &dP);
        w[i] = 2.0 / (N * (N + 1.0) * P * P);
    }
    return 0;
}

/* D[i*(N+1)+j] = l_j'(xi_i) for the Lagrange basis on the GLL nodes:
 * off-diagonal P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j)); D_00 = -N(N+1)/4,
 * D_NN = N(N+1)/4, other diagonal entries 0. */
int or_deriv(int N, const double *xi, double *D)
{
    int n = N + 1;
    double *P = (double *)malloc(sizeof(double) * n);
    if (!P) return 1;
    for (int i = 0; i < n; i++) {
        double dP;
        legendre(N, xi[i], &P[i], &dP);
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double v;
            if (i != j) v = P[i] / (P[j] * (xi[i] - xi[j]));
            else if (i == 0) v = -N * (N + 1.0) / 4.0;
            else if (i == N) v = N * (N + 1.0) / 4.0;
            else v = 0.0;
            D[i * n + j] = v;
        }
    free(P);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Mesh                                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    int Ex, Ey, Ez, N, n;
    int64_t E, n_local, n_global;
    unsigned faces;
    double rho;
    uint64_t seed;
    double *xi, *w, *D;      /* GLL nodes, weights, derivative matrix */
    double *V;               /* vertices [(Ez+1)(Ey+1)(Ex+1)][3] */
    int32_t *l2g;            /* [E][n^3], -1 for a Dirichlet node */
    double *G;               /* [E][n^3][6]: rr rs rt ss st tt */
    double *Jw;              /* [E][n^3] */
    double *X;               /* physical coordinates of local nodes [E][n^3][3] */
    double min_detJ;
    double *yL;              /* work: one element's local output [E][n^3] */
} or_mesh;

static int64_t vidx(const or_mesh *m, int a, int b, int c)
{
    return ((int64_t)c * (m->Ey + 1) + b) * (m->Ex + 1) + a;
}

/* Box vertices: lattice points (a/Ex, b/Ey, c/Ez); each vertex strictly inside
 * the box moves by (2u-1) rho h_axis along each axis. */
static void make_vertices(or_mesh *m)
{
    double h[3] = {1.0 / m->Ex, 1.0 / m->Ey, 1.0 / m->Ez};
    for (int c = 0; c <= m->Ez; c++)
        for (int b = 0; b <= m->Ey; b++)
            for (int a = 0; a <= m->Ex; a++) {
                int64_t v = vidx(m, a, b, c);
                double X[3] = {(double)a / m->Ex, (double)b / m->Ey, (double)c / m->Ez};
                int inside = a > 0 && a < m->Ex && b > 0 && b < m->Ey && c > 0 && c < m->Ez;
                for (int ax = 0; ax < 3; ax++) {
                    double off = 0.0;
                    if (inside) {
                        double u = or_u01(m->seed, 1, (uint64_t)(3 * v + ax));
                        off = (2.0 * u - 1.0) * m->rho * h[ax];
                    }
                    m->V[3 * v + ax] = X[ax] + off;
                }
            }
}

/* Global numbering: lexicographic over the lattice nodes (I,J,K), I fastest,
 * skipping the nodes on masked faces. Face bits: 0 x=0, 1 x=1, 2 y=0, 3 y=1,
 * 4 z=0, 5 z=1. */
static int make_numbering(or_mesh *m)
{
    int N = m->N, n = m->n;
    int64_t NX = (int64_t)N * m->Ex + 1, NY = (int64_t)N * m->Ey + 1, NZ = (int64_t)N * m->Ez + 1;
    int64_t *id = (int64_t *)malloc(sizeof(int64_t) * NX * NY * NZ);
    if (!id) return 1;
    int64_t next = 0;
    for (int64_t K = 0; K < NZ; K++)
        for (int64_t J = 0; J < NY; J++)
            for (int64_t I = 0; I < NX; I++) {
                int masked = ((m->faces & 1u) && I == 0) || ((m->faces & 2u) && I == NX - 1) ||
                             ((m->faces & 4u) && J == 0) || ((m->faces & 8u) && J == NY - 1) ||
                             ((m->faces & 16u) && K == 0) || ((m->faces & 32u) && K == NZ - 1);
                id[I + NX * (J + NY * K)] = masked ? -1 : next++;
            }
    m->n_global = next;
    for (int ez = 0; ez < m->Ez; ez++)
        for (int ey = 0; ey < m->Ey; ey++)
            for (int ex = 0; ex < m->Ex; ex++) {
                int64_t e = ex + (int64_t)m->Ex * (ey + (int64_t)m->Ey * ez);
                for (int k = 0; k < n; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) {
                            int64_t I = (int64_t)N * ex + i, J = (int64_t)N * ey + j, K = (int64_t)N * ez + k;
                            m->l2g[e * n * n * n + (k * n + j) * n + i] = (int32_t)id[I + NX * (J + NY * K)];
                        }
            }
    free(id);
    return 0;
}

/* The 8 vertices of element (ex,ey,ez), with the same perturbation rule as
 * make_vertices, computed directly. */
static void element_vertices(int Ex, int Ey, int Ez, double rho, uint64_t seed, int ex, int ey, int ez,
                             double Ve[2][2][2][3])
{
    double h[3] = {1.0 / Ex, 1.0 / Ey, 1.0 / Ez};
    for (int c = 0; c < 2; c++)
        for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) {
                int A = ex + a, B = ey + b, Cc = ez + c;
                int64_t v = ((int64_t)Cc * (Ey + 1) + B) * (Ex + 1) + A;
                double X[3] = {(double)A / Ex, (double)B / Ey, (double)Cc / Ez};
                int inside = A > 0 && A < Ex && B > 0 && B < Ey && Cc > 0 && Cc < Ez;
                for (int ax = 0; ax < 3; ax++) {
                    double off = 0.0;
                    if (inside) off = (2.0 * or_u01(seed, 1, (uint64_t)(3 * v + ax)) - 1.0) * rho * h[ax];
                    Ve[c][b][a][ax] = X[ax] + off;
                }
            }
}

/* Geometric factors of one element from the analytic Jacobian of the
 * trilinear map x(r,s,t) = sum_{abc} V_abc phi_a(r) phi_b(s) phi_c(t),
 * phi_0 = (1-r)/2, phi_1 = (1+r)/2, at each GLL node. G: [n^3][6], Jw: [n^3],
 * X: [n^3][3] (may be NULL). Returns the smallest det J. */
static double element_geometry(int N, const double *xi, const double *w, double Ve[2][2][2][3], double *G,
                               double *Jw, double *Xout)
{
    int n = N + 1;
    double mind = INFINITY;
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double r = xi[i], s = xi[j], t = xi[k];
                double ph[3][2] = {{0.5 * (1 - r), 0.5 * (1 + r)},
                                   {0.5 * (1 - s), 0.5 * (1 + s)},
                                   {0.5 * (1 - t), 0.5 * (1 + t)}};
                double dph[2] = {-0.5, 0.5};
                double J[3][3] = {{0}}, X[3] = {0};
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++)
                            for (int ax = 0; ax < 3; ax++) {
                                double v = Ve[c][b][a][ax];
                                X[ax] += v * ph[0][a] * ph[1][b] * ph[2][c];
                                J[ax][0] += v * dph[a] * ph[1][b] * ph[2][c];
                                J[ax][1] += v * ph[0][a] * dph[b] * ph[2][c];
                                J[ax][2] += v * ph[0][a] * ph[1][b] * dph[c];
                            }
                double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                             J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                double Ji[3][3];
                Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
                Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
                Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
                Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
                Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
                Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
                Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
                Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
                Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
                double wq = w[i] * w[j] * w[k] * det;
                int q = (k * n + j) * n + i;
                const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
                for (int f = 0; f < 6; f++) {
                    double g = 0.0;
                    for (int x = 0; x < 3; x++) g += Ji[pa[f]][x] * Ji[pb[f]][x];
                    G[6 * q + f] = wq * g;
                }
                Jw[q] = wq;
                if (Xout)
                    for (int ax = 0; ax < 3; ax++) Xout[3 * q + ax] = X[ax];
                if (det < mind) mind = det;
            }
    return mind;
}

/* Geometric factors of every element (element_geometry on the box's vertices). */
static void make_geometry(or_mesh *m)
{
    int n = m->n;
    int64_t n3 = (int64_t)n * n * n;
    double mind = INFINITY;
    for (int ez = 0; ez < m->Ez; ez++)
        for (int ey = 0; ey < m->Ey; ey++)
            for (int ex = 0; ex < m->Ex; ex++) {
                int64_t e = ex + (int64_t)m->Ex * (ey + (int64_t)m->Ey * ez);
                double Ve[2][2][2][3];
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++)
                            for (int ax = 0; ax < 3; ax++)
                                Ve[c][b][a][ax] = m->V[3 * vidx(m, ex + a, ey + b, ez + c) + ax];
                double d = element_geometry(m->N, m->xi, m->w, Ve, m->G + 6 * e * n3, m->Jw + e * n3,
                                            m->X + 3 * e * n3);
                if (d < mind) mind = d;
            }
    m->min_detJ = mind;
}

void or_mesh_free(or_mesh *m)
{
    if (!m) return;
    free(m->xi); free(m->w); free(m->D); free(m->V); free(m->l2g);
    free(m->G); free(m->Jw); free(m->X); free(m->yL);
    free(m);
}

or_mesh *or_mesh_create(int Ex, int Ey, int Ez, int N, double rho, uint64_t seed, unsigned faces)
{
    if (Ex < 1 || Ey < 1 || Ez < 1 || N < 1) return NULL;
    or_mesh *m = (or_mesh *)calloc(1, sizeof(or_mesh));
    if (!m) return NULL;
    m->Ex = Ex; m->Ey = Ey; m->Ez = Ez; m->N = N; m->n = N + 1;
    m->E = (int64_t)Ex * Ey * Ez;
    m->n_local = m->E * m->n * m->n * m->n;
    m->faces = faces; m->rho = rho; m->seed = seed;
    int n = m->n;
    int64_t nv = (int64_t)(Ex + 1) * (Ey + 1) * (Ez + 1);
    m->xi = (double *)malloc(sizeof(double) * n);
    m->w = (double *)malloc(sizeof(double) * n);
    m->D = (double *)malloc(sizeof(double) * n * n);
    m->V = (double *)malloc(sizeof(double) * 3 * nv);
    m->l2g = (int32_t *)malloc(sizeof(int32_t) * m->n_local);
    m->G = (double *)malloc(sizeof(double) * 6 * m->n_local);
    m->Jw = (double *)malloc(sizeof(double) * m->n_local);
    m->X = (double *)malloc(sizeof(double) * 3 * m->n_local);
    m->yL = (double *)malloc(sizeof(double) * m->n_local);
    if (!m->xi || !m->w || !m->D || !m->V || !m->l2g || !m->G || !m->Jw || !m->X || !m->yL) {
        or_mesh_free(m);
        return NULL;
    }
    or_gll(N, m->xi, m->w);
    or_deriv(N, m->xi, m->D);
    make_vertices(m);
    if (make_numbering(m)) { or_mesh_free(m); return NULL; }
    make_geometry(m);
    return m;
}

/* Sizes: out[0] = E, out[1] = n_local, out[2] = n_global. */
void or_mesh_sizes(const or_mesh *m, int64_t *out)
{
    out[0] = m->E; out[1] = m->n_local; out[2] = m->n_global;
}
double or_mesh_min_detJ(const or_mesh *m) { return m->min_detJ; }
void or_mesh_copy_l2g(const or_mesh *m, int32_t *out) { memcpy(out, m->l2g, sizeof(int32_t) * m->n_local); }
void or_mesh_copy_geo(const or_mesh *m, double *G6, double *Jw)
{
    memcpy(G6, m->G, sizeof(double) * 6 * m->n_local);
    memcpy(Jw, m->Jw, sizeof(double) * m->n_local);
}
void or_mesh_copy_coords(const or_mesh *m, double *X) { memcpy(X, m->X, sizeof(double) * 3 * m->n_local); }
void or_mesh_copy_vertices(const or_mesh *m, double *V)
{
    memcpy(V, m->V, sizeof(double) * 3 * (m->Ex + 1) * (m->Ey + 1) * (m->Ez + 1));
}
void or_mesh_copy_ref(const or_mesh *m, double *xi, double *w, double *D)
{
    memcpy(xi, m->xi, sizeof(double) * m->n);
    memcpy(w, m->w, sizeof(double) * m->n);
    memcpy(D, m->D, sizeof(double) * m->n * m->n);
}

/* ------------------------------------------------------------------ */
/* The operator                                                        */
/* ------------------------------------------------------------------ */

/* y_e = S_L^e u_e = Dbold^T G^e Dbold u_e for one element, with u_e = Z_e x. */
static void local_stiffness_ptr(int n, const double *D, const int32_t *l2g, const double *G, const double *x,
                                double *ye, double *u, double *ur, double *us, double *ut)
{
    int64_t n3 = (int64_t)n * n * n;
#define IX(i, j, k) (((k) * n + (j)) * n + (i))
    /* u = Z_e x (a Dirichlet node carries 0) */
    for (int q = 0; q < n3; q++) u[q] = l2g[q] >= 0 ? x[l2g[q]] : 0.0;
    /* Dbold u: (D (x) I (x) I) u, (I (x) D (x) I) u, (I (x) I (x) D) u */
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double a = 0.0, b = 0.0, c = 0.0;
                for (int p = 0; p < n; p++) {
                    a += D[i * n + p] * u[IX(p, j, k)];
                    b += D[j * n + p] * u[IX(i, p, k)];
                    c += D[k * n + p] * u[IX(i, j, p)];
                }
                ur[IX(i, j, k)] = a;
                us[IX(i, j, k)] = b;
                ut[IX(i, j, k)] = c;
            }
    /* G^e applied pointwise to (ur, us, ut) */
    for (int q = 0; q < n3; q++) {
        const double *g = G + 6 * q;
        double a = ur[q], b = us[q], c = ut[q];
        ur[q] = g[0] * a + g[1] * b + g[2] * c;
        us[q] = g[1] * a + g[3] * b + g[4] * c;
        ut[q] = g[2] * a + g[4] * b + g[5] * c;
    }
    /* Dbold^T (vr, vs, vt) */
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                double a = 0.0, b = 0.0, c = 0.0;
                for (int p = 0; p < n; p++) {
                    a += D[p * n + i] * ur[IX(p, j, k)];
                    b += D[p * n + j] * us[IX(i, p, k)];
                    c += D[p * n + k] * ut[IX(i, j, p)];
                }
                ye[IX(i, j, k)] = a + b + c;
            }
#undef IX
}

static void local_stiffness(const or_mesh *m, int64_t e, const double *x, double *ye, double *u, double *ur,
                            double *us, double *ut)
{
    int64_t n3 = (int64_t)m->n * m->n * m->n;
    local_stiffness_ptr(m->n, m->D, m->l2g + e * n3, m->G + 6 * e * n3, x, ye, u, ur, us, ut);
}

/* y = A x = Z^T S_L Z x + lambda x (screen 0, Eq. poisson) or
 *         = Z^T S_L Z x + lambda Z^T (Jw . Z x) (screen 1, mass screening).
 * Local products of different elements are independent (computed in
 * parallel when built with OpenMP); Z^T then sums them serially in element
 * order, node order, so the result does not depend on the thread count. */
int or_apply_A(or_mesh *m, int screen, double lambda, const double *x, double *y)
{
    int n = m->n;
    int64_t n3 = (int64_t)n * n * n;
    int err = 0;
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        double *wk = (double *)malloc(sizeof(double) * 4 * n3);
        if (!wk) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t e = 0; e < m->E; e++)
            if (wk) local_stiffness(m, e, x, m->yL + e * n3, wk, wk + n3, wk + 2 * n3, wk + 3 * n3);
        free(wk);
    }
    if (err) return 1;
    for (int64_t g = 0; g < m->n_global; g++) y[g] = 0.0;
    for (int64_t q = 0; q < m->n_local; q++) {
        int32_t g = m->l2g[q];
        if (g >= 0) y[g] += m->yL[q];
    }
    if (screen == 0) {
        for (int64_t g = 0; g < m->n_global; g++) y[g] += lambda * x[g];
    } else {
        for (int64_t q = 0; q < m->n_local; q++) {
            int32_t g = m->l2g[q];
            if (g >= 0) y[g] += lambda * (m->Jw[q] * x[g]);
        }
    }
    return 0;
}

/* diag(A): for each DOF the sum over its copies of the element-matrix
 * diagonal (Dbold^T G^e Dbold)_qq, written out term by term:
 *   sum_m D[m][i]^2 G_rr(m,j,k) + sum_m D[m][j]^2 G_ss(i,m,k)
 *   + sum_m D[m][k]^2 G_tt(i,j,m)
 *   + 2 D[i][i] D[j][j] G_rs + 2 D[i][i] D[k][k] G_rt + 2 D[j][j] D[k][k] G_st,
 * summed in element order, then + lambda (identity screening) or
 * + lambda * sum Jw (mass screening). */
int or_diag_A(const or_mesh *m, int screen, double lambda, double *d)
{
    int n = m->n;
    int64_t n3 = (int64_t)n * n * n;
    const double *D = m->D;
    for (int64_t g = 0; g < m->n_global; g++) d[g] = 0.0;
    for (int64_t e = 0; e < m->E; e++) {
        const double *G = m->G + 6 * e * n3;
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int64_t q = e * n3 + (k * n + j) * n + i;
                    int32_t g = m->l2g[q];
                    if (g < 0) continue;
                    double a = 0.0;
                    for (int p = 0; p < n; p++) {
                        a += D[p * n + i] * D[p * n + i] * G[6 * ((k * n + j) * n + p) + 0];
                        a += D[p * n + j] * D[p * n + j] * G[6 * ((k * n + p) * n + i) + 3];
                        a += D[p * n + k] * D[p * n + k] * G[6 * ((p * n + j) * n + i) + 5];
                    }
                    const double *gq = G + 6 * ((k * n + j) * n + i);
                    a += 2.0 * D[i * n + i] * D[j * n + j] * gq[1];
                    a += 2.0 * D[i * n + i] * D[k * n + k] * gq[2];
                    a += 2.0 * D[j * n + j] * D[k * n + k] * gq[4];
                    d[g] += a;
                }
    }
    if (screen == 0) {
        for (int64_t g = 0; g < m->n_global; g++) d[g] += lambda;
    } else {
        for (int64_t q = 0; q < m->n_local; q++) {
            int32_t g = m->l2g[q];
            if (g >= 0) d[g] += lambda * m->Jw[q];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Right-hand sides                                                    */
/* ------------------------------------------------------------------ */

/* kind 0: b_g = 2 u01(seed, 2, lattice index) - 1 at every global DOF.
 * kind 1: b = Z^T (Jw . f), f = (3 pi^2 + lambda) sin(pi x) sin(pi y) sin(pi z),
 *         the load for u = sin sin sin under -Laplace u + lambda u = f. */
void or_rhs(const or_mesh *m, int kind, uint64_t seed, double lambda, double *b)
{
    int N = m->N, n = m->n;
    int64_t n3 = (int64_t)n * n * n;
    const double pi = 3.14159265358979323846;
    for (int64_t g = 0; g < m->n_global; g++) b[g] = 0.0;
    for (int ez = 0; ez < m->Ez; ez++)
        for (int ey = 0; ey < m->Ey; ey++)
            for (int ex = 0; ex < m->Ex; ex++) {
                int64_t e = ex + (int64_t)m->Ex * (ey + (int64_t)m->Ey * ez);
                for (int k = 0; k < n; k++)
                    for (int j = 0; j < n; j++)
                        for (int i = 0; i < n; i++) {
                            int64_t q = e * n3 + (k * n + j) * n + i;
                            int32_t g = m->l2g[q];
                            if (g < 0) continue;
                            if (kind == 0) {
                                int64_t I = (int64_t)N * ex + i, J = (int64_t)N * ey + j, K = (int64_t)N * ez + k;
                                int64_t lat = I + ((int64_t)N * m->Ex + 1) * (J + ((int64_t)N * m->Ey + 1) * K);
                                b[g] = 2.0 * or_u01(seed, 2, (uint64_t)lat) - 1.0;
                            } else {
                                const double *X = m->X + 3 * q;
                                double f = (3.0 * pi * pi + lambda) * sin(pi * X[0]) * sin(pi * X[1]) * sin(pi * X[2]);
                                b[g] += m->Jw[q] * f;
                            }
                        }
            }
}

/* ------------------------------------------------------------------ */
/* Conjugate gradients (Algorithm 1)                                   */
/* ------------------------------------------------------------------ */

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* Algorithm 1 on A = S + lambda I (or mass screening). x holds x0 on entry
 * and the solution on exit. Stops when r.r <= rtol^2 b.b (rtol > 0) or after
 * max_it iterations. hist (may be NULL) receives r_j.r_j for j = 0..iters.
 * Returns 0 (done), 2 on breakdown (p.Ap <= 0 or not finite), 1 on no memory. */
int or_pcg(or_mesh *m, int screen, double lambda, const double *b, double *x, double rtol, int max_it,
           int precond, int *iters, double *rel_res, double *hist)
{
    int64_t ng = m->n_global;
    double *r = (double *)malloc(sizeof(double) * ng);
    double *p = (double *)malloc(sizeof(double) * ng);
    double *Ap = (double *)malloc(sizeof(double) * ng);
    double *z = (double *)malloc(sizeof(double) * ng);
    double *dg = precond ? (double *)malloc(sizeof(double) * ng) : NULL;
    if (!r || !p || !Ap || !z || (precond && !dg)) { free(r); free(p); free(Ap); free(z); free(dg); return 1; }
    int status = 0;
    if (precond) or_diag_A(m, screen, lambda, dg);
    /* r_0 = b - A x, z_0 = M^-1 r_0 (M = diag(A), or I), p = z_0 */
    or_apply_A(m, screen, lambda, x, Ap);
    for (int64_t i = 0; i < ng; i++) r[i] = b[i] - Ap[i];
    for (int64_t i = 0; i < ng; i++) z[i] = precond ? r[i] / dg[i] : r[i];
    for (int64_t i = 0; i < ng; i++) p[i] = z[i];
    double bb = dot(ng, b, b);
    double rr = dot(ng, r, r);
    double rz = dot(ng, r, z);
    double tol2 = rtol * rtol * bb;
    if (hist) hist[0] = rr;
    int j = 0;
    while (j < max_it && rr > tol2) {
        or_apply_A(m, screen, lambda, p, Ap);
        double pAp = dot(ng, p, Ap);
        if (!(pAp > 0.0) || !isfinite(pAp)) { status = 2; break; }
        double alpha = rz / pAp;
        for (int64_t i = 0; i < ng; i++) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < ng; i++) r[i] = r[i] - alpha * Ap[i];
        for (int64_t i = 0; i < ng; i++) z[i] = precond ? r[i] / dg[i] : r[i];
        double rz_new = dot(ng, r, z);
        double beta = rz_new / rz;
        for (int64_t i = 0; i < ng; i++) p[i] = z[i] + beta * p[i];
        rz = rz_new;
        rr = dot(ng, r, r);
        j++;
        if (hist) hist[j] = rr;
    }
    *iters = j;
    *rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    free(r); free(p); free(Ap); free(z); free(dg);
    return status;
}

/* Algorithm 1 (no preconditioner). */
int or_cg(or_mesh *m, int screen, double lambda, const double *b, double *x,
          double rtol, int max_it, int *iters, double *rel_res, double *hist)
{
    return or_pcg(m, screen, lambda, b, x, rtol, max_it, 0, iters, rel_res, hist);
}

/* Number of threads the parallel element loop uses (1 without OpenMP). */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Selected rows of A x without building the mesh                      */
/* ------------------------------------------------------------------ */

/* out[r] = (A x)[rows[r]] for the box (Ex,Ey,Ez,N,rho,seed,faces), computed
 * element by element: for each requested DOF the elements that contain it
 * (ascending element order, as or_apply_A sums them) get their vertices,
 * geometric factors and local product S_L^e Z_e x built on the spot. The
 * global id of a lattice node is its rank among the unmasked lattice nodes
 * in lexicographic order (the numbering or_mesh_create enumerates).
 * Returns 0, or 1 on a bad row or allocation failure. */
int or_apply_A_rows(int Ex, int Ey, int Ez, int N, double rho, uint64_t seed, unsigned faces, int screen,
                    double lambda, const double *x, int64_t nrows, const int64_t *rows, double *out)
{
    int n = N + 1;
    int64_t n3 = (int64_t)n * n * n;
    int64_t NX = (int64_t)N * Ex + 1, NY = (int64_t)N * Ey + 1, NZ = (int64_t)N * Ez + 1;
    int x0 = faces & 1u ? 1 : 0, x1 = faces & 2u ? 1 : 0, y0 = faces & 4u ? 1 : 0, y1 = faces & 8u ? 1 : 0;
    int z0 = faces & 16u ? 1 : 0, z1 = faces & 32u ? 1 : 0;
    int64_t NXu = NX - x0 - x1, NYu = NY - y0 - y1, NZu = NZ - z0 - z1;
    double *xi = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n), *D = malloc(sizeof(double) * n * n);
    double *G = malloc(sizeof(double) * 6 * n3), *Jw = malloc(sizeof(double) * n3);
    double *wk = malloc(sizeof(double) * 5 * n3);
    int32_t *l2g = malloc(sizeof(int32_t) * n3);
    int err = 0;
    if (!xi || !w || !D || !G || !Jw || !wk || !l2g) err = 1;
    if (!err) {
        or_gll(N, xi, w);
        or_deriv(N, xi, D);
    }
    for (int64_t r = 0; r < nrows && !err; r++) {
        int64_t g = rows[r];
        if (g < 0 || g >= NXu * NYu * NZu) { err = 1; break; }
        int64_t I = g % NXu + x0, J = (g / NXu) % NYu + y0, K = g / (NXu * NYu) + z0;
        int exs[2], eys[2], ezs[2], nx = 0, ny = 0, nz = 0;
        /* elements containing lattice coordinate I along x, ascending */
        if (I % N == 0 && I / N - 1 >= 0) exs[nx++] = (int)(I / N - 1);
        if (I / N < Ex) exs[nx++] = (int)(I / N);
        if (J % N == 0 && J / N - 1 >= 0) eys[ny++] = (int)(J / N - 1);
        if (J / N < Ey) eys[ny++] = (int)(J / N);
        if (K % N == 0 && K / N - 1 >= 0) ezs[nz++] = (int)(K / N - 1);
        if (K / N < Ez) ezs[nz++] = (int)(K / N);
        double y = 0.0, mt[8];
        int nm = 0;
        for (int cz = 0; cz < nz; cz++)
            for (int cy = 0; cy < ny; cy++)
                for (int cx = 0; cx < nx; cx++) {
                    int ex = exs[cx], ey = eys[cy], ez = ezs[cz];
                    double Ve[2][2][2][3];
                    element_vertices(Ex, Ey, Ez, rho, seed, ex, ey, ez, Ve);
                    element_geometry(N, xi, w, Ve, G, Jw, NULL);
                    for (int k = 0; k < n; k++)
                        for (int j = 0; j < n; j++)
                            for (int i = 0; i < n; i++) {
                                int64_t Il = (int64_t)N * ex + i, Jl = (int64_t)N * ey + j, Kl = (int64_t)N * ez + k;
                                int masked = (x0 && Il == 0) || (x1 && Il == NX - 1) || (y0 && Jl == 0) ||
                                             (y1 && Jl == NY - 1) || (z0 && Kl == 0) || (z1 && Kl == NZ - 1);
                                l2g[(k * n + j) * n + i] =
                                    masked ? -1 : (int32_t)((Il - x0) + NXu * ((Jl - y0) + NYu * (Kl - z0)));
                            }
                    local_stiffness_ptr(n, D, l2g, G, x, wk, wk + n3, wk + 2 * n3, wk + 3 * n3, wk + 4 * n3);
                    int q = (int)(((K - (int64_t)N * ez) * n + (J - (int64_t)N * ey)) * n + (I - (int64_t)N * ex));
                    y += wk[q];
                    mt[nm++] = lambda * (Jw[q] * x[g]);
                }
        /* screening after all element sums, copy by copy, as or_apply_A adds it */
        if (screen == 0) y += lambda * x[g];
        else
            for (int c = 0; c < nm; c++) y += mt[c];
        out[r] = y;
    }
    free(xi); free(w); free(D); free(G); free(Jw); free(wk); free(l2g);
    return err;
}
