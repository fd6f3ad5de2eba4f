// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "hipbone_gb300.h"

#define HB_MAX_N 15
#define HB_RED_BLOCKS 1216  // fixed grid of every reduction kernel (8 x 152 SMs)
#define HB_RED_MAXV 4       // values one grid reduction may carry (rows of the partials buffer)
#define HB_RED_THREADS 256

// ---------------------------------------------------------------- errors

void hb_set_error(const char *fmt, ...);
void hb_clear_error();

#define HB_TRY_CUDA(call)                                                          \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            hb_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                \
                         cudaGetErrorString(e_));                                  \
            return e_ == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;   \
        }                                                                          \
    } while (0)

#define HB_CHECK_LAUNCH() HB_TRY_CUDA(cudaGetLastError())

// Counts one kernel launch; with timing enabled also records a CUDA event pair
// around it on its stream (see hb_profile_* in the C header).
void hb_count_launch();
void hb_count_launches(unsigned long long k);
bool hb_profiling_on();
struct hb_prof_scope {
    cudaStream_t stream;
    cudaEvent_t stop;
    hb_prof_scope(const char *name, cudaStream_t s);
    ~hb_prof_scope();
};

// ---------------------------------------------------------------- CG device state

// Scalars of Algorithm 1 kept on the device so that no iteration waits on the
// host. `run` says whether the current iteration does any work; kernels of a
// finished solve return at once, so a captured run of iterations may overshoot.
struct hb_cg_state {
    double rr;        // r_j . z_j (z = M^-1 r; r_j . r_j without a preconditioner): alpha's numerator
    double rr_new;    // r_{j+1} . z_{j+1}
    double res2;      // r_j . r_j, for the stopping test
    double pAp;       // p . A p
    double alpha, beta;
    double tol2;      // rtol^2 b.b
    double bb;        // b . b
    double dot_tmp;   // scratch result of a stand-alone dot
    int it;           // iterations done
    int max_it;
    int run;          // 1 while the solve is running
    int next_run;
    int status;       // hb_status
    int pad;
};

// ---------------------------------------------------------------- mesh

struct hb_mesh {
    int device;
    hb_mesh_desc desc;
    int N, n;
    int64_t E, n_local, n_global, nnz;
    int32_t *l2g;       // [E][n^3]
    double *geo;        // [E][n][7][n^2]
    float *geo32;       // same layout (optional)
    int32_t *rowptr;    // [n_global + 1]
    int32_t *cols;      // [nnz]
    double *mdiag;      // [n_global] assembled J w (lumped mass)
    float *mdiag32;
    void *yL;           // [n_local] doubles: element-local operator output
    // workspace for reductions and CG
    double *partials;   // [HB_RED_MAXV * HB_RED_BLOCKS]
    unsigned *counters; // [4]
    hb_cg_state *state; // device CG states [4]: 0 outer/FP64, 1 inner/dot
    hb_cg_state *state_host;  // pinned mirror
    void *cg_vec;       // r, p, Ap (FP64) then FP32 inner vectors
    size_t cg_vec_bytes;
    double min_detJ;
    size_t device_bytes;
    cudaEvent_t ev0, ev1;
    int variant[3];     // element-kernel variant per precision (HB_F64, HB_F32, HB_F64X)
    // Jacobi preconditioner: 1 / diag(A) for the (screen, lambda) it was built for
    double *inv_diag;
    float *inv_diag32;
    int diag_screen;
    double diag_lambda;
    int diag_valid;
    // Z^T restricted to DOFs with a copy on an element surface (the pencil
    // kernels finish element-interior DOFs themselves)
    int64_t nsr, nnz_s;
    int32_t *srow_g;    // [nsr] global id of each surface row (ascending)
    int32_t *srowptr;   // [nsr + 1]
    int32_t *scols;     // [nnz_s] e * surf_count + surface index, ascending
    int32_t *spos;      // [E * surface nodes] CSR position of each surface copy (-1 masked); built on demand
    double *ax_partials;  // [max element-kernel blocks] per-block partials of x.y
    int64_t n_ax_partials;
    int fused_mode;     // hb_cg_solve in one cooperative kernel: 0 small meshes, 1 never, 2 whenever it fits
    // stepwise solve (hb_cg_begin / hb_cg_iterate / hb_cg_finish)
    struct cg_step {
        int active;
        hb_cg_opts o;
        const double *b;
        double *x;
        int done;
    } step;
    // captured runs of CG iterations (replayed while the key matches)
    cudaStream_t cg_stream;
    cudaEvent_t cg_ev[2];
    struct cg_graph {
        cudaGraphExec_t exec;
        const void *x, *r, *p, *Ap, *z, *inv_d;
        const hb_cg_state *st;
        int prec, screen, count, variant;
        double lambda;
        unsigned long long launches;  // kernels per replay
    } graphs[2];  // [0] FP64 runs, [1] FP32 inner runs
};

// Reference element data computed on the host for every degree 1..15 (GLL
// nodes by Newton, derivative matrix by barycentric weights).
void hb_reference_element(int N, double *xi, double *w, double *D);

// Uploads the derivative matrices (FP64 and FP32, D and D^T) of all degrees to
// the current device once per device.
hb_status hb_ensure_device_tables();
const double *hb_dev_D64(int N);
const float *hb_dev_D32(int N);

// ---------------------------------------------------------------- launchers

// y_L = S_L Z x for every element (FP64 / FP32).
hb_status hb_launch_ax_local_f64(const hb_mesh *m, const double *x, double *yL, const int *run, cudaStream_t s);
hb_status hb_launch_ax_local_f32(const hb_mesh *m, const float *x, float *yL, const int *run, cudaStream_t s);
hb_status hb_launch_ax2_f64(const hb_mesh *m, const double *x, double *ysurf, double *y, double lambda, int screen,
                            double *partials, const int *run, int eo, int eb_mult, cudaStream_t s,
                            int64_t *nblocks);
hb_status hb_launch_ax2_f32(const hb_mesh *m, const float *x, float *ysurf, float *y, double lambda, int screen,
                            double *partials, const int *run, int eo, int eb_mult, cudaStream_t s,
                            int64_t *nblocks);
int hb_surf_count(int N);  // surface nodes of one element: 2 n^2 + 4 N (N-1)
int hb_surf_pos(int N, int i, int j, int k);  // node's place in the surface block; -1 inside
hb_status hb_launch_ax2_f64_scat(const hb_mesh *m, const double *xL, double *ysurf, double *yL, double lambda,
                                 int screen, const int *run, int eo, int eb_mult, cudaStream_t s);
hb_status hb_launch_ax2_f64_range(int N, int64_t E, const double *x, const double *halo, const int32_t *l2g,
                                  const double *geo, double *ysurf, double *y, double lambda, int screen,
                                  const int *run, int eo, int eb_mult, cudaStream_t s);
hb_status hb_launch_ax2_f64x(const hb_mesh *m, const double *x, double *ysurf, double *y, double lambda, int screen,
                             double *partials, const int *run, int eb_mode, cudaStream_t s, int64_t *nblocks);
hb_status hb_ax2_upload_f64x(const double *D_all);
// Tensor-core FP64 element kernel (N = 7; see HB_VAR_TC) and its tables.
hb_status hb_tc_upload();
hb_status hb_launch_ax_tc_f64(const hb_mesh *m, const double *x, double *ysurf, double *y, double lambda,
                              int screen, double *partials, const int *run, bool csr_store, cudaStream_t s,
                              int64_t *nblocks);
hb_status hb_ax2_upload_f64(const double *D_all);
hb_status hb_ax2_upload_f32(const double *D_all);

// Element-kernel variants (bit flags): v1 = 0; HB_VAR_PENCIL = pencil kernel;
// HB_VAR_EO = even-odd split (pencil only); HB_VAR_EB2 = two element groups per
// block; HB_VAR_ONE = one element per block (with PENCIL | EO only);
// HB_VAR_TMA = bulk L2 prefetch of each block's geometric factors at its
// start (with PENCIL | EO only); HB_VAR_WS = persistent warp-specialised
// kernel staging node map and factors through shared memory (with
// PENCIL | EO only; FP32 and odd N, else the PENCIL | EO kernel runs).
// HB_VAR_CSR = surface values written straight to their CSR positions, so the
// surface gather reads contiguous runs (with PENCIL | EO, alone or with ONE).
// HB_VAR_GRID = every local value stored element-major and Z^T taken by the
// box's lattice arithmetic, one warp per lattice row (with PENCIL | EO, alone
// or with ONE).
// HB_VAR_TC = the tensor-core element kernel (alone or with HB_VAR_CSR; FP64,
// N = 7): every derivative contraction exact on tcgen05 from FP16 digit
// slices, the metric step in FP64.
enum { HB_VAR_PENCIL = 1, HB_VAR_EO = 2, HB_VAR_EB2 = 4, HB_VAR_ONE = 8, HB_VAR_TMA = 16, HB_VAR_WS = 32,
       HB_VAR_CSR = 64, HB_VAR_GRID = 128, HB_VAR_MAX = 255, HB_VAR_TC = 256 };
static inline bool hb_valid_variant(int v)
{
    if (v == 0 || v == HB_VAR_TC || v == (HB_VAR_TC | HB_VAR_CSR)) return true;
    if (v < 0 || v > HB_VAR_MAX || !(v & HB_VAR_PENCIL)) return false;
    const int extra = v & (HB_VAR_ONE | HB_VAR_TMA | HB_VAR_WS | HB_VAR_EB2);
    if (v & HB_VAR_GRID) return !(v & HB_VAR_CSR) && (v & HB_VAR_EO) && (extra == 0 || extra == HB_VAR_ONE);
    if (v & HB_VAR_CSR) return (v & HB_VAR_EO) && (extra == 0 || extra == HB_VAR_ONE);
    if (extra & (HB_VAR_ONE | HB_VAR_TMA | HB_VAR_WS))
        return (v & HB_VAR_EO) && (extra == HB_VAR_ONE || extra == HB_VAR_TMA || extra == HB_VAR_WS);
    return true;
}
// The double-float unit instantiates the even-odd pencil kernel in its base
// and one-element shapes and their CSR-store and lattice-gather forms only.
static inline bool hb_valid_variant_f64x(int v)
{
    const int base = HB_VAR_PENCIL | HB_VAR_EO;
    return v == base || v == (base | HB_VAR_ONE) || v == (base | HB_VAR_CSR) || v == (base | HB_VAR_ONE | HB_VAR_CSR) ||
           v == (base | HB_VAR_GRID) || v == (base | HB_VAR_ONE | HB_VAR_GRID);
}
// Slot of hb_mesh::variant for a precision (-1: none).
static inline int hb_variant_slot(int prec)
{
    return prec == HB_F64 ? 0 : prec == HB_F32 ? 1 : prec == HB_F64X ? 2 : -1;
}
// eb_mode of the pencil launchers for a variant (bit 8: CSR-position surface
// store; bit 16: every local value stored element-major)
static inline int hb_variant_eb_mode(int v)
{
    const int b = (v & HB_VAR_ONE) ? 0 : (v & HB_VAR_TMA) ? 3 : (v & HB_VAR_WS) ? 4 : (v & HB_VAR_EB2) ? 2 : 1;
    return b | ((v & HB_VAR_CSR) ? 8 : 0) | ((v & HB_VAR_GRID) ? 16 : 0);
}
// Builds mesh->spos if it is missing (synchronises s).
hb_status hb_mesh_ensure_spos(hb_mesh *m, cudaStream_t s);
// Fused CG (one cooperative kernel for all iterations): element groups one
// launch can keep resident for degree N (0: not available), and the run.
int hb_cg_fused_capacity(int N);
hb_status hb_cg_fused_upload(const double *D_all);
hb_status hb_cg_fused_run(const hb_mesh *m, int screen, double lambda, double *x, double *r, double *p, double *Ap,
                          hb_cg_state *st, cudaStream_t s);
// Self-tests of the bounded device waits (hb_selftest_wait): the staged
// pipeline's mbarrier wait (sets bit 0 of *err) and the fused CG's grid
// barrier (bar: a zeroed word; sets bit 1).
hb_status hb_selftest_mbar_timeout(unsigned *err, cudaStream_t s);
hb_status hb_selftest_barrier_timeout(unsigned *bar, unsigned *err, cudaStream_t s);
// Destroys the mesh's captured CG runs (before an array they use is replaced).
void hb_mesh_drop_graphs(hb_mesh *m);
// Releases a mesh whose arrays no pending work outside stream s uses: the
// stream-ordered arrays are freed on s, without waiting for the device (the
// server's retirement). hb_mesh_destroy waits for the device first.
void hb_mesh_release(hb_mesh *m, cudaStream_t s);

// Stream-ordered device memory from the library's pool (hb_mem.cu): usable on
// s at once and on other streams after s is synchronised; hb_dev_free frees on
// s in stream order. hb_dev_trim returns the pool's cached memory.
cudaError_t hb_dev_alloc(void **p, size_t bytes, cudaStream_t s);
void hb_dev_free(void *p, cudaStream_t s);
void hb_dev_trim();
// Freed pool memory kept for reuse before the rest goes back to the device
// (8 GiB unless a server raises it to its budget while it runs).
cudaError_t hb_dev_keep(uint64_t bytes);
uint64_t hb_dev_keep_default();
// Pinned host buffers of at most 256 bytes, reused.
cudaError_t hb_pinned_get(void **p, size_t bytes);
void hb_pinned_put(void *p);


// y = Z^T y_L + lambda (x or M x); optional fused x.y into st->pAp (and the
// CG breakdown test / alpha when `cg` is set).
hb_status hb_launch_assemble_f64(const hb_mesh *m, const double *yL, const double *x, double *y,
                                 int screen, double lambda, hb_cg_state *st, int dot_mode,
                                 cudaStream_t s);
hb_status hb_launch_assemble_f32(const hb_mesh *m, const float *yL, const float *x, float *y,
                                 int screen, double lambda, hb_cg_state *st, int dot_mode,
                                 cudaStream_t s);

hb_status hb_apply_A_impl(const hb_mesh *m, hb_precision prec, int screen, double lambda,
                          const void *x, void *y, hb_cg_state *st, int dot_mode, cudaStream_t s);

// 1 / diag(A) in FP64 and FP32 for (screen, lambda), built on first use and
// kept while (screen, lambda) stay the same.
hb_status hb_mesh_inv_diag(hb_mesh *m, int screen, double lambda, cudaStream_t s);

// a.b in FP64 into *out (device).
hb_status hb_launch_dot_f64(const hb_mesh *m, const double *a, const double *b, int64_t n,
                            double *out, cudaStream_t s);
hb_status hb_launch_dot_f32(const hb_mesh *m, const float *a, const float *b, int64_t n,
                            double *out, cudaStream_t s);

// dot_mode of the assembly kernel
enum { HB_DOT_NONE = 0, HB_DOT_TO_TMP = 1, HB_DOT_CG_PAP = 2 };

struct hb_device_guard {
    int prev;
    bool ok;
    explicit hb_device_guard(int dev) : prev(-1), ok(true)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~hb_device_guard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
