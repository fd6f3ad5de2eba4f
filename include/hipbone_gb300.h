/*
 * hipbone_gb300.h -- C ABI of the GB300 (sm_103a) matrix-free spectral-element
 * screened-Poisson operator and its conjugate-gradient solvers.
 *
 * The problem is the one hipBone (Chalmers, Mishra, McDougall & Warburton,
 * arXiv 2202.12477) benchmarks:
 *   - Sec. 2: a box of E hexahedral elements, polynomial degree N,
 *     (N+1)^3 Gauss-Lobatto-Legendre (GLL) nodes per element, N_L = E (N+1)^3
 *     element-local nodes and N_G assembled (global) degrees of freedom;
 *   - Eq. (poisson):   A = S + lambda I;
 *   - Eq. (stiffness): S = Z^T S_L Z with S_L^e = Dbold^T G^e Dbold;
 *   - Sec. 3.1 (DOF storage): every vector lives in assembled form, length N_G;
 *   - Algorithm 1: unpreconditioned conjugate gradients.
 *
 * Conventions for every call:
 *   - Vectors are caller-owned DEVICE buffers of length n_global (hb_mesh_info),
 *     contiguous, of the element type the precision argument names
 *     (double for HB_F64, float for HB_F32). The library never frees them.
 *   - Mesh arrays (node map, geometric factors, CSR of Z^T, workspace) are
 *     library-owned device memory, released by hb_mesh_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Calls enqueue work on it and return without waiting, except
 *     where a call says it synchronises.
 *   - A mesh carries one workspace: calls on one mesh must not overlap in
 *     time on different streams (issue them on one stream, or synchronise).
 *   - Errors come back as hb_status; hb_last_error() gives a message for the
 *     calling thread. Nothing throws across the ABI.
 *   - The device is the current CUDA device at hb_mesh_create; later calls on
 *     the mesh switch to it for their duration.
 */
#ifndef HIPBONE_GB300_H
#define HIPBONE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HB_OK = 0,
    HB_ERR_ARG = 1,            /* invalid argument (null pointer, size, mode) */
    HB_ERR_NOMEM = 2,          /* device or host allocation failed */
    HB_ERR_CUDA = 3,           /* a CUDA runtime call failed (see hb_last_error) */
    HB_ERR_GEOMETRY = 4,       /* a Jacobian determinant <= 0 at some GLL node */
    HB_ERR_BREAKDOWN = 5,      /* CG: p.Ap <= 0 or not finite (A not SPD) */
    HB_ERR_NOT_CONVERGED = 6,  /* CG: max_it reached above the requested rtol */
    HB_ERR_TIMEOUT = 7,        /* a bounded device wait ran out */
    HB_ERR_BUSY = 8,           /* resource in use (server full, slot held) */
    HB_ERR_NOT_FOUND = 9       /* unknown ticket or name */
} hb_status;

typedef enum {
    HB_F64 = 0,    /* IEEE FP64 storage and arithmetic */
    HB_F32 = 1,    /* FP32 storage and arithmetic, FP64 dot accumulation */
    HB_MIXED = 2,  /* CG only: FP32 inner CG inside an FP64 defect-correction loop */
    HB_F64X = 3    /* FP64 storage (x, y, geometric factors); the element kernel
                      computes in double-float (pairs of FP32 with error-free
                      transformations, ~47-bit significand) on the FP32 pipes,
                      gather and vector stage in FP64. Agrees with HB_F64 to
                      ~1e-14 relative; not IEEE FP64 arithmetic. */
} hb_precision;

typedef enum {
    HB_SCREEN_IDENTITY = 0,  /* A = S + lambda I, Eq. (poisson) */
    HB_SCREEN_MASS = 1       /* A = S + lambda M, M = Z^T diag(J w) Z (lumped GLL mass) */
} hb_screen;

/* Mesh description (Sec. 2: "regular mesh of E hexahedral elements" with a
 * degree-N tensor GLL basis). The box is [0,1]^3 split into ex*ey*ez equal
 * hexahedra; every vertex strictly inside the box is moved along each axis by
 * (2u-1)*perturb*h_axis with u = u01(seed, 1, 3*vertex_index+axis) (see
 * hb_u01); elements map trilinearly from their 8 vertices. */
typedef struct {
    int ex, ey, ez;            /* elements per axis, each >= 1 */
    int N;                     /* polynomial degree, 1..15 */
    double perturb;            /* rho, 0 <= rho < 0.5 */
    uint64_t seed;             /* seed of the vertex perturbation */
    unsigned dirichlet_faces;  /* bit f masks face f: 0 x=0, 1 x=1, 2 y=0, 3 y=1,
                                  4 z=0, 5 z=1; 0x3F = all faces (the paper's case) */
    int keep_fp32_copy;        /* 1: also keep FP32 geometric factors (HB_F32 and
                                  HB_MIXED need them) */
} hb_mesh_desc;

/* Read-only view of a mesh. Device pointers stay valid until hb_mesh_destroy.
 * Layouts (element e = ex + Ex*(ey + Ey*ez); local node (i,j,k), i fastest):
 *   l2g[e*(N+1)^3 + (k*(N+1)+j)*(N+1)+i]  global id of the node, -1 on a
 *       Dirichlet face (this is the mask: masked <=> l2g < 0). Global ids are
 *       lexicographic over the unmasked lattice nodes (N*ex+i, N*ey+j, N*ez+k),
 *       first coordinate fastest.
 *   geo[((e*(N+1)+k)*7 + c)*(N+1)^2 + j*(N+1)+i]  FP64 factor c of node (i,j,k):
 *       c = 0..5 the metric entries G_rr G_rs G_rt G_ss G_st G_tt (GLL weights
 *       and det J included, Sec. 2), c = 6 the quadrature weight w_i w_j w_k det J.
 *   geo32: the same in FP32 (NULL unless keep_fp32_copy).
 *   csr_rowptr[n_global+1], csr_cols[nnz]: Z^T as CSR; row g lists the local
 *       node ids that carry global id g, ascending. */
typedef struct {
    int64_t n_local;           /* N_L = E (N+1)^3 */
    int64_t n_global;          /* N_G */
    int64_t n_elem;            /* E */
    int64_t nnz;               /* unmasked local nodes = entries of Z */
    int N;
    const int32_t *l2g;
    const double *geo;
    const float *geo32;
    const int32_t *csr_rowptr;
    const int32_t *csr_cols;
    double min_detJ;           /* smallest det J over all GLL nodes */
    size_t device_bytes;       /* device memory the mesh holds */
} hb_mesh_info_t;

typedef struct hb_mesh hb_mesh;

/* Builds the mesh on the current device: GLL nodes, derivative matrix, node
 * map, CSR of Z^T and the geometric factors (Sec. 2, Sec. 3.2). The arrays are
 * allocated in stream order on `stream` from a memory pool the library owns
 * (no call here waits for other streams or the device); `stream` is
 * synchronised before the call returns, so the mesh is ready for work on any
 * stream. Returns HB_ERR_GEOMETRY (and no mesh) if det J <= 0
 * at any GLL node; HB_ERR_ARG for N outside 1..15, non-positive element counts,
 * perturb outside [0, 0.5) or more than 2^31-1 local nodes. */
hb_status hb_mesh_create(const hb_mesh_desc *desc, void *stream, hb_mesh **out);
/* Waits for the device (work on any stream may still read the mesh), then
 * frees the mesh. The pool keeps up to 8 GiB of freed memory for later meshes
 * and returns the rest to the device. */
hb_status hb_mesh_destroy(hb_mesh *mesh);
hb_status hb_mesh_info(const hb_mesh *mesh, hb_mesh_info_t *out);

/* Copies of mesh data to HOST buffers, for inspection and tests (synchronous).
 * l2g: n_local int32; geo: 7*n_local doubles in the geo layout above. */
hb_status hb_mesh_copy_l2g(const hb_mesh *mesh, int32_t *host_l2g);
hb_status hb_mesh_copy_geo(const hb_mesh *mesh, double *host_geo);

/* y = A x on assembled vectors (Eq. poisson with Eq. stiffness; Sec. 3.2):
 * gathers x through Z, applies S_L element by element (tensor-product
 * derivatives with the geometric factors), sums back with Z^T in a fixed order
 * (no atomics: results are bitwise reproducible), and adds lambda x
 * (identity screening) or lambda M x (mass screening).
 * prec HB_F64 or HB_F64X: x, y are double*; HB_F32: float* (needs
 * keep_fp32_copy). x and y must not overlap. */
hb_status hb_apply_A(const hb_mesh *mesh, hb_precision prec, hb_screen screen,
                     double lambda, const void *x, void *y, void *stream);

/* a.b over n_global entries: the inner products of Algorithm 1 (r.r, p.Ap,
 * the stopping test's norm), which Sec. 3.5 fuses into the vector kernels of
 * a CG iteration; this call is the same reduction standing alone. Accumulated
 * in FP64 (warp shuffles, then a fixed block order: bitwise reproducible).
 * prec names the element type of a and b (HB_F64: double, HB_F32: float; other
 * precisions return HB_ERR_ARG).
 * Writes the result to *out_dev (device double, may be NULL) and, if out_host
 * is not NULL, also to *out_host -- which synchronises `stream`. */
hb_status hb_dot(const hb_mesh *mesh, hb_precision prec, const void *a, const void *b,
                 double *out_dev, double *out_host, void *stream);

/* a.b like hb_dot, for callers that must not allocate device memory: it
 * needs no mesh and calls no cudaMalloc, cudaFree or allocating routine. The
 * paper has no counterpart; this exists for applications whose allocator
 * owns the whole device (a caching allocator, a serving loop with a fixed
 * memory budget) or whose latency-critical loop cannot take the device-wide
 * synchronisation an allocation may cause.
 * Scratch: a static device array inside the library (16384 block partials,
 * 128 KB), held on every GPU that loads the library until the process exits.
 * Maximum length: n <= 16384 * 1024 = 16,777,216 elements; longer vectors are
 * rejected with HB_ERR_ARG and a message. Up to 1,245,184 elements the result
 * is bitwise the same as hb_dot's; beyond, the blocks differ, so it agrees to
 * rounding (about 1e-16 of sum |a_i b_i|).
 * a, b: device vectors of n doubles (HB_F64) or floats (HB_F32). The result
 * goes to *out_dev (device double) or, if out_dev is NULL, to a slot inside
 * the static array; if out_host is not NULL it is also copied there, which
 * synchronises `stream`.
 * The first call on a device takes the array's device address (once per
 * device, with that device current) and keeps it for the life of the process;
 * make that first call before any stream capture, and do not use the entry
 * point after a cudaDeviceReset (or any teardown of the device's primary
 * context) in the same process: the kept address belongs to the old context.
 * Every call shares the one array: calls that overlap in time on the
 * GPU (different streams, or different host threads) race and give wrong
 * results; serialise them. */
hb_status hb_dot_noalloc(hb_precision prec, const void *a, const void *b, int64_t n,
                         double *out_dev, double *out_host, void *stream);

/* Right-hand side on the assembled DOFs (FP64, length n_global).
 * kind 0: b_g = 2 u01(seed, 2, I + (N ex+1)(J + (N ey+1) K)) - 1 at the global
 *         node with lattice coordinates (I,J,K) -- hipBone's pseudo-random
 *         forcing (Sec. 3), uniform in [-1, 1).
 * kind 1: b = Z^T (Jw . f), f = (3 pi^2 + lambda) sin(pi x) sin(pi y) sin(pi z):
 *         the load whose exact solution is u = sin sin sin for
 *         -Laplace u + lambda u = f (exact under mass screening; lambda = 0 for
 *         identity screening). */
hb_status hb_fill_rhs(const hb_mesh *mesh, int kind, uint64_t seed, double lambda,
                      double *b, void *stream);

typedef struct {
    hb_precision prec;     /* HB_F64, HB_F32 or HB_MIXED */
    hb_screen screen;
    double lambda;
    double rtol;           /* stop when ||r||_2 <= rtol ||b||_2; 0 runs exactly max_it */
    int max_it;            /* iteration cap (inner iterations in HB_MIXED) */
    double inner_rtol;     /* HB_MIXED: inner FP32 CG reduces its residual by this */
    int max_outer;         /* HB_MIXED: cap on FP64 defect-correction steps */
    int precond;           /* 0: none (Algorithm 1, the paper's hipBone); 1: Jacobi,
                              M = diag(A) (NekBone's diagonal preconditioner, Sec. 3) */
} hb_cg_opts;

typedef struct {
    int iters;             /* CG iterations (all inner iterations in HB_MIXED) */
    int outer_iters;       /* HB_MIXED: defect-correction steps; else 0 */
    double rel_res;        /* ||b - A x||_2 / ||b||_2 at exit, recomputed in FP64 with the
                              FP64 operator when rtol > 0 (every solver form); with
                              rtol = 0 (a fixed iteration count, no stopping test)
                              the recursive residual of Algorithm 1 */
    double time_ms;        /* device time of the solve (CUDA events) */
    hb_status status;
} hb_cg_result;

/* diag(A) for the given screening (the Jacobi preconditioner's M): the sum over
 * each DOF's copies of the element-matrix diagonal of Dbold^T G^e Dbold, plus
 * lambda (identity) or lambda M_gg (mass). Written to a HOST buffer of
 * n_global doubles; synchronises `stream`. */
hb_status hb_diag_A(hb_mesh *mesh, hb_screen screen, double lambda, double *host_diag, void *stream);

/* Solves A x = b with Algorithm 1 (x holds x0 on entry, the solution on exit;
 * both FP64 device vectors of length n_global). HB_F64 runs Algorithm 1 in FP64;
 * HB_F64X the same with the double-float element kernel.
 * HB_MIXED runs FP64 defect correction: r = b - A x in FP64, an FP32 CG on
 * A d = r to inner_rtol (FP64 dot accumulation), x += d in FP64, until
 * ||b - A x|| <= rtol ||b||. precond = 1 applies the Jacobi preconditioner
 * diag(A) (z = M^-1 r, alpha = r.z / p.Ap, beta from successive r.z, p = z + beta p;
 * in HB_MIXED to the inner FP32 CG); the stopping test stays on ||r||. The p.Ap
 * and r.r reductions are fused into the kernels that produce their operands
 * (Sec. 3.5). Synchronises `stream`.
 * Stopping test (Algorithm 1's test on the residual, taken relative: ||r|| <=
 * rtol ||b||): the recursive residual r_{j+1} = r_j - alpha A p_j drifts from
 * b - A x_{j+1} by rounding, so when it meets the tolerance the solver
 * recomputes the true residual b - A x in FP64 (FP64 operator); if that one is
 * still above rtol ||b||, Algorithm 1 restarts from x with it (p = M^-1 r) and
 * the iterations go on, while each restart lowers the true residual by at
 * least a tenth (else the rounding floor of the operator is above rtol and the
 * solve ends, HB_ERR_NOT_CONVERGED). HB_OK therefore means the true FP64
 * residual meets rtol; HB_MIXED tests the true residual at every outer step.
 * Returns HB_ERR_BREAKDOWN, HB_ERR_NOT_CONVERGED (rtol > 0 only: max_it
 * iterations ran and the true residual is above rtol) or HB_OK;
 * res (may be NULL) receives the counts, residual and device time. */
hb_status hb_cg_solve(const hb_mesh *mesh, const hb_cg_opts *opts, const double *b,
                      double *x, hb_cg_result *res, void *stream);

/* How hb_cg_solve runs HB_F64 without a preconditioner: mode 0 (default) runs
 * every iteration inside one cooperative kernel (the phases of an iteration
 * separated by grid-wide barriers instead of launches, one block per element
 * with its three line directions contracted at once) when the mesh has at
 * most 300 elements and one block per element fits on the GPU at once;
 * mode 1 never does; mode 2 does whenever they fit. The fused run computes the same
 * Algorithm 1 with its own fixed-order reductions (results agree with the
 * launched kernels to rounding, not bitwise). */
hb_status hb_set_cg_fused(hb_mesh *mesh, int mode);

/* Stepwise form of hb_cg_solve for HB_F64 / HB_F64X (with or without the
 * Jacobi preconditioner), for callers that time or interleave iterations:
 * hb_cg_begin computes r0 = b - A x0 and the solver state (enqueued on
 * `stream`, no host wait); hb_cg_iterate enqueues up to `count` more
 * iterations (never past opts->max_it; kernels of a solve that has met rtol
 * return at once) without waiting for the host; hb_cg_finish waits and fills
 * res (time_ms = 0): with rtol > 0 it recomputes the true residual b - A x in
 * FP64 (one more operator application) and returns HB_ERR_NOT_CONVERGED if it
 * is above rtol (the stepwise form does not restart: its iterations are over
 * by then). One stepwise solve
 * per mesh at a time; b and x must stay valid until hb_cg_finish, and the
 * mesh's other solver calls must not run in between. */
hb_status hb_cg_begin(hb_mesh *mesh, const hb_cg_opts *opts, const double *b, double *x, void *stream);
hb_status hb_cg_iterate(hb_mesh *mesh, int count, void *stream);
hb_status hb_cg_finish(hb_mesh *mesh, hb_cg_result *res, void *stream);

/* ---------------------------------------------------------------- partitioned operator
 * The operator split the way a distributed run applies it (Sec. 3.3,
 * "Overlapping halo and gather communication", and its operator timeline
 * figure), with the ranks emulated on one GPU: the element box is cut into
 * px x py x pz blocks of elements, one virtual rank each, every rank with its
 * own CUDA streams, element data and exchange buffers in device memory.
 *  - A node shared by elements of several ranks is a halo node; an element
 *    holding one is a halo element, the others are interior elements.
 *  - Each assembled DOF has one owner: a DOF of one rank's elements belongs to
 *    it; a halo DOF goes to one of the ranks that hold it, picked at random
 *    but fairly (uniformly among them, by u01(seed, 3, g), g its lexicographic
 *    global id).
 *  - Vectors are in partition order: rank 0's owned DOFs, then rank 1's, ...,
 *    each rank's in lexicographic order (hb_part_copy_perm gives the map).
 * y = A x runs per rank as: pack the owned values other ranks need; element
 * kernel on the first half of the interior elements while the halo values are
 * copied into the receivers' halo buffers; element kernel on the halo
 * elements; gather their partial sums at halo nodes into send buffers; element
 * kernel on the other half of the interior elements and the rank-local gather
 * Z^T while those partial sums are copied to the owners; the owners add them
 * in rank order. The result equals hb_apply_A's up to the order of the sums.
 * Precision FP64; the element kernel is the mesh's FP64 pencil variant
 * (variant 0 runs as variant 3). */
typedef struct hb_part hb_part;
typedef struct {
    int n_ranks;
    int64_t n_global;
    int64_t n_shared;        /* DOFs held by more than one rank */
    int64_t exchange_values; /* values each halo exchange moves (= each gather exchange) */
} hb_part_info_t;
typedef struct {
    int64_t n_owned, offset;          /* owned DOFs and their start in partition order */
    int64_t n_halo;                   /* DOFs other ranks own that this rank's elements hold */
    int64_t n_send;                   /* owned values sent per halo exchange */
    int64_t n_elem_interior1, n_elem_halo, n_elem_interior2;
} hb_part_rank_info_t;

/* Builds the partition of `mesh` (which must outlive it) on the mesh's device;
 * 1 <= px <= ex (same for y, z), px*py*pz <= 64. Host work O(n_local);
 * synchronises `stream`. */
hb_status hb_part_create(const hb_mesh *mesh, int px, int py, int pz, uint64_t seed, void *stream,
                         hb_part **out);
hb_status hb_part_destroy(hb_part *part);
/* The same partition planned on the host alone (no device work; what
 * hb_part_create does before it uploads): l2g_host is the mesh's node map
 * (ex*ey*ez*(N+1)^3 int32, -1 on masked nodes, e.g. from hb_mesh_copy_l2g).
 * Writes perm_host (n_global int32, as hb_part_copy_perm) and counts_host
 * (2 + 8*px*py*pz int64): n_shared, exchange_values, then per rank n_owned,
 * offset, n_halo, n_send, n_elem_interior1, n_elem_halo, n_elem_interior2 and
 * the number of owned DOFs other ranks hold. HB_ERR_ARG for bad sizes or a
 * node map that is out of range or leaves a DOF without an element. */
hb_status hb_part_plan(const int32_t *l2g_host, int ex, int ey, int ez, int N, int64_t n_global, int px, int py,
                       int pz, uint64_t seed, int32_t *perm_host, int64_t *counts_host);
hb_status hb_part_info(const hb_part *part, hb_part_info_t *out);
hb_status hb_part_rank_info(const hb_part *part, int rank, hb_part_rank_info_t *out);
/* perm_host[i] = the mesh's (lexicographic) global id of partition-order DOF i;
 * n_global int32 values; synchronous. */
hb_status hb_part_copy_perm(const hb_part *part, int32_t *perm_host);
/* y = A x with x, y FP64 device vectors of n_global values in partition order
 * (x and y must not overlap). Ordered after and before `stream`. */
hb_status hb_part_apply_A(const hb_part *part, hb_screen screen, double lambda, const double *x, double *y,
                          void *stream);
/* The halo exchange alone: fills every rank's halo buffer from x (partition
 * order); with halo_host != NULL also copies rank `rank`'s halo buffer
 * (n_halo doubles) there and synchronises. */
hb_status hb_part_halo_exchange(const hb_part *part, const double *x, int rank, double *halo_host, void *stream);
/* hb_cg_solve (HB_F64, no preconditioner) with the partitioned operator; b and x
 * in partition order. Dot products run over the concatenated owned segments
 * (the sum over ranks in rank order of each rank's part). */
hb_status hb_part_cg_solve(const hb_part *part, const hb_cg_opts *opts, const double *b, double *x,
                           hb_cg_result *res, void *stream);

/* ---------------------------------------------------------------- scattered storage
 * NekBone's storage of the DOF vectors (Sec. 2, the scattered form, and
 * Sec. 3.1 "DOF Storage"): vectors have n_local entries x_L = Z x_G, one per
 * element node (element e's node q at e (N+1)^3 + q, q = i + n (j + n k)), and
 * the operator is b_L = (Z Z^T S_L + lambda I) x_L: the element-local S_L on
 * x_L, then the gather-scatter Z Z^T, which sums the copies of each DOF and
 * writes the sum back to every copy. Masked (Dirichlet) nodes hold 0. Inner
 * products are weighted by the inverse multiplicity c_L = 1 / (Z^T Z)_gg (0 at
 * masked nodes), so (a_L, b_L)_c = a_G . b_G. The library offers it to measure
 * the paper's claim that assembled storage moves fewer bytes per CG iteration;
 * results equal the assembled path's up to rounding. FP64 only. */
typedef struct hb_scat hb_scat;
/* Builds the weights, the masked-node list and the copy map of `mesh` (which
 * must outlive it); synchronises `stream`. */
hb_status hb_scat_create(const hb_mesh *mesh, void *stream, hb_scat **out);
hb_status hb_scat_destroy(hb_scat *sc);
/* x_L = Z x_G (x_G: n_global doubles; x_L: n_local doubles; device). */
hb_status hb_scat_scatter(const hb_scat *sc, const double *xG, double *xL, void *stream);
/* y_L = (Z Z^T S_L + lambda I) x_L (identity screening) or with lambda M_gg
 * x_g at every copy (mass screening); x_L, y_L device, n_local doubles, must
 * not overlap. */
hb_status hb_scat_apply_A(const hb_scat *sc, hb_screen screen, double lambda, const double *xL, double *yL,
                          void *stream);
/* Weighted inner product sum_q c_q a_q b_q (fixed-order FP64 reduction) into
 * *out_host; synchronises `stream`. */
hb_status hb_scat_dot(const hb_scat *sc, const double *aL, const double *bL, double *out_host, void *stream);
/* Algorithm 1 on scattered vectors with weighted inner products (HB_F64, no
 * preconditioner); b_L and x_L (x0 in, solution out) device, n_local doubles. */
hb_status hb_scat_cg_solve(const hb_scat *sc, const hb_cg_opts *opts, const double *bL, double *xL,
                           hb_cg_result *res, void *stream);

/* ---------------------------------------------------------------- serving
 * A CG server with continuous batching on one GPU (the paper runs one solve at
 * a time; the server applies Algorithm 1 in the FP32-inner / FP64
 * defect-correction form of hb_cg_solve to many concurrent requests).
 * Requests queue on submit; a builder thread takes them first come, first
 * served, into free slots while the device-memory budget allows and builds
 * each one's mesh, vectors and right-hand side on its own stream. A worker
 * thread keeps every resident solve going on the slot's own stream: one
 * launch of the slot's CUDA graph (captured at creation) runs a round of
 * iters_per_launch inner iterations, and the slot's next round is launched as
 * soon as its last one has finished, so solves of different sizes advance at
 * their own pace side by side. A finished solve is retired at once (its
 * memory freed in stream order). While it runs the server lets the library's
 * memory pool keep up to 32 GiB (at most its budget) of freed memory for reuse. Every slot
 * runs on fixed grids with its own
 * reductions: a request's result does not depend on which others share the
 * GPU. The right-hand side is hb_fill_rhs kind 0 with the request's seed and
 * x0 = 0. Degrees N = 1..11; opts.prec must be HB_MIXED, opts.rtol > 0 and
 * opts.precond = 0. Requests of at most 4 Mi local nodes run on higher-priority
 * streams, and while one of their rounds is in flight a larger request's next
 * round waits (2 ms at most). The server uses two streams per slot: set
 * CUDA_DEVICE_MAX_CONNECTIONS=32 before the CUDA context is created, or the
 * streams share the default 8 hardware queues and wait on each other. */
typedef struct hb_server hb_server;
typedef struct {
    size_t mem_budget_bytes;   /* device memory the resident solves may hold */
    int max_slots;             /* concurrent solves, 1..256 */
    int iters_per_launch;      /* inner CG iterations per round, 1..256 */
} hb_server_opts;
typedef struct {
    int64_t submitted, admitted, completed, rejected, rounds;
    int active, pending;
    size_t mem_used;
    /* wall seconds spent building admitted requests (builder thread), with
     * at least one round in flight, and retiring solves (worker thread);
     * rounds counts every slot's rounds */
    double admit_s, round_s, retire_s;
    /* sums over completed requests: queued (submit to build start), building,
     * running (build end to retirement) */
    double queue_s, build_s, run_s;
} hb_server_stats_t;

hb_status hb_server_create(const hb_server_opts *opts, hb_server **out);
/* Queues a request and returns its ticket. keep_x = 1 keeps the solution for
 * hb_server_poll. The mesh description's keep_fp32_copy is ignored (always 1). */
hb_status hb_server_submit(hb_server *srv, const hb_mesh_desc *desc, const hb_cg_opts *opts,
                           uint64_t rhs_seed, int keep_x, int64_t *ticket);
/* HB_ERR_BUSY while the request is queued or running; HB_OK once it finished:
 * res receives the iteration counts, the FP64 relative residual, the solve's
 * status (HB_OK, HB_ERR_NOT_CONVERGED, HB_ERR_BREAKDOWN, or HB_ERR_NOMEM when it
 * can never fit the budget) and, in time_ms, the latency from submit to
 * completion; n_global and x_host (n_global doubles, if keep_x) as asked. A
 * request that could not be built leaves the reason in hb_last_error. A
 * finished ticket is forgotten after a successful poll (HB_ERR_NOT_FOUND then). */
hb_status hb_server_poll(hb_server *srv, int64_t ticket, hb_cg_result *res, int64_t *n_global,
                         double *x_host);
hb_status hb_server_stats(hb_server *srv, hb_server_stats_t *out);
/* Stops the worker after its current round and frees every resident solve. */
hb_status hb_server_destroy(hb_server *srv);
/* Test hook for the failure path (no device work is faulted): the worker's
 * next round behaves as if launching it had failed. The server then stops;
 * every resident solve releases its device memory and every resident or
 * queued request finishes with HB_ERR_CUDA; polls of any other ticket the
 * server issued return HB_ERR_CUDA instead of HB_ERR_BUSY, and submits are
 * refused. The failure happens at the next round, i.e. once a request is
 * resident. */
hb_status hb_server_inject_round_error(hb_server *srv);

/* The library's uniform random number, u01(seed, stream, idx) =
 * (splitmix64(seed ^ (stream * 0x9E3779B97F4A7C15) + idx) >> 11) * 2^-53, with
 * splitmix64(s) the SplitMix64 output for state s (Steele, Lea & Flood 2014). */
double hb_u01(uint64_t seed, uint64_t stream, uint64_t idx);

/* Element-kernel variants of the operator (all compute the same A x; they
 * differ in thread mapping and operation count). Bit flags:
 *   0                     one thread per t-line, D and the element in shared memory
 *   HB_VARIANT_PENCIL     every 1-D contraction by a thread owning the whole line,
 *                         D from constant memory
 *   HB_VARIANT_EVEN_ODD   (with PENCIL) even-odd split of the centro-antisymmetric D:
 *                         n^2/2 + 2n operations per line instead of n^2
 *   HB_VARIANT_EB2        (with PENCIL, N <= 10) two element groups per thread block
 *   HB_VARIANT_ONE        (with PENCIL | EVEN_ODD) one element per thread block,
 *                         which spreads small meshes over more SMs
 *   HB_VARIANT_TMA        (with PENCIL | EVEN_ODD) one thread per block issues a
 *                         bulk L2 prefetch (cp.async.bulk.prefetch) of the block's
 *                         geometric factors at its start, so their DRAM reads
 *                         overlap the x gather and the first contractions.
 *   HB_VARIANT_WS         (with PENCIL | EVEN_ODD; HB_F32, odd N) persistent
 *                         warp-specialised kernel: a producer warp stages each
 *                         element group's node map and geometric factors in shared
 *                         memory with cp.async.bulk (mbarrier-tracked) while the
 *                         other warps compute the previous group. Other precisions
 *                         and even N run PENCIL | EVEN_ODD. Its waits are bounded:
 *                         one that gives up makes the next hb_cg_solve,
 *                         hb_cg_finish or hb_autotune on the mesh return
 *                         HB_ERR_TIMEOUT.
 *   HB_VARIANT_CSR        (with PENCIL | EVEN_ODD, alone or with ONE) the element
 *                         kernel writes each surface value straight to its place
 *                         in the surface CSR order, so Z^T reads contiguous runs
 *                         instead of scattered copies. Needs an int32 per surface
 *                         copy, built when the variant is first set.
 *   HB_VARIANT_GRID       (with PENCIL | EVEN_ODD, alone or with ONE; not with
 *                         CSR) the element kernel stores every local value
 *                         element-major and Z^T is taken on every DOF by the
 *                         box's lattice arithmetic (no column array): one warp
 *                         per lattice row sums each DOF's copies in ascending
 *                         element order, as the CSR does, so y is bitwise the
 *                         same as with the other pencil variants.
 *   HB_VARIANT_TC         (alone or with CSR; HB_F64 at N = 7) the tensor-core element kernel:
 *                         every derivative contraction (D and D^T along r, s, t) runs
 *                         on the tensor cores (tcgen05.mma, FP16 inputs, FP32
 *                         accumulators in tensor memory) exactly, on an
 *                         Ozaki-style split of the element's values and of D into
 *                         seven 8-bit digits on a per-element fixed-point grid
 *                         (every product and partial sum an integer below 2^24);
 *                         the exact digit sums are combined in int64 and the
 *                         metric step runs in FP64. Error per contraction about
 *                         2^-53 of the element's largest |value| times sum |D|,
 *                         the FP64 rounding level; an element holding a
 *                         non-finite value gives NaN. Same surface store and
 *                         gather as the pencil kernels (with CSR: the CSR-position
 *                         store and contiguous gather).
 * Each of HB_F64, HB_F32 and HB_F64X keeps its own variant. HB_F64X takes
 * PENCIL | EVEN_ODD with or without ONE, and with CSR or GRID or neither (the
 * six shapes its double-float kernel is built in); other variants return
 * HB_ERR_ARG for it. The default is PENCIL | EVEN_ODD; hb_autotune measures
 * and picks per mesh and precision. */
enum { HB_VARIANT_PENCIL = 1, HB_VARIANT_EVEN_ODD = 2, HB_VARIANT_EB2 = 4, HB_VARIANT_ONE = 8,
       HB_VARIANT_TMA = 16, HB_VARIANT_WS = 32, HB_VARIANT_CSR = 64, HB_VARIANT_GRID = 128,
       HB_VARIANT_TC = 256 };
hb_status hb_set_kernel_variant(hb_mesh *mesh, hb_precision prec, int variant);
hb_status hb_get_kernel_variant(const hb_mesh *mesh, hb_precision prec, int *variant);

/* Autotuner (the paper makes its 3-D / 2-D kernel switch a configurable choice
 * made from measurements, Sec. 3.2; here every variant is timed on the mesh
 * itself). Runs one untimed and `reps` timed applications of A, each with the
 * x.y reduction a CG iteration fuses into it (p.Ap), for each
 * variant (0, PENCIL, PENCIL|EVEN_ODD, PENCIL|EB2, PENCIL|EVEN_ODD|EB2,
 * PENCIL|EVEN_ODD|ONE, PENCIL|EVEN_ODD|TMA, PENCIL|EVEN_ODD|WS, PENCIL|EVEN_ODD|CSR,
 * PENCIL|EVEN_ODD|ONE|CSR, PENCIL|EVEN_ODD|GRID, PENCIL|EVEN_ODD|ONE|GRID, and TC,
 * TC|CSR for HB_F64 at N = 7; for HB_F64X the six it takes) on `stream`, keeps the
 * fastest for `prec` (HB_F64, HB_F32 or HB_F64X) on this mesh and returns it in
 * *best_variant. ms_per_variant (may be NULL) has 512 slots
 * indexed by variant and receives the mean time of each. Allocates two scratch vectors for the
 * duration of the call; synchronises `stream`. */
hb_status hb_autotune(hb_mesh *mesh, hb_precision prec, hb_screen screen, double lambda, int reps,
                      int *best_variant, double *ms_per_variant, void *stream);

/* Measurement support (the paper times its kernels with wall clocks over
 * back-to-back launches, Sec. 4.1; here each kernel is bracketed on its own
 * stream).
 * hb_kernel_launches: number of CUDA kernels this library has launched in the
 *   process so far (all entry points, all devices).
 * hb_profile_enable(1): from now on every library kernel launch is bracketed
 *   by a pair of CUDA events recorded on its launch stream (adds two event
 *   records per launch; off by default).
 * hb_profile_read: waits for the recorded events of kernel `name` ("ax_local",
 *   "assemble", "dot", "cg_update_r", "cg_update_xp") and returns the summed
 *   device time in ms and the number of launches since the last reset.
 * hb_profile_reset: forgets the recorded launches. */
unsigned long long hb_kernel_launches(void);
hb_status hb_profile_enable(int on);
hb_status hb_profile_reset(void);
hb_status hb_profile_read(const char *name, double *total_ms, long long *launches);

/* Calibration probes (the paper calibrates its roofline with an 8-read /
 * 1-write streaming kernel, Sec. 4.1). Runs `reps` timed launches after one
 * untimed one on a scratch buffer of `bytes` bytes (allocated for the call)
 * and returns the best rate in *rate: GB/s (read + write bytes) for the
 * stream and copy kinds, GFLOP/s for HB_PROBE_FMA (bytes ignored).
 *   HB_PROBE_STREAM81_FP   8 reads, 1 write of their sum in `prec`
 *   HB_PROBE_STREAM81_BITS the same traffic combined with XOR (no FP work)
 *   HB_PROBE_COPY          16-byte vector copy
 *   HB_PROBE_FMA           independent FMA chains in `prec`
 *   HB_PROBE_DMMA          FP64 warp matrix multiply-accumulate (mma.sync m8n8k4)
 *   HB_PROBE_DMMA_FMA      the two above interleaved in one loop (prec ignored)
 *   HB_PROBE_CVT64         int64 -> FP64 -> int64 conversion chains; *rate in
 *                          G conversions/s (prec ignored) */
enum { HB_PROBE_STREAM81_FP = 0, HB_PROBE_STREAM81_BITS = 1, HB_PROBE_COPY = 2, HB_PROBE_FMA = 3,
       HB_PROBE_DMMA = 4, HB_PROBE_DMMA_FMA = 5, HB_PROBE_CVT64 = 6 };
hb_status hb_probe(int kind, hb_precision prec, size_t bytes, int reps, double *rate);

/* Self-test of the bounded device waits (every wait in this library's
 * kernels gives up after about one second of wall time, records the failure
 * in an error word and lets the kernel finish; the call that started it then
 * returns HB_ERR_TIMEOUT). which = 0 runs a kernel whose mbarrier wait (the
 * staged pipeline of HB_VARIANT_WS) never completes; which = 1 a cooperative
 * kernel whose grid barrier (the fused CG) waits for one block more than it
 * launched. Neither faults or hangs: *status receives HB_ERR_TIMEOUT when the
 * kernel gave up and reported it (the expected outcome), HB_OK if it reported
 * nothing. Takes about a second; synchronises `stream`. */
hb_status hb_selftest_wait(int which, hb_status *status, void *stream);

/* Self-check of the tensor-core operand layouts the tensor-core element
 * kernel uses (no paper counterpart: a check of the hardware interface).
 * Computes D = A B^T through tcgen05.mma kind::f16 (M = 128, N = 48, K = 48 in
 * three steps of 16; FP16 operands from shared memory, FP32 accumulator in
 * tensor memory) on one thread block. A_host: 128 x 48, B_host: 48 x 48,
 * D_host: 128 x 48 floats, row-major; inputs are rounded to FP16. mode bit 0:
 * A staged MN-major instead of K-major; bit 1: the descriptors' leading and
 * stride byte-offset fields exchanged (a wrong layout on purpose, to tell the
 * two conventions apart; it stays inside the zeroed staging area). *status
 * receives HB_OK, or HB_ERR_TIMEOUT if the bounded wait for the MMA ran out.
 * Allocates and synchronises the current device. */
hb_status hb_tc_selftest(int mode, const float *A_host, const float *B_host, float *D_host, hb_status *status);

/* Message for the last failed call on this thread ("" if none). */
const char *hb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HIPBONE_GB300_H */
