// Element-local operator, "pencil" variant (v2):
//   y_L = S_L Z x,  S_L^e = Dbold^T G^e Dbold   (hipBone Sec. 2, Sec. 3.2).
//
// Every 1-D contraction is done by a thread that owns a whole line of n = N+1
// nodes, so the n x n matrix D is applied with compile-time indices and read
// from __constant__ memory (one address per warp: a constant-bank operand,
// no registers or shared-memory reads for D). Per element, n^2 threads:
//   1. thread (i,j) gathers its t-line u(i,j,.) through l2g, forms u_t in
//      registers and copies u to shared memory;
//   2. thread (j,k) forms u_r along its r-line, thread (i,k) u_s along its
//      s-line (shared memory in, shared memory out);
//   3. thread (i,j) applies the six metric factors at its t-line (factors
//      streamed from HBM once), keeps v_t in registers, writes v_r, v_s;
//   4. D^T along r-lines, then along s-lines (accumulated), then along the
//      t-line in registers, and y_L is written.
// EO = true uses the even-odd split of D: D is centro-antisymmetric
// (D_{N-i,N-m} = -D_{i,m}), so with a_m = u_m + u_{N-m}, b_m = u_m - u_{N-m}
// (m < n/2), P_i = sum_m E_im a_m and Q_i = sum_m O_im b_m
// (E = (D_im + D_{i,N-m})/2, O = (D_im - D_{i,N-m})/2), the outputs are
// y_i = P_i + Q_i and y_{N-i} = Q_i - P_i: n^2/2 + 2n operations per line
// instead of n^2.
#pragma once

#include "hb_internal.h"
#include "hb_acc.cuh"

#ifndef HB_AX2_T
#error "define HB_AX2_T (the compute type: double, float or df) before including hb_ax2.cuh"
#endif
#ifndef HB_AX2_S
#define HB_AX2_S HB_AX2_T
#endif

#include <type_traits>

#include "hb_df.cuh"

namespace hb2 {
// Internal linkage: this header is compiled once per precision (T differs by
// translation unit), so nothing in it may share a symbol name across units.
namespace {

using T = HB_AX2_T;  // arithmetic of the element kernel
using S = HB_AX2_S;  // storage of x, y and the geometric factors

// Conversions between storage and compute types (identity unless the kernel
// computes in double-float on FP64 data).
template <typename TT, typename SS>
struct conv {
    static __device__ __forceinline__ TT c(SS v) { return v; }
    static __device__ __forceinline__ SS s(TT v) { return v; }
    static TT table(double v) { return (TT)v; }
};
template <>
struct conv<df, double> {
    static __device__ __forceinline__ df c(double v) { return df_from_double(v); }
    static __device__ __forceinline__ double s(df v) { return df_to_double(v); }
    static df table(double v)
    {
        const float h = (float)v;
        return df(h, (float)(v - (double)h));
    }
};
__device__ __forceinline__ T to_c(S v) { return conv<T, S>::c(v); }
__device__ __forceinline__ S to_s(T v) { return conv<T, S>::s(v); }
// Host: a table entry of the compute type from an FP64 value.
static inline T table_value(double v) { return conv<T, S>::table(v); }

// ------------------------------------------------------------ constant tables
// Per degree N (n = N+1, h = ceil(n/2)): D and D^T at offset off(N) =
// sum_{M<N} (M+1)^2, and the even-odd halves E, O of D and of D^T ([i][m],
// i, m < h) at offset offh(N) = sum_{M<N} h(M)^2. One copy per precision,
// in this translation unit's constant bank.
__host__ __device__ constexpr int off(int N)
{
    int o = 0;
    for (int M = 1; M < N; M++) o += (M + 1) * (M + 1);
    return o;
}
__host__ __device__ constexpr int hh(int N) { return (N + 2) / 2; }
__host__ __device__ constexpr int offh(int N)
{
    int o = 0;
    for (int M = 1; M < N; M++) o += hh(M) * hh(M);
    return o;
}
constexpr int kTable = off(HB_MAX_N + 1);
constexpr int kHalf = offh(HB_MAX_N + 1);

static __constant__ T c_D[kTable], c_Dt[kTable], c_E[kHalf], c_O[kHalf], c_Et[kHalf], c_Ot[kHalf];

// Uploads the tables of all degrees to the current device from the FP64
// derivative matrices D_all (laid out at off(N)).
static inline hb_status upload_tables(const double *D_all)
{
    static T hD[kTable], hDt[kTable], hE[kHalf], hO[kHalf], hEt[kHalf], hOt[kHalf];
    for (int N = 1; N <= HB_MAX_N; N++) {
        const int n = N + 1, h = hh(N), o = off(N), oh = offh(N);
        const double *D = D_all + o;
        for (int i = 0; i < n; i++)
            for (int m = 0; m < n; m++) {
                hD[o + i * n + m] = table_value(D[i * n + m]);
                hDt[o + i * n + m] = table_value(D[m * n + i]);
            }
        for (int i = 0; i < h; i++)
            for (int m = 0; m < h; m++) {
                const int mm = N - m;
                double e, od, et, ot;
                if (m == mm) {  // middle column (odd n)
                    e = D[i * n + m];
                    od = 0.0;
                    et = D[m * n + i];
                    ot = 0.0;
                } else {
                    e = 0.5 * (D[i * n + m] + D[i * n + mm]);
                    od = 0.5 * (D[i * n + m] - D[i * n + mm]);
                    et = 0.5 * (D[m * n + i] + D[mm * n + i]);
                    ot = 0.5 * (D[m * n + i] - D[mm * n + i]);
                }
                hE[oh + i * h + m] = table_value(e);
                hO[oh + i * h + m] = table_value(od);
                hEt[oh + i * h + m] = table_value(et);
                hOt[oh + i * h + m] = table_value(ot);
            }
    }
    HB_TRY_CUDA(cudaMemcpyToSymbol(c_D, hD, sizeof hD));
    HB_TRY_CUDA(cudaMemcpyToSymbol(c_Dt, hDt, sizeof hDt));
    HB_TRY_CUDA(cudaMemcpyToSymbol(c_E, hE, sizeof hE));
    HB_TRY_CUDA(cudaMemcpyToSymbol(c_O, hO, sizeof hO));
    HB_TRY_CUDA(cudaMemcpyToSymbol(c_Et, hEt, sizeof hEt));
    HB_TRY_CUDA(cudaMemcpyToSymbol(c_Ot, hOt, sizeof hOt));
    return HB_OK;
}

// ------------------------------------------------------------ staged pipeline
// The warp-specialised variant (WS): a producer warp copies each element
// group's node map and geometric factors (contiguous in memory) into shared
// memory with cp.async.bulk; mbarriers count the bytes in ("full") and the
// consumer warps' releases ("empty"). Every wait is bounded: after about
// kWaitNs of wall time it records bit 0 in the kernel's error word and carries
// on, so no thread ever leaves the common control flow (the results are then
// wrong and the error is reported by the host).
constexpr unsigned long long kWaitNs = 1000000000ull;

// Wall time in ns (the GPU's global timer), for bounded waits.
__device__ __forceinline__ unsigned long long wall_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Announces `bytes` on the barrier and starts the copy (addresses and size
// multiples of 16 bytes).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Waits (bounded) for phase `parity` of the barrier to complete.
__device__ __forceinline__ void mbar_wait(uint64_t *bar, unsigned parity, unsigned *err)
{
    const unsigned a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned t = 0;; t++) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return;
        if ((t & 255u) == 0) {
            const unsigned long long now = wall_ns();
            if (t == 0) t0 = now;
            else if (now - t0 > kWaitNs) break;
        }
    }
    if (err) atomicOr(err, 1u);
}

// Shared state of one WS block for the group being computed.
struct ws_ctx {
    const int32_t *lsm;  // staged node map of the group
    const void *gsm;     // staged geometric factors of the group (S)
    uint64_t *full_l, *empty_l, *full_g, *empty_g;
    unsigned parity;     // phase parity of this group's barriers
    unsigned *err;
};

// ------------------------------------------------------------ line contractions

// Applies M = D (TR = false) or D^T (TR = true) to one line held in `in`
// (clobbered) and hands each output to store(i, value) as soon as it is
// formed, so only the n inputs stay live in registers. With EO the line is
// folded in place into a_m = in_m + in_{N-m} (kept in in[m]) and
// b_m = in_m - in_{N-m} (kept in in[N-m]).
template <int N, bool TR, bool EO, class F>
__device__ __forceinline__ void line_st(T (&in)[N + 1], F &&store)
{
    constexpr int n = N + 1, o = off(N);
    const T *M = TR ? c_Dt : c_D;
    if constexpr (!EO) {
#pragma unroll
        for (int i = 0; i < n; i++) {
            T acc = M[o + i * n] * in[0];
#pragma unroll
            for (int m = 1; m < n; m++) acc = fma(M[o + i * n + m], in[m], acc);
            store(i, acc);
        }
    } else {
        constexpr int h = hh(N), oh = offh(N), half = n / 2;
        constexpr bool odd = (n & 1) != 0;
        const T *Ec = TR ? c_Et : c_E;
        const T *Oc = TR ? c_Ot : c_O;
#pragma unroll
        for (int m = 0; m < half; m++) {
            const T u = in[m], v = in[N - m];
            in[m] = u + v;
            in[N - m] = u - v;
        }
#pragma unroll
        for (int i = 0; i < half; i++) {
            T P = Ec[oh + i * h] * in[0];
            T Q = Oc[oh + i * h] * in[N];
#pragma unroll
            for (int m = 1; m < half; m++) {
                P = fma(Ec[oh + i * h + m], in[m], P);
                Q = fma(Oc[oh + i * h + m], in[N - m], Q);
            }
            if constexpr (odd) P = fma(Ec[oh + i * h + half], in[half], P);  // middle node
            store(i, P + Q);
            store(N - i, Q - P);
        }
        if constexpr (odd) {
            // middle row c = n/2: y_c = sum_{m<c} M[c][m] b_m
            T Q = M[o + half * n] * in[N];
#pragma unroll
            for (int m = 1; m < half; m++) Q = fma(M[o + half * n + m], in[N - m], Q);
            store(half, Q);
        }
    }
}

template <int N>
struct shape {
    static constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
};

// ------------------------------------------------------------ the kernel

// Arguments of the pencil kernel. Element-interior nodes (1 <= i,j,k <= N-1)
// carry a DOF no other element touches: their y = (S_L u)_node + lambda (x or
// Jw x) goes straight to y[g], and x_g y_g into this block's partial of x.y
// (partials[blockIdx.x], if partials is not null). Surface nodes go to ysurf
// in the per-element surface order of surf_index() for the Z^T gather.
struct pencil_args {
    const S *x;
    const int32_t *l2g;
    const S *geo;
    S *ysurf;
    S *y;
    int64_t E;
    const int *run;
    S lambda;
    int screen;
    double *partials;
    // l2g entries g <= -2 read halo[-2 - g] (values of DOFs another partition
    // owns, filled by a halo exchange); -1 is a masked node
    const S *halo;
    unsigned *err;  // WS kernels: bit 0 set when a bounded wait gave up
    // SP kernels: CSR position of every surface copy (e * surface nodes +
    // surface index; -1 masked); ysurf is then indexed by CSR position
    const int32_t *spos;
};

// ------------------------------------------------------------ L2 prefetch
// One thread asks the memory system to bring a block's geometric factors
// (contiguous in memory) into L2 with a bulk prefetch, so their DRAM reads
// overlap the x gather and the first contractions. Only the 16-byte-aligned
// interior of the range is named; nothing is waited for.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uintptr_t lo = (a + 15) & ~uintptr_t(15), hi = (a + bytes) & ~uintptr_t(15);
    for (uintptr_t q = lo; q < hi;) {
        const uintptr_t chunk = hi - q < (uintptr_t(1) << 20) ? hi - q : (uintptr_t(1) << 20);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"((unsigned)chunk) : "memory");
        q += chunk;
    }
}

// Position of surface node (i,j,k) in its element's surface block:
// the k = 0 face, the k = N face, then for k = 1..N-1 the ring of 4N nodes of
// that slab (j = 0 row, j = N row, then i = 0 / i = N for j = 1..N-1).
template <int N>
__host__ __device__ constexpr int surf_count() { return 2 * (N + 1) * (N + 1) + 4 * N * (N - 1); }
template <int N>
__device__ __forceinline__ int ring_index(int i, int j)
{
    return j == 0 ? i : (j == N ? N + 1 + i : 2 * (N + 1) + 2 * (j - 1) + (i == N ? 1 : 0));
}

// Shared-memory layout of one element buffer: node (i,j,k) at
// k*n*(n+1) + j*(n+1) + i (rows padded by one to spread banks).
template <int N>
struct pad {
    static constexpr int n = N + 1, rs = n + 1, ss = n * (n + 1), size = n * n * (n + 1);
    static __device__ __forceinline__ int at(int i, int j, int k) { return k * ss + j * rs + i; }
};

// Blocks per SM that shared memory allows (228 KB per SM, 1 KB reserved per
// block); the register budget is set to match so occupancy is not lost to it.
// Degrees whose kernel reads its node ids again for the interior-node
// epilogue rather than holding n of them in registers through every phase:
// where that buys more resident blocks. Measured on the full-size operator
// (about 128M local nodes): FP32 N = 3, 7, 9 and 11..13 gain 5-21% with the
// resident-block counts of f32_blocks(); N = 8, 14 and 15 gain with three
// element buffers (nbuf); at N = 5 and 10 the extra loads cost more than the
// residency gains. Double-float (with three element
// buffers below N = 11, so four blocks fit): N = 5, 7, 10 and 11.
template <int N>
__host__ __device__ constexpr bool reload_ids()
{
    if constexpr (sizeof(S) == 4) return N == 3 || N == 7 || N == 8 || N == 9 || (N >= 11 && N <= 15);
    else if constexpr (!std::is_same<T, S>::value) return N == 5 || N == 7 || N == 10 || N == 11;
    else return false;
}

// Resident blocks per SM asked of the FP32 kernel (memory-bound: latency is
// hidden by residency), per degree, from the same measurements: 4 (2 for
// n^2 > 128, whose lines need registers) unless the node ids are reloaded.
template <int N>
__host__ __device__ constexpr int f32_blocks()
{
    switch (N) {
    case 3: case 8: case 11: return 6;
    case 7: case 9: case 12: return 5;
    case 13: case 14: return 4;
    case 15: return 3;
    default: return (N + 1) * (N + 1) > 128 ? 2 : 4;
    }
}

// Element buffers in shared memory per element: 4 (u, then the r, s, t
// lines), or 3 where the t-line buffer takes the place of u once every r- and
// s-line has read it (one more block barrier; u is then gone for the
// epilogue, which reads x again). Three buffers where that lets more blocks
// reside and residency is the limit: the double-float kernel (issue-bound,
// shared memory limits it to 3 blocks per SM with 4 buffers at N <= 10) and
// the FP32 kernel at N = 8, 14, 15 (operator 4 %, 3 %, 1.5 % faster; at the
// other degrees registers limit it first or nothing was gained).
// Measured on the full-size double-float operator: N = 7 4.84 -> 4.40 ms,
// N = 8 5.60 -> 4.95, N = 10 6.99 -> 5.25, N = 1 3.82 -> 3.26; N = 2..5 and 9
// within 1 %.
template <int N>
__host__ __device__ constexpr int nbuf()
{
    if constexpr (sizeof(T) == 4) return (N == 8 || N == 14 || N == 15) ? 3 : 4;
    return (!std::is_same<T, S>::value && (N + 1) * (N + 1) <= 128) ? 3 : 4;
}

template <int N, int EB>
__host__ __device__ constexpr int pencil_min_blocks()
{
    constexpr int smem = (int)sizeof(T) * nbuf<N>() * EB * pad<N>::size + 1024;
    constexpr int by_smem = (228 * 1024) / smem;
    constexpr int by_threads = 2048 / (EB * (N + 1) * (N + 1));
    constexpr int b = by_smem < by_threads ? by_smem : by_threads;
    // FP64 is bound by the FP64 pipe: no register cap (a cap only adds spills).
    // FP32 is bound by memory: ask for the resident blocks shared memory
    // allows, up to f32_blocks().
    if constexpr (std::is_same<T, double>::value) return 1;
    // double-float: bound by the FP32 issue rate, so residency matters too
    // (up to 4, 3 at N = 9; for n^2 > 128 2, or 3 where the node ids are
    // reloaded; measured per degree like FP32)
    constexpr int cap = sizeof(T) == 4 ? f32_blocks<N>()
                                       : ((N + 1) * (N + 1) > 128 ? (reload_ids<N>() ? 3 : 2) : (N == 9 ? 3 : 4));
    return b < 1 ? 1 : (b > cap ? cap : b);
}

// One group of EB elements (group index `grp`), by the first EB*(N+1)^2
// threads of the block; further threads only join the barriers. Adds the
// group's interior-node x.y to `acc`. Every thread of the block must call it
// (it synchronises the block).
// Gather modes: GM_L2G reads x through l2g (-1 = masked); GM_HALO also reads
// halo[-2 - g] for l2g entries g <= -2 (partitioned operator); GM_SCAT reads
// scattered vectors, node q of element e at e n^3 + q (no l2g). A template
// parameter, so the common kernel carries no branch for the other two.
// GM_L2G_CG is GM_L2G for kernels that write x themselves between element
// passes (the fused CG): x is read through L2 (ld.global.cg), never through
// the non-coherent read-only path.
enum { GM_L2G = 0, GM_HALO = 1, GM_SCAT = 2, GM_L2G_CG = 3 };

// Barrier of the threads computing a group: the whole block, or (WS) the
// consumer warps only (named barrier 1), the producer warp running apart.
template <bool WS, int NC>
__device__ __forceinline__ void group_sync()
{
    if constexpr (WS) asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
    else __syncthreads();
}

template <int N, int EB>
__host__ __device__ constexpr int ws_consumers() { return (EB * (N + 1) * (N + 1) + 31) / 32 * 32; }

// KEEP_IDS: hold the node ids in registers whatever reload_ids() says (for
// kernels whose residency is fixed by other means, as the serving classes).
// NB: element buffers (4, or 3 with the t-line buffer in place of u).
// FL: every local value to ysurf[e n^3 + node] (element-major, [k][j][i]);
// no interior finish, lambda term or partial here: the lattice gather does
// all of Z^T.
template <int N, bool EO, int EB, int GM = GM_L2G, bool WS = false, bool SP = false, bool KEEP_IDS = false,
          int NB = 4, bool FL = false>
__device__ __forceinline__ void pencil_group(const pencil_args &A, int64_t grp, T *sm,
                                             hbacc::dot_acc<S> &acc, const ws_ctx *w = nullptr)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr int NC = ws_consumers<N, EB>();
    static_assert(!WS || GM == GM_L2G, "the staged pipeline reads x through l2g");
    static_assert(GM != GM_L2G_CG || std::is_same<T, S>::value, "the fused path is FP32 or FP64");
    static_assert(!(FL && (SP || WS || GM != GM_L2G)), "the element-major store is a plain-kernel mode");
    constexpr bool kReloadIds = GM != GM_SCAT && !KEEP_IDS && !FL && reload_ids<N>();
    using P = pad<N>;
    const S *__restrict__ x = A.x;
    const int32_t *__restrict__ l2g = A.l2g;
    const S *__restrict__ geo = A.geo;
    const int64_t E = A.E;
    const int tid = threadIdx.x;
    const int el = tid / n2;
    const int a = tid - el * n2;       // 0 .. n^2-1
    const int p0 = a % n, p1 = a / n;  // line owned in each direction
    const int64_t e = grp * EB + el;
    const bool active = el < EB && e < E;
    static_assert(NB == 3 || NB == 4, "three or four element buffers");
    static_assert(NB == 4 || (!WS && GM == GM_L2G), "three buffers only in the plain kernel");
    T *U = sm + el * NB * P::size;  // gathered u (with 4 buffers kept: the x values of the epilogue)
    T *B1 = U + P::size;            // r: u_r, v_r, D^T_r v_r
    T *B2 = B1 + P::size;           // s
    T *B3 = NB == 3 ? U : B2 + P::size;  // t

    int gl[n];  // node ids of this thread's t-line (i,j) = (p0,p1)
    if (active) {
        if constexpr (GM == GM_SCAT) {
            const int lbase = (int)(e * n3 + a);
#pragma unroll
            for (int k = 0; k < n; k++) {
                gl[k] = lbase + k * n2;
                U[P::at(p0, p1, k)] = to_c(__ldg(x + gl[k]));
            }
        } else {
            const int32_t *lg = WS ? w->lsm + el * n3 + a : l2g + e * n3 + a;
            if constexpr (WS) mbar_wait(w->full_l, w->parity, w->err);
#pragma unroll
            for (int k = 0; k < n; k++) {
                const int g = WS ? lg[k * n2] : (kReloadIds ? __ldg(lg + k * n2) : __ldcs(lg + k * n2));
                gl[k] = g;
                if constexpr (GM == GM_HALO) {
                    S v = S(0);
                    if (g >= 0) v = __ldg(x + g);
                    else if (g < -1) v = __ldg(A.halo + (-2 - g));
                    U[P::at(p0, p1, k)] = to_c(v);
                } else if constexpr (GM == GM_L2G_CG) {
                    U[P::at(p0, p1, k)] = g >= 0 ? to_c(__ldcg(x + g)) : T(0);
                } else {
                    U[P::at(p0, p1, k)] = g >= 0 ? to_c(__ldg(x + g)) : T(0);
                }
            }
        }
    } else if constexpr (WS) {
        mbar_wait(w->full_l, w->parity, w->err);  // keep every thread's phase in step
    }
    if constexpr (WS) {
        // this warp is done with the staged node map
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(w->empty_l);
    }
    group_sync<WS, NC>();
    if (active) {
        T in[n];
        // r-line (j,k) = (p0,p1)
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = U[P::at(m, p0, p1)];
        line_st<N, false, EO>(in, [&](int m, T v) { B1[P::at(m, p0, p1)] = v; });
        // s-line (i,k) = (p0,p1)
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = U[P::at(p0, m, p1)];
        line_st<N, false, EO>(in, [&](int m, T v) { B2[P::at(p0, m, p1)] = v; });
    }
    // three buffers: the t-lines overwrite u, so every r- and s-line must have
    // read it first (each t-line is then read whole before it is written)
    if constexpr (NB == 3) group_sync<WS, NC>();
    if (active) {
        T in[n];
        // t-line (i,j) = (p0,p1)
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = U[P::at(p0, p1, m)];
        line_st<N, false, EO>(in, [&](int m, T v) { B3[P::at(p0, p1, m)] = v; });
    }
    group_sync<WS, NC>();
    if constexpr (WS) mbar_wait(w->full_g, w->parity, w->err);
    if (active) {
        // metric factors at the t-line's nodes (coalesced rows of n^2 per factor)
        const S *ge = WS ? static_cast<const S *>(w->gsm) + el * 7 * n3 + a : geo + e * 7 * n3 + a;
#pragma unroll
        for (int k = 0; k < n; k++) {
            const S *g = ge + k * 7 * n2;
            T grr, grs, grt, gss, gst, gtt;
            if constexpr (WS) {
                grr = to_c(g[0]), grs = to_c(g[n2]), grt = to_c(g[2 * n2]);
                gss = to_c(g[3 * n2]), gst = to_c(g[4 * n2]), gtt = to_c(g[5 * n2]);
            } else {
                grr = to_c(__ldcs(g)), grs = to_c(__ldcs(g + n2)), grt = to_c(__ldcs(g + 2 * n2));
                gss = to_c(__ldcs(g + 3 * n2)), gst = to_c(__ldcs(g + 4 * n2)), gtt = to_c(__ldcs(g + 5 * n2));
            }
            const int q = P::at(p0, p1, k);
            const T ur = B1[q], us = B2[q], ut = B3[q];
            B1[q] = fma(grt, ut, fma(grs, us, grr * ur));
            B2[q] = fma(gst, ut, fma(gss, us, grs * ur));
            B3[q] = fma(gtt, ut, fma(gst, us, grt * ur));
        }
    }
    if constexpr (WS) {
        // this warp is done with the staged factors
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(w->empty_g);
    }
    group_sync<WS, NC>();
    if (active) {
        // D^T along each direction, in place (the whole line is in registers
        // before any output of it is stored)
        T in[n];
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = B1[P::at(m, p0, p1)];
        line_st<N, true, EO>(in, [&](int m, T v) { B1[P::at(m, p0, p1)] = v; });
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = B2[P::at(p0, m, p1)];
        line_st<N, true, EO>(in, [&](int m, T v) { B2[P::at(p0, m, p1)] = v; });
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = B3[P::at(p0, p1, m)];
        line_st<N, true, EO>(in, [&](int m, T v) { B3[P::at(p0, p1, m)] = v; });
    }
    group_sync<WS, NC>();
    if (FL && active) {
        // element-major: thread (p0,p1) stores its t-line, coalesced across the block
        S *yl = A.ysurf + e * n3 + a;
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int q = P::at(p0, p1, k);
            yl[k * n2] = to_s(B1[q] + B2[q] + B3[q]);
        }
    } else if (active) {
        constexpr int NS = surf_count<N>();
        S *ys = A.ysurf + e * NS;
        const bool ring = p0 == 0 || p0 == N || p1 == 0 || p1 == N;
        const int r = ring ? ring_index<N>(p0, p1) : 0;
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int q = P::at(p0, p1, k);
            const T yc = B1[q] + B2[q] + B3[q];
            if (SP && (k == 0 || k == N || ring)) {
                // straight to the copy's CSR position (the gather reads contiguous runs)
                const int sidx = k == 0 ? a : (k == N ? n2 + a : 2 * n2 + (k - 1) * 4 * N + r);
                const int pos = __ldg(A.spos + e * NS + sidx);
                if (pos >= 0) A.ysurf[pos] = to_s(yc);
            } else if (k == 0) {
                ys[a] = to_s(yc);
            } else if (k == N) {
                ys[n2 + a] = to_s(yc);
            } else if (ring) {
                ys[2 * n2 + (k - 1) * 4 * N + r] = to_s(yc);
            } else {
                // element-interior node: its DOF has no other copy (never masked)
                // (the double-float copy in U holds 47 bits of x: reload the value itself)
                const int gk = kReloadIds ? __ldg(l2g + e * n3 + a + k * n2) : gl[k];
                const S xv = (std::is_same<T, S>::value && NB == 4) ? to_s(U[q]) : __ldg(x + gk);
                const S jw = A.screen ? __ldg(geo + (e * n + k) * 7 * n2 + 6 * n2 + a) : S(1);
                S y = to_s(yc);
                y += A.lambda * (jw * xv);
                A.y[gk] = y;
                acc.add(xv, y);
            }
        }
    }
    group_sync<WS, NC>();  // the buffers are reused by the next group
}

template <int N, bool EO, int EB, bool PF = false, int GM = GM_L2G, bool SP = false, bool FL = false>
__global__ void __launch_bounds__(EB *(N + 1) * (N + 1), (pencil_min_blocks<N, EB>()))
    ax_pencil_kernel(const pencil_args A)
{
    if (A.run && *A.run == 0) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    hbacc::dot_acc<S> acc;
    if constexpr (PF) {
        if (threadIdx.x == 0) {
            constexpr int64_t n3 = (N + 1) * (N + 1) * (N + 1);
            const int64_t e0 = (int64_t)blockIdx.x * EB;
            const int64_t cnt = A.E - e0 < EB ? A.E - e0 : EB;
            prefetch_l2(A.geo + e0 * 7 * n3, (size_t)(cnt * 7 * n3) * sizeof(S));
        }
    }
    constexpr int NB = GM == GM_L2G ? nbuf<N>() : 4;
    pencil_group<N, EO, EB, GM, false, SP, false, NB, FL>(A, blockIdx.x, reinterpret_cast<T *>(smem_raw), acc);
    if (A.partials) {
        const double v = hbacc::block_sum(acc.value());
        if (threadIdx.x == 0) A.partials[blockIdx.x] = v;
    }
}

// ------------------------------------------------------------ three-group element
// One element per block on 3 (N+1)^2 threads: group d = 0, 1, 2 of n^2
// threads contracts the r-, s- or t-lines respectively (the three directions
// at once), and the gather, metric and epilogue phases split each t-line's
// k range over the groups (k = d, d + 3, ...). For a small mesh, where the
// element's own latency sets the time, this keeps all four FP64 units of an
// SM busy instead of the two that n^2 threads reach. Same arithmetic as
// pencil_group per node. Every thread of the block must call it.
template <int N, int GM = GM_L2G>
__device__ __forceinline__ void pencil_element3(const pencil_args &A, int64_t e, T *sm, hbacc::dot_acc<S> &acc)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr int NS = surf_count<N>();
    using P = pad<N>;
    const S *__restrict__ x = A.x;
    const int32_t *__restrict__ l2g = A.l2g;
    const S *__restrict__ geo = A.geo;
    const int tid = threadIdx.x;
    const int d = tid / n2;            // 0 r, 1 s, 2 t; 3+ idle
    const int a = tid - d * n2;
    const int p0 = a % n, p1 = a / n;
    const bool active = d < 3 && e < A.E;
    T *U = sm;
    T *B1 = U + P::size, *B2 = B1 + P::size, *B3 = B2 + P::size;
    T *Bd = d == 0 ? B1 : (d == 1 ? B2 : B3);
    if (active) {
        const int32_t *lg = l2g + e * n3 + a;
        for (int k = d; k < n; k += 3) {
            const int g = __ldcs(lg + k * n2);
            S v = S(0);
            if (g >= 0) v = GM == GM_L2G_CG ? __ldcg(x + g) : __ldg(x + g);
            U[P::at(p0, p1, k)] = to_c(v);
        }
    }
    __syncthreads();
    // the line this thread owns in its direction: node m of it at
    // r: (m, p0, p1), s: (p0, m, p1), t: (p0, p1, m)
    auto at_line = [&](int m) { return d == 0 ? P::at(m, p0, p1) : (d == 1 ? P::at(p0, m, p1) : P::at(p0, p1, m)); };
    if (active) {
        T in[n];
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = U[at_line(m)];
        line_st<N, false, true>(in, [&](int m, T v) { Bd[at_line(m)] = v; });
    }
    __syncthreads();
    if (active) {
        const S *ge = geo + e * 7 * n3 + a;
        for (int k = d; k < n; k += 3) {
            const S *g = ge + k * 7 * n2;
            const T grr = to_c(__ldcs(g)), grs = to_c(__ldcs(g + n2)), grt = to_c(__ldcs(g + 2 * n2));
            const T gss = to_c(__ldcs(g + 3 * n2)), gst = to_c(__ldcs(g + 4 * n2)), gtt = to_c(__ldcs(g + 5 * n2));
            const int q = P::at(p0, p1, k);
            const T ur = B1[q], us = B2[q], ut = B3[q];
            B1[q] = fma(grt, ut, fma(grs, us, grr * ur));
            B2[q] = fma(gst, ut, fma(gss, us, grs * ur));
            B3[q] = fma(gtt, ut, fma(gst, us, grt * ur));
        }
    }
    __syncthreads();
    if (active) {
        T in[n];
#pragma unroll
        for (int m = 0; m < n; m++) in[m] = Bd[at_line(m)];
        line_st<N, true, true>(in, [&](int m, T v) { Bd[at_line(m)] = v; });
    }
    __syncthreads();
    if (active) {
        S *ys = A.ysurf + e * NS;
        const bool ring = p0 == 0 || p0 == N || p1 == 0 || p1 == N;
        const int r = ring ? ring_index<N>(p0, p1) : 0;
        for (int k = d; k < n; k += 3) {
            const int q = P::at(p0, p1, k);
            const T yc = B1[q] + B2[q] + B3[q];
            if (k == 0) {
                ys[a] = to_s(yc);
            } else if (k == N) {
                ys[n2 + a] = to_s(yc);
            } else if (ring) {
                ys[2 * n2 + (k - 1) * 4 * N + r] = to_s(yc);
            } else {
                const int gk = __ldg(l2g + e * n3 + a + k * n2);
                const S xv = std::is_same<T, S>::value ? to_s(U[q]) : __ldg(x + gk);
                const S jw = A.screen ? __ldg(geo + (e * n + k) * 7 * n2 + 6 * n2 + a) : S(1);
                S y = to_s(yc);
                y += A.lambda * (jw * xv);
                A.y[gk] = y;
                acc.add(xv, y);
            }
        }
    }
    __syncthreads();  // the buffers are reused by the next element
}

// ------------------------------------------------------------ WS kernel
// Shared memory of a WS block: the four element buffers (T), then from
// 128-byte boundaries the staged factors (S) and node map of one group.
template <int N, int EB>
__host__ __device__ constexpr int ws_off_g() { return ((int)sizeof(T) * 4 * EB * pad<N>::size + 127) / 128 * 128; }
template <int N, int EB>
__host__ __device__ constexpr int ws_off_l()
{
    return (ws_off_g<N, EB>() + (int)sizeof(S) * 7 * EB * (N + 1) * (N + 1) * (N + 1) + 127) / 128 * 128;
}
template <int N, int EB>
__host__ __device__ constexpr int ws_smem() { return ws_off_l<N, EB>() + 4 * EB * (N + 1) * (N + 1) * (N + 1); }
template <int N, int EB>
__host__ __device__ constexpr int ws_min_blocks()
{
    constexpr int by_smem = (228 * 1024) / (ws_smem<N, EB>() + 1024);
    constexpr int by_threads = 2048 / (ws_consumers<N, EB>() + 32);
    constexpr int b = by_smem < by_threads ? by_smem : by_threads;
    return b < 1 ? 1 : (b > 4 ? 4 : b);
}
// Bulk copies need whole elements in 16-byte multiples (n even) and room.
template <int N, int EB>
__host__ __device__ constexpr bool ws_ok()
{
    return (N + 1) % 2 == 0 && ws_smem<N, EB>() <= 200 * 1024;
}

// Persistent: block b computes groups b, b + gridDim.x, ...; the last warp
// stages the next group's node map as soon as the consumers have read the
// current one, and its factors as soon as they have applied the current ones,
// so the DRAM reads of group i+1 overlap the computation of group i.
template <int N, int EB>
__global__ void __launch_bounds__(ws_consumers<N, EB>() + 32, (ws_min_blocks<N, EB>()))
    ax_pencil_ws_kernel(const pencil_args A)
{
    if (A.run && *A.run == 0) return;
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1), NC = ws_consumers<N, EB>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bars[4];  // full_l, empty_l, full_g, empty_g
    T *bufs = reinterpret_cast<T *>(smem_raw);
    S *gsm = reinterpret_cast<S *>(smem_raw + ws_off_g<N, EB>());
    int32_t *lsm = reinterpret_cast<int32_t *>(smem_raw + ws_off_l<N, EB>());
    const int64_t ngroups = (A.E + EB - 1) / EB;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], NC / 32);
        mbar_init(&bars[2], 1);
        mbar_init(&bars[3], NC / 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    hbacc::dot_acc<S> acc;
    if (threadIdx.x >= NC) {
        if (threadIdx.x == NC) {  // producer (one lane of the last warp)
            unsigned i = 0;
            for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x, i++) {
                const int64_t e0 = g * EB, cnt = A.E - e0 < EB ? A.E - e0 : EB;
                if (i > 0) mbar_wait(&bars[1], (i - 1) & 1, A.err);
                bulk_g2s(lsm, A.l2g + e0 * n3, (unsigned)(cnt * n3 * 4), &bars[0]);
                if (i > 0) mbar_wait(&bars[3], (i - 1) & 1, A.err);
                bulk_g2s(gsm, A.geo + e0 * 7 * n3, (unsigned)(cnt * 7 * n3 * sizeof(S)), &bars[2]);
            }
            // no copy of this block may still be in flight when it exits (the
            // consumers waited for every one; this matters only after a wait
            // of theirs gave up)
            if (i > 0) {
                mbar_wait(&bars[0], (i - 1) & 1, A.err);
                mbar_wait(&bars[2], (i - 1) & 1, A.err);
            }
        }
        __syncwarp();  // the producer warp reconverges before the block-wide barrier below
    } else {
        unsigned i = 0;
        for (int64_t g = blockIdx.x; g < ngroups; g += gridDim.x, i++) {
            const ws_ctx w{lsm, gsm, &bars[0], &bars[1], &bars[2], &bars[3], i & 1u, A.err};
            pencil_group<N, true, EB, GM_L2G, true>(A, g, bufs, acc, &w);
        }
    }
    if (A.partials) {
        const double v = hbacc::block_sum(acc.value());
        if (threadIdx.x == 0) A.partials[blockIdx.x] = v;
    }
}

}  // namespace
}  // namespace hb2

namespace hb2 {
// Internal linkage: this header is compiled once per precision (T differs by
// translation unit), so nothing in it may share a symbol name across units.
namespace {

// eb_mode: 1 = about 256 threads per block, 2 = twice that many elements
// (N <= 10), 0 = one element per block (spreads small meshes over more SMs),
// 3 = as 1 with a bulk L2 prefetch of the block's geometric factors at the
// start (even-odd only), 4 = the persistent warp-specialised kernel (even-odd,
// odd N, units that define HB_AX2_WS; else as 1). With bit 8 (modes 0 and 1,
// even-odd) surface values go to their CSR positions (A.spos); with bit 16
// (modes 0 and 1, even-odd) every local value goes to A.ysurf element-major.
template <int N, bool EO, int GM = GM_L2G>
hb_status launch(const pencil_args &A, int eb_mode, cudaStream_t s, int64_t *nblocks_out)
{
    constexpr int n = N + 1, n2 = n * n;
    constexpr int EB1 = n2 >= 256 ? 1 : 256 / n2;
    if (A.E <= 0) return HB_OK;
    static int attr_set[9][32] = {{0}};
    int dev = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    const bool sp = (eb_mode & 8) != 0;   // CSR-position surface store
    const bool fl = (eb_mode & 16) != 0;  // element-major store of every local value
    eb_mode &= 7;
    const int which = fl ? (eb_mode == 0 ? 8 : 7)
                      : sp ? (eb_mode == 0 ? 6 : 5)
                           : (eb_mode == 2 && n2 <= 128) ? 1
                                                         : (eb_mode == 0 ? 2 : (eb_mode == 3 ? 3 : (eb_mode == 4 ? 4 : 0)));
    auto go = [&](auto kern, int EB) -> hb_status {
        const size_t smem = sizeof(T) * (GM == GM_L2G ? nbuf<N>() : 4) * (size_t)EB * pad<N>::size;
        if (dev >= 0 && dev < 32 && !attr_set[which][dev]) {
            HB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            attr_set[which][dev] = 1;
        }
        const int64_t blocks = (A.E + EB - 1) / EB;
        if (nblocks_out) *nblocks_out = blocks;
        hb_prof_scope prof("ax_local", s);
        kern<<<(unsigned)blocks, EB * n2, smem, s>>>(A);
        HB_CHECK_LAUNCH();
        return HB_OK;
    };
    if constexpr (GM != GM_L2G) {
        // partitioned and scattered operators: the base block shape only
        return go(ax_pencil_kernel<N, EO, EB1, false, GM>, EB1);
    } else {
        if constexpr (EO) {
            if (which == 6) return go(ax_pencil_kernel<N, EO, 1, false, GM_L2G, true>, 1);
            if (which == 5) return go(ax_pencil_kernel<N, EO, EB1, false, GM_L2G, true>, EB1);
            if (which == 8) return go(ax_pencil_kernel<N, EO, 1, false, GM_L2G, false, true>, 1);
            if (which == 7) return go(ax_pencil_kernel<N, EO, EB1, false, GM_L2G, false, true>, EB1);
        }
        // the double-float unit keeps the block shapes the FP64 autotuner picks
        // in practice (base, one element, and their CSR-store forms); the
        // others run as the base shape there
        constexpr bool kAll = std::is_same<T, S>::value;
        if constexpr (kAll && n2 <= 128) {
            if (which == 1) return go(ax_pencil_kernel<N, EO, EB1 * 2>, EB1 * 2);
        }
        if constexpr (EO && EB1 > 1) {
            if (which == 2) return go(ax_pencil_kernel<N, EO, 1>, 1);
        }
        if constexpr (kAll && EO) {
            if (which == 3) return go(ax_pencil_kernel<N, EO, EB1, true>, EB1);
        }
#ifdef HB_AX2_WS
        if constexpr (EO && ws_ok<N, EB1>()) {
            if (which == 4) {
                // persistent grid: the blocks that fit on every SM at once
                constexpr int smem = ws_smem<N, EB1>();
                auto kern = ax_pencil_ws_kernel<N, EB1>;
                if (dev >= 0 && dev < 32 && !attr_set[4][dev]) {
                    HB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                    attr_set[4][dev] = 1;
                }
                static int grid_of[32] = {0};
                if (dev < 0 || dev >= 32) dev = 0;
                if (!grid_of[dev]) {
                    int per_sm = 0, sms = 0;
                    HB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                                              ws_consumers<N, EB1>() + 32, smem));
                    HB_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
                    grid_of[dev] = (per_sm > 0 ? per_sm : 1) * sms;
                }
                const int64_t ngroups = (A.E + EB1 - 1) / EB1;
                const int64_t blocks = ngroups < grid_of[dev] ? ngroups : grid_of[dev];
                if (nblocks_out) *nblocks_out = blocks;
                hb_prof_scope prof("ax_local", s);
                kern<<<(unsigned)blocks, ws_consumers<N, EB1>() + 32, smem, s>>>(A);
                HB_CHECK_LAUNCH();
                return HB_OK;
            }
        }
#endif
        return go(ax_pencil_kernel<N, EO, EB1>, EB1);
    }
}

}  // namespace
}  // namespace hb2
