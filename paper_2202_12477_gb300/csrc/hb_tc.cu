// Tensor-core (tcgen05) pieces of the library: a self-check of the operand
// layouts the tensor-core element kernel relies on.
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>

#include "hb_internal.h"
#include "hb_tc.cuh"
#include "hb_acc.cuh"

namespace {

constexpr unsigned long long kTcWaitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long tc_wall_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for phase `parity` of an mbarrier: about a second of wall
// time, then bit 0 of *err and return false.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity, unsigned *err)
{
    const unsigned a = hbtc::smem_addr(bar);
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
        if (done) return true;
        if ((t & 255u) == 0) {
            const unsigned long long now = tc_wall_ns();
            if (t == 0) t0 = now;
            else if (now - t0 > kTcWaitNs) break;
        }
    }
    atomicOr(err, 1u);
    return false;
}

// Self-check tile: D (128 x 48, FP32) = A (128 x 48) B^T (B: 48 x 48), FP16
// inputs, three K steps of 16. A is staged K-major (mode bit 0 clear) or
// MN-major (set), with the MN core-matrix stride 128 bytes and the K one
// 2048; B is staged K-major (N stride 128, K stride 768). Mode bit 1 swaps
// the leading and stride byte-offset fields of both descriptors (to tell the
// two conventions apart; both stay inside the zeroed staging area).
constexpr int kSelfA = 0, kSelfB = 65536, kSelfBar = 81920, kSelfSmem = 81920 + 64;

__global__ void __launch_bounds__(128) tc_selftest_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                          float *__restrict__ D, int mode, unsigned *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kSelfBar);
    unsigned *tptr = reinterpret_cast<unsigned *>(sm + kSelfBar + 8);
    const bool a_mn = (mode & 1) != 0, swap = (mode & 2) != 0;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    for (int i = tid; i < kSelfBar / 16; i += 128) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    for (int idx = tid; idx < 128 * 48; idx += 128) {
        const int mn = idx / 48, k = idx % 48;
        const int off = a_mn ? (mn % 8) * 2 + (k % 8) * 16 + (mn / 8) * 128 + (k / 8) * 2048
                             : (mn % 8) * 16 + (k % 8) * 2 + (mn / 8) * 128 + (k / 8) * 2048;
        *reinterpret_cast<__half *>(sm + kSelfA + off) = __float2half_rn(A[idx]);
    }
    for (int idx = tid; idx < 48 * 48; idx += 128) {
        const int nn = idx / 48, k = idx % 48;
        const int off = (nn % 8) * 16 + (k % 8) * 2 + (nn / 8) * 128 + (k / 8) * 768;
        *reinterpret_cast<__half *>(sm + kSelfB + off) = __float2half_rn(B[idx]);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(hbtc::smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    hbtc::fence_async_smem();
    __syncthreads();
    if (warp == 0) hbtc::tmem_alloc(tptr, 64);
    hbtc::fence_before_sync();
    __syncthreads();
    hbtc::fence_after_sync();
    const unsigned tmem = *tptr;
    if (tid == 0) {
        unsigned a_lbo = a_mn ? 128u : 2048u, a_sbo = a_mn ? 2048u : 128u;
        unsigned b_lbo = 768u, b_sbo = 128u;
        if (swap) {
            const unsigned t1 = a_lbo; a_lbo = a_sbo; a_sbo = t1;
            const unsigned t2 = b_lbo; b_lbo = b_sbo; b_sbo = t2;
        }
        const unsigned a0 = hbtc::smem_addr(sm + kSelfA), b0 = hbtc::smem_addr(sm + kSelfB);
        const uint32_t idesc = hbtc::idesc_f16(128, 48, a_mn, false);
        for (int ks = 0; ks < 3; ks++)
            hbtc::mma_f16(tmem, hbtc::smem_desc(a0 + ks * 2 * 2048, a_lbo, a_sbo),
                          hbtc::smem_desc(b0 + ks * 2 * 768, b_lbo, b_sbo), idesc, ks > 0);
        hbtc::mma_commit(bar);
    }
    tc_wait(bar, 0, err);
    hbtc::fence_after_sync();
    for (int c = 0; c < 48; c += 16) {
        uint32_t v[16];
        hbtc::tmem_ld16(tmem + ((unsigned)(32 * warp) << 16) + c, v);
        hbtc::tmem_wait_ld(v);
#pragma unroll
        for (int q = 0; q < 16; q++) D[(32 * warp + lane) * 48 + c + q] = __uint_as_float(v[q]);
    }
    hbtc::fence_before_sync();
    __syncthreads();
    if (warp == 0) hbtc::tmem_free(tmem, 64);
}

}  // namespace

extern "C" hb_status hb_tc_selftest(int mode, const float *A_host, const float *B_host, float *D_host,
                                    hb_status *status)
{
    hb_clear_error();
    if (!A_host || !B_host || !D_host || !status || mode < 0 || mode > 3) {
        hb_set_error("hb_tc_selftest: bad argument");
        return HB_ERR_ARG;
    }
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    unsigned *derr = nullptr;
    cudaError_t e = cudaMalloc(&dA, sizeof(float) * 128 * 48);
    if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(float) * 48 * 48);
    if (e == cudaSuccess) e = cudaMalloc(&dD, sizeof(float) * 128 * 48);
    if (e == cudaSuccess) e = cudaMalloc(&derr, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(dA, A_host, sizeof(float) * 128 * 48, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B_host, sizeof(float) * 48 * 48, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(derr, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(dD, 0xFF, sizeof(float) * 128 * 48);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSelfSmem);
    if (e == cudaSuccess) {
        hb_count_launch();
        tc_selftest_kernel<<<1, 128, kSelfSmem>>>(dA, dB, dD, mode, derr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(D_host, dD, sizeof(float) * 128 * 48, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(derr);
    if (e != cudaSuccess) {
        hb_set_error("hb_tc_selftest: %s", cudaGetErrorString(e));
        return HB_ERR_CUDA;
    }
    *status = herr ? HB_ERR_TIMEOUT : HB_OK;
    return HB_OK;
}

// ---------------------------------------------------------------- tensor-core FP64 element kernel
//
// y_L = S_L Z x (Sec. 2, Eq. stiffness) for N = 7 with every derivative
// contraction (D along r, s, t and D^T along r, s, t; 12 n^4 of the
// 12 n^4 + 15 n^3 flops of an element) on the tensor cores, exactly, and the
// metric step (the 6 geometric factors, 15 n^3 flops) in FP64 on the CUDA
// cores.
//
// Exact contractions from FP16 products (an Ozaki-style split into slices):
//   - the element's values u are put on one fixed-point grid,
//     X = round(u / 2^E) with 2^E the unit of the element's largest exponent
//     (|X| < 2^53: the rounding is below the last bit of the largest value),
//     and written as seven base-256 digits, X = sum_j u_j 256^(6-j), u_0
//     signed (|u_0| <= 32), u_1..u_6 unsigned bytes;
//   - D is scaled to integers D_int = round(D 2^s) (|D_int| < 2^55) and written
//     as seven balanced digits b_d in [-128, 128];
//   - digit products are integers below 2^16 and every sum the tensor core
//     forms stays below 2^24, so FP16 inputs with FP32 accumulation add them
//     without rounding. For each diagonal t = j + d <= 7 the MMA forms
//     S_t = sum_{j+d=t} sum_m b_d[i][m] u_j[m] in its own accumulator
//     column; D u = 2^(E-s) sum_t 256^(12-t) S_t up to the dropped diagonals
//     t >= 8, which weigh below 2^-58 of the largest term;
//   - a digit enters the MMA as the FP16 number 256 + u_j (384 + u_0), whose
//     bit pattern is 0x5C00 | (u_j << 2): no conversion instruction. The
//     offsets contribute a constant per accumulator column, removed inside the
//     same MMA by an eighth K block: 128 in the A operand times the constant's
//     negative / 128 (split into FP16-exact parts) in the B operand;
//   - the exact integers S_t are read back (FP32 -> int32 by adding 1.5 2^23),
//     combined in two int64 halves and turned into doubles with the exponent
//     of the element's grid (exact), summed with one FP64 add.
// Per two-element tile (128 lines per direction, M = 128) and direction: one
// MMA chain of four K = 16 steps, A = the lines' digits (128 x 64, K-major,
// K ordered (line position m, digit j) so that one node's seven digits and the
// offset-correction slot j = 7 are one 16-byte row piece), B = the digit
// stack of D (64 x 64: output index i x diagonal t by the same K), accumulator
// 128 x 64 FP32 in TMEM (r and s in columns 0..127, then t in 0..63).
namespace {
namespace tcax {

constexpr int N = 7, n = 8, n2 = 64, n3 = 512;
constexpr int NS = 2 * n2 + 4 * N * (N - 1);  // surface nodes of an element
constexpr int THREADS = 256;                  // two threads per line of a two-element tile
constexpr int KH = 4;                         // nodes of its line a thread owns (half of n)
// One direction's A operand: 8 K chunks (m) of 128 rows x 8 FP16 (16 bytes);
// rows 16 bytes apart, row chunks of 8 at 128 bytes, K chunks LBO apart. The
// r operand's K chunks sit 2064 bytes apart (16 bytes more than a chunk), so
// the eight threads of a store phase, which differ in m, hit different banks.
constexpr int LBO_R = 2064, LBO_ST = 2048;
constexpr int ABUF = 7 * LBO_R + 2048 + 112;  // 16,608 bytes, a multiple of 16
constexpr int BIMG = 64 * 64 * 2;             // one B operand image (64 x 64 FP16)
constexpr int EXS = 576;                      // padded node stride of an element in the exchange buffers
constexpr int OFF_A = 0;
constexpr int OFF_B = OFF_A + 3 * ABUF;
constexpr int OFF_MISC = OFF_B + 2 * BIMG;
constexpr int SMEM = OFF_MISC + 64;  // 66,272 bytes: three blocks per SM
// The exchange buffers (two doubles or two int64 halves per node of the
// tile) sit in the r and s operands, whose MMAs have completed by then.
static_assert(4 * EXS * 8 <= 2 * ABUF, "exchange buffers fit in the r and s operands");
// r and s accumulate in columns 0..127, then t in columns 0..63
constexpr unsigned TMEM_COLS = 128;

// B operand images of D (0) and D^T (1) in the shared-memory layout (K-major,
// N chunk stride 128 bytes, K chunk stride 1024), and s (D_int = D 2^s).
__device__ __align__(16) uint16_t g_tc_bimg[2][64 * 64];
__constant__ int c_tc_dshift;

struct tc_args {
    const double *x;
    const int32_t *l2g;
    const double *geo;
    double *ysurf;
    double *y;
    int64_t E;
    const int *run;
    double lambda;
    int screen;
    double *partials;
    unsigned *err;
    const int32_t *spos;  // SP kernels: CSR position of every surface copy (-1 masked)
};

// node (i, j, k) of element el in the padded exchange buffers
__device__ __forceinline__ int xq(int el, int i, int j, int k) { return el * EXS + k * 72 + j * 9 + i; }

__device__ __forceinline__ unsigned exp_bits(double v)
{
    return (unsigned)(__double_as_longlong(v) >> 52) & 0x7FFu;
}

// v on the grid of unit 2^(emax - 1075): round(|v| / unit) with the sign of v
// (|result| < 2^53; zero and subnormal v give 0). Integer instructions only:
// 64-bit conversions run at the FP64 rate on this GPU.
__device__ __forceinline__ long long to_fixed(double v, unsigned emax)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned e = (unsigned)(b >> 52) & 0x7FFu;
    // 2m with the implicit bit (m the 53-bit significand), 0 for zero and subnormals
    const unsigned long long m2 = e ? ((b << 1) & 0x1FFFFFFFFFFFFEull) | (1ull << 53) : 0ull;
    const unsigned sh = min(emax - e, 62u);
    // round(m / 2^sh), halves up: (floor(2m / 2^sh) + 1) / 2
    const long long X = (long long)(((m2 >> sh) + 1ull) >> 1);
    return (b >> 63) ? -X : X;
}

// T 2^off as a double, rounded to nearest (ties away from zero) from the
// integer T (any int64): normalise |T| so its top bit is bit 63, keep 53 bits,
// round on the 11 below, and let a carry out of the mantissa step into the
// exponent. Results below the normal range flush to zero, above it give
// infinity.
__device__ __forceinline__ double i64_to_double(long long T, int off)
{
    if (T == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)T & 0x8000000000000000ull;
    unsigned long long M = T < 0 ? 0ull - (unsigned long long)T : (unsigned long long)T;
    const int lz = __clzll((long long)M);
    M <<= lz;
    const unsigned long long mant = (M >> 11) + ((M >> 10) & 1ull);  // 2^52 .. 2^53
    const int ex = 1023 + 63 - lz + off;
    if (ex <= 0) return __longlong_as_double((long long)sgn);
    if (ex >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
    return __longlong_as_double((long long)(sgn | (((unsigned long long)(ex - 1) << 52) + mant)));
}

// 2^off (2^32 hi + lo) as a double: exactly as one int64 while that fits
// (|hi| < 2^30), else from its value / 2^10 rounded down (the dropped bits
// are below 2^-53 of a value of at least 2^63).
__device__ __forceinline__ double halves_to_double(long long hi, long long lo, int off)
{
    const bool small = (unsigned long long)(hi + (1ll << 30)) < (1ull << 31);
    const int sh = small ? 0 : 10;
    const long long T = (long long)((unsigned long long)hi << (32 - sh)) + (lo >> sh);
    return i64_to_double(T, off + sh);
}

// The A-operand row piece of one node: the FP16 bit patterns of the seven
// digits of X (digit j is byte 6 - j of the little-endian 64-bit word; byte 6
// is the signed leading digit u_0) as the MMA takes them -- digit u as the FP16
// number 256 + u (384 + u_0 for j = 0), pattern 0x5C00 | (u << 2) -- and the
// offset-correction slot, FP16 128.0 (0x5800).
__device__ __forceinline__ uint4 row_piece(long long X)
{
    const unsigned lo = (unsigned)X, hi = (unsigned)((unsigned long long)X >> 32);
    uint4 r;
    // __byte_perm(a, b, s): result byte n is byte (nibble n of s) of b:a; the
    // zero word supplies the empty bytes
    r.x = ((__byte_perm(hi, 0u, 0x4142u) ^ 0x00000080u) << 2) | 0x5C005C00u;           // u_0 + 128, u_1
    r.y = ((__byte_perm(lo, hi, 0x0304u) & 0x00FF00FFu) << 2) | 0x5C005C00u;           // u_2, u_3
    r.z = (__byte_perm(lo, 0u, 0x4142u) << 2) | 0x5C005C00u;                          // u_4, u_5
    r.w = ((lo & 0xFFu) << 2) | 0x58005C00u;                                          // u_6, 128.0
    return r;
}

// Stores the row pieces of the thread's nodes (ti, tj, k0 + q) in the A
// operands of the directions in `dirs` (bit 0 r, bit 1 s, bit 2 t):
//   r: row (el, k, j), K chunk m = i;  s: row (el, k, i), m = j;  t: row (el, j, i), m = k.
__device__ __forceinline__ void stage(unsigned char *Ab, int el, int ti, int tj, int k0, const long long (&X)[KH],
                                      int dirs)
{
#pragma unroll
    for (int q = 0; q < KH; q++) {
        const int k = k0 + q;
        const uint4 p = row_piece(X[q]);
        if (dirs & 1) *reinterpret_cast<uint4 *>(Ab + 0 * ABUF + ti * LBO_R + (el * 8 + k) * 128 + tj * 16) = p;
        if (dirs & 2) *reinterpret_cast<uint4 *>(Ab + 1 * ABUF + tj * LBO_ST + (el * 8 + k) * 128 + ti * 16) = p;
        if (dirs & 4) *reinterpret_cast<uint4 *>(Ab + 2 * ABUF + k * LBO_ST + (el * 8 + tj) * 128 + ti * 16) = p;
    }
}

// The r and s chains (accumulator columns 0..63 and 64..127) and, once every
// thread has read those, the t chain (columns 0..63). K step ks covers the K
// chunks m = 2 ks, 2 ks + 1 of A and B.
__device__ __forceinline__ void issue_rs(unsigned tmem, const unsigned char *Ab, const unsigned char *Bi)
{
    constexpr uint32_t idesc = hbtc::idesc_f16(128, 64, false, false);
    const unsigned b0 = hbtc::smem_addr(Bi);
#pragma unroll
    for (int dir = 0; dir < 2; dir++) {
        const unsigned a0 = hbtc::smem_addr(Ab + dir * ABUF);
        const unsigned lbo = dir == 0 ? LBO_R : LBO_ST;
#pragma unroll
        for (int ks = 0; ks < 4; ks++)
            hbtc::mma_f16(tmem + dir * 64, hbtc::smem_desc(a0 + ks * 2 * lbo, lbo, 128),
                          hbtc::smem_desc(b0 + ks * 2048, 1024, 128), idesc, ks > 0);
    }
}

__device__ __forceinline__ void issue_t(unsigned tmem, const unsigned char *Ab, const unsigned char *Bi)
{
    constexpr uint32_t idesc = hbtc::idesc_f16(128, 64, false, false);
    const unsigned b0 = hbtc::smem_addr(Bi);
    const unsigned a0 = hbtc::smem_addr(Ab + 2 * ABUF);
#pragma unroll
    for (int ks = 0; ks < 4; ks++)
        hbtc::mma_f16(tmem, hbtc::smem_desc(a0 + ks * 2 * LBO_ST, LBO_ST, 128),
                      hbtc::smem_desc(b0 + ks * 2048, 1024, 128), idesc, ks > 0);
}

// Completion of the chain in flight: warp 0 polls the barrier (bounded), the
// block meets at a barrier, which takes no issue slots.
__device__ __forceinline__ void mma_done(uint64_t *bar, unsigned &phase, int warp, unsigned *err, int &gave_up)
{
    if (warp == 0 && !tc_wait(bar, phase, err)) gave_up = 1;
    phase ^= 1u;
    __syncthreads();
    hbtc::fence_after_sync();
}

// The exact diagonal sums of output o of a 16-column chunk (diagonals 0..7)
// as the halves hi = sum_{t<4} S_t 256^(3-t), lo = sum_{t>=4} S_t 256^(7-t):
// the output is 2^72 hi + 2^40 lo in units of the element's grid times 2^-s.
// Each S_t is an integer below 2^22 in magnitude, read exactly from its float
// f as bits(f + 1.5 2^23) - 0x4B400000.
__device__ __forceinline__ void combine(const uint32_t (&v)[16], int o, long long &hi, long long &lo)
{
    // two accumulators per packed FP32 add (add.rn.f32x2): the same
    // round-to-nearest sums as one add each, half the instructions
    unsigned B[8];
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
        unsigned long long pa, pr;
        asm("mov.b64 %0, {%1, %2};" : "=l"(pa) : "r"(v[o * 8 + t]), "r"(v[o * 8 + t + 1]));
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(pr) : "l"(pa), "l"(0x4B4000004B400000ull));
        asm("mov.b64 {%0, %1}, %2;" : "=r"(B[t]), "=r"(B[t + 1]) : "l"(pr));
    }
    // S_a 256 + S_b fits an int32: form it modulo 2^32 from the raw bits
    constexpr unsigned kBias = 0x4B400000u * 257u;
    const int m0 = (int)((unsigned)B[0] * 256u + (unsigned)B[1] - kBias);
    const int m1 = (int)((unsigned)B[2] * 256u + (unsigned)B[3] - kBias);
    const int m2 = (int)((unsigned)B[4] * 256u + (unsigned)B[5] - kBias);
    const int m3 = (int)((unsigned)B[6] * 256u + (unsigned)B[7] - kBias);
    hi = (long long)m0 * 65536 + m1;
    lo = (long long)m2 * 65536 + m3;
}

__device__ __forceinline__ int ring_index7(int i, int j)
{
    return j == 0 ? i : (j == N ? N + 1 + i : 2 * (N + 1) + 2 * (j - 1) + (i == N ? 1 : 0));
}

// Largest biased exponent over element el (warps 0, 1, 4, 5 hold element 0,
// warps 2, 3, 6, 7 element 1). Every thread calls it; it synchronises.
__device__ __forceinline__ unsigned element_max(unsigned v, unsigned *wexp, int el)
{
    v = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) wexp[threadIdx.x >> 5] = v;
    __syncthreads();
    return max(max(wexp[2 * el], wexp[2 * el + 1]), max(wexp[4 + 2 * el], wexp[5 + 2 * el]));
}

// Thread tid: line tau = tid % 128 of the tile (TMEM lane tau; element
// el = tau / 64; t-line (ti, tj) = (tau % 8, tau / 8 % 8)) and half h = tid / 128:
// nodes k = 4h .. 4h + 3 of its t-line, outputs 4h .. 4h + 3 of its r-, s-
// and t-line rows. Per tile and phase (D, then D^T): stage the three operands,
// run the r and s chains, read them out (gradients to the exchange buffers in
// the r/s operands, or the exact sums of D^T along r and s), run the t chain
// into the same columns, read it out. The six metric factors are prefetched
// into L2 at the tile's start and loaded at the metric step, not held in
// registers: with 80 registers, 66 KB of shared memory and 128 TMEM columns a
// block, three blocks fit on an SM (two held 124 registers, 85 KB and 256
// columns each: 14% slower, the same bits).
template <bool SP>
__global__ void __launch_bounds__(THREADS, 3) ax_tc_kernel(const tc_args A)
{
    if (A.run && *A.run == 0) return;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tau = tid & 127, h = tid >> 7, k0 = KH * h;
    const int el = tau >> 6, a = tau & 63, ti = a & 7, tj = a >> 3;
    unsigned char *Ab = sm + OFF_A;
    unsigned char *Bi = sm + OFF_B;
    double *ExR = reinterpret_cast<double *>(sm + OFF_A);  // in the r/s operands once their MMAs are done
    double *ExS = ExR + 2 * EXS;
    long long *Yhi = reinterpret_cast<long long *>(ExR);
    long long *Ylo = reinterpret_cast<long long *>(ExS);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + OFF_MISC);
    unsigned *tptr = reinterpret_cast<unsigned *>(sm + OFF_MISC + 8);
    unsigned *wexp = reinterpret_cast<unsigned *>(sm + OFF_MISC + 16);

    for (int q = tid; q < 2 * BIMG / 16; q += THREADS)
        reinterpret_cast<uint4 *>(Bi)[q] = reinterpret_cast<const uint4 *>(&g_tc_bimg[0][0])[q];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(hbtc::smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) hbtc::tmem_alloc(tptr, TMEM_COLS);
    hbtc::fence_async_smem();
    hbtc::fence_before_sync();
    __syncthreads();
    hbtc::fence_after_sync();
    const unsigned tmem = *tptr;
    const int dshift = c_tc_dshift;
    const unsigned tl = tmem + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)(32 * h);

    hbacc::dot_acc<double> acc;
    unsigned phase = 0;
    int gave_up = 0;
    const int64_t ntiles = (A.E + 1) / 2;
    int gid_n[KH];
    double u_n[KH];
    auto gather = [&](int64_t gg) {
        const int64_t ee = 2 * gg + el;
        const bool act = gg < ntiles && ee < A.E;
        const int32_t *lg = A.l2g + ee * n3 + a;
#pragma unroll
        for (int q = 0; q < KH; q++) gid_n[q] = act ? __ldcs(lg + (k0 + q) * n2) : -1;
#pragma unroll
        for (int q = 0; q < KH; q++) u_n[q] = gid_n[q] >= 0 ? __ldg(A.x + gid_n[q]) : 0.0;
    };
    gather(blockIdx.x);
    for (int64_t g = blockIdx.x; g < ntiles; g += gridDim.x) {
        const int64_t e = 2 * g + el;
        const bool active = e < A.E;
        int gid[KH];
        double u[KH];
#pragma unroll
        for (int q = 0; q < KH; q++) {
            gid[q] = gid_n[q];
            u[q] = u_n[q];
        }
        {
            // the tile's six metric factors into L2 now (the first 6 n^2 values
            // of each element's k-slab of 7 n^2; J w only if screening reads
            // it): 24 lines of 128 bytes per slab, read at the metric step
            const int64_t e0 = 2 * g;
            const int nel = e0 + 1 < A.E ? 2 : 1;
            constexpr int kLines = 6 * n2 * 8 / 128;
            for (int L = tid; L < nel * n * kLines; L += THREADS) {
                const int eo = L / (n * kLines), k = (L / kLines) % n, line = L % kLines;
                const double *p = A.geo + (e0 + eo) * 7 * n3 + k * 7 * n2 + line * 16;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
            }
        }
        unsigned em = 0;
#pragma unroll
        for (int q = 0; q < KH; q++) em = max(em, exp_bits(u[q]));
        const unsigned eu = element_max(em, wexp, el);
        {
            long long X[KH];
#pragma unroll
            for (int q = 0; q < KH; q++) X[q] = eu == 0x7FFu ? 0 : to_fixed(u[q], eu);
            stage(Ab, el, ti, tj, k0, X, 7);
        }
        hbtc::fence_async_smem();
        hbtc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            hbtc::fence_after_sync();
            issue_rs(tmem, Ab, Bi);
            hbtc::mma_commit(bar);
        }
        mma_done(bar, phase, warp, A.err, gave_up);
        const int goff = (int)eu - 1075 - dshift + 40;
        const bool ubad = eu == 0x7FFu;
        // ---- gradients along r and s into the exchange buffers
#pragma unroll
        for (int dir = 0; dir < 2; dir++) {
            uint32_t vv[2][16];
            hbtc::tmem_ld16(tl + dir * 64, vv[0]);
            hbtc::tmem_ld16(tl + dir * 64 + 16, vv[1]);
            hbtc::tmem_wait_ld(vv[0]);
            hbtc::tmem_wait_ld(vv[1]);
#pragma unroll
            for (int c = 0; c < 2; c++) {
#pragma unroll
                for (int o = 0; o < 2; o++) {
                    long long hi, lo;
                    combine(vv[c], o, hi, lo);
                    const double gv = ubad ? __longlong_as_double(0x7FF8000000000000ll) : halves_to_double(hi, lo, goff);
                    const int out = k0 + 2 * c + o;
                    if (dir == 0) ExR[xq(el, out, tau & 7, (tau >> 3) & 7)] = gv;
                    else ExS[xq(el, tau & 7, out, (tau >> 3) & 7)] = gv;
                }
            }
        }
        // every thread has read columns 0..127: the t chain may reuse them
        hbtc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            hbtc::fence_after_sync();
            issue_t(tmem, Ab, Bi);
            hbtc::mma_commit(bar);
        }
        mma_done(bar, phase, warp, A.err, gave_up);
        double gt[KH];
        {
            uint32_t vv[2][16];
            hbtc::tmem_ld16(tl, vv[0]);
            hbtc::tmem_ld16(tl + 16, vv[1]);
            hbtc::tmem_wait_ld(vv[0]);
            hbtc::tmem_wait_ld(vv[1]);
#pragma unroll
            for (int c = 0; c < 2; c++)
#pragma unroll
                for (int o = 0; o < 2; o++) {
                    long long hi, lo;
                    combine(vv[c], o, hi, lo);
                    gt[2 * c + o] = ubad ? __longlong_as_double(0x7FF8000000000000ll) : halves_to_double(hi, lo, goff);
                }
        }
        // ---- metric (FP64): v = G grad at the thread's nodes, factors loaded here
        double vr[KH], vs[KH], vt[KH];
        unsigned evm = 0;
        {
            const double *ge = A.geo + e * 7 * n3 + a;
#pragma unroll
            for (int q = 0; q < KH; q++) {
                double G[6];
#pragma unroll
                for (int c = 0; c < 6; c++) G[c] = active ? __ldcs(ge + (k0 + q) * 7 * n2 + c * n2) : 0.0;
                const int xi = xq(el, ti, tj, k0 + q);
                const double ur = ExR[xi], us = ExS[xi], ut = gt[q];
                vr[q] = fma(G[2], ut, fma(G[1], us, G[0] * ur));
                vs[q] = fma(G[4], ut, fma(G[3], us, G[1] * ur));
                vt[q] = fma(G[5], ut, fma(G[4], us, G[2] * ur));
                evm = max(evm, max(exp_bits(vr[q]), max(exp_bits(vs[q]), exp_bits(vt[q]))));
            }
        }
        // (element_max meets the block: every exchange read is done before
        // the operands are staged over the exchange buffers)
        const unsigned ev = element_max(evm, wexp, el);
        {
            long long X[KH];
#pragma unroll
            for (int q = 0; q < KH; q++) X[q] = ev == 0x7FFu ? 0 : to_fixed(vr[q], ev);
            stage(Ab, el, ti, tj, k0, X, 1);
#pragma unroll
            for (int q = 0; q < KH; q++) X[q] = ev == 0x7FFu ? 0 : to_fixed(vs[q], ev);
            stage(Ab, el, ti, tj, k0, X, 2);
#pragma unroll
            for (int q = 0; q < KH; q++) X[q] = ev == 0x7FFu ? 0 : to_fixed(vt[q], ev);
            stage(Ab, el, ti, tj, k0, X, 4);
        }
        hbtc::fence_async_smem();
        hbtc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            hbtc::fence_after_sync();
            issue_rs(tmem, Ab, Bi + BIMG);
            hbtc::mma_commit(bar);
        }
        gather(g + gridDim.x);
        mma_done(bar, phase, warp, A.err, gave_up);
        // ---- D^T along r and s summed exactly into the exchange buffers
#pragma unroll
        for (int dir = 0; dir < 2; dir++) {
            uint32_t vv[2][16];
            hbtc::tmem_ld16(tl + dir * 64, vv[0]);
            hbtc::tmem_ld16(tl + dir * 64 + 16, vv[1]);
            hbtc::tmem_wait_ld(vv[0]);
            hbtc::tmem_wait_ld(vv[1]);
#pragma unroll
            for (int c = 0; c < 2; c++) {
#pragma unroll
                for (int o = 0; o < 2; o++) {
                    long long hi, lo;
                    combine(vv[c], o, hi, lo);
                    const int out = k0 + 2 * c + o;
                    if (dir == 0) {
                        const int q = xq(el, out, tau & 7, (tau >> 3) & 7);
                        Yhi[q] = hi;
                        Ylo[q] = lo;
                    } else {
                        const int q = xq(el, tau & 7, out, (tau >> 3) & 7);
                        Yhi[q] += hi;
                        Ylo[q] += lo;
                    }
                }
            }
            if (dir == 0) __syncthreads();
        }
        hbtc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            hbtc::fence_after_sync();
            issue_t(tmem, Ab, Bi + BIMG);
            hbtc::mma_commit(bar);
        }
        mma_done(bar, phase, warp, A.err, gave_up);
        {
            const int yoff = (int)ev - 1075 - dshift + 40;
            const bool vbad = ev == 0x7FFu;
            double *ys = A.ysurf + e * NS;
            const bool ring = ti == 0 || ti == N || tj == 0 || tj == N;
            const int r = ring ? ring_index7(ti, tj) : 0;
            uint32_t vv[2][16];
            hbtc::tmem_ld16(tl, vv[0]);
            hbtc::tmem_ld16(tl + 16, vv[1]);
            hbtc::tmem_wait_ld(vv[0]);
            hbtc::tmem_wait_ld(vv[1]);
#pragma unroll
            for (int c = 0; c < 2; c++) {
#pragma unroll
                for (int o = 0; o < 2; o++) {
                    long long hi, lo;
                    combine(vv[c], o, hi, lo);
                    const int qq = 2 * c + o, k = k0 + qq;
                    const int xi = xq(el, ti, tj, k);
                    hi += Yhi[xi];
                    lo += Ylo[xi];
                    const double yc = vbad ? __longlong_as_double(0x7FF8000000000000ll) : halves_to_double(hi, lo, yoff);
                    if (!active) continue;
                    if (SP && (k == 0 || k == N || ring)) {
                        const int sidx = k == 0 ? a : (k == N ? n2 + a : 2 * n2 + (k - 1) * 4 * N + r);
                        const int pos = __ldg(A.spos + e * NS + sidx);
                        if (pos >= 0) A.ysurf[pos] = yc;
                    } else if (k == 0) {
                        ys[a] = yc;
                    } else if (k == N) {
                        ys[n2 + a] = yc;
                    } else if (ring) {
                        ys[2 * n2 + (k - 1) * 4 * N + r] = yc;
                    } else {
                        const double xv = u[qq];
                        const double jw = A.screen ? __ldg(A.geo + (e * n + k) * 7 * n2 + 6 * n2 + a) : 1.0;
                        double yy = yc;
                        yy += A.lambda * (jw * xv);
                        A.y[gid[qq]] = yy;
                        acc.add(xv, yy);
                    }
                }
            }
        }
        // the next tile stages over the exchange buffers read above
        hbtc::fence_before_sync();
        if (__syncthreads_or(gave_up)) break;
    }
    if (A.partials) {
        const double v = hbacc::block_sum(acc.value());
        if (tid == 0) A.partials[blockIdx.x] = v;
    }
    if (__syncthreads_or(gave_up)) {
        if (tid == 0) tc_wait(bar, phase ^ 1u, A.err);
        __syncthreads();
    }
    hbtc::fence_before_sync();
    __syncthreads();
    hbtc::fence_after_sync();
    if (warp == 0) hbtc::tmem_free(tmem, TMEM_COLS);
}

// ---- host: B images and launch

// FP16 bit pattern of an integer that FP16 holds exactly.
static uint16_t fp16_exact(long long v)
{
    if (v == 0) return 0;
    const uint16_t sgn = v < 0 ? 0x8000 : 0;
    unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
    int e = 63 - __builtin_clzll(a);
    const unsigned long long f = e >= 10 ? (a >> (e - 10)) : (a << (10 - e));
    return (uint16_t)(sgn | (uint16_t)((e + 15) << 10) | (uint16_t)(f & 0x3FF));
}

// Largest part of c (toward zero) that FP16 holds exactly: its top 11 bits.
static long long fp16_part(long long c)
{
    const unsigned long long a = (unsigned long long)(c < 0 ? -c : c);
    const int e = 63 - __builtin_clzll(a);
    const unsigned long long p = e > 10 ? (a >> (e - 10)) << (e - 10) : a;
    return c < 0 ? -(long long)p : (long long)p;
}

}  // namespace tcax
}  // namespace

// Builds the B images from the degree-7 derivative matrix and uploads them to
// the current device (once per device, from hb_ensure_device_tables).
hb_status hb_tc_upload()
{
    using namespace tcax;
    double xi[n], w[n], D[n * n];
    hb_reference_element(N, xi, w, D);
    double mx = 0.0;
    for (int q = 0; q < n * n; q++) mx = std::fmax(mx, std::fabs(D[q]));
    const int s = 55 - (std::ilogb(mx) + 1);
    static uint16_t img[2][64 * 64];
    for (int tr = 0; tr < 2; tr++) {
        int b[7][n][n];  // digit d of D_int[i][m] (D^T for tr = 1), weight 256^(6-d)
        for (int i = 0; i < n; i++)
            for (int m = 0; m < n; m++) {
                const double v = tr ? D[m * n + i] : D[i * n + m];
                long long q = std::llround(std::ldexp(v, s));
                for (int d = 6; d >= 1; d--) {
                    const long long r = ((q + 128) & 255) - 128;
                    b[d][i][m] = (int)r;
                    q = (q - r) >> 8;
                }
                if (q < -128 || q > 128) {
                    hb_set_error("tensor-core split: leading digit %lld out of range", q);
                    return HB_ERR_ARG;
                }
                b[0][i][m] = (int)q;
            }
        uint16_t *im = img[tr];
        std::memset(im, 0, sizeof img[0]);
        // element (row (i, t), K (m, digit j)) at i * 128 + t * 16 + m * 1024 + j * 2
        auto put = [&](int i, int t, int j, int m, long long val) {
            im[(i * 128 + t * 16 + m * 1024 + j * 2) / 2] = fp16_exact(val);
        };
        for (int i = 0; i < n; i++)
            for (int t = 0; t < 8; t++) {
                long long beta = 0;  // what the digit offsets add to column (i, t)
                for (int j = 0; j < 7; j++) {
                    const int d = t - j;
                    if (d < 0 || d > 6) continue;
                    long long rs = 0;
                    for (int m = 0; m < n; m++) {
                        put(i, t, j, m, b[d][i][m]);
                        rs += b[d][i][m];
                    }
                    beta += (j == 0 ? 384 : 256) * rs;
                }
                // slot j = 7 of each K chunk: 128 (A side) times parts summing to -beta / 128
                long long c = -beta / 128;
                for (int m = 0; m < n && c != 0; m++) {
                    const long long p = fp16_part(c);
                    put(i, t, 7, m, p);
                    c -= p;
                }
                if (c != 0) {
                    hb_set_error("tensor-core split: offset correction does not fit");
                    return HB_ERR_ARG;
                }
            }
    }
    HB_TRY_CUDA(cudaMemcpyToSymbol(g_tc_bimg, img, sizeof img));
    HB_TRY_CUDA(cudaMemcpyToSymbol(c_tc_dshift, &s, sizeof s));
    return HB_OK;
}

// Tensor-core FP64 element kernel (N = 7): interior DOFs finished here (y,
// lambda term, partial of x.y per block), surface values to ysurf for the
// surface gather. Persistent grid: three blocks per SM at most.
hb_status hb_launch_ax_tc_f64(const hb_mesh *m, const double *x, double *ysurf, double *y, double lambda,
                              int screen, double *partials, const int *run, bool csr_store, cudaStream_t s,
                              int64_t *nblocks)
{
    using namespace tcax;
    if (m->N != N) { hb_set_error("the tensor-core element kernel is built for N = 7 only"); return HB_ERR_ARG; }
    if (!m->geo) { hb_set_error("mesh has no double geometric factors"); return HB_ERR_ARG; }
    if (m->E <= 0) return HB_OK;
    int dev = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    static int attr_set[64] = {0}, sms[64] = {0};
    if (dev < 0 || dev >= 64) { hb_set_error("device index %d unsupported", dev); return HB_ERR_ARG; }
    if (csr_store && !m->spos) { hb_set_error("surface positions missing"); return HB_ERR_ARG; }
    if (!attr_set[dev]) {
        HB_TRY_CUDA(cudaFuncSetAttribute(ax_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        HB_TRY_CUDA(cudaFuncSetAttribute(ax_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        HB_TRY_CUDA(cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev));
        attr_set[dev] = 1;
    }
    const int64_t ntiles = (m->E + 1) / 2;
    const int64_t grid = ntiles < 3 * (int64_t)sms[dev] ? ntiles : 3 * (int64_t)sms[dev];
    if (nblocks) *nblocks = grid;
    tc_args A{x, m->l2g, m->geo, ysurf, y, m->E, run, lambda, screen, partials, m->counters + 7,
              csr_store ? m->spos : nullptr};
    hb_prof_scope prof("ax_local", s);
    if (csr_store) ax_tc_kernel<true><<<(unsigned)grid, THREADS, SMEM, s>>>(A);
    else ax_tc_kernel<false><<<(unsigned)grid, THREADS, SMEM, s>>>(A);
    HB_CHECK_LAUNCH();
    return HB_OK;
}
