// Tensor-core (tcgen05) pieces of the library: a self-check of the operand
// layouts the tensor-core element kernel relies on.
#include <cuda_fp16.h>

#include "hb_internal.h"
#include "hb_tc.cuh"

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
