// Hardware probes used to calibrate the roofline (hipBone, arXiv 2202.12477,
// Sec. 4.1: the empirical streaming rate B of an 8-read / 1-write kernel).
//
// HB_PROBE_STREAM81_FP   each thread reads 8 values and writes their sum (the
//                        paper's calibration kernel; in FP64 on GB300 the 7
//                        adds per output cost more than the memory traffic)
// HB_PROBE_STREAM81_BITS the same traffic, combining the 8 words with XOR
//                        (integer pipe): the memory rate alone
// HB_PROBE_COPY          16-byte vector copy (read + write bytes)
// HB_PROBE_FMA           independent FMA chains: the arithmetic peak
#include <vector>

#include "hb_internal.h"

namespace {

template <typename T>
__global__ void probe_stream81_fp(const T *__restrict__ in, T *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T s = in[i];
#pragma unroll
        for (int q = 1; q < 8; q++) s += in[i + q * n];
        out[i] = s;
    }
}

template <typename U>
__global__ void probe_stream81_bits(const U *__restrict__ in, U *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        U s = in[i];
#pragma unroll
        for (int q = 1; q < 8; q++) s ^= in[i + q * n];
        out[i] = s;
    }
}

__global__ void probe_copy(const double2 *__restrict__ in, double2 *__restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

template <typename T>
__global__ void probe_fma(T *out, int iters, T b, T c)
{
    T a[8];
#pragma unroll
    for (int q = 0; q < 8; q++) a[q] = (T)(threadIdx.x + q) * (T)1e-7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int q = 0; q < 8; q++) a[q] = fma(a[q], b, c);
    }
    T s = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 warp-level matrix multiply-accumulate (mma.sync m8n8k4, 512 flops per
// warp and instruction): four independent accumulator tiles per warp.
// With `with_fma`, every thread also runs four independent FP64 FMA chains
// in the same loop, to see whether the two paths share one pipe.
template <bool with_fma>
__global__ void probe_dmma(double *out, int iters)
{
    const double a = 1e-7 * (threadIdx.x + 1), b = 0.9999999;
    double c[4][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    double f[4] = {a, 2 * a, 3 * a, 4 * a};
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int q = 0; q < 4; q++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[q][0]), "+d"(c[q][1])
                         : "d"(a), "d"(b));
        if (with_fma) {
#pragma unroll
            for (int q = 0; q < 4; q++) f[q] = fma(f[q], b, 1e-9);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) s += c[q][0] + c[q][1] + f[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 64-bit conversions: eight independent chains of int64 -> FP64 -> int64
// (cvt.rn.f64.s64, cvt.rni.s64.f64), two conversions and one integer add per
// step: which unit runs them decides whether they compete with FP64 FMAs.
__global__ void probe_cvt64(double *out, int iters)
{
    long long a[8];
#pragma unroll
    for (int q = 0; q < 8; q++) a[q] = (long long)threadIdx.x * 977 + q;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int q = 0; q < 8; q++) a[q] = __double2ll_rn(__ll2double_rn(a[q])) + 3;
    }
    long long s = 0;
#pragma unroll
    for (int q = 0; q < 8; q++) s += a[q];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

}  // namespace

extern "C" hb_status hb_probe(int kind, hb_precision prec, size_t bytes, int reps, double *rate)
{
    hb_clear_error();
    if (!rate || reps < 1 || (prec != HB_F64 && prec != HB_F32)) { hb_set_error("bad argument"); return HB_ERR_ARG; }
    int dev = 0, sms = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    HB_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 16, threads = 256;
    const size_t esz = prec == HB_F64 ? 8 : 4;
    void *buf = nullptr;
    size_t alloc = bytes;
    if (kind == HB_PROBE_FMA || kind == HB_PROBE_DMMA || kind == HB_PROBE_DMMA_FMA || kind == HB_PROBE_CVT64)
        alloc = (size_t)grid * threads * 8;
    if (alloc < 4096) alloc = 4096;
    HB_TRY_CUDA(cudaMalloc(&buf, alloc));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaMemset(buf, 0, alloc);
    double work = 0.0;  // bytes or flops per launch
    auto launch = [&]() {
        if (kind == HB_PROBE_STREAM81_FP || kind == HB_PROBE_STREAM81_BITS) {
            const int64_t n = (int64_t)(alloc / (9 * esz));
            work = 9.0 * n * esz;
            if (kind == HB_PROBE_STREAM81_FP) {
                if (prec == HB_F64)
                    probe_stream81_fp<double><<<grid, threads>>>((const double *)buf, (double *)buf + 8 * n, n);
                else
                    probe_stream81_fp<float><<<grid, threads>>>((const float *)buf, (float *)buf + 8 * n, n);
            } else {
                if (prec == HB_F64)
                    probe_stream81_bits<unsigned long long><<<grid, threads>>>(
                        (const unsigned long long *)buf, (unsigned long long *)buf + 8 * n, n);
                else
                    probe_stream81_bits<unsigned><<<grid, threads>>>((const unsigned *)buf, (unsigned *)buf + 8 * n,
                                                                   n);
            }
        } else if (kind == HB_PROBE_COPY) {
            const int64_t n = (int64_t)(alloc / 32);  // double2 elements in each half
            work = 2.0 * n * 16;
            probe_copy<<<grid, threads>>>((const double2 *)buf, (double2 *)buf + n, n);
        } else if (kind == HB_PROBE_DMMA || kind == HB_PROBE_DMMA_FMA) {
            const int iters = 2048;
            const double warps = (double)grid * threads / 32;
            // counted: the matrix flops (4 x 512 per warp and iteration), plus
            // with FMA the 4 x 2 flops per thread and iteration
            work = warps * iters * 4 * 512.0 + (kind == HB_PROBE_DMMA_FMA ? 8.0 * iters * (double)grid * threads : 0.0);
            if (kind == HB_PROBE_DMMA)
                probe_dmma<false><<<grid, threads>>>((double *)buf, iters);
            else
                probe_dmma<true><<<grid, threads>>>((double *)buf, iters);
        } else if (kind == HB_PROBE_CVT64) {
            const int iters = 1024;
            work = 2.0 * 8 * iters * (double)grid * threads;  // conversions
            probe_cvt64<<<grid, threads>>>((double *)buf, iters);
        } else {
            const int iters = 4096;
            work = 2.0 * 8 * iters * (double)grid * threads;
            if (prec == HB_F64)
                probe_fma<double><<<grid, threads>>>((double *)buf, iters, 0.9999999, 1e-9);
            else
                probe_fma<float><<<grid, threads>>>((float *)buf, iters, 0.9999999f, 1e-9f);
        }
        hb_count_launch();
    };
    float best = 1e30f;
    if (kind < HB_PROBE_STREAM81_FP || kind > HB_PROBE_CVT64) {
        hb_set_error("unknown probe kind %d", kind);
        e = cudaErrorInvalidValue;
    }
    for (int r = 0; r < reps + 1 && e == cudaSuccess; r++) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;  // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) {
        if (!hb_last_error()[0]) hb_set_error("probe: %s", cudaGetErrorString(e));
        return e == cudaErrorInvalidValue ? HB_ERR_ARG : HB_ERR_CUDA;
    }
    *rate = work / (best * 1e-3) / 1e9;  // GB/s or GFLOP/s
    return HB_OK;
}

extern "C" hb_status hb_selftest_wait(int which, hb_status *status, void *stream)
{
    hb_clear_error();
    if (!status) { hb_set_error("null argument"); return HB_ERR_ARG; }
    if (which != 0 && which != 1) { hb_set_error("which must be 0 or 1"); return HB_ERR_ARG; }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned *d = nullptr;  // [0..1] barrier words, [3] error word
    HB_TRY_CUDA(cudaMalloc((void **)&d, 4 * sizeof(unsigned)));
    cudaError_t e = cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), s);
    hb_status r = HB_OK;
    if (e == cudaSuccess) r = which == 0 ? hb_selftest_mbar_timeout(d + 3, s) : hb_selftest_barrier_timeout(d, d + 3, s);
    unsigned v = 0;
    if (e == cudaSuccess && r == HB_OK) e = cudaMemcpyAsync(&v, d + 3, sizeof v, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && r == HB_OK) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (r != HB_OK) return r;
    if (e != cudaSuccess) {
        hb_set_error("self-test: %s", cudaGetErrorString(e));
        return HB_ERR_CUDA;
    }
    *status = (v & (which == 0 ? 1u : 2u)) ? HB_ERR_TIMEOUT : HB_OK;
    return HB_OK;
}
