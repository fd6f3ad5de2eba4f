// Element-local part of the screened Poisson operator,
//   y_L = S_L Z x,  S_L^e = Dbold^T G^e Dbold   (hipBone Sec. 2, Sec. 3.2),
// fused with the gather Z x from assembled storage.
//
// Thread layout: a block holds EB elements; each element gets (N+1)^2 threads
// and thread (i,j) owns the t-pencil of nodes (i, j, 0..N):
//   1. gathers u(i,j,k) = x[l2g] for its pencil (coalesced l2g loads), keeps
//      the pencil in registers and copies it to shared memory;
//   2. forms u_t in registers (the pencil is contiguous along t), u_r and u_s
//      from shared memory, applies the six metric factors, keeps v_t in
//      registers and writes v_r, v_s to shared memory;
//   3. forms D^T contractions of v_r, v_s (shared) and v_t (registers) and
//      writes y_L for its pencil.
// Geometric factors are streamed once (layout [e][k][7][(N+1)^2], so a slab of
// one k is contiguous and each factor is a coalesced row of (N+1)^2 values).
#pragma once

#include "hb_internal.h"

namespace hb {

template <int N>
struct ax_shape {
    static constexpr int n = N + 1;
    static constexpr int n2 = n * n;
    static constexpr int n3 = n2 * n;
    // elements per block: about 256 threads
    static constexpr int EB = n2 >= 256 ? 1 : 256 / n2;
    static constexpr int threads = EB * n2;
    static constexpr int dpad = (n2 + 3) & ~3;
};

template <typename T>
__device__ __forceinline__ T ldg_stream(const T *p)
{
    return __ldcs(p);
}

template <int N, typename T, int EB>
__global__ void __launch_bounds__(EB *(N + 1) * (N + 1))
    ax_local_kernel(const T *__restrict__ x, const int32_t *__restrict__ l2g, const T *__restrict__ geo,
                    T *__restrict__ yL, int64_t E, const T *__restrict__ Dg, const int *__restrict__ run)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr int dpad = (n2 + 3) & ~3;
    if (run && *run == 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sD = reinterpret_cast<T *>(smem_raw);
    T *su = sD + dpad;
    T *svr = su + EB * n3;
    T *svs = svr + EB * n3;

    const int tid = threadIdx.x;
    const int el = tid / n2;
    const int ij = tid - el * n2;
    const int i = ij % n, j = ij / n;
    const int64_t e = (int64_t)blockIdx.x * EB + el;
    const bool active = e < E;

    for (int q = tid; q < n2; q += EB * n2) sD[q] = Dg[q];
    T *U = su + el * n3;
    T *VR = svr + el * n3;
    T *VS = svs + el * n3;

    T w[n];
    if (active) {
        const int32_t *lg = l2g + e * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; k++) {
            const int g = ldg_stream(lg + k * n2);
            const T v = g >= 0 ? __ldg(x + g) : T(0);
            w[k] = v;
            U[k * n2 + ij] = v;
        }
    }
    __syncthreads();
    if (active) {
        T ut[n];
#pragma unroll
        for (int k = 0; k < n; k++) {
            T a = T(0);
#pragma unroll
            for (int m = 0; m < n; m++) a += sD[k * n + m] * w[m];
            ut[k] = a;
        }
        const T *ge = geo + e * 7 * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; k++) {
            T ur = T(0), us = T(0);
#pragma unroll
            for (int m = 0; m < n; m++) {
                ur += sD[i * n + m] * U[k * n2 + j * n + m];
                us += sD[j * n + m] * U[k * n2 + m * n + i];
            }
            const T *g = ge + k * 7 * n2;
            const T grr = ldg_stream(g), grs = ldg_stream(g + n2), grt = ldg_stream(g + 2 * n2);
            const T gss = ldg_stream(g + 3 * n2), gst = ldg_stream(g + 4 * n2), gtt = ldg_stream(g + 5 * n2);
            VR[k * n2 + ij] = grr * ur + grs * us + grt * ut[k];
            VS[k * n2 + ij] = grs * ur + gss * us + gst * ut[k];
            w[k] = grt * ur + gst * us + gtt * ut[k];
        }
    }
    __syncthreads();
    if (active) {
        T *ye = yL + e * n3 + ij;
#pragma unroll
        for (int k = 0; k < n; k++) {
            T a = T(0);
#pragma unroll
            for (int m = 0; m < n; m++) {
                a += sD[m * n + i] * VR[k * n2 + j * n + m];
                a += sD[m * n + j] * VS[k * n2 + m * n + i];
                a += sD[m * n + k] * w[m];
            }
            ye[k * n2] = a;
        }
    }
}

template <int N, typename T>
hb_status launch_ax_local(const T *x, const int32_t *l2g, const T *geo, T *yL, int64_t E, const T *Dg,
                          const int *run, cudaStream_t s)
{
    using S = ax_shape<N>;
    if (E <= 0) return HB_OK;
    const size_t smem = sizeof(T) * (S::dpad + 3 * S::EB * S::n3);
    static int attr_set[32] = {0};
    int dev = 0;
    HB_TRY_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 32 && !attr_set[dev]) {
        HB_TRY_CUDA(cudaFuncSetAttribute(ax_local_kernel<N, T, S::EB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set[dev] = 1;
    }
    const int64_t blocks = (E + S::EB - 1) / S::EB;
    hb_prof_scope prof("ax_local", s);
    ax_local_kernel<N, T, S::EB><<<(unsigned)blocks, S::threads, smem, s>>>(x, l2g, geo, yL, E, Dg, run);
    HB_CHECK_LAUNCH();
    return HB_OK;
}

}  // namespace hb
