// Dot-product accumulators shared by the operator and the vector kernels.
#pragma once

namespace hbacc {

// FP64 accumulation of products. For FP32 operands the FP64 pipe of GB300 is
// slow, so the running sum is carried as an unevaluated pair of floats with
// error-free transformations (Dekker's two-product via fma, Knuth's two-sum):
// about 48 significant bits, the accuracy of an FP64 sum of these products.
template <typename T>
struct dot_acc;

template <>
struct dot_acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct dot_acc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float a, float b)
    {
        float p = a * b;
        float pe = fmaf(a, b, -p);
        float t = hi + p;
        float bp = t - hi;
        float err = (hi - (t - bp)) + (p - bp);
        hi = t;
        lo += err + pe;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Block-wide FP64 sum in a fixed order (warp shuffles, then warp 0); the
// result is valid in thread 0. Every thread of the block must call it.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

}  // namespace hbacc
