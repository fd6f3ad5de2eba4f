// Double-float arithmetic: a value is an unevaluated sum h + l of two floats
// with |l| <= ulp(h)/2 (after normalisation), about 47 significant bits
// through the operations below. Built from error-free transformations:
// Knuth's two-sum and the fma form of Dekker's two-product (see e.g.
// Muller et al., Handbook of Floating-Point Arithmetic, ch. 4 and 14).
// On GB300 every operation runs on the FP32 pipes, which issue 64 times the
// FP64 rate.
#pragma once

#include <cstdint>

struct df {
    float h, l;
    df() = default;
    __host__ __device__ constexpr df(float a) : h(a), l(0.0f) {}
    __host__ __device__ constexpr df(float a, float b) : h(a), l(b) {}
};

// a + b = s + err exactly (no condition on the magnitudes).
__device__ __forceinline__ float df_two_sum(float a, float b, float &err)
{
    const float s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
    return s;
}

__device__ __forceinline__ df df_norm(float s, float t)
{
    const float h = s + t;
    return df(h, t - (h - s));
}

__device__ __forceinline__ df operator+(const df &a, const df &b)
{
    float e;
    const float s = df_two_sum(a.h, b.h, e);
    return df_norm(s, e + (a.l + b.l));
}

__device__ __forceinline__ df operator-(const df &a) { return df(-a.h, -a.l); }

__device__ __forceinline__ df operator-(const df &a, const df &b) { return a + (-b); }

__device__ __forceinline__ df &operator+=(df &a, const df &b)
{
    a = a + b;
    return a;
}

// a * b: exact product of the high parts plus the two cross terms.
__device__ __forceinline__ df operator*(const df &a, const df &b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_norm(p, e);
}

// c + a * b for accumulation chains: the result is left unnormalised (its
// low part collects the rounding errors of the chain); every store
// normalises. The high part of the sum stays exact through two-sum.
__device__ __forceinline__ df fma(const df &a, const df &b, const df &c)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    float err;
    const float s = df_two_sum(c.h, p, err);
    return df(s, c.l + (e + err));
}

// double -> (h, l) by taking the bit fields apart: h holds the top 24 bits
// of the significand (truncated), l the next 23, so |x - (h + l)| < 2^-46 |x|.
// Integer and FP32 instructions only (no FP64 conversion anywhere, so the
// FP64 pipe stays free): magnitudes below 2^-126 become a signed zero and
// magnitudes at or above 2^128 (and infinities, NaN) a signed infinity; l is
// dropped where it would fall below the FP32 normal range (|x| < 2^-103,
// where the split keeps 24 bits).
__device__ __forceinline__ df df_from_double(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const int ef = e - 896;  // float biased exponent
    const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned hbits = ef <= 0 ? sign : (ef >= 255 ? (sign | 0x7F800000u) : (sign | ((unsigned)ef << 23) | m23));
    // the remaining 29 significand bits, top 23 of them as a float in [0,1)
    const float f1 = __uint_as_float(0x3F800000u | ((lo & 0x1FFFFFFFu) >> 6)) - 1.0f;
    const int es = e - 919;  // 2^(e - 1046) as a float exponent
    const float scale = (es > 0 && ef > 0 && ef < 255) ? __uint_as_float((unsigned)es << 23) : 0.0f;
    const float l = f1 * scale;
    return df(__uint_as_float(hbits), sign ? -l : l);
}

// float -> double exactly, by bit fields (zero and subnormals give 0).
__device__ __forceinline__ double df_float_to_double(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    const unsigned lo = (u & 0x7u) << 29;
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double df_to_double(const df &a)
{
    return df_float_to_double(a.h) + df_float_to_double(a.l);
}
