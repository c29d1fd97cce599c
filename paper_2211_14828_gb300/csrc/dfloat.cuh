// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits (Dekker, "A floating-point technique for
// extending the available precision", Numer. Math. 18, 1971; the error-free transformations
// TwoSum (Knuth, TAOCP vol. 2) and TwoProd by fused multiply-add).  Every operation runs on
// the FP32 pipes with FP32 latency: GB300 retires 2 FP64 operations per clock per SM and a
// dependent FP64 instruction waits tens of cycles, so short serial chains of small-matrix
// arithmetic (a Cholesky step, a pivot's reciprocal) run several times faster this way.
// The explicit round-to-nearest intrinsics keep the compiler from contracting or
// reassociating the error terms.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace rbki {

// Round-to-nearest FP32 operations that the compiler may not contract or reassociate: the
// device intrinsics, and on the host (the CPU tests of this header) the plain operators,
// compiled there with -ffp-contract=off.
#if defined(__CUDA_ARCH__)
#define DF_ADD(a, b) __fadd_rn(a, b)
#define DF_SUB(a, b) __fsub_rn(a, b)
#define DF_MUL(a, b) __fmul_rn(a, b)
#define DF_FMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_FMA(a, b, c) fmaf(a, b, c)
#endif
#define DF_FN __host__ __device__ __forceinline__

struct dfl {
    float hi, lo;
};

DF_FN dfl df_make(float hi, float lo) { return dfl{hi, lo}; }

// s + e == a + b exactly (no ordering assumption)
DF_FN dfl df_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    const float bb = DF_SUB(s, a);
    const float e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
    return dfl{s, e};
}

// s + e == a + b exactly, for |a| >= |b| (or a == 0)
DF_FN dfl df_quick_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    return dfl{s, DF_SUB(b, DF_SUB(s, a))};
}

DF_FN dfl df_add(dfl x, dfl y) {
    dfl s = df_two_sum(x.hi, y.hi);
    const float e = DF_ADD(s.lo, DF_ADD(x.lo, y.lo));
    return df_quick_two_sum(s.hi, e);
}

DF_FN dfl df_neg(dfl x) { return dfl{-x.hi, -x.lo}; }

DF_FN dfl df_mul(dfl x, dfl y) {
    const float p = DF_MUL(x.hi, y.hi);
    float e = DF_FMA(x.hi, y.hi, -p);                          // TwoProd: p + e == x.hi y.hi
    e = DF_FMA(x.hi, y.lo, DF_FMA(x.lo, y.hi, e));
    return df_quick_two_sum(p, e);
}

// w - x y
DF_FN dfl df_fms(dfl w, dfl x, dfl y) { return df_add(w, df_neg(df_mul(x, y))); }

DF_FN bool df_gt(dfl x, dfl y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }

// 1 / d for d > 0: the hardware's approximate FP32 reciprocal (rcp.approx, about 1 ulp)
// refined by one Newton step in double-float (relative error about 2^-46)
DF_FN float rcp_approx(float x) {
#if defined(__CUDA_ARCH__)
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#else
    return 1.0f / x;
#endif
}
DF_FN float rsqrt_approx(float x) {
#if defined(__CUDA_ARCH__)
    return rsqrtf(x);
#else
    return 1.0f / sqrtf(x);
#endif
}
DF_FN dfl df_rcp(dfl d) {
    const float y0 = rcp_approx(d.hi);
    const dfl r = df_add(dfl{1.f, 0.f}, df_neg(df_mul(d, dfl{y0, 0.f})));   // 1 - d y0
    return df_add(dfl{y0, 0.f}, df_mul(dfl{y0, 0.f}, r));
}

// 1 / sqrt(d) for d > 0: the FP32 estimate refined by two Newton steps in double-float,
// y <- y + y (1 - d y^2) / 2 (relative error about 2^-22 -> 2^-44 -> the double-float limit)
DF_FN dfl df_rsqrt(dfl d) {
    dfl y{rsqrt_approx(d.hi), 0.f};
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const dfl r = df_add(dfl{1.f, 0.f}, df_neg(df_mul(d, df_mul(y, y))));   // 1 - d y^2
        y = df_add(y, df_mul(dfl{DF_MUL(0.5f, y.hi), DF_MUL(0.5f, y.lo)}, r));
    }
    return y;
}

// FP64 <-> double-float (the caller keeps x within FP32's range)
DF_FN dfl df_from_double(double x) {
    const float hi = (float)x;
    return dfl{hi, (float)(x - (double)hi)};
}
DF_FN double df_to_double(dfl x) { return (double)x.hi + (double)x.lo; }

}  // namespace rbki
