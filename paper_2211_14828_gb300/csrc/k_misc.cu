// Sketching matrix generation (Algorithm 1 step 1), norms, precision staging.
#include "kernels.h"
#include "dfloat.cuh"

namespace rbki {
namespace {

// Y[a][s][c] = Omega^(mode)[a*C + c][s]   (FP64; layout of a TTM result so the sketch
// W = X_(n) Omega is the contraction of X with Y).
__global__ void k_omega_f64(uint64_t seed, uint32_t mode, int64_t A, int64_t C, int S,
                            double* __restrict__ Y) {
    const int npair = (S + 1) / 2;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (a, pair, c)
    int64_t total = A * npair * C;
    if (e >= total) return;
    int64_t c = e % C;
    int64_t t = e / C;
    int pair = (int)(t % npair);
    int64_t a = t / npair;
    double z0, z1;
    omega_pair_f64(seed, mode, (uint64_t)(a * C + c), (uint32_t)pair, z0, z1);
    int s = 2 * pair;
    Y[(a * S + s) * C + c] = z0;
    if (s + 1 < S) Y[(a * S + s + 1) * C + c] = z1;
}

template <typename T>
__global__ void k_sumsq(const T* __restrict__ x, int64_t n, double* __restrict__ part) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = ld_f64(x + i);
        acc += v * v;
    }
    __shared__ double red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) *out = v;
    }
}

template <typename TD> __device__ __forceinline__ TD cvt_from_f32(float v);
template <> __device__ __forceinline__ __nv_bfloat16 cvt_from_f32(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __half cvt_from_f32(float v) { return __float2half_rn(v); }

// dst = round(x) in bf16/f16 (RN) + partial sums of squares of the source (FP64)
template <typename T, typename TD>
__global__ void k_stage(const T* __restrict__ x, int64_t n, TD* __restrict__ dst,
                        double* __restrict__ part) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = ld_f64(x + i);
        acc += v * v;
        dst[i] = cvt_from_f32<TD>((float)v);
    }
    __shared__ double red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

// float4-vectorised fp32 -> bf16 staging (the common case), n % 4 == 0, 16-byte aligned.
// The squares of four elements are summed in FP32 and accumulated per thread by compensated
// FP32 summation (TwoSum: the running sum and the sum of its rounding errors, about 2^-48
// relative); the threads' sums are combined in FP64.  An FP64 accumulator here cost two FP64
// operations per 16 bytes read, about as long as the HBM traffic itself on GB300.
__global__ void k_stage_f32_bf16_v4(const float4* __restrict__ x, int64_t n4,
                                    uint2* __restrict__ dst, double* __restrict__ part) {
    float hi = 0.f, lo = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        float4 v = __ldcs(x + i);
        const dfl sq = df_two_sum(hi, v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w);
        hi = sq.hi;
        lo = __fadd_rn(lo, sq.lo);
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
        __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
        uint2 o;
        o.x = *reinterpret_cast<uint32_t*>(&a);
        o.y = *reinterpret_cast<uint32_t*>(&b);
        dst[i] = o;
    }
    double acc = (double)hi + (double)lo;
    __shared__ double red[32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

constexpr int NORM_BLOCKS = 1024;

}  // namespace

rbki_status omega_f64_cuda(uint64_t seed, int mode, int64_t A, int64_t C, int S, double* Y,
                           cudaStream_t st) {
    int64_t total = A * ((S + 1) / 2) * C;
    k_omega_f64<<<(unsigned)cdiv(total, 256), 256, 0, st>>>(seed, (uint32_t)mode, A, C, S, Y);
    RBKI_LAUNCH_CHECK("k_omega_f64");
    return RBKI_OK;
}

rbki_status sumsq_cuda(const void* x, int dtype, int64_t n, double* part, double* out,
                       cudaStream_t st) {
    int blocks = (int)std::min<int64_t>(NORM_BLOCKS, std::max<int64_t>(1, cdiv(n, 256)));
    switch (dtype) {
        case RBKI_F64: k_sumsq<<<blocks, 256, 0, st>>>((const double*)x, n, part); break;
        case RBKI_F32: k_sumsq<<<blocks, 256, 0, st>>>((const float*)x, n, part); break;
        case RBKI_BF16: k_sumsq<<<blocks, 256, 0, st>>>((const __nv_bfloat16*)x, n, part); break;
        case RBKI_F16: k_sumsq<<<blocks, 256, 0, st>>>((const __half*)x, n, part); break;
        default: return set_error(RBKI_E_INVAL, "sumsq dtype");
    }
    RBKI_LAUNCH_CHECK("k_sumsq");
    k_sum_parts<<<1, 256, 0, st>>>(part, blocks, out);
    RBKI_LAUNCH_CHECK("k_sum_parts");
    return RBKI_OK;
}

rbki_status sum_parts_cuda(const double* part, int nparts, double* out, cudaStream_t st) {
    k_sum_parts<<<1, 256, 0, st>>>(part, nparts, out);
    RBKI_LAUNCH_CHECK("k_sum_parts");
    return RBKI_OK;
}

rbki_status stage_cuda(const void* x, int dtype, int64_t n, void* dst, int dst_dtype,
                       double* part, double* norm2, cudaStream_t st) {
    int blocks = (int)std::min<int64_t>(NORM_BLOCKS, std::max<int64_t>(1, cdiv(n, 256)));
    if (dtype == RBKI_F32 && dst_dtype == RBKI_BF16 && n % 4 == 0 &&
        ((uintptr_t)x % 16) == 0 && ((uintptr_t)dst % 8) == 0) {
        k_stage_f32_bf16_v4<<<blocks, 256, 0, st>>>((const float4*)x, n / 4, (uint2*)dst, part);
    } else {
#define STG(T)                                                                              \
    if (dst_dtype == RBKI_BF16) k_stage<T, __nv_bfloat16><<<blocks, 256, 0, st>>>(           \
        (const T*)x, n, (__nv_bfloat16*)dst, part);                                          \
    else k_stage<T, __half><<<blocks, 256, 0, st>>>((const T*)x, n, (__half*)dst, part);
        switch (dtype) {
            case RBKI_F64: STG(double); break;
            case RBKI_F32: STG(float); break;
            case RBKI_BF16: STG(__nv_bfloat16); break;
            case RBKI_F16: STG(__half); break;
            default: return set_error(RBKI_E_INVAL, "stage dtype");
        }
#undef STG
    }
    RBKI_LAUNCH_CHECK("k_stage");
    k_sum_parts<<<1, 256, 0, st>>>(part, blocks, norm2);
    RBKI_LAUNCH_CHECK("k_sum_parts");
    return RBKI_OK;
}

}  // namespace rbki
