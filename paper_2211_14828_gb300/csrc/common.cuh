// Shared device/host helpers for librbki (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>
#include <algorithm>

#include "../../include/rbki.h"

namespace rbki {

// launch accounting (rbki_kernel_launches) and error capture
void note_launch();
void add_launches(uint64_t n);    // kernels launched through a CUDA graph replay
void drop_launches(uint64_t n);   // kernels recorded by a stream capture (not launched)
rbki_status set_cuda_error(cudaError_t e, const char* where);
rbki_status set_error(rbki_status s, const char* msg);

#define RBKI_LAUNCH_CHECK(where)                                             \
    do {                                                                     \
        ::rbki::note_launch();                                               \
        cudaError_t e_ = cudaGetLastError();                                 \
        if (e_ != cudaSuccess) return ::rbki::set_cuda_error(e_, where);     \
    } while (0)

#define RBKI_CUDA_TRY(call)                                                  \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ::rbki::set_cuda_error(e_, #call);     \
    } while (0)

#define RBKI_TRY(call)                                                       \
    do {                                                                     \
        rbki_status s_ = (call);                                             \
        if (s_ < 0) return s_;                                               \
    } while (0)

__host__ __device__ static inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ static inline int64_t rup(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// ---- element loads of the streamed tensor (any storage dtype) ----
template <typename T> __device__ __forceinline__ double ld_f64(const T* p);
template <> __device__ __forceinline__ double ld_f64<double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ double ld_f64<float>(const float* p) { return (double)__ldg(p); }
template <> __device__ __forceinline__ double ld_f64<__nv_bfloat16>(const __nv_bfloat16* p) {
    return (double)__bfloat162float(*p);
}
template <> __device__ __forceinline__ double ld_f64<__half>(const __half* p) {
    return (double)__half2float(*p);
}

template <typename T> __device__ __forceinline__ float ld_f32(const T* p);
template <> __device__ __forceinline__ float ld_f32<double>(const double* p) { return (float)__ldg(p); }
template <> __device__ __forceinline__ float ld_f32<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld_f32<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}
template <> __device__ __forceinline__ float ld_f32<__half>(const __half* p) { return __half2float(*p); }

// load converted straight to the accumulation type: FP32 paths never touch the FP64 pipe
// (a float <-> double conversion has 64-100 cycles of latency and FP64 throughput on GB300)
template <typename Acc> struct LdAcc;
template <> struct LdAcc<float> {
    template <typename T> __device__ __forceinline__ static float ld(const T* p) { return ld_f32(p); }
};
template <> struct LdAcc<double> {
    template <typename T> __device__ __forceinline__ static double ld(const T* p) { return ld_f64(p); }
};
template <typename Acc, typename T> __device__ __forceinline__ Acc ld_acc(const T* p) { return LdAcc<Acc>::ld(p); }

// ---- Philox4x32-10 (Salmon et al., SC'11) and the Box-Muller Gaussian of Omega ----
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        U4 o;
        o.x = hi1 ^ c.y ^ k0;
        o.y = lo1;
        o.z = hi0 ^ c.w ^ k1;
        o.w = lo0;
        c = o;
    }
    return c;
}

// Omega^(mode)[col, 2*pair] and [col, 2*pair+1] in FP64.
__device__ __forceinline__ void omega_pair_f64(uint64_t seed, uint32_t mode, uint64_t col,
                                               uint32_t pair, double& z0, double& z1) {
    U4 c{pair, mode, (uint32_t)(col & 0xffffffffu), (uint32_t)(col >> 32)};
    U4 r = philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    double u1 = ((double)(r.x >> 5) * 67108864.0 + (double)(r.y >> 6) + 1.0) * 0x1p-53;
    double u2 = ((double)(r.z >> 5) * 67108864.0 + (double)(r.w >> 6)) * 0x1p-53;
    double rho = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    z0 = rho * co;
    z1 = rho * s;
}

// Single-precision evaluation of the same Gaussian (used to feed BF16/FP16 operands): the
// two 53-bit uniforms are formed in FP32 directly (high word scaled by 2^-27 plus the low
// word by 2^-53), so the image generation never touches the FP64 pipe.
__device__ __forceinline__ void omega_pair_f32(uint64_t seed, uint32_t mode, uint64_t col,
                                               uint32_t pair, float& z0, float& z1) {
    U4 c{pair, mode, (uint32_t)(col & 0xffffffffu), (uint32_t)(col >> 32)};
    U4 r = philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const float u1 = fmaf((float)(r.x >> 5), 0x1p-27f, (float)((r.y >> 6) + 1u) * 0x1p-53f);
    const float u2 = fmaf((float)(r.z >> 5), 0x1p-27f, (float)(r.w >> 6) * 0x1p-53f);
    float rho = sqrtf(-2.0f * logf(u1));
    float s, co;
    sincospif(2.0f * u2, &s, &co);
    z0 = rho * co;
    z1 = rho * s;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace rbki
