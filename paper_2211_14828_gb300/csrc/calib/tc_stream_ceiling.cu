// Streaming ceiling of the tensor-core Krylov-step pattern on this GPU (calibration for the
// roofline of k_stream_tc; not part of librbki.so).
//
// A persistent kernel (one CTA per SM) streams a 512^3 BF16 tensor with the same TMA pattern
// as k_stream_tc (64 x 128 boxes, 128-byte swizzle, 32 KB slabs in a ring of mbarrier-guarded
// slots).  Its consumer either releases each slab at once, or first issues tcgen05.mma
// (kind::f16, M x N x 16) reading the slab and commits the slab's release to their
// completion.  Three sweeps:
//   1. release at once, ring depth 2..5 slabs          -> copy ceiling of the access pattern
//   2. 8, 16, 24, 32 MMAs per slab (M = 128, N = 32)   -> cost of one MMA
//   3. 16 MMAs per slab, M in {128, 64}, N 16..256     -> dependence of that cost on M and N
// The Krylov step issues 16 MMAs per 32 KB slab (8 for X^T Q, 8 for X Y), so sweep 2 at 16
// gives its ceiling.  Every wait is bounded; every TMA coordinate lies inside the tensor.
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o tc_ceiling \
//        paper_2211_14828_gb300/csrc/calib/tc_stream_ceiling.cu && ./tc_ceiling
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

namespace {

constexpr uint32_t WAIT_LIMIT = 1u << 26;
constexpr int SLAB = 32768;      // two 64 x 128 BF16 boxes
constexpr int BIMG = 32768;      // B operand region (zeros)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t c) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(c) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t b) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t ph, volatile int* abort_flag) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(ok) : "r"(a), "r"(ph) : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}
__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap* m, uint32_t bar, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
                 ::"r"(dst), "l"(m), "r"(bar), "r"(c0), "r"(c1), "r"(c2) : "memory");
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)layout << 61);
}
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    // D = F32, A = B = BF16, both MN-major
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// tiles: (a, 128-column block) x all I rows in 128-row slabs of 32 KB
__global__ void __launch_bounds__(64, 1) k_ceiling(const __grid_constant__ CUtensorMap tmap, int A, int I, int C,
                                                   int nslot, int nmma, int M, int N, int* err) {
    extern __shared__ __align__(1024) uint8_t raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    const uint32_t base = smem_u32(sm), bimg = base + nslot * SLAB;
    uint64_t* bars = (uint64_t*)(sm + nslot * SLAB + BIMG);
    const uint32_t b_full = smem_u32(bars), b_empty = b_full + 8 * nslot;
    volatile int* abort_flag = (volatile int*)(bars + 2 * nslot);
    uint32_t* tslot = (uint32_t*)(bars + 2 * nslot + 1);
    for (int t = threadIdx.x; t < BIMG / 4; t += blockDim.x) ((uint32_t*)(sm + nslot * SLAB))[t] = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (nmma && threadIdx.x >= 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(256) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < nslot; ++i) {
            mbar_init(b_full + 8 * i, 1);
            mbar_init(b_empty + 8 * i, 1);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int ctiles = C / 128, NS = I / 128;
    const long tiles = (long)A * ctiles;
    const long my = (tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    if (threadIdx.x == 0) {
        uint32_t slot = 0, ph = 0;
        for (long k = 0; k < my && !*abort_flag; ++k) {
            const long t = blockIdx.x + k * gridDim.x;
            const int a = (int)(t / ctiles), cc = (int)(t % ctiles) * 128;
            for (int s = 0; s < NS; ++s) {
                if (!mbar_wait(b_empty + 8 * slot, ph ^ 1, abort_flag)) break;
                mbar_expect_tx(b_full + 8 * slot, SLAB);
                tma3(base + slot * SLAB, &tmap, b_full + 8 * slot, cc, 128 * s, a);
                tma3(base + slot * SLAB + 16384u, &tmap, b_full + 8 * slot, cc + 64, 128 * s, a);
                if (++slot == (uint32_t)nslot) { slot = 0; ph ^= 1; }
            }
        }
    } else if (threadIdx.x == 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tbase = nmma ? *tslot : 0;
        const uint32_t id = idesc_bf16(M, N);
        const uint32_t blbo = (uint32_t)(N / 8) * 128u;
        uint32_t slot = 0, ph = 0;
        for (long k = 0; k < my; ++k)
            for (int s = 0; s < NS; ++s) {
                if (!mbar_wait(b_full + 8 * slot, ph, abort_flag)) { k = my; break; }
                if (nmma) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t xs = base + slot * SLAB;
                    for (int kk = 0; kk < nmma; ++kk) {
                        // A: 16 rows x M columns of the slab (MN-major, swizzled); B: zeros
                        const uint64_t ad = sdesc(xs + (kk & 7) * 2048, 16384, 1024, 2);
                        const uint64_t bd = sdesc(bimg + (uint32_t)(kk & 1) * 2u * blbo, blbo, 128, 0);
                        const uint32_t acc = (s | kk) != 0 ? 1u : 0u;
                        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                                     ::"r"(tbase), "l"(ad), "l"(bd), "r"(id), "r"(acc) : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 ::"r"(b_empty + 8 * slot) : "memory");
                } else {
                    mbar_arrive(b_empty + 8 * slot);
                }
                if (++slot == (uint32_t)nslot) { slot = 0; ph ^= 1; }
            }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (nmma && threadIdx.x >= 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tslot), "r"(256) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(err, 1);
}

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

constexpr int A_ = 512, I_ = 512, C_ = 512;
constexpr size_t BYTES = (size_t)A_ * I_ * C_ * 2;

int run(const CUtensorMap& map, int nslot, int nmma, int M, int N, int* err, float* us) {
    const size_t smem = (size_t)nslot * SLAB + BIMG + 1024 + 16 * nslot + 64;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int rep = 0; rep < 4; ++rep) {
        if (rep == 3) cudaEventRecord(e0);
        k_ceiling<<<152, 64, smem>>>(map, A_, I_, C_, nslot, nmma, M, N, err);
        if (rep == 3) cudaEventRecord(e1);
    }
    const cudaError_t e = cudaEventSynchronize(e1);
    int h = 0;
    cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || h) {
        printf("error: %s, expired wait %d\n", cudaGetErrorString(e), h);
        return 1;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *us = ms * 1e3f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return 0;
}

}  // namespace

int main() {
    void* x = nullptr;
    int* err = nullptr;
    if (cudaMalloc(&x, BYTES) != cudaSuccess || cudaMalloc(&err, 4) != cudaSuccess) {
        printf("allocation failed\n");
        return 1;
    }
    cudaMemset(x, 0, BYTES);
    cudaMemset(err, 0, 4);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        !fn) {
        printf("cuTensorMapEncodeTiled unavailable\n");
        return 1;
    }
    CUtensorMap map;
    cuuint64_t dims[3] = {(cuuint64_t)C_, (cuuint64_t)I_, (cuuint64_t)A_};
    cuuint64_t strides[2] = {(cuuint64_t)C_ * 2, (cuuint64_t)I_ * C_ * 2};
    cuuint32_t box[3] = {64, 128, 1}, es[3] = {1, 1, 1};
    if (((EncodeFn)fn)(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, x, dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        printf("tensor map encoding failed\n");
        return 1;
    }
    cudaFuncSetAttribute(k_ceiling, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    const double slabs_per_sm = BYTES / (double)SLAB / 152.0;
    float us = 0.f;
    printf("sweep 1: slab released at once (copy ceiling of the access pattern)\n");
    for (int nslot = 2; nslot <= 5; ++nslot) {
        if (run(map, nslot, 0, 128, 32, err, &us)) return 1;
        printf("  ring %d x 32 KB: %7.1f us %6.0f GB/s\n", nslot, us, BYTES / (us * 1e-6) / 1e9);
    }
    printf("sweep 2: MMAs (128 x 32 x 16) per 32 KB slab, ring 5\n");
    for (int nmma = 8; nmma <= 32; nmma += 8) {
        if (run(map, 5, nmma, 128, 32, err, &us)) return 1;
        printf("  %2d MMAs: %7.1f us %6.0f GB/s %5.0f ns per MMA per SM\n", nmma, us, BYTES / (us * 1e-6) / 1e9,
               us * 1e3 / (slabs_per_sm * nmma));
    }
    printf("sweep 3: 16 MMAs per slab, M x N x 16, ring 5\n");
    const int Ms[2] = {128, 64}, Ns[5] = {16, 32, 64, 128, 256};
    for (int mi = 0; mi < 2; ++mi)
        for (int ni = 0; ni < 5; ++ni) {
            if (run(map, 5, 16, Ms[mi], Ns[ni], err, &us)) return 1;
            printf("  M %3d N %3d: %7.1f us %6.0f GB/s %5.0f ns per MMA per SM\n", Ms[mi], Ns[ni], us,
                   BYTES / (us * 1e-6) / 1e9, us * 1e3 / (slabs_per_sm * 16));
        }
    return 0;
}
