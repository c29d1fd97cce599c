// Tensor-core Krylov step P = X_(n) (X_(n)^T Q) (Algorithm 1 step 3 / Eq. BKspace): one read
// of X from HBM per step, software-pipelined over 64-column tiles.
//
// X is viewed per mode as [A][I][C] in its native C-order layout.  A tile is 64 unfolding
// columns x all I rows; it arrives as NS = ceil(I/128) slots of 16 KB (128 rows x 64 columns,
// BF16/FP16, 128-byte swizzle) in a ring of `nslot` >= 2 NS slots, so that two tiles are
// resident while a third streams in.  Per tile k:
//   GEMM1(k)   Y_k = X_k^T Q          M = 64 tile columns, K = I, into tensor memory buffer k%2
//   epilogue   Y_k -> BF16 operand image in shared memory (hi + lo parts with `split`)
//   GEMM2(k)   P_s += X_{k,s} Y_k     M = 128 rows per slot s, K = 64, accumulators in TMEM
// GEMM1(k+1) runs while the epilogue of tile k works, so the TMA stream never waits for the
// GEMM1 -> epilogue -> GEMM2 chain of one tile; GEMM2(k) releases tile k's slots.  At the end every CTA writes its
// FP32 partial P (grid x I x N) and a fixed-order FP64 reduction sums them.
//
// Layouts (M = 64 places row m of D in TMEM lane 32 (m / 16) + m % 16):
//   C > 1 ("CFAST"): slot = one TMA box {64 c, 128 i}: 128 rows of 128 bytes.  GEMM1 reads it
//          as X^T, MN-major (one 64-element swizzle atom); GEMM2 as X, K-major.
//   C == 1 ("IFAST"): slot = two boxes {64 i, 64 a} (i 0-63 and 64-127 of the slot): 64 rows of
//          128 bytes each.  GEMM1 reads X^T K-major; GEMM2 reads X MN-major (two atoms 8 KB apart).
// Warp roles (224 threads): warp 0 TMA producer, warp 1 GEMM1 issuer + TMEM owner, warps 2-5
// epilogue, warp 6 GEMM2 issuer.  One thread issuing tcgen05.mma pays a fixed issue latency
// per instruction (about 54 cycles measured for M = 128, N = 32); two issuing threads overlap
// it (about 40 cycles per MMA combined).  Every mbarrier wait is bounded; on expiry the CTA
// raises its abort flag, every role leaves its loop, the producer waits (bounded) for each copy
// it issued and each issuer for every MMA it issued, then tensor memory is freed and the error
// word set.
#include <cuda.h>

#include "kernels.h"
#include "tc.h"
#include "tc_ptx.cuh"

namespace rbki {
namespace tc {
namespace {

constexpr int TW = 64;               // tile width in unfolding columns
constexpr int SLOT_BYTES = 16384;    // 128 rows x 64 columns x 2 bytes
constexpr int HALF_BYTES = 8192;     // one {64 i, 64 a} box of the I-fast layout
constexpr int NTHREADS = 224;
constexpr int MAX_SLOTS = 14;
constexpr int BAR_BYTES = 512;

struct KParams {
    int64_t A, I, C;
    int NS, N, Sh, split;
    int64_t tiles, ctiles;
    int nslot;
    uint32_t smem_q, smem_y, smem_bar;   // slots start at offset 0
    uint32_t tmem_cols;
    const void* qimg;
    uint32_t qimg_bytes;
    uint32_t yimg_bytes;                 // TW * N * 2
    float* part;
    int* err;
    int fp16;
    uint32_t wait_us;
    int stall;
};

// N (the MMA width, 16..64) is a template parameter so that every register array index of
// the epilogue is static (no local memory).
template <bool IFAST, int N>
__global__ void __launch_bounds__(NTHREADS, 1) k_krylov_tc(const __grid_constant__ CUtensorMap tmap, const KParams p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nslot = p.nslot, NS = p.NS;
    const uint32_t lim = p.wait_us;
    uint64_t* bars = (uint64_t*)(smem + p.smem_bar);
    const uint32_t b_full = smem_u32(bars), b_empty = b_full + 8 * nslot;
    const uint32_t b_yfull = b_empty + 8 * nslot, b_yready = b_yfull + 16, b_ysfree = b_yready + 16;
    const uint32_t b_qfull = b_ysfree + 16, b_pdone = b_qfull + 8, b_drain = b_pdone + 8, b_never = b_drain + 8;
    const uint32_t b_drain2 = b_never + 8;
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * nslot + 11);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    if (threadIdx.x == 0) {
        for (int i = 0; i < nslot; ++i) {
            mbar_init(b_full + 8 * i, 1);
            mbar_init(b_empty + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(b_yfull + 8 * i, 1);
            mbar_init(b_yready + 8 * i, 128);
            mbar_init(b_ysfree + 8 * i, 1);
        }
        mbar_init(b_qfull, 1);
        mbar_init(b_pdone, 1);
        mbar_init(b_drain, 1);
        mbar_init(b_drain2, 1);
        mbar_init(b_never, 1);   // nothing ever arrives: the planted stall of the timeout test
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), p.tmem_cols);
        tmem_relinquish();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    const int64_t my_tiles = (p.tiles - blockIdx.x + gridDim.x - 1) / gridDim.x;
    const uint32_t X0 = sbase, Q0 = sbase + p.smem_q, Y0 = sbase + p.smem_y;
    const uint32_t ycol0 = (uint32_t)(NS * N);   // TMEM columns of the two Y buffers
    const bool fp16 = p.fp16 != 0;

    if (warp == 0) {
        // ------------------------------ TMA producer ------------------------------
        if (lane == 0) {
            uint32_t issued = 0, par = 0;   // slots loaded at least once; parity of the last load
            mbar_expect_tx(b_qfull, p.qimg_bytes);
            for (uint32_t off = 0; off < p.qimg_bytes; off += 32768) {
                const uint32_t sz = min(32768u, p.qimg_bytes - off);
                bulk_load(Q0 + off, (const uint8_t*)p.qimg + off, sz, b_qfull);
            }
            uint32_t slot = 0, phase = 0;
            for (int64_t k = 0; k < my_tiles && !*abort_flag; ++k) {
                const int64_t t = blockIdx.x + k * gridDim.x;
                int ca, cc = 0;   // TMA coordinates of the tile
                if (!IFAST) {
                    ca = (int)(t / p.ctiles);
                    cc = (int)((t % p.ctiles) * TW);
                } else {
                    ca = (int)(t * TW);
                }
                for (int s = 0; s < NS; ++s) {
                    if (!mbar_wait(b_empty + 8 * slot, phase ^ 1, abort_flag, lim)) break;
                    mbar_expect_tx(b_full + 8 * slot, SLOT_BYTES);
                    const uint32_t dst = X0 + slot * SLOT_BYTES;
                    if (!IFAST) {
                        tma_load_3d(dst, &tmap, b_full + 8 * slot, cc, 128 * s, ca);
                    } else {
                        tma_load_2d(dst, &tmap, b_full + 8 * slot, 128 * s, ca);
                        tma_load_2d(dst + HALF_BYTES, &tmap, b_full + 8 * slot, 128 * s + 64, ca);
                    }
                    issued |= 1u << slot;
                    par = (par & ~(1u << slot)) | (phase << slot);
                    if (++slot == (uint32_t)nslot) { slot = 0; phase ^= 1; }
                }
            }
            // drain: every copy issued into this CTA's shared memory lands before it exits
            mbar_drain(b_qfull, 0, lim);
            for (int i = 0; i < nslot; ++i)
                if (issued >> i & 1) mbar_drain(b_full + 8 * i, par >> i & 1, lim);
        }
    } else if (warp == 1) {
        // ------------------------------ GEMM1 issuer ------------------------------
        // Y_k = X_k^T Q into tensor-memory buffer k % 2, slot by slot as slots land.  Buffer b
        // is free again once the epilogue of tile k-2 has read it (its Y-ready arrival).
        // Descriptors are built once; a slot's or K-step's descriptor adds its byte offset / 16.
        if (lane == 0) {
            const uint32_t id1 = idesc_f16(64, N, /*a_mn=*/!IFAST, /*b_mn=*/true, fp16);
            constexpr uint32_t qlbo = (uint32_t)(N / 8) * 128u;
            constexpr uint32_t qstep = (2u * qlbo) >> 4;     // one K = 16 step (16 rows) of the Q image
            // A = X^T: CFAST MN-major (a single 64-column atom), IFAST K-major
            const uint64_t dx1 = sdesc(X0, 16, 1024, LAYOUT_SW128);
            const uint64_t dq = sdesc(Q0, qlbo, 128, LAYOUT_NONE);
            bool ok = true;
            if (p.stall) ok = mbar_wait(b_never, 0, abort_flag, lim);   // expires by design
            if (ok) ok = mbar_wait(b_qfull, 0, abort_flag, lim);
            uint32_t slot = 0, phase = 0;
            for (int64_t k = 0; ok && k < my_tiles; ++k) {
                const uint32_t b = (uint32_t)(k & 1);
                if (k >= 2 && !mbar_wait(b_yready + 8 * b, (uint32_t)(((k - 2) >> 1) & 1), abort_flag, lim)) break;
                const uint32_t ytm = tbase + ycol0 + b * (uint32_t)N;
                for (int s = 0; s < NS; ++s) {
                    if (!mbar_wait(b_full + 8 * slot, phase, abort_flag, lim)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t a0 = dx1 + (uint64_t)(slot * (SLOT_BYTES >> 4));
                    const uint64_t b0 = dq + (uint64_t)(s * 8 * qstep);
                    umma_f16(ytm, a0, b0, id1, s != 0 ? 1u : 0u);
#pragma unroll
                    for (int kk = 1; kk < 8; ++kk) {
                        const uint32_t ko = IFAST ? (uint32_t)(((kk >> 2) * HALF_BYTES + (kk & 3) * 32) >> 4)
                                                  : (uint32_t)((kk * 2048) >> 4);
                        umma_f16(ytm, a0 + ko, b0 + (uint64_t)(kk * qstep), id1, 1u);
                    }
                    if (++slot == (uint32_t)nslot) { slot = 0; phase ^= 1; }
                }
                if (!ok) break;
                umma_commit(b_yfull + 8 * b);
            }
            // drain: every MMA this thread issued completes before tensor memory is freed
            umma_commit(b_drain);
            if (!mbar_drain(b_drain, 0, lim)) *abort_flag = 1;
        }
    } else if (warp == 6) {
        // ------------------------------ GEMM2 issuer ------------------------------
        // P_s += X_{k,s} Y_k once the epilogue has Y_k's operand image ready; then tile k's
        // slots go back to the producer.  Tile k occupies the NS ring slots from (k NS) % nslot.
        // A second issuing thread lets GEMM2(k) overlap GEMM1(k+1) in the tensor pipe.
        if (lane == 0) {
            const uint32_t id2 = idesc_f16(128, N, /*a_mn=*/IFAST, /*b_mn=*/true, fp16);
            // A = X: CFAST K-major, IFAST MN-major (atoms of 64 rows, 8 KB apart)
            const uint64_t dx2 = IFAST ? sdesc(X0, HALF_BYTES, 1024, LAYOUT_SW128) : sdesc(X0, 16, 1024, LAYOUT_SW128);
            const uint64_t dy = sdesc(Y0, 128, TW * 16, LAYOUT_NONE);
            bool ok = true;
            uint32_t sl = 0;
            for (int64_t k = 0; ok && k < my_tiles; ++k) {
                const uint32_t b = (uint32_t)(k & 1);
                if (!mbar_wait(b_yready + 8 * b, (uint32_t)((k >> 1) & 1), abort_flag, lim)) { ok = false; break; }
                tc_fence_after();
                const uint64_t y0 = dy + (uint64_t)((b * p.yimg_bytes) >> 4);
                for (int s = 0; s < NS; ++s) {
                    const uint64_t a0 = dx2 + (uint64_t)(sl * (SLOT_BYTES >> 4));
                    const uint32_t ptm = tbase + (uint32_t)(s * N);
                    umma_f16(ptm, a0, y0, id2, k > 0 ? 1u : 0u);
#pragma unroll
                    for (int kk = 1; kk < 4; ++kk) {
                        const uint32_t ko = IFAST ? (uint32_t)((kk * 2048) >> 4) : (uint32_t)((kk * 32) >> 4);
                        umma_f16(ptm, a0 + ko, y0 + (uint64_t)(kk * 16), id2, 1u);
                    }
                    umma_commit(b_empty + 8 * sl);
                    if (++sl == (uint32_t)nslot) sl = 0;
                }
                umma_commit(b_ysfree + 8 * b);
            }
            if (ok) umma_commit(b_pdone);
            umma_commit(b_drain2);
            if (!mbar_drain(b_drain2, 0, lim)) *abort_flag = 1;
        }
    } else {
        // ------------------------------ epilogue (warps 2-5) ------------------------------
        const int q = warp & 3;                         // TMEM sub-partition of this warp
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int col = q * 16 + lane;                  // tile column held by lanes 0-15 (M = 64)
        const int Sh = p.Sh;
        const bool split = p.split != 0;
        float v[64];
        for (int64_t k = 0; k < my_tiles; ++k) {
            const uint32_t b = (uint32_t)(k & 1);
            if (!mbar_wait(b_yfull + 8 * b, (uint32_t)((k >> 1) & 1), abort_flag, lim)) break;
            tc_fence_after();
            const uint32_t ytm = tbase + ycol0 + b * (uint32_t)N + lane_off;
            tmem_ld32(ytm, v);
            if (N > 32) tmem_ld32(ytm + 32, v + 32);
            if (split) {
                // Y = X^T (Q_hi + Q_lo), then Y = Y_hi + Y_lo again for GEMM2: hi in columns
                // s < Sh, lo in N/2 + s (columns past Sh hold zeros: Q's image is zero there)
#pragma unroll
                for (int s = 0; s < N / 2; ++s) {
                    const float y = v[s] + v[N / 2 + s];
                    const float hi = round_lo(y, fp16);
                    v[s] = hi;
                    v[N / 2 + s] = s < Sh ? y - hi : 0.f;
                }
            }
            // image b was read by GEMM2(k-2)
            if (k >= 2 && !mbar_wait(b_ysfree + 8 * b, (uint32_t)(((k - 2) >> 1) & 1), abort_flag, lim)) break;
            if (lane < 16) {
                // BF16 operand image of Y (MN-major, no swizzle): element (c, n) at
                // (n/8) * TW*16 + c*16 + (n%8)*2 bytes
                uint8_t* img = smem + p.smem_y + (size_t)b * p.yimg_bytes;
#pragma unroll
                for (int g = 0; g < N / 8; ++g) {
                    uint4 w;
                    w.x = pack2(v[8 * g + 0], v[8 * g + 1], fp16);
                    w.y = pack2(v[8 * g + 2], v[8 * g + 3], fp16);
                    w.z = pack2(v[8 * g + 4], v[8 * g + 5], fp16);
                    w.w = pack2(v[8 * g + 6], v[8 * g + 7], fp16);
                    *reinterpret_cast<uint4*>(img + g * (TW * 16) + col * 16) = w;
                }
            }
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(b_yready + 8 * b);
        }
        if (mbar_wait(b_pdone, 0, abort_flag, lim)) {
            tc_fence_after();
            float* out = p.part + (size_t)blockIdx.x * p.I * N;
            const int row = q * 32 + lane;
            for (int s = 0; s < NS; ++s) {
                const uint32_t ptm = tbase + (uint32_t)(s * N) + lane_off;
                tmem_ld32(ptm, v);
                if (N > 32) tmem_ld32(ptm + 32, v + 32);
                const int64_t i = (int64_t)s * 128 + row;
                if (i < p.I) {
                    float4* o = reinterpret_cast<float4*>(out + i * N);
#pragma unroll
                    for (int g = 0; g < N / 4; ++g) o[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tbase, p.tmem_cols);
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(p.err, 1);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn_k() {
    static const EncodeTiledFn fn = [] {   // looked up once, thread-safe
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (EncodeTiledFn)ptr;
        return (EncodeTiledFn) nullptr;
    }();
    return fn;
}

template <bool IFAST, int N>
size_t smem_limit_k() {
    static const size_t mx = max_dyn_smem(k_krylov_tc<IFAST, N>);   // thread-safe, once
    return mx;
}

template <bool IFAST>
size_t smem_limit_n(int N) {
    switch (N) {
        case 16: return smem_limit_k<IFAST, 16>();
        case 32: return smem_limit_k<IFAST, 32>();
        case 48: return smem_limit_k<IFAST, 48>();
        default: return smem_limit_k<IFAST, 64>();
    }
}

template <bool IFAST>
void launch_n(int N, int grid, size_t smem, cudaStream_t st, const CUtensorMap& map, const KParams& p) {
    switch (N) {
        case 16: k_krylov_tc<IFAST, 16><<<grid, NTHREADS, smem, st>>>(map, p); break;
        case 32: k_krylov_tc<IFAST, 32><<<grid, NTHREADS, smem, st>>>(map, p); break;
        case 48: k_krylov_tc<IFAST, 48><<<grid, NTHREADS, smem, st>>>(map, p); break;
        default: k_krylov_tc<IFAST, 64><<<grid, NTHREADS, smem, st>>>(map, p); break;
    }
}

int sm_count() {
    static const int sms = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return std::max(1, n);
    }();
    return sms;
}

// slots that fit beside the Q image, the two Y images and the barriers (0 if the launch
// cannot be configured)
int krylov_slots(const View& v, int N, size_t limit) {
    const int NS = (int)cdiv(v.I, 128);
    const size_t fixed = 1024 + (size_t)NS * 128 * N * 2 + (size_t)2 * TW * N * 2 + BAR_BYTES;
    if (limit < fixed) return 0;
    return (int)std::min<size_t>(MAX_SLOTS, (limit - fixed) / SLOT_BYTES);
}

}  // namespace

bool krylov_supported(const View& v, int N) {
    if (v.dtype != RBKI_BF16 && v.dtype != RBKI_F16) return false;
    if (N < 16 || N > 64 || N % 16) return false;
    const bool ifast = v.C == 1;
    if (ifast ? (v.I % 8) : (v.C % 8)) return false;
    if (v.A > 0x7fffffffLL || v.I > 0x7fffffffLL || v.C > 0x7fffffffLL) return false;
    const int NS = (int)cdiv(v.I, 128);
    if (NS * N + 2 * N > 512) return false;   // TMEM: P accumulators + two Y buffers
    // two whole tiles must fit the ring (GEMM1 of tile k+1 runs before GEMM2 of tile k);
    // GB300 allows 227 KB of dynamic shared memory per CTA
    return krylov_slots(v, N, 227 * 1024) >= 2 * NS;
}

int64_t krylov_tiles(const View& v) { return v.C > 1 ? v.A * cdiv(v.C, TW) : cdiv(v.A, TW); }

int krylov_grid(const View& v) { return (int)std::min<int64_t>(krylov_tiles(v), sm_count()); }

rbki_status krylov_tc(const View& v, int N, int Sh, bool split, const void* qimg, float* part, int* err,
                      cudaStream_t st, uint32_t wait_us, int stall) {
    EncodeTiledFn enc = encode_fn_k();
    if (!enc) return set_error(RBKI_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    const bool ifast = v.C == 1;
    CUtensorMap map;
    const CUtensorMapDataType dt = v.dtype == RBKI_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r;
    if (!ifast) {
        cuuint64_t dims[3] = {(cuuint64_t)v.C, (cuuint64_t)v.I, (cuuint64_t)v.A};
        cuuint64_t strides[2] = {(cuuint64_t)v.C * 2, (cuuint64_t)v.I * v.C * 2};
        cuuint32_t box[3] = {64, 128, 1};
        cuuint32_t es[3] = {1, 1, 1};
        r = enc(&map, dt, 3, const_cast<void*>(v.data), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[2] = {(cuuint64_t)v.I, (cuuint64_t)v.A};
        cuuint64_t strides[1] = {(cuuint64_t)v.I * 2};
        cuuint32_t box[2] = {64, 64};
        cuuint32_t es[2] = {1, 1};
        r = enc(&map, dt, 2, const_cast<void*>(v.data), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return set_error(RBKI_E_CUDA, "cuTensorMapEncodeTiled failed");

    KParams p{};
    p.A = v.A; p.I = v.I; p.C = v.C;
    p.NS = (int)cdiv(v.I, 128);
    p.N = N; p.Sh = Sh; p.split = split ? 1 : 0;
    p.tiles = krylov_tiles(v);
    p.ctiles = ifast ? 1 : cdiv(v.C, TW);
    p.qimg = qimg;
    p.qimg_bytes = (uint32_t)image_bytes_skinny(v, N);
    p.yimg_bytes = (uint32_t)(TW * N * 2);
    p.part = part; p.err = err;
    p.fp16 = v.dtype == RBKI_F16 ? 1 : 0;
    p.wait_us = wait_us ? wait_us : WAIT_US_DEFAULT;
    p.stall = stall;
    const uint32_t tm = (uint32_t)(p.NS * N + 2 * N);
    uint32_t cols = 32;
    while (cols < tm) cols <<= 1;
    p.tmem_cols = cols;
    const size_t limit = ifast ? smem_limit_n<true>(N) : smem_limit_n<false>(N);
    if (!limit) return set_error(RBKI_E_CUDA, "krylov_tc: shared-memory attribute");
    p.nslot = krylov_slots(v, N, limit);
    if (p.nslot < 2 * p.NS) return set_error(RBKI_E_UNSUPPORTED, "krylov_tc: two tiles do not fit");
    p.smem_q = (uint32_t)(p.nslot * SLOT_BYTES);
    p.smem_y = p.smem_q + p.qimg_bytes;
    p.smem_bar = (uint32_t)(p.smem_y + 2 * p.yimg_bytes);
    const size_t smem = 1024 + p.smem_bar + BAR_BYTES;
    const int grid = krylov_grid(v);
    if (ifast) launch_n<true>(N, grid, smem, st, map, p);
    else launch_n<false>(N, grid, smem, st, map, p);
    RBKI_LAUNCH_CHECK("k_krylov_tc");
    return RBKI_OK;
}

}  // namespace tc
}  // namespace rbki
