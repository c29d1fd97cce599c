// Batched rBKI-TK for many small decompositions (rbki_tucker_batched): a wave of requests
// runs Algorithms 1-2 in lockstep, one launch per stage for every mode of every request.
//
// The served stream (3rd-order tensors of 32..256 per mode, ranks 4..32) is bound by kernel
// launches, not by HBM: one decomposition is ~250 small launches, and the host issues about
// 200k launches/s however many threads it uses.  Here a stage is one launch whatever the
// number of requests:
//   * X is read once per mode: a work-queue kernel (k_gram_b) forms X_(n) X_(n)^T for every
//     mode of every item (I_n <= 256, so the matrix is small) and, on the Krylov-path modes,
//     the sketch W = X_(n) Omega from the same staged columns; block (x, y) of the launch is
//     unit x of item y, a block pair of the Gram matrix over a run of 32-column steps.  The
//     Krylov products are then P_j = (X_(n) X_(n)^T) Q_j in FP64, without touching X (the
//     same Krylov space as X_(n) (X_(n)^T Q_j), associated the other way);
//   * the core's mode products share a second work-queue kernel (k_ttm_b);
//   * the FP64 stages (block orthonormalisation, Z = Q^T P, the eigensolver, U = Q U~, the
//     Krylov products) are the batched twins of the single-call kernels (bat_launch): the
//     same device code and the same per-item grids.
// Every per-item partition (units, steps per unit) depends only on the item's shape and the
// reductions have a fixed order, so each item's result does not depend on its wave.
// Products with X are FP32 products of the BF16/FP16 value of each entry of X (rounded as it
// is read when the storage is wider) with FP32 Omega / U, FP32 accumulation within a unit and
// FP64 across units; orthonormalisation, the Krylov products and the eigensolver are FP64.
#include "kernels.h"
#include "plan.h"
#include "tc_ptx.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

namespace rbki {
namespace {

constexpr int GB = 64;          // rows of a block of X_(n) X_(n)^T
constexpr int KT = 32;          // columns of X_(n) per step of the Gram pass
constexpr int GP = GB + 4;      // shared-memory pitch of a staged block (16-byte rows)
constexpr int TT = 64;          // columns of X_(n) per tile of a mode product
constexpr int NTHREADS = 256;   // 8 warps

__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float round_to(float v, int rnd) {
    if (rnd == RBKI_BF16) return __bfloat162float(__float2bfloat16_rn(v));
    if (rnd == RBKI_F16) return __half2float(__float2half_rn(v));
    return v;
}

// column offsets of X_(n): colb[k] = offset of X[a][0][c] for column col0 + k, -1 past the end
__device__ __forceinline__ void column_bases(int64_t col0, int ncol, int64_t J, int I, int64_t C, int64_t* colb) {
    for (int k = threadIdx.x; k < ncol; k += NTHREADS) {
        const int64_t col = col0 + k;
        colb[k] = col < J ? (col / C) * I * C + col % C : -1;
    }
}

// ---------------------------------------------------------------------------------------
// Gram pass: G = X_(n) X_(n)^T (and W = X_(n) Omega) for I_n <= 256, one pass over X.
// Block pair (bi <= bj) of 64 x 64 rows of G, unit u = a run of 32-column steps: the two row
// blocks of the step are staged transposed (As[k][r], pitch 68), each thread accumulates a
// 4 x 4 tile (two 16-byte loads per 16 FMAs).  The diagonal pairs of a Krylov-path item also
// accumulate W's rows of their block: Omega's 32 x S entries are generated in place (Philox
// keyed by (seed, mode, column, pair)) and each thread holds S8/4 columns of one row.
// ---------------------------------------------------------------------------------------
struct gram_rec {
    const void* x;       // the item's tensor, viewed as [A][I][C]
    int dtype, rnd;      // storage dtype; rounding applied as values are read (0: none)
    int A, I, C;
    int nb, npair;       // row blocks of 64; block pairs bi <= bj
    int ksteps, kpu;     // 32-column steps of X_(n); steps per unit
    int S;               // sketch width (0: no sketch)
    uint64_t seed;
    int mode;
    float* gpart;        // [unit][I][I]: block pairs (diagonal blocks in full)
    float* wpart;        // [unit][I][S]
    int gx, gy, gz;      // npair * units, 1, 1
};

template <typename T>
__device__ __forceinline__ void stage_rows(const T* __restrict__ x, const int64_t* colb, int row0, int I, int64_t C,
                                           int rnd, float* As) {
    if (C == 1) {
        // columns are contiguous along i
#pragma unroll 4
        for (int e = threadIdx.x; e < KT * GB; e += NTHREADS) {
            const int k = e / GB, rr = e % GB, i = row0 + rr;
            const int64_t cb = colb[k];
            As[k * GP + rr] = (cb >= 0 && i < I) ? round_to(to_f32(x[cb + i]), rnd) : 0.f;
        }
    } else {
        // consecutive columns are contiguous along c
#pragma unroll 4
        for (int e = threadIdx.x; e < KT * GB; e += NTHREADS) {
            const int rr = e / KT, k = e % KT, i = row0 + rr;
            const int64_t cb = colb[k];
            As[k * GP + rr] = (cb >= 0 && i < I) ? round_to(to_f32(x[cb + (int64_t)i * C]), rnd) : 0.f;
        }
    }
}

__device__ __forceinline__ void gram_dev(const gram_rec& r, int bx) {
    extern __shared__ __align__(16) float gsm[];
    const int pair = bx % r.npair, unit = bx / r.npair;
    int bi = 0, bj = 0;
    for (int p = pair, b = 0; b < r.nb; ++b) {
        if (p < r.nb - b) {
            bi = b;
            bj = b + p;
            break;
        }
        p -= r.nb - b;
    }
    const bool diag = bi == bj, sk = diag && r.S > 0;
    const int S8 = (r.S + 7) & ~7, wn = S8 / 4;   // sketch columns per thread
    float* As = gsm;
    float* Bs = As + KT * GP;
    float* Om = Bs + KT * GP;
    int64_t* colb = reinterpret_cast<int64_t*>(Om + KT * 64);
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int rr = tid % 64, cg = tid / 64;
    const int64_t C = r.C, J = (int64_t)r.A * r.C;
    float acc[4][4], wacc[16];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) wacc[c] = 0.f;
    const int k_lo = unit * r.kpu, k_hi = min(r.ksteps, k_lo + r.kpu);
    for (int t = k_lo; t < k_hi; ++t) {
        const int64_t col0 = (int64_t)t * KT;
        __syncthreads();   // the previous step is consumed
        column_bases(col0, KT, J, r.I, C, colb);
        __syncthreads();
        switch (r.dtype) {
            case RBKI_BF16:
                stage_rows(static_cast<const __nv_bfloat16*>(r.x), colb, bi * GB, r.I, C, r.rnd, As);
                if (!diag) stage_rows(static_cast<const __nv_bfloat16*>(r.x), colb, bj * GB, r.I, C, r.rnd, Bs);
                break;
            case RBKI_F16:
                stage_rows(static_cast<const __half*>(r.x), colb, bi * GB, r.I, C, r.rnd, As);
                if (!diag) stage_rows(static_cast<const __half*>(r.x), colb, bj * GB, r.I, C, r.rnd, Bs);
                break;
            case RBKI_F32:
                stage_rows(static_cast<const float*>(r.x), colb, bi * GB, r.I, C, r.rnd, As);
                if (!diag) stage_rows(static_cast<const float*>(r.x), colb, bj * GB, r.I, C, r.rnd, Bs);
                break;
            default:
                stage_rows(static_cast<const double*>(r.x), colb, bi * GB, r.I, C, r.rnd, As);
                if (!diag) stage_rows(static_cast<const double*>(r.x), colb, bj * GB, r.I, C, r.rnd, Bs);
                break;
        }
        if (sk) {
            const int np = S8 / 2;
            for (int e = tid; e < KT * np; e += NTHREADS) {
                const int k = e / np, pr = e % np, s = 2 * pr;
                float z0 = 0.f, z1 = 0.f;
                if (colb[k] >= 0 && s < r.S)
                    omega_pair_f32(r.seed, (uint32_t)r.mode, (uint64_t)(col0 + k), (uint32_t)pr, z0, z1);
                Om[k * 64 + s] = z0;
                Om[k * 64 + s + 1] = s + 1 < r.S ? z1 : 0.f;
            }
        }
        __syncthreads();
        const float* Bsrc = diag ? As : Bs;
#pragma unroll 4
        for (int k = 0; k < KT; ++k) {
            const float4 a4 = *reinterpret_cast<const float4*>(As + k * GP + ty * 4);
            const float4 b4 = *reinterpret_cast<const float4*>(Bsrc + k * GP + tx * 4);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        if (sk) {
            for (int k = 0; k < KT; ++k) {
                const float a = As[k * GP + rr];
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c < wn) wacc[c] = fmaf(a, Om[k * 64 + cg * wn + c], wacc[c]);
            }
        }
    }
    float* g = r.gpart + (int64_t)unit * r.I * r.I;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = bi * GB + ty * 4 + a;
        if (i >= r.I) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = bj * GB + tx * 4 + b;
            if (j < r.I) g[(int64_t)i * r.I + j] = acc[a][b];
        }
    }
    if (sk) {
        const int i = bi * GB + rr;
        if (i < r.I) {
            float* w = r.wpart + ((int64_t)unit * r.I + i) * r.S;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int s = cg * wn + c;
                if (c < wn && s < r.S) w[s] = wacc[c];
            }
        }
    }
}

__global__ void __launch_bounds__(NTHREADS) k_gram_b(const __grid_constant__ BPack<gram_rec> p) {
    const gram_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    gram_dev(r, bx);
}

constexpr size_t GRAM_SMEM = (2 * KT * GP + KT * 64) * sizeof(float) + KT * sizeof(int64_t);

// ---------------------------------------------------------------------------------------
// Gram pass on the tensor cores (tcgen05, BF16/FP16 X stored in the products' format).
// CTA = (item, row block rb of 128 rows, unit of 64-column steps).  Per step the CTA stages
// X_(n)'s 64 columns for all rows (padded to whole 128-row blocks, zeros outside X) in one
// of two shared-memory buffers and one thread issues, per K = 16:
//   G[rb rows, 0:Npad] += X[rb rows, k] X[:, k]^T     (M = 128, N = Npad <= 256)
//   W[rb rows, 0:S16]  += X[rb rows, k] Omega[k, :]    (M = 128, N = S16 <= 64; Krylov path)
// with the FP32 accumulators in tensor memory.  Layouts: C > 1 (consecutive columns
// contiguous): K-major, 128-byte swizzle (row r at r*128 B, 16-byte chunk q at q ^ (r & 7));
// C == 1 (rows contiguous): MN-major without swizzle (element (r, k) at (r/8)*1024 + k*16 +
// (r%8)*2 B).  Omega's tile (BF16/FP16, from the same Philox definition) is K-major,
// 128-byte swizzle.  A buffer is refilled once the MMAs that read it have committed.  Every
// mbarrier wait is bounded (tc::mbar_wait); on expiry the CTA drains its MMAs, frees tensor
// memory, sets the error word and writes no partials.
// ---------------------------------------------------------------------------------------
constexpr int TCK = 64;                    // columns of X_(n) per step
constexpr uint32_t TC_TILE_MAX = 2 * 16384; // two 128-row blocks x 64 columns x 2 B
constexpr uint32_t TC_OM_BYTES = 8192;     // Omega tile: up to 64 rows x 128 B
constexpr uint32_t TC_BUF = TC_TILE_MAX + TC_OM_BYTES;
constexpr size_t GRAM_TC_SMEM = 1024 + 2 * (size_t)TC_BUF + 64 + TCK * sizeof(int64_t);

struct gramtc_rec {
    const void* x;       // BF16 (fp16 = 0) or FP16 (fp16 = 1) storage, [A][I][C]
    int fp16;
    int A, I, C;
    int nrb, npad;       // 128-row blocks (1 or 2); Gram columns padded to 16
    int ksteps, kpu;     // 64-column steps of X_(n); steps per unit
    int S, S16;          // sketch width and its padding to 16 (0: no sketch)
    uint64_t seed;
    int mode;
    float* gpart;        // [unit][I][I]: full rows of the CTA's row block
    float* wpart;        // [unit][I][S]
    int32_t* err;        // set when a bounded wait expires
    uint32_t tcols;      // tensor-memory columns allocated (256 or 512)
    uint32_t wait_us;
    int stall;           // diagnostics: first wait on a barrier nothing completes (expires)
    int gx, gy, gz;      // nrb * units, 1, 1
};

__device__ __forceinline__ uint32_t swz128(int r, int k) {
    return (uint32_t)r * 128u + ((uint32_t)(((k >> 3) ^ (r & 7))) << 4) + (uint32_t)(k & 7) * 2u;
}

constexpr int TCT = 256;          // threads of the tensor-core Gram pass
constexpr int TCB = 16;           // loads a thread issues before its stores (memory parallelism)

// Stages the step's 64 columns: work item e of n (e = tid + TCT u) is loaded by load(e) into a
// register and stored by store(e, v); TCB loads are in flight before the first store.
template <typename V, typename L, typename S>
__device__ __forceinline__ void stage_batched(int n, L load, S store) {
    for (int e0 = threadIdx.x; e0 < n; e0 += TCT * TCB) {
        V v[TCB];
#pragma unroll
        for (int u = 0; u < TCB; ++u) {
            const int e = e0 + u * TCT;
            v[u] = e < n ? load(e) : V{};
        }
#pragma unroll
        for (int u = 0; u < TCB; ++u) {
            const int e = e0 + u * TCT;
            if (e < n) store(e, v[u]);
        }
    }
}

template <bool IFAST>
__device__ __forceinline__ void gramtc_stage(const gramtc_rec& r, int64_t col0, const int64_t* colb, uint8_t* tile,
                                             uint8_t* om) {
    const uint16_t* x = static_cast<const uint16_t*>(r.x);
    const int rows = r.nrb * 128, I = r.I;
    const int64_t C = r.C, J = (int64_t)r.A * r.C;
    const int tid = threadIdx.x;
    if (!IFAST) {
        // colb[k] = offset of X[a][0][c] of column col0 + k (-1 past the end)
        if (C % 8 == 0) {
            // 16-byte chunks: 8 consecutive columns of one row (col0 is a multiple of 64 and C of
            // 8, so a chunk never crosses a slab of X_(n)'s columns and is 16-byte aligned)
            stage_batched<uint4>(
                rows * 8,
                [&](int e) {
                    const int rr = e >> 3;
                    const int64_t cb = colb[8 * (e & 7)];
                    return (rr < I && cb >= 0) ? __ldg(reinterpret_cast<const uint4*>(x + cb + (int64_t)rr * C))
                                               : make_uint4(0u, 0u, 0u, 0u);
                },
                [&](int e, uint4 v) { *reinterpret_cast<uint4*>(tile + swz128(e >> 3, 8 * (e & 7))) = v; });
        } else {
            // element by element, a warp reading 32 consecutive columns of one row
            stage_batched<uint16_t>(
                rows * TCK,
                [&](int e) {
                    const int rr = e / TCK;
                    const int64_t cb = colb[e % TCK];
                    return (rr < I && cb >= 0) ? x[cb + (int64_t)rr * C] : (uint16_t)0;
                },
                [&](int e, uint16_t v) { *reinterpret_cast<uint16_t*>(tile + swz128(e / TCK, e % TCK)) = v; });
        }
    } else {
        if (I % 8 == 0) {
            // 16-byte chunks: 8 consecutive rows of one column
            stage_batched<uint4>(
                (rows / 8) * TCK,
                [&](int e) {
                    const int k = e % TCK, r8 = e / TCK;
                    const int64_t col = col0 + k;
                    return (8 * r8 < I && col < J) ? __ldg(reinterpret_cast<const uint4*>(x + col * I + 8 * r8))
                                                   : make_uint4(0u, 0u, 0u, 0u);
                },
                [&](int e, uint4 v) { *reinterpret_cast<uint4*>(tile + (e / TCK) * 1024 + (e % TCK) * 16) = v; });
        } else {
            const int rsh = rows == 128 ? 7 : 8;
            stage_batched<uint16_t>(
                rows * TCK,
                [&](int e) {
                    const int k = e >> rsh, rr = e & (rows - 1);
                    const int64_t col = col0 + k;
                    return (rr < I && col < J) ? x[col * I + rr] : (uint16_t)0;
                },
                [&](int e, uint16_t v) {
                    const int k = e >> rsh, rr = e & (rows - 1);
                    *reinterpret_cast<uint16_t*>(tile + (rr >> 3) * 1024 + k * 16 + (rr & 7) * 2) = v;
                });
        }
    }
    if (r.S16 > 0) {
        // Omega[col0 + k][s] for s < S16 (zeros past S and past X_(n)'s columns), rounded to the
        // products' format, stored K-major with the 128-byte swizzle (row s, column k)
        const int np = r.S16 / 2;
        for (int e = tid; e < TCK * np; e += TCT) {
            const int k = e / np, pr = e % np, s = 2 * pr;
            float z0 = 0.f, z1 = 0.f;
            if (col0 + k < J && s < r.S)
                omega_pair_f32(r.seed, (uint32_t)r.mode, (uint64_t)(col0 + k), (uint32_t)pr, z0, z1);
            if (s + 1 >= r.S) z1 = 0.f;
            uint16_t h0, h1;
            if (r.fp16) {
                __half a = __float2half_rn(z0), b = __float2half_rn(z1);
                h0 = *reinterpret_cast<uint16_t*>(&a);
                h1 = *reinterpret_cast<uint16_t*>(&b);
            } else {
                __nv_bfloat16 a = __float2bfloat16_rn(z0), b = __float2bfloat16_rn(z1);
                h0 = *reinterpret_cast<uint16_t*>(&a);
                h1 = *reinterpret_cast<uint16_t*>(&b);
            }
            *reinterpret_cast<uint16_t*>(om + swz128(s, k)) = h0;
            *reinterpret_cast<uint16_t*>(om + swz128(s + 1, k)) = h1;
        }
    }
}

template <bool IFAST>
__device__ __forceinline__ void gramtc_dev(const gramtc_rec& r, int bx) {
    using namespace tc;
    extern __shared__ __align__(1024) uint8_t tcsm[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tcsm) + 1023) & ~uintptr_t(1023));
    uint8_t* buf[2] = {base, base + TC_BUF};
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * TC_BUF);   // [0..1] MMA done, [2] drain
    uint64_t* never = bars + 3;                                        // never completed
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 5);
    int64_t* colb = reinterpret_cast<int64_t*>(bars + 8);          // the step's column offsets
    const int rb = bx % r.nrb, unit = bx / r.nrb;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lim = r.wait_us;
    if (warp == 0) {
        tmem_alloc(smem_u32(tslot), r.tcols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        mbar_init(smem_u32(&bars[2]), 1);
        mbar_init(smem_u32(never), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t wcol = (uint32_t)((r.npad + 31) & ~31);   // W's first accumulator column
    const int k_lo = unit * r.kpu, k_hi = min(r.ksteps, k_lo + r.kpu);
    const uint32_t idg = idesc_f16(128, r.npad, IFAST, IFAST, r.fp16 != 0);
    const uint32_t idw = idesc_f16(128, r.S16 > 0 ? r.S16 : 16, IFAST, false, r.fp16 != 0);
    bool ok = true;
    if (r.stall) {
        // a planted stall (diagnostics): every thread's wait runs out, the CTA aborts
        mbar_wait(smem_u32(never), 0, abort_flag, lim);
        __syncthreads();
        ok = !*abort_flag;
    }
    for (int t = k_lo; ok && t < k_hi; ++t) {
        const int n = t - k_lo, b = n & 1;
        // buffer b was last read by the MMAs of step n - 2
        if (n >= 2) {
            bool w = mbar_wait(smem_u32(&bars[b]), (uint32_t)(((n - 2) >> 1) & 1), abort_flag, lim);
            __syncthreads();
            if (!w || *abort_flag) {
                ok = false;
                break;
            }
        }
        if (!IFAST && tid < TCK) {
            const int64_t col = (int64_t)t * TCK + tid;
            colb[tid] = col < (int64_t)r.A * r.C ? (col / r.C) * r.I * r.C + col % r.C : -1;
        }
        __syncthreads();
        gramtc_stage<IFAST>(r, (int64_t)t * TCK, colb, buf[b], buf[b] + TC_TILE_MAX);
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t tb = smem_u32(buf[b]), to = tb + TC_TILE_MAX;
            const uint64_t da = IFAST ? sdesc(tb + (uint32_t)rb * 16384u, 128, 1024, LAYOUT_NONE)
                                      : sdesc(tb + (uint32_t)rb * 16384u, 16, 1024, LAYOUT_SW128);
            const uint64_t db = IFAST ? sdesc(tb, 128, 1024, LAYOUT_NONE) : sdesc(tb, 16, 1024, LAYOUT_SW128);
            const uint64_t dom = sdesc(to, 16, 1024, LAYOUT_SW128);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ka = IFAST ? (uint64_t)(16 * kk) : (uint64_t)(2 * kk);   // K = 16 step
                const uint32_t acc = (n > 0 || kk > 0) ? 1u : 0u;
                umma_f16(tbase, da + ka, db + ka, idg, acc);
                if (r.S16 > 0) umma_f16(tbase + wcol, da + ka, dom + (uint64_t)(2 * kk), idw, acc);
            }
            umma_commit(smem_u32(&bars[b]));
        }
    }
    // the last one or two groups: wait for their commits (bounded), also on the abort path
    if (tid == 0) {
        umma_commit(smem_u32(&bars[2]));
        if (!mbar_drain(smem_u32(&bars[2]), 0, lim)) *abort_flag = 1;
    }
    __syncthreads();
    tc_fence_after();
    if (ok && !*abort_flag && k_hi > k_lo) {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 = rows 128 rb + 32 (w % 4)
        // + lane; the two warps of a sub-partition take alternate 32-column groups
        const int q = warp & 3, half = warp >> 2;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int row = rb * 128 + q * 32 + lane;
        float v[32];
        float* g = r.gpart + ((int64_t)unit * r.I + row) * r.I;
        for (int c0 = 32 * half; c0 < r.npad; c0 += 64) {
            tmem_ld32(tbase + lane_off + (uint32_t)c0, v);
            if (row < r.I)
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j < r.I) g[c0 + j] = v[j];
        }
        if (r.S16 > 0) {
            float* w = r.wpart + ((int64_t)unit * r.I + row) * r.S;
            for (int c0 = 32 * half; c0 < r.S16; c0 += 64) {
                tmem_ld32(tbase + lane_off + wcol + (uint32_t)c0, v);
                if (row < r.I)
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < r.S) w[c0 + j] = v[j];
            }
        }
    }
    if ((!ok || *abort_flag) && tid == 0) atomicExch(r.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, r.tcols);
    }
}

template <bool IFAST>
__global__ void __launch_bounds__(TCT) k_gram_tc_b(const __grid_constant__ BPack<gramtc_rec> p) {
    const gramtc_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    gramtc_dev<IFAST>(r, bx);
}

// G (FP64, I x I) = sum over units of the block pairs, in unit order; the lower blocks mirror
// the upper ones, the diagonal blocks are symmetrised: G is exactly symmetric.
struct greduce_rec {
    const float* gpart;
    int units, I;
    double* G;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_greduce_b(const __grid_constant__ BPack<greduce_rec> p) {
    const greduce_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    const int e = bx * 256 + threadIdx.x;
    if (e >= r.I * r.I) return;
    const int i = e / r.I, j = e % r.I, bi = i / GB, bj = j / GB;
    const int64_t us = (int64_t)r.I * r.I;
    auto sum = [&](int a, int b) {
        double v = 0.0;
        for (int u = 0; u < r.units; ++u) v += (double)r.gpart[u * us + (int64_t)a * r.I + b];
        return v;
    };
    r.G[e] = bi < bj ? sum(i, j) : bi > bj ? sum(j, i) : 0.5 * (sum(i, j) + sum(j, i));
}

// ---------------------------------------------------------------------------------------
// Mode product of the core chain: T[a][s][c] = sum_i X[a][i][c] U[i][s] (S = R_n <= 64).
// Unit = a run of 64-column tiles of X_(n): the tile is staged transposed (XT[t][i], odd
// pitch); warp (g, h) of the product owns columns 8g..8g+7 of U and the share h of the rows
// i, the shares meet in shared memory in a fixed order; results are written along c.
// ---------------------------------------------------------------------------------------
struct ttm_rec {
    const void* x;
    int dtype, rnd;
    int A, I, C, S;
    int tiles, tpu;
    const double* U;     // I x S, ld ldu
    int ldu;
    void* out;           // [A][S][C], FP32 or FP64 (odt)
    int odt;
    int gx, gy, gz;
};

__host__ __device__ inline int ttm_ip(int I) { return I | 1; }
__host__ __device__ inline int s8_of(int S) { return (S + 7) & ~7; }
size_t ttm_smem(const ttm_rec& r) {
    const int S8 = s8_of(r.S), ns = 8 / (S8 / 8);
    return ((size_t)TT * ttm_ip(r.I) + (size_t)r.I * S8 + (size_t)TT * S8 + (ns > 1 ? (size_t)ns * TT * S8 : 0)) *
               sizeof(float) + TT * sizeof(int64_t);
}

template <typename T>
__device__ __forceinline__ void stage_tile(const T* __restrict__ x, const int64_t* colb, int I, int Ip, int64_t C,
                                           int rnd, float* XTs) {
    const int n = TT * I;
    if (C == 1) {
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += NTHREADS) {
            const int tt = e / I, i = e - tt * I;
            const int64_t cb = colb[tt];
            XTs[tt * Ip + i] = cb >= 0 ? round_to(to_f32(x[cb + i]), rnd) : 0.f;
        }
    } else {
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += NTHREADS) {
            const int i = e / TT, tt = e % TT;
            const int64_t cb = colb[tt];
            XTs[tt * Ip + i] = cb >= 0 ? round_to(to_f32(x[cb + (int64_t)i * C]), rnd) : 0.f;
        }
    }
}

__device__ __forceinline__ void ttm_dev(const ttm_rec& r, int unit) {
    extern __shared__ __align__(16) float tsm[];
    const int I = r.I, Ip = ttm_ip(I), S = r.S, S8 = s8_of(S);
    const int G = S8 / 8, ns = 8 / G;
    float* XTs = tsm;
    float* Us = XTs + TT * Ip;
    float* Ys = Us + I * S8;
    float* Yp = Ys + TT * S8;
    int64_t* colb = reinterpret_cast<int64_t*>(Yp + (ns > 1 ? ns * TT * S8 : 0));
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t C = r.C, J = (int64_t)r.A * r.C;
    for (int e = tid; e < I * S8; e += NTHREADS) {
        const int i = e / S8, s = e % S8;
        Us[e] = s < S ? (float)r.U[(int64_t)i * r.ldu + s] : 0.f;
    }
    const bool act = w < G * ns;
    const int g = w % G, h = w / G;
    const int il = (I + ns - 1) / ns, i_lo = h * il, i_hi = min(I, i_lo + il);
    const int t_lo = unit * r.tpu, t_hi = min(r.tiles, t_lo + r.tpu);
    for (int t = t_lo; t < t_hi; ++t) {
        const int64_t col0 = (int64_t)t * TT;
        __syncthreads();
        column_bases(col0, TT, J, I, C, colb);
        __syncthreads();
        switch (r.dtype) {
            case RBKI_BF16: stage_tile(static_cast<const __nv_bfloat16*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
            case RBKI_F16: stage_tile(static_cast<const __half*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
            case RBKI_F32: stage_tile(static_cast<const float*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
            default: stage_tile(static_cast<const double*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
        }
        __syncthreads();
        if (act) {
            const int s0 = 8 * g;
            float a1[2][8];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int j = 0; j < 8; ++j) a1[u][j] = 0.f;
            for (int i = i_lo; i < i_hi; ++i) {
                const float4 qa = *reinterpret_cast<const float4*>(Us + i * S8 + s0);
                const float4 qb = *reinterpret_cast<const float4*>(Us + i * S8 + s0 + 4);
                const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
                const float x0 = XTs[lane * Ip + i], x1 = XTs[(lane + 32) * Ip + i];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    a1[0][j] = fmaf(x0, qv[j], a1[0][j]);
                    a1[1][j] = fmaf(x1, qv[j], a1[1][j]);
                }
            }
            float* dst = ns == 1 ? Ys : Yp + h * TT * S8;
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int j = 0; j < 8; ++j) dst[(lane + 32 * u) * S8 + s0 + j] = a1[u][j];
        }
        if (ns > 1) {
            __syncthreads();
            for (int e = tid; e < TT * S8; e += NTHREADS) {
                float v = 0.f;
                for (int hh = 0; hh < ns; ++hh) v += Yp[hh * TT * S8 + e];
                Ys[e] = v;
            }
        }
        __syncthreads();
        for (int e = tid; e < TT * S; e += NTHREADS) {
            const int s = e / TT, tt = e % TT;
            const int64_t col = col0 + tt;
            if (col >= J) continue;
            const int64_t a = col / C, c = col % C;
            const int64_t o = (a * S + s) * C + c;
            const float v = Ys[tt * S8 + s];
            if (r.odt == RBKI_F64) static_cast<double*>(r.out)[o] = (double)v;
            else static_cast<float*>(r.out)[o] = v;
        }
    }
}

__global__ void __launch_bounds__(NTHREADS, 2) k_ttm_b(const __grid_constant__ BPack<ttm_rec> p) {
    const ttm_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    ttm_dev(r, bx);
}

// dst[i][s] = src[i][s] for i < rows, s < cols (strided blocks: Q_{j+1} <- P_j)
struct blkcopy_rec {
    const double* src;
    int lds;
    double* dst;
    int ldd, rows, cols;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_blkcopy_b(const __grid_constant__ BPack<blkcopy_rec> p) {
    const blkcopy_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    const int e = bx * 256 + threadIdx.x;
    if (e >= r.rows * r.cols) return;
    const int i = e / r.cols, s = e % r.cols;
    r.dst[(int64_t)i * r.ldd + s] = r.src[(int64_t)i * r.lds + s];
}

// out1[i][s] (= out2[i][s]) = sum over units of part[u][i][s], in unit order, FP64
struct xreduce_rec {
    const float* part;
    int units, I, S, ldp;
    double* out1;
    int ld1;
    double* out2;
    int ld2;
    int32_t* ticket;   // the item's orthonormalisation tickets, zeroed here (or nullptr)
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_xreduce_b(const __grid_constant__ BPack<xreduce_rec> p) {
    const xreduce_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    if (bx == 0 && r.ticket && (int)threadIdx.x < ORTH_TICKETS) r.ticket[threadIdx.x] = 0;
    const int e = bx * 256 + threadIdx.x;
    if (e >= r.I * r.S) return;
    const int i = e / r.S, s = e % r.S;
    const int64_t us = (int64_t)r.I * r.ldp;
    double a = 0.0;
    for (int u = 0; u < r.units; ++u) a += (double)r.part[u * us + (int64_t)i * r.ldp + s];
    r.out1[(int64_t)i * r.ld1 + s] = a;
    if (r.out2) r.out2[(int64_t)i * r.ld2 + s] = a;
}

// Z = (Z + Z^T) / 2 in place (n x n, ld n): the upper triangle's threads write both entries
struct sym_rec {
    double* Z;
    int n;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_sym_b(const __grid_constant__ BPack<sym_rec> p) {
    const sym_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    const int e = bx * 256 + threadIdx.x;
    if (e >= r.n * r.n) return;
    const int i = e / r.n, j = e % r.n;
    if (j <= i) return;
    const double v = 0.5 * (r.Z[(int64_t)i * r.n + j] + r.Z[(int64_t)j * r.n + i]);
    r.Z[(int64_t)i * r.n + j] = v;
    r.Z[(int64_t)j * r.n + i] = v;
}

// sum of squares in FP64: part[b] = sum over chunk b (block tree), then out = sum_b part[b]
constexpr int SQ_CHUNK = 1 << 16;
struct sumsq_rec {
    const void* x;
    int dtype;
    int64_t n;
    double* part;
    double* out;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_sumsq_part_b(const __grid_constant__ BPack<sumsq_rec> p) {
    const sumsq_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    __shared__ double red[8];
    const int64_t lo = (int64_t)bx * SQ_CHUNK, hi = min(r.n, lo + SQ_CHUNK);
    double a = 0.0;
    for (int64_t e = lo + threadIdx.x; e < hi; e += 256) {
        double v;
        switch (r.dtype) {
            case RBKI_BF16: v = (double)__bfloat162float(static_cast<const __nv_bfloat16*>(r.x)[e]); break;
            case RBKI_F16: v = (double)__half2float(static_cast<const __half*>(r.x)[e]); break;
            case RBKI_F32: v = (double)static_cast<const float*>(r.x)[e]; break;
            default: v = static_cast<const double*>(r.x)[e]; break;
        }
        a += v * v;
    }
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += red[k];
        r.part[bx] = t;
    }
}

__global__ void k_sumsq_fin_b(const __grid_constant__ BPack<sumsq_rec> p) {
    const sumsq_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz) || threadIdx.x) return;
    const int nb = (int)cdiv(r.n, SQ_CHUNK);
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += r.part[b];
    *r.out = t;
}

// p[0..n) = v for every record (the error words, kept counters and orthonormalisation
// tickets of a wave in one launch)
struct fill_rec {
    int32_t* p;
    int32_t v;
    int n;
    int gx, gy, gz;
};

__global__ void k_fill_b(const __grid_constant__ BPack<fill_rec> p) {
    const fill_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    for (int e = threadIdx.x; e < r.n; e += blockDim.x) r.p[e] = r.v;
}

// info[n] = kept Krylov width (Krylov path) or I_n (Gram path); info[N+n] = path;
// info[2N] = the request's error word (nonzero: a bounded wait of the tensor-core Gram pass
// expired); q_used[n] = q or 0
struct info_rec {
    int32_t* info;
    int32_t* q_used;
    const int32_t* err;
    int N, q;
    int32_t gram[RBKI_MAX_ORDER];
    int32_t dim[RBKI_MAX_ORDER];
    const int32_t* kept[RBKI_MAX_ORDER];
    int gx, gy, gz;
};

__global__ void k_info_b(const __grid_constant__ BPack<info_rec> p) {
    const info_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    const int n = threadIdx.x;
    if (n >= r.N) return;
    if (r.info) {
        r.info[n] = r.gram[n] ? r.dim[n] : *r.kept[n];
        r.info[r.N + n] = r.gram[n];
        if (n == 0) r.info[2 * r.N] = *r.err;
    }
    if (r.q_used) r.q_used[n] = r.gram[n] ? 0 : r.q;
}

}  // namespace
}  // namespace rbki

// ---------------------------------------------------------------------------------------
// Work-queue granularity: steps (Gram pass) or tiles (mode products) per unit of an item.  A
// unit is one CTA: smaller units spread an item over more SMs, larger ones leave fewer
// partial sums to reduce.  The table holds the target steps per unit by (kind, I_n) bucket:
// a default, or the values measured by rbki_wave_autotune / read by rbki_wave_tune_load.
// ---------------------------------------------------------------------------------------
namespace rbki {
namespace {

constexpr int TUNE_KINDS = 2, TUNE_IB = 8;   // kind 0 Gram pass, 1 mode product; I_n in 32-buckets
constexpr int DEFAULT_STEPS[TUNE_KINDS] = {16, 4};
constexpr int MAX_UNITS = 32;                // bounds the partial sums of one item
std::mutex g_tune_mu;
int g_tune_steps[TUNE_KINDS][TUNE_IB];       // 0 = default
int tune_ib(int I) { return std::min(TUNE_IB - 1, std::max(0, (I - 1) / 32)); }
const char* const TUNE_NAMES[TUNE_KINDS] = {"gram", "ttm"};

int tuned_steps(int kind, int I) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int v = g_tune_steps[kind][tune_ib(I)];
    return v > 0 ? v : DEFAULT_STEPS[kind];
}

// steps per unit of an item with `steps` steps: depends only on the item's shape
int per_unit(int kind, int I, int steps) {
    const int want = tuned_steps(kind, I);
    return std::max(want, (int)cdiv(steps, MAX_UNITS));
}

}  // namespace
}  // namespace rbki

// ---------------------------------------------------------------------------------------
// Host side: plan, workspace and the lockstep schedule of one wave.
// ---------------------------------------------------------------------------------------
namespace rbki {
namespace {

constexpr size_t WAVE_ALIGN = 256;

struct WaveMode {
    const ModePlan* m = nullptr;
    double* G = nullptr;             // X_(n) X_(n)^T (I x I); the Gram path's Z
    double *Qall = nullptr, *Pall = nullptr, *Z = nullptr, *evec = nullptr, *eval = nullptr;
    double *syev_ws = nullptr, *orth_ws = nullptr, *atb_part = nullptr, *gemm_part = nullptr;
    int32_t* kept = nullptr;
    float *gpart = nullptr, *wpart = nullptr;
    int ksteps = 0, kpu = 1, units = 1;
    bool tc = false;                 // Gram pass on the tensor cores (64-column steps)
};

struct WaveReq {
    Plan pl;
    rbki_tensor X{};
    rbki_tucker_out out{};
    WaveMode mode[RBKI_MAX_ORDER];
    float* tbuf[2] = {nullptr, nullptr};
    int64_t tmax = 0;           // largest intermediate of the core chain (elements)
    double* sq_part = nullptr;
    double* norms = nullptr;    // out.norms or workspace
    int32_t* err = nullptr;     // device error word of the request's bounded waits
    int rnd = 0;                // rounding of X as it is read (RBKI_BF16 / RBKI_F16, 0: none)
};

rbki_status wave_check(const rbki_tensor* X, const rbki_params* prm, Plan& pl) {
    RBKI_TRY(make_plan(X, prm, pl));
    if (!pl.mixed) return set_error(RBKI_E_UNSUPPORTED, "batched path: BF16/FP16 products only");
    const uint32_t ok = RBKI_FLAG_SERIAL_MODES;
    if (prm->flags & ~ok) return set_error(RBKI_E_UNSUPPORTED, "batched path: flags other than SERIAL_MODES");
    if (prm->omega > 0.0 && prm->omega < 1.0) return set_error(RBKI_E_UNSUPPORTED, "batched path: column sampling");
    if (pl.N < 2) return set_error(RBKI_E_UNSUPPORTED, "batched path: order >= 2");
    if (pl.numel >= (int64_t)1 << 31) return set_error(RBKI_E_UNSUPPORTED, "batched path: tensor too large");
    for (int n = 0; n < pl.N; ++n) {
        const ModePlan& m = pl.mode[n];
        if (m.I > 256) return set_error(RBKI_E_UNSUPPORTED, "batched path: I_n > 256");
        if (m.R > 64 || m.S > 64) return set_error(RBKI_E_UNSUPPORTED, "batched path: R_n + p > 64");
        if (m.b > 192) return set_error(RBKI_E_UNSUPPORTED, "batched path: eigenproblem > 192");
    }
    return RBKI_OK;
}

struct Carve {
    char* base;
    size_t off = 0;
    template <class T> T* take(size_t count) {
        off = rup(off, WAVE_ALIGN);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

void wave_carve(WaveReq& q, Carve& cv) {
    Plan& pl = q.pl;
    int64_t cur[RBKI_MAX_ORDER];
    for (int n = 0; n < pl.N; ++n) cur[n] = pl.dims[n];
    for (int t = 0; t + 1 < pl.N; ++t) {
        cur[pl.order[t]] = pl.mode[pl.order[t]].R;
        int64_t e = 1;
        for (int n = 0; n < pl.N; ++n) e *= cur[n];
        q.tmax = std::max(q.tmax, e);
    }
    for (int n = 0; n < pl.N; ++n) {
        const ModePlan& m = pl.mode[n];
        WaveMode& w = q.mode[n];
        w.m = &m;
        const int I = (int)m.I;
        // the tensor-core Gram pass reads X in its storage format, so it needs X stored as the
        // products' 16-bit type; otherwise the CUDA-core pass rounds as it reads
        w.tc = q.X.dtype == pl.stream_dtype && (q.X.dtype == RBKI_BF16 || q.X.dtype == RBKI_F16);
        w.ksteps = (int)cdiv(m.A * m.C, w.tc ? TCK : KT);
        w.kpu = per_unit(0, I, w.ksteps);
        w.units = (int)cdiv(w.ksteps, w.kpu);
        w.gpart = cv.take<float>((size_t)w.units * I * I);
        const int ev = m.gram ? I : m.b;
        w.Z = cv.take<double>((size_t)ev * ev);
        w.evec = cv.take<double>((size_t)ev * m.R);
        w.eval = cv.take<double>((size_t)ev);
        w.syev_ws = cv.take<double>(syev_scratch_doubles(ev));
        w.kept = cv.take<int32_t>(1);
        if (m.gram) {
            w.G = w.Z;
        } else {
            w.G = cv.take<double>((size_t)I * I);
            w.wpart = cv.take<float>((size_t)w.units * I * m.S);
            w.Qall = cv.take<double>((size_t)I * m.b);
            w.Pall = cv.take<double>((size_t)I * m.b);
            w.orth_ws = cv.take<double>(orth_scratch_doubles(I, m.b - m.S, m.S));
            w.atb_part = cv.take<double>((size_t)atb_nchunks(I) * m.b * m.b);
            w.gemm_part = cv.take<double>(gemm_part_doubles(I, m.S, I));
        }
    }
    q.tbuf[0] = cv.take<float>((size_t)q.tmax);
    q.tbuf[1] = cv.take<float>((size_t)q.tmax);
    q.sq_part = cv.take<double>((size_t)cdiv(std::max(pl.numel, pl.ranks_numel), SQ_CHUNK));
    q.norms = cv.take<double>(2);
    q.err = cv.take<int32_t>(1);
}

rbki_status launch_ttm(const std::vector<ttm_rec>& recs, cudaStream_t st) {
    if (recs.empty()) return RBKI_OK;
    size_t sm = 0;
    for (const auto& r : recs) sm = std::max(sm, ttm_smem(r));
    static const size_t smax = max_dyn_smem(k_ttm_b);   // thread-safe, once
    if (sm > smax) return set_error(RBKI_E_UNSUPPORTED, "batched mode product: shared memory");
    return bat_launch(k_ttm_b, recs.data(), (int)recs.size(), NTHREADS, sm, st, "k_ttm_b");
}

// Algorithms 1-2 for every request of the wave, stage by stage.  Per Krylov-path mode the
// Krylov products are P_j = (X_(n) X_(n)^T) Q_j with X_(n) X_(n)^T formed once (I_n <= 256):
// one pass over X instead of q + 1, and FP64 products on the small matrix.
rbki_status run_wave(std::vector<WaveReq>& Q, cudaStream_t st, uint32_t wait_us = tc::WAIT_US_DEFAULT,
                     int stall = 0) {
    const int nq = (int)Q.size();
    // ---- |X|^2 ----
    {
        std::vector<sumsq_rec> sq;
        for (auto& q : Q)
            sq.push_back(sumsq_rec{q.X.data, q.X.dtype, q.pl.numel, q.sq_part, q.norms,
                                   (int)cdiv(q.pl.numel, SQ_CHUNK), 1, 1});
        RBKI_TRY(bat_launch(k_sumsq_part_b, sq.data(), nq, 256, 0, st, "k_sumsq_part_b"));
        for (auto& r : sq) r.gx = 1;
        RBKI_TRY(bat_launch(k_sumsq_fin_b, sq.data(), nq, 32, 0, st, "k_sumsq_fin_b"));
    }
    // ---- one pass per mode: X_(n) X_(n)^T, and W = X_(n) Omega (Algorithm 1 steps 1-2) on
    // Krylov-path modes; the Gram path's Z is X_(n) X_(n)^T itself ----
    int qmax = 0;
    {
        std::vector<gram_rec> gr;
        std::vector<gramtc_rec> gt[2];   // [C == 1]
        std::vector<greduce_rec> gd;
        std::vector<xreduce_rec> wd;
        std::vector<fill_rec> fk;
        for (auto& q : Q) {
            fk.push_back(fill_rec{q.err, 0, 1, 1, 1, 1});
            for (int n = 0; n < q.pl.N; ++n) {
                WaveMode& w = q.mode[n];
                const ModePlan& m = *w.m;
                const int I = (int)m.I;
                if (w.tc) {
                    gramtc_rec r{};
                    r.x = q.X.data;
                    r.fp16 = q.X.dtype == RBKI_F16 ? 1 : 0;
                    r.A = (int)m.A;
                    r.I = I;
                    r.C = (int)m.C;
                    r.nrb = (int)cdiv(I, 128);
                    r.npad = (int)rup(I, 16);
                    r.ksteps = w.ksteps;
                    r.kpu = w.kpu;
                    r.S = m.gram ? 0 : m.S;
                    r.S16 = m.gram ? 0 : (int)rup(m.S, 16);
                    r.seed = q.pl.seed;
                    r.mode = n;
                    r.gpart = w.gpart;
                    r.wpart = w.wpart;
                    r.err = q.err;
                    // G in columns [0, npad), W from rup(npad, 32); the epilogue reads whole
                    // 32-column groups, so both are counted rounded up to 32
                    r.tcols = (uint32_t)(rup(r.npad, 32) + rup(r.S16, 32) <= 256 ? 256 : 512);
                    r.wait_us = wait_us;
                    r.stall = stall;
                    r.gx = r.nrb * w.units;
                    r.gy = r.gz = 1;
                    gt[m.C == 1 ? 1 : 0].push_back(r);
                } else {
                    const int nb = (int)cdiv(I, GB), npair = nb * (nb + 1) / 2;
                    gram_rec r{};
                    r.x = q.X.data;
                    r.dtype = q.X.dtype;
                    r.rnd = q.X.dtype == q.pl.stream_dtype ? 0 : q.rnd;
                    r.A = (int)m.A;
                    r.I = I;
                    r.C = (int)m.C;
                    r.nb = nb;
                    r.npair = npair;
                    r.ksteps = w.ksteps;
                    r.kpu = w.kpu;
                    r.S = m.gram ? 0 : m.S;
                    r.seed = q.pl.seed;
                    r.mode = n;
                    r.gpart = w.gpart;
                    r.wpart = w.wpart;
                    r.gx = npair * w.units;
                    r.gy = r.gz = 1;
                    gr.push_back(r);
                }
                gd.push_back(greduce_rec{w.gpart, w.units, I, w.G, (int)cdiv((int64_t)I * I, 256), 1, 1});
                if (!m.gram) {
                    wd.push_back(xreduce_rec{w.wpart, w.units, I, m.S, m.S, w.Qall, m.b, nullptr, 0,
                                             orth_ticket(w.orth_ws), (int)cdiv((int64_t)I * m.S, 256), 1, 1});
                    fk.push_back(fill_rec{w.kept, 0, 1, 1, 1, 1});
                    qmax = std::max(qmax, m.q);
                }
            }
        }
        static const size_t gmax = max_dyn_smem(k_gram_b);
        static const size_t tmax0 = max_dyn_smem(k_gram_tc_b<false>);
        static const size_t tmax1 = max_dyn_smem(k_gram_tc_b<true>);
        if (GRAM_SMEM > gmax || GRAM_TC_SMEM > tmax0 || GRAM_TC_SMEM > tmax1)
            return set_error(RBKI_E_CUDA, "batched Gram pass: shared memory");
        RBKI_TRY(bat_launch(k_fill_b, fk.data(), (int)fk.size(), 32, 0, st, "k_fill_b"));
        RBKI_TRY(bat_launch(k_gram_tc_b<false>, gt[0].data(), (int)gt[0].size(), TCT, GRAM_TC_SMEM, st,
                            "k_gram_tc_b"));
        RBKI_TRY(bat_launch(k_gram_tc_b<true>, gt[1].data(), (int)gt[1].size(), TCT, GRAM_TC_SMEM, st,
                            "k_gram_tc_b"));
        RBKI_TRY(bat_launch(k_gram_b, gr.data(), (int)gr.size(), NTHREADS, GRAM_SMEM, st, "k_gram_b"));
        RBKI_TRY(bat_launch(k_greduce_b, gd.data(), (int)gd.size(), 256, 0, st, "k_greduce_b"));
        RBKI_TRY(bat_launch(k_xreduce_b, wd.data(), (int)wd.size(), 256, 0, st, "k_xreduce_b"));
    }
    // BCGS2 on block col0 of every listed item (two passes; the second counts kept columns)
    auto orth2 = [&](const std::vector<WaveMode*>& ws, const std::vector<int>& col0) -> rbki_status {
        std::vector<OrthItem> oi;
        for (size_t k = 0; k < ws.size(); ++k) {
            const ModePlan& m = *ws[k]->m;
            oi.push_back(OrthItem{ws[k]->Qall, m.b, m.I, col0[k], m.S, ws[k]->orth_ws, nullptr});
        }
        RBKI_TRY(orth_pass_batched(oi.data(), (int)oi.size(), TAU_DEFLATE, st));
        for (size_t k = 0; k < ws.size(); ++k) oi[k].kept = ws[k]->kept;
        return orth_pass_batched(oi.data(), (int)oi.size(), TAU_DEFLATE, st);
    };
    {
        std::vector<WaveMode*> ws;
        std::vector<int> c0;
        for (auto& q : Q)
            for (int n = 0; n < q.pl.N; ++n)
                if (!q.mode[n].m->gram) {
                    ws.push_back(&q.mode[n]);
                    c0.push_back(0);
                }
        RBKI_TRY(orth2(ws, c0));
    }
    // ---- step 3: K = [W, A W, ..., A^q W], block by block: P_j = (X X^T) Q_j (FP64) ----
    for (int j = 0; j <= qmax; ++j) {
        std::vector<GemmItem> gm;
        std::vector<blkcopy_rec> cp;
        std::vector<WaveMode*> ws;
        std::vector<int> c0;
        for (auto& q : Q)
            for (int n = 0; n < q.pl.N; ++n) {
                WaveMode& w = q.mode[n];
                const ModePlan& m = *w.m;
                if (m.gram || j > m.q) continue;
                const int I = (int)m.I;
                gm.push_back(GemmItem{false, I, m.S, I, w.G, I, w.Qall + j * m.S, m.b, w.Pall + j * m.S, m.b, 0.0,
                                      w.gemm_part});
                if (j < m.q) {
                    cp.push_back(blkcopy_rec{w.Pall + j * m.S, m.b, w.Qall + (j + 1) * m.S, m.b, I, m.S,
                                             (int)cdiv((int64_t)I * m.S, 256), 1, 1});
                    ws.push_back(&w);
                    c0.push_back((j + 1) * m.S);
                }
            }
        RBKI_TRY(gemm_f64_batched(gm.data(), (int)gm.size(), st));
        RBKI_TRY(bat_launch(k_blkcopy_b, cp.data(), (int)cp.size(), 256, 0, st, "k_blkcopy_b"));
        if (!ws.empty()) RBKI_TRY(orth2(ws, c0));
    }
    // ---- Remark 1: Z = Q^T [P_0 .. P_q]; steps 4-5: eigenvectors, U = Q U~(:, 1:R) ----
    {
        std::vector<AtbItem> ab;
        std::vector<sym_rec> sy;
        std::vector<EigItem> ei;
        std::vector<FormItem> fi;
        std::vector<CopyItem> ci;
        for (auto& q : Q)
            for (int n = 0; n < q.pl.N; ++n) {
                WaveMode& w = q.mode[n];
                const ModePlan& m = *w.m;
                const int ev = m.gram ? (int)m.I : m.b;
                if (!m.gram) {
                    ab.push_back(AtbItem{w.Qall, m.b, m.b, w.Pall, m.b, m.b, m.I, w.atb_part, w.Z, m.b});
                    sy.push_back(sym_rec{w.Z, m.b, (int)cdiv((int64_t)m.b * m.b, 256), 1, 1});
                }
                ei.push_back(EigItem{w.Z, ev, m.R, w.eval, w.evec, w.syev_ws});
                fi.push_back(m.gram ? FormItem{nullptr, 0, m.I, w.evec, ev, m.R, m.R, q.out.factors[n]}
                                    : FormItem{w.Qall, m.b, m.I, w.evec, ev, m.R, m.R, q.out.factors[n]});
                if (q.out.eigvals[n]) ci.push_back(CopyItem{w.eval, q.out.eigvals[n], m.R});
            }
        RBKI_TRY(atb_batched(ab.data(), (int)ab.size(), st));
        RBKI_TRY(bat_launch(k_sym_b, sy.data(), (int)sy.size(), 256, 0, st, "k_sym_b"));
        RBKI_TRY(syev_top_batched(ei.data(), (int)ei.size(), st));
        RBKI_TRY(form_factor_batched(fi.data(), (int)fi.size(), st));
        RBKI_TRY(copy_f64_batched(ci.data(), (int)ci.size(), st));
    }
    // ---- step 6: G = X x_1 U^(1)T ... x_N U^(N)T, largest shrink first ----
    int Nmax = 0;
    for (auto& q : Q) Nmax = std::max(Nmax, q.pl.N);
    std::vector<int64_t> cur((size_t)nq * RBKI_MAX_ORDER);
    for (int k = 0; k < nq; ++k)
        for (int n = 0; n < Q[k].pl.N; ++n) cur[k * RBKI_MAX_ORDER + n] = Q[k].pl.dims[n];
    for (int t = 0; t < Nmax; ++t) {
        std::vector<ttm_rec> tr;
        for (int k = 0; k < nq; ++k) {
            WaveReq& q = Q[k];
            const Plan& pl = q.pl;
            if (t >= pl.N) continue;
            int64_t* c = &cur[k * RBKI_MAX_ORDER];
            const int md = pl.order[t];
            const ModePlan& m = pl.mode[md];
            int64_t A = 1, Cc = 1;
            for (int i = 0; i < md; ++i) A *= c[i];
            for (int i = md + 1; i < pl.N; ++i) Cc *= c[i];
            ttm_rec r{};
            r.x = t == 0 ? q.X.data : q.tbuf[(t - 1) & 1];
            r.dtype = t == 0 ? q.X.dtype : RBKI_F32;
            r.rnd = t == 0 && q.X.dtype != pl.stream_dtype ? q.rnd : 0;
            r.A = (int)A;
            r.I = (int)c[md];
            r.C = (int)Cc;
            r.S = m.R;
            r.tiles = (int)cdiv(A * Cc, TT);
            r.tpu = per_unit(1, r.I, r.tiles);
            r.U = q.out.factors[md];
            r.ldu = m.R;
            const bool last = t == pl.N - 1;
            r.out = last ? (void*)q.out.core : (void*)q.tbuf[t & 1];
            r.odt = last ? RBKI_F64 : RBKI_F32;
            r.gx = (int)cdiv(r.tiles, r.tpu);
            r.gy = r.gz = 1;
            tr.push_back(r);
            c[md] = m.R;
        }
        RBKI_TRY(launch_ttm(tr, st));
    }
    // ---- |G|^2, info, q_used ----
    {
        std::vector<sumsq_rec> sq;
        std::vector<info_rec> in;
        for (auto& q : Q) {
            sq.push_back(sumsq_rec{q.out.core, RBKI_F64, q.pl.ranks_numel, q.sq_part, q.norms + 1,
                                   (int)cdiv(q.pl.ranks_numel, SQ_CHUNK), 1, 1});
            if (q.out.info || q.out.q_used) {
                info_rec r{};
                r.info = q.out.info;
                r.q_used = q.out.q_used;
                r.N = q.pl.N;
                r.q = q.pl.prm.q;
                for (int n = 0; n < q.pl.N; ++n) {
                    r.gram[n] = q.mode[n].m->gram ? 1 : 0;
                    r.err = q.err;
                    r.dim[n] = (int32_t)q.pl.dims[n];
                    r.kept[n] = q.mode[n].kept;
                }
                r.gx = r.gy = r.gz = 1;
                in.push_back(r);
            }
        }
        RBKI_TRY(bat_launch(k_sumsq_part_b, sq.data(), nq, 256, 0, st, "k_sumsq_part_b"));
        for (auto& r : sq) r.gx = 1;
        RBKI_TRY(bat_launch(k_sumsq_fin_b, sq.data(), nq, 32, 0, st, "k_sumsq_fin_b"));
        RBKI_TRY(bat_launch(k_info_b, in.data(), (int)in.size(), 32, 0, st, "k_info_b"));
    }
    return RBKI_OK;
}

rbki_status wave_prepare(int32_t count, const rbki_tensor* X, const rbki_params* prm, const rbki_tucker_out* out,
                         void* ws, std::vector<WaveReq>& Q, size_t* bytes) {
    if (count < 0) return set_error(RBKI_E_INVAL, "count < 0");
    if (count > 0 && (!X || !prm)) return set_error(RBKI_E_INVAL, "NULL tensor or params array");
    Q.assign((size_t)count, WaveReq());
    Carve cv{static_cast<char*>(ws)};
    for (int k = 0; k < count; ++k) {
        WaveReq& q = Q[k];
        RBKI_TRY(wave_check(&X[k], &prm[k], q.pl));
        q.X = X[k];
        q.rnd = q.pl.stream_dtype;
        if (out) {
            q.out = out[k];
            if (!q.out.core) return set_error(RBKI_E_INVAL, "out->core is NULL");
            for (int n = 0; n < q.pl.N; ++n)
                if (!q.out.factors[n]) return set_error(RBKI_E_INVAL, "out->factors[n] is NULL");
        }
        wave_carve(q, cv);
        if (q.out.norms) q.norms = q.out.norms;   // |X|^2, |G|^2 straight into the output
    }
    if (bytes) *bytes = rup(cv.off, WAVE_ALIGN);
    return RBKI_OK;
}

// ---- autotuner: the steps per unit of each kernel and I_n bucket, measured on the device ----
// A synthetic batch of 48 items (3rd-order BF16 tensors 128 x I x 128, mode 1: 16384 columns)
// runs each candidate after a warm-up launch; its time is the fastest of three timed runs of
// two launches (CUDA events on `st`); the fastest candidate replaces the default when it is
// at least 5% faster.
rbki_status autotune(cudaStream_t st, int* table) {
    const int cand[] = {2, 4, 8, 16, 32, 64};
    const int items = 48, A = 128, Cc = 128, Imax = 256, S = 32;
    const int64_t numel = (int64_t)A * Imax * Cc;
    void* x = nullptr;
    double* U = nullptr;
    float *part = nullptr, *tout = nullptr;
    const int ksteps = (int)cdiv((int64_t)A * Cc, KT), tiles = (int)cdiv((int64_t)A * Cc, TT);
    const size_t part_n = (size_t)MAX_UNITS * Imax * (Imax + S);   // one item's partials (units <= MAX_UNITS)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rbki_status rs = RBKI_OK;
    auto fail = [&](cudaError_t e, const char* w) { rs = set_cuda_error(e, w); };
    cudaError_t e;
    if ((e = cudaMalloc(&x, numel * 2)) != cudaSuccess) fail(e, "autotune: tensor");
    if (rs == RBKI_OK && (e = cudaMalloc(&U, (size_t)Imax * S * sizeof(double))) != cudaSuccess) fail(e, "autotune: U");
    if (rs == RBKI_OK && (e = cudaMalloc(&part, items * part_n * sizeof(float))) != cudaSuccess)
        fail(e, "autotune: partials");
    if (rs == RBKI_OK && (e = cudaMalloc(&tout, (size_t)items * A * S * Cc * sizeof(float))) != cudaSuccess)
        fail(e, "autotune: output");
    if (rs == RBKI_OK && (e = cudaMemsetAsync(x, 0x3f, numel * 2, st)) != cudaSuccess) fail(e, "autotune: fill");
    if (rs == RBKI_OK && (e = cudaMemsetAsync(U, 0, (size_t)Imax * S * sizeof(double), st)) != cudaSuccess)
        fail(e, "autotune: fill");
    if (rs == RBKI_OK && (e = cudaEventCreate(&e0)) != cudaSuccess) fail(e, "autotune: event");
    if (rs == RBKI_OK && (e = cudaEventCreate(&e1)) != cudaSuccess) fail(e, "autotune: event");
    static const size_t gmax = max_dyn_smem(k_gram_b);
    static const size_t tmax = max_dyn_smem(k_ttm_b);
    for (int kind = 0; kind < TUNE_KINDS && rs == RBKI_OK; ++kind) {
        for (int b = 0; b < TUNE_IB && rs == RBKI_OK; ++b) {
            const int I = 32 * (b + 1), nb = (int)cdiv(I, GB);
            float best = 1e30f, def = 1e30f;
            int arg = DEFAULT_STEPS[kind];
            for (int c : cand) {
                const int steps = kind == 0 ? ksteps : tiles;
                const int kpu = std::max(c, (int)cdiv(steps, MAX_UNITS)), units = (int)cdiv(steps, kpu);
                std::vector<gram_rec> gr;
                std::vector<ttm_rec> tr;
                for (int k = 0; k < items; ++k) {
                    if (kind == 0) {
                        gram_rec r{};
                        r.x = x;
                        r.dtype = RBKI_BF16;
                        r.A = A;
                        r.I = I;
                        r.C = Cc;
                        r.nb = nb;
                        r.npair = nb * (nb + 1) / 2;
                        r.ksteps = ksteps;
                        r.kpu = kpu;
                        r.S = S;
                        r.gpart = part + (size_t)k * part_n;
                        r.wpart = part + (size_t)k * part_n + (size_t)units * I * I;
                        r.gx = r.npair * units;
                        r.gy = r.gz = 1;
                        gr.push_back(r);
                    } else {
                        ttm_rec r{};
                        r.x = x;
                        r.dtype = RBKI_BF16;
                        r.A = A;
                        r.I = I;
                        r.C = Cc;
                        r.S = S;
                        r.tiles = tiles;
                        r.tpu = kpu;
                        r.U = U;
                        r.ldu = S;
                        r.out = tout + (size_t)k * A * S * Cc;
                        r.odt = RBKI_F32;
                        r.gx = units;
                        r.gy = r.gz = 1;
                        tr.push_back(r);
                    }
                }
                // a warm-up launch, then the fastest of 3 timed runs of 2 launches
                auto launch = [&]() -> rbki_status {
                    if (kind == 0) {
                        if (GRAM_SMEM > gmax) return set_error(RBKI_E_CUDA, "autotune: Gram shared memory");
                        return bat_launch(k_gram_b, gr.data(), items, NTHREADS, GRAM_SMEM, st, "k_gram_b");
                    }
                    const size_t sm = ttm_smem(tr[0]);
                    if (sm > tmax) return set_error(RBKI_E_CUDA, "autotune: mode-product shared memory");
                    return bat_launch(k_ttm_b, tr.data(), items, NTHREADS, sm, st, "k_ttm_b");
                };
                float ms = 1e30f;
                rs = launch();
                for (int run = 0; run < 3 && rs == RBKI_OK; ++run) {
                    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) fail(e, "autotune: record");
                    for (int l = 0; l < 2 && rs == RBKI_OK; ++l) rs = launch();
                    if (rs == RBKI_OK && (e = cudaEventRecord(e1, st)) != cudaSuccess) fail(e, "autotune: record");
                    if (rs == RBKI_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) fail(e, "autotune: sync");
                    float t = 0.f;
                    if (rs == RBKI_OK && (e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) fail(e, "autotune: time");
                    ms = std::min(ms, t);
                }
                if (rs == RBKI_OK && c == DEFAULT_STEPS[kind]) def = ms;
                if (rs == RBKI_OK && ms < best) {
                    best = ms;
                    arg = c;
                }
            }
            // keep the default unless a candidate is clearly faster (timing noise is a few %)
            table[kind * TUNE_IB + b] = best < 0.95f * def ? arg : DEFAULT_STEPS[kind];
        }
    }
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(U);
    cudaFree(part);
    cudaFree(tout);
    return rs;
}

}  // namespace
}  // namespace rbki

using namespace rbki;

extern "C" {

rbki_status rbki_wave_autotune(void* stream) {
    int table[TUNE_KINDS * TUNE_IB];
    RBKI_TRY(autotune(static_cast<cudaStream_t>(stream), table));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int k = 0; k < TUNE_KINDS; ++k)
        for (int b = 0; b < TUNE_IB; ++b) g_tune_steps[k][b] = table[k * TUNE_IB + b];
    return RBKI_OK;
}

rbki_status rbki_wave_tune_get(int32_t kind, int32_t bucket, int32_t* steps) {
    if (kind < 0 || kind >= TUNE_KINDS || bucket < 0 || bucket >= TUNE_IB || !steps)
        return set_error(RBKI_E_INVAL, "kind / bucket out of range or steps is NULL");
    *steps = tuned_steps(kind, 32 * (bucket + 1));
    return RBKI_OK;
}

rbki_status rbki_wave_tune_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& row : g_tune_steps)
        for (int& v : row) v = 0;
    return RBKI_OK;
}

rbki_status rbki_wave_tune_save(const char* path) {
    if (!path) return set_error(RBKI_E_INVAL, "path is NULL");
    FILE* f = std::fopen(path, "w");
    if (!f) return set_error(RBKI_E_INVAL, "cannot open the tuning file for writing");
    std::fprintf(f, "# rbki wave tuning table v1: kind I_n-bucket(32*(b+1)) steps-per-unit\n");
    for (int k = 0; k < TUNE_KINDS; ++k)
        for (int b = 0; b < TUNE_IB; ++b) std::fprintf(f, "%s %d %d\n", TUNE_NAMES[k], b, tuned_steps(k, 32 * (b + 1)));
    const bool ok = std::fclose(f) == 0;
    return ok ? RBKI_OK : set_error(RBKI_E_INVAL, "writing the tuning file failed");
}

rbki_status rbki_wave_tune_load(const char* path) {
    if (!path) return set_error(RBKI_E_INVAL, "path is NULL");
    FILE* f = std::fopen(path, "r");
    if (!f) return set_error(RBKI_E_NOTFOUND, "cannot open the tuning file");
    int table[TUNE_KINDS][TUNE_IB] = {};
    char line[256];
    rbki_status rs = RBKI_OK;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        char name[16];
        int b = -1, v = 0;
        if (std::sscanf(line, "%15s %d %d", name, &b, &v) != 3 || b < 0 || b >= TUNE_IB || v < 1 || v > 4096) {
            rs = set_error(RBKI_E_INVAL, "malformed line in the tuning file");
            break;
        }
        int k = -1;
        for (int i = 0; i < TUNE_KINDS; ++i)
            if (std::strcmp(name, TUNE_NAMES[i]) == 0) k = i;
        if (k < 0) {
            rs = set_error(RBKI_E_INVAL, "unknown kernel kind in the tuning file");
            break;
        }
        table[k][b] = v;
    }
    std::fclose(f);
    if (rs < 0) return rs;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (int k = 0; k < TUNE_KINDS; ++k)
        for (int b = 0; b < TUNE_IB; ++b) g_tune_steps[k][b] = table[k][b];
    return RBKI_OK;
}

rbki_status rbki_tucker_batched_workspace(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                                          size_t* bytes) {
    if (!bytes) return set_error(RBKI_E_INVAL, "bytes is NULL");
    std::vector<WaveReq> Q;
    return wave_prepare(count, X, prm, nullptr, nullptr, Q, bytes);
}

// ---- captured waves: the whole schedule of one wave as a CUDA graph, replayed per batch ----
struct rbki_batched_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;   // kernel nodes per replay
};

rbki_status rbki_batched_plan_create(int32_t count, const rbki_tensor* X, const rbki_params* prm, void* workspace,
                                     size_t workspace_bytes, const rbki_tucker_out* out, void* stream,
                                     rbki_batched_plan** plan) {
    if (!plan) return set_error(RBKI_E_INVAL, "plan is NULL");
    *plan = nullptr;
    if (count < 1) return set_error(RBKI_E_INVAL, "count must be >= 1");
    if (!out) return set_error(RBKI_E_INVAL, "out is NULL");
    size_t need = 0;
    std::vector<WaveReq> Q;
    RBKI_TRY(wave_prepare(count, X, prm, out, nullptr, Q, &need));
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    RBKI_TRY(wave_prepare(count, X, prm, out, workspace, Q, &need));
    for (const auto& q : Q)
        if (!q.X.data) return set_error(RBKI_E_INVAL, "X->data is NULL");
    cudaStream_t user = static_cast<cudaStream_t>(stream);
    // one eager run sets up every kernel's shared-memory opt-in before the capture (and
    // leaves valid outputs); the capture runs on a private stream ordered after `stream`
    RBKI_TRY(run_wave(Q, user));
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    RBKI_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    auto cleanup = [&] {
        if (ev) cudaEventDestroy(ev);
        cudaStreamDestroy(cs);
    };
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    if (e != cudaSuccess) {
        cleanup();
        return set_cuda_error(e, "batched plan: ordering");
    }
    rbki_batched_plan* p = new rbki_batched_plan();
    const uint64_t l0 = rbki_kernel_launches();
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    rbki_status rs = e == cudaSuccess ? run_wave(Q, cs) : set_cuda_error(e, "batched plan: begin capture");
    if (e == cudaSuccess) {
        const cudaError_t e2 = cudaStreamEndCapture(cs, &p->graph);
        if (rs >= 0 && e2 != cudaSuccess) rs = set_cuda_error(e2, "batched plan: end capture");
    }
    p->kernels = rbki_kernel_launches() - l0;
    drop_launches(p->kernels);   // recorded into the graph, not launched
    if (rs >= 0) {
        e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (e != cudaSuccess) rs = set_cuda_error(e, "batched plan: instantiate");
    }
    cleanup();
    if (rs < 0) {
        rbki_batched_plan_destroy(p);
        return rs;
    }
    *plan = p;
    return RBKI_OK;
}

rbki_status rbki_batched_plan_launch(rbki_batched_plan* plan, void* stream) {
    if (!plan || !plan->exec) return set_error(RBKI_E_INVAL, "plan is NULL");
    RBKI_CUDA_TRY(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)));
    add_launches(plan->kernels);
    return RBKI_OK;
}

rbki_status rbki_batched_plan_destroy(rbki_batched_plan* plan) {
    if (!plan) return set_error(RBKI_E_INVAL, "plan is NULL");
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
    return RBKI_OK;
}

rbki_status rbki_diag_batched_stall(int32_t count, const rbki_tensor* X, const rbki_params* prm, void* workspace,
                                   size_t workspace_bytes, const rbki_tucker_out* out, uint32_t wait_us,
                                   void* stream) {
    if (count < 1 || !out) return set_error(RBKI_E_INVAL, "count must be >= 1 and out non-NULL");
    if (wait_us < 1 || wait_us > tc::WAIT_US_DEFAULT) return set_error(RBKI_E_INVAL, "wait_us out of range");
    size_t need = 0;
    std::vector<WaveReq> Q;
    RBKI_TRY(wave_prepare(count, X, prm, out, nullptr, Q, &need));
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    RBKI_TRY(wave_prepare(count, X, prm, out, workspace, Q, &need));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RBKI_TRY(run_wave(Q, st, wait_us, 1));
    RBKI_CUDA_TRY(cudaStreamSynchronize(st));
    int any = 0;
    for (const auto& q : Q) {
        int32_t e = 0;
        RBKI_CUDA_TRY(cudaMemcpy(&e, q.err, sizeof(e), cudaMemcpyDeviceToHost));
        any |= e;
    }
    return any ? set_error(RBKI_E_TIMEOUT, "a bounded wait inside the Gram pass expired") : RBKI_OK;
}

rbki_status rbki_tucker_batched(int32_t count, const rbki_tensor* X, const rbki_params* prm, void* workspace,
                                size_t workspace_bytes, const rbki_tucker_out* out, void* stream) {
    if (count == 0) return RBKI_OK;
    if (!out) return set_error(RBKI_E_INVAL, "out is NULL");
    size_t need = 0;
    std::vector<WaveReq> Q;
    RBKI_TRY(wave_prepare(count, X, prm, out, nullptr, Q, &need));
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    RBKI_TRY(wave_prepare(count, X, prm, out, workspace, Q, &need));
    for (const auto& q : Q)
        if (!q.X.data) return set_error(RBKI_E_INVAL, "X->data is NULL");
    return run_wave(Q, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
