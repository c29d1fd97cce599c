// Tensor-core (tcgen05 / TMEM / TMA) streaming kernels for the mixed path on sm_103a.
//
// One kernel template streams X once per launch over the native C-order layout, viewed
// per mode as [A][I][C], in tiles of 128 unfolding columns x all I rows:
//   KRYLOV  P += X_tile (X_tile^T Q)      Algorithm 1 step 3 / Eq. BKspace: one X read per step
//   SKETCH  P += X_tile Omega_tile        Algorithm 1 step 2 (W = X Omega)
//   TTM     Y  = X_tile^T U  (stored)     Algorithm 2 step 6, first mode product of the core
// Operands are BF16 (or FP16) with FP32 accumulation in tensor memory.  With `split`, the
// skinny operand is carried as a hi + lo pair of BF16 values (N doubles), which makes the
// products accurate to ~FP32 against BF16-exact X.
//
// Data movement: TMA tiled loads with 128-byte swizzle, boxes of 64 (contiguous dim) x
// 128 rows; a "slab" is 128 rows x 128 columns = two boxes = 32 KB.  Three layouts of X in
// shared memory are consumed directly by the tensor core:
//   C > 1 ("CFAST", columns contiguous): GEMM1 reads X^T as an MN-major operand, GEMM2 reads
//        X as a K-major operand;  C == 1 ("IFAST", rows contiguous): the roles swap.
// Warp roles (192 threads): warp 0 TMA producer, warp 1 MMA issuer + TMEM owner, warps 2-5
// epilogue (TMEM -> registers -> BF16 operand image in shared memory / global stores).
// Every mbarrier wait is bounded; on expiry the CTA raises an abort flag, every role leaves
// its loop, the producer waits (bounded) for each copy it issued and the MMA issuer for every
// MMA it issued, and only then is tensor memory freed; the error word is set.
#include <cuda.h>

#include "kernels.h"
#include "tc.h"
#include "dfloat.cuh"
#include "tc_ptx.cuh"

namespace rbki {
namespace tc {
namespace {

constexpr int SLAB_BYTES = 32768;
constexpr int BOX_BYTES = 16384;
constexpr int NTHREADS = 192;

template <int MODE, bool IFAST>
__global__ void __launch_bounds__(NTHREADS, 1) k_stream_tc(const __grid_constant__ CUtensorMap tmap, const Params p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nslot = p.nslot, NS = p.NS, N = p.N;
    uint64_t* bars = (uint64_t*)(smem + p.smem_bar);
    const uint32_t b_full = smem_u32(bars), b_empty = b_full + 8 * nslot;
    const uint32_t b_yfull = b_empty + 8 * nslot, b_yready = b_yfull + 16, b_ysfree = b_yready + 16;
    const uint32_t b_omfull = b_ysfree + 16, b_qfull = b_omfull + 16, b_pdone = b_qfull + 8;
    const uint32_t b_drain = b_pdone + 8, b_never = b_drain + 8;
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * nslot + 12);
    const uint32_t lim = p.wait_us;
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
            mbar_init(b_omfull + 8 * i, 1);
        }
        mbar_init(b_qfull, 1);
        mbar_init(b_pdone, 1);
        mbar_init(b_drain, 1);
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
    const uint32_t X0 = sbase + p.smem_x, Q0 = sbase + p.smem_q, Y0 = sbase + p.smem_y;
    const uint32_t ycol0 = (MODE == TTM) ? 0u : (uint32_t)(NS * N);
    const bool fp16 = p.fp16 != 0;

    if (warp == 0) {
        // ------------------------------ TMA producer ------------------------------
        if (lane == 0) {
            // parity of the last load issued into each slot / Omega buffer, to drain them
            uint32_t issued = 0, par = 0, om_issued = 0, om_par = 0;
            if (MODE != SKETCH) {
                mbar_expect_tx(b_qfull, p.qimg_bytes);
                for (uint32_t off = 0; off < p.qimg_bytes; off += 32768) {
                    uint32_t sz = min(32768u, p.qimg_bytes - off);
                    bulk_load(Q0 + off, (const uint8_t*)p.qimg + off, sz, b_qfull);
                }
            }
            uint32_t slot = 0, phase = 0;
            for (int64_t k = 0; k < my_tiles && !*abort_flag; ++k) {
                const int64_t t = blockIdx.x + k * gridDim.x;
                int ca = 0, cc = 0;   // TMA coordinates of the tile
                if (!IFAST) {
                    ca = (int)(t / p.ctiles);
                    cc = (int)((t % p.ctiles) * 128);
                } else {
                    ca = (int)(t * 128);
                }
                if (MODE == SKETCH) {
                    const int b = (int)(k & 1);
                    if (k >= 2 && !mbar_wait(b_ysfree + 8 * b, (uint32_t)(((k - 2) >> 1) & 1), abort_flag, lim)) break;
                    mbar_expect_tx(b_omfull + 8 * b, p.yimg_bytes);
                    bulk_load(Y0 + b * p.yimg_bytes, (const uint8_t*)p.omg + (size_t)t * p.yimg_bytes, p.yimg_bytes,
                              b_omfull + 8 * b);
                    om_issued |= 1u << b;
                    om_par = (om_par & ~(1u << b)) | ((uint32_t)((k >> 1) & 1) << b);
                }
                for (int s = 0; s < NS; ++s) {
                    if (!mbar_wait(b_empty + 8 * slot, phase ^ 1, abort_flag, lim)) break;
                    mbar_expect_tx(b_full + 8 * slot, SLAB_BYTES);
                    const uint32_t dst = X0 + slot * SLAB_BYTES;
                    if (!IFAST) {
                        tma_load_3d(dst, &tmap, b_full + 8 * slot, cc, 128 * s, ca);
                        tma_load_3d(dst + BOX_BYTES, &tmap, b_full + 8 * slot, cc + 64, 128 * s, ca);
                    } else {
                        tma_load_2d(dst, &tmap, b_full + 8 * slot, 128 * s, ca);
                        tma_load_2d(dst + BOX_BYTES, &tmap, b_full + 8 * slot, 128 * s + 64, ca);
                    }
                    issued |= 1u << slot;
                    par = (par & ~(1u << slot)) | (phase << slot);
                    if (++slot == (uint32_t)nslot) { slot = 0; phase ^= 1; }
                }
            }
            // drain: every copy issued into this CTA's shared memory lands before it exits
            if (MODE != SKETCH) mbar_drain(b_qfull, 0, lim);
            for (int i = 0; i < nslot; ++i)
                if (issued >> i & 1) mbar_drain(b_full + 8 * i, par >> i & 1, lim);
            for (int i = 0; i < 2; ++i)
                if (om_issued >> i & 1) mbar_drain(b_omfull + 8 * i, om_par >> i & 1, lim);
        }
    } else if (warp == 1) {
        // ------------------------------ MMA issuer ------------------------------
        // Shared-memory descriptors are built once: a slab's or a K-step's descriptor is
        // the base descriptor plus its byte offset in 16-byte units (shared addresses stay
        // below 2^18, so the 14-bit address field never carries).  The issue loop then costs
        // a few independent adds per MMA instead of a dependent chain of shifts and masks.
        if (lane == 0) {
            const uint32_t id1 = idesc_f16(128, N, /*a_mn=*/!IFAST, /*b_mn=*/true, fp16);   // Y = X^T Q
            const uint32_t id2 = idesc_f16(128, N, /*a_mn=*/IFAST, /*b_mn=*/true, fp16);    // P += X Y
            const uint32_t qlbo = (uint32_t)(N / 8) * 128u;
            const uint64_t dx1 = IFAST ? sdesc(X0, 16, 1024, LAYOUT_SW128) : sdesc(X0, BOX_BYTES, 1024, LAYOUT_SW128);
            const uint64_t dx2 = IFAST ? sdesc(X0, BOX_BYTES, 1024, LAYOUT_SW128) : sdesc(X0, 16, 1024, LAYOUT_SW128);
            const uint64_t dq = sdesc(Q0, qlbo, 128, LAYOUT_NONE);
            const uint64_t dy = sdesc(Y0, 128, 2048, LAYOUT_NONE);
            const uint32_t qstep = (2u * qlbo) >> 4;     // one K = 16 step of the Q image
            bool ok = true;
            if (p.stall) ok = mbar_wait(b_never, 0, abort_flag, lim);   // expires by design
            if (ok && MODE != SKETCH) ok = mbar_wait(b_qfull, 0, abort_flag, lim);
            uint32_t slot = 0, phase = 0;
            for (int64_t k = 0; ok && k < my_tiles; ++k) {
                const int b = (int)(k & 1);
                const uint32_t slot0 = slot, phase0 = phase;
                if (MODE != SKETCH) {
                    if (MODE == TTM && k >= 2 && !mbar_wait(b_yready + 8 * b, (uint32_t)(((k - 2) >> 1) & 1), abort_flag, lim)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ytm = tbase + ycol0 + (uint32_t)(b * N);
                    for (int s = 0; s < NS && ok; ++s) {
                        if (!mbar_wait(b_full + 8 * slot, phase, abort_flag, lim)) { ok = false; break; }
                        tc_fence_after();
                        const uint64_t a0 = dx1 + ((slot * SLAB_BYTES) >> 4);
                        const uint64_t b0 = dq + (uint64_t)(s * 8) * qstep;
                        umma_f16(ytm, a0, b0, id1, s != 0 ? 1u : 0u);
#pragma unroll
                        for (int kk = 1; kk < 8; ++kk) {
                            const uint32_t ko = IFAST ? (uint32_t)(((kk >> 2) * BOX_BYTES + (kk & 3) * 32) >> 4)
                                                      : (uint32_t)((kk * 2048) >> 4);
                            umma_f16(ytm, a0 + ko, b0 + (uint64_t)kk * qstep, id1, 1u);
                        }
                        if (MODE == TTM) umma_commit(b_empty + 8 * slot);
                        if (++slot == (uint32_t)nslot) { slot = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    umma_commit(b_yfull + 8 * b);
                }
                if (MODE != TTM) {
                    const uint32_t rb = (MODE == KRYLOV) ? b_yready + 8 * b : b_omfull + 8 * b;
                    if (!mbar_wait(rb, (uint32_t)((k >> 1) & 1), abort_flag, lim)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t y0 = dy + (uint64_t)((b * p.yimg_bytes) >> 4);
                    uint32_t sl = slot0, ph = phase0;
                    for (int s = 0; s < NS; ++s) {
                        if (MODE == SKETCH) {
                            if (!mbar_wait(b_full + 8 * sl, ph, abort_flag, lim)) { ok = false; break; }
                            tc_fence_after();
                        }
                        const uint64_t a0 = dx2 + ((sl * SLAB_BYTES) >> 4);
                        const uint32_t ptm = tbase + (uint32_t)(s * N);
                        umma_f16(ptm, a0, y0, id2, k > 0 ? 1u : 0u);
#pragma unroll
                        for (int kk = 1; kk < 8; ++kk) {
                            const uint32_t ko = IFAST ? (uint32_t)((kk * 2048) >> 4)
                                                      : (uint32_t)(((kk >> 2) * BOX_BYTES + (kk & 3) * 32) >> 4);
                            umma_f16(ptm, a0 + ko, y0 + (uint64_t)(kk * 16), id2, 1u);
                        }
                        umma_commit(b_empty + 8 * sl);
                        if (++sl == (uint32_t)nslot) { sl = 0; ph ^= 1; }
                    }
                    if (!ok) break;
                    umma_commit(b_ysfree + 8 * b);
                    if (MODE == SKETCH) { slot = sl; phase = ph; }
                }
            }
            if (MODE != TTM && ok) umma_commit(b_pdone);
            // drain: every MMA this thread issued completes before tensor memory is freed
            umma_commit(b_drain);
            if (!mbar_drain(b_drain, 0, lim)) *abort_flag = 1;
        }
    } else {
        // ------------------------------ epilogue (warps 2-5) ------------------------------
        const int q = warp & 3;
        const int row = q * 32 + lane;                  // tile column (TMEM lane)
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float v[64];
        if (MODE != SKETCH) {
            for (int64_t k = 0; k < my_tiles; ++k) {
                const int b = (int)(k & 1);
                if (!mbar_wait(b_yfull + 8 * b, (uint32_t)((k >> 1) & 1), abort_flag, lim)) break;
                tc_fence_after();
                const uint32_t ytm = tbase + ycol0 + (uint32_t)(b * N) + lane_off;
                tmem_ld32(ytm, v);
                if (N > 32) tmem_ld32(ytm + 32, v + 32);
                const int Sh = p.Sh;
                if (p.split)
                    for (int s = 0; s < Sh; ++s) v[s] += v[N / 2 + s];
                if (MODE == TTM) {
                    tc_fence_before();
                    mbar_arrive(b_yready + 8 * b);
                    const int64_t t = blockIdx.x + k * gridDim.x;
                    if (p.yimg_out) {
                        // Y as the tile's operand image for a later SKETCH pass: element (c, n)
                        // at (n/8)*1024 + c*8 + n%8; zero past Sh and for columns outside X
                        const bool valid = !IFAST ? (t % p.ctiles) * 128 + row < p.C : t * 128 + row < p.A;
                        for (int s = 0; s < N; ++s)
                            if (!valid || s >= Sh) v[s] = 0.f;
                        uint16_t* base = (uint16_t*)p.yimg_out + (size_t)t * 128 * N;
                        for (int g = 0; g < N / 8; ++g) {
                            uint4 w;
                            w.x = pack2(v[8 * g + 0], v[8 * g + 1], fp16);
                            w.y = pack2(v[8 * g + 2], v[8 * g + 3], fp16);
                            w.z = pack2(v[8 * g + 4], v[8 * g + 5], fp16);
                            w.w = pack2(v[8 * g + 6], v[8 * g + 7], fp16);
                            *reinterpret_cast<uint4*>(base + g * 1024 + row * 8) = w;
                        }
                    } else if (!IFAST) {
                        const int64_t a = t / p.ctiles, c = (t % p.ctiles) * 128 + row;
                        if (c < p.C)
                            for (int s = 0; s < Sh; ++s) p.yout[(a * Sh + s) * p.C + c] = v[s];
                    } else {
                        const int64_t a = t * 128 + row;
                        if (a < p.A)
                            for (int s = 0; s < Sh; ++s) p.yout[a * Sh + s] = v[s];
                    }
                } else {
                    if (k >= 2 && !mbar_wait(b_ysfree + 8 * b, (uint32_t)(((k - 2) >> 1) & 1), abort_flag, lim)) break;
                    // BF16 operand image of Y (MN-major, no swizzle): element (c, n) at
                    // (n/8)*2048 + c*16 + (n%8)*2
                    uint8_t* img = smem + p.smem_y + (size_t)b * p.yimg_bytes;
                    if (p.split) {
                        for (int s = 0; s < Sh; ++s) {
                            float hi = round_lo(v[s], fp16);
                            v[N / 2 + s] = v[s] - hi;
                            v[s] = hi;
                        }
                    }
                    for (int g = 0; g < N / 8; ++g) {
                        uint4 w;
                        w.x = pack2(v[8 * g + 0], v[8 * g + 1], fp16);
                        w.y = pack2(v[8 * g + 2], v[8 * g + 3], fp16);
                        w.z = pack2(v[8 * g + 4], v[8 * g + 5], fp16);
                        w.w = pack2(v[8 * g + 6], v[8 * g + 7], fp16);
                        *reinterpret_cast<uint4*>(img + g * 2048 + row * 16) = w;
                    }
                    fence_async_smem();
                    tc_fence_before();
                    mbar_arrive(b_yready + 8 * b);
                }
            }
        }
        if (MODE != TTM) {
            if (mbar_wait(b_pdone, 0, abort_flag, lim)) {
                tc_fence_after();
                float* out = p.part + (size_t)blockIdx.x * p.I * N;
                for (int s = 0; s < NS; ++s) {
                    const uint32_t ptm = tbase + (uint32_t)(s * N) + lane_off;
                    tmem_ld32(ptm, v);
                    if (N > 32) tmem_ld32(ptm + 32, v + 32);
                    const int64_t i = (int64_t)s * 128 + row;
                    if (i < p.I) {
                        float4* o = reinterpret_cast<float4*>(out + i * N);
                        for (int g = 0; g < N / 4; ++g) o[g] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
                    }
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

// ---- operand images ----
// B image of a skinny FP64 matrix M (rows x S, ld ldm) for GEMM1: MN-major no-swizzle,
// element (i, n) at (i/8)*(N/8)*128 + (n/8)*128 + (i%8)*16 + (n%8)*2; rows padded to
// rows_pad; columns n < S hold hi (or the value), N/2 <= n < N/2 + S the lo part when
// split == 1 (S <= N/2); split == 2 puts the lo parts alone in columns n < S.
__device__ __forceinline__ void skinny_image_dev(const double* __restrict__ M, int64_t ldm, int64_t rows, int S,
                                                 int64_t rows_pad, int N, int split, int fp16, uint16_t* __restrict__ img, int bx) {
    int64_t e = (int64_t)bx * blockDim.x + threadIdx.x;
    if (e >= rows_pad * N) return;
    int64_t i = e / N;
    int n = (int)(e % N);
    float val = 0.f;
    const bool lo_half = split == 1 && n >= N / 2;
    int s = lo_half ? n - N / 2 : n;
    if (i < rows && s < S) {
        double x = M[i * ldm + s];
        float hi = fp16 ? __half2float(__double2half(x)) : __bfloat162float(__double2bfloat16(x));
        val = (lo_half || split == 2) ? (float)(x - (double)hi) : hi;
    }
    uint16_t bits;
    if (fp16) { __half h = __float2half_rn(val); bits = *reinterpret_cast<uint16_t*>(&h); }
    else { __nv_bfloat16 h = __float2bfloat16_rn(val); bits = *reinterpret_cast<uint16_t*>(&h); }
    int64_t off = (i / 8) * (N / 8) * 64 + (n / 8) * 64 + (i % 8) * 8 + (n % 8);   // in elements
    img[off] = bits;
}

__global__ void k_skinny_image(const double* __restrict__ M, int64_t ldm, int64_t rows, int S,
                               int64_t rows_pad, int N, int split, int fp16, uint16_t* __restrict__ img) {
    skinny_image_dev(M, ldm, rows, S, rows_pad, N, split, fp16, img, (int)blockIdx.x);
}

struct skinny_image_rec {
    const double* M;
    int64_t ldm;
    int64_t rows;
    int S;
    int64_t rows_pad;
    int N;
    int split;
    int fp16;
    uint16_t* img;
    int gx, gy, gz;
};

__global__ void k_skinny_image_b(const __grid_constant__ BPack<skinny_image_rec> p) {
    const skinny_image_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    skinny_image_dev(r.M, r.ldm, r.rows, r.S, r.rows_pad, r.N, r.split, r.fp16, r.img, bx);
}


// Per-tile Omega images for SKETCH: tile t covers 128 unfolding columns; element (c, n) of
// tile t at t*128*N + (n/8)*1024 + c*8 + n%8 (elements).  Columns outside the tensor are 0.
// With `split`, image column n < S holds the hi part of Omega's column n and N/2 + s the lo
// part of column s.
// element e = (tile, column c, group of 8 image columns), 0 <= e < tiles * 128 * N / 8: the
// group is written as one 16-byte vector, zeros included, so the image needs no clearing
__device__ __forceinline__ void omega_image_elem(uint64_t seed, int mode, int64_t A, int64_t C, int ifast,
                                                 int64_t ctiles, int S, int N, int split, int fp16,
                                                 uint16_t* __restrict__ img, int64_t e) {
    const int G = N / 8;
    const int g = (int)(e % G);
    const int64_t tc_ = e / G;
    const int c = (int)(tc_ & 127);
    const int64_t t = tc_ >> 7;
    int64_t col;
    bool valid;
    if (!ifast) {
        const int64_t a = t / ctiles, cc = (t % ctiles) * 128 + c;
        valid = cc < C;
        col = a * C + cc;
    } else {
        const int64_t a = t * 128 + c;
        valid = a < A;
        col = a;
    }
    float vals[8];
    int have_pair = -1;
    float z[2] = {0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int n = 8 * g + u;
        const bool lo = split && n >= N / 2;
        const int s = lo ? n - N / 2 : n;
        float v = 0.f;
        if (valid && s < S) {
            if (s / 2 != have_pair) {
                omega_pair_f32(seed, (uint32_t)mode, (uint64_t)col, (uint32_t)(s / 2), z[0], z[1]);
                have_pair = s / 2;
            }
            const float x = z[s & 1];
            const float hi = fp16 ? __half2float(__float2half_rn(x)) : __bfloat162float(__float2bfloat16_rn(x));
            v = lo ? x - hi : hi;
        }
        vals[u] = v;
    }
    uint4 w;
    w.x = pack2(vals[0], vals[1], fp16 != 0);
    w.y = pack2(vals[2], vals[3], fp16 != 0);
    w.z = pack2(vals[4], vals[5], fp16 != 0);
    w.w = pack2(vals[6], vals[7], fp16 != 0);
    *reinterpret_cast<uint4*>(img + (size_t)t * 128 * N + (size_t)g * 1024 + c * 8) = w;
}

// one thread per element
__device__ __forceinline__ void omega_images_dev(uint64_t seed, int mode, int64_t A, int64_t C, int ifast,
                                                 int64_t ctiles, int64_t tiles, int S, int N, int split,
                                                 int fp16, uint16_t* __restrict__ img, int bx) {
    const int64_t e = (int64_t)bx * blockDim.x + threadIdx.x;
    if (e >= tiles * 128 * (N / 8)) return;
    omega_image_elem(seed, mode, A, C, ifast, ctiles, S, N, split, fp16, img, e);
}

__global__ void __launch_bounds__(256) k_omega_images(uint64_t seed, int mode, int64_t A, int64_t C, int ifast,
                                                      int64_t ctiles, int64_t tiles, int S, int N, int split,
                                                      int fp16, uint16_t* __restrict__ img) {
    omega_images_dev(seed, mode, A, C, ifast, ctiles, tiles, S, N, split, fp16, img, (int)blockIdx.x);
}

struct omega_images_rec {
    uint64_t seed;
    int mode;
    int64_t A;
    int64_t C;
    int ifast;
    int64_t ctiles;
    int64_t tiles;
    int S;
    int N;
    int split;
    int fp16;
    uint16_t* img;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_omega_images_b(const __grid_constant__ BPack<omega_images_rec> p) {
    const omega_images_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    omega_images_dev(r.seed, r.mode, r.A, r.C, r.ifast, r.ctiles, r.tiles, r.S, r.N, r.split, r.fp16, r.img, bx);
}


// The staging cast of X (FP32 -> BF16, with the sum of squares) and the Omega images of every
// mode in one persistent launch: in each CTA warps 0-3 stream the cast (HBM-bound, the ALUs
// mostly idle) while warps 4-7 generate images (Philox and Box-Muller: integer- and
// FP32-ALU-bound), so the two share the SMs instead of running one after the other.  The
// staged values and the images are those of k_stage_f32_bf16_v4 and k_omega_images; the sum
// of squares is accumulated per thread by compensated FP32 summation and per CTA in FP64.
constexpr int SO_MAXREC = 8;
struct StageOmegaParams {
    const float4* x;
    int64_t n4;
    uint2* dst;
    double* part;          // one partial sum of squares per CTA
    int nrec;
    int64_t first[SO_MAXREC + 1];   // element offsets of the records' images
    omega_images_rec rec[SO_MAXREC];
};

__global__ void __launch_bounds__(256) k_stage_omega(const __grid_constant__ StageOmegaParams p) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double red[4];
    if (w < 4) {
        // warp-contiguous 32-float4 chunks, four chunks' loads in flight per thread
        const int64_t nw = (int64_t)gridDim.x * 4;
        float hi = 0.f, lo = 0.f;
        for (int64_t ch = (int64_t)blockIdx.x * 4 + w; ch * 32 < p.n4; ch += 4 * nw) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = (ch + u * nw) * 32 + lane;
                v[u] = i < p.n4 ? __ldcs(p.x + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = (ch + u * nw) * 32 + lane;
                if (i >= p.n4) continue;
                const dfl sq = df_two_sum(hi, v[u].x * v[u].x + v[u].y * v[u].y + v[u].z * v[u].z + v[u].w * v[u].w);
                hi = sq.hi;
                lo = __fadd_rn(lo, sq.lo);
                __nv_bfloat162 a = __floats2bfloat162_rn(v[u].x, v[u].y);
                __nv_bfloat162 b = __floats2bfloat162_rn(v[u].z, v[u].w);
                uint2 o;
                o.x = *reinterpret_cast<uint32_t*>(&a);
                o.y = *reinterpret_cast<uint32_t*>(&b);
                p.dst[i] = o;
            }
        }
        double acc = (double)hi + (double)lo;
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) red[w] = acc;
    } else {
        const int64_t nt = (int64_t)gridDim.x * 128;
        const int64_t total = p.first[p.nrec];
        int r = 0;
        for (int64_t e = ((int64_t)blockIdx.x * 4 + (w - 4)) * 32 + lane; e < total; e += nt) {
            while (e >= p.first[r + 1]) ++r;   // e only grows: the record index only grows
            const omega_images_rec& q = p.rec[r];
            omega_image_elem(q.seed, q.mode, q.A, q.C, q.ifast, q.ctiles, q.S, q.N, q.split, q.fp16, q.img,
                             e - p.first[r]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) p.part[blockIdx.x] = ((red[0] + red[1]) + red[2]) + red[3];
}


// out[i*ld + s] = sum_b (part[b][i][s] + split * part[b][i][N/2 + s]) in a fixed order:
// 32 outputs per CTA; warp w sums partials b = w, w+8, ... by compensated summation in FP32
// (Knuth's TwoSum: the running sum hi and the sum lo of its exact rounding errors; Ogita,
// Rump & Oishi 2005, Sum2), then the warps' hi + lo are added in order in FP64.  The
// result is as accurate as an FP64 sum of the terms up to about n^2 u32^2 sum |x| (u32 =
// 2^-24) and keeps GB300's FP64 pipe (2 operations per clock per SM) out of the loop.
// When the producing kernel reported an expired wait (*err != 0) its partials are
// incomplete, and every output is NaN instead, so the result cannot pass for a valid one.
constexpr int RED_WARPS = 8;
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
}
__device__ __forceinline__ void reduce_tc_dev(const float* __restrict__ part, int nb, int64_t I,
                                              int N, int Sh, int split, double* __restrict__ out,
                                              int64_t ld, double* __restrict__ out2, int64_t ld2,
                                              const int* __restrict__ err, int bx) {
    __shared__ double acc_sh[RED_WARPS][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)bx * 32 + lane;
    const int64_t tot = I * Sh;
    float hi = 0.f, lo = 0.f;
    if (e < tot) {
        const int64_t i = e / Sh;
        const int s = (int)(e % Sh);
        // four partials' loads in flight, then summed in partial order
        const size_t step = (size_t)RED_WARPS * I * N;
        const float* pb = part + ((size_t)w * I + i) * N + s;
        int b = w;
        for (; b + 3 * RED_WARPS < nb; b += 4 * RED_WARPS, pb += 4 * step) {
            float x[4], y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                x[u] = pb[u * step];
                y[u] = split ? pb[u * step + N / 2] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                two_sum_acc(hi, lo, x[u]);
                if (split) two_sum_acc(hi, lo, y[u]);
            }
        }
        for (; b < nb; b += RED_WARPS, pb += step) {
            two_sum_acc(hi, lo, pb[0]);
            if (split) two_sum_acc(hi, lo, pb[N / 2]);
        }
    }
    acc_sh[w][lane] = (double)hi + (double)lo;
    __syncthreads();
    if (w == 0 && e < tot) {
        double t = 0.0;
        for (int k = 0; k < RED_WARPS; ++k) t += acc_sh[k][lane];
        if (err && *err) t = __longlong_as_double(0x7ff8000000000000LL);
        const int64_t i = e / Sh;
        const int s = (int)(e % Sh);
        out[i * ld + s] = t;
        if (out2) out2[i * ld2 + s] = t;
    }
}

__global__ void __launch_bounds__(32 * RED_WARPS) k_reduce_tc(const float* __restrict__ part, int nb, int64_t I,
                                                             int N, int Sh, int split, double* __restrict__ out,
                                                             int64_t ld, double* __restrict__ out2, int64_t ld2,
                                                             const int* __restrict__ err) {
    reduce_tc_dev(part, nb, I, N, Sh, split, out, ld, out2, ld2, err, (int)blockIdx.x);
}

struct reduce_tc_rec {
    const float* part;
    int nb;
    int64_t I;
    int N;
    int Sh;
    int split;
    double* out;
    int64_t ld;
    double* out2;
    int64_t ld2;
    const int* err;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(32 * RED_WARPS) k_reduce_tc_b(const __grid_constant__ BPack<reduce_tc_rec> p) {
    const reduce_tc_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    reduce_tc_dev(r.part, r.nb, r.I, r.N, r.Sh, r.split, r.out, r.ld, r.out2, r.ld2, r.err, bx);
}


typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

template <int MODE, bool IFAST>
size_t smem_limit() {
    static const size_t mx = max_dyn_smem(k_stream_tc<MODE, IFAST>);   // thread-safe, once
    return mx;
}

}  // namespace

bool supported(const View& v, int mode, int N) {
    if (v.dtype != RBKI_BF16 && v.dtype != RBKI_F16) return false;
    if (N < 16 || N > 64 || N % 16) return false;
    const bool ifast = v.C == 1;
    if (ifast ? (v.I % 8) : (v.C % 8)) return false;
    if (v.A > 0x7fffffffLL || v.I > 0x7fffffffLL || v.C > 0x7fffffffLL) return false;
    const int NS = (int)cdiv(v.I, 128);
    const uint32_t tm = (uint32_t)((mode == TTM ? 0 : NS * N) + (mode == SKETCH ? 0 : 2 * N));
    if (tm > 512) return false;
    const size_t qimg = mode == SKETCH ? 0 : (size_t)NS * 128 * N * 2;
    const size_t yimg = mode == TTM ? 0 : (size_t)2 * 128 * N * 2;
    const size_t avail = 227 * 1024 - 2048 - qimg - yimg;
    const int nslot = (int)std::min<size_t>(8, avail / SLAB_BYTES);
    if (mode == KRYLOV ? nslot < NS : nslot < 2) return false;
    return true;
}

int64_t num_tiles(const View& v) { return v.C > 1 ? v.A * cdiv(v.C, 128) : cdiv(v.A, 128); }

size_t image_bytes_skinny(const View& v, int N) { return (size_t)cdiv(v.I, 128) * 128 * N * 2; }
size_t image_bytes_omega(const View& v, int N) { return (size_t)num_tiles(v) * 128 * N * 2; }
// One persistent CTA per SM.
int grid_size(const View& v) {
    static const int sms = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return std::max(1, n);
    }();
    return (int)std::min<int64_t>(num_tiles(v), sms);
}

rbki_status skinny_image(const double* M, int64_t ldm, int64_t rows, int S, int N, int split, bool fp16,
                         void* img, cudaStream_t st) {
    int64_t rows_pad = cdiv(rows, 128) * 128;
    int64_t tot = rows_pad * N;
    k_skinny_image<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(M, ldm, rows, S, rows_pad, N, split,
                                                             fp16 ? 1 : 0, (uint16_t*)img);
    RBKI_LAUNCH_CHECK("k_skinny_image");
    return RBKI_OK;
}

rbki_status omega_images(uint64_t seed, int mode, const View& v, int S, int N, bool split, void* img,
                         cudaStream_t st) {
    const bool ifast = v.C == 1;
    int64_t ctiles = ifast ? 1 : cdiv(v.C, 128);
    int64_t tiles = num_tiles(v);
    int64_t tot = tiles * 128 * (N / 8);
    k_omega_images<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(seed, mode, v.A, v.C, ifast ? 1 : 0, ctiles, tiles, S,
                                                             N, split ? 1 : 0, v.dtype == RBKI_F16 ? 1 : 0,
                                                             (uint16_t*)img);
    RBKI_LAUNCH_CHECK("k_omega_images");
    return RBKI_OK;
}

rbki_status stream_tc(int mode, const View& v, int N, int Sh, bool split, const void* qimg, const void* omg,
                      float* part, float* yout, int* err, cudaStream_t st, void* yimg_out, uint32_t wait_us,
                      int stall) {
    EncodeTiledFn enc = encode_fn();
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
        cuuint32_t box[2] = {64, 128};
        cuuint32_t es[2] = {1, 1};
        r = enc(&map, dt, 2, const_cast<void*>(v.data), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return set_error(RBKI_E_CUDA, "cuTensorMapEncodeTiled failed");

    Params p{};
    p.A = v.A; p.I = v.I; p.C = v.C;
    p.NS = (int)cdiv(v.I, 128);
    p.N = N; p.Sh = Sh; p.split = split ? 1 : 0;
    p.tiles = num_tiles(v);
    p.ctiles = ifast ? 1 : cdiv(v.C, 128);
    p.qimg = qimg; p.omg = omg;
    p.qimg_bytes = mode == SKETCH ? 0 : (uint32_t)image_bytes_skinny(v, N);
    p.yimg_bytes = (uint32_t)(128 * N * 2);
    p.part = part; p.yout = yout; p.err = err;
    p.yimg_out = mode == TTM ? yimg_out : nullptr;
    p.fp16 = v.dtype == RBKI_F16 ? 1 : 0;
    p.wait_us = wait_us ? wait_us : WAIT_US_DEFAULT;
    p.stall = stall;
    uint32_t tm = (uint32_t)((mode == TTM ? 0 : p.NS * N) + (mode == SKETCH ? 0 : 2 * N));
    uint32_t cols = 32;
    while (cols < tm) cols <<= 1;
    p.tmem_cols = cols;
    const size_t yimg_total = mode == TTM ? 0 : 2 * (size_t)p.yimg_bytes;
    const size_t bar_bytes = 256;
    size_t limit = 0;
#define LIM(M_, F_) limit = smem_limit<M_, F_>()
    if (mode == KRYLOV) { if (ifast) LIM(KRYLOV, true); else LIM(KRYLOV, false); }
    else if (mode == SKETCH) { if (ifast) LIM(SKETCH, true); else LIM(SKETCH, false); }
    else { if (ifast) LIM(TTM, true); else LIM(TTM, false); }
#undef LIM
    if (!limit) return set_error(RBKI_E_CUDA, "stream_tc: shared-memory attribute");
    const size_t fixed = 1024 + p.qimg_bytes + yimg_total + bar_bytes;
    if (limit < fixed + 2 * SLAB_BYTES) return set_error(RBKI_E_UNSUPPORTED, "stream_tc: shared memory");
    p.nslot = (int)std::min<size_t>(8, (limit - fixed) / SLAB_BYTES);
    if (mode == KRYLOV && p.nslot < p.NS) return set_error(RBKI_E_UNSUPPORTED, "stream_tc: tile does not fit");
    p.smem_x = 0;
    p.smem_q = (uint32_t)(p.nslot * SLAB_BYTES);
    p.smem_y = p.smem_q + p.qimg_bytes;
    p.smem_bar = (uint32_t)(p.smem_y + yimg_total);
    const size_t smem = 1024 + p.smem_bar + bar_bytes;
    const int grid = grid_size(v);
#define LAUNCH(M_, F_) k_stream_tc<M_, F_><<<grid, NTHREADS, smem, st>>>(map, p)
    if (mode == KRYLOV) { if (ifast) LAUNCH(KRYLOV, true); else LAUNCH(KRYLOV, false); }
    else if (mode == SKETCH) { if (ifast) LAUNCH(SKETCH, true); else LAUNCH(SKETCH, false); }
    else { if (ifast) LAUNCH(TTM, true); else LAUNCH(TTM, false); }
#undef LAUNCH
    RBKI_LAUNCH_CHECK("k_stream_tc");
    return RBKI_OK;
}

rbki_status reduce_parts(const float* part, int nb, int64_t I, int N, int Sh, bool split, double* out, int64_t ld,
                         double* out2, int64_t ld2, const int* err, cudaStream_t st) {
    int64_t tot = I * Sh;
    k_reduce_tc<<<(unsigned)cdiv(tot, 32), 32 * RED_WARPS, 0, st>>>(part, nb, I, N, Sh, split ? 1 : 0, out, ld, out2,
                                                                  ld2, err);
    RBKI_LAUNCH_CHECK("k_reduce_tc");
    return RBKI_OK;
}

// ---- batched forms (one launch for the items of a lockstep stage; see bat_launch) ----
rbki_status skinny_image_batched(const SkinnyItem* it, int n, cudaStream_t st) {
    std::vector<skinny_image_rec> r;
    for (int k = 0; k < n; ++k) {
        const SkinnyItem& a = it[k];
        const int64_t rows_pad = cdiv(a.rows, 128) * 128;
        r.push_back(skinny_image_rec{a.M, a.ldm, a.rows, a.S, rows_pad, a.N, a.split, a.fp16 ? 1 : 0,
                                     (uint16_t*)a.img, (int)cdiv(rows_pad * a.N, 256), 1, 1});
    }
    return bat_launch(k_skinny_image_b, r.data(), (int)r.size(), 256, 0, st, "k_skinny_image_b");
}

rbki_status omega_images_batched(const OmegaItem* it, int n, cudaStream_t st) {
    std::vector<omega_images_rec> r;
    for (int k = 0; k < n; ++k) {
        const OmegaItem& a = it[k];
        const bool ifast = a.v.C == 1;
        const int64_t ctiles = ifast ? 1 : cdiv(a.v.C, 128), tiles = num_tiles(a.v);
        r.push_back(omega_images_rec{a.seed, a.mode, a.v.A, a.v.C, ifast ? 1 : 0, ctiles, tiles, a.S, a.N,
                                     a.split ? 1 : 0, a.v.dtype == RBKI_F16 ? 1 : 0, (uint16_t*)a.img,
                                     (int)cdiv(tiles * 128 * (a.N / 8), 256), 1, 1});
    }
    return bat_launch(k_omega_images_b, r.data(), (int)r.size(), 256, 0, st, "k_omega_images_b");
}

int stage_omega_grid() {
    static const int g = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return std::max(1, sms) * 4;
    }();
    return g;
}

rbki_status stage_omega_batched(const float* x, int64_t n, void* dst, double* part, const OmegaItem* it, int n_items,
                                cudaStream_t st) {
    if (n % 4 || ((uintptr_t)x % 16) || ((uintptr_t)dst % 8)) return set_error(RBKI_E_INVAL, "stage_omega: layout");
    if (n_items < 0 || n_items > SO_MAXREC) return set_error(RBKI_E_INVAL, "stage_omega: records");
    StageOmegaParams p{};
    p.x = reinterpret_cast<const float4*>(x);
    p.n4 = n / 4;
    p.dst = reinterpret_cast<uint2*>(dst);
    p.part = part;
    p.nrec = n_items;
    p.first[0] = 0;
    for (int k = 0; k < n_items; ++k) {
        const OmegaItem& a = it[k];
        const bool ifast = a.v.C == 1;
        const int64_t ctiles = ifast ? 1 : cdiv(a.v.C, 128), tiles = num_tiles(a.v);
        p.rec[k] = omega_images_rec{a.seed, a.mode, a.v.A, a.v.C, ifast ? 1 : 0, ctiles, tiles, a.S, a.N,
                                    a.split ? 1 : 0, a.v.dtype == RBKI_F16 ? 1 : 0, (uint16_t*)a.img, 0, 1, 1};
        p.first[k + 1] = p.first[k] + tiles * 128 * (a.N / 8);
    }
    k_stage_omega<<<stage_omega_grid(), 256, 0, st>>>(p);
    RBKI_LAUNCH_CHECK("k_stage_omega");
    return RBKI_OK;
}

rbki_status reduce_parts_batched(const ReduceItem* it, int n, cudaStream_t st) {
    std::vector<reduce_tc_rec> r;
    for (int k = 0; k < n; ++k) {
        const ReduceItem& a = it[k];
        r.push_back(reduce_tc_rec{a.part, a.nb, a.I, a.N, a.Sh, a.split ? 1 : 0, a.out, a.ld, a.out2, a.ld2, a.err,
                                  (int)cdiv(a.I * a.Sh, 32), 1, 1});
    }
    return bat_launch(k_reduce_tc_b, r.data(), (int)r.size(), 32 * RED_WARPS, 0, st, "k_reduce_tc_b");
}

}  // namespace tc
}  // namespace rbki
