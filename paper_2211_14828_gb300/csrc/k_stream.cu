// CUDA-core streaming products over the strided mode-n view X = [A][I][C]:
//   * TTM     Y = X x_n M^T             (Algorithm 2 step 6; Krylov half-step X_(n)^T Q)
//   * contract P = X_(n) Y_(n)^T        (Algorithm 1 steps 2-3: sketch W = X Omega and the
//                                        Krylov product X (X^T Q); Gram X X^T when Y == X)
// These are the FP64 comparator path (FP64 accumulate) and the FP32-accumulate CUDA-core
// path for small-I Gram passes.  The unfolding is never materialised: element (i, col) of
// X_(n) is X[(col / C) * I * C + i * C + col % C].
#include "kernels.h"

namespace rbki {
namespace {

constexpr int TT_COLS = 64;   // columns of X_(n) per TTM tile
constexpr int TT_K = 16;      // rows of X_(n) per k-chunk
constexpr int MAXS = 64;      // s per tile

template <typename T, typename Acc, typename To>
__global__ void __launch_bounds__(256) k_ttm(const T* __restrict__ X, int64_t A, int64_t I,
                                             int64_t C, const double* __restrict__ M, int64_t ldm,
                                             int S, To* __restrict__ Y) {
    __shared__ Acc xs[TT_K][TT_COLS + 1];
    __shared__ Acc ms[TT_K][MAXS + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int s0 = blockIdx.y * MAXS;
    // tile -> columns
    int64_t a0, c0;
    const bool cfast = C > 1;
    if (cfast) {
        int64_t ctiles = cdiv(C, TT_COLS);
        a0 = blockIdx.x / ctiles;
        c0 = (blockIdx.x % ctiles) * TT_COLS;
    } else {
        a0 = (int64_t)blockIdx.x * TT_COLS;
        c0 = 0;
    }
    Acc acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;

    for (int64_t i0 = 0; i0 < I; i0 += TT_K) {
        // load X chunk [TT_K][TT_COLS]
        for (int e = tid; e < TT_K * TT_COLS; e += 256) {
            int ii, jj;
            if (cfast) { ii = e / TT_COLS; jj = e % TT_COLS; }
            else { jj = e / TT_K; ii = e % TT_K; }
            int64_t i = i0 + ii;
            Acc v = 0;
            if (i < I) {
                if (cfast) {
                    int64_t c = c0 + jj;
                    if (c < C) v = ld_acc<Acc>(X + (a0 * I + i) * C + c);
                } else {
                    int64_t a = a0 + jj;
                    if (a < A) v = ld_acc<Acc>(X + a * I + i);
                }
            }
            xs[ii][jj] = v;
        }
        for (int e = tid; e < TT_K * MAXS; e += 256) {
            int ii = e / MAXS, ss = e % MAXS;
            int64_t i = i0 + ii;
            int s = s0 + ss;
            ms[ii][ss] = (i < I && s < S) ? (Acc)M[i * ldm + s] : (Acc)0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TT_K; ++kk) {
            Acc xv[4], mv[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) xv[v] = xs[kk][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u) mv[u] = ms[kk][ty + 16 * u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += mv[u] * xv[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int s = s0 + ty + 16 * u;
        if (s >= S) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int jj = tx * 4 + v;
            if (cfast) {
                int64_t c = c0 + jj;
                if (c < C) Y[(a0 * S + s) * C + c] = (To)acc[u][v];
            } else {
                int64_t a = a0 + jj;
                if (a < A) Y[a * S + s] = (To)acc[u][v];
            }
        }
    }
}

constexpr int CT_ROWS = 64;   // rows of X_(n) (i) per contraction tile
constexpr int CT_K = 16;      // columns per chunk

// P_part[split][i][s] = sum over the split's columns of X[i][col] * Y[s][col]
template <typename T, typename TY, typename Acc>
__global__ void __launch_bounds__(256) k_contract(const T* __restrict__ X, int64_t A, int64_t I,
                                                  int64_t C, const TY* __restrict__ Y, int S,
                                                  int64_t cols_per_split, double* __restrict__ part) {
    __shared__ Acc xs[CT_K][CT_ROWS + 1];
    __shared__ Acc ys[CT_K][MAXS + 1];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t i0 = (int64_t)blockIdx.x * CT_ROWS;
    const int s0 = blockIdx.y * MAXS;
    const int64_t d = A * C;
    const int64_t col_lo = (int64_t)blockIdx.z * cols_per_split;
    const int64_t col_hi = min(d, col_lo + cols_per_split);
    Acc acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0;

    for (int64_t k0 = col_lo; k0 < col_hi; k0 += CT_K) {
        for (int e = tid; e < CT_K * CT_ROWS; e += 256) {
            int kk, ii;
            if (C > 1) { ii = e / CT_K; kk = e % CT_K; }     // consecutive columns: coalesced in c
            else { kk = e / CT_ROWS; ii = e % CT_ROWS; }      // C == 1: coalesced in i
            int64_t col = k0 + kk, i = i0 + ii;
            Acc v = 0;
            if (col < col_hi && i < I) {
                int64_t a = col / C, c = col - a * C;
                v = ld_acc<Acc>(X + (a * I + i) * C + c);
            }
            xs[kk][ii] = v;
        }
        for (int e = tid; e < CT_K * MAXS; e += 256) {
            int kk, ss;
            if (C > 1) { ss = e / CT_K; kk = e % CT_K; }
            else { kk = e / MAXS; ss = e % MAXS; }
            int64_t col = k0 + kk;
            int s = s0 + ss;
            Acc v = 0;
            if (col < col_hi && s < S) {
                int64_t a = col / C, c = col - a * C;
                v = ld_acc<Acc>(Y + (a * S + s) * C + c);
            }
            ys[kk][ss] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CT_K; ++kk) {
            Acc xv[4], yv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = xs[kk][ty + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) yv[v] = ys[kk][tx + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += xv[u] * yv[v];
        }
        __syncthreads();
    }
    double* out = part + (int64_t)blockIdx.z * I * S;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int64_t i = i0 + ty + 16 * u;
        if (i >= I) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int s = s0 + tx + 16 * v;
            if (s < S) out[i * S + s] = (double)acc[u][v];
        }
    }
}

// out[i*ld + s] = sum_{k < nsplit} part[k][i][s]   (fixed order: deterministic)
__global__ void k_reduce_parts(const double* __restrict__ part, int nsplit, int64_t I, int S,
                               double* __restrict__ out, int64_t ld, double* __restrict__ out2,
                               int64_t ld2) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= I * S) return;
    const int64_t stride = I * S;
    double acc = 0.0;
    int k = 0;
    for (; k + 3 < nsplit; k += 4) {
        const double v0 = part[k * stride + e], v1 = part[(k + 1) * stride + e];
        const double v2 = part[(k + 2) * stride + e], v3 = part[(k + 3) * stride + e];
        acc += (v0 + v1) + (v2 + v3);
    }
    for (; k < nsplit; ++k) acc += part[k * stride + e];
    int64_t i = e / S, s = e % S;
    out[i * ld + s] = acc;
    if (out2) out2[i * ld2 + s] = acc;
}

template <typename T>
const T* as(const void* p) { return static_cast<const T*>(p); }

// Gram matrix of a short mode (I <= IM): part[block][i][j] = sum over the block's columns of
// X_(n)[i][col] X_(n)[j][col].  One thread per column at a time (coalesced in c when C > 1),
// the I(I+1)/2 products in registers, then a fixed-order CTA reduction: an HBM-bound single
// pass for the Gram path of modes such as a video's colour mode.
template <typename T, typename Acc, int IM>
__global__ void __launch_bounds__(256) k_gram_small(const T* __restrict__ X, int64_t A, int I, int64_t C,
                                                    int64_t cols_per_block, double* __restrict__ part) {
    constexpr int NP = IM * (IM + 1) / 2;
    __shared__ Acc red[8][NP];
    Acc acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0;
    const int64_t d = A * C;
    const int64_t lo = (int64_t)blockIdx.x * cols_per_block;
    const int64_t hi = lo + cols_per_block < d ? lo + cols_per_block : d;
    int64_t col = lo + threadIdx.x;
    int64_t a = col / C, c = col - a * C;
    const int64_t step_a = (int64_t)blockDim.x / C, step_c = (int64_t)blockDim.x - step_a * C;
    for (; col < hi; col += blockDim.x) {
        Acc x[IM];
#pragma unroll
        for (int i = 0; i < IM; ++i) x[i] = i < I ? ld_acc<Acc>(X + (a * I + i) * C + c) : (Acc)0;
        int k = 0;
#pragma unroll
        for (int i = 0; i < IM; ++i)
#pragma unroll
            for (int j = i; j < IM; ++j) acc[k++] += x[i] * x[j];
        c += step_c;
        a += step_a;
        if (c >= C) { c -= C; ++a; }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const Acc v = warp_sum(acc[k]);
        if (lane == 0) red[w][k] = v;
    }
    __syncthreads();
    double* out = part + (int64_t)blockIdx.x * I * I;
    for (int e = threadIdx.x; e < NP; e += blockDim.x) {
        double v = 0.0;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) v += (double)red[ww][e];
        int i = 0, rem = e;                        // e -> (i, j), j >= i, row-major upper triangle
        while (rem >= IM - i) { rem -= IM - i; ++i; }
        const int j = i + rem;
        if (i < I && j < I) {
            out[i * I + j] = v;
            out[j * I + i] = v;
        }
    }
}

}  // namespace

rbki_status gram_small_cuda(const View& x, bool acc32, double* part, int nblocks, double* out, int64_t ld,
                            cudaStream_t st) {
    if (x.I > (acc32 ? 16 : 8)) return set_error(RBKI_E_UNSUPPORTED, "gram_small: I too large");
    const int64_t d = x.A * x.C;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(nblocks, cdiv(d, 256)));
    const int64_t cpb = cdiv(d, nb);
#define GS_L(T, ACC, IM) k_gram_small<T, ACC, IM><<<nb, 256, 0, st>>>(as<T>(x.data), x.A, (int)x.I, x.C, cpb, part)
// FP32 accumulation up to I = 16 (136 accumulators fit in registers), FP64 up to I = 8
#define GS_I(T, ACC) if (x.I <= 4) { GS_L(T, ACC, 4); } else { GS_L(T, ACC, 8); }
#define GS_D(T) if (acc32) { if (x.I > 8) { GS_L(T, float, 16); } else { GS_I(T, float) } } else { GS_I(T, double) }
    switch (x.dtype) {
        case RBKI_F64: GS_D(double); break;
        case RBKI_F32: GS_D(float); break;
        case RBKI_BF16: GS_D(__nv_bfloat16); break;
        case RBKI_F16: GS_D(__half); break;
        default: return set_error(RBKI_E_INVAL, "gram_small: dtype");
    }
#undef GS_D
#undef GS_I
#undef GS_L
    RBKI_LAUNCH_CHECK("k_gram_small");
    const int64_t n = x.I * x.I;
    k_reduce_parts<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(part, nb, x.I, (int)x.I, out, ld, nullptr, 0);
    RBKI_LAUNCH_CHECK("k_reduce_parts");
    return RBKI_OK;
}

rbki_status ttm_cuda(const View& x, const double* M, int64_t ldm, int S, void* Y, int y_dtype,
                     bool acc32, cudaStream_t st) {
    int64_t ntiles = x.C > 1 ? x.A * cdiv(x.C, TT_COLS) : cdiv(x.A, TT_COLS);
    if (ntiles > 0x7fffffff) return set_error(RBKI_E_UNSUPPORTED, "ttm: too many tiles");
    dim3 grid((unsigned)ntiles, (unsigned)cdiv(S, MAXS));
#define TTM_L(T, ACC, TO)                                                                   \
    k_ttm<T, ACC, TO><<<grid, 256, 0, st>>>(as<T>(x.data), x.A, x.I, x.C, M, ldm, S,        \
                                            static_cast<TO*>(Y))
#define TTM_D(T)                                                                            \
    if (y_dtype == RBKI_F64) { if (acc32) TTM_L(T, float, double); else TTM_L(T, double, double); } \
    else if (y_dtype == RBKI_F32) { if (acc32) TTM_L(T, float, float); else TTM_L(T, double, float); } \
    else return set_error(RBKI_E_INVAL, "ttm: output dtype");
    switch (x.dtype) {
        case RBKI_F64: TTM_D(double); break;
        case RBKI_F32: TTM_D(float); break;
        case RBKI_BF16: TTM_D(__nv_bfloat16); break;
        case RBKI_F16: TTM_D(__half); break;
        default: return set_error(RBKI_E_INVAL, "ttm: dtype");
    }
#undef TTM_D
#undef TTM_L
    RBKI_LAUNCH_CHECK("k_ttm");
    return RBKI_OK;
}

// Small mode products (the core chain after the first contraction): Y = X x_n M^T with
// S <= NSB <= 32 outputs per column.  M is staged in shared memory in chunks of TS_MI rows,
// converted to the accumulation type once.
//   C > 1: a CTA takes 32 columns c of one a; its 8 warps split the rows i (warp g takes
//          i = g mod 8), each lane keeps NSB accumulators for its column, and the 8 partial
//          sums are added in warp order through shared memory.  X reads coalesced over c.
//   C = 1: one warp per a, lanes over i, butterfly reduction of the NSB partial sums.
constexpr int TS_MI = 128;
constexpr int TS_G = 8;      // row groups (warps) per CTA of the C > 1 form
template <typename T, typename Acc, int NSB>
__global__ void __launch_bounds__(256) k_ttm_small_c(const T* __restrict__ X, int64_t A, int64_t I, int64_t C,
                                                     const double* __restrict__ M, int64_t ldm, int S,
                                                     double* __restrict__ Y) {
    static_assert(TS_G * (NSB / 2) * 32 <= TS_MI * NSB, "reduction buffer");
    __shared__ __align__(16) Acc buf[TS_MI * NSB];   // M chunk, then the reduction
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int64_t cblocks = cdiv(C, (int64_t)32);
    const int64_t a = blockIdx.x / cblocks;
    const int64_t c = (blockIdx.x % cblocks) * 32 + lane;
    Acc acc[NSB];
#pragma unroll
    for (int q = 0; q < NSB; ++q) acc[q] = 0;
    for (int64_t i0 = 0; i0 < I; i0 += TS_MI) {
        const int ni = (int)((I - i0) < TS_MI ? (I - i0) : TS_MI);
        __syncthreads();
        for (int e = threadIdx.x; e < TS_MI * NSB; e += blockDim.x) {
            const int ii = e / NSB, q = e % NSB;
            buf[e] = (ii < ni && q < S) ? (Acc)M[(i0 + ii) * ldm + q] : (Acc)0;
        }
        __syncthreads();
        if (c < C) {
            const T* xp = X + (a * I + i0) * C + c;
            // four rows' loads in flight per warp, then their products in row order
            for (int ib = g; ib < ni; ib += 4 * TS_G) {
                Acc xs[4];
#pragma unroll
                for (int u4 = 0; u4 < 4; ++u4) {
                    const int ii = ib + u4 * TS_G;
                    xs[u4] = ii < ni ? ld_acc<Acc>(xp + (int64_t)ii * C) : (Acc)0;
                }
#pragma unroll
                for (int u4 = 0; u4 < 4; ++u4) {
                    const int ii = ib + u4 * TS_G;
                    if (ii >= ni) break;
                    const Acc x = xs[u4];
                    // the row of M is the same for every lane: 16-byte broadcast reads
                    const uint4* mr = reinterpret_cast<const uint4*>(&buf[ii * NSB]);
#pragma unroll
                    for (int v = 0; v < NSB * (int)sizeof(Acc) / 16; ++v) {
                        const uint4 u = mr[v];
                        if constexpr (sizeof(Acc) == 4) {
                            acc[4 * v + 0] += x * __uint_as_float(u.x);
                            acc[4 * v + 1] += x * __uint_as_float(u.y);
                            acc[4 * v + 2] += x * __uint_as_float(u.z);
                            acc[4 * v + 3] += x * __uint_as_float(u.w);
                        } else {
                            acc[2 * v + 0] += x * __hiloint2double((int)u.y, (int)u.x);
                            acc[2 * v + 1] += x * __hiloint2double((int)u.w, (int)u.z);
                        }
                    }
                }
            }
        }
    }
    // the groups' sums, added in group order, half of the outputs at a time
    Acc* red = buf;   // [TS_G][NSB / 2][32]
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < NSB / 2; ++q) red[(g * (NSB / 2) + q) * 32 + lane] = acc[h * (NSB / 2) + q];
        __syncthreads();
        for (int e = threadIdx.x; e < (NSB / 2) * 32; e += blockDim.x) {
            const int q = e / 32, l = e % 32;
            const int qq = h * (NSB / 2) + q;
            const int64_t cc = (blockIdx.x % cblocks) * 32 + l;
            Acc t = 0;
            for (int gg = 0; gg < TS_G; ++gg) t += red[(gg * (NSB / 2) + q) * 32 + l];
            if (cc < C && qq < S) Y[(a * S + qq) * C + cc] = (double)t;
        }
    }
}

template <typename T, typename Acc, int NSB>
__global__ void __launch_bounds__(256) k_ttm_small_i(const T* __restrict__ X, int64_t A, int64_t I,
                                                     const double* __restrict__ M, int64_t ldm, int S,
                                                     double* __restrict__ Y) {
    __shared__ Acc ms[TS_MI][NSB + 1];   // odd stride: the lanes of a warp read different rows
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    Acc acc[NSB];
#pragma unroll
    for (int q = 0; q < NSB; ++q) acc[q] = 0;
    for (int64_t i0 = 0; i0 < I; i0 += TS_MI) {
        const int ni = (int)((I - i0) < TS_MI ? (I - i0) : TS_MI);
        __syncthreads();
        for (int e = threadIdx.x; e < TS_MI * NSB; e += blockDim.x) {
            const int ii = e / NSB, q = e % NSB;
            ms[ii][q] = (ii < ni && q < S) ? (Acc)M[(i0 + ii) * ldm + q] : (Acc)0;
        }
        __syncthreads();
        if (a < A)
            for (int ii = lane; ii < ni; ii += 32) {
                const Acc x = ld_acc<Acc>(X + a * I + i0 + ii);
#pragma unroll
                for (int q = 0; q < NSB; ++q) acc[q] += x * ms[ii][q];
            }
    }
    if (a >= A) return;   // whole warp
#pragma unroll
    for (int q = 0; q < NSB; ++q) {
        const Acc v = warp_sum(acc[q]);
        if (lane == 0 && q < S) Y[a * S + q] = (double)v;
    }
}

rbki_status ttm_small_cuda(const View& x, const double* M, int64_t ldm, int S, double* Y, bool acc32,
                           cudaStream_t st) {
    if (S < 1 || S > 32) return set_error(RBKI_E_UNSUPPORTED, "ttm_small: S > 32");
    if (x.dtype != RBKI_F64 && x.dtype != RBKI_F32) return set_error(RBKI_E_UNSUPPORTED, "ttm_small: dtype");
    const bool ifast = x.C == 1;
    const int64_t blocks = ifast ? cdiv(x.A, (int64_t)8) : x.A * cdiv(x.C, (int64_t)32);
    if (blocks > 0x7fffffff) return set_error(RBKI_E_UNSUPPORTED, "ttm_small: too many blocks");
#define TS_L(T, ACC, NSB)                                                                              \
    if (ifast) k_ttm_small_i<T, ACC, NSB><<<(unsigned)blocks, 256, 0, st>>>(as<T>(x.data), x.A, x.I, M, ldm, S, Y); \
    else k_ttm_small_c<T, ACC, NSB><<<(unsigned)blocks, 32 * TS_G, 0, st>>>(as<T>(x.data), x.A, x.I, x.C, M, ldm, S, Y)
#define TS_B(T, ACC)                                                                                   \
    if (S <= 8) { TS_L(T, ACC, 8); } else if (S <= 16) { TS_L(T, ACC, 16); } else if (S <= 24) { TS_L(T, ACC, 24); } \
    else { TS_L(T, ACC, 32); }
    if (x.dtype == RBKI_F64) {
        if (acc32) { TS_B(double, float) } else { TS_B(double, double) }
    } else {
        if (acc32) { TS_B(float, float) } else { TS_B(float, double) }
    }
#undef TS_B
#undef TS_L
    RBKI_LAUNCH_CHECK("k_ttm_small");
    return RBKI_OK;
}

int contract_nsplit(const View& x) {
    int64_t d = x.A * x.C;
    int64_t itiles = cdiv(x.I, CT_ROWS);
    int64_t want = cdiv(4 * 152, itiles);
    int64_t maxs = cdiv(d, 256);
    int64_t n = want < maxs ? want : maxs;
    return (int)(n < 1 ? 1 : n);
}

rbki_status contract_cuda(const View& x, const void* Y, int y_dtype, int S, bool acc32,
                          double* part, int nsplit, double* out, int64_t ld_out, double* out2,
                          int64_t ld_out2, cudaStream_t st) {
    int64_t d = x.A * x.C;
    int64_t cps = rup(cdiv(d, nsplit), CT_K);
    dim3 grid((unsigned)cdiv(x.I, CT_ROWS), (unsigned)cdiv(S, MAXS), (unsigned)nsplit);
#define CT_L(T, TY, ACC)                                                                   \
    k_contract<T, TY, ACC><<<grid, 256, 0, st>>>(as<T>(x.data), x.A, x.I, x.C, as<TY>(Y), S, \
                                                 cps, part)
#define CT_D(T)                                                                            \
    if (y_dtype == RBKI_F64) { if (acc32) CT_L(T, double, float); else CT_L(T, double, double); } \
    else if (y_dtype == x.dtype) { if (acc32) CT_L(T, T, float); else CT_L(T, T, double); }  \
    else return set_error(RBKI_E_INVAL, "contract: Y dtype");
    switch (x.dtype) {
        case RBKI_F64: CT_D(double); break;
        case RBKI_F32: CT_D(float); break;
        case RBKI_BF16: CT_D(__nv_bfloat16); break;
        case RBKI_F16: CT_D(__half); break;
        default: return set_error(RBKI_E_INVAL, "contract: dtype");
    }
#undef CT_D
#undef CT_L
    RBKI_LAUNCH_CHECK("k_contract");
    int64_t n = x.I * S;
    k_reduce_parts<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(part, nsplit, x.I, S, out, ld_out,
                                                            out2, ld_out2);
    RBKI_LAUNCH_CHECK("k_reduce_parts");
    return RBKI_OK;
}

}  // namespace rbki
