// Small dense FP64 kernels of Algorithms 1-2:
//   * A^T B with a fixed-order split reduction (block Gram-Schmidt coefficients, Gram
//     matrices, Z = Q^T P of Remark 1)
//   * one pass of block orthonormalisation: Pythagorean-inner-product block classical
//     Gram-Schmidt (BCGS-PIP, Barlow & Smoktunowicz 2013) + Cholesky QR with pivot
//     deflation (reading c3); two passes give BCGS2 / CholQR2
//   * factor formation U = Q U~(:, 1:R) with the sign convention (Algorithm 2 step 5).
#include "kernels.h"
#include "dfloat.cuh"

namespace rbki {
namespace {

constexpr int AT_T = 32;    // output tile
constexpr int AT_K = 16;    // rows per sub-chunk

// part[chunk][k][l] = sum_{r in chunk} A[r][k] B[r][l]
__device__ __forceinline__ void atb_part_dev(const double* __restrict__ A, int64_t lda, int ma,
                                             const double* __restrict__ B, int64_t ldb, int mb,
                                             int64_t rows, int64_t rows_per_chunk,
                                             double* __restrict__ part, int bx, int by, int bz) {
    __shared__ double as[AT_K][AT_T + 1];
    __shared__ double bs[AT_K][AT_T + 1];
    const int tid = threadIdx.x;
    const int tk = tid / 16, tl = tid % 16;          // 2 x 2 outputs per thread
    const int k0 = bx * AT_T, l0 = by * AT_T;
    const int64_t r_lo = (int64_t)bz * rows_per_chunk;
    const int64_t r_hi = min(rows, r_lo + rows_per_chunk);
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int64_t r0 = r_lo; r0 < r_hi; r0 += AT_K) {
        for (int e = tid; e < AT_K * AT_T; e += 256) {
            int rr = e / AT_T, cc = e % AT_T;
            int64_t r = r0 + rr;
            bool ok = r < r_hi;
            as[rr][cc] = (ok && k0 + cc < ma) ? A[r * lda + k0 + cc] : 0.0;
            bs[rr][cc] = (ok && l0 + cc < mb) ? B[r * ldb + l0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < AT_K; ++rr) {
            double a0 = as[rr][tk], a1 = as[rr][tk + 16];
            double b0 = bs[rr][tl], b1 = bs[rr][tl + 16];
            acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
            acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
        }
        __syncthreads();
    }
    double* out = part + (int64_t)bz * ma * mb;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            int k = k0 + tk + 16 * u, l = l0 + tl + 16 * v;
            if (k < ma && l < mb) out[(int64_t)k * mb + l] = acc[u][v];
        }
}

__global__ void __launch_bounds__(256) k_atb_part(const double* __restrict__ A, int64_t lda, int ma,
                                                  const double* __restrict__ B, int64_t ldb, int mb,
                                                  int64_t rows, int64_t rows_per_chunk,
                                                  double* __restrict__ part) {
    atb_part_dev(A, lda, ma, B, ldb, mb, rows, rows_per_chunk, part, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
}

struct atb_part_rec {
    const double* A;
    int64_t lda;
    int ma;
    const double* B;
    int64_t ldb;
    int mb;
    int64_t rows;
    int64_t rows_per_chunk;
    double* part;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_atb_part_b(const __grid_constant__ BPack<atb_part_rec> p) {
    const atb_part_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    atb_part_dev(r.A, r.lda, r.ma, r.B, r.ldb, r.mb, r.rows, r.rows_per_chunk, r.part, bx, by, bz);
}

// The same partials with the operands rounded to FP32 and FP32 accumulation within a chunk of
// rows (the chunks are then summed in FP64 by k_atb_reduce): for the mixed path's Z = Q^T P,
// whose P already carries the BF16 rounding of the tensor-core products (relative 2^-9), so
// the FP32 chunk sums (error <= rows_per_chunk * 2^-24 * sum |q p|) add nothing visible, and
// the products leave GB300's FP64 pipe (2 per clock per SM) for the FP32 pipes.
__device__ __forceinline__ void atb_part32_dev(const double* __restrict__ A, int64_t lda, int ma,
                                               const double* __restrict__ B, int64_t ldb, int mb,
                                               int64_t rows, int64_t rows_per_chunk,
                                               double* __restrict__ part, int bx, int by, int bz) {
    __shared__ float as[AT_K][AT_T + 1];
    __shared__ float bs[AT_K][AT_T + 1];
    const int tid = threadIdx.x;
    const int tk = tid / 16, tl = tid % 16;          // 2 x 2 outputs per thread
    const int k0 = bx * AT_T, l0 = by * AT_T;
    const int64_t r_lo = (int64_t)bz * rows_per_chunk;
    const int64_t r_hi = min(rows, r_lo + rows_per_chunk);
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int64_t r0 = r_lo; r0 < r_hi; r0 += AT_K) {
        for (int e = tid; e < AT_K * AT_T; e += 256) {
            int rr = e / AT_T, cc = e % AT_T;
            int64_t r = r0 + rr;
            bool ok = r < r_hi;
            as[rr][cc] = (ok && k0 + cc < ma) ? __double2float_rn(A[r * lda + k0 + cc]) : 0.f;
            bs[rr][cc] = (ok && l0 + cc < mb) ? __double2float_rn(B[r * ldb + l0 + cc]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < AT_K; ++rr) {
            const float a0 = as[rr][tk], a1 = as[rr][tk + 16];
            const float b0 = bs[rr][tl], b1 = bs[rr][tl + 16];
            acc[0][0] = fmaf(a0, b0, acc[0][0]); acc[0][1] = fmaf(a0, b1, acc[0][1]);
            acc[1][0] = fmaf(a1, b0, acc[1][0]); acc[1][1] = fmaf(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    double* out = part + (int64_t)bz * ma * mb;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            int k = k0 + tk + 16 * u, l = l0 + tl + 16 * v;
            if (k < ma && l < mb) out[(int64_t)k * mb + l] = (double)acc[u][v];
        }
}

__global__ void __launch_bounds__(256) k_atb_part32(const double* __restrict__ A, int64_t lda, int ma,
                                                    const double* __restrict__ B, int64_t ldb, int mb,
                                                    int64_t rows, int64_t rows_per_chunk,
                                                    double* __restrict__ part) {
    atb_part32_dev(A, lda, ma, B, ldb, mb, rows, rows_per_chunk, part, (int)blockIdx.x, (int)blockIdx.y,
                   (int)blockIdx.z);
}

__global__ void __launch_bounds__(256) k_atb_part32_b(const __grid_constant__ BPack<atb_part_rec> p) {
    const atb_part_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    atb_part32_dev(r.A, r.lda, r.ma, r.B, r.ldb, r.mb, r.rows, r.rows_per_chunk, r.part, bx, by, bz);
}


// sum over the chunks of element e of the partials: four independent loads in flight per
// step; fixed summation order
__device__ __forceinline__ double atb_sum_elem(const double* __restrict__ part, int nchunk, int64_t stride, int e) {
    double acc = 0.0;
    int c = 0;
    for (; c + 3 < nchunk; c += 4) {
        const double v0 = __ldcg(part + c * stride + e), v1 = __ldcg(part + (c + 1) * stride + e);
        const double v2 = __ldcg(part + (c + 2) * stride + e), v3 = __ldcg(part + (c + 3) * stride + e);
        acc += (v0 + v1) + (v2 + v3);
    }
    for (; c < nchunk; ++c) acc += __ldcg(part + c * stride + e);
    return acc;
}

// out = sum of the partials; sym (ma == mb): out[k][l] = (sum_kl + sum_lk) / 2, the reduction
// followed by the symmetrisation (Z + Z^T) / 2 of k_symmetrize, bit for bit
__device__ __forceinline__ void atb_reduce_dev(const double* __restrict__ part, int nchunk, int ma, int mb,
                                               double* __restrict__ out, int64_t ldo, int bx, int sym = 0) {
    int e = bx * blockDim.x + threadIdx.x;
    if (e >= ma * mb) return;
    const int64_t stride = (int64_t)ma * mb;
    const int k = e / mb, l = e % mb;
    double acc = atb_sum_elem(part, nchunk, stride, e);
    if (sym && k != l) acc = 0.5 * (acc + atb_sum_elem(part, nchunk, stride, l * mb + k));
    out[(int64_t)k * ldo + l] = acc;
}

__global__ void k_atb_reduce(const double* __restrict__ part, int nchunk, int ma, int mb,
                             double* __restrict__ out, int64_t ldo) {
    atb_reduce_dev(part, nchunk, ma, mb, out, ldo, (int)blockIdx.x);
}

struct atb_reduce_rec {
    const double* part;
    int nchunk;
    int ma;
    int mb;
    double* out;
    int64_t ldo;
    int sym;
    int gx, gy, gz;
};

__global__ void k_atb_reduce_b(const __grid_constant__ BPack<atb_reduce_rec> p) {
    const atb_reduce_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    atb_reduce_dev(r.part, r.nchunk, r.ma, r.mb, r.out, r.ldo, bx, r.sym);
}


// G'[k][l] = M[m+k][l] - sum_{r<m} M[r][k] M[r][l]  (Pythagorean Gram of the projected block)
// nu2[k] = M[m+k][k] (squared column norms before projection).
// Summation order (fixed, shared by every form): the rows r < m in tiles of GP_TILE; within a
// tile four interleaved accumulators, combined as (a0 + a1) + (a2 + a3); the tiles' sums
// added in tile order.  The batched pass computes each tile's sum on its own CTA.
constexpr int GP_TILE = 32;
// the tile's sum from its nr rows, row q at Mt + q * S (global memory or a shared copy)
template <bool SHARED>
__device__ __forceinline__ double gprime_tile_rows(const double* __restrict__ Mt, int nr, int S, int k, int l) {
    auto ld = [&](int q, int c) { return SHARED ? Mt[q * S + c] : __ldcg(Mt + (int64_t)q * S + c); };
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 3 < nr; q += 4) {
        a0 += ld(q, k) * ld(q, l);
        a1 += ld(q + 1, k) * ld(q + 1, l);
        a2 += ld(q + 2, k) * ld(q + 2, l);
        a3 += ld(q + 3, k) * ld(q + 3, l);
    }
    for (; q < nr; ++q) a0 += ld(q, k) * ld(q, l);
    return (a0 + a1) + (a2 + a3);
}
__device__ __forceinline__ double gprime_tile(const double* __restrict__ M, int m, int S, int k, int l, int t) {
    const int r0 = t * GP_TILE, r1 = min(m, r0 + GP_TILE);
    return gprime_tile_rows<false>(M + (int64_t)r0 * S, r1 - r0, S, k, l);
}

__device__ __forceinline__ void gprime_finish(const double* __restrict__ M, int m, int S, double acc,
                                              double* __restrict__ Gp, double* __restrict__ nu2, int k, int l) {
    const double g = __ldcg(M + (int64_t)(m + k) * S + l);
    Gp[k * S + l] = g - acc;
    if (k == l) nu2[k] = g;
}

__device__ __forceinline__ void gprime_elem(const double* __restrict__ M, int m, int S, double* __restrict__ Gp,
                                            double* __restrict__ nu2, int k, int l) {
    double acc = 0.0;
    for (int t = 0; t * GP_TILE < m; ++t) acc += gprime_tile(M, m, S, k, l, t);
    gprime_finish(M, m, S, acc, Gp, nu2, k, l);
}

// one CTA per column l; only the upper triangle k <= l (what the Cholesky reads)
__device__ __forceinline__ void gprime_dev(const double* __restrict__ M, int m, int S, double* __restrict__ Gp,
                                           double* __restrict__ nu2, int bx) {
    if ((int)threadIdx.x <= bx && (int)threadIdx.x < S) gprime_elem(M, m, S, Gp, nu2, (int)threadIdx.x, bx);
}

__global__ void k_gprime(const double* __restrict__ M, int m, int S, double* __restrict__ Gp,
                         double* __restrict__ nu2) {
    gprime_dev(M, m, S, Gp, nu2, (int)blockIdx.x);
}

// Cholesky G' = R^T R with pivot deflation, and Rinv (upper, zero rows/columns for
// deflated directions).  Column k is deflated when nu2[k] == 0 or its pivot (squared norm
// orthogonal to everything accepted) <= tau^2 nu2[k].  Single CTA.
//
// G' = L D L^T by elimination without square roots, carrying M = L^{-1} along (the same row
// operations applied to an identity), so that R = D^{1/2} L^T and Rinv = M^T D^{-1/2} come
// out of one loop with one barrier per step.  The elimination is a serial chain of S steps,
// so it runs in double-float (dfloat.cuh, about 2^-48 relative) on the FP32 pipes: on GB300
// a dependent FP64 instruction waits tens of cycles and the SM retires two a clock, which
// made the FP64 form take about 1.7 us per step at S = 30.  G' and the thresholds are scaled
// by an exact power of 4 (the largest nu2 into [1, 4)) so that every entry sits well inside
// FP32's range; a column whose nu2 is below about 2^-100 of the largest is treated as zero.
//   * thread 0 updates d_{k+1} first and computes 1 / d_{k+1} while the other threads update
//     the rest (lookahead);
//   * the trailing upper triangle and the rows of M are walked as one packed index list;
//   * 1 / sqrt(d_k) for all k in parallel afterwards; Rinv is written in FP64.
__device__ __forceinline__ void chol_deflate_dev(const double* __restrict__ Gp, const double* __restrict__ nu2,
                                                 int S, double tau, double* __restrict__ Rinv,
                                                 int32_t* __restrict__ kept) {
    // one S x S array holds both factors: the upper triangle (with the diagonal) is W, row k
    // = d_k L_{:,k}^T after step k; the strict lower triangle is L^{-1} (unit diagonal
    // implied).  Keeping the shared memory small (S = 30: 7.5 KB) lets this kernel share an
    // SM with the tensor-core streaming kernel running on another stream.
    extern __shared__ double sm[];
    dfl* W = reinterpret_cast<dfl*>(sm);
    dfl* inv_d = W + S * S;           // S: 1 / d_k, 0 when deflated
    dfl* aux = inv_d + S;             // S: deflation thresholds, then 1 / sqrt(d_k)
    __shared__ int p_sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid & 15, ty = tid >> 4, ny = nt >> 4;
    // p = floor(e / 2) for the largest nu2 in [2^e, 2^(e+1)): nu2 * 4^-p lies in [1, 4)
    if (tid < 32) {
        unsigned long long mx = 0;
        for (int k = tid; k < S; k += 32) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(nu2[k]);
            mx = b > mx ? b : mx;   // nu2 >= 0: the bit patterns order like the values
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
            mx = v > mx ? v : mx;
        }
        if (tid == 0) {
            const int e = (int)((mx >> 52) & 0x7ff) - 1023;
            const int pe = mx == 0 ? 0 : (e >= 0 ? e / 2 : -((1 - e) / 2));
            p_sh = pe < -500 ? -500 : (pe > 500 ? 500 : pe);   // keeps 4^-p and 2^-p normal
        }
    }
    __syncthreads();
    const int p = p_sh;
    const double sc = __longlong_as_double((long long)(1023 - 2 * p) << 52);     // 4^-p
    const double unsc = __longlong_as_double((long long)(1023 - p) << 52);       // 2^-p
    for (int e = tid; e < S * S; e += nt) W[e] = (e % S >= e / S) ? df_from_double(Gp[e] * sc) : dfl{0.f, 0.f};
    for (int k = tid; k < S; k += nt)
        aux[k] = nu2[k] > 0.0 ? df_from_double(tau * tau * nu2[k] * sc) : dfl{__int_as_float(0x7f800000), 0.f};
    __syncthreads();
    auto pivot = [&](int k) {
        const dfl d = W[k * S + k];
        inv_d[k] = df_gt(d, aux[k]) ? df_rcp(d) : dfl{0.f, 0.f};
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    const bool small = S <= 32 && ny == 16;   // 256 threads: rows ty and ty + 16 cover every i > k
    for (int k = 0; k < S; ++k) {
        const dfl ik = inv_d[k];
        const int mm = S - k - 1;
        if (ik.hi != 0.f) {                    // uniform: a deflated column eliminates nothing
            if (tid == 0 && mm > 0) {          // d_{k+1} and its reciprocal first (lookahead)
                const dfl wk = W[k * S + k + 1];
                W[(k + 1) * S + k + 1] = df_fms(W[(k + 1) * S + k + 1], df_mul(wk, ik), wk);
                pivot(k + 1);
            }
            // rows i > k on a 16-wide grid of threads (no index division): the trailing
            // upper triangle j >= i (d_{k+1} done above) and the row of L^{-1}, columns 0..k
            if (small) {
                // at most 2 rows x (2 trailing + 2 L^{-1} columns) per thread: every operand
                // is loaded before any update, so the eight double-float chains overlap
                dfl wv[8], mv[8], lv[2];
                int at[8];
                bool on[8];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int i = k + 1 + ty + 16 * a;
                    const bool rok = i < S;
                    lv[a] = rok ? df_mul(W[k * S + i], ik) : dfl{0.f, 0.f};
#pragma unroll
                    for (int b = 0; b < 2; ++b) {
                        const int j = k + 1 + tx + 16 * b, c = tx + 16 * b;
                        const int q = 4 * a + b, q2 = 4 * a + 2 + b;
                        on[q] = rok && j < S && j >= i && (i != k + 1 || j != k + 1);
                        on[q2] = rok && c <= k;
                        at[q] = i * S + j;
                        at[q2] = i * S + c;
                        wv[q] = on[q] ? W[at[q]] : dfl{0.f, 0.f};
                        mv[q] = on[q] ? W[k * S + j] : dfl{0.f, 0.f};
                        wv[q2] = on[q2] ? W[at[q2]] : dfl{0.f, 0.f};
                        mv[q2] = on[q2] ? (c == k ? dfl{1.f, 0.f} : W[k * S + c]) : dfl{0.f, 0.f};
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) wv[q] = df_fms(wv[q], lv[q / 4], mv[q]);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (on[q]) W[at[q]] = wv[q];
            } else {
                for (int i = k + 1 + ty; i < S; i += ny) {
                    const dfl li = df_mul(W[k * S + i], ik);
                    for (int j = k + 1 + tx; j < S; j += 16)
                        if (j >= i && (i != k + 1 || j != k + 1)) W[i * S + j] = df_fms(W[i * S + j], li, W[k * S + j]);
                    for (int c = tx; c <= k; c += 16) {
                        const dfl mkc = c == k ? dfl{1.f, 0.f} : W[k * S + c];   // L^{-1}[k][c]
                        W[i * S + c] = df_fms(W[i * S + c], li, mkc);
                    }
                }
            }
        } else if (tid == 0 && mm > 0) {
            pivot(k + 1);
        }
        __syncthreads();
    }
    for (int k = tid; k < S; k += nt) aux[k] = inv_d[k].hi != 0.f ? df_rsqrt(W[k * S + k]) : dfl{0.f, 0.f};
    __syncthreads();
    // Rinv[t][c] = L^{-1}[c][t] / sqrt(d_c) for t <= c, scaled back by 2^-p
    for (int e = tid; e < S * S; e += nt) {
        const int t = e / S, c = e % S;
        Rinv[e] = t < c ? df_to_double(df_mul(W[c * S + t], aux[c])) * unsc
                        : (t == c ? df_to_double(aux[c]) * unsc : 0.0);
    }
    if (tid == 0 && kept) {
        int nk = 0;
        for (int k = 0; k < S; ++k) nk += inv_d[k].hi != 0.f ? 1 : 0;
        atomicAdd(kept, nk);
    }
}

__global__ void k_chol_deflate(const double* __restrict__ Gp, const double* __restrict__ nu2,
                               int S, double tau, double* __restrict__ Rinv,
                               int32_t* __restrict__ kept) {
    chol_deflate_dev(Gp, nu2, S, tau, Rinv, kept);
}

// The head of one orthonormalisation pass in one launch, finished by ticket counters (no CTA
// waits for another):
//   1. every CTA computes its tile of the chunk partials of M = [Q_{<m} Q_m]^T Q_m (k_atb_part);
//   2. the CTA that finishes last among those of a 32-row tile of M sums that tile's partials
//      (k_atb_reduce) and, for the rows r < m it holds, the tile's sums of the Pythagorean
//      correction sum_r M[r][k] M[r][l] (gprime_tile);
//   3. the tile that finishes last adds the tiles' sums in tile order, forms G' and nu2
//      (k_gprime) and factors G' with deflation (k_chol_deflate).
// Same arithmetic in the same order as those kernels.  ticket[0] counts finished tiles and
// ticket[1 + t] the finished CTAs of tile t; the last CTA puts them back to 0.  The tickets
// must be 0 before the first pass.
struct orth_head_rec {
    const double* Q;
    int64_t ldq;
    int m;
    int S;
    int64_t rows;
    int64_t rows_per_chunk;
    int nchunk;
    double* part;
    double* M;
    double* gpart;     // [tile][S][S] sums of the Pythagorean correction per 32-row tile
    double* Gp;
    double* Rinv;
    double* nu2;
    double tau;
    int32_t* kept;
    int32_t* ticket;   // 1 + gx counters
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_orth_head_b(const __grid_constant__ BPack<orth_head_rec> p) {
    const orth_head_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    const int ma = r.m + r.S, S = r.S;
    atb_part_dev(r.Q, r.ldq, ma, r.Q + r.m, r.ldq, S, r.rows, r.rows_per_chunk, r.part, bx, by, bz);
    __shared__ int last;
    __threadfence();                   // this CTA's partials before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(r.ticket + 1 + bx, 1) == r.gy * r.gz - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();                   // the partials of this row tile are visible from here
    const int mp = ma * S;
    const int r0 = bx * AT_T, nr = min(AT_T, ma - r0);
    extern __shared__ double oh_sm[];  // this tile's rows of M (then the Cholesky's arrays)
    for (int e = threadIdx.x; e < nr * S; e += blockDim.x) {
        const double v = atb_sum_elem(r.part, r.nchunk, (int64_t)mp, r0 * S + e);
        r.M[(int64_t)r0 * S + e] = v;
        oh_sm[e] = v;
    }
    __syncthreads();                   // this tile's rows of M, for the tile sums below
    if (r0 < r.m) {
        const int nb = min(r.m, r0 + GP_TILE) - r0;
        for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
            const int k = e / S, l = e % S;
            if (k <= l) r.gpart[(int64_t)bx * S * S + e] = gprime_tile_rows<true>(oh_sm, nb, S, k, l);
        }
    }
    __syncthreads();                   // the shared rows are reused by the Cholesky
    __threadfence();                   // this tile's M rows and sums before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(r.ticket, 1) == r.gx - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();                   // every tile's M rows and sums are visible from here
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
        if (e / S > e % S) continue;   // the Cholesky reads the upper triangle only
        double acc = 0.0;
        for (int t = 0; t * GP_TILE < r.m; ++t) acc += __ldcg(r.gpart + (int64_t)t * S * S + e);
        gprime_finish(r.M, r.m, S, acc, r.Gp, r.nu2, e / S, e % S);
    }
    __syncthreads();
    chol_deflate_dev(r.Gp, r.nu2, S, r.tau, r.Rinv, r.kept);
    if (threadIdx.x == 0)
        for (int t = 0; t <= r.gx; ++t) r.ticket[t] = 0;
}

// Q[i][m+s] = sum_t (Q[i][m+t] - sum_{r<m} Q[i][r] M[r][t]) Rinv[t][s]; ORTH_ROWS rows per CTA
constexpr int ORTH_ROWS = 4;
__device__ __forceinline__ void orth_apply_dev(double* __restrict__ Q, int64_t ldq, int64_t rows, int m,
                                               int S, const double* __restrict__ M,
                                               const double* __restrict__ Rinv, int bx) {
    extern __shared__ double tmp[];   // ORTH_ROWS x S
    const int64_t i0 = (int64_t)bx * ORTH_ROWS;
    for (int e = threadIdx.x; e < ORTH_ROWS * S; e += blockDim.x) {
        int rr = e / S, s = e % S;
        int64_t i = i0 + rr;
        double v = 0.0;
        if (i < rows) {
            const double* qi = Q + i * ldq;
            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
            int r = 0;
            for (; r + 3 < m; r += 4) {
                a0 += qi[r] * M[(int64_t)r * S + s];
                a1 += qi[r + 1] * M[(int64_t)(r + 1) * S + s];
                a2 += qi[r + 2] * M[(int64_t)(r + 2) * S + s];
                a3 += qi[r + 3] * M[(int64_t)(r + 3) * S + s];
            }
            for (; r < m; ++r) a0 += qi[r] * M[(int64_t)r * S + s];
            v = qi[m + s] - ((a0 + a1) + (a2 + a3));
        }
        tmp[e] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ORTH_ROWS * S; e += blockDim.x) {
        int rr = e / S, s = e % S;
        int64_t i = i0 + rr;
        if (i >= rows) continue;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int tt = 0;
        for (; tt + 3 <= s; tt += 4) {
            a0 += tmp[rr * S + tt] * Rinv[tt * S + s];
            a1 += tmp[rr * S + tt + 1] * Rinv[(tt + 1) * S + s];
            a2 += tmp[rr * S + tt + 2] * Rinv[(tt + 2) * S + s];
            a3 += tmp[rr * S + tt + 3] * Rinv[(tt + 3) * S + s];
        }
        for (; tt <= s; ++tt) a0 += tmp[rr * S + tt] * Rinv[tt * S + s];
        Q[i * ldq + m + s] = (a0 + a1) + (a2 + a3);
    }
}

__global__ void __launch_bounds__(128) k_orth_apply(double* __restrict__ Q, int64_t ldq, int64_t rows, int m,
                                                    int S, const double* __restrict__ M,
                                                    const double* __restrict__ Rinv) {
    orth_apply_dev(Q, ldq, rows, m, S, M, Rinv, (int)blockIdx.x);
}

struct orth_apply_rec {
    double* Q;
    int64_t ldq;
    int64_t rows;
    int m;
    int S;
    const double* M;
    const double* Rinv;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(128) k_orth_apply_b(const __grid_constant__ BPack<orth_apply_rec> p) {
    const orth_apply_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    orth_apply_dev(r.Q, r.ldq, r.rows, r.m, r.S, r.M, r.Rinv, bx);
}


// U[i][k] = sum_t Q[i][t] V[t][k]  (or V[i][k] when Q == nullptr)
__device__ __forceinline__ void form_u_dev(const double* __restrict__ Q, int64_t ldq, int64_t rows,
                                           const double* __restrict__ V, int n, int ldv, int R, double* __restrict__ U, int bx) {
    int64_t e = (int64_t)bx * blockDim.x + threadIdx.x;
    if (e >= rows * R) return;
    int64_t i = e / R;
    int k = (int)(e % R);
    double acc;
    if (Q) {
        acc = 0.0;
        const double* qi = Q + i * ldq;
        for (int t = 0; t < n; ++t) acc += qi[t] * V[(int64_t)t * ldv + k];
    } else {
        acc = V[i * ldv + k];
    }
    U[e] = acc;
}

__global__ void k_form_u(const double* __restrict__ Q, int64_t ldq, int64_t rows,
                         const double* __restrict__ V, int n, int ldv, int R, double* __restrict__ U) {
    form_u_dev(Q, ldq, rows, V, n, ldv, R, U, (int)blockIdx.x);
}

struct form_u_rec {
    const double* Q;
    int64_t ldq;
    int64_t rows;
    const double* V;
    int n;
    int ldv;
    int R;
    double* U;
    int gx, gy, gz;
};

__global__ void k_form_u_b(const __grid_constant__ BPack<form_u_rec> p) {
    const form_u_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    form_u_dev(r.Q, r.ldq, r.rows, r.V, r.n, r.ldv, r.R, r.U, bx);
}


// largest-|.| entry of column k made positive (lowest row index on ties); one CTA per column
__device__ __forceinline__ void sign_fix_dev(double* __restrict__ U, int64_t rows, int R, int bx) {
    const int k = bx;
    double best = -1.0;
    int64_t bi = 0x7fffffffffffffffLL;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
        double x = fabs(U[i * R + k]);
        if (x > best) { best = x; bi = i; }
    }
    __shared__ double sb[1024];
    __shared__ int64_t si[1024];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) {
            double b2 = sb[threadIdx.x + o];
            int64_t i2 = si[threadIdx.x + o];
            if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
                sb[threadIdx.x] = b2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    int64_t piv = si[0];
    if (piv >= rows) return;
    bool flip = U[piv * R + k] < 0.0;
    __syncthreads();
    if (flip)
        for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) U[i * R + k] = -U[i * R + k];
}

__global__ void k_sign_fix(double* __restrict__ U, int64_t rows, int R) {
    sign_fix_dev(U, rows, R, (int)blockIdx.x);
}

struct sign_fix_rec {
    double* U;
    int64_t rows;
    int R;
    int gx, gy, gz;
};

__global__ void k_sign_fix_b(const __grid_constant__ BPack<sign_fix_rec> p) {
    const sign_fix_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    sign_fix_dev(r.U, r.rows, r.R, bx);
}


__device__ __forceinline__ void copy_dev(const double* __restrict__ s, double* __restrict__ d, int64_t n, int bx) {
    int64_t e = (int64_t)bx * blockDim.x + threadIdx.x;
    if (e < n) d[e] = s[e];
}

__global__ void k_copy(const double* __restrict__ s, double* __restrict__ d, int64_t n) {
    copy_dev(s, d, n, (int)blockIdx.x);
}

struct copy_rec {
    const double* s;
    double* d;
    int64_t n;
    int gx, gy, gz;
};

__global__ void k_copy_b(const __grid_constant__ BPack<copy_rec> p) {
    const copy_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    copy_dev(r.s, r.d, r.n, bx);
}

__global__ void k_fill_i32(int32_t* d, int32_t v, int n) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) d[e] = v;
}

struct fill_i32_rec {
    int32_t* d;
    int32_t v;
    int n;
    int gx, gy, gz;
};

__global__ void k_fill_i32_b(const __grid_constant__ BPack<fill_i32_rec> p) {
    const fill_i32_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    for (int e = threadIdx.x; e < r.n; e += blockDim.x) r.d[e] = r.v;
}

}  // namespace

int atb_nchunks(int64_t rows) {
    int64_t n = cdiv(rows, 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(n, 64));
}

rbki_status atb_cuda(const double* A, int64_t lda, int ma, const double* B, int64_t ldb, int mb,
                     int64_t rows, double* part, double* out, int64_t ldo, cudaStream_t st, bool f32) {
    int nch = atb_nchunks(rows);
    int64_t rpc = cdiv(rows, nch);
    dim3 grid((unsigned)cdiv(ma, AT_T), (unsigned)cdiv(mb, AT_T), (unsigned)nch);
    if (f32) k_atb_part32<<<grid, 256, 0, st>>>(A, lda, ma, B, ldb, mb, rows, rpc, part);
    else k_atb_part<<<grid, 256, 0, st>>>(A, lda, ma, B, ldb, mb, rows, rpc, part);
    RBKI_LAUNCH_CHECK("k_atb_part");
    k_atb_reduce<<<(unsigned)cdiv((int64_t)ma * mb, 256), 256, 0, st>>>(part, nch, ma, mb, out, ldo);
    RBKI_LAUNCH_CHECK("k_atb_reduce");
    return RBKI_OK;
}

// scratch: [tickets (8 doubles)] [chunk partials] [M] [G'] [Rinv] [nu2] [per-tile sums of the
// Pythagorean correction]
size_t orth_scratch_doubles(int64_t rows, int m, int S) {
    size_t mp = (size_t)(m + S) * S;
    return ORTH_TICKET_DOUBLES + (size_t)atb_nchunks(rows) * mp + mp + 2 * (size_t)S * S + S +
           (size_t)cdiv(m + S, AT_T) * S * S + 64;
}

int32_t* orth_ticket(double* scratch) { return reinterpret_cast<int32_t*>(scratch); }

rbki_status orth_pass_cuda(double* Q, int64_t ldq, int64_t rows, int m, int S, double tau,
                           double* scratch, int32_t* kept, cudaStream_t st) {
    if (S > 128) return set_error(RBKI_E_UNSUPPORTED, "orth: block width > 128");
    size_t mp = (size_t)(m + S) * S;
    double* part = scratch + ORTH_TICKET_DOUBLES;
    double* M = part + (size_t)atb_nchunks(rows) * mp;
    double* Gp = M + mp;
    double* Rinv = Gp + (size_t)S * S;
    double* nu2 = Rinv + (size_t)S * S;
    RBKI_TRY(atb_cuda(Q, ldq, m + S, Q + m, ldq, S, rows, part, M, S, st));
    k_gprime<<<S, 128, 0, st>>>(M, m, S, Gp, nu2);
    RBKI_LAUNCH_CHECK("k_gprime");
    size_t sm = ((size_t)S * S + 2 * S) * sizeof(double);   // W | L^{-1}, 1/d, 1/sqrt(d)
    static const size_t smax = max_dyn_smem(k_chol_deflate);   // thread-safe, once
    if (sm > smax) return set_error(RBKI_E_UNSUPPORTED, "orth: block too wide for shared memory");
    k_chol_deflate<<<1, 256, sm, st>>>(Gp, nu2, S, tau, Rinv, kept);
    RBKI_LAUNCH_CHECK("k_chol_deflate");
    k_orth_apply<<<(unsigned)cdiv(rows, ORTH_ROWS), 32 * ORTH_ROWS, ORTH_ROWS * S * sizeof(double), st>>>(
        Q, ldq, rows, m, S, M, Rinv);
    RBKI_LAUNCH_CHECK("k_orth_apply");
    return RBKI_OK;
}

rbki_status form_factor_cuda(const double* Q, int64_t ldq, int64_t rows, const double* V, int n,
                             int ldv, int R, double* U, cudaStream_t st) {
    int64_t tot = rows * R;
    k_form_u<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(Q, ldq, rows, V, n, ldv, R, U);
    RBKI_LAUNCH_CHECK("k_form_u");
    k_sign_fix<<<R, 256, 0, st>>>(U, rows, R);
    RBKI_LAUNCH_CHECK("k_sign_fix");
    return RBKI_OK;
}

rbki_status copy_f64_cuda(const double* src, double* dst, int64_t n, cudaStream_t st) {
    if (n <= 0) return RBKI_OK;
    k_copy<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(src, dst, n);
    RBKI_LAUNCH_CHECK("k_copy");
    return RBKI_OK;
}

rbki_status fill_i32_cuda(int32_t* dst, int32_t v, int n, cudaStream_t st) {
    if (n <= 0) return RBKI_OK;
    k_fill_i32<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(dst, v, n);
    RBKI_LAUNCH_CHECK("k_fill_i32");
    return RBKI_OK;
}

// ---- batched forms: one launch per kernel for all items (see bat_launch) ----
rbki_status atb_batched(const AtbItem* it, int n, cudaStream_t st) {
    if (n <= 0) return RBKI_OK;
    std::vector<atb_part_rec> ap, ap32;
    std::vector<atb_reduce_rec> ar(n);
    for (int k = 0; k < n; ++k) {
        const AtbItem& a = it[k];
        const int nch = atb_nchunks(a.rows);
        (a.f32 ? ap32 : ap).push_back(atb_part_rec{a.A, a.lda, a.ma, a.B, a.ldb, a.mb, a.rows, cdiv(a.rows, nch),
                                                   a.part, (int)cdiv(a.ma, AT_T), (int)cdiv(a.mb, AT_T), nch});
        if (a.sym && a.ma != a.mb) return set_error(RBKI_E_INVAL, "atb_batched: symmetric output of a non-square product");
        ar[k] = atb_reduce_rec{a.part, nch, a.ma, a.mb, a.out, a.ldo, a.sym, (int)cdiv((int64_t)a.ma * a.mb, 256), 1, 1};
    }
    RBKI_TRY(bat_launch(k_atb_part_b, ap.data(), (int)ap.size(), 256, 0, st, "k_atb_part_b"));
    RBKI_TRY(bat_launch(k_atb_part32_b, ap32.data(), (int)ap32.size(), 256, 0, st, "k_atb_part32_b"));
    return bat_launch(k_atb_reduce_b, ar.data(), n, 256, 0, st, "k_atb_reduce_b");
}

// Two launches per pass: the fused head (partials, reduction, G', Cholesky with deflation)
// and the update of the block; the same arithmetic as orth_pass_cuda's five kernels.  Each
// item's ticket (orth_ticket(scratch)) must be 0 before the first pass.
rbki_status orth_pass_batched(const OrthItem* it, int n, double tau, cudaStream_t st) {
    if (n <= 0) return RBKI_OK;
    std::vector<orth_head_rec> oh(n);
    std::vector<orth_apply_rec> oa(n);
    int smax = 0;
    for (int k = 0; k < n; ++k) {
        const OrthItem& o = it[k];
        if (o.S > 128) return set_error(RBKI_E_UNSUPPORTED, "orth: block width > 128");
        const int S = o.S, ma = o.m + S;
        const size_t mp = (size_t)ma * S;
        const int nch = atb_nchunks(o.rows);
        double* part = o.scratch + ORTH_TICKET_DOUBLES;
        double* M = part + (size_t)nch * mp;
        double* Gp = M + mp;
        double* Rinv = Gp + (size_t)S * S;
        double* nu2 = Rinv + (size_t)S * S;
        double* gpart = nu2 + S;
        if (cdiv(ma, AT_T) + 1 > (int64_t)(ORTH_TICKET_DOUBLES * 2))
            return set_error(RBKI_E_UNSUPPORTED, "orth: more row tiles than tickets");
        oh[k] = orth_head_rec{o.Q, o.ldq, o.m, S, o.rows, cdiv(o.rows, nch), nch, part, M, gpart, Gp, Rinv, nu2, tau,
                              o.kept, orth_ticket(o.scratch), (int)cdiv(ma, AT_T), (int)cdiv(S, AT_T), nch};
        oa[k] = orth_apply_rec{o.Q, o.ldq, o.rows, o.m, S, M, Rinv, (int)cdiv(o.rows, ORTH_ROWS), 1, 1};
        smax = std::max(smax, S);
    }
    // the Cholesky's arrays, or one 32-row tile of M for the tile sums
    const size_t sm = std::max((size_t)smax * smax + 2 * smax, (size_t)AT_T * smax) * sizeof(double);
    static const size_t hmax = max_dyn_smem(k_orth_head_b);   // thread-safe, once
    if (sm > hmax) return set_error(RBKI_E_UNSUPPORTED, "orth: block too wide for shared memory");
    RBKI_TRY(bat_launch(k_orth_head_b, oh.data(), n, 256, sm, st, "k_orth_head_b"));
    return bat_launch(k_orth_apply_b, oa.data(), n, 32 * ORTH_ROWS, (size_t)ORTH_ROWS * smax * sizeof(double), st,
                      "k_orth_apply_b");
}

rbki_status form_factor_batched(const FormItem* it, int n, cudaStream_t st) {
    if (n <= 0) return RBKI_OK;
    std::vector<form_u_rec> fu(n);
    std::vector<sign_fix_rec> sf(n);
    for (int k = 0; k < n; ++k) {
        const FormItem& f = it[k];
        fu[k] = form_u_rec{f.Q, f.ldq, f.rows, f.V, f.n, f.ldv, f.R, f.U, (int)cdiv(f.rows * f.R, 256), 1, 1};
        sf[k] = sign_fix_rec{f.U, f.rows, f.R, f.R, 1, 1};
    }
    RBKI_TRY(bat_launch(k_form_u_b, fu.data(), n, 256, 0, st, "k_form_u_b"));
    return bat_launch(k_sign_fix_b, sf.data(), n, 256, 0, st, "k_sign_fix_b");
}

rbki_status fill_i32_batched(const FillItem* it, int n, cudaStream_t st) {
    std::vector<fill_i32_rec> fr;
    for (int k = 0; k < n; ++k)
        if (it[k].dst && it[k].n > 0) fr.push_back(fill_i32_rec{it[k].dst, it[k].v, it[k].n, 1, 1, 1});
    return bat_launch(k_fill_i32_b, fr.data(), (int)fr.size(), 32, 0, st, "k_fill_i32_b");
}

rbki_status copy_f64_batched(const CopyItem* it, int n, cudaStream_t st) {
    std::vector<copy_rec> cp;
    for (int k = 0; k < n; ++k)
        if (it[k].n > 0) cp.push_back(copy_rec{it[k].src, it[k].dst, it[k].n, (int)cdiv(it[k].n, 256), 1, 1});
    return bat_launch(k_copy_b, cp.data(), (int)cp.size(), 256, 0, st, "k_copy_b");
}

}  // namespace rbki

// ---- general small FP64 GEMM: C = op(A) B + beta C with a split over K ----
namespace rbki {
namespace {

template <bool TRANSA>
__device__ __forceinline__ void gemm_part_dev(const double* __restrict__ A, int64_t lda,
                                              const double* __restrict__ B, int64_t ldb, int M, int N, int K,
                                              int kpc, double* __restrict__ part, int bx, int by, int bz) {
    __shared__ double as[AT_K][AT_T + 1];
    __shared__ double bs[AT_K][AT_T + 1];
    const int tid = threadIdx.x;
    const int tk = tid / 16, tl = tid % 16;
    const int m0 = bx * AT_T, n0 = by * AT_T;
    const int k_lo = bz * kpc, k_hi = min(K, k_lo + kpc);
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int k0 = k_lo; k0 < k_hi; k0 += AT_K) {
        for (int e = tid; e < AT_K * AT_T; e += 256) {
            const int kk = e / AT_T, cc = e % AT_T;
            const int k = k0 + kk;
            const bool ok = k < k_hi;
            as[kk][cc] = (ok && m0 + cc < M) ? (TRANSA ? A[(int64_t)k * lda + m0 + cc] : A[(int64_t)(m0 + cc) * lda + k]) : 0.0;
            bs[kk][cc] = (ok && n0 + cc < N) ? B[(int64_t)k * ldb + n0 + cc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < AT_K; ++kk) {
            const double a0 = as[kk][tk], a1 = as[kk][tk + 16];
            const double b0 = bs[kk][tl], b1 = bs[kk][tl + 16];
            acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
            acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
        }
        __syncthreads();
    }
    double* out = part + (int64_t)bz * M * N;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int m = m0 + tk + 16 * u, n = n0 + tl + 16 * v;
            if (m < M && n < N) out[(int64_t)m * N + n] = acc[u][v];
        }
}

template <bool TRANSA>
__global__ void __launch_bounds__(256) k_gemm_part(const double* __restrict__ A, int64_t lda,
                                                   const double* __restrict__ B, int64_t ldb, int M, int N, int K,
                                                   int kpc, double* __restrict__ part) {
    gemm_part_dev<TRANSA>(A, lda, B, ldb, M, N, K, kpc, part, (int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z);
}

struct gemm_part_rec {
    const double* A;
    int64_t lda;
    const double* B;
    int64_t ldb;
    int M;
    int N;
    int K;
    int kpc;
    double* part;
    int gx, gy, gz;
};

template <bool TRANSA>
__global__ void __launch_bounds__(256) k_gemm_part_b(const __grid_constant__ BPack<gemm_part_rec> p) {
    const gemm_part_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    gemm_part_dev<TRANSA>(r.A, r.lda, r.B, r.ldb, r.M, r.N, r.K, r.kpc, r.part, bx, by, bz);
}


__device__ __forceinline__ void gemm_reduce_dev(const double* __restrict__ part, int nchunk, int M, int N, double* __restrict__ C,
                                                int64_t ldc, double beta, int bx) {
    const int e = bx * blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    const int64_t stride = (int64_t)M * N;
    double acc = 0.0;
    int c = 0;
    for (; c + 3 < nchunk; c += 4) {
        const double v0 = part[c * stride + e], v1 = part[(c + 1) * stride + e];
        const double v2 = part[(c + 2) * stride + e], v3 = part[(c + 3) * stride + e];
        acc += (v0 + v1) + (v2 + v3);
    }
    for (; c < nchunk; ++c) acc += part[c * stride + e];
    double* cp = C + (int64_t)(e / N) * ldc + e % N;
    *cp = beta != 0.0 ? acc + beta * *cp : acc;
}

__global__ void k_gemm_reduce(const double* __restrict__ part, int nchunk, int M, int N, double* __restrict__ C,
                              int64_t ldc, double beta) {
    gemm_reduce_dev(part, nchunk, M, N, C, ldc, beta, (int)blockIdx.x);
}

struct gemm_reduce_rec {
    const double* part;
    int nchunk;
    int M;
    int N;
    double* C;
    int64_t ldc;
    double beta;
    int gx, gy, gz;
};

__global__ void k_gemm_reduce_b(const __grid_constant__ BPack<gemm_reduce_rec> p) {
    const gemm_reduce_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    gemm_reduce_dev(r.part, r.nchunk, r.M, r.N, r.C, r.ldc, r.beta, bx);
}


int gemm_nchunk(int M, int N, int K) {
    const int tiles = (int)(cdiv(M, AT_T) * cdiv(N, AT_T));
    const int want = (int)cdiv(256, tiles);
    const int maxc = (int)cdiv(K, AT_K);
    return std::max(1, std::min(want, maxc));
}

}  // namespace

size_t gemm_part_doubles(int M, int N, int K) { return (size_t)gemm_nchunk(M, N, K) * M * N; }

rbki_status gemm_f64_cuda(bool transA, int M, int N, int K, const double* A, int64_t lda, const double* B,
                          int64_t ldb, double* C, int64_t ldc, double beta, double* part, cudaStream_t st) {
    const int nch = gemm_nchunk(M, N, K);
    const int kpc = (int)rup(cdiv(K, nch), AT_K);
    dim3 grid((unsigned)cdiv(M, AT_T), (unsigned)cdiv(N, AT_T), (unsigned)nch);
    if (transA) k_gemm_part<true><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, K, kpc, part);
    else k_gemm_part<false><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, K, kpc, part);
    RBKI_LAUNCH_CHECK("k_gemm_part");
    k_gemm_reduce<<<(unsigned)cdiv((int64_t)M * N, 256), 256, 0, st>>>(part, nch, M, N, C, ldc, beta);
    RBKI_LAUNCH_CHECK("k_gemm_reduce");
    return RBKI_OK;
}

rbki_status gemm_f64_batched(const GemmItem* it, int n, cudaStream_t st) {
    if (n <= 0) return RBKI_OK;
    std::vector<gemm_part_rec> pt, pn;
    std::vector<gemm_reduce_rec> rd(n);
    for (int k = 0; k < n; ++k) {
        const GemmItem& g = it[k];
        const int nch = gemm_nchunk(g.M, g.N, g.K);
        const int kpc = (int)rup(cdiv(g.K, nch), AT_K);
        const gemm_part_rec r{g.A, g.lda, g.B, g.ldb, g.M, g.N, g.K, kpc, g.part,
                              (int)cdiv(g.M, AT_T), (int)cdiv(g.N, AT_T), nch};
        (g.transA ? pt : pn).push_back(r);
        rd[k] = gemm_reduce_rec{g.part, nch, g.M, g.N, g.C, g.ldc, g.beta, (int)cdiv((int64_t)g.M * g.N, 256), 1, 1};
    }
    RBKI_TRY(bat_launch(k_gemm_part_b<true>, pt.data(), (int)pt.size(), 256, 0, st, "k_gemm_part_b"));
    RBKI_TRY(bat_launch(k_gemm_part_b<false>, pn.data(), (int)pn.size(), 256, 0, st, "k_gemm_part_b"));
    return bat_launch(k_gemm_reduce_b, rd.data(), n, 256, 0, st, "k_gemm_reduce_b");
}

}  // namespace rbki
