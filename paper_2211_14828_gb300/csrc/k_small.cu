// Small dense FP64 kernels of Algorithms 1-2:
//   * A^T B with a fixed-order split reduction (block Gram-Schmidt coefficients, Gram
//     matrices, Z = Q^T P of Remark 1)
//   * one pass of block orthonormalisation: Pythagorean-inner-product block classical
//     Gram-Schmidt (BCGS-PIP, Barlow & Smoktunowicz 2013) + Cholesky QR with pivot
//     deflation (reading c3); two passes give BCGS2 / CholQR2
//   * factor formation U = Q U~(:, 1:R) with the sign convention (Algorithm 2 step 5).
#include "kernels.h"

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


// sum over the chunks of element e of the partials: four independent loads in flight per
// step; fixed summation order
__device__ __forceinline__ double atb_sum_elem(const double* __restrict__ part, int nchunk, int64_t stride, int e) {
    double acc = 0.0;
    int c = 0;
    for (; c + 3 < nchunk; c += 4) {
        const double v0 = part[c * stride + e], v1 = part[(c + 1) * stride + e];
        const double v2 = part[(c + 2) * stride + e], v3 = part[(c + 3) * stride + e];
        acc += (v0 + v1) + (v2 + v3);
    }
    for (; c < nchunk; ++c) acc += part[c * stride + e];
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
// nu2[k] = M[m+k][k] (squared column norms before projection).  One CTA per column l.
__device__ __forceinline__ void gprime_elem(const double* __restrict__ M, int m, int S, double* __restrict__ Gp,
                                            double* __restrict__ nu2, int k, int l) {
    double g = M[(int64_t)(m + k) * S + l];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int r = 0;
    for (; r + 3 < m; r += 4) {
        a0 += M[(int64_t)r * S + k] * M[(int64_t)r * S + l];
        a1 += M[(int64_t)(r + 1) * S + k] * M[(int64_t)(r + 1) * S + l];
        a2 += M[(int64_t)(r + 2) * S + k] * M[(int64_t)(r + 2) * S + l];
        a3 += M[(int64_t)(r + 3) * S + k] * M[(int64_t)(r + 3) * S + l];
    }
    for (; r < m; ++r) a0 += M[(int64_t)r * S + k] * M[(int64_t)r * S + l];
    Gp[k * S + l] = g - ((a0 + a1) + (a2 + a3));
    if (k == l) nu2[k] = g;
}

__device__ __forceinline__ void gprime_dev(const double* __restrict__ M, int m, int S, double* __restrict__ Gp,
                                           double* __restrict__ nu2, int bx) {
    if ((int)threadIdx.x < S) gprime_elem(M, m, S, Gp, nu2, (int)threadIdx.x, bx);
}

__global__ void k_gprime(const double* __restrict__ M, int m, int S, double* __restrict__ Gp,
                         double* __restrict__ nu2) {
    gprime_dev(M, m, S, Gp, nu2, (int)blockIdx.x);
}

struct gprime_rec {
    const double* M;
    int m;
    int S;
    double* Gp;
    double* nu2;
    int gx, gy, gz;
};

__global__ void k_gprime_b(const __grid_constant__ BPack<gprime_rec> p) {
    const gprime_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    gprime_dev(r.M, r.m, r.S, r.Gp, r.nu2, bx);
}


// Cholesky G' = R^T R with pivot deflation, and Rinv (upper, zero rows/columns for
// deflated directions).  Column k is deflated when nu2[k] == 0 or its pivot (squared norm
// orthogonal to everything accepted) <= tau^2 nu2[k].  Single CTA.
//
// G' = L D L^T by elimination without square roots, carrying M = L^{-1} along (the same row
// operations applied to an identity), so that R = D^{1/2} L^T and Rinv = M^T D^{-1/2} come
// out of one loop with one barrier per step.  FP64 on GB300 has 64 cycles of dependent
// latency and 2 FMA/clk/SM, so the serial chain is kept short and the FP64 instructions
// full:
//   * thread 0 updates d_{k+1} first and computes 1 / d_{k+1} (FP32 estimate + two FP64
//     Newton steps) while the other threads update the rest (lookahead);
//   * the trailing upper triangle and the rows of M are walked as one packed index list;
//   * 1 / sqrt(d_k) for all k in parallel afterwards.
__device__ __forceinline__ double rsqrt_f64(double d) {
    // FP32 estimate + two FP64 Newton steps: full FP64 accuracy with a short dependent chain
    double y = (double)rsqrtf((float)d);
    y = y * (1.5 - 0.5 * d * y * y);
    y = y * (1.5 - 0.5 * d * y * y);
    return y;
}
__device__ __forceinline__ double rcp_f64(double d) {
    double y = (double)__frcp_rn((float)d);
    y = y * (2.0 - d * y);
    y = y * (2.0 - d * y);
    return y;
}

__device__ __forceinline__ void chol_deflate_dev(const double* __restrict__ Gp, const double* __restrict__ nu2,
                                                 int S, double tau, double* __restrict__ Rinv,
                                                 int32_t* __restrict__ kept) {
    // one S x S array holds both factors: the upper triangle (with the diagonal) is W, row k
    // = d_k L_{:,k}^T after step k; the strict lower triangle is L^{-1} (unit diagonal
    // implied).  Keeping the shared memory small (S = 30: 7.5 KB) lets this kernel share an
    // SM with the tensor-core streaming kernel running on another stream.
    extern __shared__ double sm[];
    double* W = sm;
    double* inv_d = W + S * S;        // S: 1 / d_k, 0 when deflated
    double* rinv = inv_d + S;         // S: 1 / sqrt(d_k), 0 when deflated
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < S * S; e += nt) W[e] = (e % S >= e / S) ? Gp[e] : 0.0;
    __syncthreads();
    auto pivot = [&](int k) {
        const double d = W[k * S + k], nu = nu2[k];
        inv_d[k] = (nu > 0.0 && d > tau * tau * nu) ? rcp_f64(d) : 0.0;
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    for (int k = 0; k < S; ++k) {
        const double ik = inv_d[k];
        const int mm = S - k - 1;
        if (ik != 0.0) {                       // uniform: a deflated column eliminates nothing
            if (tid == 0 && mm > 0) {          // d_{k+1} first, then its reciprocal
                const double wk = W[k * S + k + 1];
                W[(k + 1) * S + k + 1] -= wk * wk * ik;
            }
            const int ntri = mm * (mm + 1) / 2;      // trailing upper triangle (a <= b)
            const int nm = mm * (k + 1);             // rows k+1.. of L^{-1}, columns 0..k
            for (int t = tid + 1; t < ntri + nm; t += nt) {
                if (t < ntri) {
                    // t = b (b + 1) / 2 + a, 0 <= a <= b < mm
                    int bb = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
                    if ((bb + 1) * (bb + 2) / 2 <= t) ++bb;
                    if (bb * (bb + 1) / 2 > t) --bb;
                    const int aa = t - bb * (bb + 1) / 2;
                    const int i = k + 1 + aa, j = k + 1 + bb;
                    W[i * S + j] -= W[k * S + i] * W[k * S + j] * ik;
                } else {
                    const int u = t - ntri;
                    const int i = k + 1 + u / (k + 1), c = u % (k + 1);
                    const double mkc = c == k ? 1.0 : W[k * S + c];   // L^{-1}[k][c]
                    W[i * S + c] -= (W[k * S + i] * ik) * mkc;
                }
            }
        }
        if (tid == 0 && mm > 0) pivot(k + 1);
        __syncthreads();
    }
    for (int k = tid; k < S; k += nt) rinv[k] = inv_d[k] != 0.0 ? rsqrt_f64(W[k * S + k]) : 0.0;
    __syncthreads();
    // Rinv[t][c] = L^{-1}[c][t] / sqrt(d_c) for t <= c
    for (int e = tid; e < S * S; e += nt) {
        const int t = e / S, c = e % S;
        Rinv[e] = t < c ? W[c * S + t] * rinv[c] : (t == c ? rinv[c] : 0.0);
    }
    if (tid == 0 && kept) {
        int nk = 0;
        for (int k = 0; k < S; ++k) nk += inv_d[k] != 0.0 ? 1 : 0;
        atomicAdd(kept, nk);
    }
}

__global__ void k_chol_deflate(const double* __restrict__ Gp, const double* __restrict__ nu2,
                               int S, double tau, double* __restrict__ Rinv,
                               int32_t* __restrict__ kept) {
    chol_deflate_dev(Gp, nu2, S, tau, Rinv, kept);
}

struct chol_deflate_rec {
    const double* Gp;
    const double* nu2;
    int S;
    double tau;
    double* Rinv;
    int32_t* kept;
    int gx, gy, gz;
};

__global__ void k_chol_deflate_b(const __grid_constant__ BPack<chol_deflate_rec> p) {
    const chol_deflate_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    chol_deflate_dev(r.Gp, r.nu2, r.S, r.tau, r.Rinv, r.kept);
}


// The head of one orthonormalisation pass in one launch: every CTA computes its tile of the
// chunk partials of M = [Q_{<m} Q_m]^T Q_m (k_atb_part); the CTA that finishes last (a ticket
// counter, no CTA waits for another) sums the partials (k_atb_reduce), forms the Pythagorean
// Gram G' and nu2 (k_gprime) and factors it with deflation (k_chol_deflate), with the same
// arithmetic in the same order as those three kernels, then resets the ticket to 0.  The
// ticket must be 0 before the first pass.
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
    double* Gp;
    double* Rinv;
    double* nu2;
    double tau;
    int32_t* kept;
    int32_t* ticket;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_orth_head_b(const __grid_constant__ BPack<orth_head_rec> p) {
    const orth_head_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    const int ma = r.m + r.S;
    atb_part_dev(r.Q, r.ldq, ma, r.Q + r.m, r.ldq, r.S, r.rows, r.rows_per_chunk, r.part, bx, by, bz);
    __shared__ int last;
    __threadfence();                   // this CTA's partials before its ticket
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(r.ticket, 1) == r.gx * r.gy * r.gz - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();                   // every other CTA's partials are visible from here
    const int mp = ma * r.S;
    for (int e = threadIdx.x; e < mp; e += blockDim.x)
        r.M[e] = atb_sum_elem(r.part, r.nchunk, (int64_t)mp, e);
    __syncthreads();
    for (int e = threadIdx.x; e < r.S * r.S; e += blockDim.x) gprime_elem(r.M, r.m, r.S, r.Gp, r.nu2, e % r.S, e / r.S);
    __syncthreads();
    chol_deflate_dev(r.Gp, r.nu2, r.S, r.tau, r.Rinv, r.kept);
    if (threadIdx.x == 0) *r.ticket = 0;
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
    int gx, gy, gz;
};

__global__ void k_fill_i32_b(const __grid_constant__ BPack<fill_i32_rec> p) {
    const fill_i32_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz) || threadIdx.x) return;
    *r.d = r.v;
}

}  // namespace

int atb_nchunks(int64_t rows) {
    int64_t n = cdiv(rows, 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(n, 64));
}

rbki_status atb_cuda(const double* A, int64_t lda, int ma, const double* B, int64_t ldb, int mb,
                     int64_t rows, double* part, double* out, int64_t ldo, cudaStream_t st) {
    int nch = atb_nchunks(rows);
    int64_t rpc = cdiv(rows, nch);
    dim3 grid((unsigned)cdiv(ma, AT_T), (unsigned)cdiv(mb, AT_T), (unsigned)nch);
    k_atb_part<<<grid, 256, 0, st>>>(A, lda, ma, B, ldb, mb, rows, rpc, part);
    RBKI_LAUNCH_CHECK("k_atb_part");
    k_atb_reduce<<<(unsigned)cdiv((int64_t)ma * mb, 256), 256, 0, st>>>(part, nch, ma, mb, out, ldo);
    RBKI_LAUNCH_CHECK("k_atb_reduce");
    return RBKI_OK;
}

// scratch: [ticket (8 doubles)] [chunk partials] [M] [G'] [Rinv] [nu2]
size_t orth_scratch_doubles(int64_t rows, int m, int S) {
    size_t mp = (size_t)(m + S) * S;
    return ORTH_TICKET_DOUBLES + (size_t)atb_nchunks(rows) * mp + mp + 2 * (size_t)S * S + S + 64;
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
    std::vector<atb_part_rec> ap(n);
    std::vector<atb_reduce_rec> ar(n);
    for (int k = 0; k < n; ++k) {
        const AtbItem& a = it[k];
        const int nch = atb_nchunks(a.rows);
        ap[k] = atb_part_rec{a.A, a.lda, a.ma, a.B, a.ldb, a.mb, a.rows, cdiv(a.rows, nch), a.part,
                             (int)cdiv(a.ma, AT_T), (int)cdiv(a.mb, AT_T), nch};
        if (a.sym && a.ma != a.mb) return set_error(RBKI_E_INVAL, "atb_batched: symmetric output of a non-square product");
        ar[k] = atb_reduce_rec{a.part, nch, a.ma, a.mb, a.out, a.ldo, a.sym, (int)cdiv((int64_t)a.ma * a.mb, 256), 1, 1};
    }
    RBKI_TRY(bat_launch(k_atb_part_b, ap.data(), n, 256, 0, st, "k_atb_part_b"));
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
        oh[k] = orth_head_rec{o.Q, o.ldq, o.m, S, o.rows, cdiv(o.rows, nch), nch, part, M, Gp, Rinv, nu2, tau, o.kept,
                              orth_ticket(o.scratch), (int)cdiv(ma, AT_T), (int)cdiv(S, AT_T), nch};
        oa[k] = orth_apply_rec{o.Q, o.ldq, o.rows, o.m, S, M, Rinv, (int)cdiv(o.rows, ORTH_ROWS), 1, 1};
        smax = std::max(smax, S);
    }
    const size_t sm = ((size_t)smax * smax + 2 * smax) * sizeof(double);
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
        if (it[k].dst) fr.push_back(fill_i32_rec{it[k].dst, it[k].v, 1, 1, 1});
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
