// rBKI-TK-TR (Algorithm 3): TR-ALS on the Tucker core G and the contraction of each TR core
// with its factor, FP64.
//
// Core k of the ring is Z_k (r_{k-1} x I_k x r_k), ring closed by r_{-1} = r_{N-1}; the core
// G satisfies G(i) ~ trace(Z_0(i_0) ... Z_{N-1}(i_{N-1})) (Eq. TR).  With the sub-chain
// M_c = Z_{k+1}(i_{k+1}) ... Z_{k-1}(i_{k-1}) (r_k x r_{k-1}) of unfolding column c (the
// C-order index of the other modes), G_(k) ~ Z_k(2) B^T with B[c, a r_k + b] = M_c[b, a]
// (Eq. unTR).  One ALS update is the exact least-squares solution
//   Z_k(2) = (G_(k) B) (B^T B)^{-1}
// (normal equations; reading c10).  B^T B is formed without B from transfer matrices
//   E_j[(al, al'), (be, be')] = sum_i Z_j(i)[al, be] Z_j(i)[al', be']
// as the chain E_{k+1} ... E_{k-1}; G_(k) B is a contraction of G with B laid out as
// [A][r^2][C] (the layout of the mode-k TTM result), computed by the split-reduce kernel.
// The fit after a sweep is measured from the explicit residual G_(k) - Z_k(2) B^T of the
// sweep's last update (the expansion |G|^2 - 2<G_(k)B, Z_k(2)> + <Z_k(2) B^T B, Z_k(2)>
// cancels catastrophically when the fit is close to 1).
#include "plan.h"

namespace rbki {
namespace {

constexpr int TR_RMAX = 8;

struct TrShape {
    int N;
    int64_t dims[RBKI_MAX_ORDER];   // core (Tucker rank) sizes R_n
    int r[RBKI_MAX_ORDER];          // r_n: core n is r[n-1] x dims[n] x r[n]
};

// B[a][s][c'] (column c = a*C + c' of G_(k)) = M_c[b, al], s = al * r_k + b
__global__ void k_tr_subchain(TrShape sh, int k, const double* const* cores, int64_t A, int64_t C,
                              double* __restrict__ Bout) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= A * C) return;
    const int N = sh.N;
    // multi-index of the other modes (C-order over modes != k)
    int idx[RBKI_MAX_ORDER];
    int64_t rem = c;
    for (int j = N - 1; j >= 0; --j) {
        if (j == k) continue;
        idx[j] = (int)(rem % sh.dims[j]);
        rem /= sh.dims[j];
    }
    // M = Z_{k+1}(i) Z_{k+2}(i) ... Z_{k-1}(i): rows r_k, running columns
    double M[TR_RMAX * TR_RMAX], T[TR_RMAX * TR_RMAX];
    int j = (k + 1) % N;
    int rows = sh.r[k];                       // = r_{j-1}
    int cols = sh.r[j];
    {
        const double* Z = cores[j];           // r_{j-1} x I_j x r_j
        const int64_t Ij = sh.dims[j];
        for (int p = 0; p < rows; ++p)
            for (int q = 0; q < cols; ++q) M[p * TR_RMAX + q] = Z[((int64_t)p * Ij + idx[j]) * cols + q];
    }
    for (int step = 2; step < N; ++step) {
        j = (k + step) % N;
        const double* Z = cores[j];
        const int64_t Ij = sh.dims[j];
        const int inner = cols, nc = sh.r[j];
        for (int p = 0; p < rows; ++p)
            for (int q = 0; q < nc; ++q) {
                double acc = 0.0;
                for (int t = 0; t < inner; ++t) acc += M[p * TR_RMAX + t] * Z[((int64_t)t * Ij + idx[j]) * nc + q];
                T[p * TR_RMAX + q] = acc;
            }
        for (int p = 0; p < rows; ++p)
            for (int q = 0; q < nc; ++q) M[p * TR_RMAX + q] = T[p * TR_RMAX + q];
        cols = nc;
    }
    // cols == r_{k-1}
    const int rk = sh.r[k], rkm = cols;
    const int S = rkm * rk;
    const int64_t a = c / C, cc = c - a * C;
    for (int al = 0; al < rkm; ++al)
        for (int b = 0; b < rk; ++b) Bout[(a * S + al * rk + b) * C + cc] = M[b * TR_RMAX + al];
}

// Transfer matrix of core j: E[(al, al'), (be, be')] = sum_i Z(i)[al, be] Z(i)[al', be']
__global__ void k_tr_transfer(const double* __restrict__ Z, int r0, int64_t I, int r1, double* __restrict__ E) {
    const int n0 = r0 * r0, n1 = r1 * r1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n0 * n1; t += gridDim.x * blockDim.x) {
        const int row = t / n1, col = t % n1;
        const int al = row / r0, alp = row % r0, be = col / r1, bep = col % r1;
        double acc = 0.0;
        for (int64_t i = 0; i < I; ++i) acc += Z[((int64_t)al * I + i) * r1 + be] * Z[((int64_t)alp * I + i) * r1 + bep];
        E[t] = acc;
    }
}

// One CTA: BtB = E_{k+1} ... E_{k-1} reshaped to [(al, b), (al', b')], then the normal
// equations Z_k(2) = GB (BtB)^{-1} by Cholesky (tiny diagonal shift relative to the trace
// when the Gram matrix is singular), and the fit terms.
//   E chain: entries [(b, b'), (al, al')] with b, b' over r_k and al, al' over r_{k-1}.
//   GB: I_k x S (S = r_{k-1} r_k, s = al * r_k + b).
// Writes core k (r_{k-1} x I_k x r_k).
__global__ void k_tr_solve(const double* const* Es, int nE, int rk, int rkm, const double* __restrict__ GB,
                           int64_t Ik, double* __restrict__ core, const double* __restrict__ work) {
    extern __shared__ double sm[];
    const int S = rkm * rk, S2 = S * S;
    constexpr int BS = TR_RMAX * TR_RMAX * TR_RMAX * TR_RMAX;   // every buffer holds r^4 entries
    double* P = sm;            // running chain product, (rk^2) x (cur^2)
    double* Q = P + BS;
    double* Bt = Q + BS;       // BtB S x S
    double* L = Bt + BS;       // Cholesky factor
    const int tid = threadIdx.x, nt = blockDim.x;
    // chain product of the transfer matrices (all square S x S only when r is uniform; in
    // general E_j is r_{j-1}^2 x r_j^2 and the chain goes from r_k^2 to r_{k-1}^2)
    // E list is given in order E_{k+1}, ..., E_{k-1}; dims carried in work[0..]
    const int* dd = reinterpret_cast<const int*>(work);   // dims of each E: rows, cols
    int rows = dd[0], cols = dd[1];
    for (int t = tid; t < rows * cols; t += nt) P[t] = Es[0][t];
    __syncthreads();
    for (int e = 1; e < nE; ++e) {
        const int c2 = dd[2 * e + 1];
        for (int t = tid; t < rows * c2; t += nt) {
            const int p = t / c2, q = t % c2;
            double acc = 0.0;
            for (int u = 0; u < cols; ++u) acc += P[p * cols + u] * Es[e][u * c2 + q];
            Q[t] = acc;
        }
        __syncthreads();
        for (int t = tid; t < rows * c2; t += nt) P[t] = Q[t];
        cols = c2;
        __syncthreads();
    }
    // rows = rk^2 over (b, b'), cols = rkm^2 over (al, al') -> Bt[(al, b), (al', b')]
    for (int t = tid; t < S2; t += nt) {
        const int s1 = t / S, s2 = t % S;
        const int al = s1 / rk, b = s1 % rk, alp = s2 / rk, bp = s2 % rk;
        Bt[t] = P[(b * rk + bp) * cols + (al * rkm + alp)];
    }
    __syncthreads();
    // Cholesky of Bt (S <= 64), serial over k with parallel row updates
    __shared__ double shift;
    if (tid == 0) {
        double tr = 0.0;
        for (int i = 0; i < S; ++i) tr += Bt[i * S + i];
        shift = 0.0;
        // detect singularity with a trial factorisation in thread 0 (S is small)
        for (int i = 0; i < S2; ++i) L[i] = Bt[i];
        bool ok = true;
        for (int kk = 0; kk < S && ok; ++kk) {
            double d = L[kk * S + kk];
            for (int t = 0; t < kk; ++t) d -= L[kk * S + t] * L[kk * S + t];
            if (!(d > 1e-13 * tr / S)) { ok = false; break; }
            d = sqrt(d);
            L[kk * S + kk] = d;
            for (int i = kk + 1; i < S; ++i) {
                double v = L[i * S + kk];
                for (int t = 0; t < kk; ++t) v -= L[i * S + t] * L[kk * S + t];
                L[i * S + kk] = v / d;
            }
        }
        if (!ok) {
            shift = 1e-12 * tr / S;
            for (int i = 0; i < S2; ++i) L[i] = Bt[i] + ((i / S == i % S) ? shift : 0.0);
            for (int kk = 0; kk < S; ++kk) {
                double d = L[kk * S + kk];
                for (int t = 0; t < kk; ++t) d -= L[kk * S + t] * L[kk * S + t];
                d = sqrt(fmax(d, 1e-300));
                L[kk * S + kk] = d;
                for (int i = kk + 1; i < S; ++i) {
                    double v = L[i * S + kk];
                    for (int t = 0; t < kk; ++t) v -= L[i * S + t] * L[kk * S + t];
                    L[i * S + kk] = v / d;
                }
            }
        }
    }
    __syncthreads();
    // rows of Z2: solve z (L L^T) = g  (forward then backward substitution), thread per row
    for (int64_t i = tid; i < Ik; i += nt) {
        double z[64];
        const double* g = GB + i * S;
        for (int p = 0; p < S; ++p) {
            double v = g[p];
            for (int t = 0; t < p; ++t) v -= L[p * S + t] * z[t];
            z[p] = v / L[p * S + p];
        }
        for (int p = S - 1; p >= 0; --p) {
            double v = z[p];
            for (int t = p + 1; t < S; ++t) v -= L[t * S + p] * z[t];
            z[p] = v / L[p * S + p];
        }
        for (int s = 0; s < S; ++s) {
            const int al = s / rk, b = s % rk;
            core[((int64_t)al * Ik + i) * rk + b] = z[s];
        }
    }
}

// Partial sums of squares of the residual G_(k) - Z_k(2) B^T, G viewed as [A][I][C], B as
// [A][S][C], core k as (al, i, b) with s = al * rk + b.  One partial per block.
constexpr int RES_BLOCKS = 608;
__global__ void __launch_bounds__(256) k_tr_resid(const double* __restrict__ G, int64_t A, int64_t I, int64_t C,
                                                  const double* __restrict__ B, int S, int rk,
                                                  const double* __restrict__ core, double* __restrict__ part) {
    double acc = 0.0;
    const int64_t n = A * I * C;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e % C;
        const int64_t t = e / C;
        const int64_t i = t % I, a = t / I;
        double v = G[e];
        for (int s = 0; s < S; ++s) {
            const int al = s / rk, b = s % rk;
            v -= core[((int64_t)al * I + i) * rk + b] * B[(a * S + s) * C + c];
        }
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

// Fixed-order sum of the partials (one warp) into *out.
__global__ void k_tr_sum(const double* __restrict__ part, int n, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) acc += part[i];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

// X_n[al, i, b] = sum_s U[i, s] Z_n[al, s, b]   (Algorithm 3 step 4)
__global__ void k_tr_contract(const double* __restrict__ Z, const double* __restrict__ U, int r0, int64_t Rn,
                              int r1, int64_t In, double* __restrict__ X) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)r0 * In * r1) return;
    const int b = (int)(t % r1);
    const int64_t i = (t / r1) % In;
    const int al = (int)(t / (r1 * In));
    double acc = 0.0;
    for (int64_t s = 0; s < Rn; ++s) acc += U[i * Rn + s] * Z[((int64_t)al * Rn + s) * r1 + b];
    X[t] = acc;
}

}  // namespace

struct TrPlan {
    TrShape sh;
    int64_t coreN;             // elements of G
    int64_t maxd;              // max over k of prod_{j != k} R_j
    int maxS;
    int64_t maxI;              // max over k of R_k
    int64_t maxpart;           // max over k of the contraction partials (doubles)
};

TrPlan tr_plan(int N, const int64_t* core_dims, const int32_t* ranks) {
    TrPlan p{};
    p.sh.N = N;
    p.coreN = 1;
    for (int n = 0; n < N; ++n) {
        p.sh.dims[n] = core_dims[n];
        p.sh.r[n] = ranks[n];
        p.coreN *= core_dims[n];
    }
    p.maxd = 0;
    p.maxS = 0;
    p.maxI = 0;
    p.maxpart = 0;
    for (int k = 0; k < N; ++k) {
        const int64_t d = p.coreN / core_dims[k];
        const int S = ranks[(k + N - 1) % N] * ranks[k];
        p.maxd = std::max(p.maxd, d);
        p.maxS = std::max(p.maxS, S);
        p.maxI = std::max(p.maxI, core_dims[k]);
        int64_t A = 1;
        for (int j = 0; j < k; ++j) A *= core_dims[j];
        const View v{nullptr, RBKI_F64, A, core_dims[k], d / A};
        p.maxpart = std::max(p.maxpart, (int64_t)contract_nsplit(v) * core_dims[k] * S);
    }
    return p;
}

size_t tr_workspace_doubles(const TrPlan& p) {
    size_t s = 0;
    s += (size_t)p.maxd * p.maxS + 64;                              // B
    s += (size_t)p.maxI * p.maxS + 64;                              // GB
    s += (size_t)p.maxpart + 64;                                    // contraction partials
    s += (size_t)p.sh.N * TR_RMAX * TR_RMAX * TR_RMAX * TR_RMAX + 64;   // transfer matrices
    s += 64 * RBKI_MAX_ORDER + 64;                                   // per-core metadata + stats
    s += RES_BLOCKS + 64;                                            // residual partials
    s += (size_t)p.coreN + 64;                                      // fit scratch
    return s;
}

// Runs TR-ALS on G (device, FP64, dims = core dims) from `cores` (device, initial values,
// updated in place).  fits_host[t] receives Fit_t (fraction); returns the number of sweeps.
rbki_status tr_als_cuda(const TrPlan& p, const double* G, double g_norm2, double* const* cores_dev,
                        const double* const* cores_ptr_table_dev, int maxit, double tol, double* ws,
                        double* fits_host, int* sweeps_out, cudaStream_t st) {
    const int N = p.sh.N;
    double* B = ws;
    double* GB = B + (size_t)p.maxd * p.maxS + 64;
    double* part = GB + (size_t)p.maxI * p.maxS + 64;
    double* Ebuf = part + (size_t)p.maxpart + 64;
    double* meta = Ebuf + (size_t)N * TR_RMAX * TR_RMAX * TR_RMAX * TR_RMAX + 64;
    double* stats = meta + 56 * RBKI_MAX_ORDER;
    double* rpart = meta + 64 * RBKI_MAX_ORDER + 64;
    const size_t Estride = (size_t)TR_RMAX * TR_RMAX * TR_RMAX * TR_RMAX;
    // per-core metadata (transfer-matrix dims and pointers in chain order k+1 .. k-1), built
    // once: the transfer matrices of core j live at Ebuf + j * Estride for the whole run
    struct Meta { int dims[2 * RBKI_MAX_ORDER]; const double* E[RBKI_MAX_ORDER]; };
    static thread_local Meta host_meta[RBKI_MAX_ORDER];
    for (int k = 0; k < N; ++k) {
        for (int e = 0; e < RBKI_MAX_ORDER; ++e) {
            host_meta[k].dims[2 * e] = host_meta[k].dims[2 * e + 1] = 0;
            host_meta[k].E[e] = nullptr;
        }
        for (int e = 0; e < N - 1; ++e) {
            const int j = (k + 1 + e) % N;
            const int r0 = p.sh.r[(j + N - 1) % N], r1 = p.sh.r[j];
            host_meta[k].dims[2 * e] = r0 * r0;
            host_meta[k].dims[2 * e + 1] = r1 * r1;
            host_meta[k].E[e] = Ebuf + j * Estride;
        }
    }
    Meta* dmeta = reinterpret_cast<Meta*>(meta);
    RBKI_CUDA_TRY(cudaMemcpyAsync(dmeta, host_meta, N * sizeof(Meta), cudaMemcpyHostToDevice, st));
    RBKI_CUDA_TRY(cudaStreamSynchronize(st));
    static const size_t smax = max_dyn_smem(k_tr_solve);   // thread-safe, once
    const size_t smem = 4 * (size_t)TR_RMAX * TR_RMAX * TR_RMAX * TR_RMAX * sizeof(double);
    if (smem > smax) return set_error(RBKI_E_UNSUPPORTED, "TR-ALS: ranks too large");
    double prev = -1.0;
    int sweeps = 0;
    for (int it = 0; it < maxit; ++it) {
        for (int k = 0; k < N; ++k) {
            int64_t A = 1, C = 1;
            for (int j = 0; j < k; ++j) A *= p.sh.dims[j];
            for (int j = k + 1; j < N; ++j) C *= p.sh.dims[j];
            const int rk = p.sh.r[k], rkm = p.sh.r[(k + N - 1) % N];
            const int S = rk * rkm;
            // sub-chain B in [A][S][C] layout, then GB = G_(k) B
            k_tr_subchain<<<(unsigned)cdiv(A * C, 128), 128, 0, st>>>(p.sh, k, cores_ptr_table_dev, A, C, B);
            RBKI_LAUNCH_CHECK("k_tr_subchain");
            View v{G, RBKI_F64, A, p.sh.dims[k], C};
            RBKI_TRY(contract_cuda(v, B, RBKI_F64, S, false, part, contract_nsplit(v), GB, S, nullptr, 0, st));
            // transfer matrices of the other cores (current values)
            for (int e = 0; e < N - 1; ++e) {
                const int j = (k + 1 + e) % N;
                const int r0 = p.sh.r[(j + N - 1) % N], r1 = p.sh.r[j];
                k_tr_transfer<<<(unsigned)cdiv((int64_t)r0 * r0 * r1 * r1, 128), 128, 0, st>>>(
                    cores_dev[j], r0, p.sh.dims[j], r1, Ebuf + j * Estride);
                RBKI_LAUNCH_CHECK("k_tr_transfer");
            }
            k_tr_solve<<<1, 256, smem, st>>>(dmeta[k].E, N - 1, rk, rkm, GB, p.sh.dims[k], cores_dev[k],
                                             reinterpret_cast<const double*>(dmeta[k].dims));
            RBKI_LAUNCH_CHECK("k_tr_solve");
            if (k == N - 1) {
                // |G - TR(Z)|^2 from the residual of the sweep's last update (B is current)
                const int blocks = (int)std::min<int64_t>(RES_BLOCKS, std::max<int64_t>(1, cdiv(p.coreN, 256)));
                k_tr_resid<<<blocks, 256, 0, st>>>(G, A, p.sh.dims[k], C, B, S, rk, cores_dev[k], rpart);
                RBKI_LAUNCH_CHECK("k_tr_resid");
                k_tr_sum<<<1, 32, 0, st>>>(rpart, blocks, stats);
                RBKI_LAUNCH_CHECK("k_tr_sum");
            }
        }
        // fit after the sweep
        double err2 = 0.0;
        RBKI_CUDA_TRY(cudaMemcpyAsync(&err2, stats, sizeof(double), cudaMemcpyDeviceToHost, st));
        RBKI_CUDA_TRY(cudaStreamSynchronize(st));
        const double fit = 1.0 - std::sqrt(std::max(0.0, err2) / g_norm2);
        if (fits_host) fits_host[it] = fit;
        sweeps = it + 1;
        if (prev >= -0.5 && std::fabs(fit - prev) <= tol) break;
        prev = fit;
    }
    if (sweeps_out) *sweeps_out = sweeps;
    return RBKI_OK;
}

size_t tr_workspace_doubles_for(int N, const int64_t* core_dims, const int32_t* ranks) {
    return tr_workspace_doubles(tr_plan(N, core_dims, ranks));
}

rbki_status tr_run(int N, const int64_t* core_dims, const int32_t* ranks, const double* G, double g_norm2,
                   double* const* cores_dev, const double* const* cores_table_dev, int maxit, double tol,
                   double* ws, double* fits_host, int* sweeps, cudaStream_t st) {
    for (int n = 0; n < N; ++n)
        if (ranks[n] < 1 || ranks[n] > TR_RMAX) return set_error(RBKI_E_UNSUPPORTED, "TR ranks must be in [1, 8]");
    const TrPlan p = tr_plan(N, core_dims, ranks);
    return tr_als_cuda(p, G, g_norm2, cores_dev, cores_table_dev, maxit, tol, ws, fits_host, sweeps, st);
}

// ---- TR-SVD (the alternative step 3 of Algorithm 3; Zhao et al. 2016) ----------------
// Step n takes the truncated SVD of C_n ((r_{n-1} S_n) x rest; S_1 x rest for n = 0) from
// the Gram matrix C_n C_n^T: U = its leading r eigenvectors (the FP64-refined eigensolver),
// sign-normalised,
// the remainder U^T C_n = Sigma V^T by a TTM, and the step's squared truncation error
// trace(C C^T) - sum of the r eigenvalues.  Step 0 splits the rank product r_{N-1} r_0:
// core 0 [a][i][b] = U[i][a r_0 + b], and the remainder is reordered (a, b, rest) ->
// (b, rest, a).  The last core is the remaining C_{N-1}.
namespace {

// core0[a][i][b] = U[i][a * r0 + b]
__global__ void k_trsvd_core0(const double* __restrict__ U, int64_t S, int ra, int r0, double* __restrict__ Z) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)ra * S * r0;
    if (e >= tot) return;
    const int b = (int)(e % r0);
    const int64_t i = (e / r0) % S;
    const int a = (int)(e / (r0 * S));
    Z[e] = U[i * ((int64_t)ra * r0) + (int64_t)a * r0 + b];
}

// out[b][c][a] = W[a * r0 + b][c]  (W: (ra r0) x ncol)
__global__ void k_trsvd_reorder(const double* __restrict__ W, int ra, int r0, int64_t ncol, double* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)ra * r0 * ncol;
    if (e >= tot) return;
    const int a = (int)(e % ra);
    const int64_t c = (e / ra) % ncol;
    const int b = (int)(e / (ra * ncol));
    out[e] = W[((int64_t)a * r0 + b) * ncol + c];
}

// err2 += trace(Gram) - sum_{k<r} w[k]; step 0 also records |G|^2 = trace
__global__ void k_trsvd_err(const double* __restrict__ gram, int m, const double* __restrict__ w, int r,
                            double* __restrict__ acc, int first) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tr = 0.0, top = 0.0;
    for (int i = 0; i < m; ++i) tr += gram[(int64_t)i * m + i];
    for (int k = 0; k < r; ++k) top += w[k];
    if (first) {
        acc[0] = tr;
        acc[1] = 0.0;
    }
    acc[1] += tr - top;
}

__global__ void k_trsvd_fit(const double* __restrict__ acc, double* __restrict__ fits, int nfits) {
    const int i = threadIdx.x;
    if (i >= nfits) return;
    if (i == 0) {
        const double g2 = acc[0], e2 = acc[1] > 0.0 ? acc[1] : 0.0;
        fits[0] = g2 > 0.0 ? 1.0 - sqrt(e2 / g2) : 1.0;
    } else {
        fits[i] = __longlong_as_double(0x7ff8000000000000LL);
    }
}

constexpr int TRSVD_SPLIT = 8;   // split-K partials of the Gram contraction

}  // namespace

size_t trsvd_workspace_doubles(int N, const int64_t* S, const int32_t* r) {
    int64_t numel = 1;
    for (int n = 0; n < N; ++n) numel *= S[n];
    return 2 * (size_t)rup(numel, 32) + 256 * 256 + 256 + 256 * 256 + syev_scratch_doubles(256) +
           (size_t)TRSVD_SPLIT * 256 * 256 + 64;
}

rbki_status tr_svd_cuda(int N, const int64_t* S, const int32_t* r, const double* G, double* const* cores,
                        double* ws, double* fits, int nfits, cudaStream_t st) {
    if (N < 2) return set_error(RBKI_E_INVAL, "TR-SVD needs order >= 2");
    int64_t numel = 1;
    for (int n = 0; n < N; ++n) numel *= S[n];
    double* buf[2] = {ws, ws + rup(numel, 32)};
    double* gram = buf[1] + rup(numel, 32);
    double* w = gram + 256 * 256;
    double* V = w + 256;
    double* eig_ws = V + 256 * 256;
    double* part = eig_ws + syev_scratch_doubles(256);
    double* acc = part + (size_t)TRSVD_SPLIT * 256 * 256;
    const double* C = G;
    int64_t rows = S[0], cols = numel / S[0];
    for (int n = 0; n + 1 < N; ++n) {
        const int rk = n == 0 ? r[N - 1] * r[0] : r[n];
        if (rows > 256) return set_error(RBKI_E_UNSUPPORTED, "TR-SVD: unfolding rows > 256");
        if (rk > rows || rk > cols) return set_error(RBKI_E_INVAL, "TR-SVD: rank exceeds the unfolding");
        const View v{C, RBKI_F64, 1, rows, cols};
        const int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(TRSVD_SPLIT, cdiv(cols, 256)));
        RBKI_TRY(contract_cuda(v, C, RBKI_F64, (int)rows, false, part, nsplit, gram, rows, nullptr, 0, st));
        RBKI_TRY(symmetrize_cuda(gram, (int)rows, st));
        RBKI_TRY(syev_top_cuda(gram, (int)rows, rk, w, V, eig_ws, st));
        k_trsvd_err<<<1, 32, 0, st>>>(gram, (int)rows, w, rk, acc, n == 0);
        RBKI_LAUNCH_CHECK("k_trsvd_err");
        // U = the leading eigenvectors, each column's largest-|.| entry made positive (the
        // split of step 0 mixes bond indices, so the result depends on the signs); the Gram
        // matrix is no longer needed, U takes its place
        double* U = gram;
        RBKI_TRY(form_factor_cuda(nullptr, 0, rows, V, (int)rows, rk, rk, U, st));
        double* W = C == buf[0] ? buf[1] : buf[0];                     // never the buffer C is in
        RBKI_TRY(ttm_cuda(v, U, rk, rk, W, RBKI_F64, false, st));       // W = U^T C, rk x cols
        if (n == 0) {
            const int64_t tot = (int64_t)r[N - 1] * S[0] * r[0];
            k_trsvd_core0<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(U, S[0], r[N - 1], r[0], cores[0]);
            RBKI_LAUNCH_CHECK("k_trsvd_core0");
            double* R = buf[1];                                          // W is buf[0] here
            k_trsvd_reorder<<<(unsigned)cdiv((int64_t)rk * cols, 256), 256, 0, st>>>(W, r[N - 1], r[0], cols, R);
            RBKI_LAUNCH_CHECK("k_trsvd_reorder");
            C = R;
            rows = (int64_t)r[0] * S[1];
            cols = (int64_t)cols * r[N - 1] / S[1];
        } else {
            RBKI_CUDA_TRY(cudaMemcpyAsync(cores[n], U, (size_t)rows * rk * sizeof(double), cudaMemcpyDeviceToDevice,
                                          st));
            C = W;
            rows = (int64_t)r[n] * S[n + 1];
            cols = (int64_t)rk * cols / rows;
        }
    }
    RBKI_CUDA_TRY(cudaMemcpyAsync(cores[N - 1], C, (size_t)r[N - 2] * S[N - 1] * r[N - 1] * sizeof(double),
                                  cudaMemcpyDeviceToDevice, st));
    if (fits && nfits > 0) {
        k_trsvd_fit<<<1, 1024, 0, st>>>(acc, fits, nfits > 1024 ? 1024 : nfits);
        RBKI_LAUNCH_CHECK("k_trsvd_fit");
    }
    return RBKI_OK;
}

rbki_status tr_contract_cuda(const double* Z, const double* U, int r0, int64_t Rn, int r1, int64_t In, double* X,
                             cudaStream_t st) {
    const int64_t tot = (int64_t)r0 * In * r1;
    k_tr_contract<<<(unsigned)cdiv(tot, 256), 256, 0, st>>>(Z, U, r0, Rn, r1, In, X);
    RBKI_LAUNCH_CHECK("k_tr_contract");
    return RBKI_OK;
}

}  // namespace rbki
