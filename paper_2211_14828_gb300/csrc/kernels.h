// Internal launch wrappers of librbki (host side).  Not part of the C ABI.
#pragma once

#include <vector>

#include "common.cuh"

namespace rbki {

// View of the streamed tensor for mode n: X as [A][I][C] (A = prod of dims before n,
// C = prod of dims after n).  Column `col` of X_(n) is (a, c) = (col / C, col % C).
struct View {
    const void* data;
    int dtype;  // RBKI_F64 / F32 / BF16 / F16
    int64_t A, I, C;
};

// ---- partial column sampling (k_sample.cu) ----
// the `kept` units (of nu) with the smallest Philox keys, ascending, into units[kept]
rbki_status sample_units_cuda(uint64_t seed, int mode, int64_t nu, int64_t kept, int32_t* units,
                              cudaStream_t st);
// sampled unfolding Y of the kept units: [kept][I][128] (C > 1) or [kept * 128][I] (C = 1)
rbki_status gather_units_cuda(const void* x, int dtype, int64_t A, int64_t I, int64_t C, const int32_t* units,
                              int64_t kept, void* y, cudaStream_t st);

// ---- divide-and-conquer split (k_split.cu) ----
// dst[k] (dense [A][I_k][C]) = X[:, floor(k I / parts) : floor((k+1) I / parts), :]
rbki_status split_mode_cuda(const void* x, int dtype, int64_t A, int64_t I, int64_t C, int parts, void* const* dst,
                            cudaStream_t st);

// ---- FP64/FP32 CUDA-core streaming products (k_stream.cu) ----
// Gram path of a short mode (I <= 8; I <= 16 with FP32 accumulation): out (I x I, ld) = X_(n) X_(n)^T, one pass, partials
// [nblocks][I][I] in `part`, fixed-order reduce
rbki_status gram_small_cuda(const View& x, bool acc32, double* part, int nblocks, double* out, int64_t ld,
                            cudaStream_t st);
// TTM: Y[a][s][c] = sum_i M[i*ldm + s] X[a][i][c],  s < S.  Y is [A][S][C] (Tout).
// `acc32` = accumulate in FP32 (mixed path), else FP64.
// Y (FP64, [A][S][C]) = X x_n M^T for S <= 32 (F64/F32 input): the small core-chain products
rbki_status ttm_small_cuda(const View& x, const double* M, int64_t ldm, int S, double* Y, bool acc32,
                           cudaStream_t st);
rbki_status ttm_cuda(const View& x, const double* M, int64_t ldm, int S, void* Y, int y_dtype,
                     bool acc32, cudaStream_t st);
// Contraction: P[i][s] = sum_{a,c} X[a][i][c] Y[a][s][c] (split over columns into nsplit
// partials `part` [nsplit][I][S], then a fixed-order reduce into out (ld_out) and out2).
// Y has element type y_dtype (RBKI_F64 or the tensor's dtype).  Gram: Y == X, S == I.
rbki_status contract_cuda(const View& x, const void* Y, int y_dtype, int S, bool acc32,
                          double* part, int nsplit, double* out, int64_t ld_out,
                          double* out2, int64_t ld_out2, cudaStream_t st);
int contract_nsplit(const View& x);

// FP64 Omega in the [A][S][C] layout of a TTM result (k_omega.cu).
rbki_status omega_f64_cuda(uint64_t seed, int mode, int64_t A, int64_t C, int S, double* Y,
                           cudaStream_t st);

// sum of squares of n elements (FP64 result into *out) - partials in `part` (>= 1024 doubles)
rbki_status sumsq_cuda(const void* x, int dtype, int64_t n, double* part, double* out,
                       cudaStream_t st);
// cast to bf16/f16 (dst_dtype) + sum of squares of the source
// *out = the fixed-order sum of part[0 .. nparts)
rbki_status sum_parts_cuda(const double* part, int nparts, double* out, cudaStream_t st);
rbki_status stage_cuda(const void* x, int dtype, int64_t n, void* dst, int dst_dtype,
                       double* part, double* norm2, cudaStream_t st);

// ---- small dense FP64 kernels (k_small.cu) ----
// out (ma x mb, ld ldo) = A^T B over `rows` rows; A: rows x ma (lda), B: rows x mb (ldb).
// Partial sums over chunks of rows, summed in FP64 in a fixed order; f32: the operands
// rounded to FP32 and FP32 sums within a chunk (the mixed path's Z = Q^T P).
int atb_nchunks(int64_t rows);
rbki_status atb_cuda(const double* A, int64_t lda, int ma, const double* B, int64_t ldb, int mb,
                     int64_t rows, double* part, double* out, int64_t ldo, cudaStream_t st, bool f32 = false);
// One pass of block orthonormalisation (Pythagorean-inner-product block Gram-Schmidt
// followed by Cholesky QR with pivot deflation).  Q: rows x ldq, block = columns
// [m, m+S); earlier columns [0, m) are orthonormal.  In place.
rbki_status orth_pass_cuda(double* Q, int64_t ldq, int64_t rows, int m, int S, double tau,
                           double* scratch, int32_t* kept, cudaStream_t st);
size_t orth_scratch_doubles(int64_t rows, int m, int S);
// the first ORTH_TICKET_DOUBLES of an orthonormalisation scratch hold the batched pass's
// ticket counter (orth_ticket), which must be 0 before the first orth_pass_batched on it
constexpr size_t ORTH_TICKET_DOUBLES = 8;
constexpr int ORTH_TICKETS = (int)(ORTH_TICKET_DOUBLES * 2);   // int32 words to zero
int32_t* orth_ticket(double* scratch);
// C (M x N, ld ldc) = op(A) B + beta C; op(A) = A^T (A: K x M, ld lda) when transA, else A
// (M x K); B: K x N (ld ldb).  Split over K into `part` (gemm_part_doubles), fixed-order reduce.
size_t gemm_part_doubles(int M, int N, int K);
rbki_status gemm_f64_cuda(bool transA, int M, int N, int K, const double* A, int64_t lda, const double* B,
                          int64_t ldb, double* C, int64_t ldc, double beta, double* part, cudaStream_t st);
// symmetric eigensolver (k_eig.cu), descending; V (n x n row-major) columns are eigenvectors
rbki_status syev_cuda(const double* A, int n, double* w, double* V, double* scratch,
                      cudaStream_t st);
// leading nwant eigenpairs only: w (nwant), V (n x nwant row-major)
rbki_status syev_top_cuda(const double* A, int n, int nwant, double* w, double* V, double* scratch,
                          cudaStream_t st);
size_t syev_scratch_doubles(int n);
// U[i][k] = sum_t Q[i*ldq + t] V[t*ldv + k] (k < R); then sign-normalise each column.
// Q == nullptr means identity (Gram path): U = V[:, :R].
rbki_status form_factor_cuda(const double* Q, int64_t ldq, int64_t rows, const double* V, int n,
                             int ldv, int R, double* U, cudaStream_t st);
rbki_status copy_f64_cuda(const double* src, double* dst, int64_t n, cudaStream_t st);
rbki_status fill_i32_cuda(int32_t* dst, int32_t v, int n, cudaStream_t st);

// Opt a kernel into the largest dynamic shared memory the device allows next to its static
// shared memory; returns that maximum (bytes) or 0 on error.
template <typename K>
inline size_t max_dyn_smem(K kernel) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 0;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t mx = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx) != cudaSuccess)
        return 0;
    return mx;
}

// deflation threshold of the block orthonormalisation (reading c3): a column is dropped when
// its norm orthogonal to the accepted ones is <= tau times its norm before projection
constexpr double TAU_DEFLATE = 1e-6;

// ---- batched launches ----
// The batched twin `k_x_b` of a kernel `k_x` runs one launch for up to BMAX independent
// items.  The items' arguments travel as records in the kernel parameter buffer (sm_90 and
// later accept 32 KB of parameters, so no copy precedes the launch); blockIdx.y selects the
// record and blockIdx.x is the item's own block index, flattened over the item's grid
// (gx, gy, gz).  Both kernels call the same device body, so every item does exactly the
// arithmetic, in the same order, of its single launch, whatever else shares the launch.
constexpr int BMAX = 128;
template <class R>
struct BPack {
    static_assert(sizeof(R) * BMAX <= 32000, "record too large for the kernel parameter buffer");
    R r[BMAX];
};
template <class R>
__device__ __forceinline__ bool bat_block(const R& r, int& bx, int& by, int& bz) {
    const int b = (int)blockIdx.x;
    if (b >= r.gx * r.gy * r.gz) return false;
    bx = b % r.gx;
    by = (b / r.gx) % r.gy;
    bz = b / (r.gx * r.gy);
    return true;
}
// Launches kernel(pack) over recs[0..n) in packs of BMAX; grid.x = the largest item grid.
template <class R, class K>
rbki_status bat_launch(K kernel, const R* recs, int n, int threads, size_t smem, cudaStream_t st,
                       const char* where) {
    static thread_local BPack<R> pack;
    for (int i0 = 0; i0 < n; i0 += BMAX) {
        const int cnt = std::min(BMAX, n - i0);
        int gmax = 0;
        for (int i = 0; i < cnt; ++i) {
            pack.r[i] = recs[i0 + i];
            gmax = std::max(gmax, recs[i0 + i].gx * recs[i0 + i].gy * recs[i0 + i].gz);
        }
        if (gmax == 0) continue;
        kernel<<<dim3((unsigned)gmax, (unsigned)cnt), threads, smem, st>>>(pack);
        RBKI_LAUNCH_CHECK(where);
    }
    return RBKI_OK;
}

// batched forms of the small FP64 stages (k_small.cu): item k of each array is independent
struct AtbItem {
    const double* A; int64_t lda; int ma;
    const double* B; int64_t ldb; int mb;
    int64_t rows; double* part; double* out; int64_t ldo;
    int sym = 0;   // ma == mb: out = (A^T B + B^T A) / 2, the product and its symmetrisation
    int f32 = 0;   // operands rounded to FP32, FP32 sums within a chunk of rows (atb_cuda's f32)
};
rbki_status atb_batched(const AtbItem* it, int n, cudaStream_t st);
struct OrthItem {
    double* Q; int64_t ldq; int64_t rows; int m; int S; double* scratch; int32_t* kept;
};
rbki_status orth_pass_batched(const OrthItem* it, int n, double tau, cudaStream_t st);
struct FillItem { int32_t* dst; int32_t v; int n = 1; };   // dst[0..n) = v (dst == nullptr: skipped)
rbki_status fill_i32_batched(const FillItem* it, int n, cudaStream_t st);
struct GemmItem {
    bool transA; int M, N, K;
    const double* A; int64_t lda; const double* B; int64_t ldb;
    double* C; int64_t ldc; double beta; double* part;
};
rbki_status gemm_f64_batched(const GemmItem* it, int n, cudaStream_t st);
struct FormItem {
    const double* Q; int64_t ldq; int64_t rows; const double* V; int n; int ldv; int R; double* U;
};
rbki_status form_factor_batched(const FormItem* it, int n, cudaStream_t st);
struct CopyItem {
    const double* src; double* dst; int64_t n;
};
rbki_status copy_f64_batched(const CopyItem* it, int n, cudaStream_t st);
// eigensolver (k_eig.cu): the leading nwant eigenpairs of each item's A
struct EigItem {
    const double* A; int n; int nwant; double* w; double* V; double* scratch;
};
rbki_status syev_top_batched(const EigItem* it, int n, cudaStream_t st);

// profiling hook (api.cu): returns a token for prof_end, or -1 when profiling is off
int prof_begin(int cls, cudaStream_t st);
void prof_end(int token, cudaStream_t st);

}  // namespace rbki
