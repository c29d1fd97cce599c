// Symmetric eigensolver for Algorithm 2 step 4 (Z = Q^T X X^T Q, b x b, b <= 256): FP64
// leading `nwant` eigenpairs.
//
// GB300 runs FP64 FMAs at 1/58 of the FP32 rate (1.26 vs 73 TFLOP/s measured), and an
// O(b^3) FP64 reduction on one SM takes milliseconds.  The solver therefore splits the
// work by precision:
//   1. a full eigendecomposition of Z in FP32 on one CTA:
//        Householder tridiagonalisation (Householder 1958; the symmetric rank-2 update
//        form of LAPACK's xSYTD2), bisection with Sturm counts (Givens 1954) for the
//        eigenvalues, fixed-shift inverse iteration on the tridiagonal (Gaussian
//        elimination with partial pivoting), one Cholesky QR of the eigenvector block
//        (mixes vectors only inside clusters),
//        back-transformation by the reflectors (one warp per eigenvector);
//   2. FP64 iterative refinement of the leading `nwant` eigenvectors by the method of
//        Ogita & Aishima ("Iterative refinement for symmetric eigenvalue decomposition",
//        Japan J. Indust. Appl. Math. 35, 2018), restricted to the wanted columns: with
//        X the approximate eigenvector matrix and X1 its first nwant columns,
//          G = X^T X1,  S = X^T (Z X1),  r_ij = delta_ij - g_ij,
//          lambda_j = s_jj / (1 - r_jj),
//          e_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)   (i != j, separated)
//          e_ij = r_ij / 2                                          (i == j or clustered)
//          X1 <- X1 + X E.
//      All products are FP64 GEMMs of b x b x nwant spread over many CTAs.  Two sweeps
//      take FP32-accurate vectors (~1e-6) to FP64 accuracy for eigenvalues separated
//      from the rest; within a cluster only the span is refined.
#include "kernels.h"

namespace rbki {
namespace {

template <typename T>
__device__ T block_sum(T v, T* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        T t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : (T)0;
        t = warp_sum(t);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Tridiagonalise A (n x n, symmetric, FP64 input) in precision T: d[n], e[n-1]; reflector
// k (unit vector acting on rows k+1..n-1, zero if none) stored as row k of `refl`.  The
// working matrix lives in shared memory with an odd leading dimension (n+1) when it fits,
// otherwise in `work` (global, L2 resident).
template <typename T>
__device__ __forceinline__ T block_sum1(T v, T* part, int nwarps) {
    // warp partials to shared memory, one barrier, every thread adds the partials itself
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = 0;
    for (int w = 0; w < nwarps; ++w) t += part[w];
    return t;
}

template <typename T>
__global__ void __launch_bounds__(512) k_tridiag(const double* __restrict__ A, int n, T* __restrict__ work,
                                                 int use_smem, T* __restrict__ d, T* __restrict__ e,
                                                 T* __restrict__ refl) {
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    const int ld = use_smem ? n + 1 : n;
    T* a = use_smem ? reinterpret_cast<T*>(tsm_raw) : work;
    __shared__ T v[256], u[256];
    __shared__ T part_a[16], part_b[16];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int t = tid; t < n * n; t += nt) a[(t / n) * ld + t % n] = (T)A[t];
    for (int t = tid; t < n * n; t += nt) refl[t] = (T)0;
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        const int o = k + 1;
        const T x0 = a[o * ld + k];
        T s1 = 0;
        for (int i = 1 + tid; i < m; i += nt) {
            const T x = a[(o + i) * ld + k];
            s1 += x * x;
        }
        T* part = (k & 1) ? part_b : part_a;          // alternate buffers: no reuse barrier
        s1 = block_sum1(s1, part, nw);
        if (tid == 0) d[k] = a[k * ld + k];
        if (s1 == (T)0) {
            if (tid == 0) e[k] = x0;
            __syncthreads();
            continue;
        }
        const T nrm = sqrt(x0 * x0 + s1);
        const T alpha = x0 >= (T)0 ? -nrm : nrm;
        const T v0 = x0 - alpha;
        const T inv = (T)1 / sqrt(v0 * v0 + s1);
        for (int i = tid; i < m; i += nt) {
            const T vi = (i == 0 ? v0 : a[(o + i) * ld + k]) * inv;
            v[i] = vi;
            refl[(size_t)k * n + o + i] = vi;
        }
        if (tid == 0) e[k] = alpha;
        __syncthreads();
        // u = B v with four threads per row (adjacent lanes), g = v^T u from the same pass
        T gp = 0;
        for (int base = 0; base < m; base += nt / 4) {
            const int i = base + tid / 4, q = tid & 3;
            T acc = 0;
            if (i < m) {
                const T* row = a + (size_t)(o + i) * ld + o;
                for (int j = q; j < m; j += 4) acc += row[j] * v[j];
            }
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (i < m && q == 0) {
                u[i] = acc;
                gp += acc * v[i];
            }
        }
        part = (k & 1) ? part_a : part_b;
        const T g = block_sum1(gp, part, nw);
        for (int i = tid; i < m; i += nt) u[i] = (T)2 * u[i] - (T)2 * g * v[i];   // w
        __syncthreads();
        // B -= v w^T + w v^T: warp per row on the lower triangle, mirrored
        for (int i = wid; i < m; i += nw) {
            const T vi = v[i], wi = u[i];
            T* row = a + (size_t)(o + i) * ld + o;
            for (int j = lane; j <= i; j += 32) {
                const T val = row[j] - vi * u[j] - wi * v[j];
                row[j] = val;
                a[(size_t)(o + j) * ld + o + i] = val;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            d[n - 2] = a[(n - 2) * ld + n - 2];
            e[n - 2] = a[(n - 1) * ld + n - 2];
        }
        d[n - 1] = a[(n - 1) * ld + n - 1];
    }
}

// Shared-memory variant for n where the full n x (n+1) FP32 matrix no longer fits (n > 237):
// the lower triangle, packed row by row (element (i, j), j <= i, at i (i + 1) / 2 + j: 126 KB
// for n = 256), with the same Householder steps as k_tridiag.  u = B v takes row i's
// stored part (j <= i, contiguous) and its mirrored part (j > i, read down column i); the
// rank-2 update touches the lower triangle only.
template <typename T>
__global__ void __launch_bounds__(512) k_tridiag_packed(const double* __restrict__ A, int n, T* __restrict__ d,
                                                        T* __restrict__ e, T* __restrict__ refl) {
    extern __shared__ __align__(16) unsigned char tp_raw[];
    T* a = reinterpret_cast<T*>(tp_raw);
    auto at = [&](int i, int j) -> T& { return a[(size_t)i * (i + 1) / 2 + j]; };   // j <= i
    __shared__ T v[256], u[256];
    __shared__ T part_a[16], part_b[16];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int t = tid; t < n * n; t += nt) {
        const int i = t / n, j = t % n;
        if (j <= i) at(i, j) = (T)A[t];
    }
    for (int t = tid; t < n * n; t += nt) refl[t] = (T)0;
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        const int o = k + 1;
        const T x0 = at(o, k);
        T s1 = 0;
        for (int i = 1 + tid; i < m; i += nt) {
            const T x = at(o + i, k);
            s1 += x * x;
        }
        T* part = (k & 1) ? part_b : part_a;
        s1 = block_sum1(s1, part, nw);
        if (tid == 0) d[k] = at(k, k);
        if (s1 == (T)0) {
            if (tid == 0) e[k] = x0;
            __syncthreads();
            continue;
        }
        const T nrm = sqrt(x0 * x0 + s1);
        const T alpha = x0 >= (T)0 ? -nrm : nrm;
        const T v0 = x0 - alpha;
        const T inv = (T)1 / sqrt(v0 * v0 + s1);
        for (int i = tid; i < m; i += nt) {
            const T vi = (i == 0 ? v0 : at(o + i, k)) * inv;
            v[i] = vi;
            refl[(size_t)k * n + o + i] = vi;
        }
        if (tid == 0) e[k] = alpha;
        __syncthreads();
        // u = B v: warp per row, lanes over the row's stored and mirrored parts
        T gp = 0;
        for (int i = wid; i < m; i += nw) {
            T acc = 0;
            const T* row = a + (size_t)(o + i) * (o + i + 1) / 2 + o;
            for (int j = lane; j <= i; j += 32) acc += row[j] * v[j];
            for (int j = i + 1 + lane; j < m; j += 32) acc += at(o + j, o + i) * v[j];
            acc = warp_sum(acc);
            if (lane == 0) {
                u[i] = acc;
                gp += acc * v[i];
            }
        }
        part = (k & 1) ? part_a : part_b;
        const T g = block_sum1(gp, part, nw);
        for (int i = tid; i < m; i += nt) u[i] = (T)2 * u[i] - (T)2 * g * v[i];   // w
        __syncthreads();
        // B -= v w^T + w v^T on the lower triangle
        for (int i = wid; i < m; i += nw) {
            const T vi = v[i], wi = u[i];
            T* row = a + (size_t)(o + i) * (o + i + 1) / 2 + o;
            for (int j = lane; j <= i; j += 32) row[j] -= vi * u[j] + wi * v[j];
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            d[n - 2] = at(n - 2, n - 2);
            e[n - 2] = at(n - 1, n - 2);
        }
        d[n - 1] = at(n - 1, n - 1);
    }
}

// Register-resident variant for n <= 32 * NC (and n <= 16 * NR): the working matrix is
// distributed over 16 warps, element (i, j) held by warp i % 16 (slot i / 16) and lane
// j % 32 (slot j / 32).  Per Householder step: the owners of column k publish it through
// shared memory (barrier 1); every thread forms the reflector v from it; u = B v is
// reduced across the lanes of each warp with shuffles and published with g = v^T u
// (barrier 2); the rank-2 update B -= v w^T + w v^T, w = 2u - 2 g v, runs in registers.
// Entries in rows or columns <= k are dead: v and w are zero there.
template <int NR, int NC>
__device__ __forceinline__ void tridiag_reg_dev(const double* __restrict__ A, int n, float* __restrict__ d,
                                                float* __restrict__ e, float* __restrict__ refl) {
    constexpr int NW = 16;
    __shared__ float xv[2][NR * NW];   // column k below the diagonal, double-buffered by k
    __shared__ float uv[NR * NW];
    __shared__ float part[NW], part2[NW];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    float a[NR][NC];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int i = r * NW + w, j = c * 32 + lane;
            a[r][c] = (i < n && j < n) ? (float)A[(size_t)i * n + j] : 0.f;
        }
    for (int t = tid; t < n * n; t += blockDim.x) refl[t] = 0.f;
    for (int k = 0; k + 2 < n; ++k) {
        float* x = xv[k & 1];
        const int ck = k >> 5, lk = k & 31;
        if (lane == lk) {
            float ss = 0.f;
#pragma unroll
            for (int c = 0; c < NC; ++c)
                if (c == ck) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int i = r * NW + w;
                        const float val = a[r][c];
                        if (i > k && i < n) {
                            x[i] = val;
                            if (i > k + 1) ss += val * val;
                        }
                        if (i == k) d[k] = val;
                    }
                }
            part[w] = ss;
        }
        __syncthreads();
        float s1 = part[lane & (NW - 1)];
#pragma unroll
        for (int o = NW / 2; o; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        const float x0 = x[k + 1];
        if (s1 == 0.f) {                 // already reduced: no reflector (uniform branch)
            if (tid == 0) e[k] = x0;
            __syncthreads();
            continue;
        }
        const float nrm = sqrtf(x0 * x0 + s1);
        const float alpha = x0 >= 0.f ? -nrm : nrm;
        const float v0 = x0 - alpha;
        const float inv = 1.f / sqrtf(v0 * v0 + s1);
        auto vval = [&](int i) -> float { return (i <= k || i >= n) ? 0.f : (i == k + 1 ? v0 : x[i]) * inv; };
        if (tid == 0) e[k] = alpha;
        for (int i = k + 1 + tid; i < n; i += blockDim.x) refl[(size_t)k * n + i] = vval(i);
        float vc[NC], vr[NR];
#pragma unroll
        for (int c = 0; c < NC; ++c) vc[c] = vval(c * 32 + lane);
#pragma unroll
        for (int r = 0; r < NR; ++r) vr[r] = vval(r * NW + w);
        // rows with i <= k and column slots with every column <= k are dead: skipped
        // (the row test is uniform over a warp, the slot test over the whole block)
        float gp = 0.f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int i = r * NW + w;
            if (i > k && i < n) {
                float p = 0.f;
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (c * 32 + 31 > k) p += a[r][c] * vc[c];
                p = warp_sum(p);
                if (lane == 0) uv[i] = p;
                gp += p * vr[r];
            }
        }
        if (lane == 0) part2[w] = gp;
        __syncthreads();
        float g = part2[lane & (NW - 1)];
#pragma unroll
        for (int o = NW / 2; o; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        float wc[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int j = c * 32 + lane;
            wc[c] = (j > k && j < n) ? 2.f * uv[j] - 2.f * g * vc[c] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int i = r * NW + w;
            if (i > k && i < n) {
                const float wr = 2.f * uv[i] - 2.f * g * vr[r];
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (c * 32 + 31 > k) a[r][c] -= vr[r] * wc[c] + wr * vc[c];
            }
        }
    }
    // the last 2 x 2 block
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int i = r * NW + w, j = c * 32 + lane;
            if (i < n && j < n) {
                if (i == j && i >= n - 2) d[i] = a[r][c];
                if (i == n - 1 && j == n - 2) e[n - 2] = a[r][c];
            }
        }
}

template <int NR, int NC>
__global__ void __launch_bounds__(512) k_tridiag_reg(const double* __restrict__ A, int n, float* __restrict__ d,
                                                     float* __restrict__ e, float* __restrict__ refl) {
    tridiag_reg_dev<NR, NC>(A, n, d, e, refl);
}

struct tridiag_reg_rec {
    const double* A;
    int n;
    float* d;
    float* e;
    float* refl;
    int gx, gy, gz;
};

template <int NR, int NC>
__global__ void __launch_bounds__(512) k_tridiag_reg_b(const __grid_constant__ BPack<tridiag_reg_rec> p) {
    const tridiag_reg_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tridiag_reg_dev<NR, NC>(r.A, r.n, r.d, r.e, r.refl);
}


// Row-parallel variant for n <= 128 (512 threads): the working matrix B is in shared memory
// (FP32, row stride tr_ld(n) = 4 mod 32, so the 8 rows x 4 phases of a warp hit 32 distinct
// banks) and row i belongs to the four threads 4i..4i+3, which walk its
// columns j = k+1+t, k+5+t, ...  Per Householder step k only the active block (rows and
// columns > k) is touched, so the work shrinks as k grows:
//   A  the owner (t = 0) of row i > k reads B[i][k] (written by that same thread in the
//      previous update) and contributes its square; barrier 1;
//   B  every thread forms the reflector v = (x - alpha e_1) / |x - alpha e_1| from the
//      column and the sum of squares;
//   C  u_i = sum_j B[i][j] v_j (four partial sums, two shuffles) and g = v^T u; barrier 2;
//   D  B -= v w^T + w v^T with w = 2u - 2 g v, each thread its own row slice.
// Column k+1 of the next step and the diagonal entry d[k+1] are owned by the t = 0 thread of
// their row, which also wrote them in D, so no third barrier is needed; the column, the
// partial sums and u are double-buffered by k.
constexpr int TR_TPR = 4;
__host__ __device__ inline int tr_ld(int n) { return ((n + 31) / 32) * 32 + 4; }
__device__ __forceinline__ void tridiag_rows_dev(const double* __restrict__ A, int n, float* __restrict__ d,
                                                 float* __restrict__ e, float* __restrict__ refl) {
    extern __shared__ float trs[];                  // B: n x tr_ld(n)
    __shared__ float xs[2][128], us[2][128];
    __shared__ float part[2][16], part2[2][16];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int gi = tid / TR_TPR, t = tid % TR_TPR;  // row gi, column phase t
    const int ld = tr_ld(n);
    for (int q = tid; q < n * n; q += blockDim.x) {
        const int i = q / n, j = q % n;
        trs[i * ld + j] = (float)A[q];
    }
    for (int q = tid; q < n * n; q += blockDim.x) refl[q] = 0.f;
    __syncthreads();
    const bool rowok = gi < n;
    float* Bi = trs + (size_t)(rowok ? gi : 0) * ld;
    for (int k = 0; k + 2 < n; ++k) {
        const int kb = k & 1;
        // ---- A: column k below the diagonal, sum of squares below the subdiagonal ----
        float sq = 0.f;
        if (rowok && t == 0) {
            if (gi == k) d[k] = Bi[k];
            if (gi > k) {
                const float xv = Bi[k];
                xs[kb][gi] = xv;
                if (gi > k + 1) sq = xv * xv;
            }
        }
        sq = warp_sum(sq);
        if (lane == 0) part[kb][w] = sq;
        __syncthreads();
        float s1 = part[kb][lane & 15];      // lanes 16..31 mirror 0..15: every lane, same sum
#pragma unroll
        for (int o = 8; o; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        const float x0 = xs[kb][k + 1];
        if (s1 == 0.f) {                 // already reduced: no reflector (uniform)
            if (tid == 0) e[k] = x0;
            continue;
        }
        // ---- B: the reflector ----
        const float nrm = sqrtf(x0 * x0 + s1);
        const float alpha = x0 >= 0.f ? -nrm : nrm;
        const float v0 = x0 - alpha;
        const float inv = 1.f / sqrtf(v0 * v0 + s1);
        if (tid == 0) e[k] = alpha;
        const float* xk = xs[kb];
        auto vval = [&](int j) -> float { return (j == k + 1 ? v0 : xk[j]) * inv; };
        const bool act = rowok && gi > k;
        // ---- C: u = B v over the active block, g = v^T u ----
        float ui = 0.f;
        if (act)
            for (int j = k + 1 + t; j < n; j += TR_TPR) ui += Bi[j] * vval(j);
        ui += __shfl_xor_sync(0xffffffffu, ui, 1);
        ui += __shfl_xor_sync(0xffffffffu, ui, 2);
        const float vi = act ? vval(gi) : 0.f;
        if (act && t == 0) {
            us[kb][gi] = ui;
            refl[(size_t)k * n + gi] = vi;
        }
        float gp = (t == 0) ? vi * ui : 0.f;
        gp = warp_sum(gp);
        if (lane == 0) part2[kb][w] = gp;
        __syncthreads();
        float g = part2[kb][lane & 15];
#pragma unroll
        for (int o = 8; o; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        // ---- D: rank-2 update of this thread's row slice ----
        if (act) {
            const float wi = 2.f * ui - 2.f * g * vi;
            const float* uk = us[kb];
            for (int j = k + 1 + t; j < n; j += TR_TPR) {
                const float vj = vval(j);
                const float wj = 2.f * uk[j] - 2.f * g * vj;
                Bi[j] -= vi * wj + wi * vj;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (n >= 2) {
            d[n - 2] = trs[(n - 2) * ld + (n - 2)];
            e[n - 2] = trs[(n - 1) * ld + (n - 2)];
            d[n - 1] = trs[(n - 1) * ld + (n - 1)];
        } else {
            d[0] = trs[0];
        }
    }
}

__global__ void __launch_bounds__(512) k_tridiag_rows(const double* __restrict__ A, int n, float* __restrict__ d,
                                                      float* __restrict__ e, float* __restrict__ refl) {
    tridiag_rows_dev(A, n, d, e, refl);
}

struct tridiag_rows_rec {
    const double* A;
    int n;
    float* d;
    float* e;
    float* refl;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(512) k_tridiag_rows_b(const __grid_constant__ BPack<tridiag_rows_rec> p) {
    const tridiag_rows_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tridiag_rows_dev(r.A, r.n, r.d, r.e, r.refl);
}


}  // namespace

// number of eigenvalues of T (d, e) below x, FP32 Sturm sequence
__host__ __device__ int sturm_count(const float* d, const float* e2, int n, float x, float pivmin) {
    int c = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++c;
    for (int i = 1; i < n; ++i) {
#ifdef __CUDA_ARCH__
        q = (d[i] - x) - __fdividef(e2[i - 1], q);
#else
        q = (d[i] - x) - e2[i - 1] / q;
#endif
        if (fabsf(q) < pivmin) q = -pivmin;
        if (q < 0.f) ++c;
    }
    return c;
}

// j-th smallest eigenvalue of the normalised tridiagonal by bisection on [lo, hi] (FP32)
__host__ __device__ float bisect_one(const float* df, const float* e2f, int n, int j, float lo, float hi) {
    for (int it = 0; it < 64; ++it) {
        float mid = 0.5f * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(df, e2f, n, mid, 1e-30f) > j) hi = mid; else lo = mid;
    }
    return 0.5f * (lo + hi);
}

// Inverse iteration on T (d, e).  Each solve factorises T - mu I by Gaussian elimination
// with partial pivoting fused with the forward substitution, then back-substitutes.  The
// running rows live in registers; the factor rows (1/pivot, super, second super) and y are
// strided arrays (element i at [i * stride]).
//
// Seeded start vector of eigenvector k (entries in [0.75, 1.25]).
template <typename T>
__host__ __device__ void invit_start(int n, int k, T* y, int ystride) {
    uint32_t hsh = 2166136261u ^ ((uint32_t)k * 16777619u);
    for (int i = 0; i < n; ++i) {
        hsh = hsh * 1664525u + 1013904223u;
        y[i * ystride] = (T)1 + (T)0.5 * ((T)(hsh >> 8) * (T)(1.0 / 16777216.0) - (T)0.5);
    }
}

// FP64 reciprocal on a serial chain: an FP32 estimate refined by two Newton-Raphson steps
// y <- y (2 - a y) (each doubles the correct bits: 24 -> 48 -> 96), a short dependent chain
// instead of an FP64 division; IEEE division outside the FP32 exponent range (and on the host)
__host__ __device__ __forceinline__ double rcp64_nr(double a) {
#ifdef __CUDA_ARCH__
    const double m = fabs(a);
    if (!(m > 1e-30 && m < 1e30)) return 1.0 / a;
    double y = (double)__frcp_rn((float)a);
    y = y * (2.0 - a * y);
    y = y * (2.0 - a * y);
    return y;
#else
    return 1.0 / a;
#endif
}

// reciprocal on the serial elimination chain: the hardware reciprocal for FP32 (this
// stage only needs FP32 accuracy), the Newton-refined one for FP64
template <typename T> __host__ __device__ __forceinline__ T chain_rcp(T a) { return (T)1 / a; }
template <> __host__ __device__ __forceinline__ double chain_rcp<double>(double a) { return rcp64_nr(a); }
#ifdef __CUDA_ARCH__
template <> __device__ __forceinline__ float chain_rcp<float>(float a) { return __frcp_rn(a); }
#endif

// One inverse-iteration solve y <- (T - mu I)^{-1} y, unnormalised; returns |y|^2.
// When both pivot candidates of a step are below `tiny` (a decoupled block: T's off-diagonal
// is negligible there), the diagonal one is clamped to +-tiny instead of pivoting on the
// negligible off-diagonal entry, so no multiplier exceeds 1 and no reciprocal 1 / tiny.  If
// several clamped pivots in a row still overflow the sum of squares, y is rescaled by its
// largest entry (a power-of-two factor of it) and the sum taken again.
template <typename T>
__host__ __device__ T invit_solve(const T* d, const T* e, int n, T mu, T tiny, T* rdd, T* du, T* du2, T* y,
                                       int stride, int ystride) {
    T a = d[0] - mu, b = n > 1 ? e[0] : (T)0, yi = y[0];
    for (int i = 0; i + 1 < n; ++i) {
        const T c = e[i], dn = d[i + 1] - mu, f = (i + 2 < n) ? e[i + 1] : (T)0, yn = y[(i + 1) * ystride];
        if (fabs(a) >= fabs(c) || fabs(c) < tiny) {
            if (fabs(a) < tiny) a = a >= (T)0 ? tiny : -tiny;
            const T r = chain_rcp(a), m = c * r;
            rdd[i * stride] = r; du[i * stride] = b; du2[i * stride] = 0; y[i * ystride] = yi;
            a = dn - m * b; b = f; yi = yn - m * yi;
        } else {
            const T r = chain_rcp(c), m = a * r;
            rdd[i * stride] = r; du[i * stride] = dn; du2[i * stride] = f; y[i * ystride] = yn;
            a = b - m * dn; b = -m * f; yi = yi - m * yn;
        }
    }
    if (fabs(a) < tiny) a = a >= (T)0 ? tiny : -tiny;
    T y1 = yi / a, y2 = 0;
    y[(n - 1) * ystride] = y1;
    T ss = y1 * y1;
    for (int i = n - 2; i >= 0; --i) {
        const T vv = (y[i * ystride] - du[i * stride] * y1 - du2[i * stride] * y2) * rdd[i * stride];
        y[i * ystride] = vv;
        ss += vv * vv;
        y2 = y1;
        y1 = vv;
    }
    const T big = sizeof(T) == 8 ? (T)1e300 : (T)1e36;
    if (!(ss <= big)) {
        T m = 0;
        for (int i = 0; i < n; ++i) m = fmax(m, fabs(y[i * ystride]));
        int ex = 0;
        frexp(m, &ex);
        const T sc = ldexp((T)1, -ex);   // exact power-of-two scaling: |y| <= 1 afterwards
        ss = 0;
        for (int i = 0; i < n; ++i) {
            const T v = y[i * ystride] * sc;
            y[i * ystride] = v;
            ss += v * v;
        }
    }
    return ss;
}

// Eigenvector of T for the eigenvalue nearest `mu` (optionally with Rayleigh-quotient shift
// updates); returns the final shift.
template <typename T>
__host__ __device__ T invit_one(const T* d, const T* e, int n, T mu, T tnorm, int k, T* rdd, T* du, T* du2, T* y,
                                int stride, int sweeps, int rq_update, int ystride) {
    const T eps = sizeof(T) == 8 ? (T)1.1102230246251565e-16 : (T)5.9604645e-08f;
    const T tiny = eps * tnorm + (T)(sizeof(T) == 8 ? 1e-300 : 1e-37);
    invit_start<T>(n, k, y, ystride);
    for (int it = 0; it < sweeps; ++it) {
        const T ss = invit_solve<T>(d, e, n, mu, tiny, rdd, du, du2, y, stride, ystride);
        const T sc = (T)1 / sqrt(ss);
        if (!rq_update) {
            for (int i = 0; i < n; ++i) y[i * ystride] *= sc;
            continue;
        }
        T num = 0, prev = 0, cur = y[0] * sc;
        for (int i = 0; i < n; ++i) {
            const T next = (i + 1 < n) ? y[(i + 1) * ystride] * sc : (T)0;
            y[i * ystride] = cur;
            T ti = d[i] * cur;
            if (i > 0) ti += e[i - 1] * prev;
            if (i + 1 < n) ti += e[i] * next;
            num += cur * ti;
            prev = cur;
            cur = next;
        }
        if (rq_update) mu = num;
    }
    return mu;
}
template double invit_one<double>(const double*, const double*, int, double, double, int, double*, double*, double*,
                                  double*, int, int, int, int);
template float invit_one<float>(const float*, const float*, int, float, float, int, float*, float*, float*, float*,
                                int, int, int, int);

namespace {

// Leading `nwant` eigenpairs of T (d, e):
//   k_tri_vec   bisection (FP32 Sturm counts) for the shifts + fixed-shift inverse iteration,
//               one thread per eigenvalue;
//   k_tri_runs  runs of tied shifts (consecutive shifts closer than TIE_EPS FP32 ulps of |T|:
//               a multiple eigenvalue or one FP32 cannot split): equal shifts give equal
//               factorisations, and inverse iteration then drives every start vector of the run
//               to the same direction.  The members after the first are computed in order, each
//               iterate re-orthogonalised (classical Gram-Schmidt, twice) against the earlier
//               members of its run, as in LAPACK's xSTEIN;
//   k_tri_orth  one Cholesky QR of the n x nwant eigenvector block (mixes vectors inside
//               clusters only: vectors of separated eigenvalues are already orthogonal);
//   k_tri_rq    Rayleigh quotients as eigenvalues.
// Y is n x nwant with leading dimension ld = nwant + 1 (odd: conflict-free row access).
constexpr float TIE_EPS = 4.f;
constexpr float EPS32 = 5.9604645e-08f;

__device__ __forceinline__ bool tied(const float* shift, int k) {
    return k > 0 && fabsf(shift[k] - shift[k - 1]) <= TIE_EPS * EPS32;
}

// Long runs (more than RUN_SERIAL members tied in FP32) get FP64 eigenvalues (k_run_shift64)
// and FP64 inverse-iteration vectors (k_run_vec64), member by member in parallel; only members
// still tied in FP64 (|mu_k - mu_{k-1}| <= TIE64 eps64 |T|: a numerically multiple eigenvalue)
// are left to the serial run kernel.  mu64[k] is NaN outside long runs.
// The FP64 eigenvalues are resolved to RES64 |T| (enough for inverse iteration: shifts a
// thousand times closer than the eigenvalue gaps they must separate); members whose values
// agree within twice that are tied in FP64.
constexpr int RUN_SERIAL = 8;
constexpr double RES64 = 1e-12;
constexpr double EPS64 = 1.1102230246251565e-16;
__device__ __forceinline__ bool tied64(double a, double b, double tn) { return fabs(a - b) <= 2.0 * RES64 * tn; }
__device__ __forceinline__ bool tied2(const float* shift, const double* mu64, double tn, int k) {
    if (!tied(shift, k)) return false;
    if (!mu64) return true;
    const double a = mu64[k], b = mu64[k - 1];
    if (isnan(a) || isnan(b)) return true;
    return tied64(a, b, tn);
}

template <typename T>
__device__ T tri_norm(const T* d, const T* e, int n) {
    T t = 0;
    for (int i = 0; i < n; ++i)
        t = fmax(t, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : (T)0) + (i + 1 < n ? fabs(e[i]) : (T)0));
    return t > (T)0 ? t : (T)1;
}

// shifts (normalised by |T|) of the nwant largest eigenvalues by multisection: one warp per
// eigenvalue, each round splits the bracketing interval at 32 points (one FP32 Sturm count
// per lane) and keeps the sub-interval where the count crosses the eigenvalue's index.
constexpr int SHIFT_WARPS = 8;
template <typename T>
__device__ __forceinline__ void tri_shift_dev(const T* __restrict__ d, const T* __restrict__ e,
                                              int n, int nwant, float* __restrict__ shift_out, int bx) {
    __shared__ float df[256], e2f[256];
    __shared__ float bounds[2];
    __shared__ T tn_sh;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) tn_sh = tri_norm(d, e, n);
    __syncthreads();
    const double sc = 1.0 / (double)tn_sh;     // on T / |T| (FP32 range)
    for (int i = tid; i < n; i += blockDim.x) {
        df[i] = (float)((double)d[i] * sc);
        e2f[i] = i + 1 < n ? (float)(((double)e[i] * sc) * ((double)e[i] * sc)) : 0.f;
    }
    __syncthreads();
    if (tid == 0) {
        float lo = 3.4e38f, hi = -3.4e38f;
        for (int i = 0; i < n; ++i) {
            float r = (i > 0 ? sqrtf(e2f[i - 1]) : 0.f) + (i + 1 < n ? sqrtf(e2f[i]) : 0.f);
            lo = fminf(lo, df[i] - r);
            hi = fmaxf(hi, df[i] + r);
        }
        bounds[0] = lo - 1e-5f;
        bounds[1] = hi + 1e-5f;
    }
    __syncthreads();
    const int k = bx * SHIFT_WARPS + (tid >> 5);
    if (k >= nwant) return;
    const int j = n - 1 - k;                    // index from below
    float lo = bounds[0], hi = bounds[1];
    for (int round = 0; round < 12; ++round) {
        const float h = (hi - lo) * (1.f / 33.f);
        const float p = lo + h * (float)(lane + 1);
        const unsigned above = __ballot_sync(0xffffffffu, p > lo && p < hi && sturm_count(df, e2f, n, p, 1e-30f) > j);
        const int first = above ? __ffs(above) - 1 : 32;
        const float nlo = first == 0 ? lo : lo + h * (float)first;
        const float nhi = first == 32 ? hi : lo + h * (float)(first + 1);
        if (!(nhi - nlo < hi - lo)) break;      // the interval no longer shrinks in FP32
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) shift_out[k] = 0.5f * (lo + hi);
}

template <typename T>
__global__ void __launch_bounds__(32 * SHIFT_WARPS) k_tri_shift(const T* __restrict__ d, const T* __restrict__ e,
                                                                int n, int nwant, float* __restrict__ shift_out) {
    tri_shift_dev<T>(d, e, n, nwant, shift_out, (int)blockIdx.x);
}

template <typename T>
struct tri_shift_rec {
    const T* d;
    const T* e;
    int n;
    int nwant;
    float* shift_out;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(32 * SHIFT_WARPS) k_tri_shift_b(const __grid_constant__ BPack<tri_shift_rec<T>> p) {
    const tri_shift_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tri_shift_dev<T>(r.d, r.e, r.n, r.nwant, r.shift_out, bx);
}


// fixed-shift inverse iteration (3 solves) for every eigenvalue that does not continue a run
template <typename T>
__device__ __forceinline__ void tri_vec_dev(const T* __restrict__ d, const T* __restrict__ e, int n, int nwant,
                                            const float* __restrict__ shift, T* __restrict__ Y, int bx) {
    __shared__ T tn_sh;
    const int tid = threadIdx.x;
    if (tid == 0) tn_sh = tri_norm(d, e, n);
    __syncthreads();
    const T tnorm = tn_sh;
    const int ld = nwant + 1;
    const int k = bx * blockDim.x + tid;
    if (k >= nwant || tied(shift, k)) return;
    // elimination rows of this thread in shared memory ([i][thread], conflict-free)
    extern __shared__ __align__(16) unsigned char vsm_raw[];
    T* rdd = reinterpret_cast<T*>(vsm_raw);
    T* du = rdd + (size_t)n * blockDim.x;
    T* du2 = du + (size_t)n * blockDim.x;
    // the bisection value itself: an offset that grows with k would move the shifts of a
    // dense cluster onto neighbouring eigenvalues
    const T mu = (T)shift[k] * tnorm;
    invit_one<T>(d, e, n, mu, tnorm, k, rdd + tid, du + tid, du2 + tid, Y + k, (int)blockDim.x, 3, 0, ld);
}

template <typename T>
__global__ void __launch_bounds__(64) k_tri_vec(const T* __restrict__ d, const T* __restrict__ e, int n, int nwant,
                                                const float* __restrict__ shift, T* __restrict__ Y) {
    tri_vec_dev<T>(d, e, n, nwant, shift, Y, (int)blockIdx.x);
}

template <typename T>
struct tri_vec_rec {
    const T* d;
    const T* e;
    int n;
    int nwant;
    const float* shift;
    T* Y;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(64) k_tri_vec_b(const __grid_constant__ BPack<tri_vec_rec<T>> p) {
    const tri_vec_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tri_vec_dev<T>(r.d, r.e, r.n, r.nwant, r.shift, r.Y, bx);
}


// One CTA per run of tied shifts starting at column blockIdx.x (CTAs whose column does not
// start a run with at least one follower return at once).  y lives in shared memory; the
// serial tridiagonal solve runs on thread 0.
template <typename T>
__device__ __forceinline__ void tri_runs_dev(const T* __restrict__ d, const T* __restrict__ e, int n,
                                             int nwant, const float* __restrict__ shift,
                                             const double* __restrict__ mu64, T* __restrict__ Y, int bx) {
    const int L = bx;
    __shared__ T tn0;
    if (threadIdx.x == 0) tn0 = tri_norm(d, e, n);
    __syncthreads();
    const double tnd = (double)tn0;
    if (L >= nwant || tied2(shift, mu64, tnd, L) || L + 1 >= nwant || !tied2(shift, mu64, tnd, L + 1)) return;
    int end = L + 1;
    while (end < nwant && tied2(shift, mu64, tnd, end)) ++end;   // members L .. end-1
    __shared__ T y[256], c[256], rdd[256], du[256], du2[256];
    __shared__ T red[33];
    __shared__ T tn_sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ld = nwant + 1;
    if (tid == 0) tn_sh = tri_norm(d, e, n);
    __syncthreads();
    const T tnorm = tn_sh;
    const T tiny = (T)EPS32 * tnorm + (T)1e-37;
    // y -= Y[:, L..k-1] (Y[:, L..k-1]^T y), twice, then y /= |y|
    auto cgs2 = [&](int k) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int j = L + tid; j < k; j += nt) {
                T acc = 0;
                for (int i = 0; i < n; ++i) acc += Y[(size_t)i * ld + j] * y[i];
                c[j - L] = acc;
            }
            __syncthreads();
            for (int i = tid; i < n; i += nt) {
                T acc = y[i];
                for (int j = L; j < k; ++j) acc -= c[j - L] * Y[(size_t)i * ld + j];
                y[i] = acc;
            }
            __syncthreads();
        }
        T ss = 0;
        for (int i = tid; i < n; i += nt) ss += y[i] * y[i];
        ss = block_sum(ss, red);
        const T sc = ss > (T)0 ? (T)1 / sqrt(ss) : (T)0;
        for (int i = tid; i < n; i += nt) y[i] *= sc;
        __syncthreads();
    };
    for (int k = L + 1; k < end; ++k) {
        if (tid == 0) invit_start<T>(n, k, y, 1);
        __syncthreads();
        const T mu = (mu64 && !isnan(mu64[k])) ? (T)mu64[k] : (T)shift[k] * tnorm;
        for (int sweep = 0; sweep < 3; ++sweep) {
            cgs2(k);
            if (tid == 0) invit_solve<T>(d, e, n, mu, tiny, rdd, du, du2, y, 1, 1);
            __syncthreads();
        }
        cgs2(k);
        for (int i = tid; i < n; i += nt) Y[(size_t)i * ld + k] = y[i];
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_tri_runs(const T* __restrict__ d, const T* __restrict__ e, int n,
                                                  int nwant, const float* __restrict__ shift,
                                                  const double* __restrict__ mu64, T* __restrict__ Y) {
    tri_runs_dev<T>(d, e, n, nwant, shift, mu64, Y, (int)blockIdx.x);
}

template <typename T>
struct tri_runs_rec {
    const T* d;
    const T* e;
    int n;
    int nwant;
    const float* shift;
    const double* mu64;
    T* Y;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(256) k_tri_runs_b(const __grid_constant__ BPack<tri_runs_rec<T>> p) {
    const tri_runs_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tri_runs_dev<T>(r.d, r.e, r.n, r.nwant, r.shift, r.mu64, r.Y, bx);
}


__device__ int sturm_count64(const double* d, const double* e2, int n, double x, double pivmin) {
    int c = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++c;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] * rcp64_nr(q);
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++c;
    }
    return c;
}

// one warp per CTA: every lane of a member's warp runs an FP64 chain, and GB300 issues two
// FP64 operations per clock per SM, so members are spread over as many SMs as possible
constexpr int R64_WARPS = 1;

// FP64 eigenvalue of every member of a long run: one warp per member, multisection (32 FP64
// Sturm counts per round) from the run's FP32 bracket widened by 16 FP32 ulps of |T| (the
// Gershgorin interval when the counts do not bracket the index), down to RES64 |T|.
template <typename T>
__device__ __forceinline__ void run_shift64_dev(const T* __restrict__ d, const T* __restrict__ e,
                                                int n, int nwant, const float* __restrict__ shift,
                                                double* __restrict__ mu64, int bx) {
    __shared__ double d64[256], e2[256];
    __shared__ double tn_sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < n; i += blockDim.x) {
        d64[i] = (double)d[i];
        e2[i] = i + 1 < n ? (double)e[i] * (double)e[i] : 0.0;
    }
    if (tid == 0) tn_sh = (double)tri_norm(d, e, n);
    __syncthreads();
    const int k = bx * R64_WARPS + w;
    if (k >= nwant) return;
    int L = k, end = k + 1;
    while (L > 0 && tied(shift, L)) --L;
    while (end < nwant && tied(shift, end)) ++end;
    if (end - L <= RUN_SERIAL) {
        if (lane == 0) mu64[k] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const double tn = tn_sh;
    const double pivmin = 1e-300 + EPS64 * EPS64 * tn;
    const int idx = n - 1 - k;                                     // index from below
    double lo = (double)shift[end - 1] * tn - 16.0 * (double)EPS32 * tn;
    double hi = (double)shift[L] * tn + 16.0 * (double)EPS32 * tn;
    const int clo = lane == 0 ? sturm_count64(d64, e2, n, lo, pivmin) : 0;
    const int chi = lane == 1 ? sturm_count64(d64, e2, n, hi, pivmin) : 0;
    const int c0 = __shfl_sync(0xffffffffu, clo, 0), c1 = __shfl_sync(0xffffffffu, chi, 1);
    if (!(c0 <= idx && c1 > idx)) {
        lo = -1.001 * tn;
        hi = 1.001 * tn;
    }
    for (int round = 0; round < 24; ++round) {
        const double h = (hi - lo) * (1.0 / 33.0);
        const double pt = lo + h * (double)(lane + 1);
        const unsigned above = __ballot_sync(0xffffffffu, sturm_count64(d64, e2, n, pt, pivmin) > idx);
        const int first = above ? __ffs(above) - 1 : 32;
        const double nlo = first == 0 ? lo : lo + h * (double)first;
        const double nhi = first == 32 ? hi : lo + h * (double)(first + 1);
        if (!(nhi - nlo < hi - lo)) break;
        lo = nlo;
        hi = nhi;
        if (hi - lo <= RES64 * tn) break;
    }
    if (lane == 0) mu64[k] = 0.5 * (lo + hi);
}

template <typename T>
__global__ void __launch_bounds__(32 * R64_WARPS) k_run_shift64(const T* __restrict__ d, const T* __restrict__ e,
                                                               int n, int nwant, const float* __restrict__ shift,
                                                               double* __restrict__ mu64) {
    run_shift64_dev<T>(d, e, n, nwant, shift, mu64, (int)blockIdx.x);
}

template <typename T>
struct run_shift64_rec {
    const T* d;
    const T* e;
    int n;
    int nwant;
    const float* shift;
    double* mu64;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(32 * R64_WARPS) k_run_shift64_b(const __grid_constant__ BPack<run_shift64_rec<T>> p) {
    const run_shift64_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    run_shift64_dev<T>(r.d, r.e, r.n, r.nwant, r.shift, r.mu64, bx);
}


// FP64 inverse iteration (three solves) for the long-run members that are not tied in FP64
// to their predecessor; lane 0 of the member's warp runs the serial solve, the vector is
// stored back in the working precision.  Factor rows and the iterate live in shared memory.
template <typename T>
__device__ __forceinline__ void run_vec64_dev(const T* __restrict__ d, const T* __restrict__ e, int n,
                                              int nwant, const double* __restrict__ mu64,
                                              T* __restrict__ Y, int bx) {
    extern __shared__ __align__(16) unsigned char rv_raw[];
    __shared__ double d64[256], e64[256];
    __shared__ double tn_sh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < n; i += blockDim.x) {
        d64[i] = (double)d[i];
        e64[i] = i + 1 < n ? (double)e[i] : 0.0;
    }
    if (tid == 0) tn_sh = (double)tri_norm(d, e, n);
    __syncthreads();
    const int k = bx * R64_WARPS + w;
    if (k >= nwant) return;
    const double mu = mu64[k];
    if (isnan(mu)) return;
    const double tn = tn_sh;
    if (k > 0 && !isnan(mu64[k - 1]) && tied64(mu, mu64[k - 1], tn)) return;
    double* base = reinterpret_cast<double*>(rv_raw) + (size_t)w * 4 * n;
    double *rdd = base, *du = base + n, *du2 = base + 2 * n, *y = base + 3 * n;
    if (lane == 0) invit_one<double>(d64, e64, n, mu, tn, k, rdd, du, du2, y, 1, 3, 0, 1);
    __syncwarp();
    const int ld = nwant + 1;
    for (int i = lane; i < n; i += 32) Y[(size_t)i * ld + k] = (T)y[i];
}

template <typename T>
__global__ void __launch_bounds__(32 * R64_WARPS) k_run_vec64(const T* __restrict__ d, const T* __restrict__ e, int n,
                                                             int nwant, const double* __restrict__ mu64,
                                                             T* __restrict__ Y) {
    run_vec64_dev<T>(d, e, n, nwant, mu64, Y, (int)blockIdx.x);
}

template <typename T>
struct run_vec64_rec {
    const T* d;
    const T* e;
    int n;
    int nwant;
    const double* mu64;
    T* Y;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(32 * R64_WARPS) k_run_vec64_b(const __grid_constant__ BPack<run_vec64_rec<T>> p) {
    const run_vec64_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    run_vec64_dev<T>(r.d, r.e, r.n, r.nwant, r.mu64, r.Y, bx);
}


// Orthonormalise the inverse-iteration vectors by one Cholesky QR of the whole block
// (FP32): fixed-shift inverse iteration leaves the vectors of a cluster of (near-)equal
// eigenvalues independent but not orthogonal, and the noise part of Z forms large clusters
// at FP32 resolution.  Vectors of separated eigenvalues are already orthogonal, so the
// triangular mixing acts inside clusters only.  The Gram matrix and the row update use the
// whole CTA; the factorisation and the triangular inverse run on warp 0 with warp-level
// synchronisation only.  Y (n x nwant, ld nwant+1) is processed in shared memory.
template <typename T>
__device__ __forceinline__ void tri_orth_dev(T* __restrict__ Yg, int n, int nwant, T* __restrict__ scratch,
                                             int use_smem) {
    extern __shared__ __align__(16) unsigned char osm_raw[];
    const int tid = threadIdx.x;
    const int ld = nwant + 1;
    T* ys = use_smem ? reinterpret_cast<T*>(osm_raw) : scratch;   // n x ld
    T* Gm = ys + (size_t)n * ld;                         // nwant x ld (R in the upper triangle)
    T* Ri = Gm + (size_t)nwant * ld;                     // nwant: 1 / R_kk
    for (int t = tid; t < n * ld; t += blockDim.x) ys[t] = Yg[t];
    __syncthreads();
    // G = Y^T Y, upper triangle, 4 x 4 register tiles
    const int nt4 = (nwant + 3) / 4;
    for (int t = tid; t < nt4 * nt4; t += blockDim.x) {
        const int pb = (t / nt4) * 4, qb = (t % nt4) * 4;
        if (qb + 3 < pb) continue;
        T acc[4][4] = {};
        for (int i = 0; i < n; ++i) {
            const T* yi = ys + (size_t)i * ld;
            T yp[4], yq[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                yp[u] = pb + u < nwant ? yi[pb + u] : (T)0;
                yq[u] = qb + u < nwant ? yi[qb + u] : (T)0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v2 = 0; v2 < 4; ++v2) acc[u][v2] += yp[u] * yq[v2];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v2 = 0; v2 < 4; ++v2) {
                const int pp = pb + u, qq = qb + v2;
                if (pp < nwant && qq < nwant && qq >= pp) Gm[pp * ld + qq] = acc[u][v2];
            }
    }
    __syncthreads();
    // right-looking Cholesky on the upper triangle, one barrier per step: each thread takes
    // the pivot itself; the trailing update (warp per row, lanes over columns) uses the
    // unscaled row k; rows are scaled to R after the loop.  Ri[k] keeps 1 / R_kk.
    const int lane = tid & 31, wid = tid >> 5, nwp = blockDim.x >> 5;
    // the columns are unit vectors: a pivot below 1e-6 marks a (numerically) dependent
    // column, which is left unscaled instead of being blown up to inf
    for (int k = 0; k < nwant; ++k) {
        const T dk = Gm[k * ld + k];
        const T ri = dk > (T)1e-6 ? (T)1 / sqrt(dk) : (T)1;
        if (tid == 0) Ri[k] = ri;
        const T r2 = ri * ri;
        for (int i = k + 1 + wid; i < nwant; i += nwp) {
            const T gki = Gm[k * ld + i] * r2;
            for (int j = i + lane; j < nwant; j += 32) Gm[i * ld + j] -= gki * Gm[k * ld + j];
        }
        __syncthreads();
    }
    for (int t = tid; t < nwant * nwant; t += blockDim.x) {
        const int p = t / nwant, q = t % nwant;
        if (q >= p) Gm[p * ld + q] *= Ri[p];
    }
    __syncthreads();
    // rows of Y: solve y_new R = y by forward substitution (one thread per row)
    for (int i = tid; i < n; i += blockDim.x) {
        T* yi = ys + (size_t)i * ld;
        for (int q = 0; q < nwant; ++q) {
            T a0 = yi[q], a1 = 0;
            int p = 0;
            for (; p + 1 < q; p += 2) {
                a0 -= yi[p] * Gm[p * ld + q];
                a1 -= yi[p + 1] * Gm[(p + 1) * ld + q];
            }
            for (; p < q; ++p) a0 -= yi[p] * Gm[p * ld + q];
            yi[q] = (a0 + a1) * Ri[q];
        }
    }
    __syncthreads();
    for (int t = tid; t < n * ld; t += blockDim.x) Yg[t] = ys[t];
}

template <typename T>
__global__ void __launch_bounds__(256) k_tri_orth(T* __restrict__ Yg, int n, int nwant, T* __restrict__ scratch,
                                                  int use_smem) {
    tri_orth_dev<T>(Yg, n, nwant, scratch, use_smem);
}

template <typename T>
struct tri_orth_rec {
    T* Yg;
    int n;
    int nwant;
    T* scratch;
    int use_smem;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(256) k_tri_orth_b(const __grid_constant__ BPack<tri_orth_rec<T>> p) {
    const tri_orth_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tri_orth_dev<T>(r.Yg, r.n, r.nwant, r.scratch, r.use_smem);
}


// Variant of k_tri_orth for n whose working set does not fit in shared memory: Y stays in
// global memory (L2-resident, at most 257 KB) and is updated in place, staged through
// shared memory 64 rows at a time for the Gram matrix; R lives in shared memory as the packed
// upper triangle (row p from column p: n (n + 1) / 2 floats, 128 KB for n = 256).  Same
// Gram tiles, Cholesky with the same pivot guard, and row solves.
constexpr int ORTH_CH = 64;   // rows of Y staged per pass of the Gram accumulation
template <typename T>
__device__ __forceinline__ void tri_orth_packed_dev(T* __restrict__ Yg, int n, int nwant) {
    extern __shared__ __align__(16) unsigned char op_raw[];
    T* Gp = reinterpret_cast<T*>(op_raw);
    T* Ri = Gp + (size_t)nwant * (nwant + 1) / 2;
    T* Yc = Ri + nwant;                                    // ORTH_CH x ld staged rows of Y
    auto G = [&](int p, int q) -> T& { return Gp[(size_t)p * nwant - (size_t)p * (p - 1) / 2 + (q - p)]; };
    const int tid = threadIdx.x;
    const int ld = nwant + 1;
    T* ys = Yg;
    for (int t = tid; t < nwant * (nwant + 1) / 2; t += blockDim.x) Gp[t] = (T)0;
    // G = Y^T Y over chunks of ORTH_CH rows staged in shared memory; each thread adds its own
    // 4 x 4 tiles' partial sums into G, so no two threads touch the same entry
    const int nt4 = (nwant + 3) / 4;
    for (int r0 = 0; r0 < n; r0 += ORTH_CH) {
        const int rows = n - r0 < ORTH_CH ? n - r0 : ORTH_CH;
        __syncthreads();
        for (int t = tid; t < rows * ld; t += blockDim.x) Yc[t] = ys[(size_t)r0 * ld + t];
        __syncthreads();
        for (int t = tid; t < nt4 * nt4; t += blockDim.x) {
            const int pb = (t / nt4) * 4, qb = (t % nt4) * 4;
            if (qb + 3 < pb) continue;
            T acc[4][4] = {};
            for (int i = 0; i < rows; ++i) {
                const T* yi = Yc + (size_t)i * ld;
                T yp[4], yq[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    yp[u] = pb + u < nwant ? yi[pb + u] : (T)0;
                    yq[u] = qb + u < nwant ? yi[qb + u] : (T)0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v2 = 0; v2 < 4; ++v2) acc[u][v2] += yp[u] * yq[v2];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v2 = 0; v2 < 4; ++v2) {
                    const int pp = pb + u, qq = qb + v2;
                    if (pp < nwant && qq < nwant && qq >= pp) G(pp, qq) += acc[u][v2];
                }
        }
    }
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5, nwp = blockDim.x >> 5;
    for (int k = 0; k < nwant; ++k) {
        const T dk = G(k, k);
        const T ri = dk > (T)1e-6 ? (T)1 / sqrt(dk) : (T)1;
        if (tid == 0) Ri[k] = ri;
        const T r2 = ri * ri;
        for (int i = k + 1 + wid; i < nwant; i += nwp) {
            const T gki = G(k, i) * r2;
            for (int j = i + lane; j < nwant; j += 32) G(i, j) -= gki * G(k, j);
        }
        __syncthreads();
    }
    for (int t = tid; t < nwant * nwant; t += blockDim.x) {
        const int p = t / nwant, q = t % nwant;
        if (q >= p) G(p, q) *= Ri[p];
    }
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        T* yi = ys + (size_t)i * ld;
        for (int q = 0; q < nwant; ++q) {
            T a0 = yi[q], a1 = 0;
            int p = 0;
            for (; p + 1 < q; p += 2) {
                a0 -= yi[p] * G(p, q);
                a1 -= yi[p + 1] * G(p + 1, q);
            }
            for (; p < q; ++p) a0 -= yi[p] * G(p, q);
            yi[q] = (a0 + a1) * Ri[q];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_tri_orth_packed(T* __restrict__ Yg, int n, int nwant) {
    tri_orth_packed_dev<T>(Yg, n, nwant);
}

template <typename T>
struct tri_orth_packed_rec {
    T* Yg;
    int n;
    int nwant;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(256) k_tri_orth_packed_b(const __grid_constant__ BPack<tri_orth_packed_rec<T>> p) {
    const tri_orth_packed_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tri_orth_packed_dev<T>(r.Yg, r.n, r.nwant);
}


// Cholesky QR of the eigenvector block for n <= 32 * NC (n <= 16 * NR), 512 threads.
// Y (n x n, ld n+1) is staged in shared memory; G = Y^T Y is accumulated into the same
// register distribution as k_tridiag_reg; the right-looking Cholesky publishes row k
// (double-buffered, one barrier per step) and keeps R in shared memory; then each row of
// Y is solved against R by four threads (partial sums over p = sub mod 4, two shuffles per
// column).  Same pivot guard as k_tri_orth: a pivot <= 1e-6 (the columns are unit
// vectors) leaves its column unscaled.
template <int NR, int NC>
__device__ __forceinline__ void tri_orth_reg_dev(float* __restrict__ Yg, int n) {
    constexpr int NW = 16;
    extern __shared__ __align__(16) unsigned char or_raw[];
    const int ld = n + 1;
    float* ys = reinterpret_cast<float*>(or_raw);        // n x ld
    float* Rm = ys + (size_t)n * ld;                       // n x ld, upper triangle of R
    float* ri_s = Rm + (size_t)n * ld;                     // n: multiplier of column q
    __shared__ float rowbuf[2][NC * 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int t = tid; t < n * ld; t += blockDim.x) ys[t] = Yg[t];
    __syncthreads();
    float G[NR][NC];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) G[r][c] = 0.f;
    for (int l = 0; l < n; ++l) {
        const float* yl = ys + (size_t)l * ld;
        float yi[NR], yj[NC];
#pragma unroll
        for (int r = 0; r < NR; ++r) { const int i = r * NW + w; yi[r] = i < n ? yl[i] : 0.f; }
#pragma unroll
        for (int c = 0; c < NC; ++c) { const int j = c * 32 + lane; yj[c] = j < n ? yl[j] : 0.f; }
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int c = 0; c < NC; ++c) G[r][c] += yi[r] * yj[c];
    }
    for (int k = 0; k < n; ++k) {
        float* rb = rowbuf[k & 1];
        if (w == k % NW) {
            const int rk = k / NW;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float val = 0.f;
#pragma unroll
                for (int r = 0; r < NR; ++r) val = (r == rk) ? G[r][c] : val;
                rb[c * 32 + lane] = val;
            }
        }
        __syncthreads();
        const float dk = rb[k];
        const float ri = dk > 1e-6f ? 1.f / sqrtf(dk) : 1.f;
        const float r2 = ri * ri;
        for (int j = k + tid; j < n; j += blockDim.x) Rm[(size_t)k * ld + j] = rb[j] * ri;
        if (tid == 0) ri_s[k] = ri;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int i = r * NW + w;
            if (i > k && i < n) {
                const float gi = rb[i] * r2;
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int j = c * 32 + lane;
                    if (c * 32 + 31 > k && j > k) G[r][c] -= gi * rb[j];
                }
            }
        }
    }
    __syncthreads();
    // rows of Y: y_new R = y, four threads per row.  The row loop runs to a multiple of
    // 8 rows so that every lane of a warp takes part in the shuffles; lanes past row n-1
    // contribute zeros and write nothing.
    const int sub = tid & 3;
    const int n8 = (n + 7) & ~7;
    for (int i = tid >> 2; i < n8; i += blockDim.x >> 2) {
        const bool act = i < n;
        float* yi = ys + (size_t)(act ? i : 0) * ld;
        for (int q = 0; q < n; ++q) {
            float acc = 0.f;
            if (act)
                for (int p = sub; p < q; p += 4) acc += yi[p] * Rm[(size_t)p * ld + q];
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            const float v = act ? (yi[q] - acc) * ri_s[q] : 0.f;
            __syncwarp();
            if (act && (q & 3) == sub) yi[q] = v;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int t = tid; t < n * ld; t += blockDim.x) Yg[t] = ys[t];
}

template <int NR, int NC>
__global__ void __launch_bounds__(512) k_tri_orth_reg(float* __restrict__ Yg, int n) {
    tri_orth_reg_dev<NR, NC>(Yg, n);
}

struct tri_orth_reg_rec {
    float* Yg;
    int n;
    int gx, gy, gz;
};

template <int NR, int NC>
__global__ void __launch_bounds__(512) k_tri_orth_reg_b(const __grid_constant__ BPack<tri_orth_reg_rec> p) {
    const tri_orth_reg_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tri_orth_reg_dev<NR, NC>(r.Yg, r.n);
}


template <typename T>
__device__ __forceinline__ void tri_rq_dev(const T* __restrict__ d, const T* __restrict__ e, int n, int nwant,
                                           const T* __restrict__ Y, T* __restrict__ w, int bx) {
    const int k = bx * blockDim.x + threadIdx.x;
    if (k >= nwant) return;
    const int ld = nwant + 1;
    T num = 0;
    for (int i = 0; i < n; ++i) {
        T ti = d[i] * Y[(size_t)i * ld + k];
        if (i > 0) ti += e[i - 1] * Y[(size_t)(i - 1) * ld + k];
        if (i + 1 < n) ti += e[i] * Y[(size_t)(i + 1) * ld + k];
        num += Y[(size_t)i * ld + k] * ti;
    }
    w[k] = num;
}

template <typename T>
__global__ void k_tri_rq(const T* __restrict__ d, const T* __restrict__ e, int n, int nwant,
                         const T* __restrict__ Y, T* __restrict__ w) {
    tri_rq_dev<T>(d, e, n, nwant, Y, w, (int)blockIdx.x);
}

template <typename T>
struct tri_rq_rec {
    const T* d;
    const T* e;
    int n;
    int nwant;
    const T* Y;
    T* w;
    int gx, gy, gz;
};

template <typename T>
__global__ void k_tri_rq_b(const __grid_constant__ BPack<tri_rq_rec<T>> p) {
    const tri_rq_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    tri_rq_dev<T>(r.d, r.e, r.n, r.nwant, r.Y, r.w, bx);
}


// z = H_0 H_1 ... H_{n-3} y for eigenvector column k, one warp per eigenvector (z held in
// registers, 8 entries per lane); output widened to FP64 (ld ldv).  BT_WARPS eigenvectors
// per CTA; the reflectors are staged once per CTA in shared memory when they fit
// (use_smem), otherwise read from global memory.
constexpr int BT_WARPS = 16;
template <typename T>
__device__ __forceinline__ void backtransform_dev(const T* __restrict__ refl, int n, int nwant,
                                                  const T* __restrict__ Y, double* __restrict__ V,
                                                  int ldv, int use_smem, int bx) {
    extern __shared__ __align__(16) unsigned char bt_raw[];
    const T* rf = refl;
    if (use_smem) {
        T* s = reinterpret_cast<T*>(bt_raw);
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) s[t] = refl[t];
        __syncthreads();
        rf = s;
    }
    const int lane = threadIdx.x & 31;
    const int k = bx * BT_WARPS + (threadIdx.x >> 5);
    if (k >= nwant) return;
    T z[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int i = lane + 32 * t;
        z[t] = i < n ? Y[(size_t)i * (nwant + 1) + k] : (T)0;
    }
    for (int j = n - 3; j >= 0; --j) {
        const T* vj = rf + (size_t)j * n;
        T vr[8];
        T dot = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int i = lane + 32 * t;
            vr[t] = (i > j && i < n) ? vj[i] : (T)0;
            dot += vr[t] * z[t];
        }
        dot = warp_sum(dot);
#pragma unroll
        for (int t = 0; t < 8; ++t) z[t] -= (T)2 * dot * vr[t];
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int i = lane + 32 * t;
        if (i < n) V[(size_t)i * ldv + k] = (double)z[t];
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * BT_WARPS) k_backtransform(const T* __restrict__ refl, int n, int nwant,
                                                                 const T* __restrict__ Y, double* __restrict__ V,
                                                                 int ldv, int use_smem) {
    backtransform_dev<T>(refl, n, nwant, Y, V, ldv, use_smem, (int)blockIdx.x);
}

template <typename T>
struct backtransform_rec {
    const T* refl;
    int n;
    int nwant;
    const T* Y;
    double* V;
    int ldv;
    int use_smem;
    int gx, gy, gz;
};

template <typename T>
__global__ void __launch_bounds__(32 * BT_WARPS) k_backtransform_b(const __grid_constant__ BPack<backtransform_rec<T>> p) {
    const backtransform_rec<T>& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    backtransform_dev<T>(r.refl, r.n, r.nwant, r.Y, r.V, r.ldv, r.use_smem, bx);
}


// Ogita-Aishima correction for the leading R columns: E (n x R), refined eigenvalues lam1.
// G = X^T X1, S = X^T Z X1 (n x R each), lam_all: approximate eigenvalues of every column.
__device__ __forceinline__ void oa_update_dev(const double* __restrict__ G, const double* __restrict__ S,
                                              const double* __restrict__ lam_all, int n, int R, double* __restrict__ E,
                                              double* __restrict__ lam1) {
    __shared__ double lt[256];
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        const double rjj = 1.0 - G[(size_t)j * R + j];
        lt[j] = S[(size_t)j * R + j] / (1.0 - rjj);
    }
    __syncthreads();
    // pairs closer than 16 FP32 ulps of |lambda|_max are a cluster in every sweep: the FP32
    // stage does not resolve them, and a Newton step across such a gap amplifies its error
    const double gap_floor = 1e-6 * fmax(fabs(lam_all[0]), fabs(lam_all[n - 1]));
    for (int t = threadIdx.x; t < n * R; t += blockDim.x) {
        const int i = t / R, j = t % R;
        const double rij = (i == j ? 1.0 : 0.0) - G[t];
        double eij = 0.5 * rij;
        if (i != j) {
            const double li = i < R ? lt[i] : lam_all[i];
            const double num = S[t] + lt[j] * rij, den = lt[j] - li;
            // Newton correction only while the coupling is small against the gap
            if (fabs(den) > gap_floor && fabs(num) <= 0.1 * fabs(den)) eij = num / den;
        }
        E[t] = eij;
    }
    for (int j = threadIdx.x; j < R; j += blockDim.x) lam1[j] = lt[j];
}

__global__ void k_oa_update(const double* __restrict__ G, const double* __restrict__ S,
                            const double* __restrict__ lam_all, int n, int R, double* __restrict__ E,
                            double* __restrict__ lam1) {
    oa_update_dev(G, S, lam_all, n, R, E, lam1);
}

struct oa_update_rec {
    const double* G;
    const double* S;
    const double* lam_all;
    int n;
    int R;
    double* E;
    double* lam1;
    int gx, gy, gz;
};

__global__ void k_oa_update_b(const __grid_constant__ BPack<oa_update_rec> p) {
    const oa_update_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    oa_update_dev(r.G, r.S, r.lam_all, r.n, r.R, r.E, r.lam1);
}


// descending order of the R refined pairs: w[rank] = lam[j], V[:, rank] = X1[:, j]
__device__ __forceinline__ void sort_top_dev(const double* __restrict__ lam, const double* __restrict__ X1, int n, int ldx, int R,
                                             double* __restrict__ w, double* __restrict__ V) {
    __shared__ int rank_of[256];
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        int r = 0;
        for (int t = 0; t < R; ++t) r += (lam[t] > lam[j] || (lam[t] == lam[j] && t < j)) ? 1 : 0;
        rank_of[j] = r;
        w[r] = lam[j];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * R; t += blockDim.x) {
        const int i = t / R, j = t % R;
        V[(size_t)i * R + rank_of[j]] = X1[(size_t)i * ldx + j];
    }
}

__global__ void k_sort_top(const double* __restrict__ lam, const double* __restrict__ X1, int n, int ldx, int R,
                           double* __restrict__ w, double* __restrict__ V) {
    sort_top_dev(lam, X1, n, ldx, R, w, V);
}

struct sort_top_rec {
    const double* lam;
    const double* X1;
    int n;
    int ldx;
    int R;
    double* w;
    double* V;
    int gx, gy, gz;
};

__global__ void k_sort_top_b(const __grid_constant__ BPack<sort_top_rec> p) {
    const sort_top_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    sort_top_dev(r.lam, r.X1, r.n, r.ldx, r.R, r.w, r.V);
}


// M = (3 I - G) / 2: one second-order step towards orthonormal columns (X1 <- X1 M)
__device__ __forceinline__ void halfstep_dev(const double* __restrict__ G, int R, double* __restrict__ M, int bx) {
    int t = bx * blockDim.x + threadIdx.x;
    if (t >= R * R) return;
    M[t] = ((t / R == t % R) ? 1.5 : 0.0) - 0.5 * G[t];
}

__global__ void k_halfstep(const double* __restrict__ G, int R, double* __restrict__ M) {
    halfstep_dev(G, R, M, (int)blockIdx.x);
}

struct halfstep_rec {
    const double* G;
    int R;
    double* M;
    int gx, gy, gz;
};

__global__ void k_halfstep_b(const __grid_constant__ BPack<halfstep_rec> p) {
    const halfstep_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    halfstep_dev(r.G, r.R, r.M, bx);
}


__device__ __forceinline__ void f32_to_f64_dev(const float* __restrict__ s, double* __restrict__ d, int n, int bx) {
    int e = bx * blockDim.x + threadIdx.x;
    if (e < n) d[e] = (double)s[e];
}

__global__ void k_f32_to_f64(const float* __restrict__ s, double* __restrict__ d, int n) {
    f32_to_f64_dev(s, d, n, (int)blockIdx.x);
}

struct f32_to_f64_rec {
    const float* s;
    double* d;
    int n;
    int gx, gy, gz;
};

__global__ void k_f32_to_f64_b(const __grid_constant__ BPack<f32_to_f64_rec> p) {
    const f32_to_f64_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    f32_to_f64_dev(r.s, r.d, r.n, bx);
}


__device__ __forceinline__ void copy_cols_dev(const double* __restrict__ src, int lds, double* __restrict__ dst, int ldd, int n,
                                              int R, int bx) {
    int t = bx * blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    dst[(size_t)(t / R) * ldd + t % R] = src[(size_t)(t / R) * lds + t % R];
}

__global__ void k_copy_cols(const double* __restrict__ src, int lds, double* __restrict__ dst, int ldd, int n,
                            int R) {
    copy_cols_dev(src, lds, dst, ldd, n, R, (int)blockIdx.x);
}

struct copy_cols_rec {
    const double* src;
    int lds;
    double* dst;
    int ldd;
    int n;
    int R;
    int gx, gy, gz;
};

__global__ void k_copy_cols_b(const __grid_constant__ BPack<copy_cols_rec> p) {
    const copy_cols_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    copy_cols_dev(r.src, r.lds, r.dst, r.ldd, r.n, r.R, bx);
}


struct EigLayout {
    float *work, *refl, *d, *e, *lam, *shift, *Yt, *iiw;
    double *X, *ZX1, *G, *S, *E, *T1, *lam_all, *lam1, *mu64, *part;
    size_t doubles;
};

EigLayout eig_layout(double* base, int n) {
    EigLayout L{};
    const size_t nn = (size_t)n * n;
    size_t off = 0;   // in doubles
    auto fl = [&](size_t count) {
        float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
        off += (count + 1) / 2 + 32;
        return p;
    };
    auto db = [&](size_t count) {
        double* p = base ? base + off : nullptr;
        off += count + 32;
        return p;
    };
    L.work = fl(nn);
    L.refl = fl(nn);
    L.d = fl(n);
    L.e = fl(n);
    L.lam = fl(n);
    L.shift = fl(n);
    L.Yt = fl((size_t)n * (n + 1));
    L.iiw = fl(2 * (size_t)n + 4 * (size_t)n * (n + 1) + 2 * nn + (size_t)n);
    L.X = db(nn);
    L.ZX1 = db(nn);
    L.G = db(nn);
    L.S = db(nn);
    L.E = db(nn);
    L.T1 = db(nn);
    L.lam_all = db(n);
    L.lam1 = db(n);
    L.mu64 = db(n);
    L.part = db(gemm_part_doubles(n, n, n));
    L.doubles = off + 64;
    return L;
}

}  // namespace

size_t syev_scratch_doubles(int n) { return eig_layout(nullptr, n).doubles; }

// w: nwant eigenvalues (descending); V: n x nwant row-major eigenvectors
rbki_status syev_top_cuda(const double* A, int n, int nwant, double* w, double* V, double* scratch,
                          cudaStream_t st) {
    if (n > 256 || nwant > n || nwant < 1) return set_error(RBKI_E_UNSUPPORTED, "syev: n > 256");
    const EigLayout L = eig_layout(scratch, n);
    const size_t nn = (size_t)n * n;
    // ---- 1. FP32 eigendecomposition ----
    if (n <= 128) {
        static const size_t rmax = max_dyn_smem(k_tridiag_rows);   // thread-safe, once
        const size_t rsm_t = (size_t)n * tr_ld(n) * sizeof(float);
        if (rsm_t > rmax) return set_error(RBKI_E_CUDA, "syev: tridiagonalisation shared memory");
        k_tridiag_rows<<<1, 512, rsm_t, st>>>(A, n, L.d, L.e, L.refl);
    } else if (n <= 192) {
        k_tridiag_reg<12, 6><<<1, 512, 0, st>>>(A, n, L.d, L.e, L.refl);
    } else {
        static const size_t tmax = max_dyn_smem(k_tridiag<float>);          // thread-safe, once
        static const size_t pmax = max_dyn_smem(k_tridiag_packed<float>);
        const size_t tsm = (size_t)(n + 1) * n * sizeof(float);
        const size_t psm = (size_t)n * (n + 1) / 2 * sizeof(float);
        if (tsm <= tmax)
            k_tridiag<float><<<1, 512, tsm, st>>>(A, n, L.work, 1, L.d, L.e, L.refl);
        else if (psm <= pmax)
            k_tridiag_packed<float><<<1, 512, psm, st>>>(A, n, L.d, L.e, L.refl);
        else
            k_tridiag<float><<<1, 512, 0, st>>>(A, n, L.work, 0, L.d, L.e, L.refl);
    }
    RBKI_LAUNCH_CHECK("k_tridiag");
    static const size_t vmax = max_dyn_smem(k_tri_vec<float>);
    const int vthr = 32;
    const size_t vsm = 3 * (size_t)n * vthr * sizeof(float);
    if (vsm > vmax) return set_error(RBKI_E_UNSUPPORTED, "syev: inverse-iteration rows exceed shared memory");
    k_tri_shift<float><<<(unsigned)cdiv(n, SHIFT_WARPS), 32 * SHIFT_WARPS, 0, st>>>(L.d, L.e, n, n, L.shift);
    RBKI_LAUNCH_CHECK("k_tri_shift");
    k_tri_vec<float><<<(unsigned)cdiv(n, vthr), vthr, vsm, st>>>(L.d, L.e, n, n, L.shift, L.Yt);
    RBKI_LAUNCH_CHECK("k_tri_vec");
    k_run_shift64<float><<<(unsigned)cdiv(n, R64_WARPS), 32 * R64_WARPS, 0, st>>>(L.d, L.e, n, n, L.shift, L.mu64);
    RBKI_LAUNCH_CHECK("k_run_shift64");
    {
        static const size_t rvmax = max_dyn_smem(k_run_vec64<float>);
        const size_t rvsm = (size_t)R64_WARPS * 4 * n * sizeof(double);
        if (rvsm > rvmax) return set_error(RBKI_E_UNSUPPORTED, "syev: FP64 run vectors exceed shared memory");
        k_run_vec64<float><<<(unsigned)cdiv(n, R64_WARPS), 32 * R64_WARPS, rvsm, st>>>(L.d, L.e, n, n, L.mu64, L.Yt);
        RBKI_LAUNCH_CHECK("k_run_vec64");
    }
    k_tri_runs<float><<<(unsigned)n, 256, 0, st>>>(L.d, L.e, n, n, L.shift, L.mu64, L.Yt);
    RBKI_LAUNCH_CHECK("k_tri_runs");
    const size_t rsm = (2 * (size_t)n * (n + 1) + n) * sizeof(float);
    if (n <= 128) {
        // opt-in to large dynamic shared memory once per variant (thread-safe statics)
        if (n <= 32) {
            static const size_t r0 = max_dyn_smem(k_tri_orth_reg<2, 1>);
            (void)r0;
            k_tri_orth_reg<2, 1><<<1, 512, rsm, st>>>(L.Yt, n);
        } else if (n <= 64) {
            static const size_t r1 = max_dyn_smem(k_tri_orth_reg<4, 2>);
            (void)r1;
            k_tri_orth_reg<4, 2><<<1, 512, rsm, st>>>(L.Yt, n);
        } else {
            static const size_t r2 = max_dyn_smem(k_tri_orth_reg<8, 4>);
            (void)r2;
            k_tri_orth_reg<8, 4><<<1, 512, rsm, st>>>(L.Yt, n);
        }
    } else {
        static const size_t omax = max_dyn_smem(k_tri_orth<float>);
        static const size_t opmax = max_dyn_smem(k_tri_orth_packed<float>);
        const size_t osm = (size_t)(n + 2 * n) * (n + 1) * sizeof(float);
        const size_t opsm = ((size_t)n * (n + 1) / 2 + n + (size_t)ORTH_CH * (n + 1)) * sizeof(float);
        if (osm <= omax)
            k_tri_orth<float><<<1, 256, osm, st>>>(L.Yt, n, n, L.iiw, 1);
        else if (opsm <= opmax)
            k_tri_orth_packed<float><<<1, 256, opsm, st>>>(L.Yt, n, n);
        else
            k_tri_orth<float><<<1, 256, 0, st>>>(L.Yt, n, n, L.iiw, 0);
    }
    RBKI_LAUNCH_CHECK("k_tri_orth");
    k_tri_rq<float><<<(unsigned)cdiv(n, 64), 64, 0, st>>>(L.d, L.e, n, n, L.Yt, L.lam);
    RBKI_LAUNCH_CHECK("k_tri_rq");
    static const size_t bmax = max_dyn_smem(k_backtransform<float>);
    const size_t bsm = (size_t)n * n * sizeof(float);
    const int b_smem = bsm <= bmax;
    k_backtransform<float><<<(unsigned)cdiv(n, BT_WARPS), 32 * BT_WARPS, b_smem ? bsm : 0, st>>>(
        L.refl, n, n, L.Yt, L.X, n, b_smem);
    RBKI_LAUNCH_CHECK("k_backtransform");
    k_f32_to_f64<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(L.lam, L.lam_all, n);
    RBKI_LAUNCH_CHECK("k_f32_to_f64");
    // ---- 2. FP64 refinement of the leading nwant columns ----
    const int R = nwant;
    const int sweeps = R == n ? 5 : 2;
    for (int it = 0; it < sweeps; ++it) {
        RBKI_TRY(gemm_f64_cuda(false, n, R, n, A, n, L.X, n, L.ZX1, R, 0.0, L.part, st));   // Z X1
        RBKI_TRY(gemm_f64_cuda(true, n, R, n, L.X, n, L.ZX1, R, L.S, R, 0.0, L.part, st));  // X^T Z X1
        RBKI_TRY(gemm_f64_cuda(true, n, R, n, L.X, n, L.X, n, L.G, R, 0.0, L.part, st));    // X^T X1
        k_oa_update<<<1, 256, 0, st>>>(L.G, L.S, L.lam_all, n, R, L.E, L.lam1);
        RBKI_LAUNCH_CHECK("k_oa_update");
        // X1 <- X1 + X E  (into T1, then back over the first R columns)
        k_copy_cols<<<(unsigned)cdiv((int64_t)n * R, 256), 256, 0, st>>>(L.X, n, L.T1, R, n, R);
        RBKI_LAUNCH_CHECK("k_copy_cols");
        RBKI_TRY(gemm_f64_cuda(false, n, R, n, L.X, n, L.E, R, L.T1, R, 1.0, L.part, st));
        k_copy_cols<<<(unsigned)cdiv((int64_t)n * R, 256), 256, 0, st>>>(L.T1, R, L.X, n, n, R);
        RBKI_LAUNCH_CHECK("k_copy_cols");
        RBKI_TRY(copy_f64_cuda(L.lam1, L.lam_all, R, st));
    }
    // X1 <- X1 (3I - X1^T X1) / 2 (orthonormal to second order)
    RBKI_TRY(gemm_f64_cuda(true, R, R, n, L.X, n, L.X, n, L.G, R, 0.0, L.part, st));
    k_halfstep<<<(unsigned)cdiv((int64_t)R * R, 256), 256, 0, st>>>(L.G, R, L.S);
    RBKI_LAUNCH_CHECK("k_halfstep");
    RBKI_TRY(gemm_f64_cuda(false, n, R, R, L.X, n, L.S, R, L.T1, R, 0.0, L.part, st));
    k_copy_cols<<<(unsigned)cdiv((int64_t)n * R, 256), 256, 0, st>>>(L.T1, R, L.X, n, n, R);
    RBKI_LAUNCH_CHECK("k_copy_cols");
    k_sort_top<<<1, 256, 0, st>>>(L.lam1, L.X, n, n, R, w, V);
    RBKI_LAUNCH_CHECK("k_sort_top");
    return RBKI_OK;
}

rbki_status syev_cuda(const double* A, int n, double* w, double* V, double* scratch, cudaStream_t st) {
    return syev_top_cuda(A, n, n, w, V, scratch, st);
}

}  // namespace rbki

// ---- batched form: the same stages for many independent matrices, one launch per stage and
// variant (items take exactly the kernels and shared-memory choices of syev_top_cuda) ----
namespace rbki {

rbki_status syev_top_batched(const EigItem* it, int cnt, cudaStream_t st) {
    if (cnt <= 0) return RBKI_OK;
    std::vector<EigLayout> L(cnt);
    int nmax = 0;
    for (int k = 0; k < cnt; ++k) {
        const int n = it[k].n, nw = it[k].nwant;
        if (n > 192 || nw > n || nw < 1) return set_error(RBKI_E_UNSUPPORTED, "batched syev: n > 192");
        L[k] = eig_layout(it[k].scratch, n);
        nmax = std::max(nmax, n);
    }
    // ---- 1. FP32 eigendecomposition ----
    {
        std::vector<tridiag_rows_rec> rows;
        std::vector<tridiag_reg_rec> reg;
        size_t rsm = 0;
        for (int k = 0; k < cnt; ++k) {
            const int n = it[k].n;
            if (n <= 128) {
                rows.push_back(tridiag_rows_rec{it[k].A, n, L[k].d, L[k].e, L[k].refl, 1, 1, 1});
                rsm = std::max(rsm, (size_t)n * tr_ld(n) * sizeof(float));
            } else {
                reg.push_back(tridiag_reg_rec{it[k].A, n, L[k].d, L[k].e, L[k].refl, 1, 1, 1});
            }
        }
        static const size_t rmax = max_dyn_smem(k_tridiag_rows_b);
        if (rsm > rmax) return set_error(RBKI_E_CUDA, "syev: tridiagonalisation shared memory");
        RBKI_TRY(bat_launch(k_tridiag_rows_b, rows.data(), (int)rows.size(), 512, rsm, st, "k_tridiag_rows_b"));
        RBKI_TRY(bat_launch(k_tridiag_reg_b<12, 6>, reg.data(), (int)reg.size(), 512, 0, st, "k_tridiag_reg_b"));
    }
    {
        const int vthr = 32;
        static const size_t vmax = max_dyn_smem(k_tri_vec_b<float>);
        static const size_t rvmax = max_dyn_smem(k_run_vec64_b<float>);
        const size_t vsm = 3 * (size_t)nmax * vthr * sizeof(float);
        const size_t rvsm = (size_t)R64_WARPS * 4 * nmax * sizeof(double);
        if (vsm > vmax || rvsm > rvmax) return set_error(RBKI_E_UNSUPPORTED, "syev: inverse-iteration rows exceed shared memory");
        std::vector<tri_shift_rec<float>> sh(cnt);
        std::vector<tri_vec_rec<float>> vc(cnt);
        std::vector<run_shift64_rec<float>> rs(cnt);
        std::vector<run_vec64_rec<float>> rv(cnt);
        std::vector<tri_runs_rec<float>> ru(cnt);
        for (int k = 0; k < cnt; ++k) {
            const int n = it[k].n;
            const EigLayout& l = L[k];
            sh[k] = tri_shift_rec<float>{l.d, l.e, n, n, l.shift, (int)cdiv(n, SHIFT_WARPS), 1, 1};
            vc[k] = tri_vec_rec<float>{l.d, l.e, n, n, l.shift, l.Yt, (int)cdiv(n, vthr), 1, 1};
            rs[k] = run_shift64_rec<float>{l.d, l.e, n, n, l.shift, l.mu64, (int)cdiv(n, R64_WARPS), 1, 1};
            rv[k] = run_vec64_rec<float>{l.d, l.e, n, n, l.mu64, l.Yt, (int)cdiv(n, R64_WARPS), 1, 1};
            ru[k] = tri_runs_rec<float>{l.d, l.e, n, n, l.shift, l.mu64, l.Yt, n, 1, 1};
        }
        RBKI_TRY(bat_launch(k_tri_shift_b<float>, sh.data(), cnt, 32 * SHIFT_WARPS, 0, st, "k_tri_shift_b"));
        RBKI_TRY(bat_launch(k_tri_vec_b<float>, vc.data(), cnt, vthr, vsm, st, "k_tri_vec_b"));
        RBKI_TRY(bat_launch(k_run_shift64_b<float>, rs.data(), cnt, 32 * R64_WARPS, 0, st, "k_run_shift64_b"));
        RBKI_TRY(bat_launch(k_run_vec64_b<float>, rv.data(), cnt, 32 * R64_WARPS, rvsm, st, "k_run_vec64_b"));
        RBKI_TRY(bat_launch(k_tri_runs_b<float>, ru.data(), cnt, 256, 0, st, "k_tri_runs_b"));
    }
    {
        // Cholesky QR of the inverse-iteration vectors: the variant of syev_top_cuda per item
        std::vector<tri_orth_reg_rec> o1, o2, o3;
        std::vector<tri_orth_rec<float>> og0, og1;
        std::vector<tri_orth_packed_rec<float>> op;
        size_t s1 = 0, s2 = 0, s3 = 0, sg1 = 0, spk = 0;
        static const size_t r0 = max_dyn_smem(k_tri_orth_reg_b<2, 1>);
        static const size_t r1 = max_dyn_smem(k_tri_orth_reg_b<4, 2>);
        static const size_t r2 = max_dyn_smem(k_tri_orth_reg_b<8, 4>);
        static const size_t omax = max_dyn_smem(k_tri_orth_b<float>);
        static const size_t opmax = max_dyn_smem(k_tri_orth_packed_b<float>);
        for (int k = 0; k < cnt; ++k) {
            const int n = it[k].n;
            const size_t rsm = (2 * (size_t)n * (n + 1) + n) * sizeof(float);
            if (n <= 32) {
                o1.push_back(tri_orth_reg_rec{L[k].Yt, n, 1, 1, 1});
                s1 = std::max(s1, rsm);
            } else if (n <= 64) {
                o2.push_back(tri_orth_reg_rec{L[k].Yt, n, 1, 1, 1});
                s2 = std::max(s2, rsm);
            } else if (n <= 128) {
                o3.push_back(tri_orth_reg_rec{L[k].Yt, n, 1, 1, 1});
                s3 = std::max(s3, rsm);
            } else {
                const size_t osm = (size_t)(n + 2 * n) * (n + 1) * sizeof(float);
                const size_t opsm = ((size_t)n * (n + 1) / 2 + n + (size_t)ORTH_CH * (n + 1)) * sizeof(float);
                if (osm <= omax) {
                    og1.push_back(tri_orth_rec<float>{L[k].Yt, n, n, L[k].iiw, 1, 1, 1, 1});
                    sg1 = std::max(sg1, osm);
                } else if (opsm <= opmax) {
                    op.push_back(tri_orth_packed_rec<float>{L[k].Yt, n, n, 1, 1, 1});
                    spk = std::max(spk, opsm);
                } else {
                    og0.push_back(tri_orth_rec<float>{L[k].Yt, n, n, L[k].iiw, 0, 1, 1, 1});
                }
            }
        }
        if (s1 > r0 || s2 > r1 || s3 > r2) return set_error(RBKI_E_CUDA, "syev: orthonormalisation shared memory");
        RBKI_TRY(bat_launch(k_tri_orth_reg_b<2, 1>, o1.data(), (int)o1.size(), 512, s1, st, "k_tri_orth_reg_b"));
        RBKI_TRY(bat_launch(k_tri_orth_reg_b<4, 2>, o2.data(), (int)o2.size(), 512, s2, st, "k_tri_orth_reg_b"));
        RBKI_TRY(bat_launch(k_tri_orth_reg_b<8, 4>, o3.data(), (int)o3.size(), 512, s3, st, "k_tri_orth_reg_b"));
        RBKI_TRY(bat_launch(k_tri_orth_b<float>, og1.data(), (int)og1.size(), 256, sg1, st, "k_tri_orth_b"));
        RBKI_TRY(bat_launch(k_tri_orth_packed_b<float>, op.data(), (int)op.size(), 256, spk, st,
                            "k_tri_orth_packed_b"));
        RBKI_TRY(bat_launch(k_tri_orth_b<float>, og0.data(), (int)og0.size(), 256, 0, st, "k_tri_orth_b"));
    }
    {
        static const size_t bmax = max_dyn_smem(k_backtransform_b<float>);
        std::vector<tri_rq_rec<float>> rq(cnt);
        std::vector<backtransform_rec<float>> bs, bg;
        std::vector<f32_to_f64_rec> cv(cnt);
        size_t bsm_max = 0;
        for (int k = 0; k < cnt; ++k) {
            const int n = it[k].n;
            const EigLayout& l = L[k];
            rq[k] = tri_rq_rec<float>{l.d, l.e, n, n, l.Yt, l.lam, (int)cdiv(n, 64), 1, 1};
            const size_t bsm = (size_t)n * n * sizeof(float);
            const int b_smem = bsm <= bmax;
            (b_smem ? bs : bg).push_back(backtransform_rec<float>{l.refl, n, n, l.Yt, l.X, n, b_smem,
                                                                   (int)cdiv(n, BT_WARPS), 1, 1});
            if (b_smem) bsm_max = std::max(bsm_max, bsm);
            cv[k] = f32_to_f64_rec{l.lam, l.lam_all, n, (int)cdiv(n, 256), 1, 1};
        }
        RBKI_TRY(bat_launch(k_tri_rq_b<float>, rq.data(), cnt, 64, 0, st, "k_tri_rq_b"));
        RBKI_TRY(bat_launch(k_backtransform_b<float>, bs.data(), (int)bs.size(), 32 * BT_WARPS, bsm_max, st,
                            "k_backtransform_b"));
        RBKI_TRY(bat_launch(k_backtransform_b<float>, bg.data(), (int)bg.size(), 32 * BT_WARPS, 0, st,
                            "k_backtransform_b"));
        RBKI_TRY(bat_launch(k_f32_to_f64_b, cv.data(), cnt, 256, 0, st, "k_f32_to_f64_b"));
    }
    // ---- 2. FP64 refinement of the leading nwant columns (sweeps per item as in syev_top_cuda) ----
    int max_sweeps = 0;
    for (int k = 0; k < cnt; ++k) max_sweeps = std::max(max_sweeps, it[k].nwant == it[k].n ? 5 : 2);
    std::vector<GemmItem> g;
    std::vector<oa_update_rec> ou;
    std::vector<copy_cols_rec> c1, c2;
    std::vector<CopyItem> cl;
    for (int sw = 0; sw < max_sweeps; ++sw) {
        std::vector<int> act;
        for (int k = 0; k < cnt; ++k)
            if (sw < (it[k].nwant == it[k].n ? 5 : 2)) act.push_back(k);
        const int na = (int)act.size();
        auto gemms = [&](auto make) -> rbki_status {
            g.clear();
            for (int k : act) g.push_back(make(k));
            return gemm_f64_batched(g.data(), na, st);
        };
        RBKI_TRY(gemms([&](int k) {   // Z X1
            const int n = it[k].n, R = it[k].nwant;
            return GemmItem{false, n, R, n, it[k].A, n, L[k].X, n, L[k].ZX1, R, 0.0, L[k].part};
        }));
        RBKI_TRY(gemms([&](int k) {   // X^T Z X1
            const int n = it[k].n, R = it[k].nwant;
            return GemmItem{true, n, R, n, L[k].X, n, L[k].ZX1, R, L[k].S, R, 0.0, L[k].part};
        }));
        RBKI_TRY(gemms([&](int k) {   // X^T X1
            const int n = it[k].n, R = it[k].nwant;
            return GemmItem{true, n, R, n, L[k].X, n, L[k].X, n, L[k].G, R, 0.0, L[k].part};
        }));
        ou.clear();
        c1.clear();
        c2.clear();
        cl.clear();
        for (int k : act) {
            const int n = it[k].n, R = it[k].nwant;
            const EigLayout& l = L[k];
            ou.push_back(oa_update_rec{l.G, l.S, l.lam_all, n, R, l.E, l.lam1, 1, 1, 1});
            const int gc = (int)cdiv((int64_t)n * R, 256);
            c1.push_back(copy_cols_rec{l.X, n, l.T1, R, n, R, gc, 1, 1});
            c2.push_back(copy_cols_rec{l.T1, R, l.X, n, n, R, gc, 1, 1});
            cl.push_back(CopyItem{l.lam1, l.lam_all, R});
        }
        RBKI_TRY(bat_launch(k_oa_update_b, ou.data(), na, 256, 0, st, "k_oa_update_b"));
        RBKI_TRY(bat_launch(k_copy_cols_b, c1.data(), na, 256, 0, st, "k_copy_cols_b"));
        RBKI_TRY(gemms([&](int k) {   // X1 + X E
            const int n = it[k].n, R = it[k].nwant;
            return GemmItem{false, n, R, n, L[k].X, n, L[k].E, R, L[k].T1, R, 1.0, L[k].part};
        }));
        RBKI_TRY(bat_launch(k_copy_cols_b, c2.data(), na, 256, 0, st, "k_copy_cols_b"));
        RBKI_TRY(copy_f64_batched(cl.data(), na, st));
    }
    // X1 <- X1 (3I - X1^T X1) / 2
    g.clear();
    for (int k = 0; k < cnt; ++k) {
        const int n = it[k].n, R = it[k].nwant;
        g.push_back(GemmItem{true, R, R, n, L[k].X, n, L[k].X, n, L[k].G, R, 0.0, L[k].part});
    }
    RBKI_TRY(gemm_f64_batched(g.data(), cnt, st));
    std::vector<halfstep_rec> hs(cnt);
    std::vector<copy_cols_rec> cb(cnt);
    std::vector<sort_top_rec> so(cnt);
    g.clear();
    for (int k = 0; k < cnt; ++k) {
        const int n = it[k].n, R = it[k].nwant;
        const EigLayout& l = L[k];
        hs[k] = halfstep_rec{l.G, R, l.S, (int)cdiv((int64_t)R * R, 256), 1, 1};
        g.push_back(GemmItem{false, n, R, R, l.X, n, l.S, R, l.T1, R, 0.0, l.part});
        cb[k] = copy_cols_rec{l.T1, R, l.X, n, n, R, (int)cdiv((int64_t)n * R, 256), 1, 1};
        so[k] = sort_top_rec{l.lam1, l.X, n, n, R, it[k].w, it[k].V, 1, 1, 1};
    }
    RBKI_TRY(bat_launch(k_halfstep_b, hs.data(), cnt, 256, 0, st, "k_halfstep_b"));
    RBKI_TRY(gemm_f64_batched(g.data(), cnt, st));
    RBKI_TRY(bat_launch(k_copy_cols_b, cb.data(), cnt, 256, 0, st, "k_copy_cols_b"));
    return bat_launch(k_sort_top_b, so.data(), cnt, 256, 0, st, "k_sort_top_b");
}

}  // namespace rbki
