// Symmetric eigensolver for Algorithm 2 step 4 (Z = Q^T X X^T Q, b x b, b <= 256), FP64
// results for the leading `nwant` eigenpairs.  GB300 executes FP64 FMAs at 1/58 of the
// FP32 rate, so the solver keeps FP64 arithmetic to the O(b^3) reduction that needs it and
// spreads the rest:
//   1. Householder tridiagonalisation in FP64 (Householder 1958; the symmetric rank-2
//      update form used by LAPACK's xSYTD2), one CTA, lower triangle updated and mirrored.
//   2. Bisection with Sturm counts on the tridiagonal in FP32 (Givens 1954 / Wilkinson) for
//      the wanted eigenvalues - only as shifts.
//   3. Inverse iteration in FP64 on the tridiagonal (Gaussian elimination with partial
//      pivoting), FP64 Rayleigh quotients for the eigenvalues, then classical Gram-Schmidt
//      (twice) inside clusters of close eigenvalues.
//   4. Back-transformation by the stored reflectors, one CTA per eigenvector.
#include "kernels.h"

namespace rbki {
namespace {

__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Tridiagonalise A (n x n, symmetric): d[n], e[n-1]; reflector k (unit vector acting on
// rows k+1..n-1, zero if none) stored as row k of `refl` (refl[k*n + k+1+i]).  The working
// matrix lives in shared memory with an odd leading dimension (n+1) when it fits, otherwise
// in `work` (global, L2 resident).
__global__ void __launch_bounds__(512) k_tridiag(const double* __restrict__ A, int n,
                                                 double* __restrict__ work, int use_smem,
                                                 double* __restrict__ d, double* __restrict__ e,
                                                 double* __restrict__ refl) {
    extern __shared__ double sm[];
    const int ld = use_smem ? n + 1 : n;
    double* a = use_smem ? sm : work;
    __shared__ double v[256], u[256];
    __shared__ double red[33];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int t = tid; t < n * n; t += nt) a[(t / n) * ld + t % n] = A[t];
    for (int t = tid; t < n * n; t += nt) refl[t] = 0.0;
    __syncthreads();
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        const int o = k + 1;
        double x0 = a[o * ld + k];
        double s1 = 0.0;
        for (int i = 1 + tid; i < m; i += nt) {
            double x = a[(o + i) * ld + k];
            s1 += x * x;
        }
        s1 = block_sum(s1, red);
        if (tid == 0) d[k] = a[k * ld + k];
        if (s1 == 0.0) {
            if (tid == 0) e[k] = x0;
            __syncthreads();
            continue;
        }
        double nrm = sqrt(x0 * x0 + s1);
        double alpha = x0 >= 0.0 ? -nrm : nrm;
        double v0 = x0 - alpha;
        double inv = 1.0 / sqrt(v0 * v0 + s1);
        for (int i = tid; i < m; i += nt) {
            double vi = (i == 0 ? v0 : a[(o + i) * ld + k]) * inv;
            v[i] = vi;
            refl[(size_t)k * n + o + i] = vi;
        }
        if (tid == 0) e[k] = alpha;
        __syncthreads();
        // u = B v, B = a[o:, o:]: one warp per row
        for (int i = wid; i < m; i += nw) {
            const double* row = a + (size_t)(o + i) * ld + o;
            double acc = 0.0;
            for (int j = lane; j < m; j += 32) acc += row[j] * v[j];
            acc = warp_sum(acc);
            if (lane == 0) u[i] = acc;
        }
        __syncthreads();
        double g = 0.0;
        for (int i = tid; i < m; i += nt) g += v[i] * u[i];
        g = block_sum(g, red);
        for (int i = tid; i < m; i += nt) u[i] = 2.0 * u[i] - 2.0 * g * v[i];   // w
        __syncthreads();
        // B -= v w^T + w v^T on the lower triangle, mirrored to the upper one
        for (int i = wid; i < m; i += nw) {
            const double vi = v[i], wi = u[i];
            double* row = a + (size_t)(o + i) * ld + o;
            for (int j = lane; j <= i; j += 32) {
                double val = row[j] - vi * u[j] - wi * v[j];
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

// number of eigenvalues of T (d, e) below x, FP32 Sturm sequence
__host__ __device__ int sturm_count(const float* d, const float* e2, int n, float x, float pivmin) {
    int c = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++c;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
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

// Eigenvector of T (d, e; FP64) for the eigenvalue nearest `mu` by inverse iteration with
// Rayleigh-quotient shift updates (Gaussian elimination with partial pivoting on T - mu I).
// work: 5n doubles; flags: n bytes.  Result (unit 2-norm) in y; returns the final shift.
__host__ __device__ double invit_one(const double* d, const double* e, int n, double mu, double tnorm, int k,
                                     double* work, unsigned char* swapped, double* y) {
    const double eps = 1.1102230246251565e-16;
    double* dd = work;
    double* du = dd + n;
    double* du2 = du + n;
    double* mult = du2 + n;
    double* ty = mult + n;
    uint32_t hsh = 2166136261u ^ ((uint32_t)k * 16777619u);
    for (int i = 0; i < n; ++i) {
        hsh = hsh * 1664525u + 1013904223u;
        y[i] = 1.0 + 0.5 * ((double)(hsh >> 8) * (1.0 / 16777216.0) - 0.5);
    }
    const double tiny = eps * tnorm + 1e-300;
    for (int it = 0; it < 4; ++it) {
        for (int i = 0; i < n; ++i) { dd[i] = d[i] - mu; du[i] = (i + 1 < n) ? e[i] : 0.0; du2[i] = 0.0; }
        for (int i = 0; i + 1 < n; ++i) {
            double a = dd[i], b = du[i], c = e[i], dn = dd[i + 1], f = (i + 2 < n) ? du[i + 1] : 0.0;
            if (fabs(a) >= fabs(c)) {
                if (fabs(a) < tiny) a = a >= 0 ? tiny : -tiny;
                double mlt = c / a;
                dd[i] = a;
                dd[i + 1] = dn - mlt * b;
                mult[i] = mlt;
                swapped[i] = 0;
            } else {
                double mlt = a / c;
                dd[i] = c;
                du[i] = dn;
                du2[i] = f;
                dd[i + 1] = b - mlt * dn;
                if (i + 2 < n) du[i + 1] = -mlt * f;
                mult[i] = mlt;
                swapped[i] = 1;
            }
        }
        if (fabs(dd[n - 1]) < tiny) dd[n - 1] = dd[n - 1] >= 0 ? tiny : -tiny;
        for (int i = 0; i + 1 < n; ++i) {
            if (swapped[i]) {
                double t = y[i];
                y[i] = y[i + 1];
                y[i + 1] = t - mult[i] * y[i];
            } else {
                y[i + 1] -= mult[i] * y[i];
            }
        }
        y[n - 1] /= dd[n - 1];
        if (n >= 2) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) / dd[n - 2];
        for (int i = n - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / dd[i];
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += y[i] * y[i];
        s = 1.0 / sqrt(s);
        for (int i = 0; i < n; ++i) y[i] *= s;
        // Rayleigh quotient of the new vector as the next shift
        double num = 0.0;
        for (int i = 0; i < n; ++i) {
            double ti = d[i] * y[i];
            if (i > 0) ti += e[i - 1] * y[i - 1];
            if (i + 1 < n) ti += e[i] * y[i + 1];
            ty[i] = ti;
            num += y[i] * ti;
        }
        mu = num + (k + 1) * eps * tnorm;
    }
    return mu;
}

// Leading `nwant` eigenpairs of T: eigenvalues (descending) in w, tridiagonal eigenvectors
// y (n x nwant, column k = k-th largest) in Y.  One CTA; thread k handles eigenvalue k.
__global__ void __launch_bounds__(256) k_tri_eig(const double* __restrict__ d, const double* __restrict__ e,
                                                 int n, int nwant, double* __restrict__ w,
                                                 double* __restrict__ Y, double* __restrict__ scratch) {
    __shared__ float df[256], e2f[256];
    __shared__ float lam_sh[256];
    __shared__ double red[33];
    __shared__ float bounds[2];
    __shared__ double tn_sh;
    const int tid = threadIdx.x;
    if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i)
            t = fmax(t, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0));
        tn_sh = t > 0.0 ? t : 1.0;
    }
    __syncthreads();
    const double tnorm = tn_sh;
    const double sc = 1.0 / tnorm;                      // bisection on T / |T| (FP32 range)
    for (int i = tid; i < n; i += blockDim.x) {
        df[i] = (float)(d[i] * sc);
        e2f[i] = i + 1 < n ? (float)((e[i] * sc) * (e[i] * sc)) : 0.f;
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
    // ---- bisection (FP32) ----
    for (int k = tid; k < nwant; k += blockDim.x) lam_sh[k] = bisect_one(df, e2f, n, n - 1 - k, bounds[0], bounds[1]);
    __syncthreads();
    // ---- inverse iteration with Rayleigh-quotient shifts (FP64) ----
    const double eps = 1.1102230246251565e-16;
    for (int k = tid; k < nwant; k += blockDim.x) {
        double* work = scratch + (size_t)k * 6 * n;
        double* y = work + 5 * n;
        unsigned char swapped[256];
        double mu = (double)lam_sh[k] * tnorm + (k + 1) * eps * tnorm;
        invit_one(d, e, n, mu, tnorm, k, work, swapped, y);
        for (int i = 0; i < n; ++i) Y[(size_t)i * nwant + k] = y[i];
    }
    __syncthreads();
    // ---- Gram-Schmidt (twice) inside clusters, then FP64 Rayleigh quotients ----
    const double ctol = 1e-3;                 // cluster: normalised shifts closer than this
    for (int k = 1; k < nwant; ++k) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int jv = 0; jv < k; ++jv) {
                if (fabs((double)lam_sh[jv] - (double)lam_sh[k]) > ctol) continue;
                double dot = 0.0;
                for (int i = tid; i < n; i += blockDim.x) dot += Y[(size_t)i * nwant + jv] * Y[(size_t)i * nwant + k];
                dot = block_sum(dot, red);
                for (int i = tid; i < n; i += blockDim.x) Y[(size_t)i * nwant + k] -= dot * Y[(size_t)i * nwant + jv];
                __syncthreads();
            }
        }
        double s = 0.0;
        for (int i = tid; i < n; i += blockDim.x) { double v = Y[(size_t)i * nwant + k]; s += v * v; }
        s = block_sum(s, red);
        double sc = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        for (int i = tid; i < n; i += blockDim.x) Y[(size_t)i * nwant + k] *= sc;
        __syncthreads();
    }
    for (int k = tid; k < nwant; k += blockDim.x) {
        double num = 0.0;
        for (int i = 0; i < n; ++i) {
            double ti = d[i] * Y[(size_t)i * nwant + k];
            if (i > 0) ti += e[i - 1] * Y[(size_t)(i - 1) * nwant + k];
            if (i + 1 < n) ti += e[i] * Y[(size_t)(i + 1) * nwant + k];
            num += Y[(size_t)i * nwant + k] * ti;
        }
        w[k] = num;
    }
}

// z = H_0 H_1 ... H_{n-3} y for eigenvector column k (one CTA per column); reflector j is
// refl[j*n + j+1+i], H_j = I - 2 v v^T acting on rows j+1..n-1.
__global__ void k_backtransform(const double* __restrict__ refl, int n, int nwant, const double* __restrict__ Y,
                                double* __restrict__ V) {
    __shared__ double z[256];
    __shared__ double red[33];
    const int k = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = Y[(size_t)i * nwant + k];
    __syncthreads();
    for (int j = n - 3; j >= 0; --j) {
        const int o = j + 1, m = n - o;
        double dot = 0.0;
        const double* vj = refl + (size_t)j * n + o;
        for (int i = threadIdx.x; i < m; i += blockDim.x) dot += vj[i] * z[o + i];
        dot = block_sum(dot, red);
        for (int i = threadIdx.x; i < m; i += blockDim.x) z[o + i] -= 2.0 * dot * vj[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) V[(size_t)i * nwant + k] = z[i];
}

}  // namespace

size_t syev_scratch_doubles(int n) { return 2 * (size_t)n * n + 2 * (size_t)n + (size_t)n * n + 6 * (size_t)n * n + 64; }

// w: nwant eigenvalues (descending); V: n x nwant row-major eigenvectors
rbki_status syev_top_cuda(const double* A, int n, int nwant, double* w, double* V, double* scratch,
                          cudaStream_t st) {
    if (n > 256 || nwant > n || nwant < 1) return set_error(RBKI_E_UNSUPPORTED, "syev: n > 256");
    double* work = scratch;                      // n x n working matrix (global fallback)
    double* refl = work + (size_t)n * n;         // n x n reflectors (rows)
    double* d = refl + (size_t)n * n;
    double* e = d + n;
    double* Y = e + n;                           // n x nwant
    double* iiw = Y + (size_t)n * n;             // 6 n per wanted eigenvalue
    const size_t smem = (size_t)(n + 1) * n * sizeof(double);
    static size_t smax = 0;
    if (!smax) smax = max_dyn_smem(k_tridiag);
    const int use_smem = smem <= smax;
    k_tridiag<<<1, 512, use_smem ? smem : 0, st>>>(A, n, work, use_smem, d, e, refl);
    RBKI_LAUNCH_CHECK("k_tridiag");
    k_tri_eig<<<1, 256, 0, st>>>(d, e, n, nwant, w, Y, iiw);
    RBKI_LAUNCH_CHECK("k_tri_eig");
    k_backtransform<<<nwant, 128, 0, st>>>(refl, n, nwant, Y, V);
    RBKI_LAUNCH_CHECK("k_backtransform");
    return RBKI_OK;
}

rbki_status syev_cuda(const double* A, int n, double* w, double* V, double* scratch, cudaStream_t st) {
    return syev_top_cuda(A, n, n, w, V, scratch, st);
}

}  // namespace rbki
