// Partial column sampling of the Krylov construction (Sec. 3.2, after Table 2; Fig. 5).
//
// The Krylov space of a sampled mode is built from Y, a subset of X_(n)'s columns, instead
// of X_(n).  Columns are taken in units of 128 unfolding columns (one tile of the streaming
// kernels, so a sampled pass still reads whole contiguous rows):
//   C > 1: unit u = (a, c-block): a = u / nb, c in [128 (u % nb), +128), nb = ceil(C / 128)
//   C = 1: unit u = the 128 columns a in [128 u, +128)
// of X viewed as [A][I][C].  The kept units are the `kept` ones with the smallest key
//   key(u) = word 0 of Philox4x32-10(counter (u lo, u hi, mode, 0x53414D50), key = seed),
// ties to the lower index, in ascending order: a uniformly random subset of that size.
// Y keeps the [A][I][C] streaming layout: [kept][I][128] for C > 1, [kept * 128][I] for
// C = 1; its column j * 128 + t is column t of the j-th kept unit (zero past a ragged edge).
#include "plan.h"

namespace rbki {
namespace {

constexpr uint32_t SAMPLE_TAG = 0x53414D50u;
constexpr int SEL_THREADS = 1024;
constexpr int UNIT = 128;

__device__ __forceinline__ uint32_t unit_key(uint64_t seed, uint32_t mode, uint64_t u) {
    U4 c{(uint32_t)(u & 0xffffffffu), (uint32_t)(u >> 32), mode, SAMPLE_TAG};
    return philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)).x;
}

// exclusive prefix sum over the CTA (blockDim.x = SEL_THREADS); returns the CTA total too
__device__ long long block_exclusive_scan(long long v, long long* warp_tot, long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) warp_tot[lane] = w;       // inclusive over warps
    }
    __syncthreads();
    const long long before = (wid > 0 ? warp_tot[wid - 1] : 0) + incl - v;
    total = warp_tot[nw - 1];
    __syncthreads();
    return before;
}

// One CTA.  Radix select (8 bits a pass, most significant first) finds the threshold key T
// and how many keys equal to T are kept; a compaction in unit order writes the kept units.
// Keys are recomputed in each pass (a Philox evaluation is cheaper than a scratch round trip).
__global__ void __launch_bounds__(SEL_THREADS) k_sample_units(uint64_t seed, uint32_t mode, int64_t nu,
                                                             int64_t kept, int32_t* __restrict__ units) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_prefix;
    __shared__ long long s_need;
    __shared__ long long warp_tot[32];
    const int tid = threadIdx.x;
    uint32_t prefix = 0;
    long long need = kept;                      // rank wanted among the keys matching prefix
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = tid; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const uint32_t hmask = shift == 24 ? 0u : (0xffffffffu << (shift + 8));
        for (int64_t u = tid; u < nu; u += blockDim.x) {
            const uint32_t k = unit_key(seed, mode, (uint64_t)u);
            if ((k & hmask) == (prefix & hmask)) atomicAdd(&hist[(k >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            long long acc = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (acc + (long long)hist[b] >= need) break;
                acc += hist[b];
            }
            s_prefix = prefix | ((uint32_t)b << shift);
            s_need = need - acc;
        }
        __syncthreads();
        prefix = s_prefix;
        need = s_need;
        __syncthreads();
    }
    const uint32_t T = prefix;                  // keys < T are kept, and the first `need` keys == T
    const int64_t chunk = (nu + blockDim.x - 1) / blockDim.x;
    const int64_t u0 = (int64_t)tid * chunk, u1 = u0 + chunk < nu ? u0 + chunk : nu;
    long long eq = 0, total = 0;
    for (int64_t u = u0; u < u1; ++u) eq += unit_key(seed, mode, (uint64_t)u) == T;
    const long long eq_before = block_exclusive_scan(eq, warp_tot, total);
    long long mine = 0, e = eq_before;
    for (int64_t u = u0; u < u1; ++u) {
        const uint32_t k = unit_key(seed, mode, (uint64_t)u);
        if (k < T) ++mine;
        else if (k == T) mine += (e++ < need);
    }
    long long pos = block_exclusive_scan(mine, warp_tot, total);
    e = eq_before;
    for (int64_t u = u0; u < u1; ++u) {
        const uint32_t k = unit_key(seed, mode, (uint64_t)u);
        const bool keep = k < T || (k == T && e++ < need);
        if (keep && pos < kept) units[pos++] = (int32_t)u;
    }
}

// Y[j][i][t] = X[a][i][c] (C > 1): each (j, i) row is one unit's 128-column row segment.
// Rows are copied as 16-byte vectors (VR = 128 * elem / 16 per row) when C * elem is a
// multiple of 16, so every segment starts aligned and its valid part is whole vectors;
// element by element otherwise.
template <typename E, typename IT>
__global__ void __launch_bounds__(256) k_gather_c_vec(const uint4* __restrict__ x, IT I, IT nb, int64_t cv,
                                                      const int32_t* __restrict__ units, int64_t nvec,
                                                      uint4* __restrict__ y) {
    constexpr int VR = 128 * (int)sizeof(E) / 16;         // vectors per row
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nvec;
         e += (int64_t)gridDim.x * blockDim.x) {
        const IT row = (IT)(e / VR);
        const int v = (int)(e % VR);
        const IT j = row / I, i = row - j * I;
        const IT u = (IT)units[j];
        const IT a = u / nb;
        const int64_t cvec = (int64_t)(u - a * nb) * VR + v;       // vector index within the X row
        y[e] = cvec < cv ? x[((int64_t)a * I + i) * cv + cvec] : make_uint4(0u, 0u, 0u, 0u);
    }
}

template <typename E>
__global__ void __launch_bounds__(256) k_gather_c(const E* __restrict__ x, int64_t I, int64_t C,
                                                  const int32_t* __restrict__ units, int64_t n,
                                                  E* __restrict__ y) {
    const int64_t nb = (C + UNIT - 1) / UNIT;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / UNIT;
        const int t = (int)(e - row * UNIT);
        const int64_t j = row / I, i = row - j * I;
        const int64_t u = units[j];
        const int64_t a = u / nb, c = (u - a * nb) * UNIT + t;
        y[e] = c < C ? x[(a * I + i) * C + c] : E(0);
    }
}

// Y[j*128 + t][i] = X[128 u_j + t][i] (C = 1): each kept unit is one contiguous run of
// 128 I elements of X (cut at A), copied in units of W bytes (16 when I * elem allows it)
template <typename W, typename IT>
__global__ void __launch_bounds__(256) k_gather_a(const W* __restrict__ x, int64_t A, IT wrow,
                                                  const int32_t* __restrict__ units, int64_t n,
                                                  W* __restrict__ y) {
    const IT per_unit = (IT)UNIT * wrow;                  // words per unit
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const IT j = (IT)(e / per_unit), r = (IT)(e - (int64_t)j * per_unit);
        const int64_t a = (int64_t)units[j] * UNIT + r / wrow;
        y[e] = a < A ? x[(int64_t)units[j] * per_unit + r] : W();
    }
}

}  // namespace

rbki_status sample_units_cuda(uint64_t seed, int mode, int64_t nu, int64_t kept, int32_t* units,
                              cudaStream_t st) {
    if (nu < 1 || nu > 0x7fffffff || kept < 1 || kept > nu)
        return set_error(RBKI_E_INVAL, "sample_units: unit counts out of range");
    k_sample_units<<<1, SEL_THREADS, 0, st>>>(seed, (uint32_t)mode, nu, kept, units);
    RBKI_LAUNCH_CHECK("k_sample_units");
    return RBKI_OK;
}

rbki_status gather_units_cuda(const void* x, int dtype, int64_t A, int64_t I, int64_t C, const int32_t* units,
                              int64_t kept, void* y, cudaStream_t st) {
    const int64_t es = (int64_t)dtype_size(dtype);
    // a grid of 8 CTAs per SM (152 SMs) striding over the copy
    auto grid = [](int64_t n) { return (unsigned)std::min<int64_t>(cdiv(n, 256), 152 * 8); };
    const bool al = ((uintptr_t)x % 16) == 0 && ((uintptr_t)y % 16) == 0;
    if (C > 1) {
        if (I > 0x7fffffff) return set_error(RBKI_E_UNSUPPORTED, "gather: I too large");
        if (al && (C * es) % 16 == 0) {
            const int64_t nvec = kept * I * (128 * es / 16);
            const int64_t nb = cdiv(C, 128), cv = C * es / 16;
            // 32-bit index arithmetic when the row count and unit count fit
            const bool small = kept * I < 0xffffffffLL && A * nb < 0x7fffffffLL;
#define GV(E, IT) k_gather_c_vec<E, IT><<<grid(nvec), 256, 0, st>>>((const uint4*)x, (IT)I, (IT)nb, cv, units, \
                                                                   nvec, (uint4*)y)
#define GVE(E) if (small) GV(E, uint32_t); else GV(E, int64_t)
            if (es == 2) { GVE(uint16_t); } else if (es == 4) { GVE(uint32_t); } else { GVE(uint64_t); }
#undef GVE
#undef GV
        } else {
            const int64_t n = kept * I * 128;
#define GC(E) k_gather_c<E><<<grid(n), 256, 0, st>>>((const E*)x, I, C, units, n, (E*)y)
            if (es == 2) GC(uint16_t); else if (es == 4) GC(uint32_t); else GC(uint64_t);
#undef GC
        }
    } else {
        const int64_t row_bytes = I * es;
        if (al && row_bytes % 16 == 0) {
            const int64_t n = kept * 128 * (row_bytes / 16);
            if (128 * (row_bytes / 16) < 0xffffffffLL && kept < 0x7fffffffLL)
                k_gather_a<uint4, uint32_t><<<grid(n), 256, 0, st>>>((const uint4*)x, A, (uint32_t)(row_bytes / 16),
                                                                    units, n, (uint4*)y);
            else
                k_gather_a<uint4, int64_t><<<grid(n), 256, 0, st>>>((const uint4*)x, A, row_bytes / 16, units, n,
                                                                   (uint4*)y);
        } else {
            const int64_t n = kept * 128 * I;
#define GA(E) k_gather_a<E, int64_t><<<grid(n), 256, 0, st>>>((const E*)x, A, I, units, n, (E*)y)
            if (es == 2) GA(uint16_t); else if (es == 4) GA(uint32_t); else GA(uint64_t);
#undef GA
        }
    }
    RBKI_LAUNCH_CHECK("k_gather_units");
    return RBKI_OK;
}

}  // namespace rbki
