// Batched rBKI-TK for many small decompositions (rbki_tucker_batched): a wave of requests
// runs Algorithms 1-2 in lockstep, one launch per stage for every mode of every request.
//
// The served stream (3rd-order tensors of 32..256 per mode, ranks 4..32) is bound by kernel
// launches, not by HBM: one decomposition is ~250 small launches, and the host issues about
// 200k launches/s however many threads it uses.  Here a stage is one launch whatever the
// number of requests:
//   * the X passes (sketch W = X_(n) Omega, Krylov step P = X_(n) (X_(n)^T Q), Gram
//     X_(n) X_(n)^T, the core's mode products) of all items share one work-queue kernel
//     (k_xpass_b): block (x, y) of the launch is unit x of item y, a run of 64-column tiles of
//     X_(n) whose products it accumulates in registers; a fixed-order reduction follows;
//   * the FP64 stages (block orthonormalisation, Z = Q^T P, the eigensolver, U = Q U~) are the
//     batched twins of the single-call kernels (bat_launch): the same device code and the
//     same per-item grids, so each item's result does not depend on what shares its wave.
// The products run on CUDA cores in FP32 from BF16/FP16 values of X (X rounded to the
// requested precision as it is read; FP32 Omega and Q), with FP32 accumulation per tile run
// and FP64 accumulation across runs.  Orthonormalisation and the eigensolver stay FP64.
#include "kernels.h"
#include "plan.h"

#include <cmath>
#include <cstring>
#include <mutex>

namespace rbki {
namespace {

enum XOp { XO_SKETCH = 0, XO_KRYLOV = 1, XO_GRAM = 2, XO_TTM = 3 };
constexpr int XT = 64;          // columns of X_(n) per tile
constexpr int XTHREADS = 256;   // 8 warps

__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float round_to(float v, int rnd) {
    if (rnd == RBKI_BF16) return __bfloat162float(__float2bfloat16_rn(v));
    if (rnd == RBKI_F16) return __half2float(__float2half_rn(v));
    return v;
}

// XTs[t][i] = X_(n)[i][col0 + t] for the tile's 64 columns (colb[t] = offset of X[a][0][c],
// -1 past the end); coalesced along c (C > 1) or along i (C == 1), loads unrolled by 4
template <typename T>
__device__ __forceinline__ void stage_tile(const T* __restrict__ x, const int64_t* colb, int I, int Ip, int64_t C,
                                           int rnd, float* XTs) {
    const int n = 64 * I;
    if (C == 1) {
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += 256) {
            const int tt = e / I, i = e - tt * I;
            const int64_t cb = colb[tt];
            XTs[tt * Ip + i] = cb >= 0 ? round_to(to_f32(x[cb + i]), rnd) : 0.f;
        }
    } else {
#pragma unroll 4
        for (int e = threadIdx.x; e < n; e += 256) {
            const int i = e >> 6, tt = e & 63;
            const int64_t cb = colb[tt];
            XTs[tt * Ip + i] = cb >= 0 ? round_to(to_f32(x[cb + (int64_t)i * C]), rnd) : 0.f;
        }
    }
}

struct xpass_rec {
    const void* x;          // the item's tensor, viewed as [A][I][C] for its mode
    int dtype, rnd;         // storage dtype; rounding applied as values are read (0: none)
    int A, I, C;
    int op, S;              // XOp; product width (<= 64; Gram: I, in column blocks of 64)
    int tiles, tpu;         // 64-column tiles of X_(n); tiles per unit
    const double* Q;        // KRYLOV / TTM operand, I x S (ld ldq)
    int ldq;
    uint64_t seed;          // SKETCH: Omega^(mode) (Philox4x32-10 + Box-Muller)
    int mode;
    float* part;            // SKETCH / KRYLOV / GRAM: [unit][I][ldp] partial sums
    int ldp;
    void* tout;             // TTM: [A][S][C] result, FP32 or FP64 (tdt)
    int tdt;
    int gx, gy, gz;         // units, Gram column blocks, 1
};

__host__ __device__ inline int xp_ip(int I) { return I | 1; }   // odd pitch: conflict-free columns
__host__ __device__ inline int xp_s8(int S) { return (S + 7) & ~7; }
size_t xpass_smem(const xpass_rec& r) {
    const int S = r.op == XO_GRAM ? std::min(64, r.I) : r.S;
    const int S8 = xp_s8(S);
    const bool q = r.op == XO_KRYLOV || r.op == XO_TTM;
    const int ns1 = 8 / (S8 / 8);
    return ((size_t)XT * xp_ip(r.I) + (q ? (size_t)r.I * S8 : 0) + (size_t)XT * S8 +
            (q && ns1 > 1 ? (size_t)ns1 * XT * S8 : 0)) * sizeof(float) +
           XT * sizeof(int64_t);
}

// Unit `unit` of one item: tiles [unit * tpu, (unit + 1) * tpu).  Per tile the X tile is
// staged transposed (XT[t][i], odd pitch), then
//   SKETCH:  Y[t][s] = Omega(col t, s)                      (generated in place)
//   KRYLOV:  Y = X_tile^T Q                                  (GEMM 1: warp w -> 8 columns)
//   TTM:     Y = X_tile^T U, written out as [A][S][C]
//   GRAM:    Y[t][s] = X[sb + s][t]                          (the tile itself)
// and, except for TTM, P += X_tile Y (GEMM 2: warp w -> 8 columns x a share of the rows,
// registers across all tiles of the unit).  MR bounds the 32-row groups a thread of GEMM 2
// accumulates (ceil(ceil(I/32) / warps per column group)): launches are split by MR so that
// small items run with fewer registers and less shared memory, hence more CTAs per SM.
template <int MR>
__device__ __forceinline__ void xpass_dev(const xpass_rec& r, int unit, int blk) {
    extern __shared__ __align__(16) float xsm[];
    const int I = r.I, Ip = xp_ip(I);
    const int sb = r.op == XO_GRAM ? blk * 64 : 0;
    const int S = r.op == XO_GRAM ? min(64, I - sb) : r.S;
    const int S8 = xp_s8(S);
    const bool useq = r.op == XO_KRYLOV || r.op == XO_TTM;
    const int G = S8 / 8;
    const int ns1 = 8 / G;                    // GEMM 1: warps per column group (row shares)
    const int ns2 = 8 / G;                    // GEMM 2: warps per column group (row split)
    float* XTs = xsm;
    float* Qs = XTs + XT * Ip;
    float* Ys = Qs + (useq ? I * S8 : 0);
    float* Yp = Ys + XT * S8;                 // GEMM 1 row-share partials (ns1 > 1)
    int64_t* colb = reinterpret_cast<int64_t*>(Yp + (useq && ns1 > 1 ? ns1 * XT * S8 : 0));
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t C = r.C, J = (int64_t)r.A * r.C;
    if (useq)
        for (int e = tid; e < I * S8; e += XTHREADS) {
            const int i = e / S8, s = e % S8;
            Qs[e] = s < S ? (float)r.Q[(int64_t)i * r.ldq + s] : 0.f;
        }
    const bool act1 = w < G * ns1;
    const int g1 = w % G, h1 = w / G;
    const bool act2 = w < G * ns2;
    const int g2 = w % G, h2 = w / G;
    const int nr32 = (I + 31) / 32;
    float acc[MR][8];
#pragma unroll
    for (int k = 0; k < MR; ++k)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[k][j] = 0.f;
    const int t_lo = unit * r.tpu, t_hi = min(r.tiles, t_lo + r.tpu);
    for (int t = t_lo; t < t_hi; ++t) {
        const int64_t col0 = (int64_t)t * XT;
        __syncthreads();   // the previous tile is consumed
        if (tid < XT) {
            const int64_t col = col0 + tid;
            colb[tid] = col < J ? (col / C) * I * C + col % C : -1;
        }
        __syncthreads();
        switch (r.dtype) {
            case RBKI_BF16: stage_tile(static_cast<const __nv_bfloat16*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
            case RBKI_F16: stage_tile(static_cast<const __half*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
            case RBKI_F32: stage_tile(static_cast<const float*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
            default: stage_tile(static_cast<const double*>(r.x), colb, I, Ip, C, r.rnd, XTs); break;
        }
        if (r.op == XO_SKETCH) {
            const int np = S8 / 2;
            for (int e = tid; e < XT * np; e += XTHREADS) {
                const int tt = e / np, pr = e % np, s = 2 * pr;
                float z0 = 0.f, z1 = 0.f;
                if (colb[tt] >= 0 && s < S)
                    omega_pair_f32(r.seed, (uint32_t)r.mode, (uint64_t)(col0 + tt), (uint32_t)pr, z0, z1);
                Ys[tt * S8 + s] = z0;
                Ys[tt * S8 + s + 1] = s + 1 < S ? z1 : 0.f;
            }
        }
        __syncthreads();
        if (useq) {
            // GEMM 1, Y = X_tile^T Q: warp (g, h) owns columns 8g..8g+7 and rows i of its share
            // [h*il, (h+1)*il) for both 32-column halves; the ns1 shares meet in Yp
            if (act1) {
                const int s0 = 8 * g1;
                const int il = (I + ns1 - 1) / ns1, i_lo = h1 * il, i_hi = min(I, i_lo + il);
                float a1[2][8];
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int j = 0; j < 8; ++j) a1[u][j] = 0.f;
                for (int i = i_lo; i < i_hi; ++i) {
                    const float4 qa = *reinterpret_cast<const float4*>(Qs + i * S8 + s0);
                    const float4 qb = *reinterpret_cast<const float4*>(Qs + i * S8 + s0 + 4);
                    const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
                    const float x0 = XTs[lane * Ip + i], x1 = XTs[(lane + 32) * Ip + i];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        a1[0][j] = fmaf(x0, qv[j], a1[0][j]);
                        a1[1][j] = fmaf(x1, qv[j], a1[1][j]);
                    }
                }
                float* dst = ns1 == 1 ? Ys : Yp + h1 * XT * S8;
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int j = 0; j < 8; ++j) dst[(lane + 32 * u) * S8 + s0 + j] = a1[u][j];
            }
            if (ns1 > 1) {
                __syncthreads();
                for (int e = tid; e < XT * S8; e += XTHREADS) {
                    float v = 0.f;
                    for (int h = 0; h < ns1; ++h) v += Yp[h * XT * S8 + e];
                    Ys[e] = v;
                }
            }
            __syncthreads();
            if (r.op == XO_TTM) {
                // T[a][s][c] for the tile's valid columns (coalesced along c)
                for (int e = tid; e < XT * S; e += XTHREADS) {
                    const int s = e / XT, tt = e % XT;
                    const int64_t col = col0 + tt;
                    if (col >= J) continue;
                    const int64_t a = col / C, c = col % C;
                    const int64_t o = (a * S + s) * C + c;
                    const float v = Ys[tt * S8 + s];
                    if (r.tdt == RBKI_F64) static_cast<double*>(r.tout)[o] = (double)v;
                    else static_cast<float*>(r.tout)[o] = v;
                }
                continue;
            }
        }
        if (act2) {
            const int s0 = 8 * g2;
            for (int tt = 0; tt < XT; ++tt) {
                float yv[8];
                if (r.op == XO_GRAM) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) yv[j] = s0 + j < S ? XTs[tt * Ip + sb + s0 + j] : 0.f;
                } else {
                    const float4 ya = *reinterpret_cast<const float4*>(Ys + tt * S8 + s0);
                    const float4 yb = *reinterpret_cast<const float4*>(Ys + tt * S8 + s0 + 4);
                    yv[0] = ya.x; yv[1] = ya.y; yv[2] = ya.z; yv[3] = ya.w;
                    yv[4] = yb.x; yv[5] = yb.y; yv[6] = yb.z; yv[7] = yb.w;
                }
#pragma unroll
                for (int k = 0; k < MR; ++k) {
                    const int m = h2 + k * ns2;
                    if (m >= nr32) break;
                    const int i = lane + 32 * m;
                    const float xv = i < I ? XTs[tt * Ip + i] : 0.f;
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[k][j] = fmaf(xv, yv[j], acc[k][j]);
                }
            }
        }
    }
    if (r.op == XO_TTM || !act2) return;
    float* out = r.part + (int64_t)unit * I * r.ldp + sb;
    const int s0 = 8 * g2;
#pragma unroll
    for (int k = 0; k < MR; ++k) {
        const int m = h2 + k * ns2;
        if (m >= nr32) break;
        const int i = lane + 32 * m;
        if (i >= I) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (s0 + j < S) out[(int64_t)i * r.ldp + s0 + j] = acc[k][j];
    }
}

template <int MR>
__global__ void __launch_bounds__(XTHREADS, MR <= 2 ? 3 : 2) k_xpass_b(const __grid_constant__ BPack<xpass_rec> p) {
    const xpass_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    xpass_dev<MR>(r, bx, by);
}

// row groups per GEMM-2 thread of a record (GEMM 2 only runs for SKETCH / KRYLOV / GRAM)
int xpass_mr(const xpass_rec& r) {
    const int S = r.op == XO_GRAM ? std::min(64, r.I) : r.S;
    const int G = xp_s8(S) / 8, ns2 = 8 / G, nr32 = (r.I + 31) / 32;
    return (nr32 + ns2 - 1) / ns2;
}

// out1[i][s] (= out2[i][s]) = sum over units of part[u][i][s], in unit order, FP64;
// sym: 0.5 (G[i][s] + G[s][i]) (the Gram path's Z, symmetric by construction)
struct xreduce_rec {
    const float* part;
    int units, I, S, ldp, sym;
    double* out1;
    int ld1;
    double* out2;
    int ld2;
    int gx, gy, gz;
};

__global__ void __launch_bounds__(256) k_xreduce_b(const __grid_constant__ BPack<xreduce_rec> p) {
    const xreduce_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz)) return;
    const int e = bx * 256 + threadIdx.x;
    if (e >= r.I * r.S) return;
    const int i = e / r.S, s = e % r.S;
    const int64_t us = (int64_t)r.I * r.ldp;
    double a = 0.0;
    for (int u = 0; u < r.units; ++u) a += (double)r.part[u * us + (int64_t)i * r.ldp + s];
    if (r.sym) {
        double b = 0.0;
        for (int u = 0; u < r.units; ++u) b += (double)r.part[u * us + (int64_t)s * r.ldp + i];
        a = 0.5 * (a + b);
    }
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

// *p = v for every record (the Krylov-path kept counters of a wave in one launch)
struct fill_rec {
    int32_t* p;
    int32_t v;
    int gx, gy, gz;
};

__global__ void k_fill_b(const __grid_constant__ BPack<fill_rec> p) {
    const fill_rec& r = p.r[blockIdx.y];
    int bx, by, bz;
    if (!bat_block(r, bx, by, bz) || threadIdx.x) return;
    *r.p = r.v;
}

// info[n] = kept Krylov width (Krylov path) or I_n (Gram path); info[N+n] = path;
// info[2N] = 0 (the wave's kernels have no device waits); q_used[n] = q or 0
struct info_rec {
    int32_t* info;
    int32_t* q_used;
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
        if (n == 0) r.info[2 * r.N] = 0;
    }
    if (r.q_used) r.q_used[n] = r.gram[n] ? 0 : r.q;
}

}  // namespace
}  // namespace rbki

// ---------------------------------------------------------------------------------------
// Work-queue granularity: tiles per unit of an item.  A unit is one CTA; smaller units spread
// an item over more SMs, larger ones leave fewer partial sums to reduce.  The work per unit
// comes from a table by (op, I_n, S) bucket: a default, or the values measured by
// rbki_wave_autotune / read by rbki_wave_tune_load.
// ---------------------------------------------------------------------------------------
namespace rbki {
namespace {

constexpr int TUNE_OPS = 4, TUNE_IB = 8, TUNE_SB = 8;   // I_n in 32-buckets, S in 8-buckets
constexpr double DEFAULT_WORK = 49152.0;                 // ~10 tiles of a 144 x 24 item
std::mutex g_tune_mu;
double g_tune_work[TUNE_OPS][TUNE_IB][TUNE_SB];          // work per unit; 0 = default
bool g_tune_init = false;

int tune_ib(int I) { return std::min(TUNE_IB - 1, std::max(0, (I - 1) / 32)); }
int tune_sb(int S) { return std::min(TUNE_SB - 1, std::max(0, (S - 1) / 8)); }
// cost model of one tile: the two products (I x S8 each way) and the staging of I x 64 values
double tile_cost(int I, int S) { return (double)I * (xp_s8(std::min(S, 64)) + 8); }

double tuned_work(int op, int I, int S) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const double w = g_tune_init ? g_tune_work[op][tune_ib(I)][tune_sb(S)] : 0.0;
    return w > 0.0 ? w : DEFAULT_WORK;
}

// tiles per unit of an item: about a fixed amount of work per unit (CTA), so that large and
// small items of one wave finish their units together; depends only on the item's shape
int wave_tpu(int op, int I, int S, int tiles) {
    const double t = tuned_work(op, I, S) / tile_cost(I, S);
    return (int)std::min<double>(std::max(1.0, std::floor(t)), std::max(1, tiles));
}

}  // namespace
}  // namespace rbki

// ---------------------------------------------------------------------------------------
// Host side: plan, workspace and the lockstep schedule of one wave.
// ---------------------------------------------------------------------------------------
namespace rbki {
namespace {

constexpr size_t WAVE_ALIGN = 256;

int wave_units(int tiles, int tpu) { return (int)cdiv(tiles, std::max(1, tpu)); }

struct WaveMode {
    int n = 0;
    const ModePlan* m = nullptr;
    double *Qall = nullptr, *Pall = nullptr, *Z = nullptr, *evec = nullptr, *eval = nullptr;
    double *syev_ws = nullptr, *orth_ws = nullptr, *atb_part = nullptr;
    int32_t* kept = nullptr;
    float* xpart = nullptr;
    int tiles = 0, tpu = 1, units = 1;
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
    int rnd = 0;                // RBKI_BF16 / RBKI_F16: rounding of X as it is read
    int ttm_tpu[RBKI_MAX_ORDER] = {0};
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
        w.n = n;
        w.m = &m;
        const int64_t J = m.A * m.C;
        w.tiles = (int)cdiv(J, XT);
        w.tpu = wave_tpu(m.gram ? 2 : 1, (int)m.I, m.gram ? (int)m.I : m.S, w.tiles);
        w.units = wave_units(w.tiles, w.tpu);
        const int b = m.b;
        const int ev = m.gram ? (int)m.I : b;
        w.Z = cv.take<double>((size_t)ev * ev);
        w.evec = cv.take<double>((size_t)ev * m.R);
        w.eval = cv.take<double>((size_t)ev);
        w.syev_ws = cv.take<double>(syev_scratch_doubles(ev));
        w.kept = cv.take<int32_t>(1);
        if (m.gram) {
            w.xpart = cv.take<float>((size_t)w.units * m.I * m.I);
        } else {
            w.Qall = cv.take<double>((size_t)m.I * b);
            w.Pall = cv.take<double>((size_t)m.I * b);
            w.orth_ws = cv.take<double>(orth_scratch_doubles(m.I, b - m.S, m.S));
            w.atb_part = cv.take<double>((size_t)atb_nchunks(m.I) * b * b);
            w.xpart = cv.take<float>((size_t)w.units * m.I * m.S);
        }
    }
    q.tbuf[0] = cv.take<float>((size_t)q.tmax);
    q.tbuf[1] = cv.take<float>((size_t)q.tmax);
    q.sq_part = cv.take<double>((size_t)cdiv(std::max(pl.numel, pl.ranks_numel), SQ_CHUNK));
    q.norms = cv.take<double>(2);
}

template <int MR>
rbki_status launch_xpass_class(const std::vector<xpass_rec>& recs, cudaStream_t st) {
    if (recs.empty()) return RBKI_OK;
    size_t sm = 0;
    for (const auto& r : recs) sm = std::max(sm, xpass_smem(r));
    static const size_t smax = max_dyn_smem(k_xpass_b<MR>);   // thread-safe, once per MR
    if (sm > smax) return set_error(RBKI_E_UNSUPPORTED, "batched X pass: shared memory");
    return bat_launch(k_xpass_b<MR>, recs.data(), (int)recs.size(), XTHREADS, sm, st, "k_xpass_b");
}

// one launch per register class (a TTM runs no GEMM 2: the smallest class)
rbki_status launch_xpass(const std::vector<xpass_rec>& recs, cudaStream_t st) {
    std::vector<xpass_rec> c2, c4, c8;
    for (const auto& r : recs) {
        const int mr = r.op == XO_TTM ? 1 : xpass_mr(r);
        (mr <= 2 ? c2 : mr <= 4 ? c4 : c8).push_back(r);
    }
    RBKI_TRY(launch_xpass_class<2>(c2, st));
    RBKI_TRY(launch_xpass_class<4>(c4, st));
    return launch_xpass_class<8>(c8, st);
}

xpass_rec xrec(const WaveReq& q, const WaveMode& w, int op) {
    const ModePlan& m = *w.m;
    xpass_rec r{};
    r.x = q.X.data;
    r.dtype = q.X.dtype;
    r.rnd = q.X.dtype == q.pl.stream_dtype ? 0 : q.rnd;
    r.A = (int)m.A;
    r.I = (int)m.I;
    r.C = (int)m.C;
    r.op = op;
    r.S = op == XO_GRAM ? (int)m.I : m.S;
    r.tiles = w.tiles;
    r.tpu = w.tpu;
    r.part = w.xpart;
    r.ldp = r.S;
    r.seed = q.pl.seed;
    r.mode = m.n;
    r.gx = w.units;
    r.gy = op == XO_GRAM ? (int)cdiv(m.I, 64) : 1;
    r.gz = 1;
    return r;
}

xreduce_rec rrec(const WaveMode& w, double* out1, int ld1, double* out2, int ld2) {
    const ModePlan& m = *w.m;
    const int S = m.gram ? (int)m.I : m.S;
    return xreduce_rec{w.xpart, w.units, (int)m.I, S, S, m.gram ? 1 : 0, out1, ld1, out2, ld2,
                       (int)cdiv((int64_t)m.I * S, 256), 1, 1};
}

// Algorithms 1-2 for every request of the wave, stage by stage.
rbki_status run_wave(std::vector<WaveReq>& Q, cudaStream_t st) {
    const int nq = (int)Q.size();
    // ---- |X|^2 ----
    {
        std::vector<sumsq_rec> sq;
        for (auto& q : Q)
            sq.push_back(sumsq_rec{q.X.data, q.X.dtype, q.pl.numel, q.sq_part, q.norms, (int)cdiv(q.pl.numel, SQ_CHUNK), 1, 1});
        RBKI_TRY(bat_launch(k_sumsq_part_b, sq.data(), nq, 256, 0, st, "k_sumsq_part_b"));
        for (auto& r : sq) r.gx = 1;
        RBKI_TRY(bat_launch(k_sumsq_fin_b, sq.data(), nq, 32, 0, st, "k_sumsq_fin_b"));
    }
    // ---- Algorithm 1 steps 1-2 (sketch) on Krylov modes; Z = X_(n) X_(n)^T on Gram modes ----
    int qmax = 0;
    {
        std::vector<xpass_rec> xp;
        std::vector<xreduce_rec> xr;
        std::vector<fill_rec> fk;
        for (auto& q : Q)
            for (int n = 0; n < q.pl.N; ++n) {
                WaveMode& w = q.mode[n];
                if (w.m->gram) {
                    xp.push_back(xrec(q, w, XO_GRAM));
                    xr.push_back(rrec(w, w.Z, (int)w.m->I, nullptr, 0));
                } else {
                    xp.push_back(xrec(q, w, XO_SKETCH));
                    xr.push_back(rrec(w, w.Qall, w.m->b, nullptr, 0));
                    qmax = std::max(qmax, w.m->q);
                    fk.push_back(fill_rec{w.kept, 0, 1, 1, 1});
                }
            }
        RBKI_TRY(bat_launch(k_fill_b, fk.data(), (int)fk.size(), 32, 0, st, "k_fill_b"));
        RBKI_TRY(launch_xpass(xp, st));
        RBKI_TRY(bat_launch(k_xreduce_b, xr.data(), (int)xr.size(), 256, 0, st, "k_xreduce_b"));
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
    // ---- step 3: K = [W, A W, ..., A^q W], block by block ----
    for (int j = 0; j <= qmax; ++j) {
        std::vector<xpass_rec> xp;
        std::vector<xreduce_rec> xr;
        std::vector<WaveMode*> ws;
        std::vector<int> c0;
        for (auto& q : Q)
            for (int n = 0; n < q.pl.N; ++n) {
                WaveMode& w = q.mode[n];
                const ModePlan& m = *w.m;
                if (m.gram || j > m.q) continue;
                xpass_rec r = xrec(q, w, XO_KRYLOV);
                r.Q = w.Qall + j * m.S;
                r.ldq = m.b;
                xp.push_back(r);
                const bool more = j < m.q;
                xr.push_back(rrec(w, w.Pall + j * m.S, m.b, more ? w.Qall + (j + 1) * m.S : nullptr, m.b));
                if (more) {
                    ws.push_back(&w);
                    c0.push_back((j + 1) * m.S);
                }
            }
        RBKI_TRY(launch_xpass(xp, st));
        RBKI_TRY(bat_launch(k_xreduce_b, xr.data(), (int)xr.size(), 256, 0, st, "k_xreduce_b"));
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
        std::vector<xpass_rec> xp;
        for (int k = 0; k < nq; ++k) {
            WaveReq& q = Q[k];
            const Plan& pl = q.pl;
            if (t >= pl.N) continue;
            int64_t* c = &cur[k * RBKI_MAX_ORDER];
            const int md = pl.order[t];
            const ModePlan& m = pl.mode[md];
            int64_t A = 1, C = 1;
            for (int i = 0; i < md; ++i) A *= c[i];
            for (int i = md + 1; i < pl.N; ++i) C *= c[i];
            xpass_rec r{};
            r.x = t == 0 ? q.X.data : q.tbuf[(t - 1) & 1];
            r.dtype = t == 0 ? q.X.dtype : RBKI_F32;
            r.rnd = t == 0 && q.X.dtype != pl.stream_dtype ? q.rnd : 0;
            r.A = (int)A;
            r.I = (int)c[md];
            r.C = (int)C;
            r.op = XO_TTM;
            r.S = m.R;
            r.tiles = (int)cdiv(A * C, XT);
            r.tpu = wave_tpu(3, r.I, m.R, r.tiles);
            r.Q = q.out.factors[md];
            r.ldq = m.R;
            const bool last = t == pl.N - 1;
            r.tout = last ? (void*)q.out.core : (void*)q.tbuf[t & 1];
            r.tdt = last ? RBKI_F64 : RBKI_F32;
            r.gx = wave_units(r.tiles, r.tpu);
            r.gy = r.gz = 1;
            xp.push_back(r);
            c[md] = m.R;
        }
        RBKI_TRY(launch_xpass(xp, st));
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

}  // namespace
}  // namespace rbki

using namespace rbki;

extern "C" {

rbki_status rbki_tucker_batched_workspace(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                                          size_t* bytes) {
    if (!bytes) return set_error(RBKI_E_INVAL, "bytes is NULL");
    std::vector<WaveReq> Q;
    return wave_prepare(count, X, prm, nullptr, nullptr, Q, bytes);
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
