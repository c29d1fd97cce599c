// Tensor-core streaming kernels (k_tc.cu): host interface.
#pragma once

#include "kernels.h"

namespace rbki {
namespace tc {

enum { KRYLOV = 0, SKETCH = 1, TTM = 2 };

struct Params {
    int64_t A, I, C;        // X viewed as [A][I][C]
    int NS;                 // 128-row slabs: cdiv(I, 128)
    int N;                  // MMA N (includes the lo half when split)
    int Sh;                 // logical width (N/2 when split, else the used columns)
    int split;
    int64_t tiles, ctiles;
    int nslot;
    uint32_t smem_x, smem_q, smem_y, smem_bar;
    uint32_t tmem_cols;
    const void* qimg;       // GEMM1 B image (global)
    uint32_t qimg_bytes;
    const void* omg;        // per-tile Omega images (SKETCH)
    uint32_t yimg_bytes;    // 128 * N * 2
    float* part;            // [grid][I][N] partial products (KRYLOV, SKETCH)
    float* yout;            // [A][Sh][C] TTM output
    void* yimg_out;         // TTM alternative output: per-tile BF16/FP16 images of Y in the
                            // layout SKETCH consumes (the first pass of a two-pass Krylov step)
    int* err;               // error word (bounded wait expired)
    int fp16;
    uint32_t wait_us;       // microseconds before a bounded mbarrier wait gives up
    int stall;              // nonzero: the MMA issuer first waits on a barrier nothing arrives at
                            // (the planted stall that exercises the timeout path)
};

bool supported(const View& v, int mode, int N);
int64_t num_tiles(const View& v);
int grid_size(const View& v);
size_t image_bytes_skinny(const View& v, int N);
size_t image_bytes_omega(const View& v, int N);
// split: 0 the values (rounded), 1 hi in columns < S and lo = value - hi in columns
// N/2 .. N/2+S-1 (S <= N/2), 2 the lo parts alone in columns < S
rbki_status skinny_image(const double* M, int64_t ldm, int64_t rows, int S, int N, int split, bool fp16,
                         void* img, cudaStream_t st);
rbki_status omega_images(uint64_t seed, int mode, const View& v, int S, int N, bool split, void* img,
                         cudaStream_t st);
rbki_status stream_tc(int mode, const View& v, int N, int Sh, bool split, const void* qimg, const void* omg,
                      float* part, float* yout, int* err, cudaStream_t st, void* yimg_out = nullptr,
                      uint32_t wait_us = 0, int stall = 0);
// Fused Krylov step on the pipelined kernel (k_krylov.cu): 64-column tiles, two tiles
// resident, GEMM1 of the next tile overlapping the epilogue of the current one.
bool krylov_supported(const View& v, int N);
int64_t krylov_tiles(const View& v);
int krylov_grid(const View& v);
// part: [krylov_grid(v)][I][N] FP32 partial products of P = X_(n) (X_(n)^T Q); reduce with
// reduce_parts(part, krylov_grid(v), ...).  wait_us 0 = default; stall = planted stall.
rbki_status krylov_tc(const View& v, int N, int Sh, bool split, const void* qimg, float* part, int* err,
                      cudaStream_t st, uint32_t wait_us = 0, int stall = 0);
// out (ld) [and out2 (ld2)] = sum of the grid's partial products, FP64, fixed order; NaN
// everywhere when *err is nonzero (a bounded wait of the producing kernel expired, so the
// partials are incomplete)
rbki_status reduce_parts(const float* part, int nb, int64_t I, int N, int Sh, bool split, double* out,
                         int64_t ld, double* out2, int64_t ld2, const int* err, cudaStream_t st);

// batched forms of the operand-image and reduction launches (one launch for many items)
struct SkinnyItem {
    const double* M; int64_t ldm, rows; int S, N, split; bool fp16; void* img;
};
rbki_status skinny_image_batched(const SkinnyItem* it, int n, cudaStream_t st);
struct OmegaItem {
    uint64_t seed; int mode; View v; int S, N; bool split; void* img;
};
rbki_status omega_images_batched(const OmegaItem* it, int n, cudaStream_t st);
// The FP32 -> BF16 staging of X (n elements, n % 4 == 0, x 16-byte and dst 8-byte aligned)
// with per-CTA partial sums of squares in part[0 .. stage_omega_grid()), and the Omega images
// of up to 8 items (0: the cast alone), in one launch (the two jobs share the SMs).  Same staged values and images
// as stage_cuda and omega_images_batched.
int stage_omega_grid();
rbki_status stage_omega_batched(const float* x, int64_t n, void* dst, double* part, const OmegaItem* it, int n_items,
                                cudaStream_t st);
struct ReduceItem {
    const float* part; int nb; int64_t I; int N, Sh; bool split;
    double* out; int64_t ld; double* out2; int64_t ld2; const int* err;
};
rbki_status reduce_parts_batched(const ReduceItem* it, int n, cudaStream_t st);

}  // namespace tc
}  // namespace rbki
