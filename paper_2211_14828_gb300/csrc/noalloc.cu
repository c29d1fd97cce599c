// Krylov step (P = X_(n) (X_(n)^T Q)) on the tensor-core kernel without any
// caller-provided workspace: its scratch (operand image, per-CTA partial products,
// error word) lives in a fixed array compiled into this library.
//
// Who needs it: some host applications hand all device memory to their own allocator
// at start-up, or run this step from code where calling cudaMalloc is not permitted or
// too slow (latency-critical loops, plug-ins inside a process that owns the GPU).  They
// cannot supply the workspace the other entry points ask for.
//
// Costs and rules:
//   * every GPU that loads librbki.so keeps RBKI_NOALLOC_SCRATCH_BYTES of device memory
//     for this array until the process exits;
//   * all calls share the one array: calls that overlap on the GPU (different streams,
//     or threads without ordering) race on it; serialise them;
//   * each call looks up the array's device address on the current device with
//     cudaGetSymbolAddress (no allocation; nothing is cached, so a device reset or a new
//     primary context leaves no stale address behind); the first call on a device may load
//     the library's device code, so make it before any stream capture starts;
//   * the error word is cleared at the start of each call; if a bounded wait inside the
//     kernel expires, every entry of P is set to NaN (the partial products are incomplete).
#include "plan.h"
#include "tc.h"

namespace rbki {
namespace {

constexpr size_t kScratchBytes = (size_t)RBKI_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on the current device.
rbki_status scratch_address(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = p;
    return RBKI_OK;
}

}  // namespace
}  // namespace rbki

using namespace rbki;

extern "C" rbki_status rbki_krylov_product_noalloc(const rbki_tensor* X, int32_t mode, int32_t prec,
                                                   const double* Q, int32_t s, double* P, void* stream) {
    RBKI_TRY(validate_tensor(X));
    if (mode < 0 || mode >= X->order || s < 1 || s > 32)
        return set_error(RBKI_E_INVAL, "noalloc Krylov step: mode out of range or s not in [1, 32]");
    if (!Q || !P) return set_error(RBKI_E_INVAL, "noalloc Krylov step: Q/P NULL");
    const bool split = prec < 0;
    const int pr = split ? -prec : prec;
    if (pr != RBKI_PREC_BF16 && pr != RBKI_PREC_FP16)
        return set_error(RBKI_E_INVAL, "noalloc Krylov step: precision must be BF16 or FP16 (negative = split)");
    if ((pr == RBKI_PREC_BF16 && X->dtype != RBKI_BF16) || (pr == RBKI_PREC_FP16 && X->dtype != RBKI_F16))
        return set_error(RBKI_E_INVAL, "noalloc Krylov step: X must already be stored in the product precision");
    int64_t A = 1, C = 1;
    for (int k = 0; k < mode; ++k) A *= X->dims[k];
    for (int k = mode + 1; k < X->order; ++k) C *= X->dims[k];
    const View v{X->data, X->dtype, A, X->dims[mode], C};
    const int N = (int)rup(split ? 2 * s : s, 16);
    // the same kernel choice as rbki_krylov_product, so the results are bit-identical
    const bool kp = tc::krylov_supported(v, N);
    if (!kp && !tc::supported(v, tc::KRYLOV, N))
        return set_error(RBKI_E_UNSUPPORTED, "noalloc Krylov step: shape not supported by the tensor-core kernel");
    // scratch layout: error word | operand image | partial products (grid x I x N FP32)
    const size_t img_bytes = tc::image_bytes_skinny(v, N);
    const int grid = kp ? tc::krylov_grid(v) : tc::grid_size(v);
    const size_t part_bytes = (size_t)grid * (size_t)v.I * N * sizeof(float);
    const size_t off_img = 256, off_part = rup(off_img + img_bytes, 256);
    if (off_part + part_bytes > kScratchBytes)
        return set_error(RBKI_E_NOMEM, "noalloc Krylov step: needs more than the static scratch "
                                       "(RBKI_NOALLOC_SCRATCH_BYTES); use rbki_krylov_product");
    void* base = nullptr;
    RBKI_TRY(scratch_address(&base));
    char* b = static_cast<char*>(base);
    int* err = reinterpret_cast<int*>(b);
    void* img = b + off_img;
    float* part = reinterpret_cast<float*>(b + off_part);
    cudaStream_t st = (cudaStream_t)stream;
    RBKI_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    RBKI_TRY(tc::skinny_image(Q, s, v.I, s, N, split, X->dtype == RBKI_F16, img, st));
    if (kp)
        RBKI_TRY(tc::krylov_tc(v, N, s, split, img, part, err, st));
    else
        RBKI_TRY(tc::stream_tc(tc::KRYLOV, v, N, s, split, img, nullptr, part, nullptr, err, st));
    return tc::reduce_parts(part, grid, v.I, N, s, split, P, s, nullptr, 0, err, st);
}
