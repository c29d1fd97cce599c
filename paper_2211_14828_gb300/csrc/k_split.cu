// Divide-and-conquer along one mode (Sec. 4.1.2): copy the consecutive parts of X along
// mode n into dense tensors.  Part k covers [floor(k I / K), floor((k+1) I / K)).  X is
// viewed as [A][I][C]; every (a, i) row of C elements is contiguous in both X and the part,
// and is copied in 16-byte vectors when C * elem is a multiple of 16.
#include "plan.h"

namespace rbki {
namespace {

template <typename W, typename IT>
__global__ void __launch_bounds__(256) k_split_rows(const W* __restrict__ x, IT I, IT lo, IT len, IT rw,
                                                    int64_t n, W* __restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const IT row = (IT)(e / rw), v = (IT)(e - (int64_t)row * rw);
        const IT a = row / len, il = row - a * len;
        y[e] = x[((int64_t)a * I + lo + il) * rw + v];
    }
}

template <typename W>
rbki_status launch_split(const void* x, int64_t A, int64_t I, int64_t lo, int64_t len, int64_t rw, void* y,
                         cudaStream_t st) {
    const int64_t n = A * len * rw;
    if (n == 0) return RBKI_OK;
    const unsigned grid = (unsigned)std::min<int64_t>(cdiv(n, 256), 152 * 8);
    if (A * len < 0x7fffffffLL && I < 0x7fffffffLL && rw < 0x7fffffffLL)
        k_split_rows<W, uint32_t><<<grid, 256, 0, st>>>((const W*)x, (uint32_t)I, (uint32_t)lo, (uint32_t)len,
                                                        (uint32_t)rw, n, (W*)y);
    else
        k_split_rows<W, int64_t><<<grid, 256, 0, st>>>((const W*)x, I, lo, len, rw, n, (W*)y);
    RBKI_LAUNCH_CHECK("k_split_rows");
    return RBKI_OK;
}

}  // namespace

rbki_status split_mode_cuda(const void* x, int dtype, int64_t A, int64_t I, int64_t C, int parts, void* const* dst,
                            cudaStream_t st) {
    const int64_t es = (int64_t)dtype_size(dtype);
    bool vec = (C * es) % 16 == 0 && (uintptr_t)x % 16 == 0;
    for (int k = 0; k < parts; ++k) vec = vec && (uintptr_t)dst[k] % 16 == 0;
    for (int k = 0; k < parts; ++k) {
        const int64_t lo = (int64_t)k * I / parts, hi = (int64_t)(k + 1) * I / parts;
        if (vec) {
            RBKI_TRY(launch_split<uint4>(x, A, I, lo, hi - lo, C * es / 16, dst[k], st));
        } else if (es == 2) {
            RBKI_TRY(launch_split<uint16_t>(x, A, I, lo, hi - lo, C, dst[k], st));
        } else if (es == 4) {
            RBKI_TRY(launch_split<uint32_t>(x, A, I, lo, hi - lo, C, dst[k], st));
        } else {
            RBKI_TRY(launch_split<uint64_t>(x, A, I, lo, hi - lo, C, dst[k], st));
        }
    }
    return RBKI_OK;
}

}  // namespace rbki
