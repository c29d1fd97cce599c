// RBKI_FLAG_HOST_IO: end-to-end call with X and the outputs in host memory.  The input is
// copied into the tail of the caller's workspace, the decomposition runs on the device and
// the outputs are copied back; the call returns after the stream has drained, or at once with
// RBKI_FLAG_ASYNC (calls on different streams then overlap their copies with computation).
#include "plan.h"

namespace rbki {

namespace {
struct HostIoLayout {
    size_t x_off, core_off, fac_off[RBKI_MAX_ORDER], eig_off[RBKI_MAX_ORDER], norms_off, info_off, q_off, total;
};

HostIoLayout layout(const Plan& pl) {
    HostIoLayout L{};
    size_t off = (pl.ws_bytes + 255) & ~(size_t)255;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        size_t r = off;
        off += bytes;
        return r;
    };
    L.x_off = take((size_t)pl.numel * dtype_size(pl.dtype));
    L.core_off = take((size_t)pl.ranks_numel * 8);
    for (int n = 0; n < pl.N; ++n) {
        L.fac_off[n] = take((size_t)pl.dims[n] * pl.mode[n].R * 8);
        L.eig_off[n] = take((size_t)pl.mode[n].R * 8);
    }
    L.norms_off = take(2 * 8);
    L.info_off = take((2 * RBKI_MAX_ORDER + 1) * 4);
    L.q_off = take(RBKI_MAX_ORDER * 4);
    L.total = off - pl.ws_bytes + 256;
    return L;
}
}  // namespace

size_t host_io_bytes(const Plan& pl) { return layout(pl).total; }

rbki_status run_tucker_host_io(Plan& pl, const rbki_tensor* X, const rbki_tucker_out* out,
                               void* workspace, cudaStream_t st) {
    HostIoLayout L = layout(pl);
    char* base = (char*)workspace;
    void* xdev = base + L.x_off;
    RBKI_CUDA_TRY(cudaMemcpyAsync(xdev, X->data, (size_t)pl.numel * dtype_size(pl.dtype),
                                  cudaMemcpyHostToDevice, st));
    rbki_tucker_out dout{};
    dout.core = (double*)(base + L.core_off);
    for (int n = 0; n < pl.N; ++n) {
        dout.factors[n] = (double*)(base + L.fac_off[n]);
        dout.eigvals[n] = (double*)(base + L.eig_off[n]);
    }
    dout.norms = (double*)(base + L.norms_off);
    dout.info = (int32_t*)(base + L.info_off);
    dout.q_used = (int32_t*)(base + L.q_off);
    pl.xin = xdev;
    RBKI_TRY(run_tucker(pl, &dout, st));
    RBKI_CUDA_TRY(cudaMemcpyAsync(out->core, dout.core, (size_t)pl.ranks_numel * 8,
                                  cudaMemcpyDeviceToHost, st));
    for (int n = 0; n < pl.N; ++n) {
        RBKI_CUDA_TRY(cudaMemcpyAsync(out->factors[n], dout.factors[n],
                                      (size_t)pl.dims[n] * pl.mode[n].R * 8, cudaMemcpyDeviceToHost, st));
        if (out->eigvals[n])
            RBKI_CUDA_TRY(cudaMemcpyAsync(out->eigvals[n], dout.eigvals[n], (size_t)pl.mode[n].R * 8,
                                          cudaMemcpyDeviceToHost, st));
    }
    if (out->norms)
        RBKI_CUDA_TRY(cudaMemcpyAsync(out->norms, dout.norms, 16, cudaMemcpyDeviceToHost, st));
    if (out->info)
        RBKI_CUDA_TRY(cudaMemcpyAsync(out->info, dout.info, (2 * pl.N + 1) * 4, cudaMemcpyDeviceToHost, st));
    if (out->q_used)
        RBKI_CUDA_TRY(cudaMemcpyAsync(out->q_used, dout.q_used, pl.N * 4, cudaMemcpyDeviceToHost, st));
    if (!(pl.flags & RBKI_FLAG_ASYNC)) RBKI_CUDA_TRY(cudaStreamSynchronize(st));
    return RBKI_OK;
}

}  // namespace rbki
