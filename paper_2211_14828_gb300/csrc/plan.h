// Host-side plan of one rBKI-TK call (sizes per mode + carved workspace pointers).
#pragma once

#include "kernels.h"

namespace rbki {

struct ModePlan {
    int n = 0;
    int64_t I = 0, A = 1, C = 1;   // X viewed as [A][I][C] for this mode
    int R = 0, S = 0, q = 0, b = 0;
    bool gram = false;             // b >= I: exact Gram path (reading c7)
    int nsplit = 1;
    // partial column sampling: A, C above describe the sampled unfolding Y ([kept][I][128]
    // or [kept*128][I][1]); A0, C0 the full view of X it is gathered from
    bool sampled = false;
    int64_t A0 = 1, C0 = 1, nunits = 0, kunits = 0;
    int32_t* units = nullptr;      // kept unit indices, ascending
    void* ysamp = nullptr;         // Y in the streamed dtype
    // workspace (device)
    double* Qall = nullptr;        // I x b, blocks Q_0..Q_q (ld b)
    double* Pall = nullptr;        // I x b, P_j = X X^T Q_j
    double* Y = nullptr;           // [A][S][C]: Omega, or X x_n Q_j^T
    double* part = nullptr;        // split partials
    double* small = nullptr;       // orthonormalisation scratch
    double* Z = nullptr;           // b x b
    double* evec = nullptr;        // b x b
    double* eval = nullptr;        // b
    double* syev_ws = nullptr;
    int32_t* kept = nullptr;
    // tensor-core path (mixed precision)
    bool tc = false;               // sketch + Krylov steps on tcgen05
    bool tc2 = false;              // tcgen05 too, Krylov step in two passes (Y = X^T Q to images,
                                   // then P = X Y): I_n too large for the fused step
    int N = 0;                     // MMA width (includes the lo half when split)
    void* qimg = nullptr;          // BF16 operand image of Q_j
    void* omg = nullptr;           // per-tile Omega images
    float* tpart = nullptr;        // [grid][I][N] partials (sized for the larger grid)
    int tgrid = 0;                 // grid of k_stream_tc (sketch, two-pass step)
    bool kp = false;               // fused Krylov step on the pipelined 64-column kernel
    int kgrid = 0;                 // its grid
    // Rayleigh-Ritz refinement of U (RBKI_FLAG_REFINE_FP32)
    bool refine = false;
    bool rtc = false, rkp = false; // refinement product on the tensor cores (split operand) / on
                                   // the pipelined kernel
    int rN = 0, rgrid = 0, rnsplit = 1;
    double* U0 = nullptr;          // I x R: the unrefined factor
    double* Pr = nullptr;          // I x R: X X^T U0
    double* Zr = nullptr;          // R x R
    double* Wr = nullptr;          // R x R eigenvectors of Zr
    double* lamr = nullptr;        // R refined Ritz values
    double* rsyev = nullptr;       // eigensolver scratch for R
    void* rimg = nullptr;          // split operand image of U0 (tensor cores)
    float* rpart = nullptr;        // [rgrid][I][rN] partials (tensor cores)
    double* rY = nullptr;          // [A][R][C] X x_n U0^T (CUDA cores)
    double* rsplit = nullptr;      // [rnsplit][I][R] partials (CUDA cores)
};

struct Plan {
    int N = 0, dtype = 0, prec = 0, stream_dtype = 0;
    bool mixed = false, stage = false, split = false;
    int64_t dims[RBKI_MAX_ORDER] = {0};
    int64_t numel = 0, ranks_numel = 0;
    int order[RBKI_MAX_ORDER] = {0};
    uint64_t seed = 0;
    uint32_t flags = 0;
    ModePlan mode[RBKI_MAX_ORDER];
    // workspace
    double* scal = nullptr;        // scalars + reduction partials
    char* xs = nullptr;            // staged low-precision copy of X
    double* tbuf[2] = {nullptr, nullptr};
    int32_t* err = nullptr;        // device error word (bounded waits)
    bool ttm_tc = false;           // first core TTM on tcgen05 (split factor, 2R <= 64)
    bool ttm_tc2 = false;          // ... as two plain passes (hi, then lo; 32 < R <= 64)
    int ttm_N = 0;
    void* ttm_img = nullptr;
    size_t ws_bytes = 0;
    // sequential truncation (RBKI_FLAG_SEQUENTIAL): step n works on Y_n = X x_1 U^(1)T ..
    // x_{n-1} U^(n-1)T through a plan of its own carved at the front of the workspace
    bool sequential = false;
    rbki_params prm{};
    void* ws_base = nullptr;
    void* ybuf[2] = {nullptr, nullptr};  // Y_1 .. Y_{N-1}, ping-pong (FP64, FP32 when mixed)
    int ydtype = 0;
    // bound at run time
    const void* xin = nullptr;
    const void* xstream = nullptr;
};

// TR-ALS (k_tr.cu)
struct TrPlan;
size_t tr_workspace_doubles_for(int N, const int64_t* core_dims, const int32_t* ranks);
rbki_status tr_run(int N, const int64_t* core_dims, const int32_t* ranks, const double* G, double g_norm2,
                   double* const* cores_dev, const double* const* cores_table_dev, int maxit, double tol,
                   double* ws, double* fits_host, int* sweeps, cudaStream_t st);
rbki_status tr_contract_cuda(const double* Z, const double* U, int r0, int64_t Rn, int r1, int64_t In, double* X,
                             cudaStream_t st);
size_t trsvd_workspace_doubles(int N, const int64_t* S, const int32_t* r);
rbki_status tr_svd_cuda(int N, const int64_t* S, const int32_t* r, const double* G, double* const* cores,
                        double* ws, double* fits, int nfits, cudaStream_t st);
rbki_status symmetrize_cuda(double* Z, int n, cudaStream_t st);

size_t dtype_size(int dt);
rbki_status validate_tensor(const rbki_tensor* X);
size_t host_io_bytes(const Plan& pl);
rbki_status make_plan(const rbki_tensor* X, const rbki_params* prm, Plan& pl);
void carve(Plan& pl, void* ws);    // ws == nullptr: only measures pl.ws_bytes
rbki_status step_plan(const Plan& pl, int n, const int64_t* cur, int dtype, Plan& sp);
// mode_streams: N streams for the concurrent per-mode chains (nullptr: the per-device pool)
rbki_status run_tucker(Plan& pl, const rbki_tucker_out* out, cudaStream_t st,
                       const cudaStream_t* mode_streams = nullptr);
rbki_status run_tucker_host_io(Plan& pl, const rbki_tensor* X, const rbki_tucker_out* out,
                               void* workspace, cudaStream_t st);

}  // namespace rbki
