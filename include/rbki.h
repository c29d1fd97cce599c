/*
 * rbki.h - C ABI of librbki.so: rBKI-TK Tucker decomposition and rBKI-TK-TR
 * hierarchical tensor-ring decomposition on one GB300 GPU (sm_103a).
 *
 * Method: Qiu, Sun, Zhou, Zhao, "Towards Efficient and Accurate Approximation:
 * Tensor Decomposition Based on Randomized Block Krylov Iteration", arXiv 2211.14828.
 *   Algorithm 1  tensor sketching by randomized block Krylov iteration (Eq. BKspace)
 *   Algorithm 2  rBKI-TK (randomized HOSVD with rBKI subspaces, Remark 1, Eq. tensorsketch)
 *   Algorithm 3  rBKI-TK-TR (TR-ALS on the rBKI-TK core, contraction with the factors)
 *
 * Conventions (all entry points):
 *   - Tensors are dense, C-order (last index fastest).  Mode n is 0-based here
 *     (the paper's mode n+1).  The mode-n unfolding X_(n) is never materialised;
 *     its column index is the C-order linear index of the remaining indices.
 *   - Every pointer in a struct or argument is DEVICE memory on the current CUDA
 *     device unless RBKI_FLAG_HOST_IO is set (then X and the outputs are host
 *     memory, preferably pinned, and the call copies them itself and returns
 *     after the results are back on the host).
 *   - The caller owns every buffer, including the workspace; the library
 *     allocates no device memory in these calls.  Buffers must stay alive until
 *     the work queued on `stream` has finished (or, for the server, until a
 *     terminal rbki_poll result).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is queued on it; rbki_tucker / rbki_htr return without synchronising
 *     (except with RBKI_FLAG_HOST_IO).
 *   - Errors never abort the process: a negative rbki_status is returned and
 *     nothing is written to the outputs if validation fails.  A CUDA launch
 *     error is reported as RBKI_E_CUDA; rbki_last_error() gives its text.
 *   - Outputs are FP64 whatever the input dtype and product precision.
 */
#ifndef RBKI_H
#define RBKI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RBKI_MAX_ORDER 8

typedef int32_t rbki_status;
enum {
    RBKI_OK = 0,
    RBKI_PENDING = 1,        /* server: request not finished */
    RBKI_W_DEFLATED = 2,     /* warning: a Krylov block lost directions (reading c3) */
    RBKI_E_INVAL = -1,       /* invalid argument (shape, rank, pointer, size) */
    RBKI_E_NOMEM = -2,       /* workspace too small / server budget exceeded */
    RBKI_E_CUDA = -3,        /* CUDA runtime or launch error */
    RBKI_E_UNSUPPORTED = -4, /* valid request outside what this build implements */
    RBKI_E_TIMEOUT = -5,     /* a bounded device or host wait ran out */
    RBKI_E_BUSY = -6,        /* server: no slot / queue full */
    RBKI_E_CANCELLED = -7,   /* server: request cancelled */
    RBKI_E_NOTFOUND = -8     /* server: unknown ticket */
};

/* storage dtype of the input tensor */
enum { RBKI_F64 = 0, RBKI_F32 = 1, RBKI_BF16 = 2, RBKI_F16 = 3 };

/* precision of the X-streaming products (sketch, Krylov step, Gram, first TTM).
 * Orthonormalisation, the small eigensolve and all outputs are FP64 in every mode. */
enum { RBKI_PREC_FP64 = 0, RBKI_PREC_BF16 = 1, RBKI_PREC_FP16 = 2 };

/* rbki_params.flags */
enum {
    RBKI_FLAG_HOST_IO = 1u,        /* X and outputs in host memory (end-to-end call) */
    RBKI_FLAG_SPLIT = 2u,          /* mixed path: carry the skinny operands (Q, Y, Omega, U) as
                                      hi + lo BF16 pairs: ~FP32-accurate products, 2x MMA work */
    RBKI_FLAG_SERIAL_MODES = 4u,   /* run modes one after another on `stream`, each through the
                                      per-mode kernels.  Without it, two or more Krylov-path modes
                                      with b <= 192 run in lockstep (each FP64 stage one batched
                                      launch for all modes), with the same results bit for bit;
                                      otherwise each mode runs on a stream of its own */
    RBKI_FLAG_SEQUENTIAL = 8u,     /* sequentially truncated reading of Algorithm 2 (ST-HOSVD):
                                      mode n is sketched on Y_n = X x_1 U^(1)T .. x_{n-1} U^(n-1)T,
                                      modes in the order 1..N; the default (HOSVD reading)
                                      sketches every mode on X itself */
    RBKI_FLAG_POWER = 16u,         /* power-iteration baseline (Sec. 3.1 "P-iter", GRpi):
                                      Q_{j+1} = orth(X X^T Q_j) replaces the block instead of
                                      extending it; the basis is Q_q alone (width S_n); a mode
                                      takes the Gram path when S_n >= I_n */
    RBKI_FLAG_ASYNC = 128u,        /* with RBKI_FLAG_HOST_IO: return without waiting for the
                                      stream; the host outputs are valid once `stream` has
                                      completed, and X and the outputs must be pinned host memory
                                      (calls on different streams then overlap their copies with
                                      each other's computation) */
    RBKI_FLAG_TR_SVD = 64u,        /* rbki_htr: TR-SVD (Zhao et al. 2016) on the core instead of
                                      TR-ALS (the alternative Algorithm 3 step 3 names): fixed
                                      ranks, sequential truncated SVDs, the first splitting the
                                      rank product r_{N-1} r_0; tr_init is not read (may be
                                      NULL); fits[0] = the ring's fit to G, the rest NaN.
                                      Unfolding rows r_{n-1} S_n must be <= 256 */
    RBKI_FLAG_REFINE_FP32 = 256u,  /* Rayleigh-Ritz refinement of every Krylov-path factor: one
                                      more pass of width R, P = X_(n) X_(n)^T U with FP32-accurate
                                      products (the split hi + lo operand on the tensor cores, or
                                      FP32-accumulating CUDA cores when the shape does not fit),
                                      then Z_r = U^T P (FP64), its eigenvectors W and U <- U W,
                                      eigvals <- the refined Ritz values.  U keeps its span, so
                                      the core's norm and the reconstruction error do not change;
                                      the Ritz values and the individual factor columns lose the
                                      BF16 rounding of the Krylov products.  Not with
                                      RBKI_FLAG_ADAPTIVE_Q */
    RBKI_FLAG_ADAPTIVE_Q = 32u     /* adaptive Krylov depth: q is the bound; after block j the
                                      mode's fit F_j = 1 - sqrt(|X|^2 - sum of its R_n Ritz
                                      values)/|X| is evaluated, and the mode stops at the first
                                      j >= 1 with |F_j - F_{j-1}| <= q_tol (or at j = q).  The
                                      call then synchronises `stream` once per block.  Not with
                                      RBKI_FLAG_POWER, RBKI_FLAG_SEQUENTIAL or omega sampling */
};

typedef struct {
    int32_t order;                   /* N, 1..RBKI_MAX_ORDER */
    int32_t dtype;                   /* RBKI_F64 / RBKI_F32 / RBKI_BF16 / RBKI_F16 */
    int64_t dims[RBKI_MAX_ORDER];    /* I_1..I_N, each > 0 */
    const void* data;                /* C-order, 16-byte aligned */
} rbki_tensor;

/* Algorithm 2 inputs: multilinear rank R_n, oversampling p (S_n = min(R_n + p, I_n)),
 * Krylov depth q (K has q+1 blocks, Eq. BKspace), seed of the Gaussian sketches. */
typedef struct {
    int32_t ranks[RBKI_MAX_ORDER];   /* 1 <= R_n <= I_n */
    int32_t p;                       /* >= 0 */
    int32_t q;                       /* >= 0 */
    uint64_t seed;
    int32_t prec;                    /* RBKI_PREC_* */
    uint32_t flags;                  /* RBKI_FLAG_* */
    double omega;                    /* column sampling rate of the Krylov construction
                                        (Sec. 3.2 after Table 2, Fig. 5): 0 < omega < 1
                                        builds Krylov-path modes from ceil(omega U_n) of the
                                        U_n 128-column units of X_(n) (units with the
                                        smallest Philox4x32-10 keys, counter (u lo, u hi, n,
                                        0x53414D50), key = seed); Z = Q^T Y Y^T Q on the
                                        sampled Y; the core uses all of X.  <= 0 or >= 1:
                                        no sampling.  Must be finite. */
    double q_tol;                    /* RBKI_FLAG_ADAPTIVE_Q: fit-change threshold, >= 0
                                        (+inf: stop every mode at its first check, q = 1) */
} rbki_params;

/* Algorithm 2 outputs (caller-owned). */
typedef struct {
    double* core;                    /* R_1 x ... x R_N, C-order (required) */
    double* factors[RBKI_MAX_ORDER]; /* U^(n): I_n x R_n row-major, orthonormal columns,
                                        descending Ritz values, largest-|.| entry of each
                                        column positive (required) */
    double* eigvals[RBKI_MAX_ORDER]; /* optional (NULL): leading R_n eigenvalues of Z^(n) */
    double* norms;                   /* optional: [0] = |X|_F^2, [1] = |G|_F^2; the
                                        reconstruction error is |X|^2 - |G|^2 */
    int32_t* info;                   /* optional, 2N+1 ints: [n] = kept Krylov width of mode n,
                                        [N+n] = path (0 Krylov, 1 Gram = exact T-SVD mode),
                                        [2N] = device error flags (nonzero: a bounded wait inside
                                        a kernel expired; the results are not valid) */
    int32_t* q_used;                 /* optional, N ints: Krylov depth used per mode (q, or
                                        the adaptive choice; 0 on the Gram path) */
} rbki_tucker_out;

/* Bytes of device workspace rbki_tucker needs for this problem. */
rbki_status rbki_tucker_workspace(const rbki_tensor* X, const rbki_params* prm, size_t* bytes);

/* rBKI-TK, Algorithm 2 (with Algorithm 1 per mode), HOSVD reading: every mode sketches
 * the original X; G = X x_1 U^(1)T ... x_N U^(N)T (Eq. tensorsketch).
 * Per mode: S = min(R+p, I), b = S(q+1); b >= I uses the Gram path (Z = X_(n) X_(n)^T,
 * the exact truncated-HOSVD factor); otherwise W = X_(n) Omega, Q_0 = orth(W),
 * Q_{j+1} = orth(X_(n) X_(n)^T Q_j) against all earlier blocks, Z = Q^T X X^T Q,
 * U = Q * leading eigenvectors of Z.  Omega's entries are the Philox4x32-10 +
 * Box-Muller Gaussians keyed by (seed, n, column, s).
 * RBKI_FLAG_SEQUENTIAL: the sequentially truncated reading - the same per-mode steps on
 * Y_n (dims R_1..R_{n-1}, I_n..I_N; Omega keyed by Y_n's unfolding columns), modes taken in
 * the order 1..N, Y_{n+1} = Y_n x_n U^(n)T, G = Y_{N+1}.  Works with every other flag and
 * with rbki_htr and the server; the workspace adds two buffers of the largest Y_n. */
rbki_status rbki_tucker(const rbki_tensor* X, const rbki_params* prm, void* workspace,
                        size_t workspace_bytes, const rbki_tucker_out* out, void* stream);

/* ---- batches and divide-and-conquer (Sec. 4.1.2) ----------------------------------- */
/* Workspace of a batch: the items' workspaces one after another (256-byte aligned). */
rbki_status rbki_tucker_batch_workspace(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                                        size_t* bytes);
/* `count` independent rBKI-TK decompositions (arrays X[count], prm[count], out[count];
 * device buffers, RBKI_FLAG_HOST_IO refused) run concurrently: item k on its own stream
 * (forked from and joined back to `stream`), with its own mode streams.  Results equal
 * the items' rbki_tucker calls bit for bit. */
rbki_status rbki_tucker_batch(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                              void* workspace, size_t workspace_bytes, const rbki_tucker_out* out,
                              void* stream);
/* ---- batched small decompositions (continuous batching pattern) --------------------- */
/* Workspace of rbki_tucker_batched for these items (bytes, 256-byte aligned pieces). */
rbki_status rbki_tucker_batched_workspace(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                                          size_t* bytes);
/* `count` independent rBKI-TK decompositions (Algorithm 2, HOSVD reading, the same outputs
 * as rbki_tucker) run as ONE wave on `stream`: every stage of Algorithms 1-2 is one launch
 * for all modes of all items (about 100 launches for a wave of q <= 3 requests, whatever its
 * size), so many small requests cost what one costs in launches.
 *   - X is read once per mode (I_n <= 256): one pass forms X_(n) X_(n)^T and, on Krylov-path
 *     modes, the sketch W = X_(n) Omega (Omega as in rbki_tucker); the Krylov products are
 *     P_j = (X_(n) X_(n)^T) Q_j in FP64 - the Krylov space of Eq. BKspace, the product
 *     associated the other way.  X products are FP32 products of the BF16/FP16 value of each
 *     entry (X rounded as read when stored wider), FP32 Omega, FP32 accumulation within a
 *     unit of 32-column steps, FP64 across units, fixed order.  The core's mode products
 *     likewise (FP32 intermediates).
 *   - Orthonormalisation, Z = Q^T P, the eigensolver and U = Q U~ in FP64 with the kernels
 *     of rbki_tucker (their batched forms: the same per-item arithmetic).
 * Each item's result depends only on the item (and the work-granularity table, see
 * rbki_wave_autotune), not on the other items of the wave.  Requires: prec BF16 or FP16,
 * flags 0 or RBKI_FLAG_SERIAL_MODES (no effect here), no column sampling, order >= 2,
 * every I_n <= 256, R_n + p <= 64, the eigenproblem (S(q+1), or I_n on the Gram path)
 * <= 192, fewer than 2^31 entries; otherwise RBKI_E_UNSUPPORTED.  Device buffers only;
 * outputs as rbki_tucker (info[2N] is always 0: the wave's kernels have no device waits). */
rbki_status rbki_tucker_batched(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                                void* workspace, size_t workspace_bytes, const rbki_tucker_out* out,
                                void* stream);
/* A wave captured once as a CUDA graph and replayed: for repeated batches of the same shapes
 * in the same buffers (fixed-shape request slots, frames of a stream).  _create validates
 * like rbki_tucker_batched, runs the wave once on `stream` (valid outputs), then captures its
 * launches on a private stream; X, prm, workspace and out are bound into the plan (their
 * pointers and shapes), so the caller refills X in place and calls _launch: one graph launch
 * per batch, bitwise the results of rbki_tucker_batched on the same data.  rbki_kernel_launches
 * counts a replay's kernel nodes. */
typedef struct rbki_batched_plan rbki_batched_plan;
rbki_status rbki_batched_plan_create(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                                     void* workspace, size_t workspace_bytes, const rbki_tucker_out* out,
                                     void* stream, rbki_batched_plan** plan);
rbki_status rbki_batched_plan_launch(rbki_batched_plan* plan, void* stream);
rbki_status rbki_batched_plan_destroy(rbki_batched_plan* plan);
/* Work-granularity table of rbki_tucker_batched: steps of its two work-queue kernels per CTA
 * (kind 0: the Gram pass, 32-column steps; kind 1: the core's mode products, 64-column
 * tiles) for each I_n bucket b (I_n in (32b, 32(b+1)], b = 0..7).  The summation order of an
 * item depends on these values, so results are reproducible bit for bit under one table.
 * rbki_wave_autotune times the candidates {2, 4, 8, 16, 32, 64} on a synthetic batch
 * (48 items of 128 x I x 128 BF16) on `stream` and keeps the fastest when it beats the
 * default by at least 5% (about a second; needs
 * ~500 MB of device memory for its own buffers); _save / _load write and read the table
 * as text ("<gram|ttm> <b> <steps>" lines), _reset restores the defaults. */
rbki_status rbki_wave_autotune(void* stream);
rbki_status rbki_wave_tune_get(int32_t kind, int32_t bucket, int32_t* steps);
rbki_status rbki_wave_tune_reset(void);
rbki_status rbki_wave_tune_save(const char* path);
rbki_status rbki_wave_tune_load(const char* path);
/* Divide-and-conquer split: dst[k] (device, dense C-order, dims of X with I_mode replaced by
 * hi_k - lo_k) = X restricted to mode indices [lo_k, hi_k), lo_k = floor(k I_mode / parts),
 * hi_k = floor((k+1) I_mode / parts); 1 <= parts <= I_mode.  Same dtype as X. */
rbki_status rbki_split_mode(const rbki_tensor* X, int32_t mode, int32_t parts, void* const* dst,
                            void* stream);

/* Bytes of device workspace rbki_htr needs. */
rbki_status rbki_htr_workspace(const rbki_tensor* X, const rbki_params* tk,
                               const int32_t* tr_ranks, size_t* bytes);

/* rBKI-TK-TR, Algorithm 3.  tr_ranks[n] = r_n (r_0 = r_N, ring closure; Eq. TR).
 * tr_init[n]: device, initial TR core of the Tucker core, r_{n-1} x R_n x r_n (C-order).
 * TR-ALS sweeps cores 0..N-1, exact least squares per core (normal equations, FP64),
 * stops after tr_maxit sweeps or when |Fit_t - Fit_{t-1}| <= tr_tol (Sec. 4 rule).
 * tr_cores[n]: device output r_{n-1} x I_n x r_n = G_n x_2 U^(n) (Algorithm 3 step 4).
 * fits: optional device output, tr_maxit doubles (fit per sweep, NaN after the stop);
 * tucker_out may be NULL or receive the intermediate Tucker result. */
rbki_status rbki_htr(const rbki_tensor* X, const rbki_params* tk, const int32_t* tr_ranks,
                     const double* const* tr_init, int32_t tr_maxit, double tr_tol,
                     double* const* tr_cores, double* fits, const rbki_tucker_out* tucker_out,
                     void* workspace, size_t workspace_bytes, void* stream);

/* ---- served stream (continuous batching with device-memory admission) ------------- */
typedef struct rbki_server rbki_server;

/* Creates a server on `device` that admits requests while their workspace fits in
 * mem_budget bytes.  Requests rbki_tucker_batched supports are served in waves
 * (rbki_server_create_ex with RBKI_SERVER_WAVE_THREADS workers, waves of at most
 * RBKI_SERVER_WAVE_MAX requests); every other request runs on one of max_slots slots
 * (rbki_tucker each).  The server allocates its own device memory pool of mem_budget bytes
 * once, here. */
#define RBKI_SERVER_WAVE_THREADS 4
#define RBKI_SERVER_WAVE_MAX 32
rbki_status rbki_server_create(int32_t device, size_t mem_budget, int32_t max_slots,
                               rbki_server** out);
/* As rbki_server_create with the batched path configured: wave_threads host workers (0..8;
 * 0 = every request on the slots) each run waves of up to wave_max (1..1024) requests: the
 * longest FIFO prefix of the waiting batched-path requests whose workspaces fit in the pool
 * together.  A wave item's outputs are bitwise those of rbki_tucker_batched on that request
 * alone; a slot request's those of rbki_tucker. */
rbki_status rbki_server_create_ex(int32_t device, size_t mem_budget, int32_t max_slots,
                                  int32_t wave_threads, int32_t wave_max, rbki_server** out);
/* Queues one rBKI-TK request (device buffers; RBKI_FLAG_HOST_IO is refused).  X and out
 * must stay valid until a terminal poll.  The server runs requests on its own streams: work
 * already queued on `after_stream` (a cudaStream_t as void*, typically the stream that
 * produced X) is waited for before the request's first kernel - an event is recorded on
 * it here.  NULL means "nothing to wait for": pass it only when X is complete on the device
 * (e.g. after a synchronize); the legacy default stream is passed as cudaStreamLegacy.
 * Refused at submission: invalid arguments (RBKI_E_INVAL), a workspace larger than the
 * whole budget (RBKI_E_NOMEM), a server shutting down (RBKI_E_BUSY). */
rbki_status rbki_submit(rbki_server* s, const rbki_tensor* X, const rbki_params* prm,
                        const rbki_tucker_out* out, void* after_stream, uint64_t* ticket);
/* Non-blocking.  *result = RBKI_PENDING while running, else the request's final status;
 * *latency_s = completion - submission (seconds) once finished. */
rbki_status rbki_poll(rbki_server* s, uint64_t ticket, rbki_status* result, double* latency_s);
rbki_status rbki_cancel(rbki_server* s, uint64_t ticket);
/* Waits (bounded by timeout_s) until every admitted request has finished. */
rbki_status rbki_server_drain(rbki_server* s, double timeout_s);
rbki_status rbki_server_destroy(rbki_server* s);

/* ---- step-level entry points (used by the parity tests) --------------------------- */

/* Krylov step of Algorithm 1 / Eq. BKspace on mode n: P = X_(n) (X_(n)^T Q),
 * Q: I_n x s row-major FP64 (device), P: I_n x s row-major FP64 (device).
 * prec = RBKI_PREC_*; a negative value -RBKI_PREC_BF16 / -RBKI_PREC_FP16 selects the split
 * (hi + lo) operand variant.  BF16/FP16 run on the tensor-core kernels when the shape allows
 * (contiguous extent a multiple of 8; I_n <= 640 at s <= 32, I_n <= 512 with the split
 * variant; larger I_n with plain operands in two passes), else on CUDA cores.  If a bounded
 * wait inside a tensor-core kernel expires, every entry of P is NaN. */
rbki_status rbki_krylov_product(const rbki_tensor* X, int32_t mode, int32_t prec,
                                const double* Q, int32_t s, double* P,
                                void* workspace, size_t workspace_bytes, void* stream);
rbki_status rbki_krylov_product_workspace(const rbki_tensor* X, int32_t mode, int32_t prec,
                                          int32_t s, size_t* bytes);

/* Size of the device array that rbki_krylov_product_noalloc uses instead of a workspace. */
#define RBKI_NOALLOC_SCRATCH_BYTES (20u * 1024u * 1024u)

/* The Krylov step of rbki_krylov_product, for callers that cannot allocate device memory:
 * some host applications give all device memory to their own allocator up front, or call
 * this step from code where cudaMalloc is not allowed or too slow, so they cannot pass a
 * workspace.  This variant takes none: its scratch (BF16 operand image, per-CTA partial
 * products, error word) is a fixed array of RBKI_NOALLOC_SCRATCH_BYTES compiled into the
 * library, which every GPU that loads the library keeps until the process exits.  The
 * paper has no counterpart of this entry point.
 *   X: device, already stored in the product precision (RBKI_BF16 for RBKI_PREC_BF16,
 *      RBKI_F16 for RBKI_PREC_FP16); prec < 0 selects the split (hi + lo) variant.
 *   Q: I_n x s row-major FP64 (device), 1 <= s <= 32;  P: I_n x s row-major FP64 (device).
 * Scratch needed: 256 + the operand image (ceil(I_n/128) 128 N 2 bytes) + the partial
 * products (G I_n N 4 bytes), with N = s (2s when split) rounded up to 16 and G = the kernel's
 * grid, at most the GPU's SM count.  The largest shape the kernel takes (I_n = 512, split,
 * s = 32: N = 64) needs 19.99 MB at G = 152 (GB300), inside the array; GPUs with more than 159
 * SMs get RBKI_E_NOMEM for it.  Shapes the tensor-core kernels do not take (contiguous extent
 * not a multiple of 8; I_n beyond the fused step's limits) return RBKI_E_UNSUPPORTED.  It
 * allocates nothing.  Results are bit-identical to rbki_krylov_product's (same kernels).
 * If a bounded wait inside the kernel expires, every entry of P is NaN.
 * All calls share the array: calls that overlap on the GPU race on it and must be ordered
 * by the caller.  Each call looks up the array's address on the current device
 * (cudaGetSymbolAddress, nothing cached); the first call on a device may load the library's
 * device code, so make it before any stream capture. */
rbki_status rbki_krylov_product_noalloc(const rbki_tensor* X, int32_t mode, int32_t prec,
                                        const double* Q, int32_t s, double* P, void* stream);

/* Diagnostics of the bounded device waits (no counterpart in the paper): the Krylov step of
 * rbki_krylov_product (BF16/FP16 tensor-core shapes only, else RBKI_E_UNSUPPORTED) with a
 * planted stall - the MMA-issuing thread first waits on a barrier that nothing arrives at,
 * giving up after wait_us microseconds - so the kernel's abort path runs: every role leaves its
 * loop, the copies and MMAs already issued are waited for (bounded), tensor memory is freed
 * and the error word is set.  Nothing faults or hangs.  Synchronises `stream`, then returns
 * RBKI_E_TIMEOUT when the error word is set (the expected outcome; P is then all NaN) or
 * RBKI_OK.  Workspace as rbki_krylov_product_workspace. */
rbki_status rbki_diag_krylov_stall(const rbki_tensor* X, int32_t mode, int32_t prec,
                                   const double* Q, int32_t s, double* P,
                                   void* workspace, size_t workspace_bytes,
                                   uint32_t wait_us, void* stream);

/* The same for the tensor-core Gram pass of rbki_tucker_batched: the wave runs with every
 * Gram-pass CTA first waiting on a barrier that nothing completes, giving up after wait_us
 * (1 .. 2e6) microseconds; the CTA then drains its MMAs, frees tensor memory, writes no
 * partials and sets its request's error word (info[2N]).  Synchronises `stream` and returns
 * RBKI_E_TIMEOUT when any item's error word is set (the expected outcome when an item takes
 * the tensor-core pass; the outputs are then not valid), else RBKI_OK.  Arguments otherwise
 * as rbki_tucker_batched. */
rbki_status rbki_diag_batched_stall(int32_t count, const rbki_tensor* X, const rbki_params* prm,
                                    void* workspace, size_t workspace_bytes, const rbki_tucker_out* out,
                                    uint32_t wait_us, void* stream);

/* Algorithm 1 for one mode: the orthonormal Krylov basis Q = [Q_0..Q_q] (I_n x b,
 * row-major FP64, deflated columns are zero), b = S(q+1), S = min(R_n+p, I_n). */
rbki_status rbki_mode_basis(const rbki_tensor* X, const rbki_params* prm, int32_t mode,
                            double* Q, void* workspace, size_t workspace_bytes, void* stream);

/* Partial column sampling, the choice of units alone: units[0..kept-1] (device int32) =
 * the `kept` of n_units units with the smallest keys of rbki_params.omega's rule for mode
 * `mode`, ascending.  1 <= kept <= n_units < 2^31, else RBKI_E_INVAL. */
rbki_status rbki_sample_units(uint64_t seed, int32_t mode, int64_t n_units, int64_t kept,
                              int32_t* units, void* stream);

/* Symmetric eigensolver used for Algorithm 2 step 4: A (n x n, FP64, symmetric) ->
 * eigenvalues descending in w (n) and eigenvectors as columns of V (n x n row-major). */
rbki_status rbki_syev(const double* A, int32_t n, double* w, double* V,
                      void* workspace, size_t workspace_bytes, void* stream);
rbki_status rbki_syev_workspace(int32_t n, size_t* bytes);

/* ---- diagnostics -------------------------------------------------------------------- */
/* Kernel classes timed by the profiling hook. */
enum { RBKI_PROF_KRYLOV = 0, RBKI_PROF_SKETCH = 1, RBKI_PROF_GRAM = 2, RBKI_PROF_TTM = 3,
       RBKI_PROF_STAGE = 4, RBKI_PROF_SAMPLE = 5, RBKI_PROF_COUNT = 6 };
/* When on, each streaming launch (Krylov step, sketch, Gram pass, first TTM, staging) is
 * bracketed by CUDA events recorded on the stream it runs on.  Off by default. */
void rbki_profile_enable(int32_t on);
/* Waits for the recorded events and returns, for class `cls`, the number of timed launches
 * and their summed duration in milliseconds since the last reset. */
rbki_status rbki_profile_read(int32_t cls, uint64_t* count, double* total_ms);
void rbki_profile_reset(void);

const char* rbki_status_str(rbki_status s);
const char* rbki_last_error(void);
/* Number of kernels this library has launched in this process (diagnostics). */
uint64_t rbki_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* RBKI_H */
