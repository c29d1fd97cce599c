// C ABI of librbki: argument validation, planning, workspace carving and the per-mode
// pipeline of Algorithms 1-2 (rBKI-TK) on the caller's stream, with its variants: the
// sequentially truncated reading (step plans on the contracted tensor), partial column
// sampling (Sec. 3.2), the power-iteration baseline and the adaptive Krylov depth; batches
// of independent decompositions and the divide-and-conquer split; Algorithm 3 (TR-ALS or
// TR-SVD on the core) and the step-level entry points the tests call.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "plan.h"
#include "tc.h"

namespace rbki {

static std::atomic<uint64_t> g_launches{0};
static thread_local std::string g_err;

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void drop_launches(uint64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

rbki_status set_cuda_error(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return RBKI_E_CUDA;
}

rbki_status set_error(rbki_status s, const char* msg) {
    g_err = msg;
    return s;
}

// ---- profiling hook: CUDA events around streaming launches ----
struct ProfRec { int cls; cudaEvent_t a, b; };
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static size_t g_prof_used = 0;

int prof_begin(int cls, cudaStream_t st) {
    if (!g_prof_on) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_used == g_prof.size()) {
        ProfRec r{cls, nullptr, nullptr};
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return -1;
        g_prof.push_back(r);
    }
    int tok = (int)g_prof_used++;
    g_prof[tok].cls = cls;
    cudaEventRecord(g_prof[tok].a, st);
    return tok;
}

void prof_end(int tok, cudaStream_t st) {
    if (tok < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof[tok].b, st);
}

size_t dtype_size(int dt) {
    switch (dt) {
        case RBKI_F64: return 8;
        case RBKI_F32: return 4;
        case RBKI_BF16: return 2;
        case RBKI_F16: return 2;
        default: return 0;
    }
}

// ---------------------------------------------------------------------------------
// validation + plan
// ---------------------------------------------------------------------------------
rbki_status validate_tensor(const rbki_tensor* X) {
    if (!X) return set_error(RBKI_E_INVAL, "X is NULL");
    if (X->order < 1 || X->order > RBKI_MAX_ORDER) return set_error(RBKI_E_INVAL, "order out of range");
    if (dtype_size(X->dtype) == 0) return set_error(RBKI_E_INVAL, "unknown dtype");
    for (int n = 0; n < X->order; ++n)
        if (X->dims[n] <= 0) return set_error(RBKI_E_INVAL, "dims must be positive");
    if ((uintptr_t)X->data % 16) return set_error(RBKI_E_INVAL, "X->data must be 16-byte aligned");
    return RBKI_OK;
}

rbki_status validate_params(const rbki_tensor* X, const rbki_params* prm) {
    if (!prm) return set_error(RBKI_E_INVAL, "params is NULL");
    if (prm->p < 0 || prm->q < 0) return set_error(RBKI_E_INVAL, "p and q must be >= 0");
    if (prm->prec != RBKI_PREC_FP64 && prm->prec != RBKI_PREC_BF16 && prm->prec != RBKI_PREC_FP16)
        return set_error(RBKI_E_INVAL, "unknown precision");
    if (!std::isfinite(prm->omega)) return set_error(RBKI_E_INVAL, "omega must be finite");
    if (prm->flags & RBKI_FLAG_ADAPTIVE_Q) {
        // +inf is allowed: every mode then stops at its first check (q = 1)
        if (std::isnan(prm->q_tol) || prm->q_tol < 0.0) return set_error(RBKI_E_INVAL, "q_tol must be >= 0");
        if (prm->flags & RBKI_FLAG_POWER)
            return set_error(RBKI_E_INVAL, "adaptive q applies to the block Krylov space, not power iteration");
        if (prm->flags & RBKI_FLAG_SEQUENTIAL)
            return set_error(RBKI_E_UNSUPPORTED, "adaptive q with the sequential reading");
        if (prm->omega > 0.0 && prm->omega < 1.0)
            return set_error(RBKI_E_UNSUPPORTED, "adaptive q with column sampling");
        if (prm->flags & RBKI_FLAG_REFINE_FP32)
            return set_error(RBKI_E_UNSUPPORTED, "refinement with adaptive q");
    }
    for (int n = 0; n < X->order; ++n) {
        if (prm->ranks[n] < 1 || prm->ranks[n] > X->dims[n])
            return set_error(RBKI_E_INVAL, "ranks must satisfy 1 <= R_n <= I_n");
    }
    return RBKI_OK;
}

rbki_status make_plan(const rbki_tensor* X, const rbki_params* prm, Plan& pl) {
    RBKI_TRY(validate_tensor(X));
    RBKI_TRY(validate_params(X, prm));
    pl = Plan();
    pl.N = X->order;
    pl.dtype = X->dtype;
    pl.prec = prm->prec;
    pl.numel = 1;
    for (int n = 0; n < pl.N; ++n) {
        pl.dims[n] = X->dims[n];
        pl.numel *= X->dims[n];
    }
    pl.mixed = prm->prec != RBKI_PREC_FP64;
    pl.split = pl.mixed && (prm->flags & RBKI_FLAG_SPLIT);
    pl.stream_dtype = pl.mixed ? (prm->prec == RBKI_PREC_BF16 ? RBKI_BF16 : RBKI_F16) : X->dtype;
    pl.stage = pl.mixed && X->dtype != pl.stream_dtype;
    for (int n = 0; n < pl.N; ++n) {
        ModePlan& m = pl.mode[n];
        m.n = n;
        m.I = pl.dims[n];
        m.A = 1;
        m.C = 1;
        for (int k = 0; k < n; ++k) m.A *= pl.dims[k];
        for (int k = n + 1; k < pl.N; ++k) m.C *= pl.dims[k];
        m.R = prm->ranks[n];
        m.S = (int)std::min<int64_t>(m.R + prm->p, m.I);
        m.q = prm->q;
        // power iteration keeps one block of width S (RBKI_FLAG_POWER)
        int64_t b = (prm->flags & RBKI_FLAG_POWER) ? (int64_t)m.S : (int64_t)m.S * (m.q + 1);
        m.gram = b >= m.I;
        m.b = m.gram ? (int)m.I : (int)b;
        if (m.gram && m.I > 256) return set_error(RBKI_E_UNSUPPORTED, "Gram path with I_n > 256");
        if (!m.gram && m.b > 256) return set_error(RBKI_E_UNSUPPORTED, "Krylov width S(q+1) > 256");
        if (!m.gram && m.S > 96) return set_error(RBKI_E_UNSUPPORTED, "sketch size > 96");
        // partial column sampling (Krylov-path modes, 0 < omega < 1): 128-column units
        if (!m.gram && prm->omega > 0.0 && prm->omega < 1.0) {
            m.sampled = true;
            m.A0 = m.A;
            m.C0 = m.C;
            m.nunits = m.C > 1 ? m.A * cdiv(m.C, 128) : cdiv(m.A, 128);
            if (m.nunits > 0x7fffffff) return set_error(RBKI_E_UNSUPPORTED, "too many sampling units");
            double k = std::ceil(prm->omega * (double)m.nunits);
            m.kunits = (int64_t)std::min(std::max(k, 1.0), (double)m.nunits);
            if (m.C0 > 1) {
                m.A = m.kunits;
                m.C = 128;
            } else {
                m.A = m.kunits * 128;
                m.C = 1;
            }
        }
    }
    // core chain order: largest shrink I_n / R_n first (ties -> lower mode)
    for (int n = 0; n < pl.N; ++n) pl.order[n] = n;
    std::stable_sort(pl.order, pl.order + pl.N, [&](int a, int b) {
        return (double)pl.dims[a] / prm->ranks[a] > (double)pl.dims[b] / prm->ranks[b];
    });
    pl.seed = prm->seed;
    pl.flags = prm->flags;
    pl.prm = *prm;
    pl.ranks_numel = 1;
    for (int n = 0; n < pl.N; ++n) pl.ranks_numel *= prm->ranks[n];
    pl.sequential = (prm->flags & RBKI_FLAG_SEQUENTIAL) != 0;
    if (pl.sequential) {
        // every step's plan must exist (modes already truncated take the Gram path on R_k)
        int64_t cur[RBKI_MAX_ORDER];
        for (int n = 0; n < pl.N; ++n) cur[n] = pl.dims[n];
        for (int n = 0; n < pl.N; ++n) {
            Plan sp;
            RBKI_TRY(step_plan(pl, n, cur, n == 0 ? pl.dtype : (pl.mixed ? RBKI_F32 : RBKI_F64), sp));
            cur[n] = pl.mode[n].R;
        }
    }
    return RBKI_OK;
}

// Plan of step n of the sequential reading: the tensor Y_n of dims `cur` (modes < n already
// truncated to R_k), the caller's parameters without the sequential flag.
rbki_status step_plan(const Plan& pl, int n, const int64_t* cur, int dtype, Plan& sp) {
    (void)n;
    rbki_tensor t{};
    t.order = pl.N;
    t.dtype = dtype;
    for (int k = 0; k < pl.N; ++k) t.dims[k] = cur[k];
    t.data = nullptr;
    rbki_params p = pl.prm;
    p.flags &= ~(uint32_t)RBKI_FLAG_SEQUENTIAL;
    return make_plan(&t, &p, sp);
}

// Workspace layout.  carve() with base == nullptr only measures.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base((char*)b) {}
    template <typename T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? (T*)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Sequential reading: the step plans share the front of the workspace (each carves from
// the base; the largest sets the size), then the two Y buffers, then the operand image of
// the first mode product when it runs on the tensor cores.
static void carve_sequential(Plan& pl, void* ws) {
    pl.ydtype = pl.mixed ? RBKI_F32 : RBKI_F64;
    int64_t cur[RBKI_MAX_ORDER];
    for (int n = 0; n < pl.N; ++n) cur[n] = pl.dims[n];
    size_t front = 0, ymax = 0;
    for (int n = 0; n < pl.N; ++n) {
        Plan sp;
        if (step_plan(pl, n, cur, n == 0 ? pl.dtype : pl.ydtype, sp) != RBKI_OK) continue;  // checked in make_plan
        carve(sp, nullptr);
        front = std::max(front, sp.ws_bytes);
        cur[n] = pl.mode[n].R;
        if (n < pl.N - 1) {
            size_t e = 1;
            for (int k = 0; k < pl.N; ++k) e *= (size_t)cur[k];
            ymax = std::max(ymax, e);
        }
    }
    Carver c(ws);
    c.take<char>(front);
    pl.ybuf[0] = c.take<char>(ymax * dtype_size(pl.ydtype));
    pl.ybuf[1] = c.take<char>(ymax * dtype_size(pl.ydtype));
    {
        const ModePlan& m = pl.mode[0];
        View v{nullptr, pl.stream_dtype, m.sampled ? m.A0 : m.A, m.I, m.sampled ? m.C0 : m.C};
        pl.ttm_N = (int)rup(2 * m.R, 16);
        pl.ttm_tc = pl.mixed && pl.N > 1 && m.R <= 32 && tc::supported(v, tc::TTM, pl.ttm_N);
        if (pl.ttm_tc) pl.ttm_img = c.take<char>(tc::image_bytes_skinny(v, pl.ttm_N));
    }
    pl.ws_bytes = c.off + 256;
    pl.ws_base = ws;
    pl.scal = nullptr;
    pl.err = nullptr;
    if (ws) {
        // the scalars and the error word sit at the same offsets in every step plan
        Plan sp;
        if (step_plan(pl, 0, pl.dims, pl.dtype, sp) == RBKI_OK) {
            carve(sp, ws);
            pl.scal = sp.scal;
            pl.err = sp.err;
        }
    }
}

void carve(Plan& pl, void* ws) {
    if (pl.sequential) {
        carve_sequential(pl, ws);
        return;
    }
    Carver c(ws);
    pl.scal = c.take<double>(4096);
    pl.err = c.take<int32_t>(64);
    if (pl.stage) pl.xs = c.take<char>((size_t)pl.numel * dtype_size(pl.stream_dtype));
    for (int n = 0; n < pl.N; ++n) {
        ModePlan& m = pl.mode[n];
        int64_t d = m.A * m.C;
        View v{nullptr, pl.stream_dtype, m.A, m.I, m.C};
        m.nsplit = contract_nsplit(v);
        m.Z = c.take<double>((size_t)m.b * m.b);
        m.evec = c.take<double>((size_t)m.b * m.b);
        m.eval = c.take<double>((size_t)m.b);
        m.syev_ws = c.take<double>(syev_scratch_doubles(m.b));
        m.kept = c.take<int32_t>(4);
        if (m.sampled) {
            m.units = c.take<int32_t>((size_t)m.kunits);
            m.ysamp = c.take<char>((size_t)m.A * m.I * m.C * dtype_size(pl.stream_dtype));
        }
        if (m.gram) {
            m.part = c.take<double>((size_t)m.nsplit * m.I * m.I);
        } else {
            m.Qall = c.take<double>((size_t)m.I * m.b);
            m.Pall = c.take<double>((size_t)m.I * m.b);
            m.part = c.take<double>((size_t)std::max<int64_t>((int64_t)m.nsplit * m.I * m.S,
                                                             (int64_t)atb_nchunks(m.I) * m.b * m.b));
            size_t orth = 0;
            for (int j = 0; j <= m.q; ++j)
                orth = std::max(orth, orth_scratch_doubles(m.I, j * m.S, m.S));
            m.small = c.take<double>(orth);
            m.N = (int)rup(pl.split ? 2 * m.S : m.S, 16);
            const bool kp = tc::krylov_supported(v, m.N);
            const bool kr = kp || tc::supported(v, tc::KRYLOV, m.N), sk = tc::supported(v, tc::SKETCH, m.N);
            m.tc = pl.mixed && kr && sk;
            // two-pass Krylov step when the fused one does not fit (I_n > 640); plain operands
            m.tc2 = pl.mixed && !m.tc && !pl.split && sk && tc::supported(v, tc::TTM, m.N);
            if (m.tc || m.tc2) {
                m.tgrid = tc::grid_size(v);
                m.kp = m.tc && kp;
                m.kgrid = m.kp ? tc::krylov_grid(v) : m.tgrid;
                m.qimg = c.take<char>(tc::image_bytes_skinny(v, m.N));
                m.omg = c.take<char>(tc::image_bytes_omega(v, m.N));
                m.tpart = c.take<float>((size_t)std::max(m.tgrid, m.kgrid) * m.I * m.N);
            } else {
                m.Y = c.take<double>((size_t)d * m.S);
            }
            if (pl.flags & RBKI_FLAG_REFINE_FP32) {
                const size_t IR = (size_t)m.I * m.R;
                m.refine = true;
                m.U0 = c.take<double>(IR);
                m.Pr = c.take<double>(IR);
                m.Zr = c.take<double>((size_t)m.R * m.R);
                m.Wr = c.take<double>((size_t)m.R * m.R);
                m.lamr = c.take<double>((size_t)m.R);
                m.rsyev = c.take<double>(syev_scratch_doubles(m.R));
                m.rN = (int)rup(2 * m.R, 16);
                m.rkp = pl.mixed && tc::krylov_supported(v, m.rN);
                m.rtc = m.rkp || (pl.mixed && tc::supported(v, tc::KRYLOV, m.rN));
                if (m.rtc) {
                    m.rgrid = m.rkp ? tc::krylov_grid(v) : tc::grid_size(v);
                    m.rimg = c.take<char>(tc::image_bytes_skinny(v, m.rN));
                    m.rpart = c.take<float>((size_t)m.rgrid * m.I * m.rN);
                } else {
                    m.rnsplit = contract_nsplit(v);
                    m.rY = c.take<double>((size_t)d * m.R);
                    m.rsplit = c.take<double>((size_t)m.rnsplit * m.I * m.R);
                }
            }
        }
    }
    // core chain ping-pong buffers (FP64)
    size_t maxbuf = 0;
    {
        int64_t cur[RBKI_MAX_ORDER];
        for (int n = 0; n < pl.N; ++n) cur[n] = pl.dims[n];
        for (int t = 0; t < pl.N; ++t) {
            int m = pl.order[t];
            cur[m] = pl.mode[m].R;
            int64_t sz = 1;
            for (int n = 0; n < pl.N; ++n) sz *= cur[n];
            maxbuf = std::max(maxbuf, (size_t)sz);
        }
    }
    pl.tbuf[0] = c.take<double>(maxbuf);
    pl.tbuf[1] = c.take<double>(maxbuf);
    {
        const int m0 = pl.order[0];
        const ModePlan& m = pl.mode[m0];
        // the first core product streams all of X (not a mode's column sample)
        View v{nullptr, pl.stream_dtype, m.sampled ? m.A0 : m.A, m.I, m.sampled ? m.C0 : m.C};
        // the core carries the reconstruction error |X|^2 - |G|^2: always hi + lo operands,
        // in one pass (2R columns) when they fit the MMA width, else in two (R columns each)
        pl.ttm_N = (int)rup(2 * m.R, 16);
        pl.ttm_tc = pl.mixed && m.R <= 32 && tc::supported(v, tc::TTM, pl.ttm_N);
        if (!pl.ttm_tc && pl.mixed && m.R <= 64 && tc::supported(v, tc::TTM, (int)rup(m.R, 16))) {
            pl.ttm_tc2 = true;
            pl.ttm_N = (int)rup(m.R, 16);
        }
        if (pl.ttm_tc || pl.ttm_tc2) pl.ttm_img = c.take<char>(tc::image_bytes_skinny(v, pl.ttm_N));
    }
    pl.ws_bytes = c.off + 256;
}

// ---------------------------------------------------------------------------------
// per-mode pipeline
// ---------------------------------------------------------------------------------

__global__ void k_symmetrize(double* Z, int n) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    int i = e / n, j = e % n;
    if (i < j) {
        double v = 0.5 * (Z[i * n + j] + Z[j * n + i]);
        Z[i * n + j] = v;
        Z[j * n + i] = v;
    }
}

__global__ void k_add_f32(float* __restrict__ y, const float* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

rbki_status add_f32_cuda(float* y, const float* x, int64_t n, cudaStream_t st) {
    if (n <= 0) return RBKI_OK;
    k_add_f32<<<(unsigned)std::min<int64_t>(cdiv(n, 256), 152 * 8), 256, 0, st>>>(y, x, n);
    RBKI_LAUNCH_CHECK("k_add_f32");
    return RBKI_OK;
}

rbki_status symmetrize_cuda(double* Z, int n, cudaStream_t st) {
    k_symmetrize<<<(unsigned)cdiv((int64_t)n * n, 256), 256, 0, st>>>(Z, n);
    RBKI_LAUNCH_CHECK("k_symmetrize");
    return RBKI_OK;
}

View mode_view(const Plan& pl, const ModePlan& m) {
    return View{m.sampled ? m.ysamp : pl.xstream, pl.stream_dtype, m.A, m.I, m.C};
}

// Partial column sampling: choose the kept units of mode n and gather Y from the streamed X.
static rbki_status sample_mode(const Plan& pl, const ModePlan& m, cudaStream_t st) {
    RBKI_TRY(sample_units_cuda(pl.seed, m.n, m.nunits, m.kunits, m.units, st));
    int tok = prof_begin(RBKI_PROF_SAMPLE, st);
    RBKI_TRY(gather_units_cuda(pl.xstream, pl.stream_dtype, m.A0, m.I, m.C0, m.units, m.kunits, m.ysamp, st));
    prof_end(tok, st);
    return RBKI_OK;
}

// P = X_(n) (X_(n)^T Q) for Q (I x S, ld ldq) -> out (ld ldo), out2 (optional copy)
rbki_status krylov_step(const Plan& pl, const ModePlan& m, const double* Q, int64_t ldq, int S,
                        double* out, int64_t ldo, double* out2, int64_t ldo2, cudaStream_t st) {
    View v = mode_view(pl, m);
    if (m.tc2) {
        // pass 1 writes Y = X_(n)^T Q as per-tile operand images (into the Omega image buffer,
        // free after the sketch); pass 2 is the sketch kernel with Y in place of Omega
        RBKI_TRY(tc::skinny_image(Q, ldq, m.I, S, m.N, false, pl.stream_dtype == RBKI_F16, m.qimg, st));
        int tok = prof_begin(RBKI_PROF_KRYLOV, st);
        RBKI_TRY(tc::stream_tc(tc::TTM, v, m.N, S, false, m.qimg, nullptr, nullptr, nullptr, pl.err, st, m.omg));
        RBKI_TRY(tc::stream_tc(tc::SKETCH, v, m.N, S, false, nullptr, m.omg, m.tpart, nullptr, pl.err, st));
        prof_end(tok, st);
        return tc::reduce_parts(m.tpart, m.tgrid, m.I, m.N, S, false, out, ldo, out2, ldo2, pl.err, st);
    }
    if (m.tc && m.kp) {
        RBKI_TRY(tc::skinny_image(Q, ldq, m.I, S, m.N, pl.split, pl.stream_dtype == RBKI_F16, m.qimg, st));
        int tok = prof_begin(RBKI_PROF_KRYLOV, st);
        RBKI_TRY(tc::krylov_tc(v, m.N, S, pl.split, m.qimg, m.tpart, pl.err, st));
        prof_end(tok, st);
        return tc::reduce_parts(m.tpart, m.kgrid, m.I, m.N, S, pl.split, out, ldo, out2, ldo2, pl.err, st);
    }
    if (m.tc) {
        RBKI_TRY(tc::skinny_image(Q, ldq, m.I, S, m.N, pl.split, pl.stream_dtype == RBKI_F16, m.qimg, st));
        int tok = prof_begin(RBKI_PROF_KRYLOV, st);
        RBKI_TRY(tc::stream_tc(tc::KRYLOV, v, m.N, S, pl.split, m.qimg, nullptr, m.tpart, nullptr, pl.err, st));
        prof_end(tok, st);
        return tc::reduce_parts(m.tpart, m.tgrid, m.I, m.N, S, pl.split, out, ldo, out2, ldo2, pl.err, st);
    }
    int tok = prof_begin(RBKI_PROF_KRYLOV, st);
    RBKI_TRY(ttm_cuda(v, Q, ldq, S, m.Y, RBKI_F64, pl.mixed, st));
    RBKI_TRY(contract_cuda(v, m.Y, RBKI_F64, S, pl.mixed, m.part, m.nsplit, out, ldo, out2, ldo2, st));
    prof_end(tok, st);
    return RBKI_OK;
}

rbki_status orth2(const ModePlan& m, int col0, int32_t* kept, cudaStream_t st) {
    RBKI_TRY(orth_pass_cuda(m.Qall, m.b, m.I, col0, m.S, TAU_DEFLATE, m.small, nullptr, st));
    RBKI_TRY(orth_pass_cuda(m.Qall, m.b, m.I, col0, m.S, TAU_DEFLATE, m.small, kept, st));
    return RBKI_OK;
}

// Algorithm 1 steps 1-2 for mode n: W = X_(n) Omega into block 0 of m.Qall (Omega generated
// per tile in the tensor-core images, or in the [A][S][C] layout on the CUDA-core path)
static rbki_status sketch_mode(const Plan& pl, const ModePlan& m, cudaStream_t st) {
    View v = mode_view(pl, m);
    if (m.tc || m.tc2) {
        RBKI_TRY(tc::omega_images(pl.seed, m.n, v, m.S, m.N, pl.split, m.omg, st));
        int tok = prof_begin(RBKI_PROF_SKETCH, st);
        RBKI_TRY(tc::stream_tc(tc::SKETCH, v, m.N, m.S, pl.split, nullptr, m.omg, m.tpart, nullptr, pl.err, st));
        prof_end(tok, st);
        RBKI_TRY(tc::reduce_parts(m.tpart, m.tgrid, m.I, m.N, m.S, pl.split, m.Qall, m.b, nullptr, 0, pl.err, st));
    } else {
        int tok = prof_begin(RBKI_PROF_SKETCH, st);
        RBKI_TRY(omega_f64_cuda(pl.seed, m.n, m.A, m.C, m.S, m.Y, st));
        RBKI_TRY(contract_cuda(v, m.Y, RBKI_F64, m.S, pl.mixed, m.part, m.nsplit, m.Qall, m.b,
                               nullptr, 0, st));
        prof_end(tok, st);
    }
    return RBKI_OK;
}

// Algorithm 1 for mode n: Q = [Q_0 .. Q_q] in m.Qall, P_j = A Q_j in m.Pall
rbki_status mode_basis(const Plan& pl, const ModePlan& m, int32_t* kept, cudaStream_t st) {
    RBKI_TRY(sketch_mode(pl, m, st));
    if (pl.flags & RBKI_FLAG_POWER) {
        // power iteration: each product replaces the block, orthonormalised on its own
        RBKI_TRY(orth2(m, 0, kept, st));
        for (int j = 0; j <= m.q; ++j) {
            const bool more = j < m.q;
            RBKI_TRY(krylov_step(pl, m, m.Qall, m.b, m.S, m.Pall, m.b, more ? m.Qall : nullptr, m.b, st));
            if (more) {
                RBKI_TRY(fill_i32_cuda(kept, 0, 1, st));
                RBKI_TRY(orth2(m, 0, kept, st));
            }
        }
        return RBKI_OK;
    }
    RBKI_TRY(orth2(m, 0, kept, st));
    // step 3: K = [W, A W, ..., A^q W], orthonormalised block by block (reading c2)
    for (int j = 0; j <= m.q; ++j) {
        bool more = j < m.q;
        RBKI_TRY(krylov_step(pl, m, m.Qall + j * m.S, m.b, m.S, m.Pall + j * m.S, m.b,
                             more ? m.Qall + (j + 1) * m.S : nullptr, m.b, st));
        if (more) RBKI_TRY(orth2(m, (j + 1) * m.S, kept, st));
    }
    return RBKI_OK;
}

// Rayleigh-Ritz refinement of a Krylov-path factor (RBKI_FLAG_REFINE_FP32): P = X X^T U0 at
// width R with FP32-accurate products, Z_r = U0^T P in FP64, its eigenvectors W (descending),
// U = U0 W with the sign rule; the refined Ritz values land in m.lamr.
static rbki_status refine_factor(const Plan& pl, const ModePlan& m, double* U, cudaStream_t st) {
    const View v = mode_view(pl, m);
    const int R = m.R;
    RBKI_TRY(copy_f64_cuda(U, m.U0, (int64_t)m.I * R, st));
    int tok = prof_begin(RBKI_PROF_KRYLOV, st);
    if (m.rtc) {
        RBKI_TRY(tc::skinny_image(m.U0, R, m.I, R, m.rN, 1, pl.stream_dtype == RBKI_F16, m.rimg, st));
        if (m.rkp)
            RBKI_TRY(tc::krylov_tc(v, m.rN, R, true, m.rimg, m.rpart, pl.err, st));
        else
            RBKI_TRY(tc::stream_tc(tc::KRYLOV, v, m.rN, R, true, m.rimg, nullptr, m.rpart, nullptr, pl.err, st));
        prof_end(tok, st);
        RBKI_TRY(tc::reduce_parts(m.rpart, m.rgrid, m.I, m.rN, R, true, m.Pr, R, nullptr, 0, pl.err, st));
    } else {
        RBKI_TRY(ttm_cuda(v, m.U0, R, R, m.rY, RBKI_F64, pl.mixed, st));
        RBKI_TRY(contract_cuda(v, m.rY, RBKI_F64, R, pl.mixed, m.rsplit, m.rnsplit, m.Pr, R, nullptr, 0, st));
        prof_end(tok, st);
    }
    RBKI_TRY(atb_cuda(m.U0, R, R, m.Pr, R, R, m.I, m.part, m.Zr, R, st));
    RBKI_TRY(symmetrize_cuda(m.Zr, R, st));
    RBKI_TRY(syev_top_cuda(m.Zr, R, R, m.lamr, m.Wr, m.rsyev, st));
    return form_factor_cuda(m.U0, R, m.I, m.Wr, R, R, R, U, st);
}

// Algorithm 2 steps 2-5 for mode n: U^(n) and its Ritz values
rbki_status mode_factor(const Plan& pl, const ModePlan& m, double* U, double* eigvals,
                        int32_t* info, cudaStream_t st) {
    int32_t* kept = info ? info + m.n : m.kept;
    if (m.gram) {
        // b >= I: Z = X_(n) X_(n)^T, Q = I (reading c7)
        View v = mode_view(pl, m);
        int tok = prof_begin(RBKI_PROF_GRAM, st);
        if (m.I <= (pl.mixed ? 16 : 8))
            RBKI_TRY(gram_small_cuda(v, pl.mixed, m.part, m.nsplit, m.Z, m.I, st));
        else
            RBKI_TRY(contract_cuda(v, pl.xstream, pl.stream_dtype, (int)m.I, pl.mixed, m.part,
                                   m.nsplit, m.Z, m.I, nullptr, 0, st));
        prof_end(tok, st);
        RBKI_TRY(symmetrize_cuda(m.Z, (int)m.I, st));
        RBKI_TRY(syev_top_cuda(m.Z, (int)m.I, m.R, m.eval, m.evec, m.syev_ws, st));
        RBKI_TRY(form_factor_cuda(nullptr, 0, m.I, m.evec, (int)m.I, m.R, m.R, U, st));
        if (info) RBKI_TRY(fill_i32_cuda(info + m.n, (int32_t)m.I, 1, st));
    } else {
        if (info) RBKI_TRY(fill_i32_cuda(info + m.n, 0, 1, st));
        if (m.sampled) RBKI_TRY(sample_mode(pl, m, st));
        RBKI_TRY(mode_basis(pl, m, kept, st));
        // step 3 (Remark 1): Z = Q^T X X^T Q = Q^T [P_0 .. P_q]
        RBKI_TRY(atb_cuda(m.Qall, m.b, m.b, m.Pall, m.b, m.b, m.I, m.part, m.Z, m.b, st, pl.mixed));
        RBKI_TRY(symmetrize_cuda(m.Z, m.b, st));
        // step 4: leading eigenvectors of Z; step 5: U = Q U~(:, 1:R)
        RBKI_TRY(syev_top_cuda(m.Z, m.b, m.R, m.eval, m.evec, m.syev_ws, st));
        RBKI_TRY(form_factor_cuda(m.Qall, m.b, m.I, m.evec, m.b, m.R, m.R, U, st));
        if (m.refine) RBKI_TRY(refine_factor(pl, m, U, st));
    }
    if (eigvals) RBKI_TRY(copy_f64_cuda(m.refine ? m.lamr : m.eval, eigvals, m.R, st));
    if (info) RBKI_TRY(fill_i32_cuda(info + pl.N + m.n, m.gram ? 1 : 0, 1, st));
    return RBKI_OK;
}

// Lockstep modes: whether the call's Krylov-path modes can run Algorithms 1-2 in lockstep with
// one batched launch per FP64 stage (the batched eigensolver takes b <= 192; adaptive depth,
// power iteration, sampling, refinement and the sequential reading have their own drivers;
// RBKI_FLAG_SERIAL_MODES asks for the per-mode kernels, one mode after another).
static bool lockstep_ok(const Plan& pl) {
    const uint32_t own = RBKI_FLAG_ADAPTIVE_Q | RBKI_FLAG_POWER | RBKI_FLAG_REFINE_FP32 | RBKI_FLAG_SEQUENTIAL |
                         RBKI_FLAG_SERIAL_MODES;
    if (pl.flags & own) return false;
    int krylov = 0;
    for (int n = 0; n < pl.N; ++n) {
        const ModePlan& m = pl.mode[n];
        if (m.gram) continue;
        if (m.sampled || m.b > 192) return false;
        ++krylov;
    }
    return krylov >= 2;
}

// Algorithms 1-2 for every mode on one stream, stage by stage: the X passes per mode (the
// tensor-core kernels take one tensor per launch), each FP64 stage (block orthonormalisation,
// Z = Q^T P, the eigensolver, U = Q U~) as one batched launch for all Krylov-path modes.  The
// batched kernels run each mode through the same device code and grids as the per-mode
// calls, so the results equal the concurrent per-mode chains bit for bit; the modes' FP64
// stages share launches instead of queueing on three streams.
static rbki_status run_modes_lockstep(const Plan& pl, const rbki_tucker_out* out, cudaStream_t st,
                                      bool omega_done) {
    std::vector<const ModePlan*> K;
    // one launch for the scalar outputs known up front (q_used; the Krylov-path modes' kept
    // counters and path words) and the orthonormalisation tickets
    std::vector<FillItem> fills;
    for (int n = 0; n < pl.N; ++n) {
        const ModePlan& m = pl.mode[n];
        if (out->q_used) fills.push_back(FillItem{out->q_used + n, m.gram ? 0 : m.q});
        if (m.gram) continue;
        if (out->info) {
            fills.push_back(FillItem{out->info + n, 0});
            fills.push_back(FillItem{out->info + pl.N + n, 0});
        }
        fills.push_back(FillItem{orth_ticket(m.small), 0, ORTH_TICKETS});
    }
    RBKI_TRY(fill_i32_batched(fills.data(), (int)fills.size(), st));
    for (int n = 0; n < pl.N; ++n) {
        const ModePlan& m = pl.mode[n];
        if (m.gram) RBKI_TRY(mode_factor(pl, m, out->factors[n], out->eigvals[n], out->info, st));
        else K.push_back(&m);
    }
    auto kept = [&](const ModePlan& m) { return out->info ? out->info + m.n : m.kept; };
    const bool f16 = pl.stream_dtype == RBKI_F16;
    // Algorithm 1 steps 1-2: the tensor-core modes' Omega images and reductions batched
    {
        std::vector<tc::OmegaItem> om;
        std::vector<tc::ReduceItem> rd;
        for (const ModePlan* m : K) {
            if (m->tc || m->tc2) om.push_back(tc::OmegaItem{pl.seed, m->n, mode_view(pl, *m), m->S, m->N, pl.split, m->omg});
        }
        if (!omega_done) RBKI_TRY(tc::omega_images_batched(om.data(), (int)om.size(), st));
        for (const ModePlan* m : K) {
            if (!(m->tc || m->tc2)) {
                RBKI_TRY(sketch_mode(pl, *m, st));
                continue;
            }
            int tok = prof_begin(RBKI_PROF_SKETCH, st);
            RBKI_TRY(tc::stream_tc(tc::SKETCH, mode_view(pl, *m), m->N, m->S, pl.split, nullptr, m->omg, m->tpart,
                                   nullptr, pl.err, st));
            prof_end(tok, st);
            rd.push_back(tc::ReduceItem{m->tpart, m->tgrid, m->I, m->N, m->S, pl.split, m->Qall, m->b, nullptr, 0,
                                        pl.err});
        }
        RBKI_TRY(tc::reduce_parts_batched(rd.data(), (int)rd.size(), st));
    }
    auto orth2 = [&](int j) -> rbki_status {
        std::vector<OrthItem> oi;
        for (const ModePlan* m : K)
            oi.push_back(OrthItem{m->Qall, m->b, m->I, j * m->S, m->S, m->small, nullptr});
        RBKI_TRY(orth_pass_batched(oi.data(), (int)oi.size(), TAU_DEFLATE, st));
        for (size_t k = 0; k < K.size(); ++k) oi[k].kept = kept(*K[k]);
        return orth_pass_batched(oi.data(), (int)oi.size(), TAU_DEFLATE, st);
    };
    RBKI_TRY(orth2(0));
    const int q = K[0]->q;
    for (int j = 0; j <= q; ++j) {
        // P_j = X_(n) (X_(n)^T Q_j): single-pass tensor-core modes share the Q-image and
        // reduction launches; two-pass and CUDA-core modes take krylov_step as they are
        std::vector<tc::SkinnyItem> im;
        std::vector<tc::ReduceItem> rd;
        for (const ModePlan* m : K)
            if (m->tc && !m->tc2)
                im.push_back(tc::SkinnyItem{m->Qall + j * m->S, m->b, m->I, m->S, m->N, pl.split ? 1 : 0, f16,
                                            m->qimg});
        RBKI_TRY(tc::skinny_image_batched(im.data(), (int)im.size(), st));
        for (const ModePlan* m : K) {
            double* P = m->Pall + j * m->S;
            double* Qn = j < q ? m->Qall + (j + 1) * m->S : nullptr;
            if (!(m->tc && !m->tc2)) {
                RBKI_TRY(krylov_step(pl, *m, m->Qall + j * m->S, m->b, m->S, P, m->b, Qn, m->b, st));
                continue;
            }
            const View v = mode_view(pl, *m);
            int tok = prof_begin(RBKI_PROF_KRYLOV, st);
            if (m->kp) RBKI_TRY(tc::krylov_tc(v, m->N, m->S, pl.split, m->qimg, m->tpart, pl.err, st));
            else RBKI_TRY(tc::stream_tc(tc::KRYLOV, v, m->N, m->S, pl.split, m->qimg, nullptr, m->tpart, nullptr,
                                        pl.err, st));
            prof_end(tok, st);
            rd.push_back(tc::ReduceItem{m->tpart, m->kp ? m->kgrid : m->tgrid, m->I, m->N, m->S, pl.split, P, m->b,
                                        Qn, m->b, pl.err});
        }
        RBKI_TRY(tc::reduce_parts_batched(rd.data(), (int)rd.size(), st));
        if (j < q) RBKI_TRY(orth2(j + 1));
    }
    std::vector<AtbItem> ab;
    std::vector<EigItem> ei;
    std::vector<FormItem> fi;
    for (const ModePlan* m : K) {
        // Z = Q^T P with its symmetrisation (Z + Z^T) / 2 folded into the reduction
        ab.push_back(AtbItem{m->Qall, m->b, m->b, m->Pall, m->b, m->b, m->I, m->part, m->Z, m->b, 1,
                             pl.mixed ? 1 : 0});
        ei.push_back(EigItem{m->Z, m->b, m->R, m->eval, m->evec, m->syev_ws});
        fi.push_back(FormItem{m->Qall, m->b, m->I, m->evec, m->b, m->R, m->R, out->factors[m->n]});
    }
    RBKI_TRY(atb_batched(ab.data(), (int)ab.size(), st));
    RBKI_TRY(syev_top_batched(ei.data(), (int)ei.size(), st));
    RBKI_TRY(form_factor_batched(fi.data(), (int)fi.size(), st));
    std::vector<CopyItem> ci;
    for (const ModePlan* m : K)
        if (out->eigvals[m->n]) ci.push_back(CopyItem{m->eval, out->eigvals[m->n], m->R});
    return copy_f64_batched(ci.data(), (int)ci.size(), st);
}

// Adaptive Krylov depth (RBKI_FLAG_ADAPTIVE_Q): the Krylov-path modes advance block by
// block in lockstep, each on its own stream.  After block j every active mode has the
// Rayleigh-Ritz values of Z_j = Q_{<=j}^T [P_0 .. P_j]; the host reads them (one
// synchronisation per block), forms F_j = 1 - sqrt(max(|X|^2 - sum lambda, 0) / |X|^2) in
// FP64 and stops the mode at the first j >= 1 with |F_j - F_{j-1}| <= q_tol, or at j = q.
// A stopped mode forms U from the eigenvectors of its last Z_j; a continuing one
// orthonormalises block j+1 (already written by the Krylov step).  Gram-path modes run as
// usual.  q_used[n] receives the depth.
static rbki_status run_modes_adaptive(const Plan& pl, const rbki_tucker_out* out, const double* norms,
                                      const cudaStream_t* ms, int32_t* q_used_host) {
    const double tol = pl.prm.q_tol;
    bool active[RBKI_MAX_ORDER] = {false};
    double prev_fit[RBKI_MAX_ORDER] = {0.0};
    int qmax = 0;
    for (int n = 0; n < pl.N; ++n) {
        const ModePlan& m = pl.mode[n];
        q_used_host[n] = 0;
        if (m.gram) {
            RBKI_TRY(mode_factor(pl, m, out->factors[n], out->eigvals[n], out->info, ms[n]));
            continue;
        }
        int32_t* kept = out->info ? out->info + n : m.kept;
        RBKI_TRY(fill_i32_cuda(kept, 0, 1, ms[n]));
        // Algorithm 1 steps 1-2 and Q_0 (the sketch part of mode_basis)
        View v = mode_view(pl, m);
        if (m.tc || m.tc2) {
            RBKI_TRY(tc::omega_images(pl.seed, m.n, v, m.S, m.N, pl.split, m.omg, ms[n]));
            int tok = prof_begin(RBKI_PROF_SKETCH, ms[n]);
            RBKI_TRY(tc::stream_tc(tc::SKETCH, v, m.N, m.S, pl.split, nullptr, m.omg, m.tpart, nullptr, pl.err, ms[n]));
            prof_end(tok, ms[n]);
            RBKI_TRY(tc::reduce_parts(m.tpart, m.tgrid, m.I, m.N, m.S, pl.split, m.Qall, m.b, nullptr, 0, pl.err, ms[n]));
        } else {
            int tok = prof_begin(RBKI_PROF_SKETCH, ms[n]);
            RBKI_TRY(omega_f64_cuda(pl.seed, m.n, m.A, m.C, m.S, m.Y, ms[n]));
            RBKI_TRY(contract_cuda(v, m.Y, RBKI_F64, m.S, pl.mixed, m.part, m.nsplit, m.Qall, m.b, nullptr, 0, ms[n]));
            prof_end(tok, ms[n]);
        }
        RBKI_TRY(orth2(m, 0, kept, ms[n]));
        active[n] = true;
        qmax = std::max(qmax, m.q);
    }
    std::vector<double> lam[RBKI_MAX_ORDER];
    double x2 = -1.0;
    for (int j = 0; j <= qmax; ++j) {
        bool any = false;
        for (int n = 0; n < pl.N; ++n) {
            if (!active[n]) continue;
            any = true;
            const ModePlan& m = pl.mode[n];
            const int bj = (j + 1) * m.S;
            RBKI_TRY(krylov_step(pl, m, m.Qall + j * m.S, m.b, m.S, m.Pall + j * m.S, m.b,
                                 j < m.q ? m.Qall + (j + 1) * m.S : nullptr, m.b, ms[n]));
            RBKI_TRY(atb_cuda(m.Qall, m.b, bj, m.Pall, m.b, bj, m.I, m.part, m.Z, bj, ms[n], pl.mixed));
            RBKI_TRY(symmetrize_cuda(m.Z, bj, ms[n]));
            RBKI_TRY(syev_top_cuda(m.Z, bj, m.R, m.eval, m.evec, m.syev_ws, ms[n]));
        }
        if (!any) break;
        // the Ritz values (and |X|^2, written before the fork) come back on the mode streams
        bool want_x2 = x2 < 0.0;
        for (int n = 0; n < pl.N; ++n) {
            if (!active[n]) continue;
            lam[n].resize(pl.mode[n].R);
            RBKI_CUDA_TRY(cudaMemcpyAsync(lam[n].data(), pl.mode[n].eval, pl.mode[n].R * sizeof(double),
                                          cudaMemcpyDeviceToHost, ms[n]));
            if (want_x2) {
                RBKI_CUDA_TRY(cudaMemcpyAsync(&x2, norms, sizeof(double), cudaMemcpyDeviceToHost, ms[n]));
                want_x2 = false;
            }
        }
        for (int n = 0; n < pl.N; ++n)
            if (active[n]) RBKI_CUDA_TRY(cudaStreamSynchronize(ms[n]));
        for (int n = 0; n < pl.N; ++n) {
            if (!active[n]) continue;
            const ModePlan& m = pl.mode[n];
            double sum = 0.0;
            for (int k = 0; k < m.R; ++k) sum += lam[n][k];
            const double fit = x2 > 0.0 ? 1.0 - std::sqrt(std::max(x2 - sum, 0.0) / x2) : 1.0;
            const bool stop = j == m.q || (j >= 1 && std::fabs(fit - prev_fit[n]) <= tol);
            prev_fit[n] = fit;
            if (stop) {
                const int bj = (j + 1) * m.S;
                RBKI_TRY(form_factor_cuda(m.Qall, m.b, m.I, m.evec, bj, m.R, m.R, out->factors[n], ms[n]));
                if (out->eigvals[n]) RBKI_TRY(copy_f64_cuda(m.eval, out->eigvals[n], m.R, ms[n]));
                if (out->info) RBKI_TRY(fill_i32_cuda(out->info + pl.N + n, 0, 1, ms[n]));
                q_used_host[n] = j;
                active[n] = false;
            } else {
                int32_t* kept = out->info ? out->info + n : m.kept;
                RBKI_TRY(orth2(m, (j + 1) * m.S, kept, ms[n]));
            }
        }
    }
    return RBKI_OK;
}

// step 6: G = X x_1 U^(1)T ... x_N U^(N)T, largest shrink first
// Steps t_begin .. t_end-1 of the chain; the state before t_begin (dims, source buffer and
// its dtype) follows from the plan, so the first product can run on its mode's stream as
// soon as that factor exists and the rest after the join.
rbki_status core_chain(const Plan& pl, double* const* factors, double* core, cudaStream_t st, int t_begin = 0,
                       int t_end = -1) {
    if (t_end < 0) t_end = pl.N;
    int64_t cur[RBKI_MAX_ORDER];
    for (int n = 0; n < pl.N; ++n) cur[n] = pl.dims[n];
    const void* src = pl.xstream;
    int src_dtype = pl.stream_dtype;
    for (int t = 0; t < t_begin; ++t) {
        cur[pl.order[t]] = pl.mode[pl.order[t]].R;
        src = pl.tbuf[t & 1];
        src_dtype = (t == 0 && (pl.ttm_tc || pl.ttm_tc2) && pl.N > 1) ? RBKI_F32 : RBKI_F64;
    }
    for (int t = t_begin; t < t_end; ++t) {
        int m = pl.order[t];
        int64_t A = 1, C = 1;
        for (int k = 0; k < m; ++k) A *= cur[k];
        for (int k = m + 1; k < pl.N; ++k) C *= cur[k];
        View v{src, src_dtype, A, cur[m], C};
        double* dst = (t == pl.N - 1) ? core : pl.tbuf[t & 1];
        int R = pl.mode[m].R;
        int tok = t == 0 ? prof_begin(RBKI_PROF_TTM, st) : -1;
        if (t == 0 && pl.ttm_tc && t != pl.N - 1) {
            // first mode product on tcgen05: FP32 result [A][R][C] in the ping-pong buffer
            RBKI_TRY(tc::skinny_image(factors[m], R, cur[m], R, pl.ttm_N, true, pl.stream_dtype == RBKI_F16,
                                      pl.ttm_img, st));
            RBKI_TRY(tc::stream_tc(tc::TTM, v, pl.ttm_N, R, true, pl.ttm_img, nullptr, nullptr, (float*)dst,
                                   pl.err, st));
            prof_end(tok, st);
            cur[m] = R;
            src = dst;
            src_dtype = RBKI_F32;
            continue;
        }
        if (t == 0 && pl.ttm_tc2 && t != pl.N - 1) {
            // R > 32: the hi part of the factor into dst, the lo part into the other ping-pong
            // buffer (free until step 1), then summed: the split product in two passes
            float* lo = reinterpret_cast<float*>(pl.tbuf[1]);
            const bool f16 = pl.stream_dtype == RBKI_F16;
            RBKI_TRY(tc::skinny_image(factors[m], R, cur[m], R, pl.ttm_N, 0, f16, pl.ttm_img, st));
            RBKI_TRY(tc::stream_tc(tc::TTM, v, pl.ttm_N, R, false, pl.ttm_img, nullptr, nullptr, (float*)dst,
                                   pl.err, st));
            RBKI_TRY(tc::skinny_image(factors[m], R, cur[m], R, pl.ttm_N, 2, f16, pl.ttm_img, st));
            RBKI_TRY(tc::stream_tc(tc::TTM, v, pl.ttm_N, R, false, pl.ttm_img, nullptr, nullptr, lo, pl.err, st));
            RBKI_TRY(add_f32_cuda((float*)dst, lo, A * R * C, st));
            prof_end(tok, st);
            cur[m] = R;
            src = dst;
            src_dtype = RBKI_F32;
            continue;
        }
        if (t > 0 && R <= 32 && (src_dtype == RBKI_F64 || src_dtype == RBKI_F32))
            RBKI_TRY(ttm_small_cuda(v, factors[m], R, R, dst, pl.mixed, st));
        else
            RBKI_TRY(ttm_cuda(v, factors[m], R, R, dst, RBKI_F64, pl.mixed, st));
        prof_end(tok, st);
        cur[m] = R;
        src = dst;
        src_dtype = RBKI_F64;
    }
    return RBKI_OK;
}

// Per-device pools of non-blocking streams: the N modes are independent (HOSVD reading), so
// each mode's Algorithm 1-2 chain runs on its own stream, forked from and joined back to the
// caller's stream.  Latency-bound small FP64 kernels of one mode then overlap the HBM-bound
// passes of the others.  Each caller stream gets its own set, so that calls issued on
// different streams (decompositions in flight together) do not queue behind one another on
// shared mode streams.  A device keeps at most MAX_POOLS sets; callers beyond that share
// the last one.
struct StreamPool {
    cudaStream_t owner = nullptr;
    cudaStream_t s[RBKI_MAX_ORDER];
};
constexpr int MAX_POOLS = 64;
static std::mutex g_pool_mu;
static std::vector<StreamPool> g_pools[64];

static rbki_status pool_streams(cudaStream_t caller, cudaStream_t* out, int n) {
    int dev = 0;
    RBKI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(RBKI_E_UNSUPPORTED, "device index");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    std::vector<StreamPool>& pools = g_pools[dev];
    StreamPool* p = nullptr;
    for (auto& q : pools)
        if (q.owner == caller) p = &q;
    if (!p && (int)pools.size() < MAX_POOLS) {
        StreamPool q;
        q.owner = caller;
        for (int i = 0; i < RBKI_MAX_ORDER; ++i)
            RBKI_CUDA_TRY(cudaStreamCreateWithFlags(&q.s[i], cudaStreamNonBlocking));
        pools.push_back(q);
        p = &pools.back();
    }
    if (!p) p = &pools.back();
    for (int i = 0; i < n; ++i) out[i] = p->s[i];
    return RBKI_OK;
}

// Algorithm 2, sequentially truncated reading: for n = 1..N, U^(n) from Algorithm 1 on
// Y_n (Y_1 = X), then Y_{n+1} = Y_n x_n U^(n)T; the last product is the core G.  Every step
// depends on the previous one, so all of it runs on the caller's stream.  Mixed precision:
// Y_n is kept in FP32 and streamed as BF16/FP16 (staged per step); the first product runs
// on the tensor cores from the staged X when the shape allows.
static rbki_status run_sequential(Plan& pl, const rbki_tucker_out* out, cudaStream_t st) {
    if (!pl.ws_base || !pl.scal || !pl.err) return set_error(RBKI_E_INVAL, "sequential plan not carved");
    double* norms = out->norms ? out->norms : pl.scal;
    RBKI_CUDA_TRY(cudaMemsetAsync(pl.err, 0, sizeof(int32_t), st));
    int64_t cur[RBKI_MAX_ORDER];
    for (int n = 0; n < pl.N; ++n) cur[n] = pl.dims[n];
    const void* src = pl.xin;
    int src_dtype = pl.dtype;
    for (int n = 0; n < pl.N; ++n) {
        Plan sp;
        RBKI_TRY(step_plan(pl, n, cur, src_dtype, sp));
        carve(sp, pl.ws_base);
        if (sp.err != pl.err) return set_error(RBKI_E_INVAL, "sequential plan: error word moved");
        sp.xin = src;
        const int64_t numel = sp.numel;
        double* nrm = n == 0 ? norms : sp.scal + 8;
        int tok = prof_begin(RBKI_PROF_STAGE, st);
        if (sp.stage) {
            RBKI_TRY(stage_cuda(src, src_dtype, numel, sp.xs, sp.stream_dtype, sp.scal + 64, nrm, st));
            sp.xstream = sp.xs;
        } else {
            sp.xstream = src;
            if (n == 0) RBKI_TRY(sumsq_cuda(src, src_dtype, numel, sp.scal + 64, nrm, st));
        }
        prof_end(tok, st);
        const ModePlan& m = sp.mode[n];
        RBKI_TRY(mode_factor(sp, m, out->factors[n], out->eigvals[n], out->info, st));
        // Y_{n+1} = Y_n x_n U^(n)T
        const bool last = n == pl.N - 1;
        void* dst = last ? (void*)out->core : pl.ybuf[n & 1];
        const int dst_dtype = last ? RBKI_F64 : pl.ydtype;
        const int R = m.R;
        // the product runs over all of Y_n (a sampled mode's m.A, m.C describe the sample)
        const int64_t fa = m.sampled ? m.A0 : m.A, fc = m.sampled ? m.C0 : m.C;
        tok = prof_begin(RBKI_PROF_TTM, st);
        if (n == 0 && pl.ttm_tc && !last) {
            View v{sp.xstream, sp.stream_dtype, fa, m.I, fc};
            RBKI_TRY(tc::skinny_image(out->factors[0], R, m.I, R, pl.ttm_N, true, sp.stream_dtype == RBKI_F16,
                                      pl.ttm_img, st));
            RBKI_TRY(tc::stream_tc(tc::TTM, v, pl.ttm_N, R, true, pl.ttm_img, nullptr, nullptr, (float*)dst,
                                   pl.err, st));
        } else {
            View v{src, src_dtype, fa, m.I, fc};
            if (n > 0 && dst_dtype == RBKI_F64 && R <= 32 && (src_dtype == RBKI_F64 || src_dtype == RBKI_F32))
                RBKI_TRY(ttm_small_cuda(v, out->factors[n], R, R, (double*)dst, pl.mixed, st));
            else
                RBKI_TRY(ttm_cuda(v, out->factors[n], R, R, dst, dst_dtype, pl.mixed, st));
        }
        prof_end(tok, st);
        cur[n] = R;
        src = dst;
        src_dtype = dst_dtype;
    }
    RBKI_TRY(sumsq_cuda(out->core, RBKI_F64, pl.ranks_numel, pl.scal + 64, norms + 1, st));
    if (out->info)
        RBKI_CUDA_TRY(cudaMemcpyAsync(out->info + 2 * pl.N, pl.err, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    if (out->q_used)
        for (int n = 0; n < pl.N; ++n)
            RBKI_TRY(fill_i32_cuda(out->q_used + n, pl.mode[n].gram ? 0 : pl.mode[n].q, 1, st));
    return RBKI_OK;
}

// Per-caller item streams of a batch (rbki_tucker_batch): item k of a batch issued on
// `caller` runs on item stream k mod MAX_ITEMS, which then owns its own mode-stream set.
constexpr int MAX_ITEMS = 32;
struct ItemPool {
    cudaStream_t owner = nullptr;
    std::vector<cudaStream_t> s;
};
static std::vector<ItemPool> g_items[64];

static rbki_status item_streams(cudaStream_t caller, int count, std::vector<cudaStream_t>& out) {
    int dev = 0;
    RBKI_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(RBKI_E_UNSUPPORTED, "device index");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    ItemPool* p = nullptr;
    for (auto& q : g_items[dev])
        if (q.owner == caller) p = &q;
    if (!p) {
        g_items[dev].push_back(ItemPool{caller, {}});
        p = &g_items[dev].back();
    }
    const int want = std::min(count, MAX_ITEMS);
    while ((int)p->s.size() < want) {
        cudaStream_t s;
        RBKI_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        p->s.push_back(s);
    }
    out.resize(count);
    for (int k = 0; k < count; ++k) out[k] = p->s[k % MAX_ITEMS];
    return RBKI_OK;
}

rbki_status run_tucker(Plan& pl, const rbki_tucker_out* out, cudaStream_t st, const cudaStream_t* mode_streams) {
    if (pl.sequential) return run_sequential(pl, out, st);
    double* norms = out->norms ? out->norms : pl.scal;
    RBKI_CUDA_TRY(cudaMemsetAsync(pl.err, 0, sizeof(int32_t), st));
    const bool concurrent = pl.N > 1 && !(pl.flags & RBKI_FLAG_SERIAL_MODES);
    const bool lockstep = !(pl.flags & RBKI_FLAG_ADAPTIVE_Q) && lockstep_ok(pl);
    // FP32 -> BF16 staging (every path, so that |X|^2 is summed in one order): the cast and,
    // for lockstep calls, the modes' Omega images in one launch
    std::vector<tc::OmegaItem> om;
    const bool fused = pl.stage && pl.dtype == RBKI_F32 && pl.stream_dtype == RBKI_BF16 && pl.numel % 4 == 0 &&
                       (uintptr_t)pl.xin % 16 == 0 && (uintptr_t)pl.xs % 8 == 0 &&
                       tc::stage_omega_grid() <= 4096 - 64;
    if (fused) {
        pl.xstream = pl.xs;
        for (int n = 0; n < pl.N && lockstep; ++n) {
            const ModePlan& m = pl.mode[n];
            if (!m.gram && (m.tc || m.tc2))
                om.push_back(tc::OmegaItem{pl.seed, m.n, mode_view(pl, m), m.S, m.N, pl.split, m.omg});
        }
        if (om.size() > 8) om.clear();
    }
    const bool omega_done = !om.empty();
    int tok = prof_begin(RBKI_PROF_STAGE, st);
    if (fused) {
        RBKI_TRY(tc::stage_omega_batched(static_cast<const float*>(pl.xin), pl.numel, pl.xs, pl.scal + 64, om.data(),
                                         (int)om.size(), st));
        RBKI_TRY(sum_parts_cuda(pl.scal + 64, tc::stage_omega_grid(), norms, st));
    } else if (pl.stage) {
        RBKI_TRY(stage_cuda(pl.xin, pl.dtype, pl.numel, pl.xs, pl.stream_dtype, pl.scal + 64,
                            norms, st));
        pl.xstream = pl.xs;
    } else {
        pl.xstream = pl.xin;
        RBKI_TRY(sumsq_cuda(pl.xin, pl.dtype, pl.numel, pl.scal + 64, norms, st));
    }
    prof_end(tok, st);
    int chain_from = 0;   // core-chain steps already enqueued on a mode stream
    int32_t q_used[RBKI_MAX_ORDER];
    for (int n = 0; n < pl.N; ++n) q_used[n] = pl.mode[n].gram ? 0 : pl.mode[n].q;
    if (pl.flags & RBKI_FLAG_ADAPTIVE_Q) {
        cudaStream_t ms[RBKI_MAX_ORDER];
        if (!concurrent) {
            for (int n = 0; n < pl.N; ++n) ms[n] = st;
        } else if (mode_streams) {
            for (int n = 0; n < pl.N; ++n) ms[n] = mode_streams[n];
        } else {
            RBKI_TRY(pool_streams(st, ms, pl.N));
        }
        cudaEvent_t ev;
        RBKI_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        RBKI_CUDA_TRY(cudaEventRecord(ev, st));
        for (int n = 0; n < pl.N; ++n) RBKI_CUDA_TRY(cudaStreamWaitEvent(ms[n], ev, 0));
        rbki_status rs = run_modes_adaptive(pl, out, norms, ms, q_used);
        for (int n = 0; n < pl.N && concurrent; ++n) {
            RBKI_CUDA_TRY(cudaEventRecord(ev, ms[n]));
            RBKI_CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
        }
        cudaEventDestroy(ev);
        if (rs < 0) return rs;
    } else if (lockstep) {
        RBKI_TRY(run_modes_lockstep(pl, out, st, omega_done));
    } else if (concurrent) {
        cudaStream_t ms[RBKI_MAX_ORDER];
        if (mode_streams) {
            for (int n = 0; n < pl.N; ++n) ms[n] = mode_streams[n];
        } else {
            RBKI_TRY(pool_streams(st, ms, pl.N));
        }
        cudaEvent_t fork, join[RBKI_MAX_ORDER];
        RBKI_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        RBKI_CUDA_TRY(cudaEventRecord(fork, st));
        rbki_status rs = RBKI_OK;
        for (int n = 0; n < pl.N; ++n) {
            RBKI_CUDA_TRY(cudaEventCreateWithFlags(&join[n], cudaEventDisableTiming));
            RBKI_CUDA_TRY(cudaStreamWaitEvent(ms[n], fork, 0));
            if (rs >= 0) rs = mode_factor(pl, pl.mode[n], out->factors[n], out->eigvals[n], out->info, ms[n]);
            // the first core product needs only this mode's factor: start it on this stream
            if (rs >= 0 && n == pl.order[0]) {
                rs = core_chain(pl, out->factors, out->core, ms[n], 0, 1);
                chain_from = 1;
            }
            RBKI_CUDA_TRY(cudaEventRecord(join[n], ms[n]));
            RBKI_CUDA_TRY(cudaStreamWaitEvent(st, join[n], 0));
        }
        cudaEventDestroy(fork);
        for (int n = 0; n < pl.N; ++n) cudaEventDestroy(join[n]);
        if (rs < 0) return rs;
    } else {
        for (int n = 0; n < pl.N; ++n)
            RBKI_TRY(mode_factor(pl, pl.mode[n], out->factors[n], out->eigvals[n], out->info, st));
    }
    if (out->q_used && !lockstep)   // the lockstep driver writes q_used with its first launch
        for (int n = 0; n < pl.N; ++n) RBKI_TRY(fill_i32_cuda(out->q_used + n, q_used[n], 1, st));
    RBKI_TRY(core_chain(pl, out->factors, out->core, st, chain_from));
    RBKI_TRY(sumsq_cuda(out->core, RBKI_F64, pl.ranks_numel, pl.scal + 64, norms + 1, st));
    if (out->info)
        RBKI_CUDA_TRY(cudaMemcpyAsync(out->info + 2 * pl.N, pl.err, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    return RBKI_OK;
}

}  // namespace rbki

using namespace rbki;

extern "C" {

const char* rbki_status_str(rbki_status s) {
    switch (s) {
        case RBKI_OK: return "ok";
        case RBKI_PENDING: return "pending";
        case RBKI_W_DEFLATED: return "warning: Krylov directions deflated";
        case RBKI_E_INVAL: return "invalid argument";
        case RBKI_E_NOMEM: return "out of memory / workspace too small";
        case RBKI_E_CUDA: return "CUDA error";
        case RBKI_E_UNSUPPORTED: return "unsupported";
        case RBKI_E_TIMEOUT: return "timeout";
        case RBKI_E_BUSY: return "busy";
        case RBKI_E_CANCELLED: return "cancelled";
        case RBKI_E_NOTFOUND: return "not found";
        default: return "unknown status";
    }
}

const char* rbki_last_error(void) { return g_err.c_str(); }

uint64_t rbki_kernel_launches(void) { return g_launches.load(); }

void rbki_profile_enable(int32_t on) { g_prof_on = on != 0; }

void rbki_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_used = 0;
}

rbki_status rbki_profile_read(int32_t cls, uint64_t* count, double* total_ms) {
    if (!count || !total_ms) return set_error(RBKI_E_INVAL, "NULL output");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    uint64_t c = 0;
    double t = 0.0;
    for (size_t i = 0; i < g_prof_used; ++i) {
        if (g_prof[i].cls != cls) continue;
        RBKI_CUDA_TRY(cudaEventSynchronize(g_prof[i].b));
        float ms = 0.f;
        RBKI_CUDA_TRY(cudaEventElapsedTime(&ms, g_prof[i].a, g_prof[i].b));
        t += ms;
        ++c;
    }
    *count = c;
    *total_ms = t;
    return RBKI_OK;
}

rbki_status rbki_tucker_workspace(const rbki_tensor* X, const rbki_params* prm, size_t* bytes) {
    if (!bytes) return set_error(RBKI_E_INVAL, "bytes is NULL");
    Plan pl;
    RBKI_TRY(make_plan(X, prm, pl));
    carve(pl, nullptr);
    size_t extra = 0;
    if (prm->flags & RBKI_FLAG_HOST_IO) extra = host_io_bytes(pl);
    *bytes = pl.ws_bytes + extra;
    return RBKI_OK;
}

rbki_status rbki_tucker(const rbki_tensor* X, const rbki_params* prm, void* workspace,
                        size_t workspace_bytes, const rbki_tucker_out* out, void* stream) {
    Plan pl;
    RBKI_TRY(make_plan(X, prm, pl));
    if (!out || !out->core) return set_error(RBKI_E_INVAL, "out->core is NULL");
    for (int n = 0; n < pl.N; ++n)
        if (!out->factors[n]) return set_error(RBKI_E_INVAL, "out->factors[n] is NULL");
    carve(pl, nullptr);
    size_t need = pl.ws_bytes + ((prm->flags & RBKI_FLAG_HOST_IO) ? host_io_bytes(pl) : 0);
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    carve(pl, workspace);
    if (prm->flags & RBKI_FLAG_HOST_IO) return run_tucker_host_io(pl, X, out, workspace, st);
    pl.xin = X->data;
    return run_tucker(pl, out, st);
}

// Workspace of the step-level Krylov product: staging copy, FP64 intermediates of the
// CUDA-core path or the operand image + partials of the tensor-core path.
static rbki_status krylov_product_plan(const rbki_tensor* X, int32_t mode, int32_t prec, int32_t s,
                                       uint32_t flags, Plan& pl, ModePlan& m, void* ws, size_t* bytes) {
    RBKI_TRY(validate_tensor(X));
    if (mode < 0 || mode >= X->order || s < 1 || s > 128)
        return set_error(RBKI_E_INVAL, "mode or s out of range");
    rbki_params prm{};
    for (int n = 0; n < X->order; ++n) prm.ranks[n] = 1;
    prm.prec = prec;
    prm.flags = flags;
    RBKI_TRY(make_plan(X, &prm, pl));
    m = pl.mode[mode];
    m.S = s;
    Carver c(ws);
    pl.scal = c.take<double>(4096);
    pl.err = c.take<int32_t>(64);
    if (pl.stage) pl.xs = c.take<char>((size_t)pl.numel * dtype_size(pl.stream_dtype));
    View v{nullptr, pl.stream_dtype, m.A, m.I, m.C};
    m.N = (int)rup(pl.split ? 2 * s : s, 16);
    m.tc = pl.mixed && (tc::krylov_supported(v, m.N) || tc::supported(v, tc::KRYLOV, m.N));
    m.tc2 = pl.mixed && !m.tc && !pl.split && tc::supported(v, tc::SKETCH, m.N) && tc::supported(v, tc::TTM, m.N);
    if (m.tc || m.tc2) {
        m.tgrid = tc::grid_size(v);
        m.kp = m.tc && tc::krylov_supported(v, m.N);
        m.kgrid = m.kp ? tc::krylov_grid(v) : m.tgrid;
        m.qimg = c.take<char>(tc::image_bytes_skinny(v, m.N));
        m.tpart = c.take<float>((size_t)std::max(m.tgrid, m.kgrid) * m.I * m.N);
        if (m.tc2) m.omg = c.take<char>(tc::image_bytes_omega(v, m.N));
    } else {
        m.nsplit = contract_nsplit(v);
        m.Y = c.take<double>((size_t)m.A * m.C * s);
        m.part = c.take<double>((size_t)m.nsplit * m.I * s);
    }
    if (bytes) *bytes = c.off + 256;
    return RBKI_OK;
}

rbki_status rbki_krylov_product_workspace(const rbki_tensor* X, int32_t mode, int32_t prec,
                                          int32_t s, size_t* bytes) {
    if (!bytes) return set_error(RBKI_E_INVAL, "bytes is NULL");
    Plan pl;
    ModePlan m;
    uint32_t flags = prec < 0 ? RBKI_FLAG_SPLIT : 0u;
    return krylov_product_plan(X, mode, prec < 0 ? -prec : prec, s, flags, pl, m, nullptr, bytes);
}

// prec < 0 selects the split (hi + lo) operand variant of precision -prec.
rbki_status rbki_krylov_product(const rbki_tensor* X, int32_t mode, int32_t prec, const double* Q,
                                int32_t s, double* P, void* workspace, size_t workspace_bytes,
                                void* stream) {
    size_t need = 0;
    Plan pl;
    ModePlan m;
    uint32_t flags = prec < 0 ? RBKI_FLAG_SPLIT : 0u;
    int32_t pr = prec < 0 ? -prec : prec;
    RBKI_TRY(krylov_product_plan(X, mode, pr, s, flags, pl, m, nullptr, &need));
    if (!Q || !P) return set_error(RBKI_E_INVAL, "Q/P NULL");
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    RBKI_TRY(krylov_product_plan(X, mode, pr, s, flags, pl, m, workspace, nullptr));
    cudaStream_t st = (cudaStream_t)stream;
    RBKI_CUDA_TRY(cudaMemsetAsync(pl.err, 0, sizeof(int32_t), st));
    if (pl.stage) {
        RBKI_TRY(stage_cuda(X->data, X->dtype, pl.numel, pl.xs, pl.stream_dtype, pl.scal + 64,
                            pl.scal, st));
        pl.xstream = pl.xs;
    } else {
        pl.xstream = X->data;
    }
    return krylov_step(pl, m, Q, s, s, P, s, nullptr, 0, st);
}

// Diagnostics of the bounded waits: the Krylov step of rbki_krylov_product with a planted
// stall (the MMA issuer first waits on a barrier nothing arrives at, for wait_us microseconds),
// so the abort path runs: every role leaves its loop, the copies and MMAs already issued
// are drained, tensor memory is freed and the error word set.  Synchronises the stream and
// reads the error word back.
rbki_status rbki_diag_krylov_stall(const rbki_tensor* X, int32_t mode, int32_t prec, const double* Q, int32_t s,
                                   double* P, void* workspace, size_t workspace_bytes, uint32_t wait_us,
                                   void* stream) {
    size_t need = 0;
    Plan pl;
    ModePlan m;
    uint32_t flags = prec < 0 ? RBKI_FLAG_SPLIT : 0u;
    int32_t pr = prec < 0 ? -prec : prec;
    RBKI_TRY(krylov_product_plan(X, mode, pr, s, flags, pl, m, nullptr, &need));
    if (!Q || !P) return set_error(RBKI_E_INVAL, "Q/P NULL");
    if (wait_us == 0) return set_error(RBKI_E_INVAL, "wait_us must be positive");
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    RBKI_TRY(krylov_product_plan(X, mode, pr, s, flags, pl, m, workspace, nullptr));
    if (!(m.tc || m.tc2)) return set_error(RBKI_E_UNSUPPORTED, "diag stall: not a tensor-core shape");
    cudaStream_t st = (cudaStream_t)stream;
    RBKI_CUDA_TRY(cudaMemsetAsync(pl.err, 0, sizeof(int32_t), st));
    if (pl.stage) {
        RBKI_TRY(stage_cuda(X->data, X->dtype, pl.numel, pl.xs, pl.stream_dtype, pl.scal + 64, pl.scal, st));
        pl.xstream = pl.xs;
    } else {
        pl.xstream = X->data;
    }
    const View v = mode_view(pl, m);
    const bool f16 = pl.stream_dtype == RBKI_F16;
    if (m.tc2) {
        RBKI_TRY(tc::skinny_image(Q, s, m.I, s, m.N, false, f16, m.qimg, st));
        RBKI_TRY(tc::stream_tc(tc::TTM, v, m.N, s, false, m.qimg, nullptr, nullptr, nullptr, pl.err, st, m.omg,
                               wait_us, 1));
        RBKI_TRY(tc::stream_tc(tc::SKETCH, v, m.N, s, false, nullptr, m.omg, m.tpart, nullptr, pl.err, st));
        RBKI_TRY(tc::reduce_parts(m.tpart, m.tgrid, m.I, m.N, s, false, P, s, nullptr, 0, pl.err, st));
    } else {
        RBKI_TRY(tc::skinny_image(Q, s, m.I, s, m.N, pl.split, f16, m.qimg, st));
        if (m.kp)
            RBKI_TRY(tc::krylov_tc(v, m.N, s, pl.split, m.qimg, m.tpart, pl.err, st, wait_us, 1));
        else
            RBKI_TRY(tc::stream_tc(tc::KRYLOV, v, m.N, s, pl.split, m.qimg, nullptr, m.tpart, nullptr, pl.err, st,
                                   nullptr, wait_us, 1));
        RBKI_TRY(tc::reduce_parts(m.tpart, m.kp ? m.kgrid : m.tgrid, m.I, m.N, s, pl.split, P, s, nullptr, 0,
                                  pl.err, st));
    }
    int32_t h = 0;
    RBKI_CUDA_TRY(cudaMemcpyAsync(&h, pl.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBKI_CUDA_TRY(cudaStreamSynchronize(st));
    return h ? set_error(RBKI_E_TIMEOUT, "a bounded device wait expired (planted stall)") : RBKI_OK;
}

rbki_status rbki_mode_basis(const rbki_tensor* X, const rbki_params* prm, int32_t mode, double* Q,
                            void* workspace, size_t workspace_bytes, void* stream) {
    Plan pl;
    RBKI_TRY(make_plan(X, prm, pl));
    if (mode < 0 || mode >= pl.N) return set_error(RBKI_E_INVAL, "mode out of range");
    if (pl.sequential) return set_error(RBKI_E_INVAL, "the basis is defined on X: no RBKI_FLAG_SEQUENTIAL");
    if (pl.mode[mode].gram) return set_error(RBKI_E_INVAL, "mode uses the Gram path (b >= I)");
    if (!Q) return set_error(RBKI_E_INVAL, "Q is NULL");
    carve(pl, nullptr);
    if (!workspace || workspace_bytes < pl.ws_bytes) return set_error(RBKI_E_NOMEM, "workspace too small");
    carve(pl, workspace);
    cudaStream_t st = (cudaStream_t)stream;
    pl.xin = X->data;
    if (pl.stage) {
        RBKI_TRY(stage_cuda(pl.xin, pl.dtype, pl.numel, pl.xs, pl.stream_dtype, pl.scal + 64,
                            pl.scal, st));
        pl.xstream = pl.xs;
    } else {
        pl.xstream = pl.xin;
    }
    const ModePlan& m = pl.mode[mode];
    RBKI_TRY(fill_i32_cuda(m.kept, 0, 1, st));
    if (m.sampled) RBKI_TRY(sample_mode(pl, m, st));
    RBKI_TRY(mode_basis(pl, m, m.kept, st));
    RBKI_TRY(copy_f64_cuda(m.Qall, Q, m.I * m.b, st));
    return RBKI_OK;
}

// ---- rBKI-TK-TR (Algorithm 3) ----------------------------------------------------
struct HtrLayout {
    size_t tucker, core, fac[RBKI_MAX_ORDER], eig[RBKI_MAX_ORDER], norms, info, trc[RBKI_MAX_ORDER], table, trws,
        total;
};

static rbki_status htr_layout(const Plan& pl, const rbki_params* tk, const int32_t* tr, HtrLayout& L) {
    size_t off = (pl.ws_bytes + 255) & ~(size_t)255;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        size_t r = off;
        off += bytes;
        return r;
    };
    L.tucker = 0;
    L.core = take((size_t)pl.ranks_numel * 8);
    int64_t cdims[RBKI_MAX_ORDER];
    for (int n = 0; n < pl.N; ++n) {
        L.fac[n] = take((size_t)pl.dims[n] * tk->ranks[n] * 8);
        L.eig[n] = take((size_t)tk->ranks[n] * 8);
        cdims[n] = tk->ranks[n];
    }
    L.norms = take(16);
    L.info = take((2 * RBKI_MAX_ORDER + 1) * 4);
    for (int n = 0; n < pl.N; ++n)
        L.trc[n] = take((size_t)tr[(n + pl.N - 1) % pl.N] * tk->ranks[n] * tr[n] * 8);
    L.table = take(RBKI_MAX_ORDER * sizeof(double*));
    L.trws = take(std::max(tr_workspace_doubles_for(pl.N, cdims, tr), trsvd_workspace_doubles(pl.N, cdims, tr)) * 8);
    L.total = off + 256;
    return RBKI_OK;
}

static rbki_status htr_validate(const rbki_tensor* X, const rbki_params* tk, const int32_t* tr_ranks, Plan& pl) {
    RBKI_TRY(make_plan(X, tk, pl));
    if (!tr_ranks) return set_error(RBKI_E_INVAL, "tr_ranks is NULL");
    for (int n = 0; n < pl.N; ++n)
        if (tr_ranks[n] < 1 || tr_ranks[n] > 8) return set_error(RBKI_E_UNSUPPORTED, "TR ranks must be in [1, 8]");
    if (pl.N < 2) return set_error(RBKI_E_INVAL, "a tensor ring needs order >= 2");
    if (tk->flags & RBKI_FLAG_HOST_IO) return set_error(RBKI_E_UNSUPPORTED, "rbki_htr takes device buffers");
    carve(pl, nullptr);
    return RBKI_OK;
}

rbki_status rbki_htr_workspace(const rbki_tensor* X, const rbki_params* tk, const int32_t* tr_ranks,
                               size_t* bytes) {
    if (!bytes) return set_error(RBKI_E_INVAL, "bytes is NULL");
    Plan pl;
    RBKI_TRY(htr_validate(X, tk, tr_ranks, pl));
    HtrLayout L;
    RBKI_TRY(htr_layout(pl, tk, tr_ranks, L));
    *bytes = L.total;
    return RBKI_OK;
}

// Algorithm 3: rBKI-TK, TR-ALS on the core, contraction of each TR core with its factor.
// Synchronises `stream` once per TR-ALS sweep (the stopping rule is evaluated on the host).
rbki_status rbki_htr(const rbki_tensor* X, const rbki_params* tk, const int32_t* tr_ranks,
                     const double* const* tr_init, int32_t tr_maxit, double tr_tol, double* const* tr_cores,
                     double* fits, const rbki_tucker_out* tucker_out, void* workspace, size_t workspace_bytes,
                     void* stream) {
    Plan pl;
    RBKI_TRY(htr_validate(X, tk, tr_ranks, pl));
    const bool trsvd = (tk->flags & RBKI_FLAG_TR_SVD) != 0;
    if ((!trsvd && !tr_init) || !tr_cores || tr_maxit < 1)
        return set_error(RBKI_E_INVAL, "tr_init / tr_cores / tr_maxit");
    for (int n = 0; n < pl.N; ++n)
        if ((!trsvd && !tr_init[n]) || !tr_cores[n]) return set_error(RBKI_E_INVAL, "NULL TR core pointer");
    HtrLayout L;
    RBKI_TRY(htr_layout(pl, tk, tr_ranks, L));
    if (!workspace || workspace_bytes < L.total) return set_error(RBKI_E_NOMEM, "workspace too small");
    carve(pl, workspace);
    char* base = static_cast<char*>(workspace);
    cudaStream_t st = (cudaStream_t)stream;
    rbki_tucker_out o{};
    if (tucker_out && tucker_out->core) {
        o = *tucker_out;
    } else {
        o.core = reinterpret_cast<double*>(base + L.core);
        for (int n = 0; n < pl.N; ++n) o.factors[n] = reinterpret_cast<double*>(base + L.fac[n]);
    }
    for (int n = 0; n < pl.N; ++n)
        if (!o.eigvals[n]) o.eigvals[n] = reinterpret_cast<double*>(base + L.eig[n]);
    if (!o.norms) o.norms = reinterpret_cast<double*>(base + L.norms);
    if (!o.info) o.info = reinterpret_cast<int32_t*>(base + L.info);
    pl.xin = X->data;
    RBKI_TRY(run_tucker(pl, &o, st));
    // working TR cores (initial values copied in) and their pointer table
    double* cores[RBKI_MAX_ORDER];
    int64_t cdims[RBKI_MAX_ORDER];
    if (trsvd) {
        // TR-SVD instead of TR-ALS: no initial cores, no host synchronisation; fits[0] is the
        // fit of the ring to G, the rest NaN
        for (int n = 0; n < pl.N; ++n) {
            cores[n] = reinterpret_cast<double*>(base + L.trc[n]);
            cdims[n] = tk->ranks[n];
        }
        RBKI_TRY(tr_svd_cuda(pl.N, cdims, tr_ranks, o.core, cores, reinterpret_cast<double*>(base + L.trws), fits,
                             tr_maxit, st));
        for (int n = 0; n < pl.N; ++n)
            RBKI_TRY(tr_contract_cuda(cores[n], o.factors[n], tr_ranks[(n + pl.N - 1) % pl.N], tk->ranks[n],
                                      tr_ranks[n], pl.dims[n], tr_cores[n], st));
        return RBKI_OK;
    }
    for (int n = 0; n < pl.N; ++n) {
        cores[n] = reinterpret_cast<double*>(base + L.trc[n]);
        cdims[n] = tk->ranks[n];
        const size_t cnt = (size_t)tr_ranks[(n + pl.N - 1) % pl.N] * tk->ranks[n] * tr_ranks[n];
        RBKI_CUDA_TRY(cudaMemcpyAsync(cores[n], tr_init[n], cnt * 8, cudaMemcpyDeviceToDevice, st));
    }
    double** table = reinterpret_cast<double**>(base + L.table);
    RBKI_CUDA_TRY(cudaMemcpyAsync(table, cores, pl.N * sizeof(double*), cudaMemcpyHostToDevice, st));
    double norms[2];
    RBKI_CUDA_TRY(cudaMemcpyAsync(norms, o.norms, sizeof(norms), cudaMemcpyDeviceToHost, st));
    RBKI_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> hf(tr_maxit, std::nan(""));
    int sweeps = 0;
    RBKI_TRY(tr_run(pl.N, cdims, tr_ranks, o.core, norms[1], cores, table, tr_maxit, tr_tol,
                    reinterpret_cast<double*>(base + L.trws), hf.data(), &sweeps, st));
    for (int n = 0; n < pl.N; ++n)
        RBKI_TRY(tr_contract_cuda(cores[n], o.factors[n], tr_ranks[(n + pl.N - 1) % pl.N], tk->ranks[n], tr_ranks[n],
                                  pl.dims[n], tr_cores[n], st));
    if (fits) {
        RBKI_CUDA_TRY(cudaMemcpyAsync(fits, hf.data(), tr_maxit * sizeof(double), cudaMemcpyHostToDevice, st));
        RBKI_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return RBKI_OK;
}

// ---- batches and divide-and-conquer (Sec. 4.1.2) ----
static rbki_status batch_plans(int32_t count, const rbki_tensor* X, const rbki_params* prm, std::vector<Plan>& pls,
                               std::vector<size_t>& off, size_t* total) {
    if (count < 1 || !X || !prm) return set_error(RBKI_E_INVAL, "batch: count < 1 or NULL arrays");
    pls.resize(count);
    off.resize(count);
    size_t t = 0;
    for (int k = 0; k < count; ++k) {
        if (prm[k].flags & RBKI_FLAG_HOST_IO) return set_error(RBKI_E_UNSUPPORTED, "batch items use device buffers");
        RBKI_TRY(make_plan(&X[k], &prm[k], pls[k]));
        carve(pls[k], nullptr);
        off[k] = t;
        t += (pls[k].ws_bytes + 255) & ~(size_t)255;
    }
    *total = t + 256;
    return RBKI_OK;
}

rbki_status rbki_tucker_batch_workspace(int32_t count, const rbki_tensor* X, const rbki_params* prm, size_t* bytes) {
    if (!bytes) return set_error(RBKI_E_INVAL, "bytes is NULL");
    std::vector<Plan> pls;
    std::vector<size_t> off;
    return batch_plans(count, X, prm, pls, off, bytes);
}

rbki_status rbki_tucker_batch(int32_t count, const rbki_tensor* X, const rbki_params* prm, void* workspace,
                              size_t workspace_bytes, const rbki_tucker_out* out, void* stream) {
    std::vector<Plan> pls;
    std::vector<size_t> off;
    size_t need = 0;
    RBKI_TRY(batch_plans(count, X, prm, pls, off, &need));
    if (!out) return set_error(RBKI_E_INVAL, "out is NULL");
    for (int k = 0; k < count; ++k) {
        if (!out[k].core) return set_error(RBKI_E_INVAL, "out[k].core is NULL");
        for (int n = 0; n < pls[k].N; ++n)
            if (!out[k].factors[n]) return set_error(RBKI_E_INVAL, "out[k].factors[n] is NULL");
    }
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<cudaStream_t> items;
    RBKI_TRY(item_streams(st, count, items));
    cudaEvent_t ev;
    RBKI_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    RBKI_CUDA_TRY(cudaEventRecord(ev, st));
    for (int k = 0; k < count && k < MAX_ITEMS; ++k) RBKI_CUDA_TRY(cudaStreamWaitEvent(items[k], ev, 0));
    rbki_status rs = RBKI_OK;
    for (int k = 0; k < count && rs >= 0; ++k) {
        carve(pls[k], static_cast<char*>(workspace) + off[k]);
        pls[k].xin = X[k].data;
        rs = run_tucker(pls[k], &out[k], items[k]);
    }
    for (int k = 0; k < count && k < MAX_ITEMS; ++k) {
        RBKI_CUDA_TRY(cudaEventRecord(ev, items[k]));
        RBKI_CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
    }
    cudaEventDestroy(ev);
    return rs;
}

rbki_status rbki_split_mode(const rbki_tensor* X, int32_t mode, int32_t parts, void* const* dst, void* stream) {
    RBKI_TRY(validate_tensor(X));
    if (mode < 0 || mode >= X->order) return set_error(RBKI_E_INVAL, "mode out of range");
    if (parts < 1 || parts > X->dims[mode]) return set_error(RBKI_E_INVAL, "need 1 <= parts <= I_mode");
    if (!dst) return set_error(RBKI_E_INVAL, "dst is NULL");
    for (int k = 0; k < parts; ++k)
        if (!dst[k]) return set_error(RBKI_E_INVAL, "dst[k] is NULL");
    int64_t A = 1, C = 1;
    for (int k = 0; k < mode; ++k) A *= X->dims[k];
    for (int k = mode + 1; k < X->order; ++k) C *= X->dims[k];
    return split_mode_cuda(X->data, X->dtype, A, X->dims[mode], C, parts, dst, (cudaStream_t)stream);
}

rbki_status rbki_sample_units(uint64_t seed, int32_t mode, int64_t n_units, int64_t kept, int32_t* units,
                              void* stream) {
    if (!units) return set_error(RBKI_E_INVAL, "units is NULL");
    return sample_units_cuda(seed, mode, n_units, kept, units, (cudaStream_t)stream);
}

rbki_status rbki_syev_workspace(int32_t n, size_t* bytes) {
    if (!bytes || n < 1 || n > 256) return set_error(RBKI_E_INVAL, "n out of range");
    *bytes = syev_scratch_doubles(n) * sizeof(double);
    return RBKI_OK;
}

rbki_status rbki_syev(const double* A, int32_t n, double* w, double* V, void* workspace,
                      size_t workspace_bytes, void* stream) {
    size_t need = 0;
    RBKI_TRY(rbki_syev_workspace(n, &need));
    if (!A || !w || !V) return set_error(RBKI_E_INVAL, "NULL argument");
    if (!workspace || workspace_bytes < need) return set_error(RBKI_E_NOMEM, "workspace too small");
    return syev_cuda(A, n, w, V, (double*)workspace, (cudaStream_t)stream);
}

}  // extern "C"
