// C-ABI runtime of the DOT hot path: context, setters, evaluation pipeline.
//
// Pipeline of one evaluation (each step a kernel of this library):
//   PaLS -> mu (fields.cu) -> operator coefficients -> right-hand sides [BW | CV]
//   -> block Krylov solve (krylov.cu) -> restriction S = (CV)^T U, R_s, f
//   -> sensitivity g_mu -> PaLS chain rule g_p.
// Results are cached per stage and invalidated by the setters they depend on.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dot.h"
#include "dot_internal.h"

using namespace dotk;

namespace {

// NVTX range over one phase of an evaluation (host side; a profiler shows it over the
// kernels the phase queues).  Costs a function call when no tool is attached.
struct Phase {
    explicit Phase(const char* name) { nvtxRangePushA(name); }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase&) = delete;
    Phase& operator=(const Phase&) = delete;
};

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CK(expr)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(DOT_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));       \
    } while (0)

#define TRY(expr)                  \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != DOT_OK) return rc_; \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

int ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return DOT_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return fail(DOT_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    }
    b.bytes = bytes;
    return DOT_OK;
}

// ensure() without an error record: false (and b empty) when the allocation fails.
bool try_ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.p && b.bytes >= bytes) return true;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return false;
    }
    b.bytes = bytes;
    return true;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

struct Tuning {
    bool tma;            // TMA-staged stencil
    int blocks_per_sm;   // vector kernels
    bool fused = false;  // direction update inside the TMA stencil
};

// Host-side state of one block solve in progress.
struct SolveRun {
    bool active = false, done = true;
    int kp = 0, kr = 0;
    int64_t n = 0;
    bool mixed = false;
    ElemKind inner = EK_F64;
    size_t ei = 8;
    Launch L{}, Lv{};
    ColState st{};
    DirRing ring;
    TmaStencil tma;
    bool tma_ready = false;
    bool fused_ready = false;  // the fused kernel's tensor maps and launch shape are set up
    bool fused = false;  // the direction update runs inside the TMA stencil
    OpRaw oi{}, o64{};
    double delta = 0.0;
    int maxit = 0;
    int it = 0, act = 0, upd = 0;
    bool first = true;
    Tuning cfg{true, 8, false};
    // autotuning: candidates tried one batch each, then the fastest is kept
    std::vector<Tuning> cands;
    std::vector<float> cand_ms;
    int cand_at = -1;
    bool batch_timed = false;
    // graph of one steady batch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_failed = false;
    float ms_rhs = 0.f;
};

void run_release_graph(SolveRun& r) {
    if (r.exec) cudaGraphExecDestroy(r.exec);
    if (r.graph) cudaGraphDestroy(r.graph);
    r.exec = nullptr;
    r.graph = nullptr;
}

struct TunedChoice {
    bool valid = false;
    int64_t n = 0;
    int kp = 0, inner = 0;
    bool tma = true;
    int blocks_per_sm = 8;
    bool fused = false;
    float ms = 0.f;
};

}  // namespace

int dotk::record_error(int code, const std::string& msg) { return fail(code, msg); }

struct dot_ctx {
    int device = 0;
    int num_sms = 152;
    cudaStream_t own = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int* h_flag = nullptr;  // pinned host words for polling the column counters

    bool grid_set = false;
    int nx = 0, ny = 0, nz = 0;
    double h = 0;
    int bc[6] = {0, 0, 0, 0, 0, 0};
    int64_t n = 0;
    double w = 0.0;

    bool D_set = false;
    DevBuf D;
    int mu_mode = 0;  // 0 unset, 1 direct, 2 PaLS
    DevBuf mu, phi, wdmu;
    int m0 = 0;
    DevBuf p;
    double mu_in = 0, mu_out = 0, cut = 0, eps = 1, gamma = 0;

    bool coef_valid = false;
    DevBuf cf64, dinv64, cf32, dinv32;  // packed (cx, cy, cz, dre) and Jacobi inverse diagonal
    DevBuf cf8;                         // 32-byte FP32 records (coefficients + Jacobi inverse)

    int ns = 0, nd = 0;
    DevBuf rpB, ciB, vB, rpC, ciC, vC, cpC, rwC, vCc;

    int ls = 0, ld = 0;
    DevBuf W, V;

    bool M_set = false;
    DevBuf M, MW, P;
    bool P_valid = false;

    int prec = DOT_PREC_FP64;
    double rtol = 1e-10;
    int maxit = 0;
    double delta = 1e-3;  // reliable-update threshold of the mixed-precision recurrence
    int stencil_mode = 2;  // 2: TMA stencil with the direction update fused, 1: TMA stencil, 0: direct loads

    // block vectors: FP64 right-hand side, solution and true residual; the recurrence
    // vectors x~, r~, p, q in the inner precision
    DevBuf b64, x64, r64, xi, ri, pi, qi;
    // per-column state (one allocation) and per-block partial sums
    DevBuf colbuf, partA, partB, gcount;
    bool fields_valid = false;
    int fields_status = DOT_OK;
    int kp = 0;

    bool post_valid = false;
    DevBuf Tm, S, Rs, f, gmu, gp, J, tmp;
    DevBuf bcount, boffs, bcell, bdval;  // band lists of dmu/dp per RBF (J_p and the Jacobian tensor)

    dot_stats stats{};

    // block solve in progress, graph replay and autotuning
    SolveRun run;
    bool use_graphs = true;
    bool autotune = false;
    TunedChoice tuned;
    Tuning last_cfg{false, -1, false};  // launch configuration of the last solve (blocks_per_sm -1: none yet)
    bool last_fused = false;     // the last solve ran the direction update inside the stencil
    int ring_cap = kDirRingMax;  // most direction-ring slots to try (dot_set_direction_ring)
    cudaEvent_t bev[2] = {nullptr, nullptr};

    // kernel timing (dot_set_kernel_timing)
    bool timing = false;
    // per-iteration events (4 x 8), refresh pair, one per flush of a batch (up to 4)
    cudaEvent_t tev[8 * 4 + 2 + 4] = {};
    dot_kernel_timing kt{};
};

namespace {

bool cplx(const dot_ctx* c) { return c->w != 0.0; }
size_t esz64(const dot_ctx* c) { return cplx(c) ? 16 : 8; }
size_t esz32(const dot_ctx* c) { return cplx(c) ? 8 : 4; }
void count(dot_ctx* c, int launches) { c->stats.kernel_launches += launches; }

void invalidate_coef(dot_ctx* c) {
    c->coef_valid = false;
    c->fields_valid = false;
    c->post_valid = false;
}
void invalidate_fields(dot_ctx* c) {
    c->fields_valid = false;
    c->post_valid = false;
}

int need_ctx(dot_ctx* c) {
    if (!c) return fail(DOT_EINVAL, "null context");
    CK(cudaSetDevice(c->device));
    return DOT_OK;
}

int need_grid(dot_ctx* c) {
    TRY(need_ctx(c));
    if (!c->grid_set) return fail(DOT_ESTATE, "dot_set_grid has not been called");
    return DOT_OK;
}

int upload(dot_ctx* c, DevBuf& b, const void* host, size_t bytes) {
    TRY(ensure(b, bytes));
    CK(cudaMemcpyAsync(b.p, host, bytes, cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    return DOT_OK;
}

int kp_limit_check(dot_ctx* c) {
    if (c->ls + c->ld > 1024) return fail(DOT_EINVAL, "ls + ld exceeds 1024");
    return DOT_OK;
}

OpRaw op64(const dot_ctx* c) {
    OpRaw o;
    o.cf = c->cf64.p;
    o.dinv = c->dinv64.p;
    o.w = c->w;
    o.nx = c->nx;
    o.ny = c->ny;
    o.nz = c->nz;
    return o;
}
OpRaw op32(const dot_ctx* c) {
    OpRaw o = op64(c);
    o.cf = c->cf32.p;
    o.dinv = c->dinv32.p;
    return o;
}

// ------------------------------------------------------------------ stages
int ensure_coefficients(dot_ctx* c) {
    if (c->coef_valid) return DOT_OK;
    Phase ph("dot: PaLS absorption and operator coefficients");
    if (!c->D_set) return fail(DOT_ESTATE, "dot_set_diffusion has not been called");
    if (c->mu_mode == 0) return fail(DOT_ESTATE, "neither dot_set_mua nor dot_set_pals has been called");
    const int64_t n = c->n;
    if (c->mu_mode == 2) {
        TRY(ensure(c->mu, n * 8));
        TRY(ensure(c->phi, n * 8));
        TRY(ensure(c->wdmu, n * 8));
        CK(pals_eval(c->p.as<double>(), c->m0, c->mu_in, c->mu_out, c->cut, c->eps, c->gamma, c->nx, c->ny, c->nz,
                     c->h, c->phi.as<double>(), c->mu.as<double>(), c->wdmu.as<double>(), c->s));
    }
    TRY(ensure(c->cf64, n * 32));
    TRY(ensure(c->cf32, n * 16));
    TRY(ensure(c->dinv64, n * 16));
    TRY(ensure(c->dinv32, n * 8));
    TRY(ensure(c->cf8, n * 32));
    CK(build_coefficients(c->D.as<double>(), c->mu.as<double>(), c->nx, c->ny, c->nz, c->h, c->bc, c->w, c->cf64.p,
                          c->dinv64.p, cplx(c), c->cf32.p, c->dinv32.p, c->cf8.p, c->s));
    count(c, c->mu_mode == 2 ? 2 : 1);
    c->coef_valid = true;
    return DOT_OK;
}

int alloc_colstate(dot_ctx* c, int kp, int max_grid, ColState* st) {
    const size_t n16 = (size_t)kp * 16, n8 = (size_t)kp * 8, n4 = (size_t)kp * 4;
    const size_t bytes = (4 + kDirRingMax) * n16 + 7 * n8 + 6 * n4 + 64;
    TRY(ensure(c->colbuf, bytes));
    const size_t groups = ((size_t)max_grid + kReduceGroup - 1) / kReduceGroup;
    TRY(ensure(c->partA, ((size_t)max_grid + groups) * kp * 16));
    TRY(ensure(c->partB, ((size_t)max_grid + groups) * kp * 8));
    TRY(ensure(c->gcount, groups * 4));
    CK(cudaMemsetAsync(c->colbuf.p, 0, bytes, c->s));
    CK(cudaMemsetAsync(c->gcount.p, 0, groups * 4, c->s));
    char* q = c->colbuf.as<char>();
    auto take = [&](size_t b) {
        char* r = q;
        q += b;
        return r;
    };
    st->rho = reinterpret_cast<double2*>(take(n16));
    st->rho_prev = reinterpret_cast<double2*>(take(n16));
    st->alpha = reinterpret_cast<double2*>(take(n16));
    st->alpha_hist = reinterpret_cast<double2*>(take(kDirRingMax * n16));
    st->beta = reinterpret_cast<double2*>(take(n16));
    st->rr = reinterpret_cast<double*>(take(n8));
    st->maxr = reinterpret_cast<double*>(take(n8));
    st->scale = reinterpret_cast<double*>(take(n8));
    st->ratio = reinterpret_cast<double*>(take(n8));
    st->tol2 = reinterpret_cast<double*>(take(n8));
    st->bb64 = reinterpret_cast<double*>(take(n8));
    st->rr64 = reinterpret_cast<double*>(take(n8));
    st->active = reinterpret_cast<int*>(take(n4));
    st->upd = reinterpret_cast<int*>(take(n4));
    st->iters = reinterpret_cast<int*>(take(n4));
    st->updates = reinterpret_cast<int*>(take(n4));
    st->since = reinterpret_cast<int*>(take(n4));
    st->status = reinterpret_cast<int*>(take(n4));
    int* misc = reinterpret_cast<int*>(take(64));
    st->n_active = misc;
    st->n_update = misc + 1;
    st->counter = reinterpret_cast<unsigned*>(misc + 4);
    st->error = misc + 6;
    st->partA = c->partA.as<double2>();
    st->partB = c->partB.as<double>();
    st->groupA = st->partA + (size_t)max_grid * kp;
    st->groupB = st->partB + (size_t)max_grid * kp;
    st->gcount = c->gcount.as<unsigned>();
    return DOT_OK;
}

// Reads n_active, n_update and the kernel error word after the work queued so far.
int read_counts(dot_ctx* c, const ColState& st, int* act, int* upd) {
    CK(cudaMemcpyAsync(c->h_flag, st.n_active, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    *act = c->h_flag[0];
    *upd = c->h_flag[1];
    if (c->h_flag[6] != 0) return fail(DOT_ETIMEOUT, "a bounded wait in the stencil kernel ran out");
    return DOT_OK;
}

constexpr int kPoll = 8;  // iterations between host polls

int collect_step_timing(dot_ctx* c, int steps, bool first_without_p, int H, bool fused) {
    for (int m = 0; m < steps; ++m) {
        float ms = 0.f;
        if (!(first_without_p && m == 0) && !fused) {
            CK(cudaEventElapsedTime(&ms, c->tev[4 * m], c->tev[4 * m + 1]));
            c->kt.ms[2] += ms;
            c->kt.launches[2] += 1;
        }
        CK(cudaEventElapsedTime(&ms, c->tev[4 * m + 1], c->tev[4 * m + 2]));
        c->kt.ms[0] += ms;
        c->kt.launches[0] += 1;
        CK(cudaEventElapsedTime(&ms, c->tev[4 * m + 2], c->tev[4 * m + 3]));
        c->kt.ms[1] += ms;
        c->kt.launches[1] += 1;
        if (m % H == H - 1) {
            CK(cudaEventElapsedTime(&ms, c->tev[4 * m + 3], c->tev[34 + m / H]));
            c->kt.ms[4] += ms;
            c->kt.launches[4] += 1;
        }
    }
    return DOT_OK;
}

// ------------------------------------------------------------ resumable solve
// A block solve of [BW | CV] (already in b64) into x64 runs as begin / (advance, poll)*
// / end.  advance() queues one batch of kPoll iterations (replayed from a CUDA graph once the launch configuration is
// settled); poll() waits for the context's stream, reads the column counters and runs a
// reliable-update round if a column asked for one.

int apply_tuning(dot_ctx* c, SolveRun& r, const Tuning& t) {
    r.cfg = t;
    r.Lv = vector_launch(r.n, r.kp, vector_width(r.inner), c->num_sms);
    const int64_t need = (r.n + r.Lv.slots - 1) / r.Lv.slots;
    const int64_t g = (int64_t)c->num_sms * t.blocks_per_sm;
    r.Lv.grid = (int)std::max<int64_t>(1, std::min(need, g));
    // the flush holds 8 directions per thread: two 256-thread blocks (one 1024-thread
    // block) fit per SM, so it runs one full wave of those
    const int64_t gf = (int64_t)c->num_sms * (r.Lv.threads > 256 ? 1 : 2);
    r.ring.flush_grid = (int)std::max<int64_t>(1, std::min(need, gf));
    if (t.tma && !r.tma_ready) {
        CK(tma_stencil_prepare(r.inner, r.ring, c->cf32.p, c->nx, c->ny, c->nz, r.kp, c->num_sms, &r.tma));
        r.tma.fused = false;
        // the fused kernel is an option on top of the TMA stencil: if its tensor maps or
        // launch shape cannot be set up, the solve runs the separate direction pass
        if (c->stencil_mode == 2 && dpq_eligible(r.inner, c->nx, c->ny, r.kp) &&
            dpq_prepare(r.inner, r.ring, c->ri.p, c->cf8.p, c->nx, c->ny, c->nz, r.kp, c->num_sms, &r.tma) !=
                cudaSuccess) {
            cudaGetLastError();
            r.tma.fused = false;
        }
        r.tma_ready = true;
        r.fused_ready = r.tma.fused;
    }
    // the iterations fuse the direction update into the stencil exactly when this
    // configuration asks for it (kry_step follows r.tma.fused), so that an autotuner
    // candidate with the separate direction pass runs, and is timed and counted, as one
    r.tma.fused = r.fused_ready && t.fused;
    r.fused = t.tma && r.tma.fused;
    run_release_graph(r);
    r.graph_failed = false;
    return DOT_OK;
}

int solve_begin(dot_ctx* c, int kp, int kr) {
    SolveRun& r = c->run;
    run_release_graph(r);
    r = SolveRun();
    r.active = true;
    r.done = false;
    r.kp = kp;
    r.kr = kr;
    r.n = c->n;
    r.mixed = c->prec == DOT_PREC_MIXED;
    r.inner = cplx(c) ? (r.mixed ? EK_C64 : EK_C128) : (r.mixed ? EK_F32 : EK_F64);
    r.ei = r.mixed ? esz32(c) : esz64(c);
    r.L = krylov_launch(r.n, kp, c->num_sms);
    const Launch Lmax = vector_launch(r.n, kp, vector_width(r.inner), c->num_sms);
    const int gmax = (int)std::min<int64_t>((r.n + Lmax.slots - 1) / Lmax.slots, (int64_t)c->num_sms * 16);
    TRY(alloc_colstate(c, kp, std::max(r.L.grid, std::max(gmax, 1)), &r.st));
    for (DevBuf* b : {&c->xi, &c->ri, &c->qi}) TRY(ensure(*b, (size_t)r.n * kp * r.ei));
    // direction ring: as many slots (8, 4 or 2) as device memory allows
    const size_t slot_bytes = (size_t)r.n * kp * r.ei;
    r.ring = DirRing{};
    for (int H = c->ring_cap; H >= 2; H /= 2) {
        if (kPoll % H == 0 && try_ensure(c->pi, (size_t)H * slot_bytes)) {
            r.ring = DirRing{c->pi.p, (int64_t)r.n * kp, H};
            break;
        }
    }
    if (!r.ring.base)
        return fail(DOT_ENOMEM, "cudaMalloc of the direction ring (2 x " + std::to_string(slot_bytes) +
                                    " bytes) failed");
    r.oi = r.mixed ? op32(c) : op64(c);
    r.o64 = op64(c);
    r.delta = r.mixed ? c->delta : 0.0;
    r.maxit = c->maxit > 0 ? c->maxit : 10 * (c->nx + c->ny + c->nz);
    const bool tma_ok = c->stencil_mode != 0 && tma_stencil_eligible(r.inner, c->nx, c->ny, kp);
    const bool fused_ok = tma_ok && c->stencil_mode == 2 && dpq_eligible(r.inner, c->nx, c->ny, kp);
    // five 256-thread blocks per SM: one wave at the update kernel's register limit
    Tuning base{tma_ok, 5, fused_ok};
    if (c->autotune) {
        const bool have = c->tuned.valid && c->tuned.n == r.n && c->tuned.kp == kp && c->tuned.inner == (int)r.inner;
        if (have) {
            base = Tuning{c->tuned.tma && tma_ok, c->tuned.blocks_per_sm, c->tuned.fused && fused_ok};
        } else {
            for (int bps : {4, 5, 8, 16}) {
                r.cands.push_back(Tuning{false, bps, false});
                if (tma_ok) r.cands.push_back(Tuning{true, bps, false});
                if (fused_ok) r.cands.push_back(Tuning{true, bps, true});
            }
            r.cand_ms.assign(r.cands.size(), 0.f);
            r.cand_at = 0;
            base = r.cands[0];
        }
    }
    TRY(apply_tuning(c, r, base));
    CK(solve_start(r.inner, r.oi, c->b64.p, c->x64.p, c->xi.p, c->ri.p, r.ring.base, r.n, kp, r.st, c->rtol, r.L,
                   c->s));
    count(c, 2);
    TRY(read_counts(c, r.st, &r.act, &r.upd));
    r.done = r.act == 0;
    return DOT_OK;
}

int launch_batch(dot_ctx* c, SolveRun& r, bool first_batch) {
    for (int m = 0; m < kPoll; ++m) {
        const bool with_p = !(first_batch && m == 0);
        CK(kry_step(r.inner, r.oi, c->xi.p, c->ri.p, r.ring, m, c->qi.p, r.n, r.kp, r.st, r.delta, r.maxit, with_p,
                    r.Lv, r.cfg.tma ? &r.tma : nullptr, c->s, c->timing ? &c->tev[4 * m] : nullptr,
                    c->timing ? &c->tev[34 + m / r.ring.H] : nullptr));
    }
    return DOT_OK;
}

// Queue one batch of kPoll iterations.
int solve_advance(dot_ctx* c) {
    SolveRun& r = c->run;
    if (r.done) return DOT_OK;
    Phase ph("dot: Krylov iterations");
    const bool first_batch = r.first;
    const bool tuning = r.cand_at >= 0;
    r.batch_timed = tuning;
    if (tuning) CK(cudaEventRecord(c->bev[0], c->s));
    const bool use_graph = c->use_graphs && !first_batch && !tuning && !r.graph_failed;
    if (use_graph && !r.exec) {
        // capture one steady batch of the settled configuration; fall back to direct
        // launches if the stream cannot be captured
        cudaError_t e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int rc = launch_batch(c, r, false);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(c->s, &g);
            if (rc == DOT_OK && e == cudaSuccess && g) {
                r.graph = g;
                e = cudaGraphInstantiate(&r.exec, g, 0);
            }
            if (rc != DOT_OK || e != cudaSuccess || !r.exec) {
                cudaGetLastError();
                run_release_graph(r);
                r.graph_failed = true;
            }
        } else {
            cudaGetLastError();
            r.graph_failed = true;
        }
    }
    if (use_graph && r.exec) {
        CK(cudaGraphLaunch(r.exec, c->s));
    } else {
        TRY(launch_batch(c, r, first_batch));
    }
    // direction, stencil and update per iteration (the first of a solve has no direction;
    // fused: stencil with direction and update), plus the ring flushes
    count(c, (r.fused ? kPoll * 2 : kPoll * 3 - (first_batch ? 1 : 0)) + kPoll / r.ring.H);
    if (tuning) CK(cudaEventRecord(c->bev[1], c->s));
    r.first = false;
    r.it += kPoll;
    return DOT_OK;
}

// Wait for the queued batch, read the counters, refresh if asked, and decide completion.
int solve_poll(dot_ctx* c) {
    SolveRun& r = c->run;
    if (r.done) return DOT_OK;
    const bool first_batch = r.it == kPoll;
    TRY(read_counts(c, r.st, &r.act, &r.upd));
    if (c->timing) TRY(collect_step_timing(c, kPoll, first_batch, r.ring.H, r.fused));
    if (r.batch_timed) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->bev[0], c->bev[1]));
        if (!first_batch) {  // the first batch is one launch short: time the candidate again
            r.cand_ms[r.cand_at] = ms;
            ++r.cand_at;
        }
        if (r.cand_at >= (int)r.cands.size()) {
            int best = 0;
            for (int i = 1; i < (int)r.cands.size(); ++i)
                if (r.cand_ms[i] < r.cand_ms[best]) best = i;
            c->tuned.valid = true;
            c->tuned.n = r.n;
            c->tuned.kp = r.kp;
            c->tuned.inner = (int)r.inner;
            c->tuned.tma = r.cands[best].tma;
            c->tuned.fused = r.cands[best].fused;
            c->tuned.blocks_per_sm = r.cands[best].blocks_per_sm;
            c->tuned.ms = r.cand_ms[best];
            r.cand_at = -1;
            TRY(apply_tuning(c, r, r.cands[best]));
        } else {
            TRY(apply_tuning(c, r, r.cands[r.cand_at]));
        }
        r.batch_timed = false;
    }
    if (r.upd > 0) {
        Phase ph("dot: reliable update (FP64 true residual)");
        if (c->timing) CK(cudaEventRecord(c->tev[32], c->s));
        CK(solve_refresh(r.inner, r.oi, r.o64, c->b64.p, c->x64.p, c->r64.p, c->xi.p, c->ri.p, r.n, r.kp, r.st,
                         c->rtol, r.maxit, r.L, c->num_sms, c->s));
        count(c, 3);
        if (c->timing) {
            CK(cudaEventRecord(c->tev[33], c->s));
            CK(cudaEventSynchronize(c->tev[33]));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, c->tev[32], c->tev[33]));
            c->kt.ms[3] += ms;
            c->kt.launches[3] += 3;
            c->kt.bytes[3] += (double)r.act * r.n * (6.0 * esz64(c) + 3.0 * r.ei) + (double)r.n * 4.0 * 8.0;
        }
        TRY(read_counts(c, r.st, &r.act, &r.upd));
    }
    r.done = r.act == 0 || r.it >= r.maxit + 2 * kPoll;
    return DOT_OK;
}

// Promote the last corrections, read the per-column results and fill the statistics.
int solve_end(dot_ctx* c) {
    SolveRun& r = c->run;
    const int kp = r.kp;
    c->last_cfg = r.cfg;
    c->last_fused = r.fused;
    std::vector<int> iters(kp), updates(kp), status(kp), active(kp);
    std::vector<double> rr(kp), bb(kp);
    CK(cudaMemcpyAsync(status.data(), r.st.status, kp * 4, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    bool any_bad = r.act > 0;
    for (int j = 0; j < kp; ++j) any_bad = any_bad || status[j] != DOT_OK;
    CK(solve_finish(r.inner, r.o64, c->b64.p, c->x64.p, c->r64.p, c->xi.p, r.n, kp, r.st, any_bad, r.L, c->num_sms,
                    c->s));
    count(c, any_bad ? 2 : 1);
    CK(cudaMemcpyAsync(iters.data(), r.st.iters, kp * 4, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(updates.data(), r.st.updates, kp * 4, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(status.data(), r.st.status, kp * 4, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(rr.data(), r.st.rr64, kp * 8, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(bb.data(), r.st.bb64, kp * 8, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(active.data(), r.st.active, kp * 4, cudaMemcpyDeviceToHost, c->s));
    CK(cudaEventRecord(c->ev[2], c->s));
    CK(cudaStreamSynchronize(c->s));
    run_release_graph(r);
    for (int j = 0; j < kp; ++j)
        if (active[j] && status[j] == DOT_OK) status[j] = DOT_ENOTCONV;
    if (c->timing) {
        // algorithmic bytes of the Krylov kernels: every element of a running column read or
        // written once per launch (stencil: p, q; update: r~, q read, r~ written; direction:
        // r~, old p read, new p written; flush: each direction once, x~ read and written
        // once per ring), coefficients once per launch
        double ci = 0.0;
        int itmax = 0;
        for (int j = 0; j < kp; ++j) {
            ci += iters[j];
            itmax = std::max(itmax, iters[j]);
        }
        const double nn = (double)r.n, rs = r.mixed ? 4.0 : 8.0;
        if (r.fused) {
            // fused launches read r~ and the old direction and write the new direction and
            // q (4 vectors) and one 32-byte record per cell; the first iteration of the
            // solve is a plain stencil (p and q, 16 bytes of coefficients per cell)
            double first = 0.0;
            for (int j = 0; j < kp; ++j) first += iters[j] > 0 ? 1.0 : 0.0;
            c->kt.bytes[0] += (ci - first) * nn * 4.0 * r.ei + first * nn * 2.0 * r.ei + itmax * nn * 32.0;
        } else {
            c->kt.bytes[0] += ci * nn * 2.0 * r.ei + itmax * nn * 4.0 * rs;
            c->kt.bytes[2] += ci * nn * 3.0 * r.ei + itmax * nn * r.ei;
        }
        c->kt.bytes[1] += ci * nn * 3.0 * r.ei + itmax * nn * r.ei;
        c->kt.bytes[4] += ci * nn * r.ei + ci / r.ring.H * nn * 2.0 * r.ei;
    }
    float ms_solve = 0;
    cudaEventElapsedTime(&ms_solve, c->ev[1], c->ev[2]);
    int st_all = DOT_OK;
    double relmax = 0.0;
    int itmax = 0, updmax = 0;
    int64_t itsum = 0;
    for (int j = 0; j < r.kr; ++j) {
        if (status[j] == DOT_EBREAKDOWN) st_all = DOT_EBREAKDOWN;
        else if (status[j] == DOT_ENOTCONV && st_all == DOT_OK) st_all = DOT_ENOTCONV;
        if (bb[j] > 0) relmax = std::max(relmax, std::sqrt(rr[j] / bb[j]));
        itmax = std::max(itmax, iters[j]);
        updmax = std::max(updmax, updates[j]);
        itsum += iters[j];
    }
    c->stats.k = r.kr;
    c->stats.iters_max = itmax;
    c->stats.iters_sum = itsum;
    c->stats.outer_steps = updmax;
    c->stats.status = st_all;
    c->stats.relres_max = relmax;
    c->stats.columns_solved += r.kr;
    c->stats.block_solves += 1;
    c->stats.ms_setup = r.ms_rhs;
    c->stats.ms_solve = ms_solve;
    c->kp = kp;
    c->fields_status = st_all;
    c->fields_valid = true;
    c->post_valid = false;
    r.active = false;
    return DOT_OK;
}

// Checks, right-hand sides and the start of the block solve; nothing to do when the
// fields are already valid.
int fields_begin(dot_ctx* c) {
    c->run.active = false;
    if (c->fields_valid) return DOT_OK;
    Phase ph("dot: right-hand sides and solve start");
    TRY(ensure_coefficients(c));
    if (c->ns == 0) return fail(DOT_ESTATE, "dot_set_sources has not been called");
    if (c->nd == 0) return fail(DOT_ESTATE, "dot_set_detectors has not been called");
    if (c->ls == 0 && c->ld == 0) return fail(DOT_ESTATE, "dot_set_sampling has not been called");
    TRY(kp_limit_check(c));
    const int kr = c->ls + c->ld;       // columns of the block
    const int kp = (kr + 3) & ~3;       // padded stride: 16-byte vector access in every precision
    const int64_t n = c->n;
    const size_t nk = (size_t)n * kp;
    TRY(ensure(c->b64, nk * esz64(c)));
    TRY(ensure(c->x64, nk * esz64(c)));
    TRY(ensure(c->r64, nk * esz64(c)));
    CK(cudaEventRecord(c->ev[0], c->s));
    CK(build_rhs(cplx(c), c->rpB.as<int64_t>(), c->ciB.as<int32_t>(), c->vB.as<double>(), c->W.as<double>(), c->ns,
                 c->ls, c->rpC.as<int64_t>(), c->ciC.as<int32_t>(), c->vC.as<double>(), c->V.as<double>(), c->nd,
                 c->ld, n, kp, c->b64.p, c->s));
    count(c, 1);
    CK(cudaEventRecord(c->ev[1], c->s));
    TRY(solve_begin(c, kp, kr));
    float ms_rhs = 0.f;
    cudaEventElapsedTime(&ms_rhs, c->ev[0], c->ev[1]);
    c->run.ms_rhs = ms_rhs;
    return DOT_OK;
}

bool fields_pending(dot_ctx* c) { return c->run.active && !c->run.done; }

int fields_finish(dot_ctx* c) {
    if (!c->run.active) return DOT_OK;
    return solve_end(c);
}

int ensure_fields(dot_ctx* c) {
    if (c->fields_valid) return DOT_OK;
    TRY(fields_begin(c));
    while (fields_pending(c)) {
        TRY(solve_advance(c));
        TRY(solve_poll(c));
    }
    return fields_finish(c);
}

int ensure_projection(dot_ctx* c) {
    if (c->P_valid) return DOT_OK;
    TRY(ensure(c->MW, (size_t)c->nd * std::max(c->ls, 1) * 16));
    TRY(ensure(c->P, (size_t)std::max(c->ld, 1) * std::max(c->ls, 1) * 16));
    CK(data_projection(cplx(c), c->M.as<double>(), c->nd, c->ns, c->W.as<double>(), c->ls, c->V.as<double>(), c->ld,
                       c->MW.as<double>(), c->P.as<double>(), c->s));
    count(c, 2);
    c->P_valid = true;
    return DOT_OK;
}

int ensure_post(dot_ctx* c) {
    TRY(ensure_fields(c));
    if (c->post_valid) return DOT_OK;
    Phase ph("dot: restriction and misfit");
    if (c->M_set) TRY(ensure_projection(c));
    const size_t nr = (size_t)std::max(c->ls, 1) * std::max(c->ld, 1);
    TRY(ensure(c->Tm, (size_t)c->nd * std::max(c->ls, 1) * 16));
    TRY(ensure(c->S, nr * 16));
    TRY(ensure(c->Rs, nr * 16));
    TRY(ensure(c->f, 16));
    CK(restriction_misfit(cplx(c), c->x64.p, c->kp, c->ls, c->cpC.as<int64_t>(), c->rwC.as<int32_t>(),
                          c->vCc.as<double>(), c->nd, c->V.as<double>(), c->ld, c->P.as<double>(), c->M_set,
                          c->Tm.as<double>(), c->S.as<double>(), c->Rs.as<double>(), c->f.as<double>(), c->s));
    count(c, 2);
    c->post_valid = true;
    return DOT_OK;
}

// Band lists of dmu/dp at the current PaLS parameters (ensure_coefficients has run): count
// per RBF, exclusive offsets on the host, then the cells and their five derivatives.
int build_band_lists(dot_ctx* c) {
    const int m0 = c->m0;
    TRY(ensure(c->bcount, (size_t)m0 * 8));
    TRY(ensure(c->boffs, (size_t)(m0 + 1) * 8));
    CK(pals_band_count(c->p.as<double>(), m0, c->gamma, c->nx, c->ny, c->nz, c->h, c->wdmu.as<double>(),
                       c->bcount.as<int64_t>(), c->s));
    std::vector<int64_t> cnt(m0), offs(m0 + 1, 0);
    CK(cudaMemcpyAsync(cnt.data(), c->bcount.p, (size_t)m0 * 8, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    for (int j = 0; j < m0; ++j) offs[j + 1] = offs[j] + cnt[j];
    CK(cudaMemcpyAsync(c->boffs.p, offs.data(), (size_t)(m0 + 1) * 8, cudaMemcpyHostToDevice, c->s));
    TRY(ensure(c->bcell, (size_t)std::max<int64_t>(offs[m0], 1) * 8));
    TRY(ensure(c->bdval, (size_t)std::max<int64_t>(offs[m0], 1) * 40));
    CK(pals_band_fill(c->p.as<double>(), m0, c->gamma, c->nx, c->ny, c->nz, c->h, c->wdmu.as<double>(),
                      c->boffs.as<int64_t>(), c->bcell.as<int64_t>(), c->bdval.as<double>(), c->s));
    CK(cudaStreamSynchronize(c->s));  // the host offsets must outlive the copy
    count(c, 2);
    return DOT_OK;
}

// CSC (colptr, rows) -> CSR by voxel with the column index, on the host.
void csc_to_csr(int64_t n, int ncol, const int64_t* colptr, const int32_t* rows, const double* vals,
                std::vector<int64_t>& rp, std::vector<int32_t>& ci, std::vector<double>& cv) {
    const int64_t nnz = colptr[ncol];
    rp.assign(n + 1, 0);
    for (int64_t t = 0; t < nnz; ++t) rp[rows[t] + 1]++;
    for (int64_t v = 0; v < n; ++v) rp[v + 1] += rp[v];
    ci.resize(nnz);
    cv.resize(nnz);
    std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
    for (int col = 0; col < ncol; ++col)
        for (int64_t t = colptr[col]; t < colptr[col + 1]; ++t) {
            const int64_t dst = fill[rows[t]]++;
            ci[dst] = col;
            cv[dst] = vals[t];
        }
}

int check_csc(const dot_ctx* c, int ncol, const int64_t* colptr, const int32_t* rows, const double* vals) {
    if (ncol <= 0) return fail(DOT_EINVAL, "number of columns must be positive");
    if (!colptr || (!rows && colptr[ncol] > 0) || (!vals && colptr[ncol] > 0))
        return fail(DOT_EINVAL, "null CSC array");
    if (colptr[0] != 0) return fail(DOT_EINVAL, "colptr[0] must be 0");
    for (int j = 0; j < ncol; ++j)
        if (colptr[j + 1] < colptr[j]) return fail(DOT_EINVAL, "colptr must be non-decreasing");
    for (int64_t t = 0; t < colptr[ncol]; ++t)
        if (rows[t] < 0 || rows[t] >= c->n) return fail(DOT_EINVAL, "row index out of range");
    return DOT_OK;
}

int copy_out_complex_or_real(dot_ctx* c, const DevBuf& src, size_t count, double* host) {
    // src holds `count` double2 values; real arithmetic returns the real parts only.
    std::vector<double> tmp(count * 2);
    CK(cudaMemcpyAsync(tmp.data(), src.p, count * 16, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (cplx(c))
        std::memcpy(host, tmp.data(), count * 16);
    else
        for (size_t t = 0; t < count; ++t) host[t] = tmp[2 * t];
    return DOT_OK;
}

int set_pals_common(dot_ctx* c, int m0, double mu_in, double mu_out, double cut, double eps, double gamma) {
    if (m0 <= 0) return fail(DOT_EINVAL, "m0 must be positive");
    if (!(eps > 0.0)) return fail(DOT_EINVAL, "eps must be positive");
    if (!(gamma >= 0.0)) return fail(DOT_EINVAL, "gamma must be non-negative");
    c->m0 = m0;
    c->mu_in = mu_in;
    c->mu_out = mu_out;
    c->cut = cut;
    c->eps = eps;
    c->gamma = gamma;
    c->mu_mode = 2;
    invalidate_coef(c);
    return DOT_OK;
}

}  // namespace

// ======================================================================== C ABI
extern "C" {

const char* dot_last_error(void) { return g_err.c_str(); }

int dot_create(dot_ctx** out, int device) {
    if (!out) return fail(DOT_EINVAL, "null output pointer");
    *out = nullptr;
    int count = 0;
    CK(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(DOT_EINVAL, "device ordinal out of range");
    CK(cudaSetDevice(device));
    dot_ctx* c = new dot_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_flag, 8 * sizeof(int));
    for (int t = 0; t < 4 && e == cudaSuccess; ++t) e = cudaEventCreate(&c->ev[t]);
    for (int t = 0; t < 38 && e == cudaSuccess; ++t) e = cudaEventCreate(&c->tev[t]);
    for (int t = 0; t < 2 && e == cudaSuccess; ++t) e = cudaEventCreate(&c->bev[t]);
    if (e != cudaSuccess) {
        dot_destroy(c);
        return fail(DOT_ECUDA, std::string("context creation: ") + cudaGetErrorString(e));
    }
    c->s = c->own;
    *out = c;
    return DOT_OK;
}

int dot_destroy(dot_ctx* c) {
    if (!c) return DOT_OK;
    cudaSetDevice(c->device);
    if (c->s) cudaStreamSynchronize(c->s);
    DevBuf* bufs[] = {&c->D, &c->mu, &c->phi, &c->wdmu, &c->p, &c->cf64, &c->dinv64, &c->cf32, &c->dinv32, &c->cf8, &c->rpB, &c->ciB, &c->vB, &c->rpC,
                      &c->ciC, &c->vC, &c->cpC, &c->rwC, &c->vCc, &c->W, &c->V, &c->M, &c->MW, &c->P, &c->b64,
                      &c->x64, &c->r64, &c->xi, &c->ri, &c->pi, &c->qi, &c->colbuf, &c->partA, &c->partB, &c->gcount, &c->Tm,
                      &c->S, &c->Rs, &c->f, &c->gmu, &c->gp, &c->J, &c->tmp, &c->bcount, &c->boffs, &c->bcell,
                      &c->bdval};
    for (DevBuf* b : bufs) release(*b);
    for (int t = 0; t < 4; ++t)
        if (c->ev[t]) cudaEventDestroy(c->ev[t]);
    for (int t = 0; t < 38; ++t)
        if (c->tev[t]) cudaEventDestroy(c->tev[t]);
    for (int t = 0; t < 2; ++t)
        if (c->bev[t]) cudaEventDestroy(c->bev[t]);
    run_release_graph(c->run);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
    return DOT_OK;
}

int dot_set_stream(dot_ctx* c, void* stream) {
    TRY(need_ctx(c));
    CK(cudaStreamSynchronize(c->s));
    c->s = stream ? static_cast<cudaStream_t>(stream) : c->own;
    return DOT_OK;
}

int dot_set_grid(dot_ctx* c, int nx, int ny, int nz, double h, const int bc[6]) {
    TRY(need_ctx(c));
    if (nx < 1 || ny < 1 || nz < 1) return fail(DOT_EINVAL, "grid dimensions must be positive");
    if ((int64_t)nx * ny * nz > (int64_t)1 << 31) return fail(DOT_EINVAL, "grid exceeds 2^31 cells");
    if (!(h > 0.0) || !std::isfinite(h)) return fail(DOT_EINVAL, "h must be positive and finite");
    if (!bc) return fail(DOT_EINVAL, "null bc array");
    for (int f = 0; f < 6; ++f)
        if (bc[f] != DOT_BC_ROBIN && bc[f] != DOT_BC_DIRICHLET) return fail(DOT_EINVAL, "bad boundary flag");
    const bool same_n = c->grid_set && (int64_t)nx * ny * nz == c->n;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->h = h;
    for (int f = 0; f < 6; ++f) c->bc[f] = bc[f];
    c->n = (int64_t)nx * ny * nz;
    c->grid_set = true;
    if (!same_n) {
        c->D_set = false;
        if (c->mu_mode == 1) c->mu_mode = 0;
        c->ns = c->nd = 0;
    }
    invalidate_coef(c);
    return DOT_OK;
}

int dot_set_omega(dot_ctx* c, double w) {
    TRY(need_ctx(c));
    if (!std::isfinite(w)) return fail(DOT_EINVAL, "omega/nu must be finite");
    if ((w != 0.0) != (c->w != 0.0)) c->P_valid = false;
    c->w = w;
    invalidate_coef(c);
    return DOT_OK;
}

int dot_set_diffusion(dot_ctx* c, const double* D) {
    TRY(need_grid(c));
    if (!D) return fail(DOT_EINVAL, "null D");
    for (int64_t v = 0; v < c->n; ++v)
        if (!(D[v] > 0.0) || !std::isfinite(D[v])) return fail(DOT_EINVAL, "D must be positive and finite");
    TRY(upload(c, c->D, D, c->n * 8));
    c->D_set = true;
    invalidate_coef(c);
    return DOT_OK;
}

int dot_set_mua(dot_ctx* c, const double* mu) {
    TRY(need_grid(c));
    if (!mu) return fail(DOT_EINVAL, "null mu");
    TRY(upload(c, c->mu, mu, c->n * 8));
    c->mu_mode = 1;
    invalidate_coef(c);
    return DOT_OK;
}

int dot_set_pals(dot_ctx* c, int m0, const double* p, double mu_in, double mu_out, double cut, double eps,
                 double gamma) {
    TRY(need_grid(c));
    if (!p) return fail(DOT_EINVAL, "null p");
    TRY(set_pals_common(c, m0, mu_in, mu_out, cut, eps, gamma));
    TRY(upload(c, c->p, p, (size_t)5 * m0 * 8));
    return DOT_OK;
}

int dot_set_pals_dev(dot_ctx* c, int m0, const double* p_dev, double mu_in, double mu_out, double cut, double eps,
                     double gamma) {
    TRY(need_grid(c));
    if (!p_dev) return fail(DOT_EINVAL, "null p");
    TRY(set_pals_common(c, m0, mu_in, mu_out, cut, eps, gamma));
    TRY(ensure(c->p, (size_t)5 * m0 * 8));
    CK(cudaMemcpyAsync(c->p.p, p_dev, (size_t)5 * m0 * 8, cudaMemcpyDeviceToDevice, c->s));
    return DOT_OK;
}

int dot_set_sources(dot_ctx* c, int ns, const int64_t* colptr, const int32_t* rows, const double* vals) {
    TRY(need_grid(c));
    TRY(check_csc(c, ns, colptr, rows, vals));
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> cv;
    csc_to_csr(c->n, ns, colptr, rows, vals, rp, ci, cv);
    TRY(upload(c, c->rpB, rp.data(), rp.size() * 8));
    TRY(upload(c, c->ciB, ci.data(), ci.size() * 4));
    TRY(upload(c, c->vB, cv.data(), cv.size() * 8));
    if (ns != c->ns) {
        c->ls = c->ld = 0;
        c->M_set = false;
    }
    c->ns = ns;
    c->P_valid = false;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_set_detectors(dot_ctx* c, int nd, const int64_t* colptr, const int32_t* rows, const double* vals) {
    TRY(need_grid(c));
    TRY(check_csc(c, nd, colptr, rows, vals));
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> cv;
    csc_to_csr(c->n, nd, colptr, rows, vals, rp, ci, cv);
    TRY(upload(c, c->rpC, rp.data(), rp.size() * 8));
    TRY(upload(c, c->ciC, ci.data(), ci.size() * 4));
    TRY(upload(c, c->vC, cv.data(), cv.size() * 8));
    TRY(upload(c, c->cpC, colptr, (size_t)(nd + 1) * 8));
    TRY(upload(c, c->rwC, rows, (size_t)colptr[nd] * 4));
    TRY(upload(c, c->vCc, vals, (size_t)colptr[nd] * 8));
    if (nd != c->nd) {
        c->ls = c->ld = 0;
        c->M_set = false;
    }
    c->nd = nd;
    c->P_valid = false;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_set_data(dot_ctx* c, const double* M, int is_complex) {
    TRY(need_ctx(c));
    if (c->ns == 0 || c->nd == 0) return fail(DOT_ESTATE, "set sources and detectors before data");
    if (!M) return fail(DOT_EINVAL, "null M");
    const size_t cnt = (size_t)c->nd * c->ns;
    std::vector<double> m2(cnt * 2, 0.0);
    for (size_t t = 0; t < cnt; ++t) {
        m2[2 * t] = is_complex ? M[2 * t] : M[t];
        m2[2 * t + 1] = is_complex ? M[2 * t + 1] : 0.0;
    }
    TRY(upload(c, c->M, m2.data(), cnt * 16));
    c->M_set = true;
    c->P_valid = false;
    c->post_valid = false;
    return DOT_OK;
}

int dot_set_sampling(dot_ctx* c, int ls, const double* W, int ld, const double* V) {
    TRY(need_ctx(c));
    if (c->ns == 0 || c->nd == 0) return fail(DOT_ESTATE, "set sources and detectors before sampling");
    if (ls < 1 || ld < 1) return fail(DOT_EINVAL, "ls and ld must be positive");
    if (ls + ld > 1024) return fail(DOT_EINVAL, "ls + ld exceeds 1024");
    if (!W || !V) return fail(DOT_EINVAL, "null W or V");
    TRY(upload(c, c->W, W, (size_t)c->ns * ls * 8));
    TRY(upload(c, c->V, V, (size_t)c->nd * ld * 8));
    c->ls = ls;
    c->ld = ld;
    c->P_valid = false;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_set_solver(dot_ctx* c, int precision, double rtol, int maxit) {
    TRY(need_ctx(c));
    if (precision != DOT_PREC_FP64 && precision != DOT_PREC_MIXED) return fail(DOT_EINVAL, "bad precision");
    if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(DOT_EINVAL, "rtol must lie in (0, 1)");
    if (maxit < 0) return fail(DOT_EINVAL, "maxit must be non-negative");
    c->prec = precision;
    c->rtol = rtol;
    c->maxit = maxit;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_set_refinement(dot_ctx* c, double delta) {
    TRY(need_ctx(c));
    if (!(delta > 0.0) || !(delta < 1.0)) return fail(DOT_EINVAL, "delta must lie in (0, 1)");
    c->delta = delta;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_misfit(dot_ctx* c, double* f) {
    TRY(need_grid(c));
    if (!f) return fail(DOT_EINVAL, "null f");
    if (!c->M_set) return fail(DOT_ESTATE, "dot_set_data has not been called");
    TRY(ensure_post(c));
    CK(cudaMemcpyAsync(f, c->f.p, 8, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (c->fields_status != DOT_OK) return fail(c->fields_status, "block solve did not converge in every column");
    return DOT_OK;
}

int dot_measurements(dot_ctx* c, double* S) {
    TRY(need_grid(c));
    if (!S) return fail(DOT_EINVAL, "null S");
    TRY(ensure_post(c));
    TRY(copy_out_complex_or_real(c, c->S, (size_t)c->ls * c->ld, S));
    if (c->fields_status != DOT_OK) return fail(c->fields_status, "block solve did not converge in every column");
    return DOT_OK;
}

}  // extern "C"

namespace {
// dot_gradient and dot_gradient_dev: kind says where f and g live.
int gradient_impl(dot_ctx* c, double* f, double* g, cudaMemcpyKind kind) {
    TRY(need_grid(c));
    if (!f || !g) return fail(DOT_EINVAL, "null output");
    if (!c->M_set) return fail(DOT_ESTATE, "dot_set_data has not been called");
    TRY(ensure_post(c));
    Phase ph("dot: sensitivity and PaLS chain rule");
    CK(cudaEventRecord(c->ev[3], c->s));
    TRY(ensure(c->gmu, c->n * 8));
    CK(sensitivity_gmu(cplx(c), c->x64.p, c->n, c->kp, c->ls, c->ld, c->Rs.as<double>(), c->gmu.as<double>(), c->s));
    count(c, 1);
    if (c->mu_mode == 2) {
        TRY(ensure(c->gp, (size_t)5 * c->m0 * 8));
        CK(pals_chain_gp(c->p.as<double>(), c->m0, c->gamma, c->nx, c->ny, c->nz, c->h, c->wdmu.as<double>(),
                         c->gmu.as<double>(), c->gp.as<double>(), c->s));
        count(c, 1);
        CK(cudaMemcpyAsync(g, c->gp.p, (size_t)5 * c->m0 * 8, kind, c->s));
    } else {
        CK(cudaMemcpyAsync(g, c->gmu.p, c->n * 8, kind, c->s));
    }
    CK(cudaMemcpyAsync(f, c->f.p, 8, kind, c->s));
    CK(cudaEventRecord(c->ev[2], c->s));
    CK(cudaStreamSynchronize(c->s));
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev[3], c->ev[2]);
    c->stats.ms_post = ms;
    if (c->fields_status != DOT_OK) return fail(c->fields_status, "block solve did not converge in every column");
    return DOT_OK;
}
}  // namespace

extern "C" {

int dot_gradient(dot_ctx* c, double* f, double* g) { return gradient_impl(c, f, g, cudaMemcpyDeviceToHost); }

int dot_gradient_dev(dot_ctx* c, double* f_dev, double* g_dev) {
    return gradient_impl(c, f_dev, g_dev, cudaMemcpyDeviceToDevice);
}

int dot_forward_model(dot_ctx* c, double* M) {
    TRY(need_grid(c));
    if (!M) return fail(DOT_EINVAL, "null M");
    if (c->ns == 0 || c->nd == 0) return fail(DOT_ESTATE, "set sources and detectors first");
    TRY(ensure_coefficients(c));
    const int chunk = 64;
    DevBuf saveW = c->W;
    const int save_ls = c->ls, save_ld = c->ld;
    DevBuf Wc;
    int rc = ensure(Wc, (size_t)c->ns * chunk * 8);
    int worst = DOT_OK;
    std::vector<double> hw((size_t)c->ns * chunk), ht;
    for (int s0 = 0; rc == DOT_OK && s0 < c->ns; s0 += chunk) {
        const int cw = std::min(chunk, c->ns - s0);
        std::fill(hw.begin(), hw.end(), 0.0);
        for (int i = 0; i < cw; ++i) hw[(size_t)(s0 + i) + (size_t)c->ns * i] = 1.0;
        c->W = Wc;
        c->ls = cw;
        c->ld = 0;
        invalidate_fields(c);
        rc = upload(c, Wc, hw.data(), (size_t)c->ns * cw * 8);
        if (rc == DOT_OK) rc = ensure_fields(c);
        if (rc == DOT_OK) {
            if (c->fields_status != DOT_OK && worst == DOT_OK) worst = c->fields_status;
            rc = ensure(c->Tm, (size_t)c->nd * cw * 16);
            if (rc == DOT_OK) rc = ensure(c->S, 16);
            if (rc == DOT_OK) rc = ensure(c->Rs, 16);
            if (rc == DOT_OK) rc = ensure(c->f, 16);
        }
        if (rc == DOT_OK) {
            // T = C^T U for this chunk of physical sources (the V projection is empty)
            cudaError_t e = restriction_misfit(cplx(c), c->x64.p, c->kp, cw, c->cpC.as<int64_t>(),
                                               c->rwC.as<int32_t>(), c->vCc.as<double>(), c->nd, nullptr, 0,
                                               nullptr, false, c->Tm.as<double>(), c->S.as<double>(),
                                               c->Rs.as<double>(), c->f.as<double>(), c->s);
            count(c, 2);
            ht.resize((size_t)c->nd * cw * 2);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ht.data(), c->Tm.p, (size_t)c->nd * cw * 16, cudaMemcpyDeviceToHost, c->s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
            if (e != cudaSuccess) {
                rc = fail(DOT_ECUDA, std::string("dot_forward_model: ") + cudaGetErrorString(e));
                break;
            }
            for (int i = 0; i < cw; ++i)
                for (int d = 0; d < c->nd; ++d) {
                    const size_t src = (size_t)d + (size_t)c->nd * i;
                    const size_t dst = (size_t)d + (size_t)c->nd * (s0 + i);
                    if (cplx(c)) {
                        M[2 * dst] = ht[2 * src];
                        M[2 * dst + 1] = ht[2 * src + 1];
                    } else {
                        M[dst] = ht[2 * src];
                    }
                }
        }
    }
    c->W = saveW;
    c->ls = save_ls;
    c->ld = save_ld;
    invalidate_fields(c);
    release(Wc);
    if (rc != DOT_OK) return rc;
    if (worst != DOT_OK) return fail(worst, "a forward solve did not converge");
    return DOT_OK;
}

int dot_optimized_sampling(dot_ctx* c, int qs, int qd, int maxit, double tol, int ls, const double* Ytil, int ld,
                           const double* Ztil, double* W, double* V, int* sweeps, double* objective) {
    TRY(need_grid(c));
    if (c->mu_mode != 2) return fail(DOT_ESTATE, "dot_optimized_sampling needs dot_set_pals");
    if (c->ns == 0 || c->nd == 0) return fail(DOT_ESTATE, "set sources and detectors first");
    if (qs < 1 || qd < 1 || qs > 8 || qd > 8 || qs > c->ns || qd > c->nd || ls < qs || ld < qd)
        return fail(DOT_EINVAL, "need 1 <= q <= 8, q <= n and q <= l for sources and detectors");
    if (c->ns + c->nd > 1024) return fail(DOT_EINVAL, "ns + nd exceeds 1024");
    if (!W || !V || (ls > qs && !Ytil) || (ld > qd && !Ztil)) return fail(DOT_EINVAL, "null array argument");
    if (maxit < 1 || !(tol > 0.0)) return fail(DOT_EINVAL, "maxit must be positive and tol > 0");
    TRY(ensure_coefficients(c));
    const bool cx_ = cplx(c);
    const int ns = c->ns, nd = c->nd, npar = 5 * c->m0;
    // every physical source and detector: W = I, V = I (Sec. 3.2: the full Jacobian once)
    DevBuf saveW = c->W, saveV = c->V, Wi, Vi;
    const int save_ls = c->ls, save_ld = c->ld;
    std::vector<double> eye_s((size_t)ns * ns, 0.0), eye_d((size_t)nd * nd, 0.0);
    for (int i = 0; i < ns; ++i) eye_s[(size_t)i * ns + i] = 1.0;
    for (int i = 0; i < nd; ++i) eye_d[(size_t)i * nd + i] = 1.0;
    int rc = upload(c, Wi, eye_s.data(), eye_s.size() * 8);
    if (rc == DOT_OK) rc = upload(c, Vi, eye_d.data(), eye_d.size() * 8);
    if (rc == DOT_OK) {
        c->W = Wi;
        c->V = Vi;
        c->ls = ns;
        c->ld = nd;
        invalidate_fields(c);
        rc = ensure_fields(c);
    }
    if (rc == DOT_OK) rc = ensure(c->J, (size_t)nd * ns * npar * esz64(c));
    if (rc == DOT_OK) rc = build_band_lists(c);
    if (rc == DOT_OK) {
        cudaError_t e = pals_chain_jp(cx_, c->m0, c->boffs.as<int64_t>(), c->bcell.as<int64_t>(),
                                      c->bdval.as<double>(), c->x64.p, c->kp, ns, nd, c->J.as<double>(), c->s);
        count(c, 1);
        if (e != cudaSuccess) rc = fail(DOT_ECUDA, std::string("jacobian tensor: ") + cudaGetErrorString(e));
    }
    c->W = saveW;
    c->V = saveV;
    c->ls = save_ls;
    c->ld = save_ld;
    invalidate_fields(c);
    release(Wi);
    release(Vi);
    if (rc != DOT_OK) return rc;
    DevBuf K, L, G, GP, VW;
    const int nmax = std::max(nd, ns);
    rc = ensure(K, (size_t)ns * npar * qd * esz64(c));
    if (rc == DOT_OK) rc = ensure(L, (size_t)nd * npar * qs * esz64(c));
    if (rc == DOT_OK) rc = ensure(G, (size_t)nmax * nmax * 8);
    if (rc == DOT_OK) rc = ensure(GP, (size_t)kGramPartDoubles * 8);
    if (rc == DOT_OK) rc = ensure(VW, (size_t)std::max(nd * qd, ns * qs) * 8);
    std::vector<double> What, Vhat;
    int sw = 0;
    double obj = 0.0;
    if (rc == DOT_OK)
        rc = optimize_from_tensor(cx_, c->J.p, nd, ns, npar, qs, qd, maxit, tol, K.p, L.p, G.as<double>(),
                                  GP.as<double>(), VW.as<double>(), c->s, What, Vhat, &sw, &obj);
    release(K);
    release(L);
    release(G);
    release(GP);
    release(VW);
    if (rc != DOT_OK) return rc;
    complement(ns, qs, What, ls - qs, Ytil, W);
    complement(nd, qd, Vhat, ld - qd, Ztil, V);
    if (sweeps) *sweeps = sw;
    if (objective) *objective = obj;
    return DOT_OK;
}

int dot_jacobian_mua(dot_ctx* c, double* J) {
    TRY(need_grid(c));
    if (!J) return fail(DOT_EINVAL, "null J");
    TRY(ensure_fields(c));
    const size_t cnt = (size_t)c->ls * c->ld * c->n;
    TRY(ensure(c->J, cnt * esz64(c)));
    CK(jacobian_mua(cplx(c), c->x64.p, c->n, c->kp, c->ls, c->ld, c->J.as<double>(), c->s));
    CK(cudaMemcpyAsync(J, c->J.p, cnt * esz64(c), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (c->fields_status != DOT_OK) return fail(c->fields_status, "block solve did not converge in every column");
    return DOT_OK;
}

int dot_jacobian_p(dot_ctx* c, double* Jp) {
    TRY(need_grid(c));
    if (!Jp) return fail(DOT_EINVAL, "null Jp");
    if (c->mu_mode != 2) return fail(DOT_ESTATE, "dot_jacobian_p needs dot_set_pals");
    TRY(ensure_fields(c));
    const size_t cnt = (size_t)c->ls * c->ld * 5 * c->m0;
    TRY(ensure(c->J, cnt * esz64(c)));
    TRY(build_band_lists(c));
    CK(pals_chain_jp(cplx(c), c->m0, c->boffs.as<int64_t>(), c->bcell.as<int64_t>(), c->bdval.as<double>(),
                     c->x64.p, c->kp, c->ls, c->ld, c->J.as<double>(), c->s));
    CK(cudaMemcpyAsync(Jp, c->J.p, cnt * esz64(c), cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (c->fields_status != DOT_OK) return fail(c->fields_status, "block solve did not converge in every column");
    return DOT_OK;
}

int dot_get_mua(dot_ctx* c, double* mu) {
    TRY(need_grid(c));
    if (!mu) return fail(DOT_EINVAL, "null mu");
    TRY(ensure_coefficients(c));
    CK(cudaMemcpyAsync(mu, c->mu.p, c->n * 8, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return DOT_OK;
}

int dot_get_fields(dot_ctx* c, double* U, double* Z) {
    TRY(need_grid(c));
    TRY(ensure_fields(c));
    const size_t bytes = (size_t)c->n * std::max(c->ls, c->ld) * esz64(c);
    TRY(ensure(c->tmp, bytes));
    if (U) {
        CK(blk_to_colmajor(cplx(c), c->x64.p, c->n, c->kp, 0, c->ls, c->tmp.as<double>(), c->s));
        CK(cudaMemcpyAsync(U, c->tmp.p, (size_t)c->n * c->ls * esz64(c), cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
    }
    if (Z) {
        CK(blk_to_colmajor(cplx(c), c->x64.p, c->n, c->kp, c->ls, c->ld, c->tmp.as<double>(), c->s));
        CK(cudaMemcpyAsync(Z, c->tmp.p, (size_t)c->n * c->ld * esz64(c), cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
    }
    return DOT_OK;
}

int dot_get_stats(dot_ctx* c, dot_stats* out) {
    if (!c || !out) return fail(DOT_EINVAL, "null argument");
    *out = c->stats;
    out->tuned_tma = c->last_cfg.blocks_per_sm < 0 ? -1 : (c->last_cfg.tma ? 1 : 0);
    out->tuned_blocks_per_sm = c->last_cfg.blocks_per_sm;
    out->fused_direction = c->last_cfg.blocks_per_sm < 0 ? -1 : (c->last_fused ? 1 : 0);
    return DOT_OK;
}

int dot_set_launch_options(dot_ctx* c, int graphs, int autotune) {
    TRY(need_ctx(c));
    c->use_graphs = graphs != 0;
    c->autotune = autotune != 0;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_set_direction_ring(dot_ctx* c, int slots) {
    TRY(need_ctx(c));
    if (slots != 0 && slots != 2 && slots != 4 && slots != 8)
        return fail(DOT_EINVAL, "slots must be 0 (as many as memory allows), 2, 4 or 8");
    c->ring_cap = slots == 0 ? kDirRingMax : slots;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_gradient_batch(dot_ctx* const* ctxs, int count, double* f, double* const* g) {
    if (count < 1 || !ctxs || !f || !g) return fail(DOT_EINVAL, "bad batch arguments");
    for (int i = 0; i < count; ++i) {
        dot_ctx* c = ctxs[i];
        TRY(need_grid(c));
        if (!c->M_set) return fail(DOT_ESTATE, "dot_set_data has not been called on a batch member");
        if (!g[i]) return fail(DOT_EINVAL, "null gradient output");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(DOT_EINVAL, "a context appears twice in the batch");
    }
    // The members run one after another, each on its own stream with its graph-replayed
    // block solve.  Every member's persistent kernels fill the GPU by themselves, so
    // members whose batches interleaved on concurrent streams only contended for the SMs:
    // eight uneven inversions ran 2-6% slower that way than back to back.
    int worst = DOT_OK;
    for (int i = 0; i < count; ++i) {
        TRY(need_ctx(ctxs[i]));
        const int rc = dot_gradient(ctxs[i], f + i, g[i]);
        if (rc != DOT_OK && rc != DOT_ENOTCONV && rc != DOT_EBREAKDOWN) return rc;
        if (rc != DOT_OK && worst == DOT_OK) worst = rc;
    }
    if (worst != DOT_OK) return fail(worst, "a batch member's block solve did not converge in every column");
    return DOT_OK;
}

int dot_set_stencil_path(dot_ctx* c, int mode) {
    TRY(need_ctx(c));
    if (mode < 0 || mode > 2) return fail(DOT_EINVAL, "stencil path must be 0, 1 or 2");
    c->stencil_mode = mode;
    invalidate_fields(c);
    return DOT_OK;
}

int dot_set_kernel_timing(dot_ctx* c, int enable) {
    TRY(need_ctx(c));
    c->timing = enable != 0;
    if (c->timing) c->kt = dot_kernel_timing{};
    return DOT_OK;
}

int dot_get_kernel_timing(dot_ctx* c, dot_kernel_timing* out) {
    if (!c || !out) return fail(DOT_EINVAL, "null argument");
    *out = c->kt;
    return DOT_OK;
}

int dot_apply(dot_ctx* c, int k, const double* x, double* y) {
    TRY(need_grid(c));
    if (k < 1 || !x || !y) return fail(DOT_EINVAL, "bad apply arguments");
    TRY(ensure_coefficients(c));
    const size_t bytes = (size_t)c->n * k * esz64(c);
    DevBuf xin, xb, yb;
    int rc = ensure(xin, bytes);
    if (rc == DOT_OK) rc = ensure(xb, bytes);
    if (rc == DOT_OK) rc = ensure(yb, bytes);
    if (rc == DOT_OK) {
        cudaError_t e = cudaMemcpyAsync(xin.p, x, bytes, cudaMemcpyHostToDevice, c->s);
        if (e == cudaSuccess) e = blk_from_colmajor(cplx(c), xin.as<double>(), c->n, k, k, 0, xb.p, c->s);
        if (e == cudaSuccess) e = op_apply(cplx(c) ? EK_C128 : EK_F64, op64(c), xb.p, yb.p, c->n, k, c->s);
        if (e == cudaSuccess) e = blk_to_colmajor(cplx(c), yb.p, c->n, k, 0, k, xin.as<double>(), c->s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(y, xin.p, bytes, cudaMemcpyDeviceToHost, c->s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
        if (e != cudaSuccess) rc = fail(DOT_ECUDA, std::string("dot_apply: ") + cudaGetErrorString(e));
    }
    release(xin);
    release(xb);
    release(yb);
    return rc;
}

int dot_probe_wait(dot_ctx* c, int64_t budget_cycles) {
    if (!c) return fail(DOT_EINVAL, "null context");
    if (budget_cycles < 0 || budget_cycles > 4000000000LL)
        return fail(DOT_EINVAL, "budget_cycles must lie in [0, 4e9]");
    DevBuf word;
    TRY(ensure(word, 16));
    int err = 0;
    cudaError_t e = cudaMemsetAsync(word.p, 0, 16, c->s);
    if (e == cudaSuccess) e = wait_probe(word.as<int>(), (long long)budget_cycles, c->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_flag, word.p, sizeof(int), cudaMemcpyDeviceToHost, c->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
    if (e == cudaSuccess) err = c->h_flag[0];
    release(word);
    if (e != cudaSuccess) return fail(DOT_ECUDA, std::string("dot_probe_wait: ") + cudaGetErrorString(e));
    if (err) return fail(DOT_ETIMEOUT, "dot_probe_wait: the bounded wait gave up after its budget, as intended");
    return fail(DOT_EBREAKDOWN, "dot_probe_wait: a wait that nothing completes reported completion");
}

}  // extern "C"
