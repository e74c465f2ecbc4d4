// A3-A7 host side shared by the four inner precisions: dispatch of a batch to
// its precision's launcher (solver_<precision>.cu), the launch profile, the
// synchronous and concurrent batch runners, the operator-apply dispatch and the
// allocation-free entry point with its static scratch array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace mlmc {

namespace {

// Profile of a launched batch; its stream must have been synchronised.  (Its error word is
// the context's, read by check_device_errors.)
mlmc_status finish_solve(mlmc_ctx* ctx, PendingSolve& ps_) {
    if (!ps_.active) return MLMC_OK;
    ps_.active = false;
    const int ns = ps_.ns;
    cudaEvent_t* ev = ps_.ev;
    if (ev[0]) {
        float ms = 0.f, a0 = 0.f, a1 = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (ctx->prof.t0 && cudaEventElapsedTime(&a0, ctx->prof.t0, ev[0]) == cudaSuccess &&
            cudaEventElapsedTime(&a1, ctx->prof.t0, ev[1]) == cudaSuccess)
            ctx->prof.solve_iv.emplace_back((double)a0, (double)a1);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        ev[0] = ev[1] = nullptr;
        std::vector<int32_t> stats(2 * ns);
        MLMC_CUDA_RET(ctx->err, cudaMemcpy(stats.data(), ps_.stats, sizeof(int32_t) * 2 * ns, cudaMemcpyDeviceToHost));
        const int32_t* outer = stats.data() + ns;
        double bytes = 0.0, flops = 0.0;
        int64_t iters = 0, uit = 0;
        for (int i = 0; i < ns && i < (int)ps_.unk.size(); ++i) {
            const int32_t it = stats[i];
            const int steps = std::min(outer[i], ps_.max_outer);
            bytes += (double)it * ps_.c_it[i] + (double)(steps + 1) * ps_.c_res[i] + (double)steps * ps_.c_upd[i] +
                     ps_.c_set[i];
            // the first refinement residual is r = b (x = 0): its dots only
            flops += (double)it * ps_.f_it[i] + (double)steps * ps_.f_res[i] + ps_.f_res[i] * (7.0 / 20.0) +
                     (double)steps * ps_.f_upd[i] + ps_.f_set[i];
            iters += it;
            uit += (int64_t)ps_.unk[i] * it;
        }
        mlmc_profile& A = ctx->prof.acc;
        A.solve_launches += 1;
        A.solve_ms += ms;
        A.solve_bytes += bytes;
        A.solve_flops += flops;
        A.inner_iters += iters;
        A.unknown_iters += uit;
    }
    return MLMC_OK;
}

mlmc_status launch_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                         cudaStream_t st, int slot, PendingSolve& out) {
    if (cfg.solver != MLMC_CG && cfg.solver != MLMC_MINRES) {
        ctx->err = "unknown solver";
        return MLMC_E_ARG;
    }
    switch (cfg.prec) {
        case MLMC_FP64: return solve_launch_fp64(ctx, groups, cfg, st, slot, out);
        case MLMC_FP32: return solve_launch_fp32(ctx, groups, cfg, st, slot, out);
        case MLMC_BF16S: return solve_launch_bf16s(ctx, groups, cfg, st, slot, out);
        case MLMC_FP16S: return solve_launch_fp16s(ctx, groups, cfg, st, slot, out);
        default: ctx->err = "bad precision"; return MLMC_E_ARG;
    }
}

// ---------------------------------------------------------------------------
// Autotuner (mlmc_set_autotune).  A launch shape -- inner precision, solver, preconditioner, and the
// batch's grids with their system counts rounded down to powers of two -- that has not been seen is
// solved once per candidate setting, starting from the library's own rules and changing one setting
// at a time (coordinate descent): the group size of n = 91..128 systems (2048 or 4096 chunks per
// 128-thread group), the row-pipeline depth of Jacobi-preconditioned CG (0, 2, 4 slots), the
// V-cycle's smoothing sweeps (1, 2), the inner tolerance factor theta (0.1, 0.3, 0.6) and the inner
// tolerance's floor (0.3, 1 or 3 times the precision's default).  Each
// candidate is timed twice with CUDA events on the stream (the minimum counts); a change is kept if
// it is at least 1% faster.  Every trial solves the same systems to the same accuracy, so the
// outputs of the last trial are valid results.
std::string tune_key(const std::vector<SolveGroup>& groups, const SolveConfig& cfg, int precond) {
    std::map<int, long long> cnt;
    for (const SolveGroup& g : groups)
        if (g.S > 0) cnt[g.n] += g.S;
    std::string k = "prec " + std::to_string(cfg.prec) + " solver " + std::to_string(cfg.solver) + " pc " +
                    std::to_string(precond) + ":";
    for (const auto& kv : cnt) {
        int c = 0;
        while ((2LL << c) <= kv.second) ++c;
        k += " " + std::to_string(kv.first) + "x2^" + std::to_string(c);
    }
    return k;
}

void tune_apply(const TuneChoice& t, SolveConfig& cfg) {
    cfg.med_items = t.med_items;
    cfg.ring = t.ring;
    cfg.nu = t.nu;
    cfg.mg_min = t.mg_min;
    cfg.mg_coarse = t.mg_coarse;
    cfg.mg_omega = t.mg_omega;
    cfg.mg_smem = t.mg_smem;
    cfg.theta = t.theta;
    cfg.tau_min = t.tau_min;
}

// The inner tolerance's default floor of an inner precision (the accuracy an inner solve in it can be
// relied on to reach; make_params).
double tau_floor(int prec) {
    switch (prec) {
        case MLMC_FP64: return 1e-14;
        case MLMC_FP16S: return 1e-4;
        case MLMC_BF16S: return 1e-3;
        default: return 1e-6;
    }
}

// One timed solve of the batch (minimum of `reps` runs) with the settings of t.
mlmc_status tune_time(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, SolveConfig cfg, const TuneChoice& t,
                      cudaStream_t st, int reps, float* ms) {
    tune_apply(t, cfg);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MLMC_CUDA_RET(ctx->err, cudaEventCreate(&e0));
    MLMC_CUDA_RET(ctx->err, cudaEventCreate(&e1));
    *ms = 1e30f;
    mlmc_status s = MLMC_OK;
    for (int r = 0; r < reps && s == MLMC_OK; ++r) {
        PendingSolve p;
        cudaEventRecord(e0, st);
        s = launch_batch(ctx, groups, cfg, st, 0, p);
        cudaEventRecord(e1, st);
        const cudaError_t e = cudaStreamSynchronize(st);
        if (s == MLMC_OK && e != cudaSuccess) {
            ctx->err = std::string("autotune: ") + cudaGetErrorString(e);
            s = MLMC_E_CUDA;
        }
        float x = 0.f;
        if (s == MLMC_OK && cudaEventElapsedTime(&x, e0, e1) == cudaSuccess) *ms = std::min(*ms, x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return s;
}

mlmc_status autotune_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, SolveConfig& cfg, cudaStream_t st) {
    const int precond = cfg.precond >= 0 ? cfg.precond : ctx->precond;
    const std::string key = tune_key(groups, cfg, precond);
    auto it = ctx->tune.find(key);
    if (it != ctx->tune.end()) {
        tune_apply(it->second, cfg);
        return MLMC_OK;
    }
    // which settings can matter for this shape
    bool has_mid = false, pipe_sizes = false;
    for (const SolveGroup& g : groups) {
        if (g.S <= 0) continue;
        const long long items = (long long)(g.n - 1) * ((g.n - 1) / 4 + 1);
        if (items > 2048 && items <= 4096) has_mid = true;
        if (items > 2048 && ((g.n - 1) / 4 + 1) % 32 == 0) pipe_sizes = true;
    }
    const bool mg = precond == MLMC_PC_MG;
    const bool ring_matters = cfg.solver == MLMC_CG && !mg && cfg.prec != MLMC_FP64 && pipe_sizes;
    const bool prof = ctx->prof.on;
    ctx->prof.on = false;   // trials are not part of the profile
    TuneChoice cur;
    cur.prec = cfg.prec;
    cur.solver = cfg.solver;
    cur.precond = precond;
    float best = 0.f;
    mlmc_status s = tune_time(ctx, groups, cfg, cur, st, 2, &best);
    cur.default_ms = best;
    int trials = 2;
    auto consider = [&](TuneChoice cand) {
        if (s != MLMC_OK) return;
        float ms = 0.f;
        s = tune_time(ctx, groups, cfg, cand, st, 2, &ms);
        trials += 2;
        if (s == MLMC_OK && ms < 0.99f * best) {
            best = ms;
            cur = cand;
        }
    };
    if (has_mid)
        for (int m : {2048, 4096}) {
            TuneChoice c = cur;
            c.med_items = m;
            consider(c);
        }
    if (ring_matters)
        for (int r : {0, 2, 4}) {
            TuneChoice c = cur;
            c.ring = r;
            consider(c);
        }
    if (mg) {
        // the coarsest grid: fewer or more sweeps on it, or one halving less with more sweeps (measured on
        // 100 x n = 256: 4.75 ms by default, 4.73 with 4 sweeps, 4.63 one level shallower with 16 sweeps)
        const int deeper[3][2] = {{ctx->mg_min, 4}, {ctx->mg_min, 16}, {2 * ctx->mg_min, 16}};
        for (const auto& d : deeper) {
            if (d[0] > 32 || (d[0] == ctx->mg_min && d[1] == ctx->mg_coarse)) continue;
            TuneChoice c = cur;
            c.mg_min = d[0];
            c.mg_coarse = d[1];
            consider(c);
        }
        // the smoother's damping, and the deepest grid kept in shared memory
        for (double om : {0.7, 0.9}) {
            TuneChoice c = cur;
            c.mg_omega = om;
            consider(c);
        }
        {
            TuneChoice c = cur;
            c.mg_smem = 32;
            consider(c);
        }
    }
    if (mg)
        for (int nu : {1, 2}) {
            if (nu == ctx->mg_nu) continue;
            TuneChoice c = cur;
            c.nu = nu;
            consider(c);
        }
    for (double th : {0.1, 0.6}) {
        TuneChoice c = cur;
        c.theta = th;
        consider(c);
    }
    if (ctx->inner_tau_min <= 0)
        for (double f : {0.3, 3.0}) {
            TuneChoice c = cur;
            c.tau_min = f * tau_floor(cfg.prec);
            consider(c);
        }
    ctx->prof.on = prof;
    if (s != MLMC_OK) return s;
    cur.best_ms = best;
    cur.trials = trials;
    ctx->tune[key] = cur;
    ctx->tune_order.push_back(key);
    tune_apply(cur, cfg);
    return MLMC_OK;
}

}  // namespace

mlmc_status run_solve_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg_in,
                            cudaStream_t st) {
    if (cfg_in.solver == MLMC_CHOLESKY) return run_cholesky_batch(ctx, groups, cfg_in, st, true);
    SolveConfig cfg = cfg_in;
    if (ctx->autotune) {
        const mlmc_status t = autotune_batch(ctx, groups, cfg, st);
        if (t != MLMC_OK) return t;
    }
    PendingSolve p;
    mlmc_status s = launch_batch(ctx, groups, cfg, st, 0, p);
    if (s != MLMC_OK) return s;
    MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
    s = finish_solve(ctx, p);
    const mlmc_status e = check_device_errors(ctx, st);
    return s != MLMC_OK ? s : e;
}

mlmc_status launch_solve_async(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                               cudaStream_t st) {
    // profiling reads the launch's per-system counters from its workspace, which the next call reuses;
    // tuning a new launch shape times its candidates
    if (cfg.solver == MLMC_CHOLESKY) return run_cholesky_batch(ctx, groups, cfg, st, false);
    if (ctx->prof.on || ctx->autotune) return run_solve_batch(ctx, groups, cfg, st);
    PendingSolve p;
    return launch_batch(ctx, groups, cfg, st, 0, p);
}

mlmc_status finish_solves(mlmc_ctx* ctx, std::vector<PendingSolve>& pend) {
    mlmc_status status = MLMC_OK;
    for (PendingSolve& p : pend) {
        const mlmc_status f = finish_solve(ctx, p);
        if (status == MLMC_OK) status = f;
    }
    pend.clear();
    return status;
}

mlmc_status launch_solve_batches(mlmc_ctx* ctx, const std::vector<SolveBatch>& batches, cudaStream_t st,
                                 std::vector<PendingSolve>& pend) {
    pend.clear();
    if (batches.size() <= 1) return batches.empty() ? MLMC_OK : run_solve_batch(ctx, batches[0].groups,
                                                                                 batches[0].cfg, st);
    if (batches[0].cfg.solver == MLMC_CHOLESKY) {
        // the Cholesky launches of a round run one after another
        for (const SolveBatch& b : batches) {
            const mlmc_status s = run_cholesky_batch(ctx, b.groups, b.cfg, st, true);
            if (s != MLMC_OK) return s;
        }
        return MLMC_OK;
    }
    if (batches.size() > (size_t)kSolveSlots) {
        ctx->err = "run_solve_batches: too many concurrent batches";
        return MLMC_E_ARG;
    }
    // settings of each batch (the autotuner times a new shape alone, on st, before the concurrent launch)
    std::vector<SolveConfig> cfgs;
    for (const SolveBatch& b : batches) {
        cfgs.push_back(b.cfg);
        if (ctx->autotune) {
            const mlmc_status t = autotune_batch(ctx, b.groups, cfgs.back(), st);
            if (t != MLMC_OK) return t;
        }
    }
    // fork: batch 0 on st, batch i > 0 on the context's auxiliary stream i - 1, all after st's prior work
    cudaEvent_t fork = nullptr;
    MLMC_CUDA_RET(ctx->err, cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    MLMC_CUDA_RET(ctx->err, cudaEventRecord(fork, st));
    pend.resize(batches.size());
    std::vector<cudaEvent_t> done(batches.size(), nullptr);
    mlmc_status status = MLMC_OK;
    for (size_t i = 0; i < batches.size() && status == MLMC_OK; ++i) {
        cudaStream_t si = st;
        if (i > 0) {
            if (!ctx->aux[i - 1] && cudaStreamCreateWithFlags(&ctx->aux[i - 1], cudaStreamNonBlocking) != cudaSuccess) {
                ctx->err = "run_solve_batches: cannot create a stream";
                status = MLMC_E_CUDA;
                break;
            }
            si = ctx->aux[i - 1];
            if (cudaStreamWaitEvent(si, fork, 0) != cudaSuccess) {
                ctx->err = "run_solve_batches: cudaStreamWaitEvent failed";
                status = MLMC_E_CUDA;
                break;
            }
        }
        status = launch_batch(ctx, batches[i].groups, cfgs[i], si, (int)i, pend[i]);
        if (status == MLMC_OK && i > 0) {
            // join: st waits for batch i
            if (cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(done[i], si) != cudaSuccess || cudaStreamWaitEvent(st, done[i], 0) != cudaSuccess) {
                ctx->err = "run_solve_batches: joining the streams failed";
                status = MLMC_E_CUDA;
            }
        }
    }
    // (an event may be destroyed while work it waits for is pending: it is released when that completes)
    cudaEventDestroy(fork);
    for (cudaEvent_t e : done)
        if (e) cudaEventDestroy(e);
    if (status != MLMC_OK) {
        // every launched batch is waited for, whatever failed
        for (size_t i = 1; i < batches.size(); ++i)
            if (ctx->aux[i - 1]) cudaStreamSynchronize(ctx->aux[i - 1]);
        cudaStreamSynchronize(st);
        finish_solves(ctx, pend);
    }
    return status;
}

mlmc_status run_solve_batches(mlmc_ctx* ctx, const std::vector<SolveBatch>& batches, cudaStream_t st) {
    std::vector<PendingSolve> pend;
    mlmc_status status = launch_solve_batches(ctx, batches, st, pend);
    if (status != MLMC_OK) return status;
    const cudaError_t se = cudaStreamSynchronize(st);   // st waited for every batch
    if (se != cudaSuccess) {
        ctx->err = std::string("run_solve_batches: ") + cudaGetErrorString(se);
        status = MLMC_E_CUDA;
    }
    const mlmc_status f = finish_solves(ctx, pend);
    if (status == MLMC_OK) status = f;
    if (status == MLMC_OK) status = check_device_errors(ctx, st);
    return status;
}

cudaError_t launch_apply_operator(int n, int S, const void* a, int a_fp64, int a_n, int op_prec, const void* x,
                                  void* y, int vec_fp64, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    if (vec_fp64) return apply_operator_fp64(n, S, a, a_fp64, a_n, x, y, st);
    switch (op_prec) {
        case MLMC_FP32: return apply_operator_fp32(n, S, a, a_fp64, a_n, x, y, st);
        case MLMC_BF16S: return apply_operator_bf16s(n, S, a, a_fp64, a_n, x, y, st);
        case MLMC_FP16S: return apply_operator_fp16s(n, S, a, a_fp64, a_n, x, y, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mlmc

// ===========================================================================
// Allocation-free solve (mlmc_level_solve_noalloc): the resident solve with its
// scratch in a file-scope device array instead of context workspaces.
namespace mlmc {
namespace {

constexpr size_t kNoAllocBytes = MLMC_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t noalloc_scratch(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[device] = p;
    }
    *out = g_noalloc_addr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace mlmc

extern "C" mlmc_status mlmc_level_solve_noalloc(int device, int n, int S, const void* a, mlmc_prec a_prec, int a_n,
                                                mlmc_prec prec, double delta, int max_iters, int qoi,
                                                const double* box, double f, double* Q, int32_t* iters,
                                                double* relres, int32_t* flags, void* stream) {
    using namespace mlmc;
    std::string& err = create_error();
    err.clear();
    if (n < 2 || n > 2048 || S < 0 || a_n < n || a_n % n != 0 || (a_prec != MLMC_FP64 && a_prec != MLMC_FP32) ||
        prec < MLMC_FP64 || prec > MLMC_FP16S || !(delta > 0) || max_iters < 1 || (qoi != 0 && qoi != 1) ||
        (qoi == 1 && !box) || !std::isfinite(f) || device < 0 || device >= kNoAllocMaxDevices) {
        err = "level_solve_noalloc: bad device, n, S, a_n, precision, delta, max_iters, qoi, box or f";
        return MLMC_E_ARG;
    }
    if (qoi == 1) {
        // the box must be finite, ordered, inside the unit square and on grid lines of the n-cell grid
        bool ok = std::isfinite(box[0]) && std::isfinite(box[1]) && std::isfinite(box[2]) && std::isfinite(box[3]) &&
                  box[0] >= 0.0 && box[0] < box[1] && box[1] <= 1.0 && box[2] >= 0.0 && box[2] < box[3] &&
                  box[3] <= 1.0;
        for (int k = 0; k < 4 && ok; ++k) {
            const double v = box[k] * n;
            ok = std::fabs(v - std::round(v)) <= 1e-9;
        }
        if (!ok) {
            err = "level_solve_noalloc: the QoI box must satisfy 0 <= x0 < x1 <= 1, 0 <= y0 < y1 <= 1, "
                  "with every side on a grid line of the n-cell grid";
            return MLMC_E_ARG;
        }
    }
    if (S == 0) return MLMC_OK;
    if (!a || !Q) {
        err = "level_solve_noalloc: null a or Q";
        return MLMC_E_ARG;
    }
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess) e = cudaSetDevice(device);
    void* scratch = nullptr;
    if (e == cudaSuccess) e = noalloc_scratch(device, &scratch);
    if (e != cudaSuccess) {
        err = std::string("level_solve_noalloc: set-up: ") + cudaGetErrorString(e);
        cudaSetDevice(prev);
        return MLMC_E_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int a64 = a_prec == MLMC_FP64;
    mlmc_status s;
    switch (prec) {
        case MLMC_FP64:
            s = noalloc_solve_fp64(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, Q, iters, relres, flags, st, scratch, err);
            break;
        case MLMC_FP32:
            s = noalloc_solve_fp32(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, Q, iters, relres, flags, st, scratch, err);
            break;
        case MLMC_BF16S:
            s = noalloc_solve_bf16s(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, Q, iters, relres, flags, st, scratch, err);
            break;
        default:
            s = noalloc_solve_fp16s(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, Q, iters, relres, flags, st, scratch, err);
            break;
    }
    cudaSetDevice(prev);
    return s;
}
