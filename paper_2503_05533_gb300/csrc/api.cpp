// libmlmc C ABI (include/libmlmc.h): context, entry points, the estimate loop
// of Alg. 4.1 and the round scheduler that puts every sample of every level
// of a round into one resident-solve launch per precision class.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace mlmc {

// An NVTX range for the scope (shows the estimate's rounds, field syntheses and solve launches on a
// profiler's timeline; no cost without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

std::atomic<int64_t> g_launches{0};

std::string& create_error() {
    static thread_local std::string s;
    return s;
}

// Forced allocation failure (mlmc_debug_fail_allocation): allocations left before the one that fails,
// -1 when disarmed.
static std::atomic<int64_t> g_fail_alloc{-1};

static bool forced_alloc_failure() {
    int64_t v = g_fail_alloc.load();
    while (v >= 0) {
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 0;   // 0 -> -1: this one fails
    }
    return false;
}

cudaError_t DevBuf::reserve(size_t want) {
    if (want <= bytes && ptr) return cudaSuccess;
    // calls return before their kernels finish: work still in flight may use the old buffer
    if (ptr) {
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
    }
    release();
    if (forced_alloc_failure()) return cudaErrorMemoryAllocation;
    const size_t grow = std::max(want, bytes + bytes / 4);
    cudaError_t e = cudaMalloc(&ptr, grow);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        e = cudaMalloc(&ptr, want);
        if (e != cudaSuccess) {
            ptr = nullptr;
            return e;
        }
        bytes = want;
        return cudaSuccess;
    }
    bytes = grow;
    return cudaSuccess;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}


// Chan et al. pairwise merge; compensated sums merged with TwoSum.
static void two_sum_add(double& s, double& c, double x) {
    const double t = s + x;
    const double e = (std::fabs(s) >= std::fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
    c += e;
}

void acc_merge(mlmc_acc* a, const mlmc_acc& b) {
    if (b.n == 0) return;
    if (a->n == 0) {
        *a = b;
        return;
    }
    const double na = (double)a->n, nb = (double)b.n, n = na + nb;
    const double d = b.mean - a->mean;
    a->mean = a->mean + d * (nb / n);
    a->m2 = a->m2 + b.m2 + d * d * (na * nb / n);
    a->n += b.n;
    a->sum_c += b.sum_c;
    two_sum_add(a->sum, a->sum_c, b.sum);
    a->sumsq_c += b.sumsq_c;
    two_sum_add(a->sumsq, a->sumsq_c, b.sumsq);
}

static void acc_push(mlmc_acc* a, double y) {
    a->n += 1;
    const double d = y - a->mean;
    a->mean += d / (double)a->n;
    a->m2 += d * (y - a->mean);
    two_sum_add(a->sum, a->sum_c, y);
    two_sum_add(a->sumsq, a->sumsq_c, y * y);
}

cudaError_t ctx_order_begin(mlmc_ctx* ctx, cudaStream_t st) {
    return ctx->order_recorded ? cudaStreamWaitEvent(st, ctx->order_ev, 0) : cudaSuccess;
}

cudaError_t ctx_order_end(mlmc_ctx* ctx, cudaStream_t st) {
    if (!ctx->order_ev) {
        const cudaError_t e = cudaEventCreateWithFlags(&ctx->order_ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    const cudaError_t e = cudaEventRecord(ctx->order_ev, st);
    if (e == cudaSuccess) ctx->order_recorded = true;
    return e;
}

mlmc_status check_device_errors(mlmc_ctx* ctx, cudaStream_t st) {
    unsigned w[2] = {0u, 0u};
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(w, ctx->kl_err, sizeof(w), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
    if (w[0] == 0u && w[1] == 0u) return MLMC_OK;   // KERR_NONE
    MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(ctx->kl_err, 0, sizeof(w), st));
    MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
    if (w[0] != 0u)
        ctx->err = "tensor-core KL synthesis: a bounded wait ran out (timeout); its output is not valid";
    else
        ctx->err = "resident solve: a bounded wait of the row pipeline ran out after " +
                   std::to_string(ctx->wait_timeout_s) + " s; the affected systems carry MLMC_F_TIMEOUT";
    return MLMC_E_TIMEOUT;
}

double qoi_weight_node(const mlmc_problem& p, int n, int i, int j) {
    const double h2 = 1.0 / ((double)n * n);
    if (p.qoi == 0) return h2;
    const int bx0 = (int)std::lround(p.box[0] * n), bx1 = (int)std::lround(p.box[1] * n);
    const int by0 = (int)std::lround(p.box[2] * n), by1 = (int)std::lround(p.box[3] * n);
    auto in = [&](int ci, int cj) { return (ci >= bx0 && ci < bx1 && cj >= by0 && cj < by1) ? 1 : 0; };
    const int cnt = 2 * in(i, j) + in(i - 1, j) + 2 * in(i - 1, j - 1) + in(i, j - 1);
    return h2 * cnt / 6.0;
}

}  // namespace mlmc

using namespace mlmc;

namespace {

int level_n(const mlmc_problem& p, int l) {
    long long n = p.n0;
    for (int i = 0; i < l; ++i) n *= p.m;
    return (int)n;
}

bool is_field_prec(mlmc_prec p) { return p == MLMC_FP64 || p == MLMC_FP32 || p == MLMC_FP64TC; }
bool is_master_prec(mlmc_prec p) { return p == MLMC_FP64 || p == MLMC_FP32; }   // element type of a stored field
bool is_prec(int p) { return p >= MLMC_FP64 && p <= MLMC_FP16S; }

mlmc_status fail(mlmc_ctx* ctx, mlmc_status code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

mlmc_status check_problem(const mlmc_problem* p, std::string& err) {
    if (!p) { err = "null problem"; return MLMC_E_ARG; }
    if (p->n0 < 2 || p->m < 2 || p->L_max < 0 || p->L_max >= MLMC_MAX_LEVELS) {
        err = "need n0 >= 2, m >= 2, 0 <= L_max < MLMC_MAX_LEVELS";
        return MLMC_E_ARG;
    }
    long long n = p->n0;
    for (int l = 0; l < p->L_max; ++l) n *= p->m;
    if (n > 2048) { err = "finest grid above 2048 cells per side"; return MLMC_E_ARG; }
    const mlmc_field& f = p->field;
    if (f.K < 1 || f.K > 256 || !(f.sigma2 > 0) || f.kind < 0 || f.kind > 2) {
        err = "field: need kind in 0..2, 1 <= K <= 256, sigma2 > 0";
        return MLMC_E_ARG;
    }
    if (f.kind == 0 && !(f.corr_len > 0)) { err = "field: corr_len must be > 0"; return MLMC_E_ARG; }
    if (f.kind == 2 && f.K != 1) { err = "field kind 2 needs K = 1"; return MLMC_E_ARG; }
    if (p->qoi != 0 && p->qoi != 1) { err = "qoi must be 0 or 1"; return MLMC_E_ARG; }
    if (p->qoi == 1) {
        const double* b = p->box;
        if (!(b[0] >= 0 && b[0] < b[1] && b[1] <= 1 && b[2] >= 0 && b[2] < b[3] && b[3] <= 1)) {
            err = "qoi box must satisfy 0 <= x0 < x1 <= 1, 0 <= y0 < y1 <= 1";
            return MLMC_E_ARG;
        }
        for (int k = 0; k < 4; ++k) {
            const double v = b[k] * p->n0;
            if (std::fabs(v - std::round(v)) > 1e-9) { err = "qoi box sides must lie on level-0 grid lines"; return MLMC_E_ARG; }
        }
    }
    if (!std::isfinite(p->f)) { err = "f must be finite"; return MLMC_E_ARG; }
    return MLMC_OK;
}

// Field of S samples on level l from xi (device) into a (device), in field precision.
mlmc_status synth(mlmc_ctx* ctx, int level, int S, const double* xi, void* a, long long ld, mlmc_prec field_prec,
                  cudaStream_t st) {
    const int n = level_n(ctx->prob, level);
    GridBasis& gb = ctx->basis.at(n);
    if (ld == 0) ld = (long long)(n + 1) * (n + 1);
    cudaError_t e = (field_prec == MLMC_FP64)     ? launch_kl_fp64(gb, S, xi, static_cast<double*>(a), ld, st)
                    : (field_prec == MLMC_FP64TC) ? launch_kl_tc64(ctx, gb, S, xi, static_cast<double*>(a), ld, st)
                                                  : launch_kl_fp32(ctx, gb, S, xi, static_cast<float*>(a), ld, st);
    if (e != cudaSuccess) return fail(ctx, MLMC_E_CUDA, std::string("KL synthesis: ") + cudaGetErrorString(e));
    return MLMC_OK;
}

// Inner precision rule (documented at mlmc_adapt_precision).
mlmc_prec pick_prec(double h, double delta, double contrast) {
    if (contrast <= 0) contrast = 1.0;
    const double u_single = 0x1p-24;
    if (contrast / (h * h) * u_single > 0.5) return MLMC_FP64;
    if (delta >= 1e-4) return MLMC_FP16S;
    return MLMC_FP32;
}

// The calibrated rule (mlmc_options.prec_rule = 1): the level's measured contrast in Cor. 3.4's
// condition, and IEEE half storage only where the coefficient and its inverse diagonal 1 / (4 a) stay
// in half's normal range.
mlmc_prec pick_prec_calibrated(double h, double delta, double contrast, double amin, double amax) {
    const double u_single = 0x1p-24;
    if (contrast / (h * h) * u_single > 0.5) return MLMC_FP64;
    if (delta >= 1e-4) return (amin >= 6.2e-5 && amax <= 4.0e3) ? MLMC_FP16S : MLMC_BF16S;
    return MLMC_FP32;
}

// ---------------------------------------------------------------------------
// Alg. 4.1 host loop, shared by the GPU estimate and the host-sampler variant.
struct Request {
    int level;
    int64_t first;
    int count;
};
using RoundFn = std::function<mlmc_status(const std::vector<Request>&, const std::vector<double>& delta_fine,
                                          const std::vector<double>& delta_coarse, std::vector<mlmc_acc>& out,
                                          mlmc_result* res)>;

// One JSON array of the first n values.
template <class T>
void json_array(FILE* f, const T* v, int n) {
    std::fputc('[', f);
    for (int i = 0; i < n; ++i) {
        if (i) std::fputc(',', f);
        if (std::is_integral<T>::value) std::fprintf(f, "%lld", (long long)v[i]);
        else std::fprintf(f, "%.17g", (double)v[i]);
    }
    std::fputc(']', f);
}

// Sample targets for the next round from the level accumulators (the optimal N_l of Alg. 4.1 with the
// variance budget TOL^2 / 2), never below the samples done; a level without samples starts at N_init.
// Returns whether every level already has its target.
bool next_targets(int m, const mlmc_options& o, const std::vector<mlmc_acc>& acc, std::vector<int64_t>& N) {
    const int L = (int)acc.size() - 1;
    std::vector<double> V(L + 1), C(L + 1);
    double sum_vc = 0.0;
    for (int l = 0; l <= L; ++l) {
        V[l] = acc[l].n > 0 ? acc[l].m2 / (double)acc[l].n : 0.0;
        C[l] = std::pow((double)m, o.gamma * l);
        sum_vc += std::sqrt(V[l] * C[l]);
    }
    N.assign(L + 1, 0);
    bool enough = true;
    for (int l = 0; l <= L; ++l) {
        if (acc[l].n == 0) {
            N[l] = o.N_init;
            enough = false;
            continue;
        }
        const int64_t Nopt = (int64_t)std::ceil(std::sqrt(V[l] / C[l]) * (2.0 / (o.tol * o.tol)) * sum_vc);
        N[l] = std::max<int64_t>(Nopt, acc[l].n);
        if (acc[l].n < Nopt) enough = false;
    }
    return enough;
}

mlmc_status alg41(int m, int L_max, int n0, const mlmc_options& o, const RoundFn& round, mlmc_result* res,
                  std::string& err) {
    const auto t0 = std::chrono::steady_clock::now();
    const mlmc_result* prev = o.resume;
    mlmc_result keep;
    if (prev) keep = *prev;   // res may be the checkpoint itself
    std::memset(res, 0, sizeof(*res));
    const bool fixed = o.fixed_N != nullptr;
    int L = std::min(std::max(o.L_start, 0), L_max);
    std::vector<int64_t> N(L + 1, o.N_init);
    if (fixed)
        for (int l = 0; l <= L; ++l) N[l] = o.fixed_N[l];
    std::vector<mlmc_acc> acc(L + 1);
    std::memset(acc.data(), 0, sizeof(mlmc_acc) * acc.size());
    int rounds = 0, rounds_before = 0;
    double seconds_before = 0.0;
    if (prev) {
        // checkpoint: the finest level, the level accumulators and the targets they imply
        if (fixed) {
            err = "resume: not with fixed_N";
            return MLMC_E_ARG;
        }
        if (keep.L < 0 || keep.L > L_max || keep.rounds < 0) {
            err = "resume: the checkpoint's finest level or round count is outside this problem";
            return MLMC_E_ARG;
        }
        L = keep.L;
        acc.assign(keep.acc, keep.acc + L + 1);
        for (int l = 0; l <= L; ++l)
            if (acc[l].n < 0) {
                err = "resume: negative sample count in the checkpoint";
                return MLMC_E_ARG;
            }
        next_targets(m, o, acc, N);
        rounds_before = keep.rounds;
        seconds_before = keep.seconds;
    }
    bool bias_failed = false;
    const double thr = (o.r * std::pow((double)m, o.alpha) - 1.0) * o.tol / std::sqrt(2.0);
    std::vector<double> delta;
    FILE* logf = nullptr;
    if (o.log_path) {
        logf = std::fopen(o.log_path, "a");
        if (!logf) {
            err = std::string("log_path: cannot open ") + o.log_path;
            return MLMC_E_ARG;
        }
    }
    // one line per round: the state after it and the decisions taken from it
    auto log_round = [&](bool enough, bool bias_ok) {
        if (!logf) return;
        const int Ll = (int)acc.size() - 1;
        std::vector<int64_t> n(Ll + 1);
        std::vector<double> y(Ll + 1), v(Ll + 1);
        double var = 0.0;
        for (int l = 0; l <= Ll; ++l) {
            n[l] = acc[l].n;
            y[l] = acc[l].mean;
            v[l] = acc[l].n > 0 ? acc[l].m2 / (double)acc[l].n : 0.0;
            if (acc[l].n > 0) var += v[l] / (double)acc[l].n;
        }
        const double bias = std::fabs(acc[Ll].mean) / (std::pow((double)m, o.alpha) - 1.0);
        std::fprintf(logf, "{\"round\":%d,\"L\":%d,\"N\":", rounds_before + rounds, Ll);
        json_array(logf, n.data(), Ll + 1);
        std::fprintf(logf, ",\"N_next\":");
        json_array(logf, N.data(), (int)N.size());
        std::fprintf(logf, ",\"Yhat\":");
        json_array(logf, y.data(), Ll + 1);
        std::fprintf(logf, ",\"s2\":");
        json_array(logf, v.data(), Ll + 1);
        std::fprintf(logf, ",\"delta\":");
        json_array(logf, delta.data(), (int)delta.size());
        std::fprintf(logf, ",\"rmse\":%.17g,\"bias_ok\":%s,\"enough\":%s,\"seconds\":%.6f}\n",
                     std::sqrt(bias * bias + var), bias_ok ? "true" : "false", enough ? "true" : "false",
                     seconds_before + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
        std::fflush(logf);
    };
    mlmc_status status = MLMC_OK;
    while (rounds < std::max(1, o.max_rounds)) {
        ++rounds;
        std::vector<double> h(L + 1);
        for (int l = 0; l <= L; ++l) h[l] = 1.0 / ((double)n0 * std::pow((double)m, l));
        delta.assign(L + 1, 0.0);
        std::vector<mlmc_prec> prec(L + 1);
        mlmc_adapt_precision(L, h.data(), o.kp, o.alpha1, o.alpha2, o.beta1, o.beta2, o.contrast, delta.data(),
                             prec.data());
        if (o.form == MLMC_FORM_FP64_FIXED) std::fill(delta.begin(), delta.end(), o.fixed_delta);
        // the coarse member of level l is solved to the accuracy of level l-1 (Lemma 4.6's use of delta_{l-1})
        std::vector<double> dcoarse(L + 1, 0.0);
        for (int l = 1; l <= L; ++l) dcoarse[l] = delta[l - 1];
        std::vector<Request> req;
        for (int l = 0; l <= L; ++l)
            if (N[l] > acc[l].n) req.push_back({l, acc[l].n, (int)(N[l] - acc[l].n)});
        if (!req.empty()) {
            std::vector<mlmc_acc> got(req.size());
            std::memset(got.data(), 0, sizeof(mlmc_acc) * got.size());
            status = round(req, delta, dcoarse, got, res);
            if (status != MLMC_OK) break;
            for (size_t i = 0; i < req.size(); ++i) acc_merge(&acc[req[i].level], got[i]);
        }
        if (fixed) {
            log_round(true, true);
            break;
        }
        const bool enough = next_targets(m, o, acc, N);
        bias_failed = std::fabs(acc[L].mean) > thr;
        log_round(enough, !bias_failed);
        if (bias_failed && L < L_max) {
            ++L;
            N.push_back(o.N_init);
            mlmc_acc z;
            std::memset(&z, 0, sizeof(z));
            acc.push_back(z);
            continue;
        }
        if (enough) break;
    }
    if (logf) std::fclose(logf);
    if (status != MLMC_OK) return status;
    res->L = L;
    res->rounds = rounds_before + rounds;
    res->bias_failed = bias_failed ? 1 : 0;
    double est = 0.0, var = 0.0;
    for (int l = 0; l <= L; ++l) {
        res->N[l] = acc[l].n;
        res->Yhat[l] = acc[l].mean;
        res->s2[l] = acc[l].n > 0 ? acc[l].m2 / (double)acc[l].n : 0.0;
        res->delta[l] = l < (int)delta.size() ? delta[l] : 0.0;
        res->acc[l] = acc[l];
        est += acc[l].mean;
        if (acc[l].n > 0) var += res->s2[l] / (double)acc[l].n;
    }
    const double bias = std::fabs(acc[L].mean) / (std::pow((double)m, o.alpha) - 1.0);
    res->estimate = est;
    res->var_est = var;
    res->rmse = std::sqrt(bias * bias + var);
    res->seconds = seconds_before + std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return MLMC_OK;
}

mlmc_status check_options(const mlmc_options* o, int L_max, std::string& err) {
    if (!o) { err = "null options"; return MLMC_E_ARG; }
    if (!(o->tol > 0) || o->N_init < 2 || !(o->kp > 0 && o->kp < 1) || o->L_start < 0 || o->L_start > L_max) {
        err = "options: need tol > 0, N_init >= 2, 0 < kp < 1, 0 <= L_start <= L_max";
        return MLMC_E_ARG;
    }
    if (o->form < 0 || o->form > 2 || (o->force_prec >= 0 && !is_prec(o->force_prec)) ||
        (o->solver != MLMC_CG && o->solver != MLMC_MINRES && o->solver != MLMC_CHOLESKY) || o->max_iters < 1) {
        err = "options: bad form, precision, solver or max_iters";
        return MLMC_E_ARG;
    }
    if (o->chol_table != 0 && o->chol_table != 1) {
        err = "options: chol_table must be 0 or 1";
        return MLMC_E_ARG;
    }
    if (o->prec_rule != 0 && o->prec_rule != 1) {
        err = "options: prec_rule must be 0 or 1";
        return MLMC_E_ARG;
    }
    if (o->mixed_field != MLMC_FP64TC && o->mixed_field != MLMC_FP32) {
        err = "options: mixed_field must be MLMC_FP64TC or MLMC_FP32";
        return MLMC_E_ARG;
    }
    if (o->fixed_N)
        for (int l = 0; l <= o->L_start; ++l)
            if (o->fixed_N[l] < 1) { err = "fixed_N entries must be >= 1"; return MLMC_E_ARG; }
    return MLMC_OK;
}

}  // namespace

extern "C" {

const char* mlmc_version(void) { return "libmlmc 0.1 (sm_103a)"; }

int64_t mlmc_launch_count(void) { return g_launches.load(); }

const char* mlmc_last_error(const mlmc_ctx* ctx) {
    return ctx ? ctx->err.c_str() : create_error().c_str();
}

mlmc_status mlmc_create(const mlmc_problem* prob, int device, mlmc_ctx** out) {
    if (!out) return MLMC_E_ARG;
    *out = nullptr;
    create_error().clear();
    mlmc_status st = check_problem(prob, create_error());
    if (st != MLMC_OK) return st;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || device < 0 || device >= ndev) {
        create_error() = std::string("no CUDA device ") + std::to_string(device) + ": " +
                         (e != cudaSuccess ? cudaGetErrorString(e) : "out of range");
        return MLMC_E_CUDA;
    }
    if ((e = cudaSetDevice(device)) != cudaSuccess) {
        create_error() = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    mlmc_ctx* ctx = new (std::nothrow) mlmc_ctx();
    if (!ctx) return MLMC_E_NOMEM;
    ctx->prob = *prob;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    // the device error words of the synthesis and the solves, zero until a bounded wait runs out
    if ((e = cudaMalloc(&ctx->kl_err, 2 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(ctx->kl_err, 0, 2 * sizeof(unsigned))) != cudaSuccess) {
        create_error() = std::string("error words: ") + cudaGetErrorString(e);
        ctx->kl_err = nullptr;
        mlmc_destroy(ctx);
        return e == cudaErrorMemoryAllocation ? MLMC_E_NOMEM : MLMC_E_CUDA;
    }
    ctx->solve_err = ctx->kl_err + 1;
    for (int l = 0; l <= prob->L_max; ++l) {
        const int n = level_n(*prob, l);
        std::string err;
        e = upload_basis(ctx->basis[n], prob->field, n, err);
        ctx->prof.acc.h2d_bytes += (int64_t)sizeof(double) * prob->field.K * (1 + 2 * (n + 1));
        if (e != cudaSuccess) {
            create_error() = "basis upload for n=" + std::to_string(n) + ": " +
                             (err.empty() ? std::string(cudaGetErrorString(e)) : err);
            mlmc_destroy(ctx);
            return e == cudaErrorMemoryAllocation ? MLMC_E_NOMEM : MLMC_E_CUDA;
        }
    }
    *out = ctx;
    return MLMC_OK;
}

mlmc_status mlmc_set_seed(mlmc_ctx* ctx, uint64_t seed) {
    if (!ctx) return MLMC_E_ARG;
    ctx->prob.seed = seed;
    return MLMC_OK;
}

void mlmc_destroy(mlmc_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->basis) {
        kv.second.phi64.release();
        kv.second.phi16.release();
        kv.second.phix.release();
        kv.second.phiff.release();
        kv.second.ev.release();
    }
    for (auto& p : ctx->prof.kl_pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (cudaStream_t& a : ctx->aux)
        if (a) {
            cudaStreamSynchronize(a);
            cudaStreamDestroy(a);
            a = nullptr;
        }
    Workspace& w = ctx->ws;
    for (DevBuf& b : w.solver_slot) b.release();
    for (DevBuf* b : {&w.fields, &w.xi, &w.q, &w.misc, &w.split, &w.adj, &w.chol, &w.ahead[0], &w.ahead[1]}) b->release();
    if (ctx->kl_err) cudaFree(ctx->kl_err);
    if (ctx->order_ev) cudaEventDestroy(ctx->order_ev);
    if (ctx->prof.t0) cudaEventDestroy(ctx->prof.t0);
    delete ctx;
}

mlmc_status mlmc_set_wait_timeout(mlmc_ctx* ctx, double seconds) {
    if (!ctx || !(seconds > 0)) return MLMC_E_ARG;
    ctx->wait_timeout_s = seconds;
    return MLMC_OK;
}

// Reference event of the profile's launch intervals, recorded on the legacy stream.
static mlmc_status profile_mark_t0(mlmc_ctx* ctx) {
    if (!ctx->prof.t0) MLMC_CUDA_RET(ctx->err, cudaEventCreate(&ctx->prof.t0));
    MLMC_CUDA_RET(ctx->err, cudaEventRecord(ctx->prof.t0, nullptr));
    ctx->prof.solve_iv.clear();
    return MLMC_OK;
}

mlmc_status mlmc_profile_enable(mlmc_ctx* ctx, int on) {
    if (!ctx) return MLMC_E_ARG;
    cudaSetDevice(ctx->device);
    const bool was = ctx->prof.on;
    ctx->prof.on = on != 0;
    if (ctx->prof.on && !was) return profile_mark_t0(ctx);
    return MLMC_OK;
}

mlmc_status mlmc_profile_get(mlmc_ctx* ctx, mlmc_profile* out) {
    if (!ctx || !out) return MLMC_E_ARG;
    cudaSetDevice(ctx->device);
    MLMC_CUDA_RET(ctx->err, cudaDeviceSynchronize());
    for (auto& p : ctx->prof.kl_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->prof.acc.kl_launches += 1;
            ctx->prof.acc.kl_ms += ms;
            ctx->prof.acc.kl_bytes += p.bytes;
            ctx->prof.acc.kl_flops += p.flops;
        }
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    ctx->prof.kl_pending.clear();
    // union of the solve launches' intervals
    std::vector<std::pair<double, double>> iv = ctx->prof.solve_iv;
    std::sort(iv.begin(), iv.end());
    double busy = 0.0, cs = 0.0, ce = -1.0;
    for (const auto& x : iv) {
        if (x.first > ce) {
            if (ce > cs) busy += ce - cs;
            cs = x.first;
            ce = x.second;
        } else {
            ce = std::max(ce, x.second);
        }
    }
    if (ce > cs) busy += ce - cs;
    ctx->prof.acc.solve_busy_ms = busy;
    *out = ctx->prof.acc;
    return check_device_errors(ctx, nullptr);
}

mlmc_status mlmc_profile_reset(mlmc_ctx* ctx) {
    if (!ctx) return MLMC_E_ARG;
    mlmc_profile tmp;
    mlmc_status s = mlmc_profile_get(ctx, &tmp);
    std::memset(&ctx->prof.acc, 0, sizeof(ctx->prof.acc));
    const mlmc_status t = profile_mark_t0(ctx);
    return s != MLMC_OK ? s : t;
}

mlmc_status mlmc_debug_set_wait_extra(mlmc_ctx* ctx, int extra) {
    if (!ctx || extra < 0) return MLMC_E_ARG;
    ctx->wait_extra = extra;
    return MLMC_OK;
}

mlmc_status mlmc_set_precond(mlmc_ctx* ctx, mlmc_precond pc, int nu, int coarse_sweeps, double omega) {
    if (!ctx) return MLMC_E_ARG;
    if ((pc != MLMC_PC_JACOBI && pc != MLMC_PC_MG) || nu < 0 || nu > 2 || coarse_sweeps < 0 ||
        (coarse_sweeps > 0 && (coarse_sweeps % 2 != 0 || coarse_sweeps < 2)) || !(omega >= 0.0 && omega < 1.0))
        return fail(ctx, MLMC_E_ARG, "set_precond: bad preconditioner, nu (1..2), coarse sweeps (even) or omega");
    ctx->precond = pc;
    if (nu > 0) ctx->mg_nu = nu;
    if (coarse_sweeps > 0) ctx->mg_coarse = coarse_sweeps;
    if (omega > 0.0) ctx->mg_omega = omega;
    return MLMC_OK;
}

mlmc_status mlmc_set_full_multigrid(mlmc_ctx* ctx, int on) {
    if (!ctx || (on != 0 && on != 1)) return MLMC_E_ARG;
    ctx->mg_fmg = on;
    return MLMC_OK;
}

mlmc_status mlmc_set_mg_coarsest(mlmc_ctx* ctx, int min_cells) {
    if (!ctx) return MLMC_E_ARG;
    if (min_cells < 2 || min_cells > 64) return fail(ctx, MLMC_E_ARG, "set_mg_coarsest: min_cells in 2..64");
    ctx->mg_min = min_cells;
    return MLMC_OK;
}

mlmc_status mlmc_set_inner_tolerance(mlmc_ctx* ctx, double theta, double tau_min) {
    if (!ctx) return MLMC_E_ARG;
    if (!(theta >= 0.0 && theta < 1.0) || !(tau_min < 0.5))
        return fail(ctx, MLMC_E_ARG, "set_inner_tolerance: theta in [0, 1), tau_min < 0.5");
    if (theta > 0.0) ctx->inner_theta = theta;
    ctx->inner_tau_min = tau_min > 0.0 ? tau_min : -1.0;
    return MLMC_OK;
}

mlmc_status mlmc_set_cholesky_precision(mlmc_ctx* ctx, mlmc_prec u, mlmc_prec u_r) {
    if (!ctx) return MLMC_E_ARG;
    const bool ok = (u == MLMC_FP64 && u_r == MLMC_FP64) || (u == MLMC_FP32 && (u_r == MLMC_FP32 || u_r == MLMC_FP64)) ||
                    (u == MLMC_FP16S && u_r == MLMC_FP16S);
    if (!ok)
        return fail(ctx, MLMC_E_ARG, "set_cholesky_precision: (u, u_r) must be (FP64, FP64), (FP32, FP64), "
                                     "(FP32, FP32) or (FP16S, FP16S)");
    ctx->chol_u = u;
    ctx->chol_ur = u_r;
    return MLMC_OK;
}

mlmc_status mlmc_set_sample_ahead(mlmc_ctx* ctx, int on) {
    if (!ctx || (on != 0 && on != 1)) return MLMC_E_ARG;
    ctx->sample_ahead = on != 0;
    return MLMC_OK;
}

mlmc_status mlmc_set_autotune(mlmc_ctx* ctx, int on) {
    if (!ctx) return MLMC_E_ARG;
    ctx->autotune = on != 0;
    return MLMC_OK;
}

int mlmc_autotune_count(const mlmc_ctx* ctx) { return ctx ? (int)ctx->tune_order.size() : 0; }

mlmc_status mlmc_autotune_entry(const mlmc_ctx* ctx, int i, mlmc_tune_entry* out) {
    if (!ctx || !out || i < 0 || i >= (int)ctx->tune_order.size()) return MLMC_E_ARG;
    const std::string& key = ctx->tune_order[(size_t)i];
    const TuneChoice& t = ctx->tune.at(key);
    std::memset(out, 0, sizeof(*out));
    std::strncpy(out->shape, key.c_str(), sizeof(out->shape) - 1);
    out->prec = t.prec;
    out->solver = t.solver;
    out->precond = t.precond;
    out->med_items = t.med_items;
    out->ring = t.ring;
    out->nu = t.nu;
    out->mg_min = t.mg_min;
    out->mg_coarse = t.mg_coarse;
    out->mg_omega = t.mg_omega;
    out->mg_smem = t.mg_smem;
    out->theta = t.theta;
    out->tau_min = t.tau_min;
    out->best_ms = t.best_ms;
    out->default_ms = t.default_ms;
    out->trials = t.trials;
    return MLMC_OK;
}

mlmc_status mlmc_debug_set_medium_items(mlmc_ctx* ctx, int items) {
    // a quarter's sweeps need a row's chunks (n/4 + 1) to fit its 128 threads: n <= 256 is far inside
    if (!ctx || (items != -1 && (items < 512 || items > 16384))) return MLMC_E_ARG;
    ctx->med_items = items;
    return MLMC_OK;
}

mlmc_status mlmc_debug_fail_allocation(int64_t after) {
    if (after < -1) return MLMC_E_ARG;
    g_fail_alloc.store(after);
    return MLMC_OK;
}

mlmc_status mlmc_debug_set_solve_ring(mlmc_ctx* ctx, int ring) {
    if (!ctx || ring < -1 || ring == 1 || ring > 4) return MLMC_E_ARG;
    ctx->solve_ring = ring;
    return MLMC_OK;
}

// Pitch argument of the field calls: 0 (dense) or at least the level's (n+1)^2 nodes.
bool good_pitch(const mlmc_ctx* ctx, int level, int64_t ld) {
    const int n = level_n(ctx->prob, level);
    return ld == 0 || ld >= (int64_t)(n + 1) * (n + 1);
}

mlmc_status mlmc_sample_fields(mlmc_ctx* ctx, int level, uint64_t first, int S, double* xi, void* a,
                               int64_t a_ld, mlmc_prec field_prec, void* stream) {
    if (!ctx) return MLMC_E_ARG;
    if (level < 0 || level > ctx->prob.L_max || S < 0 || (S > 0 && !a) || !is_field_prec(field_prec) ||
        !good_pitch(ctx, level, a_ld))
        return fail(ctx, MLMC_E_ARG, "sample_fields: bad level, S, output, pitch or field precision");
    if (S == 0) return MLMC_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* xbuf = xi;
    if (!xbuf) {
        MLMC_CUDA_RET(ctx->err, ctx->ws.xi.reserve(sizeof(double) * (size_t)S * ctx->prob.field.K));
        xbuf = ctx->ws.xi.as<double>();
    }
    MLMC_CUDA_RET(ctx->err, ctx_order_begin(ctx, st));
    MLMC_CUDA_RET(ctx->err, launch_philox_normals(ctx->prob.seed, level, first, S, ctx->prob.field.K, xbuf, st));
    const mlmc_status s = synth(ctx, level, S, xbuf, a, a_ld, field_prec, st);
    if (s != MLMC_OK) return s;
    MLMC_CUDA_RET(ctx->err, ctx_order_end(ctx, st));
    return MLMC_OK;
}

mlmc_status mlmc_synthesize_fields(mlmc_ctx* ctx, int level, int S, const double* xi, void* a, int64_t a_ld,
                                   mlmc_prec field_prec, void* stream) {
    if (!ctx) return MLMC_E_ARG;
    if (level < 0 || level > ctx->prob.L_max || S < 0 || (S > 0 && (!a || !xi)) || !is_field_prec(field_prec) ||
        !good_pitch(ctx, level, a_ld))
        return fail(ctx, MLMC_E_ARG, "synthesize_fields: bad level, S, pointers, pitch or field precision");
    if (S == 0) return MLMC_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MLMC_CUDA_RET(ctx->err, ctx_order_begin(ctx, st));
    const mlmc_status s = synth(ctx, level, S, xi, a, a_ld, field_prec, st);
    if (s != MLMC_OK) return s;
    MLMC_CUDA_RET(ctx->err, ctx_order_end(ctx, st));
    return MLMC_OK;
}

mlmc_status mlmc_apply_operator(int n, int S, const void* a, mlmc_prec a_prec, int a_n, mlmc_prec op_prec,
                                const void* x, void* y, mlmc_prec vec_prec, void* stream) {
    if (n < 2 || S < 0 || a_n < n || a_n % n != 0 || !is_master_prec(a_prec) || !is_prec(op_prec) ||
        !is_master_prec(vec_prec))
        return MLMC_E_ARG;
    if ((op_prec == MLMC_FP64) != (vec_prec == MLMC_FP64)) return MLMC_E_ARG;
    if (S == 0) return MLMC_OK;
    if (!a || !x || !y) return MLMC_E_ARG;
    const cudaError_t e = launch_apply_operator(n, S, a, a_prec == MLMC_FP64, a_n, op_prec, x, y,
                                                vec_prec == MLMC_FP64, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MLMC_OK : MLMC_E_CUDA;
}

mlmc_status mlmc_level_solve(mlmc_ctx* ctx, int n, int S, const void* a, mlmc_prec a_prec, int a_n, int64_t a_ld,
                             mlmc_prec prec, mlmc_solver solver, double delta, int max_iters, double* u,
                             double* Q, int32_t* iters, double* relres, int32_t* flags, void* stream) {
    if (!ctx) return MLMC_E_ARG;
    if (n < 2 || n > 2048 || S < 0 || a_n < n || a_n % n != 0 || !is_master_prec(a_prec) ||
        (a_ld != 0 && a_ld < (int64_t)(a_n + 1) * (a_n + 1)) ||
        !(is_prec(prec) || (solver == MLMC_CHOLESKY && prec == MLMC_FP8S)) ||
        (solver != MLMC_CG && solver != MLMC_MINRES && solver != MLMC_CHOLESKY) || !(delta > 0) || max_iters < 1)
        return fail(ctx, MLMC_E_ARG, "level_solve: bad n, S, a_n, a_ld, precision, solver, delta or max_iters");
    if (S == 0) return MLMC_OK;
    if (!a || !Q) return fail(ctx, MLMC_E_ARG, "level_solve: null a or Q");
    cudaSetDevice(ctx->device);
    SolveGroup g;
    g.n = n;
    g.S = S;
    g.a = a;
    g.a_fp64 = (a_prec == MLMC_FP64);
    g.a_n = a_n;
    g.a_ld = a_ld;
    g.delta = delta;
    g.Q = Q;
    g.u = u;
    g.iters = iters;
    g.relres = relres;
    g.flags = flags;
    SolveConfig cfg;
    cfg.prec = prec;
    cfg.solver = solver;
    cfg.max_iters = max_iters;
    cfg.chol_u = ctx->chol_u;
    cfg.chol_ur = ctx->chol_ur;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MLMC_CUDA_RET(ctx->err, ctx_order_begin(ctx, st));
    const mlmc_status s = launch_solve_async(ctx, {g}, cfg, st);
    if (s != MLMC_OK) return s;
    MLMC_CUDA_RET(ctx->err, ctx_order_end(ctx, st));
    return MLMC_OK;
}

mlmc_status mlmc_sync(mlmc_ctx* ctx, void* stream) {
    if (!ctx) return MLMC_E_ARG;
    cudaSetDevice(ctx->device);
    return check_device_errors(ctx, static_cast<cudaStream_t>(stream));
}

void mlmc_acc_merge(mlmc_acc* into, const mlmc_acc* other) {
    if (into && other) acc_merge(into, *other);
}

mlmc_status mlmc_level_stats(mlmc_ctx* ctx, int S, const double* Qf, const double* Qc, mlmc_acc* acc,
                             void* stream) {
    if (!ctx || S < 0 || !acc || (S > 0 && !Qf)) return ctx ? fail(ctx, MLMC_E_ARG, "level_stats: bad args") : MLMC_E_ARG;
    if (S == 0) return MLMC_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MLMC_CUDA_RET(ctx->err, ctx->ws.misc.reserve(sizeof(mlmc_acc)));
    MLMC_CUDA_RET(ctx->err, ctx_order_begin(ctx, st));
    MLMC_CUDA_RET(ctx->err, launch_level_stats(S, Qf, Qc, ctx->ws.misc.as<mlmc_acc>(), st));
    mlmc_acc got;
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(&got, ctx->ws.misc.ptr, sizeof(got), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_RET(ctx->err, ctx_order_end(ctx, st));
    MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
    ctx->prof.acc.d2h_bytes += (int64_t)sizeof(got);
    const mlmc_status s = check_device_errors(ctx, st);
    if (s != MLMC_OK) return s;
    acc_merge(acc, got);
    return MLMC_OK;
}

mlmc_status mlmc_adapt_precision(int L, const double* h, double kp, double alpha1, double alpha2, double beta1,
                                 double beta2, double contrast, double* delta, mlmc_prec* prec) {
    if (L < 0 || !h || !delta || !(kp > 0) || !(alpha2 > 0) || !(beta2 > 0)) return MLMC_E_ARG;
    for (int l = 0; l <= L; ++l) {
        if (!(h[l] > 0)) return MLMC_E_ARG;
        delta[l] = std::pow(kp * std::pow(h[l], beta1), 1.0 / beta2);
    }
    delta[L] = std::min(delta[L], std::pow(kp * std::pow(h[L], alpha1), 1.0 / alpha2));
    if (prec)
        for (int l = 0; l <= L; ++l) prec[l] = pick_prec(h[l], delta[l], contrast);
    return MLMC_OK;
}

void mlmc_default_options(mlmc_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-3;
    o->L_start = 1;
    o->N_init = 100;
    o->kp = 0.05;
    o->alpha1 = 2.0;
    o->alpha2 = 1.0;
    o->beta1 = 4.0;
    o->beta2 = 2.0;
    o->alpha = 2.0;
    o->gamma = 2.0;
    o->r = 1.0;
    o->form = MLMC_FORM_MIXED;
    o->fixed_delta = 1e-10;
    o->force_prec = -1;
    o->solver = MLMC_CG;
    o->max_iters = 100000;
    o->max_rounds = 100;
    o->fixed_N = nullptr;
    o->contrast = 1.0;
    o->mixed_field = MLMC_FP64TC;
}

mlmc_status mlmc_estimate_host(int m, int L_max, int n0, const mlmc_options* opts, mlmc_sampler_fn sampler,
                               void* user, mlmc_result* res) {
    std::string err;
    if (!sampler || !res || m < 2 || n0 < 2 || L_max < 0 || L_max >= MLMC_MAX_LEVELS) return MLMC_E_ARG;
    if (check_options(opts, L_max, err) != MLMC_OK) return MLMC_E_ARG;
    RoundFn round = [&](const std::vector<Request>& req, const std::vector<double>& df, const std::vector<double>&,
                        std::vector<mlmc_acc>& out, mlmc_result*) -> mlmc_status {
        std::vector<double> Y;
        for (size_t i = 0; i < req.size(); ++i) {
            Y.assign(req[i].count, 0.0);
            if (sampler(user, req[i].level, req[i].first, req[i].count, df.data(), Y.data()) != 0) return MLMC_E_ARG;
            for (double y : Y) acc_push(&out[i], y);
        }
        return MLMC_OK;
    };
    return alg41(m, L_max, n0, *opts, round, res, err);
}

mlmc_status mlmc_estimate(mlmc_ctx* ctx, const mlmc_options* opts, mlmc_result* res) {
    if (!ctx || !res) return MLMC_E_ARG;
    if (check_options(opts, ctx->prob.L_max, ctx->err) != MLMC_OK) return MLMC_E_ARG;
    cudaSetDevice(ctx->device);
    const mlmc_options o = *opts;
    const mlmc_problem& p = ctx->prob;
    const int K = p.field.K;
    const cudaStream_t st = nullptr;
    MLMC_CUDA_RET(ctx->err, ctx_order_begin(ctx, st));
    // the master coefficient: FP64 on the FP64 pipe for the FP64 forms; for the mixed form the option's
    // tensor-core field (FP64 to about 1e-9 in log a by default, or FP32)
    const mlmc_prec field_prec = (o.form == MLMC_FORM_MIXED) ? (mlmc_prec)o.mixed_field : MLMC_FP64;
    const size_t felem = field_prec == MLMC_FP32 ? sizeof(float) : sizeof(double);
    int32_t flags_or = 0;
    std::vector<int64_t> iters_lvl(MLMC_MAX_LEVELS, 0), dofs_lvl(MLMC_MAX_LEVELS, 0);
    std::vector<int32_t> prec_lvl(MLMC_MAX_LEVELS, -1);
    std::vector<int64_t> retries_lvl(MLMC_MAX_LEVELS, 0);
    // calibrated precision rule: per level, the largest contrast max(a) / min(a) of its samples so far
    std::vector<double> cal_contrast(MLMC_MAX_LEVELS, 0.0), cal_amin(MLMC_MAX_LEVELS, 1e300),
        cal_amax(MLMC_MAX_LEVELS, 0.0);
    const bool calibrate = o.prec_rule == 1 && o.form == MLMC_FORM_MIXED && o.solver != MLMC_CHOLESKY &&
                           o.force_prec < 0;

    // Samples solved ahead of the round that asks for them.  A round's launches leave SMs to spare beside
    // the finest level's few large systems, so extra samples of the cheap levels, which the next round of
    // Alg. 4.1 will probably ask for, cost little there; that round then copies their QoIs instead of
    // synthesising fields and launching solves, and saves its launch latencies.  How many: up to 1.25 times
    // the sample counts the last estimate on this context ended with, within a tenth of the round's
    // unknowns.
    // A wrong guess costs time, never a result: a sample's field and solve do not depend on the batch it
    // is in, the level statistics cover exactly the range each round asks for, and the counters of a
    // sample count in the round that asks for it.  Those a round does not ask for are kept for the later
    // rounds; they are used only by a round that solves their level to the same delta in the same
    // precision class, and dropped otherwise.
    struct Ahead {
        bool valid = false;
        int64_t first = 0;   // the samples first .. first + count - 1 of the level
        int count = 0;
        double df = 0.0, dc = 0.0;
        int cls_f = -1, cls_c = -1;
        size_t qf = 0, qc = 0;   // offsets (doubles) of their Qf and Qc rows in the current ahead buffer
        std::vector<int32_t> it_f, it_c, fl_f, fl_c;   // final iterations and flags of each sample
        std::vector<int64_t> abandoned;                // iterations of low-precision attempts retried in FP64
        std::vector<int32_t> retried;
    };
    std::vector<Ahead> ahead(MLMC_MAX_LEVELS);
    int ahead_buf = 0;   // the ahead buffer holding the entries' rows (the other one receives the next round's)
    // not with fixed sample counts (one round), nor under the calibrated rule (whose precision choice
    // depends on the fields of each round)
    const bool use_ahead = ctx->sample_ahead && !o.fixed_N && !calibrate;

    RoundFn round = [&](const std::vector<Request>& req, const std::vector<double>& df, const std::vector<double>& dc,
                        std::vector<mlmc_acc>& out, mlmc_result*) -> mlmc_status {
        const NvtxRange range_round("mlmc round");
        // ---- memory plan of the round
        const int L = (int)df.size() - 1;
        std::vector<double> h(L + 1);
        for (int l = 0; l <= L; ++l) h[l] = 1.0 / level_n(p, l);
        std::vector<mlmc_prec> prec_rule(L + 1);
        std::vector<double> dtmp(L + 1);
        mlmc_adapt_precision(L, h.data(), o.kp, o.alpha1, o.alpha2, o.beta1, o.beta2, o.contrast, dtmp.data(),
                             prec_rule.data());
        // precision of a solve on the grid of level g with a field of level fl (fl = g + 1 for the coarse
        // member of a level pair)
        auto prec_for = [&](int g, int fl) -> mlmc_prec {
            if (o.form != MLMC_FORM_MIXED) return MLMC_FP64;
            if (o.force_prec >= 0) return (mlmc_prec)o.force_prec;
            // the Cholesky solver of Sec. 5.2: Table 1 (right), a half factor on level 0 and single above; or
            // the quarter-precision setting, q43 (FP8 E4M3) on level 0 and half above
            if (o.solver == MLMC_CHOLESKY) {
                if (o.chol_table == 1) return g == 0 ? MLMC_FP8S : MLMC_FP16S;
                return g == 0 ? MLMC_FP16S : MLMC_FP32;
            }
            if (calibrate) return pick_prec_calibrated(h[g], df[g], cal_contrast[fl], cal_amin[fl], cal_amax[fl]);
            return prec_rule[g];
        };
        auto prec_of = [&](int l) -> mlmc_prec { return prec_for(l, l); };
        // launch class of a solve: the factor / inner precision, plus for the Cholesky solver the working
        // and residual precision (bits 4-5: 0 double, 1 single, 2 half) -- Table 1 (right): single on
        // levels 0 and 1 (hhss, ssss), double above (ssdd); the quarter-precision setting: half on level 0
        // (qhhh), single above (hhss); double throughout for the FP64 forms (dddd)
        auto class_of = [&](int g, int fl) -> int {
            const int p = prec_for(g, fl);
            if (o.solver != MLMC_CHOLESKY || o.form != MLMC_FORM_MIXED) return p;
            int w = 0;
            if (o.chol_table == 1) w = g == 0 ? 2 : 1;
            else w = g <= 1 ? 1 : 0;
            return p | (w << 4);
        };
        // each field row padded to whole 128-byte lines (32 elements), so that the synthesis writes full lines
        auto fpitch = [&](int l) -> long long {
            const int n = level_n(p, l);
            return ((long long)(n + 1) * (n + 1) + 31) / 32 * 32;
        };
        // ---- samples of each request already solved ahead (earlier rounds), and new ones to solve ahead;
        // an entry that does not fit its level's request is dropped
        std::vector<int> used(req.size(), 0);
        for (size_t i = 0; i < req.size(); ++i) {
            const int l = req[i].level;
            Ahead& a = ahead[l];
            if (a.valid && a.first == req[i].first && a.df == df[l] && a.cls_f == class_of(l, l) &&
                (l == 0 || (a.dc == dc[l] && a.cls_c == class_of(l - 1, l))))
                used[i] = std::min(req[i].count, a.count);
            else
                a.valid = false;
        }
        // the work of the round: what each request still needs, then the samples solved ahead (req < 0)
        struct Work {
            int level;
            int64_t first;
            int count;
            int req;
        };
        std::vector<Work> work;
        for (size_t i = 0; i < req.size(); ++i)
            work.push_back({req[i].level, req[i].first + used[i], req[i].count - used[i], (int)i});
        auto unknowns = [&](int l) {
            const double n = level_n(p, l), nc = n / p.m;
            return (n - 1) * (n - 1) + (l > 0 ? (nc - 1) * (nc - 1) : 0.0);
        };
        // whether a level's solves are the same in any batch: not if a member's group size follows the
        // rest of its launch (the per-launch group choice)
        auto batch_free = [&](int l) {
            const int n = level_n(p, l);
            auto fixed = [](int k) { return size_class(k, kMedItems) == size_class(k, kMedItemsWide); };
            return fixed(n) && (l == 0 || fixed(n / p.m));
        };
        if (use_ahead) {
            // up to 1.25 times the sample counts of the last estimate, on the levels where that estimate
            // went beyond this round's samples (the counts follow sampled variances: with 100 initial
            // samples they vary by about a tenth between seeds), within a tenth of the round's unknowns
            double budget = 0.0;
            for (const Request& r : req) budget += 0.1 * r.count * unknowns(r.level);
            for (size_t i = 0; i < req.size(); ++i) {
                const Request& r = req[i];
                if (!batch_free(r.level)) continue;
                // after the samples already held beyond this request
                const int64_t end = r.first + r.count + (used[i] ? ahead[r.level].count - used[i] : 0);
                const int64_t hint = ctx->ahead_hint[r.level];
                const int64_t want = hint > end ? hint + (hint + 3) / 4 - end : 0;
                const int64_t fit = (int64_t)(budget / unknowns(r.level));
                const int extra = (int)std::min<int64_t>(std::min(want, fit), 1 << 30);
                if (extra <= 0) continue;
                budget -= extra * unknowns(r.level);
                work.push_back({r.level, end, extra, -1});
            }
        }
        // QoI rows: every request's whole range (solved-ahead part first), then the samples solved ahead
        size_t fbytes = 0, xbytes = 0, qn = 0;
        std::vector<size_t> qoff(req.size());
        for (size_t i = 0; i < req.size(); ++i) {
            qoff[i] = qn;
            qn += (size_t)req[i].count;
        }
        std::vector<size_t> foff(work.size()), xoff(work.size()), wq(work.size());
        for (size_t w = 0; w < work.size(); ++w) {
            foff[w] = fbytes;
            fbytes += (size_t)work[w].count * (size_t)fpitch(work[w].level) * felem;
            fbytes = (fbytes + 255) / 256 * 256;
            xoff[w] = xbytes;
            xbytes += (size_t)work[w].count * K * sizeof(double);
            if (work[w].req >= 0) {
                wq[w] = qoff[work[w].req] + used[work[w].req];
            } else {
                wq[w] = qn;
                qn += (size_t)work[w].count;
            }
        }
        MLMC_CUDA_RET(ctx->err, ctx->ws.fields.reserve(fbytes));
        MLMC_CUDA_RET(ctx->err, ctx->ws.xi.reserve(std::max<size_t>(xbytes, 8)));
        // Qf, Qc (doubles), iters and flags for fine and coarse (int32)
        const size_t qbytes = qn * (2 * sizeof(double) + 4 * sizeof(int32_t));
        MLMC_CUDA_RET(ctx->err, ctx->ws.q.reserve(qbytes));
        MLMC_CUDA_RET(ctx->err, ctx->ws.misc.reserve(std::max(sizeof(mlmc_acc) * req.size(),
                                                               calibrate ? 2 * qn * sizeof(double) : 0)));
        char* fb = ctx->ws.fields.as<char>();
        double* xb = ctx->ws.xi.as<double>();
        double* Qf = ctx->ws.q.as<double>();
        double* Qc = Qf + qn;
        int32_t* itf = reinterpret_cast<int32_t*>(Qc + qn);
        int32_t* itc = itf + qn;
        int32_t* flf = itc + qn;
        int32_t* flc = flf + qn;
        MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(Qc, 0, qn * sizeof(double), st));
        MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(itc, 0, qn * sizeof(int32_t), st));
        MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(flc, 0, qn * sizeof(int32_t), st));
        // ---- QoIs of the samples solved ahead, into their requests' rows
        for (size_t i = 0; i < req.size(); ++i) {
            if (!used[i]) continue;
            const Ahead& a = ahead[req[i].level];
            const double* src = ctx->ws.ahead[ahead_buf].as<double>();
            MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(Qf + qoff[i], src + a.qf, used[i] * sizeof(double),
                                                    cudaMemcpyDeviceToDevice, st));
            if (req[i].level > 0)
                MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(Qc + qoff[i], src + a.qc, used[i] * sizeof(double),
                                                        cudaMemcpyDeviceToDevice, st));
        }
        // ---- fields of the work
        for (size_t w = 0; w < work.size(); ++w) {
            if (work[w].count == 0) continue;
            const NvtxRange range_fields("fields");
            const mlmc_status s = mlmc_sample_fields(ctx, work[w].level, (uint64_t)work[w].first, work[w].count,
                                                     xb + xoff[w] / sizeof(double), fb + foff[w],
                                                     fpitch(work[w].level), field_prec, (void*)st);
            if (s != MLMC_OK) return s;
        }
        // ---- calibrated rule: the contrast of every new field, per level (no samples are solved ahead
        // under this rule, so the work is the requests)
        if (calibrate) {
            double* rng = ctx->ws.misc.as<double>();
            for (size_t w = 0; w < work.size(); ++w) {
                const int n = level_n(p, work[w].level);
                MLMC_CUDA_RET(ctx->err, launch_field_range(work[w].count, (n + 1) * (n + 1), fpitch(work[w].level),
                                                           fb + foff[w], field_prec != MLMC_FP32, rng + 2 * wq[w],
                                                           st));
            }
            std::vector<double> hr(2 * qn);
            MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(hr.data(), rng, 2 * qn * sizeof(double), cudaMemcpyDeviceToHost, st));
            MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
            ctx->prof.acc.d2h_bytes += (int64_t)(2 * qn * sizeof(double));
            for (size_t w = 0; w < work.size(); ++w) {
                const int l = work[w].level;
                for (int k = 0; k < work[w].count; ++k) {
                    const double lo = hr[2 * (wq[w] + k)], hi = hr[2 * (wq[w] + k) + 1];
                    cal_amin[l] = std::min(cal_amin[l], lo);
                    cal_amax[l] = std::max(cal_amax[l], hi);
                    if (lo > 0) cal_contrast[l] = std::max(cal_contrast[l], hi / lo);
                }
            }
        }
        // ---- one resident-solve launch per inner-precision class: every fine and coarse member
        std::map<int, std::vector<SolveGroup>> classes;
        std::map<int, std::vector<int>> class_work;   // work item of each group, for the counters
        for (const Request& r : req) prec_lvl[r.level] = prec_of(r.level);
        for (size_t w = 0; w < work.size(); ++w) {
            if (work[w].count == 0) continue;
            const int l = work[w].level;
            const int n = level_n(p, l);
            SolveGroup gf;
            gf.n = n;
            gf.S = work[w].count;
            gf.a = fb + foff[w];
            gf.a_fp64 = field_prec != MLMC_FP32;
            gf.a_n = n;
            gf.a_ld = fpitch(l);
            gf.delta = df[l];
            gf.Q = Qf + wq[w];
            gf.iters = itf + wq[w];
            gf.flags = flf + wq[w];
            classes[class_of(l, l)].push_back(gf);
            class_work[class_of(l, l)].push_back((int)w);
            if (l > 0) {
                SolveGroup gc = gf;
                gc.n = n / p.m;
                gc.delta = dc[l];
                gc.Q = Qc + wq[w];
                gc.iters = itc + wq[w];
                gc.flags = flc + wq[w];
                classes[class_of(l - 1, l)].push_back(gc);
                class_work[class_of(l - 1, l)].push_back((int)w);
            }
        }
        // the classes share no data: their launches run concurrently (the smaller ones fill the
        // SMs that the finest level's few large systems leave idle)
        std::vector<SolveBatch> batches;
        for (auto& kv : classes) {
            SolveBatch b;
            b.groups = kv.second;
            b.cfg.prec = kv.first & 15;
            b.cfg.solver = o.solver;
            b.cfg.max_iters = o.max_iters;
            const int w = (kv.first >> 4) & 3;
            b.cfg.chol_u = w == 0 ? MLMC_FP64 : (w == 1 ? MLMC_FP32 : MLMC_FP16S);
            b.cfg.chol_ur = b.cfg.chol_u;
            batches.push_back(std::move(b));
        }
        // the launches are read back with the statistics below: no wait here
        std::vector<PendingSolve> pend;
        if (!batches.empty()) {
            const NvtxRange range_solves("solves");
            const mlmc_status s = launch_solve_batches(ctx, batches, st, pend);
            if (s != MLMC_OK) return s;
        }
        // ---- read-back: level statistics, iterations and flags of every solve, and the device error words,
        // with one synchronisation (a retry below, rare, reads back again)
        mlmc_acc* dacc = ctx->ws.misc.as<mlmc_acc>();
        std::vector<int32_t> hit(4 * qn);   // itf, itc, flf, flc
        auto read_back = [&]() -> mlmc_status {
            for (size_t i = 0; i < req.size(); ++i) {
                MLMC_CUDA_RET(ctx->err, launch_level_stats(req[i].count, Qf + qoff[i],
                                                            req[i].level > 0 ? Qc + qoff[i] : nullptr, dacc + i, st));
            }
            unsigned w[2] = {0u, 0u};
            MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(out.data(), dacc, sizeof(mlmc_acc) * req.size(),
                                                    cudaMemcpyDeviceToHost, st));
            MLMC_CUDA_RET(ctx->err,
                          cudaMemcpyAsync(hit.data(), itf, 4 * qn * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(w, ctx->kl_err, sizeof(w), cudaMemcpyDeviceToHost, st));
            MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
            ctx->prof.acc.d2h_bytes += (int64_t)(sizeof(mlmc_acc) * req.size() + 4 * qn * sizeof(int32_t));
            if (w[0] != 0u || w[1] != 0u) return check_device_errors(ctx, st);   // clears them, reports
            return MLMC_OK;
        };
        {
            const mlmc_status s = read_back();   // synchronises st, which waited for every solve launch
            if (s != MLMC_OK) {
                cudaStreamSynchronize(st);
                finish_solves(ctx, pend);
                return s;
            }
            const mlmc_status f = finish_solves(ctx, pend);   // the launches' counters, while profiling
            if (f != MLMC_OK) return f;
        }
        // iterations of abandoned low-precision attempts and retry counts, per QoI row
        std::vector<int64_t> abandoned(qn, 0);
        std::vector<int32_t> retried(qn, 0);
        // ---- Cor. 3.4 safety net: the low-precision conditions can fail for a sample
        // whose coefficient is rougher than the precision rule assumed; a refinement
        // that stagnated or ran out of iterations is re-run with FP64 inner arithmetic
        // to the same delta (Alg. 2.1 with u_f = u), in one more launch.
        if (o.form == MLMC_FORM_MIXED && classes.size() > (classes.count(MLMC_FP64) ? 1u : 0u)) {
            const int32_t* hfl = hit.data() + 2 * qn;   // fine then coarse flags
            const int32_t* hit2 = hit.data();           // fine then coarse iterations
            std::vector<SolveGroup> retry;
            for (auto& kv : classes) {
                if (kv.first == MLMC_FP64) continue;   // FP64 inner (or the dddd Cholesky)
                for (size_t gi = 0; gi < kv.second.size(); ++gi) {
                    const SolveGroup& g = kv.second[gi];
                    const size_t elem = g.a_fp64 ? sizeof(double) : sizeof(float);
                    const size_t aV = (size_t)field_pitch(g);
                    for (int smp = 0; smp < g.S; ++smp) {
                        const size_t q = (size_t)(g.flags - flf) + smp;
                        // a low-precision Cholesky factor that overflowed (Sec. 5.2) is retried like a stall
                        const int32_t retry_on = MLMC_F_STAGNATED | MLMC_F_MAXIT |
                                                 (o.solver == MLMC_CHOLESKY ? MLMC_F_NONFINITE : 0);
                        if (!(hfl[q] & retry_on)) continue;
                        SolveGroup r = g;
                        r.S = 1;
                        r.a = static_cast<const char*>(g.a) + smp * aV * elem;
                        r.Q = g.Q + smp;
                        r.iters = g.iters + smp;
                        r.flags = g.flags + smp;
                        retry.push_back(r);
                        // the abandoned attempt's iterations (fine member's row q, coarse member's row q)
                        const bool coarse = g.flags >= flc;
                        const size_t row = coarse ? q - qn : q;
                        abandoned[row] += hit2[q];
                        retried[row] += 1;
                    }
                }
            }
            if (!retry.empty()) {
                SolveConfig cfg;
                cfg.prec = MLMC_FP64;
                cfg.solver = o.solver;
                cfg.max_iters = o.max_iters;
                const mlmc_status s = run_solve_batch(ctx, retry, cfg, st);
                if (s != MLMC_OK) return s;
                const mlmc_status s2 = read_back();   // the statistics of the re-run samples
                if (s2 != MLMC_OK) return s2;
            }
        }
        // ---- counters of the requests: their samples solved ahead, then the rest
        for (size_t i = 0; i < req.size(); ++i) {
            const int l = req[i].level;
            const Ahead& a = ahead[l];
            for (int s = 0; s < used[i]; ++s) {
                iters_lvl[l] += a.abandoned[s] + a.it_f[s] + a.it_c[s];
                retries_lvl[l] += a.retried[s];
                flags_or |= a.fl_f[s];
                if (l > 0) flags_or |= a.fl_c[s];
            }
            dofs_lvl[l] += (int64_t)req[i].count * (int64_t)unknowns(l);
            for (int s = used[i]; s < req[i].count; ++s) {
                const size_t q = qoff[i] + s;
                iters_lvl[l] += abandoned[q] + hit[q] + hit[qn + q];
                retries_lvl[l] += retried[q];
                const int32_t ff = hit[2 * qn + q], fc = hit[3 * qn + q];
                flags_or |= ff;
                if (l > 0) flags_or |= fc;
            }
        }
        // ---- the samples held for later rounds: what is left of the earlier entries after this round's
        // requests, followed by this round's new samples, laid out afresh in the other ahead buffer
        {
            std::vector<int> taken(MLMC_MAX_LEVELS, 0);
            for (size_t i = 0; i < req.size(); ++i) taken[req[i].level] = used[i];
            std::vector<int> fresh(MLMC_MAX_LEVELS, -1);   // work item of each level's new samples
            for (size_t w = 0; w < work.size(); ++w)
                if (work[w].req < 0) fresh[work[w].level] = (int)w;
            size_t rows = 0;
            for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
                if (ahead[l].valid) rows += (size_t)(ahead[l].count - taken[l]);
                if (fresh[l] >= 0) rows += (size_t)work[fresh[l]].count;
            }
            const int nb = 1 - ahead_buf;
            if (rows) MLMC_CUDA_RET(ctx->err, ctx->ws.ahead[nb].reserve(2 * rows * sizeof(double)));
            const double* src = ctx->ws.ahead[ahead_buf].as<double>();
            double* dst = ctx->ws.ahead[nb].as<double>();
            size_t ao = 0;
            auto rows_to = [&](const double* from, size_t c) -> cudaError_t {
                if (!c) return cudaSuccess;
                const cudaError_t e = cudaMemcpyAsync(dst + ao, from, c * sizeof(double), cudaMemcpyDeviceToDevice, st);
                ao += c;
                return e;
            };
            for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
                Ahead& a = ahead[l];
                size_t keep = a.valid ? (size_t)(a.count - taken[l]) : 0;
                const int w = fresh[l];
                const size_t add = w >= 0 ? (size_t)work[w].count : 0;
                // new samples extend held ones only at the same delta and class (else the held ones go)
                if (keep && add &&
                    !(a.df == df[l] && a.cls_f == class_of(l, l) &&
                      (l == 0 || (a.dc == dc[l] && a.cls_c == class_of(l - 1, l)))))
                    keep = 0;
                if (keep + add == 0) {
                    a.valid = false;
                    continue;
                }
                const size_t t = (size_t)taken[l];
                Ahead b;
                b.valid = true;
                b.first = keep ? a.first + (int64_t)t : work[w].first;   // new samples follow held ones
                b.count = (int)(keep + add);
                if (keep) {
                    b.df = a.df, b.dc = a.dc, b.cls_f = a.cls_f, b.cls_c = a.cls_c;
                } else {
                    b.df = df[l], b.dc = l > 0 ? dc[l] : 0.0, b.cls_f = class_of(l, l);
                    b.cls_c = l > 0 ? class_of(l - 1, l) : -1;
                }
                auto tail = [&](const auto& v) { return std::decay_t<decltype(v)>(v.begin() + t, v.end()); };
                b.it_f = keep ? tail(a.it_f) : std::vector<int32_t>();
                b.it_c = keep ? tail(a.it_c) : std::vector<int32_t>();
                b.fl_f = keep ? tail(a.fl_f) : std::vector<int32_t>();
                b.fl_c = keep ? tail(a.fl_c) : std::vector<int32_t>();
                b.abandoned = keep ? tail(a.abandoned) : std::vector<int64_t>();
                b.retried = keep ? tail(a.retried) : std::vector<int32_t>();
                b.qf = ao;
                if (keep) MLMC_CUDA_RET(ctx->err, rows_to(src + a.qf + t, keep));
                if (add) MLMC_CUDA_RET(ctx->err, rows_to(Qf + wq[w], add));
                b.qc = ao;
                if (keep) MLMC_CUDA_RET(ctx->err, rows_to(src + a.qc + t, keep));
                if (add) MLMC_CUDA_RET(ctx->err, rows_to(Qc + wq[w], add));
                if (add) {
                    const size_t q0 = wq[w];
                    auto append = [&](auto& v, const auto* from) { v.insert(v.end(), from + q0, from + q0 + add); };
                    append(b.it_f, hit.data());
                    append(b.it_c, hit.data() + qn);
                    append(b.fl_f, hit.data() + 2 * qn);
                    append(b.fl_c, hit.data() + 3 * qn);
                    append(b.abandoned, abandoned.data());
                    append(b.retried, retried.data());
                }
                a = std::move(b);
            }
            ahead_buf = nb;
        }
        return MLMC_OK;
    };
    if (o.resume) {
        // checkpoint: the counters and the calibrated rule's state continue from the earlier estimate
        const mlmc_result prev = *o.resume;
        for (int l = 0; l < MLMC_MAX_LEVELS && l <= prev.L; ++l) {
            prec_lvl[l] = prev.prec[l];
            iters_lvl[l] = prev.inner_iters[l];
            dofs_lvl[l] = prev.dofs[l];
            retries_lvl[l] = prev.fp64_retries[l];
            if (calibrate) {
                cal_contrast[l] = prev.contrast[l];
                if (prev.a_min[l] > 0) cal_amin[l] = prev.a_min[l];
                cal_amax[l] = prev.a_max[l];
            }
        }
        flags_or = prev.flags_or;
    }
    nvtxRangePushA("mlmc_estimate");
    const mlmc_status s = alg41(p.m, p.L_max, p.n0, o, round, res, ctx->err);
    nvtxRangePop();
    MLMC_CUDA_RET(ctx->err, ctx_order_end(ctx, st));
    if (s != MLMC_OK) return s;
    // the next estimate's samples to solve ahead
    if (!o.fixed_N)
        for (int l = 0; l < MLMC_MAX_LEVELS; ++l) ctx->ahead_hint[l] = l <= res->L ? res->N[l] : 0;
    for (int l = 0; l <= res->L; ++l) {
        res->prec[l] = prec_lvl[l];
        res->inner_iters[l] = iters_lvl[l];
        res->dofs[l] = dofs_lvl[l];
        res->fp64_retries[l] = retries_lvl[l];
        res->contrast[l] = calibrate ? cal_contrast[l] : 0.0;
        res->a_min[l] = calibrate && cal_amin[l] < 1e300 ? cal_amin[l] : 0.0;
        res->a_max[l] = calibrate ? cal_amax[l] : 0.0;
    }
    res->flags_or = flags_or;
    const int32_t bad = MLMC_F_MAXIT | MLMC_F_STAGNATED | MLMC_F_NONFINITE;
    if (flags_or & MLMC_F_NONFINITE) return fail(ctx, MLMC_E_NONFINITE, "estimate: a solve met a non-finite value");
    if (flags_or & bad) return fail(ctx, MLMC_E_NOCONV, "estimate: some solves stopped before their tolerance");
    return MLMC_OK;
}

mlmc_status mlmc_adjoint_grad(mlmc_ctx* ctx, int level, int S, const double* xi, mlmc_prec prec, double delta,
                              int max_iters, double* Q, double* dQdxi, void* stream) {
    if (!ctx) return MLMC_E_ARG;
    if (level < 0 || level > ctx->prob.L_max || S < 0 || !is_prec(prec) || !(delta > 0) || max_iters < 1)
        return fail(ctx, MLMC_E_ARG, "adjoint_grad: bad level, S, precision, delta or max_iters");
    if (S == 0) return MLMC_OK;
    if (!xi || !Q || !dQdxi) return fail(ctx, MLMC_E_ARG, "adjoint_grad: null pointer");
    cudaSetDevice(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MLMC_CUDA_RET(ctx->err, ctx_order_begin(ctx, st));
    const int n = level_n(ctx->prob, level);
    const size_t V = (size_t)(n + 1) * (n + 1);
    // the master coefficient is FP64: on the FP64 pipe for the FP64 solve, from the tensor cores
    // (exact lead slice, about 1e-9 in log a) for the mixed-precision solves
    const mlmc_prec fp = (prec == MLMC_FP64) ? MLMC_FP64 : MLMC_FP64TC;
    const size_t felem = sizeof(double);
    // layout: a [S][V] (field precision) | u [S][V] | lam [S][V] (FP64) | w [2][S][V] (float-float) |
    // the contraction's partial sums [splits][S][K] (FP64)
    const size_t abytes = (S * V * felem + 255) / 256 * 256;
    const int splits = kl_transpose_splits(S, ctx->prob.field.K, ctx->num_sms);
    const size_t pbytes = (size_t)splits * S * ctx->prob.field.K * sizeof(double);
    MLMC_CUDA_RET(ctx->err, ctx->ws.adj.reserve(abytes + 3 * S * V * sizeof(double) + pbytes));
    char* base = ctx->ws.adj.as<char>();
    void* a = base;
    double* u = reinterpret_cast<double*>(base + abytes);
    double* lam = u + S * V;
    float* wff = reinterpret_cast<float*>(lam + S * V);
    double* part = lam + 2 * S * V;
    mlmc_status s = synth(ctx, level, S, xi, a, 0, fp, st);
    if (s != MLMC_OK) return s;
    // ||g||_2 of the adjoint right-hand side
    double g2 = 0.0;
    for (int j = 1; j < n; ++j)
        for (int i = 1; i < n; ++i) {
            const double g = qoi_weight_node(ctx->prob, n, i, j);
            g2 += g * g;
        }
    const double gnorm = std::sqrt(g2);
    MLMC_CUDA_RET(ctx->err, ctx->ws.misc.reserve(sizeof(double) * S));
    SolveGroup gf;
    gf.n = n;
    gf.S = S;
    gf.a = a;
    gf.a_fp64 = 1;
    gf.a_n = n;
    gf.delta = delta;
    gf.Q = Q;
    gf.u = u;
    SolveGroup ga = gf;
    ga.Q = ctx->ws.misc.as<double>();
    ga.u = lam;
    ga.rhs_weights = &gnorm;
    SolveConfig cfg;
    cfg.prec = prec;
    cfg.max_iters = max_iters;
    s = launch_solve_async(ctx, {gf, ga}, cfg, st);
    if (s != MLMC_OK) return s;
    MLMC_CUDA_RET(ctx->err, launch_adjoint_elements(n, S, a, 1, u, lam, wff, st));
    MLMC_CUDA_RET(ctx->err, launch_kl_transpose_ff(ctx->basis.at(n), S, wff, part, splits, dQdxi, st));
    MLMC_CUDA_RET(ctx->err, ctx_order_end(ctx, st));
    return MLMC_OK;
}

}  // extern "C"
