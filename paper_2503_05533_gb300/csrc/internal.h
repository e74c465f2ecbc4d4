// Internal host-side declarations shared by the libmlmc translation units.
// Nothing here is part of the public ABI (include/libmlmc.h).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <utility>
#include <string>
#include <vector>

#include "../../include/libmlmc.h"

namespace mlmc {

// ---------------------------------------------------------------------------
// Error plumbing: every CUDA call goes through MLMC_CUDA, which records the
// failing call in the context and returns MLMC_E_CUDA.
extern std::atomic<int64_t> g_launches;      // kernels launched by this library
std::string& create_error();                  // last mlmc_create failure

struct Status {
    mlmc_status code = MLMC_OK;
    std::string msg;
};

#define MLMC_CUDA_RET(ctxerr, call)                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (ctxerr) = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return e_ == cudaErrorMemoryAllocation ? MLMC_E_NOMEM : MLMC_E_CUDA;           \
        }                                                                                  \
    } while (0)

// ---------------------------------------------------------------------------
// Device memory owned by a context.  Buffers grow on demand and are reused.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t want);
    void release();
    template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// KL basis of one level grid on the device.
struct GridBasis {
    int n = 0;
    int K = 0;
    int nodes = 0;         // (n+1)^2
    int nodes_pad = 0;     // nodes rounded up to the tensor-core tile (256)
    int Kpad = 0;          // K rounded up to 64 (16-bit K-major rows of 128 B)
    DevBuf phi64;          // FP64 [K][nodes_pad]
    DevBuf phi16;          // FP16 [2][nodes_pad][Kpad]: hi rows then lo rows, Phi = hi + lo 2^-11 (K-major)
    DevBuf phix;           // FP16 [3][nodes_pad][Kpad]: exact-lead slices of the FP64-output synthesis (lazy)
    DevBuf phiff;          // FP32 [2][K][nodes_pad]: Phi as float-float pairs (hi rows, then lo rows) for the
                           // transposed contraction of the gradient (lazy)
    DevBuf ev;             // int [nodes_pad]: their per-node power-of-two exponents
};

constexpr int kSolveSlots = 4;   // solve batches that may run concurrently (one per precision class)
constexpr int kTuneUnset = -3;   // a SolveConfig launch setting left to the context

// Group size class of a resident solve's system: 2 a warp, 1 a 128-thread group, 0 a 512-thread CTA
// (chunk items per thread stay around 8..32).  Systems with kMedItems < items <= kMedItemsWide take a
// 128-thread group or a CTA depending on the rest of their launch (the per-launch group choice).
constexpr int kMedItems = 2048, kMedItemsWide = 4096;
inline int size_class(int n, int med_items = kMedItems) {
    const long long items = (long long)(n - 1) * ((n - 1) / 4 + 1);
    if (items <= 512) return 2;        // warp
    if (items <= med_items) return 1;  // 128 threads
    return 0;                          // 512 threads
}

// The autotuner's choice for one launch shape (see solver_common.cu): SolveConfig launch settings
// (kTuneUnset / 0: the context's own) and the timings that chose them.
struct TuneChoice {
    int prec = 0, solver = 0, precond = 0;
    int med_items = kTuneUnset, ring = kTuneUnset, nu = 0;
    int mg_min = 0, mg_coarse = 0;   // coarsest grid bound and its sweeps (0: the context's)
    double mg_omega = 0.0;           // Jacobi damping of the smoother (0: the context's)
    int mg_smem = 0;                 // largest coarse grid kept in shared memory (0: 64)
    double theta = 0.0;
    double tau_min = -1.0;      // floor of the inner tolerance (< 0: the precision's default)
    float best_ms = 0.f, default_ms = 0.f;
    int trials = 0;
};

struct Workspace {
    DevBuf solver_slot[kSolveSlots];   // solver scratch (vectors, descriptors), one per concurrent batch
    // each slot's layout at its last launch (element sizes, array offsets, and per system its grid, row
    // pitch and offsets), and the allocation it was laid out in
    std::vector<long long> slot_layout[kSolveSlots];
    void* slot_ptr[kSolveSlots] = {};
    DevBuf fields;         // coefficient fields of the estimate loop
    DevBuf xi;             // KL coefficients of the estimate loop
    DevBuf q;              // QoI values of the estimate loop
    DevBuf misc;           // small per-call scratch (flags, iteration counts)
    DevBuf split;          // split FP16 operands of the tensor-core synthesis
    DevBuf adj;            // adjoint path scratch
    DevBuf chol;           // Cholesky solver: band factors, iterates, descriptors
    DevBuf ahead[2];       // estimate loop: QoIs of samples solved ahead of their round (Qf, Qc per level),
                           // the rows of one round and those of the next
};

// Profiling state of a context (mlmc_profile_*).
struct Profile {
    bool on = false;
    mlmc_profile acc{};
    struct Pending {
        cudaEvent_t a = nullptr, b = nullptr;
        double bytes = 0, flops = 0;
    };
    std::vector<Pending> kl_pending;
    // resident-solve launch intervals [start, end) in ms after the reference event t0 (recorded when
    // profiling is switched on or reset), for the union of busy time across concurrent streams
    cudaEvent_t t0 = nullptr;
    std::vector<std::pair<double, double>> solve_iv;
};

}  // namespace mlmc

struct mlmc_ctx {
    mlmc_problem prob{};
    int device = 0;
    int num_sms = 0;
    std::string err;
    std::map<int, mlmc::GridBasis> basis;   // keyed by n
    mlmc::Workspace ws;
    double wait_timeout_s = 10.0;
    unsigned* kl_err = nullptr;   // device error words, cleared when the host reads them:
    unsigned* solve_err = nullptr;    // [0] tensor-core synthesis, [1] resident solves (KERR_*)
    cudaEvent_t order_ev = nullptr;   // end of the context's last call: later calls on any stream wait for it
    bool order_recorded = false;
    int wait_extra = 0;           // diagnostic: bytes every tensor-core wait expects and never receives
    int solve_ring = -1;          // diagnostic: row-pipeline slots of large CG solves (-1 automatic, 0 off)
    int med_items = -1;           // diagnostic: most chunks of a system solved by a 128-thread group (-1 automatic)
    int precond = MLMC_PC_MG;     // preconditioner of the CG inner solves
    int chol_u = MLMC_FP64;       // Cholesky solves: working precision of x (mlmc_set_cholesky_precision)
    int chol_ur = MLMC_FP64;      // ... and precision of the refinement residual
    int mg_nu = 1;                // multigrid: smoothing sweeps before and after the coarse correction
    int mg_coarse = 8;            // multigrid: Jacobi sweeps on the coarsest grid
    int mg_min = 4;               // multigrid: grids are halved while the half keeps at least this many cells
    double mg_omega = 0.8;        // multigrid: Jacobi damping
    int mg_fmg = 1;               // multigrid CG: the first inner solve starts from a full-multigrid guess
    double inner_theta = 0.3;     // inner tolerance tau = clamp(theta delta / rho, tau_min, 0.5)
    double inner_tau_min = -1.0;  // < 0: per-precision default
    mlmc::Profile prof;
    cudaStream_t aux[mlmc::kSolveSlots - 1] = {};   // streams of concurrent solve batches (created on demand)
    bool autotune = false;        // time candidate launch settings for every new launch shape
    std::map<std::string, mlmc::TuneChoice> tune;   // launch shape -> chosen settings
    std::vector<std::string> tune_order;            // keys in the order they were tuned
    // estimate loop: solve samples ahead of the round that asks for them (mlmc_set_sample_ahead), up to
    // the sample counts the last estimate on this context ended with
    bool sample_ahead = true;
    int64_t ahead_hint[MLMC_MAX_LEVELS] = {};
};

namespace mlmc {

// ---------------------------------------------------------------------------
// KL basis tables (kl_basis.cpp, host).
struct Basis1D {
    std::vector<double> w, theta, norm;   // exp-cov 1D eigenpairs
};
// Separable tables: Phi[k][j (n+1) + i] = coef[k] bx[k][i] by[k][j].
bool build_separable(const mlmc_field& f, int n, std::vector<double>& coef, std::vector<double>& bx,
                     std::vector<double>& by, std::string& err);
// Exponential-covariance 1D eigenpairs (roots of the characteristic equation).
Basis1D expcov_1d(double corr_len, int count);
// The K leading (i, j) products, sorted; eigenvalues sigma2 theta_i theta_j.
void expcov_modes(double sigma2, double corr_len, int K, std::vector<int>& mi, std::vector<int>& mj,
                  std::vector<double>& lam, Basis1D& b1);

// ---------------------------------------------------------------------------
// Kernel launchers (each .cu file).
// philox.cu
cudaError_t launch_philox_normals(uint64_t seed, int level, uint64_t first, int S, int K, double* xi,
                                  cudaStream_t st);
// kl_synth.cu
cudaError_t upload_basis(GridBasis& gb, const mlmc_field& f, int n, std::string& err);
// Field syntheses write sample s's (n+1)^2 nodes at a + s ld.
cudaError_t launch_kl_fp64(const GridBasis& gb, int S, const double* xi, double* a, long long ld, cudaStream_t st);
// kl_tc.cu: tensor-core synthesis into FP32
cudaError_t launch_kl_fp32(mlmc_ctx* ctx, const GridBasis& gb, int S, const double* xi, float* a,
                           long long ld, cudaStream_t st);
// kl_tc.cu: tensor-core synthesis into FP64 (exact integer lead slice, float-float exp); builds the
// grid's exact-lead basis slices on first use
cudaError_t launch_kl_tc64(mlmc_ctx* ctx, GridBasis& gb, int S, const double* xi, double* a, long long ld,
                           cudaStream_t st);
// out[s][k] = sum_v Phi[k][v] w[s][v] with w given as float-float rows wff = [2][S][V] (hi, then lo), in
// float-float arithmetic on the FP32 pipe; part: splits * S * K doubles of scratch (splits from
// kl_transpose_splits)
int kl_transpose_splits(int S, int K, int num_sms);
cudaError_t launch_kl_transpose_ff(GridBasis& gb, int S, const float* wff, double* part, int splits, double* out,
                                   cudaStream_t st);
// stencil / solver (solver.cu)
struct SolveGroup {
    int n = 0;             // solve grid
    int S = 0;             // systems in the group
    const void* a = nullptr;   // master coefficient, dense nodal layout of grid a_n
    int a_fp64 = 1;        // master precision: 1 FP64, 0 FP32
    int a_n = 0;           // grid of `a` (multiple of n)
    long long a_ld = 0;    // elements from one system's coefficient to the next (0: (a_n+1)^2)
    double delta = 1e-8;   // relative residual target
    double* Q = nullptr;   // out [S]
    double* u = nullptr;   // optional out [S][(n+1)^2]
    int32_t* iters = nullptr;
    double* relres = nullptr;
    int32_t* flags = nullptr;
    const double* rhs_weights = nullptr;  // internal: adjoint right-hand side (g) instead of f
};
inline long long field_pitch(const SolveGroup& g) {
    return g.a_ld > 0 ? g.a_ld : (long long)(g.a_n + 1) * (g.a_n + 1);
}
struct SolveConfig {
    int prec = MLMC_FP64;  // mlmc_prec of the inner solve
    int solver = MLMC_CG;
    int max_iters = 20000;
    int max_outer = 12;
    double inner_theta = 0.3;   // inner tolerance = clamp(theta * delta / rho, tau_min, tau_max)
    double tau_min = -1.0;      // <0: per-precision default
    double tau_max = 0.5;
    int tile_nodes = 2048;      // target nodes per warp tile
    int jacobi = 1;             // Jacobi-preconditioned inner CG
    int precond = -1;           // MLMC_PC_*, or -1: the context's choice (mlmc_set_precond)
    // launch settings of the autotuner, overriding the context's (kTuneUnset / 0: the context's)
    int med_items = kTuneUnset;
    int ring = kTuneUnset;
    int nu = 0;
    int mg_min = 0;             // multigrid coarsening bound (0: the context's)
    int mg_coarse = 0;          // multigrid sweeps on the coarsest grid (0: the context's)
    double mg_omega = 0.0;      // multigrid smoother damping (0: the context's)
    int mg_smem = 0;            // largest coarse grid of the 512-thread groups in shared memory (0: 64)
    double theta = 0.0;
    // Cholesky solver (MLMC_CHOLESKY): working precision u of x and residual precision u_r of Alg. 2.1
    int chol_u = MLMC_FP64;
    int chol_ur = MLMC_FP64;
};
struct SolveStats {
    int64_t inner_iters = 0;    // summed over solves (host copy, only if requested)
};
// A launched batch whose completion the host has not yet checked, with what its profile needs.
struct PendingSolve {
    bool active = false;
    const int32_t* stats = nullptr;   // device int32 [2][ns]: inner iterations, refinement steps per system
    int ns = 0;
    int max_outer = 0;
    // algorithmic bytes of system i: it_i c_it[i] + (steps_i + 1) c_res[i] + steps_i c_upd[i] + c_set[i]
    // (filled only while profiling)
    std::vector<double> unk, c_it, c_res, c_upd, c_set;
    std::vector<double> f_it, f_res, f_upd, f_set;   // the same for arithmetic operations
    cudaEvent_t ev[2] = {nullptr, nullptr};
};
// solver_<precision>.cu (solver_impl.cuh): one inner precision's batch launcher (plan, upload and
// launch on st with workspace slot `slot`), stand-alone operator apply and allocation-free solve.
#define MLMC_DECLARE_SOLVER_PRECISION(P)                                                                       \
    mlmc_status solve_launch_##P(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg, \
                                 cudaStream_t st, int slot, PendingSolve& out);                                \
    cudaError_t apply_operator_##P(int n, int S, const void* a, int a_fp64, int a_n, const void* x, void* y,  \
                                   cudaStream_t st);                                                           \
    mlmc_status noalloc_solve_##P(int n, int S, const void* a, int a_fp64, int a_n, double delta, int max_iters, \
                                  int qoi, const double* box, double f, double* Q, int32_t* iters,             \
                                  double* relres, int32_t* flags, cudaStream_t st, void* scratch,              \
                                  std::string& err);
MLMC_DECLARE_SOLVER_PRECISION(fp64)
MLMC_DECLARE_SOLVER_PRECISION(fp32)
MLMC_DECLARE_SOLVER_PRECISION(bf16s)
MLMC_DECLARE_SOLVER_PRECISION(fp16s)
#undef MLMC_DECLARE_SOLVER_PRECISION

mlmc_status run_solve_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                            cudaStream_t st);
// cholesky.cu: the batch solved by the banded Cholesky factorisation in precision cfg.prec with
// iterative refinement (working precision cfg.chol_u, residual cfg.chol_ur).  With sync, waits for
// the launch and reads its profile and error words; without, enqueues it (no profile).
mlmc_status run_cholesky_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                               cudaStream_t st, bool sync);
// The same batch enqueued on st without waiting for it (errors surface at the context's next
// synchronising call); with profiling on it synchronises to read the launch's counters.
mlmc_status launch_solve_async(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                               cudaStream_t st);
// Independent batches (e.g. one per precision class) launched concurrently: the first on st,
// the others on the context's auxiliary streams after st's prior work; returns once all are
// done (st synchronised).  At most kSolveSlots batches.
struct SolveBatch {
    std::vector<SolveGroup> groups;
    SolveConfig cfg;
};
mlmc_status run_solve_batches(mlmc_ctx* ctx, const std::vector<SolveBatch>& batches, cudaStream_t st);
// The same launches, returning without waiting: st waits for every batch, and `pend` receives the launches'
// records, which the caller finishes (finish_solves) once it has synchronised st; the device error words
// are the caller's to read.  A single batch or Cholesky batches still run to completion.  On a failure
// every launched batch has been waited for and finished.
mlmc_status launch_solve_batches(mlmc_ctx* ctx, const std::vector<SolveBatch>& batches, cudaStream_t st,
                                 std::vector<PendingSolve>& pend);
mlmc_status finish_solves(mlmc_ctx* ctx, std::vector<PendingSolve>& pend);
cudaError_t launch_apply_operator(int n, int S, const void* a, int a_fp64, int a_n, int op_prec,
                                  const void* x, void* y, int vec_fp64, cudaStream_t st);
// stats.cu
cudaError_t launch_level_stats(int S, const double* Qf, const double* Qc, mlmc_acc* out_dev,
                               cudaStream_t st);
// min and max nodal coefficient of each of S fields of V nodes: out_dev [S][2]
cudaError_t launch_field_range(int S, int V, long long ld, const void* a, int a_fp64, double* out_dev,
                               cudaStream_t st);
// adjoint.cu
// w = a_v G_v as float-float rows [2][S][(n+1)^2] (hi rows, then lo rows)
cudaError_t launch_adjoint_elements(int n, int S, const void* a, int a_fp64, const double* u,
                                    const double* lam, float* wff, cudaStream_t st);

// The context's device error words (api.cpp): synchronises `st`, reads and clears
// them; MLMC_OK, or MLMC_E_TIMEOUT when a bounded wait of a synthesis or a solve ran out
// since they were last read.
mlmc_status check_device_errors(mlmc_ctx* ctx, cudaStream_t st);
// Device-side ordering of a context's calls: work that a call enqueues on `st` starts after
// the work of the context's previous call, whatever stream that call used (the calls share
// the context's workspaces).  begin() before a call's first enqueue, end() after its last.
cudaError_t ctx_order_begin(mlmc_ctx* ctx, cudaStream_t st);
cudaError_t ctx_order_end(mlmc_ctx* ctx, cudaStream_t st);

// host helpers (api.cpp)
void acc_merge(mlmc_acc* into, const mlmc_acc& other);
double qoi_weight_node(const mlmc_problem& p, int n, int i, int j);

}  // namespace mlmc
