// Internal host-side declarations shared by the libmlmc translation units.
// Nothing here is part of the public ABI (include/libmlmc.h).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
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
};

constexpr int kSolveSlots = 4;   // solve batches that may run concurrently (one per precision class)

struct Workspace {
    DevBuf solver_slot[kSolveSlots];   // solver scratch (vectors, descriptors), one per concurrent batch
    DevBuf fields;         // coefficient fields of the estimate loop
    DevBuf xi;             // KL coefficients of the estimate loop
    DevBuf q;              // QoI values of the estimate loop
    DevBuf misc;           // small per-call scratch (flags, iteration counts)
    DevBuf split;          // split FP16 operands of the tensor-core synthesis
    DevBuf adj;            // adjoint path scratch
    void* pinned = nullptr;    // pinned host staging
    size_t pinned_bytes = 0;
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
    unsigned* kl_err = nullptr;   // error word of the tensor-core synthesis (device, 4 bytes)
    int kl_err_pending = 0;       // a synthesis ran since the word was last read
    int wait_extra = 0;           // diagnostic: bytes every tensor-core wait expects and never receives
    int solve_ring = -1;          // diagnostic: row-pipeline slots of large CG solves (-1 automatic, 0 off)
    int med_items = -1;           // diagnostic: most chunks of a system solved by a 128-thread group (-1 automatic)
    int precond = MLMC_PC_MG;     // preconditioner of the CG inner solves
    int mg_nu = 1;                // multigrid: smoothing sweeps before and after the coarse correction
    int mg_coarse = 8;            // multigrid: Jacobi sweeps on the coarsest grid
    double mg_omega = 0.8;        // multigrid: Jacobi damping
    double inner_theta = 0.3;     // inner tolerance tau = clamp(theta delta / rho, tau_min, 0.5)
    double inner_tau_min = -1.0;  // < 0: per-precision default
    mlmc::Profile prof;
    cudaStream_t aux[mlmc::kSolveSlots - 1] = {};   // streams of concurrent solve batches (created on demand)
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
cudaError_t launch_kl_fp64(const GridBasis& gb, int S, const double* xi, double* a, cudaStream_t st);
// kl_tc.cu: tensor-core synthesis into FP32
cudaError_t launch_kl_fp32(mlmc_ctx* ctx, const GridBasis& gb, int S, const double* xi, float* a,
                           cudaStream_t st);
cudaError_t launch_kl_transpose_fp64(const GridBasis& gb, int S, const double* w, double* out,
                                     cudaStream_t st);
// stencil / solver (solver.cu)
struct SolveGroup {
    int n = 0;             // solve grid
    int S = 0;             // systems in the group
    const void* a = nullptr;   // master coefficient, dense nodal layout of grid a_n
    int a_fp64 = 1;        // master precision: 1 FP64, 0 FP32
    int a_n = 0;           // grid of `a` (multiple of n)
    double delta = 1e-8;   // relative residual target
    double* Q = nullptr;   // out [S]
    double* u = nullptr;   // optional out [S][(n+1)^2]
    int32_t* iters = nullptr;
    double* relres = nullptr;
    int32_t* flags = nullptr;
    const double* rhs_weights = nullptr;  // internal: adjoint right-hand side (g) instead of f
};
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
};
struct SolveStats {
    int64_t inner_iters = 0;    // summed over solves (host copy, only if requested)
};
mlmc_status run_solve_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                            cudaStream_t st);
// Independent batches (e.g. one per precision class) launched concurrently: the first on st,
// the others on the context's auxiliary streams after st's prior work; returns once all are
// done (st synchronised).  At most kSolveSlots batches.
struct SolveBatch {
    std::vector<SolveGroup> groups;
    SolveConfig cfg;
};
mlmc_status run_solve_batches(mlmc_ctx* ctx, const std::vector<SolveBatch>& batches, cudaStream_t st);
cudaError_t launch_apply_operator(int n, int S, const void* a, int a_fp64, int a_n, int op_prec,
                                  const void* x, void* y, int vec_fp64, cudaStream_t st);
// stats.cu
cudaError_t launch_level_stats(int S, const double* Qf, const double* Qc, mlmc_acc* out_dev,
                               cudaStream_t st);
// adjoint.cu
cudaError_t launch_adjoint_elements(int n, int S, const void* a, int a_fp64, const double* u,
                                    const double* lam, double* G, cudaStream_t st);

// Error word of the last tensor-core synthesis (kl_tc.cu): MLMC_OK, or MLMC_E_TIMEOUT
// when one of its bounded waits ran out; clears the word.  Synchronises.
mlmc_status check_kl_wait(mlmc_ctx* ctx);

// host helpers (api.cpp)
void acc_merge(mlmc_acc* into, const mlmc_acc& other);
double qoi_weight_node(const mlmc_problem& p, int n, int i, int j);

}  // namespace mlmc
