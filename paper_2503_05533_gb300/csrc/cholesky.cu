// The low-precision direct solver of Sec. 5.2: Alg. 2.1 (iterative refinement)
// with a banded Cholesky factorisation computed once in precision u_f and
// reused by every correction solve, batched with one CTA per system.
//
// Unknowns are the (n-1)^2 interior nodes in natural order (k = (j-1)(n-1) +
// (i-1)); the P1 operator of Sec. 3.1 couples k with k +- 1 and k +- (n-1), so
// A is banded with half-bandwidth bw = n - 1 and its Cholesky factor L fills
// the band.  The factor is stored by columns, band[k][t] = L(k+t, k) for
// t = 0..bw, in the storage type FT: FP8 E4M3 (4 exponent and 3 mantissa bits:
// the paper's quarter precision q43), IEEE half, bfloat16, single or double.
//
// Factorisation (right-looking, column by column): d = sqrt(A(k,k)), the column
// below the diagonal is divided by d, and the trailing (bw x bw) triangle is
// updated by the outer product of that column.  Only bw + 1 columns are ever
// active, so they live in a shared-memory ring in the arithmetic type CT (FP32
// for 16- and 32-bit factors, FP64 for the double factor): column k is written
// out rounded to FT when the next column starts, and its slot takes column
// k + bw + 1 of A (nonzero only at t = 0, 1 and bw).
//
// Refinement (Alg. 2.1): x = 0; loop: r = b - A x in the residual precision
// u_r (from the master coefficient, r = b while x = 0); stop when ||r|| / ||b||
// < delta; solve L L^T d = r with the stored factor (forward and backward
// substitution, column-oriented so that every step is one scalar division and
// one bw-long update); x += d in the working precision u.  The precisions
// (u_f = u_s, u, u_r) are the paper's quadruple of Sec. 5.2, e.g. (h, h, s, s).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {
namespace {

constexpr int kCholThreads = 128;   // >= bw + 1 for n <= 128

struct CholSystem {
    int n;
    long long band_off;      // element offset of this system's band [N][bw+1]
    long long vec_off;       // element offset of its vectors (x, r) [N]
    const void* a;           // master coefficient at node (0, 0)
    long long a_row;
    int a_col;
    int a_fp64;
    int qoi, bx0, bx1, by0, by1;
    double delta, bnorm, h2, f;
    double* Q;
    double* u;
    int32_t* iters;
    double* relres;
    int32_t* flags;
    int out, sys;
};

struct CholParams {
    const CholSystem* sys;
    void* band;              // FT
    void* x;                 // WT
    void* r;                 // CT: residual, then the correction
    int32_t* sys_steps;      // per system: refinement steps (residual evaluations)
    int max_steps;
    double stag;
};

// FP8 E4M3 storage (the paper's q43); a value beyond its range becomes NaN (no saturation), so that an
// overflowing factor is detected.
struct q43 {
    __nv_fp8_storage_t b;
};
template <class T> __device__ __forceinline__ T to_t(double v) { return (T)v; }
template <> __device__ __forceinline__ q43 to_t<q43>(double v) {
    return {__nv_cvt_float_to_fp8((float)v, __NV_NOSAT, __NV_E4M3)};
}
template <> __device__ __forceinline__ __half to_t<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_t<__nv_bfloat16>(double v) { return __double2bfloat16(v); }
template <class CT> __device__ __forceinline__ CT from_t(double v) { return (CT)v; }
template <class CT> __device__ __forceinline__ CT from_t(float v) { return (CT)v; }
template <class CT> __device__ __forceinline__ CT from_t(__half v) { return (CT)__half2float(v); }
template <class CT> __device__ __forceinline__ CT from_t(__nv_bfloat16 v) { return (CT)__bfloat162float(v); }
template <class CT> __device__ __forceinline__ CT from_t(q43 v) {
    return (CT)__half2float(__half(__nv_cvt_fp8_to_halfraw(v.b, __NV_E4M3)));
}
template <class T> __device__ __forceinline__ T round_to(float v);
template <> __device__ __forceinline__ float round_to<float>(float v) { return v; }
template <> __device__ __forceinline__ __half round_to<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 round_to<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ q43 round_to<q43>(float v) { return to_t<q43>((double)v); }
template <class T> __device__ __forceinline__ T round_to(double v) { return to_t<T>(v); }

__device__ __forceinline__ double chol_master(const CholSystem& S, int i, int j) {
    const long long idx = (long long)j * S.a_row + (long long)i * S.a_col;
    return S.a_fp64 ? static_cast<const double*>(S.a)[idx] : (double)static_cast<const float*>(S.a)[idx];
}

// Edge weights of the P1 operator (times 6) in type T: east edge (i,j)-(i+1,j), north edge (i,j)-(i,j+1).
template <class T>
__device__ __forceinline__ T weight_e(const CholSystem& S, int i, int j) {
    return (T)2 * ((T)chol_master(S, i, j) + (T)chol_master(S, i + 1, j)) + (T)chol_master(S, i + 1, j + 1) +
           (T)chol_master(S, i, j - 1);
}
template <class T>
__device__ __forceinline__ T weight_n(const CholSystem& S, int i, int j) {
    return (T)2 * ((T)chol_master(S, i, j) + (T)chol_master(S, i, j + 1)) + (T)chol_master(S, i + 1, j + 1) +
           (T)chol_master(S, i - 1, j);
}

// Column k of A in the band layout (t = 0 diagonal, t = 1 east neighbour, t = bw north neighbour).
template <class CT>
__device__ __forceinline__ CT a_band(const CholSystem& S, int k, int t) {
    const int m = S.n - 1;
    const int i = 1 + k % m, j = 1 + k / m;
    if (t == 0) {
        return (weight_e<CT>(S, i, j) + weight_e<CT>(S, i - 1, j) + weight_n<CT>(S, i, j) + weight_n<CT>(S, i, j - 1)) *
               (CT)(1.0 / 6.0);
    }
    if (t == 1 && i < m) return -weight_e<CT>(S, i, j) * (CT)(1.0 / 6.0);
    if (t == m && j < m) return -weight_n<CT>(S, i, j) * (CT)(1.0 / 6.0);
    return (CT)0;
}

__device__ __forceinline__ double chol_qoi_weight(const CholSystem& S, int i, int j) {
    if (S.qoi == 0) return S.h2;
    auto in = [&](int ci, int cj) -> int { return (ci >= S.bx0 && ci < S.bx1 && cj >= S.by0 && cj < S.by1) ? 1 : 0; };
    return S.h2 * (double)(2 * in(i, j) + in(i - 1, j) + 2 * in(i - 1, j - 1) + in(i, j - 1)) * (1.0 / 6.0);
}

// CTA-wide sum of one double per thread (fixed order), the same value in every thread.
__device__ __forceinline__ double cta_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < kCholThreads / 32; ++i) s += red[i];
    return s;
}

// FT factor storage, CT factor and substitution arithmetic, WT working precision (x), RT residual
// precision (computed in RC: FP64 for a double residual, FP32 otherwise).
template <class FT, class CT, class WT, class RT>
__global__ void __launch_bounds__(kCholThreads) chol_ir_kernel(CholParams P) {
    using RC = typename std::conditional<std::is_same<RT, double>::value, double, float>::type;
    extern __shared__ __align__(16) uint8_t chol_smem[];
    __shared__ double red[kCholThreads / 32];
    const CholSystem S = P.sys[blockIdx.x];
    const int t = threadIdx.x;
    const int m = S.n - 1, N = m * m, bw = m, R = bw + 1;
    FT* band = static_cast<FT*>(P.band) + S.band_off;
    WT* X = static_cast<WT*>(P.x) + S.vec_off;
    CT* rv = reinterpret_cast<CT*>(chol_smem);   // after the factorisation: the right-hand side / solution
    bool breakdown = false;

    // ---- factorisation: ring of R columns of CT in shared memory
    {
        CT* ring = reinterpret_cast<CT*>(chol_smem);
        for (int c = 0; c < R && c < N; ++c)
            if (t <= bw) ring[c * R + t] = a_band<CT>(S, c, t);
        __syncthreads();
        for (int k = 0; k < N; ++k) {
            CT* col = ring + (k % R) * R;
            // phase A: write out column k - 1 (its slot holds L(k-1+t, k-1), the diagonal already
            // rooted) and give the slot column k - 1 + R of A; every thread reads the pivot of column k
            if (k > 0 && t <= bw) {
                CT* prev = ring + ((k - 1) % R) * R;
                const FT v = round_to<FT>(prev[t]);
                if (!isfinite((double)from_t<CT>(v))) breakdown = true;   // beyond the storage format's range
                band[(long long)(k - 1) * R + t] = v;
                const int nk = k - 1 + R;
                prev[t] = nk < N ? a_band<CT>(S, nk, t) : (CT)0;
            }
            const CT piv = col[0];
            if (!(piv > (CT)0)) breakdown = true;
            const CT d = sqrt(piv);
            __syncthreads();   // slot k-1 reloaded; every thread has read col[0]
            if (t == 0) col[0] = d;
            else if (t <= bw) col[t] = col[t] / d;
            __syncthreads();
            // phase B: trailing update A(k+i, k+j) -= L(k+i, k) L(k+j, k), 1 <= j <= i <= bw; thread t
            // owns row i = t + 1 (each (j, i) entry has one writer)
            if (t < bw) {
                const int i = t + 1;
                if (k + i < N) {
                    const CT li = col[i];
                    for (int jj = 1; jj <= i; ++jj) {
                        CT* cj = ring + ((k + jj) % R) * R;
                        cj[i - jj] -= li * col[jj];
                    }
                }
            }
            __syncthreads();
        }
        if (t <= bw) {
            CT* last = ring + ((N - 1) % R) * R;
            const FT v = round_to<FT>(last[t]);
            if (!isfinite((double)from_t<CT>(v))) breakdown = true;
            band[(long long)(N - 1) * R + t] = v;
        }
        breakdown = __syncthreads_or(breakdown ? 1 : 0) != 0;
    }

    // ---- refinement (Alg. 2.1)
    for (int k = t; k < N; k += kCholThreads) X[k] = to_t<WT>(0.0);
    __syncthreads();
    double rho = 0.0, rho_prev = 0.0;
    int steps = 0, flag = 0;
    for (;; ++steps) {
        // r = b - A x in RT, stored rounded to CT (the correction solve's precision)
        double res = 0.0;
        for (int k = t; k < N; k += kCholThreads) {
            const int i = 1 + k % m, j = 1 + k / m;
            const RC b = (RC)(S.f * S.h2);
            RC rk = b;
            if (steps > 0) {
                const RC x0 = from_t<RC>(X[k]);
                const RC xe = i < m ? from_t<RC>(X[k + 1]) : (RC)0, xw = i > 1 ? from_t<RC>(X[k - 1]) : (RC)0;
                const RC xn = j < m ? from_t<RC>(X[k + m]) : (RC)0, xs = j > 1 ? from_t<RC>(X[k - m]) : (RC)0;
                const RC ax = (weight_e<RC>(S, i, j) * (x0 - xe) + weight_e<RC>(S, i - 1, j) * (x0 - xw) +
                               weight_n<RC>(S, i, j) * (x0 - xn) + weight_n<RC>(S, i, j - 1) * (x0 - xs)) *
                              (RC)(1.0 / 6.0);
                rk = b - ax;
            }
            // the residual in u_r (a half u_r stores it rounded to half)
            const double rq = from_t<double>(to_t<RT>((double)rk));
            rv[k] = (CT)rq;
            res += rq * rq;
        }
        res = cta_sum(res, red);   // (its barriers also publish rv)
        rho = sqrt(res) / S.bnorm;
        if (breakdown) { flag = MLMC_F_NONFINITE; break; }
        if (!(rho == rho) || isinf(rho)) { flag = MLMC_F_NONFINITE; break; }
        if (rho < S.delta) { flag = MLMC_F_CONVERGED; break; }
        if (steps >= P.max_steps) { flag = MLMC_F_MAXIT; break; }
        if (steps >= 1 && rho > P.stag * rho_prev) { flag = MLMC_F_STAGNATED; break; }
        rho_prev = rho;
        // forward substitution L y = r (column-oriented): y_k = r_k / L_kk, r_{k+i} -= L_{k+i,k} y_k
        for (int k = 0; k < N; ++k) {
            const CT yk = rv[k] / from_t<CT>(band[(long long)k * R]);
            if (t >= 1 && t <= bw && k + t < N) rv[k + t] -= from_t<CT>(band[(long long)k * R + t]) * yk;
            __syncthreads();
            if (t == 0) rv[k] = yk;
            __syncthreads();
        }
        // backward substitution L^T d = y: d_k = y_k / L_kk, y_{k-i} -= L_{k,k-i} d_k
        for (int k = N - 1; k >= 0; --k) {
            const CT dk = rv[k] / from_t<CT>(band[(long long)k * R]);
            if (t >= 1 && t <= bw && k - t >= 0) rv[k - t] -= from_t<CT>(band[(long long)(k - t) * R + t]) * dk;
            __syncthreads();
            if (t == 0) rv[k] = dk;
            __syncthreads();
        }
        for (int k = t; k < N; k += kCholThreads) X[k] = to_t<WT>(from_t<double>(X[k]) + (double)rv[k]);
        __syncthreads();
    }

    // ---- QoI and outputs
    double q = 0.0;
    for (int k = t; k < N; k += kCholThreads) {
        const int i = 1 + k % m, j = 1 + k / m;
        q += chol_qoi_weight(S, i, j) * from_t<double>(X[k]);
    }
    q = cta_sum(q, red);
    if (S.u) {
        double* u = S.u + (size_t)S.out * (S.n + 1) * (S.n + 1);
        for (int v = t; v < (S.n + 1) * (S.n + 1); v += kCholThreads) {
            const int i = v % (S.n + 1), j = v / (S.n + 1);
            u[v] = (i >= 1 && i <= m && j >= 1 && j <= m) ? from_t<double>(X[(j - 1) * m + (i - 1)]) : 0.0;
        }
    }
    if (t == 0) {
        if (S.Q) S.Q[S.out] = q;
        if (S.iters) S.iters[S.out] = steps;
        if (S.relres) S.relres[S.out] = rho;
        if (S.flags) S.flags[S.out] = flag;
        P.sys_steps[S.sys] = steps;
    }
}

size_t chol_align(size_t v) { return (v + 255) / 256 * 256; }

template <class FT, class CT, class WT, class RT>
mlmc_status chol_launch_typed(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                              cudaStream_t st, std::vector<int>& ns, int32_t** steps_dev) {
    std::vector<CholSystem> sys;
    long long bandn = 0, vecn = 0;
    const mlmc_problem& pb = ctx->prob;
    int nmax = 0;
    for (const SolveGroup& g : groups) {
        if (g.S <= 0) continue;
        const int n = g.n, m = n - 1;
        const int stride = g.a_n / n;
        const size_t elem = g.a_fp64 ? sizeof(double) : sizeof(float);
        const long long aV = field_pitch(g);
        const double h = 1.0 / n;
        int bx0 = 0, bx1 = n, by0 = 0, by1 = n;
        if (pb.qoi == 1) {
            bx0 = (int)std::lround(pb.box[0] * n);
            bx1 = (int)std::lround(pb.box[1] * n);
            by0 = (int)std::lround(pb.box[2] * n);
            by1 = (int)std::lround(pb.box[3] * n);
        }
        for (int s = 0; s < g.S; ++s) {
            CholSystem d{};
            d.n = n;
            d.band_off = bandn;
            bandn += (long long)m * m * n;   // N (bw + 1)
            d.vec_off = vecn;
            vecn += (long long)m * m;
            d.a = static_cast<const char*>(g.a) + (size_t)s * aV * elem;
            d.a_row = (long long)stride * (g.a_n + 1);
            d.a_col = stride;
            d.a_fp64 = g.a_fp64;
            d.qoi = pb.qoi;
            d.bx0 = bx0; d.bx1 = bx1; d.by0 = by0; d.by1 = by1;
            d.delta = g.delta;
            d.h2 = h * h;
            d.f = pb.f;
            d.bnorm = std::fabs(pb.f) * h * h * (double)m;
            d.Q = g.Q;
            d.u = g.u;
            d.iters = g.iters;
            d.relres = g.relres;
            d.flags = g.flags;
            d.out = s;
            d.sys = (int)sys.size();
            sys.push_back(d);
            ns.push_back(n);
            nmax = std::max(nmax, n);
        }
    }
    const int nsys = (int)sys.size();
    if (nsys == 0) return MLMC_OK;
    // workspace: band (FT) | x (WT) | r unused in global | descriptors | steps
    const size_t o_band = 0;
    const size_t o_x = chol_align(o_band + (size_t)bandn * sizeof(FT));
    const size_t o_sys = chol_align(o_x + (size_t)vecn * sizeof(WT));
    const size_t o_steps = chol_align(o_sys + sizeof(CholSystem) * nsys);
    const size_t total = chol_align(o_steps + sizeof(int32_t) * nsys);
    MLMC_CUDA_RET(ctx->err, ctx->ws.chol.reserve(total));
    char* base = ctx->ws.chol.as<char>();
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(base + o_sys, sys.data(), sizeof(CholSystem) * nsys, cudaMemcpyHostToDevice, st));
    CholParams P;
    P.sys = reinterpret_cast<const CholSystem*>(base + o_sys);
    P.band = base + o_band;
    P.x = base + o_x;
    P.r = nullptr;
    P.sys_steps = reinterpret_cast<int32_t*>(base + o_steps);
    P.max_steps = cfg.max_outer;
    P.stag = 0.5;
    const int m = nmax - 1;
    // shared memory: the factor ring (R x R of CT) and, afterwards, one vector of N entries of CT
    const size_t smem = std::max((size_t)(m + 1) * (m + 1), (size_t)m * m) * sizeof(CT);
    if (smem > 227 * 1024) {
        ctx->err = "cholesky: a system of this size needs more shared memory than a CTA has";
        return MLMC_E_UNSUPPORTED;
    }
    MLMC_CUDA_RET(ctx->err, cudaFuncSetAttribute(chol_ir_kernel<FT, CT, WT, RT>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    chol_ir_kernel<FT, CT, WT, RT><<<nsys, kCholThreads, smem, st>>>(P);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    MLMC_CUDA_RET(ctx->err, cudaGetLastError());
    ctx->prof.acc.h2d_bytes += (int64_t)(sizeof(CholSystem) * nsys);
    *steps_dev = P.sys_steps;
    return MLMC_OK;
}

template <class FT, class CT>
mlmc_status chol_dispatch_w(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                            cudaStream_t st, std::vector<int>& ns, int32_t** steps) {
    // (u, u_r): (d, d), (s, d), (s, s), (h, h)
    if (cfg.chol_u == MLMC_FP64) return chol_launch_typed<FT, CT, double, double>(ctx, groups, cfg, st, ns, steps);
    if (cfg.chol_u == MLMC_FP16S) return chol_launch_typed<FT, CT, __half, __half>(ctx, groups, cfg, st, ns, steps);
    return cfg.chol_ur == MLMC_FP64 ? chol_launch_typed<FT, CT, float, double>(ctx, groups, cfg, st, ns, steps)
                                    : chol_launch_typed<FT, CT, float, float>(ctx, groups, cfg, st, ns, steps);
}

double prec_bits(int p) {
    switch (p) {
        case MLMC_FP64: return 64.0;
        case MLMC_FP32: return 32.0;
        case MLMC_FP8S: return 8.0;
        default: return 16.0;
    }
}

}  // namespace

mlmc_status run_cholesky_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                               cudaStream_t st, bool sync) {
    sync = sync || ctx->prof.on;   // the profile needs the launch's step counts
    for (const SolveGroup& g : groups)
        if (g.S > 0 && (g.n < 2 || g.n > 128)) {
            ctx->err = "cholesky: grids of 2 to 128 cells per side (half-bandwidth n - 1 <= 127)";
            return MLMC_E_UNSUPPORTED;
        }
    std::vector<int> ns;
    int32_t* steps_dev = nullptr;
    mlmc_status s;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (ctx->prof.on) {
        MLMC_CUDA_RET(ctx->err, cudaEventCreate(&ev[0]));
        MLMC_CUDA_RET(ctx->err, cudaEventCreate(&ev[1]));
        MLMC_CUDA_RET(ctx->err, cudaEventRecord(ev[0], st));
    }
    switch (cfg.prec) {
        case MLMC_FP64: s = chol_dispatch_w<double, double>(ctx, groups, cfg, st, ns, &steps_dev); break;
        case MLMC_FP32: s = chol_dispatch_w<float, float>(ctx, groups, cfg, st, ns, &steps_dev); break;
        case MLMC_BF16S: s = chol_dispatch_w<__nv_bfloat16, float>(ctx, groups, cfg, st, ns, &steps_dev); break;
        case MLMC_FP16S: s = chol_dispatch_w<__half, float>(ctx, groups, cfg, st, ns, &steps_dev); break;
        case MLMC_FP8S: s = chol_dispatch_w<q43, float>(ctx, groups, cfg, st, ns, &steps_dev); break;
        default: ctx->err = "cholesky: bad factor precision"; s = MLMC_E_ARG;
    }
    if (s != MLMC_OK) return s;
    if (ev[0]) MLMC_CUDA_RET(ctx->err, cudaEventRecord(ev[1], st));
    if (!sync) return MLMC_OK;
    MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
    if (ev[0]) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        std::vector<int32_t> steps(ns.size());
        if (!ns.empty())
            MLMC_CUDA_RET(ctx->err, cudaMemcpy(steps.data(), steps_dev, sizeof(int32_t) * ns.size(),
                                               cudaMemcpyDeviceToHost));
        // the cost model of Sec. 5.2: bits of every factor entry and vector entry computed and stored --
        // the factor's nonzeros in u_f, x_0 in u, each residual in u_r, each correction and update in u
        const double bf = prec_bits(cfg.prec), bu = prec_bits(cfg.chol_u), br = prec_bits(cfg.chol_ur);
        double bits = 0.0;
        for (size_t i = 0; i < ns.size(); ++i) {
            const double m = ns[i] - 1, N = m * m;
            const double nnz = N * (m + 1) - m * (m + 1) / 2;
            const double it = steps[i];
            bits += nnz * bf + N * bu + (it + 1) * N * br + it * 2.0 * N * bu;
        }
        mlmc_profile& A = ctx->prof.acc;
        A.solve_launches += 1;
        A.solve_ms += ms;
        A.chol_bits += bits;
    }
    return check_device_errors(ctx, st);
}

}  // namespace mlmc
