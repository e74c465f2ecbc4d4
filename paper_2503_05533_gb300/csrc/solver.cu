// A3-A7: matrix-free P1 operator, batched inner Krylov solve, FP64 iterative
// refinement and the QoI, for many independent systems in one persistent
// cooperative kernel.
//
// Operator (Sec. 3.1, P1 elements on the uniform grid with SW-NE diagonals,
// a_T = mean of the vertex values).  Right-angled P1 triangles couple only
// along their legs, so A is 5-point with edge weights
//   wE(i,j) = (a_T1(i,j) + a_T2(i,j-1)) / 2 = (2a(i,j) + 2a(i+1,j) + a(i+1,j+1) + a(i,j-1)) / 6
//   wN(i,j) = (a_T2(i,j) + a_T1(i-1,j)) / 2 = (2a(i,j) + 2a(i,j+1) + a(i+1,j+1) + a(i-1,j)) / 6
//   (A x)_ij = sum over the 4 edges of w (x_ij - x_nbr),  x = 0 on the boundary,
// and b_i = f h^2 (six triangles of area h^2/2, one third each).
//
// Solve (Alg. 2.1 with the factorisation replaced by a Krylov method):
//   x = 0; loop: r = b - A x (FP64, master coefficient); stop if ||r||/||b|| < delta
//   (Eq. (2.1), C = 1); else solve A d = r with CG (Sec. 2.2) in the inner
//   precision to relative residual tau = clamp(theta delta / rho, tau_min, tau_max);
//   x += d (FP64).
// QoI (Problem 4.5): Q = sum_i g_i x_i, g_i = int_B phi_i (B = D: g_i = h^2).
//
// Execution: all systems of a batch share one cooperative launch.  A system's
// interior rows are cut into row tiles; CTAs take tiles grid-stride.  Phases
// are separated by a bounded grid barrier.  Each tile writes one partial sum
// per reduction; every CTA that needs a system's scalar (alpha, beta, rho,
// stop decisions) sums the same partials in the same order, so all CTAs agree
// bit for bit without an extra barrier.  Per-system state that must outlive a
// phase is written by the CTA owning the system's first tile only.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {

namespace {

constexpr int BLOCK = 256;

struct DevSolve {
    int n, ld;
    long long off;           // node offset of this system's workspace grid
    const void* a;           // master coefficient at node (0,0)
    long long a_row;         // element stride between rows of `a`
    int a_col;               // element stride between columns of `a`
    int a_fp64;              // master precision (1: FP64, 0: FP32)
    int tile0, ntiles;
    int cpr;                 // 4-node chunks per row
    int rhs_mode;            // 0: b_i = f h^2 ; 1: b_i = g_i (adjoint right-hand side)
    int qoi;                 // 0: int_D ; 1: int_B
    int bx0, bx1, by0, by1;  // QoI box as cell index bounds
    double delta, bnorm, h2, f;
    double* Q;
    double* u;
    int32_t* iters;
    double* relres;
    int32_t* flags;
    int out;                 // index into the output arrays
};

struct DevTile {
    int solve, j0, j1;
};

struct Params {
    unsigned nbar;       // CTAs a grid barrier waits for (the grid, plus a diagnostic surplus)
    const DevSolve* solves;
    const DevTile* tiles;
    int nsolves, ntiles;
    double* x64;
    void* r;
    void* p0;
    void* p1;
    void* d;
    void* as;
    double* part_res;
    double* part_rr0;
    double* part_rr;     // [2][ntiles]
    double* part_sig;
    double* part_q;
    int* conv_outer;     // outer index at which the system stopped (INT_MAX: running)
    int* inner_tag;      // o + 1 once the inner solve of outer step o finished
    int* iters_acc;      // inner iterations so far
    double* rho_hist;    // [2][nsolves]
    double* rho_final;
    int* flags_acc;
    int* active_count;   // [max_outer + 1]
    int* done_count;     // [max_outer + 1]
    unsigned* bar;
    unsigned* err;
    int max_outer, max_iters;
    double theta, tau_min, tau_max, stag;
    unsigned long long timeout_ns;
};

// ---------------------------------------------------------------------------
// The 5-point P1 stencil at one node from its coefficient neighbourhood.
//   a: a(i-1..i+1, j-1..j+1) as a[dy][dx] (dy, dx in 0..2, centre a[1][1]),
//   x: centre, E, W, N, S values.
template <class CT>
__device__ __forceinline__ CT stencil_point(CT a00, CT aE, CT aW, CT aN, CT aS, CT aNE, CT aSW, CT x0, CT xE,
                                            CT xW, CT xN, CT xS) {
    const CT two = (CT)2;
    const CT wE = two * (a00 + aE) + aNE + aS;
    const CT wW = two * (aW + a00) + aN + aSW;
    const CT wN = two * (a00 + aN) + aNE + aW;
    const CT wS = two * (aS + a00) + aE + aSW;
    const CT y = wE * (x0 - xE) + wW * (x0 - xW) + wN * (x0 - xN) + wS * (x0 - xS);
    return y * (CT)(1.0 / 6.0);
}

// Coefficient neighbourhood of a 4-node chunk (columns 4c-1 .. 4c+4 of rows j-1, j, j+1).
template <class ST, class CT>
__device__ __forceinline__ void load_coef_chunk(const ST* as, int ld, int n, int j, int c, CT a[3][6]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const ST* row = as + (size_t)(j - 1 + r) * ld;
        CoefLoad<ST, CT>::load4(row + 4 * c, &a[r][1]);
        a[r][0] = (c > 0) ? CoefLoad<ST, CT>::load1(row + 4 * c - 1) : (CT)0;
        a[r][5] = (4 * c + 4 <= n) ? CoefLoad<ST, CT>::load1(row + 4 * c + 4) : (CT)0;
    }
}

// Vector neighbourhood of a chunk: south row (4), centre row with one halo each
// side (6), north row (4).
template <class VT>
__device__ __forceinline__ void load_vec_chunk(const VT* v, int ld, int n, int j, int c, VT s[4], VT cc[6],
                                               VT nn[4]) {
    const VT* row = v + (size_t)j * ld;
    Vec4<VT>::load(row - ld + 4 * c, s);
    Vec4<VT>::load(row + 4 * c, &cc[1]);
    Vec4<VT>::load(row + ld + 4 * c, nn);
    cc[0] = (c > 0) ? __ldcg(row + 4 * c - 1) : (VT)0;
    cc[5] = (4 * c + 4 <= n) ? __ldcg(row + 4 * c + 4) : (VT)0;
}

template <class CT>
__device__ __forceinline__ void apply_chunk(const CT a[3][6], const CT s[4], const CT cc[6], const CT nn[4],
                                            int n, int c, CT y[4]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int ii = t + 1;
        const int i = 4 * c + t;
        const CT v = stencil_point<CT>(a[1][ii], a[1][ii + 1], a[1][ii - 1], a[2][ii], a[0][ii], a[2][ii + 1],
                                       a[0][ii - 1], cc[ii], cc[ii + 1], cc[ii - 1], nn[t], s[t]);
        y[t] = (i >= 1 && i <= n - 1) ? v : (CT)0;
    }
}

__device__ __forceinline__ double master_a(const DevSolve& S, int i, int j) {
    const long long idx = (long long)j * S.a_row + (long long)i * S.a_col;
    return S.a_fp64 ? __ldg(static_cast<const double*>(S.a) + idx)
                    : (double)__ldg(static_cast<const float*>(S.a) + idx);
}

__device__ __forceinline__ double qoi_weight(const DevSolve& S, int i, int j) {
    if (S.qoi == 0) return S.h2;
    auto in = [&](int ci, int cj) -> int {
        return (ci >= S.bx0 && ci < S.bx1 && cj >= S.by0 && cj < S.by1) ? 1 : 0;
    };
    const int cnt = 2 * in(i, j) + in(i - 1, j) + 2 * in(i - 1, j - 1) + in(i, j - 1);
    return S.h2 * (double)cnt * (1.0 / 6.0);
}

__device__ __forceinline__ double rhs_value(const DevSolve& S, int i, int j) {
    return S.rhs_mode == 0 ? S.f * S.h2 : qoi_weight(S, i, j);
}

// Inner tolerance for the current refinement step.
__device__ __forceinline__ double inner_tau(const Params& P, const DevSolve& S, double rho) {
    double t = P.theta * S.delta / rho;
    t = fmin(fmax(t, P.tau_min), P.tau_max);
    return t;
}

// Stop decision of outer step o from the residual partials (identical in every CTA).
// Returns 0 to continue, else the MLMC_F_* reason.
__device__ __forceinline__ int stop_reason(const Params& P, const DevSolve& S, int s, int o, double rho) {
    if (!(rho == rho) || isinf(rho)) return MLMC_F_NONFINITE;
    if (rho < S.delta) return MLMC_F_CONVERGED;
    if (o >= P.max_outer) return MLMC_F_MAXIT;
    if (__ldcg(P.iters_acc + s) >= P.max_iters) return MLMC_F_MAXIT;
    if (o >= 1) {
        const double prev = __ldcg(P.rho_hist + (size_t)((o - 1) & 1) * P.nsolves + s);
        if (rho > P.stag * prev) return MLMC_F_STAGNATED;
    }
    return 0;
}

__device__ __forceinline__ double solve_rho(const Params& P, const DevSolve& S) {
    const double rr = warp_sum_partials(P.part_res, S.tile0, S.ntiles);
    return sqrt(rr) / S.bnorm;
}

// ---------------------------------------------------------------------------
// Per-tile decision of one phase, made by warp 0 and broadcast to the block so
// that every thread takes the same branch (other CTAs may update a system's
// words concurrently; reading them once keeps the block uniform).
struct TileDecision {
    int go;
    double s0, s1;
};

template <class VT, class ST>
__global__ void __launch_bounds__(BLOCK) persistent_solve(Params P) {
    __shared__ double red[2 * BLOCK / 32];
    __shared__ TileDecision sh;
    const unsigned nb = gridDim.x;
    const int lane = threadIdx.x & 31;
    const bool w0 = threadIdx.x < 32;
    double* x64 = P.x64;
    VT* r = static_cast<VT*>(P.r);
    VT* pb[2] = {static_cast<VT*>(P.p0), static_cast<VT*>(P.p1)};
    VT* d = static_cast<VT*>(P.d);
    ST* as = static_cast<ST*>(P.as);

    // ---- setup: coefficient in the inner storage precision (all rows 0..n)
    for (int t = blockIdx.x; t < P.ntiles; t += nb) {
        const DevTile T = P.tiles[t];
        const DevSolve& S = P.solves[T.solve];
        const int jlo = (T.j0 == 1) ? 0 : T.j0;
        const int jhi = (T.j1 == S.n) ? S.n + 1 : T.j1;
        const int width = S.n + 1;
        for (int it = threadIdx.x; it < (jhi - jlo) * width; it += BLOCK) {
            const int j = jlo + it / width, i = it % width;
            as[S.off + (size_t)j * S.ld + i] = to_store<ST>(master_a(S, i, j));
        }
    }
    if (!grid_barrier(P.bar, P.nbar, P.err, P.timeout_ns)) return;

    for (int o = 0; o <= P.max_outer; ++o) {
        // ---- R: r = b - A x in FP64 with the master coefficient; d = 0
        for (int t = blockIdx.x; t < P.ntiles; t += nb) {
            const DevTile T = P.tiles[t];
            const DevSolve& S = P.solves[T.solve];
            __syncthreads();
            if (threadIdx.x == 0) sh.go = (__ldcg(P.conv_outer + T.solve) >= o);
            __syncthreads();
            if (!sh.go) continue;
            double acc64 = 0.0, accv = 0.0;
            const int items = (T.j1 - T.j0) * S.cpr;
            for (int it = threadIdx.x; it < items; it += BLOCK) {
                const int j = T.j0 + it / S.cpr, c = it % S.cpr;
                double xs[4], xc[6], xn[4];
                load_vec_chunk<double>(x64 + S.off, S.ld, S.n, j, c, xs, xc, xn);
                VT rv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 4 * c + q;
                    double rq = 0.0;
                    if (i >= 1 && i <= S.n - 1) {
                        const double a00 = master_a(S, i, j), aE = master_a(S, i + 1, j), aW = master_a(S, i - 1, j);
                        const double aN = master_a(S, i, j + 1), aS = master_a(S, i, j - 1);
                        const double aNE = master_a(S, i + 1, j + 1), aSW = master_a(S, i - 1, j - 1);
                        const double ax = stencil_point<double>(a00, aE, aW, aN, aS, aNE, aSW, xc[q + 1], xc[q + 2],
                                                                xc[q], xn[q], xs[q]);
                        rq = rhs_value(S, i, j) - ax;
                    }
                    rv[q] = (VT)rq;
                    acc64 += rq * rq;
                    accv += (double)rv[q] * (double)rv[q];
                }
                const size_t base = S.off + (size_t)j * S.ld + 4 * c;
                Vec4<VT>::store(r + base, rv);
                const VT z[4] = {(VT)0, (VT)0, (VT)0, (VT)0};
                Vec4<VT>::store(d + base, z);
            }
            const double2 tot = block_sum2<BLOCK>(acc64, accv, red);
            if (threadIdx.x == 0) {
                P.part_res[t] = tot.x;
                P.part_rr0[t] = tot.y;
                P.part_rr[t] = tot.y;   // rho_0 of the inner solve, parity 0
            }
        }
        if (!grid_barrier(P.bar, P.nbar, P.err, P.timeout_ns)) return;

        // ---- decide: the CTA owning a system's first tile records the outcome
        if (w0) {
            for (int t = blockIdx.x; t < P.ntiles; t += nb) {
                const DevTile T = P.tiles[t];
                const DevSolve& S = P.solves[T.solve];
                if (t != S.tile0 || __ldcg(P.conv_outer + T.solve) < o) continue;
                const double rho = solve_rho(P, S);
                const int why = stop_reason(P, S, T.solve, o, rho);
                if (lane == 0) {
                    P.rho_hist[(size_t)(o & 1) * P.nsolves + T.solve] = rho;
                    P.rho_final[T.solve] = rho;
                    if (why) {
                        P.conv_outer[T.solve] = o;
                        P.flags_acc[T.solve] = why;
                    } else {
                        atomicAdd(P.active_count + o, 1);
                    }
                }
            }
        }
        if (o == P.max_outer) break;

        // ---- inner CG on A d = r
        for (int k = 0;; ++k) {
            const int cur = k & 1;
            // I1: beta, p = r + beta p_old, sigma = (p, A p)
            for (int t = blockIdx.x; t < P.ntiles; t += nb) {
                const DevTile T = P.tiles[t];
                const DevSolve& S = P.solves[T.solve];
                const int s = T.solve;
                __syncthreads();
                if (w0) {
                    int go = 1;
                    double beta = 0.0;
                    const int co = __ldcg(P.conv_outer + s);
                    if (co <= o || __ldcg(P.inner_tag + s) == o + 1) {
                        go = 0;
                    } else {
                        const double rho = solve_rho(P, S);
                        if (k == 0 && stop_reason(P, S, s, o, rho)) {
                            go = 0;
                        } else {
                            const double rrk =
                                warp_sum_partials(P.part_rr + (size_t)cur * P.ntiles, S.tile0, S.ntiles);
                            const double rr0 = warp_sum_partials(P.part_rr0, S.tile0, S.ntiles);
                            const double tau = inner_tau(P, S, rho);
                            const int budget = P.max_iters - __ldcg(P.iters_acc + s);
                            const bool finite = (rrk == rrk) && !isinf(rrk);
                            const bool done = !finite || rrk <= tau * tau * rr0 || rrk == 0.0 || k >= budget;
                            if (done) {
                                go = 0;
                                if (t == S.tile0 && lane == 0) {
                                    P.inner_tag[s] = o + 1;
                                    P.iters_acc[s] += k;
                                    atomicAdd(P.done_count + o, 1);
                                }
                            } else if (k > 0) {
                                const double rrp = warp_sum_partials(P.part_rr + (size_t)(cur ^ 1) * P.ntiles,
                                                                     S.tile0, S.ntiles);
                                beta = rrk / rrp;
                            }
                        }
                    }
                    if (lane == 0) {
                        sh.go = go;
                        sh.s0 = beta;
                    }
                }
                __syncthreads();
                if (!sh.go) continue;
                const VT vb = (VT)sh.s0;
                const VT* pold = pb[cur ^ 1] + S.off;
                VT* pnew = pb[cur] + S.off;
                const VT* rr = r + S.off;
                VT acc = 0;
                const int items = (T.j1 - T.j0) * S.cpr;
                for (int it = threadIdx.x; it < items; it += BLOCK) {
                    const int j = T.j0 + it / S.cpr, c = it % S.cpr;
                    VT rs[4], rc[6], rn[4];
                    load_vec_chunk<VT>(rr, S.ld, S.n, j, c, rs, rc, rn);
                    if (k > 0) {
                        VT ps[4], pc[6], pn[4];
                        load_vec_chunk<VT>(pold, S.ld, S.n, j, c, ps, pc, pn);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            rs[q] = rs[q] + vb * ps[q];
                            rn[q] = rn[q] + vb * pn[q];
                        }
#pragma unroll
                        for (int q = 0; q < 6; ++q) rc[q] = rc[q] + vb * pc[q];
                    }
                    VT a[3][6];
                    load_coef_chunk<ST, VT>(as + S.off, S.ld, S.n, j, c, a);
                    VT y[4];
                    apply_chunk<VT>(a, rs, rc, rn, S.n, c, y);
                    Vec4<VT>::store(pnew + (size_t)j * S.ld + 4 * c, &rc[1]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc += rc[q + 1] * y[q];
                }
                const double tot = block_sum<BLOCK>((double)acc, red);
                if (threadIdx.x == 0) P.part_sig[t] = tot;
            }
            if (!grid_barrier(P.bar, P.nbar, P.err, P.timeout_ns)) return;
            if (__ldcg(P.done_count + o) >= __ldcg(P.active_count + o)) break;

            // I2: alpha = rr / sigma; d += alpha p; r -= alpha A p; rr_new = (r, r)
            for (int t = blockIdx.x; t < P.ntiles; t += nb) {
                const DevTile T = P.tiles[t];
                const DevSolve& S = P.solves[T.solve];
                const int s = T.solve;
                __syncthreads();
                if (w0) {
                    int go = 1;
                    double alpha = 0.0;
                    if (__ldcg(P.conv_outer + s) <= o || __ldcg(P.inner_tag + s) == o + 1) {
                        go = 0;
                    } else {
                        const double rrk = warp_sum_partials(P.part_rr + (size_t)cur * P.ntiles, S.tile0, S.ntiles);
                        const double sig = warp_sum_partials(P.part_sig, S.tile0, S.ntiles);
                        alpha = rrk / sig;
                    }
                    if (lane == 0) {
                        sh.go = go;
                        sh.s0 = alpha;
                    }
                }
                __syncthreads();
                if (!sh.go) continue;
                const VT va = (VT)sh.s0;
                const VT* pk = pb[cur] + S.off;
                VT* rr = r + S.off;
                VT* dd = d + S.off;
                VT acc = 0;
                const int items = (T.j1 - T.j0) * S.cpr;
                for (int it = threadIdx.x; it < items; it += BLOCK) {
                    const int j = T.j0 + it / S.cpr, c = it % S.cpr;
                    VT ps[4], pc[6], pn[4];
                    load_vec_chunk<VT>(pk, S.ld, S.n, j, c, ps, pc, pn);
                    VT a[3][6];
                    load_coef_chunk<ST, VT>(as + S.off, S.ld, S.n, j, c, a);
                    VT y[4];
                    apply_chunk<VT>(a, ps, pc, pn, S.n, c, y);
                    const size_t base = (size_t)j * S.ld + 4 * c;
                    VT dv[4], rv[4];
                    Vec4<VT>::load(dd + base, dv);
                    Vec4<VT>::load(rr + base, rv);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        dv[q] = dv[q] + va * pc[q + 1];
                        rv[q] = rv[q] - va * y[q];
                        acc += rv[q] * rv[q];
                    }
                    Vec4<VT>::store(dd + base, dv);
                    Vec4<VT>::store(rr + base, rv);
                }
                const double tot = block_sum<BLOCK>((double)acc, red);
                if (threadIdx.x == 0) P.part_rr[(size_t)(cur ^ 1) * P.ntiles + t] = tot;
            }
            if (!grid_barrier(P.bar, P.nbar, P.err, P.timeout_ns)) return;
        }
        if (__ldcg(P.active_count + o) == 0) break;

        // ---- U: x += d in FP64
        for (int t = blockIdx.x; t < P.ntiles; t += nb) {
            const DevTile T = P.tiles[t];
            const DevSolve& S = P.solves[T.solve];
            __syncthreads();
            if (threadIdx.x == 0) sh.go = (__ldcg(P.conv_outer + T.solve) > o);
            __syncthreads();
            if (!sh.go) continue;
            const int items = (T.j1 - T.j0) * S.cpr;
            for (int it = threadIdx.x; it < items; it += BLOCK) {
                const int j = T.j0 + it / S.cpr, c = it % S.cpr;
                const size_t base = S.off + (size_t)j * S.ld + 4 * c;
                double xv[4];
                VT dv[4];
                Vec4<double>::load(x64 + base, xv);
                Vec4<VT>::load(d + base, dv);
#pragma unroll
                for (int q = 0; q < 4; ++q) xv[q] += (double)dv[q];
                Vec4<double>::store(x64 + base, xv);
            }
        }
        if (!grid_barrier(P.bar, P.nbar, P.err, P.timeout_ns)) return;
    }

    // ---- Q: G(u) = sum g_i x_i; optional dense copy of u
    for (int t = blockIdx.x; t < P.ntiles; t += nb) {
        const DevTile T = P.tiles[t];
        const DevSolve& S = P.solves[T.solve];
        double acc = 0.0;
        const int items = (T.j1 - T.j0) * S.cpr;
        for (int it = threadIdx.x; it < items; it += BLOCK) {
            const int j = T.j0 + it / S.cpr, c = it % S.cpr;
            double xv[4];
            Vec4<double>::load(x64 + S.off + (size_t)j * S.ld + 4 * c, xv);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = 4 * c + q;
                if (i >= 1 && i <= S.n - 1) acc += qoi_weight(S, i, j) * xv[q];
            }
        }
        if (S.u) {
            double* u = S.u + (size_t)S.out * (S.n + 1) * (S.n + 1);
            const int jlo = (T.j0 == 1) ? 0 : T.j0;
            const int jhi = (T.j1 == S.n) ? S.n + 1 : T.j1;
            const int width = S.n + 1;
            for (int it = threadIdx.x; it < (jhi - jlo) * width; it += BLOCK) {
                const int j = jlo + it / width, i = it % width;
                const bool inner = (i >= 1 && i <= S.n - 1 && j >= 1 && j <= S.n - 1);
                u[(size_t)j * width + i] = inner ? x64[S.off + (size_t)j * S.ld + i] : 0.0;
            }
        }
        const double tot = block_sum<BLOCK>(acc, red);
        if (threadIdx.x == 0) P.part_q[t] = tot;
    }
    if (!grid_barrier(P.bar, P.nbar, P.err, P.timeout_ns)) return;
    if (w0) {
        for (int t = blockIdx.x; t < P.ntiles; t += nb) {
            const DevTile T = P.tiles[t];
            const DevSolve& S = P.solves[T.solve];
            if (t != S.tile0) continue;
            const double q = warp_sum_partials(P.part_q, S.tile0, S.ntiles);
            if (lane == 0) {
                if (S.Q) S.Q[S.out] = q;
                if (S.iters) S.iters[S.out] = P.iters_acc[T.solve];
                if (S.relres) S.relres[S.out] = P.rho_final[T.solve];
                if (S.flags) S.flags[S.out] = P.flags_acc[T.solve];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Stand-alone operator application y = A x (dense nodal layouts), for testing
// the stencil against element-by-element assembly.  The coefficient passes
// through the storage type ST exactly as inside the solver.
template <class VT, class ST>
__global__ void apply_operator_kernel(int n, int S, const void* a, int a_fp64, int a_n, const VT* x, VT* y) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int V = (n + 1) * (n + 1);
    if (tid >= (long long)S * V) return;
    const int s = (int)(tid / V);
    const int v = (int)(tid - (long long)s * V);
    const int i = v % (n + 1), j = v / (n + 1);
    const int st = a_n / n;
    const long long aV = (long long)(a_n + 1) * (a_n + 1);
    auto A = [&](int ii, int jj) -> VT {
        const long long idx = (long long)s * aV + (long long)(jj * st) * (a_n + 1) + (long long)ii * st;
        const double val = a_fp64 ? static_cast<const double*>(a)[idx] : (double)static_cast<const float*>(a)[idx];
        return widen<VT>(to_store<ST>(val));
    };
    VT out = (VT)0;
    if (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1) {
        const VT* xs = x + (size_t)s * V;
        auto X = [&](int ii, int jj) -> VT {
            return (ii >= 1 && ii <= n - 1 && jj >= 1 && jj <= n - 1) ? xs[jj * (n + 1) + ii] : (VT)0;
        };
        out = stencil_point<VT>(A(i, j), A(i + 1, j), A(i - 1, j), A(i, j + 1), A(i, j - 1), A(i + 1, j + 1),
                                A(i - 1, j - 1), X(i, j), X(i + 1, j), X(i - 1, j), X(i, j + 1), X(i, j - 1));
    }
    y[(size_t)s * V + v] = out;
}

// Occupancy-derived co-resident grid for each instantiation.
template <class VT, class ST>
int max_coresident(int num_sms) {
    static int cached = -1;
    if (cached < 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_solve<VT, ST>, BLOCK, 0) !=
                cudaSuccess ||
            per_sm <= 0)
            per_sm = 1;
        cached = per_sm;
    }
    return cached * num_sms;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <class VT, class ST>
mlmc_status run_typed(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                      cudaStream_t st) {
    // ---- host plan
    std::vector<DevSolve> solves;
    std::vector<DevTile> tiles;
    long long total = 0;
    const mlmc_problem& pb = ctx->prob;
    for (const SolveGroup& g : groups) {
        if (g.S <= 0) continue;
        const int n = g.n;
        const int ld = (int)align_up((size_t)n + 1, 4);
        const int stride = g.a_n / n;
        const size_t elem = g.a_fp64 ? sizeof(double) : sizeof(float);
        const long long aV = (long long)(g.a_n + 1) * (g.a_n + 1);
        const int rpt = std::max(1, std::min(n - 1, cfg.tile_nodes / ld));
        const int nt = (n - 1 + rpt - 1) / rpt;
        const double h = 1.0 / n;
        int bx0 = 0, bx1 = n, by0 = 0, by1 = n;
        if (pb.qoi == 1) {
            bx0 = (int)std::lround(pb.box[0] * n);
            bx1 = (int)std::lround(pb.box[1] * n);
            by0 = (int)std::lround(pb.box[2] * n);
            by1 = (int)std::lround(pb.box[3] * n);
        }
        double gnorm = 0.0;
        if (g.rhs_weights) gnorm = *g.rhs_weights;   // precomputed ||g||_2 for the adjoint rhs
        for (int s = 0; s < g.S; ++s) {
            DevSolve d{};
            d.n = n;
            d.ld = ld;
            d.off = total;
            total += (long long)align_up((size_t)(n + 1) * ld, 64);
            d.a = static_cast<const char*>(g.a) + (size_t)s * aV * elem;
            d.a_row = (long long)stride * (g.a_n + 1);
            d.a_col = stride;
            d.a_fp64 = g.a_fp64;
            d.tile0 = (int)tiles.size();
            d.ntiles = nt;
            d.cpr = (n - 1) / 4 + 1;
            d.rhs_mode = g.rhs_weights ? 1 : 0;
            d.qoi = pb.qoi;
            d.bx0 = bx0; d.bx1 = bx1; d.by0 = by0; d.by1 = by1;
            d.delta = g.delta;
            d.h2 = h * h;
            d.f = pb.f;
            d.bnorm = g.rhs_weights ? gnorm : std::fabs(pb.f) * h * h * (double)(n - 1);
            d.Q = g.Q;
            d.u = g.u;
            d.iters = g.iters;
            d.relres = g.relres;
            d.flags = g.flags;
            d.out = s;
            for (int tt = 0; tt < nt; ++tt) {
                DevTile T;
                T.solve = (int)solves.size();
                T.j0 = 1 + tt * rpt;
                T.j1 = std::min(n, T.j0 + rpt);
                tiles.push_back(T);
            }
            solves.push_back(d);
        }
    }
    const int ns = (int)solves.size(), ntl = (int)tiles.size();
    if (ns == 0) return MLMC_OK;
    const int max_outer = cfg.max_outer;

    // ---- workspace layout (256-byte aligned sections)
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_x = take(sizeof(double) * total);
    const size_t o_r = take(sizeof(VT) * total);
    const size_t o_p0 = take(sizeof(VT) * total);
    const size_t o_p1 = take(sizeof(VT) * total);
    const size_t o_d = take(sizeof(VT) * total);
    const size_t o_as = take(sizeof(ST) * total);
    const size_t zero_begin = off;   // everything below is cleared per launch except descriptors
    const size_t o_pres = take(sizeof(double) * ntl);
    const size_t o_prr0 = take(sizeof(double) * ntl);
    const size_t o_prr = take(sizeof(double) * 2 * ntl);
    const size_t o_psig = take(sizeof(double) * ntl);
    const size_t o_pq = take(sizeof(double) * ntl);
    const size_t o_inner = take(sizeof(int) * ns);
    const size_t o_iters = take(sizeof(int) * ns);
    const size_t o_rhoh = take(sizeof(double) * 2 * ns);
    const size_t o_rhof = take(sizeof(double) * ns);
    const size_t o_flags = take(sizeof(int) * ns);
    const size_t o_act = take(sizeof(int) * (max_outer + 1));
    const size_t o_done = take(sizeof(int) * (max_outer + 1));
    const size_t o_bar = take(sizeof(unsigned) * 4);
    const size_t zero_end = off;
    const size_t o_conv = take(sizeof(int) * ns);
    const size_t o_solves = take(sizeof(DevSolve) * ns);
    const size_t o_tiles = take(sizeof(DevTile) * ntl);
    const size_t need = off;

    mlmc::DevBuf& buf = ctx->ws.solver;
    MLMC_CUDA_RET(ctx->err, buf.reserve(need));
    char* base = buf.as<char>();
    // vectors start at zero (boundary and padding entries stay zero forever)
    MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(base, 0, zero_end, st));
    MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(base + o_conv, 0x7f, sizeof(int) * ns, st));
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(base + o_solves, solves.data(), sizeof(DevSolve) * ns,
                                            cudaMemcpyHostToDevice, st));
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(base + o_tiles, tiles.data(), sizeof(DevTile) * ntl,
                                            cudaMemcpyHostToDevice, st));
    (void)zero_begin;

    Params P{};
    P.solves = reinterpret_cast<const DevSolve*>(base + o_solves);
    P.tiles = reinterpret_cast<const DevTile*>(base + o_tiles);
    P.nsolves = ns;
    P.ntiles = ntl;
    P.x64 = reinterpret_cast<double*>(base + o_x);
    P.r = base + o_r;
    P.p0 = base + o_p0;
    P.p1 = base + o_p1;
    P.d = base + o_d;
    P.as = base + o_as;
    P.part_res = reinterpret_cast<double*>(base + o_pres);
    P.part_rr0 = reinterpret_cast<double*>(base + o_prr0);
    P.part_rr = reinterpret_cast<double*>(base + o_prr);
    P.part_sig = reinterpret_cast<double*>(base + o_psig);
    P.part_q = reinterpret_cast<double*>(base + o_pq);
    P.conv_outer = reinterpret_cast<int*>(base + o_conv);
    P.inner_tag = reinterpret_cast<int*>(base + o_inner);
    P.iters_acc = reinterpret_cast<int*>(base + o_iters);
    P.rho_hist = reinterpret_cast<double*>(base + o_rhoh);
    P.rho_final = reinterpret_cast<double*>(base + o_rhof);
    P.flags_acc = reinterpret_cast<int*>(base + o_flags);
    P.active_count = reinterpret_cast<int*>(base + o_act);
    P.done_count = reinterpret_cast<int*>(base + o_done);
    P.bar = reinterpret_cast<unsigned*>(base + o_bar);
    P.err = P.bar + 2;
    P.max_outer = max_outer;
    P.max_iters = cfg.max_iters;
    P.theta = cfg.inner_theta;
    // Refining the inner solve below what its operator can deliver wastes iterations:
    // a refinement step contracts the residual by about the storage unit roundoff.
    double tmin = 1e-6;
    if (cfg.prec == MLMC_FP64) tmin = 1e-14;
    if (cfg.prec == MLMC_FP16S) tmin = 1e-4;
    if (cfg.prec == MLMC_BF16S) tmin = 1e-3;
    P.tau_min = cfg.tau_min > 0 ? cfg.tau_min : tmin;
    P.tau_max = cfg.tau_max;
    P.stag = 0.5;
    P.timeout_ns = (unsigned long long)(ctx->wait_timeout_s * 1e9);

    const int grid = std::max(1, std::min(ntl, max_coresident<VT, ST>(ctx->num_sms)));
    P.nbar = (unsigned)(grid + std::max(0, ctx->barrier_extra));
    void* args[] = {&P};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (ctx->prof.on) {
        MLMC_CUDA_RET(ctx->err, cudaEventCreate(&ev[0]));
        MLMC_CUDA_RET(ctx->err, cudaEventCreate(&ev[1]));
        MLMC_CUDA_RET(ctx->err, cudaEventRecord(ev[0], st));
    }
    MLMC_CUDA_RET(ctx->err, cudaLaunchCooperativeKernel((const void*)persistent_solve<VT, ST>, dim3(grid),
                                                        dim3(BLOCK), args, 0, st));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (ctx->prof.on) MLMC_CUDA_RET(ctx->err, cudaEventRecord(ev[1], st));
    unsigned kerr = 0;
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(&kerr, P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_RET(ctx->err, cudaStreamSynchronize(st));
    ctx->prof.acc.h2d_bytes += (int64_t)(sizeof(DevSolve) * ns + sizeof(DevTile) * ntl);
    ctx->prof.acc.d2h_bytes += (int64_t)sizeof(unsigned);
    if (ctx->prof.on) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        std::vector<int> it(ns), co(ns);
        MLMC_CUDA_RET(ctx->err, cudaMemcpy(it.data(), P.iters_acc, sizeof(int) * ns, cudaMemcpyDeviceToHost));
        MLMC_CUDA_RET(ctx->err, cudaMemcpy(co.data(), P.conv_outer, sizeof(int) * ns, cudaMemcpyDeviceToHost));
        const double pv = sizeof(VT), ps = sizeof(ST);
        double bytes = 0.0;
        int64_t iters = 0, uit = 0;
        for (int i = 0; i < ns; ++i) {
            const double unk = (double)(solves[i].n - 1) * (solves[i].n - 1);
            const double pm = solves[i].a_fp64 ? 8.0 : 4.0;
            const int steps = std::min(co[i], max_outer);   // refinement (inner) solves
            bytes += unk * ((double)it[i] * (8 * pv + 2 * ps) + (double)(steps + 1) * (8 + pm + 2 * pv) +
                            (double)steps * (16 + pv) + (8 + pm + ps));
            iters += it[i];
            uit += (int64_t)unk * it[i];
        }
        mlmc_profile& A = ctx->prof.acc;
        A.solve_launches += 1;
        A.solve_ms += ms;
        A.solve_bytes += bytes;
        A.inner_iters += iters;
        A.unknown_iters += uit;
    }
    if (kerr == KERR_TIMEOUT) {
        ctx->err = "persistent solve: a grid barrier wait ran out (timeout)";
        return MLMC_E_TIMEOUT;
    }
    if (kerr != KERR_NONE) {
        ctx->err = "persistent solve: kernel error word set";
        return MLMC_E_CUDA;
    }
    return MLMC_OK;
}

}  // namespace

mlmc_status run_solve_batch(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                            cudaStream_t st) {
    if (cfg.solver != MLMC_CG) {
        ctx->err = "solver not available in this build";
        return MLMC_E_UNSUPPORTED;
    }
    switch (cfg.prec) {
        case MLMC_FP64: return run_typed<double, double>(ctx, groups, cfg, st);
        case MLMC_FP32: return run_typed<float, float>(ctx, groups, cfg, st);
        case MLMC_BF16S: return run_typed<float, __nv_bfloat16>(ctx, groups, cfg, st);
        case MLMC_FP16S: return run_typed<float, __half>(ctx, groups, cfg, st);
        default: ctx->err = "bad precision"; return MLMC_E_ARG;
    }
}

cudaError_t launch_apply_operator(int n, int S, const void* a, int a_fp64, int a_n, int op_prec, const void* x,
                                  void* y, int vec_fp64, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const long long work = (long long)S * (n + 1) * (n + 1);
    const unsigned grid = (unsigned)((work + 255) / 256);
    if (vec_fp64) {
        apply_operator_kernel<double, double><<<grid, 256, 0, st>>>(n, S, a, a_fp64, a_n,
                                                                    static_cast<const double*>(x),
                                                                    static_cast<double*>(y));
    } else {
        const float* xf = static_cast<const float*>(x);
        float* yf = static_cast<float*>(y);
        switch (op_prec) {
            case MLMC_FP32: apply_operator_kernel<float, float><<<grid, 256, 0, st>>>(n, S, a, a_fp64, a_n, xf, yf); break;
            case MLMC_BF16S:
                apply_operator_kernel<float, __nv_bfloat16><<<grid, 256, 0, st>>>(n, S, a, a_fp64, a_n, xf, yf);
                break;
            case MLMC_FP16S: apply_operator_kernel<float, __half><<<grid, 256, 0, st>>>(n, S, a, a_fp64, a_n, xf, yf); break;
            default: return cudaErrorInvalidValue;
        }
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mlmc

// ===========================================================================
// Allocation-free solve (mlmc_level_solve_noalloc): the persistent solve with
// its scratch in a file-scope device array instead of context workspaces.
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

// Descriptors of a batch of equal-shaped systems, written on the device.
__global__ void noalloc_plan_kernel(DevSolve proto, int S, long long stride_nodes, long long a_elems,
                                    int a_elem_bytes, int ntile_per, int rpt, DevSolve* solves, DevTile* tiles) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)S * ntile_per) return;
    const int s = (int)(idx / ntile_per), tt = (int)(idx % ntile_per);
    if (tt == 0) {
        DevSolve d = proto;
        d.off = s * stride_nodes;
        d.a = static_cast<const char*>(proto.a) + (size_t)s * a_elems * a_elem_bytes;
        d.tile0 = s * ntile_per;
        d.out = s;
        solves[s] = d;
    }
    DevTile T;
    T.solve = s;
    T.j0 = 1 + tt * rpt;
    T.j1 = min(proto.n, T.j0 + rpt);
    tiles[idx] = T;
}

template <class VT, class ST>
mlmc_status noalloc_typed(int n, int S, const void* a, int a_fp64, int a_n, double delta, int max_iters, int qoi,
                          const double* box, double f, int prec, double* Q, int32_t* iters, double* relres,
                          int32_t* flags, cudaStream_t st, void* scratch, int num_sms, std::string& err) {
    const int ld = (int)align_up((size_t)n + 1, 4);
    const int tile_nodes = 4096, max_outer = 12;
    const int rpt = std::max(1, std::min(n - 1, tile_nodes / ld));
    const int nt = (n - 1 + rpt - 1) / rpt;
    const long long stride = (long long)align_up((size_t)(n + 1) * ld, 64);
    const long long total = stride * S;
    const int ns = S, ntl = S * nt;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    const size_t o_x = take(sizeof(double) * total);
    const size_t o_r = take(sizeof(VT) * total);
    const size_t o_p0 = take(sizeof(VT) * total);
    const size_t o_p1 = take(sizeof(VT) * total);
    const size_t o_d = take(sizeof(VT) * total);
    const size_t o_as = take(sizeof(ST) * total);
    const size_t o_pres = take(sizeof(double) * ntl);
    const size_t o_prr0 = take(sizeof(double) * ntl);
    const size_t o_prr = take(sizeof(double) * 2 * ntl);
    const size_t o_psig = take(sizeof(double) * ntl);
    const size_t o_pq = take(sizeof(double) * ntl);
    const size_t o_inner = take(sizeof(int) * ns);
    const size_t o_iters = take(sizeof(int) * ns);
    const size_t o_rhoh = take(sizeof(double) * 2 * ns);
    const size_t o_rhof = take(sizeof(double) * ns);
    const size_t o_flags = take(sizeof(int) * ns);
    const size_t o_act = take(sizeof(int) * (max_outer + 1));
    const size_t o_done = take(sizeof(int) * (max_outer + 1));
    const size_t o_bar = take(sizeof(unsigned) * 4);
    const size_t zero_end = off;
    const size_t o_conv = take(sizeof(int) * ns);
    const size_t o_solves = take(sizeof(DevSolve) * ns);
    const size_t o_tiles = take(sizeof(DevTile) * ntl);
    if (off > kNoAllocBytes) {
        err = "level_solve_noalloc: the batch needs " + std::to_string(off) + " bytes of scratch, above the " +
              std::to_string(kNoAllocBytes) + "-byte maximum (MLMC_NOALLOC_SCRATCH_BYTES); use fewer systems";
        return MLMC_E_ARG;
    }
    char* base = static_cast<char*>(scratch);
    cudaError_t e;
    if ((e = cudaMemsetAsync(base, 0, zero_end, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + o_conv, 0x7f, sizeof(int) * ns, st)) != cudaSuccess) {
        err = std::string("level_solve_noalloc: cudaMemsetAsync: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    DevSolve proto{};
    proto.n = n;
    proto.ld = ld;
    proto.a = a;
    const int stridea = a_n / n;
    proto.a_row = (long long)stridea * (a_n + 1);
    proto.a_col = stridea;
    proto.a_fp64 = a_fp64;
    proto.ntiles = nt;
    proto.cpr = (n - 1) / 4 + 1;
    proto.rhs_mode = 0;
    proto.qoi = qoi;
    proto.bx0 = 0; proto.bx1 = n; proto.by0 = 0; proto.by1 = n;
    if (qoi == 1) {
        proto.bx0 = (int)std::lround(box[0] * n);
        proto.bx1 = (int)std::lround(box[1] * n);
        proto.by0 = (int)std::lround(box[2] * n);
        proto.by1 = (int)std::lround(box[3] * n);
    }
    const double h = 1.0 / n;
    proto.delta = delta;
    proto.h2 = h * h;
    proto.f = f;
    proto.bnorm = std::fabs(f) * h * h * (double)(n - 1);
    proto.Q = Q;
    proto.iters = iters;
    proto.relres = relres;
    proto.flags = flags;
    const long long a_elems = (long long)(a_n + 1) * (a_n + 1);
    noalloc_plan_kernel<<<(unsigned)((ntl + 255) / 256), 256, 0, st>>>(
        proto, S, stride, a_elems, a_fp64 ? 8 : 4, nt, rpt, reinterpret_cast<DevSolve*>(base + o_solves),
        reinterpret_cast<DevTile*>(base + o_tiles));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        err = std::string("level_solve_noalloc: plan kernel: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    Params P{};
    P.solves = reinterpret_cast<const DevSolve*>(base + o_solves);
    P.tiles = reinterpret_cast<const DevTile*>(base + o_tiles);
    P.nsolves = ns;
    P.ntiles = ntl;
    P.x64 = reinterpret_cast<double*>(base + o_x);
    P.r = base + o_r;
    P.p0 = base + o_p0;
    P.p1 = base + o_p1;
    P.d = base + o_d;
    P.as = base + o_as;
    P.part_res = reinterpret_cast<double*>(base + o_pres);
    P.part_rr0 = reinterpret_cast<double*>(base + o_prr0);
    P.part_rr = reinterpret_cast<double*>(base + o_prr);
    P.part_sig = reinterpret_cast<double*>(base + o_psig);
    P.part_q = reinterpret_cast<double*>(base + o_pq);
    P.conv_outer = reinterpret_cast<int*>(base + o_conv);
    P.inner_tag = reinterpret_cast<int*>(base + o_inner);
    P.iters_acc = reinterpret_cast<int*>(base + o_iters);
    P.rho_hist = reinterpret_cast<double*>(base + o_rhoh);
    P.rho_final = reinterpret_cast<double*>(base + o_rhof);
    P.flags_acc = reinterpret_cast<int*>(base + o_flags);
    P.active_count = reinterpret_cast<int*>(base + o_act);
    P.done_count = reinterpret_cast<int*>(base + o_done);
    P.bar = reinterpret_cast<unsigned*>(base + o_bar);
    P.err = P.bar + 2;
    P.max_outer = max_outer;
    P.max_iters = max_iters;
    P.theta = 0.3;
    double tmin = 1e-6;
    if (prec == MLMC_FP64) tmin = 1e-14;
    if (prec == MLMC_FP16S) tmin = 1e-4;
    if (prec == MLMC_BF16S) tmin = 1e-3;
    P.tau_min = tmin;
    P.tau_max = 0.5;
    P.stag = 0.5;
    P.timeout_ns = 10000000000ull;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_solve<VT, ST>, BLOCK, 0) != cudaSuccess ||
        per_sm <= 0)
        per_sm = 1;
    const int grid = std::max(1, std::min(ntl, per_sm * num_sms));
    P.nbar = (unsigned)grid;
    void* args[] = {&P};
    if ((e = cudaLaunchCooperativeKernel((const void*)persistent_solve<VT, ST>, dim3(grid), dim3(BLOCK), args, 0,
                                         st)) != cudaSuccess) {
        err = std::string("level_solve_noalloc: cooperative launch: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    unsigned kerr = 0;
    if ((e = cudaMemcpyAsync(&kerr, P.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        err = std::string("level_solve_noalloc: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    if (kerr == KERR_TIMEOUT) {
        err = "level_solve_noalloc: a grid barrier wait ran out (timeout)";
        return MLMC_E_TIMEOUT;
    }
    return kerr == KERR_NONE ? MLMC_OK : MLMC_E_CUDA;
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
    if (S == 0) return MLMC_OK;
    if (!a || !Q) {
        err = "level_solve_noalloc: null a or Q";
        return MLMC_E_ARG;
    }
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess) e = cudaSetDevice(device);
    int num_sms = 0;
    void* scratch = nullptr;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
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
            s = noalloc_typed<double, double>(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, prec, Q, iters,
                                              relres, flags, st, scratch, num_sms, err);
            break;
        case MLMC_FP32:
            s = noalloc_typed<float, float>(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, prec, Q, iters, relres,
                                            flags, st, scratch, num_sms, err);
            break;
        case MLMC_BF16S:
            s = noalloc_typed<float, __nv_bfloat16>(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, prec, Q, iters,
                                                    relres, flags, st, scratch, num_sms, err);
            break;
        default:
            s = noalloc_typed<float, __half>(n, S, a, a64, a_n, delta, max_iters, qoi, box, f, prec, Q, iters,
                                             relres, flags, st, scratch, num_sms, err);
            break;
    }
    cudaSetDevice(prev);
    return s;
}
