// A3-A7: matrix-free P1 operator, batched inner Krylov solve, FP64 iterative
// refinement and the QoI, for every system of a batch in one launch.
//
// This file holds the kernels and launchers of one inner precision; each
// solver_<precision>.cu defines MLMC_SOLVER_PREC (an mlmc_prec value) and
// includes it, so the four precisions compile as separate translation units.
// solver_common.cu dispatches to them.
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
//   x = 0; loop: r = b - A x (FP64, master coefficient; r = b while x = 0); stop if
//   ||r||/||b|| < delta (Eq. (2.1), C = 1); else solve A d = r with CG or MINRES
//   (Sec. 2.2), preconditioned by a geometric multigrid V-cycle or by Jacobi, in the
//   inner precision to ||r_k|| <= tau ||r_0||, tau = clamp(theta delta / rho,
//   tau_min, tau_max); x += d (FP64).  With the V-cycle, CG's first inner solve
//   starts from the full-multigrid (nested iteration) guess of d instead of 0.
// QoI (Problem 4.5): Q = sum_i g_i x_i, g_i = int_B phi_i (B = D: g_i = h^2).
//
// Execution: each system is solved start to finish by one group of threads --
// a 512-thread CTA for large grids, a 128-thread quarter of a CTA for medium
// grids, a warp for small grids -- so every synchronisation is group-local
// (__syncthreads, a named barrier, __syncwarp) and nothing waits on another
// group.  One launch covers all systems of a precision class: CTA b takes either
// one large system, four medium ones or sixteen small ones.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {

namespace {

constexpr int CTA = 512;              // threads per CTA
constexpr int G_BIG = 512, G_MED = 128, G_SMALL = 32;

struct DevSolve {
    int n, ld;
    long long off;           // node offset of this system's workspace grid
    const void* a;           // master coefficient at node (0,0)
    long long a_row;         // element stride between rows of `a`
    int a_col;               // element stride between columns of `a`
    int a_fp64;              // master precision (1: FP64, 0: FP32)
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
    int sys;                 // index of the system in the batch
    int mg_levels;           // multigrid: coarse levels below this grid (0: none)
    long long mg_off;        // multigrid: node offset of this system's coarse levels
};

struct Params {
    const DevSolve* solves;
    const int* order;        // systems in launch order: big, then medium, then small
    int nbig, nmed, nsmall;
    double* x64;
    void* r;
    void* p0;
    void* p1;
    void* d;
    void* as;
    void* dinv;              // inverse diagonal in the storage type (Jacobi)
    void* vb;                // MINRES: second Lanczos vector buffer
    void* w0;                // MINRES: search directions (two buffers)
    void* w1;
    int solver;              // MLMC_CG or MLMC_MINRES
    int32_t* sys_iters;      // per system: inner iterations
    int32_t* sys_outer;      // per system: refinement steps
    int max_outer, max_iters;
    double theta, tau_min, tau_max, stag;
    int jacobi;
    int ring;                // row-pipeline slots per team of a 512-thread CG group (0: no pipeline)
    int mg;                  // CG preconditioner: 0 Jacobi, 1 geometric multigrid V-cycle
    int mg_nu;               // multigrid: damped-Jacobi sweeps before and after the coarse correction
    int mg_coarse;           // multigrid: Jacobi sweeps on the coarsest grid (even)
    double mg_omega;         // multigrid: Jacobi damping
    int mg_smem_nmax;        // multigrid: coarse levels of at most this many cells sit in shared memory
    int mg_smem_off;         // ... at this offset of the dynamic shared memory (512-thread groups)
    int fmg;                 // multigrid CG: the first inner solve starts from a full-multigrid guess
    void* mz;                // multigrid: preconditioned residual z (fine grid)
    void* mt;                // multigrid: fine-grid scratch
    void* cx;                // multigrid: coarse-level iterate, scratch and right-hand side
    void* ct;
    void* cb;
    void* cas;               // multigrid: coarse-level coefficient and inverse diagonal (storage type)
    void* cdi;
    double* we;              // FP64 edge weights of the master operator, 6 wE and 6 wN (refinement residual)
    double* wn;
    unsigned* err;           // error word of the launch (KERR_*)
    unsigned long long timeout_ns;   // bound of every pipeline wait
    unsigned extra_tx;       // diagnostic: bytes a team's first full barrier expects and never receives
};

// Shared memory of the row pipeline.  A system of n cells is swept by
// nseg = 512 / cpr teams of cpr threads (cpr = 4-node chunks per row); each
// team owns `ring` slots large enough for the five rows (three vectors, two
// storage-type arrays) of one step of the update sweep.
__host__ __device__ constexpr int pipe_nseg(int n) { return (512 / ((n - 1) / 4 + 1)) > 1 ? 512 / ((n - 1) / 4 + 1) : 1; }
__host__ __device__ constexpr int pipe_slot_bytes(int ld, int pv, int ps) { return ((3 * pv + 2 * ps) * ld + 127) / 128 * 128; }
__host__ __device__ constexpr int pipe_bar_bytes(int n, int ring) { return (16 * ring * pipe_nseg(n) + 127) / 128 * 128; }
__host__ __device__ constexpr int pipe_smem_bytes(int n, int ld, int ring, int pv, int ps) {
    return pipe_bar_bytes(n, ring) + pipe_nseg(n) * ring * pipe_slot_bytes(ld, pv, ps);
}

// Workspace row pitch: a multiple of 8 elements, so that every row of every
// array (8- to 2-byte elements) starts on a 16-byte boundary for bulk copies.
__host__ __device__ constexpr int row_pitch(int n) { return (n + 1 + 7) / 8 * 8; }

// Multigrid hierarchy of an n-cell grid: halve while the grid is even and the
// half has at least 4 cells.  Level k >= 1 (n >> k cells) occupies
// mg_level_nodes(n >> k) nodes of the coarse-level arrays, levels in order.
constexpr int kMgMinN = 4;
__host__ __device__ constexpr int mg_level_count(int n, int min_n = kMgMinN) {
    int l = 0;
    while (n % 2 == 0 && n / 2 >= min_n) {
        n /= 2;
        ++l;
    }
    return l;
}
__host__ __device__ constexpr long long mg_level_nodes(int nk) {
    return ((long long)(nk + 1) * row_pitch(nk) + 63) / 64 * 64;
}
__host__ __device__ constexpr long long mg_coarse_nodes(int n, int nl) {
    long long t = 0;
    for (int k = 1; k <= nl; ++k) t += mg_level_nodes(n >> k);
    return t;
}
// Coarse levels of at most `nmax` cells of a 512-thread group live in its shared memory:
// per level x, scratch and b (p_v bytes each) and the coefficient and inverse diagonal
// (p_s bytes each) over the level's padded grid, 16-byte aligned, deepest levels last.
__host__ __device__ constexpr int mg_smem_array(int nk, int p) { return ((nk + 1) * row_pitch(nk) * p + 15) / 16 * 16; }
__host__ __device__ constexpr int mg_smem_level_bytes(int nk, int pv, int ps) {
    return 3 * mg_smem_array(nk, pv) + 2 * mg_smem_array(nk, ps);
}
// Bytes of the shared-memory levels of an n-cell grid with nl coarse levels, from level 1 up to
// (not including) level `upto`.
__host__ __device__ constexpr int mg_smem_bytes(int n, int nl, int nmax, int pv, int ps, int upto) {
    int t = 0;
    for (int k = 1; k <= nl && k < upto; ++k)
        if ((n >> k) <= nmax) t += mg_smem_level_bytes(n >> k, pv, ps);
    return t;
}

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

// The same from memory that may be shared or global (plain generic loads).
template <class ST, class CT>
__device__ __forceinline__ void load_coef_chunk_any(const ST* as, int ld, int n, int j, int c, CT a[3][6]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const ST* row = as + (size_t)(j - 1 + r) * ld;
        SmemLoad<ST, CT>::load4(row + 4 * c, &a[r][1]);
        a[r][0] = (c > 0) ? SmemLoad<ST, CT>::load1(row + 4 * c - 1) : (CT)0;
        a[r][5] = (4 * c + 4 <= n) ? SmemLoad<ST, CT>::load1(row + 4 * c + 4) : (CT)0;
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
    cc[0] = (c > 0) ? row[4 * c - 1] : (VT)0;
    cc[5] = (4 * c + 4 <= n) ? row[4 * c + 4] : (VT)0;
}

// Storage-type values at the chunk's cross neighbourhood (same shape as load_vec_chunk).
template <class ST, class CT>
__device__ __forceinline__ void load_coef_cross(const ST* v, int ld, int n, int j, int c, CT s[4], CT cc[6],
                                                CT nn[4]) {
    const ST* row = v + (size_t)j * ld;
    CoefLoad<ST, CT>::load4(row - ld + 4 * c, s);
    CoefLoad<ST, CT>::load4(row + 4 * c, &cc[1]);
    CoefLoad<ST, CT>::load4(row + ld + 4 * c, nn);
    cc[0] = (c > 0) ? CoefLoad<ST, CT>::load1(row + 4 * c - 1) : (CT)0;
    cc[5] = (4 * c + 4 <= n) ? CoefLoad<ST, CT>::load1(row + 4 * c + 4) : (CT)0;
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

// The master coefficient at node (i, j) in the compute type CT: FP32 masters are read as FP32
// (no FP64 conversion when CT is float).
template <class CT>
__device__ __forceinline__ CT master_a_as(const DevSolve& S, int i, int j) {
    const long long idx = (long long)j * S.a_row + (long long)i * S.a_col;
    return S.a_fp64 ? (CT)__ldg(static_cast<const double*>(S.a) + idx)
                    : (CT)__ldg(static_cast<const float*>(S.a) + idx);
}

// Inverse diagonal of the P1 operator at fine-grid node (i, j) of the grid whose nodes are 2^k
// fine nodes apart (k = 0: the grid itself), from the master coefficient, in the compute type
// of the inner solve (it only enters the preconditioner).
template <class CT>
__device__ __forceinline__ CT stencil_inv_diag(const DevSolve& S, int i, int j, int k) {
    const int d = 1 << k;
    const CT a00 = master_a_as<CT>(S, i, j), aE = master_a_as<CT>(S, i + d, j), aW = master_a_as<CT>(S, i - d, j);
    const CT aN = master_a_as<CT>(S, i, j + d), aS = master_a_as<CT>(S, i, j - d);
    const CT aNE = master_a_as<CT>(S, i + d, j + d), aSW = master_a_as<CT>(S, i - d, j - d);
    const CT two = (CT)2;
    const CT diag = (two * (a00 + aE) + aNE + aS + two * (aW + a00) + aN + aSW + two * (a00 + aN) + aNE + aW +
                     two * (aS + a00) + aE + aSW) * (CT)(1.0 / 6.0);
    return (CT)1 / diag;
}

// A master value in the storage type, converted from the compute type.
template <class ST, class CT> __device__ __forceinline__ ST store_from(CT v);
template <> __device__ __forceinline__ double store_from<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float store_from<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __half store_from<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 store_from<__nv_bfloat16, float>(float v) {
    return __float2bfloat16_rn(v);
}

__device__ __forceinline__ double rhs_value(const DevSolve& S, int i, int j) {
    return S.rhs_mode == 0 ? S.f * S.h2 : qoi_weight(S, i, j);
}


// ---------------------------------------------------------------------------
// Groups of GT threads that solve one system.
template <class T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;   // an xor butterfly leaves the same bits in every lane: addition commutes
}

template <int GT>
struct Group {
    int rank, gid;           // thread rank in the group, group index in the CTA
    double* red;             // 3 * (GT / 32) doubles of shared scratch
    double* bc;              // 4 doubles: results broadcast by the group's first thread
    __device__ __forceinline__ void sync() const {
        if (GT == 32) {
            __syncwarp();
        } else if (GT == CTA) {
            __syncthreads();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(GT) : "memory");
        }
    }
    // Sums over the group of three per-thread values of type T -- a butterfly
    // in T within each warp, then the warp sums in FP64 in a fixed order by the
    // first warp -- then fn(sum_a, sum_b, sum_c, r) evaluated once (by every
    // lane of a one-warp group, by thread 0 otherwise).  Every thread returns
    // the same r[0..3], converted to OT.
    template <class T, class OT, class FN>
    __device__ __forceinline__ void reduce(T a, T b, T c, FN fn, OT out[4]) const {
        a = warp_allsum(a);
        b = warp_allsum(b);
        c = warp_allsum(c);
        if (GT == 32) {
            double r[4] = {0.0, 0.0, 0.0, 0.0};
            fn((double)a, (double)b, (double)c, r);
#pragma unroll
            for (int i = 0; i < 4; ++i) out[i] = (OT)r[i];
            return;
        }
        constexpr int W = GT / 32;
        const int w = rank >> 5, lane = rank & 31;
        if (lane == 0) {
            red[w] = (double)a;
            red[W + w] = (double)b;
            red[2 * W + w] = (double)c;
        }
        sync();
        if (w == 0) {
            double ta = lane < W ? red[lane] : 0.0;
            double tb = lane < W ? red[W + lane] : 0.0;
            double tc = lane < W ? red[2 * W + lane] : 0.0;
            ta = warp_allsum(ta);
            tb = warp_allsum(tb);
            tc = warp_allsum(tc);
            if (lane == 0) {
                double r[4] = {0.0, 0.0, 0.0, 0.0};
                fn(ta, tb, tc, r);
                OT* o = reinterpret_cast<OT*>(bc);
#pragma unroll
                for (int i = 0; i < 4; ++i) o[i] = (OT)r[i];
            }
        }
        sync();
        const OT* o = reinterpret_cast<const OT*>(bc);
#pragma unroll
        for (int i = 0; i < 4; ++i) out[i] = o[i];
    }
    // Plain group sums, the same bits in every thread.
    template <class T>
    __device__ __forceinline__ void sum3(T a, T b, T c, double& sa, double& sb, double& sc) const {
        double o[4];
        reduce<T, double>(a, b, c, [](double x, double y, double z, double* r) { r[0] = x; r[1] = y; r[2] = z; },
                          o);
        sa = o[0];
        sb = o[1];
        sc = o[2];
    }
};

__device__ __forceinline__ double inner_tau(const Params& P, const DevSolve& S, double rho) {
    return fmin(fmax(P.theta * S.delta / rho, P.tau_min), P.tau_max);
}


// ---------------------------------------------------------------------------
// Row sweeps of the inner iteration.  A thread owns one 4-node column chunk c
// and marches down its row segment [ja, jb), keeping a 3-row window of the
// direction and of the coefficient in registers, so each row costs one vector
// load (plus two halo scalars) per array instead of the full 3 x 6 stencil
// neighbourhood.

// The stencil on a 4-node chunk from three coefficient rows (south, centre, north).
template <class CT>
__device__ __forceinline__ void apply_rows(const CT* aS, const CT* aC, const CT* aN, const CT* s, const CT* cc,
                                           const CT* nn, int n, int c, CT y[4]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int ii = t + 1;
        const int i = 4 * c + t;
        const CT v = stencil_point<CT>(aC[ii], aC[ii + 1], aC[ii - 1], aN[ii], aS[ii], aN[ii + 1], aS[ii - 1], cc[ii],
                                       cc[ii + 1], cc[ii - 1], nn[t], s[t]);
        y[t] = (i >= 1 && i <= n - 1) ? v : (CT)0;
    }
}

// Halo columns 4c-1 and 4c+4 of a chunk row: every lane loads its own, in the
// same batch as the row's four values (columns outside 0..n give 0).  Loading
// them beats fetching them from the neighbouring lanes by shuffles here: the
// sweeps are latency-bound, the loads overlap with the row's own loads and hit
// L1, whereas a shuffle adds a dependent step after them.
template <class T, class F>
__device__ __forceinline__ void halo_edges(int n, int c, F edge, T v[6]) {
    v[0] = (c > 0) ? edge(4 * c - 1) : (T)0;
    v[5] = (4 * c + 4 <= n) ? edge(4 * c + 4) : (T)0;
}

// Rounded-to-nearest products and FMAs, so that a value is formed with the same
// roundings wherever it is formed (its owner lane or a neighbour's halo).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// p = z + beta p_old with z = D^-1 r (JAC) or r, and p_old only when PREV.
template <class VT, bool JAC, bool PREV>
__device__ __forceinline__ VT dir_value(VT r, VT dinv, VT po, VT beta) {
    VT z = JAC ? mul_rn(r, dinv) : r;
    return PREV ? fma_rn(beta, po, z) : z;
}

// One row of the storage-type coefficient at columns 4c-1 .. 4c+4.
template <class ST, class CT>
__device__ __forceinline__ void coef_row(const ST* AS, int ld, int n, int jj, int c, CT v[6]) {
    const ST* rowb = AS + (size_t)jj * ld;
    CoefLoad<ST, CT>::load4(rowb + 4 * c, &v[1]);
    halo_edges<CT>(n, c, [&](int col) -> CT { return CoefLoad<ST, CT>::load1(rowb + col); }, v);
}

// One row of a vector at columns 4c-1 .. 4c+4.
template <class VT>
__device__ __forceinline__ void vec_row(const VT* V, int ld, int n, int jj, int c, VT v[6]) {
    const VT* rowb = V + (size_t)jj * ld;
    Vec4<VT>::load(rowb + 4 * c, &v[1]);
    halo_edges<VT>(n, c, [&](int col) -> VT { return rowb[col]; }, v);
}

// Direction at one row (columns 4c-1 .. 4c+4).
template <class VT, class ST, bool JAC, bool PREV>
__device__ __forceinline__ void dir_row(const VT* R, const ST* DI, const VT* PO, VT beta, int ld, int n, int jj,
                                        int c, VT v[6]) {
    const size_t rb = (size_t)jj * ld;
    VT r4[4], d4[4] = {(VT)0, (VT)0, (VT)0, (VT)0}, o4[4] = {(VT)0, (VT)0, (VT)0, (VT)0};
    Vec4<VT>::load(R + rb + 4 * c, r4);
    if (JAC) CoefLoad<ST, VT>::load4(DI + rb + 4 * c, d4);
    if (PREV) Vec4<VT>::load(PO + rb + 4 * c, o4);
    halo_edges<VT>(n, c,
                   [&](int col) -> VT {
                       return dir_value<VT, JAC, PREV>(R[rb + col], JAC ? CoefLoad<ST, VT>::load1(DI + rb + col) : (VT)0,
                                                       PREV ? PO[rb + col] : (VT)0, beta);
                   },
                   v);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q + 1] = dir_value<VT, JAC, PREV>(r4[q], d4[q], o4[q], beta);
}

// I1 sweep: writes p_new on rows [ja, jb) and returns this thread's part of (p, A p).
template <class VT, class ST, bool JAC, bool PREV>
__device__ __forceinline__ VT sweep_dir(const VT* R, const ST* DI, const VT* PO, VT* PN, const ST* AS, VT beta,
                                            int ld, int n, int c, int ja, int jb) {
    VT pm[6], p0[6], pp[6], am[6], a0[6], ap[6];
    dir_row<VT, ST, JAC, PREV>(R, DI, PO, beta, ld, n, ja - 1, c, pm);
    dir_row<VT, ST, JAC, PREV>(R, DI, PO, beta, ld, n, ja, c, p0);
    coef_row<ST, VT>(AS, ld, n, ja - 1, c, am);
    coef_row<ST, VT>(AS, ld, n, ja, c, a0);
    VT acc = 0;
    for (int j = ja; j < jb; ++j) {
        dir_row<VT, ST, JAC, PREV>(R, DI, PO, beta, ld, n, j + 1, c, pp);
        coef_row<ST, VT>(AS, ld, n, j + 1, c, ap);
        VT y[4];
        apply_rows<VT>(am, a0, ap, &pm[1], p0, &pp[1], n, c, y);
        Vec4<VT>::store(PN + (size_t)j * ld + 4 * c, &p0[1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc += p0[q + 1] * y[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            pm[q] = p0[q];
            p0[q] = pp[q];
            am[q] = a0[q];
            a0[q] = ap[q];
        }
    }
    return acc;
}

// I2 sweep: d += alpha p, r -= alpha A p on rows [ja, jb); returns (||r||^2, (r, z)) parts.
template <class VT, class ST, bool JAC>
__device__ __forceinline__ void sweep_upd(const VT* PK, VT* R, VT* D, const ST* DI, const ST* AS, VT alpha, int ld,
                                          int n, int c, int ja, int jb, VT& rr, VT& rz) {
    VT pm[6], p0[6], pp[6], am[6], a0[6], ap[6];
    vec_row<VT>(PK, ld, n, ja - 1, c, pm);
    vec_row<VT>(PK, ld, n, ja, c, p0);
    coef_row<ST, VT>(AS, ld, n, ja - 1, c, am);
    coef_row<ST, VT>(AS, ld, n, ja, c, a0);
    VT acc_r = 0, acc_z = 0;
    for (int j = ja; j < jb; ++j) {
        vec_row<VT>(PK, ld, n, j + 1, c, pp);
        coef_row<ST, VT>(AS, ld, n, j + 1, c, ap);
        const size_t base = (size_t)j * ld + 4 * c;
        VT dv[4], rv[4], zz[4];
        Vec4<VT>::load(D + base, dv);
        Vec4<VT>::load(R + base, rv);
        if (JAC) CoefLoad<ST, VT>::load4(DI + base, zz);
        VT y[4];
        apply_rows<VT>(am, a0, ap, &pm[1], p0, &pp[1], n, c, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dv[q] = dv[q] + alpha * p0[q + 1];
            rv[q] = rv[q] - alpha * y[q];
            acc_r += rv[q] * rv[q];
            acc_z += JAC ? rv[q] * (rv[q] * zz[q]) : rv[q] * rv[q];
        }
        Vec4<VT>::store(D + base, dv);
        Vec4<VT>::store(R + base, rv);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            pm[q] = p0[q];
            p0[q] = pp[q];
            am[q] = a0[q];
            a0[q] = ap[q];
        }
    }
    rr = acc_r;
    rz = acc_z;
}


// ---------------------------------------------------------------------------
// Stencil from the stored FP64 edge weights (the FP64 inner solve, whose storage
// type is FP64 too): (A x)_ij = (WE(i,j)(x - x_E) + WE(i-1,j)(x - x_W)
//   + WN(i,j)(x - x_N) + WN(i,j-1)(x - x_S)) / 6, about 9 FP64 operations per
// node instead of about 21 for rebuilding the weights from the nodal coefficient.
__device__ __forceinline__ void we_row(const double* WE, int ld, int j, int c, double w[5]) {
    const double* row = WE + (size_t)j * ld + 4 * c;
    Vec4<double>::load(row, &w[1]);
    w[0] = c > 0 ? row[-1] : 0.0;
}
__device__ __forceinline__ void wn_row(const double* WN, int ld, int j, int c, double w[4]) {
    Vec4<double>::load(WN + (size_t)j * ld + 4 * c, w);
}
template <class VT>
__device__ __forceinline__ void apply_rows_w(const double we[5], const double ws[4], const double wn[4], const VT* s,
                                             const VT* cc, const VT* nn, int n, int c, VT y[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = 4 * c + q;
        const VT x0 = cc[q + 1];
        const VT v = (we[q + 1] * (x0 - cc[q + 2]) + we[q] * (x0 - cc[q]) + wn[q] * (x0 - nn[q]) + ws[q] * (x0 - s[q])) *
                     (VT)(1.0 / 6.0);
        y[q] = (i >= 1 && i <= n - 1) ? v : (VT)0;
    }
}

// I1 sweep with stored weights (same recurrences as sweep_dir).
template <class VT, class ST, bool JAC, bool PREV>
__device__ __forceinline__ VT sweep_dir_w(const VT* R, const ST* DI, const VT* PO, VT* PN, const double* WE,
                                          const double* WN, VT beta, int ld, int n, int c, int ja, int jb) {
    VT pm[6], p0[6], pp[6];
    double ws[4], we[5], wn[4];
    dir_row<VT, ST, JAC, PREV>(R, DI, PO, beta, ld, n, ja - 1, c, pm);
    dir_row<VT, ST, JAC, PREV>(R, DI, PO, beta, ld, n, ja, c, p0);
    wn_row(WN, ld, ja - 1, c, ws);
    VT acc = 0;
    for (int j = ja; j < jb; ++j) {
        dir_row<VT, ST, JAC, PREV>(R, DI, PO, beta, ld, n, j + 1, c, pp);
        we_row(WE, ld, j, c, we);
        wn_row(WN, ld, j, c, wn);
        VT y[4];
        apply_rows_w<VT>(we, ws, wn, &pm[1], p0, &pp[1], n, c, y);
        Vec4<VT>::store(PN + (size_t)j * ld + 4 * c, &p0[1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc += p0[q + 1] * y[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            pm[q] = p0[q];
            p0[q] = pp[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) ws[q] = wn[q];
    }
    return acc;
}

// I2 sweep with stored weights (same recurrences as sweep_upd).
template <class VT, class ST, bool JAC>
__device__ __forceinline__ void sweep_upd_w(const VT* PK, VT* R, VT* D, const ST* DI, const double* WE,
                                            const double* WN, VT alpha, int ld, int n, int c, int ja, int jb, VT& rr,
                                            VT& rz) {
    VT pm[6], p0[6], pp[6];
    double ws[4], we[5], wn[4];
    vec_row<VT>(PK, ld, n, ja - 1, c, pm);
    vec_row<VT>(PK, ld, n, ja, c, p0);
    wn_row(WN, ld, ja - 1, c, ws);
    VT acc_r = 0, acc_z = 0;
    for (int j = ja; j < jb; ++j) {
        vec_row<VT>(PK, ld, n, j + 1, c, pp);
        we_row(WE, ld, j, c, we);
        wn_row(WN, ld, j, c, wn);
        const size_t base = (size_t)j * ld + 4 * c;
        VT dv[4], rv[4], zz[4];
        Vec4<VT>::load(D + base, dv);
        Vec4<VT>::load(R + base, rv);
        if (JAC) CoefLoad<ST, VT>::load4(DI + base, zz);
        VT y[4];
        apply_rows_w<VT>(we, ws, wn, &pm[1], p0, &pp[1], n, c, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dv[q] = dv[q] + alpha * p0[q + 1];
            rv[q] = rv[q] - alpha * y[q];
            acc_r += rv[q] * rv[q];
            acc_z += JAC ? rv[q] * (rv[q] * zz[q]) : rv[q] * rv[q];
        }
        Vec4<VT>::store(D + base, dv);
        Vec4<VT>::store(R + base, rv);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            pm[q] = p0[q];
            p0[q] = pp[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) ws[q] = wn[q];
    }
    rr = acc_r;
    rz = acc_z;
}

// ---------------------------------------------------------------------------
// Row pipeline of the 512-thread CG groups.  The row segments of a system are
// teams of cpr threads.  A team streams the rows its sweep needs through a ring
// of shared-memory slots: its first thread issues bulk asynchronous copies of
// whole rows (the TMA engine) ring - 1 steps ahead of the row being computed,
// so loads never wait on HBM latency.  Slot s has a `full` mbarrier (one
// arrival plus the copied bytes) and an `empty` mbarrier (one arrival per team
// thread, when it has read the slot).  Every wait is bounded in wall time; on
// expiry the CTA raises its abort flag and the launch's error word, every
// later wait returns at once, the sweeps run to their ends on whatever the
// slots hold, and the solve stops at its next reduction.
struct Pipe {
    uint8_t* slots = nullptr;    // this team's ring
    uint64_t* full = nullptr;
    uint64_t* empty = nullptr;
    int ring = 0, slot_bytes = 0;
    // consumer position (the same in every team thread): slot and parity of the next step
    int cslot = 0;
    unsigned cphase = 0;
    // producer position (team leader): slot, parity and count of the next step to issue
    int pslot = 0;
    unsigned pphase = 0;
    unsigned issued = 0;
    bool leader = false;         // lane 0 of the leader warp: owns the producer position
    bool lead_warp = false;      // the team's first warp issues the copies
    int* abort = nullptr;        // CTA abort flag (shared memory)
    unsigned* err = nullptr;
    unsigned long long timeout_ns = 0;
    unsigned extra_tx = 0;
};

__device__ __forceinline__ bool pipe_aborted(const Pipe& p) { return *(volatile int*)p.abort != 0; }

__device__ __forceinline__ bool pipe_wait(Pipe& p, uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (pipe_aborted(p)) return false;
        if (global_ns() - t0 > p.timeout_ns) {
            *(volatile int*)p.abort = 1;
            atomicCAS(p.err, KERR_NONE, KERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Leader: claim the slot of the next step once every team thread has read its
// previous contents (the empty phase one lap earlier), and announce `bytes` on
// its full barrier.  nullptr after an abort.
__device__ __forceinline__ uint8_t* pipe_produce(Pipe& p, uint32_t bytes, uint64_t*& bar) {
    const int s = p.pslot;
    if (p.issued >= (unsigned)p.ring && !pipe_wait(p, p.empty + s, p.pphase ^ 1u)) return nullptr;
    if (pipe_aborted(p)) return nullptr;
    bar = p.full + s;
    mbar_expect_tx(bar, bytes + (p.issued == 0 ? p.extra_tx : 0u));
    ++p.issued;
    if (++p.pslot == p.ring) {
        p.pslot = 0;
        p.pphase ^= 1u;
    }
    return p.slots + (size_t)s * p.slot_bytes;
}

// Every team thread: wait for the next step's rows, then release the slot once read.
__device__ __forceinline__ const uint8_t* pipe_acquire(Pipe& p) {
    pipe_wait(p, p.full + p.cslot, p.cphase);
    return p.slots + (size_t)p.cslot * p.slot_bytes;
}
__device__ __forceinline__ void pipe_release(Pipe& p) {
    mbar_arrive(p.empty + p.cslot);
    if (++p.cslot == p.ring) {
        p.cslot = 0;
        p.cphase ^= 1u;
    }
}

// Leader, after an abort: wait (bounded) for the copies of each slot's last issued step.
__device__ __forceinline__ void pipe_drain(Pipe& p) {
    for (int s = 0; s < p.ring; ++s) {
        if (p.issued <= (unsigned)s) continue;
        const unsigned g = p.issued - 1u - ((p.issued - 1u - (unsigned)s) % (unsigned)p.ring);
        mbar_wait(p.full + s, (g / (unsigned)p.ring) & 1u, p.timeout_ns);
    }
}

// Leader warp: issue one pipeline step -- lane 0 claims the slot and posts the
// step's `total` bytes, then every lane holding a copy (src != nullptr) issues
// it into slot + off.  Returns false after an abort.
__device__ __forceinline__ bool pipe_issue_step(Pipe& p, uint32_t total, const void* src, uint32_t off,
                                                uint32_t bytes) {
    const int lane = threadIdx.x & 31;
    uint8_t* dst = nullptr;
    uint64_t* bar = nullptr;
    if (lane == 0) dst = pipe_produce(p, total, bar);
    dst = reinterpret_cast<uint8_t*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(dst), 0));
    bar = reinterpret_cast<uint64_t*>(__shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(bar), 0));
    if (!dst) return false;
    if (src) bulk_g2s(dst + off, src, bytes, bar);
    return true;
}

// A row of a vector (columns 4c-1 .. 4c+4) from a shared-memory slot.
template <class VT>
__device__ __forceinline__ void srow_vec(const VT* row, int n, int c, VT v[6]) {
    Vec4<VT>::load(row + 4 * c, &v[1]);
    halo_edges<VT>(n, c, [&](int col) -> VT { return row[col]; }, v);
}
// A row of a storage-type array (columns 4c-1 .. 4c+4) from a shared-memory slot.
template <class ST, class CT>
__device__ __forceinline__ void srow_coef(const ST* row, int n, int c, CT v[6]) {
    SmemLoad<ST, CT>::load4(row + 4 * c, &v[1]);
    halo_edges<CT>(n, c, [&](int col) -> CT { return SmemLoad<ST, CT>::load1(row + col); }, v);
}

// I1 sweep through the pipeline: the same arithmetic as sweep_dir.  Step t
// carries row ja - 1 + t of r, D^-1, p_old and the coefficient.
template <class VT, class ST, bool JAC, bool PREV>
__device__ __forceinline__ VT sweep_dir_staged(Pipe& p, const VT* R, const ST* DI, const VT* PO, VT* PN,
                                               const ST* AS, VT beta, int ld, int n, int c, int ja, int jb) {
    const uint32_t rv = (uint32_t)ld * sizeof(VT), rs = (uint32_t)ld * sizeof(ST);
    const uint32_t o_di = rv, o_po = o_di + (JAC ? rs : 0u), o_as = o_po + (PREV ? rv : 0u);
    const uint32_t total = o_as + rs;
    const int nsteps = jb - ja + 2;                 // rows ja-1 .. jb
    int next = 0;                                   // leader warp: next step of this sweep to issue
    auto issue_to = [&](int upto) {
        for (; next < upto && next < nsteps; ++next) {
            const size_t row = (size_t)(ja - 1 + next) * ld;
            // lane 0: r; lane 1: D^-1 (JAC); next lane: p_old (PREV); next lane: coefficient
            constexpr int l_di = JAC ? 1 : -1, l_po = PREV ? (JAC ? 2 : 1) : -1, l_as = 1 + JAC + PREV;
            const int lane = threadIdx.x & 31;
            const void* src = nullptr;
            uint32_t off = 0, by = 0;
            if (lane == 0) { src = R + row; off = 0; by = rv; }
            if (lane == l_di) { src = DI + row; off = o_di; by = rs; }
            if (lane == l_po) { src = PO + row; off = o_po; by = rv; }
            if (lane == l_as) { src = AS + row; off = o_as; by = rs; }
            if (!pipe_issue_step(p, total, src, off, by)) {
                next = nsteps;
                break;
            }
        }
    };
    const int depth = p.ring - 1;
    int taken = 0;
    auto take = [&](VT* pv, VT* av) {
        const uint8_t* sl = pipe_acquire(p);
        const VT* rrow = reinterpret_cast<const VT*>(sl);
        const ST* drow = reinterpret_cast<const ST*>(sl + o_di);
        const VT* prow = reinterpret_cast<const VT*>(sl + o_po);
        VT r4[4], d4[4] = {(VT)0, (VT)0, (VT)0, (VT)0}, o4[4] = {(VT)0, (VT)0, (VT)0, (VT)0};
        Vec4<VT>::load(rrow + 4 * c, r4);
        if (JAC) SmemLoad<ST, VT>::load4(drow + 4 * c, d4);
        if (PREV) Vec4<VT>::load(prow + 4 * c, o4);
        halo_edges<VT>(n, c,
                       [&](int col) -> VT {
                           return dir_value<VT, JAC, PREV>(rrow[col], JAC ? SmemLoad<ST, VT>::load1(drow + col) : (VT)0,
                                                           PREV ? prow[col] : (VT)0, beta);
                       },
                       pv);
#pragma unroll
        for (int q = 0; q < 4; ++q) pv[q + 1] = dir_value<VT, JAC, PREV>(r4[q], d4[q], o4[q], beta);
        srow_coef<ST, VT>(reinterpret_cast<const ST*>(sl + o_as), n, c, av);
        pipe_release(p);
        ++taken;
        if (p.lead_warp) issue_to(taken + depth);
    };
    if (p.lead_warp) issue_to(depth);
    VT pm[6], p0[6], pp[6], am[6], a0[6], ap[6];
    take(pm, am);
    take(p0, a0);
    VT acc = 0;
    for (int j = ja; j < jb; ++j) {
        take(pp, ap);
        VT y[4];
        apply_rows<VT>(am, a0, ap, &pm[1], p0, &pp[1], n, c, y);
        Vec4<VT>::store(PN + (size_t)j * ld + 4 * c, &p0[1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc += p0[q + 1] * y[q];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            pm[q] = p0[q];
            p0[q] = pp[q];
            am[q] = a0[q];
            a0[q] = ap[q];
        }
    }
    fence_proxy_async_global();
    return acc;
}

// I2 sweep through the pipeline: the same arithmetic as sweep_upd.  Steps 0
// and 1 carry rows ja-1 and ja of p and the coefficient; step 2+q carries row
// ja+q+1 of p and the coefficient and row ja+q of d, r and D^-1.
template <class VT, class ST, bool JAC>
__device__ __forceinline__ void sweep_upd_staged(Pipe& p, const VT* PK, VT* R, VT* D, const ST* DI, const ST* AS,
                                                 VT alpha, int ld, int n, int c, int ja, int jb, VT& rr, VT& rz) {
    const uint32_t rv = (uint32_t)ld * sizeof(VT), rs = (uint32_t)ld * sizeof(ST);
    const uint32_t o_as = rv, o_d = o_as + rs, o_r = o_d + rv, o_di = o_r + rv;
    const int nsteps = jb - ja + 2;
    int next = 0;
    auto issue_to = [&](int upto) {
        for (; next < upto && next < nsteps; ++next) {
            const size_t rowk = (size_t)(ja - 1 + next) * ld;
            const size_t rowo = (size_t)(ja - 2 + next) * ld;
            // lanes 0, 1: p and coefficient at row ja-1+next; lanes 2, 3, 4: d, r, D^-1 at row ja-2+next
            const int lane = threadIdx.x & 31;
            const bool own = next >= 2;
            const void* src = nullptr;
            uint32_t off = 0, by = 0;
            if (lane == 0) { src = PK + rowk; off = 0; by = rv; }
            if (lane == 1) { src = AS + rowk; off = o_as; by = rs; }
            if (own && lane == 2) { src = D + rowo; off = o_d; by = rv; }
            if (own && lane == 3) { src = R + rowo; off = o_r; by = rv; }
            if (own && JAC && lane == 4) { src = DI + rowo; off = o_di; by = rs; }
            const uint32_t total = own ? o_di + (JAC ? rs : 0u) : o_d;
            if (!pipe_issue_step(p, total, src, off, by)) {
                next = nsteps;
                break;
            }
        }
    };
    const int depth = p.ring - 1;
    int taken = 0;
    if (p.lead_warp) issue_to(depth);
    VT pm[6], p0[6], pp[6], am[6], a0[6], ap[6];
    {
        const uint8_t* sl = pipe_acquire(p);
        srow_vec<VT>(reinterpret_cast<const VT*>(sl), n, c, pm);
        srow_coef<ST, VT>(reinterpret_cast<const ST*>(sl + o_as), n, c, am);
        pipe_release(p);
        ++taken;
        if (p.lead_warp) issue_to(taken + depth);
        sl = pipe_acquire(p);
        srow_vec<VT>(reinterpret_cast<const VT*>(sl), n, c, p0);
        srow_coef<ST, VT>(reinterpret_cast<const ST*>(sl + o_as), n, c, a0);
        pipe_release(p);
        ++taken;
        if (p.lead_warp) issue_to(taken + depth);
    }
    VT acc_r = 0, acc_z = 0;
    for (int j = ja; j < jb; ++j) {
        const uint8_t* sl = pipe_acquire(p);
        srow_vec<VT>(reinterpret_cast<const VT*>(sl), n, c, pp);
        srow_coef<ST, VT>(reinterpret_cast<const ST*>(sl + o_as), n, c, ap);
        VT dv[4], rv4[4], zz[4];
        Vec4<VT>::load(reinterpret_cast<const VT*>(sl + o_d) + 4 * c, dv);
        Vec4<VT>::load(reinterpret_cast<const VT*>(sl + o_r) + 4 * c, rv4);
        if (JAC) SmemLoad<ST, VT>::load4(reinterpret_cast<const ST*>(sl + o_di) + 4 * c, zz);
        pipe_release(p);
        ++taken;
        if (p.lead_warp) issue_to(taken + depth);
        VT y[4];
        apply_rows<VT>(am, a0, ap, &pm[1], p0, &pp[1], n, c, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dv[q] = dv[q] + alpha * p0[q + 1];
            rv4[q] = rv4[q] - alpha * y[q];
            acc_r += rv4[q] * rv4[q];
            acc_z += JAC ? rv4[q] * (rv4[q] * zz[q]) : rv4[q] * rv4[q];
        }
        const size_t base = (size_t)j * ld + 4 * c;
        Vec4<VT>::store(D + base, dv);
        Vec4<VT>::store(R + base, rv4);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            pm[q] = p0[q];
            p0[q] = pp[q];
            am[q] = a0[q];
            a0[q] = ap[q];
        }
    }
    fence_proxy_async_global();
    rr = acc_r;
    rz = acc_z;
}


// ---------------------------------------------------------------------------
// MINRES sweeps (preconditioned Lanczos with Givens rotations, Paige-Saunders).
// zn_j = Z_j / gamma_j is the normalised preconditioned Lanczos vector.

// Pending update of iteration j-1, elementwise at one chunk:
// w_new = (zn_prev - a3 w_old - a2 w_new_prev) / a1 (stored over w_old), d += cst w_new.
template <class VT>
__device__ __forceinline__ void minres_update_chunk(const VT* ZP, VT gpi, VT* WO, const VT* WN, VT* D, VT a1i, VT a2,
                                                    VT a3, VT cst, size_t base) {
    VT zp[4], wo[4], wn[4], dv[4];
    Vec4<VT>::load(ZP + base, zp);
    Vec4<VT>::load(WO + base, wo);
    Vec4<VT>::load(WN + base, wn);
    Vec4<VT>::load(D + base, dv);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const VT w = (zp[q] * gpi - a3 * wo[q] - a2 * wn[q]) * a1i;
        wo[q] = w;
        dv[q] = dv[q] + cst * w;
    }
    Vec4<VT>::store(WO + base, wo);
    Vec4<VT>::store(D + base, dv);
}

// Sweep A: this thread's part of delta_j = (A zn_j, zn_j); with UPD, also the pending update.
template <class VT, class ST, bool UPD>
__device__ __forceinline__ VT sweep_minres_a(const VT* ZC, VT gci, const ST* AS, int ld, int n, int c, int ja,
                                                 int jb, const VT* ZP, VT gpi, VT* WO, const VT* WN, VT* D, VT a1i,
                                                 VT a2, VT a3, VT cst) {
    VT zm[6], z0[6], zp[6], am[6], a0[6], ap[6];
    vec_row<VT>(ZC, ld, n, ja - 1, c, zm);
    vec_row<VT>(ZC, ld, n, ja, c, z0);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        zm[q] *= gci;
        z0[q] *= gci;
    }
    coef_row<ST, VT>(AS, ld, n, ja - 1, c, am);
    coef_row<ST, VT>(AS, ld, n, ja, c, a0);
    VT acc = 0;
    for (int j = ja; j < jb; ++j) {
        vec_row<VT>(ZC, ld, n, j + 1, c, zp);
#pragma unroll
        for (int q = 0; q < 6; ++q) zp[q] *= gci;
        coef_row<ST, VT>(AS, ld, n, j + 1, c, ap);
        VT y[4];
        apply_rows<VT>(am, a0, ap, &zm[1], z0, &zp[1], n, c, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc += z0[q + 1] * y[q];
        if (UPD) minres_update_chunk<VT>(ZP, gpi, WO, WN, D, a1i, a2, a3, cst, (size_t)j * ld + 4 * c);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            zm[q] = z0[q];
            z0[q] = zp[q];
            am[q] = a0[q];
            a0[q] = ap[q];
        }
    }
    return acc;
}

// Sweep B: v_{j+1} = A zn_j - cA v_j - cB v_{j-1} (over v_{j-1}), z_{j+1} = D^-1 v_{j+1} or v_{j+1};
// returns this thread's part of (z_{j+1}, v_{j+1}).
template <class VT, class ST, bool JAC>
__device__ __forceinline__ VT sweep_minres_b(const VT* ZC, VT gci, const ST* AS, VT* VP, const VT* VC,
                                                 const ST* DI, VT* ZN, VT cA, VT cB, int ld, int n, int c, int ja,
                                                 int jb) {
    VT zm[6], z0[6], zp[6], am[6], a0[6], ap[6];
    vec_row<VT>(ZC, ld, n, ja - 1, c, zm);
    vec_row<VT>(ZC, ld, n, ja, c, z0);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        zm[q] *= gci;
        z0[q] *= gci;
    }
    coef_row<ST, VT>(AS, ld, n, ja - 1, c, am);
    coef_row<ST, VT>(AS, ld, n, ja, c, a0);
    VT acc = 0;
    for (int j = ja; j < jb; ++j) {
        vec_row<VT>(ZC, ld, n, j + 1, c, zp);
#pragma unroll
        for (int q = 0; q < 6; ++q) zp[q] *= gci;
        coef_row<ST, VT>(AS, ld, n, j + 1, c, ap);
        VT y[4];
        apply_rows<VT>(am, a0, ap, &zm[1], z0, &zp[1], n, c, y);
        const size_t base = (size_t)j * ld + 4 * c;
        VT vp[4], vc[4], dd[4];
        Vec4<VT>::load(VP + base, vp);
        Vec4<VT>::load(VC + base, vc);
        if (JAC) CoefLoad<ST, VT>::load4(DI + base, dd);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            vp[q] = y[q] - cA * vc[q] - cB * vp[q];
            vc[q] = JAC ? dd[q] * vp[q] : vp[q];
            acc += vc[q] * vp[q];
        }
        Vec4<VT>::store(VP + base, vp);
        Vec4<VT>::store(ZN + base, vc);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            zm[q] = z0[q];
            z0[q] = zp[q];
            am[q] = a0[q];
            a0[q] = ap[q];
        }
    }
    return acc;
}

// ---------------------------------------------------------------------------
// Geometric multigrid V-cycle: the CG preconditioner when P.mg != 0 (the
// optimal solver the cost model of Sec. 4 assumes, cost per sample ~ unknowns).
//  - Level k >= 1 is the grid of n >> k cells.  Its nodal coefficient is the
//    master coefficient injected at the coarse nodes, a_k(I, J) = a(2^k I, 2^k J),
//    and its operator is the P1 operator of Sec. 3.1 re-discretised on it.
//  - Prolongation P is P1 interpolation on the SW-NE triangulation: even nodes
//    copy the coarse value, edge midpoints (horizontal, vertical and the SW-NE
//    diagonal) average its two ends.  Restriction is P^T.
//  - Smoothing: nu damped-Jacobi sweeps before and nu after the coarse
//    correction; the coarsest grid takes mg_coarse sweeps from zero.
// Every step is a fixed linear map and the post-smoother is the adjoint of the
// pre-smoother, so z = B r is symmetric in r, as CG needs.  Each pass is one
// group-strided loop over 4-node chunks followed by a group barrier.
template <class VT, class ST>
struct MGLevel {
    int n, ld, cpr;
    VT* x;          // iterate (level 0: z)
    VT* t;          // scratch
    VT* b;          // right-hand side (level 0: r, read only)
    const ST* a;    // coefficient in the storage type
    const ST* di;   // inverse diagonal in the storage type (zero off the interior)
    const double* we;   // FP64 inner solve, grid level: stored edge weights (else nullptr)
    const double* wn;
};

template <class VT, class ST>
__device__ __forceinline__ MGLevel<VT, ST> mg_level(const Params& P, const DevSolve& S, int k, VT* Z, VT* T,
                                                   const VT* R, const ST* AS, const ST* DI, uint8_t* cs) {
    MGLevel<VT, ST> L;
    if (k == 0) {
        L.n = S.n;
        L.ld = S.ld;
        L.x = Z;
        L.t = T;
        L.b = const_cast<VT*>(R);
        L.a = AS;
        L.di = DI;
        // the FP64 inner solve applies its grid operator from the stored FP64 edge weights
        const bool w64 = sizeof(VT) == 8 && sizeof(ST) == 8;
        L.we = w64 ? P.we + S.off : nullptr;
        L.wn = w64 ? P.wn + S.off : nullptr;
    } else {
        L.we = nullptr;
        L.wn = nullptr;
        L.n = S.n >> k;
        L.ld = row_pitch(L.n);
        if (cs && L.n <= P.mg_smem_nmax) {
            uint8_t* q = cs + mg_smem_bytes(S.n, S.mg_levels, P.mg_smem_nmax, (int)sizeof(VT), (int)sizeof(ST), k);
            const int av = mg_smem_array(L.n, (int)sizeof(VT)), as = mg_smem_array(L.n, (int)sizeof(ST));
            L.x = reinterpret_cast<VT*>(q);
            L.t = reinterpret_cast<VT*>(q + av);
            L.b = reinterpret_cast<VT*>(q + 2 * av);
            L.a = reinterpret_cast<const ST*>(q + 3 * av);
            L.di = reinterpret_cast<const ST*>(q + 3 * av + as);
        } else {
            const long long off = S.mg_off + mg_coarse_nodes(S.n, k - 1);
            L.x = static_cast<VT*>(P.cx) + off;
            L.t = static_cast<VT*>(P.ct) + off;
            L.b = static_cast<VT*>(P.cb) + off;
            L.a = static_cast<const ST*>(P.cas) + off;
            L.di = static_cast<const ST*>(P.cdi) + off;
        }
    }
    L.cpr = (L.n - 1) / 4 + 1;
    return L;
}

// The loads of one 4-node chunk of a smoothing or residual pass.  Passes handle
// two chunks per step, loading both before using either, so that each thread
// keeps two chunks' loads in flight.
template <class VT>
struct MGChunk {
    VT b4[4], d4[4], a3[3][6], xs[4], xc[6], xn[4];
};
// Stored-weight form (FP64 inner solve, grid level): the edge weights replace the coefficient.
template <class VT>
struct MGChunkW {
    VT b4[4], d4[4], xs[4], xc[6], xn[4];
    double we[5], ws[4], wn[4];
};
template <class VT, bool W> using MGChunkT = typename std::conditional<W, MGChunkW<VT>, MGChunk<VT>>::type;

template <class VT, class ST, bool IN, bool DI, bool W = false>
__device__ __forceinline__ void mg_load(const MGLevel<VT, ST>& L, const VT* in, int it, MGChunkT<VT, W>& C) {
    const int j = 1 + it / L.cpr, c = it - (j - 1) * L.cpr;
    const size_t base = (size_t)j * L.ld + 4 * c;
    Vec4<VT>::load(L.b + base, C.b4);
    if (DI) SmemLoad<ST, VT>::load4(L.di + base, C.d4);    // levels may live in shared memory
    if (IN) {
        if constexpr (W) {
            we_row(L.we, L.ld, j, c, C.we);
            wn_row(L.wn, L.ld, j - 1, c, C.ws);
            wn_row(L.wn, L.ld, j, c, C.wn);
        } else {
            load_coef_chunk_any<ST, VT>(L.a, L.ld, L.n, j, c, C.a3);
        }
        load_vec_chunk<VT>(in, L.ld, L.n, j, c, C.xs, C.xc, C.xn);
    }
}

template <class VT>
__device__ __forceinline__ void mg_apply(const MGChunk<VT>& C, int n, int c, VT y[4]) {
    apply_chunk<VT>(C.a3, C.xs, C.xc, C.xn, n, c, y);
}
template <class VT>
__device__ __forceinline__ void mg_apply(const MGChunkW<VT>& C, int n, int c, VT y[4]) {
    apply_rows_w<VT>(C.we, C.ws, C.wn, C.xs, C.xc, C.xn, n, c, y);
}

// Smoothing step on one loaded chunk: out = in + w D^-1 (b - A in); returns (b, out) when RZ.
template <class VT, class ST, bool IN, bool RZ, bool W = false>
__device__ __forceinline__ VT mg_smooth_store(const MGLevel<VT, ST>& L, VT* out, int it, const MGChunkT<VT, W>& C,
                                              VT w) {
    const int j = 1 + it / L.cpr, c = it - (j - 1) * L.cpr;
    VT y[4] = {(VT)0, (VT)0, (VT)0, (VT)0}, x4[4] = {(VT)0, (VT)0, (VT)0, (VT)0};
    if (IN) {
        mg_apply<VT>(C, L.n, c, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) x4[q] = C.xc[q + 1];
    }
    VT o4[4], acc = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) o4[q] = fma_rn(mul_rn(w, C.d4[q]), C.b4[q] - y[q], x4[q]);
    Vec4<VT>::store(out + (size_t)j * L.ld + 4 * c, o4);
    if (RZ) {
#pragma unroll
        for (int q = 0; q < 4; ++q) acc += C.b4[q] * o4[q];
    }
    return acc;
}

// out = in + w D^-1 (b - A in) (in == nullptr: out = w D^-1 b); returns this
// thread's part of (b, out) when RZ.
template <class VT, class ST, int GT, bool RZ, bool W>
__device__ __forceinline__ VT mg_smooth_in(const Group<GT>& G, const MGLevel<VT, ST>& L, const VT* in, VT* out,
                                           VT w, int items) {
    VT acc = 0;
    for (int it0 = G.rank; it0 < items; it0 += 2 * GT) {
        const bool two = it0 + GT < items;
        const int it1 = two ? it0 + GT : it0;     // a second valid chunk, or a repeat that is not stored
        MGChunkT<VT, W> c0, c1;
        mg_load<VT, ST, true, true, W>(L, in, it0, c0);
        mg_load<VT, ST, true, true, W>(L, in, it1, c1);
        acc += mg_smooth_store<VT, ST, true, RZ, W>(L, out, it0, c0, w);
        if (two) acc += mg_smooth_store<VT, ST, true, RZ, W>(L, out, it1, c1, w);
    }
    return acc;
}

template <class VT, class ST, int GT, bool RZ>
__device__ __forceinline__ VT mg_smooth(const Group<GT>& G, const MGLevel<VT, ST>& L, const VT* in, VT* out, VT w) {
    const int items = (L.n - 1) * L.cpr;
    VT acc = 0;
    if constexpr (sizeof(VT) == 8 && sizeof(ST) == 8) {
        if (in && L.we) {
            acc = mg_smooth_in<VT, ST, GT, RZ, true>(G, L, in, out, w, items);
            G.sync();
            return acc;
        }
    }
    for (int it0 = G.rank; it0 < items; it0 += 2 * GT) {
        const bool two = it0 + GT < items;
        const int it1 = two ? it0 + GT : it0;     // a second valid chunk, or a repeat that is not stored
        MGChunk<VT> c0, c1;
        if (in) {
            mg_load<VT, ST, true, true>(L, in, it0, c0);
            mg_load<VT, ST, true, true>(L, in, it1, c1);
            acc += mg_smooth_store<VT, ST, true, RZ>(L, out, it0, c0, w);
            if (two) acc += mg_smooth_store<VT, ST, true, RZ>(L, out, it1, c1, w);
        } else {
            mg_load<VT, ST, false, true>(L, in, it0, c0);
            mg_load<VT, ST, false, true>(L, in, it1, c1);
            acc += mg_smooth_store<VT, ST, false, RZ>(L, out, it0, c0, w);
            if (two) acc += mg_smooth_store<VT, ST, false, RZ>(L, out, it1, c1, w);
        }
    }
    G.sync();
    return acc;
}

// t = b - A x on level L.
template <class VT, class ST, int GT, bool W>
__device__ __forceinline__ void mg_residual_pass(const Group<GT>& G, const MGLevel<VT, ST>& L) {
    const int items = (L.n - 1) * L.cpr;
    auto finish = [&](int it, const MGChunkT<VT, W>& C) {
        const int j = 1 + it / L.cpr, c = it - (j - 1) * L.cpr;
        VT y[4], r4[4];
        mg_apply<VT>(C, L.n, c, y);
#pragma unroll
        for (int q = 0; q < 4; ++q) r4[q] = C.b4[q] - y[q];
        Vec4<VT>::store(L.t + (size_t)j * L.ld + 4 * c, r4);
    };
    for (int it0 = G.rank; it0 < items; it0 += 2 * GT) {
        const bool two = it0 + GT < items;
        const int it1 = two ? it0 + GT : it0;
        MGChunkT<VT, W> c0, c1;
        mg_load<VT, ST, true, false, W>(L, L.x, it0, c0);
        mg_load<VT, ST, true, false, W>(L, L.x, it1, c1);
        finish(it0, c0);
        if (two) finish(it1, c1);
    }
}

template <class VT, class ST, int GT>
__device__ __forceinline__ void mg_residual(const Group<GT>& G, const MGLevel<VT, ST>& L) {
    if constexpr (sizeof(VT) == 8 && sizeof(ST) == 8) {
        if (L.we) mg_residual_pass<VT, ST, GT, true>(G, L);
        else mg_residual_pass<VT, ST, GT, false>(G, L);
    } else {
        mg_residual_pass<VT, ST, GT, false>(G, L);
    }
    G.sync();
}

// Coarse right-hand side C.b = P^T F.t: each interior coarse node gathers its
// fine node and half of its six P1 neighbours (E, W, N, S, NE, SW).
template <class VT, class ST, int GT>
__device__ __forceinline__ void mg_restrict(const Group<GT>& G, const MGLevel<VT, ST>& F, const MGLevel<VT, ST>& C) {
    const int nc = C.n, items = (nc - 1) * C.cpr;
    const VT half = (VT)0.5;
    for (int it = G.rank; it < items; it += GT) {
        const int J = 1 + it / C.cpr, Cc = it - (J - 1) * C.cpr;
        // fine rows 2J-1 .. 2J+1, columns 8Cc-1 .. 8Cc+7: two aligned 4-wide loads and one halo
        // value per row (columns past n are padding, which stays zero, and lie within the row pitch)
        VT v[3][9];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const VT* row = F.t + (size_t)(2 * J - 1 + r) * F.ld + 8 * Cc;
            Vec4<VT>::load(row, &v[r][1]);
            Vec4<VT>::load(row + 4, &v[r][5]);
            v[r][0] = Cc > 0 ? row[-1] : (VT)0;
        }
        VT o4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int I = 4 * Cc + q, m = 2 * q + 1;
            const VT nb = v[1][m + 1] + v[1][m - 1] + v[2][m] + v[0][m] + v[2][m + 1] + v[0][m - 1];
            o4[q] = (I >= 1 && I <= nc - 1) ? fma_rn(half, nb, v[1][m]) : (VT)0;
        }
        Vec4<VT>::store(C.b + (size_t)J * C.ld + 4 * Cc, o4);
    }
    G.sync();
}

// out = F.x + P C.x on the interior of level F (out may be F.x).
template <class VT, class ST, int GT>
__device__ __forceinline__ void mg_prolong(const Group<GT>& G, const MGLevel<VT, ST>& C, const MGLevel<VT, ST>& F,
                                           VT* out) {
    const int n = F.n, cpr = F.cpr, items = (n - 1) * cpr;
    const VT half = (VT)0.5;
    for (int it = G.rank; it < items; it += GT) {
        const int j = 1 + it / cpr, c = it - (j - 1) * cpr;
        const size_t base = (size_t)j * F.ld + 4 * c;
        const int Ja = j >> 1, Jb = (j + 1) >> 1;      // equal for even j
        VT ca[3], cb[3];                               // coarse columns 2c .. 2c+2 of rows Ja and Jb
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int col = 2 * c + m;
            ca[m] = col <= C.n ? C.x[(size_t)Ja * C.ld + col] : (VT)0;
            cb[m] = col <= C.n ? C.x[(size_t)Jb * C.ld + col] : (VT)0;
        }
        const bool odd = (j & 1) != 0;
        VT pv[4];
        // even columns 4c, 4c+2 take (2c, 2c+1); odd columns take their SW and NE (odd row) or W and E ends
        pv[0] = odd ? half * (ca[0] + cb[0]) : ca[0];
        pv[1] = odd ? half * (ca[0] + cb[1]) : half * (ca[0] + ca[1]);
        pv[2] = odd ? half * (ca[1] + cb[1]) : ca[1];
        pv[3] = odd ? half * (ca[1] + cb[2]) : half * (ca[1] + ca[2]);
        VT x4[4];
        Vec4<VT>::load(F.x + base, x4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 4 * c + q;
            x4[q] = (i >= 1 && i <= n - 1) ? x4[q] + pv[q] : x4[q];
        }
        Vec4<VT>::store(out + base, x4);
    }
    G.sync();
}

// nu sweeps from zero, alternating t and x so that the last lands in x.
template <class VT, class ST, int GT>
__device__ __forceinline__ void mg_sweeps_from_zero(const Group<GT>& G, const MGLevel<VT, ST>& L, int nu, VT w) {
    const VT* in = nullptr;
    for (int s = 1; s <= nu; ++s) {
        VT* out = ((nu - s) % 2 == 0) ? L.x : L.t;
        mg_smooth<VT, ST, GT, false>(G, L, in, out, w);
        in = out;
    }
}

// z = B r; returns this thread's part of (r, z).
template <class VT, class ST, int GT>
__device__ VT mg_vcycle(const Params& P, const DevSolve& S, const Group<GT>& G, VT* Z, VT* T, const VT* R,
                        const ST* AS, const ST* DI, uint8_t* cs) {
    const int nl = S.mg_levels, nu = P.mg_nu;
    const VT w = (VT)P.mg_omega;
    for (int k = 0; k < nl; ++k) {
        const MGLevel<VT, ST> L = mg_level<VT, ST>(P, S, k, Z, T, R, AS, DI, cs);
        mg_sweeps_from_zero<VT, ST, GT>(G, L, nu, w);
        mg_residual<VT, ST, GT>(G, L);
        mg_restrict<VT, ST, GT>(G, L, mg_level<VT, ST>(P, S, k + 1, Z, T, R, AS, DI, cs));
    }
    mg_sweeps_from_zero<VT, ST, GT>(G, mg_level<VT, ST>(P, S, nl, Z, T, R, AS, DI, cs), P.mg_coarse, w);
    VT rz = 0;
    for (int k = nl - 1; k >= 0; --k) {
        const MGLevel<VT, ST> L = mg_level<VT, ST>(P, S, k, Z, T, R, AS, DI, cs);
        // corrected iterate into t for odd nu, in place for even nu, so that nu sweeps end in x
        VT* corr = (nu % 2) ? L.t : L.x;
        mg_prolong<VT, ST, GT>(G, mg_level<VT, ST>(P, S, k + 1, Z, T, R, AS, DI, cs), L, corr);
        const VT* in = corr;
        for (int s = 1; s <= nu; ++s) {
            VT* out = ((nu - s) % 2 == 0) ? L.x : L.t;
            if (k == 0 && s == nu)
                rz = mg_smooth<VT, ST, GT, true>(G, L, in, out, w);
            else
                mg_smooth<VT, ST, GT, false>(G, L, in, out, w);
            in = out;
        }
    }
    if (nl == 0) {
        // no coarse grid: the coarsest sweeps ran on the fine grid itself; (r, z) separately
        const MGLevel<VT, ST> L = mg_level<VT, ST>(P, S, 0, Z, T, R, AS, DI, cs);
        const int n = L.n, ld = L.ld, cpr = L.cpr, items = (n - 1) * cpr;
        for (int it = G.rank; it < items; it += GT) {
            const int j = 1 + it / cpr, c = it - (j - 1) * cpr;
            const size_t base = (size_t)j * ld + 4 * c;
            VT b4[4], z4[4];
            Vec4<VT>::load(R + base, b4);
            Vec4<VT>::load(Z + base, z4);
#pragma unroll
            for (int q = 0; q < 4; ++q) rz += b4[q] * z4[q];
        }
    }
    return rz;
}

// v = 0 on the interior chunks of level L.
template <class VT, class ST, int GT>
__device__ __forceinline__ void mg_zero(const Group<GT>& G, const MGLevel<VT, ST>& L, VT* v) {
    const int items = (L.n - 1) * L.cpr;
    const VT z[4] = {(VT)0, (VT)0, (VT)0, (VT)0};
    for (int it = G.rank; it < items; it += GT) {
        const int j = 1 + it / L.cpr, c = it - (j - 1) * L.cpr;
        Vec4<VT>::store(v + (size_t)j * L.ld + 4 * c, z);
    }
    G.sync();
}

// Full-multigrid guess for A d = r (d = 0 on entry): r restricted down the hierarchy, the coarsest grid
// smoothed from zero, then on each finer grid the prolonged coarser solution improved by one V-cycle (nu
// sweeps, coarse correction from zero, nu sweeps).  Leaves d in D and r - A d in R.  Level 0 of this
// hierarchy is (x D, scratch T, right-hand side R); the coarse levels are the V-cycle's.
// (Not inlined: its own register allocation leaves the solve's sweep loops as they are.)
template <class VT, class ST, int GT>
__device__ __noinline__ void mg_fmg(const Params& P, const DevSolve& S, const Group<GT>& G, VT* D, VT* T, VT* R,
                                    const ST* AS, const ST* DI, uint8_t* cs) {
    const int nl = S.mg_levels, nu = P.mg_nu;
    const VT w = (VT)P.mg_omega;
    for (int k = 0; k < nl; ++k) {
        MGLevel<VT, ST> F = mg_level<VT, ST>(P, S, k, D, T, R, AS, DI, cs);
        F.t = F.b;   // restrict the right-hand side itself
        mg_restrict<VT, ST, GT>(G, F, mg_level<VT, ST>(P, S, k + 1, D, T, R, AS, DI, cs));
    }
    mg_sweeps_from_zero<VT, ST, GT>(G, mg_level<VT, ST>(P, S, nl, D, T, R, AS, DI, cs), P.mg_coarse, w);
    for (int k = nl - 1; k >= 0; --k) {
        MGLevel<VT, ST> L = mg_level<VT, ST>(P, S, k, D, T, R, AS, DI, cs);
        if (k > 0) mg_zero<VT, ST, GT>(G, L, L.x);
        mg_prolong<VT, ST, GT>(G, mg_level<VT, ST>(P, S, k + 1, D, T, R, AS, DI, cs), L, L.x);
        // nu sweeps from the prolonged guess, alternating x and t (the iterate is in L.x after each pair)
        for (int s = 0; s < nu; ++s) {
            mg_smooth<VT, ST, GT, false>(G, L, L.x, L.t, w);
            VT* q = L.x;
            L.x = L.t;
            L.t = q;
        }
        mg_residual<VT, ST, GT>(G, L);
        mg_restrict<VT, ST, GT>(G, L, mg_level<VT, ST>(P, S, k + 1, D, T, R, AS, DI, cs));
        // coarse correction from zero on levels k + 1 .. nl (the V-cycle's descent and ascent)
        for (int j = k + 1; j < nl; ++j) {
            const MGLevel<VT, ST> C = mg_level<VT, ST>(P, S, j, D, T, R, AS, DI, cs);
            mg_sweeps_from_zero<VT, ST, GT>(G, C, nu, w);
            mg_residual<VT, ST, GT>(G, C);
            mg_restrict<VT, ST, GT>(G, C, mg_level<VT, ST>(P, S, j + 1, D, T, R, AS, DI, cs));
        }
        mg_sweeps_from_zero<VT, ST, GT>(G, mg_level<VT, ST>(P, S, nl, D, T, R, AS, DI, cs), P.mg_coarse, w);
        for (int j = nl - 1; j > k; --j) {
            const MGLevel<VT, ST> C = mg_level<VT, ST>(P, S, j, D, T, R, AS, DI, cs);
            VT* corr = (nu % 2) ? C.t : C.x;
            mg_prolong<VT, ST, GT>(G, mg_level<VT, ST>(P, S, j + 1, D, T, R, AS, DI, cs), C, corr);
            const VT* in = corr;
            for (int s = 1; s <= nu; ++s) {
                VT* out = ((nu - s) % 2 == 0) ? C.x : C.t;
                mg_smooth<VT, ST, GT, false>(G, C, in, out, w);
                in = out;
            }
        }
        mg_prolong<VT, ST, GT>(G, mg_level<VT, ST>(P, S, k + 1, D, T, R, AS, DI, cs), L, L.x);
        for (int s = 0; s < nu; ++s) {
            mg_smooth<VT, ST, GT, false>(G, L, L.x, L.t, w);
            VT* q = L.x;
            L.x = L.t;
            L.t = q;
        }
    }
    // r = r - A d (in place: each chunk reads its own r before writing it)
    MGLevel<VT, ST> L0 = mg_level<VT, ST>(P, S, 0, D, T, R, AS, DI, cs);
    L0.t = L0.b;
    mg_residual<VT, ST, GT>(G, L0);
}

// One system, start to finish: set-up, refinement loop with the inner PCG, QoI.
// `pipe` is non-null for a 512-thread CG group whose sweeps stream rows
// through shared memory.
template <class VT, class ST, int SOLVER, int GT>
__device__ void solve_system(const Params& P, const DevSolve& S, const Group<GT>& G, Pipe* pipe, uint8_t* cs) {
    const int n = S.n, ld = S.ld, cpr = S.cpr;
    const int items = (n - 1) * cpr;
    const int tr = G.rank;
    double* X = P.x64 + S.off;
    VT* R = static_cast<VT*>(P.r) + S.off;
    VT* PB0 = static_cast<VT*>(P.p0) + S.off;
    VT* PB1 = static_cast<VT*>(P.p1) + S.off;
    VT* D = static_cast<VT*>(P.d) + S.off;
    ST* AS = static_cast<ST*>(P.as) + S.off;
    ST* DI = static_cast<ST*>(P.dinv) + S.off;
    const bool jac = P.jacobi != 0;
    constexpr bool minres = SOLVER == MLMC_MINRES;
    // the FP64 inner solve applies its grid operator from the stored FP64 edge weights
    constexpr bool W64 = sizeof(VT) == 8 && sizeof(ST) == 8;
    const bool pipe_on = pipe != nullptr;
    VT* VB = minres ? static_cast<VT*>(P.vb) + S.off : nullptr;
    VT* W0 = minres ? static_cast<VT*>(P.w0) + S.off : nullptr;
    VT* W1 = minres ? static_cast<VT*>(P.w1) + S.off : nullptr;
    VT* MZ = P.mg ? static_cast<VT*>(P.mz) + S.off : nullptr;
    VT* MT = P.mg ? static_cast<VT*>(P.mt) + S.off : nullptr;
    // row-sweep mapping: GT / cpr row segments, each thread one chunk column of one segment
    const int nseg = max(1, GT / cpr);
    const int seg_rows = (n - 1 + nseg - 1) / nseg;
    const int sc = tr % cpr, seg = tr / cpr;
    const int ja = 1 + seg * seg_rows, jb = min(n, ja + seg_rows);
    const bool sweep_on = seg < nseg && ja < jb;

    // ---- set-up: coefficient (and inverse diagonal) in the inner storage precision, on the
    // grid and, with multigrid, on every coarse level (coefficient injected at the coarse nodes)
    const bool mg = P.mg != 0;
    const bool need_di = jac || mg;
    for (int it = tr; it < (n + 1) * (n + 1); it += GT) {
        const int j = it / (n + 1), i = it - j * (n + 1);
        AS[(size_t)j * ld + i] = store_from<ST, VT>(master_a_as<VT>(S, i, j));
        if (need_di && i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1)
            DI[(size_t)j * ld + i] = store_from<ST, VT>(stencil_inv_diag<VT>(S, i, j, 0));
    }
    // FP64 edge weights of the master operator (6 wE, 6 wN), formed once and reused by every
    // refinement residual: WE(i,j) = 2 (a(i,j) + a(i+1,j)) + a(i+1,j+1) + a(i,j-1) on the edge
    // (i,j)-(i+1,j), WN(i,j) = 2 (a(i,j) + a(i,j+1)) + a(i+1,j+1) + a(i-1,j) on (i,j)-(i,j+1).
    {
        double* WE = P.we + S.off;
        double* WN = P.wn + S.off;
        for (int it = tr; it < (n + 1) * (n + 1); it += GT) {
            const int j = it / (n + 1), i = it - j * (n + 1);
            double we = 0.0, wn = 0.0;
            if (i <= n - 1 && j >= 1 && j <= n - 1)
                we = 2.0 * (master_a(S, i, j) + master_a(S, i + 1, j)) + master_a(S, i + 1, j + 1) +
                     master_a(S, i, j - 1);
            if (j <= n - 1 && i >= 1 && i <= n - 1)
                wn = 2.0 * (master_a(S, i, j) + master_a(S, i, j + 1)) + master_a(S, i + 1, j + 1) +
                     master_a(S, i - 1, j);
            WE[(size_t)j * ld + i] = we;
            WN[(size_t)j * ld + i] = wn;
        }
    }
    if (mg) {
        if (cs) {
            // shared-memory levels start at zero (boundary and padding entries stay zero)
            const int bytes = mg_smem_bytes(n, S.mg_levels, P.mg_smem_nmax, (int)sizeof(VT), (int)sizeof(ST),
                                            S.mg_levels + 1);
            for (int i = tr; i < bytes / 16; i += GT) reinterpret_cast<uint4*>(cs)[i] = make_uint4(0, 0, 0, 0);
            G.sync();
        }
        for (int k = 1; k <= S.mg_levels; ++k) {
            const int nk = n >> k, ldk = row_pitch(nk);
            const MGLevel<VT, ST> Lk = mg_level<VT, ST>(P, S, k, nullptr, nullptr, nullptr, AS, DI, cs);
            ST* ca = const_cast<ST*>(Lk.a);
            ST* cd = const_cast<ST*>(Lk.di);
            for (int it = tr; it < (nk + 1) * (nk + 1); it += GT) {
                const int J = it / (nk + 1), I = it - J * (nk + 1);
                ca[(size_t)J * ldk + I] = store_from<ST, VT>(master_a_as<VT>(S, I << k, J << k));
                if (I >= 1 && I <= nk - 1 && J >= 1 && J <= nk - 1)
                    cd[(size_t)J * ldk + I] = store_from<ST, VT>(stencil_inv_diag<VT>(S, I << k, J << k, k));
            }
        }
    }
    if (pipe_on) fence_proxy_async_global();
    G.sync();

    double rho = 0.0, rho_prev = 0.0;
    int iters = 0, flag = 0, o = 0;
    // right-hand side b_i = f h^2 (or the adjoint's g_i), formed once
    const bool rhs_mode0 = S.rhs_mode == 0;
    const double b0 = S.f * S.h2;
    for (;; ++o) {
        // ---- R: r = b - A x in FP64 with the master coefficient (r = b while x = 0); d = 0
        // the FP64 residual norm decides the refinement; the inner solve's starting (r, r) and (r, z) are
        // the inner type's, summed like the sweeps' (and summed across the group in FP64)
        double res = 0.0;
        VT rr0v = 0, rz0v = 0;
        for (int it = tr; it < items; it += GT) {
            const int j = 1 + it / cpr, c = it - (j - 1) * cpr;
            const size_t base = (size_t)j * ld + 4 * c;
            VT rv[4], zv[4];
            if (jac) CoefLoad<ST, VT>::load4(DI + base, zv);
            double r4[4];
            if (o == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 4 * c + q;
                    r4[q] = (i >= 1 && i <= n - 1) ? (rhs_mode0 ? b0 : rhs_value(S, i, j)) : 0.0;
                }
            } else {
                // (A x)_ij = (WE(i,j)(x - x_E) + WE(i-1,j)(x - x_W) + WN(i,j)(x - x_N) + WN(i,j-1)(x - x_S)) / 6
                const double* WE = P.we + S.off;
                const double* WN = P.wn + S.off;
                double xs[4], xc[6], xn[4], we[5], wn[4], ws[4];
                load_vec_chunk<double>(X, ld, n, j, c, xs, xc, xn);
                Vec4<double>::load(WE + base, &we[1]);
                we[0] = c > 0 ? WE[base - 1] : 0.0;
                Vec4<double>::load(WN + base, wn);
                Vec4<double>::load(WN + base - ld, ws);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 4 * c + q;
                    const double x0 = xc[q + 1];
                    const double ax = (we[q + 1] * (x0 - xc[q + 2]) + we[q] * (x0 - xc[q]) + wn[q] * (x0 - xn[q]) +
                                       ws[q] * (x0 - xs[q])) * (1.0 / 6.0);
                    r4[q] = (i >= 1 && i <= n - 1) ? (rhs_mode0 ? b0 : rhs_value(S, i, j)) - ax : 0.0;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double rq = r4[q];
                rv[q] = (VT)rq;
                res += rq * rq;
                rr0v += rv[q] * rv[q];
                rz0v += jac ? rv[q] * (rv[q] * zv[q]) : rv[q] * rv[q];
            }
            Vec4<VT>::store(R + base, rv);
            const VT z[4] = {(VT)0, (VT)0, (VT)0, (VT)0};
            Vec4<VT>::store(D + base, z);
            if (minres) {
                // v_1 = r (in R), z_1 = D^-1 v_1 (in PB0), v_0 = w_0 = w_1 = 0
                VT z1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) z1[q] = jac ? rv[q] * zv[q] : rv[q];
                Vec4<VT>::store(PB0 + base, z1);
                Vec4<VT>::store(VB + base, z);
                Vec4<VT>::store(W0 + base, z);
                Vec4<VT>::store(W1 + base, z);
            }
        }
        if (pipe_on) fence_proxy_async_global();
        double rr0, rz0;
        {
            double a0, b0s, c0s;
            G.template sum3<double>(res, (double)rr0v, (double)rz0v, a0, b0s, c0s);
            res = a0;
            rr0 = b0s;
            rz0 = c0s;
        }
        rho = sqrt(res) / S.bnorm;
        if (pipe_on && pipe_aborted(*pipe)) { flag = MLMC_F_TIMEOUT; break; }
        if (!(rho == rho) || isinf(rho)) { flag = MLMC_F_NONFINITE; break; }
        if (rho < S.delta) { flag = MLMC_F_CONVERGED; break; }
        if (o >= P.max_outer || iters >= P.max_iters) { flag = MLMC_F_MAXIT; break; }
        if (o >= 1 && rho > P.stag * rho_prev) { flag = MLMC_F_STAGNATED; break; }
        rho_prev = rho;
        const double tau = inner_tau(P, S, rho);
        if constexpr (!minres) {
            // the first inner solve starts from a full-multigrid guess (d and r replaced)
            if (mg && P.fmg && o == 0 && S.mg_levels > 0) {
                mg_fmg<VT, ST, GT>(P, S, G, D, MT, R, AS, DI, cs);
                if (pipe_on) fence_proxy_async_global();
            }
        }

        int k = 0;
        if (minres) {
            // ---- inner preconditioned MINRES on A d = r; |eta| is ||r_k|| in the M^-1 norm, with
            // M^-1 = D^-1 (Jacobi) or the V-cycle B (multigrid, z_1 = B v_1 here and z_j+1 = B v_j+1
            // after sweep B); the V-cycle is symmetric positive definite, as MINRES needs
            if (mg) {
                const VT zp = mg_vcycle<VT, ST, GT>(P, S, G, PB0, MT, R, AS, DI, cs);
                double zz, u1, u2;
                G.template sum3<VT>(zp, (VT)0, (VT)0, zz, u1, u2);
                rz0 = zz;
            }
            double g0 = 1.0, g1 = sqrt(rz0), c0 = 1.0, c1 = 1.0, s0 = 0.0, s1 = 0.0;
            double eta = g1;
            const double eta0 = g1;
            VT *Vp = VB, *Vc = R, *Zc = PB0, *Zn = PB1, *Wo = W0, *Wn = W1;
            bool pend = false;
            VT pa1i = 0, pa2 = 0, pa3 = 0, pcst = 0, pgi = 0;
            while ((eta == eta) && !isinf(eta) && fabs(eta) > tau * eta0 && eta0 > 0.0 && iters + k < P.max_iters) {
                const VT gci = (VT)(1.0 / g1);
                VT dlp = 0;
                if (sweep_on)
                    dlp = pend ? sweep_minres_a<VT, ST, true>(Zc, gci, AS, ld, n, sc, ja, jb, Zn, pgi, Wo, Wn, D, pa1i,
                                                              pa2, pa3, pcst)
                               : sweep_minres_a<VT, ST, false>(Zc, gci, AS, ld, n, sc, ja, jb, Zn, pgi, Wo, Wn, D,
                                                               pa1i, pa2, pa3, pcst);
                double dl, t1, t2;
                G.template sum3<VT>(dlp, (VT)0, (VT)0, dl, t1, t2);
                if (pend) {
                    VT* tw = Wo;
                    Wo = Wn;
                    Wn = tw;
                }
                VT zvp = 0;
                const VT cA = (VT)(dl / g1), cB = (VT)(g1 / g0);
                if (sweep_on) {
                    if (jac && !mg)
                        zvp = sweep_minres_b<VT, ST, true>(Zc, gci, AS, Vp, Vc, DI, Zn, cA, cB, ld, n, sc, ja, jb);
                    else
                        zvp = sweep_minres_b<VT, ST, false>(Zc, gci, AS, Vp, Vc, DI, Zn, cA, cB, ld, n, sc, ja, jb);
                }
                if (mg) {
                    // z_j+1 = B v_j+1 and (v_j+1, z_j+1)
                    G.sync();
                    zvp = mg_vcycle<VT, ST, GT>(P, S, G, Zn, MT, Vp, AS, DI, cs);
                }
                double zv, t3, t4;
                G.template sum3<VT>(zvp, (VT)0, (VT)0, zv, t3, t4);
                const double g2 = sqrt(fmax(zv, 0.0));
                const double al0 = c1 * dl - c0 * s1 * g1;
                const double al1 = sqrt(al0 * al0 + g2 * g2);
                const double al2 = s1 * dl + c0 * c1 * g1;
                const double al3 = s0 * g1;
                const double c2 = al0 / al1, s2 = g2 / al1;
                pend = true;
                pa1i = (VT)(1.0 / al1);
                pa2 = (VT)al2;
                pa3 = (VT)al3;
                pcst = (VT)(c2 * eta);
                pgi = gci;
                eta = -s2 * eta;
                c0 = c1; c1 = c2; s0 = s1; s1 = s2; g0 = g1; g1 = g2;
                VT* tv = Vp; Vp = Vc; Vc = tv;
                VT* tz = Zc; Zc = Zn; Zn = tz;
                ++k;
                if (g2 == 0.0) break;
            }
            if (pend) {
                for (int it = tr; it < items; it += GT) {
                    const int j = 1 + it / cpr, c = it - (j - 1) * cpr;
                    minres_update_chunk<VT>(Zn, pgi, Wo, Wn, D, pa1i, pa2, pa3, pcst, (size_t)j * ld + 4 * c);
                }
                G.sync();
            }
        } else {
            // ---- inner PCG on A d = r: z = D^-1 r (Jacobi), z = B r (multigrid V-cycle) or z = r.
            // The scalars are formed once per reduction from the FP64 group sums and broadcast.
            const double tau2rr0 = tau * tau * rr0;
            double rzk = rz0;              // (r, z) of the current residual, kept where the scalars are formed
            VT beta = 0;
            const bool dj = jac && !mg;    // the sweeps form z = D^-1 r themselves
            const VT* zsrc = mg ? MZ : R;
            bool cont = (rr0 == rr0) && !isinf(rr0) && rr0 > tau2rr0 && rr0 != 0.0 && iters < P.max_iters;
            while (cont) {
                const VT* pold = (k & 1) ? PB0 : PB1;
                VT* pnew = (k & 1) ? PB1 : PB0;
                if (mg) {
                    // z = B r and (r, z); beta = (r, z) / (r, z)_previous
                    const VT rzp = mg_vcycle<VT, ST, GT>(P, S, G, MZ, MT, R, AS, DI, cs);
                    VT sc0[4];
                    const int k0 = k;
                    G.template reduce<VT, VT>(rzp, (VT)0, (VT)0,
                                              [&](double rz, double, double, double* r) {
                                                  r[0] = k0 > 0 ? rz / rzk : 0.0;
                                                  rzk = rz;
                                              },
                                              sc0);
                    beta = sc0[0];
                }
                // I1: p = z + beta p_old on the segment rows (recomputed on the halo rows); sigma = (p, A p)
                VT sig = 0;
                if (sweep_on) {
                    if (pipe_on) {
                        if (dj)
                            sig = (k > 0) ? sweep_dir_staged<VT, ST, true, true>(*pipe, zsrc, DI, pold, pnew, AS, beta,
                                                                                 ld, n, sc, ja, jb)
                                          : sweep_dir_staged<VT, ST, true, false>(*pipe, zsrc, DI, pold, pnew, AS,
                                                                                  beta, ld, n, sc, ja, jb);
                        else
                            sig = (k > 0) ? sweep_dir_staged<VT, ST, false, true>(*pipe, zsrc, DI, pold, pnew, AS,
                                                                                  beta, ld, n, sc, ja, jb)
                                          : sweep_dir_staged<VT, ST, false, false>(*pipe, zsrc, DI, pold, pnew, AS,
                                                                                   beta, ld, n, sc, ja, jb);
                    } else if constexpr (W64) {
                        const double* WE = P.we + S.off;
                        const double* WN = P.wn + S.off;
                        if (dj)
                            sig = (k > 0) ? sweep_dir_w<VT, ST, true, true>(zsrc, DI, pold, pnew, WE, WN, beta, ld, n,
                                                                            sc, ja, jb)
                                          : sweep_dir_w<VT, ST, true, false>(zsrc, DI, pold, pnew, WE, WN, beta, ld,
                                                                             n, sc, ja, jb);
                        else
                            sig = (k > 0) ? sweep_dir_w<VT, ST, false, true>(zsrc, DI, pold, pnew, WE, WN, beta, ld,
                                                                             n, sc, ja, jb)
                                          : sweep_dir_w<VT, ST, false, false>(zsrc, DI, pold, pnew, WE, WN, beta, ld,
                                                                              n, sc, ja, jb);
                    } else {
                        if (dj)
                            sig = (k > 0) ? sweep_dir<VT, ST, true, true>(zsrc, DI, pold, pnew, AS, beta, ld, n, sc,
                                                                          ja, jb)
                                          : sweep_dir<VT, ST, true, false>(zsrc, DI, pold, pnew, AS, beta, ld, n, sc,
                                                                           ja, jb);
                        else
                            sig = (k > 0) ? sweep_dir<VT, ST, false, true>(zsrc, DI, pold, pnew, AS, beta, ld, n, sc,
                                                                           ja, jb)
                                          : sweep_dir<VT, ST, false, false>(zsrc, DI, pold, pnew, AS, beta, ld, n,
                                                                            sc, ja, jb);
                    }
                }
                VT sc1[4];
                G.template reduce<VT, VT>(sig, (VT)0, (VT)0,
                                          [&](double sg, double, double, double* r) { r[0] = rzk / sg; }, sc1);
                const VT alpha = sc1[0];
                // I2: d += alpha p; r -= alpha A p; ||r||^2 and, with Jacobi, (r, D^-1 r)
                VT nrr = 0, nrz = 0;
                if (sweep_on) {
                    if (pipe_on) {
                        if (dj)
                            sweep_upd_staged<VT, ST, true>(*pipe, pnew, R, D, DI, AS, alpha, ld, n, sc, ja, jb, nrr, nrz);
                        else
                            sweep_upd_staged<VT, ST, false>(*pipe, pnew, R, D, DI, AS, alpha, ld, n, sc, ja, jb, nrr,
                                                            nrz);
                    } else if constexpr (W64) {
                        const double* WE = P.we + S.off;
                        const double* WN = P.wn + S.off;
                        if (dj)
                            sweep_upd_w<VT, ST, true>(pnew, R, D, DI, WE, WN, alpha, ld, n, sc, ja, jb, nrr, nrz);
                        else
                            sweep_upd_w<VT, ST, false>(pnew, R, D, DI, WE, WN, alpha, ld, n, sc, ja, jb, nrr, nrz);
                    } else {
                        if (dj)
                            sweep_upd<VT, ST, true>(pnew, R, D, DI, AS, alpha, ld, n, sc, ja, jb, nrr, nrz);
                        else
                            sweep_upd<VT, ST, false>(pnew, R, D, DI, AS, alpha, ld, n, sc, ja, jb, nrr, nrz);
                    }
                }
                VT sc2[4];
                const int kk = k;
                G.template reduce<VT, VT>(nrr, nrz, (VT)0,
                                          [&](double rr, double rz, double, double* r) {
                                              const bool ab = pipe_on && pipe_aborted(*pipe);
                                              const bool go = (rr == rr) && !isinf(rr) && rr > tau2rr0 && rr != 0.0 &&
                                                              iters + kk + 1 < P.max_iters && !ab;
                                              if (!mg) {
                                                  r[0] = rz / rzk;
                                                  rzk = rz;
                                              }
                                              r[1] = go ? 1.0 : 0.0;
                                          },
                                          sc2);
                if (!mg) beta = sc2[0];
                cont = sc2[1] != (VT)0;
                ++k;
            }
        }
        iters += k;

        // ---- U: x += d in FP64
        for (int it = tr; it < items; it += GT) {
            const int j = 1 + it / cpr, c = it - (j - 1) * cpr;
            const size_t base = (size_t)j * ld + 4 * c;
            double xv[4];
            VT dvv[4];
            Vec4<double>::load(X + base, xv);
            Vec4<VT>::load(D + base, dvv);
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[q] += (double)dvv[q];
            Vec4<double>::store(X + base, xv);
        }
        G.sync();
    }

    // ---- Q: G(u) = sum g_i x_i; optional dense copy of u
    double qsum = 0.0;
    for (int it = tr; it < items; it += GT) {
        const int j = 1 + it / cpr, c = it - (j - 1) * cpr;
        double xv[4];
        Vec4<double>::load(X + (size_t)j * ld + 4 * c, xv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 4 * c + q;
            if (i >= 1 && i <= n - 1) qsum += qoi_weight(S, i, j) * xv[q];
        }
    }
    if (S.u) {
        double* u = S.u + (size_t)S.out * (n + 1) * (n + 1);
        for (int it = tr; it < (n + 1) * (n + 1); it += GT) {
            const int j = it / (n + 1), i = it - j * (n + 1);
            const bool inner = (i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1);
            u[it] = inner ? X[(size_t)j * ld + i] : 0.0;
        }
    }
    double qs, t4, t5;
    G.template sum3<double>(qsum, 0.0, 0.0, qs, t4, t5);
    if (tr == 0) {
        if (S.Q) S.Q[S.out] = qs;
        if (S.iters) S.iters[S.out] = iters;
        if (S.relres) S.relres[S.out] = rho;
        if (S.flags) S.flags[S.out] = flag;
        P.sys_iters[S.sys] = iters;
        P.sys_outer[S.sys] = o;
    }
}

// One launch for every system: CTA b < nbig solves one large system; the next
// ceil(nmed / 4) CTAs solve four medium systems each (128-thread groups); the
// rest solve sixteen small systems each (one warp each).  A large CG system
// streams its sweeps through the row pipeline when P.ring >= 2 (dynamic
// shared memory of pipe_smem_bytes).
template <class VT, class ST, int SOLVER>
__global__ void __launch_bounds__(CTA, 1) resident_solve(Params P) {
    extern __shared__ __align__(128) uint8_t dsm[];
    __shared__ double red[3 * (CTA / 32)];
    __shared__ double bcast[4 * (CTA / G_MED)];
    __shared__ int s_abort;
    const int b = blockIdx.x;
    const int nmed_cta = (P.nmed + 3) / 4;
    if (b < P.nbig) {
        const DevSolve& S = P.solves[P.order[b]];
        Group<G_BIG> G{(int)threadIdx.x, 0, red, bcast};
        if (SOLVER == MLMC_CG && P.ring >= 2 && S.cpr % 32 == 0) {
            const int cpr = S.cpr, nseg = pipe_nseg(S.n), ring = P.ring;
            uint64_t* bars = reinterpret_cast<uint64_t*>(dsm);
            if (threadIdx.x == 0) {
                s_abort = 0;
                for (int i = 0; i < ring * nseg; ++i) {
                    mbar_init(bars + i, 1);
                    mbar_init(bars + ring * nseg + i, (uint32_t)cpr);
                }
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            }
            __syncthreads();
            Pipe pipe;
            pipe.ring = ring;
            pipe.abort = &s_abort;
            pipe.err = P.err;
            pipe.timeout_ns = P.timeout_ns;
            pipe.extra_tx = P.extra_tx;
            const int seg = (int)threadIdx.x / cpr;
            if (seg < nseg) {
                pipe.slot_bytes = pipe_slot_bytes(S.ld, (int)sizeof(VT), (int)sizeof(ST));
                pipe.slots = dsm + pipe_bar_bytes(S.n, ring) + (size_t)seg * ring * pipe.slot_bytes;
                pipe.full = bars + seg * ring;
                pipe.empty = bars + ring * nseg + seg * ring;
                pipe.leader = ((int)threadIdx.x % cpr) == 0;
                pipe.lead_warp = ((int)threadIdx.x % cpr) < 32;
            }
            solve_system<VT, ST, SOLVER, G_BIG>(P, S, G, &pipe, P.mg_smem_nmax > 0 ? dsm + P.mg_smem_off : nullptr);
            if (pipe.leader && pipe_aborted(pipe)) pipe_drain(pipe);
            return;
        }
        solve_system<VT, ST, SOLVER, G_BIG>(P, S, G, nullptr, P.mg_smem_nmax > 0 ? dsm + P.mg_smem_off : nullptr);
        return;
    }
    if (b < P.nbig + nmed_cta) {
        const int gid = threadIdx.x / G_MED;
        const int idx = (b - P.nbig) * 4 + gid;
        if (idx >= P.nmed) return;
        Group<G_MED> G{(int)(threadIdx.x % G_MED), gid, red + gid * 3 * (G_MED / 32), bcast + 4 * gid};
        solve_system<VT, ST, SOLVER, G_MED>(P, P.solves[P.order[P.nbig + idx]], G, nullptr, nullptr);
        return;
    }
    const int gid = threadIdx.x / G_SMALL;
    const int idx = (b - P.nbig - nmed_cta) * (CTA / G_SMALL) + gid;
    if (idx >= P.nsmall) return;
    Group<G_SMALL> G{(int)(threadIdx.x % G_SMALL), gid, nullptr, nullptr};
    solve_system<VT, ST, SOLVER, G_SMALL>(P, P.solves[P.order[P.nbig + P.nmed + idx]], G, nullptr, nullptr);
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

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


// Algorithmic bytes of one V-cycle summed over the unknowns of every level:
// per unknown, a sweep from zero reads b and D^-1 and writes x (2 p_v + p_s),
// a sweep reads x, b, a, D^-1 and writes x (3 p_v + 2 p_s), the residual reads
// x, b, a and writes t (3 p_v + p_s), restriction reads t and writes the coarse
// b, prolongation reads the coarse x and x and writes x.
double mg_iter_bytes(int n, int nl, int nu, int ncs, double pv, double ps) {
    double bytes = 0.0;
    for (int k = 0; k <= nl; ++k) {
        const double u = (double)((n >> k) - 1) * ((n >> k) - 1);
        if (k < nl) {
            const double pre = (2 * pv + ps) + (nu - 1) * (3 * pv + 2 * ps), post = nu * (3 * pv + 2 * ps);
            const double uc = (double)((n >> (k + 1)) - 1) * ((n >> (k + 1)) - 1);
            bytes += u * (pre + (3 * pv + ps) + pv + 2 * pv + post) + uc * (2 * pv);
        } else {
            bytes += u * ((2 * pv + ps) + (ncs - 1) * (3 * pv + 2 * ps));
        }
    }
    return bytes;
}

// Arithmetic operations per interior unknown, as the kernels execute them: a stencil point from
// the nodal coefficient (four edge weights of 4 operations each, then 4 differences, 4 products,
// 3 sums and the 1/6 scaling) or from stored FP64 edge weights (the FP64 inner solve's grid level).
constexpr double kFlopStencil = 28.0, kFlopStencilW = 12.0;

// Operations of one V-cycle summed over the unknowns of every level: a smoothing sweep from zero
// 2 (omega D^-1 b), a later sweep a stencil plus 4 (b - A x, D^-1, omega, update), the residual a
// stencil plus 1, restriction 8 per coarse unknown (the fine node and half of six neighbours),
// prolongation 3 per fine unknown, and (r, z) on the grid 2.  The grid level uses stencil `s0`.
double mg_iter_flops(int n, int nl, int nu, int ncs, double s0) {
    double fl = 0.0;
    for (int k = 0; k <= nl; ++k) {
        const double u = (double)((n >> k) - 1) * ((n >> k) - 1);
        const double st = k == 0 ? s0 : kFlopStencil;
        if (k < nl) {
            const double uc = (double)((n >> (k + 1)) - 1) * ((n >> (k + 1)) - 1);
            fl += u * (2.0 + (nu - 1) * (st + 4.0) + (st + 1.0) + 3.0 + nu * (st + 4.0)) + uc * 8.0;
        } else {
            fl += u * (2.0 + (ncs - 1) * (st + 4.0));
        }
    }
    return fl + 2.0 * (double)(n - 1) * (n - 1);
}

// The full-multigrid start (mg_fmg), once per solve: the right-hand side restricted down the hierarchy
// (2 p_v per coarse unknown), the coarsest sweeps, and on each finer level k the guess cleared (k > 0) and
// prolonged (3 p_v per unknown) and a V-cycle of levels k .. nl from it (counted as one from zero), then
// the fine residual r - A d (3 p_v + p_s per unknown).
double mg_fmg_bytes(int n, int nl, int nu, int ncs, double pv, double ps) {
    auto unk = [&](int k) { return (double)((n >> k) - 1) * ((n >> k) - 1); };
    double b = unk(nl) * ((2 * pv + ps) + (ncs - 1) * (3 * pv + 2 * ps)) + unk(0) * (3 * pv + ps);
    for (int k = 0; k < nl; ++k)
        b += unk(k + 1) * 2 * pv + unk(k) * (k > 0 ? 3 : 2) * pv + mg_iter_bytes(n >> k, nl - k, nu, ncs, pv, ps);
    return b;
}
// Its operations: restriction 8 per coarse unknown, the coarsest sweeps, per finer level the prolongation
// (2 per unknown) and a V-cycle, and the fine residual (a stencil plus 1).
double mg_fmg_flops(int n, int nl, int nu, int ncs, double s0) {
    auto unk = [&](int k) { return (double)((n >> k) - 1) * ((n >> k) - 1); };
    double f = unk(nl) * (2.0 + (ncs - 1) * (kFlopStencil + 4.0)) + unk(0) * (s0 + 1.0);
    for (int k = 0; k < nl; ++k)
        f += unk(k + 1) * 8.0 + unk(k) * 2.0 + mg_iter_flops(n >> k, nl - k, nu, ncs, k == 0 ? s0 : kFlopStencil);
    return f;
}

// Workspace of a batch: vectors, coefficient storage, descriptors, launch order.
struct Layout {
    size_t o_x, o_r, o_p0, o_p1, o_d, o_as, o_dinv, o_vb, o_w0, o_w1, o_mz, o_mt, o_cx, o_ct, o_cb, o_cas, o_cdi,
        o_we, o_wn, o_stats, o_err, zero_end, o_solves, o_order, total;
};

template <class VT, class ST>
Layout make_layout(long long nodes, int ns, bool jacobi, bool minres, bool mg = false, long long cnodes = 0) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.o_x = take(sizeof(double) * nodes);
    L.o_r = take(sizeof(VT) * nodes);
    L.o_p0 = take(sizeof(VT) * nodes);
    L.o_p1 = take(sizeof(VT) * nodes);
    L.o_d = take(sizeof(VT) * nodes);
    L.o_as = take(sizeof(ST) * nodes);
    L.o_dinv = take(jacobi || mg ? sizeof(ST) * nodes : 0);
    L.o_vb = take(minres ? sizeof(VT) * nodes : 0);
    L.o_w0 = take(minres ? sizeof(VT) * nodes : 0);
    L.o_w1 = take(minres ? sizeof(VT) * nodes : 0);
    L.o_mz = take(mg ? sizeof(VT) * nodes : 0);
    L.o_mt = take(mg ? sizeof(VT) * nodes : 0);
    L.o_cx = take(mg ? sizeof(VT) * cnodes : 0);
    L.o_ct = take(mg ? sizeof(VT) * cnodes : 0);
    L.o_cb = take(mg ? sizeof(VT) * cnodes : 0);
    L.o_cas = take(mg ? sizeof(ST) * cnodes : 0);
    L.o_cdi = take(mg ? sizeof(ST) * cnodes : 0);
    L.o_we = take(sizeof(double) * nodes);
    L.o_wn = take(sizeof(double) * nodes);
    L.o_stats = take(sizeof(int32_t) * 2 * ns);
    L.o_err = take(sizeof(unsigned));
    L.zero_end = off;
    L.o_solves = take(sizeof(DevSolve) * ns);
    L.o_order = take(sizeof(int) * ns);
    L.total = off;
    return L;
}

template <class VT, class ST>
Params make_params(char* base, const Layout& L, int ns, int nbig, int nmed, int nsmall, int max_outer,
                   int max_iters, int prec, int jacobi, int solver, double theta, double tau_max) {
    Params P{};
    P.solves = reinterpret_cast<const DevSolve*>(base + L.o_solves);
    P.order = reinterpret_cast<const int*>(base + L.o_order);
    P.nbig = nbig;
    P.nmed = nmed;
    P.nsmall = nsmall;
    P.x64 = reinterpret_cast<double*>(base + L.o_x);
    P.r = base + L.o_r;
    P.p0 = base + L.o_p0;
    P.p1 = base + L.o_p1;
    P.d = base + L.o_d;
    P.as = base + L.o_as;
    P.dinv = base + L.o_dinv;
    P.vb = base + L.o_vb;
    P.w0 = base + L.o_w0;
    P.w1 = base + L.o_w1;
    P.mz = base + L.o_mz;
    P.mt = base + L.o_mt;
    P.cx = base + L.o_cx;
    P.ct = base + L.o_ct;
    P.cb = base + L.o_cb;
    P.cas = base + L.o_cas;
    P.cdi = base + L.o_cdi;
    P.we = reinterpret_cast<double*>(base + L.o_we);
    P.wn = reinterpret_cast<double*>(base + L.o_wn);
    P.mg = 0;
    P.mg_nu = 1;
    P.mg_coarse = 8;
    P.mg_omega = 0.8;
    P.mg_smem_nmax = 0;
    P.mg_smem_off = 0;
    P.solver = solver;
    P.sys_iters = reinterpret_cast<int32_t*>(base + L.o_stats);
    P.sys_outer = P.sys_iters + ns;
    P.max_outer = max_outer;
    P.max_iters = max_iters;
    P.theta = theta;
    // Refining the inner solve below what its operator can deliver wastes iterations:
    // a refinement step contracts the residual by about the storage unit roundoff.
    double tmin = 1e-6;
    if (prec == MLMC_FP64) tmin = 1e-14;
    if (prec == MLMC_FP16S) tmin = 1e-4;
    if (prec == MLMC_BF16S) tmin = 1e-3;
    P.tau_min = tmin;
    P.tau_max = tau_max;
    P.stag = 0.5;
    P.jacobi = jacobi;
    P.ring = 0;
    P.err = reinterpret_cast<unsigned*>(base + L.o_err);
    P.timeout_ns = 10000000000ull;
    P.extra_tx = 0;
    return P;
}

// Workspace row pitch: a multiple of 8 elements, so that every row of every
// array (8- to 2-byte elements) starts on a 16-byte boundary for bulk copies.

constexpr int kPipeSmemMax = 220 * 1024;   // dynamic shared memory budget of the row pipeline

// Slots per team for the large systems of a CG launch: the deepest ring
// (max_ring, or 4 when max_ring < 0, down to 2) whose shared memory fits every
// large system; 0 (no pipeline) if none does, if max_ring == 0, or if
// max_ring < 0 and fewer systems of the largest size than SMs.  Only systems with
// warp-aligned teams (chunks per row a multiple of 32) use the pipeline.
// `smem` receives the dynamic shared memory of the launch.
template <class VT, class ST>
int choose_ring(const std::vector<int>& big_n, size_t& smem, int max_ring, int num_sms) {
    smem = 0;
    if (big_n.empty() || max_ring == 0) return 0;
    // The FP64 inner solve streams stored FP64 edge weights, not the coefficient rows the
    // pipeline carries; it runs on plain loads.
    if (sizeof(VT) == 8) return 0;
    // Automatic: the pipeline pays when the largest systems -- the launch's
    // critical path -- occupy every SM (DRAM latency under full load is what it
    // hides; on a partly filled GPU the L1-cached plain loads keep up and cost
    // fewer issue slots).
    if (max_ring < 0) {
        const int nmax = *std::max_element(big_n.begin(), big_n.end());
        if ((int)std::count(big_n.begin(), big_n.end(), nmax) < num_sms) return 0;
    }
    for (int ring = max_ring < 0 ? 4 : max_ring; ring >= 2; --ring) {
        size_t need = 0;
        for (int n : big_n)
            need = std::max(need, (size_t)pipe_smem_bytes(n, row_pitch(n), ring, (int)sizeof(VT), (int)sizeof(ST)));
        if (need <= (size_t)kPipeSmemMax) {
            smem = need;
            return ring;
        }
    }
    return 0;
}

// Launch the CG or MINRES kernel (the row pipeline is CG-only).
template <class VT, class ST>
cudaError_t launch_resident(const Params& P, int solver, int grid, size_t smem, cudaStream_t st) {
    if (solver == MLMC_MINRES) {
        if (smem > 0) {
            const cudaError_t e = cudaFuncSetAttribute(resident_solve<VT, ST, MLMC_MINRES>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        resident_solve<VT, ST, MLMC_MINRES><<<grid, CTA, smem, st>>>(P);
    } else {
        if (smem > 0) {
            const cudaError_t e = cudaFuncSetAttribute(resident_solve<VT, ST, MLMC_CG>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        resident_solve<VT, ST, MLMC_CG><<<grid, CTA, smem, st>>>(P);
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

int grid_of(int nbig, int nmed, int nsmall) {
    return nbig + (nmed + 3) / 4 + (nsmall + CTA / G_SMALL - 1) / (CTA / G_SMALL);
}

// Plan, upload and launch one batch on stream st using workspace slot `slot`; the host
// checks it later with finish_solve (after st has been synchronised).
template <class VT, class ST>
mlmc_status launch_typed(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups, const SolveConfig& cfg,
                         cudaStream_t st, int slot, PendingSolve& out) {
    out = PendingSolve();
    // ---- host plan
    std::vector<DevSolve> solves;
    long long total = 0, ctotal = 0;
    const mlmc_problem& pb = ctx->prob;
    const int precond = cfg.precond >= 0 ? cfg.precond : ctx->precond;
    const bool mg = precond == MLMC_PC_MG;
    for (const SolveGroup& g : groups) {
        if (g.S <= 0) continue;
        const int n = g.n;
        const int ld = row_pitch(n);
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
        const double gnorm = g.rhs_weights ? *g.rhs_weights : 0.0;
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
            d.sys = (int)solves.size();
            d.mg_levels = mg ? mg_level_count(n, cfg.mg_min > 0 ? cfg.mg_min : ctx->mg_min) : 0;
            d.mg_off = ctotal;
            ctotal += mg ? mg_coarse_nodes(n, d.mg_levels) : 0;
            solves.push_back(d);
        }
    }
    const int ns = (int)solves.size();
    if (ns == 0) return MLMC_OK;
    // launch order: large systems first (largest first), then medium, then small
    std::vector<int> order(ns);
    for (int i = 0; i < ns; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return solves[x].n > solves[y].n; });
    // Mid-size systems (2048 < chunks <= 4096, n = 91..128) go four to a CTA when the launch also holds
    // systems at least twice their size and the CTAs of those and of the mid-size quarters fit one wave:
    // a quarter then takes about as long as one of the largest systems on a whole CTA, every long CTA
    // starts at once, and the small systems' CTAs fill in behind them.  Otherwise a whole CTA each.
    int med_items = cfg.med_items != kTuneUnset ? cfg.med_items : ctx->med_items;
    if (med_items < 0) {
        int nmax = 0, mid_nmax = 0, nmid = 0, nlarge = 0;
        for (const DevSolve& d : solves) {
            nmax = std::max(nmax, d.n);
            if (size_class(d.n, kMedItemsWide) == 0) {
                ++nlarge;
            } else if (size_class(d.n, kMedItems) == 0) {
                ++nmid;
                mid_nmax = std::max(mid_nmax, d.n);
            }
        }
        const bool wide = nmid > 0 && nlarge > 0 && 2 * mid_nmax <= nmax && nlarge + (nmid + 3) / 4 <= ctx->num_sms;
        med_items = wide ? kMedItemsWide : kMedItems;
    }
    int nbig = 0, nmed = 0, nsmall = 0;
    for (int i : order) {
        const int c = size_class(solves[i].n, med_items);
        nbig += c == 0;
        nmed += c == 1;
        nsmall += c == 2;
    }
    const Layout L = make_layout<VT, ST>(total, ns, cfg.jacobi != 0, cfg.solver == MLMC_MINRES, mg, ctotal);
    mlmc::DevBuf& buf = ctx->ws.solver_slot[slot];
    MLMC_CUDA_RET(ctx->err, buf.reserve(L.total));
    char* base = buf.as<char>();
    // Vectors start at zero.  Boundary and padding entries are never written and stay zero, and every
    // interior entry except x (which the refinement accumulates) is written before it is read; so when
    // the slot's last launch had this very layout, only x, the counters and the error word are cleared
    // (the whole clear moved about 0.7 GB for the 5-level estimate's largest launch).
    std::vector<long long> layout = {(long long)sizeof(VT), (long long)sizeof(ST), (long long)L.total};
    for (size_t o : {L.o_x, L.o_r, L.o_p0, L.o_p1, L.o_d, L.o_as, L.o_dinv, L.o_vb, L.o_w0, L.o_w1, L.o_mz, L.o_mt,
                     L.o_cx, L.o_ct, L.o_cb, L.o_cas, L.o_cdi, L.o_we, L.o_wn, L.o_stats, L.o_err, L.zero_end})
        layout.push_back((long long)o);
    for (const DevSolve& d : solves) {
        layout.push_back(d.n);
        layout.push_back(d.ld);
        layout.push_back(d.off);
        layout.push_back(d.mg_levels);
        layout.push_back(d.mg_off);
    }
    if (buf.ptr == ctx->ws.slot_ptr[slot] && layout == ctx->ws.slot_layout[slot]) {
        MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(base + L.o_x, 0, L.o_r - L.o_x, st));
        MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(base + L.o_stats, 0, L.zero_end - L.o_stats, st));
    } else {
        ctx->ws.slot_ptr[slot] = nullptr;   // until the clear below is enqueued
        MLMC_CUDA_RET(ctx->err, cudaMemsetAsync(base, 0, L.zero_end, st));
        ctx->ws.slot_ptr[slot] = buf.ptr;
        ctx->ws.slot_layout[slot] = std::move(layout);
    }
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(base + L.o_solves, solves.data(), sizeof(DevSolve) * ns,
                                            cudaMemcpyHostToDevice, st));
    MLMC_CUDA_RET(ctx->err, cudaMemcpyAsync(base + L.o_order, order.data(), sizeof(int) * ns,
                                            cudaMemcpyHostToDevice, st));
    Params P = make_params<VT, ST>(base, L, ns, nbig, nmed, nsmall, cfg.max_outer, cfg.max_iters, cfg.prec,
                                   cfg.jacobi, cfg.solver, cfg.theta > 0 ? cfg.theta : ctx->inner_theta,
                                   cfg.tau_max);
    if (ctx->inner_tau_min > 0) P.tau_min = ctx->inner_tau_min;
    if (cfg.tau_min > 0) P.tau_min = cfg.tau_min;
    if (mg) {
        P.mg = 1;
        P.mg_nu = cfg.nu > 0 ? cfg.nu : ctx->mg_nu;
        P.mg_coarse = cfg.mg_coarse > 0 ? cfg.mg_coarse : ctx->mg_coarse;
        P.mg_omega = cfg.mg_omega > 0 ? cfg.mg_omega : ctx->mg_omega;
        P.fmg = ctx->mg_fmg;
    }
    size_t smem = 0;
    if (cfg.solver == MLMC_CG) {
        std::vector<int> big_n;
        for (int i : order)
            if (size_class(solves[i].n, med_items) == 0) big_n.push_back(solves[i].n);
        // automatic choice with multigrid: no pipeline.  Its ring would take the shared memory that
        // the coarse levels and L1 serve the V-cycle passes from (measured: 4096 x n = 512 sweep
        // 0.593 s without, 0.700 s with), and it only speeds up the CG sweeps.
        const int ring_req = cfg.ring != kTuneUnset ? cfg.ring : ctx->solve_ring;
        const int want = (mg && ring_req < 0) ? 0 : ring_req;
        P.ring = choose_ring<VT, ST>(big_n, smem, want, ctx->num_sms);
    }
    // multigrid: the deepest coarse levels of the 512-thread groups in shared memory, as deep a cut
    // (coarse grids of at most 64, 32 or 16 cells) as fits beside the row pipeline
    if (mg && nbig > 0) {
        const size_t pipe_end = smem ? (smem + 127) / 128 * 128 : 0;
        for (int nmax : {64, 32, 16}) {
            if (cfg.mg_smem > 0 && nmax > cfg.mg_smem) continue;
            // every large system's shared-memory levels must fit (halving chains differ by grid)
            size_t need = 0;
            for (int i : order) {
                const int ni = solves[i].n;
                if (size_class(ni, med_items) != 0) continue;
                need = std::max(need, (size_t)mg_smem_bytes(ni, solves[i].mg_levels, nmax, (int)sizeof(VT),
                                                            (int)sizeof(ST), solves[i].mg_levels + 1));
            }
            if (need > 0 && pipe_end + need <= (size_t)kPipeSmemMax) {
                P.mg_smem_nmax = nmax;
                P.mg_smem_off = (int)pipe_end;
                smem = pipe_end + need;
                break;
            }
        }
    }
    P.timeout_ns = (unsigned long long)(ctx->wait_timeout_s * 1e9);
    P.extra_tx = 16u * (unsigned)ctx->wait_extra;
    P.err = ctx->solve_err;   // the context's word: it outlives the workspace, read at the next synchronising call
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (ctx->prof.on) {
        MLMC_CUDA_RET(ctx->err, cudaEventCreate(&ev[0]));
        MLMC_CUDA_RET(ctx->err, cudaEventCreate(&ev[1]));
        MLMC_CUDA_RET(ctx->err, cudaEventRecord(ev[0], st));
    }
    MLMC_CUDA_RET(ctx->err, (launch_resident<VT, ST>(P, cfg.solver, grid_of(nbig, nmed, nsmall), smem, st)));
    if (ctx->prof.on) MLMC_CUDA_RET(ctx->err, cudaEventRecord(ev[1], st));
    ctx->prof.acc.h2d_bytes += (int64_t)((sizeof(DevSolve) + sizeof(int)) * ns);
    out.active = true;
    out.stats = reinterpret_cast<const int32_t*>(base + L.o_stats);
    out.ns = ns;
    out.max_outer = cfg.max_outer;
    out.ev[0] = ev[0];
    out.ev[1] = ev[1];
    if (ctx->prof.on) {
        // algorithmic bytes of each system, per unit of its counters (inner iterations, refinement steps)
        const double pv = sizeof(VT), ps = sizeof(ST);
        const double pd = cfg.jacobi ? ps : 0.0;   // inverse diagonal read once per inner iteration
        for (const DevSolve& d : solves) {
            const double unk = (double)(d.n - 1) * (d.n - 1);
            const double pm = d.a_fp64 ? 8.0 : 4.0;
            const double vcyc = mg ? mg_iter_bytes(d.n, d.mg_levels, P.mg_nu, P.mg_coarse, pv, ps) / unk : 0.0;
            const double per_it = cfg.solver == MLMC_MINRES ? (mg ? vcyc + 14 * pv + 2 * ps : 14 * pv + 2 * ps + pd)
                                                            : (mg ? vcyc + 8 * pv + 2 * ps : 8 * pv + 2 * ps + pd);
            out.unk.push_back(unk);
            out.c_it.push_back(unk * per_it);
            // refinement residual: x, the two FP64 edge weights, r and d (and D^-1); update: x and d;
            // set-up: the master coefficient read for the storage copy and the weights, the copy, D^-1 and
            // the weights written
            out.c_res.push_back(unk * (8 + 16 + 2 * pv + pd));
            out.c_upd.push_back(unk * (16 + pv));
            const bool fmg = mg && P.fmg && cfg.solver == MLMC_CG && d.mg_levels > 0;
            out.c_set.push_back(unk * (8 + pm + ps + pd + 16) +
                                (fmg ? mg_fmg_bytes(d.n, d.mg_levels, P.mg_nu, P.mg_coarse, pv, ps) : 0.0));
            // operations: per inner iteration two stencil sweeps with their recurrences and dots, plus
            // the V-cycle (CG: 12 + 2 S with Jacobi, 10 + 2 S with multigrid; MINRES: 18 + 2 S and
            // 17 + 2 S); per refinement step the FP64 residual from the stored weights with its three
            // dots (20) and the update (1); set-up: the edge weights (8), the inverse diagonal (21;
            // 7 more for the coarse levels) and the QoI (2)
            const double S_ = (sizeof(VT) == 8 && sizeof(ST) == 8) ? kFlopStencilW : kFlopStencil;
            const double vf = mg ? mg_iter_flops(d.n, d.mg_levels, P.mg_nu, P.mg_coarse, S_) / unk : 0.0;
            const double fit = cfg.solver == MLMC_MINRES ? (mg ? 17.0 : 18.0) + 2.0 * S_ + vf
                                                         : (mg ? 10.0 : 12.0) + 2.0 * S_ + vf;
            out.f_it.push_back(unk * fit);
            out.f_res.push_back(unk * 20.0);
            out.f_upd.push_back(unk * 1.0);
            out.f_set.push_back(unk * (8.0 + 21.0 + (mg ? 7.0 : 0.0) + 2.0) +
                                (fmg ? mg_fmg_flops(d.n, d.mg_levels, P.mg_nu, P.mg_coarse, S_) : 0.0));
        }
    }
    return MLMC_OK;
}

// Descriptors and launch order of a batch of equal-shaped systems, written on the device.
__global__ void noalloc_plan_kernel(DevSolve proto, int S, long long stride_nodes, long long a_elems,
                                    int a_elem_bytes, DevSolve* solves, int* order) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    DevSolve d = proto;
    d.off = s * stride_nodes;
    d.a = static_cast<const char*>(proto.a) + (size_t)s * a_elems * a_elem_bytes;
    d.out = s;
    d.sys = s;
    solves[s] = d;
    order[s] = s;
}

template <class VT, class ST>
mlmc_status noalloc_typed(int n, int S, const void* a, int a_fp64, int a_n, double delta, int max_iters, int qoi,
                          const double* box, double f, int prec, double* Q, int32_t* iters, double* relres,
                          int32_t* flags, cudaStream_t st, void* scratch, std::string& err) {
    const int ld = row_pitch(n);
    const long long stride = (long long)align_up((size_t)(n + 1) * ld, 64);
    const Layout L = make_layout<VT, ST>(stride * S, S, true, false);
    if (L.total > (size_t)MLMC_NOALLOC_SCRATCH_BYTES) {
        err = "level_solve_noalloc: the batch needs " + std::to_string(L.total) + " bytes of scratch, above the " +
              std::to_string((size_t)MLMC_NOALLOC_SCRATCH_BYTES) + "-byte maximum (MLMC_NOALLOC_SCRATCH_BYTES); use fewer systems";
        return MLMC_E_ARG;
    }
    char* base = static_cast<char*>(scratch);
    cudaError_t e;
    if ((e = cudaMemsetAsync(base, 0, L.zero_end, st)) != cudaSuccess) {
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
    noalloc_plan_kernel<<<(unsigned)((S + 255) / 256), 256, 0, st>>>(
        proto, S, stride, a_elems, a_fp64 ? 8 : 4, reinterpret_cast<DevSolve*>(base + L.o_solves),
        reinterpret_cast<int*>(base + L.o_order));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        err = std::string("level_solve_noalloc: plan kernel: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    const int c = size_class(n);
    const int nbig = c == 0 ? S : 0, nmed = c == 1 ? S : 0, nsmall = c == 2 ? S : 0;
    Params P = make_params<VT, ST>(base, L, S, nbig, nmed, nsmall, 12, max_iters, prec, 1, MLMC_CG, 0.3, 0.5);
    size_t smem = 0;
    int sms = 0, cur = 0;
    if ((e = cudaGetDevice(&cur)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cur)) != cudaSuccess) {
        err = std::string("level_solve_noalloc: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    P.ring = nbig > 0 ? choose_ring<VT, ST>(std::vector<int>((size_t)nbig, n), smem, -1, sms) : 0;
    if ((e = launch_resident<VT, ST>(P, MLMC_CG, grid_of(nbig, nmed, nsmall), smem, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
        err = std::string("level_solve_noalloc: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    unsigned kerr = 0;
    if ((e = cudaMemcpy(&kerr, base + L.o_err, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        err = std::string("level_solve_noalloc: ") + cudaGetErrorString(e);
        return MLMC_E_CUDA;
    }
    if (kerr != KERR_NONE) {
        err = "level_solve_noalloc: a bounded wait of the row pipeline ran out; the affected systems carry "
              "MLMC_F_TIMEOUT";
        return MLMC_E_TIMEOUT;
    }
    return MLMC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// The entry points of this precision (declared in internal.h).
#if MLMC_SOLVER_PREC == 0
#define MLMC_SOLVER_NAME(x) x##_fp64
using SolverVT = double;
using SolverST = double;
#elif MLMC_SOLVER_PREC == 1
#define MLMC_SOLVER_NAME(x) x##_fp32
using SolverVT = float;
using SolverST = float;
#elif MLMC_SOLVER_PREC == 2
#define MLMC_SOLVER_NAME(x) x##_bf16s
using SolverVT = float;
using SolverST = __nv_bfloat16;
#elif MLMC_SOLVER_PREC == 3
#define MLMC_SOLVER_NAME(x) x##_fp16s
using SolverVT = float;
using SolverST = __half;
#else
#error "MLMC_SOLVER_PREC must be an mlmc_prec value"
#endif

mlmc_status MLMC_SOLVER_NAME(solve_launch)(mlmc_ctx* ctx, const std::vector<SolveGroup>& groups,
                                           const SolveConfig& cfg, cudaStream_t st, int slot, PendingSolve& out) {
    return launch_typed<SolverVT, SolverST>(ctx, groups, cfg, st, slot, out);
}

cudaError_t MLMC_SOLVER_NAME(apply_operator)(int n, int S, const void* a, int a_fp64, int a_n, const void* x, void* y,
                                             cudaStream_t st) {
    const long long work = (long long)S * (n + 1) * (n + 1);
    const unsigned grid = (unsigned)((work + 255) / 256);
    apply_operator_kernel<SolverVT, SolverST><<<grid, 256, 0, st>>>(n, S, a, a_fp64, a_n,
                                                                     static_cast<const SolverVT*>(x),
                                                                     static_cast<SolverVT*>(y));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

mlmc_status MLMC_SOLVER_NAME(noalloc_solve)(int n, int S, const void* a, int a_fp64, int a_n, double delta,
                                            int max_iters, int qoi, const double* box, double f, double* Q,
                                            int32_t* iters, double* relres, int32_t* flags, cudaStream_t st,
                                            void* scratch, std::string& err) {
    return noalloc_typed<SolverVT, SolverST>(n, S, a, a_fp64, a_n, delta, max_iters, qoi, box, f, MLMC_SOLVER_PREC, Q,
                                             iters, relres, flags, st, scratch, err);
}

}  // namespace mlmc
