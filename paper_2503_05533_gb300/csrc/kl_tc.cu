// A2 on the tensor cores: a[s][v] = exp(sum_k xi[s][k] Phi[k][v]) (Sec. 5.1,
// Eq. (5.2); the KL field of the configurations) as a (samples x KL terms) x
// (KL terms x nodes) contraction on tcgen05 with FP16 operands and FP32
// accumulation in tensor memory, in two forms:
//
// FP32 output.  Both operands are split x = hi + lo 2^-11 (hi = fp16(x),
// lo = fp16((x - hi) 2^11), which keeps lo in FP16's normal range); the basis
// is scaled by log2(e) before the split, and two accumulators hold
// D0 = Phi_hi xi_hi^T and D1 = Phi_hi xi_lo^T + Phi_lo xi_hi^T over all K, so
// log2 a = D0 + 2^-11 D1 (the lo*lo term, 2^-22 relative, dropped) and
// a = 2^(log2 a) by the SFU's exp2.  About 1e-6 relative error in a.
//
// FP64 output (the master coefficient of the mixed-precision solves, where the
// refinement residual of Alg. 2.1 is FP64).  Each sample row of xi is scaled by
// a power of two 2^-e_s so that its largest entry lies in [1/2, 1), and each
// node's column of Phi likewise by 2^-e_v; the scaled values times 2^9 are
// split into an integer lead slice (|lead| <= 512, exact in FP16) and two FP16
// slices h and l of the remainder (X = lead + h + 2^-11 l up to 2^-23 for
// |X| <= 512).  Three accumulators hold, per 64-term K block,
//   E0 = lead_x lead_y^T                                  (integers below 2^24:
//        exact in FP32, whatever order the tensor core adds them in),
//   E1 = lead_x h_y^T + h_x lead_y^T + h_x h_y^T,
//   E2 = lead_x l_y^T + l_x lead_y^T + h_x l_y^T + l_x h_y^T,
// and the epilogue adds the K blocks: E0 as exact 32-bit integers, E1 + 2^-11 E2
// in FP32, then log a = 2^(e_s + e_v - 18) (sum E0 + sum (E1 + 2^-11 E2)) as a
// float-float pair.  The slices represent each operand to 2^-23 of |X| <= 512,
// which bounds the log-a error by 2^-32 (2^e_v sum_k |xi_k| + 2^e_s sum_k
// |Phi_k(x_v)|) + K 2^(e_s + e_v - 42); the FP32 accumulation of E1 (terms at
// most 2^-9 of the E0 scale, at most 12 additions per K block) adds at most
// about six times that; E0 adds nothing.  Rounding errors of opposite signs
// cancel, and the error is typically near 1e-10.
// a = exp(log a) is formed in float-float arithmetic by the table-driven method
// of P. T. P. Tang (ACM TOMS 15(2), 1989): N = round(32 log a / ln 2),
// r = log a - N ln 2 / 32 with ln 2 / 32 split into three parts so that the
// reduction is exact to float-float precision, exp(r) - 1 by its Taylor
// polynomial to r^5 (|r| <= ln 2 / 64), times the table value 2^(j/32) stored as
// a float-float pair and 2^((N - j) / 32); the pair is written as one FP64
// value.  The FP32 pipe does all of this work: GB300's FP64 pipe is narrow.
//
// Execution: a persistent kernel, one CTA per SM walking output tiles of 128
// nodes x TN samples.  The MMA's A operand is the basis (M = 128 node rows),
// its B operand xi (N = TN sample rows), so a tensor-memory lane holds one node
// and a column one sample.  Warp 0 streams the operand slices of every 64-term
// K block by TMA (128-byte swizzle) through a ring of shared-memory stages;
// warp 1 issues the MMAs (M = 128, N = TN, K = 16) into one of two tensor-
// memory buffers and signals through mbarriers; 16 epilogue warps drain the
// other buffer (each warp 32 sample columns of one TMEM lane quarter in the
// FP32 form, 16 in the FP64 form).
// Loads of tile t+1 and the epilogue of tile t overlap its MMAs.  Output rows
// (one per sample) are `ldo` elements apart.  When they are whole 128-byte
// lines (ldo a multiple of 32, aligned base: the layout the estimate uses),
// each warp writes, sample by sample, the 32 consecutive nodes of its lanes
// as one full line straight from registers.  Otherwise (dense rows of
// (n+1)^2 elements, which start at any 4-byte offset) the FP32 form stages
// each 32-sample chunk in shared memory and writes whole 128-node rows with
// 16-byte stores, so that no store straddles two lines needlessly.  Every mbarrier wait is bounded in wall time; on expiry the CTA records
// the context's error word, every role leaves its loop, the producer waits
// (bounded) for its copies in flight, and the TMEM is freed.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {
namespace {

constexpr int TM = 128;              // nodes per tile (MMA M, TMEM lanes)
constexpr int TKB = 64;              // terms per K block: 64 FP16 = one 128-byte swizzle row
constexpr uint32_t kATile = TM * TKB * 2;   // 16 KiB: one slice of 128 node rows
constexpr int kStgPitch = TM + 4;           // floats per staging row (528 bytes, a multiple of 16)

// MODE 0: FP32 output (2 slices per operand) through the shared-memory staging of the epilogue;
// MODE 2: the same into rows of whole 128-byte lines, stored straight from registers (a third TMA stage
// in place of the staging area); MODE 1: FP64 output (3 slices, exact lead).
template <int MODE> struct KLCfg;
// Warp 0 issues the TMA copies, warp 1 the MMAs; EW = 4 TN / CW epilogue warps follow, each draining one
// CW-column chunk of one TMEM lane quarter (its warp index mod 4).  The FP64 form's long per-element
// epilogue takes 16-column chunks, so that twice as many warps hide its latency.
template <> struct KLCfg<0> {
    static constexpr int NA = 2, NB = 2, TN = 128, NACC = 2, NSTAGE = 2, CW = 32, EW = 4 * TN / CW;
    static constexpr bool DRAIN = false;   // accumulate the whole K range in TMEM
    using Out = float;
};
template <> struct KLCfg<2> {
    static constexpr int NA = 2, NB = 2, TN = 128, NACC = 2, NSTAGE = 3, CW = 32, EW = 4 * TN / CW;
    static constexpr bool DRAIN = false;
    using Out = float;
};
template <> struct KLCfg<1> {
    static constexpr int NA = 3, NB = 3, TN = 64, NACC = 3, NSTAGE = 3, CW = 16, EW = 4 * TN / CW;
    static constexpr bool DRAIN = true;    // the epilogue drains every K block
    using Out = double;
};

template <int MODE> struct KLLayout {
    using C = KLCfg<MODE>;
    static constexpr uint32_t kBTile = C::TN * TKB * 2;
    static constexpr uint32_t kStage = C::NA * kATile + C::NB * kBTile;   // multiple of 1024
    static constexpr uint32_t kOffStg = C::NSTAGE * kStage;
    // FP32 form: per 32-sample chunk, 32 staging rows of kStgPitch floats (a tile row of 128 nodes plus a
    // shift of up to 3 that aligns it with the output's 16-byte boundaries).  Two TMA stages make room
    // for it; two rounds of 16 rows beside a third stage measured slower (the extra barriers).
    // FP64 form: the exponential's table 2^(j/32) = th + tl (64 floats), indexed per lane
    static constexpr uint32_t kStgBytes = MODE == 0 ? (C::TN / 32) * 32 * kStgPitch * 4 : (MODE == 1 ? 64 * 4 : 0);
    static constexpr int kThreads = 64 + 32 * C::EW;
    static constexpr uint32_t kOffBar = (kOffStg + kStgBytes + 15) / 16 * 16;
    // full[NSTAGE], empty[NSTAGE], tfull[2], tempty[2], then the TMEM address and the abort flag
    static constexpr uint32_t kBarBytes = 8 * (2 * C::NSTAGE + 4) + 16;
    static constexpr uint32_t kSmem = kOffBar + kBarBytes + 1024;          // + 1 KiB for 1024-byte alignment
    static constexpr uint32_t kTmemCols = 512;                             // 2 buffers x NACC x TN <= 512
    static_assert(2 * C::NACC * C::TN <= 512, "tensor memory");
    static_assert(kSmem <= 227 * 1024, "shared memory");
};

// Float-float exponential tables (host-computed): 2^(j/32) = th[j] + tl[j]; ln 2 / 32 = l1 + l2 + l3
// with l1 of at most 12 significant bits; inv = 32 / ln 2.
struct FFExp {
    float th[32], tl[32];
    float l1, l2, l3, inv;
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), fixed version bits 0b001.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// Instruction descriptor, kind::f16: D FP32, A and B FP16, both K-major, M = 128, N = TN.
template <int TN>
constexpr uint32_t idesc() {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

template <int TN>
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc<TN>()), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// 2^x by the SFU's approximation (maximum relative error about 2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// Named barrier `id` over `count` threads that also returns the OR of every thread's `v`.
__device__ __forceinline__ bool bar_or(int id, int count, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "barrier.cta.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void bar_sync_n(int id, int count) {
    asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Tile t -> (sample tile st, node tile nt).  Node tiles go in groups of G; a group's tiles are
// taken node tile fastest, so the tiles in flight at any time cover about G consecutive node tiles
// of every sample row they touch (long contiguous runs of output per row), while the group's basis
// rows stay in L2 for all its sample tiles.
__device__ __forceinline__ void tile_coords(int t, int num_st, int num_nt, int G, int& st, int& nt) {
    const int g = t / (G * num_st);
    const int Gg = min(G, num_nt - g * G);
    const int r = t - g * G * num_st;
    nt = g * G + r % Gg;
    st = r / Gg;
}

// Bounded wait that also gives up once another role has aborted the CTA.
__device__ __forceinline__ bool kl_wait(uint64_t* bar, uint32_t parity, volatile int* abort, unsigned* err,
                                        uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (global_ns() - t0 > timeout_ns) {
            *abort = 1;
            atomicCAS(err, KERR_NONE, KERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// The same wait for a whole warp: lane 0 waits (bounded), the warp agrees on the outcome, and on
// success every lane observes the completed phase itself (at once: it has completed), so that the
// warp's later .sync.aligned tensor-memory loads are never split by a timeout.
__device__ __forceinline__ bool kl_warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort, unsigned* err,
                                             uint64_t timeout_ns) {
    bool ok = false;
    if ((threadIdx.x & 31) == 0) ok = kl_wait(bar, parity, abort, err, timeout_ns);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    if (ok) mbar_wait(bar, parity, timeout_ns);
    return ok;
}

// x 2^e: one product with the power of two when 2^e is a normal float (the same single rounding as
// ldexpf), else ldexpf.
__device__ __forceinline__ float scale2(float x, int e) {
    return (e >= -126 && e <= 127) ? __fmul_rn(x, __int_as_float((e + 127) << 23)) : ldexpf(x, e);
}
// The rare cases of ff_to_double, on the FP64 pipe (kept out of line, so that the common path never
// executes FP64 instructions under a predicate).
__device__ __noinline__ double ff_to_double_fp64(float ah, float al) { return (double)ah + (double)al; }

// (double)ah + (double)al rounded to nearest, for a float-float pair with |al| <= ulp(ah) / 2, without the
// FP64 pipe (GB300's is narrow): ah's double has its float mantissa followed by 29 zero bits, so al
// amounts to k = al / ulp_double(ah) units of the last place, |k| <= 2^28; al 2^(52 - e) is an exact
// power-of-two scaling, its rounding to the nearest integer (ties to even) is the rounding of the sum
// (the last bit of the result is k's), and k is added to the bit pattern.  A sum that leaves ah's
// binade downwards (ah a power of two, |ah + al| < |ah|), where the last place halves, and exponents
// outside [-60, 100] take the FP64 instructions.
__device__ __forceinline__ double ff_to_double(float ah, float al) {
    const uint32_t u = __float_as_uint(ah);
    const int Eb = (int)((u >> 23) & 0xFFu);
    const uint32_t M = u & 0x7FFFFFu;
    const int e = Eb - 127;
    const bool down = (M == 0u) && ((al < 0.0f) != (ah < 0.0f)) && al != 0.0f;
    if (e < -60 || e > 100 || down) return ff_to_double_fp64(ah, al);
    const unsigned long long bits =
        ((unsigned long long)((u & 0x80000000u) | ((uint32_t)(Eb + 896) << 20) | (M >> 3)) << 32) |
        (unsigned long long)(u << 29);
    int k = __float2int_rn(__fmul_rn(al, __int_as_float((52 - e + 127) << 23)));
    if (u >> 31) k = -k;    // the bits hold |ah|: a negative ah grows in magnitude with a negative al
    return __longlong_as_double((long long)(bits + (unsigned long long)(long long)k));
}

// exp(xh + xl) as a float-float pair (Tang's table-driven method, see the file comment); th, tl: the
// table 2^(j/32) = th[j] + tl[j] (shared memory).
__device__ __forceinline__ void ff_exp(float xh, float xl, const FFExp& T, const float* th_s, const float* tl_s,
                                       float& rh, float& rl) {
    const int N = __float2int_rn(__fmul_rn(xh, T.inv));
    const float nf = (float)N;
    const int j = N & 31;
    const int m = (N - j) / 32;
    // r = x - N ln2/32: xh - N l1 is exact (N l1 has at most 24 bits and is within a factor 2 of xh)
    const float t = __fsub_rn(xh, __fmul_rn(nf, T.l1));
    float p, pe, s, se;
    ff_two_prod(nf, T.l2, p, pe);
    ff_two_sum(t, -p, s, se);
    const float lo = __fsub_rn(__fadd_rn(se, xl), __fmaf_rn(nf, T.l3, pe));
    float r, rlo;
    ff_fast_two_sum(s, lo, r, rlo);
    // exp(r) - 1 = r + r^2/2 + r^3 (1/6 + r (1/24 + r/120))
    float sq, sqe;
    ff_two_prod(r, r, sq, sqe);
    const float r3 = __fmul_rn(__fmul_rn(sq, r),
                               __fmaf_rn(r, __fmaf_rn(r, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f));
    float qh, qe;
    ff_two_sum(r, __fmul_rn(0.5f, sq), qh, qe);
    const float ql0 = __fadd_rn(__fadd_rn(qe, rlo), __fadd_rn(__fmaf_rn(0.5f, sqe, __fmul_rn(r, rlo)), r3));
    float q, ql;
    ff_fast_two_sum(qh, ql0, q, ql);
    // 2^(j/32) (1 + q)
    const float th = th_s[j], tl = tl_s[j];
    float ph, phe, s1, s1e;
    ff_two_prod(th, q, ph, phe);
    ff_two_sum(th, ph, s1, s1e);
    const float lo2 = __fadd_rn(__fadd_rn(s1e, phe), __fmaf_rn(th, ql, __fmaf_rn(tl, q, tl)));
    float h, l;
    ff_fast_two_sum(s1, lo2, h, l);
    rh = scale2(h, m);
    rl = scale2(l, m);
}

template <int MODE>
__global__ void __launch_bounds__(KLLayout<MODE>::kThreads, 1)
    kl_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int S, int Spad,
                 int V, int Vpad, int Kpad, int num_st, int num_tiles, int tile_group, const int* __restrict__ es,
                 const int* __restrict__ ev, const __grid_constant__ FFExp ffx, typename KLCfg<MODE>::Out* __restrict__ out,
                 long long ldo,
                 unsigned* err, unsigned long long timeout_ns, unsigned extra_tx) {
    using C = KLCfg<MODE>;
    using Lay = KLLayout<MODE>;
    using Out = typename C::Out;
    constexpr int TN = C::TN;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::kOffBar);
    uint64_t* empty = full + C::NSTAGE;
    uint64_t* tfull = empty + C::NSTAGE;
    uint64_t* tempty = tfull + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = Kpad / TKB;
    // FP64 form: the exponential's table in shared memory (lanes index it by their own j; the kernel
    // parameter's constant bank would serialise distinct indices)
    float* ffx_th = reinterpret_cast<float*>(smem + Lay::kOffStg);
    float* ffx_tl = ffx_th + 32;
    if (MODE == 1 && threadIdx.x < 32) {
        ffx_th[threadIdx.x] = ffx.th[threadIdx.x];
        ffx_tl[threadIdx.x] = ffx.tl[threadIdx.x];
    }

    if (threadIdx.x == 0) {
        for (int i = 0; i < C::NSTAGE; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull + i, 1);
            mbar_init(tempty + i, C::EW);   // one arrival per epilogue warp
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(Lay::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            unsigned issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                int st_, nt_;
                tile_coords(t, num_st, num_tiles / num_st, tile_group, st_, nt_);
                const int s0 = st_ * TN, v0 = nt_ * TM;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!kl_wait(empty + stage, phase ^ 1u, abort, err, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + (size_t)stage * Lay::kStage;
                    mbar_expect_tx(full + stage, Lay::kStage + (issued == 0 ? extra_tx : 0u));
                    ++issued;
#pragma unroll
                    for (int q = 0; q < C::NA; ++q) tma_load_2d(st + q * kATile, &mapA, kb * TKB, q * Vpad + v0, full + stage);
#pragma unroll
                    for (int q = 0; q < C::NB; ++q)
                        tma_load_2d(st + C::NA * kATile + q * Lay::kBTile, &mapB, kb * TKB, q * Spad + s0, full + stage);
                    if (++stage == C::NSTAGE) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // let the copies in flight land before the CTA's shared memory goes away: the last
                // NSTAGE issues, each on its own stage (bounded; a copy that never completes its
                // barrier is waited for only until the timeout)
                const unsigned n = issued < (unsigned)C::NSTAGE ? issued : (unsigned)C::NSTAGE;
                for (unsigned i = 0; i < n; ++i) {
                    const unsigned g = issued - 1u - i;
                    mbar_wait(full + (g % C::NSTAGE), (g / C::NSTAGE) & 1u, timeout_ns);
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            int stage = 0, tb = 0;
            uint32_t phase = 0, tphase = 0;
            bool ok = true;
            uint64_t* last_bar = nullptr;   // barrier and parity of the last commit, for a clean abort
            uint32_t last_par = 0;
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                if (!C::DRAIN && !kl_wait(tempty + tb, tphase ^ 1u, abort, err, timeout_ns)) break;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (C::DRAIN && !kl_wait(tempty + tb, tphase ^ 1u, abort, err, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    if (!kl_wait(full + stage, phase, abort, err, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + (size_t)stage * Lay::kStage);
                    const uint32_t sb = sa + C::NA * kATile;
                    const uint32_t d0 = tmem + (uint32_t)(tb * C::NACC * TN);
#pragma unroll
                    for (int k = 0; k < TKB / 16; ++k) {
                        const uint32_t koff = (uint32_t)k * 32u;   // 16 FP16 = 32 bytes along the swizzled row
                        const bool first = C::DRAIN ? (k == 0) : (kb == 0 && k == 0);
                        const uint64_t a0 = desc_sw128(sa + koff), b0 = desc_sw128(sb + koff);
                        const uint64_t a1 = desc_sw128(sa + kATile + koff), b1 = desc_sw128(sb + Lay::kBTile + koff);
                        mma_f16<TN>(d0, a0, b0, first ? 0u : 1u);
                        mma_f16<TN>(d0 + TN, a0, b1, first ? 0u : 1u);
                        mma_f16<TN>(d0 + TN, a1, b0, 1u);
                        if (MODE == 1) {
                            const uint64_t a2 = desc_sw128(sa + 2 * kATile + koff);
                            const uint64_t b2 = desc_sw128(sb + 2 * Lay::kBTile + koff);
                            mma_f16<TN>(d0 + TN, a1, b1, 1u);
                            mma_f16<TN>(d0 + 2 * TN, a0, b2, first ? 0u : 1u);
                            mma_f16<TN>(d0 + 2 * TN, a2, b0, 1u);
                            mma_f16<TN>(d0 + 2 * TN, a1, b2, 1u);
                            mma_f16<TN>(d0 + 2 * TN, a2, b1, 1u);
                        }
                    }
                    mma_commit(empty + stage);   // the stage is free once these MMAs have read it
                    last_bar = empty + stage;
                    last_par = phase;
                    if (++stage == C::NSTAGE) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    if (C::DRAIN) {
                        mma_commit(tfull + tb);
                        if (++tb == 2) {
                            tb = 0;
                            tphase ^= 1u;
                        }
                    }
                }
                if (!ok) break;
                if (!C::DRAIN) {
                    mma_commit(tfull + tb);
                    if (++tb == 2) {
                        tb = 0;
                        tphase ^= 1u;
                    }
                }
            }
            // after an abort, the MMAs already issued finish before the tensor memory is freed
            if (*abort && last_bar) mbar_wait(last_bar, last_par, timeout_ns);
        }
    } else {
        // ---- epilogue: warp 2 + e drains TMEM lanes 32 (warp % 4) .. + 31 -- one node per lane -- of the
        // tile's sample chunk e / 4 (32 columns, one sample each) and writes, for every sample, the 32
        // consecutive nodes of its lanes with one coalesced store
        const int e = warp - 2;
        const int q4 = warp & 3;
        const int c = e >> 2;
        const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
        // the output's offset from a 16-byte boundary, in elements (FP32 form)
        const int mis = (int)((reinterpret_cast<uintptr_t>(out) / sizeof(Out)) & 3);
        // FP32 form: rows of whole 128-byte lines (see the epilogue)
        constexpr bool lines = MODE == 2;
        int tb = 0;
        uint32_t tphase = 0;
        for (int t = blockIdx.x; t < num_tiles; t += gridDim.x) {
            int st_, nt_;
            tile_coords(t, num_st, num_tiles / num_st, tile_group, st_, nt_);
            const int s0 = st_ * TN, v0 = nt_ * TM;
            const int v = v0 + q4 * 32 + lane;       // this lane's node
            const int sc0 = s0 + c * C::CW;          // the chunk's first sample
            if constexpr (MODE != 1) {
                // Output rows (one per sample) are `ldo` elements apart.  When ldo is a multiple of 32 and
                // the output starts on a 128-byte boundary, every 32-node piece of a row is one full line:
                // each warp stores its 32 nodes of every sample straight from registers.  Otherwise a row
                // of the tile starts at any 4-byte offset and such a store would straddle two lines, so the
                // four warps of chunk c (one per lane quarter) stage the chunk's 32 samples x 128 nodes in
                // shared memory and each writes 8 whole rows of 128 nodes with 16-byte stores.
                const bool ok = kl_warp_wait(tfull + tb, tphase, abort, err, timeout_ns);
                uint32_t r0[32], r1[32];
                if (ok) {
                    tc_fence_after();
                    const uint32_t base = tmem + lane_base + (uint32_t)(tb * C::NACC * TN + c * C::CW);
                    tmem_ld_x32(base, r0);
                    tmem_ld_x32(base + (uint32_t)TN, r1);
                    tmem_wait_ld();
                    // this warp's values are in registers: its share of the buffer goes back to the MMA warp
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty + tb);
                }
                if (++tb == 2) {
                    tb = 0;
                    tphase ^= 1u;
                }
                if constexpr (lines) {
                    if (!ok) break;
                    if (v < V) {
                        // the basis tables carry log2(e): the accumulators hold log2 a; one running pointer
                        // down the chunk's 32 sample rows
                        Out* p = out + (size_t)sc0 * ldo + v;
                        if (sc0 + 32 <= S) {
#pragma unroll
                            for (int j = 0; j < 32; ++j, p += ldo)
                                *p = (Out)ex2_approx(
                                    __fmaf_rn(__uint_as_float(r1[j]), 1.0f / 2048.0f, __uint_as_float(r0[j])));
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j, p += ldo)
                                if (sc0 + j < S)
                                    *p = (Out)ex2_approx(
                                        __fmaf_rn(__uint_as_float(r1[j]), 1.0f / 2048.0f, __uint_as_float(r0[j])));
                        }
                    }
                } else {
                    // the chunk's warps agree to go on (a failed wait anywhere stops all four together); it also
                    // orders their previous tile's reads of the staging rows before the writes below
                    if (bar_or(1 + c, 128, !ok)) break;
                    float* stg = reinterpret_cast<float*>(smem + Lay::kOffStg) + (size_t)c * 32 * kStgPitch;
                    const int nv = min(TM, V - v0);   // nodes of this tile inside the grid
                    // output index of (sample sc0, node v0) plus the output's offset, mod 4 (32-bit arithmetic
                    // suffices for a residue mod 4); sample sc0 + j adds j ldo
                    const uint32_t g4 = (uint32_t)sc0 * (uint32_t)ldo + (uint32_t)v0 + (uint32_t)mis;
                    // staging row j holds sample sc0 + j, node v0 + k at slot k + sh_j with sh_j = (output index
                    // + mis) mod 4, so that 16-byte-aligned output addresses meet 16-byte-aligned slots
                    const uint32_t d4 = (uint32_t)ldo & 3u;
                    uint32_t shj = g4 & 3u;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float l2 = __fmaf_rn(__uint_as_float(r1[j]), 1.0f / 2048.0f, __uint_as_float(r0[j]));
                        stg[j * kStgPitch + (int)shj + q4 * 32 + lane] = ex2_approx(l2);
                        shj = (shj + d4) & 3u;
                    }
                    bar_sync_n(1 + c, 128);
                    // warp q4 writes staging rows 8 q4 .. 8 q4 + 7, one running pointer down them
                    const int j0 = q4 * 8;
                    Out* dst = out + (size_t)(sc0 + j0) * ldo + v0;
                    uint32_t shr = (g4 + (uint32_t)j0 * (uint32_t)ldo) & 3u;
                    const int jn = min(8, S - (sc0 + j0));
#pragma unroll 1
                    for (int jj = 0; jj < jn && nv > 0; ++jj, dst += ldo, shr = (shr + d4) & 3u) {
                        const int sh = (int)shr;
                        const int h = min((4 - sh) & 3, nv);    // elements before the first aligned one
                        const int nb = (nv - h) >> 2;           // aligned groups of four
                        const int t0 = h + 4 * nb;              // first element of the tail
                        const float* row = stg + (j0 + jj) * kStgPitch + sh;
                        if (lane < h) dst[lane] = row[lane];
                        if (lane < nb)
                            *reinterpret_cast<float4*>(dst + h + 4 * lane) =
                                *reinterpret_cast<const float4*>(row + h + 4 * lane);
                        if (lane < nv - t0) dst[t0 + lane] = row[t0 + lane];
                    }
                }
            } else {
                int s0i[C::CW];        // sum over K blocks of E0 (exact integers)
                float s1f[C::CW];      // sum over K blocks of E1 + 2^-11 E2
#pragma unroll
                for (int j = 0; j < C::CW; ++j) {
                    s0i[j] = 0;
                    s1f[j] = 0.0f;
                }
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!kl_warp_wait(tfull + tb, tphase, abort, err, timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = tmem + lane_base + (uint32_t)(tb * C::NACC * TN + c * C::CW);
                    uint32_t r0[C::CW], r1[C::CW], r2[C::CW];
                    tmem_ld_x16(base, r0);
                    tmem_ld_x16(base + (uint32_t)TN, r1);
                    tmem_ld_x16(base + (uint32_t)(2 * TN), r2);
                    tmem_wait_ld();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty + tb);
                    if (++tb == 2) {
                        tb = 0;
                        tphase ^= 1u;
                    }
#pragma unroll
                    for (int j = 0; j < C::CW; ++j) {
                        s0i[j] += __float2int_rn(__uint_as_float(r0[j]));
                        s1f[j] = __fmaf_rn(__uint_as_float(r2[j]), 1.0f / 2048.0f,
                                           __fadd_rn(s1f[j], __uint_as_float(r1[j])));
                    }
                }
                if (!ok) break;
                const int evv = ev[v < Vpad ? v : Vpad - 1];
                // lane l holds the exponent of sample sc0 + l; sample j's is taken from lane j
                const int esl = es[min(sc0 + lane, Spad - 1)];
                Out* p = out + (size_t)sc0 * ldo + v;
                const int jend = min(C::CW, S - sc0);
#pragma unroll
                for (int j = 0; j < C::CW; ++j, p += ldo) {
                    const int sc = __shfl_sync(0xffffffffu, esl, j) + evv - 18;
                    // float-float of the integer sum (up to 2^26) plus the FP32 correction sum
                    const int ii = s0i[j];
                    const float ih = (float)ii;
                    const float il = (float)(ii - (int)ih);
                    float h, e2;
                    ff_two_sum(ih, s1f[j], h, e2);
                    float lh, ll;
                    ff_fast_two_sum(h, __fadd_rn(e2, il), lh, ll);
                    lh = scale2(lh, sc);
                    ll = scale2(ll, sc);
                    float ah, al;
                    ff_exp(lh, ll, ffx, ffx_th, ffx_tl, ah, al);
                    if (j < jend && v < V) *p = ff_to_double(ah, al);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lay::kTmemCols)
                     : "memory");
    }
}

// xi (FP64 [S][K]) -> split FP16 operand [2][Spad][Kpad] (hi rows, then lo rows).
__global__ void split_xi_kernel(int S, int K, int Spad, int Kpad, const double* __restrict__ xi,
                                __half* __restrict__ a16) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Spad * Kpad) return;
    const int s = (int)(idx / Kpad), k = (int)(idx % Kpad);
    const double x = (s < S && k < K) ? xi[(size_t)s * K + k] : 0.0;
    const __half hi = __double2half(x);
    a16[idx] = hi;
    a16[(size_t)Spad * Kpad + idx] = __double2half((x - (double)__half2float(hi)) * 2048.0);
}

// Exact-lead slices of a row x[0..K) (FP64, read with stride `stride`): scale 2^-e with
// max |x_k| 2^-e in [1/2, 1) (e = 0 for an all-zero row), X = x 2^(9 - e), lead = rint(X),
// h = fp16(X - lead), l = fp16((X - lead - h) 2^11); written to out[q * slice + k], q = 0, 1, 2.
// One warp per row.
__device__ __forceinline__ void exact_slices_row(const double* x, long long stride, int K, int Kpad, __half* out,
                                                 size_t slice, int* e_out) {
    const int lane = threadIdx.x & 31;
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(x[(long long)k * stride]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);   // mx = f 2^e, f in [1/2, 1)
    const double sc = ldexp(1.0, 9 - e);
    for (int k = lane; k < Kpad; k += 32) {
        const double X = k < K ? x[(long long)k * stride] * sc : 0.0;
        const double lead = rint(X);
        const double rem = X - lead;                      // exact: |rem| <= 1/2
        const __half h = __double2half(rem);
        const __half l = __double2half((rem - (double)__half2float(h)) * 2048.0);
        out[k] = __double2half(lead);                    // |lead| <= 512: exact
        out[slice + k] = h;
        out[2 * slice + k] = l;
    }
    if (lane == 0) *e_out = e;
}

// xi (FP64 [S][K]) -> exact-lead operand [3][Spad][Kpad] and row exponents es[Spad].
__global__ void split_xi_exact_kernel(int S, int K, int Spad, int Kpad, const double* __restrict__ xi,
                                      __half* __restrict__ a16, int* __restrict__ es) {
    const int s = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (s >= Spad) return;
    const size_t slice = (size_t)Spad * Kpad;
    if (s < S) {
        exact_slices_row(xi + (size_t)s * K, 1, K, Kpad, a16 + (size_t)s * Kpad, slice, es + s);
    } else {
        const int lane = threadIdx.x & 31;
        for (int k = lane; k < Kpad; k += 32) {
            a16[(size_t)s * Kpad + k] = __float2half(0.0f);
            a16[slice + (size_t)s * Kpad + k] = __float2half(0.0f);
            a16[2 * slice + (size_t)s * Kpad + k] = __float2half(0.0f);
        }
        if (lane == 0) es[s] = 0;
    }
}

// Basis columns Phi[.][v] (FP64 [K][ld64]) -> exact-lead operand [3][Vpad][Kpad] and node exponents ev[Vpad].
__global__ void split_basis_exact_kernel(int K, int Kpad, int V, int Vpad, int ld64, const double* __restrict__ phi64,
                                         __half* __restrict__ b16, int* __restrict__ ev) {
    const int v = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (v >= Vpad) return;
    // padding nodes (v >= V) are zero columns of phi64
    exact_slices_row(phi64 + v, ld64, K, Kpad, b16 + (size_t)v * Kpad, (size_t)Vpad * Kpad, ev + v);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2D FP16 tensor [rows][cols] (cols contiguous), box {64, box_rows}, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * sizeof(__half)};
    const cuuint32_t box[2] = {TKB, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tang's tables in float-float, from long-double host arithmetic.
FFExp make_ffexp() {
    FFExp T;
    for (int j = 0; j < 32; ++j) {
        const long double t = std::exp2((long double)j / 32.0L);
        T.th[j] = (float)t;
        T.tl[j] = (float)(t - (long double)T.th[j]);
    }
    const long double L = std::log(2.0L) / 32.0L;
    // l1: L rounded to 12 significant bits (so that N l1 is exact for |N| < 2^12)
    int e = 0;
    const long double f = std::frexp(L, &e);               // L = f 2^e, f in [1/2, 1)
    const long double l1 = std::ldexp(std::round(std::ldexp(f, 12)), e - 12);
    T.l1 = (float)l1;
    T.l2 = (float)(L - l1);
    T.l3 = (float)(L - l1 - (long double)T.l2);
    T.inv = (float)(1.0L / L);
    return T;
}

template <int MODE>
cudaError_t kl_launch(mlmc_ctx* ctx, int S, int Spad, int Kpad, int nodes, int nodes_pad, const void* aops,
                      const void* bops, const int* es, const int* ev, void* out, long long ldo, cudaStream_t st) {
    using C = KLCfg<MODE>;
    using Lay = KLLayout<MODE>;
    // MMA operand A: the basis slices (128 node rows), B: the xi slices (TN sample rows)
    CUtensorMap mapA, mapB;
    if (!make_map(&mapA, bops, (uint64_t)C::NA * nodes_pad, (uint64_t)Kpad, TM) ||
        !make_map(&mapB, aops, (uint64_t)C::NB * Spad, (uint64_t)Kpad, C::TN))
        return cudaErrorInvalidValue;
    static bool attr = false;
    cudaError_t e;
    if (!attr) {
        if ((e = cudaFuncSetAttribute(kl_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)Lay::kSmem)) != cudaSuccess)
            return e;
        attr = true;
    }
    static const FFExp ffx = make_ffexp();
    const int num_st = Spad / C::TN;
    const int num_tiles = num_st * (nodes_pad / TM);
    const int grid = num_tiles < ctx->num_sms ? num_tiles : ctx->num_sms;
    Profile::Pending pend;
    if (ctx->prof.on) {
        if ((e = cudaEventCreate(&pend.a)) != cudaSuccess) return e;
        if ((e = cudaEventCreate(&pend.b)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(pend.a, st)) != cudaSuccess) return e;
    }
    kl_tc_kernel<MODE><<<(unsigned)grid, Lay::kThreads, Lay::kSmem, st>>>(
        mapA, mapB, S, Spad, nodes, nodes_pad, Kpad, num_st, num_tiles, std::max(1, grid / 8), es, ev, ffx,
        static_cast<typename C::Out*>(out), ldo, ctx->kl_err, (unsigned long long)(ctx->wait_timeout_s * 1e9),
        16u * (unsigned)ctx->wait_extra);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ctx->prof.on) {
        if ((e = cudaEventRecord(pend.b, st)) != cudaSuccess) return e;
        // written output, one read of both operands' slices (and the exponents)
        pend.bytes = (double)S * nodes * sizeof(typename C::Out) + (double)C::NA * Spad * Kpad * 2.0 +
                     (double)C::NB * nodes_pad * Kpad * 2.0 + (MODE == 1 ? 4.0 * (Spad + nodes_pad) : 0.0);
        const int mmas = MODE == 1 ? 8 : 3;   // MMAs per 16-term step
        pend.flops = 2.0 * mmas * Spad * (double)Kpad * nodes_pad;
        ctx->prof.kl_pending.push_back(pend);
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_kl_fp32(mlmc_ctx* ctx, const GridBasis& gb, int S, const double* xi, float* a, long long ld,
                           cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(a) % sizeof(float) != 0) return cudaErrorMisalignedAddress;
    const int Spad = (S + TM - 1) / TM * TM;
    const int Kpad = gb.Kpad;
    cudaError_t e = ctx->ws.split.reserve((size_t)2 * Spad * Kpad * sizeof(__half));
    if (e != cudaSuccess) return e;
    __half* a16 = ctx->ws.split.as<__half>();
    const long long work = (long long)Spad * Kpad;
    split_xi_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(S, gb.K, Spad, Kpad, xi, a16);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // rows of whole 128-byte lines take the direct-store form
    if (ld % 32 == 0 && reinterpret_cast<uintptr_t>(a) % 128 == 0)
        return kl_launch<2>(ctx, S, Spad, Kpad, gb.nodes, gb.nodes_pad, a16, gb.phi16.ptr, nullptr, nullptr, a, ld, st);
    return kl_launch<0>(ctx, S, Spad, Kpad, gb.nodes, gb.nodes_pad, a16, gb.phi16.ptr, nullptr, nullptr, a, ld, st);
}

cudaError_t launch_kl_tc64(mlmc_ctx* ctx, GridBasis& gb, int S, const double* xi, double* a, long long ld,
                           cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    cudaError_t e;
    if (!gb.phix.ptr) {
        // exact-lead basis slices and node exponents, built once per grid from the FP64 basis
        if ((e = gb.phix.reserve((size_t)3 * gb.nodes_pad * gb.Kpad * sizeof(__half))) != cudaSuccess) return e;
        if ((e = gb.ev.reserve((size_t)gb.nodes_pad * sizeof(int))) != cudaSuccess) {
            gb.phix.release();
            return e;
        }
        const long long threads = (long long)gb.nodes_pad * 32;
        split_basis_exact_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
            gb.K, gb.Kpad, gb.nodes, gb.nodes_pad, gb.nodes_pad, gb.phi64.as<double>(), gb.phix.as<__half>(),
            gb.ev.as<int>());
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int Spad = (S + TM - 1) / TM * TM;
    const int Kpad = gb.Kpad;
    const size_t abytes = ((size_t)3 * Spad * Kpad * sizeof(__half) + 255) / 256 * 256;
    if ((e = ctx->ws.split.reserve(abytes + (size_t)Spad * sizeof(int))) != cudaSuccess) return e;
    __half* a16 = ctx->ws.split.as<__half>();
    int* es = reinterpret_cast<int*>(ctx->ws.split.as<char>() + abytes);
    const long long threads = (long long)Spad * 32;
    split_xi_exact_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(S, gb.K, Spad, Kpad, xi, a16, es);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return kl_launch<1>(ctx, S, Spad, Kpad, gb.nodes, gb.nodes_pad, a16, gb.phix.ptr, es, gb.ev.as<int>(), a, ld, st);
}

}  // namespace mlmc
