// A2 on the tensor cores: a[s][v] = exp(sum_k xi[s][k] Phi[k][v]) in FP32.
//
// The contraction (samples x KL terms) x (KL terms x nodes) runs on tcgen05
// with FP16 operands and FP32 accumulation.  FP16 alone would give ~1e-3
// relative error in log a, so both operands are split, x = hi + lo 2^-11
// (hi = fp16(x), lo = fp16((x - hi) 2^11), which keeps lo in FP16's normal
// range), and two TMEM accumulators hold
//   D1 = xi_hi Phi_hi^T,   D2 = xi_hi Phi_lo^T + xi_lo Phi_hi^T,
// so log a = D1 + 2^-11 D2 with the lo*lo term (2^-22 relative) dropped.
//
// One CTA computes a 128-sample x 128-node tile.  Thread 0 streams 64-term K
// blocks of the four operand tiles with TMA (128-byte swizzle) into shared
// memory and issues the MMAs (M = 128, N = 128, K = 16); tcgen05.commit
// signals completion through an mbarrier.  The four warps then read their 32
// TMEM lanes (one sample each), form exp(D1 + 2^-11 D2), and write the tile
// through a shared-memory transpose so that stores are row-contiguous.
// Every mbarrier wait is bounded in wall time; on expiry the CTA records an
// error word, waits (bounded) for its own copies in flight, frees its TMEM
// and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {
namespace {

constexpr int TM = 128;              // samples per tile (MMA M, TMEM lanes)
constexpr int TN = 128;              // nodes per tile (MMA N)
constexpr int TKB = 64;              // terms per K block: 64 FP16 = one 128-byte swizzle row
constexpr int kTmemCols = 256;       // D1 in columns [0, 128), D2 in [128, 256)
constexpr uint32_t kTileBytes = TM * TKB * 2;                  // 16 KiB (A tile; B tile is the same size)
constexpr uint32_t kOffAhi = 0, kOffAlo = kTileBytes, kOffBhi = 2 * kTileBytes, kOffBlo = 3 * kTileBytes;
constexpr uint32_t kOffStage = 4 * kTileBytes;                 // 4 warps x 32 x 33 floats
constexpr uint32_t kStageBytes = 4 * 32 * 33 * 4;
constexpr uint32_t kOffBar = kOffStage + kStageBytes;          // 2 mbarriers + TMEM slot + status
constexpr uint32_t kSmemBytes = kOffBar + 64 + 1024;           // + 1 KiB for 1024-byte alignment

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
// Instruction descriptor, kind::f16: D FP32, A and B FP16, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum));
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

__global__ void __launch_bounds__(128, 1) kl_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                                                       const __grid_constant__ CUtensorMap mapB, int S, int Spad,
                                                       int V, int Vpad, int Kpad, int num_m,
                                                       float* __restrict__ out, unsigned* err,
                                                       unsigned long long timeout_ns, unsigned extra_tx) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bar_full = reinterpret_cast<uint64_t*>(smem + kOffBar);
    uint64_t* bar_done = bar_full + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_full + 2);
    uint32_t* status = tmem_slot + 1;
    float* stage = reinterpret_cast<float*>(smem + kOffStage);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m_tile = blockIdx.x % num_m, n_tile = blockIdx.x / num_m;
    const int s0 = m_tile * TM, v0 = n_tile * TN;

    if (threadIdx.x == 0) {
        mbar_init(bar_full, 1);
        mbar_init(bar_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *status = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        const int nkb = Kpad / TKB;
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            mbar_expect_tx(bar_full, 4 * kTileBytes + extra_tx);
            tma_load_2d(smem + kOffAhi, &mapA, kb * TKB, s0, bar_full);
            tma_load_2d(smem + kOffAlo, &mapA, kb * TKB, Spad + s0, bar_full);
            tma_load_2d(smem + kOffBhi, &mapB, kb * TKB, v0, bar_full);
            tma_load_2d(smem + kOffBlo, &mapB, kb * TKB, Vpad + v0, bar_full);
            if (!mbar_wait(bar_full, (uint32_t)(kb & 1), timeout_ns)) {
                atomicCAS(err, KERR_NONE, KERR_TIMEOUT);
                mbar_wait(bar_full, (uint32_t)(kb & 1), timeout_ns);   // let in-flight copies land
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aH = smem_u32(smem + kOffAhi), aL = smem_u32(smem + kOffAlo);
            const uint32_t bH = smem_u32(smem + kOffBhi), bL = smem_u32(smem + kOffBlo);
#pragma unroll
            for (int k = 0; k < TKB / 16; ++k) {
                const uint32_t koff = (uint32_t)k * 32u;   // 16 FP16 = 32 bytes along the swizzled row
                const uint64_t dAH = desc_sw128(aH + koff), dAL = desc_sw128(aL + koff);
                const uint64_t dBH = desc_sw128(bH + koff), dBL = desc_sw128(bL + koff);
                const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
                mma_f16(tmem + 0, dAH, dBH, acc);
                mma_f16(tmem + TN, dAH, dBL, acc);
                mma_f16(tmem + TN, dAL, dBH, 1u);
            }
            mma_commit(bar_done);
            if (!mbar_wait(bar_done, (uint32_t)(kb & 1), timeout_ns)) {
                atomicCAS(err, KERR_NONE, KERR_TIMEOUT);
                mbar_wait(bar_done, (uint32_t)(kb & 1), timeout_ns);
                ok = false;
                break;
            }
        }
        *status = ok ? 1u : 0u;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (*status) {
        float* stg = stage + warp * 32 * 33;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int c = 0; c < TN / 32; ++c) {
            uint32_t r1[32], r2[32];
            tmem_ld_x32(tmem + lane_base + (uint32_t)(c * 32), r1);
            tmem_ld_x32(tmem + lane_base + (uint32_t)(TN + c * 32), r2);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float lg = __uint_as_float(r1[j]) + __uint_as_float(r2[j]) * (1.0f / 2048.0f);
                stg[lane * 33 + j] = expf(lg);
            }
            __syncwarp();
            const int v = v0 + c * 32 + lane;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const int s = s0 + warp * 32 + rr;
                if (s < S && v < V) out[(size_t)s * V + v] = stg[rr * 33 + lane];
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
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

// 2D FP16 tensor [rows][cols] (cols contiguous), box {64, 128}, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * sizeof(__half)};
    const cuuint32_t box[2] = {TKB, 128};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t launch_kl_fp32(mlmc_ctx* ctx, const GridBasis& gb, int S, const double* xi, float* a, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const int Spad = (S + TM - 1) / TM * TM;
    const int Kpad = gb.Kpad;
    // split operand + error word
    const size_t abytes = (size_t)2 * Spad * Kpad * sizeof(__half);
    cudaError_t e = ctx->ws.split.reserve(abytes + 256);
    if (e != cudaSuccess) return e;
    __half* a16 = ctx->ws.split.as<__half>();
    // the error word is the context's (cleared when the host reads it)
    unsigned* errw = ctx->kl_err;
    const long long work = (long long)Spad * Kpad;
    split_xi_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(S, gb.K, Spad, Kpad, xi, a16);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap mapA, mapB;
    if (!make_map(&mapA, a16, (uint64_t)2 * Spad, (uint64_t)Kpad) ||
        !make_map(&mapB, gb.phi16.ptr, (uint64_t)2 * gb.nodes_pad, (uint64_t)Kpad))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        if ((e = cudaFuncSetAttribute(kl_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes)) !=
            cudaSuccess)
            return e;
        attr = true;
    }
    const int num_m = Spad / TM;
    const int num_n = (gb.nodes + TN - 1) / TN;
    Profile::Pending pend;
    if (ctx->prof.on) {
        if ((e = cudaEventCreate(&pend.a)) != cudaSuccess) return e;
        if ((e = cudaEventCreate(&pend.b)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(pend.a, st)) != cudaSuccess) return e;
    }
    kl_tc_kernel<<<(unsigned)(num_m * num_n), 128, kSmemBytes, st>>>(
        mapA, mapB, S, Spad, gb.nodes, gb.nodes_pad, Kpad, num_m, a, errw,
        (unsigned long long)(ctx->wait_timeout_s * 1e9), 16u * (unsigned)ctx->wait_extra);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ctx->prof.on) {
        if ((e = cudaEventRecord(pend.b, st)) != cudaSuccess) return e;
        const double npad = (double)num_n * TN;
        pend.bytes = (double)S * gb.nodes * 4.0 + 2.0 * Spad * Kpad * 2.0 + 2.0 * (double)gb.nodes_pad * Kpad * 2.0;
        pend.flops = 6.0 * Spad * (double)Kpad * npad;
        ctx->prof.kl_pending.push_back(pend);
    }
    return cudaSuccess;
}

}  // namespace mlmc
