// Device helpers shared by the libmlmc kernels: bounded grid barrier,
// deterministic block reductions and 4-wide loads of the storage types.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mlmc {

// Error codes a kernel can leave in its error word (host maps them to mlmc_status).
enum : unsigned { KERR_NONE = 0, KERR_TIMEOUT = 1, KERR_BAD_LAUNCH = 2 };

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// bar[0] = arrivals, bar[1] = generation, err = shared error word.
// Every wait is bounded by `timeout_ns` of wall time: on expiry the CTA sets
// KERR_TIMEOUT and returns false; every CTA then leaves the kernel at its next
// barrier (which also returns false once err is set).
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* err,
                                             uint64_t timeout_ns) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ok = 1;
        __threadfence();
        const unsigned gen = ld_acquire_u32(&bar[1]);
        __threadfence();
        const unsigned arrived = atomicAdd(&bar[0], 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            const uint64_t t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_u32(&bar[1]) == gen) {
                if (ld_acquire_u32(err) != KERR_NONE) break;
                if ((++spins & 63u) == 0u && global_ns() - t0 > timeout_ns) {
                    atomicCAS(err, KERR_NONE, KERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ld_acquire_u32(err) != KERR_NONE) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum of one double per thread over the block, fixed order (warp xor tree,
// then warps in index order).  Result valid in thread 0.
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* smem /* >= BLOCK/32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) smem[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < BLOCK / 32; ++i) t += smem[i];
    }
    __syncthreads();
    return t;
}

// Two sums at once (same order guarantees as block_sum).
template <int BLOCK>
__device__ __forceinline__ double2 block_sum2(double a, double b, double* smem /* >= BLOCK/16 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        smem[2 * w] = a;
        smem[2 * w + 1] = b;
    }
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < BLOCK / 32; ++i) {
            t.x += smem[2 * i];
            t.y += smem[2 * i + 1];
        }
    }
    __syncthreads();
    return t;
}

// Sum of a solve's per-tile partials, fixed order, computed by one warp; all
// lanes return the same value.  Every CTA that evaluates this for the same
// range gets the same bits.
__device__ __forceinline__ double warp_sum_partials(const double* part, int t0, int nt) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int t = lane; t < nt; t += 32) v += __ldcg(part + t0 + t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Storage types of the nodal coefficient and vectors: 4 consecutive values
// starting at a 4-aligned index, widened to the compute type.
//
// Cache policy.  Vectors that the persistent solve rewrites (x, r, p, d) are
// read with ordinary L1-cached loads: no phase reads a location that another
// CTA writes in the same phase, and the grid barrier between phases performs
// a gpu-scope acquire, which discards stale L1 lines.  The coefficient and its
// inverse diagonal are read-only after set-up and use the read-only path.
template <class T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float* p, const float v[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void load(const double* p, double v[4]) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double* p, const double v[4]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
        *(reinterpret_cast<double2*>(p) + 1) = make_double2(v[2], v[3]);
    }
};

// Coefficient storage (read-only while it is read): load 4 values of ST widened to CT.
template <class ST, class CT> struct CoefLoad;
template <class CT> struct CoefLoad<double, CT> {
    static __device__ __forceinline__ void load4(const double* p, CT v[4]) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        v[0] = (CT)a.x; v[1] = (CT)a.y; v[2] = (CT)b.x; v[3] = (CT)b.y;
    }
    static __device__ __forceinline__ CT load1(const double* p) { return (CT)__ldg(p); }
};
template <class CT> struct CoefLoad<float, CT> {
    static __device__ __forceinline__ void load4(const float* p, CT v[4]) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = (CT)q.x; v[1] = (CT)q.y; v[2] = (CT)q.z; v[3] = (CT)q.w;
    }
    static __device__ __forceinline__ CT load1(const float* p) { return (CT)__ldg(p); }
};
template <class CT> struct CoefLoad<__half, CT> {
    static __device__ __forceinline__ void load4(const __half* p, CT v[4]) {
        const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
        const __half2 lo = *reinterpret_cast<const __half2*>(&q.x);
        const __half2 hi = *reinterpret_cast<const __half2*>(&q.y);
        const float2 a = __half22float2(lo), b = __half22float2(hi);
        v[0] = (CT)a.x; v[1] = (CT)a.y; v[2] = (CT)b.x; v[3] = (CT)b.y;
    }
    static __device__ __forceinline__ CT load1(const __half* p) { return (CT)__half2float(__ldg(p)); }
};
template <class CT> struct CoefLoad<__nv_bfloat16, CT> {
    static __device__ __forceinline__ void load4(const __nv_bfloat16* p, CT v[4]) {
        const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
        const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
        const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
        const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
        v[0] = (CT)a.x; v[1] = (CT)a.y; v[2] = (CT)b.x; v[3] = (CT)b.y;
    }
    static __device__ __forceinline__ CT load1(const __nv_bfloat16* p) {
        return (CT)__bfloat162float(__ldg(p));
    }
};

// Widen one stored coefficient value (a register, not memory) to the compute type.
template <class CT> __device__ __forceinline__ CT widen(double v) { return (CT)v; }
template <class CT> __device__ __forceinline__ CT widen(float v) { return (CT)v; }
template <class CT> __device__ __forceinline__ CT widen(__half v) { return (CT)__half2float(v); }
template <class CT> __device__ __forceinline__ CT widen(__nv_bfloat16 v) { return (CT)__bfloat162float(v); }

template <class ST> __device__ __forceinline__ ST to_store(double v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __half to_store<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) {
    return __double2bfloat16(v);
}

}  // namespace mlmc
