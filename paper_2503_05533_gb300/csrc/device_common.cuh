// Device helpers shared by the libmlmc kernels: the global timer for bounded
// waits, mbarriers and bulk asynchronous copies, and 4-wide loads of the
// storage types.
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

// ---------------------------------------------------------------------------
// mbarriers and bulk asynchronous copies (the TMA engine).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// One arrival that also raises the phase's expected transaction count by `bytes`.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// True once the phase of parity `phase` has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase has not completed within timeout_ns of wall time.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint64_t timeout_ns) {
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, phase))
        if (global_ns() - t0 > timeout_ns) return false;
    return true;
}
// Copy `bytes` (a multiple of 16; both addresses 16-byte aligned) from global
// memory into this CTA's shared memory; completion is counted in bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Orders this thread's earlier global writes (generic proxy) before later bulk
// copies (async proxy) that read them.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Storage types of the nodal coefficient and vectors: 4 consecutive values
// starting at a 4-aligned index, widened to the compute type.
//
// Cache policy.  Vectors that the solve rewrites (x, r, p, d) are read with
// ordinary L1-cached loads: every system is solved by threads of one CTA, no
// phase reads a location that another thread writes in the same phase, and the
// CTA barrier between phases orders global memory for the whole CTA.  The
// coefficient and its inverse diagonal are read-only after set-up and use the
// read-only path.
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

// Storage-type values from shared memory (same conversions as CoefLoad).
template <class ST, class CT> struct SmemLoad;
template <class CT> struct SmemLoad<double, CT> {
    static __device__ __forceinline__ void load4(const double* p, CT v[4]) {
        const double2 a = *reinterpret_cast<const double2*>(p);
        const double2 b = *(reinterpret_cast<const double2*>(p) + 1);
        v[0] = (CT)a.x; v[1] = (CT)a.y; v[2] = (CT)b.x; v[3] = (CT)b.y;
    }
    static __device__ __forceinline__ CT load1(const double* p) { return (CT)*p; }
};
template <class CT> struct SmemLoad<float, CT> {
    static __device__ __forceinline__ void load4(const float* p, CT v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = (CT)q.x; v[1] = (CT)q.y; v[2] = (CT)q.z; v[3] = (CT)q.w;
    }
    static __device__ __forceinline__ CT load1(const float* p) { return (CT)*p; }
};
template <class CT> struct SmemLoad<__half, CT> {
    static __device__ __forceinline__ void load4(const __half* p, CT v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        v[0] = (CT)a.x; v[1] = (CT)a.y; v[2] = (CT)b.x; v[3] = (CT)b.y;
    }
    static __device__ __forceinline__ CT load1(const __half* p) { return (CT)__half2float(*p); }
};
template <class CT> struct SmemLoad<__nv_bfloat16, CT> {
    static __device__ __forceinline__ void load4(const __nv_bfloat16* p, CT v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q.y));
        v[0] = (CT)a.x; v[1] = (CT)a.y; v[2] = (CT)b.x; v[3] = (CT)b.y;
    }
    static __device__ __forceinline__ CT load1(const __nv_bfloat16* p) { return (CT)__bfloat162float(*p); }
};

// ---------------------------------------------------------------------------
// Float-float arithmetic: a value h + l with |l| <= ulp(h) / 2 (about 48 significant bits) on
// the FP32 pipe, GB300's FP64 pipe being narrow.  Error-free transformations (Knuth's TwoSum,
// Dekker's FastTwoSum, the FMA product error) with explicit round-to-nearest operations, which
// the compiler never contracts.
struct __align__(8) ff2 {
    float h, l;
};
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b| or a = 0
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void ff_two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ ff2 ff_add(ff2 a, ff2 b) {
    float s, e, h, l;
    ff_two_sum(a.h, b.h, s, e);
    ff_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.l, b.l)), h, l);
    return {h, l};
}
__device__ __forceinline__ ff2 ff_neg(ff2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff2 ff_sub(ff2 a, ff2 b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff2 ff_mul(ff2 a, ff2 b) {
    float p, e, h, l;
    ff_two_prod(a.h, b.h, p, e);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    ff_fast_two_sum(p, e, h, l);
    return {h, l};
}
__device__ __forceinline__ ff2 ff_add_f(ff2 a, float b) {
    float s, e, h, l;
    ff_two_sum(a.h, b, s, e);
    ff_fast_two_sum(s, __fadd_rn(e, a.l), h, l);
    return {h, l};
}
// Nearest float-float of a double (two conversions and a subtraction on the FP64 pipe).
__device__ __forceinline__ ff2 ff_from_d(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double ff_to_d(ff2 a) { return (double)a.h + (double)a.l; }

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
