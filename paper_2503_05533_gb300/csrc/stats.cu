// A8: level statistics of Y_l = Q_l - Q_{l-1} (Sec. 4.1, Eq. (4.1)) for the
// sample mean Y_hat_l and s_l^2 = (1/N) sum (Y - Y_hat)^2 (Eq. (4.2)).
//
// One CTA: thread t takes a contiguous chunk of the batch and runs Welford's
// update plus compensated (TwoSum) sums of Y and Y^2; the 256 partial states
// are merged pairwise (Chan, Golub, LeVeque) in a fixed tree order, so the
// result does not depend on scheduling.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {
namespace {

struct Acc {
    double n, mean, m2, s, sc, q, qc;
};

__device__ __forceinline__ void two_sum_add(double& s, double& c, double x) {
    const double t = s + x;
    const double e = (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
    c += e;
}

__device__ __forceinline__ void acc_push(Acc& a, double y) {
    a.n += 1.0;
    const double d = y - a.mean;
    a.mean += d / a.n;
    a.m2 += d * (y - a.mean);
    two_sum_add(a.s, a.sc, y);
    two_sum_add(a.q, a.qc, __dmul_rn(y, y));
}

__device__ __forceinline__ Acc acc_merge_dev(const Acc& a, const Acc& b) {
    if (b.n == 0.0) return a;
    if (a.n == 0.0) return b;
    Acc r;
    r.n = a.n + b.n;
    const double d = b.mean - a.mean;
    r.mean = a.mean + d * (b.n / r.n);
    r.m2 = a.m2 + b.m2 + d * d * (a.n * b.n / r.n);
    r.s = a.s;
    r.sc = a.sc + b.sc;
    two_sum_add(r.s, r.sc, b.s);
    r.q = a.q;
    r.qc = a.qc + b.qc;
    two_sum_add(r.q, r.qc, b.q);
    return r;
}

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) level_stats_kernel(int S, const double* __restrict__ Qf,
                                                               const double* __restrict__ Qc,
                                                               mlmc_acc* __restrict__ out) {
    __shared__ Acc sh[kThreads];
    const int t = threadIdx.x;
    const int chunk = (S + kThreads - 1) / kThreads;
    const int lo = t * chunk, hi = min(S, lo + chunk);
    Acc a{0, 0, 0, 0, 0, 0, 0};
    for (int i = lo; i < hi; ++i) acc_push(a, Qf[i] - (Qc ? Qc[i] : 0.0));
    sh[t] = a;
    __syncthreads();
    for (int w = 1; w < kThreads; w <<= 1) {
        if ((t % (2 * w)) == 0) sh[t] = acc_merge_dev(sh[t], sh[t + w]);
        __syncthreads();
    }
    if (t == 0) {
        out->n = (int64_t)sh[0].n;
        out->mean = sh[0].mean;
        out->m2 = sh[0].m2;
        out->sum = sh[0].s;
        out->sum_c = sh[0].sc;
        out->sumsq = sh[0].q;
        out->sumsq_c = sh[0].qc;
    }
}

// Smallest and largest nodal coefficient of every sample (the contrast that bounds kappa(A): A is
// the P1 operator with element means of a, so min(a) L <= A <= max(a) L for the Laplacian L).
// One CTA per sample.
__global__ void __launch_bounds__(kThreads) field_range_kernel(int V, long long ld, const void* __restrict__ a,
                                                               int a_fp64, double* __restrict__ out) {
    __shared__ double smin[kThreads], smax[kThreads];
    const int s = blockIdx.x, t = threadIdx.x;
    double lo = INFINITY, hi = -INFINITY;
    for (int v = t; v < V; v += kThreads) {
        const size_t idx = (size_t)s * ld + v;
        const double x = a_fp64 ? static_cast<const double*>(a)[idx] : (double)static_cast<const float*>(a)[idx];
        lo = fmin(lo, x);
        hi = fmax(hi, x);
    }
    smin[t] = lo;
    smax[t] = hi;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (t < w) {
            smin[t] = fmin(smin[t], smin[t + w]);
            smax[t] = fmax(smax[t], smax[t + w]);
        }
        __syncthreads();
    }
    if (t == 0) {
        out[2 * s] = smin[0];
        out[2 * s + 1] = smax[0];
    }
}

}  // namespace

cudaError_t launch_field_range(int S, int V, long long ld, const void* a, int a_fp64, double* out_dev,
                               cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    field_range_kernel<<<S, kThreads, 0, st>>>(V, ld, a, a_fp64, out_dev);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_level_stats(int S, const double* Qf, const double* Qc, mlmc_acc* out_dev, cudaStream_t st) {
    level_stats_kernel<<<1, kThreads, 0, st>>>(S, Qf, Qc, out_dev);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mlmc
