// A1: random inputs xi[s][k] ~ N(0,1) of the KL expansion.
//
// The paper draws omega_j ~ N(0, sigma^2) (Sec. 5.1, Eq. (5.2)) and reuses a
// draw for both members of Y_l = Q_l - Q_{l-1} (Sec. 4.1, Eq. (4.1)).  Here a
// counter-based generator makes sample k of level l reproducible from
// (seed, l, k) alone:
//   Philox4x32-10 (Salmon et al., SC'11), key (seed lo, seed hi),
//   counter (k lo, k hi, l, j >> 1); words (0,1) for even j, (2,3) for odd j;
//   u = (M + 1/2) 2^-52 with the 52-bit M = (w_a << 20) | (w_b >> 12);
//   xi = AS241(u) (Wichura, Applied Statistics 37 (1988)), whose tail uses a
//   log written out from log m = 2 atanh((m-1)/(m+1)).
// Every FP64 operation is an explicit round-to-nearest intrinsic, so the
// compiler cannot fuse them and the bits are fixed by the operation sequence.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mlmc {
namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kM0, c[0]), lo0 = kM0 * c[0];
        const uint32_t hi1 = __umulhi(kM1, c[2]), lo1 = kM1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += kW0; k1 += kW1;
    }
}

__device__ __forceinline__ double uniform52(uint32_t wa, uint32_t wb) {
    const uint64_t m = ((uint64_t)wa << 20) | (uint64_t)(wb >> 12);
    return __dmul_rn(__dadd_rn((double)m, 0.5), 0x1p-52);
}

// log x for 0 < x <= 1; same operation sequence as the oracle's log_series.
__device__ __forceinline__ double log_series(double x) {
    const double kLn2Hi = 0x1.62e42fee00000p-1;
    const double kLn2Lo = 0x1.a39ef35793c76p-33;
    const double kSqrt2 = 0x1.6a09e667f3bcdp+0;
    const double c[11] = {0x1.5555555555555p-2, 0x1.999999999999ap-3, 0x1.2492492492492p-3,
                          0x1.c71c71c71c71cp-4, 0x1.745d1745d1746p-4, 0x1.3b13b13b13b14p-4,
                          0x1.1111111111111p-4, 0x1.e1e1e1e1e1e1ep-5, 0x1.af286bca1af28p-5,
                          0x1.8618618618618p-5, 0x1.642c8590b2164p-5};   // 1/3, 1/5, ..., 1/23
    int e;
    double m = frexp(x, &e);          // exact: m in [0.5, 1)
    m = __dmul_rn(m, 2.0);
    e -= 1;
    if (m > kSqrt2) {
        m = __dmul_rn(m, 0.5);
        e += 1;
    }
    const double f = __dsub_rn(m, 1.0);
    const double s = __ddiv_rn(f, __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    double p = c[10];
#pragma unroll
    for (int i = 9; i >= 0; --i) {
        p = __dmul_rn(p, z);
        p = __dadd_rn(p, c[i]);
    }
    const double t = __dadd_rn(s, s);
    const double zp = __dmul_rn(z, p);
    double lm = __dmul_rn(t, zp);
    lm = __dadd_rn(t, lm);
    const double de = (double)e;
    lm = __dadd_rn(lm, __dmul_rn(de, kLn2Lo));
    return __dadd_rn(__dmul_rn(de, kLn2Hi), lm);
}

__device__ __forceinline__ double horner8(const double* k, double r) {
    double p = k[7];
#pragma unroll
    for (int i = 6; i >= 0; --i) {
        p = __dmul_rn(p, r);
        p = __dadd_rn(p, k[i]);
    }
    return p;
}

__device__ double as241(double u) {
    const double A[8] = {3.3871328727963666080e0, 1.3314166789178437745e+2, 1.9715909503065514427e+3,
                         1.3731693765509461125e+4, 4.5921953931549871457e+4, 6.7265770927008700853e+4,
                         3.3430575583588128105e+4, 2.5090809287301226727e+3};
    const double B[8] = {1.0, 4.2313330701600911252e+1, 6.8718700749205790830e+2, 5.3941960214247511077e+3,
                         2.1213794301586595867e+4, 3.9307895800092710610e+4, 2.8729085735721942674e+4,
                         5.2264952788528545610e+3};
    const double C[8] = {1.42343711074968357734e0, 4.63033784615654529590e0, 5.76949722146069140550e0,
                         3.64784832476320460504e0, 1.27045825245236838258e0, 2.41780725177450611770e-1,
                         2.27238449892691845833e-2, 7.74545014278341407640e-4};
    const double D[8] = {1.0, 2.05319162663775882187e0, 1.67638483018380384940e0, 6.89767334985100004550e-1,
                         1.48103976427480074590e-1, 1.51986665636164571966e-2, 5.47593808499534494600e-4,
                         1.05075007164441684324e-9};
    const double E[8] = {6.65790464350110377720e0, 5.46378491116411436990e0, 1.78482653991729133580e0,
                         2.96560571828504891230e-1, 2.65321895265761230930e-2, 1.24266094738807843860e-3,
                         2.71155556874348757815e-5, 2.01033439929228813265e-7};
    const double F[8] = {1.0, 5.99832206555887937690e-1, 1.36929880922735805310e-1, 1.48753612908506148525e-2,
                         7.86869131145613259100e-4, 1.84631831751005468180e-5, 1.42151175831644588870e-7,
                         2.04426310338993978564e-15};
    const double q = __dsub_rn(u, 0.5);
    if (fabs(q) <= 0.425) {
        const double r = __dsub_rn(0.180625, __dmul_rn(q, q));
        const double num = __dmul_rn(q, horner8(A, r));
        return __ddiv_rn(num, horner8(B, r));
    }
    double r = (q < 0.0) ? u : __dsub_rn(1.0, u);
    r = __dsqrt_rn(-log_series(r));
    double z;
    if (r <= 5.0) {
        const double rn = __dsub_rn(r, 1.6);
        z = __ddiv_rn(horner8(C, rn), horner8(D, rn));
    } else {
        const double rf = __dsub_rn(r, 5.0);
        z = __ddiv_rn(horner8(E, rf), horner8(F, rf));
    }
    return (q < 0.0) ? -z : z;
}

// One thread per (sample, pair of terms).
__global__ void __launch_bounds__(256) philox_normal_kernel(uint64_t seed, uint32_t level, uint64_t first,
                                                            int S, int K, double* __restrict__ xi) {
    const int pairs = (K + 1) >> 1;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)S * pairs) return;
    const int s = (int)(tid / pairs);
    const int jp = (int)(tid - (long long)s * pairs);
    const uint64_t k = first + (uint64_t)s;
    uint32_t c[4] = {(uint32_t)(k & 0xFFFFFFFFu), (uint32_t)(k >> 32), level, (uint32_t)jp};
    philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    const int j0 = 2 * jp;
    double* row = xi + (size_t)s * K;
    row[j0] = as241(uniform52(c[0], c[1]));
    if (j0 + 1 < K) row[j0 + 1] = as241(uniform52(c[2], c[3]));
}

}  // namespace

cudaError_t launch_philox_normals(uint64_t seed, int level, uint64_t first, int S, int K, double* xi,
                                  cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const long long work = (long long)S * ((K + 1) / 2);
    const int block = 256;
    const long long grid = (work + block - 1) / block;
    philox_normal_kernel<<<(unsigned)grid, block, 0, st>>>(seed, (uint32_t)level, first, S, K, xi);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mlmc
