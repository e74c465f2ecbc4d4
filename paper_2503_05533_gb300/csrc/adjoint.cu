// A12: element part of the QoI gradient.
//
// With A x = b, A lambda = g (A symmetric) and Q = g^T x, dQ = -lambda^T dA x.
// A = sum_T a_T Khat_T with a_T the mean of T's vertex values, so
//   dQ/da_v = G_v = -(1/3) sum_{T contains v} |T| grad(lambda_h).grad(u_h)|_T,
// and with a_v = exp(sum_k xi_k Phi_k(v)), dQ/dxi_k = sum_v Phi_k(v) a_v G_v
// (the transposed KL contraction, kl_synth.cu).  This kernel forms
// w[s][v] = a_v G_v on every node v of the (n+1)^2 grid, in FP64, and stores it as
// a float-float pair (hi = w rounded to FP32, lo = the remainder rounded to FP32; 48
// significant bits) for the contraction, which runs on the FP32 pipe.
//
// On the right triangles T1(i,j) = (SW, SE, NE) and T2(i,j) = (SW, NE, NW) of
// cell (i,j) with legs h, |T| grad(l).grad(u) = 1/2 (sum over the two legs of
// the products of the leg differences).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {
namespace {

__device__ __forceinline__ double leg_energy_t1(const double* u, const double* l, int n, int i, int j) {
    // cell (i,j): SW = (i,j), SE = (i+1,j), NE = (i+1,j+1)
    const int w = n + 1;
    const double uSW = u[j * w + i], uSE = u[j * w + i + 1], uNE = u[(j + 1) * w + i + 1];
    const double lSW = l[j * w + i], lSE = l[j * w + i + 1], lNE = l[(j + 1) * w + i + 1];
    return 0.5 * ((lSE - lSW) * (uSE - uSW) + (lNE - lSE) * (uNE - uSE));
}

__device__ __forceinline__ double leg_energy_t2(const double* u, const double* l, int n, int i, int j) {
    // cell (i,j): SW = (i,j), NE = (i+1,j+1), NW = (i,j+1)
    const int w = n + 1;
    const double uSW = u[j * w + i], uNE = u[(j + 1) * w + i + 1], uNW = u[(j + 1) * w + i];
    const double lSW = l[j * w + i], lNE = l[(j + 1) * w + i + 1], lNW = l[(j + 1) * w + i];
    return 0.5 * ((lNE - lNW) * (uNE - uNW) + (lNW - lSW) * (uNW - uSW));
}

__global__ void adjoint_elements_kernel(int n, int S, const void* a, int a_fp64, const double* __restrict__ u,
                                        const double* __restrict__ lam, float* __restrict__ wff) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int V = (n + 1) * (n + 1);
    if (tid >= (long long)S * V) return;
    const int s = (int)(tid / V);
    const int v = (int)(tid - (long long)s * V);
    const int i = v % (n + 1), j = v / (n + 1);
    const double* us = u + (size_t)s * V;
    const double* ls = lam + (size_t)s * V;
    double e = 0.0;
    const bool hasE = i < n, hasW = i > 0, hasN = j < n, hasS = j > 0;
    if (hasE && hasN) e += leg_energy_t1(us, ls, n, i, j) + leg_energy_t2(us, ls, n, i, j);      // NE cell
    if (hasW && hasN) e += leg_energy_t1(us, ls, n, i - 1, j);                                   // NW cell
    if (hasW && hasS) e += leg_energy_t1(us, ls, n, i - 1, j - 1) + leg_energy_t2(us, ls, n, i - 1, j - 1);  // SW
    if (hasE && hasS) e += leg_energy_t2(us, ls, n, i, j - 1);                                   // SE cell
    const double av = a_fp64 ? static_cast<const double*>(a)[(size_t)s * V + v]
                             : (double)static_cast<const float*>(a)[(size_t)s * V + v];
    const double wv = -av * e * (1.0 / 3.0);
    const float hi = __double2float_rn(wv);
    wff[(size_t)s * V + v] = hi;
    wff[(size_t)S * V + (size_t)s * V + v] = __double2float_rn(wv - (double)hi);
}

}  // namespace

cudaError_t launch_adjoint_elements(int n, int S, const void* a, int a_fp64, const double* u, const double* lam,
                                    float* G, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const long long work = (long long)S * (n + 1) * (n + 1);
    adjoint_elements_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(n, S, a, a_fp64, u, lam, G);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mlmc
