// A2: KL synthesis of the coefficient, a[s][v] = exp(sum_k xi[s][k] Phi[k][v]).
//
// This file holds the basis expansion on the device, the FP64 contraction
// (plain FP64 form; GB300's FP64 rate makes it ALU-bound) and the transposed
// contraction used by the adjoint gradient.  The tensor-core FP32 form is in
// kl_tc.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <vector>

#include "device_common.cuh"
#include "internal.h"

namespace mlmc {
namespace {

// Phi64[k][v] (row stride ld64) and the split FP16 operand phi16 = [hi; lo],
// each [Vpad][Kpad] (K contiguous): log2(e) Phi = hi + lo 2^-11.
__global__ void expand_basis_kernel(int n, int K, int Kpad, int V, int Vpad, int ld64,
                                    const double* __restrict__ coef, const double* __restrict__ bx,
                                    const double* __restrict__ by, double* __restrict__ phi64,
                                    __half* __restrict__ phi16) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)Vpad * Kpad) return;
    const int v = (int)(tid / Kpad);
    const int k = (int)(tid - (long long)v * Kpad);
    double phi = 0.0;
    if (v < V && k < K) {
        const int i = v % (n + 1), j = v / (n + 1);
        phi = coef[k] * bx[(size_t)k * (n + 1) + i] * by[(size_t)k * (n + 1) + j];
        phi64[(size_t)k * ld64 + v] = phi;
    }
    // the tensor-core FP32 synthesis contracts log2(e) Phi, so that its accumulators hold log2 a
    const double phi2 = phi * 1.4426950408889634;
    const __half hi = __double2half(phi2);
    const double rem = (phi2 - (double)__half2float(hi)) * 2048.0;
    phi16[tid] = hi;
    phi16[(size_t)Vpad * Kpad + tid] = __double2half(rem);
}

// out[s][v] = exp(sum_k xi[s][k] Phi[k][v]) in FP64.  Block (64, 4): thread
// (tx, ty) owns nodes 4 tx .. 4 tx + 3 of the block's 256 and samples
// 8 ty .. 8 ty + 7 of its 32.
template <class OutT>
__global__ void __launch_bounds__(256) kl_fp64_kernel(int S, int K, int V, int ld64,
                                                      const double* __restrict__ xi,
                                                      const double* __restrict__ phi,
                                                      OutT* __restrict__ out, long long ldo) {
    constexpr int KC = 32;
    __shared__ double sx[32][KC + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 64 + tx;
    const int v0 = blockIdx.x * 256 + 4 * tx;
    const int s0 = blockIdx.y * 32;
    double acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < K; k0 += KC) {
        __syncthreads();
        for (int e = tid; e < 32 * KC; e += 256) {
            const int ss = e / KC, kk = e % KC;
            const int s = s0 + ss, k = k0 + kk;
            sx[ss][kk] = (s < S && k < K) ? xi[(size_t)s * K + k] : 0.0;
        }
        __syncthreads();
        const int kend = min(KC, K - k0);
        for (int kk = 0; kk < kend; ++kk) {
            double p[4];
            Vec4<double>::load(phi + (size_t)(k0 + kk) * ld64 + v0, p);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const double x = sx[ty * 8 + a][kk];
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(x, p[b], acc[a][b]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int s = s0 + ty * 8 + a;
        if (s >= S) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int v = v0 + b;
            if (v < V) out[(size_t)s * ldo + v] = (OutT)exp(acc[a][b]);
        }
    }
}

// out[s][k] = sum_v Phi[k][v] w[s][v] (FP64).  Block of 256 threads handles
// 4 samples x 16 terms; threads stride over v; fixed-order reduction.
__global__ void __launch_bounds__(256) kl_transpose_kernel(int S, int K, int V, int ld64,
                                                           const double* __restrict__ phi,
                                                           const double* __restrict__ w,
                                                           double* __restrict__ out) {
    constexpr int SB = 4, KB = 16;
    __shared__ double red[8][SB][KB];
    const int s0 = blockIdx.y * SB, k0 = blockIdx.x * KB;
    double acc[SB][KB];
#pragma unroll
    for (int a = 0; a < SB; ++a)
#pragma unroll
        for (int b = 0; b < KB; ++b) acc[a][b] = 0.0;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        double wv[SB];
#pragma unroll
        for (int a = 0; a < SB; ++a) wv[a] = (s0 + a < S) ? w[(size_t)(s0 + a) * V + v] : 0.0;
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            const double p = (k0 + b < K) ? phi[(size_t)(k0 + b) * ld64 + v] : 0.0;
#pragma unroll
            for (int a = 0; a < SB; ++a) acc[a][b] = fma(p, wv[a], acc[a][b]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < SB; ++a)
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            double t = acc[a][b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[warp][a][b] = t;
        }
    __syncthreads();
    if (threadIdx.x < SB * KB) {
        const int a = threadIdx.x / KB, b = threadIdx.x % KB;
        double t = 0.0;
        for (int wi = 0; wi < 8; ++wi) t += red[wi][a][b];
        if (s0 + a < S && k0 + b < K) out[(size_t)(s0 + a) * K + k0 + b] = t;
    }
}

}  // namespace

cudaError_t upload_basis(GridBasis& gb, const mlmc_field& f, int n, std::string& err) {
    std::vector<double> coef, bx, by;
    if (!build_separable(f, n, coef, bx, by, err)) return cudaErrorInvalidValue;
    gb.n = n;
    gb.K = f.K;
    gb.nodes = (n + 1) * (n + 1);
    gb.nodes_pad = (gb.nodes + 255) / 256 * 256;
    gb.Kpad = (f.K + 63) / 64 * 64;
    cudaError_t e;
    if ((e = gb.phi64.reserve((size_t)gb.K * gb.nodes_pad * sizeof(double))) != cudaSuccess) return e;
    if ((e = gb.phi16.reserve((size_t)2 * gb.nodes_pad * gb.Kpad * sizeof(__half))) != cudaSuccess) return e;
    DevBuf tmp;
    const size_t nb = coef.size() + bx.size() + by.size();
    if ((e = tmp.reserve(nb * sizeof(double))) != cudaSuccess) return e;
    double* d = tmp.as<double>();
    e = cudaMemcpy(d, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d + coef.size(), bx.data(), bx.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d + coef.size() + bx.size(), by.data(), by.size() * sizeof(double),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(gb.phi64.ptr, 0, (size_t)gb.K * gb.nodes_pad * sizeof(double));
    if (e == cudaSuccess) {
        const long long work = (long long)gb.nodes_pad * gb.Kpad;
        expand_basis_kernel<<<(unsigned)((work + 255) / 256), 256>>>(
            n, gb.K, gb.Kpad, gb.nodes, gb.nodes_pad, gb.nodes_pad, d, d + coef.size(),
            d + coef.size() + bx.size(), gb.phi64.as<double>(), gb.phi16.as<__half>());
        g_launches.fetch_add(1, std::memory_order_relaxed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    tmp.release();
    return e;
}

template <class OutT>
static cudaError_t kl_fp64_launch(const GridBasis& gb, int S, const double* xi, OutT* a, long long ld,
                                  cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    dim3 block(64, 4);
    dim3 grid((gb.nodes + 255) / 256, (S + 31) / 32);
    kl_fp64_kernel<OutT><<<grid, block, 0, st>>>(S, gb.K, gb.nodes, gb.nodes_pad, xi, gb.phi64.as<double>(), a, ld);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

cudaError_t launch_kl_fp64(const GridBasis& gb, int S, const double* xi, double* a, long long ld, cudaStream_t st) {
    return kl_fp64_launch<double>(gb, S, xi, a, ld, st);
}

cudaError_t launch_kl_transpose_fp64(const GridBasis& gb, int S, const double* w, double* out,
                                     cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    dim3 grid((gb.K + 15) / 16, (S + 3) / 4);
    kl_transpose_kernel<<<grid, 256, 0, st>>>(S, gb.K, gb.nodes, gb.nodes_pad, gb.phi64.as<double>(), w, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

}  // namespace mlmc
