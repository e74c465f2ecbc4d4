// A2: KL synthesis of the coefficient, a[s][v] = exp(sum_k xi[s][k] Phi[k][v]).
//
// This file holds the basis expansion on the device, the FP64 contraction
// (plain FP64 form; GB300's FP64 rate makes it ALU-bound) and the transposed
// contraction used by the adjoint gradient (float-float on the FP32 pipe).  The
// tensor-core forms are in kl_tc.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
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

// Phi as float-float rows: phiff[k][v] = hi, phiff[K + k][v] = lo, Phi = hi + lo to 48 bits.
__global__ void split_phi_ff_kernel(int K, int Vpad, int ld64, const double* __restrict__ phi64,
                                    float* __restrict__ phiff) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)K * Vpad) return;
    const int k = (int)(tid / Vpad), v = (int)(tid - (long long)k * Vpad);
    const double x = phi64[(size_t)k * ld64 + v];
    const float hi = __double2float_rn(x);
    phiff[tid] = hi;
    phiff[(size_t)K * Vpad + tid] = __double2float_rn(x - (double)hi);
}

// (ah, al) += (wh + wl)(ph + pl) in float-float: the product of the leading parts exactly (an FMA
// recovers its rounding error), the two cross terms in FP32 (the lo * lo term, 2^-48 relative, dropped),
// the sum by Knuth's two-sum.
__device__ __forceinline__ void ff_mac(float& ah, float& al, float wh, float wl, float ph, float pl) {
    const float p = __fmul_rn(wh, ph);
    const float pe = __fmaf_rn(wh, ph, -p);
    const float t = __fmaf_rn(wh, pl, __fmaf_rn(wl, ph, pe));
    const float sum = __fadd_rn(ah, p);
    const float bb = __fsub_rn(sum, ah);
    const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
    ah = sum;
    al = __fadd_rn(al, __fadd_rn(err, t));
}

// The gradient's transposed contraction as a GEMM out (S x K) = w (S x V) Phi^T (V x K) on the FP32
// pipe in float-float arithmetic (GB300's FP64 pipe is narrow): a block computes a 64-sample x
// 64-term tile over its share of V (split-V), 32 nodes at a time staged in shared memory; a thread
// holds 4 x 4 float-float accumulators, renormalised after every 32 nodes.  The block writes its
// partial sums as FP64; kl_transpose_sum_kernel adds the splits in a fixed order.
constexpr int kTT = 64, kTV = 32, kTP = kTT + 4;   // tile, nodes per stage, staging pitch (16-byte rows)
__global__ void __launch_bounds__(256) kl_transpose_ff_kernel(int S, int K, int V, int Vpad, int vper,
                                                              const float* __restrict__ phiff,
                                                              const float* __restrict__ wff,
                                                              double* __restrict__ part) {
    __shared__ __align__(16) float sWh[kTV][kTP], sWl[kTV][kTP], sPh[kTV][kTP], sPl[kTV][kTP];
    const int k0 = blockIdx.x * kTT, s0 = blockIdx.y * kTT, split = blockIdx.z;
    const int vb = split * vper, ve = min(V, vb + vper);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const float* wh = wff;
    const float* wl = wff + (size_t)S * V;
    const float* ph = phiff;
    const float* pl = phiff + (size_t)K * Vpad;
    float ah[4][4], al[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ah[i][j] = 0.0f;
            al[i][j] = 0.0f;
        }
    for (int v0 = vb; v0 < ve; v0 += kTV) {
        __syncthreads();
        // 64 rows x 32 nodes of each array: a warp loads 32 consecutive nodes of one row
#pragma unroll
        for (int i = 0; i < (kTT * kTV) / 256; ++i) {
            const int e = t + 256 * i, r = e >> 5, vv = e & 31, v = v0 + vv;
            const bool vin = v < ve;
            const int s = s0 + r, k = k0 + r;
            sWh[vv][r] = (vin && s < S) ? wh[(size_t)s * V + v] : 0.0f;
            sWl[vv][r] = (vin && s < S) ? wl[(size_t)s * V + v] : 0.0f;
            sPh[vv][r] = (vin && k < K) ? ph[(size_t)k * Vpad + v] : 0.0f;
            sPl[vv][r] = (vin && k < K) ? pl[(size_t)k * Vpad + v] : 0.0f;
        }
        __syncthreads();
#pragma unroll 4
        for (int vv = 0; vv < kTV; ++vv) {
            const float4 wh4 = *reinterpret_cast<const float4*>(&sWh[vv][4 * ty]);
            const float4 wl4 = *reinterpret_cast<const float4*>(&sWl[vv][4 * ty]);
            const float4 ph4 = *reinterpret_cast<const float4*>(&sPh[vv][4 * tx]);
            const float4 pl4 = *reinterpret_cast<const float4*>(&sPl[vv][4 * tx]);
            const float whs[4] = {wh4.x, wh4.y, wh4.z, wh4.w}, wls[4] = {wl4.x, wl4.y, wl4.z, wl4.w};
            const float phs[4] = {ph4.x, ph4.y, ph4.z, ph4.w}, pls[4] = {pl4.x, pl4.y, pl4.z, pl4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) ff_mac(ah[i][j], al[i][j], whs[i], wls[i], phs[j], pls[j]);
        }
        // renormalise, so that al stays below half an ulp of ah
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float sum = __fadd_rn(ah[i][j], al[i][j]);
                al[i][j] = __fsub_rn(al[i][j], __fsub_rn(sum, ah[i][j]));
                ah[i][j] = sum;
            }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = s0 + 4 * ty + i, k = k0 + 4 * tx + j;
            if (s < S && k < K) part[((size_t)split * S + s) * K + k] = (double)ah[i][j] + (double)al[i][j];
        }
}

__global__ void kl_transpose_sum_kernel(int S, int K, int splits, const double* __restrict__ part,
                                        double* __restrict__ out) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= (long long)S * K) return;
    double acc = 0.0;
    for (int p = 0; p < splits; ++p) acc += part[(size_t)p * S * K + tid];
    out[tid] = acc;
}

}  // namespace

int kl_transpose_splits(int S, int K, int num_sms) {
    const int tiles = ((K + kTT - 1) / kTT) * ((S + kTT - 1) / kTT);
    return std::max(1, std::min(64, (4 * num_sms + tiles - 1) / tiles));
}

cudaError_t launch_kl_transpose_ff(GridBasis& gb, int S, const float* wff, double* part, int splits, double* out,
                                   cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    cudaError_t e;
    if (!gb.phiff.ptr) {
        if ((e = gb.phiff.reserve((size_t)2 * gb.K * gb.nodes_pad * sizeof(float))) != cudaSuccess) return e;
        const long long work = (long long)gb.K * gb.nodes_pad;
        split_phi_ff_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(gb.K, gb.nodes_pad, gb.nodes_pad,
                                                                          gb.phi64.as<double>(),
                                                                          gb.phiff.as<float>());
        g_launches.fetch_add(1, std::memory_order_relaxed);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int vper = ((gb.nodes + splits - 1) / splits + kTV - 1) / kTV * kTV;
    dim3 grid((gb.K + kTT - 1) / kTT, (S + kTT - 1) / kTT, splits);
    kl_transpose_ff_kernel<<<grid, 256, 0, st>>>(S, gb.K, gb.nodes, gb.nodes_pad, vper, gb.phiff.as<float>(), wff,
                                                part);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const long long outs = (long long)S * gb.K;
    kl_transpose_sum_kernel<<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(S, gb.K, splits, part, out);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
}

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


}  // namespace mlmc
