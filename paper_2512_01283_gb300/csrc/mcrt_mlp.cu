// mcrt_mlp.cu -- learned surrogate of the grain optics (the paper's Sec. 2.2 allows
// the Mueller matrix to come from analytic forms, tables or neural networks; Sec. 4
// motivates networks for multi-dimensional grain optics).
//
// The network maps (n_i, n_s, s) -- incident and scattered directions in the grain
// frame and the position s in [-1, 1] of ln x between the first and last tabulated
// size parameter -- to 20 numbers: ln M11 of the 4x4 scattering matrix in the
// scattering-plane basis and its other 15 entries relative to M11 (the rotations into
// and out of the plane stay exact geometry in the kernels that use the network), the
// extinction elements alpha1..3 at the incident polar angle, and ln N(s), N(s) = max
// P11.  Architecture 16 (7 inputs, zero padded) -> 128 -> 128 ->
// 128 -> 128 -> 24 (20 used), SiLU; BF16 weights and activations, FP32 accumulation on
// the tensor cores (mma.sync m16n8k16), FP32 master weights and Adam.
//
// Training labels are generated on the GPU from the method's own tables, a fresh
// Philox-drawn batch every step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mcrt.h"
#include "mcrt_device.cuh"
#include "mcrt_internal.h"
#include "mcrt_mlp_infer.cuh"
#include "mcrt_mlp_tc.cuh"

namespace mcrt {
namespace {

typedef __nv_bfloat16 bf16;

using mlp::kHid;
using mlp::kIn;
using mlp::kInPad;
using mlp::kLayers;
using mlp::kOut;
using mlp::kOutPad;
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kInPad : kHid; }
__host__ __device__ constexpr int layer_out(int l) { return l == kLayers - 1 ? kOutPad : kHid; }
// parameter layout: per layer W [out][in] then b [out], layers in order
__host__ __device__ constexpr int layer_offset(int l) {
    int off = 0;
    for (int i = 0; i < l; ++i) off += layer_out(i) * layer_in(i) + layer_out(i);
    return off;
}
constexpr int kParams = layer_offset(kLayers);
__host__ __device__ constexpr int wbf_offset(int l) {
    int off = 0;
    for (int i = 0; i < l; ++i) off += layer_out(i) * layer_in(i);
    return off;
}
constexpr int kWeights = wbf_offset(kLayers);

// ---------------------------------------------------------------------------------
// training labels from the tables
// ---------------------------------------------------------------------------------
struct LabelTables {
    const float4* bins;  // [n_bins][n_theta][2] (P11,P12,P22,P33),(P34,P44,0,0)
    const float4* kext;  // [n_ktheta]
    int n_bins, n_theta, n_ktheta;
};

__device__ void interp_row(const LabelTables& T, int k, int j, float f, float w, float P[6]) {
    const float4 a0 = T.bins[((size_t)k * T.n_theta + j) * 2], a1 = T.bins[((size_t)k * T.n_theta + j) * 2 + 1];
    const float4 b0 = T.bins[((size_t)k * T.n_theta + j + 1) * 2], b1 = T.bins[((size_t)k * T.n_theta + j + 1) * 2 + 1];
    const float g = 1.f - f;
    P[0] += w * (g * a0.x + f * b0.x);
    P[1] += w * (g * a0.y + f * b0.y);
    P[2] += w * (g * a0.z + f * b0.z);
    P[3] += w * (g * a0.w + f * b0.w);
    P[4] += w * (g * a1.x + f * b1.x);
    P[5] += w * (g * a1.y + f * b1.y);
}

// 20 targets for (n_i, n_s, s): tables interpolated linearly in the scattering angle
// and in ln x between bins; the scattering-plane matrix M as ln M11 and M_rc / M11;
// alpha1..3; ln of the maximum interpolated P11.
__device__ void surrogate_label(const LabelTables& T, const V3<float>& ni, const V3<float>& ns, float s,
                                float out[kOut]) {
    // bins k and k1 = k + 1 around s (one bin: k = k1 = 0)
    int k = 0, k1 = 0;
    float fb = 0.f;
    if (T.n_bins > 1) {
        const float b = (fminf(fmaxf(s, -1.f), 1.f) + 1.f) * 0.5f * (float)(T.n_bins - 1);
        k = (int)floorf(b);
        k = k > T.n_bins - 2 ? T.n_bins - 2 : (k < 0 ? 0 : k);
        k1 = k + 1;
        fb = b - (float)k;
    }
    float N = 0.f;
    for (int j = 0; j < T.n_theta; ++j) {
        const float v = (1.f - fb) * T.bins[((size_t)k * T.n_theta + j) * 2].x +
                        fb * T.bins[((size_t)k1 * T.n_theta + j) * 2].x;
        N = fmaxf(N, v);
    }
    const float mu = fminf(fmaxf(dot(ni, ns), -1.f), 1.f);
    const float x = acosf(mu) * 0.31830988618379067f * (float)(T.n_theta - 1);
    int j = (int)floorf(x);
    j = j > T.n_theta - 2 ? T.n_theta - 2 : (j < 0 ? 0 : j);
    const float ft = x - (float)j;
    float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    interp_row(T, k, j, ft, 1.f - fb, P);
    interp_row(T, k1, j, ft, fb, P);
    // scattering-plane matrix [[P11,P12,0,0],[P12,P22,0,0],[0,0,P33,P34],[0,0,-P34,P44]]
    // as ln M11 and the entries relative to M11 (equal relative accuracy over the
    // decades that P11 spans)
    const float inv = 1.f / P[0];
    const float Z[16] = {P[0], P[1], 0.f, 0.f, P[1], P[2], 0.f, 0.f, 0.f, 0.f, P[3], P[4], 0.f, 0.f, -P[4], P[5]};
    out[0] = logf(P[0]);
    for (int k = 1; k < 16; ++k) out[k] = Z[k] * inv;
    const float xk = acosf(fminf(fmaxf(ni.z, -1.f), 1.f)) * 0.31830988618379067f * (float)(T.n_ktheta - 1);
    int jk = (int)floorf(xk);
    jk = jk > T.n_ktheta - 2 ? T.n_ktheta - 2 : (jk < 0 ? 0 : jk);
    const float fk = xk - (float)jk;
    const float4 ka = T.kext[jk], kb = T.kext[jk + 1];
    out[16] = (1.f - fk) * ka.x + fk * kb.x;
    out[17] = (1.f - fk) * ka.y + fk * kb.y;
    out[18] = (1.f - fk) * ka.z + fk * kb.z;
    out[19] = logf(N);
}

__device__ V3<float> iso_unit(float ua, float ub) {
    const float ct = 2.f * ua - 1.f;
    float st = (1.f - ct) * (1.f + ct);
    st = st > 0.f ? sqrtf(st) : 0.f;
    float sp, cp;
    sincospif(2.f * ub, &sp, &cp);
    return V3<float>{st * cp, st * sp, ct};
}

// Training batch of step step0 + *iter: inputs (zero-padded to 16, BF16) and targets.
__global__ void k_gen_batch(LabelTables T, unsigned seed, unsigned step0, const unsigned* __restrict__ iter, int B,
                            bf16* __restrict__ X, float* __restrict__ Y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const unsigned step = step0 + *iter;
    const Draw4<float> u0 = draw4<float>(i, step, 0x51u, seed, 0x5A17u);
    const Draw4<float> u1 = draw4<float>(i, step, 0x52u, seed, 0x5A17u);
    const V3<float> ni = iso_unit(u0.a, u0.b), ns = iso_unit(u0.c, u0.d);
    const float s = 2.f * u1.a - 1.f;
    const float in[kIn] = {ni.x, ni.y, ni.z, ns.x, ns.y, ns.z, s};
    mlp::store_input_row(X + (size_t)i * kInPad, in);
    float out[kOut];
    surrogate_label(T, ni, ns, s, out);
    for (int c = 0; c < kOut; ++c) Y[(size_t)i * kOut + c] = out[c];
}

// Labels of given inputs [n][7] (diagnostics and the error map).
__global__ void k_labels(LabelTables T, int n, const float* __restrict__ in, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* u = in + (size_t)i * kIn;
    float o[kOut];
    surrogate_label(T, V3<float>{u[0], u[1], u[2]}, V3<float>{u[3], u[4], u[5]}, u[6], o);
    for (int c = 0; c < kOut; ++c) out[(size_t)i * kOut + c] = o[c];
}

__global__ void k_pack_inputs(int n, const float* __restrict__ in, bf16* __restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float u[kIn];
    for (int c = 0; c < kIn; ++c) u[c] = in[(size_t)i * kIn + c];
    mlp::store_input_row(X + (size_t)i * kInPad, u);
}

// ---------------------------------------------------------------------------------
// BF16 tensor-core GEMM with fused epilogues:  C[m][n] = sum_k A(m,k) B(k,n)
//   A(m,k) = a_t ? A[k*lda + m] : A[m*lda + k]
//   B(k,n) = b_kn ? B[k*ldb + n] : B[n*ldb + k]
// Block tile 64x64x32, 4 warps of 32x32, mma.sync.m16n8k16 (BF16 in, FP32 accumulate).
// ---------------------------------------------------------------------------------
enum { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DX = 2, EPI_DW = 3 };

struct GemmArgs {
    int M, N, K;
    const bf16* A;
    int lda, a_t;
    const bf16* B;
    int ldb, b_kn;
    const float* bias;    // HIDDEN, OUT
    float* Zout;          // HIDDEN: pre-activation; OUT: output; DW: gradient
    int ldz;
    bf16* Hout;           // HIDDEN: SiLU(Z); DX: dZ of the previous layer
    int ldh;
    const float* Zprev;   // DX: pre-activation of the previous layer
};

constexpr int kTM = 64, kTN = 64, kTK = 32, kPadK = 40;

__device__ __forceinline__ void mma_bf16(float c[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_f(float z) { return mlp::silu(z); }
__device__ __forceinline__ float silu_grad_f(float z) { return mlp::silu_grad(z); }

template <int EPI> __global__ void __launch_bounds__(128) k_gemm(const GemmArgs g) {
    __shared__ __align__(16) bf16 As[kTM][kPadK];
    __shared__ __align__(16) bf16 Bs[kTN][kPadK];
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gr = lane >> 2, tc = lane & 3;
    float acc[2][4][4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 4; ++j)
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    // weight gradients split K (the batch) over gridDim.z blocks, which add their
    // partial sums to the zeroed gradient; the other epilogues take the whole K
    int kb = 0, ke = g.K;
    if (EPI == EPI_DW && gridDim.z > 1) {
        const int per = ((g.K + gridDim.z - 1) / gridDim.z + kTK - 1) / kTK * kTK;
        kb = blockIdx.z * per;
        ke = kb + per < g.K ? kb + per : g.K;
    }
    for (int k0 = kb; k0 < ke; k0 += kTK) {
        for (int i = tid; i < kTM * kTK; i += blockDim.x) {
            const int mm = i / kTK, kk = i % kTK, m = m0 + mm, k = k0 + kk;
            bf16 v = zero;
            if (m < g.M && k < ke) v = g.a_t ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
            As[mm][kk] = v;
        }
        for (int i = tid; i < kTN * kTK; i += blockDim.x) {
            const int nn = i / kTK, kk = i % kTK, n = n0 + nn, k = k0 + kk;
            bf16 v = zero;
            if (n < g.N && k < ke) v = g.b_kn ? g.B[(size_t)k * g.ldb + n] : g.B[(size_t)n * g.ldb + k];
            Bs[nn][kk] = v;
        }
        __syncthreads();
        for (int ks = 0; ks < kTK; ks += 16) {
            unsigned a[2][4], b[4][2];
            for (int mt = 0; mt < 2; ++mt) {
                const int r = wm + mt * 16 + gr, c = ks + tc * 2;
                a[mt][0] = *reinterpret_cast<const unsigned*>(&As[r][c]);
                a[mt][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][c]);
                a[mt][2] = *reinterpret_cast<const unsigned*>(&As[r][c + 8]);
                a[mt][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][c + 8]);
            }
            for (int nt = 0; nt < 4; ++nt) {
                const int n = wn + nt * 8 + gr, c = ks + tc * 2;
                b[nt][0] = *reinterpret_cast<const unsigned*>(&Bs[n][c]);
                b[nt][1] = *reinterpret_cast<const unsigned*>(&Bs[n][c + 8]);
            }
            for (int mt = 0; mt < 2; ++mt)
                for (int nt = 0; nt < 4; ++nt)
                    mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
        }
        __syncthreads();
    }
    // epilogue: c0,c1 at (row gr, cols 2tc, 2tc+1), c2,c3 at row gr + 8
    for (int mt = 0; mt < 2; ++mt)
        for (int nt = 0; nt < 4; ++nt)
            for (int h = 0; h < 2; ++h)
                for (int e = 0; e < 2; ++e) {
                    const int m = m0 + wm + mt * 16 + gr + h * 8, n = n0 + wn + nt * 8 + tc * 2 + e;
                    if (m >= g.M || n >= g.N) continue;
                    const float v = acc[mt][nt][h * 2 + e];
                    if (EPI == EPI_HIDDEN) {
                        const float z = v + g.bias[n];
                        g.Zout[(size_t)m * g.ldz + n] = z;
                        g.Hout[(size_t)m * g.ldh + n] = __float2bfloat16(silu_f(z));
                    } else if (EPI == EPI_OUT) {
                        g.Zout[(size_t)m * g.ldz + n] = v + g.bias[n];
                    } else if (EPI == EPI_DX) {
                        g.Hout[(size_t)m * g.ldh + n] = __float2bfloat16(v * silu_grad_f(g.Zprev[(size_t)m * g.ldz + n]));
                    } else {
                        if (gridDim.z > 1)
                            atomicAdd(&g.Zout[(size_t)m * g.ldz + n], v);
                        else
                            g.Zout[(size_t)m * g.ldz + n] = v;
                    }
                }
}

template <int EPI> cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
    (void)cudaGetLastError();
    dim3 grid((g.N + kTN - 1) / kTN, (g.M + kTM - 1) / kTM);
    // weight gradients (small M x N, K = the batch): split K so that the GPU fills;
    // the output (d_grads) is zeroed before the backward pass
    if (EPI == EPI_DW) {
        int z = 256 / (int)(grid.x * grid.y);
        const int kmax = (g.K + 4 * kTK - 1) / (4 * kTK);  // at least four k-tiles per block
        z = z < kmax ? z : kmax;
        grid.z = z > 1 ? z : 1;
    }
    k_gemm<EPI><<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// FP32 mode of the training passes, for gradient checks at FP32 accuracy: the same
// layers and fused epilogues with FP32 operands and activations on the FP32 pipe (no
// BF16 rounding anywhere), C[m][n] = sum_k A(m,k) B(k,n) with the index rules of
// GemmArgs.  Block tile 64x64x16, 256 threads of 4x4 outputs each.
// ---------------------------------------------------------------------------------
struct GemmArgs32 {
    int M, N, K;
    const float* A;
    int lda, a_t;
    const float* B;
    int ldb, b_kn;
    const float* bias;
    float* Zout;
    int ldz;
    float* Hout;
    int ldh;
    const float* Zprev;
};

constexpr int kT32 = 64, kK32 = 16;

template <int EPI> __global__ void __launch_bounds__(256) k_gemm32(const GemmArgs32 g) {
    __shared__ float As[kK32][kT32 + 4];  // [k][m]
    __shared__ float Bs[kK32][kT32 + 4];  // [k][n]
    const int m0 = blockIdx.y * kT32, n0 = blockIdx.x * kT32;
    const int tid = threadIdx.x, tm = (tid / 16) * 4, tn = (tid % 16) * 4;
    float acc[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    int kb = 0, ke = g.K;
    if (EPI == EPI_DW && gridDim.z > 1) {
        const int per = ((g.K + gridDim.z - 1) / gridDim.z + kK32 - 1) / kK32 * kK32;
        kb = blockIdx.z * per;
        ke = kb + per < g.K ? kb + per : g.K;
    }
    for (int k0 = kb; k0 < ke; k0 += kK32) {
        for (int i = tid; i < kT32 * kK32; i += blockDim.x) {
            const int r = i / kK32, kk = i % kK32, k = k0 + kk;
            const int m = m0 + r, n = n0 + r;
            float a = 0.f, b = 0.f;
            if (m < g.M && k < ke) a = g.a_t ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
            if (n < g.N && k < ke) b = g.b_kn ? g.B[(size_t)k * g.ldb + n] : g.B[(size_t)n * g.ldb + k];
            As[kk][r] = a;
            Bs[kk][r] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kK32; ++kk) {
            float a[4], b[4];
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tm + i];
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tn + j];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tm + i, n = n0 + tn + j;
            if (m >= g.M || n >= g.N) continue;
            const float v = acc[i][j];
            if (EPI == EPI_HIDDEN) {
                const float z = v + g.bias[n];
                g.Zout[(size_t)m * g.ldz + n] = z;
                g.Hout[(size_t)m * g.ldh + n] = silu_f(z);
            } else if (EPI == EPI_OUT) {
                g.Zout[(size_t)m * g.ldz + n] = v + g.bias[n];
            } else if (EPI == EPI_DX) {
                g.Hout[(size_t)m * g.ldh + n] = v * silu_grad_f(g.Zprev[(size_t)m * g.ldz + n]);
            } else {
                if (gridDim.z > 1)
                    atomicAdd(&g.Zout[(size_t)m * g.ldz + n], v);
                else
                    g.Zout[(size_t)m * g.ldz + n] = v;
            }
        }
}

template <int EPI> cudaError_t gemm32(const GemmArgs32& g, cudaStream_t s) {
    (void)cudaGetLastError();
    dim3 grid((g.N + kT32 - 1) / kT32, (g.M + kT32 - 1) / kT32);
    if (EPI == EPI_DW) {
        int z = 256 / (int)(grid.x * grid.y);
        const int kmax = (g.K + 4 * kK32 - 1) / (4 * kK32);
        z = z < kmax ? z : kmax;
        grid.z = z > 1 ? z : 1;
    }
    k_gemm32<EPI><<<grid, 256, 0, s>>>(g);
    return cudaGetLastError();
}

// FP32 inputs [n][7] as the first 7 of 16 columns (the rest zero): in FP32 the input
// needs no high and low parts.
__global__ void k_pack_inputs32(int n, const float* __restrict__ in, float* __restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < kInPad; ++c) X[(size_t)i * kInPad + c] = c < kIn ? in[(size_t)i * kIn + c] : 0.f;
}

// dY = 2 w (Y - T) / (B * 20) in FP32 and the loss sum (the FP32 twin of k_loss_grad).
__global__ void k_loss_grad32(int B, const float* __restrict__ Y, const float* __restrict__ T,
                              const float* __restrict__ w, float* __restrict__ dY, double* __restrict__ loss) {
    __shared__ double part[256];
    double acc = 0.0;
    const float scale = 2.f / ((float)B * (float)kOut);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * kOutPad; i += gridDim.x * blockDim.x) {
        const int b = i / kOutPad, o = i % kOutPad;
        float d = 0.f;
        if (o < kOut) {
            const float r = Y[(size_t)b * kOutPad + o] - T[(size_t)b * kOut + o];
            acc += (double)(w[o] * r * r);
            d = scale * w[o] * r;
        }
        dY[i] = d;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, part[0] / ((double)B * kOut));
}

// db[n] = sum over rows of dZ[b][n] (FP32 input).
__global__ void k_colsum32(int B, int N, const float* __restrict__ dZ, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = blockIdx.y; b < B; b += gridDim.y) s += dZ[(size_t)b * N + n];
    atomicAdd(&db[n], s);
}

// dY = 2 w (Y - T) / (B * 20) (BF16, zero in the padding columns) and the loss sum,
// added to loss[*iter] (loss[0] without an iteration counter).
__global__ void k_loss_grad(int B, const float* __restrict__ Y, const float* __restrict__ T,
                            const float* __restrict__ w, bf16* __restrict__ dY, double* __restrict__ loss,
                            const unsigned* __restrict__ iter) {
    __shared__ double part[256];
    double acc = 0.0;
    const float scale = 2.f / ((float)B * (float)kOut);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * kOutPad; i += gridDim.x * blockDim.x) {
        const int b = i / kOutPad, o = i % kOutPad;
        float d = 0.f;
        if (o < kOut) {
            const float r = Y[(size_t)b * kOutPad + o] - T[(size_t)b * kOut + o];
            acc += (double)(w[o] * r * r);
            d = scale * w[o] * r;
        }
        dY[i] = __float2bfloat16(d);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss + (iter ? *iter : 0u), part[0] / ((double)B * kOut));
}

// db[n] = sum over rows of dZ[b][n] (BF16 input, FP32 output).
__global__ void k_colsum(int B, int N, const bf16* __restrict__ dZ, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = blockIdx.y; b < B; b += gridDim.y) s += __bfloat162float(dZ[(size_t)b * N + n]);
    atomicAdd(&db[n], s);
}

// Adam on the FP32 master parameters; the learning rate and the two bias corrections
// of the iteration are sched[3 * *iter + 0..2].
__global__ void k_adam(int P, float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, const float* __restrict__ sched, const unsigned* __restrict__ iter,
                       float b1, float b2, float eps) {
    const float* sc = sched + 3 * (size_t)*iter;
    const float lr = sc[0], c1 = sc[1], c2 = sc[2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of the weights for the training GEMMs.  Layer 0 columns 7-13 repeat
// columns 0-6 (they multiply the low parts of the split inputs).  As the last kernel
// of a training step it also advances the step's iteration counter (iter_inc).
__global__ void k_pack_weights(const float* __restrict__ p, bf16* __restrict__ wbf, unsigned* __restrict__ iter_inc) {
    if (iter_inc && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(iter_inc, 1u);
    for (int l = 0; l < kLayers; ++l) {
        const int n = layer_out(l) * layer_in(l);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            int src = i;
            float v;
            if (l == 0) {
                const int o = i / kInPad, c = i % kInPad;
                src = o * kInPad + (c < kIn ? c : c - kIn);
                v = c < 2 * kIn ? p[layer_offset(0) + src] : 0.f;
            } else {
                v = p[layer_offset(l) + src];
            }
            wbf[wbf_offset(l) + i] = __float2bfloat16(v);
        }
    }
}

// Layer-0 weight gradient: a master weight feeds both the hi and the lo column, so
// its gradient is the sum of the two; the unused columns get zero.
__global__ void k_fold_l0(float* __restrict__ g) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= kHid) return;
    float* row = g + (size_t)o * kInPad;
    for (int c = 0; c < kIn; ++c) row[c] += row[c + kIn];
    for (int c = kIn; c < kInPad; ++c) row[c] = 0.f;
}

// Inference image (layout in mcrt_mlp_infer.cuh) from the FP32 parameters.
__global__ void k_pack_image(const float* __restrict__ p, unsigned char* __restrict__ img) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int l = 0; l < kLayers; ++l) {
        const int ld = l == 0 ? mlp::kLd0 : mlp::kLdH;
        bf16* w = reinterpret_cast<bf16*>(img + mlp::img_w(l));
        const int rows = layer_out(l), n = rows * ld;
        for (int i = tid; i < n; i += nth) {
            const int o = i / ld, c = i % ld;
            float v = 0.f;
            if (l == 0) {
                if (c < 2 * kIn) v = p[layer_offset(0) + o * kInPad + (c < kIn ? c : c - kIn)];
            } else if (c < layer_in(l)) {
                v = p[layer_offset(l) + o * layer_in(l) + c];
            }
            w[i] = __float2bfloat16(v);
        }
        float* b = reinterpret_cast<float*>(img + mlp::kImgBias) + mlp::bias_off(l);
        for (int i = tid; i < rows; i += nth) b[i] = p[layer_offset(l) + rows * layer_in(l) + i];
    }
}

// Weights N(0, 1/fan_in) (Box-Muller on Philox draws), biases zero.
__global__ void k_init_params(float* __restrict__ p, unsigned seed) {
    for (int l = 0; l < kLayers; ++l) {
        const int nw = layer_out(l) * layer_in(l), nb = layer_out(l);
        const float sd = rsqrtf((float)(l == 0 ? kIn : layer_in(l)));
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + nb; i += gridDim.x * blockDim.x) {
            float v = 0.f;
            if (i < nw) {
                const int col = i % layer_in(l);
                if (l == 0 && col >= kIn) {
                    v = 0.f;
                } else {
                    const Draw4<float> u = draw4<float>(i, (unsigned)l, 0x1A17u, seed, 0x5A17u);
                    v = sd * sqrtf(-2.f * logf(u.a)) * cospif(2.f * u.b);
                }
            }
            p[layer_offset(l) + i] = v;
        }
    }
}

// Inference image for the tcgen05 engine (mcrt_mlp_tc.cuh layout) from the FP32
// parameters: weights in 8x16-byte core matrices, layer 0 columns 7-13 repeating
// columns 0-6, output rows 24-31 zero; biases, output ones padded with zeros.  The
// hidden layers hold W / 2 and b / 2 (exact), so their epilogue gets z / 2 directly.
__global__ void k_pack_image_tc(const float* __restrict__ p, unsigned char* __restrict__ img) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int l = 0; l < kLayers; ++l) {
        const int K = l == 0 ? 16 : 128, N = l == kLayers - 1 ? tc::kN4 : 128;
        __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(img + tc::w_off(l));
        for (int i = tid; i < N * K; i += nth) {
            const int r = i / K, k = i % K;
            float v = 0.f;
            if (l == 0) {
                if (k < 2 * kIn) v = p[layer_offset(0) + r * kInPad + (k < kIn ? k : k - kIn)];
            } else if (r < layer_out(l)) {
                v = p[layer_offset(l) + r * layer_in(l) + k];
            }
            const float half = l < kLayers - 1 ? 0.5f : 1.f;
            w[tc::core_off(r, k, K) / 2] = __float2bfloat16(v * half);
        }
        float* b = reinterpret_cast<float*>(img + tc::kBias) + 128 * l;
        const float half = l < kLayers - 1 ? 0.5f : 1.f;
        for (int i = tid; i < N; i += nth)
            b[i] = i < layer_out(l) ? half * p[layer_offset(l) + layer_out(l) * layer_in(l) + i] : 0.f;
    }
}

// outputs [n][20] of inputs [n][7] on the tcgen05 engine: 128 rows per tile, kTcGroups
// tiles in flight per CTA
constexpr int kTcGroups = 3;
__global__ void __launch_bounds__(tc::kRows * kTcGroups, 1)
    k_infer_tc(const unsigned char* __restrict__ img, long long n, const float* __restrict__ in,
               float* __restrict__ out, unsigned* __restrict__ error) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long mbar[kTcGroups];
    __shared__ unsigned tmem_slot;
    const tc::Group g = tc::setup(kTcGroups, sm, img, mbar, &tmem_slot);
    unsigned phase = 0;
    bool failed = false;
    const long long ntile = (n + tc::kRows - 1) / tc::kRows;
    const int gi = threadIdx.x / tc::kRows;
    for (long long tile = (long long)blockIdx.x * kTcGroups + gi; tile < ntile; tile += (long long)gridDim.x * kTcGroups) {
        const long long row = tile * tc::kRows + g.t;
        float u[kIn];
        for (int c = 0; c < kIn; ++c) u[c] = row < n ? in[row * kIn + c] : 0.f;
        tc::store_input(g, u);
        float y[24];
        if (!tc::forward(g, y, phase, 2000000000ull)) {
            failed = true;
            if (g.t == 0) atomicOr(error, 1u);
            break;
        }
        if (row < n)
            for (int o = 0; o < kOut; ++o) out[row * kOut + o] = y[o];
        tc::group_sync(g);  // every row has read its outputs before the next tile's layer 0
    }
    tc::teardown(kTcGroups, g, failed, phase, 2000000000ull);
}

// ---------------------------------------------------------------------------------
// fused inference (mcrt_mlp_infer.cuh): evaluation, error map, extinction table
// ---------------------------------------------------------------------------------
constexpr int kInferBlock = 256;
struct WarpTile {
    bf16 in[16 * mlp::kLd0];
    float out[16 * mlp::kOutLd];
};
static_assert(sizeof(WarpTile) % 16 == 0, "tiles stay 16-byte aligned");
constexpr size_t kInferSmem = mlp::kImgBytes + (kInferBlock / 32) * sizeof(WarpTile);

__device__ __forceinline__ WarpTile& warp_tile(unsigned char* sm) {
    return reinterpret_cast<WarpTile*>(sm + mlp::kImgBytes)[threadIdx.x >> 5];
}

// outputs [n][20] of inputs [n][7]
__global__ void __launch_bounds__(kInferBlock) k_infer(const unsigned char* __restrict__ img, long long n,
                                                       const float* __restrict__ in, float* __restrict__ out) {
    extern __shared__ __align__(128) unsigned char sm[];
    mlp::load_image(sm, img);
    __syncthreads();
    WarpTile& wt = warp_tile(sm);
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const long long ntile = (n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntile; tile += (long long)gridDim.x * wpb) {
        const long long row = tile * 16 + lane;
        if (lane < 16) {
            float u[kIn];
            for (int c = 0; c < kIn; ++c) u[c] = row < n ? in[row * kIn + c] : 0.f;
            mlp::store_input_row(wt.in + lane * mlp::kLd0, u);
        }
        __syncwarp();
        mlp::warp_mlp16(sm, wt.in, wt.out, lane);
        __syncwarp();
        if (lane < 16 && row < n)
            for (int o = 0; o < kOut; ++o) out[row * kOut + o] = wt.out[lane * mlp::kOutLd + o];
        __syncwarp();
    }
}

// Error map: for n samples (uniform directions, uniform s) the largest error of the
// network's scattering matrix against the tables relative to the true M11, per cell
// of (cos theta_i, cos theta_s, delta phi, s).  map: 4096 floats, zeroed by the
// caller (non-negative floats compare like their bit patterns).
__global__ void __launch_bounds__(kInferBlock) k_errmap(const unsigned char* __restrict__ img, LabelTables T,
                                                        long long n, unsigned seed, float* __restrict__ map) {
    extern __shared__ __align__(128) unsigned char sm[];
    mlp::load_image(sm, img);
    __syncthreads();
    WarpTile& wt = warp_tile(sm);
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const long long ntile = (n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntile; tile += (long long)gridDim.x * wpb) {
        const long long i = tile * 16 + lane;
        float lab[kOut];
        V3<float> ni{0.f, 0.f, 1.f}, ns{0.f, 0.f, 1.f};
        float s = 0.f;
        if (lane < 16) {
            const Draw4<float> u0 = draw4<float>(i, 0u, 0x61u, seed, 0xE77u);
            const Draw4<float> u1 = draw4<float>(i, 0u, 0x62u, seed, 0xE77u);
            ni = iso_unit(u0.a, u0.b);
            ns = iso_unit(u0.c, u0.d);
            s = 2.f * u1.a - 1.f;
            surrogate_label(T, ni, ns, s, lab);
            const float u[kIn] = {ni.x, ni.y, ni.z, ns.x, ns.y, ns.z, s};
            mlp::store_input_row(wt.in + lane * mlp::kLd0, u);
        }
        __syncwarp();
        mlp::warp_mlp16(sm, wt.in, wt.out, lane);
        __syncwarp();
        if (lane < 16 && i < n) {
            const float* y = wt.out + lane * mlp::kOutLd;
            const float r = __expf(y[0] - lab[0]);  // M11 of the network / true M11
            float e = fabsf(r - 1.f);
            for (int o = 1; o < 16; ++o) e = fmaxf(e, fabsf(r * y[o] - lab[o]));
            if (!(e <= 3.0e38f)) e = 3.0e38f;  // NaN or inf: always falls back
            const int idx = mlp::errmap_index(ni.z, ns.z, atan2f(ns.y, ns.x) - atan2f(ni.y, ni.x), s);
            atomicMax(reinterpret_cast<int*>(map) + idx, __float_as_int(e));
        }
        __syncwarp();
    }
}

// Extinction elements alpha1..3 of the network on the grid theta'_j = pi j / (n_k - 1):
// the mean over 16 scattered directions and sizes of outputs 16..18 at
// n_i = (sin theta', 0, cos theta').  Rows that are not realizable (alpha1 <= 0 or
// |alpha2| >= alpha1) keep the table's row and are counted.
__global__ void __launch_bounds__(kInferBlock) k_distill_kext(const unsigned char* __restrict__ img, int n_k,
                                                              const float4* __restrict__ table,
                                                              float4* __restrict__ out, unsigned* __restrict__ n_fixed) {
    extern __shared__ __align__(128) unsigned char sm[];
    mlp::load_image(sm, img);
    __syncthreads();
    WarpTile& wt = warp_tile(sm);
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int j = blockIdx.x * wpb + (threadIdx.x >> 5); j < n_k; j += gridDim.x * wpb) {
        if (lane < 16) {
            float st, ct, sp, cp;
            sincospif((float)j / (float)(n_k - 1), &st, &ct);
            const float z = 1.f - (2.f * lane + 1.f) / 16.f, rho = sqrtf(fmaxf(0.f, 1.f - z * z));
            sincosf(2.39996323f * (float)lane, &sp, &cp);
            const float u[kIn] = {st, 0.f, ct, rho * cp, rho * sp, z, -1.f + (2.f * lane + 1.f) / 16.f};
            mlp::store_input_row(wt.in + lane * mlp::kLd0, u);
        }
        __syncwarp();
        mlp::warp_mlp16(sm, wt.in, wt.out, lane);
        __syncwarp();
        if (lane == 0) {
            float a[3] = {0.f, 0.f, 0.f};
            for (int r = 0; r < 16; ++r)
                for (int e = 0; e < 3; ++e) a[e] += wt.out[r * mlp::kOutLd + 16 + e] * (1.f / 16.f);
            const bool ok = a[0] > 0.f && fabsf(a[1]) < a[0] && fabsf(a[2]) < 3.0e38f;
            if (ok) {
                out[j] = make_float4(a[0], a[1], a[2], 0.f);
            } else {
                out[j] = table[j];
                atomicAdd(n_fixed, 1u);
            }
        }
        __syncwarp();
    }
}

}  // namespace

// ---------------------------------------------------------------------------------
// host side: the surrogate object
// ---------------------------------------------------------------------------------
struct SurrogateBuffers {
    int B = 0;
    bf16* x0 = nullptr;
    float* z[4] = {nullptr, nullptr, nullptr, nullptr};
    bf16* h[4] = {nullptr, nullptr, nullptr, nullptr};
    float* y = nullptr;
    float* t = nullptr;
    bf16* dy = nullptr;
    bf16* dz[2] = {nullptr, nullptr};
};

}  // namespace mcrt

using namespace mcrt;

struct mcrt_surrogate {
    cudaStream_t stream = nullptr;
    float4* d_bins = nullptr;
    float4* d_kext = nullptr;
    int n_bins = 0, n_theta = 0, n_ktheta = 0;
    float* d_params = nullptr;
    float* d_grads = nullptr;
    float* d_m = nullptr;
    float* d_v = nullptr;
    float* d_w = nullptr;  // loss weights [20]
    bf16* d_wbf = nullptr;
    double* d_loss = nullptr;
    float* d_in = nullptr;  // staging of user inputs
    size_t in_cap = 0;
    SurrogateBuffers buf;
    unsigned seed = 0;
    long long step = 0;
    unsigned char* d_image = nullptr;  // inference image of the current parameters
    float* d_map = nullptr;            // error map [4096]
    bool map_valid = false;
    int n_sm = 0;
};

namespace {

#define SK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            (void)cudaGetLastError();                                                                   \
            return mcrt_fail_noctx(MCRT_E_CUDA, "surrogate: %s: %s", #call, cudaGetErrorString(e_));    \
        }                                                                                               \
    } while (0)

void free_buffers(SurrogateBuffers& b) {
    cudaFree(b.x0);
    for (int i = 0; i < 4; ++i) {
        cudaFree(b.z[i]);
        cudaFree(b.h[i]);
    }
    cudaFree(b.y);
    cudaFree(b.t);
    cudaFree(b.dy);
    cudaFree(b.dz[0]);
    cudaFree(b.dz[1]);
    b = SurrogateBuffers{};
}

cudaError_t ensure_buffers(SurrogateBuffers& b, int B) {
    if (b.B >= B) return cudaSuccess;
    free_buffers(b);
    cudaError_t e = cudaMalloc(&b.x0, (size_t)B * kInPad * sizeof(bf16));
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
        e = cudaMalloc(&b.z[i], (size_t)B * kHid * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&b.h[i], (size_t)B * kHid * sizeof(bf16));
    }
    if (e == cudaSuccess) e = cudaMalloc(&b.y, (size_t)B * kOutPad * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b.t, (size_t)B * kOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b.dy, (size_t)B * kOutPad * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc(&b.dz[0], (size_t)B * kHid * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc(&b.dz[1], (size_t)B * kHid * sizeof(bf16));
    if (e != cudaSuccess) {
        free_buffers(b);
        return e;
    }
    b.B = B;
    return cudaSuccess;
}

LabelTables tables_of(const mcrt_surrogate* s) {
    return LabelTables{s->d_bins, s->d_kext, s->n_bins, s->n_theta, s->n_ktheta};
}

// Forward pass on buf.x0 rows [0, B): hidden activations and the output buf.y.
mcrt_status forward(mcrt_surrogate* s, int B) {
    SurrogateBuffers& b = s->buf;
    for (int l = 0; l < kLayers; ++l) {
        GemmArgs g{};
        g.M = B;
        g.N = layer_out(l);
        g.K = layer_in(l);
        g.A = l == 0 ? b.x0 : b.h[l - 1];
        g.lda = layer_in(l);
        g.a_t = 0;
        g.B = s->d_wbf + wbf_offset(l);
        g.ldb = layer_in(l);
        g.b_kn = 0;
        g.bias = s->d_params + layer_offset(l) + layer_out(l) * layer_in(l);
        if (l < kLayers - 1) {
            g.Zout = b.z[l];
            g.ldz = kHid;
            g.Hout = b.h[l];
            g.ldh = kHid;
            SK(gemm<EPI_HIDDEN>(g, s->stream));
        } else {
            g.Zout = b.y;
            g.ldz = kOutPad;
            SK(gemm<EPI_OUT>(g, s->stream));
        }
    }
    return MCRT_OK;
}

// Backward pass after forward() and the loss gradient in buf.dy: gradients of all
// parameters into d_grads (FP32).
mcrt_status backward(mcrt_surrogate* s, int B) {
    SurrogateBuffers& b = s->buf;
    SK(cudaMemsetAsync(s->d_grads, 0, sizeof(float) * kParams, s->stream));
    const bf16* dZ = b.dy;  // gradient w.r.t. the pre-activation of layer l
    int cur = 0;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int no = layer_out(l), ni = layer_in(l);
        const bf16* Hin = l == 0 ? b.x0 : b.h[l - 1];
        // dW = dZ^T Hin : M = no, N = ni, K = B
        GemmArgs gw{};
        gw.M = no;
        gw.N = ni;
        gw.K = B;
        gw.A = dZ;
        gw.lda = no;
        gw.a_t = 1;
        gw.B = Hin;
        gw.ldb = ni;
        gw.b_kn = 1;
        gw.Zout = s->d_grads + layer_offset(l);
        gw.ldz = ni;
        SK(gemm<EPI_DW>(gw, s->stream));
        // db = column sums of dZ
        {
            (void)cudaGetLastError();
            const dim3 grid((no + 127) / 128, 64);
            k_colsum<<<grid, 128, 0, s->stream>>>(B, no, dZ, s->d_grads + layer_offset(l) + no * ni);
            SK(cudaGetLastError());
        }
        if (l == 0) {
            k_fold_l0<<<1, kHid, 0, s->stream>>>(s->d_grads + layer_offset(0));
            SK(cudaGetLastError());
            break;
        }
        // dZ_{l-1} = (dZ W) * SiLU'(Z_{l-1}) : M = B, N = ni, K = no
        GemmArgs gx{};
        gx.M = B;
        gx.N = ni;
        gx.K = no;
        gx.A = dZ;
        gx.lda = no;
        gx.a_t = 0;
        gx.B = s->d_wbf + wbf_offset(l);
        gx.ldb = ni;
        gx.b_kn = 1;
        gx.Zprev = b.z[l - 1];
        gx.ldz = kHid;
        gx.Hout = b.dz[cur];
        gx.ldh = kHid;
        SK(gemm<EPI_DX>(gx, s->stream));
        dZ = b.dz[cur];
        cur ^= 1;
    }
    return MCRT_OK;
}

mcrt_status stage_inputs(mcrt_surrogate* s, const float* in, long long n) {
    const size_t bytes = (size_t)n * kIn * sizeof(float);
    if (s->in_cap < bytes) {
        cudaFree(s->d_in);
        s->d_in = nullptr;
        s->in_cap = 0;
        SK(cudaMalloc(&s->d_in, bytes));
        s->in_cap = bytes;
    }
    SK(cudaMemcpyAsync(s->d_in, in, bytes, cudaMemcpyDefault, s->stream));
    return MCRT_OK;
}

// Inference image of the current parameters (on the surrogate's stream).
mcrt_status pack_image(mcrt_surrogate* s) {
    (void)cudaGetLastError();
    k_pack_image<<<64, 256, 0, s->stream>>>(s->d_params, s->d_image);
    SK(cudaGetLastError());
    return MCRT_OK;
}

template <typename K> mcrt_status infer_attr(K kernel) {
    SK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem));
    return MCRT_OK;
}

int infer_grid(const mcrt_surrogate* s, long long tiles) {
    const long long per_block = kInferBlock / 32;
    long long g = (tiles + per_block - 1) / per_block;
    const long long cap = (long long)(s->n_sm > 0 ? s->n_sm : 1) * 1;
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

mcrt_status compute_error_map(mcrt_surrogate* s, long long n_samples) {
    mcrt_status st = pack_image(s);
    if (st != MCRT_OK) return st;
    st = infer_attr(k_errmap);
    if (st != MCRT_OK) return st;
    SK(cudaMemsetAsync(s->d_map, 0, sizeof(float) * kErrMapCells, s->stream));
    k_errmap<<<infer_grid(s, (n_samples + 15) / 16), kInferBlock, kInferSmem, s->stream>>>(
        s->d_image, tables_of(s), n_samples, s->seed ^ 0x9E3779B9u, s->d_map);
    SK(cudaGetLastError());
    SK(cudaStreamSynchronize(s->stream));
    s->map_valid = true;
    return MCRT_OK;
}

}  // namespace

// Inference data of the surrogate for a model's transport: the inference image, the
// error map (computed with 2^22 samples if not yet done) and the distilled extinction
// table on n_ktheta angles (rows that are not realizable come from `table`).
mcrt_status mcrt_surrogate_export(mcrt_surrogate* s, int n_ktheta, const float4* table, unsigned char* d_image,
                                  unsigned char* d_image_tc, float* d_map, float4* d_kext, int* n_fixed) {
    if (!s->map_valid) {
        mcrt_status st = compute_error_map(s, 1ll << 22);
        if (st != MCRT_OK) return st;
    }
    mcrt_status st = pack_image(s);
    if (st != MCRT_OK) return st;
    st = infer_attr(k_distill_kext);
    if (st != MCRT_OK) return st;
    unsigned* d_fixed = nullptr;
    SK(cudaMalloc(&d_fixed, sizeof(unsigned)));
    cudaError_t e = cudaMemsetAsync(d_fixed, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) {
        (void)cudaGetLastError();
        k_distill_kext<<<infer_grid(s, n_ktheta), kInferBlock, kInferSmem, s->stream>>>(s->d_image, n_ktheta, table,
                                                                                      d_kext, d_fixed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_image, s->d_image, mlp::kImgBytes, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) {
        k_pack_image_tc<<<64, 256, 0, s->stream>>>(s->d_params, d_image_tc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_map, s->d_map, sizeof(float) * kErrMapCells, cudaMemcpyDeviceToDevice, s->stream);
    unsigned fixed = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fixed, d_fixed, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d_fixed);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return mcrt_fail_noctx(MCRT_E_CUDA, "surrogate export: %s", cudaGetErrorString(e));
    }
    if (n_fixed) *n_fixed = (int)fixed;
    return MCRT_OK;
}

extern "C" {

mcrt_status mcrt_surrogate_create(mcrt_surrogate** out, const mcrt_ctx* optics, uint32_t seed) {
    if (!out) return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_create: out is NULL");
    *out = nullptr;
    TablesDev t{};
    if (mcrt_ctx_tables(optics, &t) != MCRT_OK || t.model != MCRT_SCAT_TABLE)
        return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_create: the model needs tabulated optics");
    mcrt_surrogate* s = new (std::nothrow) mcrt_surrogate();
    if (!s) return mcrt_fail_noctx(MCRT_E_NOMEM, "mcrt_surrogate_create: host allocation");
    s->n_bins = t.n_bins;
    s->n_theta = t.n_theta;
    s->n_ktheta = t.n_ktheta;
    s->seed = seed;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    const size_t nbins = (size_t)t.n_bins * t.n_theta * 2;
    if (e == cudaSuccess) e = cudaMalloc(&s->d_bins, nbins * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_kext, (size_t)t.n_ktheta * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_params, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_grads, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_m, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_v, sizeof(float) * kParams);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_w, sizeof(float) * kOut);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_wbf, sizeof(bf16) * kWeights);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_image, mlp::kImgBytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_map, sizeof(float) * kErrMapCells);
    if (e == cudaSuccess) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_bins, t.bins, nbins * sizeof(float4), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_kext, t.kext, (size_t)t.n_ktheta * sizeof(float4), cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_m, 0, sizeof(float) * kParams, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_v, 0, sizeof(float) * kParams, s->stream);
    if (e == cudaSuccess) {
        std::vector<float> w(kOut, 1.f);
        e = cudaMemcpyAsync(s->d_w, w.data(), sizeof(float) * kOut, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    if (e == cudaSuccess) {
        (void)cudaGetLastError();
        k_init_params<<<64, 256, 0, s->stream>>>(s->d_params, seed);
        k_pack_weights<<<64, 256, 0, s->stream>>>(s->d_params, s->d_wbf, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        mcrt_surrogate_destroy(s);
        return mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_create: %s", cudaGetErrorString(e));
    }
    *out = s;
    return MCRT_OK;
}

mcrt_status mcrt_surrogate_train(mcrt_surrogate* s, int64_t n_steps, int32_t batch, double lr, double* loss_history) {
    if (!s || n_steps < 0 || batch < 64 || batch > (1 << 20) || n_steps > (1ll << 31))
        return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_train: bad arguments");
    SK(ensure_buffers(s->buf, batch));
    s->map_valid = false;
    if (n_steps == 0) return MCRT_OK;
    const LabelTables T = tables_of(s);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    // schedule of every step: cosine decay of the learning rate over the call's steps
    // and Adam's bias corrections of the global step
    std::vector<float> sched((size_t)n_steps * 3);
    for (long long it = 0; it < n_steps; ++it) {
        const unsigned step = (unsigned)(s->step + it);
        const double frac = n_steps > 1 ? (double)it / (double)(n_steps - 1) : 0.0;
        sched[3 * it] = (float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * frac))));
        sched[3 * it + 1] = 1.f - std::pow(b1, (float)(step + 1));
        sched[3 * it + 2] = 1.f - std::pow(b2, (float)(step + 1));
    }
    // one allocation: loss per step (FP64), schedule, iteration counter
    const size_t hist_bytes = (size_t)n_steps * sizeof(double), sched_bytes = sched.size() * sizeof(float);
    unsigned char* work = nullptr;
    SK(cudaMalloc(&work, hist_bytes + sched_bytes + 16));
    double* d_hist = reinterpret_cast<double*>(work);
    float* d_sched = reinterpret_cast<float*>(work + hist_bytes);
    unsigned* d_iter = reinterpret_cast<unsigned*>(work + hist_bytes + sched_bytes);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto done = [&](mcrt_status st) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamSynchronize(s->stream);
        cudaFree(work);
        return st;
    };
    cudaError_t e = cudaMemcpyAsync(d_sched, sched.data(), sched_bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_hist, 0, hist_bytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_iter, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // the schedule left the host buffer
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return done(mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_train: %s", cudaGetErrorString(e)));
    }
    // one training step, captured once and replayed: every launch of the step reads its
    // iteration from d_iter, which the step's last kernel advances
    (void)cudaGetLastError();
    e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return done(mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_train: %s", cudaGetErrorString(e)));
    mcrt_status st = MCRT_OK;
    k_gen_batch<<<(batch + 127) / 128, 128, 0, s->stream>>>(T, s->seed, (unsigned)s->step, d_iter, batch, s->buf.x0,
                                                            s->buf.t);
    if (cudaGetLastError() != cudaSuccess) st = MCRT_E_CUDA;
    if (st == MCRT_OK) st = forward(s, batch);
    if (st == MCRT_OK) {
        k_loss_grad<<<256, 256, 0, s->stream>>>(batch, s->buf.y, s->buf.t, s->d_w, s->buf.dy, d_hist, d_iter);
        if (cudaGetLastError() != cudaSuccess) st = MCRT_E_CUDA;
    }
    if (st == MCRT_OK) st = backward(s, batch);
    if (st == MCRT_OK) {
        k_adam<<<128, 256, 0, s->stream>>>(kParams, s->d_params, s->d_grads, s->d_m, s->d_v, d_sched, d_iter, b1, b2,
                                           eps);
        k_pack_weights<<<64, 256, 0, s->stream>>>(s->d_params, s->d_wbf, d_iter);
        if (cudaGetLastError() != cudaSuccess) st = MCRT_E_CUDA;
    }
    e = cudaStreamEndCapture(s->stream, &graph);
    if (st != MCRT_OK) return done(mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_train: capture of the step failed"));
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    for (long long it = 0; it < n_steps && e == cudaSuccess; ++it) e = cudaGraphLaunch(exec, s->stream);
    if (e == cudaSuccess && loss_history)
        e = cudaMemcpyAsync(loss_history, d_hist, hist_bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return done(mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_train: %s", cudaGetErrorString(e)));
    }
    s->step += n_steps;
    return done(MCRT_OK);
}

mcrt_status mcrt_surrogate_eval(mcrt_surrogate* s, int64_t n, const float* inputs, float* outputs) {
    if (!s || n < 0 || (n > 0 && (!inputs || !outputs))) return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_eval: bad arguments");
    if (n == 0) return MCRT_OK;
    mcrt_status st = stage_inputs(s, inputs, n);
    if (st != MCRT_OK) return st;
    st = pack_image(s);
    if (st != MCRT_OK) return st;
    st = infer_attr(k_infer);
    if (st != MCRT_OK) return st;
    float* d_out = nullptr;
    SK(cudaMalloc(&d_out, (size_t)n * kOut * sizeof(float)));
    (void)cudaGetLastError();
    k_infer<<<infer_grid(s, (n + 15) / 16), kInferBlock, kInferSmem, s->stream>>>(s->d_image, n, s->d_in, d_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(outputs, d_out, (size_t)n * kOut * sizeof(float), cudaMemcpyDefault, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d_out);
    if (e != cudaSuccess) return mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_eval: %s", cudaGetErrorString(e));
    return MCRT_OK;
}

mcrt_status mcrt_surrogate_eval_engine(mcrt_surrogate* s, int32_t engine, int64_t n, const float* inputs,
                                       float* outputs) {
    if (engine == MCRT_ENGINE_MMA_SYNC) return mcrt_surrogate_eval(s, n, inputs, outputs);
    if (!s || engine != MCRT_ENGINE_TCGEN05 || n < 0 || (n > 0 && (!inputs || !outputs)))
        return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_eval_engine: bad arguments");
    if (n == 0) return MCRT_OK;
    mcrt_status st = stage_inputs(s, inputs, n);
    if (st != MCRT_OK) return st;
    unsigned char* d_img = nullptr;
    float* d_out = nullptr;
    unsigned* d_err = nullptr;
    unsigned err = 0;
    cudaError_t e = cudaMalloc(&d_img, tc::kImgBytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)n * kOut * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(unsigned), s->stream);
    if (e == cudaSuccess) {
        (void)cudaGetLastError();
        k_pack_image_tc<<<64, 256, 0, s->stream>>>(s->d_params, d_img);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::smem_bytes(kTcGroups));
    if (e == cudaSuccess) {
        const long long tiles = (n + tc::kRows * kTcGroups - 1) / (tc::kRows * kTcGroups);
        const int grid = (int)(tiles < s->n_sm ? tiles : s->n_sm);
        k_infer_tc<<<grid, tc::kRows * kTcGroups, tc::smem_bytes(kTcGroups), s->stream>>>(d_img, n, s->d_in, d_out, d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(outputs, d_out, (size_t)n * kOut * sizeof(float), cudaMemcpyDefault, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d_img);
    cudaFree(d_out);
    cudaFree(d_err);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_eval_engine: %s", cudaGetErrorString(e));
    }
    if (err) return mcrt_fail_noctx(MCRT_E_TIMEOUT, "mcrt_surrogate_eval_engine: a tensor-core wait timed out");
    return MCRT_OK;
}

mcrt_status mcrt_surrogate_error_map(mcrt_surrogate* s, int64_t n_samples, float* map) {
    if (!s || n_samples < 16 || n_samples > (1ll << 34))
        return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_error_map: bad arguments");
    mcrt_status st = compute_error_map(s, n_samples);
    if (st != MCRT_OK) return st;
    if (map) {
        SK(cudaMemcpyAsync(map, s->d_map, sizeof(float) * kErrMapCells, cudaMemcpyDefault, s->stream));
        SK(cudaStreamSynchronize(s->stream));
    }
    return MCRT_OK;
}

mcrt_status mcrt_surrogate_labels(mcrt_surrogate* s, int64_t n, const float* inputs, float* labels) {
    if (!s || n < 0 || (n > 0 && (!inputs || !labels))) return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_labels: bad arguments");
    if (n == 0) return MCRT_OK;
    mcrt_status st = stage_inputs(s, inputs, n);
    if (st != MCRT_OK) return st;
    float* d_out = nullptr;
    SK(cudaMalloc(&d_out, (size_t)n * kOut * sizeof(float)));
    (void)cudaGetLastError();
    k_labels<<<(unsigned)((n + 127) / 128), 128, 0, s->stream>>>(tables_of(s), (int)n, s->d_in, d_out);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(labels, d_out, (size_t)n * kOut * sizeof(float), cudaMemcpyDefault, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(d_out);
    if (e != cudaSuccess) return mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_labels: %s", cudaGetErrorString(e));
    return MCRT_OK;
}

mcrt_status mcrt_surrogate_grad(mcrt_surrogate* s, int64_t n, const float* inputs, const float* targets,
                                const float* loss_weights, float* grads, double* loss) {
    if (!s || n < 1 || n > (1 << 20) || !inputs || !targets || !grads)
        return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_grad: bad arguments");
    mcrt_status st = stage_inputs(s, inputs, n);
    if (st != MCRT_OK) return st;
    SK(ensure_buffers(s->buf, (int)n));
    (void)cudaGetLastError();
    k_pack_inputs<<<(unsigned)((n + 127) / 128), 128, 0, s->stream>>>((int)n, s->d_in, s->buf.x0);
    SK(cudaGetLastError());
    SK(cudaMemcpyAsync(s->buf.t, targets, (size_t)n * kOut * sizeof(float), cudaMemcpyDefault, s->stream));
    std::vector<float> w(kOut, 1.f);
    if (loss_weights) std::memcpy(w.data(), loss_weights, sizeof(float) * kOut);
    SK(cudaMemcpyAsync(s->d_w, w.data(), sizeof(float) * kOut, cudaMemcpyHostToDevice, s->stream));
    st = forward(s, (int)n);
    if (st != MCRT_OK) return st;
    SK(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    k_loss_grad<<<256, 256, 0, s->stream>>>((int)n, s->buf.y, s->buf.t, s->d_w, s->buf.dy, s->d_loss, nullptr);
    SK(cudaGetLastError());
    st = backward(s, (int)n);
    if (st != MCRT_OK) return st;
    SK(cudaMemcpyAsync(grads, s->d_grads, sizeof(float) * kParams, cudaMemcpyDefault, s->stream));
    double l = 0.0;
    SK(cudaMemcpyAsync(&l, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    std::vector<float> ones(kOut, 1.f);
    SK(cudaMemcpyAsync(s->d_w, ones.data(), sizeof(float) * kOut, cudaMemcpyHostToDevice, s->stream));
    SK(cudaStreamSynchronize(s->stream));
    if (loss) *loss = l;
    return MCRT_OK;
}

// The FP32 mode of mcrt_surrogate_grad: forward, loss gradient and backward with FP32
// operands, activations and gradients (k_gemm32), the FP32 master weights as they
// are.  Its buffers live for the call only.
mcrt_status mcrt_surrogate_grad_fp32(mcrt_surrogate* s, int64_t n, const float* inputs, const float* targets,
                                     const float* loss_weights, float* grads, double* loss) {
    if (!s || n < 1 || n > (1 << 20) || !inputs || !targets || !grads)
        return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_grad_fp32: bad arguments");
    mcrt_status st = stage_inputs(s, inputs, n);
    if (st != MCRT_OK) return st;
    const int B = (int)n;
    // x [B][16], z and h [4][B][128], y [B][24], t [B][20], dy [B][24], dz [2][B][128]
    const size_t nx = (size_t)B * kInPad, nh = (size_t)B * kHid, ny = (size_t)B * kOutPad;
    const size_t total = nx + 8 * nh + ny + (size_t)B * kOut + ny + 2 * nh;
    float* base = nullptr;
    SK(cudaMalloc(&base, total * sizeof(float)));
    float* x = base;
    float* z[4];
    float* h[4];
    for (int i = 0; i < 4; ++i) {
        z[i] = x + nx + (size_t)(2 * i) * nh;
        h[i] = z[i] + nh;
    }
    float* y = x + nx + 8 * nh;
    float* t = y + ny;
    float* dy = t + (size_t)B * kOut;
    float* dzb[2] = {dy + ny, dy + ny + nh};
    cudaError_t e = cudaSuccess;
    auto ck = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    k_pack_inputs32<<<(unsigned)((n + 127) / 128), 128, 0, s->stream>>>(B, s->d_in, x);
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(t, targets, (size_t)n * kOut * sizeof(float), cudaMemcpyDefault, s->stream));
    std::vector<float> w(kOut, 1.f);
    if (loss_weights) std::memcpy(w.data(), loss_weights, sizeof(float) * kOut);
    ck(cudaMemcpyAsync(s->d_w, w.data(), sizeof(float) * kOut, cudaMemcpyHostToDevice, s->stream));
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        GemmArgs32 g{};
        g.M = B;
        g.N = layer_out(l);
        g.K = layer_in(l);
        g.A = l == 0 ? x : h[l - 1];
        g.lda = layer_in(l);
        g.B = s->d_params + layer_offset(l);
        g.ldb = layer_in(l);
        g.bias = s->d_params + layer_offset(l) + layer_out(l) * layer_in(l);
        if (l < kLayers - 1) {
            g.Zout = z[l];
            g.ldz = kHid;
            g.Hout = h[l];
            g.ldh = kHid;
            ck(gemm32<EPI_HIDDEN>(g, s->stream));
        } else {
            g.Zout = y;
            g.ldz = kOutPad;
            ck(gemm32<EPI_OUT>(g, s->stream));
        }
    }
    ck(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
    if (e == cudaSuccess) {
        k_loss_grad32<<<256, 256, 0, s->stream>>>(B, y, t, s->d_w, dy, s->d_loss);
        ck(cudaGetLastError());
    }
    ck(cudaMemsetAsync(s->d_grads, 0, sizeof(float) * kParams, s->stream));
    const float* dZ = dy;
    int cur = 0;
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
        const int no = layer_out(l), ni = layer_in(l);
        GemmArgs32 gw{};
        gw.M = no;
        gw.N = ni;
        gw.K = B;
        gw.A = dZ;
        gw.lda = no;
        gw.a_t = 1;
        gw.B = l == 0 ? x : h[l - 1];
        gw.ldb = ni;
        gw.b_kn = 1;
        gw.Zout = s->d_grads + layer_offset(l);
        gw.ldz = ni;
        ck(gemm32<EPI_DW>(gw, s->stream));
        k_colsum32<<<dim3((no + 127) / 128, 64), 128, 0, s->stream>>>(B, no, dZ,
                                                                      s->d_grads + layer_offset(l) + no * ni);
        ck(cudaGetLastError());
        if (l == 0) break;
        GemmArgs32 gx{};
        gx.M = B;
        gx.N = ni;
        gx.K = no;
        gx.A = dZ;
        gx.lda = no;
        gx.B = s->d_params + layer_offset(l);
        gx.ldb = ni;
        gx.b_kn = 1;
        gx.Zprev = z[l - 1];
        gx.ldz = kHid;
        gx.Hout = dzb[cur];
        gx.ldh = kHid;
        ck(gemm32<EPI_DX>(gx, s->stream));
        dZ = dzb[cur];
        cur ^= 1;
    }
    double lv = 0.0;
    ck(cudaMemcpyAsync(grads, s->d_grads, sizeof(float) * kParams, cudaMemcpyDefault, s->stream));
    ck(cudaMemcpyAsync(&lv, s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    std::vector<float> ones(kOut, 1.f);
    ck(cudaMemcpyAsync(s->d_w, ones.data(), sizeof(float) * kOut, cudaMemcpyHostToDevice, s->stream));
    ck(cudaStreamSynchronize(s->stream));
    cudaFree(base);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_surrogate_grad_fp32: %s", cudaGetErrorString(e));
    }
    if (loss) *loss = lv;
    return MCRT_OK;
}

mcrt_status mcrt_surrogate_params(mcrt_surrogate* s, float* params, int32_t set) {
    if (!s || !params) return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_params: bad arguments");
    if (set) {
        s->map_valid = false;
        SK(cudaMemcpyAsync(s->d_params, params, sizeof(float) * kParams, cudaMemcpyDefault, s->stream));
        (void)cudaGetLastError();
        k_pack_weights<<<64, 256, 0, s->stream>>>(s->d_params, s->d_wbf, nullptr);
        SK(cudaGetLastError());
    } else {
        SK(cudaMemcpyAsync(params, s->d_params, sizeof(float) * kParams, cudaMemcpyDefault, s->stream));
    }
    SK(cudaStreamSynchronize(s->stream));
    return MCRT_OK;
}

int64_t mcrt_surrogate_param_count(void) { return kParams; }

mcrt_status mcrt_surrogate_destroy(mcrt_surrogate* s) {
    if (!s) return MCRT_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    free_buffers(s->buf);
    cudaFree(s->d_bins);
    cudaFree(s->d_kext);
    cudaFree(s->d_params);
    cudaFree(s->d_grads);
    cudaFree(s->d_m);
    cudaFree(s->d_v);
    cudaFree(s->d_w);
    cudaFree(s->d_wbf);
    cudaFree(s->d_loss);
    cudaFree(s->d_in);
    cudaFree(s->d_image);
    cudaFree(s->d_map);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return MCRT_OK;
}

}  // extern "C"
