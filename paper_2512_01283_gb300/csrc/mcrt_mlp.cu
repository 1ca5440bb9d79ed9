// mcrt_mlp.cu -- learned surrogate of the grain optics (the paper's Sec. 2.2 allows
// the Mueller matrix to come from analytic forms, tables or neural networks; Sec. 4
// motivates networks for multi-dimensional grain optics).
//
// The network maps (n_i, n_s, s) -- incident and scattered directions in the grain
// frame and the position s in [-1, 1] of ln x between the first and last tabulated
// size parameter -- to 20 numbers: the 4x4 grain-basis scattering matrix divided by
// its normaliser N(s) = max P11, the extinction elements alpha1..3 at the incident
// polar angle, and ln N(s).  Architecture 16 (7 inputs, zero padded) -> 128 -> 128 ->
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

namespace mcrt {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kLayers = 5;
constexpr int kIn = 7, kInPad = 16, kHid = 128, kOut = 20, kOutPad = 24;
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
// and in ln x between bins; grain-basis matrix from the scattering-plane transfer of
// the four unit Stokes vectors; normalised by the maximum interpolated P11.
__device__ void surrogate_label(const LabelTables& T, const V3<float>& ni, const V3<float>& ns, float s,
                                float out[kOut]) {
    const float b = (fminf(fmaxf(s, -1.f), 1.f) + 1.f) * 0.5f * (float)(T.n_bins - 1);
    int k = (int)floorf(b);
    k = k > T.n_bins - 2 ? T.n_bins - 2 : (k < 0 ? 0 : k);
    const float fb = b - (float)k;
    float N = 0.f;
    for (int j = 0; j < T.n_theta; ++j) {
        const float v = (1.f - fb) * T.bins[((size_t)k * T.n_theta + j) * 2].x +
                        fb * T.bins[((size_t)(k + 1) * T.n_theta + j) * 2].x;
        N = fmaxf(N, v);
    }
    const float mu = fminf(fmaxf(dot(ni, ns), -1.f), 1.f);
    const float x = acosf(mu) * 0.31830988618379067f * (float)(T.n_theta - 1);
    int j = (int)floorf(x);
    j = j > T.n_theta - 2 ? T.n_theta - 2 : (j < 0 ? 0 : j);
    const float ft = x - (float)j;
    float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    interp_row(T, k, j, ft, 1.f - fb, P);
    interp_row(T, k + 1, j, ft, fb, P);
    V3<float> thi, phi, ths, phs;
    stokes_basis(ni, thi, phi);
    stokes_basis(ns, ths, phs);
    const PlaneRot<float> r = plane_rotation(ni, thi, phi, ns, ths, phs);
    const float invN = 1.f / N;
    for (int c = 0; c < 4; ++c) {
        float e[4] = {0.f, 0.f, 0.f, 0.f}, y[4];
        e[c] = 1.f;
        apply_plane(r, P, e, y);
        for (int rr = 0; rr < 4; ++rr) out[rr * 4 + c] = y[rr] * invN;
    }
    const float xk = acosf(fminf(fmaxf(ni.z, -1.f), 1.f)) * 0.31830988618379067f * (float)(T.n_ktheta - 1);
    int jk = (int)floorf(xk);
    jk = jk > T.n_ktheta - 2 ? T.n_ktheta - 2 : (jk < 0 ? 0 : jk);
    const float fk = xk - (float)jk;
    const float4 k0 = T.kext[jk], k1 = T.kext[jk + 1];
    out[16] = (1.f - fk) * k0.x + fk * k1.x;
    out[17] = (1.f - fk) * k0.y + fk * k1.y;
    out[18] = (1.f - fk) * k0.z + fk * k1.z;
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

// Training batch of step `step`: inputs (zero-padded to 16, BF16) and targets.
__global__ void k_gen_batch(LabelTables T, unsigned seed, unsigned step, int B, bf16* __restrict__ X,
                            float* __restrict__ Y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    const Draw4<float> u0 = draw4<float>(i, step, 0x51u, seed, 0x5A17u);
    const Draw4<float> u1 = draw4<float>(i, step, 0x52u, seed, 0x5A17u);
    const V3<float> ni = iso_unit(u0.a, u0.b), ns = iso_unit(u0.c, u0.d);
    const float s = 2.f * u1.a - 1.f;
    const float in[kIn] = {ni.x, ni.y, ni.z, ns.x, ns.y, ns.z, s};
    for (int c = 0; c < kInPad; ++c) X[(size_t)i * kInPad + c] = __float2bfloat16(c < kIn ? in[c] : 0.f);
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
    for (int c = 0; c < kInPad; ++c) X[(size_t)i * kInPad + c] = __float2bfloat16(c < kIn ? in[(size_t)i * kIn + c] : 0.f);
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

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float sg = 1.f / (1.f + __expf(-z));
    return sg * (1.f + z * (1.f - sg));
}

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
    for (int k0 = 0; k0 < g.K; k0 += kTK) {
        for (int i = tid; i < kTM * kTK; i += blockDim.x) {
            const int mm = i / kTK, kk = i % kTK, m = m0 + mm, k = k0 + kk;
            bf16 v = zero;
            if (m < g.M && k < g.K) v = g.a_t ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k];
            As[mm][kk] = v;
        }
        for (int i = tid; i < kTN * kTK; i += blockDim.x) {
            const int nn = i / kTK, kk = i % kTK, n = n0 + nn, k = k0 + kk;
            bf16 v = zero;
            if (n < g.N && k < g.K) v = g.b_kn ? g.B[(size_t)k * g.ldb + n] : g.B[(size_t)n * g.ldb + k];
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
                        g.Zout[(size_t)m * g.ldz + n] = v;
                    }
                }
}

template <int EPI> cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
    (void)cudaGetLastError();
    const dim3 grid((g.N + kTN - 1) / kTN, (g.M + kTM - 1) / kTM);
    k_gemm<EPI><<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

// dY = 2 w (Y - T) / (B * 20) (BF16, zero in the padding columns) and the loss sum.
__global__ void k_loss_grad(int B, const float* __restrict__ Y, const float* __restrict__ T,
                            const float* __restrict__ w, bf16* __restrict__ dY, double* __restrict__ loss) {
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
    if (threadIdx.x == 0) atomicAdd(loss, part[0] / ((double)B * kOut));
}

// db[n] = sum over rows of dZ[b][n] (BF16 input, FP32 output).
__global__ void k_colsum(int B, int N, const bf16* __restrict__ dZ, float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = blockIdx.y; b < B; b += gridDim.y) s += __bfloat162float(dZ[(size_t)b * N + n]);
    atomicAdd(&db[n], s);
}

// Adam on the FP32 master parameters, then the BF16 copies of the weights.
__global__ void k_adam(int P, float* __restrict__ p, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_pack_weights(const float* __restrict__ p, bf16* __restrict__ wbf) {
    for (int l = 0; l < kLayers; ++l) {
        const int n = layer_out(l) * layer_in(l);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
            wbf[wbf_offset(l) + i] = __float2bfloat16(p[layer_offset(l) + i]);
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
        if (l == 0) break;
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

}  // namespace

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
        k_pack_weights<<<64, 256, 0, s->stream>>>(s->d_params, s->d_wbf);
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
    if (!s || n_steps < 0 || batch < 64 || batch > (1 << 20))
        return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_train: bad arguments");
    SK(ensure_buffers(s->buf, batch));
    const LabelTables T = tables_of(s);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long long it = 0; it < n_steps; ++it) {
        const unsigned step = (unsigned)(s->step++);
        (void)cudaGetLastError();
        k_gen_batch<<<(batch + 127) / 128, 128, 0, s->stream>>>(T, s->seed, step, batch, s->buf.x0, s->buf.t);
        SK(cudaGetLastError());
        mcrt_status st = forward(s, batch);
        if (st != MCRT_OK) return st;
        SK(cudaMemsetAsync(s->d_loss, 0, sizeof(double), s->stream));
        k_loss_grad<<<256, 256, 0, s->stream>>>(batch, s->buf.y, s->buf.t, s->d_w, s->buf.dy, s->d_loss);
        SK(cudaGetLastError());
        st = backward(s, batch);
        if (st != MCRT_OK) return st;
        // cosine decay of the learning rate over the call's steps
        const double frac = n_steps > 1 ? (double)it / (double)(n_steps - 1) : 0.0;
        const float lr_t = (float)(lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(3.141592653589793 * frac))));
        const float c1 = 1.f - std::pow(b1, (float)(step + 1)), c2 = 1.f - std::pow(b2, (float)(step + 1));
        k_adam<<<128, 256, 0, s->stream>>>(kParams, s->d_params, s->d_grads, s->d_m, s->d_v, lr_t, b1, b2, eps, c1, c2);
        k_pack_weights<<<64, 256, 0, s->stream>>>(s->d_params, s->d_wbf);
        SK(cudaGetLastError());
        if (loss_history) SK(cudaMemcpyAsync(&loss_history[it], s->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    }
    SK(cudaStreamSynchronize(s->stream));
    return MCRT_OK;
}

mcrt_status mcrt_surrogate_eval(mcrt_surrogate* s, int64_t n, const float* inputs, float* outputs) {
    if (!s || n < 0 || (n > 0 && (!inputs || !outputs))) return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_eval: bad arguments");
    if (n == 0) return MCRT_OK;
    mcrt_status st = stage_inputs(s, inputs, n);
    if (st != MCRT_OK) return st;
    const int chunk = 1 << 16;
    SK(ensure_buffers(s->buf, chunk > s->buf.B ? chunk : s->buf.B));
    std::vector<float> y((size_t)chunk * kOutPad);
    for (long long i0 = 0; i0 < n; i0 += chunk) {
        const int m = (int)(n - i0 < chunk ? n - i0 : chunk);
        (void)cudaGetLastError();
        k_pack_inputs<<<(m + 127) / 128, 128, 0, s->stream>>>(m, s->d_in + (size_t)i0 * kIn, s->buf.x0);
        SK(cudaGetLastError());
        st = forward(s, m);
        if (st != MCRT_OK) return st;
        SK(cudaMemcpyAsync(y.data(), s->buf.y, (size_t)m * kOutPad * sizeof(float), cudaMemcpyDeviceToHost, s->stream));
        SK(cudaStreamSynchronize(s->stream));
        for (int i = 0; i < m; ++i)
            for (int o = 0; o < kOut; ++o) outputs[((size_t)i0 + i) * kOut + o] = y[(size_t)i * kOutPad + o];
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
    k_loss_grad<<<256, 256, 0, s->stream>>>((int)n, s->buf.y, s->buf.t, s->d_w, s->buf.dy, s->d_loss);
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

mcrt_status mcrt_surrogate_params(mcrt_surrogate* s, float* params, int32_t set) {
    if (!s || !params) return mcrt_fail_noctx(MCRT_E_INVAL, "mcrt_surrogate_params: bad arguments");
    if (set) {
        SK(cudaMemcpyAsync(s->d_params, params, sizeof(float) * kParams, cudaMemcpyDefault, s->stream));
        (void)cudaGetLastError();
        k_pack_weights<<<64, 256, 0, s->stream>>>(s->d_params, s->d_wbf);
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
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return MCRT_OK;
}

}  // extern "C"
