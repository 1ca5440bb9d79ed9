// mcrt_mlp_infer.cuh -- fused inference of the grain-optics network on the tensor
// cores: one warp evaluates 16 rows through all five layers with the activations held
// in registers (the accumulator fragments of layer l are repacked in place as the A
// fragments of layer l+1) and the BF16 weights read from shared memory with
// ldmatrix.  mma.sync m16n8k16, BF16 operands, FP32 accumulation; SiLU between
// layers.  Used by the surrogate transport (tally and scattering kernels), the error
// map and the evaluation entry point.
//
// Network: 16 inputs -> 128 -> 128 -> 128 -> 128 -> 24 (20 used).  The 7 inputs
// (n_i, n_s, s) enter split into BF16 high and low parts, x = hi + lo, in columns
// 0-6 and 7-13; layer 0 carries each weight column twice, so it sees the inputs to
// about 16 significant bits although its operands are BF16.
#pragma once

#include <cuda_bf16.h>

namespace mcrt {
namespace mlp {

constexpr int kLayers = 5;
constexpr int kIn = 7, kInPad = 16, kHid = 128, kOut = 20, kOutPad = 24;

// Inference image: BF16 weight rows padded so that the eight rows read by one
// ldmatrix fall into distinct shared-memory bank groups, then FP32 biases.  The same
// bytes live in global memory and, per block, in shared memory.
constexpr int kLd0 = 24;   // row stride (elements) of layer 0, K = 16
constexpr int kLdH = 136;  // row stride of layers 1-4, K = 128
// byte offset of layer l's weights; float offset of its biases from kImgBias
__host__ __device__ constexpr int img_w(int l) { return l == 0 ? 0 : kHid * kLd0 * 2 + (l - 1) * kHid * kLdH * 2; }
__host__ __device__ constexpr int bias_off(int l) { return l * kHid; }
constexpr int kImgBias = img_w(kLayers - 1) + kOutPad * kLdH * 2;  // 117120
constexpr int kImgBytes = kImgBias + (4 * kHid + kOutPad) * 4;     // 119264
constexpr int kOutLd = 25;  // row stride (floats) of a warp's output tile

static_assert(img_w(1) == 6144 && img_w(4) == 110592 && kImgBias == 117120, "image layout");
static_assert(kImgBytes % 16 == 0, "image is copied in 16-byte units");

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(unsigned a, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(unsigned a, unsigned& r0, unsigned& r1) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(a));
}
// the input tile is written by the warp just before: keep the load after those stores
__device__ __forceinline__ void ldsm_x4_fenced(unsigned a, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a)
                 : "memory");
}

__device__ __forceinline__ void mma16816(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float tanh_apx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// SiLU(z) = z sigma(z) with sigma(z) = (1 + tanh(z/2)) / 2
__device__ __forceinline__ float silu(float z) {
    const float h = 0.5f * z;
    return fmaf(h, tanh_apx(h), h);
}
__device__ __forceinline__ float silu_grad(float z) {
    const float sg = 0.5f + 0.5f * tanh_apx(0.5f * z);
    return sg * (1.f + z * (1.f - sg));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

// Input row of 16 BF16: hi parts of the 7 inputs, lo parts, two zeros.
__device__ __forceinline__ void store_input_row(__nv_bfloat16* row, const float u[kIn]) {
#pragma unroll
    for (int c = 0; c < kIn; ++c) {
        const __nv_bfloat16 h = __float2bfloat16_rn(u[c]);
        row[c] = h;
        row[kIn + c] = __float2bfloat16_rn(u[c] - __bfloat162float(h));
    }
    row[14] = __float2bfloat16_rn(0.f);
    row[15] = __float2bfloat16_rn(0.f);
}

// Hidden layer, N = 128 in two halves of 64 columns.  ain: A fragments of the
// layer input (KT k-tiles of 16); aout: A fragments of the layer output (8 k-tiles).
template <int KT>
__device__ __forceinline__ void hidden_layer(unsigned w_base, int ld, const float* bias, const unsigned (&ain)[8][4],
                                             unsigned (&aout)[8][4], int lane) {
    const int t = lane & 3;
    const int mi = lane >> 3, r = lane & 7;
    // ldmatrix row of this lane: matrices (n-tile 2jp, k lo), (2jp, k hi), (2jp+1, k lo), (2jp+1, k hi)
    const unsigned lane_off = (unsigned)(((r + (mi >> 1) * 8) * ld + (mi & 1) * 8) * 2);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = 64 * h + 8 * j + 2 * t;
            const float b0 = bias[col], b1 = bias[col + 1];
            acc[j][0] = b0;
            acc[j][1] = b1;
            acc[j][2] = b0;
            acc[j][3] = b1;
        }
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
#pragma unroll
            for (int jp = 0; jp < 4; ++jp) {
                unsigned b0, b1, b2, b3;
                ldsm_x4(w_base + lane_off + (unsigned)(((64 * h + 16 * jp) * ld + 16 * kk) * 2), b0, b1, b2, b3);
                mma16816(acc[2 * jp], ain[kk], b0, b1);
                mma16816(acc[2 * jp + 1], ain[kk], b2, b3);
            }
        }
        // accumulators of n-tiles (2jj, 2jj+1) form k-tile 4h + jj of the next layer
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            aout[4 * h + jj][0] = pack_bf16(silu(acc[2 * jj][0]), silu(acc[2 * jj][1]));
            aout[4 * h + jj][1] = pack_bf16(silu(acc[2 * jj][2]), silu(acc[2 * jj][3]));
            aout[4 * h + jj][2] = pack_bf16(silu(acc[2 * jj + 1][0]), silu(acc[2 * jj + 1][1]));
            aout[4 * h + jj][3] = pack_bf16(silu(acc[2 * jj + 1][2]), silu(acc[2 * jj + 1][3]));
        }
    }
}

// 16 rows of the calling warp (all 32 lanes take part): in_s [16][kLd0] BF16 input
// rows in shared memory, out_s [16][kOutLd] FP32 (columns 0-23 written).  img: the
// inference image in shared memory.
__device__ __forceinline__ void warp_mlp16(const unsigned char* img, const __nv_bfloat16* in_s, float* out_s,
                                           int lane) {
    const unsigned base = smem_addr(img);
    const float* bias = reinterpret_cast<const float*>(img + kImgBias);
    unsigned a[8][4], c[8][4];
    {
        const int mi = lane >> 3, r = lane & 7;
        const __nv_bfloat16* p = in_s + (r + (mi & 1) * 8) * kLd0 + (mi >> 1) * 8;
        ldsm_x4_fenced(smem_addr(p), a[0][0], a[0][1], a[0][2], a[0][3]);
    }
    hidden_layer<1>(base + img_w(0), kLd0, bias + bias_off(0), a, c, lane);
    hidden_layer<8>(base + img_w(1), kLdH, bias + bias_off(1), c, a, lane);
    hidden_layer<8>(base + img_w(2), kLdH, bias + bias_off(2), a, c, lane);
    hidden_layer<8>(base + img_w(3), kLdH, bias + bias_off(3), c, a, lane);
    // output layer, N = 24: n-tiles 0, 1 with ldmatrix.x4, n-tile 2 with .x2
    const int g = lane >> 2, t = lane & 3;
    const int mi = lane >> 3, r = lane & 7;
    const float* b4 = bias + bias_off(4);
    float acc[3][4];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float b0 = b4[8 * j + 2 * t], b1 = b4[8 * j + 2 * t + 1];
        acc[j][0] = b0;
        acc[j][1] = b1;
        acc[j][2] = b0;
        acc[j][3] = b1;
    }
    const unsigned w4 = base + img_w(4);
    const unsigned off01 = (unsigned)(((r + (mi >> 1) * 8) * kLdH + (mi & 1) * 8) * 2);
    const unsigned off2 = (unsigned)(((16 + r) * kLdH + (mi & 1) * 8) * 2);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        unsigned b0, b1, b2, b3, e0, e1;
        ldsm_x4(w4 + off01 + kk * 32, b0, b1, b2, b3);
        ldsm_x2(w4 + off2 + kk * 32, e0, e1);
        mma16816(acc[0], a[kk], b0, b1);
        mma16816(acc[1], a[kk], b2, b3);
        mma16816(acc[2], a[kk], e0, e1);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        out_s[g * kOutLd + 8 * j + 2 * t] = acc[j][0];
        out_s[g * kOutLd + 8 * j + 2 * t + 1] = acc[j][1];
        out_s[(g + 8) * kOutLd + 8 * j + 2 * t] = acc[j][2];
        out_s[(g + 8) * kOutLd + 8 * j + 2 * t + 1] = acc[j][3];
    }
}

// Block-wide copy of the inference image into shared memory (caller synchronizes).
__device__ __forceinline__ void load_image(unsigned char* dst, const unsigned char* src) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int i = threadIdx.x; i < kImgBytes / 16; i += blockDim.x) d[i] = __ldg(&s[i]);
}

// Error-map cell of (cos theta_i, cos theta_s, delta phi, s): 8 bins per coordinate.
__device__ __forceinline__ int errmap_index(float ci, float cs, float dphi, float s) {
    auto bin = [](float x, float lo, float w) {
        int b = (int)floorf((x - lo) * w);
        return b < 0 ? 0 : (b > 7 ? 7 : b);
    };
    float d = dphi;
    if (d < 0.f) d += 6.283185307179586f;
    return ((bin(ci, -1.f, 4.f) * 8 + bin(cs, -1.f, 4.f)) * 8 + bin(d, 0.f, 1.2732395447351628f)) * 8 + bin(s, -1.f, 4.f);
}

}  // namespace mlp
}  // namespace mcrt
