// mcrt_mlp_tc.cuh -- the grain-optics network on the 5th-generation tensor cores
// (tcgen05): one CTA of 128 threads evaluates 128 rows per tile, thread t owning
// row t (its TMEM lane).  Per layer one thread issues tcgen05.mma (kind::f16, BF16
// operands from shared memory, FP32 accumulator in TMEM, K = 16 per instruction)
// and commits to an mbarrier; the 128 threads then read their row of the
// accumulator with tcgen05.ld, add the bias, apply SiLU and write the row back to
// shared memory as the next layer's A operand.
//
// Operands are K-major without swizzling, in 8-row x 16-byte core matrices: element
// (r, k) of an operand with K columns sits at byte
//   ((r / 8) * (K / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so core matrices adjacent in K are 128 bytes apart (leading byte offset) and
// 8-row groups K / 8 * 128 bytes apart (stride byte offset).
//
// Same network and inputs as mcrt_mlp_infer.cuh (inputs split into BF16 high and
// low parts, layer 0 weights duplicated for them, SiLU in the tanh form).
#pragma once

#include <cuda_bf16.h>

#include "mcrt_mlp_infer.cuh"

namespace mcrt {
namespace tc {

constexpr int kRows = 128;  // rows per tile = TMEM lanes = threads of the CTA
constexpr int kN4 = 32;     // output layer N (24 outputs padded to a multiple of 16)

// image layout (bytes): weights W_l [N][K] in the core-matrix layout, then biases;
// layers 0-3 (those followed by SiLU) hold W / 2 and b / 2
__host__ __device__ constexpr int operand_bytes(int rows, int k) { return rows * k * 2; }
constexpr int kW0 = 0;                                       // 128 x 16
constexpr int kW1 = kW0 + operand_bytes(128, 16);            // 128 x 128
constexpr int kW2 = kW1 + operand_bytes(128, 128);
constexpr int kW3 = kW2 + operand_bytes(128, 128);
constexpr int kW4 = kW3 + operand_bytes(128, 128);           // 32 x 128
constexpr int kBias = kW4 + operand_bytes(kN4, 128);         // 4 x 128 + 32 floats
constexpr int kImgBytes = kBias + (4 * 128 + kN4) * 4;       // 112768
static_assert(kImgBytes % 16 == 0, "16-byte copies");
__host__ __device__ constexpr int w_off(int l) { return l == 0 ? kW0 : (l == 1 ? kW1 : (l == 2 ? kW2 : (l == 3 ? kW3 : kW4))); }

__host__ __device__ constexpr int core_off(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// ---------------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, leading byte offset >> 4, stride byte
// offset >> 4, descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0)
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3fffu) | ((unsigned long long)((lbo >> 4) & 0x3fffu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28
__host__ __device__ constexpr unsigned instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                        unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned mbar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0u;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity, at most limit_ns of wall time.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity, unsigned long long limit_ns) {
    const unsigned long long t0 = now_ns();
    while (!mbar_try_wait(mbar, parity))
        if (now_ns() - t0 > limit_ns) return false;
    return true;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM allocation by one full warp; the address lands in *slot (shared memory)
__device__ __forceinline__ void tmem_alloc(unsigned slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float v[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float v[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------------
// the engine: G groups of 128 threads per CTA, each with a tile in flight (its own
// input / activation tiles, TMEM accumulator, mbarrier and named barrier), sharing
// the weights.  While one group runs its epilogue on the CUDA cores another group's
// MMAs run on the tensor cores.
// ---------------------------------------------------------------------------------
constexpr int kA0Bytes = operand_bytes(kRows, 16);    // input tile (4 KB), later the group's staging rows
constexpr int kActBytes = operand_bytes(kRows, 128);  // activation tile (32 KB)
constexpr int kGroupBytes = kA0Bytes + kActBytes;
__host__ __device__ constexpr int smem_bytes(int groups) { return kImgBytes + groups * kGroupBytes; }
__host__ __device__ constexpr unsigned tmem_cols(int groups) { return groups <= 1 ? 128u : (groups == 2 ? 256u : 512u); }

struct Group {
    unsigned char* img;  // weights + biases (shared by the groups)
    unsigned char* a0;   // input tile, 128 x 16 BF16; free after layer 0
    unsigned char* act;  // activation tile, 128 x 128 BF16
    unsigned mbar;       // shared address of the group's MMA-completion mbarrier
    unsigned tmem;       // TMEM address of the group's 128 accumulator columns
    int bar;             // named barrier id of the group (1 + group)
    int t;               // row = thread index within the group
};

__device__ __forceinline__ void group_sync(const Group& g) {
    asm volatile("bar.sync %0, %1;" ::"r"(g.bar), "r"(kRows) : "memory");
}
__device__ __forceinline__ bool group_and(const Group& g, bool v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v ? 1u : 0u), "r"(g.bar), "r"(kRows)
        : "memory");
    return r != 0u;
}

// Row t of the group's input tile from 7 inputs (BF16 high parts, low parts, zeros).
__device__ __forceinline__ void store_input(const Group& g, const float u[mlp::kIn]) {
    __nv_bfloat16 v[16];
#pragma unroll
    for (int c = 0; c < mlp::kIn; ++c) {
        const __nv_bfloat16 h = __float2bfloat16_rn(u[c]);
        v[c] = h;
        v[mlp::kIn + c] = __float2bfloat16_rn(u[c] - __bfloat162float(h));
    }
    v[14] = v[15] = __float2bfloat16_rn(0.f);
    const uint4* src = reinterpret_cast<const uint4*>(v);
    *reinterpret_cast<uint4*>(g.a0 + core_off(g.t, 0, 16)) = src[0];
    *reinterpret_cast<uint4*>(g.a0 + core_off(g.t, 8, 16)) = src[1];
}

// One layer: D (TMEM) = A (shared, rows x K) * W^T; issued by the group's thread 0,
// completion on its mbarrier (parity `phase`).  Returns false in every thread of the
// group when the MMAs did not complete within limit_ns.
__device__ __forceinline__ bool layer_mma(const Group& g, unsigned a_addr, int K, int l, int N, unsigned& phase,
                                          unsigned long long limit_ns) {
    // the group's smem writes -> visible to the tensor core; its TMEM reads finished
    // before the accumulator is overwritten
    fence_async_smem();
    fence_before();
    group_sync(g);
    fence_after();
    if (g.t == 0) {
        const unsigned w_addr = smem_u32(g.img) + (unsigned)w_off(l);
        const unsigned sbo = (unsigned)(K / 8) * 128u;
        const unsigned idesc = instr_desc(kRows, N);
        for (int k = 0; k < K / 16; ++k) {
            const unsigned long long ad = smem_desc(a_addr + (unsigned)k * 256u, 128u, sbo);
            const unsigned long long bd = smem_desc(w_addr + (unsigned)k * 256u, 128u, sbo);
            mma_f16(g.tmem, ad, bd, idesc, k > 0 ? 1u : 0u);
        }
        mma_commit(g.mbar);
    }
    const bool ok = group_and(g, mbar_wait(g.mbar, phase, limit_ns));
    phase ^= 1u;
    fence_after();
    return ok;
}

// TMEM address of row t's lane (warp w reaches lanes 32 (w mod 4) .. + 31)
__device__ __forceinline__ unsigned lane_addr(const Group& g) { return g.tmem + ((unsigned)(g.t & ~31) << 16); }


// wait for this thread's TMEM loads, with the destination registers tied to the wait so
// that no use of them is scheduled before it
__device__ __forceinline__ void tmem_wait_ld32(float (&v)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                   "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]),
                   "+f"(v[16]), "+f"(v[17]), "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]), "+f"(v[22]), "+f"(v[23]),
                   "+f"(v[24]), "+f"(v[25]), "+f"(v[26]), "+f"(v[27]), "+f"(v[28]), "+f"(v[29]), "+f"(v[30]), "+f"(v[31])
                 :
                 : "memory");
}
// packed FP32 pairs (add / fma .f32x2: one instruction for two lanes of arithmetic,
// each rounded as the scalar operation)
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(unsigned long long d, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(d));
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Hidden-layer epilogue of 32 columns of row t: D + bias, SiLU, BF16, into the
// activation tile.  The hidden layers' weights and biases are stored halved (exact in
// BF16 and FP32), so D + bias is h = z / 2 and SiLU(z) = z sigma(z) = h + h tanh(h).
__device__ __forceinline__ void epi_chunk(const Group& g, const float* bias, int j, const float (&v)[32]) {
    unsigned p[16];
    const unsigned long long* b2 = reinterpret_cast<const unsigned long long*>(bias + j);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const unsigned long long h = f2_add(f2_pack(v[2 * i], v[2 * i + 1]), b2[i]);
        float h0, h1;
        f2_unpack(h, h0, h1);
        const unsigned long long r = f2_fma(h, f2_pack(mlp::tanh_apx(h0), mlp::tanh_apx(h1)), h);
        float r0, r1;
        f2_unpack(r, r0, r1);
        p[i] = mlp::pack_bf16(r0, r1);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(g.act + core_off(g.t, j + 8 * c, 128)) =
            make_uint4(p[4 * c], p[4 * c + 1], p[4 * c + 2], p[4 * c + 3]);
}

// Hidden-layer epilogue of row t, 128 columns: the next 32 columns are loaded from
// tensor memory while the current ones are converted.
__device__ __forceinline__ void hidden_epilogue(const Group& g, const float* bias) {
    const unsigned la = lane_addr(g);
    float va[32], vb[32];
    tmem_ld32(la, va);
    tmem_wait_ld32(va);
    tmem_ld32(la + 32u, vb);
    epi_chunk(g, bias, 0, va);
    tmem_wait_ld32(vb);
    tmem_ld32(la + 64u, va);
    epi_chunk(g, bias, 32, vb);
    tmem_wait_ld32(va);
    tmem_ld32(la + 96u, vb);
    epi_chunk(g, bias, 64, va);
    tmem_wait_ld32(vb);
    epi_chunk(g, bias, 96, vb);
}

// The network on the group's 128 rows (inputs in a0): out[0..23] of row t.  All
// threads of the group call it.  Returns false (in all of them) on an MMA timeout.
__device__ __forceinline__ bool forward(const Group& g, float out[24], unsigned& phase, unsigned long long limit_ns) {
    const float* bias = reinterpret_cast<const float*>(g.img + kBias);
    if (!layer_mma(g, smem_u32(g.a0), 16, 0, 128, phase, limit_ns)) return false;
    hidden_epilogue(g, bias);
    for (int l = 1; l < 4; ++l) {
        if (!layer_mma(g, smem_u32(g.act), 128, l, 128, phase, limit_ns)) return false;
        hidden_epilogue(g, bias + 128 * l);
    }
    if (!layer_mma(g, smem_u32(g.act), 128, 4, kN4, phase, limit_ns)) return false;
    float v[32];
    tmem_ld32(lane_addr(g), v);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 24; ++i) out[i] = v[i] + bias[512 + i];
    return true;
}

// CTA set-up for `groups` groups of 128 threads: image into shared memory, one
// mbarrier per group, TMEM (warp 0 allocates for all).  All threads call it; it ends
// with a CTA barrier.  mbar: `groups` 8-byte words in shared memory.
__device__ __forceinline__ Group setup(int groups, unsigned char* smem, const unsigned char* img_global,
                                       unsigned long long* mbar, unsigned* tmem_slot) {
    const uint4* src = reinterpret_cast<const uint4*>(img_global);
    uint4* dst = reinterpret_cast<uint4*>(smem);
    for (int i = threadIdx.x; i < kImgBytes / 16; i += blockDim.x) dst[i] = __ldg(&src[i]);
    if (threadIdx.x == 0) {
        for (int k = 0; k < groups; ++k) mbar_init(smem_u32(&mbar[k]), 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) tmem_alloc(smem_u32(tmem_slot), tmem_cols(groups));
    fence_before();
    __syncthreads();
    fence_after();
    const int gi = threadIdx.x / kRows;
    Group g;
    g.img = smem;
    g.a0 = smem + kImgBytes + gi * kGroupBytes;
    g.act = g.a0 + kA0Bytes;
    g.mbar = smem_u32(&mbar[gi]);
    g.tmem = *tmem_slot + (unsigned)(gi * 128);
    g.bar = 1 + gi;
    g.t = threadIdx.x % kRows;
    return g;
}

// After a timeout one more bounded wait for the group's MMA in flight (its phase was
// already flipped by layer_mma), then warp 0 releases the TMEM in any case.
__device__ __forceinline__ void teardown(int groups, const Group& g, bool failed, unsigned phase,
                                         unsigned long long limit_ns) {
    if (failed && g.t == 0) (void)mbar_wait(g.mbar, phase ^ 1u, limit_ns);
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32) tmem_dealloc(g.tmem, tmem_cols(groups));  // warp 0: group 0, column base
}

}  // namespace tc
}  // namespace mcrt
