// mcrt_wave.cu -- round-based step 1 of the two-step scheme (Sec. 2.2-2.3): the
// surrogate path, with the grain optics of Sec. 2.2 taken from the network of
// mcrt_mlp.cu instead of the tables, and the table rounds (FP32 table launches),
// whose transport kernel scatters in place and leaves 32-byte records that
// k_tab_tally adds for every camera with one FP64 bulk reduction per record.
//
// The network is a dense contraction, so it runs where the rows are dense: the
// transport kernel (k_transport, surrogate instantiation) moves every packet in
// flight to its next scattering, applies extinction, and leaves one 64-byte record
// per tallying segment (direction, flight size, path integral, grain quaternion,
// cell); at the scattering the packet itself waits in a 128-byte slot.  Then
//  - k_sur_tally_tc evaluates the network for every (record, camera) row on the
//    5th-generation tensor cores (mcrt_mlp_tc.cuh, 128-row tiles), or k_sur_tally on
//    mma.sync, 16 rows per warp (mcrt_mlp_infer.cuh), and adds Z W to the FP64
//    source tally with TMA bulk reductions;
//  - k_sur_scatter runs the rejection sampling of the waiting packets, each warp
//    evaluating up to 16 trials at once (trials of the same packet in order, the
//    first accepted one wins, which is exactly the sequential rule);
// and the survivors resume in the next transport launch, with new packets filling
// the rest of the round's capacity.  Rounds repeat until no packet is left.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <cmath>

#include "mcrt_device.cuh"
#include "mcrt_internal.h"
#include "mcrt_mlp_infer.cuh"
#include "mcrt_mlp_tc.cuh"
#include "mcrt_packet.cuh"

namespace cg = cooperative_groups;

namespace mcrt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWaveBlock = 384;  // 12 warps per SM share one copy of the network

struct TallyWarp {
    __nv_bfloat16 in[16 * mlp::kLd0];
    float out[16 * mlp::kOutLd];
    double stage[16 * 4];  // Stokes rows of the tile's records, source of the bulk reductions
};
struct ScatWarp {
    __nv_bfloat16 in[16 * mlp::kLd0];
    float out[16 * mlp::kOutLd];
};
static_assert(sizeof(TallyWarp) % 16 == 0 && sizeof(ScatWarp) % 16 == 0, "16-byte aligned tiles");
constexpr size_t kCamBytes = kMaxCams * 12 * sizeof(float);
constexpr size_t kTallySmem = mlp::kImgBytes + kCamBytes + (kWaveBlock / 32) * sizeof(TallyWarp);
constexpr size_t kScatSmem = mlp::kImgBytes + (kWaveBlock / 32) * sizeof(ScatWarp);

// Realizability of a network matrix (outputs: ln M11, then M_rc / M11 row-major
// without (0,0)): M11 = e^{y0} > 0, and neither a polarized input nor an unpolarized
// one may give more polarization than intensity, |row 1| <= M11 and |column 1| <=
// M11.  Matrices within 5% of that boundary (in the squared norms) are scaled back
// onto it -- fully polarizing directions sit exactly there and the network lands on
// either side -- and the rest fail.  m receives the 16 ratios (m[0] = 1).
__device__ __forceinline__ bool realizable(const float* y, float m[16]) {
    m[0] = 1.f;
#pragma unroll
    for (int k = 1; k < 16; ++k) m[k] = y[k];
    const float r = m[1] * m[1] + m[2] * m[2] + m[3] * m[3];
    const float c = m[4] * m[4] + m[8] * m[8] + m[12] * m[12];
    if (!(fabsf(y[0]) < 80.f) || !(r <= 1.05f) || !(c <= 1.05f)) return false;
    if (r > 1.f) {
        const float f = rsqrtf(r);
        m[1] *= f;
        m[2] *= f;
        m[3] *= f;
    }
    if (c > 1.f) {
        const float f = rsqrtf(c);
        m[4] *= f;
        m[8] *= f;
        m[12] *= f;
    }
    return true;
}

__device__ __forceinline__ bool map_says_fallback(const SurrogateDev& s, const V3<float>& a, const V3<float>& b,
                                                  float size) {
    const int idx = mlp::errmap_index(a.z, b.z, atan2f(b.y, b.x) - atan2f(a.y, a.x), size);
    return !(__ldg(&s.err_map[idx]) <= s.bound);
}

// Round set-up: new packets taken by the previous round are counted, the packets
// waiting from the previous round become this round's resume list (written by the
// scattering kernel, or, with swap, the previous transport's suspend buffer itself),
// and new packets fill the capacity left.
__global__ void k_wave_begin(WaveCtl* c, unsigned long long total, unsigned long long cap, int swap, int slot) {
    c->next_pid += c->n_new;
    c->n_resume = swap ? c->n_suspend : c->n_resume_next;
    c->n_resume_next = 0;
    const unsigned long long left = total > c->next_pid ? total - c->next_pid : 0;
    const unsigned long long room = cap > c->n_resume ? cap - c->n_resume : 0;
    c->n_new = left < room ? left : room;
    c->claim = 0;
    c->n_suspend = 0;
    c->n_born = 0;
    c->n_rec[slot] = 0;
    c->full = 0;
    c->cnt[kCntIterations] += 1;
}

__device__ __forceinline__ void flush_counters(WaveCtl* ctl, unsigned long long* s_cnt, const unsigned long long* v,
                                               int n, const int* which) {
    for (int k = 0; k < n; ++k)
        if (v[k]) atomicAdd(&s_cnt[k], v[k]);
    __syncthreads();
    if (threadIdx.x < n && s_cnt[threadIdx.x]) atomicAdd(&ctl->cnt[which[threadIdx.x]], s_cnt[threadIdx.x]);
}

// Source tally of the queued segments: row (record, camera) -> the network at
// (n_GF, Omega_c,GF, s) gives the scattering-plane matrix M -> rotate W into the
// plane of n -> Omega_c, apply M, rotate into the camera basis -> S[cell][camera].
// The rows of one record are consecutive (cameras padded to 1, 2, 4, 8 or 16), so
// a record's cameras are one contiguous FP64 bulk reduction.
__global__ void __launch_bounds__(kWaveBlock, 1) k_sur_tally(const __grid_constant__ TransportParams P) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ unsigned long long s_cnt[3];
    mlp::load_image(sm, P.sur.image);
    float* s_cam = reinterpret_cast<float*>(sm + mlp::kImgBytes);
    for (int i = threadIdx.x; i < 12 * P.n_cam; i += blockDim.x) {
        const CameraDev& cd = P.cam[i / 12];
        const int e = i % 12, v = e / 4, w = e % 4;
        s_cam[i] = w == 3 ? 0.f : (float)(v == 0 ? cd.dir[w] : (v == 1 ? cd.th[w] : cd.ph[w]));
    }
    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0ull;
    __syncthreads();
    TallyWarp& tw = reinterpret_cast<TallyWarp*>(sm + mlp::kImgBytes + kCamBytes)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const unsigned long long nreq = P.sur.ctl->n_rec[P.sur.rec_slot];
    const unsigned long long nrec = nreq < P.sur.rec_cap ? nreq : P.sur.rec_cap;
    const int ncam = P.n_cam;
    const int ncp = ncam <= 1 ? 1 : (ncam <= 2 ? 2 : (ncam <= 4 ? 4 : (ncam <= 8 ? 8 : 16)));
    const int per_tile = 16 / ncp;
    const unsigned long long ntile = (nrec + per_tile - 1) / per_tile;
    unsigned long long c_rows = 0, c_map = 0, c_real = 0;
    for (unsigned long long tile = (unsigned long long)blockIdx.x * wpb + (threadIdx.x >> 5); tile < ntile;
         tile += (unsigned long long)gridDim.x * wpb) {
        bulk_wait_read();  // this lane's reductions of the previous tile have read the staging rows
        __syncwarp();
        const int cam = lane % ncp;
        bool valid = false, fb = false;
        unsigned cell = 0;
        float s = 0.f, W[4] = {0.f, 0.f, 0.f, 0.f}, mu = 1.f;
        PlaneRot<float> pr{1.f, 0.f, 1.f, 0.f};
        if (lane < 16) {
            float u[mlp::kIn] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const unsigned long long rec = tile * per_tile + (unsigned)(lane / ncp);
            if (rec < nrec) {
                const float4* r = P.sur.records + rec * kRecordF4;
                cell = __float_as_uint(r[3].x);
                valid = cam < ncam && cell != 0xffffffffu;
                if (valid) {
                    const float4 r0 = r[0], r1 = r[1], q = r[2];
                    const V3<float> n{r0.x, r0.y, r0.z};
                    s = r0.w;
                    W[0] = r1.x;
                    W[1] = r1.y;
                    W[2] = r1.z;
                    W[3] = r1.w;
                    V3<float> th, ph, Om, thc, phc;
                    stokes_basis(n, th, ph);
                    load_camera(s_cam + 12 * cam, Om, thc, phc);
                    // scattering plane of n -> Omega_c, in the lab frame (as the table path)
                    pr = plane_rotation(n, th, ph, Om, thc, phc);
                    mu = dot(n, Om);
                    // the network sees both directions in the grain frame
                    const V3<float> nGF = quat_to_grain(q, n), cGF = quat_to_grain(q, Om);
                    u[0] = nGF.x;
                    u[1] = nGF.y;
                    u[2] = nGF.z;
                    u[3] = cGF.x;
                    u[4] = cGF.y;
                    u[5] = cGF.z;
                    u[6] = s;
                    fb = map_says_fallback(P.sur, nGF, cGF, s);
                }
            }
            mlp::store_input_row(tw.in + lane * mlp::kLd0, u);
        }
        __syncwarp();
        mlp::warp_mlp16(sm, tw.in, tw.out, lane);
        __syncwarp();
        if (valid) {
            const float* y = tw.out + lane * mlp::kOutLd;
            float Y[4], m[16];
            const bool real = realizable(y, m);
            if (!fb && real) {
                apply_plane_full(pr, __expf(y[0]), m, W, Y);
            } else {
                float Pm[6];
                table_at(P.t, s, mu, Pm);
                apply_plane(pr, Pm, W, Y);
                if (fb)
                    ++c_map;
                else
                    ++c_real;
            }
            ++c_rows;
            double2* d2 = reinterpret_cast<double2*>(tw.stage + lane * 4);
            d2[0] = make_double2((double)Y[0], (double)Y[1]);
            d2[1] = make_double2((double)Y[2], (double)Y[3]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncwarp();
        if (valid && cam == 0)
            bulk_reduce_add_f64(P.S + (size_t)cell * (size_t)ncam * 4, tw.stage + lane * 4, (unsigned)ncam * 32u);
    }
    bulk_wait_all();
    const unsigned long long v[3] = {c_rows, c_map, c_real};
    const int which[3] = {kCntTallyRows, kCntFallbackMap, kCntFallbackReal};
    flush_counters(P.sur.ctl, s_cnt, v, 3, which);
}

// The same tally on the 5th-generation tensor cores: a CTA of kTcGroups groups of
// 128 threads, each group taking tiles of 128 rows, thread t building row t's inputs,
// reading row t of the network's output from tensor memory (mcrt_mlp_tc.cuh) and
// finishing row t; while one group works on the CUDA cores another's MMAs run.  A
// record's rows (at most 16 cameras) lie in one warp, whose first-camera lane issues
// the bulk reduction from the group's staging rows (they reuse its input tile).
constexpr int kTcGroups = 3;
constexpr size_t kTallyTcSmem = tc::smem_bytes(kTcGroups) + kCamBytes;
constexpr unsigned long long kTensorWaitNs = 2000000000ull;
static_assert(tc::kA0Bytes >= tc::kRows * 4 * (int)sizeof(double), "staging rows fit the input tile");

__global__ void __launch_bounds__(tc::kRows * kTcGroups, 1) k_sur_tally_tc(const __grid_constant__ TransportParams P) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long mbar[kTcGroups];
    __shared__ unsigned tmem_slot;
    __shared__ unsigned long long s_cnt[3];
    if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0ull;
    float* s_cam = reinterpret_cast<float*>(sm + tc::smem_bytes(kTcGroups));
    for (int i = threadIdx.x; i < 12 * P.n_cam; i += blockDim.x) {
        const CameraDev& cd = P.cam[i / 12];
        const int e = i % 12, v = e / 4, w = e % 4;
        s_cam[i] = w == 3 ? 0.f : (float)(v == 0 ? cd.dir[w] : (v == 1 ? cd.th[w] : cd.ph[w]));
    }
    const tc::Group g = tc::setup(kTcGroups, sm, P.sur.image_tc, mbar, &tmem_slot);  // ends with a barrier
    double* stage = reinterpret_cast<double*>(g.a0);
    const int t = g.t, gi = threadIdx.x / tc::kRows;
    const unsigned long long nreq = P.sur.ctl->n_rec[P.sur.rec_slot];
    const unsigned long long nrec = nreq < P.sur.rec_cap ? nreq : P.sur.rec_cap;
    const int ncam = P.n_cam;
    const int ncp = ncam <= 1 ? 1 : (ncam <= 2 ? 2 : (ncam <= 4 ? 4 : (ncam <= 8 ? 8 : 16)));
    const int per_tile = tc::kRows / ncp;
    const unsigned long long ntile = (nrec + per_tile - 1) / per_tile;
    unsigned long long c_rows = 0, c_map = 0, c_real = 0;
    unsigned phase = 0;
    bool failed = false;
    const int cam = t % ncp;
    const unsigned long long stride = (unsigned long long)gridDim.x * kTcGroups;
    // row t's record of a tile (cell word 0xffffffff past the end); the next tile's is
    // loaded while this tile runs through the network
    auto load = [&](unsigned long long tl, float4 (&r)[4]) {
        const unsigned long long rec = tl * per_tile + (unsigned)(t / ncp);
        if (tl < ntile && rec < nrec) {
            const float4* src = P.sur.records + rec * kRecordF4;
            r[0] = src[0];
            r[1] = src[1];
            r[2] = src[2];
            r[3] = src[3];
        } else {
            r[3].x = __uint_as_float(0xffffffffu);
        }
    };
    float4 nxt[4];
    unsigned long long tile = (unsigned long long)blockIdx.x * kTcGroups + gi;
    load(tile, nxt);
    for (; tile < ntile; tile += stride) {
        // the staging rows share the input tile: every reduction of the previous tile
        // has read them before any row is overwritten
        bulk_wait_read();
        tc::group_sync(g);
        const float4 r0 = nxt[0], r1 = nxt[1], q = nxt[2];
        const unsigned cell = __float_as_uint(nxt[3].x);
        load(tile + stride, nxt);
        bool valid = cam < ncam && cell != 0xffffffffu, fb = false;
        float s = 0.f, W[4] = {0.f, 0.f, 0.f, 0.f}, mu = 1.f;
        PlaneRot<float> pr{1.f, 0.f, 1.f, 0.f};
        float u[mlp::kIn] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        {
            if (valid) {
                const V3<float> n{r0.x, r0.y, r0.z};
                s = r0.w;
                W[0] = r1.x;
                W[1] = r1.y;
                W[2] = r1.z;
                W[3] = r1.w;
                V3<float> th, ph, Om, thc, phc;
                stokes_basis(n, th, ph);
                load_camera(s_cam + 12 * cam, Om, thc, phc);
                pr = plane_rotation(n, th, ph, Om, thc, phc);
                mu = dot(n, Om);
                const V3<float> nGF = quat_to_grain(q, n), cGF = quat_to_grain(q, Om);
                u[0] = nGF.x;
                u[1] = nGF.y;
                u[2] = nGF.z;
                u[3] = cGF.x;
                u[4] = cGF.y;
                u[5] = cGF.z;
                u[6] = s;
                fb = map_says_fallback(P.sur, nGF, cGF, s);
            }
        }
        tc::store_input(g, u);
        float y[24];
        if (!tc::forward(g, y, phase, kTensorWaitNs)) {
            failed = true;
            break;
        }
        if (valid) {
            float Y[4], m[16];
            const bool real = realizable(y, m);
            if (!fb && real) {
                apply_plane_full(pr, __expf(y[0]), m, W, Y);
            } else {
                float Pm[6];
                table_at(P.t, s, mu, Pm);
                apply_plane(pr, Pm, W, Y);
                if (fb)
                    ++c_map;
                else
                    ++c_real;
            }
            ++c_rows;
            double2* d2 = reinterpret_cast<double2*>(stage + t * 4);
            d2[0] = make_double2((double)Y[0], (double)Y[1]);
            d2[1] = make_double2((double)Y[2], (double)Y[3]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncwarp();
        if (valid && cam == 0)
            bulk_reduce_add_f64(P.S + (size_t)cell * (size_t)ncam * 4, stage + t * 4, (unsigned)ncam * 32u);
    }
    bulk_wait_all();
    if (failed && t == 0) atomicOr(P.status, (unsigned)MCRT_STATUS_DEVICE_TIMEOUT);
    const unsigned long long v[3] = {c_rows, c_map, c_real};
    const int which[3] = {kCntTallyRows, kCntFallbackMap, kCntFallbackReal};
    flush_counters(P.sur.ctl, s_cnt, v, 3, which);
    tc::teardown(kTcGroups, g, failed, phase, kTensorWaitNs);
}

// Scattering of the waiting packets (Sec. 2.2 rejection sampling): lanes 0-15 own
// one packet each; every round the unresolved packets share the warp's 16 rows,
// packet k taking trials t_k .. t_k + T - 1 (T = 16 / unresolved) with the same
// Philox counters, proposals and envelope as the table path; the network gives
// the target (Z X)_0 of each trial.
__global__ void __launch_bounds__(kWaveBlock, 1) k_sur_scatter(const __grid_constant__ TransportParams P) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ BlockTotals bt;
    __shared__ unsigned long long s_cnt[4];
    mlp::load_image(sm, P.sur.image);
    if (threadIdx.x < 6) bt.e[threadIdx.x] = 0.0;
    if (threadIdx.x < 10) bt.n[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) bt.status = 0u;
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0ull;
    __syncthreads();
    ScatWarp& sw = reinterpret_cast<ScatWarp*>(sm + mlp::kImgBytes)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const TablesDev& tabs = P.t;
    const int nint = tabs.n_theta - 1;
    const float widen_env = 1.f + P.sur.env_margin;
    const unsigned long long nsus = P.sur.ctl->n_suspend;
    const unsigned long long nbatch = (nsus + 15) / 16;
    unsigned long long c_rows = 0, c_map = 0, c_real = 0, c_miss = 0;
    for (unsigned long long batch = (unsigned long long)blockIdx.x * wpb + (threadIdx.x >> 5); batch < nbatch;
         batch += (unsigned long long)gridDim.x * wpb) {
        Packet<float> pk;
        pk.X0 = pk.X1 = pk.X2 = pk.X3 = 0.f;
        pk.pid = 0;
        pk.n_sca = 0;
        bool live = false;
        float us_a = 0.5f, us_d = 0.5f, sk = 0.f;
        int bin = 0;
        float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
        V3<float> n{0.f, 0.f, 1.f}, th{1.f, 0.f, 0.f}, ph{0.f, 1.f, 0.f}, nGF{0.f, 0.f, 1.f};
        const unsigned long long i = batch * 16 + (unsigned)lane;
        bool parked = false;
        if (lane < 16 && i < nsus) parked = __float_as_uint(P.sur.suspend[i * kStateF4 + 7].y) != 0u;
        if (parked) {
            // stopped inside its flight: straight to the resume buffer
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(&P.sur.ctl->n_resume_next, (unsigned long long)grp.size());
            base = grp.shfl(base, 0);
            const float4* src = P.sur.suspend + i * kStateF4;
            float4* dst = P.sur.resume + (base + grp.thread_rank()) * kStateF4;
#pragma unroll
            for (int e = 0; e < kStateF4; ++e) dst[e] = src[e];
        }
        if (lane < 16 && i < nsus && !parked) {
            load_state(P.sur.suspend + i * kStateF4, pk);
            const Draw4<float> us = draw4<float>(pk.pid, pk.n_sca, 0u, P.seed, P.stream);
            us_a = us.a;
            us_d = us.d;
            live = true;
            if (P.roulette_thr > 0.0 && (double)pk.X0 < P.roulette_thr * (double)pk.I_birth) {
                if ((double)us.b < P.roulette_surv) {
                    const float gmul = (float)(1.0 / P.roulette_surv);
                    pk.e_gain += pk.X0 * (gmul - 1.f);
                    pk.X0 *= gmul;
                    pk.X1 *= gmul;
                    pk.X2 *= gmul;
                    pk.X3 *= gmul;
                } else {
                    finish(P, pk, 2, bt);
                    live = false;
                }
            }
            if (live) {
                bin = tabs.n_bins - 1;
                for (int k = 0; k < tabs.n_bins; ++k)
                    if (us.c < tabs.bin_cdf_f[k]) {
                        bin = k;
                        break;
                    }
                sk = tabs.n_bins > 1 ? -1.f + 2.f * (float)bin / (float)(tabs.n_bins - 1) : 0.f;
                const long long c = ((long long)pk.iz * P.g.n[1] + pk.iy) * P.g.n[0] + pk.ix;
                q = __ldg(&P.g.cells[2 * c]);
                n = V3<float>{pk.nx, pk.ny, pk.nz};
                stokes_basis(n, th, ph);
                nGF = quat_to_grain(q, n);
            }
        }
        const unsigned pid_lo = (unsigned)((unsigned long long)pk.pid & 0xffffffffull);
        const unsigned pid_hi = (unsigned)((unsigned long long)pk.pid >> 32);
        unsigned U = __ballot_sync(kFull, live);
        int t_next = 0;
        bool resolved = false;
        V3<float> n2s{0.f, 0.f, 1.f};
        float Ys[4] = {0.f, 0.f, 0.f, 0.f};
        while (U) {
            const int nu = __popc(U), T = 16 / nu;
            int owner = 0, j = 0;
            bool rowv = false;
            if (lane < 16) {
                const int slot = lane / T;
                if (slot < nu) {
                    owner = (int)__fns(U, 0u, slot + 1);
                    j = lane % T;
                    rowv = true;
                }
            }
            // the owning packet's data
            const float onx = __shfl_sync(kFull, n.x, owner), ony = __shfl_sync(kFull, n.y, owner),
                        onz = __shfl_sync(kFull, n.z, owner);
            const float otx = __shfl_sync(kFull, th.x, owner), oty = __shfl_sync(kFull, th.y, owner),
                        otz = __shfl_sync(kFull, th.z, owner);
            const float opx = __shfl_sync(kFull, ph.x, owner), opy = __shfl_sync(kFull, ph.y, owner),
                        opz = __shfl_sync(kFull, ph.z, owner);
            const float4 oq = make_float4(__shfl_sync(kFull, q.x, owner), __shfl_sync(kFull, q.y, owner),
                                          __shfl_sync(kFull, q.z, owner), __shfl_sync(kFull, q.w, owner));
            const V3<float> og{__shfl_sync(kFull, nGF.x, owner), __shfl_sync(kFull, nGF.y, owner),
                               __shfl_sync(kFull, nGF.z, owner)};
            const float oX[4] = {__shfl_sync(kFull, pk.X0, owner), __shfl_sync(kFull, pk.X1, owner),
                                 __shfl_sync(kFull, pk.X2, owner), __shfl_sync(kFull, pk.X3, owner)};
            const float oX0 = oX[0];
            const int obin = __shfl_sync(kFull, bin, owner);
            const float osk = __shfl_sync(kFull, sk, owner);
            const unsigned opl = __shfl_sync(kFull, pid_lo, owner), oph = __shfl_sync(kFull, pid_hi, owner);
            const unsigned onsca = __shfl_sync(kFull, pk.n_sca, owner);
            const int ot = __shfl_sync(kFull, t_next, owner) + j;
            rowv = rowv && ot < P.max_trials;
            float bound = 0.f, bmax = 0.f, mu = 1.f;
            V3<float> n2{0.f, 0.f, 1.f};
            PlaneRot<float> pr{1.f, 0.f, 1.f, 0.f};
            bool fb = false;
            if (lane < 16) {
                float u[mlp::kIn] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (rowv) {
                    const long long opid = (long long)(((unsigned long long)oph << 32) | (unsigned long long)opl);
                    const Draw4<float> ut = draw4<float>(opid, onsca, 1u + (unsigned)ot, P.seed, P.stream);
                    // interval of the piecewise-constant envelope of bin obin, then the
                    // angle inside it and the azimuth (as the table path)
                    const float* cdf = tabs.env_cdf_f + (size_t)obin * nint;
                    int lo = 0, hi = nint - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (ut.a < cdf[mid])
                            hi = mid;
                        else
                            lo = mid + 1;
                    }
                    float s0, c0, s1, c1;
                    sincospif((float)lo / (float)nint, &s0, &c0);
                    sincospif((float)(lo + 1) / (float)nint, &s1, &c1);
                    mu = c0 - ut.b * (c0 - c1);
                    float sn = (1.f - mu) * (1.f + mu);
                    sn = sn > 0.f ? sqrtf(sn) : 0.f;
                    float sa, ca;
                    sincospif(2.f * ut.c, &sa, &ca);
                    n2 = V3<float>{mu * onx + sn * (ca * otx + sa * opx), mu * ony + sn * (ca * oty + sa * opy),
                                   mu * onz + sn * (ca * otz + sa * opz)};
                    bmax = 2.f * tabs.env[(size_t)obin * nint + lo] * oX0 * widen_env;
                    bound = ut.d * bmax;
                    V3<float> th2, ph2;
                    stokes_basis(n2, th2, ph2);
                    pr = plane_rotation(V3<float>{onx, ony, onz}, V3<float>{otx, oty, otz}, V3<float>{opx, opy, opz},
                                        n2, th2, ph2);
                    const V3<float> n2GF = quat_to_grain(oq, n2);
                    u[0] = og.x;
                    u[1] = og.y;
                    u[2] = og.z;
                    u[3] = n2GF.x;
                    u[4] = n2GF.y;
                    u[5] = n2GF.z;
                    u[6] = osk;
                    fb = map_says_fallback(P.sur, og, n2GF, osk);
                }
                mlp::store_input_row(sw.in + lane * mlp::kLd0, u);
            }
            __syncwarp();
            mlp::warp_mlp16(sm, sw.in, sw.out, lane);
            __syncwarp();
            bool acc = false;
            float Yr[4] = {0.f, 0.f, 0.f, 0.f};
            if (rowv) {
                const float* y = sw.out + lane * mlp::kOutLd;
                float m[16];
                const bool real = realizable(y, m);
                if (!fb && real) {
                    apply_plane_full(pr, __expf(y[0]), m, oX, Yr);
                } else {
                    float Pm[6];
                    table_at(tabs, osk, mu, Pm);
                    apply_plane(pr, Pm, oX, Yr);
                    if (fb)
                        ++c_map;
                    else
                        ++c_real;
                }
                ++c_rows;
                if (Yr[0] > bmax) ++c_miss;
                acc = bound < Yr[0];
            }
            __syncwarp();
            // each owner takes its first accepted row, in trial order
            const unsigned A = __ballot_sync(kFull, rowv && acc);
            const unsigned V = __ballot_sync(kFull, rowv);
            const bool mine = lane < 16 && ((U >> lane) & 1u);
            int src = lane, examined = 0;
            bool got = false;
            if (mine) {
                const int sp = __popc(U & ((1u << lane) - 1u));
                const unsigned m = ((1u << T) - 1u) << (sp * T);
                const unsigned a = A & m;
                if (a) {
                    src = __ffs(a) - 1;
                    got = true;
                    examined = src - sp * T + 1;
                } else {
                    examined = __popc(V & m);
                }
            }
            float g[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) g[e] = __shfl_sync(kFull, Yr[e], src);
            const float gx = __shfl_sync(kFull, n2.x, src), gy = __shfl_sync(kFull, n2.y, src),
                        gz = __shfl_sync(kFull, n2.z, src);
            if (mine) {
                pk.trials += (unsigned)examined;
                t_next += T;
                if (got) {
                    resolved = true;
                    for (int e = 0; e < 4; ++e) Ys[e] = g[e];
                    n2s = V3<float>{gx, gy, gz};
                } else if (t_next >= P.max_trials) {
                    finish(P, pk, 4, bt);
                    live = false;
                }
            }
            U = __ballot_sync(kFull, live && !resolved);
        }
        if (resolved) {
            // Ys is in the lab basis of the new direction; the intensity is kept
            const float norm = pk.X0 / Ys[0];
            pk.X0 = Ys[0] * norm;
            pk.X1 = Ys[1] * norm;
            pk.X2 = Ys[2] * norm;
            pk.X3 = Ys[3] * norm;
            pk.nx = n2s.x;
            pk.ny = n2s.y;
            pk.nz = n2s.z;
            tau_set(pk.tau, -logf(us_a));
            pk.s_flight = flight_size(tabs, us_d);
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(&P.sur.ctl->n_resume_next, (unsigned long long)grp.size());
            base = grp.shfl(base, 0);
            store_state(P.sur.resume + (base + grp.thread_rank()) * kStateF4, pk);
        }
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        if (bt.e[threadIdx.x] != 0.0) atomicAdd(&P.stats[threadIdx.x], bt.e[threadIdx.x]);
    } else if (threadIdx.x < 16) {
        unsigned long long* c = reinterpret_cast<unsigned long long*>(P.stats + 6);
        if (bt.n[threadIdx.x - 6]) atomicAdd(&c[threadIdx.x - 6], bt.n[threadIdx.x - 6]);
    } else if (threadIdx.x == 16 && bt.status) {
        atomicOr(P.status, bt.status);
    }
    const unsigned long long v[4] = {c_rows, c_map, c_real, c_miss};
    const int which[4] = {kCntScatRows, kCntFallbackMap, kCntFallbackReal, kCntEnvelopeMiss};
    flush_counters(P.sur.ctl, s_cnt, v, 4, which);
}

// The rejection trials of the waiting packets on the 5th-generation tensor cores: a CTA
// of kScatGroups groups of 128 threads (the engine of mcrt_mlp_tc.cuh, one weight copy per
// CTA); a group takes 128 waiting packets at a time, thread k owning packet k.  Every
// round the unresolved packets share the group's 128 trial rows -- packet k takes trials
// t_k .. t_k + T - 1 with T = 128 / (unresolved packets), at most 8 -- each row a proposal with the
// table path's Philox counters, envelope and angles, and the network evaluates all 128
// rows in one tile; each packet then takes its first accepted trial in trial order,
// which is the sequential rule.  The decisions are those of k_sur_scatter up to the FP32
// summation order of the two tensor-core engines.
constexpr int kScatGroups = 2;
constexpr int kScatPk = tc::kRows;  // one packet per thread of the group
struct ScatPkt {     // a waiting packet as its trial rows read it (shared memory)
    float n[3], th[3], ph[3], g[3];  // direction, its Stokes basis, the direction in the grain frame
    float4 q;                        // grain quaternion of the packet's cell
    float X[4];
    float sk;                        // size coordinate of the drawn bin
    int bin, t_next, want;           // want: live and not yet resolved
    int slot_owner;                  // entry k: the k-th unresolved packet
    unsigned pid_lo, pid_hi, n_sca;
};
struct ScatRow {     // a trial's outcome (over the activation tile once the network is done)
    float Y[4], n2[3];
    int acc;
};
constexpr size_t kScatTcSmem = tc::smem_bytes(kScatGroups) + kScatGroups * kScatPk * sizeof(ScatPkt);
static_assert(sizeof(ScatRow) * tc::kRows <= (size_t)tc::kActBytes, "trial rows fit in the activation tile");

__global__ void __launch_bounds__(tc::kRows * kScatGroups, 1) k_sur_scatter_tc(const __grid_constant__ TransportParams P) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long mbar[kScatGroups];
    __shared__ unsigned tmem_slot;
    __shared__ BlockTotals bt;
    __shared__ unsigned long long s_cnt[4];
    __shared__ int n_unres[kScatGroups][tc::kRows / 32];
    if (threadIdx.x < 6) bt.e[threadIdx.x] = 0.0;
    if (threadIdx.x < 10) bt.n[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) bt.status = 0u;
    if (threadIdx.x < 4) s_cnt[threadIdx.x] = 0ull;
    const tc::Group g = tc::setup(kScatGroups, sm, P.sur.image_tc, mbar, &tmem_slot);  // ends with a barrier
    const int t = g.t, gi = threadIdx.x / tc::kRows;
    ScatPkt* pkt = reinterpret_cast<ScatPkt*>(sm + tc::smem_bytes(kScatGroups)) + gi * kScatPk;
    ScatRow* rows = reinterpret_cast<ScatRow*>(g.act);
    const TablesDev& tabs = P.t;
    const int nint = tabs.n_theta - 1;
    const float widen_env = 1.f + P.sur.env_margin;
    const unsigned long long nsus = P.sur.ctl->n_suspend;
    const unsigned long long nbatch = (nsus + kScatPk - 1) / kScatPk;
    unsigned long long c_rows = 0, c_map = 0, c_real = 0, c_miss = 0;
    unsigned phase = 0;
    bool failed = false;
    for (unsigned long long batch = (unsigned long long)blockIdx.x * kScatGroups + gi; batch < nbatch;
         batch += (unsigned long long)gridDim.x * kScatGroups) {
        Packet<float> pk;
        pk.X0 = pk.X1 = pk.X2 = pk.X3 = 0.f;
        pk.pid = 0;
        pk.n_sca = 0;
        bool live = false, resolved = false;
        float us_a = 0.5f, us_d = 0.5f;
        V3<float> n2s{0.f, 0.f, 1.f};
        float Ys[4] = {0.f, 0.f, 0.f, 0.f};
        if (t < kScatPk) {
            const unsigned long long i = batch * kScatPk + (unsigned)t;
            const bool parked = i < nsus && __float_as_uint(P.sur.suspend[i * kStateF4 + 7].y) != 0u;
            if (parked) {
                // stopped inside its flight: straight to the resume buffer
                cg::coalesced_group grp = cg::coalesced_threads();
                unsigned long long base = 0;
                if (grp.thread_rank() == 0) base = atomicAdd(&P.sur.ctl->n_resume_next, (unsigned long long)grp.size());
                base = grp.shfl(base, 0);
                const float4* src = P.sur.suspend + i * kStateF4;
                float4* dst = P.sur.resume + (base + grp.thread_rank()) * kStateF4;
#pragma unroll
                for (int e = 0; e < kStateF4; ++e) dst[e] = src[e];
            }
            ScatPkt& sp = pkt[t];
            sp.want = 0;
            sp.t_next = 0;
            if (i < nsus && !parked) {
                load_state(P.sur.suspend + i * kStateF4, pk);
                const Draw4<float> us = draw4<float>(pk.pid, pk.n_sca, 0u, P.seed, P.stream);
                us_a = us.a;
                us_d = us.d;
                live = true;
                if (P.roulette_thr > 0.0 && (double)pk.X0 < P.roulette_thr * (double)pk.I_birth) {
                    if ((double)us.b < P.roulette_surv) {
                        const float gmul = (float)(1.0 / P.roulette_surv);
                        pk.e_gain += pk.X0 * (gmul - 1.f);
                        pk.X0 *= gmul;
                        pk.X1 *= gmul;
                        pk.X2 *= gmul;
                        pk.X3 *= gmul;
                    } else {
                        finish(P, pk, 2, bt);
                        live = false;
                    }
                }
                if (live) {
                    int bin = tabs.n_bins - 1;
                    for (int k = 0; k < tabs.n_bins; ++k)
                        if (us.c < tabs.bin_cdf_f[k]) {
                            bin = k;
                            break;
                        }
                    const long long c = ((long long)pk.iz * P.g.n[1] + pk.iy) * P.g.n[0] + pk.ix;
                    const float4 q = __ldg(&P.g.cells[2 * c]);
                    const V3<float> n{pk.nx, pk.ny, pk.nz};
                    V3<float> th, ph;
                    stokes_basis(n, th, ph);
                    const V3<float> gf = quat_to_grain(q, n);
                    sp.n[0] = n.x; sp.n[1] = n.y; sp.n[2] = n.z;
                    sp.th[0] = th.x; sp.th[1] = th.y; sp.th[2] = th.z;
                    sp.ph[0] = ph.x; sp.ph[1] = ph.y; sp.ph[2] = ph.z;
                    sp.g[0] = gf.x; sp.g[1] = gf.y; sp.g[2] = gf.z;
                    sp.q = q;
                    sp.X[0] = pk.X0; sp.X[1] = pk.X1; sp.X[2] = pk.X2; sp.X[3] = pk.X3;
                    sp.bin = bin;
                    sp.sk = tabs.n_bins > 1 ? -1.f + 2.f * (float)bin / (float)(tabs.n_bins - 1) : 0.f;
                    sp.pid_lo = (unsigned)((unsigned long long)pk.pid & 0xffffffffull);
                    sp.pid_hi = (unsigned)((unsigned long long)pk.pid >> 32);
                    sp.n_sca = pk.n_sca;
                    sp.want = 1;
                }
            }
        }
        tc::group_sync(g);
        for (;;) {
            // the unresolved packets in packet order (slot_owner) and their number, by warp
            // ballots and the counts of the group's earlier warps
            const bool want = pkt[t].want != 0;
            const unsigned wb = __ballot_sync(0xffffffffu, want);
            const int w = t >> 5, lane = t & 31;
            if (lane == 0) n_unres[gi][w] = __popc(wb);
            tc::group_sync(g);
            int before = 0, nu = 0;
            for (int k = 0; k < tc::kRows / 32; ++k) {
                before += k < w ? n_unres[gi][k] : 0;
                nu += n_unres[gi][k];
            }
            const int my_slot = before + __popc(wb & ((1u << lane) - 1u));
            if (want) pkt[my_slot].slot_owner = t;
            tc::group_sync(g);
            if (nu == 0) break;  // the same in every thread of the group
            const int T = tc::kRows / nu < 8 ? tc::kRows / nu : 8;
            const int slot = t / T, j = t % T;
            const int owner = slot < nu ? pkt[slot].slot_owner : 0;
            const ScatPkt& o = pkt[owner];
            const int ot = o.t_next + j;
            const bool rowv = slot < nu && ot < P.max_trials;
            float bound = 0.f, bmax = 0.f, mu = 1.f;
            V3<float> n2{0.f, 0.f, 1.f};
            PlaneRot<float> pr{1.f, 0.f, 1.f, 0.f};
            bool fb = false;
            float u[mlp::kIn] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            const V3<float> on{o.n[0], o.n[1], o.n[2]}, oth{o.th[0], o.th[1], o.th[2]}, oph{o.ph[0], o.ph[1], o.ph[2]};
            if (rowv) {
                const long long opid = (long long)(((unsigned long long)o.pid_hi << 32) | (unsigned long long)o.pid_lo);
                const Draw4<float> ut = draw4<float>(opid, o.n_sca, 1u + (unsigned)ot, P.seed, P.stream);
                // interval of the piecewise-constant envelope of the drawn bin, then the angle
                // inside it and the azimuth (as the table path)
                const float* cdf = tabs.env_cdf_f + (size_t)o.bin * nint;
                int lo = 0, hi = nint - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (ut.a < cdf[mid])
                        hi = mid;
                    else
                        lo = mid + 1;
                }
                float s0, c0, s1, c1;
                sincospif((float)lo / (float)nint, &s0, &c0);
                sincospif((float)(lo + 1) / (float)nint, &s1, &c1);
                mu = c0 - ut.b * (c0 - c1);
                float sn = (1.f - mu) * (1.f + mu);
                sn = sn > 0.f ? sqrtf(sn) : 0.f;
                float sa, ca;
                sincospif(2.f * ut.c, &sa, &ca);
                n2 = V3<float>{mu * on.x + sn * (ca * oth.x + sa * oph.x), mu * on.y + sn * (ca * oth.y + sa * oph.y),
                               mu * on.z + sn * (ca * oth.z + sa * oph.z)};
                bmax = 2.f * tabs.env[(size_t)o.bin * nint + lo] * o.X[0] * widen_env;
                bound = ut.d * bmax;
                V3<float> th2, ph2;
                stokes_basis(n2, th2, ph2);
                pr = plane_rotation(on, oth, oph, n2, th2, ph2);
                const V3<float> og{o.g[0], o.g[1], o.g[2]};
                const V3<float> n2GF = quat_to_grain(o.q, n2);
                u[0] = og.x;
                u[1] = og.y;
                u[2] = og.z;
                u[3] = n2GF.x;
                u[4] = n2GF.y;
                u[5] = n2GF.z;
                u[6] = o.sk;
                fb = map_says_fallback(P.sur, og, n2GF, o.sk);
            }
            tc::store_input(g, u);
            float y[24];
            if (!tc::forward(g, y, phase, kTensorWaitNs)) {  // false in every thread of the group
                failed = true;
                break;
            }
            ScatRow r;
            r.acc = 0;
            r.Y[0] = r.Y[1] = r.Y[2] = r.Y[3] = 0.f;
            r.n2[0] = n2.x;
            r.n2[1] = n2.y;
            r.n2[2] = n2.z;
            if (rowv) {
                float m[16];
                const float oX[4] = {o.X[0], o.X[1], o.X[2], o.X[3]};
                const bool real = realizable(y, m);
                if (!fb && real) {
                    apply_plane_full(pr, __expf(y[0]), m, oX, r.Y);
                } else {
                    float Pm[6];
                    table_at(tabs, o.sk, mu, Pm);
                    apply_plane(pr, Pm, oX, r.Y);
                    if (fb)
                        ++c_map;
                    else
                        ++c_real;
                }
                ++c_rows;
                if (r.Y[0] > bmax) ++c_miss;
                r.acc = bound < r.Y[0] ? 1 : 2;  // 1 accepted, 2 rejected, 0 no trial
            }
            rows[t] = r;
            tc::group_sync(g);
            if (want) {
                // this packet's rows, in trial order: the first accepted one wins
                const int sp = my_slot;
                int examined = 0, src = -1;
                for (int k = sp * T; k < sp * T + T; ++k) {
                    if (rows[k].acc == 0) break;
                    ++examined;
                    if (rows[k].acc == 1) {
                        src = k;
                        break;
                    }
                }
                pk.trials += (unsigned)examined;
                pkt[t].t_next += T;
                if (src >= 0) {
                    resolved = true;
                    for (int e = 0; e < 4; ++e) Ys[e] = rows[src].Y[e];
                    n2s = V3<float>{rows[src].n2[0], rows[src].n2[1], rows[src].n2[2]};
                    pkt[t].want = 0;
                } else if (pkt[t].t_next >= P.max_trials) {
                    finish(P, pk, 4, bt);
                    live = false;
                    pkt[t].want = 0;
                }
            }
            tc::group_sync(g);
        }
        if (failed) break;
        if (t < kScatPk && live && resolved) {
            // Ys is in the lab basis of the new direction; the intensity is kept
            const float norm = pk.X0 / Ys[0];
            pk.X0 = Ys[0] * norm;
            pk.X1 = Ys[1] * norm;
            pk.X2 = Ys[2] * norm;
            pk.X3 = Ys[3] * norm;
            pk.nx = n2s.x;
            pk.ny = n2s.y;
            pk.nz = n2s.z;
            tau_set(pk.tau, -logf(us_a));
            pk.s_flight = flight_size(tabs, us_d);
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(&P.sur.ctl->n_resume_next, (unsigned long long)grp.size());
            base = grp.shfl(base, 0);
            store_state(P.sur.resume + (base + grp.thread_rank()) * kStateF4, pk);
        }
        tc::group_sync(g);  // the packet table is read before the next batch overwrites it
    }
    if (failed && t == 0) atomicOr(P.status, (unsigned)MCRT_STATUS_DEVICE_TIMEOUT);
    __syncthreads();
    if (threadIdx.x < 6) {
        if (bt.e[threadIdx.x] != 0.0) atomicAdd(&P.stats[threadIdx.x], bt.e[threadIdx.x]);
    } else if (threadIdx.x < 16) {
        unsigned long long* c = reinterpret_cast<unsigned long long*>(P.stats + 6);
        if (bt.n[threadIdx.x - 6]) atomicAdd(&c[threadIdx.x - 6], bt.n[threadIdx.x - 6]);
    } else if (threadIdx.x == 16 && bt.status) {
        atomicOr(P.status, bt.status);
    }
    const unsigned long long v[4] = {c_rows, c_map, c_real, c_miss};
    const int which[4] = {kCntScatRows, kCntFallbackMap, kCntFallbackReal, kCntEnvelopeMiss};
    flush_counters(P.sur.ctl, s_cnt, v, 4, which);
    tc::teardown(kScatGroups, g, failed, phase, kTensorWaitNs);
}

// Source tally of queued table-path segments: one record per lane, its cameras in
// turn (the record's Stokes basis once, then per camera the matrix at the scattering
// angle, the plane rotation and the Stokes product), the mixture table and the
// cameras in shared memory.  Each lane stages its record's camera rows (32 B each) in
// a row of its own and issues one contiguous FP64 bulk reduction into S[cell]; lanes
// share nothing, so no lane waits for another.  Same arithmetic as the in-place tally
// of k_transport (table_matrix, plane_rotation, apply_plane).
constexpr int kTabBlock = 128;
constexpr int kTabSlots = 2;  // staging rows per lane (1 or 2), alternated from tile to tile
// a lane's staging row: the cameras' rows, padded by 16 B so that the 16-byte stores of
// a quarter-warp's lanes (rows 8 c + 4 words apart) fall in different bank groups
__host__ __device__ constexpr int tab_row_bytes(int ncam) { return ncam * 32 + 16; }

__global__ void __launch_bounds__(kTabBlock) k_tab_tally(const __grid_constant__ TransportParams P) {
    extern __shared__ __align__(16) unsigned char sm[];
    float4* s_mix = reinterpret_cast<float4*>(sm);
    const int n_mix = 2 * P.t.n_theta;
    float* s_cam = reinterpret_cast<float*>(s_mix + n_mix);
    unsigned char* s_stage = reinterpret_cast<unsigned char*>(s_cam + 12 * kMaxCams);
    for (int i = threadIdx.x; i < n_mix; i += blockDim.x) s_mix[i] = P.t.mix[i];
    for (int i = threadIdx.x; i < 12 * P.n_cam; i += blockDim.x) {
        const CameraDev& cd = P.cam[i / 12];
        const int e = i % 12, v = e / 4, w = e % 4;
        s_cam[i] = w == 3 ? 0.f : (float)(v == 0 ? cd.dir[w] : (v == 1 ? cd.th[w] : cd.ph[w]));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int ncam = P.n_cam;
    const int row = tab_row_bytes(ncam);
    // row of (warp, slot, lane) at index (warp * kTabSlots + slot) * 32 + lane
    unsigned char* const rows = s_stage + ((size_t)(threadIdx.x >> 5) * kTabSlots * 32 + lane) * row;
    const unsigned long long nreq = P.sur.ctl->n_rec[P.sur.rec_slot];
    const unsigned long long nrec = nreq < P.sur.rec_cap ? nreq : P.sur.rec_cap;
    const unsigned long long ntile = (nrec + 31) / 32;
    const unsigned long long stride = (unsigned long long)gridDim.x * wpb;
    // the next tile's record is loaded while this one is converted; a lane's two rows
    // alternate, so that a row is rewritten only once the reduction issued from it two
    // tiles before has read it (every lane commits one bulk group per tile, empty when
    // it issues none, so "all but the newest group" is that reduction)
    auto load = [&](unsigned long long t, float4& a, float4& b) {
        const unsigned long long rec = t * 32 + (unsigned)lane;
        if (t < ntile && rec < nrec) {
            const float4* r = P.sur.records + rec * kTableRecordF4;
            a = r[0];
            b = r[1];
        } else {
            b.w = __uint_as_float(0xffffffffu);
        }
    };
    float4 n0 = make_float4(0.f, 0.f, 0.f, 0.f), n1 = n0;
    unsigned long long tile = (unsigned long long)blockIdx.x * wpb + (threadIdx.x >> 5);
    load(tile, n0, n1);
    for (unsigned it = 0; tile < ntile; ++it, tile += stride) {
        const float4 r0 = n0, r1 = n1;
        load(tile + stride, n0, n1);
        const unsigned cell = __float_as_uint(r1.w);
        if (cell != 0xffffffffu) {
            unsigned char* const dst = rows + (size_t)(it % kTabSlots) * 32 * row;
            if constexpr (kTabSlots == 1)
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            else
                asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            const V3<float> n{r0.x, r0.y, r0.z};
            const float W[4] = {r0.w, r1.x, r1.y, r1.z};
            V3<float> th, ph;
            stokes_basis(n, th, ph);
            for (int k = 0; k < ncam; ++k) {
                V3<float> Om, thc, phc;
                load_camera(s_cam + 12 * k, Om, thc, phc);
                float Pm[6], Y[4];
                table_matrix(s_mix, P.t.n_theta, dot(n, Om), Pm);
                const PlaneRot<float> pr = plane_rotation(n, th, ph, Om, thc, phc);
                apply_plane(pr, Pm, W, Y);
                // FP32 -> FP64: half of the conversions on the (narrow) FP64 pipe, half with
                // integer operations, which balances the two pipes (all on the FP64 pipe or all
                // in integers measured 2 % slower)
                double2* d2 = reinterpret_cast<double2*>(dst + 32 * k);
                d2[0] = make_double2(widen(Y[0]), widen(Y[1]));
                d2[1] = make_double2((double)Y[2], (double)Y[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const unsigned src = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(
                             P.S + (size_t)cell * (size_t)ncam * 4),
                         "r"(src), "r"((unsigned)ncam * 32u)
                         : "memory");
        }
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    bulk_wait_all();
}

size_t tab_tally_smem(const TransportParams& p) {
    return (size_t)2 * p.t.n_theta * sizeof(float4) + 12 * kMaxCams * sizeof(float) +
           (size_t)(kTabBlock / 32) * kTabSlots * 32 * (size_t)tab_row_bytes(p.n_cam > 0 ? p.n_cam : 1);
}

}  // namespace

cudaError_t run_round_transport(const TransportParams& p_in, int model, int n_sm, unsigned long long cap,
                                int* iterations, float* ms_out, float* ms_kernels, cudaStream_t s) {
    const bool sur = model == kScatSurrogate;
    TransportParams p = p_in;
    p.sur.deferred = model;
    p.sur.rec_slot = 0;
    cudaError_t e = cudaSuccess;
    int tab_grid = n_sm;
    const size_t tab_smem = tab_tally_smem(p);
    if (sur) {
        e = cudaFuncSetAttribute(k_sur_tally, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallySmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sur_tally_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTallyTcSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sur_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sur_scatter_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatTcSmem);
    } else {
        if (tab_smem > 48 * 1024)
            e = cudaFuncSetAttribute(k_tab_tally, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab_smem);
        int nb = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tab_tally, kTabBlock, tab_smem);
        tab_grid = n_sm * (nb > 0 ? nb : 1);
    }
    if (e != cudaSuccess) return e;
    const unsigned long long total = (unsigned long long)(p.pid_end - p.pid_begin);
    const int block = 128;
    const size_t tsmem = transport_smem_bytes(p, MCRT_FP32, block);
    const int bps = transport_max_blocks_per_sm(MCRT_FP32, model, false, block, tsmem, p.g.n_patches > 0);
    const int tgrid = n_sm * bps;
    float4* const bufs[2] = {p_in.sur.resume, p_in.sur.suspend};
    cudaEvent_t e0 = nullptr, e1 = nullptr, ek[4] = {nullptr, nullptr, nullptr, nullptr};
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&ek[k]);
    float kms[3] = {0.f, 0.f, 0.f};  // transport, tally, scattering kernels
    if (e == cudaSuccess) e = cudaMemsetAsync(p.sur.ctl, 0, sizeof(WaveCtl), s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    unsigned long long C = cap;
    // a packet advances by at least one event per round
    const long long max_rounds = p.max_events + (long long)(total / 256) + 1000;
    WaveCtl h{};
    int it = 0;
    for (; e == cudaSuccess; ++it) {
        if (it >= max_rounds) {
            e = cudaErrorUnknown;
            break;
        }
        if (!sur) {  // parked packets wait in the other buffer: the two swap roles every round
            p.sur.resume = bufs[it & 1];
            p.sur.suspend = bufs[(it + 1) & 1];
        }
        k_wave_begin<<<1, 1, 0, s>>>(p.sur.ctl, total, C, sur ? 0 : 1, 0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ek[0], s);
        if (e == cudaSuccess && !sur) e = launch_births(p, n_sm, s);
        if (e == cudaSuccess) e = launch_transport(p, MCRT_FP32, block, tgrid, s);
        if (e == cudaSuccess) e = cudaEventRecord(ek[1], s);
        if (e == cudaSuccess) {
            if (sur && p.sur.tally_engine == MCRT_ENGINE_TCGEN05)
                k_sur_tally_tc<<<n_sm, tc::kRows * kTcGroups, kTallyTcSmem, s>>>(p);
            else if (sur)
                k_sur_tally<<<n_sm, kWaveBlock, kTallySmem, s>>>(p);
            else
                k_tab_tally<<<tab_grid, kTabBlock, tab_smem, s>>>(p);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ek[2], s);
        if (e == cudaSuccess && sur) {
            if (p.sur.tally_engine == MCRT_ENGINE_TCGEN05)
                k_sur_scatter_tc<<<n_sm, tc::kRows * kScatGroups, kScatTcSmem, s>>>(p);
            else
                k_sur_scatter<<<n_sm, kWaveBlock, kScatSmem, s>>>(p);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ek[3], s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, p.sur.ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, ek[k], ek[k + 1]);
            kms[k] += t;
        }
        if (e != cudaSuccess) break;
        const unsigned long long waiting = sur ? h.n_resume_next : h.n_suspend;
        if (waiting == 0 && h.next_pid + h.n_new >= total) {
            ++it;
            break;
        }
        // surrogate rounds end at each packet's scattering: keep their records within
        // the queue (capacity from this round's records per work item, factor 2 of
        // headroom).  Table rounds run packets to their end and are meant to stop on a
        // full queue, which parks what is left: they keep the full capacity.
        const unsigned long long items = h.n_resume + h.n_new;
        if (sur && items > 0 && h.n_rec[0] > 0) {
            const double per = (double)h.n_rec[0] / (double)items;
            double want = 0.5 * (double)p.sur.rec_cap / per;
            if (want > (double)cap) want = (double)cap;
            if (want < 1024.0) want = 1024.0;
            C = (unsigned long long)want;
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int k = 0; k < 4; ++k)
        if (ek[k]) cudaEventDestroy(ek[k]);
    if (iterations) *iterations = it;
    if (ms_out) *ms_out = ms;
    if (ms_kernels)
        for (int k = 0; k < 3; ++k) ms_kernels[k] = kms[k];
    return e;
}

cudaError_t run_table_rounds_overlapped(const TransportParams& p_in, int n_sm, unsigned long long cap, int tbps,
                                        int tally_bps, int* iterations, float* ms_out, float* ms_kernels,
                                        cudaStream_t s, cudaStream_t s2) {
    TransportParams p = p_in;
    p.sur.deferred = kScatTableDeferred;
    const size_t tab_smem = tab_tally_smem(p);
    cudaError_t e = cudaSuccess;
    if (tab_smem > 48 * 1024)
        e = cudaFuncSetAttribute(k_tab_tally, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab_smem);
    if (e != cudaSuccess) return e;
    const unsigned long long total = (unsigned long long)(p.pid_end - p.pid_begin);
    const int tgrid = n_sm * (tbps > 0 ? tbps : 1), tab_grid = n_sm * (tally_bps > 0 ? tally_bps : 1);
    float4* const bufs[2] = {p_in.sur.resume, p_in.sur.suspend};
    float4* const recs[2] = {p_in.sur.records, p_in.sur.records + p_in.sur.rec_cap * kTableRecordF4};
    cudaEvent_t e0 = nullptr, e1 = nullptr, tb = nullptr, te = nullptr, join = nullptr;
    cudaEvent_t ab[2] = {nullptr, nullptr}, ae[2] = {nullptr, nullptr};
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventCreate(&tb);
    if (e == cudaSuccess) e = cudaEventCreate(&te);
    if (e == cudaSuccess) e = cudaEventCreate(&join);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        e = cudaEventCreate(&ab[k]);
        if (e == cudaSuccess) e = cudaEventCreate(&ae[k]);
    }
    float kms[3] = {0.f, 0.f, 0.f};
    bool pending[2] = {false, false};  // a tally kernel of this slot has not been accounted yet
    auto account = [&](int slot) -> cudaError_t {
        if (!pending[slot]) return cudaSuccess;
        cudaError_t r = cudaEventSynchronize(ae[slot]);
        float t = 0.f;
        if (r == cudaSuccess) r = cudaEventElapsedTime(&t, ab[slot], ae[slot]);
        kms[1] += t;
        pending[slot] = false;
        return r;
    };
    if (e == cudaSuccess) e = cudaMemsetAsync(p.sur.ctl, 0, sizeof(WaveCtl), s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    const long long max_rounds = p.max_events + (long long)(total / 256) + 1000;
    WaveCtl h{};
    int it = 0;
    for (; e == cudaSuccess; ++it) {
        if (it >= max_rounds) {
            e = cudaErrorUnknown;
            break;
        }
        const int slot = it & 1;
        // the tally of round it-2 read this slot's records and counter
        if (pending[slot]) e = cudaStreamWaitEvent(s, ae[slot], 0);
        if (e == cudaSuccess) e = account(slot);
        p.sur.resume = bufs[it & 1];
        p.sur.suspend = bufs[(it + 1) & 1];
        p.sur.records = recs[slot];
        p.sur.rec_slot = slot;
        if (e == cudaSuccess) {
            k_wave_begin<<<1, 1, 0, s>>>(p.sur.ctl, total, cap, 1, slot);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(tb, s);
        if (e == cudaSuccess) e = launch_births(p, n_sm, s);
        if (e == cudaSuccess) e = launch_transport(p, MCRT_FP32, 128, tgrid, s);
        if (e == cudaSuccess) e = cudaEventRecord(te, s);
        // this round's tally runs beside the next round's transport
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s2, te, 0);
        if (e == cudaSuccess) e = cudaEventRecord(ab[slot], s2);
        if (e == cudaSuccess) {
            k_tab_tally<<<tab_grid, kTabBlock, tab_smem, s2>>>(p);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ae[slot], s2);
        if (e == cudaSuccess) pending[slot] = true;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, p.sur.ctl, sizeof(WaveCtl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, tb, te);
        kms[0] += t;
        if (e != cudaSuccess) break;
        if (h.n_suspend == 0 && h.next_pid + h.n_new >= total) {
            ++it;
            break;
        }
    }
    // the last tallies join the main stream before the end of the launch
    if (e == cudaSuccess) e = cudaEventRecord(join, s2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, join, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = account(k);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEvent_t all[] = {e0, e1, tb, te, join, ab[0], ab[1], ae[0], ae[1]};
    for (cudaEvent_t x : all)
        if (x) cudaEventDestroy(x);
    if (iterations) *iterations = it;
    if (ms_out) *ms_out = ms;
    if (ms_kernels)
        for (int k = 0; k < 3; ++k) ms_kernels[k] = kms[k];
    return e;
}

}  // namespace mcrt
