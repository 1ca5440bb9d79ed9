// mcrt_packet.cuh -- packet state and per-packet helpers shared by the transport
// kernels (mcrt_transport.cu) and the scattering kernel of the surrogate path
// (mcrt_wave.cu): the register-resident packet, block totals, the end-of-packet
// accounting, table lookups, and the 128-byte form in which a packet waits between
// kernels.
#pragma once

#include "mcrt_device.cuh"
#include "mcrt_internal.h"

namespace mcrt {
namespace {

// camera record in shared memory: Omega, theta-hat, phi-hat, each padded to 4
__device__ __forceinline__ void load_camera(const float* cm, V3<float>& Om, V3<float>& th, V3<float>& ph) {
    const float4 a = reinterpret_cast<const float4*>(cm)[0], b = reinterpret_cast<const float4*>(cm)[1],
                 c = reinterpret_cast<const float4*>(cm)[2];
    Om = V3<float>{a.x, a.y, a.z};
    th = V3<float>{b.x, b.y, b.z};
    ph = V3<float>{c.x, c.y, c.z};
}
__device__ __forceinline__ void load_camera(const double* cm, V3<double>& Om, V3<double>& th, V3<double>& ph) {
    Om = V3<double>{cm[0], cm[1], cm[2]};
    th = V3<double>{cm[4], cm[5], cm[6]};
    ph = V3<double>{cm[8], cm[9], cm[10]};
}

// TMA bulk reduction (global += shared, FP64) of one thread's staging slot, and the
// waits on this thread's bulk groups.
__device__ __forceinline__ void bulk_reduce_add_f64(double* gdst, const double* ssrc, unsigned bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(ssrc);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f64 [%0], [%1], %2;" ::"l"(gdst), "r"(s),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// alpha1..3 at cos(theta'), linear in theta' on the table grid
template <typename T>
__device__ __forceinline__ void kext_eval(const TablesDev& t, const float4* kx, T cos_tp, T& a1, T& a2, T& a3) {
    if (t.k_const) {
        const float4 k = kx[0];
        a1 = k.x;
        a2 = k.y;
        a3 = k.z;
        return;
    }
    const T c = cos_tp > T(1) ? T(1) : (cos_tp < T(-1) ? T(-1) : cos_tp);
    const T x = t_acos(c) * T(0.31830988618379067) * T(t.n_ktheta - 1);
    int j = (int)floor(x);
    j = j > t.n_ktheta - 2 ? t.n_ktheta - 2 : (j < 0 ? 0 : j);
    const T f = x - T(j);
    const float4 k0 = kx[j], k1 = kx[j + 1];
    a1 = (T(1) - f) * T(k0.x) + f * T(k1.x);
    a2 = (T(1) - f) * T(k0.y) + f * T(k1.y);
    a3 = (T(1) - f) * T(k0.z) + f * T(k1.z);
}

// scattering matrix of a table (rows of two float4) at mu, linear in the angle
template <typename T> __device__ __forceinline__ void table_matrix(const float4* tab, int n_theta, T mu, T P[6]) {
    const T c = mu > T(1) ? T(1) : (mu < T(-1) ? T(-1) : mu);
    const T x = t_acos(c) * T(0.31830988618379067) * T(n_theta - 1);
    int j = (int)floor(x);
    j = j > n_theta - 2 ? n_theta - 2 : (j < 0 ? 0 : j);
    const T f = x - T(j), g = T(1) - f;
    const float4 a0 = tab[2 * j], a1 = tab[2 * j + 1], b0 = tab[2 * j + 2], b1 = tab[2 * j + 3];
    P[0] = g * T(a0.x) + f * T(b0.x);
    P[1] = g * T(a0.y) + f * T(b0.y);
    P[2] = g * T(a0.z) + f * T(b0.z);
    P[3] = g * T(a0.w) + f * T(b0.w);
    P[4] = g * T(a1.x) + f * T(b1.x);
    P[5] = g * T(a1.y) + f * T(b1.y);
}

// Packet state, held in registers for the packet's lifetime (scalar fields only,
// so that nothing is indexed at run time and nothing lands in local memory).
template <typename T> struct Packet {
    T px, py, pz, nx, ny, nz;
    T X0, X1, X2, X3;
    T I_birth, e_abs, e_gain;
    T s_flight;  // surrogate path: grain-size coordinate of the current flight's tally
    bool park;     // round-based paths: stop before the next segment (record queue near its end)
    bool pending;  // a scattering waits for the warp's next scattering phase
    double tau;  // remaining scattering optical depth (FP64 running sum)
    long long pid;
    const JobDev* job;  // batched launches: the packet's job
    unsigned events, n_seg, n_sca, n_tally, n_abs, trials;
    int ix, iy, iz, src;
    int lvl;        // composite grids: 0 in the root grid, p + 1 in patch p
    float4 cq, cr;  // record of the current cell: q_B and (kappa_abs, kappa_sca, B, 0)
};

// Launch totals of one block (shared memory), folded in once per packet.
struct BlockTotals {
    double e[6];               // emitted, escaped, absorbed, roulette lost, roulette gain, capped
    unsigned long long n[10];  // events, segments, scatterings, emitted, escaped, killed, capped,
                               // trials, tally segments, absorbing segments
    unsigned status;
};

template <typename T> __device__ __forceinline__ T pick(float f, double d);
template <> __device__ __forceinline__ float pick<float>(float f, double) { return f; }
template <> __device__ __forceinline__ double pick<double>(float, double d) { return d; }

// Widening of an FP32 value to FP64 with integer operations only (the FP64 pipe of
// GB300 is narrow): exact for normal numbers, infinities and NaN; FP32 subnormals
// (|x| < 1.2e-38) become signed zero.
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = u & 0x7f800000u;
    const unsigned sign = u & 0x80000000u;
    // exponent and mantissa moved into the double's fields, exponent rebased by 1023 - 127
    unsigned hi = sign | (((u & 0x7fffffffu) >> 3) + 0x38000000u);
    hi = e == 0x7f800000u ? (sign | 0x7ff00000u | ((u & 0x007fffffu) >> 3)) : hi;
    hi = e == 0u ? sign : hi;
    const unsigned lo = e == 0u ? 0u : (u << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// The remaining optical depth is an FP64 running sum (FP32 steps widened exactly).
__device__ __forceinline__ void tau_set(double& t, float v) { t = (double)v; }
__device__ __forceinline__ void tau_set(double& t, double v) { t = v; }
__device__ __forceinline__ bool tau_below(double t, float d) { return t < widen(d); }
__device__ __forceinline__ bool tau_below(double t, double d) { return t < d; }
__device__ __forceinline__ void tau_sub(double& t, float d) { t -= widen(d); }
__device__ __forceinline__ void tau_sub(double& t, double d) { t -= d; }
__device__ __forceinline__ double tau_value(double t) { return t; }
// 8 bytes of the waiting form of a packet
__device__ __forceinline__ void tau_pack(double t, float& a, float& b) {
    a = __int_as_float(__double2loint(t));
    b = __int_as_float(__double2hiint(t));
}
__device__ __forceinline__ void tau_unpack(double& t, float a, float b) {
    t = __hiloint2double(__float_as_int(b), __float_as_int(a));
}
__device__ __forceinline__ double widen(double d) { return d; }

// Packet end: optional trace record, then the packet's totals into the block's.
template <typename T>
__device__ void finish(const TransportParams& P, const Packet<T>& pk, int flag, BlockTotals& bt) {
    atomicAdd(&bt.e[0], (double)pk.I_birth);
    atomicAdd(&bt.e[2], (double)pk.e_abs);
    if (pk.e_gain != T(0)) atomicAdd(&bt.e[4], (double)pk.e_gain);
    if (flag == 1) {
        atomicAdd(&bt.e[1], (double)pk.X0);
        atomicAdd(&bt.n[4], 1ull);
    } else if (flag == 2) {
        atomicAdd(&bt.e[3], (double)pk.X0);
        atomicAdd(&bt.n[5], 1ull);
    } else {
        atomicAdd(&bt.e[5], (double)pk.X0);
        atomicAdd(&bt.n[6], 1ull);
        atomicOr(&bt.status, flag == 3 ? (unsigned)MCRT_STATUS_EVENT_CAP : (unsigned)MCRT_STATUS_TRIAL_CAP);
    }
    atomicAdd(&bt.n[0], (unsigned long long)pk.events);
    atomicAdd(&bt.n[1], (unsigned long long)pk.n_seg);
    atomicAdd(&bt.n[2], (unsigned long long)pk.n_sca);
    atomicAdd(&bt.n[3], 1ull);
    atomicAdd(&bt.n[7], (unsigned long long)pk.trials);
    atomicAdd(&bt.n[8], (unsigned long long)pk.n_tally);
    atomicAdd(&bt.n[9], (unsigned long long)pk.n_abs);
    if (P.trace && pk.pid < P.n_trace) {
        double* tr = P.trace + pk.pid * 16;
        tr[0] = pk.X0;
        tr[1] = pk.X1;
        tr[2] = pk.X2;
        tr[3] = pk.X3;
        tr[4] = pk.px;
        tr[5] = pk.py;
        tr[6] = pk.pz;
        tr[7] = pk.nx;
        tr[8] = pk.ny;
        tr[9] = pk.nz;
        tr[10] = (double)pk.n_sca;
        tr[11] = (double)pk.n_seg;
        tr[12] = (double)flag;
        tr[13] = (double)pk.I_birth;
        tr[14] = (double)pk.src;
        tr[15] = (double)pk.events;
    }
}

// Grain-size coordinate s in [-1, 1] of the bin drawn with u from the bin weights
// (bin k of n sits at s = -1 + 2k / (n - 1)); 0 for a single bin.
template <typename T> __device__ __forceinline__ T flight_size(const TablesDev& t, T u) {
    if (t.n_bins <= 1) return T(0);
    int bin = t.n_bins - 1;
    for (int k = 0; k < t.n_bins; ++k)
        if (u < cdf_at<T>(t.bin_cdf, t.bin_cdf_f, k)) {
            bin = k;
            break;
        }
    return T(-1) + T(2) * T(bin) / T(t.n_bins - 1);
}

// Scattering-plane matrix from the tables at size coordinate s (bin tables linear
// in ln x between neighbouring bins, a single bin as it is) and cos Theta = mu: the
// function the network approximates.
__device__ __forceinline__ void table_at(const TablesDev& t, float s, float mu, float P[6]) {
    int k = 0;
    float f = 0.f;
    if (t.n_bins > 1) {
        const float x = (fminf(fmaxf(s, -1.f), 1.f) + 1.f) * 0.5f * (float)(t.n_bins - 1);
        k = (int)floorf(x);
        k = k > t.n_bins - 2 ? t.n_bins - 2 : (k < 0 ? 0 : k);
        f = x - (float)k;
    }
    table_matrix(t.bins + (size_t)k * t.n_theta * 2, t.n_theta, mu, P);
    if (f > 0.f) {
        float P2[6];
        table_matrix(t.bins + (size_t)(k + 1) * t.n_theta * 2, t.n_theta, mu, P2);
#pragma unroll
        for (int e = 0; e < 6; ++e) P[e] = (1.f - f) * P[e] + f * P2[e];
    }
}

// A general 4x4 scattering-plane matrix z * m (m row-major, m[0] = 1) applied with
// the plane rotations r: X in the basis of the incident direction, Y in that of the
// scattered one (the six-element case is apply_plane).
__device__ __forceinline__ void apply_plane_full(const PlaneRot<float>& r, float z, const float m[16], const float X[4],
                                                 float Y[4]) {
    const float Xs[4] = {X[0], r.c1 * X[1] + r.s1 * X[2], -r.s1 * X[1] + r.c1 * X[2], X[3]};
    float Ys[4];
#pragma unroll
    for (int row = 0; row < 4; ++row)
        Ys[row] = z * (m[4 * row] * Xs[0] + m[4 * row + 1] * Xs[1] + m[4 * row + 2] * Xs[2] + m[4 * row + 3] * Xs[3]);
    Y[0] = Ys[0];
    Y[1] = r.c2 * Ys[1] + r.s2 * Ys[2];
    Y[2] = -r.s2 * Ys[1] + r.c2 * Ys[2];
    Y[3] = Ys[3];
}

// A packet waiting between kernels: 8 float4 (128 bytes); its cell record is
// reloaded from (ix, iy, iz) and its level (root grid or patch) when it resumes.  parked = 1: stopped inside its flight
// (nothing to do before it resumes), 0: waiting for its scattering.
__device__ __forceinline__ void store_state(float4* d, const Packet<float>& pk, unsigned parked = 0u) {
    const unsigned long long pid = (unsigned long long)pk.pid;
    d[0] = make_float4(pk.px, pk.py, pk.pz, pk.X0);
    d[1] = make_float4(pk.nx, pk.ny, pk.nz, pk.X1);
    d[2] = make_float4(pk.X2, pk.X3, pk.I_birth, pk.e_abs);
    d[3] = make_float4(pk.e_gain, pk.s_flight, __int_as_float(pk.src), 0.f);
    float ta, tb;
    tau_pack(pk.tau, ta, tb);
    d[4] = make_float4(__uint_as_float((unsigned)(pid & 0xffffffffull)), __uint_as_float((unsigned)(pid >> 32)), ta, tb);
    d[5] = make_float4(__uint_as_float(pk.events), __uint_as_float(pk.n_seg), __uint_as_float(pk.n_sca),
                       __uint_as_float(pk.n_tally));
    d[6] = make_float4(__uint_as_float(pk.n_abs), __uint_as_float(pk.trials), __int_as_float(pk.ix),
                       __int_as_float(pk.iy));
    d[7] = make_float4(__int_as_float(pk.iz), __uint_as_float(parked), __int_as_float(pk.lvl), 0.f);
}

__device__ __forceinline__ void load_state(const float4* d, Packet<float>& pk) {
    const float4 a = d[0], b = d[1], c = d[2], e = d[3], f = d[4], g = d[5], h = d[6], k = d[7];
    pk.px = a.x;
    pk.py = a.y;
    pk.pz = a.z;
    pk.X0 = a.w;
    pk.nx = b.x;
    pk.ny = b.y;
    pk.nz = b.z;
    pk.X1 = b.w;
    pk.X2 = c.x;
    pk.X3 = c.y;
    pk.I_birth = c.z;
    pk.e_abs = c.w;
    pk.e_gain = e.x;
    pk.s_flight = e.y;
    pk.src = __float_as_int(e.z);
    pk.pid = (long long)(((unsigned long long)__float_as_uint(f.y) << 32) | (unsigned long long)__float_as_uint(f.x));
    tau_unpack(pk.tau, f.z, f.w);
    pk.events = __float_as_uint(g.x);
    pk.n_seg = __float_as_uint(g.y);
    pk.n_sca = __float_as_uint(g.z);
    pk.n_tally = __float_as_uint(g.w);
    pk.n_abs = __float_as_uint(h.x);
    pk.trials = __float_as_uint(h.y);
    pk.ix = __float_as_int(h.z);
    pk.iy = __float_as_int(h.w);
    pk.iz = __float_as_int(k.x);
    pk.lvl = __float_as_int(k.z);
    pk.job = nullptr;
    pk.park = false;
    pk.pending = false;
}

}  // namespace
}  // namespace mcrt
