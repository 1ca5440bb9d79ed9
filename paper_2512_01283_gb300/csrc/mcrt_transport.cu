// mcrt_transport.cu -- step 1 of the two-step scheme (Kratos-polrad, arXiv:2512.01283,
// Sec. 2.2-2.3): persistent, thread-per-packet Monte-Carlo transport of Stokes
// packets through the grid.
//
// Design (GB300): one warp holds 32 independent packets in registers; a lane whose
// packet ends takes the next packet id from a global counter (one atomic per warp,
// via a coalesced group) and is reborn in place, so warps stay full until the pool
// drains.  Each loop iteration moves every live packet by one cell segment (DDA),
// applies the in-cell analytic extinction (App. A) in the grain-meridian basis
// (eq. rotation-angle / stokes-rotation, quaternions of eq. grain-quaternion), and
// adds the segment's path integral through Z(Omega_cam; Omega_pp) to the FP64
// source tally of every camera (eq. scat-disc-sum).  Lanes of a warp in the same
// cell are found with __match_any_sync and their tally contributions are summed in
// registers before one FP64 atomic per group.  Scattering events draw a new
// direction by rejection sampling of the polarization-aware cross section.
// Per-step arithmetic runs in T (float or double); the remaining scattering optical
// depth and all tallies are FP64.
#include <cooperative_groups.h>

#include "mcrt_device.cuh"
#include "mcrt_internal.h"

namespace cg = cooperative_groups;

namespace mcrt {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDefaultBlock = 256;

template <typename T> struct Packet {
    T p[3], n[3], X[4];
    double tau;  // remaining scattering optical depth
    T I_birth;
    long long pid;
    long long events, n_seg;
    unsigned n_sca;
    int idx[3];
    int src;
};

struct LocalStats {
    double e_emit, e_esc, e_abs, lost, gain, cap_lost;
    unsigned long long events, seg, sca, emitted, escaped, killed, caps, trials, tally_seg, abs_seg;
    unsigned status;
};

template <typename T> struct Smem {
    const T* cam;        // [n_cam][9]: Omega, theta-hat, phi-hat
    const float4* mix;   // [n_theta][2]
    const float4* kext;  // [n_ktheta]
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T> __device__ __forceinline__ void iso_dir(T u_cos, T u_phi, T n[3]) {
    const T ct = T(2) * u_cos - T(1);
    T st = (T(1) - ct) * (T(1) + ct);
    st = st > T(0) ? t_sqrt(st) : T(0);
    T sp, cp;
    t_sincospi(T(2) * u_phi, &sp, &cp);
    n[0] = st * cp;
    n[1] = st * sp;
    n[2] = ct;
}

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

template <typename T>
__device__ __forceinline__ T group_sum(unsigned mask, unsigned peers, T v, unsigned gmax) {
    T acc = T(0);
    unsigned m = peers;
    const int lane = threadIdx.x & 31;
    for (unsigned k = 0; k < gmax; ++k) {
        const int src = m ? (__ffs(m) - 1) : lane;
        const T x = __shfl_sync(mask, v, src);
        if (m) {
            acc += x;
            m &= m - 1;
        }
    }
    return acc;
}

template <typename T>
__device__ void finish(const TransportParams& P, const Packet<T>& pk, int flag, LocalStats& st) {
    if (flag == 1) {
        st.e_esc += (double)pk.X[0];
        st.escaped++;
    } else if (flag == 2) {
        st.killed++;
    } else {
        st.cap_lost += (double)pk.X[0];
        st.caps++;
        st.status |= (flag == 3) ? MCRT_STATUS_EVENT_CAP : MCRT_STATUS_TRIAL_CAP;
    }
    if (P.trace && pk.pid < P.n_trace) {
        double* tr = P.trace + pk.pid * 16;
        tr[0] = pk.X[0];
        tr[1] = pk.X[1];
        tr[2] = pk.X[2];
        tr[3] = pk.X[3];
        tr[4] = pk.p[0];
        tr[5] = pk.p[1];
        tr[6] = pk.p[2];
        tr[7] = pk.n[0];
        tr[8] = pk.n[1];
        tr[9] = pk.n[2];
        tr[10] = (double)pk.n_sca;
        tr[11] = (double)pk.n_seg;
        tr[12] = (double)flag;
        tr[13] = (double)pk.I_birth;
        tr[14] = (double)pk.src;
        tr[15] = (double)pk.events;
    }
}

// Packet birth, event 0: slot 0 = (tau, cos theta, phi, cell), slot 1 = (x, y, z, -).
template <typename T>
__device__ bool emit(const TransportParams& P, const GridT<T>& g, const Smem<T>& sm, long long pid, Packet<T>& pk,
                     LocalStats& st) {
    int s = 0;
    while (s < P.n_src - 1 && pid >= P.src[s].start + P.src[s].count) ++s;
    const SourceDev& src = P.src[s];
    const Draw4<T> u0 = draw4<T>(pid, 0u, 0u, P.seed, P.stream);
    const Draw4<T> u1 = draw4<T>(pid, 0u, 1u, P.seed, P.stream);
    pk.pid = pid;
    pk.src = s;
    pk.events = 1;
    pk.n_seg = 0;
    pk.n_sca = 0;
    const T eps = T(src.eps);
    pk.X[0] = eps;
    pk.X[1] = pk.X[2] = pk.X[3] = T(0);
    bool inside;
    if (src.type == MCRT_SRC_POINT) {
        pk.p[0] = T(src.pos[0]);
        pk.p[1] = T(src.pos[1]);
        pk.p[2] = T(src.pos[2]);
        iso_dir(u0.b, u0.c, pk.n);
        inside = locate(g, pk.p, pk.n, pk.idx);
    } else if (src.type == MCRT_SRC_BEAM) {
        pk.p[0] = T(P.g.lo[0] + (double)u1.a * (P.g.hi[0] - P.g.lo[0]));
        pk.p[1] = T(P.g.lo[1] + (double)u1.b * (P.g.hi[1] - P.g.lo[1]));
        pk.p[2] = T(src.beam_dir > 0 ? P.g.lo[2] : P.g.hi[2]);
        pk.n[0] = T(0);
        pk.n[1] = T(0);
        pk.n[2] = src.beam_dir > 0 ? T(1) : T(-1);
        inside = locate(g, pk.p, pk.n, pk.idx);
    } else {
        // first cell whose cumulative emission weight exceeds u * total
        const double target = (double)u0.d * P.thermal_total;
        long long lo = 0, hi = P.g.ncell - 1;
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (P.thermal_cdf[mid] > target)
                hi = mid;
            else
                lo = mid + 1;
        }
        const long long c = lo;
        pk.idx[0] = (int)(c % g.n[0]);
        pk.idx[1] = (int)((c / g.n[0]) % g.n[1]);
        pk.idx[2] = (int)(c / ((long long)g.n[0] * g.n[1]));
        const T uu[3] = {u1.a, u1.b, u1.c};
        for (int a = 0; a < 3; ++a) pk.p[a] = g.lo[a] + (T(pk.idx[a]) + uu[a]) * g.d[a];
        iso_dir(u0.b, u0.c, pk.n);
        inside = true;
        // emission alpha_abs B (1,0,0,0) in the grain-meridian basis
        const float4 q = P.g.cells[2 * c];
        const float4 r = P.g.cells[2 * c + 1];
        const T kext = T(r.x) + T(r.y);
        const T omega = kext > T(0) ? T(r.y) / kext : T(0);
        V3<T> n{pk.n[0], pk.n[1], pk.n[2]}, th, ph;
        stokes_basis(n, th, ph);
        const GrainFrame<T> f = grain_frame(q, n, ph);
        T a1, a2, a3;
        kext_eval(P.t, sm.kext, f.cos_tp, a1, a2, a3);
        const T w = (a1 - omega) / (T(P.t.alpha1_mean) - omega);
        pk.X[0] = eps * w;
        pk.X[1] = eps * w * a2 / (a1 - omega);
        rotate_qu(pk.X[1], pk.X[2], f.c2, -f.s2);
    }
    pk.tau = -(double)t_log(u0.a);
    pk.I_birth = pk.X[0];
    st.e_emit += (double)pk.X[0];
    st.emitted++;
    st.events++;
    if (!inside) finish(P, pk, 1, st);
    return inside;
}

// One event of a live packet: a cell segment, followed by a scattering when the
// sampled optical depth runs out inside the cell.  `work` = live lanes of the warp.
template <typename T, int SCAT>
__device__ void step(const TransportParams& P, const GridT<T>& g, const Smem<T>& sm, Packet<T>& pk, bool& alive,
                     LocalStats& st, unsigned work) {
    const long long c = ((long long)pk.idx[2] * g.n[1] + pk.idx[1]) * g.n[0] + pk.idx[0];
    const bool capped = pk.events >= P.max_events;
    const float4 q = __ldg(&P.g.cells[2 * c]);
    const float4 r = __ldg(&P.g.cells[2 * c + 1]);
    const T ks = T(r.y);
    const T kext = T(r.x) + ks;
    int axis;
    const T ell_exit = exit_distance(g, pk.idx, pk.p, pk.n, axis);
    // a packet without a finite exit (non-finite direction) ends as escaped
    const bool lost = !capped && axis < 0;
    const bool want_A = !capped && !lost && kext > T(0);
    const bool want_S = want_A && ks > T(0) && P.n_cam > 0;
    // converged point: same-cell groups for the aggregated tallies; lanes that
    // leave below are outside actA / actS
    const unsigned peers = __match_any_sync(work, (unsigned)c);
    const unsigned actA = __ballot_sync(work, want_A);
    const unsigned actS = __ballot_sync(work, want_S);
    if (capped || lost) {
        finish(P, pk, capped ? 3 : 1, st);
        alive = false;
        return;
    }
    const T omega = kext > T(0) ? ks / kext : T(0);
    const T dsca_exit = ks * ell_exit;
    const bool scatter_here = (ks > T(0)) && (pk.tau < (double)dsca_exit);
    const T ell = scatter_here ? T(pk.tau) / ks : ell_exit;
    const V3<T> n{pk.n[0], pk.n[1], pk.n[2]};
    V3<T> th, ph;
    stokes_basis(n, th, ph);
    const int lane = threadIdx.x & 31;
    // same-cell lanes that tally (a capped lane may share the cell but has left)
    const unsigned group = peers & actA;
    const int leader = __ffs(group) - 1;

    if (want_A) {
        T c2 = T(1), s2 = T(0), a1, a2, a3;
        if (P.t.k_iso) {
            a1 = T(sm.kext[0].x);
            a2 = T(0);
            a3 = T(0);
        } else {
            const GrainFrame<T> f = grain_frame(q, n, ph);
            c2 = f.c2;
            s2 = f.s2;
            kext_eval(P.t, sm.kext, f.cos_tp, a1, a2, a3);
        }
        const T a = a1 - omega;
        const T dtau = kext * ell;
        T Xg[4] = {pk.X[0], pk.X[1], pk.X[2], pk.X[3]};
        rotate_qu(Xg[1], Xg[2], c2, s2);
        T Yg[4], Wg[4];
        transfer(Xg, a, a2, a3, dtau, Yg, Wg, want_S, ell);
        rotate_qu(Yg[1], Yg[2], c2, -s2);
        // absorbed energy, one FP64 atomic per same-cell group
        {
            const unsigned gmax = __reduce_max_sync(actA, (unsigned)__popc(group));
            T dI = pk.X[0] - Yg[0];
            st.e_abs += (double)dI;
            if (dI != T(0)) st.abs_seg++;
            if (gmax > 1u) dI = group_sum(actA, group, dI, gmax);
            if (lane == leader && dI != T(0)) atomicAdd(&P.absorbed[c], (double)dI);
        }
        if (want_S) {
            rotate_qu(Wg[1], Wg[2], c2, -s2);
            const T W[4] = {Wg[0], Wg[1], Wg[2], Wg[3]};
            const unsigned gmax = __reduce_max_sync(actS, (unsigned)__popc(group));
            st.tally_seg++;
            double* Sc = P.S + (size_t)c * (size_t)P.n_cam * 4;
            for (int k = 0; k < P.n_cam; ++k) {
                const T* cm = sm.cam + 9 * k;
                const V3<T> Om{cm[0], cm[1], cm[2]}, thc{cm[3], cm[4], cm[5]}, phc{cm[6], cm[7], cm[8]};
                const T mu = dot(n, Om);
                T Pm[6];
                if (SCAT == MCRT_SCAT_RAYLEIGH)
                    rayleigh_matrix(mu, Pm);
                else
                    table_matrix(sm.mix, P.t.n_theta, mu, Pm);
                const PlaneRot<T> pr = plane_rotation(n, th, ph, Om, thc, phc);
                T s[4];
                apply_plane(pr, Pm, W, s);
                if (gmax > 1u) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) s[e] = group_sum(actS, group, s[e], gmax);
                }
                if (lane == leader) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) atomicAdd(Sc + 4 * k + e, (double)s[e]);
                }
            }
        }
        pk.X[0] = Yg[0];
        pk.X[1] = Yg[1];
        pk.X[2] = Yg[2];
        pk.X[3] = Yg[3];
    }
    pk.n_seg++;
    pk.events++;
    st.seg++;
    st.events++;

    if (!scatter_here) {
        pk.tau -= (double)dsca_exit;
        if (!cross_face(g, pk.idx, pk.p, pk.n, ell_exit, axis)) {
            finish(P, pk, 1, st);
            alive = false;
        }
        return;
    }

    // ---- scattering; the packet keeps its cell ----
    for (int a = 0; a < 3; ++a) pk.p[a] += ell * pk.n[a];
    pk.n_sca++;
    pk.events++;
    st.sca++;
    st.events++;
    const Draw4<T> us = draw4<T>(pk.pid, pk.n_sca, 0u, P.seed, P.stream);
    if (P.roulette_thr > 0.0 && (double)pk.X[0] < P.roulette_thr * (double)pk.I_birth) {
        if ((double)us.b < P.roulette_surv) {
            const T gmul = T(1.0 / P.roulette_surv);
            st.gain += (double)pk.X[0] * ((double)gmul - 1.0);
            for (int e = 0; e < 4; ++e) pk.X[e] *= gmul;
        } else {
            st.lost += (double)pk.X[0];
            finish(P, pk, 2, st);
            alive = false;
            return;
        }
    }
    int bin = 0;
    const float4* tab = nullptr;
    if (SCAT == MCRT_SCAT_TABLE) {
        bin = P.t.n_bins - 1;
        for (int k = 0; k < P.t.n_bins; ++k)
            if (us.c < T(P.t.bin_cdf[k])) {
                bin = k;
                break;
            }
        tab = P.t.bins + (size_t)bin * P.t.n_theta * 2;
    }
    V3<T> n2;
    T Pm[6];
    bool accepted = false;
    for (int t = 0; t < P.max_trials; ++t) {
        const Draw4<T> ut = draw4<T>(pk.pid, pk.n_sca, 1u + (unsigned)t, P.seed, P.stream);
        st.trials++;
        T bound;
        if (SCAT == MCRT_SCAT_RAYLEIGH) {
            T g2[3];
            iso_dir(ut.a, ut.b, g2);
            n2 = quat_to_lab(q, V3<T>{g2[0], g2[1], g2[2]});
            rayleigh_matrix(dot(n, n2), Pm);
            bound = ut.c * T(2) * T(0.11936620731892133) * pk.X[0];  // 2 * 3/(8 pi)
        } else {
            // interval j of the piecewise-constant envelope of P11: first j with u < cdf_j
            const int nint = P.t.n_theta - 1;
            const double* cdf = P.t.env_cdf + (size_t)bin * nint;
            int lo = 0, hi = nint - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (ut.a < T(cdf[mid]))
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const int j = lo;
            T s0, c0, s1, c1;
            t_sincospi(T(j) / T(nint), &s0, &c0);
            t_sincospi(T(j + 1) / T(nint), &s1, &c1);
            const T mu = c0 - ut.b * (c0 - c1);
            T sn = (T(1) - mu) * (T(1) + mu);
            sn = sn > T(0) ? t_sqrt(sn) : T(0);
            T sa, ca;
            t_sincospi(T(2) * ut.c, &sa, &ca);
            n2 = V3<T>{mu * n.x + sn * (ca * th.x + sa * ph.x), mu * n.y + sn * (ca * th.y + sa * ph.y),
                       mu * n.z + sn * (ca * th.z + sa * ph.z)};
            table_matrix(tab, P.t.n_theta, mu, Pm);
            bound = ut.d * T(2) * T(P.t.env[(size_t)bin * nint + j]) * pk.X[0];
        }
        const T Qs = plane_Q(n, th, ph, n2, pk.X);
        if (bound < Pm[0] * pk.X[0] + Pm[1] * Qs) {
            accepted = true;
            break;
        }
    }
    if (!accepted) {
        finish(P, pk, 4, st);
        alive = false;
        return;
    }
    V3<T> th2, ph2;
    stokes_basis(n2, th2, ph2);
    const PlaneRot<T> pr = plane_rotation(n, th, ph, n2, th2, ph2);
    T Y[4];
    apply_plane(pr, Pm, pk.X, Y);
    const T norm = pk.X[0] / Y[0];
    for (int e = 0; e < 4; ++e) pk.X[e] = Y[e] * norm;
    pk.n[0] = n2.x;
    pk.n[1] = n2.y;
    pk.n[2] = n2.z;
    pk.tau = -(double)t_log(us.a);
}

template <typename T, int SCAT>
__global__ void __launch_bounds__(kDefaultBlock) k_transport(const __grid_constant__ TransportParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // shared layout: kext table, mixture table (TABLE), cameras
    float4* s_kext = reinterpret_cast<float4*>(smem_raw);
    float4* s_mix = s_kext + P.t.n_ktheta;
    const int n_mix = (SCAT == MCRT_SCAT_TABLE) ? 2 * P.t.n_theta : 0;
    T* s_cam = reinterpret_cast<T*>(s_mix + n_mix);
    for (int i = threadIdx.x; i < P.t.n_ktheta; i += blockDim.x) s_kext[i] = P.t.kext[i];
    for (int i = threadIdx.x; i < n_mix; i += blockDim.x) s_mix[i] = P.t.mix[i];
    for (int i = threadIdx.x; i < 9 * P.n_cam; i += blockDim.x) {
        const CameraDev& cd = P.cam[i / 9];
        const int e = i % 9;
        s_cam[i] = T(e < 3 ? cd.dir[e] : (e < 6 ? cd.th[e - 3] : cd.ph[e - 6]));
    }
    __syncthreads();

    GridT<T> g;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = P.g.n[a];
        g.lo[a] = T(P.g.lo[a]);
        g.d[a] = T(P.g.d[a]);
    }
    const Smem<T> sm{s_cam, s_mix, s_kext};
    LocalStats st = {};
    Packet<T> pk;
    bool alive = false, pool_done = false;
    const unsigned long long t0 = global_ns();

    for (;;) {
        if (!alive && !pool_done) {
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(P.counter, (unsigned long long)grp.size());
            base = grp.shfl(base, 0);
            const long long pid = P.pid_begin + (long long)(base + grp.thread_rank());
            bool late = false;
            if (P.time_budget_ns > 0.0 && (double)(global_ns() - t0) > P.time_budget_ns) late = true;
            if (pid >= P.pid_end || late) {
                pool_done = true;
                if (late && pid < P.pid_end) st.status |= MCRT_STATUS_TIMEOUT;
            } else {
                alive = emit<T>(P, g, sm, pid, pk, st);
            }
        }
        const unsigned work = __ballot_sync(kFull, alive);
        if (work == 0u) {
            if (__all_sync(kFull, pool_done)) break;
            continue;
        }
        if (alive) step<T, SCAT>(P, g, sm, pk, alive, st, work);
    }

    // reduce the per-thread totals: warp shuffle, then one atomic per warp
    double dv[6] = {st.e_emit, st.e_esc, st.e_abs, st.lost, st.gain, st.cap_lost};
    unsigned long long cv[10] = {st.events, st.seg,    st.sca,   st.emitted,   st.escaped,
                                 st.killed, st.caps, st.trials, st.tally_seg, st.abs_seg};
    unsigned status = st.status;
    for (int off = 16; off > 0; off >>= 1) {
        for (int i = 0; i < 6; ++i) dv[i] += __shfl_down_sync(kFull, dv[i], off);
        for (int i = 0; i < 10; ++i) cv[i] += __shfl_down_sync(kFull, cv[i], off);
        status |= __shfl_down_sync(kFull, status, off);
    }
    if ((threadIdx.x & 31) == 0) {
        for (int i = 0; i < 6; ++i) atomicAdd(&P.stats[i], dv[i]);
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(P.stats + 6);
        for (int i = 0; i < 10; ++i) atomicAdd(&cnt[i], cv[i]);
        if (status) atomicOr(P.status, status);
    }
}

}  // namespace

size_t transport_smem_bytes(const TransportParams& p, int precision) {
    const size_t tsize = precision == MCRT_FP64 ? sizeof(double) : sizeof(float);
    const size_t mix = p.t.model == MCRT_SCAT_TABLE ? 2 * (size_t)p.t.n_theta * sizeof(float4) : 0;
    return (size_t)p.t.n_ktheta * sizeof(float4) + mix + 9 * (size_t)p.n_cam * tsize;
}

static const void* kernel_ptr(int precision, int model) {
    if (precision == MCRT_FP64)
        return model == MCRT_SCAT_TABLE ? (const void*)k_transport<double, MCRT_SCAT_TABLE>
                                        : (const void*)k_transport<double, MCRT_SCAT_RAYLEIGH>;
    return model == MCRT_SCAT_TABLE ? (const void*)k_transport<float, MCRT_SCAT_TABLE>
                                    : (const void*)k_transport<float, MCRT_SCAT_RAYLEIGH>;
}

int transport_max_blocks_per_sm(int precision, int model, int block, size_t smem) {
    int nb = 0;
    const void* k = kernel_ptr(precision, model);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_transport(const TransportParams& p, int precision, int block, int grid, cudaStream_t s) {
    const size_t smem = transport_smem_bytes(p, precision);
    const void* k = kernel_ptr(precision, p.t.model);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {const_cast<TransportParams*>(&p)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace mcrt
