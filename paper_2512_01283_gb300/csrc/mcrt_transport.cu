// mcrt_transport.cu -- step 1 of the two-step scheme (Kratos-polrad, arXiv:2512.01283,
// Sec. 2.2-2.3): persistent, thread-per-packet Monte-Carlo transport of Stokes
// packets through the grid.
//
// Design (GB300): one warp holds 32 independent packets in registers; lanes whose
// packets end take the next packet ids from a global counter (one atomic per group
// of lanes, via a coalesced group) and are reborn in place, so warps stay full until
// the pool drains.  Each loop iteration moves every live packet by one cell segment
// (DDA), applies the in-cell analytic extinction (App. A) in the grain-meridian basis
// (eq. rotation-angle / stokes-rotation, quaternions of eq. grain-quaternion), adds
// its absorbed energy with one FP64 atomic, and tallies the segment's path integral
// through Z(Omega_cam; Omega_pp) for every camera (eq. scat-disc-sum): in place, one
// FP64 bulk reduction of the cell's camera rows per lane, or (table rounds and the
// surrogate) as a record that a tally kernel of its own adds.  Scatterings draw a new
// direction by rejection sampling of the polarization-aware cross section, for the
// warp's waiting lanes together.  Per-step arithmetic runs in T (float or double);
// the remaining scattering optical depth and all tallies are FP64.
#include <cooperative_groups.h>

#include "mcrt_device.cuh"
#include "mcrt_internal.h"
#include "mcrt_packet.cuh"
#include "mcrt_refine.cuh"

namespace cg = cooperative_groups;

namespace mcrt {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDefaultBlock = 128;
// resident blocks per SM the FP32 kernels are compiled for (register budget 96);
// shared memory (tables + 272 B of tally staging per thread) allows 5 such blocks
#ifndef MCRT_MIN_BLOCKS
#define MCRT_MIN_BLOCKS 5
#endif
// lanes of a warp that wait before the warp runs the scattering code (or takes new
// packets) for all of them at once.  Measured on GB300: the in-place kernels run fastest
// with 4 and 4; the table rounds of the 192^3 disk, whose births run in a kernel of their
// own, with 6 scatterings (transport 718 ms per 1e8-packet step, against 728 with 4 and
// 738 with 3) and 4 resumed packets (752 ms with 1 or 8); the batched launch of the
// 256-job sweep with 8 and 4 (9.4e9 events/s; 8.7e9 with 4 and 4, 7.5e9 with 1 and 1)
#ifndef MCRT_SCATTER_BATCH
#define MCRT_SCATTER_BATCH 4
#endif
#ifndef MCRT_SCATTER_BATCH_ROUNDS
#define MCRT_SCATTER_BATCH_ROUNDS 6
#endif
#ifndef MCRT_SCATTER_BATCH_JOBS
#define MCRT_SCATTER_BATCH_JOBS 8
#endif
#ifndef MCRT_REFILL_BATCH
#define MCRT_REFILL_BATCH 4
#endif
template <bool B, int SCAT> constexpr int scatter_batch() {
    return B ? MCRT_SCATTER_BATCH_JOBS : (SCAT == kScatTableDeferred ? MCRT_SCATTER_BATCH_ROUNDS : MCRT_SCATTER_BATCH);
}
// per-thread staging slot for the TMA bulk reduction of one segment's source
// contributions: up to 8 cameras x 4 Stokes FP64 (256 B), padded to 272 B so that
// the 16-byte stores of a warp spread over all shared-memory banks
constexpr int kStageCams = 8;
constexpr int kStageDoubles = 34;

template <typename T> struct Smem {
    const T* cam;        // [n_cam][12]: Omega, theta-hat, phi-hat (each padded to 4)
    const float4* mix;   // [n_theta][2]
    const float4* kext;  // [n_ktheta]
    double* stage;       // [blockDim][kStageDoubles]
    unsigned long long* chunk;  // round-based paths: per warp, next and end of its record slots
};

constexpr unsigned kRecChunk = 32u * MCRT_REC_CHUNK;
// Same-cell lanes of a warp pre-sum their absorbed energy before one FP64 atomic (1), or
// every lane adds its own (0, round-based kernels only: there is no in-place tally
// needing the same-cell groups).  Packets of a warp rarely share a cell: without the
// match the table-round transport takes 852 ms per 1e8-packet disk step, 909 ms with it.
#ifndef MCRT_ABS_GROUPS
#define MCRT_ABS_GROUPS 0
#endif
// In-place kernels: same-cell lanes pre-sum their source and absorbed terms (1) or
// every lane reduces its own (0).  Without the match: batched sweep 9.6e9 -> 1.1e10
// events/s, plane-parallel slab 1.15e10 -> 1.25e10, spheroids 1.54e10 -> 1.76e10,
// refined disk 3.8e9 -> 5.1e9.
#ifndef MCRT_INPLACE_GROUPS
#define MCRT_INPLACE_GROUPS 0
#endif

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


// Model-dependent data a packet reads: for a single-model launch the kernel
// parameters and the tables staged in shared memory; for a batched launch the
// packet's record in the job table (tables read through L1).
template <typename T, bool B> struct JobRef;

template <typename T> struct JobRef<T, false> {
    const TransportParams& P;
    const float4* kx;
    const float4* mx;
    __device__ __forceinline__ int n(int a) const { return P.g.n[a]; }
    __device__ __forceinline__ int periodic() const { return P.g.periodic; }
    __device__ __forceinline__ T lo(int a) const { return pick<T>(P.lo_f[a], P.g.lo[a]); }
    __device__ __forceinline__ T d(int a) const { return pick<T>(P.d_f[a], P.g.d[a]); }
    __device__ __forceinline__ double lo_d(int a) const { return P.g.lo[a]; }
    __device__ __forceinline__ double hi_d(int a) const { return P.g.hi[a]; }
    __device__ __forceinline__ long long ncell() const { return P.g.ncell; }
    __device__ __forceinline__ const float4* cells() const { return P.g.cells; }
    __device__ __forceinline__ double* S() const { return P.S; }
    __device__ __forceinline__ double* absorbed() const { return P.absorbed; }
    __device__ __forceinline__ const TablesDev& t() const { return P.t; }
    __device__ __forceinline__ const float4* kext() const { return kx; }
    __device__ __forceinline__ const float4* mix() const { return mx; }
    __device__ __forceinline__ unsigned stream() const { return P.stream; }
    __device__ __forceinline__ double eps(int s) const { return P.src[s].eps; }
    __device__ __forceinline__ const double* cdf() const { return P.thermal_cdf; }
    __device__ __forceinline__ double cdf_total() const { return P.thermal_total; }
    __device__ __forceinline__ const long long* guide() const { return P.thermal_guide; }
    __device__ __forceinline__ long long n_guide() const { return P.n_guide; }
    __device__ __forceinline__ unsigned index() const { return 0u; }
    __device__ __forceinline__ int n_patches() const { return P.g.n_patches; }
    __device__ __forceinline__ const PatchDev* patches() const { return P.g.patches; }
    __device__ __forceinline__ long long ncell_root() const { return P.g.ncell_root; }
};

template <typename T> struct JobRef<T, true> {
    const JobDev* j;
    __device__ __forceinline__ int n(int a) const { return j->n[a]; }
    __device__ __forceinline__ int periodic() const { return j->periodic; }
    __device__ __forceinline__ T lo(int a) const { return pick<T>(j->lo_f[a], j->lo[a]); }
    __device__ __forceinline__ T d(int a) const { return pick<T>(j->d_f[a], j->d[a]); }
    __device__ __forceinline__ double lo_d(int a) const { return j->lo[a]; }
    __device__ __forceinline__ double hi_d(int a) const { return j->hi[a]; }
    __device__ __forceinline__ long long ncell() const { return j->ncell; }
    __device__ __forceinline__ const float4* cells() const { return j->cells; }
    __device__ __forceinline__ double* S() const { return j->S; }
    __device__ __forceinline__ double* absorbed() const { return j->absorbed; }
    __device__ __forceinline__ const TablesDev& t() const { return j->t; }
    __device__ __forceinline__ const float4* kext() const { return j->t.kext; }
    __device__ __forceinline__ const float4* mix() const { return j->t.mix; }
    __device__ __forceinline__ unsigned stream() const { return j->stream; }
    __device__ __forceinline__ double eps(int s) const { return j->src_eps[s]; }
    __device__ __forceinline__ const double* cdf() const { return j->thermal_cdf; }
    __device__ __forceinline__ double cdf_total() const { return j->thermal_total; }
    __device__ __forceinline__ const long long* guide() const { return j->thermal_guide; }
    __device__ __forceinline__ long long n_guide() const { return j->n_guide; }
    __device__ __forceinline__ unsigned index() const { return j->index; }
    // batched launches refuse refined grids
    __device__ __forceinline__ int n_patches() const { return 0; }
    __device__ __forceinline__ const PatchDev* patches() const { return nullptr; }
    __device__ __forceinline__ long long ncell_root() const { return j->ncell; }
};

template <typename T, bool B>
__device__ __forceinline__ JobRef<T, B> job_of(const TransportParams& P, const Smem<T>& sm, const Packet<T>& pk) {
    if constexpr (B)
        return JobRef<T, true>{pk.job};
    else
        return JobRef<T, false>{P, sm.kext, sm.mix};
}


template <typename J>
__device__ __forceinline__ void load_cell(const J& job, int ix, int iy, int iz, float4& q, float4& r) {
    const long long c = ((long long)iz * job.n(1) + iy) * job.n(0) + ix;
    q = __ldg(&job.cells()[2 * c]);
    r = __ldg(&job.cells()[2 * c + 1]);
}

// Composite grids: a packet that has just entered a root cell covered by a patch moves
// into the patch cell that holds its position (entry cell for its direction).
template <typename T, typename J> __device__ __forceinline__ void descend(const J& job, Packet<T>& pk) {
    const int q = covering_patch(pk.cr);
    if (q < 0) return;
    const PatchDev& pq = job.patches()[q];
    int idx[3];
    patch_locate<T>(pq, pk.px, pk.py, pk.pz, pk.nx, pk.ny, pk.nz, idx);
    pk.ix = idx[0];
    pk.iy = idx[1];
    pk.iz = idx[2];
    pk.lvl = q + 1;
    const long long c = patch_cell(pq, idx[0], idx[1], idx[2]);
    pk.cq = __ldg(&job.cells()[2 * c]);
    pk.cr = __ldg(&job.cells()[2 * c + 1]);
}

// Exit of the current patch cell along n (as exit_face, with the patch's geometry).
template <typename T>
__device__ __forceinline__ T exit_face_patch(const PatchDev& q, const Packet<T>& pk, int& axis, T& face) {
    T best = T(INFINITY);
    axis = -1;
    face = T(0);
    const T p[3] = {pk.px, pk.py, pk.pz}, n[3] = {pk.nx, pk.ny, pk.nz};
    const int id[3] = {pk.ix, pk.iy, pk.iz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (n[a] != T(0)) {
            const T f = patch_lo<T>(q, a) + T(n[a] > T(0) ? id[a] + 1 : id[a]) * patch_d<T>(q, a);
            T t = t_div(f - p[a], n[a]);
            t = t < T(0) ? T(0) : t;
            if (t < best) {
                best = t;
                axis = a;
                face = f;
            }
        }
    }
    return best;
}


// First cell whose cumulative emission weight exceeds `target`: a guide table over
// equal steps of the total narrows the search, and the answer is checked against
// the definition (full binary search when the check fails).
template <typename J> __device__ __forceinline__ long long thermal_cell(const J& job, double u) {
    const double* cdf = job.cdf();
    const double target = u * job.cdf_total();
    const long long last = job.ncell() - 1;
    long long lo = 0, hi = last;
    const long long* guide = job.guide();
    if (guide) {
        const long long ng = job.n_guide();
        long long k = (long long)(u * (double)ng);
        k = k < 0 ? 0 : (k >= ng ? ng - 1 : k);
        lo = guide[k];
        hi = guide[k + 1];
    }
    while (lo < hi) {
        const long long mid = lo + (hi - lo) / 2;
        if (cdf[mid] > target)
            hi = mid;
        else
            lo = mid + 1;
    }
    const bool ok = cdf[lo] > target || lo == last;
    const bool ok_prev = lo == 0 || !(cdf[lo - 1] > target);
    if (ok && ok_prev) return lo;
    lo = 0;
    hi = last;
    while (lo < hi) {
        const long long mid = lo + (hi - lo) / 2;
        if (cdf[mid] > target)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// Packet birth, event 0: slot 0 = (tau, cos theta, phi, cell), slot 1 = (x, y, z, -).
// pid is the packet id within its model.  Returns false when the packet starts
// outside the grid (it is then finished).
// WP: the instantiation walks composite grids (births in patch cells).
template <typename T, bool B, bool WP>
__device__ bool emit(const TransportParams& P, const JobRef<T, B>& job, long long pid, Packet<T>& pk, BlockTotals& bt) {
    int s = 0;
    while (s < P.n_src - 1 && pid >= P.src[s].start + P.src[s].count) ++s;
    const SourceDev& src = P.src[s];
    const Draw4<T> u0 = draw4<T>(pid, 0u, 0u, P.seed, job.stream());
    const Draw4<T> u1 = draw4<T>(pid, 0u, 1u, P.seed, job.stream());
    pk.pid = pid;
    pk.src = s;
    pk.s_flight = flight_size(job.t(), u1.d);
    pk.pending = false;
    pk.events = 1;
    pk.n_seg = pk.n_sca = pk.n_tally = pk.n_abs = pk.trials = 0;
    pk.e_abs = pk.e_gain = T(0);
    const T eps = T(job.eps(s));
    pk.X0 = eps;
    pk.X1 = pk.X2 = pk.X3 = T(0);
    bool inside;
    pk.lvl = 0;
    if (src.type == MCRT_SRC_THERMAL) {
        const long long c = thermal_cell(job, (double)u0.d);
        if (WP && job.n_patches() > 0 && c >= job.ncell_root()) {
            // a cell of a refined patch
            int q = job.n_patches() - 1;
            while (q > 0 && job.patches()[q].offset > c) --q;
            const PatchDev& pq = job.patches()[q];
            const long long l = c - pq.offset;
            pk.ix = (int)(l % pq.n[0]);
            pk.iy = (int)((l / pq.n[0]) % pq.n[1]);
            pk.iz = (int)(l / ((long long)pq.n[0] * pq.n[1]));
            pk.px = patch_lo<T>(pq, 0) + (T(pk.ix) + u1.a) * patch_d<T>(pq, 0);
            pk.py = patch_lo<T>(pq, 1) + (T(pk.iy) + u1.b) * patch_d<T>(pq, 1);
            pk.pz = patch_lo<T>(pq, 2) + (T(pk.iz) + u1.c) * patch_d<T>(pq, 2);
            pk.lvl = q + 1;
            pk.cq = __ldg(&job.cells()[2 * c]);
            pk.cr = __ldg(&job.cells()[2 * c + 1]);
        } else {
            pk.ix = (int)(c % job.n(0));
            pk.iy = (int)((c / job.n(0)) % job.n(1));
            pk.iz = (int)(c / ((long long)job.n(0) * job.n(1)));
            pk.px = job.lo(0) + (T(pk.ix) + u1.a) * job.d(0);
            pk.py = job.lo(1) + (T(pk.iy) + u1.b) * job.d(1);
            pk.pz = job.lo(2) + (T(pk.iz) + u1.c) * job.d(2);
            load_cell(job, pk.ix, pk.iy, pk.iz, pk.cq, pk.cr);
        }
        T n[3];
        iso_dir(u0.b, u0.c, n);
        pk.nx = n[0];
        pk.ny = n[1];
        pk.nz = n[2];
        inside = true;
        // emission alpha_abs B (1,0,0,0) in the grain-meridian basis, with alpha_abs the
        // absorption part of K (K minus its scattering part (s11, s12)); weight
        // alpha_abs,11(theta') over its mean over directions (mean alpha1 - omega)
        const T kext = T(pk.cr.x) + T(pk.cr.y);
        const T omega = kext > T(0) ? T(pk.cr.y) / kext : T(0);
        const V3<T> nv{pk.nx, pk.ny, pk.nz};
        V3<T> th, ph;
        stokes_basis(nv, th, ph);
        const GrainFrame<T> f = grain_frame(pk.cq, nv, ph);
        const TablesDev& tb = job.t();
        T a1, a2, a3, s11 = omega, s12 = T(0);
        if (tb.model == MCRT_SCAT_DIPOLE) {
            const DipoleConst<T> dc = dipole_const<T>(tb.dip);
            dipole_K(dc.ca0, dc.ca1, dc.cs0, dc.cs1, T(pk.cr.x) / kext, omega,
                     f.cos_tp, a1, a2, s11, s12);
            a3 = T(0);
        } else {
            kext_eval(tb, job.kext(), f.cos_tp, a1, a2, a3);
        }
        const T w = (a1 - s11) / (T(tb.alpha1_mean) - omega);
        pk.X0 = eps * w;
        pk.X1 = (a1 - s11) > T(0) ? eps * w * (a2 - s12) / (a1 - s11) : T(0);
        rotate_qu(pk.X1, pk.X2, f.c2, -f.s2);
    } else {
        T p[3], n[3];
        if (src.type == MCRT_SRC_POINT) {
            p[0] = T(src.pos[0]);
            p[1] = T(src.pos[1]);
            p[2] = T(src.pos[2]);
            iso_dir(u0.b, u0.c, n);
        } else {
            p[0] = T(job.lo_d(0) + (double)u1.a * (job.hi_d(0) - job.lo_d(0)));
            p[1] = T(job.lo_d(1) + (double)u1.b * (job.hi_d(1) - job.lo_d(1)));
            p[2] = T(src.beam_dir > 0 ? job.lo_d(2) : job.hi_d(2));
            n[0] = T(0);
            n[1] = T(0);
            n[2] = src.beam_dir > 0 ? T(1) : T(-1);
        }
        GridT<T> g;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g.n[a] = job.n(a);
            g.lo[a] = job.lo(a);
            g.d[a] = job.d(a);
        }
        int idx[3];
        inside = locate(g, p, n, idx);
        pk.px = p[0];
        pk.py = p[1];
        pk.pz = p[2];
        pk.nx = n[0];
        pk.ny = n[1];
        pk.nz = n[2];
        pk.ix = idx[0];
        pk.iy = idx[1];
        pk.iz = idx[2];
        if (inside) load_cell(job, pk.ix, pk.iy, pk.iz, pk.cq, pk.cr);
        if constexpr (WP)
            if (inside && job.n_patches() > 0) descend(job, pk);
    }
    tau_set(pk.tau, -t_log(u0.a));
    pk.I_birth = pk.X0;
    if (!inside) finish(P, pk, 1, bt);
    return inside;
}

// Exit of the current cell along n: distance, axis (ties to the lowest axis) and the
// coordinate of the exit face.
template <typename T, typename J>
__device__ __forceinline__ T exit_face(const J& job, const Packet<T>& pk, int& axis, T& face) {
    T best = T(INFINITY);
    axis = -1;
    face = T(0);
    if (pk.nx != T(0)) {
        const T f = job.lo(0) + T(pk.nx > T(0) ? pk.ix + 1 : pk.ix) * job.d(0);
        T t = t_div(f - pk.px, pk.nx);
        t = t < T(0) ? T(0) : t;
        if (t < best) {
            best = t;
            axis = 0;
            face = f;
        }
    }
    if (pk.ny != T(0)) {
        const T f = job.lo(1) + T(pk.ny > T(0) ? pk.iy + 1 : pk.iy) * job.d(1);
        T t = t_div(f - pk.py, pk.ny);
        t = t < T(0) ? T(0) : t;
        if (t < best) {
            best = t;
            axis = 1;
            face = f;
        }
    }
    if (pk.nz != T(0)) {
        const T f = job.lo(2) + T(pk.nz > T(0) ? pk.iz + 1 : pk.iz) * job.d(2);
        T t = t_div(f - pk.pz, pk.nz);
        t = t < T(0) ? T(0) : t;
        if (t < best) {
            best = t;
            axis = 2;
            face = f;
        }
    }
    return best;
}

__host__ __device__ constexpr bool table_optics(int scat) { return scat == MCRT_SCAT_TABLE || scat == kScatTableDeferred; }
__host__ __device__ constexpr bool round_based(int scat) { return scat == kScatSurrogate || scat == kScatTableDeferred; }
// instantiations that may walk composite grids (static mesh refinement): single-model
// launches with the in-place tally or the table rounds; the kernels for grids with
// patches (R) are instantiated apart, so that plain grids keep the plain walk
__host__ __device__ constexpr bool walks_patches(int scat, bool batch) { return !batch && scat != kScatSurrogate; }

// Round-based paths: the packet leaves this launch for the suspend buffer (one slot per
// work item of the launch, so it cannot run over), waiting for its scattering
// (parked = 0) or stopped inside its flight (parked = 1).
template <typename T>
__device__ __forceinline__ void suspend_packet(const TransportParams& P, const Packet<T>& pk, unsigned parked) {
    if constexpr (sizeof(T) == 4) {
        cg::coalesced_group grp = cg::coalesced_threads();
        unsigned long long base = 0;
        if (grp.thread_rank() == 0) base = atomicAdd(&P.sur.ctl->n_suspend, (unsigned long long)grp.size());
        base = grp.shfl(base, 0);
        store_state(P.sur.suspend + (base + grp.thread_rank()) * kStateF4, pk, parked);
    }
}
template <typename T> __device__ __forceinline__ void park_packet(const TransportParams& P, Packet<T>& pk, bool& alive) {
    pk.park = false;
    suspend_packet(P, pk, 1u);
    alive = false;
}

// A tally-record slot that holds no record (skipped by the tally kernels).
template <int SCAT> __device__ __forceinline__ void empty_record(const TransportParams& P, unsigned long long k) {
    if constexpr (SCAT == kScatSurrogate)
        P.sur.records[k * kRecordF4 + 3] = make_float4(__uint_as_float(0xffffffffu), 0.f, 0.f, 0.f);
    else
        P.sur.records[k * kTableRecordF4 + 1] = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xffffffffu));
}

// One event of a live packet: a cell segment, then a scattering when the sampled
// optical depth runs out inside the cell.  `work` = live lanes of the warp.
template <typename T, int SCAT, bool B, bool R>
__device__ __forceinline__ void step(const TransportParams& P, const Smem<T>& sm, Packet<T>& pk, bool& alive,
                                     BlockTotals& bt, unsigned work) {
    const JobRef<T, B> job = job_of<T, B>(P, sm, pk);
    const TablesDev& tabs = job.t();
    const T ks = T(pk.cr.y);
    const T kext = T(pk.cr.x) + ks;
    const bool capped = pk.events >= (unsigned)P.max_events;
    int axis;
    T face;
    // composite grids: the patch the packet is in (nullptr in the root grid)
    const PatchDev* pt = nullptr;
    if constexpr (R)
        if (pk.lvl > 0) pt = &job.patches()[pk.lvl - 1];
    const T ell_exit = pt ? exit_face_patch(*pt, pk, axis, face) : exit_face(job, pk, axis, face);
    // a packet without a finite exit (non-finite direction) ends as escaped
    const bool lost = !capped && axis < 0;
    const bool want_A = !capped && !lost && kext > T(0);
    const bool want_S = want_A && ks > T(0) && P.n_cam > 0;
    const unsigned c32 = pt ? (unsigned)patch_cell(*pt, pk.ix, pk.iy, pk.iz)
                            : (unsigned)(((long long)pk.iz * job.n(1) + pk.iy) * job.n(0) + pk.ix);
    // converged point: same-cell groups (of the same model) for the aggregated
    // tallies; lanes that leave below are outside actA / actS
    constexpr bool kGroups = round_based(SCAT) ? MCRT_ABS_GROUPS : MCRT_INPLACE_GROUPS;
    const unsigned long long key = ((unsigned long long)job.index() << 32) | c32;
    const unsigned peers = kGroups ? __match_any_sync(work, key) : (1u << (threadIdx.x & 31));
    const unsigned actA = __ballot_sync(work, want_A);
    const unsigned actS = __ballot_sync(work, want_S);
    if (capped || lost) {
        finish(P, pk, capped ? 3 : 1, bt);
        alive = false;
        return;
    }
    // scattering rate along n: kappa_sca for Theta-only optics; for aligned spheroids the
    // unpolarized rate kappa_ext s11(theta'), which needs the grain frame first
    T ks_n = ks;
    GrainFrame<T> dip_f{T(1), T(0), T(1)};
    if constexpr (SCAT == MCRT_SCAT_DIPOLE) {
        if (kext > T(0)) {
            const V3<T> n0{pk.nx, pk.ny, pk.nz};
            V3<T> th0, ph0;
            stokes_basis(n0, th0, ph0);
            dip_f = grain_frame(pk.cq, n0, ph0);
            T S2 = (T(1) - dip_f.cos_tp) * (T(1) + dip_f.cos_tp);
            S2 = S2 > T(0) ? S2 : T(0);
            const DipoleConst<T> dc = dipole_const<T>(tabs.dip);
            ks_n = ks * (dc.cs0 + (dc.cs1 - dc.cs0) * T(0.5) * S2);
        }
    }
    const T omega = kext > T(0) ? t_div(ks_n, kext) : T(0);
    const T dsca_exit = ks_n * ell_exit;
    const bool scatter_here = (ks_n > T(0)) && tau_below(pk.tau, dsca_exit);
    const T ell = scatter_here ? T(tau_value(pk.tau)) / ks_n : ell_exit;

    // the next cell's record is requested before the segment arithmetic
    int nix = pk.ix, niy = pk.iy, niz = pk.iz;
    bool next_in = true;
    float4 nq = pk.cq, nr = pk.cr;
    if (!scatter_here) {
        int* ni = axis == 0 ? &nix : (axis == 1 ? &niy : &niz);
        const T na = axis == 0 ? pk.nx : (axis == 1 ? pk.ny : pk.nz);
        const int nn = pt ? pt->n[axis] : job.n(axis);
        *ni += na > T(0) ? 1 : -1;
        next_in = *ni >= 0 && *ni < nn;
        if (pt) {
            // within the patch; leaving it is resolved below, once the packet is on the face
            if (next_in) {
                const long long c = patch_cell(*pt, nix, niy, niz);
                nq = __ldg(&job.cells()[2 * c]);
                nr = __ldg(&job.cells()[2 * c + 1]);
            }
        } else {
            if (!next_in && ((job.periodic() >> axis) & 1)) {
                // a periodic axis: the packet re-enters on the opposite face
                face = na > T(0) ? job.lo(axis) : job.lo(axis) + T(nn) * job.d(axis);
                *ni = na > T(0) ? 0 : nn - 1;
                next_in = true;
            }
            if (next_in) load_cell(job, nix, niy, niz, nq, nr);
        }
    }

    const V3<T> n{pk.nx, pk.ny, pk.nz};
    V3<T> th, ph;
    stokes_basis(n, th, ph);
    const int lane = threadIdx.x & 31;
    const unsigned group = peers & actA;  // same-cell lanes that tally
    const int leader = __ffs(group) - 1;

    if (want_A) {
        T c2 = T(1), s2 = T(0), a1, a2, a3;
        T s12 = T(0);  // aligned spheroids: polarization-dependent part of the scattering rate
        if constexpr (SCAT == MCRT_SCAT_DIPOLE) {
            c2 = dip_f.c2;
            s2 = dip_f.s2;
            T s11;
            const DipoleConst<T> dc = dipole_const<T>(tabs.dip);
            dipole_K(dc.ca0, dc.ca1, dc.cs0, dc.cs1,
                     t_div(T(pk.cr.x), kext), t_div(ks, kext), dip_f.cos_tp, a1, a2, s11, s12);
            a3 = T(0);
        } else if (tabs.k_iso) {
            a1 = T(job.kext()[0].x);
            a2 = T(0);
            a3 = T(0);
        } else {
            const GrainFrame<T> f = grain_frame(pk.cq, n, ph);
            c2 = f.c2;
            s2 = f.s2;
            kext_eval(tabs, job.kext(), f.cos_tp, a1, a2, a3);
        }
        const T a = a1 - omega;
        const T dtau = kext * ell;
        T Xg[4] = {pk.X0, pk.X1, pk.X2, pk.X3};
        rotate_qu(Xg[1], Xg[2], c2, s2);
        T Yg[4], Wg[4];
        transfer(Xg, a, a2, a3, dtau, Yg, Wg, want_S || SCAT == MCRT_SCAT_DIPOLE, ell);
        rotate_qu(Yg[1], Yg[2], c2, -s2);
        // absorbed energy, one FP64 atomic per same-cell group
        {
            const unsigned gmax = kGroups ? __reduce_max_sync(actA, (unsigned)__popc(group)) : 1u;
            // the absorbed energy is int (K_abs X)_0 dl = kappa_ext (a W_I + (a2 - s12) W_Q) over the
            // segment, from the path integral where it is computed: I0 - I1 would cancel in
            // optically thin cells (FP32: nothing absorbed below dtau ~ 6e-8).  For aligned
            // spheroids the decrease of I also holds kappa_ext s12 int Q dl, which the scattering
            // weight returns in expectation, hence a2 - s12.
            T dI = pk.X0 - Yg[0];
            if (want_S || SCAT == MCRT_SCAT_DIPOLE) dI = kext * (a * Wg[0] + (a2 - s12) * Wg[1]);
            pk.e_abs += dI;
            if (dI != T(0)) pk.n_abs++;
            if (gmax > 1u) dI = group_sum(actA, group, dI, gmax);
            if (lane == leader && dI != T(0)) atomicAdd(&job.absorbed()[c32], widen(dI));
        }
        bool queued = false;
        if constexpr (round_based(SCAT)) {
            if (want_S) {
                // the segment's tally waits for its own kernel: one record per lane (64 B
                // with the network's inputs, 32 B for the tables), the warp's records in
                // consecutive slots; a warp that would run past the queue's end writes
                // empty records and tallies in place below
                T Wl1 = Wg[1], Wl2 = Wg[2];  // path integral in the packet's basis
                rotate_qu(Wl1, Wl2, c2, -s2);
                const int lead = __ffs(actS) - 1;
                const unsigned cnt = (unsigned)__popc(actS);
                unsigned long long base = 0;
                const unsigned rank = (unsigned)__popc(actS & ((1u << lane) - 1u));
                unsigned long long idx, last;  // this lane's slot; the step's highest slot
                if constexpr (kRecChunk > 0) {
                    // slots from the warp's chunk; when it runs out, the first lanes take its
                    // rest and the others the start of a new chunk
                    unsigned long long* ch = sm.chunk + 2 * (threadIdx.x >> 5);
                    unsigned long long next = ch[0], end = ch[1];
                    const unsigned long long rest = end - next;
                    if (rest >= cnt) {
                        idx = next + rank;
                        last = next + cnt - 1;
                        next += cnt;
                    } else {
                        unsigned long long nb = 0;
                        if (lane == lead) nb = atomicAdd(&P.sur.ctl->n_rec[P.sur.rec_slot], (unsigned long long)kRecChunk);
                        nb = __shfl_sync(actS, nb, lead);
                        idx = rank < rest ? next + rank : nb + (rank - rest);
                        last = nb + (cnt - rest) - 1;
                        next = nb + (cnt - rest);
                        end = nb + kRecChunk;
                    }
                    __syncwarp(actS);
                    if (lane == lead) {
                        ch[0] = next;
                        ch[1] = end;
                    }
                    __syncwarp(actS);
                } else {
                    if (lane == lead) base = atomicAdd(&P.sur.ctl->n_rec[P.sur.rec_slot], (unsigned long long)cnt);
                    base = __shfl_sync(actS, base, lead);
                    idx = base + rank;
                    last = base + cnt - 1;
                }
                queued = last < P.sur.rec_cap;
                if (idx < P.sur.rec_cap) {
                    if constexpr (SCAT == kScatSurrogate) {
                        float4* r = P.sur.records + idx * kRecordF4;
                        if (queued) {
                            r[0] = make_float4((float)n.x, (float)n.y, (float)n.z, (float)pk.s_flight);
                            r[1] = make_float4((float)Wg[0], (float)Wl1, (float)Wl2, (float)Wg[3]);
                            r[2] = pk.cq;
                            r[3] = make_float4(__uint_as_float(c32), 0.f, 0.f, 0.f);
                        } else {
                            r[3] = make_float4(__uint_as_float(0xffffffffu), 0.f, 0.f, 0.f);
                        }
                    } else {
                        float4* r = P.sur.records + idx * kTableRecordF4;
                        if (queued) {
                            r[0] = make_float4((float)n.x, (float)n.y, (float)n.z, (float)Wg[0]);
                            r[1] = make_float4((float)Wl1, (float)Wl2, (float)Wg[3], __uint_as_float(c32));
                        } else {
                            r[1] = make_float4(0.f, 0.f, 0.f, __uint_as_float(0xffffffffu));
                        }
                    }
                    if (queued) pk.n_tally++;
                }
                // a lane whose record lands past the soft limit parks its packet before its
                // next segment and parks all work it takes afterwards, so each thread adds
                // at most one record beyond it and the queue cannot run over (the in-place
                // tally below is a guard that stays unused)
                if (idx >= P.sur.rec_soft) pk.park = true;
                if (lane == lead && last >= P.sur.rec_soft) atomicExch(&P.sur.ctl->full, 1ull);
                if (!queued && lane == lead) atomicAdd(&P.sur.ctl->cnt[kCntOverflow], (unsigned long long)cnt);
            }
        }
        // the table rounds keep no in-place tally (smaller kernel): a segment that finds
        // no queue space is counted and fails the launch, which the soft limit rules out
        if (SCAT != kScatTableDeferred && want_S && !queued) {
            rotate_qu(Wg[1], Wg[2], c2, -s2);
            const unsigned gmax = kGroups ? __reduce_max_sync(actS, (unsigned)__popc(group)) : 1u;
            pk.n_tally++;
            double* Sc = job.S() + (size_t)c32 * (size_t)P.n_cam * 4;
            double* slot = sm.stage + threadIdx.x * kStageDoubles;
            V3<T> ax{T(0), T(0), T(1)};
            if constexpr (SCAT == MCRT_SCAT_DIPOLE) ax = quat_to_lab(pk.cq, ax);
            for (int k0 = 0; k0 < P.n_cam; k0 += kStageCams) {
                const int kn = P.n_cam - k0 < kStageCams ? P.n_cam - k0 : kStageCams;
                if (lane == leader) bulk_wait_read();  // the slot's previous reduction has read it
                for (int k = 0; k < kn; ++k) {
                    V3<T> Om, thc, phc;
                    load_camera(sm.cam + 12 * (k0 + k), Om, thc, phc);
                    T sv[4];
                    if constexpr (SCAT == MCRT_SCAT_DIPOLE) {
                        const DipoleConst<T> dc = dipole_const<T>(tabs.dip);
                        dipole_apply(dc.rho_re, dc.rho_im, dc.zn, ax, th, ph, thc, phc, Wg,
                                     sv);
                    } else {
                        const T mu = dot(n, Om);
                        T Pm[6];
                        if (SCAT == MCRT_SCAT_RAYLEIGH)
                            rayleigh_matrix(mu, Pm);
                        else
                            table_matrix(job.mix(), tabs.n_theta, mu, Pm);
                        const PlaneRot<T> pr = plane_rotation(n, th, ph, Om, thc, phc);
                        apply_plane(pr, Pm, Wg, sv);
                    }
                    if (gmax > 1u) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) sv[e] = group_sum(actS, group, sv[e], gmax);
                    }
                    if (lane == leader) {
                        double2* d2 = reinterpret_cast<double2*>(slot + 4 * k);
                        d2[0] = make_double2(widen(sv[0]), widen(sv[1]));
                        d2[1] = make_double2(widen(sv[2]), widen(sv[3]));
                    }
                }
                if (lane == leader) bulk_reduce_add_f64(Sc + 4 * k0, slot, (unsigned)kn * 32u);
            }
        }
        pk.X0 = Yg[0];
        pk.X1 = Yg[1];
        pk.X2 = Yg[2];
        pk.X3 = Yg[3];
    }
    pk.n_seg++;
    pk.events++;

    if (!scatter_here) {
        tau_sub(pk.tau, dsca_exit);
        pk.px += ell_exit * pk.nx;
        pk.py += ell_exit * pk.ny;
        pk.pz += ell_exit * pk.nz;
        if (axis == 0)
            pk.px = face;
        else if (axis == 1)
            pk.py = face;
        else
            pk.pz = face;
        if constexpr (R) {
            if (pt && !next_in) {
                // out of the patch: the root cell beyond its face (across a periodic face
                // of the root box, the one on the opposite side)
                const T na = axis == 0 ? pk.nx : (axis == 1 ? pk.ny : pk.nz);
                int r[3] = {pt->box[0] + nix / pt->factor, pt->box[1] + niy / pt->factor, pt->box[2] + niz / pt->factor};
                r[axis] = na > T(0) ? pt->box[3 + axis] : pt->box[axis] - 1;
                next_in = r[axis] >= 0 && r[axis] < job.n(axis);
                if (!next_in && ((job.periodic() >> axis) & 1)) {
                    r[axis] = na > T(0) ? 0 : job.n(axis) - 1;
                    const T f = na > T(0) ? job.lo(axis) : job.lo(axis) + T(job.n(axis)) * job.d(axis);
                    if (axis == 0)
                        pk.px = f;
                    else if (axis == 1)
                        pk.py = f;
                    else
                        pk.pz = f;
                    next_in = true;
                }
                nix = r[0];
                niy = r[1];
                niz = r[2];
                pk.lvl = 0;
                if (next_in) load_cell(job, nix, niy, niz, nq, nr);
            }
        }
        pk.ix = nix;
        pk.iy = niy;
        pk.iz = niz;
        if (!next_in) {
            finish(P, pk, 1, bt);
            alive = false;
            return;
        }
        pk.cq = nq;
        pk.cr = nr;
        if constexpr (R)
            if (pk.lvl == 0 && job.n_patches() > 0) descend(job, pk);
        return;
    }

    // ---- scattering; the packet keeps its cell ----
    pk.px += ell * pk.nx;
    pk.py += ell * pk.ny;
    pk.pz += ell * pk.nz;
    pk.n_sca++;
    pk.events++;
    if constexpr (SCAT == kScatSurrogate) {
        // the scattering is done by the network's kernel; the packet waits in the
        // suspend buffer, whose capacity is the launch's number of work items
        suspend_packet(P, pk, 0u);
        alive = false;
        return;
    }
    // the rejection sampling waits until enough lanes of the warp need it (scatter_event)
    pk.pending = true;
}

// Russian roulette at a scattering of a packet whose intensity fell below the threshold
// fraction of its birth intensity: it survives with probability surv, its Stokes
// vector scaled by 1 / surv.  Returns false when the packet ends here.
template <typename T>
__device__ __forceinline__ bool roulette(const TransportParams& P, Packet<T>& pk, T u, BlockTotals& bt) {
    if (P.roulette_thr > 0.0 && (double)pk.X0 < P.roulette_thr * (double)pk.I_birth) {
        if ((double)u < P.roulette_surv) {
            const T gmul = T(1.0 / P.roulette_surv);
            pk.e_gain += pk.X0 * (gmul - T(1));
            pk.X0 *= gmul;
            pk.X1 *= gmul;
            pk.X2 *= gmul;
            pk.X3 *= gmul;
        } else {
            finish(P, pk, 2, bt);
            return false;
        }
    }
    return true;
}

// Size bin of a scattering: the first bin whose cumulative weight exceeds u.
template <typename T> __device__ __forceinline__ int size_bin(const TablesDev& tabs, T u) {
    for (int k = 0; k < tabs.n_bins; ++k)
        if (u < cdf_at<T>(tabs.bin_cdf, tabs.bin_cdf_f, k)) return k;
    return tabs.n_bins - 1;
}

// One trial of the rejection sampling of a tabulated scattering (Sec. 2.2): a scattering
// angle from the piecewise-constant envelope of P11 of the size bin (interval j with
// probability proportional to its envelope mass, cos theta uniform inside it), an
// azimuth uniform around n, accepted when u 2 env_j I lies below the scattered
// intensity P11 I + P12 Q_s.  Returns the proposed direction n2, mu = cos theta and the
// matrix at mu.
template <typename T>
__device__ __forceinline__ bool table_trial(const TablesDev& tabs, int bin, const Draw4<T>& ut, const V3<T>& n,
                                            const V3<T>& th, const V3<T>& ph, const T X[4], V3<T>& n2, T& mu,
                                            T Pm[6]) {
    const float4* tab = tabs.bins + (size_t)bin * tabs.n_theta * 2;
    // interval j of the envelope: first j with u < cdf_j
    const int nint = tabs.n_theta - 1;
    const size_t c0i = (size_t)bin * nint;
    int lo = 0, hi = nint - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ut.a < cdf_at<T>(tabs.env_cdf, tabs.env_cdf_f, c0i + mid))
            hi = mid;
        else
            lo = mid + 1;
    }
    const int j = lo;
    T s0, c0, s1, c1;
    t_sincospi(T(j) / T(nint), &s0, &c0);
    t_sincospi(T(j + 1) / T(nint), &s1, &c1);
    mu = c0 - ut.b * (c0 - c1);
    T sn = (T(1) - mu) * (T(1) + mu);
    sn = sn > T(0) ? t_sqrt(sn) : T(0);
    T sa, ca;
    t_sincospi(T(2) * ut.c, &sa, &ca);
    n2 = V3<T>{mu * n.x + sn * (ca * th.x + sa * ph.x), mu * n.y + sn * (ca * th.y + sa * ph.y),
               mu * n.z + sn * (ca * th.z + sa * ph.z)};
    table_matrix(tab, tabs.n_theta, mu, Pm);
    const T bound = ut.d * T(2) * T(tabs.env[c0i + j]) * X[0];
    const T Qs = plane_Q(th, ph, n2, X);
    return bound < Pm[0] * X[0] + Pm[1] * Qs;
}

// Scattering of a packet at its current position (Sec. 2.2): roulette, size bin, then
// rejection sampling of the new direction; run for the warp's waiting lanes together.
template <typename T, int SCAT, bool B>
__device__ __forceinline__ void scatter_event(const TransportParams& P, const Smem<T>& sm, Packet<T>& pk, bool& alive,
                                              BlockTotals& bt) {
    const JobRef<T, B> job = job_of<T, B>(P, sm, pk);
    const TablesDev& tabs = job.t();
    const V3<T> n{pk.nx, pk.ny, pk.nz};
    V3<T> th, ph;
    stokes_basis(n, th, ph);
    const Draw4<T> us = draw4<T>(pk.pid, pk.n_sca, 0u, P.seed, job.stream());
    if (!roulette(P, pk, us.b, bt)) {
        alive = false;
        return;
    }
    if constexpr (SCAT == MCRT_SCAT_DIPOLE) {
        // aligned spheroid: isotropic proposal, envelope env I >= (Zhat X)_0; the new
        // Stokes vector is Zhat X (K_sca X)_0 / (s11 (Zhat X)_0), i.e. Zhat X renormalised
        // to I + (s12 / s11) Q with Q in the grain-meridian basis
        const DipoleConst<T> dp = dipole_const<T>(tabs.dip);
        const V3<T> ax = quat_to_lab(pk.cq, V3<T>{T(0), T(0), T(1)});
        const GrainFrame<T> f = grain_frame(pk.cq, n, ph);
        T Qg = pk.X1, Ug = pk.X2;
        rotate_qu(Qg, Ug, f.c2, f.s2);
        T S2 = (T(1) - f.cos_tp) * (T(1) + f.cos_tp);
        S2 = S2 > T(0) ? S2 : T(0);
        const T hs = (dp.cs1 - dp.cs0) * T(0.5) * S2;
        const T Iw = pk.X0 + t_div(hs, dp.cs0 + hs) * Qg;
        const T X[4] = {pk.X0, pk.X1, pk.X2, pk.X3};
        const T rho_re = dp.rho_re, rho_im = dp.rho_im, zn = dp.zn, env = dp.env;
        V3<T> n2;
        T Y[4];
        bool accepted = false;
        for (int t = 0; t < P.max_trials; ++t) {
            const Draw4<T> ut = draw4<T>(pk.pid, pk.n_sca, 1u + (unsigned)t, P.seed, job.stream());
            pk.trials++;
            T g2[3];
            iso_dir(ut.a, ut.b, g2);
            n2 = quat_to_lab(pk.cq, V3<T>{g2[0], g2[1], g2[2]});
            V3<T> th2, ph2;
            stokes_basis(n2, th2, ph2);
            dipole_apply(rho_re, rho_im, zn, ax, th, ph, th2, ph2, X, Y);
            if (ut.c * env * X[0] < Y[0]) {
                accepted = true;
                break;
            }
        }
        if (!accepted) {
            finish(P, pk, 4, bt);
            alive = false;
            return;
        }
        const T norm = Iw / Y[0];
        pk.X0 = Y[0] * norm;
        pk.X1 = Y[1] * norm;
        pk.X2 = Y[2] * norm;
        pk.X3 = Y[3] * norm;
        pk.nx = n2.x;
        pk.ny = n2.y;
        pk.nz = n2.z;
        tau_set(pk.tau, -t_log(us.a));
        return;
    }
    const int bin = table_optics(SCAT) ? size_bin(tabs, us.c) : 0;
    const T X[4] = {pk.X0, pk.X1, pk.X2, pk.X3};
    V3<T> n2;
    T Pm[6];
    bool accepted = false;
    for (int t = 0; t < P.max_trials; ++t) {
        const Draw4<T> ut = draw4<T>(pk.pid, pk.n_sca, 1u + (unsigned)t, P.seed, job.stream());
        pk.trials++;
        bool acc;
        if (SCAT == MCRT_SCAT_RAYLEIGH) {
            T g2[3];
            iso_dir(ut.a, ut.b, g2);
            n2 = quat_to_lab(pk.cq, V3<T>{g2[0], g2[1], g2[2]});
            rayleigh_matrix(dot(n, n2), Pm);
            const T bound = ut.c * T(2) * T(0.11936620731892133) * X[0];  // 2 * 3/(8 pi)
            const T Qs = plane_Q(th, ph, n2, X);
            acc = bound < Pm[0] * X[0] + Pm[1] * Qs;
        } else {
            T mu;
            acc = table_trial(tabs, bin, ut, n, th, ph, X, n2, mu, Pm);
        }
        if (acc) {
            accepted = true;
            break;
        }
    }
    if (!accepted) {
        finish(P, pk, 4, bt);
        alive = false;
        return;
    }
    V3<T> th2, ph2;
    stokes_basis(n2, th2, ph2);
    const PlaneRot<T> pr = plane_rotation(n, th, ph, n2, th2, ph2);
    T Y[4];
    apply_plane(pr, Pm, X, Y);
    const T norm = X[0] / Y[0];
    pk.X0 = Y[0] * norm;
    pk.X1 = Y[1] * norm;
    pk.X2 = Y[2] * norm;
    pk.X3 = Y[3] * norm;
    pk.nx = n2.x;
    pk.ny = n2.y;
    pk.nz = n2.z;
    tau_set(pk.tau, -t_log(us.a));
}

// Lane of the k-th set bit of m (k < popc(m)), by halving.
__device__ __forceinline__ int nth_set_lane(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const unsigned lo = m & ((1u << w) - 1u);
        const int c = __popc(lo);
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        } else {
            m = lo;
        }
    }
    return pos;
}

// Scatterings of the warp's waiting lanes with their rejection trials spread over all
// 32 lanes (launches with tabulated optics; in batched launches each trial lane reads
// the tables of its packet's job).  Each owner first takes its roulette and size bin;
// then, round after round, every unresolved packet gets floor(32 / unresolved) lanes
// that evaluate its next trials in trial order, and the packet takes its first
// accepted trial.  Direction, matrix and trial count are thus those of the sequential
// rule (same random numbers, same arithmetic; the trial reads I, Q and U only, so V
// is not passed).  All 32 lanes call it.
template <typename T, bool B>
__device__ __forceinline__ void scatter_coop(const TransportParams& P, const Smem<T>& sm, Packet<T>& pk, bool& alive,
                                             BlockTotals& bt) {
    const int lane = threadIdx.x & 31;
    bool live = false;
    int bin = 0;
    T u_tau = T(1);
    if (alive && pk.pending) {
        pk.pending = false;
        const JobRef<T, B> job = job_of<T, B>(P, sm, pk);
        const TablesDev& tabs = job.t();
        const Draw4<T> us = draw4<T>(pk.pid, pk.n_sca, 0u, P.seed, job.stream());
        live = roulette(P, pk, us.b, bt);
        alive = live;
        bin = size_bin(tabs, us.c);
        u_tau = us.a;
    }
    unsigned todo = __ballot_sync(kFull, live);
    int t_next = 0;          // owner: first trial of its next round
    bool accepted = false;   // owner: a trial was accepted
    V3<T> n2a{T(0), T(0), T(1)};
    T mua = T(1);
    while (todo != 0u) {
        const int nu = __popc(todo);
        const int per = 32 / nu;
        const int k = lane / per;  // packet this lane evaluates (rank among the unresolved)
        const int src = k < nu ? nth_set_lane(todo, k) : lane;
        const V3<T> n{__shfl_sync(kFull, pk.nx, src), __shfl_sync(kFull, pk.ny, src), __shfl_sync(kFull, pk.nz, src)};
        const T X[4] = {__shfl_sync(kFull, pk.X0, src), __shfl_sync(kFull, pk.X1, src),
                        __shfl_sync(kFull, pk.X2, src), T(0)};
        const long long pid = __shfl_sync(kFull, pk.pid, src);
        const unsigned nsca = __shfl_sync(kFull, pk.n_sca, src);
        const int tb = __shfl_sync(kFull, bin, src);
        const int t = __shfl_sync(kFull, t_next, src) + lane % per;
        // the packet's job (batched launches)
        Packet<T> jp;
        if constexpr (B)
            jp.job = reinterpret_cast<const JobDev*>(
                __shfl_sync(kFull, reinterpret_cast<unsigned long long>(pk.job), src));
        bool acc = false;
        V3<T> n2{T(0), T(0), T(1)};
        T mu = T(1);
        if (k < nu && t < P.max_trials) {
            const JobRef<T, B> job = job_of<T, B>(P, sm, jp);
            V3<T> th, ph;
            stokes_basis(n, th, ph);
            const Draw4<T> ut = draw4<T>(pid, nsca, 1u + (unsigned)t, P.seed, job.stream());
            T Pm[6];
            acc = table_trial(job.t(), tb, ut, n, th, ph, X, n2, mu, Pm);
        }
        const unsigned am = __ballot_sync(kFull, acc);
        // each owner: the first accepted trial among its lanes
        const bool own = (todo >> lane) & 1u;
        const int kr = __popc(todo & ((1u << lane) - 1u));
        const unsigned seg = own ? (per >= 32 ? kFull : ((1u << per) - 1u) << (kr * per)) : 0u;
        const unsigned hit = am & seg;
        const int w = hit != 0u ? __ffs(hit) - 1 : lane;
        n2.x = __shfl_sync(kFull, n2.x, w);
        n2.y = __shfl_sync(kFull, n2.y, w);
        n2.z = __shfl_sync(kFull, n2.z, w);
        mu = __shfl_sync(kFull, mu, w);
        if (own) {
            if (hit != 0u) {
                pk.trials += (unsigned)(w - kr * per + 1);
                accepted = true;
                n2a = n2;
                mua = mu;
            } else {
                const int left = P.max_trials - t_next;
                pk.trials += (unsigned)(left < per ? (left > 0 ? left : 0) : per);
                t_next += per;
            }
        }
        todo = __ballot_sync(kFull, own && hit == 0u && t_next < P.max_trials);
    }
    if (!live) return;
    if (!accepted) {
        finish(P, pk, 4, bt);
        alive = false;
        return;
    }
    const TablesDev& tabs = job_of<T, B>(P, sm, pk).t();
    const V3<T> n{pk.nx, pk.ny, pk.nz};
    V3<T> th, ph, th2, ph2;
    stokes_basis(n, th, ph);
    stokes_basis(n2a, th2, ph2);
    T Pm[6];
    table_matrix(tabs.bins + (size_t)bin * tabs.n_theta * 2, tabs.n_theta, mua, Pm);
    const PlaneRot<T> pr = plane_rotation(n, th, ph, n2a, th2, ph2);
    const T X[4] = {pk.X0, pk.X1, pk.X2, pk.X3};
    T Y[4];
    apply_plane(pr, Pm, X, Y);
    const T norm = X[0] / Y[0];
    pk.X0 = Y[0] * norm;
    pk.X1 = Y[1] * norm;
    pk.X2 = Y[2] * norm;
    pk.X3 = Y[3] * norm;
    pk.nx = n2a.x;
    pk.ny = n2a.y;
    pk.nz = n2a.z;
    tau_set(pk.tau, -t_log(u_tau));
}

// Job of a batch packet index: the last job whose first index is <= gpid.
__device__ __forceinline__ int job_index(const TransportParams& P, long long gpid) {
    int lo = 0, hi = P.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.jobs[mid].pid_start <= gpid)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// resident blocks per SM of the table-round instantiation: without the camera loop
// and its staging slots it fits more warps per SM
#ifndef MCRT_ROUND_MIN_BLOCKS
#define MCRT_ROUND_MIN_BLOCKS 7
#endif
template <typename T, int SCAT>
constexpr int min_blocks() {
    return sizeof(T) != 4 ? 1 : (SCAT == kScatTableDeferred ? MCRT_ROUND_MIN_BLOCKS : MCRT_MIN_BLOCKS);
}

template <typename T, int SCAT, bool B, bool R>
__global__ void __launch_bounds__(kDefaultBlock, (min_blocks<T, SCAT>()))
    k_transport(const __grid_constant__ TransportParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockTotals bt;
    __shared__ unsigned long long s_chunk[2 * (kDefaultBlock / 32)];
    // shared layout: kext table and mixture table (single model, TABLE), cameras,
    // tally staging
    float4* s_kext = reinterpret_cast<float4*>(smem_raw);
    const int n_k = B ? 0 : P.t.n_ktheta;
    float4* s_mix = s_kext + n_k;
    const int n_mix = (!B && SCAT != MCRT_SCAT_RAYLEIGH && SCAT != MCRT_SCAT_DIPOLE) ? 2 * P.t.n_theta : 0;
    T* s_cam = reinterpret_cast<T*>(s_mix + n_mix);
    const int cam_bytes = 12 * P.n_cam * (int)sizeof(T);
    double* s_stage = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(s_cam) + cam_bytes);
    for (int i = threadIdx.x; i < n_k; i += blockDim.x) s_kext[i] = P.t.kext[i];
    for (int i = threadIdx.x; i < n_mix; i += blockDim.x) s_mix[i] = P.t.mix[i];
    for (int i = threadIdx.x; i < 12 * P.n_cam; i += blockDim.x) {
        const CameraDev& cd = P.cam[i / 12];
        const int e = i % 12, v = e / 4, w = e % 4;
        s_cam[i] = w == 3 ? T(0) : T(v == 0 ? cd.dir[w] : (v == 1 ? cd.th[w] : cd.ph[w]));
    }
    if (threadIdx.x < 6) bt.e[threadIdx.x] = 0.0;
    if (threadIdx.x < 10) bt.n[threadIdx.x] = 0ull;
    if (threadIdx.x < 2 * (kDefaultBlock / 32)) s_chunk[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) bt.status = 0u;
    __syncthreads();

    const Smem<T> sm{s_cam, s_mix, s_kext, s_stage, s_chunk};
    Packet<T> pk;
    pk.job = nullptr;
    bool alive = false, pool_done = false;
    bool stop = false;  // round-based paths: this lane's record went past the soft limit
    const unsigned long long t0 = global_ns();
    // surrogate path: packets resumed after their scattering, then new packets
    unsigned long long w_resume = 0, w_new = 0, w_next = 0;
    if constexpr (SCAT == kScatTableDeferred) {
        // table rounds: the birth kernel stored the round's new packets after the resume list
        w_resume = P.sur.ctl->n_resume + P.sur.ctl->n_born;
    } else if constexpr (round_based(SCAT)) {
        w_resume = P.sur.ctl->n_resume;
        w_new = P.sur.ctl->n_new;
        w_next = P.sur.ctl->next_pid;
    }

    for (;;) {
        // dead lanes take new work in groups, so that the birth code runs for several
        // lanes at once (or when no lane can move otherwise)
        const unsigned need = __ballot_sync(kFull, !alive && !pool_done);
        const unsigned busy = __ballot_sync(kFull, alive && !pk.pending);
        const bool refill = need != 0u && (__popc(need) >= MCRT_REFILL_BATCH || busy == 0u);
        if constexpr (round_based(SCAT)) {
            if (refill && !alive && !pool_done) {
                cg::coalesced_group grp = cg::coalesced_threads();
                unsigned long long base = 0;
                if (grp.thread_rank() == 0) base = atomicAdd(&P.sur.ctl->claim, (unsigned long long)grp.size());
                base = grp.shfl(base, 0);
                const unsigned long long idx = base + grp.thread_rank();
                // the record queue is near its end: work items taken now wait for the
                // next round without a segment
                const bool full = *reinterpret_cast<volatile unsigned long long*>(&P.sur.ctl->full) != 0ull;
                pk.park = false;
                const JobRef<T, false> jr{P, sm.kext, sm.mix};
                if (idx < w_resume) {
                    if constexpr (sizeof(T) == 4) {
                        load_state(P.sur.resume + idx * kStateF4, pk);
                        if constexpr (!R) pk.lvl = 0;  // plain grids: the root level throughout
                        if (R && pk.lvl > 0) {  // a cell of a refined patch
                            const long long c = patch_cell(jr.patches()[pk.lvl - 1], pk.ix, pk.iy, pk.iz);
                            pk.cq = __ldg(&jr.cells()[2 * c]);
                            pk.cr = __ldg(&jr.cells()[2 * c + 1]);
                        } else {
                            load_cell(jr, pk.ix, pk.iy, pk.iz, pk.cq, pk.cr);
                        }
                        alive = true;
                    }
                } else if (SCAT != kScatTableDeferred && idx - w_resume < w_new) {
                    // the surrogate path emits here; the table rounds hold no birth code
                    if constexpr (SCAT != kScatTableDeferred) {
                        const long long pid = P.pid_begin + (long long)(w_next + (idx - w_resume));
                        alive = emit<T, false, R>(P, jr, pid, pk, bt);
                        pk.park = false;
                    }
                } else {
                    pool_done = true;
                }
                if (alive && (full || stop)) park_packet(P, pk, alive);
            }
            if (alive && pk.park && !pk.pending) {  // before the next segment, outside collective steps
                stop = true;
                park_packet(P, pk, alive);
            }
        } else if (refill && !alive && !pool_done) {
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(P.counter, (unsigned long long)grp.size());
            base = grp.shfl(base, 0);
            const long long pid = P.pid_begin + (long long)(base + grp.thread_rank());
            const bool late = P.time_budget_ns > 0.0 && (double)(global_ns() - t0) > P.time_budget_ns;
            if (pid >= P.pid_end || late) {
                pool_done = true;
                if (late && pid < P.pid_end) atomicOr(&bt.status, (unsigned)MCRT_STATUS_TIMEOUT);
            } else if constexpr (B) {
                long long local;
                if (P.job_interleave) {
                    pk.job = &P.jobs[pid % P.n_jobs];
                    local = pid / P.n_jobs;
                } else {
                    pk.job = &P.jobs[job_index(P, pid)];
                    local = pid - pk.job->pid_start;
                }
                alive = emit<T, true, false>(P, JobRef<T, true>{pk.job}, local, pk, bt);
            } else {
                alive = emit<T, false, R>(P, JobRef<T, false>{P, sm.kext, sm.mix}, pid, pk, bt);
            }
        }
        const unsigned pend = __ballot_sync(kFull, alive && pk.pending);
        const unsigned work = __ballot_sync(kFull, alive && !pk.pending);
        if (work == 0u && pend == 0u) {
            if (__all_sync(kFull, pool_done)) break;
            continue;
        }
        // scatterings of the warp run together once enough lanes wait for one
        if (pend != 0u && (__popc(pend) >= scatter_batch<B, SCAT>() || work == 0u)) {
            if constexpr (table_optics(SCAT)) {
                scatter_coop<T, B>(P, sm, pk, alive, bt);  // every lane runs trials of the waiting packets
            } else if constexpr (SCAT != kScatSurrogate) {  // the surrogate scatters in its own kernel
                if (alive && pk.pending) {
                    pk.pending = false;
                    scatter_event<T, SCAT, B>(P, sm, pk, alive, bt);
                }
            }
            continue;
        }
        if (alive && !pk.pending) step<T, SCAT, B, R>(P, sm, pk, alive, bt, work);
    }

    if constexpr (round_based(SCAT) && kRecChunk > 0) {
        // the warp's unused record slots hold no record
        __syncwarp();
        const unsigned long long next = s_chunk[2 * (threadIdx.x >> 5)], end = s_chunk[2 * (threadIdx.x >> 5) + 1];
        for (unsigned long long k = next + (threadIdx.x & 31); k < end && k < P.sur.rec_cap; k += 32)
            empty_record<SCAT>(P, k);
    }
    bulk_wait_all();  // this thread's reductions have completed before the block ends
    __syncthreads();
    if (threadIdx.x < 6) {
        atomicAdd(&P.stats[threadIdx.x], bt.e[threadIdx.x]);
    } else if (threadIdx.x < 16) {
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(P.stats + 6);
        atomicAdd(&cnt[threadIdx.x - 6], bt.n[threadIdx.x - 6]);
    } else if (threadIdx.x == 16 && bt.status) {
        atomicOr(P.status, bt.status);
    }
}

// Births of a round of the FP32 table path, in a kernel of their own: one thread per
// new packet of the round (so births run with every lane busy and their thermal-cell
// searches overlap), each born packet stored in the 128-byte waiting form after the
// packets resumed from the previous round, where the round's transport kernel takes it
// like a resumed one.  The transport kernel of the table rounds thus holds no birth
// code.  The packet is the one emit() gives inside the transport kernel: the same
// random numbers and FP32 values (the waiting form keeps them exactly), so the
// trajectories do not change.  Packets that start outside the grid are finished here.
constexpr int kBirthBlock = 256;

template <bool R> __global__ void __launch_bounds__(kBirthBlock) k_birth(const __grid_constant__ TransportParams P) {
    __shared__ BlockTotals bt;
    if (threadIdx.x < 6) bt.e[threadIdx.x] = 0.0;
    if (threadIdx.x < 10) bt.n[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) bt.status = 0u;
    __syncthreads();
    const unsigned long long n_new = P.sur.ctl->n_new, first = P.sur.ctl->n_resume, next = P.sur.ctl->next_pid;
    const JobRef<float, false> jr{P, P.t.kext, P.t.mix};
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_new;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        Packet<float> pk;
        pk.job = nullptr;
        const long long pid = P.pid_begin + (long long)(next + i);
        if (emit<float, false, R>(P, jr, pid, pk, bt)) {
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(&P.sur.ctl->n_born, (unsigned long long)grp.size());
            base = grp.shfl(base, 0);
            store_state(P.sur.resume + (first + base + grp.thread_rank()) * kStateF4, pk, 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        if (bt.e[threadIdx.x] != 0.0) atomicAdd(&P.stats[threadIdx.x], bt.e[threadIdx.x]);
    } else if (threadIdx.x < 16) {
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(P.stats + 6);
        if (bt.n[threadIdx.x - 6]) atomicAdd(&cnt[threadIdx.x - 6], bt.n[threadIdx.x - 6]);
    } else if (threadIdx.x == 16 && bt.status) {
        atomicOr(P.status, bt.status);
    }
}

}  // namespace

cudaError_t launch_births(const TransportParams& p, int n_sm, cudaStream_t s) {
    (void)cudaGetLastError();
    const int grid = n_sm * 8;
    if (p.g.n_patches > 0)
        k_birth<true><<<grid, kBirthBlock, 0, s>>>(p);
    else
        k_birth<false><<<grid, kBirthBlock, 0, s>>>(p);
    return cudaGetLastError();
}

size_t transport_smem_bytes(const TransportParams& p, int precision, int block) {
    const bool batch = p.jobs != nullptr;
    const size_t tsize = precision == MCRT_FP64 ? sizeof(double) : sizeof(float);
    const size_t kx = batch ? 0 : (size_t)p.t.n_ktheta * sizeof(float4);
    const size_t mix = (!batch && p.t.model == MCRT_SCAT_TABLE) ? 2 * (size_t)p.t.n_theta * sizeof(float4) : 0;
    const size_t cams = 12 * (size_t)p.n_cam * tsize;
    // the table rounds tally in their own kernel: no staging slots
    const size_t stage = p.sur.deferred == kScatTableDeferred ? 0 : (size_t)block * kStageDoubles * sizeof(double);
    return kx + mix + cams + stage;
}

template <typename T, int SCAT, bool B> const void* kernel_of(bool refined) {
    if constexpr (walks_patches(SCAT, B))
        if (refined) return (const void*)k_transport<T, SCAT, B, true>;
    return (const void*)k_transport<T, SCAT, B, false>;
}

template <typename T> const void* kernel_of_model(int model, bool batch, bool refined) {
    if (model == MCRT_SCAT_DIPOLE)  // single-model launches only
        return kernel_of<T, MCRT_SCAT_DIPOLE, false>(refined);
    if (model == MCRT_SCAT_TABLE)
        return batch ? kernel_of<T, MCRT_SCAT_TABLE, true>(false) : kernel_of<T, MCRT_SCAT_TABLE, false>(refined);
    return batch ? kernel_of<T, MCRT_SCAT_RAYLEIGH, true>(false) : kernel_of<T, MCRT_SCAT_RAYLEIGH, false>(refined);
}

const void* transport_kernel(int precision, int model, bool batch, bool refined) {
    return precision == MCRT_FP64 ? kernel_of_model<double>(model, batch, refined)
                                  : kernel_of_model<float>(model, batch, refined);
}

const void* transport_kernel_rounds(int model, bool refined) {
    if (model == kScatSurrogate) return (const void*)k_transport<float, kScatSurrogate, false, false>;
    return refined ? (const void*)k_transport<float, kScatTableDeferred, false, true>
                   : (const void*)k_transport<float, kScatTableDeferred, false, false>;
}

int transport_max_blocks_per_sm(int precision, int model, bool batch, int block, size_t smem, bool refined) {
    int nb = 0;
    const void* k = round_based(model) ? transport_kernel_rounds(model, refined)
                                        : transport_kernel(precision, model, batch, refined);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_transport(const TransportParams& p, int precision, int block, int grid, cudaStream_t s) {
    const size_t smem = transport_smem_bytes(p, precision, block);
    const void* k = p.sur.deferred ? transport_kernel_rounds(p.sur.deferred, p.g.n_patches > 0)
                                   : transport_kernel(precision, p.t.model, p.jobs != nullptr, p.g.n_patches > 0);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {const_cast<TransportParams*>(&p)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem, s);
}

}  // namespace mcrt
