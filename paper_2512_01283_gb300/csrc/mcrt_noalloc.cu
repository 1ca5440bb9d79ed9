// mcrt_noalloc.cu -- a transport launch that allocates no memory.
//
// Some callers cannot allocate device memory at all: code running inside another
// framework's memory pool or a pre-planned memory budget, or a process whose
// allocator is locked down.  mcrt_launch_packets_noalloc serves them: the caller
// passes every input and output as device memory it already owns, and the
// launch's scratch (cell records with the grain quaternions, prepared scattering
// tables, the packet counter and the launch totals) lives in the file-scope array
// below instead of in cudaMalloc'd buffers.  The array is part of the library
// image, so every GPU that loads the library holds it until the process exits.
//
// The kernels launched are the library's usual set-up and transport kernels; only
// the origin of their scratch differs.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>

#include "mcrt.h"
#include "mcrt_internal.h"

namespace {

using namespace mcrt;

// Limits of the static scratch (documented in include/mcrt.h).
constexpr long long kMaxCells = MCRT_NOALLOC_MAX_CELLS;
constexpr int kMaxBins = MCRT_NOALLOC_MAX_BINS;
constexpr int kMaxTheta = MCRT_NOALLOC_MAX_THETA;

constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
// byte layout of the scratch array
constexpr size_t kOffCells = 0;
constexpr size_t kOffMix = kOffCells + round256((size_t)kMaxCells * 2 * sizeof(float4));
constexpr size_t kOffBins = kOffMix + round256((size_t)kMaxTheta * 2 * sizeof(float4));
constexpr size_t kOffEnvCdf = kOffBins + round256((size_t)kMaxBins * kMaxTheta * 2 * sizeof(float4));
constexpr size_t kOffEnv = kOffEnvCdf + round256((size_t)kMaxBins * (kMaxTheta - 1) * (sizeof(double) + sizeof(float)));
constexpr size_t kOffBinCdf = kOffEnv + round256((size_t)kMaxBins * (kMaxTheta - 1) * sizeof(float));
constexpr size_t kOffKext = kOffBinCdf + round256((size_t)kMaxBins * (sizeof(double) + sizeof(float)));
constexpr size_t kOffWork = kOffKext + round256((size_t)kMaxTheta * sizeof(float4));
// work area: packet counter (8 B), 16 totals (128 B), status (8 B), alpha1 mean (8 B),
// invalid-input flag (8 B)
constexpr size_t kWorkBytes = 8 + 128 + 8 + 8 + 8;
constexpr size_t kScratchBytes = kOffWork + round256(kWorkBytes);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device, looked up on every call
// with that device current: after a cudaDeviceReset, or in another context on the same
// device, the module is loaded anew and the array can sit elsewhere, so no address is
// kept between calls.  The first lookup on a device may load the library's device code.
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

// Device memory of the current device (or managed memory): the kernels read and write
// these buffers directly, so memory of another GPU is refused.
bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

void basis(const double n[3], double th[3], double ph[3]) {
    const double r2 = n[0] * n[0] + n[1] * n[1];
    if (r2 > 0) {
        const double r = 1.0 / std::sqrt(r2);
        ph[0] = -n[1] * r;
        ph[1] = n[0] * r;
        ph[2] = 0.0;
    } else {
        ph[0] = 0.0;
        ph[1] = 1.0;
        ph[2] = 0.0;
    }
    th[0] = ph[1] * n[2] - ph[2] * n[1];
    th[1] = ph[2] * n[0] - ph[0] * n[2];
    th[2] = ph[0] * n[1] - ph[1] * n[0];
}

#define NA_CK(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            (void)cudaGetLastError();                                                        \
            return mcrt_fail_noctx(MCRT_E_CUDA, "mcrt_launch_packets_noalloc: %s: %s", #call, \
                                   cudaGetErrorString(e_));                                  \
        }                                                                                    \
    } while (0)

}  // namespace

extern "C" mcrt_status mcrt_launch_packets_noalloc(const mcrt_noalloc_problem* pr, const mcrt_launch_desc* d,
                                                   mcrt_stats* out_stats) {
    const char* me = "mcrt_launch_packets_noalloc";
    if (!pr || !d) return mcrt_fail_noctx(MCRT_E_INVAL, "%s: problem or desc is NULL", me);
    if (pr->nx < 1 || pr->ny < 1 || pr->nz < 1) return mcrt_fail_noctx(MCRT_E_INVAL, "%s: bad grid shape", me);
    const long long ncell = (long long)pr->nx * pr->ny * pr->nz;
    if (ncell > kMaxCells)
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: %lld cells exceed the static limit of %lld", me, ncell, kMaxCells);
    for (int a = 0; a < 3; ++a)
        if (!(pr->hi[a] > pr->lo[a]) || !std::isfinite(pr->lo[a]) || !std::isfinite(pr->hi[a]))
            return mcrt_fail_noctx(MCRT_E_INVAL, "%s: empty or non-finite box on axis %d", me, a);
    if (pr->model != MCRT_SCAT_RAYLEIGH && pr->model != MCRT_SCAT_TABLE)
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: unknown scattering model %d", me, pr->model);
    const bool table = pr->model == MCRT_SCAT_TABLE;
    if (pr->n_ktheta < 2 || pr->n_ktheta > kMaxTheta)
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: need 2 <= n_ktheta <= %d", me, kMaxTheta);
    if (table && (pr->n_bins < 1 || pr->n_bins > kMaxBins || pr->n_theta < 2 || pr->n_theta > kMaxTheta))
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: need 1 <= n_bins <= %d and 2 <= n_theta <= %d", me, kMaxBins,
                               kMaxTheta);
    if (!on_device(pr->kappa_abs) || !on_device(pr->kappa_sca) || !on_device(pr->kext) ||
        (pr->bfield && !on_device(pr->bfield)) || (table && (!on_device(pr->mueller) || !on_device(pr->bin_weight))))
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: grid and optics inputs must be device memory", me);
    if (!on_device(pr->absorbed) || (d->n_cameras > 0 && !on_device(pr->source)))
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: source and absorbed outputs must be device memory", me);
    if (d->n_sources < 1 || d->n_sources > kMaxSources || !d->sources)
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: need 1..%d sources", me, kMaxSources);
    if (d->n_cameras < 0 || d->n_cameras > kMaxCams || (d->n_cameras > 0 && !d->cameras))
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: need 0..%d cameras", me, kMaxCams);
    if (d->precision != MCRT_FP32 && d->precision != MCRT_FP64)
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: bad precision", me);
    if (d->roulette_threshold < 0.0 ||
        (d->roulette_threshold > 0.0 && !(d->roulette_survival > 0.0 && d->roulette_survival <= 1.0)))
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: bad roulette parameters", me);
    if (d->n_trace < 0 || (d->n_trace > 0 && !on_device(d->trace)))
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: the trace buffer must be device memory", me);
    if (d->optics != MCRT_OPTICS_TABLES) return mcrt_fail_noctx(MCRT_E_INVAL, "%s: tables only", me);

    cudaStream_t s = (cudaStream_t)pr->cuda_stream;
    unsigned char* base = nullptr;
    NA_CK(scratch_address(&base));

    // extinction rows on the host (stack buffer) for the checks and table flags
    float hk[kMaxTheta * 3];
    NA_CK(cudaMemcpyAsync(hk, pr->kext, (size_t)pr->n_ktheta * 3 * sizeof(float), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    bool k_const = true;
    for (int j = 0; j < pr->n_ktheta; ++j) {
        if (!(hk[3 * j] > 0.f) || !(std::fabs(hk[3 * j + 1]) <= hk[3 * j]) || !std::isfinite(hk[3 * j + 2]))
            return mcrt_fail_noctx(MCRT_E_INVAL, "%s: invalid kext row %d", me, j);
        for (int e = 0; e < 3; ++e)
            if (hk[3 * j + e] != hk[e]) k_const = false;
    }

    TransportParams P{};
    P.g.n[0] = pr->nx;
    P.g.n[1] = pr->ny;
    P.g.n[2] = pr->nz;
    for (int a = 0; a < 3; ++a) {
        P.g.lo[a] = pr->lo[a];
        P.g.hi[a] = pr->hi[a];
        P.g.d[a] = (pr->hi[a] - pr->lo[a]) / P.g.n[a];
        P.lo_f[a] = (float)P.g.lo[a];
        P.d_f[a] = (float)P.g.d[a];
    }
    P.g.ncell = ncell;
    P.g.cells = reinterpret_cast<const float4*>(base + kOffCells);
    unsigned char* work = base + kOffWork;

    // set-up kernels write the cell records and prepared tables into the scratch
    NA_CK(cudaMemsetAsync(work, 0, kWorkBytes, s));
    NA_CK(launch_setup_cells(pr->kappa_abs, pr->kappa_sca, pr->bfield, nullptr, ncell,
                             reinterpret_cast<float4*>(base + kOffCells), reinterpret_cast<unsigned*>(work + 152), s));
    NA_CK(launch_prepare_tables(pr->model, table ? pr->n_bins : 0, table ? pr->n_theta : 0, pr->n_ktheta, pr->mueller,
                                pr->bin_weight, pr->kext, reinterpret_cast<float4*>(base + kOffMix),
                                reinterpret_cast<float4*>(base + kOffBins), reinterpret_cast<double*>(base + kOffEnvCdf),
                                reinterpret_cast<float*>(base + kOffEnv), reinterpret_cast<double*>(base + kOffBinCdf),
                                reinterpret_cast<float4*>(base + kOffKext), reinterpret_cast<double*>(work + 144), s));
    unsigned bad = 0;
    NA_CK(cudaMemcpyAsync(&bad, work + 152, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (bad) return mcrt_fail_noctx(MCRT_E_INVAL, "%s: negative or non-finite values in the input grids", me);

    TablesDev& t = P.t;
    t.model = pr->model;
    t.n_bins = table ? pr->n_bins : 0;
    t.n_theta = table ? pr->n_theta : 0;
    t.n_ktheta = pr->n_ktheta;
    t.k_const = k_const ? 1 : 0;
    t.k_iso = (k_const && hk[1] == 0.f && hk[2] == 0.f) ? 1 : 0;
    t.mix = reinterpret_cast<const float4*>(base + kOffMix);
    t.bins = reinterpret_cast<const float4*>(base + kOffBins);
    t.env_cdf = reinterpret_cast<const double*>(base + kOffEnvCdf);
    t.env = reinterpret_cast<const float*>(base + kOffEnv);
    t.bin_cdf = reinterpret_cast<const double*>(base + kOffBinCdf);
    // the FP32 copies follow the FP64 tables (as k_prepare_tables writes them)
    t.env_cdf_f = reinterpret_cast<const float*>(t.env_cdf + (size_t)t.n_bins * (t.n_theta > 1 ? t.n_theta - 1 : 0));
    t.bin_cdf_f = reinterpret_cast<const float*>(t.bin_cdf + t.n_bins);
    t.kext = reinterpret_cast<const float4*>(base + kOffKext);
    t.alpha1_mean = 1.0;  // used by thermal sources only, which are not accepted here

    long long total = 0, start = 0;
    for (int i = 0; i < d->n_sources; ++i) {
        const mcrt_source& src = d->sources[i];
        if (src.type == MCRT_SRC_THERMAL)
            return mcrt_fail_noctx(MCRT_E_INVAL, "%s: thermal sources need per-cell emission scratch; use "
                                                 "mcrt_launch_packets", me);
        if (src.type != MCRT_SRC_POINT && src.type != MCRT_SRC_BEAM)
            return mcrt_fail_noctx(MCRT_E_INVAL, "%s: bad source type %d", me, src.type);
        if (src.n_packets < 0) return mcrt_fail_noctx(MCRT_E_INVAL, "%s: negative n_packets", me);
        if (src.type == MCRT_SRC_POINT)
            for (int a = 0; a < 3; ++a)
                if (!(src.pos[a] >= pr->lo[a] && src.pos[a] <= pr->hi[a]))
                    return mcrt_fail_noctx(MCRT_E_INVAL, "%s: point source outside the grid", me);
        if (src.type == MCRT_SRC_BEAM && src.beam_dir != 1 && src.beam_dir != -1)
            return mcrt_fail_noctx(MCRT_E_INVAL, "%s: beam_dir must be +1 or -1", me);
        SourceDev& o = P.src[i];
        o.type = src.type;
        o.beam_dir = src.beam_dir;
        o.start = start;
        o.count = src.n_packets;
        o.eps = src.n_packets > 0 ? src.luminosity / (double)src.n_packets : 0.0;
        for (int a = 0; a < 3; ++a) o.pos[a] = src.pos[a];
        start += src.n_packets;
        total += src.n_packets;
    }
    P.n_src = d->n_sources;
    for (int k = 0; k < d->n_cameras; ++k) {
        const mcrt_camera& cm = d->cameras[k];
        const double nn = std::sqrt(cm.dir[0] * cm.dir[0] + cm.dir[1] * cm.dir[1] + cm.dir[2] * cm.dir[2]);
        if (!(nn > 0.0)) return mcrt_fail_noctx(MCRT_E_INVAL, "%s: bad camera %d", me, k);
        for (int a = 0; a < 3; ++a) P.cam[k].dir[a] = cm.dir[a] / nn;
        basis(P.cam[k].dir, P.cam[k].th, P.cam[k].ph);
    }
    P.n_cam = d->n_cameras;
    const long long pb = d->pid_begin, pe = d->pid_end <= 0 ? total : d->pid_end;
    if (pb < 0 || pe > total || pb > pe) return mcrt_fail_noctx(MCRT_E_INVAL, "%s: bad packet id range", me);

    if (!d->accumulate) {
        if (d->n_cameras > 0)
            NA_CK(cudaMemsetAsync(pr->source, 0, (size_t)ncell * d->n_cameras * 4 * sizeof(double), s));
        NA_CK(cudaMemsetAsync(pr->absorbed, 0, (size_t)ncell * sizeof(double), s));
    }
    if (d->n_trace > 0) NA_CK(cudaMemsetAsync(d->trace, 0, (size_t)d->n_trace * 16 * sizeof(double), s));
    P.S = pr->source;
    P.absorbed = pr->absorbed;
    P.seed = d->seed;
    P.stream = d->stream;
    P.pid_begin = pb;
    P.pid_end = pe;
    P.roulette_thr = d->roulette_threshold;
    P.roulette_surv = d->roulette_survival > 0.0 ? d->roulette_survival : 1.0;
    P.max_events = d->max_events > 0 ? (d->max_events < 2147483647ll ? d->max_events : 2147483647ll) : 100000;
    P.max_trials = d->max_trials > 0 ? d->max_trials : 1000;
    P.time_budget_ns = d->time_budget_s > 0.0 ? d->time_budget_s * 1e9 : 0.0;
    P.counter = reinterpret_cast<unsigned long long*>(work);
    P.stats = reinterpret_cast<double*>(work + 8);
    P.status = reinterpret_cast<unsigned*>(work + 136);
    P.trace = d->n_trace > 0 ? d->trace : nullptr;
    P.n_trace = d->n_trace;

    const int block = d->block_size > 0 ? d->block_size : 128;
    if (block % 32 != 0 || block > 128)
        return mcrt_fail_noctx(MCRT_E_INVAL, "%s: block_size must be a multiple of 32, <= 128", me);
    int dev = 0, nsm = 0;
    NA_CK(cudaGetDevice(&dev));
    NA_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = transport_smem_bytes(P, d->precision, block);
    int bps = transport_max_blocks_per_sm(d->precision, P.t.model, false, block, smem);
    if (d->blocks_per_sm > 0 && d->blocks_per_sm < bps) bps = d->blocks_per_sm;
    const long long nwork = pe - pb;
    long long grid = (long long)nsm * bps;
    const long long need = (nwork + block - 1) / block;
    if (need < grid) grid = need > 0 ? need : 1;
    if (nwork > 0) NA_CK(launch_transport(P, d->precision, block, (int)grid, s));

    // the launch's status word is always read (event or trial cap, time budget), the
    // totals when out_stats is given
    double raw[16];
    unsigned status = 0;
    if (out_stats) NA_CK(cudaMemcpyAsync(raw, work + 8, sizeof raw, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&status, work + 136, sizeof status, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (out_stats) {
        std::memset(out_stats, 0, sizeof(*out_stats));
        const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(raw + 6);
        out_stats->emitted_energy = raw[0];
        out_stats->escaped_energy = raw[1];
        out_stats->absorbed_energy = raw[2];
        out_stats->roulette_lost = raw[3];
        out_stats->roulette_gain = raw[4];
        out_stats->cap_lost = raw[5];
        out_stats->events = (double)cnt[0];
        out_stats->segments = (double)cnt[1];
        out_stats->scatterings = (double)cnt[2];
        out_stats->emitted = (double)cnt[3];
        out_stats->escaped = (double)cnt[4];
        out_stats->roulette_killed = (double)cnt[5];
        out_stats->cap_hits = (double)cnt[6];
        out_stats->trials = (double)cnt[7];
        out_stats->tally_segments = (double)cnt[8];
        out_stats->absorb_segments = (double)cnt[9];
        out_stats->status_bits = (double)status;
    }
    if (status & MCRT_STATUS_TIMEOUT) return mcrt_fail_noctx(MCRT_E_TIMEOUT, "%s: time budget exhausted", me);
    if (status & (MCRT_STATUS_EVENT_CAP | MCRT_STATUS_TRIAL_CAP))
        return mcrt_fail_noctx(MCRT_E_EVENT_CAP, "%s: packets reached the event or trial cap", me);
    return MCRT_OK;
}
