// mcrt_api.cu -- host side of the C ABI declared in include/mcrt.h: argument
// validation, device residency of the model, launch set-up and error reporting.
// All arithmetic of the method runs in the kernels of mcrt_transport.cu and
// mcrt_image.cu; this file only moves data and fills launch parameters.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mcrt.h"
#include "mcrt_internal.h"

using namespace mcrt;

struct mcrt_ctx {
    GridDev g{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_sm = 0;
    float4* d_cells = nullptr;
    bool has_emissivity = false;
    // optics
    bool tables_set = false;
    TablesDev t{};
    float4 *d_mix = nullptr, *d_bins = nullptr, *d_kext = nullptr;
    double *d_env_cdf = nullptr, *d_bin_cdf = nullptr, *d_alpha1 = nullptr;
    float* d_env = nullptr;
    // thermal emission CDF
    double* d_cdf = nullptr;
    double* d_block_sums = nullptr;
    long long* d_guide = nullptr;
    long long n_guide = 0;
    bool cdf_valid = false;
    double thermal_total = 0.0;
    // tallies of the last launch
    int n_cam = 0;
    size_t S_elems = 0;
    double* d_S = nullptr;
    double* d_absorbed = nullptr;
    mcrt_camera cams[kMaxCams];
    bool launched = false;
    int precision = MCRT_FP32;  // arithmetic of the last launch, reused by its images
    // work area: counter (8 B), stats (16 x 8 B), status (8 B)
    unsigned char* d_work = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    char err[512] = {0};
};

namespace {

thread_local char g_err[512] = "";

mcrt_status fail(mcrt_ctx* ctx, mcrt_status st, const char* fmt, ...) {
    char* dst = ctx ? ctx->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return st;
}

#define CK(ctx, call)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return fail((ctx), MCRT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device copy of a caller buffer: the buffer itself if it is device memory, else
// a temporary allocation filled from host memory.
struct DevIn {
    const void* ptr = nullptr;
    void* owned = nullptr;
    ~DevIn() {
        if (owned) cudaFree(owned);
    }
};

cudaError_t stage(DevIn& d, const void* src, size_t bytes, cudaStream_t s) {
    if (!src) return cudaSuccess;
    if (is_device_ptr(src)) {
        d.ptr = src;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(&d.owned, bytes);
    if (e != cudaSuccess) return e;
    d.ptr = d.owned;
    return cudaMemcpyAsync(d.owned, src, bytes, cudaMemcpyHostToDevice, s);
}

// Stokes basis of a unit vector on the host (phi-hat = (-y, x, 0)/rho,
// theta-hat = phi-hat x n; phi-hat = y-hat at the poles).
void host_basis(const double n[3], double th[3], double ph[3]) {
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

void free_tables(mcrt_ctx* c) {
    cudaFree(c->d_mix);
    cudaFree(c->d_bins);
    cudaFree(c->d_kext);
    cudaFree(c->d_env_cdf);
    cudaFree(c->d_bin_cdf);
    cudaFree(c->d_alpha1);
    cudaFree(c->d_env);
    c->d_mix = c->d_bins = c->d_kext = nullptr;
    c->d_env_cdf = c->d_bin_cdf = c->d_alpha1 = nullptr;
    c->d_env = nullptr;
    c->tables_set = false;
}

constexpr size_t kWorkBytes = 8 + 16 * 8 + 8;

}  // namespace

mcrt_status mcrt_fail_noctx(mcrt_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

extern "C" {

const char* mcrt_last_error(const mcrt_ctx* ctx) { return ctx ? ctx->err : g_err; }

mcrt_status mcrt_create_grid(mcrt_ctx** out, int32_t nx, int32_t ny, int32_t nz, const double lo[3],
                             const double hi[3], const float* kappa_abs, const float* kappa_sca, const float* bfield,
                             const float* emissivity, int32_t boundary, void* cuda_stream) {
    if (!out) return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: bad shape %d %d %d", nx, ny, nz);
    const long long ncell = (long long)nx * ny * nz;
    if (ncell >= (1ll << 31)) return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: %lld cells exceed 2^31", ncell);
    if (!lo || !hi) return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: lo/hi is NULL");
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] > lo[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a]))
            return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: empty or non-finite box on axis %d", a);
    if (!kappa_abs || !kappa_sca) return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: kappa_abs/kappa_sca is NULL");
    if (boundary != MCRT_BOUNDARY_OUTFLOW)
        return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: only MCRT_BOUNDARY_OUTFLOW is supported");

    mcrt_ctx* c = new (std::nothrow) mcrt_ctx();
    if (!c) return fail(nullptr, MCRT_E_NOMEM, "mcrt_create_grid: host allocation failed");
    c->stream = (cudaStream_t)cuda_stream;
    c->g.n[0] = nx;
    c->g.n[1] = ny;
    c->g.n[2] = nz;
    for (int a = 0; a < 3; ++a) {
        c->g.lo[a] = lo[a];
        c->g.hi[a] = hi[a];
        c->g.d[a] = (hi[a] - lo[a]) / c->g.n[a];
    }
    c->g.ncell = ncell;
    c->has_emissivity = emissivity != nullptr;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cells, (size_t)ncell * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_work, kWorkBytes);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) {
        mcrt_status st = fail(nullptr, e == cudaErrorMemoryAllocation ? MCRT_E_NOMEM : MCRT_E_CUDA,
                              "mcrt_create_grid: %s", cudaGetErrorString(e));
        mcrt_destroy(c);
        return st;
    }
    c->g.cells = c->d_cells;
    unsigned bad = 0;
    {
        DevIn ka, ks, bf, em;
        const size_t fb = (size_t)ncell * sizeof(float);
        e = stage(ka, kappa_abs, fb, c->stream);
        if (e == cudaSuccess) e = stage(ks, kappa_sca, fb, c->stream);
        if (e == cudaSuccess) e = stage(bf, bfield, 3 * fb, c->stream);
        if (e == cudaSuccess) e = stage(em, emissivity, fb, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_work, 0, kWorkBytes, c->stream);
        if (e == cudaSuccess)
            e = launch_setup_cells((const float*)ka.ptr, (const float*)ks.ptr, (const float*)bf.ptr,
                                   (const float*)em.ptr, ncell, c->d_cells, (unsigned*)c->d_work, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, c->d_work, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e == cudaSuccess && bad) {
        mcrt_destroy(c);
        return fail(nullptr, MCRT_E_INVAL, "mcrt_create_grid: negative or non-finite values in the input grids");
    }
    if (e != cudaSuccess) {
        mcrt_status st = fail(nullptr, e == cudaErrorMemoryAllocation ? MCRT_E_NOMEM : MCRT_E_CUDA,
                              "mcrt_create_grid: %s", cudaGetErrorString(e));
        mcrt_destroy(c);
        return st;
    }
    *out = c;
    return MCRT_OK;
}

mcrt_status mcrt_set_dust_tables(mcrt_ctx* ctx, int32_t model, int32_t n_bins, int32_t n_theta, const float* mueller,
                                 const float* bin_weight, int32_t n_ktheta, const float* kext) {
    if (!ctx) return fail(nullptr, MCRT_E_INVAL, "mcrt_set_dust_tables: ctx is NULL");
    if (model != MCRT_SCAT_RAYLEIGH && model != MCRT_SCAT_TABLE)
        return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: unknown model %d", model);
    if (!kext || n_ktheta < 2 || n_ktheta > 721)
        return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: need 2 <= n_ktheta <= 721 and kext");
    if (model == MCRT_SCAT_TABLE) {
        if (!mueller || !bin_weight) return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: tables are NULL");
        if (n_bins < 1 || n_bins > 32 || n_theta < 2 || n_theta > 721)
            return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: need 1 <= n_bins <= 32, 2 <= n_theta <= 721");
    } else {
        n_bins = 0;
        n_theta = 0;
    }
    // host copies for the validity checks and the table flags
    std::vector<float> hk((size_t)n_ktheta * 3), hw((size_t)(n_bins > 0 ? n_bins : 1));
    CK(ctx, cudaMemcpy(hk.data(), kext, hk.size() * sizeof(float), cudaMemcpyDefault));
    if (model == MCRT_SCAT_TABLE) CK(ctx, cudaMemcpy(hw.data(), bin_weight, n_bins * sizeof(float), cudaMemcpyDefault));
    double wsum = 0.0;
    for (int k = 0; k < n_bins; ++k) {
        if (!(hw[k] >= 0.f)) return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: negative bin weight");
        wsum += hw[k];
    }
    if (model == MCRT_SCAT_TABLE && !(wsum > 0.0))
        return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: bin weights sum to zero");
    bool k_const = true;
    for (int j = 0; j < n_ktheta; ++j) {
        for (int e = 0; e < 3; ++e)
            if (!std::isfinite(hk[3 * j + e])) return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: non-finite kext");
        if (!(hk[3 * j] > 0.f)) return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: alpha1 must be > 0");
        if (std::fabs(hk[3 * j + 1]) > hk[3 * j])
            return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_tables: |alpha2| > alpha1 at row %d", j);
        for (int e = 0; e < 3; ++e)
            if (hk[3 * j + e] != hk[e]) k_const = false;
    }
    const bool k_iso = k_const && hk[1] == 0.f && hk[2] == 0.f;

    free_tables(ctx);
    ctx->cdf_valid = false;
    const int nint = n_theta > 1 ? n_theta - 1 : 1;
    const int nb = n_bins > 0 ? n_bins : 1;
    const int nt = n_theta > 0 ? n_theta : 1;
    cudaError_t e = cudaMalloc(&ctx->d_kext, n_ktheta * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_alpha1, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_mix, (size_t)nt * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_bins, (size_t)nb * nt * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_env_cdf, (size_t)nb * nint * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_env, (size_t)nb * nint * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_bin_cdf, (size_t)nb * sizeof(double));
    if (e != cudaSuccess) {
        free_tables(ctx);
        return fail(ctx, MCRT_E_NOMEM, "mcrt_set_dust_tables: %s", cudaGetErrorString(e));
    }
    double a1m = 0.0;
    {
        DevIn dm, dw, dk;
        e = stage(dk, kext, (size_t)n_ktheta * 3 * sizeof(float), ctx->stream);
        if (e == cudaSuccess && model == MCRT_SCAT_TABLE)
            e = stage(dm, mueller, (size_t)n_bins * n_theta * 6 * sizeof(float), ctx->stream);
        if (e == cudaSuccess && model == MCRT_SCAT_TABLE) e = stage(dw, bin_weight, (size_t)n_bins * sizeof(float), ctx->stream);
        if (e == cudaSuccess)
            e = launch_prepare_tables(model, n_bins, n_theta, n_ktheta, (const float*)dm.ptr, (const float*)dw.ptr,
                                      (const float*)dk.ptr, ctx->d_mix, ctx->d_bins, ctx->d_env_cdf, ctx->d_env,
                                      ctx->d_bin_cdf, ctx->d_kext, ctx->d_alpha1, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&a1m, ctx->d_alpha1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (e != cudaSuccess) {
        free_tables(ctx);
        return fail(ctx, MCRT_E_CUDA, "mcrt_set_dust_tables: %s", cudaGetErrorString(e));
    }
    TablesDev& t = ctx->t;
    t.model = model;
    t.n_bins = n_bins;
    t.n_theta = n_theta;
    t.n_ktheta = n_ktheta;
    t.k_iso = k_iso ? 1 : 0;
    t.k_const = k_const ? 1 : 0;
    t.mix = ctx->d_mix;
    t.bins = ctx->d_bins;
    t.env_cdf = ctx->d_env_cdf;
    t.env = ctx->d_env;
    t.bin_cdf = ctx->d_bin_cdf;
    t.kext = ctx->d_kext;
    t.alpha1_mean = a1m;
    ctx->tables_set = true;
    return MCRT_OK;
}

static mcrt_status launch_one(mcrt_ctx* ctx, const mcrt_launch_desc* d, uint32_t stream_key, mcrt_stats* st_out,
                              bool want_sync) {
    if (!ctx->tables_set) return fail(ctx, MCRT_E_STATE, "mcrt_launch_packets: mcrt_set_dust_tables not called");
    if (d->n_sources < 1 || d->n_sources > kMaxSources || !d->sources)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: need 1..%d sources", kMaxSources);
    if (d->n_cameras < 0 || d->n_cameras > kMaxCams || (d->n_cameras > 0 && !d->cameras))
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: need 0..%d cameras", kMaxCams);
    if (d->precision != MCRT_FP32 && d->precision != MCRT_FP64)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad precision %d", d->precision);
    if (d->roulette_threshold < 0.0 || (d->roulette_threshold > 0.0 && !(d->roulette_survival > 0.0 && d->roulette_survival <= 1.0)))
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad roulette parameters");
    if (d->n_trace < 0 || (d->n_trace > 0 && !d->trace)) return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad trace");

    TransportParams P{};
    P.g = ctx->g;
    P.t = ctx->t;
    long long total = 0;
    bool need_thermal = false;
    for (int s = 0; s < d->n_sources; ++s) {
        const mcrt_source& src = d->sources[s];
        if (src.type < MCRT_SRC_POINT || src.type > MCRT_SRC_THERMAL)
            return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad source type %d", src.type);
        if (src.n_packets < 0) return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: negative n_packets");
        if (src.type == MCRT_SRC_POINT)
            for (int a = 0; a < 3; ++a)
                if (!(src.pos[a] >= ctx->g.lo[a] && src.pos[a] <= ctx->g.hi[a]))
                    return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: point source outside the grid");
        if (src.type == MCRT_SRC_BEAM && src.beam_dir != 1 && src.beam_dir != -1)
            return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: beam_dir must be +1 or -1");
        if (src.type == MCRT_SRC_THERMAL) need_thermal = true;
        total += src.n_packets;
    }
    if (need_thermal && !ctx->has_emissivity)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: thermal source needs an emissivity grid");
    if (need_thermal && !ctx->cdf_valid) {
        const int nb = thermal_cdf_blocks(ctx->g.ncell);
        if (!ctx->d_cdf) CK(ctx, cudaMalloc(&ctx->d_cdf, (size_t)ctx->g.ncell * sizeof(double)));
        if (!ctx->d_block_sums) CK(ctx, cudaMalloc(&ctx->d_block_sums, (size_t)nb * sizeof(double)));
        CK(ctx, launch_thermal_cdf(ctx->g, ctx->t.alpha1_mean, ctx->d_cdf, ctx->d_block_sums, nb, ctx->stream));
        ctx->n_guide = ctx->g.ncell < (1ll << 22) ? ctx->g.ncell : (1ll << 22);
        if (!ctx->d_guide) CK(ctx, cudaMalloc(&ctx->d_guide, (size_t)(ctx->n_guide + 1) * sizeof(long long)));
        CK(ctx, launch_thermal_guide(ctx->d_cdf, ctx->g.ncell, ctx->d_guide, ctx->n_guide, ctx->stream));
        CK(ctx, cudaMemcpyAsync(&ctx->thermal_total, ctx->d_cdf + (ctx->g.ncell - 1), sizeof(double),
                                cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->cdf_valid = true;
    }
    if (need_thermal && !(ctx->thermal_total > 0.0))
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: thermal source but the grid emits nothing");
    long long start = 0;
    for (int s = 0; s < d->n_sources; ++s) {
        const mcrt_source& src = d->sources[s];
        SourceDev& o = P.src[s];
        o.type = src.type;
        o.beam_dir = src.beam_dir;
        o.start = start;
        o.count = src.n_packets;
        double L = src.luminosity;
        if (src.type == MCRT_SRC_THERMAL && L <= 0.0) L = 4.0 * 3.141592653589793 * ctx->thermal_total;
        o.eps = src.n_packets > 0 ? L / (double)src.n_packets : 0.0;
        for (int a = 0; a < 3; ++a) o.pos[a] = src.pos[a];
        start += src.n_packets;
    }
    P.n_src = d->n_sources;
    for (int k = 0; k < d->n_cameras; ++k) {
        const mcrt_camera& cm = d->cameras[k];
        const double nn = std::sqrt(cm.dir[0] * cm.dir[0] + cm.dir[1] * cm.dir[1] + cm.dir[2] * cm.dir[2]);
        if (!(nn > 0.0) || cm.npix[0] < 1 || cm.npix[1] < 1 || !(cm.fov[0] > 0.0) || !(cm.fov[1] > 0.0))
            return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad camera %d", k);
        CameraDev& cd = P.cam[k];
        for (int a = 0; a < 3; ++a) cd.dir[a] = cm.dir[a] / nn;
        host_basis(cd.dir, cd.th, cd.ph);
    }
    P.n_cam = d->n_cameras;
    P.thermal_cdf = ctx->d_cdf;
    P.thermal_total = ctx->thermal_total;
    P.thermal_guide = ctx->d_guide;
    P.n_guide = ctx->n_guide;
    for (int a = 0; a < 3; ++a) {
        P.lo_f[a] = (float)ctx->g.lo[a];
        P.d_f[a] = (float)ctx->g.d[a];
    }

    long long pb = d->pid_begin, pe = d->pid_end <= 0 ? total : d->pid_end;
    if (pb < 0 || pe > total || pb > pe) return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad packet id range");

    // tallies
    const size_t S_elems = (size_t)ctx->g.ncell * (size_t)(d->n_cameras > 0 ? d->n_cameras : 1) * 4;
    if (d->accumulate && (!ctx->launched || ctx->n_cam != d->n_cameras))
        return fail(ctx, MCRT_E_STATE, "mcrt_launch_packets: accumulate needs a previous launch with the same cameras");
    if (ctx->S_elems != S_elems) {
        cudaFree(ctx->d_S);
        ctx->d_S = nullptr;
        ctx->S_elems = 0;
        cudaError_t e = cudaMalloc(&ctx->d_S, S_elems * sizeof(double));
        if (e != cudaSuccess) return fail(ctx, MCRT_E_NOMEM, "mcrt_launch_packets: source tally: %s", cudaGetErrorString(e));
        ctx->S_elems = S_elems;
    }
    if (!ctx->d_absorbed) CK(ctx, cudaMalloc(&ctx->d_absorbed, (size_t)ctx->g.ncell * sizeof(double)));
    if (!d->accumulate) {
        CK(ctx, cudaMemsetAsync(ctx->d_S, 0, S_elems * sizeof(double), ctx->stream));
        CK(ctx, cudaMemsetAsync(ctx->d_absorbed, 0, (size_t)ctx->g.ncell * sizeof(double), ctx->stream));
    }
    ctx->n_cam = d->n_cameras;
    ctx->precision = d->precision;
    for (int k = 0; k < d->n_cameras; ++k) ctx->cams[k] = d->cameras[k];

    P.S = ctx->d_S;
    P.absorbed = ctx->d_absorbed;
    P.seed = d->seed;
    P.stream = stream_key;
    P.pid_begin = pb;
    P.pid_end = pe;
    P.roulette_thr = d->roulette_threshold;
    P.roulette_surv = d->roulette_survival > 0.0 ? d->roulette_survival : 1.0;
    P.max_events = d->max_events > 0 ? (d->max_events < 2147483647ll ? d->max_events : 2147483647ll) : 100000;
    P.max_trials = d->max_trials > 0 ? d->max_trials : 1000;
    P.time_budget_ns = d->time_budget_s > 0.0 ? d->time_budget_s * 1e9 : 0.0;
    P.counter = reinterpret_cast<unsigned long long*>(ctx->d_work);
    P.stats = reinterpret_cast<double*>(ctx->d_work + 8);
    P.status = reinterpret_cast<unsigned*>(ctx->d_work + 8 + 16 * 8);
    CK(ctx, cudaMemsetAsync(ctx->d_work, 0, kWorkBytes, ctx->stream));

    // trace buffer
    DevIn trace_dev;
    double* trace_host = nullptr;
    if (d->n_trace > 0) {
        const size_t tb = (size_t)d->n_trace * 16 * sizeof(double);
        if (is_device_ptr(d->trace)) {
            P.trace = d->trace;
            CK(ctx, cudaMemsetAsync(d->trace, 0, tb, ctx->stream));
        } else {
            CK(ctx, cudaMalloc(&trace_dev.owned, tb));
            CK(ctx, cudaMemsetAsync(trace_dev.owned, 0, tb, ctx->stream));
            P.trace = (double*)trace_dev.owned;
            trace_host = d->trace;
        }
        P.n_trace = d->n_trace;
    }

    const int block = d->block_size > 0 ? d->block_size : 128;
    if (block % 32 != 0 || block > 128)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: block_size must be a multiple of 32, <= 128");
    const size_t smem = transport_smem_bytes(P, d->precision, block);
    int bps = transport_max_blocks_per_sm(d->precision, P.t.model, block, smem);
    if (d->blocks_per_sm > 0 && d->blocks_per_sm < bps) bps = d->blocks_per_sm;
    const long long work = pe - pb;
    long long grid = (long long)ctx->n_sm * bps;
    const long long need = (work + block - 1) / block;
    if (need < grid) grid = need > 0 ? need : 1;

    CK(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
    if (work > 0) CK(ctx, launch_transport(P, d->precision, block, (int)grid, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    ctx->launched = true;

    if (trace_host)
        CK(ctx, cudaMemcpyAsync(trace_host, P.trace, (size_t)d->n_trace * 16 * sizeof(double), cudaMemcpyDeviceToHost,
                                ctx->stream));
    if (!(want_sync || trace_host)) return MCRT_OK;
    double raw[16];
    unsigned status = 0;
    CK(ctx, cudaMemcpyAsync(raw, ctx->d_work + 8, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(&status, ctx->d_work + 8 + 16 * 8, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    CK(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    if (st_out) {
        const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(raw + 6);
        st_out->emitted_energy += raw[0];
        st_out->escaped_energy += raw[1];
        st_out->absorbed_energy += raw[2];
        st_out->roulette_lost += raw[3];
        st_out->roulette_gain += raw[4];
        st_out->cap_lost += raw[5];
        st_out->events += (double)cnt[0];
        st_out->segments += (double)cnt[1];
        st_out->scatterings += (double)cnt[2];
        st_out->emitted += (double)cnt[3];
        st_out->escaped += (double)cnt[4];
        st_out->roulette_killed += (double)cnt[5];
        st_out->cap_hits += (double)cnt[6];
        st_out->trials += (double)cnt[7];
        st_out->tally_segments += (double)cnt[8];
        st_out->absorb_segments += (double)cnt[9];
        st_out->kernel_ms += ms;
        st_out->status_bits = (double)((unsigned)st_out->status_bits | status);
    }
    if (status & MCRT_STATUS_TIMEOUT) return fail(ctx, MCRT_E_TIMEOUT, "mcrt_launch_packets: time budget exhausted");
    if (status & (MCRT_STATUS_EVENT_CAP | MCRT_STATUS_TRIAL_CAP))
        return fail(ctx, MCRT_E_EVENT_CAP, "mcrt_launch_packets: packets reached the event or trial cap");
    return MCRT_OK;
}

mcrt_status mcrt_launch_packets(mcrt_ctx* const* models, int32_t n_models, const mcrt_launch_desc* desc,
                                mcrt_stats* out_stats) {
    if (!models || n_models < 1 || !desc) return fail(nullptr, MCRT_E_INVAL, "mcrt_launch_packets: no models or desc");
    for (int m = 0; m < n_models; ++m)
        if (!models[m]) return fail(nullptr, MCRT_E_INVAL, "mcrt_launch_packets: model %d is NULL", m);
    if (out_stats) std::memset(out_stats, 0, sizeof(*out_stats));
    mcrt_status worst = MCRT_OK;
    for (int m = 0; m < n_models; ++m) {
        mcrt_status s = launch_one(models[m], desc, desc->stream + (uint32_t)m, out_stats, out_stats != nullptr);
        if (s == MCRT_E_EVENT_CAP || s == MCRT_E_TIMEOUT) {
            worst = s;
            continue;
        }
        if (s != MCRT_OK) {
            std::snprintf(g_err, sizeof g_err, "model %d: %s", m, models[m]->err);
            return s;
        }
    }
    return worst;
}

mcrt_status mcrt_image_stokes(mcrt_ctx* ctx, int32_t camera, double* out) {
    if (!ctx) return fail(nullptr, MCRT_E_INVAL, "mcrt_image_stokes: ctx is NULL");
    if (!ctx->launched) return fail(ctx, MCRT_E_STATE, "mcrt_image_stokes: no launch yet");
    if (camera < 0 || camera >= ctx->n_cam) return fail(ctx, MCRT_E_INVAL, "mcrt_image_stokes: camera %d out of range", camera);
    if (!out) return fail(ctx, MCRT_E_INVAL, "mcrt_image_stokes: out is NULL");
    const mcrt_camera& cm = ctx->cams[camera];
    ImageParams p{};
    p.g = ctx->g;
    p.t = ctx->t;
    const double nn = std::sqrt(cm.dir[0] * cm.dir[0] + cm.dir[1] * cm.dir[1] + cm.dir[2] * cm.dir[2]);
    for (int a = 0; a < 3; ++a) p.cam.dir[a] = cm.dir[a] / nn;
    host_basis(p.cam.dir, p.cam.th, p.cam.ph);
    for (int a = 0; a < 3; ++a) p.center[a] = cm.center[a];
    p.fov[0] = cm.fov[0];
    p.fov[1] = cm.fov[1];
    p.npix[0] = cm.npix[0];
    p.npix[1] = cm.npix[1];
    p.cam_index = camera;
    p.n_cam = ctx->n_cam;
    p.S = ctx->d_S;
    const size_t bytes = (size_t)4 * cm.npix[0] * cm.npix[1] * sizeof(double);
    DevIn tmp;
    const bool dev = is_device_ptr(out);
    if (dev) {
        p.out = out;
    } else {
        CK(ctx, cudaMalloc(&tmp.owned, bytes));
        p.out = (double*)tmp.owned;
    }
    CK(ctx, launch_image(p, ctx->precision, ctx->stream));
    if (!dev) {
        CK(ctx, cudaMemcpyAsync(out, p.out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return MCRT_OK;
}

mcrt_status mcrt_get_tallies(mcrt_ctx* ctx, double* source, double* absorbed) {
    if (!ctx) return fail(nullptr, MCRT_E_INVAL, "mcrt_get_tallies: ctx is NULL");
    if (!ctx->launched) return fail(ctx, MCRT_E_STATE, "mcrt_get_tallies: no launch yet");
    if (source && ctx->n_cam > 0)
        CK(ctx, cudaMemcpyAsync(source, ctx->d_S, (size_t)ctx->g.ncell * ctx->n_cam * 4 * sizeof(double),
                                cudaMemcpyDefault, ctx->stream));
    if (absorbed)
        CK(ctx, cudaMemcpyAsync(absorbed, ctx->d_absorbed, (size_t)ctx->g.ncell * sizeof(double), cudaMemcpyDefault,
                                ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

mcrt_status mcrt_destroy(mcrt_ctx* ctx) {
    if (!ctx) return MCRT_OK;
    free_tables(ctx);
    cudaFree(ctx->d_cells);
    cudaFree(ctx->d_cdf);
    cudaFree(ctx->d_block_sums);
    cudaFree(ctx->d_guide);
    cudaFree(ctx->d_S);
    cudaFree(ctx->d_absorbed);
    cudaFree(ctx->d_work);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return MCRT_OK;
}

mcrt_status mcrt_unit_eval(int32_t fn, int32_t precision, int64_t n, const double* in, double* out) {
    static const int in_w[6] = {6, 7, 10, 12, 8, 16};
    static const int out_w[6] = {4, 8, 6, 4, 4, 4};
    if (fn < 0 || fn > 5) return fail(nullptr, MCRT_E_INVAL, "mcrt_unit_eval: unknown fn %d", fn);
    if (precision != MCRT_FP32 && precision != MCRT_FP64) return fail(nullptr, MCRT_E_INVAL, "mcrt_unit_eval: precision");
    if (n < 0 || (n > 0 && (!in || !out))) return fail(nullptr, MCRT_E_INVAL, "mcrt_unit_eval: bad buffers");
    if (n == 0) return MCRT_OK;
    DevIn din, dout;
    const size_t ib = (size_t)n * in_w[fn] * sizeof(double), ob = (size_t)n * out_w[fn] * sizeof(double);
    CK(nullptr, cudaMalloc(&din.owned, ib));
    CK(nullptr, cudaMalloc(&dout.owned, ob));
    CK(nullptr, cudaMemcpy(din.owned, in, ib, cudaMemcpyDefault));
    CK(nullptr, launch_unit_eval(fn, precision, n, (const double*)din.owned, (double*)dout.owned, nullptr));
    CK(nullptr, cudaMemcpy(out, dout.owned, ob, cudaMemcpyDefault));
    return MCRT_OK;
}

}  // extern "C"
