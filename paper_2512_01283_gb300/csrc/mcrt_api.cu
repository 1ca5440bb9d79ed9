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
#include "mcrt_mlp_infer.cuh"
#include "mcrt_mlp_tc.cuh"

using namespace mcrt;

struct mcrt_ctx {
    GridDev g{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_sm = 0;
    float4* d_cells = nullptr;
    PatchDev* d_patches = nullptr;  // static mesh refinement
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
    // attached surrogate: network image, error map, distilled extinction table
    bool sur_set = false;
    unsigned char* d_sur_image = nullptr;
    unsigned char* d_sur_image_tc = nullptr;
    float* d_sur_map = nullptr;
    float4* d_sur_kext = nullptr;
    float sur_bound = 0.05f;
    int sur_kext_fixed = 0;
    int last_optics = MCRT_OPTICS_TABLES;
    // surrogate launches: control block, tally records, waiting packets
    WaveCtl* d_wave = nullptr;
    cudaStream_t tally_stream = nullptr;  // table rounds: tally kernels beside the next transport
    float4* d_records = nullptr;
    unsigned long long rec_cap = 0;
    size_t rec_bytes = 0;  // size of the tally-record queue allocation
    float4 *d_susp = nullptr, *d_res = nullptr;
    unsigned long long wave_cap = 0;
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

#define CK(ctx, call)                                                                             \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            (void)cudaGetLastError();                                                             \
            return fail((ctx), MCRT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));             \
        }                                                                                         \
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

void free_surrogate(mcrt_ctx* c) {
    cudaFree(c->d_sur_image);
    cudaFree(c->d_sur_image_tc);
    cudaFree(c->d_sur_map);
    cudaFree(c->d_sur_kext);
    c->d_sur_image = nullptr;
    c->d_sur_image_tc = nullptr;
    c->d_sur_map = nullptr;
    c->d_sur_kext = nullptr;
    c->sur_set = false;
}

void free_wave(mcrt_ctx* c) {
    cudaFree(c->d_wave);
    cudaFree(c->d_records);
    cudaFree(c->d_susp);
    cudaFree(c->d_res);
    c->d_wave = nullptr;
    c->d_records = nullptr;
    c->d_susp = c->d_res = nullptr;
    c->rec_cap = c->wave_cap = 0;
    c->rec_bytes = 0;
}

void free_tables(mcrt_ctx* c) {
    free_surrogate(c);  // the network was attached for these tables
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

mcrt_status mcrt_ctx_tables(const mcrt_ctx* ctx, TablesDev* out) {
    if (!ctx || !ctx->tables_set || !out) return MCRT_E_STATE;
    *out = ctx->t;
    return MCRT_OK;
}

mcrt_status mcrt_fail_noctx(mcrt_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

extern "C" {

const char* mcrt_last_error(const mcrt_ctx* ctx) { return ctx ? ctx->err : g_err; }

// Grid creation with an optional list of refined patches (validated here).
static mcrt_status create_grid(const char* me, mcrt_ctx** out, int32_t nx, int32_t ny, int32_t nz, const double lo[3],
                               const double hi[3], const float* kappa_abs, const float* kappa_sca, const float* bfield,
                               const float* emissivity, int32_t boundary, int32_t n_patches,
                               const mcrt_patch* patches, void* cuda_stream) {
    if (!out) return fail(nullptr, MCRT_E_INVAL, "%s: out is NULL", me);
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, MCRT_E_INVAL, "%s: bad shape %d %d %d", me, nx, ny, nz);
    const long long nroot = (long long)nx * ny * nz;
    if (!lo || !hi) return fail(nullptr, MCRT_E_INVAL, "%s: lo/hi is NULL", me);
    for (int a = 0; a < 3; ++a)
        if (!(hi[a] > lo[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a]))
            return fail(nullptr, MCRT_E_INVAL, "%s: empty or non-finite box on axis %d", me, a);
    if (!kappa_abs || !kappa_sca) return fail(nullptr, MCRT_E_INVAL, "%s: kappa_abs/kappa_sca is NULL", me);
    if (boundary < 0 || boundary > (MCRT_BOUNDARY_PERIODIC_X | MCRT_BOUNDARY_PERIODIC_Y | MCRT_BOUNDARY_PERIODIC_Z))
        return fail(nullptr, MCRT_E_INVAL, "%s: boundary must be an MCRT_BOUNDARY_* mask", me);
    if (n_patches < 0 || n_patches > kMaxPatches || (n_patches > 0 && !patches))
        return fail(nullptr, MCRT_E_INVAL, "%s: need 0..%d patches", me, kMaxPatches);
    const int root_n[3] = {nx, ny, nz};
    std::vector<PatchDev> hp((size_t)n_patches);
    long long ncell = nroot;
    for (int q = 0; q < n_patches; ++q) {
        const mcrt_patch& Q = patches[q];
        if (Q.factor < 2 || Q.factor > 16) return fail(nullptr, MCRT_E_INVAL, "%s: patch %d: factor must be 2..16", me, q);
        if (!Q.kappa_abs || !Q.kappa_sca) return fail(nullptr, MCRT_E_INVAL, "%s: patch %d: kappa arrays are NULL", me, q);
        if ((Q.bfield != nullptr) != (bfield != nullptr) || (Q.emissivity != nullptr) != (emissivity != nullptr))
            return fail(nullptr, MCRT_E_INVAL, "%s: patch %d: field and emission arrays must match the root's", me, q);
        PatchDev& P = hp[q];
        for (int a = 0; a < 3; ++a) {
            if (Q.box[a] < 0 || Q.box[3 + a] > root_n[a] || Q.box[3 + a] <= Q.box[a])
                return fail(nullptr, MCRT_E_INVAL, "%s: patch %d: box outside the root grid or empty", me, q);
            P.box[a] = Q.box[a];
            P.box[3 + a] = Q.box[3 + a];
            P.n[a] = (Q.box[3 + a] - Q.box[a]) * Q.factor;
            const double dr = (hi[a] - lo[a]) / root_n[a];
            P.lo[a] = lo[a] + Q.box[a] * dr;
            P.d[a] = dr / Q.factor;
            P.lo_f[a] = (float)P.lo[a];
            P.d_f[a] = (float)P.d[a];
        }
        P.factor = Q.factor;
        P.offset = ncell;
        ncell += (long long)P.n[0] * P.n[1] * P.n[2];
        for (int k = 0; k < q; ++k) {
            bool overlap = true;
            for (int a = 0; a < 3; ++a)
                overlap = overlap && hp[k].box[a] < P.box[3 + a] && P.box[a] < hp[k].box[3 + a];
            if (overlap) return fail(nullptr, MCRT_E_INVAL, "%s: patches %d and %d overlap", me, k, q);
        }
    }
    if (ncell >= (1ll << 31)) return fail(nullptr, MCRT_E_INVAL, "%s: %lld cells exceed 2^31", me, ncell);

    mcrt_ctx* c = new (std::nothrow) mcrt_ctx();
    if (!c) return fail(nullptr, MCRT_E_NOMEM, "%s: host allocation failed", me);
    c->stream = (cudaStream_t)cuda_stream;
    for (int a = 0; a < 3; ++a) {
        c->g.n[a] = root_n[a];
        c->g.lo[a] = lo[a];
        c->g.hi[a] = hi[a];
        c->g.d[a] = (hi[a] - lo[a]) / c->g.n[a];
    }
    c->g.ncell = ncell;
    c->g.ncell_root = nroot;
    c->g.periodic = boundary;
    c->has_emissivity = emissivity != nullptr;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cells, (size_t)ncell * 2 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_work, kWorkBytes);
    if (e == cudaSuccess && n_patches > 0) e = cudaMalloc(&c->d_patches, hp.size() * sizeof(PatchDev));
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) {
        mcrt_status st = fail(nullptr, e == cudaErrorMemoryAllocation ? MCRT_E_NOMEM : MCRT_E_CUDA, "%s: %s", me,
                              cudaGetErrorString(e));
        mcrt_destroy(c);
        return st;
    }
    c->g.cells = c->d_cells;
    c->g.n_patches = n_patches;
    c->g.patches = c->d_patches;
    unsigned bad = 0;
    e = cudaMemsetAsync(c->d_work, 0, kWorkBytes, c->stream);
    // cell records of one level: its arrays staged on the device, then k_setup_cells
    auto level = [&](const float* ka_in, const float* ks_in, const float* bf_in, const float* em_in, long long count,
                     float4* dst) {
        DevIn ka, ks, bf, em;
        const size_t fb = (size_t)count * sizeof(float);
        cudaError_t r = stage(ka, ka_in, fb, c->stream);
        if (r == cudaSuccess) r = stage(ks, ks_in, fb, c->stream);
        if (r == cudaSuccess) r = stage(bf, bf_in, 3 * fb, c->stream);
        if (r == cudaSuccess) r = stage(em, em_in, fb, c->stream);
        if (r == cudaSuccess)
            r = launch_setup_cells((const float*)ka.ptr, (const float*)ks.ptr, (const float*)bf.ptr,
                                   (const float*)em.ptr, count, dst, (unsigned*)c->d_work, c->stream);
        // the staged copies are freed when this returns: finish the kernel first
        if (r == cudaSuccess) r = cudaStreamSynchronize(c->stream);
        return r;
    };
    if (e == cudaSuccess) e = level(kappa_abs, kappa_sca, bfield, emissivity, nroot, c->d_cells);
    for (int q = 0; q < n_patches && e == cudaSuccess; ++q) {
        const mcrt_patch& Q = patches[q];
        const long long cnt = (long long)hp[q].n[0] * hp[q].n[1] * hp[q].n[2];
        e = level(Q.kappa_abs, Q.kappa_sca, Q.bfield, Q.emissivity, cnt, c->d_cells + 2 * hp[q].offset);
    }
    if (e == cudaSuccess && n_patches > 0)
        e = cudaMemcpyAsync(c->d_patches, hp.data(), hp.size() * sizeof(PatchDev), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && n_patches > 0) e = launch_mark_covered(c->g, hp.data(), c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, c->d_work, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && bad) {
        mcrt_destroy(c);
        return fail(nullptr, MCRT_E_INVAL, "%s: negative or non-finite values in the input grids", me);
    }
    if (e != cudaSuccess) {
        mcrt_status st = fail(nullptr, e == cudaErrorMemoryAllocation ? MCRT_E_NOMEM : MCRT_E_CUDA, "%s: %s", me,
                              cudaGetErrorString(e));
        mcrt_destroy(c);
        return st;
    }
    *out = c;
    return MCRT_OK;
}

mcrt_status mcrt_create_grid(mcrt_ctx** out, int32_t nx, int32_t ny, int32_t nz, const double lo[3],
                             const double hi[3], const float* kappa_abs, const float* kappa_sca, const float* bfield,
                             const float* emissivity, int32_t boundary, void* cuda_stream) {
    return create_grid("mcrt_create_grid", out, nx, ny, nz, lo, hi, kappa_abs, kappa_sca, bfield, emissivity, boundary,
                       0, nullptr, cuda_stream);
}

mcrt_status mcrt_create_grid_refined(mcrt_ctx** out, int32_t nx, int32_t ny, int32_t nz, const double lo[3],
                                     const double hi[3], const float* kappa_abs, const float* kappa_sca,
                                     const float* bfield, const float* emissivity, int32_t boundary,
                                     int32_t n_patches, const mcrt_patch* patches, void* cuda_stream) {
    return create_grid("mcrt_create_grid_refined", out, nx, ny, nz, lo, hi, kappa_abs, kappa_sca, bfield, emissivity,
                       boundary, n_patches, patches, cuda_stream);
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
    // cumulative tables: FP64, then their FP32 copies
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_env_cdf, (size_t)nb * nint * (sizeof(double) + sizeof(float)));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_env, (size_t)nb * nint * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_bin_cdf, (size_t)nb * (sizeof(double) + sizeof(float)));
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
    t.env_cdf_f = reinterpret_cast<const float*>(ctx->d_env_cdf + (size_t)nb * nint);
    t.bin_cdf_f = reinterpret_cast<const float*>(ctx->d_bin_cdf + nb);
    t.kext = ctx->d_kext;
    t.alpha1_mean = a1m;
    ctx->tables_set = true;
    return MCRT_OK;
}

static mcrt_status dipole_args(mcrt_ctx* ctx, const char* me, double eps_re, double eps_im, double aspect,
                               double x) {
    if (!std::isfinite(eps_re) || !std::isfinite(eps_im) || !std::isfinite(aspect) || !std::isfinite(x))
        return fail(ctx, MCRT_E_INVAL, "%s: non-finite parameter", me);
    if (eps_im < 0.0) return fail(ctx, MCRT_E_INVAL, "%s: eps_im < 0 (a gain medium)", me);
    if (eps_re == 1.0 && eps_im == 0.0) return fail(ctx, MCRT_E_INVAL, "%s: eps = 1 (no grain)", me);
    if (!(aspect > 0.0)) return fail(ctx, MCRT_E_INVAL, "%s: aspect must be > 0", me);
    if (x < 0.0) return fail(ctx, MCRT_E_INVAL, "%s: size_x must be >= 0", me);
    return MCRT_OK;
}

// The 20 constants of k_dipole_setup, on the host.
static cudaError_t dipole_setup_host(double eps_re, double eps_im, double aspect, double x, double out[20],
                                     cudaStream_t s) {
    DevIn d;
    cudaError_t e = cudaMalloc(&d.owned, 20 * sizeof(double));
    if (e == cudaSuccess) e = launch_dipole_setup(eps_re, eps_im, aspect, x, (double*)d.owned, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d.owned, 20 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

mcrt_status mcrt_set_dust_dipole(mcrt_ctx* ctx, double eps_re, double eps_im, double aspect, double size_x) {
    if (!ctx) return fail(nullptr, MCRT_E_INVAL, "mcrt_set_dust_dipole: ctx is NULL");
    const mcrt_status st = dipole_args(ctx, "mcrt_set_dust_dipole", eps_re, eps_im, aspect, size_x);
    if (st != MCRT_OK) return st;
    double c[20];
    CK(ctx, dipole_setup_host(eps_re, eps_im, aspect, size_x, c, ctx->stream));
    for (int k = 0; k < 20; ++k)
        if (!std::isfinite(c[k])) return fail(ctx, MCRT_E_INVAL, "mcrt_set_dust_dipole: singular polarizability");
    free_tables(ctx);
    ctx->cdf_valid = false;
    TablesDev t{};
    t.model = MCRT_SCAT_DIPOLE;
    t.alpha1_mean = 1.0;  // K is relative to its orientation average
    t.dip.rho_re = c[12];
    t.dip.rho_im = c[13];
    t.dip.zn = c[14];
    t.dip.env = c[15];
    t.dip.ca[0] = c[16];
    t.dip.ca[1] = c[17];
    t.dip.cs[0] = c[18];
    t.dip.cs[1] = c[19];
    t.dip.f_rho_re = (float)t.dip.rho_re;
    t.dip.f_rho_im = (float)t.dip.rho_im;
    t.dip.f_zn = (float)t.dip.zn;
    t.dip.f_env = (float)t.dip.env;
    for (int k = 0; k < 2; ++k) {
        t.dip.f_ca[k] = (float)t.dip.ca[k];
        t.dip.f_cs[k] = (float)t.dip.cs[k];
    }
    ctx->t = t;
    ctx->tables_set = true;
    return MCRT_OK;
}

mcrt_status mcrt_dipole_constants(double eps_re, double eps_im, double aspect, double size_x, double* out) {
    if (!out) return fail(nullptr, MCRT_E_INVAL, "mcrt_dipole_constants: out is NULL");
    const mcrt_status st = dipole_args(nullptr, "mcrt_dipole_constants", eps_re, eps_im, aspect, size_x);
    if (st != MCRT_OK) return st;
    double c[20];
    CK(nullptr, dipole_setup_host(eps_re, eps_im, aspect, size_x, c, nullptr));
    std::memcpy(out, c, 16 * sizeof(double));
    return MCRT_OK;
}

// Checks of a launch description that do not depend on the model.
static mcrt_status check_desc(mcrt_ctx* ctx, const mcrt_launch_desc* d) {
    if (d->n_sources < 1 || d->n_sources > kMaxSources || !d->sources)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: need 1..%d sources", kMaxSources);
    if (d->n_cameras < 0 || d->n_cameras > kMaxCams || (d->n_cameras > 0 && !d->cameras))
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: need 0..%d cameras", kMaxCams);
    if (d->precision != MCRT_FP32 && d->precision != MCRT_FP64)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad precision %d", d->precision);
    if (d->roulette_threshold < 0.0 || (d->roulette_threshold > 0.0 && !(d->roulette_survival > 0.0 && d->roulette_survival <= 1.0)))
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad roulette parameters");
    if (d->n_trace < 0 || (d->n_trace > 0 && !d->trace)) return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad trace");
    if (d->optics != MCRT_OPTICS_TABLES && d->optics != MCRT_OPTICS_SURROGATE)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad optics %d", d->optics);
    if (d->optics == MCRT_OPTICS_SURROGATE && (d->precision != MCRT_FP32 || d->time_budget_s > 0.0))
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: surrogate launches are FP32 without a time budget");
    for (int s = 0; s < d->n_sources; ++s) {
        const mcrt_source& src = d->sources[s];
        if (src.type < MCRT_SRC_POINT || src.type > MCRT_SRC_THERMAL)
            return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad source type %d", src.type);
        if (src.n_packets < 0) return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: negative n_packets");
        if (src.type == MCRT_SRC_BEAM && src.beam_dir != 1 && src.beam_dir != -1)
            return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: beam_dir must be +1 or -1");
    }
    for (int k = 0; k < d->n_cameras; ++k) {
        const mcrt_camera& cm = d->cameras[k];
        const double nn = std::sqrt(cm.dir[0] * cm.dir[0] + cm.dir[1] * cm.dir[1] + cm.dir[2] * cm.dir[2]);
        if (!(nn > 0.0) || cm.npix[0] < 1 || cm.npix[1] < 1 || !(cm.fov[0] > 0.0) || !(cm.fov[1] > 0.0))
            return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad camera %d", k);
    }
    return MCRT_OK;
}

static long long desc_total(const mcrt_launch_desc* d) {
    long long total = 0;
    for (int s = 0; s < d->n_sources; ++s) total += d->sources[s].n_packets;
    return total;
}

// Launch-wide parameters: sources (without energies), cameras, random-number key,
// roulette, caps.
static void fill_common(const mcrt_launch_desc* d, TransportParams& P) {
    long long start = 0;
    for (int s = 0; s < d->n_sources; ++s) {
        const mcrt_source& src = d->sources[s];
        SourceDev& o = P.src[s];
        o.type = src.type;
        o.beam_dir = src.beam_dir;
        o.start = start;
        o.count = src.n_packets;
        for (int a = 0; a < 3; ++a) o.pos[a] = src.pos[a];
        start += src.n_packets;
    }
    P.n_src = d->n_sources;
    for (int k = 0; k < d->n_cameras; ++k) {
        const mcrt_camera& cm = d->cameras[k];
        const double nn = std::sqrt(cm.dir[0] * cm.dir[0] + cm.dir[1] * cm.dir[1] + cm.dir[2] * cm.dir[2]);
        CameraDev& cd = P.cam[k];
        for (int a = 0; a < 3; ++a) cd.dir[a] = cm.dir[a] / nn;
        host_basis(cd.dir, cd.th, cd.ph);
    }
    P.n_cam = d->n_cameras;
    P.seed = d->seed;
    P.stream = d->stream;
    P.roulette_thr = d->roulette_threshold;
    P.roulette_surv = d->roulette_survival > 0.0 ? d->roulette_survival : 1.0;
    P.max_events = d->max_events > 0 ? (d->max_events < 2147483647ll ? d->max_events : 2147483647ll) : 100000;
    P.max_trials = d->max_trials > 0 ? d->max_trials : 1000;
    P.time_budget_ns = d->time_budget_s > 0.0 ? d->time_budget_s * 1e9 : 0.0;
}

// Model part of a launch: checks the description against the model, builds the
// thermal-emission CDF when a thermal source needs it, sizes the tallies and zeroes
// them unless accumulating, and fills the model's job record.
static mcrt_status prepare_model(mcrt_ctx* ctx, const mcrt_launch_desc* d, uint32_t stream_key, JobDev& job) {
    if (!ctx->tables_set) return fail(ctx, MCRT_E_STATE, "mcrt_launch_packets: mcrt_set_dust_tables not called");
    bool need_thermal = false;
    for (int s = 0; s < d->n_sources; ++s) {
        const mcrt_source& src = d->sources[s];
        if (src.type == MCRT_SRC_POINT)
            for (int a = 0; a < 3; ++a)
                if (!(src.pos[a] >= ctx->g.lo[a] && src.pos[a] <= ctx->g.hi[a]))
                    return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: point source outside the grid");
        if (src.type == MCRT_SRC_THERMAL) need_thermal = true;
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

    job = JobDev{};
    for (int a = 0; a < 3; ++a) {
        job.n[a] = ctx->g.n[a];
        job.periodic = ctx->g.periodic;
        job.lo[a] = ctx->g.lo[a];
        job.hi[a] = ctx->g.hi[a];
        job.d[a] = ctx->g.d[a];
        job.lo_f[a] = (float)ctx->g.lo[a];
        job.d_f[a] = (float)ctx->g.d[a];
    }
    job.ncell = ctx->g.ncell;
    job.cells = ctx->d_cells;
    job.S = ctx->d_S;
    job.absorbed = ctx->d_absorbed;
    job.t = ctx->t;
    job.thermal_cdf = ctx->d_cdf;
    job.thermal_total = ctx->thermal_total;
    job.thermal_guide = ctx->d_guide;
    job.n_guide = ctx->n_guide;
    for (int s = 0; s < d->n_sources; ++s) {
        const mcrt_source& src = d->sources[s];
        double L = src.luminosity;
        if (src.type == MCRT_SRC_THERMAL && L <= 0.0) L = 4.0 * 3.141592653589793 * ctx->thermal_total;
        job.src_eps[s] = src.n_packets > 0 ? L / (double)src.n_packets : 0.0;
    }
    job.stream = stream_key;
    return MCRT_OK;
}

static void add_wave_stats(mcrt_stats* st, const WaveCtl& w) {
    st->mlp_tally_rows += (double)w.cnt[kCntTallyRows];
    st->mlp_scatter_rows += (double)w.cnt[kCntScatRows];
    st->mlp_fallback_map += (double)w.cnt[kCntFallbackMap];
    st->mlp_fallback_realizability += (double)w.cnt[kCntFallbackReal];
    st->tally_overflow += (double)w.cnt[kCntOverflow];
    st->envelope_miss += (double)w.cnt[kCntEnvelopeMiss];
    st->wave_iterations += (double)w.cnt[kCntIterations];
}

static void add_stats(mcrt_stats* st, const double raw[16], unsigned status, float ms) {
    const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(raw + 6);
    st->emitted_energy += raw[0];
    st->escaped_energy += raw[1];
    st->absorbed_energy += raw[2];
    st->roulette_lost += raw[3];
    st->roulette_gain += raw[4];
    st->cap_lost += raw[5];
    st->events += (double)cnt[0];
    st->segments += (double)cnt[1];
    st->scatterings += (double)cnt[2];
    st->emitted += (double)cnt[3];
    st->escaped += (double)cnt[4];
    st->roulette_killed += (double)cnt[5];
    st->cap_hits += (double)cnt[6];
    st->trials += (double)cnt[7];
    st->tally_segments += (double)cnt[8];
    st->absorb_segments += (double)cnt[9];
    st->kernel_ms += ms;
    st->status_bits = (double)((unsigned)st->status_bits | status);
}

static mcrt_status status_of(mcrt_ctx* ctx, unsigned status) {
    if (status & MCRT_STATUS_DEVICE_TIMEOUT)
        return fail(ctx, MCRT_E_TIMEOUT, "mcrt_launch_packets: a tensor-core wait timed out; tallies incomplete");
    if (status & MCRT_STATUS_TIMEOUT) return fail(ctx, MCRT_E_TIMEOUT, "mcrt_launch_packets: time budget exhausted");
    if (status & (MCRT_STATUS_EVENT_CAP | MCRT_STATUS_TRIAL_CAP))
        return fail(ctx, MCRT_E_EVENT_CAP, "mcrt_launch_packets: packets reached the event or trial cap");
    return MCRT_OK;
}

static mcrt_status launch_batched(mcrt_ctx* const* models, int32_t n_models, const mcrt_launch_desc* desc,
                                  mcrt_stats* out_stats);

static mcrt_status launch_one(mcrt_ctx* ctx, const mcrt_launch_desc* d, mcrt_stats* st_out, bool want_sync) {
    mcrt_status st = check_desc(ctx, d);
    if (st != MCRT_OK) return st;
    JobDev job;
    st = prepare_model(ctx, d, d->stream, job);
    if (st != MCRT_OK) return st;
    const bool sur = d->optics == MCRT_OPTICS_SURROGATE;
    if (sur && !ctx->sur_set) return fail(ctx, MCRT_E_STATE, "mcrt_launch_packets: no surrogate attached (mcrt_set_surrogate)");
    if (sur && ctx->g.n_patches > 0)
        return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: refined grids take table, Rayleigh or dipole optics");
    // FP32 table launches tally in a kernel of their own unless asked not to
    const bool deferred_table = !sur && ctx->t.model == MCRT_SCAT_TABLE && d->precision == MCRT_FP32 &&
                                d->n_cameras > 0 && !(d->time_budget_s > 0.0) && !(d->flags & MCRT_FLAG_INLINE_TALLY);
    const bool rounds = sur || deferred_table;
    TransportParams P{};
    fill_common(d, P);
    P.g = ctx->g;
    P.t = ctx->t;
    const bool validate = sur && ctx->sur_bound < 0.f;  // every evaluation from the tables
    if (sur && !validate) {  // extinction and emission from the network's alpha table
        P.t.kext = ctx->d_sur_kext;
        P.t.k_iso = 0;
        P.t.k_const = 0;
    }
    for (int a = 0; a < 3; ++a) {
        P.lo_f[a] = job.lo_f[a];
        P.d_f[a] = job.d_f[a];
    }
    for (int s = 0; s < d->n_sources; ++s) P.src[s].eps = job.src_eps[s];
    P.thermal_cdf = job.thermal_cdf;
    P.thermal_total = job.thermal_total;
    P.thermal_guide = job.thermal_guide;
    P.n_guide = job.n_guide;
    P.S = job.S;
    P.absorbed = job.absorbed;
    const long long total = desc_total(d);
    const long long pb = d->pid_begin, pe = d->pid_end <= 0 ? total : d->pid_end;
    if (pb < 0 || pe > total || pb > pe) return fail(ctx, MCRT_E_INVAL, "mcrt_launch_packets: bad packet id range");
    P.pid_begin = pb;
    P.pid_end = pe;
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
    int bps = transport_max_blocks_per_sm(d->precision, P.t.model, false, block, smem, P.g.n_patches > 0);
    if (d->blocks_per_sm > 0 && d->blocks_per_sm < bps) bps = d->blocks_per_sm;
    const long long work = pe - pb;
    long long grid = (long long)ctx->n_sm * bps;
    const long long need = (work + block - 1) / block;
    if (need < grid) grid = need > 0 ? need : 1;

    if (rounds) {
        // capacity of a round: up to 2^21 packets in flight, 32 tally records each
        unsigned long long cap = work < (1ll << 21) ? (unsigned long long)(work > 0 ? work : 1) : (1ull << 21);
        // soft limit: room for one more record per thread of the transport grid
        // slots taken past the soft limit: one record per resident thread, plus (chunked
        // reservation) one chunk per resident warp
        const unsigned long long margin =
            (unsigned long long)ctx->n_sm * (16ull * 128ull + 64ull * 32ull * (unsigned long long)MCRT_REC_CHUNK);
        // queue: 32 records per packet in flight for the network's 64-byte records,
        // MCRT_TABLE_ROUND_RECORDS for the tables' 32-byte records, two slots of them (the
        // overlapped rounds fill one while the tally reads the other)
        const unsigned long long per_packet = sur ? 32ull : (unsigned long long)MCRT_TABLE_ROUND_RECORDS;
        const size_t rec_bytes = (size_t)(sur ? kRecordF4 : 2 * kTableRecordF4) * sizeof(float4);
        unsigned long long rec_cap = cap * per_packet;
        if (rec_cap < 4 * margin) rec_cap = 4 * margin;
        if (!ctx->d_wave) CK(ctx, cudaMalloc(&ctx->d_wave, sizeof(WaveCtl)));
        if (ctx->wave_cap < cap) {
            cudaFree(ctx->d_susp);
            cudaFree(ctx->d_res);
            ctx->d_susp = ctx->d_res = nullptr;
            ctx->wave_cap = 0;
            cudaError_t e = cudaMalloc(&ctx->d_susp, (size_t)cap * kStateF4 * sizeof(float4));
            if (e == cudaSuccess) e = cudaMalloc(&ctx->d_res, (size_t)cap * kStateF4 * sizeof(float4));
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(ctx, MCRT_E_NOMEM, "mcrt_launch_packets: surrogate packet buffers: %s", cudaGetErrorString(e));
            }
            ctx->wave_cap = cap;
        }
        if (ctx->rec_bytes < (size_t)rec_cap * rec_bytes) {
            cudaFree(ctx->d_records);
            ctx->d_records = nullptr;
            ctx->rec_bytes = 0;
            cudaError_t e = cudaMalloc(&ctx->d_records, (size_t)rec_cap * rec_bytes);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(ctx, MCRT_E_NOMEM, "mcrt_launch_packets: surrogate tally queue: %s", cudaGetErrorString(e));
            }
            ctx->rec_bytes = (size_t)rec_cap * rec_bytes;
        }
        ctx->rec_cap = rec_cap;
        P.sur.image = ctx->d_sur_image;
        P.sur.image_tc = ctx->d_sur_image_tc;
        P.sur.tally_engine = (d->flags & MCRT_FLAG_MMA_SYNC_TALLY) ? MCRT_ENGINE_MMA_SYNC : MCRT_ENGINE_TCGEN05;
        P.sur.err_map = ctx->d_sur_map;
        P.sur.bound = ctx->sur_bound;
        P.sur.env_margin = validate ? 0.f : 0.05f;
        P.sur.ctl = ctx->d_wave;
        P.sur.records = ctx->d_records;
        P.sur.rec_cap = ctx->rec_cap;
        P.sur.rec_soft = ctx->rec_cap - margin;
        P.sur.suspend = ctx->d_susp;
        P.sur.resume = ctx->d_res;
        int n_rounds = 0;
        float ms = 0.f, kms[3] = {0.f, 0.f, 0.f};
        // overlap of a round's tally with the next transport is opt-in: measured slower on the
        // disk (the latency-bound transport slows down under the tally's DRAM traffic)
        const bool overlap = !sur && d->tally_blocks_per_sm > 0;
        if (overlap && !ctx->tally_stream) {
            int lo = 0, hi = 0;
            CK(ctx, cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CK(ctx, cudaStreamCreateWithPriority(&ctx->tally_stream, cudaStreamNonBlocking, hi));
        }
        if (work > 0 && overlap) {
            // the transport leaves room on every SM for the tally kernels of the round before
            P.sur.deferred = kScatTableDeferred;
            const size_t tsm = transport_smem_bytes(P, MCRT_FP32, 128);
            const int bmax = transport_max_blocks_per_sm(MCRT_FP32, kScatTableDeferred, false, 128, tsm, P.g.n_patches > 0);
            int tbps = d->blocks_per_sm > 0 ? d->blocks_per_sm : (bmax > 2 ? bmax - 2 : 1);
            if (tbps > bmax) tbps = bmax;
            const int abps = d->tally_blocks_per_sm;
            CK(ctx, run_table_rounds_overlapped(P, ctx->n_sm, cap, tbps, abps, &n_rounds, &ms, kms, ctx->stream,
                                                ctx->tally_stream));
        } else if (work > 0) {
            CK(ctx, run_round_transport(P, sur ? kScatSurrogate : kScatTableDeferred, ctx->n_sm, cap, &n_rounds, &ms,
                                        kms, ctx->stream));
        }
        ctx->launched = true;
        ctx->last_optics = sur ? MCRT_OPTICS_SURROGATE : MCRT_OPTICS_TABLES;
        if (trace_host)
            CK(ctx, cudaMemcpyAsync(trace_host, P.trace, (size_t)d->n_trace * 16 * sizeof(double),
                                    cudaMemcpyDeviceToHost, ctx->stream));
        double raw[16];
        unsigned status = 0;
        WaveCtl w{};
        CK(ctx, cudaMemcpyAsync(raw, ctx->d_work + 8, 16 * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaMemcpyAsync(&status, ctx->d_work + 8 + 16 * 8, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
        if (work > 0) CK(ctx, cudaMemcpyAsync(&w, ctx->d_wave, sizeof(WaveCtl), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        if (st_out) {
            add_stats(st_out, raw, status, ms);
            add_wave_stats(st_out, w);
            st_out->ms_transport += kms[0];
            st_out->ms_tally += kms[1];
            st_out->ms_scatter += kms[2];
        }
        if (!sur && w.cnt[kCntOverflow] > 0)
            return fail(ctx, MCRT_E_CUDA, "mcrt_launch_packets: internal error, tally queue overflow");
        return status_of(ctx, status);
    }

    CK(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
    if (work > 0) CK(ctx, launch_transport(P, d->precision, block, (int)grid, ctx->stream));
    CK(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
    ctx->launched = true;
    ctx->last_optics = MCRT_OPTICS_TABLES;

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
    if (st_out) add_stats(st_out, raw, status, ms);
    return status_of(ctx, status);
}

mcrt_status mcrt_launch_packets(mcrt_ctx* const* models, int32_t n_models, const mcrt_launch_desc* desc,
                                mcrt_stats* out_stats) {
    if (!models || n_models < 1 || !desc) return fail(nullptr, MCRT_E_INVAL, "mcrt_launch_packets: no models or desc");
    for (int m = 0; m < n_models; ++m)
        if (!models[m]) return fail(nullptr, MCRT_E_INVAL, "mcrt_launch_packets: model %d is NULL", m);
    if (out_stats) std::memset(out_stats, 0, sizeof(*out_stats));
    if (n_models == 1) return launch_one(models[0], desc, out_stats, out_stats != nullptr);
    return launch_batched(models, n_models, desc, out_stats);
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
    if (ctx->last_optics == MCRT_OPTICS_SURROGATE && ctx->sur_set && ctx->sur_bound >= 0.f) {
        p.t.kext = ctx->d_sur_kext;
        p.t.k_iso = 0;
        p.t.k_const = 0;
    }
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

mcrt_status mcrt_microbench(int32_t kind, uint64_t bytes, uint64_t n_ops, double* ms_out) {
    if ((kind != 0 && kind != 1) || bytes < 256 || !ms_out) return fail(nullptr, MCRT_E_INVAL, "mcrt_microbench: bad arguments");
    int dev = 0, n_sm = 0;
    CK(nullptr, cudaGetDevice(&dev));
    CK(nullptr, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    DevIn buf;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf.owned, bytes);
    if (e == cudaErrorMemoryAllocation) {
        (void)cudaGetLastError();
        return fail(nullptr, MCRT_E_NOMEM, "mcrt_microbench: %llu bytes", (unsigned long long)bytes);
    }
    if (e == cudaSuccess) e = cudaMemset(buf.owned, 0, bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch_microbench(kind, (double*)buf.owned, bytes, n_ops, n_sm, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
    if (e == cudaSuccess) e = launch_microbench(kind, (double*)buf.owned, bytes, n_ops, n_sm, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(nullptr, MCRT_E_CUDA, "mcrt_microbench: %s", cudaGetErrorString(e));
    *ms_out = ms;
    return MCRT_OK;
}

mcrt_status mcrt_set_tallies(mcrt_ctx* ctx, const double* source, const double* absorbed) {
    if (!ctx) return fail(nullptr, MCRT_E_INVAL, "mcrt_set_tallies: ctx is NULL");
    if (!ctx->launched) return fail(ctx, MCRT_E_STATE, "mcrt_set_tallies: no launch yet");
    if (source && ctx->n_cam > 0)
        CK(ctx, cudaMemcpyAsync(ctx->d_S, source, (size_t)ctx->g.ncell * ctx->n_cam * 4 * sizeof(double),
                                cudaMemcpyDefault, ctx->stream));
    if (absorbed)
        CK(ctx, cudaMemcpyAsync(ctx->d_absorbed, absorbed, (size_t)ctx->g.ncell * sizeof(double), cudaMemcpyDefault,
                                ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MCRT_OK;
}

mcrt_status mcrt_tally_buffers(mcrt_ctx* ctx, double** source, double** absorbed, int64_t* source_count,
                               int64_t* absorbed_count) {
    if (!ctx) return fail(nullptr, MCRT_E_INVAL, "mcrt_tally_buffers: ctx is NULL");
    if (!ctx->launched) return fail(ctx, MCRT_E_STATE, "mcrt_tally_buffers: no launch yet");
    if (source) *source = ctx->n_cam > 0 ? ctx->d_S : nullptr;
    if (absorbed) *absorbed = ctx->d_absorbed;
    if (source_count) *source_count = ctx->n_cam > 0 ? (int64_t)ctx->g.ncell * ctx->n_cam * 4 : 0;
    if (absorbed_count) *absorbed_count = (int64_t)ctx->g.ncell;
    return MCRT_OK;
}

mcrt_status mcrt_set_surrogate(mcrt_ctx* ctx, mcrt_surrogate* s, double bound) {
    if (!ctx || !s) return fail(ctx, MCRT_E_INVAL, "mcrt_set_surrogate: ctx or surrogate is NULL");
    if (!ctx->tables_set || ctx->t.model != MCRT_SCAT_TABLE)
        return fail(ctx, MCRT_E_STATE, "mcrt_set_surrogate: the model needs MCRT_SCAT_TABLE optics as the fallback");
    if (!(bound == bound)) return fail(ctx, MCRT_E_INVAL, "mcrt_set_surrogate: bound is NaN");
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (!ctx->d_sur_image) {
        cudaError_t e = cudaMalloc(&ctx->d_sur_image, mlp::kImgBytes);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_sur_image_tc, tc::kImgBytes);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_sur_map, sizeof(float) * kErrMapCells);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            free_surrogate(ctx);
            return fail(ctx, MCRT_E_NOMEM, "mcrt_set_surrogate: %s", cudaGetErrorString(e));
        }
    }
    cudaFree(ctx->d_sur_kext);
    ctx->d_sur_kext = nullptr;
    CK(ctx, cudaMalloc(&ctx->d_sur_kext, (size_t)ctx->t.n_ktheta * sizeof(float4)));
    ctx->sur_set = false;
    int fixed = 0;
    const mcrt_status st = mcrt_surrogate_export(s, ctx->t.n_ktheta, ctx->d_kext, ctx->d_sur_image,
                                                 ctx->d_sur_image_tc, ctx->d_sur_map, ctx->d_sur_kext, &fixed);
    if (st != MCRT_OK) return fail(ctx, st, "mcrt_set_surrogate: %s", mcrt_last_error(nullptr));
    ctx->sur_bound = bound > 0.0 ? (float)bound : (bound < 0.0 ? -1.f : 0.05f);
    ctx->sur_kext_fixed = fixed;
    ctx->sur_set = true;
    return MCRT_OK;
}

mcrt_status mcrt_destroy(mcrt_ctx* ctx) {
    if (!ctx) return MCRT_OK;
    free_tables(ctx);
    cudaFree(ctx->d_cells);
    cudaFree(ctx->d_patches);
    cudaFree(ctx->d_cdf);
    cudaFree(ctx->d_block_sums);
    cudaFree(ctx->d_guide);
    cudaFree(ctx->d_S);
    cudaFree(ctx->d_absorbed);
    cudaFree(ctx->d_work);
    free_wave(ctx);
    if (ctx->tally_stream) cudaStreamDestroy(ctx->tally_stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return MCRT_OK;
}

mcrt_status mcrt_unit_eval(int32_t fn, int32_t precision, int64_t n, const double* in, double* out) {
    static const int in_w[8] = {6, 7, 10, 12, 8, 16, 16, 8};
    static const int out_w[8] = {4, 8, 6, 4, 4, 4, 4, 4};
    if (fn < 0 || fn > 7) return fail(nullptr, MCRT_E_INVAL, "mcrt_unit_eval: unknown fn %d", fn);
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

// ---------------------------------------------------------------------------------
// Batched launches: many models (e.g. one per wavelength) in one persistent launch
// ---------------------------------------------------------------------------------
struct mcrt_batch {
    std::vector<mcrt_ctx*> models;
    mcrt_launch_desc desc{};
    std::vector<mcrt_source> sources;
    std::vector<mcrt_camera> cameras;
    cudaStream_t stream = nullptr;  // private stream: the launch sequence is captured on it
    std::vector<JobDev> jobs;
    JobDev* d_jobs = nullptr;
    JobDev* d_trial = nullptr;
    unsigned char* d_work = nullptr;
    TransportParams P{};
    long long per_job = 0;
    int n_sm = 0, block = 128, bps = 0, interleave = 0;
    double* d_images = nullptr;
    std::vector<size_t> img_off;  // [job][camera] offsets into d_images
    size_t img_elems = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t kernel_node = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

#define BK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            (void)cudaGetLastError();                                                             \
            return fail(nullptr, MCRT_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
        }                                                                                         \
    } while (0)

void batch_free(mcrt_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_jobs);
    cudaFree(b->d_trial);
    cudaFree(b->d_work);
    cudaFree(b->d_images);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Job table, work area and launch parameters for the models; tallies of every model
// are sized and zeroed (prepare_model).
mcrt_status batch_build(mcrt_batch** out, mcrt_ctx* const* models, int32_t n_models, const mcrt_launch_desc* desc,
                        bool images) {
    *out = nullptr;
    if (!models || n_models < 1 || !desc) return fail(nullptr, MCRT_E_INVAL, "batch: no models or desc");
    mcrt_status st = check_desc(nullptr, desc);
    if (st != MCRT_OK) return st;
    if (desc->n_trace > 0 || desc->accumulate || desc->pid_begin != 0 || desc->pid_end > 0)
        return fail(nullptr, MCRT_E_INVAL, "batch: traces, accumulation and packet id ranges are single-model options");
    if (desc->optics != MCRT_OPTICS_TABLES)
        return fail(nullptr, MCRT_E_INVAL, "batch: surrogate optics are a single-model option");
    for (int m = 0; m < n_models; ++m) {
        if (!models[m]) return fail(nullptr, MCRT_E_INVAL, "batch: model %d is NULL", m);
        if (!models[m]->tables_set) return fail(nullptr, MCRT_E_STATE, "batch: model %d has no optics", m);
        if (models[m]->t.model != models[0]->t.model)
            return fail(nullptr, MCRT_E_INVAL, "batch: all models need the same scattering model");
        if (models[m]->t.model == MCRT_SCAT_DIPOLE)
            return fail(nullptr, MCRT_E_INVAL, "batch: aligned-spheroid optics are a single-model option");
        if (models[m]->g.n_patches > 0)
            return fail(nullptr, MCRT_E_INVAL, "batch: refined grids are a single-model option");
    }
    mcrt_batch* b = new (std::nothrow) mcrt_batch();
    if (!b) return fail(nullptr, MCRT_E_NOMEM, "batch: host allocation failed");
    b->models.assign(models, models + n_models);
    b->desc = *desc;
    b->sources.assign(desc->sources, desc->sources + desc->n_sources);
    b->cameras.assign(desc->cameras, desc->cameras + desc->n_cameras);
    b->desc.sources = b->sources.data();
    b->desc.cameras = b->cameras.data();
    b->per_job = desc_total(desc);
    b->jobs.resize(n_models);
    for (int m = 0; m < n_models; ++m) {
        st = prepare_model(models[m], &b->desc, desc->stream + (uint32_t)m, b->jobs[m]);
        if (st != MCRT_OK) {
            std::snprintf(g_err, sizeof g_err, "batch: model %d: %s", m, models[m]->err);
            batch_free(b);
            return st;
        }
        b->jobs[m].pid_start = (long long)m * b->per_job;
        b->jobs[m].index = (unsigned)m;
        if (cudaStreamSynchronize(models[m]->stream) != cudaSuccess) {
            batch_free(b);
            return fail(nullptr, MCRT_E_CUDA, "batch: model %d stream failed", m);
        }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_jobs, sizeof(JobDev) * n_models);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_trial, sizeof(JobDev) * n_models);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_work, kWorkBytes);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_jobs, b->jobs.data(), sizeof(JobDev) * n_models, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && images) {
        for (int m = 0; m < n_models; ++m)
            for (int k = 0; k < desc->n_cameras; ++k) {
                b->img_off.push_back(b->img_elems);
                b->img_elems += (size_t)4 * desc->cameras[k].npix[0] * desc->cameras[k].npix[1];
            }
        if (b->img_elems) e = cudaMalloc(&b->d_images, b->img_elems * sizeof(double));
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        batch_free(b);
        return fail(nullptr, e == cudaErrorMemoryAllocation ? MCRT_E_NOMEM : MCRT_E_CUDA, "batch: %s",
                    cudaGetErrorString(e));
    }
    TransportParams& P = b->P;
    fill_common(&b->desc, P);
    P.t = models[0]->t;  // selects the kernel; the tables themselves come from the jobs
    P.jobs = b->d_jobs;
    P.n_jobs = n_models;
    P.pid_begin = 0;
    P.pid_end = (long long)n_models * b->per_job;
    P.counter = reinterpret_cast<unsigned long long*>(b->d_work);
    P.stats = reinterpret_cast<double*>(b->d_work + 8);
    P.status = reinterpret_cast<unsigned*>(b->d_work + 8 + 16 * 8);
    b->block = desc->block_size > 0 ? desc->block_size : 128;
    if (b->block % 32 != 0 || b->block > 128) {
        batch_free(b);
        return fail(nullptr, MCRT_E_INVAL, "batch: block_size must be a multiple of 32, <= 128");
    }
    b->bps = desc->blocks_per_sm;
    *out = b;
    return MCRT_OK;
}

int batch_grid(const mcrt_batch* b, const TransportParams& P, int block, int bps_req) {
    const size_t smem = transport_smem_bytes(P, b->desc.precision, block);
    int bps = transport_max_blocks_per_sm(b->desc.precision, P.t.model, true, block, smem);
    if (bps_req > 0 && bps_req < bps) bps = bps_req;
    long long grid = (long long)b->n_sm * bps;
    const long long work = P.pid_end - P.pid_begin;
    const long long need = (work + block - 1) / block;
    if (need < grid) grid = need > 0 ? need : 1;
    return (int)grid;
}

// Queues one batched transport launch (and optionally the images) on b->stream.
mcrt_status batch_enqueue(mcrt_batch* b, const TransportParams& P, int block, int bps, bool zero_tallies,
                          bool images, bool capturing = false) {
    // inside a stream capture the timing events must become event-record nodes
    const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    BK(cudaMemsetAsync(b->d_work, 0, kWorkBytes, b->stream));
    if (zero_tallies)
        for (mcrt_ctx* c : b->models) {
            BK(cudaMemsetAsync(c->d_S, 0, c->S_elems * sizeof(double), b->stream));
            BK(cudaMemsetAsync(c->d_absorbed, 0, (size_t)c->g.ncell * sizeof(double), b->stream));
        }
    BK(cudaEventRecordWithFlags(b->ev0, b->stream, ev_flags));
    if (P.pid_end > P.pid_begin) BK(launch_transport(P, b->desc.precision, block, batch_grid(b, P, block, bps), b->stream));
    BK(cudaEventRecordWithFlags(b->ev1, b->stream, ev_flags));
    if (images && b->d_images) {
        size_t i = 0;
        for (size_t m = 0; m < b->models.size(); ++m) {
            const mcrt_ctx* c = b->models[m];
            for (int k = 0; k < b->desc.n_cameras; ++k, ++i) {
                const mcrt_camera& cm = b->cameras[k];
                ImageParams ip{};
                ip.g = c->g;
                ip.t = c->t;
                const double nn = std::sqrt(cm.dir[0] * cm.dir[0] + cm.dir[1] * cm.dir[1] + cm.dir[2] * cm.dir[2]);
                for (int a = 0; a < 3; ++a) ip.cam.dir[a] = cm.dir[a] / nn;
                host_basis(ip.cam.dir, ip.cam.th, ip.cam.ph);
                for (int a = 0; a < 3; ++a) ip.center[a] = cm.center[a];
                ip.fov[0] = cm.fov[0];
                ip.fov[1] = cm.fov[1];
                ip.npix[0] = cm.npix[0];
                ip.npix[1] = cm.npix[1];
                ip.cam_index = k;
                ip.n_cam = b->desc.n_cameras;
                ip.S = c->d_S;
                ip.out = b->d_images + b->img_off[i];
                BK(launch_image(ip, b->desc.precision, b->stream));
            }
        }
    }
    return MCRT_OK;
}

mcrt_status batch_read_stats(mcrt_batch* b, mcrt_stats* out) {
    double raw[16];
    unsigned status = 0;
    BK(cudaMemcpyAsync(raw, b->d_work + 8, sizeof raw, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaMemcpyAsync(&status, b->d_work + 8 + 16 * 8, sizeof status, cudaMemcpyDeviceToHost, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    float ms = 0.f;
    BK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    if (out) {
        std::memset(out, 0, sizeof(*out));
        add_stats(out, raw, status, ms);
    }
    return status_of(nullptr, status);
}

// Captures memsets + transport + images into a CUDA graph and finds the transport node.
mcrt_status batch_capture(mcrt_batch* b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    // dynamic shared memory attributes are set outside the capture
    batch_grid(b, b->P, b->block, b->bps);
    BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    mcrt_status st = batch_enqueue(b, b->P, b->block, b->bps, true, true, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (st != MCRT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(nullptr, MCRT_E_CUDA, "batch: capture: %s", cudaGetErrorString(e));
    b->graph = g;
    BK(cudaGraphInstantiate(&b->exec, b->graph, 0));
    size_t n = 0;
    BK(cudaGraphGetNodes(b->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    BK(cudaGraphGetNodes(b->graph, nodes.data(), &n));
    const void* kfn = transport_kernel(b->desc.precision, b->P.t.model, true);
    b->kernel_node = nullptr;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        BK(cudaGraphNodeGetType(nd, &ty));
        if (ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp;
        BK(cudaGraphKernelNodeGetParams(nd, &kp));
        if (kp.func == kfn) b->kernel_node = nd;
    }
    if (!b->kernel_node && b->P.pid_end > b->P.pid_begin)
        return fail(nullptr, MCRT_E_CUDA, "batch: transport node not found in the captured graph");
    return MCRT_OK;
}

}  // namespace

extern "C" {

mcrt_status mcrt_batch_create(mcrt_batch** out, mcrt_ctx* const* models, int32_t n_models,
                              const mcrt_launch_desc* desc) {
    if (!out) return fail(nullptr, MCRT_E_INVAL, "mcrt_batch_create: out is NULL");
    mcrt_batch* b = nullptr;
    mcrt_status st = batch_build(&b, models, n_models, desc, true);
    if (st != MCRT_OK) return st;
    st = batch_capture(b);
    if (st != MCRT_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return MCRT_OK;
}

mcrt_status mcrt_batch_run(mcrt_batch* b, uint32_t seed, mcrt_stats* out_stats) {
    if (!b || !b->exec) return fail(nullptr, MCRT_E_INVAL, "mcrt_batch_run: no batch");
    if (b->kernel_node) {
        TransportParams Pr = b->P;
        Pr.seed = seed;
        cudaKernelNodeParams kp;
        BK(cudaGraphKernelNodeGetParams(b->kernel_node, &kp));
        void* args[] = {&Pr};
        kp.kernelParams = args;
        kp.extra = nullptr;
        BK(cudaGraphExecKernelNodeSetParams(b->exec, b->kernel_node, &kp));
    }
    BK(cudaGraphLaunch(b->exec, b->stream));
    for (mcrt_ctx* c : b->models) c->launched = true;
    if (!out_stats) return MCRT_OK;
    return batch_read_stats(b, out_stats);
}

mcrt_status mcrt_batch_tune(mcrt_batch* b, int64_t packets_per_job, mcrt_tune_report* report) {
    if (!b) return fail(nullptr, MCRT_E_INVAL, "mcrt_batch_tune: no batch");
    if (packets_per_job < 1) return fail(nullptr, MCRT_E_INVAL, "mcrt_batch_tune: packets_per_job < 1");
    const long long trial = packets_per_job < b->per_job ? packets_per_job : b->per_job;
    std::vector<JobDev> tj = b->jobs;
    for (size_t m = 0; m < tj.size(); ++m) tj[m].pid_start = (long long)m * trial;
    BK(cudaMemcpy(b->d_trial, tj.data(), sizeof(JobDev) * tj.size(), cudaMemcpyHostToDevice));
    mcrt_tune_report rep{};
    double best = -1.0;
    const int blocks[3] = {64, 96, 128};
    for (int bi = 0; bi < 3; ++bi)
        for (int occ = 0; occ < 2; ++occ)
            for (int il = 0; il < 2; ++il) {
                TransportParams Pt = b->P;
                Pt.jobs = b->d_trial;
                Pt.pid_end = (long long)tj.size() * trial;
                Pt.job_interleave = il;
                const size_t smem = transport_smem_bytes(Pt, b->desc.precision, blocks[bi]);
                const int bmax = transport_max_blocks_per_sm(b->desc.precision, Pt.t.model, true, blocks[bi], smem);
                const int bps = occ == 0 ? bmax : (bmax > 1 ? bmax - 1 : 1);
                if (occ == 1 && bmax <= 1) continue;
                mcrt_status st = batch_enqueue(b, Pt, blocks[bi], bps, false, false);
                if (st != MCRT_OK) return st;
                mcrt_stats s{};
                st = batch_read_stats(b, &s);
                if (st != MCRT_OK && st != MCRT_E_EVENT_CAP) return st;
                const double rate = s.kernel_ms > 0 ? s.events / (s.kernel_ms * 1e-3) : 0.0;
                if (rep.n < 16) {
                    rep.block_size[rep.n] = blocks[bi];
                    rep.blocks_per_sm[rep.n] = bps;
                    rep.interleave[rep.n] = il;
                    rep.events_per_s[rep.n] = rate;
                    if (rate > best) {
                        best = rate;
                        rep.best = rep.n;
                    }
                    rep.n++;
                }
            }
    b->block = rep.block_size[rep.best];
    b->bps = rep.blocks_per_sm[rep.best];
    b->interleave = rep.interleave[rep.best];
    b->P.job_interleave = b->interleave;
    if (report) *report = rep;
    return batch_capture(b);
}

mcrt_status mcrt_batch_images(mcrt_batch* b, double* out) {
    if (!b || !out) return fail(nullptr, MCRT_E_INVAL, "mcrt_batch_images: no batch or out");
    if (!b->d_images) return MCRT_OK;
    BK(cudaMemcpyAsync(out, b->d_images, b->img_elems * sizeof(double), cudaMemcpyDefault, b->stream));
    BK(cudaStreamSynchronize(b->stream));
    return MCRT_OK;
}

mcrt_status mcrt_batch_destroy(mcrt_batch* b) {
    if (b) cudaStreamSynchronize(b->stream);
    batch_free(b);
    return MCRT_OK;
}

}  // extern "C"

// n_models > 1: one persistent launch over the job table of all models (no graph).
static mcrt_status launch_batched(mcrt_ctx* const* models, int32_t n_models, const mcrt_launch_desc* desc,
                                  mcrt_stats* out_stats) {
    mcrt_batch* b = nullptr;
    mcrt_status st = batch_build(&b, models, n_models, desc, false);
    if (st != MCRT_OK) return st;
    st = batch_enqueue(b, b->P, b->block, b->bps, false, false);
    if (st == MCRT_OK) {
        for (mcrt_ctx* c : b->models) c->launched = true;
        mcrt_stats tmp{};
        st = batch_read_stats(b, out_stats ? out_stats : &tmp);
    }
    batch_free(b);
    return st;
}
