// mcrt_internal.h -- device-side layouts shared by the translation units of the
// library (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "mcrt.h"

namespace mcrt {

constexpr int kMaxPatches = 64;
// Round-based paths: a warp reserves its tally-record slots in chunks of this many per
// lane (one atomic per chunk instead of one per tallying step); 0 reserves per step.
// Measured when introduced, on the 192^3 disk: table-round transport 910 ms per 1e8-packet
// step with 4 or 8, 924 ms with 16 and 1027 ms per step without chunks.
#ifndef MCRT_REC_CHUNK
#define MCRT_REC_CHUNK 4
#endif
// Table rounds: tally records of queue per packet in flight (2^21 packets per round).
// On the 192^3 disk, 32 (107 rounds per 1e8-packet step) beat 64 and 128 (65 and 48
// rounds): the transport took 853, 862 and 906 ms.
#ifndef MCRT_TABLE_ROUND_RECORDS
#define MCRT_TABLE_ROUND_RECORDS 32
#endif
constexpr int kMaxCams = MCRT_MAX_CAMERAS;
constexpr int kMaxSources = MCRT_MAX_SOURCES;
// scattering-model id of the transport instantiation that defers the optics to the
// network (internal; the tables stay MCRT_SCAT_TABLE)
constexpr int kScatSurrogate = 2;
// table optics with the source tally deferred to a separate coherent kernel (FP32,
// one model): the transport kernel leaves 32-byte records instead of the camera loop
constexpr int kScatTableDeferred = 3;
constexpr int kTableRecordF4 = 2;  // table tally record: 2 float4 (32 bytes)
constexpr int kErrMapCells = 4096;  // 8^4 cells of (cos theta_i, cos theta_s, delta phi, s)
constexpr int kStateF4 = 8;         // suspended packet: 8 float4 (128 bytes)
constexpr int kRecordF4 = 4;        // tally record: 4 float4 (64 bytes)

// Cell record, 32 bytes = one DRAM sector: q_B (float4) then
// (kappa_abs, kappa_sca, emissivity, 0).
// A statically refined patch of the root grid (one level of a composite mesh): the
// root cells of `box` (half-open, root-cell indices) are replaced by a uniform grid of
// `factor` cells per root cell along each axis, numbered from `offset` on.
struct PatchDev {
    int box[6];
    int factor;
    int n[3];
    long long offset;
    double lo[3], d[3];
    float lo_f[3], d_f[3];
};

struct GridDev {
    int n[3];      // root grid
    int periodic;  // bit a: axis a periodic (MCRT_BOUNDARY_PERIODIC_*)
    double lo[3], hi[3], d[3];
    long long ncell;       // all cells: the root's, then each patch's
    long long ncell_root;  // root cells
    const float4* cells;   // [ncell][2]; a covered root cell holds (1,0,0,0), (0, 0, 0, patch + 1 as bits)
    int n_patches;
    const PatchDev* patches;  // [n_patches], device
};

// Aligned dipole spheroids (MCRT_SCAT_DIPOLE): index 0 a principal axis perpendicular
// to the symmetry axis, 1 the symmetry axis.
struct DipoleDev {
    double rho_re, rho_im;  // alpha'_1 / alpha'_0
    double ca[2], cs[2];    // absorption and scattering cross sections over their orientation averages
    double zn;              // Zhat = zn M(J), 1/sr
    double env;             // bound of (Zhat X)_0 / I
    // the same constants rounded once to FP32 on the host, for the FP32 kernels (no FP64
    // conversion per segment on GB300's narrow FP64 pipe)
    float f_rho_re, f_rho_im, f_ca[2], f_cs[2], f_zn, f_env;
};

// Dipole constants in the kernel's arithmetic type.
template <typename T> struct DipoleConst {
    T rho_re, rho_im, ca0, ca1, cs0, cs1, zn, env;
};
template <typename T> __host__ __device__ inline DipoleConst<T> dipole_const(const DipoleDev& d);
template <> __host__ __device__ inline DipoleConst<float> dipole_const<float>(const DipoleDev& d) {
    return DipoleConst<float>{d.f_rho_re, d.f_rho_im, d.f_ca[0], d.f_ca[1], d.f_cs[0], d.f_cs[1], d.f_zn, d.f_env};
}
template <> __host__ __device__ inline DipoleConst<double> dipole_const<double>(const DipoleDev& d) {
    return DipoleConst<double>{d.rho_re, d.rho_im, d.ca[0], d.ca[1], d.cs[0], d.cs[1], d.zn, d.env};
}

struct TablesDev {
    int model;            // MCRT_SCAT_*
    int n_bins, n_theta, n_ktheta;
    int k_iso;            // alpha2 = alpha3 = 0 everywhere and alpha1 constant
    int k_const;          // alpha does not depend on theta'
    const float4* mix;    // [n_theta][2] (P11,P12,P22,P33),(P34,P44,0,0) of the bin mixture
    const float4* bins;   // [n_bins][n_theta][2]
    const double* env_cdf;  // [n_bins][n_theta-1] normalised cumulative envelope weights
    const float* env;     // [n_bins][n_theta-1] envelope max(P11_j, P11_j+1)
    const double* bin_cdf;  // [n_bins] normalised cumulative bin weights
    // the two cumulative weights rounded to FP32 once (stored after the FP64 ones), for
    // the FP32 kernels, which compare in FP32: no FP64 conversion per search step
    const float* env_cdf_f;
    const float* bin_cdf_f;
    const float4* kext;   // [n_ktheta] (alpha1, alpha2, alpha3, 0)
    double alpha1_mean;
    DipoleDev dip;        // MCRT_SCAT_DIPOLE constants
};

// Entry i of a cumulative weight table in the kernel's arithmetic type.
template <typename T> __device__ __forceinline__ T cdf_at(const double* d, const float* f, size_t i);
template <> __device__ __forceinline__ float cdf_at<float>(const double*, const float* f, size_t i) { return f[i]; }
template <> __device__ __forceinline__ double cdf_at<double>(const double* d, const float*, size_t i) { return d[i]; }

struct SourceDev {
    int type, beam_dir;
    long long start, count;
    double eps;  // energy per packet
    double pos[3];
};

struct CameraDev {
    double dir[3], th[3], ph[3];
};

// One job of a batched launch (a model, e.g. at one wavelength): its grid, tallies,
// tables, thermal-emission CDF and the energy per packet of each source.
struct JobDev {
    int n[3];
    int periodic;
    float lo_f[3], d_f[3];
    double lo[3], hi[3], d[3];
    long long ncell;
    const float4* cells;
    double* S;
    double* absorbed;
    TablesDev t;
    const double* thermal_cdf;
    double thermal_total;
    const long long* thermal_guide;
    long long n_guide;
    double src_eps[kMaxSources];
    long long pid_start;  // first index of the job in the batch's packet index space
    unsigned stream;      // Philox key word 1
    unsigned index;
};

// Control block of the surrogate path (device memory, rewritten by its kernels):
// packets in flight wait in two buffers between the transport launch, which moves
// them to their next scattering and queues the tally segments of the way, and the
// kernels that evaluate the network for the tallies and for the scattering.
struct WaveCtl {
    unsigned long long next_pid;       // new packets taken so far (relative to pid_begin)
    unsigned long long n_new;          // new packets of the current transport launch
    unsigned long long claim;          // work items claimed in the current transport launch
    unsigned long long n_resume;       // packets to resume in the current transport launch
    unsigned long long n_resume_next;  // packets written to the resume buffer by the scattering kernel
    unsigned long long n_suspend;      // packets suspended at a scattering by the current launch
    unsigned long long n_born;         // table rounds: new packets the birth kernel stored after the
                                       // resume list (packets born outside the grid are not stored)
    unsigned long long n_rec[2];       // tally records requested per record buffer (the table
                                       // rounds alternate two buffers; the surrogate uses [0])
    unsigned long long full;           // the record queue passed its soft limit: packets park
    // totals: network rows (tally, scattering), fallbacks (error map, realizability),
    // tally segments tallied in place for want of record space, envelope misses
    unsigned long long cnt[8];
};
enum { kCntTallyRows = 0, kCntScatRows, kCntFallbackMap, kCntFallbackReal, kCntOverflow, kCntEnvelopeMiss, kCntIterations };

struct SurrogateDev {
    const unsigned char* image;  // inference image (mcrt_mlp_infer.cuh layout)
    const unsigned char* image_tc;  // the same network for the tcgen05 engine (mcrt_mlp_tc.cuh)
    int tally_engine;            // MCRT_ENGINE_* of the tally kernel
    const float* err_map;        // [kErrMapCells] largest error per cell, units of N(s)
    float bound;                 // cells with a larger error use the tables
    float env_margin;            // rejection envelope factor (1 + margin)
    WaveCtl* ctl;
    float4* records;             // [rec_cap][kRecordF4]
    unsigned long long rec_cap;
    unsigned long long rec_soft;  // rec_cap minus the threads of the transport grid (one
                                  // more record each at most once the soft limit is passed)
    float4* suspend;             // [cap][kStateF4]
    float4* resume;              // [cap][kStateF4]
    int deferred;                // which round-based instantiation runs (kScat* id), 0: none
    int rec_slot;                // record buffer (and counter n_rec[rec_slot]) of this launch
};

struct TransportParams {
    GridDev g;
    float lo_f[3], d_f[3];  // FP32 copies of g.lo, g.d
    TablesDev t;
    int n_src;
    SourceDev src[kMaxSources];
    int n_cam;
    CameraDev cam[kMaxCams];
    const double* thermal_cdf;  // [ncell] inclusive cumulative emission weights
    double thermal_total;
    const long long* thermal_guide;  // [n_guide + 1]: first cell with cdf > k total / n_guide
    long long n_guide;
    double* S;         // [ncell][n_cam][4]
    double* absorbed;  // [ncell]
    unsigned seed, stream;
    long long pid_begin, pid_end;
    double roulette_thr, roulette_surv;
    long long max_events;
    int max_trials;
    double time_budget_ns;  // <= 0: none
    unsigned long long* counter;  // next packet index (relative to pid_begin)
    double* stats;  // [6] FP64 energy sums, then [10] u64 counters
    unsigned* status;
    double* trace;
    long long n_trace;
    // batched launch: job table (nullptr for a single model); packet indices
    // [0, total) are split over the jobs by JobDev::pid_start
    const JobDev* jobs;
    int n_jobs;
    int job_interleave;  // 1: packet index i belongs to job i % n_jobs (equal packet counts)
    SurrogateDev sur;    // surrogate path only
};

struct ImageParams {
    GridDev g;
    TablesDev t;
    CameraDev cam;
    double center[3], fov[2];
    int npix[2];
    int cam_index, n_cam;
    const double* S;  // [ncell][n_cam][4] or nullptr
    double* out;      // [4][ny][nx]
};

// launchers (defined in the .cu files)
cudaError_t launch_transport(const TransportParams& p, int precision, int block, int grid, cudaStream_t s);
// Births of a round of the FP32 table path (k_birth): the round's new packets in the
// waiting form after the resume list, before the round's transport launch.
cudaError_t launch_births(const TransportParams& p, int n_sm, cudaStream_t s);
const void* transport_kernel(int precision, int model, bool batch, bool refined = false);
int transport_max_blocks_per_sm(int precision, int model, bool batch, int block, size_t smem, bool refined = false);
size_t transport_smem_bytes(const TransportParams& p, int precision, int block);
cudaError_t launch_image(const ImageParams& p, int precision, cudaStream_t s);
cudaError_t launch_setup_cells(const float* ka, const float* ks, const float* bf, const float* em, long long ncell,
                               float4* cells, unsigned* bad, cudaStream_t s);
cudaError_t launch_prepare_tables(int model, int n_bins, int n_theta, int n_ktheta, const float* mueller,
                                  const float* bin_weight, const float* kext, float4* mix, float4* bins,
                                  double* env_cdf, float* env, double* bin_cdf, float4* kext4, double* alpha1_mean,
                                  cudaStream_t s);
cudaError_t launch_thermal_cdf(const GridDev& g, double alpha1_mean, double* cdf, double* block_sums, int n_blocks,
                               cudaStream_t s);
int thermal_cdf_blocks(long long ncell);
cudaError_t launch_thermal_guide(const double* cdf, long long ncell, long long* guide, long long n_guide,
                                 cudaStream_t s);
cudaError_t launch_unit_eval(int fn, int precision, long long n, const double* in, double* out, cudaStream_t s);
// FP64 reduction throughput kernels (kind 0 scalar atomics, 1 bulk 256-byte rows)
cudaError_t launch_microbench(int kind, double* buf, unsigned long long bytes, unsigned long long n_ops, int n_sm,
                              cudaStream_t s);
// marks the root cells covered by patches (records of patch p + 1, zero opacity and emission)
cudaError_t launch_mark_covered(const GridDev& g, const PatchDev* host_patches, cudaStream_t s);
// one-thread kernel: the 16 constants of mcrt_dipole_constants into out (device)
cudaError_t launch_dipole_setup(double eps_re, double eps_im, double aspect, double x, double* out, cudaStream_t s);
// round-based paths (mcrt_wave.cu): the transport loop of one launch with the tally
// (and, for the surrogate, the scattering) in kernels of their own; model is
// kScatSurrogate or kScatTableDeferred; ms_out: device time of the whole loop;
// ms_kernels[3]: summed times of the transport, tally and scattering kernels
cudaError_t run_round_transport(const TransportParams& p, int model, int n_sm, unsigned long long cap,
                                int* iterations, float* ms_out, float* ms_kernels, cudaStream_t s);
// table rounds with the tally of round r on stream s2 overlapping the transport of
// round r+1 on s: tbps transport blocks and tally_bps tally blocks per SM; the record
// queue (p.sur.records, capacity p.sur.rec_cap each) is two buffers back to back
cudaError_t run_table_rounds_overlapped(const TransportParams& p, int n_sm, unsigned long long cap, int tbps,
                                        int tally_bps, int* iterations, float* ms_out, float* ms_kernels,
                                        cudaStream_t s, cudaStream_t s2);

}  // namespace mcrt

// Optics tables of a model (device pointers owned by the model); MCRT_E_STATE when
// none are set.
mcrt_status mcrt_ctx_tables(const mcrt_ctx* ctx, mcrt::TablesDev* out);

// Records `fmt` as the calling thread's context-less error message (read with
// mcrt_last_error(NULL)) and returns st.
mcrt_status mcrt_fail_noctx(mcrt_status st, const char* fmt, ...);

// Inference data of a trained surrogate (mcrt_mlp.cu) for a model: inference image,
// error map and the extinction table distilled on n_ktheta angles.
mcrt_status mcrt_surrogate_export(mcrt_surrogate* s, int n_ktheta, const float4* table, unsigned char* d_image,
                                  unsigned char* d_image_tc, float* d_map, float4* d_kext, int* n_fixed);
