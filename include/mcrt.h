/*
 * mcrt.h -- C ABI of the GB300 polarized Monte-Carlo radiative transfer library.
 *
 * The library transports photon packets that carry the full Stokes vector
 * (I,Q,U,V) through a Cartesian grid of dust with magnetically aligned grains and
 * tallies them into the two-step polarimetry images of Kratos-polrad
 * (arXiv:2512.01283).  All compute runs in hand-written CUDA kernels for sm_103a;
 * nothing falls back to the CPU.  Every function returns an mcrt_status; no C++
 * exception crosses this boundary.
 *
 * Conventions shared by all calls
 *  - Grids are C-ordered [nz][ny][nx]; cell (i,j,k) spans
 *    [lo + (i,j,k) d, lo + (i+1,j+1,k+1) d] with d = (hi - lo) / (nx,ny,nz).
 *  - Stokes vectors of light travelling along n are given in the basis
 *    theta-hat = (cos t cos p, cos t sin p, -sin t), phi-hat = (-sin p, cos p, 0)
 *    of n = (t, p) (paper Sec. 2.1); Q > 0 means polarization along theta-hat;
 *    at the poles p = 0.
 *  - Pointer arguments may be host or device memory (detected with
 *    cudaPointerGetAttributes) unless stated otherwise.  Inputs are copied; the
 *    caller keeps ownership of every buffer it passes.
 *  - Work is queued on the stream given to mcrt_create_grid (NULL: the legacy
 *    default stream).  Calls that return data to host memory synchronize that
 *    stream before returning.
 *  - Errors: a failing call returns a negative mcrt_status and leaves a message
 *    readable with mcrt_last_error(ctx) (or mcrt_last_error(NULL) for failures
 *    without a context); the context stays usable unless the status is
 *    MCRT_E_CUDA from a sticky CUDA error.
 *  - Results are deterministic for a given (seed, stream, packet ids) up to the
 *    order of floating-point atomic additions in the tallies.
 */
#ifndef MCRT_H
#define MCRT_H

#include <stdint.h>

#if defined(__GNUC__)
#define MCRT_API __attribute__((visibility("default")))
#else
#define MCRT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcrt_ctx mcrt_ctx; /* opaque, owned by the library */

typedef enum {
    MCRT_OK = 0,
    MCRT_E_INVAL = -1,     /* bad argument; nothing was queued */
    MCRT_E_NOMEM = -2,     /* device or host allocation failed */
    MCRT_E_CUDA = -3,      /* a CUDA call failed; message holds cudaGetErrorString */
    MCRT_E_EVENT_CAP = -4, /* some packets hit the per-packet event or trial cap */
    MCRT_E_TIMEOUT = -5,   /* the launch's time budget ran out; tallies are partial */
    MCRT_E_STATE = -6      /* call out of order (e.g. image before any launch) */
} mcrt_status;

/* Boundary of the grid box, per axis: packets leaving through an outflow face escape;
 * through a face of a periodic axis they re-enter on the opposite face (the paper's
 * dust-cylinder test, Sec. 3, uses periodic conditions).  Combine the PERIODIC bits. */
enum {
    MCRT_BOUNDARY_OUTFLOW = 0,
    MCRT_BOUNDARY_PERIODIC_X = 1,
    MCRT_BOUNDARY_PERIODIC_Y = 2,
    MCRT_BOUNDARY_PERIODIC_Z = 4
};
enum { MCRT_SRC_POINT = 0, MCRT_SRC_BEAM = 1, MCRT_SRC_THERMAL = 2 };
/* Grain optics: Rayleigh (dipole of a sphere) and tables use mcrt_set_dust_tables;
 * aligned dipole spheroids use mcrt_set_dust_dipole. */
enum { MCRT_SCAT_RAYLEIGH = 0, MCRT_SCAT_TABLE = 1, MCRT_SCAT_DIPOLE = 4 };
enum { MCRT_FP32 = 0, MCRT_FP64 = 1 };
enum { MCRT_OPTICS_TABLES = 0, MCRT_OPTICS_SURROGATE = 1 };
/* Launch flags (mcrt_launch_desc.flags). */
enum {
    MCRT_FLAG_INLINE_TALLY = 1,  /* FP32 table launches: tally inside the transport kernel instead of the
                                    default rounds (transport, then a tally kernel over the queued segments) */
    MCRT_FLAG_MMA_SYNC_TALLY = 2 /* surrogate launches: the network of the tally and of the rejection
                                    trials on warp-level mma.sync instead of the default
                                    5th-generation tensor cores (tcgen05) */
};
enum { MCRT_MAX_SOURCES = 8, MCRT_MAX_CAMERAS = 16 };

/* Status bits reported in mcrt_stats.status_bits. */
enum {
    MCRT_STATUS_EVENT_CAP = 1u, /* a packet reached max_events */
    MCRT_STATUS_TRIAL_CAP = 2u, /* a scattering found no accepted proposal in max_trials */
    MCRT_STATUS_TIMEOUT = 4u,   /* time budget exhausted before the packet pool */
    MCRT_STATUS_DEVICE_TIMEOUT = 8u /* a tensor-core operation did not complete in time; the kernel
                                       stopped and the tallies are incomplete */
};

/* A packet source (paper Sec. 2.2: packets are emitted, then transported). */
typedef struct {
    int32_t type;       /* MCRT_SRC_POINT: isotropic unpolarized point at pos.
                           MCRT_SRC_BEAM: unpolarized plane beam entering the lo_z face
                           along +z (beam_dir = +1) or the hi_z face along -z (-1),
                           uniform over the face.
                           MCRT_SRC_THERMAL: emission alpha_abs B of the grid's
                           emissivity (eq. polarized-rt), cells drawn in proportion to
                           kappa_ext (mean alpha1 - omega) B V, isotropic directions. */
    int32_t beam_dir;
    double luminosity;  /* total power of the source's packets; THERMAL: <= 0 means
                           4 pi sum kappa_ext (mean alpha1 - omega) B V */
    double pos[3];      /* POINT: position, inside the grid box */
    int64_t n_packets;  /* packets of this source; sources take consecutive packet ids */
} mcrt_source;

/* A camera of the two-step imaging (paper Sec. 2.3). */
typedef struct {
    double dir[3];      /* Omega_cam: unit vector from the model toward the observer */
    double center[3];   /* point of the model imaged at the image centre */
    double fov[2];      /* image extent along e_x = phi-hat(Omega), e_y = -theta-hat(Omega) */
    int32_t npix[2];    /* pixels along e_x, e_y */
} mcrt_camera;

/* One transport launch. */
typedef struct {
    int32_t n_sources;
    const mcrt_source *sources;   /* host memory */
    int32_t n_cameras;            /* 0..MCRT_MAX_CAMERAS; 0 skips the step-1 tally */
    const mcrt_camera *cameras;   /* host memory */
    uint32_t seed;                /* Philox key word 0 */
    uint32_t stream;              /* Philox key word 1 (job index in batched launches) */
    int32_t precision;            /* MCRT_FP32 (per-step transport math in FP32) or MCRT_FP64 */
    int32_t accumulate;           /* 0: zero the tallies first; 1: add to the previous launch
                                     (resume: launch the remaining packet ids) */
    int64_t pid_begin, pid_end;   /* packet ids to run; pid_end <= 0 means all ids */
    double roulette_threshold;    /* Russian roulette when I < threshold * I_birth at a
                                     scattering; 0 disables */
    double roulette_survival;     /* survival probability (weight / survival on survival) */
    int64_t max_events;           /* per-packet event cap (emission + segments + scatterings) */
    int32_t max_trials;           /* rejection-sampling trial cap per scattering */
    int32_t block_size;           /* threads per block (multiple of 32, <= 128); 0 = 128 */
    int32_t blocks_per_sm;        /* resident blocks per SM of the persistent grid; 0 = max */
    double time_budget_s;         /* > 0: stop taking new packets after this many seconds
                                     of kernel time and return MCRT_E_TIMEOUT */
    int64_t n_trace;              /* final state of packets with id < n_trace is written */
    double *trace;                /* [n_trace][16]: I,Q,U,V, x,y,z, nx,ny,nz, scatterings,
                                     segments, flag (1 escaped, 2 roulette, 3 event cap,
                                     4 trial cap), I_birth, source, events; host or device;
                                     nullable */
    int32_t optics;               /* MCRT_OPTICS_TABLES: the optics set with
                                     mcrt_set_dust_tables; MCRT_OPTICS_SURROGATE: the
                                     network attached with mcrt_set_surrogate (FP32, one
                                     model, no time budget) */
    int32_t flags;                /* MCRT_FLAG_* */
    int32_t tally_blocks_per_sm;  /* FP32 table rounds: 0 runs each round's transport and tally
                                     kernels one after the other (default); > 0 runs a round's
                                     tally, with this many blocks per SM, beside the next round's
                                     transport, whose blocks per SM are then blocks_per_sm (0 = its
                                     maximum minus 2).  Measured slower on the disk workload. */
} mcrt_launch_desc;

/* Totals of a launch (FP64 sums over packets). */
typedef struct {
    double emitted_energy, escaped_energy, absorbed_energy;
    double roulette_lost, roulette_gain, cap_lost;
    double events, segments, scatterings, emitted, escaped, roulette_killed, cap_hits, trials;
    double kernel_ms;             /* device time of the transport kernel(s) */
    double status_bits;           /* MCRT_STATUS_* bits, as a number */
    double tally_segments;        /* segments that added to the source tally */
    double absorb_segments;       /* segments that added to the absorbed-energy tally */
    /* surrogate launches only (zero otherwise) */
    double mlp_tally_rows;        /* network evaluations for the source tally (segment x camera) */
    double mlp_scatter_rows;      /* network evaluations for rejection trials */
    double mlp_fallback_map;      /* evaluations replaced by the tables: error-map cell above bound */
    double mlp_fallback_realizability; /* ... network matrix not physically realizable */
    double tally_overflow;        /* tally segments done with the tables for want of queue space */
    double envelope_miss;         /* trials whose target exceeded the (widened) envelope */
    double wave_iterations;       /* transport / network rounds of the launch */
    double ms_transport, ms_tally, ms_scatter; /* device time of the rounds' transport,
                                     network-tally and network-scattering kernels */
} mcrt_stats;

/*
 * Create a model: the grid of inverse mean free paths (eq. mfp-matrices, read per
 * cell as in Sec. 2.2) and the grain alignment field (Sec. 2.1).
 *   kappa_abs, kappa_sca  [nz][ny][nx] FP32, 1/length, >= 0
 *   bfield     [nz][ny][nx][3] FP32 field direction (any norm; zero means no
 *              alignment, q_B = 1) or NULL for none; converted once to the grain
 *              quaternion q_B of eq. (grain-quaternion)
 *   emissivity [nz][ny][nx] FP32 Planck function B per cell, or NULL
 *   boundary   MCRT_BOUNDARY_OUTFLOW (packets leaving the box escape) or a combination
 *              of MCRT_BOUNDARY_PERIODIC_X/Y/Z (re-entry on the opposite face along those
 *              axes; step-2 images still cover the box itself)
 *   cuda_stream  cudaStream_t on which this context queues all its work
 * On success *out owns device copies of the grid (32 bytes per cell).
 * Errors: MCRT_E_INVAL for bad sizes or NULL required pointers, MCRT_E_NOMEM,
 * MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_create_grid(mcrt_ctx **out, int32_t nx, int32_t ny, int32_t nz, const double lo[3],
                             const double hi[3], const float *kappa_abs, const float *kappa_sca,
                             const float *bfield, const float *emissivity, int32_t boundary,
                             void *cuda_stream);

/*
 * A statically refined patch of the root grid (Sec. 2: a composite mesh, optionally with
 * static mesh refinement).  The root cells of `box` (root-cell indices i0, j0, k0, i1,
 * j1, k1, half-open, inside the root grid) are replaced by a uniform grid with `factor`
 * cells per root cell along each axis, nx = (i1 - i0) factor and so on.
 *   kappa_abs, kappa_sca  [nz][ny][nx] FP32 of the patch, host or device
 *   bfield, emissivity    as the root grid's: given exactly when the root's are
 */
typedef struct {
    int32_t box[6];
    int32_t factor;  /* 2..16 */
    const float *kappa_abs, *kappa_sca, *bfield, *emissivity;
} mcrt_patch;

/*
 * mcrt_create_grid with static mesh refinement: up to 64 patches (disjoint boxes, one
 * level).  Cells are numbered root first ([z][y][x]), then each patch in order
 * ([z][y][x] within the patch); tallies (mcrt_get_tallies) use that numbering and hold
 * zeros for covered root cells, whose root values are not used.  Packets descend into
 * a patch on entering a covered root cell and return to the root cell beyond the
 * patch face they leave through; step 2 marches through the same cells.  Refined
 * models take Rayleigh, table or dipole optics in single-model launches (FP32 table
 * launches run in rounds with the tally kernel, as on plain grids); batched, surrogate
 * and no-allocation launches refuse them.
 * Errors: as mcrt_create_grid, and MCRT_E_INVAL for overlapping or out-of-range boxes,
 * bad factors, or field/emission arrays present on one level only.
 */
MCRT_API mcrt_status mcrt_create_grid_refined(mcrt_ctx **out, int32_t nx, int32_t ny, int32_t nz, const double lo[3],
                                     const double hi[3], const float *kappa_abs, const float *kappa_sca,
                                     const float *bfield, const float *emissivity, int32_t boundary,
                                     int32_t n_patches, const mcrt_patch *patches, void *cuda_stream);

/*
 * Grain optics (Sec. 2.2: the Mueller matrix and cross sections are user-defined,
 * as analytic forms or tables; App. A: extinction elements alpha_i).
 *   model    MCRT_SCAT_RAYLEIGH: dipole scattering matrix (n_bins, mueller and
 *            bin_weight ignored); MCRT_SCAT_TABLE: tables below.
 *   mueller  [n_bins][n_theta][6] FP32 P11,P12,P22,P33,P34,P44 in the scattering-
 *            plane basis, on scattering angles theta_j = pi j / (n_theta - 1),
 *            interpolated linearly in theta, each bin normalised so that
 *            2 pi int P11 sin(theta) dtheta = 1 (1/sr)
 *   bin_weight [n_bins] FP32 share of the scattering cross section per bin
 *   kext     [n_ktheta][3] FP32 alpha1, alpha2, alpha3 per unit extinction optical
 *            depth at grain-frame angles theta'_j = pi j / (n_ktheta - 1), linear in
 *            theta', in the grain-meridian basis; the extinction matrix is
 *            K = [[a1,a2,0,0],[a2,a1,0,0],[0,0,a1,a3],[0,0,-a3,a1]]
 * Limits: 2 <= n_theta <= 721, 1 <= n_bins <= 32, 2 <= n_ktheta <= 721.
 * Errors: MCRT_E_INVAL, MCRT_E_NOMEM, MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_set_dust_tables(mcrt_ctx *ctx, int32_t model, int32_t n_bins, int32_t n_theta,
                                 const float *mueller, const float *bin_weight, int32_t n_ktheta,
                                 const float *kext);

/*
 * Grain optics of aligned spheroids in the dipole approximation (Sec. 2.1: the dipole
 * approximation; Sec. 3: K from the optical theorem with no phase lag between the
 * dipole excitations, so no U-V term).  The grain's symmetry axis lies along the
 * cell's field (the grain frame of eq. grain-quaternion).
 *   eps_re, eps_im  dielectric function of the grain material, eps_im >= 0, eps != 1
 *   aspect          equatorial over symmetry semi-axis: > 1 oblate, < 1 prolate, 1 a
 *                   sphere (then identical in distribution to MCRT_SCAT_RAYLEIGH)
 *   size_x          size parameter 2 pi a_eff / lambda >= 0 (a_eff: radius of the sphere
 *                   of equal volume), entering through the radiative-reaction correction
 * On the device: depolarization factors L (closed forms of the ellipsoid integral),
 * polarizabilities alpha_j = (eps-1)/(3(1+L_j(eps-1))) a_eff^3 with the radiative
 * reaction alpha'_j = alpha_j / (1 - (2i/3) x^3 alpha_j / a_eff^3), and per axis the
 * cross sections C_ext = 4 pi k Im alpha', C_sca = (8 pi/3) k^4 |alpha'|^2,
 * C_abs = C_ext - C_sca.  The grid's kappa_abs and kappa_sca are read as the
 * orientation-averaged opacities; along a direction n the extinction matrix is
 *   K = kappa_abs Khat_abs(n) + kappa_sca Khat_sca(n)
 * with each dichroic part relative to its orientation average, the scattering matrix
 * Z = kappa_sca Zhat with Zhat from the Jones matrix of the induced dipole.  Packets
 * sample scatterings at the unpolarized rate along n and take the weight
 * (K_sca X)_0 / (K_sca,11 (Z X)_0) at each scattering.
 * Replaces any optics set before.  Not accepted by batched launches, the surrogate
 * (which learns tables) or mcrt_launch_packets_noalloc.
 * Errors: MCRT_E_INVAL (bad parameters), MCRT_E_NOMEM, MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_set_dust_dipole(mcrt_ctx *ctx, double eps_re, double eps_im, double aspect,
                                          double size_x);

/*
 * The constants mcrt_set_dust_dipole computes on the device, for checks:
 *   out [16] host: L_perp, L_par, Re/Im alpha'_perp, Re/Im alpha'_par (per a_eff^3),
 *        Qext_perp, Qext_par, Qsca_perp, Qsca_par, Qabs_perp, Qabs_par (efficiencies,
 *        cross section over pi a_eff^2), Re/Im rho = alpha'_par / alpha'_perp,
 *        zn (Zhat scale, 1/sr), env (rejection envelope of (Zhat X)_0 / I, 1/sr)
 * Errors: MCRT_E_INVAL, MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_dipole_constants(double eps_re, double eps_im, double aspect, double size_x, double *out);

/*
 * Step 1 of the two-step scheme (Sec. 2.2, 2.3): emit and transport packets,
 * accumulating per model the absorbed energy per cell and the source tally
 *   T_c[cell] = sum over path segments of Z(Omega_c; Omega_pp) int I_pp ds
 * (eq. scat-disc-sum, path-integral estimator, FP64) for each camera c.
 * With n_models > 1 the same description runs for every model in one persistent
 * launch (see the batch calls below), model m using Philox stream desc->stream + m.
 * out_stats (nullable, host) receives the totals summed over models after the
 * stream has been synchronized.
 * Errors: MCRT_E_INVAL, MCRT_E_STATE (tables not set), MCRT_E_NOMEM, MCRT_E_CUDA,
 * MCRT_E_EVENT_CAP (results valid, some packets were cut), MCRT_E_TIMEOUT.
 */
MCRT_API mcrt_status mcrt_launch_packets(mcrt_ctx *const *models, int32_t n_models, const mcrt_launch_desc *desc,
                                mcrt_stats *out_stats);

/*
 * Step 2 (Sec. 2.3, App. A): ray-march every pixel of camera `camera` of the last
 * launch from the far side of the grid toward the observer, integrating
 * dX/dtau = -K X + alpha_abs B + S cell by cell with S = omega / V * T_c.
 *   out  [4][npix_y][npix_x] FP64 Stokes image (I,Q,U,V) in the basis of Omega_cam;
 *        host or device.
 * Errors: MCRT_E_INVAL (camera out of range), MCRT_E_STATE (no launch yet),
 * MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_image_stokes(mcrt_ctx *ctx, int32_t camera, double *out);

/*
 * Copy the step-1 tallies of the last launch: source [ncell][n_cameras][4] FP64
 * (length-weighted Stokes sums T_c, camera basis) and absorbed [ncell] FP64.  Either
 * pointer may be NULL.  Host or device.
 */
MCRT_API mcrt_status mcrt_get_tallies(mcrt_ctx *ctx, double *source, double *absorbed);

/*
 * Throughput of the FP64 reductions the step-1 tallies are made of, on the current
 * device: n_ops additions into a zeroed device buffer of `bytes` bytes at spread
 * positions (a multiplicative hash of the op index).
 *   kind 0: scalar FP64 atomic adds without return value (one double per op)
 *   kind 1: 256-byte bulk reduce-adds of FP64 rows from shared memory (one row per op)
 * One untimed launch, then *ms_out = the CUDA-event time of one launch of n_ops ops.
 * Errors: MCRT_E_INVAL (kind, or bytes < 256), MCRT_E_NOMEM, MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_microbench(int32_t kind, uint64_t bytes, uint64_t n_ops, double *ms_out);

/*
 * Replace the step-1 tallies of the last launch (layouts as in mcrt_get_tallies), e.g.
 * with their sum over ranks that each ran a share of the packet ids: step 2 is linear
 * in the tallies (Sec. 2.3), so images of the summed tallies are the images of all
 * packets.  Either pointer may be NULL (that tally is kept).  Host or device; the
 * caller keeps ownership.
 * Errors: MCRT_E_INVAL, MCRT_E_STATE (no launch yet), MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_set_tallies(mcrt_ctx *ctx, const double *source, const double *absorbed);

/*
 * Device addresses of the step-1 tallies of the last launch, owned by the library
 * (layouts as in mcrt_get_tallies), for collectives that work on them in place: the
 * sum over ranks of a sharded run (Sec. 2.3: step 2 is linear in the tallies) can run
 * directly on these buffers instead of a copy out and back.  Writes through them
 * replace the tallies as mcrt_set_tallies does.  The caller orders its work on them
 * after the launch and before the next call that uses ctx (the launch has
 * synchronized ctx's stream when it returned with out_stats; otherwise synchronize
 * that stream first).  Valid until the next launch or mcrt_destroy of ctx.  Any
 * output pointer may be NULL; source is NULL (count 0) when the launch had no camera.
 * Errors: MCRT_E_INVAL, MCRT_E_STATE (no launch yet).
 */
MCRT_API mcrt_status mcrt_tally_buffers(mcrt_ctx *ctx, double **source, double **absorbed, int64_t *source_count,
                                        int64_t *absorbed_count);

/* Release the context and its device memory; NULL is accepted. */
MCRT_API mcrt_status mcrt_destroy(mcrt_ctx *ctx);

/* Last error message of ctx, or of the calling thread's context-less calls when
 * ctx is NULL.  Never NULL; owned by the library. */
MCRT_API const char *mcrt_last_error(const mcrt_ctx *ctx);

/*
 * Diagnostics: evaluate one device building block on n inputs (host buffers),
 * for unit tests against the CPU reference.  fn selects the block; in/out layouts:
 *   0 Philox4x32-10: in [n][6] (ctr0..3, key0, key1 as doubles) -> out [n][4]
 *   1 grain quaternion rotation: in [n][7] (bx,by,bz, vx,vy,vz, unused) ->
 *     out [n][8] (q0..q3, v in the grain frame)
 *   2 eta rotation into the grain-meridian basis: in [n][10] (bx,by,bz, nx,ny,nz,
 *     I,Q,U,V) -> out [n][6] (I,Q,U,V in that basis, cos theta', unused)
 *   3 in-cell solution: in [n][12] (I,Q,U,V, alpha1,alpha2,alpha3, S1..S4, dtau)
 *     -> out [n][4]
 *   4 path integral: in [n][8] (I,Q,U,V, a, alpha2, alpha3, dtau) -> out [n][4]
 *   5 scattering-matrix transfer: in [n][16] (I,Q,U,V, n, n2, P11,P12,P22,P33,P34,
 *     P44) -> out [n][4] (Stokes in the basis of n2)
 *   6 dipole-spheroid scattering: in [n][16] (I,Q,U,V, n, n2, axis, Re rho, Im rho,
 *     zn) -> out [n][4] (Zhat X in the basis of n2)
 *   7 dipole-spheroid extinction: in [n][8] (ca_perp, ca_par, cs_perp, cs_par,
 *     kappa_abs/kappa_ext, kappa_sca/kappa_ext, cos theta', unused) with ca, cs the
 *     absorption and scattering cross sections over their orientation averages ->
 *     out [n][4] (alpha1, alpha2, s11, s12: K and its scattering part per unit
 *     kappa_ext, first row, grain-meridian basis)
 * precision selects the FP32 or FP64 instantiation.
 */
MCRT_API mcrt_status mcrt_unit_eval(int32_t fn, int32_t precision, int64_t n, const double *in, double *out);

/*
 * Batched launches (many models, e.g. one grid per wavelength, in one persistent
 * launch).  The paper runs one model per launch; batching is a throughput layer
 * over the same transport.  Job m of a batch is model m with Philox stream
 * desc->stream + m, so its tallies equal those of a single launch of that model
 * with that stream, up to the order of floating-point additions.
 *
 * mcrt_batch_create copies the description, sizes every model's tallies, builds
 * the job table and captures one CUDA graph holding: zeroing of all tallies, the
 * transport kernel over all jobs, and step 2 for every (model, camera) into
 * batch-owned image buffers.  All models need the same scattering model; traces,
 * accumulation and packet-id ranges are not available in a batch.  Errors of the
 * batch calls are read with mcrt_last_error(NULL).
 * mcrt_batch_run replays the graph with `seed` (Philox key word 0) on the batch's
 * own stream; out_stats (nullable) holds the totals over all jobs after the run.
 * mcrt_batch_tune runs short trial launches of packets_per_job packets per job for
 * block sizes 64/96/128, full or one-less resident blocks per SM, and job-major or
 * interleaved packet order, keeps the fastest and re-captures the graph; the
 * trials overwrite the models' tallies.  report (nullable) lists the trials.
 * mcrt_batch_images copies all images, [model][camera][4][ny][nx] FP64 (each
 * camera with its own npix), to host or device memory.
 * After a run, mcrt_get_tallies and mcrt_image_stokes work on each model as after
 * a single launch.
 */
typedef struct mcrt_batch mcrt_batch;

typedef struct {
    int32_t n, best;
    int32_t block_size[16], blocks_per_sm[16], interleave[16];
    double events_per_s[16];
} mcrt_tune_report;

MCRT_API mcrt_status mcrt_batch_create(mcrt_batch **out, mcrt_ctx *const *models, int32_t n_models,
                                       const mcrt_launch_desc *desc);
MCRT_API mcrt_status mcrt_batch_run(mcrt_batch *batch, uint32_t seed, mcrt_stats *out_stats);
MCRT_API mcrt_status mcrt_batch_tune(mcrt_batch *batch, int64_t packets_per_job, mcrt_tune_report *report);
MCRT_API mcrt_status mcrt_batch_images(mcrt_batch *batch, double *out);
MCRT_API mcrt_status mcrt_batch_destroy(mcrt_batch *batch); /* NULL-safe */

/*
 * Learned surrogate of the grain optics (Sec. 2.2 lets the Mueller matrix come from
 * analytic forms, tables or neural networks; Sec. 4 proposes networks for
 * multi-dimensional grain optics).  The network maps u = (n_i[3], n_s[3], s) --
 * incident and scattered directions in the grain frame and s in [-1, 1], the
 * position of ln x between the first and last tabulated size parameter -- to 20
 * outputs for the 4x4 scattering matrix M in the scattering-plane basis (Sec. 2.1;
 * the rotations into and out of the plane are applied exactly by the kernels): ln M11
 * (M in 1/sr) and the other 15 entries divided by M11 (row-major, (0,0) left out);
 * then alpha1..3 at the polar angle of n_i and ln N(s), N(s) = max P11 over the
 * scattering angle.  Layers 16 (7 inputs, zero padded) -> 128 -> 128 -> 128
 * -> 128 -> 24 (20 used), SiLU; BF16 weights and activations with FP32 accumulation
 * on the tensor cores; FP32 master weights and Adam.
 *   create: copies the tables of `optics` (MCRT_SCAT_TABLE) as the label source and
 *           initialises the weights from `seed`.
 *   train:  n_steps Adam steps on fresh batches of `batch` samples generated on the
 *           GPU from the tables (uniform directions, uniform s); learning rate `lr`
 *           with cosine decay; loss_history (host, nullable) gets the mean squared
 *           error of each step.  One step is captured once as a CUDA graph on the
 *           surrogate's own stream and replayed n_steps times; the call allocates
 *           20 bytes of device memory per step (losses, schedule) for its duration
 *           and returns when the steps have run.
 *   eval:   outputs [n][20] (host or device) for inputs [n][7].
 *   labels: the training targets [n][20] of inputs [n][7].
 *   grad:   loss sum_b sum_o w_o (y - t)^2 / (20 n) and its gradient with respect
 *           to every parameter (layout of params) for given inputs and targets
 *           [n][20]; loss_weights [20] nullable (ones).
 *   params: get (set = 0) or set (set = 1) the FP32 parameters, per layer W[out][in]
 *           then b[out]; mcrt_surrogate_param_count() of them.
 * Errors of these calls are read with mcrt_last_error(NULL).
 */
typedef struct mcrt_surrogate mcrt_surrogate;

MCRT_API mcrt_status mcrt_surrogate_create(mcrt_surrogate **out, const mcrt_ctx *optics, uint32_t seed);
MCRT_API mcrt_status mcrt_surrogate_train(mcrt_surrogate *s, int64_t n_steps, int32_t batch, double lr,
                                          double *loss_history);
MCRT_API mcrt_status mcrt_surrogate_eval(mcrt_surrogate *s, int64_t n, const float *inputs, float *outputs);
MCRT_API mcrt_status mcrt_surrogate_labels(mcrt_surrogate *s, int64_t n, const float *inputs, float *labels);
MCRT_API mcrt_status mcrt_surrogate_grad(mcrt_surrogate *s, int64_t n, const float *inputs, const float *targets,
                                         const float *loss_weights, float *grads, double *loss);
/*
 * The FP32 mode of mcrt_surrogate_grad, for checking the backward pass at FP32
 * accuracy: the same loss and gradient with FP32 operands, activations and gradients
 * throughout (FP32 FMA on the CUDA cores, no BF16 rounding; the inputs enter as FP32
 * without high and low parts) and the FP32 master weights as they are.  Allocates
 * its activation buffers for the duration of the call.  Same arguments and errors.
 */
MCRT_API mcrt_status mcrt_surrogate_grad_fp32(mcrt_surrogate *s, int64_t n, const float *inputs,
                                              const float *targets, const float *loss_weights, float *grads,
                                              double *loss);
MCRT_API mcrt_status mcrt_surrogate_params(mcrt_surrogate *s, float *params, int32_t set);
MCRT_API int64_t mcrt_surrogate_param_count(void);
MCRT_API mcrt_status mcrt_surrogate_destroy(mcrt_surrogate *s); /* NULL-safe */

/*
 * Error map of the current network: n_samples inputs drawn uniformly (directions on
 * the sphere, s in [-1, 1]) are evaluated by the network and by the tables; each of
 * the 8^4 cells of (cos theta_i, cos theta_s, delta phi = phi_s - phi_i in [0, 2 pi),
 * s), 8 equal bins per coordinate, index ((i*8 + j)*8 + k)*8 + l, gets the largest
 * error max_e |M_net,e - M_e| / M11 over its samples (relative to the true M11).  map (host or device,
 * [4096] FP32, nullable) receives it.  Training or setting parameters invalidates it.
 */
MCRT_API mcrt_status mcrt_surrogate_error_map(mcrt_surrogate *s, int64_t n_samples, float *map);

/*
 * Evaluation on a chosen tensor-core engine: MCRT_ENGINE_MMA_SYNC (warp-level
 * mma.sync m16n8k16, the engine of mcrt_surrogate_eval) or MCRT_ENGINE_TCGEN05 (5th-
 * generation tensor cores: tcgen05.mma with the accumulator in tensor memory, 128
 * rows per CTA).  Same network, inputs and outputs as mcrt_surrogate_eval; the two
 * engines differ only in the order of FP32 additions.  MCRT_E_TIMEOUT if a
 * tensor-core operation did not complete within 2 s (the kernel then stops).
 */
enum { MCRT_ENGINE_MMA_SYNC = 0, MCRT_ENGINE_TCGEN05 = 1 };
MCRT_API mcrt_status mcrt_surrogate_eval_engine(mcrt_surrogate *s, int32_t engine, int64_t n, const float *inputs,
                                                float *outputs);

/*
 * Attach the network to a model for launches with desc->optics =
 * MCRT_OPTICS_SURROGATE.  The model needs MCRT_SCAT_TABLE optics: they remain the
 * fallback.  Copies the network (BF16 weights, FP32 biases), its error map (computed
 * with 2^22 samples if not yet done) and the extinction elements alpha1..3 that the
 * network gives on the model's n_ktheta angles (averaged over 16 scattered
 * directions and sizes; rows with alpha1 <= 0 or |alpha2| >= alpha1 keep the table's
 * row).  In surrogate launches
 *  - each tallying segment and camera evaluates the network at the grain-frame
 *    directions of the packet and the camera and at the size s of the packet's
 *    current flight (a grain-size bin drawn with the bin weights at every emission
 *    and scattering, so that the tally averages to the bin mixture);
 *  - each rejection trial evaluates it at the proposed direction and the size bin
 *    drawn for the scattering; the proposals and the envelope are the tables' (the
 *    envelope widened by 5%);
 *  - an evaluation uses the tables instead when its error-map cell exceeds `bound`
 *    (relative to M11) or when the network's matrix fails the realizability check
 *    M11^2 >= M12^2 + M13^2 + M14^2 and M11^2 >= M21^2 + M31^2 + M41^2 by more than 5%
 *    in those squared norms (smaller excesses are scaled back onto the boundary);
 *  - extinction and emission use the distilled alpha1..3; step-2 images of such a
 *    launch too.
 * The surrogate may be destroyed afterwards.  bound = 0 means 0.05.  bound < 0 is a
 * validation mode: the surrogate path's kernels run but every evaluation takes the
 * tables, the envelope is not widened and extinction uses the tables' alpha, so the
 * packets follow the table path's trajectories exactly (same random numbers and
 * decisions, up to rounding); only the tally differs, sampling one size bin per flight
 * instead of the bin mixture, with the same expectation.
 * Errors: MCRT_E_INVAL, MCRT_E_STATE (no MCRT_SCAT_TABLE optics), MCRT_E_NOMEM,
 * MCRT_E_CUDA.
 */
MCRT_API mcrt_status mcrt_set_surrogate(mcrt_ctx *ctx, mcrt_surrogate *s, double bound);

/*
 * Transport without allocation.  The paper has no counterpart to this entry point;
 * it exists for callers that cannot allocate device memory themselves or through
 * this library: code running inside another framework's memory pool or under a
 * fixed memory plan, or a process whose allocator must not be touched after
 * start-up.  mcrt_launch_packets_noalloc performs the same step-1 transport as
 * mcrt_launch_packets, but
 *  - every input and output is caller-owned DEVICE memory passed in `prob`
 *    (kappa_abs, kappa_sca, bfield, the optics tables, and the outputs source
 *    [ncell][n_cameras][4] FP64 and absorbed [ncell] FP64, zeroed by the call unless
 *    desc->accumulate is set); desc->trace, if used, must be device memory too;
 *  - its scratch (cell records with the grain quaternions, prepared tables, the
 *    packet counter and the launch totals) lives in one static device array of
 *    about 4.3 MB that the library image carries; every GPU that loads the library
 *    holds that array until the process exits;
 *  - it calls no cudaMalloc, cudaFree or other allocating routine.
 * Limits (MCRT_E_INVAL beyond them): at most MCRT_NOALLOC_MAX_CELLS cells,
 * MCRT_NOALLOC_MAX_BINS grain bins, MCRT_NOALLOC_MAX_THETA angles per table; point
 * and beam sources only (thermal sources need per-cell emission scratch).
 * Every call looks up the array's device address on the current device (the first
 * lookup on a device can load the library's device code); make the first call on a
 * device before any stream capture.  Inputs, outputs and the trace must be memory of
 * the current device (or managed memory); memory of another GPU is refused.
 * All calls share the one array, so calls whose GPU work overlaps (different
 * streams or host threads without ordering between them) race on it; each call
 * clears what must start at zero.  Work runs on prob->cuda_stream, and the call
 * synchronizes that stream three times before it returns: after copying the kext
 * rows to the host for their checks, after the set-up kernels' check of the grids,
 * and after the transport, to read the launch's status word.  It therefore blocks
 * the calling host thread until all work queued on the stream has finished.  The
 * status is read whether or not out_stats is given: MCRT_E_EVENT_CAP or
 * MCRT_E_TIMEOUT report packets cut by the caps or the time budget (the outputs hold
 * the rest).  out_stats (nullable, host) receives the launch totals.
 */
enum { MCRT_NOALLOC_MAX_CELLS = 131072, MCRT_NOALLOC_MAX_BINS = 8, MCRT_NOALLOC_MAX_THETA = 181 };

typedef struct {
    int32_t nx, ny, nz;
    double lo[3], hi[3];
    const float *kappa_abs, *kappa_sca; /* device, [nz][ny][nx] */
    const float *bfield;                /* device, [nz][ny][nx][3], or NULL */
    int32_t model, n_bins, n_theta;     /* as in mcrt_set_dust_tables */
    const float *mueller, *bin_weight;  /* device (MCRT_SCAT_TABLE only) */
    int32_t n_ktheta;
    const float *kext;                  /* device, [n_ktheta][3] */
    double *source;                     /* device output, [ncell][n_cameras][4] */
    double *absorbed;                   /* device output, [ncell] */
    void *cuda_stream;
} mcrt_noalloc_problem;

MCRT_API mcrt_status mcrt_launch_packets_noalloc(const mcrt_noalloc_problem *prob, const mcrt_launch_desc *desc,
                                                 mcrt_stats *out_stats);

#ifdef __cplusplus
}
#endif

#endif /* MCRT_H */
