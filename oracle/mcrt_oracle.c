/*
 * mcrt_oracle.c -- plain, slow, FP64 CPU reference of the polarized Monte-Carlo
 * transport and two-step imaging of Kratos-polrad (arXiv:2512.01283).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the tests, the package smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the CUDA
 * path: every formula is written here a second time, directly from the paper, in
 * the paper's order and notation, with no blocking or fusion.
 *
 * Passages followed (paper sections / equations):
 *   Sec. 2.1  eq. (grain-quaternion)   q_B from (theta_B, phi_B)
 *             eq. (vector-transform)   (0, n_GF) = q_B^* (0, n) q_B
 *             Stokes basis theta-hat, phi-hat; Q > 0 along theta-hat
 *             eq. (rotation-angle), eq. (stokes-rotation): basis rotation by eta.
 *             Here the rotation is done by projecting the coherency matrix onto
 *             the new basis vectors, which needs no angle convention; the signed
 *             eta of the CUDA path is checked against it.
 *   Sec. 2.2  eq. (polarized-rt), eq. (mfp-matrices), eq. (scattering-source);
 *             exponential scattering optical depth drawn at emission and after
 *             each scattering; cell-to-cell traversal; rejection sampling of the
 *             polarization-aware differential cross section.
 *   Sec. 2.3  eq. (scat-disc-sum): every path segment adds Z(Omega_cam;Omega_pp) I_pp
 *             to S(Omega_cam, x); step 2 ray-marches toward the camera with the
 *             same cell-by-cell analytic integration.
 *   App. A    analytic in-cell solution (the printed I_s..V_s and cosh/sinh,
 *             cos/sin solution; the extinction matrix is taken as the one that
 *             solution solves, K = [[a1,a2,0,0],[a2,a1,0,0],[0,0,a1,a3],[0,0,-a3,a1]]).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - Random numbers: Philox4x32-10 (Salmon et al. 2011), key = (seed, stream),
 *     counter = (pid_lo, pid_hi, event, slot); u = ((x >> 8) | 1) * 2^-24.
 *   - Scattering optical depth is sampled with the scalar kappa_sca; between
 *     events the Stokes vector is attenuated by K - omega*1 (absorption and all
 *     dichroism) and the absorbed I is tallied.
 *   - The step-1 tally uses the exact path integral of the attenuated Stokes
 *     vector over the segment (length units); step 2 uses S = omega/V * tally.
 *   - Rayleigh: isotropic proposal in the grain frame with envelope 2*max Z11.
 *     Tables: proposal from a piecewise-constant envelope of P11 over the
 *     tabulated scattering-angle intervals, azimuth uniform about n.
 *   - Aligned spheroids (Sec. 2.1 and Sec. 3: dipole approximation, K from the
 *     optical theorem with no phase lag, so no U-V term): polarizability tensor of
 *     a spheroid with the radiative-reaction correction; the scattered field is the
 *     transverse part of the induced dipole (a Jones matrix, applied to the
 *     coherency matrix).  The cell's kappa_abs and kappa_sca are the orientation-
 *     averaged opacities; the dichroic parts of K are relative to those averages.
 *     Scatterings are sampled along n at the unpolarized rate s11 kappa_ext
 *     (direction-dependent) and the packet is attenuated by K - s11 kappa_ext 1; at a
 *     scattering the new Stokes vector is Z X (K_sca X)_0 / (s11 (Z X)_0) (the weight
 *     that keeps the estimator unbiased when the scattering cross section depends on
 *     direction and polarization).  Isotropic proposal, envelope max(1,|rho|^2) zn.
 *
 * All arithmetic is double precision.  Tallies from several threads are added
 * with compare-and-swap; with one thread the results are deterministic.
 */
#define _POSIX_C_SOURCE 199309L
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------- */
/* Problem description (mirrored field by field in oracle.py).               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t type;       /* 0 point, 1 plane beam, 2 thermal emission of the grid */
    int32_t beam_dir;   /* beam: +1 travels +z from the lo_z face, -1 travels -z from hi_z */
    double luminosity;  /* total power of this source; thermal: <= 0 means computed */
    double pos[3];      /* point source position */
    int64_t n_packets;
} orc_source;

typedef struct {
    double dir[3];      /* unit vector pointing from the model toward the observer */
    double center[3];   /* image centre */
    double fov[2];      /* image extent along e_x, e_y (length units) */
    int32_t npix[2];    /* nx, ny */
} orc_camera;

/* A statically refined patch: the root cells of `box` (root-cell indices i0, j0, k0,
 * i1, j1, k1, half-open) are replaced by a uniform grid of `factor` cells per root cell
 * along each axis, with its own arrays [nz][ny][nx] (bfield and emissivity as the
 * root's: NULL when the root's are). */
typedef struct {
    int32_t box[6];
    int32_t factor;
    const float *kappa_abs, *kappa_sca, *bfield, *emissivity;
} orc_patch;

typedef struct {
    int32_t n[3];
    double lo[3], hi[3];
    const float *kappa_abs;   /* [nz][ny][nx], 1/length */
    const float *kappa_sca;   /* [nz][ny][nx], 1/length */
    const float *bfield;      /* [nz][ny][nx][3] or NULL (no alignment) */
    const float *emissivity;  /* [nz][ny][nx] B_lambda(T) or NULL */
    int32_t scat_model;       /* 0 Rayleigh (analytic dipole), 1 tables, 2 aligned dipole spheroids */
    int32_t n_bins, n_theta;
    const float *mueller;     /* [n_bins][n_theta][6] P11,P12,P22,P33,P34,P44 */
    const float *bin_weight;  /* [n_bins] */
    int32_t n_ktheta;
    const float *kext;        /* [n_ktheta][3] alpha1, alpha2, alpha3 on theta' in [0, pi] */
    int32_t n_sources;
    const orc_source *sources;
    int32_t n_cam;
    const orc_camera *cams;
    uint32_t seed, stream;
    int64_t pid_begin, pid_end;
    double roulette_threshold, roulette_survival;
    int64_t max_events;
    int32_t max_trials;
    int32_t n_threads;
    int64_t n_trace;
    int32_t periodic;         /* bit a set: axis a is periodic (a packet leaving the box there re-enters
                                 on the opposite face), else packets leaving escape */
    double eps_re, eps_im;    /* scat_model 2: dielectric function of the grain material */
    double aspect;            /* scat_model 2: equatorial over symmetry semi-axis (> 1 oblate) */
    double size_x;            /* scat_model 2: size parameter 2 pi a_eff / lambda */
    int32_t n_patches;        /* static mesh refinement: patches of the root grid (one level,
                                 disjoint boxes); the root arrays' values in covered cells
                                 are not used */
    const orc_patch *patches;
} orc_problem;

typedef struct {
    double *S;          /* [ncell][n_cam][4] path-integral tally, caller zeroes */
    double *absorbed;   /* [ncell] */
    double *trace;      /* [n_trace][16] final packet states, or NULL */
    double stats[16];
} orc_result;

enum {
    ST_EMITTED_E = 0, ST_ESCAPED_E, ST_ABSORBED_E, ST_ROULETTE_LOST, ST_ROULETTE_GAIN,
    ST_CAP_LOST, ST_EVENTS, ST_SEGMENTS, ST_SCATTERS, ST_EMITTED_N, ST_ESCAPED_N,
    ST_KILLED_N, ST_CAP_N, ST_TRIALS, ST_STATUS, ST_SPARE
};

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw (SC'11), Sec. 5.                */
/* ------------------------------------------------------------------------- */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_uniform(uint32_t x)
{
    return (double)((x >> 8) | 1u) * (1.0 / 16777216.0);
}

/* Four uniforms of (pid, event, slot). */
static void draw4(const orc_problem *P, int64_t pid, uint32_t event, uint32_t slot, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)((uint64_t)pid & 0xffffffffu), (uint32_t)((uint64_t)pid >> 32), event, slot};
    uint32_t key[2] = {P->seed, P->stream};
    uint32_t x[4];
    orc_philox(ctr, key, x);
    for (int i = 0; i < 4; ++i) u[i] = orc_uniform(x[i]);
}

/* ------------------------------------------------------------------------- */
/* Vectors and Hamilton quaternions (Sec. 2.1).                              */
/* ------------------------------------------------------------------------- */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3])
{
    double x = a[1] * b[2] - a[2] * b[1];
    double y = a[2] * b[0] - a[0] * b[2];
    double z = a[0] * b[1] - a[1] * b[0];
    c[0] = x; c[1] = y; c[2] = z;
}

/* Hamilton product with i^2 = j^2 = k^2 = ijk = -1. */
static void qmul(const double a[4], const double b[4], double c[4])
{
    double r0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double r1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double r2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double r3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    c[0] = r0; c[1] = r1; c[2] = r2; c[3] = r3;
}

/* eq. (grain-quaternion): q_B from the field direction angles (theta_B, phi_B);
 * phi_B = 0 when B is along z, q_B = 1 when B = 0. */
void orc_grain_quaternion(double bx, double by, double bz, double q[4])
{
    double b = sqrt(bx * bx + by * by + bz * bz);
    if (b == 0.0) {
        q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
        return;
    }
    double c = bz / b;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double thetaB = acos(c);
    double phiB = (bx == 0.0 && by == 0.0) ? 0.0 : atan2(by, bx);
    q[0] = cos(phiB / 2) * cos(thetaB / 2);
    q[1] = -sin(phiB / 2) * sin(thetaB / 2);
    q[2] = cos(phiB / 2) * sin(thetaB / 2);
    q[3] = sin(phiB / 2) * cos(thetaB / 2);
}

/* eq. (vector-transform): (0, v_GF) = q^* (0, v) q. */
void orc_to_grain(const double q[4], const double v[3], double out[3])
{
    double qc[4] = {q[0], -q[1], -q[2], -q[3]};
    double pv[4] = {0.0, v[0], v[1], v[2]};
    double t[4], r[4];
    qmul(qc, pv, t);
    qmul(t, q, r);
    out[0] = r[1]; out[1] = r[2]; out[2] = r[3];
}

/* Inverse of eq. (vector-transform): (0, v) = q (0, v_GF) q^*. */
void orc_to_lab(const double q[4], const double v[3], double out[3])
{
    double qc[4] = {q[0], -q[1], -q[2], -q[3]};
    double pv[4] = {0.0, v[0], v[1], v[2]};
    double t[4], r[4];
    qmul(q, pv, t);
    qmul(t, qc, r);
    out[0] = r[1]; out[1] = r[2]; out[2] = r[3];
}

/* Sec. 2.1 Stokes reference basis for light travelling along n = (theta, phi):
 * theta-hat = (cos t cos p, cos t sin p, -sin t), phi-hat = (-sin p, cos p, 0);
 * at the poles phi = 0. */
void orc_stokes_basis(const double n[3], double th[3], double ph[3])
{
    double c = n[2];
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double t = acos(c);
    double p = (n[0] == 0.0 && n[1] == 0.0) ? 0.0 : atan2(n[1], n[0]);
    th[0] = cos(t) * cos(p); th[1] = cos(t) * sin(p); th[2] = -sin(t);
    ph[0] = -sin(p); ph[1] = cos(p); ph[2] = 0.0;
}

/* Re-express a Stokes vector given in the basis (a1, a2) in the basis (b1, b2),
 * both orthonormal and perpendicular to the propagation direction.  The field
 * components transform as E_b = T E_a with T_jk = b_j . a_k; the coherency matrix
 * C = <E E^dagger> = 1/2 [[I+Q, U+iV], [U-iV, I-Q]] transforms as T C T^T.  This is
 * the explicit projection behind eq. (stokes-rotation). */
void orc_change_basis(const double X[4], const double a1[3], const double a2[3],
                      const double b1[3], const double b2[3], double out[4])
{
    double T[2][2] = {{dot3(b1, a1), dot3(b1, a2)}, {dot3(b2, a1), dot3(b2, a2)}};
    double complex C[2][2];
    C[0][0] = 0.5 * (X[0] + X[1]);
    C[1][1] = 0.5 * (X[0] - X[1]);
    C[0][1] = 0.5 * (X[2] + I * X[3]);
    C[1][0] = 0.5 * (X[2] - I * X[3]);
    double complex D[2][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) {
            double complex s = 0.0;
            for (int l = 0; l < 2; ++l)
                for (int m = 0; m < 2; ++m) s += T[j][l] * C[l][m] * T[k][m];
            D[j][k] = s;
        }
    out[0] = creal(D[0][0] + D[1][1]);
    out[1] = creal(D[0][0] - D[1][1]);
    out[2] = 2.0 * creal(D[0][1]);
    out[3] = 2.0 * cimag(D[0][1]);
}

/* ------------------------------------------------------------------------- */
/* App. A: analytic solution inside one cell.                                */
/* ------------------------------------------------------------------------- */

/* The printed solution with source (S1..S4) per unit extinction optical depth,
 * entering Stokes X0 and cell optical depth dtau. */
void orc_cell_solution(const double X0[4], double alpha1, double alpha2, double alpha3,
                       const double S[4], double dtau, double out[4])
{
    double Is = (alpha1 * S[0] - alpha2 * S[1]) / (alpha1 * alpha1 - alpha2 * alpha2);
    double Qs = (alpha1 * S[1] - alpha2 * S[0]) / (alpha1 * alpha1 - alpha2 * alpha2);
    double Us = (alpha1 * S[2] - alpha3 * S[3]) / (alpha1 * alpha1 + alpha3 * alpha3);
    double Vs = (alpha1 * S[3] + alpha3 * S[2]) / (alpha1 * alpha1 + alpha3 * alpha3);
    double e = exp(-alpha1 * dtau);
    double ch = cosh(-alpha2 * dtau), sh = sinh(-alpha2 * dtau);
    double co = cos(-alpha3 * dtau), si = sin(-alpha3 * dtau);
    out[0] = Is + (X0[0] - Is) * e * ch + (X0[1] - Qs) * e * sh;
    out[1] = Qs + (X0[0] - Is) * e * sh + (X0[1] - Qs) * e * ch;
    out[2] = Us + (X0[2] - Us) * e * co + (X0[3] - Vs) * e * si;
    out[3] = Vs - (X0[2] - Us) * e * si + (X0[3] - Vs) * e * co;
}

/* App. A with S = 0 and diagonal rate a (= alpha1 - omega in step 1). */
void orc_attenuate(const double X0[4], double a, double alpha2, double alpha3, double dtau, double out[4])
{
    double e = exp(-a * dtau);
    double ch = cosh(-alpha2 * dtau), sh = sinh(-alpha2 * dtau);
    double co = cos(-alpha3 * dtau), si = sin(-alpha3 * dtau);
    out[0] = X0[0] * e * ch + X0[1] * e * sh;
    out[1] = X0[0] * e * sh + X0[1] * e * ch;
    out[2] = X0[2] * e * co + X0[3] * e * si;
    out[3] = -X0[2] * e * si + X0[3] * e * co;
}

/* Integral over t in [0, dtau] of exp(-M t) X0 with M = [[a,a2,0,0],[a2,a,0,0],
 * [0,0,a,a3],[0,0,-a3,a]], from the eigen-decomposition of the two blocks:
 * I+Q and I-Q decay at a+a2 and a-a2, U+iV at a-i a3; int_0^T e^{-z t} dt =
 * (1 - e^{-z T})/z, equal to T when z = 0. */
static double complex decay_integral(double complex z, double T)
{
    if (z == 0.0) return T;
    /* 1 - e^{-w} for w = x + i y, written with expm1 and 1 - cos y = 2 sin^2(y/2)
     * so that small |w| keeps full relative precision */
    double x = creal(z) * T, y = cimag(z) * T;
    double s = sin(0.5 * y);
    double re = -expm1(-x) + 2.0 * exp(-x) * s * s;
    double im = exp(-x) * sin(y);
    return (re + I * im) / z;
}

void orc_segment_integral(const double X0[4], double a, double alpha2, double alpha3, double dtau, double out[4])
{
    double p = creal(decay_integral(a + alpha2, dtau)) * (X0[0] + X0[1]);
    double m = creal(decay_integral(a - alpha2, dtau)) * (X0[0] - X0[1]);
    double complex w = decay_integral(a - I * alpha3, dtau) * (X0[2] + I * X0[3]);
    out[0] = 0.5 * (p + m);
    out[1] = 0.5 * (p - m);
    out[2] = creal(w);
    out[3] = cimag(w);
}

/* ------------------------------------------------------------------------- */
/* Grain optics.                                                             */
/* ------------------------------------------------------------------------- */

/* Dipole (Rayleigh) scattering matrix normalised to int P11 dOmega = 1, in the
 * scattering-plane basis (e_par, e_perp): P11,P12,P22,P33,P34,P44. */
void orc_rayleigh(double mu, double P[6])
{
    double f = 3.0 / (16.0 * M_PI);
    P[0] = f * (1.0 + mu * mu);
    P[1] = f * (mu * mu - 1.0);
    P[2] = f * (1.0 + mu * mu);
    P[3] = f * 2.0 * mu;
    P[4] = 0.0;
    P[5] = f * 2.0 * mu;
}

/* Table row interpolation, linear in the scattering angle on a uniform grid. */
static void table_mueller(const float *tab, int n_theta, double mu, double P[6])
{
    if (mu > 1.0) mu = 1.0;
    if (mu < -1.0) mu = -1.0;
    double x = acos(mu) / M_PI * (n_theta - 1);
    int j = (int)floor(x);
    if (j > n_theta - 2) j = n_theta - 2;
    if (j < 0) j = 0;
    double f = x - j;
    for (int e = 0; e < 6; ++e)
        P[e] = (1.0 - f) * tab[j * 6 + e] + f * tab[(j + 1) * 6 + e];
}

/* Scattering matrix of the bin mixture used by the step-1 tally. */
static void mixture_mueller(const orc_problem *P, double mu, double Z[6])
{
    if (P->scat_model == 0) {
        orc_rayleigh(mu, Z);
        return;
    }
    double wsum = 0.0;
    for (int k = 0; k < P->n_bins; ++k) wsum += P->bin_weight[k];
    for (int e = 0; e < 6; ++e) Z[e] = 0.0;
    for (int k = 0; k < P->n_bins; ++k) {
        double Pk[6];
        table_mueller(P->mueller + (size_t)k * P->n_theta * 6, P->n_theta, mu, Pk);
        for (int e = 0; e < 6; ++e) Z[e] += P->bin_weight[k] / wsum * Pk[e];
    }
}

/* Extinction elements alpha1..3 at grain-frame polar angle theta', linear in theta'. */
static void kext_eval(const orc_problem *P, double thetap, double al[3])
{
    double x = thetap / M_PI * (P->n_ktheta - 1);
    int j = (int)floor(x);
    if (j > P->n_ktheta - 2) j = P->n_ktheta - 2;
    if (j < 0) j = 0;
    double f = x - j;
    for (int e = 0; e < 3; ++e) al[e] = (1.0 - f) * P->kext[j * 3 + e] + f * P->kext[(j + 1) * 3 + e];
}

/* Average of alpha1 over the sphere, 1/2 int alpha1(theta') sin theta' dtheta',
 * integrating the linear interpolant exactly on each interval. */
static double kext_alpha1_mean(const orc_problem *P)
{
    double h = M_PI / (P->n_ktheta - 1), s = 0.0;
    for (int j = 0; j + 1 < P->n_ktheta; ++j) {
        double ta = j * h, tb = (j + 1) * h;
        double A = P->kext[j * 3], B = (P->kext[(j + 1) * 3] - A) / h;
        s += A * (cos(ta) - cos(tb)) + B * (-(tb - ta) * cos(tb) + sin(tb) - sin(ta));
    }
    return 0.5 * s;
}

/* Apply a scattering matrix Z (block form) for the scattering n -> n2 to X given
 * in the Stokes basis of n; the result is in the Stokes basis of n2.  The
 * scattering plane basis is e_perp = n x n2 / |n x n2|, e_par = e_perp x n on
 * the incident side and e_perp x n2 on the scattered side (Q = I_par - I_perp).
 * The plane is taken as undefined when sin(Theta) = |n x n2| < 1e-6; e_perp is
 * then the phi-hat of n (for a realizable matrix the result is continuous there:
 * P12, P34 -> 0 and P33 -> +-P11). */
void orc_mueller_apply(const double X[4], const double n[3], const double n2[3], const double Z[6], double out[4])
{
    double th[3], ph[3], th2[3], ph2[3];
    orc_stokes_basis(n, th, ph);
    orc_stokes_basis(n2, th2, ph2);
    double ep[3];
    cross3(n, n2, ep);
    double len = sqrt(dot3(ep, ep));
    if (len < 1e-6) {
        ep[0] = ph[0]; ep[1] = ph[1]; ep[2] = ph[2];
    } else {
        ep[0] /= len; ep[1] /= len; ep[2] /= len;
    }
    double epar_in[3], epar_out[3];
    cross3(ep, n, epar_in);
    cross3(ep, n2, epar_out);
    double Xs[4], Y[4];
    orc_change_basis(X, th, ph, epar_in, ep, Xs);
    Y[0] = Z[0] * Xs[0] + Z[1] * Xs[1];
    Y[1] = Z[1] * Xs[0] + Z[2] * Xs[1];
    Y[2] = Z[3] * Xs[2] + Z[4] * Xs[3];
    Y[3] = -Z[4] * Xs[2] + Z[5] * Xs[3];
    orc_change_basis(Y, epar_out, ep, th2, ph2, out);
}

/* (Z X)_0 / I for the proposal n -> n2: the polarization-aware differential
 * cross section relative to its unpolarized value, evaluated in the
 * scattering-plane basis. */
static double scattered_I(const double X[4], const double n[3], const double n2[3], const double Z[6])
{
    double th[3], ph[3];
    orc_stokes_basis(n, th, ph);
    double ep[3];
    cross3(n, n2, ep);
    double len = sqrt(dot3(ep, ep));
    if (len < 1e-6) {
        ep[0] = ph[0]; ep[1] = ph[1]; ep[2] = ph[2];
    } else {
        ep[0] /= len; ep[1] /= len; ep[2] /= len;
    }
    double epar_in[3];
    cross3(ep, n, epar_in);
    double Xs[4];
    orc_change_basis(X, th, ph, epar_in, ep, Xs);
    return Z[0] * Xs[0] + Z[1] * Xs[1];
}

/* ------------------------------------------------------------------------- */
/* Aligned spheroids in the dipole approximation (Sec. 2.1, Sec. 3: grain     */
/* optics from the dipole approximation, K from the optical theorem).        */
/* ------------------------------------------------------------------------- */

/* Depolarization factor L along the symmetry axis of a spheroid whose equatorial
 * semi-axis is s times its symmetry semi-axis (s > 1 oblate, s < 1 prolate, s = 1 a
 * sphere).  With g = s^2 - 1 the closed forms for oblate and prolate spheroids
 * (Bohren & Huffman 1983, eqs. 5.34, 5.35) are both L = s^2 F(g) with
 * F(g) = sum_k (-g)^k / (2k + 3): for g > 0, F = (1 - atan(sqrt g) / sqrt g) / g;
 * for g < 0, F = (atanh(sqrt -g) / sqrt -g - 1) / (-g).  The series is summed for
 * |g| < 0.5, where the closed forms cancel. */
double orc_spheroid_L(double s)
{
    double g = s * s - 1.0, F;
    if (fabs(g) < 0.5) {
        F = 0.0;
        double t = 1.0;
        for (int k = 0; k < 200; ++k) {
            F += t / (2 * k + 3);
            t *= -g;
        }
    } else if (g > 0.0) {
        double f = sqrt(g);
        F = (1.0 - atan(f) / f) / g;
    } else {
        double e = sqrt(-g);
        F = (atanh(e) / e - 1.0) / (-g);
    }
    return s * s * F;
}

/* Per-grain constants of the aligned dipole spheroid: dielectric function eps,
 * shape s (as above), size parameter x = 2 pi a_eff / lambda (a_eff the radius of
 * the sphere of equal volume).  Index 0 is a principal axis perpendicular to the
 * symmetry axis, index 1 the symmetry axis.
 *   polarizability per a_eff^3 (Clausius-Mossotti for an ellipsoid):
 *       alpha_j = (eps - 1) / (3 (1 + L_j (eps - 1))),  L_0 = (1 - L_1) / 2
 *   with the radiative-reaction correction alpha'_j = alpha_j / (1 - (2i/3) x^3 alpha_j)
 *   efficiencies (cross section over pi a_eff^2) for the field along axis j:
 *       Q_ext,j = 4 x Im alpha'_j          (optical theorem)
 *       Q_sca,j = (8/3) x^4 |alpha'_j|^2   (power radiated by the dipole)
 *       Q_abs,j = Q_ext,j - Q_sca,j
 * A field e (unit, transverse) sees C(e) = C_0 (1 - w) + C_1 w with w = (a . e)^2,
 * a the symmetry axis; over random orientation and polarization <w> = 1/3. */
typedef struct {
    double L[2];
    double complex al[2];     /* alpha'_j per a_eff^3 */
    double q_ext[2], q_sca[2], q_abs[2];
    double complex rho;       /* alpha'_1 / alpha'_0 */
    double zn;                /* 1 / N, N = (8 pi / 3) (2 + |rho|^2) / 3 */
    double env;               /* max(1, |rho|^2) zn: bound of (Z X)_0 / I */
} orc_dipole;

static void dipole_setup(double eps_re, double eps_im, double s, double x, orc_dipole *D)
{
    double complex eps = eps_re + I * eps_im;
    D->L[1] = orc_spheroid_L(s);
    D->L[0] = 0.5 * (1.0 - D->L[1]);
    for (int j = 0; j < 2; ++j) {
        double complex a = (eps - 1.0) / (3.0 * (1.0 + D->L[j] * (eps - 1.0)));
        double complex ap = a / (1.0 - I * (2.0 / 3.0) * x * x * x * a);
        D->al[j] = ap;
        D->q_ext[j] = 4.0 * x * cimag(ap);
        D->q_sca[j] = (8.0 / 3.0) * pow(x, 4) * creal(ap * conj(ap));
        D->q_abs[j] = D->q_ext[j] - D->q_sca[j];
    }
    D->rho = D->al[1] / D->al[0];
    double r2 = creal(D->rho * conj(D->rho));
    D->zn = 1.0 / ((8.0 * M_PI / 3.0) * (2.0 + r2) / 3.0);
    D->env = (r2 > 1.0 ? r2 : 1.0) * D->zn;
}

/* Test export: [L0, L1, Re a'0, Im a'0, Re a'1, Im a'1, Qext0, Qext1, Qsca0, Qsca1,
 * Qabs0, Qabs1, Re rho, Im rho, zn, env]. */
void orc_dipole_constants(double eps_re, double eps_im, double s, double x, double out[16])
{
    orc_dipole D;
    dipole_setup(eps_re, eps_im, s, x, &D);
    double v[16] = {D.L[0], D.L[1], creal(D.al[0]), cimag(D.al[0]), creal(D.al[1]), cimag(D.al[1]),
                    D.q_ext[0], D.q_ext[1], D.q_sca[0], D.q_sca[1], D.q_abs[0], D.q_abs[1],
                    creal(D.rho), cimag(D.rho), D.zn, D.env};
    memcpy(out, v, sizeof v);
}

/* Cross section for the transverse field e, relative to its average over random
 * orientation and polarization: c[0] perpendicular, c[1] along the axis. */
static double relative_cross_section(const double c[2], double w)
{
    double mean = (2.0 * c[0] + c[1]) / 3.0;
    if (!(mean > 0.0)) return 1.0;  /* no such process: any shape, the cell kappa is 0 */
    return (c[0] * (1.0 - w) + c[1] * w) / mean;
}

/* First-row elements (K11, K12) of a dichroic matrix, per unit of its orientation
 * average, for a packet along n in the basis (e1, e2) transverse to n: K11 and K12 are
 * the mean and half difference of the cross sections for fields along e1 and e2
 * (light polarized along e1, Q = I, is removed at K11 + K12). */
static void dichroic_row(const double c[2], const double axis[3], const double e1[3], const double e2[3],
                         double K[2])
{
    double w1 = dot3(axis, e1), w2 = dot3(axis, e2);
    double C1 = relative_cross_section(c, w1 * w1), C2 = relative_cross_section(c, w2 * w2);
    K[0] = 0.5 * (C1 + C2);
    K[1] = 0.5 * (C1 - C2);
}

/* Scattered Stokes vector Z X for the scattering n -> n2 by a grain with symmetry
 * axis `axis` (lab frame); X in the Stokes basis of n, the result in that of n2.  The
 * induced dipole is p = alpha'_0 (1 + (rho - 1) axis axis^T) E and the far field along
 * n2 is the part of p transverse to n2, so between the bases (th, ph) of n and (th2,
 * ph2) of n2 the Jones matrix is J_jk = f2_j . (1 + (rho - 1) axis axis^T) . f_k; the
 * coherency matrix C = 1/2 [[I+Q, U+iV], [U-iV, I-Q]] goes to J C J^dagger.  Scaled by
 * zn, so that int Z11 dOmega averaged over orientation is 1 (1/sr). */
static void dipole_scatter(const orc_dipole *D, const double axis[3], const double X[4], const double n[3],
                           const double n2[3], double out[4])
{
    double th[3], ph[3], th2[3], ph2[3];
    orc_stokes_basis(n, th, ph);
    orc_stokes_basis(n2, th2, ph2);
    const double *f[2] = {th, ph}, *f2[2] = {th2, ph2};
    double complex J[2][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k)
            J[j][k] = dot3(f2[j], f[k]) + (D->rho - 1.0) * dot3(f2[j], axis) * dot3(axis, f[k]);
    double complex Cm[2][2] = {{0.5 * (X[0] + X[1]), 0.5 * (X[2] + I * X[3])},
                               {0.5 * (X[2] - I * X[3]), 0.5 * (X[0] - X[1])}};
    double complex Dm[2][2];
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < 2; ++k) {
            double complex acc = 0.0;
            for (int l = 0; l < 2; ++l)
                for (int m = 0; m < 2; ++m) acc += J[j][l] * Cm[l][m] * conj(J[k][m]);
            Dm[j][k] = acc;
        }
    out[0] = D->zn * creal(Dm[0][0] + Dm[1][1]);
    out[1] = D->zn * creal(Dm[0][0] - Dm[1][1]);
    out[2] = D->zn * 2.0 * creal(Dm[0][1]);
    out[3] = D->zn * 2.0 * cimag(Dm[0][1]);
}

/* Test export of dipole_scatter: grain axis `axis`, out = Z X (1/sr). */
void orc_dipole_scatter(double eps_re, double eps_im, double s, double x, const double axis[3], const double X[4],
                        const double n[3], const double n2[3], double out[4])
{
    orc_dipole D;
    dipole_setup(eps_re, eps_im, s, x, &D);
    dipole_scatter(&D, axis, X, n, n2, out);
}

/* ------------------------------------------------------------------------- */
/* Grid and cell-to-cell traversal.                                          */
/* ------------------------------------------------------------------------- */
static double cell_size(const orc_problem *P, int a) { return (P->hi[a] - P->lo[a]) / P->n[a]; }

/* Cell holding p for travel along n; a point on a face belongs to the cell that
 * n points into.  Returns 0 when that cell is outside the grid. */
static int locate(const int n3[3], const double lo[3], const double hi[3], const double p[3],
                  const double n[3], int idx[3])
{
    for (int a = 0; a < 3; ++a) {
        double d = (hi[a] - lo[a]) / n3[a];
        double x = (p[a] - lo[a]) / d;
        int i = (int)floor(x);
        if ((double)i == x && n[a] < 0.0) i -= 1;
        idx[a] = i;
        if (i < 0 || i >= n3[a]) return 0;
    }
    return 1;
}

/* Distance to the exit face of cell idx along n and the axis crossed; equal
 * distances go to the lowest axis. */
static double exit_distance(const int n3[3], const double lo[3], const double hi[3], const int idx[3],
                            const double p[3], const double n[3], int *axis)
{
    double best = INFINITY;
    *axis = -1;
    for (int a = 0; a < 3; ++a) {
        double d = (hi[a] - lo[a]) / n3[a];
        double t;
        if (n[a] > 0.0)
            t = (lo[a] + (idx[a] + 1) * d - p[a]) / n[a];
        else if (n[a] < 0.0)
            t = (lo[a] + idx[a] * d - p[a]) / n[a];
        else
            continue;
        if (t < 0.0) t = 0.0;
        if (t < best) {
            best = t;
            *axis = a;
        }
    }
    return best;
}

/* Move p to the exit face and step the cell index; returns 0 on leaving the grid.
 * Along a periodic axis (bit axis of `periodic`) leaving the grid re-enters it on the
 * opposite face: index wrapped, coordinate set to that face. */
static int cross_face_p(const int n3[3], const double lo[3], const double hi[3], int idx[3], double p[3],
                        const double n[3], double ell, int axis, int periodic)
{
    double d = (hi[axis] - lo[axis]) / n3[axis];
    for (int a = 0; a < 3; ++a) p[a] += ell * n[a];
    if (n[axis] > 0.0) {
        p[axis] = lo[axis] + (idx[axis] + 1) * d;
        idx[axis] += 1;
    } else {
        p[axis] = lo[axis] + idx[axis] * d;
        idx[axis] -= 1;
    }
    if (idx[axis] >= 0 && idx[axis] < n3[axis]) return 1;
    if (!((periodic >> axis) & 1)) return 0;
    if (idx[axis] >= n3[axis]) {
        idx[axis] = 0;
        p[axis] = lo[axis];
    } else {
        idx[axis] = n3[axis] - 1;
        p[axis] = lo[axis] + n3[axis] * d;
    }
    return 1;
}

static int cross_face(const int n3[3], const double lo[3], const double hi[3], int idx[3], double p[3],
                      const double n[3], double ell, int axis)
{
    return cross_face_p(n3, lo, hi, idx, p, n, ell, axis, 0);
}

/* ------------------------------------------------------------------------- */
/* Composite grid: the root grid and its statically refined patches (Sec. 2:  */
/* a composite mesh with optional static mesh refinement).                    */
/* ------------------------------------------------------------------------- */
/* Cells are numbered root first ([z][y][x]), then each patch in order ([z][y][x]
 * within the patch).  A position in the grid is (g, idx): g = -1 for the root grid,
 * else the patch number. */
typedef struct {
    int g;
    int idx[3];
} where_t;

static int64_t root_cells(const orc_problem *P) { return (int64_t)P->n[0] * P->n[1] * P->n[2]; }

static void patch_dims(const orc_problem *P, int q, int n3[3])
{
    const orc_patch *Q = &P->patches[q];
    for (int a = 0; a < 3; ++a) n3[a] = (Q->box[3 + a] - Q->box[a]) * Q->factor;
}

static int64_t patch_offset(const orc_problem *P, int q)
{
    int64_t off = root_cells(P);
    for (int k = 0; k < q; ++k) {
        int m[3];
        patch_dims(P, k, m);
        off += (int64_t)m[0] * m[1] * m[2];
    }
    return off;
}

int64_t orc_n_cells(const orc_problem *P) { return patch_offset(P, P->n_patches); }

/* Cell counts and box of grid g (root or patch). */
static void grid_geom(const orc_problem *P, int g, int n3[3], double lo[3], double hi[3])
{
    if (g < 0) {
        for (int a = 0; a < 3; ++a) {
            n3[a] = P->n[a];
            lo[a] = P->lo[a];
            hi[a] = P->hi[a];
        }
        return;
    }
    patch_dims(P, g, n3);
    for (int a = 0; a < 3; ++a) {
        double d = (P->hi[a] - P->lo[a]) / P->n[a];
        lo[a] = P->lo[a] + P->patches[g].box[a] * d;
        hi[a] = P->lo[a] + P->patches[g].box[3 + a] * d;
    }
}

static int64_t cell_index(const orc_problem *P, const where_t *w)
{
    int n3[3];
    double lo[3], hi[3];
    grid_geom(P, w->g, n3, lo, hi);
    int64_t local = ((int64_t)w->idx[2] * n3[1] + w->idx[1]) * n3[0] + w->idx[0];
    return w->g < 0 ? local : patch_offset(P, w->g) + local;
}

static void cell_where(const orc_problem *P, int64_t c, where_t *w)
{
    w->g = -1;
    for (int q = P->n_patches - 1; q >= 0; --q)
        if (c >= patch_offset(P, q)) {
            w->g = q;
            c -= patch_offset(P, q);
            break;
        }
    int n3[3];
    double lo[3], hi[3];
    grid_geom(P, w->g, n3, lo, hi);
    w->idx[0] = (int)(c % n3[0]);
    w->idx[1] = (int)((c / n3[0]) % n3[1]);
    w->idx[2] = (int)(c / ((int64_t)n3[0] * n3[1]));
}

static double grid_cell_volume(const orc_problem *P, int g)
{
    int n3[3];
    double lo[3], hi[3];
    grid_geom(P, g, n3, lo, hi);
    return (hi[0] - lo[0]) / n3[0] * (hi[1] - lo[1]) / n3[1] * (hi[2] - lo[2]) / n3[2];
}

/* Cell data of composite cell c. */
static const float *cell_array(const orc_problem *P, int64_t c, int which, int64_t *local)
{
    *local = c;
    if (c < root_cells(P)) {
        const float *root[4] = {P->kappa_abs, P->kappa_sca, P->bfield, P->emissivity};
        return root[which];
    }
    for (int q = P->n_patches - 1; q >= 0; --q) {
        int64_t off = patch_offset(P, q);
        if (c >= off) {
            const orc_patch *Q = &P->patches[q];
            const float *arr[4] = {Q->kappa_abs, Q->kappa_sca, Q->bfield, Q->emissivity};
            *local = c - off;
            return arr[which];
        }
    }
    return NULL;
}

static double cell_ka(const orc_problem *P, int64_t c)
{
    int64_t l;
    return cell_array(P, c, 0, &l)[l];
}

static double cell_ks(const orc_problem *P, int64_t c)
{
    int64_t l;
    return cell_array(P, c, 1, &l)[l];
}

static double cell_em(const orc_problem *P, int64_t c)
{
    int64_t l;
    const float *e = cell_array(P, c, 3, &l);
    return e ? e[l] : 0.0;
}

/* Field direction of cell c; 0 when the model has no field. */
static int cell_field(const orc_problem *P, int64_t c, double b[3])
{
    int64_t l;
    const float *f = cell_array(P, c, 2, &l);
    if (!f) return 0;
    b[0] = f[3 * l];
    b[1] = f[3 * l + 1];
    b[2] = f[3 * l + 2];
    return 1;
}

/* Patch covering root cell ridx, or -1. */
static int covering_patch(const orc_problem *P, const int ridx[3])
{
    for (int q = 0; q < P->n_patches; ++q) {
        const int32_t *b = P->patches[q].box;
        if (ridx[0] >= b[0] && ridx[0] < b[3] && ridx[1] >= b[1] && ridx[1] < b[4] && ridx[2] >= b[2] &&
            ridx[2] < b[5])
            return q;
    }
    return -1;
}

/* Root cell ridx entered at p along n: the cell itself, or the cell of the patch that
 * covers it, found like locate (a point on a face belongs to the cell n points into)
 * and clamped to the patch. */
static void enter_root_cell(const orc_problem *P, const int ridx[3], const double p[3], const double n[3],
                            where_t *w)
{
    int q = covering_patch(P, ridx);
    w->g = q;
    if (q < 0) {
        for (int a = 0; a < 3; ++a) w->idx[a] = ridx[a];
        return;
    }
    int n3[3];
    double lo[3], hi[3];
    grid_geom(P, q, n3, lo, hi);
    for (int a = 0; a < 3; ++a) {
        double d = (hi[a] - lo[a]) / n3[a];
        double x = (p[a] - lo[a]) / d;
        int i = (int)floor(x);
        if ((double)i == x && n[a] < 0.0) i -= 1;
        if (i < 0) i = 0;
        if (i >= n3[a]) i = n3[a] - 1;
        w->idx[a] = i;
    }
}

static int composite_locate(const orc_problem *P, const double p[3], const double n[3], where_t *w)
{
    int ridx[3];
    if (!locate(P->n, P->lo, P->hi, p, n, ridx)) return 0;
    enter_root_cell(P, ridx, p, n, w);
    return 1;
}

static double composite_exit(const orc_problem *P, const where_t *w, const double p[3], const double n[3],
                             int *axis)
{
    int n3[3];
    double lo[3], hi[3];
    grid_geom(P, w->g, n3, lo, hi);
    return exit_distance(n3, lo, hi, w->idx, p, n, axis);
}

/* Move p to the exit face of the current cell and into the next cell of the composite
 * grid; 0 when the packet leaves the grid.  Leaving a patch leads to the root cell
 * beyond its face (or, through a periodic face of the root box, the one on the
 * opposite side), which may itself be covered by a patch. */
static int composite_cross(const orc_problem *P, where_t *w, double p[3], const double n[3], double ell, int axis,
                           int periodic)
{
    int n3[3];
    double lo[3], hi[3];
    grid_geom(P, w->g, n3, lo, hi);
    if (w->g < 0) {
        if (!cross_face_p(n3, lo, hi, w->idx, p, n, ell, axis, periodic)) return 0;
        int ridx[3] = {w->idx[0], w->idx[1], w->idx[2]};
        enter_root_cell(P, ridx, p, n, w);
        return 1;
    }
    if (cross_face_p(n3, lo, hi, w->idx, p, n, ell, axis, 0)) return 1;
    const orc_patch *Q = &P->patches[w->g];
    int ridx[3];
    for (int a = 0; a < 3; ++a) ridx[a] = Q->box[a] + w->idx[a] / Q->factor;
    ridx[axis] = n[axis] > 0.0 ? Q->box[3 + axis] : Q->box[axis] - 1;
    if (ridx[axis] < 0 || ridx[axis] >= P->n[axis]) {
        if (!((periodic >> axis) & 1)) return 0;
        ridx[axis] = ridx[axis] < 0 ? P->n[axis] - 1 : 0;
        p[axis] = ridx[axis] == 0 ? P->lo[axis] : P->hi[axis];
    }
    enter_root_cell(P, ridx, p, n, w);
    return 1;
}

/* Composite cells and chord lengths along a ray from p0 (for the refinement pins). */
int64_t orc_dda_walk_composite(const orc_problem *P, const double p0[3], const double n[3], int64_t max_cells,
                               int64_t *cells, double *lengths)
{
    where_t w;
    double p[3] = {p0[0], p0[1], p0[2]};
    if (!composite_locate(P, p, n, &w)) return 0;
    int64_t k = 0;
    while (k < max_cells) {
        int axis;
        double ell = composite_exit(P, &w, p, n, &axis);
        cells[k] = cell_index(P, &w);
        lengths[k] = ell;
        ++k;
        if (!composite_cross(P, &w, p, n, ell, axis, 0)) break;
    }
    return k;
}

/* Brute list of cells and chord lengths along a ray (for the DDA pins). */
int64_t orc_dda_walk(const int32_t n3[3], const double lo[3], const double hi[3], const double p0[3],
                     const double n[3], int64_t max_cells, int64_t *cells, double *lengths)
{
    int idx[3];
    double p[3] = {p0[0], p0[1], p0[2]};
    if (!locate(n3, lo, hi, p, n, idx)) return 0;
    int64_t k = 0;
    while (k < max_cells) {
        int axis;
        double ell = exit_distance(n3, lo, hi, idx, p, n, &axis);
        cells[k] = ((int64_t)idx[2] * n3[1] + idx[1]) * n3[0] + idx[0];
        lengths[k] = ell;
        ++k;
        if (!cross_face(n3, lo, hi, idx, p, n, ell, axis)) break;
    }
    return k;
}

/* ------------------------------------------------------------------------- */
/* Per-cell local frame: grain quaternion, grain-meridian basis, K elements.  */
/* ------------------------------------------------------------------------- */
typedef struct {
    double th[3], ph[3];   /* lab Stokes basis of n */
    double gth[3], gph[3]; /* grain-meridian basis of n, in lab coordinates */
    double alpha[3];       /* alpha1..3 at theta' (extinction per unit kappa_ext) */
    double sca[2];         /* scattering part (s11, s12) of the first row of K per unit
                              kappa_ext, grain-meridian basis; s11 kappa_ext is the rate
                              at which scatterings are sampled along n */
    double gsca;           /* that rate over kappa_sca (1 for Theta-only optics) */
    double thetap;
    double axis[3];        /* grain symmetry axis in the lab frame */
    orc_dipole dip;        /* scat_model 2 constants */
} local_frame;

static void cell_quaternion(const orc_problem *P, int64_t c, double q[4])
{
    double b[3];
    if (!cell_field(P, c, b)) {
        q[0] = 1.0; q[1] = q[2] = q[3] = 0.0;
        return;
    }
    orc_grain_quaternion(b[0], b[1], b[2], q);
}

static void make_local_frame(const orc_problem *P, int64_t c, const double n[3], local_frame *F)
{
    double q[4], nGF[3], th_g[3], ph_g[3];
    cell_quaternion(P, c, q);
    orc_stokes_basis(n, F->th, F->ph);
    orc_to_grain(q, n, nGF);
    orc_stokes_basis(nGF, th_g, ph_g);
    orc_to_lab(q, th_g, F->gth);
    orc_to_lab(q, ph_g, F->gph);
    double cz = nGF[2];
    if (cz > 1.0) cz = 1.0;
    if (cz < -1.0) cz = -1.0;
    F->thetap = acos(cz);
    const double zg[3] = {0.0, 0.0, 1.0};
    orc_to_lab(q, zg, F->axis);
    double ka = cell_ka(P, c), ks = cell_ks(P, c);
    double kext = ka + ks;
    double omega = kext > 0.0 ? ks / kext : 0.0;
    if (P->scat_model == 2) {
        /* K = kappa_abs Khat_abs + kappa_sca Khat_sca, each dichroic part relative to its
         * orientation average; no U-V terms (no phase lag in the optical theorem) */
        dipole_setup(P->eps_re, P->eps_im, P->aspect, P->size_x, &F->dip);
        double fa = kext > 0.0 ? ka / kext : 0.0, Ka[2], Ks[2];
        dichroic_row(F->dip.q_abs, F->axis, F->gth, F->gph, Ka);
        dichroic_row(F->dip.q_sca, F->axis, F->gth, F->gph, Ks);
        F->alpha[0] = fa * Ka[0] + omega * Ks[0];
        F->alpha[1] = fa * Ka[1] + omega * Ks[1];
        F->alpha[2] = 0.0;
        F->sca[0] = omega * Ks[0];
        F->sca[1] = omega * Ks[1];
        F->gsca = Ks[0];
    } else {
        kext_eval(P, F->thetap, F->alpha);
        F->sca[0] = omega;
        F->sca[1] = 0.0;
        F->gsca = 1.0;
    }
}

/* Public wrapper for the frame tests: grain-meridian basis and theta'. */
void orc_grain_meridian(const double q[4], const double n[3], double gth[3], double gph[3], double *thetap)
{
    double nGF[3], th_g[3], ph_g[3];
    orc_to_grain(q, n, nGF);
    orc_stokes_basis(nGF, th_g, ph_g);
    orc_to_lab(q, th_g, gth);
    orc_to_lab(q, ph_g, gph);
    double cz = nGF[2];
    if (cz > 1.0) cz = 1.0;
    if (cz < -1.0) cz = -1.0;
    *thetap = acos(cz);
}

/* ------------------------------------------------------------------------- */
/* Tallies (compare-and-swap when several threads run).                      */
/* ------------------------------------------------------------------------- */
static int g_threads_shared = 0;

static void add_double(double *dst, double v)
{
    if (!g_threads_shared) {
        *dst += v;
        return;
    }
    uint64_t *p = (uint64_t *)dst;
    uint64_t old = __atomic_load_n(p, __ATOMIC_RELAXED);
    for (;;) {
        double cur;
        memcpy(&cur, &old, 8);
        double nv = cur + v;
        uint64_t nb;
        memcpy(&nb, &nv, 8);
        if (__atomic_compare_exchange_n(p, &old, nb, 0, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) return;
    }
}

/* ------------------------------------------------------------------------- */
/* Step 1: Monte-Carlo transport of one packet.                              */
/* ------------------------------------------------------------------------- */
typedef struct {
    const orc_problem *P;
    orc_result *R;
    const double *cdf;     /* thermal emission CDF over cells (unnormalised), or NULL */
    double cdf_total;
    double alpha1_mean;
    double thermal_L;
    double stats[16];
} run_ctx;

static int find_source(const orc_problem *P, int64_t pid, int64_t *first)
{
    int64_t start = 0;
    for (int s = 0; s < P->n_sources; ++s) {
        if (pid < start + P->sources[s].n_packets) {
            *first = start;
            return s;
        }
        start += P->sources[s].n_packets;
    }
    *first = start;
    return -1;
}

static double source_luminosity(const run_ctx *C, int s)
{
    const orc_source *src = &C->P->sources[s];
    if (src->type == 2 && src->luminosity <= 0.0) return C->thermal_L;
    return src->luminosity;
}

static void isotropic(double u_cos, double u_phi, double n[3])
{
    double ct = 2.0 * u_cos - 1.0;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = 2.0 * M_PI * u_phi;
    n[0] = st * cos(ph); n[1] = st * sin(ph); n[2] = ct;
}

/* Packet birth, event 0 (Sec. 2.2): position, direction and Stokes vector in the
 * lab basis of n.  Slot 0 = (tau, cos theta, phi, cell), slot 1 = (x, y, z, -). */
static int emit_packet(const run_ctx *C, int64_t pid, int s, double eps, double p[3], double n[3],
                       double X[4], where_t *w, double *tau)
{
    const orc_problem *P = C->P;
    const orc_source *src = &P->sources[s];
    const int64_t ncell = orc_n_cells(P);
    double u0[4], u1[4];
    draw4(P, pid, 0, 0, u0);
    draw4(P, pid, 0, 1, u1);
    X[0] = eps; X[1] = X[2] = X[3] = 0.0;
    int inside;
    if (src->type == 0) {
        p[0] = src->pos[0]; p[1] = src->pos[1]; p[2] = src->pos[2];
        isotropic(u0[1], u0[2], n);
        inside = composite_locate(P, p, n, w);
    } else if (src->type == 1) {
        p[0] = P->lo[0] + u1[0] * (P->hi[0] - P->lo[0]);
        p[1] = P->lo[1] + u1[1] * (P->hi[1] - P->lo[1]);
        p[2] = src->beam_dir > 0 ? P->lo[2] : P->hi[2];
        n[0] = 0.0; n[1] = 0.0; n[2] = src->beam_dir > 0 ? 1.0 : -1.0;
        inside = composite_locate(P, p, n, w);
    } else {
        /* thermal: first cell whose cumulative weight exceeds u * total */
        double target = u0[3] * C->cdf_total;
        int64_t lo = 0, hi = ncell - 1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (C->cdf[mid] > target) hi = mid; else lo = mid + 1;
        }
        int64_t c = lo;
        cell_where(P, c, w);
        int n3[3];
        double glo[3], ghi[3];
        grid_geom(P, w->g, n3, glo, ghi);
        for (int a = 0; a < 3; ++a) p[a] = glo[a] + (w->idx[a] + u1[a]) * ((ghi[a] - glo[a]) / n3[a]);
        isotropic(u0[1], u0[2], n);
        inside = 1;
        /* emission alpha_abs B with alpha_abs the absorption part of K acting on
         * (1,0,0,0), in the grain-meridian basis; weight alpha_abs,11(theta') over its
         * mean over directions (mean alpha1 - omega) */
        local_frame F;
        make_local_frame(P, c, n, &F);
        double ka = cell_ka(P, c), ks = cell_ks(P, c);
        double omega = (ka + ks) > 0.0 ? ks / (ka + ks) : 0.0;
        /* absorption part of K's first row along n */
        double kab1 = F.alpha[0] - F.sca[0], kab2 = F.alpha[1] - F.sca[1];
        double w = kab1 / (C->alpha1_mean - omega);
        double Xg[4] = {eps * w, kab1 > 0.0 ? eps * w * kab2 / kab1 : 0.0, 0.0, 0.0};
        orc_change_basis(Xg, F.gth, F.gph, F.th, F.ph, X);
    }
    *tau = -log(u0[0]);
    return inside;
}

/* Rejection sampling of the polarization-aware differential cross section at
 * scattering number n_sca (Sec. 2.2 and Sec. 3).  Trial t uses slot 1 + t.
 * On acceptance n2 is the new direction and Y the scattered Stokes vector in the
 * lab basis of n2, renormalised to the incident I.  Returns the number of trials,
 * negative when no proposal was accepted within max_trials. */
static int scatter_sample(const orc_problem *P, int64_t pid, uint32_t n_sca, int bin, const double X[4],
                          const double n[3], const double q[4], double n2[3], double Y[4])
{
    const float *tab = NULL;
    double *env_cdf = NULL, env_cdf_total = 0.0;
    const int dip = P->scat_model == 2;
    orc_dipole D;
    double axis[3], I_w = X[0];
    if (dip) {
        /* aligned spheroid: the total scattered power (K_sca X)_0 depends on the
         * polarization; the new Stokes vector is Z X (K_sca X)_0 / (s11 (Z X)_0) with
         * s11 the sampling rate (Sec. 2.2 weight for direction-dependent cross sections),
         * i.e. Z X renormalised to I + (s12 / s11) Q in the grain-meridian basis */
        const double zg[3] = {0.0, 0.0, 1.0};
        double gth[3], gph[3], th[3], ph[3], tp, Xg[4], Ks[2];
        dipole_setup(P->eps_re, P->eps_im, P->aspect, P->size_x, &D);
        orc_to_lab(q, zg, axis);
        orc_grain_meridian(q, n, gth, gph, &tp);
        orc_stokes_basis(n, th, ph);
        orc_change_basis(X, th, ph, gth, gph, Xg);
        dichroic_row(D.q_sca, axis, gth, gph, Ks);
        I_w = X[0] + Ks[1] / Ks[0] * Xg[1];
    }
    if (P->scat_model == 1) {
        tab = P->mueller + (size_t)bin * P->n_theta * 6;
        /* piecewise-constant envelope of P11 over [theta_j, theta_j+1] */
        env_cdf = (double *)malloc(sizeof(double) * (P->n_theta - 1));
        for (int j = 0; j + 1 < P->n_theta; ++j) {
            double t0 = M_PI * j / (P->n_theta - 1), t1 = M_PI * (j + 1) / (P->n_theta - 1);
            double env = fmax(tab[j * 6], tab[(j + 1) * 6]);
            env_cdf_total += env * (cos(t0) - cos(t1));
            env_cdf[j] = env_cdf_total;
        }
    }
    int result = -P->max_trials;
    for (int t = 0; t < P->max_trials; ++t) {
        double ut[4];
        draw4(P, pid, n_sca, (uint32_t)(1 + t), ut);
        double Z[6], bound, Yd[4];
        if (dip) {
            /* isotropic proposal, envelope max(1, |rho|^2) zn I >= (Z X)_0 */
            double nGF2[3];
            isotropic(ut[0], ut[1], nGF2);
            orc_to_lab(q, nGF2, n2);
            dipole_scatter(&D, axis, X, n, n2, Yd);
            bound = ut[2] * D.env * X[0];
        } else if (P->scat_model == 0) {
            /* isotropic proposal in the grain frame, envelope 2 max Z11 */
            double nGF2[3];
            isotropic(ut[0], ut[1], nGF2);
            orc_to_lab(q, nGF2, n2);
            orc_rayleigh(dot3(n, n2), Z);
            bound = ut[2] * 2.0 * (3.0 / (8.0 * M_PI)) * X[0];
        } else {
            int j = P->n_theta - 2;
            for (int jj = 0; jj + 1 < P->n_theta; ++jj)
                if (ut[0] < env_cdf[jj] / env_cdf_total) {
                    j = jj;
                    break;
                }
            double t0 = M_PI * j / (P->n_theta - 1), t1 = M_PI * (j + 1) / (P->n_theta - 1);
            double mu = cos(t0) - ut[1] * (cos(t0) - cos(t1));
            double sn = sqrt(fmax(0.0, 1.0 - mu * mu));
            double az = 2.0 * M_PI * ut[2];
            double th[3], ph[3];
            orc_stokes_basis(n, th, ph);
            for (int a = 0; a < 3; ++a) n2[a] = mu * n[a] + sn * (cos(az) * th[a] + sin(az) * ph[a]);
            table_mueller(tab, P->n_theta, mu, Z);
            double env = fmax(tab[j * 6], tab[(j + 1) * 6]);
            bound = ut[3] * 2.0 * env * X[0];
        }
        if (dip ? bound < Yd[0] : bound < scattered_I(X, n, n2, Z)) {
            if (dip)
                for (int e = 0; e < 4; ++e) Y[e] = Yd[e];
            else
                orc_mueller_apply(X, n, n2, Z, Y);
            double norm = I_w / Y[0];
            for (int e = 0; e < 4; ++e) Y[e] *= norm;
            result = t + 1;
            break;
        }
    }
    free(env_cdf);
    return result;
}

/* Grain bin k with probability proportional to its weight: the first k whose
 * cumulative normalised weight exceeds u. */
static int choose_bin(const orc_problem *P, double u)
{
    if (P->scat_model != 1) return 0;
    double wsum = 0.0, acc = 0.0;
    for (int k = 0; k < P->n_bins; ++k) wsum += P->bin_weight[k];
    for (int k = 0; k < P->n_bins; ++k) {
        acc += P->bin_weight[k];
        if (u < acc / wsum) return k;
    }
    return P->n_bins - 1;
}

static void transport_packet(run_ctx *C, int64_t pid)
{
    const orc_problem *P = C->P;
    orc_result *R = C->R;
    int64_t first;
    int s = find_source(P, pid, &first);
    if (s < 0) return;
    const orc_source *src = &P->sources[s];
    double eps = source_luminosity(C, s) / (double)src->n_packets;

    double p[3], n[3], X[4], tau_rem;
    where_t w;
    int inside = emit_packet(C, pid, s, eps, p, n, X, &w, &tau_rem);
    double I_birth = X[0];
    C->stats[ST_EMITTED_E] += X[0];
    C->stats[ST_EMITTED_N] += 1.0;
    C->stats[ST_EVENTS] += 1.0;

    int64_t n_seg = 0, n_sca = 0, events = 1;
    int flag = 0; /* 1 escaped, 2 roulette, 3 event cap, 4 trial cap */
    if (!inside) flag = 1;

    while (!flag) {
        if (events >= P->max_events) {
            flag = 3;
            break;
        }
        int64_t c = cell_index(P, &w);
        double ka = cell_ka(P, c), ks = cell_ks(P, c);
        double kext = ka + ks;
        int axis;
        double ell_exit = composite_exit(P, &w, p, n, &axis);
        local_frame F;
        if (kext > 0.0) make_local_frame(P, c, n, &F);
        /* scattering optical depth sampled along n: kappa_sca for Theta-only optics, the
         * direction-dependent unpolarized rate s11 kappa_ext for aligned spheroids */
        double ks_n = (P->scat_model == 2 && kext > 0.0) ? ks * F.gsca : ks;
        double dtau_sca_exit = ks_n * ell_exit;
        int scatter_here = (ks_n > 0.0 && tau_rem < dtau_sca_exit);
        double ell = scatter_here ? tau_rem / ks_n : ell_exit;

        /* ---- extinction, absorption and the step-1 tally over the segment ---- */
        if (kext > 0.0) {
            double dtau = kext * ell;
            double a = F.alpha[0] - F.sca[0];
            double Xg[4], Yg[4], Wg[4], Y[4];
            orc_change_basis(X, F.th, F.ph, F.gth, F.gph, Xg);
            orc_attenuate(Xg, a, F.alpha[1], F.alpha[2], dtau, Yg);
            orc_change_basis(Yg, F.gth, F.gph, F.th, F.ph, Y);
            double dI = X[0] - Y[0];
            if (P->scat_model == 2) {
                /* the decrease of I holds kappa_ext s12 int Q dl, the polarization-dependent
                 * part of the scattering rate; it is not absorption and returns in
                 * expectation through the scattering weight, so the absorbed tally is
                 * int (K_abs X)_0 dl */
                double Wt[4];
                orc_segment_integral(Xg, a, F.alpha[1], F.alpha[2], dtau, Wt);
                dI -= F.sca[1] * Wt[1];
            }
            if (ks > 0.0 && P->n_cam > 0) {
                double W[4];
                orc_segment_integral(Xg, a, F.alpha[1], F.alpha[2], dtau, Wg);
                for (int e = 0; e < 4; ++e) Wg[e] /= kext;
                orc_change_basis(Wg, F.gth, F.gph, F.th, F.ph, W);
                for (int k = 0; k < P->n_cam; ++k) {
                    double Z[6], Sc[4];
                    /* eq. (scat-disc-sum): Z(Omega_cam; Omega_pp) applied to the path
                     * integral of I_pp, in the Stokes basis of Omega_cam */
                    if (P->scat_model == 2) {
                        dipole_scatter(&F.dip, F.axis, W, n, P->cams[k].dir, Sc);
                    } else {
                        mixture_mueller(P, dot3(n, P->cams[k].dir), Z);
                        orc_mueller_apply(W, n, P->cams[k].dir, Z, Sc);
                    }
                    for (int e = 0; e < 4; ++e) add_double(&R->S[((size_t)c * P->n_cam + k) * 4 + e], Sc[e]);
                }
            }
            if (dI != 0.0) {
                add_double(&R->absorbed[c], dI);
                C->stats[ST_ABSORBED_E] += dI;
            }
            for (int e = 0; e < 4; ++e) X[e] = Y[e];
        }
        n_seg++;
        events++;
        C->stats[ST_SEGMENTS] += 1.0;
        C->stats[ST_EVENTS] += 1.0;

        if (!scatter_here) {
            tau_rem -= dtau_sca_exit;
            if (!composite_cross(P, &w, p, n, ell_exit, axis, P->periodic)) {
                flag = 1;
                break;
            }
            continue;
        }

        /* ---- scattering event: the packet stays in cell idx ---- */
        for (int a = 0; a < 3; ++a) p[a] += ell * n[a];
        n_sca++;
        events++;
        C->stats[ST_SCATTERS] += 1.0;
        C->stats[ST_EVENTS] += 1.0;
        double us[4];
        draw4(P, pid, (uint32_t)n_sca, 0, us);
        if (P->roulette_threshold > 0.0 && X[0] < P->roulette_threshold * I_birth) {
            if (us[1] < P->roulette_survival) {
                double g = 1.0 / P->roulette_survival;
                C->stats[ST_ROULETTE_GAIN] += X[0] * (g - 1.0);
                for (int e = 0; e < 4; ++e) X[e] *= g;
            } else {
                C->stats[ST_ROULETTE_LOST] += X[0];
                flag = 2;
                break;
            }
        }
        double q[4], n2[3], Y[4];
        cell_quaternion(P, c, q);
        int trials = scatter_sample(P, pid, (uint32_t)n_sca, choose_bin(P, us[2]), X, n, q, n2, Y);
        C->stats[ST_TRIALS] += (double)(trials > 0 ? trials : -trials);
        if (trials < 0) {
            flag = 4;
            break;
        }
        for (int e = 0; e < 4; ++e) X[e] = Y[e];
        for (int a = 0; a < 3; ++a) n[a] = n2[a];
        tau_rem = -log(us[0]);
    }

    if (flag == 1) {
        C->stats[ST_ESCAPED_E] += X[0];
        C->stats[ST_ESCAPED_N] += 1.0;
    } else if (flag == 2) {
        C->stats[ST_KILLED_N] += 1.0;
    } else if (flag == 3 || flag == 4) {
        C->stats[ST_CAP_LOST] += X[0];
        C->stats[ST_CAP_N] += 1.0;
    }
    if (R->trace && pid < P->n_trace) {
        double *tr = R->trace + (size_t)pid * 16;
        tr[0] = X[0]; tr[1] = X[1]; tr[2] = X[2]; tr[3] = X[3];
        tr[4] = p[0]; tr[5] = p[1]; tr[6] = p[2];
        tr[7] = n[0]; tr[8] = n[1]; tr[9] = n[2];
        tr[10] = (double)n_sca; tr[11] = (double)n_seg; tr[12] = (double)flag;
        tr[13] = I_birth; tr[14] = (double)s; tr[15] = (double)events;
    }
}

typedef struct {
    run_ctx *C;
    int64_t b, e;
} thread_arg;

static void *thread_main(void *arg)
{
    thread_arg *A = (thread_arg *)arg;
    for (int64_t pid = A->b; pid < A->e; ++pid) transport_packet(A->C, pid);
    return NULL;
}

/* Thermal source set-up: cell weights kappa_ext (mean alpha1 - omega) B V (V the cell's
 * own volume; root cells covered by a patch weigh 0) and the luminosity 4 pi sum of
 * them. */
static int thermal_setup(run_ctx *C)
{
    const orc_problem *P = C->P;
    int need = 0;
    for (int s = 0; s < P->n_sources; ++s)
        if (P->sources[s].type == 2) need = 1;
    /* the dipole's K is relative to its orientation average: mean alpha1 = 1 */
    C->alpha1_mean = P->scat_model == 2 ? 1.0 : kext_alpha1_mean(P);
    if (!need) return 0;
    if (!P->emissivity) return -1;
    const int64_t ncell = orc_n_cells(P);
    double *cdf = (double *)malloc(sizeof(double) * ncell);
    double acc = 0.0;
    int64_t c = 0;
    /* level by level: the root grid, then each patch, each with its cells' volume */
    for (int g = -1; g < P->n_patches; ++g) {
        int n3[3];
        double glo[3], ghi[3];
        grid_geom(P, g, n3, glo, ghi);
        const double V = grid_cell_volume(P, g);
        const float *ka = g < 0 ? P->kappa_abs : P->patches[g].kappa_abs;
        const float *ks = g < 0 ? P->kappa_sca : P->patches[g].kappa_sca;
        const float *em = g < 0 ? P->emissivity : P->patches[g].emissivity;
        const int64_t count = (int64_t)n3[0] * n3[1] * n3[2];
        for (int64_t l = 0; l < count; ++l, ++c) {
            double kext = (double)ka[l] + (double)ks[l];
            double omega = kext > 0.0 ? ks[l] / kext : 0.0;
            double w = kext * (C->alpha1_mean - omega) * (em ? em[l] : 0.0) * V;
            if (w < 0.0) w = 0.0;
            if (g < 0 && P->n_patches > 0) {
                int ridx[3] = {(int)(l % n3[0]), (int)((l / n3[0]) % n3[1]), (int)(l / ((int64_t)n3[0] * n3[1]))};
                if (covering_patch(P, ridx) >= 0) w = 0.0;
            }
            acc += w;
            cdf[c] = acc;
        }
    }
    C->cdf = cdf;
    C->cdf_total = acc;
    C->thermal_L = 4.0 * M_PI * acc;
    return 0;
}

double orc_thermal_luminosity(const orc_problem *P)
{
    run_ctx C;
    memset(&C, 0, sizeof C);
    C.P = P;
    if (thermal_setup(&C) != 0) return -1.0;
    free((void *)C.cdf);
    return C.thermal_L;
}

int orc_transport(const orc_problem *P, orc_result *R)
{
    if (P->n_cam > 64) return -1;
    run_ctx C;
    memset(&C, 0, sizeof C);
    C.P = P;
    C.R = R;
    if (thermal_setup(&C) != 0) return -2;
    int nt = P->n_threads > 0 ? P->n_threads : 1;
    int64_t total = P->pid_end - P->pid_begin;
    if (nt > total) nt = total > 0 ? (int)total : 1;
    /* wall time of the packet loop alone (set-up above excluded), for the CPU baseline */
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    if (nt == 1) {
        g_threads_shared = 0;
        for (int64_t pid = P->pid_begin; pid < P->pid_end; ++pid) transport_packet(&C, pid);
        memcpy(R->stats, C.stats, sizeof C.stats);
    } else {
        g_threads_shared = 1;
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
        thread_arg *A = (thread_arg *)malloc(sizeof(thread_arg) * nt);
        run_ctx *Cs = (run_ctx *)malloc(sizeof(run_ctx) * nt);
        for (int t = 0; t < nt; ++t) {
            Cs[t] = C;
            A[t].C = &Cs[t];
            A[t].b = P->pid_begin + total * t / nt;
            A[t].e = P->pid_begin + total * (t + 1) / nt;
            pthread_create(&th[t], NULL, thread_main, &A[t]);
        }
        memset(R->stats, 0, sizeof R->stats);
        for (int t = 0; t < nt; ++t) {
            pthread_join(th[t], NULL);
            for (int k = 0; k < 16; ++k) R->stats[k] += Cs[t].stats[k];
        }
        g_threads_shared = 0;
        free(th);
        free(A);
        free(Cs);
    }
    clock_gettime(CLOCK_MONOTONIC, &t1);
    R->stats[15] = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
    free((void *)C.cdf);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Step 2: deterministic ray-march toward the camera (Sec. 2.3, App. A).     */
/* ------------------------------------------------------------------------- */

/* S is the step-1 tally [ncell][n_cam][4]; scale_S multiplies it (1 / number of
 * packet batches or similar, normally 1).  out is [4][ny][nx]. */
int orc_image(const orc_problem *P, const double *S, int cam, double scale_S, double *out)
{
    const orc_camera *K = &P->cams[cam];
    double Om[3] = {K->dir[0], K->dir[1], K->dir[2]};
    double cth[3], cph[3];
    orc_stokes_basis(Om, cth, cph);
    double ex[3] = {cph[0], cph[1], cph[2]};
    double ey[3] = {-cth[0], -cth[1], -cth[2]};
    const int nx = K->npix[0], ny = K->npix[1];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double a = ((i + 0.5) / nx - 0.5) * K->fov[0];
            double b = ((j + 0.5) / ny - 0.5) * K->fov[1];
            double o[3];
            for (int d = 0; d < 3; ++d) o[d] = K->center[d] + a * ex[d] + b * ey[d];
            /* entry and exit of the box along Om */
            double tin = -INFINITY, tout = INFINITY;
            int miss = 0;
            for (int d = 0; d < 3; ++d) {
                if (Om[d] != 0.0) {
                    double t1 = (P->lo[d] - o[d]) / Om[d], t2 = (P->hi[d] - o[d]) / Om[d];
                    if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; }
                    if (t1 > tin) tin = t1;
                    if (t2 < tout) tout = t2;
                } else if (o[d] < P->lo[d] || o[d] > P->hi[d]) {
                    miss = 1;
                }
            }
            double X[4] = {0.0, 0.0, 0.0, 0.0};
            if (!miss && tin < tout) {
                double p[3];
                int ridx[3];
                where_t w;
                for (int d = 0; d < 3; ++d) p[d] = o[d] + tin * Om[d];
                for (int d = 0; d < 3; ++d) {
                    double dd = cell_size(P, d);
                    double x = (p[d] - P->lo[d]) / dd;
                    int ii = (int)floor(x);
                    if ((double)ii == x && Om[d] < 0.0) ii -= 1;
                    if (ii < 0) ii = 0;
                    if (ii >= P->n[d]) ii = P->n[d] - 1;
                    ridx[d] = ii;
                }
                enter_root_cell(P, ridx, p, Om, &w);
                for (;;) {
                    int axis;
                    double ell = composite_exit(P, &w, p, Om, &axis);
                    int64_t c = cell_index(P, &w);
                    double ka = cell_ka(P, c), ks = cell_ks(P, c);
                    double kext = ka + ks;
                    if (kext > 0.0 && ell > 0.0) {
                        double omega = ks / kext;
                        double V = grid_cell_volume(P, w.g);
                        local_frame F;
                        make_local_frame(P, c, Om, &F);
                        double Bc = cell_em(P, c);
                        double Sg[4] = {(F.alpha[0] - F.sca[0]) * Bc, (F.alpha[1] - F.sca[1]) * Bc, 0.0, 0.0};
                        if (S && ks > 0.0) {
                            double Sc[4], Sgs[4];
                            for (int e = 0; e < 4; ++e)
                                Sc[e] = scale_S * omega / V * S[((size_t)c * P->n_cam + cam) * 4 + e];
                            orc_change_basis(Sc, F.th, F.ph, F.gth, F.gph, Sgs);
                            for (int e = 0; e < 4; ++e) Sg[e] += Sgs[e];
                        }
                        double Xg[4], Yg[4];
                        orc_change_basis(X, F.th, F.ph, F.gth, F.gph, Xg);
                        orc_cell_solution(Xg, F.alpha[0], F.alpha[1], F.alpha[2], Sg, kext * ell, Yg);
                        orc_change_basis(Yg, F.gth, F.gph, F.th, F.ph, X);
                    }
                    if (!composite_cross(P, &w, p, Om, ell, axis, 0)) break;
                }
            }
            for (int e = 0; e < 4; ++e) out[((size_t)e * ny + j) * nx + i] = X[e];
        }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exported pieces for the tests.                                            */
/* ------------------------------------------------------------------------- */

/* Birth of packet pid: out = [x,y,z, nx,ny,nz, I,Q,U,V, tau, inside, source]. */
int orc_emit(const orc_problem *P, int64_t pid, double out[13])
{
    run_ctx C;
    memset(&C, 0, sizeof C);
    C.P = P;
    if (thermal_setup(&C) != 0) return -2;
    int64_t first;
    int s = find_source(P, pid, &first);
    if (s < 0) {
        free((void *)C.cdf);
        return -1;
    }
    double eps = source_luminosity(&C, s) / (double)P->sources[s].n_packets;
    double p[3], n[3], X[4], tau;
    where_t w;
    int inside = emit_packet(&C, pid, s, eps, p, n, X, &w, &tau);
    for (int a = 0; a < 3; ++a) { out[a] = p[a]; out[3 + a] = n[a]; }
    for (int e = 0; e < 4; ++e) out[6 + e] = X[e];
    out[10] = tau; out[11] = inside; out[12] = s;
    free((void *)C.cdf);
    return 0;
}

/* Local frame of cell c for direction n: out = [alpha1, alpha2, alpha3, s11, s12, gsca,
 * theta', gth(3), gph(3)]. */
void orc_frame(const orc_problem *P, int64_t c, const double n[3], double out[13])
{
    local_frame F;
    make_local_frame(P, c, n, &F);
    double v[13] = {F.alpha[0], F.alpha[1], F.alpha[2], F.sca[0], F.sca[1], F.gsca, F.thetap,
                    F.gth[0], F.gth[1], F.gth[2], F.gph[0], F.gph[1], F.gph[2]};
    memcpy(out, v, sizeof v);
}

/* One scattering of packet pid at scattering number n_sca with cell quaternion q:
 * out = [n2x,n2y,n2z, I,Q,U,V]; returns the trial count (negative: no acceptance). */
int orc_scatter(const orc_problem *P, int64_t pid, uint32_t n_sca, int bin, const double X[4],
                const double n[3], const double q[4], double out[7])
{
    double n2[3], Y[4];
    int t = scatter_sample(P, pid, n_sca, bin, X, n, q, n2, Y);
    for (int a = 0; a < 3; ++a) out[a] = n2[a];
    for (int e = 0; e < 4; ++e) out[3 + e] = Y[e];
    return t;
}
