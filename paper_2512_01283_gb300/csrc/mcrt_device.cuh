// mcrt_device.cuh -- device building blocks of the polarized Monte-Carlo transport
// (Kratos-polrad, arXiv:2512.01283), templated on the arithmetic type T (float for
// the production path, double for the FP64 instantiation).
//
// Frames follow Sec. 2.1: the grain frame is reached with the quaternion q_B of
// eq. (grain-quaternion) through (0, n_GF) = q_B^* (0, n) q_B (eq. vector-transform);
// Stokes bases are rotated by the signed angle eta of eq. (rotation-angle),
// sin(eta) = (phi_GF x phi') . n_GF, cos(eta) = phi_GF . phi', applied through the
// double-angle form of eq. (stokes-rotation) so that no trigonometric call is needed.
// The in-cell transfer is App. A written as e^{-K dtau} X0 + dtau E(K dtau) S with
// E(x) = (1 - e^{-x}) / x evaluated with expm1, which equals the printed
// I_s + (I0 - I_s) e^{...} form and stays accurate in thin cells.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mcrt {

// ---------------------------------------------------------------------------------
// scalar helpers that pick the float or double routine
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float t_exp(float x) { return expf(x); }
__device__ __forceinline__ double t_exp(double x) { return exp(x); }
__device__ __forceinline__ float t_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double t_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float t_log(float x) { return logf(x); }
__device__ __forceinline__ double t_log(double x) { return log(x); }
__device__ __forceinline__ float t_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double t_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float t_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double t_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float t_acos(float x) { return acosf(x); }
__device__ __forceinline__ double t_acos(double x) { return acos(x); }
__device__ __forceinline__ void t_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void t_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void t_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void t_sincos(double x, double* s, double* c) { sincos(x, s, c); }

template <typename T> struct V3 {
    T x, y, z;
};
template <typename T> __device__ __forceinline__ V3<T> v3(T x, T y, T z) { return V3<T>{x, y, z}; }
template <typename T> __device__ __forceinline__ T dot(const V3<T>& a, const V3<T>& b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename T> __device__ __forceinline__ V3<T> cross(const V3<T>& a, const V3<T>& b) {
    return V3<T>{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename T> __device__ __forceinline__ V3<T> axpy(T s, const V3<T>& a, const V3<T>& b) {
    return V3<T>{s * a.x + b.x, s * a.y + b.y, s * a.z + b.z};
}

// ---------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies with
// the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// kept out of line so that the kernel holds one copy of the ten rounds
static __host__ __device__ __noinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                  uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t a = 0xD2511F53u * c0, ah = mulhi32(0xD2511F53u, c0);
        const uint32_t b = 0xCD9E8D57u * c2, bh = mulhi32(0xCD9E8D57u, c2);
        const uint32_t n0 = bh ^ c1 ^ k0;
        const uint32_t n2 = ah ^ c3 ^ k1;
        c0 = n0;
        c1 = b;
        c2 = n2;
        c3 = a;
    }
    return U4{c0, c1, c2, c3};
}

// u = ((x >> 8) | 1) 2^-24: odd multiples of 2^-24 in (0, 1), exact in FP32 and FP64.
template <typename T> __device__ __forceinline__ T u01(uint32_t x) {
    return T((x >> 8) | 1u) * T(5.9604644775390625e-8);
}

template <typename T> struct Draw4 {
    T a, b, c, d;
};

// counter = (pid_lo, pid_hi, event, slot), key = (seed, stream)
template <typename T>
__device__ __forceinline__ Draw4<T> draw4(long long pid, uint32_t event, uint32_t slot, uint32_t seed,
                                          uint32_t stream) {
    const U4 r = philox4x32_10((uint32_t)((unsigned long long)pid & 0xffffffffull),
                               (uint32_t)((unsigned long long)pid >> 32), event, slot, seed, stream);
    return Draw4<T>{u01<T>(r.x), u01<T>(r.y), u01<T>(r.z), u01<T>(r.w)};
}

// ---------------------------------------------------------------------------------
// quaternion rotations with q = (s, w), |q| = 1
//   to_lab:   q (0,v) q^*  = v + 2 s (w x v) + 2 w x (w x v)
//   to_grain: q^* (0,v) q  = v - 2 s (w x v) + 2 w x (w x v)
// ---------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ V3<T> quat_to_lab(const float4& q, const V3<T>& v) {
    const V3<T> w{T(q.y), T(q.z), T(q.w)};
    const T s = T(q.x);
    const V3<T> t = cross(w, v);
    const V3<T> tt = cross(w, t);
    return V3<T>{v.x + T(2) * (s * t.x + tt.x), v.y + T(2) * (s * t.y + tt.y), v.z + T(2) * (s * t.z + tt.z)};
}
template <typename T> __device__ __forceinline__ V3<T> quat_to_grain(const float4& q, const V3<T>& v) {
    const V3<T> w{T(q.y), T(q.z), T(q.w)};
    const T s = T(q.x);
    const V3<T> t = cross(w, v);
    const V3<T> tt = cross(w, t);
    return V3<T>{v.x + T(2) * (tt.x - s * t.x), v.y + T(2) * (tt.y - s * t.y), v.z + T(2) * (tt.z - s * t.z)};
}

// ---------------------------------------------------------------------------------
// Stokes basis of n without trigonometry: phi-hat = (-n_y, n_x, 0) / rho,
// theta-hat = phi-hat x n; at the poles phi-hat = (0, 1, 0).
// ---------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ void stokes_basis(const V3<T>& n, V3<T>& th, V3<T>& ph) {
    const T r2 = n.x * n.x + n.y * n.y;
    if (r2 > T(0)) {
        const T r = t_rsqrt(r2);
        ph = V3<T>{-n.y * r, n.x * r, T(0)};
    } else {
        ph = V3<T>{T(0), T(1), T(0)};
    }
    th = cross(ph, n);
}

__device__ __forceinline__ float t_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double t_rcp(double x) { return 1.0 / x; }
// quotient: the fast reciprocal-based form in FP32 (about 2 ulp), exact in FP64
__device__ __forceinline__ float t_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double t_div(double a, double b) { return a / b; }

// (cos 2psi, sin 2psi) from any (A, B) proportional to (cos psi, sin psi); (1, 0)
// for A = B = 0.  Tiny inputs are rescaled first so that 1/r cannot overflow.
template <typename T> __device__ __forceinline__ void double_angle(T A, T B, T& c2, T& s2) {
    T r = A * A + B * B;
    if (!(r >= T(1e-30))) {
        const T m = fmax(fabs(A), fabs(B));
        if (!(m > T(0))) {
            c2 = T(1);
            s2 = T(0);
            return;
        }
        A = A / m;
        B = B / m;
        r = A * A + B * B;
    }
    const T inv = t_rcp(r);
    c2 = (A * A - B * B) * inv;
    s2 = T(2) * A * B * inv;
}

// eq. (stokes-rotation): (Q', U') = [[c2, s2], [-s2, c2]] (Q, U)
template <typename T> __device__ __forceinline__ void rotate_qu(T& Q, T& U, T c2, T s2) {
    const T q = c2 * Q + s2 * U;
    const T u = -s2 * Q + c2 * U;
    Q = q;
    U = u;
}

// Grain-meridian frame of direction n in a cell with grain quaternion q:
// (cos 2eta, sin 2eta) of eq. (rotation-angle) (signed) and cos theta'.
template <typename T> struct GrainFrame {
    T c2, s2, cos_tp;
};

template <typename T>
__device__ __forceinline__ GrainFrame<T> grain_frame(const float4& q, const V3<T>& n, const V3<T>& ph_lab) {
    const V3<T> nGF = quat_to_grain(q, n);
    const V3<T> phGF = quat_to_grain(q, ph_lab);
    // phi' of n_GF up to a positive factor; (0, 1, 0) along the grain axis
    V3<T> php{-nGF.y, nGF.x, T(0)};
    if (php.x == T(0) && php.y == T(0)) php.y = T(1);
    const T cos_eta = dot(phGF, php);
    const T sin_eta = dot(cross(phGF, php), nGF);
    GrainFrame<T> f;
    double_angle(cos_eta, sin_eta, f.c2, f.s2);
    f.cos_tp = nGF.z;
    return f;
}

// ---------------------------------------------------------------------------------
// App. A transfer over optical depth dtau for the block matrix
//   M = [[a, a2, 0, 0], [a2, a, 0, 0], [0, 0, a, a3], [0, 0, -a3, a]]
// Y = e^{-M dtau} X  and  W = int_0^dtau e^{-M t} dt X  (both optional)
// I+Q, I-Q decay at a +- a2; U + iV at a - i a3.
// ---------------------------------------------------------------------------------
// E(x) = (1 - e^{-x}) / x
template <typename T> __device__ __forceinline__ T e1(T x) {
    if (fabs(x) < T(1e-4)) return T(1) - x * (T(0.5) - x * T(1.0 / 6.0));
    return t_div(-t_expm1(-x), x);
}

// int_0^1 e^{-(x - i y) s} ds = (re, im)
template <typename T> __device__ __forceinline__ void e1_complex(T x, T y, T& re, T& im) {
    if (y == T(0)) {
        re = e1(x);
        im = T(0);
        return;
    }
    if (fabs(x) + fabs(y) < T(1e-4)) {
        re = T(1) - x * T(0.5) + (x * x - y * y) * T(1.0 / 6.0);
        im = y * T(0.5) - x * y * T(1.0 / 3.0);
        return;
    }
    T sh, ch, sy, cy;
    t_sincos(T(0.5) * y, &sh, &ch);
    sy = T(2) * sh * ch;
    const T ex = t_exp(-x);
    const T nr = -t_expm1(-x) + T(2) * ex * sh * sh;  // 1 - e^{-x} cos y
    const T ni = ex * sy;                               // e^{-x} sin y
    const T den = t_rcp(x * x + y * y);
    re = (nr * x + ni * y) * den;
    im = (nr * y - ni * x) * den;
    (void)cy;
}

// Y = e^{-M dtau} X; with want_W also W = wscale * int_0^1 e^{-M dtau s} ds X
// (wscale = dtau gives the optical-depth integral, wscale = ell the path-length one,
// which needs no division by kappa_ext).  For |a2 dtau| <= 10 the I-Q block uses the
// cosh/sinh form of App. A (no cancellation in Q); beyond, the eigen-decay form, whose
// factors underflow to zero instead of overflowing.
template <typename T>
__device__ __forceinline__ void transfer(const T X[4], T a, T a2, T a3, T dtau, T Y[4], T W[4], bool want_W,
                                         T wscale) {
    const T xa = a * dtau, xb = a2 * dtau, ya = a3 * dtau;
    const T xp = xa + xb, xm = xa - xb;
    const T ea = t_exp(-xa);
    if (fabs(xb) <= T(10)) {
        // e^{-xb} - 1 = -m / (1 + m) with m = e^{xb} - 1: no cancellation, one expm1
        const T e1p = t_expm1(xb), e1m = -e1p * t_rcp(T(1) + e1p);
        const T sh = T(0.5) * (e1p - e1m), ch = T(1) + T(0.5) * (e1p + e1m);
        Y[0] = ea * (ch * X[0] - sh * X[1]);
        Y[1] = ea * (ch * X[1] - sh * X[0]);
    } else {
        const T sp = X[0] + X[1], sm = X[0] - X[1];
        const T ep = t_exp(-xp), em = t_exp(-xm);
        Y[0] = T(0.5) * (ep * sp + em * sm);
        Y[1] = T(0.5) * (ep * sp - em * sm);
    }
    T s3 = T(0), c3 = T(1);
    if (ya != T(0)) t_sincos(ya, &s3, &c3);
    Y[2] = ea * (c3 * X[2] - s3 * X[3]);
    Y[3] = ea * (s3 * X[2] + c3 * X[3]);
    if (want_W) {
        const T sp = X[0] + X[1], sm = X[0] - X[1];
        const T Ep = wscale * e1(xp), Em = wscale * e1(xm);
        W[0] = T(0.5) * (Ep * sp + Em * sm);
        W[1] = T(0.5) * (Ep * sp - Em * sm);
        T re, im;
        e1_complex(xa, ya, re, im);
        re *= wscale;
        im *= wscale;
        W[2] = re * X[2] - im * X[3];
        W[3] = re * X[3] + im * X[2];
    }
}

// Full App. A cell step with source S (per unit dtau) and the extinction matrix K:
// X <- e^{-K dtau} X + (int_0^dtau e^{-K t} dt) S
template <typename T> __device__ __forceinline__ void cell_step(T X[4], T a1, T a2, T a3, const T S[4], T dtau) {
    T Y[4], W[4], Z[4];
    transfer(X, a1, a2, a3, dtau, Y, W, false, dtau);
    transfer(S, a1, a2, a3, dtau, Z, W, true, dtau);
    for (int e = 0; e < 4; ++e) X[e] = Y[e] + W[e];
}

// ---------------------------------------------------------------------------------
// scattering matrices in the scattering-plane basis: P11,P12,P22,P33,P34,P44
// ---------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ void rayleigh_matrix(T mu, T P[6]) {
    const T f = T(0.059683103659460665);  // 3 / (16 pi)
    P[0] = f * (T(1) + mu * mu);
    P[1] = f * (mu * mu - T(1));
    P[2] = P[0];
    P[3] = f * T(2) * mu;
    P[4] = T(0);
    P[5] = P[3];
}

// Transfer of X (basis of n) through a scattering n -> n2 with matrix P to the
// basis (th2, ph2) of n2.  Scattering-plane basis: e_perp ~ n x n2 and
// e_par = e_perp x n (x n2 after scattering); when sin(Theta) < 1e-6 the plane is
// undefined and e_perp = phi-hat(n).
template <typename T> struct PlaneRot {
    T c1, s1, c2, s2;
};

// With e = n x n2 the rotation inputs are projections: e.phi(n) = n2.theta(n),
// -e.theta(n) = n2.phi(n), e.phi(n2) = -n.theta(n2), e.theta(n2) = n.phi(n2).
template <typename T>
__device__ __forceinline__ PlaneRot<T> plane_rotation(const V3<T>& n, const V3<T>& th, const V3<T>& ph,
                                                      const V3<T>& n2, const V3<T>& th2, const V3<T>& ph2) {
    T A1 = dot(n2, th), B1 = dot(n2, ph);
    T A2 = -dot(n, th2), B2 = dot(n, ph2);
    if (A1 * A1 + B1 * B1 < T(1e-12)) {  // sin(Theta) < 1e-6: plane undefined, e_perp = phi(n)
        A1 = T(1);
        B1 = T(0);
        A2 = dot(ph, ph2);
        B2 = dot(ph, th2);
    }
    PlaneRot<T> r;
    double_angle(A1, B1, r.c1, r.s1);
    double_angle(A2, B2, r.c2, r.s2);
    return r;
}

// Incident Q in the scattering-plane basis only (rejection test).
template <typename T>
__device__ __forceinline__ T plane_Q(const V3<T>& th, const V3<T>& ph, const V3<T>& n2, const T X[4]) {
    const T A1 = dot(n2, th), B1 = dot(n2, ph);
    if (A1 * A1 + B1 * B1 < T(1e-12)) return X[1];
    T c1, s1;
    double_angle(A1, B1, c1, s1);
    return c1 * X[1] + s1 * X[2];
}

template <typename T> __device__ __forceinline__ void apply_plane(const PlaneRot<T>& r, const T P[6], const T X[4], T Y[4]) {
    const T Qs = r.c1 * X[1] + r.s1 * X[2];
    const T Us = -r.s1 * X[1] + r.c1 * X[2];
    const T I2 = P[0] * X[0] + P[1] * Qs;
    const T Q2 = P[1] * X[0] + P[2] * Qs;
    const T U2 = P[3] * Us + P[4] * X[3];
    const T V2 = -P[4] * Us + P[5] * X[3];
    Y[0] = I2;
    Y[1] = r.c2 * Q2 + r.s2 * U2;
    Y[2] = -r.s2 * Q2 + r.c2 * U2;
    Y[3] = V2;
}

// ---------------------------------------------------------------------------------
// aligned dipole spheroids (Sec. 2.1 dipole approximation, Sec. 3 optical theorem)
// ---------------------------------------------------------------------------------
// First row of K per unit kappa_ext in the grain-meridian basis at cos theta' = ct, and
// its scattering part (s11, s12).  A field along theta-hat' sees the symmetry axis with
// weight sin^2 theta', one along phi-hat' not at all; each process' cross section is
// c0 + (c1 - c0) w over its orientation average (ca: absorption, cs: scattering), and
// fa, fs are kappa_abs / kappa_ext and kappa_sca / kappa_ext.
template <typename T>
__device__ __forceinline__ void dipole_K(T ca0, T ca1, T cs0, T cs1, T fa, T fs, T ct, T& a1, T& a2, T& s11, T& s12) {
    T S2 = (T(1) - ct) * (T(1) + ct);
    S2 = S2 > T(0) ? S2 : T(0);
    const T ha = (ca1 - ca0) * T(0.5) * S2;
    const T hs = (cs1 - cs0) * T(0.5) * S2;
    s11 = fs * (cs0 + hs);
    s12 = fs * hs;
    a1 = fa * (ca0 + ha) + s11;
    a2 = fa * ha + s12;
}

// Y = Zhat X for the scattering n -> n2 by a spheroid with symmetry axis ax: X in the
// Stokes basis (th, ph) of n, Y in the basis (th2, ph2) of n2.  The induced dipole is
// alpha'_0 (1 + (rho - 1) ax ax^T) E and the far field along n2 its transverse part, so
// the Jones matrix is J_jk = f2_j . f_k + (rho - 1) (f2_j . ax)(ax . f_k); the coherency
// matrix C = 1/2 [[I+Q, U+iV], [U-iV, I-Q]] goes to J C J^H, scaled by zn.
template <typename T>
__device__ __forceinline__ void dipole_apply(T rho_re, T rho_im, T zn, const V3<T>& ax, const V3<T>& th,
                                             const V3<T>& ph, const V3<T>& th2, const V3<T>& ph2, const T X[4],
                                             T Y[4]) {
    const T rr = rho_re - T(1);
    const T g0 = dot(th2, ax), g1 = dot(ph2, ax), b0 = dot(ax, th), b1 = dot(ax, ph);
    // J = (Jr + i Ji)
    const T Jr00 = dot(th2, th) + rr * g0 * b0, Ji00 = rho_im * g0 * b0;
    const T Jr01 = dot(th2, ph) + rr * g0 * b1, Ji01 = rho_im * g0 * b1;
    const T Jr10 = dot(ph2, th) + rr * g1 * b0, Ji10 = rho_im * g1 * b0;
    const T Jr11 = dot(ph2, ph) + rr * g1 * b1, Ji11 = rho_im * g1 * b1;
    // C (Hermitian): c00, c11 real, c01 = cr + i ci, c10 = conj(c01)
    const T c00 = T(0.5) * (X[0] + X[1]), c11 = T(0.5) * (X[0] - X[1]);
    const T cr = T(0.5) * X[2], ci = T(0.5) * X[3];
    // M = J C
    const T Mr00 = Jr00 * c00 + Jr01 * cr + Ji01 * ci, Mi00 = Ji00 * c00 + Ji01 * cr - Jr01 * ci;
    const T Mr01 = Jr00 * cr - Ji00 * ci + Jr01 * c11, Mi01 = Jr00 * ci + Ji00 * cr + Ji01 * c11;
    const T Mr10 = Jr10 * c00 + Jr11 * cr + Ji11 * ci, Mi10 = Ji10 * c00 + Ji11 * cr - Jr11 * ci;
    const T Mr11 = Jr10 * cr - Ji10 * ci + Jr11 * c11, Mi11 = Jr10 * ci + Ji10 * cr + Ji11 * c11;
    // D = M J^H: D_jk = sum_l M_jl conj(J_kl)
    const T D00 = Mr00 * Jr00 + Mi00 * Ji00 + Mr01 * Jr01 + Mi01 * Ji01;
    const T D11 = Mr10 * Jr10 + Mi10 * Ji10 + Mr11 * Jr11 + Mi11 * Ji11;
    const T Dr01 = Mr00 * Jr10 + Mi00 * Ji10 + Mr01 * Jr11 + Mi01 * Ji11;
    const T Di01 = Mi00 * Jr10 - Mr00 * Ji10 + Mi01 * Jr11 - Mr01 * Ji11;
    Y[0] = zn * (D00 + D11);
    Y[1] = zn * (D00 - D11);
    Y[2] = zn * T(2) * Dr01;
    Y[3] = zn * T(2) * Di01;
}

// ---------------------------------------------------------------------------------
// uniform grid: exit distance of cell idx along n; ties go to the lowest axis
// ---------------------------------------------------------------------------------
template <typename T> struct GridT {
    int n[3];
    T lo[3], d[3];
};

template <typename T>
__device__ __forceinline__ T exit_distance(const GridT<T>& g, const int idx[3], const T p[3], const T n[3], int& axis) {
    T best = T(INFINITY);
    axis = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T t;
        if (n[a] > T(0))
            t = (g.lo[a] + T(idx[a] + 1) * g.d[a] - p[a]) / n[a];
        else if (n[a] < T(0))
            t = (g.lo[a] + T(idx[a]) * g.d[a] - p[a]) / n[a];
        else
            continue;
        if (t < T(0)) t = T(0);
        if (t < best) {
            best = t;
            axis = a;
        }
    }
    return best;
}

// Moves p to the exit face and steps the index; false when the packet leaves the grid.
template <typename T>
__device__ __forceinline__ bool cross_face(const GridT<T>& g, int idx[3], T p[3], const T n[3], T ell, int axis) {
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] += ell * n[a];
    if (n[axis] > T(0)) {
        p[axis] = g.lo[axis] + T(idx[axis] + 1) * g.d[axis];
        idx[axis] += 1;
    } else {
        p[axis] = g.lo[axis] + T(idx[axis]) * g.d[axis];
        idx[axis] -= 1;
    }
    return idx[axis] >= 0 && idx[axis] < g.n[axis];
}

// Cell of p for travel along n (a point on a face belongs to the cell n points
// into); false outside the grid.
template <typename T> __device__ __forceinline__ bool locate(const GridT<T>& g, const T p[3], const T n[3], int idx[3]) {
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T x = (p[a] - g.lo[a]) / g.d[a];
        int i = (int)floor(x);
        if (T(i) == x && n[a] < T(0)) i -= 1;
        idx[a] = i;
        in = in && (i >= 0 && i < g.n[a]);
    }
    return in;
}

}  // namespace mcrt
