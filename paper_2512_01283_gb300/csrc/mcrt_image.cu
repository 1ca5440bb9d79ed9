// mcrt_image.cu -- step 2 of the two-step scheme (Kratos-polrad, arXiv:2512.01283,
// Sec. 2.3): deterministic ray-march of every pixel toward the camera, integrating
// the vector transfer equation (eq. polarized-rt) cell by cell with the analytic
// in-cell solution of App. A.  The per-cell source is the emission alpha_abs B plus
// the step-1 scattering source S = omega / V * T_c, both turned into the
// grain-meridian basis with the signed eta rotation of Sec. 2.1.
#include <cuda/std/complex>

#include "mcrt_device.cuh"
#include "mcrt_internal.h"
#include "mcrt_refine.cuh"

namespace mcrt {

namespace {

template <typename T>
__device__ __forceinline__ void kext_lookup(const TablesDev& t, T cos_tp, T& a1, T& a2, T& a3) {
    if (t.k_const) {
        const float4 k = t.kext[0];
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
    const float4 k0 = t.kext[j], k1 = t.kext[j + 1];
    a1 = (T(1) - f) * T(k0.x) + f * T(k1.x);
    a2 = (T(1) - f) * T(k0.y) + f * T(k1.y);
    a3 = (T(1) - f) * T(k0.z) + f * T(k1.z);
}

template <typename T> __global__ void __launch_bounds__(128) k_image(const __grid_constant__ ImageParams P) {
    const int nx = P.npix[0], ny = P.npix[1];
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (long long)nx * ny) return;
    const int ix = (int)(pix % nx), iy = (int)(pix / nx);
    GridT<T> g;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = P.g.n[a];
        g.lo[a] = T(P.g.lo[a]);
        g.d[a] = T(P.g.d[a]);
    }
    const V3<T> Om{T(P.cam.dir[0]), T(P.cam.dir[1]), T(P.cam.dir[2])};
    const V3<T> thc{T(P.cam.th[0]), T(P.cam.th[1]), T(P.cam.th[2])};
    const V3<T> phc{T(P.cam.ph[0]), T(P.cam.ph[1]), T(P.cam.ph[2])};
    // image plane: e_x = phi-hat(Omega), e_y = -theta-hat(Omega)
    const T a = (T((double)(ix) + 0.5) / T(nx) - T(0.5)) * T(P.fov[0]);
    const T b = (T((double)(iy) + 0.5) / T(ny) - T(0.5)) * T(P.fov[1]);
    const T o[3] = {T(P.center[0]) + a * phc.x - b * thc.x, T(P.center[1]) + a * phc.y - b * thc.y,
                    T(P.center[2]) + a * phc.z - b * thc.z};
    const T dir[3] = {Om.x, Om.y, Om.z};
    T tin = -T(INFINITY), tout = T(INFINITY);
    bool miss = false;
    for (int d = 0; d < 3; ++d) {
        if (dir[d] != T(0)) {
            T t1 = (T(P.g.lo[d]) - o[d]) / dir[d], t2 = (T(P.g.hi[d]) - o[d]) / dir[d];
            if (t1 > t2) {
                const T tt = t1;
                t1 = t2;
                t2 = tt;
            }
            tin = t1 > tin ? t1 : tin;
            tout = t2 < tout ? t2 : tout;
        } else if (o[d] < T(P.g.lo[d]) || o[d] > T(P.g.hi[d])) {
            miss = true;
        }
    }
    T X[4] = {T(0), T(0), T(0), T(0)};
    if (!miss && tin < tout) {
        T p[3];
        int idx[3];
        for (int d = 0; d < 3; ++d) p[d] = o[d] + tin * dir[d];
        for (int d = 0; d < 3; ++d) {
            const T x = (p[d] - g.lo[d]) / g.d[d];
            int i = (int)floor(x);
            if (T(i) == x && dir[d] < T(0)) i -= 1;
            i = i < 0 ? 0 : (i >= g.n[d] ? g.n[d] - 1 : i);
            idx[d] = i;
        }
        const T inv_vol_root = T(1.0 / (P.g.d[0] * P.g.d[1] * P.g.d[2]));
        T inv_vol = inv_vol_root;
        // composite grid: the current level's geometry (root, or the patch the ray is in)
        GridT<T> gc = g;
        int lvl = 0;
        auto descend = [&]() {
            const long long rc = ((long long)idx[2] * g.n[1] + idx[1]) * g.n[0] + idx[0];
            const int q = covering_patch(P.g.cells[2 * rc + 1]);
            if (q < 0) return;
            const PatchDev& pq = P.g.patches[q];
            lvl = q + 1;
            for (int a = 0; a < 3; ++a) {
                gc.n[a] = pq.n[a];
                gc.lo[a] = patch_lo<T>(pq, a);
                gc.d[a] = patch_d<T>(pq, a);
            }
            inv_vol = T(1.0 / (pq.d[0] * pq.d[1] * pq.d[2]));
            patch_locate<T>(pq, p[0], p[1], p[2], dir[0], dir[1], dir[2], idx);
        };
        if (P.g.n_patches > 0) descend();
        const long long max_steps =
            (long long)(g.n[0] + g.n[1] + g.n[2]) * (P.g.n_patches > 0 ? 3 * 16 + 1 : 1) + 3;
        for (long long step = 0; step < max_steps; ++step) {
            int axis;
            const T ell = exit_distance(gc, idx, p, dir, axis);
            if (axis < 0) break;
            const long long c = lvl == 0 ? ((long long)idx[2] * g.n[1] + idx[1]) * g.n[0] + idx[0]
                                         : patch_cell(P.g.patches[lvl - 1], idx[0], idx[1], idx[2]);
            const float4 r = P.g.cells[2 * c + 1];
            const T ks = T(r.y);
            const T kext = T(r.x) + ks;
            if (kext > T(0) && ell > T(0)) {
                const T omega = ks / kext;
                T c2 = T(1), s2 = T(0), a1, a2, a3;
                T s11 = omega, s12 = T(0);  // scattering part of K's first row
                if (P.t.model == MCRT_SCAT_DIPOLE) {
                    const GrainFrame<T> f = grain_frame(P.g.cells[2 * c], Om, phc);
                    c2 = f.c2;
                    s2 = f.s2;
                    const DipoleConst<T> dp = dipole_const<T>(P.t.dip);
                    dipole_K(dp.ca0, dp.ca1, dp.cs0, dp.cs1, T(r.x) / kext, omega, f.cos_tp, a1,
                             a2, s11, s12);
                    a3 = T(0);
                } else if (P.t.k_iso) {
                    a1 = T(P.t.kext[0].x);
                    a2 = T(0);
                    a3 = T(0);
                } else {
                    const float4 q = P.g.cells[2 * c];
                    const GrainFrame<T> f = grain_frame(q, Om, phc);
                    c2 = f.c2;
                    s2 = f.s2;
                    kext_lookup(P.t, f.cos_tp, a1, a2, a3);
                }
                const T B = T(r.z);
                // emission: the absorption part of K acting on (B, 0, 0, 0)
                T S[4] = {(a1 - s11) * B, (a2 - s12) * B, T(0), T(0)};
                if (P.S && ks > T(0)) {
                    const double* Sc = P.S + ((size_t)c * P.n_cam + P.cam_index) * 4;
                    const T f = omega * inv_vol;
                    T s1 = f * T(Sc[1]), s2v = f * T(Sc[2]);
                    rotate_qu(s1, s2v, c2, s2);
                    S[0] += f * T(Sc[0]);
                    S[1] += s1;
                    S[2] += s2v;
                    S[3] += f * T(Sc[3]);
                }
                rotate_qu(X[1], X[2], c2, s2);
                cell_step(X, a1, a2, a3, S, kext * ell);
                rotate_qu(X[1], X[2], c2, -s2);
            }
            if (lvl == 0) {
                if (!cross_face(g, idx, p, dir, ell, axis)) break;
                if (P.g.n_patches > 0) descend();
            } else if (!cross_face(gc, idx, p, dir, ell, axis)) {
                // out of the patch: the root cell beyond its face
                const PatchDev& pq = P.g.patches[lvl - 1];
                for (int a = 0; a < 3; ++a) idx[a] = pq.box[a] + (a == axis ? 0 : idx[a] / pq.factor);
                idx[axis] = dir[axis] > T(0) ? pq.box[3 + axis] : pq.box[axis] - 1;
                lvl = 0;
                gc = g;
                inv_vol = inv_vol_root;
                if (idx[axis] < 0 || idx[axis] >= g.n[axis]) break;
                descend();
            }
        }
    }
    for (int e = 0; e < 4; ++e) P.out[((size_t)e * ny + iy) * nx + ix] = (double)X[e];
}

// ---------------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------------

// q_B of eq. (grain-quaternion) from the field direction angles (theta_B, phi_B),
// computed in FP64; phi_B = 0 along z; q_B = 1 for a zero field.
__device__ float4 quat_from_field(double bx, double by, double bz) {
    const double bn = sqrt(bx * bx + by * by + bz * bz);
    if (!(bn > 0.0)) return make_float4(1.f, 0.f, 0.f, 0.f);
    double cz = bz / bn;
    cz = cz > 1.0 ? 1.0 : (cz < -1.0 ? -1.0 : cz);
    const double thB = acos(cz);
    const double phB = (bx == 0.0 && by == 0.0) ? 0.0 : atan2(by, bx);
    double sp, cp, st, ct;
    sincos(0.5 * phB, &sp, &cp);
    sincos(0.5 * thB, &st, &ct);
    return make_float4((float)(cp * ct), (float)(-sp * st), (float)(cp * st), (float)(sp * ct));
}

// Cell records: q_B as float4, then (kappa_abs, kappa_sca, emissivity, 0).  Inputs
// that are negative or not finite set *bad.
__global__ void k_setup_cells(const float* __restrict__ ka, const float* __restrict__ ks,
                              const float* __restrict__ bf, const float* __restrict__ em, long long ncell,
                              float4* __restrict__ cells, unsigned* __restrict__ bad) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const float a = ka[c], s = ks[c], e = em ? em[c] : 0.f;
        bool ok = isfinite(a) && isfinite(s) && isfinite(e) && a >= 0.f && s >= 0.f && e >= 0.f;
        float4 q = make_float4(1.f, 0.f, 0.f, 0.f);
        if (bf) {
            const float bx = bf[3 * c], by = bf[3 * c + 1], bz = bf[3 * c + 2];
            ok = ok && isfinite(bx) && isfinite(by) && isfinite(bz);
            if (ok) q = quat_from_field(bx, by, bz);
        }
        if (!ok) atomicOr(bad, 1u);
        cells[2 * c] = q;
        cells[2 * c + 1] = make_float4(ok ? a : 0.f, ok ? s : 0.f, ok ? e : 0.f, 0.f);
    }
}

// Table preparation (one block): mixture matrix for the tally, per-bin rows,
// piecewise-constant envelope of P11 with its normalised cumulative weights,
// cumulative bin weights, extinction rows and the sphere average of alpha1.  The two
// cumulative tables are followed by their FP32 copies (env_cdf holds n_bins (n_theta - 1)
// doubles and as many floats, bin_cdf n_bins doubles and n_bins floats).
__global__ void k_prepare_tables(int model, int n_bins, int n_theta, int n_ktheta, const float* __restrict__ mueller,
                                 const float* __restrict__ bin_weight, const float* __restrict__ kext,
                                 float4* __restrict__ mix, float4* __restrict__ bins, double* __restrict__ env_cdf,
                                 float* __restrict__ env, double* __restrict__ bin_cdf, float4* __restrict__ kext4,
                                 double* __restrict__ alpha1_mean) {
    const double pi = 3.141592653589793;
    for (int j = threadIdx.x; j < n_ktheta; j += blockDim.x)
        kext4[j] = make_float4(kext[3 * j], kext[3 * j + 1], kext[3 * j + 2], 0.f);
    if (threadIdx.x == 0) {
        const double h = pi / (n_ktheta - 1);
        double s = 0.0;
        for (int j = 0; j + 1 < n_ktheta; ++j) {
            const double ta = j * h, tb = (j + 1) * h;
            const double A = kext[3 * j], B = ((double)kext[3 * (j + 1)] - A) / h;
            s += A * (cos(ta) - cos(tb)) + B * (-(tb - ta) * cos(tb) + sin(tb) - sin(ta));
        }
        *alpha1_mean = 0.5 * s;
    }
    if (model != MCRT_SCAT_TABLE) return;
    __shared__ double wsum_s;
    if (threadIdx.x == 0) {
        double ws = 0.0;
        for (int k = 0; k < n_bins; ++k) ws += bin_weight[k];
        double acc = 0.0;
        for (int k = 0; k < n_bins; ++k) {
            acc += bin_weight[k];
            bin_cdf[k] = acc / ws;
        }
        wsum_s = ws;
    }
    __syncthreads();
    const double ws = wsum_s;
    for (int j = threadIdx.x; j < n_theta; j += blockDim.x) {
        double m[6] = {0, 0, 0, 0, 0, 0};
        for (int k = 0; k < n_bins; ++k) {
            const float* row = mueller + ((size_t)k * n_theta + j) * 6;
            bins[((size_t)k * n_theta + j) * 2] = make_float4(row[0], row[1], row[2], row[3]);
            bins[((size_t)k * n_theta + j) * 2 + 1] = make_float4(row[4], row[5], 0.f, 0.f);
            for (int e = 0; e < 6; ++e) m[e] += (double)bin_weight[k] / ws * row[e];
        }
        mix[2 * j] = make_float4((float)m[0], (float)m[1], (float)m[2], (float)m[3]);
        mix[2 * j + 1] = make_float4((float)m[4], (float)m[5], 0.f, 0.f);
    }
    const int nint = n_theta - 1;
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) {
        const float* tab = mueller + (size_t)k * n_theta * 6;
        double tot = 0.0;
        for (int j = 0; j < nint; ++j) {
            const double e = fmax((double)tab[j * 6], (double)tab[(j + 1) * 6]);
            tot += e * (cos(pi * j / nint) - cos(pi * (j + 1) / nint));
            env[(size_t)k * nint + j] = (float)e;
            env_cdf[(size_t)k * nint + j] = tot;
        }
        for (int j = 0; j < nint; ++j) env_cdf[(size_t)k * nint + j] /= tot;
    }
    // FP32 copies after the FP64 tables
    __syncthreads();
    float* env_cdf_f = reinterpret_cast<float*>(env_cdf + (size_t)n_bins * nint);
    float* bin_cdf_f = reinterpret_cast<float*>(bin_cdf + n_bins);
    for (int i = threadIdx.x; i < n_bins * nint; i += blockDim.x) env_cdf_f[i] = (float)env_cdf[i];
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) bin_cdf_f[k] = (float)bin_cdf[k];
}

// Thermal emission weights kappa_ext (mean alpha1 - omega) B V and their inclusive
// prefix sum over cells (block scan, block-sum scan, add).
constexpr int kScanBlock = 256;
constexpr int kScanItems = 16;

__global__ void k_scan_local(const float4* __restrict__ cells, long long ncell, double alpha1_mean, double vol,
                             long long ncell_root, int n_patches, const PatchDev* __restrict__ patches,
                             double* __restrict__ cdf, double* __restrict__ block_sums) {
    __shared__ double sh[kScanBlock];
    const long long base = (long long)blockIdx.x * kScanBlock * kScanItems + (long long)threadIdx.x * kScanItems;
    double v[kScanItems];
    double run = 0.0;
    for (int i = 0; i < kScanItems; ++i) {
        const long long c = base + i;
        double w = 0.0;
        if (c < ncell) {
            const float4 r = cells[2 * c + 1];
            const double kext = (double)r.x + (double)r.y;
            const double omega = kext > 0.0 ? (double)r.y / kext : 0.0;
            double v = vol;  // the cell's own volume; covered root cells hold no emission
            if (c >= ncell_root)
                for (int q = n_patches - 1; q >= 0; --q)
                    if (c >= patches[q].offset) {
                        v = patches[q].d[0] * patches[q].d[1] * patches[q].d[2];
                        break;
                    }
            w = kext * (alpha1_mean - omega) * (double)r.z * v;
            if (w < 0.0) w = 0.0;
        }
        run += w;
        v[i] = run;
    }
    sh[threadIdx.x] = run;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {
        const double add = threadIdx.x >= off ? sh[threadIdx.x - off] : 0.0;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    const double prefix = threadIdx.x > 0 ? sh[threadIdx.x - 1] : 0.0;
    for (int i = 0; i < kScanItems; ++i) {
        const long long c = base + i;
        if (c < ncell) cdf[c] = v[i] + prefix;
    }
    if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_sums(double* __restrict__ block_sums, int n) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) {
            acc += block_sums[i];
            block_sums[i] = acc;
        }
    }
}

__global__ void k_scan_add(double* __restrict__ cdf, long long ncell, const double* __restrict__ block_sums) {
    const long long span = (long long)kScanBlock * kScanItems;
    const int b = blockIdx.x;
    if (b == 0) return;
    const double add = block_sums[b - 1];
    for (long long c = (long long)b * span + threadIdx.x; c < (long long)(b + 1) * span && c < ncell; c += blockDim.x)
        cdf[c] += add;
}

// ---------------------------------------------------------------------------------
// unit evaluation of device building blocks (diagnostics)
// ---------------------------------------------------------------------------------
template <typename T> __global__ void k_unit(int fn, long long n, const double* __restrict__ in, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (fn == 0) {
        const double* a = in + 6 * i;
        const U4 r = philox4x32_10((uint32_t)a[0], (uint32_t)a[1], (uint32_t)a[2], (uint32_t)a[3], (uint32_t)a[4],
                                   (uint32_t)a[5]);
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    } else if (fn == 1) {
        const double* a = in + 7 * i;
        const float4 q = quat_from_field((float)a[0], (float)a[1], (float)a[2]);
        const V3<T> v{T(a[3]), T(a[4]), T(a[5])};
        const V3<T> g = quat_to_grain(q, v);
        double* o = out + 8 * i;
        o[0] = q.x;
        o[1] = q.y;
        o[2] = q.z;
        o[3] = q.w;
        o[4] = g.x;
        o[5] = g.y;
        o[6] = g.z;
        o[7] = 0.0;
    } else if (fn == 2) {
        const double* a = in + 10 * i;
        const float4 q = quat_from_field((float)a[0], (float)a[1], (float)a[2]);
        const V3<T> n{T(a[3]), T(a[4]), T(a[5])};
        V3<T> th, ph;
        stokes_basis(n, th, ph);
        const GrainFrame<T> f = grain_frame(q, n, ph);
        T Q = T(a[7]), U = T(a[8]);
        rotate_qu(Q, U, f.c2, f.s2);
        double* o = out + 6 * i;
        o[0] = a[6];
        o[1] = Q;
        o[2] = U;
        o[3] = a[9];
        o[4] = f.cos_tp;
        o[5] = 0.0;
    } else if (fn == 3) {
        const double* a = in + 12 * i;
        T X[4] = {T(a[0]), T(a[1]), T(a[2]), T(a[3])};
        const T S[4] = {T(a[7]), T(a[8]), T(a[9]), T(a[10])};
        cell_step(X, T(a[4]), T(a[5]), T(a[6]), S, T(a[11]));
        for (int e = 0; e < 4; ++e) out[4 * i + e] = X[e];
    } else if (fn == 4) {
        const double* a = in + 8 * i;
        const T X[4] = {T(a[0]), T(a[1]), T(a[2]), T(a[3])};
        T Y[4], W[4];
        transfer(X, T(a[4]), T(a[5]), T(a[6]), T(a[7]), Y, W, true, T(a[7]));
        for (int e = 0; e < 4; ++e) out[4 * i + e] = W[e];
    } else if (fn == 5) {
        const double* a = in + 16 * i;
        const T X[4] = {T(a[0]), T(a[1]), T(a[2]), T(a[3])};
        const V3<T> n{T(a[4]), T(a[5]), T(a[6])}, n2{T(a[7]), T(a[8]), T(a[9])};
        const T P[6] = {T(a[10]), T(a[11]), T(a[12]), T(a[13]), T(a[14]), T(a[15])};
        V3<T> th, ph, th2, ph2;
        stokes_basis(n, th, ph);
        stokes_basis(n2, th2, ph2);
        const PlaneRot<T> r = plane_rotation(n, th, ph, n2, th2, ph2);
        T Y[4];
        apply_plane(r, P, X, Y);
        for (int e = 0; e < 4; ++e) out[4 * i + e] = Y[e];
    } else if (fn == 6) {
        const double* a = in + 16 * i;
        const T X[4] = {T(a[0]), T(a[1]), T(a[2]), T(a[3])};
        const V3<T> n{T(a[4]), T(a[5]), T(a[6])}, n2{T(a[7]), T(a[8]), T(a[9])}, ax{T(a[10]), T(a[11]), T(a[12])};
        V3<T> th, ph, th2, ph2;
        stokes_basis(n, th, ph);
        stokes_basis(n2, th2, ph2);
        T Y[4];
        dipole_apply(T(a[13]), T(a[14]), T(a[15]), ax, th, ph, th2, ph2, X, Y);
        for (int e = 0; e < 4; ++e) out[4 * i + e] = Y[e];
    } else if (fn == 7) {
        const double* a = in + 8 * i;
        T a1, a2, s11, s12;
        dipole_K(T(a[0]), T(a[1]), T(a[2]), T(a[3]), T(a[4]), T(a[5]), T(a[6]), a1, a2, s11, s12);
        out[4 * i] = a1;
        out[4 * i + 1] = a2;
        out[4 * i + 2] = s11;
        out[4 * i + 3] = s12;
    }
}

// Depolarization factor along the symmetry axis of a spheroid whose equatorial
// semi-axis is s times the symmetry one.  With g = s^2 - 1 the oblate and prolate
// closed forms of the ellipsoid integral are both s^2 F(g), F(g) = sum_k (-g)^k/(2k+3):
// atan form for g > 0, atanh form for g < 0, and near the sphere (|g| < 0.25) the
// series, whose terms then fall by 4x each.
__device__ double spheroid_depolarization(double s) {
    const double g = s * s - 1.0;
    double F;
    if (fabs(g) < 0.25) {
        F = 0.0;
        double t = 1.0;
        for (int k = 0; k < 40; ++k) {
            F += t / (2.0 * k + 3.0);
            t *= -g;
        }
    } else if (g > 0.0) {
        const double f = sqrt(g);
        F = (1.0 - atan(f) / f) / g;
    } else {
        const double e = sqrt(-g);
        F = (atanh(e) / e - 1.0) / (-g);
    }
    return s * s * F;
}

// Constants of aligned dipole spheroids (one thread): out[0..15] as documented for
// mcrt_dipole_constants, then out[16..19] = ca_perp, ca_par, cs_perp, cs_par (cross
// sections over their orientation averages (2 c_perp + c_par) / 3).
__global__ void k_dipole_setup(double eps_re, double eps_im, double aspect, double x, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    using cplx = cuda::std::complex<double>;
    const cplx eps(eps_re, eps_im);
    double L[2];
    L[1] = spheroid_depolarization(aspect);
    L[0] = 0.5 * (1.0 - L[1]);
    cplx al[2];
    double qe[2], qs[2], qa[2];
    const double x3 = x * x * x;
    for (int j = 0; j < 2; ++j) {
        const cplx a = (eps - 1.0) / (3.0 * (1.0 + L[j] * (eps - 1.0)));
        al[j] = a / (1.0 - cplx(0.0, 2.0 / 3.0 * x3) * a);  // radiative reaction
        qe[j] = 4.0 * x * al[j].imag();
        qs[j] = 8.0 / 3.0 * x3 * x * cuda::std::norm(al[j]);
        qa[j] = qe[j] - qs[j];
    }
    const cplx rho = al[1] / al[0];
    const double r2 = cuda::std::norm(rho);
    const double zn = 1.0 / (8.0 * 3.14159265358979323846 / 3.0 * (2.0 + r2) / 3.0);
    const double o[16] = {L[0], L[1], al[0].real(), al[0].imag(), al[1].real(), al[1].imag(), qe[0], qe[1],
                          qs[0], qs[1], qa[0], qa[1], rho.real(), rho.imag(), zn, (r2 > 1.0 ? r2 : 1.0) * zn};
    for (int k = 0; k < 16; ++k) out[k] = o[k];
    const double ma = (2.0 * qa[0] + qa[1]) / 3.0, ms = (2.0 * qs[0] + qs[1]) / 3.0;
    // a process with zero cross section has no shape (its cell opacity must be 0)
    out[16] = ma > 0.0 ? qa[0] / ma : 1.0;
    out[17] = ma > 0.0 ? qa[1] / ma : 1.0;
    out[18] = ms > 0.0 ? qs[0] / ms : 1.0;
    out[19] = ms > 0.0 ? qs[1] / ms : 1.0;
}

}  // namespace

// Root cells of a patch's box: q_B = 1, no opacity or emission, patch + 1 in the last word.
__global__ void k_mark_covered(float4* __restrict__ cells, int nx, int ny, int i0, int j0, int k0, int ni, int nj,
                               int nk, unsigned tag) {
    const long long total = (long long)ni * nj * nk;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = i0 + (int)(t % ni), j = j0 + (int)((t / ni) % nj), k = k0 + (int)(t / ((long long)ni * nj));
        const long long c = ((long long)k * ny + j) * nx + i;
        cells[2 * c] = make_float4(1.f, 0.f, 0.f, 0.f);
        cells[2 * c + 1] = make_float4(0.f, 0.f, 0.f, __uint_as_float(tag));
    }
}

cudaError_t launch_mark_covered(const GridDev& g, const PatchDev* hp, cudaStream_t s) {
    (void)cudaGetLastError();  // report these launches' errors only
    for (int q = 0; q < g.n_patches; ++q) {
        const PatchDev& P = hp[q];
        const int ni = P.box[3] - P.box[0], nj = P.box[4] - P.box[1], nk = P.box[5] - P.box[2];
        const long long total = (long long)ni * nj * nk;
        const unsigned grid = (unsigned)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
        k_mark_covered<<<grid, 256, 0, s>>>(const_cast<float4*>(g.cells), g.n[0], g.n[1], P.box[0], P.box[1],
                                            P.box[2], ni, nj, nk, (unsigned)(q + 1));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_dipole_setup(double eps_re, double eps_im, double aspect, double x, double* out, cudaStream_t s) {
    (void)cudaGetLastError();  // report this launch's error only
    k_dipole_setup<<<1, 32, 0, s>>>(eps_re, eps_im, aspect, x, out);
    return cudaGetLastError();
}

cudaError_t launch_image(const ImageParams& p, int precision, cudaStream_t s) {
    const long long npix = (long long)p.npix[0] * p.npix[1];
    const int block = 128;
    const unsigned grid = (unsigned)((npix + block - 1) / block);
    (void)cudaGetLastError();  // report this launch's error only
    if (precision == MCRT_FP64)
        k_image<double><<<grid, block, 0, s>>>(p);
    else
        k_image<float><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_setup_cells(const float* ka, const float* ks, const float* bf, const float* em, long long ncell,
                               float4* cells, unsigned* bad, cudaStream_t s) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (ncell + 255) / 256;
    const unsigned grid = (unsigned)(want < (long long)nsm * 8 ? (want > 0 ? want : 1) : (long long)nsm * 8);
    (void)cudaGetLastError();  // report this launch's error only
    k_setup_cells<<<grid, 256, 0, s>>>(ka, ks, bf, em, ncell, cells, bad);
    return cudaGetLastError();
}

cudaError_t launch_prepare_tables(int model, int n_bins, int n_theta, int n_ktheta, const float* mueller,
                                  const float* bin_weight, const float* kext, float4* mix, float4* bins,
                                  double* env_cdf, float* env, double* bin_cdf, float4* kext4, double* alpha1_mean,
                                  cudaStream_t s) {
    (void)cudaGetLastError();  // report this launch's error only
    k_prepare_tables<<<1, 256, 0, s>>>(model, n_bins, n_theta, n_ktheta, mueller, bin_weight, kext, mix, bins,
                                       env_cdf, env, bin_cdf, kext4, alpha1_mean);
    return cudaGetLastError();
}

cudaError_t launch_thermal_cdf(const GridDev& g, double alpha1_mean, double* cdf, double* block_sums, int n_blocks,
                               cudaStream_t s) {
    const double vol = g.d[0] * g.d[1] * g.d[2];
    (void)cudaGetLastError();  // report these launches' errors only
    k_scan_local<<<n_blocks, kScanBlock, 0, s>>>(g.cells, g.ncell, alpha1_mean, vol,
                                                 g.n_patches > 0 ? g.ncell_root : g.ncell, g.n_patches, g.patches,
                                                 cdf, block_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_sums<<<1, 32, 0, s>>>(block_sums, n_blocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_add<<<n_blocks, kScanBlock, 0, s>>>(cdf, g.ncell, block_sums);
    return cudaGetLastError();
}

// guide[k] = first cell whose cumulative weight exceeds k * total / n_guide, for
// k = 0..n_guide (binary search of the definition).
__global__ void k_thermal_guide(const double* __restrict__ cdf, long long ncell, long long* __restrict__ guide,
                                long long n_guide) {
    const double total = cdf[ncell - 1];
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k <= n_guide;
         k += (long long)gridDim.x * blockDim.x) {
        const double b = (double)k * total / (double)n_guide;
        long long lo = 0, hi = ncell - 1;
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (cdf[mid] > b)
                hi = mid;
            else
                lo = mid + 1;
        }
        guide[k] = lo;
    }
}

cudaError_t launch_thermal_guide(const double* cdf, long long ncell, long long* guide, long long n_guide,
                                 cudaStream_t s) {
    const long long n = n_guide + 1;
    const unsigned grid = (unsigned)((n + 255) / 256 < 65535 ? (n + 255) / 256 : 65535);
    (void)cudaGetLastError();  // report this launch's error only
    k_thermal_guide<<<grid, 256, 0, s>>>(cdf, ncell, guide, n_guide);
    return cudaGetLastError();
}

int thermal_cdf_blocks(long long ncell) { return (int)((ncell + (long long)kScanBlock * kScanItems - 1) / ((long long)kScanBlock * kScanItems)); }

cudaError_t launch_unit_eval(int fn, int precision, long long n, const double* in, double* out, cudaStream_t s) {
    const int block = 128;
    const unsigned grid = (unsigned)((n + block - 1) / block);
    (void)cudaGetLastError();  // report this launch's error only
    if (precision == MCRT_FP64)
        k_unit<double><<<grid, block, 0, s>>>(fn, n, in, out);
    else
        k_unit<float><<<grid, block, 0, s>>>(fn, n, in, out);
    return cudaGetLastError();
}

}  // namespace mcrt
