"""Seeded synthetic inputs for the transport: grids, field directions, grain optics
tables, sources and cameras.

This module only builds input arrays (numpy, FP32 fields, FP64 geometry).  It holds
none of the transport or imaging arithmetic, and is the one module that both the CPU
oracle's tests and the CUDA path draw their inputs from.

Workloads (sizes as stated):
  rayleigh_sphere   uniform sphere of radius 1 on a 32^3 grid over [-1,1]^3, radial
                    optical depth 1, albedo 1, dipole (Rayleigh) grains, central
                    isotropic unpolarized point source, 1e5 packets, one 64^2 camera.
  dichroic_slab     aligned-grain slab on a 64^3 grid over [0,1]^3, uniform field at
                    45 deg to the line of sight, alpha2/alpha1 = -0.05, alpha3 = 0,
                    no scattering, plane beam along +z, 1e6 packets.
  disk              flared disk on a 192^3 grid over [-1,1]^3: rho ~ (R/R0)^-1
                    exp(-z^2/2H^2), H/R = 0.1 (R/R0)^0.25, inner radius 0.1, outer 1,
                    midplane radial optical depth 1e3; toroidal+poloidal field with a
                    30 deg pitch; 8 grain-size bins of tabulated scattering matrices
                    (181 angles); star plus thermal emission; 8 cameras at 256^2.
  twisted_slab      slab with a field rotating by 2 pi per unit optical depth (the
                    twisted-field test of Sec. 3.2).
  spheroid_sphere   uniform sphere of aligned oblate dipole spheroids (aspect 2:1,
                    m = 2.30 + 0.0228 i, as in the circumstellar test of Sec. 3.5) on a
                    32^3 grid over [-1,1]^3, field along z, radial optical depth 0.01, 1
                    or 10, central star, camera along x.
  spheroid_atmosphere  plane-parallel slab of aligned spheroids with aspect 1.03 (the
                    atmosphere test of Sec. 3.4), periodic in x and y, field along x,
                    thermal emission, cameras at 45 deg inclination and a range of
                    azimuths.
  disk_refined      the flared disk on a 128^3 root grid with one statically refined patch
                    (4x) over the inner quarter in x, y and the middle eighth in z, the
                    fields evaluated at the patch's own cell centres.
  inclined_thin_disk  the inclined-disk scene of Sec. 3.1: a geometrically and optically
                    thin annulus of Rayleigh grains (one cell layer |z| <= h, inner radius
                    0.3, outer 1, radial optical depth 1e-3) around a central isotropic
                    star, so that the light reaching the grains travels in the disk
                    plane; field along x; cameras at inclinations 0..90 deg, 256^2.
  sweep             batched sweep: 32 models with edges drawn uniformly in 32..192, clumpy
                    log-normal density (sigma_ln = 1), mean optical depth log-uniform in
                    [1, 100], times 8 wavelengths 0.5-3 um (kappa ~ lambda^-1.5); central
                    star; one camera at 45 deg, 128^2.

The grain tables are synthetic (no measured optical constants are available): per bin
a Henyey-Greenstein P11, P12/P11 = -p (1-c^2)/(1+c^2), P22 = P11,
P33/P11 = P44/P11 = 2c/(1+c^2), P34 = 0, which is a realizable scattering matrix for
0 <= p <= 1.  Their extinction has the dipole form alpha1 = 1, alpha2 = -p_max sin^2
theta' with p_max from 0.1 (smallest bin) to 0.02 (largest); the mixture's table holds
the extinction-weighted mean of the bins' p_max.
"""
from __future__ import annotations

import math

import numpy as np

N_THETA = 181


def _centres(n, lo, hi):
    d = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * d


def cell_centres(shape_zyx, lo, hi):
    nz, ny, nx = shape_zyx
    z = _centres(nz, lo[2], hi[2])[:, None, None]
    y = _centres(ny, lo[1], hi[1])[None, :, None]
    x = _centres(nx, lo[0], hi[0])[None, None, :]
    return x, y, z


# ----------------------------------------------------------------------------------
# grain optics inputs
# ----------------------------------------------------------------------------------
def kext_isotropic():
    """alpha1 = 1, alpha2 = alpha3 = 0 on theta' in [0, pi] (spherical grains)."""
    return np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0]], dtype=np.float32)


def kext_constant(alpha2, alpha3=0.0):
    return np.array([[1.0, alpha2, alpha3], [1.0, alpha2, alpha3]], dtype=np.float32)


def kext_dipole(p_max, alpha3_over_alpha2=0.0, n=N_THETA):
    """alpha1 = 1, alpha2 = -p_max sin^2 theta', alpha3 = ratio * alpha2."""
    t = np.linspace(0.0, math.pi, n)
    a2 = -p_max * np.sin(t) ** 2
    return np.stack([np.ones(n), a2, alpha3_over_alpha2 * a2], axis=1).astype(np.float32)


def _interp_norm(p11, n_theta):
    """2 pi int P11(theta) sin(theta) dtheta of the interpolant linear in theta."""
    h = math.pi / (n_theta - 1)
    ta = np.arange(n_theta - 1) * h
    tb = ta + h
    A = p11[:-1]
    B = (p11[1:] - p11[:-1]) / h
    return 2 * math.pi * np.sum(A * (np.cos(ta) - np.cos(tb)) + B * (-(tb - ta) * np.cos(tb) + np.sin(tb) - np.sin(ta)))


def synthetic_bins(n_bins=8, n_theta=N_THETA):
    """Per-bin scattering tables [n_bins][n_theta][6] (P11,P12,P22,P33,P34,P44),
    normalised so that the theta-linear interpolant of P11 integrates to 1 over the
    sphere, and the bin weights (fractions of the scattering cross section)."""
    x = np.logspace(-1, 1, n_bins)
    g = np.linspace(0.0, 0.8, n_bins)
    p = np.linspace(1.0, 0.3, n_bins)
    th = np.linspace(0.0, math.pi, n_theta)
    c = np.cos(th)
    tabs = np.zeros((n_bins, n_theta, 6))
    for k in range(n_bins):
        p11 = (1 - g[k] ** 2) / (4 * math.pi * (1 + g[k] ** 2 - 2 * g[k] * c) ** 1.5)
        p11 = p11 / _interp_norm(p11, n_theta)
        tabs[k, :, 0] = p11
        tabs[k, :, 1] = -p[k] * (1 - c * c) / (1 + c * c) * p11
        tabs[k, :, 2] = p11
        tabs[k, :, 3] = 2 * c / (1 + c * c) * p11
        tabs[k, :, 4] = 0.0
        tabs[k, :, 5] = 2 * c / (1 + c * c) * p11
    w = np.sqrt(x)
    w = w / w.sum()
    return tabs.astype(np.float32), w.astype(np.float32), x


def dipole_optics(eps=complex(2.30, 0.0228) ** 2, aspect=2.0, x=0.3):
    """Aligned spheroids in the dipole approximation: complex dielectric function
    `eps`, equatorial over symmetry semi-axis `aspect` (> 1 oblate, < 1 prolate; the
    symmetry axis lies along the field), size parameter x = 2 pi a_eff / lambda.  The
    cells' kappa_abs and kappa_sca are the orientation-averaged opacities."""
    return {"model": "dipole", "eps": complex(eps), "aspect": float(aspect), "x": float(x)}


def rayleigh_optics():
    return {"model": "rayleigh", "kext": kext_isotropic()}


def rayleigh_table(n_theta=N_THETA):
    """The dipole-sphere (Rayleigh) scattering matrix as a one-bin table [1][n_theta][6]:
    P11 = P22 = 1 + c^2, P12 = c^2 - 1, P33 = P44 = 2c, P34 = 0, normalised like
    ``synthetic_bins`` (theta-linear interpolant of P11 integrating to 1)."""
    c = np.cos(np.linspace(0.0, math.pi, n_theta))
    tab = np.zeros((1, n_theta, 6))
    tab[0, :, 0] = tab[0, :, 2] = 1 + c * c
    tab[0, :, 1] = c * c - 1
    tab[0, :, 3] = tab[0, :, 5] = 2 * c
    tab /= _interp_norm(tab[0, :, 0], n_theta)
    return tab.astype(np.float32)


def bin_p_max(n_bins=8):
    """Dichroism of the synthetic size bins: p_max from 0.1 (smallest grains) to 0.02."""
    return np.linspace(0.1, 0.02, n_bins)


def table_optics(n_bins=8, p_max=None):
    """Synthetic bin tables with the dipole extinction form.  ``p_max`` None: each bin
    k has its own alpha2 = -p_max,k sin^2 theta' (``bin_p_max``); the table given is
    that of the mixture, the bins weighted by their share of the extinction (all bins
    share the cell's albedo, so that share is ``bin_weight``).  A number: one p_max."""
    tabs, w, _ = synthetic_bins(n_bins)
    p = float(np.dot(w.astype(np.float64), bin_p_max(n_bins))) if p_max is None else float(p_max)
    return {"model": "table", "mueller": tabs, "bin_weight": w, "kext": kext_dipole(p)}


# ----------------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------------
def camera(direction, npix, fov, center=None):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    cam = {"dir": tuple(float(v) for v in d), "npix": (int(npix[0]), int(npix[1])),
           "fov": (float(fov[0]), float(fov[1]))}
    if center is not None:
        cam["center"] = tuple(float(v) for v in center)
    return cam


def inclination_cameras(n_cam=8, npix=256, fov=2.0):
    """Cameras at inclinations linspace(0, 90 deg, n_cam), azimuth 0."""
    cams = []
    for i in np.linspace(0.0, math.pi / 2, n_cam):
        cams.append(camera((math.sin(i), 0.0, math.cos(i)), (npix, npix), (fov, fov)))
    return cams


# ----------------------------------------------------------------------------------
# models
# ----------------------------------------------------------------------------------
def rayleigh_sphere(n=32, tau=1.0, radius=1.0, bfield=None):
    """Uniform Rayleigh sphere: kappa_ext = tau/radius where the cell centre lies
    within ``radius`` of the origin, albedo 1."""
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    x, y, z = cell_centres((n, n, n), lo, hi)
    r = np.sqrt(x * x + y * y + z * z)
    ks = np.where(r <= radius, tau / radius, 0.0).astype(np.float32)
    model = {"lo": lo, "hi": hi, "kappa_abs": np.zeros_like(ks), "kappa_sca": ks,
             "bfield": bfield, "emissivity": None, "optics": rayleigh_optics()}
    return model


def rayleigh_sphere_run(n_packets=100000, seed=0, npix=64):
    return {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": n_packets}],
            "cameras": [camera((1.0, 0.0, 0.0), (npix, npix), (2.0, 2.0))],
            "seed": seed, "roulette_threshold": 1e-4, "roulette_survival": 0.1}


def dichroic_slab(n=64, tau=1.0, p=0.05, b_angle_deg=45.0, albedo=0.0, emissivity=None):
    """Aligned-grain slab over [0,1]^3 with uniform kappa_ext = tau and a uniform
    field in the x-z plane at ``b_angle_deg`` from +z."""
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    kext = np.full((n, n, n), tau, dtype=np.float32)
    a = math.radians(b_angle_deg)
    bf = np.zeros((n, n, n, 3), dtype=np.float32)
    bf[..., 0] = math.sin(a)
    bf[..., 2] = math.cos(a)
    em = None if emissivity is None else np.full((n, n, n), emissivity, dtype=np.float32)
    return {"lo": lo, "hi": hi, "kappa_abs": (kext * (1 - albedo)).astype(np.float32),
            "kappa_sca": (kext * albedo).astype(np.float32), "bfield": bf, "emissivity": em,
            "optics": {"model": "rayleigh", "kext": kext_constant(-p, 0.0)}}


def plane_parallel_slab(nxy=4, nz=16, tau=1.0, albedo=0.9, periodic=3, b_angle_deg=None, p=0.0):
    """Plane-parallel slab: z in [0, 1] with uniform kappa_ext = tau (vertical optical
    depth tau), x, y in [0, 1] periodic (bit a of ``periodic``: axis a), dipole grains;
    optionally a uniform field in the x-z plane at ``b_angle_deg`` from +z with
    dichroism alpha2 = -p."""
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    shape = (nz, nxy, nxy)
    kext = np.full(shape, tau, dtype=np.float32)
    bf = None
    if b_angle_deg is not None:
        a = math.radians(b_angle_deg)
        bf = np.zeros(shape + (3,), dtype=np.float32)
        bf[..., 0] = math.sin(a)
        bf[..., 2] = math.cos(a)
    return {"lo": lo, "hi": hi, "kappa_abs": (kext * (1 - albedo)).astype(np.float32),
            "kappa_sca": (kext * albedo).astype(np.float32), "bfield": bf, "emissivity": None,
            "periodic": int(periodic),
            "optics": {"model": "rayleigh", "kext": kext_constant(-p, 0.0) if p else kext_isotropic()}}


def spheroid_sphere(n=32, tau=1.0, albedo=0.5, radius=1.0, optics=None, b=(0.0, 0.0, 1.0)):
    """Uniform sphere of aligned dipole spheroids (radial extinction optical depth tau,
    given albedo) with a uniform field `b`."""
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    x, y, z = cell_centres((n, n, n), lo, hi)
    r = np.sqrt(x * x + y * y + z * z)
    kext = np.where(r <= radius, tau / radius, 0.0)
    bf = np.zeros((n, n, n, 3), dtype=np.float32)
    bf[...] = np.asarray(b, dtype=np.float32)
    return {"lo": lo, "hi": hi, "kappa_abs": (kext * (1 - albedo)).astype(np.float32),
            "kappa_sca": (kext * albedo).astype(np.float32), "bfield": bf, "emissivity": None,
            "optics": optics or dipole_optics()}


def spheroid_atmosphere(nxy=4, nz=32, tau=1.0, albedo=0.5, optics=None, emissivity=1.0):
    """Plane-parallel slab (z in [0, 1], vertical extinction optical depth tau),
    periodic in x and y, aligned spheroids with the field along x, uniform thermal
    emission."""
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    shape = (nz, nxy, nxy)
    kext = np.full(shape, tau, dtype=np.float64)
    bf = np.zeros(shape + (3,), dtype=np.float32)
    bf[..., 0] = 1.0
    return {"lo": lo, "hi": hi, "kappa_abs": (kext * (1 - albedo)).astype(np.float32),
            "kappa_sca": (kext * albedo).astype(np.float32), "bfield": bf,
            "emissivity": np.full(shape, emissivity, dtype=np.float32), "periodic": 3,
            "optics": optics or dipole_optics(aspect=1.03)}


def atmosphere_cameras(n_az=8, incl_deg=45.0, npix=8):
    """Cameras at inclination `incl_deg` from +z and azimuths 0..180 deg."""
    i = math.radians(incl_deg)
    return [camera((math.sin(i) * math.cos(a), math.sin(i) * math.sin(a), math.cos(i)), (npix, npix), (1.0, 1.0),
                   center=(0.5, 0.5, 0.5))
            for a in np.linspace(0.0, math.pi, n_az)]


def center_source_run(n_packets, seed=5, cameras=None, pos=(0.5, 0.5, 0.5)):
    """Isotropic unpolarized point source (luminosity 1) at ``pos``."""
    return {"sources": [{"type": "point", "pos": tuple(pos), "luminosity": 1.0, "n_packets": int(n_packets)}],
            "cameras": cameras or [], "seed": seed}


def beam_run(n_packets, seed=1, direction=+1, cameras=None, roulette_threshold=0.0):
    return {"sources": [{"type": "beam", "beam_dir": direction, "luminosity": 1.0, "n_packets": n_packets}],
            "cameras": cameras or [], "seed": seed, "roulette_threshold": roulette_threshold,
            "roulette_survival": 0.1}


def twisted_slab(tau, p0=0.01, nz_per_tau=200, nxy=2, coupling=True):
    """Slab of optical depth ``tau`` (kappa = 1) over z in [0, tau]; the field lies
    in the x-y plane at angle 2 pi z from +x, i.e. 2 pi tau' with tau' the optical
    depth above the z = 0 face.  alpha2 = -p0 (field perpendicular to the beam);
    alpha3 = -alpha2 when ``coupling`` (the artificial U-V term of Sec. 3.2)."""
    nz = max(1, int(round(nz_per_tau * tau)))
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, float(tau))
    z = _centres(nz, 0.0, tau)
    bf = np.zeros((nz, nxy, nxy, 3), dtype=np.float32)
    bf[..., 0] = np.cos(2 * math.pi * z)[:, None, None]
    bf[..., 1] = np.sin(2 * math.pi * z)[:, None, None]
    ka = np.ones((nz, nxy, nxy), dtype=np.float32)
    a3 = p0 if coupling else 0.0
    return {"lo": lo, "hi": hi, "kappa_abs": ka, "kappa_sca": np.zeros_like(ka), "bfield": bf,
            "emissivity": None, "optics": {"model": "rayleigh", "kext": kext_constant(-p0, a3)}}


def _disk_fields(x, y, z, tau_mid, r_in, r_out, albedo, pitch_deg, T0, lam_um):
    """Cell arrays of the flared disk at cell centres (x, y, z): kappa_abs, kappa_sca,
    field, unnormalised emissivity."""
    R = np.sqrt(x * x + y * y) + 0.0 * z
    H = 0.1 * np.maximum(R, 1e-30) ** 1.25
    rho = np.where((R >= r_in) & (R <= r_out), np.maximum(R, 1e-30) ** -1.0 * np.exp(-z * z / (2 * H * H)), 0.0)
    k0 = tau_mid / math.log(r_out / r_in)
    kext = (k0 * rho).astype(np.float32)
    ks = (albedo * kext).astype(np.float32)
    ka = (kext - ks).astype(np.float32)
    pitch = math.radians(pitch_deg)
    Rs = np.maximum(R, 1e-30)
    bf = np.zeros(np.broadcast(x, y, z).shape + (3,), dtype=np.float32)
    bf[..., 0] = (math.cos(pitch) * (-y / Rs)) * (R > 0)
    bf[..., 1] = (math.cos(pitch) * (x / Rs)) * (R > 0)
    bf[..., 2] = math.sin(pitch)
    T = T0 * Rs ** -0.5
    hc_k = 14387.77 / lam_um
    em = np.where(rho > 0, 1.0 / np.expm1(np.minimum(hc_k / T, 700.0)), 0.0)
    return ka, ks, bf, em


def disk(n=192, tau_mid=1e3, r_in=0.1, r_out=1.0, albedo=0.6, pitch_deg=30.0, T0=1000.0,
         lam_um=1.0, n_bins=8, p_max=None):
    """Flared disk; see the module docstring."""
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    x, y, z = cell_centres((n, n, n), lo, hi)
    ka, ks, bf, em = _disk_fields(x, y, z, tau_mid, r_in, r_out, albedo, pitch_deg, T0, lam_um)
    em = (em / max(em.max(), 1e-300)).astype(np.float32)
    return {"lo": lo, "hi": hi, "kappa_abs": ka, "kappa_sca": ks, "bfield": bf, "emissivity": em,
            "optics": table_optics(n_bins, p_max)}


def disk_refined(n=128, box=None, factor=4, tau_mid=1e3, r_in=0.1, r_out=1.0, albedo=0.6, pitch_deg=30.0,
                 T0=1000.0, lam_um=1.0, n_bins=8, p_max=None):
    """Flared disk on a composite grid: an n^3 root grid plus one statically refined
    patch over root-cell box `box` (default: the inner quarter of x and y, the middle
    eighth of z) with `factor` cells per root cell, the disk's fields evaluated at the
    patch's own cell centres (emissivity normalised like the root's)."""
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    if box is None:
        q, e = n // 2 - n // 8, n // 2 - n // 16
        box = (q, q, e, n - q, n - q, n - e)
    x, y, z = cell_centres((n, n, n), lo, hi)
    ka, ks, bf, em = _disk_fields(x, y, z, tau_mid, r_in, r_out, albedo, pitch_deg, T0, lam_um)
    norm = max(em.max(), 1e-300)
    d = [(h - l) / n for l, h in zip(lo, hi)]
    plo = [l + b * dd for l, b, dd in zip(lo, box[:3], d)]
    phi = [l + b * dd for l, b, dd in zip(lo, box[3:], d)]
    shape = tuple((box[3 + a] - box[a]) * factor for a in (2, 1, 0))
    px, py, pz = cell_centres(shape, plo, phi)
    pka, pks, pbf, pem = _disk_fields(px, py, pz, tau_mid, r_in, r_out, albedo, pitch_deg, T0, lam_um)
    patch = {"box": tuple(int(b) for b in box), "factor": int(factor), "kappa_abs": pka, "kappa_sca": pks,
             "bfield": pbf, "emissivity": (pem / norm).astype(np.float32)}
    return {"lo": lo, "hi": hi, "kappa_abs": ka, "kappa_sca": ks, "bfield": bf,
            "emissivity": (em / norm).astype(np.float32), "optics": table_optics(n_bins, p_max), "refine": [patch]}


def refine_uniform(model, patches):
    """The same model on a composite grid: each (box, factor) of `patches` becomes a
    refined patch whose cells copy their parent root cell's values (a finer grid of the
    same medium)."""
    out = dict(model)
    out["refine"] = []
    for box, f in patches:
        i0, j0, k0, i1, j1, k1 = box
        rep = {}
        for key in ("kappa_abs", "kappa_sca", "bfield", "emissivity"):
            a = model.get(key)
            if a is None:
                rep[key] = None
                continue
            sub = np.asarray(a)[k0:k1, j0:j1, i0:i1]
            sub = np.repeat(np.repeat(np.repeat(sub, f, axis=0), f, axis=1), f, axis=2)
            rep[key] = np.ascontiguousarray(sub, dtype=np.float32)
        out["refine"].append(dict(rep, box=tuple(box), factor=int(f)))
    return out


def disk_run(n_packets=100_000_000, seed=2, n_cam=8, npix=256, star_luminosity=1.0):
    """Half of the packets from the star at the origin, half from thermal emission."""
    n_star = n_packets // 2
    return {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": star_luminosity,
                         "n_packets": n_star},
                        {"type": "thermal", "luminosity": 0.0, "n_packets": n_packets - n_star}],
            "cameras": inclination_cameras(n_cam, npix, 2.0), "seed": seed,
            "roulette_threshold": 1e-4, "roulette_survival": 0.1}


def inclined_thin_disk(n=64, h=0.01, r_in=0.3, r_out=1.0, tau=1e-3, table=False):
    """Thin annulus of Rayleigh grains (Sec. 3.1, inclined-disk test): grid
    [-1,1]^2 x [-h,h] with one cell layer of n x n cells; kappa_sca = tau / (r_out - r_in)
    where the cell centre's cylindrical radius lies in [r_in, r_out] (radial scattering
    optical depth tau), albedo 1; field along +x (the paper puts the grain frame's axis
    along x in this test).  ``table``: the Rayleigh matrix as a 181-angle table
    (MCRT_SCAT_TABLE) instead of the closed form."""
    lo, hi = (-1.0, -1.0, -float(h)), (1.0, 1.0, float(h))
    x, y, z = cell_centres((1, n, n), lo, hi)
    R = np.sqrt(x * x + y * y) + 0.0 * z
    ks = np.where((R >= r_in) & (R <= r_out), tau / (r_out - r_in), 0.0).astype(np.float32)
    bf = np.zeros(ks.shape + (3,), dtype=np.float32)
    bf[..., 0] = 1.0
    optics = rayleigh_optics()
    if table:
        optics = {"model": "table", "mueller": rayleigh_table(), "bin_weight": np.ones(1, np.float32),
                  "kext": kext_isotropic()}
    return {"lo": lo, "hi": hi, "kappa_abs": np.zeros_like(ks), "kappa_sca": ks, "bfield": bf, "emissivity": None,
            "optics": optics, "geometry": {"h": float(h), "r_in": float(r_in), "r_out": float(r_out)}}


def thin_disk_run(n_packets, seed=6, npix=256, incl_deg=(0, 15, 30, 45, 60, 75, 90)):
    """Central isotropic star (luminosity 1) and cameras at inclinations ``incl_deg``
    from the disk axis toward +x, FOV 2 x 2; no roulette (albedo 1)."""
    cams = [camera((math.sin(math.radians(a)), 0.0, math.cos(math.radians(a))), (npix, npix), (2.0, 2.0))
            for a in incl_deg]
    return {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": int(n_packets)}],
            "cameras": cams, "seed": seed, "roulette_threshold": 0.0, "roulette_survival": 0.1}


def clumpy_density(n, seed, smooth_cells=2.0):
    """rho = exp(g - 1/2), g a unit-variance Gaussian random field: white noise
    smoothed with a Gaussian of ``smooth_cells`` cells, rescaled to unit variance
    (so that <rho> = 1 for a log-normal field with sigma_ln = 1)."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    g = gaussian_filter(rng.standard_normal((n, n, n)), smooth_cells, mode="wrap")
    g = (g - g.mean()) / g.std()
    return np.exp(g - 0.5)


def sweep_models(n_models=32, n_lambda=8, n_min=32, n_max=192, albedo=0.6, seed0=1000, edges=None):
    """Model dicts of the batched sweep, ordered model-major: [m][lambda].  Grid
    [-1,1]^3; the mean extinction optical depth across the box (length 2) is
    tau_m at 1 um, log-uniform in [1, 100]; kappa scales as (lambda / 1 um)^-1.5."""
    lams = np.logspace(np.log10(0.5), np.log10(3.0), n_lambda)
    optics = table_optics()
    out = []
    for m in range(n_models):
        rng = np.random.default_rng(seed0 + m)
        n = int(rng.integers(n_min, n_max + 1)) if edges is None else int(edges[m])
        tau = 10 ** rng.uniform(0.0, 2.0)
        rho = clumpy_density(n, seed0 + m)
        for lam in lams:
            kext = (tau / 2.0 * lam ** -1.5 * rho).astype(np.float32)
            ks = (albedo * kext).astype(np.float32)
            out.append({"lo": (-1.0, -1.0, -1.0), "hi": (1.0, 1.0, 1.0), "kappa_abs": (kext - ks).astype(np.float32),
                        "kappa_sca": ks, "bfield": None, "emissivity": None, "optics": optics,
                        "edge": n, "tau": tau, "lambda_um": float(lam)})
    return out


def sweep_run(n_packets=10_000_000, seed=4, npix=128):
    return {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": n_packets}],
            "cameras": [camera((math.sin(math.pi / 4), 0.0, math.cos(math.pi / 4)), (npix, npix), (2.0, 2.0))],
            "seed": seed, "roulette_threshold": 1e-4, "roulette_survival": 0.1}
