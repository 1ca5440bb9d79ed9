"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a published
test vector, a closed form printed in the paper, an independent construction
(rotation matrices, scipy's matrix exponential, quadrature, brute-force geometry)
or an invariant.  CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.linalg import expm

from oracle import oracle as O
from paper_2512_01283_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def rand_dirs(k, rng=RNG):
    v = rng.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def f32(x):
    return float(np.float32(x))


# ---------------------------------------------------------------------------------
# random numbers
# ---------------------------------------------------------------------------------
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al. 2011)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_open_interval_and_float32_exact():
    for x in [0, 1, 255, 256, 0x7fffffff, 0xffffff00, 0xffffffff]:
        u = O.uniform(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
        assert u == (((x >> 8) | 1) / 2.0 ** 24)


# ---------------------------------------------------------------------------------
# Sec. 2.1: quaternions, Stokes bases, basis rotation
# ---------------------------------------------------------------------------------
def rot_z(a):
    return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])


def rot_y(a):
    return np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])


def test_grain_quaternion_is_rz_ry_rotation():
    """eq. (grain-quaternion): q_B rotates z-hat to B-hat; the lab->grain map of
    eq. (vector-transform) equals (R_z(phi_B) R_y(theta_B))^T built from plain
    rotation matrices."""
    for b in rand_dirs(50):
        th, ph = math.acos(b[2]), math.atan2(b[1], b[0])
        R = rot_z(ph) @ rot_y(th)
        q = O.grain_quaternion(b * 3.7)
        assert abs(np.dot(q, q) - 1.0) < 1e-14
        assert np.allclose(O.to_lab(q, [0, 0, 1]), b, atol=1e-14)
        assert np.allclose(O.to_grain(q, b), [0, 0, 1], atol=1e-14)
        v = rand_dirs(1)[0]
        assert np.allclose(O.to_grain(q, v), R.T @ v, atol=1e-14)
        assert np.allclose(O.to_lab(q, O.to_grain(q, v)), v, atol=1e-14)


def test_grain_quaternion_special_cases():
    assert np.allclose(O.grain_quaternion([0, 0, 0]), [1, 0, 0, 0])
    assert np.allclose(O.grain_quaternion([0, 0, 2]), [1, 0, 0, 0])
    # field along -z: theta_B = pi, phi_B = 0 -> rotation by pi about y
    q = O.grain_quaternion([0, 0, -1])
    assert np.allclose(O.to_lab(q, [0, 0, 1]), [0, 0, -1], atol=1e-15)
    assert np.allclose(O.to_lab(q, [1, 0, 0]), [-1, 0, 0], atol=1e-15)


def test_stokes_basis_right_handed_and_poles():
    for n in rand_dirs(50):
        th, ph = O.stokes_basis(n)
        assert np.allclose(np.cross(th, ph), n, atol=1e-14)
        assert abs(np.dot(th, n)) < 1e-14 and abs(np.dot(ph, n)) < 1e-14
        assert ph[2] == 0.0
    th, ph = O.stokes_basis([0, 0, 1])
    assert np.allclose(th, [1, 0, 0]) and np.allclose(ph, [0, 1, 0])
    th, ph = O.stokes_basis([0, 0, -1])
    assert np.allclose(th, [-1, 0, 0]) and np.allclose(ph, [0, 1, 0])


def test_change_basis_matches_eta_rotation():
    """eq. (rotation-angle) + eq. (stokes-rotation), with the signed reading
    sin(eta) = (phi_GF x phi') . n: projecting onto the rotated basis equals the
    printed (Q,U) rotation; I and V are unchanged."""
    for n in rand_dirs(40):
        th, ph = O.stokes_basis(n)
        psi = RNG.uniform(-math.pi, math.pi)
        th2 = math.cos(psi) * th + math.sin(psi) * ph
        ph2 = np.cross(n, th2)
        cos_eta = np.dot(ph, ph2)
        sin_eta = np.dot(np.cross(ph, ph2), n)
        eta = math.atan2(sin_eta, cos_eta)
        X = np.array([1.0, *(RNG.uniform(-0.5, 0.5, 3))])
        Q = math.cos(2 * eta) * X[1] + math.sin(2 * eta) * X[2]
        U = -math.sin(2 * eta) * X[1] + math.cos(2 * eta) * X[2]
        Y = O.change_basis(X, th, ph, th2, ph2)
        assert np.allclose(Y, [X[0], Q, U, X[3]], atol=1e-14)


def test_change_basis_handedness_flip_and_field_picture():
    # linear polarization along theta-hat: Q = I
    n = unit([0.3, -0.2, 0.9])
    th, ph = O.stokes_basis(n)
    # field at angle chi from theta-hat: Q = cos 2chi, U = sin 2chi
    chi = 0.4
    e = math.cos(chi) * th + math.sin(chi) * ph
    Y = O.change_basis([1, math.cos(2 * chi), math.sin(2 * chi), 0], th, ph, e, np.cross(n, e))
    assert np.allclose(Y, [1, 1, 0, 0], atol=1e-14)
    # swapping to a left-handed basis flips V
    Y = O.change_basis([1, 0.1, 0.2, 0.3], th, ph, th, -ph)
    assert np.allclose(Y, [1, 0.1, -0.2, -0.3], atol=1e-14)


def test_grain_meridian_basis():
    """theta-hat' of the grain-frame direction lies along minus the projection of
    B-hat on the plane normal to n; theta' is the angle between n and B-hat."""
    for _ in range(30):
        b, n = rand_dirs(2)
        q = O.grain_quaternion(b)
        gth, gph, tp = O.grain_meridian(q, n)
        assert abs(tp - math.acos(np.clip(np.dot(n, b), -1, 1))) < 1e-12
        bperp = b - np.dot(b, n) * n
        assert np.allclose(gth, -unit(bperp), atol=1e-12)
        assert np.allclose(np.cross(gth, gph), n, atol=1e-12)


# ---------------------------------------------------------------------------------
# App. A: in-cell analytic solution
# ---------------------------------------------------------------------------------
def kmat(a1, a2, a3):
    return np.array([[a1, a2, 0, 0], [a2, a1, 0, 0], [0, 0, a1, a3], [0, 0, -a3, a1]], dtype=np.float64)


def test_cell_solution_against_matrix_exponential():
    """App. A printed solution = e^{-K dtau} X0 + K^{-1}(1 - e^{-K dtau}) S (scipy expm)."""
    for _ in range(200):
        a1 = RNG.uniform(0.2, 3.0)
        a2 = RNG.uniform(-0.9, 0.9) * a1
        a3 = RNG.uniform(-2, 2)
        X0 = np.array([1.0, *RNG.uniform(-0.5, 0.5, 3)])
        S = RNG.uniform(-1, 1, 4)
        dt = 10 ** RNG.uniform(-3, 1.3)
        K = kmat(a1, a2, a3)
        E = expm(-K * dt)
        ref = E @ X0 + np.linalg.solve(K, (np.eye(4) - E) @ S)
        got = O.cell_solution(X0, (a1, a2, a3), S, dt)
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-12 * (1 + np.abs(ref).max()))


def test_cell_solution_solves_the_ode_not_the_printed_matrix():
    """The printed solution solves dX/dtau = -K X + S for the symmetric I-Q block
    and antisymmetric U-V block (reading of App. A); finite difference check."""
    a1, a2, a3 = 1.3, -0.4, 0.7
    X0 = np.array([1.0, 0.2, -0.1, 0.05])
    S = np.array([0.3, -0.1, 0.2, 0.05])
    t, h = 0.8, 1e-5
    Xp = O.cell_solution(X0, (a1, a2, a3), S, t + h)
    Xm = O.cell_solution(X0, (a1, a2, a3), S, t - h)
    X = O.cell_solution(X0, (a1, a2, a3), S, t)
    d = (Xp - Xm) / (2 * h)
    assert np.allclose(d, -kmat(a1, a2, a3) @ X + S, atol=1e-8)
    printed = np.array([[a1, a2, 0, 0], [-a2, a1, 0, 0], [0, 0, a1, a3], [0, 0, a3, a1]])
    assert not np.allclose(d, -printed @ X + S, atol=1e-3)


def test_attenuate_is_cell_solution_without_source():
    for _ in range(50):
        a = RNG.uniform(0.0, 2.0)
        a2 = RNG.uniform(-0.5, 0.5) * max(a, 0.1)
        a3 = RNG.uniform(-1, 1)
        X0 = np.array([1.0, *RNG.uniform(-0.5, 0.5, 3)])
        dt = RNG.uniform(0, 5)
        ref = expm(-kmat(a, a2, a3) * dt) @ X0
        assert np.allclose(O.attenuate(X0, a, a2, a3, dt), ref, rtol=1e-12, atol=1e-14)


def test_segment_integral_against_quadrature():
    """Path integral of the attenuated Stokes vector: int_0^dtau e^{-M t} dt X0,
    against adaptive quadrature of scipy's expm."""
    cases = [(0.0, 0.0, 0.0, 2.0), (0.4, -0.05, 0.0, 3.0), (1.0, 0.3, 0.6, 0.7), (0.2, 0.2, -0.3, 12.0),
             (1e-9, 0.0, 1e-9, 0.5)]
    for a, a2, a3, dt in cases:
        X0 = np.array([1.0, 0.3, -0.2, 0.1])
        M = kmat(a, a2, a3)
        ref = np.array([quad(lambda t, i=i: (expm(-M * t) @ X0)[i], 0, dt, epsabs=1e-13, epsrel=1e-12)[0]
                        for i in range(4)])
        assert np.allclose(O.segment_integral(X0, a, a2, a3, dt), ref, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------------
# Grain optics: dipole scattering, Sec. 3.1 inclined disk
# ---------------------------------------------------------------------------------
def test_rayleigh_normalisation_and_polarization():
    """Dipole scattering: int P11 dOmega = 1; unpolarized light scattered by Theta
    has p = (1 - cos^2)/(1 + cos^2) perpendicular to the scattering plane."""
    norm = quad(lambda mu: 2 * math.pi * O.rayleigh(mu)[0], -1, 1)[0]
    assert abs(norm - 1.0) < 1e-12
    for n, n2 in zip(rand_dirs(40), rand_dirs(40)):
        mu = float(np.dot(n, n2))
        Y = O.mueller_apply([1, 0, 0, 0], n, n2, O.rayleigh(mu))
        assert abs(Y[0] - 3 / (16 * math.pi) * (1 + mu * mu)) < 1e-14
        p = math.hypot(Y[1], Y[2]) / Y[0]
        assert abs(p - (1 - mu * mu) / (1 + mu * mu)) < 1e-12
        # electric vector direction from (Q, U) in the basis of n2
        th, ph = O.stokes_basis(n2)
        chi = 0.5 * math.atan2(Y[2], Y[1])
        e = math.cos(chi) * th + math.sin(chi) * ph
        assert abs(np.dot(e, unit(np.cross(n, n2)))) > 1 - 1e-10
        assert abs(Y[3]) < 1e-15


def test_rayleigh_matches_dipole_field_projection():
    """Scattered coherency of a dipole: E_out ~ E_in minus its component along n2.
    Checks the full Mueller + both basis rotations for polarized input."""
    for n, n2 in zip(rand_dirs(30), rand_dirs(30)):
        th, ph = O.stokes_basis(n)
        th2, ph2 = O.stokes_basis(n2)
        E = RNG.normal(size=2) + 1j * RNG.normal(size=2)
        Evec = E[0] * th + E[1] * ph
        Eo = Evec - np.dot(n2, Evec) * n2
        e1, e2 = np.dot(Eo, th2), np.dot(Eo, ph2)
        X = [abs(E[0]) ** 2 + abs(E[1]) ** 2, abs(E[0]) ** 2 - abs(E[1]) ** 2,
             2 * (E[0] * np.conj(E[1])).real, 2 * (E[0] * np.conj(E[1])).imag]
        ref = np.array([abs(e1) ** 2 + abs(e2) ** 2, abs(e1) ** 2 - abs(e2) ** 2,
                        2 * (e1 * np.conj(e2)).real, 2 * (e1 * np.conj(e2)).imag]) * 3 / (8 * math.pi)
        Y = O.mueller_apply(X, n, n2, O.rayleigh(float(np.dot(n, n2))))
        assert np.allclose(Y, ref, atol=1e-13)


@pytest.mark.parametrize("incl_deg", [0, 15, 30, 45, 60, 75, 90])
def test_inclined_disk_polarization(incl_deg):
    """Sec. 3.1: single dipole scattering of an in-plane isotropic radiation field,
    seen at inclination i, has p = sin^2 i / (2 + sin^2 i), Q > 0 and U = 0, summed
    through the step-1 camera tally kernel (Z(Omega_cam; Omega_pp) I_pp)."""
    i = math.radians(incl_deg)
    cam = np.array([math.sin(i), 0.0, math.cos(i)])
    tot = np.zeros(4)
    for a in np.arange(16) * 2 * math.pi / 16:
        n = np.array([math.cos(a), math.sin(a), 0.0])
        tot += O.mueller_apply([1, 0, 0, 0], n, cam, O.rayleigh(float(np.dot(n, cam))))
    s2 = math.sin(i) ** 2
    assert abs(tot[1] / tot[0] - s2 / (2 + s2)) < 1e-13
    assert abs(tot[2] / tot[0]) < 1e-13


def test_single_scattering_tally_of_a_thin_slab():
    """eq. (scat-disc-sum) in the single-scattering limit: an unpolarized beam along +z
    through a thin Rayleigh slab (tau = 1e-3, albedo 1, no dichroism).  Between events
    the packet is attenuated by K - omega 1 = 0 and leaves the beam where it scatters,
    so the tally of a z-layer of thickness dz starting at z is, in expectation,
    L Z(Omega_c; z-hat) (1, 0, 0, 0) (e^{-kappa z} - e^{-kappa (z + dz)}) / kappa, with
    Z the Rayleigh matrix 3/(16 pi) (1 + mu^2, mu^2 - 1) at mu = Omega_c . z-hat; scattered
    packets add O(tau).  With Omega_c in the x-z plane the camera's theta-hat lies in the
    scattering plane, so the light, polarized across it, has Q = Z21 I < 0 and U = V = 0."""
    n, tau = 6, 1e-3
    model = W.dichroic_slab(n=n, tau=tau, p=0.0, albedo=1.0)
    angles = [math.radians(d) for d in (30.0, 90.0, 150.0)]
    cams = [W.camera((math.sin(a), 0.0, math.cos(a)), (2, 2), (1.0, 1.0)) for a in angles]
    run = dict(W.beam_run(4000, cameras=cams), n_threads=4)
    o = O.transport(model, run)
    S = o["S"].reshape(n, n, n, len(cams), 4)  # [z][y][x][camera][I,Q,U,V]
    dz = 1.0 / n
    for c, a in enumerate(angles):
        mu = math.cos(a)
        z11, z21 = 3.0 / (16.0 * math.pi) * (1.0 + mu * mu), 3.0 / (16.0 * math.pi) * (mu * mu - 1.0)
        for k in range(n):
            w = (math.exp(-tau * k * dz) - math.exp(-tau * (k + 1) * dz)) / tau
            layer = S[k].sum(axis=(0, 1))[c]
            assert abs(layer[0] - z11 * w) < 3e-3 * z11 * w, (a, k, layer)
            assert abs(layer[1] - z21 * w) < 3e-3 * z11 * w, (a, k, layer)
            assert abs(layer[2]) < 3e-3 * z11 * w and abs(layer[3]) < 1e-12 * z11 * w, (a, k, layer)


def test_single_scattering_tally_with_a_bin_mixture():
    """The same thin-slab limit with tabulated optics of three grain-size bins (Sec. 2.2,
    Mueller elements linear in the scattering angle between tabulated angles): the layer
    sums follow the weighted mixture sum_b w_b (P11_b, P12_b)(Theta) / sum_b w_b, the
    tables interpolated here with numpy at angles between grid points."""
    n, tau = 6, 1e-3
    model = W.dichroic_slab(n=n, tau=tau, p=0.0, albedo=1.0)
    model["optics"] = W.table_optics(n_bins=3, p_max=0.0)
    tabs = np.asarray(model["optics"]["mueller"], dtype=np.float64)
    w = np.asarray(model["optics"]["bin_weight"], dtype=np.float64)
    w = w / w.sum()
    grid = np.linspace(0.0, math.pi, tabs.shape[1])
    angles = [math.radians(d) for d in (37.3, 90.4, 141.7)]
    cams = [W.camera((math.sin(a), 0.0, math.cos(a)), (2, 2), (1.0, 1.0)) for a in angles]
    run = dict(W.beam_run(4000, cameras=cams), n_threads=4)
    o = O.transport(model, run)
    S = o["S"].reshape(n, n, n, len(cams), 4)
    dz = 1.0 / n
    for c, a in enumerate(angles):
        p11 = sum(w[b] * np.interp(a, grid, tabs[b, :, 0]) for b in range(3))
        p12 = sum(w[b] * np.interp(a, grid, tabs[b, :, 1]) for b in range(3))
        for k in range(n):
            f = (math.exp(-tau * k * dz) - math.exp(-tau * (k + 1) * dz)) / tau
            layer = S[k].sum(axis=(0, 1))[c]
            assert abs(layer[0] - p11 * f) < 3e-3 * p11 * f, (a, k, layer)
            assert abs(layer[1] - p12 * f) < 3e-3 * p11 * f, (a, k, layer)


def test_thin_slab_image_carries_the_scattered_power():
    """Step 2's normalisation end to end (S = omega / V * tally per unit extinction optical
    depth, Sec. 2.3 and App. A): for the thin slab above, the image summed over pixels
    times the pixel area is the power scattered per steradian toward the camera,
    L omega (1 - e^{-tau}) Z11(Theta) for I and L omega (1 - e^{-tau}) Z21(Theta) for Q (the
    beam decays with the extinction, a fraction omega of it scattered), up to the slab's
    own extinction of the scattered light and multiple scattering, both O(tau).  Albedo
    0.5, so that a dropped or doubled omega shows."""
    n, tau, omega = 6, 1e-3, 0.5
    model = W.dichroic_slab(n=n, tau=tau, p=0.0, albedo=omega)
    for deg in (30.0, 90.0, 150.0):
        a = math.radians(deg)
        cam = W.camera((math.sin(a), 0.0, math.cos(a)), (90, 90), (3.0, 3.0), center=(0.5, 0.5, 0.5))
        run = dict(W.beam_run(4000, cameras=[cam]), n_threads=4)
        o = O.transport(model, run)
        img = O.image(model, run, o["S"], 0)
        apix = (3.0 / 90) ** 2
        mu = math.cos(a)
        z11, z21 = 3.0 / (16.0 * math.pi) * (1.0 + mu * mu), 3.0 / (16.0 * math.pi) * (mu * mu - 1.0)
        scat = omega * (1.0 - math.exp(-tau))
        assert img[0].sum() * apix == pytest.approx(scat * z11, rel=3e-3), deg
        assert img[1].sum() * apix == pytest.approx(scat * z21, rel=4e-3), deg
        assert abs(img[2].sum() * apix) < 1e-3 * scat * z11 and np.all(img[3] == 0.0), deg


# ---------------------------------------------------------------------------------
# Rejection sampling of the polarization-aware cross section
# ---------------------------------------------------------------------------------
def test_rayleigh_sampler_dipole_pattern():
    """Scattering of light polarized along x travelling along +z follows the dipole
    pattern 1 - n_x^2: <n_x^2> = 1/5, <n_y^2> = <n_z^2> = 2/5.  Unpolarized light:
    cos Theta distributed as 1 + mu^2 (mean mu^2 = 2/5)."""
    model = W.rayleigh_sphere(n=4)
    run = W.rayleigh_sphere_run(n_packets=1)
    k = 20000
    dirs = np.array([O.scatter(model, run, pid, 1, 0, [1, 1, 0, 0], [0, 0, 1])[1] for pid in range(k)])
    m = (dirs ** 2).mean(axis=0)
    sig = 0.3 / math.sqrt(k)
    assert abs(m[0] - 0.2) < 5 * sig and abs(m[1] - 0.4) < 5 * sig and abs(m[2] - 0.4) < 5 * sig
    trials = [O.scatter(model, run, pid, 1, 0, [1, 0, 0, 0], [0, 0, 1]) for pid in range(k)]
    mu = np.array([t[1][2] for t in trials])
    assert abs((mu ** 2).mean() - 0.4) < 5 * 0.3 / math.sqrt(k)
    acc = k / sum(t[0] for t in trials)
    assert abs(acc - 1 / 3) < 0.02
    for t in trials[:200]:
        Y = t[2]
        assert abs(Y[0] - 1.0) < 1e-14
        assert Y[0] ** 2 >= Y[1] ** 2 + Y[2] ** 2 + Y[3] ** 2 - 1e-14


def test_table_sampler_follows_p11():
    """Table proposal + rejection: for unpolarized light the scattering-angle
    distribution is the theta-linear interpolant of P11 (checked on 12 angle bins
    against exact integrals of the interpolant)."""
    model = W.rayleigh_sphere(n=4)
    model["optics"] = W.table_optics(n_bins=8)
    run = W.rayleigh_sphere_run(n_packets=1)
    tab = model["optics"]["mueller"][5].astype(np.float64)
    k = 30000
    mu = np.array([O.scatter(model, run, pid, 1, 5, [1, 0, 0, 0], [0, 0, 1])[1][2] for pid in range(k)])
    theta = np.arccos(np.clip(mu, -1, 1))
    edges = np.linspace(0, math.pi, 13)
    hist = np.histogram(theta, edges)[0]
    tg = np.linspace(0, math.pi, tab.shape[0])

    def p11(t):
        return np.interp(t, tg, tab[:, 0])

    expect = np.array([2 * math.pi * quad(lambda t: p11(t) * math.sin(t), a, b, limit=200)[0]
                       for a, b in zip(edges[:-1], edges[1:])]) * k
    chi2 = np.sum((hist - expect) ** 2 / np.maximum(expect, 1))
    assert chi2 < 40, chi2


# ---------------------------------------------------------------------------------
# Cell-to-cell traversal
# ---------------------------------------------------------------------------------
def test_dda_brute_force_tiny_grids():
    """Sum of segment lengths = chord length of the box; the cell sequence equals
    the one obtained by sorting all plane crossings along the ray."""
    rng = np.random.default_rng(7)
    for _ in range(300):
        shape = rng.integers(1, 5, size=3)
        lo = rng.uniform(-1, 0, 3)
        hi = lo + rng.uniform(0.5, 2, 3)
        p0 = lo + rng.uniform(0.01, 0.99, 3) * (hi - lo)
        n = rand_dirs(1, rng)[0]
        cells, lens = O.dda_walk(shape, lo, hi, p0, n)
        # chord from p0 to the box exit
        t_exit = min(((hi[a] if n[a] > 0 else lo[a]) - p0[a]) / n[a] for a in range(3) if n[a] != 0)
        assert abs(lens.sum() - t_exit) < 1e-12
        # crossings
        d = (hi - lo) / shape
        ts = [0.0]
        for a in range(3):
            for k in range(shape[a] + 1):
                if n[a] != 0:
                    t = (lo[a] + k * d[a] - p0[a]) / n[a]
                    if 1e-12 < t < t_exit - 1e-12:
                        ts.append(t)
        ts = sorted(ts) + [t_exit]
        mids = [(a + b) / 2 for a, b in zip(ts[:-1], ts[1:]) if b - a > 1e-12]
        ref = []
        for t in mids:
            x = p0 + t * n
            ix = np.clip(np.floor((x - lo) / d).astype(int), 0, shape - 1)
            ref.append((ix[2] * shape[1] + ix[1]) * shape[0] + ix[0])
        got = [c for c, l in zip(cells, lens) if l > 1e-12]
        assert got == ref


def test_dda_face_ownership_and_ties():
    # a point on a vertex travelling into the negative octant starts in cell (0,0,0)
    cells, lens = O.dda_walk((2, 2, 2), (-1, -1, -1), (1, 1, 1), (0, 0, 0), unit([-1, -1, -1]))
    assert cells[0] == 0 and len(cells) == 1
    # exact tie along a diagonal in the x-y plane: the x step comes first (lowest axis)
    cells, lens = O.dda_walk((2, 2, 1), (0, 0, 0), (2, 2, 1), (0.5, 0.5, 0.5), unit([1, 1, 0]))
    assert list(cells) == [0, 1, 3]
    assert lens[1] == 0.0


# ---------------------------------------------------------------------------------
# Sec. 3.3: dichroic extinction slab, eq. (ptau)
# ---------------------------------------------------------------------------------
TAUS = [0.1, 1.0, 10.0, 30.0]


@pytest.mark.parametrize("tau", TAUS)
def test_dichroic_slab_transmission(tau):
    """Unpolarized beam through a uniformly aligned slab (alpha2 = -0.05, field at
    45 deg): I/I0 = e^-tau cosh(0.05 tau), Q/I = +tanh(0.05 tau) (along the
    projected field), U = V = 0, absorbed = 1 - I/I0.  Inputs are FP32, so the
    closed form is evaluated at the FP32 values of tau and 0.05."""
    t, p = f32(tau), -f32(-0.05)
    model = W.dichroic_slab(n=8, tau=tau)
    run = W.beam_run(8, seed=1)
    run["n_trace"] = 8
    out = O.transport(model, run)
    tr = out["trace"]
    I = tr[:, 0] / tr[:, 13]
    assert np.allclose(I, math.exp(-t) * math.cosh(p * t), rtol=1e-12)
    assert np.allclose(tr[:, 1] / tr[:, 0], math.tanh(p * t), rtol=1e-12)
    assert np.all(np.abs(tr[:, 2:4] / tr[:, :1]) < 1e-15)
    st = out["stats"]
    assert abs(st["absorbed_energy"] + st["escaped_energy"] - st["emitted_energy"]) < 1e-14
    assert abs(st["absorbed_energy"] - (1 - math.exp(-t) * math.cosh(p * t))) < 1e-12


@pytest.mark.parametrize("tau", TAUS)
@pytest.mark.parametrize("n", [1, 8])
def test_ptau_emission_through_imaging(tau, n):
    """eq. (ptau), Hildebrand (2000): an isothermal aligned slab seen face-on has
    |Q|/I = e^-tau sinh(p0 tau) / (1 - e^-tau cosh(p0 tau)), polarized across the
    projected field (Q < 0 here), via step 2 with the emission source alpha_abs B.
    Tolerance: 1e-5 relative, floored at 1e-15 in Q/I (FP64 rounding of the basis
    rotations leaks ~1e-16 of I into Q)."""
    t, p = f32(tau), -f32(-0.05)
    model = W.dichroic_slab(n=n, tau=tau, emissivity=1.0)
    run = W.beam_run(1, cameras=[W.camera((0, 0, 1), (3, 3), (0.5, 0.5))])
    img = O.image(model, run, None, 0)
    P = math.exp(-t) * math.sinh(p * t) / (1 - math.exp(-t) * math.cosh(p * t))
    I, Q, U, V = img[:, 1, 1]
    assert abs(I - (1 - math.exp(-t) * math.cosh(p * t))) < 1e-13
    assert abs(-Q / I - P) <= max(1e-5 * P, 1e-15)
    assert abs(U) < 1e-15 and abs(V) < 1e-15


# ---------------------------------------------------------------------------------
# Sec. 3.2: twisted field, eq. (analytical-qu)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("tau", [0.125, 0.3, 0.5, 0.8, 1.0])
def test_twisted_field_slab(tau):
    """Unpolarized light generated at optical depth tau travelling to the face
    through a field rotating by 2 pi per unit tau, with the artificial U-V term
    alpha3 = -alpha2 (K_VU = K_QI): Q/I, U/I and V/I follow eq. (analytical-qu) to
    O(p0^3); with p0 = 0.01 that is < 1e-7 absolute on Q/I, U/I and 1e-3 relative
    on V/I at 400 layers per unit tau."""
    p0 = 0.01
    model = W.twisted_slab(tau, p0=p0, nz_per_tau=400)
    run = W.beam_run(1, seed=3, direction=-1)
    run["n_trace"] = 1
    tr = O.transport(model, run)["trace"][0]
    I, Q, U, V = tr[:4]
    k = p0 / (4 * math.pi)
    x = 4 * math.pi * tau
    assert abs(Q / I - k * math.sin(x)) < 1e-7
    assert abs(U / I + k * (1 - math.cos(x))) < 1e-7
    v_ref = k * k * (math.sin(x) - x)
    assert abs(V / I - v_ref) < 1e-3 * abs(v_ref)
    # without the artificial term no circular polarization appears
    model = W.twisted_slab(tau, p0=p0, nz_per_tau=400, coupling=False)
    tr = O.transport(model, run)["trace"][0]
    assert abs(tr[3] / tr[0]) < 1e-15


# ---------------------------------------------------------------------------------
# Invariants of the full transport
# ---------------------------------------------------------------------------------
def test_energy_conservation_and_realizability_rayleigh_sphere():
    """Albedo 1: every packet escapes with its birth energy; escaped + absorbed =
    emitted; I^2 >= Q^2 + U^2 + V^2 at the end of every packet."""
    model = W.rayleigh_sphere(n=16, tau=2.0)
    run = W.rayleigh_sphere_run(n_packets=3000, npix=16)
    run["n_trace"] = 3000
    out = O.transport(model, run)
    st = out["stats"]
    assert st["escaped"] == 3000
    assert abs(st["escaped_energy"] - st["emitted_energy"]) < 1e-12
    assert abs(st["absorbed_energy"]) < 1e-12  # only basis-rotation rounding of I
    tr = out["trace"]
    assert np.all(tr[:, 0] ** 2 >= (tr[:, 1:4] ** 2).sum(axis=1) * (1 - 1e-12))
    assert np.allclose(np.linalg.norm(tr[:, 7:10], axis=1), 1.0, atol=1e-12)
    assert tr[:, 10].mean() > 0.5  # radial optical depth 2 scatters most packets


def test_energy_balance_absorbing_disk_with_roulette():
    """Absorbing medium with roulette and both sources: escaped + absorbed +
    roulette losses - roulette gains + capped = emitted, to rounding."""
    model = W.disk(n=24)
    run = W.disk_run(n_packets=1000, n_cam=2, npix=8)
    run["n_trace"] = 1000
    out = O.transport(model, run)
    st = out["stats"]
    bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
    assert abs(bal - st["emitted_energy"]) < 1e-10 * st["emitted_energy"]
    assert abs(out["absorbed"].sum() - st["absorbed_energy"]) < 1e-10 * st["emitted_energy"]
    tr = out["trace"]
    assert np.all(tr[:, 0] ** 2 >= (tr[:, 1:4] ** 2).sum(axis=1) * (1 - 1e-12))
    assert st["roulette_killed"] > 0 and st["scatterings"] > 0


def test_point_and_beam_births_follow_their_definitions():
    """Packet birth (Sec. 2.2): a point source emits unpolarized packets of energy L/N
    from its position in isotropic directions (n_z and the azimuth uniform); a plane
    beam enters uniformly over the face it starts on, along +z or -z.  Kolmogorov-
    Smirnov distances against the uniform law (bound 1.63 / sqrt(N), the 1 % level)."""
    from scipy import stats

    model = W.dichroic_slab(n=4, tau=1.0, albedo=0.5)
    N = 20000
    crit = 1.63 / math.sqrt(N)
    run = {"sources": [{"type": "point", "pos": (0.3, 0.6, 0.5), "luminosity": 2.0, "n_packets": N},
                       {"type": "beam", "beam_dir": 1, "luminosity": 1.0, "n_packets": N},
                       {"type": "beam", "beam_dir": -1, "luminosity": 3.0, "n_packets": N}], "seed": 17}
    rows = O.emit(model, run, range(3 * N))
    pt, up, down = rows[:N], rows[N:2 * N], rows[2 * N:]
    assert np.all(pt[:, 12] == 0) and np.all(up[:, 12] == 1) and np.all(down[:, 12] == 2)
    # point source: fixed position, energy L / N, unpolarized, isotropic
    assert np.allclose(pt[:, 0:3], (0.3, 0.6, 0.5), atol=1e-15)
    assert np.allclose(pt[:, 6], 2.0 / N, rtol=1e-14) and np.all(pt[:, 7:10] == 0.0)
    assert np.allclose(np.linalg.norm(pt[:, 3:6], axis=1), 1.0, atol=1e-14)
    assert stats.kstest((pt[:, 5] + 1) / 2, "uniform").statistic < crit
    phi = (np.arctan2(pt[:, 4], pt[:, 3]) + math.pi) / (2 * math.pi)
    assert stats.kstest(phi, "uniform").statistic < crit
    # beams: on their face, uniform over it, along the axis, energy L / N
    for b, z0, nz, L in ((up, 0.0, 1.0, 1.0), (down, 1.0, -1.0, 3.0)):
        assert np.all(b[:, 2] == z0) and np.all(b[:, 5] == nz) and np.all(b[:, 3:5] == 0.0)
        assert np.allclose(b[:, 6], L / N, rtol=1e-14) and np.all(b[:, 7:10] == 0.0)
        for a in (0, 1):
            assert stats.kstest(b[:, a], "uniform").statistic < crit
    # the optical depth to the first scattering is exponential with mean 1
    assert stats.kstest(pt[:, 10], "expon").statistic < crit


def test_thermal_birth_polarization():
    """Thermal emission alpha_abs B: at birth the packet is polarized across the
    projected field with degree |alpha2| / (alpha1 - omega)."""
    model = W.dichroic_slab(n=4, tau=1.0, albedo=0.3, emissivity=1.0)
    run = {"sources": [{"type": "thermal", "n_packets": 200}], "seed": 9}
    rows = O.emit(model, run, range(200))
    b = unit([math.sin(math.radians(45)), 0, math.cos(math.radians(45))])
    for r in rows:
        n, X = r[3:6], r[6:10]
        sin2 = 1 - np.dot(n, b) ** 2
        th, ph = O.stokes_basis(n)
        bperp = unit(b - np.dot(b, n) * n)
        chi = math.atan2(np.dot(bperp, ph), np.dot(bperp, th))  # field direction angle
        kap = f32(0.7) + f32(0.3)
        omega = f32(0.3) / kap
        degree = f32(0.05) / (1 - omega)
        # constant alpha2 table: the degree does not depend on theta'
        assert abs(math.hypot(X[1], X[2]) / X[0] - degree) < 1e-6
        # polarized perpendicular to the projected field: angle chi + 90 deg
        assert abs(X[1] / X[0] - degree * math.cos(2 * chi + math.pi)) < 1e-6
        assert abs(X[2] / X[0] - degree * math.sin(2 * chi + math.pi)) < 1e-6
        assert sin2 >= 0


def test_thermal_cell_selection_follows_weights():
    """Birth cells are drawn in proportion to kappa_abs B V."""
    model = W.dichroic_slab(n=2, tau=1.0, emissivity=1.0)
    em = np.array([[[1, 2], [3, 4]], [[0, 1], [5, 0]]], dtype=np.float32)
    model["emissivity"] = em
    run = {"sources": [{"type": "thermal", "n_packets": 20000}], "seed": 11}
    rows = O.emit(model, run, range(20000))
    idx = np.floor(rows[:, :3] / 0.5).astype(int)
    cell = (idx[:, 2] * 2 + idx[:, 1]) * 2 + idx[:, 0]
    h = np.bincount(cell, minlength=8) / 20000
    w = em.ravel() / em.sum()
    assert np.all(np.abs(h - w) < 5 * np.sqrt(w * (1 - w) / 20000) + 1e-12)
    L = O.thermal_luminosity(model, run)
    assert abs(L - 4 * math.pi * em.sum() * f32(1.0) * 0.125) < 1e-9


# ---------------------------------------------------------------------------------
# App. A and eq. polarized-rt with extinction elements that depend on theta'
# ---------------------------------------------------------------------------------
# alpha1..3 on 5 nodes theta'_j = 45 j deg; FP32 as the ABI takes them
KEXT5 = np.array([[1.0, 0.0, 0.0], [1.3, -0.1, 0.02], [2.0, -0.3, 0.05], [1.5, -0.05, 0.01], [1.1, 0.0, 0.0]],
                 dtype=np.float32)
NODES5 = np.radians([0.0, 45.0, 90.0, 135.0, 180.0])


def alpha_by_hand(thetap):
    """alpha1..3 at theta', linear in theta' between the two nodes around it."""
    return np.array([np.interp(thetap, NODES5, KEXT5[:, e].astype(np.float64)) for e in range(3)])


def aligned_slab(tau, b, albedo=0.0, emissivity=None, n=4):
    """[0,1]^3 slab, kappa_ext = tau, uniform field b, the 5-node extinction table."""
    shape = (n, n, n)
    kext = np.full(shape, tau, dtype=np.float32)
    bf = np.zeros(shape + (3,), dtype=np.float32)
    bf[...] = np.asarray(b, dtype=np.float32)
    em = None if emissivity is None else np.full(shape, emissivity, dtype=np.float32)
    return {"lo": (0.0, 0.0, 0.0), "hi": (1.0, 1.0, 1.0), "kappa_abs": (kext * (1 - albedo)).astype(np.float32),
            "kappa_sca": (kext * albedo).astype(np.float32), "bfield": bf, "emissivity": em,
            "optics": {"model": "rayleigh", "kext": KEXT5}}


@pytest.mark.parametrize("theta_b,phi_b", [(30.0, 0.0), (30.0, 30.0), (100.0, -70.0), (160.0, 10.0)])
def test_dichroic_slab_with_angle_dependent_extinction(theta_b, phi_b):
    """App. A: an unpolarized beam along +z through a uniformly aligned slab with the
    field at polar angle theta_B (so theta' = theta_B for every packet) leaves with
    I/I0 = e^(-alpha1 tau) cosh(alpha2 tau) and degree tanh(|alpha2| tau) along the
    projected field, alpha_i interpolated by hand linearly in theta' between the
    table's nodes.  Interpolating in cos theta', or taking theta' from the lab polar
    angle of n, gives other alphas."""
    tau = 2.0
    tb, pb = math.radians(theta_b), math.radians(phi_b)
    b32 = np.array([math.sin(tb) * math.cos(pb), math.sin(tb) * math.sin(pb), math.cos(tb)], dtype=np.float32)
    b = b32.astype(np.float64)
    thetap = math.atan2(math.hypot(b[0], b[1]), b[2])
    a1, a2, _ = alpha_by_hand(thetap)
    t = f32(tau)
    model = aligned_slab(tau, b32)
    run = W.beam_run(4, seed=1)
    run["n_trace"] = 4
    out = O.transport(model, run)
    tr = out["trace"]
    I = tr[:, 0] / tr[:, 13]
    ref_I = math.exp(-a1 * t) * math.cosh(a2 * t)
    assert np.allclose(I, ref_I, rtol=1e-10), (I, ref_I)
    # n = +z: theta-hat = x-hat, phi-hat = y-hat; the projected field is at angle phi_B
    deg = math.tanh(abs(a2) * t)
    chi = math.atan2(b[1], b[0])
    assert np.allclose(tr[:, 1] / tr[:, 0], deg * math.cos(2 * chi), atol=1e-12)
    assert np.allclose(tr[:, 2] / tr[:, 0], deg * math.sin(2 * chi), atol=1e-12)
    assert np.all(np.abs(tr[:, 3] / tr[:, 0]) < 1e-15)
    assert abs(out["stats"]["absorbed_energy"] - (1 - ref_I)) < 1e-10


def alpha1_sphere_mean_by_quadrature():
    """1/2 int_0^pi alpha1(theta') sin theta' dtheta' of the theta'-linear interpolant."""
    f = lambda th: float(alpha_by_hand(th)[0]) * math.sin(th)
    return 0.5 * sum(quad(f, NODES5[j], NODES5[j + 1], epsabs=1e-14, epsrel=1e-13)[0] for j in range(4))


def test_thermal_luminosity_uses_the_sphere_average_of_alpha1():
    """eq. polarized-rt: the emission alpha_abs B summed over directions is
    4 pi kappa_ext (<alpha1> - omega) B per unit volume, <alpha1> the average of
    alpha1(theta') over the sphere (scipy quadrature of the interpolant; its plain
    mean over theta' would differ by 8 %)."""
    for albedo in (0.0, 0.3):
        model = aligned_slab(1.5, (0.6, 0.0, 0.8), albedo=albedo, emissivity=2.0)
        run = {"sources": [{"type": "thermal", "n_packets": 10}], "seed": 9}
        ka, ks = float(model["kappa_abs"][0, 0, 0]), float(model["kappa_sca"][0, 0, 0])
        kext = ka + ks
        omega = ks / kext
        L = O.thermal_luminosity(model, run)
        ref = 4 * math.pi * kext * (alpha1_sphere_mean_by_quadrature() - omega) * 2.0 * 1.0
        assert abs(L - ref) < 1e-12 * ref, (L, ref)


def test_thermal_births_with_angle_dependent_extinction():
    """eq. polarized-rt with alpha_abs = K - omega 1 acting on (B,0,0,0): a packet
    emitted along n carries weight (alpha1(theta') - omega) / (<alpha1> - omega) and
    degree |alpha2(theta')| / (alpha1(theta') - omega) across the projected field,
    theta' the angle between n and the field."""
    albedo = 0.3
    b32 = np.array([0.6, 0.0, 0.8], dtype=np.float32)
    b = unit(b32.astype(np.float64))
    model = aligned_slab(1.5, b32, albedo=albedo, emissivity=1.0)
    N = 400
    run = {"sources": [{"type": "thermal", "luminosity": 1.0, "n_packets": N}], "seed": 9}
    rows = O.emit(model, run, range(N))
    ka, ks = float(model["kappa_abs"][0, 0, 0]), float(model["kappa_sca"][0, 0, 0])
    omega = ks / (ka + ks)
    mean1 = alpha1_sphere_mean_by_quadrature()
    eps = 1.0 / N
    thetaps = []
    for r in rows:
        n, X = r[3:6], r[6:10]
        thetap = math.acos(max(-1.0, min(1.0, float(np.dot(n, b)))))
        thetaps.append(thetap)
        a1, a2, _ = alpha_by_hand(thetap)
        assert abs(X[0] / eps - (a1 - omega) / (mean1 - omega)) < 1e-9
        th, ph = O.stokes_basis(n)
        bperp = b - np.dot(b, n) * n
        chi = math.atan2(np.dot(bperp, ph), np.dot(bperp, th))
        deg = abs(a2) / (a1 - omega)
        assert abs(X[1] / X[0] - deg * math.cos(2 * chi + math.pi)) < 1e-9
        assert abs(X[2] / X[0] - deg * math.sin(2 * chi + math.pi)) < 1e-9
    # the draw covers several table intervals
    assert len(np.unique(np.digitize(thetaps, NODES5))) >= 4


# ---------------------------------------------------------------------------------
# Sec. 3.1: the inclined-disk test through step 1 and step 2
# ---------------------------------------------------------------------------------
def test_inclined_thin_disk_through_both_steps():
    """Sec. 3.1 (Yang et al. 2016): light of a central star reaching a geometrically and
    optically thin annulus of Rayleigh grains travels in the disk plane; scattered once
    and imaged at inclination i its integrated Q/I is sin^2 i / (2 + sin^2 i) and U/I = 0.
    Step 1 (tally) and step 2 (images, 512^2) of the oracle with 32 M packets; the gate
    is 4 sigma plus 1e-4 for the pixel quadrature of the images, sigma from the spread
    of 16 packet batches of the tally.  The light is in the plane only to h / r_in: the
    expectation includes its <k_z^2>."""
    import closed_forms as CF

    model = W.inclined_thin_disk()
    g = model["geometry"]
    kz2 = CF.thin_annulus_kz2(g["h"], g["r_in"], g["r_out"])
    assert kz2 < 2e-4
    nb, per = 16, 2_000_000
    run = W.thin_disk_run(nb * per, npix=512)
    S = None
    sums = np.zeros((nb, len(run["cameras"]), 4))
    for b in range(nb):
        o = O.transport(model, dict(run, pid_begin=b * per, pid_end=(b + 1) * per, n_threads=os.cpu_count() or 1))
        sums[b] = o["S"].sum(axis=0)
        S = o["S"] if S is None else S + o["S"]
    for k, a in enumerate((0, 15, 30, 45, 60, 75, 90)):
        i = math.radians(a)
        img = O.image(model, run, S, k).sum(axis=(1, 2))
        q = sums[:, k, 1] / sums[:, k, 0]
        u = sums[:, k, 2] / sums[:, k, 0]
        sq, su = q.std(ddof=1) / math.sqrt(nb), u.std(ddof=1) / math.sqrt(nb)
        p = CF.inclined_disk_p(i, kz2)
        assert abs(img[1] / img[0] - p) < 4 * sq + 1e-4, (a, img[1] / img[0], p, sq)
        assert abs(img[2] / img[0]) < 4 * su + 1e-4, (a, img[2] / img[0], su)
        assert abs(img[3]) < 1e-12 * img[0]
    # the expectation moves with i as the paper's curve: 0 face-on, 1/3 edge-on
    assert CF.inclined_disk_p(0.0) == 0.0 and abs(CF.inclined_disk_p(math.pi / 2) - 1 / 3) < 1e-15


def test_sweep_generator_statistics():
    """Batched-sweep inputs: ln rho has unit variance (sigma_ln = 1) and <rho> ~ 1;
    kappa scales as lambda^-1.5 between the wavelengths of one model."""
    r = W.clumpy_density(48, 3)
    assert abs(np.log(r).std() - 1.0) < 1e-9
    assert abs(r.mean() - 1.0) < 0.1
    ms = W.sweep_models(n_models=2, n_lambda=3, n_min=8, n_max=10)
    for m in range(2):
        a, b = ms[3 * m], ms[3 * m + 2]
        k_a = a["kappa_abs"] + a["kappa_sca"]
        k_b = b["kappa_abs"] + b["kappa_sca"]
        ratio = (b["lambda_um"] / a["lambda_um"]) ** -1.5
        assert np.allclose(k_b, k_a * ratio, rtol=1e-5)
        assert 1.0 <= a["tau"] <= 100.0


# ---------------------------------------------------------------------------------
# grain-optics surrogate: labels and the FP64 MLP reference
# ---------------------------------------------------------------------------------
def test_surrogate_labels_reduce_to_the_tables():
    """At the tabulated sizes the label matrix is the bin table in the scattering-plane
    basis; applied with the plane rotations it is the oracle's scattering transfer;
    between sizes it interpolates in ln x; alpha follows the extinction table;
    realizable (M11 >= |row 1|, |column 1|)."""
    from oracle import mlp_oracle as MO

    opt = W.table_optics(n_bins=8)
    tabs, kext = opt["mueller"], opt["kext"]
    rng = np.random.default_rng(5)
    for trial in range(40):
        ni, ns = rand_dirs(2, rng)
        k = trial % 8
        s = -1.0 + 2.0 * k / 7
        lab = MO.label(np.r_[ni, ns, s], tabs, kext)
        N = math.exp(lab[19])
        Z = MO.matrix(lab)
        mu = float(np.dot(ni, ns))
        P = MO.theta_interp(tabs[k].astype(np.float64), mu)
        assert abs(N - tabs[k][:, 0].max()) < 1e-6 * N
        # the 4x4 form of the six table elements
        ref = np.array([[P[0], P[1], 0, 0], [P[1], P[2], 0, 0], [0, 0, P[3], P[4]], [0, 0, -P[4], P[5]]])
        assert np.allclose(Z, ref, rtol=1e-12, atol=1e-12 * P[0])
        # with the plane rotations: the oracle's scattering transfer of a polarized input
        X = np.array([1.0, 0.3, -0.2, 0.1])
        Zg = np.array([O.mueller_apply(e, ni, ns, P) for e in np.eye(4)]).T
        assert np.allclose(Zg @ X, O.mueller_apply(X, ni, ns, Z[[0, 0, 1, 2, 2, 3], [0, 1, 1, 2, 3, 3]]))
        assert Z[0, 0] ** 2 >= Z[0, 1] ** 2 + Z[0, 2] ** 2 + Z[0, 3] ** 2 - 1e-12
        a = MO.kext_interp(kext, ni[2])
        assert np.allclose(lab[16:19], a)
    # halfway between bins 2 and 3 in ln x
    ni, ns = rand_dirs(2, rng)
    s = -1.0 + 2.0 * 2.5 / 7
    lab = MO.label(np.r_[ni, ns, s], tabs, kext)
    mid = 0.5 * (tabs[2].astype(np.float64) + tabs[3].astype(np.float64))
    P = MO.theta_interp(mid, float(np.dot(ni, ns)))
    assert abs(math.exp(lab[0]) - (MO.matrix(lab) @ [1, 0, 0, 0])[0]) < 1e-12 * math.exp(lab[0])
    assert abs((MO.matrix(lab) @ [1, 0, 0, 0])[0] - P[0]) < 1e-6 * P[0]
    # the ratios of a realizable matrix: row 1 and column 1 within the unit ball
    assert lab[1] ** 2 + lab[2] ** 2 + lab[3] ** 2 <= 1 + 1e-12
    assert lab[4] ** 2 + lab[8] ** 2 + lab[12] ** 2 <= 1 + 1e-12


def test_mlp_reference_gradients_by_central_differences():
    from oracle import mlp_oracle as MO

    rng = np.random.default_rng(9)
    params = [(rng.normal(scale=1 / math.sqrt(ni), size=(no, ni)), rng.normal(scale=0.1, size=no))
              for ni, no in MO.LAYERS]
    x = MO.pad_inputs(rng.uniform(-1, 1, size=(5, MO.N_IN)))
    t = rng.normal(size=(5, MO.N_OUT))
    w = rng.uniform(0.5, 2.0, size=MO.N_OUT)
    loss, grads = MO.loss_and_grads(params, x, t, w)
    h = 1e-6
    for li in (0, 2, 4):
        W, b = params[li]
        for (i, j) in [(0, 0), (3, 5), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp = W.copy(); Wp[i, j] += h
            Wm = W.copy(); Wm[i, j] -= h
            pp = list(params); pp[li] = (Wp, b)
            pm = list(params); pm[li] = (Wm, b)
            num = (MO.loss_and_grads(pp, x, t, w)[0] - MO.loss_and_grads(pm, x, t, w)[0]) / (2 * h)
            assert abs(num - grads[li][0][i, j]) < 1e-7 * max(1.0, abs(num)), (li, i, j)
        bp = b.copy(); bp[1] += h
        bm = b.copy(); bm[1] -= h
        pp = list(params); pp[li] = (W, bp)
        pm = list(params); pm[li] = (W, bm)
        num = (MO.loss_and_grads(pp, x, t, w)[0] - MO.loss_and_grads(pm, x, t, w)[0]) / (2 * h)
        assert abs(num - grads[li][1][1]) < 1e-7 * max(1.0, abs(num))


# ---------------------------------------------------------------------------------
# periodic boundaries (the paper's periodic conditions of its dust-cylinder test)
# ---------------------------------------------------------------------------------
def test_periodic_slab_oblique_escape_closed_form():
    """Absorbing slab z in [0, 1] (kappa = tau), x and y periodic, isotropic point
    source at the centre: a packet can only leave through z = 0 or z = 1, after the
    path 0.5 / |n_z| whatever the number of periodic re-entries, so
    I = (L / N) exp(-tau 0.5 / |n_z|) exactly.  Without the periodic faces packets
    escape sideways with more intensity."""
    tau, N = 1.5, 3000
    model = W.plane_parallel_slab(nxy=4, nz=8, tau=tau, albedo=0.0, periodic=3)
    run = dict(W.center_source_run(N), n_trace=N, max_events=10_000_000)
    o = O.transport(model, run)
    tr = o["trace"]
    esc = tr[:, 12] == 1
    assert esc.mean() > 0.999
    nz = tr[esc, 9]
    zf = tr[esc, 6]
    assert np.all(np.isclose(zf, 0.0, atol=1e-12) | np.isclose(zf, 1.0, atol=1e-12))
    expect = (1.0 / N) * np.exp(-tau * 0.5 / np.abs(nz))
    assert np.allclose(tr[esc, 0], expect, rtol=1e-10, atol=1e-300)
    # no dichroism: unpolarized up to the basis rotations' rounding (of the birth intensity)
    assert np.all(np.abs(tr[esc, 1:4]) <= 1e-14 * tr[esc, 13:14])
    st = o["stats"]
    assert abs(st["escaped_energy"] + st["absorbed_energy"] + st["cap_lost"] - st["emitted_energy"]) < 1e-12
    # the same slab with outflow sides: some packets leave through x or y, brighter
    model0 = dict(model, periodic=0)
    o0 = O.transport(model0, run)
    side = ~(np.isclose(o0["trace"][:, 6], 0.0) | np.isclose(o0["trace"][:, 6], 1.0))
    assert side.mean() > 0.3
    assert o0["stats"]["escaped_energy"] > st["escaped_energy"]


def test_periodic_scattering_slab_conserves_energy_and_symmetry():
    """Scattering slab with periodic x, y: energy conservation, and the absorbed energy
    per z layer is mirror-symmetric about the source's midplane (to Monte-Carlo
    accuracy)."""
    model = W.plane_parallel_slab(nxy=4, nz=10, tau=2.0, albedo=0.7, periodic=3)
    run = dict(W.center_source_run(20_000), n_threads=4)
    o = O.transport(model, run)
    st = o["stats"]
    bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
    assert abs(bal - st["emitted_energy"]) < 1e-9 * st["emitted_energy"]
    layers = o["absorbed"].reshape(10, 16).sum(axis=1)
    assert np.abs(layers - layers[::-1]).max() < 0.05 * layers.max()
