"""Pins of the oracle's aligned-spheroid dipole optics (grain optics in the dipole
approximation with K from the optical theorem, Sec. 2.1 and Sec. 3; the general
scattering weight for direction- and polarization-dependent cross sections).

Each pin checks the oracle against something other than its own formulas: the
depolarization factor against numerical quadrature of the ellipsoid integral, the
polarizabilities against the sphere limit and exact energy conservation, the Jones
scattering against the Rayleigh matrix, the dipole radiation integral and purity,
K against the optical-theorem cross section of arbitrary linear polarizations, and the
transport against closed forms (unscattered fractions, a deterministic single-segment
tally) and expectation values (energy balance of a pure scatterer)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.linalg import expm

from oracle import oracle as O
from paper_2512_01283_gb300 import workloads as W

RNG = np.random.default_rng(2468)
EPS = complex(2.30, 0.0228) ** 2  # refractory grains of the circumstellar test (Sec. 3.5)


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def rand_dir():
    return unit(RNG.normal(size=3))


def rand_stokes(pure=False):
    p = 1.0 if pure else RNG.uniform(0, 1)
    v = unit(RNG.normal(size=3)) * p
    return np.array([1.0, v[0], v[1], v[2]]) * RNG.uniform(0.5, 2.0)


# ---------------------------------------------------------------------------------
# grain constants
# ---------------------------------------------------------------------------------
def quad_L(s):
    """Ellipsoid depolarization integral L_i = (abc/2) int dq / ((a_i^2 + q) f(q)),
    f = sqrt((a^2+q)(b^2+q)(c^2+q)), for the symmetry semi-axis 1 and equatorial s."""
    sym = quad(lambda q: 1.0 / ((1.0 + q) ** 1.5 * (q + s * s)), 0, np.inf, epsabs=0, epsrel=1e-13, limit=500)[0]
    eq = quad(lambda q: 1.0 / ((s * s + q) ** 2 * math.sqrt(1.0 + q)), 0, np.inf, epsabs=0, epsrel=1e-13,
              limit=500)[0]
    return 0.5 * s * s * sym, 0.5 * s * s * eq


@pytest.mark.parametrize("s", [0.2, 0.5, 0.8, 0.95, 1.0, 1.03, 1.2, 1.22, 1.25, 1.5, 2.0, 4.0, 10.0])
def test_spheroid_depolarization_factor_against_quadrature(s):
    Ls, Le = quad_L(s)
    assert abs(Ls + 2 * Le - 1.0) < 1e-10  # sum rule of the quadratures themselves
    assert abs(O.spheroid_L(s) - Ls) < 1e-10
    d = O.dipole_constants(EPS, s, 0.1)
    assert abs(d["L1"] - Ls) < 1e-10 and abs(d["L0"] - Le) < 1e-10


def test_depolarization_limits():
    assert O.spheroid_L(1.0) == pytest.approx(1 / 3, abs=1e-15)
    assert O.spheroid_L(1e4) > 0.999  # flat disk: the field along the normal is screened
    assert O.spheroid_L(1e-3) < 1e-4  # needle


def test_sphere_limit_is_the_rayleigh_sphere():
    """s = 1: alpha = (eps - 1)/(eps + 2) a^3 and the small-particle efficiencies
    Q_abs = 4 x Im((eps-1)/(eps+2)), Q_sca = (8/3) x^4 |(eps-1)/(eps+2)|^2."""
    x = 1e-3
    d = O.dipole_constants(EPS, 1.0, x)
    cm = (EPS - 1) / (EPS + 2)
    for j in (0, 1):
        a = complex(d["al%d_re" % j], d["al%d_im" % j])
        assert abs(a - cm) < 1e-8 * abs(cm)
        assert d["q_abs%d" % j] == pytest.approx(4 * x * cm.imag, rel=1e-6)
        assert d["q_sca%d" % j] == pytest.approx(8 / 3 * x ** 4 * abs(cm) ** 2, rel=1e-6)
    assert complex(d["rho_re"], d["rho_im"]) == pytest.approx(1.0, abs=1e-14)
    assert d["zn"] == pytest.approx(3 / (8 * math.pi), rel=1e-14)


@pytest.mark.parametrize("s", [0.5, 1.0, 2.0])
def test_radiative_reaction_conserves_energy(s):
    """A non-absorbing grain (real eps) absorbs nothing: Q_ext = Q_sca exactly (the
    optical theorem with the radiative-reaction correction); an absorbing one has
    Q_abs > 0 on both axes."""
    for x in (0.05, 0.3, 1.0):
        d = O.dipole_constants(2.25, s, x)
        for j in (0, 1):
            assert abs(d["q_abs%d" % j]) <= 1e-13 * d["q_ext%d" % j]
        d = O.dipole_constants(EPS, s, x)
        assert d["q_abs0"] > 0 and d["q_abs1"] > 0


def test_oblate_grains_respond_less_along_their_short_axis():
    d = O.dipole_constants(EPS, 2.0, 0.3)
    assert d["q_abs1"] < d["q_abs0"] and d["q_sca1"] < d["q_sca0"]
    d = O.dipole_constants(EPS, 0.5, 0.3)  # prolate: the symmetry axis is the long one
    assert d["q_abs1"] > d["q_abs0"] and d["q_sca1"] > d["q_sca0"]


# ---------------------------------------------------------------------------------
# scattering matrix
# ---------------------------------------------------------------------------------
def coherency(X):
    return 0.5 * np.array([[X[0] + X[1], X[2] + 1j * X[3]], [X[2] - 1j * X[3], X[0] - X[1]]])


def radiated_power(d, axis, X, n):
    """Power radiated by the induced dipole, (8 pi / 3) <|p|^2>, with p = A E,
    A = 1 + (rho - 1) axis axis^T, in units of alpha'_0, times zn."""
    rho = complex(d["rho_re"], d["rho_im"])
    A = np.eye(3) + (rho - 1) * np.outer(axis, axis)
    th, ph = O.stokes_basis(n)
    F = np.stack([th, ph], axis=1)  # 3 x 2
    G = F @ coherency(X) @ F.T  # 3-d coherency of E
    return d["zn"] * 8 * math.pi / 3 * np.trace(A @ G @ A.conj().T).real


def test_sphere_scattering_matrix_is_rayleigh():
    for _ in range(40):
        X, n, n2, axis = rand_stokes(), rand_dir(), rand_dir(), rand_dir()
        got = O.dipole_scatter(EPS, 1.0, 0.2, axis, X, n, n2)
        want = O.mueller_apply(X, n, n2, O.rayleigh(float(np.dot(n, n2))))
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14 * X[0])


def test_incidence_along_the_axis_scatters_like_a_sphere():
    """With n along the symmetry axis the incident field only excites alpha_0, so the
    pattern is Rayleigh's scaled by zn / (3 / 8 pi)."""
    d = O.dipole_constants(EPS, 2.0, 0.3)
    for _ in range(20):
        X, axis, n2 = rand_stokes(), rand_dir(), rand_dir()
        got = O.dipole_scatter(EPS, 2.0, 0.3, axis, X, axis, n2)
        want = O.mueller_apply(X, axis, n2, O.rayleigh(float(np.dot(axis, n2)))) * d["zn"] / (3 / (8 * math.pi))
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14 * X[0])


@pytest.mark.parametrize("s", [0.5, 2.0])
def test_scattered_power_integrates_to_the_dipole_radiation(s):
    """int (Z X)_0 dOmega over the sphere (Gauss-Legendre x uniform azimuth) equals
    the closed-form radiated power of the induced dipole."""
    d = O.dipole_constants(EPS, s, 0.3)
    mu, wmu = np.polynomial.legendre.leggauss(24)
    phis = (np.arange(48) + 0.5) * 2 * math.pi / 48
    for _ in range(4):
        X, n, axis = rand_stokes(), rand_dir(), rand_dir()
        tot = 0.0
        for m, w in zip(mu, wmu):
            st = math.sqrt(1 - m * m)
            for p in phis:
                n2 = np.array([st * math.cos(p), st * math.sin(p), m])
                tot += w * (2 * math.pi / 48) * O.dipole_scatter(EPS, s, 0.3, axis, X, n, n2)[0]
        assert tot == pytest.approx(radiated_power(d, axis, X, n), rel=1e-12)


def test_orientation_average_of_the_scattered_power_is_one():
    """zn normalises the scattering matrix to the orientation-averaged cross section:
    the mean over random axes of the radiated power of unpolarized light is 1."""
    d = O.dipole_constants(EPS, 2.0, 0.3)
    n = np.array([0.0, 0.0, 1.0])
    mu, wmu = np.polynomial.legendre.leggauss(16)
    acc = 0.0
    for m, w in zip(mu, wmu):  # the power depends only on the axis' polar angle
        axis = np.array([math.sqrt(1 - m * m), 0.0, m])
        acc += 0.5 * w * radiated_power(d, axis, [1, 0, 0, 0], n)
    assert acc == pytest.approx(1.0, rel=1e-12)


def test_pure_states_stay_pure_and_the_envelope_bounds():
    d = O.dipole_constants(EPS, 2.0, 0.3)
    for _ in range(300):
        X, n, n2, axis = rand_stokes(pure=True), rand_dir(), rand_dir(), rand_dir()
        Y = O.dipole_scatter(EPS, 2.0, 0.3, axis, X, n, n2)
        assert Y[0] ** 2 == pytest.approx(Y[1] ** 2 + Y[2] ** 2 + Y[3] ** 2, rel=1e-10)
        X = rand_stokes()
        Y = O.dipole_scatter(EPS, 2.0, 0.3, axis, X, n, n2)
        assert Y[0] <= d["env"] * X[0] * (1 + 1e-12)
        assert Y[0] ** 2 >= (Y[1] ** 2 + Y[2] ** 2 + Y[3] ** 2) * (1 - 1e-12)


def test_circular_polarization_needs_a_phase_lag():
    """Real eps in the small-particle limit (rho real: the radiative reaction adds a
    phase of order x^3) makes no V from linear polarization; an absorbing grain
    (complex rho) does."""
    vmax_real, vmax_abs = 0.0, 0.0
    for _ in range(100):
        X, n, n2, axis = rand_stokes(), rand_dir(), rand_dir(), rand_dir()
        X[3] = 0.0
        vmax_real = max(vmax_real, abs(O.dipole_scatter(2.25, 2.0, 1e-4, axis, X, n, n2)[3]) / X[0])
        vmax_abs = max(vmax_abs, abs(O.dipole_scatter(complex(3.0, 2.0), 2.0, 0.3, axis, X, n, n2)[3]) / X[0])
    assert vmax_real < 1e-10 and vmax_abs > 1e-3


# ---------------------------------------------------------------------------------
# extinction matrix, emission and sampling in a cell
# ---------------------------------------------------------------------------------
def one_cell(b, ka=0.4, ks=0.6, s=2.0, x=0.3, emissivity=None, n=(1, 1, 1)):
    shape = (n[2], n[1], n[0])
    bf = np.zeros(shape + (3,), dtype=np.float32)
    bf[...] = np.asarray(b, dtype=np.float32)
    return {"lo": (0.0, 0.0, 0.0), "hi": (1.0, 1.0, 1.0),
            "kappa_abs": np.full(shape, ka, dtype=np.float32), "kappa_sca": np.full(shape, ks, dtype=np.float32),
            "bfield": bf, "emissivity": None if emissivity is None else np.full(shape, emissivity, np.float32),
            "optics": W.dipole_optics(EPS, s, x)}


def cross_section(d, kind, axis, e):
    """Optical-theorem (ext) or radiated (sca) cross section of linear polarization e,
    relative to the orientation average, as a field along e sees the principal axes."""
    w = float(np.dot(axis, e)) ** 2
    c0, c1 = d["q_%s0" % kind], d["q_%s1" % kind]
    return (c0 * (1 - w) + c1 * w) / ((2 * c0 + c1) / 3)


def test_extinction_of_any_linear_polarization():
    """K applied to light linearly polarized along e at angle chi in the
    grain-meridian basis is removed at kappa_abs C_abs(e) + kappa_sca C_sca(e) (each
    relative to its orientation average): K11 + K12 cos 2chi, with no U coupling."""
    ka, ks = 0.4, 0.6
    for _ in range(30):
        b, n = rand_dir(), rand_dir()
        m = one_cell(b, ka, ks)
        f = O.frame(m, 0, n)
        d = O.dipole_constants(EPS, 2.0, 0.3)
        axis = unit(np.asarray(b, dtype=np.float32).astype(np.float64))
        a1, a2, a3 = f["alpha"]
        assert a3 == 0.0
        for chi in np.linspace(0, math.pi, 7):
            e = math.cos(chi) * f["gth"] + math.sin(chi) * f["gph"]
            want = ka * cross_section(d, "abs", axis, e) + ks * cross_section(d, "sca", axis, e)
            got = (a1 + a2 * math.cos(2 * chi)) * (ka + ks)
            assert got == pytest.approx(want, rel=2e-6)  # FP32 field direction
            want_s = ks * cross_section(d, "sca", axis, e)
            assert (f["sca"][0] + f["sca"][1] * math.cos(2 * chi)) * (ka + ks) == pytest.approx(want_s, rel=2e-6)
        ka32, ks32 = float(np.float32(ka)), float(np.float32(ks))  # the grid is FP32
        assert f["gsca"] * ks32 == pytest.approx(f["sca"][0] * (ka32 + ks32), rel=1e-12)


def test_mean_extinction_over_directions_is_kappa_ext():
    """The cell's opacities are orientation averages: the mean of alpha1 over
    directions is 1 and its scattering part averages to omega."""
    m = one_cell((0.3, -0.2, 0.9))
    mu, wmu = np.polynomial.legendre.leggauss(16)
    a_mean, s_mean = 0.0, 0.0
    for mm, w in zip(mu, wmu):
        for p in (np.arange(16) + 0.5) * 2 * math.pi / 16:
            st = math.sqrt(1 - mm * mm)
            f = O.frame(m, 0, [st * math.cos(p), st * math.sin(p), mm])
            a_mean += w / 2 / 16 * f["alpha"][0]
            s_mean += w / 2 / 16 * f["sca"][0]
    assert a_mean == pytest.approx(1.0, rel=1e-6)
    assert s_mean == pytest.approx(0.6, rel=1e-6)


def test_oblate_grains_polarize_transmitted_light_along_the_projected_field():
    """alpha2 < 0: the field along the projected axis (theta-hat') is extinguished
    less, so starlight gets polarized along the projected field."""
    m = one_cell((0, 0, 1))
    f = O.frame(m, 0, [1, 0, 0])
    assert f["alpha"][1] < 0 and f["sca"][1] < 0
    assert abs(np.dot(f["gth"], [0, 0, 1])) == pytest.approx(1.0)


def test_thermal_emission_follows_the_absorption_cross_section():
    """A thermal packet is born with I proportional to C_abs along n relative to its
    average, polarized with Q/I = K_abs,12 / K_abs,11 in the grain-meridian basis."""
    b = unit([0.5, 0.1, 0.8])
    m = one_cell(b, emissivity=1.0)
    d = O.dipole_constants(EPS, 2.0, 0.3)
    run = {"sources": [{"type": "thermal", "n_packets": 4000}], "seed": 3}
    rows = O.emit(m, run, range(4000))
    axis = unit(np.asarray(b, dtype=np.float32).astype(np.float64))
    # the thermal luminosity is 4 pi kappa_abs B V; the run gives the source luminosity
    # 1, so each packet carries 1/4000 times its direction's weight
    assert O.thermal_luminosity(m, run) == pytest.approx(4 * math.pi * np.float32(0.4), rel=1e-7)
    eps_p = 1.0 / 4000
    for r in rows[:200]:
        n, X = r[3:6], r[6:10]
        f = O.frame(m, 0, n)
        ct, cp = cross_section(d, "abs", axis, f["gth"]), cross_section(d, "abs", axis, f["gph"])
        th, ph = O.stokes_basis(n)
        Xg = O.change_basis(X, th, ph, f["gth"], f["gph"])
        assert Xg[0] == pytest.approx(eps_p * 0.5 * (ct + cp), rel=1e-9)
        assert Xg[1] / Xg[0] == pytest.approx((ct - cp) / (ct + cp), rel=1e-9, abs=1e-12)
        assert abs(Xg[2]) < 1e-12 * Xg[0] and Xg[3] == 0.0
    wsum = rows[:, 6].mean() / eps_p
    assert wsum == pytest.approx(1.0, abs=0.02)  # mean of C_abs over directions


def test_scattering_sampler_density_and_weight():
    """Accepted directions follow (Z X)_0 (chi-square on the cosine to the axis); the
    scattered Stokes vector is Z X renormalised to I + (s12/s11) Q_grain-meridian."""
    b = unit([0.2, 0.4, 0.9])
    m = one_cell(b)
    axis = unit(np.asarray(b, dtype=np.float32).astype(np.float64))
    X = np.array([1.0, 0.4, -0.3, 0.2])
    n = unit([1.0, 0.2, -0.3])
    f = O.frame(m, 0, n)
    th, ph = O.stokes_basis(n)
    Xg = O.change_basis(X, th, ph, f["gth"], f["gph"])
    Iw = X[0] + f["sca"][1] / f["sca"][0] * Xg[1]
    q = O.grain_quaternion(np.asarray(b, dtype=np.float32))
    run = {"sources": [{"type": "point", "n_packets": 1}], "cameras": []}
    nb = 10
    counts = np.zeros(nb)
    N = 6000
    for pid in range(N):
        t, n2, Y = O.scatter(m, run, pid, 1, 0, X, n, q)
        assert t > 0
        Z = O.dipole_scatter(EPS, 2.0, 0.3, axis, X, n, n2)
        assert np.allclose(Y, Z * Iw / Z[0], rtol=1e-10, atol=1e-14)
        counts[min(nb - 1, int((np.dot(n2, axis) + 1) / 2 * nb))] += 1
    # expected: int over the band of (Z X)_0, by quadrature in (cos to axis, azimuth)
    e1 = unit(np.cross(axis, [1.0, 0.0, 0.0]))
    e2 = np.cross(axis, e1)
    expect = np.zeros(nb)
    gm, gw = np.polynomial.legendre.leggauss(8)
    for k in range(nb):
        lo, hi = -1 + 2 * k / nb, -1 + 2 * (k + 1) / nb
        for m_, w_ in zip(gm, gw):
            c = 0.5 * (lo + hi) + 0.5 * (hi - lo) * m_
            sc = math.sqrt(1 - c * c)
            for p in (np.arange(32) + 0.5) * 2 * math.pi / 32:
                n2 = c * axis + sc * (math.cos(p) * e1 + math.sin(p) * e2)
                expect[k] += 0.5 * (hi - lo) * w_ * (2 * math.pi / 32) * O.dipole_scatter(EPS, 2.0, 0.3, axis, X, n,
                                                                                         n2)[0]
    expect *= N / expect.sum()
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 30.0  # 9 degrees of freedom: p ~ 4e-4


# ---------------------------------------------------------------------------------
# transport
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("b", [(1, 0, 0), (0, 0, 1), (0.6, 0, 0.8)])
def test_unscattered_fraction_follows_the_directional_scattering_rate(b):
    """A beam along +z through a slab of optical thickness kappa_sca L: the share of
    packets crossing without scattering is exp(-kappa_sca C_sca(n) L), with C_sca(n)
    the unpolarized scattering cross section along n relative to its average."""
    m = one_cell(b, ka=0.0, ks=1.5, n=(1, 1, 4))
    run = W.beam_run(20000, seed=11)
    run["n_trace"] = 20000
    out = O.transport(m, run)
    f = O.frame(m, 0, [0, 0, 1])
    p = math.exp(-1.5 * f["gsca"])
    frac = np.mean(out["trace"][:, 10] == 0)
    assert abs(frac - p) < 4 * math.sqrt(p * (1 - p) / 20000)


def test_pure_scatterer_conserves_energy_in_expectation():
    """kappa_abs = 0: the polarization-dependent weights change a packet's I but the
    mean escaped energy equals the emitted energy (unbiased general weight)."""
    m = W.spheroid_sphere(n=12, tau=2.0, albedo=1.0, b=(1.0, 0.0, 0.0),
                          optics=W.dipole_optics(EPS, 2.0, 0.3))
    N = 40000
    run = {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": N}],
           "cameras": [], "seed": 21, "roulette_threshold": 0.0, "n_trace": N, "n_threads": 8}
    out = O.transport(m, run)
    tr = out["trace"]
    assert np.all(tr[:, 12] == 1)  # all escaped
    e = tr[:, 0] * N  # escaped I per packet over the birth I
    assert tr[:, 10].mean() > 1.5  # most packets scatter, several times
    assert e.std() > 1e-3  # the weights do vary
    assert abs(e.mean() - 1.0) < 4 * e.std() / math.sqrt(N)
    assert np.all(tr[:, 0] ** 2 >= (tr[:, 1:4] ** 2).sum(axis=1) * (1 - 1e-12))


def test_absorbing_medium_balances_energy_in_expectation():
    """Absorbing and scattering spheroids: escaped + absorbed = emitted in expectation
    (over 16 independent seeds, 4 standard errors).  The absorbed tally is the
    integral of (K_abs X)_0; the decrease of I also holds the polarization-dependent
    part of the scattering rate, which the scattering weight returns."""
    m = W.spheroid_sphere(n=12, tau=3.0, albedo=0.5, b=(1.0, 0.0, 0.0), optics=W.dipole_optics(EPS, 2.0, 0.3))
    bal = []
    for seed in range(16):
        run = {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": 4000}],
               "cameras": [], "seed": 100 + seed, "roulette_threshold": 0.0, "n_threads": 8}
        st = O.transport(m, run)["stats"]
        bal.append((st["escaped_energy"] + st["absorbed_energy"] + st["cap_lost"]) / st["emitted_energy"] - 1.0)
    bal = np.array(bal)
    assert abs(bal.mean()) < 4 * bal.std(ddof=1) / math.sqrt(len(bal)) + 1e-12, (bal.mean(), bal.std())


def test_single_segment_tally_closed_form():
    """A beam along +z through one cell with (almost) no scattering: the step-1 tally
    is Z(Omega_c; z) applied to int_0^L exp(-(K - s11 kappa_ext) l) X0 dl, computed here
    with the matrix exponential and the dipole radiation of the induced dipole."""
    b = unit([1.0, 0.0, 0.6])
    m = one_cell(b, ka=2.0, ks=1e-9)
    cam = unit([0.3, 0.5, 0.8])
    run = W.beam_run(50, seed=2, cameras=[W.camera(cam, (4, 4), (1.0, 1.0))])
    out = O.transport(m, run)
    assert out["stats"]["scatterings"] == 0
    n = np.array([0.0, 0.0, 1.0])
    f = O.frame(m, 0, n)
    a1, a2, _ = f["alpha"]
    kext = float(np.float32(2.0)) + float(np.float32(1e-9))  # FP32 grid, FP64 sum
    # K - s11 kappa_ext 1 in the grain-meridian basis (only the diagonal loses s11)
    Kg = kext * np.array([[a1 - f["sca"][0], a2, 0, 0], [a2, a1 - f["sca"][0], 0, 0],
                          [0, 0, a1 - f["sca"][0], 0], [0, 0, 0, a1 - f["sca"][0]]])
    Wg = quad_vec(lambda l: expm(-Kg * l) @ np.array([1.0, 0, 0, 0]), 0.0, 1.0)
    th, ph = O.stokes_basis(n)
    Wl = O.change_basis(Wg, f["gth"], f["gph"], th, ph)
    axis = unit(np.asarray(b, dtype=np.float32).astype(np.float64))
    want = O.dipole_scatter(EPS, 2.0, 0.3, axis, Wl, n, cam)  # per unit birth I
    got = out["S"][0, 0] / out["stats"]["emitted_energy"]
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12 * abs(want[0]))


def quad_vec(fn, a, b, k=40):
    x, w = np.polynomial.legendre.leggauss(k)
    return sum(0.5 * (b - a) * wi * fn(0.5 * (a + b) + 0.5 * (b - a) * xi) for xi, wi in zip(x, w))


def test_thin_cell_emission_image():
    """Step 2 of an optically thin emitting cell: the pixel sees kappa_abs C_abs(e) B L
    for each linear polarization e (here only thermal emission, no scattering)."""
    b = unit([0.0, 0.0, 1.0])
    m = one_cell(b, ka=1e-4, ks=0.0, emissivity=1.0)
    cam = np.array([1.0, 0.0, 0.0])
    run = {"sources": [], "cameras": [W.camera(cam, (1, 1), (0.5, 0.5), center=(0.5, 0.5, 0.5))]}
    img = O.image(m, run, None, 0)[:, 0, 0]
    d = O.dipole_constants(EPS, 2.0, 0.3)
    th, ph = O.stokes_basis(cam)
    ct, cp = cross_section(d, "abs", b, th), cross_section(d, "abs", b, ph)
    tau = np.float32(1e-4)
    # optically thin: I = tau B (ct + cp)/2, Q = tau B (ct - cp)/2 in the camera's basis
    assert img[0] == pytest.approx(tau * 0.5 * (ct + cp), rel=1e-3)
    assert img[1] == pytest.approx(tau * 0.5 * (ct - cp), rel=1e-3)
    assert abs(img[2]) < 1e-12 and abs(img[3]) < 1e-12
