"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, on the same
seeded inputs.  Needs a GB300: run with ``-m gpu``.

Tolerances (stated per test): FP64 kernels agree with the oracle to rounding
(<= 1e-9 relative on traces); FP32 kernels to 1e-4 relative per packet trace for
>= 99.9 % of packets, 1e-3 of the total intensity on integrated image Stokes, and
closed forms to 1e-5 relative with an absolute floor in Q/I of 64 x 2^-24 (FP32,
one rounding per cell of a 64-cell slab) or 1e-15 (FP64).
"""
import math

import numpy as np
import pytest

from accuracy_report import integrated_error, record
from oracle import oracle as O
from paper_2512_01283_gb300 import build as B
from paper_2512_01283_gb300 import mcrt as M
from paper_2512_01283_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2024)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    B.build()
    M.lib()


def rand_dirs(k):
    v = RNG.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def f32(x):
    return float(np.float32(x))


def gpu_run(model, run, precision="fp32", n_trace=0, **kw):
    m = M.Model(model)
    trace = np.zeros((max(1, n_trace), 16))
    st = M.launch(m, run, precision=precision, trace=trace if n_trace else None, n_trace=n_trace, **kw)
    n_cam = len(run.get("cameras", []))
    S, A = m.tallies(n_cam)
    imgs = []
    for k, c in enumerate(run.get("cameras", [])):
        out = np.zeros((4, c["npix"][1], c["npix"][0]))
        m.image(k, out)
        imgs.append(out)
    m.close()
    return {"stats": st, "trace": trace[:n_trace], "S": S, "absorbed": A, "images": imgs}


def oracle_run(model, run, n_trace=0, images=True, n_threads=1):
    r = dict(run)
    r["n_trace"] = n_trace
    r["n_threads"] = n_threads
    out = O.transport(model, r)
    out["images"] = [O.image(model, r, out["S"], k) for k in range(len(run.get("cameras", [])))] if images else []
    return out


def trace_match_fraction(tg, to, rtol):
    """Fraction of packets whose final (I,Q,U,V) agree to rtol relative to I."""
    I = np.abs(to[:, 0:1]) + 1e-300
    err = np.max(np.abs(tg[:, 0:4] - to[:, 0:4]) / I, axis=1)
    same_fate = tg[:, 12] == to[:, 12]
    return float(np.mean((err < rtol) & same_fate))


# ---------------------------------------------------------------------------------
# building blocks against the oracle
# ---------------------------------------------------------------------------------
def test_philox_bitwise():
    ins = RNG.integers(0, 2 ** 32, size=(4096, 6), dtype=np.uint64).astype(np.float64)
    for prec in ("fp32", "fp64"):
        out = M.unit_eval(0, ins, prec)
        ref = np.array([O.philox(r[:4].astype(np.uint64), r[4:6].astype(np.uint64)) for r in ins], dtype=np.float64)
        assert np.array_equal(out, ref)


def test_grain_quaternion_rotation():
    b = rand_dirs(500) * RNG.uniform(0.1, 3, size=(500, 1))
    v = rand_dirs(500)
    ins = np.concatenate([b, v, np.zeros((500, 1))], axis=1)
    for prec, tol in (("fp32", 2e-6), ("fp64", 2e-7)):
        out = M.unit_eval(1, ins, prec)
        for r, o in zip(ins, out):
            q = O.grain_quaternion(r[:3].astype(np.float32))
            assert np.allclose(o[:4], q, atol=1e-7)
            assert np.allclose(o[4:7], O.to_grain(q, r[3:6]), atol=tol)


def test_eta_rotation_equals_projection():
    """Signed eta of eq. (rotation-angle) applied by eq. (stokes-rotation) equals the
    oracle's projection of the coherency matrix on the grain-meridian basis."""
    b = rand_dirs(500)
    n = rand_dirs(500)
    X = np.concatenate([np.ones((500, 1)), RNG.uniform(-0.5, 0.5, (500, 3))], axis=1)
    ins = np.concatenate([b, n, X], axis=1)
    for prec, tol in (("fp32", 3e-6), ("fp64", 3e-7)):
        out = M.unit_eval(2, ins, prec)
        for r, o in zip(ins, out):
            q = O.grain_quaternion(r[:3].astype(np.float32))
            th, ph = O.stokes_basis(r[3:6])
            gth, gph, tp = O.grain_meridian(q, r[3:6])
            ref = O.change_basis(r[6:10], th, ph, gth, gph)
            assert np.allclose(o[:4], ref, atol=tol)
            assert abs(o[4] - math.cos(tp)) < tol


def test_cell_solution_and_path_integral():
    k = 400
    a1 = RNG.uniform(0.3, 2.0, k)
    a2 = RNG.uniform(-0.9, 0.9, k) * a1
    a3 = RNG.uniform(-1.5, 1.5, k)
    X = np.concatenate([np.ones((k, 1)), RNG.uniform(-0.5, 0.5, (k, 3))], axis=1)
    S = RNG.uniform(-0.5, 1.0, (k, 4))
    dt = 10 ** RNG.uniform(-4, 1.5, k)
    ins = np.concatenate([X, a1[:, None], a2[:, None], a3[:, None], S, dt[:, None]], axis=1)
    for prec, rtol in (("fp32", 2e-5), ("fp64", 1e-10)):
        out = M.unit_eval(3, ins, prec)
        for r, o in zip(ins, out):
            ref = O.cell_solution(r[:4], r[4:7], r[7:11], r[11])
            scale = 1.0 + np.abs(ref).max() + np.abs(r[7:11]).max() / r[4]
            assert np.allclose(o, ref, atol=rtol * scale), (r, o, ref)
    ins2 = np.concatenate([X, (a1 * 0.7)[:, None], (a2 * 0.5)[:, None], a3[:, None], dt[:, None]], axis=1)
    for prec, rtol in (("fp32", 2e-5), ("fp64", 1e-11)):
        out = M.unit_eval(4, ins2, prec)
        for r, o in zip(ins2, out):
            ref = O.segment_integral(r[:4], r[4], r[5], r[6], r[7])
            assert np.allclose(o, ref, rtol=rtol, atol=rtol * r[7])


def test_scattering_matrix_transfer():
    k = 400
    n, n2 = rand_dirs(k), rand_dirs(k)
    n2[:5] = n[:5]          # forward, degenerate scattering plane
    n2[5:10] = -n[5:10]     # backward
    n[10:12] = [[0, 0, 1], [0, 0, -1]]  # poles
    X = np.concatenate([np.ones((k, 1)), RNG.uniform(-0.5, 0.5, (k, 3))], axis=1)
    P = np.array([O.rayleigh(float(np.dot(a, b))) for a, b in zip(n, n2)])
    # a circular term away from Theta = 0, pi only: a realizable matrix has P34 = 0
    # where the scattering plane is undefined
    P[10:, 4] = RNG.uniform(-0.02, 0.02, k - 10)
    ins = np.concatenate([X, n, n2, P], axis=1)
    for prec, tol in (("fp32", 3e-6), ("fp64", 1e-12)):
        out = M.unit_eval(5, ins, prec)
        for r, o in zip(ins, out):
            ref = O.mueller_apply(r[:4], r[4:7], r[7:10], r[10:16])
            assert np.allclose(o, ref, atol=tol), (r, o, ref)


# ---------------------------------------------------------------------------------
# dichroic slab (64^3, 1e6 packets, FP32): closed forms and oracle traces
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("tau", [0.1, 1.0, 10.0, 30.0])
def test_dichroic_slab_full_size(tau):
    t, p = f32(tau), -f32(-0.05)
    model = W.dichroic_slab(n=64, tau=tau)
    run = W.beam_run(1_000_000, seed=1)
    g = gpu_run(model, run, "fp32", n_trace=256)
    st = g["stats"]
    assert st["emitted"] == 1_000_000 and st["escaped"] == 1_000_000
    assert st["events"] == 1_000_000 * 65
    tr = g["trace"]
    I = tr[:, 0] / tr[:, 13]
    ref_I = math.exp(-t) * math.cosh(p * t)
    assert np.allclose(I, ref_I, rtol=1e-5, atol=0.0)
    assert np.allclose(tr[:, 1] / tr[:, 0], math.tanh(p * t), rtol=1e-5, atol=64 * 2.0 ** -24)
    assert np.all(np.abs(tr[:, 2:4]) <= 1e-6 * tr[:, :1])
    assert abs(st["escaped_energy"] - ref_I) < 1e-5 * ref_I
    assert abs(st["absorbed_energy"] + st["escaped_energy"] - 1.0) < 1e-5
    o = oracle_run(model, dict(run, pid_end=256), n_trace=256, images=False)
    assert trace_match_fraction(tr, o["trace"], 1e-5) == 1.0


# absolute floors in Q/I: FP32 = 64 cells x 2^-24 (one rounding of Q per cell),
# FP64 = the 1e-15 of the oracle pin
@pytest.mark.parametrize("prec,floor", [("fp32", 64 * 2.0 ** -24), ("fp64", 1e-15)])
@pytest.mark.parametrize("tau", [0.1, 1.0, 10.0, 30.0])
def test_ptau_emission_imaging(tau, prec, floor):
    """eq. (ptau) through the GPU step-2 kernel (emission source only)."""
    t, p = f32(tau), -f32(-0.05)
    model = W.dichroic_slab(n=64, tau=tau, emissivity=1.0)
    run = W.beam_run(1, cameras=[W.camera((0, 0, 1), (4, 4), (0.5, 0.5))])
    g = gpu_run(model, run, prec)
    P = math.exp(-t) * math.sinh(p * t) / (1 - math.exp(-t) * math.cosh(p * t))
    I, Q, U, V = g["images"][0][:, 1, 2]
    assert abs(I - (1 - math.exp(-t) * math.cosh(p * t))) < max(1e-5 * I, floor)
    assert abs(-Q / I - P) <= max(1e-5 * P, floor)
    assert abs(U) <= floor and abs(V) <= floor


# ---------------------------------------------------------------------------------
# Rayleigh sphere (32^3, 1e5 packets)
# ---------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def sphere_oracle():
    model = W.rayleigh_sphere()
    run = W.rayleigh_sphere_run(100_000, seed=0)
    return model, run, oracle_run(model, run, n_trace=100_000)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rayleigh_sphere_parity(sphere_oracle, prec):
    """Per-packet Stokes traces within 1e-4 relative for >= 99.9 % of packets;
    integrated I,Q,U,V of the image within 1e-3 of the total I; tallies."""
    model, run, o = sphere_oracle
    g = gpu_run(model, run, prec, n_trace=100_000)
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= 0.999, frac
    if prec == "fp64":
        assert frac >= 0.9999
    gi, oi = g["images"][0], o["images"][0]
    Itot = oi[0].sum()
    for e in range(4):
        assert abs(gi[e].sum() - oi[e].sum()) < 1e-3 * Itot, e
    for key in ("emitted", "escaped", "scatterings", "segments"):
        assert abs(g["stats"][key] - o["stats"][key]) <= 2e-4 * o["stats"][key] + 2, key
    dS = np.linalg.norm(g["S"] - o["S"]) / np.linalg.norm(o["S"])
    assert dS < (1e-9 if prec == "fp64" else 1e-3), dS
    assert abs(g["stats"]["escaped_energy"] - g["stats"]["emitted_energy"]) < 1e-6


def test_rayleigh_sphere_chi2_independent_seeds(sphere_oracle):
    """Images from independent seeds agree within Monte-Carlo error:
    chi^2/dof < 1.2 with per-pixel sigma from 32 packet batches of each run."""
    model, run, _ = sphere_oracle
    nb, per = 32, 100_000 // 32
    total = nb * per
    mdl = M.Model(model)
    gimgs = []
    for b in range(nb):
        r = dict(run, seed=7, pid_begin=b * per, pid_end=(b + 1) * per)
        r["sources"] = [dict(run["sources"][0], n_packets=total)]
        M.launch(mdl, r, precision="fp32")
        out = np.zeros((4, 64, 64))
        mdl.image(0, out)
        gimgs.append(out * nb)
    mdl.close()
    oimgs = []
    for b in range(nb):
        r = dict(run, seed=11, pid_begin=b * per, pid_end=(b + 1) * per)
        r["sources"] = [dict(run["sources"][0], n_packets=total)]
        o = O.transport(model, r)
        oimgs.append(O.image(model, r, o["S"], 0) * nb)
    G, Oo = np.array(gimgs), np.array(oimgs)
    for e in range(3):
        mg, mo = G[:, e].mean(0), Oo[:, e].mean(0)
        var = G[:, e].var(0, ddof=1) / nb + Oo[:, e].var(0, ddof=1) / nb
        mask = var > 0
        chi2 = np.sum((mg - mo)[mask] ** 2 / var[mask]) / mask.sum()
        assert chi2 < 1.2, (e, chi2)


# ---------------------------------------------------------------------------------
# flared disk with grain tables, star + thermal emission
# ---------------------------------------------------------------------------------
def test_small_disk_parity():
    """24^3 disk, star + thermal, 4 cameras, 1e5 packets: traces (>= 99.9 % FP64, 99 %
    FP32: the optically thick disk flips more FP32 decisions), integrated image Stokes
    within 1e-3 of the total I, energy balance."""
    model = W.disk(n=24)
    n = 100_000
    run = W.disk_run(n_packets=n, n_cam=4, npix=32)
    o = oracle_run(model, run, n_trace=n, n_threads=16)
    for prec in ("fp64", "fp32"):
        g = gpu_run(model, run, prec, n_trace=n)
        frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
        assert frac >= (0.999 if prec == "fp64" else 0.99), (prec, frac)
        err = integrated_error(g["images"], o["images"])
        record("flared disk 24^3, star + thermal, 4 cameras, 1e5 packets, " + prec, "max integrated |dX|/I", err,
               1e-3)
        record("flared disk 24^3, star + thermal, 4 cameras, 1e5 packets, " + prec, "trace match fraction at 1e-4",
               frac, 0.999 if prec == "fp64" else 0.99, "min")
        assert err < (1e-9 if prec == "fp64" else 1e-3), (prec, err)
        st = g["stats"]
        bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
        assert abs(bal - st["emitted_energy"]) < (1e-9 if prec == "fp64" else 1e-5) * st["emitted_energy"]
        assert abs(st["emitted_energy"] - o["stats"]["emitted_energy"]) < 1e-6 * o["stats"]["emitted_energy"]
        if prec == "fp64":
            # the warp's rejection trials run on all its lanes, the first accepted one in
            # trial order wins: scatterings and trials total as the oracle's sequential rule
            for k in ("scatterings", "trials"):
                assert abs(st[k] - o["stats"][k]) <= 1e-5 * o["stats"][k], (k, st[k], o["stats"][k])


def test_full_size_disk_sampled_parity():
    """192^3 disk, 8 cameras of 256^2, in the benchmark's launch configuration:
    the first 2000 packet ids of a 2e6-packet launch against the oracle."""
    model = W.disk(n=192)
    run = W.disk_run(n_packets=2_000_000)
    n_s = 2000
    g = gpu_run(model, run, "fp32", n_trace=n_s)
    o = O.transport(model, dict(run, pid_end=n_s, n_trace=n_s, n_threads=8))
    # both halves of the id range: star ids [0, 1e6) only here; thermal ids sampled below
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= 0.99, frac
    r2 = dict(run, pid_begin=1_000_000, pid_end=1_000_000 + n_s)
    mdl = M.Model(model)
    tr = np.zeros((1_000_000 + n_s, 16))
    M.launch(mdl, r2, precision="fp32", trace=tr, n_trace=1_000_000 + n_s)
    mdl.close()
    o2 = O.transport(model, dict(r2, n_trace=1_000_000 + n_s, n_threads=8))
    frac2 = trace_match_fraction(tr[1_000_000:], o2["trace"][1_000_000:], 1e-4)
    assert frac2 >= 0.99, frac2
    st = g["stats"]
    bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
    assert abs(bal - st["emitted_energy"]) < 1e-5 * st["emitted_energy"]


# ---------------------------------------------------------------------------------
# edge cases and error paths
# ---------------------------------------------------------------------------------
def test_empty_and_degenerate_inputs():
    # no dust: every packet escapes unchanged after crossing the grid
    model = W.rayleigh_sphere(n=8)
    model["kappa_sca"][:] = 0
    run = W.rayleigh_sphere_run(5000, npix=8)
    g = gpu_run(model, run, "fp32", n_trace=100)
    assert g["stats"]["escaped"] == 5000 and g["stats"]["scatterings"] == 0
    assert np.all(g["images"][0] == 0.0)
    # one-cell grid
    model = W.dichroic_slab(n=1, tau=2.0)
    g = gpu_run(model, W.beam_run(64), "fp64", n_trace=4)
    t, p = 2.0, -f32(-0.05)
    assert np.allclose(g["trace"][:, 0] / g["trace"][:, 13], math.exp(-t) * math.cosh(p * t), rtol=1e-12)
    # zero packets
    m = M.Model(W.rayleigh_sphere(n=4))
    st = M.launch(m, W.rayleigh_sphere_run(0, npix=4))
    assert st["emitted"] == 0
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eight_sources_with_empty_and_single_packet_sources(prec):
    """The most sources a launch takes (8): point, beam and thermal sources mixed, two
    with no packets and one with a single packet, against the oracle (packet ids run
    through the sources in order, each source's energy split over its own packets); a
    ninth source is refused."""
    model = W.dichroic_slab(n=8, tau=1.5, p=0.05, b_angle_deg=35.0, albedo=0.6, emissivity=1.0)
    model["optics"] = W.table_optics(n_bins=2)
    sources = [{"type": "point", "pos": (0.3, 0.6, 0.5), "luminosity": 2.0, "n_packets": 0},
               {"type": "beam", "beam_dir": 1, "luminosity": 1.0, "n_packets": 1},
               {"type": "point", "pos": (0.5, 0.5, 0.5), "luminosity": 0.7, "n_packets": 33_700},
               {"type": "thermal", "luminosity": 0.0, "n_packets": 0},
               {"type": "beam", "beam_dir": -1, "luminosity": 0.4, "n_packets": 9_500},
               {"type": "point", "pos": (0.81, 0.22, 0.13), "luminosity": 1.3, "n_packets": 100_000},
               {"type": "thermal", "luminosity": 0.0, "n_packets": 64_000},
               {"type": "point", "pos": (0.05, 0.95, 0.5), "luminosity": 0.1, "n_packets": 3}]
    n = sum(s["n_packets"] for s in sources)
    run = {"sources": sources, "cameras": [W.camera((0.3, 0.2, 0.93), (9, 9), (1.2, 1.2), center=(0.5, 0.5, 0.5))],
           "seed": 21, "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    o = oracle_run(model, run, n_trace=n, n_threads=16)
    g = gpu_run(model, run, prec, n_trace=n)
    # every packet is born at the source its id falls in
    assert np.array_equal(g["trace"][:, 14], o["trace"][:, 14])
    assert np.array_equal(np.bincount(g["trace"][:, 14].astype(int), minlength=8),
                          [s["n_packets"] for s in sources])
    assert trace_match_fraction(g["trace"], o["trace"], 1e-4) >= (0.999 if prec == "fp64" else 0.99)
    tol = 1e-7 if prec == "fp64" else 2e-3
    assert np.linalg.norm(g["S"] - o["S"]) < tol * np.linalg.norm(o["S"])
    assert g["stats"]["emitted_energy"] == pytest.approx(o["stats"]["emitted_energy"], rel=1e-6)
    err = integrated_error(g["images"], o["images"])
    record("eight sources, 8^3 slab, 2 bins, 2.07e5 packets, " + prec, "max integrated |dX|/I", err, 1e-3)
    # FP64: the cell record keeps the grain quaternion of the 35-degree field in FP32
    assert err < (1e-7 if prec == "fp64" else 1e-3), err
    m = M.Model(model)
    with pytest.raises(M.McrtError) as err:
        M.launch(m, dict(run, sources=sources + [sources[2]]))
    assert err.value.status == M.MCRT_E_INVAL
    m.close()


def _step2_model(kind):
    if kind == "disk":
        return W.disk(n=16), {}
    if kind == "refined disk":
        return W.disk_refined(n=16, factor=2), {}
    # aligned dipole spheroids with a central star (imaging adds their own emission); 10
    # cells, so that no pixel ray runs along a cell face, where the two precisions may
    # image different neighbours
    m = W.spheroid_sphere(n=10, tau=1.5, albedo=0.6, b=(0.6, 0.0, 0.8))
    m["emissivity"] = np.full(m["kappa_abs"].shape, 0.3, dtype=np.float32)
    return m, {"sources": [{"type": "point", "pos": (0.05, -0.02, 0.01), "luminosity": 1.0, "n_packets": 6000}]}


@pytest.mark.parametrize("kind", ["disk", "refined disk", "spheroids"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step2_images_pixelwise_on_the_oracle_tallies(kind, prec):
    """Step 2 alone: the oracle's step-1 tallies set into the GPU model (mcrt_set_tallies)
    and imaged by both sides, pixel by pixel, on a plain grid with tables, a composite
    grid and aligned spheroids.  Cameras with non-square pixel counts and fields of
    view, one looking down -z (the pole of the Stokes basis), one along +y, one oblique
    with an off-centre image centre, and a single pixel."""
    model, extra = _step2_model(kind)
    cams = [W.camera((0, 0, -1), (7, 5), (1.7, 1.1)),
            W.camera((0, 1, 0), (6, 9), (2.0, 1.3)),
            W.camera((0.4, -0.3, 0.6), (11, 4), (1.4, 0.6), center=(0.1, -0.2, 0.05)),
            W.camera((0.2, 0.7, -0.3), (1, 1), (0.3, 0.3))]
    run = dict(W.disk_run(n_packets=6000), cameras=cams, **extra)
    r = dict(run, n_threads=4)
    o = O.transport(model, r)
    m = M.Model(model)
    M.launch(m, run, precision=prec)
    m.set_tallies(np.ascontiguousarray(o["S"]), np.ascontiguousarray(o["absorbed"]))
    # FP64: the cell record keeps the grain quaternion in FP32, which the oracle does not
    tol = 1e-7 if prec == "fp64" else 2e-5
    for k, c in enumerate(cams):
        ref = O.image(model, r, o["S"], k)
        out = np.zeros((4, c["npix"][1], c["npix"][0]))
        m.image(k, out)
        assert out.shape == ref.shape
        scale = np.abs(ref[0]).max()
        assert scale > 0
        assert np.abs(out - ref).max() < tol * scale, (k, np.abs(out - ref).max() / scale)
    m.close()


def test_ragged_packet_counts_and_resume():
    """Odd packet counts (not multiples of a warp) and a launch split into two id
    ranges with accumulate give the same tallies as one launch."""
    model = W.rayleigh_sphere(n=16)
    run = W.rayleigh_sphere_run(12_345, npix=16)
    one = gpu_run(model, run, "fp64")
    m = M.Model(model)
    M.launch(m, dict(run, pid_end=5_001), precision="fp64")
    M.launch(m, dict(run, pid_begin=5_001), precision="fp64", accumulate=1)
    S, A = m.tallies(1)
    m.close()
    assert np.allclose(S, one["S"], rtol=1e-9, atol=1e-15)


def test_invalid_arguments_are_rejected():
    m = M.Model(W.rayleigh_sphere(n=4))
    bad = W.rayleigh_sphere_run(10, npix=4)
    bad["sources"][0]["pos"] = (5.0, 0.0, 0.0)
    with pytest.raises(M.McrtError) as e:
        M.launch(m, bad)
    assert e.value.status == M.MCRT_E_INVAL
    with pytest.raises(M.McrtError) as e:
        m.image(3, np.zeros((4, 4, 4)))
    assert e.value.status in (M.MCRT_E_STATE, M.MCRT_E_INVAL)
    m.close()


def test_event_cap_and_time_budget_report_status():
    """The per-packet event cap and the launch time budget end the kernel with a
    status the host reads; the context stays usable afterwards."""
    model = W.rayleigh_sphere(n=32, tau=20.0)
    m = M.Model(model)
    run = dict(W.rayleigh_sphere_run(2000, npix=8), max_events=5)
    st = M.launch(m, run, raise_on_cap=False)
    assert st["status"] == M.MCRT_E_EVENT_CAP and st["cap_hits"] > 0
    st = M.launch(m, W.rayleigh_sphere_run(5_000_000, npix=8), raise_on_cap=False, time_budget_s=1e-6)
    assert st["status"] == M.MCRT_E_TIMEOUT and st["emitted"] < 5_000_000
    st = M.launch(m, W.rayleigh_sphere_run(1000, npix=8))
    assert st["status"] == M.MCRT_OK and st["emitted"] == 1000
    m.close()


def test_table_rounds_equal_the_in_place_tally():
    """FP32 table launches run in rounds (transport, then a tally kernel over the queued
    segments) by default; the in-place tally (MCRT_FLAG_INLINE_TALLY) and the rounds
    with each tally beside the next transport (tally_blocks_per_sm > 0) give the same
    packets and the same tallies up to FP32 rounding of the per-segment terms."""
    model = W.disk(n=24)
    run = W.disk_run(n_packets=20_000, n_cam=4, npix=32)
    ref = gpu_run(model, run, "fp32", n_trace=20_000, inline_tally=True)
    for kw in ({}, {"tally_blocks_per_sm": 2}):
        g = gpu_run(model, run, "fp32", n_trace=20_000, **kw)
        assert g["stats"]["events"] == ref["stats"]["events"]
        assert g["stats"]["wave_iterations"] >= 1
        assert trace_match_fraction(g["trace"], ref["trace"], 1e-6) >= 0.999
        assert np.linalg.norm(g["S"] - ref["S"]) < 1e-6 * np.linalg.norm(ref["S"])
        # absorbed: the in-place kernel pre-sums same-cell lanes in FP32 before widening, the
        # round kernels widen each lane's term
        assert np.linalg.norm(g["absorbed"] - ref["absorbed"]) < 1e-7 * np.linalg.norm(ref["absorbed"])
        for k in range(4):
            assert np.linalg.norm(g["images"][k] - ref["images"][k]) < 1e-6 * np.linalg.norm(ref["images"][k])


@pytest.mark.parametrize("n_cam", [1, 3, 16])
def test_table_rounds_camera_counts(n_cam):
    """The tally kernel pads each record's cameras to 1, 2, 4, 8 or 16 rows: odd and
    extreme camera counts give the in-place tally's result."""
    model = W.disk(n=20)
    run = dict(W.disk_run(n_packets=6_000, n_cam=8, npix=16))
    run["cameras"] = W.inclination_cameras(n_cam=n_cam, npix=16)
    ref = gpu_run(model, run, "fp32", inline_tally=True)
    g = gpu_run(model, run, "fp32")
    assert g["stats"]["events"] == ref["stats"]["events"]
    assert g["S"].shape == ref["S"].shape == (20 ** 3, n_cam, 4)
    assert np.linalg.norm(g["S"] - ref["S"]) < 1e-6 * np.linalg.norm(ref["S"])


def test_table_rounds_resume_ranges_and_ragged_counts():
    """Rounds with packet-id sub-ranges and accumulate (several launches adding to the
    same tallies), and odd packet counts, equal one launch over all ids."""
    model = W.disk(n=20)
    run = W.disk_run(n_packets=12_345, n_cam=2, npix=16)
    one = gpu_run(model, run, "fp32")
    m = M.Model(model)
    M.launch(m, dict(run, pid_end=5_001), precision="fp32")
    M.launch(m, dict(run, pid_begin=5_001, pid_end=9_999), precision="fp32", accumulate=1)
    M.launch(m, dict(run, pid_begin=9_999), precision="fp32", accumulate=1)
    S, A = m.tallies(2)
    m.close()
    # FP32 launches pre-sum the absorbed energy of same-cell lanes of a warp in FP32, and
    # the warps differ between the split and the single launch
    assert np.linalg.norm(S - one["S"]) < 1e-6 * np.linalg.norm(one["S"])
    assert np.linalg.norm(A - one["absorbed"]) < 1e-6 * np.linalg.norm(one["absorbed"])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_slab_oblique_escape_on_gpu(prec):
    """Absorbing slab with periodic x and y: every packet leaves through z = 0 or 1 with
    I = (L/N) exp(-tau 0.5 / |n_z|) (the oracle's closed-form pin), on both paths."""
    tau, N = 1.5, 20_000
    model = W.plane_parallel_slab(nxy=4, nz=8, tau=tau, albedo=0.0, periodic=3)
    run = dict(W.center_source_run(N), max_events=10_000_000)
    g = gpu_run(model, run, prec, n_trace=N)
    tr = g["trace"]
    esc = tr[:, 12] == 1
    assert esc.mean() > 0.999
    zf = tr[esc, 6]
    assert np.all(np.isclose(zf, 0.0, atol=1e-5) | np.isclose(zf, 1.0, atol=1e-5))
    expect = (1.0 / N) * np.exp(-tau * 0.5 / np.abs(tr[esc, 9]))
    rtol = 1e-10 if prec == "fp64" else 2e-4
    ok = np.isclose(tr[esc, 0], expect, rtol=rtol, atol=1e-30)
    assert ok.mean() > (0.9999 if prec == "fp64" else 0.995)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_periodic_scattering_slab_parity(prec):
    """Scattering, dichroic slab with periodic x and y (tables off, dipole grains):
    packet traces against the oracle, energy conservation."""
    model = W.plane_parallel_slab(nxy=4, nz=12, tau=3.0, albedo=0.8, periodic=3, b_angle_deg=30.0, p=0.05)
    run = dict(W.center_source_run(10_000, cameras=[W.camera((0.3, 0.2, 1.0), (8, 8), (1.0, 1.0))]))
    o = oracle_run(model, run, n_trace=10_000, images=False, n_threads=8)
    g = gpu_run(model, run, prec, n_trace=10_000)
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= (0.999 if prec == "fp64" else 0.99), frac
    st = g["stats"]
    bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
    assert abs(bal - st["emitted_energy"]) < 1e-6 * st["emitted_energy"]
    assert np.linalg.norm(g["S"] - o["S"]) < 2e-3 * np.linalg.norm(o["S"])


def test_rank_shares_and_the_tally_exchange():
    """Two ranks' shares of the packet ids run on two models (as two GPUs would), the
    tallies summed through CUDA tensors with get/set_tallies: tallies and images equal a
    single launch over all ids, up to the order of the FP64 additions."""
    import torch

    from paper_2512_01283_gb300 import multigpu as MG

    model = W.disk(n=24)
    run = W.disk_run(n_packets=20_000, n_cam=2, npix=16)
    ref = gpu_run(model, run, "fp32")
    mods, S_sum, A_sum = [], None, None
    for r in range(2):
        m = M.Model(model)
        MG.rank_launch(lambda rr, acc: M.launch(m, rr, precision="fp32", accumulate=acc), run, r, 2)
        S = torch.empty((m.ncell, 2, 4), dtype=torch.float64, device="cuda")
        A = torch.empty((m.ncell,), dtype=torch.float64, device="cuda")
        m.tallies_into(S, A)
        S_sum = S if S_sum is None else S_sum + S
        A_sum = A if A_sum is None else A_sum + A
        mods.append(m)
    m0 = mods[0]
    m0.set_tallies(S_sum, A_sum)
    S0, A0 = m0.tallies(2)
    assert np.allclose(S0, ref["S"], rtol=1e-9, atol=1e-12 * np.abs(ref["S"]).max())
    # absorbed: same-cell lanes of a warp are pre-summed in FP32 before the FP64 atomic, and
    # which packets share a warp differs between one launch and two shares
    assert np.allclose(A0, ref["absorbed"], rtol=1e-6, atol=1e-9 * np.abs(ref["absorbed"]).max())
    for k in range(2):
        out = np.zeros((4, 16, 16))
        m0.image(k, out)
        assert np.allclose(out, ref["images"][k], rtol=1e-9, atol=1e-12 * np.abs(ref["images"][k]).max())
    for m in mods:
        m.close()
    # the same sum in place on the library's own buffers (mcrt_tally_buffers), as the
    # NCCL all-reduce of a sharded run does it
    mods = []
    for r in range(2):
        m = M.Model(model)
        MG.rank_launch(lambda rr, acc: M.launch(m, rr, precision="fp32", accumulate=acc), run, r, 2)
        mods.append(m)
    (S0v, A0v), (S1v, A1v) = mods[0].tally_tensors(2), mods[1].tally_tensors(2)
    assert S0v.shape == (mods[0].ncell, 2, 4) and A0v.shape == (mods[0].ncell,)
    S0v.add_(S1v)
    A0v.add_(A1v)
    torch.cuda.synchronize()
    S0, A0 = mods[0].tallies(2)
    assert np.allclose(S0, ref["S"], rtol=1e-9, atol=1e-12 * np.abs(ref["S"]).max())
    assert np.allclose(A0, ref["absorbed"], rtol=1e-6, atol=1e-9 * np.abs(ref["absorbed"]).max())
    for k in range(2):
        out = np.zeros((4, 16, 16))
        mods[0].image(k, out)
        assert np.allclose(out, ref["images"][k], rtol=1e-9, atol=1e-12 * np.abs(ref["images"][k]).max())
    for m in mods:
        m.close()


def test_reduction_microbench_runs_and_checks_arguments():
    """mcrt_microbench: both reduction forms run on a small buffer; bad arguments are refused."""
    for kind in (0, 1):
        assert M.microbench(kind, 1 << 20, 1 << 16) > 0.0
    for bad in ((2, 1 << 20, 10), (0, 64, 10)):
        with pytest.raises(M.McrtError) as e:
            M.microbench(*bad)
        assert e.value.status == M.MCRT_E_INVAL
