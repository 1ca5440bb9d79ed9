"""Parity of the aligned-spheroid dipole optics on the CUDA path (through the C ABI)
with the FP64 oracle on the same seeded inputs.  Needs a GB300: run with ``-m gpu``.

Tolerances: device constants to 1e-12 relative (both FP64); unit kernels to 1e-12 of
the envelope (FP64) or 2e-6 (FP32); transport traces within 1e-4 relative for >= 99.9 %
(FP64) or 99 % (FP32) of packets; tallies and integrated image Stokes to 1e-7 (FP64:
the cell record keeps the grain quaternion in FP32, so the grain axis carries a
2^-24 rounding that the oracle, which builds it in FP64 from the same FP32 field, does
not) or 2e-3 of the total I (FP32).
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
RNG = np.random.default_rng(77)
EPS = complex(2.30, 0.0228) ** 2
FP64_AXIS_TOL = 1e-7  # FP64 runs: the FP32 grain quaternion of the cell record


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    B.build()
    M.lib()


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def rand_dirs(k):
    v = RNG.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def gpu_run(model, run, precision, n_trace=0, **kw):
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


def oracle_run(model, run, n_trace=0):
    r = dict(run, n_trace=n_trace, n_threads=8)
    out = O.transport(model, r)
    out["images"] = [O.image(model, r, out["S"], k) for k in range(len(run.get("cameras", [])))]
    return out


def trace_match_fraction(tg, to, rtol):
    I = np.abs(to[:, 0:1]) + 1e-300
    err = np.max(np.abs(tg[:, 0:4] - to[:, 0:4]) / I, axis=1)
    return float(np.mean((err < rtol) & (tg[:, 12] == to[:, 12])))


GRAINS = [(EPS, 2.0, 0.3), (EPS, 0.5, 0.1), (EPS, 1.03, 0.5), (EPS, 1.22, 0.2), (2.25, 1.0, 1e-3),
          (complex(3.0, 2.0), 4.0, 0.05), (complex(1.5, 0.01), 0.95, 1.0)]


@pytest.mark.parametrize("eps,s,x", GRAINS)
def test_device_constants_match_the_oracle(eps, s, x):
    g, o = M.dipole_constants(eps, s, x), O.dipole_constants(eps, s, x)
    for k in M.DIPOLE_KEYS:
        assert g[k] == pytest.approx(o[k], rel=1e-12, abs=1e-15 * max(1.0, abs(o[k]))), k


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_jones_scattering_unit(prec, tol):
    d = O.dipole_constants(EPS, 2.0, 0.3)
    n, n2, ax = rand_dirs(2000), rand_dirs(2000), rand_dirs(2000)
    X = np.zeros((2000, 4))
    X[:, 0] = 1.0
    X[:, 1:] = rand_dirs(2000) * RNG.uniform(0, 1, size=(2000, 1))
    # poles of the Stokes basis and incidence along the axis
    n[0], n[1], ax[2] = (0, 0, 1), (0, 0, -1), n[2]
    ins = np.hstack([X, n, n2, ax, np.tile([d["rho_re"], d["rho_im"], d["zn"]], (2000, 1))])
    got = M.unit_eval(6, ins, prec)
    for i in range(2000):
        want = O.dipole_scatter(EPS, 2.0, 0.3, ax[i], X[i], n[i], n2[i])
        assert np.all(np.abs(got[i] - want) <= tol * d["env"]), (i, got[i], want)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_extinction_unit_matches_the_oracle_frame(prec, tol):
    d = O.dipole_constants(EPS, 2.0, 0.3)
    ma, ms = (2 * d["q_abs0"] + d["q_abs1"]) / 3, (2 * d["q_sca0"] + d["q_sca1"]) / 3
    ca, cs = (d["q_abs0"] / ma, d["q_abs1"] / ma), (d["q_sca0"] / ms, d["q_sca1"] / ms)
    rows, want = [], []
    for _ in range(200):
        b, n = rand_dirs(1)[0], rand_dirs(1)[0]
        ka, ks = RNG.uniform(0, 2), RNG.uniform(0, 2)
        shape = (1, 1, 1)
        m = {"lo": (0, 0, 0), "hi": (1, 1, 1), "kappa_abs": np.full(shape, ka, np.float32),
             "kappa_sca": np.full(shape, ks, np.float32), "bfield": np.asarray(b, np.float32).reshape(1, 1, 1, 3),
             "emissivity": None, "optics": W.dipole_optics(EPS, 2.0, 0.3)}
        f = O.frame(m, 0, n)
        ka, ks = float(np.float32(ka)), float(np.float32(ks))
        rows.append([ca[0], ca[1], cs[0], cs[1], ka / (ka + ks), ks / (ka + ks), math.cos(f["thetap"]), 0.0])
        want.append([f["alpha"][0], f["alpha"][1], f["sca"][0], f["sca"][1]])
    got = M.unit_eval(7, np.array(rows), prec)
    assert np.max(np.abs(got - np.array(want))) < tol * 4


def spheroid_case(n_packets=20_000):
    model = W.spheroid_sphere(n=16, tau=1.0, albedo=0.6, b=(0.6, 0.0, 0.8))
    run = {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": n_packets}],
           "cameras": [W.camera((1, 0, 0), (16, 16), (2.0, 2.0)), W.camera(unit((0.3, 0.4, 0.85)), (16, 16), (2.0, 2.0))],
           "seed": 5, "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    return model, run


@pytest.fixture(scope="module")
def sphere_oracle():
    model, run = spheroid_case()
    return model, run, oracle_run(model, run, n_trace=20_000)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spheroid_sphere_parity(sphere_oracle, prec):
    model, run, o = sphere_oracle
    g = gpu_run(model, run, prec, n_trace=20_000)
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= (0.999 if prec == "fp64" else 0.99), frac
    dS = np.linalg.norm(g["S"] - o["S"]) / np.linalg.norm(o["S"])
    assert dS < (FP64_AXIS_TOL if prec == "fp64" else 2e-3), dS
    # absorbed tally: the integral of (K_abs X)_0 on both sides
    dA = np.linalg.norm(g["absorbed"] - o["absorbed"]) / np.linalg.norm(o["absorbed"])
    assert dA < (FP64_AXIS_TOL if prec == "fp64" else 2e-3), dA
    err = integrated_error(g["images"], o["images"])
    record("aligned spheroid sphere 16^3, 2e4 packets, " + prec, "max integrated |dX|/I", err, 1e-3)
    assert err < (FP64_AXIS_TOL if prec == "fp64" else 1e-3), err
    for key in ("emitted", "escaped", "scatterings", "segments"):
        assert abs(g["stats"][key] - o["stats"][key]) <= 2e-3 * o["stats"][key] + 2, key
    st = g["stats"]
    assert st["scatterings"] > 5000 and st["trials"] > st["scatterings"]
    assert st["absorbed_energy"] == pytest.approx(o["stats"]["absorbed_energy"], rel=1e-6 if prec == "fp64" else 2e-3)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_AXIS_TOL), ("fp32", 2e-5)])
def test_single_segment_tally_on_gpu(prec, tol):
    """Deterministic case: a beam through one absorbing cell with (almost) no
    scattering; every packet adds the same Zhat-weighted path integral."""
    b = unit([1.0, 0.0, 0.6])
    shape = (1, 1, 1)
    model = {"lo": (0.0, 0.0, 0.0), "hi": (1.0, 1.0, 1.0), "kappa_abs": np.full(shape, 2.0, np.float32),
             "kappa_sca": np.full(shape, 1e-9, np.float32), "bfield": np.asarray(b, np.float32).reshape(1, 1, 1, 3),
             "emissivity": None, "optics": W.dipole_optics(EPS, 2.0, 0.3)}
    run = W.beam_run(4096, seed=2, cameras=[W.camera(unit([0.3, 0.5, 0.8]), (4, 4), (1.0, 1.0)),
                                            W.camera((0, 0, 1), (4, 4), (1.0, 1.0))])
    o = O.transport(model, run)
    g = gpu_run(model, run, prec)
    assert g["stats"]["scatterings"] == 0 and o["stats"]["scatterings"] == 0
    assert np.allclose(g["S"], o["S"], rtol=tol, atol=tol * np.abs(o["S"]).max())
    assert np.allclose(g["absorbed"], o["absorbed"], rtol=tol)


def atmosphere_case(n_packets=20_000):
    model = W.spheroid_atmosphere(nxy=4, nz=16, tau=1.0, albedo=0.5)
    run = {"sources": [{"type": "thermal", "luminosity": 0.0, "n_packets": n_packets}],
           "cameras": W.atmosphere_cameras(n_az=4, npix=4), "seed": 8, "roulette_threshold": 1e-4,
           "roulette_survival": 0.1}
    return model, run


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_thermal_spheroid_atmosphere_parity(prec):
    """Periodic plane-parallel slab of aligned s = 1.03 spheroids with thermal
    emission: traces, tallies and images (emission and scattering) against the
    oracle."""
    model, run = atmosphere_case()
    o = oracle_run(model, run, n_trace=20_000)
    g = gpu_run(model, run, prec, n_trace=20_000)
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= (0.999 if prec == "fp64" else 0.99), frac
    dS = np.linalg.norm(g["S"] - o["S"]) / np.linalg.norm(o["S"])
    assert dS < (FP64_AXIS_TOL if prec == "fp64" else 2e-3), dS
    assert g["stats"]["emitted_energy"] == pytest.approx(o["stats"]["emitted_energy"], rel=1e-6)
    err = integrated_error(g["images"], o["images"])
    record("spheroid atmosphere 4x4x16, thermal, 2e4 packets, " + prec, "max integrated |dX|/I", err, 1e-3)
    assert err < (FP64_AXIS_TOL if prec == "fp64" else 1e-3), err
    for k in range(len(run["cameras"])):
        gi, oi = g["images"][k], o["images"][k]
        Itot = oi[0].sum()
        # thermal emission of grains aligned along x is polarized: Q or U is non-zero
        assert np.abs(oi[1:3]).sum() > 1e-3 * Itot


def test_invalid_dipole_arguments_and_unsupported_paths():
    model, run = spheroid_case(100)
    m = M.Model(model)
    for bad in [dict(eps=complex(2.0, -0.1)), dict(aspect=0.0), dict(eps=1.0), dict(x=-1.0),
                dict(aspect=float("nan"))]:
        opt = dict(W.dipole_optics(EPS, 2.0, 0.3), **bad)
        with pytest.raises(M.McrtError) as e:
            m.set_optics(opt)
        assert e.value.status == M.MCRT_E_INVAL
    m.set_optics(W.dipole_optics(EPS, 2.0, 0.3))
    # the surrogate learns tables: no surrogate launch on dipole optics
    with pytest.raises(M.McrtError) as e:
        M.launch(m, run, precision="fp32", optics="surrogate")
    assert e.value.status == M.MCRT_E_STATE
    m2 = M.Model(model)
    with pytest.raises(M.McrtError) as e:
        M.Batch([m, m2], run)
    assert e.value.status == M.MCRT_E_INVAL
    m.close()
    m2.close()
    with pytest.raises(M.McrtError):
        M.dipole_constants(complex(2.0, -1.0), 1.0, 0.1)


@pytest.mark.parametrize("grain", [(EPS, 0.5, 0.2), (EPS, 1.0, 0.3), (complex(3.0, 2.0), 4.0, 0.05)],
                         ids=["prolate", "sphere", "absorbing-flat"])
def test_spheroid_shapes_parity_fp32(grain):
    """Prolate, spherical and strongly absorbing flat grains: FP32 traces and tallies
    against the oracle (the sphere case is Rayleigh scattering with the dipole code)."""
    eps, s, x = grain
    model = W.spheroid_sphere(n=12, tau=1.0, albedo=0.6, b=(0.3, 0.5, 0.81), optics=W.dipole_optics(eps, s, x))
    run = {"sources": [{"type": "point", "pos": (0.02, 0.03, -0.01), "luminosity": 1.0, "n_packets": 8000}],
           "cameras": [W.camera((0.2, 0.9, 0.39), (13, 13), (2.0, 2.0))], "seed": 12,
           "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    o = oracle_run(model, run, n_trace=8000)
    g = gpu_run(model, run, "fp32", n_trace=8000)
    assert trace_match_fraction(g["trace"], o["trace"], 1e-4) >= 0.99
    assert np.linalg.norm(g["S"] - o["S"]) < 2e-3 * np.linalg.norm(o["S"])
    assert np.linalg.norm(g["absorbed"] - o["absorbed"]) < 2e-3 * np.linalg.norm(o["absorbed"])
