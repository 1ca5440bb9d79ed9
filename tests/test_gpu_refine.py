"""Static mesh refinement on the CUDA path (through the C ABI) against the FP64 oracle
on the same seeded inputs.  Needs a GB300: run with ``-m gpu``.

Tolerances as in the other parity tests: traces within 1e-4 relative for >= 99.9 %
(FP64) or 99 % (FP32) of packets; tallies and integrated image Stokes to 1e-7 (FP64;
the grain quaternion is stored in FP32) or 2e-3 of the total I (FP32).
"""
import numpy as np
import pytest

from accuracy_report import integrated_error, record
from oracle import oracle as O
from paper_2512_01283_gb300 import build as B
from paper_2512_01283_gb300 import mcrt as M
from paper_2512_01283_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    B.build()
    M.lib()


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


@pytest.fixture(scope="module")
def refined_disk():
    model = W.disk_refined(n=24, factor=3)
    run = W.disk_run(n_packets=20_000, n_cam=2, npix=16)
    return model, run, oracle_run(model, run, n_trace=20_000)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_refined_disk_parity(refined_disk, prec):
    """The flared disk with a 3x refined inner patch (fields at the patch's own cell
    centres), star and thermal emission: traces, tallies, absorbed energy and images."""
    model, run, o = refined_disk
    assert O.n_cells(model) == 24 ** 3 + 18 * 18 * 6
    g = gpu_run(model, run, prec, n_trace=20_000)
    assert g["S"].shape[0] == O.n_cells(model)
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= (0.999 if prec == "fp64" else 0.99), frac
    tol = 1e-7 if prec == "fp64" else 2e-3
    dS = np.linalg.norm(g["S"] - o["S"]) / np.linalg.norm(o["S"])
    dA = np.linalg.norm(g["absorbed"] - o["absorbed"]) / np.linalg.norm(o["absorbed"])
    assert dS < tol and dA < tol, (dS, dA)
    # the patch holds tallies of its own
    assert np.abs(o["S"][24 ** 3:]).sum() > 0.05 * np.abs(o["S"]).sum()
    err = integrated_error(g["images"], o["images"])
    record("refined disk 24^3 + 3x patch, star + thermal, 2e4 packets, " + prec, "max integrated |dX|/I", err, 1e-3)
    assert err < (1e-7 if prec == "fp64" else 1e-3), err
    assert g["stats"]["emitted_energy"] == pytest.approx(o["stats"]["emitted_energy"], rel=1e-6)


def test_refined_table_rounds_equal_the_in_place_tally():
    """FP32 table launches on a refined grid run in rounds like plain grids: the same
    packets and tallies as the in-place tally, over several rounds between which packets
    wait, some of them inside patches."""
    model = W.disk_refined(n=48, factor=3)
    run = W.disk_run(n_packets=4_000_000, n_cam=4, npix=16)
    ref = gpu_run(model, run, "fp32", n_trace=200_000, inline_tally=True)
    assert ref["stats"]["wave_iterations"] == 0
    g = gpu_run(model, run, "fp32", n_trace=200_000)
    assert g["stats"]["wave_iterations"] >= 2  # packets parked and resumed
    assert g["stats"]["events"] == ref["stats"]["events"]
    assert trace_match_fraction(g["trace"], ref["trace"], 1e-6) >= 0.999
    assert np.linalg.norm(g["S"] - ref["S"]) < 1e-6 * np.linalg.norm(ref["S"])
    assert np.abs(g["S"][48 ** 3:]).sum() > 0.05 * np.abs(g["S"]).sum()
    assert np.linalg.norm(g["absorbed"] - ref["absorbed"]) < 1e-6 * np.linalg.norm(ref["absorbed"])
    for k in range(4):
        assert np.linalg.norm(g["images"][k] - ref["images"][k]) < 1e-6 * np.linalg.norm(ref["images"][k])
    # the packet ids split over three launches that add to the same tallies
    m = M.Model(model)
    M.launch(m, dict(run, pid_end=1_300_001), precision="fp32")
    M.launch(m, dict(run, pid_begin=1_300_001, pid_end=2_633_333), precision="fp32", accumulate=1)
    M.launch(m, dict(run, pid_begin=2_633_333), precision="fp32", accumulate=1)
    S, A = m.tallies(4)
    m.close()
    assert np.linalg.norm(S - ref["S"]) < 1e-6 * np.linalg.norm(ref["S"])
    assert np.linalg.norm(A - ref["absorbed"]) < 1e-6 * np.linalg.norm(ref["absorbed"])


def test_refined_copy_equals_the_plain_grid_on_gpu():
    """A patch copying its parents' values is the same medium: the FP64 traces equal the
    plain grid's and the patch tallies fold back onto their parents."""
    m0 = W.dichroic_slab(n=8, tau=2.0, p=0.05, b_angle_deg=30.0, albedo=0.7)
    m0["optics"] = W.table_optics(n_bins=2)
    box, f = (2, 2, 2, 5, 6, 4), 2
    m1 = W.refine_uniform(m0, [(box, f)])
    run = {"sources": [{"type": "point", "pos": (0.41, 0.52, 0.47), "luminosity": 1.0, "n_packets": 5000}],
           "cameras": [W.camera((0.3, 0.2, 0.93), (8, 8), (1.0, 1.0))], "seed": 4,
           "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    a, b = gpu_run(m0, run, "fp64", n_trace=5000), gpu_run(m1, run, "fp64", n_trace=5000)
    assert np.allclose(b["trace"][:, 0:10], a["trace"][:, 0:10], rtol=1e-9, atol=1e-12)
    assert np.array_equal(b["trace"][:, 10], a["trace"][:, 10])
    S = b["S"][:512].copy()
    i0, j0, k0, i1, j1, k1 = box
    pn = ((k1 - k0) * f, (j1 - j0) * f, (i1 - i0) * f)
    k, j, i = np.meshgrid(np.arange(pn[0]), np.arange(pn[1]), np.arange(pn[2]), indexing="ij")
    parent = ((k0 + k // f) * 8 + (j0 + j // f)) * 8 + (i0 + i // f)
    np.add.at(S, parent.ravel(), b["S"][512:])
    assert np.allclose(S, a["S"], rtol=1e-9, atol=1e-12 * np.abs(a["S"]).max())


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_refined_periodic_slab_parity(prec):
    """Patches on the periodic faces of a slab: leaving them through the face wraps."""
    m0 = W.plane_parallel_slab(nxy=6, nz=8, tau=2.0, albedo=0.8, periodic=3, b_angle_deg=40.0, p=0.05)
    m = W.refine_uniform(m0, [((4, 0, 2, 6, 3, 6), 2), ((0, 3, 1, 2, 6, 4), 3)])
    run = dict(W.center_source_run(10_000, cameras=[W.camera((0, 0, 1), (6, 6), (1.0, 1.0))]), roulette_threshold=1e-4,
               roulette_survival=0.1)
    o = oracle_run(m, run, n_trace=10_000)
    g = gpu_run(m, run, prec, n_trace=10_000)
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= (0.999 if prec == "fp64" else 0.99), frac
    dS = np.linalg.norm(g["S"] - o["S"]) / np.linalg.norm(o["S"])
    assert dS < (1e-7 if prec == "fp64" else 2e-3), dS


def test_refined_grid_errors():
    base = W.dichroic_slab(n=8, tau=1.0, albedo=0.5)
    bad = [
        [((0, 0, 0, 4, 4, 4), 2), ((3, 3, 3, 6, 6, 6), 2)],  # overlap
        [((0, 0, 0, 2, 2, 2), 1)],                           # factor 1
        [((6, 0, 0, 9, 2, 2), 2)],                           # outside the root grid
        [((2, 2, 2, 2, 4, 4), 2)],                           # empty box
    ]
    for patches in bad:
        with pytest.raises(M.McrtError) as e:
            M.Model(W.refine_uniform(base, patches))
        assert e.value.status == M.MCRT_E_INVAL
    m = W.refine_uniform(base, [((0, 0, 0, 2, 2, 2), 2)])
    m["refine"][0]["bfield"] = None  # the root has a field
    with pytest.raises(M.McrtError) as e:
        M.Model(m)
    assert e.value.status == M.MCRT_E_INVAL
    good = M.Model(W.refine_uniform(base, [((0, 0, 0, 2, 2, 2), 2)]))
    other = M.Model(base)
    run = W.beam_run(100)
    with pytest.raises(M.McrtError) as e:
        M.Batch([good, other], run)
    assert e.value.status == M.MCRT_E_INVAL
    good.close()
    other.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_refined_spheroid_sphere_parity(prec):
    """Aligned dipole spheroids on a refined grid: a 2x patch over the centre of the
    spheroid sphere, central star, two cameras (13 pixels: no pixel ray runs exactly along
    a cell face, where the two precisions may take different neighbours)."""
    base = W.spheroid_sphere(n=12, tau=1.5, albedo=0.6, b=(0.6, 0.0, 0.8))
    m = W.refine_uniform(base, [((3, 3, 3, 9, 9, 9), 2)])
    run = {"sources": [{"type": "point", "pos": (0.05, -0.02, 0.01), "luminosity": 1.0, "n_packets": 10_000}],
           "cameras": [W.camera((1, 0, 0), (13, 13), (2.0, 2.0)), W.camera((0.3, 0.4, 0.866), (13, 13), (2.0, 2.0))],
           "seed": 6, "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    o = oracle_run(m, run, n_trace=10_000)
    g = gpu_run(m, run, prec, n_trace=10_000)
    frac = trace_match_fraction(g["trace"], o["trace"], 1e-4)
    assert frac >= (0.999 if prec == "fp64" else 0.99), frac
    tol = 1e-7 if prec == "fp64" else 2e-3
    dS = np.linalg.norm(g["S"] - o["S"]) / np.linalg.norm(o["S"])
    assert dS < tol, dS
    err = integrated_error(g["images"], o["images"])
    assert err < (1e-7 if prec == "fp64" else 1e-3), err


def test_many_patches_largest_factor_parity():
    """The limits of a composite grid: 64 single-cell patches of factor 2 over a 8x8
    plane of a slab, one patch of factor 16 and patches on every face; FP64 traces and
    tallies against the oracle."""
    base = W.dichroic_slab(n=10, tau=1.5, p=0.05, b_angle_deg=35.0, albedo=0.7, emissivity=1.0)
    base["optics"] = W.table_optics(n_bins=2)
    patches = [((i, j, 4, i + 1, j + 1, 5), 2) for i in range(1, 9) for j in range(1, 9)]
    assert len(patches) == 64
    m = W.refine_uniform(base, patches[:60] + [((0, 0, 0, 1, 1, 1), 16), ((9, 9, 9, 10, 10, 10), 3),
                                               ((0, 5, 8, 10, 6, 10), 2), ((4, 0, 0, 6, 10, 2), 2)])
    run = {"sources": [{"type": "point", "pos": (0.31, 0.42, 0.47), "luminosity": 1.0, "n_packets": 6000},
                       {"type": "thermal", "luminosity": 0.0, "n_packets": 6000}],
           "cameras": [W.camera((0.3, 0.2, 0.93), (11, 11), (1.2, 1.2), center=(0.5, 0.5, 0.5))], "seed": 14,
           "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    o = oracle_run(m, run, n_trace=12_000)
    g = gpu_run(m, run, "fp64", n_trace=12_000)
    assert trace_match_fraction(g["trace"], o["trace"], 1e-4) >= 0.999
    assert np.linalg.norm(g["S"] - o["S"]) < 1e-7 * np.linalg.norm(o["S"])
    Itot = o["images"][0][0].sum()
    for e in range(4):
        assert abs(g["images"][0][e].sum() - o["images"][0][e].sum()) < 1e-7 * Itot
    # a 65th patch is refused
    with pytest.raises(M.McrtError):
        M.Model(W.refine_uniform(base, patches + [((0, 0, 9, 1, 1, 10), 2)]))
