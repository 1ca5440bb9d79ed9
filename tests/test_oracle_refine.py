"""Pins of the oracle's composite grid with static mesh refinement (Sec. 2: a
composite mesh, optionally with static mesh refinement).

The composite traversal is checked against a brute-force walk (every plane crossing
of the root and patch grids, each interval's midpoint located by box tests), and the
transport against refinement invariance: a patch whose cells copy their parent's
values is the same medium, so packets follow the same paths (to rounding), the patch
cells' tallies add up to their parent's, emission images do not change and the
thermal luminosity stays the same.  A patch on a periodic face checks the wrap."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2512_01283_gb300 import workloads as W

RNG = np.random.default_rng(31)


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def tiny_model():
    shape = (5, 3, 4)  # nz, ny, nx
    m = {"lo": (-1.0, 0.0, 0.5), "hi": (1.0, 1.5, 3.0), "kappa_abs": np.ones(shape, np.float32),
         "kappa_sca": np.zeros(shape, np.float32), "bfield": None, "emissivity": None,
         "optics": W.rayleigh_optics()}
    return W.refine_uniform(m, [((1, 0, 1, 3, 2, 3), 2), ((0, 2, 3, 2, 3, 5), 3)])


def brute_walk(m, p0, n):
    """Cells and lengths from all plane crossings; each interval's cell by box tests."""
    lo, hi = np.array(m["lo"]), np.array(m["hi"])
    nz, ny, nx = m["kappa_abs"].shape
    N = np.array([nx, ny, nz])
    d = (hi - lo) / N
    ts = [0.0]
    # exit of the box
    t_out = min(((hi[a] if n[a] > 0 else lo[a]) - p0[a]) / n[a] for a in range(3) if n[a] != 0)
    planes = [list(lo[a] + np.arange(N[a] + 1) * d[a]) for a in range(3)]
    patches = m["refine"]
    for q in patches:
        b, f = q["box"], q["factor"]
        for a in range(3):
            planes[a] += list(lo[a] + (b[a] + np.arange((b[3 + a] - b[a]) * f + 1) / f) * d[a])
    for a in range(3):
        if n[a] != 0:
            for x in planes[a]:
                t = (x - p0[a]) / n[a]
                if 0 < t < t_out:
                    ts.append(t)
    ts = sorted(set(ts + [t_out]))
    offs = [nx * ny * nz]
    for q in patches:
        b, f = q["box"], q["factor"]
        offs.append(offs[-1] + int(np.prod([(b[3 + a] - b[a]) * f for a in range(3)])))
    cells, lens = [], []
    for t0, t1 in zip(ts[:-1], ts[1:]):
        if t1 - t0 < 1e-13:
            continue
        x = p0 + 0.5 * (t0 + t1) * n
        r = np.floor((x - lo) / d).astype(int)
        c = (r[2] * ny + r[1]) * nx + r[0]
        for k, q in enumerate(patches):
            b, f = q["box"], q["factor"]
            if all(b[a] <= r[a] < b[3 + a] for a in range(3)):
                pn = [(b[3 + a] - b[a]) * f for a in range(3)]
                pl = lo + np.array(b[:3]) * d
                i = np.floor((x - pl) / (d / f)).astype(int)
                c = offs[k] + (i[2] * pn[1] + i[1]) * pn[0] + i[0]
        if cells and cells[-1] == c:
            lens[-1] += t1 - t0
        else:
            cells.append(int(c))
            lens.append(t1 - t0)
    return cells, lens


def test_composite_walk_matches_brute_force():
    m = tiny_model()
    assert O.n_cells(m) == 60 + 2 * 2 * 2 * 8 + 2 * 1 * 2 * 27
    lo, hi = np.array(m["lo"]), np.array(m["hi"])
    for _ in range(300):
        p0 = lo + RNG.uniform(0.02, 0.98, 3) * (hi - lo)
        n = unit(RNG.normal(size=3))
        cells, lens = O.dda_walk_composite(m, p0, n)
        bc, bl = brute_walk(m, p0, n)
        assert list(cells) == bc
        assert np.allclose(lens, bl, rtol=0, atol=1e-12)
    # rays along the axes through patch faces
    for n in np.eye(3).tolist() + (-np.eye(3)).tolist():
        p0 = np.array([0.1, 0.61, 1.2])
        cells, lens = O.dda_walk_composite(m, p0, n)
        bc, bl = brute_walk(m, p0, np.array(n))
        assert list(cells) == bc and np.allclose(lens, bl, atol=1e-12)


def medium():
    m = W.dichroic_slab(n=8, tau=2.0, p=0.05, b_angle_deg=30.0, albedo=0.7, emissivity=1.0)
    m["optics"] = W.table_optics(n_bins=2)
    return m


PATCHES = [((2, 2, 2, 5, 6, 4), 2), ((5, 0, 4, 8, 3, 7), 3)]


def test_refined_copy_is_the_same_medium_for_packets():
    """Same packets (point and beam sources) on the plain grid and on the grid with
    patches that copy their parents: identical traces to rounding, patch tallies that
    add up to their parent cells', the same absorbed energy per parent."""
    m0 = medium()
    m1 = W.refine_uniform(m0, PATCHES)
    cams = [W.camera((0.3, 0.2, 0.93), (8, 8), (1.0, 1.0)), W.camera((1, 0, 0), (8, 8), (1.0, 1.0))]
    run = {"sources": [{"type": "point", "pos": (0.41, 0.52, 0.47), "luminosity": 1.0, "n_packets": 3000},
                       {"type": "beam", "beam_dir": 1, "luminosity": 0.5, "n_packets": 2000}],
           "cameras": cams, "seed": 4, "n_trace": 5000, "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    a, b = O.transport(m0, run), O.transport(m1, run)
    ta, tb = a["trace"], b["trace"]
    assert np.allclose(tb[:, 0:10], ta[:, 0:10], rtol=1e-9, atol=1e-12)
    assert np.array_equal(tb[:, 10], ta[:, 10]) and np.array_equal(tb[:, 12], ta[:, 12])
    assert b["stats"]["segments"] > a["stats"]["segments"]  # the patches split segments
    # fold the patch cells back onto their parents
    nroot = 8 ** 3
    S, A = b["S"][:nroot].copy(), b["absorbed"][:nroot].copy()
    off = nroot
    for box, f in PATCHES:
        i0, j0, k0, i1, j1, k1 = box
        pn = ((k1 - k0) * f, (j1 - j0) * f, (i1 - i0) * f)
        cnt = pn[0] * pn[1] * pn[2]
        k, j, i = np.meshgrid(np.arange(pn[0]), np.arange(pn[1]), np.arange(pn[2]), indexing="ij")
        parent = ((k0 + k // f) * 8 + (j0 + j // f)) * 8 + (i0 + i // f)
        np.add.at(S, parent.ravel(), b["S"][off:off + cnt])
        np.add.at(A, parent.ravel(), b["absorbed"][off:off + cnt])
        off += cnt
    assert off == O.n_cells(m1)
    scale = np.abs(a["S"]).max()
    assert np.allclose(S, a["S"], rtol=1e-9, atol=1e-12 * scale)
    assert np.allclose(A, a["absorbed"], rtol=1e-9, atol=1e-12 * np.abs(a["absorbed"]).max())


def test_refined_copy_keeps_emission_images_and_luminosity():
    """Step 2 of the pure emission (no scattering source): the analytic cell solution
    composes exactly over sub-cells of a homogeneous cell, so the images agree to
    rounding; the thermal luminosity (cell weights times the cells' own volumes) too."""
    m0 = medium()
    m1 = W.refine_uniform(m0, PATCHES)
    cams = [W.camera(unit((0.3, -0.4, 0.8)), (12, 12), (1.2, 1.2), center=(0.5, 0.5, 0.5)),
            W.camera((0, 1, 0), (12, 12), (1.2, 1.2), center=(0.5, 0.5, 0.5))]
    run = {"sources": [{"type": "thermal", "luminosity": 0.0, "n_packets": 10}], "cameras": cams}
    for k in range(2):
        i0, i1 = O.image(m0, run, None, k), O.image(m1, run, None, k)
        assert np.abs(i0[0]).max() > 0
        assert np.allclose(i1, i0, rtol=1e-9, atol=1e-12 * np.abs(i0[0]).max())
    assert O.thermal_luminosity(m1, run) == pytest.approx(O.thermal_luminosity(m0, run), rel=1e-12)


def test_thermal_births_fill_patch_cells_by_weight():
    """A patch with its own (finer) emissivity: the share of thermal births inside the
    patch equals its share of the emission weights (binomial, 4 sigma)."""
    m = W.refine_uniform(medium(), [((2, 2, 2, 6, 6, 6), 2)])
    q = m["refine"][0]
    q["emissivity"] = (q["emissivity"] * (1.0 + RNG.uniform(0, 3, q["emissivity"].shape))).astype(np.float32)
    N = 4000
    run = {"sources": [{"type": "thermal", "luminosity": 0.0, "n_packets": N}], "seed": 12}
    rows = O.emit(m, run, range(N))
    pos = rows[:, 0:3]
    inside = np.all((pos >= 0.25) & (pos < 0.75), axis=1)
    kext = 2.0
    w_patch = (kext * 0.3 * q["emissivity"].astype(np.float64)).sum() * (1 / 16) ** 3
    w_root = (kext * 0.3 * m["emissivity"].astype(np.float64)).sum() * (1 / 8) ** 3
    w_root -= (kext * 0.3 * m["emissivity"][2:6, 2:6, 2:6].astype(np.float64)).sum() * (1 / 8) ** 3
    share = w_patch / (w_patch + w_root)
    assert abs(inside.mean() - share) < 4 * math.sqrt(share * (1 - share) / N)


def test_patch_on_a_periodic_face():
    """A patch touching the periodic x faces of a slab: leaving it through the face wraps
    to the opposite root cells; traces equal the unrefined periodic slab's."""
    m0 = W.plane_parallel_slab(nxy=6, nz=8, tau=2.0, albedo=0.8, periodic=3)
    m1 = W.refine_uniform(m0, [((4, 0, 2, 6, 3, 6), 2), ((0, 3, 1, 2, 6, 4), 2)])
    run = dict(W.center_source_run(3000, cameras=[W.camera((0, 0, 1), (6, 6), (1.0, 1.0))]), n_trace=3000)
    a, b = O.transport(m0, run), O.transport(m1, run)
    assert np.allclose(b["trace"][:, 0:10], a["trace"][:, 0:10], rtol=1e-9, atol=1e-12)
    assert np.array_equal(b["trace"][:, 10], a["trace"][:, 10])
