"""The inclined-disk test of Sec. 3.1 on the GPU, through step 1 (transport and
tally) and step 2 (images), in the kernels the library launches for it: the in-place
tally with the Rayleigh closed form, and the table rounds with the Rayleigh matrix as
a 181-angle table.  Needs a GB300: run with ``-m gpu``.

Light of a central star reaching a thin annulus of dipole grains travels in the disk
plane; scattered once and seen at inclination i, the integrated Q/I is
sin^2 i / (2 + sin^2 i) and U/I = 0 (closed form with the small out-of-plane part in
``closed_forms.inclined_disk_p``).
"""
import math

import numpy as np
import pytest

import closed_forms as CF
from accuracy_report import record
from oracle import oracle as O
from paper_2512_01283_gb300 import build as B
from paper_2512_01283_gb300 import mcrt as M
from paper_2512_01283_gb300 import workloads as W

pytestmark = pytest.mark.gpu
INCL = (0, 15, 30, 45, 60, 75, 90)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    B.build()
    M.lib()


def gpu_batches(model, run, nb, per, precision):
    """Stokes sums [nb][n_cam][4] of the images of nb launches of `per` ids each."""
    mdl = M.Model(model)
    out = np.zeros((nb, len(run["cameras"]), 4))
    try:
        for b in range(nb):
            st = M.launch(mdl, dict(run, pid_begin=b * per, pid_end=(b + 1) * per), precision=precision)
            assert st["emitted"] == per and st["escaped"] == per
            for k, c in enumerate(run["cameras"]):
                img = np.zeros((4, c["npix"][1], c["npix"][0]))
                mdl.image(k, img)
                out[b, k] = img.sum(axis=(1, 2)) * nb
    finally:
        mdl.close()
    return out


@pytest.mark.parametrize("table", [False, True])
def test_inclined_thin_disk_polarization(table):
    """1e9 packets in 16 launches, FP32, images of 1024^2 pixels.  Gate: 4 batch sigma
    plus 1e-4 on Q/I and U/I at every inclination (the pixel quadrature of a thin disk
    seen at 75 deg errs by 9e-4 at 256^2, 7e-5 at 512^2 and 2e-5 at 1024^2 in Q/I, the
    oracle's images against its own volume sums).  The table path adds the
    theta-linear interpolation of the Rayleigh matrix, below 1e-4 in Q/I."""
    model = W.inclined_thin_disk(table=table)
    g = model["geometry"]
    kz2 = CF.thin_annulus_kz2(g["h"], g["r_in"], g["r_out"])
    nb, per = 16, 62_500_000
    run = W.thin_disk_run(nb * per, seed=21, npix=1024)
    sums = gpu_batches(model, run, nb, per, "fp32")
    tot = sums.mean(axis=0)
    for k, a in enumerate(INCL):
        q = sums[:, k, 1] / sums[:, k, 0]
        u = sums[:, k, 2] / sums[:, k, 0]
        sq, su = q.std(ddof=1) / math.sqrt(nb), u.std(ddof=1) / math.sqrt(nb)
        p = CF.inclined_disk_p(math.radians(a), kz2)
        record("inclined thin disk (Sec. 3.1), 1e9 packets, fp32, " + ("table rounds" if table else "in place"),
               "|Q/I - p(i)| at i = %d deg" % a, abs(tot[k, 1] / tot[k, 0] - p), 4 * sq + 1e-4)
        assert abs(tot[k, 1] / tot[k, 0] - p) < 4 * sq + 1e-4, (a, tot[k, 1] / tot[k, 0], p, sq)
        assert abs(tot[k, 2] / tot[k, 0]) < 4 * su + 1e-4, (a, tot[k, 2] / tot[k, 0], su)
        assert abs(tot[k, 3]) < 1e-6 * tot[k, 0]
        assert sq < 2e-4


def test_inclined_thin_disk_images_equal_the_oracle_fp64():
    """Same seed, FP64 kernels: every pixel of every inclination equals the oracle's
    to 1e-7 of the image's largest pixel (trace-identical packets; the cell record
    keeps the grain quaternion of the field along x, cos 45 deg, in FP32)."""
    model = W.inclined_thin_disk()
    run = W.thin_disk_run(1_000_000, seed=22, npix=256)  # pixel rows inside the layer edge-on
    mdl = M.Model(model)
    M.launch(mdl, run, precision="fp64")
    gimgs = []
    for k in range(len(INCL)):
        img = np.zeros((4, 256, 256))
        mdl.image(k, img)
        gimgs.append(img)
    mdl.close()
    o = O.transport(model, dict(run, n_threads=8))
    for k in range(len(INCL)):
        oi = O.image(model, run, o["S"], k)
        scale = np.abs(oi[0]).max()
        assert scale > 0
        assert np.max(np.abs(gimgs[k] - oi)) < 1e-7 * scale, k
