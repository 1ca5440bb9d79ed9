"""mcrt_launch_packets_noalloc: the transport entry point for callers that cannot
allocate device memory (code inside another framework's memory pool or under a fixed
memory plan).  The caller owns every input and output; the call's scratch lives in a
static device array.  Checked through the C ABI against mcrt_launch_packets on the
same problem, on two calls in a row (the shared array keeps the previous call's
contents, so each call must clear what starts at zero).

Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

from paper_2512_01283_gb300 import build as B
from paper_2512_01283_gb300 import mcrt as M
from paper_2512_01283_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("a CUDA GPU is required for -m gpu tests")
    B.build()
    M.lib()
    return torch


def to_device(torch, model):
    dev = {"lo": model["lo"], "hi": model["hi"]}
    for k in ("kappa_abs", "kappa_sca", "bfield"):
        dev[k] = None if model.get(k) is None else torch.from_numpy(np.ascontiguousarray(model[k], dtype=np.float32)).cuda()
    opt = {"model": model["optics"]["model"]}
    for k in ("mueller", "bin_weight", "kext"):
        if k in model["optics"]:
            opt[k] = torch.from_numpy(np.ascontiguousarray(model["optics"][k], dtype=np.float32)).cuda()
    dev["optics"] = opt
    return dev


def reference(model, run, precision):
    # the no-allocation entry point tallies inside the transport kernel: compare with the
    # allocating entry point on that same path (its FP32 default tallies in rounds)
    m = M.Model(model)
    st = M.launch(m, run, precision=precision, inline_tally=True)
    S, A = m.tallies(len(run["cameras"]))
    m.close()
    return st, S, A


CASES = [
    ("rayleigh sphere 32^3, 1 camera, fp64", lambda: (W.rayleigh_sphere(), W.rayleigh_sphere_run(50_000, npix=16)),
     "fp64"),
    ("disk 24^3 with grain tables, star only, 4 cameras, fp32",
     lambda: (W.disk(n=24), dict(W.disk_run(40_000, n_cam=4, npix=16),
                                 sources=[{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0,
                                           "n_packets": 40_000}])), "fp32"),
]


@pytest.mark.parametrize("name,make,precision", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_entry_point(torch_cuda, name, make, precision):
    torch = torch_cuda
    model, run = make()
    ref_st, ref_S, ref_A = reference(model, run, precision)
    dev = to_device(torch, model)
    ncell = model["kappa_abs"].size
    n_cam = len(run["cameras"])
    source = torch.empty((ncell, n_cam, 4), dtype=torch.float64, device="cuda")
    absorbed = torch.empty(ncell, dtype=torch.float64, device="cuda")
    for call in range(2):
        # garbage in the outputs: the call must zero them itself
        source.fill_(7.0)
        absorbed.fill_(-3.0)
        free_before = torch.cuda.mem_get_info()[0]
        st = M.launch_noalloc(dev, run, source, absorbed, precision=precision)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        assert st["status"] == M.MCRT_OK
        for key in ("emitted", "escaped", "events", "segments", "scatterings", "tally_segments"):
            assert st[key] == ref_st[key], (call, key)
        for key in ("emitted_energy", "escaped_energy", "absorbed_energy"):
            assert abs(st[key] - ref_st[key]) <= 1e-9 * abs(ref_st["emitted_energy"]), (call, key)
        S = source.cpu().numpy()
        A = absorbed.cpu().numpy()
        assert np.linalg.norm(S - ref_S) <= 1e-9 * np.linalg.norm(ref_S), call
        assert np.linalg.norm(A - ref_A) <= 1e-9 * max(np.linalg.norm(ref_A), 1e-300), call


def test_noalloc_beam_source_fp32(torch_cuda):
    """A plane beam into a scattering, absorbing slab with aligned grains (FP32,
    Rayleigh, two cameras), twice in a row, against the allocating entry point."""
    torch = torch_cuda
    model = W.dichroic_slab(n=16, tau=2.0, albedo=0.5)
    run = W.beam_run(30_000, seed=3, cameras=[W.camera((0, 0, 1), (8, 8), (1.0, 1.0)),
                                              W.camera((0.6, 0, 0.8), (8, 8), (1.0, 1.0))])
    ref_st, ref_S, ref_A = reference(model, run, "fp32")
    dev = to_device(torch, model)
    source = torch.empty((model["kappa_abs"].size, 2, 4), dtype=torch.float64, device="cuda")
    absorbed = torch.empty(model["kappa_abs"].size, dtype=torch.float64, device="cuda")
    for call in range(2):
        source.fill_(5.0)
        absorbed.fill_(5.0)
        st = M.launch_noalloc(dev, run, source, absorbed, precision="fp32")
        assert st["status"] == M.MCRT_OK
        for key in ("emitted", "escaped", "events", "scatterings", "tally_segments"):
            assert st[key] == ref_st[key], (call, key)
        S, A = source.cpu().numpy(), absorbed.cpu().numpy()
        assert np.linalg.norm(S - ref_S) <= 1e-6 * np.linalg.norm(ref_S), call
        assert np.linalg.norm(A - ref_A) <= 1e-6 * np.linalg.norm(ref_A), call


def test_noalloc_half_ranges_accumulate_to_one_call(torch_cuda):
    """Two calls over the halves of the packet ids, the second with accumulate = 1 (the
    outputs kept while the shared scratch's counters start again at zero), equal one
    allocating call over all ids."""
    torch = torch_cuda
    model = W.disk(n=24)
    run = dict(W.disk_run(20_000, n_cam=2, npix=8),
               sources=[{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": 20_000}])
    ref_st, ref_S, ref_A = reference(model, run, "fp32")
    dev = to_device(torch, model)
    source = torch.full((model["kappa_abs"].size, 2, 4), 9.0, dtype=torch.float64, device="cuda")
    absorbed = torch.full((model["kappa_abs"].size,), 9.0, dtype=torch.float64, device="cuda")
    st1 = M.launch_noalloc(dev, dict(run, pid_begin=0, pid_end=10_000), source, absorbed, precision="fp32")
    st2 = M.launch_noalloc(dev, dict(run, pid_begin=10_000, pid_end=20_000), source, absorbed, precision="fp32",
                           accumulate=1)
    for key in ("emitted", "escaped", "events", "segments", "scatterings", "tally_segments"):
        assert st1[key] + st2[key] == ref_st[key], key
    S, A = source.cpu().numpy(), absorbed.cpu().numpy()
    assert np.linalg.norm(S - ref_S) <= 1e-6 * np.linalg.norm(ref_S)
    assert np.linalg.norm(A - ref_A) <= 1e-6 * np.linalg.norm(ref_A)


def test_noalloc_without_cameras(torch_cuda):
    """No camera and no source-tally buffer: only the absorbed tally is written."""
    torch = torch_cuda
    model = W.disk(n=24)
    run = dict(W.disk_run(10_000, n_cam=0),
               sources=[{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": 10_000}])
    run["cameras"] = []
    ref_st, _, ref_A = reference(model, run, "fp32")
    dev = to_device(torch, model)
    absorbed = torch.full((model["kappa_abs"].size,), -1.0, dtype=torch.float64, device="cuda")
    st = M.launch_noalloc(dev, run, None, absorbed, precision="fp32")
    assert st["events"] == ref_st["events"] and st["tally_segments"] == 0
    A = absorbed.cpu().numpy()
    assert np.linalg.norm(A - ref_A) <= 1e-6 * np.linalg.norm(ref_A)
    # the absorbed total sums each packet's FP32 absorbed energy, the tally widened terms
    assert abs(A.sum() - st["absorbed_energy"]) <= 1e-7 * st["emitted_energy"]


def test_noalloc_rejects_sizes_beyond_its_limit(torch_cuda):
    torch = torch_cuda
    model = W.rayleigh_sphere(n=4)
    big = np.zeros((64, 64, 33), dtype=np.float32)  # 135168 cells > 131072
    model["kappa_abs"] = big
    model["kappa_sca"] = big
    dev = to_device(torch, model)
    absorbed = torch.empty(big.size, dtype=torch.float64, device="cuda")
    with pytest.raises(M.McrtError) as e:
        M.launch_noalloc(dev, W.rayleigh_sphere_run(10, npix=4) | {"cameras": []}, None, absorbed)
    assert e.value.status == M.MCRT_E_INVAL and "static limit" in str(e.value)
    # thermal sources need per-cell emission scratch and are refused
    model = W.dichroic_slab(n=8, tau=1.0, emissivity=1.0)
    dev = to_device(torch, model)
    absorbed = torch.empty(512, dtype=torch.float64, device="cuda")
    with pytest.raises(M.McrtError) as e:
        M.launch_noalloc(dev, {"sources": [{"type": "thermal", "n_packets": 10}], "cameras": []}, None, absorbed)
    assert e.value.status == M.MCRT_E_INVAL
