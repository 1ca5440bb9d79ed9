"""Python binding of the C ABI in ``include/mcrt.h`` (ctypes; argument marshalling
only -- every step of the transport and imaging runs in the CUDA kernels of
``libmcrt.so``).  There is no CPU fallback: if the library is missing or no GPU is
present the calls raise.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device memory);
torch is used only as a device-memory and stream container.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmcrt.so")

MCRT_OK, MCRT_E_INVAL, MCRT_E_NOMEM, MCRT_E_CUDA, MCRT_E_EVENT_CAP, MCRT_E_TIMEOUT, MCRT_E_STATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "MCRT_OK", -1: "MCRT_E_INVAL", -2: "MCRT_E_NOMEM", -3: "MCRT_E_CUDA", -4: "MCRT_E_EVENT_CAP",
                -5: "MCRT_E_TIMEOUT", -6: "MCRT_E_STATE"}
SRC = {"point": 0, "beam": 1, "thermal": 2}
SCAT = {"rayleigh": 0, "table": 1, "dipole": 4}
PRECISION = {"fp32": 0, "fp64": 1}


class McrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Source(C.Structure):
    _fields_ = [("type", C.c_int32), ("beam_dir", C.c_int32), ("luminosity", C.c_double),
                ("pos", C.c_double * 3), ("n_packets", C.c_int64)]


class Camera(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("center", C.c_double * 3), ("fov", C.c_double * 2),
                ("npix", C.c_int32 * 2)]


class LaunchDesc(C.Structure):
    _fields_ = [("n_sources", C.c_int32), ("sources", C.POINTER(Source)),
                ("n_cameras", C.c_int32), ("cameras", C.POINTER(Camera)),
                ("seed", C.c_uint32), ("stream", C.c_uint32), ("precision", C.c_int32), ("accumulate", C.c_int32),
                ("pid_begin", C.c_int64), ("pid_end", C.c_int64),
                ("roulette_threshold", C.c_double), ("roulette_survival", C.c_double),
                ("max_events", C.c_int64), ("max_trials", C.c_int32), ("block_size", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("time_budget_s", C.c_double),
                ("n_trace", C.c_int64), ("trace", C.c_void_p), ("optics", C.c_int32), ("flags", C.c_int32),
                ("tally_blocks_per_sm", C.c_int32)]

FLAG_INLINE_TALLY = 1
FLAG_MMA_SYNC_TALLY = 2

OPTICS = {"tables": 0, "surrogate": 1}


STAT_FIELDS = ["emitted_energy", "escaped_energy", "absorbed_energy", "roulette_lost", "roulette_gain", "cap_lost",
               "events", "segments", "scatterings", "emitted", "escaped", "roulette_killed", "cap_hits", "trials",
               "kernel_ms", "status_bits", "tally_segments", "absorb_segments",
               "mlp_tally_rows", "mlp_scatter_rows", "mlp_fallback_map", "mlp_fallback_realizability",
               "tally_overflow", "envelope_miss", "wave_iterations", "ms_transport", "ms_tally", "ms_scatter"]


class Stats(C.Structure):
    _fields_ = [(f, C.c_double) for f in STAT_FIELDS]


class TuneReport(C.Structure):
    _fields_ = [("n", C.c_int32), ("best", C.c_int32), ("block_size", C.c_int32 * 16),
                ("blocks_per_sm", C.c_int32 * 16), ("interleave", C.c_int32 * 16), ("events_per_s", C.c_double * 16)]


class Patch(C.Structure):
    _fields_ = [("box", C.c_int32 * 6), ("factor", C.c_int32), ("kappa_abs", C.c_void_p), ("kappa_sca", C.c_void_p),
                ("bfield", C.c_void_p), ("emissivity", C.c_void_p)]


class NoAllocProblem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("kappa_abs", C.c_void_p), ("kappa_sca", C.c_void_p),
                ("bfield", C.c_void_p), ("model", C.c_int32), ("n_bins", C.c_int32), ("n_theta", C.c_int32),
                ("mueller", C.c_void_p), ("bin_weight", C.c_void_p), ("n_ktheta", C.c_int32),
                ("kext", C.c_void_p), ("source", C.c_void_p), ("absorbed", C.c_void_p),
                ("cuda_stream", C.c_void_p)]


_lib = None

# symbols of include/mcrt.h
SYMBOLS = ["mcrt_create_grid", "mcrt_set_dust_tables", "mcrt_launch_packets", "mcrt_image_stokes",
           "mcrt_get_tallies", "mcrt_destroy", "mcrt_last_error", "mcrt_unit_eval", "mcrt_launch_packets_noalloc",
           "mcrt_batch_create", "mcrt_batch_run", "mcrt_batch_tune", "mcrt_batch_images", "mcrt_batch_destroy",
           "mcrt_surrogate_create", "mcrt_surrogate_train", "mcrt_surrogate_eval", "mcrt_surrogate_labels",
           "mcrt_surrogate_grad", "mcrt_surrogate_grad_fp32", "mcrt_surrogate_params", "mcrt_surrogate_param_count", "mcrt_surrogate_destroy",
           "mcrt_surrogate_error_map", "mcrt_set_surrogate", "mcrt_surrogate_eval_engine", "mcrt_set_dust_dipole",
           "mcrt_dipole_constants", "mcrt_set_tallies", "mcrt_create_grid_refined", "mcrt_microbench", "mcrt_tally_buffers"]


def lib():
    """Load ``libmcrt.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libmcrt.so is not built (run paper_2512_01283_gb300.build.build()); "
                           "there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dp, fp = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.c_void_p
    L.mcrt_create_grid.argtypes = [C.POINTER(C.c_void_p), i32, i32, i32, dp, dp, fp, fp, fp, fp, i32, vp]
    L.mcrt_create_grid_refined.argtypes = [C.POINTER(C.c_void_p), i32, i32, i32, dp, dp, fp, fp, fp, fp, i32, i32,
                                           C.POINTER(Patch), vp]
    L.mcrt_set_dust_tables.argtypes = [vp, i32, i32, i32, fp, fp, i32, fp]
    L.mcrt_launch_packets.argtypes = [C.POINTER(C.c_void_p), i32, C.POINTER(LaunchDesc), C.POINTER(Stats)]
    L.mcrt_image_stokes.argtypes = [vp, i32, vp]
    L.mcrt_get_tallies.argtypes = [vp, vp, vp]
    L.mcrt_set_tallies.argtypes = [vp, vp, vp]
    L.mcrt_tally_buffers.argtypes = [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]
    L.mcrt_microbench.argtypes = [i32, C.c_uint64, C.c_uint64, C.POINTER(C.c_double)]
    L.mcrt_destroy.argtypes = [vp]
    L.mcrt_last_error.argtypes = [vp]
    L.mcrt_last_error.restype = C.c_char_p
    L.mcrt_unit_eval.argtypes = [i32, i32, i64, vp, vp]
    L.mcrt_launch_packets_noalloc.argtypes = [C.POINTER(NoAllocProblem), C.POINTER(LaunchDesc), C.POINTER(Stats)]
    L.mcrt_batch_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), i32, C.POINTER(LaunchDesc)]
    L.mcrt_batch_run.argtypes = [vp, C.c_uint32, C.POINTER(Stats)]
    L.mcrt_batch_tune.argtypes = [vp, i64, C.POINTER(TuneReport)]
    L.mcrt_batch_images.argtypes = [vp, vp]
    L.mcrt_batch_destroy.argtypes = [vp]
    L.mcrt_surrogate_create.argtypes = [C.POINTER(C.c_void_p), vp, C.c_uint32]
    L.mcrt_surrogate_train.argtypes = [vp, i64, i32, C.c_double, vp]
    L.mcrt_surrogate_eval.argtypes = [vp, i64, vp, vp]
    L.mcrt_surrogate_labels.argtypes = [vp, i64, vp, vp]
    L.mcrt_surrogate_grad.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.mcrt_surrogate_grad_fp32.argtypes = [vp, i64, vp, vp, vp, vp, vp]
    L.mcrt_surrogate_params.argtypes = [vp, vp, i32]
    L.mcrt_surrogate_param_count.argtypes = []
    L.mcrt_surrogate_param_count.restype = C.c_int64
    L.mcrt_surrogate_destroy.argtypes = [vp]
    L.mcrt_surrogate_error_map.argtypes = [vp, i64, vp]
    L.mcrt_set_surrogate.argtypes = [vp, vp, C.c_double]
    L.mcrt_surrogate_eval_engine.argtypes = [vp, i32, i64, vp, vp]
    d = C.c_double
    L.mcrt_set_dust_dipole.argtypes = [vp, d, d, d, d]
    L.mcrt_dipole_constants.argtypes = [d, d, d, d, C.POINTER(C.c_double)]
    for name in SYMBOLS:
        if name not in ("mcrt_last_error", "mcrt_surrogate_param_count"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status, ctx=None):
    if status != MCRT_OK:
        msg = lib().mcrt_last_error(ctx).decode(errors="replace")
        raise McrtError(status, msg)


def _ptr(a, dtype):
    """Pointer and keep-alive object for a numpy array or a CUDA torch tensor."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return C.c_void_p(arr.ctypes.data), arr


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


DIPOLE_KEYS = ["L0", "L1", "al0_re", "al0_im", "al1_re", "al1_im", "q_ext0", "q_ext1", "q_sca0", "q_sca1",
               "q_abs0", "q_abs1", "rho_re", "rho_im", "zn", "env"]


def microbench(kind, nbytes, n_ops):
    """mcrt_microbench: CUDA-event milliseconds of n_ops FP64 reductions (kind 0 scalar
    atomics, 1 bulk 256-byte rows) into a buffer of nbytes."""
    ms = C.c_double()
    _check(lib().mcrt_microbench(int(kind), int(nbytes), int(n_ops), C.byref(ms)))
    return ms.value


def dipole_constants(eps, aspect, x):
    """Constants of aligned dipole spheroids as the device computes them
    (mcrt_dipole_constants); index 0 perpendicular to the symmetry axis, 1 along it."""
    eps = complex(eps)
    out = (C.c_double * 16)()
    _check(lib().mcrt_dipole_constants(eps.real, eps.imag, float(aspect), float(x), out))
    return dict(zip(DIPOLE_KEYS, list(out)))


class Model:
    """A device-resident model: grid (mcrt_create_grid) plus optics (mcrt_set_dust_tables)."""

    def __init__(self, model: dict, stream=None):
        L = lib()
        ka = model["kappa_abs"]
        nz, ny, nx = tuple(ka.shape)
        self.shape = (nz, ny, nx)
        self.ncell = nx * ny * nz
        self.center = tuple((float(a) + float(b)) / 2 for a, b in zip(model["lo"], model["hi"]))
        keep = []
        pk, k1 = _ptr(ka, np.float32)
        ps, k2 = _ptr(model["kappa_sca"], np.float32)
        pb, k3 = _ptr(model.get("bfield"), np.float32)
        pe, k4 = _ptr(model.get("emissivity"), np.float32)
        keep += [k1, k2, k3, k4]
        lo = (C.c_double * 3)(*model["lo"])
        hi = (C.c_double * 3)(*model["hi"])
        h = C.c_void_p()
        patches = model.get("refine") or []
        self.ncell = nx * ny * nz
        if patches:
            arr = (Patch * len(patches))()
            for i, q in enumerate(patches):
                arr[i].box = (C.c_int32 * 6)(*q["box"])
                arr[i].factor = int(q["factor"])
                for key in ("kappa_abs", "kappa_sca", "bfield", "emissivity"):
                    ptr, k = _ptr(q.get(key), np.float32)
                    keep.append(k)
                    setattr(arr[i], key, ptr)
                self.ncell += int(np.prod([(q["box"][3 + a] - q["box"][a]) * q["factor"] for a in range(3)]))
            st = L.mcrt_create_grid_refined(C.byref(h), nx, ny, nz, lo, hi, pk, ps, pb, pe, int(model.get("periodic", 0)),
                                            len(patches), arr, _stream_handle(stream))
        else:
            st = L.mcrt_create_grid(C.byref(h), nx, ny, nz, lo, hi, pk, ps, pb, pe, int(model.get("periodic", 0)),
                                    _stream_handle(stream))
        _check(st)
        self.h = h
        try:
            self.set_optics(model["optics"])
        except Exception:
            self.close()
            raise

    def set_optics(self, optics: dict):
        L = lib()
        m = SCAT[optics["model"]]
        if m == SCAT["dipole"]:
            eps = complex(optics["eps"])
            _check(L.mcrt_set_dust_dipole(self.h, eps.real, eps.imag, float(optics["aspect"]), float(optics["x"])),
                   self.h)
            return
        pkx, kx = _ptr(optics["kext"], np.float32)
        n_k = int(np.asarray(optics["kext"]).shape[0]) if not hasattr(optics["kext"], "is_cuda") else optics["kext"].shape[0]
        if m == 1:
            pm, km = _ptr(optics["mueller"], np.float32)
            pw, kw = _ptr(optics["bin_weight"], np.float32)
            nb, nt = optics["mueller"].shape[0], optics["mueller"].shape[1]
        else:
            pm = pw = None
            nb = nt = 0
        _check(L.mcrt_set_dust_tables(self.h, m, nb, nt, pm, pw, n_k, pkx), self.h)

    def image(self, camera: int, out=None):
        """Stokes image [4][ny][nx] (FP64) of a camera of the last launch."""
        L = lib()
        if out is None:
            raise ValueError("pass out (numpy float64 [4][ny][nx] or CUDA tensor)")
        p, keep = _ptr(out, np.float64)
        _check(L.mcrt_image_stokes(self.h, int(camera), p), self.h)
        return out

    def set_surrogate(self, sur: "Surrogate", bound=0.05):
        """mcrt_set_surrogate: attach a trained network (launch with optics="surrogate")."""
        _check(lib().mcrt_set_surrogate(self.h, sur.h, float(bound)), self.h)

    def tallies(self, n_cam: int):
        L = lib()
        S = np.zeros((self.ncell, max(1, n_cam), 4))
        A = np.zeros(self.ncell)
        _check(L.mcrt_get_tallies(self.h, C.c_void_p(S.ctypes.data) if n_cam > 0 else None,
                                  C.c_void_p(A.ctypes.data)), self.h)
        return S[:, :n_cam], A

    def tallies_into(self, source=None, absorbed=None):
        """mcrt_get_tallies into caller buffers (numpy or CUDA tensors, FP64, contiguous)."""
        for b in (source, absorbed):
            if isinstance(b, np.ndarray) and (b.dtype != np.float64 or not b.flags.c_contiguous):
                raise ValueError("tally buffers must be contiguous float64")
        ps, ks = _ptr(source, np.float64)
        pa, ka = _ptr(absorbed, np.float64)
        _check(lib().mcrt_get_tallies(self.h, ps, pa), self.h)

    def set_tallies(self, source=None, absorbed=None):
        """mcrt_set_tallies: replace the last launch's tallies (e.g. with their sum over ranks)."""
        ps, ks = _ptr(source, np.float64)
        pa, ka = _ptr(absorbed, np.float64)
        _check(lib().mcrt_set_tallies(self.h, ps, pa), self.h)

    def tally_tensors(self, n_cam: int):
        """The library's own tally buffers of the last launch as CUDA torch tensors
        (mcrt_tally_buffers; no copy): source [ncell][n_cam][4] (None without cameras)
        and absorbed [ncell], FP64, valid until the next launch or close."""
        import torch

        ps, pa = C.c_void_p(), C.c_void_p()
        ns, na = C.c_int64(), C.c_int64()
        _check(lib().mcrt_tally_buffers(self.h, C.byref(ps), C.byref(pa), C.byref(ns), C.byref(na)), self.h)

        class _View:  # a device buffer described by the CUDA array interface
            def __init__(self, ptr, shape):
                self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape, "typestr": "<f8",
                                                 "version": 3, "strides": None, "stream": None}

        src = None
        if ns.value > 0:
            assert ns.value == self.ncell * n_cam * 4
            src = torch.as_tensor(_View(ps.value, (self.ncell, n_cam, 4)), device="cuda")
        ab = torch.as_tensor(_View(pa.value, (na.value,)), device="cuda")
        return src, ab

    def close(self):
        if getattr(self, "h", None):
            lib().mcrt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_desc(run: dict, precision="fp32", trace=None, n_trace=0, default_center=(0.0, 0.0, 0.0), **kw):
    """mcrt_launch_desc from a run dict (sources, cameras, seed, roulette...);
    cameras without a centre image ``default_center``."""
    keep = []
    srcs = run["sources"]
    sa = (Source * len(srcs))()
    for i, s in enumerate(srcs):
        sa[i].type = SRC[s["type"]]
        sa[i].beam_dir = int(s.get("beam_dir", 1))
        sa[i].luminosity = float(s.get("luminosity", 1.0))
        sa[i].pos = (C.c_double * 3)(*s.get("pos", (0.0, 0.0, 0.0)))
        sa[i].n_packets = int(s["n_packets"])
    keep.append(sa)
    cams = run.get("cameras", [])
    ca = (Camera * max(1, len(cams)))()
    for i, c in enumerate(cams):
        ca[i].dir = (C.c_double * 3)(*c["dir"])
        ca[i].center = (C.c_double * 3)(*c.get("center", default_center))
        ca[i].fov = (C.c_double * 2)(*c["fov"])
        ca[i].npix = (C.c_int32 * 2)(*c["npix"])
    keep.append(ca)
    d = LaunchDesc()
    d.n_sources = len(srcs)
    d.sources = sa
    d.n_cameras = len(cams)
    d.cameras = ca
    d.seed = int(run.get("seed", 0)) & 0xffffffff
    d.stream = int(run.get("stream", 0)) & 0xffffffff
    d.precision = PRECISION[precision]
    d.accumulate = int(kw.get("accumulate", 0))
    d.pid_begin = int(run.get("pid_begin", 0))
    d.pid_end = int(run.get("pid_end", 0))
    d.roulette_threshold = float(run.get("roulette_threshold", 1e-4))
    d.roulette_survival = float(run.get("roulette_survival", 0.1))
    d.max_events = int(run.get("max_events", 100000))
    d.max_trials = int(run.get("max_trials", 1000))
    d.block_size = int(kw.get("block_size", 0))
    d.blocks_per_sm = int(kw.get("blocks_per_sm", 0))
    d.time_budget_s = float(kw.get("time_budget_s", 0.0))
    d.optics = OPTICS[kw.get("optics", "tables")]
    d.flags = (FLAG_INLINE_TALLY if kw.get("inline_tally", False) else 0) | \
        (FLAG_MMA_SYNC_TALLY if kw.get("tally_engine", "tcgen05") == "mma" else 0)
    d.tally_blocks_per_sm = int(kw.get("tally_blocks_per_sm", 0))
    if trace is not None:
        p, k = _ptr(trace, np.float64)
        keep.append(k)
        d.trace = p
        d.n_trace = int(n_trace)
    return d, keep


def launch(models, run: dict, precision="fp32", trace=None, n_trace=0, sync=True, raise_on_cap=True, **kw):
    """mcrt_launch_packets over one or more Model objects; returns the stats dict
    (with key ``status`` = returned mcrt_status)."""
    L = lib()
    if isinstance(models, Model):
        models = [models]
    arr = (C.c_void_p * len(models))(*[m.h for m in models])
    d, keep = make_desc(run, precision, trace, n_trace, default_center=models[0].center, **kw)
    st = Stats()
    status = L.mcrt_launch_packets(arr, len(models), C.byref(d), C.byref(st) if sync else None)
    if status not in (MCRT_OK, MCRT_E_EVENT_CAP, MCRT_E_TIMEOUT) or (raise_on_cap and status == MCRT_E_EVENT_CAP):
        _check(status, None if len(models) > 1 else models[0].h)
    out = {f: getattr(st, f) for f in STAT_FIELDS}
    out["status"] = status
    del keep
    return out


def unit_eval(fn: int, inputs, precision="fp32"):
    """mcrt_unit_eval: evaluate a device building block on host inputs."""
    L = lib()
    widths_out = [4, 8, 6, 4, 4, 4, 4, 4]
    a = np.ascontiguousarray(np.asarray(inputs, dtype=np.float64))
    n = a.shape[0]
    out = np.zeros((n, widths_out[fn]))
    _check(L.mcrt_unit_eval(int(fn), PRECISION[precision], n, C.c_void_p(a.ctypes.data), C.c_void_p(out.ctypes.data)))
    return out


def launch_noalloc(model_dev: dict, run: dict, source, absorbed, precision="fp32", trace=None, n_trace=0,
                   stream=None, **kw):
    """mcrt_launch_packets_noalloc: transport with caller-owned device buffers only.

    ``model_dev`` holds CUDA tensors (kappa_abs, kappa_sca, optional bfield, and the
    optics tensors under "optics") plus "lo"/"hi"; ``source`` and ``absorbed`` are
    CUDA float64 tensors the call writes.  Returns the stats dict."""
    L = lib()
    ka = model_dev["kappa_abs"]
    nz, ny, nx = tuple(ka.shape)
    pr = NoAllocProblem()
    pr.nx, pr.ny, pr.nz = nx, ny, nz
    pr.lo = (C.c_double * 3)(*model_dev["lo"])
    pr.hi = (C.c_double * 3)(*model_dev["hi"])
    pr.kappa_abs = ka.data_ptr()
    pr.kappa_sca = model_dev["kappa_sca"].data_ptr()
    pr.bfield = model_dev["bfield"].data_ptr() if model_dev.get("bfield") is not None else None
    opt = model_dev["optics"]
    pr.model = SCAT[opt["model"]]
    if pr.model == 1:
        pr.n_bins, pr.n_theta = opt["mueller"].shape[0], opt["mueller"].shape[1]
        pr.mueller = opt["mueller"].data_ptr()
        pr.bin_weight = opt["bin_weight"].data_ptr()
    pr.n_ktheta = opt["kext"].shape[0]
    pr.kext = opt["kext"].data_ptr()
    pr.source = source.data_ptr() if source is not None else None
    pr.absorbed = absorbed.data_ptr()
    pr.cuda_stream = _stream_handle(stream)
    center = tuple((float(a) + float(b)) / 2 for a, b in zip(model_dev["lo"], model_dev["hi"]))
    d, keep = make_desc(run, precision, trace, n_trace, default_center=center, **kw)
    st = Stats()
    status = L.mcrt_launch_packets_noalloc(C.byref(pr), C.byref(d), C.byref(st))
    if status not in (MCRT_OK, MCRT_E_EVENT_CAP, MCRT_E_TIMEOUT):
        _check(status)
    out = {f: getattr(st, f) for f in STAT_FIELDS}
    out["status"] = status
    del keep
    return out


class Batch:
    """mcrt_batch_*: many models in one persistent launch captured in a CUDA graph."""

    def __init__(self, models, run: dict, precision="fp32", **kw):
        L = lib()
        self.models = list(models)
        self.run = run
        arr = (C.c_void_p * len(self.models))(*[mm.h for mm in self.models])
        d, self._keep = make_desc(run, precision, default_center=self.models[0].center, **kw)
        h = C.c_void_p()
        _check(L.mcrt_batch_create(C.byref(h), arr, len(self.models), C.byref(d)))
        self.h = h
        cams = run.get("cameras", [])
        self.image_shape = [(4, c["npix"][1], c["npix"][0]) for c in cams]

    def tune(self, packets_per_job):
        rep = TuneReport()
        _check(lib().mcrt_batch_tune(self.h, int(packets_per_job), C.byref(rep)))
        rows = [{"block_size": rep.block_size[i], "blocks_per_sm": rep.blocks_per_sm[i],
                 "interleave": rep.interleave[i], "events_per_s": rep.events_per_s[i]} for i in range(rep.n)]
        return {"trials": rows, "best": rep.best}

    def launch(self, seed):
        st = Stats()
        status = lib().mcrt_batch_run(self.h, int(seed) & 0xffffffff, C.byref(st))
        if status not in (MCRT_OK, MCRT_E_EVENT_CAP, MCRT_E_TIMEOUT):
            _check(status)
        out = {f: getattr(st, f) for f in STAT_FIELDS}
        out["status"] = status
        return out

    def images(self, out=None):
        """All images, [model][camera] -> array [4][ny][nx]."""
        n = sum(int(np.prod(s)) for s in self.image_shape) * len(self.models)
        flat = np.zeros(n) if out is None else out
        p, keep = _ptr(flat, np.float64)
        _check(lib().mcrt_batch_images(self.h, p))
        if out is not None:
            return out
        res, off = [], 0
        for _ in self.models:
            row = []
            for s in self.image_shape:
                k = int(np.prod(s))
                row.append(flat[off:off + k].reshape(s))
                off += k
            res.append(row)
        return res

    def close(self):
        if getattr(self, "h", None):
            lib().mcrt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """mcrt_surrogate_*: the MLP surrogate of the grain optics (GPU training and
    evaluation; marshalling only)."""

    N_IN, N_OUT = 7, 20
    LAYERS = [(16, 128), (128, 128), (128, 128), (128, 128), (128, 24)]

    def __init__(self, model: "Model", seed=3):
        h = C.c_void_p()
        _check(lib().mcrt_surrogate_create(C.byref(h), model.h, int(seed) & 0xffffffff))
        self.h = h
        self.n_params = int(lib().mcrt_surrogate_param_count())

    def train(self, n_steps, batch=8192, lr=2e-3):
        hist = np.zeros(max(1, int(n_steps)))
        _check(lib().mcrt_surrogate_train(self.h, int(n_steps), int(batch), float(lr),
                                          C.c_void_p(hist.ctypes.data)))
        return hist[:int(n_steps)]

    ENGINES = {"mma": 0, "tcgen05": 1}

    def eval(self, inputs, engine="mma"):
        """Network outputs [n][20]; engine "mma" (mma.sync) or "tcgen05"."""
        x = np.ascontiguousarray(np.asarray(inputs, dtype=np.float32))
        out = np.zeros((x.shape[0], self.N_OUT), dtype=np.float32)
        _check(lib().mcrt_surrogate_eval_engine(self.h, self.ENGINES[engine], x.shape[0], C.c_void_p(x.ctypes.data),
                                                C.c_void_p(out.ctypes.data)))
        return out

    def labels(self, inputs):
        x = np.ascontiguousarray(np.asarray(inputs, dtype=np.float32))
        out = np.zeros((x.shape[0], self.N_OUT), dtype=np.float32)
        _check(lib().mcrt_surrogate_labels(self.h, x.shape[0], C.c_void_p(x.ctypes.data),
                                           C.c_void_p(out.ctypes.data)))
        return out

    def grad(self, inputs, targets, loss_weights=None, precision="bf16"):
        """Loss and per-layer gradients (mcrt_surrogate_grad; precision "fp32":
        mcrt_surrogate_grad_fp32)."""
        fn = lib().mcrt_surrogate_grad_fp32 if precision == "fp32" else lib().mcrt_surrogate_grad
        x = np.ascontiguousarray(np.asarray(inputs, dtype=np.float32))
        t = np.ascontiguousarray(np.asarray(targets, dtype=np.float32))
        w = None if loss_weights is None else np.ascontiguousarray(np.asarray(loss_weights, dtype=np.float32))
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_double()
        _check(fn(self.h, x.shape[0], C.c_void_p(x.ctypes.data), C.c_void_p(t.ctypes.data),
                  C.c_void_p(w.ctypes.data) if w is not None else None, C.c_void_p(g.ctypes.data), C.byref(loss)))
        return loss.value, self.unflatten(g)

    def error_map(self, n_samples=1 << 22):
        """mcrt_surrogate_error_map: largest error per (cos theta_i, cos theta_s,
        delta phi, s) cell, shape (8, 8, 8, 8)."""
        m = np.zeros(4096, dtype=np.float32)
        _check(lib().mcrt_surrogate_error_map(self.h, int(n_samples), C.c_void_p(m.ctypes.data)))
        return m.reshape(8, 8, 8, 8)

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        _check(lib().mcrt_surrogate_params(self.h, C.c_void_p(p.ctypes.data), 0))
        return self.unflatten(p)

    def set_params(self, layers):
        p = np.ascontiguousarray(self.flatten(layers), dtype=np.float32)
        _check(lib().mcrt_surrogate_params(self.h, C.c_void_p(p.ctypes.data), 1))

    def unflatten(self, p):
        out, off = [], 0
        for ni, no in self.LAYERS:
            W = np.asarray(p[off:off + no * ni]).reshape(no, ni)
            off += no * ni
            b = np.asarray(p[off:off + no])
            off += no
            out.append((W, b))
        return out

    def flatten(self, layers):
        return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])

    def close(self):
        if getattr(self, "h", None):
            lib().mcrt_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
