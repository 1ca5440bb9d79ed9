"""ctypes front end of the FP64 CPU oracle (``mcrt_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.

The problem is passed as plain numpy arrays and dicts; the dict keys follow the
fields of ``orc_problem`` in the C file.  Every function here only marshals
arguments: the arithmetic is in the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcrt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, plain C11, FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Source(C.Structure):
    _fields_ = [("type", C.c_int32), ("beam_dir", C.c_int32), ("luminosity", C.c_double),
                ("pos", C.c_double * 3), ("n_packets", C.c_int64)]


class Camera(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("center", C.c_double * 3), ("fov", C.c_double * 2),
                ("npix", C.c_int32 * 2)]


_f32p = C.POINTER(C.c_float)
_f64p = C.POINTER(C.c_double)


class Patch(C.Structure):
    _fields_ = [("box", C.c_int32 * 6), ("factor", C.c_int32), ("kappa_abs", _f32p), ("kappa_sca", _f32p),
                ("bfield", _f32p), ("emissivity", _f32p)]


class Problem(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("kappa_abs", _f32p), ("kappa_sca", _f32p), ("bfield", _f32p), ("emissivity", _f32p),
                ("scat_model", C.c_int32), ("n_bins", C.c_int32), ("n_theta", C.c_int32),
                ("mueller", _f32p), ("bin_weight", _f32p), ("n_ktheta", C.c_int32), ("kext", _f32p),
                ("n_sources", C.c_int32), ("sources", C.POINTER(Source)),
                ("n_cam", C.c_int32), ("cams", C.POINTER(Camera)),
                ("seed", C.c_uint32), ("stream", C.c_uint32),
                ("pid_begin", C.c_int64), ("pid_end", C.c_int64),
                ("roulette_threshold", C.c_double), ("roulette_survival", C.c_double),
                ("max_events", C.c_int64), ("max_trials", C.c_int32), ("n_threads", C.c_int32),
                ("n_trace", C.c_int64), ("periodic", C.c_int32),
                ("eps_re", C.c_double), ("eps_im", C.c_double), ("aspect", C.c_double), ("size_x", C.c_double),
                ("n_patches", C.c_int32), ("patches", C.POINTER(Patch))]


class Result(C.Structure):
    _fields_ = [("S", _f64p), ("absorbed", _f64p), ("trace", _f64p), ("stats", C.c_double * 16)]


STAT_NAMES = ["emitted_energy", "escaped_energy", "absorbed_energy", "roulette_lost", "roulette_gain",
              "cap_lost", "events", "segments", "scatterings", "emitted", "escaped", "roulette_killed",
              "cap_hits", "trials", "status", "loop_seconds"]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.orc_philox.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = C.c_double
            L.orc_grain_quaternion.argtypes = [C.c_double, C.c_double, C.c_double, _f64p]
            L.orc_to_grain.argtypes = [_f64p, _f64p, _f64p]
            L.orc_to_lab.argtypes = [_f64p, _f64p, _f64p]
            L.orc_stokes_basis.argtypes = [_f64p, _f64p, _f64p]
            L.orc_change_basis.argtypes = [_f64p] * 6
            L.orc_cell_solution.argtypes = [_f64p, C.c_double, C.c_double, C.c_double, _f64p, C.c_double, _f64p]
            L.orc_attenuate.argtypes = [_f64p, C.c_double, C.c_double, C.c_double, C.c_double, _f64p]
            L.orc_segment_integral.argtypes = [_f64p, C.c_double, C.c_double, C.c_double, C.c_double, _f64p]
            L.orc_rayleigh.argtypes = [C.c_double, _f64p]
            L.orc_mueller_apply.argtypes = [_f64p, _f64p, _f64p, _f64p, _f64p]
            L.orc_grain_meridian.argtypes = [_f64p, _f64p, _f64p, _f64p, _f64p]
            L.orc_dda_walk.argtypes = [C.POINTER(C.c_int32), _f64p, _f64p, _f64p, _f64p, C.c_int64,
                                       C.POINTER(C.c_int64), _f64p]
            L.orc_dda_walk.restype = C.c_int64
            L.orc_transport.argtypes = [C.POINTER(Problem), C.POINTER(Result)]
            L.orc_transport.restype = C.c_int
            L.orc_image.argtypes = [C.POINTER(Problem), _f64p, C.c_int, C.c_double, _f64p]
            L.orc_image.restype = C.c_int
            L.orc_thermal_luminosity.argtypes = [C.POINTER(Problem)]
            L.orc_thermal_luminosity.restype = C.c_double
            L.orc_emit.argtypes = [C.POINTER(Problem), C.c_int64, _f64p]
            L.orc_emit.restype = C.c_int
            L.orc_scatter.argtypes = [C.POINTER(Problem), C.c_int64, C.c_uint32, C.c_int, _f64p, _f64p, _f64p,
                                      _f64p]
            L.orc_scatter.restype = C.c_int
            L.orc_frame.argtypes = [C.POINTER(Problem), C.c_int64, _f64p, _f64p]
            L.orc_n_cells.argtypes = [C.POINTER(Problem)]
            L.orc_n_cells.restype = C.c_int64
            L.orc_dda_walk_composite.argtypes = [C.POINTER(Problem), _f64p, _f64p, C.c_int64,
                                                 C.POINTER(C.c_int64), _f64p]
            L.orc_dda_walk_composite.restype = C.c_int64
            L.orc_spheroid_L.argtypes = [C.c_double]
            L.orc_spheroid_L.restype = C.c_double
            L.orc_dipole_constants.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _f64p]
            L.orc_dipole_scatter.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double] + [_f64p] * 5
    return _lib


def _d(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.shape, n)
    return a


def _pd(a):
    return a.ctypes.data_as(_f64p)


# ----------------------------------------------------------------------------------
# unit functions
# ----------------------------------------------------------------------------------
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return [int(x) for x in o]


def uniform(x):
    return lib().orc_uniform(int(x) & 0xffffffff)


def grain_quaternion(b):
    q = np.zeros(4)
    lib().orc_grain_quaternion(float(b[0]), float(b[1]), float(b[2]), _pd(q))
    return q


def to_grain(q, v):
    q, v, o = _d(q, 4), _d(v, 3), np.zeros(3)
    lib().orc_to_grain(_pd(q), _pd(v), _pd(o))
    return o


def to_lab(q, v):
    q, v, o = _d(q, 4), _d(v, 3), np.zeros(3)
    lib().orc_to_lab(_pd(q), _pd(v), _pd(o))
    return o


def stokes_basis(n):
    n, th, ph = _d(n, 3), np.zeros(3), np.zeros(3)
    lib().orc_stokes_basis(_pd(n), _pd(th), _pd(ph))
    return th, ph


def change_basis(X, a1, a2, b1, b2):
    X, a1, a2, b1, b2 = _d(X, 4), _d(a1, 3), _d(a2, 3), _d(b1, 3), _d(b2, 3)
    o = np.zeros(4)
    lib().orc_change_basis(_pd(X), _pd(a1), _pd(a2), _pd(b1), _pd(b2), _pd(o))
    return o


def cell_solution(X0, alpha, S, dtau):
    X0, S, o = _d(X0, 4), _d(S, 4), np.zeros(4)
    lib().orc_cell_solution(_pd(X0), float(alpha[0]), float(alpha[1]), float(alpha[2]), _pd(S), float(dtau), _pd(o))
    return o


def attenuate(X0, a, alpha2, alpha3, dtau):
    X0, o = _d(X0, 4), np.zeros(4)
    lib().orc_attenuate(_pd(X0), float(a), float(alpha2), float(alpha3), float(dtau), _pd(o))
    return o


def segment_integral(X0, a, alpha2, alpha3, dtau):
    X0, o = _d(X0, 4), np.zeros(4)
    lib().orc_segment_integral(_pd(X0), float(a), float(alpha2), float(alpha3), float(dtau), _pd(o))
    return o


def rayleigh(mu):
    o = np.zeros(6)
    lib().orc_rayleigh(float(mu), _pd(o))
    return o


def mueller_apply(X, n, n2, Z):
    X, n, n2, Z, o = _d(X, 4), _d(n, 3), _d(n2, 3), _d(Z, 6), np.zeros(4)
    lib().orc_mueller_apply(_pd(X), _pd(n), _pd(n2), _pd(Z), _pd(o))
    return o


def grain_meridian(q, n):
    q, n = _d(q, 4), _d(n, 3)
    gth, gph, tp = np.zeros(3), np.zeros(3), np.zeros(1)
    lib().orc_grain_meridian(_pd(q), _pd(n), _pd(gth), _pd(gph), _pd(tp))
    return gth, gph, float(tp[0])


DIPOLE_KEYS = ["L0", "L1", "al0_re", "al0_im", "al1_re", "al1_im", "q_ext0", "q_ext1", "q_sca0", "q_sca1",
               "q_abs0", "q_abs1", "rho_re", "rho_im", "zn", "env"]


def spheroid_L(s):
    return lib().orc_spheroid_L(float(s))


def dipole_constants(eps, aspect, x):
    """Per-grain constants of the aligned dipole spheroid (index 0: a principal axis
    perpendicular to the symmetry axis, 1: the symmetry axis)."""
    o = np.zeros(16)
    eps = complex(eps)
    lib().orc_dipole_constants(eps.real, eps.imag, float(aspect), float(x), _pd(o))
    return dict(zip(DIPOLE_KEYS, o.tolist()))


def dipole_scatter(eps, aspect, x, axis, X, n, n2):
    """Z X (1/sr) for the scattering n -> n2 by a spheroid with symmetry axis `axis`."""
    eps = complex(eps)
    axis, X, n, n2, o = _d(axis, 3), _d(X, 4), _d(n, 3), _d(n2, 3), np.zeros(4)
    lib().orc_dipole_scatter(eps.real, eps.imag, float(aspect), float(x), _pd(axis), _pd(X), _pd(n), _pd(n2), _pd(o))
    return o


def frame(model, cell, n):
    """Local frame of `cell` (flat index) for direction n: dict with alpha (K per unit
    kappa_ext, grain-meridian basis), sca (s11, s12), gsca, thetap, gth, gph."""
    keep = make_problem(model, {"sources": [], "cameras": []})
    o, n = np.zeros(13), _d(n, 3)
    lib().orc_frame(C.byref(keep.P), int(cell), _pd(n), _pd(o))
    return {"alpha": o[0:3].copy(), "sca": o[3:5].copy(), "gsca": float(o[5]), "thetap": float(o[6]),
            "gth": o[7:10].copy(), "gph": o[10:13].copy()}


def dda_walk(shape_xyz, lo, hi, p0, n, max_cells=100000):
    n3 = (C.c_int32 * 3)(*shape_xyz)
    lo, hi, p0, n = _d(lo, 3), _d(hi, 3), _d(p0, 3), _d(n, 3)
    cells = np.zeros(max_cells, dtype=np.int64)
    lens = np.zeros(max_cells)
    k = lib().orc_dda_walk(n3, _pd(lo), _pd(hi), _pd(p0), _pd(n), max_cells,
                           cells.ctypes.data_as(C.POINTER(C.c_int64)), _pd(lens))
    return cells[:k].copy(), lens[:k].copy()


# ----------------------------------------------------------------------------------
# transport and imaging
# ----------------------------------------------------------------------------------
class _Keep:
    """Holds the numpy buffers a Problem points into."""


def make_problem(model: dict, run: dict):
    """Build the C problem from a model dict (grid and optics, see
    ``paper_2512_01283_gb300.workloads``) and a run dict (sources, cameras, seed...)."""
    keep = _Keep()
    P = Problem()
    nz, ny, nx = model["kappa_abs"].shape
    P.n = (C.c_int32 * 3)(nx, ny, nz)
    P.lo = (C.c_double * 3)(*model["lo"])
    P.hi = (C.c_double * 3)(*model["hi"])

    def f32(name, arr):
        if arr is None:
            return None
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float32))
        setattr(keep, name, a)
        return a.ctypes.data_as(_f32p)

    P.kappa_abs = f32("ka", model["kappa_abs"])
    P.kappa_sca = f32("ks", model["kappa_sca"])
    P.bfield = f32("bf", model.get("bfield"))
    P.emissivity = f32("em", model.get("emissivity"))
    optics = model["optics"]
    P.scat_model = {"rayleigh": 0, "table": 1, "dipole": 2}[optics["model"]]
    if P.scat_model == 2:
        eps = complex(optics["eps"])
        P.eps_re, P.eps_im = eps.real, eps.imag
        P.aspect = float(optics["aspect"])
        P.size_x = float(optics["x"])
    if P.scat_model == 1:
        mu = np.asarray(optics["mueller"], dtype=np.float32)
        P.n_bins, P.n_theta = mu.shape[0], mu.shape[1]
        P.mueller = f32("mu", mu)
        P.bin_weight = f32("bw", optics["bin_weight"])
    if P.scat_model != 2:  # the dipole spheroid computes its own K
        kx = np.asarray(optics["kext"], dtype=np.float32)
        P.n_ktheta = kx.shape[0]
        P.kext = f32("kx", kx)
    srcs = run["sources"]
    arr = (Source * max(1, len(srcs)))()
    for i, s in enumerate(srcs):
        arr[i].type = {"point": 0, "beam": 1, "thermal": 2}[s["type"]]
        arr[i].beam_dir = int(s.get("beam_dir", 1))
        arr[i].luminosity = float(s.get("luminosity", 1.0))
        arr[i].pos = (C.c_double * 3)(*s.get("pos", (0.0, 0.0, 0.0)))
        arr[i].n_packets = int(s["n_packets"])
    keep.src = arr
    P.n_sources = len(srcs)
    P.sources = arr
    cams = run.get("cameras", [])
    carr = (Camera * max(1, len(cams)))()
    for i, c in enumerate(cams):
        carr[i].dir = (C.c_double * 3)(*c["dir"])
        carr[i].center = (C.c_double * 3)(*c.get("center", [(a + b) / 2 for a, b in zip(model["lo"], model["hi"])]))
        carr[i].fov = (C.c_double * 2)(*c["fov"])
        carr[i].npix = (C.c_int32 * 2)(*c["npix"])
    keep.cams = carr
    P.n_cam = len(cams)
    P.cams = carr
    P.seed = int(run.get("seed", 0)) & 0xffffffff
    P.stream = int(run.get("stream", 0)) & 0xffffffff
    total = sum(int(s["n_packets"]) for s in srcs)
    P.pid_begin = int(run.get("pid_begin", 0))
    P.pid_end = int(run.get("pid_end", total))
    P.roulette_threshold = float(run.get("roulette_threshold", 1e-4))
    P.roulette_survival = float(run.get("roulette_survival", 0.1))
    P.max_events = int(run.get("max_events", 100000))
    P.max_trials = int(run.get("max_trials", 1000))
    P.n_threads = int(run.get("n_threads", 1))
    P.n_trace = int(run.get("n_trace", 0))
    P.periodic = int(model.get("periodic", 0))  # bit a: axis a periodic
    patches = model.get("refine", [])
    parr = (Patch * max(1, len(patches)))()
    for i, q in enumerate(patches):
        parr[i].box = (C.c_int32 * 6)(*q["box"])
        parr[i].factor = int(q["factor"])
        parr[i].kappa_abs = f32("pka%d" % i, q["kappa_abs"])
        parr[i].kappa_sca = f32("pks%d" % i, q["kappa_sca"])
        parr[i].bfield = f32("pbf%d" % i, q.get("bfield"))
        parr[i].emissivity = f32("pem%d" % i, q.get("emissivity"))
    keep.patches = parr
    P.n_patches = len(patches)
    P.patches = parr
    keep.P = P
    return keep


def n_cells(model: dict) -> int:
    """Cells of the composite grid: the root's, then each refined patch's."""
    keep = make_problem(model, {"sources": [], "cameras": []})
    return int(lib().orc_n_cells(C.byref(keep.P)))


def dda_walk_composite(model: dict, p0, n, max_cells=100000):
    """Composite cells and chord lengths along a ray through a refined grid."""
    keep = make_problem(model, {"sources": [], "cameras": []})
    p0, n = _d(p0, 3), _d(n, 3)
    cells = np.zeros(max_cells, dtype=np.int64)
    lens = np.zeros(max_cells)
    k = lib().orc_dda_walk_composite(C.byref(keep.P), _pd(p0), _pd(n), max_cells,
                                     cells.ctypes.data_as(C.POINTER(C.c_int64)), _pd(lens))
    return cells[:k].copy(), lens[:k].copy()


def transport(model: dict, run: dict, S_out=None, absorbed_out=None):
    """Step 1 (Sec. 2.2, 2.3).  Returns dict with S [ncell][n_cam][4], absorbed
    [ncell], trace [n_trace][16] and stats.  S_out / absorbed_out: FP64 buffers of
    those shapes to add the tallies to instead of fresh zeroed ones (a timing loop
    reuses them, so that first-touch page faults stay out of the packet loop)."""
    keep = make_problem(model, run)
    P = keep.P
    ncell = int(lib().orc_n_cells(C.byref(P)))
    S = np.zeros((ncell, max(1, P.n_cam), 4)) if S_out is None else S_out
    absorbed = np.zeros(ncell) if absorbed_out is None else absorbed_out
    for a, shape in ((S, (ncell, max(1, P.n_cam), 4)), (absorbed, (ncell,))):
        if a.shape != shape or a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("tally buffer of shape %s, contiguous float64, expected" % (shape,))
    trace = np.zeros((max(1, P.n_trace), 16))
    R = Result()
    R.S = _pd(S)
    R.absorbed = _pd(absorbed)
    R.trace = _pd(trace) if P.n_trace > 0 else None
    rc = lib().orc_transport(C.byref(P), C.byref(R))
    if rc != 0:
        raise RuntimeError("oracle transport failed: %d" % rc)
    stats = {k: R.stats[i] for i, k in enumerate(STAT_NAMES)}
    return {"S": S[:, :P.n_cam], "absorbed": absorbed, "trace": trace[:P.n_trace], "stats": stats}


def image(model: dict, run: dict, S, cam: int, scale_S: float = 1.0):
    """Step 2 (Sec. 2.3, App. A): Stokes image [4][ny][nx] of camera ``cam``."""
    keep = make_problem(model, run)
    P = keep.P
    c = run["cameras"][cam]
    nx, ny = c["npix"]
    out = np.zeros((4, ny, nx))
    Sarr = None
    if S is not None:
        Sarr = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
        assert Sarr.shape[1] == P.n_cam
    rc = lib().orc_image(C.byref(P), _pd(Sarr) if Sarr is not None else None, int(cam), float(scale_S), _pd(out))
    if rc != 0:
        raise RuntimeError("oracle image failed: %d" % rc)
    return out


def thermal_luminosity(model: dict, run: dict) -> float:
    keep = make_problem(model, run)
    return lib().orc_thermal_luminosity(C.byref(keep.P))


def emit(model: dict, run: dict, pids):
    """Birth of each packet id: rows [x,y,z, nx,ny,nz, I,Q,U,V, tau, inside, source]."""
    keep = make_problem(model, run)
    out = np.zeros((len(pids), 13))
    for i, pid in enumerate(pids):
        rc = lib().orc_emit(C.byref(keep.P), int(pid), _pd(out[i]))
        if rc != 0:
            raise RuntimeError("oracle emit failed: %d" % rc)
    return out


def scatter(model: dict, run: dict, pid, n_sca, bin_index, X, n, q=(1.0, 0.0, 0.0, 0.0)):
    """One scattering draw: (trials, new direction, scattered Stokes)."""
    keep = make_problem(model, run)
    X, n, q, out = _d(X, 4), _d(n, 3), _d(q, 4), np.zeros(7)
    t = lib().orc_scatter(C.byref(keep.P), int(pid), int(n_sca), int(bin_index), _pd(X), _pd(n), _pd(q), _pd(out))
    return t, out[:3].copy(), out[3:].copy()
