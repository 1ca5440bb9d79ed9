#!/usr/bin/env python
"""Throughput of the polarized Monte-Carlo transport + two-step imaging on one GB300.

Workload (default): flared protoplanetary disk on a 192^3 grid, 8 grain-size bins of
tabulated scattering matrices (181 angles), aligned grains (toroidal + poloidal field,
30 deg pitch), star plus thermal emission, 1e8 packets per step, 8 cameras at 256^2.
A step = step 1 (all packets emitted, transported, tallied) + step 2 (all 8 images).
Metric: packet-events/s (emission + cell segments + scatterings), inputs resident in
HBM.  Synthetic seeded inputs (paper_2512_01283_gb300.workloads).

``--impl reference`` times the FP64 CPU oracle on bounded samples of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "packet-events/s on 1 GB300 at fixed Stokes-map error; surrogate vs table path"
UNIT = "packet-events/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--packets", type=float, default=1e8)
    ap.add_argument("--grid", type=int, default=192)
    ap.add_argument("--cpu-chunks", type=int, default=CPU_CHUNKS, help="chunks of packet ids in the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--sweep-packets", type=float, default=1e7, help="packets per job of the batched sweep")
    ap.add_argument("--sweep-runs", type=int, default=1, help="timed graph replays of the batched sweep")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-plane-parallel", action="store_true")
    ap.add_argument("--no-spheroids", action="store_true", help="skip the aligned-spheroid line")
    ap.add_argument("--no-refined", action="store_true", help="skip the static-mesh-refinement line")
    ap.add_argument("--no-microbench", action="store_true", help="skip the FP64 reduction microbenchmark")
    ap.add_argument("--inline-tally", action="store_true",
                    help="table path: tally inside the transport kernel instead of a tally kernel per round")
    ap.add_argument("--tally-bps", type=int, default=0,
                    help="table rounds: > 0 overlaps each tally (this many blocks per SM) with the next transport")
    ap.add_argument("--transport-bps", type=int, default=0, help="table rounds: transport blocks per SM (0: auto)")
    ap.add_argument("--sur-steps", type=int, default=1, help="timed launches of the surrogate path")
    ap.add_argument("--sur-train-samples", type=float, default=2e7, help="training samples of the network")
    ap.add_argument("--sur-bound", type=float, default=0.05, help="error-map bound of the table fallback")
    ap.add_argument("--fixed-error-measured", action="store_true",
                    help="surrogate line: run both paths to a fixed map error against a 10-launch table reference")
    return ap.parse_args()


def workload_config(args):
    return {"workload": "flared disk %d^3, 8 grain-size bins (181-angle scattering tables), aligned grains, "
                        "star + thermal emission, %.0e packets, 8 cameras at 256^2" % (args.grid, args.packets),
            "grid": args.grid, "packets_per_step": int(args.packets), "n_cameras": 8, "npix": 256,
            "precision": "fp32 per-step transport math, fp64 optical-depth sum and tallies",
            "l2": "no flush: the source tally (1.81 GB) and grid (226 MB) exceed the 129 MB L2"}


CPU_CHUNK = 8192  # packet ids per source half in one chunk of the oracle baseline
CPU_CHUNKS = 48   # chunks of the GPU arm's baseline (about 13 s of loop time); the reference arm cycles through them


def oracle_sample(model, run, chunks, n_threads, bufs=None):
    """The FP64 oracle on chunks of the workload's packet ids: chunk c is ids
    [c * CPU_CHUNK, (c + 1) * CPU_CHUNK) of the star half and the same offsets into
    the thermal half, each half one oracle call over all host threads.  The time is the
    packet loops' alone, measured inside the oracle: its per-call set-up (problem
    marshalling, the thermal emission CDF over all cells) is excluded, and the tally
    buffers are allocated and touched once beforehand.  Returns (events, seconds,
    packets, bufs)."""
    from oracle import oracle as O

    if bufs is None:
        ncell = O.n_cells(model)
        bufs = (np.zeros((ncell, max(1, len(run["cameras"])), 4)), np.zeros(ncell))
        for b in bufs:
            b.fill(0.0)
    n_star = run["sources"][0]["n_packets"]
    events = wall = 0.0
    packets = 0
    for c in chunks:
        for base in (c * CPU_CHUNK, n_star + c * CPU_CHUNK):
            out = O.transport(model, dict(run, pid_begin=base, pid_end=base + CPU_CHUNK, n_threads=n_threads),
                              S_out=bufs[0], absorbed_out=bufs[1])
            events += out["stats"]["events"]
            wall += out["stats"]["loop_seconds"]
            packets += CPU_CHUNK
    return events, wall, packets, bufs


def oracle_sample_text(chunks, packets, total):
    return ("chunks %s of %d star + %d thermal packet ids (chunk c: ids from c x %d in each half) of the "
            "%.0e-packet workload, %d packets; packet loops timed inside the oracle, its set-up excluded"
            % (chunks, CPU_CHUNK, CPU_CHUNK, CPU_CHUNK, total, packets))


KERNEL_SOURCES = ("paper_2512_01283_gb300/csrc/mcrt_transport.cu", "paper_2512_01283_gb300/csrc/mcrt_device.cuh",
                  "paper_2512_01283_gb300/csrc/mcrt_internal.h", "paper_2512_01283_gb300/csrc/mcrt_packet.cuh",
                  "paper_2512_01283_gb300/csrc/mcrt_wave.cu")


def code_only(text):
    """C++ source without its comments and blank space, so that a comment edit does not
    mark a profile of the same code as stale."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_sha(read=None):
    """Hash of the code (comments and blank space dropped) of the table-round kernels'
    sources; `read(path)` gives a file's text (default: the working tree)."""
    import hashlib

    read = read or (lambda f: open(os.path.join(ROOT, f), encoding="utf-8").read())
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(code_only(read(f)).encode())
    return h.hexdigest()[:16]


def profiled_fields():
    """The key: value lines of the committed ncu summary of the disk workload's table
    rounds, or {} when the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "rounds_disk192.md")
    if not os.path.exists(path):
        return {}
    fields = {}
    for line in open(path):
        if ":" in line and not line.startswith(("|", "#", "`")):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    return fields if fields.get("kernel_source_sha") == kernel_source_sha() else {}


def profiled_traffic(kernel, units_per_launch):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu summary of
    the disk workload: bytes per unit (segment of the transport kernel, record of the
    tally kernel) of the captured small launch times this launch's units; None when
    the kernel sources changed since the capture."""
    v = profiled_fields().get("%s_traffic_bytes_per_unit" % kernel)
    return None if v is None else float(v) * units_per_launch


def profiled_issue(kernel):
    """Issue utilisation of `kernel` in the same capture (duration-weighted over its
    launches): share of cycles an instruction issued, and active threads per warp
    instruction; None when the kernel sources changed since the capture."""
    f = profiled_fields()
    a, t = f.get("%s_issue_active_pct" % kernel), f.get("%s_threads_per_warp_instruction" % kernel)
    if a is None or t is None:
        return None
    return {"issue_active": float(a) / 100.0, "threads_per_warp_instruction": float(t), "source": "ncu"}


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", os.environ.get("LOCAL_RANK", "0")],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def run_sweep(args, M, W, torch, rank=0, world=1, dist=None):
    """Batched sweep: 32 clumpy models (edges 32..192) x 8 wavelengths = 256 jobs in one
    persistent launch replayed from a CUDA graph, schedule from the autotuner.  Over
    several ranks the jobs are split (rank r takes jobs r, r + world, ...), with no
    collective but the timing reduction: events summed, time the slowest rank's."""
    models = W.sweep_models()[rank::world]
    run = W.sweep_run(n_packets=int(args.sweep_packets))
    t0 = time.perf_counter()
    mdls = [M.Model(m) for m in models]
    batch = M.Batch(mdls, run, precision="fp32")
    tune = batch.tune(packets_per_job=max(1000, int(args.sweep_packets) // 100))
    setup_s = time.perf_counter() - t0
    # the tuner's trial launches ran the same kernels: no separate warm-up replay
    torch.cuda.synchronize()
    runs = []
    for s in range(args.sweep_runs):
        t1 = time.perf_counter()
        st = batch.launch(seed=11 + s)
        runs.append((st, time.perf_counter() - t1))
    ev = sum(r[0]["events"] for r in runs)
    wall = sum(r[1] for r in runs)
    kms = sum(r[0]["kernel_ms"] for r in runs)
    if world > 1:
        from paper_2512_01283_gb300 import multigpu as MG

        ms_max, ev = MG.reduce_timing(1e3 * wall, ev, dist, device="cuda")
        wall = 1e-3 * ms_max
        kms_max, _ = MG.reduce_timing(kms, 0.0, dist, device="cuda")
        kms = kms_max
    best = tune["trials"][tune["best"]]
    out = {"workload": "batched sweep: 32 models (edges 32..192, clumpy log-normal density, mean tau 1..100) x "
                       "8 wavelengths 0.5..3 um = 256 jobs, central star, one 128^2 camera each, %.0e packets "
                       "per job, one persistent launch replayed from a CUDA graph" % args.sweep_packets,
           "value": ev / wall, "unit": UNIT, "transport_events_per_s": ev / (kms * 1e-3),
           "events_per_run": ev / len(runs), "ms_per_run": 1e3 * wall / len(runs),
           "schedule": best, "tune_trials": len(tune["trials"]), "setup_s": setup_s,
           "scaling": "strong: the 256 jobs split over %d rank(s)" % world,
           "cells_total": int(sum(m["kappa_abs"].size for m in models))}
    batch.close()
    for m in mdls:
        m.close()
    return out


def run_plane_parallel(M, W, torch):
    """Plane-parallel atmosphere: 64 x 64 x 128 slab, periodic in x and y, vertical
    optical depth 10, albedo 0.9, aligned dichroic grains (field 30 deg from z, alpha2 =
    -0.05), central point source, 1e7 packets, FP32."""
    model = W.plane_parallel_slab(nxy=64, nz=128, tau=10.0, albedo=0.9, periodic=3, b_angle_deg=30.0, p=0.05)
    run = W.center_source_run(10_000_000, cameras=[W.camera((0.0, 0.0, 1.0), (64, 64), (1.0, 1.0)),
                                                    W.camera((0.5, 0.0, 0.866), (64, 64), (1.0, 1.0))])
    m = M.Model(model)
    M.launch(m, dict(run, seed=90), precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = M.launch(m, dict(run, seed=91), precision="fp32")
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    m.close()
    bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
    return {"workload": "plane-parallel slab 64x64x128, periodic x and y, tau 10, albedo 0.9, dichroic aligned grains, "
                        "central point source, 1e7 packets, 2 cameras",
            "value": st["events"] / wall, "unit": UNIT, "events": st["events"], "seconds": wall,
            "energy_balance_rel": abs(bal - st["emitted_energy"]) / st["emitted_energy"]}


def run_spheroids(M, W, torch):
    """Aligned oblate dipole spheroids (2:1, m = 2.30 + 0.0228 i, x = 0.3), the
    circumstellar scene of Sec. 3.5 at a benchmark size: uniform sphere on a 128^3
    grid, radial optical depth 1, albedo 0.5, field along z, central star, 1e7
    packets, cameras along x and z at 256^2, FP32."""
    model = W.spheroid_sphere(n=128, tau=1.0, albedo=0.5)
    run = {"sources": [{"type": "point", "pos": (0.0, 0.0, 0.0), "luminosity": 1.0, "n_packets": 10_000_000}],
           "cameras": [W.camera((1.0, 0.0, 0.0), (256, 256), (2.0, 2.0)), W.camera((0.0, 0.0, 1.0), (256, 256), (2.0, 2.0))],
           "roulette_threshold": 1e-4, "roulette_survival": 0.1}
    m = M.Model(model)
    M.launch(m, dict(run, seed=92), precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = M.launch(m, dict(run, seed=93), precision="fp32")
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    img = np.zeros((4, 256, 256))
    m.image(0, img)
    m.close()
    bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
    return {"workload": "aligned oblate dipole spheroids (2:1, m = 2.30+0.0228i, x = 0.3), uniform sphere 128^3, "
                        "tau 1, albedo 0.5, field along z, central star, 1e7 packets, 2 cameras at 256^2",
            "value": st["events"] / wall, "unit": UNIT, "events": st["events"], "seconds": wall,
            "scatterings": st["scatterings"], "trials_per_scattering": st["trials"] / max(1.0, st["scatterings"]),
            # zero in expectation (Monte-Carlo noise): the polarization-dependent scattering
            # weights change single packets' energy
            "energy_balance_rel": (bal - st["emitted_energy"]) / st["emitted_energy"],
            "image_x": {"I": float(img[0].sum()), "Q_over_I": float(img[1].sum() / img[0].sum()),
                        "V_over_I": float(img[3].sum() / img[0].sum())}}


def run_refined(M, W, torch):
    """Static mesh refinement: the flared disk on a 128^3 root grid with a 4x refined
    patch over the inner quarter in x, y and the middle eighth in z (1.05e6 patch cells,
    the fields at their own centres), star + thermal, 1e7 packets, 8 cameras at 256^2,
    FP32: in rounds with the tally kernel (the default, as on plain grids) and, for
    comparison, with the in-place tally."""
    model = W.disk_refined(n=128, factor=4)
    run = W.disk_run(n_packets=10_000_000)
    m = M.Model(model)
    out = {}
    for name, kw in (("rounds", {}), ("in_place", {"inline_tally": True})):
        M.launch(m, dict(run, seed=94), precision="fp32", **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = M.launch(m, dict(run, seed=95), precision="fp32", **kw)
        torch.cuda.synchronize()
        out[name] = (st, time.perf_counter() - t0)
    S, _ = m.tallies(len(run["cameras"]))
    m.close()
    st, wall = out["rounds"]
    nroot = 128 ** 3
    bal = st["escaped_energy"] + st["absorbed_energy"] + st["roulette_lost"] - st["roulette_gain"] + st["cap_lost"]
    return {"workload": "flared disk, 128^3 root grid + 4x refined inner patch (1.05e6 cells), star + thermal, "
                        "1e7 packets, 8 cameras at 256^2, table rounds (transport + tally kernel)",
            "value": st["events"] / wall, "unit": UNIT, "events": st["events"], "seconds": wall,
            "rounds": st["wave_iterations"], "kernel_ms": {"transport": st["ms_transport"], "tally": st["ms_tally"]},
            "in_place_tally_value": out["in_place"][0]["events"] / out["in_place"][1],
            "patch_tally_share": float(np.abs(S[nroot:]).sum() / max(np.abs(S).sum(), 1e-300)),
            "energy_balance_rel": abs(bal - st["emitted_energy"]) / st["emitted_energy"]}


def run_reduction_peaks(M):
    """Throughput of the FP64 reductions the tallies are made of (mcrt_microbench): scalar
    atomic adds and 256-byte bulk reduce-adds at spread positions, into 32 MB (inside the
    L2) and 8 GB (far beyond it).  For comparison with the tally kernel, the bulk rate is
    also given as read-modify-write bytes (2 x 256 B per row), the way its algorithmic
    bytes count the source rows."""
    out = {}
    for tag, nbytes in (("l2", 32 << 20), ("dram", 8 << 30)):
        n_red = 1 << 28
        ms = M.microbench(0, nbytes, n_red)
        out["f64_atomic_per_s_" + tag] = n_red / (ms * 1e-3)
        n_rows = 1 << 24
        ms = M.microbench(1, nbytes, n_rows)
        out["bulk_rows_per_s_" + tag] = n_rows / (ms * 1e-3)
        out["bulk_rmw_GBs_" + tag] = n_rows * 512.0 / (ms * 1e-3) / 1e9
    out["note"] = ("scalar atomics: 2^28 FP64 adds; bulk: 2^24 rows of 32 doubles (cp.reduce.async.bulk add.f64); "
                   "positions spread by a multiplicative hash")
    return out


def image_diff(a, b):
    """Relative L2 differences of Stokes image stacks [cam][4][ny][nx]: I, and
    (Q, U) against I; plus the largest relative difference of integrated I."""
    a, b = np.asarray(a), np.asarray(b)
    dI = np.sqrt(np.sum((a[:, 0] - b[:, 0]) ** 2, axis=(1, 2)) / np.sum(b[:, 0] ** 2, axis=(1, 2)))
    dP = np.sqrt(np.sum((a[:, 1:3] - b[:, 1:3]) ** 2, axis=(1, 2, 3)) / np.sum(b[:, 0] ** 2, axis=(1, 2)))
    tot = np.abs(a[:, 0].sum(axis=(1, 2)) - b[:, 0].sum(axis=(1, 2))) / b[:, 0].sum(axis=(1, 2))
    return {"I_rel_l2": float(dI.mean()), "QU_rel_l2": float(dP.mean()), "I_total_rel_max": float(tot.max())}


def map_d2(a, b, ref):
    """Mean over cameras of the squared L2 difference of the I maps and of the (Q, U)
    maps of two image stacks [cam][4][ny][nx], relative to the I maps of `ref`."""
    a, b, ref = np.asarray(a), np.asarray(b), np.asarray(ref)
    nI = np.sum(ref[:, 0] ** 2, axis=(1, 2))
    dI = np.sum((a[:, 0] - b[:, 0]) ** 2, axis=(1, 2)) / nI
    dP = np.sum((a[:, 1:3] - b[:, 1:3]) ** 2, axis=(1, 2, 3)) / nI
    return float(dI.mean()), float(dP.mean())


def fixed_error(t1, t2, s1, s2, packets, table_s, sur_s, targets=(0.01, 0.02, 0.05)):
    """Table and surrogate paths at a fixed map error.  From two seeds of each path at
    `packets` packets: the Monte-Carlo variance of a map, sigma^2 = d^2(seed 1, seed 2) / 2,
    for each path, and the surrogate's systematic difference from the table path,
    b^2 = d^2(s1, t1) - sigma_s^2 - sigma_t^2.  A path's error after N packets against the
    table method's expected map is then eps^2 = b^2 + sigma^2 packets / N, which gives the
    packets, and with each path's measured time per packet the seconds, to reach eps."""
    out = {"packets_per_run": packets, "seconds_per_run": {"table": table_s, "surrogate": sur_s}}
    for name, k in (("I", 0), ("QU", 1)):
        vt = map_d2(t1, t2, t1)[k] / 2.0
        vs = map_d2(s1, s2, t1)[k] / 2.0
        b2 = max(0.0, map_d2(s1, t1, t1)[k] - vs - vt)
        rows = []
        for eps in targets:
            nt = packets * vt / eps ** 2
            ns = packets * vs / (eps ** 2 - b2) if eps ** 2 > b2 else None
            st = nt / packets * table_s
            ss = ns / packets * sur_s if ns is not None else None
            rows.append({"eps": eps, "table_packets": nt, "table_s": st, "surrogate_packets": ns, "surrogate_s": ss,
                         "table_over_surrogate_time": st / ss if ss else None})
        out[name] = {"sigma_table": vt ** 0.5, "sigma_surrogate": vs ** 0.5, "bias_surrogate": b2 ** 0.5,
                     "targets": rows}
    return out


def fixed_error_measured(M, torch, mdl_t, mdl_s, run, n_cam, npix, n_ref=10, targets=(0.05, 0.03), n_max=1.6e8):
    """Both paths run to a fixed map error, measured: a reference of n_ref table launches
    of the run's packets (seeds 7000 + k, 10^9 packets at the default size), then each
    path at 1e7, 2e7, 4e7, ... packets (fresh seeds) until its I map is within the
    smallest target of the reference.  The error of a map is the relative L2 difference
    of its I maps (and of its Q, U maps against I) from the reference's, over the
    cameras; the reference's own Monte-Carlo noise (its batch spread / sqrt(n_ref)) is
    taken out in quadrature.  Seconds are each path's measured launch times."""
    total = sum(int(src["n_packets"]) for src in run["sources"])

    def images(m, r, optics):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        M.launch(m, r, precision="fp32", optics=optics)
        out = np.zeros((n_cam, 4, npix[1], npix[0]))
        for k in range(n_cam):
            m.image(k, out[k])
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    refs = [images(mdl_t, dict(run, seed=7000 + k), "tables")[0] for k in range(n_ref)]
    ref = np.mean(refs, axis=0)
    nI = np.sum(ref[:, 0] ** 2, axis=(1, 2))
    var_ref = np.var(refs, axis=0, ddof=1) / n_ref
    noise_I = float(np.mean(np.sum(var_ref[:, 0], axis=(1, 2)) / nI))
    noise_QU = float(np.mean(np.sum(var_ref[:, 1:3], axis=(1, 2, 3)) / nI))

    def errors(img):
        dI = float(np.mean(np.sum((img[:, 0] - ref[:, 0]) ** 2, axis=(1, 2)) / nI))
        dQU = float(np.mean(np.sum((img[:, 1:3] - ref[:, 1:3]) ** 2, axis=(1, 2, 3)) / nI))
        return max(0.0, dI - noise_I) ** 0.5, max(0.0, dQU - noise_QU) ** 0.5

    out = {"reference": {"packets": n_ref * total, "I_noise": noise_I ** 0.5, "QU_noise": noise_QU ** 0.5}}
    for name, m, optics in (("table", mdl_t, "tables"), ("surrogate", mdl_s, "surrogate")):
        runs, n, k = [], 1e7, 0
        while n <= n_max:
            half = int(n) // 2
            r = dict(run, seed=8000 + 100 * k + (0 if name == "table" else 50),
                     sources=[dict(run["sources"][0], n_packets=half),
                              dict(run["sources"][1], n_packets=int(n) - half)])
            img, sec = images(m, r, optics)
            eI, eQU = errors(img)
            runs.append({"packets": int(n), "seconds": sec, "I_error": eI, "QU_error": eQU})
            if eI <= min(targets) and eQU <= min(targets):
                break
            n *= 2
            k += 1
        reach = {}
        for eps in targets:
            hit = [x for x in runs if x["I_error"] <= eps and x["QU_error"] <= eps]
            reach["%g" % eps] = hit[0] if hit else None
        out[name] = {"runs": runs, "first_within": reach}
    for eps in targets:
        a, b = out["table"]["first_within"]["%g" % eps], out["surrogate"]["first_within"]["%g" % eps]
        out["table_over_surrogate_time_%g" % eps] = (a["seconds"] / b["seconds"]) if (a and b) else None
    return out


def run_surrogate(args, M, W, torch, model, run, table_imgs, table_step, table_value, table_step_s, table_mdl=None):
    """The same disk with the grain optics from the MLP surrogate: trained here on the
    tables (2e7 samples), table fallback above the error-map bound; throughput and
    the images' difference from the table path's, next to the table path's own
    Monte-Carlo difference between two seeds."""
    mdl = M.Model(model)
    t0 = time.perf_counter()
    sur = M.Surrogate(mdl, seed=5)
    n_train = int(round(args.sur_train_samples / 2048))
    hist = sur.train(n_steps=n_train, batch=2048, lr=3e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    t1 = time.perf_counter()
    emap = sur.error_map(1 << 22)
    mdl.set_surrogate(sur, args.sur_bound)
    setup_s = time.perf_counter() - t1
    n_cam = len(run["cameras"])
    npix = run["cameras"][0]["npix"]
    imgs = np.zeros((n_cam, 4, npix[1], npix[0]))
    # warm-up on the first 2^21 packets (kernels loaded, round buffers at full size)
    total = sum(int(src["n_packets"]) for src in run["sources"])
    M.launch(mdl, dict(run, seed=77, pid_end=min(1 << 21, total)), precision="fp32", optics="surrogate")
    torch.cuda.synchronize()
    sts = []
    t2 = time.perf_counter()
    for k in range(args.sur_steps):
        # a seed of its own: compared with the table images like a second table seed is
        sts.append(M.launch(mdl, dict(run, seed=5000 + k), precision="fp32", optics="surrogate"))
        for c in range(n_cam):
            mdl.image(c, imgs[c])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t2
    ev = sum(st["events"] for st in sts)
    value = ev / wall
    st = sts[-1]
    rows = st["mlp_tally_rows"] + st["mlp_scatter_rows"]
    fb = st["mlp_fallback_map"] + st["mlp_fallback_realizability"]
    # algorithmic FLOPs of one evaluation of the 7 -> 128 x 4 -> 20 network (the padded
    # input and output columns the kernel also multiplies are not counted)
    flop_row = 2.0 * (7 * 128 + 3 * 128 * 128 + 128 * 20)
    try:
        peak_bf16 = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"])
    except (OSError, KeyError, ValueError):
        peak_bf16 = 1700.0
    other = np.zeros_like(imgs)
    table_step(2000 + args.steps, other)
    # a second surrogate seed (untimed) for the fixed-error comparison
    imgs2 = np.zeros_like(imgs)
    M.launch(mdl, dict(run, seed=6000), precision="fp32", optics="surrogate")
    for c in range(n_cam):
        mdl.image(c, imgs2[c])
    out = {"workload": "flared disk %d^3 as the table line, grain optics from the MLP surrogate (7 -> 128 x 4 -> 20, "
                       "SiLU, BF16 weights, FP32 accumulation; tally and rejection trials on tcgen05), "
                       "trained on %.0e samples from the "
                       "tables, table fallback above error bound %g; %.0e packets"
                       % (args.grid, n_train * 2048, args.sur_bound, args.packets),
           "value": value, "unit": UNIT, "ms_per_step": 1e3 * wall / args.sur_steps,
           "vs_table_path": value / table_value,
           "train": {"samples": n_train * 2048, "steps": n_train, "batch": 2048, "seconds": train_s,
                     "loss_first": float(hist[0]), "loss_last": float(np.mean(hist[-20:]))},
           "error_map": {"median": float(np.median(emap)), "p90": float(np.quantile(emap, 0.9)),
                         "max": float(emap.max()), "cells_above_bound": int(np.sum(emap > args.sur_bound)),
                         "setup_s": setup_s},
           "mlp_rows_per_step": rows, "fallback_fraction": fb / max(rows, 1.0),
           "envelope_miss_fraction": st["envelope_miss"] / max(st["mlp_scatter_rows"], 1.0),
           "tally_overflow": st["tally_overflow"], "rounds": st["wave_iterations"],
           "mlp_tflops_over_launch": rows * flop_row / (wall / args.sur_steps) / 1e12,
           "kernel_ms": {"transport": st["ms_transport"], "tally": st["ms_tally"], "scatter": st["ms_scatter"],
                         "rounds_total": st["kernel_ms"]},
           "roofline": {"bound": "tensor", "kernel": "k_sur_tally_tc (tcgen05.mma kind::f16, BF16 x BF16 -> FP32 in "
                                                     "tensor memory, 3 tiles of 128 rows in flight per SM)",
                        "achieved": st["mlp_tally_rows"] * flop_row / (st["ms_tally"] * 1e-3) / 1e12,
                        "peak": peak_bf16, "unit": "TFLOP/s",
                        "frac": st["mlp_tally_rows"] * flop_row / (st["ms_tally"] * 1e-3) / 1e12 / peak_bf16,
                        "traffic": None, "peak_source": "measured bf16_tflops_sustained (kernel inside a long step)",
                        "flop_per_row": flop_row},
           "image_error": {"surrogate_vs_table": image_diff(imgs, table_imgs),
                           "table_vs_table_other_seed": image_diff(other, table_imgs),
                           "surrogate_vs_surrogate_other_seed": image_diff(imgs2, imgs)},
           "fixed_error": fixed_error(table_imgs, other, imgs, imgs2, args.packets, table_step_s,
                                      wall / args.sur_steps),
           "fixed_error_measured": (fixed_error_measured(M, torch, table_mdl, mdl, run, n_cam, npix)
                                    if args.fixed_error_measured else None),
           "gpu_launches_per_step": int(st["wave_iterations"]) * 4 + n_cam}
    sur.close()
    mdl.close()
    return out


def run_reference(args, rank):
    """Reference arm: the FP64 CPU oracle, each step one chunk of the workload's packet
    ids (steps cycle through the chunks the GPU arm's cpu_baseline times), the packet
    loops timed inside the oracle."""
    if rank != 0:
        return
    from paper_2512_01283_gb300 import workloads as W

    model = W.disk(n=args.grid)
    run = W.disk_run(n_packets=int(args.packets))
    cores = os.cpu_count() or 1
    bufs = None
    ev = wall = 0.0
    npk = 0
    timed = []
    for s in range(args.warmup + args.steps):
        c = s % CPU_CHUNKS
        e, w, n, bufs = oracle_sample(model, run, [c], cores, bufs)
        if s >= args.warmup:
            ev, wall, npk = ev + e, wall + w, npk + n
            timed.append(c)
    value = ev / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": oracle_sample_text(sorted(set(timed)), npk, args.packets)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    from paper_2512_01283_gb300 import build as B
    from paper_2512_01283_gb300 import mcrt as M
    from paper_2512_01283_gb300 import multigpu as MG
    from paper_2512_01283_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    B.build()

    model = W.disk(n=args.grid)
    # weak scaling: the whole job has `world` times the packets, each rank runs its share
    # of every source's packet ids (all of them on one rank); no collective on the transport
    run = MG.scaled_run(W.disk_run(n_packets=int(args.packets)), world)
    n_cam = len(run["cameras"])
    npix = run["cameras"][0]["npix"]
    mdl = M.Model(model)
    imgs = torch.empty((n_cam, 4, npix[1], npix[0]), dtype=torch.float64, device="cuda")

    def launch_share(m_, seed, **kw):
        return MG.rank_launch(lambda r, acc: M.launch(m_, dict(r, seed=seed), precision="fp32", accumulate=acc, **kw),
                              run, rank, world)

    def exchange(m_):
        # the one exchange of a sharded run: FP64 tallies summed over ranks before step 2,
        # in place on the library's own buffers (no copy out and back)
        if world > 1:
            src, ab = m_.tally_tensors(n_cam)
            MG.combine_tallies(src, ab, dist)

    my_cams = MG.rank_cameras(n_cam, rank, world)

    def image_step(m_, host=None):
        # step 2 split by camera over ranks, the images gathered (one all-reduce)
        if world == 1:
            for k in my_cams:
                m_.image(k, host[k] if host is not None else imgs[k])
            return
        imgs.zero_()
        for k in my_cams:
            m_.image(k, imgs[k])
        MG.combine_images(imgs, dist)
        if host is not None:
            host[:] = imgs.cpu().numpy()

    def step(seed):
        st = launch_share(mdl, seed, inline_tally=args.inline_tally, tally_blocks_per_sm=args.tally_bps,
                          blocks_per_sm=args.transport_bps)
        exchange(mdl)
        image_step(mdl)
        return st

    for w in range(args.warmup):
        step(1000 + w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stats = []
    # the raw nvidia-smi samples (their summary goes into the JSON line); MCRT_CLOCKS_DIR keeps them
    import tempfile

    clocks_dir = os.environ.get("MCRT_CLOCKS_DIR", tempfile.gettempdir())
    clocks_path = os.path.join(clocks_dir, "bench_clocks_rank%d.csv" % rank)
    os.makedirs(clocks_dir, exist_ok=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(clocks_path) as cs:
        e0.record()
        for s in range(args.steps):
            stats.append(step(2000 + s))
        e1.record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    events = sum(s["events"] for s in stats)
    ms_max, ev_all = MG.reduce_timing(ms, events, dist, device="cuda")
    value = ev_all / (ms_max * 1e-3)
    _, tal_all = MG.reduce_timing(ms, sum(s["tally_segments"] for s in stats), dist, device="cuda")

    # rooflines: the method's algorithmic bytes (per segment: 4 B kappa + 16 B grain
    # quaternion read; 8 B absorbed-energy read + write per absorbing segment; 4 Stokes x
    # 8 B read + write per camera per tallying segment, the source tally being far larger
    # than L2) over each kernel's CUDA-event time measured inside the library on its
    # launching stream.  FP32 table launches run in rounds: the transport kernel carries
    # the kappa, quaternion and absorbed bytes, the tally kernel the source bytes; the
    # longer of the two is `roofline`.  The bytes this design moves besides (32-byte cell
    # records, 32-byte tally records between the kernels) are given as design_bytes.
    seg = sum(s["segments"] for s in stats)
    tal = sum(s["tally_segments"] for s in stats)
    ab = sum(s["absorb_segments"] for s in stats)
    kms = sum(s["kernel_ms"] for s in stats)
    t_ms = sum(s["ms_transport"] for s in stats)
    a_ms = sum(s["ms_tally"] for s in stats)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    alg_t = 20.0 * seg + 16.0 * ab
    alg_a = 64.0 * n_cam * tal
    kernels = {}
    if t_ms > 0 and a_ms > 0:
        kernels["transport"] = {"kernel": "k_transport<float, table rounds>", "bound": "hbm",
                                "achieved": alg_t / (t_ms * 1e-3) / 1e9, "ms_per_step": t_ms / args.steps,
                                "bytes_per_unit": "4 kappa + 16 quaternion per segment, + 16 absorbed read/write "
                                                  "per absorbing segment",
                                "design_bytes_per_unit": "32 cell record per segment + 16 absorbed per absorbing "
                                                         "segment + 32 tally record per tallying segment",
                                "design_GBs": (32.0 * seg + 16.0 * ab + 32.0 * tal) / (t_ms * 1e-3) / 1e9,
                                "traffic": profiled_traffic("transport", seg / args.steps),
                                "issue": profiled_issue("transport")}
        kernels["tally"] = {"kernel": "k_tab_tally", "bound": "hbm", "achieved": alg_a / (a_ms * 1e-3) / 1e9,
                            "ms_per_step": a_ms / args.steps,
                            "bytes_per_unit": "n_cam x 4 Stokes x 8 B, read + write, per tallying segment",
                            "design_bytes_per_unit": "32 tally record + n_cam x 64 source read/write per record",
                            "design_GBs": (32.0 + 64.0 * n_cam) * tal / (a_ms * 1e-3) / 1e9,
                            "traffic": profiled_traffic("tally", tal / args.steps),
                            "issue": profiled_issue("tally")}
        for k in kernels.values():
            k.update({"peak": peak, "unit": "GB/s", "frac": k["achieved"] / peak, "peak_source": src})
            k["traffic_per_launch_note"] = "ncu dram bytes of a 2e6-packet capture, scaled to the step's units"
        dom = kernels["transport"] if t_ms >= a_ms else kernels["tally"]
        roofline = dict(dom)
    else:
        achieved = (alg_t + alg_a) / (kms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": None, "peak_source": src, "kernel": "k_transport<float, table> (tally in place)",
                    "bytes_per_unit": "20 per segment + 16 per absorbing segment + 64 x n_cam per tallying segment"}
    alg_step = alg_t + alg_a
    roofline_step = {"achieved": alg_step / (ms_max * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg_step / (ms_max * 1e-3) / 1e9 / peak, "bytes_per_step": alg_step / args.steps,
                     "note": "the method's bytes of step 1 (as roofline) over the whole step time, images included"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
            "roofline": roofline, "roofline_kernels": kernels, "roofline_step": roofline_step,
            "gpu_launches": int(sum(3 * s["wave_iterations"] if s["wave_iterations"] else 1 for s in stats)
                                + args.steps * len(my_cams)),
            "clocks": cs.summary(),
            "tally_segments_per_s": tal_all / (ms_max * 1e-3),
            "detail": {"events_per_step": events / args.steps, "segments_per_step": seg / args.steps,
                       "scatterings_per_step": sum(s["scatterings"] for s in stats) / args.steps,
                       "tally_segments_per_step": tal / args.steps,
                       "transport_ms_per_step": kms / args.steps,
                       "imaging_ms_per_step": ms / args.steps - kms / args.steps,
                       "rounds_per_step": sum(s["wave_iterations"] for s in stats) / args.steps,
                       "round_kernels_ms_per_step": {"transport": sum(s["ms_transport"] for s in stats) / args.steps,
                                                     "tally": sum(s["ms_tally"] for s in stats) / args.steps}}}

    # end to end through the public API with host buffers: H2D of the model, both
    # steps, D2H of the images, every step
    if not args.no_e2e:
        # the step's inputs and the images' host buffer in pinned host memory, as a
        # pipeline feeding the GPU would hold them
        keep = []  # the pinned tensors behind the arrays

        def pinned(a):
            keep.append(torch.from_numpy(np.ascontiguousarray(a)).pin_memory())
            return keep[-1].numpy()

        host_model = dict(model)
        for k in ("kappa_abs", "kappa_sca", "bfield", "emissivity"):
            host_model[k] = pinned(model[k])
        host_imgs = pinned(np.zeros((n_cam, 4, npix[1], npix[0])))
        h2d = sum(np.asarray(model[k]).nbytes for k in ("kappa_abs", "kappa_sca", "bfield", "emissivity"))
        h2d += sum(np.asarray(model["optics"][k]).nbytes for k in ("mueller", "bin_weight", "kext"))
        d2h = host_imgs.nbytes
        e_ev, e_t = 0.0, 0.0
        with ClockSampler(os.path.join(clocks_dir, "bench_clocks_e2e_rank%d.csv" % rank)) as cs_e:
            for s in range(args.steps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                m2 = M.Model(host_model)
                st = launch_share(m2, 3000 + s)
                exchange(m2)
                image_step(m2, host_imgs)
                m2.close()
                torch.cuda.synchronize()
                e_t += time.perf_counter() - t0
                e_ev += st["events"]
        e_ms_max, e_ev_all = MG.reduce_timing(1e3 * e_t, e_ev, dist, device="cuda")
        e_val = e_ev_all / (e_ms_max * 1e-3)
        line["e2e"] = {"value": e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": e_ms_max / args.steps, "host_buffers": "pinned", "clocks": cs_e.summary()}
        line["gpu_launches_e2e_per_step"] = int(3 * st["wave_iterations"]) + len(my_cams) + 5

    if not args.no_sweep:
        line["batched_sweep"] = run_sweep(args, M, W, torch, rank, world, dist)

    if not args.no_plane_parallel and world == 1:
        line["plane_parallel"] = run_plane_parallel(M, W, torch)

    if not args.no_spheroids and world == 1:
        line["spheroids"] = run_spheroids(M, W, torch)

    if not args.no_refined and world == 1:
        line["refined"] = run_refined(M, W, torch)

    if not args.no_microbench and world == 1:
        red = run_reduction_peaks(M)
        line["reduction_peaks"] = red
        if "tally" in line.get("roofline_kernels", {}):
            tk = line["roofline_kernels"]["tally"]
            tk["frac_of_bulk_reduction_dram"] = tk["achieved"] / red["bulk_rmw_GBs_dram"]

    if not args.no_surrogate and world == 1:
        table_imgs = imgs.cpu().numpy()

        def table_step(seed, out):
            M.launch(mdl, dict(run, seed=seed), precision="fp32")
            for k in range(n_cam):
                mdl.image(k, out[k])

        line["surrogate"] = run_surrogate(args, M, W, torch, model, run, table_imgs, table_step, value,
                                          ms_max / args.steps * 1e-3, table_mdl=mdl)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        chunks = list(range(args.cpu_chunks))
        ev, wall, npk, _ = oracle_sample(model, run, chunks, cores)
        line["cpu_baseline"] = {"value": ev / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": oracle_sample_text(chunks, npk, args.packets), "seconds": wall}
    mdl.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
