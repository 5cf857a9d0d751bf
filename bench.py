#!/usr/bin/env python3
"""Benchmark of the fictitious-wave CSEM gradient hot path.

One step = one full gradient for the workload's source batch, every row of
the hot path: coefficient set-up from the model, forward run with the fused
damped transform into all frequencies (volumes kept), misfit and weighted
residual, adjoint-source basis (CGNR), adjoint run driven by the basis
series, and the cell gradient with respect to ln(rho).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` counts cell updates of both runs
(cells incl. CPML x nt x sources x 2) per second of device time, inputs
resident in HBM.  `e2e` repeats the measurement through the same public calls
with the model and observed data copied from pinned host memory and the
gradient and misfit copied back inside the timed region.  The reference arm
times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s; batched gradient s/source vs plain path; % of HBM roofline"
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="thin_reservoir")
    ap.add_argument("--vti", action="store_true", help="VTI medium: models (rho_h, rho_v), split gradient")
    ap.add_argument("--order", type=int, default=2, choices=[2, 4],
                    help="spatial order of the staggered differences (4: four-point kernels)")
    ap.add_argument("--inversion", type=int, default=0, help="run this many iterations of the outer inversion loop")
    ap.add_argument("--route", default="basis", choices=["basis", "td"],
                    help="gradient route of --inversion: basis-function adjoint or time-domain adjoint")
    ap.add_argument("--max-src", type=int, default=0,
                    help="use only the first K sources of the workload (side measurements of large configs)")
    ap.add_argument("--oracle-timings", action="store_true",
                    help="time the FP64 oracle (1 thread and all cores) beside the device on three workloads")
    ap.add_argument("--early-stop-volumes", type=float, default=0.0,
                    help="time gradients with the early end of the forward and adjoint volume runs")
    ap.add_argument("--early-stop", type=float, default=0.0,
                    help="time forward data runs with the early end at this tolerance against full runs")
    ap.add_argument("--td", type=int, default=0,
                    help="time this many time-domain adjoint gradients against the basis route")
    ap.add_argument("--cpu-steps", type=int, default=2000, help="time steps in the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batched-vs-plain", action="store_true",
                    help="side measurement on batched_towline: one batched Kahan gradient vs one source per launch")
    ap.add_argument("--nt", type=int, default=0, help="time steps for --batched-vs-plain (0: the workload's)")
    ap.add_argument("--check-sources", type=int, default=4, help="sources scored against FP64 in --batched-vs-plain")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                if self.uuid and self.uuid not in p[0]:
                    continue
                rows.append(p)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_workload(name, rank, world, vti=False, max_src=0):
    from paper_2211_16665_gb300 import dist as D
    from paper_2211_16665_gb300 import workloads as W
    wl = W.ALL[name]()
    if max_src and wl.src.n > max_src:
        wl.src = wl.src.subset(list(range(max_src)))     # a side measurement on the first sources
    if vti:
        # VTI medium (Sec. 2): rho_v = 2 rho_h below the water, capped at the CFL resistivity
        water = wl.rho.min()
        def split(r):
            rv = np.where(r > water, np.minimum(2.0 * r, wl.rho_max), r)
            return np.stack([r, rv])
        wl.rho, wl.rho_true = split(wl.rho), split(wl.rho_true)
    if world > 1:
        # weak scaling: a towline of `world` sources on the same model, one share per rank
        line = D.towline(wl.src, world * wl.src.n)
        wl.src = line.subset(list(D.shard(line.n, rank, world)))
    return wl


def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_bytes(wl, eng):
    """Algorithmic bytes per launch of each stepping kernel (one source batch).

    Per cell (the work domain of the step kernels) and source, with r the real
    size and f the CPML slab fraction sum_axes 2 npml / n_axis (two CPML
    arrays per axis per half-step, read + written, inside the slabs only):
      k_h     read E^n 3r, read + write H 6r, CPML 4 r f
      k_e     read E^n 3r, write E^{n+1} 3r, read H 3r, read dt/eps 3r, CPML 4 r f
      k_step  (fused) read E^n 3r, read H 3r, write H 3r, read dt/eps 3r,
              write E^{n+1} 3r, CPML 8 r f
      k_dft   one flush of M snapshots, per lattice node: read 3 M r, read + write
              the 3 nf complex accumulators 3 nf 4r, and their Kahan terms as
              much again
    """
    r = 4 if eng.precision == 32 else 8
    cells = wl.nx * wl.ny * wl.nz * wl.src.n
    nodes = (wl.nx + 1) * (wl.ny + 1) * (wl.nz + 1) * wl.src.n
    f = sum(2 * wl.npml / n for n in (wl.nx, wl.ny, wl.nz))
    per = {"k_h": 9 * r + 4 * r * f,
           "k_e": 12 * r + 4 * r * f,
           "k_step": 15 * r + 8 * r * f,
           "k_dft": 3 * eng.flush_block() * r + 3 * eng.nf * 4 * r * (2 if eng.info.kahan else 1)}
    units = {"k_h": cells, "k_e": cells, "k_step": cells, "k_dft": nodes}
    return {k: v * units[k] for k, v in per.items()}, per


# DRAM bytes (read + write) per launch of a kernel from ncu captures of
# dram__bytes_read.sum and dram__bytes_write.sum (cold cache, 128x128x96 thin reservoir,
# nt = 256 through the profile driver with the launch configurations of
# profiles/traffic_lean_thin_reservoir.md; the mean over the captured launches), valid only
# for the source they were taken on: keyed by workload, kernel, launch code (Engine.kz
# entry) and the SHA-1 of the kernel's source file, with the shared header's SHA-1
# checked separately.  Any other kernel reports null.
_LEAN = "78b60ad8187d51577bc248ded4ea5cffa931c7e7"
_STEP = "2b13003dc0a546c8de35f6b3b533bac6c5297935"
NCU_TRAFFIC = {
    ("thin_reservoir_128x128x96_fp32", "k_e", 16422, _LEAN): 66.875e6 + 1.251e6,
    ("thin_reservoir_128x128x96_fp32", "k_h", 16422, _LEAN): 47.268e6 + 0.002e6,
    ("thin_reservoir_128x128x96_fp32", "k_e", 16424, _LEAN): 66.885e6 + 1.476e6,
    ("thin_reservoir_128x128x96_fp32", "k_h", 16424, _LEAN): 47.270e6 + 0.001e6,
    ("thin_reservoir_128x128x96_fp32", "k_dft", 129, _STEP): 980.377e6 + 288.796e6,
    ("thin_reservoir_128x128x96_fp32", "k_dft", 131, _STEP): 980.487e6 + 288.802e6,
}
_HEADER_SHA = "d4d538b5843a1f7202e9ae15e2c39d39f857e817"


def ncu_traffic(wl, eng, kernel):
    import hashlib
    code = {"k_h": eng.kz[0], "k_e": eng.kz[1], "k_dft": eng.kz[2]}.get(kernel) if eng.kz else None
    src = {"k_h": "kern_lean.cu", "k_e": "kern_lean.cu", "k_dft": "kern_step.cu"}.get(kernel)
    if code is None or src is None:
        return None
    d = os.path.join(ROOT, "paper_2211_16665_gb300", "csrc")
    sha = lambda f: hashlib.sha1(open(os.path.join(d, f), "rb").read()).hexdigest()
    if sha("csem_internal.cuh") != _HEADER_SHA:
        return None
    return NCU_TRAFFIC.get((wl.name, kernel, code, sha(src)))


def cpu_baseline(wl, nt_sample, order=2):
    from oracle import fdtd
    pb = fdtd.problem_from_workload(wl, order=order)
    nt_sample = min(nt_sample, pb.nt)
    t0 = time.perf_counter()
    fdtd.forward(pb, wl.rho, wl.src.subset([0]), wl.rec, keep_volume=True, nt_run=nt_sample)
    t = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": wl.cells * nt_sample / t / 1e9, "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, {nt_sample} of {pb.nt} steps of one source with the volumetric transform "
                      f"into {wl.freqs.size} frequencies on the full {wl.nx}x{wl.ny}x{wl.nz} grid "
                      f"(a gradient is 2 such runs per source); {t:.1f} s"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2211_16665_gb300 import _capi
    from paper_2211_16665_gb300 import dist as D
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine, misfit

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = make_workload(args.workload, rank, world, vti=args.vti, max_src=args.max_src)
    eng = Engine.from_workload(wl, vti=args.vti, order=args.order)
    S = wl.src.n
    rho = eng.model_tensor(wl.rho)
    rho_true = eng.model_tensor(wl.rho_true)
    d_obs = eng.fwd_model(rho_true, wl.src, wl.rec)
    d_obs = torch.as_tensor(W.add_noise(d_obs.cpu().numpy(), wl.noise, wl.noise_seed), device=dev)
    torch.cuda.synchronize()

    def step(rho_in, d_obs_in):
        d, E = eng.fwd_model(rho_in, wl.src, wl.rec, keep_volume=True)
        phi, r = misfit(d_obs_in, d)
        basis, fit, its = eng.estimate_adjoint_basis(gamma=1e-12, relative=True, fit_target=1e-3)
        V = eng.adjoint_model(rho_in, wl.rec, r, basis)
        g = eng.gradient(rho_in, E, V, wrt="lnrho")
        D.sum_over_ranks(g, phi)          # the one exchange: sum of the per-source gradients
        return phi, g, fit

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(rho, d_obs)
    barrier()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    n0 = _capi.launch_count()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        phi, g, fit = step(rho, d_obs)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (_capi.launch_count() - n0) // args.steps
    clk = clocks.stop()
    ms = D.max_over_ranks(ms, device=dev)

    cell_updates = 2.0 * wl.cells * eng.nt * S * world
    value = cell_updates / (ms / 1e3) / 1e9

    # the adjoint-source basis solve alone (it is part of every timed step above; it blocks
    # until its fit residual is on the host)
    torch.cuda.synchronize()
    tb = time.perf_counter()
    eng.estimate_adjoint_basis(gamma=1e-12, relative=True, fit_target=1e-3)
    basis_ms = (time.perf_counter() - tb) * 1e3

    # roofline of the dominant kernel, timed live with CUDA events on its stream
    _, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    from paper_2211_16665_gb300.engine import _ptr, _stream
    kms = dict(zip(("k_h", "k_step", "k_e", "k_dft"), _capi.time_step_kernels(eng.ctx, S, _ptr(E), 200, _stream())))
    bytes_launch, per_unit = kernel_bytes(wl, eng)
    fused = kms["k_step"] > 0
    per_step_ms = ({"k_step": kms["k_step"]} if fused else {"k_h": kms["k_h"], "k_e": kms["k_e"]})
    per_step_ms["k_dft"] = kms["k_dft"] / eng.flush_block()
    dom = max(per_step_ms, key=per_step_ms.get)
    peak, peak_kind = hbm_peak()
    gbs = {k: round(bytes_launch[k] / (kms[k] / 1e3) / 1e9, 1) for k in kms if kms[k] > 0}
    achieved = gbs[dom]
    tot = sum(per_step_ms.values())
    roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind, "traffic": ncu_traffic(wl, eng, dom),
            "bytes_per_unit": round(per_unit[dom], 1), "unit_of_work": "lattice node" if dom == "k_dft" else "cell",
            "ms_per_launch": {k: round(v, 5) for k, v in kms.items()},
            "step_share": {k: round(v / tot, 3) for k, v in per_step_ms.items()},
            "all_kernels_gbs": gbs}
    del E

    # end to end: host model in, host gradient out
    e2e = None
    if not args.no_e2e:
        rho_h = rho.cpu().pin_memory()
        dobs_h = d_obs.cpu().pin_memory()
        g_h = torch.empty(g.shape, dtype=g.dtype).pin_memory()
        phi_h = torch.empty((), dtype=torch.float64).pin_memory()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            r_dev = rho_h.to(dev, non_blocking=True)
            o_dev = dobs_h.to(dev, non_blocking=True)
            phi2, g2, _ = step(r_dev, o_dev)
            g_h.copy_(g2, non_blocking=True)
            phi_h.copy_(phi2, non_blocking=True)
        e1.record(stream)
        barrier()
        ems = D.max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
        e2e = {"value": round(cell_updates / (ems / 1e3) / 1e9, 3), "unit": "Gcell-updates/s",
               "ms_per_step": round(ems, 3),
               "h2d_bytes_per_step": int(rho_h.numel() * rho_h.element_size() + dobs_h.numel() * dobs_h.element_size()),
               "d2h_bytes_per_step": int(g_h.numel() * g_h.element_size() + 8)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_steps, args.order)

    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 3), "unit": "Gcell-updates/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32" if eng.precision == 32 else "f64",
               "data": "synthetic",
               "config": {"workload": wl.name, "cells": wl.cells, "grid": [wl.nx, wl.ny, wl.nz], "nt": eng.nt,
                          "dt": eng.dt, "n_src_per_gpu": S, "n_rec": wl.rec.n, "freqs_hz": list(map(float, wl.freqs)),
                          "kahan": bool(eng.info.kahan), "launch": eng.launch_config(), "l2": "inputs larger than L2 (each step streams "
                          f"{2 * 3 * eng.nf * eng.vol * 8 * S * (2 if eng.info.kahan else 1) / 2**20:.0f} MiB of "
                          "transform volumes)", "parallelism": f"sources sharded, dp{world}",
                          "medium": "vti" if args.vti else "isotropic", "order": eng.order},
               "grad_s_per_source": round(ms / 1e3 / S, 4),
               "basis_fit": fit, "basis_gamma_rel": eng.basis_gamma, "basis_ms": round(basis_ms, 3),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
               "clocks": clk}
        print(json.dumps(out), flush=True)
    eng.close()
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    from oracle import fdtd
    wl = make_workload(args.workload, 0, 1, vti=args.vti)
    pb = fdtd.problem_from_workload(wl)
    src = wl.src.subset([0])
    # calibrate: size each step so that warmup + steps take ~2.5 minutes
    t0 = time.perf_counter()
    fdtd.forward(pb, wl.rho, src, wl.rec, keep_volume=True, nt_run=3)
    per = (time.perf_counter() - t0) / 3
    nt_s = int(max(5, min(pb.nt, 150.0 / max(1, args.steps + args.warmup) / per)))
    for _ in range(args.warmup):
        fdtd.forward(pb, wl.rho, src, wl.rec, keep_volume=True, nt_run=nt_s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fdtd.forward(pb, wl.rho, src, wl.rec, keep_volume=True, nt_run=nt_s)
    t = (time.perf_counter() - t0) / args.steps
    value = wl.cells * nt_s / t / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "Gcell-updates/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "cells": wl.cells, "grid": [wl.nx, wl.ny, wl.nz], "nt": pb.nt,
                      "nt_sample": nt_s, "medium": "vti" if args.vti else "isotropic"},
           "cpu_baseline": {"value": round(value, 5), "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
                            "sample": f"{nt_s} of {pb.nt} steps of one forward run with the volumetric transform"},
           "e2e": {"value": round(value, 5), "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched_vs_plain(args):
    """Gradient seconds per source: all sources in one launch (FP32 + Kahan) against one
    source per launch (FP32, plain transform), and each gradient's error against FP64."""
    import torch
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine, misfit

    torch.cuda.set_device(0)
    wl = W.batched_towline()
    S = wl.src.n

    def gradient(eng, src, d_obs, out):
        rho = eng.model_tensor(wl.rho)
        d, E = eng.fwd_model(rho, src, wl.rec, keep_volume=True)
        phi, r = misfit(d_obs, d)
        basis, _, _ = eng.estimate_adjoint_basis()
        V = eng.adjoint_model(rho, wl.rec, r, basis)
        eng.gradient(rho, E, V, out=out)
        del E, V

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    Z = W.cell_centres(wl.xn, wl.yn, wl.zn)[2]
    rho_obs = np.where(Z >= 1000.0, 1.3 * wl.rho, wl.rho)     # observed data: sediment 30 % more resistive
    out = {"mode": "batched_vs_plain", "workload": wl.name, "n_src": S, "nt": None}
    # batched: every source in each launch, compensated transform
    eb = Engine.from_workload(wl, nt=args.nt or None, max_src=S, kahan=1)
    out["nt"] = eb.nt
    d_obs = eb.fwd_model(eb.model_tensor(rho_obs), wl.src, wl.rec)
    gb = torch.zeros((wl.nz, wl.ny, wl.nx), dtype=torch.float32, device="cuda")
    gradient(eb, wl.src, d_obs, gb)                       # warm-up
    gb.zero_()
    tb = timed(lambda: gradient(eb, wl.src, d_obs, gb))
    out["batched"] = {"s_per_source": tb / S, "launch": eb.launch_config(), "kahan": True}
    eb.close()
    # plain: one source per launch, plain FP32 transform
    ep = Engine.from_workload(wl, nt=args.nt or None, max_src=1, kahan=0)
    gp = torch.zeros_like(gb)
    gradient(ep, wl.src.subset([0]), d_obs[:1].contiguous(), gp)
    gp.zero_()
    tp = timed(lambda: [gradient(ep, wl.src.subset([s]), d_obs[s:s + 1].contiguous(), gp) for s in range(S)])
    out["plain"] = {"s_per_source": tp / S, "launch": ep.launch_config(), "kahan": False}
    ep.close()
    # error of each path's gradient on the first sources against the FP64 engine
    k = min(args.check_sources, S)
    sub = wl.src.subset(list(range(k)))
    errs = {}
    ref = None
    for name, prec, kahan in (("fp64", 64, 0), ("batched", 32, 1), ("plain", 32, 0)):
        e = Engine.from_workload(wl, nt=args.nt or None, max_src=k, precision=prec, kahan=kahan)
        g = torch.zeros((wl.nz, wl.ny, wl.nx), dtype=e.real, device="cuda")
        gradient(e, sub, d_obs[:k].contiguous(), g)
        g = g.double().cpu().numpy()
        e.close()
        if ref is None:
            ref = g
        else:
            errs[name] = float(np.linalg.norm(g - ref) / np.linalg.norm(ref))
    out["batched"]["grad_rel_l2_vs_fp64"] = errs["batched"]
    out["plain"]["grad_rel_l2_vs_fp64"] = errs["plain"]
    out["speedup_per_source"] = out["plain"]["s_per_source"] / out["batched"]["s_per_source"]
    out["note"] = (f"nt = {out['nt']} time steps per run; the per-step cost does not depend on nt; errors on the "
                   f"first {k} sources")
    print(json.dumps(out), flush=True)


def run_inversion(args):
    """K iterations of the outer inversion loop (Sec. 3.5) on the thin reservoir (FP32):
    noisy synthetic data, a 600 m offset mute, 3 % relative-error weights, the
    sediment free and the water fixed, start model without the reservoir."""
    import math
    import torch
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine
    from paper_2211_16665_gb300.inversion import Inversion
    torch.cuda.set_device(0)
    wl = make_workload(args.workload, 0, 1)
    eng = Engine.from_workload(wl)
    d_true = eng.fwd_model(eng.model_tensor(wl.rho_true), wl.src, wl.rec).cpu().numpy()
    if args.early_stop > 0:
        eng.set_early_stop(args.early_stop)    # the line-search forwards keep no volumes
    d_obs = W.add_noise(d_true, wl.noise, wl.noise_seed)
    dx = wl.rec.x[None, :] - wl.src.x[:, None]
    dy = wl.rec.y[None, :] - wl.src.y[:, None]
    mute = (np.hypot(dx, dy) >= 600.0).astype(float)[:, :, None].repeat(wl.freqs.size, axis=2)
    w = mute / (0.03 * np.abs(d_obs) + 1e-30)
    free = wl.rho > wl.rho.min()
    basis, fit, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    inv = Inversion(eng, wl.src, wl.rec, torch.as_tensor(d_obs), wl.rho, free, basis, weights=w,
                    xn=wl.xn, yn=wl.yn, zn=wl.zn, m_max=math.log(wl.rho_max), route=args.route)
    runs = {"fwd": 0}
    calls = eng.fwd_model

    def counted(*a, **k):
        runs["fwd"] += 1
        return calls(*a, **k)

    eng.fwd_model = counted
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m, hist = inv.run(torch.log(torch.as_tensor(wl.rho)), args.inversion)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    slab = wl.rho_true > 10.0
    upd = np.abs(m.cpu().numpy() - np.log(wl.rho))
    kz = int(np.unravel_index(int(np.argmax(upd)), upd.shape)[0])
    out = {"mode": "inversion", "workload": wl.name, "iterations": len(hist), "s_total": round(t, 3),
           "s_per_iteration": round(t / max(1, len(hist)), 3), "forward_runs": runs["fwd"],
           "adjoint_runs": len(hist), "phi": [round(h["phi"], 6) for h in hist],
           "directions": [h["direction"] for h in hist], "steps": [h["step"] for h in hist],
           "reservoir_mean_rho": {"start": float(np.exp(np.log(wl.rho[slab]).mean())),
                                  "end": float(np.exp(m.cpu().numpy()[slab].mean())),
                                  "true": float(wl.rho_true[slab].mean())},
           "largest_update": {"ln_rho": float(upd.max()), "depth_m": float(0.5 * (wl.zn[kz] + wl.zn[kz + 1]))},
           "basis_fit": fit, "early_stop_tol": args.early_stop, "gradient_route": args.route,
           "data": "synthetic, 1 % noise (seed 42), 600 m mute, 3 % relative-error weights"}
    print(json.dumps(out))


def run_td(args):
    """The time-domain adjoint gradient (appendix) against the basis-function route on
    the thin reservoir (FP32, the same residual): seconds per gradient, steps run,
    the checkpoint plan, and the relative L2 difference of the two gradients."""
    import torch
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine, misfit
    torch.cuda.set_device(0)
    wl = make_workload(args.workload, 0, 1)
    eng = Engine.from_workload(wl)
    rho = eng.model_tensor(wl.rho)
    d_obs = torch.as_tensor(W.add_noise(eng.fwd_model(eng.model_tensor(wl.rho_true), wl.src, wl.rec).cpu().numpy(),
                                        wl.noise, wl.noise_seed), device=eng.device)
    d = eng.fwd_model(rho, wl.src, wl.rec)
    _, r = misfit(d_obs, d)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)

    def basis_route():
        _, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
        V = eng.adjoint_model(rho, wl.rec, r, basis)
        return eng.gradient(rho, E, V)

    def td_route():
        return eng.gradient_td(rho, wl.src, wl.rec, r)

    out = {"mode": "td_adjoint", "workload": wl.name, "nt": eng.nt, "cells": int(np.prod(eng.model_shape))}
    grads = {}
    for name, fn in (("basis", basis_route), ("td", td_route)):
        for _ in range(max(1, args.warmup)):
            g = fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.td):
            g = fn()
        torch.cuda.synchronize()
        out[f"s_per_gradient_{name}"] = round((time.perf_counter() - t0) / args.td, 4)
        grads[name] = g.double().cpu().numpy()
    seg = eng.last_td["segment"]
    K = -(-eng.nt // seg)
    out.update(segment=seg, segments=K, workspace_gb=round(eng.last_td["workspace_bytes"] / 1e9, 3),
               forward_steps_td=(K - 1) * seg + eng.nt, adjoint_steps_td=eng.nt,
               rel_l2_td_vs_basis=float(np.linalg.norm(grads["td"] - grads["basis"]) / np.linalg.norm(grads["basis"])),
               gcell_per_s_td=round(out["cells"] * ((K - 1) * seg + 2 * eng.nt) / out["s_per_gradient_td"] / 1e9, 2),
               data="synthetic, 1 % noise (seed 42); the same residual for both routes")
    print(json.dumps(out))


def run_oracle_timings(args):
    """The FP64 oracle timed on the host cores, single-threaded and on all cores, on bounded
    samples of the tiny FP64 box, the thin reservoir and the 116^3 crop of the heterogeneous
    model (one source, forward run with the volumetric transform), beside the device's
    gradient on the same workloads (Gcell-updates/s over both runs of all sources)."""
    import torch
    from oracle import fdtd
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine, misfit
    torch.cuda.set_device(0)
    all_threads = os.cpu_count() or 1
    out = {"mode": "oracle_timings", "host_cores": all_threads, "rows": []}
    for name, nt_sample in (("plain_tiny", 300), ("thin_reservoir", 200), ("heterogeneous_crop96", 200)):
        wl = W.ALL[name]()
        row = {"workload": wl.name, "cells": wl.cells, "precision": wl.precision}
        pb = fdtd.problem_from_workload(wl)
        n = min(nt_sample, pb.nt)
        for threads in (1, all_threads):
            fdtd.set_threads(threads)
            t0 = time.perf_counter()
            fdtd.forward(pb, wl.rho, wl.src.subset([0]), wl.rec, keep_volume=True, nt_run=n)
            t = time.perf_counter() - t0
            row[f"oracle_gcell_s_{threads}_threads"] = round(wl.cells * n / t / 1e9, 5)
        row["oracle_sample"] = f"{n} of {pb.nt} steps, one source, volumetric transform"
        fdtd.set_threads(all_threads)
        eng = Engine.from_workload(wl)
        rho = eng.model_tensor(wl.rho)
        d_obs = eng.fwd_model(eng.model_tensor(wl.rho_true), wl.src, wl.rec)
        basis, _, _ = eng.estimate_adjoint_basis()

        def grad():
            d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
            _, r = misfit(d_obs, d)
            V = eng.adjoint_model(rho, wl.rec, r, basis)
            return eng.gradient(rho, E, V)
        grad()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grad()
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        row["gpu_gcell_s"] = round(2.0 * wl.cells * eng.nt * wl.src.n / t / 1e9, 3)
        row["gpu_s_per_gradient_per_source"] = round(t / wl.src.n, 4)
        row["n_src"] = wl.src.n
        row["gpu_over_oracle_all_cores"] = round(row["gpu_gcell_s"] / row[f"oracle_gcell_s_{all_threads}_threads"], 1)
        eng.close()
        out["rows"].append(row)
    print(json.dumps(out))


def run_early_stop_volumes(args):
    """Gradients on the thin reservoir with the early end applied to the volumetric
    transforms of the forward and adjoint runs (Sec. 2) against full gradients: seconds per
    gradient, the steps each run took, and the relative L2 change of the gradient."""
    import torch
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine, misfit
    torch.cuda.set_device(0)
    wl = make_workload(args.workload, 0, 1)
    eng = Engine.from_workload(wl)
    rho = eng.model_tensor(wl.rho)
    d_obs = torch.as_tensor(W.add_noise(eng.fwd_model(eng.model_tensor(wl.rho_true), wl.src, wl.rec).cpu().numpy(),
                                        wl.noise, wl.noise_seed), device=eng.device)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True, fit_target=1e-3)
    out = {"mode": "early_stop_volumes", "workload": wl.name, "nt": eng.nt, "tol": args.early_stop_volumes}
    grads = {}
    for name, tol in (("full", 0.0), ("early", args.early_stop_volumes)):
        eng.set_early_stop_volumes(tol)

        def grad():
            d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
            sf = eng.last_run_steps()
            _, r = misfit(d_obs, d)
            V = eng.adjoint_model(rho, wl.rec, r, basis)
            sa = eng.last_run_steps()
            return eng.gradient(rho, E, V), sf, sa
        for _ in range(max(1, args.warmup)):
            grad()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            g, sf, sa = grad()
        torch.cuda.synchronize()
        out[f"s_per_gradient_{name}"] = round((time.perf_counter() - t0) / args.steps, 4)
        out[f"steps_{name}"] = {"forward": sf, "adjoint": sa}
        grads[name] = g.double().cpu().numpy()
    out["speedup"] = round(out["s_per_gradient_full"] / out["s_per_gradient_early"], 3)
    out["rel_l2_gradient_change"] = float(np.linalg.norm(grads["early"] - grads["full"]) /
                                          np.linalg.norm(grads["full"]))
    print(json.dumps(out))


def run_early_stop(args):
    """Forward data runs (receivers only) on the thin reservoir with the early end of Sec. 2
    at the given tolerance against full runs: ms per run, steps, relative L2 change of the data."""
    import torch
    from paper_2211_16665_gb300.engine import Engine
    torch.cuda.set_device(0)
    wl = make_workload(args.workload, 0, 1)
    eng = Engine.from_workload(wl)
    rho = eng.model_tensor(wl.rho)
    out = {"mode": "early_stop", "workload": wl.name, "nt": eng.nt, "tol": args.early_stop}
    data = {}
    for name, tol in (("full", 0.0), ("early", args.early_stop)):
        eng.set_early_stop(tol)
        for _ in range(args.warmup):
            d = eng.fwd_model(rho, wl.src, wl.rec)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            d = eng.fwd_model(rho, wl.src, wl.rec)
        ev1.record()
        torch.cuda.synchronize()
        out[f"ms_per_run_{name}"] = round(ev0.elapsed_time(ev1) / args.steps, 3)
        out[f"steps_{name}"] = eng.last_run_steps()
        data[name] = d.cpu().numpy()
    out["speedup"] = round(out["ms_per_run_full"] / out["ms_per_run_early"], 3)
    out["rel_l2_data_change"] = float(np.linalg.norm(data["early"] - data["full"]) / np.linalg.norm(data["full"]))
    print(json.dumps(out))


def main():
    args = parse()
    if args.oracle_timings:
        run_oracle_timings(args)
        return
    if args.inversion:
        run_inversion(args)
        return
    if args.early_stop_volumes > 0:
        run_early_stop_volumes(args)
        return
    if args.early_stop > 0:
        run_early_stop(args)
        return
    if args.td:
        run_td(args)
        return
    if args.batched_vs_plain:
        run_batched_vs_plain(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
