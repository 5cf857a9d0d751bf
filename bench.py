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
    ap.add_argument("--workload", default="batched_towline")
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
    ap.add_argument("--es-floor", type=float, default=1e-4,
                    help="--early-stop-volumes: entries below this fraction of their frequency's largest get an "
                         "absolute bound")
    ap.add_argument("--early-stop", type=float, default=0.0,
                    help="time forward data runs with the early end at this tolerance against full runs")
    ap.add_argument("--td", type=int, default=0,
                    help="time this many time-domain adjoint gradients against the basis route")
    ap.add_argument("--cpu-steps", type=int, default=300, help="time steps in the oracle sample")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="--impl reference: wall-clock budget of its warm-up and timed steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=2,
                    help="sources per launch: each step runs one batched gradient of the next batch of the "
                         "workload's sources")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-source-per-launch comparison")
    ap.add_argument("--check-sources", type=int, default=1,
                    help="sources of the first batch whose gradients are scored against the FP64 engine")
    ap.add_argument("--e2e-steps", type=int, default=2, help="steps of the end-to-end measurement")
    ap.add_argument("--batch-sweep", default="",
                    help="comma-separated sources per launch (e.g. 1,2,4,8,16,32): one JSON line per batch size "
                         "with the gradient seconds per source, compensated, and the plain path at 1 source")
    ap.add_argument("--nt", type=int, default=0, help="--batch-sweep: time steps per run (0: the workload's)")
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
    # weak scaling: a towline of world x the workload's sources on the same model, one share per rank
    wl.src = D.rank_sources(wl.src, rank, world)
    return wl


def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def stencil_bytes(wl, eng):
    """Algorithmic bytes of one fused H+E step per cell (the floor of the byte model): the six
    field components read and written once (6 x 2 x r), one material value per cell (r per
    conductivity: 2 in a VTI medium), and the CPML memory, four arrays read and written on the
    cells of each axis' two slabs (4 x 2 x r x sum over axes of 2 npml / n)."""
    r = 4 if eng.precision == 32 else 8
    f = sum(2 * wl.npml / n for n in (wl.nx, wl.ny, wl.nz))
    return 12 * r + r * (2 if eng.vti else 1) + 8 * r * f


def flush_bytes(wl, eng):
    """Algorithmic bytes of one transform flush of M snapshots per lattice node: the M
    snapshots read (3 M r) and the 3 n_freq complex accumulators read and written once
    (3 n_freq 2r x 2), and their compensation terms as much again with Kahan."""
    r = 4 if eng.precision == 32 else 8
    M = eng.flush_block()
    return 3 * M * r + 3 * eng.nf * 2 * r * 2 * (2 if eng.info.kahan else 1)


# DRAM bytes (read + write) per launch from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum) of the named kernel on the named workload, per source of a launch,
# valid only while the kernel's source file and the shared header are the ones captured
# (SHA-1 of each); the figure is scaled by the sources of a launch.  Anything else reports null.
# Stencil pair on the 256x256x128 towline, 2 sources per launch, lean H (2 cells, 4 planes,
# 8 blocks/SM) and lean E (the same): 654.1 + 776.4 MB per launch, cold cache, the mean of
# 149 launches of each in the profiling module's forward run (nt 256) under ncu.
NCU_TRAFFIC = {
    ("batched_towline_256x256x128_32src", "k_h_lean+k_e_lean", "kern_lean.cu",
     "e04bd69a59f373a283c3077b61bb51e2bfd75cf6", "c841fae235235a812cf25a4a18317b28f55113ae"): (654.1e6 + 776.4e6) / 2,
}


def ncu_traffic(wl, kernel, S):
    import hashlib
    d = os.path.join(ROOT, "paper_2211_16665_gb300", "csrc")
    sha = lambda f: hashlib.sha1(open(os.path.join(d, f), "rb").read()).hexdigest()
    for (name, kern, src, src_sha, hdr_sha), per_src in NCU_TRAFFIC.items():
        if name == wl.name and kern == kernel and sha(src) == src_sha and sha("csem_internal.cuh") == hdr_sha:
            return per_src * S
    return None


def cpu_baseline(wl, nt_sample, order=2, threads=0):
    """The CPU baseline leg: the FP64 oracle, as it stands, timed on a bounded sample (one
    source's forward run with the volumetric transform for nt_sample steps) on `threads` host
    threads (0: all, or OMP_NUM_THREADS)."""
    from oracle import fdtd
    pb = fdtd.problem_from_workload(wl, order=order)
    nt_sample = min(nt_sample, pb.nt)
    prev = fdtd.get_threads()
    if threads:
        fdtd.set_threads(threads)
    try:
        t0 = time.perf_counter()
        fdtd.forward(pb, wl.rho, wl.src.subset([0]), wl.rec, keep_volume=True, nt_run=nt_sample)
        t = time.perf_counter() - t0
    finally:
        fdtd.set_threads(prev)
    cores = threads or int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": wl.cells * nt_sample / t / 1e9, "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
            "nt_sample": nt_sample, "nt": pb.nt,
            "sample": f"FP64 oracle, {nt_sample} of {pb.nt} steps of one source with the volumetric transform "
                      f"into {wl.freqs.size} frequencies on the full {wl.nx}x{wl.ny}x{wl.nz} grid "
                      f"(a gradient is 2 such runs per source); {t:.1f} s"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def gradient_step(eng, rho, src, rec, d_obs):
    """One gradient of the hot path for a source batch: coefficient set-up and forward run
    with the volumetric transform, misfit and residual, adjoint-source basis, adjoint run,
    cell gradient with respect to ln rho."""
    from paper_2211_16665_gb300.engine import misfit
    d, E = eng.fwd_model(rho, src, rec, keep_volume=True)
    phi, r = misfit(d_obs, d)
    basis, fit, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True, fit_target=1e-3)
    V = eng.adjoint_model(rho, rec, r, basis)
    g = eng.gradient(rho, E, V, wrt="lnrho")
    del E, V
    return phi, g, fit


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2211_16665_gb300 import _capi
    from paper_2211_16665_gb300 import dist as D
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine, _ptr, _stream

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    wl = make_workload(args.workload, rank, world, vti=args.vti, max_src=args.max_src)
    S_all = wl.src.n
    B = max(1, min(args.batch, S_all))
    nb = S_all // B
    batches = [wl.src.subset(list(range(b * B, (b + 1) * B))) for b in range(nb)]
    eng = Engine.from_workload(wl, max_src=B, vti=args.vti, order=args.order)
    nt, dt, prec = eng.nt, eng.dt, eng.precision
    rho = eng.model_tensor(wl.rho)
    rho_true = eng.model_tensor(wl.rho_true)
    # observed data of every batch (the true model; data-only runs end early at 1e-6)
    eng.set_early_stop(1e-6)
    d_obs = []
    for b in range(nb):
        d = eng.fwd_model(rho_true, batches[b], wl.rec).cpu().numpy()
        d_obs.append(torch.as_tensor(W.add_noise(d, wl.noise, wl.noise_seed + b), device=dev))
    eng.set_early_stop(0.0)
    torch.cuda.synchronize()

    def step(t, rho_in=None, d_in=None):
        b = t % nb
        phi, g, fit = gradient_step(eng, rho if rho_in is None else rho_in, batches[b], wl.rec,
                                    d_obs[b] if d_in is None else d_in)
        D.sum_over_ranks(g, phi)          # the one exchange: sum of the per-source gradients
        return phi, g, fit

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for t in range(args.warmup):
        step(t)
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
    for t in range(args.steps):
        phi, g, fit = step(args.warmup + t)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    launches = (_capi.launch_count() - n0) // args.steps
    clk = clocks.stop()
    ms = D.max_over_ranks(ms, device=dev)

    cell_updates = 2.0 * wl.cells * nt * B * world
    value = cell_updates / (ms / 1e3) / 1e9

    # the adjoint-source basis solve alone (part of every timed step above; it blocks until
    # its fit residual is on the host)
    torch.cuda.synchronize()
    tb = time.perf_counter()
    eng.estimate_adjoint_basis(gamma=1e-12, relative=True, fit_target=1e-3)
    basis_ms = (time.perf_counter() - tb) * 1e3

    # roofline: the stencil (split H + E pair or fused step) and the transform flush, timed
    # live with CUDA events on the stream they are launched on
    _, E = eng.fwd_model(rho, batches[0], wl.rec, keep_volume=True)
    kms = dict(zip(("k_h", "k_step", "k_e", "k_dft"), _capi.time_step_kernels(eng.ctx, B, _ptr(E), 100, _stream())))
    del E
    fused = kms["k_step"] > 0
    st_ms = kms["k_step"] if fused else kms["k_h"] + kms["k_e"]
    lc = eng.launch_config()
    st_name = ({"fused one-pass H+E": "k_step_fz", "fused warp-specialised H+E": "k_step_ws",
                "wave-ordered H+E": "k_step_wave"}.get(
        lc["step"]["kernel"], "k_step")) if fused else \
        "+".join(f"k_{w}_{lc['step'][w]['kernel'].split()[0]}" if eng.order == 2 else
                 (f"k_{w}_ho4" if lc["step"][w]["kernel"] == "lean" else f"k_{w}_ho") for w in ("h", "e"))
    b_cell = stencil_bytes(wl, eng)
    nodes = (wl.nx + 1) * (wl.ny + 1) * (wl.nz + 1)
    M = eng.flush_block()
    b_flush = flush_bytes(wl, eng)
    peak, peak_kind = hbm_peak()
    st_gbs = b_cell * wl.cells * B / (st_ms / 1e3) / 1e9
    fl_gbs = b_flush * nodes * B / (kms["k_dft"] / 1e3) / 1e9
    per_step = {"stencil": st_ms, "flush": kms["k_dft"] / M}
    # the floor of one gradient step per cell update: the stencil's bytes plus the flush's per
    # snapshot share (nodes per cell), both runs alike
    floor_update = b_cell + b_flush / M * nodes / wl.cells
    whole = floor_update * cell_updates / world / (ms / 1e3) / 1e9
    roof = {"kernel": st_name, "bound": "hbm", "achieved": round(st_gbs, 1), "peak": peak, "unit": "GB/s",
            "frac": round(st_gbs / peak, 4), "peak_kind": peak_kind,
            "traffic": ncu_traffic(wl, st_name, B),
            "bytes_per_unit": round(b_cell, 2), "unit_of_work": "cell (one H + E step, every source of the launch)",
            "units_per_launch": wl.cells * B, "ms_per_launch": round(st_ms, 5),
            "flush": {"kernel": ("k_dft_stream" if M >= 64 else "k_dft_bulk") if lc["flush"]["kernel"] == "bulk-copy"
                      else "k_dft",
                      "snapshots": M, "bytes_per_node": b_flush, "achieved": round(fl_gbs, 1),
                      "frac": round(fl_gbs / peak, 4), "ms_per_launch": round(kms["k_dft"], 5)},
            "step_share": {k: round(v / sum(per_step.values()), 3) for k, v in per_step.items()},
            "whole_step": {"bytes_per_cell_update": round(floor_update, 2), "achieved": round(whole, 1),
                           "frac": round(whole / peak, 4)}}

    # end to end: host model and data in, host gradient and misfit out, every step
    e2e = None
    if not args.no_e2e:
        k_e2e = max(1, min(args.steps, args.e2e_steps))
        rho_h = rho.cpu().pin_memory()
        dobs_h = [d.cpu().pin_memory() for d in d_obs]
        g_h = torch.empty(g.shape, dtype=g.dtype).pin_memory()
        phi_h = torch.empty((), dtype=torch.float64).pin_memory()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for t in range(k_e2e):
            r_dev = rho_h.to(dev, non_blocking=True)
            o_dev = dobs_h[t % nb].to(dev, non_blocking=True)
            phi2, g2, _ = step(t, r_dev, o_dev)
            g_h.copy_(g2, non_blocking=True)
            phi_h.copy_(phi2, non_blocking=True)
        e1.record(stream)
        barrier()
        ems = D.max_over_ranks(e0.elapsed_time(e1) / k_e2e, device=dev)
        e2e = {"value": round(cell_updates / (ems / 1e3) / 1e9, 3), "unit": "Gcell-updates/s",
               "ms_per_step": round(ems, 3), "steps": k_e2e,
               "h2d_bytes_per_step": int(rho_h.numel() * rho_h.element_size() +
                                         dobs_h[0].numel() * dobs_h[0].element_size()),
               "d2h_bytes_per_step": int(g_h.numel() * g_h.element_size() + 8)}

    # batched (B sources per launch, compensated transform) against the plain path (one
    # source per launch, plain FP32 transform) on the sources of the first batch, and each
    # path's gradient against the FP64 engine on the first sources
    bvp = None
    if rank == 0 and not args.no_plain and B > 1:
        eng.close()
        del eng
        torch.cuda.empty_cache()
        ep = Engine.from_workload(wl, max_src=1, kahan=0, vti=args.vti, order=args.order)
        rp = ep.model_tensor(wl.rho)
        singles = [batches[0].subset([u]) for u in range(B)]
        gradient_step(ep, rp, singles[0], wl.rec, d_obs[0][:1].contiguous())      # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for u in range(B):
            gradient_step(ep, rp, singles[u], wl.rec, d_obs[0][u:u + 1].contiguous())
        e1.record(stream)
        torch.cuda.synchronize()
        plain_s = e0.elapsed_time(e1) / 1e3 / B
        bvp = {"batched": {"s_per_source": round(ms / 1e3 / B, 4), "sources_per_launch": B, "kahan": True,
                           "launch": lc},
               "plain": {"s_per_source": round(plain_s, 4), "sources_per_launch": 1, "kahan": False,
                         "launch": ep.launch_config()},
               "batched_over_plain": round(plain_s / (ms / 1e3 / B), 4)}
        if args.check_sources > 0:
            k = min(args.check_sources, B)
            grads = {}
            gp = torch.zeros_like(g)
            for u in range(k):
                gp += gradient_step(ep, rp, singles[u], wl.rec, d_obs[0][u:u + 1].contiguous())[1]
            grads["plain"] = gp.double().cpu().numpy()
            ep.close()
            del ep
            torch.cuda.empty_cache()
            for name, prec, kahan in (("fp64", 64, 0), ("batched", 32, 1)):
                e = Engine.from_workload(wl, max_src=k, precision=prec, kahan=kahan, vti=args.vti, order=args.order)
                sub = batches[0].subset(list(range(k)))
                gg = gradient_step(e, e.model_tensor(wl.rho), sub, wl.rec, d_obs[0][:k].contiguous())[1]
                grads[name] = gg.double().cpu().numpy()
                e.close()
                del e
                torch.cuda.empty_cache()
            ref = grads["fp64"]
            for name in ("batched", "plain"):
                bvp[name]["grad_rel_l2_vs_fp64"] = float(np.linalg.norm(grads[name] - ref) / np.linalg.norm(ref))
            bvp["checked_sources"] = k
        else:
            ep.close()
    else:
        eng.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_steps, args.order)

    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 3), "unit": "Gcell-updates/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == 32 else "f64",
               "data": "synthetic",
               "config": {"workload": wl.name, "cells": wl.cells, "grid": [wl.nx, wl.ny, wl.nz], "nt": nt, "dt": dt,
                          "n_src_per_gpu": S_all, "sources_per_step": B, "batches": nb,
                          "n_rec": wl.rec.n, "freqs_hz": list(map(float, wl.freqs)),
                          "kahan": True, "launch": lc,
                          "l2": "inputs larger than L2 (each step streams "
                          f"{2 * 3 * wl.freqs.size * nodes * 8 * B * 2 / 2**20:.0f} MiB of transform volumes and "
                          f"{2 * 6 * wl.cells * 4 * B / 2**20:.0f} MiB of fields per time step)",
                          "parallelism": f"sources sharded, dp{world}",
                          "medium": "vti" if args.vti else "isotropic", "order": args.order},
               "grad_s_per_source": round(ms / 1e3 / B, 4),
               "batched_vs_plain": bvp,
               "basis_fit": fit, "basis_ms": round(basis_ms, 3),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
               "clocks": clk}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
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
    # calibrate: size each step so that warmup + steps take --ref-seconds (2.5 minutes by default)
    t0 = time.perf_counter()
    fdtd.forward(pb, wl.rho, src, wl.rec, keep_volume=True, nt_run=3)
    per = (time.perf_counter() - t0) / 3
    nt_s = int(max(5, min(pb.nt, args.ref_seconds / max(1, args.steps + args.warmup) / per)))
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
    from paper_2211_16665_gb300 import workloads as W
    from paper_2211_16665_gb300.engine import Engine, misfit
    torch.cuda.set_device(0)
    all_threads = os.cpu_count() or 1
    out = {"mode": "oracle_timings", "host_cores": all_threads, "rows": []}
    for name, nt_sample in (("plain_tiny", 300), ("thin_reservoir", 200), ("heterogeneous_crop96", 200)):
        wl = W.ALL[name]()
        row = {"workload": wl.name, "cells": wl.cells, "precision": wl.precision}
        for threads in (1, all_threads):         # the cpu_baseline leg on one and on all host threads
            cb = cpu_baseline(wl, nt_sample, threads=threads)
            row[f"oracle_gcell_s_{threads}_threads"] = round(cb["value"], 5)
        row["oracle_sample"] = f"{cb['nt_sample']} of {cb['nt']} steps, one source, volumetric transform"
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
    out = {"mode": "early_stop_volumes", "workload": wl.name, "nt": eng.nt, "tol": args.early_stop_volumes,
           "floor": args.es_floor}
    grads = {}
    for name, tol in (("full", 0.0), ("early", args.early_stop_volumes)):
        eng.set_early_stop_volumes(tol, args.es_floor)

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


def run_batch_sweep(args):
    """Gradient seconds per source against the sources per launch: each batch size gets its
    own context (ring sized against free memory, autotuned kernels and flush), one warm-up
    gradient and args.steps timed ones over the first B sources of the workload; the plain
    path (1 source, no compensation) last."""
    import torch
    from paper_2211_16665_gb300.engine import Engine
    torch.cuda.set_device(0)
    wl = make_workload(args.workload, 0, 1)
    sizes = [int(v) for v in args.batch_sweep.split(",") if v.strip()]
    runs = [(B, 1) for B in sizes] + [(1, 0)]
    for B, kahan in runs:
        B = min(B, wl.src.n)
        src = wl.src.subset(list(range(B)))
        eng = Engine.from_workload(wl, max_src=B, kahan=kahan, nt=args.nt)
        rho, rho_t = eng.model_tensor(wl.rho), eng.model_tensor(wl.rho_true)
        eng.set_early_stop(1e-6)
        d_obs = eng.fwd_model(rho_t, src, wl.rec)
        eng.set_early_stop(0.0)
        gradient_step(eng, rho, src, wl.rec, d_obs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            gradient_step(eng, rho, src, wl.rec, d_obs)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3 / args.steps
        print(json.dumps({"mode": "batch_sweep", "workload": wl.name, "nt": eng.nt, "sources_per_launch": B,
                          "kahan": bool(kahan), "s_per_gradient": round(s, 4), "s_per_source": round(s / B, 5),
                          "gcell_updates_per_s": round(2.0 * wl.cells * eng.nt * B / s / 1e9, 3),
                          "launch": eng.launch_config()}), flush=True)
        eng.close()
        del eng
        torch.cuda.empty_cache()


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
    if args.batch_sweep:
        run_batch_sweep(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
