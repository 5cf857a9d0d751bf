"""Writes thin_reservoir_oracle.json: FP64 oracle outputs for the full-size
thin-reservoir workload (128x128x96 cells, nt from the CFL step, 4 frequencies,
1 source, 41 receivers), used by the full-size GPU parity test.

Calls only `oracle/` (and the seeded input generators).  Stored:
  * d_obs (true model, before noise) and d_syn (starting model) at the receivers;
  * the misfit with the 1 % seeded noise, and the basis fit;
  * the ln(rho) gradient at 600 cells (the 300 largest |g| and 300 seeded
    random core cells) and its global L2 norm.
Takes ~30 min on 8 cores.

    python tests/golden/make_thin_reservoir_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fdtd  # noqa: E402
from paper_2211_16665_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "thin_reservoir_oracle.json")


def cplx(a):
    a = np.asarray(a)
    return {"re": a.real.tolist(), "im": a.imag.tolist()}


def main():
    t0 = time.time()
    wl = W.thin_reservoir()
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d_obs_noisy = W.add_noise(d_obs, wl.noise, wl.noise_seed)
    d_syn, E = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs_noisy, d_syn)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho")
    flat = g.ravel()
    top = np.argsort(-np.abs(flat))[:300]
    rng = np.random.default_rng(0)
    nz, ny, nx = g.shape
    core = []
    while len(core) < 300:
        k, j, i = rng.integers(10, nz - 10), rng.integers(10, ny - 10), rng.integers(10, nx - 10)
        c = (k * ny + j) * nx + i
        if c not in core and c not in set(top.tolist()):
            core.append(int(c))
    cells = [int(c) for c in top] + core
    out = {
        "what": "FP64 oracle, thin_reservoir workload, full size",
        "dt": pb.dt, "nt": pb.nt, "freqs": wl.freqs.tolist(),
        "d_obs": cplx(d_obs[0]), "d_obs_noisy": cplx(d_obs_noisy[0]), "d_syn": cplx(d_syn[0]),
        "phi": phi, "basis_fit": fit,
        "grad_cells": cells, "grad_values": flat[cells].tolist(), "grad_norm": float(np.linalg.norm(flat)),
        "seconds": time.time() - t0,
    }
    json.dump(out, open(OUT, "w"))
    print(f"wrote {OUT} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
