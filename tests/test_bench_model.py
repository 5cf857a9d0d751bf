"""The byte model the bench's roofline fractions are computed on (CPU): the stencil floor per
cell-update and the flush bytes per lattice node, for the workloads whose figures are quoted
(256x256x128 towline 62.0 B and 1152 B per 64 snapshots with compensation; thin reservoir
68.67 B; 512x512x256 heterogeneous model 57.0 B), and the traffic lookup that is null for a
kernel or workload that was not captured; and the reference arm's JSON line."""
import os
import types

import pytest

import bench
from paper_2211_16665_gb300 import workloads as W


def fake_engine(precision=32, vti=False, M=64, nf=4, kahan=1):
    return types.SimpleNamespace(precision=precision, vti=vti, nf=nf, info=types.SimpleNamespace(kahan=kahan),
                                 flush_block=lambda: M)


@pytest.mark.parametrize("name, floor", [("batched_towline", 62.0), ("thin_reservoir", 68.67),
                                         ("heterogeneous", 57.0)])
def test_stencil_floor(name, floor):
    wl = W.ALL[name]()
    assert bench.stencil_bytes(wl, fake_engine()) == pytest.approx(floor, abs=0.005)
    # one more conductivity per cell in a VTI medium; twice the bytes in FP64
    assert bench.stencil_bytes(wl, fake_engine(vti=True)) == pytest.approx(floor + 4.0, abs=0.005)
    assert bench.stencil_bytes(wl, fake_engine(precision=64)) == pytest.approx(2 * floor, abs=0.01)


def test_flush_bytes():
    wl = W.ALL["batched_towline"]()
    assert bench.flush_bytes(wl, fake_engine(M=64)) == 3 * 64 * 4 + 3 * 4 * 8 * 2 * 2 == 1152
    assert bench.flush_bytes(wl, fake_engine(M=32)) == 768
    assert bench.flush_bytes(wl, fake_engine(M=64, kahan=0)) == 960
    assert bench.flush_bytes(wl, fake_engine(M=64, nf=3)) == 1056


def test_traffic_lookup_only_for_the_captured_kernel():
    wl = W.ALL["batched_towline"]()
    per_launch = bench.ncu_traffic(wl, "k_h_lean+k_e_lean", 2)
    assert per_launch is None or per_launch == pytest.approx(1430.5e6)
    assert bench.ncu_traffic(wl, "k_step_fz", 2) is None
    assert bench.ncu_traffic(W.ALL["thin_reservoir"](), "k_h_lean+k_e_lean", 1) is None


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the FP64 oracle on the host (the reference of this
    build) and prints one JSON line with the keys the measurement contract names."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "plain_tiny", "--steps", "2", "--warmup", "1", "--ref-seconds", "2"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "Gcell-updates/s"
    assert line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 1
    assert line["config"]["workload"] and line["config"]["cells"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
