"""Failure detection of the bulk-copy kernels on the GPU, without a fault.

Every wait of a kernel on the barrier of its shared-memory copies is bounded
(about a second).  The test hook csem_set_copy_fault makes the first stage of
every block expect 16 bytes more than its copies bring, so that wait runs out:
the block leaves without writing, the kernel returns, and csem_check reports
CSEM_ERR_TIMEOUT naming the kernel family.  The context stays usable: with the
hook off, the next run gives the results of an engine that never saw the hook,
bit for bit.  Covered: the transform flush (16 snapshots held at once, and 64
streamed through a ring of stages), the row-staged H/E step kernels and the
fused one-pass step kernel; the warp-specialised fused step, whose producer
warps skip their first hand-over under the hook; and the wave-ordered step, whose E
tiles wait under the hook for one H tile more than there are (the first ones give
up, the rest skip the wait), after which its counters are back at zero for the next run.
"""
import dataclasses

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300._capi import CsemError  # noqa: E402
from paper_2211_16665_gb300.engine import Engine  # noqa: E402

TIMEOUT = -6

CASES = {
    # family: (launch configuration, steps per run, words the timeout message names[, frequencies])
    "flush": (dict(kz_h=2, mb_h=8, lean_h=2, kz_e=2, mb_e=8, lean_e=2, flush_mode=1, block=16), 16, "flush"),
    "streamed flush": (dict(kz_h=2, mb_h=8, lean_h=2, kz_e=2, mb_e=8, lean_e=2, flush_mode=1, block=64), 64, "flush"),
    # with eight frequencies the streamed flush reads its accumulators at the end, not on a barrier
    "streamed flush, 8 frequencies": (dict(kz_h=2, mb_h=8, lean_h=2, kz_e=2, mb_e=8, lean_e=2, flush_mode=1,
                                           block=64), 64, "flush", 8),
    "row-staged": (dict(kz_h=4, mb_h=4, kz_e=4, mb_e=4, tma_h=2, tma_e=2, flush_mode=0, block=16), 2, "row-staged"),
    "one-pass": (dict(onepass=(8, 4, 4), flush_mode=0, block=16), 2, "one-pass"),
    "warp-specialised": (dict(wspec=(8, 4, 3), flush_mode=0, block=16), 2, "warp-specialised"),
    "wave-ordered": (dict(wave=(2, 4, 8), flush_mode=0, block=16), 2, "wave-ordered"),
}


@pytest.mark.parametrize("family", list(CASES))
def test_bounded_wait_reports_timeout_and_context_recovers(family):
    launch, nt, word = CASES[family][:3]
    wl = W.small_box(n_core=24, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2)
    if len(CASES[family]) > 3:
        wl = dataclasses.replace(wl, freqs=np.linspace(0.25, 1.5, CASES[family][3]))

    def engine():
        e = Engine.from_workload(wl, precision=32, kahan=1, autotune=False, nt=nt)
        e.set_launch(**launch)
        return e

    ref = engine()
    rho = ref.model_tensor(wl.rho)
    d_ref, E_ref = ref.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    ref.check()
    eng = engine()
    eng.set_copy_fault(16)
    eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    with pytest.raises(CsemError) as err:
        eng.check()
    assert err.value.code == TIMEOUT and word in str(err.value)
    eng.set_copy_fault(0)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    eng.check()
    assert torch.equal(d, d_ref) and torch.equal(E, E_ref)
    with pytest.raises(CsemError):
        eng.set_copy_fault(8)            # not a multiple of 16
    eng.close()
    ref.close()
