"""The allocation-free adjoint-basis entry point.

Callers that cannot allocate device memory (an application whose memory
belongs to another allocator, or a path where an allocation's implicit
synchronisation is not acceptable) use csem_estimate_adjoint_basis_noalloc,
whose scratch is a static device array inside the library.  These tests call
it through the C ABI and check it against csem_estimate_adjoint_basis, the
allocating entry point, on two calls in a row (the static array is shared by
every call and must not leak one call's values into the next), plus its size
limit.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2211_16665_gb300 import _capi  # noqa: E402


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _rel_l2(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


CASES = [
    # (dt, nt, freqs): the paper's worked example, the thin-reservoir workload's set, and the
    # 400x400x200 workload's eight log-spaced frequencies over 19 492 steps (a 16-column basis)
    (0.004, 1000, [0.25, 0.75, 2.25]),
    (9.0374e-4, 12328, [0.25, 0.5, 0.75, 1.0]),
    (9.0374e-4, 19492, list(np.logspace(np.log10(0.1), np.log10(1.5), 8))),
]


def test_noalloc_matches_allocating_entry_point_twice_in_a_row():
    for (dt, nt, freqs) in CASES:
        ref = torch.empty((nt, 2 * len(freqs)), dtype=torch.float64, device="cuda")
        fit_r, its_r = _capi.estimate_adjoint_basis(dt, nt, freqs, 1.0, 1e-12, 1, 200, 1e-15, _vp(ref), _stream())
        for call in range(2):
            out = torch.full_like(ref, float("nan"))
            fit, its = _capi.estimate_adjoint_basis_noalloc(dt, nt, freqs, 1.0, 1e-12, 1, 200, 1e-15, _vp(out),
                                                            _stream())
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            # the same kernels on the same inputs: within the basis tolerance of the parity tests (1e-7)
            assert _rel_l2(out, ref) <= 1e-7, (call, _rel_l2(out, ref))
            assert abs(fit - fit_r) <= 1e-6 + 1e-3 * fit_r
            assert its == its_r


def test_noalloc_rejects_sizes_beyond_its_array():
    out = torch.empty((40000, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(_capi.CsemError) as e:
        _capi.estimate_adjoint_basis_noalloc(1e-3, 40000, [0.5], 1.0, 1e-12, 1, 50, 1e-14, _vp(out), _stream())
    assert e.value.code == _capi.ERR_INVALID_ARG
    assert "nt <= 32768" in str(e.value)
