"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances (relative L2 over all outputs of a kind):
  FP64 stencil: 1e-10 (same arithmetic, rounding order only);
  FP32 stencil: receivers 1e-5, volumes / gradient 1e-3 (the targets stated
  for the hot path; the FP32 field over a few thousand lossless steps carries
  ~1e-6 relative round-off).
Sizes span several thread blocks in every direction and ragged tails.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import fdtd  # noqa: E402
from paper_2211_16665_gb300 import workloads as W  # noqa: E402
from paper_2211_16665_gb300.engine import Engine, misfit  # noqa: E402
from paper_2211_16665_gb300._capi import CsemError  # noqa: E402


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_volume(eng, v):
    """[S,3,F,NZ,NY,pitch] device -> numpy [S,3,F,NZ,NY,NX]."""
    return v.cpu().numpy()[..., : eng.nx + 1].astype(np.complex128)


@pytest.fixture(scope="module")
def box():
    wl = W.small_box(n_core=24, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2)
    pb = fdtd.problem_from_workload(wl)
    return wl, pb


@pytest.fixture(scope="module")
def box_oracle(box):
    wl, pb = box
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E, tr = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True, return_trace=True)
    phi, r = fdtd.misfit(d_obs, d)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho")
    gs = fdtd.gradient(pb, wl.rho, E, V, wrt="sigma")
    return dict(d_obs=d_obs, d=d, E=E, tr=tr, phi=phi, r=r, Bp=Bp, V=V, g=g, gs=gs)


@pytest.mark.parametrize("precision", [64, 32])
def test_forward_receivers_traces_volumes(box, box_oracle, precision):
    wl, pb = box
    o = box_oracle
    eng = Engine.from_workload(wl, precision=precision, kahan=1)
    assert abs(eng.dt - pb.dt) <= 1e-14 * pb.dt and eng.nt == pb.nt
    rho = eng.model_tensor(wl.rho)
    d, E, tr = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True, trace=True)
    torch.cuda.synchronize()
    tol_r, tol_v = (1e-10, 1e-10) if precision == 64 else (1e-5, 1e-3)
    assert rel_l2(tr.cpu().numpy(), o["tr"]) <= (1e-10 if precision == 64 else 1e-4)
    assert rel_l2(d.cpu().numpy(), o["d"]) <= tol_r
    Eg = gpu_volume(eng, E)
    assert rel_l2(Eg, o["E"]) <= tol_v
    # row padding and off-lattice entries stay zero
    assert torch.count_nonzero(E[..., eng.nx + 1:]) == 0
    eng.check()
    eng.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_adjoint_and_gradient(box, box_oracle, precision):
    wl, pb = box
    o = box_oracle
    eng = Engine.from_workload(wl, precision=precision, kahan=1)
    rho = eng.model_tensor(wl.rho)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    d_obs = torch.as_tensor(o["d_obs"], device=eng.device)
    phi, r = misfit(d_obs, d)
    phi_tol = 1e-4 if precision == 32 else 1e-10
    assert abs(phi.item() - o["phi"]) <= phi_tol * o["phi"]
    basis, fit, its = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    assert rel_l2(basis.cpu().numpy(), o["Bp"]) <= 1e-7
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    tol = 1e-9 if precision == 64 else 1e-3
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= tol
    g = eng.gradient(rho, E, V, wrt="lnrho")
    gs = eng.gradient(rho, E, V, wrt="sigma")
    assert rel_l2(g.cpu().numpy(), o["g"]) <= tol
    assert rel_l2(gs.cpu().numpy(), o["gs"]) <= tol
    eng.close()


LAUNCH_VARIANTS = [
    dict(kz_h=1, mb_h=8, kz_e=4, mb_e=6, fused_kz=0, flush_mode=0, block=16),
    dict(kz_h=2, mb_h=4, kz_e=1, mb_e=6, vec_h=1, vec_e=1, flush_mode=1, block=32),
    dict(kz_h=8, mb_h=6, kz_e=4, mb_e=4, vec_h=1, vec_e=0, flush_mode=1, block=16),
    dict(kz_h=4, mb_h=8, kz_e=8, mb_e=4, vec_h=0, vec_e=1, flush_mode=0, block=16),
    dict(kz_h=4, mb_h=4, kz_e=2, mb_e=4, tma_h=4, tma_e=4, flush_mode=1, block=32),
    dict(kz_h=16, mb_h=4, kz_e=8, mb_e=4, tma_h=1, tma_e=2, flush_mode=1, block=16),
    dict(kz_h=2, mb_h=4, kz_e=16, mb_e=4, tma_h=2, tma_e=1, vec_h=0, flush_mode=0, block=16),
    dict(kz_h=8, mb_h=4, kz_e=2, mb_e=4, fused_kz=0, flush_mode=1, block=16),
    dict(fused_kz=4, flush_mode=1, block=32),
    dict(fused_kz=8, flush_mode=0, block=16),
    dict(fused_kz=16, flush_mode=1, block=16),
    dict(kz_h=1, mb_h=4, kz_e=4, mb_e=6, vec_h=1, flush_mode=3, block=32),
    dict(kz_h=2, mb_h=6, kz_e=2, mb_e=4, vec_e=1, flush_mode=3, block=16),
    dict(kz_h=4, mb_h=4, kz_e=4, mb_e=4, flush_mode=2, block=16),
    dict(fused_kz=8, flush_mode=3, block=32),
    dict(kz_h=1, mb_h=8, lean_h=1, kz_e=1, mb_e=6, lean_e=1, flush_mode=3, block=32),
    dict(kz_h=2, mb_h=6, lean_h=2, kz_e=4, mb_e=4, lean_e=2, flush_mode=1, block=16),
    dict(kz_h=2, mb_h=8, lean_h=2, kz_e=2, mb_e=6, lean_e=2, flush_mode=1, block=64),
    dict(kz_h=2, mb_h=4, lean_h=2, kz_e=1, mb_e=4, lean_e=2, flush_mode=3, block=64),
    dict(kz_h=4, mb_h=4, kz_e=4, mb_e=6, flush_mode=0, block=64),
    dict(onepass=(8, 4, 4), flush_mode=1, block=32),
    dict(onepass=(16, 8, 2), flush_mode=3, block=16),
    dict(onepass=(5, 4, 6), flush_mode=0, block=64),
    dict(onepass=(64, 8, 3), flush_mode=1, block=16),
    dict(kz_h=4, mb_h=8, lean_h=2, kz_e=4, mb_e=8, lean_e=2, flush_mode=1, block=128),
    dict(kz_h=4, mb_h=4, kz_e=4, mb_e=4, flush_mode=0, block=128),
    dict(wspec=(8, 4, 3), flush_mode=1, block=32),
    dict(wspec=(16, 8, 2), flush_mode=3, block=16),
    dict(wave=(2, 4, 8), flush_mode=1, block=32),
    dict(wave=(1, 2, 6), flush_mode=3, block=16),
    dict(wave=(4, 4, 6), flush_mode=0, block=64),
    dict(wave=(99, 2, 8), flush_mode=1, block=128),     # lag beyond the z blocks: every H tile first
]

LEAN_VARIANTS = [
    dict(kz_h=1, mb_h=6, lean_h=1, kz_e=1, mb_e=8, lean_e=1, flush_mode=3, block=32),
    dict(kz_h=2, mb_h=4, lean_h=2, kz_e=4, mb_e=6, lean_e=2, flush_mode=1, block=16),
    dict(kz_h=4, mb_h=6, lean_h=1, kz_e=2, mb_e=8, lean_e=2, flush_mode=0, block=16),
    dict(kz_h=1, mb_h=6, lean_h=2, kz_e=4, mb_e=8, lean_e=1, flush_mode=2, block=16),
    dict(kz_h=4, mb_h=8, lean_h=1, vec_e=1, kz_e=1, mb_e=4, flush_mode=3, block=16),
    dict(onepass=(8, 4, 4), flush_mode=1, block=16),
    dict(onepass=(3, 8, 2), flush_mode=3, block=32),
    dict(onepass=(16, 4, 6), flush_mode=0, block=16),
    dict(onepass=(44, 8, 3), flush_mode=1, block=64),
    dict(wspec=(8, 4, 3), flush_mode=1, block=16),
    dict(wspec=(3, 4, 2), flush_mode=3, block=32),
    dict(wspec=(16, 6, 2), flush_mode=0, block=16),
    dict(wspec=(44, 8, 1), flush_mode=1, block=64),
    dict(wspec=(5, 8, 2), flush_mode=1, block=16),
    dict(wave=(1, 4, 8), flush_mode=1, block=16),
    dict(wave=(3, 2, 6), flush_mode=3, block=32),
    dict(wave=(2, 4, 6), flush_mode=0, block=64),
]


@pytest.fixture(scope="module")
def ragged():
    """52 x 45 x 43 cells: ragged for 1 or 2 cells per thread over 32-thread rows,
    8-row blocks and 2- or 4-plane z blocks."""
    wl = W.small_box(n_core=28, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2, n_core_y=21, n_core_z=19)
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E, tr = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True, return_trace=True)
    phi, r = fdtd.misfit(d_obs, d)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho")
    return wl, dict(d_obs=d_obs, d=d, E=E, tr=tr, V=V, g=g)


@pytest.mark.parametrize("variant", range(len(LEAN_VARIANTS)))
def test_lean_kernels_match_oracle_on_a_ragged_box(ragged, variant):
    wl, o = ragged
    eng = Engine.from_workload(wl, precision=32, kahan=1, autotune=False)
    eng.set_launch(**LEAN_VARIANTS[variant])
    rho = eng.model_tensor(wl.rho)
    d, E, tr = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True, trace=True)
    assert rel_l2(tr.cpu().numpy(), o["tr"]) <= 1e-4
    assert rel_l2(d.cpu().numpy(), o["d"]) <= 1e-5
    Eg = gpu_volume(eng, E)
    assert rel_l2(Eg, o["E"]) <= 1e-3
    assert torch.count_nonzero(E[..., eng.nx + 1:]) == 0
    basis, _, _ = eng.estimate_adjoint_basis()
    d_obs = torch.as_tensor(o["d_obs"], device=eng.device)
    phi, r = misfit(d_obs, d)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= 1e-3
    assert rel_l2(eng.gradient(rho, E, V).cpu().numpy(), o["g"]) <= 1e-3
    eng.check()
    eng.close()


def test_lean_kernels_refused_where_they_do_not_apply():
    odd = W.small_box(n_core=20, h=100.0, npml=8, ratio=1.05, n_st=3, n_rec=6, n_freq=2)   # nx = 42
    assert odd.nx % 4 != 0
    eng = Engine.from_workload(odd, precision=32, autotune=False)
    with pytest.raises(CsemError):
        eng.set_launch(kz_h=1, mb_h=8, lean_h=1)
    eng.close()
    box = W.small_box(n_core=24, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2)
    eng = Engine.from_workload(box, precision=64, autotune=False)
    with pytest.raises(CsemError):
        eng.set_launch(kz_e=1, mb_e=4, lean_e=2)
    eng.close()
    eng = Engine.from_workload(box, precision=32, autotune=False)
    for bad in (dict(lean_h=3, kz_h=1), dict(lean_e=1, kz_e=8), dict(lean_h=1, kz_h=1, mb_h=4),
                dict(lean_e=2, kz_e=1, mb_e=3)):
        with pytest.raises(CsemError):
            eng.set_launch(**bad)
    eng.close()


def test_onepass_step_refused_where_it_does_not_apply():
    """The fused one-pass step needs FP32, second order, nx even and a supported block shape."""
    odd = W.small_box(n_core=21, h=100.0, npml=8, ratio=1.05, n_st=3, n_rec=6, n_freq=2)
    assert odd.nx % 2 == 1
    eng = Engine.from_workload(odd, precision=32, autotune=False)
    with pytest.raises(CsemError):
        eng.set_launch(onepass=(8, 4, 4))
    eng.close()
    box = W.small_box(n_core=24, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2)
    eng = Engine.from_workload(box, precision=64, autotune=False)
    with pytest.raises(CsemError):
        eng.set_launch(onepass=(8, 4, 4))
    eng.close()
    eng = Engine.from_workload(box, precision=32, autotune=False)
    for bad in ((8, 4, 3), (8, 2, 4), (1, 4, 4), (8, 8, 4)):
        with pytest.raises(CsemError):
            eng.set_launch(onepass=bad)
    eng.set_launch(onepass=(8, 8, 3))
    assert eng.launch_config()["step"] == {"kernel": "fused one-pass H+E", "z_planes": 8, "rows_per_block": 8,
                                           "blocks_per_sm": 3}
    for bad in ((8, 4, 4), (8, 6, 3), (1, 4, 3), (8, 2, 2)):
        with pytest.raises(CsemError):
            eng.set_launch(wspec=bad)
    eng.set_launch(wspec=(16, 6, 2))
    assert eng.launch_config()["step"] == {"kernel": "fused warp-specialised H+E", "z_planes": 16,
                                           "rows_per_block": 6, "blocks_per_sm": 2}
    eng.close()
    eng = Engine.from_workload(box, precision=64, autotune=False)
    with pytest.raises(CsemError):
        eng.set_launch(wspec=(8, 4, 3))
    with pytest.raises(CsemError):
        eng.set_launch(wave=(2, 4, 8))
    eng.close()


@pytest.mark.parametrize("wave", [(1, 4, 8), (2, 2, 6), (3, 4, 6), (99, 2, 8)])
def test_wave_step_is_bitwise_the_lean_pair(ragged, wave):
    """The wave-ordered step runs the lean H and E tiles' arithmetic in one launch, so a run
    with it equals a run with the split lean pair bit for bit (receivers, traces, volumes,
    adjoint volumes), on the ragged box with two sources per launch."""
    wl, o = ragged
    two = W.Points.make([[30.0, 0.0, wl.src.z[0]], [-250.0, 40.0, wl.src.z[0]]], 0)
    out = []
    for launch in (dict(kz_h=wave[1], mb_h=wave[2], lean_h=2, kz_e=wave[1], mb_e=wave[2], lean_e=2),
                   dict(wave=wave)):
        eng = Engine.from_workload(wl, precision=32, kahan=1, autotune=False, max_src=2)
        eng.set_launch(flush_mode=1, block=64, **launch)
        rho = eng.model_tensor(wl.rho)
        d, E, tr = eng.fwd_model(rho, two, wl.rec, keep_volume=True, trace=True)
        basis, _, _ = eng.estimate_adjoint_basis()
        V = eng.adjoint_model(rho, wl.rec, d, basis)
        eng.check()
        out.append((d.clone(), E.clone(), tr.clone(), V.clone()))
        eng.close()
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_wave_step_refused_where_it_does_not_apply():
    """The wave-ordered step needs FP32, second order, nx a multiple of 4, a lag of at least
    one z block, 2 or 4 planes and 6 or 8 blocks per SM."""
    odd = W.small_box(n_core=20, h=100.0, npml=8, ratio=1.05, n_st=3, n_rec=6, n_freq=2)   # nx = 42
    eng = Engine.from_workload(odd, precision=32, autotune=False)
    with pytest.raises(CsemError):
        eng.set_launch(wave=(2, 4, 8))
    eng.close()
    box = W.small_box(n_core=24, h=100.0, npml=8, ratio=1.08, n_st=4, n_rec=6, n_freq=2)
    eng = Engine.from_workload(box, precision=32, autotune=False, order=4)
    with pytest.raises(CsemError):
        eng.set_launch(wave=(2, 4, 8))
    eng.close()
    eng = Engine.from_workload(box, precision=32, autotune=False)
    for bad in ((0, 4, 8), (2, 8, 8), (2, 1, 8), (2, 4, 4), (2, 4, 7)):
        with pytest.raises(CsemError):
            eng.set_launch(wave=bad)
    eng.set_launch(wave=(3, 2, 6))
    assert eng.launch_config()["step"] == {"kernel": "wave-ordered H+E", "lag": 3, "z_planes": 2,
                                           "blocks_per_sm": 6}
    eng.close()


@pytest.mark.parametrize("variant", range(len(LAUNCH_VARIANTS)))
def test_every_launch_variant_matches_oracle(box, box_oracle, variant):
    """Split / fused step kernels and register / bulk-copy flushes give the oracle's results."""
    wl, pb = box
    o = box_oracle
    eng = Engine.from_workload(wl, precision=32, kahan=1, autotune=False)
    eng.set_launch(**LAUNCH_VARIANTS[variant])
    rho = eng.model_tensor(wl.rho)
    d, E, tr = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True, trace=True)
    assert rel_l2(tr.cpu().numpy(), o["tr"]) <= 1e-4
    assert rel_l2(d.cpu().numpy(), o["d"]) <= 1e-5
    assert rel_l2(gpu_volume(eng, E), o["E"]) <= 1e-3
    basis, _, _ = eng.estimate_adjoint_basis()
    d_obs = torch.as_tensor(o["d_obs"], device=eng.device)
    phi, r = misfit(d_obs, d)
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    assert rel_l2(gpu_volume(eng, V), o["V"]) <= 1e-3
    assert rel_l2(eng.gradient(rho, E, V).cpu().numpy(), o["g"]) <= 1e-3
    eng.check()
    eng.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("nt", [40, 64, 200, 0])
def test_overlapped_flush_is_bitwise_the_in_order_flush(box, precision, nt):
    """The transform flush on the side stream (overlapping the next block) gives
    the in-order flush's receivers, traces and volumes bit for bit: below one
    captured chunk, exactly one chunk, chunks plus a ragged remainder, the full nt."""
    wl, pb = box
    modes = [(0, 16), (2, 16), (0, 32), (2, 32), (0, 64), (2, 64)]
    if precision == 32:
        modes += [(1, 16), (3, 16), (1, 32), (3, 32), (1, 64), (3, 64)]
    out = {}
    for fm, m in modes:
        eng = Engine.from_workload(wl, precision=precision, kahan=1, autotune=False, nt=nt)
        eng.set_launch(kz_h=4, mb_h=4, kz_e=4, mb_e=4, flush_mode=fm, block=m)
        d, E, tr = eng.fwd_model(eng.model_tensor(wl.rho), wl.src, wl.rec, keep_volume=True, trace=True)
        out[(fm, m)] = (d.clone(), E.clone(), tr.clone())
        eng.check()
        eng.close()
    for (fm, m), got in out.items():
        if fm & 2:
            ref = out[(fm & 1, m)]
            for a, b in zip(got, ref):
                assert torch.equal(a, b), (fm, m)


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("nt", [40, 64, 100, 128, 192, 250, 320, 0])
def test_128_snapshot_flush_is_the_64_snapshot_sum(box, precision, nt):
    """With 128 snapshots per flush the chunks alternate between a graph without a flush and
    one that transforms both chunks' snapshots; an odd last chunk and the remainder are
    transformed together at the end.  Only the grouping of the sums changes: receivers (FP64)
    and traces equal the 64-snapshot run's to rounding, volumes within the compensated FP32
    grouping error, below one chunk, at whole and odd chunk counts, with remainders and at
    the full nt."""
    wl, pb = box
    kinds = [0, 1] if precision == 32 else [0]
    for fm in kinds:
        out = {}
        for m in (64, 128):
            eng = Engine.from_workload(wl, precision=precision, kahan=1, autotune=False, nt=nt)
            eng.set_launch(kz_h=4, mb_h=4, kz_e=4, mb_e=4, flush_mode=fm, block=m)
            assert eng.launch_config()["flush"]["snapshots"] == m
            d, E, tr = eng.fwd_model(eng.model_tensor(wl.rho), wl.src, wl.rec, keep_volume=True, trace=True)
            out[m] = (d.cpu().numpy(), gpu_volume(eng, E), tr.cpu().numpy())
            eng.check()
            eng.close()
        (d1, E1, t1), (d2, E2, t2) = out[64], out[128]
        assert np.array_equal(t1, t2)
        assert rel_l2(d2, d1) <= 1e-12
        assert rel_l2(E2, E1) <= (1e-12 if precision == 64 else 1e-6)


def test_early_end_runs_flush_at_most_64_snapshots(box):
    """Runs with an early end check after every 64-step chunk, so a context set to 128
    snapshots per flush transforms 64 at a time there: the same data and volumes as a
    context set to 64."""
    wl, pb = box
    out = {}
    for m in (64, 128):
        eng = Engine.from_workload(wl, precision=32, kahan=1, autotune=False)
        eng.set_launch(kz_h=4, mb_h=4, kz_e=4, mb_e=4, flush_mode=1, block=m)
        rho = eng.model_tensor(wl.rho)
        eng.set_early_stop(1e-6)
        d = eng.fwd_model(rho, wl.src, wl.rec)
        s1 = eng.last_run_steps()
        eng.set_early_stop(0.0)
        eng.set_early_stop_volumes(1e-6)
        dv, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
        s2 = eng.last_run_steps()
        eng.check()
        out[m] = (d.clone(), s1, dv.clone(), E.clone(), s2)
        eng.close()
    a, b = out[64], out[128]
    assert a[1] == b[1] and a[4] == b[4]
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])


def test_fused_and_split_steps_agree_in_fp64(box):
    wl, pb = box
    out = []
    for fused in (0, 8):
        eng = Engine.from_workload(wl, precision=64, autotune=False)
        eng.set_launch(fused_kz=fused)
        d, E = eng.fwd_model(eng.model_tensor(wl.rho), wl.src, wl.rec, keep_volume=True)
        out.append((d.cpu().numpy(), E.cpu().numpy()))
        eng.close()
    assert rel_l2(out[1][0], out[0][0]) <= 1e-13
    assert rel_l2(out[1][1], out[0][1]) <= 1e-13


def test_basis_matches_oracle_on_workload_sets():
    from oracle import basis as ob
    for (dt, nt, freqs) in ((0.004, 1000, [0.25, 0.75, 2.25]), (9.04e-4, 12328, [0.25, 0.5, 0.75, 1.0])):
        B = ob.basis_matrix(dt, nt, freqs, 1.0)
        g = ob.gamma_from_relative(B, 1e-12)
        ref = ob.pinv_pushthrough(B, g)
        eng_basis = torch.empty((nt, 2 * len(freqs)), dtype=torch.float64, device="cuda")
        from paper_2211_16665_gb300 import _capi
        import ctypes
        fit, its = _capi.estimate_adjoint_basis(dt, nt, freqs, 1.0, 1e-12, 1, 200, 1e-15,
                                                ctypes.c_void_p(eng_basis.data_ptr()),
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rel_l2(eng_basis.cpu().numpy(), ref) <= 1e-7
        assert abs(fit - ob.fit_residual(B, ref)) <= 1e-6 + 1e-3 * ob.fit_residual(B, ref)
        assert 1 <= its <= 200


def test_batched_equals_single_source_runs(box):
    wl, pb = box
    src = W.Points.make([[0.0, 0.0, wl.src.z[0]], [150.0, -120.0, wl.src.z[0]], [-260.0, 40.0, wl.src.z[0]]], [0, 1, 0])
    eng = Engine.from_workload(wl, precision=32, kahan=1, max_src=3)
    rho = eng.model_tensor(wl.rho)
    d3, E3 = eng.fwd_model(rho, src, wl.rec, keep_volume=True)
    for s in range(3):
        d1, E1 = eng.fwd_model(rho, src.subset([s]), wl.rec, keep_volume=True)
        assert torch.equal(d1[0], d3[s])
        assert torch.equal(E1[0], E3[s])
    eng.close()


def test_wavelet_invariance_on_gpu(box):
    wl, pb = box
    eng = Engine.from_workload(wl, precision=64)
    rho = eng.model_tensor(wl.rho_true)
    d_imp = eng.fwd_model(rho, wl.src, wl.rec).cpu().numpy()
    t = (np.arange(eng.nt) + 0.5) * eng.dt
    a = (np.pi * 5.0 * (t - 0.3)) ** 2
    eng.set_wavelet((1 - 2 * a) * np.exp(-a))
    d_ric = eng.fwd_model(rho, wl.src, wl.rec).cpu().numpy()
    assert rel_l2(d_ric, d_imp) <= 1e-9
    eng.close()


def test_plain_tiny_fp64_forward_adjoint_gradient():
    wl = W.plain_tiny()
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d, E = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs, d)
    Bp, fit = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    g = fdtd.gradient(pb, wl.rho, E, V)

    eng = Engine.from_workload(wl)
    assert eng.precision == 64 and eng.nt == 1500
    rho = eng.model_tensor(wl.rho)
    dg, Eg = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    assert rel_l2(dg.cpu().numpy(), d) <= 1e-10
    phig, rg = misfit(torch.as_tensor(d_obs, device="cuda"), dg)
    basis, fitg, _ = eng.estimate_adjoint_basis()
    Vg = eng.adjoint_model(rho, wl.rec, rg, basis)
    gg = eng.gradient(rho, Eg, Vg)
    assert rel_l2(gg.cpu().numpy(), g) <= 1e-8
    eng.close()


def test_error_statuses(box):
    wl, pb = box
    eng = Engine.from_workload(wl, precision=32)
    rho = eng.model_tensor(wl.rho)
    outside = W.Points.make([[1e6, 0.0, 500.0]], 0)
    with pytest.raises(CsemError) as e:
        eng.fwd_model(rho, outside, wl.rec)
    assert e.value.code == -2
    too_many = W.Points.make([[0.0, 0.0, 500.0]] * 2, 0)
    with pytest.raises(CsemError) as e:
        eng.fwd_model(rho, too_many, wl.rec)
    assert e.value.code == -1
    bad = rho.clone()
    bad[3, 4, 5] = float("nan")
    eng.fwd_model(bad, wl.src, wl.rec)
    with pytest.raises(CsemError) as e:
        eng.check()
    assert e.value.code == -5
    eng.close()
    with pytest.raises(CsemError) as e:
        Engine(wl.xn, wl.yn, wl.zn, wl.npml, wl.freqs, rho_max=wl.rho_max, dt=1.0)
    assert e.value.code == -3


@pytest.mark.parametrize("launch", [None, dict(kz_h=2, mb_h=8, lean_h=2, kz_e=2, mb_e=8, lean_e=2, flush_mode=1, block=64),
                                    dict(wspec=(8, 4, 3), flush_mode=1, block=16)])
def test_single_frequency_and_a_run_without_receivers(launch):
    """One frequency (the flush kernels' two-frequency padding, a two-column basis) through
    forward, adjoint and gradient against the oracle, autotuned and on the streamed 64-snapshot
    flush and the warp-specialised step; a forward run without receivers gives the same volumes."""
    wl = W.small_box(n_core=20, h=100.0, npml=6, ratio=1.08, n_st=2, n_rec=5, n_freq=1)
    pb = fdtd.problem_from_workload(wl)
    d_obs = fdtd.forward(pb, wl.rho_true, wl.src, wl.rec)
    d_o, E_o = fdtd.forward(pb, wl.rho, wl.src, wl.rec, keep_volume=True)
    phi_o, r_o = fdtd.misfit(d_obs, d_o)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    V_o = fdtd.adjoint(pb, wl.rho, wl.rec, r_o, Bp)
    g_o = fdtd.gradient(pb, wl.rho, E_o, V_o, wrt="lnrho")
    eng = Engine.from_workload(wl, precision=32, kahan=1, autotune=launch is None)
    if launch:
        eng.set_launch(**launch)
    rho = eng.model_tensor(wl.rho)
    d, E = eng.fwd_model(rho, wl.src, wl.rec, keep_volume=True)
    assert rel_l2(d.cpu().numpy(), d_o) <= 1e-5
    assert rel_l2(gpu_volume(eng, E), E_o) <= 1e-3
    phi, r = misfit(torch.as_tensor(d_obs, device=eng.device), d)
    basis, _, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    assert basis.shape[-1] == 2
    V = eng.adjoint_model(rho, wl.rec, r, basis)
    assert rel_l2(gpu_volume(eng, V), V_o) <= 1e-3
    assert rel_l2(eng.gradient(rho, E, V, wrt="lnrho").cpu().numpy(), g_o) <= 1e-3
    none = W.Points.make(np.zeros((0, 3)), 0)
    d0, E0 = eng.fwd_model(rho, wl.src, none, keep_volume=True)
    assert d0.shape[1] == 0 and torch.equal(E0, E)
    with pytest.raises(CsemError) as e:            # no sources: refused, nothing runs
        eng.fwd_model(rho, none, wl.rec)
    assert e.value.code == -1
    eng.check()
    eng.close()


def test_basis_fit_target_on_eight_widely_spaced_frequencies():
    """The Gram matrix of 8 log-spaced frequencies 0.1-1.5 Hz over 19 492 steps has a
    condition number near 1e12: gamma = 1e-12 relative leaves a fit residual of 0.19, and
    the fit target lowers gamma until the device basis fits the oracle's B to 1e-3."""
    from oracle import basis as OB
    wl = W.large_gradient()
    pb = fdtd.problem_from_workload(wl)
    M = OB.basis_matrix(pb.dt, pb.nt, pb.freqs, pb.f0)
    small = W.small_box(n_core=10, h=100.0, npml=4, n_freq=2)
    eng = Engine.from_workload(small, autotune=False)
    eng.dt, eng.nt, eng.freqs, eng.nf = pb.dt, pb.nt, np.asarray(pb.freqs), pb.freqs.size
    b12, fit12, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True)
    assert fit12 > 0.1 and abs(fit12 - OB.fit_residual(M, b12.cpu().numpy())) <= 1e-6
    b, fit, _ = eng.estimate_adjoint_basis(gamma=1e-12, relative=True, fit_target=1e-3)
    assert eng.basis_gamma < 1e-12 and fit <= 1e-3
    assert OB.fit_residual(M, b.cpu().numpy()) <= 1e-3
    eng.close()
