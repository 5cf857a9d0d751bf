"""Host logic of the source-parallel path on CPU: sharding covers every source
exactly once; two gloo ranks that each sum a per-source contribution end with
the serial total and agree on the maximum time; and two gloo ranks that each
compute the FP64 oracle's gradient of their share of a towline (the sharding
bench.py uses) sum to the serial oracle gradient of the whole towline."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2211_16665_gb300 import dist as D
from paper_2211_16665_gb300 import workloads as W


def test_shard_covers_every_item_once():
    for n in (1, 2, 5, 32, 64, 100):
        for world in (1, 2, 3, 4, 8):
            seen = []
            sizes = []
            for r in range(world):
                sh = D.shard(n, r, world)
                seen += list(sh)
                sizes.append(len(sh))
            assert seen == list(range(n))
            assert max(sizes) - min(sizes) <= 1


def test_towline_spacing_and_centre():
    p = D.towline(W.Points.make([[100.0, 5.0, 950.0]], 0), 4)
    assert np.allclose(np.diff(p.x), 250.0) and p.x[2] == 100.0 and np.all(p.z == 950.0)


def _per_source(s, shape):
    rng = np.random.default_rng(1000 + s)
    return rng.standard_normal(shape), float(rng.uniform())


def _worker(rank, world, port, n_src, shape, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = torch.zeros(shape, dtype=torch.float64)
    phi = torch.zeros((), dtype=torch.float64)
    for s in D.shard(n_src, rank, world):
        gs, ps = _per_source(s, shape)
        g += torch.from_numpy(gs)
        phi += ps
    D.sum_over_ranks(g, phi)
    t = D.max_over_ranks(float(rank + 1))
    out[rank] = (g.numpy().copy(), float(phi), t)
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n_src", [2, 5])
def test_two_gloo_ranks_sum_the_source_gradients(n_src):
    shape = (3, 4, 5)
    mgr = mp.Manager()
    out = mgr.dict()
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), n_src, shape, out), nprocs=world, join=True)
    g_ref = sum(_per_source(s, shape)[0] for s in range(n_src))
    phi_ref = sum(_per_source(s, shape)[1] for s in range(n_src))
    for r in range(world):
        g, phi, t = out[r]
        assert np.allclose(g, g_ref, rtol=1e-12, atol=1e-12)
        assert abs(phi - phi_ref) <= 1e-12
        assert t == float(world)


def _oracle_box():
    from oracle import fdtd
    wl = W.small_box(n_core=8, h=100.0, npml=4, ratio=1.05, n_st=2, n_rec=4, n_freq=2, nt=240)
    return wl, fdtd.problem_from_workload(wl)


def _oracle_gradient(wl, pb, src):
    """Per-batch FP64 oracle gradient (ln rho) and misfit of the method's hot path."""
    from oracle import fdtd
    d_obs = fdtd.forward(pb, wl.rho_true, src, wl.rec)
    d, E = fdtd.forward(pb, wl.rho, src, wl.rec, keep_volume=True)
    phi, r = fdtd.misfit(d_obs, d)
    Bp, _ = fdtd.adjoint_basis(pb, 1e-12)
    V = fdtd.adjoint(pb, wl.rho, wl.rec, r, Bp)
    return fdtd.gradient(pb, wl.rho, E, V, wrt="lnrho"), float(phi)


def _gradient_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import fdtd
    fdtd.set_threads(2)
    wl, pb = _oracle_box()
    src = D.rank_sources(wl.src, rank, world)          # the sharding bench.py uses under torchrun
    g, phi = _oracle_gradient(wl, pb, src)
    gt = torch.from_numpy(np.ascontiguousarray(g))
    pt = torch.tensor(phi, dtype=torch.float64)
    D.sum_over_ranks(gt, pt)
    out[rank] = (gt.numpy().copy(), float(pt), list(map(float, src.x)))
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_oracle_gradients_to_the_serial_gradient():
    """Each rank takes its share of a towline (the bench's weak-scaling sharding), computes
    the FP64 oracle's gradient and misfit for it, and one all-reduce gives every rank the
    serial gradient of all the towline's sources."""
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_gradient_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    wl, pb = _oracle_box()
    line = D.towline(wl.src, world * wl.src.n)
    g_ref, phi_ref = _oracle_gradient(wl, pb, line)
    xs = sorted(x for r in range(world) for x in out[r][2])
    assert xs == sorted(map(float, line.x))            # every towline source modelled exactly once
    for r in range(world):
        g, phi, _ = out[r]
        assert np.abs(g - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
        assert abs(phi - phi_ref) <= 1e-12 * abs(phi_ref)
