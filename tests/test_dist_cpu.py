"""Host logic of the source-parallel path on CPU: sharding covers every source
exactly once, and two gloo ranks that each sum a per-source contribution end
with the serial total (gradient volume and misfit), and agree on the maximum
time."""
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
