"""Multi-rank VMC exchange (global energy statistics, gradient weights and the
gradient sum) on two gloo ranks on the CPU, against the single-process
oracle on all samples.  The per-rank gradients come from the oracle's reverse
sweep, so this checks the exchange the GPU step uses, not the kernels."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import model as om, vmc as ov
from paper_2507_18700_gb300 import dist as vdist, inputs

N, D, B_RANK, WORLD = 10, 8, 24, 2


def _data():
    mod = om.Model(om.GRU1D, N, d_h=D)
    pf = inputs.xavier_params(1, D, seed=3, noise_std=0.1)
    sig = inputs.random_configs(B_RANK * WORLD, N, seed=4).astype(np.int64)
    e = inputs.random_weights(B_RANK * WORLD, seed=5, scale=2.0) - 7.0
    return mod, pf, sig, e


def _rank(rank, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        mod, pf, sig, e = _data()
        lo, hi = rank * B_RANK, (rank + 1) * B_RANK
        eloc = torch.tensor(e[lo:hi], dtype=torch.float32)
        stats = vdist.global_energy_stats(eloc)
        w = vdist.vmc_weights(eloc, stats)
        g = torch.tensor(ov.logpsi_grad(mod, pf, sig[lo:hi], w.double().numpy()))
        vdist.allreduce_grad(g)
        q.put((rank, stats.numpy(), w.numpy(), g.numpy(), vdist.rank_seed(11)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_exchange_matches_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = dict((r, rest) for r, *rest in (q.get(timeout=120) for _ in range(WORLD)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mod, pf, sig, e = _data()
    e = e.astype(np.float32).astype(np.float64)        # the ranks hold float32 energies, as on the GPU
    ref_stats = ov.energy_stats(e)
    ref_grad = ov.vmc_gradient(mod, pf, sig, e)
    w_ref = 2.0 * (e - e.mean()) / e.size
    for r in range(WORLD):
        stats, w, g, seed = out[r]
        np.testing.assert_allclose(stats, ref_stats, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(w, w_ref[r * B_RANK:(r + 1) * B_RANK], rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(g, ref_grad, rtol=1e-6, atol=1e-9)
    assert out[0][3] != out[1][3]            # distinct sampling streams per rank
