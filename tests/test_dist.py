"""Data-parallel VMC step on two gloo ranks on the CPU against one rank.

The library calls are replaced by a CPU stand-in built from the float64
oracle (sampling with the global sample offset, local energies by full
re-evaluation, the energy sums and the centred gradient share), so this checks
the exchange and the sample partition that ``paper_2507_18700_gb300.dist``
performs around the kernels: the two ranks together must draw bitwise the
samples of one rank with the whole batch, and reach the same statistics and
gradient.  The kernels' own pieces (nqs_energy_sums, nqs_vmc_grad_global,
the sample offset) are checked against the single-rank calls on the GPU in
tests/test_parity_dist_gpu.py.
"""
import os
import socket
import types

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import hamiltonian as oh, model as om, philox, vmc as ov
from paper_2507_18700_gb300 import dist as vdist, inputs

N, D, B_RANK, WORLD, SEED, STEP, GAMMA = 10, 8, 24, 2, 11, 3, 0.8


def _oracle_api():
    """CPU stand-in for the library calls dist.py makes (torch CPU tensors in and out)."""
    mod = om.Model(om.GRU1D, N, d_h=D)
    pf = inputs.xavier_params(1, D, seed=3, noise_std=0.1).astype(np.float32).astype(np.float64)

    def sample(desc, params, B, seed, step, ws=None, sample_offset=0):
        u = philox.sampling_uniforms(seed, step, B, N, sample_offset=sample_offset)
        s = om.sample(mod, pf, u)["sigma"]
        return torch.tensor(s.astype(np.uint8)), None, None

    def local_energy(desc, params, ham, sigma, hc, ws=None):
        s = sigma.numpy().astype(np.int64)
        e = oh.tfim_local_energy(N, 1.0, GAMMA, s, lambda x: om.logpsi(mod, pf, x))
        return torch.tensor(e, dtype=torch.float32)

    def energy_sums(eloc):
        e = eloc.double().numpy()
        return torch.tensor([e.sum(), (e * e).sum(), float(e.size)], dtype=torch.float64)

    def vmc_grad_global(desc, params, sigma, hc, eloc, sums, ws=None):
        M = float(sums[2])
        mean = float(sums[0]) / M
        stats = torch.tensor([mean, float(sums[1]) / M - mean * mean, M], dtype=torch.float64)
        w = 2.0 * (eloc.double().numpy() - mean) / M
        g = ov.logpsi_grad(mod, pf, sigma.numpy().astype(np.int64), w)
        return torch.tensor(g, dtype=torch.float64), stats

    return types.SimpleNamespace(sample=sample, local_energy=local_energy, energy_sums=energy_sums,
                                 vmc_grad_global=vmc_grad_global)


def _rank(rank, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        g, stats, sigma, eloc = vdist.vmc_step(None, None, None, B_RANK, SEED, STEP, api=_oracle_api())
        q.put((rank, g.numpy(), stats.numpy(), sigma.numpy(), eloc.numpy()))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_step_matches_one_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = dict((r, rest) for r, *rest in (q.get(timeout=180) for _ in range(WORLD)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # one rank with the whole batch (no process group: world size 1)
    g1, st1, s1, e1 = vdist.vmc_step(None, None, None, B_RANK * WORLD, SEED, STEP, api=_oracle_api())
    sig = np.concatenate([out[r][2] for r in range(WORLD)])
    assert np.array_equal(sig, s1.numpy())                   # the same global batch, bitwise
    np.testing.assert_array_equal(np.concatenate([out[r][3] for r in range(WORLD)]), e1.numpy())
    for r in range(WORLD):
        g, stats = out[r][0], out[r][1]
        np.testing.assert_allclose(stats, st1.numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(g, g1.numpy(), rtol=1e-10, atol=1e-12)
    # and the exchange reaches the oracle's single-process estimator
    ref = ov.vmc_gradient(om.Model(om.GRU1D, N, d_h=D),
                          inputs.xavier_params(1, D, seed=3, noise_std=0.1).astype(np.float32).astype(np.float64),
                          s1.numpy().astype(np.int64), e1.double().numpy())
    np.testing.assert_allclose(out[0][0], ref, rtol=1e-9, atol=1e-12)
