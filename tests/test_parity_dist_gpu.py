"""The library's data-parallel pieces on one GPU: ranks emulated one after the
other (no kernel waits on another), their buffers summed on the host side as
an all-reduce would.

* nqs_sample with sample_offset = r * B: the ranks' samples, log psi and cache
  are bitwise the rows of one call with the whole batch;
* nqs_energy_sums + nqs_vmc_grad_global: with the summed energy sums the
  statistics equal the one-call statistics to FP64 rounding and the summed
  gradient shares equal the one-call gradient to FP32 rounding of the per-block
  partials (relative L2 1e-5: the samples meet in other CTAs); with one rank they are bitwise nqs_vmc_grad's (the gradient before
  its rounding to float).
"""
import numpy as np
import pytest
import torch

from oracle import model as om, philox
from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _setup(cell, precision):
    if cell == nqs.GRU1D:
        N, Lx, Ly, d, sz0, ham = 40, 40, 1, 32, False, nqs.tfim(1.0, 0.9)
    else:
        N, Lx, Ly, d, sz0, ham = 16, 4, 4, 32, True, nqs.heisenberg()
    flat = inputs.xavier_params(cell, d, seed=31, noise_std=0.05).astype(np.float32)
    desc = nqs.model_desc(cell, Lx, Ly, d, sz0=sz0, precision=precision)
    return desc, ham, flat, torch.tensor(flat, device=DEV)


@pytest.mark.parametrize("cell,precision", [(nqs.GRU1D, nqs.FP32), (nqs.GRU1D, nqs.BF16),
                                            (nqs.GRU2D, nqs.FP32), (nqs.GRU2D, nqs.BF16)])
def test_emulated_ranks_equal_one_rank(cell, precision):
    desc, ham, flat, p = _setup(cell, precision)
    R, B = 3, 97
    s1, lp1, hc1 = nqs.sample(desc, p, R * B, seed=17, step=5)
    e1 = nqs.local_energy(desc, p, ham, s1, hc1)
    g1, st1 = nqs.vmc_grad(desc, p, s1, hc1, e1)
    parts = []
    for r in range(R):
        s, lp, hc = nqs.sample(desc, p, B, seed=17, step=5, sample_offset=r * B)
        e = nqs.local_energy(desc, p, ham, s, hc)
        parts.append((s, lp, hc, e, nqs.energy_sums(e)))
    torch.cuda.synchronize()
    assert torch.equal(torch.cat([x[0] for x in parts]), s1)
    assert torch.equal(torch.cat([x[1] for x in parts]), lp1)
    assert torch.equal(torch.cat([x[2] for x in parts]), hc1)
    assert torch.equal(torch.cat([x[3] for x in parts]), e1)
    sums = sum(x[4] for x in parts)                       # the all-reduce of the energy sums
    grad = torch.zeros(g1.numel(), dtype=torch.float64, device=DEV)
    for s, lp, hc, e, _ in parts:
        g, st = nqs.vmc_grad_global(desc, p, s, hc, e, sums)
        grad += g                                         # the all-reduce of the gradient shares
        torch.cuda.synchronize()
        np.testing.assert_allclose(st.cpu().numpy(), st1.cpu().numpy(), rtol=1e-13, atol=1e-13)
    ref = g1.double()
    rel = float((grad - ref).norm() / ref.norm())
    assert rel <= 1e-5, rel
    # one rank: bitwise nqs_vmc_grad
    g_one, st_one = nqs.vmc_grad_global(desc, p, s1, hc1, e1, nqs.energy_sums(e1))
    torch.cuda.synchronize()
    assert torch.equal(st_one, st1)
    assert torch.equal(g_one.float(), g1)


def test_sample_offset_matches_oracle_uniforms():
    """A call with sample_offset draws the oracle's uniforms of those global
    sample indices: the same configurations as injecting them."""
    desc, _, flat, p = _setup(nqs.GRU1D, nqs.FP32)
    B, off = 64, 1000
    s, lp, _ = nqs.sample(desc, p, B, seed=4, step=2, sample_offset=off)
    u = torch.tensor(philox.sampling_uniforms(4, 2, B, desc.N, sample_offset=off), dtype=torch.float32,
                     device=DEV)
    s2, lp2, _ = nqs.sample(desc, p, B, seed=4, step=2, uniforms=u)
    torch.cuda.synchronize()
    assert torch.equal(s, s2) and torch.equal(lp, lp2)
    mod = om.Model(om.GRU1D, desc.N, d_h=desc.d_h)
    np.testing.assert_allclose(lp.cpu().numpy(), om.logpsi(mod, flat.astype(np.float64),
                                                           s.cpu().numpy().astype(np.int64)), atol=1e-4)
