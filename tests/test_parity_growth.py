"""Parity of nqs_grow_hidden (Sec. II B, Fig. 2(b)) with the float64 oracle."""
import numpy as np
import pytest
import torch

from oracle import exact, growth, model as om
from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("cell,Lx,Ly,d,D", [(1, 100, 1, 16, 32), (1, 100, 1, 32, 64), (1, 100, 1, 64, 128),
                                            (1, 12, 1, 8, 8), (2, 4, 4, 8, 16), (2, 8, 8, 32, 64)])
def test_growth_matches_oracle(cell, Lx, Ly, d, D):
    small = nqs.model_desc(cell, Lx, Ly, d)
    big = nqs.model_desc(cell, Lx, Ly, D)
    ps = inputs.xavier_params(cell, d, seed=3, noise_std=0.1).astype(np.float32)
    pb = nqs.grow_hidden(small, torch.tensor(ps, device=DEV), big, seed=2, eps=1e-3)
    torch.cuda.synchronize()
    ref = growth.grow(om.Model(cell, Lx, Ly, d_h=d), ps.astype(np.float64), om.Model(cell, Lx, Ly, d_h=D),
                      seed=2, eps=1e-3)
    got = pb.cpu().numpy().astype(np.float64)
    old = np.abs(ref) > 5e-2            # carried entries are bit-exact copies
    np.testing.assert_allclose(got, ref, atol=2e-9, rtol=1e-5)
    assert np.array_equal(got[old], ref[old])


def test_growth_with_zero_noise_keeps_logpsi_on_device():
    N, d, D, B = 20, 16, 32, 256
    small = nqs.model_desc(1, N, 1, d)
    big = nqs.model_desc(1, N, 1, D)
    ps = torch.tensor(inputs.xavier_params(1, d, seed=4, noise_std=0.2).astype(np.float32), device=DEV)
    pb = nqs.grow_hidden(small, ps, big, seed=2, eps=0.0)
    sig = torch.tensor(inputs.random_configs(B, N, seed=5), device=DEV)
    a, _ = nqs.logpsi(small, ps, sig, hcache=None)
    b, _ = nqs.logpsi(big, pb, sig, hcache=None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(a.cpu().numpy(), b.cpu().numpy(), atol=2e-6)
