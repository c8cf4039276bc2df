"""Hidden-state checkpointing (FP32 1D GRU): the forward keeps every k-th state,
the reverse sweep recomputes each k-site segment from its checkpoint.

* log psi bitwise equal to nqs_logpsi (the same cells in the same order) and
  every checkpoint bitwise equal to the corresponding prefix-cache row;
* the gradient equal to nqs_logpsi_grad's to FP32 rounding of the per-block
  partials (relative L2 1e-6: the segments' partial rows are summed apart)
  and to the oracle's reverse sweep (relative 1e-4), for k = 1, sqrt(N), a
  ragged last segment and k >= N (one segment, no checkpoint);
* the autograd.Function with checkpoint = k gives the checkpointed gradient.
"""
import numpy as np
import pytest
import torch

from oracle import model as om, vmc as ov
from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("N,d,B,k", [(100, 64, 300, 10), (37, 16, 129, 6), (20, 32, 70, 1), (12, 8, 40, 12),
                                     (12, 8, 40, 50), (50, 128, 33, 7)])
def test_checkpointed_logpsi_and_gradient(N, d, B, k):
    flat = inputs.xavier_params(1, d, seed=51, noise_std=0.1).astype(np.float32)
    p = torch.tensor(flat, device=DEV)
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d)
    sig = torch.tensor(inputs.random_configs(B, N, seed=52), device=DEV)
    w = torch.tensor(inputs.random_weights(B, seed=53).astype(np.float32), device=DEV)
    lp, hc = nqs.logpsi(desc, p, sig)
    lpc, ck = nqs.logpsi_ckpt(desc, p, sig, k)
    g = nqs.logpsi_grad(desc, p, sig, hc, w)
    gc = nqs.logpsi_grad_ckpt(desc, p, sig, k, ck, w)
    torch.cuda.synchronize()
    assert torch.equal(lp, lpc)
    nck = (N + k - 1) // k - 1
    assert ck.numel() == B * nck * d
    if nck:
        rows = hc[:, [(j + 1) * k - 1 for j in range(nck)], :]
        assert torch.equal(ck.view(B, nck, d), rows)
    rel = float((gc.double() - g.double()).norm() / g.double().norm())
    assert rel <= 1e-6, rel
    ref = ov.logpsi_grad(om.Model(om.GRU1D, N, d_h=d), flat.astype(np.float64), sig.cpu().numpy().astype(np.int64),
                         w.double().cpu().numpy())
    gg = gc.double().cpu().numpy()
    assert np.linalg.norm(gg - ref) / np.linalg.norm(ref) <= 1e-4


def test_autograd_function_with_checkpoints():
    N, d, B = 64, 32, 100
    flat = inputs.xavier_params(1, d, seed=54, noise_std=0.1).astype(np.float32)
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d)
    sig = torch.tensor(inputs.random_configs(B, N, seed=55), device=DEV)
    w = torch.tensor(inputs.random_weights(B, seed=56).astype(np.float32), device=DEV)
    grads = []
    for k in (None, 8):
        pa = torch.tensor(flat, device=DEV).requires_grad_(True)
        (nqs.LogPsi.apply(pa, sig, desc, k) * w).sum().backward()
        grads.append(pa.grad.double())
    torch.cuda.synchronize()
    assert float((grads[1] - grads[0]).norm() / grads[0].norm()) <= 1e-6


def test_checkpoint_rejects_other_models():
    for desc in (nqs.model_desc(nqs.GRU1D, 20, 1, 32, precision=nqs.BF16), nqs.model_desc(nqs.GRU2D, 4, 4, 16),
                 nqs.model_desc(nqs.GRU1D, 20, 1, 32, phase=True)):
        assert nqs.lib().nqs_ckpt_workspace_bytes(desc, 10, 4) == 0
