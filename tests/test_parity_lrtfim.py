"""Long-range TFIM (Sec. III C) local energies on the GPU against the float64
oracle, on configurations drawn from the model.

The flips run the TFIM's prefix-cached chains; the diagonal
-J sum_{i<j} s_i s_j / |i - j|^alpha is summed in FP64 per sample and rounded
to float once (a relative 6e-8 of |E_loc|, which reaches ~10^3 at N = 80).
Per sample: FP32 within 2e-5 N (1 + Gamma) + 1e-7 |E|; BF16 within
4e-3 Gamma S + 1e-5 N + 1e-7 |E| (S = sum of the flip ratios; the bound of
the BF16 TFIM chains)."""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as oh, model as om, philox
from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("N,d,B,alpha,Gamma,precision", [
    (80, 32, 96, 0.1, 1.0, nqs.FP32), (80, 64, 64, 0.1, 1.0, nqs.BF16), (37, 16, 129, 1.5, 0.6, nqs.FP32),
    (50, 32, 70, 3.0, 1.2, nqs.BF16), (20, 16, 40, float("inf"), 1.0, nqs.FP32)])
def test_lr_tfim_local_energy(N, d, B, alpha, Gamma, precision):
    flat = inputs.xavier_params(1, d, seed=27, noise_std=0.1).astype(np.float32)
    pf = flat.astype(np.float64)
    mod = om.Model(om.GRU1D, N, d_h=d)
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d, precision=precision)
    p = torch.tensor(flat, device=DEV)
    sig = om.sample(mod, pf, philox.sampling_uniforms(28, 0, B, N))["sigma"]
    sg = torch.tensor(sig.astype(np.uint8), device=DEV)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    el = nqs.local_energy(desc, p, nqs.lr_tfim(alpha, 1.0, Gamma), sg, hc, ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    ref = oh.lr_tfim_local_energy(N, alpha, 1.0, Gamma, sig, lambda x: om.logpsi(mod, pf, x))
    got = el.double().cpu().numpy()
    err = np.abs(got - ref)
    if precision == nqs.FP32:
        tol = 2e-5 * N * (1 + Gamma) + 1e-7 * np.abs(ref)
    else:
        S = (oh.lr_tfim_local_energy(N, alpha, 1.0, 0.0, sig, lambda x: np.zeros(len(x))) - ref) / Gamma
        tol = 4e-3 * Gamma * S + 1e-5 * N + 1e-7 * np.abs(ref)
    assert np.all(err <= tol), (err / tol).max()
    if alpha == float("inf"):
        el_nn = nqs.local_energy(desc, p, nqs.tfim(1.0, Gamma), sg, hc, ws=ws)
        torch.cuda.synchronize()
        np.testing.assert_allclose(got, el_nn.double().cpu().numpy(), rtol=1e-6, atol=1e-5)


def test_lr_tfim_rejects_bad_alpha_and_2d():
    desc = nqs.model_desc(nqs.GRU1D, 10, 1, 8)
    p = torch.zeros(nqs.param_count(desc), device=DEV)
    s = torch.zeros((4, 10), dtype=torch.uint8, device=DEV)
    hc = torch.zeros((4, 10, 8), device=DEV)
    with pytest.raises(nqs.NqsError):
        nqs.local_energy(desc, p, nqs.lr_tfim(-1.0), s, hc)
    d2 = nqs.model_desc(nqs.GRU2D, 4, 4, 8)
    with pytest.raises(nqs.NqsError):
        nqs.local_energy(d2, torch.zeros(nqs.param_count(d2), device=DEV), nqs.lr_tfim(0.5),
                         torch.zeros((4, 16), dtype=torch.uint8, device=DEV), torch.zeros((4, 16, 8), device=DEV))
