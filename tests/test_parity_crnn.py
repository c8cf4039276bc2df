"""cRNN (phase head, Eq. softsign) and the cluster-state Hamiltonian (Sec.
III D) on the FP32 1D path against the float64 oracle.

Bounds (FP32 state and readout): log|psi| 1e-4 absolute at N = 64 (as the
pRNN); phi = sum of N terms pi softsign(z) with |d softsign / dz| <= 1, so
its error is about pi times the summed logit error, 2e-4 absolute; E_loc per
sample (complex) 2e-5 N (1 + |E|/N) absolute, as the TFIM chains (N ratios,
each from up to N float32 log-probability and phase differences); the
gradient relative L2 error 1e-4 against the oracle's reverse sweep; growth
bit-exact on carried entries.
"""
import numpy as np
import pytest
import torch

from oracle import growth, hamiltonian as oh, model as om, philox, vmc as ov
from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def setup(N, d, seed=40, phase=True, noise=0.3):
    flat = inputs.xavier_params(1, d, seed=seed, noise_std=noise, phase=phase).astype(np.float32)
    return (nqs.model_desc(nqs.GRU1D, N, 1, d, phase=phase), om.Model(om.GRU1D, N, d_h=d, phase=phase),
            flat.astype(np.float64), torch.tensor(flat, device=DEV))


@pytest.mark.parametrize("N,d,B", [(64, 16, 100), (20, 32, 129), (37, 64, 70), (12, 128, 33)])
def test_crnn_logpsi_phase_and_sampling(N, d, B):
    desc, mod, pf, p = setup(N, d)
    sig = inputs.random_configs(B, N, seed=41)
    lp, hc = nqs.logpsi(desc, p, torch.tensor(sig, device=DEV))
    torch.cuda.synchronize()
    ref = om.run(mod, pf, sigma=sig.astype(np.int64))
    got = lp.cpu().numpy()
    assert got.shape == (B, 2)
    np.testing.assert_allclose(got[:, 0], ref["logpsi"], atol=1e-4, rtol=0)
    np.testing.assert_allclose(got[:, 1], ref["phase"], atol=2e-4, rtol=0)
    np.testing.assert_allclose(hc.cpu().numpy(), ref["hidden"], atol=2e-5, rtol=0)
    # sampling: the phase head does not change the draws
    s, lps, _ = nqs.sample(desc, p, B, seed=3, step=1)
    torch.cuda.synchronize()
    u = philox.sampling_uniforms(3, 1, B, N)
    ref_s = om.sample(mod, pf, u)
    near = (np.abs(u - ref_s["p0"]) < 1e-6).any(axis=1)
    assert np.array_equal(s.cpu().numpy()[~near], ref_s["sigma"][~near])
    np.testing.assert_allclose(lps.cpu().numpy()[~near, 1], ref_s["phase"][~near], atol=2e-4, rtol=0)


@pytest.mark.parametrize("N,d,B,phase", [(64, 16, 60, True), (30, 32, 77, True), (16, 64, 40, True),
                                         (9, 128, 20, True), (40, 32, 50, False), (3, 16, 30, True)])
def test_cluster_local_energy(N, d, B, phase):
    desc, mod, pf, p = setup(N, d, seed=42, phase=phase)
    sig = om.sample(mod, pf, philox.sampling_uniforms(43, 0, B, N))["sigma"]
    sg = torch.tensor(sig.astype(np.uint8), device=DEV)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    el = nqs.local_energy(desc, p, nqs.cluster(), sg, hc, ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    ref = oh.cluster_local_energy(N, sig, lambda x: om.logpsi(mod, pf, x),
                                  (lambda x: om.phase(mod, pf, x)) if phase else (lambda x: np.zeros(len(x))))
    got = el.double().cpu().numpy()
    got = got[:, 0] + 1j * got[:, 1] if phase else got
    if not phase:
        assert np.abs(ref.imag).max() == 0.0
    tol = 2e-5 * N * (1.0 + np.abs(ref) / N)
    assert np.all(np.abs(got - ref) <= tol), (np.abs(got - ref) / tol).max()


@pytest.mark.parametrize("N,d,B", [(64, 16, 100), (25, 64, 70), (10, 128, 17)])
def test_crnn_vmc_gradient(N, d, B):
    desc, mod, pf, p = setup(N, d, seed=44)
    sig = om.sample(mod, pf, philox.sampling_uniforms(45, 0, B, N))["sigma"]
    sg = torch.tensor(sig.astype(np.uint8), device=DEV)
    _, hc = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.cluster(), sg, hc)
    g, st = nqs.vmc_grad(desc, p, sg, hc, el)
    torch.cuda.synchronize()
    e = el.double().cpu().numpy()
    ec = e[:, 0] + 1j * e[:, 1]
    ref_st = ov.energy_stats(ec)
    np.testing.assert_allclose(st.cpu().numpy(), ref_st, rtol=1e-10, atol=1e-12)
    ref = ov.vmc_gradient(mod, pf, sig, ec)
    gg = g.double().cpu().numpy()
    rel = np.linalg.norm(gg - ref) / np.linalg.norm(ref)
    assert rel <= 1e-4, rel


def test_crnn_logpsi_grad_and_autograd():
    N, d, B = 20, 32, 90
    desc, mod, pf, p = setup(N, d, seed=46)
    sig = inputs.random_configs(B, N, seed=47)
    w = np.stack([inputs.random_weights(B, seed=48), inputs.random_weights(B, seed=49)], axis=1).astype(np.float32)
    sg = torch.tensor(sig, device=DEV)
    _, hc = nqs.logpsi(desc, p, sg)
    g = nqs.logpsi_grad(desc, p, sg, hc, torch.tensor(w, device=DEV))
    pa = p.clone().requires_grad_(True)
    out = nqs.LogPsi.apply(pa, sg, desc)
    (out * torch.tensor(w, device=DEV)).sum().backward()
    torch.cuda.synchronize()
    ref = ov.logpsi_grad(mod, pf, sig.astype(np.int64), w[:, 0].astype(np.float64),
                         phase_weights=w[:, 1].astype(np.float64))
    gg = g.double().cpu().numpy()
    assert np.linalg.norm(gg - ref) / np.linalg.norm(ref) <= 1e-4
    assert torch.equal(pa.grad, g)


def test_crnn_growth_matches_oracle():
    N, d, D = 30, 16, 32
    small = nqs.model_desc(nqs.GRU1D, N, 1, d, phase=True)
    big = nqs.model_desc(nqs.GRU1D, N, 1, D, phase=True)
    ps = inputs.xavier_params(1, d, seed=50, noise_std=0.1, phase=True).astype(np.float32)
    pb = nqs.grow_hidden(small, torch.tensor(ps, device=DEV), big, seed=2, eps=1e-3)
    torch.cuda.synchronize()
    ref = growth.grow(om.Model(1, N, d_h=d, phase=True), ps.astype(np.float64), om.Model(1, N, d_h=D, phase=True),
                      seed=2, eps=1e-3)
    got = pb.cpu().numpy().astype(np.float64)
    old = np.abs(ref) > 5e-2
    np.testing.assert_allclose(got, ref, atol=2e-9, rtol=1e-5)
    assert np.array_equal(got[old], ref[old])
