"""Parity of the CUDA 1D GRU path (through the C ABI) with the float64 oracle.

Inputs come from the seeded generators (``inputs``) or the oracle's own
sampler; expected values come from the oracle only.  Tolerances (FP32 path):
  log psi      1e-4 absolute at N = 100 (float32 rounding of ~N softplus terms);
  E_loc        per sample 2e-5 * N * (1 + |Gamma|) absolute; mean per site 1e-6;
  gradient     relative L2 error 1e-4, cosine >= 0.9999;
  sampling     identical configurations except samples with a draw whose
               uniform lies within 1e-6 of the oracle's threshold (<= 1e-4 of draws).
"""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as oh, model as om, philox, vmc as ov
from paper_2507_18700_gb300 import inputs, nqs
from _draws import check_draws

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def setup(N, d, seed, noise):
    flat = inputs.xavier_params(1, d, seed=seed, noise_std=noise)
    p32 = flat.astype(np.float32)
    return nqs.model_desc(nqs.GRU1D, N, 1, d), om.Model(om.GRU1D, N, d_h=d), p32.astype(np.float64), dev(p32)


def compare_samples(mod, pf, sig_gpu, seed, step):
    B, N = sig_gpu.shape
    u = philox.sampling_uniforms(seed, step, B, N)
    ref = om.sample(mod, pf, u)
    near = np.abs(u - ref["p0"]) < 1e-6             # 1D: sampling position == lattice index
    assert near.mean() <= 1e-4
    clean = ~near.any(axis=1)
    assert np.array_equal(sig_gpu[clean], ref["sigma"][clean])
    # every draw along the GPU's own path (the oracle teacher-forced on it)
    frac, _ = check_draws(mod, pf, sig_gpu, u, 1e-6)
    assert frac <= 1e-4
    return ref


@pytest.mark.parametrize("N,d,B", [(12, 8, 512), (37, 16, 100), (20, 32, 129), (100, 64, 256), (9, 128, 70)])
def test_sampling_and_logpsi(N, d, B):
    desc, mod, pf, p = setup(N, d, seed=0, noise=0.1)
    sig, lp, hc = nqs.sample(desc, p, B, seed=5, step=3)
    torch.cuda.synchronize()
    s = sig.cpu().numpy().astype(np.int64)
    ref = compare_samples(mod, pf, s, 5, 3)
    clean = np.array_equal(s, ref["sigma"])
    # teacher forcing on the oracle's samples
    lp2, hc2 = nqs.logpsi(desc, p, dev(ref["sigma"], torch.uint8))
    torch.cuda.synchronize()
    np.testing.assert_allclose(lp2.cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)
    np.testing.assert_allclose(hc2.cpu().numpy(), ref["hidden"], atol=2e-5, rtol=0)
    if clean:
        np.testing.assert_allclose(lp.cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)
        np.testing.assert_allclose(hc.cpu().numpy(), ref["hidden"], atol=2e-5, rtol=0)


def test_injected_uniforms_equal_internal_philox():
    desc, mod, pf, p = setup(30, 16, seed=2, noise=0.2)
    B = 300
    u = philox.sampling_uniforms(9, 77, B, 30)
    s1, lp1, _ = nqs.sample(desc, p, B, seed=9, step=77, hcache=None)
    s2, lp2, _ = nqs.sample(desc, p, B, uniforms=dev(u), hcache=None)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2)
    assert torch.equal(lp1, lp2)


def test_step_and_seed_change_the_draws():
    desc, mod, pf, p = setup(16, 8, seed=3, noise=0.5)
    a = nqs.sample(desc, p, 256, seed=1, step=0, hcache=None)[0]
    b = nqs.sample(desc, p, 256, seed=1, step=1, hcache=None)[0]
    c = nqs.sample(desc, p, 256, seed=2, step=0, hcache=None)[0]
    assert not torch.equal(a, b) and not torch.equal(a, c)


def eloc_case(N, d, B, Gamma, J=1.0, seed=1, noise=0.1):
    desc, mod, pf, p = setup(N, d, seed=seed, noise=noise)
    sig = inputs.random_configs(B, N, seed=seed + 100)
    sg = dev(sig, torch.uint8)
    lp, hc = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.tfim(J, Gamma), sg, hc)
    torch.cuda.synchronize()
    ref = oh.tfim_local_energy(N, J, Gamma, sig.astype(np.int64), lambda x: om.logpsi(mod, pf, x))
    got = el.cpu().numpy()
    tol = 2e-5 * N * (1 + abs(Gamma))
    np.testing.assert_allclose(got, ref, atol=tol, rtol=0)
    assert abs(got.mean() - ref.mean()) / N < 1e-6
    return got, ref


@pytest.mark.parametrize("N,d,B,Gamma", [(12, 8, 512, 1.0), (7, 16, 37, 0.5), (2, 8, 5, 2.0),
                                         (33, 32, 65, 1.5), (24, 128, 40, 1.0), (100, 64, 48, 1.0)])
def test_tfim_local_energy(N, d, B, Gamma):
    eloc_case(N, d, B, Gamma)


def test_tfim_local_energy_single_site_and_empty_batch():
    eloc_case(1, 8, 9, 1.0)
    desc, mod, pf, p = setup(10, 8, seed=0, noise=0.1)
    empty = torch.empty((0, 10), dtype=torch.uint8, device=DEV)
    lp, hc = nqs.logpsi(desc, p, empty)
    el = nqs.local_energy(desc, p, nqs.tfim(), empty, hc)
    torch.cuda.synchronize()
    assert lp.numel() == 0 and el.numel() == 0


def grad_check(g, ref):
    g = g.double().cpu().numpy()
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    assert rel < 1e-4 and cos > 0.9999, (rel, cos)


@pytest.mark.parametrize("N,d,B", [(12, 8, 512), (21, 16, 77), (15, 32, 100), (40, 64, 200), (10, 128, 50)])
def test_logpsi_grad(N, d, B):
    desc, mod, pf, p = setup(N, d, seed=4, noise=0.2)
    sig = inputs.random_configs(B, N, seed=40)
    w = inputs.random_weights(B, seed=41)
    sg = dev(sig, torch.uint8)
    _, hc = nqs.logpsi(desc, p, sg)
    g = nqs.logpsi_grad(desc, p, sg, hc, dev(w))
    torch.cuda.synchronize()
    grad_check(g, ov.logpsi_grad(mod, pf, sig.astype(np.int64), w.astype(np.float32).astype(np.float64)))


def test_vmc_grad_and_stats():
    N, d, B = 12, 8, 512
    desc, mod, pf, p = setup(N, d, seed=0, noise=0.0)
    sig = inputs.random_configs(B, N, seed=50)
    e = inputs.random_weights(B, seed=51, scale=3.0) - 14.0
    e32 = e.astype(np.float32)
    sg = dev(sig, torch.uint8)
    _, hc = nqs.logpsi(desc, p, sg)
    g, st = nqs.vmc_grad(desc, p, sg, hc, dev(e32))
    torch.cuda.synchronize()
    np.testing.assert_allclose(st.cpu().numpy(), ov.energy_stats(e32.astype(np.float64)), rtol=1e-12, atol=1e-12)
    grad_check(g, ov.vmc_gradient(mod, pf, sig.astype(np.int64), e32.astype(np.float64)))


def test_autograd_function_matches_oracle():
    N, d, B = 10, 16, 64
    desc, mod, pf, p = setup(N, d, seed=6, noise=0.1)
    sig = inputs.random_configs(B, N, seed=60)
    w = inputs.random_weights(B, seed=61).astype(np.float32)
    pp = p.clone().requires_grad_(True)
    lp = nqs.LogPsi.apply(pp, dev(sig, torch.uint8), desc)
    (lp * dev(w)).sum().backward()
    torch.cuda.synchronize()
    np.testing.assert_allclose(lp.detach().cpu().numpy(), om.logpsi(mod, pf, sig.astype(np.int64)), atol=1e-5)
    grad_check(pp.grad, ov.logpsi_grad(mod, pf, sig.astype(np.int64), w.astype(np.float64)))


def test_full_size_tfim_n100_d64_b4096():
    """The benchmark workload: 1D TFIM N = 100, d_h = 64, 4096 samples (launch
    configuration of bench.py).  Sampling is compared on every sample; local
    energies on 48 samples the oracle evaluates one by one; the gradient on all
    samples with generator weights."""
    N, d, B = 100, 64, 4096
    desc, mod, pf, p = setup(N, d, seed=1, noise=0.1)
    sig, lp, hc = nqs.sample(desc, p, B, seed=11, step=0)
    torch.cuda.synchronize()
    ref = compare_samples(mod, pf, sig.cpu().numpy().astype(np.int64), 11, 0)
    sg = dev(ref["sigma"], torch.uint8)
    lp2, hc2 = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.tfim(1.0, 1.0), sg, hc2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(lp2.cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)
    pick = np.random.default_rng(0).choice(B, 48, replace=False)
    s_pick = ref["sigma"][pick]
    e_ref = oh.tfim_local_energy(N, 1.0, 1.0, s_pick, lambda x: om.logpsi(mod, pf, x))
    np.testing.assert_allclose(el.cpu().numpy()[pick], e_ref, atol=2e-5 * N * 2, rtol=0)
    w = inputs.random_weights(B, seed=12).astype(np.float32)
    g = nqs.logpsi_grad(desc, p, sg, hc2, dev(w))
    torch.cuda.synchronize()
    grad_check(g, ov.logpsi_grad(mod, pf, ref["sigma"], w.astype(np.float64)))
