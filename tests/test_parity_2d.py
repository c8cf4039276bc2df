"""Parity of the CUDA 2D GRU + GLU path (zig-zag order, Heisenberg local energy
with the Marshall sign, zero-magnetisation mask) with the float64 oracle.

Weights are Xavier-uniform plus Gaussian noise of std <= 0.1: the 2D cell's
mixing path U_mix h' has no squashing, and with much larger weights the hidden
state grows geometrically across the lattice (8 x 8, d_h = 64, std 0.2:
max |h| ~ 1e7), where no float32 evaluation can match float64.

Tolerances as for 1D (FP32 path): log psi 1e-4 absolute; E_loc per sample
2e-5 absolute per bond and the mean per site 1e-6; gradient relative L2 error
1e-4 and cosine 0.9999; sampling identical except samples with a draw within
1e-6 of the oracle's threshold (<= 1e-4 of draws).
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


def setup(Lx, Ly, d, sz0, seed=0, noise=0.1):
    # the noise is kept relative to the Xavier scale: the spectral norm of a
    # d x 2d Gaussian perturbation grows like sqrt(d)
    noise = noise * min(1.0, np.sqrt(64.0 / d))
    flat = inputs.xavier_params(2, d, seed=seed, noise_std=noise).astype(np.float32)
    return (nqs.model_desc(nqs.GRU2D, Lx, Ly, d, sz0=sz0), om.Model(om.GRU2D, Lx, Ly, d_h=d, sz0=sz0),
            flat.astype(np.float64), dev(flat))


def order_index(mod):
    return np.array([mod.lattice_index(i, j) for (i, j) in mod.order()])


def compare_samples(mod, pf, sig_gpu, seed, step):
    B, N = sig_gpu.shape
    u = philox.sampling_uniforms(seed, step, B, N)          # [B, position]
    ref = om.sample(mod, pf, u)
    p0_pos = ref["p0"][:, order_index(mod)]
    near = np.abs(u - p0_pos) < 1e-6
    assert near.mean() <= 1e-4
    clean = ~near.any(axis=1)
    assert np.array_equal(sig_gpu[clean], ref["sigma"][clean])
    # every draw along the GPU's own path (the oracle teacher-forced on it)
    frac, _ = check_draws(mod, pf, sig_gpu, u, 1e-6)
    assert frac <= 1e-4
    return ref


@pytest.mark.parametrize("Lx,Ly,d,B,sz0", [(4, 4, 16, 512, True), (3, 3, 8, 300, False), (8, 8, 64, 256, True),
                                           (5, 6, 32, 77, False), (3, 4, 128, 40, True), (4, 4, 256, 24, True)])
def test_sampling_and_logpsi_2d(Lx, Ly, d, B, sz0):
    desc, mod, pf, p = setup(Lx, Ly, d, sz0)
    sig, lp, hc = nqs.sample(desc, p, B, seed=3, step=1)
    torch.cuda.synchronize()
    s = sig.cpu().numpy().astype(np.int64)
    if sz0:
        assert np.all(s.sum(axis=1) == mod.N // 2)
    ref = compare_samples(mod, pf, s, 3, 1)
    lp2, hc2 = nqs.logpsi(desc, p, dev(ref["sigma"], torch.uint8))
    torch.cuda.synchronize()
    np.testing.assert_allclose(lp2.cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)
    np.testing.assert_allclose(hc2.cpu().numpy(), ref["hidden"], atol=2e-5, rtol=0)
    if np.array_equal(s, ref["sigma"]):
        np.testing.assert_allclose(lp.cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)


def heis_case(Lx, Ly, d, B, sz0, marshall=True, J=1.0, seed=2):
    desc, mod, pf, p = setup(Lx, Ly, d, sz0, seed=seed)
    sig = inputs.random_configs(B, mod.N, seed=seed + 50, sz0=sz0)
    sg = dev(sig, torch.uint8)
    _, hc = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.heisenberg(J, marshall), sg, hc)
    torch.cuda.synchronize()
    ref = oh.heisenberg_local_energy(Lx, Ly, J, marshall, sig.astype(np.int64),
                                     lambda x: om.logpsi(mod, pf, x))
    nb = len(oh.square_bonds(Lx, Ly))
    got = el.cpu().numpy()
    np.testing.assert_allclose(got, ref, atol=2e-5 * nb, rtol=0)
    assert abs(got.mean() - ref.mean()) / mod.N < 1e-6


@pytest.mark.parametrize("Lx,Ly,d,B,sz0,marshall", [(4, 4, 16, 64, True, True), (2, 2, 8, 16, True, True),
                                                    (3, 4, 32, 50, True, False), (4, 3, 16, 40, False, True),
                                                    (8, 8, 64, 24, True, True), (2, 6, 128, 12, True, True),
                                                    (5, 2, 8, 33, False, False), (4, 4, 256, 10, True, True)])
def test_heisenberg_local_energy(Lx, Ly, d, B, sz0, marshall):
    heis_case(Lx, Ly, d, B, sz0, marshall)


def grad_check(g, ref):
    g = g.double().cpu().numpy()
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    assert rel < 1e-4 and cos > 0.9999, (rel, cos)


@pytest.mark.parametrize("Lx,Ly,d,B,sz0", [(4, 4, 16, 100, True), (3, 3, 8, 40, False), (8, 8, 64, 64, True),
                                           (2, 4, 128, 20, True), (5, 3, 32, 37, False), (3, 4, 256, 12, True)])
def test_logpsi_grad_2d(Lx, Ly, d, B, sz0):
    # noise 0.05: the mixing path U_mix h' is not squashed, so much larger
    # weights make the hidden state grow geometrically over the lattice and the
    # float32 result is then ill-conditioned against float64
    desc, mod, pf, p = setup(Lx, Ly, d, sz0, seed=5, noise=0.05)
    sig = inputs.random_configs(B, mod.N, seed=6, sz0=sz0)
    w = inputs.random_weights(B, seed=7).astype(np.float32)
    sg = dev(sig, torch.uint8)
    _, hc = nqs.logpsi(desc, p, sg)
    g = nqs.logpsi_grad(desc, p, sg, hc, dev(w))
    torch.cuda.synchronize()
    grad_check(g, ov.logpsi_grad(mod, pf, sig.astype(np.int64), w.astype(np.float64)))


def test_vmc_grad_2d():
    Lx, Ly, d, B = 4, 4, 16, 128
    desc, mod, pf, p = setup(Lx, Ly, d, True, seed=8)
    sig = inputs.random_configs(B, mod.N, seed=9, sz0=True)
    e = (inputs.random_weights(B, seed=10, scale=0.5) - 9.0).astype(np.float32)
    sg = dev(sig, torch.uint8)
    _, hc = nqs.logpsi(desc, p, sg)
    g, st = nqs.vmc_grad(desc, p, sg, hc, dev(e))
    torch.cuda.synchronize()
    np.testing.assert_allclose(st.cpu().numpy(), ov.energy_stats(e.astype(np.float64)), rtol=1e-12, atol=1e-12)
    grad_check(g, ov.vmc_gradient(mod, pf, sig.astype(np.int64), e.astype(np.float64)))


def test_full_size_heisenberg_8x8_d64_b2048():
    """8 x 8 open lattice, Marshall sign, zero magnetisation, d_h = 64, 2048 samples."""
    Lx = Ly = 8
    d, B = 64, 2048
    desc, mod, pf, p = setup(Lx, Ly, d, True, seed=0, noise=0.0)
    sig, lp, hc = nqs.sample(desc, p, B, seed=21, step=0)
    torch.cuda.synchronize()
    ref = compare_samples(mod, pf, sig.cpu().numpy().astype(np.int64), 21, 0)
    sg = dev(ref["sigma"], torch.uint8)
    lp2, hc2 = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.heisenberg(1.0, True), sg, hc2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(lp2.cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)
    pick = np.random.default_rng(1).choice(B, 16, replace=False)
    e_ref = oh.heisenberg_local_energy(Lx, Ly, 1.0, True, ref["sigma"][pick], lambda x: om.logpsi(mod, pf, x))
    np.testing.assert_allclose(el.cpu().numpy()[pick], e_ref, atol=2e-5 * 112, rtol=0)
    w = inputs.random_weights(B, seed=22).astype(np.float32)
    g = nqs.logpsi_grad(desc, p, sg, hc2, dev(w))
    torch.cuda.synchronize()
    grad_check(g, ov.logpsi_grad(mod, pf, ref["sigma"], w.astype(np.float64)))


def test_largest_model_16x16_d256():
    """The largest configuration's model: 16 x 16 open lattice, d_h = 256, Marshall
    sign, zero magnetisation, Xavier weights (seed 3), at a batch the oracle can
    follow: sampling on every sample, local energies on 2 samples evaluated one by
    one, gradient on 4 samples."""
    Lx = Ly = 16
    d, B = 256, 32
    desc, mod, pf, p = setup(Lx, Ly, d, True, seed=3, noise=0.0)
    sig, lp, hc = nqs.sample(desc, p, B, seed=31, step=0)
    torch.cuda.synchronize()
    ref = compare_samples(mod, pf, sig.cpu().numpy().astype(np.int64), 31, 0)
    sg = dev(ref["sigma"], torch.uint8)
    lp2, hc2 = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.heisenberg(1.0, True), sg, hc2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(lp2.cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)
    e_ref = oh.heisenberg_local_energy(Lx, Ly, 1.0, True, ref["sigma"][:2], lambda x: om.logpsi(mod, pf, x))
    np.testing.assert_allclose(el.cpu().numpy()[:2], e_ref, atol=2e-5 * 480, rtol=0)
    w = inputs.random_weights(4, seed=32).astype(np.float32)
    sg4 = sg[:4].contiguous()
    _, hc4 = nqs.logpsi(desc, p, sg4)
    g = nqs.logpsi_grad(desc, p, sg4, hc4, dev(w))
    torch.cuda.synchronize()
    grad_check(g, ov.logpsi_grad(mod, pf, ref["sigma"][:4], w.astype(np.float64)))
