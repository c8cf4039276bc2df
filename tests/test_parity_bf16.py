"""BF16 tensor-core path (1D GRU) against the float64 oracle.

The cell GEMMs take BF16 operands (h and the weights rounded to 8 significant
bits) with FP32 accumulation; state, gates and readout stay FP32.  Each
site's logits then carry a relative error of about 2^-8, so the bounds are:
  log psi       2e-4 * N absolute (the N per-site errors add with random signs;
                measured mean 5e-5 per site at N = 100, d_h = 64);
  energy/site   |mean E_loc(BF16) - mean E_loc(oracle)| / N <= 1e-4 on the
                same configurations (the acceptance bound for the BF16 step);
  E_loc         per sample |E(BF16) - E(oracle)| <= 4e-3 Gamma S + 1e-5 N with
                S = sum_i psi(flip_i)/psi: each log ratio Delta_i sums up to N
                per-site log-probability differences, each off by at most the
                logit error (measured r.m.s. 7.5e-4 at N = 100, d_h = 64), so
                Delta_i is off by about 7.5e-4 sqrt(N) / 2 ~ 4e-3 (measured
                worst relative error 8.7e-4 of Gamma S);
  sampling      every draw along the GPU's path equals the oracle's decision
                u < p0 (float64, teacher-forced on that path) unless
                |u - p0| < 1e-3, twice the largest BF16 p0 error measured
                (4.8e-4 at N = 100, d_h = 64, logit error up to 2.1e-3); at
                most 1 % of the draws may fall in that window (expected 0.2 %);
  gradient      cosine similarity >= 0.999 with the oracle's gradient, also at
                the full bench size on a subsample of the batch.
"""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as oh, model as om, philox, vmc as ov
from paper_2507_18700_gb300 import inputs, nqs
from _draws import check_draws

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
W_SAMPLE = 1e-3          # sampling window (see the module docstring)
EPS_DELTA = 4e-3         # per-sample local-energy bound (see the module docstring)


def tfim_offdiag(sig, ref_e, J, Gamma):
    """S = sum_i psi(flip_i)/psi from the oracle's E_loc: E = diag - Gamma S."""
    s = 1 - 2 * np.asarray(sig, dtype=np.int64)
    return (-J * (s[:, :-1] * s[:, 1:]).sum(axis=1) - ref_e) / Gamma


def assert_eloc_per_sample(got, ref, sig, J, Gamma, N):
    S = tfim_offdiag(sig, ref, J, Gamma)
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    tol = EPS_DELTA * abs(Gamma) * S + 1e-5 * N
    assert np.all(err <= tol), (err / tol).max()


def setup(N, d, seed=1, noise=0.1):
    flat = inputs.xavier_params(1, d, seed=seed, noise_std=noise).astype(np.float32)
    return (nqs.model_desc(nqs.GRU1D, N, 1, d, precision=nqs.BF16), om.Model(om.GRU1D, N, d_h=d),
            flat.astype(np.float64), torch.tensor(flat, device=DEV))


@pytest.mark.parametrize("N,d,B", [(12, 16, 256), (40, 32, 300), (100, 64, 200), (7, 64, 129), (100, 128, 130)])
def test_bf16_logpsi_and_cache(N, d, B):
    desc, mod, pf, p = setup(N, d)
    sig = inputs.random_configs(B, N, seed=5)
    lp, hc = nqs.logpsi(desc, p, torch.tensor(sig, device=DEV))
    torch.cuda.synchronize()
    ref = om.run(mod, pf, sigma=sig.astype(np.int64))
    np.testing.assert_allclose(lp.cpu().numpy(), ref["logpsi"], atol=2e-4 * N, rtol=0)
    # the cache error grows with the number of BF16 products per gate (d_h + 16)
    np.testing.assert_allclose(hc.cpu().numpy(), ref["hidden"], atol=1e-2 if d <= 64 else 2e-2, rtol=0)


@pytest.mark.parametrize("N,d,B", [(20, 16, 512), (100, 64, 256)])
def test_bf16_sampling(N, d, B):
    desc, mod, pf, p = setup(N, d)
    sig, lp, hc = nqs.sample(desc, p, B, seed=9, step=4)
    lp_t, _ = nqs.logpsi(desc, p, sig, hcache=None)
    torch.cuda.synchronize()
    assert torch.equal(lp, lp_t)            # same kernel arithmetic in both modes
    u = philox.sampling_uniforms(9, 4, B, N)
    frac, _ = check_draws(mod, pf, sig.cpu().numpy(), u, W_SAMPLE)
    assert frac <= 1e-2, frac


@pytest.mark.parametrize("N,d,B,Gamma", [(12, 16, 512, 1.0), (30, 32, 256, 0.5), (100, 64, 256, 1.0)])
def test_bf16_energy_per_site(N, d, B, Gamma):
    # configurations drawn from the model (by the oracle's sampler), as in a VMC
    # step: uniformly random spins have vanishing probability, so their ratios
    # psi(sigma')/psi(sigma) are exponentially large and amplify any rounding
    desc, mod, pf, p = setup(N, d)
    sig = om.sample(mod, pf, philox.sampling_uniforms(11, 0, B, N))["sigma"].astype(np.uint8)
    sg = torch.tensor(sig, device=DEV)
    _, hc = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.tfim(1.0, Gamma), sg, hc)
    torch.cuda.synchronize()
    ref = oh.tfim_local_energy(N, 1.0, Gamma, sig.astype(np.int64), lambda x: om.logpsi(mod, pf, x))
    assert abs(el.cpu().numpy().mean() - ref.mean()) / N <= 1e-4
    assert_eloc_per_sample(el.cpu().numpy(), ref, sig, 1.0, Gamma, N)


def test_bf16_vmc_gradient_cosine():
    N, d, B = 40, 32, 256
    desc, mod, pf, p = setup(N, d)
    sig = inputs.random_configs(B, N, seed=12)
    e = (inputs.random_weights(B, seed=13, scale=2.0) - 50.0).astype(np.float32)
    sg = torch.tensor(sig, device=DEV)
    _, hc = nqs.logpsi(desc, p, sg)
    g, st = nqs.vmc_grad(desc, p, sg, hc, torch.tensor(e, device=DEV))
    torch.cuda.synchronize()
    ref = ov.vmc_gradient(mod, pf, sig.astype(np.int64), e.astype(np.float64))
    g = g.double().cpu().numpy()
    assert g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref)) >= 0.999


def test_bf16_full_size_step_n100_d64_b4096():
    """Bench workload in BF16: energy per site of the whole step within 1e-4 of
    the oracle's on 64 of its samples evaluated one by one (each also within
    the per-sample bound), and of the FP32 path; the reverse sweep at the full
    batch (the launch configuration of the step) against the oracle's
    gradient on those 64 samples (weights zero elsewhere)."""
    N, d, B = 100, 64, 4096
    desc, mod, pf, p = setup(N, d)
    d32 = nqs.model_desc(nqs.GRU1D, N, 1, d)
    u = philox.sampling_uniforms(21, 0, B, N)
    ref = om.sample(mod, pf, u)
    sg = torch.tensor(ref["sigma"], dtype=torch.uint8, device=DEV)
    _, hc = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.tfim(), sg, hc)
    _, hc32 = nqs.logpsi(d32, p, sg)
    el32 = nqs.local_energy(d32, p, nqs.tfim(), sg, hc32)
    g, st = nqs.vmc_grad(desc, p, sg, hc, el)
    ws = nqs.Workspace(DEV)
    sig, lp, hcs = nqs.sample(desc, p, B, seed=21, step=0, ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    # the step's own sampling at the full batch, every draw
    frac, _ = check_draws(mod, pf, sig.cpu().numpy(), u, W_SAMPLE)
    assert frac <= 1e-2, frac
    e16, e32 = el.double().cpu().numpy(), el32.double().cpu().numpy()
    assert abs(e16.mean() - e32.mean()) / N <= 1e-4
    pick = np.random.default_rng(2).choice(B, 64, replace=False)
    e_ref = oh.tfim_local_energy(N, 1.0, 1.0, ref["sigma"][pick], lambda x: om.logpsi(mod, pf, x))
    assert abs(e16[pick].mean() - e_ref.mean()) / N <= 1e-4
    assert_eloc_per_sample(e16[pick], e_ref, ref["sigma"][pick], 1.0, 1.0, N)
    assert np.isfinite(g.cpu().numpy()).all()
    # the VMC weights of the step, kept on the 64 picked samples only
    w = np.zeros(B, dtype=np.float32)
    w[pick] = (2.0 * (e16[pick] - e16.mean()) / B).astype(np.float32)
    gp = nqs.logpsi_grad(desc, p, sg, hc, torch.tensor(w, device=DEV), ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    g_ref = ov.logpsi_grad(mod, pf, ref["sigma"][pick], w[pick].astype(np.float64))
    gp = gp.double().cpu().numpy()
    cos = gp @ g_ref / (np.linalg.norm(gp) * np.linalg.norm(g_ref))
    rel = np.linalg.norm(gp - g_ref) / np.linalg.norm(g_ref)
    assert cos >= 0.999 and rel <= 2e-2, (cos, rel)


@pytest.mark.parametrize("N,d,B", [(12, 16, 300), (40, 32, 200), (100, 64, 256), (30, 64, 1)])
def test_bf16_reverse_sweep(N, d, B):
    """The BF16 reverse sweep (tensor-core recompute, dh and weight-gradient
    GEMMs; G and X read as transposed operands) against the oracle's gradient of
    sum_b w_b log psi_b: cosine >= 0.999 and relative L2 error <= 2e-2 (BF16
    operands, about 2^-8 per product, summed over B N terms)."""
    desc, mod, pf, p = setup(N, d)
    sig = inputs.random_configs(B, N, seed=14)
    w = inputs.random_weights(B, seed=15).astype(np.float32)
    sg = torch.tensor(sig, device=DEV)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    g = nqs.logpsi_grad(desc, p, sg, hc, torch.tensor(w, device=DEV), ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    ref = ov.logpsi_grad(mod, pf, sig.astype(np.int64), w.astype(np.float64))
    g = g.double().cpu().numpy()
    assert g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref)) >= 0.999
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) <= 2e-2


def test_autotuned_variants_agree_bitwise():
    """Every tile variant (1, 2 or 4 threads per row; 128, 64 or 32 rows per
    tile) computes bitwise the same samples, cache, local energies and energy
    statistics, and so does the autotuned choice (tuning off = first variant).
    The gradient is a sum over samples whose per-CTA grouping depends on the
    rows per tile: bitwise equal among variants with the same rows per tile,
    equal to FP32 rounding across them (relative L2 difference <= 1e-5)."""
    N, d, B = 60, 64, 700
    desc, mod, pf, p = setup(N, d)
    outs = []
    runs = [(None, False), (None, True), (None, True)] + [(v, True) for v in range(9)]
    for variant, tune in runs:
        nqs.set_autotune(tune)
        nqs.set_tile_variant(variant)
        s, lp, hc = nqs.sample(desc, p, B, seed=3, step=2)
        el = nqs.local_energy(desc, p, nqs.tfim(), s, hc)
        g, st = nqs.vmc_grad(desc, p, s, hc, el)
        torch.cuda.synchronize()
        outs.append((variant, s.clone(), lp.clone(), hc.clone(), el.clone(), st.clone(), g.clone()))
    nqs.set_tile_variant(None)
    nqs.set_autotune(True)
    ref = outs[0]
    for o in outs[1:]:
        for x, y in zip(ref[1:6], o[1:6]):
            assert torch.equal(x, y)
        rel = float((o[6].double() - ref[6].double()).norm() / ref[6].double().norm())
        assert rel <= 1e-5, rel
    # pinned variants 0-2 (128 rows), 3-5 (64 rows) and 6-8 (32 rows): bitwise
    # within each class
    for lo, hi in ((3, 6), (6, 9), (9, 12)):
        for o in outs[lo + 1:hi]:
            assert torch.equal(o[6], outs[lo][6])

def test_bf16_d128_against_oracle():
    """d_h = 128 on the tensor cores (one 128-row tile per CTA, the x_in block
    from an FP32 table, 2 or 4 threads per row): log psi and cache, every
    sampling draw (window 2e-3: twice the d_h = 64 window, the gate GEMMs sum
    twice as many BF16 products), per-sample local energies, and the gradient
    of the BF16 reverse sweep (tape pass, sequential sweep, weight-gradient
    GEMMs) at the d_h <= 64 bounds."""
    N, d, B = 60, 128, 200
    desc, mod, pf, p = setup(N, d)
    sig = inputs.random_configs(B, N, seed=61)
    lp, hc = nqs.logpsi(desc, p, torch.tensor(sig, device=DEV))
    torch.cuda.synchronize()
    ref = om.run(mod, pf, sigma=sig.astype(np.int64))
    np.testing.assert_allclose(lp.cpu().numpy(), ref["logpsi"], atol=2e-4 * N, rtol=0)
    np.testing.assert_allclose(hc.cpu().numpy(), ref["hidden"], atol=2e-2, rtol=0)
    s, lps, hcs = nqs.sample(desc, p, B, seed=9, step=4)
    torch.cuda.synchronize()
    frac, _ = check_draws(mod, pf, s.cpu().numpy(), philox.sampling_uniforms(9, 4, B, N), 2e-3)
    assert frac <= 1e-2, frac
    sm = om.sample(mod, pf, philox.sampling_uniforms(62, 0, B, N))["sigma"]
    sg = torch.tensor(sm.astype(np.uint8), device=DEV)
    ws = nqs.Workspace(DEV)
    _, hc2 = nqs.logpsi(desc, p, sg, ws=ws)
    el = nqs.local_energy(desc, p, nqs.tfim(1.0, 1.0), sg, hc2, ws=ws)
    g, st = nqs.vmc_grad(desc, p, sg, hc2, el, ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    e_ref = oh.tfim_local_energy(N, 1.0, 1.0, sm, lambda x: om.logpsi(mod, pf, x))
    e16 = el.double().cpu().numpy()
    assert abs(e16.mean() - e_ref.mean()) / N <= 1e-4
    assert_eloc_per_sample(e16, e_ref, sm, 1.0, 1.0, N)
    g_ref = ov.vmc_gradient(mod, pf, sm.astype(np.int64), e_ref)
    gg = g.double().cpu().numpy()
    assert gg @ g_ref / (np.linalg.norm(gg) * np.linalg.norm(g_ref)) >= 0.999
    assert np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref) <= 2e-2


@pytest.mark.parametrize("N,B", [(60, 200), (17, 129), (100, 33), (3, 300)])
def test_bf16_d128_logpsi_grad(N, B):
    """The d_h = 128 BF16 reverse sweep on random configurations and weights
    (ragged tiles, short and long chains) against the oracle's reverse sweep:
    cosine >= 0.999 and relative L2 error <= 2e-2, as at d_h <= 64."""
    d = 128
    desc, mod, pf, p = setup(N, d, seed=63)
    sig = inputs.random_configs(B, N, seed=64)
    w = inputs.random_weights(B, seed=65).astype(np.float32)
    sg = torch.tensor(sig, device=DEV)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    g = nqs.logpsi_grad(desc, p, sg, hc, torch.tensor(w, device=DEV), ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    ref = ov.logpsi_grad(mod, pf, sig.astype(np.int64), w.astype(np.float64))
    gg = g.double().cpu().numpy()
    cos = gg @ ref / (np.linalg.norm(gg) * np.linalg.norm(ref))
    rel = np.linalg.norm(gg - ref) / np.linalg.norm(ref)
    assert cos >= 0.999 and rel <= 2e-2, (cos, rel)


def test_bf16_d128_variants_agree_bitwise():
    """Every d_h = 128 tile variant (2 or 4 threads per row; 128, 64 or 32 rows
    per tile for sampling / teacher forcing) gives bitwise the same samples,
    log psi, cache and local energies."""
    N, d, B = 40, 128, 300
    desc, mod, pf, p = setup(N, d)
    outs = []
    for v in range(6):
        nqs.set_tile_variant(v)
        s, lp, hc = nqs.sample(desc, p, B, seed=5, step=1)
        lpt, hct = nqs.logpsi(desc, p, s)
        el = nqs.local_energy(desc, p, nqs.tfim(), s, hc)
        torch.cuda.synchronize()
        outs.append((s.clone(), lp.clone(), hc.clone(), lpt.clone(), hct.clone(), el.clone()))
    nqs.set_tile_variant(None)
    assert torch.isfinite(outs[0][5]).all()
    for o in outs[1:]:
        for x, y in zip(outs[0], o):
            assert torch.equal(x, y)
    assert torch.equal(outs[0][1], outs[0][3]) and torch.equal(outs[0][2], outs[0][4])
