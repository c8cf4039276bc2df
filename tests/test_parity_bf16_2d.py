"""BF16 tensor-core 2D path (GRU + GLU, zig-zag order, Heisenberg local energy
with the Marshall sign and the zero-magnetisation mask) against the float64
oracle.

Both cell GEMMs and the GLU GEMM take BF16 operands (states and weights
rounded to 8 significant bits; biases and one-hot input weights carried as
BF16 hi + lo pairs) with FP32 accumulation; gates, readout and log-probability
sums stay FP32.  Bounds, as for the 1D BF16 path:
  log psi       6e-4 * N absolute on uniformly random configurations: the
                cell and GLU take 8 d^2 BF16 weights per unit (3 d^2 in 1D),
                each rounded by up to 2^-9, and a random configuration visits
                sites whose logits are far from 0, where that relative error
                becomes an absolute one (measured at 8 x 8, d_h = 64: mean
                6e-5, worst of 256 configurations 4.8e-4 per site);
  cache         3e-2 absolute (the cached states are FP32 values of a BF16 path);
  energy/site   |mean E_loc(BF16) - mean E_loc(oracle)| / N <= 1e-4 on the same
                configurations, drawn from the model;
  E_loc         per sample |E(BF16) - E(oracle)| <= 1e-2 S + 1e-5 N with S the
                summed magnitude of the exchange terms, J/2 exp(Delta) over the
                antiparallel bonds: each Delta sums up to N per-site
                log-probability differences whose logit errors were measured
                at r.m.s. 4e-4 (first row) to 5.3e-3 (last row) at 8 x 8,
                d_h = 64, so Delta is off by about 2.5e-3 sqrt(N) / 2 ~ 1e-2
                (measured worst relative error 2.1e-3 of S);
  sampling      every draw along the GPU's path equals the oracle's decision
                u < p0 (float64, teacher-forced on that path; forced draws of
                the mask must take the forced value) unless |u - p0| lies
                within 8e-4 (j + 1) at row j: the largest BF16 p0 error
                measured at 8 x 8, d_h = 64 grows with the row, from 2.3e-4
                (row 0) to 4.0e-3 (row 7), as the states' rounding compounds
                through the vertical inputs; at most 1 % of the free draws may
                fall in the window (expected 0.7 %);
  gradient      cosine similarity >= 0.999 and relative L2 error <= 2e-2 for the
                BF16 tensor-core reverse sweep (gate gradients rounded to BF16
                in the backward and weight-gradient GEMMs).
"""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as oh, model as om, philox, vmc as ov
from paper_2507_18700_gb300 import inputs, nqs
from _bf16 import bf16_weight_model, draw_window
from _draws import check_draws

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EPS_DELTA = 1e-2          # per-sample local-energy bound (see the module docstring)


def sample_window(mod):
    """Per sampling position: 8e-4 (j + 1) for a site of row j."""
    return np.array([8e-4 * (j + 1) for (i, j) in mod.order()])


def assert_eloc_per_sample(got, ref, sig, Lx, Ly, J, N):
    s = np.asarray(sig, dtype=np.int64)
    diag = np.zeros(s.shape[0])
    for a, b in oh.square_bonds(Lx, Ly):
        diag += np.where(s[:, a] == s[:, b], 0.25 * J, -0.25 * J)
    S = np.abs(ref - diag)
    err = np.abs(np.asarray(got, dtype=np.float64) - ref)
    tol = EPS_DELTA * S + 1e-5 * N
    assert np.all(err <= tol), (err / tol).max()


def dev(x, dtype=torch.float32):
    return torch.tensor(np.asarray(x), dtype=dtype, device=DEV)


def setup(Lx, Ly, d, sz0, seed=0, noise=0.1):
    noise = noise * min(1.0, np.sqrt(64.0 / d))
    flat = inputs.xavier_params(2, d, seed=seed, noise_std=noise).astype(np.float32)
    return (nqs.model_desc(nqs.GRU2D, Lx, Ly, d, sz0=sz0, precision=nqs.BF16),
            nqs.model_desc(nqs.GRU2D, Lx, Ly, d, sz0=sz0),
            om.Model(om.GRU2D, Lx, Ly, d_h=d, sz0=sz0), flat.astype(np.float64), dev(flat))


@pytest.mark.parametrize("Lx,Ly,d,B,sz0", [(4, 4, 32, 300, True), (8, 8, 64, 256, True), (3, 5, 32, 129, False),
                                           (6, 4, 64, 40, True)])
def test_bf16_2d_logpsi_and_cache(Lx, Ly, d, B, sz0):
    desc, _, mod, pf, p = setup(Lx, Ly, d, sz0)
    sig = inputs.random_configs(B, mod.N, seed=4, sz0=sz0)
    lp, hc = nqs.logpsi(desc, p, dev(sig, torch.uint8))
    torch.cuda.synchronize()
    ref = om.run(mod, pf, sigma=sig.astype(np.int64))
    np.testing.assert_allclose(lp.cpu().numpy(), ref["logpsi"], atol=6e-4 * mod.N, rtol=0)
    np.testing.assert_allclose(hc.cpu().numpy(), ref["hidden"], atol=3e-2, rtol=0)


@pytest.mark.parametrize("Lx,Ly,d,B,sz0", [(4, 4, 32, 512, True), (8, 8, 64, 256, True), (5, 3, 32, 200, False)])
def test_bf16_2d_sampling(Lx, Ly, d, B, sz0):
    desc, _, mod, pf, p = setup(Lx, Ly, d, sz0)
    sig, lp, hc = nqs.sample(desc, p, B, seed=3, step=1)
    lp_t, _ = nqs.logpsi(desc, p, sig, hcache=None)
    torch.cuda.synchronize()
    assert torch.equal(lp, lp_t)            # same kernel arithmetic in both modes
    s = sig.cpu().numpy().astype(np.int64)
    if sz0:
        assert np.all(s.sum(axis=1) == mod.N // 2)
    u = philox.sampling_uniforms(3, 1, B, mod.N)
    frac, _ = check_draws(mod, pf, s, u, sample_window(mod))
    assert frac <= 1e-2, frac


@pytest.mark.parametrize("Lx,Ly,d,B,sz0,marshall", [(4, 4, 32, 64, True, True), (8, 8, 64, 24, True, True),
                                                    (3, 4, 32, 50, True, False), (4, 3, 64, 40, False, True)])
def test_bf16_2d_energy_per_site(Lx, Ly, d, B, sz0, marshall):
    # configurations drawn from the model (by the oracle's sampler), as in a VMC step
    desc, d32, mod, pf, p = setup(Lx, Ly, d, sz0, seed=2)
    sig = om.sample(mod, pf, philox.sampling_uniforms(17, 0, B, mod.N))["sigma"].astype(np.uint8)
    sg = dev(sig, torch.uint8)
    ham = nqs.heisenberg(1.0, marshall)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    el = nqs.local_energy(desc, p, ham, sg, hc, ws=ws)
    _, hc32 = nqs.logpsi(d32, p, sg)
    el32 = nqs.local_energy(d32, p, ham, sg, hc32)
    torch.cuda.synchronize()
    assert ws.status() == 0
    ref = oh.heisenberg_local_energy(Lx, Ly, 1.0, marshall, sig.astype(np.int64), lambda x: om.logpsi(mod, pf, x))
    e16 = el.double().cpu().numpy()
    assert np.isfinite(e16).all()
    assert abs(e16.mean() - ref.mean()) / mod.N <= 1e-4
    assert abs(e16.mean() - el32.double().cpu().numpy().mean()) / mod.N <= 1e-4
    assert_eloc_per_sample(e16, ref, sig, Lx, Ly, 1.0, mod.N)


def test_bf16_2d_vmc_gradient_cosine():
    Lx, Ly, d, B = 4, 4, 32, 128
    desc, _, mod, pf, p = setup(Lx, Ly, d, True, seed=8, noise=0.05)
    sig = om.sample(mod, pf, philox.sampling_uniforms(19, 0, B, mod.N))["sigma"].astype(np.uint8)
    sg = dev(sig, torch.uint8)
    _, hc = nqs.logpsi(desc, p, sg)
    el = nqs.local_energy(desc, p, nqs.heisenberg(), sg, hc)
    g, st = nqs.vmc_grad(desc, p, sg, hc, el)
    torch.cuda.synchronize()
    e_ref = oh.heisenberg_local_energy(Lx, Ly, 1.0, True, sig.astype(np.int64), lambda x: om.logpsi(mod, pf, x))
    ref = ov.vmc_gradient(mod, pf, sig.astype(np.int64), e_ref)
    g = g.double().cpu().numpy()
    assert g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref)) >= 0.999


@pytest.mark.parametrize("Lx,Ly,d,B,sz0", [(4, 4, 32, 100, True), (8, 8, 64, 64, True), (3, 5, 32, 77, False),
                                           (4, 6, 64, 130, True)])
def test_bf16_2d_logpsi_grad(Lx, Ly, d, B, sz0):
    desc, d32, mod, pf, p = setup(Lx, Ly, d, sz0, seed=5, noise=0.05)
    sig = inputs.random_configs(B, mod.N, seed=6, sz0=sz0)
    w = inputs.random_weights(B, seed=7).astype(np.float32)
    sg = dev(sig, torch.uint8)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    g = nqs.logpsi_grad(desc, p, sg, hc, dev(w), ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    ref = ov.logpsi_grad(mod, pf, sig.astype(np.int64), w.astype(np.float64))
    g = g.double().cpu().numpy()
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert cos >= 0.999 and rel <= 2e-2, (cos, rel)


@pytest.mark.parametrize("Lx,Ly,B", [(8, 8, 300), (6, 4, 77)])
def test_bf16_2d_forward_tile_rows_agree(Lx, Ly, B):
    """Sampling and teacher forcing at d_h = 64 on 32-sample CTAs (every A row
    in all four TMEM lane quarters, the units split over the quarters' warps)
    and on 128-sample CTAs give bitwise the same samples, log psi and cache:
    the readout sums 16-unit chunks in order and the chunks by a fixed tree in
    both.  B is not a multiple of 32 (ragged last CTA)."""
    desc, _, mod, pf, p = setup(Lx, Ly, 64, True, seed=12)
    out = []
    for v in (0, 1):
        nqs.set_tile_variant(v)
        s, lp, hc = nqs.sample(desc, p, B, seed=4, step=3)
        lp_t, hc_t = nqs.logpsi(desc, p, s)
        out.append((s.clone(), lp.clone(), hc.clone(), lp_t.clone(), hc_t.clone()))
    nqs.set_tile_variant(None)
    torch.cuda.synchronize()
    assert torch.isfinite(out[0][1]).all()
    for x, y in zip(out[0], out[1]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("Lx,Ly,d,B", [(4, 4, 32, 90), (8, 8, 64, 70), (8, 8, 64, 1500), (6, 6, 32, 2000),
                                        (16, 16, 64, 40)])
def test_bf16_2d_chains_split_rows_agree(Lx, Ly, d, B):
    """The Heisenberg chains on two 128-row tiles per CTA with one thread per
    row (the default, variant 2) or two (variant 3), on one tile with one
    thread per row (variant 0) and on one tile with the units of a row split
    over several warps (variant 1); with split rows part 0 pulls the jobs and
    publishes them.  All give bitwise the same local energies.  The larger batches
    hold more chain jobs than the grid has rows, so rows take several jobs from
    the queue; 16 x 16 runs on 256-bit configuration masks."""
    desc, _, mod, pf, p = setup(Lx, Ly, d, True, seed=13, noise=0.0 if Lx * Ly > 128 else 0.1)
    sg = dev(inputs.random_configs(B, mod.N, seed=14, sz0=True), torch.uint8)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    out = []
    for v in (None, 0, 1, 2, 3):
        nqs.set_tile_variant(v)
        out.append(nqs.local_energy(desc, p, nqs.heisenberg(), sg, hc, ws=ws).clone())
    nqs.set_tile_variant(None)
    torch.cuda.synchronize()
    assert ws.status() == 0
    assert torch.isfinite(out[0]).all()
    for k in range(1, len(out)):
        assert torch.equal(out[0], out[k]), k


@pytest.mark.parametrize("Lx,Ly,d,B", [(4, 4, 32, 300), (6, 4, 64, 200)])
def test_bf16_2d_grad_tile_rows_agree(Lx, Ly, d, B):
    """The sequential sweep on 32-sample tiles (the TMEM lane quarters split the
    units and exchange dh' through shared memory) and on 128-sample tiles gives
    bitwise the same gradient: the MMA rows are independent and the exchange
    copies FP32 values.  B is not a multiple of 128 (ragged last tile)."""
    desc, d32, mod, pf, p = setup(Lx, Ly, d, True, seed=9, noise=0.05)
    sig = inputs.random_configs(B, mod.N, seed=10, sz0=True)
    w = inputs.random_weights(B, seed=11).astype(np.float32)
    sg = dev(sig, torch.uint8)
    ws = nqs.Workspace(DEV)
    _, hc = nqs.logpsi(desc, p, sg, ws=ws)
    out = []
    for v in (0, 1):
        nqs.set_tile_variant(v)
        out.append(nqs.logpsi_grad(desc, p, sg, hc, dev(w), ws=ws).clone())
    nqs.set_tile_variant(None)
    torch.cuda.synchronize()
    assert ws.status() == 0
    assert torch.isfinite(out[0]).all()
    assert torch.equal(out[0], out[1])


def test_bf16_2d_full_size_8x8_d64_b2048():
    """Heisenberg 8 x 8 workload in BF16: every draw of the step's sampling;
    energy per site of the whole step within 1e-4 of the FP32 path on the same
    samples and of the oracle on 12 of them (each also within the per-sample
    bound); the reverse sweep at the full batch (the step's launch
    configuration) against the oracle's gradient on 32 samples (weights zero
    elsewhere)."""
    Lx, Ly, d, B = 8, 8, 64, 2048
    desc, d32, mod, pf, p = setup(Lx, Ly, d, True, seed=0)
    ws = nqs.Workspace(DEV)
    sig, lp, hc = nqs.sample(desc, p, B, seed=5, step=0, ws=ws)
    el = nqs.local_energy(desc, p, nqs.heisenberg(), sig, hc, ws=ws)
    g, st = nqs.vmc_grad(desc, p, sig, hc, el, ws=ws)
    _, hc32 = nqs.logpsi(d32, p, sig)
    el32 = nqs.local_energy(d32, p, nqs.heisenberg(), sig, hc32)
    torch.cuda.synchronize()
    assert ws.status() == 0
    e16, e32 = el.double().cpu().numpy(), el32.double().cpu().numpy()
    assert abs(e16.mean() - e32.mean()) / mod.N <= 1e-4
    s = sig.cpu().numpy().astype(np.int64)
    frac, _ = check_draws(mod, pf, s, philox.sampling_uniforms(5, 0, B, mod.N), sample_window(mod))
    assert frac <= 1e-2, frac
    pick = np.random.default_rng(3).choice(B, 12, replace=False)
    e_ref = oh.heisenberg_local_energy(Lx, Ly, 1.0, True, s[pick], lambda x: om.logpsi(mod, pf, x))
    assert abs(e16[pick].mean() - e_ref.mean()) / mod.N <= 1e-4
    assert_eloc_per_sample(e16[pick], e_ref, s[pick], Lx, Ly, 1.0, mod.N)
    assert np.isfinite(g.cpu().numpy()).all()
    gpick = np.random.default_rng(4).choice(B, 32, replace=False)
    w = np.zeros(B, dtype=np.float32)
    w[gpick] = (2.0 * (e16[gpick] - e16.mean()) / B).astype(np.float32)
    gp = nqs.logpsi_grad(desc, p, sig, hc, dev(w), ws=ws)
    torch.cuda.synchronize()
    assert ws.status() == 0
    g_ref = ov.logpsi_grad(mod, pf, s[gpick], w[gpick].astype(np.float64))
    gp = gp.double().cpu().numpy()
    cos = gp @ g_ref / (np.linalg.norm(gp) * np.linalg.norm(g_ref))
    rel = np.linalg.norm(gp - g_ref) / np.linalg.norm(g_ref)
    assert cos >= 0.999 and rel <= 2e-2, (cos, rel)


@pytest.mark.parametrize("d", [32, 64])
def test_bf16_2d_16x16(d):
    """256 sites at d_h 32 / 64 (256-bit configuration masks, NW = 4 engine):
    log psi and cache against the BF16-weight model (2e-6 N, 5e-4 max |h|)
    and the exact one (6e-4 N, 3e-2); every draw against both models
    (windows: 1e-4, and the exact / BF16-weight p0 gap + 1e-4); per-sample
    local energies against the FP32 path and on 2 samples the oracle; the
    reverse sweep against the oracle's gradient.  Xavier weights without
    noise: with noise the 16 x 16 map expands and the exact model leaves the
    BF16 one."""
    Lx = Ly = 16
    desc, d32, mod, pf, p = setup(Lx, Ly, d, True, seed=9, noise=0.0)
    sig = inputs.random_configs(6, mod.N, seed=4, sz0=True)
    lp, hc = nqs.logpsi(desc, p, dev(sig, torch.uint8))
    torch.cuda.synchronize()
    ref_b = om.run(mod, bf16_weight_model(mod, pf), sigma=sig.astype(np.int64))
    np.testing.assert_allclose(lp.cpu().numpy(), ref_b["logpsi"], atol=2e-6 * mod.N, rtol=0)
    np.testing.assert_allclose(hc.cpu().numpy(), ref_b["hidden"], atol=5e-4 * np.abs(ref_b["hidden"]).max(), rtol=0)
    ref = om.run(mod, pf, sigma=sig.astype(np.int64))
    np.testing.assert_allclose(lp.cpu().numpy(), ref["logpsi"], atol=6e-4 * mod.N, rtol=0)
    np.testing.assert_allclose(hc.cpu().numpy(), ref["hidden"], atol=3e-2, rtol=0)
    # sampling
    B = 24
    s, _, _ = nqs.sample(desc, p, B, seed=3, step=1)
    torch.cuda.synchronize()
    s = s.cpu().numpy().astype(np.int64)
    assert np.all(s.sum(axis=1) == mod.N // 2)
    u = philox.sampling_uniforms(3, 1, B, mod.N)
    frac_b, _ = check_draws(mod, bf16_weight_model(mod, pf), s, u, 1e-4)
    assert frac_b <= 1e-3, frac_b
    frac, _ = check_draws(mod, pf, s, u, draw_window(mod, pf, s))
    assert frac <= 1e-2, frac
    # local energies
    sm = om.sample(mod, pf, philox.sampling_uniforms(17, 0, 16, mod.N))["sigma"].astype(np.uint8)
    sg = dev(sm, torch.uint8)
    ws = nqs.Workspace(DEV)
    _, hcs = nqs.logpsi(desc, p, sg, ws=ws)
    el = nqs.local_energy(desc, p, nqs.heisenberg(), sg, hcs, ws=ws)
    _, hc32 = nqs.logpsi(d32, p, sg)
    el32 = nqs.local_energy(d32, p, nqs.heisenberg(), sg, hc32)
    torch.cuda.synchronize()
    assert ws.status() == 0
    e16, e32 = el.double().cpu().numpy(), el32.double().cpu().numpy()
    assert abs(e16.mean() - e32.mean()) / mod.N <= 1e-4
    assert_eloc_per_sample(e16, e32, sm, Lx, Ly, 1.0, mod.N)
    e_ref = oh.heisenberg_local_energy(Lx, Ly, 1.0, True, sm[:2].astype(np.int64), lambda x: om.logpsi(mod, pf, x))
    assert_eloc_per_sample(e16[:2], e_ref, sm[:2], Lx, Ly, 1.0, mod.N)
    # reverse sweep
    w = inputs.random_weights(6, seed=7).astype(np.float32)
    g = nqs.logpsi_grad(desc, p, dev(sig, torch.uint8), hc, dev(w))
    torch.cuda.synchronize()
    g_ref = ov.logpsi_grad(mod, pf, sig.astype(np.int64), w.astype(np.float64))
    g = g.double().cpu().numpy()
    cos = g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref))
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert cos >= 0.999 and rel <= 2e-2, (cos, rel)


@pytest.mark.parametrize("Lx,Ly,d", [(4, 4, 128), (17, 16, 64), (4, 4, 16), (16, 17, 32)])
def test_bf16_2d_unsupported_shapes(Lx, Ly, d):
    desc = nqs.model_desc(nqs.GRU2D, Lx, Ly, d, sz0=True, precision=nqs.BF16)
    p = torch.zeros(nqs.param_count(desc), device=DEV)
    with pytest.raises(nqs.NqsError):
        nqs.sample(desc, p, 8, seed=0, step=0)
