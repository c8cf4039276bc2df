"""Training loop and final evaluation on the GPU.

* nqs_adam_step against the oracle's float64 Adam over steps that cross the
  schedules' switch points (FP32 parameters and moments: relative 1e-5);
* a captured CUDA graph of k training steps reproduces k eager steps bitwise
  (samples drawn from the device step counter, statistics log, Adam state);
* growth carries the moments with zero padding;
* a short training run of the 12-site TFIM (GRU d_h 8, B 512, Xavier seed 0)
  lowers the energy toward the exact ground energy and stays above it;
* nqs_evaluate agrees with one large sampling + local-energy call (FP64 sums
  grouped by chunk) and, with 2e5 samples of the 12-site model, with the
  exact energy by enumeration within 4 standard errors.
"""
import numpy as np
import pytest
import torch

from oracle import adam as oa, exact, hamiltonian as oh, model as om
from paper_2507_18700_gb300 import inputs, nqs
from paper_2507_18700_gb300.train import Trainer

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_adam_step_matches_oracle():
    P = 1000
    x0 = inputs.random_weights(P, seed=1).astype(np.float32)
    grads = [inputs.random_weights(P, seed=10 + k, scale=0.5).astype(np.float32) for k in range(6)]
    for sched, ref_fn in ((nqs.lr_step(5e-3, 5e-4, 3), oa.lr_step(5e-3, 5e-4, 3)),
                          (nqs.lr_inverse(1e-2, 2.0, 2), oa.lr_inverse(1e-2, 2.0, 2))):
        p = torch.tensor(x0, device=DEV)
        m, v = torch.zeros_like(p), torch.zeros_like(p)
        t = torch.zeros((1,), dtype=torch.int64, device=DEV)
        for g in grads:
            nqs.adam_step(p, m, v, torch.tensor(g, device=DEV), nqs.adam_desc(), sched, t_dev=t)
        torch.cuda.synchronize()
        assert int(t.item()) == len(grads)
        xr, mr, vr = oa.adam(x0.astype(np.float64), [g.astype(np.float64) for g in grads], ref_fn)
        # FP32 moments: each of the 6 updates rounds terms of size up to |g|
        # (m) and g^2 (v), so the absolute error is a few 1e-8 |g|_max where
        # the moment itself cancels to a small value
        gmax = max(np.abs(g).max() for g in grads)
        np.testing.assert_allclose(p.cpu().numpy(), xr, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(m.cpu().numpy(), mr, rtol=1e-5, atol=1e-7 * gmax)
        np.testing.assert_allclose(v.cpu().numpy(), vr, rtol=1e-5, atol=1e-7 * gmax ** 2)
    # a float64 gradient (the rank-summed one) and a host step give the same update
    p1 = torch.tensor(x0, device=DEV)
    p2 = p1.clone()
    z = [torch.zeros_like(p1) for _ in range(4)]
    g = torch.tensor(grads[0], device=DEV)
    nqs.adam_step(p1, z[0], z[1], g, nqs.adam_desc(), nqs.lr_constant(1e-3), t=4)
    nqs.adam_step(p2, z[2], z[3], g.double(), nqs.adam_desc(), nqs.lr_constant(1e-3), t=4)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)


@pytest.mark.parametrize("precision", [nqs.FP32, nqs.BF16])
def test_graph_replay_equals_eager_steps(precision):
    N, d, B, k = 20, 16, 256, 4
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d, precision=precision)
    p0 = torch.tensor(inputs.xavier_params(1, d, seed=3, noise_std=0.05).astype(np.float32), device=DEV)
    a = Trainer(desc, p0, nqs.tfim(1.0, 1.0), B, seed=5, sched=nqs.lr_constant(1e-2))
    b = Trainer(desc, p0, nqs.tfim(1.0, 1.0), B, seed=5, sched=nqs.lr_constant(1e-2))
    a.capture(k)                              # one eager warm-up step, then k steps recorded
    a.replay()
    for _ in range(k + 1):
        b.step()
    torch.cuda.synchronize()
    assert a.steps_done() == b.steps_done() == k + 1
    for x, y in ((a.params, b.params), (a.m, b.m), (a.v, b.v), (a.sigma, b.sigma), (a.log, b.log)):
        assert torch.equal(x, y)
    h = a.history()
    assert h.shape[0] == k + 1 and list(h[:, 0].long()) == list(range(k + 1))


def test_growth_carries_moments_with_zero_padding():
    N, d = 12, 8
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d)
    p0 = torch.tensor(inputs.xavier_params(1, d, seed=0).astype(np.float32), device=DEV)
    tr = Trainer(desc, p0, nqs.tfim(), 128, seed=1, sched=nqs.lr_constant(1e-2))
    for _ in range(3):
        tr.step()
    m_small, v_small = tr.m.clone(), tr.v.clone()
    tr.grow(16)
    torch.cuda.synchronize()
    big = om.Model(om.GRU1D, N, d_h=16)
    small = om.Model(om.GRU1D, N, d_h=d)
    from oracle import growth
    ref_m = growth.grow(small, m_small.double().cpu().numpy(), big, seed=2, eps=0.0)
    ref_v = growth.grow(small, v_small.double().cpu().numpy(), big, seed=2, eps=0.0)
    np.testing.assert_array_equal(tr.m.double().cpu().numpy(), ref_m)
    np.testing.assert_array_equal(tr.v.double().cpu().numpy(), ref_v)
    tr.step()
    torch.cuda.synchronize()
    assert tr.steps_done() == 4 and torch.isfinite(tr.params).all()


def test_short_training_lowers_the_energy():
    """12-site TFIM at Gamma = 1 (exact ground energy -14.925971...): 120 Adam
    steps at lr 1e-2 from Xavier weights; the mean energy of the last 20 steps
    is below that of the first 20 by at least 0.5 and above E0 - 0.05 (the
    variational bound, up to the sampling error of 512 samples)."""
    N, d, B = 12, 8, 512
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d)
    p0 = torch.tensor(inputs.xavier_params(1, d, seed=0).astype(np.float32), device=DEV)
    tr = Trainer(desc, p0, nqs.tfim(1.0, 1.0), B, seed=0, sched=nqs.lr_constant(1e-2))
    tr.capture(20)
    for _ in range(6):
        tr.replay()
    torch.cuda.synchronize()
    h = tr.history().numpy()
    assert h.shape[0] == 121
    e = h[:, 1]
    e0 = exact.tfim_closed_form_critical(N)
    assert e[-20:].mean() < e[:20].mean() - 0.5, (e[:20].mean(), e[-20:].mean())
    assert e[-20:].mean() > e0 - 0.05
    assert np.all(h[:, 2] >= 0)


@pytest.mark.parametrize("precision", [nqs.FP32, nqs.BF16])
def test_evaluate_equals_one_large_call(precision):
    N, d, M, chunk = 40, 32, 10007, 3000
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d, precision=precision)
    p = torch.tensor(inputs.xavier_params(1, d, seed=6, noise_std=0.05).astype(np.float32), device=DEV)
    ham = nqs.tfim(1.0, 0.8)
    st = nqs.evaluate(desc, p, ham, M, chunk=chunk, seed=7, step=2)
    s, _, hc = nqs.sample(desc, p, M, seed=7, step=2)
    el = nqs.local_energy(desc, p, ham, s, hc).double()
    torch.cuda.synchronize()
    mean = el.mean().item()
    var = (el * el).mean().item() - mean * mean
    got = st.cpu().numpy()
    assert got[2] == M
    np.testing.assert_allclose(got[0], mean, rtol=1e-12)
    np.testing.assert_allclose(got[1], var, rtol=1e-9)
    np.testing.assert_allclose(got[3], np.sqrt(var / M), rtol=1e-9)
    np.testing.assert_allclose(got[4], var * np.sqrt(2.0 / (M - 1)), rtol=1e-9)


def test_evaluate_matches_exact_energy():
    N, d = 12, 8
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d)
    flat = inputs.xavier_params(1, d, seed=0, noise_std=0.3).astype(np.float32)
    st = nqs.evaluate(desc, torch.tensor(flat, device=DEV), nqs.tfim(1.0, 1.0), 200_000, chunk=65536, seed=3)
    torch.cuda.synchronize()
    mod = om.Model(om.GRU1D, N, d_h=d)
    pf = flat.astype(np.float64)
    configs = exact.all_configs(N)
    P = np.exp(2 * om.logpsi(mod, pf, configs))
    el = oh.tfim_local_energy(N, 1.0, 1.0, configs, lambda x: om.logpsi(mod, pf, x))
    e_exact = exact.exact_energy(P, el)
    var_exact = float(np.sum(P * el * el) - e_exact ** 2)
    got = st.cpu().numpy()
    assert abs(got[0] - e_exact) < 4 * got[3], (got[0], e_exact, got[3])
    assert abs(got[1] - var_exact) < 5 * got[4] + 1e-6, (got[1], var_exact, got[4])
