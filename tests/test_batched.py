"""Batched VMC step over replicas of uneven hidden size (the Adaptive growth
family, Sec. II B) against the float64 oracle, and its CUDA-graph replay."""
import numpy as np
import pytest
import torch

from oracle import hamiltonian as oh, model as om, philox, vmc as ov
from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def make_models(N, specs, seed=3):
    models = []
    for i, (d, B, Gamma) in enumerate(specs):
        flat = inputs.xavier_params(1, d, seed=seed + i, noise_std=0.1).astype(np.float32)
        models.append((nqs.model_desc(nqs.GRU1D, N, 1, d), nqs.tfim(1.0, Gamma), B, 100 + i,
                       torch.tensor(flat, device=DEV)))
    return models


def test_batched_step_matches_oracle_per_replica():
    N = 20
    specs = [(16, 64, 0.5), (32, 100, 1.0), (64, 37, 1.5), (128, 50, 2.0), (16, 129, 1.0)]
    models = make_models(N, specs)
    batch = nqs.ReplicaBatch(models)
    out = batch.step(step_no=3)
    torch.cuda.synchronize()
    assert batch.ws.status() == 0
    for (desc, ham, B, seed, p), o in zip(models, out):
        mod = om.Model(om.GRU1D, N, d_h=desc.d_h)
        pf = p.double().cpu().numpy()
        u = philox.sampling_uniforms(seed, 3, B, N)
        ref = om.sample(mod, pf, u)
        assert not (np.abs(u - ref["p0"]) < 1e-6).any()
        np.testing.assert_array_equal(o["sigma"].cpu().numpy(), ref["sigma"])
        np.testing.assert_allclose(o["logpsi"].cpu().numpy(), ref["logpsi"], atol=1e-4, rtol=0)
        e_ref = oh.tfim_local_energy(N, 1.0, ham.h, ref["sigma"], lambda x: om.logpsi(mod, pf, x))
        np.testing.assert_allclose(o["eloc"].cpu().numpy(), e_ref, atol=2e-5 * N * (1 + ham.h), rtol=0)
        np.testing.assert_allclose(o["stats"].cpu().numpy(),
                                   ov.energy_stats(o["eloc"].double().cpu().numpy()), rtol=1e-9, atol=1e-9)
        g_ref = ov.vmc_gradient(mod, pf, ref["sigma"], e_ref)
        g = o["grad"].double().cpu().numpy()
        rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
        assert rel < 1e-3, rel


def test_batched_step_equals_single_model_calls():
    N = 30
    specs = [(16, 80, 1.0), (64, 120, 0.7)]
    models = make_models(N, specs, seed=11)
    out = nqs.ReplicaBatch(models).step(step_no=5)
    for (desc, ham, B, seed, p), o in zip(models, out):
        s, lp, hc = nqs.sample(desc, p, B, seed=seed, step=5)
        el = nqs.local_energy(desc, p, ham, s, hc)
        g, st = nqs.vmc_grad(desc, p, s, hc, el)
        torch.cuda.synchronize()
        assert torch.equal(s, o["sigma"]) and torch.equal(lp, o["logpsi"])
        assert torch.equal(el, o["eloc"]) and torch.equal(st, o["stats"])
        torch.testing.assert_close(g, o["grad"], rtol=1e-5, atol=1e-7)


def test_device_step_counter_and_graph_replay():
    N = 16
    specs = [(16, 64, 1.0), (32, 64, 2.0)]
    models = make_models(N, specs, seed=21)
    eager = nqs.ReplicaBatch(models, device_step=True)
    ref = []
    for k in range(3):
        o = eager.step()
        torch.cuda.synchronize()
        ref.append([x["sigma"].clone() for x in o] + [x["grad"].clone() for x in o])
    assert int(eager.step_dev.item()) == 3
    assert not torch.equal(ref[0][0], ref[1][0])
    # same three steps through a captured graph
    graphed = nqs.ReplicaBatch(models, device_step=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        graphed.step()                       # warm-up outside the capture: module loading, step 0
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = [x["sigma"].clone() for x in graphed.out] + [x["grad"].clone() for x in graphed.out]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        graphed.step()
    for k in (1, 2):
        g.replay()
        torch.cuda.synchronize()
        got = [x["sigma"] for x in graphed.out] + [x["grad"] for x in graphed.out]
        for a, b in zip(got, ref[k]):
            assert torch.equal(a, b)
    for a, b in zip(first, ref[0]):
        assert torch.equal(a, b)
    assert int(graphed.step_dev.item()) == 3


def test_batched_rejects_unsupported_replicas():
    flat = torch.zeros(nqs.param_count(nqs.model_desc(1, 10, 1, 8)), device=DEV)
    with pytest.raises(nqs.NqsError):
        nqs.ReplicaBatch([(nqs.model_desc(1, 10, 1, 8), nqs.tfim(), 4, 0, flat)])      # d_h 8
    p2 = torch.zeros(nqs.param_count(nqs.model_desc(2, 4, 4, 16)), device=DEV)
    with pytest.raises(nqs.NqsError):
        nqs.ReplicaBatch([(nqs.model_desc(2, 4, 4, 16), nqs.heisenberg(), 4, 0, p2)])  # 2D


def make_mixed(N, specs, seed=31):
    """specs: (d_h, B, Gamma, precision)."""
    models = []
    for i, (d, B, Gamma, prec) in enumerate(specs):
        flat = inputs.xavier_params(1, d, seed=seed + i, noise_std=0.1).astype(np.float32)
        models.append((nqs.model_desc(nqs.GRU1D, N, 1, d, precision=prec), nqs.tfim(1.0, Gamma), B, 200 + i,
                       torch.tensor(flat, device=DEV)))
    return models


def test_batched_bf16_replicas_equal_single_model_calls():
    """BF16 replicas (d_h 16..128) in one batched call with FP32 ones: each BF16
    replica's samples, log psi, local energies, statistics and gradient are
    bitwise those of its own tensor-core calls; the FP32 replicas as before."""
    N = 40
    specs = [(16, 90, 1.0, nqs.BF16), (32, 64, 0.5, nqs.FP32), (64, 130, 1.5, nqs.BF16), (128, 70, 2.0, nqs.BF16),
             (128, 33, 1.0, nqs.FP32)]
    models = make_mixed(N, specs)
    batch = nqs.ReplicaBatch(models)
    out = batch.step(step_no=7)
    torch.cuda.synchronize()
    assert batch.ws.status() == 0
    for (desc, ham, B, seed, p), o in zip(models, out):
        s, lp, hc = nqs.sample(desc, p, B, seed=seed, step=7)
        el = nqs.local_energy(desc, p, ham, s, hc)
        g, st = nqs.vmc_grad(desc, p, s, hc, el)
        torch.cuda.synchronize()
        assert torch.equal(s, o["sigma"]) and torch.equal(lp, o["logpsi"])
        assert torch.equal(el, o["eloc"]) and torch.equal(st, o["stats"])
        if desc.precision == nqs.BF16:
            assert torch.equal(g, o["grad"])
        else:
            torch.testing.assert_close(g, o["grad"], rtol=1e-5, atol=1e-7)


def test_batched_bf16_graph_replay():
    """All-BF16 replicas with the device step counter: graph replays equal eager
    steps bitwise, and the counter advances once per step."""
    N = 24
    specs = [(16, 64, 1.0, nqs.BF16), (64, 64, 2.0, nqs.BF16), (128, 40, 0.7, nqs.BF16)]
    models = make_mixed(N, specs, seed=41)
    eager = nqs.ReplicaBatch(models, device_step=True)
    ref = []
    for k in range(3):
        o = eager.step()
        torch.cuda.synchronize()
        ref.append([x["sigma"].clone() for x in o] + [x["grad"].clone() for x in o])
    assert int(eager.step_dev.item()) == 3
    graphed = nqs.ReplicaBatch(models, device_step=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        graphed.step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        graphed.step()
    for k in (1, 2):
        g.replay()
        torch.cuda.synchronize()
        got = [x["sigma"] for x in graphed.out] + [x["grad"] for x in graphed.out]
        for a, b in zip(got, ref[k]):
            assert torch.equal(a, b)
    assert int(graphed.step_dev.item()) == 3
