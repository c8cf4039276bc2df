"""Failure detection without a GPU fault: a non-finite value met on the device
is reported through the workspace status word (NQS_ENONFINITE), the call
itself returns normally, and the next call on the same workspace starts from
a clean word.  The failure is made on the host: one weight is set to NaN."""
import numpy as np
import pytest
import torch

from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ENONFINITE = 6


@pytest.mark.parametrize("cell,Lx,Ly,d,sz0,precision", [
    (nqs.GRU1D, 30, 1, 16, False, nqs.FP32), (nqs.GRU1D, 30, 1, 32, False, nqs.BF16),
    (nqs.GRU2D, 4, 4, 16, True, nqs.FP32), (nqs.GRU2D, 4, 4, 32, True, nqs.BF16)])
def test_nan_weight_sets_nonfinite_status(cell, Lx, Ly, d, sz0, precision):
    desc = nqs.model_desc(cell, Lx, Ly, d, sz0=sz0, precision=precision)
    ham = nqs.tfim() if cell == nqs.GRU1D else nqs.heisenberg()
    flat = inputs.xavier_params(cell, d, seed=1, noise_std=0.05).astype(np.float32)
    good = torch.tensor(flat, device=DEV)
    bad = good.clone()
    bad[3] = float("nan")                     # a recurrent weight of the first gate block
    ws = nqs.Workspace(DEV)
    B = 64
    # sampling and local energy with the NaN weight: the calls return, the word says why
    s, lp, hc = nqs.sample(desc, bad, B, seed=1, step=0, ws=ws)
    assert ws.status() == ENONFINITE
    assert not torch.isfinite(lp).all()
    el = nqs.local_energy(desc, bad, ham, s, hc, ws=ws)
    assert ws.status() == ENONFINITE
    assert not torch.isfinite(el).all()
    # the same workspace serves a clean call afterwards
    s, lp, hc = nqs.sample(desc, good, B, seed=1, step=0, ws=ws)
    el = nqs.local_energy(desc, good, ham, s, hc, ws=ws)
    g, st = nqs.vmc_grad(desc, good, s, hc, el, ws=ws)
    assert ws.status() == 0
    torch.cuda.synchronize()
    assert torch.isfinite(lp).all() and torch.isfinite(el).all() and torch.isfinite(g).all()


@pytest.mark.parametrize("cell,Lx,Ly,d,sz0", [(nqs.GRU1D, 30, 1, 32, False), (nqs.GRU2D, 4, 4, 32, True)])
def test_wait_that_gives_up_sets_timeout_status(cell, Lx, Ly, d, sz0):
    """With the wait bound at 0 polls every tensor-core wait that may give up
    does so at once: each call (sampling, teacher forcing, local energy,
    gradient) records NQS_ETIMEOUT and returns; the kernels free their tensor
    memory only after their MMAs drained, so the context stays usable and the
    next calls with the default bound reproduce the clean results bitwise.
    The inputs of the timed-out calls are the clean run's (valid) ones."""
    ETIMEOUT = 5
    desc = nqs.model_desc(cell, Lx, Ly, d, sz0=sz0, precision=nqs.BF16)
    ham = nqs.tfim() if cell == nqs.GRU1D else nqs.heisenberg()
    p = torch.tensor(inputs.xavier_params(cell, d, seed=2, noise_std=0.05).astype(np.float32), device=DEV)
    ws = nqs.Workspace(DEV)
    B = 200
    nqs.set_autotune(False)                  # no tuning on timed-out runs
    try:
        s, lp, hc = nqs.sample(desc, p, B, seed=3, step=1, ws=ws)
        el = nqs.local_energy(desc, p, ham, s, hc, ws=ws)
        g, st = nqs.vmc_grad(desc, p, s, hc, el, ws=ws)
        assert ws.status() == 0
        nqs.set_wait_limit(0)
        try:
            nqs.sample(desc, p, B, seed=3, step=1, ws=ws)
            assert ws.status() == ETIMEOUT
            nqs.logpsi(desc, p, s, ws=ws)
            assert ws.status() == ETIMEOUT
            nqs.local_energy(desc, p, ham, s, hc, ws=ws)
            assert ws.status() == ETIMEOUT
            nqs.vmc_grad(desc, p, s, hc, el, ws=ws)
            assert ws.status() == ETIMEOUT
        finally:
            nqs.set_wait_limit(None)
        s2, lp2, hc2 = nqs.sample(desc, p, B, seed=3, step=1, ws=ws)
        el2 = nqs.local_energy(desc, p, ham, s2, hc2, ws=ws)
        g2, st2 = nqs.vmc_grad(desc, p, s2, hc2, el2, ws=ws)
        assert ws.status() == 0
        torch.cuda.synchronize()
        for x, y in ((s, s2), (lp, lp2), (hc, hc2), (el, el2), (g, g2), (st, st2)):
            assert torch.equal(x, y)
    finally:
        nqs.set_autotune(True)
