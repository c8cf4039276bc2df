"""nqs_local_energy_static: local energies with no caller workspace.

Callers that cannot allocate device memory (a plugin whose host owns every
allocation, a latency-critical loop, a binding without a device allocator)
use this entry point; its scratch is a fixed device array inside the library.
The test calls it through the C ABI twice in a row, on different batches, and
checks each result against nqs_local_energy (the workspace version) within the
local-energy tolerance of the parity tests.  It builds its own inputs, so it
passes alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2507_18700_gb300 import build as nqs_build
from paper_2507_18700_gb300 import inputs, nqs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def entry_point():
    nqs_build.build()
    L = nqs.lib()
    f = L.nqs_local_energy_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(nqs.ModelDesc), ctypes.c_void_p, ctypes.POINTER(nqs.HamDesc),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    return f


def call_static(f, desc, p, ham, sigma, hcache, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(ctypes.byref(desc), ctypes.c_void_p(p.data_ptr()), ctypes.byref(ham),
             ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(hcache.data_ptr()),
             sigma.shape[0], ctypes.c_void_p(out.data_ptr()), stream)


def test_static_scratch_local_energy_matches_workspace_version():
    f = entry_point()
    torch.cuda.set_device(DEV)
    N, d, Gamma = 100, 64, 1.0
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d)
    ham = nqs.tfim(1.0, Gamma)
    p = torch.tensor(inputs.xavier_params(1, d, seed=1, noise_std=0.1).astype(np.float32), device=DEV)
    tol = 2e-5 * N * (1 + Gamma)
    for B, seed in ((4096, 7), (333, 8)):          # two calls in a row on the shared array
        sig = torch.tensor(inputs.random_configs(B, N, seed=seed), device=DEV)
        _, hc = nqs.logpsi(desc, p, sig)
        ref = nqs.local_energy(desc, p, ham, sig, hc)
        out = torch.full((B,), float("nan"), dtype=torch.float32, device=DEV)
        assert call_static(f, desc, p, ham, sig, hc, out) == 0
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), atol=tol, rtol=0)


def test_static_scratch_rejects_batches_beyond_its_capacity():
    f = entry_point()
    N, d = 100, 64
    desc = nqs.model_desc(nqs.GRU1D, N, 1, d)
    ham = nqs.tfim()
    fake = ctypes.c_void_p(0x1000)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    too_many = 1 << 20                              # B * N = 1e8 floats, far beyond 16 MiB
    assert f(ctypes.byref(desc), fake, ctypes.byref(ham), fake, fake, too_many, fake, stream) == 3
