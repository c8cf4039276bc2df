"""The C-ABI library: it loads, exports every declared symbol, and rejects bad
arguments on the host before touching the GPU (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

from oracle import model as om
from paper_2507_18700_gb300 import build as nqs_build
from paper_2507_18700_gb300 import inputs, nqs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    nqs_build.build()
    return nqs.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "nqs.h")).read()
    return sorted(set(re.findall(r"^\s*(?:size_t|nqs_status|const char\*|void)\s+(nqs_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    assert sorted(names) == sorted(nqs.EXPORTS)


@pytest.mark.parametrize("cell,Lx,Ly,d", [(1, 12, 1, 8), (1, 100, 1, 64), (1, 20, 1, 128),
                                          (2, 8, 8, 64), (2, 4, 4, 16), (2, 16, 16, 256)])
def test_param_count_matches_layouts(L, cell, Lx, Ly, d):
    desc = nqs.model_desc(cell, Lx, Ly, d)
    n = L.nqs_param_count(ctypes.byref(desc))
    if cell == 2 and d == 256:
        assert n in (0, om.Model(cell, Lx, Ly, d_h=d).param_count())
        return
    assert n == om.Model(cell, Lx, Ly, d_h=d).param_count() == inputs.param_count(cell, d)


@pytest.mark.parametrize("d", [16, 64, 128])
def test_param_count_of_the_crnn(L, d):
    desc = nqs.model_desc(1, 30, 1, d, phase=True)
    assert L.nqs_param_count(ctypes.byref(desc)) == om.Model(1, 30, 1, d_h=d, phase=True).param_count() \
        == inputs.param_count(1, d, phase=True)
    # built only on the FP32 1D path with d_h >= 16, and only with the cluster Hamiltonian
    fake = ctypes.c_void_p(0x1000)
    for bad in (nqs.model_desc(1, 30, 1, 8, phase=True), nqs.model_desc(1, 30, 1, 32, phase=True, precision=1)):
        assert L.nqs_logpsi(ctypes.byref(bad), fake, fake, 4, fake, None, fake, 1 << 30, None) == 7
    assert L.nqs_local_energy(ctypes.byref(desc), fake, ctypes.byref(nqs.tfim()), fake, fake, 4, fake, fake,
                              1 << 30, None) == 7
    assert nqs.ModelDesc(1, 30, 1, d, 0, 0, 0, 2).phase == 2
    assert L.nqs_param_count(ctypes.byref(nqs.ModelDesc(1, 30, 1, d, 0, 0, 0, 2))) == 0


def test_bad_descriptors_are_rejected(L):
    bad = [nqs.model_desc(3, 10, 1, 8), nqs.model_desc(1, 10, 2, 8), nqs.model_desc(1, 10, 1, 12),
           nqs.model_desc(1, 0, 1, 8), nqs.model_desc(2, 3, 3, 8, sz0=True),
           nqs.model_desc(1, 10, 1, 8, precision=7), nqs.model_desc(2, 4, 4, 16, d_model=8)]
    for desc in bad:
        assert L.nqs_param_count(ctypes.byref(desc)) == 0
        assert L.nqs_workspace_bytes(ctypes.byref(desc), None, 16, nqs.OP_SAMPLE) == 0
    assert L.nqs_param_count(None) == 0


def test_host_checks_return_status_without_launching(L):
    desc = nqs.model_desc(1, 12, 1, 8)
    fake = ctypes.c_void_p(0x1000)
    ws_unaligned = ctypes.c_void_p(0x1010)
    # null params
    assert L.nqs_sample(ctypes.byref(desc), None, 4, 0, 0, None, 0, None, fake, fake, None, fake, 1 << 20, None) == 1
    # the global sample index must fit the 32-bit Philox counter word
    assert L.nqs_sample(ctypes.byref(desc), fake, 4, 0, 0, None, (1 << 32) - 3, None, fake, fake, None, fake,
                        1 << 20, None) == 1
    # training and evaluation calls: bad arguments are rejected on the host
    adam, sched = nqs.adam_desc(), nqs.lr_constant(1e-3)
    assert L.nqs_adam_step(fake, fake, fake, fake, fake, 10, ctypes.byref(adam), ctypes.byref(sched), 0, None,
                           None) == 1                      # both gradient pointers
    assert L.nqs_adam_step(None, None, fake, fake, fake, 10, ctypes.byref(adam), ctypes.byref(sched), 0, None,
                           None) == 1                      # no gradient
    bad_sched = nqs.lr_inverse(1e-3, 0.0)
    assert L.nqs_adam_step(fake, None, fake, fake, fake, 10, ctypes.byref(adam), ctypes.byref(bad_sched), 0, None,
                           None) == 1
    bad_adam = nqs.adam_desc(beta1=1.0)
    assert L.nqs_adam_step(fake, None, fake, fake, fake, 10, ctypes.byref(bad_adam), ctypes.byref(sched), 0, None,
                           None) == 1
    assert L.nqs_record_stats(fake, fake, 0, fake, None) == 1
    ham = nqs.tfim()
    assert L.nqs_evaluate_workspace_bytes(ctypes.byref(desc), ctypes.byref(ham), 0) == 0
    assert L.nqs_evaluate_workspace_bytes(ctypes.byref(desc), ctypes.byref(ham), 1000) > 1000 * 12 * 8 * 4
    assert L.nqs_evaluate(ctypes.byref(desc), fake, ctypes.byref(ham), 0, 10, 0, 0, fake, fake, 1 << 30,
                          None) == 1                       # no samples
    assert L.nqs_evaluate(ctypes.byref(desc), fake, ctypes.byref(ham), 100, 10, 0, 0, fake, fake, 16,
                          None) == 3                       # workspace too small
    # data-parallel calls: null pointers are rejected before any launch
    assert L.nqs_energy_sums(None, 4, fake, None) == 1
    assert L.nqs_energy_sums(fake, 4, None, None) == 1
    assert L.nqs_vmc_grad_global(ctypes.byref(desc), fake, fake, fake, fake, 4, None, fake, fake, fake,
                                 1 << 20, None) == 1
    # null descriptor
    assert L.nqs_logpsi(None, fake, fake, 4, fake, None, fake, 1 << 20, None) == 1
    # workspace too small / misaligned / missing
    assert L.nqs_logpsi(ctypes.byref(desc), fake, fake, 4, fake, None, fake, 16, None) == 3
    assert L.nqs_logpsi(ctypes.byref(desc), fake, fake, 4, fake, None, ws_unaligned, 1 << 20, None) == 3
    assert L.nqs_logpsi(ctypes.byref(desc), fake, fake, 4, fake, None, None, 1 << 20, None) == 3
    # negative batch
    assert L.nqs_logpsi(ctypes.byref(desc), fake, fake, -1, fake, None, fake, 1 << 20, None) == 1
    # local energy needs a Hamiltonian and the prefix cache
    assert L.nqs_local_energy(ctypes.byref(desc), fake, None, fake, fake, 4, fake, fake, 1 << 20, None) == 1
    ham = nqs.tfim()
    assert L.nqs_local_energy(ctypes.byref(desc), fake, ctypes.byref(ham), fake, None, 4, fake, fake,
                              1 << 20, None) == 1
    # an empty batch needs no data pointers
    assert L.nqs_local_energy(ctypes.byref(desc), fake, ctypes.byref(ham), None, None, 0, None, fake,
                              1 << 20, None) == 0
    bad_ham = nqs.HamDesc(9, 0, 1.0, 1.0)
    assert L.nqs_local_energy(ctypes.byref(desc), fake, ctypes.byref(bad_ham), fake, fake, 4, fake, fake,
                              1 << 20, None) == 1
    # vmc_grad needs at least one sample
    st = ctypes.c_void_p(0x2000)
    assert L.nqs_vmc_grad(ctypes.byref(desc), fake, fake, fake, fake, 0, fake, st, fake, 1 << 20, None) == 1
    # growth may not shrink or change the lattice
    big = nqs.model_desc(1, 12, 1, 16)
    other = nqs.model_desc(1, 10, 1, 16)
    assert L.nqs_grow_hidden(ctypes.byref(big), fake, ctypes.byref(desc), fake, 2, 1e-3, None) == 2
    assert L.nqs_grow_hidden(ctypes.byref(desc), fake, ctypes.byref(other), fake, 2, 1e-3, None) == 2
    assert L.nqs_grow_hidden(ctypes.byref(desc), fake, ctypes.byref(big), fake, 2, -1.0, None) == 1
    for code in range(8):
        assert L.nqs_status_string(code).startswith(b"NQS_")


def test_workspace_grows_with_batch(L):
    desc = nqs.model_desc(1, 100, 1, 64)
    ham = nqs.tfim()
    a = L.nqs_workspace_bytes(ctypes.byref(desc), ctypes.byref(ham), 100, nqs.OP_LOCAL_ENERGY)
    b = L.nqs_workspace_bytes(ctypes.byref(desc), ctypes.byref(ham), 4096, nqs.OP_LOCAL_ENERGY)
    assert 0 < a < b and a % 256 == 0 and b % 256 == 0
    assert L.nqs_workspace_bytes(ctypes.byref(desc), None, 100, nqs.OP_LOCAL_ENERGY) == 0


def test_static_scratch_call_rejects_bad_descriptors_like_the_workspace_call(L):
    """nqs_local_energy_static returns the status nqs_local_energy returns for
    an invalid descriptor (both check on the host before any launch)."""
    fake = ctypes.c_void_p(0x1000)
    ham = nqs.tfim()
    f = L.nqs_local_energy_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(nqs.ModelDesc), ctypes.c_void_p, ctypes.POINTER(nqs.HamDesc), ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    bad = [nqs.model_desc(1, 12, 1, 8, precision=5), nqs.ModelDesc(1, 12, 1, 8, 0, 2, 0),
           nqs.model_desc(1, 12, 2, 8), nqs.model_desc(1, (1 << 20) + 1, 1, 8), nqs.model_desc(7, 12, 1, 8),
           nqs.model_desc(1, 12, 1, 12), nqs.model_desc(1, 0, 1, 8)]
    for desc in bad:
        want = L.nqs_local_energy(ctypes.byref(desc), fake, ctypes.byref(ham), fake, fake, 4, fake, fake,
                                  1 << 20, None)
        assert want in (1, 2)
        assert f(ctypes.byref(desc), fake, ctypes.byref(ham), fake, fake, 4, fake, None) == want, desc.precision
    # valid descriptors off the call's single path
    assert f(ctypes.byref(nqs.model_desc(1, 12, 1, 8, precision=nqs.BF16)), fake, ctypes.byref(ham), fake, fake,
             4, fake, None) == 7
    assert f(ctypes.byref(nqs.model_desc(2, 4, 4, 8)), fake, ctypes.byref(ham), fake, fake, 4, fake, None) == 7


def test_sweep_segment_bounds_the_wide_gradient_workspace(L):
    """Passes of k positions in the d_h = 256 2D BF16 reverse sweep keep tapes
    for B k cells instead of B N: the gradient workspace at 16 x 16, B = 8192
    shrinks with k, and 0 restores the one-pass size."""
    desc = nqs.model_desc(nqs.GRU2D, 16, 16, 256, sz0=True, precision=nqs.BF16)
    size = lambda: L.nqs_workspace_bytes(ctypes.byref(desc), None, 8192, nqs.OP_LOGPSI_GRAD)
    try:
        one = size()
        L.nqs_set_sweep_segment(16)
        k16 = size()
        L.nqs_set_sweep_segment(64)
        k64 = size()
    finally:
        L.nqs_set_sweep_segment(0)
    assert size() == one
    # tapes ~7.2 KB per (sample, position): B N of them in one pass
    assert one > 8192 * 256 * 7000
    assert k16 < k64 < one
    assert k16 < one / 10
