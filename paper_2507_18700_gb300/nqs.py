"""Python binding of libnqs (include/nqs.h): argument marshalling only.

Every function takes torch CUDA tensors, passes their device pointers, sizes
and the current CUDA stream to the C ABI, and raises ``NqsError`` on a non-OK
status.  All arithmetic runs in the library's kernels; there is no CPU or
PyTorch fallback, and importing this module without a built ``libnqs.so``
raises.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnqs.so")

GRU1D, GRU2D = 1, 2
FP32, BF16 = 0, 1
TFIM, HEISENBERG, LRTFIM, CLUSTER = 1, 2, 3, 4
OP_SAMPLE, OP_LOGPSI, OP_LOCAL_ENERGY, OP_LOGPSI_GRAD, OP_VMC_GRAD = 1, 2, 3, 4, 5

STATUS = {0: "NQS_OK", 1: "NQS_EINVAL", 2: "NQS_ESHAPE", 3: "NQS_EWORKSPACE", 4: "NQS_ECUDA",
          5: "NQS_ETIMEOUT", 6: "NQS_ENONFINITE", 7: "NQS_EUNSUPPORTED"}

EXPORTS = ["nqs_param_count", "nqs_workspace_bytes", "nqs_grow_hidden", "nqs_sample", "nqs_logpsi",
           "nqs_local_energy", "nqs_local_energy_static", "nqs_logpsi_grad", "nqs_vmc_grad", "nqs_workspace_status",
           "nqs_status_string", "nqs_vmc_step_batched_workspace_bytes", "nqs_vmc_step_batched",
           "nqs_set_autotune", "nqs_set_tile_variant", "nqs_set_sweep_segment", "nqs_energy_sums", "nqs_vmc_grad_global", "nqs_set_wait_limit", "nqs_adam_step",
           "nqs_record_stats", "nqs_evaluate_workspace_bytes", "nqs_evaluate", "nqs_ckpt_floats",
           "nqs_ckpt_workspace_bytes", "nqs_logpsi_ckpt", "nqs_logpsi_grad_ckpt"]


class NqsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s" % (where, STATUS.get(code, code)))


class ModelDesc(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_int32), ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
                ("d_h", ctypes.c_int32), ("d_model", ctypes.c_int32), ("sz0", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("phase", ctypes.c_int32)]

    @property
    def N(self):
        return self.Lx * self.Ly


class HamDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("marshall", ctypes.c_int32), ("J", ctypes.c_double),
                ("h", ctypes.c_double), ("alpha", ctypes.c_double)]


class LrSchedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("lr0", ctypes.c_double),
                ("lr1", ctypes.c_double), ("t_switch", ctypes.c_int64), ("decay", ctypes.c_double)]


class AdamDesc(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double)]


LR_CONSTANT, LR_STEP, LR_INVERSE = 1, 2, 3


def lr_constant(lr):
    return LrSchedule(LR_CONSTANT, 0, lr, 0.0, 0, 1.0)


def lr_step(lr0, lr1, t_switch):
    return LrSchedule(LR_STEP, 0, lr0, lr1, int(t_switch), 1.0)


def lr_inverse(lr0, decay, t_switch=0):
    return LrSchedule(LR_INVERSE, 0, lr0, 0.0, int(t_switch), float(decay))


def adam_desc(beta1=0.9, beta2=0.999, eps=1e-8):
    return AdamDesc(beta1, beta2, eps)


class Replica(ctypes.Structure):
    _fields_ = [("desc", ModelDesc), ("ham", HamDesc), ("B", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("params", ctypes.c_void_p), ("sigma", ctypes.c_void_p), ("logpsi", ctypes.c_void_p),
                ("hcache", ctypes.c_void_p), ("eloc", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("stats", ctypes.c_void_p)]


MAX_REPLICAS = 16


def model_desc(cell, Lx, Ly=1, d_h=8, d_model=0, sz0=False, precision=FP32, phase=False):
    return ModelDesc(cell, Lx, Ly, d_h, d_model, int(bool(sz0)), precision, int(bool(phase)))


def tfim(J=1.0, Gamma=1.0):
    return HamDesc(TFIM, 0, J, Gamma, 0.0)


def lr_tfim(alpha, J=1.0, Gamma=1.0):
    """Long-range TFIM of Sec. III C: -J sum_{i<j} Z_i Z_j / |i-j|^alpha - Gamma sum X_i."""
    return HamDesc(LRTFIM, 0, J, Gamma, alpha)


def cluster(J=1.0):
    """Cluster-state Hamiltonian of Sec. III D (stabiliser reading; ground energy -J N)."""
    return HamDesc(CLUSTER, 0, J, 0.0, 0.0)


def heisenberg(J=1.0, marshall=True):
    return HamDesc(HEISENBERG, int(bool(marshall)), J, 0.0, 0.0)


_lib = None


def lib():
    """Load the in-tree libnqs.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libnqs.so is not built (run __graft_entry__.build()); there is no fallback")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i64, u64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    L.nqs_param_count.restype = sz
    L.nqs_param_count.argtypes = [P(ModelDesc)]
    L.nqs_workspace_bytes.restype = sz
    L.nqs_workspace_bytes.argtypes = [P(ModelDesc), P(HamDesc), i64, ctypes.c_int]
    L.nqs_grow_hidden.restype = ctypes.c_int
    L.nqs_grow_hidden.argtypes = [P(ModelDesc), vp, P(ModelDesc), vp, u64, ctypes.c_float, vp]
    L.nqs_sample.restype = ctypes.c_int
    L.nqs_sample.argtypes = [P(ModelDesc), vp, i64, u64, u64, vp, u64, vp, vp, vp, vp, vp, sz, vp]
    L.nqs_ckpt_floats.restype = sz
    L.nqs_ckpt_floats.argtypes = [P(ModelDesc), i64, ctypes.c_int32]
    L.nqs_ckpt_workspace_bytes.restype = sz
    L.nqs_ckpt_workspace_bytes.argtypes = [P(ModelDesc), i64, ctypes.c_int32]
    L.nqs_logpsi_ckpt.restype = ctypes.c_int
    L.nqs_logpsi_ckpt.argtypes = [P(ModelDesc), vp, vp, i64, ctypes.c_int32, vp, vp, vp, sz, vp]
    L.nqs_logpsi_grad_ckpt.restype = ctypes.c_int
    L.nqs_logpsi_grad_ckpt.argtypes = [P(ModelDesc), vp, vp, i64, ctypes.c_int32, vp, vp, vp, vp, sz, vp]
    L.nqs_adam_step.restype = ctypes.c_int
    L.nqs_adam_step.argtypes = [vp, vp, vp, vp, vp, i64, P(AdamDesc), P(LrSchedule), u64, vp, vp]
    L.nqs_record_stats.restype = ctypes.c_int
    L.nqs_record_stats.argtypes = [vp, vp, i64, vp, vp]
    L.nqs_evaluate_workspace_bytes.restype = sz
    L.nqs_evaluate_workspace_bytes.argtypes = [P(ModelDesc), P(HamDesc), i64]
    L.nqs_evaluate.restype = ctypes.c_int
    L.nqs_evaluate.argtypes = [P(ModelDesc), vp, P(HamDesc), i64, i64, u64, u64, vp, vp, sz, vp]
    L.nqs_logpsi.restype = ctypes.c_int
    L.nqs_logpsi.argtypes = [P(ModelDesc), vp, vp, i64, vp, vp, vp, sz, vp]
    L.nqs_local_energy.restype = ctypes.c_int
    L.nqs_local_energy.argtypes = [P(ModelDesc), vp, P(HamDesc), vp, vp, i64, vp, vp, sz, vp]
    L.nqs_logpsi_grad.restype = ctypes.c_int
    L.nqs_logpsi_grad.argtypes = [P(ModelDesc), vp, vp, vp, vp, i64, vp, vp, sz, vp]
    L.nqs_vmc_grad.restype = ctypes.c_int
    L.nqs_vmc_grad.argtypes = [P(ModelDesc), vp, vp, vp, vp, i64, vp, vp, vp, sz, vp]
    L.nqs_energy_sums.restype = ctypes.c_int
    L.nqs_energy_sums.argtypes = [vp, i64, vp, vp]
    L.nqs_vmc_grad_global.restype = ctypes.c_int
    L.nqs_vmc_grad_global.argtypes = [P(ModelDesc), vp, vp, vp, vp, i64, vp, vp, vp, vp, sz, vp]
    L.nqs_set_wait_limit.restype = ctypes.c_int
    L.nqs_set_wait_limit.argtypes = [i64]
    L.nqs_workspace_status.restype = ctypes.c_int
    L.nqs_workspace_status.argtypes = [vp, P(ctypes.c_int32), vp]
    L.nqs_vmc_step_batched_workspace_bytes.restype = sz
    L.nqs_vmc_step_batched_workspace_bytes.argtypes = [ctypes.c_int, P(Replica)]
    L.nqs_vmc_step_batched.restype = ctypes.c_int
    L.nqs_vmc_step_batched.argtypes = [ctypes.c_int, P(Replica), u64, vp, vp, sz, vp]
    L.nqs_set_autotune.restype = None
    L.nqs_set_autotune.argtypes = [ctypes.c_int]
    L.nqs_set_tile_variant.restype = None
    L.nqs_set_tile_variant.argtypes = [ctypes.c_int]
    L.nqs_set_sweep_segment.restype = None
    L.nqs_set_sweep_segment.argtypes = [ctypes.c_int32]
    L.nqs_status_string.restype = ctypes.c_char_p
    L.nqs_status_string.argtypes = [ctypes.c_int]
    _lib = L
    return L


def _check(code, where):
    if code != 0:
        raise NqsError(code, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _per_sample(desc, B):
    """Shape of a per-sample log psi / local energy / weight: [B] or, for a
    cRNN, [B, 2] (real and imaginary parts)."""
    return (B, 2) if desc.phase else (B,)


def _need(t, dtype, shape, name):
    if t is None:
        raise ValueError("%s is required" % name)
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError("%s must be a contiguous CUDA %s tensor of shape %s, got %s %s %s"
                         % (name, dtype, tuple(shape), t.device, t.dtype, tuple(t.shape)))


def set_autotune(on):
    """Turn the tile-shape autotuner of the tensor-core kernels on or off."""
    lib().nqs_set_autotune(1 if on else 0)


def set_wait_limit(polls):
    """Bound of the tensor-core waits that may give up (None: the default);
    0 makes every such wait give up at once (testing NQS_ETIMEOUT)."""
    _check(lib().nqs_set_wait_limit(-1 if polls is None else int(polls)), "nqs_set_wait_limit")


def set_sweep_segment(positions):
    """Positions per pass of the d_h = 256 2D BF16 reverse sweep (None or 0:
    one pass); workspace sizes follow the setting."""
    lib().nqs_set_sweep_segment(0 if positions is None else int(positions))


def set_tile_variant(variant):
    """Pin the tile variant of the tensor-core kernels (None or < 0: normal selection)."""
    lib().nqs_set_tile_variant(-1 if variant is None else int(variant))


def param_count(desc):
    n = lib().nqs_param_count(ctypes.byref(desc))
    if n == 0:
        raise NqsError(1, "nqs_param_count")
    return n


def workspace_bytes(desc, B, op, ham=None):
    n = lib().nqs_workspace_bytes(ctypes.byref(desc), ctypes.byref(ham) if ham is not None else None,
                                  int(B), op)
    if n == 0:
        raise NqsError(1, "nqs_workspace_bytes")
    return n


class Workspace:
    """Caller-owned workspace buffer that grows on demand (256-byte aligned)."""

    def __init__(self, device=None):
        self.device = device
        self.buf = None

    def get(self, nbytes):
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256) + 256, dtype=torch.uint8, device=self.device)
        off = (-self.buf.data_ptr()) % 256
        return ctypes.c_void_p(self.buf.data_ptr() + off), self.buf.numel() - off

    def status(self):
        if self.buf is None:
            return 0
        ptr, _ = self.get(256)
        v = ctypes.c_int32(0)
        _check(lib().nqs_workspace_status(ptr, ctypes.byref(v), _stream()), "nqs_workspace_status")
        return v.value


_default_ws = {}


def _ws(ws, device):
    if ws is not None:
        return ws
    key = str(device)
    if key not in _default_ws:
        _default_ws[key] = Workspace(device)
    return _default_ws[key]


def sample(desc, params, B, seed=0, step=0, uniforms=None, hcache=True, ws=None, sample_offset=0,
           step_dev=None, out=None):
    """Autoregressive sampling: returns (sigma uint8 [B,N], logpsi [B], hcache [B,N,d_h] or None).
    sample_offset is the global index of the first sample (the Philox counter);
    step_dev (a CUDA uint64/int64 tensor of one element) replaces `step` by a
    device counter; out = (sigma, logpsi) reuses output buffers."""
    dev = params.device
    N, d = desc.N, desc.d_h
    _need(params, torch.float32, (param_count(desc),), "params")
    if uniforms is not None:
        _need(uniforms, torch.float32, (B, N), "uniforms")
    if out is None:
        sigma = torch.empty((B, N), dtype=torch.uint8, device=dev)
        logpsi = torch.empty(_per_sample(desc, B), dtype=torch.float32, device=dev)
    else:
        sigma, logpsi = out
        _need(sigma, torch.uint8, (B, N), "sigma")
        _need(logpsi, torch.float32, _per_sample(desc, B), "logpsi")
    hc = torch.empty((B, N, d), dtype=torch.float32, device=dev) if hcache is True else hcache
    if hc is not None and hcache is not True:
        _need(hc, torch.float32, (B, N, d), "hcache")
    w = _ws(ws, dev)
    wp, wn = w.get(workspace_bytes(desc, B, OP_SAMPLE))
    _check(lib().nqs_sample(ctypes.byref(desc), _ptr(params), int(B), int(seed), int(step), _ptr(step_dev),
                            int(sample_offset), _ptr(uniforms), _ptr(sigma), _ptr(logpsi), _ptr(hc), wp, wn, _stream()),
           "nqs_sample")
    return sigma, logpsi, hc


def logpsi(desc, params, sigma, hcache=True, ws=None):
    """Teacher-forced log psi: returns (logpsi [B], hcache or None)."""
    dev = params.device
    B, N = sigma.shape
    _need(params, torch.float32, (param_count(desc),), "params")
    _need(sigma, torch.uint8, (B, desc.N), "sigma")
    out = torch.empty(_per_sample(desc, B), dtype=torch.float32, device=dev)
    hc = torch.empty((B, N, desc.d_h), dtype=torch.float32, device=dev) if hcache is True else hcache
    w = _ws(ws, dev)
    wp, wn = w.get(workspace_bytes(desc, B, OP_LOGPSI))
    _check(lib().nqs_logpsi(ctypes.byref(desc), _ptr(params), _ptr(sigma), int(B), _ptr(out), _ptr(hc),
                            wp, wn, _stream()), "nqs_logpsi")
    return out, hc


def local_energy(desc, params, ham, sigma, hcache, ws=None, out=None):
    dev = params.device
    B = sigma.shape[0]
    _need(params, torch.float32, (param_count(desc),), "params")
    _need(sigma, torch.uint8, (B, desc.N), "sigma")
    _need(hcache, torch.float32, (B, desc.N, desc.d_h), "hcache")
    eloc = torch.empty(_per_sample(desc, B) if ham.kind == CLUSTER else (B,), dtype=torch.float32,
                       device=dev) if out is None else out
    w = _ws(ws, dev)
    wp, wn = w.get(workspace_bytes(desc, B, OP_LOCAL_ENERGY, ham))
    _check(lib().nqs_local_energy(ctypes.byref(desc), _ptr(params), ctypes.byref(ham), _ptr(sigma),
                                  _ptr(hcache), int(B), _ptr(eloc), wp, wn, _stream()),
           "nqs_local_energy")
    return eloc


def logpsi_grad(desc, params, sigma, hcache, weights, ws=None, out=None):
    dev = params.device
    B = sigma.shape[0]
    P = param_count(desc)
    _need(params, torch.float32, (P,), "params")
    _need(sigma, torch.uint8, (B, desc.N), "sigma")
    _need(hcache, torch.float32, (B, desc.N, desc.d_h), "hcache")
    _need(weights, torch.float32, _per_sample(desc, B), "weights")
    grad = torch.empty((P,), dtype=torch.float32, device=dev) if out is None else out
    w = _ws(ws, dev)
    wp, wn = w.get(workspace_bytes(desc, B, OP_LOGPSI_GRAD))
    _check(lib().nqs_logpsi_grad(ctypes.byref(desc), _ptr(params), _ptr(sigma), _ptr(hcache),
                                 _ptr(weights), int(B), _ptr(grad), wp, wn, _stream()),
           "nqs_logpsi_grad")
    return grad


def vmc_grad(desc, params, sigma, hcache, eloc, ws=None, grad=None, stats=None):
    """Returns (grad [P] float32, stats [3] float64 = mean E_loc, variance, M)."""
    dev = params.device
    B = sigma.shape[0]
    P = param_count(desc)
    _need(params, torch.float32, (P,), "params")
    _need(sigma, torch.uint8, (B, desc.N), "sigma")
    _need(hcache, torch.float32, (B, desc.N, desc.d_h), "hcache")
    _need(eloc, torch.float32, _per_sample(desc, B), "eloc")
    g = torch.empty((P,), dtype=torch.float32, device=dev) if grad is None else grad
    st = torch.empty((4 if desc.phase else 3,), dtype=torch.float64, device=dev) if stats is None else stats
    w = _ws(ws, dev)
    wp, wn = w.get(workspace_bytes(desc, B, OP_VMC_GRAD))
    _check(lib().nqs_vmc_grad(ctypes.byref(desc), _ptr(params), _ptr(sigma), _ptr(hcache), _ptr(eloc),
                              int(B), _ptr(g), _ptr(st), wp, wn, _stream()), "nqs_vmc_grad")
    return g, st


def energy_sums(eloc, out=None):
    """This rank's [sum E_loc, sum E_loc^2, B] (float64 [3]) for the data-parallel step."""
    _need(eloc, torch.float32, (eloc.shape[0],), "eloc")
    s = torch.empty((3,), dtype=torch.float64, device=eloc.device) if out is None else out
    _check(lib().nqs_energy_sums(_ptr(eloc), int(eloc.shape[0]), _ptr(s), _stream()), "nqs_energy_sums")
    return s


def vmc_grad_global(desc, params, sigma, hcache, eloc, sums, ws=None, grad=None, stats=None):
    """This rank's share of the VMC gradient (float64 [P]) with weights centred
    by the global sums of all ranks; returns (grad, stats [3] = global mean,
    variance, M)."""
    dev = params.device
    B = sigma.shape[0]
    P = param_count(desc)
    _need(params, torch.float32, (P,), "params")
    _need(sigma, torch.uint8, (B, desc.N), "sigma")
    _need(hcache, torch.float32, (B, desc.N, desc.d_h), "hcache")
    _need(eloc, torch.float32, (B,), "eloc")
    _need(sums, torch.float64, (3,), "sums")
    g = torch.empty((P,), dtype=torch.float64, device=dev) if grad is None else grad
    st = torch.empty((3,), dtype=torch.float64, device=dev) if stats is None else stats
    w = _ws(ws, dev)
    wp, wn = w.get(workspace_bytes(desc, B, OP_VMC_GRAD))
    _check(lib().nqs_vmc_grad_global(ctypes.byref(desc), _ptr(params), _ptr(sigma), _ptr(hcache), _ptr(eloc),
                                     int(B), _ptr(sums), _ptr(g), _ptr(st), wp, wn, _stream()),
           "nqs_vmc_grad_global")
    return g, st


def adam_step(params, m, v, grad, adam, sched, t=0, t_dev=None):
    """One Adam update in place (grad float32 or float64); t_dev advances."""
    P = params.numel()
    _need(params, torch.float32, (P,), "params")
    _need(m, torch.float32, (P,), "m")
    _need(v, torch.float32, (P,), "v")
    g32 = grad if grad.dtype == torch.float32 else None
    g64 = grad if grad.dtype == torch.float64 else None
    _need(grad, grad.dtype if grad.dtype in (torch.float32, torch.float64) else torch.float32, (P,), "grad")
    _check(lib().nqs_adam_step(_ptr(g32), _ptr(g64), _ptr(params), _ptr(m), _ptr(v), int(P), ctypes.byref(adam),
                               ctypes.byref(sched), int(t), _ptr(t_dev), _stream()), "nqs_adam_step")


def record_stats(stats, log, t_dev):
    _check(lib().nqs_record_stats(_ptr(stats), _ptr(log), int(log.shape[0]), _ptr(t_dev), _stream()),
           "nqs_record_stats")


def evaluate(desc, params, ham, M, chunk=65536, seed=0, step=0, ws=None):
    """Final evaluation: float64 [5] = mean E_loc, variance, M, error of the mean, error of the variance."""
    dev = params.device
    _need(params, torch.float32, (param_count(desc),), "params")
    n = lib().nqs_evaluate_workspace_bytes(ctypes.byref(desc), ctypes.byref(ham), int(min(chunk, M)))
    if n == 0:
        raise NqsError(1, "nqs_evaluate_workspace_bytes")
    st = torch.empty((5,), dtype=torch.float64, device=dev)
    w = _ws(ws, dev)
    wp, wn = w.get(n)
    _check(lib().nqs_evaluate(ctypes.byref(desc), _ptr(params), ctypes.byref(ham), int(M), int(chunk), int(seed),
                              int(step), _ptr(st), wp, wn, _stream()), "nqs_evaluate")
    return st


def grow_hidden(small, p_small, big, seed=2, eps=1e-3):
    _need(p_small, torch.float32, (param_count(small),), "p_small")
    p_big = torch.empty((param_count(big),), dtype=torch.float32, device=p_small.device)
    _check(lib().nqs_grow_hidden(ctypes.byref(small), _ptr(p_small), ctypes.byref(big), _ptr(p_big),
                                 int(seed), float(eps), _stream()), "nqs_grow_hidden")
    return p_big


def logpsi_ckpt(desc, params, sigma, k, ws=None):
    """Teacher-forced log psi keeping every k-th state: (logpsi [B], ckpt)."""
    B = sigma.shape[0]
    _need(params, torch.float32, (param_count(desc),), "params")
    _need(sigma, torch.uint8, (B, desc.N), "sigma")
    n = lib().nqs_ckpt_floats(ctypes.byref(desc), int(B), int(k))
    out = torch.empty((B,), dtype=torch.float32, device=params.device)
    ck = torch.empty((max(n, 1),), dtype=torch.float32, device=params.device)
    w = _ws(ws, params.device)
    wp, wn = w.get(lib().nqs_ckpt_workspace_bytes(ctypes.byref(desc), int(B), int(k)))
    _check(lib().nqs_logpsi_ckpt(ctypes.byref(desc), _ptr(params), _ptr(sigma), int(B), int(k), _ptr(out),
                                 _ptr(ck), wp, wn, _stream()), "nqs_logpsi_ckpt")
    return out, ck[:n]


def logpsi_grad_ckpt(desc, params, sigma, k, ckpt, weights, ws=None):
    """Gradient of sum_b w_b log psi_b from the checkpoints of logpsi_ckpt."""
    B = sigma.shape[0]
    P = param_count(desc)
    _need(params, torch.float32, (P,), "params")
    _need(weights, torch.float32, (B,), "weights")
    grad = torch.empty((P,), dtype=torch.float32, device=params.device)
    w = _ws(ws, params.device)
    wp, wn = w.get(lib().nqs_ckpt_workspace_bytes(ctypes.byref(desc), int(B), int(k)))
    _check(lib().nqs_logpsi_grad_ckpt(ctypes.byref(desc), _ptr(params), _ptr(sigma), int(B), int(k),
                                      _ptr(ckpt) if ckpt.numel() else None, _ptr(weights), _ptr(grad), wp, wn,
                                      _stream()), "nqs_logpsi_grad_ckpt")
    return grad


class LogPsi(torch.autograd.Function):
    """log psi(sigma) with the library's reverse sweep as its backward.

    forward(params, sigma, desc, checkpoint=None) -> logpsi [B] ([B, 2] for a
    cRNN); backward gives d params of sum_b grad_out_b * logpsi_b (sigma is not
    differentiable).  With checkpoint = k the forward keeps every k-th hidden
    state only (FP32 1D GRU) and the backward recomputes the segments.
    """

    @staticmethod
    def forward(ctx, params, sigma, desc, checkpoint=None):
        ctx.desc, ctx.k = desc, checkpoint
        if checkpoint:
            lp, ck = logpsi_ckpt(desc, params.detach(), sigma, int(checkpoint))
            ctx.save_for_backward(params, sigma, ck)
            return lp
        lp, hc = logpsi(desc, params.detach(), sigma, hcache=True)
        ctx.save_for_backward(params, sigma, hc)
        return lp

    @staticmethod
    def backward(ctx, grad_out):
        params, sigma, saved = ctx.saved_tensors
        if ctx.k:
            g = logpsi_grad_ckpt(ctx.desc, params.detach(), sigma, int(ctx.k), saved, grad_out.contiguous().float())
        else:
            g = logpsi_grad(ctx.desc, params.detach(), sigma, saved, grad_out.contiguous().float())
        return g, None, None, None


class ReplicaBatch:
    """Device buffers of a batch of 1D replicas and their batched VMC step.

    models: list of (desc, ham, B, seed, params) with params a CUDA float32
    tensor.  step(step_no) runs nqs_vmc_step_batched; with device_step=True the
    step number lives in a device counter that every call advances (usable
    inside a captured CUDA graph).
    """

    def __init__(self, models, device=None, device_step=False):
        if not 1 <= len(models) <= MAX_REPLICAS:
            raise ValueError("1 to %d replicas" % MAX_REPLICAS)
        self.models = models
        dev = models[0][4].device if device is None else device
        self.out = []
        reps = (Replica * len(models))()
        for i, (desc, ham, B, seed, params) in enumerate(models):
            P = param_count(desc)
            _need(params, torch.float32, (P,), "params")
            o = dict(sigma=torch.empty((B, desc.N), dtype=torch.uint8, device=dev),
                     logpsi=torch.empty((B,), dtype=torch.float32, device=dev),
                     hcache=torch.empty((B, desc.N, desc.d_h), dtype=torch.float32, device=dev),
                     eloc=torch.empty((B,), dtype=torch.float32, device=dev),
                     grad=torch.empty((P,), dtype=torch.float32, device=dev),
                     stats=torch.empty((3,), dtype=torch.float64, device=dev), params=params)
            self.out.append(o)
            reps[i] = Replica(desc, ham, B, seed, params.data_ptr(), o["sigma"].data_ptr(),
                              o["logpsi"].data_ptr(), o["hcache"].data_ptr(), o["eloc"].data_ptr(),
                              o["grad"].data_ptr(), o["stats"].data_ptr())
        self.reps = reps
        n = lib().nqs_vmc_step_batched_workspace_bytes(len(models), reps)
        if n == 0:
            raise NqsError(1, "nqs_vmc_step_batched_workspace_bytes")
        self.ws = Workspace(dev)
        self.ws_ptr, self.ws_n = self.ws.get(n)
        self.step_dev = torch.zeros((1,), dtype=torch.int64, device=dev) if device_step else None

    def step(self, step_no=0):
        _check(lib().nqs_vmc_step_batched(len(self.models), self.reps, int(step_no), _ptr(self.step_dev),
                                          self.ws_ptr, self.ws_n, _stream()), "nqs_vmc_step_batched")
        return self.out
