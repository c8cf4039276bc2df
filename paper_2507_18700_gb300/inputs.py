"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: it only draws parameter vectors
(Xavier-uniform per matrix, optional Gaussian noise) and spin configurations
with numpy's PCG64 generator, in the flat parameter layout documented in
``include/nqs.h``.  Both the CUDA path and the float64 oracle consume what it
returns.
"""
import numpy as np

GRU1D = 1
GRU2D = 2


def tensor_shapes(cell, d_h, d_model=None, phase=False):
    """(name, shape) of every tensor of the flat layout, in order (phase: the
    cRNN's phase layer U_phi, c_phi after the amplitude head)."""
    d = d_h
    m = d_h if d_model is None else d_model
    if cell == GRU1D:
        return [("W_g", (d, d + 2)), ("W_r", (d, d + 2)), ("W_h", (d, d)),
                ("W_in", (d, 2)), ("b_g", (d,)), ("b_r", (d,)), ("b_h", (d,)),
                ("b_in", (d,)), ("U", (2, d)), ("c", (2,))] + (
                    [("U_phi", (2, d)), ("c_phi", (2,))] if phase else [])
    if cell == GRU2D:
        return [("W", (d, 2 * d + 4)), ("W_g", (d, 2 * d + 4)), ("U_mix", (d, 2 * d)),
                ("b", (d,)), ("b_g", (d,)), ("W_1", (m, d)), ("b_1", (m,)),
                ("W_2", (m, d)), ("b_2", (m,)), ("U_out", (2, m)), ("c", (2,))]
    raise ValueError("unknown cell")


def param_count(cell, d_h, d_model=None, phase=False):
    return sum(int(np.prod(s)) for _, s in tensor_shapes(cell, d_h, d_model, phase))


def xavier_params(cell, d_h, seed, noise_std=0.0, d_model=None, phase=False):
    """Xavier-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)) per matrix,
    zero biases, plus N(0, noise_std^2) on every entry when noise_std > 0.
    Returned as float64; callers cast to float32 for the device."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for _, shape in tensor_shapes(cell, d_h, d_model, phase):
        if len(shape) == 2:
            a = np.sqrt(6.0 / (shape[0] + shape[1]))
            parts.append(rng.uniform(-a, a, size=shape).reshape(-1))
        else:
            parts.append(np.zeros(shape))
    flat = np.concatenate(parts)
    if noise_std > 0:
        flat = flat + rng.normal(0.0, noise_std, size=flat.shape)
    return flat


def random_configs(B, N, seed, sz0=False):
    """B random spin configurations (uint8, lattice order); with sz0, exactly N/2 ones."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if not sz0:
        return rng.integers(0, 2, size=(B, N)).astype(np.uint8)
    base = np.zeros(N, dtype=np.uint8)
    base[: N // 2] = 1
    return np.stack([rng.permutation(base) for _ in range(B)]).astype(np.uint8)


def random_weights(B, seed, scale=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.normal(0.0, scale, size=B)
