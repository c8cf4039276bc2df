"""The model the BF16 tensor-core 2D path evaluates exactly (up to FP32
accumulation and the 16-bit hi + lo states): the float64 oracle on weights
rounded to BF16 where the GEMMs read BF16 weights (W and W_g on the states, U_mix,
W_1, W_2); the input-spin columns and the biases enter as hi + lo pairs and
the readout U_out, c in FP32, so they stay as they are.

Where the lattice map expands (hidden states growing over the lattice), the
exact model and the BF16-weight model drift apart by the weight rounding
amplified along the zig-zag path; comparing against the BF16-weight model
checks the kernels at a tolerance that does not depend on that amplification.
"""
import numpy as np

from oracle import model as om


def bf16_round(x):
    """Round float32 values to the nearest BF16 (ties to even), as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_weight_model(mod, flat):
    """Flat parameters of the 2D GRU + GLU with the GEMM weights rounded to BF16."""
    t = {k: v.copy() for k, v in mod.unpack(flat).items()}
    d = mod.d
    for k in ("W", "W_g"):
        t[k][:, :2 * d] = bf16_round(t[k][:, :2 * d])
    for k in ("U_mix", "W_1", "W_2"):
        t[k] = bf16_round(t[k])
    return mod.pack(t)


def draw_window(mod, pf, s):
    """Per draw (sampling order): the gap between the exact and the
    BF16-weight models' p0 along the path, plus 1e-4 for the kernels' own
    error against the BF16-weight model."""
    gap = np.abs(om.run(mod, pf, sigma=s)["p0"] - om.run(mod, bf16_weight_model(mod, pf), sigma=s)["p0"])
    order = np.array([mod.lattice_index(i, j) for (i, j) in mod.order()])
    return gap[:, order] + 1e-4
