"""Hidden-dimension growth, Fig. 2(b) and Sec. II B (test infrastructure).

The paper pads the smaller model's weights and biases with small random numbers
up to the larger size.  Reading used here:

* every old block keeps its indices: old hidden units are units 0..d-1 of the
  new model, and each hidden-input column group ([h] in 1D; [h_hor | h_ver] in
  2D) is laid out as [old units | new units];
* the one-hot input columns keep their meaning and follow the hidden columns;
* d_model grows with d_h in 2D (d_model = d_h, App. A);
* every entry that has no counterpart in the old model is eps * z, with z a
  standard normal drawn by Philox keyed by (seed, tensor index in the flat
  layout, row, column) and Box-Muller (``philox.growth_normals``).
"""
import numpy as np

from . import model as M
from .philox import growth_normals


def _index_map(cell, name, small, big):
    """For one tensor: (row map, column map) from old indices to new indices."""
    d, D = small.d, big.d
    m, Mm = small.m, big.m
    rows_h = np.arange(d)
    if cell == M.GRU1D:
        if name in ("W_g", "W_r"):
            return rows_h, np.concatenate([np.arange(d), D + np.arange(2)])
        if name == "W_h":
            return rows_h, np.arange(d)
        if name == "W_in":
            return rows_h, np.arange(2)
        if name in ("b_g", "b_r", "b_h", "b_in"):
            return rows_h, None
        if name in ("U", "U_phi"):
            return np.arange(2), np.arange(d)
        if name in ("c", "c_phi"):
            return np.arange(2), None
    else:
        hcols = np.concatenate([np.arange(d), D + np.arange(d)])
        if name in ("W", "W_g"):
            return rows_h, np.concatenate([hcols, 2 * D + np.arange(4)])
        if name == "U_mix":
            return rows_h, hcols
        if name in ("b", "b_g"):
            return rows_h, None
        if name in ("W_1", "W_2"):
            return np.arange(m), np.arange(d)
        if name in ("b_1", "b_2"):
            return np.arange(m), None
        if name == "U_out":
            return np.arange(2), np.arange(m)
        if name == "c":
            return np.arange(2), None
    raise KeyError(name)


def grow(small, p_small, big, seed, eps):
    """Embed the parameters of ``small`` into the larger model ``big``."""
    if small.cell != big.cell or small.Lx != big.Lx or small.Ly != big.Ly or small.phase != big.phase:
        raise ValueError("growth keeps the cell and the lattice")
    if big.d < small.d or big.m < small.m:
        raise ValueError("growth cannot shrink the model")
    ps = small.unpack(p_small)
    out = {}
    for t, (name, shape) in enumerate(big.shapes()):
        rows = shape[0]
        cols = shape[1] if len(shape) == 2 else 1
        noise = eps * growth_normals(seed, t, rows, cols)
        new = noise.copy()
        rmap, cmap = _index_map(big.cell, name, small, big)
        old = ps[name]
        if cmap is None:
            new[rmap, 0] = old
        else:
            new[np.ix_(rmap, cmap)] = old
        out[name] = new.reshape(shape)
    return big.pack(out)
