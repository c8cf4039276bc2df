"""Per-draw check of GPU samples against the oracle along the GPU's own path.

The oracle is evaluated teacher-forced on the configurations the GPU drew, so
every draw of every sample is checked against u < p0 computed in float64 from
the same prefix; a divergence at one draw does not hide the later ones.  Draws
whose uniform lies within `window` of the oracle's threshold are not checked
(the GPU's p0 differs from the float64 one by its rounding), and their
fraction is returned.  Draws that the zero-magnetisation mask forces must take
the forced value.
"""
import numpy as np

from oracle import model as om


def check_draws(mod, flat, sigma_gpu, u, window):
    """sigma_gpu [B, N] lattice order (numpy), u [B, N] sampling order,
    window scalar or [N] per sampling position.  Raises on a mismatch outside
    the window; returns (fraction of unforced draws inside the window,
    number of mismatches inside it)."""
    s_lat = np.asarray(sigma_gpu, dtype=np.int64)
    ref = om.run(mod, flat, sigma=s_lat)
    order = np.array([mod.lattice_index(i, j) for (i, j) in mod.order()])
    p0 = ref["p0"][:, order]
    s = s_lat[:, order]
    B, N = s.shape
    n_up = np.concatenate([np.zeros((B, 1), dtype=np.int64), np.cumsum(s == 0, axis=1)[:, :-1]], axis=1)
    n_dn = np.arange(N)[None, :] - n_up
    if mod.sz0:
        forced_dn, forced_up = n_up >= N // 2, n_dn >= N // 2
    else:
        forced_dn = forced_up = np.zeros_like(s, dtype=bool)
    free = ~(forced_dn | forced_up)
    expected = np.where(forced_dn, 1, np.where(forced_up, 0, (u >= p0).astype(np.int64)))
    near = free & (np.abs(u - p0) < np.broadcast_to(np.asarray(window, dtype=np.float64), (B, N)))
    bad = (s != expected) & ~near
    if bad.any():
        b, n = np.argwhere(bad)[0]
        raise AssertionError("draw (sample %d, position %d) differs: u = %.9f, p0 = %.9f, forced %s"
                             % (b, n, u[b, n], p0[b, n], bool(~free[b, n])))
    return float(near.sum() / max(free.sum(), 1)), int(((s != expected) & near).sum())
