"""RNN wave functions in float64 (test infrastructure; see the package docstring).

Conventions (the paper leaves them open; these are the readings used
throughout):

* spins sigma_n in {0, 1}; sigma = 0 is spin up (sigma^z = +1); the one-hot
  encoding of sigma is e_sigma and the "no input" vector (sigma_0, and a
  neighbour outside the lattice) is the zero vector (Eq. 2, h_0 = 0, sigma_0 = 0);
* configurations are stored in lattice order, index j*Lx + i for column i and
  row j (1D: Ly = 1);
* sampling order: 1D left to right; 2D zig-zag over rows, row 0 left to right,
  row j odd right to left (Sec. II, Fig. 1(b): the horizontal neighbour is
  i - (-1)^j, the vertical one (i, j-1));
* zero-magnetisation mask (optional): once the prefix holds N/2 up spins every
  remaining spin is down with conditional probability 1, and vice versa.

Flat parameter layout (row-major, in this order; also the C-ABI layout):

1D GRU (App. A), d = d_h:
  W_g[d, d+2], W_r[d, d+2], W_h[d, d], W_in[d, 2], b_g[d], b_r[d], b_h[d],
  b_in[d], U[2, d], c[2]                 -- columns of W_g, W_r: [h | sigma]
  cRNN (phase head, Eq. softsign) appends U_phi[2, d], c_phi[2]
2D GRU + GLU (App. A), d = d_h, m = d_model:
  W[d, 2d+4], W_g[d, 2d+4], U_mix[d, 2d], b[d], b_g[d], W_1[m, d], b_1[m],
  W_2[m, d], b_2[m], U_out[2, m], c[2]   -- columns: [h_hor | h_ver | s_hor | s_ver]
"""
import numpy as np

GRU1D = 1
GRU2D = 2


class Model:
    """Shape of one RNN wave function."""

    def __init__(self, cell, Lx, Ly=1, d_h=8, d_model=None, sz0=False, phase=False):
        self.cell = cell
        self.Lx = Lx
        self.Ly = Ly
        self.N = Lx * Ly
        self.d = d_h
        self.m = d_h if d_model is None else d_model
        self.sz0 = bool(sz0)
        self.phase = bool(phase)
        if cell == GRU1D and Ly != 1:
            raise ValueError("1D GRU needs Ly == 1")
        if phase and cell != GRU1D:
            raise ValueError("the phase head is built for the 1D GRU")

    def shapes(self):
        d, m = self.d, self.m
        if self.cell == GRU1D:
            base = [("W_g", (d, d + 2)), ("W_r", (d, d + 2)), ("W_h", (d, d)),
                    ("W_in", (d, 2)), ("b_g", (d,)), ("b_r", (d,)), ("b_h", (d,)),
                    ("b_in", (d,)), ("U", (2, d)), ("c", (2,))]
            # cRNN (Eq. softsign): phase layer U_phi h_n + c_phi after the amplitude head
            return base + ([("U_phi", (2, d)), ("c_phi", (2,))] if self.phase else [])
        return [("W", (d, 2 * d + 4)), ("W_g", (d, 2 * d + 4)), ("U_mix", (d, 2 * d)),
                ("b", (d,)), ("b_g", (d,)), ("W_1", (m, d)), ("b_1", (m,)),
                ("W_2", (m, d)), ("b_2", (m,)), ("U_out", (2, m)), ("c", (2,))]

    def param_count(self):
        return sum(int(np.prod(s)) for _, s in self.shapes())

    def unpack(self, flat):
        flat = np.asarray(flat, dtype=np.float64)
        if flat.size != self.param_count():
            raise ValueError("parameter vector has the wrong length")
        out, off = {}, 0
        for name, shape in self.shapes():
            size = int(np.prod(shape))
            out[name] = flat[off:off + size].reshape(shape)
            off += size
        return out

    def pack(self, tensors):
        return np.concatenate([np.asarray(tensors[name], dtype=np.float64).reshape(-1)
                               for name, _ in self.shapes()])

    # ---- ordering -------------------------------------------------------------
    def order(self):
        """List of (i, j) in sampling order."""
        out = []
        for j in range(self.Ly):
            cols = range(self.Lx) if j % 2 == 0 else range(self.Lx - 1, -1, -1)
            out.extend((i, j) for i in cols)
        return out

    def lattice_index(self, i, j):
        return j * self.Lx + i


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def onehot(s):
    """One-hot rows e_sigma for an integer array s of 0/1."""
    s = np.asarray(s)
    out = np.zeros(s.shape + (2,))
    out[..., 0] = (s == 0)
    out[..., 1] = (s == 1)
    return out


def log_softmax2(z):
    """log Softmax over the two outcomes (Eq. 3), z: [..., 2]."""
    return z - np.logaddexp(z[..., :1], z[..., 1:])


def gru1d_cell(p, h, x):
    """One 1D GRU step (App. A).  h: [B, d] previous state, x: [B, 2] one-hot input."""
    hx = np.concatenate([h, x], axis=1)
    u = sigmoid(hx @ p["W_g"].T + p["b_g"])
    r = sigmoid(hx @ p["W_r"].T + p["b_r"])
    h_cand = np.tanh(r * (h @ p["W_h"].T + p["b_h"]) + x @ p["W_in"].T + p["b_in"])
    return (1.0 - u) * h + u * h_cand


def gru2d_cell(p, h_hor, h_ver, x_hor, x_ver):
    """One 2D GRU step (App. A) on h' = [h_hor; h_ver], sigma' = [x_hor; x_ver]."""
    hp = np.concatenate([h_hor, h_ver], axis=1)
    inp = np.concatenate([hp, x_hor, x_ver], axis=1)
    h_cand = np.tanh(inp @ p["W"].T + p["b"])
    u = sigmoid(inp @ p["W_g"].T + p["b_g"])
    return u * h_cand + (1.0 - u) * (hp @ p["U_mix"].T)


def glu(p, h):
    """Gated linear unit applied to the 2D hidden state before the softmax (App. A)."""
    return (h @ p["W_1"].T + p["b_1"]) * sigmoid(h @ p["W_2"].T + p["b_2"])


def readout_logits(model, p, h):
    if model.cell == GRU1D:
        return h @ p["U"].T + p["c"]
    return glu(p, h) @ p["U_out"].T + p["c"]


def softsign(x):
    return x / (1.0 + np.abs(x))


def phase_logits(p, h):
    """cRNN phase layer (Eq. softsign): z_phi = U_phi h + c_phi, one entry per spin value."""
    return h @ p["U_phi"].T + p["c_phi"]


def _mask_logp(model, logp, n_up, n_dn):
    """Zero-magnetisation mask: forced spins get log p = 0 and the other -inf."""
    if not model.sz0:
        return logp
    half = model.N // 2
    logp = logp.copy()
    force_dn = n_up >= half
    force_up = n_dn >= half
    logp[force_dn, 0] = -np.inf
    logp[force_dn, 1] = 0.0
    logp[force_up, 0] = 0.0
    logp[force_up, 1] = -np.inf
    return logp


def run(model, flat, sigma=None, uniforms=None):
    """Evaluate (teacher forcing) or sample the RNN along the sampling order.

    sigma: [B, N] in lattice order (teacher forcing) or None (sampling with
    uniforms [B, N] indexed by sampling position: sigma_n = 0 iff u_n < p_n(0)).
    Returns dict with sigma, logp [B, N] (log p_n(sigma_n), lattice order),
    p0 [B, N] (unmasked p_n(0)), logits [B, N, 2], hidden [B, N, d], logpsi [B].
    """
    p = model.unpack(flat)
    N, d = model.N, model.d
    sampling = sigma is None
    if sampling:
        uniforms = np.asarray(uniforms, dtype=np.float64)
        B = uniforms.shape[0]
        sigma = np.zeros((B, N), dtype=np.int64)
    else:
        sigma = np.asarray(sigma, dtype=np.int64).copy()
        B = sigma.shape[0]
    hid = np.zeros((B, N, d))
    logits = np.zeros((B, N, 2))
    logp_site = np.zeros((B, N))
    phi_site = np.zeros((B, N))
    phlog = np.zeros((B, N, 2))
    p0 = np.zeros((B, N))
    n_up = np.zeros(B, dtype=np.int64)
    n_dn = np.zeros(B, dtype=np.int64)
    zeros_h = np.zeros((B, d))
    zeros_x = np.zeros((B, 2))
    for pos, (i, j) in enumerate(model.order()):
        k = model.lattice_index(i, j)
        if model.cell == GRU1D:
            if pos == 0:
                h = gru1d_cell(p, zeros_h, zeros_x)
            else:
                h = gru1d_cell(p, hid[:, k - 1], onehot(sigma[:, k - 1]))
        else:
            ih = i - (-1) ** j
            if 0 <= ih < model.Lx:
                kh = model.lattice_index(ih, j)
                h_hor, x_hor = hid[:, kh], onehot(sigma[:, kh])
            else:
                h_hor, x_hor = zeros_h, zeros_x
            if j >= 1:
                kv = model.lattice_index(i, j - 1)
                h_ver, x_ver = hid[:, kv], onehot(sigma[:, kv])
            else:
                h_ver, x_ver = zeros_h, zeros_x
            h = gru2d_cell(p, h_hor, h_ver, x_hor, x_ver)
        hid[:, k] = h
        z = readout_logits(model, p, h)
        logits[:, k] = z
        lp = _mask_logp(model, log_softmax2(z), n_up, n_dn)
        p0[:, k] = np.exp(log_softmax2(z)[:, 0])
        if sampling:
            s = np.where(uniforms[:, pos] < np.exp(lp[:, 0]), 0, 1)
            sigma[:, k] = s
        s = sigma[:, k]
        logp_site[:, k] = lp[np.arange(B), s]
        if model.phase:
            # phi_n = pi Softsign(U_phi h_n + c_phi) . onehot(sigma_n) (Eq. softsign)
            zp = phase_logits(p, h)
            phlog[:, k] = zp
            phi_site[:, k] = np.pi * softsign(zp[np.arange(B), s])
        n_up += (s == 0)
        n_dn += (s == 1)
    return {"sigma": sigma, "logp": logp_site, "p0": p0, "logits": logits,
            "hidden": hid, "logpsi": 0.5 * logp_site.sum(axis=1),
            "phase_logits": phlog, "phase": phi_site.sum(axis=1)}


def logpsi(model, flat, sigma):
    """log psi(sigma) = 1/2 sum_n log p_n(sigma_n) (Eq. 1 and the pRNN amplitude)."""
    return run(model, flat, sigma=sigma)["logpsi"]


def phase(model, flat, sigma):
    """phi(sigma) = sum_n phi_n of the cRNN (Sec. II, Eq. softsign); 0 for a pRNN."""
    return run(model, flat, sigma=sigma)["phase"]


def sample(model, flat, uniforms):
    """Exact autoregressive sampling with given uniforms (one per site, sampling order)."""
    return run(model, flat, uniforms=uniforms)
