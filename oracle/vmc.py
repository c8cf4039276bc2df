"""VMC estimators and the reverse-mode gradient of log psi (test infrastructure).

Sec. III: the energy E = <psi|H|psi> (psi normalised by construction, Eq. 1) is
estimated by the sample mean of E_loc; the paper trains with the scheme of
Hibat-Allah et al. (2020) and prints no gradient formula.  Reading used here:

  g = (2/M) sum_s (E_loc(sigma_s) - mean E_loc) d log psi(sigma_s) / d theta,

with E_loc and its mean held constant.  The variance uses the 1/M normaliser.

``logpsi_grad`` differentiates L = sum_s w_s log psi(sigma_s) by an explicit
reverse sweep over the unrolled recurrence (the chain rule written out cell by
cell from the App. A equations); it shares nothing with the CUDA adjoint.
"""
import numpy as np

from . import model as M


def energy_stats(eloc):
    """[mean, variance (1/M), M] of the local energies, in float64; for complex
    local energies (cRNN) [Re mean, mean |E - mean|^2, M, Im mean]."""
    if np.iscomplexobj(eloc):
        e = np.asarray(eloc, dtype=np.complex128)
        mean = e.mean()
        return np.array([mean.real, np.mean(np.abs(e - mean) ** 2), float(e.size), mean.imag])
    e = np.asarray(eloc, dtype=np.float64)
    mean = e.mean()
    return np.array([mean, (e * e).mean() - mean * mean, float(e.size)])


def vmc_weights(eloc):
    """w_s = 2 (E_loc,s - mean) / M, the per-sample factor of the VMC gradient
    (complex for a complex E_loc)."""
    e = np.asarray(eloc)
    e = e.astype(np.complex128) if np.iscomplexobj(e) else e.astype(np.float64)
    return 2.0 * (e - e.mean()) / e.size


def vmc_gradient(model, flat, sigma, eloc):
    """g = (2/M) sum_s Re[(E_s - mean)^* d log psi_s]: for a real psi the sum of
    (E_s - mean) d log psi_s; for a cRNN, log psi = log|psi| + i phi, so
    g = (2/M) sum_s [Re(E_s - mean) d log|psi_s| + Im(E_s - mean) d phi_s]."""
    w = vmc_weights(eloc)
    if np.iscomplexobj(w):
        return logpsi_grad(model, flat, sigma, w.real, phase_weights=w.imag)
    return logpsi_grad(model, flat, sigma, w)


def _dlogits(model, z, s, n_up, n_dn, coef):
    """d(coef * log p_n(s)) / dz for the two-outcome softmax; 0 where the mask forces s."""
    prob = np.exp(M.log_softmax2(z))
    dz = coef[:, None] * (M.onehot(s) - prob)
    if model.sz0:
        half = model.N // 2
        forced = (n_up >= half) | (n_dn >= half)
        dz[forced] = 0.0
    return dz


def logpsi_grad(model, flat, sigma, weights, phase_weights=None):
    """d/dtheta of sum_s [w_s log|psi(sigma_s)| + v_s phi(sigma_s)] (v = phase_weights,
    cRNN only), as a flat float64 vector."""
    p = model.unpack(flat)
    sigma = np.asarray(sigma, dtype=np.int64)
    w = np.asarray(weights, dtype=np.float64)
    vph = None if phase_weights is None else np.asarray(phase_weights, dtype=np.float64)
    B, N = sigma.shape
    d = model.d
    g = {name: np.zeros(shape) for name, shape in model.shapes()}
    order = model.order()
    # forward sweep, keeping what the reverse sweep needs
    hid = np.zeros((B, N, d))
    tape = []
    n_up = np.zeros(B, dtype=np.int64)
    n_dn = np.zeros(B, dtype=np.int64)
    zeros_h, zeros_x = np.zeros((B, d)), np.zeros((B, 2))
    for pos, (i, j) in enumerate(order):
        k = model.lattice_index(i, j)
        rec = {"k": k, "n_up": n_up.copy(), "n_dn": n_dn.copy()}
        if model.cell == M.GRU1D:
            if pos == 0:
                h_prev, x, kp = zeros_h, zeros_x, None
            else:
                h_prev, x, kp = hid[:, k - 1], M.onehot(sigma[:, k - 1]), k - 1
            hx = np.concatenate([h_prev, x], axis=1)
            u = M.sigmoid(hx @ p["W_g"].T + p["b_g"])
            r = M.sigmoid(hx @ p["W_r"].T + p["b_r"])
            q = h_prev @ p["W_h"].T + p["b_h"]
            c = np.tanh(r * q + x @ p["W_in"].T + p["b_in"])
            h = (1.0 - u) * h_prev + u * c
            rec.update(h_prev=h_prev, x=x, hx=hx, u=u, r=r, q=q, c=c, kp=kp)
            z = h @ p["U"].T + p["c"]
        else:
            ih = i - (-1) ** j
            kh = model.lattice_index(ih, j) if 0 <= ih < model.Lx else None
            kv = model.lattice_index(i, j - 1) if j >= 1 else None
            h_hor = hid[:, kh] if kh is not None else zeros_h
            x_hor = M.onehot(sigma[:, kh]) if kh is not None else zeros_x
            h_ver = hid[:, kv] if kv is not None else zeros_h
            x_ver = M.onehot(sigma[:, kv]) if kv is not None else zeros_x
            hp = np.concatenate([h_hor, h_ver], axis=1)
            inp = np.concatenate([hp, x_hor, x_ver], axis=1)
            c = np.tanh(inp @ p["W"].T + p["b"])
            u = M.sigmoid(inp @ p["W_g"].T + p["b_g"])
            mix = hp @ p["U_mix"].T
            h = u * c + (1.0 - u) * mix
            y1 = h @ p["W_1"].T + p["b_1"]
            s2 = M.sigmoid(h @ p["W_2"].T + p["b_2"])
            gl = y1 * s2
            rec.update(kh=kh, kv=kv, hp=hp, inp=inp, c=c, u=u, mix=mix, y1=y1, s2=s2, gl=gl)
            z = gl @ p["U_out"].T + p["c"]
        hid[:, k] = h
        rec.update(h=h, z=z)
        tape.append(rec)
        n_up += sigma[:, k] == 0
        n_dn += sigma[:, k] == 1
    # reverse sweep
    carry = np.zeros((B, N, d))           # dL/dh_k accumulated from later cells
    for rec in reversed(tape):
        k, h, z = rec["k"], rec["h"], rec["z"]
        dz = _dlogits(model, z, sigma[:, k], rec["n_up"], rec["n_dn"], 0.5 * w)
        g["c"] += dz.sum(axis=0)
        if model.cell == M.GRU1D:
            g["U"] += dz.T @ h
            dh = dz @ p["U"] + carry[:, k]
            if model.phase and vph is not None:
                # phi_k = pi softsign(z_phi[s_k]); d softsign / dz = 1 / (1 + |z|)^2
                zp = M.phase_logits(p, h)
                sel = M.onehot(sigma[:, k])
                zs = (zp * sel).sum(axis=1)
                dzp = sel * (vph * np.pi / (1.0 + np.abs(zs)) ** 2)[:, None]
                g["U_phi"] += dzp.T @ h
                g["c_phi"] += dzp.sum(axis=0)
                dh = dh + dzp @ p["U_phi"]
            u, r, q, c, h_prev = rec["u"], rec["r"], rec["q"], rec["c"], rec["h_prev"]
            dc = dh * u
            du = dh * (c - h_prev)
            dh_prev = dh * (1.0 - u)
            dac = dc * (1.0 - c * c)
            dau = du * u * (1.0 - u)
            dq = dac * r
            dar = dac * q * r * (1.0 - r)
            g["W_in"] += dac.T @ rec["x"]
            g["b_in"] += dac.sum(axis=0)
            g["W_h"] += dq.T @ h_prev
            g["b_h"] += dq.sum(axis=0)
            g["W_g"] += dau.T @ rec["hx"]
            g["b_g"] += dau.sum(axis=0)
            g["W_r"] += dar.T @ rec["hx"]
            g["b_r"] += dar.sum(axis=0)
            dh_prev = dh_prev + dau @ p["W_g"][:, :d] + dar @ p["W_r"][:, :d] + dq @ p["W_h"]
            if rec["kp"] is not None:
                carry[:, rec["kp"]] += dh_prev
        else:
            g["U_out"] += dz.T @ rec["gl"]
            dgl = dz @ p["U_out"]
            s2, y1 = rec["s2"], rec["y1"]
            dy1 = dgl * s2
            dy2 = dgl * y1 * s2 * (1.0 - s2)
            g["W_1"] += dy1.T @ h
            g["b_1"] += dy1.sum(axis=0)
            g["W_2"] += dy2.T @ h
            g["b_2"] += dy2.sum(axis=0)
            dh = dy1 @ p["W_1"] + dy2 @ p["W_2"] + carry[:, k]
            u, c, mix = rec["u"], rec["c"], rec["mix"]
            dc = dh * u
            du = dh * (c - mix)
            dmix = dh * (1.0 - u)
            da = dc * (1.0 - c * c)
            dg = du * u * (1.0 - u)
            g["W"] += da.T @ rec["inp"]
            g["b"] += da.sum(axis=0)
            g["W_g"] += dg.T @ rec["inp"]
            g["b_g"] += dg.sum(axis=0)
            g["U_mix"] += dmix.T @ rec["hp"]
            dinp = da @ p["W"] + dg @ p["W_g"]
            dhp = dinp[:, :2 * d] + dmix @ p["U_mix"]
            if rec["kh"] is not None:
                carry[:, rec["kh"]] += dhp[:, :d]
            if rec["kv"] is not None:
                carry[:, rec["kv"]] += dhp[:, d:]
    return model.pack(g)
