"""Exact references used to pin the oracle (test infrastructure).

* ``all_configs``          every configuration of N spins (lattice order)
* ``tfim_hamiltonian``     sparse Eq. (tfim) in the sigma basis
* ``heisenberg_hamiltonian`` sparse Eq. (heisenberg), optionally Marshall-rotated
* ``lr_tfim_hamiltonian``  sparse long-range TFIM (Sec. III C)
* ``cluster_hamiltonian``  sparse cluster Hamiltonian (Sec. III D)
* ``ground_state``         exact diagonalisation (scipy eigsh / dense eigh)
* ``tfim_free_fermion``    ground energy of the open TFIM from free fermions:
                           E0 = -1/2 sum_k eps_k, with eps_k the singular values
                           of the N x N upper-bidiagonal matrix with 2*Gamma on
                           the diagonal and 2*J above it (Jordan-Wigner,
                           Lieb-Schultz-Mattis); at J = Gamma = 1 this is
                           E0 = 1 - csc(pi / (2 (2N + 1))) (Pfeuty, 1970)
* ``exact_energy``         sum_sigma P(sigma) E_loc(sigma) by enumeration
* ``exact_gradient``       sum_sigma P (E_loc - E) d log P / d theta
* ``central_fd``           central finite differences of a scalar function

Basis convention: configuration sigma (lattice order) is basis index
sum_k sigma_k 2^k; sigma_k = 0 is spin up, Z_k = +1.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hamiltonian as H
from . import vmc


def all_configs(N):
    idx = np.arange(2 ** N, dtype=np.int64)
    return ((idx[:, None] >> np.arange(N)[None, :]) & 1).astype(np.int64)


def sz0_configs(N):
    c = all_configs(N)
    return c[c.sum(axis=1) == N // 2]


def tfim_hamiltonian(N, J, Gamma):
    dim = 2 ** N
    idx = np.arange(dim, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(N)[None, :]) & 1
    z = 1 - 2 * bits
    diag = -J * (z[:, :-1] * z[:, 1:]).sum(axis=1)
    rows = [idx]
    cols = [idx]
    vals = [diag.astype(np.float64)]
    for k in range(N):
        rows.append(idx)
        cols.append(idx ^ (1 << k))
        vals.append(np.full(dim, -Gamma, dtype=np.float64))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(dim, dim))


def lr_tfim_hamiltonian(N, alpha, J, Gamma):
    """Sparse long-range TFIM (Sec. III C) in the sigma basis."""
    dim = 2 ** N
    idx = np.arange(dim, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(N)[None, :]) & 1
    z = 1 - 2 * bits
    diag = np.zeros(dim)
    for i in range(N):
        for j in range(i + 1, N):
            diag -= J * z[:, i] * z[:, j] / float(j - i) ** alpha
    rows = [idx]
    cols = [idx]
    vals = [diag]
    for k in range(N):
        rows.append(idx)
        cols.append(idx ^ (1 << k))
        vals.append(np.full(dim, -Gamma, dtype=np.float64))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(dim, dim))


def cluster_hamiltonian(N):
    """Sparse cluster Hamiltonian (Sec. III D, the stabiliser reading of
    ``hamiltonian.cluster_terms``): <sigma^(k)| -K_k |sigma> = -s_k(sigma)."""
    dim = 2 ** N
    idx = np.arange(dim, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(N)[None, :]) & 1
    z = 1 - 2 * bits
    rows, cols, vals = [], [], []
    for k, flips in H.cluster_terms(N):
        mask = 0
        for f in flips:
            mask |= 1 << f
        rows.append(idx ^ mask)
        cols.append(idx)
        vals.append(-z[:, k].astype(np.float64))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(dim, dim))


def heisenberg_hamiltonian(Lx, Ly, J=1.0, marshall=False):
    """Eq. (heisenberg) with Pauli matrices and prefactor J/4 on every open-lattice bond.

    X_a X_b + Y_a Y_b maps |..s_a..s_b..> with s_a != s_b to 2|..s_b..s_a..>;
    Z_a Z_b is +1 / -1 for parallel / antiparallel.  ``marshall`` conjugates
    by the diagonal sign (-1)^(number of up spins on the sublattice i + j even).
    """
    N = Lx * Ly
    dim = 2 ** N
    idx = np.arange(dim, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(N)[None, :]) & 1
    sub_a = np.array([((k % Lx) + (k // Lx)) % 2 == 0 for k in range(N)])
    sign = (-1.0) ** ((bits[:, sub_a] == 0).sum(axis=1))
    diag = np.zeros(dim)
    rows, cols, vals = [], [], []
    for a, b in H.square_bonds(Lx, Ly):
        par = bits[:, a] == bits[:, b]
        diag += np.where(par, 0.25 * J, -0.25 * J)
        anti = idx[~par]
        tgt = anti ^ ((1 << a) | (1 << b))
        rows.append(anti)
        cols.append(tgt)
        v = np.full(anti.size, 0.5 * J)
        if marshall:
            v = v * sign[anti] * sign[tgt]
        vals.append(v)
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(dim, dim))


def ground_state(Hm, restrict=None):
    """(E0, psi0) of a sparse Hamiltonian, optionally restricted to basis subset ``restrict``."""
    if restrict is not None:
        Hm = Hm[restrict][:, restrict]
    if Hm.shape[0] <= 2048:
        w, v = np.linalg.eigh(Hm.toarray())
        return w[0], v[:, 0]
    w, v = spla.eigsh(Hm, k=1, which="SA", tol=1e-13, maxiter=100000)
    return w[0], v[:, 0]


def tfim_free_fermion(N, J, Gamma):
    Bm = np.diag(np.full(N, 2.0 * Gamma)) + np.diag(np.full(N - 1, 2.0 * J), 1)
    return -0.5 * np.linalg.svd(Bm, compute_uv=False).sum()


def tfim_closed_form_critical(N):
    return 1.0 - 1.0 / np.sin(np.pi / (2.0 * (2 * N + 1)))


def basis_index(sigma):
    sigma = np.asarray(sigma, dtype=np.int64)
    return (sigma << np.arange(sigma.shape[1])[None, :]).sum(axis=1)


def exact_energy(probs, eloc):
    return float(np.sum(probs * eloc))


def exact_gradient(model, flat, configs, probs, eloc):
    """Exact dE/dtheta = sum_sigma P (E_loc - E) d log P / d theta = 2 sum P (E_loc - E) d log psi;
    for a complex E_loc (cRNN), 2 sum P [Re(E_loc - E) d log|psi| + Im(E_loc - E) d phi]."""
    E = np.sum(probs * eloc)
    w = 2.0 * probs * (eloc - E)
    if np.iscomplexobj(w):
        return vmc.logpsi_grad(model, flat, configs, w.real, phase_weights=w.imag)
    return vmc.logpsi_grad(model, flat, configs, w)


def central_fd(f, x, h=1e-5, idx=None):
    x = np.asarray(x, dtype=np.float64)
    idx = np.arange(x.size) if idx is None else np.asarray(idx)
    out = np.zeros(len(idx))
    for t, k in enumerate(idx):
        xp = x.copy()
        xm = x.copy()
        xp[k] += h
        xm[k] -= h
        out[t] = (f(xp) - f(xm)) / (2 * h)
    return out
