"""Local energies by full re-evaluation (test infrastructure; see the package docstring).

E_loc(sigma) = sum_sigma' H[sigma, sigma'] psi(sigma') / psi(sigma) for a
positive wave function psi = exp(logpsi).  Every connected configuration is
evaluated from scratch with ``logpsi_fn`` (no prefix re-use), so the CUDA
path's prefix-cached evaluation is checked against the definition.

TFIM, Eq. (tfim), open chain:
  H = -J sum_{i<N} Z_i Z_{i+1} - Gamma sum_i X_i
  E_loc = -J sum_i s_i s_{i+1} - Gamma sum_i psi(flip_i sigma) / psi(sigma),
  with s = +1 for sigma = 0 (spin up) and -1 for sigma = 1.

Long-range TFIM, Sec. III C, open chain:
  H = -J sum_{i<j} Z_i Z_j / |i - j|^alpha - Gamma sum_i X_i
  (the paper's J = 1; alpha -> infinity is the nearest-neighbour chain).

Cluster state, Sec. III D, open chain of N sites: H = -sum_k K_k with the
stabilisers K_1 = Z_1 X_2, K_k = X_{k-1} Z_k X_{k+1} (1 < k < N) and
K_N = X_{N-1} Z_N.  The paper's boundary terms are garbled; this reading keeps
every stabiliser of the (Hadamard-rotated) cluster state, whose ground energy
is then exactly -N.  E_loc is complex for a cRNN:
  E_loc = -sum_k s_k psi(sigma^(k)) / psi(sigma),
with sigma^(k) the configuration with the X sites of K_k flipped.

Heisenberg, Eq. (heisenberg), open Lx x Ly square lattice, Pauli matrices with
the prefactor 1/4 (so J S_i.S_j per bond):
  diagonal  +J/4 for a parallel bond, -J/4 for an antiparallel bond;
  exchange  an antiparallel bond swaps the two spins with matrix element +J/2,
            or -J/2 after the Marshall rotation (Sec. III B: every off-diagonal
            element of the rotated Hamiltonian is negative).
"""
import numpy as np


def tfim_local_energy(N, J, Gamma, sigma, logpsi_fn):
    """E_loc for the open 1D TFIM; sigma: [B, N] in {0, 1}."""
    sigma = np.asarray(sigma, dtype=np.int64)
    B = sigma.shape[0]
    s = 1 - 2 * sigma
    diag = -J * (s[:, :-1] * s[:, 1:]).sum(axis=1)
    lp = logpsi_fn(sigma)
    flipped = np.repeat(sigma[:, None, :], N, axis=1)          # [B, N, N]
    idx = np.arange(N)
    flipped[:, idx, idx] = 1 - flipped[:, idx, idx]
    lp_f = logpsi_fn(flipped.reshape(B * N, N)).reshape(B, N)
    return diag - Gamma * np.exp(lp_f - lp[:, None]).sum(axis=1)


def square_bonds(Lx, Ly):
    """Nearest-neighbour bonds of the open Lx x Ly lattice, as lattice-index pairs."""
    bonds = []
    for j in range(Ly):
        for i in range(Lx):
            k = j * Lx + i
            if i + 1 < Lx:
                bonds.append((k, k + 1))
            if j + 1 < Ly:
                bonds.append((k, k + Lx))
    return bonds


def heisenberg_local_energy(Lx, Ly, J, marshall, sigma, logpsi_fn):
    """E_loc for the open square-lattice Heisenberg model; sigma: [B, N]."""
    sigma = np.asarray(sigma, dtype=np.int64)
    B, N = sigma.shape
    bonds = square_bonds(Lx, Ly)
    lp = logpsi_fn(sigma)
    off = -0.5 * J if marshall else 0.5 * J
    eloc = np.zeros(B)
    swapped = np.repeat(sigma[:, None, :], len(bonds), axis=1)  # [B, nb, N]
    for t, (a, b) in enumerate(bonds):
        swapped[:, t, a] = sigma[:, b]
        swapped[:, t, b] = sigma[:, a]
    lp_s = logpsi_fn(swapped.reshape(B * len(bonds), N)).reshape(B, len(bonds))
    for t, (a, b) in enumerate(bonds):
        par = sigma[:, a] == sigma[:, b]
        ratio = np.where(par, 0.0, np.exp(np.where(par, 0.0, lp_s[:, t] - lp)))
        eloc += np.where(par, 0.25 * J, -0.25 * J + off * ratio)
    return eloc


def lr_tfim_local_energy(N, alpha, J, Gamma, sigma, logpsi_fn):
    """E_loc of the long-range TFIM (Sec. III C), open chain:
    H = -J sum_{i<j} Z_i Z_j / |i - j|^alpha - Gamma sum_i X_i; the flips as
    in the TFIM, the diagonal summed over every pair."""
    sigma = np.asarray(sigma, dtype=np.int64)
    B = sigma.shape[0]
    s = 1 - 2 * sigma
    diag = np.zeros(B)
    for i in range(N):
        for j in range(i + 1, N):
            diag -= J * s[:, i] * s[:, j] / float(j - i) ** alpha
    lp = logpsi_fn(sigma)
    flipped = np.repeat(sigma[:, None, :], N, axis=1)
    idx = np.arange(N)
    flipped[:, idx, idx] = 1 - flipped[:, idx, idx]
    lp_f = logpsi_fn(flipped.reshape(B * N, N)).reshape(B, N)
    return diag - Gamma * np.exp(lp_f - lp[:, None]).sum(axis=1)


def cluster_terms(N):
    """[(k, flipped sites)] of the cluster Hamiltonian, 0-based (see the module docstring)."""
    if N < 2:
        raise ValueError("the cluster chain needs N >= 2")
    out = [(0, (1,))]
    out += [(k, (k - 1, k + 1)) for k in range(1, N - 1)]
    out.append((N - 1, (N - 2,)))
    return out


def cluster_local_energy(N, sigma, logamp_fn, phase_fn):
    """Complex E_loc of the cluster Hamiltonian for psi = exp(logamp + i phase)."""
    sigma = np.asarray(sigma, dtype=np.int64)
    s = 1 - 2 * sigma
    la, ph = logamp_fn(sigma), phase_fn(sigma)
    e = np.zeros(sigma.shape[0], dtype=np.complex128)
    for k, flips in cluster_terms(N):
        sp = sigma.copy()
        for f in flips:
            sp[:, f] = 1 - sp[:, f]
        e -= s[:, k] * np.exp(logamp_fn(sp) - la + 1j * (phase_fn(sp) - ph))
    return e
