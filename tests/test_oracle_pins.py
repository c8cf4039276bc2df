"""Pins of the float64 oracle against what the paper and the physics fix (CPU only).

Each test checks the oracle against something other than itself: published
known-answer vectors, values printed in the paper, closed forms, exact
diagonalisation, a library routine that reduces to the same cell, invariants
(autoregressive normalisation, constant local energy on an eigenstate) and
finite differences.
"""
import os

import numpy as np
import pytest
import scipy.stats

from oracle import exact, growth, hamiltonian, model as M, philox, vmc
from paper_2507_18700_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lp_fn(mod, flat):
    return lambda s: M.logpsi(mod, flat, s)


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = philox.philox4x32_10([np.array([c]) for c in v[:4]], (v[4], v[5]))
        assert [int(o[0]) for o in out] == v[6:]


def test_philox_uniforms_are_uniform():
    u = philox.sampling_uniforms(seed=7, step=3, B=2000, N=50).ravel()
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3
    assert scipy.stats.kstest(u, "uniform").pvalue > 1e-3
    z = philox.growth_normals(2, 5, 300, 300).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-3


# ------------------------------------------------------------------ cells ----
def test_gru1d_cell_is_the_reset_after_gru_of_torch():
    """The App. A cell equals torch.nn.GRUCell with z = 1 - u (weights mapped)."""
    torch = pytest.importorskip("torch")
    d = 5
    mod = M.Model(M.GRU1D, 4, d_h=d)
    p = mod.unpack(inputs.xavier_params(1, d, seed=3, noise_std=0.3))
    cell = torch.nn.GRUCell(2, d).double()
    with torch.no_grad():
        cell.weight_ih.copy_(torch.from_numpy(np.concatenate(
            [p["W_r"][:, d:], -p["W_g"][:, d:], p["W_in"]])))
        cell.weight_hh.copy_(torch.from_numpy(np.concatenate(
            [p["W_r"][:, :d], -p["W_g"][:, :d], p["W_h"]])))
        cell.bias_ih.copy_(torch.from_numpy(np.concatenate([p["b_r"], -p["b_g"], p["b_in"]])))
        cell.bias_hh.copy_(torch.from_numpy(np.concatenate([np.zeros(d), np.zeros(d), p["b_h"]])))
    rng = np.random.default_rng(0)
    h = rng.normal(size=(7, d))
    x = M.onehot(rng.integers(0, 2, size=7))
    ref = cell(torch.from_numpy(x), torch.from_numpy(h)).detach().numpy()
    np.testing.assert_allclose(M.gru1d_cell(p, h, x), ref, rtol=1e-13, atol=1e-13)


# --------------------------------------------------- normalisation (Eq. 1) ----
@pytest.mark.parametrize("cell,Lx,Ly,d,sz0", [
    (M.GRU1D, 10, 1, 6, False),
    (M.GRU1D, 8, 1, 4, True),
    (M.GRU2D, 3, 3, 4, False),
    (M.GRU2D, 2, 4, 3, True),
    (M.GRU2D, 4, 2, 3, False),
])
def test_autoregressive_normalisation(cell, Lx, Ly, d, sz0):
    """sum_sigma P(sigma) = 1; a conditional that read a later spin would break it."""
    mod = M.Model(cell, Lx, Ly, d_h=d, sz0=sz0)
    flat = inputs.xavier_params(cell, d, seed=11, noise_std=0.5)
    configs = exact.all_configs(mod.N)
    P = np.exp(2.0 * M.logpsi(mod, flat, configs))
    assert abs(P.sum() - 1.0) < 1e-12
    if sz0:
        outside = configs.sum(axis=1) != mod.N // 2
        assert np.all(P[outside] == 0.0)


# -------------------------------------------------------------- sampling ----
@pytest.mark.parametrize("cell,Lx,Ly,d,sz0", [(M.GRU1D, 6, 1, 4, False),
                                             (M.GRU2D, 2, 3, 3, True)])
def test_sampling_frequencies_match_probabilities(cell, Lx, Ly, d, sz0):
    mod = M.Model(cell, Lx, Ly, d_h=d, sz0=sz0)
    flat = inputs.xavier_params(cell, d, seed=5, noise_std=0.7)
    n = 200_000
    u = philox.sampling_uniforms(seed=1, step=0, B=n, N=mod.N)
    out = M.sample(mod, flat, u)
    configs = exact.all_configs(mod.N)
    P = np.exp(2.0 * M.logpsi(mod, flat, configs))
    counts = np.bincount(exact.basis_index(out["sigma"]), minlength=configs.shape[0])
    keep = P > 0
    assert counts[~keep].sum() == 0
    chi2 = ((counts[keep] - n * P[keep]) ** 2 / (n * P[keep])).sum()
    dof = keep.sum() - 1
    assert scipy.stats.chi2.sf(chi2, dof) > 1e-4
    np.testing.assert_allclose(out["logpsi"], M.logpsi(mod, flat, out["sigma"]), atol=1e-12)


# ------------------------------------------------ ground energies (pins) ----
def test_free_fermion_matches_closed_form_and_ed():
    for N in (2, 5, 10):
        assert abs(exact.tfim_free_fermion(N, 1.0, 1.0) - exact.tfim_closed_form_critical(N)) < 1e-12
    for G in (0.5, 1.0, 1.5, 2.0):
        e_ed, _ = exact.ground_state(exact.tfim_hamiltonian(10, 1.0, G))
        assert abs(e_ed - exact.tfim_free_fermion(10, 1.0, G)) < 1e-10


def test_closed_form_matches_table1():
    """Table I prints E_RNN and (E_RNN - E_DMRG)/|E_DMRG|; the closed form is E_DMRG."""
    for line in open(os.path.join(GOLDEN, "table1_tfim_energies.txt")):
        if line.startswith("#") or not line.strip():
            continue
        N, _, E, _, rel, drel = line.split()
        e0 = exact.tfim_closed_form_critical(int(N))
        got = (float(E) - e0) / abs(e0) * 1e7
        assert float(E) >= e0                       # variational bound
        assert abs(got - float(rel)) <= float(drel) + 1.0


def test_heisenberg_textbook_ground_energies():
    # two spins: singlet -3/4; 2x2 open square = four-site ring: -2
    assert abs(exact.ground_state(exact.heisenberg_hamiltonian(2, 1))[0] + 0.75) < 1e-12
    assert abs(exact.ground_state(exact.heisenberg_hamiltonian(2, 2))[0] + 2.0) < 1e-12
    # four-site open chain: -(3/4 + sqrt(3)/2)
    assert abs(exact.ground_state(exact.heisenberg_hamiltonian(4, 1))[0]
               + 0.75 + np.sqrt(3) / 2) < 1e-12
    # the Marshall rotation is a unitary: same spectrum
    for Lx, Ly in ((2, 3), (3, 2), (2, 4)):
        a = np.linalg.eigvalsh(exact.heisenberg_hamiltonian(Lx, Ly).toarray())
        b = np.linalg.eigvalsh(exact.heisenberg_hamiltonian(Lx, Ly, marshall=True).toarray())
        np.testing.assert_allclose(a, b, atol=1e-11)


# ----------------------------------- local energy on an exact eigenstate ----
@pytest.mark.parametrize("Gamma", [0.5, 1.0, 2.0])
def test_tfim_local_energy_is_constant_on_ground_state(Gamma):
    N = 10
    e0, v = exact.ground_state(exact.tfim_hamiltonian(N, 1.0, Gamma))
    psi = np.abs(v)                       # Perron-Frobenius: one sign
    table = np.log(psi)
    lp = lambda s: table[exact.basis_index(s)]
    configs = exact.all_configs(N)
    el = hamiltonian.tfim_local_energy(N, 1.0, Gamma, configs, lp)
    np.testing.assert_allclose(el, e0, atol=1e-9)
    assert abs(e0 - exact.tfim_free_fermion(N, 1.0, Gamma)) < 1e-10


@pytest.mark.parametrize("Lx,Ly", [(2, 2), (2, 4), (4, 3)])
def test_heisenberg_local_energy_is_constant_on_ground_state(Lx, Ly):
    N = Lx * Ly
    configs = exact.sz0_configs(N)
    sector = exact.basis_index(configs)
    Hm = exact.heisenberg_hamiltonian(Lx, Ly, marshall=True)
    e0, v = exact.ground_state(Hm, restrict=sector)
    psi = np.abs(v)
    assert np.all(psi > 1e-12)            # positive after the Marshall rotation
    full = np.full(2 ** N, -np.inf)
    full[sector] = np.log(psi)
    lp = lambda s: full[exact.basis_index(s)]
    el = hamiltonian.heisenberg_local_energy(Lx, Ly, 1.0, True, configs, lp)
    np.testing.assert_allclose(el, e0, atol=1e-8)
    e_plain, _ = exact.ground_state(exact.heisenberg_hamiltonian(Lx, Ly), restrict=sector)
    assert abs(e0 - e_plain) < 1e-10


# ---------------------------------------- exact energy by two routes ----
def test_rnn_energy_two_routes_tfim():
    N, d = 8, 5
    mod = M.Model(M.GRU1D, N, d_h=d)
    flat = inputs.xavier_params(1, d, seed=2, noise_std=0.3)
    configs = exact.all_configs(N)
    lpsi = M.logpsi(mod, flat, configs)
    P = np.exp(2 * lpsi)
    el = hamiltonian.tfim_local_energy(N, 1.0, 1.0, configs, _lp_fn(mod, flat))
    e_sum = exact.exact_energy(P, el)
    psi = np.exp(lpsi)
    Hm = exact.tfim_hamiltonian(N, 1.0, 1.0)
    assert abs(e_sum - psi @ (Hm @ psi)) < 1e-11
    assert e_sum >= exact.tfim_free_fermion(N, 1.0, 1.0)


def test_rnn_energy_two_routes_heisenberg():
    Lx, Ly, d = 2, 4, 4
    mod = M.Model(M.GRU2D, Lx, Ly, d_h=d, sz0=True)
    flat = inputs.xavier_params(2, d, seed=4, noise_std=0.3)
    configs = exact.sz0_configs(mod.N)
    lpsi = M.logpsi(mod, flat, configs)
    P = np.exp(2 * lpsi)
    el = hamiltonian.heisenberg_local_energy(Lx, Ly, 1.0, True, configs, _lp_fn(mod, flat))
    e_sum = exact.exact_energy(P, el)
    psi = np.zeros(2 ** mod.N)
    psi[exact.basis_index(configs)] = np.exp(lpsi)
    Hm = exact.heisenberg_hamiltonian(Lx, Ly, marshall=True)
    assert abs(e_sum - psi @ (Hm @ psi)) < 1e-11
    e0, _ = exact.ground_state(Hm, restrict=exact.basis_index(configs))
    assert e_sum >= e0


def test_energy_stats():
    st = vmc.energy_stats([1.0, 2.0, 3.0, 6.0])
    np.testing.assert_allclose(st, [3.0, 3.5, 4.0])


# ------------------------------------------------------------- gradients ----
@pytest.mark.parametrize("cell,Lx,Ly,d,sz0", [(M.GRU1D, 5, 1, 3, False),
                                             (M.GRU2D, 2, 3, 3, False),
                                             (M.GRU2D, 3, 2, 2, True)])
def test_logpsi_gradient_matches_finite_differences(cell, Lx, Ly, d, sz0):
    mod = M.Model(cell, Lx, Ly, d_h=d, sz0=sz0)
    flat = inputs.xavier_params(cell, d, seed=8, noise_std=0.4)
    sig = inputs.random_configs(6, mod.N, seed=9, sz0=sz0).astype(np.int64)
    w = inputs.random_weights(6, seed=10)
    g = vmc.logpsi_grad(mod, flat, sig, w)
    fd = exact.central_fd(lambda x: float(w @ M.logpsi(mod, x, sig)), flat, h=1e-5)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_exact_gradient_matches_fd_of_exact_energy():
    """d/dtheta <psi|H|psi> (dense H, enumeration) = sum P (E_loc - E) d log P."""
    N, d = 6, 3
    mod = M.Model(M.GRU1D, N, d_h=d)
    flat = inputs.xavier_params(1, d, seed=12, noise_std=0.4)
    configs = exact.all_configs(N)
    Hm = exact.tfim_hamiltonian(N, 1.0, 0.7)

    def energy(x):
        psi = np.exp(M.logpsi(mod, x, configs))
        return psi @ (Hm @ psi)

    P = np.exp(2 * M.logpsi(mod, flat, configs))
    el = hamiltonian.tfim_local_energy(N, 1.0, 0.7, configs, _lp_fn(mod, flat))
    g = exact.exact_gradient(mod, flat, configs, P, el)
    fd = exact.central_fd(energy, flat, h=1e-5)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


# ---------------------------------------------------------------- growth ----
@pytest.mark.parametrize("cell,Lx,Ly,sz0", [(M.GRU1D, 8, 1, False), (M.GRU2D, 2, 4, True)])
def test_growth_with_zero_noise_keeps_the_wave_function(cell, Lx, Ly, sz0):
    small = M.Model(cell, Lx, Ly, d_h=3, sz0=sz0)
    big = M.Model(cell, Lx, Ly, d_h=6, sz0=sz0)
    ps = inputs.xavier_params(cell, 3, seed=13, noise_std=0.3)
    pb = growth.grow(small, ps, big, seed=2, eps=0.0)
    configs = exact.sz0_configs(small.N) if sz0 else exact.all_configs(small.N)
    np.testing.assert_allclose(M.logpsi(big, pb, configs), M.logpsi(small, ps, configs),
                               atol=1e-13)
    pe = growth.grow(small, ps, big, seed=2, eps=1e-3)
    diff = np.abs(M.logpsi(big, pe, configs) - M.logpsi(small, ps, configs))
    assert 0 < diff.max() < 1e-3 * small.N
    new = np.abs(pe - pb)
    assert np.count_nonzero(new) == big.param_count() - small.param_count()
    assert abs(new[new > 0].mean() - 1e-3 * np.sqrt(2 / np.pi)) < 2e-4


# ------------------------------------ sample estimator of the gradient ----
def test_vmc_weights_hand_computed():
    """Three local energies 1, 2, 6: mean 3, w = 2 (E - 3) / 3 = (-4/3, -2/3, 2)."""
    np.testing.assert_allclose(vmc.vmc_weights([1.0, 2.0, 6.0]), [-4.0 / 3, -2.0 / 3, 2.0],
                               rtol=0, atol=1e-15)


def _estimator_setup():
    N, d, Gamma = 6, 3, 0.7
    mod = M.Model(M.GRU1D, N, d_h=d)
    flat = inputs.xavier_params(1, d, seed=21, noise_std=0.6)
    configs = exact.all_configs(N)
    el_all = hamiltonian.tfim_local_energy(N, 1.0, Gamma, configs, _lp_fn(mod, flat))
    return mod, flat, configs, el_all, exact.tfim_hamiltonian(N, 1.0, Gamma)


def test_vmc_gradient_is_unbiased_for_fd_of_exact_energy():
    """The sample estimator g = (2/M) sum_s (E_s - mean) d log psi_s, on M = 2e5
    exact autoregressive samples, equals the central finite difference of the
    exact energy <psi|H|psi> (dense H) within 4 standard errors per component.
    A dropped factor 2 or a sign error fails by many standard errors (checked)."""
    mod, flat, configs, el_all, Hm = _estimator_setup()
    Msamp = 200_000
    u = philox.sampling_uniforms(seed=5, step=0, B=Msamp, N=mod.N)
    sig = M.sample(mod, flat, u)["sigma"]
    idx = exact.basis_index(sig)
    eloc = el_all[idx]
    g = vmc.vmc_gradient(mod, flat, sig, eloc)

    def energy(x):
        psi = np.exp(M.logpsi(mod, x, configs))
        return psi @ (Hm @ psi)

    fd = exact.central_fd(energy, flat, h=1e-5)
    # per-sample contributions 2 (E_s - mean) d log psi(sigma_s) for the standard error
    jac = np.stack([vmc.logpsi_grad(mod, flat, configs[k:k + 1], np.ones(1))
                    for k in range(configs.shape[0])])
    contrib = 2.0 * (eloc - eloc.mean())[:, None] * jac[idx]
    np.testing.assert_allclose(contrib.mean(axis=0), g, rtol=1e-9, atol=1e-12)
    se = contrib.std(axis=0) / np.sqrt(Msamp) + 1e-12
    z = np.abs(g - fd) / se
    assert z.max() < 4.0, z.max()
    # the test has power: half the estimator, or its negative, is far outside
    assert (np.abs(0.5 * g - fd) / se).max() > 20.0
    assert (np.abs(-g - fd) / se).max() > 20.0


def test_vmc_gradient_is_invariant_to_an_energy_shift():
    """Adding a constant to H adds it to every E_loc and leaves dE/dtheta unchanged;
    the mean subtraction makes the sample estimator invariant exactly (up to
    rounding), which an estimator without the centring is not (checked)."""
    mod, flat, configs, el_all, _ = _estimator_setup()
    sig = inputs.random_configs(64, mod.N, seed=22).astype(np.int64)
    eloc = el_all[exact.basis_index(sig)]
    g0 = vmc.vmc_gradient(mod, flat, sig, eloc)
    g1 = vmc.vmc_gradient(mod, flat, sig, eloc + 17.25)
    np.testing.assert_allclose(g1, g0, rtol=1e-10, atol=1e-12)
    raw = lambda e: vmc.logpsi_grad(mod, flat, sig, 2.0 * np.asarray(e) / len(e))
    assert np.abs(raw(eloc + 17.25) - raw(eloc)).max() > 1e-2


# ---------------------------------------------------- long-range TFIM ----
def _lmg_ground_energy(N, J, Gamma):
    """alpha = 0: sum_{i<j} Z_i Z_j = (M^2 - N) / 2 with M = sum Z = 2 S_z, so
    H = -J (4 S_z^2 - N) / 2 - 2 Gamma S_x (the Lipkin-Meshkov-Glick form); its
    ground state lies in the symmetric sector S = N/2, an (N + 1)-dimensional
    matrix in the S_z basis with S_x from the ladder operators."""
    S = N / 2.0
    m = np.arange(-S, S + 1.0)
    Hm = np.diag(-J * (4.0 * m * m - N) / 2.0)
    for k in range(len(m) - 1):
        x = 0.5 * np.sqrt(S * (S + 1) - m[k] * (m[k] + 1))      # <m+1|S_x|m>
        Hm[k, k + 1] = Hm[k + 1, k] = -2.0 * Gamma * x
    return np.linalg.eigvalsh(Hm)[0]


def test_lr_tfim_alpha_zero_matches_the_symmetric_sector():
    for N, G in ((6, 0.7), (9, 1.3)):
        e_ed, _ = exact.ground_state(exact.lr_tfim_hamiltonian(N, 0.0, 1.0, G))
        assert abs(e_ed - _lmg_ground_energy(N, 1.0, G)) < 1e-10


def test_lr_tfim_alpha_infinity_is_the_nearest_neighbour_chain():
    N, d = 9, 4
    mod = M.Model(M.GRU1D, N, d_h=d)
    flat = inputs.xavier_params(1, d, seed=23, noise_std=0.3)
    sig = inputs.random_configs(40, N, seed=24).astype(np.int64)
    a = hamiltonian.lr_tfim_local_energy(N, np.inf, 1.0, 0.8, sig, _lp_fn(mod, flat))
    b = hamiltonian.tfim_local_energy(N, 1.0, 0.8, sig, _lp_fn(mod, flat))
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-13)
    e_lr, _ = exact.ground_state(exact.lr_tfim_hamiltonian(8, np.inf, 1.0, 1.0))
    assert abs(e_lr - exact.tfim_free_fermion(8, 1.0, 1.0)) < 1e-10


def test_lr_tfim_classical_and_mean_field_limits():
    """Gamma = 0: the all-up state has E = -sum_{r>=1} (N - r) r^-alpha (pairs
    counted by distance); alpha = 0: E_loc = -(M^2 - N) / 2 for every sigma."""
    N = 11
    up = np.zeros((1, N), dtype=np.int64)
    for alpha in (0.1, 1.0, 2.5):
        e = hamiltonian.lr_tfim_local_energy(N, alpha, 1.0, 0.0, up, lambda s: np.zeros(len(s)))
        assert abs(e[0] + sum((N - r) * r ** -alpha for r in range(1, N))) < 1e-12
    sig = inputs.random_configs(30, N, seed=25).astype(np.int64)
    Mz = (1 - 2 * sig).sum(axis=1)
    e0 = hamiltonian.lr_tfim_local_energy(N, 0.0, 1.0, 0.0, sig, lambda s: np.zeros(len(s)))
    np.testing.assert_allclose(e0, -(Mz * Mz - N) / 2.0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("alpha", [0.1, 1.0, 3.0])
def test_lr_tfim_local_energy_is_constant_on_ground_state(alpha):
    N = 10
    e0, v = exact.ground_state(exact.lr_tfim_hamiltonian(N, alpha, 1.0, 1.0))
    table = np.log(np.abs(v))
    lp = lambda s: table[exact.basis_index(s)]
    el = hamiltonian.lr_tfim_local_energy(N, alpha, 1.0, 1.0, exact.all_configs(N), lp)
    np.testing.assert_allclose(el, e0, atol=1e-8)


def test_lr_tfim_energy_two_routes():
    N, d, alpha = 8, 5, 0.5
    mod = M.Model(M.GRU1D, N, d_h=d)
    flat = inputs.xavier_params(1, d, seed=26, noise_std=0.3)
    configs = exact.all_configs(N)
    lpsi = M.logpsi(mod, flat, configs)
    el = hamiltonian.lr_tfim_local_energy(N, alpha, 1.0, 1.0, configs, _lp_fn(mod, flat))
    psi = np.exp(lpsi)
    Hm = exact.lr_tfim_hamiltonian(N, alpha, 1.0, 1.0)
    assert abs(exact.exact_energy(np.exp(2 * lpsi), el) - psi @ (Hm @ psi)) < 1e-10
    assert exact.exact_energy(np.exp(2 * lpsi), el) >= exact.ground_state(Hm)[0]


# ------------------------------------------- cRNN and the cluster state ----
def test_cluster_hamiltonian_ground_energy_is_minus_n():
    """All N stabilisers commute and are independent, so the ground state is
    the unique joint +1 eigenstate with energy exactly -N, and the first
    excited level (one stabiliser at -1) is -N + 2."""
    for N in (3, 4, 7, 9):
        w = np.linalg.eigvalsh(exact.cluster_hamiltonian(N).toarray())
        assert abs(w[0] + N) < 1e-10 and abs(w[1] - (-N + 2)) < 1e-10


def test_cluster_local_energy_is_constant_on_ground_state():
    N = 8
    e0, v = exact.ground_state(exact.cluster_hamiltonian(N))
    nz = np.abs(v) > 1e-12
    la = np.where(nz, np.log(np.where(nz, np.abs(v), 1.0)), -np.inf)
    ph = np.where(v < 0, np.pi, 0.0)
    configs = exact.all_configs(N)[nz]
    el = hamiltonian.cluster_local_energy(N, configs, lambda s: la[exact.basis_index(s)],
                                          lambda s: ph[exact.basis_index(s)])
    np.testing.assert_allclose(el, e0, atol=1e-9)
    assert abs(e0 + N) < 1e-10
    assert (v < -1e-12).any()                   # the ground state has a sign structure


def _crnn(N, d, seed):
    mod = M.Model(M.GRU1D, N, d_h=d, phase=True)
    return mod, inputs.xavier_params(1, d, seed=seed, noise_std=0.4, phase=True)


def test_crnn_phase_range_and_normalisation():
    mod, flat = _crnn(7, 4, 30)
    configs = exact.all_configs(7)
    out = M.run(mod, flat, sigma=configs)
    assert abs(np.exp(2 * out["logpsi"]).sum() - 1.0) < 1e-12
    assert np.all(np.abs(out["phase"]) < 7 * np.pi)
    # phi_n of the spin that was not chosen does not enter phi
    zp = out["phase_logits"]
    phi = np.pi * M.softsign(zp[np.arange(len(configs))[:, None], np.arange(7)[None, :], configs]).sum(axis=1)
    np.testing.assert_allclose(out["phase"], phi, rtol=0, atol=1e-13)


def test_crnn_cluster_energy_two_routes():
    N, d = 7, 4
    mod, flat = _crnn(N, d, 31)
    configs = exact.all_configs(N)
    la, ph = M.logpsi(mod, flat, configs), M.phase(mod, flat, configs)
    el = hamiltonian.cluster_local_energy(N, configs, lambda s: M.logpsi(mod, flat, s),
                                          lambda s: M.phase(mod, flat, s))
    P = np.exp(2 * la)
    e_sum = np.sum(P * el)
    psi = np.exp(la + 1j * ph)
    e_h = np.vdot(psi, exact.cluster_hamiltonian(N) @ psi)
    assert abs(e_sum - e_h) < 1e-11 and abs(e_sum.imag) < 1e-11
    assert e_sum.real >= -N - 1e-12


def test_crnn_gradient_matches_fd_of_exact_energy():
    """d <psi|H|psi> / d theta for the cRNN on the cluster Hamiltonian (dense
    H, complex psi) = 2 sum P [Re(E_loc - E) d log|psi| + Im(E_loc - E) d phi]."""
    N, d = 5, 3
    mod, flat = _crnn(N, d, 32)
    configs = exact.all_configs(N)
    Hm = exact.cluster_hamiltonian(N).toarray()

    def energy(x):
        psi = np.exp(M.logpsi(mod, x, configs) + 1j * M.phase(mod, x, configs))
        return float(np.vdot(psi, Hm @ psi).real)

    P = np.exp(2 * M.logpsi(mod, flat, configs))
    el = hamiltonian.cluster_local_energy(N, configs, lambda s: M.logpsi(mod, flat, s),
                                          lambda s: M.phase(mod, flat, s))
    g = exact.exact_gradient(mod, flat, configs, P, el)
    fd = exact.central_fd(energy, flat, h=1e-5)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_crnn_phase_gradient_matches_fd():
    N, d = 6, 3
    mod, flat = _crnn(N, d, 33)
    sig = inputs.random_configs(5, N, seed=34).astype(np.int64)
    w = inputs.random_weights(5, seed=35)
    v = inputs.random_weights(5, seed=36)
    g = vmc.logpsi_grad(mod, flat, sig, w, phase_weights=v)
    fd = exact.central_fd(lambda x: float(w @ M.logpsi(mod, x, sig) + v @ M.phase(mod, x, sig)), flat)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)
