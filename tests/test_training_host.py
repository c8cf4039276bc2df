"""Host-side pieces of the training loop, on the CPU: the float64 Adam of the
oracle against closed forms, the learning-rate schedules against values
computed by hand from Tab. III, and the product's early-stopping rule against
the oracle's on synthetic variance sequences (plus a case whose trigger step
is known by hand)."""
import numpy as np

from oracle import adam as oa
from paper_2507_18700_gb300 import inputs
from paper_2507_18700_gb300.train import EarlyStopping, fixed_interval_plan


def test_adam_first_step_is_lr_times_sign():
    """After one update m_hat = g and v_hat = g^2 exactly, so the step is
    lr g / (|g| + eps)."""
    x0 = inputs.random_weights(50, seed=1)
    g = inputs.random_weights(50, seed=2, scale=3.0)
    x1, m, v = oa.adam(x0, [g], oa.lr_constant(1e-2), eps=1e-8)
    np.testing.assert_allclose(x1, x0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_adam_constant_gradient_moves_lr_per_step():
    """With the same gradient every step the bias-corrected moments equal g
    and g^2 exactly, so each of k steps moves by lr g / (|g| + eps)."""
    x0 = inputs.random_weights(20, seed=3)
    g = inputs.random_weights(20, seed=4)
    k = 7
    xk, _, _ = oa.adam(x0, [g] * k, oa.lr_constant(3e-3), eps=1e-8)
    np.testing.assert_allclose(xk, x0 - k * 3e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-13)


def test_schedules_of_table_iii():
    step = oa.lr_step(5e-3, 5e-4, 25_000)            # 1D TFIM Adaptive
    assert step(0) == 5e-3 and step(24_999) == 5e-3 and step(25_000) == 5e-4
    inv = oa.lr_inverse(5e-4, 5000.0)                # 2D Heisenberg Static
    assert inv(0) == 5e-4 and abs(inv(5000) - 2.5e-4) < 1e-18 and abs(inv(15000) - 1.25e-4) < 1e-18
    adp = oa.lr_inverse(5e-4, 5000.0, 100_000)       # 2D Heisenberg Adaptive (reading of the garbled formula)
    assert adp(99_999) == 5e-4 and adp(100_000) == 5e-4 and abs(adp(105_000) - 2.5e-4) < 1e-18


def test_early_stopping_hand_case():
    """window 3, patience 2, delta 0.5: variances 10, 10, 10 (metric 10, best),
    then 10 (metric 10, no improvement: 1), 1 (metric 7, improvement), 10
    (metric 7, 1), 10 (metric 7, 2: trigger) -> triggers at the 7th value."""
    for rule in (EarlyStopping(4, window=3, patience=2, delta=0.5),
                 oa.EarlyStopping(4, window=3, patience=2, delta=0.5)):
        out = [rule.update(x) for x in (10, 10, 10, 10, 1, 10, 10)]
        assert out == [False] * 6 + [True]


def test_early_stopping_matches_oracle_and_delta_rule():
    rng = np.random.default_rng(5)
    for d in (2, 16, 256):
        a, b = EarlyStopping(d, window=50, patience=80), oa.EarlyStopping(d, window=50, patience=80)
        assert abs(a.delta - 10.0 ** (-0.5 * np.log2(d))) < 1e-15 and a.delta == b.delta
        seq = np.exp(-np.arange(2000) / 300.0) * 5 + rng.exponential(0.2, 2000)
        ta = [a.update(x) for x in seq]
        tb = [b.update(x) for x in seq]
        assert ta == tb


def test_fixed_interval_plan():
    assert fixed_interval_plan(2, 256, 50_000) == [(2 ** k, 6250) for k in range(1, 9)]
