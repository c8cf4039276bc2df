"""Adam and the learning-rate schedules of the training loop (test infrastructure).

The paper trains every model with Adam (Sec. III and its hyperparameter
appendix, citing Kingma and Ba 2014) and carries the optimiser's moment
estimates over to the larger model at every growth step.  This module writes
Adam's update (Kingma and Ba, Algorithm 1) in float64 and the schedules of
Tab. III:

* 1D TFIM Adaptive: 5e-3 for the first 25,000 steps, then 5e-4 (a step);
* 2D Heisenberg Static: 5e-4 / (1 + t / 5000) (an inverse decay);
* 2D Heisenberg Adaptive: the table's formula is garbled; it is read as
  5e-4 for t < 100,000 and 5e-4 / (1 + (t - 100,000) / 5000) afterwards (the
  floor term switches the decay on for the second half of training).

Early stopping (the hyperparameter appendix): the monitored metric is the
moving average of the energy variance over a window of 500 steps; a step
improves when the metric falls below the best value so far minus
delta = 10^(-log2(d_h) / 2); training of a model stops after `patience`
(10,000) consecutive steps without improvement.
"""
import numpy as np


def lr_constant(lr0):
    return lambda t: lr0


def lr_step(lr0, lr1, t_switch):
    return lambda t: lr0 if t < t_switch else lr1


def lr_inverse(lr0, decay, t_switch=0):
    return lambda t: lr0 if t < t_switch else lr0 / (1.0 + (t - t_switch) / decay)


def adam(params, grads, lr_fn, beta1=0.9, beta2=0.999, eps=1e-8, m=None, v=None, t0=0):
    """Apply Adam to `params` for the gradients in `grads` (one per step, the
    step numbers t0, t0 + 1, ...).  Returns (params, m, v) in float64."""
    x = np.asarray(params, dtype=np.float64).copy()
    m = np.zeros_like(x) if m is None else np.asarray(m, dtype=np.float64).copy()
    v = np.zeros_like(x) if v is None else np.asarray(v, dtype=np.float64).copy()
    for i, g in enumerate(grads):
        t = t0 + i                       # 0-based training step
        k = t + 1                        # Algorithm 1 counts updates from 1
        g = np.asarray(g, dtype=np.float64)
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        m_hat = m / (1.0 - beta1 ** k)
        v_hat = v / (1.0 - beta2 ** k)
        x = x - lr_fn(t) * m_hat / (np.sqrt(v_hat) + eps)
    return x, m, v


class EarlyStopping:
    """Moving average of the energy variance over `window` steps; a step
    improves when it is below the best average so far by more than `delta`;
    `triggered` after `patience` consecutive steps without improvement."""

    def __init__(self, d_h, window=500, patience=10000, delta=None):
        self.window = window
        self.patience = patience
        self.delta = 10.0 ** (-0.5 * np.log2(d_h)) if delta is None else delta
        self.values = []
        self.best = np.inf
        self.since = 0

    def update(self, variance):
        self.values.append(float(variance))
        if len(self.values) < self.window:
            return False
        metric = float(np.mean(self.values[-self.window:]))
        if metric < self.best - self.delta:
            self.best = metric
            self.since = 0
        else:
            self.since += 1
        return self.since >= self.patience
