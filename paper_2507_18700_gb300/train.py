"""Adaptive training loop around the library's VMC step (Sec. II B, Sec. III,
Fig. 2 and the hyperparameter appendix, Tab. III).

A ``Trainer`` holds one model's parameters, its Adam moments and a device step
counter, and runs training steps entirely in library calls on the current
stream: sampling (Philox step read from the device counter), local energies,
the VMC gradient with its FP64 statistics, a per-step record of the
statistics, and the Adam update that advances the counter.  Because nothing in
a step depends on the host, ``capture(k)`` records k steps as one CUDA graph
and every ``replay()`` runs k fresh steps.  ``grow(d_h)`` embeds the model
into the next hidden size with ``nqs_grow_hidden`` and carries the moment
estimates over the same way with zero padding (the appendix carries both the
parameters and the momentum states to the new model).

The schedule helpers (fixed-interval growth, early stopping on the moving
average of the energy variance) are host bookkeeping between graph replays;
all arithmetic on device data runs in the library.
"""
import math

import torch

from . import nqs


class EarlyStopping:
    """Early-stopping rule of the appendix: the metric is the moving average of
    the energy variance over `window` steps; a step improves when the metric
    is below the best so far by more than delta = 10^(-log2(d_h) / 2); the
    rule triggers after `patience` consecutive steps without improvement.
    The metric is first formed once `window` values have been seen."""

    def __init__(self, d_h, window=500, patience=10000, delta=None):
        self.window, self.patience = int(window), int(patience)
        self.delta = 10.0 ** (-0.5 * math.log2(d_h)) if delta is None else float(delta)
        self.buf = []
        self.total = 0.0
        self.best = math.inf
        self.since = 0

    def update(self, variance):
        self.buf.append(float(variance))
        self.total += self.buf[-1]
        if len(self.buf) > self.window:
            self.total -= self.buf.pop(0)
        if len(self.buf) < self.window:
            return False
        metric = self.total / self.window
        if metric < self.best - self.delta:
            self.best = metric
            self.since = 0
        else:
            self.since += 1
        return self.since >= self.patience


class Trainer:
    """One model of the Adaptive sequence and its optimiser state on a device."""

    def __init__(self, desc, params, ham, B, seed=0, sched=None, adam=None, log_cap=4096, t0=0):
        self.dev = params.device
        self.ham, self.B, self.seed = ham, int(B), int(seed)
        self.sched = nqs.lr_constant(1e-3) if sched is None else sched
        self.adam = nqs.adam_desc() if adam is None else adam
        self.t = torch.full((1,), int(t0), dtype=torch.int64, device=self.dev)
        self.log = torch.zeros((int(log_cap), 4), dtype=torch.float64, device=self.dev)
        self.ws = nqs.Workspace(self.dev)
        self._set_model(desc, params.detach().clone(), torch.zeros_like(params), torch.zeros_like(params))

    def _set_model(self, desc, params, m, v):
        self.desc, self.params, self.m, self.v = desc, params, m, v
        N, d, B, dev = desc.N, desc.d_h, self.B, self.dev
        self.sigma = torch.empty((B, N), dtype=torch.uint8, device=dev)
        self.logpsi = torch.empty((B,), dtype=torch.float32, device=dev)
        self.hcache = torch.empty((B, N, d), dtype=torch.float32, device=dev)
        self.eloc = torch.empty((B,), dtype=torch.float32, device=dev)
        self.grad = torch.empty_like(params)
        self.stats = torch.empty((3,), dtype=torch.float64, device=dev)
        need = max(nqs.workspace_bytes(desc, B, nqs.OP_SAMPLE), nqs.workspace_bytes(desc, B, nqs.OP_VMC_GRAD),
                   nqs.workspace_bytes(desc, B, nqs.OP_LOCAL_ENERGY, self.ham))
        self.ws.get(need)                    # sized before any capture: no reallocation inside a graph
        self.graph = None

    def step(self):
        """One training step, enqueued on the current stream."""
        nqs.sample(self.desc, self.params, self.B, seed=self.seed, step_dev=self.t, hcache=self.hcache,
                   out=(self.sigma, self.logpsi), ws=self.ws)
        nqs.local_energy(self.desc, self.params, self.ham, self.sigma, self.hcache, ws=self.ws, out=self.eloc)
        nqs.vmc_grad(self.desc, self.params, self.sigma, self.hcache, self.eloc, ws=self.ws, grad=self.grad,
                     stats=self.stats)
        nqs.record_stats(self.stats, self.log, self.t)
        nqs.adam_step(self.params, self.m, self.v, self.grad, self.adam, self.sched, t_dev=self.t)

    def capture(self, k):
        """Record k steps as one CUDA graph (after one eager warm-up step on a
        side stream, which also settles the tile autotuner)."""
        side = torch.cuda.Stream(self.dev)
        side.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.stream(side):
            self.step()
        torch.cuda.current_stream(self.dev).wait_stream(side)
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(int(k)):
                self.step()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def history(self):
        """(t, mean E_loc, variance, M) of the logged steps, oldest first (host)."""
        rows = self.log.cpu()
        rows = rows[rows[:, 3] > 0]
        return rows[torch.argsort(rows[:, 0])]

    def steps_done(self):
        return int(self.t.item())

    def grow(self, d_new, seed=2, eps=1e-3):
        """Embed the model into hidden size d_new (Fig. 2(b)); the moments are
        embedded with zero padding."""
        big = nqs.model_desc(self.desc.cell, self.desc.Lx, self.desc.Ly, d_new, sz0=bool(self.desc.sz0),
                             precision=self.desc.precision)
        p = nqs.grow_hidden(self.desc, self.params, big, seed=seed, eps=eps)
        m = nqs.grow_hidden(self.desc, self.m, big, seed=seed, eps=0.0)
        v = nqs.grow_hidden(self.desc, self.v, big, seed=seed, eps=0.0)
        self._set_model(big, p, m, v)

    def evaluate(self, M=1_000_000, chunk=65536, seed=None, step=0):
        """Final evaluation of the current model (Tab. I): float64 [5]."""
        return nqs.evaluate(self.desc, self.params, self.ham, M, chunk=chunk,
                            seed=self.seed + 1 if seed is None else seed, step=step)


def fixed_interval_plan(d_start, d_final, total_steps):
    """Hidden sizes and step counts of the fixed-interval Adaptive schedule:
    d_h doubles from d_start to d_final with the steps split evenly (1D TFIM:
    2 -> 256 over 50,000 steps, every 6,250 steps)."""
    sizes = []
    d = d_start
    while d <= d_final:
        sizes.append(d)
        d *= 2
    per = total_steps // len(sizes)
    return [(d, per) for d in sizes]


def run_adaptive(trainer, plan, graph_steps=50, stopper=None, on_stage=None):
    """Train through `plan` [(d_h, steps), ...]: each stage runs its steps as
    graph replays of `graph_steps` steps (plus eager steps for the remainder)
    and grows to the next size.  With `stopper(d_h)` returning an
    EarlyStopping, a stage also ends when the rule triggers (checked after
    every replay from the logged variances)."""
    for si, (d, steps) in enumerate(plan):
        if trainer.desc.d_h != d:
            trainer.grow(d)
        rule = stopper(d) if stopper else None
        done = 0
        if steps >= graph_steps:
            trainer.capture(graph_steps)
            done = 1                                   # the capture's warm-up step
        stop = False
        while done + graph_steps <= steps and not stop:
            t_before = trainer.steps_done()
            trainer.replay()
            done += graph_steps
            if rule is not None:
                h = trainer.history()
                for row in h[h[:, 0] >= t_before]:
                    if rule.update(float(row[2])):
                        stop = True
                        break
        while done < steps and not stop:
            trainer.step()
            done += 1
        if on_stage is not None:
            on_stage(si, d, trainer)
    return trainer
