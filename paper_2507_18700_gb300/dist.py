"""Data-parallel VMC step over ranks (one process per GPU).

Samples are independent (Sec. III), so each rank draws and evaluates its own
share of the batch with the replicated weights.  Rank r draws the samples
with global indices r*B .. r*B + B - 1 of one Philox stream (the library's
sample offset), so the union over ranks is bitwise the batch one rank would
draw and the result does not depend on the rank count.  The step has one real
exchange: the gradient weights w_b = 2 (E_loc,b - mean) / M need the energy
sums of all ranks, and the gradient is the sum of the ranks' shares.  All of
the arithmetic runs in the library (nqs_energy_sums, nqs_vmc_grad_global);
this module only moves buffers through all-reduces.
"""
import torch.distributed as dist

from . import nqs


def _world(group):
    return dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1


def _rank(group):
    return dist.get_rank(group) if _world(group) > 1 else 0


def allreduce(t, group=None):
    """Sum a library-filled buffer over ranks, in place (no-op on one rank)."""
    if _world(group) > 1:
        dist.all_reduce(t, group=group)
    return t


def sample_offset(B, group=None):
    """Global index of this rank's first sample when every rank draws B."""
    return _rank(group) * B


def global_gradient(desc, params, sigma, hcache, eloc, ws=None, group=None, api=nqs):
    """(grad float64 [P], stats float64 [3]) of all ranks' samples: the energy
    sums are all-reduced, the library forms the centred weights and this
    rank's gradient share, and the shares are all-reduced."""
    sums = allreduce(api.energy_sums(eloc), group)
    grad, stats = api.vmc_grad_global(desc, params, sigma, hcache, eloc, sums, ws=ws)
    return allreduce(grad, group), stats


def vmc_step(desc, params, ham, B, seed, step, ws=None, group=None, api=nqs):
    """One VMC step on this rank's B samples (every rank passes the same B,
    seed and step).  Returns (grad, stats, sigma, eloc); grad and stats are
    global."""
    sigma, _, hc = api.sample(desc, params, B, seed=seed, step=step, ws=ws,
                              sample_offset=sample_offset(B, group))
    eloc = api.local_energy(desc, params, ham, sigma, hc, ws=ws)
    grad, stats = global_gradient(desc, params, sigma, hc, eloc, ws=ws, group=group, api=api)
    return grad, stats, sigma, eloc
