"""Data-parallel VMC step over ranks (one process per GPU).

Samples are independent, so each rank draws and evaluates its own batch with
the replicated weights.  The step has one real exchange (Sec. III): the
gradient weights w_b = 2 (E_loc,b - E_mean) / M need the mean energy and the
sample count over all ranks, and the gradient is the sum of the ranks' sums.
Both are all-reduces of small tensors; the kernels stay per rank.
"""
import torch
import torch.distributed as dist

from . import nqs


def _world(group):
    return dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1


def global_energy_stats(eloc, group=None):
    """[mean, variance, M] of the local energies of all ranks, in float64: one
    all-reduce of (sum E, sum E^2, M)."""
    e = eloc.double()
    s = torch.stack([e.sum(), (e * e).sum(), torch.tensor(float(e.numel()), dtype=torch.float64, device=e.device)])
    if _world(group) > 1:
        dist.all_reduce(s, group=group)
    M = s[2]
    mean = s[0] / M
    return torch.stack([mean, s[1] / M - mean * mean, M])


def vmc_weights(eloc, stats):
    """w_b = 2 (E_loc,b - mean) / M with the global statistics (float32)."""
    return (2.0 * (eloc.double() - stats[0]) / stats[2]).float()


def allreduce_grad(grad, group=None):
    """Sum the ranks' partial gradients in place."""
    if _world(group) > 1:
        dist.all_reduce(grad, group=group)
    return grad


def rank_seed(seed, group=None):
    """Sampling seed of this rank: distinct Philox streams per rank."""
    r = dist.get_rank(group) if _world(group) > 1 else 0
    return seed + 1000003 * r


def vmc_step(desc, params, ham, B, seed, step, ws=None, group=None):
    """One VMC step on this rank's B samples with the exchange above.
    Returns (grad, stats, sigma, eloc); grad and stats are global."""
    sigma, _, hc = nqs.sample(desc, params, B, seed=rank_seed(seed, group), step=step, ws=ws)
    eloc = nqs.local_energy(desc, params, ham, sigma, hc, ws=ws)
    stats = global_energy_stats(eloc, group)
    grad = nqs.logpsi_grad(desc, params, sigma, hc, vmc_weights(eloc, stats), ws=ws)
    return allreduce_grad(grad, group), stats, sigma, eloc
