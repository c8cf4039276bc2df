"""VMC step throughput of the RNN-wave-function hot path on GB300.

One step = autoregressive sampling of B configurations, local energies of all
of them (every Hamiltonian-connected configuration, prefix-cached) and the VMC
gradient with its energy statistics, on one set of weights.  Workload: the 1D
transverse-field Ising chain, N = 100, Gamma = J = 1, open boundaries; 1D GRU
wave function with d_h = 64; B = 4096 samples per step; Xavier-uniform weights
plus N(0, 0.1^2) noise from seed 1 (synthetic: the paper's trained weights are
not available and none are needed).

Prints one JSON line (rank 0).  ``--impl reference`` times the float64 CPU
oracle on the host cores instead (a bounded sample of each step).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_SITES, D_H, BATCH, GAMMA, J = 100, 64, 4096, 1.0, 1.0
METRIC = "VMC samples/sec/GPU (sample+E_loc+grad), BF16 vs FP32 at <=1e-4 energy/site"
WORKLOAD = "1D TFIM N=100 OBC, Gamma=J=1, GRU d_h=64, 4096 samples/step"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def flops_per_sample(N, d):
    """Algorithmic FLOPs of one sample's step: 2 * MAC_cell * (N + N(N-1)/2 + 2N),
    MAC_cell = 3 d^2 + 2 d (gate GEMMs on h and the readout)."""
    mac = 3 * d * d + 2 * d
    return 2 * mac * (N + N * (N - 1) // 2 + 2 * N)


def chain_flops(B, N, d):
    return 2 * (3 * d * d + 2 * d) * B * (N * (N - 1) // 2)


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def oracle_step_seconds(n_samples, seed):
    """Float64 oracle for n_samples of the workload: sampling, local energies by
    full re-evaluation, VMC gradient.  Returns seconds."""
    import numpy as np
    from oracle import hamiltonian as oh, model as om, philox, vmc as ov
    from paper_2507_18700_gb300 import inputs
    mod = om.Model(om.GRU1D, N_SITES, d_h=D_H)
    flat = inputs.xavier_params(1, D_H, seed=1, noise_std=0.1)
    t0 = time.perf_counter()
    u = philox.sampling_uniforms(seed, 0, n_samples, N_SITES)
    s = om.sample(mod, flat, u)["sigma"]
    e = oh.tfim_local_energy(N_SITES, J, GAMMA, s, lambda x: om.logpsi(mod, flat, x))
    ov.energy_stats(e)
    ov.vmc_gradient(mod, flat, s, e)
    return time.perf_counter() - t0


def cpu_baseline(target_s=12.0):
    n = 16
    t = oracle_step_seconds(n, seed=100)
    n2 = max(16, min(BATCH, int(n * target_s / max(t, 1e-3))))
    t2 = oracle_step_seconds(n2, seed=101)
    return {"value": n2 / t2, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d of the 4096 samples of one step (sampling, E_loc by full re-evaluation, "
                      "gradient), float64 numpy on all host cores" % n2,
            "seconds": t2}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 32
    oracle_step_seconds(8, seed=1)
    times = []
    for k in range(args.warmup + args.steps):
        dt = oracle_step_seconds(n, seed=200 + k)
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "samples_per_step_timed": n,
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "samples/s", "kind": "oracle",
                             "cores": os.cpu_count(),
                             "sample": "%d samples per step of the same workload" % n},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2507_18700_gb300 import inputs, nqs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    precision = nqs.FP32
    desc = nqs.model_desc(nqs.GRU1D, N_SITES, 1, D_H, precision=precision)
    ham = nqs.tfim(J, GAMMA)
    flat = inputs.xavier_params(1, D_H, seed=1, noise_std=0.1).astype(np.float32)
    params = torch.tensor(flat, device=dev)
    P = params.numel()
    ws = nqs.Workspace(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    st = torch.cuda.current_stream()
    step_seed = 1000 + rank

    def step(k, p):
        sigma, lp, hc = nqs.sample(desc, p, BATCH, seed=step_seed, step=k, ws=ws)
        eloc = nqs.local_energy(desc, p, ham, sigma, hc, ws=ws)
        grad, stats = nqs.vmc_grad(desc, p, sigma, hc, eloc, ws=ws)
        return grad, stats, eloc

    def loc_events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    for k in range(args.warmup):
        step(k, params)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    step_ms, le_ms = [], []
    for k in range(args.steps):
        flush.zero_()
        a, b = loc_events()
        la, lb = loc_events()
        torch.cuda.synchronize()
        a.record(st)
        sigma, lp, hc = nqs.sample(desc, params, BATCH, seed=step_seed, step=args.warmup + k, ws=ws)
        la.record(st)
        eloc = nqs.local_energy(desc, params, ham, sigma, hc, ws=ws)
        lb.record(st)
        grad, stats = nqs.vmc_grad(desc, params, sigma, hc, eloc, ws=ws)
        b.record(st)
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
        le_ms.append(la.elapsed_time(lb))
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    energy_per_site = float(stats[0].item()) / N_SITES

    # end to end through the public API with host buffers: params in, grad + stats out
    host_p = torch.from_numpy(flat).pin_memory()
    host_g = torch.empty(P, dtype=torch.float32).pin_memory()
    host_s = torch.empty(3, dtype=torch.float64).pin_memory()
    dev_p = torch.empty_like(params)
    e2e_ms = []
    for k in range(args.steps):
        flush.zero_()
        a, b = loc_events()
        torch.cuda.synchronize()
        a.record(st)
        dev_p.copy_(host_p, non_blocking=True)
        g, s, _ = step(10_000 + k, dev_p)
        host_g.copy_(g, non_blocking=True)
        host_s.copy_(s, non_blocking=True)
        b.record(st)
        torch.cuda.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_total = sum(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_total], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())

    pk, src = peaks()
    alu_peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12   # FP32 FMA TFLOP/s
    le_avg = sum(le_ms) / len(le_ms)
    achieved = chain_flops(BATCH, N_SITES, D_H) / (le_avg * 1e-3) / 1e12
    value = world * BATCH * args.steps / (total_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": BATCH * world, "seq_len": N_SITES,
                   "parallelism": "replicas" if world > 1 else "single", "precision": "fp32",
                   "l2": "flushed (256 MB write) before every timed step",
                   "energy_per_site": energy_per_site},
        "roofline": {"bound": "alu", "kernel": "nqs_local_energy (prefix-cached chains)",
                     "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": None,
                     "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x %s MHz (%s)"
                                    % (pk.get("sm_max_mhz", 2070.0), src)},
        "e2e": {"value": world * BATCH * args.steps / (e2e_total * 1e-3), "unit": "samples/s",
                "h2d_bytes_per_step": P * 4, "d2h_bytes_per_step": P * 4 + 24},
        "gpu_launches": 11 * args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
