"""VMC step throughput of the RNN-wave-function hot path on GB300.

One step = autoregressive sampling of B configurations, local energies of all
of them (every Hamiltonian-connected configuration, prefix-cached) and the VMC
gradient with its energy statistics, on one set of weights.

Default workload (--workload tfim100): the 1D transverse-field Ising chain,
N = 100, Gamma = J = 1, open boundaries; 1D GRU wave function with d_h = 64;
B = 4096 samples per step; Xavier-uniform weights plus N(0, 0.1^2) noise from
seed 1.  --workload heis8x8: the Marshall-rotated Heisenberg model on the open
8 x 8 lattice with the zero-magnetisation mask, 2D GRU + GLU with d_h = 64,
B = 2048, Xavier-uniform weights from seed 0.  Inputs are synthetic (the
paper's trained weights are not available and none are needed).

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

METRIC = "VMC samples/sec/GPU (sample+E_loc+grad), BF16 vs FP32 at <=1e-4 energy/site"

WORKLOADS = {
    "tfim100": dict(cell=1, Lx=100, Ly=1, d=64, B=4096, sz0=False, ham="tfim", J=1.0, Gamma=1.0,
                    seed=1, noise=0.1,
                    name="1D TFIM N=100 OBC, Gamma=J=1, GRU d_h=64, 4096 samples/step"),
    "heis8x8": dict(cell=2, Lx=8, Ly=8, d=64, B=2048, sz0=True, ham="heis", J=1.0, Gamma=0.0,
                    seed=0, noise=0.0,
                    name="2D Heisenberg 8x8 OBC, Marshall sign, S_z=0, 2D GRU+GLU d_h=64, 2048 samples/step"),
    "heis16x16": dict(cell=2, Lx=16, Ly=16, d=256, B=8192, sz0=True, ham="heis", J=1.0, Gamma=0.0,
                      seed=3, noise=0.0,
                      name="2D Heisenberg 16x16 OBC, Marshall sign, S_z=0, 2D GRU+GLU d_h=256, 8192 samples/step"),
    "cluster64": dict(cell=1, Lx=64, Ly=1, d=128, B=4096, sz0=False, ham="cluster", J=1.0, Gamma=0.0,
                      seed=4, noise=0.0, phase=True,
                      name="1D cluster state N=64 (Sec. III D), cRNN (GRU d_h=128 + softsign phase layer), "
                           "4096 samples/step, FP32"),
    "eval1m": dict(cell=1, Lx=100, Ly=1, d=64, B=1_000_000, sz0=False, ham="tfim", J=1.0, Gamma=1.0,
                   seed=1, noise=0.1, chunk=65536,
                   name="final evaluation: 1D TFIM N=100, Gamma=J=1, GRU d_h=64, 10^6 samples in chunks of 65,536 "
                        "(sampling + E_loc, FP64 statistics)"),
    "replicas16": dict(cell=1, Lx=100, Ly=1, d=None, B=2048, sz0=False, ham="tfim", J=1.0, Gamma=None,
                       seed=10, noise=0.0, fields=(0.5, 1.0, 1.5, 2.0), sizes=(16, 32, 64, 128),
                       name="16 replicas: 1D TFIM N=100, Gamma in {0.5,1,1.5,2} x GRU d_h in {16,32,64,128} "
                            "grown from d_h=16 (seed 2, eps 1e-3), 2048 samples each, one batched step, CUDA graph"),
}


def mac_cell(w):
    d = w["d"]
    if w["cell"] == 1:
        return 3 * d * d + 2 * d + (2 * d if w.get("phase") else 0)   # cRNN: the phase layer
    return 8 * d * d + 2 * d


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def chain_cells(w, sigma):
    """Cells recomputed by the prefix-cached local energy for configurations sigma
    (numpy [B, N]): N(N-1)/2 per sample for the TFIM; for the Heisenberg model
    N-1-pos(a) per antiparallel bond (a, b), pos(a) < pos(b)."""
    import numpy as np
    B, N = sigma.shape
    if w["ham"] == "tfim":
        return B * (N * (N - 1) // 2)
    if w["ham"] == "cluster":
        # term k restarts at its first flipped site f: 1 (k = 0), k - 1, N - 2 (k = N - 1)
        firsts = [1] + list(range(0, N - 2)) + [N - 2]
        return B * sum(N - 1 - f for f in firsts)
    Lx, Ly = w["Lx"], w["Ly"]
    pos = np.empty(N, dtype=np.int64)
    for j in range(Ly):
        for i in range(Lx):
            pos[j * Lx + i] = j * Lx + (i if j % 2 == 0 else Lx - 1 - i)
    total = 0
    for j in range(Ly):
        for i in range(Lx):
            k = j * Lx + i
            for q in ([k + 1] if i + 1 < Lx else []) + ([k + Lx] if j + 1 < Ly else []):
                anti = sigma[:, k] != sigma[:, q]
                total += int(anti.sum()) * (N - 1 - min(pos[k], pos[q]))
    return total


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


def _oracle_model(w):
    from oracle import model as om
    from paper_2507_18700_gb300 import inputs
    mod = om.Model(w["cell"], w["Lx"], w["Ly"], d_h=w["d"], sz0=w["sz0"], phase=w.get("phase", False))
    flat = inputs.xavier_params(w["cell"], w["d"], seed=w["seed"], noise_std=w["noise"], phase=w.get("phase", False))
    return mod, flat


def oracle_step_seconds(w, n_samples, seed):
    """Float64 oracle for n_samples of the workload: sampling, local energies by
    full re-evaluation, VMC gradient.  Returns seconds."""
    from oracle import hamiltonian as oh, model as om, philox, vmc as ov
    mod, flat = _oracle_model(w)
    t0 = time.perf_counter()
    u = philox.sampling_uniforms(seed, 0, n_samples, mod.N)
    s = om.sample(mod, flat, u)["sigma"]
    lp = lambda x: om.logpsi(mod, flat, x)
    if w["ham"] == "tfim":
        e = oh.tfim_local_energy(mod.N, w["J"], w["Gamma"], s, lp)
    elif w["ham"] == "cluster":
        e = w["J"] * oh.cluster_local_energy(mod.N, s, lp, lambda x: om.phase(mod, flat, x))
    else:
        e = oh.heisenberg_local_energy(w["Lx"], w["Ly"], w["J"], True, s, lp)
    ov.energy_stats(e)
    ov.vmc_gradient(mod, flat, s, e)
    return time.perf_counter() - t0


def _single_thread_blas():
    """Pool initializer: one BLAS thread per worker (set before numpy loads)."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_share(job):
    w, n, seed = job
    return oracle_step_seconds(w, n, seed), n


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def cpu_baseline(w, target_s=8.0):
    """The float64 oracle on the host: single-threaded, and one single-threaded
    worker process per core (spawned, so no process is forked after the GPU
    calls) on disjoint samples; throughput = samples / the slowest worker's
    time (worker start-up excluded)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    cores = os.cpu_count() or 1
    with ctx.Pool(1, initializer=_single_thread_blas) as pool:
        t, _ = pool.apply(_oracle_share, ((w, 4, 100),))
        n1 = max(4, min(w["B"], int(4 * target_s / max(t, 1e-3))))
        t1, _ = pool.apply(_oracle_share, ((w, n1, 101),))
    single = n1 / t1
    per = max(2, min(max(1, w["B"] // cores), int(single * target_s)))
    with ctx.Pool(cores, initializer=_single_thread_blas) as pool:
        res = pool.map(_oracle_share, [(w, per, 200 + i) for i in range(cores)])
    slowest = max(r[0] for r in res)
    return {"value": per * cores / slowest, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "single_thread": single, "cpu_model": cpu_model(),
            "sample": "one single-threaded worker per core on %d samples each (%d of the %d samples of a step "
                      "in all; sampling, E_loc by full re-evaluation, gradient; float64 numpy); single thread: "
                      "%d samples" % (per, per * cores, w["B"], n1),
            "seconds": slowest}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 32 if w["cell"] == 1 else 8
    oracle_step_seconds(w, 4, seed=1)
    times = []
    for k in range(args.warmup + args.steps):
        dt = oracle_step_seconds(w, n, seed=200 + k)
        if k >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = n * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "samples_per_step_timed": n,
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "samples/s", "kind": "oracle",
                             "cores": os.cpu_count(),
                             "sample": "%d samples per step of the same workload" % n},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_gpu(args, w):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2507_18700_gb300 import dist as vdist, inputs, nqs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    B = args.batch or w["B"]
    N = w["Lx"] * w["Ly"]
    phase = w.get("phase", False)
    ham = (nqs.tfim(w["J"], w["Gamma"]) if w["ham"] == "tfim" else
           nqs.cluster(w["J"]) if w["ham"] == "cluster" else nqs.heisenberg(w["J"], True))
    flat = inputs.xavier_params(w["cell"], w["d"], seed=w["seed"], noise_std=w["noise"],
                                phase=phase).astype(np.float32)
    params = torch.tensor(flat, device=dev)
    P = params.numel()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    st = torch.cuda.current_stream()
    step_seed = 1000          # one Philox stream; rank r draws global samples r*B .. r*B + B - 1
    offset = vdist.sample_offset(B)

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def vmc_grad(desc, sigma, hc, eloc, ws, p=None):
        """The step's gradient: one rank, nqs_vmc_grad; several ranks, the
        library's energy sums and gradient share with an all-reduce of each
        (3 and P doubles, inside the timed step)."""
        p = params if p is None else p
        if world == 1:
            return nqs.vmc_grad(desc, p, sigma, hc, eloc, ws=ws)
        return vdist.global_gradient(desc, p, sigma, hc, eloc, ws=ws)

    def measure(precision):
        """Time args.steps VMC steps at one precision (after args.warmup untimed ones)."""
        desc = nqs.model_desc(w["cell"], w["Lx"], w["Ly"], w["d"], sz0=w["sz0"], precision=precision, phase=phase)
        ws = nqs.Workspace(dev)
        for k in range(args.warmup):
            s_, _, h_ = nqs.sample(desc, params, B, seed=step_seed, step=k, ws=ws, sample_offset=offset)
            e_ = nqs.local_energy(desc, params, ham, s_, h_, ws=ws)
            vmc_grad(desc, s_, h_, e_, ws)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        step_ms, le_ms, cells = [], [], []
        for k in range(args.steps):
            flush.zero_()
            a, b = events()
            la, lb = events()
            torch.cuda.synchronize()
            a.record(st)
            sigma, lp, hc = nqs.sample(desc, params, B, seed=step_seed, step=args.warmup + k, ws=ws,
                                         sample_offset=offset)
            la.record(st)
            eloc = nqs.local_energy(desc, params, ham, sigma, hc, ws=ws)
            lb.record(st)
            grad, stats = vmc_grad(desc, sigma, hc, eloc, ws)
            b.record(st)
            torch.cuda.synchronize()
            step_ms.append(a.elapsed_time(b))
            le_ms.append(la.elapsed_time(lb))
            cells.append(chain_cells(w, sigma.cpu().numpy()))
        clk = clocks.stop()
        total_ms = sum(step_ms)
        if world > 1:
            t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        # end to end through the public API with host buffers: params in, grad + stats out
        host_p = torch.from_numpy(flat).pin_memory()
        gdt = torch.float32 if world == 1 else torch.float64    # several ranks: the FP64 all-reduced gradient
        host_g = torch.empty(P, dtype=gdt).pin_memory()
        host_s = torch.empty(4 if phase else 3, dtype=torch.float64).pin_memory()
        dev_p = torch.empty_like(params)
        e2e_ms = []
        for k in range(args.steps):
            flush.zero_()
            a, b = events()
            torch.cuda.synchronize()
            a.record(st)
            dev_p.copy_(host_p, non_blocking=True)
            s_, _, h_ = nqs.sample(desc, dev_p, B, seed=step_seed, step=10_000 + k, ws=ws, sample_offset=offset)
            e_ = nqs.local_energy(desc, dev_p, ham, s_, h_, ws=ws)
            g_, st_ = vmc_grad(desc, s_, h_, e_, ws, dev_p)
            host_g.copy_(g_, non_blocking=True)
            host_s.copy_(st_, non_blocking=True)
            b.record(st)
            torch.cuda.synchronize()
            e2e_ms.append(a.elapsed_time(b))
        e2e_total = sum(e2e_ms)
        if world > 1:
            t = torch.tensor([e2e_total], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_total = float(t.item())
        return dict(desc=desc, ws=ws, total_ms=total_ms, le_ms=le_ms, cells=cells, clk=clk,
                    e2e_ms=e2e_total, energy_per_site=float(stats[0].item()) / N, status=ws.status())

    def accuracy_check(d16, d32):
        """BF16 against FP32 on the same configurations: energy per site and gradient cosine."""
        sigma, _, _ = nqs.sample(d32, params, B, seed=77, step=0)
        out = {}
        for name, desc in (("bf16", d16), ("fp32", d32)):
            _, hc = nqs.logpsi(desc, params, sigma)
            el = nqs.local_energy(desc, params, ham, sigma, hc)
            g, stt = nqs.vmc_grad(desc, params, sigma, hc, el)
            out[name] = (float(stt[0].item()) / N, g.double())
        cos = float((out["bf16"][1] @ out["fp32"][1]) /
                    (out["bf16"][1].norm() * out["fp32"][1].norm()))
        de = abs(out["bf16"][0] - out["fp32"][0])
        return {"energy_per_site_diff": de, "grad_cosine": cos, "pass": bool(de <= 1e-4 and cos >= 0.999)}

    r32 = measure(nqs.FP32)
    chosen, r16, check = r32, None, None
    bf16_ok = args.precision != "fp32" and not phase and (w["d"] in (16, 32, 64, 128) if w["cell"] == 1
                                                          else (w["d"] in (32, 64) and N <= 256)
                                                          or (w["d"] == 256 and N <= 256))
    if bf16_ok:
        r16 = measure(nqs.BF16)
        check = accuracy_check(r16["desc"], r32["desc"])
        if check["pass"] or args.precision == "bf16":
            chosen = r16
    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    flop_per_cell = 2 * mac_cell(w)
    achieved = sum(chosen["cells"]) * flop_per_cell / (sum(chosen["le_ms"]) * 1e-3) / 1e12
    if chosen is r16:
        peak = pk.get("bf16_tflops", 1887.4)
        d = w["d"]
        mufu = sum(chosen["cells"]) * 3 * d / (sum(chosen["le_ms"]) * 1e-3) / 1e12
        mufu_peak = 152 * 16 * sm_mhz * 1e6 / 1e12
        # DRAM bytes of one chain launch, from an ncu capture of the 1D chain
        # kernel as it stands at B = 1024 (dram__bytes_read.sum 26,536,448,
        # write 0: the prefix cache read once), scaled by B (traffic grows
        # with B)
        traffic = (26536448 * B / 1024.0) if (w["cell"] == 1 and w["d"] == 64 and N == 100) else None
        roof = {"bound": "tensor",
                "kernel": "nqs_local_energy (prefix-cached %s chains, tcgen05 BF16)"
                          % ("TFIM" if w["cell"] == 1 else "Heisenberg"),
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": "bf16_tflops (burst) of measured peaks (%s)" % src,
                "epilogue_sfu": {"achieved": mufu, "peak": mufu_peak, "unit": "Tops/s",
                                 "frac": mufu / mufu_peak,
                                 "note": "3 MUFU ops (hardware tanh) per hidden unit per cell (two sigmoids, one tanh); "
                                         "SFU peak 16/clk/SM x 152 SMs x max SM clock"}}
    else:
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": "nqs_local_energy (prefix-cached chains, FP32 CUDA cores)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x %s MHz (%s)" % (sm_mhz, src)}
    value = world * B * args.steps / (chosen["total_ms"] * 1e-3)
    # kernels of one step (memsets excluded): 1D FP32 sample 2, E_loc 4, gradient 5;
    # 1D BF16 sample 3, E_loc 5, gradient 9 (statistics, weights, three packs,
    # tape, sweep, two reductions); 2D FP32 sample 2, E_loc 5, gradient 5;
    # 2D BF16 sample 2, E_loc 7 (pack, bonds, cached-path tables, job count,
    # jobs, chains, energies), gradient 8 (statistics, weights, pack, tape,
    # sweep, weight gradients, readout gradient, reduction); 2D BF16 at d_h =
    # 256: E_loc 8 (the tables' up-spin prefix counts as one more), gradient 11
    # (statistics, weights, two packs, up-spin prefix, tape, sweep, weight
    # gradients, readout gradients, final reduction, conversion)
    wide = w["cell"] == 2 and w["d"] == 256
    if w["cell"] == 1:
        launches = 17 if chosen is r16 else 11
    else:
        launches = (21 if wide else 17) if chosen is r16 else 12
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": chosen["total_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if chosen is r16 else "f32",
        "data": "synthetic",
        "config": {"workload": w["name"], "global_batch": B * world, "seq_len": N,
                   "parallelism": "dp%d (samples split over ranks; all-reduce of energy statistics and gradient)"
                                  % world if world > 1 else "single",
                   "precision": ("bf16 tensor-core cell GEMMs, fp32 state" if w["cell"] == 1 else
                                 "bf16 tensor-core cell and GLU GEMMs (states as bf16 hi+lo pairs, weights "
                                 "streamed from L2 through a shared-memory ring) and reverse sweep, fp32 state"
                                 if wide else
                                 "bf16 tensor-core cell and GLU GEMMs (states as bf16 hi+lo pairs) "
                                 "and reverse sweep, fp32 state") if chosen is r16 else "fp32",
                   "fp32_value": world * B * args.steps / (r32["total_ms"] * 1e-3),
                   "fp32_ms_per_step": r32["total_ms"] / args.steps,
                   "bf16_check": check,
                   "l2": "flushed (256 MB write) before every timed step",
                   "energy_per_site": chosen["energy_per_site"],
                   "chain_cells_per_step": sum(chosen["cells"]) / len(chosen["cells"]),
                   "device_status": chosen["status"]},
        "roofline": roof,
        "e2e": {"value": world * B * args.steps / (chosen["e2e_ms"] * 1e-3), "unit": "samples/s",
                "h2d_bytes_per_step": P * 4,
                "d2h_bytes_per_step": P * (4 if world == 1 else 8) + (32 if phase else 24)},
        "gpu_launches": launches * args.steps,
        "clocks": {"sm_mhz": chosen["clk"]["sm_mhz"], "sm_max_mhz": chosen["clk"]["sm_max_mhz"],
                   "reasons": chosen["clk"]["reasons"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def replica_models(w, dev, precision=None):
    """The growth family: for each field a Xavier d_h = 16 model, embedded into
    d_h = 32, 64, 128 by nqs_grow_hidden (seed 2, eps 1e-3)."""
    import numpy as np
    import torch
    from paper_2507_18700_gb300 import inputs, nqs
    precision = nqs.FP32 if precision is None else precision
    models = []
    for fi, G in enumerate(w["fields"]):
        small = nqs.model_desc(nqs.GRU1D, w["Lx"], 1, w["sizes"][0])
        p = torch.tensor(inputs.xavier_params(1, w["sizes"][0], seed=w["seed"] + fi).astype(np.float32), device=dev)
        for si, d in enumerate(w["sizes"]):
            desc = nqs.model_desc(nqs.GRU1D, w["Lx"], 1, d)
            if si > 0:
                p = nqs.grow_hidden(small, p, desc, seed=2, eps=1e-3)
            models.append((nqs.model_desc(nqs.GRU1D, w["Lx"], 1, d, precision=precision), nqs.tfim(w["J"], G),
                           w["B"], 5000 + 16 * fi + si, p))
            small = desc
    return models


def oracle_replicas_seconds(w, per_replica, seed):
    """Float64 oracle: per_replica samples of each of the 16 replicas (no growth: Xavier weights)."""
    from oracle import hamiltonian as oh, model as om, philox, vmc as ov
    from paper_2507_18700_gb300 import inputs
    t0 = time.perf_counter()
    for fi, G in enumerate(w["fields"]):
        for d in w["sizes"]:
            mod = om.Model(om.GRU1D, w["Lx"], d_h=d)
            flat = inputs.xavier_params(1, d, seed=w["seed"] + fi)
            s = om.sample(mod, flat, philox.sampling_uniforms(seed, 0, per_replica, mod.N))["sigma"]
            e = oh.tfim_local_energy(mod.N, w["J"], G, s, lambda x: om.logpsi(mod, flat, x))
            ov.vmc_gradient(mod, flat, s, e)
    return time.perf_counter() - t0


def run_replicas(args, w):
    import torch
    from paper_2507_18700_gb300 import nqs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def events():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def measure(models):
        """(1) the batched step captured in a CUDA graph with the device step
        counter, (2) the same step without the graph, (3) 3 x R separate calls,
        (4) end to end: parameters in from pinned host memory, gradients and
        statistics out."""
        batch = nqs.ReplicaBatch(models, device_step=True)
        side = torch.cuda.Stream()
        side.wait_stream(st)
        with torch.cuda.stream(side):
            for _ in range(args.warmup):
                batch.step()
        st.wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            batch.step()
        graph.replay()
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        g_ms = []
        for k in range(args.steps):
            flush.zero_()
            a, b = events()
            torch.cuda.synchronize()
            a.record(st)
            graph.replay()
            b.record(st)
            torch.cuda.synchronize()
            g_ms.append(a.elapsed_time(b))
        clk = clocks.stop()
        e_ms, s_ms = [], []
        ws = nqs.Workspace(dev)
        for k in range(args.steps):
            flush.zero_()
            a, b = events()
            torch.cuda.synchronize()
            a.record(st)
            batch.step()
            b.record(st)
            torch.cuda.synchronize()
            e_ms.append(a.elapsed_time(b))
            flush.zero_()
            a, b = events()
            torch.cuda.synchronize()
            a.record(st)
            for (desc, ham, B, seed, p) in models:
                sg, _, hc = nqs.sample(desc, p, B, seed=seed, step=k, ws=ws)
                el = nqs.local_energy(desc, p, ham, sg, hc, ws=ws)
                nqs.vmc_grad(desc, p, sg, hc, el, ws=ws)
            b.record(st)
            torch.cuda.synchronize()
            s_ms.append(a.elapsed_time(b))
        host_p = [m[4].cpu().pin_memory() for m in models]
        host_g = [torch.empty_like(h).pin_memory() for h in host_p]
        host_s = [torch.empty(3, dtype=torch.float64).pin_memory() for _ in models]
        x_ms = []
        for k in range(args.steps):
            flush.zero_()
            a, b = events()
            torch.cuda.synchronize()
            a.record(st)
            for hp, m in zip(host_p, models):
                m[4].copy_(hp, non_blocking=True)
            graph.replay()
            for hg, hs, o in zip(host_g, host_s, batch.out):
                hg.copy_(o["grad"], non_blocking=True)
                hs.copy_(o["stats"], non_blocking=True)
            b.record(st)
            torch.cuda.synchronize()
            x_ms.append(a.elapsed_time(b))
        return dict(step_ms=sum(g_ms) / len(g_ms), no_graph_ms=sum(e_ms) / len(e_ms),
                    separate_ms=sum(s_ms) / len(s_ms), e2e_ms=sum(x_ms) / len(x_ms), clk=clk,
                    status=batch.ws.status(), P_bytes=sum(h.numel() * 4 for h in host_p),
                    energy_per_site=[float(o["stats"][0].item()) / w["Lx"] for o in batch.out])

    m32 = replica_models(w, dev, nqs.FP32)
    m16 = [(nqs.model_desc(1, d.Lx, 1, d.d_h, precision=nqs.BF16), h, B, sd, p) for (d, h, B, sd, p) in m32]
    r32 = measure(m32)
    r16 = measure(m16) if args.precision != "fp32" else None
    # BF16 against FP32 on the same configurations, replica by replica
    check = None
    if r16 is not None:
        de, cos_min = 0.0, 1.0
        for (d32, ham, B, seed, p), (d16, _, _, _, _) in zip(m32, m16):
            sg, _, _ = nqs.sample(d32, p, B, seed=77, step=0, hcache=None)
            res = []
            for desc in (d16, d32):
                _, hc = nqs.logpsi(desc, p, sg)
                el = nqs.local_energy(desc, p, ham, sg, hc)
                g, stt = nqs.vmc_grad(desc, p, sg, hc, el)
                res.append((float(stt[0].item()) / w["Lx"], g.double()))
            de = max(de, abs(res[0][0] - res[1][0]))
            cos_min = min(cos_min, float(res[0][1] @ res[1][1] / (res[0][1].norm() * res[1][1].norm())))
        check = {"max_energy_per_site_diff": de, "min_grad_cosine": cos_min,
                 "pass": bool(de <= 1e-4 and cos_min >= 0.999)}
    chosen = r16 if (r16 is not None and (check["pass"] or args.precision == "bf16")) else r32
    models = m16 if chosen is r16 else m32
    R = len(models)
    total_B = sum(m[2] for m in models)
    pk, src = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    N = w["Lx"]
    flops = sum(2 * (3 * m[0].d_h ** 2 + 2 * m[0].d_h) * m[2] * (N + N * (N - 1) // 2 + 2 * N) for m in models)
    step_s = chosen["step_ms"] * 1e-3
    achieved = flops / step_s / 1e12
    if chosen is r16:
        peak = pk.get("bf16_tflops", 1887.4)
        roof = {"bound": "tensor", "kernel": "nqs_vmc_step_batched (whole step, BF16 tcgen05 replicas)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "bf16_tflops (burst) of measured peaks (%s)" % src}
    else:
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": "nqs_vmc_step_batched (whole step; chains dominate)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x %s MHz (%s)" % (sm_mhz, src)}
    line = {
        "metric": METRIC, "value": total_B / step_s, "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": chosen["step_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if chosen is r16 else "f32", "data": "synthetic",
        "config": {"workload": w["name"], "global_batch": total_B, "seq_len": N, "replicas": R,
                   "parallelism": "single",
                   "precision": ("bf16 tensor-core replicas (d_h 16-128) and reverse sweeps"
                                 if chosen is r16 else "fp32"),
                   "fp32_value": total_B / (r32["step_ms"] * 1e-3), "fp32_ms_per_step": r32["step_ms"],
                   "bf16_check": check,
                   "l2": "flushed (256 MB write) before every timed step",
                   "no_graph_ms_per_step": chosen["no_graph_ms"],
                   "separate_calls_ms_per_step": chosen["separate_ms"],
                   "energy_per_site": chosen["energy_per_site"],
                   "device_status": chosen["status"]},
        "roofline": roof,
        "e2e": {"value": total_B / (chosen["e2e_ms"] * 1e-3), "unit": "samples/s",
                "h2d_bytes_per_step": chosen["P_bytes"], "d2h_bytes_per_step": chosen["P_bytes"] + 24 * R},
        "gpu_launches": (10 if chosen is r32 else 17 * R + 3 * R) * args.steps,
        "clocks": {"sm_mhz": chosen["clk"]["sm_mhz"], "sm_max_mhz": chosen["clk"]["sm_max_mhz"],
                   "reasons": chosen["clk"]["reasons"]},
    }
    if not args.no_cpu_baseline:
        n = 2
        t = oracle_replicas_seconds(w, n, seed=300)
        line["cpu_baseline"] = {"value": n * R / t, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "%d samples of each of the %d replicas (float64 numpy, BLAS on all "
                                          "host cores)" % (n, R), "seconds": t}
    print(json.dumps(line))


def run_eval(args, w):
    """Final-evaluation mode (Tab. I: 10^6 samples after training): nqs_evaluate."""
    import numpy as np
    import torch
    from paper_2507_18700_gb300 import inputs, nqs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flat = inputs.xavier_params(1, w["d"], seed=w["seed"], noise_std=w["noise"]).astype(np.float32)
    params = torch.tensor(flat, device=dev)
    ham = nqs.tfim(w["J"], w["Gamma"])
    M, chunk = args.batch or w["B"], w["chunk"]
    st = torch.cuda.current_stream()
    out = {}
    for name, prec in (("fp32", nqs.FP32), ("bf16", nqs.BF16)):
        desc = nqs.model_desc(1, w["Lx"], 1, w["d"], precision=prec)
        ws = nqs.Workspace(dev)
        for k in range(args.warmup):
            nqs.evaluate(desc, params, ham, M, chunk=chunk, seed=11, step=k, ws=ws)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        ms = []
        for k in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            stats = nqs.evaluate(desc, params, ham, M, chunk=chunk, seed=11, step=100 + k, ws=ws)
            b.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        clk = clocks.stop()
        out[name] = dict(ms=sum(ms) / len(ms), stats=stats.cpu().tolist(), clk=clk, status=ws.status())
    N = w["Lx"]
    pk, src = peaks()
    c = out["bf16"]
    cells = M * (N + N * (N - 1) // 2)
    achieved = cells * 2 * mac_cell(w) / (c["ms"] * 1e-3) / 1e12
    line = {"metric": "final-evaluation samples/sec/GPU (sampling + E_loc, FP64 energy and variance)",
            "value": M / (c["ms"] * 1e-3), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": c["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": w["name"], "samples": M, "chunk": chunk,
                       "fp32_value": M / (out["fp32"]["ms"] * 1e-3),
                       "energy_per_site": {k: v["stats"][0] / N for k, v in out.items()},
                       "error_of_mean_per_site": {k: v["stats"][3] / N for k, v in out.items()},
                       "variance_per_site": {k: v["stats"][1] / N for k, v in out.items()},
                       "device_status": {k: v["status"] for k, v in out.items()},
                       "l2": "inputs (10^6 x 100 configurations, 1.7 GB of cache traffic per pass) exceed L2"},
            "roofline": {"bound": "tensor", "kernel": "nqs_evaluate (sampling + prefix-cached chains, BF16)",
                         "achieved": achieved, "peak": pk.get("bf16_tflops", 1887.4), "unit": "TFLOP/s",
                         "frac": achieved / pk.get("bf16_tflops", 1887.4), "traffic": None,
                         "peak_source": "bf16_tflops (burst) of measured peaks (%s)" % src},
            # per chunk: sampling 3 (two packs, engine), local energy 5, two status merges, one
            # sum; plus the final statistics
            "gpu_launches": args.steps * (11 * ((M + chunk - 1) // chunk) + 1),
            "clocks": {"sm_mhz": c["clk"]["sm_mhz"], "sm_max_mhz": c["clk"]["sm_max_mhz"],
                       "reasons": c["clk"]["reasons"]}}
    print(json.dumps(line))


def run_chain_variants(args, w):
    """Diagnostic: the BF16 chain kernel in each tile variant, pinned with the
    autotuner off, on one sampled batch: prints per-variant CUDA-event times of
    the local-energy call (median of --steps after --warmup).  1D TFIM: one and
    two threads per row (with the MUFU tanh rate they imply); 2D Heisenberg:
    the two-tile chain kernel with two and with one thread per row, the
    one-tile engine with one thread per row and with split rows (bitwise the
    same energies, checked here).  Under
    ncu each variant's chain launch is the only launch of its template
    instance."""
    import numpy as np
    import torch
    from paper_2507_18700_gb300 import inputs, nqs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B, d = args.batch or w["B"], w["d"]
    two = w["cell"] == 2
    N = w["Lx"] * w["Ly"]
    p = torch.tensor(inputs.xavier_params(w["cell"], d, seed=w["seed"], noise_std=w["noise"]).astype(np.float32),
                     device=dev)
    desc = nqs.model_desc(w["cell"], w["Lx"], w["Ly"], d, sz0=w["sz0"], precision=nqs.BF16)
    ham = nqs.heisenberg(w["J"]) if two else nqs.tfim(w["J"], w["Gamma"])
    nqs.set_autotune(False)
    s, _, hc = nqs.sample(desc, p, B, seed=1, step=0)
    ws = nqs.Workspace(dev)
    out, res = {}, []
    variants = ((None, "default"), (3, "two_tiles_two_threads_per_row"), (2, "two_tiles_one_thread_per_row"),
                (0, "one_tile"), (1, "one_tile_split_rows")) if two else \
        ((0, "threads_per_row_1"), (1, "threads_per_row_2"))
    for v, name in variants:
        nqs.set_tile_variant(v)
        ts = []
        for k in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            e = nqs.local_energy(desc, p, ham, s, hc, ws=ws)
            b.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(a.elapsed_time(b))
        res.append(e.clone())
        ms = float(np.median(ts))
        out[name] = {"ms": ms}
        if not two:
            out[name]["tanh_per_clock_per_sm"] = 3 * d * B * N * (N - 1) / 2 / (ms * 1e-3 * 2.07e9 * 152)
    nqs.set_tile_variant(None)
    nqs.set_autotune(True)
    line = {"probe": "chain-variants", "workload": w["name"], "batch": B, "variants": out,
            "bitwise_equal": all(bool(torch.equal(res[0], r)) for r in res[1:]), "device_status": ws.status()}
    print(json.dumps(line))


def run_ckpt_probe(args, w):
    """Diagnostic: teacher forcing + gradient of sum_b w_b log psi_b with the
    full prefix cache against hidden-state checkpoints every k sites (FP32 1D
    GRU): CUDA-event times (median of --steps after --warmup) and the bytes of
    saved states per sample."""
    import numpy as np
    import torch
    from paper_2507_18700_gb300 import inputs, nqs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B, N, d = args.batch or w["B"], w["Lx"], w["d"]
    p = torch.tensor(inputs.xavier_params(1, d, seed=w["seed"], noise_std=w["noise"]).astype(np.float32), device=dev)
    desc = nqs.model_desc(1, N, 1, d)
    sig, _, _ = nqs.sample(desc, p, B, seed=1, step=0, hcache=None)
    wts = torch.tensor(inputs.random_weights(B, seed=2).astype(np.float32), device=dev)
    ws = nqs.Workspace(dev)

    def timed(fn):
        ts = []
        for k in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    def full():
        _, hc = nqs.logpsi(desc, p, sig, ws=ws)
        nqs.logpsi_grad(desc, p, sig, hc, wts, ws=ws)

    out = {"full_cache": {"ms": timed(full), "saved_bytes_per_sample": N * d * 4}}
    for k in sorted({int(round(N ** 0.5)), 4, 25}):
        def ck(k=k):
            _, c = nqs.logpsi_ckpt(desc, p, sig, k, ws=ws)
            nqs.logpsi_grad_ckpt(desc, p, sig, k, c, wts, ws=ws)
        out["ckpt_every_%d" % k] = {"ms": timed(ck), "saved_bytes_per_sample": ((N + k - 1) // k - 1) * d * 4}
    print(json.dumps({"probe": "ckpt", "workload": w["name"], "precision": "fp32", "batch": B, "runs": out}))


def run_segment_probe(args, w):
    """Diagnostic: the gradient of sum_b w_b log psi_b of the 2D GRU at d_h =
    256 in BF16 with its reverse sweep in one pass and in passes of k
    positions: CUDA-event times (median of --steps after --warmup) and the
    workspace bytes of the gradient call."""
    import numpy as np
    import torch
    from paper_2507_18700_gb300 import inputs, nqs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B, d, N = args.batch or w["B"], w["d"], w["Lx"] * w["Ly"]
    p = torch.tensor(inputs.xavier_params(2, d, seed=w["seed"], noise_std=w["noise"]).astype(np.float32), device=dev)
    desc = nqs.model_desc(2, w["Lx"], w["Ly"], d, sz0=w["sz0"], precision=nqs.BF16)
    sig, _, hc = nqs.sample(desc, p, B, seed=1, step=0)
    wts = torch.tensor(inputs.random_weights(B, seed=2).astype(np.float32), device=dev)
    out, ref = {}, None
    for k in (0, 128, 64, 16):
        nqs.set_sweep_segment(k)
        ws = nqs.Workspace(dev)
        ts = []
        for it in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g = nqs.logpsi_grad(desc, p, sig, hc, wts, ws=ws)
            b.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                ts.append(a.elapsed_time(b))
        g = g.double()
        ref = g if ref is None else ref
        out["one_pass" if k == 0 else "passes_of_%d" % k] = {
            "ms": float(np.median(ts)), "workspace_bytes": nqs.workspace_bytes(desc, B, nqs.OP_LOGPSI_GRAD),
            "rel_diff_to_one_pass": float((g - ref).norm() / ref.norm()), "status": ws.status()}
        del ws
        torch.cuda.empty_cache()
    nqs.set_sweep_segment(0)
    print(json.dumps({"probe": "sweep-segment", "workload": w["name"], "precision": "bf16", "batch": B,
                      "cache_bytes": B * N * d * 4, "runs": out}))


def run_batched_probe(args, w):
    """Diagnostic: the replica family's batched step on the BF16 path, eagerly
    (no graph), for launch lists: prints the median step time."""
    import numpy as np
    import torch
    from paper_2507_18700_gb300 import nqs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    m32 = replica_models(w, dev, nqs.FP32)
    models = [(nqs.model_desc(1, d.Lx, 1, d.d_h, precision=nqs.BF16), h, B, sd, p) for (d, h, B, sd, p) in m32]
    batch = nqs.ReplicaBatch(models)
    ts = []
    for k in range(args.warmup + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        batch.step(step_no=k)
        b.record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            ts.append(a.elapsed_time(b))
    print(json.dumps({"probe": "batched", "workload": w["name"], "precision": "bf16",
                      "ms_per_step": float(np.median(ts)), "device_status": batch.ws.status()}))


def run_step_probe(args, w):
    """Diagnostic: the workload's VMC step at one precision (--precision, BF16
    for auto), without the FP32 comparison: CUDA-event times of sampling,
    local energy and gradient (median of --steps after --warmup) and the
    chain FLOP rate of the local-energy call.  A short target for launch
    lists."""
    import numpy as np
    import torch
    from paper_2507_18700_gb300 import inputs, nqs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B = args.batch or w["B"]
    prec = nqs.FP32 if args.precision == "fp32" else nqs.BF16
    p = torch.tensor(inputs.xavier_params(w["cell"], w["d"], seed=w["seed"], noise_std=w["noise"]).astype(np.float32),
                     device=dev)
    desc = nqs.model_desc(w["cell"], w["Lx"], w["Ly"], w["d"], sz0=w["sz0"], precision=prec)
    ham = nqs.tfim(w["J"], w["Gamma"]) if w["ham"] == "tfim" else nqs.heisenberg(w["J"], True)
    ws = nqs.Workspace(dev)
    ph = {"sample": [], "local_energy": [], "gradient": []}
    cells = 0
    for k in range(args.warmup + args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        s, _, hc = nqs.sample(desc, p, B, seed=1, step=k, ws=ws)
        ev[1].record()
        el = nqs.local_energy(desc, p, ham, s, hc, ws=ws)
        ev[2].record()
        nqs.vmc_grad(desc, p, s, hc, el, ws=ws)
        ev[3].record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            for i, name in enumerate(ph):
                ph[name].append(ev[i].elapsed_time(ev[i + 1]))
            cells = chain_cells(w, s.cpu().numpy())
    ms = {k: float(np.median(v)) for k, v in ph.items()}
    print(json.dumps({"probe": "step", "workload": w["name"], "precision": "fp32" if prec == nqs.FP32 else "bf16",
                      "batch": B, "ms": ms, "ms_per_step": sum(ms.values()),
                      "chain_tflops": cells * 2 * mac_cell(w) / (ms["local_energy"] * 1e-3) / 1e12,
                      "device_status": ws.status()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tfim100", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0, help="samples per step (default: the workload's)")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp32", "bf16"],
                    help="auto: report BF16 when it passes the accuracy check against FP32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--probe", default=None, choices=["chain-variants", "ckpt", "batched", "step", "sweep-segment"],
                    help="diagnostic run instead of the bench line")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.probe == "chain-variants":
        run_chain_variants(args, w)
        return
    if args.probe == "ckpt":
        run_ckpt_probe(args, w)
        return
    if args.probe == "sweep-segment":
        run_segment_probe(args, w)
        return
    if args.probe == "batched":
        run_batched_probe(args, w)
        return
    if args.probe == "step":
        run_step_probe(args, w)
        return
    if args.impl == "reference":
        if args.workload == "replicas16":
            t = oracle_replicas_seconds(w, 1, seed=7)
            print(json.dumps({"impl": "reference", "metric": METRIC, "value": 16 / t, "unit": "samples/s",
                              "n_gpus": args.gpus, "steps": 1, "warmup": 0, "ms_per_step": t * 1e3,
                              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                              "dtype": "f64", "data": "synthetic",
                              "config": {"workload": w["name"], "samples_per_step_timed": 16},
                              "cpu_baseline": {"value": 16 / t, "unit": "samples/s", "kind": "oracle",
                                               "cores": os.cpu_count(), "sample": "1 sample per replica"},
                              "e2e": {"value": 16 / t, "unit": "samples/s", "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}))
        else:
            run_reference(args, w)
    elif args.workload == "replicas16":
        run_replicas(args, w)
    elif args.workload == "eval1m":
        run_eval(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
