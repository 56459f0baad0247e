"""Throughput of the GB300 Metropolis sweep on the large batched spin-glass workload.

Workload (one "step" = one vegas_run over the whole schedule of the workload): 32
temperature replicas (T geometric 0.1 -> 2.0) of a 256^3 periodic simple-cubic +-J spin
glass, uniform-on-sphere trial moves, 200 MCS, FP32 spins with FP64 per-MCS E/M history.
Metric: Metropolis spin-update attempts per second (one attempt per site per MCS).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mcs M]

With N > 1 (launched by torchrun) every rank sweeps its own 32 replicas (instances
32*rank ...): weak scaling with no collective on the data path; value is the sum over
ranks divided by the slowest rank's time. `--impl reference` times the CPU FP64 oracle on
this host's cores on a bounded sample of the same workload (one MCS of one replica per
core per step).

Other lines: `--workload NAME` times one run of a secondary workload's schedule (the 8^3 FP64
ferromagnet, the 64^3 hysteresis loop, the core/shell particle, the 256 nanoparticles; under
torchrun the nanoparticles are split over the ranks), with `--impl reference` the oracle on a
bounded sample of it; `--policy`, `--variant`, `--type-stats`, `--snapshots` select the path;
`--analysis` and `--ising` time the history analysis and the Ising model; `--quick` times the
sweep alone (profiling runs).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Metropolis spin-update attempts/s on 1 GB300; batched vs plain; % HBM roofline"
UNIT = "attempts/s"
L_SIDE, REPLICAS, MCS, SEED = 256, 32, 200, 1
L_DEPTH = 0  # z extent of the lattice, 0: the side (profiling cases may be flatter)
# algorithmic bytes per attempt: 16 B read + 16 B write of the FP32 spin (float4), plus one
# row of six (int32 col, f32 J) links = 48 B shared by the 32 replicas that sweep it together
BYTES_PER_ATTEMPT = 16 + 16 + 48.0 / REPLICAS
CSRC = os.path.join(ROOT, "paper_1803_07030_gb300", "csrc")
# per sweep variant: the kernel that sweeps, its committed ncu summary, the sources it is built
# from (the summary's counters are used only while their hash matches), and how many colour
# classes one launch covers
SWEEP_KERNELS = {
    "per_class": ("pass32_r32", os.path.join(ROOT, "profiles", "pass32_r32_sg256x32.txt"),
                  [os.path.join(CSRC, f) for f in ("vegas_r32.cuh", "vegas_staged.cuh", "vegas_device.cuh")], 1),
    "wave": ("wave32_r32", os.path.join(ROOT, "profiles", "wave32_r32_sg256x32.txt"),
             [os.path.join(CSRC, f) for f in ("vegas_wave.cu", "vegas_staged.cuh", "vegas_device.cuh")], 2),
}


def sweep_kernel(variant: int):
    return SWEEP_KERNELS["wave" if variant == 4 else "per_class"]


def workload_desc(mcs):
    return {
        "workload": f"sg{L_SIDE}x32: 32 temperature replicas (T 0.1->2.0 geometric) of a {L_SIDE}^3 periodic sc +-J "
                    f"spin glass, random moves, {mcs} MCS per step, FP32 spins / FP64 history",
        "sites_per_replica": L_SIDE * L_SIDE * (L_DEPTH or L_SIDE),
        "replicas_per_gpu": REPLICAS,
        "mcs_per_step": mcs,
        "l2": "inputs larger than L2 (8.6 GB of spins + 0.8 GB of links per GPU)",
        "seed": SEED,
    }


def temperatures():
    return 0.1 * 20.0 ** (np.arange(REPLICAS) / (REPLICAS - 1.0))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_instances(rank: int, world: int, replicas: int = REPLICAS) -> list:
    """Instance ids a rank sweeps: every rank owns its own block of replicas (weak scaling;
    instances are independent, so no data-path collective is needed)."""
    return list(range(rank * replicas, (rank + 1) * replicas))


def workload_share(w, rank: int, world: int) -> dict:
    """The part of a secondary workload one rank runs. A workload of several samples is split
    into contiguous blocks of samples balanced by attempts (total work fixed: strong scaling);
    a workload of one sample runs whole on every rank as an independent copy whose instance ids
    start at rank * n_inst (weak scaling). Instance ids keep the sample-major numbering either
    way, so a rank's results are those of the same instances in a single run."""
    from paper_1803_07030_gb300.shard import contiguous_shards, sample_costs

    R = w.replicas
    costs = sample_costs(w.samples, R, w.n_steps, w.mcs)
    if len(w.samples) > 1:
        shards = contiguous_shards(costs, world)
        b, e = shards[rank]
        loads = [sum(costs[x:y]) for x, y in shards]
        return {"samples": w.samples[b:e], "T": w.T[b * R:e * R], "B": w.B[b * R:e * R], "inst_base": b * R,
                "range": (b, e), "attempts": loads[rank], "job_attempts": sum(costs), "scaling": "strong",
                "max_over_mean": max(loads) * world / max(1, sum(costs))}
    return {"samples": w.samples, "T": w.T, "B": w.B, "inst_base": rank * w.n_inst, "range": (0, len(w.samples)),
            "attempts": sum(costs), "job_attempts": sum(costs) * world, "scaling": "weak", "max_over_mean": 1.0}


def sum_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def slowest_rank_ms(ms: float, world: int, device=None) -> float:
    """Max over ranks of the timed region (the job ends with its slowest rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sweep_kernel_names(bits: int) -> list:
    from paper_1803_07030_gb300.vegas import sweep_kernel_names as names

    return names(bits)


def peaks():
    """Measured HBM copy bandwidth (GB/s) of this GPU model if the file has it, else the
    fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            v = float(json.load(f).get("hbm_gbs", 0.0))
        if v > 0.0:
            return v, "measured"
    except (OSError, ValueError, TypeError, AttributeError):
        pass
    return 6800.0, "fallback"


def kernel_hash(sources):
    h = hashlib.sha256()
    for path in sources:
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(summary, sources):
    """DRAM bytes per sweep launch from the committed ncu summary, if it still describes
    the current kernel source (else None)."""
    if not os.path.exists(summary):
        return None
    vals = {}
    with open(summary) as f:
        for line in f:
            if ":" in line and line.split(":", 1)[0].strip() in ("kernel_source_sha256_16", "dram_bytes_per_launch"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_hash(sources) or "dram_bytes_per_launch" not in vals:
        return None
    return float(vals["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"vegas_clocks_{os.getpid()}.csv")

    def __enter__(self):
        self.f = None
        self.proc = None
        if shutil.which("nvidia-smi") is None:  # no sampler: the line says the clocks are unknown
            return self
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:  # no nvidia-smi (or no temporary file): the line says the clocks are unknown
            self.proc = None
            if self.f:
                self.f.close()
                os.remove(self.path)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=10)
            except subprocess.TimeoutExpired:
                self.proc.kill()  # the sampler this object started, by its own handle
                self.proc.wait()
            self.f.close()
        return False

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline_run(sample, n_threads, mcs=1):
    """Oracle (CPU FP64, as it stands) on n_threads replicas of the full lattice, one per thread."""
    import oracle

    T = temperatures()[:n_threads, None]
    t0 = time.perf_counter()
    oracle.run(sample, T, np.zeros_like(T), mcs, seed=SEED, n_threads=n_threads)
    dt = time.perf_counter() - t0
    return n_threads * sample.n_sites * mcs / dt, dt


PRECISION_BOUND = 1e-3  # |d(E/N)| the FP32 path must stay below (per result)


def precision_statement(ctx, samples, replicas, B_last, instances) -> dict:
    """The deterministic precision figure of a result, taken in the oracle leg after the timed
    region: for a few instances, the last history record's E/N (FP32 spins, FP64 sums) against
    the oracle's FP64 energy (Eq. 1-3) of the same instance's final spins (read with
    vegas_get_spins). The spins are read after the step's FP64 renormalisation, which moves
    each spin by at most a few FP32 ulps, so the figure also bounds what the renormalisation
    changes. B_last: the field of the last step, per instance."""
    import oracle

    H = ctx.history()
    worst, rows = 0.0, []
    for i in instances:
        smp = samples[i // replicas]
        S = ctx.spins(i)
        e_ref = oracle.energy(smp, S, float(B_last[i]))
        d = abs(float(H[i, -1, 0]) - e_ref) / smp.n_sites
        worst = max(worst, d)
        rows.append({"instance": int(i), "sites": int(smp.n_sites), "e_per_site": e_ref / smp.n_sites,
                     "d_e_per_site": d})
    return {"d_e_per_site": worst, "bound": PRECISION_BOUND, "ok": bool(worst < PRECISION_BOUND),
            "method": "last history record's E/N against the oracle's FP64 energy of the same final spins",
            "checked": rows}


POLICY_CODES = {"random": 0, "flip": 1, "small": 2, "gauss": 3, "hn": 4, "adaptive": 5}
POLICY_DEFAULT_PARAM = {"random": 0.0, "flip": 0.0, "small": 0.5, "gauss": 0.4, "hn": 0.5, "adaptive": 1.0}


def apply_policy(samples, spec):
    """spec: comma list of policy[:param], one per site type (the last one repeats for higher
    types), e.g. "adaptive" or "random,hn:0.26". Sets each sample's policy table."""
    if not spec:
        return None
    entries = []
    for item in spec.split(","):
        name, _, par = item.partition(":")
        if name not in POLICY_CODES:
            raise SystemExit(f"unknown policy {name!r}; choose from {sorted(POLICY_CODES)}")
        entries.append((POLICY_CODES[name], float(par) if par else POLICY_DEFAULT_PARAM[name]))
    for smp in samples:
        n_types = int(smp.type.max()) + 1 if smp.type is not None else 1
        table = [entries[min(k, len(entries) - 1)] for k in range(max(n_types, len(entries)))]
        smp.with_policy([c for c, _ in table], [p for _, p in table])
    return spec


def host_description() -> dict:
    """The host the CPU baseline ran on: CPU model and the oracle's compiler (best effort; a
    missing tool leaves its field empty)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    compiler = ""
    try:
        compiler = subprocess.run(["gcc", "--version"], capture_output=True, text=True, timeout=10).stdout.splitlines()[0]
    except (OSError, subprocess.SubprocessError, IndexError):
        pass
    return {"cpu_model": model, "logical_cpus": os.cpu_count() or 0, "compiler": compiler,
            "build": "gcc -O2 -ffp-contract=off (oracle)"}


def workload_oracle_sample(w, budget: int = 10_000_000):
    """Oracle (CPU FP64, as it stands, one thread) on a bounded sample of a secondary workload:
    the first samples in order, each over the first temperature/field steps of its schedule
    (or the first MCS of its first step, when one step is already larger) that keep its
    attempts within `budget`, until `budget` attempts are done. Returns (attempts, seconds,
    description)."""
    import oracle

    R = w.replicas
    done, secs, parts = 0, 0.0, []
    for p, smp in enumerate(w.samples):
        per_step = smp.n_sites * R * w.mcs
        if per_step <= budget:
            steps, mcs = min(w.n_steps, budget // per_step), w.mcs
        else:
            steps, mcs = 1, max(1, budget // (smp.n_sites * R))
        rows = slice(p * R, (p + 1) * R)
        t0 = time.perf_counter()
        oracle.run(smp, w.T[rows, :steps], w.B[rows, :steps], mcs, seed=w.seed, inst_base=p * R)
        secs += time.perf_counter() - t0
        done += smp.n_sites * R * steps * mcs
        parts.append((steps, mcs))
        if done >= budget:
            break
    st = sorted({f"{a} x {b}" for a, b in parts})
    desc = (f"{len(parts)} of the {len(w.samples)} samples ({R} replica(s) each), steps x MCS from the start "
            f"of the schedule: {', '.join(st[:3])}{' ...' if len(st) > 3 else ''}; one thread: {done} attempts "
            f"in {secs:.2f} s")
    return done, secs, desc


def workload_bytes_per_attempt(w) -> float:
    """Algorithmic bytes per attempt of a workload: the spin read and written (float4 FP32 or
    double4 FP64) plus the site's links (int32 neighbour + J as f32 or f64) shared by the
    replicas that sweep them together; per-site parameters are left out."""
    vec = 32 if w.precision == 64 else 16
    link = 4 + (8 if w.precision == 64 else 4)
    sites = sum(s.n_sites for s in w.samples)
    edges = sum(s.n_edges for s in w.samples)
    return 2.0 * vec + link * edges / (sites * w.replicas)


def workload_config(w, args, policy, attempts_per_step):
    return {"workload": args.workload, "instances": w.n_inst, "sites": w.n_sites_total,
            "steps_x_mcs": [w.n_steps, w.mcs], "attempts_per_step": attempts_per_step,
            "l2": "working set inside L2" if w.n_sites_total * 16 < 100e6 else "larger than L2",
            "policy": policy or "random", "type_stats": bool(args.type_stats), "snapshots": bool(args.snapshots)}


def run_reference_workload(args):
    """The oracle on a secondary workload: one bounded sample (workload_oracle_sample) per step."""
    from lattices import workload
    import oracle

    oracle.build()
    w = workload(args.workload, mcs=args.mcs if args.mcs != MCS else None)
    policy = apply_policy(w.samples, args.policy)
    for _ in range(args.warmup):
        workload_oracle_sample(w)
    attempts, secs, desc = 0, 0.0, ""
    for _ in range(args.steps):
        a, t, desc = workload_oracle_sample(w)
        attempts += a
        secs += t
    value = attempts / secs
    rank, world, _ = dist_env()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps, "higher_is_better": True,
        "scaling": "strong" if len(w.samples) > 1 else "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, args, policy, w.attempts()),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc + " per step",
                         "host": host_description()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.analysis or args.ising:
        print(json.dumps({"impl": "reference", "unavailable": "the analysis and Ising lines time the oracle "
                          "themselves (their cpu_baseline); there is no separate reference arm for them"}), flush=True)
        return 0
    if args.workload != "sg256x32":
        return run_reference_workload(args)
    from lattices import sc_periodic
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    n_threads = min(REPLICAS, cores)
    s = sc_periodic(L_SIDE, bimodal_seed=SEED)
    for _ in range(args.warmup):
        cpu_baseline_run(s, n_threads)
    total, vals = 0.0, []
    for _ in range(args.steps):
        v, dt = cpu_baseline_run(s, n_threads)
        total += dt
        vals.append(v)
    value = args.steps * n_threads * s.n_sites / total
    sample = f"1 MCS of {n_threads} replicas (one per host thread) of the {L_SIDE}^3 lattice per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_desc(args.mcs),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_threads, "kind": "oracle", "sample": sample,
                         "host": host_description()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import paper_1803_07030_gb300 as vg
    from lattices import sc_periodic

    vg.build()
    mcs = args.mcs
    s = sc_periodic(L_SIDE if L_DEPTH in (0, L_SIDE) else (L_SIDE, L_SIDE, L_DEPTH), bimodal_seed=SEED)
    policy = apply_policy([s], args.policy)
    T = temperatures()[:, None]
    B = np.zeros_like(T)
    stream = torch.cuda.current_stream()
    inst_base = rank_instances(rank, world)[0]
    t0 = time.perf_counter()
    ctx = vg.Context([s], precision=32, replicas=REPLICAS, seed=SEED, inst_base=inst_base, device=dev,
                     stream=int(stream.cuda_stream), timing=True, variant=args.variant)
    create_s = time.perf_counter() - t0

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.run(T, B, mcs)
    barrier()
    st0 = ctx.stats()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.run(T, B, mcs)
        ev1.record(stream)
        barrier()
    st1 = ctx.stats()
    ms = slowest_rank_ms(ev0.elapsed_time(ev1), world, device="cuda")
    attempts_rank = REPLICAS * s.n_sites * mcs * args.steps
    value = attempts_rank * world / (ms / 1000.0)
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    sweeps = st1["sweep_launches"] - st0["sweep_launches"]
    sweep_ms = (st1["sweep_ms"] - st0["sweep_ms"]) / max(sweeps, 1)
    kname, ksummary, ksources, kclasses = sweep_kernel(st1["variant"])
    # one colour class of the checkerboard per launch, or both (wavefront sweep)
    attempts_per_launch = REPLICAS * s.n_sites * kclasses // 2
    peak, peak_kind = peaks()
    achieved = BYTES_PER_ATTEMPT * attempts_per_launch / (sweep_ms / 1000.0) / 1e9
    # the committed counters are those of the 256^3 workload; another side has none
    traffic = profiled_traffic(ksummary, ksources) if L_SIDE == 256 and L_DEPTH in (0, 256) else None

    if args.quick or policy:
        if rank == 0:
            cfg = dict(workload_desc(mcs))
            if policy:
                cfg["policy"] = policy
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms / args.steps,
                              "config": cfg, "quick": True, "avg_launch_ms": sweep_ms,
                              "achieved_gbs": achieved, "gpu_launches": launches, "variant": st1["variant"],
                              "clocks": clk.summary()}),
                  flush=True)
        ctx.close()
        return 0

    # end to end through the public API with host buffers: schedule in, history out
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(args.steps):
        ctx.run(T, B, mcs)
        h = ctx.history()
    e2e_s = time.perf_counter() - te
    e2e_value = attempts_rank * world / e2e_s
    h2d = T.size * 2 * 8 + 40
    d2h = REPLICAS * mcs * 4 * 8 + 4

    # the oracle leg (rank 0, after every timed region of this context): precision statement
    precision = precision_statement(ctx, [s], REPLICAS, B[:, -1], (0, REPLICAS // 2, REPLICAS - 1)) \
        if rank == 0 else None

    # plain single-instance path on the same lattice: one replica per context, R = 1
    ctx.close()
    torch.cuda.synchronize()
    plain_reps = (0, REPLICAS - 1)
    plain_ms = 0.0
    for p in plain_reps:
        with vg.Context([s], precision=32, replicas=1, seed=SEED, inst_base=inst_base + p, device=dev,
                        stream=int(stream.cuda_stream)) as q:
            q.run(T[p:p + 1], B[p:p + 1], 2)  # warm-up
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            q.run(T[p:p + 1], B[p:p + 1], mcs)
            b.record(stream)
            torch.cuda.synchronize()
            plain_ms += a.elapsed_time(b)
    plain_value = len(plain_reps) * s.n_sites * mcs / (plain_ms / 1000.0)

    line = None
    if rank == 0:
        cores = min(REPLICAS, os.cpu_count() or 1)
        cpu_v, cpu_dt = cpu_baseline_run(s, cores)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_desc(mcs),
            "precision": precision,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_basis": "sweep kernel: algorithmic bytes of one launch / its mean CUDA-event time",
                         "headline_achieved": BYTES_PER_ATTEMPT * value / world / 1e9,
                         "headline_frac": BYTES_PER_ATTEMPT * value / world / 1e9 / peak,
                         "headline_basis": "whole step: algorithmic bytes per attempt x attempts/s per GPU "
                                           "(every launch of the step, reductions and renormalisation included)",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s",
                         "kernel": kname, "bytes_per_attempt": BYTES_PER_ATTEMPT,
                         "attempts_per_launch": attempts_per_launch, "avg_launch_ms": sweep_ms},
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_description(),
                             "sample": f"1 MCS of {cores} replicas (one per host thread) of the {L_SIDE}^3 lattice, "
                                       f"{cpu_dt:.1f} s"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "vegas_run(host T, B) + vegas_history(host buffer)"},
            "plain": {"value": plain_value, "unit": UNIT, "replicas_timed": len(plain_reps),
                      "note": "same lattice, one replica per context (R = 1), one launch per colour class"},
            "batched_over_plain": value / world / plain_value,
            "gpu_launches": launches,
            "variant": st1["variant"],
            "sweep_kernels": sweep_kernel_names(st1.get("sweep_kernels", 0)),
            "create_s": create_s,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_workload(args):
    """One step = one vegas_run of the whole schedule of a secondary workload (the 8^3 FP64
    ferromagnet, the 64^3 hysteresis loop, the field-cooled core/shell particle, the 256
    nanoparticles). Under torchrun the 256 nanoparticles are split over the ranks in contiguous
    blocks balanced by attempts, and a one-sample workload runs as an independent copy per rank
    (`workload_share`); no collective touches the data path. For np256 at one GPU the plain
    comparison runs every particle in its own context, one after another, for a bounded number
    of MCS."""
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import paper_1803_07030_gb300 as vg
    from lattices import workload

    vg.build()
    w = workload(args.workload, mcs=args.mcs if args.mcs != MCS else None)
    policy = apply_policy(w.samples, args.policy)
    share = workload_share(w, rank, world)
    stream = torch.cuda.current_stream()
    ctx = None
    if share["samples"]:
        ctx = vg.Context(share["samples"], precision=w.precision, replicas=w.replicas, seed=w.seed,
                         inst_base=share["inst_base"], device=dev, stream=int(stream.cuda_stream),
                         variant=args.variant, type_stats=args.type_stats, snapshots=args.snapshots,
                         resident_smem=args.resident_smem, graphs=args.graphs,
                         cluster_blocks=args.cluster_blocks, cluster_threads=args.cluster_threads,
                         cluster_split=args.cluster_split, group_threads=args.group_threads,
                         group_sites=16 * args.group_threads)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        if ctx is not None:
            ctx.run(share["T"], share["B"], w.mcs)
    barrier()
    st0 = ctx.stats() if ctx is not None else None
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        a.record(stream)
        for _ in range(args.steps):
            if ctx is not None:
                ctx.run(share["T"], share["B"], w.mcs)
        b.record(stream)
        barrier()
    ms = slowest_rank_ms(a.elapsed_time(b), world, device="cuda")
    st1 = ctx.stats() if ctx is not None else None
    precision = None
    if rank == 0 and ctx is not None and not args.quick:
        # the oracle leg, after the timed region: the first instance, the largest sample's
        # first replica and the last instance
        R = w.replicas
        big = int(np.argmax([smp.n_sites for smp in share["samples"]]))
        insts = sorted({0, big * R, len(share["samples"]) * R - 1})
        precision = precision_statement(ctx, share["samples"], R, np.asarray(share["B"])[:, -1], insts)
    mine = float(st1["kernel_launches"] - st0["kernel_launches"]) if ctx is not None else 0.0
    launches = sum_over_ranks(mine, world, device="cuda")
    value = share["job_attempts"] * args.steps / (ms / 1000.0)
    if ctx is not None:
        ctx.close()
    if rank == 0:
        shape = {k: st1[k] for k in ("variant", "block_threads", "cluster_blocks", "split_sites", "group_threads",
                                     "group_sites")} if st1 else {}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": share["scaling"], "vs_baseline": None, "dtype": "f64" if w.precision == 64 else "f32",
            "data": "synthetic",
            "config": workload_config(w, args, policy, share["job_attempts"]),
            **shape,
            "sweep_kernels": sweep_kernel_names(st1.get("sweep_kernels", 0)) if st1 else [],
            "precision": precision,
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        bpa = workload_bytes_per_attempt(w)
        peak, peak_kind = peaks()
        line["effective_roofline"] = {
            "bytes_per_attempt": bpa, "achieved": bpa * value / 1e9, "peak": peak, "unit": "GB/s",
            "frac": bpa * value / 1e9 / peak, "peak_source": f"{peak_kind} HBM copy bandwidth",
            "note": "algorithmic bytes x attempts/s; the working set stays in L2, so this is an effective "
                    "figure that can exceed 1" if w.n_sites_total * 16 < 100e6 else
                    "algorithmic bytes x attempts/s against the HBM peak"}
        if not args.quick:
            att, secs, desc = workload_oracle_sample(w)
            line["cpu_baseline"] = {"value": att / secs, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                                    "host": host_description()}
        if world > 1:
            line["config"]["sharding"] = {
                "by": "contiguous sample blocks balanced by attempts" if share["scaling"] == "strong"
                else "one independent copy per rank", "max_over_mean_attempts": share["max_over_mean"]}
        if args.workload == "np256" and world == 1 and not policy and not args.type_stats and not args.snapshots \
                and not args.quick:
            plain_mcs = min(w.mcs, 100)
            plain_ms, plain_att = 0.0, 0
            for p, smp in enumerate(w.samples):
                with vg.Context([smp], precision=32, seed=w.seed, inst_base=p, variant=0,
                                stream=int(stream.cuda_stream)) as q:
                    Tp, Bp = w.T[p:p + 1], w.B[p:p + 1]
                    q.run(Tp, Bp, 2)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    q.run(Tp, Bp, plain_mcs)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    plain_ms += e0.elapsed_time(e1)
                    plain_att += smp.n_sites * plain_mcs
            line["plain"] = {"value": plain_att / (plain_ms / 1000.0), "unit": UNIT,
                             "note": f"each of the {len(w.samples)} particles in its own context, one launch per "
                                     f"colour class, {plain_mcs} MCS each, run one after another"}
            line["batched_over_plain"] = value / line["plain"]["value"]
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_analysis(args):
    """Times the history analysis on the GPU (C-ABI, host arrays in and out, copies included):
    thermal averages of 1024 histories of 10,000 records (AR(1) energies with tau ~ 10), and
    multiple-histogram reweighting of 32 runs x 20,000 samples. The oracle (numpy) is timed on
    a bounded sample of the same work."""
    import torch
    import paper_1803_07030_gb300 as vg

    vg.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(SEED)
    ns, ln, phi = 1024, 10000, 0.9
    x = np.zeros((ns, ln))
    xi = rng.normal(size=(ns, ln)) * np.sqrt(1 - phi * phi)
    for i in range(1, ln):
        x[:, i] = phi * x[:, i - 1] + xi[:, i]
    H = np.stack([-3000.0 + 30.0 * x, 50.0 * rng.normal(size=(ns, ln)), 50.0 * x, 300.0 + 40.0 * x], axis=2)
    Tv = np.linspace(0.5, 2.5, ns)
    for _ in range(args.warmup):
        vg.thermal_averages(H, 2000, 20, Tv, 1000.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vg.thermal_averages(H, 2000, 20, Tv, 1000.0)
    ta = (time.perf_counter() - t0) / args.steps
    K, n = 32, 20000
    betas = np.linspace(0.4, 1.2, K)
    E = np.stack([rng.normal(-1000.0 * b, 30.0, n) for b in betas])
    O = np.stack([np.column_stack([E[k], E[k] ** 2]) for k in range(K)])
    vg.reweight(E, O, betas, betas, max_iter=50, tol=1e-300)
    t0 = time.perf_counter()
    _, _, it = vg.reweight(E, O, betas, np.linspace(0.4, 1.2, 64), max_iter=200, tol=1e-300)
    tr = time.perf_counter() - t0
    from oracle import analysis as ora_an

    t0 = time.perf_counter()
    for s_ in range(8):
        ora_an.thermal_averages(H[s_], 2000, 20, Tv[s_], 1000.0)
    to = (time.perf_counter() - t0) / 8
    t0 = time.perf_counter()
    ora_an.reweight(E, O, betas, np.linspace(0.4, 1.2, 64), max_iter=5, tol=1e-300)
    tro = (time.perf_counter() - t0) / 5
    line = {
        "metric": "history records analysed/s (thermal averages, errors, tau) on 1 GB300", "value": ns * ln / ta,
        "unit": "records/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * ta,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "1024 histories x 10,000 records (AR(1), tau ~ 10), cut 2000, 20 bins; "
                               "reweighting 32 runs x 20,000 samples to 64 temperatures"},
        "reweight": {"iterations": it, "s": tr, "sample_iterations_per_s": K * n * it / tr},
        "cpu_baseline": {"value": ln / to, "unit": "records/s", "cores": 1, "kind": "oracle", "host": host_description(),
                         "sample": "8 of the 1024 histories", "reweight_sample_iterations_per_s": K * n / tro},
    }
    print(json.dumps(line), flush=True)
    return 0


ISING_PROFILE = os.path.join(ROOT, "profiles", "ising_pass_2d16384x32.txt")


def run_ising(args):
    """The Ising workload (spin flip, Sec. II; the 2D Ising systems of Sec. IV.B, IV.E): a
    periodic 16384^2 square lattice, 32 replicas (temperatures 1.5 .. 3.5), multi-spin coded.
    A step is one vegas_ising_run of --mcs MCS (default 20). The kernel is bound by integer
    issue (Philox and the bit logic), not by HBM: the roofline is warp instructions per second
    against the issue peak, 152 SMs x 4 schedulers x the median SM clock."""
    import torch
    import paper_1803_07030_gb300 as vg

    vg.build()
    torch.cuda.set_device(0)
    L, R = 16384, 32
    mcs = args.mcs if args.mcs != MCS else 20
    T = np.linspace(1.5, 3.5, R)[:, None]
    h = np.zeros_like(T)
    stream = torch.cuda.current_stream()
    with vg.IsingContext(2, L, replicas=R, seed=SEED, stream=int(stream.cuda_stream), timing=True) as c:
        for _ in range(args.warmup):
            c.run(T, h, mcs)
        torch.cuda.synchronize()
        st0 = c.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                c.run(T, h, mcs)
            e1.record(stream)
            torch.cuda.synchronize()
        st1 = c.stats()
        ms = e0.elapsed_time(e1)
    attempts = L * L * R * mcs * args.steps
    value = attempts / (ms / 1000.0)
    sweeps = st1["sweep_launches"] - st0["sweep_launches"]
    launch_ms = (st1["sweep_ms"] - st0["sweep_ms"]) / max(sweeps, 1)
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = 152 * 4 * sm_mhz * 1e6 / 1e9  # G warp-instructions/s
    inst = None
    if os.path.exists(ISING_PROFILE):
        for line in open(ISING_PROFILE):
            if line.startswith("warp_instructions_per_attempt:"):
                inst = float(line.split(":", 1)[1])
    per_launch = L * L * R // 2
    achieved = None if inst is None else inst * per_launch / (launch_ms / 1000.0) / 1e9
    from oracle import ising_run

    t0 = time.perf_counter()
    ising_run(2, 256, 1.0, np.full((4, 1), 2.27), np.zeros((4, 1)), 10, seed=SEED)
    cpu_dt = time.perf_counter() - t0
    line = {
        "metric": "Ising spin-flip attempts/s on 1 GB300", "value": value, "unit": "attempts/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "2D Ising, periodic 16384^2, 32 replicas (T 1.5..3.5), J = 1, h = 0, "
                               f"{mcs} MCS per step, multi-spin coded", "l2": "inputs larger than L2 (1 GiB)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G warp-instructions/s",
                     "frac": None if achieved is None else achieved / peak,
                     "peak_source": "152 SMs x 4 issue slots x median SM clock (derived)",
                     "kernel": "ising_pass_kernel<2>", "warp_instructions_per_attempt": inst,
                     "attempts_per_launch": per_launch, "avg_launch_ms": launch_ms},
        "cpu_baseline": {"value": 256 * 256 * 4 * 10 / cpu_dt, "unit": "attempts/s", "cores": 1, "kind": "oracle", "host": host_description(),
                         "sample": "256^2 x 4 replicas x 10 MCS"},
        "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"], "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    global L_SIDE, L_DEPTH
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--mcs", type=int, default=MCS)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=L_SIDE, help="lattice side (smaller cases for ncu captures)")
    ap.add_argument("--depth", type=int, default=0, help="z extent of the lattice (0: the side); profiling cases")
    ap.add_argument("--workload", default="sg256x32",
                    choices=["sg256x32", "sc8_fp64", "sc64_hyst", "coreshell_fc", "np256"],
                    help="sg256x32 is the headline line; the others time one run of their schedule")
    ap.add_argument("--policy", default="",
                    help="update policy per site type, e.g. 'adaptive' or 'random,hn:0.26' (policy[:param], one "
                         "per type; names: " + ", ".join(POLICY_CODES) + "); the line then reports that path")
    ap.add_argument("--variant", type=int, default=-1, choices=[-1, 0, 1, 2, 3, 4],
                    help="sweep variant: -1 automatic (timed on the first run), 0 per colour class, 1 resident, 3 cluster, "
                         "2 cooperative, 4 wavefront (both classes per launch); profiling commands fix it because ncu "
                         "distorts the automatic timing")
    ap.add_argument("--resident-smem", type=int, default=0, choices=[-1, 0, 1],
                    help="secondary workloads: 1 keeps spins in shared memory in the resident or cluster sweep, "
                         "-1 never, 0 automatic (profiling commands fix it with --variant)")
    ap.add_argument("--cluster-blocks", type=int, default=0,
                    help="secondary workloads with --variant 3: blocks per cluster (0 automatic); with the next "
                         "three, the shape the automatic choice keeps, for profiling commands")
    ap.add_argument("--cluster-threads", type=int, default=0, help="threads per block of the cluster sweep (0 automatic)")
    ap.add_argument("--cluster-split", type=int, default=0,
                    help="cluster sweep: instances of at most this many sites swept by one block each (0: all by clusters)")
    ap.add_argument("--group-threads", type=int, default=0,
                    help="resident or cluster sweep: threads per small instance swept several to a block "
                         "(up to 16 sites per thread; 0 off)")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1, 2],
                    help="secondary workloads: 1 a run as one CUDA graph, 2 a graph per step, 0 direct launches "
                         "(profilers see the kernels of graphs without conditional nodes only)")
    ap.add_argument("--analysis", action="store_true", help="time the history analysis instead of the sweep")
    ap.add_argument("--ising", action="store_true", help="time the multi-spin-coded Ising workload")
    ap.add_argument("--type-stats", action="store_true", help="secondary workloads: record per-type magnetization")
    ap.add_argument("--snapshots", action="store_true", help="secondary workloads: keep the final state of every step")
    ap.add_argument("--quick", action="store_true",
                    help="time the sweep only (no e2e, plain-path or CPU-baseline legs); for profiling runs")
    args = ap.parse_args()
    L_SIDE = args.side
    L_DEPTH = args.depth
    if args.impl == "reference":
        return run_reference(args)
    if args.analysis:
        return run_analysis(args)
    if args.ising:
        return run_ising(args)
    if args.workload != "sg256x32":
        return run_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
