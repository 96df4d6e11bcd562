"""Benchmark: active pair interactions per second (density + force) of the SPH
hot path on the 2,097,152-particle clustered workload (uniform background plus
64 Plummer spheres, time bins spanning ~2^13), batched versus plain.

One timed step = one full kick-drift-kick step (mark active, drift, density
with the smoothing-length iteration, force, kicks, time bins).  K steps are
timed from the initial conditions (step 0 has every particle active, the rest
only the particles of the active bins); W warm-up steps run first on the same
initial conditions, after which the state is restored.  Each step is timed with
CUDA events on the launching stream, with the L2 cache flushed between steps
(a 256 MiB write, outside the timed interval).

value       useful pairs (density: i active, j != i, r < H_i at the final h;
            force: r < max(H_i, H_j)) over all timed steps / summed step time,
            batched form (persistent kernels + CUDA graph);
plain       the same for the per-bin launch form;
e2e         the batched form through the C ABI with host buffers: each step
            copies the particle state host->device (pinned) and back;
roofline    the dominant pair-loop kernel: algorithmic FLOPs per useful pair
            (density 29, force 61) x useful pairs per launch / mean launch time
            (CUDA events in the library, on the launching stream), against the
            FP32 peak: the SMs the device reports x 128 lanes x 2 x the median
            SM clock sampled during the timed steps; `executed` counts instead
            every candidate test and every pair term of every h iteration; its
            `traffic` is the DRAM bytes per launch from the kernel's ncu summary
            under profiles/, reported only while that summary's source digest
            matches the sources;
cell_build_ms  one cell build of the initial state (CUDA events; a rebuild
            inside a timed step is part of that step's time);
cpu_baseline  the FP64 oracle on a bounded sample of the same workload.

--impl reference times the oracle alone (the CPU reference of this method).
--ablation prints, instead, the cost per unit simulated time of relevant-only
drift, drift-all and one global time step (Sec. III-D); --adjoint the times
of the forward and reverse pass of the differentiation workload.
Under torchrun every rank runs its own replica (the method does not shard
across GPUs here); value sums the ranks' pairs over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "active pair interactions/s (density+force) at 2.1M clustered; batched vs plain"
UNIT = "pairs/s"
WORKLOAD = "c3_clustered_2m"
# algorithmic FP32 operations per useful pair (FMA = 2; sqrt, rsqrt, divide = 1)
FLOP_DENSITY = 29
FLOP_FORCE = 61
# executed FP32 operations per candidate test (3 differences, r^2 by one multiply
# and two FMAs, the compare; the force test compares with both supports)
FLOP_TEST_DENSITY = 9
FLOP_TEST_FORCE = 10
FP32_LANES_PER_SM = 128  # FP32 lanes per SM (sm_103a)


def fp32_peak(sms: int, sm_mhz: float) -> float:
    """FP32 peak in TFLOP/s from the SM count and the SM clock (FMA = 2)."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
DEFAULT_LAUNCH = dict(threads_per_particle=1, leaf_max=16, cell_margin=2.0, list_cap=512,
                      search_margin=1.02, staging_depth=1, heavy_factor=2.0)
KNOBS = ("threads_per_particle", "leaf_max", "cell_margin", "list_cap", "search_margin",
         "staging_depth", "heavy_factor")


def kernel_source_digest() -> str:
    """First 16 hex digits of the SHA-256 of the pair-kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for f in ("sph_pairs.cu", "sph_pairloop.cuh", "sph_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1807_01341_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def launch_key(launch: dict) -> str:
    return " ".join(f"{k}={launch[k]}" for k in KNOBS)


def profiled_traffic(kernel: str, workload: str, launch: dict, profiles_dir: str | None = None):
    """DRAM bytes per launch of a pair kernel from its committed ncu summary,
    or None when the summary is missing or was taken from other sources or
    another launch configuration."""
    path = os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), f"k_{kernel}_{workload}.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    fields = dict(re.findall(
        r"^(kernel_source_digest|traffic_bytes_per_launch|launch_config):\s*(\S.*?)\s*$",
        text, flags=re.M))
    if fields.get("kernel_source_digest") != kernel_source_digest():
        return None
    if fields.get("launch_config") != launch_key(launch):
        return None
    try:
        return int(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def parse_launch(text: str | None) -> dict:
    """--launch "knob=value,knob=value" (knobs of KNOBS) as a dict."""
    out = {}
    for item in (text or "").split(","):
        if not item.strip():
            continue
        k, v = item.split("=", 1)
        k = k.strip()
        if k not in KNOBS:
            raise SystemExit(f"--launch: unknown knob {k!r} (one of {', '.join(KNOBS)})")
        out[k] = type(DEFAULT_LAUNCH[k])(float(v)) if isinstance(DEFAULT_LAUNCH[k], int) \
            else float(v)
    return out


def reduce_over_ranks(max_values, sum_values, device):
    """Across the ranks of the process group: the largest of each time-like
    value (the job takes as long as its slowest rank) and the sum of each
    count (the work of the whole job)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(max_values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor(sum_values, dtype=torch.float64, device=device)
    dist.all_reduce(s)
    return [float(x) for x in t.tolist()], [float(x) for x in s.tolist()]


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if len(s) > 2 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 2 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, name in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import torch
    import sph_ics
    from sph_ics import workloads
    from paper_1807_01341_gb300 import _lib, autotune, build, sim

    build.build()
    dev = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    ic = workloads.make(args.workload)
    t_ic = time.time() - t0
    n = ic["pos"].shape[0]
    base = workloads.PARAMS[args.workload]
    tuned = dict(DEFAULT_LAUNCH)
    tuned.update(parse_launch(args.launch))
    tune_info = None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    if not args.no_autotune:
        # trials time the benchmark's own step count, L2 flushed between steps
        t = autotune.tune(ic, base, args.workload, steps=args.steps, flush=flush.zero_)
        tuned = {k: t[k] for k in KNOBS}
        tune_info = {"cached": t.get("cached"),
                     "trials": [dict(r["cand"], pairs_per_s=r["rate"]) for r in t.get("trials", [])]}
    params = sim.Params(**base, **tuned)
    ctx = sim.Context(params, n)
    p = sim.Particles.from_ics(ic, with_counts=False, with_gradients=False)
    ctx.build_cells(p)
    snapshot = {k: t.clone() for k, t in p.arrays().items()}
    stream = torch.cuda.Stream()

    build_ms = []

    def restore():
        """The initial state, its cell build timed (CUDA events on the
        stream; the build also synchronises on the host to size its grid)."""
        for k, t in p.arrays().items():
            t.copy_(snapshot[k])
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.build_cells(p, stream)
        e1.record(stream)
        e1.synchronize()
        build_ms.append(e0.elapsed_time(e1))
        ctx.begin_run(stream)
        ctx.reset_kernel_times()

    def one_step(form, timed):
        """One step: [ev0, enqueue, ev1] then a host sync outside the interval;
        a step stopped by a cell overflow is redone after the rebuild and its
        attempts and the rebuild are all counted."""
        total = 0.0
        while True:
            if timed:
                flush.zero_()
                torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                ev0.record(stream)
                ctx.step_async(p, form, stream)
                ev1.record(stream)
            tw = time.perf_counter()
            done = ctx.step_sync(p, stream)
            total += ev0.elapsed_time(ev1)
            if done:
                return total
            total += (time.perf_counter() - tw) * 1e3  # the rebuild (wall clock)

    forms = {"batched": _lib.SPH_FORM_BATCHED, "plain": _lib.SPH_FORM_PLAIN}
    results = {}
    ctx.set_profiling(True)
    for name in ([] if args.no_plain else ["plain"]) + ["batched"]:
        form = forms[name]
        restore()
        for _ in range(args.warmup):
            one_step(form, False)
        restore()
        ctx.reset_counters(stream)
        torch.cuda.synchronize()
        launches0 = ctx.counters()["kernel_launches"]
        if world > 1:
            torch.distributed.barrier()
        ms = []
        with Clocks(dev) as clk:
            for _ in range(args.steps):
                ms.append(one_step(form, True))
        torch.cuda.synchronize()
        c = ctx.counters()
        kt = ctx.kernel_times()
        results[name] = dict(ms=ms, counters=c, ktimes=kt, clocks=clk.summary(),
                             grid=ctx.grid_info(),
                             launches=c["kernel_launches"] - launches0)
    res = results["batched"]
    pairs = res["counters"]["pairs_density"] + res["counters"]["pairs_force"]
    total_ms = sum(res["ms"])

    # e2e: the same steps through the C ABI from a host copy of the state (one
    # pinned buffer holding every particle array, as the device state does)
    host = torch.empty(p.storage.shape, dtype=torch.uint8, pin_memory=True)
    restore()
    host.copy_(p.storage)
    h2d = host.numel()  # bytes moved each way per step
    ctx.reset_counters(stream)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        t_step = 0.0
        while True:
            flush.zero_()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                ev0.record(stream)
                p.storage.copy_(host, non_blocking=True)
                ctx.step_async(p, _lib.SPH_FORM_BATCHED, stream)
                host.copy_(p.storage, non_blocking=True)
                ev1.record(stream)
            done = ctx.step_sync(p, stream)
            t_step += ev0.elapsed_time(ev1)
            if done:
                break
            # the cells were rebuilt on the device: fetch the reordered state
            tw = time.perf_counter()
            host.copy_(p.storage)
            torch.cuda.synchronize()
            t_step += (time.perf_counter() - tw) * 1e3
        e2e_ms.append(t_step)
    ce = ctx.counters()
    e2e_pairs = ce["pairs_density"] + ce["pairs_force"]

    # roofline of the dominant pair-loop kernel (batched form)
    kt = res["ktimes"]
    c = res["counters"]
    dens = dict(ms=kt["density_ms"], n=max(kt["density_launches"], 1),
                flops=FLOP_DENSITY * c["pairs_density"],
                executed=FLOP_TEST_DENSITY * c["cand_density"] + FLOP_DENSITY * c["evals_density"])
    forc = dict(ms=kt["force_ms"], n=max(kt["force_launches"], 1),
                flops=FLOP_FORCE * c["pairs_force"],
                executed=FLOP_TEST_FORCE * c["cand_force"] + FLOP_FORCE * c["pairs_force"])
    dom_name, dom = max((("density", dens), ("force", forc)), key=lambda kv: kv[1]["ms"])
    per_launch_s = dom["ms"] / dom["n"] / 1e3
    achieved = dom["flops"] / dom["n"] / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    executed = dom["executed"] / dom["n"] / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = dict(pairs=pairs, total_ms=total_ms, res=results, e2e_ms=sum(e2e_ms),
               sms=sms, build_ms=statistics.median(build_ms) if build_ms else None,
               e2e_pairs=e2e_pairs, h2d=h2d, n=n, t_ic=t_ic,
               roofline=dict(kernel=dom_name, achieved=achieved, executed=executed,
                             per_launch_ms=per_launch_s * 1e3,
                             density_ms=kt["density_ms"], force_ms=kt["force_ms"]),
               gpu_state={k: t for k, t in p.arrays().items()} if rank == 0 else None,
               ic=ic, tuned=tuned, tune_info=tune_info)
    return out


# ---------------------------------------------------------------------------
# --ablation: the time-stepping schemes of Sec. III-D compared (Fig. 2 analogue)
# ---------------------------------------------------------------------------
def run_ablation(args):
    """K steps from the initial conditions under three schemes, each timed
    with CUDA events (after one warm-up step and a restore):
    relevant-only drift (the default), drift of every particle each step, and
    one global time step (every particle active every step).  The individual
    schemes advance the tick by what their bins allow; the global scheme's
    time step is the smallest particle step of the initial bins (the
    Gadget-2-style global step), so its cost per unit simulated time is its
    cost per all-active step over that step."""
    import torch
    from paper_1807_01341_gb300 import _lib, sim
    from sph_ics import workloads
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ic = workloads.make(args.workload)
    n = ic["pos"].shape[0]
    base = dict(workloads.PARAMS[args.workload])
    stream = torch.cuda.Stream()
    schemes = {"relevant_only_drift": dict(drift_all=0),
               "drift_all": dict(drift_all=1),
               "global_step": dict(drift_all=0, bin_cap=0)}
    out, b_min = {}, None
    for name, kw in schemes.items():
        prm = dict(base, **DEFAULT_LAUNCH)
        prm.update(kw)
        ctx = sim.Context(sim.Params(**prm), n)
        p = sim.Particles.from_ics(ic, with_counts=False)
        snap = {k: t.clone() for k, t in p.arrays().items()}

        def restore():
            for k, t in p.arrays().items():
                t.copy_(snap[k])
            torch.cuda.synchronize()
            ctx.build_cells(p, stream)
            ctx.begin_run(stream)
        restore()
        ctx.step_async(p, _lib.SPH_FORM_BATCHED, stream)
        ctx.step_sync(p, stream)
        if name == "relevant_only_drift":
            b_min = int(p.numpy()["bin"].min())  # the initial bins (from step 0)
        restore()
        ctx.reset_counters(stream)
        ti0 = ctx.get_time()[0]
        ms = 0.0
        for _ in range(args.steps):
            while True:
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    ev0.record(stream)
                    ctx.step_async(p, _lib.SPH_FORM_BATCHED, stream)
                    ev1.record(stream)
                done = ctx.step_sync(p, stream)
                ms += ev0.elapsed_time(ev1)
                if done:
                    break
        ti1 = ctx.get_time()[1]  # the tick the next step would start at
        c = ctx.counters()
        sim_t = (ti1 - ti0) * base["dt_min"]
        out[name] = {"gpu_ms": ms, "ms_per_step": ms / args.steps,
                     "active_per_step": c["active_particles"] / args.steps,
                     "pairs": c["pairs_density"] + c["pairs_force"],
                     "sim_time": sim_t, "ms_per_sim_time": ms / sim_t if sim_t > 0 else None,
                     "rebuilds": c["rebuilds"]}
        ctx.close()
        del p, snap
        torch.cuda.empty_cache()
    # the global scheme at the Gadget-2 global step: the smallest initial bin
    g = out["global_step"]
    g["global_dt"] = (2 ** b_min) * base["dt_min"]
    g["ms_per_sim_time"] = g["ms_per_step"] / g["global_dt"]
    ref = out["relevant_only_drift"]["ms_per_sim_time"]
    line = {"experiment": "time-to-solution of the time-stepping schemes (Sec. III-D, Fig. 2)",
            "workload": args.workload, "n_particles": n, "steps": args.steps,
            "data": "synthetic", "schemes": out,
            "speedup_vs_global_step": g["ms_per_sim_time"] / ref if ref else None,
            "speedup_vs_drift_all": out["drift_all"]["ms_per_sim_time"] / ref if ref else None}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# --adjoint: the differentiation workload (forward and reverse pass timed)
# ---------------------------------------------------------------------------
def run_adjoint(args):
    """The 32,768-particle clumpy set, 20 steps, loss = sum of squared
    differences of the final density on a 32^3 grid against the same run from
    perturbed initial conditions (positions + N(0, 0.05 spacing), energies
    x (1 + N(0, 0.05)), seed 5; computed on the GPU).  Times, with CUDA events
    after W warm-up repetitions, K repetitions of the forward run (checkpoints
    every 5 steps, grid density) and of the backward pass (the grid-density
    adjoint, then per segment the recomputed steps and sph_step_bwd over
    them), and reports the gradient evaluations per second."""
    import torch
    from paper_1807_01341_gb300 import adjoint, build, sim
    from sph_ics import workloads
    build.build()
    torch.cuda.set_device(0)
    name = "c4_clumpy_32k"
    ic = workloads.make(name)
    n = ic["pos"].shape[0]
    n_steps, n_grid, k = workloads.STEPS[name], 32, 5
    params = sim.Params(**workloads.PARAMS[name], **DEFAULT_LAUNCH)
    run = adjoint.Run(params, ic["m"], ic["h0"], n_steps, n_grid, checkpoint_every=k)
    dev = torch.device("cuda")
    pos0 = torch.as_tensor(ic["pos"], dtype=torch.float64, device=dev)
    vel0 = torch.as_tensor(ic["vel"], dtype=torch.float32, device=dev)
    u0 = torch.as_tensor(np.broadcast_to(np.asarray(ic["u"], np.float64), (n,)).copy(),
                         dtype=torch.float32, device=dev)
    rng = np.random.default_rng(5)
    posp = torch.as_tensor((ic["pos"] + rng.normal(0.0, 0.05 / 32, size=ic["pos"].shape)) % 1.0,
                           dtype=torch.float64, device=dev)
    up = u0 * torch.as_tensor(1.0 + 0.05 * rng.normal(size=n), dtype=torch.float32, device=dev)
    target = run.forward(posp, vel0, up).clone()
    fwd, bwd = [], []
    loss = grad_rms = None
    for rep in range(args.warmup + args.steps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record()
        rho = run.forward(pos0, vel0, u0)
        diff = rho - target
        e[1].record()
        gpos, gvel, gu = run.backward(2.0 * diff)
        e[2].record()
        torch.cuda.synchronize()
        if rep >= args.warmup:
            fwd.append(e[0].elapsed_time(e[1]))
            bwd.append(e[1].elapsed_time(e[2]))
        loss = float((diff * diff).sum())
        grad_rms = float(gpos.pow(2).mean().sqrt())
    run.close()
    f, b = statistics.median(fwd), statistics.median(bwd)
    line = {"experiment": "reverse pass of the differentiation workload (checkpoint-and-recompute)",
            "workload": name, "n_particles": n, "steps": n_steps, "grid": n_grid,
            "checkpoint_every": k, "repetitions": args.steps, "warmup": args.warmup,
            "data": "synthetic", "forward_ms": f, "backward_ms": b, "backward_over_forward": b / f,
            "gradients_per_s": 1e3 / (f + b), "loss": loss, "grad_pos_rms": grad_rms,
            "timing": "CUDA events, median over repetitions; the backward includes the "
                      "recomputation of every segment"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# oracle on a bounded sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(ic, sample=2048, seed=0):
    """The FP64 oracle on a seeded sample of active particles of the workload:
    its density loop with the smoothing-length iteration (from the same initial
    h) and its force loop for the sample (neighbour h, rho, f, P, c taken from
    the initial state: the loop's cost and pair count do not depend on them).
    Returns useful pairs, seconds, threads."""
    import oracle
    from sph_ics import subsample_active
    n = ic["pos"].shape[0]
    act = subsample_active(n, sample, seed)
    gamma = 5.0 / 3.0
    t0 = time.perf_counter()
    d = oracle.density(ic["pos"], ic["m"], ic["h0"], act)
    t1 = time.perf_counter()
    h = np.where(act == 1, d["h"], ic["h0"])
    rho = np.where(act == 1, d["rho"], ic["m"] * (1.2348 / ic["h0"]) ** 3)
    f = np.ones(n)
    A = oracle.entropy_from_u(ic["u"], rho, gamma)
    P, cs = oracle.eos(A, rho, gamma)
    t2 = time.perf_counter()
    fr = oracle.force(ic["pos"], ic["vel"], ic["m"], h, rho, f, P, cs, act)
    t3 = time.perf_counter()
    pairs = int(d["count"][act == 1].sum()) + int(fr["count"][act == 1].sum())
    return dict(pairs=pairs, seconds=(t1 - t0) + (t3 - t2), threads=oracle.num_threads(),
                sample=f"{sample} seeded active particles of the {n}-particle workload: "
                       "density with h iteration + force, FP64, cell-grid neighbour search")


def run_reference(args, rank, world):
    import oracle
    from sph_ics import workloads
    oracle.build()
    ic = workloads.make(args.workload)
    runs = []
    for k in range(args.warmup + args.steps):
        r = oracle_sample(ic, args.ref_sample, seed=k)
        if k >= args.warmup:
            runs.append(r)
    pairs = sum(r["pairs"] for r in runs)
    secs = sum(r["seconds"] for r in runs)
    v = pairs / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "form": "oracle sample"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": runs[0]["threads"],
                             "kind": "oracle", "sample": runs[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=2048)
    ap.add_argument("--cpu-sample", type=int, default=2048)
    ap.add_argument("--launch", default=None,
                    help="launch knobs, e.g. 'list_cap=128,staging_depth=2' (with "
                         "--no-autotune: used as given; otherwise the autotuner's start)")
    ap.add_argument("--adjoint", action="store_true",
                    help="instead of the benchmark line, time the forward and reverse pass "
                         "of the differentiation workload")
    ap.add_argument("--ablation", action="store_true",
                    help="instead of the benchmark line, print the comparison of "
                         "relevant-only drift, drift-all and one global step")
    args = ap.parse_args()
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank, world)
        return

    if args.ablation:
        if rank == 0:
            run_ablation(args)
        return
    if args.adjoint:
        if rank == 0:
            run_adjoint(args)
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    out = run_ours(args, rank, world)
    total_ms = out["total_ms"]
    pairs = out["pairs"]
    e2e_ms = out["e2e_ms"]
    if world > 1:
        (total_ms, e2e_ms), (pairs_all, e2e_pairs) = reduce_over_ranks(
            [total_ms, e2e_ms], [float(pairs), float(out["e2e_pairs"])], "cuda")
    else:
        pairs_all, e2e_pairs = float(pairs), float(out["e2e_pairs"])
    if rank == 0:
        res = out["res"]
        b = res["batched"]
        rf = out["roofline"]
        plain = None
        if "plain" in res:
            pr = res["plain"]
            pp = pr["counters"]["pairs_density"] + pr["counters"]["pairs_force"]
            plain = {"value": pp / (sum(pr["ms"]) / 1e3) * world, "ms_per_step":
                     sum(pr["ms"]) / len(pr["ms"]), "unit": UNIT}
        cpu = None
        if not args.no_cpu_baseline:
            r = oracle_sample(out["ic"], args.cpu_sample, seed=0)
            cpu = {"value": r["pairs"] / r["seconds"], "unit": UNIT, "cores": r["threads"],
                   "kind": "oracle", "sample": r["sample"]}
        c = b["counters"]
        # the roofline denominator: FP32 lanes of the SMs the device reports, at
        # the median SM clock sampled during the timed steps (else the maximum)
        mhz = b["clocks"].get("sm_mhz") or b["clocks"].get("sm_max_mhz") or 2070.0
        peak = fp32_peak(out["sms"], mhz)
        line = {
            "metric": METRIC, "value": pairs_all / (total_ms / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 pair arithmetic, f64 positions/h test",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_particles": out["n"],
                       "form": "batched (persistent kernels + CUDA graph)",
                       "steps_from": "initial conditions (step 0 all active)",
                       "l2": "flushed between timed steps (256 MiB write)",
                       "grid_cells_per_axis": b["grid"][0], "leaves": b["grid"][1],
                       "launch": out["tuned"],
                       "autotuned": not args.no_autotune},
            "autotune": out["tune_info"],
            "plain": plain,
            "e2e": {"value": e2e_pairs / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": out["h2d"], "d2h_bytes_per_step": out["h2d"]},
            "roofline": {"bound": "alu", "kernel": rf["kernel"], "achieved": rf["achieved"],
                         "peak": peak, "unit": "TFLOP/s",
                         "frac": rf["achieved"] / peak,
                         "traffic": profiled_traffic(rf["kernel"], args.workload, out["tuned"]),
                         "peak_source": f"{out['sms']} SMs (queried) x {FP32_LANES_PER_SM} FP32 "
                                        f"lanes x 2 x {mhz:.0f} MHz (median SM clock sampled "
                                        "during the timed steps)",
                         "achieved_counts": (
                             "algorithmic FLOPs of the useful pairs (at the final h)"
                             if rf["kernel"] == "density" else
                             "algorithmic FLOPs of the useful pairs (r < max(H_i, H_j))"),
                         "executed": {"achieved": rf["executed"], "frac": rf["executed"] / peak,
                                      "counts": (
                                          "FP32 work executed: every candidate test and every "
                                          "pair term of every h iteration"
                                          if rf["kernel"] == "density" else
                                          "FP32 work executed: every candidate test and every "
                                          "pair term")},
                         "launch_ms": rf["per_launch_ms"], "density_ms": rf["density_ms"],
                         "force_ms": rf["force_ms"]},
            "cell_build_ms": out["build_ms"],
            "cpu_baseline": cpu,
            "gpu_launches": b["launches"],
            # useful pairs / tested (record, particle) pairs; the density loop's
            # tests include every h iteration, its useful pairs the final one
            "candidate_efficiency": {
                "density": c["pairs_density"] / max(c["cand_density"], 1),
                "force": c["pairs_force"] / max(c["cand_force"], 1)},
            "counters": {k: c[k] for k in ("pairs_density", "pairs_force", "cand_density",
                                           "cand_force", "iters_density", "gathers_density",
                                           "list_overflows", "evals_density", "active_particles",
                                           "steps", "rebuilds", "redone_steps")},
            "clocks": b["clocks"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
