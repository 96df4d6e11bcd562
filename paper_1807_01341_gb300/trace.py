"""Per-step trace of a run: one record (and, on request, one JSON line) per
kick-drift-kick step.

Each record holds what the paper follows step by step (the wall-clock time
of a step against its active count, Sec. IV-B, and the occupancy of the time
bins, Fig. 1): the step's tick and time, the largest active bin (Eq. 2: every bin
n with the tick a multiple of 2^n), the active particles, the useful pairs
and density iterations of the step, the time of the step and of its two
pair-loop kernels (CUDA events on the launching stream), the rebuilds it
needed, the bin histogram after it and, optionally, the FP64 energy and
momentum (sph_diagnostics).  Library calls only.
"""
from __future__ import annotations

import json

import torch

from . import _lib
from .sim import Context, Particles


def max_active_bin(ti: int) -> int:
    """The largest bin whose particles are active at tick ti (ctz(ti); every
    bin at tick 0)."""
    return (ti & -ti).bit_length() - 1 if ti > 0 else 63


def run(ctx: Context, p: Particles, n_steps: int, out=None, form: int = _lib.SPH_FORM_BATCHED,
        stream=None, energy: bool = False) -> list:
    """Advances n_steps steps (rebuilding the cells when the library asks)
    and returns their records; with `out` (a path, appended to, or an open
    text file) each record is also written as one JSON line."""
    stream = stream if stream is not None else torch.cuda.current_stream()
    fh = open(out, "a") if isinstance(out, str) else out
    records = []
    ctx.set_profiling(True)
    try:
        for _ in range(n_steps):
            c0 = ctx.counters()
            ctx.reset_kernel_times()
            ms, attempts = 0.0, 0
            while True:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.step_async(p, form, stream)
                e1.record(stream)
                done = ctx.step_sync(p, stream)
                ms += e0.elapsed_time(e1)
                attempts += 1
                if done:
                    break
            c1 = ctx.counters()
            kt = ctx.kernel_times()
            ti, ti_next = ctx.get_time()
            bins = ctx.bin_counts(64, stream)
            top = max((b for b, c in enumerate(bins) if c), default=-1)
            rec = {
                "step": int(c1["steps"]), "ti": ti, "t": ctx.params.t_begin + ti * ctx.params.dt_min,
                "ti_next": ti_next, "max_active_bin": max_active_bin(ti),
                "active": c1["active_particles"] - c0["active_particles"],
                "pairs_density": c1["pairs_density"] - c0["pairs_density"],
                "pairs_force": c1["pairs_force"] - c0["pairs_force"],
                "iters_density": c1["iters_density"] - c0["iters_density"],
                "step_ms": ms, "density_ms": kt["density_ms"], "force_ms": kt["force_ms"],
                "attempts": attempts, "rebuilds": c1["rebuilds"] - c0["rebuilds"],
                "bins": bins[:top + 1],
            }
            if energy:
                rec["diagnostics"] = ctx.diagnostics(p, ti, stream)
            records.append(rec)
            if fh is not None:
                fh.write(json.dumps(rec) + "\n")
                fh.flush()
    finally:
        if isinstance(out, str) and fh is not None:
            fh.close()
    return records
