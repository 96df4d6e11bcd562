"""Shared helpers of the GPU parity tests (the oracle is only used as the reference)."""
from __future__ import annotations

import numpy as np

ETA = 1.2348
GAMMA = 5.0 / 3.0


def gpu_setup(ic, params, bins=None, ti=0):
    """Context + particles built into cells; optional per-particle bins
    (steps start at tick 0 and end at the next multiple of 2^bin)."""
    import torch
    from paper_1807_01341_gb300 import sim
    n = ic["pos"].shape[0]
    ctx = sim.Context(params, max(n, 1))
    p = sim.Particles.from_ics(ic)
    if bins is not None:
        b = np.asarray(bins, dtype=np.int64)
        p.bin.copy_(torch.as_tensor(b.astype(np.int8)))
        p.ti_begin.zero_()
        p.ti_end.copy_(torch.as_tensor(np.left_shift(1, b)))
        p.ti_drift.fill_(ti)
    ctx.build_cells(p)
    return ctx, p


def sorted_inputs(ic, perm):
    """The IC arrays in the library's cell order (out[k] = in[perm[k]])."""
    return {k: (v[perm] if isinstance(v, np.ndarray) and v.shape[:1] == ic["pos"].shape[:1] else v)
            for k, v in ic.items() if k != "meta"}


def wrapped(pos, box=1.0):
    x = pos.copy()
    x[x < 0] += box
    x[x >= box] -= box
    return x


def band_pairs(pos, h, idx, box=1.0, band=1e-6, gamma_k=1.825742):
    """Per particle i in idx: number of j with |r_ij^2 - H_i^2| < band H_i^2
    (pairs whose neighbour status FP32 rounding may flip)."""
    out = np.zeros(len(idx), dtype=np.int64)
    for k, i in enumerate(idx):
        d = pos - pos[i]
        d -= box * np.round(d / box)
        r2 = (d * d).sum(1)
        H2 = (gamma_k * h[i]) ** 2
        out[k] = int((np.abs(r2 - H2) < band * H2).sum())
    return out


def band_pairs_sym(pos, h, idx, box=1.0, band=1e-6, gamma_k=1.825742):
    """As band_pairs for the symmetric force support max(H_i, H_j)."""
    out = np.zeros(len(idx), dtype=np.int64)
    H = gamma_k * h
    for k, i in enumerate(idx):
        d = pos - pos[i]
        d -= box * np.round(d / box)
        r2 = (d * d).sum(1)
        R2 = np.maximum(H[i], H) ** 2
        out[k] = int((np.abs(r2 - R2) < band * R2).sum())
    return out
