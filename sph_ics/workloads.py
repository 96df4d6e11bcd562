"""Named synthetic workloads: an initial-condition recipe plus the run
parameters of each, shared by the benchmark and the tests.

C1  4,096-particle jittered lattice (16^3), all active, one density + force pass.
C2  262,144-particle Sedov blast (64^3), 100 kick-drift-kick steps, CFL 0.1,
    time bins up to 2^10.
C3  2,097,152 particles: 1,048,576 uniform background + 64 Plummer spheres of
    16,384 (scale radii log-uniform in [1e-3, 3e-2]), 50 steps, bins spanning
    ~2^13; the benchmark workload (batched vs plain).
C4  32,768-particle jittered 32^3 lattice with 4,096 particles moved into 8
    Plummer clumps of 512, 20 steps, bins up to 2^12: the differentiation
    workload (loss on the final density sampled on a 32^3 grid).
C5  16,777,216-particle Zel'dovich-displaced 256^3 lattice, 20 steps, bins up
    to 2^14.
"""
from __future__ import annotations

import sph_ics

# Run parameters (a subset of the library's sph_params) per workload.
PARAMS = {
    "c1_lattice_4k": dict(cfl=0.1, bin_cap=0, dt_min=1e-4),
    "c2_sedov_262k": dict(cfl=0.1, bin_cap=10, dt_min=2.0 ** -24),
    "c3_clustered_2m": dict(cfl=0.1, bin_cap=20, dt_min=2.0 ** -28),
    "c4_clumpy_32k": dict(cfl=0.1, bin_cap=12, dt_min=2.0 ** -24),
    "c5_zeldovich_16m": dict(cfl=0.1, bin_cap=14, dt_min=2.0 ** -24),
}

STEPS = {"c1_lattice_4k": 1, "c2_sedov_262k": 100, "c3_clustered_2m": 50,
         "c4_clumpy_32k": 20, "c5_zeldovich_16m": 20}


def make(name: str):
    if name == "c1_lattice_4k":
        return sph_ics.lattice(16, 0.1, seed=1)
    if name == "c2_sedov_262k":
        return sph_ics.sedov(64, seed=2)
    if name == "c3_clustered_2m":
        return sph_ics.clustered(seed=3)
    if name == "c4_clumpy_32k":
        return sph_ics.clumpy_lattice(32, 8, 512, seed=4)
    if name == "c5_zeldovich_16m":
        return sph_ics.zeldovich(256, seed=5)
    raise KeyError(name)
