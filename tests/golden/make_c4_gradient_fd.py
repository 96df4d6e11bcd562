"""Writes c4_gradient_fd.json: central finite differences of the oracle's loss
for the differentiation workload (32^3 jittered lattice with 8 Plummer clumps
of 512, 20 kick-drift-kick steps, SPH density on a 32^3 grid against the
target of the same run from perturbed initial conditions: positions displaced
by N(0, 0.05 spacing), energies scaled by 1 + N(0, 0.05)), on 64 seeded
coordinates of the initial positions (step 1e-6) and on the internal energies
of 16 seeded clump particles (step 1e-4 relative: within 20 steps u moves the
loss only through the clumps' pressure, and a smaller step would not resolve
that change of the loss).

Calls only the oracle.  Run:  python tests/golden/make_c4_gradient_fd.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import sph_ics  # noqa: E402
from oracle import adjoint as adj  # noqa: E402

RECIPE = dict(nside=32, n_clumps=8, per_clump=512, seed=4, n_steps=20, n_grid=32,
              cfl=0.1, dt_min=2.0 ** -24, bin_cap=12, target_seed=5, target_sigma_cells=0.05,
              target_u_sigma=0.05,
              coord_seed=2024, n_pos=64, n_u=16, eps_pos=1e-6, eps_u_rel=1e-4)


def workload():
    r = RECIPE
    ic = sph_ics.clumpy_lattice(r["nside"], r["n_clumps"], r["per_clump"], seed=r["seed"])
    kw = dict(cfl=r["cfl"], dt_min=r["dt_min"], bin_cap=r["bin_cap"])
    rng = np.random.default_rng(r["target_seed"])
    icp = dict(ic)
    icp["pos"] = (ic["pos"] + rng.normal(0.0, r["target_sigma_cells"] / r["nside"],
                                          size=ic["pos"].shape)) % 1.0
    n = ic["pos"].shape[0]
    icp["u"] = np.asarray(ic["u"], dtype=np.float64) * (1.0 + r["target_u_sigma"] *
                                                        rng.normal(size=n))
    _, _, simt = adj.oracle_loss(icp, r["n_steps"], r["n_grid"], np.zeros(r["n_grid"] ** 3), **kw)
    target = adj.grid_density(simt.pos, simt.h, simt.m, r["n_grid"])
    return ic, kw, target


def coordinates(ic):
    """Seeded position coordinates over all particles; energy coordinates over
    the clump particles (initial h below half the lattice value)."""
    r = RECIPE
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(r["coord_seed"])
    pos = [(int(rng.integers(n)), int(rng.integers(3))) for _ in range(r["n_pos"])]
    clump = np.nonzero(ic["h0"] < 0.5 * np.median(ic["h0"]))[0]
    u = [int(clump[rng.integers(clump.size)]) for _ in range(r["n_u"])]
    return pos, u


def main():
    r = RECIPE
    t0 = time.time()
    ic, kw, target = workload()
    n = ic["pos"].shape[0]
    L0, bins0, _ = adj.oracle_loss(ic, r["n_steps"], r["n_grid"], target, **kw)
    pos_c, u_c = coordinates(ic)
    u0 = np.broadcast_to(np.asarray(ic["u"], dtype=np.float64), (n,)).copy()
    out_pos, out_u = [], []
    for (i, k) in pos_c:
        vals, same = [], True
        for s in (1.0, -1.0):
            p = ic["pos"].copy()
            p[i, k] += s * r["eps_pos"]
            L, b, _ = adj.oracle_loss(ic, r["n_steps"], r["n_grid"], target, pos0=p, **kw)
            vals.append(L)
            same = same and bool((b == bins0).all())
        out_pos.append(dict(i=i, k=k, fd=(vals[0] - vals[1]) / (2 * r["eps_pos"]), bins_same=same))
    for i in u_c:
        vals, same = [], True
        eps = r["eps_u_rel"] * u0[i]
        for s in (1.0, -1.0):
            u = u0.copy()
            u[i] += s * eps
            L, b, _ = adj.oracle_loss(ic, r["n_steps"], r["n_grid"], target, u0=u, **kw)
            vals.append(L)
            same = same and bool((b == bins0).all())
        out_u.append(dict(i=i, fd=(vals[0] - vals[1]) / (2 * eps), bins_same=same))
    doc = dict(description=__doc__.strip().splitlines()[0], recipe=RECIPE, loss=L0,
               pos=out_pos, u=out_u, seconds=time.time() - t0)
    with open(os.path.join(HERE, "c4_gradient_fd.json"), "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote c4_gradient_fd.json in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
