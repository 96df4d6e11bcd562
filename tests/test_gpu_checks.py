"""The build with device bounds checks (libsph_gb300_checks.so, -DSPH_CHECKS).

Each case runs in a child process that loads the checks build
(SPH_GB300_CHECKS=1), so that the parent keeps the plain library:
  * whole steps in every form agree with the plain library (integers exactly,
    floating point to rounding), with no check failing;
  * a work-group index planted past the last group (test_bad_group, accepted
    only by the checks build) is caught by the SPH_CHECK_GROUP check before it
    is used: the step stops with SPH_ERR_BOUNDS, the report names the site, the
    index and the bound, nothing traps, and after the status is cleared the
    same context completes the step like a run that never saw the index."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if __name__ != "__main__":
    pytestmark = pytest.mark.gpu

STEP_PARAMS = dict(dt_min=1e-6, bin_cap=14, cfl=0.1)
FIELDS = ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "A", "Adot", "h", "rho", "f", "P",
          "c", "vsig", "bin", "ti_begin", "ti_end", "ti_drift", "active")


def _ic(seed=47):
    import sph_ics
    ic = sph_ics.clumpy_lattice(nside=12, n_clumps=1, per_clump=200, seed=seed)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(seed)
    ic["vel"] = rng.normal(scale=0.1, size=(n, 3))
    ic["u"] = rng.uniform(0.5, 2.0, n)
    return ic


def _run(mode):
    """Steps of the clumpy case in the library this process loaded; returns
    the final state and what the status word and the check report said."""
    import torch
    from paper_1807_01341_gb300 import _lib, sim
    ic = _ic()
    out = {}
    bad = 1 if mode == "plant" else 0
    ctx = sim.Context(sim.Params(**STEP_PARAMS, test_bad_group=bad), ic["pos"].shape[0])
    p = sim.Particles.from_ics(ic)
    ctx.build_cells(p)
    if mode == "plant":
        try:
            ctx.step(p, _lib.SPH_FORM_BATCHED)
            out["first_code"] = 0
        except _lib.SphError as e:
            out["first_code"] = e.code
        out["status"] = ctx.status()[0]
        out["report"] = ctx.check_report()
        out["steps_after_failure"] = ctx.counters()["steps"]
        ctx.clear_status()
        ctx.step(p, _lib.SPH_FORM_BATCHED)
    else:
        for form in (_lib.SPH_FORM_BATCHED, _lib.SPH_FORM_PLAIN, _lib.SPH_FORM_BATCHED_NOGRAPH):
            for _ in range(3):
                ctx.step(p, form)
    torch.cuda.synchronize()
    out["final_status"] = ctx.status()[0]
    out["final_report"] = ctx.check_report()
    out["steps"] = ctx.counters()["steps"]
    st = p.numpy()
    out["state"] = {k: st[k] for k in FIELDS}
    out["checks"] = _lib.load().sph_built_with_checks()
    ctx.close()
    return out


def _child(mode, tmp_path):
    path = str(tmp_path / f"{mode}.npy")
    env = dict(os.environ, SPH_GB300_CHECKS="1", PYTHONPATH=ROOT + os.pathsep + os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), mode, path], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(path, allow_pickle=True).item()


@pytest.fixture(scope="module")
def plain():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_01341_gb300 import build, _lib
    build.build()
    assert _lib.load().sph_built_with_checks() == 0
    return _lib


def test_checks_build_agrees_with_the_plain_library(plain, tmp_path):
    """No check fails over nine steps, and the state agrees with the plain
    library's: exactly for every integer result, to rounding for the floating
    point ones (the branches of the checks change where the compiler fuses a
    multiply and an add, so the two builds may round differently)."""
    got = _child("clean", tmp_path)
    assert got["checks"] == 1
    assert got["final_status"] == 0 and got["final_report"][0] == plain.SPH_CHECK_NONE
    ref = _run("clean")
    assert ref["checks"] == 0 and ref["steps"] == got["steps"] == 9
    a, b = got["state"], ref["state"]
    for k in ("bin", "ti_begin", "ti_end", "ti_drift", "active"):
        assert np.array_equal(a[k], b[k]), k
    d = np.stack([a[k] - b[k] for k in ("x", "y", "z")], 1)
    d -= np.round(d)
    assert np.abs(d).max() < 1e-9, np.abs(d).max()
    for k in ("h", "rho", "f", "P", "c", "vsig", "A"):
        rel = np.max(np.abs(a[k].astype(np.float64) / b[k] - 1))
        assert rel < 1e-5, (k, rel)
    for vec in (("vx", "vy", "vz"), ("ax", "ay", "az")):
        va = np.stack([a[k] for k in vec], 1).astype(np.float64)
        vb = np.stack([b[k] for k in vec], 1).astype(np.float64)
        err = np.abs(va - vb).max() / np.sqrt((vb ** 2).sum(1).mean())
        assert err < 1e-4, (vec, err)


def test_bounds_check_catches_a_planted_group(plain, tmp_path):
    got = _child("plant", tmp_path)
    assert got["checks"] == 1
    assert got["first_code"] == plain.SPH_ERR_BOUNDS
    assert got["status"] == plain.SPH_ERR_BOUNDS
    site, index, bound = got["report"]
    assert site == plain.SPH_CHECK_GROUP
    assert bound > 0 and index == bound + 7
    assert got["steps_after_failure"] == 0
    assert got["final_status"] == 0 and got["final_report"][0] == plain.SPH_CHECK_NONE
    assert got["steps"] == 1
    # the same step in the plain library, never disturbed
    import torch
    from paper_1807_01341_gb300 import sim
    ic = _ic()
    ctx = sim.Context(sim.Params(**STEP_PARAMS), ic["pos"].shape[0])
    p = sim.Particles.from_ics(ic)
    ctx.build_cells(p)
    ctx.step(p, plain.SPH_FORM_BATCHED)
    torch.cuda.synchronize()
    ref = p.numpy()
    ctx.close()
    st = got["state"]
    for k in ("x", "y", "z", "active", "ti_drift"):
        assert np.array_equal(st[k], ref[k]), k
    # the redone step starts its h iteration from partly updated guesses:
    # the same roots to the convergence tolerance
    for k in ("h", "rho"):
        assert np.max(np.abs(st[k] / ref[k] - 1)) < 1e-5, k
    a = np.stack([st["ax"], st["ay"], st["az"]], 1)
    a_ref = np.stack([ref["ax"], ref["ay"], ref["az"]], 1)
    assert np.max(np.abs(a - a_ref)) < 1e-4 * np.sqrt((a_ref ** 2).sum(1).mean())


if __name__ == "__main__":
    res = _run(sys.argv[1])
    np.save(sys.argv[2], res, allow_pickle=True)
