"""The per-step trace (trace.py) and the bin histogram (sph_get_bin_counts)
against the library's counters and the state."""
import json

import numpy as np
import pytest

import sph_ics
from _gpu_helpers import gpu_setup

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_01341_gb300 import build
    build.build()
    from paper_1807_01341_gb300 import sim as S
    return S


def test_trace_records_match_counters_and_state(sim, tmp_path):
    """Eight steps of a clumpy set with individual bins: the records' active
    counts, pairs and iterations add up to the run's counters; each record's
    largest active bin is ctz(tick); the bin histogram after each step counts
    every particle and equals the histogram of the state's own bins; the
    step time covers the two pair loops; the JSON lines read back equal."""
    from paper_1807_01341_gb300 import trace
    ic = sph_ics.clumpy_lattice(nside=10, n_clumps=1, per_clump=150, seed=31)
    n = ic["pos"].shape[0]
    rng = np.random.default_rng(31)
    ic["vel"] = rng.normal(scale=0.1, size=(n, 3))
    ctx, p = gpu_setup(ic, sim.Params(cfl=0.1, dt_min=1e-6, bin_cap=14))
    ctx.begin_run()
    path = str(tmp_path / "trace.jsonl")
    recs = trace.run(ctx, p, 8, out=path, energy=True)
    c = ctx.counters()
    assert [r["step"] for r in recs] == list(range(1, 9))
    assert sum(r["active"] for r in recs) == c["active_particles"]
    assert sum(r["pairs_density"] for r in recs) == c["pairs_density"]
    assert sum(r["pairs_force"] for r in recs) == c["pairs_force"]
    assert sum(r["iters_density"] for r in recs) == c["iters_density"]
    assert recs[0]["active"] == n and recs[0]["ti"] == 0
    for r in recs:
        assert r["max_active_bin"] == (63 if r["ti"] == 0 else (r["ti"] & -r["ti"]).bit_length() - 1)
        assert sum(r["bins"]) == n
        assert r["ti_next"] > r["ti"]
        assert r["step_ms"] >= r["density_ms"] + r["force_ms"] > 0.0
        assert r["diagnostics"]["mass"] > 0.0
    st = p.numpy()
    hist = np.bincount(st["bin"].astype(np.int64), minlength=len(recs[-1]["bins"]))
    assert list(hist[:len(recs[-1]["bins"])]) == recs[-1]["bins"]
    assert len(set(np.nonzero(hist)[0])) > 1
    with open(path) as f:
        back = [json.loads(line) for line in f]
    assert back == json.loads(json.dumps(recs))
    ctx.close()
