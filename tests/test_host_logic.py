"""Host-side logic of the benchmark and the autotuner (no GPU): when a profile's
DRAM traffic is reported, and which launch configuration the autotuner keeps."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _profile(tmp_path, digest, launch, traffic=123456):
    import bench
    text = (f"# k_density<1>\n\nkernel_source_digest: {digest}\n"
            f"launch_config: {bench.launch_key(launch)}\ntraffic_bytes_per_launch: {traffic}\n")
    (tmp_path / "k_density_w.md").write_text(text)


def test_traffic_reported_only_for_matching_sources_and_launch(tmp_path):
    import bench
    launch = dict(bench.DEFAULT_LAUNCH)
    _profile(tmp_path, bench.kernel_source_digest(), launch)
    assert bench.profiled_traffic("density", "w", launch, str(tmp_path)) == 123456
    other = dict(launch, leaf_max=32)
    assert bench.profiled_traffic("density", "w", other, str(tmp_path)) is None
    _profile(tmp_path, "0" * 16, launch)  # counters taken from other sources
    assert bench.profiled_traffic("density", "w", launch, str(tmp_path)) is None
    assert bench.profiled_traffic("force", "w", launch, str(tmp_path)) is None  # no summary


def _fake_trials(monkeypatch, rates):
    from paper_1807_01341_gb300 import autotune
    calls = []

    def trial(ic, base, cand, steps, flush=None):
        calls.append(cand)
        return dict(cand=cand, ms=1.0, pairs=1, rate=rates[len(calls) - 1])
    monkeypatch.setattr(autotune, "trial", trial)
    return autotune, calls


@pytest.mark.parametrize("rates,expect", [
    ([1.00, 1.015, 0.9], 0),   # 1.5 % faster: inside the margin, the default stays
    ([1.00, 1.03, 0.9], 1),    # 3 % faster: chosen
    ([1.00, 0.98, 0.97], 0),   # the default is fastest
])
def test_autotune_keeps_default_inside_margin(monkeypatch, tmp_path, rates, expect):
    pytest.importorskip("torch")
    autotune, calls = _fake_trials(monkeypatch, rates)
    cands = [dict(threads_per_particle=1, leaf_max=16, cell_margin=2.0),
             dict(threads_per_particle=1, leaf_max=24, cell_margin=2.5),
             dict(threads_per_particle=2, leaf_max=16, cell_margin=2.0)]
    import numpy as np
    ic = {"pos": np.zeros((10, 3))}
    cache = str(tmp_path / "tune.json")
    got = autotune.tune(ic, {}, "w", steps=3, candidates=cands, cache_path=cache)
    assert {k: got[k] for k in cands[0]} == cands[expect]
    assert not got["cached"] and len(calls) == 3
    # the choice is cached per workload key, particle count and step count
    again = autotune.tune(ic, {}, "w", steps=3, candidates=cands, cache_path=cache)
    assert again["cached"] and {k: again[k] for k in cands[0]} == cands[expect]
    assert len(calls) == 3
    with open(cache) as f:
        assert "w:n=10:steps=3:knobs=cell_margin,leaf_max,threads_per_particle" in json.load(f)
