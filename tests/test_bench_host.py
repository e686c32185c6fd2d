"""Host-side checks of bench.py (no GPU): the reference arm's JSON contract, the
workload description both arms share, and the partner-tile count behind the
SpMM's on-chip roofline."""
import importlib.util
import json
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_partner_tiles(bench):
    """Partner tiles per 1024-state tile: the 12 single-site flips above the tile bits of
    the 22-spin transverse-field model, every tile; for all-to-all XX+YY (J^x = J^y) the
    12 (15) groups of one high and one low spin, every tile, plus the C(12,2) = 66
    (C(15,2) = 105) pairs of high spins, each copied only by the half of the tiles where
    the two spins differ; none for a 10-spin chain (all flips inside the tile)."""
    import workloads as W
    assert bench._partner_tiles(W.config_c2(0)["spec"]) == 12
    assert bench._partner_tiles(W.long_range_xxz(22, 1, 1.0, 1.0, 0.1)) == 12 + 66 / 2
    assert bench._partner_tiles(W.config_c3()["spec"]) == 15 + 105 / 2
    assert bench._partner_tiles(W.config_c1()["spec"]) == 0
    spec = W.long_range_xxz(22, 1, 1.0, 1.0, 0.1)
    spec.jy[:] = 0.5 * spec.jx  # J^x != J^y: every pair hops, every tile copies it
    assert bench._partner_tiles(spec) == 12 + 66


def test_both_arms_describe_the_same_workload(bench):
    a = types.SimpleNamespace(n_sites=22, k=60, n_v=32, model="tfim")
    c = bench._config(a, 1)
    assert c["workload"] == bench.WORKLOAD and c["block_columns"] == 128 and c["n_sys"] == 2
    assert bench._bench_case(a)
    x = types.SimpleNamespace(n_sites=24, k=6, n_v=64, model="xxz")
    cx = bench._config(x, 1)
    assert not bench._bench_case(x) and cx["workload"].startswith("profiling_xxz_N24")
    assert cx["block_columns"] == 128 and cx["n_sys"] == 1


def test_reference_arm_prints_the_contract_line():
    """`--impl reference` times the oracle on the host and prints one JSON line with the
    contract's keys (one bounded sample: about ten seconds of CPU)."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "0", "--oracle-cores", "2", "--ref-steps", "1"],
                       capture_output=True, text=True, env=env, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "lr_tfim_N22_Ns2_nv32_k60_beta1_fp32"
    # the steps it reports were run: their time fits the run's own wall time
    assert d["steps"] == 2 and d["ms_per_step"] * d["steps"] <= 1000.0 * d["wall_s"]
    assert d["cpu_baseline"]["cores"] == 2


def test_world_size_must_match_gpus(bench, monkeypatch):
    """Under torchrun `--gpus N` must equal the world size; outside it N = 1 runs here."""
    a = types.SimpleNamespace(gpus=2)
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench._launch_ranks(a) == 2
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench._launch_ranks(a) is None
    monkeypatch.delenv("WORLD_SIZE")
    assert bench._launch_ranks(types.SimpleNamespace(gpus=1)) is None
