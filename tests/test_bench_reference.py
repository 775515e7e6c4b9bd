"""The bench's reference arm (the FP64 oracle timed on the host) keeps the
one-JSON-line contract: same metric and unit as the GPU arm, impl "reference",
a cpu_baseline describing the run and an e2e with no host-device bytes.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "energyscapes/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == bench.WORKLOAD
    for k in ("n_mics", "n_samples", "n_dirs"):
        assert d["config"][k] == getattr(bench, k.upper()), k
    # ms_per_step is the measured step; value scales the sampled DAS time to all directions
    vb = d["value_basis"]
    assert vb["scale_factor"] == bench.N_DIRS / vb["dirs_per_step"]
    t_full = vb["matched_filter_s_per_step"] + vb["scale_factor"] * vb["das_s_per_step"]
    assert abs(d["value"] - 1.0 / t_full) <= 1e-9 * d["value"]
    assert d["ms_per_step"] < 1e3 * t_full


def test_all_cores_oracle_baseline_runs_in_spawned_workers():
    import bench
    rate, procs = bench.oracle_pool_rate(2, procs=2)
    assert procs == 2 and rate > 0
    entry = bench.all_cores_baseline(2)
    assert entry["kind"] == "oracle" and entry["cores"] >= 1 and entry["value"] > 0


def test_error_vs_oracle_entry_aligns_sampled_rows():
    # the bench's oracle sample rows line up with the full energyscape's rows: the oracle
    # against itself gives zero error and the same peak; a perturbed copy shows its error
    import numpy as np

    import bench
    import oracle
    import synth
    cfg = synth.single_sensor(n_samples=4096, n_dirs=20)
    _, _, _, pick, o_td, o_fd = bench.oracle_sample(cfg, 6, seed=3)
    full_td = oracle.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"])
    full_fd = oracle.energyscape(cfg["x"], cfg["chirp"], cfg["mic_xyz"], cfg["dirs"], cfg["fs"], cfg["c"], path="fd")
    e = bench.oracle_error_entry(pick, {"td": (o_td, full_td), "fd": (o_fd, full_fd)})
    assert e["directions_sampled"] == 6
    for k in ("td", "fd"):
        assert e[k]["max_abs_err_over_peak"] < 1e-12 and e[k]["peak_index_match"]
    bumped = full_td.copy()
    bumped[pick[2], 7] += 1e-3 * o_td.max()
    assert abs(bench.oracle_error_entry(pick, {"td": (o_td, bumped)})["td"]["max_abs_err_over_peak"] - 1e-3) < 1e-9
