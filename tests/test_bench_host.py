"""Host-side logic of bench.py that needs no GPU: the traffic figure's source
guard, the clock-sample summary and the per-step kernel count."""
import os
import types

import bench


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    import hashlib
    sources = {rel: hashlib.sha256(open(os.path.join(bench.ROOT, rel), "rb").read()).hexdigest()
               for rel in bench.RASTER_BWD_TRAFFIC["sources"]}
    same = dict(bench.RASTER_BWD_TRAFFIC, sources=sources, blend_bytes=1000, projection_bytes=500, pairs=10,
                n=100, views=2)
    monkeypatch.setattr(bench, "RASTER_BWD_TRAFFIC", same)
    assert bench.raster_bwd_traffic() == 1500
    assert bench.raster_bwd_traffic(40) == 4500  # the blend's bytes scaled by the pairs
    # the projection reverse's by its algorithmic bytes: 2 -> 8 views of 112-byte cotangent rows, each
    # read and cleared, next to the 236-byte parameter column and two 236-byte output columns (SH degree 3,
    # two probes)
    assert bench.projection_reverse_bytes(100, 2) == 100 * (236 + 2 * 2 * 112 + 2 * 236)
    want = 4000 + 500 * (236 + 2 * 8 * 112 + 472) / (236 + 2 * 2 * 112 + 472)
    assert bench.raster_bwd_traffic(40, 100, 8) == round(want)
    changed = dict(same, sources=dict(sources))
    first = next(iter(changed["sources"]))
    changed["sources"][first] = "0" * 64
    monkeypatch.setattr(bench, "RASTER_BWD_TRAFFIC", changed)
    assert bench.raster_bwd_traffic() is None


def test_clock_summary_reads_samples_and_removes_them(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1401.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbled line",
    ]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    c.proc = object()  # as if nvidia-smi had been started
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.path)
    # without nvidia-smi the summary says so instead of inventing clocks
    c2 = bench.ClockSampler(0)
    assert c2.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_kernel_count_per_step():
    # 1920 x 1080 in 16 x 16 tiles: 120 x 68 tiles per view, 8 views -> 16 tile
    # bits, two 8-bit pair passes; 4 record passes
    eng = types.SimpleNamespace(Tx=120, Ty=68)
    # step counter 1, projection 1, sort 40, forward 1, reverse 3 (workspace
    # check, reverse blend, projection reverse), update 1; the ncu launch list of
    # a step shows the same kernels
    assert bench.kernel_launches_per_step(eng) == 47


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference`: the oracle on the host cores, whole steps
    (here of a 20k-Gaussian scene), in the same JSON contract as the CUDA arm."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.abspath(bench.__file__))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--n", "20000"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    # the line reports the whole steps it timed, nothing scaled
    assert abs(d["value"] * d["ms_per_step"] * 1e-3 - 1.0) < 1e-9
    assert "nothing scaled" in d["cpu_baseline"]["sample"]
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
