"""Host logic of bench.py that needs no GPU: the DRAM traffic of a fused launch is
the per-node figure of the committed ncu capture scaled by the node count, and only
while the kernel sources are those the capture was taken on; the clock sampler
reports the throttle reasons that were active; the growth-rate fit."""
import os
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _copy_sources(tmp_path):
    root = tmp_path / "repo"
    for rel in bench.KERNEL_SOURCES:
        (root / os.path.dirname(rel)).mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), root / rel)
    return root


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_traffic_scales_per_node_while_the_sources_match(tmp_path, monkeypatch, storage):
    root = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    per_node, sha = bench.FUSED_TRAFFIC[storage]
    assert bench.kernel_source_sha() == sha          # the committed figure is current
    assert bench.fused_traffic(1, storage) == per_node > 1000
    assert bench.fused_traffic(4096 * 4096, storage) == pytest.approx(per_node * 4096 * 4096)
    # the profile summary names the same sources and figure
    name = "step_fused_kernel_kolmogorov_512x512_nq32" + ("" if storage == "fp32" else "_fp16")
    text = open(os.path.join(ROOT, "profiles", name + ".md")).read()
    assert sha in text and f"**{per_node:.0f} B**" in text
    # any change of a kernel source makes the counters stale: no traffic
    with open(root / bench.KERNEL_SOURCES[1], "ab") as f:
        f.write(b"\n// changed\n")
    assert bench.fused_traffic(4096 * 4096, storage) is None


def test_traffic_is_none_without_a_capture(tmp_path, monkeypatch):
    root = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.fused_traffic(100, "fp8") is None


def test_growth_rate_fit_uses_the_second_half():
    t = np.arange(1, 21) * 9.0
    e = np.where(t < 90, 1.0, np.exp(2e-3 * (t - 90)))   # flat, then growing
    assert bench._growth_rate(t, e) == pytest.approx(2e-3, rel=1e-9)


def test_clock_sampler_parses_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("0, 2070, 2070, 400.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                    "0, 2070, 2070, 420.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                    "garbage line\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc, s.path, s.out = Done(), str(path), open(os.devnull, "w")
    r = s.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["power_w_max"] == 1390.0
    assert r["reasons"] == ["sw_power_cap"]
    assert not path.exists()
