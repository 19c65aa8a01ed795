"""Host logic of bench.py that needs no GPU: the measured DRAM traffic is taken
from the committed ncu summary only while the kernel source still matches it,
and the clock sampler reports the throttle reasons that were active."""
import hashlib
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

NAME = "step_fused_kernel_kolmogorov_512x512_nq32"


def _copy_tree(tmp_path):
    """bench's inputs for the traffic lookup: the profile summaries and the kernel source."""
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "profiles"), root / "profiles")
    csrc = root / "paper_2201_10132_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "paper_2201_10132_gb300", "csrc", "tfkt_fused.cu"), csrc)
    return root


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_traffic_scales_per_node_while_the_source_matches(tmp_path, monkeypatch, storage):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    text = open(root / "profiles" / (NAME + ("" if storage == "fp32" else "_fp16") + ".md")).read()
    src = open(root / "paper_2201_10132_gb300" / "csrc" / "tfkt_fused.cu", "rb").read()
    assert hashlib.sha256(src).hexdigest()[:16] in text   # the committed summary is current
    per_node = bench._measured_traffic(1, storage)
    assert per_node is not None and per_node > 1000
    assert bench._measured_traffic(4096 * 4096, storage) == pytest.approx(per_node * 4096 * 4096)
    # any change of the kernel source makes the counters stale: no traffic
    with open(root / "paper_2201_10132_gb300" / "csrc" / "tfkt_fused.cu", "ab") as f:
        f.write(b"\n// changed\n")
    assert bench._measured_traffic(4096 * 4096, storage) is None


def test_traffic_is_none_without_a_summary(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._measured_traffic(100, "fp8") is None


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
