"""JSONL run log (host logic only): records, the NaN stop and the Mach guard,
driven by a fake solver that follows a scripted diagnostics trajectory."""
import io
import json
import math

import numpy as np
import pytest

from paper_2201_10132_gb300 import monitor

DIAGS = ["mass_s", "ke", "umax", "qrms_max"]
ENAN = 4


class _Err(RuntimeError):
    def __init__(self, status):
        super().__init__(f"status {status}")
        self.status = status


class FakeSolver:
    """step(n) advances a counter; diagnostics follow umax(step), with NaN
    from step `nan_at` on, or another error status from step `err_at` on."""

    def __init__(self, umax, nan_at=None, err_at=None):
        self.t, self.umax, self.nan_at, self.err_at = 0, umax, nan_at, err_at
        self.calls = []

    def step(self, n):
        self.calls.append(n)
        self.t += n

    def diagnostics_into(self, out):
        out[:] = [100.0, 0.5 * self.t, self.umax(self.t), 0.2]
        if self.err_at is not None and self.t >= self.err_at:
            raise _Err(3)
        if self.nan_at is not None and self.t >= self.nan_at:
            out[1] = math.nan
            raise _Err(ENAN)


def _run(s, steps, every, **kw):
    buf = io.StringIO()
    last = monitor.run_logged(s, steps, every, buf, diags=DIAGS, nan_status=ENAN, **kw)
    return last, [json.loads(line) for line in buf.getvalue().splitlines()]


def test_records_every_k_steps_and_ragged_end():
    s = FakeSolver(lambda t: 0.01)
    last, recs = _run(s, 23, 10)
    assert [r["step"] for r in recs] == [0, 10, 20, 23]
    assert s.calls == [10, 10, 3]
    assert all(r["status"] == "ok" for r in recs) and last == recs[-1]
    assert recs[2]["ke"] == 10.0 and recs[2]["mass_s"] == 100.0
    assert recs[0]["mach"] == pytest.approx(0.01 * math.sqrt(3.0))
    assert all(r["wall_ms"] >= 0 for r in recs)


def test_zero_steps_writes_one_record():
    s = FakeSolver(lambda t: 0.0)
    last, recs = _run(s, 0, 5)
    assert len(recs) == 1 and recs[0]["step"] == 0 and s.calls == []


def test_nan_stops_with_step_and_null_values():
    s = FakeSolver(lambda t: 0.01, nan_at=15)
    last, recs = _run(s, 100, 10)
    assert [r["step"] for r in recs] == [0, 10, 20]
    assert last["status"] == "nan" and last["step"] == 20
    assert last["ke"] is None and last["mass_s"] == 100.0
    assert "message" in last
    assert s.t == 20   # nothing stepped after the NaN was seen


def test_mach_guard_stops():
    s = FakeSolver(lambda t: 0.002 * t)    # Mach 0.3 is reached at t ~ 86.6
    last, recs = _run(s, 500, 10, mach_limit=0.3)
    assert last["status"] == "mach" and last["step"] == 90
    assert last["mach"] > 0.3 and all(r["mach"] <= 0.3 for r in recs[:-1])


def test_other_errors_propagate():
    s = FakeSolver(lambda t: 0.01, err_at=10)
    with pytest.raises(_Err):
        _run(s, 50, 10)


def test_bad_arguments():
    with pytest.raises(ValueError):
        _run(FakeSolver(lambda t: 0.0), 10, 0)


def test_record_nonfinite_is_null_and_json_strict():
    r = monitor.record(7, {"a": math.inf, "umax": math.nan, "b": 1.5}, 2.0)
    text = json.dumps(r, allow_nan=False)   # raises if any NaN/inf slipped through
    assert json.loads(text) == {"step": 7, "status": "ok", "a": None, "umax": None, "b": 1.5,
                                "mach": None, "wall_ms": 2.0}
    assert np.isclose(monitor.CS, 1 / np.sqrt(3))


def test_defaults_come_from_the_binding():
    """Without explicit names the log uses the library's diagnostics (including
    the maxima umax and qrms_max) and its TFKT_ENAN status."""
    from paper_2201_10132_gb300 import tfkt

    class Fake:
        def __init__(self):
            self.t = 0

        def step(self, n):
            self.t += n

        def diagnostics_into(self, out):
            out[:] = np.arange(len(out), dtype=float) + 0.5
            out[tfkt.DIAGS.index("umax")] = 0.01
            if self.t >= 4:
                e = RuntimeError("non-finite diagnostic ke at step 4")
                e.status = tfkt.ENAN
                raise e

    buf = io.StringIO()
    last = monitor.run_logged(Fake(), 10, 2, buf)
    recs = [json.loads(line) for line in buf.getvalue().splitlines()]
    assert set(tfkt.DIAGS) <= set(recs[0]) and "umax" in tfkt.DIAGS and "qrms_max" in tfkt.DIAGS
    assert [r["step"] for r in recs] == [0, 2, 4] and last["status"] == "nan"
    assert recs[0]["mach"] == pytest.approx(0.01 * math.sqrt(3.0))
