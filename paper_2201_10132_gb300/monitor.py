"""JSONL run log: the global diagnostics every K steps, with a Mach guard.

One JSON object per line. Each record holds the step, every diagnostic of
``tfkt_diagnostics`` (masses, momentum, kinetic energy, enstrophy, mean and
largest Q_rms of Sec. VII, largest |u|), the Mach number max|u| / c_s with
c_s = 1/sqrt(3) of the D2Q9 lattice (Sec. VI A), and the wall time since the
previous record (the K steps and this record's diagnostics call, which
synchronises). Non-finite values are written as null (JSON has no NaN).

The run stops early, with a last record saying why, when
- a diagnostic is not finite (``TFKT_ENAN``): status "nan", with the step and
  the library's message; the device state is kept as it is, for inspection;
- the Mach number exceeds ``mach_limit``: status "mach". The lattice scheme
  holds only for |u| well below c_s, so a run past that limit has left the
  regime the method is valid in.

Every step runs in the solver's CUDA kernels; this module only decides when
to read the diagnostics and writes the records.
"""
from __future__ import annotations

import json
import math
import time

CS = 1.0 / math.sqrt(3.0)


def _finite_or_none(v: float):
    return v if math.isfinite(v) else None


def record(step: int, diag: dict, wall_ms: float, status: str = "ok", message: str = "") -> dict:
    """One log record from a diagnostics dict (as ``Solver.diagnostics``)."""
    r = {"step": int(step), "status": status}
    for k, v in diag.items():
        r[k] = _finite_or_none(float(v))
    umax = float(diag.get("umax", float("nan")))
    r["mach"] = _finite_or_none(umax / CS)
    r["wall_ms"] = float(wall_ms)
    if message:
        r["message"] = message
    return r


def run_logged(solver, steps: int, every: int, out, mach_limit: float = 0.3,
               diags=None, nan_status=None) -> dict:
    """Advance ``solver`` by ``steps`` steps, logging every ``every`` steps.

    ``solver`` needs ``step(n)`` and ``diagnostics_into(array)`` as in
    ``tfkt.Solver`` (``diagnostics_into`` fills the array even when it raises
    for a non-finite value). ``out`` is a writable text stream. ``diags`` (the
    diagnostic names) and ``nan_status`` (the status code of a non-finite
    diagnostic) default to the library's. Returns the last record; the record
    at step 0 is written before the first step.
    """
    import numpy as np

    if every <= 0 or steps < 0:
        raise ValueError("every must be > 0 and steps >= 0")
    if diags is None or nan_status is None:
        from . import tfkt
        diags = tfkt.DIAGS if diags is None else diags
        nan_status = tfkt.ENAN if nan_status is None else nan_status
    buf = np.zeros(len(diags))
    done = 0
    t0 = time.perf_counter()
    while True:
        try:
            solver.diagnostics_into(buf)
            status, msg = "ok", ""
        except RuntimeError as e:   # tfkt.TfktError
            if getattr(e, "status", None) != nan_status:
                raise
            status, msg = "nan", str(e)
        wall = (time.perf_counter() - t0) * 1e3
        rec = record(done, dict(zip(diags, buf.tolist())), wall, status, msg)
        if status == "ok" and rec["mach"] is not None and rec["mach"] > mach_limit:
            rec["status"] = "mach"
            rec["message"] = f"Mach {rec['mach']:.4g} above the limit {mach_limit:g}"
        out.write(json.dumps(rec) + "\n")
        out.flush()
        if rec["status"] != "ok" or done >= steps:
            return rec
        n = min(every, steps - done)
        t0 = time.perf_counter()
        solver.step(n)
        done += n
