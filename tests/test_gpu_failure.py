"""Failure detection on the GPU without a GPU fault.

A NaN placed in the host-side initial state (the velocity perturbation that
tfkt_create uploads) must surface as TFKT_ENAN from the next diagnostics call,
which names the diagnostic and the step. The context stays usable: it steps,
its fields read back, the NaN stays local (each step reaches a few nodes:
streaming, and the central differences of the velocity and the polymer
stress), and the state is not reset. The JSONL monitor stops on it, and its
Mach guard stops a run whose largest |u| exceeds the limit."""
import io
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NX, NY, XN, YN = 64, 32, 9, 5   # grid (two 32 x 8 tiles wide) and the poisoned node


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_2201_10132_gb300 import build, tfkt
    build.build()
    return tfkt


def _params(T, prec):
    return T.Params(NX, NY, 6, 3.0, 5.0, 0.5, 0.2, 0.05, 1, 0.0, 0.0, 1, getattr(T, prec))


def _poisoned():
    from paper_2201_10132_gb300.inputs import perturbation
    pert = perturbation(NX, NY, 7, 0.05, 0.05)
    pert[0, YN, XN] = np.nan
    return pert


def _distance():
    """Periodic Chebyshev distance of every node from the poisoned one."""
    y, x = np.mgrid[:NY, :NX]
    dx = np.abs(x - XN)
    dy = np.abs(y - YN)
    return np.maximum(np.minimum(dx, NX - dx), np.minimum(dy, NY - dy))


@pytest.mark.parametrize("prec", ["FP64", "FP32", "FP16"])
def test_injected_nan_gives_enan_and_keeps_state(T, prec):
    with T.Solver(_params(T, prec), _poisoned()) as s:
        out = np.zeros(len(T.DIAGS))
        with pytest.raises(T.TfktError) as e:
            s.diagnostics_into(out)
        assert e.value.status == T.ENAN and "at step 0" in str(e.value)
        assert np.isnan(out[T.DIAGS.index("umax")])      # the maximum keeps the NaN
        s.step(2)
        with pytest.raises(T.TfktError) as e:
            s.diagnostics()
        assert e.value.status == T.ENAN and "at step 2" in str(e.value)
        assert s.get_info()["step"] == 2
        g = s.moments(["ux", "uy", "rho_s", "psi_tot"])
        far = _distance() > 4 * 3
        for k in ("ux", "uy", "rho_s", "psi_tot"):
            assert np.isnan(g[k][YN, XN]), k
            assert np.isfinite(g[k][far]).all(), k
    # a fresh context on the same device is unaffected
    from paper_2201_10132_gb300.inputs import perturbation
    with T.Solver(_params(T, prec), perturbation(NX, NY, 7, 0.05, 0.05)) as s:
        s.step(2)
        assert np.isfinite(list(s.diagnostics().values())).all()


def test_monitor_logs_and_stops_on_nan(T):
    from paper_2201_10132_gb300 import monitor
    from paper_2201_10132_gb300.inputs import perturbation
    p = _params(T, "FP64")
    buf = io.StringIO()
    with T.Solver(p, perturbation(NX, NY, 7, 0.05, 0.05)) as s:
        last = monitor.run_logged(s, 12, 5, buf)
    recs = [json.loads(line) for line in buf.getvalue().splitlines()]
    assert [r["step"] for r in recs] == [0, 5, 10, 12] and last["status"] == "ok"
    m0 = recs[0]["mass_s"] + recs[0]["mass_p"]
    for r in recs:
        assert set(T.DIAGS) <= set(r)
        assert r["mass_s"] + r["mass_p"] == pytest.approx(m0, rel=1e-12)   # mass is conserved
        assert 0.05 < r["mach"] < 0.3 and r["qrms_max"] >= r["qrms_mean"]
    buf = io.StringIO()
    with T.Solver(p, _poisoned()) as s:
        last = monitor.run_logged(s, 12, 5, buf)
        assert s.get_info()["step"] == 0
    assert last["status"] == "nan" and last["step"] == 0 and last["umax"] is None


def test_monitor_mach_guard(T):
    from paper_2201_10132_gb300 import monitor
    from paper_2201_10132_gb300.inputs import perturbation
    buf = io.StringIO()
    with T.Solver(_params(T, "FP32"), perturbation(NX, NY, 7, 0.05, 0.05)) as s:
        last = monitor.run_logged(s, 12, 5, buf, mach_limit=0.05)
    assert last["status"] == "mach" and last["step"] == 0 and last["mach"] > 0.05


def test_workspace_errors_leave_nothing_behind(T):
    """A caller workspace that is too small gives TFKT_ENOMEM, a misaligned one
    TFKT_EINVAL; neither creates a context, and an exact-size one works."""
    import torch
    p = _params(T, "FP32")
    need = T.required_bytes(p)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.TfktError) as e:
        T.Solver(p, None, workspace=small)
    assert e.value.status == 2   # TFKT_ENOMEM
    big = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.TfktError) as e:
        T.Solver(p, None, workspace=big[16:])
    assert e.value.status == T.EINVAL
    exact = torch.empty(need, dtype=torch.uint8, device="cuda")
    from paper_2201_10132_gb300.inputs import perturbation
    with T.Solver(p, perturbation(NX, NY, 7, 0.05, 0.05), workspace=exact) as s:
        s.step(3)
        d = s.diagnostics()
    assert np.isfinite(list(d.values())).all()
