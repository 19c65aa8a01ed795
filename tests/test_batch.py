"""Batched ensembles (tfkt_batch_*): independent runs advanced by one launch of
each kernel per step must give the results of the same runs stepped one by one
up to float rounding: the kernels share one tile routine, but the batched one
sums a Q-node's moments velocity by velocity and the single-run one by velocity
pairs, and other tile heights move the tile borders (finished by the fix-up)."""
import numpy as np
import pytest

RUNS = [
    # nx, ny, S, R, re, wi, beta, kp, ic, seed
    (64, 32, 6, 3.0, 5.0, 0.5, 0.2, 1, 1, 3),
    (32, 16, 4, 2.0, 3.0, 1.0, 0.5, 1, 0, 4),
    (96, 24, 6, 3.0, 8.0, 0.3, 0.1, 2, 1, 5),
]


@pytest.fixture(scope="module")
def T():
    from paper_2201_10132_gb300 import build, tfkt
    build.build()
    return tfkt


def _params(T, r, precision=None):
    nx, ny, S, R, re, wi, beta, kp, ic, _ = r
    return T.Params(nx, ny, S, R, re, wi, beta, 0.05, kp, 0.0, 0.0, ic,
                    T.FP32 if precision is None else precision)


def test_batch_rejects_unsupported_runs(T):
    with pytest.raises(T.TfktError):
        T.batch_required_bytes([_params(T, RUNS[0], T.FP64)])
    ragged = list(RUNS[0])
    ragged[0] = 70
    with pytest.raises(T.TfktError):
        T.batch_required_bytes([_params(T, tuple(ragged))])
    short = list(RUNS[0])
    short[1] = 12                       # runs must admit the single-run 8-row tile
    with pytest.raises(T.TfktError):
        T.batch_required_bytes([_params(T, tuple(short))])
    assert T.batch_required_bytes([_params(T, r) for r in RUNS]) > 0


@pytest.mark.gpu
@pytest.mark.parametrize("steps", [1, 7])
def test_batch_matches_single_runs(T, steps, monkeypatch):
    """At the single-run tile height (8 rows): fields and diagnostics."""
    from paper_2201_10132_gb300.inputs import perturbation
    monkeypatch.setenv("TFKT_BATCH_TILE_HEIGHT", "8")
    params = [_params(T, r) for r in RUNS]
    perts = [perturbation(r[0], r[1], r[9], 0.05, 0.05) for r in RUNS]
    with T.Batch(params, perts) as b:
        assert b.tile_height()[0] == 8
        b.step(steps)
        got = [b.run(i).moments() for i in range(len(RUNS))]
        diag = [b.run(i).diagnostics() for i in range(len(RUNS))]
        assert all(b.run(i).get_info()["step"] == steps for i in range(len(RUNS)))
    for i, (p, pert) in enumerate(zip(params, perts)):
        with T.Solver(p, pert) as s:
            s.step(steps)
            ref = s.moments()
            dref = s.diagnostics()
        _close(got[i], ref)
        for k, v in dref.items():
            assert diag[i][k] == pytest.approx(v, rel=1e-5, abs=1e-8 * dref["mass_s"]), (i, k)


def _single(T, p, pert, steps):
    with T.Solver(p, pert) as s:
        s.step(steps)
        return s.moments()


def _close(got, ref):
    """The FP32 tolerance of the oracle parity tests: 2e-5 of the field's largest
    magnitude, velocity-derived fields against the largest velocity."""
    uscale = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    for k in ref:
        scale = uscale if k in ("ux", "uy", "vort") else np.abs(ref[k]).max()
        err = float(np.abs(got[k] - ref[k]).max()) / max(scale, 1e-30)
        assert err < 2e-5, (k, err)


@pytest.mark.gpu
@pytest.mark.parametrize("ty", [4, 16])
def test_batch_tile_heights_match_single_runs(T, ty, monkeypatch):
    """Other tile heights change only which CTA updates a node; each node's
    collision is the same, so the fields agree with the single runs."""
    from paper_2201_10132_gb300.inputs import perturbation
    runs = RUNS[:2] if ty == 16 else RUNS       # ny = 24 is not a multiple of 16
    monkeypatch.setenv("TFKT_BATCH_TILE_HEIGHT", str(ty))
    params = [_params(T, r) for r in runs]
    perts = [perturbation(r[0], r[1], r[9], 0.05, 0.05) for r in runs]
    steps = 7
    with T.Batch(params, perts) as b:
        assert b.tile_height()[0] == ty
        b.step(steps)
        got = [b.run(i).moments() for i in range(len(runs))]
    for i, (p, pert) in enumerate(zip(params, perts)):
        _close(got[i], _single(T, p, pert, steps))


@pytest.mark.gpu
def test_batch_autotune_picks_fastest(T, monkeypatch):
    from paper_2201_10132_gb300.inputs import perturbation
    monkeypatch.delenv("TFKT_BATCH_TILE_HEIGHT", raising=False)
    monkeypatch.delenv("TFKT_BATCH_PER_RUN", raising=False)
    runs = RUNS[:2]
    params = [_params(T, r) for r in runs]
    perts = [perturbation(r[0], r[1], r[9], 0.05, 0.05) for r in runs]
    with T.Batch(params, perts) as b:
        plan = b.plan()
        ms = plan["ms"]
        assert all(np.isfinite(m) and m > 0 for m in ms.values())
        chosen = "per_run" if plan["per_run"] else str(plan["tile_height"])
        assert ms[chosen] == min(ms.values())
        assert all(b.run(i).get_info()["step"] == 0 for i in range(len(runs)))
        b.step(3)
        got = [b.run(i).moments() for i in range(len(runs))]
    for i, (p, pert) in enumerate(zip(params, perts)):
        _close(got[i], _single(T, p, pert, 3))


@pytest.mark.gpu
@pytest.mark.parametrize("steps", [1, 6, 7])
def test_batch_per_run_plan_is_bit_identical(T, steps, monkeypatch):
    """Each run's own single-run kernels as graph branches: the runs advance
    exactly as when stepped alone (graph replays two steps; odd counts end with
    a plain step)."""
    from paper_2201_10132_gb300.inputs import perturbation
    monkeypatch.setenv("TFKT_BATCH_PER_RUN", "1")
    params = [_params(T, r) for r in RUNS]
    perts = [perturbation(r[0], r[1], r[9], 0.05, 0.05) for r in RUNS]
    with T.Batch(params, perts) as b:
        assert b.plan()["per_run"]
        b.step(steps)
        got = [b.run(i).moments() for i in range(len(RUNS))]
        diag = [_raw_diagnostics(T, b.run(i)) for i in range(len(RUNS))]
    for i, (p, pert) in enumerate(zip(params, perts)):
        with T.Solver(p, pert) as s:
            s.step(steps)
            ref = s.moments()
            dref = _raw_diagnostics(T, s)
        for k in ref:
            assert np.array_equal(got[i][k], ref[k], equal_nan=True), (i, k)
        assert diag[i][0] == dref[0] and np.array_equal(diag[i][1], dref[1], equal_nan=True), i


def _raw_diagnostics(T, s):
    """tfkt_diagnostics' status and values, also when a value is not finite (the
    third run's Q_rms is NaN at step 6: on its 12-node forcing wavelength the
    over-relaxed stress mode rings, and the trace of C is negative on alternate
    early steps, where Q_rms = sqrt(trace) is NaN, as in the oracle)."""
    import ctypes
    out = np.zeros(len(T.DIAGS))
    st = T.lib().tfkt_diagnostics(s._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return st, out


@pytest.mark.gpu
def test_batch_forced_height_must_fit(T, monkeypatch):
    monkeypatch.setenv("TFKT_BATCH_TILE_HEIGHT", "16")
    with pytest.raises(T.TfktError):
        T.Batch([_params(T, RUNS[2])], None)         # ny = 24


# Runs of different grid sizes, Re, Wi and beta, one with tau2 > tau1; every ny
# is a multiple of 16 so that each tile height can take every run.
ORACLE_RUNS = [
    # nx, ny, S, R, re, wi, beta, kp, tau2, ic, seed
    (64, 32, 6, 3.0, 5.0, 0.5, 0.2, 1, 0.0, 1, 3),
    (32, 16, 4, 2.0, 3.0, 1.0, 0.5, 1, 0.0, 0, 4),
    (96, 16, 6, 3.0, 8.0, 0.3, 0.1, 1, 0.0, 1, 5),
    (64, 48, 6, 3.0, 4.0, 1.0, 0.5, 1, 0.3, 1, 6),
]


@pytest.mark.gpu
@pytest.mark.parametrize("plan", ["4", "8", "16", "per_run"])
def test_batch_matches_oracle(T, oracle_mod, plan, monkeypatch):
    """Every run of a heterogeneous batch, under each plan, against the FP64 oracle
    at the FP32 parity tolerance (fields and global diagnostics)."""
    from paper_2201_10132_gb300.inputs import perturbation
    monkeypatch.delenv("TFKT_BATCH_TILE_HEIGHT", raising=False)
    monkeypatch.delenv("TFKT_BATCH_PER_RUN", raising=False)
    if plan == "per_run":
        monkeypatch.setenv("TFKT_BATCH_PER_RUN", "1")
    else:
        monkeypatch.setenv("TFKT_BATCH_TILE_HEIGHT", plan)
    steps = 9
    params, perts = [], []
    for nx, ny, S, R, re, wi, beta, kp, tau2, ic, seed in ORACLE_RUNS:
        params.append(T.Params(nx, ny, S, R, re, wi, beta, 0.05, kp, tau2, 0.0, ic, T.FP32))
        perts.append(perturbation(nx, ny, seed, 0.05, 0.05))
    with T.Batch(params, perts) as b:
        pl = b.plan()
        assert pl["per_run"] if plan == "per_run" else pl["tile_height"] == int(plan)
        b.step(steps)
        got = [b.run(i).moments() for i in range(len(params))]
        diag = [b.run(i).diagnostics() for i in range(len(params))]
    for i, (r, pert) in enumerate(zip(ORACLE_RUNS, perts)):
        nx, ny, S, R, re, wi, beta, kp, tau2, ic, _ = r
        lat = oracle_mod.map_params(nx, ny, S, R, re, wi, beta, 0.05, kp, tau2)
        o = oracle_mod.Oracle(lat)
        o.init(pert, ic)
        o.step(steps)
        f = o.fields()
        _close(got[i], {k: f[k] for k in got[i]})
        od = o.diagnostics()
        uscale = max(np.abs(f["ux"]).max(), np.abs(f["uy"]).max())
        du = 2e-5 * uscale
        rho = f["rho_s"] + f["psi_tot"]
        tol = {"mass_s": 2e-5 * od["mass_s"], "mass_p": 2e-5 * max(od["mass_p"], 1e-30),
               "px": 2 * du * rho.sum(), "py": 2 * du * rho.sum(),
               "ke": 2 * du * (rho * (np.abs(f["ux"]) + np.abs(f["uy"]))).sum() + 1e-30,
               "enstrophy": 4 * du * np.abs(f["vort"]).sum() + 1e-30,
               "qrms_mean": 2e-5 * max(od["qrms_mean"], 1e-30),
               "ey2": 2 * du * np.abs(f["uy"]).sum() + 1e-30}
        for k, t in tol.items():
            assert abs(diag[i][k] - od[k]) <= t, (plan, i, k, diag[i][k], od[k], t)
