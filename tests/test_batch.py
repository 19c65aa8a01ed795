"""Batched ensembles (tfkt_batch_*): independent runs advanced by one launch of
each kernel per step must give exactly the results of the same runs stepped
one by one (the kernels share one tile routine and sum in a fixed order)."""
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
    assert T.batch_required_bytes([_params(T, r) for r in RUNS]) > 0


@pytest.mark.gpu
@pytest.mark.parametrize("steps", [1, 7])
def test_batch_equals_single_runs(T, steps):
    from paper_2201_10132_gb300.inputs import perturbation
    params = [_params(T, r) for r in RUNS]
    perts = [perturbation(r[0], r[1], r[9], 0.05, 0.05) for r in RUNS]
    with T.Batch(params, perts) as b:
        b.step(steps)
        got = [b.run(i).moments() for i in range(len(RUNS))]
        diag = [b.run(i).diagnostics() for i in range(len(RUNS))]
        assert all(b.run(i).get_info()["step"] == steps for i in range(len(RUNS)))
    for i, (p, pert) in enumerate(zip(params, perts)):
        with T.Solver(p, pert) as s:
            s.step(steps)
            ref = s.moments()
            dref = s.diagnostics()
        for k in ref:
            assert np.array_equal(got[i][k], ref[k]), (i, k)
        assert diag[i] == dref
