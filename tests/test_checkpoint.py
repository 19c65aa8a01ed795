"""Checkpoint and restart (tfkt_save / tfkt_load): a run saved after n steps and
resumed in a fresh context follows the uninterrupted run bit for bit, on the
fused, two-pass, FP16 and stress-QE paths; wrong parameters, corrupt,
truncated, foreign and missing files are refused with the documented status."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# nx, ny, S, R, re, wi, beta, kp, ic, precision, qe  (precision/qe as names)
CASES = [
    (64, 32, 6, 3.0, 5.0, 0.5, 0.2, 1, 1, "FP32", 0),     # fused
    (30, 20, 4, 2.0, 3.0, 1.0, 0.5, 1, 1, "FP64", 0),     # two-pass, ragged tiles
    (64, 32, 6, 3.0, 5.0, 0.5, 0.2, 1, 0, "FP16", 0),     # fused, half storage
    (64, 16, 4, 2.0, 4.0, 0.8, 0.3, 1, 1, "FP32", 1),     # stress quasi-equilibrium
]


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_2201_10132_gb300 import build, tfkt
    build.build()
    return tfkt


def _params(T, c, re=None):
    nx, ny, S, R, r, wi, beta, kp, ic, prec, qe = c
    return T.Params(nx, ny, S, R, r if re is None else re, wi, beta, 0.05, kp, 0.0, 0.0, ic,
                    getattr(T, prec), 0.0, qe)


def _pert(c):
    from paper_2201_10132_gb300.inputs import perturbation
    return perturbation(c[0], c[1], 11, 0.05, 0.05)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[9]}-qe{c[10]}-{c[0]}x{c[1]}")
def test_resume_is_bit_exact(T, tmp_path, case):
    p = _params(T, case)
    path = str(tmp_path / "run.ckpt")
    with T.Solver(p, _pert(case)) as s:
        s.step(5)
        s.save(path)
        s.step(7)
        ref_m, ref_p = s.moments(), s.populations()
    assert os.path.exists(path) and not os.path.exists(path + ".part")
    with T.Solver(p) as s:          # created from rest: the load replaces the state
        s.load(path)
        assert s.get_info()["step"] == 5
        s.step(7)
        got_m, got_p = s.moments(), s.populations()
        assert s.get_info()["step"] == 12
    for k in ref_m:
        assert np.array_equal(got_m[k], ref_m[k]), k
    assert np.array_equal(got_p, ref_p)


def test_refuses_other_parameters(T, tmp_path):
    c = CASES[0]
    path = str(tmp_path / "a.ckpt")
    with T.Solver(_params(T, c), _pert(c)) as s:
        s.step(2)
        s.save(path)
    with T.Solver(_params(T, c, re=6.0)) as s:
        before = s.moments()
        with pytest.raises(T.TfktError) as e:
            s.load(path)
        assert e.value.status == T.EINVAL
        assert s.get_info()["step"] == 0
        after = s.moments()
        assert all(np.array_equal(before[k], after[k]) for k in before)


def _saved(T, tmp_path, steps=3):
    c = CASES[0]
    path = str(tmp_path / "b.ckpt")
    with T.Solver(_params(T, c), _pert(c)) as s:
        s.step(steps)
        s.save(path)
    return c, path


def test_refuses_corrupt_payload_and_resets(T, tmp_path):
    c, path = _saved(T, tmp_path)
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40                     # one bit of one population
    open(path, "wb").write(bytes(raw))
    with T.Solver(_params(T, c), _pert(c)) as s:
        s.step(1)
        with pytest.raises(T.TfktError) as e:
            s.load(path)
        assert e.value.status == T.EIO
        assert s.get_info()["step"] == 0            # reset to the initial state
        with T.Solver(_params(T, c)) as r:
            rest = r.moments()
        got = s.moments()
        assert all(np.array_equal(got[k], rest[k]) for k in rest)


def test_refuses_changed_step_field(T, tmp_path):
    c, path = _saved(T, tmp_path)
    raw = bytearray(open(path, "rb").read())
    # header: magic 8, version 4, 9 int32, 2 uint64, 12 double, then the step (int64)
    o = 8 + 4 + 9 * 4 + 2 * 8 + 12 * 8
    assert int.from_bytes(raw[o:o + 8], "little") == 3
    raw[o] = 4
    open(path, "wb").write(bytes(raw))
    with T.Solver(_params(T, c)) as s:
        with pytest.raises(T.TfktError) as e:
            s.load(path)
        assert e.value.status == T.EIO


@pytest.mark.parametrize("how", ["truncated", "trailing", "foreign", "missing"])
def test_refuses_bad_files(T, tmp_path, how):
    c, path = _saved(T, tmp_path)
    raw = open(path, "rb").read()
    if how == "truncated":
        open(path, "wb").write(raw[:-100])
    elif how == "trailing":
        open(path, "wb").write(raw + b"\0")
    elif how == "foreign":
        open(path, "wb").write(b"NOTACKPT" + raw[8:])
    else:
        os.remove(path)
    with T.Solver(_params(T, c)) as s:
        with pytest.raises(T.TfktError) as e:
            s.load(path)
        assert e.value.status == T.EIO


def test_batch_runs_save_but_do_not_load(T, tmp_path):
    c = CASES[0]
    p = _params(T, c)
    path = str(tmp_path / "c.ckpt")
    with T.Batch([p, p], [_pert(c), None]) as b:
        b.step(4)
        b.run(0).save(path)
        ref = b.run(0).moments()
        with pytest.raises(T.TfktError) as e:
            b.run(1).load(path)
        assert e.value.status == T.EINVAL
    with T.Solver(p) as s:
        s.load(path)
        assert s.get_info()["step"] == 4
        got = s.moments()
    assert all(np.array_equal(got[k], ref[k]) for k in ref)
