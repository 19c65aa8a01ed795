"""Oracle pins: velocity sets, weights and isotropy (Sec. VI-A, VI-B), Q-grid masking.

Checked against the constants the paper prints (tests/golden/lattice_constants.json)
and against brute-force moment sums: isotropy to 4th order with c_s^2 = 1/3
(reading: the printed 4th-order condition has c_sP^2 where c_sP^4 is meant).
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_constants.json")


def _frac(p):
    return Fraction(p[0], p[1])


def _moments(c, w, order):
    d = c.shape[1]
    out = {}
    for idx in itertools.product(range(d), repeat=order):
        s = Fraction(0)
        for k in range(len(w)):
            term = Fraction(w[k]).limit_denominator(1000)
            for a in idx:
                term *= int(c[k, a])
            s += term
        out[idx] = s
    return out


def _delta(a, b):
    return 1 if a == b else 0


@pytest.mark.parametrize("which", ["d2q9", "d4q25"])
def test_isotropy_to_fourth_order(oracle_mod, which):
    c, w, opp = getattr(oracle_mod, which)()
    cs2 = Fraction(1, 3)
    assert sum(Fraction(x).limit_denominator(1000) for x in w) == 1
    for idx, s in _moments(c, w, 1).items():
        assert s == 0
    for (a, b), s in _moments(c, w, 2).items():
        assert s == cs2 * _delta(a, b)
    for idx, s in _moments(c, w, 3).items():
        assert s == 0
    for (a, b, g, t), s in _moments(c, w, 4).items():
        iso = _delta(a, b) * _delta(g, t) + _delta(a, g) * _delta(b, t) + _delta(a, t) * _delta(b, g)
        assert s == cs2 * cs2 * iso, (a, b, g, t)
    # opposite velocity
    for i in range(len(w)):
        assert np.array_equal(c[opp[i]], -c[i])
        assert w[opp[i]] == w[i]


def test_printed_constants(oracle_mod):
    gold = json.load(open(GOLDEN))
    c, w, _ = oracle_mod.d2q9()
    for k in range(9):
        sp = int((c[k] ** 2).sum())
        num, den = gold["d2q9"]["weights_by_speed2"][str(sp)][1:]
        assert Fraction(w[k]).limit_denominator(1000) == Fraction(num, den)
    c, w, _ = oracle_mod.d4q25()
    g = gold["d4q25"]
    assert Fraction(w[0]).limit_denominator(1000) == _frac(g["w_rest"])
    assert np.all(c[0] == 0)
    moving = [k for k in range(25) if np.any(c[k] != 0)]
    assert len(moving) == g["n_moving"]
    assert all(Fraction(w[k]).limit_denominator(1000) == _frac(g["w_moving"]) for k in moving)
    # every moving velocity has exactly two components +-1 (Table dis_vel rows)
    seen = {}
    for k in moving:
        nz = tuple(int(a) for a in np.nonzero(c[k])[0])
        assert len(nz) == 2 and all(abs(c[k][a]) == 1 for a in nz)
        seen[nz] = seen.get(nz, 0) + 1
    for cls in g["classes"]:
        assert seen[tuple(cls["nonzero_axes"])] == cls["count"]
    assert len({tuple(x) for x in c.tolist()}) == 25


@pytest.mark.parametrize("S,R,expected", [(6, 3.0, 32), (8, 4.0, 52), (2, 1.0, 4), (1, 1.0, 1)])
def test_q_grid(oracle_mod, S, R, expected):
    lat = oracle_mod.Lattice(nx=1, ny=1, q_side=S, q_radius=R, tau1=0.5, tau2=0.5, sigma_q2=1.0,
                             ell=2 ** 0.5)
    o = oracle_mod.Oracle(lat)
    qx, qy = o.q_nodes()
    # brute-force count of cell centres inside the disk
    cnt = 0
    for j in range(S):
        for i in range(S):
            x, y = i - (S - 1) / 2, j - (S - 1) / 2
            cnt += x * x + y * y <= R * R
    assert o.nq == cnt == expected
    assert np.all(qx ** 2 + qy ** 2 <= R * R + 1e-12)
    # symmetric under Q -> -Q (so the Q-drift has no preferred direction)
    pts = {(a, b) for a, b in zip(qx.tolist(), qy.tolist())}
    assert all((-a, -b) in pts for a, b in pts)
