"""Oracle pins: physical -> lattice parameter mapping (Sec. VII definitions).

Re = U0 l / nu, Wi = U0 lambda_H / l, beta = eta_s / (eta_s + eta_p), F = eta U0 / l^2,
and the dumbbell relations lambda_H = zeta / (4 H), zeta = 1 / tau2, Q-diffusivity
2 kT / zeta (ell = sqrt(2)); the derived identities below follow from them.
"""
import math

import pytest


def test_definitions_round_trip(oracle_mod):
    O = oracle_mod
    ny, kp, u0, re, wi, beta = 64, 1, 0.05, 5.0, 0.5, 0.2
    lat = O.map_params(64, ny, 8, 4.0, re, wi, beta, u0, kp)
    l = ny / (2 * math.pi * kp)
    assert u0 * l / lat.nu == pytest.approx(re, rel=1e-14)
    assert u0 * lat.lambda_h / l == pytest.approx(wi, rel=1e-14)
    assert lat.nu_s / lat.nu == pytest.approx(beta, rel=1e-14)
    assert lat.tau1 / 3.0 == pytest.approx(lat.nu_s, rel=1e-14)          # nu_s = c_s^2 tau1
    assert lat.a0 == pytest.approx(lat.nu * u0 / l ** 2, rel=1e-14)       # F = eta U / l^2
    assert 4 * lat.H * lat.lambda_h * lat.tau2 == pytest.approx(1.0, rel=1e-14)
    assert 2 * lat.kappa * lat.lambda_h == pytest.approx(1.0, rel=1e-14)  # C relaxes at 1/lambda
    assert lat.ell == pytest.approx(math.sqrt(2.0), rel=1e-15)
    # equilibrium variance kT/H in Q-lattice units: D_Q / kappa with D_Q = tau2/3
    assert lat.sigma_q2 == pytest.approx((lat.tau2 / 3) / lat.kappa, rel=1e-14)
    # eta_p = (H/2) ell^2 psi_tot sigma_Q^2 lambda_H  (psi counts beads)
    eta_p = (1 - beta) * lat.nu
    assert 0.5 * lat.H * lat.ell ** 2 * lat.psi_tot * lat.sigma_q2 * lat.lambda_h == \
        pytest.approx(eta_p, rel=1e-13)
    # worked numbers for the 64^2 case (nu = 0.10186, tau1 = 0.0611, lambda_H = 101.86)
    assert lat.nu == pytest.approx(0.101859, abs=1e-6)
    assert lat.tau1 == pytest.approx(0.061115, abs=1e-6)
    assert lat.lambda_h == pytest.approx(101.859, abs=1e-3)


@pytest.mark.parametrize("kw", [dict(beta=0.0), dict(beta=1.5), dict(re=0.0), dict(u0=-1.0),
                                dict(wi=0.0), dict(tau2=1e-4), dict(q_radius=0.0)])
def test_invalid_inputs_rejected(oracle_mod, kw):
    args = dict(nx=8, ny=8, q_side=4, q_radius=2.0, re=5.0, wi=0.5, beta=0.2, u0=0.05,
                k_periods=1, tau2=0.0)
    args.update(kw)
    with pytest.raises(ValueError):
        oracle_mod.map_params(**args)


def test_newtonian_has_no_polymer(oracle_mod):
    lat = oracle_mod.map_params(8, 8, 2, 1.0, 5.0, 0.0, 1.0, 0.05, 1)
    assert lat.psi_tot == 0.0 and lat.H == 0.0 and lat.kappa == 0.0
