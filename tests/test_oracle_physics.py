"""Oracle pins: limits where the scheme must reproduce known physics.

- Homogeneous shear on one r-node (Appendix A, homogeneous dilute limit: the
  Smoluchowski equation for Q with drift Q . grad U - 2F/zeta and diffusivity
  2 kT/zeta): the conformation reaches the upper-convected Maxwell steady state
  C_xy = lambda gd C_eq, C_xx - C_eq = 2 (lambda gd)^2 C_eq, C_yy = C_eq, and
  after the shear stops C_xy decays at exactly 1/lambda_H.
- Polymer r-diffusion (Appendix A, density equation): without springs the bead
  density diffuses at kT/zeta = tau2/3; at conformational equilibrium the
  centre of mass diffuses at kT/zeta - (1/(2 zeta)) Theta/n, i.e.
  tau2 (1/3 - (H/2) <Q_x^2>) with <Q_x^2> the lattice equilibrium value.
- Newtonian Kolmogorov flow (Sec. VII: F = eta U / l^2 drives U cos(y/l)): the
  steady profile is a0/(nu k^2) sin(k y), converging at least at second order.
"""
import ctypes

import numpy as np
import pytest


def _one_node(O, tau2, sigma2, S, R, tau1_frac=0.5):
    kappa = tau2 / (3 * sigma2)
    lat = O.Lattice(nx=1, ny=1, q_side=S, q_radius=R, tau1=tau2 * tau1_frac, tau2=tau2,
                    H=kappa / (2 * tau2), kappa=kappa, ell=2 ** 0.5, psi_tot=1e-3,
                    sigma_q2=sigma2, a0=0.0, kf=1.0, u0=0.0)
    return lat, 1.0 / (2 * kappa)


@pytest.mark.parametrize("tau2,sigma2,S,R", [(0.1, 4.0, 24, 12.0), (0.05, 4.0, 24, 12.0)])
def test_homogeneous_shear_ucm(oracle_mod, tau2, sigma2, S, R):
    O = oracle_mod
    lat, lam = _one_node(O, tau2, sigma2, S, R)
    wi = 0.5
    gd = wi / lam
    o = O.Oracle(lat)
    o.init(None, 0)
    o.impose_gradient([[0.0, 0.0], [gd, 0.0]])  # d_y U_x = gd
    o.step(int(15 * lam))
    f = o.fields()
    l2 = lat.ell ** 2
    cxx, cxy, cyy = (f[k][0, 0] / l2 for k in ("cxx", "cxy", "cyy"))
    assert cxy == pytest.approx(wi * sigma2, rel=3e-4)
    assert cxx - sigma2 == pytest.approx(2 * wi ** 2 * sigma2, rel=5e-4)
    assert cyy == pytest.approx(sigma2, rel=1e-4)
    # switch the shear off: C_xy decays at 1/lambda_H (second-order time error)
    o.impose_gradient([[0.0, 0.0], [0.0, 0.0]])
    h = int(lam / 2)
    c = []
    for _ in range(3):
        o.step(h)
        c.append(o.fields()["cxy"][0, 0])
    rate = np.log(c[0] / c[1]) / h
    assert rate == pytest.approx(1.0 / lam, rel=3e-3)
    assert np.log(c[1] / c[2]) / h == pytest.approx(rate, rel=1e-5)


def test_homogeneous_shear_direction(oracle_mod):
    """d_x U_y instead of d_y U_x stretches along y, not x (catches a transposed gradient)."""
    O = oracle_mod
    lat, lam = _one_node(O, 0.1, 4.0, 24, 12.0)
    o = O.Oracle(lat)
    o.init(None, 0)
    o.impose_gradient([[0.0, 0.5 / lam], [0.0, 0.0]])
    o.step(int(15 * lam))
    f = o.fields()
    assert f["cyy"][0, 0] / 2 == pytest.approx(4.0 * (1 + 2 * 0.25), rel=5e-4)
    assert f["cxx"][0, 0] / 2 == pytest.approx(4.0, rel=1e-4)


def _diffusion_rate(O, lat_kw, nx, gp_profile, T1, T2, k):
    lat = O.Lattice(nx=nx, ny=1, **lat_kw)
    o = O.Oracle(lat)
    c9, w9, _ = O.d2q9()
    x = np.arange(nx)
    prof = 1 + 0.01 * np.cos(k * x)
    gs = np.broadcast_to(w9, (1, nx, 9)).copy()
    gp = (gp_profile[None, None] * prof[None, :, None, None]).copy()
    o.set_g(gs, gp)

    def amp():
        pt = o.fields()["psi_tot"][0]
        return 2 * np.abs(np.fft.rfft(pt)[1]) / nx

    o.step(T1)
    a1 = amp()
    o.step(T2 - T1)
    a2 = amp()
    return np.log(a1 / a2) / (T2 - T1) / k ** 2


def test_bead_diffusion_without_springs(oracle_mod):
    O = oracle_mod
    tau2 = 0.2
    kw = dict(q_side=28, q_radius=14.0, tau1=0.1, tau2=tau2, H=0.0, kappa=0.0, ell=2 ** 0.5,
              psi_tot=1e-3, sigma_q2=2.0, a0=0.0, kf=1.0, u0=0.0)
    c25, w25, _ = O.d4q25()
    errs = []
    for nx, T2 in ((16, 120), (32, 300)):
        probe = O.Oracle(O.Lattice(nx=1, ny=1, **kw))
        prof = w25[None, :] * probe.psi0()[:, None]
        D = _diffusion_rate(O, kw, nx, prof, 20, T2, 2 * np.pi / nx)
        errs.append(abs(D / (tau2 / 3) - 1))
    assert errs[1] < 5e-3
    assert errs[0] / errs[1] > 3.0  # second-order convergence in k


def test_centre_of_mass_diffusion(oracle_mod):
    """At conformational equilibrium the polymer density diffuses at the centre-of-mass
    rate tau2 (1/3 - (H/2) ell^2 <Q_x^2>) of the density equation in Appendix A.
    Without the bead-counting factor 1/2 in the spring term the rate would be
    tau2 (1/3 - H ell^2 <Q_x^2>), about a quarter of this."""
    O = oracle_mod
    tau2, sigma2, S, R = 0.2, 4.0, 10, 5.0
    lat1, lam = _one_node(O, tau2, sigma2, S, R)
    one = O.Oracle(lat1)
    one.init(None, 0)
    one.step(int(30 * lam))
    _, gp1 = one.get_g()
    cxx = one.fields()["cxx"][0, 0]  # ell^2 <Q_x^2>, r-lengths
    kw = {k: getattr(lat1, k) for k, _ in O.Lattice._fields_ if k not in ("nx", "ny")}
    nx = 48
    D = _diffusion_rate(O, kw, nx, gp1[0, 0], 40, 700, 2 * np.pi / nx)
    pred = tau2 * (1.0 / 3.0 - 0.5 * lat1.H * cxx)
    assert D == pytest.approx(pred, rel=0.02)


def test_newtonian_kolmogorov_profile(oracle_mod):
    O = oracle_mod
    errs = []
    for ny in (16, 32, 64):
        nu = 1.0 / 6.0
        re = 0.05 * ny / (2 * np.pi * nu)
        lat = O.map_params(4, ny, 1, 1.0, re, 0.0, 1.0, 0.05, 1)  # beta = 1: no polymer
        assert lat.psi_tot == 0.0 and lat.tau1 == pytest.approx(0.5)
        o = O.Oracle(lat)
        o.init(None, 1)
        o.step(int(14 / (lat.nu * lat.kf ** 2)))
        f = o.fields()
        y = np.arange(ny)
        ref = lat.a0 / (lat.nu * lat.kf ** 2) * np.sin(lat.kf * y)
        assert np.abs(f["uy"]).max() < 1e-13
        errs.append(np.abs(f["ux"][:, 0] - ref).max() / np.abs(ref).max())
    assert errs[0] < 2e-4
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
