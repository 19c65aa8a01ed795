"""Oracle pins for FENE springs (Sec. VI-D: spring force H Q / (1 - Q^2/Q0^2),
Q0^2 = b kT/H, Q-domain a disk inside |Q| < Q0 with bounce-back at its edge).

The spring factor phi(Q) = 1/(1 - Q^2/Q0^2) enters three places: the Q-space
drift of the polymer equilibrium, the bead-force term of the r-space flux and
the polymer stress. The pins below are fixed by the Smoluchowski equation of
Appendix A (homogeneous limit) and need no FENE closure:

- Second-moment balance: for any spring law the homogeneous Fokker-Planck
  equation gives d<QQ>/dt = G^T<QQ> + <QQ>G - 2 kappa <phi QQ> + 2 kappa sigma^2 I
  (kappa = H-rate, sigma^2 = kT/H). At rest its steady state is the
  equipartition identity <phi Q_a Q_b> = sigma^2 delta_ab (the stress of any
  spring law at equilibrium is n kT I); in steady shear d_y U_x = gd it fixes
  <phi Q_x Q_y> = lambda gd <Q_y^2> and <phi Q_x^2> = sigma^2 + 2 lambda gd <Q_x Q_y>.
  The stress field measures <phi QQ>, the conformation field <QQ>, so a
  missing or misplaced phi in the drift or in the stress fails these.
- The 2-D FENE equilibrium (1 - Q^2/Q0^2)^(b/2) has <Q^2> = 2 b sigma^2/(b+4)
  (a Beta-function integral), against 2 sigma^2 for Hookean springs.
- Centre-of-mass diffusion at equilibrium runs at tau2 (1/3 - (H/2) ell^2
  <phi Q_x^2>) = tau2 (1/3 - H ell^2 sigma^2 / 2) by the identity above: the
  bead-force term must carry phi.
- b -> infinity recovers the Hookean scheme.
"""
import numpy as np
import pytest

SIGMA2 = 4.0


def _one_node(O, tau2, S, R, b, psi_tot=1e-3, nx=1):
    kappa = tau2 / (3 * SIGMA2)
    lat = O.Lattice(nx=nx, ny=1, q_side=S, q_radius=R, tau1=tau2 * 0.5, tau2=tau2,
                    H=kappa / (2 * tau2), kappa=kappa, ell=2 ** 0.5, psi_tot=psi_tot,
                    sigma_q2=SIGMA2, a0=0.0, kf=1.0, u0=0.0, fene_b=b)
    return lat, 1.0 / (2 * kappa)


def _moments(lat, f):
    l2 = lat.ell ** 2
    hl = 0.5 * lat.H * l2 * lat.psi_tot
    c = {k: f[k][0, 0] / l2 for k in ("cxx", "cxy", "cyy")}
    t = {k: f[k][0, 0] / hl for k in ("thxx", "thxy", "thyy")}
    return c, t


def _from_gaussian(O, tau2, S, R, b):
    """A FENE run started from the sampled Gaussian (the Hookean equilibrium)."""
    lat_h, _ = _one_node(O, tau2, S, R, 0.0)
    h = O.Oracle(lat_h)
    h.init(None, 0)
    gs, gp = h.get_g()
    lat, lam = _one_node(O, tau2, S, R, b)
    o = O.Oracle(lat)
    o.set_g(gs, gp)
    return lat, lam, o


def test_fene_equilibrium_identity_and_extension(oracle_mod):
    O = oracle_mod
    b = 50.0
    lat, lam, o = _from_gaussian(O, 0.1, 22, 11.0, b)
    o.impose_gradient([[0.0, 0.0], [0.0, 0.0]])
    o.step(int(20 * lam))
    c, t = _moments(lat, o.fields())
    assert t["thxx"] == pytest.approx(SIGMA2, rel=1e-4)
    assert t["thyy"] == pytest.approx(SIGMA2, rel=1e-4)
    assert abs(t["thxy"]) < 1e-10
    q2 = c["cxx"] + c["cyy"]
    cont = 2 * b * SIGMA2 / (b + 4)
    assert q2 == pytest.approx(cont, rel=6e-3)  # Q-lattice spacing sigma/2: midpoint-rule error
    assert abs(q2 / (2 * SIGMA2) - 1) > 0.05  # and clearly not the Hookean extension


def test_fene_initial_state_is_the_fene_equilibrium(oracle_mod):
    O = oracle_mod
    for b in (10.0, 50.0):
        S = 22
        R = min(11.0, 0.98 * np.sqrt(b * SIGMA2))
        lat, _ = _one_node(O, 0.1, S, R, b)
        o = O.Oracle(lat)
        o.init(None, 0)
        c, t = _moments(lat, o.fields())
        # sampled (1 - Q^2/Q0^2)^(b/2) on a grid of spacing sigma/2, cut at R: its <Q^2>
        # is the continuum value up to the midpoint rule and the tail beyond R
        assert c["cxx"] + c["cyy"] == pytest.approx(2 * b * SIGMA2 / (b + 4), rel=1e-2)
        assert c["cxx"] == pytest.approx(c["cyy"], rel=1e-12)


@pytest.mark.parametrize("wi", [0.5, 1.0])
def test_fene_shear_second_moment_balance(oracle_mod, wi):
    O = oracle_mod
    lat, lam, o = _from_gaussian(O, 0.1, 22, 11.0, 50.0)
    gd = wi / lam
    o.impose_gradient([[0.0, 0.0], [gd, 0.0]])
    o.step(int(20 * lam))
    c, t = _moments(lat, o.fields())
    assert t["thxy"] == pytest.approx(lam * gd * c["cyy"], rel=5e-4)
    assert t["thxx"] == pytest.approx(SIGMA2 + 2 * lam * gd * c["cxy"], rel=5e-4)
    assert t["thyy"] == pytest.approx(SIGMA2, rel=5e-4)
    # FENE springs stretch less than Hookean ones (UCM: C_xx = sigma^2 (1 + 2 Wi^2))
    assert c["cxx"] < SIGMA2 * (1 + 2 * wi ** 2) * 0.99


def test_fene_large_b_is_hookean(oracle_mod):
    O = oracle_mod
    out = []
    for b in (0.0, 1e10):
        lat, lam = _one_node(O, 0.1, 16, 8.0, b)
        o = O.Oracle(lat)
        o.init(None, 0)
        o.impose_gradient([[0.0, 0.0], [0.5 / lam, 0.0]])
        o.step(200)
        out.append(_moments(lat, o.fields()))
    for k in ("cxx", "cxy", "cyy"):
        assert out[1][0][k] == pytest.approx(out[0][0][k], rel=1e-8)
    for k in ("thxx", "thxy", "thyy"):
        assert out[1][1][k] == pytest.approx(out[0][1][k], rel=1e-8)


def test_fene_centre_of_mass_diffusion(oracle_mod):
    """Equilibrated FENE polymer density diffuses at tau2 (1/3 - H ell^2 sigma^2 / 2);
    with the bead-force term lacking phi it would run at tau2 (1/3 - (H/2) ell^2 <Q_x^2>),
    which for b = 10 on this disk is about 28% faster. The disk is cut at 0.79 Q0:
    nodes with a large phi Q_x^2 / sigma^2 make the first-order bead-force flux
    anti-diffusive enough to destabilise the r-space modes."""
    O = oracle_mod
    from test_oracle_physics import _diffusion_rate

    tau2, b, S, R = 0.2, 10.0, 10, 5.0
    lat1, lam = _one_node(O, tau2, S, R, b)
    one = O.Oracle(lat1)
    one.init(None, 0)
    one.step(int(30 * lam))
    _, gp1 = one.get_g()
    c, t = _moments(lat1, one.fields())
    kw = {k: getattr(lat1, k) for k, _ in O.Lattice._fields_ if k not in ("nx", "ny")}
    nx = 48
    D = _diffusion_rate(O, kw, nx, gp1[0, 0], 40, 700, 2 * np.pi / nx)
    pred = tau2 * (1.0 / 3.0 - 0.5 * lat1.H * lat1.ell ** 2 * t["thxx"])
    assert D == pytest.approx(pred, rel=0.02)
    without_phi = tau2 * (1.0 / 3.0 - 0.5 * lat1.H * lat1.ell ** 2 * c["cxx"])
    assert abs(without_phi / pred - 1) > 0.15


def test_fene_map_params_rejects_disk_beyond_q0(oracle_mod):
    O = oracle_mod
    lat = O.map_params(64, 64, 8, 4.0, 5.0, 0.5, 0.2, 0.05, 1, fene_b=25.0)
    q0 = np.sqrt(25.0 * lat.sigma_q2)
    assert lat.fene_b == 25.0 and q0 > 4.0
    with pytest.raises(ValueError):
        O.map_params(64, 64, 8, 1.01 * q0, 5.0, 0.5, 0.2, 0.05, 1, fene_b=25.0)
    with pytest.raises(ValueError):  # the same disk is too large on a coarser r-grid
        O.map_params(8, 8, 8, 4.0, 5.0, 0.5, 0.2, 0.05, 1, fene_b=25.0)
    with pytest.raises(ValueError):
        O.map_params(64, 64, 8, 4.0, 5.0, 0.5, 0.2, 0.05, 1, fene_b=-1.0)
