"""Oracle pins: the observables of Sec. VII and the initial state of Sec. VI-D.

States with known answers are built here directly from the lattice definitions
(D2Q9 and D4Q25 equilibria about a prescribed velocity, Sec. VI-A and VI-B),
so the expected values are closed forms, not re-runs of the oracle:

- the rest state: masses N rho_S and N psi_tot, no momentum, no kinetic energy,
  no enstrophy, and Q_rms = sqrt(ell^2 <psi |Q|^2> / <psi>) of the Gaussian on
  the masked Q-grid;
- a uniform flow U: momentum rho U N and kinetic energy (1/2) rho |U|^2 N with
  rho = rho_S + psi_tot (the mixture density, not the solvent's);
- the shear U_x = A sin(k y): vorticity -A sin(k) cos(k y) from the central
  difference, enstrophy (1/2) sum omega^2 = A^2 sin^2(k) N / 4;
- the rotation sense: U = (-A sin(k y), A sin(k x)) turns counter-clockwise
  near the origin, so omega = d_x U_y - d_y U_x is positive there (2 A sin k);
- the mean Q_rms is the plain mean over all r-nodes of the local Q_rms;
- the initial state carries psi = psi0(q), J^r = psi U and
  J^Q = psi (Q . grad U - kappa phi Q) (Eq. poly_imposed_vel with grad_r psi = 0),
  and, without body force, it is a fixed point of the first collision (g = f^eq
  with f* = f^eq), which ties its drift term to the collision's (pinned by the
  homogeneous-shear tests).
"""
import numpy as np
import pytest

ELL = 2 ** 0.5


def _lattice(O, nx, ny, S=6, R=3.0, tau1=0.4, tau2=0.9, H=0.02, psi_tot=0.2, a0=0.0,
             fene_b=0.0):
    kappa = 2 * H * tau2
    return O.Lattice(nx=nx, ny=ny, q_side=S, q_radius=R, tau1=tau1, tau2=tau2, H=H,
                     kappa=kappa, ell=ELL, psi_tot=psi_tot, sigma_q2=tau2 / (3 * kappa),
                     a0=a0, kf=2 * np.pi / ny, u0=0.05, fene_b=fene_b)


def _q_grid(S, R):
    """The cell-centred S x S Q-grid masked to |Q| <= R, row-major over (j, i)."""
    c = np.arange(S) - 0.5 * (S - 1)
    qx, qy = np.meshgrid(c, c)
    keep = qx ** 2 + qy ** 2 <= R * R + 1e-9
    return qx[keep], qy[keep]


def _gaussian_psi0(S, R, sigma_q2, psi_tot):
    qx, qy = _q_grid(S, R)
    g = np.exp(-(qx ** 2 + qy ** 2) / (2 * sigma_q2))
    return psi_tot * g / g.sum()


def _equilibrium_state(O, lat, rho_s, ux, uy, psi):
    """D2Q9 solvent equilibrium about (ux, uy) with density rho_s (quadratic,
    Sec. VI-A), and D4Q25 polymer populations w_i [psi + 3 psi U . v_i] (linear
    equilibrium with J^r = psi U, J^Q = 0, Sec. VI-B). psi: [ny, nx, nq]."""
    c9, w9, _ = O.d2q9()
    c25, w25, _ = O.d4q25()
    cu = c9[None, None, :, 0] * ux[..., None] + c9[None, None, :, 1] * uy[..., None]
    u2 = (ux * ux + uy * uy)[..., None]
    gs = w9 * rho_s[..., None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * u2)
    vu = c25[:, 0] * ux[..., None] + c25[:, 1] * uy[..., None]         # [ny, nx, 25]
    gp = w25 * psi[..., None] * (1 + 3 * vu[:, :, None, :])
    return gs, gp


def _fields_and_diag(O, lat, gs, gp):
    o = O.Oracle(lat)
    o.set_g(gs, gp)
    return o.fields(), o.diagnostics(), o


def test_rest_state(oracle_mod):
    O = oracle_mod
    nx, ny = 7, 5
    lat = _lattice(O, nx, ny)
    psi0 = _gaussian_psi0(6, 3.0, lat.sigma_q2, lat.psi_tot)
    z = np.zeros((ny, nx))
    gs, gp = _equilibrium_state(O, lat, z + 1.0, z, z, np.broadcast_to(psi0, (ny, nx, psi0.size)))
    f, d, _ = _fields_and_diag(O, lat, gs, gp)
    N = nx * ny
    assert d["mass_s"] == pytest.approx(N, rel=1e-14)
    assert d["mass_p"] == pytest.approx(N * lat.psi_tot, rel=1e-13)
    for k in ("px", "py", "ke", "enstrophy", "ey2"):
        assert abs(d[k]) < 1e-28, k
    qx, qy = _q_grid(6, 3.0)
    qrms = np.sqrt(ELL ** 2 * (psi0 * (qx ** 2 + qy ** 2)).sum() / psi0.sum())
    assert d["qrms_mean"] == pytest.approx(qrms, rel=1e-13)
    np.testing.assert_allclose(f["qrms"], qrms, rtol=1e-13)
    # conformation of the rest state: ell^2 <Q_a Q_b>, isotropic on the symmetric grid
    cxx = ELL ** 2 * (psi0 * qx * qx).sum() / psi0.sum()
    np.testing.assert_allclose(f["cxx"], cxx, rtol=1e-13)
    np.testing.assert_allclose(f["cyy"], cxx, rtol=1e-13)
    assert np.abs(f["cxy"]).max() < 1e-15


def test_uniform_flow(oracle_mod):
    """Mixture density weights the momentum and the kinetic energy."""
    O = oracle_mod
    nx, ny = 6, 4
    lat = _lattice(O, nx, ny, psi_tot=0.3)
    psi0 = _gaussian_psi0(6, 3.0, lat.sigma_q2, lat.psi_tot)
    U = (0.031, -0.017)
    rho_s = 1.3
    one = np.ones((ny, nx))
    gs, gp = _equilibrium_state(O, lat, rho_s * one, U[0] * one, U[1] * one,
                                np.broadcast_to(psi0, (ny, nx, psi0.size)))
    f, d, _ = _fields_and_diag(O, lat, gs, gp)
    N = nx * ny
    rho = rho_s + lat.psi_tot
    np.testing.assert_allclose(f["ux"], U[0], rtol=1e-13)
    np.testing.assert_allclose(f["uy"], U[1], rtol=1e-13)
    assert d["mass_s"] == pytest.approx(rho_s * N, rel=1e-14)
    assert d["px"] == pytest.approx(rho * U[0] * N, rel=1e-13)
    assert d["py"] == pytest.approx(rho * U[1] * N, rel=1e-13)
    assert d["ke"] == pytest.approx(0.5 * rho * (U[0] ** 2 + U[1] ** 2) * N, rel=1e-13)
    assert d["ey2"] == pytest.approx(U[1] ** 2 * N, rel=1e-13)
    assert abs(d["enstrophy"]) < 1e-28
    assert np.abs(f["vort"]).max() < 1e-17


@pytest.mark.parametrize("ny", [8, 12])
def test_shear_vorticity_and_enstrophy(oracle_mod, ny):
    O = oracle_mod
    nx = 5
    lat = _lattice(O, nx, ny)
    psi0 = _gaussian_psi0(6, 3.0, lat.sigma_q2, lat.psi_tot)
    A, k = 0.04, 2 * np.pi / ny
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = A * np.sin(k * y)
    gs, gp = _equilibrium_state(O, lat, np.ones((ny, nx)), ux, np.zeros((ny, nx)),
                                np.broadcast_to(psi0, (ny, nx, psi0.size)))
    f, d, _ = _fields_and_diag(O, lat, gs, gp)
    N = nx * ny
    np.testing.assert_allclose(f["ux"], ux, atol=1e-16)
    # omega = -d_y U_x = -A (sin k(y+1) - sin k(y-1)) / 2 = -A sin(k) cos(k y)
    np.testing.assert_allclose(f["vort"], -A * np.sin(k) * np.cos(k * y), atol=1e-16)
    assert d["enstrophy"] == pytest.approx(A * A * np.sin(k) ** 2 * N / 4, rel=1e-12)
    rho = 1.0 + lat.psi_tot
    assert d["ke"] == pytest.approx(rho * A * A * N / 4, rel=1e-12)
    assert abs(d["px"]) < 1e-15 and abs(d["ey2"]) < 1e-30


def test_vorticity_rotation_sense(oracle_mod):
    """A counter-clockwise eddy at the origin has positive vorticity."""
    O = oracle_mod
    n = 16
    lat = _lattice(O, n, n)
    psi0 = _gaussian_psi0(6, 3.0, lat.sigma_q2, lat.psi_tot)
    A, k = 0.03, 2 * np.pi / n
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ux = -A * np.sin(k * y)
    uy = A * np.sin(k * x)
    gs, gp = _equilibrium_state(O, lat, np.ones((n, n)), ux, uy,
                                np.broadcast_to(psi0, (n, n, psi0.size)))
    f, _, _ = _fields_and_diag(O, lat, gs, gp)
    # near (0, 0): U ~ (-A k y, A k x), a rigid counter-clockwise rotation
    assert f["vort"][0, 0] > 0
    assert f["vort"][0, 0] == pytest.approx(2 * A * np.sin(k), rel=1e-12)
    np.testing.assert_allclose(f["vort"], A * np.sin(k) * (np.cos(k * x) + np.cos(k * y)),
                               atol=1e-16)


def test_qrms_mean_is_plain_mean_over_nodes(oracle_mod):
    """Nodes with different psi_tot and different Q-spreads: the mean is over
    the r-nodes, not weighted by psi."""
    O = oracle_mod
    nx, ny = 4, 3
    lat = _lattice(O, nx, ny, psi_tot=0.1)
    qx, qy = _q_grid(6, 3.0)
    q2 = qx ** 2 + qy ** 2
    wide = np.exp(-q2 / 8.0)
    narrow = np.exp(-q2 / 1.0)
    psi = np.empty((ny, nx, q2.size))
    psi[:, :2] = 0.05 * wide / wide.sum()
    psi[:, 2:] = 0.4 * narrow / narrow.sum()
    gs, gp = _equilibrium_state(O, lat, np.ones((ny, nx)), np.zeros((ny, nx)),
                                np.zeros((ny, nx)), psi)
    f, d, _ = _fields_and_diag(O, lat, gs, gp)
    q_w = np.sqrt(ELL ** 2 * (wide * q2).sum() / wide.sum())
    q_n = np.sqrt(ELL ** 2 * (narrow * q2).sum() / narrow.sum())
    np.testing.assert_allclose(f["qrms"][:, :2], q_w, rtol=1e-13)
    np.testing.assert_allclose(f["qrms"][:, 2:], q_n, rtol=1e-13)
    assert d["qrms_mean"] == pytest.approx(0.5 * (q_w + q_n), rel=1e-13)
    assert d["mass_p"] == pytest.approx(ny * 2 * (0.05 + 0.4), rel=1e-13)


def _fene_phi(S, R, b, sigma_q2):
    qx, qy = _q_grid(S, R)
    return 1.0 / (1.0 - (qx ** 2 + qy ** 2) / (b * sigma_q2))


@pytest.mark.parametrize("fene_b", [0.0, 4.0])
def test_initial_state_moments(oracle_mod, fene_b):
    from paper_2201_10132_gb300.inputs import perturbation
    O = oracle_mod
    nx, ny = 10, 8
    lat = _lattice(O, nx, ny, fene_b=fene_b)
    pert = perturbation(nx, ny, 3, 0.3, 0.05)
    o = O.Oracle(lat)
    o.init(pert, 1)
    gs, gp = o.get_g()
    c9, _, _ = O.d2q9()
    c25, _, _ = O.d4q25()
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = lat.u0 * np.sin(lat.kf * y) + pert[0]
    uy = pert[1]
    # solvent: rho_S = 1, J_S = U
    np.testing.assert_allclose(gs.sum(-1), 1.0, rtol=1e-14)
    np.testing.assert_allclose(gs @ c9[:, 0], ux, atol=1e-16)
    np.testing.assert_allclose(gs @ c9[:, 1], uy, atol=1e-16)
    # polymer: psi(q) is the spring's equilibrium normalised to psi_tot
    qx, qy = _q_grid(6, 3.0)
    q2 = qx ** 2 + qy ** 2
    if fene_b > 0:
        phi = _fene_phi(6, 3.0, fene_b, lat.sigma_q2)
        g0 = (1.0 - q2 / (fene_b * lat.sigma_q2)) ** (fene_b / 2)
    else:
        phi = np.ones_like(q2)
        g0 = np.exp(-q2 / (2 * lat.sigma_q2))
    psi0 = lat.psi_tot * g0 / g0.sum()
    psi = gp.sum(-1)
    np.testing.assert_allclose(psi, np.broadcast_to(psi0, psi.shape), rtol=1e-13)
    # J^r = psi U
    jrx = gp @ c25[:, 0]
    jry = gp @ c25[:, 1]
    np.testing.assert_allclose(jrx, psi0 * ux[..., None], atol=1e-16)
    np.testing.assert_allclose(jry, psi0 * uy[..., None], atol=1e-16)
    # J^Q = psi (Q . grad U - kappa phi Q), grad U by central differences
    d = lambda a, ax: 0.5 * (np.roll(a, -1, axis=ax) - np.roll(a, 1, axis=ax))
    dxux, dyux, dxuy, dyuy = d(ux, 1), d(ux, 0), d(uy, 1), d(uy, 0)
    jqx = psi0 * (qx * dxux[..., None] + qy * dyux[..., None] - lat.kappa * phi * qx)
    jqy = psi0 * (qx * dxuy[..., None] + qy * dyuy[..., None] - lat.kappa * phi * qy)
    scale = np.abs(jqx).max()
    np.testing.assert_allclose(gp @ c25[:, 2], jqx, atol=1e-13 * scale)
    np.testing.assert_allclose(gp @ c25[:, 3], jqy, atol=1e-13 * scale)
    # the velocity-gradient part alone is non-trivial in this state
    assert np.abs(psi0 * qy * dyux[..., None]).max() > 0.05 * scale


@pytest.mark.parametrize("fene_b", [0.0, 4.0])
def test_initial_state_is_a_fixed_point_of_the_collision(oracle_mod, fene_b):
    """Without body force, g = f^eq: the g -> f momenta equal the equilibrium
    ones, so f* = f^eq and the update returns g unchanged."""
    from paper_2201_10132_gb300.inputs import perturbation
    O = oracle_mod
    nx, ny = 10, 8
    lat = _lattice(O, nx, ny, fene_b=fene_b, a0=0.0)
    o = O.Oracle(lat)
    o.init(perturbation(nx, ny, 3, 0.3, 0.05), 1)
    gs, gp = o.get_g()
    o.collide()
    hs, hp = o.get_gpost()
    np.testing.assert_allclose(hs, gs, rtol=0, atol=1e-15)
    np.testing.assert_allclose(hp, gp, rtol=0, atol=1e-14 * np.abs(gp).max())
