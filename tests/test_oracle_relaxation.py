"""Oracle pins: closed-form relaxation of the g-scheme (Sec. VI-C).

With g = f - (dt/2) Omega (reading of Eq. aux with the sign that makes the
update explicit), one collision of a spatially uniform state must
- relax the momentum difference J(g) - J_eq by exactly (2 tau2 - 1)/(2 tau2 + 1),
  for the solvent and for every polymer Q-node (both r and Q momenta);
- relax the non-equilibrium stress by exactly 1 - 2 beta = (2 tau1 - 1)/(2 tau1 + 1);
- reduce, for tau1 = tau2, to the textbook single-relaxation BGK lattice
  Boltzmann update with relaxation time tau + 1/2 and the Guo et al. (2002)
  forcing term (1 - 1/(2 tau_BGK)) F_i.
"""
import numpy as np


def _uniform_lattice(O, tau1, tau2, a0=0.0, H=0.0, psi_tot=0.01, S=4, R=2.0, nx=3, ny=3):
    kappa = 2 * H * tau2
    return O.Lattice(nx=nx, ny=ny, q_side=S, q_radius=R, tau1=tau1, tau2=tau2, H=H, kappa=kappa,
                     ell=2 ** 0.5, psi_tot=psi_tot, sigma_q2=1.0, a0=a0, kf=2 * np.pi / ny,
                     u0=0.05)


def _uniform_state(O, o, us, up, seed=0):
    c9, w9, _ = O.d2q9()
    c25, w25, _ = O.d4q25()
    psi0 = o.psi0()
    cu = c9 @ np.asarray(us)
    fs = w9 * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * np.dot(us, us))
    rng = np.random.default_rng(seed)
    jq = 0.02 * rng.standard_normal((o.nq, 2))
    fp = w25[None, :] * (psi0[:, None] * (1 + 3 * (c25[:, :2] @ np.asarray(up))[None, :])
                         + 3 * psi0[:, None] * (jq @ c25[:, 2:].T))
    gs = np.broadcast_to(fs, (o.ny, o.nx, 9)).copy()
    gp = np.broadcast_to(fp, (o.ny, o.nx, o.nq, 25)).copy()
    return gs, gp


def test_momentum_relaxation_factor(oracle_mod):
    O = oracle_mod
    tau1, tau2 = 0.3, 1.7
    o = O.Oracle(_uniform_lattice(O, tau1, tau2))
    gs, gp = _uniform_state(O, o, [0.02, -0.01], [-0.03, 0.015])
    o.set_g(gs, gp)
    o.collide()
    hs, hp = o.get_gpost()
    c9, _, _ = O.d2q9()
    c25, _, _ = O.d4q25()
    rho_s = gs[0, 0].sum()
    psi = gp[0, 0].sum(-1)
    rho = rho_s + psi.sum()
    J = gs[0, 0] @ c9 + (gp[0, 0] @ c25[:, :2]).sum(0)
    U = J / rho
    fac = (2 * tau2 - 1) / (2 * tau2 + 1)
    dS0 = gs[0, 0] @ c9 - rho_s * U
    dS1 = hs[0, 0] @ c9 - rho_s * U
    np.testing.assert_allclose(dS1, fac * dS0, rtol=1e-12)
    dR0 = gp[0, 0] @ c25[:, :2] - psi[:, None] * U[None, :]
    dR1 = hp[0, 0] @ c25[:, :2] - psi[:, None] * U[None, :]
    np.testing.assert_allclose(dR1, fac * dR0, rtol=1e-11, atol=1e-20)
    # H = 0 and grad U = 0: J^Q_eq = 0, so J^Q(g) itself decays by the same factor
    np.testing.assert_allclose(hp[0, 0] @ c25[:, 2:], fac * (gp[0, 0] @ c25[:, 2:]), rtol=1e-11,
                               atol=1e-20)


def test_stress_relaxation_factor(oracle_mod):
    O = oracle_mod
    tau1, tau2 = 0.45, 2.0
    o = O.Oracle(_uniform_lattice(O, tau1, tau2, psi_tot=0.0))
    c9, w9, _ = O.d2q9()
    # zero-momentum state with a traceless stress perturbation
    pert = 0.01 * (c9[:, 0] ** 2 - c9[:, 1] ** 2) + 0.004 * c9[:, 0] * c9[:, 1]
    fs = w9 * (1.0 + pert)
    gs = np.broadcast_to(fs, (o.ny, o.nx, 9)).copy()
    o.set_g(gs, np.zeros((o.ny, o.nx, o.nq, 25)))
    o.collide()
    hs, _ = o.get_gpost()
    P0 = np.einsum("i,ia,ib->ab", gs[0, 0], c9, c9)
    P1 = np.einsum("i,ia,ib->ab", hs[0, 0], c9, c9)
    Peq = np.eye(2) * gs[0, 0].sum() / 3.0
    fac = (2 * tau1 - 1) / (2 * tau1 + 1)
    np.testing.assert_allclose(P1 - Peq, fac * (P0 - Peq), rtol=1e-12, atol=4e-16)


def test_single_relaxation_reduces_to_textbook_bgk(oracle_mod):
    """tau1 = tau2 = tau: BGK with tau_BGK = tau + 1/2 and Guo forcing (textbook LBM)."""
    O = oracle_mod
    tau = 0.37
    ny = 5
    lat = _uniform_lattice(O, tau, tau, a0=2e-3, psi_tot=0.0, nx=4, ny=ny)
    o = O.Oracle(lat)
    c9, w9, _ = O.d2q9()
    rng = np.random.default_rng(7)
    gs = w9[None, None, :] * (1 + 0.05 * rng.standard_normal((ny, 4, 9)))
    o.set_g(gs, np.zeros((ny, 4, o.nq, 25)))
    o.collide()
    hs, _ = o.get_gpost()
    # textbook: tau_B = tau + 1/2; u = (sum c f + F/2)/rho; f' = f - (f - feq)/tau_B + (1 - 1/(2 tau_B)) S
    tB = tau + 0.5
    rho = gs.sum(-1)
    Fx = rho * lat.a0 * np.sin(lat.kf * np.arange(ny))[:, None]
    ux = (gs @ c9[:, 0] + 0.5 * Fx) / rho
    uy = (gs @ c9[:, 1]) / rho
    ref = np.empty_like(gs)
    for i in range(9):
        cx, cy = c9[i]
        cu = cx * ux + cy * uy
        feq = w9[i] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (ux ** 2 + uy ** 2))
        Si = w9[i] * (3 * (cx - ux) + 9 * cu * cx) * Fx
        ref[..., i] = gs[..., i] - (gs[..., i] - feq) / tB + (1 - 1 / (2 * tB)) * Si
    np.testing.assert_allclose(hs, ref, rtol=1e-13, atol=1e-16)
