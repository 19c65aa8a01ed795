"""Oracle pins of the stress quasi-equilibrium model (Sec. V, Eq. quasieq2; the
discrete f*_S and f**_P of Sec. VI with the component stresses quasi-conserved).

With the stresses as the quasi-conserved variables, the roles of the two
relaxation times swap (Sec. V): momenta relax at tau1, stresses at tau2. One
collision of a uniform state must therefore
- relax J(g) - J_eq by exactly (2 tau1 - 1)/(2 tau1 + 1) (solvent, and r and Q
  momenta of every polymer Q-node);
- relax P(g) - P_eq by exactly (2 tau2 - 1)/(2 tau2 + 1) (solvent stress, and the
  three polymer blocks P^r, P^rQ, P^Q);
- coincide with the momentum model when tau1 = tau2.
The physics that does not depend on the model must survive the swap: the
Newtonian Kolmogorov profile (viscosity from the stress relaxation time), the
upper-convected Maxwell response of the dumbbells in homogeneous shear and the
bead diffusivity, both set by the momentum relaxation time.
"""
import numpy as np
import pytest

from test_oracle_relaxation import _uniform_state


def _lattice(O, tau1, tau2, qe, a0=0.0, H=0.0, psi_tot=0.01, S=4, R=2.0, nx=3, ny=3):
    tau_m = tau1 if qe == 1 else tau2
    return O.Lattice(nx=nx, ny=ny, q_side=S, q_radius=R, tau1=tau1, tau2=tau2, H=H,
                     kappa=2 * H * tau_m, ell=2 ** 0.5, psi_tot=psi_tot, sigma_q2=1.0, a0=a0,
                     kf=2 * np.pi / ny, u0=0.05, qe_model=qe)


def test_momentum_relaxes_at_tau1(oracle_mod):
    O = oracle_mod
    tau1, tau2 = 0.3, 1.7
    o = O.Oracle(_lattice(O, tau1, tau2, 1))
    gs, gp = _uniform_state(O, o, [0.02, -0.01], [-0.03, 0.015])
    o.set_g(gs, gp)
    o.collide()
    hs, hp = o.get_gpost()
    c9, _, _ = O.d2q9()
    c25, _, _ = O.d4q25()
    rho_s = gs[0, 0].sum()
    psi = gp[0, 0].sum(-1)
    rho = rho_s + psi.sum()
    U = (gs[0, 0] @ c9 + (gp[0, 0] @ c25[:, :2]).sum(0)) / rho
    fac = (2 * tau1 - 1) / (2 * tau1 + 1)
    np.testing.assert_allclose(hs[0, 0] @ c9 - rho_s * U, fac * (gs[0, 0] @ c9 - rho_s * U),
                               rtol=1e-11)
    np.testing.assert_allclose(hp[0, 0] @ c25[:, :2] - psi[:, None] * U,
                               fac * (gp[0, 0] @ c25[:, :2] - psi[:, None] * U), rtol=1e-10,
                               atol=1e-20)
    np.testing.assert_allclose(hp[0, 0] @ c25[:, 2:], fac * (gp[0, 0] @ c25[:, 2:]), rtol=1e-10,
                               atol=1e-20)


def test_solvent_stress_relaxes_at_tau2(oracle_mod):
    O = oracle_mod
    tau1, tau2 = 0.45, 2.0
    o = O.Oracle(_lattice(O, tau1, tau2, 1, psi_tot=0.0))
    c9, w9, _ = O.d2q9()
    pert = 0.01 * (c9[:, 0] ** 2 - c9[:, 1] ** 2) + 0.004 * c9[:, 0] * c9[:, 1]
    gs = np.broadcast_to(w9 * (1.0 + pert), (o.ny, o.nx, 9)).copy()
    o.set_g(gs, np.zeros((o.ny, o.nx, o.nq, 25)))
    o.collide()
    hs, _ = o.get_gpost()
    P0 = np.einsum("i,ia,ib->ab", gs[0, 0], c9, c9)
    P1 = np.einsum("i,ia,ib->ab", hs[0, 0], c9, c9)
    Peq = np.eye(2) * gs[0, 0].sum() / 3.0
    fac = (2 * tau2 - 1) / (2 * tau2 + 1)
    np.testing.assert_allclose(P1 - Peq, fac * (P0 - Peq), rtol=1e-12, atol=4e-16)


def test_polymer_stress_blocks_relax_at_tau2(oracle_mod):
    O = oracle_mod
    tau1, tau2 = 0.35, 1.4
    o = O.Oracle(_lattice(O, tau1, tau2, 1, S=4, R=2.0))
    c25, w25, _ = O.d4q25()
    c9, w9, _ = O.d2q9()
    rng = np.random.default_rng(3)
    psi0 = o.psi0()
    # zero momenta, a random symmetric second-moment perturbation of each Q-node
    A = rng.normal(0, 0.05, (o.nq, 4, 4))
    A = A + A.transpose(0, 2, 1)
    herm = np.einsum("qab,ia,ib->qi", A, c25, c25) - np.einsum("qaa->q", A)[:, None] / 3.0
    fp = w25[None, :] * psi0[:, None] * (1.0 + herm)
    gs = np.broadcast_to(w9, (o.ny, o.nx, 9)).copy()
    gp = np.broadcast_to(fp, (o.ny, o.nx, o.nq, 25)).copy()
    o.set_g(gs, gp)
    o.collide()
    _, hp = o.get_gpost()
    P0 = np.einsum("qi,ia,ib->qab", gp[0, 0], c25, c25)
    P1 = np.einsum("qi,ia,ib->qab", hp[0, 0], c25, c25)
    psi = gp[0, 0].sum(-1)
    Peq = psi[:, None, None] * np.eye(4)[None] / 3.0
    fac = (2 * tau2 - 1) / (2 * tau2 + 1)
    assert np.abs(P0 - Peq).max() > 1e-6                # the test state is off equilibrium
    np.testing.assert_allclose(P1 - Peq, fac * (P0 - Peq), rtol=1e-10, atol=1e-18)


def test_equal_times_reduce_to_the_momentum_model(oracle_mod):
    O = oracle_mod
    out = []
    for qe in (0, 1):
        o = O.Oracle(_lattice(O, 0.6, 0.6, qe, a0=1e-3, H=0.01, nx=5, ny=4))
        gs, gp = _uniform_state(O, o, [0.02, -0.01], [-0.03, 0.015], seed=4)
        rng = np.random.default_rng(5)
        gs = gs * (1 + 0.01 * rng.standard_normal(gs.shape))
        gp = gp * (1 + 0.01 * rng.standard_normal(gp.shape))
        o.set_g(gs, gp)
        o.collide()
        out.append(o.get_gpost())
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-13, atol=1e-17)
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-11, atol=1e-18)


def test_mapping_orders_the_times(oracle_mod):
    O = oracle_mod
    a = O.map_params(32, 32, 4, 2.0, 5.0, 0.5, 0.2, 0.05, 1, qe_model=1)
    assert a.qe_model == 1 and a.tau1 == a.tau2          # default: tau_m = tau_s
    tau_s = a.tau2
    b = O.map_params(32, 32, 4, 2.0, 5.0, 0.5, 0.2, 0.05, 1, tau2=0.5 * tau_s, qe_model=1)
    assert b.tau1 == pytest.approx(0.5 * tau_s) and b.tau2 == pytest.approx(tau_s)
    assert b.kappa == pytest.approx(2 * b.H * b.tau1)
    with pytest.raises(ValueError):       # the momentum model needs tau_m >= tau_s
        O.map_params(32, 32, 4, 2.0, 5.0, 0.5, 0.2, 0.05, 1, tau2=0.5 * tau_s, qe_model=0)
    with pytest.raises(ValueError):       # the stress model needs tau_m <= tau_s
        O.map_params(32, 32, 4, 2.0, 5.0, 0.5, 0.2, 0.05, 1, tau2=2.0 * tau_s, qe_model=1)


def test_newtonian_profile_with_stress_model(oracle_mod):
    """Viscosity c_s^2 tau2 (the stress relaxation time) whatever the faster tau1: the
    steady profile converges to a0/(nu k^2) sin(k y) at second order in the grid
    (unlike the single-relaxation case, the two relaxation times leave an O(k^2 tau^2)
    error, about 0.4% at 32 nodes per wavelength)."""
    O = oracle_mod
    nu = 1.0 / 6.0
    errs = []
    for ny in (16, 32, 64):
        re = 0.05 * ny / (2 * np.pi * nu)
        lat = O.map_params(4, ny, 1, 1.0, re, 0.0, 1.0, 0.05, 1, tau2=0.2, qe_model=1)
        assert lat.tau1 == pytest.approx(0.2) and lat.tau2 == pytest.approx(0.5)
        o = O.Oracle(lat)
        o.init(None, 1)
        o.step(int(14 / (lat.nu * lat.kf ** 2)))
        f = o.fields()
        y = np.arange(ny)
        ref = lat.a0 / (lat.nu * lat.kf ** 2) * np.sin(lat.kf * y)
        errs.append(np.abs(f["ux"][:, 0] - ref).max() / np.abs(ref).max())
    assert errs[2] < 2e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_ucm_shear_with_stress_model(oracle_mod):
    """The dumbbells' Q-space drift and diffusion come from the momentum relaxation time
    (tau1 here): the UCM steady shear and its decay at 1/lambda_H hold as in the
    momentum model."""
    O = oracle_mod
    tau_m, tau_s, sigma2 = 0.05, 0.2, 4.0
    kappa = tau_m / (3 * sigma2)
    lat = O.Lattice(nx=1, ny=1, q_side=24, q_radius=12.0, tau1=tau_m, tau2=tau_s,
                    H=kappa / (2 * tau_m), kappa=kappa, ell=2 ** 0.5, psi_tot=1e-3,
                    sigma_q2=sigma2, a0=0.0, kf=1.0, u0=0.0, qe_model=1)
    lam = 1.0 / (2 * kappa)
    wi = 0.5
    o = O.Oracle(lat)
    o.init(None, 0)
    o.impose_gradient([[0.0, 0.0], [wi / lam, 0.0]])
    o.step(int(15 * lam))
    f = o.fields()
    l2 = lat.ell ** 2
    assert f["cxy"][0, 0] / l2 == pytest.approx(wi * sigma2, rel=1e-3)
    assert f["cxx"][0, 0] / l2 - sigma2 == pytest.approx(2 * wi ** 2 * sigma2, rel=2e-3)
    assert f["cyy"][0, 0] / l2 == pytest.approx(sigma2, rel=1e-3)


def test_bead_diffusion_with_stress_model(oracle_mod):
    """Without springs the bead density diffuses at c_s^2 tau_m = tau1 / 3."""
    O = oracle_mod
    from test_oracle_physics import _diffusion_rate
    tau_m, tau_s = 0.2, 0.6
    kw = dict(q_side=28, q_radius=14.0, tau1=tau_m, tau2=tau_s, H=0.0, kappa=0.0, ell=2 ** 0.5,
              psi_tot=1e-3, sigma_q2=2.0, a0=0.0, kf=1.0, u0=0.0, qe_model=1)
    c25, w25, _ = O.d4q25()
    probe = O.Oracle(O.Lattice(nx=1, ny=1, **kw))
    prof = w25[None, :] * probe.psi0()[:, None]
    nx = 32
    D = _diffusion_rate(O, kw, nx, prof, 20, 300, 2 * np.pi / nx)
    assert D == pytest.approx(tau_m / 3, rel=5e-3)


def test_momentum_budget_with_stress_model(oracle_mod):
    """Node by node the collision adds E + rho a to the total momentum (the polymer's
    J^r_eq carries tau1 D, and beta (1 + 2 tau1) = 1 closes the budget)."""
    O = oracle_mod
    from test_oracle_invariants import _random_state, _lattice as inv_lattice
    import test_oracle_invariants as inv
    inv.o_mod = O
    lat = inv_lattice(O, tau1=0.3, tau2=0.7)
    lat.qe_model = 1
    lat.kappa = 2 * lat.H * lat.tau1
    o = O.Oracle(lat)
    gs, gp = _random_state(o, np.random.default_rng(2))
    o.set_g(gs, gp)
    c9, _, _ = O.d2q9()
    c25, _, _ = O.d4q25()
    f = o.fields(with_e=True)
    rho = f["rho_s"] + f["psi_tot"]
    a = lat.a0 * np.sin(lat.kf * np.arange(o.ny))[:, None]
    o.collide()
    hs, hp = o.get_gpost()
    dJ = (np.einsum("yxi,ia->ayx", hs - gs, c9) + np.einsum("yxqi,ia->ayx", hp - gp, c25[:, :2]))
    np.testing.assert_allclose(dJ[0], f["ex"] + rho * a, atol=1e-15)
    np.testing.assert_allclose(dJ[1], f["ey"], atol=1e-15)
    np.testing.assert_allclose(hs.sum(-1), gs.sum(-1), rtol=1e-14)
    np.testing.assert_allclose(hp.sum(-1), gp.sum(-1), rtol=1e-13, atol=1e-18)
