"""Oracle pins: conservation laws and structural invariants of the step.

- the collision conserves rho_S and every psi(r, q) node by node (Sec. VI: the
  equilibria share the zeroth moments of f; the g-transform keeps them);
- the collision changes the total momentum by exactly sum (rho a) + sum E, and
  sum E = 0 on a periodic grid (Sec. III: the elastic impulse is a divergence,
  Eq. IDef), so the budget closes to roundoff;
- the elastic force the step uses equals the central-difference divergence of
  the stress Theta = H ell^2 sum_q psi Q Q computed from the fields;
- streaming is a permutation of the populations (bit-exact), with a single
  population landing where the velocity sends it or bounced back at the disk;
- translating the initial state by whole cells in x translates the result
  (bit-exact); point inversion r -> -r maps a solution to a solution.
"""
import numpy as np
import pytest


def _lattice(O, nx=6, ny=5, S=6, R=3.0, tau1=0.3, tau2=0.7, H=0.02, ell=2 ** 0.5, a0=1e-3,
             kf=None, psi_tot=0.01):
    kf = 2 * np.pi / ny if kf is None else kf
    kappa = 2 * H * tau2
    return O.Lattice(nx=nx, ny=ny, q_side=S, q_radius=R, tau1=tau1, tau2=tau2, H=H,
                     kappa=kappa, ell=ell, psi_tot=psi_tot,
                     sigma_q2=tau2 / (3 * kappa) if kappa > 0 else 1.0, a0=a0, kf=kf, u0=0.05)


def _random_state(o, rng, amp=0.02):
    c9, w9, _ = o_mod.d2q9()
    c25, w25, _ = o_mod.d4q25()
    gs = w9[None, None, :] * (1.0 + amp * rng.standard_normal((o.ny, o.nx, 9)))
    psi0 = o.psi0()
    gp = (w25[None, None, None, :] * psi0[None, None, :, None]
          * (1.0 + amp * rng.standard_normal((o.ny, o.nx, o.nq, 25))))
    return gs, gp


o_mod = None


@pytest.fixture(autouse=True)
def _mod(oracle_mod):
    global o_mod
    o_mod = oracle_mod


def test_collision_conserves_zeroth_moments(oracle_mod):
    O = oracle_mod
    o = O.Oracle(_lattice(O))
    rng = np.random.default_rng(1)
    gs, gp = _random_state(o, rng)
    o.set_g(gs, gp)
    o.collide()
    hs, hp = o.get_gpost()
    np.testing.assert_allclose(hs.sum(-1), gs.sum(-1), rtol=1e-14, atol=0)
    np.testing.assert_allclose(hp.sum(-1), gp.sum(-1), rtol=1e-13, atol=1e-18)


def test_collision_momentum_budget(oracle_mod):
    O = oracle_mod
    lat = _lattice(O)
    o = O.Oracle(lat)
    rng = np.random.default_rng(2)
    gs, gp = _random_state(o, rng)
    o.set_g(gs, gp)
    c9, _, _ = O.d2q9()
    c25, _, _ = O.d4q25()
    f = o.fields(with_e=True)
    rho = f["rho_s"] + f["psi_tot"]
    a = lat.a0 * np.sin(lat.kf * np.arange(o.ny))[:, None]
    o.collide()
    hs, hp = o.get_gpost()
    P0 = np.einsum("yxi,ia->a", gs, c9) + np.einsum("yxqi,ia->a", gp, c25[:, :2])
    P1 = np.einsum("yxi,ia->a", hs, c9) + np.einsum("yxqi,ia->a", hp, c25[:, :2])
    # node by node: Delta J = E + rho a
    dJ = (np.einsum("yxi,ia->ayx", hs - gs, c9) + np.einsum("yxqi,ia->ayx", hp - gp, c25[:, :2]))
    np.testing.assert_allclose(dJ[0], f["ex"] + rho * a, atol=1e-15)
    np.testing.assert_allclose(dJ[1], f["ey"], atol=1e-15)
    assert abs(f["ex"].sum()) < 1e-16 and abs(f["ey"].sum()) < 1e-16
    np.testing.assert_allclose(P1 - P0, [(rho * a).sum(), 0.0], atol=1e-14)


def test_elastic_force_is_divergence_of_stress(oracle_mod):
    O = oracle_mod
    o = O.Oracle(_lattice(O, nx=7, ny=6))
    rng = np.random.default_rng(3)
    gs, gp = _random_state(o, rng, amp=0.1)
    o.set_g(gs, gp)
    f = o.fields(with_e=True)

    def dx(a):
        return 0.5 * (np.roll(a, -1, axis=1) - np.roll(a, 1, axis=1))

    def dy(a):
        return 0.5 * (np.roll(a, -1, axis=0) - np.roll(a, 1, axis=0))

    ex = dx(f["thxx"]) + dy(f["thxy"])
    ey = dx(f["thxy"]) + dy(f["thyy"])
    scale = np.abs(f["ex"]).max()
    assert scale > 0
    np.testing.assert_allclose(f["ex"], ex, atol=1e-12 * scale)
    np.testing.assert_allclose(f["ey"], ey, atol=1e-12 * scale)


def test_stream_is_permutation(oracle_mod):
    O = oracle_mod
    o = O.Oracle(_lattice(O))
    rng = np.random.default_rng(4)
    hs = rng.standard_normal((o.ny, o.nx, 9))
    hp = rng.standard_normal((o.ny, o.nx, o.nq, 25))
    o.set_gpost(hs, hp)
    o.stream()
    gs, gp = o.get_g()
    assert np.array_equal(np.sort(gs.ravel()), np.sort(hs.ravel()))
    assert np.array_equal(np.sort(gp.ravel()), np.sort(hp.ravel()))


def test_stream_single_population(oracle_mod):
    O = oracle_mod
    o = O.Oracle(_lattice(O, nx=5, ny=4, S=6, R=3.0))
    c25, _, opp = O.d4q25()
    qx, qy = o.q_nodes()
    qindex = {(a, b): k for k, (a, b) in enumerate(zip(qx.tolist(), qy.tolist()))}
    # the velocity (+1 r_x, 0, +1 Q_x, 0)
    i = [k for k in range(25) if list(c25[k]) == [1, 0, 1, 0]][0]
    # interior Q-node (0.5, 0.5) -> (1.5, 0.5), and r (4, 2) -> (0, 2) periodic
    hp = np.zeros((o.ny, o.nx, o.nq, 25))
    hp[2, 4, qindex[(0.5, 0.5)], i] = 7.0
    o.set_gpost(np.zeros((o.ny, o.nx, 9)), hp)
    o.stream()
    _, gp = o.get_g()
    assert gp[2, 0, qindex[(1.5, 0.5)], i] == 7.0 and np.count_nonzero(gp) == 1
    # edge Q-node (2.5, 0.5) moving +Q_x leaves the disk: bounces back in place as -i
    hp[:] = 0
    hp[1, 3, qindex[(2.5, 0.5)], i] = 5.0
    o.set_gpost(None, hp)
    o.stream()
    _, gp = o.get_g()
    assert gp[1, 3, qindex[(2.5, 0.5)], opp[i]] == 5.0 and np.count_nonzero(gp) == 1
    # solvent: velocity (1, 1) moves (x, y) -> (x+1, y+1)
    c9, _, _ = O.d2q9()
    j = [k for k in range(9) if list(c9[k]) == [1, 1]][0]
    hs = np.zeros((o.ny, o.nx, 9))
    hs[3, 4, j] = 3.0
    o.set_gpost(hs, np.zeros_like(hp))
    o.stream()
    gs, _ = o.get_g()
    assert gs[0, 0, j] == 3.0 and np.count_nonzero(gs) == 1


def test_translation_invariance_x(oracle_mod):
    from paper_2201_10132_gb300.inputs import perturbation
    O = oracle_mod
    lat = O.map_params(12, 8, 4, 2.0, 5.0, 0.5, 0.5, 0.05, 1)
    p = perturbation(12, 8, 11, 0.05, 0.05)
    a = O.Oracle(lat)
    a.init(p, 1)
    a.step(5)
    b = O.Oracle(lat)
    b.init(np.roll(p, 5, axis=2), 1)
    b.step(5)
    ga, pa = a.get_g()
    gb, pb = b.get_g()
    assert np.array_equal(np.roll(ga, 5, axis=1), gb)
    assert np.array_equal(np.roll(pa, 5, axis=1), pb)


def test_point_inversion_symmetry(oracle_mod):
    """r -> -r with U -> -U, Q -> -Q maps a run onto a run (the forcing sin(k y) is odd)."""
    from paper_2201_10132_gb300.inputs import perturbation
    O = oracle_mod
    nx, ny = 8, 8
    lat = O.map_params(nx, ny, 6, 3.0, 5.0, 0.5, 0.5, 0.05, 1)
    p = perturbation(nx, ny, 5, 0.1, 0.05)
    ix = (-np.arange(nx)) % nx
    iy = (-np.arange(ny)) % ny
    pm = -p[:, iy][:, :, ix]
    a = O.Oracle(lat)
    a.init(p, 1)
    a.step(6)
    b = O.Oracle(lat)
    b.init(pm, 1)
    b.step(6)
    fa = a.fields(with_psi=True)
    fb = b.fields(with_psi=True)
    inv = lambda f: f[iy][:, ix]
    np.testing.assert_allclose(inv(fa["ux"]), -fb["ux"], atol=1e-14)
    np.testing.assert_allclose(inv(fa["uy"]), -fb["uy"], atol=1e-14)
    np.testing.assert_allclose(inv(fa["rho_s"]), fb["rho_s"], rtol=1e-13)
    qx, qy = a.q_nodes()
    qi = {(x, y): k for k, (x, y) in enumerate(zip(qx.tolist(), qy.tolist()))}
    qneg = np.array([qi[(-x, -y)] for x, y in zip(qx.tolist(), qy.tolist())])
    np.testing.assert_allclose(inv(fa["psi"])[:, :, qneg], fb["psi"], rtol=1e-12,
                               atol=1e-12 * fa["psi"].max())
