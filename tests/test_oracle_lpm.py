"""Pins of the learned-macro-step oracle (oracle/lpm_oracle.py).

The network: bfloat16 rounding against hand-made values, GELU against the
normal CDF's closed-form values, backpropagation against central finite
differences of the loss, one Adam step against its closed form. The lattice
pieces: the solvent sub-step against the C oracle's plain solvent step
(Newtonian limit) and the momentum budget, the reshape's moment conditions,
advection on fields it must move exactly, the feature layout on a field with
a known gradient, and a whole block in the Newtonian limit against 1 + K plain
steps of the C oracle.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def L(oracle_mod):
    from oracle import lpm_oracle
    return lpm_oracle


def test_bf16_rounding(L):
    one = 1.0
    cases = [(one, one), (one + 2 ** -8, one),                  # halfway: ties to even (down)
             (one + 3 * 2 ** -8, one + 2 ** -6),                # halfway: ties to even (up)
             (one + 2 ** -8 + 2 ** -20, one + 2 ** -7),         # above halfway
             (-(one + 2 ** -8 + 2 ** -20), -(one + 2 ** -7)), (3.0, 3.0), (0.0, 0.0),
             (1000.0, 1000.0), (1001.0, 1000.0)]                # 1001 = 1000 + 1 < half-ulp (4)
    x = np.array([c[0] for c in cases])
    assert np.array_equal(L.bf16(x), np.array([c[1] for c in cases]))


def test_gelu_values(L):
    # Phi(1) and Phi(-1) of the standard normal distribution
    assert L.gelu(np.array(1.0)) == pytest.approx(0.8413447460685429, rel=1e-15)
    assert L.gelu(np.array(-1.0)) == pytest.approx(-0.15865525393145707, rel=1e-14)
    assert L.gelu(np.array(0.0)) == 0.0
    assert L.gelu_grad(np.array(0.0)) == pytest.approx(0.5, rel=1e-15)
    assert L.gelu(np.array(12.0)) == pytest.approx(12.0, rel=1e-15)
    assert abs(L.gelu(np.array(-12.0))) < 1e-30
    z = np.linspace(-4, 4, 17)
    h = 1e-6
    fd = (L.gelu(z + h) - L.gelu(z - h)) / (2 * h)
    assert np.abs(fd - L.gelu_grad(z)).max() < 1e-9


def test_backprop_matches_finite_differences(L):
    rng = np.random.default_rng(3)
    P = {"W1": rng.normal(0, 0.5, (7, 5)), "b1": rng.normal(0, 0.1, 7),
         "W2": rng.normal(0, 0.5, (6, 7)), "b2": rng.normal(0, 0.1, 6),
         "W3": rng.normal(0, 0.5, (3, 6)), "b3": rng.normal(0, 0.1, 3)}
    X = rng.normal(0, 1, (9, 5))
    T = rng.normal(0, 1, (9, 3))
    _, g = L.loss_and_grads(P, X, T)
    h = 1e-6
    for k, v in P.items():
        for idx in list(np.ndindex(v.shape))[:12]:
            Pp = {kk: vv.copy() for kk, vv in P.items()}
            Pm = {kk: vv.copy() for kk, vv in P.items()}
            Pp[k][idx] += h
            Pm[k][idx] -= h
            fd = (L.loss_and_grads(Pp, X, T)[0] - L.loss_and_grads(Pm, X, T)[0]) / (2 * h)
            assert g[k][idx] == pytest.approx(fd, rel=1e-6, abs=1e-9), (k, idx)


def test_adam_first_step_closed_form(L):
    master = {"W": np.array([[0.5, -0.25]]), "b": np.array([1.0])}
    grads = {"W": np.array([[2.0, -1e-3]]), "b": np.array([0.0])}
    st = {}
    L.adam(master, grads, st, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step lr g / (|g| + eps)
    assert master["W"][0, 0] == pytest.approx(0.5 - 0.01 * 2.0 / (2.0 + 1e-8), rel=1e-15)
    assert master["W"][0, 1] == pytest.approx(-0.25 + 0.01 * 1e-3 / (1e-3 + 1e-8), rel=1e-14)
    assert master["b"][0] == 1.0


def _newtonian(O, nx=24, ny=16):
    from paper_2201_10132_gb300.inputs import perturbation
    lat = O.map_params(nx, ny, 1, 1.0, 5.0, 0.0, 1.0, 0.05, 1)   # beta = 1: no polymer
    o = O.Oracle(lat)
    o.init(perturbation(nx, ny, 2, 0.2, 0.05), 1)
    o.step(3)
    return lat, o


def test_solvent_substep_is_the_plain_solvent_step(L, oracle_mod):
    O = oracle_mod
    lat, o = _newtonian(O)
    s = L.Setup(lat, K=4, tile=8)
    gs, _ = o.get_g()
    g = np.moveaxis(gs, -1, 0).copy()
    zero_c = np.zeros((3, lat.ny, lat.nx))
    mine = L.collide(s, g, np.zeros((lat.ny, lat.nx)), zero_c)
    o.collide()
    ref, _ = o.get_gpost()
    assert np.abs(mine - np.moveaxis(ref, -1, 0)).max() < 1e-15
    o.stream()
    pulled, _ = o.get_g()
    assert np.array_equal(L.pull(s, mine), np.moveaxis(pulled, -1, 0)) or \
        np.abs(L.pull(s, mine) - np.moveaxis(pulled, -1, 0)).max() < 1e-15


def test_substep_momentum_budget(L, oracle_mod):
    """With the polymer slaved (dP = 0) each collision adds exactly E + rho a to J_S."""
    O = oracle_mod
    lat = O.map_params(32, 24, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1)
    s = L.Setup(lat, K=4, tile=8)
    rng = np.random.default_rng(1)
    y, x = np.mgrid[0:24, 0:32]
    psi = lat.psi_tot * (1 + 0.1 * np.sin(2 * np.pi * x / 32))
    C = np.stack([s.c_e * (1 + 0.3 * np.cos(2 * np.pi * y / 24)), 0.2 * s.c_e * np.sin(2 * np.pi * x / 32),
                  s.c_e * np.ones((24, 32))])
    g = s.w9[:, None, None] * (1 + 0.01 * rng.normal(size=(9, 24, 32)))
    out = L.collide(s, g, psi, C)
    E = L.elastic_force(s, psi, C)
    rho = g.sum(0) + psi
    for a in range(2):
        dj = ((out - g) * s.c9[:, a, None, None]).sum(0)
        force = E[a] + (rho * s.arow[:, None] if a == 0 else 0.0)
        assert np.abs(dj - force).max() < 1e-15    # |J_S| ~ 1e-2: rounding of the sums
    assert np.abs(out.sum(0) - g.sum(0)).max() < 1e-15                      # mass
    assert abs(E.sum()) < 1e-18 * E.size                                      # div of a periodic field


def test_reshape_moment_conditions(L, oracle_mod):
    from paper_2201_10132_gb300.inputs import perturbation
    O = oracle_mod
    lat = O.map_params(32, 32, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1)
    o = O.Oracle(lat)
    o.init(perturbation(32, 32, 4, 0.3, 0.05), 1)
    o.step(20)
    s = L.Setup(lat, K=4, tile=16)
    gs, gp = o.get_g()
    C = L.conformation(o.fields())
    target = C * np.array([1.05, 0.9, 0.97])[:, None, None] + np.array([0.0, 0.05, 0.0])[:, None, None]
    dg = L.reshape_increment(s, np.moveaxis(gs, -1, 0), gp, target)
    o.set_g(gs, gp + dg)
    f = o.fields()
    assert np.abs(L.conformation(f) - target).max() < 1e-12 * np.abs(target).max()
    c25, _, _ = O.d4q25()
    assert np.abs(dg.sum((-1, -2))).max() < 1e-18                           # polymer mass per node
    for a in range(2):
        assert np.abs((dg * c25[:, a]).sum((-1, -2))).max() < 1e-19         # r-momentum per node


def test_advect_moves_fields_exactly(L, oracle_mod):
    O = oracle_mod
    lat = O.map_params(32, 16, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1)
    s = L.Setup(lat, K=4, tile=16)
    rng = np.random.default_rng(0)
    F = rng.normal(size=(2, 16, 32))
    U = np.stack([np.full((16, 32), 0.5), np.full((16, 32), -0.25)])          # K U = (2, -1)
    assert np.array_equal(L.advect(s, F, U), np.roll(np.roll(F, 2, axis=-1), -1, axis=-2))
    # bilinear interpolation reproduces an affine field away from the periodic seam
    y, x = np.mgrid[0:16, 0:32].astype(float)
    A = 0.3 * x - 0.7 * y + 2.0
    U = np.stack([0.11 + 0.01 * np.sin(y), -0.07 + 0.01 * np.cos(x)])
    out = L.advect(s, A, U)
    ref = 0.3 * (x - 4 * U[0]) - 0.7 * (y - 4 * U[1]) + 2.0
    inner = (slice(3, -3), slice(3, -3))
    assert np.abs(out[inner] - ref[inner]).max() < 1e-13


def test_feature_layout(L, oracle_mod):
    O = oracle_mod
    lat = O.map_params(32, 16, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1)
    s = L.Setup(lat, K=4, tile=16)
    y, x = np.mgrid[0:16, 0:32].astype(float)
    kx, ky = 2 * np.pi / 32, 2 * np.pi / 16
    U = np.stack([np.sin(ky * y), np.cos(kx * x)])        # only dU_x/dy and dU_y/dx are non-zero
    C = np.stack([s.c_e * np.ones_like(x), np.zeros_like(x), s.c_e * np.ones_like(x)])
    X = L.features(s, U, C).reshape(16, 32, 40)
    assert np.abs(X[..., :3]).max() == 0.0
    assert np.allclose(X[..., 39], 4 / lat.lambda_h)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            base = 3 + 4 * ((dy + 1) * 3 + (dx + 1))
            yy, xx = (y + dy) % 16, (x + dx) % 32
            # central differences of sin / cos: exact discrete derivatives
            dux_dy = np.sin(ky) * np.cos(ky * yy)
            duy_dx = -np.sin(kx) * np.sin(kx * xx)
            assert np.abs(X[..., base + 0]).max() < 1e-15
            assert np.abs(X[..., base + 1] - 4 * duy_dx).max() < 1e-14
            assert np.abs(X[..., base + 2] - 4 * dux_dy).max() < 1e-14
            assert np.abs(X[..., base + 3]).max() < 1e-15


def test_newtonian_block_is_plain_steps(L, oracle_mod):
    """Without polymer a block (any mode) is 1 + K plain steps."""
    O = oracle_mod
    lat, o = _newtonian(O)
    ref = O.Oracle(lat)
    ref.set_g(*o.get_g())
    s = L.Setup(lat, K=4, tile=8)
    L.block(s, o, None, "frozen")
    ref.step(1 + s.K)
    a, b = o.fields(), ref.fields()
    for k in ("rho_s", "ux", "uy"):
        assert np.abs(a[k] - b[k]).max() < 1e-15, k


def test_slaved_polymer_momentum_closure(L, oracle_mod):
    """Solvent sub-steps fed with the plain run's own polymer stress follow the plain
    run: the velocity error after K = 8 steps is a few per cent of the velocity change."""
    from paper_2201_10132_gb300.inputs import perturbation
    O = oracle_mod
    lat = O.map_params(32, 32, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1)
    o = O.Oracle(lat)
    o.init(perturbation(32, 32, 6, 0.3, 0.05), 1)
    o.step(60)
    s = L.Setup(lat, K=8, tile=16)
    gs, gp = o.get_g()
    f0 = o.fields()
    dP = L.polymer_momentum_offset(s, gs, gp, f0)
    g = np.moveaxis(gs, -1, 0).copy()
    U0 = np.stack([f0["ux"], f0["uy"]])
    for _ in range(s.K):
        f = o.fields()
        g = L.pull(s, L.collide(s, g, f["psi_tot"], L.conformation(f), dP))
        o.step(1)
    f = o.fields()
    U_ref = np.stack([f["ux"], f["uy"]])
    _, U, _, _ = L.velocity(s, g, f["psi_tot"], L.conformation(f), dP)
    assert np.abs(U - U_ref).max() < 0.05 * np.abs(U_ref - U0).max()
