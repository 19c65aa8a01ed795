"""FP64 oracle of the learned polymer macro-step (numpy + the C oracle).

TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing else. It restates,
plainly and slowly, what the CUDA library's learned mode computes, and shares
no code with it.

The paper has no learned step; this one is built on the paper's scheme. A
block advances the state (the plain scheme's populations) by 1 + K lattice
steps:

 1. One plain step of the scheme (Sec. VI), t -> t + 1. The conformation
    C = ell^2 sum_q psi Q Q / psi_tot (r-lengths^2) before and after it gives
    the plain update's rate r = C(t + 1) - C(t), and U(t + 1) is the mixture
    velocity of the new state.
 2. The parcel arriving at r during the next K steps left from r - K U(r):
    C_dep is C(t + 1) interpolated there (bilinear, periodic).
 3. Features per node (40): (C_dep - c_e I)/c_e (3; c_e the lattice
    equilibrium C_xx), K dU_b/dr_a at the 3 x 3 stencil around the node (36,
    order dy, dx, then dU_x/dx, dU_y/dx, dU_x/dy, dU_y/dy), and K / lambda_H.
    A multilayer perceptron 40 -> 64 -> 64 -> 3 (GELU, BF16 weights, FP32
    biases) predicts o = (C(t + 1 + K) - C_dep) / c_e: C_new = C_dep + c_e o.
 4. Check and fallback: per node e = max_ab |C_new - C(t + 1) - K r| / c_e,
    the network's change against the plain update's rate carried over the K
    steps; every T x T tile whose largest e exceeds the threshold keeps the
    plain update's C(t + 1) (no learned change) on all its nodes instead.
 5. K solvent sub-steps; sub-step j (j = 0..K-1) sees the polymer stress
    Theta = (H / 2) psi_tot C of C(t + 1) + (j / K)(C_new - C(t + 1)) (Sec. III:
    (H ell^2 / 2) sum_q psi Q Q), E = div Theta by central differences. The
    polymer momentum is slaved to psi_tot U + tau2 E + dP, dP its offset in the
    plain state at t + 1, which turns the mixture velocity of Sec. VI-C into
    rho_S U = J_S(g) + (tau2 + 1/2) E + rho a / 2 + dP (rho = rho_S + psi_tot);
    the solvent then collides exactly as in the plain step (two relaxations,
    Guo source of the force rho a).
 6. The polymer populations of t + 1 (pulled) are reshaped at every node so
    that their conformation is C_new: psi(q) changes by dpsi(q) = psi_tot p0(q)
    sum_ab w_ab beta_ab (Q_a Q_b - m0_ab) (p0 the normalised equilibrium, m0 its
    second moments, w = 1, 2, 1), the three beta from the constant 3 x 3 system
    that makes the change of the second moments (C_new - C) / ell^2 (psi_tot is
    unchanged; weighting by the equilibrium rather than by the node's own psi
    keeps the system well conditioned where psi(q) is far from equilibrium or
    partly negative, as it is in strong shear on a truncated disk); dpsi enters as the
    linear quasi-equilibrium of Sec. VI-B (populations w_i [dpsi + 3 (v_i .
    dpsi U + Qdot_i . dpsi (Q . grad U - kappa Q))]), U and grad U those of the
    reshaped state. The solvent populations are those of the last sub-step.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import oracle as O

NIN, NH, NOUT = 40, 64, 3


# ---------------------------------------------------------------- the network
def bf16(a) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    """GELU(z) = z Phi(z), Phi the standard normal CDF (Hendrycks & Gimpel 2016)."""
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(seed: int, nin=NIN, nh=NH, nout=NOUT):
    """FP32 master parameters: weights uniform in +-sqrt(6 / (fan_in + fan_out))
    (Glorot & Bengio 2010), zero biases; the output layer scaled by 0.1."""
    rng = np.random.default_rng(seed)
    def glorot(o, i, s=1.0):
        lim = s * np.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, (o, i)).astype(np.float32).astype(np.float64)
    return {"W1": glorot(nh, nin), "b1": np.zeros(nh), "W2": glorot(nh, nh), "b2": np.zeros(nh),
            "W3": glorot(nout, nh, 0.1), "b3": np.zeros(nout)}


def compute_weights(master):
    """The weights the network computes with: BF16 matrices, FP32 biases."""
    out = {}
    for k, v in master.items():
        out[k] = bf16(v) if k.startswith("W") else np.float32(v).astype(np.float64)
    return out


def forward(P, X):
    """Two GELU hidden layers and a linear output; X [N, nin] -> O [N, nout]."""
    z1 = X @ P["W1"].T + P["b1"]
    a1 = gelu(z1)
    z2 = a1 @ P["W2"].T + P["b2"]
    a2 = gelu(z2)
    o = a2 @ P["W3"].T + P["b3"]
    return o, (X, z1, a1, z2, a2)


def apply(net, X):
    """The trained network on raw features: inputs standardised by (mx, sx), outputs
    rescaled by (st, mt): o = st * MLP((X - mx) / sx) + mt."""
    o, _ = forward(net, (X - net["mx"]) / net["sx"])
    return o * net["st"] + net["mt"]


def loss_and_grads(P, X, T):
    """L = (1/N) sum_n sum_j (o_nj - t_nj)^2 and dL/dparameter by the chain rule."""
    n = X.shape[0]
    o, (x, z1, a1, z2, a2) = forward(P, X)
    r = o - T
    loss = float((r * r).sum() / n)
    do = 2.0 * r / n
    g = {"W3": do.T @ a2, "b3": do.sum(0)}
    dz2 = (do @ P["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return loss, g


def adam(master, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on the FP32 master parameters, in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in master:
        m = state.setdefault("m_" + k, np.zeros_like(master[k]))
        v = state.setdefault("v_" + k, np.zeros_like(master[k]))
        m[...] = b1 * m + (1 - b1) * grads[k]
        v[...] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        master[k] = master[k] - lr * mh / (np.sqrt(vh) + eps)


# ---------------------------------------------------------------- lattice pieces
class Setup:
    """Lattice parameters and tables of one learned run (from the C oracle's mapping)."""

    def __init__(self, lat: O.Lattice, K: int = 8, tile: int = 32, threshold: float = 0.05):
        self.lat = lat
        self.K = K
        self.tile = tile
        self.threshold = threshold
        self.nx, self.ny = lat.nx, lat.ny
        c9, w9, _ = O.d2q9()
        self.c9, self.w9 = c9.astype(np.float64), w9
        one = O.Oracle(O.Lattice(**{**lat.as_dict(), "nx": 1, "ny": 1}))
        self.qx, self.qy = one.q_nodes()
        psi0 = one.psi0()
        # lattice equilibrium C_xx (1 when there is no polymer: it only scales features)
        self.c_e = lat.ell ** 2 * (psi0 * self.qx * self.qx).sum() / psi0.sum() if psi0.sum() > 0 \
            else 1.0
        self.qq = np.stack([self.qx * self.qx, self.qx * self.qy, self.qy * self.qy])  # [3, nq]
        self.p0 = psi0 / psi0.sum() if psi0.sum() > 0 else np.zeros_like(psi0)
        self.m0 = self.qq @ self.p0                        # equilibrium second moments
        y = np.arange(self.ny)
        self.arow = lat.a0 * np.sin(lat.kf * y)
        self.beta = 1.0 / (2.0 * lat.tau1 + 1.0)


def _shift(a, dx, dy):
    """a evaluated at (x + dx, y + dy), periodic; a [..., ny, nx]."""
    return np.roll(np.roll(a, -dy, axis=-2), -dx, axis=-1)


def _ddx(a):
    return 0.5 * (_shift(a, 1, 0) - _shift(a, -1, 0))


def _ddy(a):
    return 0.5 * (_shift(a, 0, 1) - _shift(a, 0, -1))


def pull(s: Setup, gpost):
    """g_i(x) = g'_i(x - c_i), periodic (Sec. VI-A streaming); [9, ny, nx]."""
    g = np.empty_like(gpost)
    for i in range(9):
        g[i] = _shift(gpost[i], -int(s.c9[i, 0]), -int(s.c9[i, 1]))
    return g


def elastic_force(s: Setup, psi, C):
    """E = div Theta, Theta = (H / 2) psi_tot C, central differences."""
    th = 0.5 * s.lat.H * psi[None] * C           # [3, ny, nx]: xx, xy, yy
    return np.stack([_ddx(th[0]) + _ddy(th[1]), _ddx(th[1]) + _ddy(th[2])])


def velocity(s: Setup, g, psi, C, dP=0.0):
    """rho_S, U, the mixture force density rho a and J_S(g) of the pulled solvent g
    under (psi, C). The polymer momentum is slaved: J_P(g) = psi_tot U + tau2 E + dP
    (psi_tot U + tau2 E is the sum over Q of J^r_eq = psi U + tau2 D, as sum_q D = E;
    dP, held over the block, is what the plain state at its start has beyond it), so
    rho U = J_S + J_P + (E + rho a) / 2 gives
    rho_S U = J_S(g) + (tau2 + 1/2) E + rho a / 2 + dP."""
    rho_s = g.sum(0)
    jx = (g * s.c9[:, 0, None, None]).sum(0)
    jy = (g * s.c9[:, 1, None, None]).sum(0)
    E = elastic_force(s, psi, C)
    rho = rho_s + psi
    fa = rho * s.arow[:, None]
    t = s.lat.tau2 + 0.5
    dP = np.broadcast_to(dP, (2,) + rho_s.shape)
    U = np.stack([(jx + t * E[0] + 0.5 * fa + dP[0]) / rho_s, (jy + t * E[1] + dP[1]) / rho_s])
    return rho_s, U, fa, np.stack([jx, jy])


def polymer_momentum_offset(s: Setup, gs, gp, f):
    """dP = J_P(g) - psi_tot U - tau2 E of a plain state (oracle layouts; f its fields)."""
    c25, _, _ = O.d4q25()
    jp = np.stack([(gp * c25[:, 0]).sum((-1, -2)), (gp * c25[:, 1]).sum((-1, -2))])
    C = conformation(f)
    E = elastic_force(s, f["psi_tot"], C)
    U = np.stack([f["ux"], f["uy"]])
    return jp - f["psi_tot"] * U - s.lat.tau2 * E


def collide(s: Setup, g, psi, C, dP=0.0):
    """Solvent sub-step: the solvent collision of Sec. VI-C with the U above,
    J_S(f) = (2 tau2 J_S(g) + rho_S U + tau2 rho a) / (2 tau2 + 1), u_S = J_S(f) / rho_S,
    g' = (1 - 2 beta) g + 2 beta [(1 - tau1/tau2) f^eq(u_S) + (tau1/tau2) f^eq(U)]
         + (1 - beta) S_i, S_i the Guo source of the force (rho a, 0)."""
    rho_s, U, fa, J = velocity(s, g, psi, C, dP)
    lat = s.lat
    c2 = 2.0 * lat.tau2
    usx = (c2 * J[0] + rho_s * U[0] + lat.tau2 * fa) / (c2 + 1.0) / rho_s
    usy = (c2 * J[1] + rho_s * U[1]) / (c2 + 1.0) / rho_s
    r = lat.tau1 / lat.tau2
    b = s.beta
    out = np.empty_like(g)
    for i in range(9):
        cx, cy = s.c9[i]
        cu = cx * U[0] + cy * U[1]
        cs = cx * usx + cy * usy
        feq = s.w9[i] * rho_s * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (U[0] ** 2 + U[1] ** 2))
        fst = s.w9[i] * rho_s * (1.0 + 3.0 * cs + 4.5 * cs * cs - 1.5 * (usx ** 2 + usy ** 2))
        src = s.w9[i] * (3.0 * (cx - U[0]) + 9.0 * cu * cx) * fa
        out[i] = (1.0 - 2.0 * b) * g[i] + 2.0 * b * ((1.0 - r) * fst + r * feq) + (1.0 - b) * src
    return out


def grad_u(U):
    """G[a][b] = dU_b / dr_a by central differences: [2, 2, ny, nx]."""
    return np.array([[_ddx(U[0]), _ddx(U[1])], [_ddy(U[0]), _ddy(U[1])]])


def features(s: Setup, U, C_dep):
    """[ny * nx, 40] network inputs (node order y-major)."""
    K, ce = s.K, s.c_e
    G = grad_u(U)
    cols = [(C_dep[0] - ce) / ce, C_dep[1] / ce, (C_dep[2] - ce) / ce]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            for a, b in ((0, 0), (0, 1), (1, 0), (1, 1)):
                cols.append(K * _shift(G[a, b], dx, dy))
    cols.append(np.full(U[0].shape, K / s.lat.lambda_h))
    return np.stack([c.ravel() for c in cols], axis=1)


def advect(s: Setup, F, U):
    """Bilinear interpolation of F [..., ny, nx] at r - K U(r), periodic."""
    ny, nx = s.ny, s.nx
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    px = xx - s.K * U[0]
    py = yy - s.K * U[1]
    x0 = np.floor(px)
    y0 = np.floor(py)
    fx, fy = px - x0, py - y0
    x0 = x0.astype(np.int64) % nx
    y0 = y0.astype(np.int64) % ny
    x1, y1 = (x0 + 1) % nx, (y0 + 1) % ny
    return ((1 - fy) * ((1 - fx) * F[..., y0, x0] + fx * F[..., y0, x1]) +
            fy * ((1 - fx) * F[..., y1, x0] + fx * F[..., y1, x1]))


def reshape_dpsi(s: Setup, psi_q, C_new):
    """dpsi[ny, nx, nq]: the change of psi(q) that moves the conformation of psi_q
    [ny, nx, nq] to C_new [3, ny, nx] at unchanged psi_tot: the equilibrium-weighted
    second-order form dpsi(q) = psi_tot p0(q) sum_ab w_ab beta_ab (Q_a Q_b - m0_ab)
    (p0 the normalised equilibrium, m0 its second moments, w = 1, 2, 1 for xx, xy, yy),
    with beta from M0 beta = (C_new - C) / ell^2, M0 = sum_q p0 QQ (w (QQ - m0))^T a
    constant, well-conditioned 3 x 3 matrix."""
    l2 = s.lat.ell ** 2
    pt = psi_q.sum(-1)
    C = l2 * np.einsum("yxq,cq->cyx", psi_q, s.qq) / pt[None]
    w = np.array([1.0, 2.0, 1.0])
    dev0 = s.qq - s.m0[:, None]                            # [3, nq]
    M0 = (s.p0[None, :] * s.qq) @ (w[:, None] * dev0).T    # [3, 3]
    beta = np.einsum("ab,byx->ayx", np.linalg.inv(M0), (C_new - C) / l2)
    shape = np.einsum("ayx,aq->yxq", beta * w[:, None, None], dev0)
    return pt[..., None] * s.p0[None, None, :] * shape


def reshape_increment(s: Setup, gs, gp, C_new):
    """Equilibrium-shaped change of the pulled polymer populations gp [ny, nx, nq, 25]
    that moves their conformation to C_new: dpsi from reshape_dpsi, carried as the
    linear quasi-equilibrium of Sec. VI-B,
    dg_i = w_i [dpsi + 3 (v_i . dpsi U + Qdot_i . dpsi (Q . grad U - kappa Q))],
    with U the mixture velocity of the reshaped state (pulled solvent gs [9, ny, nx]):
    rho U = J_S + J_P + (E + rho a) / 2, E = div Theta of C_new (dg carries no momentum
    and no mass, so J_P and rho are those of gp)."""
    psi_q = gp.sum(-1)
    if not s.lat.psi_tot > 0:                             # no polymer: nothing to reshape
        return np.zeros_like(gp)
    dpsi = reshape_dpsi(s, psi_q, C_new)                              # [ny, nx, nq]
    c25, w25, _ = O.d4q25()
    psi_tot = psi_q.sum(-1)
    rho_s = gs.sum(0)
    rho = rho_s + psi_tot
    E = elastic_force(s, psi_tot, C_new)
    jx = (gs * s.c9[:, 0, None, None]).sum(0) + (gp * c25[:, 0]).sum((-1, -2))
    jy = (gs * s.c9[:, 1, None, None]).sum(0) + (gp * c25[:, 1]).sum((-1, -2))
    U = np.stack([(jx + 0.5 * (E[0] + rho * s.arow[:, None])) / rho, (jy + 0.5 * E[1]) / rho])
    G = grad_u(U)
    qx, qy = s.qx[None, None], s.qy[None, None]
    jrx = dpsi * U[0][..., None]
    jry = dpsi * U[1][..., None]
    jqx = dpsi * (qx * G[0, 0][..., None] + qy * G[1, 0][..., None] - s.lat.kappa * qx)
    jqy = dpsi * (qx * G[0, 1][..., None] + qy * G[1, 1][..., None] - s.lat.kappa * qy)
    return w25 * (dpsi[..., None] + 3.0 * (jrx[..., None] * c25[:, 0] + jry[..., None] * c25[:, 1] +
                                           jqx[..., None] * c25[:, 2] + jqy[..., None] * c25[:, 3]))


def conformation(f):
    return np.stack([f["cxx"], f["cxy"], f["cyy"]])


# ---------------------------------------------------------------- the block
def block(s: Setup, o: O.Oracle, P, mode: str = "mlp"):
    """Advance the C-oracle state o by one block of 1 + K steps. mode: "mlp" (network,
    check and fallback), "frozen" (C_new = C(t + 1) on every tile: the plain update
    alone, the method without the network), "plain" (K more plain steps).
    Returns info (flagged tiles, indicator per tile, features)."""
    C_t = conformation(o.fields())
    o.step(1)
    f1 = o.fields()
    C1 = conformation(f1)
    if mode == "plain":
        o.step(s.K)
        return {"flagged": [], "C1": C1}
    U1 = np.stack([f1["ux"], f1["uy"]])
    psi1 = f1["psi_tot"]
    r = C1 - C_t
    C_dep = advect(s, C1, U1)
    X = features(s, U1, C_dep) if mode == "mlp" else None
    ce = s.c_e
    flagged, worst = [], {}
    if mode == "mlp":
        out = apply(P, X)
        C_new = C_dep + ce * out.T.reshape(3, s.ny, s.nx)
        e = np.abs(C_new - C1 - s.K * r).max(0) / ce
        T = s.tile
        for ty in range(0, s.ny, T):
            for tx in range(0, s.nx, T):
                worst[(tx, ty)] = float(e[ty:ty + T, tx:tx + T].max())
                if worst[(tx, ty)] > s.threshold:
                    flagged.append((tx, ty))
                    C_new[:, ty:ty + T, tx:tx + T] = C1[:, ty:ty + T, tx:tx + T]
    else:
        C_new = C1.copy()
    gs, gp = o.get_g()                                    # pulled populations at t + 1
    dP = polymer_momentum_offset(s, gs, gp, f1)
    g = np.moveaxis(gs, -1, 0).copy()
    for j in range(s.K):
        fr = j / s.K
        g = pull(s, collide(s, g, psi1, C1 + fr * (C_new - C1), dP))
    gs_k = np.ascontiguousarray(np.moveaxis(g, 0, -1))
    o.set_g(gs_k, gp + reshape_increment(s, g, gp, C_new))
    return {"flagged": flagged, "worst": worst, "X": X, "C_dep": C_dep, "C1": C1, "C_new": C_new,
            "U1": U1}


def targets(s: Setup, C_dep, C_end):
    """Training targets (C(t + 1 + K) - C_dep) / c_e, [N, 3]."""
    d = (C_end - C_dep) / s.c_e
    return np.stack([d[0].ravel(), d[1].ravel(), d[2].ravel()], axis=1)
