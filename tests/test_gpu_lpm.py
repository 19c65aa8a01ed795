"""GPU parity of the learned macro-step against its FP64 oracle (oracle/lpm_oracle.py).

The network's forward pass, loss, gradient and Adam step run in FP32 with
bfloat16 matrices; the oracle runs in FP64 with the same bfloat16-rounded
matrices. FP32 accumulation over 40 and 64 terms and over the batch leaves
relative errors of order 1e-6 per output; the tolerances below allow 1e-4 of
each tensor's largest magnitude. The learned block is compared field by field
after whole blocks on grids of several 32 x 8 tiles, with the block's own FP32
arithmetic (each sub-step re-rounds the state) against FP64: 1e-4 of the
velocity scale for U and of C's largest magnitude for C.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    assert torch.cuda.is_available()
    from paper_2201_10132_gb300 import build, tfkt
    build.build()
    return tfkt


@pytest.fixture(scope="module")
def L(oracle_mod):
    from oracle import lpm_oracle
    return lpm_oracle


def _random_net(L, T, seed, out_scale=1.0):
    """A seeded network with non-trivial input and output standardisation."""
    rng = np.random.default_rng(seed)
    P = L.init_params(seed)
    P["W3"] = P["W3"] * 10 * out_scale
    P["b1"] = rng.normal(0, 0.1, 64).astype(np.float32).astype(np.float64)
    P["b2"] = rng.normal(0, 0.1, 64).astype(np.float32).astype(np.float64)
    P["b3"] = rng.normal(0, 0.1, 3).astype(np.float32).astype(np.float64)
    norm = {"mx": rng.normal(0, 0.1, 40), "sx": rng.uniform(0.5, 2.0, 40),
            "mt": rng.normal(0, 0.01, 3), "st": rng.uniform(0.01, 0.05, 3)}
    norm = {k: v.astype(np.float32).astype(np.float64) for k, v in norm.items()}
    vec = T.pack_mlp(P["W1"], P["b1"], P["W2"], P["b2"], P["W3"], P["b3"], norm["mx"], norm["sx"],
                     norm["mt"], norm["st"])
    net = dict(L.compute_weights(P), **norm)
    return vec, P, net


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def test_forward_matches_oracle(T, L):
    import torch
    vec, _, net = _random_net(L, T, 1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1.5, (1000, 40)).astype(np.float32)
    Y = torch.zeros((1000, 3), dtype=torch.float32, device="cuda")
    m = T.Mlp(vec)
    Xd = _dev(X)
    m.forward(Xd.data_ptr(), 1000, Y.data_ptr())
    torch.cuda.synchronize()
    ref = L.apply(net, X.astype(np.float64))
    err = np.abs(Y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-4, err
    m.close()


@pytest.mark.parametrize("n", [1000, 128, 1])
def test_loss_and_gradient_match_oracle(T, L, n):
    """n = 1000 spans seven full blocks of 128 samples and a ragged one."""
    import torch
    vec, P, net = _random_net(L, T, 3)
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1.5, (n, 40)).astype(np.float32)
    Tg = rng.normal(0, 0.03, (n, 3)).astype(np.float32)
    m = T.Mlp(vec)
    g = torch.zeros(T.MLP_NWEIGHTS, dtype=torch.float32, device="cuda")
    Xd, Td = _dev(X), _dev(Tg)
    loss = m.loss_grad(Xd.data_ptr(), Td.data_ptr(), n, g.data_ptr())
    xn = (X.astype(np.float64) - net["mx"]) / net["sx"]
    tn = (Tg.astype(np.float64) - net["mt"]) / net["st"]
    ref_loss, ref_g = L.loss_and_grads(net, xn, tn)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    gd = T.unpack_mlp(np.concatenate([g.cpu().numpy(), np.zeros(86, np.float32)]))
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.abs(gd[k] - ref_g[k]).max() / np.abs(ref_g[k]).max()
        assert err < 1e-4, (k, err)
    m.close()


def test_adam_step_matches_oracle(T, L):
    import torch
    vec, P, net = _random_net(L, T, 5)
    rng = np.random.default_rng(6)
    X = rng.normal(0, 1.5, (512, 40)).astype(np.float32)
    Tg = rng.normal(0, 0.03, (512, 3)).astype(np.float32)
    m = T.Mlp(vec)
    Xd, Td = _dev(X), _dev(Tg)
    lr = 1e-3
    for _ in range(3):
        m.loss_grad(Xd.data_ptr(), Td.data_ptr(), 512)
        m.adam(lr)
    got = T.unpack_mlp(m.get())
    master = {k: P[k].copy() for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    st = {}
    xn = (X.astype(np.float64) - net["mx"]) / net["sx"]
    tn = (Tg.astype(np.float64) - net["mt"]) / net["st"]
    for _ in range(3):
        w = dict(L.compute_weights(master))
        _, g = L.loss_and_grads(w, xn, tn)
        L.adam(master, g, st, lr)
    for k in master:
        # Adam's steps are ~lr in size whatever the gradient: compare against lr
        assert np.abs(got[k] - master[k]).max() < 0.05 * lr, k
    m.close()


def _pair(T, O, L, nx, ny, wi, steps0, seed, K=4, tile=16, threshold=1e9):
    from paper_2201_10132_gb300.inputs import perturbation
    pert = perturbation(nx, ny, seed, 0.3, 0.05)
    lat = O.map_params(nx, ny, 6, 3.0, 10.0, wi, 0.2, 0.05, 1)
    o = O.Oracle(lat)
    o.init(pert, 1)
    o.step(steps0)
    p = T.Params(nx, ny, 6, 3.0, 10.0, wi, 0.2, 0.05, 1, 0.0, 0.0, 1, T.FP32)
    s = T.Solver(p, pert)
    s.step(steps0)
    setup = L.Setup(lat, K=K, tile=tile, threshold=threshold)
    return o, s, setup


def test_network_wait_timeout_is_reported_and_leaves_a_valid_block(T, L):
    """The network kernel bounds its waits for the tensor cores. With the fault
    injection it issues no tensor-core work, so every wait runs out after a few
    polls: tfkt_lpm_run returns TFKT_ETIMEOUT, every tile has fallen back to the
    plain step's conformation (the state is then bit-identical to a block without
    the network), and the context stays usable."""
    from paper_2201_10132_gb300.inputs import perturbation
    vec, _, _ = _random_net(L, T, 7, out_scale=0.2)
    pert = perturbation(64, 32, 3, 0.3, 0.05)
    p = T.Params(64, 32, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1, 0.0, 0.0, 1, T.FP32)
    m = T.Mlp(vec)
    with T.Solver(p, pert) as a, T.Solver(p, pert) as b:
        a.step(5)
        b.step(5)
        with pytest.raises(T.TfktError) as e:
            T.lpm_run(a, m, 1, K=4, tile=16, threshold=1e9, inject_wait_timeout=True)
        assert e.value.status == T.ETIMEOUT
        assert T.lpm_run(b, None, 1, K=4, tile=16, threshold=1e9, mode=T.LPM_FROZEN) == 0
        assert a.get_info()["step"] == b.get_info()["step"] == 5 + 5
        fa, fb = a.moments(), b.moments()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
        # the context is not poisoned: a normal block and plain steps follow
        assert T.lpm_run(a, m, 1, K=4, tile=16, threshold=1e9) == 0
        a.step(2)
        d = a.diagnostics()
        assert all(np.isfinite(v) for v in d.values())
    m.close()


def _compare(o, s, L):
    f = o.fields()
    g = s.moments()
    uscale = max(np.abs(f["ux"]).max(), np.abs(f["uy"]).max())
    err_u = max(np.abs(g[k] - f[k]).max() for k in ("ux", "uy")) / uscale
    cs = max(np.abs(f[k]).max() for k in ("cxx", "cxy", "cyy"))
    err_c = max(np.abs(g[k] - f[k]).max() for k in ("cxx", "cxy", "cyy")) / cs
    err_p = np.abs(g["psi_tot"] - f["psi_tot"]).max() / np.abs(f["psi_tot"]).max()
    return err_u, err_c, err_p


@pytest.mark.parametrize("mode", ["mlp", "frozen", "fallback"])
def test_block_matches_oracle(T, L, oracle_mod, mode):
    O = oracle_mod
    vec, _, net = _random_net(L, T, 7, out_scale=0.2)
    thr = 0.0 if mode == "fallback" else 1e9
    o, s, setup = _pair(T, O, L, 64, 32, 1.0, 40, 3, K=4, tile=16, threshold=thr)
    m = T.Mlp(vec)
    flagged = T.lpm_run(s, m if mode != "frozen" else None, 2, K=4, tile=16, threshold=thr,
                        mode=T.LPM_FROZEN if mode == "frozen" else T.LPM_NET)
    nfl = 0
    for _ in range(2):
        info = L.block(setup, o, net, "frozen" if mode == "frozen" else "mlp")
        nfl += len(info["flagged"])
    assert flagged == nfl == (2 * 8 if mode == "fallback" else 0)
    assert s.get_info()["step"] == 40 + 2 * 5
    err_u, err_c, err_p = _compare(o, s, L)
    assert err_u < 1e-4 and err_c < 1e-4 and err_p < 1e-5, (err_u, err_c, err_p)
    # a plain step after the blocks: the increments reached the populations
    o.step(1)
    s.step(1)
    err_u, err_c, err_p = _compare(o, s, L)
    assert err_u < 1e-4 and err_c < 1e-4 and err_p < 1e-5, (err_u, err_c, err_p)
    s.close()
    m.close()


def test_features_and_targets_match_oracle(T, L, oracle_mod):
    import torch
    O = oracle_mod
    o, s, setup = _pair(T, O, L, 64, 32, 0.5, 30, 5, K=4)
    N = 64 * 32
    X = torch.zeros((N, 40), dtype=torch.float32, device="cuda")
    Cd = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    Tt = torch.zeros((N, 3), dtype=torch.float32, device="cuda")
    T.lpm_features(s, 4, X.data_ptr(), Cd.data_ptr())
    f = o.fields()
    U = np.stack([f["ux"], f["uy"]])
    Cdep = L.advect(setup, L.conformation(f), U)
    Xr = L.features(setup, U, Cdep)
    Xg = X.cpu().numpy()
    for cols in (slice(0, 3), slice(3, 39), slice(39, 40)):
        scale = np.abs(Xr[:, cols]).max()
        assert np.abs(Xg[:, cols] - Xr[:, cols]).max() < 1e-4 * scale, cols
    o.step(4)
    s.step(4)
    T.lpm_targets(s, Cd.data_ptr(), Tt.data_ptr())
    Tr = L.targets(setup, Cdep, L.conformation(o.fields()))
    assert np.abs(Tt.cpu().numpy() - Tr).max() < 1e-3 * np.abs(Tr).max()
    s.close()


@pytest.mark.parametrize("kw,K", [(dict(precision=0), 4), (dict(), 3), (dict(fene_b=25.0), 4),
                                  (dict(nx=40), 4)])
def test_rejects_unsupported(T, kw, K):
    args = dict(nx=64, ny=32, q_side=6, q_radius=3.0, re=10.0, wi=1.0, beta=0.2, ic_mode=1,
                precision=T.FP32)
    args.update(kw)
    with T.Solver(T.Params(**args)) as s:
        with pytest.raises(T.TfktError) as e:
            T.lpm_run(s, None, 1, K=K, mode=T.LPM_FROZEN)
        assert e.value.status == 1


def test_trained_network_gains_over_the_block_without_it(T):
    """The committed network against the same block without it (every tile keeping
    the plain step's conformation), both against the plain solver, on a flow it was
    not trained on (256^2, seed 123, laminar start with a 5% perturbation)."""
    from paper_2201_10132_gb300 import train_lpm
    from paper_2201_10132_gb300.inputs import Workload, perturbation
    params, meta = train_lpm.load()
    K, thr = meta["K"], meta["threshold"]
    w = Workload("gain-256", 256, 256, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 4, 123, 0.05, ic_mode=1)
    p = T.Params.from_workload(w, T.FP32)
    pert = perturbation(w.nx, w.ny, w.seed, w.amp, w.u0)
    net = T.Mlp(params)
    sols = {m: T.Solver(p, pert) for m in ("plain", "net", "frozen")}
    ey2 = {m: [] for m in sols}
    fl = 0
    nblk = 40
    for s in sols.values():
        s.step(600)
    for _ in range(nblk):
        sols["plain"].step(1 + K)
        fl += T.lpm_run(sols["net"], net, 1, K=K, tile=32, threshold=thr)
        T.lpm_run(sols["frozen"], None, 1, K=K, tile=32, threshold=thr, mode=T.LPM_FROZEN)
        for m, s in sols.items():
            ey2[m].append(s.diagnostics()["ey2"])
    f = {m: s.moments(["ux", "uy", "cxx", "cxy", "cyy"]) for m, s in sols.items()}
    us = max(np.abs(f["plain"][k]).max() for k in ("ux", "uy"))
    cs = max(np.abs(f["plain"][k]).max() for k in ("cxx", "cxy", "cyy"))
    t = np.arange(1, nblk + 1) * (1 + K)
    rate = {m: np.polyfit(t[nblk // 2:], np.log(ey2[m][nblk // 2:]), 1)[0] for m in sols}
    err = {}
    for m in ("net", "frozen"):
        err[m] = (max(np.abs(f[m][k] - f["plain"][k]).max() for k in ("ux", "uy")) / us,
                  max(np.abs(f[m][k] - f["plain"][k]).max() for k in ("cxx", "cxy", "cyy")) / cs,
                  abs(rate[m] / rate["plain"] - 1))
    assert fl == 0
    assert err["net"][0] < 0.5 * err["frozen"][0], err       # velocity
    assert err["net"][1] < 0.25 * err["frozen"][1], err      # conformation
    assert err["net"][2] < 0.02 and err["net"][2] < err["frozen"][2], err   # growth rate
    for s in sols.values():
        s.close()
    net.close()


def test_pending_increment_flush_equals_fused_pull(T, L, oracle_mod):
    """A block leaves its increment to the next step's pull; reading the populations
    in between adds it to the stored populations instead. Both orders give the same
    next state."""
    O = oracle_mod
    vec, _, _ = _random_net(L, T, 9, out_scale=0.2)
    m = T.Mlp(vec)
    out = []
    for flush in (False, True):
        o, s, _ = _pair(T, O, L, 64, 32, 1.0, 40, 3, K=4, tile=16)
        T.lpm_run(s, m, 2, K=4, tile=16, threshold=1e9)
        if flush:
            s.populations()
        s.step(2)
        out.append(s.moments(["ux", "uy", "cxx", "cxy", "cyy", "psi_tot"]))
        s.close()
    for k in out[0]:
        scale = np.abs(out[0][k]).max()
        assert np.abs(out[0][k] - out[1][k]).max() <= 1e-5 * scale, k
    m.close()


def test_paper_run_low_weissenberg(T):
    """The paper's 72^2 run at Wi = 0.1 (Sec. VII): the inflectional instability lowers
    the enstrophy from its laminar plateau early on, and the polymer stays at its
    equilibrium extension, Q_rms ~ 0.2 of the maximum extension sqrt(b)."""
    from paper_2201_10132_gb300 import paper_run
    r = paper_run.run(0.1, 150.0, 5.0)
    s = paper_run.summarise(r)
    assert r["blowup_time"] is None
    assert s["onset_time"] is not None and 20 < s["onset_time"] < 120, s
    assert 0.15 < s["qrms_over_q0_late"] < 0.25, s
