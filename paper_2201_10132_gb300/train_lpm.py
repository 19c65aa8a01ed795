"""Train the learned macro-step's network on trajectories of the plain solver.

Everything numerical runs in the library's kernels: the plain step generates
the trajectories, tfkt_lpm_features / tfkt_lpm_targets extract the training
pairs, tfkt_mlp_loss_grad / tfkt_mlp_adam train the network. PyTorch only
holds device memory and gathers the sampled rows; numpy shuffles and computes
the standardisation on the host.

Trajectories: 1024^2 Kolmogorov flows with the local resolution of the 4096^2
workload (forcing wavelength 64 nodes, 6 x 6 Q-grid masked to R = 3), Re = 10,
beta = 0.2, Wi in {0.5, 1, 2}, from rest and from the laminar profile, with
small and moderate seeded perturbations; a pair (features at t, conformation
at t + K) every `every` steps, 1/32 of the nodes per snapshot.

    python -m paper_2201_10132_gb300.train_lpm [--out PATH] [--steps N]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import tfkt
from .inputs import Workload, perturbation

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "weights", "lpm_re10_beta0.2_nq32.npz")


def training_runs(side: int = 1024):
    runs = []
    for wi in (0.5, 1.0, 2.0):
        for ic, amp in ((0, 1e-3), (1, 0.1), (0, 0.1)):
            runs.append(Workload(f"train-wi{wi}-ic{ic}-amp{amp}", side, side, 6, 3.0, 10.0, wi, 0.2,
                                 0.05, side // 64, int(wi * 100) + 10 * ic + (amp > 0.01), amp,
                                 ic_mode=ic))
    return runs


def collect(runs, K: int, nsteps: int, every: int, keep: int, seed: int):
    """Training pairs (X [n, 40], T [n, 3]) on the host."""
    import torch
    rng = np.random.default_rng(seed)
    Xs, Ts = [], []
    for w in runs:
        p = tfkt.Params.from_workload(w, tfkt.FP32)
        pert = perturbation(w.nx, w.ny, w.seed, w.amp, w.u0)
        N = w.nx * w.ny
        X = torch.empty((N, tfkt.MLP_IN), dtype=torch.float32, device="cuda")
        Cd = torch.empty((N, 3), dtype=torch.float32, device="cuda")
        T = torch.empty((N, 3), dtype=torch.float32, device="cuda")
        t0 = time.time()
        with tfkt.Solver(p, pert) as s:
            t = 0
            while t + every <= nsteps:
                s.step(every - K)
                t += every - K
                tfkt.lpm_features(s, K, X.data_ptr(), Cd.data_ptr())
                s.step(K)
                t += K
                tfkt.lpm_targets(s, Cd.data_ptr(), T.data_ptr())
                idx = torch.as_tensor(rng.choice(N, N // keep, replace=False), device="cuda")
                Xs.append(X.index_select(0, idx).cpu().numpy())
                Ts.append(T.index_select(0, idx).cpu().numpy())
        print(f"  {w.name}: {t} steps, {len(Xs)} snapshots so far, {time.time() - t0:.1f} s",
              flush=True)
    return np.concatenate(Xs), np.concatenate(Ts)


def train(X, T, seed: int, epochs: int, batch: int, lr: float, log=print):
    """Adam on standardised data; returns the packed parameters and the losses."""
    import torch
    rng = np.random.default_rng(seed)
    mx, sx = X.mean(0), X.std(0)
    sx = np.where(sx > 1e-12, sx, 1.0)            # constant inputs (K / lambda_H of one run)
    mt, st = T.mean(0), T.std(0)
    st = np.where(st > 1e-12, st, 1.0)
    perm = rng.permutation(len(X))
    nval = max(len(X) // 20, 1)
    val, tr = perm[:nval], perm[nval:]
    Xtr = torch.as_tensor(np.ascontiguousarray(X[tr]), device="cuda")
    Ttr = torch.as_tensor(np.ascontiguousarray(T[tr]), device="cuda")
    Xva = torch.as_tensor(np.ascontiguousarray(X[val]), device="cuda")
    Tva = torch.as_tensor(np.ascontiguousarray(T[val]), device="cuda")
    # Glorot-uniform weights, zero biases, the output layer scaled by 0.1
    def glorot(o, i, s=1.0):
        lim = s * np.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, (o, i))
    H, I, O = tfkt.MLP_HID, tfkt.MLP_IN, tfkt.MLP_OUT
    vec = tfkt.pack_mlp(glorot(H, I), np.zeros(H), glorot(H, H), np.zeros(H), glorot(O, H, 0.1),
                        np.zeros(O), mx, sx, mt, st)
    net = tfkt.Mlp(vec)
    ntr = len(tr)
    nb = ntr // batch
    hist = []
    step = 0
    total = epochs * nb
    for ep in range(epochs):
        order = rng.permutation(nb)
        for b in order:
            lr_now = lr if step < 0.6 * total else (lr * 0.25 if step < 0.85 * total else lr * 0.05)
            net.loss_grad(Xtr[b * batch:].data_ptr(), Ttr[b * batch:].data_ptr(), batch)
            net.adam(lr_now)
            step += 1
        lv = net.loss_grad(Xva.data_ptr(), Tva.data_ptr(), len(val))
        lt = net.loss_grad(Xtr.data_ptr(), Ttr.data_ptr(), min(ntr, 1 << 20))
        hist.append((ep, lt, lv))
        log(f"  epoch {ep}: train loss {lt:.5f}, validation loss {lv:.5f} (standardised, 3 outputs)")
    out = net.get()
    net.close()
    return out, hist


def calibrate(params, K: int, side: int, tile: int, warm: int, blocks: int, fraction: float,
              log=print):
    """Smallest threshold (of a geometric ladder) at which at most `fraction` of the
    tiles fall back on a held-out run, times 4: a tile falls back only when the
    network disagrees with the plain rate well beyond what it does on flows like
    the ones it was trained on."""
    w = Workload("calibrate", side, side, 6, 3.0, 10.0, 1.0, 0.2, 0.05, side // 64, 97, 0.05,
                 ic_mode=1)
    p = tfkt.Params.from_workload(w, tfkt.FP32)
    pert = perturbation(w.nx, w.ny, w.seed, w.amp, w.u0)
    net = tfkt.Mlp(params)
    ntiles = (side // tile) ** 2 * blocks
    chosen = None
    for thr in (1e-4, 2e-4, 5e-4, 1e-3, 2e-3, 5e-3, 0.01, 0.02, 0.05, 0.1, 0.2, 0.5, 1.0):
        with tfkt.Solver(p, pert) as s:
            s.step(warm)
            fl = tfkt.lpm_run(s, net, blocks, K=K, tile=tile, threshold=thr)
        log(f"  threshold {thr}: {fl} of {ntiles} tiles fell back")
        if fl <= fraction * ntiles:
            chosen = 4.0 * thr
            break
    net.close()
    return chosen if chosen is not None else 2.0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--side", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=4800)
    ap.add_argument("--every", type=int, default=240)
    ap.add_argument("--keep", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    t0 = time.time()
    runs = training_runs(args.side)
    print(f"collecting pairs from {len(runs)} plain runs", flush=True)
    X, T = collect(runs, args.K, args.steps, args.every, args.keep, args.seed)
    print(f"{len(X)} pairs, {time.time() - t0:.0f} s", flush=True)
    params, hist = train(X, T, args.seed, args.epochs, args.batch, args.lr)
    print(f"trained, {time.time() - t0:.0f} s", flush=True)
    thr = calibrate(params, args.K, 256, 32, 600, 20, 0.005)
    meta = {"K": args.K, "threshold": thr, "pairs": int(len(X)), "loss_history": hist,
            "runs": [w.as_dict() for w in runs], "steps_per_run": args.steps,
            "every": args.every, "keep_one_in": args.keep, "epochs": args.epochs,
            "batch": args.batch, "lr": args.lr, "seed": args.seed}
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.savez(args.out, params=params, meta=json.dumps(meta))
    print(f"saved {args.out} (threshold {thr}), {time.time() - t0:.0f} s", flush=True)


def load(path: str = DEFAULT_OUT):
    """(packed parameters, metadata) of a trained network."""
    d = np.load(path)
    return d["params"].astype(np.float32), json.loads(str(d["meta"]))


if __name__ == "__main__":
    main()
