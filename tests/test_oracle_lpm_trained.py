"""The committed network in the FP64 oracle of the learned block (CPU): it reproduces
the plain scheme better than the same block without it, on a 64^2 flow with the
training flows' local resolution (forcing wavelength 64 nodes)."""
import json

import numpy as np
import pytest


def _net(L):
    from paper_2201_10132_gb300 import train_lpm, tfkt
    params, meta = train_lpm.load()
    d = tfkt.unpack_mlp(params)
    P = {k: d[k].astype(np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    net = dict(L.compute_weights(P))
    net.update({k: d[k].astype(np.float64) for k in ("mx", "sx", "mt", "st")})
    return net, meta


def test_weights_file_is_consistent():
    from paper_2201_10132_gb300 import train_lpm, tfkt
    params, meta = train_lpm.load()
    assert params.shape == (tfkt.MLP_NPARAM,) and np.isfinite(params).all()
    d = tfkt.unpack_mlp(params)
    assert (d["sx"] > 0).all() and (d["st"] > 0).all()
    assert meta["K"] % 2 == 0 and meta["threshold"] > 0 and meta["pairs"] > 10 ** 6
    assert meta["loss_history"][-1][2] < 0.1        # validation loss, standardised


def test_trained_network_gains_in_the_oracle(oracle_mod):
    from oracle import lpm_oracle as L
    from paper_2201_10132_gb300.inputs import perturbation
    O = oracle_mod
    net, meta = _net(L)
    K = meta["K"]
    nx = ny = 64
    lat = O.map_params(nx, ny, 6, 3.0, 10.0, 1.0, 0.2, 0.05, 1)
    base = O.Oracle(lat)
    base.init(perturbation(nx, ny, 31, 0.05, 0.05), 1)
    base.step(300)
    s = L.Setup(lat, K=K, tile=32, threshold=meta["threshold"])
    runs = {m: O.Oracle(lat) for m in ("plain", "mlp", "frozen")}
    for o in runs.values():
        o.set_g(*base.get_g())
    flagged = 0
    for _ in range(12):
        for m, o in runs.items():
            info = L.block(s, o, net, m)
            flagged += len(info["flagged"])
    f = {m: o.fields() for m, o in runs.items()}
    cs = max(np.abs(f["plain"][k]).max() for k in ("cxx", "cxy", "cyy"))
    us = max(np.abs(f["plain"][k]).max() for k in ("ux", "uy"))
    ec = {m: max(np.abs(f[m][k] - f["plain"][k]).max() for k in ("cxx", "cxy", "cyy")) / cs
          for m in ("mlp", "frozen")}
    eu = {m: max(np.abs(f[m][k] - f["plain"][k]).max() for k in ("ux", "uy")) / us
          for m in ("mlp", "frozen")}
    assert flagged == 0
    assert ec["mlp"] < 0.25 * ec["frozen"], ec
    assert eu["mlp"] < 0.5 * eu["frozen"], eu
