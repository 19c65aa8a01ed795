"""The paper's viscoelastic Kolmogorov run (Sec. VII): a 72 x 72 periodic cell with
four forcing periods, Re = 3.5, beta = 0.5, FENE dumbbells with b = 25, Wi in
{0.1, 2.5, 5}, started from rest with a seeded random perturbation, followed
to t = 2000 convective times (l / U0). Records the enstrophy and the polymer's
root-mean-square extension, the two global quantities the paper follows.

The paper reports (Sec. VII, figures without numbers): the enstrophy rises to
the laminar plateau, then drops at the onset of the inflectional instability,
early for Wi = 0.1, later and by marginally less for Wi = 2.5, never for
Wi = 5; Q_rms stays near the equilibrium extension at Wi = 0.1 and reaches about
twice it at Wi = 5.

Lattice choices (the paper gives none): U0 = 0.05; the 6 x 6 Q-grid masked to
R = 3 of the throughput workload; a momentum relaxation time tau_m that makes
sigma_Q = 2 Q-lattice units at every Wi (sigma_Q^2 = 2 lambda_H tau_m / 3), with the
momentum quasi-equilibrium where tau_m >= 3 beta nu and the stress one where it is
smaller; seed amplitude 1e-2 U0. The Schmidt number this implies, about
3 beta nu / tau_m, runs from 0.06 (Wi = 0.1) to 2.9 (Wi = 5), inside the range
0.05-4 that the paper states. A disk reaching Q0 = sqrt(b) sigma_Q, as in the
paper, is not stable with the first-order bead-force closure on this Q-lattice
(it blows up within a few hundred steps for R >= 3 sigma_Q), so the disk here
holds 1.5 sigma_Q and the FENE force is mild on it (phi <= 1.1).

    python -m paper_2201_10132_gb300.paper_run [--tmax 2000] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import tfkt
from .inputs import perturbation

N, KP, RE, BETA, U0, B = 72, 4, 3.5, 0.5, 0.05, 25.0


SIGMA2 = 4.0


def relaxation(wi: float):
    """(tau_m, qe_model): sigma_Q^2 = 2 lambda_H tau_m / 3 = SIGMA2 in the library's mapping."""
    l = N / (2 * math.pi * KP)
    tau_s = 3 * BETA * U0 * l / RE
    tau_m = 3 * SIGMA2 / (2 * wi * l / U0)
    return tau_m, (tfkt.QE_MOMENTUM if tau_m >= tau_s else tfkt.QE_STRESS)


def run(wi: float, tmax: float, every: float, seed: int = 0, amp: float = 1e-2,
        precision: int = tfkt.FP32, plain_times: bool = False):
    """plain_times: keep the momentum model with tau_m = 3 beta nu (sigma_Q then grows
    with Wi) and size the Q-grid to a disk of 1.5 sigma_Q instead."""
    l = N / (2 * math.pi * KP)
    if plain_times:
        tau_m, qe = 3 * BETA * U0 * l / RE, tfkt.QE_MOMENTUM
        s2 = 2 * (wi * l / U0) * tau_m / 3
        R = 1.5 * math.sqrt(s2)
        S = max(2, int(math.ceil(2 * R - 1e-9)))
    else:
        s2 = SIGMA2
        R, S = 3.0, 6
        tau_m, qe = relaxation(wi)
    q0 = math.sqrt(B * s2)
    p = tfkt.Params(N, N, S, R, RE, wi, BETA, U0, KP, 0.0 if plain_times else tau_m, 0.0, 0,
                    precision, B, qe)
    tconv = l / U0                          # lattice steps per convective time
    nsteps = int(round(tmax * tconv))
    chunk = max(1, int(round(every * tconv)))
    t, ens, qrms = [], [], []
    blowup = None
    with tfkt.Solver(p, perturbation(N, N, seed, amp, U0)) as s:
        info = s.get_info()
        ell = info["ell"]
        done = 0
        while done < nsteps:
            k = min(chunk, nsteps - done)
            s.step(k)
            done += k
            try:
                d = s.diagnostics()
            except tfkt.TfktError:          # non-finite state: the run ends here
                blowup = done / tconv
                break
            t.append(done / tconv)
            ens.append(d["enstrophy"])
            qrms.append(d["qrms_mean"] / ell)   # Q lattice units
    sig = math.sqrt(s2)
    return {"wi": wi, "q_radius": R, "nq": info["nq"], "sigma_q": sig, "q0": q0,
            "tau_m": tau_m, "qe_model": qe, "schmidt": 3 * BETA * U0 * l / RE / tau_m,
            "steps_per_convective_time": tconv, "blowup_time": blowup, "t": t, "enstrophy": ens,
            "qrms_over_sigma": [q / sig for q in qrms], "qrms_over_q0": [q / q0 for q in qrms]}


def summarise(r: dict) -> dict:
    t = np.array(r["t"])
    e = np.array(r["enstrophy"])
    if len(t) == 0:
        return {"wi": r["wi"], "blowup_time": r["blowup_time"]}
    plateau = float(e[t <= 40].max()) if (t <= 40).any() else float(e.max())
    below = np.nonzero((t > 10) & (e < 0.9 * plateau))[0]
    late = t >= 0.8 * t[-1]
    return {"wi": r["wi"], "plateau_enstrophy": plateau, "final_enstrophy": float(e[-1]),
            "onset_time": float(t[below[0]]) if len(below) else None,
            "qrms_over_sigma_late": float(np.mean(np.array(r["qrms_over_sigma"])[late])),
            "qrms_over_q0_late": float(np.mean(np.array(r["qrms_over_q0"])[late])),
            "nq": r["nq"], "q_radius": r["q_radius"], "q0": r["q0"], "qe_model": r["qe_model"],
            "schmidt": r["schmidt"], "blowup_time": r["blowup_time"], "t_end": float(t[-1])}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--tmax", type=float, default=2000.0)
    ap.add_argument("--every", type=float, default=5.0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--wi", type=float, nargs="*", default=[0.1, 2.5, 5.0])
    ap.add_argument("--plain-times", action="store_true",
                    help="tau_m = 3 beta nu and a 1.5 sigma_Q disk instead of sigma_Q = 2")
    args = ap.parse_args(argv)
    res = {}
    for wi in args.wi:
        t0 = time.time()
        r = run(wi, args.tmax, args.every, precision=tfkt.FP64 if args.fp64 else tfkt.FP32,
                plain_times=args.plain_times)
        res[str(wi)] = r
        print(json.dumps({"summary": summarise(r), "seconds": round(time.time() - t0, 1)}),
              flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    main()
