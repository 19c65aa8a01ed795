"""Throughput of the two-fluid kinetic step (GLUPS = 1e9 r-node updates / s).

Workload: Kolmogorov flow on 4096 x 4096 r-nodes, N_Q = 32 Q-nodes (6 x 6 grid
masked to R = 3), Re 10, Wi 1, beta 0.2, forcing wavelength 64 nodes, FP32
storage; synthetic seeded perturbation. One step = pull-stream, moments,
collision and write-back of all 9 + 25 N_Q populations of every node.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank advances its own independent run (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129e6


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per r-node of one
# fused-kernel launch, from the ncu capture of the 512^2 case of the same lattice
# parameters (profiles/step_fused_kernel_kolmogorov_512x512_nq32*.md; traffic grows
# in proportion to the node count), with the sha256 prefix of the kernel sources
# the capture was taken on.
FUSED_TRAFFIC = {
    "fp32": (6657.4, "0574d80a66975595"),
    "fp16": (3480.5, "0574d80a66975595"),
}
KERNEL_SOURCES = ("paper_2201_10132_gb300/csrc/tfkt_fused.cu",
                  "paper_2201_10132_gb300/csrc/tfkt_fused.cuh")


def kernel_source_sha() -> str:
    """sha256 prefix (16 hex digits) of the fused kernel's sources, in order."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def fused_traffic(nodes: int, storage: str = "fp32"):
    """DRAM bytes of one fused-kernel launch over `nodes` r-nodes, scaled from the
    512^2 capture; None for a storage without a capture, or once the kernel sources
    differ from those the counters were taken on."""
    if storage not in FUSED_TRAFFIC:
        return None
    per_node, sha = FUSED_TRAFFIC[storage]
    try:
        if kernel_source_sha() != sha:
            return None
    except OSError:
        return None
    return per_node * nodes


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="tfkt_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


def max_over_ranks(x: float, dist=None, device: str = "cuda") -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank advances its own independent run (weak scaling): its own seed."""
    return base_seed + rank


def aggregate_glups(world: int, nodes: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: r-node updates of all ranks over the slowest rank's time."""
    return world * nodes * steps / seconds / 1e9


def host_cpu() -> str:
    """The host CPU's model name (x86 'model name'; Arm implementer and part numbers)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model"):
        for line in info.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = (t.strip() for t in line.split(":", 1))
            fields.setdefault(k, v)
    return f"implementer {fields.get('CPU implementer', '?')} part {fields.get('CPU part', '?')}"


def oracle_sample(W, target_s: float = 12.0, threads: int | None = None):
    """Time the CPU oracle on a bounded sample of the workload: 256 x 256 r-nodes
    with the same lattice parameters (forcing wavelength 64 nodes), N_Q = 32, on
    all host cores (or `threads`)."""
    from oracle import oracle as O
    from paper_2201_10132_gb300.inputs import perturbation
    n = 256
    kp = W.k_periods * n // W.ny
    cores = O.set_threads(threads or os.cpu_count() or 1)
    lat = O.map_params(n, n, W.q_side, W.q_radius, W.re, W.wi, W.beta, W.u0, kp, W.tau2)
    o = O.Oracle(lat)
    o.init(perturbation(n, n, W.seed, W.amp, W.u0), W.ic_mode)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    steps = max(1, int(target_s / max(t1 - t0, 1e-6)))
    t1 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t1
    return {"value": n * n * steps / dt / 1e9, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n}x{n} r-nodes, N_Q={o.nq}, {steps} steps, FP64, same lattice "
                      f"parameters as the workload, {dt:.1f} s"}


def run_reference(args, W):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    total_nodes = 0
    from oracle import oracle as O  # noqa: F401  (the oracle is the reference arm)
    for k in range(args.warmup + args.steps):
        r = oracle_sample(W, target_s=max(2.0, 60.0 / max(1, args.steps + args.warmup)))
        if k >= args.warmup:
            per_step.append(r)
    value = sum(r["value"] for r in per_step) / len(per_step)
    line = {"impl": "reference", "metric": "GLUPS (1e9 r-node updates/s), 4096^2 two-fluid step",
            "value": value, "unit": "GLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W.name, "sample": per_step[-1]["sample"]},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": per_step[-1]["cores"],
                             "kind": "oracle", "sample": per_step[-1]["sample"],
                             "host": {"cpu": host_cpu(), "nproc": os.cpu_count()}},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def precision_sweep(W, steps: int):
    """FP64 vs FP32 vs FP16 storage from the identical seeded state: per-field relative
    L2 / Linf errors against the FP64 run after `steps` steps, the growth rate of
    sum U_y^2 (the instability indicator) over the run, and the fused-kernel time."""
    import numpy as np
    import torch
    from paper_2201_10132_gb300 import tfkt
    from paper_2201_10132_gb300.inputs import perturbation
    pert = perturbation(W.nx, W.ny, W.seed, W.amp, W.u0)
    names = ["ux", "uy", "rho_s", "cxy", "thxy"]
    out, ref = {}, None
    for label, prec in (("fp64", tfkt.FP64), ("fp32", tfkt.FP32), ("fp16", tfkt.FP16)):
        p = tfkt.Params.from_workload(W, prec)
        ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
        s = tfkt.Solver(p, pert, workspace=ws)
        e0 = s.diagnostics()["ey2"]
        kms = np.zeros(len(tfkt.KERNELS))
        n = np.zeros(len(tfkt.KERNELS), np.int64)
        s.step_profiled(steps, kms, n)
        e1 = s.diagnostics()["ey2"]
        f = s.moments(names)
        s.close()
        del s, ws
        torch.cuda.empty_cache()
        k = tfkt.KERNELS.index("fused")
        r = {"fused_ms": kms[k] / max(n[k], 1), "ey2_rate": math.log(e1 / e0) / steps}
        if ref is None:
            ref = f
        else:
            uscale = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
            for name in names:
                d = f[name] - ref[name]
                scale = uscale if name in ("ux", "uy") else np.abs(ref[name]).max()
                r[name + "_linf"] = float(np.abs(d).max() / scale)
                r[name + "_l2"] = float(np.sqrt(np.mean(d * d)) /
                                        max(np.sqrt(np.mean(ref[name] ** 2)), 1e-300))
            r["ey2_rate_rel_err"] = abs(r["ey2_rate"] - out["fp64"]["ey2_rate"]) / max(
                abs(out["fp64"]["ey2_rate"]), 1e-300)
        out[label] = r
    for label in ("fp32", "fp16"):
        out[label]["speedup_vs_fp32"] = out["fp32"]["fused_ms"] / out[label]["fused_ms"]
    return out


def capacity_run(steps: int, warmup: int):
    """The largest run that one GPU holds: 8192^2 r-nodes, N_Q = 32, with FP16 polymer
    storage (FP32 solvent); FP32 storage would need more memory than the GPU has. Time
    per step, GLUPS, the fused kernel's algorithmic bandwidth, and mass conservation
    over the timed steps. Skipped (with the sizes) when the workspace does not fit."""
    import numpy as np
    import torch
    from paper_2201_10132_gb300 import tfkt
    from paper_2201_10132_gb300.inputs import KOLMOGOROV_8192 as W, perturbation
    p = tfkt.Params.from_workload(W, tfkt.FP16)
    need16 = tfkt.required_bytes(p)
    need32 = tfkt.required_bytes(tfkt.Params.from_workload(W, tfkt.FP32))
    free, total = torch.cuda.mem_get_info()
    out = {"workload": W.name, "storage": "fp16 polymer (scaled deviations), fp32 solvent",
           "workspace_gb": need16 / 1e9, "fp32_workspace_gb": need32 / 1e9,
           "device_total_gb": total / 1e9, "device_free_gb": free / 1e9}
    if need16 > 0.97 * free:
        out["skipped"] = "workspace does not fit the free device memory"
        return out
    ws = torch.empty(need16, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    with tfkt.Solver(p, perturbation(W.nx, W.ny, W.seed, W.amp, W.u0), workspace=ws,
                     stream=stream.cuda_stream) as s:
        s.step(warmup)
        d0 = s.diagnostics()
        kms = np.zeros(len(tfkt.KERNELS))
        n = np.zeros(len(tfkt.KERNELS), np.int64)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step_profiled(steps, kms, n)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        d1 = s.diagnostics()
        info = s.info
    k = tfkt.KERNELS.index("fused")
    fused_ms = kms[k] / max(n[k], 1)
    nodes = W.nx * W.ny
    peak, kind = _peaks()
    gbs = info["bytes_per_node_step"] * nodes / (fused_ms / 1e3) / 1e9
    m0, m1 = d0["mass_s"] + d0["mass_p"], d1["mass_s"] + d1["mass_p"]
    out.update({"steps": steps, "ms_per_step": ms, "value": aggregate_glups(1, nodes, steps, ms * steps / 1e3),
                "unit": "GLUPS", "fused_ms": fused_ms, "fused_algorithmic_gbs": gbs,
                "fused_frac_of_hbm": gbs / peak, "peak_kind": kind,
                "bytes_per_node_step": info["bytes_per_node_step"],
                "mass_rel_drift": abs(m1 - m0) / m0, "umax": d1["umax"]})
    return out


def learned_vs_plain(W, nblocks: int, warm: int, only: bool = False):
    """The learned macro-step (1 plain step + K solvent sub-steps per block, the
    committed network) against the plain FP32 step and the FP64 step on the same
    seeded workload: time per block against 1 + K plain steps, per-field errors
    against the plain FP32 run after the blocks, and the growth rate of sum U_y^2
    over the blocks against the FP64 run. The block without the network (every tile
    keeping the plain step's conformation) is reported beside it."""
    import numpy as np
    import torch
    from paper_2201_10132_gb300 import tfkt, train_lpm
    from paper_2201_10132_gb300.inputs import perturbation
    params, meta = train_lpm.load()
    K, thr = meta["K"], meta["threshold"]
    pert = perturbation(W.nx, W.ny, W.seed, W.amp, W.u0)
    names = ["ux", "uy", "cxx", "cxy", "cyy"]
    net = tfkt.Mlp(params)
    res, fields = {}, {}
    for label in (("net",) if only else ("fp64", "fp32", "net", "frozen")):
        p = tfkt.Params.from_workload(W, tfkt.FP64 if label == "fp64" else tfkt.FP32)
        ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
        st = torch.cuda.Stream()
        s = tfkt.Solver(p, pert, workspace=ws, stream=st.cuda_stream)
        s.step(warm)
        ey2, ms, fl = [], 0.0, 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for b in range(nblocks):
            s.sync()
            e0.record(st)
            if label in ("fp64", "fp32"):
                s.step(1 + K)
            elif label == "net":
                fl += tfkt.lpm_run(s, net, 1, K=K, tile=32, threshold=thr)
            else:
                tfkt.lpm_run(s, None, 1, K=K, tile=32, threshold=thr, mode=tfkt.LPM_FROZEN)
            e1.record(st)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            ey2.append(s.diagnostics()["ey2"])
        if label != "fp64":
            fields[label] = s.moments(names)
        s.close()
        del s, ws
        torch.cuda.empty_cache()
        t = np.arange(1, nblocks + 1) * (1 + K)
        h = nblocks // 2
        res[label] = {"ms_per_block": ms / nblocks, "fallback_tiles": fl,
                      "glups_equivalent": W.nx * W.ny * (1 + K) / (ms / nblocks / 1e3) / 1e9,
                      "ey2_rate": float(np.polyfit(t[h:], np.log(ey2[h:]), 1)[0])}
    net.close()
    if only:
        return {"K": K, "threshold": thr, "blocks": nblocks, "warm_plain_steps": warm, "modes": res}
    ref = fields["fp32"]
    us = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    cs = max(np.abs(ref[k]).max() for k in ("cxx", "cxy", "cyy"))
    for label in ("fp32", "net", "frozen"):
        r = res[label]
        r["ey2_rate_rel_err_vs_fp64"] = abs(r["ey2_rate"] / res["fp64"]["ey2_rate"] - 1)
        r["speedup_vs_fp32"] = res["fp32"]["ms_per_block"] / r["ms_per_block"]
        if label != "fp32":
            r["u_linf_vs_fp32"] = max(float(np.abs(fields[label][k] - ref[k]).max()) for k in
                                      ("ux", "uy")) / us
            r["c_linf_vs_fp32"] = max(float(np.abs(fields[label][k] - ref[k]).max()) for k in
                                      ("cxx", "cxy", "cyy")) / cs
    return {"K": K, "threshold": thr, "blocks": nblocks, "warm_plain_steps": warm, "modes": res}


def ensemble_throughput(n_runs: int, steps: int, warmup: int):
    """Aggregate GLUPS of a seeded ensemble advanced as one batch (one launch of the
    fused kernel and one of its fix-up per step, replayed from a CUDA graph)."""
    import torch
    from paper_2201_10132_gb300 import tfkt
    from paper_2201_10132_gb300.inputs import ensemble, perturbation
    runs = ensemble(n_runs)
    params = [tfkt.Params.from_workload(w, tfkt.FP32) for w in runs]
    perts = [perturbation(w.nx, w.ny, w.seed, w.amp, w.u0) for w in runs]
    ws = torch.empty(tfkt.batch_required_bytes(params), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    nodes = sum(w.nx * w.ny for w in runs)
    with tfkt.Batch(params, perts, workspace=ws, stream=stream.cuda_stream) as b:
        b.step(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        diag = [b.run(i).diagnostics() for i in (0, n_runs - 1)]
        plan = b.plan()
    assert all(math.isfinite(v) for d in diag for v in d.values())
    return {"runs": n_runs, "r_nodes": nodes, "steps": steps, "ms_per_step": ms / steps,
            "plan": "per-run kernels" if plan["per_run"] else f"batched kernel, tile 32x{plan['tile_height']}",
            "tuned_ms_per_step": plan["ms"],
            "value": aggregate_glups(1, nodes, steps, ms / 1e3), "unit": "GLUPS",
            "workspace_gb": ws.numel() / 1e9, "nq": 9}


SUB_FIELDS = ["ux", "uy", "cxx", "cxy", "cyy"]


def _hbm_roofline(kernel: str, bytes_per_launch: float, ms: float, traffic=None, **extra):
    peak, kind = _peaks()
    ach = bytes_per_launch / (ms / 1e3) / 1e9
    r = {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "GB/s",
         "frac": ach / peak, "peak_kind": kind, "bytes_per_launch": bytes_per_launch,
         "traffic": traffic}
    r.update(extra)
    return r


def fp16_sub(W, steps: int, warmup: int, fp32_ms_per_step: float, fp32_fused_ms: float,
             ref_fields: dict):
    """The throughput workload with FP16 polymer storage (FP32 solvent, FP32
    arithmetic) from the identical seeded state: time per step, the fused kernel
    against the HBM roofline at its own algorithmic bytes, the speedup over the FP32
    line just measured, and the largest field errors against that FP32 run after
    the same number of steps (velocity against the velocity scale, conformation
    against the largest diagonal conformation)."""
    import numpy as np
    import torch
    from paper_2201_10132_gb300 import tfkt
    from paper_2201_10132_gb300.inputs import perturbation
    p = tfkt.Params.from_workload(W, tfkt.FP16)
    ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    s = tfkt.Solver(p, perturbation(W.nx, W.ny, W.seed, W.amp, W.u0), workspace=ws,
                    stream=stream.cuda_stream)
    info = s.info
    s.step(warmup)
    s.sync()
    kms = np.zeros(len(tfkt.KERNELS))
    n = np.zeros(len(tfkt.KERNELS), np.int64)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step_profiled(steps, kms, n)
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    f = s.moments(SUB_FIELDS)
    s.close()
    del s, ws
    torch.cuda.empty_cache()
    nodes = W.nx * W.ny
    k = tfkt.KERNELS.index("fused")
    fused_ms = kms[k] / max(n[k], 1)
    pb = 9 * 4 + 25 * info["nq"] * 2
    nm = info["nq"] + 6
    us = max(np.abs(ref_fields["ux"]).max(), np.abs(ref_fields["uy"]).max())
    cs = max(np.abs(ref_fields["cxx"]).max(), np.abs(ref_fields["cyy"]).max())
    err = {name: float(np.abs(f[name] - ref_fields[name]).max() /
                       (us if name in ("ux", "uy") else cs)) for name in SUB_FIELDS}
    return {"storage": "fp16 polymer deviations (scaled), fp32 solvent deviations; fp32 arithmetic",
            "ms_per_step": ms, "value": nodes / (ms / 1e3) / 1e9, "unit": "GLUPS",
            "fused_ms": fused_ms, "speedup_vs_fp32_step": fp32_ms_per_step / ms,
            "speedup_vs_fp32_fused": fp32_fused_ms / fused_ms,
            "roofline": _hbm_roofline("fused", nodes * (2 * pb + 2 * nm * 4), fused_ms,
                                      fused_traffic(nodes, "fp16"),
                                      traffic_source="ncu capture of the 512^2 case, scaled by r-nodes"),
            "linf_vs_fp32_after_steps": err, "steps": steps,
            "gpu_launches": int(n.sum()), "clocks": clocks}


def ensemble_sub(n_runs: int, steps: int, warmup: int):
    """The seeded 256-run ensemble advanced as one batch: the autotuned plan's time per
    step for all runs together, and the step's algorithmic bytes against the HBM
    roofline (the step is a replayed graph of each run's fused and fix-up kernels, so
    the time is the whole step's)."""
    import torch
    from paper_2201_10132_gb300.inputs import ensemble
    torch.cuda.empty_cache()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    r = ensemble_throughput(n_runs, steps, warmup)
    r["clocks"] = sampler.stop()
    nq = r["nq"]
    per_node = 2 * (9 + 25 * nq) * 4 + 2 * (nq + 6) * 4
    r["roofline"] = _hbm_roofline("fused + fix-up of every run (whole step)",
                                  r["r_nodes"] * per_node, r["ms_per_step"],
                                  algorithmic_bytes_per_node=per_node)
    r["workload"] = f"{n_runs} seeded runs: square grids 128-1024, Re 1-20, Wi 0.1-2, " \
                    f"beta 0.1/0.2/0.5, N_Q = {nq}, FP32"
    return r


def slab_sub(W, steps: int, warmup: int, ref_fields: dict, fp32_ms_per_step: float, parts: int = 2):
    """The throughput workload split into `parts` y-slabs on this one GPU (one run,
    slab contexts with ghost rows refreshed from the neighbours before every step,
    device-to-device halo copies on one stream): time per step with the exchange,
    the exchange alone, its bytes, and whether the owned rows equal the FP32
    single-domain run after the same number of steps bit for bit."""
    import numpy as np
    import torch
    from paper_2201_10132_gb300 import slabs as S, tfkt
    from paper_2201_10132_gb300.inputs import perturbation
    torch.cuda.empty_cache()
    p = tfkt.Params.from_workload(W, tfkt.FP32)
    pert = perturbation(W.nx, W.ny, W.seed, W.amp, W.u0)
    stream = torch.cuda.Stream()
    sl, bufs, wss = [], [], []
    for y0, n in S.partition(W.ny, parts):
        ws = torch.empty(tfkt.slab_required_bytes(p, n), dtype=torch.uint8, device="cuda")
        s = tfkt.Slab(p, y0, n, S.local_perturbation(pert, y0, n), workspace=ws,
                      stream=stream.cuda_stream)
        nb = s.halo_bytes()
        sl.append(s)
        wss.append(ws)
        bufs.append((torch.empty(nb, dtype=torch.uint8, device="cuda"),
                     torch.empty(nb, dtype=torch.uint8, device="cuda")))
    del pert

    def step():
        for s in sl:
            s.step(1)
        S.exchange_local(sl, bufs)

    S.exchange_local(sl, bufs)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the exchange alone (it leaves the state unchanged: the ghost rows are already current)
    e0.record(stream)
    for _ in range(steps):
        S.exchange_local(sl, bufs)
    e1.record(stream)
    e1.synchronize()
    xms = e0.elapsed_time(e1) / steps
    clocks = sampler.stop()
    same = True
    for k in SUB_FIELDS:
        got = np.concatenate([s.owned(s.moments([k])[k]) for s in sl])
        same = same and bool(np.array_equal(got, ref_fields[k]))
    nb = sl[0].halo_bytes()
    for s in sl:
        s.close()
    del sl, wss, bufs
    torch.cuda.empty_cache()
    nodes = W.nx * W.ny
    return {"slabs": parts, "ghost_rows_per_side": S.GHOST, "ms_per_step": ms,
            "value": nodes / (ms / 1e3) / 1e9, "unit": "GLUPS",
            "exchange_ms_per_step": xms, "halo_bytes_per_side": nb,
            "exchange_bytes_per_step": 2 * parts * nb,
            "overhead_vs_single_domain": ms / fp32_ms_per_step - 1,
            "owned_rows_bit_identical_to_single_domain": same, "steps": steps,
            "clocks": clocks}


def _growth_rate(t, ey2):
    """Least-squares slope of log(sum U_y^2) against steps over the second half."""
    import numpy as np
    h = len(t) // 2
    return float(np.polyfit(np.asarray(t[h:], float), np.log(np.asarray(ey2[h:])), 1)[0])


def learned_sub(W, blocks: int = 6, warm: int = 40, grid: int = 512, growth_warm: int = 1000,
                growth_blocks: int = 60):
    """The learned macro-step (one plain step, the network in place of K polymer
    steps, K solvent sub-steps; the committed weights) against the plain step:
    (1) speed at the throughput workload's size, block against 1 + K plain steps;
    (2) the growth rate of sum U_y^2 in a growing phase against the FP64 plain run:
    the same lattice parameters on grid^2 r-nodes (forcing wavelength kept) started
    on the laminar profile with the seeded perturbation; after `growth_warm` plain
    steps (in each run's own precision) the instability grows (sum U_y^2 by about
    e^1 over the window), and `growth_blocks` blocks follow, the rate fitted over
    their second half; the plain FP32 run and the block without the network are
    reported beside it."""
    import numpy as np
    import torch
    from dataclasses import replace
    from paper_2201_10132_gb300 import tfkt, train_lpm
    from paper_2201_10132_gb300.inputs import perturbation
    vec, meta = train_lpm.load()
    K, thr = meta["K"], meta["threshold"]
    torch.cuda.empty_cache()
    net = tfkt.Mlp(vec)
    out = {"K": K, "threshold": thr}
    # (1) speed at the full size
    p = tfkt.Params.from_workload(W, tfkt.FP32)
    ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    s = tfkt.Solver(p, perturbation(W.nx, W.ny, W.seed, W.amp, W.u0), workspace=ws,
                    stream=st.cuda_stream)
    s.step(warm)
    tfkt.lpm_run(s, net, 1, K=K, tile=32, threshold=thr)     # warm-up block
    s.sync()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kms = np.zeros(len(tfkt.KERNELS))
    n = np.zeros(len(tfkt.KERNELS), np.int64)
    e0.record(st)
    s.step_profiled(1 + K, kms, n)
    e1.record(st)
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1)
    fl = 0
    e0.record(st)
    for _ in range(blocks):
        fl += tfkt.lpm_run(s, net, 1, K=K, tile=32, threshold=thr)
    e1.record(st)
    e1.synchronize()
    block_ms = e0.elapsed_time(e1) / blocks
    # every tile falling back (threshold 0): the block keeps the plain step's conformation
    fl_all = 0
    e0.record(st)
    for _ in range(blocks):
        fl_all += tfkt.lpm_run(s, net, 1, K=K, tile=32, threshold=0.0)
    e1.record(st)
    e1.synchronize()
    fallback_ms = e0.elapsed_time(e1) / blocks
    clocks = sampler.stop()
    nq = s.info["nq"]
    s.close()
    del s, ws
    torch.cuda.empty_cache()
    nodes = W.nx * W.ny
    k = tfkt.KERNELS.index("fused")
    fused_ms = kms[k] / max(n[k], 1)
    info_bytes = 2 * (9 + 25 * nq) * 4 + 2 * (nq + 6) * 4
    out["speed"] = {"workload": W.name, "ms_per_block": block_ms, "plain_ms_per_1_plus_K": plain_ms,
                    "speedup_vs_fp32": plain_ms / block_ms,
                    "glups_equivalent": nodes * (1 + K) / (block_ms / 1e3) / 1e9,
                    "fallback_tiles": fl, "blocks": blocks,
                    "ms_per_block_all_tiles_falling_back": fallback_ms,
                    "tiles_falling_back_in_that_run": fl_all,
                    "roofline": _hbm_roofline("fused (the block's plain step)", nodes * info_bytes,
                                              fused_ms,
                                              share_of_block=fused_ms / block_ms),
                    "clocks": clocks}
    # (2) growth rate in a growing phase
    G = replace(W, name=f"laminar-start-{grid}x{grid}-nq32", nx=grid, ny=grid,
                k_periods=W.k_periods * grid // W.ny, ic_mode=1)
    pert = perturbation(G.nx, G.ny, G.seed, G.amp, G.u0)
    rates, ey = {}, {}
    for label in ("fp64", "fp32", "net", "frozen"):
        pg = tfkt.Params.from_workload(G, tfkt.FP64 if label == "fp64" else tfkt.FP32)
        sg = tfkt.Solver(pg, pert)
        sg.step(growth_warm)
        t, e = [], []
        for b in range(growth_blocks):
            if label in ("fp64", "fp32"):
                sg.step(1 + K)
            elif label == "net":
                tfkt.lpm_run(sg, net, 1, K=K, tile=32, threshold=thr)
            else:
                tfkt.lpm_run(sg, None, 1, K=K, tile=32, threshold=thr, mode=tfkt.LPM_FROZEN)
            t.append((b + 1) * (1 + K))
            e.append(sg.diagnostics()["ey2"])
        sg.close()
        rates[label] = _growth_rate(t, e)
        ey[label] = (e[0], e[-1])
    net.close()
    torch.cuda.empty_cache()
    out["growth"] = {"workload": G.name, "warm_plain_steps": growth_warm,
                     "steps": growth_blocks * (1 + K),
                     "ey2_first_last": ey, "ey2_rate_per_step": rates,
                     "rate_rel_err_vs_fp64": {k: abs(rates[k] / rates["fp64"] - 1)
                                              for k in ("fp32", "net", "frozen")},
                     "growing": rates["fp64"] > 0}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kolmogorov-4096x4096-nq32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16"],
                    help="population storage of the throughput run (compute is FP32 in both)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--ensemble", type=int, default=0, metavar="RUNS",
                    help="instead of the throughput line: a seeded ensemble advanced as one batch")
    ap.add_argument("--precision-sweep", type=int, default=0, metavar="STEPS",
                    help="instead of the throughput line: FP64 vs FP32 vs FP16 errors and times")
    ap.add_argument("--capacity", action="store_true",
                    help="instead of the throughput line: the 8192^2 run in FP16 storage")
    ap.add_argument("--learned", type=int, default=0, metavar="BLOCKS",
                    help="instead of the throughput line: the learned macro-step against the "
                         "plain step (speed, field and growth-rate errors)")
    ap.add_argument("--learned-warm", type=int, default=240)
    ap.add_argument("--learned-only", action="store_true",
                    help="time the learned block alone (no reference runs; for profiling)")
    ap.add_argument("--no-sub", action="store_true",
                    help="the throughput line only, without the fp16 / ensemble / learned "
                         "sub-records (profiling runs)")
    args = ap.parse_args()
    from paper_2201_10132_gb300.inputs import WORKLOADS
    W = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, W)

    if args.ensemble:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"ensemble": ensemble_throughput(args.ensemble, args.steps,
                                                          args.warmup)}), flush=True)
        return
    if args.capacity:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"capacity": capacity_run(args.steps, args.warmup)}), flush=True)
        return
    if args.learned:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"learned": learned_vs_plain(W, args.learned, args.learned_warm,
                                                      args.learned_only),
                          "workload": W.name}), flush=True)
        return
    if args.precision_sweep:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps({"precision_sweep": precision_sweep(W, args.precision_sweep),
                          "workload": W.name, "steps": args.precision_sweep}), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import numpy as np
    import torch
    from paper_2201_10132_gb300 import tfkt
    from paper_2201_10132_gb300.inputs import perturbation
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    p = tfkt.Params.from_workload(W, tfkt.FP16 if args.storage == "fp16" else tfkt.FP32)
    nodes = W.nx * W.ny
    ws = torch.empty(tfkt.required_bytes(p), dtype=torch.uint8, device="cuda")
    pert = torch.from_numpy(perturbation(W.nx, W.ny, replica_seed(W.seed, rank), W.amp,
                                         W.u0)).pin_memory()
    stream = torch.cuda.Stream()
    solver = tfkt.Solver(p, pert.numpy(), workspace=ws, stream=stream.cuda_stream)
    info = solver.info
    solver.step(args.warmup)
    solver.sync()

    kms = np.zeros(len(tfkt.KERNELS))
    launches = np.zeros(len(tfkt.KERNELS), np.int64)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step_profiled(args.steps, kms, launches)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    diag = solver.diagnostics()
    assert all(math.isfinite(v) for v in diag.values()), diag
    subs = rank == 0 and world == 1 and not args.no_sub
    ref_fields = solver.moments(SUB_FIELDS) if subs and args.storage == "fp32" else None
    solver.close()

    # end to end through the C-ABI with pinned host buffers: create from the host
    # perturbation, per step a step and a diagnostics read-back, then the velocity
    # and density fields back to the host
    e2e = None
    if not args.no_e2e:
        out_diag = torch.zeros(len(tfkt.DIAGS), dtype=torch.float64).pin_memory()
        names = ["rho_s", "ux", "uy"]
        host_f = torch.empty((len(names), W.ny, W.nx), dtype=torch.float64).pin_memory()
        barrier()
        t0 = time.perf_counter()
        s2 = tfkt.Solver(p, pert.numpy(), workspace=ws, stream=stream.cuda_stream)
        for _ in range(args.steps):
            s2.step(1)
            s2.diagnostics_into(out_diag.numpy())
        s2.moments_into(tfkt.field_mask(names), host_f.numpy())
        s2.close()
        t_e2e = max_over_ranks(time.perf_counter() - t0, dist)
        e2e = {"value": aggregate_glups(world, nodes, args.steps, t_e2e), "unit": "GLUPS",
               "h2d_bytes_per_step": pert.numel() * 8 / args.steps,
               "d2h_bytes_per_step": (args.steps * out_diag.numel() * 8 + host_f.numel() * 8)
               / args.steps}

    if rank == 0:
        hbm_peak, peak_kind = _peaks()
        s = 4  # bytes per moment value (FP32)
        npl, nm = 9 + 25 * info["nq"], info["nq"] + 6
        # bytes of a node's populations: FP32, or FP32 solvent and FP16 polymer
        pb = npl * s if args.storage == "fp32" else 9 * 4 + 25 * info["nq"] * 2
        # algorithmic bytes per launch: each population read once and written once;
        # moment planes read once (and written once where the kernel produces them)
        model = {"moments": nodes * (pb + nm * s), "step": nodes * (2 * pb + nm * s),
                 "fused": nodes * (2 * pb + 2 * nm * s), "fixup": None}
        per = {}
        for k, name in enumerate(tfkt.KERNELS):
            if launches[k]:
                ms_l = kms[k] / launches[k]
                b = model[name]
                per[name] = {"launches": int(launches[k]), "ms_per_launch": ms_l,
                             "bytes_per_launch": b,
                             "achieved_gbs": None if b is None else b / (ms_l / 1e3) / 1e9}
        top = max(per, key=lambda k: per[k]["ms_per_launch"] * per[k]["launches"])
        value = aggregate_glups(world, nodes, args.steps, ms / 1e3)
        ach = per[top]["achieved_gbs"]
        line = {
            "metric": "GLUPS (1e9 r-node updates/s), 4096^2 two-fluid step",
            "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": W.name, "nx": W.nx, "ny": W.ny, "nq": info["nq"],
                       "re": W.re, "wi": W.wi, "beta": W.beta, "k_periods": W.k_periods,
                       "storage": "fp32 deviations from rest" if args.storage == "fp32" else
                                  "fp16 polymer deviations (scaled), fp32 solvent deviations",
                       "l2": f"inputs larger than L2 (populations {nodes * pb / 1e9:.2f} GB "
                             "per buffer, L2 129 MB)",
                       "parallelism": f"{world} independent runs"},
            "roofline": {"bound": "hbm", "kernel": top + "_kernel", "achieved": ach,
                         "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                         "peak_kind": peak_kind,
                         "traffic": fused_traffic(nodes, args.storage) if top == "fused" else None,
                         "traffic_source": "ncu capture of the 512^2 case, scaled by r-nodes",
                         "bytes_per_launch": per[top]["bytes_per_launch"],
                         "step_model_gbs": nodes * (2 * pb + 2 * nm * s) / (ms / args.steps / 1e3) / 1e9,
                         "kernels": per},
            "updates": {"hyper_lattice_per_s": value * 1e9 * info["nq"],
                        "populations_per_s": value * 1e9 * npl},
            "e2e": e2e,
            "gpu_launches": int(launches.sum()),
            "clocks": clocks,
            "cpu_baseline": None,
        }
        if subs:
            # the side modes, each timed on its own with its own clock record
            del ws
            torch.cuda.empty_cache()
            sub_launches = 0
            if ref_fields is not None:
                line["fp16"] = fp16_sub(W, args.steps, args.warmup, ms / args.steps,
                                        per["fused"]["ms_per_launch"], ref_fields)
                sub_launches += line["fp16"]["gpu_launches"]
            line["slab"] = slab_sub(W, args.steps, args.warmup, ref_fields, ms / args.steps) \
                if "ux" in (ref_fields or {}) else None
            line["ensemble"] = ensemble_sub(256, 4, 2)
            line["learned"] = learned_sub(W)
            line["gpu_launches_sub_records"] = sub_launches
        if world == 1 and not args.no_cpu_baseline:
            # the oracle on the host cores, after every GPU timing so that its
            # threads share the host with none of them
            cpu_base = oracle_sample(W)
            one = oracle_sample(W, target_s=4.0, threads=1)
            cpu_base["single_thread"] = {"value": one["value"], "sample": one["sample"]}
            cpu_base["host"] = {"cpu": host_cpu(), "nproc": os.cpu_count()}
            line["cpu_baseline"] = cpu_base
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
