"""Seeded synthetic inputs of the Kolmogorov-flow workloads.

This module holds no arithmetic of the two-fluid scheme: it only draws the
random initial velocity perturbation (Sec. VII seeds the instability with a
random field) and names the workload presets. Both the CUDA path (through the
C-ABI, which takes the perturbation as an input array) and the CPU oracle use
it, so both start from the same bytes.

Perturbation recipe: a divergence-free field from the stream function
    phi(x, y) = sum_{1<=|m|,|n|<=4} cos(2 pi (m x / nx + n y / ny) + theta_mn),
    u'_x = d phi / dy,  u'_y = -d phi / dx  (analytic derivatives),
with phases theta_mn = 2 pi * U[0,1) drawn from splitmix64(seed) in the order
m = -4..4, n = -4..4 (zeros skipped), scaled so that rms |u'| = amp * u0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict

import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(seed: int):
    """Counter-based splitmix64 stream (Steele, Lea & Flood 2014)."""
    state = seed & _MASK
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        yield z ^ (z >> 31)


def perturbation(nx: int, ny: int, seed: int, amp: float, u0: float,
                 kmax: int = 4) -> np.ndarray:
    """Random divergence-free velocity perturbation, float64 array [2, ny, nx]."""
    rng = splitmix64(seed)
    modes = []
    for m in range(-kmax, kmax + 1):
        for n in range(-kmax, kmax + 1):
            if m == 0 or n == 0:
                continue
            theta = 2.0 * math.pi * ((next(rng) >> 11) * 2.0 ** -53)
            modes.append((m, n, theta))
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    # sin(a + b) = sin(a) cos(b) + cos(a) sin(b), a = 2 pi m x / nx, b = 2 pi n y / ny + theta:
    # each component is a sum of rank-1 products, evaluated as one matrix product.
    nm = len(modes)
    ay = np.zeros((ny, 2 * nm))
    ax = np.zeros((2 * nm, nx))
    by = np.zeros((ny, 2 * nm))
    for k, (m, n, th) in enumerate(modes):
        a = 2.0 * math.pi * m * x / nx
        b = 2.0 * math.pi * n * y / ny + th
        kx, ky = 2.0 * math.pi * m / nx, 2.0 * math.pi * n / ny
        # u_x = d phi/dy = -ky sin(a + b);  u_y = -d phi/dx = kx sin(a + b)
        ay[:, 2 * k] = -ky * np.cos(b)
        ay[:, 2 * k + 1] = -ky * np.sin(b)
        by[:, 2 * k] = kx * np.cos(b)
        by[:, 2 * k + 1] = kx * np.sin(b)
        ax[2 * k] = np.sin(a)
        ax[2 * k + 1] = np.cos(a)
    ux = ay @ ax
    uy = by @ ax
    rms = math.sqrt(float(np.mean(ux * ux + uy * uy)))
    scale = amp * u0 / rms if rms > 0 else 0.0
    return np.ascontiguousarray(np.stack([ux * scale, uy * scale]))


@dataclass(frozen=True)
class Workload:
    """A Kolmogorov run: grid, Q-grid, dimensionless groups, forcing, seed."""
    name: str
    nx: int
    ny: int
    q_side: int
    q_radius: float
    re: float
    wi: float
    beta: float
    u0: float
    k_periods: int
    seed: int
    amp: float
    tau2: float = 0.0
    ic_mode: int = 0

    def as_dict(self):
        return asdict(self)


# Small FP64 case: 64^2, Re 5, Wi 0.5, beta 0.2, 8x8 Q-grid masked to R = 4 (52 nodes).
KOLMOGOROV_64 = Workload("kolmogorov-64x64-nq52", 64, 64, 8, 4.0, 5.0, 0.5, 0.2, 0.05, 1, 0, 1e-3)
# Throughput case: 4096^2, Re 10, Wi 1, beta 0.2, 6x6 Q-grid masked to R = 3 (32 nodes),
# forcing wavelength 64 nodes (k_periods = 64).
KOLMOGOROV_4096 = Workload("kolmogorov-4096x4096-nq32", 4096, 4096, 6, 3.0, 10.0, 1.0, 0.2, 0.05,
                           64, 0, 1e-3)
# Profiling case: same lattice parameters at 1024^2 (forcing wavelength 64 nodes).
KOLMOGOROV_1024 = Workload("kolmogorov-1024x1024-nq32", 1024, 1024, 6, 3.0, 10.0, 1.0, 0.2, 0.05,
                           16, 0, 1e-3)
# Profiling case small enough for a full ncu capture (inputs still larger than L2).
KOLMOGOROV_512 = Workload("kolmogorov-512x512-nq32", 512, 512, 6, 3.0, 10.0, 1.0, 0.2, 0.05,
                          8, 0, 1e-3)
# Capacity case: the same lattice parameters at 8192^2 (forcing wavelength 64 nodes); it
# fits one GPU's memory only with FP16 polymer storage.
KOLMOGOROV_8192 = Workload("kolmogorov-8192x8192-nq32", 8192, 8192, 6, 3.0, 10.0, 1.0, 0.2, 0.05,
                           128, 0, 1e-3)
WORKLOADS = {w.name: w for w in (KOLMOGOROV_64, KOLMOGOROV_512, KOLMOGOROV_1024, KOLMOGOROV_4096,
                                 KOLMOGOROV_8192)}


def ensemble(n: int = 256, seed: int = 0, q_side: int = 3, q_radius: float = 1.5):
    """A seeded ensemble of independent Kolmogorov runs: square grids drawn from
    {128, 256, 512, 1024}, Re uniform in [1, 20], Wi uniform in [0.1, 2], beta from
    {0.1, 0.2, 0.5}, forcing wavelength 64 nodes, a small Q-grid (3 x 3 masked to
    R = 1.5: 9 nodes) so that ~89 M r-nodes fit in memory in FP32. Wi is kept away
    from 0, where the dilute polymer density psi_tot = 3 eta_p / lambda_H diverges."""
    rng = splitmix64(seed ^ 0x5EED)
    u = lambda: (next(rng) >> 11) * 2.0 ** -53
    sizes = (128, 256, 512, 1024)
    betas = (0.1, 0.2, 0.5)
    runs = []
    for k in range(n):
        side = sizes[int(u() * 4) % 4]
        re = 1.0 + 19.0 * u()
        wi = 0.1 + 1.9 * u()
        beta = betas[int(u() * 3) % 3]
        runs.append(Workload(f"ensemble-{k}", side, side, q_side, q_radius, re, wi, beta, 0.05,
                             side // 64, seed * 100003 + k, 1e-3))
    return runs
