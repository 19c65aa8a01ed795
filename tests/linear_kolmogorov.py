"""Linear stability of Newtonian Kolmogorov flow U = sin y (units of U0 and
l): the largest growth rate of a long-wave mode e^{i alpha x} by a Fourier-
Galerkin solution of the linearised vorticity equation (stream function
phi = sum_n a_n e^{i n y}, k_n^2 = alpha^2 + n^2),

    sigma k_n^2 a_n = -(alpha/2) [(k_{n-1}^2 - 1) a_{n-1} - (k_{n+1}^2 - 1) a_{n+1}]
                      - (1/Re) k_n^4 a_n,

and the onset Re_c(alpha) by bisection. Test helper, shared by the oracle's and
the GPU path's growth-rate tests; it is checked against the textbook limits in
tests/test_oracle_onset.py."""
import numpy as np


def sigma(alpha, re, n_modes=40):
    n = np.arange(-n_modes, n_modes + 1)
    k2 = alpha ** 2 + n ** 2
    m = len(n)
    A = np.zeros((m, m))
    A[np.arange(m), np.arange(m)] = -(k2 ** 2) / re
    A[np.arange(1, m), np.arange(m - 1)] = -(alpha / 2) * (k2[:-1] - 1)
    A[np.arange(m - 1), np.arange(1, m)] = (alpha / 2) * (k2[1:] - 1)
    ev = np.linalg.eigvals(A / k2[:, None])
    return ev[np.argmax(ev.real)]


def onset(alpha):
    lo, hi = 1.0, 4.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        if sigma(alpha, mid).real > 0:
            hi = mid
        else:
            lo = mid
    return hi
