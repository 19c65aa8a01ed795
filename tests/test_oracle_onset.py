"""Oracle pin: linear instability of Newtonian Kolmogorov flow (Sec. VII, beta = 1).

The laminar profile U0 sin(y/l) of the forced flow becomes unstable to
long-wave perturbations e^{i alpha x / l} above a Reynolds number Re_c(alpha)
that tends to sqrt(2) as alpha -> 0 (Meshalkin & Sinai 1961; the long-wave
growth rate is alpha^2 (Re/2 - 1/Re) U0/l, the "negative eddy viscosity" of
Sivashinsky 1985).

The growth rates are computed here independently of the oracle, by a Fourier-
Galerkin solution of the linearised vorticity equation about U = sin y
(stream function phi = sum_n a_n e^{i n y}, k_n^2 = alpha^2 + n^2):

    sigma k_n^2 a_n = -(alpha/2) [(k_{n-1}^2 - 1) a_{n-1} - (k_{n+1}^2 - 1) a_{n+1}]
                      - (1/Re) k_n^4 a_n,

in units of U0/l. The eigen-solver is itself checked against the two textbook
limits above; the oracle (lattice units, one forcing period across ny, box
nx = ny/alpha) must then reproduce the growth or decay rate of the leading
x-mode, on both sides of the onset.
"""
import numpy as np
import pytest


from linear_kolmogorov import onset as _onset, sigma as _sigma


def test_eigen_solver_textbook_limits():
    assert _onset(0.05) == pytest.approx(np.sqrt(2.0), rel=5e-3)
    for re in (2.0, 3.0):
        long_wave = 0.05 ** 2 * (re / 2 - 1 / re)
        assert _sigma(0.05, re).real == pytest.approx(long_wave, rel=3e-2)
    # finite boxes: the onset moves up as the longest wave shortens
    assert np.sqrt(2.0) < _onset(0.125) < _onset(0.25) < _onset(0.5)


def _oracle_rate(O, ny, alpha, re, u0, steps, chunk=200):
    from paper_2201_10132_gb300.inputs import perturbation
    nx = int(round(ny / alpha))
    lat = O.map_params(nx, ny, 1, 1.0, re, 0.0, 1.0, u0, 1)  # beta = 1: Newtonian
    o = O.Oracle(lat)
    o.init(perturbation(nx, ny, 3, 1e-4, u0), 1)  # laminar profile + small seed field
    t, amp = [], []
    for k in range(steps // chunk):
        o.step(chunk)
        uy = o.fields()["uy"]
        amp.append(np.sqrt((np.abs(np.fft.fft(uy, axis=1)[:, 1]) ** 2).sum()))
        t.append((k + 1) * chunk)
    t, la = np.array(t), np.log(amp)
    h = len(t) // 2  # the second half, after the faster-decaying modes have gone
    return np.polyfit(t[h:], la[h:], 1)[0], lat


@pytest.mark.parametrize("re", [1.2, 1.3, 1.8, 2.5])
def test_kolmogorov_growth_rate_matches_linear_theory(oracle_mod, re):
    """Box 4 forcing wavelengths long (alpha = 1/4, Re_c = 1.552), 32 nodes per
    wavelength, U0 = 0.05 (Mach 0.087). Near the onset the rate is a small
    difference of O(alpha^2) terms, so their O(dx^2) and O(Ma^2) lattice errors
    show as a few per cent of it: the tolerance is 4%."""
    alpha, ny, u0 = 0.25, 32, 0.05
    sig = _sigma(alpha, re)
    assert abs(sig.imag) < 1e-12  # the leading mode is stationary
    pred = sig.real * u0 * (2 * np.pi / ny)  # U0/l -> per lattice step
    steps = int(min(12000, max(4000, 3 / abs(pred)))) // 200 * 200  # ~3 e-foldings
    rate, lat = _oracle_rate(oracle_mod, ny, alpha, re, u0, steps)
    assert np.sign(rate) == np.sign(pred) == (1 if re > _onset(alpha) else -1)
    assert rate == pytest.approx(pred, rel=0.04)
