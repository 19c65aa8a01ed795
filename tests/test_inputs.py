"""The seeded input generators shared by the CUDA path and the oracle (host only):
the splitmix64 stream, the divergence-free perturbation and the ensemble draw."""
import numpy as np
import pytest

from paper_2201_10132_gb300.inputs import WORKLOADS, ensemble, perturbation, splitmix64


def test_splitmix64_published_value():
    # splitmix64 (Steele, Lea & Flood 2014) from state 0: first output 0xE220A8397B1DCDAF
    g = splitmix64(0)
    assert next(g) == 0xE220A8397B1DCDAF
    assert next(splitmix64(7)) != next(splitmix64(8))


@pytest.mark.parametrize("nx,ny", [(64, 64), (96, 40), (33, 17)])
def test_perturbation_is_divergence_free_with_requested_rms(nx, ny):
    u = perturbation(nx, ny, 3, 1e-3, 0.05)
    assert u.shape == (2, ny, nx) and u.dtype == np.float64 and u.flags.c_contiguous
    assert np.sqrt(np.mean(u[0] ** 2 + u[1] ** 2)) == pytest.approx(1e-3 * 0.05, rel=1e-12)
    # spectral divergence: i kx ux_hat + i ky uy_hat = 0 for every mode
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    ky = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    div = kx * np.fft.fft2(u[0]) + ky * np.fft.fft2(u[1])
    assert np.abs(div).max() < 1e-12 * np.abs(np.fft.fft2(u[0])).max()
    # only modes 1 <= |m|, |n| <= 4 are present
    spec = np.abs(np.fft.fft2(u[0])) + np.abs(np.fft.fft2(u[1]))
    m = np.abs(np.fft.fftfreq(nx) * nx)[None, :]
    n = np.abs(np.fft.fftfreq(ny) * ny)[:, None]
    outside = (m == 0) | (n == 0) | (m > 4) | (n > 4)
    assert spec[outside].max() < 1e-12 * spec.max()


def test_perturbation_is_seeded():
    a = perturbation(32, 32, 5, 1e-3, 0.05)
    assert np.array_equal(a, perturbation(32, 32, 5, 1e-3, 0.05))
    assert not np.array_equal(a, perturbation(32, 32, 6, 1e-3, 0.05))
    assert not perturbation(32, 32, 5, 0.0, 0.05).any()


def test_ensemble_draw():
    runs = ensemble(256)
    assert len(runs) == 256 and runs == ensemble(256)
    assert {r.nx for r in runs} <= {128, 256, 512, 1024}
    assert all(r.nx == r.ny and r.k_periods == r.ny // 64 for r in runs)
    assert all(1.0 <= r.re <= 20.0 and 0.1 <= r.wi <= 2.0 and r.beta in (0.1, 0.2, 0.5) for r in runs)
    assert len({r.seed for r in runs}) == 256
    assert len({r.nx for r in runs}) == 4     # every size occurs


def test_presets_keep_the_forcing_wavelength():
    for w in WORKLOADS.values():
        if w.nx >= 512:
            assert w.ny // w.k_periods == 64, w.name
