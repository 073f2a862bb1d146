"""Texture fit of Eq. (10): the oracle (scipy curve_fit) pinned to exact and
sampled Gaussians, and the library's host fit against the oracle."""
import numpy as np
import pytest


def _gauss_hist(g, N):
    import oracle
    phi = oracle.folded_centres()
    p = np.exp(-phi ** 2 / (2 * g * g)) / (g * np.sqrt(2 * np.pi))
    return np.rint(p / p.sum() * N).astype(np.int64)


@pytest.mark.parametrize("g", [3.0, 6.0, 9.0, 12.0])
def test_oracle_fit_recovers_exact_gaussian(oracle, g):
    # the histogram holds the Gaussian's values at the bin centres; for these
    # widths the fold at +-45 degrees truncates less than 2e-4 of the mass
    fit = oracle.texture_fit(_gauss_hist(g, 10 ** 12))
    assert abs(fit - g) < 1e-3 * g, fit


@pytest.mark.parametrize("g", [6.0, 12.0])
def test_oracle_fit_sampled_gaussian(oracle, g):
    rng = np.random.default_rng(int(g))
    fits = []
    for _ in range(20):
        phi = rng.normal(0.0, g, size=200_000)
        phi = phi[np.abs(phi) < 45]
        theta = np.where(phi < 0, phi + 90.0, phi)
        h = np.bincount(np.floor(theta).astype(int), minlength=90)[:90]
        fits.append(oracle.texture_fit(h))
    fits = np.array(fits)
    assert abs(fits.mean() - g) < 4 * fits.std(ddof=1) / np.sqrt(len(fits)) + 0.01 * g


def test_library_fit_matches_oracle(oracle):
    from paper_1007_3509_gb300 import build, hmcpotts as hm
    build.build()
    rng = np.random.default_rng(3)
    for g in (4.0, 9.0, 20.0):
        h = _gauss_hist(g, 10 ** 6) + rng.integers(0, 50, size=90)
        gl, _ = hm.hp_texture_fit(h)
        assert abs(gl - oracle.texture_fit(h)) < 1e-4 * gl
    with pytest.raises(hm.HPError):
        hm.hp_texture_fit(np.zeros(90, dtype=np.int64))
