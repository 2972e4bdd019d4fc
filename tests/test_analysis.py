"""The chi^2 spectral fit (Sec. 4.3): on histograms drawn from known
distributions it recovers k and sigma, and a Maxwellian gives k = 3 with
sigma = kT / 2, as the paper states."""
import numpy as np
import pytest

from paper_2502_13695_gb300.analysis import fit_chi2

stats = pytest.importorskip("scipy.stats")


@pytest.mark.parametrize("k, sigma", [(3.0, 2.5), (0.7, 4.0), (1.86, 1.0), (2.56, 7.0)])
def test_fit_recovers_parameters(k, sigma):
    rng = np.random.default_rng(7)
    # f(E; k, sigma) is a gamma law of shape k / 2 and scale 2 sigma
    E = rng.gamma(k / 2, 2 * sigma, size=400000)
    edges = np.linspace(0.0, np.quantile(E, 0.999), 121)
    w, _ = np.histogram(E, bins=edges)
    fit = fit_chi2(edges, w)
    assert fit["k"] == pytest.approx(k, rel=0.02)
    assert fit["sigma"] == pytest.approx(sigma, rel=0.03)


def test_maxwellian_gives_k3_and_half_kT():
    rng = np.random.default_rng(11)
    kT = 5.0  # eV
    v = rng.normal(size=(300000, 3)) * np.sqrt(kT)  # m = 1
    E = 0.5 * (v * v).sum(1)
    edges = np.linspace(0.0, 60.0, 151)
    w, _ = np.histogram(E, bins=edges)
    fit = fit_chi2(edges, w)
    assert fit["k"] == pytest.approx(3.0, rel=0.02)
    assert fit["sigma"] == pytest.approx(kT / 2, rel=0.02)


def test_fit_rejects_bad_input():
    with pytest.raises(ValueError):
        fit_chi2([0, 1, 2], [1.0])
    with pytest.raises(ValueError):
        fit_chi2([0, 1, 2], [0.0, 0.0])
