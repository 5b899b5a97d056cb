"""The seeded input generators: the paper's coefficient map (Sec. 4.1) and its
multi-level data (Appendix, Algorithm "Generate Multi-Level Data")."""
import numpy as np
import pytest

from paper_2312_11093_gb300 import inputs


def test_linear_resize_keeps_samples_and_is_exact_on_bilinear_fields():
    """Interpolation from m^2 to (2(m-1)+1)^2 keeps every sample (they sit on
    every other node) and reproduces a bilinear field exactly at any size."""
    rng = np.random.default_rng(0)
    a = rng.uniform(size=(5, 5))
    b = inputs._resize_linear(a, 9)
    assert np.array_equal(b[::2, ::2], a)
    j, i = np.meshgrid(np.arange(5.0), np.arange(5.0), indexing="ij")
    bil = 1.0 + 2.0 * i - 3.0 * j + 0.5 * i * j
    t = np.linspace(0.0, 4.0, 13)
    J, I = np.meshgrid(t, t, indexing="ij")
    assert np.allclose(inputs._resize_linear(bil, 13), 1.0 + 2.0 * I - 3.0 * J + 0.5 * I * J, atol=1e-12)


def test_multilevel_noise_follows_the_algorithm():
    """Replaying the algorithm's draws by hand: levels = 0 is the interpolated
    initial noise; each level doubles the size and adds noise of weight 2^-i."""
    n = 63
    a = inputs.multilevel_noise(n, 0, np.random.default_rng(1))
    r = np.random.default_rng(1)
    assert np.array_equal(a, inputs._resize_linear(r.uniform(0.0, 1.0, size=(5, 5)), n))
    r = np.random.default_rng(2)
    d = r.uniform(0.0, 1.0, size=(5, 5))
    for i in (1, 2, 3):
        d = inputs._resize_linear(d, 2 * d.shape[0])
        d = d + 2.0 ** (-i) * r.uniform(0.0, 1.0, size=d.shape)
    assert d.shape == (40, 40)
    assert np.array_equal(inputs.multilevel_noise(n, 3, np.random.default_rng(2)), inputs._resize_linear(d, n))


@pytest.mark.parametrize("Re", [10.0, 1000.0])
def test_paper_coefficient_range(Re):
    """coef = 10^(-power), power linear in the tensor from 0 to log10 Re: the range
    is exactly [1/Re, 1] with both ends attained, and the map is monotone."""
    rng = np.random.default_rng(3)
    x = inputs.multilevel_noise(31, 2, rng)
    c = inputs.paper_coefficient(x, Re)
    assert np.isclose(c.max(), 1.0, rtol=1e-15) and np.isclose(c.min(), 1.0 / Re, rtol=1e-12)
    order = np.argsort(x.ravel())
    assert np.all(np.diff(c.ravel()[order]) <= 0.0)


def test_mldata_fields_are_seeded_and_shaped():
    n = 127
    mu = inputs.paper_mldata_mu(n, np.random.default_rng(4))
    k = inputs.paper_mldata_k(n, np.random.default_rng(4))
    assert mu.shape == (n, n) and k.shape == (n + 2, n + 2)
    assert np.array_equal(mu, inputs.paper_mldata_mu(n, np.random.default_rng(4)))
    coef = mu * (n + 1)                                     # the paper's coef = mu / h
    assert np.isclose(coef.min(), 1e-3, rtol=1e-12) and np.isclose(coef.max(), 1.0, rtol=1e-15)
    assert k.min() >= 1e-3 * (1 - 1e-12) and k.max() <= 1.0 + 1e-15
    # smoother than white noise: neighbouring values are strongly correlated
    d = np.diff(np.log10(mu), axis=1)
    assert np.std(d) < 0.25 * np.std(np.log10(mu))
