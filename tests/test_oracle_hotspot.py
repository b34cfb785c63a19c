"""Pins of the oracle's hot-spot initial state (3D thermal box workload).

The sampled radial density must follow rho(r) ∝ T(r)^3 with
T(r) = T0 + dT exp(-r^2 / 2w^2) (chi^2 over shells against the integral of
4 pi r^2 rho(r), normalised with the closed-form Gaussian moments), and each
particle's energy must be Gamma(3, T) at its own T(r) (KS on E / T(r))."""
import math

import numpy as np
from scipy import integrate, stats

from oracle import oracle as O
import physics as PH


def test_hotspot_density_and_local_spectrum():
    L, T0, dT, w = 12.8, 0.4, 0.2, 1.0
    n = 400000
    p = O.make_params(L=(L, L, L), n=(16, 16, 16), dt=0.1, sigma_fm2=0.5, n_test=1.0, seed=4)
    st = O.init_hotspot(p, n, T0, dT, w)
    assert st[:3].min() >= 0.0 and st[:3].max() <= L
    r = np.sqrt(((st[:3] - L / 2) ** 2).sum(axis=0))

    def rho(x):
        return (T0 + dT * math.exp(-x * x / (2 * w * w))) ** 3

    # normalisation: T0^3 L^3 + sum_k binom(3,k) T0^(3-k) dT^k (2 pi w^2 / k)^(3/2)
    Z = T0 ** 3 * L ** 3
    for k, c in ((1, 3), (2, 3), (3, 1)):
        Z += c * T0 ** (3 - k) * dT ** k * (2 * math.pi * w * w / k) ** 1.5
    edges = np.array([0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 4.0])
    obs = np.histogram(r, bins=edges)[0]
    exp = np.array([integrate.quad(lambda x: 4 * math.pi * x * x * rho(x), a, b)[0] / Z * n
                    for a, b in zip(edges[:-1], edges[1:])])
    chi2 = np.sum((obs - exp) ** 2 / exp)
    assert stats.chi2.sf(chi2, len(obs)) > 1e-4
    # the hot spot is visible: the innermost shell is denser than the base gas
    assert obs[0] / exp[0] > 0.9 and exp[0] / (n * 4 / 3 * math.pi * 0.5 ** 3 * T0 ** 3 / Z) > 2.5
    # local thermal spectrum
    Tloc = T0 + dT * np.exp(-r * r / (2 * w * w))
    E = np.sqrt((st[3:] ** 2).sum(axis=0))
    assert stats.kstest(E / Tloc, PH.gamma3_cdf).pvalue > 1e-3
