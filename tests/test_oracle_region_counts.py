"""The oracle's split of the particles over initial regions (Sec. 5).

A Boltzmann gluon gas has number density n ∝ T^3, so a region of volume V at
temperature T receives a share ∝ T^3 V of the test particles; the integer
counts follow the largest-remainder rule, ties going to the lower region.
Expected counts below are worked out by hand from that definition:

- the 20 000-particle Riemann run (box 10 x 1 x 1 fm split at x = 5 fm,
  T = 400 / 320 MeV): shares 0.064 : 0.032768, i.e. 13 227.51 / 6 772.49,
  floors 13 227 / 6 772, the larger remainder (0.513) takes the last one:
  13 228 / 6 772;
- the 16 M-particle run: 10 582 010.58 / 5 417 989.42 -> 10 582 011 / 5 417 989;
- three regions of unequal volume, T = 0.3, 0.5, 0.2 GeV, V = 2, 1, 3 fm^3,
  1000 particles: weights 0.054, 0.125, 0.024 give 266.01 / 615.76 / 118.23,
  floors 266 / 615 / 118, the one left over goes to the largest remainder
  (0.76): 266 / 616 / 118;
- ties: 5 particles over two equal regions -> 3 / 2; 7 over three -> 3 / 2 / 2.

A T^2 weighting (or a dropped volume factor) changes every one of these.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _regions(specs):
    return [((x0, 0.0, 0.0), (x1, 1.0, 1.0), T) for (x0, x1, T) in specs]


@pytest.mark.parametrize("n,expected", [(20000, [13228, 6772]), (16000000, [10582011, 5417989])])
def test_riemann_split_by_t_cubed(n, expected):
    regs = O.riemann_regions((10.0, 1.0, 1.0), 0.4, 0.32)
    got = O.region_counts(n, regs)
    assert list(got) == expected


def test_three_regions_unequal_volumes():
    regs = _regions([(0.0, 2.0, 0.3), (2.0, 3.0, 0.5), (3.0, 6.0, 0.2)])
    assert list(O.region_counts(1000, regs)) == [266, 616, 118]


def test_ties_go_to_the_lower_region():
    assert list(O.region_counts(5, _regions([(0.0, 1.0, 0.4), (1.0, 2.0, 0.4)]))) == [3, 2]
    assert list(O.region_counts(7, _regions([(0.0, 1.0, 0.4), (1.0, 2.0, 0.4), (2.0, 3.0, 0.4)]))) == [3, 2, 2]


def test_counts_sum_and_lie_within_one_particle_of_the_share():
    rng = np.random.default_rng(3)
    for _ in range(50):
        k = int(rng.integers(1, 6))
        edges = np.sort(rng.uniform(0.0, 10.0, size=k + 1))
        edges[0], edges[-1] = 0.0, 10.0
        if np.any(np.diff(edges) <= 1e-6):
            continue
        Ts = rng.uniform(0.1, 0.8, size=k)
        regs = _regions([(edges[r], edges[r + 1], Ts[r]) for r in range(k)])
        n = int(rng.integers(0, 10 ** 6))
        got = np.asarray(O.region_counts(n, regs), dtype=np.int64)
        assert got.sum() == n
        share = n * Ts ** 3 * np.diff(edges) / np.sum(Ts ** 3 * np.diff(edges))
        assert np.all(np.abs(got - share) < 1.0)


def test_init_thermal_fills_regions_in_generation_order():
    """Particles are generated region by region: the first 13 228 of the
    20 000-particle Riemann state lie in the left half, the rest in the right."""
    L = (10.0, 1.0, 1.0)
    regs = O.riemann_regions(L, 0.4, 0.32)
    p = O.make_params(L=L, n=(100, 1, 1), dt=0.05, sigma_fm2=1.0, n_test=195.9, seed=0)
    st = O.init_thermal(p, 20000, regs)
    x = st[0]
    assert np.all(x[:13228] <= 5.0) and np.all(x[13228:] >= 5.0)
