"""Seeded synthetic inputs shaped like the paper's runs (Sec. 5).

No arithmetic of the method lives here: only the sizes of the workloads and a
numpy sampler of initial states (uniform positions per region, isotropic
directions, massless Boltzmann energies E ~ Gamma(3, T)), used by the tests
and by the end-to-end benchmark leg as host-side input.

There is no public dataset behind the paper's runs; these synthetic states
stand in for its 1D Riemann problem (two halves at T_left / T_right).
"""
import math

import numpy as np

HBARC_GEV_FM = 0.1973269804
FM2_PER_MB = 0.1
GLUON_DOF = 16.0


def gluon_density(T, g=GLUON_DOF):
    """Boltzmann number density g T^3 / (pi^2 (hbar c)^3), fm^-3, T in GeV."""
    return g * T ** 3 / (math.pi ** 2 * HBARC_GEV_FM ** 3)


def riemann_regions(L, T_left, T_right):
    half = 0.5 * L[0]
    return [((0.0, 0.0, 0.0), (half, L[1], L[2]), T_left),
            ((half, 0.0, 0.0), (L[0], L[1], L[2]), T_right)]


def n_test_for(n_particles, regions, g=GLUON_DOF):
    """Test particles per physical particle for a gas filling `regions`."""
    nphys = 0.0
    for lo, hi, T in regions:
        vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        nphys += gluon_density(T, g) * vol
    return n_particles / nphys


def region_split(n, regions):
    """Particles per region in proportion to T^3 V, largest remainder."""
    w = np.array([T ** 3 * np.prod(np.subtract(hi, lo)) for lo, hi, T in regions], dtype=float)
    q = n * w / w.sum()
    c = np.floor(q).astype(np.int64)
    frac = q - c
    for _ in range(int(n - c.sum())):
        k = int(np.argmax(frac))
        c[k] += 1
        frac[k] = -1.0
    return c


def thermal_state(n, regions, seed, dtype=np.float64):
    """(6, n) state: x, y, z, px, py, pz, region by region (unsorted)."""
    rng = np.random.default_rng(seed)
    counts = region_split(n, regions)
    st = np.empty((6, n), dtype=np.float64)
    k0 = 0
    for (lo, hi, T), m in zip(regions, counts):
        m = int(m)
        for a in range(3):
            st[a, k0:k0 + m] = rng.uniform(lo[a], hi[a], m)
        E = rng.gamma(3.0, T, m)
        ct = rng.uniform(-1.0, 1.0, m)
        phi = rng.uniform(0.0, 2.0 * math.pi, m)
        s = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
        st[3, k0:k0 + m] = E * s * np.cos(phi)
        st[4, k0:k0 + m] = E * s * np.sin(phi)
        st[5, k0:k0 + m] = E * ct
        k0 += m
    for a in range(3):
        L = max(hi[a] for _, hi, _ in regions)
        np.clip(st[a], 0.0, L, out=st[a])
    return st.astype(dtype)


# Workloads of the benchmark and of the parity tests.  Sizes follow the
# paper's 1D Riemann problem (Sec. 5), scaled as described in the design doc.
def riemann_1d(n_particles, n_cells, dt, sigma_mb, T_left=0.4, T_right=0.32, L=(10.0, 1.0, 1.0)):
    regs = riemann_regions(L, T_left, T_right)
    return dict(L=L, n_cells=(n_cells, 1, 1), dt=dt, sigma_fm2=sigma_mb * FM2_PER_MB,
                n_test=n_test_for(n_particles, regs), n=n_particles, regions=regs,
                T_left=T_left, T_right=T_right)


RIEMANN_SMALL = dict(name="riemann-1d-20k", n=20000, n_cells=100, dt=0.05, sigma_mb=10.0, steps=100)
RIEMANN_16M = dict(name="riemann-1d-16M", n=16_000_000, n_cells=2000, dt=0.0025, sigma_mb=10.0, steps=500)
