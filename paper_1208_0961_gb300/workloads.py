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
# paper's 1D Riemann problem (Sec. 5): the 20 k-particle, 100-cell box and
# its 16 M-particle, 2000-cell scale-up at the same temperatures.
def riemann_1d(n_particles, n_cells, dt, sigma_mb, T_left=0.4, T_right=0.32, L=(10.0, 1.0, 1.0)):
    regs = riemann_regions(L, T_left, T_right)
    return dict(L=L, n_cells=(n_cells, 1, 1), dt=dt, sigma_fm2=sigma_mb * FM2_PER_MB,
                n_test=n_test_for(n_particles, regs), n=n_particles, regions=regs,
                T_left=T_left, T_right=T_right)


RIEMANN_SMALL = dict(name="riemann-1d-20k", n=20000, n_cells=100, dt=0.05, sigma_mb=10.0, steps=100)
RIEMANN_16M = dict(name="riemann-1d-16M", n=16_000_000, n_cells=2000, dt=0.0025, sigma_mb=10.0, steps=500)


def hotspot_3d(n_particles, cells_per_axis, dt, sigma_mb, L=12.8, T0=0.4, dT=0.2, width=1.0):
    """3D thermal box with a Gaussian hot spot, T(r) = T0 + dT exp(-r^2/2w^2)
    about the centre, density ∝ T^3.  N_test from the physical number
    g/(pi^2 (hbar c)^3) ∫ T(r)^3 dV, the integral in closed form (the Gaussian
    terms lie well inside the box)."""
    Z = T0 ** 3 * L ** 3
    for k, c in ((1, 3), (2, 3), (3, 1)):
        Z += c * T0 ** (3 - k) * dT ** k * (2 * math.pi * width * width / k) ** 1.5
    n_phys = GLUON_DOF * Z / (math.pi ** 2 * HBARC_GEV_FM ** 3)
    return dict(L=(L, L, L), n_cells=(cells_per_axis,) * 3, dt=dt, sigma_fm2=sigma_mb * FM2_PER_MB,
                n_test=n_particles / n_phys, n=n_particles, T0=T0, dT=dT, width=width)


def hotspot_state(n, cfg, seed, dtype=np.float64, chunk=1 << 24):
    """(6, n) state of the hot-spot box: positions uniform in the box, kept
    with probability (T(r) / T_max)^3 (density ∝ T^3), then a massless
    Boltzmann energy E ~ Gamma(3, T(r)) and an isotropic direction."""
    rng = np.random.default_rng(seed)
    L = np.asarray(cfg["L"], dtype=np.float64)
    T0, dT, w = cfg["T0"], cfg["dT"], cfg["width"]
    tmax = T0 + dT
    st = np.empty((6, n), dtype=np.float64)
    k = 0
    while k < n:
        x = rng.uniform(0.0, 1.0, (3, chunk)) * L[:, None]
        r2 = ((x - 0.5 * L[:, None]) ** 2).sum(axis=0)
        T = T0 + dT * np.exp(-r2 / (2.0 * w * w))
        keep = rng.uniform(0.0, 1.0, chunk) < (T / tmax) ** 3
        m = min(int(keep.sum()), n - k)
        st[:3, k:k + m] = x[:, keep][:, :m]
        Tk = T[keep][:m]
        E = rng.gamma(3.0, Tk)
        ct = rng.uniform(-1.0, 1.0, m)
        phi = rng.uniform(0.0, 2.0 * math.pi, m)
        s = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
        st[3, k:k + m] = E * s * np.cos(phi)
        st[4, k:k + m] = E * s * np.sin(phi)
        st[5, k:k + m] = E * ct
        k += m
    return st.astype(dtype)


HOTSPOT_64M = dict(name="hotspot-3d-64M", n=64_000_000, cells=128, dt=0.01, sigma_mb=5.0, steps=200)
