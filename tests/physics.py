"""Closed-form physics used to pin the oracle (no code shared with it).

* Free streaming of a massless gas with isotropic momenta between specular
  walls: the exact solution of the collisionless Boltzmann equation, obtained
  by unfolding the box into its even, 2L-periodic extension (method of
  images).  For the 1D Riemann initial condition it reduces, away from the
  walls, to eps = eps_R + (eps_L - eps_R) (1 - xi) / 2 and
  T0x = (eps_L - eps_R) (1 - xi^2) / 4 with xi = (x - L/2) / t.
* The ideal-fluid (eps = 3P, c_s^2 = 1/3) Riemann problem: left rarefaction,
  plateau, right-moving shock, from the Riemann invariant and the
  energy-momentum jump conditions.  This is the large-sigma limit of the
  transport solution (Results section, Figs. 2-3).
"""
import math

import numpy as np
from scipy.optimize import brentq

CS = 1.0 / math.sqrt(3.0)


def fold(X, L):
    """Position in [0, L] of an unfolded coordinate of the even 2L-periodic extension."""
    Y = np.mod(X, 2.0 * L)
    return np.where(Y > L, 2.0 * L - Y, Y)


def free_stream_profile(edges, t, L, eps0, nmu=4001, nsub=16):
    """Cell averages of T00 and T0x at time t of a collisionless massless gas.

    eps0: callable giving the initial energy density at positions in [0, L];
    the momentum distribution is isotropic everywhere.  The direction cosine
    mu = p_x / E is uniform on [-1, 1], so
        T00(x, t) = 1/2 int dmu eps0_ext(x - mu t),
        T0x(x, t) = 1/2 int dmu mu eps0_ext(x - mu t),
    with eps0_ext the even 2L-periodic extension.  Averages over each cell use
    nsub sample points; the mu integral uses the trapezoid rule.
    """
    mu = np.linspace(-1.0, 1.0, nmu)
    w = np.full(nmu, 2.0 / (nmu - 1))
    w[0] *= 0.5
    w[-1] *= 0.5
    T00 = np.zeros(len(edges) - 1)
    T0x = np.zeros(len(edges) - 1)
    for c in range(len(edges) - 1):
        xs = edges[c] + (np.arange(nsub) + 0.5) / nsub * (edges[c + 1] - edges[c])
        src = fold(xs[:, None] - mu[None, :] * t, L)
        e = eps0(src)
        T00[c] = np.mean(0.5 * (e * w[None, :]).sum(axis=1))
        T0x[c] = np.mean(0.5 * (e * (mu * w)[None, :]).sum(axis=1))
    return T00, T0x


def _fluid_T(eps, v):
    g2 = 1.0 / (1.0 - v * v)
    T00 = 4.0 / 3.0 * eps * g2 - eps / 3.0
    T0x = 4.0 / 3.0 * eps * g2 * v
    Txx = 4.0 / 3.0 * eps * g2 * v * v + eps / 3.0
    return T00, T0x, Txx


def rarefaction_eps(eps_l, v):
    """Energy density on the left simple wave: eps_L ((1-v)/(1+v))^(2/sqrt 3)."""
    return eps_l * ((1.0 - v) / (1.0 + v)) ** (2.0 / math.sqrt(3.0))


def ideal_riemann(eps_l, eps_r):
    """Plateau (eps*, v*) and shock speed of the ideal conformal-fluid Riemann problem."""
    if eps_l <= eps_r:
        raise ValueError("expects eps_l > eps_r")

    def mismatch(v):
        e = rarefaction_eps(eps_l, v)
        T00, T0x, Txx = _fluid_T(e, v)
        return T0x * T0x - (T00 - eps_r) * (Txx - eps_r / 3.0)

    # The plateau of a compressive shock lies between eps_r and eps_l: bracket
    # v* between 0 (eps* = eps_l, mismatch < 0) and the velocity at which the
    # rarefaction reaches eps_r (mismatch > 0 there).
    r = (eps_r / eps_l) ** (math.sqrt(3.0) / 2.0)
    v_max = (1.0 - r) / (1.0 + r)
    v = brentq(mismatch, 1e-14, v_max, xtol=1e-15)
    e = rarefaction_eps(eps_l, v)
    T00, T0x, _ = _fluid_T(e, v)
    vsh = T0x / (T00 - eps_r)
    return e, v, vsh


def ideal_profile(xi, eps_l, eps_r):
    """(eps, v, T00, T0x) of the self-similar ideal solution at xi = (x - x0)/t."""
    e_s, v_s, vsh = ideal_riemann(eps_l, eps_r)
    xi_tail = (v_s - CS) / (1.0 - v_s * CS)
    xi = np.asarray(xi, dtype=float)
    eps = np.empty_like(xi)
    vel = np.empty_like(xi)
    left = xi < -CS
    fan = (xi >= -CS) & (xi < xi_tail)
    plat = (xi >= xi_tail) & (xi < vsh)
    right = xi >= vsh
    eps[left] = eps_l
    vel[left] = 0.0
    vf = (xi[fan] + CS) / (1.0 + xi[fan] * CS)
    vel[fan] = vf
    eps[fan] = rarefaction_eps(eps_l, vf)
    eps[plat] = e_s
    vel[plat] = v_s
    eps[right] = eps_r
    vel[right] = 0.0
    T00, T0x, _ = _fluid_T(eps, vel)
    return eps, vel, T00, T0x


def gamma3_cdf(x):
    """CDF of E/T for a massless Boltzmann gas (Gamma(3, 1)): 1 - e^-x (1 + x + x^2/2)."""
    x = np.asarray(x, dtype=float)
    return 1.0 - np.exp(-x) * (1.0 + x + 0.5 * x * x)
