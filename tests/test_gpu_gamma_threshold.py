"""The FP64 threshold of the FP32 kinematics (FP64 only for CM
boosts above a stated Lorentz factor).  Pairs with a chosen CM gamma are
boosted by the device's FP32 path with no FP64 fallback and compared with the
oracle's FP64 kinematics on the same (float-rounded) momenta.  Relative to
the pair energy the error grows about like gamma eps_32 (the parity bar is
1e-5 of the pair energy); relative to a particle's own energy it grows like
gamma^2 eps_32 (the soft backward particle of a fast pair).  The library's
threshold (8) keeps both below 1e-5 for every pair it boosts in FP32; the
sweep prints both errors per gamma (run with -s)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba

pytestmark = pytest.mark.gpu

KEY = 0x5EED


def _pairs(gamma, n, rng):
    """n pairs of equal energies with CM Lorentz factor gamma, random orientation."""
    ct = 1.0 - 2.0 / gamma ** 2          # opening angle: gamma^2 = 2 / (1 - cos)
    th = math.acos(max(-1.0, min(1.0, ct)))
    out = np.zeros((n, 6))
    for k in range(n):
        E = rng.uniform(0.1, 2.0)
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        b = rng.normal(size=3)
        b -= a * (a @ b)
        b /= np.linalg.norm(b)
        out[k, :3] = E * a
        out[k, 3:] = E * (math.cos(th) * a + math.sin(th) * b)
    return out.astype(np.float32)


def _errors(pin, gamma_fp64):
    import torch
    n = len(pin)
    d_in = torch.from_numpy(pin).cuda()
    d_out = torch.zeros_like(d_in)
    d_u = torch.zeros(n, dtype=torch.int32, device="cuda")
    cuba.cuba_kinematics_fp32(d_in, n, KEY, 3, gamma_fp64, d_out, d_u)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().astype(np.float64)
    used = d_u.cpu().numpy()
    err_pair = np.zeros(n)
    err_own = np.zeros(n)
    for k in range(n):
        pi, pj = pin[k, :3].astype(np.float64), pin[k, 3:].astype(np.float64)
        ok, a, b = O.kinematics([KEY & 0xFFFFFFFF, KEY >> 32], 3, 0, 2 * k, 2 * k + 1, pi, pj)
        s = np.linalg.norm(pi) + np.linalg.norm(pj)
        da, db = np.abs(got[k, :3] - a).max(), np.abs(got[k, 3:] - b).max()
        err_pair[k] = max(da, db) / s
        err_own[k] = max(da / np.linalg.norm(a), db / np.linalg.norm(b))
    return err_pair, err_own, used


def test_fp32_kinematics_error_and_default_threshold():
    rng = np.random.default_rng(1)
    gammas = [1.05, 2.0, 4.0, 8.0, 16.0, 64.0, 256.0, 1024.0]
    worst = {}
    for g in gammas:
        ep, eo, used = _errors(_pairs(g, 400, rng), 1e30)   # FP32 always
        assert not used.any()
        worst[g] = (ep.max(), eo.max())
        print("gamma %8.2f  max err / pair energy %.3e  max err / own energy %.3e" % (g, ep.max(), eo.max()))
    # the per-particle error grows with gamma: it crosses 1e-5 above the default
    assert worst[8.0][1] < 1e-5 and worst[1024.0][1] > 1e-5
    assert worst[1024.0][0] > worst[2.0][0]
    # with the default threshold every pair meets both bars
    for g in gammas:
        ep, eo, used = _errors(_pairs(g, 200, rng), 8.0)
        assert ep.max() < 1e-5 and eo.max() < 1e-5, (g, ep.max(), eo.max())
        if g != 8.0:
            assert used.all() == (g > 8.0)
