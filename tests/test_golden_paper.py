"""Values the paper prints (tests/golden/paper_numbers.txt, Secs. 5-6).

The cross section of the first run is quoted in GeV^-2; converting it with
hbar c gives 0.3894 fm^2 = 3.894 mb, the unit the oracle and library use.  The
two quoted run times give the quoted speed-up of about 13.
"""
import os

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_numbers.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, _unit = line.split(None, 2)
            vals[name] = float(value)
    return vals


def test_cross_section_units():
    g = _golden()
    sigma_fm2 = g["sigma_gev_minus2"] * O.HBARC_GEV_FM ** 2
    assert abs(sigma_fm2 - 0.38938) < 1e-4
    assert abs(sigma_fm2 / O.FM2_PER_MB - 3.8938) < 1e-3


def test_quoted_speedup():
    g = _golden()
    assert round(g["bamps_seconds"] / g["cuba_seconds"]) == g["speedup_about"]


def test_paper_first_run_is_valid_input():
    """dt = 0.1 fm/c must stay below the cell size (Sec. 5); with the quoted
    box and temperatures the oracle accepts a 32-cell grid and rejects dt >= dx."""
    g = _golden()
    L = g["box_edge"]
    ok = O.make_params(L=(L, L, L), n=(32, 1, 1), dt=g["dt_fm"], sigma_fm2=0.389, n_test=10.0)
    assert O.p22_scale(ok) > 0
    bad = O.make_params(L=(L, L, L), n=(320, 1, 1), dt=g["dt_fm"], sigma_fm2=0.389, n_test=10.0)
    import numpy as np
    import pytest
    with pytest.raises(ValueError):
        O.keys(bad, np.zeros((6, 1)))
