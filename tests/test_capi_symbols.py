"""The C-ABI library loads without a GPU and exports every entry point that
include/cuba.h declares; the binding's struct layouts match the header."""
import ctypes
import os
import re

from paper_1208_0961_gb300 import cuba

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "cuba.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(cuba_[a-z0-9_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    lib = cuba.load()
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match_header_layout():
    # cuba_params: 3 doubles, 3 int32 (+4 pad), 3 doubles, int32 (+4 pad), uint64, double
    assert ctypes.sizeof(cuba.cuba_params) == 24 + 16 + 24 + 8 + 8 + 8
    assert ctypes.sizeof(cuba.cuba_region) == 56
    assert ctypes.sizeof(cuba.cuba_counters) == 64


def test_invalid_parameters_are_rejected_without_a_gpu():
    # dt >= dx and sigma < 0 fail in parameter validation, before any CUDA call
    p = cuba.make_params(L=(1, 1, 1), n_cells=(10, 1, 1), dt=0.2)
    try:
        cuba.cuba_create(p, 10)
        raised = None
    except cuba.CubaError as e:
        raised = e
    assert raised is not None and raised.code == cuba.CUBA_ERR_INVALID
    assert "cell edge" in cuba.cuba_last_error()
    p = cuba.make_params(L=(1, 1, 1), n_cells=(2, 1, 1), dt=0.1, sigma_fm2=100.0, n_test=1.0)
    try:
        cuba.cuba_create(p, 10)
        raised = None
    except cuba.CubaError as e:
        raised = e
    assert raised is not None and raised.code == cuba.CUBA_ERR_P22
