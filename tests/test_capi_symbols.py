"""The C-ABI library loads without a GPU and exports every entry point that
include/cuba.h declares; the binding's struct layouts match the header."""
import ctypes
import os
import re
import subprocess

import pytest

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


def test_struct_sizes_match_header_layout(tmp_path):
    # the C compiler's layout of the header's structs against the binding's
    structs = {"cuba_params": cuba.cuba_params, "cuba_region": cuba.cuba_region,
               "cuba_counters": cuba.cuba_counters, "cuba_batch_config": cuba.cuba_batch_config,
               "cuba_allocator": cuba.cuba_allocator}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cuba.h"', 'int main(void) {']
    for name, ct in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in ct._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name, ct in structs.items():
        assert int(got[name]) == ctypes.sizeof(ct), name
        for f, _ in ct._fields_:
            assert int(got["%s.%s" % (name, f)]) == getattr(ct, f).offset, (name, f)


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


@pytest.mark.parametrize("kw,code,msg", [
    (dict(dt=-0.01), "CUBA_ERR_INVALID", "dt must be > 0"),
    (dict(sigma_fm2=-1.0), "CUBA_ERR_INVALID", "sigma"),
    (dict(sigma_fm2=float("nan")), "CUBA_ERR_INVALID", "sigma"),
    (dict(n_test=0.0), "CUBA_ERR_INVALID", "n_test"),
    (dict(kappa=0.6), "CUBA_ERR_INVALID", "kappa"),
    (dict(mass=-0.1), "CUBA_ERR_INVALID", "mass"),
    (dict(mu=-0.1), "CUBA_ERR_INVALID", "mu"),
    (dict(n_cells=(0, 1, 1)), "CUBA_ERR_INVALID", "n_cells"),
    (dict(L=(0.0, 1.0, 1.0)), "CUBA_ERR_INVALID", "L[0]"),
    (dict(acceptance=7), "CUBA_ERR_INVALID", "acceptance"),
    (dict(precision=3), "CUBA_ERR_INVALID", "precision"),
    # 2C = 1.0 exactly is allowed for the all-pairs test (P22 <= 2C), but
    # skip-ahead needs 2.0001 C < 1
    (dict(sigma_fm2=5.0, n_test=1.0, acceptance=1), "CUBA_ERR_P22", "skip-ahead"),
])
def test_parameter_validation_without_a_gpu(kw, code, msg):
    # every check runs in parameter validation, before any CUDA call
    args = dict(L=(1.0, 1.0, 1.0), n_cells=(10, 1, 1), dt=0.01, sigma_fm2=1.0, n_test=1.0)
    args.update(kw)
    p = cuba.make_params(**args)
    with pytest.raises(cuba.CubaError) as e:
        cuba.cuba_create(p, 10)
    assert e.value.code == getattr(cuba, code)
    assert msg in cuba.cuba_last_error()
