"""The library's device Philox4x32-10 against the oracle's (bit-exact, all four
counter words and both key words) and against cuRAND's device generator,
whose curand_init(seed, subsequence, offset) starts at counter
(offset/4 low, offset/4 high, subsequence low, subsequence high).  Together
with the CPU pin of the oracle against cuRAND's host generator this fixes
every counter word of the generator both sides use."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _curand_ref():
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libcurand_ref.so")
    src = os.path.join(HERE, "helpers", "curand_ref.cu")
    if not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler",
                        "-fPIC", "-o", lib, src], check=True)
    L = ctypes.CDLL(lib)
    L.curand_ref_philox.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_void_p]
    return L


def test_device_philox_matches_oracle_bit_exact():
    import torch
    rng = np.random.default_rng(0)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0x80000000, 5, 6, 0x40000007]]
    for key in (0, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF):
        d_ctr = torch.from_numpy(np.ascontiguousarray(ctr).view(np.int32)).cuda()
        d_out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
        cuba.cuba_philox(d_ctr, n, key, d_out)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().astype(np.uint32)
        kk = [key & 0xFFFFFFFF, key >> 32]
        for k in list(range(16)) + list(range(16, n, 97)):
            assert list(got[k]) == list(O.philox(ctr[k], kk)), k


def test_device_philox_matches_curand_device_api():
    import torch
    L = _curand_ref()
    rng = np.random.default_rng(1)
    n = 512
    sub = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    off = (rng.integers(0, 2 ** 61, size=n, dtype=np.uint64) // 4) * 4
    seed = 0x1234_5678_9ABC_DEF0
    d_sub = torch.from_numpy(sub.view(np.int64)).cuda()
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    d_ref = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    assert L.curand_ref_philox(seed, d_sub.data_ptr(), d_off.data_ptr(), n, d_ref.data_ptr()) == 0
    ref = d_ref.cpu().numpy().astype(np.uint32)
    q = off // 4
    ctr = np.stack([q & 0xFFFFFFFF, q >> 32, sub & 0xFFFFFFFF, sub >> 32], axis=1).astype(np.uint32)
    d_ctr = torch.from_numpy(np.ascontiguousarray(ctr).view(np.int32)).cuda()
    d_out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    cuba.cuba_philox(d_ctr, n, seed, d_out)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().astype(np.uint32)
    assert np.array_equal(got, ref)
