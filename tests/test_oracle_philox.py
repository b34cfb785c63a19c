"""Pins of the oracle's Philox4x32-10 and of the pair random word u_ij.

The oracle writes Philox4x32-10 (Salmon et al., SC'11) itself; here it is
checked against an independent implementation, cuRAND's host-side
PHILOX4_32_10 generator (a library routine that runs on the CPU), whose block
k of four outputs is Philox with counter (0, 0, k, 0) and key = the 64-bit
seed split into two words.  That fixes the round function, the multipliers,
the key schedule and counter word 2; the remaining counter words are pinned on
the GPU against cuRAND's device API.  Statistical checks cover the derived
pair word used in the acceptance test (Eq. 3's Monte-Carlo draw).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    return None


CURAND = _curand()


def curand_host(seed, offset, n):
    g = ctypes.c_void_p()
    assert CURAND.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert CURAND.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert CURAND.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        buf = np.zeros(n, dtype=np.uint32)
        assert CURAND.curandGenerate(g, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        CURAND.curandDestroyGenerator(g)
    return buf


@pytest.mark.skipif(CURAND is None, reason="libcurand not found")
@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(seed):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    nb = 2048
    ref = curand_host(seed, 0, 4 * nb).reshape(nb, 4)
    for k in list(range(0, 64)) + list(range(64, nb, 37)):
        assert list(O.philox([0, 0, k, 0], key)) == list(ref[k]), k
    # an offset into the stream: blocks 40000.. of the same generator
    ref2 = curand_host(seed, 4 * 40000, 8).reshape(2, 4)
    assert list(O.philox([0, 0, 40000, 0], key)) == list(ref2[0])
    assert list(O.philox([0, 0, 40001, 0], key)) == list(ref2[1])


def test_philox_counter_words_all_matter():
    """Changing any single counter or key word changes every output word."""
    base = O.philox([1, 2, 3, 4], [5, 6])
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        out = O.philox(c, [5, 6])
        assert np.all(out != base)
    for w in range(2):
        k = [5, 6]
        k[w] ^= 1
        assert np.all(O.philox([1, 2, 3, 4], k) != base)


def test_pair_word_uniform_and_independent():
    """u_ij = r_ij 2^-32 is uniform (KS) and its top byte is uniform (chi^2)."""
    key = [12345, 678]
    words = np.array([O.pair_word(key, 7, c, i, j)
                      for c in range(3) for i in range(40) for j in range(i + 1, 120)],
                     dtype=np.uint64)
    u = words.astype(np.float64) * 2.0 ** -32
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    top = (words >> np.uint64(24)).astype(np.int64)
    counts = np.bincount(top, minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
    # adjacent columns of a row are not correlated
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5.0 / np.sqrt(len(u))


def test_pair_word_structure():
    """Top byte from block (step, cell, i, j/16), next byte from the block
    (step, cell, i, TAG_MID | j/16), low 16 bits from (step, cell, i, TAG_FINE | j)."""
    key = [1, 2]
    w = O.pair_word(key, 3, 4, 5, 37)
    blk = O.philox([3, 4, 5, 37 >> 4], key)
    top = (int(blk[(37 >> 2) & 3]) >> (8 * (37 & 3))) & 0xFF
    mid_blk = O.philox([3, 4, 5, 0x20000000 | (37 >> 4)], key)
    mid = (int(mid_blk[(37 >> 2) & 3]) >> (8 * (37 & 3))) & 0xFF
    fine = O.philox([3, 4, 5, 0x40000000 | 37], key)
    assert (w >> 24) == top
    assert ((w >> 16) & 0xFF) == mid
    assert (w & 0xFFFF) == (int(fine[0]) >> 16)


def test_pair_word_parts_are_independent():
    """Top byte, middle byte and low half of u_ij are uncorrelated."""
    key = [9, 10]
    w = np.array([O.pair_word(key, 1, 2, i, j) for i in range(30) for j in range(i + 1, 200)], dtype=np.uint64)
    top = (w >> np.uint64(24)).astype(float)
    mid = ((w >> np.uint64(16)) & np.uint64(0xFF)).astype(float)
    low = (w & np.uint64(0xFFFF)).astype(float)
    lim = 5.0 / np.sqrt(len(w))
    for a, b in ((top, mid), (top, low), (mid, low)):
        assert abs(np.corrcoef(a, b)[0, 1]) < lim
