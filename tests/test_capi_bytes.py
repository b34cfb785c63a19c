"""cuba_batch_bytes and cuba_sim_bytes cover every buffer a simulation or a
batch allocates (pure arithmetic: no GPU needed).

The buffers, restated from the arena's data layout: two SoA state copies
(6 components), keys and permutation ping-pong (4 B each, two copies), per
cell start/work/skip/accept-count/active tables, the radix histograms (two
2048-entry rows per 4096-particle tile, plus one tile), the scan scratch
(at least the 2 x 512 + 1 rows of 2048 words the digit scan uses), counters,
the byte-filter survivor list (16 B x max(2^21, particles / 2)), the greedy
bitmap, the neighbour-move tables (27 + 1 words per cell, arenas of more
than 2048 cells), per-simulation counters and descriptors (a descriptor is
more than its 33-entry skip-ahead table of 8-byte words), the observables
scratch (20 B per cell) and totals, and the smallest accepted-pair list
(2^20 entries of 8 B).
"""
import pytest

from paper_1208_0961_gb300 import cuba

TILE = 4096
BINS = 2048


def _restated(precision, P, Cc, S):
    es = 8 if precision == cuba.CUBA_FP64 else 4
    b = 2 * 6 * P * es                      # state ping-pong
    b += 2 * 4 * P + 2 * 4 * P              # keys, permutation
    b += (Cc + 1) * (4 + 8 + 4) + 2 * 4 * Cc  # cell_start, work, skip work, acc count, active
    b += 4 * 2 * BINS * ((P + TILE - 1) // TILE + 1)
    b += 4 * (2 * 512 + 1) * BINS           # digit-scan scratch
    b += 64                                 # counters
    b += 16 * max(1 << 21, P // 2)          # survivors
    b += 4 * (P // 32 + 2)                  # greedy bitmap
    if Cc > BINS:
        b += 4 * 27 * Cc + 4 * (Cc + 1)     # neighbour-move tables
    b += S * (8 * 8 + 33 * 8)               # counters and descriptors (lower bound)
    b += 20 * Cc + 64 + 64                  # observables, totals
    b += 8 * (1 << 20)                      # smallest accepted list
    return b


@pytest.mark.parametrize("precision,P,Cc,S", [
    (cuba.CUBA_FP32, 1, 1, 1),
    (cuba.CUBA_FP32, 16_000_000, 2000, 1),
    (cuba.CUBA_FP64, 20_000, 100, 1),
    (cuba.CUBA_FP32, 64_000_000, 128 ** 3, 1),           # neighbour tables, survivors P / 2
    (cuba.CUBA_FP32, 300_000_000, 600_000, 256),          # ensemble-sized batch
    (cuba.CUBA_FP64, 5_000_000, 3000, 17),
])
def test_batch_bytes_cover_every_buffer(precision, P, Cc, S):
    cfg = cuba.make_batch_config(precision, max_sims=S, max_particles=P, max_cells=Cc)
    got = cuba.cuba_batch_bytes(cfg)
    need = _restated(precision, P, Cc, S)
    assert got >= need
    # and not wildly above it: the restatement misses only scan padding and
    # the descriptors' other fields
    assert got <= need + 4 * 1024 * 1024 + S * 1024


def test_sim_bytes_match_a_one_member_batch():
    p = cuba.make_params(L=(10.0, 1.0, 1.0), n_cells=(2000, 1, 1), dt=0.0025, sigma_fm2=1.0, n_test=156732.0,
                         precision=cuba.CUBA_FP32)
    cfg = cuba.make_batch_config(cuba.CUBA_FP32, max_sims=1, max_particles=16_000_000, max_cells=2000)
    assert cuba.cuba_sim_bytes(p, 16_000_000) == cuba.cuba_batch_bytes(cfg)
    assert cuba.cuba_sim_bytes(p, 16_000_000) >= _restated(cuba.CUBA_FP32, 16_000_000, 2000, 1)


def test_bytes_reject_invalid_arguments():
    cfg = cuba.make_batch_config(cuba.CUBA_FP32, max_sims=0, max_particles=10, max_cells=10)
    assert cuba.cuba_batch_bytes(cfg) == -1
    p = cuba.make_params(L=(1, 1, 1), n_cells=(10, 1, 1), dt=0.2)  # dt above the cell edge
    assert cuba.cuba_sim_bytes(p, 10) == -1
