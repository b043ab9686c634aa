"""Pins for the oracle's random draws: Philox-4x32-10 against its published known-answer
vectors, and the alpha-initialisation / probe constructions against their definitions'
invariants (range, exactness in FP32, sign balance, independence across counters)."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(v, 16) for v in line.split()]
        yield w[:4], w[4:6], w[6:10]


def test_philox_known_answer_vectors():
    rows = list(_kat_rows())
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = [int(v) for v in philox.philox4x32_10(*ctr, *key)]
        assert got == want, (ctr, key, [hex(v) for v in got])


def test_philox_vectorised_matches_scalar():
    ctr = np.arange(37, dtype=np.uint64)
    out = philox.philox4x32_10(ctr, 5, 7, 9, 11, 13)
    for i in (0, 1, 17, 36):
        one = philox.philox4x32_10(int(ctr[i]), 5, 7, 9, 11, 13)
        assert [int(o[i]) for o in out] == [int(v) for v in one]


def test_alpha_init_open_unit_interval_and_fp32_exact():
    a = philox.alpha_init(1234, 3, 1000)
    assert a.shape == (3, 1000)
    assert np.all(a > 0.0) and np.all(a < 1.0)
    assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
    # clusters get distinct draws; the mean of 3000 uniforms is near 1/2
    assert not np.array_equal(a[0], a[1])
    assert abs(a.mean() - 0.5) < 4 * np.sqrt(1 / 12 / a.size)


def test_alpha_init_seed_high_word_matters():
    a = philox.alpha_init(1, 1, 16)
    b = philox.alpha_init(1 + (1 << 32), 1, 16)
    assert not np.array_equal(a, b)


def test_probes_are_rademacher_and_balanced():
    P = philox.probes(7, 3, 2, 1, 4, 64, 517)          # ragged D, not a multiple of 128
    assert P.shape == (64, 517)
    assert set(np.unique(P)) <= {-1.0, 1.0}
    m = P.mean()
    assert abs(m) < 4 / np.sqrt(P.size)


def test_probes_depend_on_every_counter_field():
    base = philox.probes(7, 3, 2, 1, 4, 4, 256)
    assert not np.array_equal(base, philox.probes(8, 3, 2, 1, 4, 4, 256))   # seed
    assert not np.array_equal(base, philox.probes(7, 4, 2, 1, 4, 4, 256))   # EM iteration
    assert not np.array_equal(base, philox.probes(7, 3, 3, 1, 4, 4, 256))   # task
    assert not np.array_equal(base, philox.probes(7, 3, 2, 2, 4, 4, 256))   # cluster
    assert not np.array_equal(base[0], base[1])                             # probe index
    # coordinates of different 128-blocks come from different counters
    assert not np.array_equal(base[:, :128], base[:, 128:256])


def test_probe_bit_extraction_against_counter_words():
    """Coordinate d takes bit d % 32 of word (d // 32) % 4 of the call with counter d // 128."""
    seed, e, t, c, C = 99, 5, 3, 1, 2
    P = philox.probes(seed, e, t, c, C, 1, 256)[0]
    for d in (0, 31, 32, 77, 127, 128, 255):
        w = philox.philox4x32_10(d // 128, 0, t * C + c, (e << 4) | 1, seed, 0)
        bit = (int(w[(d // 32) % 4]) >> (d % 32)) & 1
        assert P[d] == (1.0 if bit == 0 else -1.0)
