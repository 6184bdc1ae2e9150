"""Pins of the oracle's Philox4x32-10 against published known-answer vectors."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_counter_sensitivity(orc):
    # every counter and key word feeds the output (a dropped word would leave it unchanged)
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for pos in range(6):
        ctr = [1, 2, 3, 4]
        key = [5, 6]
        if pos < 4:
            ctr[pos] ^= 1
        else:
            key[pos - 4] ^= 1
        out = orc.philox(ctr, key)
        assert np.count_nonzero(out != base) == 4


def test_philox_uniformity(orc):
    # 2^14 blocks: the top byte of each word is uniform (chi^2, 255 dof)
    from scipy import stats
    words = np.array([orc.philox([i, 7, 0x02000003, 11], [123, 456]) for i in range(1 << 14)]).reshape(-1)
    hist = np.bincount(words >> 24, minlength=256)
    assert stats.chisquare(hist).pvalue > 1e-4


def test_series_sincos_against_libm(orc):
    """The Maclaurin-series sin/cos used for Metropolis steps and initial spins
    agrees with libm to 2e-15 absolute on [-pi, pi] and is exact at 0."""
    xs = np.concatenate([np.linspace(-np.pi, np.pi, 4001), [0.0, 1e-8, -1e-8, np.pi, -np.pi]])
    worst = 0.0
    for x in xs:
        sn, cs = orc.sincos_series(x)
        worst = max(worst, abs(sn - np.sin(x)), abs(cs - np.cos(x)))
    assert worst < 2e-15
    assert orc.sincos_series(0.0) == (0.0, 1.0)
