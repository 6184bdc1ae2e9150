"""Pins of the oracle's Philox4x32-10 against an independent implementation,
cuRAND's host-side Philox4x32-10 generator (libcurand, run on the CPU).

Seeded with s, cuRAND's generator keys Philox with (s mod 2^32, s >> 32); a
generator offset of 4b words starts its output at block b, and block b is
Philox at counter (b >> 16 mod 2^32, b >> 48, b mod 2^16, 0) in its default
ordering (65536 interleaved subsequences), as observed from its output.
Random keys and offsets therefore cover every key bit, counter words 0 and 2
and the low 14 bits of word 1; all four words are covered on the GPU
(tests/test_gpu_rng.py) by cuRAND's device block function.
"""
import ctypes as C
import ctypes.util
import os

import numpy as np
import pytest

_PHILOX4_32_10 = 161  # curandRngType_t CURAND_RNG_PSEUDO_PHILOX4_32_10


def _libcurand():
    for name in (ctypes.util.find_library("curand"), "/usr/local/cuda/lib64/libcurand.so",
                 "/usr/local/cuda/lib64/libcurand.so.10"):
        if name and (os.path.exists(name) or not name.startswith("/")):
            try:
                return C.CDLL(name)
            except OSError:
                continue
    pytest.skip("libcurand not found")


def _curand_blocks(lib, seed, first_block, n_blocks):
    gen = C.c_void_p()
    assert lib.curandCreateGeneratorHost(C.byref(gen), _PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, C.c_ulonglong(4 * first_block)) == 0
        out = (C.c_uint32 * (4 * n_blocks))()
        assert lib.curandGenerate(gen, out, C.c_size_t(4 * n_blocks)) == 0
        return np.frombuffer(out, np.uint32).reshape(-1, 4).copy()
    finally:
        lib.curandDestroyGenerator(gen)


def _counter(b):
    return [(b >> 16) & 0xFFFFFFFF, b >> 48, b & 0xFFFF, 0]


def test_philox_matches_curand(orc):
    lib = _libcurand()
    rng = np.random.default_rng(5)
    seeds = [0, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF] + [int(x) for x in rng.integers(0, 2 ** 63, 5)]
    for seed in seeds:
        key = [seed & 0xFFFFFFFF, seed >> 32]
        # a run of consecutive blocks from block 0 (counters (0, 0, j, 0) then (1, 0, j, 0))
        got = _curand_blocks(lib, seed, 0, 70000)
        for b in [0, 1, 2, 65535, 65536, 65537, 69999] + [int(x) for x in rng.integers(0, 70000, 200)]:
            assert np.array_equal(got[b], orc.philox(_counter(b), key)), (hex(seed), b)
        # single blocks at random offsets: counter words 0 and 1 far from zero
        # (the offset counts 32-bit words in 64 bits, so blocks stay below 2^62)
        for b in [(1 << 48) + 5, (1 << 62) - 1] + [int(x) for x in rng.integers(0, 2 ** 62, 20)]:
            one = _curand_blocks(lib, seed, b, 1)[0]
            assert np.array_equal(one, orc.philox(_counter(b), key)), (hex(seed), hex(b))


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
