"""Pins the oracle's Philox4x32-10 to a library implementation.

cuRAND's host-side generator (CURAND_RNG_PSEUDO_PHILOX4_32_10) runs on the CPU
without a GPU; its output stream is block j = philox(ctr = (0, 0, j_lo, j_hi),
key = (seed_lo, seed_hi)), four words per block.  The oracle must reproduce it
word for word for any seed.
"""
import ctypes
import os

import numpy as np
import pytest

from oracle import oracle as O

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so.10", "libcurand.so", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def _curand_stream(L, seed, nwords):
    g = ctypes.c_void_p()
    if L.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(nwords, np.uint32)
        assert L.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
    finally:
        L.curandDestroyGenerator(g)
    return out


@pytest.mark.parametrize("seed", [0, 1, 42, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF, 0xDEADBEEF00000000])
def test_philox_matches_curand_host_generator(seed):
    L = _curand()
    if L is None:
        pytest.skip("libcurand not found")
    blocks = 257
    ref = _curand_stream(L, seed, 4 * blocks)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(blocks):
        got = O.philox4x32_10([0, 0, j & 0xFFFFFFFF, j >> 32], key)
        assert np.array_equal(got, ref[4 * j:4 * j + 4]), (seed, j)


def test_philox_words_are_uniform():
    # chi-square on the top byte of 4 * 4096 words over varied counters
    words = np.concatenate([O.philox4x32_10([i, 7 * i + 1, i >> 3, 5], [11, 13]) for i in range(4096)])
    hist = np.bincount(words >> 24, minlength=256)
    from scipy import stats
    assert stats.chisquare(hist).pvalue > 1e-4
