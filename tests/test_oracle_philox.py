"""Pins the oracle's Philox4x32-10 to two library implementations.

cuRAND's host-side generator (CURAND_RNG_PSEUDO_PHILOX4_32_10) runs on the CPU
without a GPU; its output stream is block j = philox(ctr = (0, 0, j_lo, j_hi),
key = (seed_lo, seed_hi)), four words per block.  The oracle must reproduce it
word for word for any seed.  cuRAND's stream leaves counter words 0 and 1 at
zero, so a second reference covers all four: Triton's philox (its language
library, run by its CPU interpreter) with random counters and keys.
"""
import ctypes
import json
import os
import subprocess
import sys
import textwrap

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


_TRITON_PHILOX = textwrap.dedent("""
    import json, sys
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, out_ptr, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c_ptr + 4 * i), tl.load(c_ptr + 4 * i + 1),
                               tl.load(c_ptr + 4 * i + 2), tl.load(c_ptr + 4 * i + 3))
        tl.store(out_ptr + 4 * i, a)
        tl.store(out_ptr + 4 * i + 1, b)
        tl.store(out_ptr + 4 * i + 2, c)
        tl.store(out_ptr + 4 * i + 3, d)

    job = json.load(sys.stdin)
    res = []
    for seed, ctrs in job:
        c = torch.from_numpy(np.array(ctrs, np.uint32).view(np.int32).copy())
        out = torch.zeros_like(c)
        k[(1,)](c, out, seed, N=c.shape[0])
        res.append(out.numpy().view(np.uint32).tolist())
    json.dump(res, sys.stdout)
""")


def test_philox_matches_triton_on_all_counter_words():
    pytest.importorskip("triton")
    g = np.random.default_rng(2024)
    seeds = [0, 1, 0xFFFFFFFFFFFFFFFF, int(g.integers(0, 2**63)) * 2 + 1]
    job = [[s, g.integers(0, 2**32, (64, 4), dtype=np.uint64).tolist()] for s in seeds]
    job[0][1][0] = [0, 0, 0, 0]
    job[1][1][0] = [0xFFFFFFFF] * 4
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=json.dumps(job), capture_output=True, text=True,
                       env=env, timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + r.stderr.strip().splitlines()[-1][:200])
    ref = json.loads(r.stdout)
    for (seed, ctrs), words in zip(job, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for c, w in zip(ctrs, words):
            assert np.array_equal(O.philox4x32_10(c, key), np.array(w, np.uint32)), (seed, c)
