"""Pins of the oracle's random numbers (the uniform(0,1) draws of Algorithm 1).

Philox4x32-10 is pinned twice, by things other than the oracle itself:
  * the published known-answer vectors (tests/golden/philox4x32_10_kat.txt);
  * curand's host-side Philox4_32_10 generator, run as a black-box library on the
    CPU: block j of seed K is Philox(counter (0, 0, j, 0), key (K lo, K hi)).
The uniform mapping ((x >> 9) * 2 + 1) / 2^24 is pinned by its defining
properties (odd multiples of 2^-24, never 0, 1 or 1/2, exact in FP32).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    seed = key[0] | (key[1] << 32)
    w = oracle.philox_words(seed, ctr[1], ctr[2], ctr[3], ctr[0], 1)[0]
    assert [int(x) for x in w] == expect


def _curand():
    for cand in ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so", ctypes.util.find_library("curand")]:
        if not cand:
            continue
        try:
            return ctypes.CDLL(cand)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFF00000001])
def test_philox_matches_curand_host_generator(seed):
    cur = _curand()
    if cur is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161  # curand.h enum value
    if cur.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("curand host generator unavailable")
    try:
        assert cur.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n_blocks = 64
        out = np.zeros(4 * n_blocks, np.uint32)
        assert cur.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        cur.curandDestroyGenerator(gen)
    for j in range(n_blocks):
        w = oracle.philox_words(seed, 0, j, 0, 0, 1)[0]
        assert list(w) == list(out[4 * j:4 * j + 4]), f"block {j}"


def test_philox_counter_words_all_matter():
    base = oracle.philox_words(7, 1, 2, 3, 0, 1)[0]
    for changed in [oracle.philox_words(7, 1, 2, 3, 1, 1)[0], oracle.philox_words(7, 9, 2, 3, 0, 1)[0],
                    oracle.philox_words(7, 1, 9, 3, 0, 1)[0], oracle.philox_words(7, 1, 2, 9, 0, 1)[0],
                    oracle.philox_words(8, 1, 2, 3, 0, 1)[0], oracle.philox_words(7 | (1 << 40), 1, 2, 3, 0, 1)[0]]:
        assert not np.array_equal(base, changed)


def test_uniform_mapping_properties():
    words = np.array([0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF], np.uint32)
    u = oracle.u01(words)
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24 and u[2] == 2.0 ** -24
    assert u[3] == 3 * 2.0 ** -24
    assert u[-1] == 1.0 - 2.0 ** -24
    assert np.all((u > 0) & (u < 1)) and not np.any(u == 0.5)
    # exact in FP32 and equal to the C implementation
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    for x in words:
        assert oracle.lib().orc_u01(int(x)) == oracle.u01(np.array([x]))[0]
    # uniformity of Philox output through the mapping (chi-square over 64 bins)
    w = oracle.philox_words(3, 0, 0, 0, 0, 1 << 14).reshape(-1)
    counts = np.bincount((oracle.u01(w) * 64).astype(int), minlength=64)
    expected = w.size / 64
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert chi2 < 120.0  # 63 dof: p ~ 2e-5
