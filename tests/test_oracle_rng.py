"""Pins for the oracle's Philox4x32-10 (the counter-based generator that both the
oracle and the CUDA path implement from its published definition).

The pin is cuRAND's host-side PHILOX4_32_10 generator, run here on the CPU.  Its
output word i with seed s and offset o is word (o+i) % 4 of the Philox block with
key (s lo, s hi) and counter (C lo, C hi, j, 0), where the block index
(o+i)//4 = C * 65536 + j.  This covers counter words 0, 1 and 2 and both key words.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = [ctypes.util.find_library("curand"), "/usr/local/cuda/lib64/libcurand.so",
             "/usr/local/cuda/lib64/libcurand.so.10"]
    cands += [os.path.join(d, "libcurand.so") for d in ("/usr/local/cuda/targets/sbsa-linux/lib",
                                                         "/usr/local/cuda/targets/x86_64-linux/lib")]
    for c in cands:
        if c and os.path.exists(c) or (c and not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    pytest.skip("libcurand not found")


def _host_philox(lib, seed, n, offset):
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_first_blocks(orc, seed):
    lib = _curand()
    out = _host_philox(lib, seed, 4 * 64, 0).reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(64):
        np.testing.assert_array_equal(orc.philox([0, 0, j, 0], key), out[j])


@pytest.mark.parametrize("C,j", [(1, 0), (3, 7), (1 << 32, 0), ((1 << 32) + 5, 9), ((7 << 32) + 0xFFFFFFFF, 65535)])
def test_philox_matches_curand_high_counter_words(orc, C, j):
    lib = _curand()
    seed = 0x0F1E2D3C4B5A6978
    offset = 4 * (C * 65536 + j)
    out = _host_philox(lib, seed, 4, offset)
    ctr = [C & 0xFFFFFFFF, C >> 32, j, 0]
    np.testing.assert_array_equal(orc.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32]), out)


def test_philox_words_uniform(orc):
    """Chi-square of the top 6 bits of 40000 words over counters (c0, sweep, walker, tag)."""
    words = []
    for w in range(100):
        for c0 in range(100):
            words.extend(orc.philox([c0, 5, w, 1], [12345, 678]))
    words = np.array(words, dtype=np.uint64)
    counts = np.bincount((words >> 26).astype(np.int64), minlength=64)
    exp = words.size / 64
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 120  # 63 dof: p < 1e-5 above this
    # distinct tags give distinct streams
    assert not np.array_equal(orc.philox([0, 0, 0, 0], [1, 2]), orc.philox([0, 0, 0, 1], [1, 2]))
