"""Pins of the oracle's Philox4x32-10 against sources other than itself:
the published Random123 known-answer vectors and cuRAND's host-side Philox
generator (a library run on the CPU)."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle import estimator as E

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert E.philox4x32_10(ctr, key).tolist() == expect


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10",
                 ctypes.util.find_library("curand")):
        if cand and (os.path.exists(cand) or not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                continue
    return None


def _curand_host_stream(seed: int, offset: int, count: int) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    PHILOX4_32_10 = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10 in curand.h
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4_32_10 lays its output out as 65536 interleaved
    streams: output block b is the Philox block of counter
    (b // 65536, 0, b % 65536, 0) under key (seed_lo, seed_hi).  This pins
    counter words 0 and 2 and both key words; the known-answer vectors pin
    words 1 and 3."""
    streams = 65536
    n_blocks = 2 * streams + 64
    ref = _curand_host_stream(seed, 0, 4 * n_blocks)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in list(range(40)) + [4095, 4096, streams - 1, streams, streams + 1, 2 * streams + 63]:
        ours = E.philox4x32_10([b // streams, 0, b % streams, 0], key)
        assert np.array_equal(ours, ref[4 * b:4 * b + 4]), b
