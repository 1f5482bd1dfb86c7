"""Pins for the oracle's Philox4x32-10 (Salmon et al., SC'11).

The reference is cuRAND's host-side PHILOX4_32_10 generator, run through its
public API (outputs only): with seed s its output block b (four words) is the
Philox block of counter (b >> 16, 0, b & 0xffff, 0) under key (lo32 s, hi32 s).
"""
import ctypes as C

import numpy as np
import pytest

from oracle import ctaux


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 985456376, 0x0123456789ABCDEF])
def test_philox_matches_curand_host_generator(seed):
    L = _curand()
    if L is None:
        pytest.skip("libcurand not available")
    gen = C.c_void_p()
    assert L.curandCreateGeneratorHost(C.byref(gen), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        n = 4 * (2 * 65536 + 64)
        buf = np.zeros(n, np.uint32)
        assert L.curandGenerate(gen, C.c_void_p(buf.ctypes.data), C.c_size_t(n)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    blocks = buf.reshape(-1, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in list(range(0, 40)) + [65536, 65536 + 7, 131072 + 3]:
        ctr = [b >> 16, 0, b & 0xFFFF, 0]
        assert ctaux.philox4x32_10(ctr, key) == [int(x) for x in blocks[b]], b


def test_philox_is_a_function_of_every_word():
    base = ctaux.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert ctaux.philox4x32_10(c, [5, 6]) != base
    for i in range(2):
        k = [5, 6]
        k[i] ^= 1
        assert ctaux.philox4x32_10([1, 2, 3, 4], k) != base
