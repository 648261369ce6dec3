"""Pins of the oracle's Philox4x32-10 generator against cuRAND's host generator
(a library implementation of the same published algorithm), and of the
uniform-variate mapping."""
import ctypes
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O

CURAND = "/usr/local/cuda/lib64/libcurand.so"


@pytest.mark.skipif(not os.path.exists(CURAND), reason="cuRAND not installed")
@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's host Philox4_32_10 generator at offset 0 emits block i as
    philox(counter = (0, 0, i, 0), key = (seed lo, seed hi))."""
    cr = ctypes.CDLL(CURAND)
    gen = ctypes.c_void_p()
    assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4096, np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        cr.curandDestroyGenerator(gen)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for i in range(0, 1024, 7):
        assert O.philox4x32_10((0, 0, i, 0), key) == tuple(int(v) for v in out[4 * i:4 * i + 4])


def test_uniforms_are_24_bit_and_uniform():
    u = np.array([O.uniform(7, p, s, slot) for p in range(50) for s in range(20) for slot in range(20)])
    assert np.all((u >= 0) & (u < 1))
    assert np.all(u * 2 ** 24 == np.floor(u * 2 ** 24))
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    # distinct streams per pixel, sample and slot
    assert len(np.unique(u)) > 0.99 * len(u)
