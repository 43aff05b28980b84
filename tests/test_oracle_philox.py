"""Pins of the oracle's Philox-4x32-10 (no GPU)."""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle import philox as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        a, b = line.split(":")
        rows.append(([int(x, 16) for x in a.split()], [int(x, 16) for x in b.split()]))
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for inp, out in rows:
        got = ph.philox4x32_10(*inp)
        assert [int(g) for g in got] == out


def _curand():
    for cand in ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]:
        if cand and os.path.exists(cand):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    return None


@pytest.mark.parametrize("seed", [0, 1234, 0x0123456789ABCDEF, 2**64 - 1])
def test_matches_curand_host_generator(seed):
    """curand's host Philox4x32-10 generator emits block b as philox(ctr=(0,0,b,0),
    key=(seed lo, seed hi)) -- a library routine computed on the CPU."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n_blocks = 64
        buf = (ctypes.c_uint32 * (4 * n_blocks))()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(4 * n_blocks)) == 0
        got = np.array(buf, dtype=np.uint64).reshape(n_blocks, 4)
        b = np.arange(n_blocks, dtype=np.uint64)
        k0, k1 = ph.key_of(seed)
        ref = ph.philox4x32_10(np.zeros(n_blocks, np.uint64), np.zeros(n_blocks, np.uint64), b,
                               np.zeros(n_blocks, np.uint64), k0, k1)
        np.testing.assert_array_equal(got, np.stack(ref, axis=1))
    finally:
        lib.curandDestroyGenerator(gen)


def test_bijective_on_sample():
    c = np.arange(1 << 16, dtype=np.uint64)
    out = ph.stream(c * np.uint64(2654435761), 3, 0, 99)
    packed = (out[0] << np.uint64(32)) | out[1]
    assert len(np.unique(packed)) == len(c)


def test_stream_word_layout():
    """stream() puts the 64-bit counter in words 0/1, word2 and purpose in 2/3."""
    c = np.array([5 + (7 << 32)], dtype=np.uint64)
    a = ph.stream(c, 11, 2, (13 << 32) | 17)
    b = ph.philox4x32_10(5, 7, 11, 2, 17, 13)
    assert [int(x[0]) for x in a] == [int(x) for x in b]
