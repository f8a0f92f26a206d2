"""Pins for the oracle's random-number layer.

* Philox4x32-10 is checked against an independent implementation: cuRAND's
  host-side PHILOX4_32_10 generator (a library routine, run on the CPU).  Its
  output block b is Philox with counter (b // 65536 low word, high word,
  b % 65536, 0) under key (seed low, seed high), so an offset into its stream
  selects exactly the counters (slot, event, purpose, 0) the method uses.
* The uniform mapping is exact in float32 and stays inside (0, 1).
* Box-Muller normals and log-normal smearing are checked statistically against
  their closed-form distributions (fixed seeds, so the tests are deterministic).
"""
import ctypes as C
import os

import numpy as np
import pytest
from scipy import stats

import oracle

P_MIN = 1e-3  # acceptance level of the statistical pins


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return C.CDLL(path)
        except OSError:
            continue
    return None


def _curand_block(lib, seed: int, block: int) -> np.ndarray:
    gen = C.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(C.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, C.c_ulonglong(4 * block)) == 0
        out = np.zeros(4, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(C.c_void_p), C.c_size_t(4)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_matches_curand_host_generator():
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    lib.curandCreateGeneratorHost.argtypes = [C.c_void_p, C.c_int]
    lib.curandSetPseudoRandomGeneratorSeed.argtypes = [C.c_void_p, C.c_ulonglong]
    lib.curandSetGeneratorOffset.argtypes = [C.c_void_p, C.c_ulonglong]
    lib.curandGenerate.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
    lib.curandDestroyGenerator.argtypes = [C.c_void_p]
    n_checked = 0
    for seed in (0, 1, 42, 0x0123456789ABCDEF, 2**64 - 1):
        key = (seed & 0xFFFFFFFF, seed >> 32)
        for slot in (0, 1, 403, 65535, 2**32 - 1):
            for event in (0, 1, 99, 16383):
                for purpose in (1, 2, 3, 4):
                    block = ((event << 32) | slot) * 65536 + purpose
                    ref = _curand_block(lib, seed, block)
                    got = oracle.philox((slot, event, purpose, 0), key)
                    assert np.array_equal(ref, got), (seed, slot, event, purpose)
                    n_checked += 1
    assert n_checked == 400


def test_philox_counter_words_all_matter():
    key = (0x12345678, 0x9ABCDEF0)
    base = oracle.philox((5, 6, 7, 8), key)
    for word in range(4):
        ctr = [5, 6, 7, 8]
        ctr[word] ^= 1
        other = oracle.philox(ctr, key)
        # every output word changes (avalanche after ten rounds)
        assert np.all(other != base), word
    assert np.all(oracle.philox((5, 6, 7, 8), (key[0] ^ 1, key[1])) != base)


def test_u01_exact_and_open_interval():
    assert oracle.u01(0) == 2.0**-24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0**-24
    assert oracle.u01(0x80000000) == 0.5 + 2.0**-24
    rng = np.random.default_rng(7)
    for w in rng.integers(0, 2**32, 1000, dtype=np.uint64):
        u = oracle.u01(int(w))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u  # representable in float32: both sides share it exactly
        # only the top 23 bits matter
        assert oracle.u01(int(w) | 0x1FF) == u


def _philox_words(n, purpose, seed=2024):
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 1] = 12345
    ctr[:, 2] = purpose
    return oracle.philox_n(ctr, (seed & 0xFFFFFFFF, seed >> 32))


def test_philox_words_uniform():
    w = _philox_words(200_000, 1)
    for k in range(4):
        u = (w[:, k] >> 9).astype(np.float64) / 2**23
        assert stats.kstest(u, "uniform").pvalue > P_MIN


def test_box_muller_normal_distribution():
    n = 1_000_000
    w = _philox_words(n, 3)
    z = oracle.normal_n(w[:, 0], w[:, 1])
    assert stats.kstest(z, "norm").pvalue > P_MIN
    # mean 0 and variance 1 (z-tests with the exact sampling variances 1/n, 2/n)
    assert abs(z.mean()) / np.sqrt(1.0 / n) < stats.norm.isf(P_MIN / 2)
    assert abs(z.var() - 1.0) / np.sqrt(2.0 / n) < stats.norm.isf(P_MIN / 2)
    # the smallest uniform is 2^-24, so |z| <= sqrt(48 ln 2)
    assert np.abs(z).max() <= np.sqrt(-2.0 * np.log(2.0**-24)) + 1e-12


@pytest.mark.parametrize("x", [0.3, 1.0, 7.0, 120.0])
@pytest.mark.parametrize("rel", [0.01, 0.2, 1.0, 2.0])
def test_lognormal_moments(x, rel):
    """Mean x and standard deviation rel*x (closed-form log-normal moments)."""
    n = 1_000_000
    w = _philox_words(n, 4, seed=int(x * 1000) + int(rel * 100))
    z = oracle.normal_n(w[:, 0], w[:, 1])
    xs = oracle.lognormal_n(x, rel, z)
    assert np.all(xs > 0)
    q = 1.0 + rel * rel
    # E[X^k] = x^k q^(k(k-1)/2) for a log-normal with mean x and variance (rel x)^2
    m1, m2, m4 = x, x * x * q, x**4 * q**6
    zcrit = stats.norm.isf(P_MIN / 2)
    assert abs(xs.mean() - m1) / np.sqrt((m2 - m1 * m1) / n) < zcrit
    x2 = xs * xs
    assert abs(x2.mean() - m2) / np.sqrt((m4 - m2 * m2) / n) < zcrit
    # log(X/x) ~ N(-s^2/2, s^2) with s^2 = log(1 + rel^2)
    s2 = np.log1p(rel * rel)
    lx = np.log(xs / x)
    assert stats.kstest(lx, stats.norm(loc=-0.5 * s2, scale=np.sqrt(s2)).cdf).pvalue > P_MIN


def test_eff_threshold_exact():
    assert oracle.eff_threshold(1.0) == 2**32
    assert oracle.eff_threshold(1.5) == 2**32
    assert oracle.eff_threshold(0.0) == 0
    assert oracle.eff_threshold(-0.1) == 0
    assert oracle.eff_threshold(0.5) == 2**31
    assert oracle.eff_threshold(0.95) == 4080218931  # floor(0.95 * 4294967296) = floor(4080218931.2)
    assert oracle.eff_threshold(0.25) == 2**30
    # eff = 1 accepts every 32-bit word, eff = 0 none
    assert (2**32 - 1) < oracle.eff_threshold(1.0)
    assert not (0 < oracle.eff_threshold(0.0))
