"""Pins of the oracle's row sampler (CPU only).

The paper fixes the row probabilities ||a_i||^2/||A||_F^2 (Section 1, before
Eq. (2)); the generator behind them (Philox4x32-10, Salmon et al. SC'11) and the
alias table (Walker's method, built by one sweep over integer masses) are this
project's choice.  Each is pinned to something other
than the oracle itself:
  * Philox4x32-10 against cuRAND's host Philox4_32_10 generator, run here on the
    CPU (its documented layout: 65536 subsequences, counter word 2 = subsequence,
    words 0-1 = 64-bit position, key = the 64-bit seed);
  * the alias table against the exact probabilities it encodes, which must equal
    w_i/F up to the 2^-32 threshold quantisation;
  * the drawn rows against w_i/F by a chi-square test.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

_CURAND_PATHS = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]


def _curand():
    for p in _CURAND_PATHS:
        if p and (os.path.exists(p) or not p.startswith("/")):
            try:
                return ctypes.CDLL(p)
            except OSError:
                continue
    pytest.skip("libcurand not available")


def _curand_philox_host(lib, seed, count, offset):
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 42, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("step", [0, 1, 2**32 - 1, 2**33 + 5])
def test_philox_matches_curand_host_generator(seed, step):
    lib = _curand()
    T = 65536  # subsequences of the host generator
    out = _curand_philox_host(lib, seed, 4 * T * 2, offset=4 * T * step)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for s in (step, step + 1):  # step + 1 crosses into counter word 1 for 2^32 - 1
        for t in (0, 1, 2, 777, T - 1):
            blk = (s - step) * T + t
            ctr = [s & 0xFFFFFFFF, (s >> 32) & 0xFFFFFFFF, t, 0]
            np.testing.assert_array_equal(out[4 * blk:4 * blk + 4], oracle.philox4x32_10(ctr, key))


def test_philox_is_a_bijection_sample():
    # distinct counters give distinct outputs (a keyed bijection of 128 bits)
    key = [0x12345678, 0x9ABCDEF0]
    seen = {tuple(oracle.philox4x32_10([c, 0, 0, 0], key)) for c in range(4096)}
    assert len(seen) == 4096


def _alias_probabilities(thr, alias, uniform):
    m = thr.shape[0]
    if uniform:
        return np.full(m, 1.0 / m)
    keep = thr.astype(np.float64) / 2.0**32
    p = keep.copy()
    np.add.at(p, alias.astype(np.int64), 1.0 - keep)
    return p / m


@pytest.mark.parametrize("m,kind", [(1, "lognormal"), (2, "lognormal"), (7, "spiky"),
                                    (64, "lognormal"), (1000, "lognormal"), (100_000, "lognormal"),
                                    (4096, "near_unit"), (333, "one_heavy")])
def test_alias_table_encodes_row_probabilities(m, kind):
    rng = np.random.default_rng(m)
    if kind == "lognormal":
        w = np.exp(2 * rng.standard_normal(m))
    elif kind == "spiky":
        w = np.array([1e-12, 1.0, 1e6, 3.0, 1e-3, 7.0, 2.0])[:m]
    elif kind == "near_unit":
        w = 1.0 + rng.integers(-3, 4, size=m) * np.finfo(np.float64).eps
    else:
        w = np.ones(m)
        w[17] = 1e4
    F = float(np.sum(w))
    thr, alias, uniform = oracle.alias_table(w, F)
    assert uniform == 0 or np.all(w == w[0])
    assert np.all(alias < m)
    p = _alias_probabilities(thr, alias, uniform)
    # each threshold is quantised to 2^-32 and every bucket aliasing to row i
    # carries that error into p_i; FP64 rounding of the q updates adds ~1e-12
    n_alias = np.bincount(alias.astype(np.int64), minlength=m) if not uniform else np.zeros(m)
    tol = (1.0 + n_alias) / 2.0**32 / m + 1e-12 * (w / F) + 1e-15
    assert np.all(np.abs(p - w / F) <= tol)
    assert abs(np.sum(p) - 1.0) < 1e-12


def test_alias_uniform_shortcut_only_for_identical_weights():
    w = np.ones(50)
    thr, alias, uniform = oracle.alias_table(w, 50.0)
    assert uniform == 1
    w[3] = np.nextafter(1.0, 2.0)
    thr, alias, uniform = oracle.alias_table(w, float(np.sum(w)))
    assert uniform == 0


def _masses(thr, alias, m):
    """Units of 2^-32 of a bucket that the table gives each row."""
    M = thr.astype(np.int64).copy()
    full = thr == 0xFFFFFFFF
    M[full] = 1 << 32  # a full bucket (2^32 - 1 is the stored maximum)
    np.add.at(M, alias.astype(np.int64), np.where(full, 0, (1 << 32) - M))
    return M


@pytest.mark.parametrize("scale", [1.0, 1.0 - 1e-9, 1.0 + 1e-9])
def test_alias_table_is_a_whole_distribution(scale):
    # whatever F the table is given, the buckets hand out exactly m buckets'
    # worth of mass (probabilities that add up to 1 with no unit of 2^-32 lost
    # or created); each row's share stays w_i / sum(w), off by the 2^-32
    # quantisation and, when F is off by a factor, by at most that factor's
    # share of the total mass moved to renormalise
    m = 1000
    w = np.exp(2 * np.random.default_rng(8).standard_normal(m))
    F = float(np.sum(w)) * scale
    thr, alias, uniform = oracle.alias_table(w, F)
    M = _masses(thr, alias, m)
    assert int(M.sum()) == m << 32
    p = M / float(m << 32)
    n_alias = np.bincount(alias.astype(np.int64), minlength=m)
    target = w / math.fsum(w)
    moved = 2.0 * abs(1.0 / scale - 1.0)
    assert np.all(np.abs(p - target) <= (1 + n_alias) / 2.0**32 / m + moved + 1e-12 * target)
    assert np.sum(np.abs(p - target)) <= moved + (1 + n_alias).sum() / 2.0**32 / m


def test_drawn_rows_follow_row_weights_chi_square():
    m = 64
    rng = np.random.default_rng(5)
    w = np.exp(rng.standard_normal(m))
    F = float(np.sum(w))
    thr, alias, uniform = oracle.alias_table(w, F)
    rows = oracle.draw_rows(0xC0FFEE, 0, 0, 1_000_000, thr, alias, uniform)
    counts = np.bincount(rows, minlength=m)
    expected = w / F * rows.size
    chi2, p = stats.chisquare(counts, expected)
    assert p > 1e-3, (chi2, p)


def test_draws_depend_on_stream_and_position():
    w = np.ones(1 << 20)
    thr, alias, uniform = oracle.alias_table(w, float(w.size))
    a = oracle.draw_rows(1, 0, 0, 1000, thr, alias, uniform)
    b = oracle.draw_rows(1, 1, 0, 1000, thr, alias, uniform)
    c = oracle.draw_rows(1, 0, 500, 500, thr, alias, uniform)
    assert np.mean(a != b) > 0.99
    np.testing.assert_array_equal(a[500:], c)


def test_bucket_is_the_high_word_of_u0_times_m():
    # uniform weights: the draw is floor(u0 * m / 2^32) of Philox at counter (j, 0, stream, 0)
    m = 12345
    w = np.ones(m)
    thr, alias, uniform = oracle.alias_table(w, float(m))
    seed = 0xABCDEF0123
    rows = oracle.draw_rows(seed, 3, 2**32 - 2, 4, thr, alias, uniform)
    for t in range(4):
        j = 2**32 - 2 + t
        u = oracle.philox4x32_10([j & 0xFFFFFFFF, j >> 32, 3, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert rows[t] == (int(u[0]) * m) >> 32
