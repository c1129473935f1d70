"""Pins of the oracle's two variants (CPU only).

Shuffled sweeps (the paper's implementation samples without replacement,
reshuffled after each scan, Section 5):
  * every sweep's order is a bijection of the rows, for awkward m too;
  * sweeps differ, and a row's position is uniform over many sweeps (chi-square);
  * an orthogonal system is solved exactly after one sweep (each row once).

Single-coordinate update (Algorithm 1):
  * the exact one-step expectation, enumerating every (row, entry) pair, equals
    ||e||^2 - (2 gamma/F)||Ae||^2 + (gamma^2/F) sum_i theta_i (a_i^T e)^2
    (the identity E_t[theta P_t a] = a of the proof of Theorem 1 gives the cross
    term); a missing theta, a wrong norm or a wrong entry breaks it;
  * with unit rows and gamma = 1/mu (psi = mu when tau = 0), the mean error
    obeys Theorem 1's bound (1 - lambda_min gamma (2 - gamma psi)/m)^J.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1401_4780_gb300 import synth


@pytest.mark.parametrize("m", [1, 2, 3, 5, 7, 8, 64, 1000, 4097, 65537])
def test_each_sweep_is_a_permutation(m):
    w = np.ones(m)
    thr, alias, uniform = oracle.alias_table(w, float(m))
    for k in (0, 1, 12345):
        rows = oracle.draw_rows(99, 3, k * m, m, thr, alias, uniform, sampling=oracle.SAMPLE_SHUFFLED)
        assert np.array_equal(np.sort(rows), np.arange(m))
        assert all(oracle.shuffle(99, 3, k, m, q) == rows[q] for q in range(0, m, max(1, m // 17)))


def test_sweeps_differ_and_positions_are_uniform():
    m = 50
    w = np.ones(m)
    thr, alias, uniform = oracle.alias_table(w, float(m))
    sweeps = 20000
    rows = oracle.draw_rows(7, 0, 0, sweeps * m, thr, alias, uniform,
                            sampling=oracle.SAMPLE_SHUFFLED).reshape(sweeps, m)
    assert np.mean(np.any(rows[1:] != rows[:-1], axis=1)) > 0.999
    first = np.bincount(rows[:, 0], minlength=m)
    assert stats.chisquare(first).pvalue > 1e-3
    pos_of_row0 = np.argmax(rows == 0, axis=1)
    assert stats.chisquare(np.bincount(pos_of_row0, minlength=m)).pvalue > 1e-3
    # the stream word changes the order
    other = oracle.draw_rows(7, 1, 0, m, thr, alias, uniform, sampling=oracle.SAMPLE_SHUFFLED)
    assert np.any(other != rows[0])


def test_orthogonal_rows_are_exact_after_one_shuffled_sweep():
    H = np.array([[1.0]])
    for _ in range(3):
        H = np.block([[H, H], [H, -H]])
    rng = np.random.default_rng(3)
    A = H * np.exp(rng.standard_normal(8))[:, None]
    row_ptr = np.arange(0, 65, 8, dtype=np.int64)
    col = np.tile(np.arange(8, dtype=np.int32), 8)
    xs = rng.standard_normal(8)
    b = A @ xs
    x = np.zeros(8)
    oracle.rk_steps(8, 8, row_ptr, col, A.reshape(-1), b, x, 1.0, 11, 0, 0, 7,
                    sampling=oracle.SAMPLE_SHUFFLED)
    assert np.linalg.norm(x - xs) > 1e-3
    oracle.rk_steps(8, 8, row_ptr, col, A.reshape(-1), b, x, 1.0, 11, 0, 7, 1,
                    sampling=oracle.SAMPLE_SHUFFLED)
    assert np.linalg.norm(x - xs) <= 1e-14 * np.linalg.norm(xs)


def _draw_t(seed, j, theta):
    u = oracle.philox4x32_10([j & 0xFFFFFFFF, j >> 32, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
    return (int(u[2]) * theta) >> 32


@pytest.mark.parametrize("gamma", [1.0, 0.3])
def test_single_coordinate_expectation_by_enumeration(gamma):
    s = synth.make_system(24, 10, (2, 5), 5, row_norms="lognormal", value_dtype="f64")
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    x0 = s.x_true + np.random.default_rng(1).standard_normal(s.n)
    seed = 21
    # a sequence position j drawing each (row, entry) pair
    where = {}
    rows = oracle.draw_rows(seed, 0, 0, 3_000_000, samp.thr, samp.alias, samp.uniform)
    for j in range(rows.size):
        i = int(rows[j])
        theta = int(s.row_ptr[i + 1] - s.row_ptr[i])
        where.setdefault((i, _draw_t(seed, j, theta)), j)
        if len(where) == s.nnz:
            break
    assert len(where) == s.nnz
    F = samp.F
    expect = 0.0
    for (i, t), j in where.items():
        theta = int(s.row_ptr[i + 1] - s.row_ptr[i])
        x = x0.copy()
        oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, seed, 0, j, 1,
                        sampler=samp, update=oracle.UPDATE_SINGLE)
        d = x - s.x_true
        expect += samp.w[i] / F / theta * float(d @ d)
    A = oracle.dense(s.m, s.n, s.row_ptr, s.col, s.val64)
    e = x0 - s.x_true
    r = A @ e
    theta_all = np.diff(s.row_ptr)
    exact = float(e @ e) - 2 * gamma / F * float(r @ r) + gamma**2 / F * float(theta_all @ (r * r))
    assert abs(expect - exact) <= 1e-12 * float(e @ e)


def test_single_coordinate_rate_bound_theorem1():
    s = synth.make_system(200, 50, 5, 23, row_norms="unit", value_dtype="f64")
    lmin, lmax = oracle.spectrum(s.m, s.n, s.row_ptr, s.col, s.val64)
    mu, _ = oracle.mu_nu(s.m, s.n, s.row_ptr, s.col)
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    gamma = 1.0 / mu  # psi = mu when tau = 0
    J = 20 * s.m
    ratios = []
    for seed in range(48):
        x = np.zeros(s.n)
        oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, 500 + seed, 0, 0, J,
                        sampler=samp, update=oracle.UPDATE_SINGLE)
        d = x - s.x_true
        ratios.append(float(d @ d) / float(s.x_true @ s.x_true))
    ratios = np.array(ratios)
    F = samp.F  # = m for unit rows
    bound = (1.0 - lmin * gamma * (2.0 - gamma * mu) / F) ** J
    assert ratios.mean() <= bound + 3 * ratios.std(ddof=1) / np.sqrt(ratios.size)
    assert bound < 0.2 and ratios.mean() < 0.2
