"""Pins of the oracle's RK iteration against facts the paper and algebra fix (CPU only).

  * Eq. (2) per step: for a consistent system and the projection with step
    length gamma, ||e_{j+1}||^2 = ||e_j||^2 - gamma (2 - gamma) r^2 / ||a_i||^2
    exactly (the derivation before Eq. (3); gamma = 1 is the printed case).
  * Eq. (3), middle line: with rows drawn with probability ||a_i||^2/||A||_F^2,
    E_i ||e_{j+1}||^2 = ||e_j||^2 - gamma (2 - gamma) ||A e_j||^2 / ||A||_F^2,
    checked by enumerating every row of a small system.
  * Eq. (3), last line, and the matching lower bound from the same identity:
    (1 - g lambda_max/F)^J <= E ||e_J||^2 / ||e_0||^2 <= (1 - g lambda_min/F)^J
    with g = gamma (2 - gamma), lambda from a dense eigendecomposition.
  * Special cases: orthogonal rows (RK is exact once every row has been used),
    a one-row system (solved in one step), the row just projected onto has zero
    residual.
  * lambda_max <= mu nu (Section 1, "Notation and Assumption").
  * The problem checks of Section 1 (no zero rows) and of the CSR layout.
"""
import numpy as np
import pytest

import oracle
from paper_1401_4780_gb300 import synth


def _small(m=96, n=24, L=6, seed=3, norms="lognormal"):
    return synth.make_system(m, n, L, seed, row_norms=norms, value_dtype="f64")


def _err2(x, xs):
    d = x - xs
    return float(d @ d)


@pytest.mark.parametrize("gamma", [1.0, 0.5, 1.5])
@pytest.mark.parametrize("norms", ["lognormal", "unit"])
def test_per_step_pythagoras_identity(gamma, norms):
    s = _small(norms=norms)
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    x = np.zeros(s.n)
    nsteps = 4 * s.m
    rows, r, e2 = oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, 77, 0, 0,
                                  nsteps, sampler=samp, x_true=s.x_true, trace=True)
    e2_next = np.append(e2[1:], _err2(x, s.x_true))
    w = samp.w[rows]
    predicted = e2 - gamma * (2.0 - gamma) * r * r / w
    ok = e2 > (1e-9 ** 2) * float(s.x_true @ s.x_true)  # above b's rounding floor
    assert ok.sum() > nsteps // 2
    rel = np.abs(e2_next - predicted)[ok] / e2[ok]
    assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("gamma", [1.0, 0.7])
def test_expected_decrease_by_enumerating_rows(gamma):
    s = _small(m=40, n=12, L=4, seed=11)
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    rng = np.random.default_rng(0)
    x0 = s.x_true + rng.standard_normal(s.n)
    # find, for every row, a position j of the sequence that draws it
    rows = oracle.draw_rows(9, 0, 0, 4_000_000, samp.thr, samp.alias, samp.uniform)
    uniq, pos = np.unique(rows, return_index=True)
    assert uniq.size == s.m
    first = dict(zip(uniq.tolist(), pos.tolist()))
    expect = 0.0
    for i in range(s.m):
        x = x0.copy()
        got = oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, 9, 0, first[i], 1,
                              sampler=samp, trace=True)
        assert got[0][0] == i
        expect += samp.w[i] / samp.F * _err2(x, s.x_true)
    A = oracle.dense(s.m, s.n, s.row_ptr, s.col, s.val64)
    e0 = x0 - s.x_true
    Ae = A @ e0
    exact = float(e0 @ e0) - gamma * (2 - gamma) * float(Ae @ Ae) / samp.F
    assert abs(expect - exact) <= 1e-12 * float(e0 @ e0)


def test_linear_rate_bounds_from_spectrum():
    s = synth.make_system(256, 64, 6, 21, row_norms="unit", value_dtype="f64")
    lmin, lmax = oracle.spectrum(s.m, s.n, s.row_ptr, s.col, s.val64)
    mu, nu = oracle.mu_nu(s.m, s.n, s.row_ptr, s.col)
    assert lmax <= mu * nu + 1e-9
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    F = samp.F
    J = 3 * s.m
    ratios = []
    for seed in range(48):
        x = np.zeros(s.n)
        oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, 1.0, 1000 + seed, 0, 0, J,
                        sampler=samp)
        ratios.append(_err2(x, s.x_true) / float(s.x_true @ s.x_true))
    ratios = np.array(ratios)
    upper = (1.0 - lmin / F) ** J
    lower = (1.0 - lmax / F) ** J
    mean = ratios.mean()
    se = ratios.std(ddof=1) / np.sqrt(ratios.size)
    assert mean <= upper + 3 * se, (mean, upper, se)
    assert mean >= lower - 3 * se, (mean, lower, se)
    # the bounds are not vacuous here: they differ from 0 and 1 by orders
    assert upper < 0.5 and lower > 1e-30


def test_orthogonal_rows_are_exact_after_every_row_is_used():
    # a signed, scaled 8x8 Hadamard block: orthogonal rows, 8 nonzeros each
    H = np.array([[1]])
    for _ in range(3):
        H = np.block([[H, H], [H, -H]])
    rng = np.random.default_rng(1)
    scale = np.exp(rng.standard_normal(8))
    A = H * scale[:, None]
    m = n = 8
    row_ptr = np.arange(0, 65, 8, dtype=np.int64)
    col = np.tile(np.arange(8, dtype=np.int32), 8)
    val = A.reshape(-1)
    xs = rng.standard_normal(8)
    b = A @ xs
    samp = oracle.Sampler(m, row_ptr, val)
    rows = oracle.draw_rows(5, 0, 0, 400, samp.thr, samp.alias, samp.uniform)
    last_new = max(int(np.argmax(rows == i)) for i in range(m))
    assert all((rows == i).any() for i in range(m))
    x = np.zeros(n)
    oracle.rk_steps(m, n, row_ptr, col, val, b, x, 1.0, 5, 0, 0, last_new, sampler=samp)
    assert np.linalg.norm(x - xs) > 1e-3  # one row is still unused
    oracle.rk_steps(m, n, row_ptr, col, val, b, x, 1.0, 5, 0, last_new, 1, sampler=samp)
    assert np.linalg.norm(x - xs) <= 1e-14 * np.linalg.norm(xs)


def test_single_row_system_is_solved_in_one_step():
    n = 10
    rng = np.random.default_rng(2)
    val = rng.standard_normal(n) * 3.0
    row_ptr = np.array([0, n], dtype=np.int64)
    col = np.arange(n, dtype=np.int32)
    b = np.array([2.5])
    x = rng.standard_normal(n)
    x0 = x.copy()
    oracle.rk_steps(1, n, row_ptr, col, val, b, x, 1.0, 0, 0, 0, 1)
    assert abs(val @ x - 2.5) <= 1e-14 * (np.abs(val) @ np.abs(x) + 2.5)
    # the step is along a_1 (minimum-norm correction)
    d = x - x0
    assert np.linalg.norm(d - (d @ val) / (val @ val) * val) <= 1e-14 * np.linalg.norm(d)


def test_projected_row_has_zero_residual():
    s = _small()
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    x = np.random.default_rng(4).standard_normal(s.n)
    rows, _, _ = oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, 1.0, 3, 0, 123, 1,
                                 sampler=samp, trace=True)
    i = rows[0]
    sl = slice(s.row_ptr[i], s.row_ptr[i + 1])
    ai_x = float(s.val64[sl] @ x[s.col[sl]])
    assert abs(ai_x - s.b[i]) <= 1e-13 * (abs(s.b[i]) + np.abs(s.val64[sl]) @ np.abs(x[s.col[sl]]))


def test_solve_stops_at_first_sweep_meeting_tolerance():
    s = synth.plain_f64_system(m=1024, n=256, L=8)
    seed = synth.solver_seed(s.seed)
    x = np.zeros(s.n)
    res = oracle.rk_solve(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, 1.0, seed, 1e-8, 500,
                          x_true=s.x_true)
    assert res.status == oracle.OK and res.rel_err <= 1e-8
    assert res.steps == res.sweeps * s.m
    x2 = np.zeros(s.n)
    res2 = oracle.rk_solve(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x2, 1.0, seed, 1e-8,
                           res.sweeps - 1, x_true=s.x_true)
    assert res2.status == oracle.NOT_CONVERGED and res2.rel_err > 1e-8
    # same sequence: the first sweeps - 1 sweeps of both runs agree bit for bit
    x3 = np.zeros(s.n)
    oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x3, 1.0, seed, 0, 0,
                    (res.sweeps - 1) * s.m)
    np.testing.assert_array_equal(x2, x3)


def test_residual_measures_match_dense_algebra():
    s = _small()
    A = oracle.dense(s.m, s.n, s.row_ptr, s.col, s.val64)
    x = np.random.default_rng(8).standard_normal(s.n)
    nrm, r = oracle.residual(s.m, s.row_ptr, s.col, s.val64, s.b, x)
    np.testing.assert_allclose(r, s.b - A @ x, rtol=0, atol=1e-12)
    assert abs(nrm - np.linalg.norm(s.b - A @ x)) <= 1e-12 * nrm
    g = oracle.normal_residual(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x)
    np.testing.assert_allclose(g, A.T @ (A @ x - s.b), rtol=0, atol=1e-11)


def test_gamma_outside_open_interval_is_rejected_and_divergence_reported():
    s = _small()
    for g in (0.0, 2.0, -1.0):
        res = oracle.rk_solve(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, np.zeros(s.n), g, 1, 1e-6,
                              5, x_true=s.x_true)
        assert res.status == oracle.EINVAL


@pytest.mark.parametrize("defect", ["zero_row", "unsorted", "duplicate", "out_of_range",
                                    "negative", "nan", "zero_values", "row_ptr0", "b_inf"])
def test_problem_checks(defect):
    m, n = 4, 6
    row_ptr = np.array([0, 2, 4, 6, 8], dtype=np.int64)
    col = np.array([0, 3, 1, 2, 4, 5, 0, 5], dtype=np.int32)
    val = np.arange(1.0, 9.0)
    b = np.ones(m)
    assert oracle.validate(m, n, row_ptr, col, val, b) == oracle.OK
    if defect == "zero_row":
        row_ptr = np.array([0, 2, 2, 4, 6], dtype=np.int64)
        col, val = col[:6], val[:6]
    elif defect == "unsorted":
        col[0], col[1] = 3, 0
    elif defect == "duplicate":
        col[1] = 0
    elif defect == "out_of_range":
        col[7] = 6
    elif defect == "negative":
        col[2] = -1
    elif defect == "nan":
        val[3] = np.nan
    elif defect == "zero_values":
        val[2:4] = 0.0
    elif defect == "row_ptr0":
        row_ptr = row_ptr + 1
    elif defect == "b_inf":
        b[2] = np.inf
    assert oracle.validate(m, n, row_ptr, col, val, b) == oracle.EINVAL


def test_underdetermined_system_converges_to_the_minimum_norm_solution():
    # m < n: the solutions form an affine set; every RK step moves x along a row
    # of A, so from x0 = 0 the iterates stay in range(A^T) and the limit is the
    # projection of 0 onto the solution set, pinv(A) b (a closed form)
    s = synth.make_system(120, 300, ("poisson", 6), 17, row_norms="unit", value_dtype="f64")
    A = oracle.dense(s.m, s.n, s.row_ptr, s.col, s.val64)
    x_mn = np.linalg.pinv(A) @ s.b
    x = np.zeros(s.n)
    oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, 1.0, 3, 0, 0, 600 * s.m)
    assert np.linalg.norm(x - x_mn) <= 1e-10 * np.linalg.norm(x_mn)
    assert np.linalg.norm(x - s.x_true) > 1e-2 * np.linalg.norm(s.x_true)  # x* is not the limit
    g = oracle.normal_residual(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x)
    assert float(g @ g) < 1e-18
