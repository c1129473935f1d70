"""Plant plausible mistakes in a copy of the oracle and check that its pins catch them.

Each case rewrites one expression of ``oracle/asyrk_oracle.c`` in a temporary
copy, builds it, runs the oracle's Python API on that build and asserts that the
pin named beside the mistake fails.  The real oracle is never modified.
"""
import math
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1401_4780_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "asyrk_oracle.c")


def _build_variant(tmp_path, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, old
    path = tmp_path / "variant.c"
    path.write_text(text.replace(old, new))
    lib = tmp_path / "libvariant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(lib), str(path), "-lm"])
    return str(lib)


def pin_step_identity():
    s = synth.make_system(96, 24, 6, 3, row_norms="lognormal", value_dtype="f64")
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    gamma = 0.5
    x = np.zeros(s.n)
    rows, r, e2 = oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, 77, 0, 0,
                                  2 * s.m, sampler=samp, x_true=s.x_true, trace=True)
    d = x - s.x_true
    e2_next = np.append(e2[1:], d @ d)
    # the weights from the dense definition, not from the oracle under test
    w = np.array([np.sum(s.val64[s.row_ptr[i]:s.row_ptr[i + 1]] ** 2) for i in rows])
    pred = e2 - gamma * (2 - gamma) * r * r / w
    return np.max(np.abs(e2_next - pred) / e2) <= 1e-12


def pin_row_frequencies():
    m = 64
    w = np.exp(np.random.default_rng(5).standard_normal(m))
    row_ptr = np.arange(m + 1, dtype=np.int64)
    samp = oracle.Sampler(m, row_ptr, np.sqrt(w))
    rows = oracle.draw_rows(0xC0FFEE, 0, 0, 400_000, samp.thr, samp.alias, samp.uniform)
    _, p = stats.chisquare(np.bincount(rows, minlength=m), w / w.sum() * rows.size)
    return p > 1e-3


def pin_alias_probabilities():
    m = 1000
    w = np.exp(2 * np.random.default_rng(1).standard_normal(m))
    thr, alias, uniform = oracle.alias_table(w, float(w.sum()))
    keep = thr / 2.0**32
    p = keep.copy()
    np.add.at(p, alias.astype(np.int64), 1 - keep)
    # every bucket that aliases to row i adds at most one 2^-32 quantum to p_i
    n_alias = np.bincount(alias.astype(np.int64), minlength=m)
    return bool(np.all(np.abs(p / m - w / w.sum()) <= (1 + n_alias) / 2.0**32 / m + 1e-15))


def pin_philox_counter_words():
    # two counters that differ only in word 1 / word 2 / the key must differ,
    # and the known first block for key 0 (cuRAND host generator, seed 0) holds
    out = oracle.philox4x32_10([0, 0, 0, 0], [0, 0])
    return list(out) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


def pin_solver_reaches_tolerance():
    s = synth.plain_f64_system(m=512, n=128, L=8)
    x = np.zeros(s.n)
    res = oracle.rk_solve(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, 1.0, 5, 1e-8, 200,
                          x_true=s.x_true)
    err = np.linalg.norm(x - s.x_true) / np.linalg.norm(s.x_true)
    return res.status == oracle.OK and err <= 1e-8


def pin_shuffle_is_permutation():
    m = 1000
    w = np.ones(m)
    thr, alias, uniform = oracle.alias_table(w, float(m))
    rows = oracle.draw_rows(5, 0, 0, m, thr, alias, uniform, sampling=oracle.SAMPLE_SHUFFLED)
    return np.array_equal(np.sort(rows), np.arange(m))


def pin_single_coordinate_expectation():
    s = synth.make_system(24, 10, (2, 5), 5, row_norms="lognormal", value_dtype="f64")
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    x0 = s.x_true + np.random.default_rng(1).standard_normal(s.n)
    seed, gamma = 21, 0.3
    where = {}
    rows = oracle.draw_rows(seed, 0, 0, 3_000_000, samp.thr, samp.alias, samp.uniform)
    for j in range(rows.size):
        i = int(rows[j])
        theta = int(s.row_ptr[i + 1] - s.row_ptr[i])
        u = oracle.philox4x32_10([j & 0xFFFFFFFF, j >> 32, 0, 0], [seed, 0])
        where.setdefault((i, (int(u[2]) * theta) >> 32), j)
        if len(where) == s.nnz:
            break
    expect = 0.0
    for (i, t), j in where.items():
        theta = int(s.row_ptr[i + 1] - s.row_ptr[i])
        x = x0.copy()
        oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, seed, 0, j, 1,
                        sampler=samp, update=oracle.UPDATE_SINGLE)
        d = x - s.x_true
        expect += samp.w[i] / samp.F / theta * float(d @ d)
    A = oracle.dense(s.m, s.n, s.row_ptr, s.col, s.val64)
    e = x0 - s.x_true
    r = A @ e
    th = np.diff(s.row_ptr)
    exact = float(e @ e) - 2 * gamma / samp.F * float(r @ r) + gamma**2 / samp.F * float(th @ (r * r))
    return abs(expect - exact) <= 1e-12 * float(e @ e)


def pin_lsq_solution():
    m, n, phi = 120, 30, 2.0
    s = synth.make_system(m, n, 6, 9, row_norms="unit", value_dtype="f64")
    b = s.b + 0.3 * np.random.default_rng(10).standard_normal(m)
    A = oracle.dense(m, n, s.row_ptr, s.col, s.val64)
    x_ls = np.linalg.lstsq(A, b, rcond=None)[0]
    zeta = np.linalg.svd(A, compute_uv=False).min() / np.sqrt(2)
    rows, cols, rp, col, val, rhs = oracle.lsq_augment(m, n, s.row_ptr, s.col, s.val64, b, zeta,
                                                       phi)
    z = np.zeros(cols)
    oracle.rk_steps(rows, cols, rp, col, val, rhs, z, 1.0, 3, 0, 0, 3000 * rows)
    return np.max(np.abs(z[:n] / zeta - x_ls)) <= 1e-8 * np.abs(x_ls).max()


def pin_lsq_spectrum():
    m, n, zeta, phi = 40, 12, 0.2, 2.5
    s = synth.make_system(m, n, 5, 3, row_norms="lognormal", value_dtype="f64")
    rows, cols, rp, col, val, rhs = oracle.lsq_augment(m, n, s.row_ptr, s.col, s.val64, s.b, zeta,
                                                       phi)
    got = np.sort(np.linalg.svd(oracle.dense(rows, cols, rp, col, val), compute_uv=False))
    sv = np.linalg.svd(oracle.dense(m, n, s.row_ptr, s.col, s.val64), compute_uv=False)
    want = []
    for x in sv:
        want.extend(np.linalg.svd(np.array([[0.0, phi * x], [x, -zeta]]), compute_uv=False))
    want = np.sort(np.array(want + [zeta] * (m - sv.size) + [0.0] * (n - sv.size)))
    return got.shape == want.shape and np.allclose(got, want, rtol=1e-12, atol=1e-12 * want.max())


def pin_frobenius_exact():
    # F = ||A||_F^2 (Section 1's row probabilities divide by it) is the exact
    # sum of the w_i, rounded once: checked against Python's correctly rounded
    # math.fsum on weights whose plain or blocked running sums round away
    # thousands of small terms
    m = 6000
    val = np.full(m, 2.0**-27)          # w_i = 2^-54: below half an ulp of 1
    val[0] = 1.0
    val[2500] = 3.0
    row_ptr = np.arange(m + 1, dtype=np.int64)
    w, F = oracle.row_weights(m, row_ptr, val)
    # a tie broken by one bit far below it: 1 + 2^-53 + 2^-1074 rounds up
    tie = np.array([1.0, 2.0**-53, 2.0**-1074])
    return (F == math.fsum(w) and oracle.exact_sum(w[::-1]) == F
            and oracle.exact_sum(tie) == math.fsum(tie) == 1.0 + 2.0**-52)


MUTATIONS = [
    ("dropped gamma", "double s = gamma * r / w[i];", "double s = r / w[i];", pin_step_identity),
    ("sign of b", "double r = dot - b[i];", "double r = dot + b[i];", pin_step_identity),
    ("update sign", "x[col[k]] -= s * val[k];", "x[col[k]] += s * val[k];", pin_step_identity),
    ("norm not squared", "double s = gamma * r / w[i];", "double s = gamma * r / sqrt(w[i]);",
     pin_step_identity),
    ("last nonzero skipped in dot",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) dot += val[k] * x[col[k]];",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1] - 1; ++k) dot += val[k] * x[col[k]];",
     pin_step_identity),
    ("alias ignored", "return (u[1] < thr[bucket]) ? (int64_t)bucket : (int64_t)alias[bucket];",
     "return (int64_t)bucket;", pin_row_frequencies),
    ("alias coin inverted", "return (u[1] < thr[bucket]) ? (int64_t)bucket : (int64_t)alias[bucket];",
     "return (u[1] >= thr[bucket]) ? (int64_t)bucket : (int64_t)alias[bucket];",
     pin_row_frequencies),
    ("heavy's residual not carried to the next heavy", "R = M[heavy[t + 1]] - (U - R);",
     "R = M[heavy[t + 1]];", pin_alias_probabilities),
    ("light's deficit not taken from the heavy", "R -= U - M[l];", "R -= M[l];",
     pin_alias_probabilities),
    ("rounding of the masses not redistributed",
     "M[i] += D / m + (i < D % m ? 1 : 0);", "M[i] += 0;", pin_alias_probabilities),
    ("weights not squared", "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += val[k] * val[k];",
     "for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s += fabs(val[k]);",
     pin_row_frequencies),
    ("Philox key schedule", "k1 += PHILOX_W1;", "k1 += PHILOX_W0;", pin_philox_counter_words),
    ("Philox word swap", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c3 ^ k0;",
     pin_philox_counter_words),
    ("single update without theta", "x[col[k]] -= ((double)theta * s) * val[k];",
     "x[col[k]] -= s * val[k];", pin_single_coordinate_expectation),
    ("single update picks the wrong entry",
     "const int64_t k = row_ptr[i] + pick;", "const int64_t k = row_ptr[i];",
     pin_single_coordinate_expectation),
    ("Feistel round not a permutation",
     "uint64_t nr = L ^ ((uint64_t)fmix32((uint32_t)R ^ K[r]) & mask);",
     "uint64_t nr = R ^ ((uint64_t)fmix32((uint32_t)L ^ K[r]) & mask);",
     pin_shuffle_is_permutation),
    ("least squares: sign of zeta", "aval[e] = -zeta;", "aval[e] = zeta;", pin_lsq_solution),
    ("least squares: right side without phi", "ab[r] = phi * s;", "ab[r] = s;",
     pin_lsq_solution),
    ("least squares: A^T block without phi", "aval[e] = phi * tval[p];", "aval[e] = tval[p];",
     pin_lsq_spectrum),
    ("least squares: right side over the wrong b",
     "s += tval[p] * b[trow[p]];", "s += tval[p] * b[p - cstart[j]];", pin_lsq_solution),
    ("F summed by a plain running sum", "return oracle_exact_sum(m, w);",
     "double F = 0.0;\n    for (int64_t i = 0; i < m; ++i) F += w[i];\n    return F;",
     pin_frobenius_exact),
    ("F summed in blocks of 2048 rows", "return oracle_exact_sum(m, w);",
     "double F = 0.0;\n    for (int64_t b0 = 0; b0 < m; b0 += 2048) {\n"
     "        double part = 0.0;\n"
     "        for (int64_t i = b0; i < m && i < b0 + 2048; ++i) part += w[i];\n"
     "        F += part;\n    }\n    return F;",
     pin_frobenius_exact),
    ("exact sum drops the sticky bit", "sticky = exact_bit(digits, b);", "sticky = 0;",
     pin_frobenius_exact),
    ("stop test on wrong measure", "if (meas <= tol) status = OR_OK;\n    }",
     "if (meas <= 1e3 * tol) status = OR_OK;\n    }", pin_solver_reaches_tolerance),
]


def test_pins_hold_on_the_real_oracle():
    for _, _, _, pin in MUTATIONS:
        assert pin()


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pin):
    lib = _build_variant(tmp_path, old, new)
    with oracle.swapped_library(lib):
        assert not pin(), "pin did not catch: " + name
