"""Pins of the oracle's least-squares system (Section 6), CPU only.

The square system [[0, phi A^T], [A, -zeta I]] (x, y) = (phi A^T b, 0):
  * its singular values are those of the 2x2 blocks [[0, phi s], [s, -zeta]]
    for the singular values s of A, zeta (m - r times) and 0 (n - r times),
    the decomposition of Section 6; for phi = 1 the smallest nonzero one is
    min{zeta, -zeta/2 + sqrt(zeta^2 + 4 s_r^2)/2};
  * ||.||_F^2 = (1 + phi^2) ||A||_F^2 + m zeta^2;
  * the right side's block is phi A^T b (against scipy's sparse product);
  * RK on it reaches x = zeta x_LS, x_LS from numpy's lstsq, and y = A x_LS;
    for a rank-deficient A, x / zeta is pinv(A) b;
  * at phi = 1, zeta = s_r/sqrt(2) the ratio sigma_min^2/||.||_F^2 is
    s_r^2/(4 ||A||_F^2 + m s_r^2) and moving zeta or phi lowers it;
  * an empty column of A gives no row.
"""
from types import SimpleNamespace

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1401_4780_gb300 import synth


def _dense_aug(m, n, zeta, phi, s):
    rows, cols, rp, col, val, rhs = oracle.lsq_augment(m, n, s.row_ptr, s.col, s.val64, s.b,
                                                       zeta, phi)
    return oracle.dense(rows, cols, rp, col, val), rhs, (rows, cols, rp, col, val, rhs)


def _inconsistent(m, n, L, seed, row_norms="unit"):
    s = synth.make_system(m, n, L, seed, row_norms=row_norms, value_dtype="f64")
    s.b = s.b + 0.3 * np.random.default_rng(seed + 1).standard_normal(m)
    return s


def _block_singular_values(sv, zeta, phi, m, n):
    r = sv.size
    out = []
    for x in sv:
        out.extend(np.linalg.svd(np.array([[0.0, phi * x], [x, -zeta]]), compute_uv=False))
    out.extend([zeta] * (m - r))
    out.extend([0.0] * (n - r))
    return np.sort(np.array(out))


@pytest.mark.parametrize("zeta,phi", [(0.7, 1.0), (0.2, 2.5), (1.9, 0.4)])
def test_singular_values_follow_section6_decomposition(zeta, phi):
    m, n = 40, 12
    s = _inconsistent(m, n, 5, 3, row_norms="lognormal")
    A = oracle.dense(m, n, s.row_ptr, s.col, s.val64)
    assert np.all(np.any(A != 0, axis=0))
    At, _, _ = _dense_aug(m, n, zeta, phi, s)
    assert At.shape == (n + m, n + m)
    got = np.sort(np.linalg.svd(At, compute_uv=False))
    sv = np.linalg.svd(A, compute_uv=False)
    want = _block_singular_values(sv, zeta, phi, m, n)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * want.max())
    if phi == 1.0:
        sr = sv.min()
        smin = min(zeta, -zeta / 2 + 0.5 * np.sqrt(zeta**2 + 4 * sr**2))
        assert abs(got[got > 1e-10].min() - smin) <= 1e-12 * smin


def test_frobenius_norm_and_right_side():
    m, n, zeta, phi = 300, 90, 0.37, 1.7
    s = _inconsistent(m, n, 6, 5, row_norms="lognormal")
    rows, cols, rp, col, val, rhs = oracle.lsq_augment(m, n, s.row_ptr, s.col, s.val64, s.b,
                                                       zeta, phi)
    fro_a = float(np.sum(s.val64 ** 2))
    assert abs(float(np.sum(val ** 2)) - ((1 + phi**2) * fro_a + m * zeta**2)) <= 1e-12 * fro_a
    A = sp.csr_matrix((s.val64, s.col, s.row_ptr), shape=(m, n))
    nonempty = np.flatnonzero(np.diff(A.tocsc().indptr) > 0)
    np.testing.assert_allclose(rhs[:nonempty.size], phi * (A.T @ s.b)[nonempty], rtol=1e-13,
                               atol=1e-13 * np.abs(rhs).max())
    assert np.all(rhs[nonempty.size:] == 0.0)
    assert rows == nonempty.size + m and cols == n + m
    # every row strictly ascending (a valid CSR for the solver)
    for i in range(rows):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)


def _rk_lsq(s, m, n, zeta, phi, sweeps, seed=3):
    rows, cols, rp, col, val, rhs = oracle.lsq_augment(m, n, s.row_ptr, s.col, s.val64, s.b,
                                                       zeta, phi)
    z = np.zeros(cols)
    oracle.rk_steps(rows, cols, rp, col, val, rhs, z, 1.0, seed, 0, 0, sweeps * rows)
    return z[:n], z[n:]


@pytest.mark.parametrize("phi", [1.0, 2.0])
def test_rk_on_the_system_gives_least_squares(phi):
    m, n = 120, 30
    s = _inconsistent(m, n, 6, 9)
    A = oracle.dense(m, n, s.row_ptr, s.col, s.val64)
    x_ls = np.linalg.lstsq(A, s.b, rcond=None)[0]
    assert np.linalg.norm(A @ x_ls - s.b) > 0.1  # really inconsistent
    sr = np.linalg.svd(A, compute_uv=False).min()
    zeta = sr / np.sqrt(2)
    x, y = _rk_lsq(s, m, n, zeta, phi, 3000)
    np.testing.assert_allclose(x / zeta, x_ls, rtol=0, atol=1e-8 * np.abs(x_ls).max())
    np.testing.assert_allclose(y, A @ x_ls, rtol=0, atol=1e-8 * np.abs(A @ x_ls).max())


def test_rank_deficient_gives_minimum_norm_least_squares():
    m, n = 80, 20
    s = _inconsistent(m, n, 5, 13)
    # make column 7 a copy of column 3 (same rows, same values): rank n - 1
    A = oracle.dense(m, n, s.row_ptr, s.col, s.val64)
    A[:, 7] = A[:, 3]
    keep = np.linalg.norm(A, axis=1) > 0
    A, b = A[keep], s.b[keep]
    m = A.shape[0]
    A = A / np.linalg.norm(A, axis=1, keepdims=True)
    Ac = sp.csr_matrix(A)
    Ac.sort_indices()
    s = SimpleNamespace(row_ptr=Ac.indptr.astype(np.int64), col=Ac.indices.astype(np.int32),
                        val64=Ac.data.astype(np.float64), b=b)
    sv = np.linalg.svd(A, compute_uv=False)
    sr = sv[sv > 1e-10 * sv[0]].min()
    zeta = sr / np.sqrt(2)
    x, _ = _rk_lsq(s, m, n, zeta, 1.0, 4000)
    x_mn = np.linalg.pinv(A) @ b
    np.testing.assert_allclose(x / zeta, x_mn, rtol=0, atol=1e-8 * np.abs(x_mn).max())


def test_section6_choice_maximises_the_ratio():
    m, n = 60, 20
    s = _inconsistent(m, n, 5, 21)
    A = oracle.dense(m, n, s.row_ptr, s.col, s.val64)
    sr = np.linalg.svd(A, compute_uv=False).min()
    fro = float(np.sum(A * A))

    def ratio(zeta, phi):
        At, _, _ = _dense_aug(m, n, zeta, phi, s)
        sv = np.linalg.svd(At, compute_uv=False)
        return sv[sv > 1e-10 * sv[0]].min() ** 2 / float(np.sum(At * At))

    best = ratio(sr / np.sqrt(2), 1.0)
    assert abs(best - sr**2 / (4 * fro + m * sr**2)) <= 1e-10 * best
    for zeta, phi in [(sr, 1.0), (sr / 2, 1.0), (sr / np.sqrt(2), 0.5), (sr / np.sqrt(2), 2.0)]:
        assert ratio(zeta, phi) < best


def test_empty_column_gives_no_row():
    rp = np.array([0, 2, 3], dtype=np.int64)
    col = np.array([0, 2, 1], dtype=np.int32)
    val = np.array([1.0, 2.0, 3.0])
    b = np.array([1.0, -1.0])
    rows, cols, arp, acol, aval, rhs = oracle.lsq_augment(2, 4, rp, col, val, b, 0.5, 2.0)
    assert rows == 5 and cols == 6
    assert list(arp) == [0, 1, 2, 3, 6, 8]
    assert list(acol) == [4, 5, 4, 0, 2, 4, 1, 5]
    assert list(aval) == [2.0, 6.0, 4.0, 1.0, 2.0, -0.5, 3.0, -0.5]
    assert list(rhs) == [2.0, -6.0, 4.0, 0.0, 0.0]
