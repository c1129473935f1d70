"""Sequential FP64 CPU oracle for randomized Kaczmarz (AsyRK paper, arXiv:1401.4780).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library never
calls it, and it never calls the CUDA library: the two meet only through the
seeded input generator (``paper_1401_4780_gb300.synth``), which holds none of the
method's arithmetic.

The arithmetic lives in ``asyrk_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module only loads it through ctypes and marshals
numpy arrays.  ``spectrum()`` adds the dense eigenvalue computation used by the
rate pins (numpy ``eigvalsh`` on A^T A).

Paper passages followed (section / equation):
  * problem and row probabilities ||a_i||^2/||A||_F^2: Section 1, before Eq. (2);
  * the projection: Eq. (2), with a step-length factor gamma;
  * full-row update, single thread equals the usual RK: Section 5;
  * the expected one-step decrease and the rate 1 - lambda_min/||A||_F^2: Eq. (3);
  * sampling without replacement, reshuffled each scan (the paper's
    implementation, Section 5) and the single-coordinate update (Algorithm 1);
  * lambda_min, lambda_max, mu, nu: Section 1, "Notation and Assumption".
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asyrk_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SAMPLE_WEIGHTED, SAMPLE_SHUFFLED = 0, 1
UPDATE_ROW, UPDATE_SINGLE = 0, 1

OK = 0
EINVAL = -1
ENOMEM = -2
NOT_CONVERGED = 1
DIVERGED = 2


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class OracleResult(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("rel_err", ctypes.c_double), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _bind(path):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, u64, u32, i32, f64 = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                               ctypes.c_int32, ctypes.c_double)
    lib.oracle_philox4x32_10.argtypes = [P, P, P]
    lib.oracle_philox4x32_10.restype = None
    lib.oracle_validate.argtypes = [i64, i64, P, P, P, P]
    lib.oracle_validate.restype = ctypes.c_int
    lib.oracle_row_weights.argtypes = [i64, P, P, P]
    lib.oracle_row_weights.restype = f64
    lib.oracle_exact_sum.argtypes = [i64, P]
    lib.oracle_exact_sum.restype = f64
    lib.oracle_alias_build.argtypes = [i64, P, f64, P, P]
    lib.oracle_alias_build.restype = ctypes.c_int
    lib.oracle_draw_rows.argtypes = [u64, u32, u64, i64, i64, P, P, ctypes.c_int, P]
    lib.oracle_draw_rows.restype = None
    lib.oracle_residual_norm.argtypes = [i64, P, P, P, P, P, P]
    lib.oracle_residual_norm.restype = f64
    lib.oracle_normal_residual.argtypes = [i64, i64, P, P, P, P, P, P]
    lib.oracle_normal_residual.restype = None
    lib.oracle_rk_steps.argtypes = [i64, P, P, P, P, P, P, P, ctypes.c_int, u64, u32,
                                    f64, u64, i64, P, i64, P, P, P, P]
    lib.oracle_rk_steps.restype = None
    lib.oracle_rk_solve.argtypes = [i64, i64, P, P, P, P, P, f64, u64, u32, u64, f64,
                                    i64, i64, P, ctypes.POINTER(OracleResult)]
    lib.oracle_rk_solve.restype = ctypes.c_int
    lib.oracle_shuffle.argtypes = [u64, u32, u64, i64, i64]
    lib.oracle_shuffle.restype = i64
    lib.oracle_draw_rows_ex.argtypes = [u64, u32, u64, i64, i64, P, P, ctypes.c_int, ctypes.c_int,
                                        P]
    lib.oracle_draw_rows_ex.restype = None
    lib.oracle_rk_steps_ex.argtypes = [i64, P, P, P, P, P, P, P, ctypes.c_int, u64, u32, f64, u64,
                                       i64, P, i64, P, P, P, P, ctypes.c_int, ctypes.c_int]
    lib.oracle_rk_steps_ex.restype = None
    lib.oracle_rk_solve_ex.argtypes = [i64, i64, P, P, P, P, P, f64, u64, u32, u64, f64, i64, i64,
                                       P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(OracleResult)]
    lib.oracle_rk_solve_ex.restype = ctypes.c_int
    lib.oracle_lsq_augment.argtypes = [i64, i64, P, P, P, P, f64, f64, P, P, P, P]
    lib.oracle_lsq_augment.restype = i64
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


@contextlib.contextmanager
def swapped_library(path):
    """Run the oracle's Python API on another build of ``asyrk_oracle.c``.

    Used by the tests that plant mistakes in a copy of the oracle and check that
    the pins reject it."""
    global _lib
    prev = _load()
    _lib = _bind(path)
    try:
        yield
    finally:
        _lib = prev


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr(row_ptr, col, val):
    return (np.ascontiguousarray(row_ptr, dtype=np.int64),
            np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


# --------------------------------------------------------------------------
# Sampler
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) of one 128-bit counter."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    assert c.shape == (4,) and k.shape == (2,)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def exact_sum(v):
    """The sum of finite values v_i >= 0, exact until one final rounding to the
    nearest double (ties to even)."""
    a = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().oracle_exact_sum(a.shape[0], _p(a)))


def row_weights(m, row_ptr, val):
    """w_i = ||a_i||^2 (FP64, CSR order) and F = ||A||_F^2, the w_i's exact sum
    rounded once."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    v = np.ascontiguousarray(val, dtype=np.float64)
    w = np.zeros(m, dtype=np.float64)
    F = _load().oracle_row_weights(m, _p(rp), _p(v), _p(w))
    return w, F


def alias_table(w, F):
    """Alias table (thr, alias, uniform) for probabilities w_i / F (the sweep over
    integer masses stated in asyrk_oracle.c)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    m = w.shape[0]
    thr = np.zeros(m, dtype=np.uint32)
    alias = np.zeros(m, dtype=np.uint32)
    u = _load().oracle_alias_build(m, _p(w), float(F), _p(thr), _p(alias))
    if u < 0:
        raise MemoryError("oracle alias table")
    return thr, alias, int(u)


def draw_rows(seed, stream, j0, count, thr, alias, uniform, sampling=SAMPLE_WEIGHTED):
    """Rows i(j) for j = j0 .. j0+count-1 of the row sequence (Philox/alias, or
    shuffled sweeps)."""
    m = thr.shape[0]
    out = np.zeros(count, dtype=np.int32)
    _load().oracle_draw_rows_ex(seed, stream, j0, count, m, _p(thr), _p(alias), int(uniform),
                                int(sampling), _p(out))
    return out


def shuffle(seed, stream, k, m, q):
    """pi_k(q): position q of sweep k in the shuffled order of rows 0..m-1."""
    return int(_load().oracle_shuffle(seed, stream, k, m, q))


# --------------------------------------------------------------------------
# Measures
# --------------------------------------------------------------------------
def validate(m, n, row_ptr, col, val, b=None):
    rp, c, v = _csr(row_ptr, col, val)
    bb = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    return _load().oracle_validate(m, n, _p(rp), _p(c), _p(v), _p(bb))


def residual(m, row_ptr, col, val, b, x):
    """(||b - A x||, r = b - A x) in FP64."""
    rp, c, v = _csr(row_ptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    r = np.zeros(m, dtype=np.float64)
    nrm = _load().oracle_residual_norm(m, _p(rp), _p(c), _p(v), _p(bb), _p(xx), _p(r))
    return nrm, r


def normal_residual(m, n, row_ptr, col, val, b, x):
    """A^T (A x - b) in FP64 (Table 2's measure is its squared norm)."""
    rp, c, v = _csr(row_ptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    g = np.zeros(n, dtype=np.float64)
    _load().oracle_normal_residual(m, n, _p(rp), _p(c), _p(v), _p(bb), _p(xx), _p(g))
    return g


def lsq_augment(m, n, row_ptr, col, val, b, zeta, phi=1.0):
    """Section 6's square consistent system for min ||A x - b||.

    Returns (rows, cols, row_ptr, col, val, rhs) of the matrix
    [[0, phi A^T], [A, -zeta I]] over (x, y), rows of empty columns left out;
    its solutions have x = zeta x_LS."""
    rp, c, v = _csr(row_ptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    nnz = int(rp[-1])
    arp = np.zeros(n + m + 1, dtype=np.int64)
    acol = np.zeros(2 * nnz + m, dtype=np.int32)
    aval = np.zeros(2 * nnz + m, dtype=np.float64)
    ab = np.zeros(n + m, dtype=np.float64)
    rows = _load().oracle_lsq_augment(m, n, _p(rp), _p(c), _p(v), _p(bb), float(zeta), float(phi),
                                      _p(arp), _p(acol), _p(aval), _p(ab))
    e = int(arp[rows])
    return rows, n + m, arp[:rows + 1].copy(), acol[:e].copy(), aval[:e].copy(), ab[:rows].copy()


# --------------------------------------------------------------------------
# RK iteration
# --------------------------------------------------------------------------
class Sampler:
    """Row weights and alias table of one matrix, built once."""

    def __init__(self, m, row_ptr, val):
        self.m = m
        self.w, self.F = row_weights(m, row_ptr, val)
        self.thr, self.alias, self.uniform = alias_table(self.w, self.F)


def rk_steps(m, n, row_ptr, col, val, b, x, gamma, seed, stream, j0, nsteps,
             sampler=None, x_true=None, trace=False, sampling=SAMPLE_WEIGHTED, update=UPDATE_ROW):
    """Apply steps j0..j0+nsteps-1 of Eq. (2) (step length gamma) to x in place.

    With ``trace`` returns (rows, r, err2): the row of each step, its residual
    a_i^T x - b_i before the step and, given x_true, ||x - x*||^2 before it.
    """
    rp, c, v = _csr(row_ptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    s = sampler or Sampler(m, rp, v)
    xt = None if x_true is None else np.ascontiguousarray(x_true, dtype=np.float64)
    rows = np.zeros(nsteps, dtype=np.int32) if trace else None
    rr = np.zeros(nsteps, dtype=np.float64) if trace else None
    e2 = np.zeros(nsteps, dtype=np.float64) if (trace and xt is not None) else None
    _load().oracle_rk_steps_ex(m, _p(rp), _p(c), _p(v), _p(bb), _p(s.w), _p(s.thr), _p(s.alias),
                               int(s.uniform), seed, stream, float(gamma), j0, nsteps, _p(x), n,
                               _p(xt), _p(rows), _p(rr), _p(e2), int(sampling), int(update))
    return (rows, rr, e2) if trace else None


def rk_solve(m, n, row_ptr, col, val, b, x, gamma, seed, tol, max_sweeps,
             check_every=1, x_true=None, stream=0, j0=0, sampling=SAMPLE_WEIGHTED,
             update=UPDATE_ROW):
    """Sequential RK to tolerance; x is updated in place.  Returns OracleResult."""
    rp, c, v = _csr(row_ptr, col, val)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    assert x.dtype == np.float64 and x.flags.c_contiguous
    xt = None if x_true is None else np.ascontiguousarray(x_true, dtype=np.float64)
    res = OracleResult()
    _load().oracle_rk_solve_ex(m, n, _p(rp), _p(c), _p(v), _p(bb), _p(x), float(gamma), seed,
                               stream, j0, float(tol), max_sweeps, check_every, _p(xt),
                               int(sampling), int(update), ctypes.byref(res))
    return res


# --------------------------------------------------------------------------
# Problem statistics (Section 1, "Notation and Assumption")
# --------------------------------------------------------------------------
def dense(m, n, row_ptr, col, val):
    A = np.zeros((m, n), dtype=np.float64)
    rp = np.asarray(row_ptr)
    for i in range(m):
        A[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return A


def spectrum(m, n, row_ptr, col, val):
    """(lambda_min nonzero, lambda_max) of A^T A by dense eigendecomposition."""
    A = dense(m, n, row_ptr, col, val)
    ev = np.linalg.eigvalsh(A.T @ A)
    tol = ev[-1] * max(m, n) * np.finfo(np.float64).eps * 10
    nz = ev[ev > tol]
    return float(nz[0]), float(ev[-1])


def mu_nu(m, n, row_ptr, col):
    """mu = max_i ||a_i||_0, nu = max_j ||abar_j||_0."""
    rp = np.asarray(row_ptr)
    mu = int(np.max(np.diff(rp)))
    nu = int(np.max(np.bincount(np.asarray(col), minlength=n)))
    return mu, nu


# --------------------------------------------------------------------------
# Step-length theory (Theorem 2, Corollary 2): formulas for reports and tests
# --------------------------------------------------------------------------
def theorem2_psi(mu, lmax, m, tau, rho):
    """psi = mu + 2 lambda_max tau rho^tau / m (the quantity of Theorem 2)."""
    return mu + 2.0 * lmax * tau * rho ** tau / m


def theorem2_step_bounds(mu, alpha, lmax, m, tau, rho):
    """The three upper bounds Theorem 2 puts on gamma: 1/psi,
    m (rho - 1) / (2 lambda_max rho^(tau+1)) and
    m sqrt((rho - 1) / (rho^tau (m alpha^2 + lambda_max^2 tau rho^tau)))."""
    psi = theorem2_psi(mu, lmax, m, tau, rho)
    b1 = 1.0 / psi
    b2 = m * (rho - 1.0) / (2.0 * lmax * rho ** (tau + 1))
    b3 = m * np.sqrt((rho - 1.0) / (rho ** tau * (m * alpha ** 2 + lmax ** 2 * tau * rho ** tau)))
    return b1, b2, b3


def corollary2(mu, lmax, m, tau):
    """(rho, psi, gamma) of Corollary 2: rho = 1 + 2 e lambda_max (tau + 1) / m,
    gamma = 1/psi; its assumption is 2 e lambda_max (tau + 1) / m <= 1."""
    rho = 1.0 + 2.0 * np.e * lmax * (tau + 1) / m
    psi = theorem2_psi(mu, lmax, m, tau, rho)
    return rho, psi, 1.0 / psi
