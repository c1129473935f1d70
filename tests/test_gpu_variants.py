"""GPU parity of the two variants against the FP64 oracle, through the C ABI.

Shuffled sweeps (rows without replacement, a fresh order each sweep, Section 5):
  * the GPU's row sequence equals the oracle's bit for bit, across sweep
    boundaries, at awkward m and at a 2^22-row system (sampled);
  * the single-worker FP64 iterate matches the oracle's to 1e-12;
  * async FP32 solves converge, and on a Table 2 shape they need no more
    sweeps than the oracle's sequential shuffled solve (x1.5);
  * the multi-system engine runs them too.

Single-coordinate update (Algorithm 1, x_t -= gamma theta_i A_it r / ||a_i||^2):
  * the single-worker FP64 iterate matches the oracle's to 1e-12, with both
    samplers;
  * async solves with tau inside Corollary 2's range and gamma = 1/(mu + 1)
    reach 1e-6 within Theorem 3's projection count.
"""
import numpy as np
import pytest

import oracle
from paper_1401_4780_gb300 import asyrk, synth

pytestmark = pytest.mark.gpu

SH = oracle.SAMPLE_SHUFFLED


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    asyrk.load()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("m", [7, 1000, 4097, 65537])
def test_shuffled_sequence_is_bit_exact(m):
    s = synth.make_system(m, 64, 4, 17 + m, row_norms="lognormal", value_dtype="f32")
    seed = synth.solver_seed(s.seed)
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    with asyrk.Problem.from_system(s) as p:
        for j0, count, stream in [(0, 5 * m + 3, 0), (m - 2, 3 * m, 5),
                                  (2**32 - 700, 1400, 0), (2**40 + 3 * m, m, 9)]:
            got = p.draw_rows(j0, count, stream, sampling=asyrk.SAMPLE_SHUFFLED)
            want = oracle.draw_rows(seed, stream, j0, count, samp.thr, samp.alias, samp.uniform,
                                    sampling=SH)
            np.testing.assert_array_equal(got, want)
        # a whole sweep is a permutation of the rows on the GPU as well
        k0 = 3 * m
        sweep = p.draw_rows(k0, m, 2, sampling=asyrk.SAMPLE_SHUFFLED)
        assert np.array_equal(np.sort(sweep), np.arange(m))


def test_shuffled_sequence_large_system_sampled():
    m = 1 << 22
    s = synth.make_system(m, 1 << 10, 2, 3, row_norms="unit", value_dtype="f32")
    seed = synth.solver_seed(s.seed)
    samp = oracle.Sampler(s.m, s.row_ptr, s.val64)
    with asyrk.Problem.from_system(s) as p:
        got = p.draw_rows(m - 50_000, 100_000, 1, sampling=asyrk.SAMPLE_SHUFFLED)
        want = oracle.draw_rows(seed, 1, m - 50_000, 100_000, samp.thr, samp.alias, samp.uniform,
                                sampling=SH)
        np.testing.assert_array_equal(got, want)
        sweep = p.draw_rows(7 * m, m, 0, sampling=asyrk.SAMPLE_SHUFFLED)
        assert np.array_equal(np.sort(sweep), np.arange(m))


def _oracle_iterate(s, seed, nsteps, gamma, sampling, update):
    x = np.zeros(s.n)
    oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, gamma, seed, 0, 0, nsteps,
                    sampling=sampling, update=update)
    return x


CASES = [
    ("shuffled rows", oracle.SAMPLE_SHUFFLED, oracle.UPDATE_ROW),
    ("weighted single", oracle.SAMPLE_WEIGHTED, oracle.UPDATE_SINGLE),
    ("shuffled single", oracle.SAMPLE_SHUFFLED, oracle.UPDATE_SINGLE),
]


@pytest.mark.parametrize("name,sampling,update", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("subwarp", [1, 4, 32])
def test_sequential_iterate_matches_oracle(name, sampling, update, subwarp):
    s = synth.make_system(3001, 700, (1, 40), 8, row_norms="lognormal", value_dtype="f64")
    seed = synth.solver_seed(s.seed)
    gamma = 0.7 if update == oracle.UPDATE_ROW else 1.0 / oracle.mu_nu(s.m, s.n, s.row_ptr,
                                                                         s.col)[0]
    sweeps = 4
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, gamma=gamma, tol=0.0, max_sweeps=sweeps,
                           mode=asyrk.MODE_SEQUENTIAL, subwarp=subwarp, sampling=sampling,
                           update=update)
        assert st == asyrk.OK and info.projections == sweeps * s.m
    xo = _oracle_iterate(s, seed, sweeps * s.m, gamma, sampling, update)
    assert _rel(x, xo) <= 1e-12


@pytest.mark.parametrize("form", [asyrk.FORM_THROUGHPUT, asyrk.FORM_LATENCY])
def test_async_one_worker_shuffled_sweeps_match_oracle(form):
    # both forms of the ASYNC kernel on Section 5's shuffled sweeps: with one
    # worker the iterate is the oracle's sequential one on the same permutations
    s = synth.make_system(3001, 700, (1, 40), 8, row_norms="lognormal", value_dtype="f64")
    seed = synth.solver_seed(s.seed)
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, gamma=0.7, tol=0.0, max_sweeps=3, mode=asyrk.MODE_ASYNC,
                           workers=1, subwarp=4, sampling=asyrk.SAMPLE_SHUFFLED,
                           kernel_form=form)
        assert st == asyrk.OK and info.projections == 3 * s.m
    xo = _oracle_iterate(s, seed, 3 * s.m, 0.7, oracle.SAMPLE_SHUFFLED, oracle.UPDATE_ROW)
    assert _rel(x, xo) <= 1e-12


def test_async_shuffled_converges():
    s = synth.plain_f64_system()
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, tol=1e-10, max_sweeps=400, sampling=asyrk.SAMPLE_SHUFFLED,
                           x_true=s.x_true)
        assert st == asyrk.OK, info.as_dict()
    assert _rel(x, s.x_true) <= 1e-10


def _oracle_shuffled_sweeps_to_normal(s, tol, seed, max_sweeps=3000):
    x = np.zeros(s.n)
    for k in range(1, max_sweeps + 1):
        oracle.rk_steps(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x, 1.0, seed, 0,
                        (k - 1) * s.m, s.m, sampling=SH)
        g = oracle.normal_residual(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x)
        if float(g @ g) <= tol:
            return k
    raise AssertionError("oracle did not reach the threshold")


def test_async_shuffled_table2_measure_within_oracle_sweeps():
    s = synth.make_system(8000, 10000, ("poisson", 10), 41, row_norms="unit", value_dtype="f32")
    seed = synth.solver_seed(s.seed)
    med = np.median([_oracle_shuffled_sweeps_to_normal(s, 1e-5, seed + k) for k in range(3)])
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, tol=1e-5, max_sweeps=3000, measure=asyrk.MEASURE_NORMAL_RESIDUAL,
                           sampling=asyrk.SAMPLE_SHUFFLED)
        assert st == asyrk.OK, info.as_dict()
        assert info.sweeps <= 1.5 * med, (info.sweeps, med)
    g = oracle.normal_residual(s.m, s.n, s.row_ptr, s.col, s.val64, s.b, x)
    assert float(g @ g) <= 1e-5


@pytest.mark.parametrize("sampling", [asyrk.SAMPLE_WEIGHTED, asyrk.SAMPLE_SHUFFLED])
def test_async_single_coordinate_meets_theorem3_count(sampling):
    # unit rows, so Algorithm 1's setting; tau = workers within Corollary 2's
    # 2 e lambda_max (tau + 1) / m <= 1, and gamma = 1/(mu + 1) <= 1/psi
    s = synth.make_system(8192, 2048, 16, 12, row_norms="unit", value_dtype="f64")
    lmin, lmax = oracle.spectrum(s.m, s.n, s.row_ptr, s.col, s.val64)
    mu, _ = oracle.mu_nu(s.m, s.n, s.row_ptr, s.col)
    workers = 128
    assert 2 * np.e * lmax * (workers + 1) / s.m <= 1.0
    tol, eta = 1e-6, 0.1
    # Theorem 3: j >= m (mu + 1)/lambda_min |log(||x0 - x*||^2 / (eta eps))| projections
    # give ||x_j - x*||^2 <= eps with probability >= 1 - eta (x0 = 0, eps = tol^2 ||x*||^2)
    j_bound = s.m * (mu + 1) / lmin * abs(np.log(1.0 / (eta * tol * tol)))
    with asyrk.Problem.from_system(s) as p:
        x = np.zeros(s.n)
        st, info = p.solve(x, gamma=1.0 / (mu + 1), tol=tol, max_sweeps=int(j_bound / s.m) + 1,
                           workers=workers, update=asyrk.UPDATE_SINGLE, sampling=sampling,
                           x_true=s.x_true)
        assert st == asyrk.OK, info.as_dict()
        assert info.projections <= j_bound
    assert _rel(x, s.x_true) <= tol


@pytest.mark.parametrize("sampling,update", [(asyrk.SAMPLE_SHUFFLED, asyrk.UPDATE_ROW),
                                             (asyrk.SAMPLE_WEIGHTED, asyrk.UPDATE_SINGLE)])
def test_batch_runs_the_variants(sampling, update):
    systems = [synth.make_system(2000 + 500 * k, 400, 8, 60 + k, row_norms="unit",
                                 value_dtype="f32") for k in range(3)]
    probs = [asyrk.Problem.from_system(s) for s in systems]
    try:
        gammas = [1.0 if update == asyrk.UPDATE_ROW
                  else 1.0 / oracle.mu_nu(s.m, s.n, s.row_ptr, s.col)[0] for s in systems]
        with asyrk.Batch(probs, sampling=sampling, update=update) as b:
            xs = [np.zeros(s.n) for s in systems]
            st, infos, _ = b.solve(xs, gammas=gammas, tols=[1e-6] * 3, max_sweeps=3000,
                                   x_trues=[s.x_true for s in systems])
            assert st == asyrk.OK, [i.as_dict() for i in infos]
        for x, s in zip(xs, systems):
            assert _rel(x, s.x_true) <= 1e-6
    finally:
        for p in probs:
            p.close()
