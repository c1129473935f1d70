"""Theorem 2 / Corollary 2 formulas of the oracle's tooling (CPU only).

  * where rho^tau <= e holds (2 e lambda_max (tau+1) tau / m <= 1), Corollary 2's
    step 1/psi satisfies all three of Theorem 2's bounds on gamma (with
    alpha = sqrt(lambda_max) mu, the bound alpha <= ||A|| mu stated with the
    notation, which the proof uses) and psi <= mu + 1, as the proof concludes;
  * with only the corollary's stated assumption 2 e lambda_max (tau+1)/m <= 1,
    rho^tau can exceed e and psi exceed mu + 1: the proof bounds rho^tau as if
    rho were 1 + 2 e lambda_max / m (the reading the GPU test of Algorithm 1
    follows by taking gamma = 1/(mu + 1));
  * on a real matrix, the rate of Theorem 2 with gamma = 1/(mu+1) and tau = 0 is
    Theorem 1's, pinned elsewhere by simulation.
"""
import numpy as np

import oracle


def test_corollary2_step_meets_theorem2_where_rho_tau_is_at_most_e():
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(2000):
        m = int(rng.integers(100, 10**7))
        lmax = float(rng.uniform(0.5, 20.0))
        mu = int(rng.integers(1, 200))
        tau = int(rng.integers(0, 1000))
        if 2 * np.e * lmax * (tau + 1) * max(tau, 1) / m > 1.0:
            continue
        rho, psi, gamma = oracle.corollary2(mu, lmax, m, tau)
        assert rho ** tau <= np.e * (1 + 1e-12)
        assert psi <= mu + 1 + 1e-12
        # alpha <= ||A|| mu = sqrt(lambda_max) mu (Section 1), the bound the proof uses
        b1, b2, b3 = oracle.theorem2_step_bounds(mu, np.sqrt(lmax) * mu, lmax, m, tau, rho)
        assert gamma <= b1 * (1 + 1e-12) and gamma <= b2 and gamma <= b3
        checked += 1
    assert checked > 200


def test_the_stated_assumption_alone_does_not_keep_psi_below_mu_plus_one():
    m, lmax, mu, tau = 1000, 1.0, 16, 50
    assert 2 * np.e * lmax * (tau + 1) / m <= 1.0  # the corollary's assumption holds
    rho, psi, gamma = oracle.corollary2(mu, lmax, m, tau)
    assert rho ** tau > np.e and psi > mu + 1
    # Theorem 2 still holds for gamma = 1/psi (it meets all three bounds) ...
    b1, b2, b3 = oracle.theorem2_step_bounds(mu, 4.0 * mu, lmax, m, tau, rho)
    assert gamma <= b1 * (1 + 1e-12) and gamma <= b2 and gamma <= b3
    # ... but its rate 1 - lambda_min gamma (2 - gamma psi)/m = 1 - lambda_min/(m psi) is
    # slower than the corollary's 1 - lambda_min/(m (mu + 1))
    assert 1.0 / psi < 1.0 / (mu + 1)
