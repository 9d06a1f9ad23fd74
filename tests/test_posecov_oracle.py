"""Pins of the pose-covariance oracle (oracle/posecov.py).

The main pins do not use the oracle's arithmetic: for samples of a 6-D
Gaussian, a fit to the ones inside 3 sigma has covariance
Sigma P(chi2_8 <= 9) / P(chi2_6 <= 9) (the second moment of a chi2_6
variable below c is 6 P(chi2_8 <= c)), and refitting over and over
shrinks it to the fixed point s^2 Sigma of
s^2 = P(chi2_8 <= 9 s^2) / P(chi2_6 <= 9 s^2)."""
import numpy as np
import pytest
from scipy import optimize, stats

from oracle import geometry, posecov

EPS = 1e-12


def _spd(rng, scale):
    A = rng.normal(size=(6, 6))
    S = A @ A.T / 6 + np.eye(6)
    D = np.diag(np.sqrt(scale))
    return D @ S @ D / np.mean(np.diag(S))


def _draw(rng, mu, Sigma, n):
    L = np.linalg.cholesky(Sigma)
    return [geometry.compose(mu, geometry.se3_exp(L @ rng.normal(size=6))) for _ in range(n)]


def _mu(rng):
    return geometry.se3_exp(np.concatenate([rng.normal(size=3) * 0.1, rng.normal(size=3)]))


def test_one_3_sigma_round_gives_the_truncated_chi2_moment():
    # one round from the true Gaussian keeps P(chi2_6 <= 9) of the samples
    # and fits E[d d^T | d^T S^-1 d <= 9] = S P(chi2_8 <= 9) / P(chi2_6 <= 9)
    rng = np.random.default_rng(0)
    Sigma = _spd(rng, np.array([1e-6] * 3 + [4e-6] * 3))
    mu = _mu(rng)
    samples = _draw(rng, mu, Sigma, 20000)
    shrink = stats.chi2.cdf(9, 8) / stats.chi2.cdf(9, 6)
    m, S, n_in, rounds, deg = posecov.fit(samples, mu, EPS, sigma0=Sigma, max_rounds=1)
    assert not deg and rounds == 1
    assert n_in / len(samples) == pytest.approx(stats.chi2.cdf(9, 6), abs=0.01)
    err = np.linalg.norm(S - shrink * Sigma) / np.linalg.norm(shrink * Sigma)
    assert err < 0.05, (err, shrink)
    dm = geometry.se3_log(geometry.compose(geometry.inverse(mu), m))
    assert np.all(np.abs(dm) < 4 * np.sqrt(np.diag(Sigma) / 1000))


def test_repeated_rounds_approach_the_chi2_fixed_point():
    # repeated rounds shrink it to s^2 S, s^2 = P(chi2_8 <= 9 s^2) / P(chi2_6 <= 9 s^2)
    # (the fit's sensitivity near that point, 1 / (1 - 0.83), widens the band)
    rng = np.random.default_rng(6)
    Sigma = _spd(rng, np.array([1e-6] * 3 + [4e-6] * 3))
    mu = _mu(rng)
    samples = _draw(rng, mu, Sigma, 6000)
    g = lambda s2: s2 - stats.chi2.cdf(9 * s2, 8) / stats.chi2.cdf(9 * s2, 6)
    s2 = optimize.brentq(g, 0.3, 1.0)
    _, S, _, rounds, deg = posecov.fit(samples, mu, EPS, sigma0=Sigma, max_rounds=400)
    assert not deg and rounds < 400
    assert np.linalg.norm(S - s2 * Sigma) / np.linalg.norm(s2 * Sigma) < 0.3


def test_outliers_are_discarded():
    rng = np.random.default_rng(1)
    Sigma = _spd(rng, np.array([4e-6] * 3 + [1e-4] * 3))
    mu = _mu(rng)
    inl = _draw(rng, mu, Sigma, 3000)
    out = [geometry.compose(mu, geometry.se3_exp(np.concatenate(
        [rng.normal(size=3) * rng.uniform(0.3, 1.0), rng.normal(size=3)]))) for _ in range(1000)]
    mixed = list(inl) + out
    rng.shuffle(mixed)
    _, S_clean, _, _, _ = posecov.fit(inl, mu, EPS)
    m, S, n_in, _, deg = posecov.fit(mixed, mu, EPS)
    assert not deg and n_in <= len(inl)
    assert np.linalg.norm(S - S_clean) / np.linalg.norm(S_clean) < 0.1


def test_symmetric_star_closed_form():
    # samples mu exp(+-a e_k), k = 1..6: mean mu, Sigma = (2 a^2 / 12) I
    mu = _mu(np.random.default_rng(2))
    a = 1e-3
    samples = [geometry.compose(mu, geometry.se3_exp(sg * a * np.eye(6)[k]))
               for k in range(6) for sg in (1.0, -1.0)]
    m, S, n_in, rounds, deg = posecov.fit(samples, mu, EPS, sigma0=a * a * np.eye(6))
    assert not deg and n_in == 12 and rounds == 2
    assert np.allclose(S, a * a / 6 * np.eye(6), rtol=1e-9, atol=1e-18)
    assert np.allclose(m, mu, atol=1e-12)


def test_eigenvalue_floor_and_symmetry():
    rng = np.random.default_rng(3)
    mu = _mu(rng)
    # rotation-only samples: the translation block has zero variance
    samples = [geometry.compose(mu, geometry.se3_exp(np.concatenate([rng.normal(size=3) * 1e-3,
                                                                     np.zeros(3)])))
               for _ in range(200)]
    eps = 1e-10
    _, S, _, _, deg = posecov.fit(samples, mu, eps)
    assert not deg and np.array_equal(S, S.T) or np.allclose(S, S.T, atol=1e-20)
    w = np.linalg.eigvalsh(S)
    assert np.sum(np.isclose(w, eps, rtol=1e-6)) == 3 and np.all(w >= eps * (1 - 1e-9))


def test_few_samples_are_degenerate_and_the_fit_is_a_fixed_point():
    rng = np.random.default_rng(4)
    mu = _mu(rng)
    sigma0 = np.diag([1e-6] * 3 + [1e-4] * 3)
    few = _draw(rng, mu, sigma0, 5)
    m, S, n_in, rounds, deg = posecov.fit(few, mu, EPS)
    assert deg and np.array_equal(m, mu) and np.allclose(S, EPS * np.eye(6))
    samples = _draw(rng, mu, sigma0, 400)
    m, S, _, _, deg = posecov.fit(samples, mu, EPS)
    m2, S2, _, rounds2, deg2 = posecov.fit(samples, m, EPS, sigma0=S)
    assert not deg and not deg2 and rounds2 == 2
    assert np.allclose(m2, m, atol=1e-12) and np.allclose(S2, S, rtol=1e-9, atol=1e-20)


def test_six_samples_cannot_give_a_covariance():
    # a 6-D covariance needs 7 samples: 6 (however spread) are degenerate
    mu = _mu(np.random.default_rng(8))
    a = 1e-3
    six = [geometry.compose(mu, geometry.se3_exp(sg * a * np.eye(6)[k]))
           for k in range(3) for sg in (1.0, -1.0)]
    m, S, n_in, rounds, deg = posecov.fit(six, mu, EPS, sigma0=a * a * np.eye(6))
    assert deg and n_in == 6 and rounds == 0


def test_robust_start_is_the_gaussian_scale_and_ignores_outliers():
    # median |x| of N(0, s^2) is 0.67449 s, so 1.4826 median |x| = s
    rng = np.random.default_rng(7)
    sd = np.array([2e-3, 1e-3, 3e-3, 0.05, 0.02, 0.04])
    mu = _mu(rng)
    samples = _draw(rng, mu, np.diag(sd ** 2), 20000)
    s = np.sqrt(np.diag(posecov.robust_start(samples, mu)))
    assert np.allclose(s, sd, rtol=0.03)
    # a third of the samples replaced by wild ones: the scale moves by the
    # quantile shift of a 2/3 mixture, not by the outliers' size
    wild = [geometry.compose(mu, geometry.se3_exp(np.concatenate(
        [rng.normal(size=3), rng.normal(size=3) * 10]))) for _ in range(10000)]
    s2 = np.sqrt(np.diag(posecov.robust_start(samples[:20000] + wild, mu)))
    assert np.all(s2 < 2.5 * sd) and np.all(s2 > sd)
