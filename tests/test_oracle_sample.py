"""Pins for the oracle's Born-rule sampling (the shots of Section VII) against
facts that do not come from it: exact rational inverse-CDF draws on states
whose probabilities are dyadic (every sum exact in FP64, so the draw is
decided exactly), closed-form outcomes of GHZ and basis states, the rule
that an outcome of probability zero is never drawn, and the empirical
frequencies of many draws against |psi|^2."""

from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(77)


def dyadic_state(n, rng, zero_frac=0.3):
    """Amplitudes (re, im) that are multiples of 1/16 in [-1, 1]: every
    |psi_i|^2 and every partial sum is an exact binary fraction in FP64."""
    N = 1 << n
    re = rng.integers(-16, 17, size=N) / 16.0
    im = rng.integers(-16, 17, size=N) / 16.0
    z = rng.random(N) < zero_frac
    re[z] = 0.0
    im[z] = 0.0
    if not np.any(re ** 2 + im ** 2):
        re[rng.integers(0, N)] = 0.5
    return (re + 1j * im).astype(np.complex128)


def exact_draw(psi, u):
    """Smallest i with sum_{j<=i} p_j > r in exact rationals, where
    r = u * sum_j p_j is the FP64 product (the precision the sampler
    decides in; u clamped to [0, 1]); the largest i with p_i > 0 when none
    exceeds. On dyadic states the total is exact, so r is the only rounding."""
    p = [Fraction(float(a.real)) ** 2 + Fraction(float(a.imag)) ** 2 for a in psi]
    total = sum(p)
    if total == 0:
        return -1
    assert float(total) == total  # exact in FP64
    uu = min(max(float(u), 0.0), 1.0) if u == u else 0.0
    r = Fraction(float(np.float64(uu) * np.float64(float(total))))
    s = Fraction(0)
    for i, pi in enumerate(p):
        s += pi
        if s > r:
            return i
    return max(i for i, pi in enumerate(p) if pi > 0)


def dyadic_uniforms(psi, rng, count):
    """Uniforms that land exactly on CDF boundaries (u = cdf_i / total, an
    exact FP64 value here) and just beside them, plus random ones."""
    p = np.abs(psi) ** 2
    c = np.cumsum(p)
    total = c[-1]
    picks = rng.integers(0, len(psi), size=count)
    on = c[picks] / total
    return np.concatenate([on, np.nextafter(on, 0), np.nextafter(on, 2), rng.random(count), [0.0, 1.0]])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_sample_matches_exact_rational_inverse_cdf(n):
    for trial in range(3):
        psi = dyadic_state(n, RNG)
        u = dyadic_uniforms(psi, RNG, 40)
        got = oracle.sample(psi, u)
        want = [exact_draw(psi, x) for x in u]
        assert list(got) == want


def test_sample_ghz_and_basis_states():
    for n in (2, 6, 12):
        psi = oracle.run_circuit(synth.ghz(n), synth.basis_state(n, 0))
        u = np.concatenate([RNG.random(500), [0.0, 1.0, np.nextafter(1.0, 0)]])
        got = oracle.sample(psi, u)
        assert set(got.tolist()) <= {0, (1 << n) - 1}
        # cdf_0 = |1/sqrt 2|^2 and the total = 2 |1/sqrt 2|^2 (exact doubling):
        # u below cdf_0 / total = 1/2 draws |0...0>, u at or above it |1...1>
        half = oracle.cdf(psi)[0] / oracle.cdf(psi)[-1]
        assert half == 0.5
        assert np.array_equal(got == 0, u < 0.5)
    for j in (0, 5, 31):
        psi = synth.basis_state(5, j) * (0.6 - 0.8j)
        assert set(oracle.sample(psi, RNG.random(100)).tolist()) == {j}


def test_sample_never_draws_zero_probability_and_clamps():
    psi = np.zeros(16, dtype=np.complex128)
    psi[[3, 4, 11]] = [0.5, 0.5j, np.sqrt(0.5)]
    u = np.array([0.0, -3.0, np.nan, 1.0, 7.0, 0.2499999, 0.25, 0.4999, 0.5, 0.99])
    got = oracle.sample(psi, u)
    assert list(got) == [3, 3, 3, 11, 11, 3, 4, 4, 11, 11]
    assert list(oracle.sample(np.zeros(8, complex), [0.1, 0.9])) == [-1, -1]


def test_sample_frequencies_follow_born_rule():
    """200 000 draws on a random 8-qubit state: Pearson chi-square of the
    counts against N p_i, with 255 degrees of freedom (mean 255, sd 22.6);
    a bound of 255 + 8 sd is exceeded with probability < 1e-9."""
    psi = synth.random_state(8, RNG)
    p = np.abs(psi) ** 2
    p /= p.sum()
    shots = 200_000
    idx = oracle.sample(psi, np.random.default_rng(5).random(shots))
    counts = np.bincount(idx, minlength=256)
    expected = shots * p
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    assert chi2 < 255 + 8 * 22.6, chi2


def test_sample_pins_reject_planted_mistakes():
    """Variants of the definition with a planted mistake fail the exact
    rational pin above: >= in place of > (draws at exact CDF boundaries),
    the CDF taken from the top of the index range, and r = u without the
    total."""
    psi = dyadic_state(5, np.random.default_rng(1), zero_frac=0.2) * 0.5
    u = dyadic_uniforms(psi, np.random.default_rng(2), 40)
    want = np.array([exact_draw(psi, x) for x in u])
    p = np.abs(psi) ** 2
    c = np.cumsum(p)
    ge = np.searchsorted(c, u * c[-1], side="left")            # smallest i with cdf_i >= r
    rev_c = np.cumsum(p[::-1])
    rev = len(p) - 1 - np.searchsorted(rev_c, u * c[-1], side="right")
    unnorm = np.minimum(np.searchsorted(c, u, side="right"), len(p) - 1)
    assert np.array_equal(oracle.sample(psi, u), want)
    for bad in (ge, rev, unnorm):
        assert not np.array_equal(bad, want)
