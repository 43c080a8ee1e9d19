"""GPU parity of the FP64 reductions: norm, Pauli-sum expectation and the
Pauli-sum apply lambda = H psi."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, dev, host, maxerr

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(99)


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _random_obs(n, terms, complex_coeff=False):
    xs = RNG.integers(0, 1 << n, size=terms).astype(np.uint64)
    zs = RNG.integers(0, 1 << n, size=terms).astype(np.uint64)
    xs[: terms // 3] = 0  # several terms share the zero X mask
    cs = RNG.standard_normal(terms) + (1j * RNG.standard_normal(terms) if complex_coeff else 0)
    return synth.Observable(xs, zs, cs)


@pytest.mark.parametrize("n", [1, 5, 12, 17])
def test_norm(api, n):
    psi = synth.random_state(n, RNG) * 1.7
    assert abs(api.norm(dev(psi)) - oracle.norm2(psi)) <= 1e-13 * oracle.norm2(psi)
    p32 = dev(psi, torch.complex64)
    ref32 = oracle.norm2(host(p32))
    assert abs(api.norm(p32) - ref32) <= 1e-6 * ref32


@pytest.mark.parametrize("n", [1, 6, 11, 15])
def test_expect_matches_oracle(api, n):
    psi = synth.random_state(n, RNG)
    for complex_coeff in (False, True):
        obs = _random_obs(n, 9, complex_coeff)
        want = oracle.expect(psi, obs)
        got = api.expect(dev(psi), obs.xmask, obs.zmask, obs.coeff)
        assert abs(got - want) <= TOL_C128
        p32 = dev(psi, torch.complex64)
        want32 = oracle.expect(host(p32), obs)
        got32 = api.expect(p32, obs.xmask, obs.zmask, obs.coeff)
        assert abs(got32 - want32) <= 1e-6 * float(np.sum(np.abs(obs.coeff)))


def test_expect_special_cases(api):
    n = 8
    ghz = oracle.run_circuit(synth.ghz(n), synth.basis_state(n, 0))
    g = dev(ghz)
    for i, j in ((0, 1), (2, 7), (3, 5)):
        assert abs(api.expect(g, [0], [(1 << i) | (1 << j)], [1.0]) - 1.0) < 1e-15
    assert abs(api.expect(g, [(1 << n) - 1], [0], [1.0]) - 1.0) < 1e-15
    assert abs(api.expect(g, [0], [1], [1.0])) < 1e-15
    plus = dev(np.full(1 << n, 1 / math.sqrt(1 << n), dtype=np.complex128))
    for q in range(n):
        assert abs(api.expect(plus, [1 << q], [0], [1.0]) - 1.0) < 1e-15
        assert abs(api.expect(plus, [1 << q], [1 << q], [1.0])) < 1e-15
    for j in (0, 37, 255):
        b = dev(synth.basis_state(n, j))
        for q in range(n):
            assert api.expect(b, [0], [1 << q], [1.0]) == (-1.0 if (j >> q) & 1 else 1.0)
    assert api.expect(g, [], [], []) == 0  # empty observable


@pytest.mark.parametrize("n", [2, 9, 14])
def test_pauli_sum_apply(api, n):
    psi = synth.random_state(n, RNG)
    obs = _random_obs(n, 7, complex_coeff=True)
    lam = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    api.apply_pauli_sum(dev(psi), lam, obs.xmask, obs.zmask, obs.coeff)
    assert maxerr(host(lam), oracle.apply_pauli_sum(psi, obs)) <= TOL_C128 * max(1, float(np.sum(np.abs(obs.coeff))))


def test_reductions_deterministic(api):
    n = 20
    p = dev(synth.random_state(n, RNG))
    obs = synth.ansatz_observable(n)
    a = [api.norm(p) for _ in range(3)]
    b = [api.expect(p, obs.xmask, obs.zmask, obs.coeff) for _ in range(3)]
    assert len(set(a)) == 1 and len(set(b)) == 1


def test_reduction_errors(api):
    from paper_2405_01250_gb300._native import DiaqError
    p = dev(synth.random_state(4, RNG))
    with pytest.raises(DiaqError, match="qubit"):
        api.expect(p, [1 << 5], [0], [1.0])
    with pytest.raises(DiaqError, match="overlap"):
        api.apply_pauli_sum(p, p, [0], [1], [1.0])
