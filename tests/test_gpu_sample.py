"""GPU parity of Born-rule shot sampling (diaq_sample) against the oracle's
inverse-CDF draws on the same uniforms.

Bit-exact where the cumulative sums are exact (dyadic probabilities, GHZ);
on general states the GPU sums in another order, so a uniform whose r lies
within the summation-rounding bound of a CDF boundary may draw the
neighbouring index: such shots are detected, counted and printed, and every
other shot must match exactly."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import qft_amplitudes

pytestmark = pytest.mark.gpu

DTYPES = [torch.complex128, torch.complex64]


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _dyadic(n, rng, zero_frac=0.3):
    N = 1 << n
    re = rng.integers(-16, 17, size=N) / 16.0
    im = rng.integers(-16, 17, size=N) / 16.0
    z = rng.random(N) < zero_frac
    re[z] = 0.0
    im[z] = 0.0
    re[rng.integers(0, N)] = 0.75
    return (re + 1j * im).astype(np.complex128)


def _uniforms(psi, rng, count):
    """Random uniforms plus ones that hit CDF boundaries exactly and just
    beside them, and the ends of [0, 1]."""
    c = oracle.cdf(psi)
    on = c[rng.integers(0, len(psi), size=count)] / c[-1]
    return np.concatenate([rng.random(count), on, np.nextafter(on, 0), np.nextafter(on, 2),
                           [0.0, 1.0, np.nextafter(1.0, 0), -0.5, 2.0, np.nan]])


def _gpu_sample(api, psi, u, dtype):
    x = torch.as_tensor(psi).to(device="cuda", dtype=dtype)
    return api.sample(x, torch.as_tensor(u, dtype=torch.float64).cuda()).cpu().numpy()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 5, 10, 11, 12, 13, 16, 19, 22])
def test_sample_bit_exact_on_dyadic_states(api, n, dtype):
    """Probabilities that are multiples of 2^-8: every partial sum on both
    sides is exact, so every draw - including uniforms exactly on a CDF
    boundary - must equal the oracle's. n spans a partial tile (< 2048
    amplitudes), one and several tiles, and 1 to 3 tree levels above them."""
    rng = np.random.default_rng(100 + n)
    psi = _dyadic(n, rng)
    u = _uniforms(psi, rng, 300)
    want = oracle.sample(psi, u)
    got = _gpu_sample(api, psi, u, dtype)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


@pytest.mark.parametrize("dtype", DTYPES)
def test_sample_ghz12_only_two_outcomes(api, dtype):
    n = 12
    x = torch.zeros(1 << n, dtype=dtype, device="cuda")
    x[0] = 1
    for g in synth.ghz(n).gates:
        api.apply(api.build(g, n, dtype=dtype), x, x)
    u = np.random.default_rng(3).random(1024)
    got = api.sample(x, u).cpu().numpy()
    assert set(got.tolist()) <= {0, (1 << n) - 1}
    assert np.array_equal(got, oracle.sample(x.cpu().numpy().astype(np.complex128), u))
    assert 400 < int(np.sum(got == 0)) < 624  # 1024 fair coin flips


def _ambiguity_bound(n, dtype, total):
    """Largest possible difference between the GPU's and the oracle's running
    sums at any index: each is a sum of at most N + 2 rounded FP64
    operations per term chain (recursive-summation bound (N + 2) u sum|x|),
    the complex64 runs add their FP32-pair error (below 2^-40 relative), and
    r = u * total is rounded on each side."""
    N = 1 << n
    u64 = 2.0 ** -53
    b = 2 * (N + 4) * u64 * total
    if dtype == torch.complex64:
        b += 2.0 ** -40 * total
    return b


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("zero_frac", [0.0, 0.5])
def test_sample_random20_matches_oracle_outside_rounding_ties(api, dtype, zero_frac):
    n = 20
    rng = np.random.default_rng(7)
    psi = synth.random_state(n, rng)
    psi[rng.random(1 << n) < zero_frac] = 0
    psi = psi.astype(np.complex64 if dtype == torch.complex64 else np.complex128).astype(np.complex128)
    u = np.concatenate([rng.random(4096), [0.0, 1.0, np.nextafter(1.0, 0)]])
    want = oracle.sample(psi, u)
    got = _gpu_sample(api, psi, u, dtype)
    p = np.abs(psi) ** 2
    assert np.all(p[got] > 0)  # never an outcome of zero probability
    c = oracle.cdf(psi)
    delta = _ambiguity_bound(n, dtype, c[-1])
    ties = 0
    for s in np.nonzero(got != want)[0]:
        a, b = sorted((int(got[s]), int(want[s])))
        r = u[s] * c[-1]
        assert np.all(np.abs(c[a:b] - r) <= delta), (s, got[s], want[s])
        ties += 1
    print(f"random-{n} {dtype} zeros {zero_frac}: {len(u)} shots, {ties} within rounding of a CDF "
          f"boundary (bound {delta:.2e} of total {c[-1]:.6f})")
    assert ties <= 8


@pytest.mark.parametrize("dtype", DTYPES)
def test_sample_edge_cases(api, dtype):
    # a single amplitude at the very end, zeros before it
    psi = np.zeros(1 << 13, dtype=np.complex128)
    psi[-1] = 1j
    u = np.array([0.0, 0.5, 1.0, -1.0, np.nan, 3.0])
    assert _gpu_sample(api, psi, u, dtype).tolist() == [8191] * 6
    # the first amplitude only
    psi = np.zeros(1 << 12, dtype=np.complex128)
    psi[0] = 0.5
    assert _gpu_sample(api, psi, u, dtype).tolist() == [0] * 6
    # a zero state: -1 for every shot
    assert _gpu_sample(api, np.zeros(1 << 9, complex), u, dtype).tolist() == [-1] * 6
    # no shots: nothing to do
    x = torch.zeros(16, dtype=dtype, device="cuda")
    assert api.sample(x, torch.zeros(0, dtype=torch.float64, device="cuda")).numel() == 0


def test_sample_frequencies_follow_born_rule(api):
    """One million GPU shots of a random 12-qubit complex128 state: Pearson
    chi-square against shots * p_i with 4095 degrees of freedom (sd 90.5);
    the bound 4095 + 8 sd is exceeded with probability below 1e-9."""
    n = 12
    psi = synth.random_state(n, np.random.default_rng(8))
    u = torch.rand(1_000_000, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    got = api.sample(torch.as_tensor(psi).cuda(), u).cpu().numpy()
    p = np.abs(psi) ** 2
    p /= p.sum()
    counts = np.bincount(got, minlength=1 << n)
    e = 1_000_000 * p
    chi2 = float(np.sum((counts - e) ** 2 / e))
    assert chi2 < 4095 + 8 * 90.5, chi2


def test_sample_full_size_qft28_and_ghz30(api):
    """Full size in the benchmark's configuration: the QFT-28 state of a
    basis state has |psi_k|^2 = 1/N for every k (closed form), so shot u draws
    floor(u N) up to one index of rounding; GHZ-30 in complex64 (8 GiB)
    draws only |0...0> and |1...1>."""
    n = 28
    circ, j = synth.qft(n, seed=0)
    x = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    x[j] = 1
    y = torch.empty_like(x)
    for g in circ.gates:
        api.apply(api.build(g, n), x, y)
        x, y = y, x
    del y
    ks = np.random.default_rng(1).integers(0, 1 << n, size=64)
    got_amp = x[torch.as_tensor(ks).cuda()].cpu().numpy()
    assert np.max(np.abs(got_amp - qft_amplitudes(n, j, ks))) < 1e-12
    u = np.random.default_rng(2).random(1024)
    idx = api.sample(x, u).cpu().numpy()
    assert np.all(np.abs(idx - np.floor(u * (1 << n))) <= 1)
    del x
    torch.cuda.empty_cache()
    n = 30
    x = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    x[0] = 1
    for g in synth.ghz(n).gates:
        api.apply(api.build(g, n, dtype=torch.complex64), x, x)
    idx = api.sample(x, u).cpu().numpy()
    assert set(idx.tolist()) <= {0, (1 << n) - 1}
    assert np.array_equal(idx == 0, u < 0.5)
    del x
    torch.cuda.empty_cache()


def test_sample_rejects_bad_arguments(api):
    from paper_2405_01250_gb300 import _native
    L = _native.lib()
    x = torch.zeros(16, dtype=torch.complex128, device="cuda")
    u = torch.zeros(4, dtype=torch.float64, device="cuda")
    o = torch.zeros(4, dtype=torch.int64, device="cuda")
    import ctypes
    vp = ctypes.c_void_p
    assert L.diaq_sample(None, 4, 1, vp(u.data_ptr()), 4, vp(o.data_ptr()), None) == 1
    assert L.diaq_sample(vp(x.data_ptr()), 4, 1, None, 4, vp(o.data_ptr()), None) == 1
    assert L.diaq_sample(vp(x.data_ptr()), 4, 1, vp(u.data_ptr()), -1, vp(o.data_ptr()), None) == 1
    assert L.diaq_sample(vp(x.data_ptr()), 4, 1, vp(u.data_ptr() + 4), 2, vp(o.data_ptr()), None) == 1
    assert L.diaq_sample(vp(x.data_ptr()), 4, 1, None, 0, None, None) == 0
