"""GPU parity of the DiaQ gate apply (both variants), the builder's stored
diagonals, fusion and the GHZ / QFT workloads against the FP64 oracle."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, dev, host, maxerr, qft_amplitudes, tol_c64

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(2024)
KINDS = ["dense", "real", "diag", "perm", "monomial", "sparse"]


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _check(api, n, targets, m, dtype, variant, inplace=False):
    x = synth.random_state(n, RNG)
    want = oracle.apply_gate(x, targets, m)
    xt = dev(x, dtype)
    op = api.build(synth.Gate(tuple(targets), m), n, dtype=dtype, variant=variant)
    yt = xt if inplace else torch.empty_like(xt)
    api.apply(op, xt, yt)
    got = host(yt)
    if dtype == torch.complex128:
        tol = TOL_C128
    else:
        tol = tol_c64(len(targets), float(np.max(np.abs(x))) * float(np.max(np.abs(m))))
    err = maxerr(got, want)
    assert err <= tol, (n, targets, variant, dtype, err, tol)
    return op


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_onthefly_small_k_all_classes_and_placements(api, dtype, k):
    for n in (k, k + 2, 9, 14):
        for kind in KINDS:
            t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
            _check(api, n, t, synth.random_gate(k, RNG, kind), dtype, "onthefly")
        # extreme placements: lowest, highest, reversed order
        _check(api, n, list(range(k)), synth.random_gate(k, RNG), dtype, "onthefly")
        _check(api, n, list(range(n - 1, n - 1 - k, -1)), synth.random_gate(k, RNG), dtype, "onthefly")


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("k", [4, 5, 6])
def test_onthefly_large_k(api, dtype, k):
    for n in (k, k + 3, 13):
        for kind in ("dense", "diag", "perm", "sparse"):
            t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
            _check(api, n, t, synth.random_gate(k, RNG, kind), dtype, "onthefly")


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_onthefly_in_place(api, dtype):
    for k in (1, 2, 3, 5):
        n = 11
        t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
        _check(api, n, t, synth.random_gate(k, RNG), dtype, "onthefly", inplace=True)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_stored_variant(api, dtype, k):
    for n in (k, k + 2, 10):
        for kind in ("dense", "real", "diag", "perm", "sparse"):
            t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
            _check(api, n, t, synth.random_gate(k, RNG, kind), dtype, "stored")


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_stored_real_or_imaginary_entries(api, dtype):
    """Stored gate ops whose entries are each real or purely imaginary (RX,
    Y, iSWAP and products of such) take the kernel that multiplies one half
    of each value; ops with a complex entry and all-real ops the others."""
    rx = np.array([[math.cos(0.35), -1j * math.sin(0.35)], [-1j * math.sin(0.35), math.cos(0.35)]])
    y = np.array([[0, -1j], [1j, 0]])
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    iswap = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]])
    gates = [rx, y, iswap, np.kron(y, rx), np.kron(np.kron(y, x), rx), np.kron(rx, iswap)]
    n = 10
    for m in gates:
        assert np.all((m.real == 0) | (m.imag == 0))
        k = int(math.log2(m.shape[0]))
        for _ in range(2):
            t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
            _check(api, n, t, m, dtype, "stored")
        op = api.build(synth.Gate(tuple(range(k)), m), n, dtype=dtype, variant="stored")
        assert not op.info()["real_values"]


def test_stored_diagonals_match_oracle(api):
    """Builder (stored): full-system offsets and every diagonal's values."""
    for n, k in ((5, 1), (6, 2), (7, 3)):
        for kind in ("dense", "sparse", "diag"):
            t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
            m = synth.random_gate(k, RNG, kind)
            op = api.build(synth.Gate(tuple(t), m), n, dtype=torch.complex128, variant="stored")
            offs, vals = oracle.gate_diaq(n, t, m)
            assert list(op.offsets()) == list(offs)
            for q in range(len(offs)):
                np.testing.assert_array_equal(op.diagonal(q), vals[q])
            info = op.info()
            assert info["stored_bytes"] == 16 * sum(len(v) for v in vals)
            op32 = api.build(synth.Gate(tuple(t), m), n, dtype=torch.complex64, variant="stored")
            for q in range(len(offs)):
                np.testing.assert_array_equal(op32.diagonal(q), vals[q].astype(np.complex64))


def test_classes(api):
    n = 6
    cases = {"diagonal": synth.cphase(0.3), "permutation": synth.SWAP, "real": synth.H,
             "monomial": np.array([[0, -1j], [1j, 0]]), "general": synth.haar_u2(RNG)}
    real = {"diagonal": False, "permutation": True, "real": True, "monomial": False, "general": False}
    for want, m in cases.items():
        k = int(math.log2(m.shape[0]))
        op = api.build(synth.Gate(tuple(range(k)), m), n)
        assert op.info()["class"] == want
        assert op.info()["real_values"] == real[want]


def test_raw_diaq_apply(api):
    """A DiaQ matrix given by the user (Section IV) times a state (Algorithm 2)."""
    n = 9
    N = 1 << n
    idx = [-300, -17, -1, 0, 2, 64, 511]
    vals = [RNG.standard_normal(N - abs(d)) + 1j * RNG.standard_normal(N - abs(d)) for d in idx]
    vals[2][::3] = 0.0  # exact zeros inside a diagonal
    x = synth.random_state(n, RNG)
    want = oracle.diaq_matvec(idx, vals, x)
    for dtype, tol in ((torch.complex128, TOL_C128), (torch.complex64, 5e-6)):
        op = api.build_diaq(n, idx, vals, dtype=dtype)
        y = torch.empty(N, dtype=dtype, device="cuda")
        api.apply(op, dev(x, dtype), y)
        assert maxerr(host(y), want) <= tol * max(1.0, float(np.max(np.abs(want))))
        assert op.info()["class"] == "raw"


@pytest.mark.parametrize("real", [False, True])
@pytest.mark.parametrize("n_diag", [1, 2, 3, 4, 5, 15, 16, 17, 40])
def test_raw_diaq_apply_diagonal_counts(api, n_diag, real):
    """Stored SpMV with zero, one, real and complex entries (or real entries
    only, which take the kernel without the imaginary half), across the
    switch from offsets passed by value (up to 16 diagonals) to offsets read
    from device memory."""
    n = 10
    N = 1 << n
    idx = sorted(int(d) for d in RNG.choice(np.arange(-N + 1, N), size=n_diag, replace=False))
    vals = [RNG.standard_normal(N - abs(d)) + (0 if real else 1j) * RNG.standard_normal(N - abs(d)) for d in idx]
    for v in vals:
        v[::5] = 0.0
        v[1::7] = 1.0
        v[2::9] = RNG.standard_normal(len(v[2::9]))  # real entries
    x = synth.random_state(n, RNG)
    want = oracle.diaq_matvec(idx, vals, x)
    scale = max(1.0, float(np.max(np.abs(want))))
    for dtype, tol in ((torch.complex128, TOL_C128), (torch.complex64, 5e-6)):
        op = api.build_diaq(n, idx, vals, dtype=dtype)
        y = torch.empty(N, dtype=dtype, device="cuda")
        api.apply(op, dev(x, dtype), y)
        assert maxerr(host(y), want) <= tol * scale * n_diag, (n_diag, dtype)


def test_fuse_gate_ops(api):
    n = 10
    for trial in range(5):
        gates = []
        union = set()
        while len(gates) < 4:
            k = int(RNG.integers(1, 3))
            t = tuple(int(q) for q in RNG.choice(n, size=k, replace=False))
            if len(union | set(t)) > 5:
                break
            union |= set(t)
            gates.append(synth.Gate(t, synth.random_gate(k, RNG, ["dense", "diag", "real"][trial % 3])))
        x = synth.random_state(n, RNG)
        want = x
        for g in gates:
            want = oracle.apply_gate(want, g.targets, g.matrix)
        for variant in ("onthefly", "stored"):
            ops = [api.build(g, n) for g in gates]
            f = api.fuse(ops, variant=variant)
            y = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
            api.apply(f, dev(x), y)
            assert maxerr(host(y), want) <= TOL_C128


def test_fuse_raw_ops_on_device(api):
    """Algorithm 1 on full-system DiaQ operands, on the device."""
    n = 7
    N = 1 << n
    mats = []
    ops = []
    for _ in range(3):
        idx = sorted(set(int(d) for d in RNG.integers(-N + 1, N, size=4)) | {0})
        vals = [RNG.standard_normal(N - abs(d)) + 1j * RNG.standard_normal(N - abs(d)) for d in idx]
        A = np.zeros((N, N), dtype=np.complex128)
        for d, v in zip(idx, vals):
            t = np.arange(len(v))
            A[max(0, -d) + t, max(0, d) + t] = v
        mats.append(A)
        ops.append(api.build_diaq(n, idx, vals))
    f = api.fuse(ops)
    P = mats[2] @ mats[1] @ mats[0]
    x = synth.random_state(n, RNG)
    y = torch.empty(N, dtype=torch.complex128, device="cuda")
    api.apply(f, dev(x), y)
    assert maxerr(host(y), P @ x) <= 1e-11 * max(1.0, float(np.max(np.abs(P @ x))))
    # real operands give a real product (applied without the imaginary half);
    # one complex operand makes it complex again
    rops = [api.build_diaq(n, list(range(-3, 4)), [RNG.standard_normal(N - abs(d)) for d in range(-3, 4)])
            for _ in range(2)]
    rm = [np.zeros((N, N), dtype=np.complex128) for _ in range(2)]
    for o, A in zip(rops, rm):
        for q, d in enumerate(o.offsets()):
            t = np.arange(N - abs(d))
            A[max(0, -d) + t, max(0, d) + t] = o.diagonal(q)
    assert all(o.info()["real_values"] for o in rops) and not ops[1].info()["real_values"]
    for pair, want, real in (((rops[0], rops[1]), rm[1] @ rm[0], True), ((rops[0], ops[1]), mats[1] @ rm[0], False)):
        f = api.fuse(list(pair))
        assert f.info()["real_values"] == real
        assert f.prune().info()["real_values"] == real
        api.apply(f, dev(x), y)
        assert maxerr(host(y), want @ x) <= 1e-11 * max(1.0, float(np.max(np.abs(want @ x))))


@pytest.mark.parametrize("variant", ["stored", "onthefly"])
def test_ghz12_both_variants(api, variant):
    """GHZ-12: each gate as a 4096 x 4096 DiaQ matrix (offsets 0, +-2^k),
    applied by the DiaQ SpMV; equals (|0..0> + |1..1>)/sqrt(2) and the oracle."""
    n = 12
    circ = synth.ghz(n)
    ops = [api.build(g, n, variant=variant) for g in circ.gates]
    for g, op in zip(circ.gates[1:], ops[1:]):
        k = g.targets[0]
        assert list(op.offsets()) == [-(2 << k), 0, 2 << k]
    x = dev(synth.basis_state(n, 0))
    y = torch.empty_like(x)
    for op in ops:
        api.apply(op, x, y)
        x, y = y, x
    got = host(x)
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert maxerr(got, ref) <= 2.3e-16
    assert maxerr(got, oracle.run_circuit(circ, synth.basis_state(n, 0))) <= TOL_C128


@pytest.mark.parametrize("n", [5, 13, 18])
def test_qft_matches_oracle_and_closed_form(api, n):
    circ, j = synth.qft(n, seed=n)
    ops = [api.build(g, n) for g in circ.gates]
    x = dev(synth.basis_state(n, j))
    y = torch.empty_like(x)
    for op in ops:
        api.apply(op, x, y)
        x, y = y, x
    got = host(x)
    assert maxerr(got, qft_amplitudes(n, j, np.arange(1 << n))) <= TOL_C128
    if n <= 13:
        assert maxerr(got, oracle.run_circuit(circ, synth.basis_state(n, j))) <= TOL_C128


def _run_qft_full(api, n, variant):
    circ, j = synth.qft(n, seed=0)
    x = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    x[j] = 1.0
    y = torch.empty_like(x)
    if variant == "onthefly":
        ops = [api.build(g, n) for g in circ.gates]
        for op in ops:
            api.apply(op, x, y)
            x, y = y, x
    else:
        for g in circ.gates:  # materialise one op at a time (bounded memory)
            op = api.build(g, n, variant="stored")
            api.apply(op, x, y)
            x, y = y, x
            op.close()
    torch.cuda.synchronize()
    return x, j


@pytest.mark.parametrize("variant", ["onthefly", "stored"])
def test_qft28_full_size_sampled(api, variant):
    """QFT-28 (4 GiB complex128 state, 420 ops) in the launch configuration
    the benchmark uses; sampled amplitudes against the closed form, and the
    norm."""
    n = 28
    free, _ = torch.cuda.mem_get_info()
    need = (2 if variant == "onthefly" else 6) * (16 << n)
    assert free > need, "not enough device memory for the full-size case"
    x, j = _run_qft_full(api, n, variant)
    ks = np.concatenate([np.arange(64), (1 << n) - 1 - np.arange(64),
                         np.random.default_rng(5).integers(0, 1 << n, size=8192)])
    got = x[torch.as_tensor(ks, device="cuda")].cpu().numpy()
    assert maxerr(got, qft_amplitudes(n, j, ks)) <= TOL_C128
    assert abs(api.norm(x) - 1.0) <= 1e-12


def test_error_paths(api):
    from paper_2405_01250_gb300._native import DiaqError
    op = api.build(synth.Gate((0,), synth.H), 6, variant="stored")
    x = torch.zeros(64, dtype=torch.complex128, device="cuda")
    with pytest.raises(DiaqError, match="in place"):
        api.apply(op, x, x)
    big = torch.zeros(128, dtype=torch.complex128, device="cuda")
    with pytest.raises(DiaqError, match="overlap"):
        api.apply(op, big[:64], big[32:96])
    with pytest.raises(DiaqError, match="SHAPE"):
        api.fuse([api.build(synth.Gate((0,), synth.H), 6), api.build(synth.Gate((0,), synth.H), 7)])
    with pytest.raises(DiaqError, match="UNSUPPORTED"):
        api.fuse([api.build(synth.Gate((q,), synth.H), 8) for q in range(7)])


def test_zero_operator_both_variants(api):
    """Degenerate gate with no non-zero entry: no diagonals, y = 0."""
    n = 6
    for variant in ("onthefly", "stored"):
        op = api.build(synth.Gate((2, 4), np.zeros((4, 4), dtype=complex)), n, variant=variant)
        assert len(op.offsets()) == 0
        x = dev(synth.random_state(n, RNG))
        y = torch.full_like(x, 7.0)
        api.apply(op, x, y)
        assert np.all(host(y) == 0)
