"""GPU parity of the in-place apply that skips identity rows (a controlled
phase or CZ changes a quarter of the rows, a CNOT or SWAP half; Section
III-A): bit-identical to the full out-of-place pass, within 1e-12 of the FP64
oracle, and its byte accounting."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, dev, host, maxerr, qft_amplitudes, tol_c64

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(77)


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _controlled(k, rng):
    """identity on the local rows whose top bit is 0, a Haar block on the rest"""
    d = 1 << k
    m = np.eye(d, dtype=np.complex128)
    m[d // 2:, d // 2:] = synth.haar_u2(rng, d // 2)
    return m


def _partial_identity(k, rng):
    """a random subset of rows kept as identity rows, the others random"""
    d = 1 << k
    m = synth.random_gate(k, rng, "sparse")
    keep = rng.random(d) < 0.5
    for r in range(d):
        if keep[r]:
            m[r, :] = 0
            m[r, r] = 1
    return m


def _gates(k, rng):
    out = [synth.random_gate(k, rng, "diag"), synth.random_gate(k, rng, "perm"), _controlled(k, rng),
           _partial_identity(k, rng)]
    if k == 2:
        out += [synth.CNOT, synth.CZ, synth.SWAP, synth.cphase(0.37)]
    if k == 1:
        out += [np.diag([1.0, -1.0]).astype(np.complex128), np.diag([1.0, 1j]).astype(np.complex128)]
    return out


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_inplace_skip_bit_identical_to_full_pass(api, dtype, k):
    for n in (k, k + 1, 10, 13):
        for m in _gates(k, RNG):
            t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
            x = synth.random_state(n, RNG)
            xt = dev(x, dtype)
            op = api.build(synth.Gate(tuple(t), m), n, dtype=dtype)
            y_full = torch.empty_like(xt)
            api.apply(op, xt, y_full)
            api.apply(op, xt, xt)  # in place: identity rows skipped
            torch.cuda.synchronize()
            assert torch.equal(xt, y_full), (n, t, dtype)
            want = oracle.apply_gate(x, t, m)
            tol = TOL_C128 if dtype == torch.complex128 else tol_c64(k, float(np.max(np.abs(x))) * float(np.max(np.abs(m))))
            assert maxerr(host(xt), want) <= tol


def test_apply_bytes_accounting(api):
    n = 12
    N = 1 << n
    cases = [
        (synth.Gate((3, 7), synth.cphase(0.2)), 16 * 2 * N // 4),
        (synth.Gate((3, 7), synth.CZ), 16 * 2 * N // 4),
        (synth.Gate((5, 1), synth.CNOT), 16 * N),
        (synth.Gate((0, 11), synth.SWAP), 16 * N),
        (synth.Gate((4,), synth.H), 16 * 2 * N),
        (synth.Gate((4,), np.eye(2, dtype=np.complex128)), 0),
    ]
    for g, want in cases:
        op = api.build(g, n)
        assert op.apply_bytes(in_place=False) == 2 * N * 16
        assert op.apply_bytes(in_place=True) == want, g.name
    op = api.build(synth.Gate((3, 7), synth.CZ), n, dtype=torch.complex64)
    assert op.apply_bytes(in_place=True) == 8 * 2 * N // 4
    st = api.build(synth.Gate((3, 7), synth.CZ), n, variant="stored")
    assert st.apply_bytes(in_place=False) == 2 * N * 16 + st.info()["stored_bytes"]
    with pytest.raises(Exception):
        st.apply_bytes(in_place=True)
    # stored H on qubit q: each row reads its own two entries (main diagonal
    # and the one to its partner), not the zeros stored where the diagonals
    # +-2^q cross rows of the other class
    for q in (0, 5, 11):
        st = api.build(synth.Gate((q,), synth.H), n, variant="stored")
        assert st.info()["stored_bytes"] == 16 * (3 * N - 2 * (1 << q))
        assert st.apply_bytes() == 2 * N * 16 + 2 * N * 16
    # zero entries are not read: SWAP and a controlled phase one entry per
    # row, RX two
    for g, per_row in ((synth.Gate((2, 8), synth.SWAP), 1), (synth.Gate((2, 8), synth.cphase(0.4)), 1),
                       (synth.Gate((6,), np.array([[0.8, -0.6j], [-0.6j, 0.8]])), 2)):
        st = api.build(g, n, variant="stored")
        assert st.apply_bytes() == 2 * N * 16 + per_row * N * 16, g.name
    # a dense two-qubit gate: four entries per row; raw ops read every value
    st = api.build(synth.Gate((4, 9), synth.haar_u2(RNG, 4)), n, variant="stored")
    assert st.apply_bytes() == 2 * N * 16 + 4 * N * 16
    raw = api.build_diaq(n, [-3, 0, 5], [np.ones(N - 3), np.ones(N), np.ones(N - 5)])
    assert raw.apply_bytes() == 2 * N * 16 + 16 * (3 * N - 8)


def test_identity_gate_in_place_leaves_state(api):
    n = 9
    x = synth.random_state(n, RNG)
    xt = dev(x)
    before = xt.clone()
    op = api.build(synth.Gate((2, 5), np.eye(4, dtype=np.complex128)), n)
    api.apply(op, xt, xt)
    torch.cuda.synchronize()
    assert torch.equal(xt, before)


@pytest.mark.parametrize("n", [12, 20])
def test_qft_in_place_closed_form(api, n):
    """QFT in place through diaq_simulate (controlled phases and SWAPs take
    the skip path, H the full kernel) against the closed form."""
    circ, j = synth.qft(n, seed=5)
    ops = [api.build(g, n) for g in circ.gates]
    hin = np.zeros(1 << n, dtype=np.complex128)
    hin[j] = 1
    out = np.empty_like(hin)
    w = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    api.simulate(ops, hin, out, w)
    want = qft_amplitudes(n, j, np.arange(1 << n))
    assert maxerr(out, want) <= TOL_C128


def test_qft28_in_place_full_size_sampled(api):
    """Full size (2^28 amplitudes), in place: sampled amplitudes against the
    closed form, and the in-place state equal to the out-of-place one."""
    n = 28
    circ, j = synth.qft(n, seed=0)
    ops = [api.build(g, n) for g in circ.gates]
    a = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    a[j] = 1
    b = torch.empty_like(a)
    c = a.clone()
    x, y = a, b
    for op in ops:
        api.apply(op, x, y)
        x, y = y, x
    for op in ops:
        api.apply(op, c, c)
    torch.cuda.synchronize()
    assert torch.equal(x, c)
    ks = np.concatenate([np.arange(64), RNG.integers(0, 1 << n, size=4096), [(1 << n) - 1]]).astype(np.int64)
    got = c[torch.as_tensor(ks, device="cuda")].cpu().numpy()
    assert maxerr(got, qft_amplitudes(n, j, ks)) <= TOL_C128
    assert abs(api.norm(c) - 1.0) < 1e-12


def _sim_circuits(n, rng):
    qft, j = synth.qft(n, seed=4)
    mixed = [synth.Gate((n - 1,), synth.H), synth.Gate((0, 5), synth.random_gate(2, rng, "dense")),
             synth.Gate((2, n - 2, 7), synth.random_gate(3, rng, "dense")),
             synth.Gate((1, 3, 4, 6), synth.random_gate(4, rng, "dense")), synth.Gate((3,), synth.H),
             synth.Gate((n - 3, 1), synth.CZ)]
    return {"qft": (qft.gates, synth.basis_state(n, j)), "mixed": (mixed, synth.random_state(n, rng)),
            "one_op_top": ([synth.Gate((n - 1,), synth.H)], synth.random_state(n, rng)),
            "one_op_low": ([synth.Gate((1, 0), synth.random_gate(2, rng, "dense"))], synth.random_state(n, rng))}


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("stored_ends", [False, True])
def test_simulate_host_pipelined_equals_device_path(api, dtype, stored_ends):
    """diaq_simulate from and to pinned host memory overlaps the copies with
    the first and last ops slice by slice; the state must be bit-identical
    to the same ops run on device buffers, and match the oracle. With
    stored ops at both ends no slice overlap applies (the plain path)."""
    n = 16
    rng = np.random.default_rng(31)
    for name, (gates, psi0) in _sim_circuits(n, rng).items():
        variants = ["onthefly"] * len(gates)
        if stored_ends:
            variants[0] = variants[-1] = "stored"
        ops = [api.build(g, n, dtype=dtype, variant=v) for g, v in zip(gates, variants)]
        hin = torch.as_tensor(psi0).to(dtype).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        w0 = torch.empty(1 << n, dtype=dtype, device="cuda")
        w1 = torch.empty_like(w0)
        _, tl = api.simulate(ops, hin, hout, w0, w1, timeline=True)
        assert 0.0 <= tl[0] <= tl[2] and tl[1] <= tl[2]
        din = hin.cuda()
        dout = torch.empty_like(din)
        api.simulate(ops, din, dout, torch.empty_like(w0), torch.empty_like(w1))
        assert torch.equal(hout, dout.cpu()), name
        want = psi0
        for g in gates:
            want = oracle.apply_gate(want, g.targets, g.matrix)
        tol = TOL_C128 if dtype == torch.complex128 else 64 * 2.0 ** -24
        assert maxerr(hout.numpy().astype(np.complex128), want) <= tol, name
