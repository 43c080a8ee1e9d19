"""GPU parity of diagonal ops of 4 to 6 qubits (one table lookup and one
complex multiply per row; in place, rows whose entry is exactly 1 are not
touched) and of the QFT with its runs of controlled phases fused into such
ops (plan_fusion_diagonal), against the FP64 oracle and the QFT's closed
form."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, dev, host, maxerr, qft_amplitudes, tol_c64

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(2024)


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _diag_gate(k, rng):
    """Random phases with exact 1, -1, i and 0 entries mixed in."""
    d = np.exp(1j * rng.uniform(0, 2 * np.pi, size=1 << k))
    pick = rng.permutation(1 << k)
    d[pick[: (1 << k) // 3]] = 1.0
    d[pick[(1 << k) // 3]] = -1.0
    d[pick[(1 << k) // 3 + 1]] = 1j
    d[pick[(1 << k) // 3 + 2]] = 0.0
    return np.diag(d).astype(np.complex128)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("k", [4, 5, 6])
def test_diagonal_op_out_of_place_and_in_place(api, dtype, k):
    for n in (k, k + 1, 11, 14):
        t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
        m = _diag_gate(k, RNG)
        psi = synth.random_state(n, RNG)
        want = oracle.apply_gate(psi, t, m)
        op = api.build(synth.Gate(tuple(t), m), n, dtype=dtype)
        assert op.info()["class"] == "diagonal"
        x = dev(psi, dtype)
        y = torch.empty_like(x)
        api.apply(op, x, y)
        z = x.clone()
        api.apply(op, z, z)
        tol = TOL_C128 if dtype == torch.complex128 else tol_c64(0, 1.0)
        assert maxerr(host(y), want) <= tol
        assert torch.equal(y, z)  # in place: the same bits
        # rows whose entry is exactly 1 are left as they were, bit for bit
        idx = np.arange(1 << n)
        loc = np.zeros_like(idx)
        for a, q in enumerate(t):
            loc |= ((idx >> q) & 1) << (k - 1 - a)
        ones = np.diag(m)[loc] == 1.0
        assert torch.equal(z[torch.as_tensor(np.nonzero(ones)[0], device="cuda")],
                           x[torch.as_tensor(np.nonzero(ones)[0], device="cuda")])
        s = 16 if dtype == torch.complex128 else 8
        changed = int(np.count_nonzero(np.diag(m) != 1.0))
        assert op.apply_bytes(in_place=True) == 2 * s * ((1 << n) >> k) * changed
        assert op.apply_bytes() == 2 * s * (1 << n)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("n", [7, 12, 16])
def test_qft_with_fused_phase_runs(api, dtype, n):
    circ, j = synth.qft(n, seed=n)
    ops = api.build_fused(circ.gates, n, 6, 64, dtype=dtype, diagonal=True)
    assert len(ops) < len(circ.gates)
    want = qft_amplitudes(n, j, np.arange(1 << n))
    x = torch.zeros(1 << n, dtype=dtype, device="cuda")
    x[j] = 1
    c = x.clone()
    y = torch.empty_like(x)
    for op in ops:
        api.apply(op, x, y)
        x, y = y, x
    for op in ops:
        api.apply(op, c, c)
    tol = TOL_C128 if dtype == torch.complex128 else 64 * 2.0 ** -24
    assert maxerr(host(x), want) <= tol
    assert maxerr(host(c), want) <= tol


def test_qft28_fused_phase_runs_full_size_sampled(api):
    n = 28
    circ, j = synth.qft(n, seed=0)
    ops = api.build_fused(circ.gates, n, 6, 64, diagonal=True)
    assert len(ops) == 129
    c = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    c[j] = 1
    for op in ops:
        api.apply(op, c, c)
    ks = np.concatenate([np.arange(64), RNG.integers(0, 1 << n, size=4096), [(1 << n) - 1]]).astype(np.int64)
    got = c[torch.as_tensor(ks, device="cuda")].cpu().numpy()
    assert maxerr(got, qft_amplitudes(n, j, ks)) <= TOL_C128
    assert abs(api.norm(c) - 1.0) < 1e-12
