"""GPU parity of unitary simulation (Section II-A) by chained device DiaQ
products (Algorithm 1): after every time step the diagonals, their values
and the non-zero count match the oracle's dense product of the time-step
unitaries; GHZ(10) stays at least 99.8 % sparse (Section III-A)."""

import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, dev, host, maxerr

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(99)


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _dense_step(n, gate, theta):
    """Full-system matrix of one gate from the oracle's DiaQ diagonals."""
    N = 1 << n
    offs, vals = oracle.gate_diaq(n, gate.targets, oracle.gate_matrix(gate, theta))
    m = np.zeros((N, N), dtype=np.complex128)
    for d, v in zip(offs, vals):
        r0, c0 = max(0, -d), max(0, d)
        idx = np.arange(len(v))
        m[r0 + idx, c0 + idx] = v
    return m


def _dense_chain(n, gates, theta=None):
    U = np.eye(1 << n, dtype=np.complex128)
    out = []
    for g in gates:
        U = _dense_step(n, g, theta) @ U
        out.append(U.copy())
    return out


def _nonzero_diagonals(U):
    N = U.shape[0]
    r, c = np.nonzero(U)
    return np.unique(c - r)


def _check_op_equals_dense(op, U, tol):
    N = U.shape[0]
    offs = op.offsets()
    for q, d in enumerate(offs):
        got = op.diagonal(q)
        want = np.diagonal(U, offset=int(d))
        assert maxerr(got, want) <= tol, (q, d)
    # every diagonal of U with a value above the tolerance is stored
    big = [d for d in _nonzero_diagonals(U).tolist() if np.max(np.abs(np.diagonal(U, offset=d))) > tol]
    assert set(big) <= set(offs.tolist())


def test_ghz10_chain_matches_dense_per_step(api):
    g = json.load(open(os.path.join(GOLDEN, "ghz10_sparsity.json")))
    n = g["n_qubits"]
    N = 1 << n
    circ = synth.ghz(n)
    dense = _dense_chain(n, circ.gates)
    for t in range(len(circ.gates)):
        op, nd, nz = api.unitary_chain(circ.gates[: t + 1], n, prune=True)
        U = dense[t]
        assert nz[t] == np.count_nonzero(U)
        assert nd[t] == len(_nonzero_diagonals(U))  # pruned: exactly the non-zero diagonals
        assert 1.0 - nz[t] / (N * N) >= g["min_sparsity"]
        _check_op_equals_dense(op, U, TOL_C128)
    # the per-step records of one chain equal the separate chains' last entries
    op, nd, nz = api.unitary_chain(circ.gates, n, prune=True)
    assert list(nz) == [np.count_nonzero(U) for U in dense]
    assert list(nd) == [len(_nonzero_diagonals(U)) for U in dense]
    assert nz[-1] == 2 * N  # permutations times one Hadamard: two non-zeros per column


def test_chain_without_prune_keeps_structural_diagonals(api):
    n = 8
    circ = synth.ghz(n)
    opp, ndp, nzp = api.unitary_chain(circ.gates, n, prune=True)
    opf, ndf, nzf = api.unitary_chain(circ.gates, n, prune=False)
    assert np.all(ndf >= ndp)
    assert list(nzf) == list(nzp)
    U = _dense_chain(n, circ.gates)[-1]
    _check_op_equals_dense(opf, U, TOL_C128)
    nnz = opf.diagonal_nnz()
    assert int(nnz.sum()) == np.count_nonzero(U)
    pr = opf.prune()
    assert list(pr.offsets()) == list(opp.offsets())


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_tfim_chain_and_apply(api, dtype):
    n = 6
    circ = synth.tfim(n, 2, 0.2, J=1.0, h=0.7)
    op, nd, nz = api.unitary_chain(circ.gates, n, dtype=dtype, theta=circ.theta)
    U = _dense_chain(n, circ.gates, circ.theta)[-1]
    tol = TOL_C128 if dtype == torch.complex128 else len(circ.gates) * 8 * 3 * 2.0 ** -24
    _check_op_equals_dense(op, U, tol)
    assert nd[-1] <= 2 * (1 << n) - 1
    # the unitary applied by the stored DiaQ SpMV equals running the circuit
    x = synth.random_state(n, RNG)
    xt = dev(x, dtype)
    yt = torch.empty_like(xt)
    api.apply(op, xt, yt)
    want = oracle.run_circuit(circ, x)
    assert maxerr(host(yt), want) <= (TOL_C128 if dtype == torch.complex128 else 4 * tol)


def test_chain_edge_cases(api):
    # one gate, one qubit
    op, nd, nz = api.unitary_chain([synth.Gate((0,), synth.H)], 1)
    assert list(op.offsets()) == [-1, 0, 1] and nz[0] == 4
    # an identity gate leaves only the principal diagonal after pruning
    op, nd, nz = api.unitary_chain([synth.Gate((1, 0), np.eye(4, dtype=np.complex128))], 3)
    assert list(op.offsets()) == [0] and nz[0] == 8
    # H twice: the off-diagonals cancel to exact zeros only where rounding allows;
    # pruning never changes a value, so U stays within rounding of I
    op, nd, nz = api.unitary_chain([synth.Gate((2,), synth.H), synth.Gate((2,), synth.H)], 4)
    _check_op_equals_dense(op, _dense_chain(4, [synth.Gate((2,), synth.H)] * 2)[-1], 1e-15)
    with pytest.raises(Exception):
        api.unitary_chain([synth.Gate((0,), synth.H)], 16)
    with pytest.raises(Exception):
        api.unitary_chain([], 4)
