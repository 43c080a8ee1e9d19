"""Full-size and maximum-size cases in the benchmark's launch configuration,
checked through properties that hold at any size (the circuit followed by
its inverse returns the initial state; the norm is preserved) or against
closed forms and the oracle on sampled instances."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _inverse(gates):
    return [synth.Gate(g.targets, np.asarray(g.matrix).conj().T) for g in reversed(gates)]


@pytest.mark.parametrize("dtype,depth,tol", [(torch.complex64, 40, 2e-4), (torch.complex128, 8, 1e-12)])
def test_random30_circuit_then_inverse(api, dtype, depth, tol):
    """Random layered circuit on 30 qubits (8 or 16 GiB state), on the fly,
    in place; then its inverse: the state must return to |0...0>."""
    n = 30
    circ = synth.random_layered(n, depth, seed=0)
    x = torch.zeros(1 << n, dtype=dtype, device="cuda")
    x[0] = 1
    for g in circ.gates:
        api.apply(api.build(g, n, dtype=dtype), x, x)
    nrm = api.norm(x)
    assert abs(nrm - 1.0) < (1e-12 if dtype == torch.complex128 else 1e-4)
    assert abs(x[0].item()) < 0.5  # the circuit moved the state
    for g in _inverse(circ.gates):
        api.apply(api.build(g, n, dtype=dtype), x, x)
    assert abs(x[0].item() - 1.0) <= tol
    x[0] = 0
    assert float(x.abs().max().item()) <= tol


def test_33_qubit_state_64bit_indexing(api):
    """A 2^33-amplitude complex128 state (128 GiB): gates on the top and
    bottom qubits index past 2^32 amplitudes; the result is a product state
    whose amplitudes are known exactly."""
    n = 33
    free, _ = torch.cuda.mem_get_info()
    assert free > (16 << n) + (8 << 30), "needs a GB300-class device"
    x = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    x[0] = 1
    phi = 0.7
    for g in (synth.Gate((32,), synth.H), synth.Gate((0,), synth.H), synth.Gate((0, 32), synth.cphase(phi)),
              synth.Gate((31, 32), synth.SWAP)):
        api.apply(api.build(g, n), x, x)
    # after H(32), H(0): (|0> + |1>)_32 (|0> + |1>)_0 / 2; CP adds e^{i phi} to |1...1>; SWAP(31, 32) moves bit 32 to 31
    idx = [0, 1, 1 << 31, (1 << 31) | 1]
    want = [0.5, 0.5, 0.5, 0.5 * complex(math.cos(phi), math.sin(phi))]
    got = x[torch.tensor(idx, device="cuda")].cpu().numpy()
    assert np.max(np.abs(got - np.array(want))) <= 1e-15
    assert abs(api.norm(x) - 1.0) <= 1e-12
    x[torch.tensor(idx, device="cuda")] = 0
    assert api.norm(x) == 0.0  # every other amplitude is exactly zero
    del x


def test_qaoa_batch_full_size_sampled(api):
    """All 256 QAOA circuits (n = 14..22, p = 4) in one batched launch:
    every energy and gradient against the plain per-circuit adjoint path
    (itself oracle-checked), and two 14-qubit circuits against the oracle's
    parameter-shift gradient."""
    inst = synth.qaoa_batch(256, seed=0)
    theta = np.concatenate([c.theta for c, _ in inst])
    b = api.Batch([(c.n, c.gates, c.n_params, (o.xmask, o.zmask, o.coeff)) for c, o in inst])
    E, G = b.run(theta)
    b.close()
    for i in range(0, 256, 17):
        c, o = inst[i]
        p0 = torch.zeros(1 << c.n, dtype=torch.complex128, device="cuda")
        p0[0] = 1
        e, g = api.adjoint_grad(c.gates, c.theta, o.xmask, o.zmask, o.coeff, p0, torch.empty_like(p0),
                                torch.empty_like(p0))
        assert abs(E[i] - e) <= 1e-11 and np.max(np.abs(G[i] - g)) <= 1e-10
    small = [i for i, (c, _) in enumerate(inst) if c.n == 14][:2]
    for i in small:
        c, o = inst[i]
        psi0 = synth.basis_state(c.n, 0)
        assert abs(E[i] - oracle.energy(c, o, psi0)) <= 1e-11
        assert np.max(np.abs(G[i] - oracle.param_shift_grad(c, o, psi0))) <= 1e-9
