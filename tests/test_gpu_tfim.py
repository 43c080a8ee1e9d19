"""GPU parity on the Trotterised transverse-field Ising workload (the paper's
Hamiltonian-simulation benchmark, Section VII, read out as the average
magnetisation): states and magnetisations against the FP64 oracle, the
adjoint gradient with respect to the two shared angles against the exact
parameter-shift gradient, and full-size (28-qubit) runs against the closed
forms of the decoupled limits."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, host, maxerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _run(api, circ, dtype=torch.complex128, in_place=False):
    n = circ.n
    ops = [api.build(g, n, dtype=dtype, theta=circ.theta) for g in circ.gates]
    x = torch.zeros(1 << n, dtype=dtype, device="cuda")
    x[0] = 1
    y = x if in_place else torch.empty_like(x)
    for op in ops:
        api.apply(op, x, y)
        if not in_place:
            x, y = y, x
    return x


@pytest.mark.parametrize("n,steps", [(3, 2), (12, 6), (15, 3)])
def test_tfim_state_and_magnetisation_c128(api, n, steps):
    circ = synth.tfim(n, steps, 0.1, J=1.0, h=0.7)
    want = oracle.run_circuit(circ, synth.basis_state(n, 0))
    obs = synth.magnetisation_observable(n)
    for in_place in (False, True):
        x = _run(api, circ, in_place=in_place)
        assert maxerr(host(x), want) <= TOL_C128
        m = api.expect(x, obs.xmask, obs.zmask, obs.coeff).real
        assert abs(m - oracle.expect(want, obs).real) <= TOL_C128


def test_tfim_c64_against_fp64_oracle(api):
    n, steps = 12, 6
    circ = synth.tfim(n, steps, 0.1, J=1.0, h=0.7)
    want = oracle.run_circuit(circ, synth.basis_state(n, 0))
    x = _run(api, circ, dtype=torch.complex64)
    # per gate at most 2^k products, each with three FP32 roundings, relative
    # to amplitudes <= 1; errors add over the circuit's gates
    bound = len(circ.gates) * 2 * 4 * 3 * 2.0 ** -24
    assert maxerr(host(x), want) <= bound
    assert oracle.fidelity(host(x), want) >= 1 - 1e-9


def test_tfim_adjoint_gradient_of_magnetisation(api):
    """dM/dtheta for the two shared angles (every bond gate shares theta[0],
    every field gate theta[1])."""
    n = 8
    circ = synth.tfim(n, 4, 0.15, J=1.0, h=0.7)
    obs = synth.magnetisation_observable(n)
    p0 = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    p0[0] = 1
    e, g = api.adjoint_grad(circ.gates, circ.theta, obs.xmask, obs.zmask, obs.coeff, p0, torch.empty_like(p0),
                            torch.empty_like(p0))
    psi0 = synth.basis_state(n, 0)
    assert abs(e - oracle.energy(circ, obs, psi0)) <= TOL_C128
    assert np.max(np.abs(g - oracle.param_shift_grad(circ, obs, psi0))) <= 1e-10
    assert np.max(np.abs(g - oracle.fd_grad(circ, obs, psi0, h=1e-4))) <= 1e-6


def test_tfim28_full_size_decoupled_limits(api):
    """28 qubits (4 GiB state), in place: with J = 0 every qubit precesses,
    so M_z = cos(2 h t); with h = 0 the state stays |0...0> up to the phase
    exp(i J t (n-1))."""
    n, steps, dt = 28, 3, 0.11
    obs = synth.magnetisation_observable(n)
    x = _run(api, synth.tfim(n, steps, dt, J=0.0, h=0.8), in_place=True)
    m = api.expect(x, obs.xmask, obs.zmask, obs.coeff).real
    assert abs(m - math.cos(2 * 0.8 * steps * dt)) <= TOL_C128
    assert abs(api.norm(x) - 1.0) <= TOL_C128
    del x
    x = _run(api, synth.tfim(n, steps, dt, J=1.3, h=0.0), in_place=True)
    a0 = complex(x[0].item())
    assert abs(a0 - complex(math.cos(1.3 * steps * dt * (n - 1)), math.sin(1.3 * steps * dt * (n - 1)))) <= TOL_C128
    x[0] = 0
    assert float(x.abs().max().item()) == 0.0
