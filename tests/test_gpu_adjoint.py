"""GPU parity of the adjoint gradient (energy and dE/dtheta for every
parameter in one sweep) against the oracle's parameter-shift gradient and
central finite differences; the autograd binding."""

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


def _run(api, circ, obs, n, dtype=torch.complex128, theta=None):
    p0 = torch.zeros(1 << n, dtype=dtype, device="cuda")
    p0[0] = 1
    th = circ.theta if theta is None else theta
    return api.adjoint_grad(circ.gates, th, obs.xmask, obs.zmask, obs.coeff, p0, torch.empty_like(p0),
                            torch.empty_like(p0))


@pytest.mark.parametrize("n,layers", [(2, 1), (5, 2), (8, 2)])
def test_ansatz_gradient_c128(api, n, layers):
    circ = synth.ansatz(n=n, layers=layers, seed=n)
    obs = synth.ansatz_observable(n)
    e, g = _run(api, circ, obs, n)
    psi0 = synth.basis_state(n, 0)
    assert abs(e - oracle.energy(circ, obs, psi0)) <= 1e-12
    g_ps = oracle.param_shift_grad(circ, obs, psi0)
    assert np.max(np.abs(g - g_ps)) <= 1e-10
    g_fd = oracle.fd_grad(circ, obs, psi0, h=1e-4)
    assert np.max(np.abs(g - g_fd)) <= 1e-6


def test_ansatz_gradient_c64(api):
    n = 8
    circ = synth.ansatz(n=n, layers=2, seed=3)
    obs = synth.ansatz_observable(n)
    e, g = _run(api, circ, obs, n, dtype=torch.complex64)
    psi0 = synth.basis_state(n, 0)
    g_ps = oracle.param_shift_grad(circ, obs, psi0)
    # FP32 state, FP64 accumulation: error grows with depth; bound from the
    # state error (~ gates * 2^-24 * sum|c|)
    bound = len(circ.gates) * 2.0 ** -24 * float(np.sum(np.abs(obs.coeff))) * 8
    assert abs(e - oracle.energy(circ, obs, psi0)) <= bound
    assert np.max(np.abs(g - g_ps)) <= bound


def test_qaoa_shared_parameters(api):
    circ, obs = synth.qaoa_instance(8, np.random.default_rng(4), p=2)
    e, g = _run(api, circ, obs, 8)
    psi0 = synth.basis_state(8, 0)
    assert abs(e - oracle.energy(circ, obs, psi0)) <= 1e-12
    assert np.max(np.abs(g - oracle.param_shift_grad(circ, obs, psi0))) <= 1e-10


def test_scaled_and_multi_qubit_generators(api):
    n = 5
    rng = np.random.default_rng(8)
    gates = [synth.Gate((q,), synth.H) for q in range(n)]
    gates += [synth.Gate((0, 3), None, param=0, gen="XY", scale=0.5),
              synth.Gate((4, 1, 2), None, param=1, gen="ZXY", scale=-1.5),
              synth.Gate((2,), synth.haar_u2(rng)),
              synth.Gate((1, 4), None, param=0, gen="YY", scale=2.0)]
    circ = synth.Circuit(n, gates, theta=rng.uniform(0, 2 * np.pi, 2))
    obs = synth.Observable(np.array([0b10101, 0, 3], np.uint64), np.array([0b00110, 0b11000, 1], np.uint64),
                           np.array([0.7, -1.1, 0.4]))
    e, g = _run(api, circ, obs, n)
    psi0 = synth.basis_state(n, 0)
    assert abs(e - oracle.energy(circ, obs, psi0)) <= 1e-12
    assert np.max(np.abs(g - oracle.param_shift_grad(circ, obs, psi0))) <= 1e-10


def test_ansatz20_sampled_parameters(api):
    """Full-size ansatz (20 qubits, 8 layers, 320 parameters): the adjoint
    gradient on sampled parameters against parameter shift."""
    n = 20
    circ = synth.ansatz(n=n, layers=8, seed=0)
    obs = synth.ansatz_observable(n)
    e, g = _run(api, circ, obs, n)
    psi0 = synth.basis_state(n, 0)
    sample = [0, 1, 157, 319]
    g_ps = oracle.param_shift_grad(circ, obs, psi0, params=sample)
    assert np.max(np.abs(g[sample] - g_ps[sample])) <= 1e-10
    assert abs(e - oracle.energy(circ, obs, psi0)) <= 1e-11


def test_autograd_function(api):
    n = 4
    circ = synth.ansatz(n=n, layers=1, seed=9)
    obs = synth.ansatz_observable(n)
    theta = torch.tensor(circ.theta, dtype=torch.float64, requires_grad=True)
    p0 = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    p0[0] = 1
    E = api.DiaqEnergy.apply(theta, circ.gates, (obs.xmask, obs.zmask, obs.coeff), p0)
    (2.0 * E).backward()
    g_ps = oracle.param_shift_grad(circ, obs, synth.basis_state(n, 0))
    assert np.max(np.abs(theta.grad.numpy() - 2 * g_ps)) <= 1e-10


def test_empty_circuit_and_no_params(api):
    n = 3
    obs = synth.Observable(np.array([0], np.uint64), np.array([1], np.uint64), np.array([1.0]))
    circ = synth.Circuit(n, [], theta=np.zeros(0))
    e, g = _run(api, circ, obs, n)
    assert e == 1.0 and len(g) == 0


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_adjoint_plan_graph_replay(api, dtype):
    """The graph-recorded sweep matches the oracle for several theta on one
    plan, from |0..0> and from a given initial state."""
    n = 7
    circ = synth.ansatz(n=n, layers=2, seed=11)
    obs = synth.ansatz_observable(n)
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
    rng = np.random.default_rng(12)
    tol_e, tol_g = (1e-12, 1e-10) if dtype == torch.complex128 else (2e-5, 2e-5)
    for trial in range(3):
        th = rng.uniform(0, 2 * np.pi, circ.n_params)
        e, g = plan.run(th)
        psi0 = synth.basis_state(n, 0)
        c2 = synth.Circuit(n, circ.gates, theta=th)
        assert abs(e - oracle.energy(c2, obs, psi0)) <= tol_e
        assert np.max(np.abs(g - oracle.param_shift_grad(c2, obs, psi0))) <= tol_g
    start = synth.random_state(n, rng)
    p0 = torch.as_tensor(start).to(device="cuda", dtype=dtype)
    e, g = plan.run(circ.theta, psi0=p0)
    ref_start = p0.cpu().numpy().astype(np.complex128)
    assert abs(e - oracle.energy(circ, obs, ref_start)) <= tol_e
    assert np.max(np.abs(g - oracle.param_shift_grad(circ, obs, ref_start))) <= tol_g


def test_autograd_with_plan(api):
    n = 5
    circ = synth.ansatz(n=n, layers=1, seed=13)
    obs = synth.ansatz_observable(n)
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n)
    theta = torch.tensor(circ.theta, dtype=torch.float64, requires_grad=True)
    E = api.DiaqEnergy.apply(theta, plan, None, None)
    E.backward()
    g_ps = oracle.param_shift_grad(circ, obs, synth.basis_state(n, 0))
    assert np.max(np.abs(theta.grad.numpy() - g_ps)) <= 1e-10


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_plan_and_batch_lambda_groups_sharing_an_x_mask(api, dtype):
    """lambda = H psi for an observable whose term groups share X masks with
    bits among 5..7 and many equal-weight terms (counted for eight amplitudes
    at once), beside a group of unequal weights, single terms and Y letters;
    the plan and the batch against the oracle."""
    rng = np.random.default_rng(21)
    n = 10
    circ = synth.ansatz(n=n, layers=2, seed=6)
    xs, zs, cs = [], [], []
    for x in (0, (1 << 6) | (1 << 2), (1 << 7) | (1 << 5) | 1):
        for _ in range(7):  # equal weights: the count form
            xs.append(x)
            zs.append(int(rng.integers(0, 1 << n)))
            cs.append(0.3)
    for _ in range(5):  # one X mask, unequal weights
        xs.append(1 << 9)
        zs.append(int(rng.integers(0, 1 << n)))
        cs.append(float(rng.uniform(-1, 1)))
    xs.append(1 << 3)
    zs.append(1 << 3)  # a Y letter
    cs.append(0.7)
    obs = synth.Observable(np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64), np.array(cs))
    psi0 = synth.basis_state(n, 0)
    e_ref = oracle.energy(circ, obs, psi0)
    g_ref = oracle.param_shift_grad(circ, obs, psi0)
    tol_e, tol_g = (1e-11, 1e-10) if dtype == torch.complex128 else (2e-5, 5e-5)
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
    e, g = plan.run(circ.theta)
    plan.close()
    assert abs(e - e_ref) < tol_e and np.max(np.abs(g - g_ref)) < tol_g
    b = api.Batch([(n, circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff))], dtype=dtype)
    E, G = b.run(circ.theta)
    b.close()
    assert abs(E[0] - e_ref) < tol_e and np.max(np.abs(G[0] - g_ref)) < tol_g
