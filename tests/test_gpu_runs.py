"""Diagonal runs of the adjoint sweep (phase.cuh): runs of Z-type rotations,
fixed single-qubit diagonals and CZs applied as one diagonal operator, with
each rotation's gradient term taken once for the run. Checked against the
same sweep gate by gate (runs off) and against the FP64 oracle's
parameter-shift gradient, for the adjoint plan (weight and chunk forms) and
the batch (weight form), including runs too long for either form."""

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


S_GATE = np.diag([1, 1j]).astype(np.complex128)
T_GATE = np.diag([1, np.exp(1j * math.pi / 4)]).astype(np.complex128)


def _mixed(n, rng):
    """Rotations with Z-only generators (single Z, ZZ, IZ), fixed S, T and CZ
    gates, repeated rotations on one qubit, and non-diagonal gates between
    them on disjoint and on shared qubits."""
    g = []
    g.append(synth.Gate((0,), synth.H))
    g.append(synth.Gate((1,), synth.H))
    g.append(synth.Gate((2,), None, param=0, gen="Z"))
    g.append(synth.Gate((3,), S_GATE))
    g.append(synth.Gate((5,), None, param=1, gen="Y"))          # disjoint: moves ahead
    g.append(synth.Gate((1, 4), synth.CZ))
    g.append(synth.Gate((2,), None, param=2, gen="Z", scale=-0.5))
    g.append(synth.Gate((0, 6), None, param=3, gen="IZ"))        # a single Z on qubit 6
    g.append(synth.Gate((4,), T_GATE))
    g.append(synth.Gate((2, 3), None, param=4, gen="XY"))        # shares qubits: closes the run
    g.append(synth.Gate((0, 1), None, param=5, gen="ZZ"))        # weight 2, own parameter
    g.append(synth.Gate((3, 5), None, param=5, gen="ZZ"))
    g.append(synth.Gate((6,), synth.random_gate(1, rng, "dense")))
    g.append(synth.Gate((1,), None, param=6, gen="Z"))
    g.append(synth.Gate((6,), None, param=6, gen="Z"))
    g.append(synth.Gate((0, 5), synth.CZ))
    return synth.Circuit(n, g, theta=rng.uniform(0, 2 * math.pi, size=7))


def _plan_grad(api, circ, obs, n, dtype, runs):
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
    plan.set_runs(runs)
    e, g = plan.run(circ.theta)
    info = plan.runs()
    plan.close()
    return e, g, info


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("which", ["ansatz", "mixed", "qaoa"])
def test_plan_runs_match_gate_by_gate_and_oracle(api, dtype, which):
    rng = np.random.default_rng(3)
    if which == "ansatz":
        n = 10
        circ = synth.ansatz(n=n, layers=3, seed=1)
        obs = synth.ansatz_observable(n)
    elif which == "mixed":
        n = 8
        circ = _mixed(n, rng)
        obs = synth.ansatz_observable(n)
    else:
        n = 10
        circ, obs = synth.qaoa_instance(n, rng, p=3)
    e_on, g_on, info = _plan_grad(api, circ, obs, n, dtype, True)
    e_off, g_off, info_off = _plan_grad(api, circ, obs, n, dtype, False)
    assert info[0] and info[1] >= 1 and info[2] < len(circ.gates)  # runs formed, fewer launches
    assert not info_off[0] and info_off[2] == len(circ.gates)
    psi0 = synth.basis_state(n, 0)
    e_ref = oracle.energy(circ, obs, psi0)
    g_ref = oracle.param_shift_grad(circ, obs, psi0)
    if dtype == torch.complex128:
        assert abs(e_on - e_off) < 1e-12 and np.max(np.abs(g_on - g_off)) < 1e-12
        assert abs(e_on - e_ref) < 1e-11 and np.max(np.abs(g_on - g_ref)) < 1e-10
    else:
        assert abs(e_on - e_ref) < 2e-5 and np.max(np.abs(g_on - g_ref)) < 5e-5


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("which", ["ansatz-5", "ansatz-7", "qaoa-6"])
def test_plan_runs_on_states_below_one_block(api, dtype, which):
    """States of fewer than 256 amplitudes: the run kernels' blocks of 256
    are partial (lanes and rows past the state's end take no part)."""
    rng = np.random.default_rng(11)
    if which.startswith("ansatz"):
        n = int(which.split("-")[1])
        circ = synth.ansatz(n=n, layers=2, seed=3)
        obs = synth.ansatz_observable(n)
    else:
        n = 6
        circ, obs = synth.qaoa_instance(n, rng, p=2)
    e_on, g_on, info = _plan_grad(api, circ, obs, n, dtype, True)
    assert info[0] and info[1] >= 1
    psi0 = synth.basis_state(n, 0)
    tol_e, tol_g = (1e-11, 1e-10) if dtype == torch.complex128 else (2e-5, 5e-5)
    assert abs(e_on - oracle.energy(circ, obs, psi0)) < tol_e
    assert np.max(np.abs(g_on - oracle.param_shift_grad(circ, obs, psi0))) < tol_g


def test_plan_runs_beyond_form_limits_fall_back(api):
    """A run of 60 one-parameter ZZ rotations (over the weight form's 48) and
    a run of 28 single-qubit rotations (over the chunk form's 24) are applied
    gate by gate; the gradient still matches the oracle."""
    rng = np.random.default_rng(9)
    n = 14
    g = [synth.Gate((q,), synth.H) for q in range(n)]
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)][:60]
    g += [synth.Gate(pq, None, param=0, gen="ZZ") for pq in pairs]
    g += [synth.Gate((q,), None, param=1, gen="X") for q in range(n)]
    g += [synth.Gate((q % n,), None, param=2 + q, gen="Z") for q in range(28)]
    circ = synth.Circuit(n, g, theta=rng.uniform(0, 2 * math.pi, size=30))
    obs = synth.ansatz_observable(n)
    e_on, g_on, info = _plan_grad(api, circ, obs, n, torch.complex128, True)
    assert info[1] == 0  # neither run fits a form
    psi0 = synth.basis_state(n, 0)
    assert abs(e_on - oracle.energy(circ, obs, psi0)) < 1e-11
    assert np.max(np.abs(g_on - oracle.param_shift_grad(circ, obs, psi0))) < 1e-10


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_batch_runs_match_gate_by_gate_and_oracle(api, dtype):
    inst = synth.qaoa_batch(12, seed=4, sizes=(8, 10, 12))
    desc = [(c.n, c.gates, c.n_params, (o.xmask, o.zmask, o.coeff)) for c, o in inst]
    theta = np.concatenate([c.theta for c, _ in inst])
    res = {}
    for on in (True, False):
        b = api.Batch(desc, dtype=dtype)
        b.set_runs(on)
        assert b.runs()[0] == on and (b.runs()[1] == (4 * len(inst) if on else 0))
        b.set_launch(2, 128)
        res[on] = b.run(theta)
        b.close()
    E1, G1 = res[True]
    E0, G0 = res[False]
    if dtype == torch.complex128:
        assert np.max(np.abs(E1 - E0)) < 1e-12
        assert max(float(np.max(np.abs(a - b))) for a, b in zip(G1, G0)) < 1e-12
    for i in (0, 5):
        c, o = inst[i]
        p0 = synth.basis_state(c.n, 0)
        tol_e, tol_g = (1e-11, 1e-10) if dtype == torch.complex128 else (2e-5, 5e-5)
        assert abs(E1[i] - oracle.energy(c, o, p0)) < tol_e
        assert np.max(np.abs(G1[i] - oracle.param_shift_grad(c, o, p0))) < tol_g
