"""GPU parity of the window-fused adjoint sweep: gates grouped into blocks of
at most w qubits (moved only past gates on disjoint qubits), each block run
in one launch over shared-memory groups. Energies and gradients must match
the FP64 oracle (parameter shift) and the one-launch-per-gate sweep."""

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
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return A


def _tols(dtype, circ, obs):
    if dtype == torch.complex128:
        return 1e-12, 1e-10
    # FP32 states: each gate adds about 2^-24 relative error per amplitude,
    # weighted by the observable's norm bound sum |c|
    b = len(circ.gates) * 2.0 ** -24 * float(np.sum(np.abs(obs.coeff))) * 8
    return b, b


def _mixed_circuit(n, rng):
    gates = [synth.Gate((q,), synth.H) for q in range(n)]
    gates += [synth.Gate((0, 3), None, param=0, gen="XY", scale=0.5),
              synth.Gate((2,), synth.haar_u2(rng)),
              synth.Gate((4, 1), synth.haar_u2(rng, 4)),
              synth.Gate((1, 4), None, param=1, gen="YY", scale=2.0),
              synth.Gate((3,), None, param=2, gen="Z"),
              synth.Gate((2, 0), None, param=0, gen="ZX", scale=-1.5),
              synth.Gate((5, 2), synth.CNOT),
              synth.Gate((5,), None, param=1, gen="Y"),
              synth.Gate((0, 5), synth.CZ)]
    return synth.Circuit(n, gates, theta=rng.uniform(0, 2 * np.pi, 3))


def _cases():
    rng = np.random.default_rng(31)
    a = synth.ansatz(n=7, layers=2, seed=11)
    out = [("ansatz7", a, synth.ansatz_observable(7))]
    q, qo = synth.qaoa_instance(10, rng, p=2)
    out.append(("qaoa10", q, qo))
    m = _mixed_circuit(6, rng)
    mo = synth.Observable(np.array([0b101010, 0, 3], np.uint64), np.array([0b000110, 0b110000, 1], np.uint64),
                          np.array([0.7, -1.1, 0.4]))
    out.append(("mixed6", m, mo))
    t = synth.tfim(8, 3, 0.15, J=1.0, h=0.7)
    out.append(("tfim8", t, synth.magnetisation_observable(8)))
    return out


CASES = _cases()


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_window_fused_plan_matches_oracle(api, dtype, case):
    name, circ, obs = CASES[case]
    n = circ.n
    psi0 = synth.basis_state(n, 0)
    e_ref = oracle.energy(circ, obs, psi0)
    g_ref = oracle.param_shift_grad(circ, obs, psi0)
    tol_e, tol_g = _tols(dtype, circ, obs)
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
    e0, g0 = plan.run(circ.theta)
    for w in (2, 3, 4, 5):
        for lanes in (1, 4):
            plan.set_sweep(w, lanes)
            win, ln, launches = plan.sweep()
            assert win == w and ln == lanes and 0 < launches <= len(circ.gates)
            e, g = plan.run(circ.theta)
            assert abs(e - e_ref) <= tol_e, (name, w, lanes)
            assert np.max(np.abs(g - g_ref)) <= tol_g, (name, w, lanes)
            if dtype == torch.complex128:
                assert abs(e - e0) <= 1e-12 and np.max(np.abs(g - g0)) <= 1e-12
    # back to one launch per gate
    plan.set_window(0)
    assert plan.window() == (0, len(circ.gates))
    e, g = plan.run(circ.theta)
    assert abs(e - e0) == 0.0 and np.array_equal(g, g0)
    plan.close()


def test_window_plan_replays_new_theta_and_initial_state(api):
    name, circ, obs = CASES[0]
    n = circ.n
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n)
    plan.set_window(4)
    rng = np.random.default_rng(5)
    for _ in range(3):
        th = rng.uniform(0, 2 * np.pi, circ.n_params)
        e, g = plan.run(th)
        c2 = synth.Circuit(n, circ.gates, theta=th)
        psi0 = synth.basis_state(n, 0)
        assert abs(e - oracle.energy(c2, obs, psi0)) <= 1e-12
        assert np.max(np.abs(g - oracle.param_shift_grad(c2, obs, psi0))) <= 1e-10
    start = synth.random_state(n, rng)
    p0 = torch.as_tensor(start).cuda()
    e, g = plan.run(circ.theta, psi0=p0)
    assert abs(e - oracle.energy(circ, obs, start)) <= 1e-12
    assert np.max(np.abs(g - oracle.param_shift_grad(circ, obs, start))) <= 1e-10


def test_window_plan_full_size_ansatz20(api):
    """Ansatz-20 (320 parameters, 472 gates): windows 3, 4 and 5 give the
    per-gate sweep's energy and full gradient; a sample against parameter
    shift."""
    n = 20
    circ = synth.ansatz(n=n, layers=8, seed=0)
    obs = synth.ansatz_observable(n)
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n)
    e0, g0 = plan.run(circ.theta)
    for w in (3, 4, 5):
        for lanes in (1, 4):
            plan.set_sweep(w, lanes)
            e, g = plan.run(circ.theta)
            assert abs(e - e0) <= 1e-11 and np.max(np.abs(g - g0)) <= 1e-11, (w, lanes)
    sample = [0, 1, 200, 319]
    g_ps = oracle.param_shift_grad(circ, obs, synth.basis_state(n, 0), params=sample)
    assert np.max(np.abs(g[sample] - g_ps[sample])) <= 1e-10


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_plan_autotune_keeps_parity(api, dtype):
    name, circ, obs = CASES[1]
    n = circ.n
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
    rep = plan.autotune(circ.theta, reps=2)
    assert {(w, ln) for w, ln, _, _ in rep["tried"]} == {(0, 1), (3, 1), (4, 1), (5, 1), (3, 4), (4, 4), (5, 4)}
    assert all(b == 0 for w, _, b, _ in rep["tried"] if w > 0)
    assert all(b > 0 for w, _, b, _ in rep["tried"] if w == 0)
    assert plan.sweep()[:2] == (rep["best_window"], rep["best_lanes"])
    if rep["best_window"] == 0:
        assert plan.blocks() == rep["best_blocks"] > 0
    e, g = plan.run(circ.theta)
    psi0 = synth.basis_state(n, 0)
    tol_e, tol_g = _tols(dtype, circ, obs)
    assert abs(e - oracle.energy(circ, obs, psi0)) <= tol_e
    assert np.max(np.abs(g - oracle.param_shift_grad(circ, obs, psi0))) <= tol_g


def test_window_argument_errors(api):
    circ = synth.ansatz(n=3, layers=1, seed=1)
    obs = synth.ansatz_observable(3)
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), 3)
    for bad in (1, 6, -1):
        with pytest.raises(Exception):
            plan.set_window(bad)
    for bad_lanes in (0, 2, 8):
        with pytest.raises(Exception):
            plan.set_sweep(4, bad_lanes)
    e, g = plan.run(circ.theta)
    assert abs(e - oracle.energy(circ, obs, synth.basis_state(3, 0))) <= 1e-12
    empty = api.AdjointPlan([], 0, (obs.xmask, obs.zmask, obs.coeff), 3)
    empty.set_window(4)
    e, g = empty.run(np.zeros(0))
    assert abs(e - oracle.expect(synth.basis_state(3, 0), obs).real) <= 1e-12 and len(g) == 0
