"""Scaled rotations of the complex128 adjoint sweep (rot.cuh rot_groups_s):
each Pauli rotation is applied divided by the larger of |cos(a/2)| and
|sin(a/2)|, one fused multiply-add per real component, and the factor the
states then carry is divided out of the energy and of each gradient term.
Checked against the unscaled sweep and the FP64 oracle's parameter-shift
gradient for the adjoint plan and the batch: one- and two-qubit generators
with even and odd Y counts, angles on both sides of |cos| = |sin| and at
the special angles, runs on and off, and a circuit past the rotation bound
(where the unscaled form runs)."""

import math

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GENS1 = ["X", "Y", "Z"]
GENS2 = ["XX", "XY", "YX", "YY", "ZX", "XZ", "YZ", "ZY", "ZZ", "IX", "YI"]


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _pauli_circuit(n, rng, count, theta=None):
    """Random Pauli rotations on one and two (possibly reversed,
    non-adjacent) qubits, with fixed H and CZ gates between them."""
    g = [synth.Gate((q,), synth.H) for q in range(n)]
    p = 0
    for i in range(count):
        if i % 5 == 4:
            a, b = rng.choice(n, size=2, replace=False)
            g.append(synth.Gate((int(a), int(b)), synth.CZ))
            continue
        if rng.random() < 0.5:
            g.append(synth.Gate((int(rng.integers(n)),), None, param=p, gen=GENS1[int(rng.integers(3))],
                                scale=float(rng.choice([1.0, -0.5, 2.0]))))
        else:
            a, b = rng.choice(n, size=2, replace=False)
            g.append(synth.Gate((int(a), int(b)), None, param=p, gen=GENS2[int(rng.integers(len(GENS2)))]))
        p += 1
    th = rng.uniform(0, 2 * math.pi, size=p) if theta is None else theta(p)
    return synth.Circuit(n, g, theta=th)


def _plan(api, circ, obs, n, dtype, scaled, runs=True):
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
    plan.set_runs(runs)
    plan.set_scaled(scaled)
    state = plan.scaled()
    e, g = plan.run(circ.theta)
    plan.close()
    return e, g, state


def _check_vs_oracle(circ, obs, n, e, g):
    psi0 = synth.basis_state(n, 0)
    assert abs(e - oracle.energy(circ, obs, psi0)) < 1e-11
    assert np.max(np.abs(g - oracle.param_shift_grad(circ, obs, psi0))) < 1e-10


@pytest.mark.parametrize("which", ["pauli", "ansatz", "qaoa"])
@pytest.mark.parametrize("runs", [True, False])
def test_plan_scaled_matches_unscaled_and_oracle(api, which, runs):
    rng = np.random.default_rng(21)
    if which == "pauli":
        n = 9
        circ = _pauli_circuit(n, rng, 60)
        obs = synth.ansatz_observable(n)
    elif which == "ansatz":
        n = 10
        circ = synth.ansatz(n=n, layers=3, seed=5)
        obs = synth.ansatz_observable(n)
    else:
        n = 10
        circ, obs = synth.qaoa_instance(n, rng, p=3)
    e1, g1, st1 = _plan(api, circ, obs, n, torch.complex128, True, runs)
    e0, g0, st0 = _plan(api, circ, obs, n, torch.complex128, False, runs)
    assert st1 == (True, True) and st0 == (False, False)
    assert abs(e1 - e0) < 1e-12 and np.max(np.abs(g1 - g0)) < 1e-12
    _check_vs_oracle(circ, obs, n, e1, g1)


def test_plan_scaled_special_angles(api):
    """Angles where cos(a/2) or sin(a/2) is 0, where |cos| = |sin|, and just
    either side of it: both forms of the scaled rotation and their switch."""
    rng = np.random.default_rng(8)
    n = 8
    q = math.pi / 2
    special = np.array([0.0, math.pi, 2 * math.pi, q, 3 * q, -q, q + 1e-9, q - 1e-9, math.pi - 1e-12, 1e-12])
    circ = _pauli_circuit(n, rng, 50, theta=lambda p: np.resize(special, p))
    obs = synth.ansatz_observable(n)
    e1, g1, st = _plan(api, circ, obs, n, torch.complex128, True)
    e0, g0, _ = _plan(api, circ, obs, n, torch.complex128, False)
    assert st == (True, True)
    assert abs(e1 - e0) < 1e-12 and np.max(np.abs(g1 - g0)) < 1e-12
    _check_vs_oracle(circ, obs, n, e1, g1)


def test_plan_scaled_not_used_for_complex64_or_past_the_bound(api):
    rng = np.random.default_rng(2)
    n = 6
    circ = synth.ansatz(n=n, layers=2, seed=3)
    obs = synth.ansatz_observable(n)
    _, _, st = _plan(api, circ, obs, n, torch.complex64, True)
    assert st == (True, False)
    # 500 non-diagonal rotations: 1000 forward and reverse applications > 960
    g = [synth.Gate((q,), synth.H) for q in range(4)]
    g += [synth.Gate((i % 4,), None, param=i, gen="XY"[i % 2]) for i in range(500)]
    big = synth.Circuit(4, g, theta=rng.uniform(0, 2 * math.pi, size=500))
    obs4 = synth.ansatz_observable(4)
    e, gr, st = _plan(api, big, obs4, 4, torch.complex128, True)
    assert st == (True, False)
    _check_vs_oracle(big, obs4, 4, e, gr)


def test_batch_scaled_matches_unscaled_and_oracle(api):
    inst = synth.qaoa_batch(10, seed=6, sizes=(8, 10, 12))
    desc = [(c.n, c.gates, c.n_params, (o.xmask, o.zmask, o.coeff)) for c, o in inst]
    theta = np.concatenate([c.theta for c, _ in inst])
    res = {}
    for on in (True, False):
        b = api.Batch(desc, dtype=torch.complex128)
        b.set_scaled(on)
        b.set_launch(2, 128)
        assert b.scaled() == (on, on)
        res[on] = b.run(theta)
        b.close()
    (E1, G1), (E0, G0) = res[True], res[False]
    assert np.max(np.abs(E1 - E0)) < 1e-12
    assert max(float(np.max(np.abs(a - b))) for a, b in zip(G1, G0)) < 1e-12
    for i in (0, 3, 7):
        c, o = inst[i]
        p0 = synth.basis_state(c.n, 0)
        assert abs(E1[i] - oracle.energy(c, o, p0)) < 1e-11
        assert np.max(np.abs(G1[i] - oracle.param_shift_grad(c, o, p0))) < 1e-10
    # complex64 batches keep the unscaled form
    b = api.Batch(desc, dtype=torch.complex64)
    assert b.scaled() == (True, False)
    b.close()


def _xy_circuit(n, rng, layers):
    """Layers of one-qubit X and Y rotations (runs of them pair up in the
    sweep), some on the same qubit back to back, with CZs and a dense fixed
    gate between layers."""
    g = [synth.Gate((q,), synth.H) for q in range(n)]
    p = 0
    for _ in range(layers):
        qs = list(rng.permutation(n)) + [int(rng.integers(n))]
        for q in qs:
            g.append(synth.Gate((int(q),), None, param=p, gen="XY"[int(rng.integers(2))],
                                scale=float(rng.choice([1.0, -0.5]))))
            p += 1
        g.append(synth.Gate((0, n - 1), synth.CZ))
        g.append(synth.Gate((int(rng.integers(n)),), synth.random_gate(1, rng, "dense")))
    return synth.Circuit(n, g, theta=rng.uniform(0, 2 * math.pi, size=p))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("scaled", [True, False])
def test_plan_rotation_pairs_match_single_launches_and_oracle(api, dtype, scaled):
    rng = np.random.default_rng(31)
    n = 9
    circ = _xy_circuit(n, rng, 4)
    obs = synth.ansatz_observable(n)
    res = {}
    for pairs in (True, False):
        plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
        plan.set_scaled(scaled)
        plan.set_pairs(pairs)
        assert plan.pairs() == pairs
        res[pairs] = plan.run(circ.theta)
        plan.close()
    (e1, g1), (e0, g0) = res[True], res[False]
    psi0 = synth.basis_state(n, 0)
    e_ref = oracle.energy(circ, obs, psi0)
    g_ref = oracle.param_shift_grad(circ, obs, psi0)
    if dtype == torch.complex128:
        assert abs(e1 - e0) < 1e-12 and np.max(np.abs(g1 - g0)) < 1e-12
        assert abs(e1 - e_ref) < 1e-11 and np.max(np.abs(g1 - g_ref)) < 1e-10
    else:
        assert abs(e1 - e_ref) < 2e-5 and np.max(np.abs(g1 - g_ref)) < 5e-5


def _layer_circuit(n, rng):
    """A leading layer of dense one-qubit gates on all qubits but the last
    (written directly as a product state), a second gate on qubit 3 (which
    ends the layer), then rotations and CZs."""
    g = [synth.Gate((q,), synth.random_gate(1, rng, "dense")) for q in range(n - 1)]
    g.append(synth.Gate((3,), synth.H))
    p = 0
    for i in range(3 * n):
        g.append(synth.Gate((int(rng.integers(n)),), None, param=p, gen="XYZ"[i % 3]))
        p += 1
        if i % 5 == 4:
            a, b = rng.choice(n, size=2, replace=False)
            g.append(synth.Gate((int(a), int(b)), synth.CZ))
    return synth.Circuit(n, g, theta=rng.uniform(0, 2 * math.pi, size=p))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_leading_product_layer_plan_and_batch(api, dtype):
    rng = np.random.default_rng(12)
    n = 10
    circs = [_layer_circuit(n, rng) for _ in range(3)]
    obs = synth.ansatz_observable(n)
    psi0 = synth.basis_state(n, 0)
    tol_e, tol_g = (1e-11, 1e-10) if dtype == torch.complex128 else (2e-5, 5e-5)
    for c in circs[:1]:
        plan = api.AdjointPlan(c.gates, c.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
        e, g = plan.run(c.theta)
        plan.close()
        assert abs(e - oracle.energy(c, obs, psi0)) < tol_e
        assert np.max(np.abs(g - oracle.param_shift_grad(c, obs, psi0))) < tol_g
    desc = [(c.n, c.gates, c.n_params, (obs.xmask, obs.zmask, obs.coeff)) for c in circs]
    b = api.Batch(desc, dtype=dtype)
    b.set_launch(2, 128)
    E, G = b.run(np.concatenate([c.theta for c in circs]))
    b.close()
    for i, c in enumerate(circs):
        assert abs(E[i] - oracle.energy(c, obs, psi0)) < tol_e
        assert np.max(np.abs(G[i] - oracle.param_shift_grad(c, obs, psi0))) < tol_g


@pytest.mark.parametrize("launch", [(2, 128), (4, 256), (1, 64)])
def test_complex64_batch_rotation_tiles_match_complex128_and_oracle(api, launch):
    """complex64 teams take up to three consecutive one-qubit X/Y rotations on
    distinct qubits per pass (tiles of 2 and 3, lone rotations where a qubit
    repeats, both sweeps); against the complex128 batch (pairs) and the
    oracle."""
    rng = np.random.default_rng(41)
    n = 9
    circs = [_xy_circuit(n, rng, 3 + i) for i in range(3)]
    obs = synth.ansatz_observable(n)
    desc = [(c.n, c.gates, c.n_params, (obs.xmask, obs.zmask, obs.coeff)) for c in circs]
    theta = np.concatenate([c.theta for c in circs])
    out = {}
    for dt in (torch.complex64, torch.complex128):
        b = api.Batch(desc, dtype=dt)
        b.set_launch(*launch)
        out[dt] = b.run(theta)
        b.close()
    (E1, G1), (E2, G2) = out[torch.complex64], out[torch.complex128]
    psi0 = synth.basis_state(n, 0)
    for i, c in enumerate(circs):
        assert abs(E2[i] - oracle.energy(c, obs, psi0)) < 1e-11
        assert abs(E1[i] - E2[i]) < 2e-5
        g_ref = oracle.param_shift_grad(c, obs, psi0)
        assert np.max(np.abs(G2[i] - g_ref)) < 1e-10
        assert np.max(np.abs(G1[i] - g_ref)) < 5e-5


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("kind", ["xy", "ansatz"])
def test_plan_blocks_keep_parity(api, dtype, kind):
    """The per-gate sweep at other block counts (more partial columns per
    gradient term, fewer groups per thread, clamped at one group per thread)
    gives the same energy and gradient; 0 restores two blocks per SM. The
    ansatz's RZ layers run as chunk-form diagonal runs, whose reverse step
    takes the terms of rotations on low bits from per-thread totals: with 1,
    3, 2, 8 and 16 blocks the split between those bits and the per-amplitude
    ones moves (it depends on the trailing zero bits of the block count)."""
    rng = np.random.default_rng(7)
    if kind == "xy":
        n = 11
        circ = _xy_circuit(n, rng, 3)
    else:
        n = 13
        circ = synth.ansatz(n=n, layers=3, seed=4)
    obs = synth.ansatz_observable(n)
    plan = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), n, dtype=dtype)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    want = (2 ** n // 2 + 255) // 256
    assert plan.blocks() == min(want, 2 * sms)
    e0, g0 = plan.run(circ.theta)
    psi0 = synth.basis_state(n, 0)
    tol_e, tol_g = (1e-11, 1e-10) if dtype == torch.complex128 else (2e-5, 5e-5)
    assert abs(e0 - oracle.energy(circ, obs, psi0)) < tol_e
    g_ref = oracle.param_shift_grad(circ, obs, psi0)
    assert np.max(np.abs(g0 - g_ref)) < tol_g
    for b in (1, 3, 2, 8, 16, 1000000):
        plan.set_blocks(b)
        assert plan.blocks() == max(1, min(b, want, 64 * sms))
        e, g = plan.run(circ.theta)
        if dtype == torch.complex128:
            assert abs(e - e0) < 1e-12 and np.max(np.abs(g - g0)) < 1e-12, b
        assert abs(e - oracle.energy(circ, obs, psi0)) < tol_e
        assert np.max(np.abs(g - g_ref)) < tol_g
    plan.set_blocks(0)
    assert plan.blocks() == min(want, 2 * sms)
    plan.close()
