"""GPU parity of the batched persistent launch (energies and adjoint
gradients of many circuits of uneven sizes) and of the autotuners and the
fusion planner."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, dev, host, maxerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _instances(rng, sizes, p=2):
    out = []
    for n in sizes:
        circ, obs = synth.qaoa_instance(n, rng, p=p)
        out.append((circ, obs))
    a = synth.ansatz(n=5, layers=1, seed=4)
    out.append((a, synth.ansatz_observable(5)))
    return out


def _ref(instances):
    E, G = [], []
    for circ, obs in instances:
        psi0 = synth.basis_state(circ.n, 0)
        E.append(oracle.energy(circ, obs, psi0))
        G.append(oracle.param_shift_grad(circ, obs, psi0))
    return E, G


def _batch(api, instances, dtype):
    return api.Batch([(c.n, c.gates, c.n_params, (o.xmask, o.zmask, o.coeff)) for c, o in instances], dtype=dtype)


def test_batch_matches_oracle_all_shapes(api):
    rng = np.random.default_rng(21)
    inst = _instances(rng, [4, 6, 8, 10, 6, 4])
    E_ref, G_ref = _ref(inst)
    theta = np.concatenate([c.theta for c, _ in inst])
    b = _batch(api, inst, torch.complex128)
    for cluster in (1, 2, 4, 8):
        for threads in (64, 256):
            b.set_launch(cluster, threads)
            E, G = b.run(theta)
            assert np.max(np.abs(E - E_ref)) <= 1e-12, (cluster, threads)
            for g, gr in zip(G, G_ref):
                assert np.max(np.abs(g - gr)) <= 1e-10, (cluster, threads)
    # a second theta through the same captured graph
    theta2 = theta + 0.37
    inst2 = [(synth.Circuit(c.n, c.gates, theta=c.theta + 0.37), o) for c, o in inst]
    E_ref2, G_ref2 = _ref(inst2)
    E, G = b.run(theta2)
    assert np.max(np.abs(E - E_ref2)) <= 1e-12
    assert max(np.max(np.abs(g - gr)) for g, gr in zip(G, G_ref2)) <= 1e-10


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_batch_window_fused_matches_oracle(api, dtype):
    """The window-fused team kernel (blocks of <= w qubits, one cluster
    barrier per block) gives the oracle's energies and gradients for every
    window and cluster size, and the per-gate kernel's to rounding."""
    rng = np.random.default_rng(24)
    inst = _instances(rng, [4, 6, 8, 10, 12, 6])
    E_ref, G_ref = _ref(inst)
    theta = np.concatenate([c.theta for c, _ in inst])
    b = _batch(api, inst, dtype)
    E0, G0 = b.run(theta)
    for w, lanes in ((2, 1), (3, 1), (4, 1), (5, 1), (3, 4), (4, 4), (5, 4)):
        b.set_sweep(w, lanes)
        assert b.window() == w and b.sweep() == (w, lanes)
        for cluster in (1, 2, 8):
            b.set_launch(cluster, 128)
            E, G = b.run(theta)
            for (c, o), e, er, g, gr, e0, g0 in zip(inst, E, E_ref, G, G_ref, E0, G0):
                if dtype == torch.complex128:
                    assert abs(e - er) <= 1e-12 and np.max(np.abs(g - gr)) <= 1e-10, (w, lanes, cluster)
                    assert abs(e - e0) <= 1e-12 and np.max(np.abs(g - g0)) <= 1e-12, (w, lanes, cluster)
                else:
                    bound = len(c.gates) * 2.0 ** -24 * float(np.sum(np.abs(o.coeff))) * 8
                    assert abs(e - er) <= bound and np.max(np.abs(g - gr)) <= bound, (w, lanes, cluster)
    with pytest.raises(Exception):
        b.set_launch(2, 256)  # the window-fused kernel runs 128 threads per block
    b.set_window(0)
    b.set_launch(1, 256)
    E, G = b.run(theta)
    assert np.array_equal(E, E0)
    with pytest.raises(Exception):
        b.set_window(6)
    with pytest.raises(Exception):
        b.set_sweep(4, 3)


def test_batch_c64(api):
    rng = np.random.default_rng(22)
    inst = _instances(rng, [6, 8, 10])
    E_ref, G_ref = _ref(inst)
    theta = np.concatenate([c.theta for c, _ in inst])
    b = _batch(api, inst, torch.complex64)
    E, G = b.run(theta)
    for (c, o), e, er, g, gr in zip(inst, E, E_ref, G, G_ref):
        bound = len(c.gates) * 2.0 ** -24 * float(np.sum(np.abs(o.coeff))) * 8
        assert abs(e - er) <= bound
        assert np.max(np.abs(g - gr)) <= bound


def test_batch_deterministic_and_autotune(api):
    rng = np.random.default_rng(23)
    inst = _instances(rng, [8, 12, 14, 10, 12])
    theta = np.concatenate([c.theta for c, _ in inst])
    b = _batch(api, inst, torch.complex128)
    rep = b.autotune(theta, reps=1)
    assert rep["tried"] and rep["best_cluster"] in (1, 2, 4, 8)
    assert {(w, ln) for _, _, w, ln, _ in rep["tried"]} >= {(0, 1), (3, 1), (4, 1), (3, 4), (4, 4)}
    q = b.query()
    assert q["cluster"] == rep["best_cluster"] and q["threads"] == rep["best_threads"]
    assert b.sweep() == (rep["best_window"], rep["best_lanes"])
    E1, G1 = b.run(theta)
    E2, G2 = b.run(theta)
    assert np.array_equal(E1, E2) and all(np.array_equal(a, c) for a, c in zip(G1, G2))
    E_ref, G_ref = _ref(inst)
    assert np.max(np.abs(E1 - E_ref)) <= 1e-12


def test_autotune_apply_keeps_parity(api):
    n = 16
    x = torch.empty(1 << n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    rep = api.autotune_apply(n, x, y, reps=2)
    assert len(rep["rows"]) == 27 and set(rep["best"]) == {1, 2, 3}
    rng = np.random.default_rng(24)
    for k in (1, 2, 3):
        for threads, groups in ((128, 4), (64, 1), tuple(rep["best"][k][:2])):
            api.set_apply_launch(torch.complex128, k, threads, groups)
            for nn in (k, 9, 13):
                t = [int(q) for q in rng.choice(nn, size=k, replace=False)]
                m = synth.random_gate(k, rng)
                xs = synth.random_state(nn, rng)
                op = api.build(synth.Gate(tuple(t), m), nn)
                yt = torch.empty(1 << nn, dtype=torch.complex128, device="cuda")
                api.apply(op, dev(xs), yt)
                assert maxerr(host(yt), oracle.apply_gate(xs, t, m)) <= TOL_C128
        api.set_apply_launch(torch.complex128, k, 256, 0)


def test_fused_circuit_and_fusion_autotune(api):
    n = 12
    circ = synth.random_layered(n, 3, seed=7)
    psi0 = synth.basis_state(n, 0)
    want = oracle.run_circuit(circ, psi0)
    for max_k, depth in ((2, 4), (4, 4), (6, 8)):
        for variant in ("onthefly", "stored"):
            ops = api.build_fused(circ.gates, n, max_k, depth, variant=variant)
            assert len(ops) < len(circ.gates) or depth == 1
            x = dev(psi0)
            y = torch.empty_like(x)
            for op in ops:
                api.apply(op, x, y)
                x, y = y, x
            assert maxerr(host(x), want) <= TOL_C128
    w = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    rep = api.autotune_fusion(circ.gates, n, w, max_k=4, max_depth=4)
    assert 1 <= rep["best_depth"] <= 4 and rep["ops"][0] == len(circ.gates)


def test_commuting_fused_circuit(api):
    n = 12
    circ = synth.random_layered(n, 4, seed=8)
    psi0 = synth.basis_state(n, 0)
    want = oracle.run_circuit(circ, psi0)
    for max_k, depth in ((2, 4), (3, 8)):
        for dtype, tol in ((torch.complex128, TOL_C128), (torch.complex64, 2e-5)):
            ops = api.build_fused(circ.gates, n, max_k, depth, dtype=dtype, commuting=True)
            assert len(ops) < len(circ.gates) // 2
            x = dev(psi0, dtype)
            for op in ops:
                api.apply(op, x, x)
            assert maxerr(host(x), want) <= tol
    w = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    rep = api.autotune_fusion(circ.gates, n, w, max_k=2, max_depth=4, commuting=True)
    assert rep["ops"][0] == len(circ.gates) and rep["ops"][3] < rep["ops"][0]
