"""Host logic that needs no GPU: the fusion planner and the batch argument
checks (which run before any device call)."""

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def test_plan_fusion_respects_limits(api):
    rng = np.random.default_rng(3)
    n = 12
    gates = []
    for _ in range(200):
        k = int(rng.integers(1, 3))
        gates.append(synth.Gate(tuple(int(q) for q in rng.choice(n, size=k, replace=False)), synth.random_gate(k, rng)))
    for max_k in (2, 3, 4, 6):
        for depth in (1, 2, 4, 8):
            grp = api.plan_fusion(gates, max_k, depth)
            assert grp[0] == 0 and all(b - a in (0, 1) for a, b in zip(grp, grp[1:]))
            for g in set(grp):
                members = [gates[i] for i in range(len(gates)) if grp[i] == g]
                assert 1 <= len(members) <= depth
                assert len({q for m in members for q in m.targets}) <= max_k
            if depth == 1:
                assert grp == list(range(len(gates)))


def test_plan_fusion_greedy_example(api):
    H, CZ = synth.H, synth.CZ
    gates = [synth.Gate((0,), H), synth.Gate((1,), H), synth.Gate((0, 1), CZ), synth.Gate((2,), H),
             synth.Gate((2, 3), CZ), synth.Gate((0,), H)]
    assert api.plan_fusion(gates, 2, 4) == [0, 0, 0, 1, 1, 2]
    assert api.plan_fusion(gates, 3, 4) == [0, 0, 0, 0, 1, 1]
    assert api.plan_fusion(gates, 4, 2) == [0, 0, 1, 1, 2, 2]


def test_plan_fusion_rejects_bad_limits(api):
    from paper_2405_01250_gb300._native import DiaqError
    g = [synth.Gate((0, 1), synth.CZ)]
    with pytest.raises(DiaqError, match="max_k"):
        api.plan_fusion(g, 1, 2)
    with pytest.raises(DiaqError):
        api.plan_fusion(g, 7, 2)
    with pytest.raises(DiaqError):
        api.plan_fusion(g, 2, 0)


def _batch_args(api, instances):
    import torch  # noqa: F401
    return instances


def test_batch_validation_before_device(api):
    from paper_2405_01250_gb300._native import DiaqError
    obs = ([0], [3], [1.0])
    with pytest.raises(DiaqError, match="1 or 2 qubits"):
        api.Batch([(4, [synth.Gate((0, 1, 2), synth.random_gate(3, np.random.default_rng(0)))], 0, obs)])
    with pytest.raises(DiaqError, match="n_qubits"):
        api.Batch([(1, [synth.Gate((0,), synth.H)], 0, ([0], [1], [1.0]))])
    with pytest.raises(DiaqError, match="parameter"):
        api.Batch([(3, [synth.Gate((0,), None, param=2, gen="X")], 1, obs)])
    with pytest.raises(DiaqError, match="qubit"):
        api.Batch([(2, [synth.Gate((0,), synth.H)], 0, ([0], [1 << 5], [1.0]))])


def test_plan_fusion_commuting_valid_and_exact(api):
    """Commutation-aware grouping: the order is a permutation that moves a
    gate only past gates on disjoint qubits, groups respect the limits, and
    the reordered circuit is the same operator (checked with the oracle)."""
    import oracle
    for seed in range(3):
        circ = synth.random_layered(8, 4, seed=seed)
        for max_k, depth in ((2, 4), (3, 8), (4, 6)):
            order, grp = api.plan_fusion_commuting(circ.gates, max_k, depth)
            assert sorted(order) == list(range(len(circ.gates)))
            assert grp[0] == 0 and all(b - a in (0, 1) for a, b in zip(grp, grp[1:]))
            for g in set(grp):
                members = [circ.gates[order[p]] for p in range(len(order)) if grp[p] == g]
                assert len(members) <= depth
                assert len({q for m in members for q in m.targets}) <= max_k
            # any two gates that swapped relative order act on disjoint qubits
            pos = {gi: p for p, gi in enumerate(order)}
            for a in range(len(circ.gates)):
                for b in range(a + 1, len(circ.gates)):
                    if pos[a] > pos[b]:
                        assert not set(circ.gates[a].targets) & set(circ.gates[b].targets)
            psi = synth.random_state(8, np.random.default_rng(seed))
            ref = oracle.run_circuit(circ, psi)
            got = psi
            for gi in order:
                got = oracle.apply_gate(got, circ.gates[gi].targets, circ.gates[gi].matrix)
            assert np.max(np.abs(got - ref)) < 1e-13
    # the random-layer structure fuses to one group per CZ pair and layer at max_k = 2
    circ = synth.random_layered(30, 4, seed=0)
    _, grp = api.plan_fusion_commuting(circ.gates, 2, 4)
    assert max(grp) + 1 == 60


def test_plan_fusion_diagonal_keeps_classes_apart(api):
    """Runs of diagonal gates (fixed diagonal matrices, Z-only rotations)
    fuse within max_k qubits and max_depth gates; every other gate is a
    group of its own; the fused circuit equals the original (oracle)."""
    import oracle
    rng = np.random.default_rng(5)
    n = 8
    circ, j = synth.qft(n, seed=2)
    extra = [synth.Gate((1, 4), None, param=0, gen="ZZ"), synth.Gate((3,), None, param=0, gen="Z"),
             synth.Gate((2, 5), None, param=0, gen="ZX"), synth.Gate((0, 6), synth.CZ)]
    gates = list(circ.gates[:10]) + extra + list(circ.gates[10:])
    theta = np.array([0.37])
    diag = [g.matrix is None and set(g.gen) <= {"Z", "I"} or
            (g.matrix is not None and np.count_nonzero(g.matrix - np.diag(np.diag(g.matrix))) == 0) for g in gates]
    for max_k, depth in ((2, 64), (4, 3), (6, 64)):
        grp = api.plan_fusion_diagonal(gates, max_k, depth)
        assert grp[0] == 0 and all(b - a in (0, 1) for a, b in zip(grp, grp[1:]))
        for gi in set(grp):
            members = [i for i in range(len(gates)) if grp[i] == gi]
            if len(members) > 1:
                assert all(diag[i] for i in members)
                assert len(members) <= depth
                assert len({q for i in members for q in gates[i].targets}) <= max_k
        psi = synth.random_state(n, rng)
        want = psi
        for g in gates:
            want = oracle.apply_gate(want, g.targets, oracle.gate_matrix(g, theta))
        got = psi
        for gi in sorted(set(grp)):
            members = [gates[i] for i in range(len(gates)) if grp[i] == gi]
            union, F = oracle.fuse([(m.targets, oracle.gate_matrix(m, theta)) for m in members])
            got = oracle.apply_gate(got, list(union), F)
        assert np.max(np.abs(got - want)) < 1e-13
    # QFT-28: 28 H, 87 runs of controlled phases (5 per run beside the
    # shared target, 6 qubits), 14 SWAPs
    c28, _ = synth.qft(28, seed=0)
    assert max(api.plan_fusion_diagonal(c28.gates, 6, 64)) + 1 == 28 + 87 + 14
