"""Host logic of the sharded state, on CPU: the exchange schedule of
diaq_shard_schedule is a correct program for every circuit, shard count and
restore setting (its steps replayed by the oracle on the state in physical
index order equal the circuit run directly), and two gloo ranks that each
hold half of a state and trade packed halves through TorchDistTransport
reproduce the oracle's state."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _three_qubit_circuit(n, seed):
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(12):
        k = int(rng.integers(1, 4))
        t = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
        gates.append(synth.Gate(t, synth.random_gate(k, rng, "dense")))
    return synth.Circuit(n, gates)


def _circuits(n):
    qft, j = synth.qft(n, seed=1)
    return [("qft", qft, synth.basis_state(n, j)), ("random", synth.random_layered(n, 3, seed=2),
                                                     synth.random_state(n, np.random.default_rng(3))),
            ("k3", _three_qubit_circuit(n, 4), synth.random_state(n, np.random.default_rng(5)))]


def replay_physical(steps, gates, n, n_local, psi_phys, theta=None):
    """Run a step list on the whole state in physical index order with the
    oracle: a gate on its local positions, an exchange as the SWAP of
    physical bits n_local + G and l, a local SWAP on its two positions."""
    psi = psi_phys
    for s in steps:
        if s["kind"] == "apply":
            g = gates[s["gate"]]
            psi = oracle.apply_gate(psi, list(s["targets"]), oracle.gate_matrix(g, theta))
        elif s["kind"] == "exchange":
            psi = oracle.apply_gate(psi, [n_local + s["global_bit"], s["local_bit"]], synth.SWAP)
        else:
            psi = oracle.apply_gate(psi, list(s["targets"]), synth.SWAP)
    return psi


def logical_from_physical(psi_phys, fmap):
    """State in logical index order: bit q of the logical index is bit
    fmap[q] of the physical one."""
    n = len(fmap)
    L = np.arange(1 << n)
    P = np.zeros_like(L)
    for q in range(n):
        P |= ((L >> q) & 1) << fmap[q]
    return psi_phys[P]


@pytest.mark.parametrize("g", [1, 2, 3])
@pytest.mark.parametrize("restore", [True, False])
def test_schedule_replays_to_the_circuit(api, g, restore):
    n = 8
    for name, circ, psi0 in _circuits(n):
        steps, fmap = api.shard_schedule(circ.gates, n, g, restore)
        assert sorted(fmap) == list(range(n))
        if restore:
            assert fmap == list(range(n))
        for s in steps:
            assert all(0 <= t < n - g for t in s["targets"]), (name, s)
            if s["kind"] == "exchange":
                assert 0 <= s["global_bit"] < g and 0 <= s["local_bit"] < n - g
        assert [s["gate"] for s in steps if s["kind"] == "apply"] == list(range(len(circ.gates)))
        got = logical_from_physical(replay_physical(steps, circ.gates, n, n - g, psi0, circ.theta), fmap)
        want = oracle.run_circuit(circ, psi0)
        assert np.max(np.abs(got - want)) < 1e-13, name


def test_schedule_without_global_targets_has_no_exchange(api):
    n = 10
    circ = synth.random_layered(6, 4, seed=0)  # qubits 0..5 only
    steps, fmap = api.shard_schedule(circ.gates, n, 3, True)
    assert all(s["kind"] == "apply" for s in steps) and fmap == list(range(n))


def test_schedule_rejects_gates_wider_than_a_shard(api):
    from paper_2405_01250_gb300._native import DiaqError
    g3 = synth.Gate((0, 1, 2), synth.random_gate(3, np.random.default_rng(0), "dense"))
    with pytest.raises(DiaqError, match="UNSUPPORTED"):
        api.shard_schedule([g3], 4, 2)
    with pytest.raises(DiaqError, match="ARG"):
        api.shard_schedule([g3], 4, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pack(shard, l, value):
    """Amplitudes of the shard whose local bit l equals value, in index order."""
    idx = np.arange(len(shard))
    return shard[((idx >> l) & 1) == value].copy()


def _unpack(shard, buf, l, value):
    idx = np.arange(len(shard))
    shard[((idx >> l) & 1) == value] = buf


def _rank_main(rank, world, port, n, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    import synth as S
    from paper_2405_01250_gb300 import api as A
    g = world.bit_length() - 1
    n_local = n - g
    results = {}
    for name, circ, psi0 in _circuits(n):
        shard = psi0.reshape(world, -1)[rank].copy()
        steps, fmap = A.shard_schedule(circ.gates, n, g, restore=True)
        tr = A.TorchDistTransport()
        for s in steps:
            if s["kind"] == "exchange":
                value = 1 - ((rank >> s["global_bit"]) & 1)
                send = torch.from_numpy(_pack(shard, s["local_bit"], value))
                recv = torch.empty_like(send)
                tr.exchange(rank ^ (1 << s["global_bit"]), send, recv)
                _unpack(shard, recv.numpy(), s["local_bit"], value)
            else:
                m = O.gate_matrix(circ.gates[s["gate"]], circ.theta) if s["kind"] == "apply" else S.SWAP
                shard = O.apply_gate(shard, list(s["targets"]), m)
        results[name] = shard
    out[rank] = results
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_exchange_halves_and_match_oracle(world):
    n = 8
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    for name, circ, psi0 in _circuits(n):
        got = np.concatenate([res[r][name] for r in range(world)])
        assert np.max(np.abs(got - oracle.run_circuit(circ, psi0))) < 1e-13, name
