"""GPU parity of the sharded state on one device: 2 and 4 shards of one
state in one process, run by the native runner (diaq_sharded_simulate, with
the in-place pair swap) and by the rank-structured path (ShardRank: pack,
buffer trade, unpack, as separate ranks would do with NCCL; the trade here
is a device copy), against the FP64 oracle; sharded norm and expectation;
the slice-move kernels against the index permutation they define."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, c64_circuit_bound, host, qft_amplitudes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def logical(psi_phys, fmap):
    n = len(fmap)
    L = np.arange(1 << n)
    P = np.zeros_like(L)
    for q in range(n):
        P |= ((L >> q) & 1) << fmap[q]
    return psi_phys[P]


@pytest.mark.parametrize("g", [1, 2])
def test_qft18_on_shards_matches_closed_form(api, g):
    n = 18
    circ, j = synth.qft(n, seed=3)
    full = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    full[j] = 1
    st = api.ShardedState.from_full(full, g).simulate(circ.gates, restore=True)
    assert st.map == list(range(n))
    got = host(st.physical())
    assert np.max(np.abs(got - qft_amplitudes(n, j, np.arange(1 << n)))) <= TOL_C128
    assert abs(st.norm() - 1.0) < 1e-12


@pytest.mark.parametrize("g", [1, 2])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("restore", [True, False])
def test_random16_on_shards_matches_oracle(api, g, dtype, restore):
    n = 16
    circ = synth.random_layered(n, 6, seed=g)
    psi0 = synth.random_state(n, np.random.default_rng(9))
    want = oracle.run_circuit(circ, psi0)
    st = api.ShardedState.from_full(torch.as_tensor(psi0).to(device="cuda", dtype=dtype), g)
    st.simulate(circ.gates, restore=restore)
    got = logical(host(st.physical()), st.map)
    if dtype == torch.complex128:
        assert np.max(np.abs(got - want)) <= TOL_C128
    else:
        # exchanges and SWAPs move amplitudes exactly; the bound is the gates'
        ks = [0 if gt.name == "cz" else gt.k for gt in circ.gates]
        assert np.max(np.abs(got - want)) <= c64_circuit_bound(ks) + 2.0 ** -24
    if not restore:
        assert sorted(st.map) == list(range(n))


def test_parametric_and_three_qubit_gates_on_shards(api):
    n = 12
    rng = np.random.default_rng(4)
    gates = [synth.Gate((11, 0, 6), synth.random_gate(3, rng, "dense")),
             synth.Gate((10, 11), None, param=0, gen="XY"),
             synth.Gate((1, 10, 5), None, param=1, gen="ZYX", scale=0.5),
             synth.Gate((11,), synth.H)]
    theta = np.array([0.7, -1.9])
    circ = synth.Circuit(n, gates, theta=theta)
    psi0 = synth.random_state(n, rng)
    st = api.ShardedState.from_full(torch.as_tensor(psi0).cuda(), 2).simulate(gates, theta=theta)
    assert np.max(np.abs(host(st.physical()) - oracle.run_circuit(circ, psi0))) <= TOL_C128


@pytest.mark.parametrize("g", [1, 2])
def test_sharded_norm_and_expect(api, g):
    n = 14
    circ = synth.random_layered(n, 3, seed=5)
    psi0 = synth.basis_state(n, 0)
    want = oracle.run_circuit(circ, psi0)
    st = api.ShardedState.from_full(torch.as_tensor(psi0).cuda(), g).simulate(circ.gates, restore=False)
    assert abs(st.norm() - oracle.norm2(want)) < 1e-13
    # Z on every qubit pair (global ones included), X and Y on qubits that
    # the final map keeps local
    local_q = [q for q in range(n) if st.map[q] < n - g]
    terms = [({q: "Z", (q + 1) % n: "Z"}, 0.7) for q in range(n)]
    terms += [({q: "X"}, 0.3) for q in local_q[:4]] + [({local_q[0]: "Y", local_q[2]: "X", n - 1: "Z"}, -1.1)]
    xs, zs, cs = [], [], []
    for letters, c in terms:
        x, z = synth.pauli_masks(letters)
        xs.append(x)
        zs.append(z)
        cs.append(c)
    obs = synth.Observable(np.array(xs, np.uint64), np.array(zs, np.uint64), np.array(cs))
    got = st.expect(obs.xmask, obs.zmask, obs.coeff)
    assert abs(got - oracle.expect(want, obs)) < 1e-12
    # an X on a qubit held on a global bit is refused
    gq = [q for q in range(n) if st.map[q] >= n - g][0]
    from paper_2405_01250_gb300._native import DiaqError
    with pytest.raises(DiaqError, match="UNSUPPORTED"):
        st.expect([1 << gq], [0], [1.0])


@pytest.mark.parametrize("g", [1, 2])
def test_rank_structured_path_equals_native_runner(api, g):
    """2^g ShardRank objects stepped together, each exchange as pack ->
    device copy of the partner's buffer -> unpack: the same bits as the
    native runner (every move is exact, every local op the same kernel)."""
    n = 16
    circ, j = synth.qft(n, seed=8)
    full = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    full[j] = 1
    ref = api.ShardedState.from_full(full, g).simulate(circ.gates, restore=True)
    ranks = [api.ShardRank(r, n, g, s.clone()) for r, s in enumerate(full.reshape(1 << g, -1))]
    plans = [rk.plan(circ.gates) for rk in ranks]
    steps = plans[0]
    assert all(p == steps for p in plans)
    for i, s in enumerate(steps):
        if s["kind"] == "exchange":
            for rk in ranks:
                rk.pack(s)
            for rk in ranks:
                rk.recv.copy_(ranks[rk.partner(s)].send)
            for rk in ranks:
                rk.unpack(s)
        else:
            for rk in ranks:
                rk.apply_step(i, s)
    got = torch.cat([rk.shard for rk in ranks])
    assert torch.equal(got, ref.physical())


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("n_local,l", [(1, 0), (5, 0), (5, 3), (13, 12), (13, 7)])
def test_slice_move_kernels(api, dtype, n_local, l):
    from paper_2405_01250_gb300 import _native
    L = _native.lib()
    code = 1 if dtype == torch.complex128 else 0
    rng = np.random.default_rng(n_local * 10 + l)
    a0 = synth.random_state(n_local, rng)
    b0 = synth.random_state(n_local, rng)
    a = torch.as_tensor(a0).to(device="cuda", dtype=dtype)
    b = torch.as_tensor(b0).to(device="cuda", dtype=dtype)
    idx = np.arange(1 << n_local)
    hi = ((idx >> l) & 1) == 1
    vp = ctypes.c_void_p
    assert L.diaq_shard_swap(vp(a.data_ptr()), vp(b.data_ptr()), n_local, code, l, None) == 0
    wa, wb = a0.copy(), b0.copy()
    wa[hi], wb[~hi] = b0[~hi], a0[hi]
    cast = np.complex64 if dtype == torch.complex64 else np.complex128
    assert np.array_equal(host(a), wa.astype(cast).astype(np.complex128))
    assert np.array_equal(host(b), wb.astype(cast).astype(np.complex128))
    buf = torch.empty(max(1, (1 << n_local) // 2), dtype=dtype, device="cuda")
    for value in (0, 1):
        assert L.diaq_shard_pack(vp(a.data_ptr()), n_local, code, l, value, vp(buf.data_ptr()), None) == 0
        sel = (((idx >> l) & 1) == value)
        assert np.array_equal(host(buf), host(a)[sel])
        c = torch.zeros_like(a)
        assert L.diaq_shard_unpack(vp(buf.data_ptr()), vp(c.data_ptr()), n_local, code, l, value, None) == 0
        assert np.array_equal(host(c)[sel], host(a)[sel]) and not np.any(host(c)[~sel])
    # overlapping shards and an out-of-range bit are refused
    assert L.diaq_shard_swap(vp(a.data_ptr()), vp(a.data_ptr()), n_local, code, l, None) == 1
    assert L.diaq_shard_pack(vp(a.data_ptr()), n_local, code, n_local, 0, vp(buf.data_ptr()), None) == 1
