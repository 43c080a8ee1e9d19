"""Failure detection without a GPU fault: the library's allocations are made
to fail on the host, one position at a time (diaq_debug_inject_alloc_failure),
for operations that allocate device or pinned memory. Each call either
succeeds with the right result or fails with a status, releases what it had
allocated, and leaves the library usable; afterwards the same operations give
the same results and device memory has not leaked."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL_C128, dev, host, maxerr

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(55)


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    yield A
    A.inject_alloc_failure(-1)


def _ops(api):
    """(name, callable returning a float array) for operations that allocate."""
    n = 9
    x = synth.random_state(n, RNG)
    xt = dev(x)
    circ = synth.ansatz(n=6, layers=1, seed=7)
    obs = synth.ansatz_observable(6)
    qa, qo = synth.qaoa_instance(6, RNG, p=1)
    m2 = synth.random_gate(2, RNG)

    def stored_apply():
        op = api.build(synth.Gate((4, 1), m2), n, variant="stored")
        y = torch.empty_like(xt)
        api.apply(op, xt, y)
        return host(y).view(np.float64)

    def raw_fuse():
        ops = []
        for q in (0, 3):
            offs, vals = oracle.gate_diaq(n, (q,), synth.H)
            ops.append(api.build_diaq(n, offs, vals))
        f = api.fuse(ops)
        y = torch.empty_like(xt)
        api.apply(f, xt, y)
        return host(y).view(np.float64)

    def chain():
        op, nd, nz = api.unitary_chain(synth.ghz(5).gates, 5)
        return np.concatenate([nd, nz]).astype(np.float64)

    def reductions():
        e = api.expect(xt, obs.xmask[:3], obs.zmask[:3], obs.coeff[:3])
        return np.array([api.norm(xt), e.real, e.imag])

    def adjoint():
        p0 = torch.zeros(64, dtype=torch.complex128, device="cuda")
        p0[0] = 1
        e, g = api.adjoint_grad(circ.gates, circ.theta, obs.xmask, obs.zmask, obs.coeff, p0,
                                torch.empty_like(p0), torch.empty_like(p0))
        return np.concatenate([[e], g])

    def plan():
        pl = api.AdjointPlan(circ.gates, circ.n_params, (obs.xmask, obs.zmask, obs.coeff), 6)
        pl.set_sweep(4, 4)
        e, g = pl.run(circ.theta)
        pl.close()
        return np.concatenate([[e], g])

    def batch():
        b = api.Batch([(6, qa.gates, qa.n_params, (qo.xmask, qo.zmask, qo.coeff))] * 2)
        b.set_sweep(3, 1)
        b.set_launch(2, 128)
        E, G = b.run(np.concatenate([qa.theta, qa.theta]))
        b.close()
        return np.concatenate([E, G[0], G[1]])

    return [("stored_apply", stored_apply), ("raw_fuse", raw_fuse), ("chain", chain),
            ("reductions", reductions), ("adjoint", adjoint), ("plan", plan), ("batch", batch)]


def test_injected_allocation_failures_are_clean(api):
    from paper_2405_01250_gb300._native import DiaqError
    ops = _ops(api)
    ref = {name: f() for name, f in ops}
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for name, f in ops:
        for k in range(0, 14):
            api.inject_alloc_failure(k)
            try:
                got = f()
            except DiaqError as e:
                failures += 1
                assert "ERR_ALLOC" in str(e) or "ERR_CUDA" in str(e), (name, k, str(e))
            else:
                assert maxerr(got, ref[name]) <= TOL_C128, (name, k)
            finally:
                api.inject_alloc_failure(-1)
        # the library is usable afterwards and gives the same result
        assert maxerr(f(), ref[name]) <= TOL_C128, name
    assert failures >= len(ops)  # every operation met at least one injected failure
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (128 << 20), (free0, free1)


def test_injection_argument_check(api):
    from paper_2405_01250_gb300._native import DiaqError
    with pytest.raises(DiaqError):
        api.inject_alloc_failure(-2)
    api.inject_alloc_failure(-1)
