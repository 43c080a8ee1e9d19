"""C-ABI checks that need no GPU: the library loads and exports every symbol
include/diaq.h declares, and the host parts of the path (builder offsets,
Algorithm 1 product, gate fusion, argument validation) agree with the
oracle."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RNG = np.random.default_rng(77)


@pytest.fixture(scope="module")
def api():
    from paper_2405_01250_gb300 import build as B
    B.build()
    from paper_2405_01250_gb300 import api as A
    return A


def _header_functions():
    txt = open(os.path.join(ROOT, "include", "diaq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(diaq_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(api):
    from paper_2405_01250_gb300 import _native
    names = _header_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(_native.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_native.SIGNATURES), "binding and header disagree"
    assert "sm_103a" in api.version()


@pytest.mark.parametrize("n,k", [(3, 1), (6, 2), (8, 3), (5, 2), (7, 4), (8, 5), (8, 6)])
def test_gate_offsets_match_oracle(api, n, k):
    for kind in ("dense", "sparse", "perm", "diag", "monomial"):
        t = [int(q) for q in RNG.choice(n, size=k, replace=False)]
        m = synth.random_gate(k, RNG, kind)
        got = api.gate_offsets(synth.Gate(tuple(t), m), n)
        want, _ = oracle.gate_diaq(n, t, m)
        assert list(got) == list(want), (kind, t)


def test_gate_offsets_paper_patterns(api):
    # Fig. 3: single H in a 4-qubit circuit; Section III-A: Z is the principal diagonal
    for q, below in ((3, 8), (2, 4), (1, 2), (0, 1)):
        assert list(api.gate_offsets(synth.Gate((q,), synth.H), 4)) == [-below, 0, below]
        assert list(api.gate_offsets(synth.Gate((q,), np.diag([1, -1]).astype(complex)), 4)) == [0]
    # CNOT chain of GHZ-12: offsets 0, +-2^(k+1)
    for k in range(11):
        assert list(api.gate_offsets(synth.Gate((k, k + 1), synth.CNOT), 12)) == [-(2 << k), 0, 2 << k]
    # parametric gates: structure of I and the generator, independent of theta
    g = synth.Gate((2, 5), None, param=0, gen="ZZ")
    assert list(api.gate_offsets(g, 6)) == [0]
    g = synth.Gate((3,), None, param=0, gen="Y")
    assert list(api.gate_offsets(g, 6)) == [-8, 0, 8]


def _dense_from(N, idx, vals):
    A = np.zeros((N, N), dtype=np.complex128)
    for d, v in zip(idx, vals):
        r0, c0 = max(0, -int(d)), max(0, int(d))
        t = np.arange(len(v))
        A[r0 + t, c0 + t] = v
    return A


def test_algorithm1_product_matches_dense(api):
    for N in (1, 5, 16, 33):
        A = RNG.standard_normal((N, N)) + 1j * RNG.standard_normal((N, N))
        B = RNG.standard_normal((N, N)) + 1j * RNG.standard_normal((N, N))
        A *= RNG.random((N, N)) < 0.2
        B *= RNG.random((N, N)) < 0.2
        ai, av = oracle.dense_to_diaq(A)
        bi, bv = oracle.dense_to_diaq(B)
        ci, cv = api.diaq_matmul_host(N, ai, av, bi, bv)
        assert list(ci) == sorted(ci)
        np.testing.assert_allclose(_dense_from(N, ci, cv), A @ B, atol=1e-12)


def test_algorithm1_accumulates_coinciding_diagonals(api):
    """H * H: three (a, b) pairs meet on index 0. Overwriting (a literal
    reading of the listing) would not give the identity."""
    ai, av = oracle.dense_to_diaq(synth.H)
    ci, cv = api.diaq_matmul_host(2, ai, av, ai, av)
    np.testing.assert_allclose(_dense_from(2, ci, cv), np.eye(2), atol=1e-15)


def test_fuse_gates_host_matches_oracle(api):
    n = 8
    for trial in range(6):
        gates = []
        for _ in range(int(RNG.integers(1, 5))):
            k = int(RNG.integers(1, 3))
            t = tuple(int(q) for q in RNG.choice(n, size=k, replace=False))
            gates.append(synth.Gate(t, synth.random_gate(k, RNG, ["dense", "diag", "perm"][trial % 3])))
        union = []
        for g in gates:
            for q in g.targets:
                if q not in union:
                    union.append(q)
        if len(union) > 6:
            continue
        ut, F = api.fuse_gates_host(gates)
        uo, Fo = oracle.fuse([(g.targets, g.matrix) for g in gates])
        assert tuple(ut) == tuple(uo)
        np.testing.assert_allclose(F, Fo, atol=1e-13)


def test_fuse_gates_host_parametric(api):
    th = np.array([0.7, -1.3])
    gates = [synth.Gate((0,), None, param=0, gen="Y"), synth.Gate((0, 1), None, param=1, gen="ZZ", scale=2.0)]
    ut, F = api.fuse_gates_host(gates, th)
    _, Fo = oracle.fuse([(g.targets, oracle.gate_matrix(g, th)) for g in gates])
    np.testing.assert_allclose(F, Fo, atol=1e-14)


def test_argument_validation_without_gpu(api):
    from paper_2405_01250_gb300._native import DiaqError
    with pytest.raises(DiaqError, match="ERR_ARG"):
        api.gate_offsets(synth.Gate((1, 1), synth.CNOT), 4)     # repeated target
    with pytest.raises(DiaqError, match="ERR_ARG"):
        api.gate_offsets(synth.Gate((4,), synth.H), 4)          # target outside register
    with pytest.raises(DiaqError, match="ERR_SHAPE"):
        api.gate_offsets(synth.Gate((0, 1, 2), synth.random_gate(3, RNG)), 2)  # k > n
    with pytest.raises(DiaqError, match="ERR_ARG"):
        api.gate_offsets(synth.Gate((0,), None, param=0, gen="Q"), 3)  # bad generator letter
    with pytest.raises(DiaqError, match="ERR_SHAPE"):
        api.diaq_matmul_host(4, [5], [np.zeros(1)], [0], [np.ones(4)])  # index outside the matrix
    with pytest.raises(DiaqError, match="ERR_UNSUPPORTED"):
        api.fuse_gates_host([synth.Gate((q,), synth.H) for q in range(7)])


def test_device_entry_points_fail_loudly_without_gpu(api):
    """On a machine with no GPU the device path reports an error; it never
    falls back to a CPU computation."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2405_01250_gb300._native import DiaqError
    with pytest.raises(DiaqError):
        api.build(synth.Gate((0,), synth.H), 4, stream=0)


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of include/diaq.h has the same size and field offsets in
    C (gcc, from the header itself) as in the ctypes binding."""
    import subprocess

    from paper_2405_01250_gb300 import _native as N
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = open(os.path.join(root, "include", "diaq.h")).read()
    structs = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(diaq_\w+);", hdr, re.S):
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"(\w+)\s*(?:\[[^\]]*\])?\s*;", body)
        structs[name] = fields
    assert set(structs) == {"diaq_gate", "diaq_op_info", "diaq_plan_tuning", "diaq_apply_tuning",
                            "diaq_fusion_tuning", "diaq_batch_tuning", "diaq_shard_step"}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "diaq.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    c_layout = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = ln.split()
        c_layout[(a, b)] = int(v)
    for name, fields in structs.items():
        cls = getattr(N, name)
        assert [f[0] for f in cls._fields_] == fields, name
        assert ctypes.sizeof(cls) == c_layout[(name, "size")], name
        for f in fields:
            assert getattr(cls, f).offset == c_layout[(name, f)], (name, f)


def test_binding_signatures_match_the_header():
    """Every function the header declares has a binding entry with the same
    number of arguments, each of the same kind (32-bit integer or enum,
    64-bit integer, double, pointer or handle), and the same return kind."""
    import ctypes as C

    from paper_2405_01250_gb300 import _native as N
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(root, "include", "diaq.h")).read(), flags=re.S)
    protos = re.findall(r"(diaq_status|const char\s*\*)\s*(diaq_\w+)\s*\(([^;]*?)\)\s*;", hdr, re.S)
    assert len(protos) == len(N.SIGNATURES)

    def c_kind(decl):
        decl = " ".join(decl.split())
        if "*" in decl or re.match(r"(const )?diaq_\w+_t\b", decl):
            return "ptr"
        base = decl.split()[0] if not decl.startswith("const ") else decl.split()[1]
        if base in ("int32_t", "int", "diaq_dtype", "diaq_variant"):
            return "i32"
        if base in ("int64_t", "uint64_t"):
            return "i64"
        if base == "double":
            return "f64"
        raise AssertionError(f"unclassified C parameter type: {decl}")

    def py_kind(t):
        if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
            return "ptr"
        if C.sizeof(t) == 4 and t in (C.c_int32, C.c_int):
            return "i32"
        if t in (C.c_int64, C.c_uint64):
            return "i64"
        if t is C.c_double:
            return "f64"
        raise AssertionError(f"unclassified ctypes type: {t}")

    for ret, name, params in protos:
        assert name in N.SIGNATURES, name
        res, args = N.SIGNATURES[name]
        params = params.strip()
        kinds = [] if params in ("", "void") else [c_kind(p) for p in params.split(",")]
        assert [py_kind(a) for a in args] == kinds, name
        assert (res is C.c_char_p) == ret.startswith("const char"), name


def test_debug_bounds_status_plumbing():
    """The debug build's status path on the CPU: the recorded word decodes to
    DIAQ_ERR_BOUNDS with the site and the index (negative indices included);
    an empty word is DIAQ_OK; the normal build reports its checks as off and
    the debug build as on."""
    import ctypes as C
    import subprocess
    import sys

    from paper_2405_01250_gb300 import _native as N
    L = N.lib()
    assert L.diaq_debug_bounds_status(0) == 0
    site, idx = 6, 123456789
    w = (1 << 63) | (site << 48) | idx
    assert L.diaq_debug_bounds_status(w) == 6
    msg = L.diaq_last_error().decode()
    assert "stored SpMV column" in msg and "123456789" in msg
    neg = (1 << 63) | (10 << 48) | ((-5) & 0xFFFFFFFFFFFF)
    assert L.diaq_debug_bounds_status(neg) == 6 and "index -5" in L.diaq_last_error().decode()
    on = C.c_int32(7)
    assert L.diaq_debug_bounds_enabled(C.byref(on)) == 0
    assert on.value == (1 if N.DEBUG_BOUNDS else 0)
    # the debug build compiles and reports its checks as on (in a fresh process)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import ctypes, sys; sys.path.insert(0, %r); "
            "from paper_2405_01250_gb300 import build as B; p = B.build(debug_bounds=True); "
            "L = ctypes.CDLL(p); v = ctypes.c_int32(0); "
            "assert L.diaq_debug_bounds_enabled(ctypes.byref(v)) == 0 and v.value == 1; print('dbg ok')" % root)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert "dbg ok" in out.stdout, out.stderr[-2000:]
