"""Seeded circuit, state and observable generators (input data only).

Conventions, shared as *data layout* by both sides of every parity check:

* Qubit ``q`` is bit ``q`` of the basis index (qubit 0 is the least significant
  bit); a state of ``n`` qubits has ``N = 2**n`` complex amplitudes.
* A gate on targets ``(t_0, ..., t_{k-1})`` carries a ``2**k x 2**k`` matrix
  in the local basis whose most significant bit is ``t_0``: a CNOT with
  control ``c`` and target ``t`` is ``Gate((c, t), CNOT)``.
* A parametric gate carries no matrix. It names a Pauli generator ``gen``
  (one letter per target, first letter on ``t_0``), a parameter index and a
  scale; its operator is ``exp(-i * scale * theta[param] / 2 * P)``. Each
  consumer builds that matrix itself.
* An observable is a real-weighted Pauli sum given as ``(xmask, zmask,
  coeff)`` triples: bit ``q`` of ``xmask``/``zmask`` set means an X/Z factor
  on qubit ``q``; both set means Y.

The circuits stand in for the paper's SupermarQ GHZ and Hamiltonian-simulation
(TFIM) and QASMBench QFT workloads (Section VII), which are not available
here; the random-layer,
ansatz and QAOA circuits exercise the precision, adjoint and batching paths.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Fixed gate matrices (input constants)
# ----------------------------------------------------------------------------

H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
CNOT = np.array(
    [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128
)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
SWAP = np.array(
    [[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128
)


def cphase(phi: float) -> np.ndarray:
    """Controlled phase diag(1, 1, 1, e^{i phi})."""
    m = np.eye(4, dtype=np.complex128)
    m[3, 3] = complex(math.cos(phi), math.sin(phi))
    return m


def haar_u2(rng: np.random.Generator, dim: int = 2) -> np.ndarray:
    """Haar-random unitary by QR of a complex Gaussian with the phase fix of
    Mezzadri, "How to generate random matrices from the classical compact
    groups" (2007)."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return (q * (d / np.abs(d))).astype(np.complex128)


# ----------------------------------------------------------------------------
# Data classes
# ----------------------------------------------------------------------------


@dataclass(frozen=True)
class Gate:
    targets: tuple
    matrix: np.ndarray | None = None
    param: int = -1
    gen: str = ""
    scale: float = 1.0
    name: str = ""

    @property
    def k(self) -> int:
        return len(self.targets)

    @property
    def parametric(self) -> bool:
        return self.param >= 0


@dataclass
class Circuit:
    n: int
    gates: list
    theta: np.ndarray = field(default_factory=lambda: np.zeros(0))
    meta: dict = field(default_factory=dict)

    @property
    def n_params(self) -> int:
        return int(len(self.theta))


@dataclass
class Observable:
    xmask: np.ndarray
    zmask: np.ndarray
    coeff: np.ndarray

    @property
    def n_terms(self) -> int:
        return int(len(self.coeff))


def pauli_masks(letters: dict) -> tuple:
    """{qubit: 'X'|'Y'|'Z'|'I'} -> (xmask, zmask)."""
    x = z = 0
    for q, p in letters.items():
        p = p.upper()
        if p in ("X", "Y"):
            x |= 1 << q
        if p in ("Z", "Y"):
            z |= 1 << q
    return x, z


def _observable(terms: list) -> Observable:
    xs, zs, cs = [], [], []
    for letters, c in terms:
        x, z = pauli_masks(letters)
        xs.append(x)
        zs.append(z)
        cs.append(c)
    return Observable(
        np.array(xs, dtype=np.uint64), np.array(zs, dtype=np.uint64), np.array(cs, dtype=np.float64)
    )


# ----------------------------------------------------------------------------
# States
# ----------------------------------------------------------------------------


def basis_state(n: int, j: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[j] = 1.0
    return psi


def random_state(n: int, rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return (v / np.linalg.norm(v)).astype(np.complex128)


# ----------------------------------------------------------------------------
# Circuits
# ----------------------------------------------------------------------------


def ghz(n: int) -> Circuit:
    """GHZ preparation: H on qubit 0, then the CNOT chain q_k -> q_{k+1}."""
    gates = [Gate((0,), H, name="h")]
    for k in range(n - 1):
        gates.append(Gate((k, k + 1), CNOT, name="cx"))
    return Circuit(n, gates, meta={"workload": f"ghz-{n}"})


def qft(n: int, seed: int = 0) -> tuple:
    """QFT of a seeded basis state |j>, textbook interleaved order with
    qubit 0 as the least significant bit:

        for b = n-1 .. 0:  H(b); for c = b-1 .. 0: CP(c, b, 2*pi / 2**(b-c+1))
        then SWAP(b, n-1-b) for b < n/2.

    Returns (circuit, j). The intended output is e^{2 pi i j k / 2^n} / sqrt(2^n).
    """
    rng = np.random.default_rng(seed)
    j = int(rng.integers(0, 1 << n))
    gates = []
    for b in range(n - 1, -1, -1):
        gates.append(Gate((b,), H, name="h"))
        for c in range(b - 1, -1, -1):
            m = b - c + 1
            gates.append(Gate((c, b), cphase(2.0 * math.pi / (1 << m)), name="cp"))
    for b in range(n // 2):
        gates.append(Gate((b, n - 1 - b), SWAP, name="swap"))
    return Circuit(n, gates, meta={"workload": f"qft-{n}", "j": j}), j


def random_layered(n: int, depth: int, seed: int = 0) -> Circuit:
    """Layers of Haar U(2) on every qubit followed by CZ on a seeded random
    perfect matching (n even)."""
    if n % 2:
        raise ValueError("random_layered needs an even qubit count")
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(depth):
        for q in range(n):
            gates.append(Gate((q,), haar_u2(rng), name="u2"))
        perm = rng.permutation(n)
        for a in range(0, n, 2):
            u, v = int(perm[a]), int(perm[a + 1])
            gates.append(Gate((u, v), CZ, name="cz"))
    return Circuit(n, gates, meta={"workload": f"random-{n}-d{depth}"})


def ansatz(n: int = 20, layers: int = 8, seed: int = 0) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(theta) then RZ(phi) on each
    qubit (circuit order), then the CZ ladder CZ(i, i+1), i = 0..n-2.
    Parameters uniform in [0, 2 pi); RY on qubit q of layer l uses index
    2*(l*n + q), RZ the next one."""
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=2 * n * layers)
    gates = []
    for l in range(layers):
        for q in range(n):
            p = 2 * (l * n + q)
            gates.append(Gate((q,), None, param=p, gen="Y", name="ry"))
            gates.append(Gate((q,), None, param=p + 1, gen="Z", name="rz"))
        for q in range(n - 1):
            gates.append(Gate((q, q + 1), CZ, name="cz"))
    return Circuit(n, gates, theta=theta, meta={"workload": f"ansatz-{n}-l{layers}"})


def ansatz_observable(n: int = 20) -> Observable:
    """H = sum_i Z_i Z_{i+1} (open chain) + 0.5 sum_i X_i."""
    terms = [({i: "Z", i + 1: "Z"}, 1.0) for i in range(n - 1)]
    terms += [({i: "X"}, 0.5) for i in range(n)]
    return _observable(terms)


def tfim(n: int, steps: int, dt: float, J: float = 1.0, h: float = 1.0) -> Circuit:
    """First-order Trotter circuit of the 1D transverse-field Ising model
    H = -J sum_{i<n-1} Z_i Z_{i+1} - h sum_i X_i (open chain), the paper's
    Hamiltonian-simulation (HAM) workload, from |0...0>. Each of `steps`
    steps applies exp(+i J dt Z_i Z_{i+1}) on every bond (i = 0..n-2), then
    exp(+i h dt X_i) on every qubit. As parametric gates exp(-i a/2 P):
    every bond gate uses theta[0] = -2 J dt (generator ZZ), every field gate
    theta[1] = -2 h dt (generator X)."""
    gates = []
    for _ in range(steps):
        for i in range(n - 1):
            gates.append(Gate((i, i + 1), None, param=0, gen="ZZ", name="rzz"))
        for q in range(n):
            gates.append(Gate((q,), None, param=1, gen="X", name="rx"))
    theta = np.array([-2.0 * J * dt, -2.0 * h * dt], dtype=np.float64)
    return Circuit(n, gates, theta=theta,
                   meta={"workload": f"tfim-{n}-s{steps}", "J": J, "h": h, "dt": dt, "steps": steps})


def magnetisation_observable(n: int) -> Observable:
    """Average magnetisation M_z = (1/n) sum_i Z_i."""
    return _observable([({i: "Z"}, 1.0 / n) for i in range(n)])


def _random_3_regular(n: int, rng: np.random.Generator) -> list:
    """Pairing (configuration) model with rejection of loops and multi-edges."""
    if (3 * n) % 2:
        raise ValueError("3-regular graph needs an even vertex count")
    for _ in range(10000):
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        edges = set()
        ok = True
        for a in range(0, len(stubs), 2):
            u, v = int(stubs[a]), int(stubs[a + 1])
            if u == v:
                ok = False
                break
            e = (min(u, v), max(u, v))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)
    raise RuntimeError("no simple 3-regular graph found")


def qaoa_instance(n: int, rng: np.random.Generator, p: int = 4) -> tuple:
    """QAOA MaxCut on a seeded random 3-regular graph: |+>^n by H on every
    qubit, then per layer l RZZ(gamma_l) on every edge and RX(beta_l) on every
    qubit. theta = (gamma_1..gamma_p, beta_1..beta_p), uniform in [0, pi).
    Returns (circuit, observable H_C = sum_edges Z_u Z_v)."""
    edges = _random_3_regular(n, rng)
    gamma = rng.uniform(0.0, math.pi, size=p)
    beta = rng.uniform(0.0, math.pi, size=p)
    gates = [Gate((q,), H, name="h") for q in range(n)]
    for l in range(p):
        for (u, v) in edges:
            gates.append(Gate((u, v), None, param=l, gen="ZZ", name="rzz"))
        for q in range(n):
            gates.append(Gate((q,), None, param=p + l, gen="X", name="rx"))
    obs = _observable([({u: "Z", v: "Z"}, 1.0) for (u, v) in edges])
    circ = Circuit(n, gates, theta=np.concatenate([gamma, beta]),
                   meta={"workload": f"qaoa-{n}-p{p}", "edges": edges})
    return circ, obs


def qaoa_batch(count: int = 256, seed: int = 0, sizes=(14, 16, 18, 20, 22), p: int = 4) -> list:
    """`count` QAOA instances with n drawn uniformly from `sizes`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(sizes[int(rng.integers(0, len(sizes)))])
        out.append(qaoa_instance(n, rng, p))
    return out


# ----------------------------------------------------------------------------
# Random gates for parity tests
# ----------------------------------------------------------------------------


def random_gate(k: int, rng: np.random.Generator, kind: str = "dense") -> np.ndarray:
    """A random 2^k x 2^k gate matrix of a given structural class:
    'dense' (Haar), 'real' (real orthogonal), 'diag' (random phases),
    'perm' (permutation), 'monomial' (permutation times phases),
    'sparse' (Haar with a random pattern of exact zeros; not unitary)."""
    d = 1 << k
    if kind == "dense":
        return haar_u2(rng, d)
    if kind == "real":
        q, r = np.linalg.qr(rng.standard_normal((d, d)))
        return (q * np.sign(np.diag(r))).astype(np.complex128)
    if kind == "diag":
        return np.diag(np.exp(1j * rng.uniform(0, 2 * math.pi, d))).astype(np.complex128)
    if kind == "perm":
        return np.eye(d, dtype=np.complex128)[rng.permutation(d)]
    if kind == "monomial":
        m = np.eye(d, dtype=np.complex128)[rng.permutation(d)]
        return m * np.exp(1j * rng.uniform(0, 2 * math.pi, d))[:, None]
    if kind == "sparse":
        m = haar_u2(rng, d)
        mask = rng.random((d, d)) < 0.5
        return np.where(mask, 0.0, m).astype(np.complex128)
    raise ValueError(kind)
