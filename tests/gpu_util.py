"""Helpers for the GPU parity tests (tolerances, transfers)."""

import math

import numpy as np
import torch

# complex128: the maximum absolute amplitude error allowed against the FP64 oracle
TOL_C128 = 1e-12


def tol_c64(k: int, scale: float) -> float:
    """One gate in complex64: each output sums 2^k products, each with a
    rounded input (2^-24), a rounded matrix entry (2^-24) and a rounded
    product/sum (2^-24) relative to |M||x| <= scale; a factor of 2 margin."""
    return 2.0 * (2 ** k) * 3 * 2.0 ** -24 * scale


def dev(x: np.ndarray, dtype=torch.complex128) -> torch.Tensor:
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype).contiguous()


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128)


def maxerr(a, b) -> float:
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0


def qft_amplitudes(n: int, j: int, ks: np.ndarray) -> np.ndarray:
    """Closed-form QFT output e^{2 pi i j k / 2^n} / sqrt(2^n), phase reduced
    exactly modulo 2^n in integers before the FP64 sincos."""
    N = 1 << n
    ks = np.asarray(ks, dtype=np.uint64)
    ph = ((np.uint64(j) * ks) % np.uint64(N)).astype(np.float64) / N
    return np.exp(2j * np.pi * ph) / math.sqrt(N)


U32 = 2.0 ** -24  # unit roundoff of FP32


def c64_gate_bound(k: int) -> float:
    """Worst-case growth of the 2-norm error vector, in units of FP32's unit
    roundoff u, when a k-qubit unitary M (stored in FP32) is applied in
    complex64 to a state of 2-norm 1. Each output row sums 2^k complex
    products, i.e. 2^(k+1) real products per real component, so its rounding
    error is at most gamma_{2^(k+1)+1} * (|M||x|)_r; rounding the entries of
    M to FP32 adds u |M| |x| (sqrt(2) for the two parts). Over a group of 2^k
    rows the 2-norm of |M||x| is at most ||M||_F ||x|| = 2^(k/2) ||x||, and
    the groups are orthogonal, so the whole state's error grows by at most
    ((2^(k+1) + 1) * 1.01 + sqrt(2)) * 2^(k/2) * u."""
    return ((2 ** (k + 1) + 1) * 1.01 + math.sqrt(2.0)) * 2.0 ** (k / 2.0)


def c64_circuit_bound(ks) -> float:
    """Bound B on ||psi_c64 - psi_exact||_2 (hence on the largest amplitude
    error) for a circuit of unitary gates on k_i qubits applied in complex64
    to a unit state: the error of gate l is carried forward unchanged in norm
    by the later (unitary) gates, so the per-gate bounds add. Gates whose
    entries are all 0 or +-1 (CZ, CNOT, SWAP) are exact in FP32 and pass
    k = 0 here."""
    return 1.01 * U32 * sum(c64_gate_bound(k) for k in ks if k > 0)


def fidelity_loss_bound(b: float) -> float:
    """For unit a and b = a + d with ||d|| <= B: 1 - |<a|b>|^2 / ||b||^2 =
    (||d||^2 - |<a|d>|^2) / ||b||^2 <= B^2 / (1 - B)^2."""
    return b * b / (1.0 - b) ** 2
