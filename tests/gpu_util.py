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
