"""The index arithmetic the diagonal-run and lambda kernels rely on, checked
on the CPU by enumerating their loop order (no GPU): amplitudes by aligned
blocks of 256, warp w of the grid taking blocks w, w + W, ..., lane l the
amplitudes l + 32 j (j = 0..7) of each.

- Every amplitude is visited exactly once, also for states below one block.
- In the reverse chunk-form kernel (256 threads per block, P blocks,
  W = 8 P warps) bits 5..7 of the index are j, bits 8..10 the warp within
  its block and bits 11 .. 10 + z (z = trailing zero bits of P) the block
  index: the bits whose gradient terms come from per-thread totals.
- The weight form's W(i) = sum_g (-1)^popc(i & z_g), and lambda's count of
  odd parities of a group sharing an X mask, follow for the eight amplitudes
  of a lane from per-class sums over the masks' other bits and a
  Walsh-Hadamard transform over j."""

import numpy as np
import pytest


def popc(v):
    return bin(v).count("1")


def order(n, P):
    """(block index, warp, lane, j, amplitude) in the kernels' loop order."""
    N = 1 << n
    nblk = (N + 255) >> 8
    W = 8 * P
    for b in range(P):
        for warp in range(8):
            blk = b * 8 + warp
            while blk < nblk:
                base = blk << 8
                for lane in range(32):
                    for j in range(8):
                        i = base + lane + 32 * j
                        if i >= N:
                            break
                        yield b, warp, lane, j, i
                blk += W


@pytest.mark.parametrize("n", [2, 5, 8, 9, 13])
@pytest.mark.parametrize("P", [1, 3, 4, 6, 16])
def test_block_order_visits_every_amplitude_once_with_fixed_bits(n, P):
    N = 1 << n
    f = 11 + ((P & -P).bit_length() - 1)
    seen = np.zeros(N, dtype=np.int64)
    for b, warp, lane, j, i in order(n, P):
        seen[i] += 1
        assert i & 31 == lane and (i >> 5) & 7 == j
        for q in range(8, min(f, n)):
            want = (warp >> (q - 8)) & 1 if q < 11 else (b >> (q - 11)) & 1
            assert (i >> q) & 1 == want
    assert np.all(seen == 1)


def _class_counts(y_masked, zs):
    """Per-class sizes and odd-parity sums of masks grouped by bits 5..7."""
    n_k = [0] * 8
    odd_k = [0] * 8
    for z in zs:
        k = (z >> 5) & 7
        n_k[k] += 1
        odd_k[k] += popc(y_masked & z) & 1
    return n_k, odd_k


def _wht8(d):
    d = list(d)
    h = 1
    while h < 8:
        for k in range(8):
            if not k & h:
                d[k], d[k + h] = d[k] + d[k + h], d[k] - d[k + h]
        h <<= 1
    return d


@pytest.mark.parametrize("seed", range(6))
def test_weight_form_and_lambda_counts_by_class_transform(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 13))
    N = 1 << n
    zs = [int(rng.integers(0, N)) for _ in range(int(rng.integers(2, 30)))]
    x = int(rng.integers(0, N))
    for blk in range((N + 255) >> 8):
        base = blk << 8
        for lane in range(32):
            # weight form: W_j = WHT_j(C), C_k = n_k - 2 odd_k with y = base | lane
            n_k, odd_k = _class_counts((base | lane) & ~0xE0, zs)
            Wj = _wht8([n_k[k] - 2 * odd_k[k] for k in range(8)])
            # lambda: odd count of (i ^ x) & z_u for the eight j
            n2, odd2 = _class_counts(((base | lane) ^ x) & ~0xE0, zs)
            D = _wht8([n2[k] - 2 * odd2[k] for k in range(8)])
            dtot = len(zs) - 2 * sum(odd2)
            xj = (x >> 5) & 7
            for j in range(8):
                i = base + lane + 32 * j
                if i >= N:
                    break
                assert Wj[j] == sum(-1 if popc(i & z) & 1 else 1 for z in zs)
                assert sum(odd2) + (dtot - D[j ^ xj]) // 2 == sum(popc((i ^ x) & z) & 1 for z in zs)


def test_cross_chunk_cz_sign_per_block():
    """A CZ with both bits at or above 8 signs the whole block; one with its
    low bit a below 8 flips the amplitudes with bit a set when its high bit
    is set in the block's base."""
    rng = np.random.default_rng(3)
    n = 14
    cz = [(1 << 7) | (1 << 8), (1 << 3) | (1 << 12), (1 << 9) | (1 << 13), (1 << 3) | (1 << 10)]
    for blk in rng.integers(0, 1 << (n - 8), size=20):
        base = int(blk) << 8
        bneg, lmask = 0, 0
        for m in cz:
            low = m & 255
            if low == 0:
                bneg ^= int(popc(base & m) == 2)
            elif base & m:
                lmask ^= low
        for lo in range(256):
            i = base + lo
            want = 0
            for m in cz:
                want ^= int(popc(i & m) == 2)
            assert bneg ^ (popc(lo & lmask) & 1) == want
