// Window-fused gate sweeps: device records and the per-group gate
// application shared by the adjoint plan and the batched kernel.
//
// A block of gates acts on at most WIN_MAX qubits (the window). A thread
// takes a group (the 2^w amplitudes that share their bits outside the
// window), stages it in shared memory (one column per thread, stride T, so
// a warp's accesses are consecutive), runs the block's gates on it there and
// writes it back: the state is read and written once per block instead of
// once per gate. Gates have 1 or 2 targets; rotations exp(-i a/2 P) use the
// (cos, kappa) form of rot.cuh, fixed gates their matrix with typed entries.
#pragma once

#include "common.cuh"
#include "rot.cuh"

namespace diaq {

constexpr int WIN_MAX = 5;     // window qubits
constexpr int WIN_MAXG = 32;   // gates per block
constexpr int WIN_THREADS = 128;

struct WinBlock {
    int nq;                     // window qubits
    int q[WIN_MAX];             // ascending
    int64_t off[1 << WIN_MAX];  // full-system offset of window index e (bit a -> qubit q[a])
    int first, count;           // entries of this block in the window gate list
    int np;                     // parametric gates
    int slot[WIN_MAXG];         // partial row of parametric gate j
};

struct WinGate {
    int g;       // gate index
    int b0, b1;  // window bits of targets t[0] and t[1]
    int j;       // parametric index within the block, -1 for a fixed gate
};

// A gate of the block as the sweep applies it, staged in shared memory.
template <typename R>
struct WinOp {
    int k, b0, b1, j;
    int xl, zl, ny;       // rotation generator (local masks), j >= 0
    R cs, kr, ki;         // rotation: cos(a/2) and kappa of this direction
    R mre[16], mim[16];   // fixed gate: M (forward) or M^dag (reverse)
    uint8_t ty[16];
};

__device__ __forceinline__ int ins0(int h, int b) { return ((h >> b) << (b + 1)) | (h & ((1 << b) - 1)); }

// window index of gate-local index c (bit k-1-a of c is target a)
__device__ __forceinline__ int win_row(int base, int c, int k, int b0, int b1) {
    if (k == 1) return base | ((c & 1) << b0);
    return base | (((c >> 1) & 1) << b0) | ((c & 1) << b1);
}

// Rotation rows of one gate subspace: partial (reverse) and update, with
// the generator's X mask XL fixed at compile time so every partner
// amplitude is a register.
template <typename R, int XL>
__device__ __forceinline__ void win_rot(const WinOp<R>& op, int Dk, amp_t<R>* v, amp_t<R>* w, bool rev,
                                        Acc<R>* acc) {
    using A = amp_t<R>;
    if (rev) {
        // Im conj(l_r) i^ny s_r p_{r ^ xl}
        R sr = R(0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (r < Dk) {
                const A q = mul_ipow(v[r ^ XL], op.ny);
                const R t = w[r].x * q.y - w[r].y * q.x;
                sr += (__popc((r ^ XL) & op.zl) & 1) ? -t : t;
            }
        }
        acc->add(sr);
    }
    const bool kimag = op.kr == R(0), kreal = op.ki == R(0);
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1 && !rev) break;
        A* x = pass == 0 ? v : w;
        A o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (r < Dk) {
                const bool neg = (__popc((r ^ XL) & op.zl) & 1) != 0;
                const R krr = neg ? -op.kr : op.kr, kir = neg ? -op.ki : op.ki;
                const A a = x[r], b = x[r ^ XL];
                if (kimag) {
                    o[r].x = fma(op.cs, a.x, -kir * b.y);
                    o[r].y = fma(op.cs, a.y, kir * b.x);
                } else if (kreal) {
                    o[r].x = fma(op.cs, a.x, krr * b.x);
                    o[r].y = fma(op.cs, a.y, krr * b.y);
                } else {
                    o[r].x = fma(op.cs, a.x, fma(krr, b.x, -kir * b.y));
                    o[r].y = fma(op.cs, a.y, fma(krr, b.y, kir * b.x));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < Dk) x[r] = o[r];
    }
}

// One gate on the staged column of psi (and, in the reverse sweep, lambda),
// stride T in shared memory; a rotation in the reverse sweep also adds its
// partial into acc before the update.
template <typename R>
__device__ __forceinline__ void win_apply(const WinOp<R>& op, amp_t<R>* p, amp_t<R>* l, int D, int T,
                                          Acc<R>* acc) {
    using A = amp_t<R>;
    const int k = op.k, Dk = 1 << k;
    const int lo = k == 1 ? op.b0 : min(op.b0, op.b1), hi = k == 1 ? 0 : max(op.b0, op.b1);
    const int H = D >> k;
    const bool rev = l != nullptr;
    for (int h = 0; h < H; ++h) {
        const int base = k == 1 ? ins0(h, lo) : ins0(ins0(h, lo), hi);
        int row[4];
        A v[4], w[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            row[c] = 0;
            if (c < Dk) {
                row[c] = win_row(base, c, k, op.b0, op.b1) * T;
                v[c] = p[row[c]];
                if (rev) w[c] = l[row[c]];
            }
        }
        if (op.j >= 0) {
            switch (op.xl) {
                case 0: win_rot<R, 0>(op, Dk, v, w, rev, acc); break;
                case 1: win_rot<R, 1>(op, Dk, v, w, rev, acc); break;
                case 2: win_rot<R, 2>(op, Dk, v, w, rev, acc); break;
                default: win_rot<R, 3>(op, Dk, v, w, rev, acc); break;
            }
        } else {
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1 && !rev) break;
                A* x = pass == 0 ? v : w;
                A o[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (r < Dk) {
                        A s;
                        s.x = R(0);
                        s.y = R(0);
                        bool first = true;
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            if (c < Dk) mac_typed<R>(s, first, op.ty[r * Dk + c], op.mre[r * Dk + c], op.mim[r * Dk + c], x[c]);
                        o[r] = s;
                    }
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (r < Dk) x[r] = o[r];
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c < Dk) {
                p[row[c]] = v[c];
                if (rev) l[row[c]] = w[c];
            }
        }
    }
}

}  // namespace diaq
