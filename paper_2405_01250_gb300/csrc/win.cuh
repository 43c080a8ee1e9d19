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
// Lanes per group of the four-lane kernels: a group's 2^w amplitudes are
// shared by WIN_LANES threads of one warp, which split its subspaces gate by
// gate (a __syncwarp between gates), so a block of 128 threads works on 32
// groups at once and a thread's chain of dependent steps per gate is
// WIN_LANES times shorter.
constexpr int WIN_LANES = 4;

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

// One rotation exp(-i a/2 P) over every subspace of the window, with the
// gate's shape fixed at compile time: K targets, the generator's local X
// mask XL, NYP = parity of its Y count (kappa = -i sin(a/2) i^ny is then
// imaginary for even ny and real for odd ny, and i^ny turns the partial's
// Im into a Re), and REV (reverse sweep: partial Im <l|P|p> before U^dag,
// and the same update of l). The per-row signs s_r are folded into kappa
// once. Rows of a subspace are registers; subspaces of one column are
// disjoint, so iterations do not depend on each other.
template <typename R, int K, int XL, int NYP, bool REV, int UNR>
__device__ __noinline__ void win_rot_loop(amp_t<R>* __restrict__ p, amp_t<R>* __restrict__ l, int D, int T,
                                          int h0, int hs, int b0, int b1, int zl, bool negp, R cs, R kr, R ki,
                                          Acc<R>* acc) {
    using A = amp_t<R>;
    constexpr int Dk = 1 << K;
    const int lo = K == 1 ? b0 : min(b0, b1), hi = K == 1 ? 0 : max(b0, b1);
    int ro[Dk];
#pragma unroll
    for (int c = 0; c < Dk; ++c)
        ro[c] = (K == 1 ? ((c & 1) << b0) : ((((c >> 1) & 1) << b0) | ((c & 1) << b1))) * T;
    bool sneg[Dk];
    R kk[Dk];
#pragma unroll
    for (int r = 0; r < Dk; ++r) {
        sneg[r] = (__popc((r ^ XL) & zl) & 1) != 0;
        const R kv = NYP ? kr : ki;  // the non-zero part of kappa
        kk[r] = sneg[r] ? -kv : kv;
    }
    Acc<R> loc;
    const int H = D >> K;
#pragma unroll UNR
    for (int h = h0; h < H; h += hs) {
        const int base = (K == 1 ? ins0(h, lo) : ins0(ins0(h, lo), hi)) * T;
        A v[Dk], w[Dk];
#pragma unroll
        for (int c = 0; c < Dk; ++c) {
            v[c] = p[base + ro[c]];
            if (REV) w[c] = l[base + ro[c]];
        }
        if (REV) {
            // Im conj(w_r) i^ny s_r v_{r^XL}: a cross product for even ny,
            // a dot product for odd ny; the sign of i^ny (ny & 2) is applied
            // to the sum at the end
            R sr = R(0);
#pragma unroll
            for (int r = 0; r < Dk; ++r) {
                const A q = v[r ^ XL];
                const R t = NYP ? fma(w[r].x, q.x, w[r].y * q.y) : fma(w[r].x, q.y, -w[r].y * q.x);
                sr += sneg[r] ? -t : t;
            }
            loc.add(sr);
        }
#pragma unroll
        for (int pass = 0; pass < (REV ? 2 : 1); ++pass) {
            A* x = pass == 0 ? v : w;
            A o[Dk];
#pragma unroll
            for (int r = 0; r < Dk; ++r) {
                const A a = x[r], b = x[r ^ XL];
                if (NYP) {  // kappa real
                    o[r].x = fma(cs, a.x, kk[r] * b.x);
                    o[r].y = fma(cs, a.y, kk[r] * b.y);
                } else {    // kappa = i kk
                    o[r].x = fma(cs, a.x, -kk[r] * b.y);
                    o[r].y = fma(cs, a.y, kk[r] * b.x);
                }
            }
#pragma unroll
            for (int r = 0; r < Dk; ++r) x[r] = o[r];
        }
#pragma unroll
        for (int c = 0; c < Dk; ++c) {
            p[base + ro[c]] = v[c];
            if (REV) l[base + ro[c]] = w[c];
        }
    }
    if (REV && acc) {
        const double v = loc.value();
        acc->add(R(negp ? -v : v));
    }
}

// One fixed gate (its matrix, or M^dag in the reverse sweep, staged in op)
// over every subspace of the window; REV also updates l.
template <typename R, int K, bool REV, int UNR>
__device__ __noinline__ void win_fixed_loop(const WinOp<R>& op, amp_t<R>* __restrict__ p, amp_t<R>* __restrict__ l,
                                            int D, int T, int h0, int hs) {
    using A = amp_t<R>;
    constexpr int Dk = 1 << K;
    const int b0 = op.b0, b1 = op.b1;
    const int lo = K == 1 ? b0 : min(b0, b1), hi = K == 1 ? 0 : max(b0, b1);
    int ro[Dk];
#pragma unroll
    for (int c = 0; c < Dk; ++c)
        ro[c] = (K == 1 ? ((c & 1) << b0) : ((((c >> 1) & 1) << b0) | ((c & 1) << b1))) * T;
    R mr[Dk * Dk], mi[Dk * Dk];
    uint8_t ty[Dk * Dk];
#pragma unroll
    for (int e = 0; e < Dk * Dk; ++e) {
        mr[e] = op.mre[e];
        mi[e] = op.mim[e];
        ty[e] = op.ty[e];
    }
    const int H = D >> K;
#pragma unroll UNR
    for (int h = h0; h < H; h += hs) {
        const int base = (K == 1 ? ins0(h, lo) : ins0(ins0(h, lo), hi)) * T;
#pragma unroll
        for (int pass = 0; pass < (REV ? 2 : 1); ++pass) {
            A* col = pass == 0 ? p : l;
            A x[Dk], o[Dk];
#pragma unroll
            for (int c = 0; c < Dk; ++c) x[c] = col[base + ro[c]];
#pragma unroll
            for (int r = 0; r < Dk; ++r) {
                A s;
                s.x = R(0);
                s.y = R(0);
                bool first = true;
#pragma unroll
                for (int c = 0; c < Dk; ++c) mac_typed<R>(s, first, ty[r * Dk + c], mr[r * Dk + c], mi[r * Dk + c], x[c]);
                o[r] = s;
            }
#pragma unroll
            for (int c = 0; c < Dk; ++c) col[base + ro[c]] = o[c];
        }
    }
}

template <typename R, int K, bool REV, int UNR>
__device__ __forceinline__ void win_rot_dispatch(const WinOp<R>& op, amp_t<R>* p, amp_t<R>* l, int D, int T,
                                                 int h0, int hs, Acc<R>* acc) {
    const int nyp = op.ny & 1;
    const bool negp = (op.ny & 2) != 0;
    const R cs = op.cs, kr = op.kr, ki = op.ki;
    const int b0 = op.b0, b1 = op.b1, zl = op.zl;
#define DIAQ_WROT(XL, NYP) win_rot_loop<R, K, XL, NYP, REV, UNR>(p, l, D, T, h0, hs, b0, b1, zl, negp, cs, kr, ki, acc)
    if (K == 1) {
        if (op.xl == 0) {
            if (nyp) DIAQ_WROT(0, 1); else DIAQ_WROT(0, 0);
        } else {
            if (nyp) DIAQ_WROT(1, 1); else DIAQ_WROT(1, 0);
        }
    } else {
        switch (op.xl) {
            case 0: if (nyp) DIAQ_WROT(0, 1); else DIAQ_WROT(0, 0); break;
            case 1: if (nyp) DIAQ_WROT(1, 1); else DIAQ_WROT(1, 0); break;
            case 2: if (nyp) DIAQ_WROT(2, 1); else DIAQ_WROT(2, 0); break;
            default: if (nyp) DIAQ_WROT(3, 1); else DIAQ_WROT(3, 0); break;
        }
    }
#undef DIAQ_WROT
}

// One gate of a block on the staged amplitudes p (and, in the reverse
// sweep, l): window row r of the group is p[r * T]; this thread takes the
// gate's subspaces h0, h0 + hs, ... (a group may be shared by hs threads),
// UNR of them per loop trip. A rotation in the reverse sweep also adds its
// partial into acc (if acc is not NULL). The gate's kind is resolved here,
// once, ahead of the loop.
template <typename R, int UNR = 2>
__device__ __forceinline__ void win_apply(const WinOp<R>& op, amp_t<R>* p, amp_t<R>* l, int D, int T,
                                          Acc<R>* acc, int h0 = 0, int hs = 1) {
    if (op.j >= 0) {
        if (l) {
            if (op.k == 1) win_rot_dispatch<R, 1, true, UNR>(op, p, l, D, T, h0, hs, acc);
            else win_rot_dispatch<R, 2, true, UNR>(op, p, l, D, T, h0, hs, acc);
        } else {
            if (op.k == 1) win_rot_dispatch<R, 1, false, UNR>(op, p, l, D, T, h0, hs, acc);
            else win_rot_dispatch<R, 2, false, UNR>(op, p, l, D, T, h0, hs, acc);
        }
    } else if (l) {
        if (op.k == 1) win_fixed_loop<R, 1, true, UNR>(op, p, l, D, T, h0, hs);
        else win_fixed_loop<R, 2, true, UNR>(op, p, l, D, T, h0, hs);
    } else {
        if (op.k == 1) win_fixed_loop<R, 1, false, UNR>(op, p, l, D, T, h0, hs);
        else win_fixed_loop<R, 2, false, UNR>(op, p, l, D, T, h0, hs);
    }
}

}  // namespace diaq
