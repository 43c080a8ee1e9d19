// Pauli rotations exp(-i a/2 P) on k <= 2 targets, the parametric gates of
// the adjoint sweep, with their structure resolved at compile time.
//
// For a Pauli string P on the targets with local X mask xl, local Z mask zl
// and ny Y letters, P|c> = i^ny (-1)^{popc(c & zl)} |c ^ xl>, so
//   (P x)_r = i^ny s_r x_{r ^ xl},  s_r = (-1)^{popc((r ^ xl) & zl)},
// and U = cos(a/2) I - i sin(a/2) P gives
//   (U x)_r = cos x_r + kappa s_r x_{r ^ xl},  kappa = -i sin(a/2) i^ny
// (U^dag: kappa' = +i sin(a/2) i^ny). Every row has at most two terms and
// xl is a template parameter, so the partner x_{r ^ xl} is a register, not
// an indexed load; the angle enters as three numbers (cos, kappa).
#pragma once

#include "bounds.cuh"
#include "common.cuh"

namespace diaq {

// Sign flip of v when the mask is 0x80000000: an integer XOR on the word
// that holds the sign bit, so no floating-point pipe slot is spent on it.
__device__ __forceinline__ double flip_sign(double v, unsigned m) {
    return __hiloint2double(__double2hiint(v) ^ int(m), __double2loint(v));
}
__device__ __forceinline__ float flip_sign(float v, unsigned m) { return __int_as_float(__float_as_int(v) ^ int(m)); }

struct RotShape {
    int st[2];          // targets ascending
    int64_t off[4];     // full-system offset of local index c
    int zl;             // local Z mask
    int ny;             // number of Y letters mod 4
};

// z * i^q
template <typename A>
__device__ __forceinline__ A mul_ipow(A z, int q) {
    A w;
    switch (q & 3) {
        case 0: w = z; break;
        case 1: w.x = -z.y; w.y = z.x; break;
        case 2: w.x = -z.x; w.y = -z.y; break;
        default: w.x = z.y; w.y = -z.x; break;
    }
    return w;
}

// One rotation over a grid-stride share of the groups, in place on psi
// (and lam). cs = cos(a/2); (kr, ki) = kappa for the direction applied.
// With lam (reverse step), returns this thread's share of
// Im <lam|P|psi> taken before the update; otherwise 0. Each thread takes U
// groups per iteration, all loads issued before any arithmetic.
// KT fixes kappa's form when the caller knows the parity of the Y count
// (kappa = -i sin(a/2) i^ny): 1 imaginary (even ny), 2 real (odd ny), 0 read
// from the values. With KT != 0 the partial's i^ny is a cross (even) or a
// dot (odd) product, its sign applied once to the sum: the same values.
template <typename R, int K, int XL, int U, int KT = 0>
__device__ __noinline__ double rot_groups_u(amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam, int n,
                                            const RotShape& sh, R cs, R kr, R ki, int64_t tid, int64_t nthreads) {
    constexpr int D = 1 << K;
    using A = amp_t<R>;
    int st[K];
    int64_t off[D];
#pragma unroll
    for (int a = 0; a < K; ++a) st[a] = sh.st[a];
#pragma unroll
    for (int c = 0; c < D; ++c) off[c] = sh.off[c];
    // per-row sign s_r folded into kappa once, so the loop spends no
    // arithmetic on it; gradient terms are summed per row and signed at the end
    R krr[D], kir[D];
    bool sneg[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
        sneg[r] = (__popc((r ^ XL) & sh.zl) & 1) != 0;
        krr[r] = sneg[r] ? -kr : kr;
        kir[r] = sneg[r] ? -ki : ki;
    }
    const bool kreal = ki == R(0), kimag = kr == R(0);
    const int ny = sh.ny;
    Acc<R> accr[D];
    const int64_t G = int64_t(1) << (n - K);
    for (int64_t g0 = tid; g0 < G; g0 += int64_t(U) * nthreads) {
        int64_t b[U];
        A p[U][D], l[U][D];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t gi = g0 + int64_t(u) * nthreads;
            b[u] = gi < G ? insert_zeros<K>(gi, st) : int64_t(-1);
            if (b[u] >= 0 && !DIAQ_BOUNDS_OK(b[u] + off[D - 1], int64_t(1) << n, BS_ROTATION)) b[u] = -1;
            if (b[u] >= 0) {
#pragma unroll
                for (int c = 0; c < D; ++c) p[u][c] = psi[b[u] + off[c]];
                if (lam) {
#pragma unroll
                    for (int c = 0; c < D; ++c) l[u][c] = lam[b[u] + off[c]];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b[u] < 0) continue;
            if (lam) {
                // Im conj(l_r) i^ny p_{r ^ XL}, per row (signed after the loop)
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    if (KT == 1) {
                        const A q = p[u][r ^ XL];
                        accr[r].add_cross(l[u][r].x, q.y, l[u][r].y, q.x);
                    } else if (KT == 2) {
                        const A q = p[u][r ^ XL];
                        accr[r].add_dot(l[u][r].x, q.x, l[u][r].y, q.y);
                    } else {
                        const A q = mul_ipow(p[u][r ^ XL], ny);
                        accr[r].add_cross(l[u][r].x, q.y, l[u][r].y, q.x);
                    }
                }
            }
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1 && !lam) break;
                const A* v = pass == 0 ? p[u] : l[u];
                A* dst = pass == 0 ? psi : lam;
                A o[D];
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    const A x = v[r], y = v[r ^ XL];
                    A w;
                    if (KT == 1 || (KT == 0 && kimag)) {  // kappa_r = i ki_r: w = cs x + i ki_r y
                        w.x = fma(cs, x.x, -kir[r] * y.y);
                        w.y = fma(cs, x.y, kir[r] * y.x);
                    } else if (KT == 2 || (KT == 0 && kreal)) {  // kappa_r = kr_r
                        w.x = fma(cs, x.x, krr[r] * y.x);
                        w.y = fma(cs, x.y, krr[r] * y.y);
                    } else {
                        w.x = fma(cs, x.x, fma(krr[r], y.x, -kir[r] * y.y));
                        w.y = fma(cs, x.y, fma(krr[r], y.y, kir[r] * y.x));
                    }
                    o[r] = w;
                }
#pragma unroll
                for (int r = 0; r < D; ++r) dst[b[u] + off[r]] = o[r];
            }
        }
    }
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < D; ++r) acc += sneg[r] ? -accr[r].value() : accr[r].value();
    if (KT != 0 && (ny & 2)) acc = -acc;  // i^ny = -1 or -i
    return acc;
}

// Scaled form of a rotation: U = sigma V, applied as V alone, with sigma
// the larger in magnitude of cos(a/2) and kappa's non-zero part (kappa is
// real for an odd Y count, imaginary for an even one), so |sigma| >= 1/sqrt(2)
// and V's other coefficient is at most 1 in magnitude. Row r of V x is
//   M1 = 0 (sigma = cos):   x_r + tau s_r (i)x_{r ^ xl},   tau = kappa / cos
//   M1 = 1 (sigma = kappa): c x_r + s_r (i)x_{r ^ xl},     c = cos / kappa
// (the factor i only when kappa is imaginary), one fused multiply-add per
// real component instead of a multiply and a fused multiply-add: the
// unit coefficient's sign is an integer flip. The caller tracks the
// product of the 1/sigma factors (the stored state is the true one times
// it) and rescales energies and gradient terms. The partial
// Im <lam|P|psi> is taken before the update, as in rot_groups_u.
template <typename R, int K, int XL, int U, int KT, int M1>
__device__ __noinline__ double rot_groups_s(amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam, int n,
                                            const RotShape& sh, R cf, int64_t tid, int64_t nthreads) {
    static_assert(KT == 1 || KT == 2, "kappa's form must be known");
    constexpr int D = 1 << K;
    using A = amp_t<R>;
    int st[K];
    int64_t off[D];
#pragma unroll
    for (int a = 0; a < K; ++a) st[a] = sh.st[a];
#pragma unroll
    for (int c = 0; c < D; ++c) off[c] = sh.off[c];
    // per row: the coefficient of the partner term (M1 = 0) or the sign
    // mask of the unit partner coefficient (M1 = 1), for each component
    R tx[D], ty[D];
    unsigned mx[D], my[D];
    bool sneg[D];
#pragma unroll
    for (int r = 0; r < D; ++r) {
        sneg[r] = (__popc((r ^ XL) & sh.zl) & 1) != 0;
        const R t = sneg[r] ? -cf : cf;
        // kappa real: w = x + t y; kappa imaginary: w.x = x.x - t y.y, w.y = x.y + t y.x
        tx[r] = KT == 2 ? t : -t;
        ty[r] = t;
        const unsigned neg = sneg[r] ? 0x80000000u : 0u;
        mx[r] = KT == 2 ? neg : (neg ^ 0x80000000u);
        my[r] = neg;
    }
    const int ny = sh.ny;
    Acc<R> accr[D];
    const int64_t G = int64_t(1) << (n - K);
    for (int64_t g0 = tid; g0 < G; g0 += int64_t(U) * nthreads) {
        int64_t b[U];
        A p[U][D], l[U][D];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t gi = g0 + int64_t(u) * nthreads;
            b[u] = gi < G ? insert_zeros<K>(gi, st) : int64_t(-1);
            if (b[u] >= 0 && !DIAQ_BOUNDS_OK(b[u] + off[D - 1], int64_t(1) << n, BS_ROTATION)) b[u] = -1;
            if (b[u] >= 0) {
#pragma unroll
                for (int c = 0; c < D; ++c) p[u][c] = psi[b[u] + off[c]];
                if (lam) {
#pragma unroll
                    for (int c = 0; c < D; ++c) l[u][c] = lam[b[u] + off[c]];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b[u] < 0) continue;
            if (lam) {
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    const A q = p[u][r ^ XL];
                    if (KT == 1) accr[r].add_cross(l[u][r].x, q.y, l[u][r].y, q.x);
                    else accr[r].add_dot(l[u][r].x, q.x, l[u][r].y, q.y);
                }
            }
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1 && !lam) break;
                const A* v = pass == 0 ? p[u] : l[u];
                A* dst = pass == 0 ? psi : lam;
                A o[D];
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    const A x = v[r], y = v[r ^ XL];
                    // the partner component feeding each output component
                    const R yx = KT == 2 ? y.x : y.y;
                    const R yy = KT == 2 ? y.y : y.x;
                    A w;
                    if (M1 == 0) {
                        w.x = fma(tx[r], yx, x.x);
                        w.y = fma(ty[r], yy, x.y);
                    } else {
                        w.x = fma(cf, x.x, flip_sign(yx, mx[r]));
                        w.y = fma(cf, x.y, flip_sign(yy, my[r]));
                    }
                    o[r] = w;
                }
#pragma unroll
                for (int r = 0; r < D; ++r) dst[b[u] + off[r]] = o[r];
            }
        }
    }
    double acc = 0.0;
#pragma unroll
    for (int r = 0; r < D; ++r) acc += sneg[r] ? -accr[r].value() : accr[r].value();
    if (ny & 2) acc = -acc;  // i^ny = -1 or -i
    return acc;
}

// Scaled rotation with the form chosen per gate (m1 is uniform).
template <typename R, int K, int XL, int U, int KT>
__device__ __forceinline__ double rot_groups_sc(amp_t<R>* psi, amp_t<R>* lam, int n, const RotShape& sh, bool m1,
                                                R cf, int64_t tid, int64_t nthreads) {
    if (m1) return rot_groups_s<R, K, XL, U, KT, 1>(psi, lam, n, sh, cf, tid, nthreads);
    return rot_groups_s<R, K, XL, U, KT, 0>(psi, lam, n, sh, cf, tid, nthreads);
}

// One-qubit rotation about X (G = 1) or Y (G = 2) on a pair of amplitudes
// (x0: target bit 0, x1: target bit 1), for the fused pair kernels. With
// sc = false, (c0, c1) = (cos(a/2), kappa's non-zero part): X rows are
// cos x_r + kappa_i i x_{1-r} (kappa imaginary), Y rows cos x_r + s_r kappa
// x_{1-r} with s_0 = -1, s_1 = +1 (kappa real). With sc = true the scaled
// form of rot_groups_s, c0 = V's coefficient and m1 its form: m1 = 0 gives
// x_r + c0 s_r (i)x_{1-r}, m1 = 1 gives c0 x_r + s_r (i)x_{1-r}. Either way
// each real component costs one fused multiply-add (scaled) or a multiply
// and a fused multiply-add (unscaled); in the scaled form the operands are
// selected on the uniform m1 and a unit coefficient's sign is an integer
// flip, so no FP64 instruction is issued twice.
template <typename R, int G, bool SC>
struct Rot1 {
    R c0, c1;
    bool m1;

    __device__ __forceinline__ amp_t<R> row(amp_t<R> x, amp_t<R> y, int r) const {
        amp_t<R> w;
        // partner component feeding each output component and its sign s
        // (X: w.x gets -y.y, w.y gets +y.x; Y: both get s_r y, s_0 = -1)
        const R px = G == 1 ? y.y : y.x, py = G == 1 ? y.x : y.y;
        const bool nx = G == 1 ? true : (r == 0), ny_ = G == 1 ? false : (r == 0);
        if (!SC) {
            w.x = fma(c0, x.x, (nx ? -c1 : c1) * px);
            w.y = fma(c0, x.y, (ny_ ? -c1 : c1) * py);
        } else {
            const R tx = nx ? -c0 : c0, ty = ny_ ? -c0 : c0;
            const R fx = flip_sign(px, nx ? 0x80000000u : 0u), fy = flip_sign(py, ny_ ? 0x80000000u : 0u);
            w.x = fma(m1 ? c0 : tx, m1 ? x.x : px, m1 ? fx : x.x);
            w.y = fma(m1 ? c0 : ty, m1 ? x.y : py, m1 ? fy : x.y);
        }
        return w;
    }
    __device__ __forceinline__ void apply(amp_t<R>& x0, amp_t<R>& x1) const {
        const amp_t<R> w0 = row(x0, x1, 0), w1 = row(x1, x0, 1);
        x0 = w0;
        x1 = w1;
    }
    // Im <l|P|p> over the pair, into the positive and negative sums: X gives
    // Im conj(l_r) p_{1-r}; Y gives s_r Re conj(l_r) p_{1-r}
    __device__ __forceinline__ void partial(const amp_t<R>& l0, const amp_t<R>& l1, const amp_t<R>& p0,
                                            const amp_t<R>& p1, Acc<R>& pos, Acc<R>& neg) const {
        if (G == 1) {
            pos.add_cross(l0.x, p1.y, l0.y, p1.x);
            pos.add_cross(l1.x, p0.y, l1.y, p0.x);
        } else {
            neg.add_dot(l0.x, p1.x, l0.y, p1.y);
            pos.add_dot(l1.x, p0.x, l1.y, p0.y);
        }
    }
};

// Two one-qubit X/Y rotations A (on qubit qa) then B (on qb != qa), fused:
// each thread takes groups of the 4 amplitudes that share every other bit
// and applies A along qa and B along qb in registers (forward), or - with
// lam - takes B's partial, undoes B on psi and lam, takes A's partial and
// undoes A (reverse), so a pair costs one read and one write of the states
// instead of two. Partials go to pa and pb (this thread's shares).
template <typename R, int GA, int GB, bool SC, int U>
__device__ __noinline__ void rot2_groups(amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam, int n, int qa,
                                         int qb, const Rot1<R, GA, SC> A, const Rot1<R, GB, SC> B, int64_t tid,
                                         int64_t nthreads, double* pa, double* pb) {
    using Am = amp_t<R>;
    int st[2] = {qa < qb ? qa : qb, qa < qb ? qb : qa};
    const int64_t oa = int64_t(1) << qa, ob = int64_t(1) << qb;
    const int64_t off[4] = {0, oa, ob, oa + ob};  // bit 0 of the index: qa, bit 1: qb
    Acc<R> a_pos, a_neg, b_pos, b_neg;
    const int64_t G = int64_t(1) << (n - 2);
    for (int64_t g0 = tid; g0 < G; g0 += int64_t(U) * nthreads) {
        int64_t b[U];
        Am p[U][4], l[U][4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t gi = g0 + int64_t(u) * nthreads;
            b[u] = gi < G ? insert_zeros<2>(gi, st) : int64_t(-1);
            if (b[u] >= 0 && !DIAQ_BOUNDS_OK(b[u] + off[3], int64_t(1) << n, BS_ROTATION)) b[u] = -1;
            if (b[u] >= 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c) p[u][c] = psi[b[u] + off[c]];
                if (lam) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) l[u][c] = lam[b[u] + off[c]];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b[u] < 0) continue;
            if (!lam) {
                A.apply(p[u][0], p[u][1]);
                A.apply(p[u][2], p[u][3]);
                B.apply(p[u][0], p[u][2]);
                B.apply(p[u][1], p[u][3]);
            } else {
                B.partial(l[u][0], l[u][2], p[u][0], p[u][2], b_pos, b_neg);
                B.partial(l[u][1], l[u][3], p[u][1], p[u][3], b_pos, b_neg);
                B.apply(p[u][0], p[u][2]);
                B.apply(p[u][1], p[u][3]);
                B.apply(l[u][0], l[u][2]);
                B.apply(l[u][1], l[u][3]);
                A.partial(l[u][0], l[u][1], p[u][0], p[u][1], a_pos, a_neg);
                A.partial(l[u][2], l[u][3], p[u][2], p[u][3], a_pos, a_neg);
                A.apply(p[u][0], p[u][1]);
                A.apply(p[u][2], p[u][3]);
                A.apply(l[u][0], l[u][1]);
                A.apply(l[u][2], l[u][3]);
#pragma unroll
                for (int c = 0; c < 4; ++c) lam[b[u] + off[c]] = l[u][c];
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) psi[b[u] + off[c]] = p[u][c];
        }
    }
    *pa = a_pos.value() - a_neg.value();
    *pb = b_pos.value() - b_neg.value();
}

// One-qubit rotation about X or Y with the generator's structure taken at
// run time, for the complex64 rotation tiles (FP32 work is cheap there, the
// passes over the states are not): rows w_r = a x_r + b_r x_{1-r} with
// a = cos(a/2) and b_r = kappa s_r, and the gradient term
// sum_r Im conj(l_r) pi_r p_{1-r}, pi_r = i^ny s_r (+-1 for X, +-i for Y).
template <typename R>
struct RotG {
    R a;
    R br[2], bi[2];
    R pr[2], pi[2];

    __device__ __forceinline__ void apply(amp_t<R>& x0, amp_t<R>& x1) const {
        amp_t<R> w0, w1;
        w0.x = fma(a, x0.x, fma(br[0], x1.x, -bi[0] * x1.y));
        w0.y = fma(a, x0.y, fma(br[0], x1.y, bi[0] * x1.x));
        w1.x = fma(a, x1.x, fma(br[1], x0.x, -bi[1] * x0.y));
        w1.y = fma(a, x1.y, fma(br[1], x0.y, bi[1] * x0.x));
        x0 = w0;
        x1 = w1;
    }
    __device__ __forceinline__ void partial(const amp_t<R>& l0, const amp_t<R>& l1, const amp_t<R>& p0,
                                            const amp_t<R>& p1, Acc<R>& acc) const {
        // t_r = pi_r p_{1-r}; Im conj(l_r) t_r = l.x t.y - l.y t.x
        const R t0x = pr[0] * p1.x - pi[0] * p1.y, t0y = pr[0] * p1.y + pi[0] * p1.x;
        const R t1x = pr[1] * p0.x - pi[1] * p0.y, t1y = pr[1] * p0.y + pi[1] * p0.x;
        acc.add_cross(l0.x, t0y, l0.y, t0x);
        acc.add_cross(l1.x, t1y, l1.y, t1x);
    }
};

// A tile of NQ one-qubit X/Y rotations on distinct qubits q[0..NQ-1],
// applied in that order (forward) or undone in reverse order with each
// rotation's partial taken before it is undone (reverse, lam != NULL), on
// groups of 2^NQ amplitudes held in registers: the states are read and
// written once per tile. Bit j of a group's local index is qubit q[j].
template <typename R, int NQ>
__device__ __forceinline__ void rotq_groups(amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam, int n,
                                         const int* q, const RotG<R>* rot, int64_t tid, int64_t nthreads,
                                         double* part) {
    constexpr int D = 1 << NQ;
    using Am = amp_t<R>;
    int st[NQ];
    int64_t o[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        st[j] = q[j];
        o[j] = int64_t(1) << q[j];
    }
    // ascending targets for insert_zeros (a few swaps of a tiny array)
#pragma unroll
    for (int x = 0; x < NQ; ++x)
#pragma unroll
        for (int y = 0; y + 1 < NQ - x; ++y)
            if (st[y] > st[y + 1]) {
                const int t = st[y];
                st[y] = st[y + 1];
                st[y + 1] = t;
            }
    Acc<R> acc[NQ];
    const int64_t G = int64_t(1) << (n - NQ);
    for (int64_t g = tid; g < G; g += nthreads) {
        const int64_t b = insert_zeros<NQ>(g, st);
        int64_t last = b;
#pragma unroll
        for (int j = 0; j < NQ; ++j) last += o[j];
        if (!DIAQ_BOUNDS_OK(last, int64_t(1) << n, BS_ROTATION)) continue;
        Am p[D], l[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            int64_t off = 0;
#pragma unroll
            for (int j = 0; j < NQ; ++j)
                if ((c >> j) & 1) off += o[j];
            p[c] = psi[b + off];
            if (lam) l[c] = lam[b + off];
        }
        if (!lam) {
#pragma unroll
            for (int j = 0; j < NQ; ++j)
#pragma unroll
                for (int c = 0; c < D; ++c)
                    if (!((c >> j) & 1)) rot[j].apply(p[c], p[c | (1 << j)]);
        } else {
#pragma unroll
            for (int j = NQ - 1; j >= 0; --j) {
#pragma unroll
                for (int c = 0; c < D; ++c)
                    if (!((c >> j) & 1)) rot[j].partial(l[c], l[c | (1 << j)], p[c], p[c | (1 << j)], acc[j]);
#pragma unroll
                for (int c = 0; c < D; ++c)
                    if (!((c >> j) & 1)) {
                        rot[j].apply(p[c], p[c | (1 << j)]);
                        rot[j].apply(l[c], l[c | (1 << j)]);
                    }
            }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            int64_t off = 0;
#pragma unroll
            for (int j = 0; j < NQ; ++j)
                if ((c >> j) & 1) off += o[j];
            psi[b + off] = p[c];
            if (lam) lam[b + off] = l[c];
        }
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) part[j] = acc[j].value();
}

// The scaled form's coefficients from (cos, kappa) of one direction: the
// form (m1), V's coefficient cf and sigma (U = sigma V).
__host__ __device__ __forceinline__ void rot_scaled_coefs(double cs, double kr, double ki, int ny, int* m1, double* cf,
                                                          double* sigma) {
    const double kv = (ny & 1) ? kr : ki;  // kappa's non-zero part
    if (fabs(cs) >= fabs(kv)) {
        *m1 = 0;
        *cf = kv / cs;
        *sigma = cs;
    } else {
        *m1 = 1;
        *cf = cs / kv;
        *sigma = kv;
    }
}

// Groups per iteration: enough 16-byte loads in flight without spilling.
template <typename R, int K, int XL, int KT = 0>
__device__ __forceinline__ double rot_groups(amp_t<R>* psi, amp_t<R>* lam, int n, const RotShape& sh, R cs, R kr,
                                             R ki, int64_t tid, int64_t nthreads) {
    constexpr int U = K == 1 ? 4 : (sizeof(R) == 4 ? 2 : 1);
    if (lam) return rot_groups_u<R, K, XL, U, KT>(psi, lam, n, sh, cs, kr, ki, tid, nthreads);
    return rot_groups_u<R, K, XL, (K == 1 ? 4 : 2), KT>(psi, lam, n, sh, cs, kr, ki, tid, nthreads);
}

// Dispatch on (k, xl, parity of the Y count) for the persistent batch
// kernel: one group per iteration, so its register budget (shared with
// every other gate path of that kernel) is not exceeded.
template <typename R, int KT>
__device__ __forceinline__ double rot_dispatch_kt(int k, int xl, amp_t<R>* psi, amp_t<R>* lam, int n,
                                                  const RotShape& sh, R cs, R kr, R ki, int64_t tid, int64_t nth) {
    if (k == 1) {
        if (xl == 0) return rot_groups_u<R, 1, 0, 1, KT>(psi, lam, n, sh, cs, kr, ki, tid, nth);
        return rot_groups_u<R, 1, 1, 1, KT>(psi, lam, n, sh, cs, kr, ki, tid, nth);
    }
    switch (xl) {
        case 0: return rot_groups_u<R, 2, 0, 1, KT>(psi, lam, n, sh, cs, kr, ki, tid, nth);
        case 1: return rot_groups_u<R, 2, 1, 1, KT>(psi, lam, n, sh, cs, kr, ki, tid, nth);
        case 2: return rot_groups_u<R, 2, 2, 1, KT>(psi, lam, n, sh, cs, kr, ki, tid, nth);
        default: return rot_groups_u<R, 2, 3, 1, KT>(psi, lam, n, sh, cs, kr, ki, tid, nth);
    }
}

// The scaled form (rot_groups_s) for the persistent batch kernel, one group
// per iteration; m1 and cf as returned by rot_scaled_coefs.
template <typename R, int KT>
__device__ __forceinline__ double rot_dispatch_s_kt(int k, int xl, amp_t<R>* psi, amp_t<R>* lam, int n,
                                                    const RotShape& sh, bool m1, R cf, int64_t tid, int64_t nth) {
    if (k == 1) {
        if (xl == 0) return rot_groups_sc<R, 1, 0, 1, KT>(psi, lam, n, sh, m1, cf, tid, nth);
        return rot_groups_sc<R, 1, 1, 1, KT>(psi, lam, n, sh, m1, cf, tid, nth);
    }
    switch (xl) {
        case 0: return rot_groups_sc<R, 2, 0, 1, KT>(psi, lam, n, sh, m1, cf, tid, nth);
        case 1: return rot_groups_sc<R, 2, 1, 1, KT>(psi, lam, n, sh, m1, cf, tid, nth);
        case 2: return rot_groups_sc<R, 2, 2, 1, KT>(psi, lam, n, sh, m1, cf, tid, nth);
        default: return rot_groups_sc<R, 2, 3, 1, KT>(psi, lam, n, sh, m1, cf, tid, nth);
    }
}

template <typename R>
__device__ __forceinline__ double rot_dispatch_s(int k, int xl, amp_t<R>* psi, amp_t<R>* lam, int n,
                                                 const RotShape& sh, bool m1, R cf, int64_t tid, int64_t nth) {
    if (sh.ny & 1) return rot_dispatch_s_kt<R, 2>(k, xl, psi, lam, n, sh, m1, cf, tid, nth);
    return rot_dispatch_s_kt<R, 1>(k, xl, psi, lam, n, sh, m1, cf, tid, nth);
}

template <typename R>
__device__ __forceinline__ double rot_dispatch(int k, int xl, amp_t<R>* psi, amp_t<R>* lam, int n,
                                               const RotShape& sh, R cs, R kr, R ki, int64_t tid, int64_t nth) {
    if (sh.ny & 1) return rot_dispatch_kt<R, 2>(k, xl, psi, lam, n, sh, cs, kr, ki, tid, nth);
    return rot_dispatch_kt<R, 1>(k, xl, psi, lam, n, sh, cs, kr, ki, tid, nth);
}

}  // namespace diaq
