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
