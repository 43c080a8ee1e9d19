// Gate-apply kernels of libdiaq_gb300: the DiaQ SpMV y[i] = sum_d A_d(i) x[i+d]
// of arXiv 2405.01250, in its two variants.
//
//  * On the fly (Algorithm 3, generalised to any target placement): the
//    full-system diagonals of I_above (x) M (x) I_below are never formed.
//    Row i of the operator has its non-zeros at columns i + d(r, c), where
//    r is i's local index on the targets, c runs over the 2^k local columns
//    and d(r, c) = sum_a (c_a - r_a) 2^{t_a} is the diagonal M[r][c] lies
//    on. The 2^k rows that share their non-target bits (a "group") read the
//    same 2^k amplitudes, so each thread loads a group once into registers
//    and produces all of its rows: every amplitude is read once and written
//    once, with 16-byte coalesced accesses across the warp.
//  * Stored (Algorithm 2): the diagonals live in device memory, one array of
//    N - |d| values per index d; each output row sums over the diagonals,
//    reading A_d(i) and, where it is non-zero, x[i + d]. Rows are visited
//    in an order that keeps whole groups inside one block when the op has
//    gate structure, so the shifted reads of x hit cache.
//
// Both write y exactly once per row (no atomics) and sum the terms of a row
// in a fixed order.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "bounds.cuh"
#include "common.cuh"
#include "internal.h"

DIAQ_BOUNDS_TU(apply)

namespace diaq {

// ---------------------------------------------------------------------------
// On-the-fly apply, k <= 3: matrix, entry types and offsets in kernel params.
// ---------------------------------------------------------------------------
template <typename R, int K>
struct SmallGateArgs {
    int64_t g_base;              // first group of the launch
    int64_t n_groups;            // one past the last group
    int64_t N;                   // amplitudes of the state
    int st[K];                   // targets, ascending
    int64_t off[1 << K];         // full-system offset of local index c
    R re[1 << (2 * K)];
    R im[1 << (2 * K)];
    uint8_t type[1 << (2 * K)];
    // k = 1 only: both rows start with the same non-zero entry in column 0
    // (a Hadamard, any [[a, b], [a, d]]), so the product m00 x0 that opens
    // both rows' sums is formed once. Same roundings, fewer FP64 instructions.
    // 1: every entry real and non-zero (the butterfly, written out with no
    // entry-type dispatch); 2: any other such matrix.
    int share_col0;
    // k = 1 only: every entry general complex (a Haar U(2)): the rows are
    // written out as fused multiply-adds in the order of the typed path,
    // with no entry-type dispatch.
    int dense1;
    // Other patterns written out the same way (same operations, same order
    // as the typed path): 1 every entry real and non-zero (RY), 2 real
    // non-zero diagonal with imaginary non-zero off-diagonal (RX),
    // 3 diagonal, every diagonal entry general complex (RZ; RZZ for k = 2).
    int pattern;
    // k = 1 only, scaled form (launch_gate_scaled1): each output component
    // is one fused multiply-add, fma(sc_a, in[sc_mul], +-in[sc_add]), with
    // in = (own.re, own.im, partner.re, partner.im) of the row and the sign
    // an integer flip (sc_neg); the caller tracks the dropped factor.
    int scaled1;
    R sc_a[2][2];
    uint8_t sc_mul[2][2], sc_add[2][2];
    uint32_t sc_neg[2][2];
};

// v with its sign bit XORed with m (0 or 0x80000000): an integer operation
__device__ __forceinline__ double flip_mask(double v, uint32_t m) {
    return __hiloint2double(__double2hiint(v) ^ int(m), __double2loint(v));
}
__device__ __forceinline__ float flip_mask(float v, uint32_t m) { return __int_as_float(__float_as_int(v) ^ int(m)); }

template <typename R>
__device__ __forceinline__ R pick4(int code, const amp_t<R>& own, const amp_t<R>& par) {
    return code == 0 ? own.x : (code == 1 ? own.y : (code == 2 ? par.x : par.y));
}

template <typename R, int K, int G>
__global__ void __launch_bounds__(256)
k_apply_small(const amp_t<R>* x, amp_t<R>* y, const __grid_constant__ SmallGateArgs<R, K> a) {
    constexpr int D = 1 << K;
    using A = amp_t<R>;
    const int64_t T = blockDim.x;
    const int64_t g0 = a.g_base + (int64_t)blockIdx.x * T * G + threadIdx.x;
    A v[G][D];
    int64_t b[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const int64_t g = g0 + j * T;
        b[j] = g < a.n_groups ? insert_zeros<K>(g, a.st) : int64_t(-1);
        // every row of the group lies in [b, b + off[D-1]]
        if (b[j] >= 0 && !DIAQ_BOUNDS_OK(b[j] + a.off[D - 1], a.N, BS_APPLY_SMALL)) b[j] = -1;
        if (b[j] >= 0) {
#pragma unroll
            for (int c = 0; c < D; ++c) v[j][c] = ld_stream(x + b[j] + a.off[c]);
        }
    }
    if (K == 1 && a.scaled1) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (b[j] < 0) continue;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const A own = v[j][r], par = v[j][1 - r];
                A w;
                w.x = fma(a.sc_a[r][0], pick4<R>(a.sc_mul[r][0], own, par),
                          flip_mask(pick4<R>(a.sc_add[r][0], own, par), a.sc_neg[r][0]));
                w.y = fma(a.sc_a[r][1], pick4<R>(a.sc_mul[r][1], own, par),
                          flip_mask(pick4<R>(a.sc_add[r][1], own, par), a.sc_neg[r][1]));
                st_stream(y + b[j] + a.off[r], w);
            }
        }
        return;
    }
    if (K == 1 && a.dense1) {
        // y_r = m_r0 x0 + m_r1 x1, each complex product as in mac_typed:
        // first term re = mr x.re - mi x.im (a product, then an FMA), then two FMAs per part
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (b[j] < 0) continue;
            const A x0 = v[j][0], x1 = v[j][1];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const R ar = a.re[2 * r], ai = a.im[2 * r], br = a.re[2 * r + 1], bi = a.im[2 * r + 1];
                A acc;
                acc.x = ar * x0.x;
                acc.x = fma(-ai, x0.y, acc.x);
                acc.y = ar * x0.y;
                acc.y = fma(ai, x0.x, acc.y);
                acc.x = fma(br, x1.x, acc.x);
                acc.x = fma(-bi, x1.y, acc.x);
                acc.y = fma(br, x1.y, acc.y);
                acc.y = fma(bi, x1.x, acc.y);
                st_stream(y + b[j] + a.off[r], acc);
            }
        }
        return;
    }
    if (a.pattern == 3) {
        // diagonal phases: y_r = m_rr x_r, first-general product then FMA
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (b[j] < 0) continue;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                const R mr = a.re[r * D + r], mi = a.im[r * D + r];
                const A x = v[j][r];
                A acc;
                acc.x = mr * x.x;
                acc.x = fma(-mi, x.y, acc.x);
                acc.y = mr * x.y;
                acc.y = fma(mi, x.x, acc.y);
                st_stream(y + b[j] + a.off[r], acc);
            }
        }
        return;
    }
    if (K == 1 && (a.pattern == 1 || a.pattern == 2)) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (b[j] < 0) continue;
            const A x0 = v[j][0], x1 = v[j][1];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const R d = a.re[3 * r];  // real diagonal entry m_rr
                const A xd = r == 0 ? x0 : x1, xo = r == 0 ? x1 : x0;
                A acc;
                if (r == 0) {  // column 0 first: the diagonal entry opens the sum
                    acc.x = d * xd.x;
                    acc.y = d * xd.y;
                } 
                if (a.pattern == 1) {  // real off-diagonal m_r,1-r
                    const R o = a.re[r == 0 ? 1 : 2];
                    if (r == 0) {
                        acc.x = fma(o, xo.x, acc.x);
                        acc.y = fma(o, xo.y, acc.y);
                    } else {  // row 1: column 0 (off-diagonal) opens the sum
                        acc.x = o * xo.x;
                        acc.y = o * xo.y;
                        acc.x = fma(d, xd.x, acc.x);
                        acc.y = fma(d, xd.y, acc.y);
                    }
                } else {  // imaginary off-diagonal i*o
                    const R o = a.im[r == 0 ? 1 : 2];
                    if (r == 0) {
                        acc.x = fma(-o, xo.y, acc.x);
                        acc.y = fma(o, xo.x, acc.y);
                    } else {
                        acc.x = -o * xo.y;
                        acc.y = o * xo.x;
                        acc.x = fma(d, xd.x, acc.x);
                        acc.y = fma(d, xd.y, acc.y);
                    }
                }
                st_stream(y + b[j] + a.off[r], acc);
            }
        }
        return;
    }
    if (K == 1 && a.share_col0 == 1) {
        // real butterfly: p = a x0 (two products), y_r = fma(m_r1, x1, p)
        const R m00 = a.re[0], m01 = a.re[1], m11 = a.re[3];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (b[j] < 0) continue;
            const A x0 = v[j][0], x1 = v[j][1];
            const R px = m00 * x0.x, py = m00 * x0.y;
            A y0, y1;
            y0.x = fma(m01, x1.x, px);
            y0.y = fma(m01, x1.y, py);
            y1.x = fma(m11, x1.x, px);
            y1.y = fma(m11, x1.y, py);
            st_stream(y + b[j] + a.off[0], y0);
            st_stream(y + b[j] + a.off[1], y1);
        }
        return;
    }
    if (K == 1 && a.share_col0) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (b[j] < 0) continue;
            A p;
            bool first = true;
            mac_typed<R>(p, first, a.type[0], a.re[0], a.im[0], v[j][0]);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                A acc = p;
                bool f = false;
                mac_typed<R>(acc, f, a.type[r * D + 1], a.re[r * D + 1], a.im[r * D + 1], v[j][1]);
                st_stream(y + b[j] + a.off[r], acc);
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < G; ++j) {
        if (b[j] < 0) continue;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            A acc;
            acc.x = R(0);
            acc.y = R(0);
            bool first = true;
#pragma unroll
            for (int c = 0; c < D; ++c)
                mac_typed<R>(acc, first, a.type[r * D + c], a.re[r * D + c], a.im[r * D + c], v[j][c]);
            st_stream(y + b[j] + a.off[r], acc);
        }
    }
}

// ---------------------------------------------------------------------------
// On-the-fly apply, 4 <= k <= 6: the local matrix is staged in shared memory
// from the op's device copy; each block processes chunks of B groups whose
// 2^k * B amplitudes it loads into shared memory (group index fastest, so
// the loads coalesce), then writes the rows back.
// ---------------------------------------------------------------------------
struct LargeGateArgs {
    int64_t n_groups;
    int64_t N;
    int k;
    int st[DIAQ_MAX_K];
    int64_t off[1 << DIAQ_MAX_K];
};

template <typename R>
__global__ void __launch_bounds__(256)
k_apply_large(const amp_t<R>* x, amp_t<R>* y, const void* dmat, const __grid_constant__ LargeGateArgs a,
              int B) {
    using A = amp_t<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int k = a.k;
    const int D = 1 << k;
    const int DD = D * D;
    R* mre = reinterpret_cast<R*>(smem);
    R* mim = mre + DD;
    uint8_t* mty = reinterpret_cast<uint8_t*>(mim + DD);
    A* xs = reinterpret_cast<A*>(smem + ((2 * DD * sizeof(R) + DD + 15) / 16) * 16);
    // dmat layout: re[DD], im[DD] (R), type[DD] (uint8)
    const R* gre = reinterpret_cast<const R*>(dmat);
    const R* gim = gre + DD;
    const uint8_t* gty = reinterpret_cast<const uint8_t*>(gim + DD);
    for (int e = threadIdx.x; e < DD; e += blockDim.x) {
        mre[e] = gre[e];
        mim[e] = gim[e];
        mty[e] = gty[e];
    }
    __syncthreads();
    const int64_t n_chunks = (a.n_groups + B - 1) / B;
    const int per = B * D;
    for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        for (int e = threadIdx.x; e < per; e += blockDim.x) {
            const int gi = e % B, c = e / B;
            const int64_t g = ch * B + gi;
            if (g < a.n_groups) {
                const int64_t i = insert_zeros_rt(g, a.st, k) + a.off[c];
                A v;
                v.x = R(0);
                v.y = R(0);
                if (DIAQ_BOUNDS_OK(i, a.N, BS_APPLY_LARGE)) v = ld_stream(x + i);
                xs[c * B + gi] = v;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < per; e += blockDim.x) {
            const int gi = e % B, r = e / B;
            const int64_t g = ch * B + gi;
            if (g >= a.n_groups) continue;
            A acc;
            acc.x = R(0);
            acc.y = R(0);
            bool first = true;
            for (int c = 0; c < D; ++c)
                mac_typed<R>(acc, first, mty[r * D + c], mre[r * D + c], mim[r * D + c], xs[c * B + gi]);
            const int64_t i = insert_zeros_rt(g, a.st, k) + a.off[r];
            if (DIAQ_BOUNDS_OK(i, a.N, BS_APPLY_LARGE)) st_stream(y + i, acc);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host launch helpers
// ---------------------------------------------------------------------------
static void sorted_targets(const GateDesc& g, int* st) {
    for (int a = 0; a < g.k; ++a) st[a] = g.targets[a];
    std::sort(st, st + g.k);
}

static void local_offsets(const GateDesc& g, int64_t* off) {
    const int D = 1 << g.k;
    for (int c = 0; c < D; ++c) {
        int64_t o = 0;
        for (int a = 0; a < g.k; ++a)
            if ((c >> (g.k - 1 - a)) & 1) o += int64_t(1) << g.targets[a];
        off[c] = o;
    }
}

static int default_groups(diaq_dtype dt, int k) {
    // enough independent 16-byte loads in flight per thread
    if (k == 1) return dt == DIAQ_C128 ? 2 : 4;
    if (k == 2) return dt == DIAQ_C128 ? 1 : 2;
    return 1;
}

LaunchCfg& launch_cfg(diaq_dtype dt, int k) {
    static LaunchCfg table[2][DIAQ_MAX_K + 1];
    return table[dt == DIAQ_C128 ? 1 : 0][k < 0 ? 0 : (k > DIAQ_MAX_K ? DIAQ_MAX_K : k)];
}

template <typename R, int K, int G>
static diaq_status launch_small_G(int n, const GateDesc& g, const void* x, void* y, int threads,
                                  int64_t g_begin, int64_t g_end, cudaStream_t s) {
    SmallGateArgs<R, K> a;
    std::memset(&a, 0, sizeof(a));
    a.g_base = g_begin;
    a.n_groups = g_end;
    a.N = int64_t(1) << n;
    sorted_targets(g, a.st);
    local_offsets(g, a.off);
    constexpr int DD = 1 << (2 * K);
    for (int e = 0; e < DD; ++e) {
        a.re[e] = R(g.m[e].real());
        a.im[e] = R(g.m[e].imag());
        // classify after rounding to R so a c64 entry that rounds to 1 is exact
        a.type[e] = entry_type(cplx(double(a.re[e]), double(a.im[e])));
    }
    if (K == 1) {
        const bool shared = a.type[0] != ET_ZERO && a.type[2] == a.type[0] && a.re[2] == a.re[0] && a.im[2] == a.im[0];
        const bool butterfly = shared && a.type[0] == ET_REAL && a.type[1] == ET_REAL && a.type[3] == ET_REAL;
        a.share_col0 = butterfly ? 1 : (shared ? 2 : 0);
        a.dense1 = a.type[0] == ET_GENERAL && a.type[1] == ET_GENERAL && a.type[2] == ET_GENERAL &&
                   a.type[3] == ET_GENERAL;
        if (!a.dense1 && a.share_col0 != 1) {
            const bool rd = a.type[0] == ET_REAL && a.type[3] == ET_REAL;  // real diagonal, not 0 or 1
            if (rd && a.type[1] == ET_REAL && a.type[2] == ET_REAL) a.pattern = 1;
            else if (rd && a.type[1] == ET_IMAG && a.type[2] == ET_IMAG) a.pattern = 2;
        }
    }
    {
        bool diag = true;
        for (int r = 0; r < (1 << K); ++r)
            for (int c = 0; c < (1 << K); ++c)
                if (r == c ? a.type[r * (1 << K) + c] != ET_GENERAL : a.type[r * (1 << K) + c] != ET_ZERO) diag = false;
        if (diag) a.pattern = 3;
    }
    const int64_t per_block = int64_t(threads) * G;
    const int64_t blocks = (g_end - g_begin + per_block - 1) / per_block;
    if (blocks <= 0) return DIAQ_OK;
    DIAQ_PRELAUNCH("k_apply_small");
    k_apply_small<R, K, G><<<dim3((unsigned)blocks), threads, 0, s>>>(
        reinterpret_cast<const amp_t<R>*>(x), reinterpret_cast<amp_t<R>*>(y), a);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

// The scaled form of a one-qubit gate whose diagonal entries are real and
// non-zero and whose off-diagonal entries are both real or both imaginary
// and non-zero (RX, RY, H and the like), with |m00| = |m11|: U = sigma V,
// sigma = max(|m_rr|, |m_r,1-r|), the same for both rows. Every row of V has
// one entry of magnitude 1 (+-1 or +-i), so each output component is one
// fused multiply-add: fma(m / sigma, term, +-unit term). Writes sigma; false
// when the gate has no such form.
static bool scaled1_form(const GateDesc& g, double* sigma, double sc_a[2][2], uint8_t mul[2][2], uint8_t add[2][2],
                         uint32_t neg[2][2]) {
    if (g.k != 1 || g.m.size() != 4) return false;
    const cplx m00 = g.m[0], m01 = g.m[1], m10 = g.m[2], m11 = g.m[3];
    if (m00.imag() != 0.0 || m11.imag() != 0.0 || m00.real() == 0.0 || m11.real() == 0.0) return false;
    int P;  // 1: real off-diagonal, 2: imaginary off-diagonal
    if (m01.imag() == 0.0 && m10.imag() == 0.0 && m01.real() != 0.0 && m10.real() != 0.0) P = 1;
    else if (m01.real() == 0.0 && m10.real() == 0.0 && m01.imag() != 0.0 && m10.imag() != 0.0) P = 2;
    else return false;
    const double d[2] = {m00.real(), m11.real()};
    const double o[2] = {P == 1 ? m01.real() : m01.imag(), P == 1 ? m10.real() : m10.imag()};
    const double s0 = std::max(std::fabs(d[0]), std::fabs(o[0])), s1 = std::max(std::fabs(d[1]), std::fabs(o[1]));
    if (s0 != s1 || !(s0 > 0.0)) return false;
    const double sg = s0;
    constexpr uint32_t NEG = 0x80000000u;
    for (int r = 0; r < 2; ++r) {
        // input codes: 0 own.re, 1 own.im, 2 partner.re, 3 partner.im
        if (std::fabs(d[r]) == sg) {  // own term +-1: fma(o/sigma, partner part, +-own)
            const double A = o[r] / sg;
            const uint32_t on = d[r] < 0.0 ? NEG : 0u;
            if (P == 1) {
                sc_a[r][0] = A; mul[r][0] = 2; add[r][0] = 0; neg[r][0] = on;
                sc_a[r][1] = A; mul[r][1] = 3; add[r][1] = 1; neg[r][1] = on;
            } else {  // (i A) partner = (-A p.im, A p.re)
                sc_a[r][0] = -A; mul[r][0] = 3; add[r][0] = 0; neg[r][0] = on;
                sc_a[r][1] = A; mul[r][1] = 2; add[r][1] = 1; neg[r][1] = on;
            }
        } else {  // partner term +-1 or +-i: fma(d/sigma, own part, +-partner part)
            const double A = d[r] / sg;
            const bool un = o[r] < 0.0;
            if (P == 1) {
                sc_a[r][0] = A; mul[r][0] = 0; add[r][0] = 2; neg[r][0] = un ? NEG : 0u;
                sc_a[r][1] = A; mul[r][1] = 1; add[r][1] = 3; neg[r][1] = un ? NEG : 0u;
            } else {  // (+-i) partner = (-+p.im, +-p.re)
                sc_a[r][0] = A; mul[r][0] = 0; add[r][0] = 3; neg[r][0] = un ? 0u : NEG;
                sc_a[r][1] = A; mul[r][1] = 1; add[r][1] = 2; neg[r][1] = un ? NEG : 0u;
            }
        }
    }
    *sigma = sg;
    return true;
}

bool gate_scaled1_sigma(const GateDesc& g, double* sigma) {
    double a[2][2];
    uint8_t mul[2][2], add[2][2];
    uint32_t neg[2][2];
    return scaled1_form(g, sigma, a, mul, add, neg);
}

template <int G>
static diaq_status launch_scaled1_G(int n, const GateDesc& g, const void* x, void* y, int threads, int64_t g_begin,
                                    int64_t g_end, double* sigma, cudaStream_t s) {
    SmallGateArgs<double, 1> a;
    std::memset(&a, 0, sizeof(a));
    double ca[2][2];
    if (!scaled1_form(g, sigma, ca, a.sc_mul, a.sc_add, a.sc_neg))
        return fail(DIAQ_ERR_UNSUPPORTED, "gate has no scaled one-qubit form");
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) a.sc_a[r][c] = ca[r][c];
    a.scaled1 = 1;
    a.g_base = g_begin;
    a.n_groups = g_end;
    a.N = int64_t(1) << n;
    sorted_targets(g, a.st);
    local_offsets(g, a.off);
    const int64_t per_block = int64_t(threads) * G;
    const int64_t blocks = (g_end - g_begin + per_block - 1) / per_block;
    if (blocks <= 0) return DIAQ_OK;
    DIAQ_PRELAUNCH("k_apply_small");
    k_apply_small<double, 1, G><<<dim3((unsigned)blocks), threads, 0, s>>>(
        reinterpret_cast<const double2*>(x), reinterpret_cast<double2*>(y), a);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

// Groups [g_begin, g_end) of a complex128 one-qubit gate in the scaled form
// (V = U / sigma, *sigma written); DIAQ_ERR_UNSUPPORTED without one.
diaq_status launch_gate_scaled1_range(int n, const GateDesc& g, const void* x, void* y, int64_t g_begin,
                                      int64_t g_end, double* sigma, cudaStream_t s) {
    const LaunchCfg& cfg = launch_cfg(DIAQ_C128, 1);
    const int G = cfg.groups > 0 ? cfg.groups : default_groups(DIAQ_C128, 1);
    switch (G) {
        case 1: return launch_scaled1_G<1>(n, g, x, y, cfg.threads, g_begin, g_end, sigma, s);
        case 2: return launch_scaled1_G<2>(n, g, x, y, cfg.threads, g_begin, g_end, sigma, s);
        default: return launch_scaled1_G<4>(n, g, x, y, cfg.threads, g_begin, g_end, sigma, s);
    }
}

// ---------------------------------------------------------------------------
// Two one-qubit gates on different qubits, a then b, in one in-place pass
// (diaq_simulate): each thread takes groups of the 4 amplitudes that share
// every other bit, applies a along qa and b along qb in registers, and
// writes them back, so the state is read and written once for both. Each
// gate is either in the scaled form (the selectors of scaled1_form: one
// fused multiply-add per real component) or a general 2 x 2 complex matrix
// (the rows as in the dense one-qubit path).
// ---------------------------------------------------------------------------
template <typename R>
struct Pair1Gate {
    R re[4], im[4];                 // general form: row-major
    R sa[2][2];                     // scaled form: coefficient per row and component
    uint8_t smul[2][2], sadd[2][2];
    uint32_t sneg[2][2];
};

template <typename R>
struct Pair1Args {
    int64_t n_groups;
    int64_t N;
    int st[2];                      // targets, ascending
    int64_t oa, ob;                 // offsets of a's and b's target bits
    Pair1Gate<R> a, b;
};

template <typename R, bool SC>
__device__ __forceinline__ void pair1_apply(const Pair1Gate<R>& g, amp_t<R>& x0, amp_t<R>& x1) {
    using A = amp_t<R>;
    A w[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const A own = r == 0 ? x0 : x1, par = r == 0 ? x1 : x0;
        if (SC) {
            w[r].x = fma(g.sa[r][0], pick4<R>(g.smul[r][0], own, par),
                         flip_mask(pick4<R>(g.sadd[r][0], own, par), g.sneg[r][0]));
            w[r].y = fma(g.sa[r][1], pick4<R>(g.smul[r][1], own, par),
                         flip_mask(pick4<R>(g.sadd[r][1], own, par), g.sneg[r][1]));
        } else {
            const R ar = g.re[2 * r], ai = g.im[2 * r], br = g.re[2 * r + 1], bi = g.im[2 * r + 1];
            A acc;
            acc.x = ar * x0.x;
            acc.x = fma(-ai, x0.y, acc.x);
            acc.y = ar * x0.y;
            acc.y = fma(ai, x0.x, acc.y);
            acc.x = fma(br, x1.x, acc.x);
            acc.x = fma(-bi, x1.y, acc.x);
            acc.y = fma(br, x1.y, acc.y);
            acc.y = fma(bi, x1.x, acc.y);
            w[r] = acc;
        }
    }
    x0 = w[0];
    x1 = w[1];
}

template <typename R, bool SCA, bool SCB>
__global__ void __launch_bounds__(256) k_apply_pair1(amp_t<R>* x, const __grid_constant__ Pair1Args<R> a) {
    using A = amp_t<R>;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n_groups; g += T) {
        const int64_t b = insert_zeros<2>(g, a.st);
        if (!DIAQ_BOUNDS_OK(b + a.oa + a.ob, a.N, BS_APPLY_SMALL)) continue;
        A v[4];
        v[0] = ld_stream(x + b);
        v[1] = ld_stream(x + b + a.oa);
        v[2] = ld_stream(x + b + a.ob);
        v[3] = ld_stream(x + b + a.oa + a.ob);
        pair1_apply<R, SCA>(a.a, v[0], v[1]);
        pair1_apply<R, SCA>(a.a, v[2], v[3]);
        pair1_apply<R, SCB>(a.b, v[0], v[2]);
        pair1_apply<R, SCB>(a.b, v[1], v[3]);
        st_stream(x + b, v[0]);
        st_stream(x + b + a.oa, v[1]);
        st_stream(x + b + a.ob, v[2]);
        st_stream(x + b + a.oa + a.ob, v[3]);
    }
}

template <typename R>
static bool pair1_gate(const GateDesc& g, bool scaled, Pair1Gate<R>* out) {
    std::memset(out, 0, sizeof(*out));
    if (scaled) {
        double sig, ca[2][2];
        if (!scaled1_form(g, &sig, ca, out->smul, out->sadd, out->sneg)) return false;
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) out->sa[r][c] = R(ca[r][c]);
        return true;
    }
    for (int e = 0; e < 4; ++e) {
        out->re[e] = R(g.m[size_t(e)].real());
        out->im[e] = R(g.m[size_t(e)].imag());
    }
    return true;
}

// One in-place pass of one-qubit gates a then b (distinct targets) on the
// whole state; sa / sb: that gate in the scaled form (complex128; the
// caller tracks the dropped factor), else general.
diaq_status launch_pair1_inplace(int n, diaq_dtype dt, const GateDesc& ga, bool sa, const GateDesc& gb, bool sb,
                                 void* x, cudaStream_t s) {
    if (ga.k != 1 || gb.k != 1 || ga.targets[0] == gb.targets[0] || n < 2)
        return fail(DIAQ_ERR_ARG, "a pair needs two one-qubit gates on different qubits");
    if ((sa || sb) && dt != DIAQ_C128) return fail(DIAQ_ERR_UNSUPPORTED, "the scaled form is complex128 only");
    const int qa = ga.targets[0], qb = gb.targets[0];
    const int64_t groups = int64_t(1) << (n - 2);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((groups + 255) / 256, int64_t(device_sm_count()) * 8));
    DIAQ_PRELAUNCH("k_apply_pair1");
    if (dt == DIAQ_C128) {
        Pair1Args<double> a;
        std::memset(&a, 0, sizeof(a));
        a.n_groups = groups;
        a.N = int64_t(1) << n;
        a.st[0] = std::min(qa, qb);
        a.st[1] = std::max(qa, qb);
        a.oa = int64_t(1) << qa;
        a.ob = int64_t(1) << qb;
        if (!pair1_gate(ga, sa, &a.a) || !pair1_gate(gb, sb, &a.b))
            return fail(DIAQ_ERR_UNSUPPORTED, "gate has no scaled one-qubit form");
        double2* xd = reinterpret_cast<double2*>(x);
        if (sa && sb) k_apply_pair1<double, true, true><<<unsigned(blocks), 256, 0, s>>>(xd, a);
        else if (sa) k_apply_pair1<double, true, false><<<unsigned(blocks), 256, 0, s>>>(xd, a);
        else if (sb) k_apply_pair1<double, false, true><<<unsigned(blocks), 256, 0, s>>>(xd, a);
        else k_apply_pair1<double, false, false><<<unsigned(blocks), 256, 0, s>>>(xd, a);
    } else {
        Pair1Args<float> a;
        std::memset(&a, 0, sizeof(a));
        a.n_groups = groups;
        a.N = int64_t(1) << n;
        a.st[0] = std::min(qa, qb);
        a.st[1] = std::max(qa, qb);
        a.oa = int64_t(1) << qa;
        a.ob = int64_t(1) << qb;
        pair1_gate(ga, false, &a.a);
        pair1_gate(gb, false, &a.b);
        k_apply_pair1<float, false, false><<<unsigned(blocks), 256, 0, s>>>(reinterpret_cast<float2*>(x), a);
    }
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

template <typename R, int K>
static diaq_status launch_small(int n, diaq_dtype dt, const GateDesc& g, const void* x, void* y,
                                int64_t g_begin, int64_t g_end, cudaStream_t s) {
    const LaunchCfg& cfg = launch_cfg(dt, K);
    const int G = cfg.groups > 0 ? cfg.groups : default_groups(dt, K);
    const int threads = cfg.threads;
    switch (G) {
        case 1: return launch_small_G<R, K, 1>(n, g, x, y, threads, g_begin, g_end, s);
        case 2: return launch_small_G<R, K, 2>(n, g, x, y, threads, g_begin, g_end, s);
        default: return launch_small_G<R, K, 4>(n, g, x, y, threads, g_begin, g_end, s);
    }
}

// Groups [g_begin, g_end) of a k <= 3 gate (all of them: 0, 2^(n-k)).
diaq_status launch_gate_local_range(int n, diaq_dtype dt, const GateDesc& g, const void* x, void* y,
                                    int64_t g_begin, int64_t g_end, cudaStream_t s) {
    if (g.k < 1 || g.k > 3) return fail(DIAQ_ERR_UNSUPPORTED, "group ranges need k <= 3 (k = %d)", g.k);
    if (dt == DIAQ_C128) {
        switch (g.k) {
            case 1: return launch_small<double, 1>(n, dt, g, x, y, g_begin, g_end, s);
            case 2: return launch_small<double, 2>(n, dt, g, x, y, g_begin, g_end, s);
            default: return launch_small<double, 3>(n, dt, g, x, y, g_begin, g_end, s);
        }
    }
    switch (g.k) {
        case 1: return launch_small<float, 1>(n, dt, g, x, y, g_begin, g_end, s);
        case 2: return launch_small<float, 2>(n, dt, g, x, y, g_begin, g_end, s);
        default: return launch_small<float, 3>(n, dt, g, x, y, g_begin, g_end, s);
    }
}

static size_t large_smem_bytes(diaq_dtype dt, int k, int B) {
    const size_t DD = size_t(1) << (2 * k);
    const size_t rs = dt == DIAQ_C128 ? 8 : 4;
    const size_t head = ((2 * DD * rs + DD + 15) / 16) * 16;
    return head + size_t(B) * (size_t(1) << k) * amp_bytes(dt);
}

template <typename R>
static diaq_status launch_large(int n, diaq_dtype dt, const GateDesc& g, const void* dmat,
                                const void* x, void* y, cudaStream_t s) {
    LargeGateArgs a;
    std::memset(&a, 0, sizeof(a));
    a.k = g.k;
    a.n_groups = int64_t(1) << (n - g.k);
    a.N = int64_t(1) << n;
    sorted_targets(g, a.st);
    local_offsets(g, a.off);
    const int B = 32;
    const size_t smem = large_smem_bytes(dt, g.k, B);
    DIAQ_CUDA(cudaFuncSetAttribute(k_apply_large<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0;
    DIAQ_CUDA(cudaGetDevice(&dev));
    DIAQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t n_chunks = (a.n_groups + B - 1) / B;
    const int64_t blocks = std::min<int64_t>(n_chunks, int64_t(sms) * 8);
    DIAQ_PRELAUNCH("k_apply_large");
    k_apply_large<R><<<dim3((unsigned)blocks), 256, smem, s>>>(
        reinterpret_cast<const amp_t<R>*>(x), reinterpret_cast<amp_t<R>*>(y), dmat, a, B);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

// Device copy of a local matrix for the k >= 4 kernel: re[DD], im[DD], type[DD].
diaq_status upload_matrix(diaq_op_s* op) {
    const int k = op->gate.k;
    const size_t DD = size_t(1) << (2 * k);
    const size_t rs = op->dtype == DIAQ_C128 ? 8 : 4;
    std::vector<unsigned char> buf(2 * DD * rs + DD);
    for (size_t e = 0; e < DD; ++e) {
        const cplx v = op->gate.m[e];
        uint8_t t;
        if (rs == 8) {
            reinterpret_cast<double*>(buf.data())[e] = v.real();
            reinterpret_cast<double*>(buf.data())[DD + e] = v.imag();
            t = entry_type(v);
        } else {
            const float fr = float(v.real()), fi = float(v.imag());
            reinterpret_cast<float*>(buf.data())[e] = fr;
            reinterpret_cast<float*>(buf.data())[DD + e] = fi;
            t = entry_type(cplx(fr, fi));
        }
        buf[2 * DD * rs + e] = t;
    }
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, buf.size());
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMalloc of %zu bytes for the gate matrix failed: %s",
                                      buf.size(), cudaGetErrorString(e));
    e = cudaMemcpy(d, buf.data(), buf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "cudaMemcpy(gate matrix)");
    }
    op->d_matrix = d;
    return DIAQ_OK;
}

diaq_status launch_gate_local(int n, diaq_dtype dt, const GateDesc& g, const void* d_matrix,
                              const void* x, void* y, cudaStream_t s) {
    if (g.k <= 3) return launch_gate_local_range(n, dt, g, x, y, 0, int64_t(1) << (n - g.k), s);
    if (is_diagonal(g)) return launch_diag(n, dt, g, x, y, s);
    if (!d_matrix) return fail(DIAQ_ERR_ARG, "k = %d op has no device matrix", g.k);
    return dt == DIAQ_C128 ? launch_large<double>(n, dt, g, d_matrix, x, y, s)
                           : launch_large<float>(n, dt, g, d_matrix, x, y, s);
}

diaq_status launch_onthefly(const diaq_op_s* op, const void* x, void* y, cudaStream_t s) {
    return launch_gate_local(op->n, op->dtype, op->gate, op->d_matrix, x, y, s);
}

// ---------------------------------------------------------------------------
// Stored variant: materialise the diagonals, then the DiaQ SpMV.
// ---------------------------------------------------------------------------
struct RowMap {
    // Row order that keeps whole groups inside a block: linear row j ->
    // group g = (j_high << L) | j_low, local index c = (j >> L) & (2^k - 1),
    // row = insert_zeros(g) + off[c]. k = 0 means identity.
    int k;
    int L;
    int st[DIAQ_MAX_K];
    int64_t off[1 << DIAQ_MAX_K];
};

__device__ __forceinline__ int64_t map_row(int64_t j, const RowMap& m) {
    if (m.k == 0) return j;
    const int64_t lowmask = (int64_t(1) << m.L) - 1;
    const int64_t c = (j >> m.L) & ((int64_t(1) << m.k) - 1);
    const int64_t g = ((j >> (m.L + m.k)) << m.L) | (j & lowmask);
    return insert_zeros_rt(g, m.st, m.k) + m.off[c];
}

// A stored value is zero when both halves of its bit pattern are zero once
// the sign bit is masked (-0 counts as zero, NaN does not). The tests run on
// the integer pipes: FP64 compares would compete with the arithmetic for
// the FP64 pipe.
__device__ __forceinline__ bool zero_bits(double v) {
    return ((__double2hiint(v) & 0x7fffffff) | __double2loint(v)) == 0;
}
__device__ __forceinline__ bool zero_bits(float v) { return (__float_as_int(v) & 0x7fffffff) == 0; }

// -v when neg, else v, by flipping the sign bit with an integer operation.
__device__ __forceinline__ double flip_sign(double v, bool neg) {
    return __hiloint2double(__double2hiint(v) ^ (neg ? int(0x80000000) : 0), __double2loint(v));
}
__device__ __forceinline__ float flip_sign(float v, bool neg) {
    return __int_as_float(__float_as_int(v) ^ (neg ? int(0x80000000) : 0));
}

// acc += a * v for one stored diagonal of a raw op, with warp-uniform
// control flow: a lane whose value is zero adds fma(0, v, acc) = acc, so no
// lane branches on its own value. The warp skips the diagonal when it is
// zero on every lane, and the imaginary half when every lane's value is real
// (CPLX = false: the op's values are all real, so there is no imaginary
// half). The skip is nested around the imaginary half on purpose: measured,
// without that nesting the compiler predicates the whole skip, and
// predicated-off FP64 instructions still occupy the FP64 pipe.
template <typename R, bool CPLX>
__device__ __forceinline__ void stored_mac(amp_t<R>& acc, amp_t<R> a, amp_t<R> v) {
    const bool cplx = CPLX && !zero_bits(a.y);
    const bool nz = cplx || !zero_bits(a.x);
    if (!__any_sync(0xffffffffu, nz)) return;
    acc.x = fma(a.x, v.x, acc.x);
    acc.y = fma(a.x, v.y, acc.y);
    if (CPLX && __any_sync(0xffffffffu, cplx)) {
        acc.x = fma(-a.y, v.y, acc.x);
        acc.y = fma(a.y, v.x, acc.y);
    }
}

// Offsets and value starts of up to STORED_PARAM_D diagonals, passed by
// value so that no thread waits on a load before it can address x and the
// values; ops with more diagonals read them from device memory.
//
// For a gate op on k <= STORED_CLS_K targets, also the terms of each local
// row class: a row whose target bits are c (the matrix's local row index)
// has A[i][i+d] = M[c][c2] for d = off[c2] - off[c], that column is always
// inside the state, and every other entry of the row is zero. cls[c][e]
// (e < ecount) codes the term of one entry M[c][c2] != 0 as (q << 1) | h:
// the stored diagonal q and, for ops whose entries are each real or
// imaginary (STORED_TERMS_HALF), whether the term multiplies the value's
// imaginary part (h = 1). Entries M[c][c2] = 0 have no term. 0xff marks the
// end of a class's terms.
constexpr int STORED_PARAM_D = 16;
constexpr int STORED_CLS_K = 3;
constexpr int STORED_THREADS = 256;  // launch shape of k_stored_spmv
constexpr int STORED_G = 2;          // rows per thread
// Kind of the terms, fixed per op: all values real (2 FMAs per term); each
// value real or imaginary (2 FMAs, the half chosen per term); complex values
// (4 FMAs per term).
constexpr int STORED_TERMS_REAL = 0;
constexpr int STORED_TERMS_HALF = 1;
constexpr int STORED_TERMS_COMPLEX = 2;
struct StoredDiags {
    int64_t off[STORED_PARAM_D];
    int64_t start[STORED_PARAM_D];
    int ecount;  // 0: no class table (raw ops, k > STORED_CLS_K)
    uint8_t cls[1 << STORED_CLS_K][1 << STORED_CLS_K];
};

// Algorithm 2 over the stored diagonals. Each thread takes G rows (grouped
// by the row map so that a block holds every row its targets couple).
//
// CLS (gate ops, k <= 3): each row walks only the terms of its local row
// class (from the class table) and multiplies them without testing the
// values: the class is warp-uniform under the row map, so no warp diverges
// or votes, and each row does its own multiply-adds only. The FMAs per term
// follow the op's KIND; for STORED_TERMS_HALF the half a term multiplies is
// chosen with integer selects and a sign flip, never with a branch (a
// branch around FP64 work is predicated by the compiler, and predicated-off
// FP64 instructions still occupy the FP64 pipe). Measured, splitting a
// complex entry into two half terms was slower than one 4-FMA term.
//
// Otherwise (raw ops): each row walks every diagonal in stored order, with
// the warp-uniform skips of stored_mac. Threads past N keep running with
// zero values so that every warp vote sees full warps.
//
// Both issue a diagonal's value and x loads together. (Issuing several
// diagonals' loads before using any of them was measured slower: the extra
// registers cost more occupancy than the shorter dependency chain gained.)
// KIND = STORED_TERMS_REAL only for ops whose stored values are all real;
// STORED_TERMS_HALF only with CLS.
template <typename R, int G, int KIND, bool CLS>
__global__ void __launch_bounds__(256)
k_stored_spmv(const amp_t<R>* x, amp_t<R>* y, int64_t N, int D, const int64_t* __restrict__ offs,
              const int64_t* __restrict__ starts, const amp_t<R>* __restrict__ vals,
              const __grid_constant__ RowMap map, const __grid_constant__ StoredDiags sd) {
    using A = amp_t<R>;
    const int64_t T = blockDim.x;
    const int64_t j0 = (int64_t)blockIdx.x * T * G + threadIdx.x;
    const bool by_value = D <= STORED_PARAM_D;
    int64_t row[G];
    int cls[G];
    A acc[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
        const int64_t j = j0 + u * T;
        row[u] = j < N ? map_row(j, map) : int64_t(-1);
        cls[u] = CLS ? int((j >> map.L) & ((int64_t(1) << map.k) - 1)) : 0;
        acc[u].x = R(0);
        acc[u].y = R(0);
    }
    const int E = CLS ? sd.ecount : D;
    for (int e = 0; e < E; ++e) {
        A a[G], xv[G];
        bool imag_half[G];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const int code = CLS ? int(sd.cls[cls[u]][e]) : (e << 1);
            const int q = code >> 1;
            imag_half[u] = (code & 1) != 0;
            bool ok = row[u] >= 0 && code != 0xff;
            int64_t d = 0, p = 0, st = 0;
            if (ok) {
                d = CLS || by_value ? sd.off[q] : offs[q];
                st = CLS || by_value ? sd.start[q] : starts[q];
                p = row[u] - (d < 0 ? -d : 0);
                ok = p >= 0 && p < N - (d < 0 ? -d : d);
            }
            if (ok) ok = DIAQ_BOUNDS_OK(row[u] + d, N, BS_STORED_X) && DIAQ_BOUNDS_OK(row[u], N, BS_STORED_VALUE);
            if (ok) {
                a[u] = ld_stream(vals + st + p);
                xv[u] = x[row[u] + d];
            } else {
                a[u].x = R(0);
                a[u].y = R(0);
                xv[u].x = R(0);
                xv[u].y = R(0);
            }
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (CLS && KIND == STORED_TERMS_REAL) {
                acc[u].x = fma(a[u].x, xv[u].x, acc[u].x);
                acc[u].y = fma(a[u].x, xv[u].y, acc[u].y);
            } else if (CLS && KIND == STORED_TERMS_COMPLEX) {
                acc[u].x = fma(a[u].x, xv[u].x, acc[u].x);
                acc[u].x = fma(-a[u].y, xv[u].y, acc[u].x);
                acc[u].y = fma(a[u].x, xv[u].y, acc[u].y);
                acc[u].y = fma(a[u].y, xv[u].x, acc[u].y);
            } else if (CLS) {
                // real half: acc += re(a) (x.x, x.y); imaginary half:
                // acc += im(a) (-x.y, x.x)
                const bool h = imag_half[u];
                const R m = h ? a[u].y : a[u].x;
                const R x0 = flip_sign(h ? xv[u].y : xv[u].x, h);
                const R x1 = h ? xv[u].x : xv[u].y;
                acc[u].x = fma(m, x0, acc[u].x);
                acc[u].y = fma(m, x1, acc[u].y);
            } else {
                stored_mac<R, KIND != STORED_TERMS_REAL>(acc[u], a[u], xv[u]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < G; ++u)
        if (row[u] >= 0) st_stream(y + row[u], acc[u]);
}

// v_q[t] = A[i][i+d], i = t + max(0, -d): M[local(i)][local(i+d)] when i
// and i+d agree outside the targets, else 0.
struct MatArgs {
    int k;
    int t[DIAQ_MAX_K];  // targets in gate order (t[0] = most significant local bit)
    int64_t tmask;
};

template <typename R>
__global__ void __launch_bounds__(256)
k_materialise(amp_t<R>* vals, int64_t N, const int64_t* __restrict__ offs,
              const int64_t* __restrict__ starts, const R* __restrict__ mre, const R* __restrict__ mim,
              const __grid_constant__ MatArgs ma) {
    using A = amp_t<R>;
    const int q = blockIdx.y;
    const int64_t d = offs[q];
    const int64_t len = N - (d < 0 ? -d : d);
    const int64_t shift = d < 0 ? -d : 0;
    const int k = ma.k;
    const int D = 1 << k;
    A* out = vals + starts[q];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t + shift, j = i + d;
        A v;
        v.x = R(0);
        v.y = R(0);
        if (((i ^ j) & ~ma.tmask) == 0 && DIAQ_BOUNDS_OK(j, N, BS_MATERIALISE)) {
            int r = 0, c = 0;
            for (int a = 0; a < k; ++a) {
                r |= int((i >> ma.t[a]) & 1) << (k - 1 - a);
                c |= int((j >> ma.t[a]) & 1) << (k - 1 - a);
            }
            v.x = mre[r * D + c];
            v.y = mim[r * D + c];
        }
        st_stream(out + t, v);
    }
}

static RowMap make_rowmap(const GateDesc& g, int n, int threads, int G) {
    RowMap m;
    std::memset(&m, 0, sizeof(m));
    m.k = g.k;
    for (int a = 0; a < g.k; ++a) m.st[a] = g.targets[a];
    std::sort(m.st, m.st + g.k);
    local_offsets(g, m.off);
    // low group bits per block: a block covers threads*G rows = 2^(L+k)
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= int64_t(threads) * G) ++lg;
    m.L = std::max(0, std::min(lg - g.k, n - g.k));
    return m;
}

// Class table of a gate op on k <= STORED_CLS_K targets: for each local row
// class c, one term per entry M[c][c2] != 0 (diagonal d = off[c2] - off[c]),
// in stored order, and the op's term kind in *kind. *values_read (if not
// NULL) gets the number of stored values the SpMV reads, N / 2^k x the
// non-zero entries. Returns false when the op takes the generic path (raw
// ops, k > STORED_CLS_K, more than STORED_PARAM_D diagonals).
static bool stored_class_table(const diaq_op_s* op, const RowMap& map, int D, StoredDiags* sd, int* kind,
                               int64_t* values_read) {
    if (op->op_class == DIAQ_CLASS_RAW || map.k < 1 || map.k > STORED_CLS_K || D > STORED_PARAM_D) return false;
    const int K = 1 << map.k;
    bool any_imag = false, any_complex = false;
    for (const cplx& m : op->gate.m) {
        any_imag |= m.imag() != 0.0;
        any_complex |= m.real() != 0.0 && m.imag() != 0.0;
    }
    *kind = any_complex ? STORED_TERMS_COMPLEX : any_imag ? STORED_TERMS_HALF : STORED_TERMS_REAL;
    std::memset(sd->cls, 0xff, sizeof(sd->cls));
    sd->ecount = 0;
    int64_t entries = 0;
    for (int c = 0; c < K; ++c) {
        int e = 0;
        for (int q = 0; q < D; ++q)
            for (int c2 = 0; c2 < K; ++c2)
                if (op->offsets[size_t(q)] == map.off[c2] - map.off[c]) {
                    const cplx m = op->gate.m[size_t(c) * K + c2];
                    if (m.real() != 0.0 || m.imag() != 0.0) {
                        const int h = *kind == STORED_TERMS_HALF && m.imag() != 0.0 ? 1 : 0;
                        sd->cls[c][e++] = uint8_t((q << 1) | h);
                        ++entries;
                    }
                    break;
                }
        sd->ecount = std::max(sd->ecount, e);
    }
    if (values_read) *values_read = (int64_t(1) << (op->n - map.k)) * entries;
    return true;
}

template <typename R, int G>
static void stored_launch(int kind, bool cls, dim3 grid, int threads, cudaStream_t s, const void* x, void* y,
                          int64_t N, int D, const diaq_op_s* op, const RowMap& map, const StoredDiags& sd) {
    using A = amp_t<R>;
    const A* xa = reinterpret_cast<const A*>(x);
    A* ya = reinterpret_cast<A*>(y);
    const A* va = reinterpret_cast<const A*>(op->d_values);
    const int64_t* o = op->d_offsets;
    const int64_t* t = op->d_starts;
    if (cls && kind == STORED_TERMS_REAL)
        k_stored_spmv<R, G, STORED_TERMS_REAL, true><<<grid, threads, 0, s>>>(xa, ya, N, D, o, t, va, map, sd);
    else if (cls && kind == STORED_TERMS_HALF)
        k_stored_spmv<R, G, STORED_TERMS_HALF, true><<<grid, threads, 0, s>>>(xa, ya, N, D, o, t, va, map, sd);
    else if (cls)
        k_stored_spmv<R, G, STORED_TERMS_COMPLEX, true><<<grid, threads, 0, s>>>(xa, ya, N, D, o, t, va, map, sd);
    else if (kind == STORED_TERMS_REAL)
        k_stored_spmv<R, G, STORED_TERMS_REAL, false><<<grid, threads, 0, s>>>(xa, ya, N, D, o, t, va, map, sd);
    else
        k_stored_spmv<R, G, STORED_TERMS_COMPLEX, false><<<grid, threads, 0, s>>>(xa, ya, N, D, o, t, va, map, sd);
}

diaq_status launch_stored(const diaq_op_s* op, const void* x, void* y, cudaStream_t s) {
    const int64_t N = int64_t(1) << op->n;
    const int threads = STORED_THREADS, G = STORED_G;
    RowMap map;
    if (op->op_class == DIAQ_CLASS_RAW) {
        std::memset(&map, 0, sizeof(map));
    } else {
        map = make_rowmap(op->gate, op->n, threads, G);
    }
    const int64_t blocks = (N + int64_t(threads) * G - 1) / (int64_t(threads) * G);
    const int D = (int)op->offsets.size();
    if (D == 0) {
        // the zero operator: y = 0
        DIAQ_CUDA(cudaMemsetAsync(y, 0, size_t(N) * amp_bytes(op->dtype), s));
        return DIAQ_OK;
    }
    StoredDiags sd;
    std::memset(&sd, 0, sizeof(sd));
    for (int q = 0; q < D && q < STORED_PARAM_D; ++q) {
        sd.off[q] = op->offsets[size_t(q)];
        sd.start[q] = op->starts[size_t(q)];
    }
    int kind = op->real_values ? STORED_TERMS_REAL : STORED_TERMS_COMPLEX;
    const bool cls = stored_class_table(op, map, D, &sd, &kind, nullptr);
    DIAQ_PRELAUNCH("k_stored_spmv");
    const dim3 grid((unsigned)blocks);
    if (op->dtype == DIAQ_C128)
        stored_launch<double, G>(kind, cls, grid, threads, s, x, y, N, D, op, map, sd);
    else
        stored_launch<float, G>(kind, cls, grid, threads, s, x, y, N, D, op, map, sd);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

int64_t stored_values_read(const diaq_op_s* op) {
    const int D = (int)op->offsets.size();
    if (op->op_class == DIAQ_CLASS_RAW || D == 0) return op->stored_elems;
    const RowMap map = make_rowmap(op->gate, op->n, STORED_THREADS, STORED_G);
    StoredDiags sd;
    std::memset(&sd, 0, sizeof(sd));
    int kind = 0;
    int64_t values_read = 0;
    if (!stored_class_table(op, map, D, &sd, &kind, &values_read)) return op->stored_elems;
    return values_read;
}

diaq_status launch_materialise(diaq_op_s* op, cudaStream_t s) {
    const int64_t N = int64_t(1) << op->n;
    const int k = op->gate.k;
    const int D = 1 << k;
    // matrix (re, im) in the op's precision, temporary device copy
    const size_t rs = op->dtype == DIAQ_C128 ? 8 : 4;
    std::vector<unsigned char> buf(2 * size_t(D) * D * rs);
    for (int e = 0; e < D * D; ++e) {
        if (rs == 8) {
            reinterpret_cast<double*>(buf.data())[e] = op->gate.m[e].real();
            reinterpret_cast<double*>(buf.data())[D * D + e] = op->gate.m[e].imag();
        } else {
            reinterpret_cast<float*>(buf.data())[e] = float(op->gate.m[e].real());
            reinterpret_cast<float*>(buf.data())[D * D + e] = float(op->gate.m[e].imag());
        }
    }
    void* dm = nullptr;
    cudaError_t e = cudaMallocAsync(&dm, buf.size(), s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(gate matrix): %s", cudaGetErrorString(e));
    DIAQ_CUDA(cudaMemcpyAsync(dm, buf.data(), buf.size(), cudaMemcpyHostToDevice, s));
    MatArgs ma;
    std::memset(&ma, 0, sizeof(ma));
    ma.k = k;
    for (int a = 0; a < k; ++a) {
        ma.t[a] = op->gate.targets[a];
        ma.tmask |= int64_t(1) << op->gate.targets[a];
    }
    const int Dq = (int)op->offsets.size();
    if (Dq == 0) {
        // the zero operator: no diagonal to fill (its SpMV writes y = 0)
        DIAQ_CUDA(cudaStreamSynchronize(s));
        DIAQ_CUDA(cudaFreeAsync(dm, s));
        return DIAQ_OK;
    }
    const int64_t bx = std::min<int64_t>((N + 255) / 256, 4096);
    DIAQ_PRELAUNCH("k_materialise");
    if (op->dtype == DIAQ_C128)
        k_materialise<double><<<dim3((unsigned)bx, (unsigned)Dq), 256, 0, s>>>(
            reinterpret_cast<double2*>(op->d_values), N, op->d_offsets, op->d_starts,
            reinterpret_cast<const double*>(dm), reinterpret_cast<const double*>(dm) + D * D, ma);
    else
        k_materialise<float><<<dim3((unsigned)bx, (unsigned)Dq), 256, 0, s>>>(
            reinterpret_cast<float2*>(op->d_values), N, op->d_offsets, op->d_starts,
            reinterpret_cast<const float*>(dm), reinterpret_cast<const float*>(dm) + D * D, ma);
    DIAQ_CUDA(cudaGetLastError());
    // the host buffer must outlive the async copy
    DIAQ_CUDA(cudaStreamSynchronize(s));
    DIAQ_CUDA(cudaFreeAsync(dm, s));
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// Device DiaQ product (Algorithm 1, accumulating): C_e(i) = sum over pairs
// (a, b) with a + b = e of A(i, i+a) B(i+a, i+a+b), for the rows where both
// factors exist. One thread per output element; pairs in fixed order.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_spgemm(amp_t<R>* cvals, const int64_t* __restrict__ c_offs, const int64_t* __restrict__ c_starts,
         const int32_t* __restrict__ pair_first, const int32_t* __restrict__ pair_a,
         const int32_t* __restrict__ pair_b, const amp_t<R>* __restrict__ avals,
         const int64_t* __restrict__ a_offs, const int64_t* __restrict__ a_starts,
         const amp_t<R>* __restrict__ bvals, const int64_t* __restrict__ b_offs,
         const int64_t* __restrict__ b_starts, int64_t N) {
    using A = amp_t<R>;
    const int q = blockIdx.y;
    const int64_t e = c_offs[q];
    const int64_t len = N - (e < 0 ? -e : e);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t + (e < 0 ? -e : 0);
        A acc;
        acc.x = R(0);
        acc.y = R(0);
        for (int p = pair_first[q]; p < pair_first[q + 1]; ++p) {
            const int qa = pair_a[p], qb = pair_b[p];
            const int64_t a = a_offs[qa], b = b_offs[qb];
            const int64_t m = i + a;
            if (m < 0 || m >= N || m + b < 0 || m + b >= N) continue;
            if (!DIAQ_BOUNDS_OK(i - (a < 0 ? -a : 0), N - (a < 0 ? -a : a), BS_SPGEMM)) continue;
            const A av = avals[a_starts[qa] + (i - (a < 0 ? -a : 0))];
            const A bv = bvals[b_starts[qb] + (m - (b < 0 ? -b : 0))];
            acc.x = fma(av.x, bv.x, acc.x);
            acc.x = fma(-av.y, bv.y, acc.x);
            acc.y = fma(av.x, bv.y, acc.y);
            acc.y = fma(av.y, bv.x, acc.y);
        }
        cvals[c_starts[q] + t] = acc;
    }
}

diaq_status launch_spgemm(const diaq_op_s* A, const diaq_op_s* B, diaq_op_s* C, cudaStream_t s) {
    // host: result indices and the (a, b) pairs meeting on each
    const int64_t N = int64_t(1) << A->n;
    std::vector<std::pair<int64_t, std::pair<int32_t, int32_t>>> pairs;
    for (size_t qa = 0; qa < A->offsets.size(); ++qa)
        for (size_t qb = 0; qb < B->offsets.size(); ++qb) {
            const int64_t a = A->offsets[qa], b = B->offsets[qb], e = a + b;
            const int64_t lo = std::max<int64_t>({0, -a, -e});
            const int64_t hi = std::min<int64_t>({N, N - a, N - e});
            if (lo >= hi) continue;  // no overlap: the product diagonal is not valid
            pairs.push_back({e, {int32_t(qa), int32_t(qb)}});
        }
    std::stable_sort(pairs.begin(), pairs.end(),
                     [](const auto& u, const auto& v) { return u.first < v.first; });
    std::vector<int64_t> offs;
    std::vector<int32_t> first, pa, pb;
    for (size_t p = 0; p < pairs.size(); ++p) {
        if (offs.empty() || offs.back() != pairs[p].first) {
            offs.push_back(pairs[p].first);
            first.push_back(int32_t(p));
        }
        pa.push_back(pairs[p].second.first);
        pb.push_back(pairs[p].second.second);
    }
    first.push_back(int32_t(pairs.size()));
    C->offsets = offs;
    C->starts.resize(offs.size());
    int64_t tot = 0;
    for (size_t q = 0; q < offs.size(); ++q) {
        C->starts[q] = tot;
        tot += N - (offs[q] < 0 ? -offs[q] : offs[q]);
    }
    C->stored_elems = tot;
    const size_t ab = amp_bytes(C->dtype);
    cudaError_t e;
    if ((e = cudaMalloc(&C->d_values, size_t(std::max<int64_t>(tot, 1)) * ab)) != cudaSuccess ||
        (e = cudaMalloc((void**)&C->d_offsets, std::max<size_t>(offs.size(), 1) * 8)) != cudaSuccess ||
        (e = cudaMalloc((void**)&C->d_starts, std::max<size_t>(offs.size(), 1) * 8)) != cudaSuccess)
        return fail(DIAQ_ERR_ALLOC, "device allocation for the DiaQ product failed: %s", cudaGetErrorString(e));
    int32_t* dp = nullptr;
    const size_t pbytes = (first.size() + pa.size() + pb.size()) * 4;
    if ((e = cudaMallocAsync((void**)&dp, pbytes, s)) != cudaSuccess)
        return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(pairs): %s", cudaGetErrorString(e));
    std::vector<int32_t> packed(first);
    packed.insert(packed.end(), pa.begin(), pa.end());
    packed.insert(packed.end(), pb.begin(), pb.end());
    DIAQ_CUDA(cudaMemcpyAsync(dp, packed.data(), pbytes, cudaMemcpyHostToDevice, s));
    DIAQ_CUDA(cudaMemcpyAsync(C->d_offsets, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, s));
    DIAQ_CUDA(cudaMemcpyAsync(C->d_starts, C->starts.data(), offs.size() * 8, cudaMemcpyHostToDevice, s));
    if (!offs.empty()) {
        DIAQ_PRELAUNCH("k_spgemm");
        const int64_t bx = std::min<int64_t>((N + 255) / 256, 4096);
        const int32_t* d_first = dp;
        const int32_t* d_pa = dp + first.size();
        const int32_t* d_pb = d_pa + pa.size();
        if (C->dtype == DIAQ_C128)
            k_spgemm<double><<<dim3((unsigned)bx, (unsigned)offs.size()), 256, 0, s>>>(
                reinterpret_cast<double2*>(C->d_values), C->d_offsets, C->d_starts, d_first, d_pa, d_pb,
                reinterpret_cast<const double2*>(A->d_values), A->d_offsets, A->d_starts,
                reinterpret_cast<const double2*>(B->d_values), B->d_offsets, B->d_starts, N);
        else
            k_spgemm<float><<<dim3((unsigned)bx, (unsigned)offs.size()), 256, 0, s>>>(
                reinterpret_cast<float2*>(C->d_values), C->d_offsets, C->d_starts, d_first, d_pa, d_pb,
                reinterpret_cast<const float2*>(A->d_values), A->d_offsets, A->d_starts,
                reinterpret_cast<const float2*>(B->d_values), B->d_offsets, B->d_starts, N);
        DIAQ_CUDA(cudaGetLastError());
    }
    DIAQ_CUDA(cudaStreamSynchronize(s));  // host vectors feed async copies
    DIAQ_CUDA(cudaFreeAsync(dp, s));
    return DIAQ_OK;
}

}  // namespace diaq
