// Diagonal ops of 4 to 6 qubits. Z-type and controlled-phase gates hold
// their values on the principal diagonal only (Section III-A), and so does
// any product of them: a fused run of a QFT's controlled phases (Section VI
// fuses gates with the DIA x DIA product of Algorithm 1) is one diagonal
// op whose single DiaQ diagonal is index 0. Row i is then
// y[i] = M[c][c] x[i], with c the row's local index on the targets: one
// table lookup and one complex multiply, where the general 4..6-qubit
// kernel spends 2^k complex multiply-adds per row.
//
// In place (y == x), a row whose entry is exactly 1 is neither read nor
// written (a fused controlled-phase group leaves every row with the target
// bit clear unchanged); out of place it is copied. The product is the one
// the typed path forms for a general complex entry (a product, then a
// fused multiply-add, per part), so results match it bit for bit.
//
// Algorithmic bytes: out of place 2 N s; in place
// 2 s N / 2^k x (entries that are not exactly 1).

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "bounds.cuh"
#include "common.cuh"
#include "internal.h"

DIAQ_BOUNDS_TU(diag)

namespace diaq {
namespace {

template <typename R>
struct DiagArgs {
    int64_t N;
    int k;
    int t[DIAQ_MAX_K];      // targets; t[0] is the most significant local bit
    uint64_t one;           // bit c set: entry c is exactly 1 in R
    R re[1 << DIAQ_MAX_K];
    R im[1 << DIAQ_MAX_K];
};

constexpr int kDiagUnroll = 4;

template <typename R, bool INPLACE>
__global__ void __launch_bounds__(256) k_apply_diag(const amp_t<R>* x, amp_t<R>* y,
                                                    const __grid_constant__ DiagArgs<R> a) {
    using A = amp_t<R>;
    // The entries go to shared memory first: the lanes of a warp index them
    // by their own row class, and indexed reads of kernel parameters with
    // different addresses across a warp are served one address at a time.
    __shared__ A tab[1 << DIAQ_MAX_K];
    for (int c = threadIdx.x; c < (1 << a.k); c += blockDim.x) {
        A e;
        e.x = a.re[c];
        e.y = a.im[c];
        tab[c] = e;
    }
    __syncthreads();
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < a.N; i0 += T * kDiagUnroll) {
        int c[kDiagUnroll];
        A v[kDiagUnroll];
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) {
            const int64_t i = i0 + u * T;
            int cc = -1;
            if (i < a.N && DIAQ_BOUNDS_OK(i, a.N, BS_APPLY_DIAG)) {
                cc = 0;
                for (int q = 0; q < a.k; ++q) cc = (cc << 1) | int((i >> a.t[q]) & 1);
                if (((a.one >> cc) & 1) && INPLACE) cc = -1;  // unchanged: no read, no write
            }
            c[u] = cc;
            if (cc >= 0) v[u] = ld_stream(x + i);
        }
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) {
            if (c[u] < 0) continue;
            const int64_t i = i0 + u * T;
            if ((a.one >> c[u]) & 1) {  // out of place only
                st_stream(y + i, v[u]);
                continue;
            }
            const A m = tab[c[u]];
            const R mr = m.x, mi = m.y;
            A o;
            o.x = mr * v[u].x;
            o.x = fma(-mi, v[u].y, o.x);
            o.y = mr * v[u].y;
            o.y = fma(mi, v[u].x, o.y);
            st_stream(y + i, o);
        }
    }
}

template <typename R>
diaq_status launch_diag_t(int n, const GateDesc& g, const void* x, void* y, cudaStream_t s) {
    DiagArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.N = int64_t(1) << n;
    a.k = g.k;
    const int D = 1 << g.k;
    for (int q = 0; q < g.k; ++q) a.t[q] = g.targets[q];
    for (int c = 0; c < D; ++c) {
        a.re[c] = R(g.m[size_t(c) * D + c].real());
        a.im[c] = R(g.m[size_t(c) * D + c].imag());
        if (a.re[c] == R(1) && a.im[c] == R(0)) a.one |= uint64_t(1) << c;
    }
    const int64_t want = (a.N + 256 * kDiagUnroll - 1) / (256 * kDiagUnroll);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 16));
    DIAQ_PRELAUNCH("k_apply_diag");
    if (x == y)
        k_apply_diag<R, true><<<blocks, 256, 0, s>>>(reinterpret_cast<const amp_t<R>*>(x), reinterpret_cast<amp_t<R>*>(y), a);
    else
        k_apply_diag<R, false><<<blocks, 256, 0, s>>>(reinterpret_cast<const amp_t<R>*>(x), reinterpret_cast<amp_t<R>*>(y), a);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

// A diagonal over up to DIAG_BIG_K qubits from a table in device memory:
// diaq_simulate merges runs of consecutive diagonal ops (a QFT's controlled
// phases, a TFIM layer's ZZ rotations) into one such pass when their union
// of targets is small enough, so each amplitude takes one complex multiply
// for the whole run instead of one per op. Row i's entry is table[c],
// c = sum_q (bit t[q] of i) << q; rows whose entry is exactly 1 (bit set in
// skip) are neither read nor written. In place.
template <typename R>
__global__ void __launch_bounds__(256) k_apply_bigdiag(amp_t<R>* x, int64_t N, const __grid_constant__ BigDiagArgs a,
                                                       const double2* __restrict__ table,
                                                       const uint32_t* __restrict__ skip) {
    using A = amp_t<R>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int E = 1 << a.k;
    A* tab = reinterpret_cast<A*>(smem);
    uint32_t* sk = reinterpret_cast<uint32_t*>(smem + sizeof(A) * size_t(E));
    for (int c = threadIdx.x; c < E; c += blockDim.x) {
        const double2 v = table[c];
        A e;
        e.x = R(v.x);
        e.y = R(v.y);
        tab[c] = e;
    }
    for (int w = threadIdx.x; w < (E + 31) / 32; w += blockDim.x) sk[w] = skip[w];
    __syncthreads();
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < N; i0 += T * kDiagUnroll) {
        int c[kDiagUnroll];
        A v[kDiagUnroll];
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) {
            const int64_t i = i0 + u * T;
            int cc = -1;
            if (i < N && DIAQ_BOUNDS_OK(i, N, BS_APPLY_DIAG)) {
                cc = 0;
                for (int q = 0; q < a.k; ++q) cc |= int((i >> a.t[q]) & 1) << q;
                if ((sk[cc >> 5] >> (cc & 31)) & 1) cc = -1;  // entry exactly 1: untouched
            }
            c[u] = cc;
            if (cc >= 0) v[u] = ld_stream(x + i);
        }
#pragma unroll
        for (int u = 0; u < kDiagUnroll; ++u) {
            if (c[u] < 0) continue;
            const A m = tab[c[u]];
            A o;
            o.x = m.x * v[u].x;
            o.x = fma(-m.y, v[u].y, o.x);
            o.y = m.x * v[u].y;
            o.y = fma(m.y, v[u].x, o.y);
            st_stream(x + i0 + u * T, o);
        }
    }
}

}  // namespace

diaq_status launch_bigdiag_inplace(int n, diaq_dtype dt, const BigDiagArgs& a, const double2* table,
                                   const uint32_t* skip, void* x, cudaStream_t s) {
    if (a.k < 1 || a.k > DIAG_BIG_K) return fail(DIAQ_ERR_ARG, "merged diagonal over %d qubits", a.k);
    const int64_t N = int64_t(1) << n;
    const size_t E = size_t(1) << a.k;
    const size_t smem = (dt == DIAQ_C128 ? 16 : 8) * E + 4 * ((E + 31) / 32);
    const int64_t want = (N + 256 * kDiagUnroll - 1) / (256 * kDiagUnroll);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 6));
    DIAQ_PRELAUNCH("k_apply_bigdiag");
    if (dt == DIAQ_C128)
        k_apply_bigdiag<double><<<blocks, 256, smem, s>>>(reinterpret_cast<double2*>(x), N, a, table, skip);
    else
        k_apply_bigdiag<float><<<blocks, 256, smem, s>>>(reinterpret_cast<float2*>(x), N, a, table, skip);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

bool is_diagonal(const GateDesc& g) {
    const int D = 1 << g.k;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            if (r != c && g.m[size_t(r) * D + c] != cplx(0, 0)) return false;
    return true;
}

int64_t diag_inplace_bytes(int n, diaq_dtype dt, const GateDesc& g) {
    const int D = 1 << g.k;
    int64_t changed = 0;
    for (int c = 0; c < D; ++c) {
        const cplx v = g.m[size_t(c) * D + c];
        const bool one = dt == DIAQ_C128 ? (v.real() == 1.0 && v.imag() == 0.0)
                                         : (float(v.real()) == 1.0f && float(v.imag()) == 0.0f);
        if (!one) ++changed;
    }
    return 2 * (int64_t(1) << (n - g.k)) * changed * int64_t(amp_bytes(dt));
}

diaq_status launch_diag(int n, diaq_dtype dt, const GateDesc& g, const void* x, void* y, cudaStream_t s) {
    return dt == DIAQ_C128 ? launch_diag_t<double>(n, g, x, y, s) : launch_diag_t<float>(n, g, x, y, s);
}

}  // namespace diaq
