// In-place on-the-fly apply that skips identity rows.
//
// A time-step unitary I_above (x) M (x) I_below (Section II-C) changes only
// the rows whose local row of M differs from the identity: a controlled
// phase or CZ changes one local row in four, a CNOT or SWAP two in four
// (Section III-A: many gates are diagonal or permutations). When the op runs
// in place (y == x), a row whose local row of M is exactly e_r keeps its
// amplitude, so it needs neither a read nor a write. This kernel reads the
// local columns that the changed rows use and writes the changed rows only.
// It does the same arithmetic, in the same order, as the full kernel for
// those rows, so the state it leaves is bit-identical to the full kernel's.
//
// Algorithmic bytes per launch: 2^(n-k) groups x (columns read + rows
// written) x bytes per amplitude.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "bounds.cuh"
#include "common.cuh"
#include "internal.h"

DIAQ_BOUNDS_TU(inplace)

namespace diaq {

template <typename R, int K>
struct RowsArgs {
    int64_t g_base;         // first group of the launch
    int64_t n_groups;       // one past the last group
    int64_t N;              // amplitudes of the state
    int st[K];              // targets, ascending
    int64_t off[1 << K];    // full-system offset of local index c
    uint32_t ld_mask;       // local columns read by the changed rows
    uint32_t st_mask;       // local rows that differ from the identity
    R re[1 << (2 * K)];
    R im[1 << (2 * K)];
    uint8_t type[1 << (2 * K)];
};

template <typename R, int K, int G>
__global__ void __launch_bounds__(256)
k_apply_rows(amp_t<R>* x, const __grid_constant__ RowsArgs<R, K> a) {
    constexpr int D = 1 << K;
    using A = amp_t<R>;
    const int64_t T = blockDim.x;
    const int64_t g0 = a.g_base + (int64_t)blockIdx.x * T * G + threadIdx.x;
    A v[G][D];
    int64_t b[G];
    // every load of a group precedes its stores: the group is read whole
    // (the columns it needs) into registers before any row is written
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const int64_t g = g0 + j * T;
        b[j] = g < a.n_groups ? insert_zeros<K>(g, a.st) : int64_t(-1);
        if (b[j] >= 0 && !DIAQ_BOUNDS_OK(b[j] + a.off[D - 1], a.N, BS_APPLY_ROWS)) b[j] = -1;
        if (b[j] >= 0) {
#pragma unroll
            for (int c = 0; c < D; ++c)
                if ((a.ld_mask >> c) & 1u) v[j][c] = ld_stream(x + b[j] + a.off[c]);
        }
    }
#pragma unroll
    for (int j = 0; j < G; ++j) {
        if (b[j] < 0) continue;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            if (!((a.st_mask >> r) & 1u)) continue;
            A acc;
            acc.x = R(0);
            acc.y = R(0);
            bool first = true;
#pragma unroll
            for (int c = 0; c < D; ++c)
                if ((a.ld_mask >> c) & 1u)
                    mac_typed<R>(acc, first, a.type[r * D + c], a.re[r * D + c], a.im[r * D + c], v[j][c]);
            st_stream(x + b[j] + a.off[r], acc);
        }
    }
}

// Entry types of the local matrix after rounding to the op's precision.
static void rounded_types(const GateDesc& g, diaq_dtype dt, uint8_t* type) {
    const int DD = 1 << (2 * g.k);
    for (int e = 0; e < DD; ++e) {
        const cplx v = g.m[e];
        type[e] = dt == DIAQ_C128 ? entry_type(v) : entry_type(cplx(double(float(v.real())), double(float(v.imag()))));
    }
}

void inplace_masks(const GateDesc& g, diaq_dtype dt, uint32_t* ld_mask, uint32_t* st_mask) {
    const int D = 1 << g.k;
    uint8_t type[1 << (2 * DIAQ_MAX_K)];
    rounded_types(g, dt, type);
    uint32_t ld = 0, st = 0;
    for (int r = 0; r < D && g.k <= 3; ++r) {
        bool ident = true;
        for (int c = 0; c < D; ++c) {
            const uint8_t t = type[r * D + c];
            if (c == r ? t != ET_ONE : t != ET_ZERO) ident = false;
        }
        if (ident) continue;
        st |= 1u << r;
        for (int c = 0; c < D; ++c)
            if (type[r * D + c] != ET_ZERO) ld |= 1u << c;
    }
    if (g.k > 3) {
        ld = st = 0xffffffffu;  // the rows kernel covers k <= 3 only
    }
    *ld_mask = ld;
    *st_mask = st;
}

int64_t inplace_bytes(int n, diaq_dtype dt, const GateDesc& g) {
    const int64_t N = int64_t(1) << n;
    const int64_t s = int64_t(amp_bytes(dt));
    if (g.k > 3) return is_diagonal(g) ? diag_inplace_bytes(n, dt, g) : 2 * N * s;
    uint32_t ld, st;
    inplace_masks(g, dt, &ld, &st);
    const uint32_t full = (1u << (1 << g.k)) - 1u;
    if (st == full) return 2 * N * s;  // no identity row: the full kernel runs
    return (N >> g.k) * int64_t(__builtin_popcount(ld) + __builtin_popcount(st)) * s;
}

template <typename R, int K, int G>
static diaq_status launch_rows_G(int n, const GateDesc& g, uint32_t ld, uint32_t stm, void* x, int64_t g_begin,
                                 int64_t g_end, cudaStream_t s) {
    RowsArgs<R, K> a;
    std::memset(&a, 0, sizeof(a));
    a.g_base = g_begin;
    a.n_groups = g_end;
    a.N = int64_t(1) << n;
    for (int i = 0; i < K; ++i) a.st[i] = g.targets[i];
    std::sort(a.st, a.st + K);
    for (int c = 0; c < (1 << K); ++c) {
        int64_t o = 0;
        for (int i = 0; i < K; ++i)
            if ((c >> (K - 1 - i)) & 1) o += int64_t(1) << g.targets[i];
        a.off[c] = o;
    }
    a.ld_mask = ld;
    a.st_mask = stm;
    constexpr int DD = 1 << (2 * K);
    for (int e = 0; e < DD; ++e) {
        a.re[e] = R(g.m[e].real());
        a.im[e] = R(g.m[e].imag());
        a.type[e] = entry_type(cplx(double(a.re[e]), double(a.im[e])));
    }
    const int threads = 256;
    const int64_t per_block = int64_t(threads) * G;
    const int64_t blocks = (g_end - g_begin + per_block - 1) / per_block;
    if (blocks <= 0) return DIAQ_OK;
    DIAQ_PRELAUNCH("k_apply_rows");
    k_apply_rows<R, K, G><<<dim3((unsigned)blocks), threads, 0, s>>>(reinterpret_cast<amp_t<R>*>(x), a);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

template <typename R>
static diaq_status launch_rows(int n, const GateDesc& g, uint32_t ld, uint32_t st, void* x, int64_t g_begin,
                               int64_t g_end, cudaStream_t s) {
    // groups per thread: enough independent loads in flight, registers bounded
    constexpr bool dbl = sizeof(R) == 8;
    switch (g.k) {
        case 1: return launch_rows_G<R, 1, 4>(n, g, ld, st, x, g_begin, g_end, s);
        case 2: return launch_rows_G<R, 2, dbl ? 2 : 4>(n, g, ld, st, x, g_begin, g_end, s);
        default: return launch_rows_G<R, 3, dbl ? 1 : 2>(n, g, ld, st, x, g_begin, g_end, s);
    }
}

diaq_status launch_inplace_skip(const diaq_op_s* op, void* x, cudaStream_t s, bool* launched) {
    return op->gate.k >= 1 && op->gate.k <= 3
               ? launch_inplace_skip_range(op, x, 0, int64_t(1) << (op->n - op->gate.k), s, launched)
               : launch_inplace_skip_range(op, x, 0, 0, s, launched);
}

diaq_status launch_inplace_skip_range(const diaq_op_s* op, void* x, int64_t g_begin, int64_t g_end, cudaStream_t s,
                                      bool* launched) {
    *launched = false;
    if (op->variant != DIAQ_ONTHEFLY || op->op_class == DIAQ_CLASS_RAW || op->gate.k > 3) return DIAQ_OK;
    uint32_t ld, st;
    inplace_masks(op->gate, op->dtype, &ld, &st);
    const uint32_t full = (1u << (1 << op->gate.k)) - 1u;
    if (st == full) return DIAQ_OK;  // every row changes: the full kernel is the right one
    *launched = true;
    if (st == 0) return DIAQ_OK;     // the identity: nothing changes in place
    return op->dtype == DIAQ_C128 ? launch_rows<double>(op->n, op->gate, ld, st, x, g_begin, g_end, s)
                                  : launch_rows<float>(op->n, op->gate, ld, st, x, g_begin, g_end, s);
}

}  // namespace diaq
