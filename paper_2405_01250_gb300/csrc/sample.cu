// Shots: Born-rule sampling of basis states from a device state (the
// measurement behind a run's shots; Section VII runs every benchmark for
// 1024 shots). Outcome i is drawn with probability |psi_i|^2 / ||psi||^2 by
// the inverse of the cumulative distribution in index order, one caller
// uniform u per shot: the smallest i whose running sum of |psi|^2 exceeds
// r = u * ||psi||^2.
//
// No cumulative array of N entries is written. One pass over the state
// builds a tree of sums in which every node is the SEQUENTIAL sum, in index
// order, of its children, and stores each group of siblings as inclusive
// running sums (prefixes):
//   run    16 consecutive amplitudes                (one thread; not stored)
//   seg    16 runs = 256 amplitudes                 (run prefixes stored)
//   tile   16 segs = 4096 amplitudes, one block     (seg prefixes stored)
//   level  groups of 256 nodes of the level below   (prefixes stored, up to one node)
// A shot descends from the total: in each group it binary-searches the
// first prefix that exceeds its remaining r, subtracts the prefix before it,
// and finally walks the 16 amplitudes of one run with the same operation
// sequence as the tile pass, which reproduces the stored run prefix bit for
// bit. Prefixes are non-negative doubles, so they are compared as their
// 64-bit patterns on the integer pipe.
//
// Because every running sum is sequential, a child of zero total leaves its
// prefix unchanged, so a zero-probability outcome is never entered. When
// rounding leaves the remaining r at or above a group's last prefix (or
// u = 1), the descent takes the group's last child of non-zero total, then
// the last one below that, and so on: the outcome still has non-zero
// probability.
//
// Cost. complex128 accumulates re^2 then im^2 with FP64 fused multiply-adds
// (two FP64 instructions per amplitude, the fewest for |psi|^2 in FP64);
// complex64 keeps each run as an unevaluated FP32 pair hi + lo fed with the
// exact squares (two-product and two-sum, about 48 bits), converted to FP64
// once per run. The sequential sums above the runs are done by one thread
// per group, so a tile spends 32 warp-wide FP64 additions on them, not one
// per lane: on this GPU a warp-wide FP64 instruction occupies the SM's FP64
// pipe for about 19 cycles whatever its active mask.

#include <cuda_runtime.h>

#include <algorithm>

#include "bounds.cuh"
#include "common.cuh"
#include "internal.h"

DIAQ_BOUNDS_TU(sample)

namespace diaq {
namespace {

constexpr int kRun = 16;                  // amplitudes per run
constexpr int kSegRuns = 16;              // runs per seg
constexpr int kTileSegs = 16;             // segs per tile
constexpr int kTileRuns = kSegRuns * kTileSegs;   // 256 runs: one per thread
constexpr int kTile = kRun * kTileRuns;   // 4096 amplitudes
constexpr int kWarpRuns = 32;             // runs staged by one warp
constexpr int kFan = 256;                 // group size above the tiles
constexpr int kMaxLevels = 8;             // 2^34 / 4096 = 2^22 tiles -> 4 levels

// Running sum of |psi_i|^2 over one run, in one fixed operation sequence
// shared by the tile pass and the descent.
template <typename R>
struct RunSum;

template <>
struct RunSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double2 v) {
        s = __fma_rn(v.x, v.x, s);
        s = __fma_rn(v.y, v.y, s);
    }
    __device__ __forceinline__ double value() const { return s; }
};

template <>
struct RunSum<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add1(float a) {
        const float p = __fmul_rn(a, a);
        const float e = __fmaf_rn(a, a, -p);  // a^2 = p + e exactly
        const float t = __fadd_rn(hi, p);     // hi + p = t + err exactly (two-sum)
        const float bb = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(p, bb));
        hi = t;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ void add(float2 v) {
        add1(v.x);
        add1(v.y);
    }
    __device__ __forceinline__ double value() const { return __dadd_rn(double(hi), double(lo)); }
};

template <typename R>
__device__ __forceinline__ amp_t<R> zero_amp();
template <>
__device__ __forceinline__ double2 zero_amp<double>() { return make_double2(0.0, 0.0); }
template <>
__device__ __forceinline__ float2 zero_amp<float>() { return make_float2(0.0f, 0.0f); }

// Ordering of non-negative doubles by their bit patterns.
__device__ __forceinline__ long long key(double v) { return __double_as_longlong(v); }

// Running sums of 16 values in place, sequential from acc: loads first, then
// the chain of additions in registers, then the stores.
__device__ __forceinline__ double prefix16(double* v, double acc) {
    double x[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) x[t] = v[t];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        acc = __dadd_rn(acc, x[t]);
        x[t] = acc;
    }
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = x[t];
    return acc;
}

// Half a run per staging pass.
constexpr int kHalf = kRun / 2;

template <typename R>
constexpr int tile_smem_bytes() {
    return 8 * kWarpRuns * (kHalf + 1) * int(sizeof(amp_t<R>));
}

// ---------------------------------------------------------------------------
// Tile pass: one block of 256 threads per 4096 amplitudes; warp w owns runs
// 32 w .. 32 w + 31, lane l run 32 w + l. In two passes the warp stages the
// first and then the second half of each of its runs in shared memory (load
// j covers 4 runs, 8 consecutive amplitudes of each: four whole 128-byte
// segments; one padding amplitude per run keeps the per-lane reads free of
// bank conflicts), and each lane continues its run's sum over the 8 staged
// amplitudes, so the sum is sequential in index order as before. Staging
// half runs halves the shared memory per block, so twice as many blocks
// fit on an SM. Threads 0..15 then form the run prefixes of seg t, thread 0
// the seg prefixes of the tile.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_sample_tiles(const amp_t<R>* __restrict__ psi, int64_t N,
                                                      double* __restrict__ run_pre, double* __restrict__ seg_pre,
                                                      double* __restrict__ tile_tot) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using A = amp_t<R>;
    A(*stage)[kWarpRuns][kHalf + 1] = reinterpret_cast<A(*)[kWarpRuns][kHalf + 1]>(smem_raw);
    __shared__ double rp[kTileRuns];
    __shared__ double sp[kTileSegs];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)warp * (kWarpRuns * kRun);
    RunSum<R> rs;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        // load j: runs 4 j + lane / 8, amplitude half * 8 + lane % 8 of each;
        // all 8 loads in flight before the first shared-memory store
        A v[kHalf];
#pragma unroll
        for (int j = 0; j < kHalf; ++j) {
            const int64_t i = base + int64_t(kRun) * (4 * j + lane / kHalf) + half * kHalf + lane % kHalf;
            v[j] = i < N && DIAQ_BOUNDS_OK(i, N, BS_SAMPLE_TILES) ? ld_stream(psi + i) : zero_amp<R>();
        }
        if (half) __syncwarp();  // every lane has read the first half
#pragma unroll
        for (int j = 0; j < kHalf; ++j) stage[warp][4 * j + lane / kHalf][lane % kHalf] = v[j];
        __syncwarp();
#pragma unroll
        for (int e = 0; e < kHalf; ++e) rs.add(stage[warp][lane][e]);
    }
    rp[threadIdx.x] = rs.value();
    __syncthreads();
    static_assert(kSegRuns == 16 && kTileSegs == 16, "prefix16 walks groups of 16");
    if (threadIdx.x < kTileSegs) sp[threadIdx.x] = prefix16(rp + threadIdx.x * kSegRuns, 0.0);
    __syncthreads();
    run_pre[(int64_t)blockIdx.x * kTileRuns + threadIdx.x] = rp[threadIdx.x];
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = prefix16(sp, 0.0);
    __syncthreads();
    if (threadIdx.x < kTileSegs) seg_pre[(int64_t)blockIdx.x * kTileSegs + threadIdx.x] = sp[threadIdx.x];
}

// One level up: group j of 256 values becomes their running sums (pre) and
// its total (parent[j]). One block per group, coalesced loads.
__global__ void __launch_bounds__(256) k_sample_level(const double* __restrict__ child, int64_t n_child,
                                                      double* __restrict__ pre, double* __restrict__ parent) {
    __shared__ double v[kFan];
    const int64_t c = (int64_t)blockIdx.x * kFan + threadIdx.x;
    v[threadIdx.x] = c < n_child ? child[c] : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        // values past the end are 0 and leave the running sum unchanged
        double acc = 0.0;
        for (int t = 0; t < kFan; t += 16) acc = prefix16(v + t, acc);
        parent[blockIdx.x] = acc;
    }
    __syncthreads();
    if (c < n_child) pre[c] = v[threadIdx.x];
}

struct Levels {
    const double* pre[kMaxLevels];  // pre[L]: running sums of level L within groups of 256
    int64_t count[kMaxLevels];      // nodes at level L (level 0: tiles); count[m-1] == 1
    const double* total;            // the single node above level m-2 (or the tile total if m == 1)
    const double* run_pre;          // per tile: 256 run prefixes (within segs)
    const double* seg_pre;          // per tile: 16 seg prefixes
    int m;
};

// In the running sums pre[b .. e) (non-decreasing, pre[e-1] the group total):
// the first position whose running sum exceeds r, or - when none does, and
// whenever take_last is set - the position where the running sum last
// increased (the last child of non-zero total); -1 if the group total is 0.
// r becomes the remainder past the positions before the chosen one.
__device__ int64_t pick(const double* __restrict__ pre, int64_t b, int64_t e, double& r, bool& take_last) {
    const long long last = key(pre[e - 1]);
    if (last == 0) return -1;
    int64_t lo = b, hi = e - 1;
    if (!take_last && key(r) < last) {  // smallest c with pre[c] > r
        const long long kr = key(r);
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (key(pre[mid]) > kr)
                hi = mid;
            else
                lo = mid + 1;
        }
    } else {  // smallest c with pre[c] == pre[e-1]
        take_last = true;
        while (lo < hi) {
            const int64_t mid = lo + ((hi - lo) >> 1);
            if (key(pre[mid]) >= last)
                hi = mid;
            else
                lo = mid + 1;
        }
    }
    if (lo > b) r = __dsub_rn(r, pre[lo - 1]);
    return lo;
}

// One thread per shot.
template <typename R>
__global__ void __launch_bounds__(128) k_sample_search(const amp_t<R>* __restrict__ psi, int64_t N, Levels lv,
                                                       const double* __restrict__ uniforms, int64_t shots,
                                                       int64_t* __restrict__ out) {
    const int64_t shot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (shot >= shots) return;
    double u = uniforms[shot];
    if (!(u > 0.0)) u = 0.0;  // also maps NaN to 0
    if (u > 1.0) u = 1.0;
    double r = __dmul_rn(u, *lv.total);
    bool take_last = false;
    int64_t node = 0, idx = -1;
    for (int L = lv.m - 2; L >= 0 && node >= 0; --L) {
        const int64_t b = node * kFan;
        const int64_t e = b + kFan < lv.count[L] ? b + kFan : lv.count[L];
        node = pick(lv.pre[L], b, e, r, take_last);
    }
    if (node >= 0 && !DIAQ_BOUNDS_OK(node, lv.count[0], BS_SAMPLE_SEARCH)) node = -1;
    if (node >= 0) {  // node: the tile
        const int64_t seg = pick(lv.seg_pre + node * kTileSegs, 0, kTileSegs, r, take_last);
        if (seg >= 0) {
            const double* rpre = lv.run_pre + node * kTileRuns + seg * kSegRuns;
            const int64_t run = pick(rpre, 0, kSegRuns, r, take_last);
            if (run >= 0) {
                const int64_t first = node * kTile + (seg * kSegRuns + run) * kRun;
                RunSum<R> rs;
                long long prev = 0;
                int last_e = -1;
                const long long kr = key(r);
                for (int e = 0; e < kRun; ++e) {
                    rs.add(first + e < N ? psi[first + e] : zero_amp<R>());
                    const long long cur = key(rs.value());
                    if (!take_last && cur > kr) {
                        idx = first + e;
                        break;
                    }
                    if (cur > prev) last_e = e;
                    prev = cur;
                }
                if (idx < 0 && last_e >= 0) idx = first + last_e;
            }
        }
    }
    out[shot] = idx;
}

}  // namespace
}  // namespace diaq

using namespace diaq;

extern "C" diaq_status diaq_sample(const void* psi, int32_t n_qubits, diaq_dtype dtype, const double* uniforms,
                                   int64_t n_shots, int64_t* out_indices, diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();  // discard a non-sticky error left by the caller's own calls
    if (!psi) return fail(DIAQ_ERR_ARG, "state is NULL");
    if (n_qubits < 1 || n_qubits > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_qubits = %d out of range", n_qubits);
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (reinterpret_cast<uintptr_t>(psi) & 15) return fail(DIAQ_ERR_ARG, "state buffer must be 16-byte aligned");
    if (n_shots < 0 || n_shots > (int64_t(1) << 31)) return fail(DIAQ_ERR_ARG, "n_shots = %lld out of range [0, 2^31]", (long long)n_shots);
    if (n_shots == 0) return DIAQ_OK;
    if (!uniforms || !out_indices) return fail(DIAQ_ERR_ARG, "uniforms or out_indices is NULL");
    if ((reinterpret_cast<uintptr_t>(uniforms) | reinterpret_cast<uintptr_t>(out_indices)) & 7)
        return fail(DIAQ_ERR_ARG, "uniforms and out_indices must be 8-byte aligned");
    const int64_t N = int64_t(1) << n_qubits;
    const int64_t tiles = (N + kTile - 1) / kTile;
    // scratch: run prefixes, seg prefixes, then per level its running sums
    // and the totals of its groups (the next level's nodes)
    Levels lv{};
    int64_t count[kMaxLevels + 1];
    int m = 0;
    for (int64_t c = tiles;; c = (c + kFan - 1) / kFan) {
        count[m++] = c;
        if (c == 1) break;
    }
    int64_t total_doubles = tiles * (kTileRuns + kTileSegs) + count[0];
    for (int L = 0; L + 1 < m; ++L) total_doubles += count[L] + count[L + 1];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, sizeof(double) * total_doubles, s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(sample tree, %lld doubles): %s",
                                      (long long)total_doubles, cudaGetErrorString(e));
    double* run_pre = scratch;
    double* seg_pre = run_pre + tiles * kTileRuns;
    double* node_tot = seg_pre + tiles * kTileSegs;  // level 0 totals (tiles)
    double* cursor = node_tot + count[0];
    lv.m = m;
    lv.run_pre = run_pre;
    lv.seg_pre = seg_pre;
    for (int L = 0; L < m; ++L) lv.count[L] = count[L];
    const double* level_tot = node_tot;
    diaq_status st = DIAQ_OK;
    if (dtype == DIAQ_C128) {
        constexpr int sm = tile_smem_bytes<double>();
        e = cudaFuncSetAttribute(k_sample_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess)
            k_sample_tiles<double><<<(unsigned)tiles, 256, sm, s>>>(reinterpret_cast<const double2*>(psi), N, run_pre,
                                                                     seg_pre, node_tot);
    } else {
        constexpr int sm = tile_smem_bytes<float>();
        e = cudaFuncSetAttribute(k_sample_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e == cudaSuccess)
            k_sample_tiles<float><<<(unsigned)tiles, 256, sm, s>>>(reinterpret_cast<const float2*>(psi), N, run_pre,
                                                                    seg_pre, node_tot);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    for (int L = 0; L + 1 < m && e == cudaSuccess; ++L) {
        double* pre = cursor;
        double* parent = cursor + count[L];
        cursor = parent + count[L + 1];
        k_sample_level<<<(unsigned)count[L + 1], kFan, 0, s>>>(level_tot, count[L], pre, parent);
        e = cudaGetLastError();
        lv.pre[L] = pre;
        level_tot = parent;
    }
    lv.total = level_tot;
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n_shots + 127) / 128);
        if (dtype == DIAQ_C128)
            k_sample_search<double><<<blocks, 128, 0, s>>>(reinterpret_cast<const double2*>(psi), N, lv, uniforms,
                                                           n_shots, out_indices);
        else
            k_sample_search<float><<<blocks, 128, 0, s>>>(reinterpret_cast<const float2*>(psi), N, lv, uniforms,
                                                          n_shots, out_indices);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_fail(e, "sampling kernels");
    cudaFreeAsync(scratch, s);
    return st;
}
