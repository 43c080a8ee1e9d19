// Shots: Born-rule sampling of basis states from a device state (the
// measurement behind a run's shots; Section VII runs every benchmark for
// 1024 shots). Outcome i is drawn with probability |psi_i|^2 / ||psi||^2 by
// the inverse of the cumulative distribution in index order, one caller
// uniform u per shot: the smallest i whose running sum of |psi|^2 exceeds
// r = u * ||psi||^2.
//
// No cumulative array is written. The state is read once to build a sum
// tree of fixed fan-out whose every node is the SEQUENTIAL sum, in index
// order, of its children:
//   run   16 consecutive amplitudes            (one thread)
//   seg   32 runs = 512 amplitudes             (one warp)
//   tile  4 segs  = 2048 amplitudes            (one block; totals stored)
//   level 256 nodes of the level below         (stored, up to the single total)
// A shot then descends from the total: at each node it walks the children's
// running sum and enters the first child whose running sum exceeds the
// shot's remaining r, subtracting the sum before it. Inside a tile the seg,
// run and amplitude sums are recomputed with the same operation sequence as
// the tile pass, so they reproduce its totals bit for bit.
//
// Because every running sum is sequential, a child of zero total leaves it
// unchanged, so a zero-probability outcome is never entered. When rounding
// leaves the remaining r at or above a node's own total (or u = 1), the
// descent takes the node's last child of non-zero total, then the last one
// below that, and so on: the outcome still has non-zero probability.
//
// Sums: complex128 accumulates re^2 then im^2 with FP64 fused multiply-adds
// (two FP64 instructions per amplitude, the fewest for |psi|^2 in FP64);
// complex64 keeps each run as an unevaluated FP32 pair hi + lo fed with the
// exact squares (two-product and two-sum, about 48 bits), converted to FP64
// once per run, so the FP64 pipe is not used per amplitude.

#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace diaq {
namespace {

constexpr int kRun = 16;                            // amplitudes per run
constexpr int kSegRuns = 32;                        // runs per seg (one per lane)
constexpr int kSeg = kRun * kSegRuns;               // 512 amplitudes
constexpr int kTileSegs = 4;                        // segs per tile (one per warp)
constexpr int kTile = kSeg * kTileSegs;             // 2048 amplitudes
constexpr int kFan = 256;                           // children per node above the tiles
constexpr int kMaxLevels = 8;                       // 2^34 / 2048 = 2^23 tiles -> 4 levels
constexpr unsigned kFull = 0xffffffffu;

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

// Sequential sum over the warp's lanes, in lane order, of one value per
// lane; every lane gets the total.
__device__ __forceinline__ double lane_ordered_sum(double v) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < 32; ++l) s = __dadd_rn(s, __shfl_sync(kFull, v, l));
    return s;
}

// ---------------------------------------------------------------------------
// Tile pass: one block of 4 warps per 2048 amplitudes. Each warp stages its
// seg in shared memory with coalesced loads (one padding amplitude per run
// keeps the per-lane reads free of bank conflicts), then lane l sums run l.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(128) k_sample_tiles(const amp_t<R>* __restrict__ psi, int64_t N,
                                                      double* __restrict__ tile_tot) {
    __shared__ amp_t<R> stage[kTileSegs][kSegRuns][kRun + 1];
    __shared__ double seg_tot[kTileSegs];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t seg_base = (int64_t)blockIdx.x * kTile + (int64_t)warp * kSeg;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        const int g = 32 * j + lane;
        const int64_t i = seg_base + g;
        stage[warp][g / kRun][g % kRun] = i < N ? ld_stream(psi + i) : zero_amp<R>();
    }
    __syncwarp();
    RunSum<R> rs;
#pragma unroll
    for (int e = 0; e < kRun; ++e) rs.add(stage[warp][lane][e]);
    const double seg = lane_ordered_sum(rs.value());
    if (lane == 0) seg_tot[warp] = seg;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int s = 0; s < kTileSegs; ++s) t = __dadd_rn(t, seg_tot[s]);
        tile_tot[blockIdx.x] = t;
    }
}

// One level up: parent j = sequential sum of children [256 j, 256 j + 256).
__global__ void __launch_bounds__(128) k_sample_level(const double* __restrict__ child, int64_t n_child,
                                                      double* __restrict__ parent, int64_t n_parent) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_parent) return;
    const int64_t b = j * kFan, e = b + kFan < n_child ? b + kFan : n_child;
    double s = 0.0;
    for (int64_t c = b; c < e; ++c) s = __dadd_rn(s, child[c]);
    parent[j] = s;
}

struct Levels {
    const double* lv[kMaxLevels];  // lv[0]: tile totals ... lv[m-1]: the total (one node)
    int64_t count[kMaxLevels];
    int m;
};

// Among stored children [b, e): the first whose running sum exceeds r (r
// becomes the remainder past the children before it), else - and from then
// on, take_last - the last child of non-zero total. Warp-uniform: every
// lane walks the same sequence. Returns -1 if every child is zero.
__device__ int64_t pick_stored(const double* __restrict__ v, int64_t b, int64_t e, double& r, bool& take_last) {
    const int lane = threadIdx.x & 31;
    double prefix = 0.0;
    int64_t last_pos = -1;
    for (int64_t c0 = b; c0 < e; c0 += 32) {
        const int64_t c = c0 + lane;
        const double mine = c < e ? v[c] : 0.0;
        const unsigned pos = __ballot_sync(kFull, mine > 0.0);
        if (pos) last_pos = c0 + 31 - __clz((int)pos);
        if (take_last) continue;
        const int cnt = e - c0 < 32 ? (int)(e - c0) : 32;
        for (int k = 0; k < cnt; ++k) {
            const double x = __shfl_sync(kFull, mine, k);
            const double np = __dadd_rn(prefix, x);
            if (np > r) {
                r = __dsub_rn(r, prefix);
                return c0 + k;
            }
            prefix = np;
        }
    }
    take_last = true;
    return last_pos;
}

// Inside one tile: seg (recomputed), run (the lanes' run sums), amplitude.
template <typename R>
__device__ int64_t pick_in_tile(const amp_t<R>* __restrict__ psi, int64_t N, int64_t tile, double r,
                                bool take_last) {
    const int lane = threadIdx.x & 31;
    const int64_t tile_base = tile * kTile;
    // the seg: its lanes' run sums stay in registers once chosen
    double run = 0.0;
    int seg = -1;
    {
        double prefix = 0.0;
        int last_seg = -1;
        double last_run = 0.0;
        for (int s = 0; s < kTileSegs; ++s) {
            const int64_t base = tile_base + (int64_t)s * kSeg + (int64_t)lane * kRun;
            RunSum<R> rs;
            for (int e = 0; e < kRun; ++e) rs.add(base + e < N ? psi[base + e] : zero_amp<R>());
            const double my_run = rs.value();
            const double tot = lane_ordered_sum(my_run);
            if (tot > 0.0) {
                last_seg = s;
                last_run = my_run;
            }
            if (!take_last) {
                const double np = __dadd_rn(prefix, tot);
                if (np > r) {
                    r = __dsub_rn(r, prefix);
                    seg = s;
                    run = my_run;
                    break;
                }
                prefix = np;
            }
        }
        if (seg < 0) {
            take_last = true;
            seg = last_seg;
            run = last_run;
        }
    }
    if (seg < 0) return -1;
    // the run
    int L = -1;
    {
        double prefix = 0.0;
        int last_l = -1;
        for (int k = 0; k < 32; ++k) {
            const double x = __shfl_sync(kFull, run, k);
            if (x > 0.0) last_l = k;
            if (!take_last && L < 0) {
                const double np = __dadd_rn(prefix, x);
                if (np > r) {
                    r = __dsub_rn(r, prefix);
                    L = k;
                } else {
                    prefix = np;
                }
            }
        }
        if (L < 0) {
            take_last = true;
            L = last_l;
        }
    }
    if (L < 0) return -1;
    // the amplitude: the run's running sum, element by element
    const int64_t base = tile_base + (int64_t)seg * kSeg + (int64_t)L * kRun;
    RunSum<R> rs;
    double prev = 0.0;
    int last_e = -1;
    for (int e = 0; e < kRun; ++e) {
        rs.add(base + e < N ? psi[base + e] : zero_amp<R>());
        const double cur = rs.value();
        if (!take_last && cur > r) return base + e;
        if (cur > prev) last_e = e;
        prev = cur;
    }
    return last_e < 0 ? -1 : base + last_e;
}

// One warp per shot.
template <typename R>
__global__ void __launch_bounds__(128) k_sample_search(const amp_t<R>* __restrict__ psi, int64_t N, Levels lv,
                                                       const double* __restrict__ uniforms, int64_t shots,
                                                       int64_t* __restrict__ out) {
    const int64_t shot = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (shot >= shots) return;  // whole warps leave together
    double u = uniforms[shot];
    if (!(u > 0.0)) u = 0.0;  // also maps NaN to 0
    if (u > 1.0) u = 1.0;
    double r = __dmul_rn(u, lv.lv[lv.m - 1][0]);
    bool take_last = false;
    int64_t node = 0;
    for (int L = lv.m - 2; L >= 0; --L) {
        const int64_t b = node * kFan;
        const int64_t e = b + kFan < lv.count[L] ? b + kFan : lv.count[L];
        node = pick_stored(lv.lv[L], b, e, r, take_last);
        if (node < 0) break;
    }
    // with a single tile (lv.m == 1) the descent starts inside it
    const int64_t idx = node >= 0 ? pick_in_tile<R>(psi, N, node, r, take_last) : -1;
    if ((threadIdx.x & 31) == 0) out[shot] = idx;
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
    Levels lv{};
    int64_t off[kMaxLevels];
    int64_t total = 0;
    int64_t count = (N + kTile - 1) / kTile;
    lv.m = 0;
    for (;;) {
        lv.count[lv.m] = count;
        off[lv.m] = total;
        total += count;
        ++lv.m;
        if (count == 1) break;
        count = (count + kFan - 1) / kFan;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, sizeof(double) * total, s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(sample tree, %lld doubles): %s",
                                      (long long)total, cudaGetErrorString(e));
    for (int l = 0; l < lv.m; ++l) lv.lv[l] = scratch + off[l];
    diaq_status st = DIAQ_OK;
    if (dtype == DIAQ_C128)
        k_sample_tiles<double><<<(unsigned)lv.count[0], 128, 0, s>>>(reinterpret_cast<const double2*>(psi), N, scratch);
    else
        k_sample_tiles<float><<<(unsigned)lv.count[0], 128, 0, s>>>(reinterpret_cast<const float2*>(psi), N, scratch);
    e = cudaGetLastError();
    for (int l = 1; l < lv.m && e == cudaSuccess; ++l) {
        k_sample_level<<<(unsigned)((lv.count[l] + 127) / 128), 128, 0, s>>>(lv.lv[l - 1], lv.count[l - 1],
                                                                             scratch + off[l], lv.count[l]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n_shots + 3) / 4);
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
