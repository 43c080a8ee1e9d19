// Slice moves of the sharded state: a state vector larger than one device's
// memory is split across devices (Section II-A; Section VI names the
// multi-node backend, diaq-mpi), here over 2^g shards by the top g bits of
// the basis index. Exchanging global bit G of the shard index with local
// bit l moves, between the shard pair (s with bit G clear, s | 2^G), the
// amplitudes whose local bit l differs from the shard's bit G: the half of
// shard s with bit l = 1 trades places with the half of its partner with
// bit l = 0. Each half is N_local / 2 amplitudes in chunks of 2^l.
//
// k_shard_swap does the trade in place for two shards in one address space;
// k_shard_pack / k_shard_unpack gather a half into a contiguous buffer and
// scatter it back, for shards held by separate ranks that exchange the
// buffers (NCCL send/recv). Every kernel is a pure move: HBM-bound,
// 16 or 8 bytes read and written per amplitude moved.

#include <cuda_runtime.h>

#include <algorithm>

#include "bounds.cuh"
#include "common.cuh"
#include "internal.h"

DIAQ_BOUNDS_TU(shard)

namespace diaq {
namespace {

// Index with bit l equal to `value` and the other bits taken from t.
__device__ __forceinline__ int64_t with_bit(int64_t t, int l, int value) {
    const int64_t lo = t & ((int64_t(1) << l) - 1);
    return ((t - lo) << 1) | (int64_t(value) << l) | lo;
}

template <typename R>
__global__ void __launch_bounds__(256) k_shard_swap(amp_t<R>* __restrict__ lo_shard, amp_t<R>* __restrict__ hi_shard,
                                                    int64_t half, int l) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride) {
        const int64_t a = with_bit(t, l, 1), b = with_bit(t, l, 0);
        if (!DIAQ_BOUNDS_OK(a, 2 * half, BS_SHARD_MOVE)) continue;
        const amp_t<R> va = ld_stream(lo_shard + a);
        const amp_t<R> vb = ld_stream(hi_shard + b);
        st_stream(lo_shard + a, vb);
        st_stream(hi_shard + b, va);
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_shard_pack(const amp_t<R>* __restrict__ shard, amp_t<R>* __restrict__ buf,
                                                    int64_t half, int l, int value) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride)
        if (DIAQ_BOUNDS_OK(with_bit(t, l, value), 2 * half, BS_SHARD_MOVE))
            st_stream(buf + t, ld_stream(shard + with_bit(t, l, value)));
}

template <typename R>
__global__ void __launch_bounds__(256) k_shard_unpack(const amp_t<R>* __restrict__ buf, amp_t<R>* __restrict__ shard,
                                                      int64_t half, int l, int value) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride)
        if (DIAQ_BOUNDS_OK(with_bit(t, l, value), 2 * half, BS_SHARD_MOVE))
            st_stream(shard + with_bit(t, l, value), ld_stream(buf + t));
}

int move_blocks(int64_t half) {
    const int64_t want = (half + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 16));
}

diaq_status check_move(const void* a, int n_local, diaq_dtype dt, int l) {
    if (!a) return fail(DIAQ_ERR_ARG, "shard or buffer is NULL");
    if (n_local < 1 || n_local > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_local = %d out of range", n_local);
    if (dt != DIAQ_C64 && dt != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dt);
    if (l < 0 || l >= n_local) return fail(DIAQ_ERR_ARG, "local bit %d outside [0, %d)", l, n_local);
    if (reinterpret_cast<uintptr_t>(a) & 15) return fail(DIAQ_ERR_ARG, "shard buffers must be 16-byte aligned");
    return DIAQ_OK;
}

bool spans_overlap(const void* a, size_t a_bytes, const void* b, size_t b_bytes) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + b_bytes && y < x + a_bytes;
}

}  // namespace

diaq_status launch_shard_swap(void* lo, void* hi, int n_local, diaq_dtype dt, int l, cudaStream_t s) {
    const int64_t half = int64_t(1) << (n_local - 1);
    DIAQ_PRELAUNCH("k_shard_swap");
    if (dt == DIAQ_C128)
        k_shard_swap<double><<<move_blocks(half), 256, 0, s>>>(static_cast<double2*>(lo), static_cast<double2*>(hi), half, l);
    else
        k_shard_swap<float><<<move_blocks(half), 256, 0, s>>>(static_cast<float2*>(lo), static_cast<float2*>(hi), half, l);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

}  // namespace diaq

using namespace diaq;

extern "C" diaq_status diaq_shard_swap(void* lo_shard, void* hi_shard, int32_t n_local, diaq_dtype dtype,
                                       int32_t local_bit, diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    DIAQ_TRY(check_move(lo_shard, n_local, dtype, local_bit));
    DIAQ_TRY(check_move(hi_shard, n_local, dtype, local_bit));
    const size_t bytes = (size_t(1) << n_local) * amp_bytes(dtype);
    if (spans_overlap(lo_shard, bytes, hi_shard, bytes))
        return fail(DIAQ_ERR_ARG, "the two shards overlap");
    return launch_shard_swap(lo_shard, hi_shard, n_local, dtype, local_bit, static_cast<cudaStream_t>(stream));
}

extern "C" diaq_status diaq_shard_pack(const void* shard, int32_t n_local, diaq_dtype dtype, int32_t local_bit,
                                       int32_t value, void* buf, diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    DIAQ_TRY(check_move(shard, n_local, dtype, local_bit));
    DIAQ_TRY(check_move(buf, n_local, dtype, local_bit));
    if (value != 0 && value != 1) return fail(DIAQ_ERR_ARG, "value must be 0 or 1");
    const int64_t half = int64_t(1) << (n_local - 1);
    if (spans_overlap(shard, size_t(2 * half) * amp_bytes(dtype), buf, size_t(half) * amp_bytes(dtype)))
        return fail(DIAQ_ERR_ARG, "shard and buffer overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DIAQ_PRELAUNCH("k_shard_pack");
    if (dtype == DIAQ_C128)
        k_shard_pack<double><<<move_blocks(half), 256, 0, s>>>(static_cast<const double2*>(shard), static_cast<double2*>(buf),
                                                               half, local_bit, value);
    else
        k_shard_pack<float><<<move_blocks(half), 256, 0, s>>>(static_cast<const float2*>(shard), static_cast<float2*>(buf),
                                                              half, local_bit, value);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

extern "C" diaq_status diaq_shard_unpack(const void* buf, void* shard, int32_t n_local, diaq_dtype dtype,
                                         int32_t local_bit, int32_t value, diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    DIAQ_TRY(check_move(shard, n_local, dtype, local_bit));
    DIAQ_TRY(check_move(buf, n_local, dtype, local_bit));
    if (value != 0 && value != 1) return fail(DIAQ_ERR_ARG, "value must be 0 or 1");
    const int64_t half = int64_t(1) << (n_local - 1);
    if (spans_overlap(shard, size_t(2 * half) * amp_bytes(dtype), buf, size_t(half) * amp_bytes(dtype)))
        return fail(DIAQ_ERR_ARG, "shard and buffer overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DIAQ_PRELAUNCH("k_shard_unpack");
    if (dtype == DIAQ_C128)
        k_shard_unpack<double><<<move_blocks(half), 256, 0, s>>>(static_cast<const double2*>(buf), static_cast<double2*>(shard),
                                                                 half, local_bit, value);
    else
        k_shard_unpack<float><<<move_blocks(half), 256, 0, s>>>(static_cast<const float2*>(buf), static_cast<float2*>(shard),
                                                                half, local_bit, value);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}
