// diaq_norm_noalloc: the FP64 norm reduction of diaq_norm without any
// device allocation. The per-block partial sums and the total live in a
// fixed array compiled into the library instead of memory obtained from
// cudaMallocAsync.
//
// This is for callers whose device memory is not theirs to allocate from:
// an application whose memory manager has reserved the whole device heap
// up front (a library cudaMalloc would fail or bypass its accounting), or a
// latency-critical loop that cannot afford the implicit synchronisation and
// pool growth an allocation can trigger.

#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

// Scratch of the no-alloc norm: DIAQ_NOALLOC_SCRATCH_DOUBLES doubles
// (32 KiB), present on every device that loads the library until the process
// exits. Slots [0, P) hold the block partials of one call, slot P the total.
static __device__ __align__(256) double g_noalloc_scratch[DIAQ_NOALLOC_SCRATCH_DOUBLES];

namespace diaq {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};

// Device address of the scratch array for the current device. In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
diaq_status scratch_for_current_device(double** out, int* sms) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(DIAQ_ERR_UNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute(SM count)");
        g_sm_count[dev] = n > 0 ? n : 1;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    *sms = g_sm_count[dev];
    return DIAQ_OK;
}

// Same per-thread order, block tree and grid as the norm of diaq_norm, so
// the two entry points return the same bits.
template <typename R>
__global__ void __launch_bounds__(256) k_norm_partials_noalloc(const amp_t<R>* __restrict__ psi, int64_t N,
                                                               double* part) {
    __shared__ double warps[32];
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const amp_t<R> v = ld_stream(psi + i);
        if constexpr (sizeof(R) == 8) {
            acc = fma(double(v.x), double(v.x), acc);
            acc = fma(double(v.y), double(v.y), acc);
        } else {
            acc += double(fmaf(v.x, v.x, v.y * v.y));
        }
    }
    acc = block_sum(acc, warps);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) k_norm_total_noalloc(const double* __restrict__ part, int cols, double* out) {
    __shared__ double warps[32];
    double s = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += part[c];
    s = block_sum(s, warps);
    if (threadIdx.x == 0) *out = s;
}

}  // namespace
}  // namespace diaq

using namespace diaq;

extern "C" diaq_status diaq_norm_noalloc(const void* psi, int32_t n_qubits, diaq_dtype dtype, double* out,
                                         diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();  // discard a non-sticky error left by the caller's own calls
    if (!psi || !out) return fail(DIAQ_ERR_ARG, "psi or out is NULL");
    if (n_qubits < 1 || n_qubits > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_qubits = %d out of range", n_qubits);
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (reinterpret_cast<uintptr_t>(psi) & 15) return fail(DIAQ_ERR_ARG, "state buffer must be 16-byte aligned");
    double* scratch = nullptr;
    int sms = 1;
    DIAQ_TRY(scratch_for_current_device(&scratch, &sms));
    const int64_t N = int64_t(1) << n_qubits;
    // grid of the diaq_norm reduction: one block per 1024 amplitudes, at most 8 per SM
    const int64_t want = (N / 4 + 255) / 256;
    const int P = (int)std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 8));
    if (P + 1 > DIAQ_NOALLOC_SCRATCH_DOUBLES)
        return fail(DIAQ_ERR_UNSUPPORTED,
                    "no-alloc norm needs %d doubles of scratch but the fixed array holds %d (DIAQ_NOALLOC_SCRATCH_DOUBLES)",
                    P + 1, DIAQ_NOALLOC_SCRATCH_DOUBLES);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Every slot read below (partials [0, P) and the total at P) is written
    // earlier in this same call, so no slot needs clearing first.
    if (dtype == DIAQ_C128)
        k_norm_partials_noalloc<double><<<P, 256, 0, s>>>(reinterpret_cast<const double2*>(psi), N, scratch);
    else
        k_norm_partials_noalloc<float><<<P, 256, 0, s>>>(reinterpret_cast<const float2*>(psi), N, scratch);
    DIAQ_CUDA(cudaGetLastError());
    k_norm_total_noalloc<<<1, 256, 0, s>>>(scratch, P, scratch + P);
    DIAQ_CUDA(cudaGetLastError());
    DIAQ_CUDA(cudaMemcpyAsync(out, scratch + P, sizeof(double), cudaMemcpyDeviceToHost, s));
    DIAQ_CUDA(cudaStreamSynchronize(s));
    return DIAQ_OK;
}
