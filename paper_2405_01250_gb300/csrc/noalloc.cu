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

#include "common.cuh"
#include "internal.h"

// Scratch of the no-alloc norm: DIAQ_NOALLOC_SCRATCH_DOUBLES doubles
// (32 KiB), present on every device that loads the library until the process
// exits. Slots [0, P) hold the block partials of one call, slot P the total.
static __device__ __align__(256) double g_noalloc_scratch[DIAQ_NOALLOC_SCRATCH_DOUBLES];

namespace diaq {
namespace {

// Device address of the scratch array in the current context. In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with the device current. It is looked up on
// every call rather than cached: the lookup is cheap once the library's
// module is loaded on the device, and a context that the host application
// tore down and recreated (cudaDeviceReset) may place the array elsewhere.
diaq_status scratch_for_current_device(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    *out = static_cast<double*>(p);
    return DIAQ_OK;
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
    // the grid of diaq_norm: one block per 1024 amplitudes, at most 8 per SM
    const int P = norm_partials(n_qubits);
    if (P + 1 > DIAQ_NOALLOC_SCRATCH_DOUBLES)
        return fail(DIAQ_ERR_UNSUPPORTED,
                    "no-alloc norm needs %d doubles of scratch but the fixed array holds %d (DIAQ_NOALLOC_SCRATCH_DOUBLES)",
                    P + 1, DIAQ_NOALLOC_SCRATCH_DOUBLES);
    double* scratch = nullptr;
    DIAQ_TRY(scratch_for_current_device(&scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Every slot read (partials [0, P) and the total at P) is written earlier
    // in this same call, so no slot needs clearing first.
    DIAQ_TRY(launch_norm(psi, n_qubits, dtype, scratch, s));
    DIAQ_CUDA(cudaMemcpyAsync(out, scratch + P, sizeof(double), cudaMemcpyDeviceToHost, s));
    DIAQ_CUDA(cudaStreamSynchronize(s));
    return DIAQ_OK;
}
