// Kernels for unitary simulation (Section II-A) with DiaQ matrices: the
// circuit's unitary is the chain of its time-step unitaries multiplied by
// the DiaQ product of Algorithm 1 (launch_spgemm), and Section III-A tracks
// how many diagonals and non-zeros it holds after each time step. These
// kernels count the non-zero values of each stored diagonal and gather the
// diagonals that hold any, so a product can drop diagonals that came out
// exactly zero without changing a value.

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace diaq {

// counts[q] += number of values of diagonal q that are not exactly zero.
// One grid row per diagonal; integer counts, so the order of the atomic
// additions does not change the result.
template <typename R>
__global__ void __launch_bounds__(256)
k_diag_nnz(const amp_t<R>* __restrict__ vals, const int64_t* __restrict__ starts,
           const int64_t* __restrict__ lens, unsigned long long* __restrict__ counts) {
    const int q = blockIdx.y;
    const int64_t len = lens[q];
    const amp_t<R>* v = vals + starts[q];
    unsigned int c = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
        const amp_t<R> a = v[t];
        c += (a.x != R(0) || a.y != R(0)) ? 1u : 0u;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(counts + q, (unsigned long long)c);
}

// dst diagonal q = src diagonal map[q]: copy lens[q] values.
template <typename R>
__global__ void __launch_bounds__(256)
k_gather_diagonals(amp_t<R>* __restrict__ dst, const int64_t* __restrict__ dst_starts,
                   const amp_t<R>* __restrict__ src, const int64_t* __restrict__ src_starts,
                   const int64_t* __restrict__ lens) {
    const int q = blockIdx.y;
    const int64_t len = lens[q];
    amp_t<R>* d = dst + dst_starts[q];
    const amp_t<R>* s = src + src_starts[q];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x)
        d[t] = s[t];
}

static unsigned grid_x(int64_t max_len) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((max_len + 255) / 256, 1024));
}

diaq_status count_diagonal_nnz(const diaq_op_s* op, std::vector<int64_t>* nnz, cudaStream_t s) {
    const int64_t N = int64_t(1) << op->n;
    const size_t D = op->offsets.size();
    nnz->assign(D, 0);
    if (D == 0) return DIAQ_OK;
    std::vector<int64_t> lens(D);
    int64_t max_len = 0;
    for (size_t q = 0; q < D; ++q) {
        const int64_t d = op->offsets[q];
        lens[q] = N - (d < 0 ? -d : d);
        max_len = std::max(max_len, lens[q]);
    }
    // device scratch: lens (int64) then counts (uint64)
    void* buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, 2 * D * sizeof(int64_t), s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(diagonal counts): %s", cudaGetErrorString(e));
    int64_t* d_lens = static_cast<int64_t*>(buf);
    unsigned long long* d_counts = reinterpret_cast<unsigned long long*>(d_lens + D);
    diaq_status st = DIAQ_OK;
    do {
        if ((e = cudaMemcpyAsync(d_lens, lens.data(), D * sizeof(int64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(d_counts, 0, D * sizeof(int64_t), s)) != cudaSuccess) {
            st = cuda_fail(e, "cudaMemcpyAsync/cudaMemsetAsync(diagonal counts)");
            break;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) {
            st = cuda_fail(e, "an earlier CUDA call (pending before launch of k_diag_nnz)");
            break;
        }
        const dim3 grid(grid_x(max_len), (unsigned)D);
        if (op->dtype == DIAQ_C128)
            k_diag_nnz<double><<<grid, 256, 0, s>>>(static_cast<const double2*>(op->d_values), op->d_starts, d_lens,
                                                     d_counts);
        else
            k_diag_nnz<float><<<grid, 256, 0, s>>>(static_cast<const float2*>(op->d_values), op->d_starts, d_lens,
                                                    d_counts);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            st = cuda_fail(e, "launch of k_diag_nnz");
            break;
        }
        if ((e = cudaMemcpyAsync(nnz->data(), d_counts, D * sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            st = cuda_fail(e, "reading diagonal counts");
            break;
        }
    } while (false);
    cudaFreeAsync(buf, s);
    return st;
}

diaq_status launch_gather_diagonals(const diaq_op_s* src, const std::vector<int32_t>& keep, diaq_op_s* dst,
                                    cudaStream_t s) {
    const size_t K = keep.size();
    if (K == 0) return DIAQ_OK;
    const int64_t N = int64_t(1) << src->n;
    std::vector<int64_t> host(3 * K);
    int64_t max_len = 0;
    for (size_t q = 0; q < K; ++q) {
        const int64_t d = src->offsets[keep[q]];
        host[q] = dst->starts[q];
        host[K + q] = src->starts[keep[q]];
        host[2 * K + q] = N - (d < 0 ? -d : d);
        max_len = std::max(max_len, host[2 * K + q]);
    }
    void* buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, host.size() * sizeof(int64_t), s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(diagonal map): %s", cudaGetErrorString(e));
    int64_t* m = static_cast<int64_t*>(buf);
    diaq_status st = DIAQ_OK;
    if ((e = cudaMemcpyAsync(m, host.data(), host.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        st = cuda_fail(e, "cudaMemcpyAsync(diagonal map)");
    } else if ((e = cudaGetLastError()) != cudaSuccess) {
        st = cuda_fail(e, "an earlier CUDA call (pending before launch of k_gather_diagonals)");
    } else {
        const dim3 grid(grid_x(max_len), (unsigned)K);
        if (src->dtype == DIAQ_C128)
            k_gather_diagonals<double><<<grid, 256, 0, s>>>(static_cast<double2*>(dst->d_values), m,
                                                            static_cast<const double2*>(src->d_values), m + K, m + 2 * K);
        else
            k_gather_diagonals<float><<<grid, 256, 0, s>>>(static_cast<float2*>(dst->d_values), m,
                                                           static_cast<const float2*>(src->d_values), m + K, m + 2 * K);
        if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(e, "launch of k_gather_diagonals");
    }
    // the host map must outlive the asynchronous copy
    const cudaError_t es = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    if (st == DIAQ_OK && es != cudaSuccess) st = cuda_fail(es, "cudaStreamSynchronize(gather diagonals)");
    return st;
}

}  // namespace diaq
