// Reductions and the adjoint reverse step of libdiaq_gb300.
//
// All sums accumulate in FP64 whatever the state precision, per thread in
// index order, then over the block with a fixed shuffle tree, then over the
// blocks of a fixed-size grid in a second kernel: the result is the same
// bit pattern on every run for a given n_qubits, dtype and gate.
//
// Pauli strings are encoded by masks (bit q of xmask: X or Y on qubit q;
// bit q of zmask: Z or Y). A string P maps |j> to i^{#Y} (-1)^{popc(j & z)}
// |j ^ x>, so <psi|P|psi> = sum_j conj(psi[j ^ x]) psi[j] i^{#Y}
// (-1)^{popc(j & z)} and (P psi)[i] = i^{#Y} (-1)^{popc((i ^ x) & z)}
// psi[i ^ x]. Terms that share an X mask are summed in one pass.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <vector>

#include "bounds.cuh"
#include "common.cuh"
#include "internal.h"

DIAQ_BOUNDS_TU(reduce)

namespace diaq {

// SM count of the current device, looked up once per device ordinal (it
// does not change while the process runs, whatever happens to contexts).
int device_sm_count() {
    constexpr int kMaxDevices = 64;
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    if (dev >= kMaxDevices) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 1;
    }
    int sms = cache[dev].load(std::memory_order_relaxed);
    if (!sms) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        cache[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

static int reduce_blocks(int64_t work_items) {
    const int64_t want = (work_items + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, int64_t(device_sm_count()) * 8));
}

template <typename R>
__device__ __forceinline__ double2 to_d2(amp_t<R> v) {
    return make_double2(double(v.x), double(v.y));
}

// ---------------------------------------------------------------------------
// Final sums: out[r] = sum_c part[r * cols + c].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sum_rows(const double* __restrict__ part, int cols, double* out) {
    __shared__ double warps[32];
    const double* p = part + (int64_t)blockIdx.x * cols;
    double s = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += p[c];
    s = block_sum(s, warps);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

diaq_status launch_sum_rows(const double* partials, int rows, int cols, double* out, cudaStream_t s) {
    if (rows <= 0) return DIAQ_OK;
    DIAQ_PRELAUNCH("k_sum_rows");
    k_sum_rows<<<rows, 256, 0, s>>>(partials, cols, out);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// Norm: sum |psi_i|^2. complex128 accumulates in FP64; complex64 forms each
// |psi_i|^2 in FP32 and sums a thread's share with Kahan compensation
// (Acc<float>), so the FP64 pipe is used only from the block sum on.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_norm(const amp_t<R>* __restrict__ psi, int64_t N, double* part) {
    __shared__ double warps[32];
    Acc<R> acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const amp_t<R> v = ld_stream(psi + i);
        acc.add_dot(v.x, v.x, v.y, v.y);
    }
    const double t = block_sum(acc.value(), warps);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

int norm_partials(int n) { return reduce_blocks((int64_t(1) << n) / 4); }

diaq_status launch_norm(const void* psi, int n, diaq_dtype dt, double* scratch, cudaStream_t s) {
    const int64_t N = int64_t(1) << n;
    const int P = norm_partials(n);
    DIAQ_PRELAUNCH("k_norm");
    if (dt == DIAQ_C128)
        k_norm<double><<<P, 256, 0, s>>>(reinterpret_cast<const double2*>(psi), N, scratch);
    else
        k_norm<float><<<P, 256, 0, s>>>(reinterpret_cast<const float2*>(psi), N, scratch);
    DIAQ_CUDA(cudaGetLastError());
    return launch_sum_rows(scratch, 1, P, scratch + P, s);
}

diaq_status run_norm(const void* psi, int n, diaq_dtype dt, double* out, cudaStream_t s) {
    const int P = norm_partials(n);
    double* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, sizeof(double) * (P + 1), s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(norm partials): %s", cudaGetErrorString(e));
    diaq_status st = launch_norm(psi, n, dt, d, s);
    if (st == DIAQ_OK) {
        e = cudaMemcpyAsync(out, d + P, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync(norm)");
    }
    cudaFreeAsync(d, s);
    if (st != DIAQ_OK) return st;
    DIAQ_CUDA(cudaStreamSynchronize(s));
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// Pauli groups
// ---------------------------------------------------------------------------
diaq_status make_pauli_groups(int n_qubits, int n_terms, const uint64_t* xm, const uint64_t* zm,
                              const double* coeff, bool real_only, PauliGroups* out) {
    const uint64_t valid = n_qubits >= 64 ? ~uint64_t(0) : ((uint64_t(1) << n_qubits) - 1);
    std::vector<int> order(n_terms);
    for (int t = 0; t < n_terms; ++t) {
        if ((xm[t] & ~valid) || (zm[t] & ~valid))
            return fail(DIAQ_ERR_ARG, "Pauli term %d acts on a qubit >= n_qubits (%d)", t, n_qubits);
        order[t] = t;
    }
    // stable: groups in order of first appearance of their X mask, terms in input order
    std::vector<uint64_t> keys;
    std::vector<std::vector<int>> members;
    for (int t = 0; t < n_terms; ++t) {
        size_t g = 0;
        for (; g < keys.size(); ++g)
            if (keys[g] == xm[t]) break;
        if (g == keys.size()) {
            keys.push_back(xm[t]);
            members.emplace_back();
        }
        members[g].push_back(t);
    }
    out->xmask = keys;
    out->first.clear();
    out->zmask.clear();
    out->kappa.clear();
    int pos = 0;
    for (size_t g = 0; g < keys.size(); ++g) {
        out->first.push_back(pos);
        for (int t : members[g]) {
            const int ny = __builtin_popcountll(xm[t] & zm[t]) & 3;
            const double cr = coeff[2 * t], ci = real_only ? 0.0 : coeff[2 * t + 1];
            // kappa = c * i^ny
            double kr = cr, ki = ci;
            for (int r = 0; r < ny; ++r) {
                const double tr = -ki, ti = kr;
                kr = tr;
                ki = ti;
            }
            out->zmask.push_back(zm[t]);
            out->kappa.push_back(kr);
            out->kappa.push_back(ki);
            ++pos;
        }
    }
    out->first.push_back(pos);
    return DIAQ_OK;
}

struct DevGroups {
    const uint64_t* xmask;
    const int32_t* first;
    const uint64_t* zmask;
    const double* kappa;
    int n_groups;
};

// Device copy of the groups in one temporary stream-ordered allocation.
static diaq_status upload_groups(const PauliGroups& pg, cudaStream_t s, void** mem, DevGroups* dg) {
    const size_t ng = pg.xmask.size(), nt = pg.zmask.size();
    const size_t bytes = 8 * ng + 4 * (ng + 1) + 4 /*pad*/ + 8 * nt + 16 * nt + 16;
    std::vector<unsigned char> buf(bytes, 0);
    size_t o = 0;
    const size_t o_x = o; o += 8 * ng;
    const size_t o_z = o; o += 8 * nt;
    const size_t o_k = o; o += 16 * nt;
    const size_t o_f = o; o += 4 * (ng + 1);
    if (ng) std::memcpy(buf.data() + o_x, pg.xmask.data(), 8 * ng);
    if (nt) std::memcpy(buf.data() + o_z, pg.zmask.data(), 8 * nt);
    if (nt) std::memcpy(buf.data() + o_k, pg.kappa.data(), 16 * nt);
    std::memcpy(buf.data() + o_f, pg.first.data(), 4 * (ng + 1));
    unsigned char* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, bytes, s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(Pauli terms): %s", cudaGetErrorString(e));
    e = cudaMemcpyAsync(d, buf.data(), bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        cudaFreeAsync(d, s);
        return cuda_fail(e, "cudaMemcpyAsync(Pauli terms)");
    }
    // pageable source: the copy has completed when cudaMemcpyAsync returns
    // for pageable memory only after staging; synchronise to be safe.
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFreeAsync(d, s);
        return cuda_fail(e, "cudaStreamSynchronize");
    }
    dg->xmask = reinterpret_cast<const uint64_t*>(d + o_x);
    dg->zmask = reinterpret_cast<const uint64_t*>(d + o_z);
    dg->kappa = reinterpret_cast<const double*>(d + o_k);
    dg->first = reinterpret_cast<const int32_t*>(d + o_f);
    dg->n_groups = (int)ng;
    *mem = d;
    return DIAQ_OK;
}

// W_g(j) = sum_{t in g} kappa_t (-1)^{popc(j & z_t)}
__device__ __forceinline__ double2 group_weight(const DevGroups& G, int g, uint64_t j) {
    double wr = 0.0, wi = 0.0;
    for (int t = G.first[g]; t < G.first[g + 1]; ++t) {
        const double kr = G.kappa[2 * t], ki = G.kappa[2 * t + 1];
        if (__popcll(j & G.zmask[t]) & 1) {
            wr -= kr;
            wi -= ki;
        } else {
            wr += kr;
            wi += ki;
        }
    }
    return make_double2(wr, wi);
}

// ---------------------------------------------------------------------------
// Expectation: sum_g sum_j conj(psi[j ^ x_g]) psi[j] W_g(j).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_expect(const amp_t<R>* __restrict__ psi, int64_t N, const DevGroups G, double* part) {
    __shared__ double warps[32];
    double ar = 0.0, ai = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) {
        const double2 pj = to_d2<R>(psi[j]);
        for (int g = 0; g < G.n_groups; ++g) {
            const int64_t jk = j ^ (int64_t)G.xmask[g];
            if (!DIAQ_BOUNDS_OK(jk, N, BS_EXPECT)) continue;
            const double2 pk = to_d2<R>(psi[jk]);
            // w = conj(pk) * pj
            const double wr = pk.x * pj.x + pk.y * pj.y;
            const double wi = pk.x * pj.y - pk.y * pj.x;
            const double2 W = group_weight(G, g, (uint64_t)j);
            ar = fma(W.x, wr, ar);
            ar = fma(-W.y, wi, ar);
            ai = fma(W.x, wi, ai);
            ai = fma(W.y, wr, ai);
        }
    }
    ar = block_sum(ar, warps);
    ai = block_sum(ai, warps);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = ar;
        part[gridDim.x + blockIdx.x] = ai;
    }
}

diaq_status run_expect(const void* psi, int n, diaq_dtype dt, const PauliGroups& pg, double* out,
                       cudaStream_t s) {
    if (pg.zmask.empty()) {
        out[0] = out[1] = 0.0;
        return DIAQ_OK;
    }
    void* gm = nullptr;
    DevGroups G;
    DIAQ_TRY(upload_groups(pg, s, &gm, &G));
    const int64_t N = int64_t(1) << n;
    const int P = reduce_blocks(N / 4);
    double* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, sizeof(double) * (2 * P + 2), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(gm, s);
        return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(expect partials): %s", cudaGetErrorString(e));
    }
    DIAQ_PRELAUNCH("k_expect");
    if (dt == DIAQ_C128)
        k_expect<double><<<P, 256, 0, s>>>(reinterpret_cast<const double2*>(psi), N, G, d);
    else
        k_expect<float><<<P, 256, 0, s>>>(reinterpret_cast<const float2*>(psi), N, G, d);
    DIAQ_CUDA(cudaGetLastError());
    DIAQ_TRY(launch_sum_rows(d, 2, P, d + 2 * P, s));
    double res[2];
    DIAQ_CUDA(cudaMemcpyAsync(res, d + 2 * P, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    DIAQ_CUDA(cudaFreeAsync(d, s));
    DIAQ_CUDA(cudaFreeAsync(gm, s));
    DIAQ_CUDA(cudaStreamSynchronize(s));
    out[0] = res[0];
    out[1] = res[1];
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// lambda[i] = sum_g psi[i ^ x_g] W_g(i ^ x_g)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_pauli_apply(const amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam, int64_t N, const DevGroups G) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        R lr = R(0), li = R(0);
        for (int g = 0; g < G.n_groups; ++g) {
            const uint64_t j = (uint64_t)i ^ G.xmask[g];
            if (!DIAQ_BOUNDS_OK(int64_t(j), N, BS_PAULI_APPLY)) continue;
            const amp_t<R> p = psi[j];
            // W_g(j) in the state's precision
            R wr = R(0), wi = R(0);
            for (int t = G.first[g]; t < G.first[g + 1]; ++t) {
                const R kr = R(G.kappa[2 * t]), ki = R(G.kappa[2 * t + 1]);
                const bool neg = (__popcll(j & G.zmask[t]) & 1) != 0;
                wr += neg ? -kr : kr;
                wi += neg ? -ki : ki;
            }
            lr = fma(wr, p.x, fma(-wi, p.y, lr));
            li = fma(wr, p.y, fma(wi, p.x, li));
        }
        amp_t<R> o;
        o.x = lr;
        o.y = li;
        lam[i] = o;
    }
}

diaq_status run_pauli_apply(const void* psi, void* lam, int n, diaq_dtype dt, const PauliGroups& pg,
                            cudaStream_t s) {
    const int64_t N = int64_t(1) << n;
    if (pg.zmask.empty()) {
        DIAQ_CUDA(cudaMemsetAsync(lam, 0, size_t(N) * amp_bytes(dt), s));
        return DIAQ_OK;
    }
    void* gm = nullptr;
    DevGroups G;
    DIAQ_TRY(upload_groups(pg, s, &gm, &G));
    const int P = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, int64_t(device_sm_count()) * 16));
    DIAQ_PRELAUNCH("k_pauli_apply");
    if (dt == DIAQ_C128)
        k_pauli_apply<double><<<P, 256, 0, s>>>(reinterpret_cast<const double2*>(psi),
                                                reinterpret_cast<double2*>(lam), N, G);
    else
        k_pauli_apply<float><<<P, 256, 0, s>>>(reinterpret_cast<const float2*>(psi),
                                               reinterpret_cast<float2*>(lam), N, G);
    DIAQ_CUDA(cudaGetLastError());
    DIAQ_CUDA(cudaFreeAsync(gm, s));
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// Re <a|b> into partials (P blocks).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_inner_re(const amp_t<R>* __restrict__ a, const amp_t<R>* __restrict__ b, int64_t N, double* part) {
    __shared__ double warps[32];
    Acc<R> acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const amp_t<R> u = a[i], v = b[i];
        acc.add_dot(u.x, v.x, u.y, v.y);
    }
    const double t = block_sum(acc.value(), warps);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

int inner_partials(int n) { return reduce_blocks((int64_t(1) << n) / 4); }

diaq_status launch_inner_re(const void* a, const void* b, int n, diaq_dtype dt, double* partials,
                            int n_partials, cudaStream_t s) {
    const int64_t N = int64_t(1) << n;
    DIAQ_PRELAUNCH("k_inner_re");
    if (dt == DIAQ_C128)
        k_inner_re<double><<<n_partials, 256, 0, s>>>(reinterpret_cast<const double2*>(a),
                                                      reinterpret_cast<const double2*>(b), N, partials);
    else
        k_inner_re<float><<<n_partials, 256, 0, s>>>(reinterpret_cast<const float2*>(a),
                                                     reinterpret_cast<const float2*>(b), N, partials);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// Adjoint reverse step for a gate of k <= 3 qubits: per group, the partial
// Im sum_r conj(lam_r) (P psi)_r (if the gate is parametric), then
// psi <- U^dag psi and lam <- U^dag lam in place.
// ---------------------------------------------------------------------------
template <typename R, int K>
struct AdjArgs {
    int64_t n_groups;
    int st[K];
    int64_t off[1 << K];
    R ure[1 << (2 * K)], uim[1 << (2 * K)];
    uint8_t utype[1 << (2 * K)];
    R pre[1 << (2 * K)], pim[1 << (2 * K)];
    uint8_t ptype[1 << (2 * K)];
    int has_p;
};

template <typename R, int K>
__global__ void __launch_bounds__(256)
k_adjoint_step(amp_t<R>* psi, amp_t<R>* lam, double* part, const __grid_constant__ AdjArgs<R, K> a) {
    constexpr int D = 1 << K;
    using A = amp_t<R>;
    __shared__ double warps[32];
    Acc<R> acc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.n_groups; g += stride) {
        const int64_t b = insert_zeros<K>(g, a.st);
        A p[D], l[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            p[c] = psi[b + a.off[c]];
            l[c] = lam[b + a.off[c]];
        }
        if (a.has_p) {
#pragma unroll
            for (int r = 0; r < D; ++r) {
                A q;
                q.x = R(0);
                q.y = R(0);
                bool first = true;
#pragma unroll
                for (int c = 0; c < D; ++c) mac_typed<R>(q, first, a.ptype[r * D + c], a.pre[r * D + c], a.pim[r * D + c], p[c]);
                // Im(conj(l) q) = l.x q.y - l.y q.x
                acc.add_cross(l[r].x, q.y, l[r].y, q.x);
            }
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
            A u, w;
            u.x = R(0);
            u.y = R(0);
            w.x = R(0);
            w.y = R(0);
            bool f1 = true, f2 = true;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                mac_typed<R>(u, f1, a.utype[r * D + c], a.ure[r * D + c], a.uim[r * D + c], p[c]);
                mac_typed<R>(w, f2, a.utype[r * D + c], a.ure[r * D + c], a.uim[r * D + c], l[c]);
            }
            psi[b + a.off[r]] = u;
            lam[b + a.off[r]] = w;
        }
    }
    if (part) {
        const double t = block_sum(acc.value(), warps);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

int adjoint_partials(int n, diaq_dtype, int k) { return reduce_blocks(int64_t(1) << (n - k)); }

template <typename R, int K>
static diaq_status launch_adj(int n, diaq_dtype dt, const GateDesc& u, const GateDesc* pauli, void* psi,
                              void* lam, double* partials, int n_partials, cudaStream_t s) {
    AdjArgs<R, K> a;
    std::memset(&a, 0, sizeof(a));
    a.n_groups = int64_t(1) << (n - K);
    for (int i = 0; i < K; ++i) a.st[i] = u.targets[i];
    std::sort(a.st, a.st + K);
    for (int c = 0; c < (1 << K); ++c) {
        int64_t o = 0;
        for (int i = 0; i < K; ++i)
            if ((c >> (K - 1 - i)) & 1) o += int64_t(1) << u.targets[i];
        a.off[c] = o;
    }
    for (int e = 0; e < (1 << (2 * K)); ++e) {
        a.ure[e] = R(u.m[e].real());
        a.uim[e] = R(u.m[e].imag());
        a.utype[e] = entry_type(cplx(double(a.ure[e]), double(a.uim[e])));
        if (pauli) {
            a.pre[e] = R(pauli->m[e].real());
            a.pim[e] = R(pauli->m[e].imag());
            a.ptype[e] = entry_type(pauli->m[e]);
        }
    }
    a.has_p = pauli ? 1 : 0;
    DIAQ_PRELAUNCH("k_adjoint_step");
    k_adjoint_step<R, K><<<n_partials, 256, 0, s>>>(reinterpret_cast<amp_t<R>*>(psi),
                                                    reinterpret_cast<amp_t<R>*>(lam), pauli ? partials : nullptr, a);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

diaq_status launch_adjoint_step(int n, diaq_dtype dt, const GateDesc& udag, const GateDesc* pauli,
                                void* psi, void* lam, double* partials, int n_partials, cudaStream_t s) {
    const bool d = dt == DIAQ_C128;
    switch (udag.k) {
        case 1: return d ? launch_adj<double, 1>(n, dt, udag, pauli, psi, lam, partials, n_partials, s)
                         : launch_adj<float, 1>(n, dt, udag, pauli, psi, lam, partials, n_partials, s);
        case 2: return d ? launch_adj<double, 2>(n, dt, udag, pauli, psi, lam, partials, n_partials, s)
                         : launch_adj<float, 2>(n, dt, udag, pauli, psi, lam, partials, n_partials, s);
        case 3: return d ? launch_adj<double, 3>(n, dt, udag, pauli, psi, lam, partials, n_partials, s)
                         : launch_adj<float, 3>(n, dt, udag, pauli, psi, lam, partials, n_partials, s);
        default: return fail(DIAQ_ERR_UNSUPPORTED, "adjoint step supports gates of at most 3 qubits (got %d)", udag.k);
    }
}

}  // namespace diaq
