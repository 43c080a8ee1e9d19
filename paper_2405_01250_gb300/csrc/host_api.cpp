// Host side of libdiaq_gb300: argument checks, the DiaQ builder (offsets,
// classes), the host DiaQ product of Algorithm 1 used for gate fusion, op
// lifecycle and the C ABI entry points declared in include/diaq.h.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <mutex>
#include <vector>

#include "bounds.cuh"
#include "internal.h"

namespace diaq {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_error;

diaq_status fail(diaq_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
    return s;
}

void clear_error() { g_error.clear(); }

// Device entry points: also discard a non-sticky error that an earlier,
// unchecked runtime call of the host application left pending, so the
// launch checks below report only this call's own failures. (A sticky
// error, such as a fault, persists and is reported by the next call.)
static void clear_error_device() {
    g_error.clear();
    cudaGetLastError();
}

diaq_status cuda_fail(cudaError_t e, const char* what) {
    return fail(DIAQ_ERR_CUDA, "%s failed: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Gate description
// ---------------------------------------------------------------------------
uint8_t entry_type(cplx v) {
    if (v.real() == 0.0 && v.imag() == 0.0) return ET_ZERO;
    if (v.imag() == 0.0) return v.real() == 1.0 ? ET_ONE : ET_REAL;
    if (v.real() == 0.0) return ET_IMAG;
    return ET_GENERAL;
}

std::vector<cplx> pauli_matrix(const char* gen, int k) {
    std::vector<cplx> m(1, cplx(1.0, 0.0));
    int dim = 1;
    for (int a = 0; a < k; ++a) {
        cplx p[4];
        switch (gen[a]) {
            case 'X': case 'x': p[0] = 0; p[1] = 1; p[2] = 1; p[3] = 0; break;
            case 'Y': case 'y': p[0] = 0; p[1] = cplx(0, -1); p[2] = cplx(0, 1); p[3] = 0; break;
            case 'Z': case 'z': p[0] = 1; p[1] = 0; p[2] = 0; p[3] = -1; break;
            default: p[0] = 1; p[1] = 0; p[2] = 0; p[3] = 1; break;
        }
        // kron(m, p): earlier letters are more significant
        std::vector<cplx> r(static_cast<size_t>(4) * dim * dim);
        const int nd = 2 * dim;
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < dim; ++j)
                for (int u = 0; u < 2; ++u)
                    for (int v = 0; v < 2; ++v) r[(2 * i + u) * nd + (2 * j + v)] = m[i * dim + j] * p[2 * u + v];
        m.swap(r);
        dim = nd;
    }
    return m;
}

static diaq_status check_gate_shape(const diaq_gate* g, int n_qubits) {
    if (!g) return fail(DIAQ_ERR_ARG, "gate is NULL");
    if (n_qubits < 1 || n_qubits > DIAQ_MAX_QUBITS)
        return fail(DIAQ_ERR_ARG, "n_qubits = %d outside [1, %d]", n_qubits, DIAQ_MAX_QUBITS);
    if (g->k < 1 || g->k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "gate k = %d outside [1, %d]", g->k, DIAQ_MAX_K);
    if (g->k > n_qubits) return fail(DIAQ_ERR_SHAPE, "gate on %d qubits does not fit %d qubits", g->k, n_qubits);
    for (int a = 0; a < g->k; ++a) {
        if (g->targets[a] < 0 || g->targets[a] >= n_qubits)
            return fail(DIAQ_ERR_ARG, "target %d = %d outside [0, %d)", a, g->targets[a], n_qubits);
        for (int b = 0; b < a; ++b)
            if (g->targets[a] == g->targets[b]) return fail(DIAQ_ERR_ARG, "repeated target %d", g->targets[a]);
    }
    return DIAQ_OK;
}

static diaq_status check_gen(const diaq_gate* g) {
    const size_t len = strnlen(g->gen, sizeof(g->gen));
    if (len != size_t(g->k)) return fail(DIAQ_ERR_ARG, "generator \"%.*s\" must have one letter per target (k = %d)",
                                         (int)len, g->gen, g->k);
    for (int a = 0; a < g->k; ++a)
        if (!strchr("IXYZixyz", g->gen[a])) return fail(DIAQ_ERR_ARG, "generator letter '%c' not in IXYZ", g->gen[a]);
    return DIAQ_OK;
}

diaq_status gate_desc_from(const diaq_gate* g, int n_qubits, const double* theta, GateDesc* out) {
    DIAQ_TRY(check_gate_shape(g, n_qubits));
    out->k = g->k;
    for (int a = 0; a < g->k; ++a) out->targets[a] = g->targets[a];
    const size_t DD = size_t(1) << (2 * g->k);
    out->m.assign(DD, cplx(0, 0));
    if (g->param < 0) {
        if (!g->m) return fail(DIAQ_ERR_ARG, "fixed gate has no matrix");
        for (size_t e = 0; e < DD; ++e) {
            out->m[e] = cplx(g->m[2 * e], g->m[2 * e + 1]);
            if (!std::isfinite(g->m[2 * e]) || !std::isfinite(g->m[2 * e + 1]))
                return fail(DIAQ_ERR_ARG, "gate matrix entry %zu is not finite", e);
        }
        return DIAQ_OK;
    }
    DIAQ_TRY(check_gen(g));
    if (!theta) return fail(DIAQ_ERR_ARG, "parametric gate needs theta");
    const double a = g->scale * theta[g->param];
    if (!std::isfinite(a)) return fail(DIAQ_ERR_ARG, "parameter angle is not finite");
    const std::vector<cplx> P = pauli_matrix(g->gen, g->k);
    const double c = std::cos(0.5 * a), s = std::sin(0.5 * a);
    const int D = 1 << g->k;
    for (int r = 0; r < D; ++r)
        for (int q = 0; q < D; ++q) out->m[r * D + q] = (r == q ? cplx(c, 0) : cplx(0, 0)) + cplx(0, -s) * P[r * D + q];
    return DIAQ_OK;
}

int classify(const std::vector<cplx>& m, int k) {
    const int D = 1 << k;
    bool diag = true, real = true, mono = true, perm = true;
    std::vector<int> colcount(D, 0);
    for (int r = 0; r < D; ++r) {
        int rowcount = 0;
        for (int c = 0; c < D; ++c) {
            const cplx v = m[r * D + c];
            if (v.imag() != 0.0) real = false;
            if (v != cplx(0, 0)) {
                if (r != c) diag = false;
                ++rowcount;
                ++colcount[c];
                if (v != cplx(1, 0)) perm = false;
            }
        }
        if (rowcount != 1) mono = perm = false;
    }
    for (int c = 0; c < D; ++c)
        if (colcount[c] != 1) mono = perm = false;
    if (diag) return DIAQ_CLASS_DIAGONAL;
    if (perm) return DIAQ_CLASS_PERMUTATION;
    if (mono) return DIAQ_CLASS_MONOMIAL;
    if (real) return DIAQ_CLASS_REAL;
    return DIAQ_CLASS_GENERAL;
}

std::vector<int64_t> full_offsets(const GateDesc& g, const std::vector<uint8_t>* pattern) {
    const int D = 1 << g.k;
    std::vector<int64_t> out;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            const bool nz = pattern ? (*pattern)[r * D + c] != 0 : g.m[r * D + c] != cplx(0, 0);
            if (!nz) continue;
            int64_t d = 0;
            for (int a = 0; a < g.k; ++a) {
                const int64_t rb = (r >> (g.k - 1 - a)) & 1, cb = (c >> (g.k - 1 - a)) & 1;
                d += (cb - rb) * (int64_t(1) << g.targets[a]);
            }
            out.push_back(d);
        }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
    return out;
}

// Structural pattern: non-zeros of M for a fixed gate, of I and P for a
// parametric one (so the offsets do not depend on the angle).
static std::vector<uint8_t> gate_pattern(const diaq_gate* g, const GateDesc& d) {
    const int D = 1 << d.k;
    std::vector<uint8_t> p(static_cast<size_t>(D) * D, 0);
    if (g->param < 0) {
        for (int e = 0; e < D * D; ++e) p[e] = d.m[e] != cplx(0, 0);
    } else {
        const std::vector<cplx> P = pauli_matrix(g->gen, g->k);
        for (int e = 0; e < D * D; ++e) p[e] = (P[e] != cplx(0, 0)) || (e / D == e % D);
    }
    return p;
}

// ---------------------------------------------------------------------------
// Host DiaQ product (Algorithm 1, accumulating reading)
// ---------------------------------------------------------------------------
using DiaMap = std::map<int64_t, std::vector<cplx>>;

static int64_t dlen(int64_t N, int64_t d) { return N - (d < 0 ? -d : d); }

// C = A B. Row form: A(i, i+a) sits at position i - max(0, -a) of diagonal a.
static DiaMap diaq_matmul(int64_t N, const DiaMap& A, const DiaMap& B) {
    DiaMap C;
    for (const auto& [a, va] : A)
        for (const auto& [b, vb] : B) {
            const int64_t e = a + b;
            const int64_t lo = std::max<int64_t>({0, -a, -e});
            const int64_t hi = std::min<int64_t>({N, N - a, N - e});
            if (lo >= hi) continue;  // "isValid": the product diagonal has no element
            auto it = C.find(e);
            if (it == C.end()) it = C.emplace(e, std::vector<cplx>(size_t(dlen(N, e)), cplx(0, 0))).first;
            std::vector<cplx>& vc = it->second;
            const int64_t sa = a < 0 ? -a : 0, sb = b < 0 ? -b : 0, sc = e < 0 ? -e : 0;
            for (int64_t i = lo; i < hi; ++i) vc[size_t(i - sc)] += va[size_t(i - sa)] * vb[size_t(i + a - sb)];
        }
    return C;
}

static DiaMap dense_to_map(const std::vector<cplx>& m, int64_t N) {
    DiaMap out;
    for (int64_t d = -(N - 1); d <= N - 1; ++d) {
        const int64_t len = dlen(N, d), r0 = d < 0 ? -d : 0, c0 = d > 0 ? d : 0;
        bool nz = false;
        for (int64_t t = 0; t < len && !nz; ++t) nz = m[size_t((r0 + t) * N + c0 + t)] != cplx(0, 0);
        if (!nz) continue;
        std::vector<cplx> v(static_cast<size_t>(len));
        for (int64_t t = 0; t < len; ++t) v[size_t(t)] = m[size_t((r0 + t) * N + c0 + t)];
        out.emplace(d, std::move(v));
    }
    return out;
}

static std::vector<cplx> map_to_dense(const DiaMap& A, int64_t N) {
    std::vector<cplx> m(static_cast<size_t>(N * N), cplx(0, 0));
    for (const auto& [d, v] : A) {
        const int64_t r0 = d < 0 ? -d : 0, c0 = d > 0 ? d : 0;
        for (int64_t t = 0; t < int64_t(v.size()); ++t) m[size_t((r0 + t) * N + c0 + t)] = v[size_t(t)];
    }
    return m;
}

// Embedding of a gate in a union target space (union[0] most significant).
static std::vector<cplx> embed(const GateDesc& g, const int* uni, int K) {
    const int64_t DU = int64_t(1) << K;
    int pos[DIAQ_MAX_K];
    for (int a = 0; a < g.k; ++a)
        for (int u = 0; u < K; ++u)
            if (uni[u] == g.targets[a]) pos[a] = K - 1 - u;
    int64_t gmask = 0;
    for (int a = 0; a < g.k; ++a) gmask |= int64_t(1) << pos[a];
    const int D = 1 << g.k;
    std::vector<cplx> E(static_cast<size_t>(DU * DU), cplx(0, 0));
    for (int64_t R = 0; R < DU; ++R)
        for (int64_t C = 0; C < DU; ++C) {
            if ((R & ~gmask) != (C & ~gmask)) continue;
            int r = 0, c = 0;
            for (int a = 0; a < g.k; ++a) {
                r |= int((R >> pos[a]) & 1) << (g.k - 1 - a);
                c |= int((C >> pos[a]) & 1) << (g.k - 1 - a);
            }
            E[size_t(R * DU + C)] = g.m[size_t(r * D + c)];
        }
    return E;
}

static diaq_status fuse_descs(const std::vector<GateDesc>& gs, GateDesc* out) {
    int uni[DIAQ_MAX_K];
    int K = 0;
    for (const GateDesc& g : gs)
        for (int a = 0; a < g.k; ++a) {
            bool seen = false;
            for (int u = 0; u < K; ++u) seen |= uni[u] == g.targets[a];
            if (seen) continue;
            if (K == DIAQ_MAX_K)
                return fail(DIAQ_ERR_UNSUPPORTED, "fused gates span more than %d qubits", DIAQ_MAX_K);
            uni[K++] = g.targets[a];
        }
    const int64_t DU = int64_t(1) << K;
    DiaMap acc;
    {
        std::vector<cplx> I(static_cast<size_t>(DU * DU), cplx(0, 0));
        for (int64_t i = 0; i < DU; ++i) I[size_t(i * DU + i)] = 1.0;
        acc = dense_to_map(I, DU);
    }
    for (const GateDesc& g : gs) acc = diaq_matmul(DU, dense_to_map(embed(g, uni, K), DU), acc);
    out->k = K;
    for (int u = 0; u < K; ++u) out->targets[u] = uni[u];
    out->m = map_to_dense(acc, DU);
    return DIAQ_OK;
}

}  // namespace diaq

using namespace diaq;

// ---------------------------------------------------------------------------
// Allocation-failure injection (testing hook)
// ---------------------------------------------------------------------------
static std::atomic<int> g_fail_in{-1};

// true if this allocation is the one chosen to fail
static bool inject_now() {
    int v = g_fail_in.load();
    while (v >= 0) {
        if (g_fail_in.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

namespace diaq {
cudaError_t inj_malloc(void** p, size_t n) {
    if (inject_now()) return cudaErrorMemoryAllocation;
    return (cudaMalloc)(p, n);
}
cudaError_t inj_malloc_async(void** p, size_t n, cudaStream_t s) {
    if (inject_now()) return cudaErrorMemoryAllocation;
    return (cudaMallocAsync)(p, n, s);
}
cudaError_t inj_malloc_host(void** p, size_t n) {
    if (inject_now()) return cudaErrorMemoryAllocation;
    return (cudaMallocHost)(p, n);
}
}  // namespace diaq

// ---------------------------------------------------------------------------
// Debug bounds checks (the build with -DDIAQ_DEBUG_BOUNDS)
// ---------------------------------------------------------------------------
extern "C" diaq_status diaq_debug_bounds_enabled(int32_t* enabled) {
    clear_error();
    if (!enabled) return fail(DIAQ_ERR_ARG, "enabled is NULL");
#ifdef DIAQ_DEBUG_BOUNDS
    *enabled = 1;
#else
    *enabled = 0;
#endif
    return DIAQ_OK;
}

extern "C" diaq_status diaq_debug_bounds_status(uint64_t word) {
    clear_error();
    if (word == 0) return DIAQ_OK;
    static const char* names[] = {"?", "on-the-fly apply (k <= 3)", "in-place row skip", "on-the-fly apply (k >= 4)",
                                  "diagonal op", "stored SpMV row", "stored SpMV column", "materialise",
                                  "expectation", "Pauli-sum apply", "rotation", "sampling tile pass",
                                  "sampling descent", "shard move", "DiaQ product", "window sweep"};
    if (word == ~uint64_t(0)) return fail(DIAQ_ERR_CUDA, "a bounds word could not be read from the device");
    const int site = int((word >> 48) & 0x7fff);
    const uint64_t idx = word & 0xffffffffffffull;
    const int64_t sidx = (idx >> 47) ? int64_t(idx | ~0xffffffffffffull) : int64_t(idx);  // sign-extend 48 bits
    return fail(DIAQ_ERR_BOUNDS, "device index check failed in %s (site %d): index %lld", site < BS_SITES ? names[site] : "?",
                site, (long long)sidx);
}

extern "C" diaq_status diaq_debug_bounds_check(int32_t clear, uint64_t* word) {
    clear_error();
    unsigned long long first = 0;
    unsigned long long (*const tus[])(bool) = {bounds_word_apply, bounds_word_inplace, bounds_word_diag,
                                               bounds_word_reduce, bounds_word_batch, bounds_word_sample,
                                               bounds_word_shard};
    for (auto f : tus) {
        const unsigned long long w = f(clear != 0);
        if (w && !first) first = w;
    }
    if (word) *word = first;
    return diaq_debug_bounds_status(first);
}

extern "C" diaq_status diaq_debug_inject_alloc_failure(int32_t after) {
    clear_error();
    if (after < -1) return fail(DIAQ_ERR_ARG, "after = %d: use -1 (off) or >= 0", after);
    g_fail_in.store(after);
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// Op helpers
// ---------------------------------------------------------------------------
static diaq_status check_op(diaq_op_t op) {
    if (!op) return fail(DIAQ_ERR_ARG, "op is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != op->device)
        return fail(DIAQ_ERR_ARG, "op was built on device %d but device %d is current", op->device, dev);
    return DIAQ_OK;
}

static diaq_status free_op_memory(diaq_op_s* op) {
    cudaError_t first = cudaSuccess;
    // the stored values return to the pool (cudaFree waits for the device
    // first, as for the other buffers)
    for (void* p : {op->d_values, static_cast<void*>(op->d_offsets), static_cast<void*>(op->d_starts), op->d_matrix}) {
        if (!p) continue;
        const cudaError_t e = cudaFree(p);
        if (e != cudaSuccess && first == cudaSuccess) first = e;
    }
    op->d_values = nullptr;
    op->d_offsets = nullptr;
    op->d_starts = nullptr;
    op->d_matrix = nullptr;
    return first == cudaSuccess ? DIAQ_OK : cuda_fail(first, "cudaFree(op memory)");
}

// Stored diagonals come from a library-owned stream-ordered pool per device
// that keeps up to 32 GiB of released memory for reuse, so the build,
// apply, release cycle of a circuit of stored ops (up to 12 GiB each at 28
// qubits) does not return to the operating system between ops. Memory above
// that threshold goes back at the next synchronisation.
static diaq_status values_pool(int dev, cudaMemPool_t* out) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return fail(DIAQ_ERR_UNSUPPORTED, "device ordinal %d >= 64", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        DIAQ_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t keep = uint64_t(32) << 30;
        DIAQ_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
        pools[dev] = p;
    }
    *out = pools[dev];
    return DIAQ_OK;
}

static diaq_status alloc_stored(diaq_op_s* op, cudaStream_t s) {
    const int64_t N = int64_t(1) << op->n;
    op->starts.resize(op->offsets.size());
    int64_t tot = 0;
    for (size_t q = 0; q < op->offsets.size(); ++q) {
        op->starts[q] = tot;
        tot += dlen(N, op->offsets[q]);
    }
    op->stored_elems = tot;
    const size_t bytes = size_t(std::max<int64_t>(tot, 1)) * amp_bytes(op->dtype);
    cudaMemPool_t pool = nullptr;
    DIAQ_TRY(values_pool(op->device, &pool));
    cudaError_t e = inject_now() ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync(&op->d_values, bytes, pool, s);
    if (e != cudaSuccess) {
        op->d_values = nullptr;
        return fail(DIAQ_ERR_ALLOC, "allocation of %zu bytes for stored diagonals failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    const size_t ob = std::max<size_t>(op->offsets.size(), 1) * sizeof(int64_t);
    if ((e = cudaMalloc((void**)&op->d_offsets, ob)) != cudaSuccess ||
        (e = cudaMalloc((void**)&op->d_starts, ob)) != cudaSuccess)
        return fail(DIAQ_ERR_ALLOC, "cudaMalloc for diagonal indices failed: %s", cudaGetErrorString(e));
    if (!op->offsets.empty()) {
        // ordered on the build stream (the host vectors live as long as the op)
        DIAQ_CUDA(cudaMemcpyAsync(op->d_offsets, op->offsets.data(), op->offsets.size() * 8, cudaMemcpyHostToDevice, s));
        DIAQ_CUDA(cudaMemcpyAsync(op->d_starts, op->starts.data(), op->starts.size() * 8, cudaMemcpyHostToDevice, s));
    }
    return DIAQ_OK;
}

// Finish a gate-structured op: class, offsets, device data.
static diaq_status finish_gate_op(diaq_op_s* op, const std::vector<uint8_t>* pattern, cudaStream_t s) {
    op->op_class = classify(op->gate.m, op->gate.k);
    op->real_values = std::all_of(op->gate.m.begin(), op->gate.m.end(), [](const cplx& v) { return v.imag() == 0.0; });
    op->offsets = full_offsets(op->gate, pattern);
    if (op->variant == DIAQ_ONTHEFLY) {
        if (op->gate.k > 3) DIAQ_TRY(upload_matrix(op));
        return DIAQ_OK;
    }
    DIAQ_TRY(alloc_stored(op, s));
    return launch_materialise(op, s);
}

static bool overlaps(const void* a, const void* b, size_t bytes) {
    const char* x = static_cast<const char*>(a);
    const char* y = static_cast<const char*>(b);
    return x < y + bytes && y < x + bytes;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* diaq_last_error(void) { return g_error.c_str(); }

const char* diaq_version(void) { return "diaq_gb300 0.1 (sm_103a)"; }

diaq_status diaq_gate_offsets(const diaq_gate* g, int32_t n_qubits, int64_t* offsets, int64_t cap,
                              int64_t* count) {
    clear_error();
    if (!count) return fail(DIAQ_ERR_ARG, "count is NULL");
    GateDesc d;
    // structure only: a parametric gate's offsets do not depend on theta
    if (g && g->param >= 0) {
        DIAQ_TRY(check_gate_shape(g, n_qubits));
        DIAQ_TRY(check_gen(g));
        d.k = g->k;
        for (int a = 0; a < g->k; ++a) d.targets[a] = g->targets[a];
        d.m.assign(size_t(1) << (2 * g->k), cplx(0, 0));
    } else {
        DIAQ_TRY(gate_desc_from(g, n_qubits, nullptr, &d));
    }
    const std::vector<uint8_t> pat = gate_pattern(g, d);
    const std::vector<int64_t> offs = full_offsets(d, &pat);
    *count = int64_t(offs.size());
    if (int64_t(offs.size()) > cap || (!offsets && !offs.empty()))
        return fail(DIAQ_ERR_ARG, "offset buffer holds %lld, need %zu", (long long)cap, offs.size());
    std::copy(offs.begin(), offs.end(), offsets);
    return DIAQ_OK;
}

diaq_status diaq_diaq_matmul_host(int64_t N, int64_t a_count, const int64_t* a_idx, const double* a_values,
                                  int64_t b_count, const int64_t* b_idx, const double* b_values,
                                  int64_t* c_count, int64_t* c_idx, int64_t* c_values_len,
                                  double* c_values) {
    clear_error();
    if (N < 1) return fail(DIAQ_ERR_ARG, "N = %lld < 1", (long long)N);
    if (a_count < 0 || b_count < 0 || (a_count && (!a_idx || !a_values)) || (b_count && (!b_idx || !b_values)))
        return fail(DIAQ_ERR_ARG, "bad operand arrays");
    if (!c_count || !c_values_len) return fail(DIAQ_ERR_ARG, "c_count / c_values_len is NULL");
    auto load = [&](int64_t cnt, const int64_t* idx, const double* vals, DiaMap* m, const char* nm) -> diaq_status {
        const double* p = vals;
        for (int64_t q = 0; q < cnt; ++q) {
            const int64_t d = idx[q];
            if (d <= -N || d >= N) return fail(DIAQ_ERR_SHAPE, "%s index %lld outside (-N, N)", nm, (long long)d);
            if (m->count(d)) return fail(DIAQ_ERR_ARG, "%s index %lld repeated", nm, (long long)d);
            std::vector<cplx> v(static_cast<size_t>(dlen(N, d)));
            for (size_t t = 0; t < v.size(); ++t) v[t] = cplx(p[2 * t], p[2 * t + 1]);
            p += 2 * v.size();
            m->emplace(d, std::move(v));
        }
        return DIAQ_OK;
    };
    DiaMap A, B;
    DIAQ_TRY(load(a_count, a_idx, a_values, &A, "A"));
    DIAQ_TRY(load(b_count, b_idx, b_values, &B, "B"));
    const DiaMap C = diaq_matmul(N, A, B);
    int64_t len = 0;
    for (const auto& kv : C) len += int64_t(kv.second.size());
    *c_count = int64_t(C.size());
    *c_values_len = len;
    if (!c_values) return DIAQ_OK;
    if (!c_idx) return fail(DIAQ_ERR_ARG, "c_idx is NULL");
    double* p = c_values;
    int64_t q = 0;
    for (const auto& [d, v] : C) {
        c_idx[q++] = d;
        for (const cplx& z : v) {
            *p++ = z.real();
            *p++ = z.imag();
        }
    }
    return DIAQ_OK;
}

diaq_status diaq_fuse_gates_host(const diaq_gate* gates, int32_t count, const double* theta,
                                 int32_t* union_k, int32_t* union_targets, double* fused_m) {
    clear_error();
    if (!gates || count < 1) return fail(DIAQ_ERR_ARG, "need at least one gate");
    if (!union_k || !union_targets || !fused_m) return fail(DIAQ_ERR_ARG, "NULL output");
    int nq = 0;
    for (int i = 0; i < count; ++i)
        for (int a = 0; a < gates[i].k && a < DIAQ_MAX_K; ++a) nq = std::max(nq, gates[i].targets[a] + 1);
    std::vector<GateDesc> ds(static_cast<size_t>(count));
    for (int i = 0; i < count; ++i) DIAQ_TRY(gate_desc_from(&gates[i], std::max(nq, 1), theta, &ds[size_t(i)]));
    GateDesc f;
    DIAQ_TRY(fuse_descs(ds, &f));
    *union_k = f.k;
    for (int u = 0; u < f.k; ++u) union_targets[u] = f.targets[u];
    for (size_t e = 0; e < f.m.size(); ++e) {
        fused_m[2 * e] = f.m[e].real();
        fused_m[2 * e + 1] = f.m[e].imag();
    }
    return DIAQ_OK;
}

diaq_status diaq_build(const diaq_gate* g, int32_t n_qubits, diaq_dtype dtype, diaq_variant variant,
                       const double* theta, diaq_stream_t stream, diaq_op_t* out) {
    clear_error_device();
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (variant != DIAQ_ONTHEFLY && variant != DIAQ_STORED) return fail(DIAQ_ERR_ARG, "bad variant %d", (int)variant);
    GateDesc d;
    DIAQ_TRY(gate_desc_from(g, n_qubits, theta, &d));
    const std::vector<uint8_t> pat = gate_pattern(g, d);
    diaq_op_s* op = new (std::nothrow) diaq_op_s();
    if (!op) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
    op->n = n_qubits;
    op->dtype = dtype;
    op->variant = variant;
    op->gate = d;
    cudaError_t e = cudaGetDevice(&op->device);
    if (e != cudaSuccess) {
        delete op;
        return cuda_fail(e, "cudaGetDevice");
    }
    diaq_status s = finish_gate_op(op, &pat, static_cast<cudaStream_t>(stream));
    if (s != DIAQ_OK) {
        free_op_memory(op);
        delete op;
        return s;
    }
    *out = op;
    return DIAQ_OK;
}

diaq_status diaq_build_diaq(int32_t n_qubits, int64_t count, const int64_t* indices, const double* values,
                            diaq_dtype dtype, diaq_stream_t stream, diaq_op_t* out) {
    clear_error_device();
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_qubits = %d out of range", n_qubits);
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (count < 0 || (count && (!indices || !values))) return fail(DIAQ_ERR_ARG, "bad diagonal arrays");
    const int64_t N = int64_t(1) << n_qubits;
    std::vector<std::pair<int64_t, int64_t>> idx;  // (index, input position)
    for (int64_t q = 0; q < count; ++q) {
        if (indices[q] <= -N || indices[q] >= N)
            return fail(DIAQ_ERR_SHAPE, "diagonal index %lld outside (-N, N)", (long long)indices[q]);
        idx.push_back({indices[q], q});
    }
    std::sort(idx.begin(), idx.end());
    for (size_t q = 1; q < idx.size(); ++q)
        if (idx[q].first == idx[q - 1].first) return fail(DIAQ_ERR_ARG, "diagonal index %lld repeated", (long long)idx[q].first);
    // input start of each diagonal
    std::vector<int64_t> in_start(static_cast<size_t>(count));
    int64_t pos = 0;
    for (int64_t q = 0; q < count; ++q) {
        in_start[size_t(q)] = pos;
        pos += dlen(N, indices[q]);
    }
    diaq_op_s* op = new (std::nothrow) diaq_op_s();
    if (!op) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
    op->n = n_qubits;
    op->dtype = dtype;
    op->variant = DIAQ_STORED;
    op->op_class = DIAQ_CLASS_RAW;
    cudaError_t e = cudaGetDevice(&op->device);
    if (e != cudaSuccess) {
        delete op;
        return cuda_fail(e, "cudaGetDevice");
    }
    for (auto& p : idx) op->offsets.push_back(p.first);
    op->real_values = true;
    for (int64_t t = 0; t < pos && op->real_values; ++t) op->real_values = values[2 * t + 1] == 0.0;
    diaq_status s = alloc_stored(op, static_cast<cudaStream_t>(stream));
    if (s == DIAQ_OK) {
        // host staging in the op's precision, sorted order
        const size_t ab = amp_bytes(dtype);
        std::vector<unsigned char> buf(static_cast<size_t>(std::max<int64_t>(op->stored_elems, 1)) * ab);
        for (size_t q = 0; q < idx.size(); ++q) {
            const double* src = values + 2 * in_start[size_t(idx[q].second)];
            const int64_t len = dlen(N, idx[q].first);
            for (int64_t t = 0; t < len; ++t) {
                const size_t at = size_t(op->starts[q] + t);
                if (dtype == DIAQ_C128) {
                    reinterpret_cast<double*>(buf.data())[2 * at] = src[2 * t];
                    reinterpret_cast<double*>(buf.data())[2 * at + 1] = src[2 * t + 1];
                } else {
                    reinterpret_cast<float*>(buf.data())[2 * at] = float(src[2 * t]);
                    reinterpret_cast<float*>(buf.data())[2 * at + 1] = float(src[2 * t + 1]);
                }
            }
        }
        e = cudaMemcpyAsync(op->d_values, buf.data(), size_t(op->stored_elems) * ab, cudaMemcpyHostToDevice,
                            static_cast<cudaStream_t>(stream));
        if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) s = cuda_fail(e, "upload of DiaQ diagonals");
    }
    if (s != DIAQ_OK) {
        free_op_memory(op);
        delete op;
        return s;
    }
    *out = op;
    return DIAQ_OK;
}

diaq_status diaq_op_destroy(diaq_op_t op) {
    clear_error();
    if (!op) return DIAQ_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != op->device) cudaSetDevice(op->device);
    cudaError_t e = cudaDeviceSynchronize();
    diaq_status s = free_op_memory(op);
    if (cur >= 0 && cur != op->device) cudaSetDevice(cur);
    delete op;
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize (op destroy)");
    return s;
}

diaq_status diaq_op_query(diaq_op_t op, diaq_op_info* info) {
    clear_error();
    if (!op || !info) return fail(DIAQ_ERR_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n_qubits = op->n;
    info->dtype = op->dtype;
    info->variant = op->variant;
    info->op_class = op->op_class;
    info->k = op->op_class == DIAQ_CLASS_RAW ? 0 : op->gate.k;
    for (int a = 0; a < info->k; ++a) info->targets[a] = op->gate.targets[a];
    info->n_diagonals = int64_t(op->offsets.size());
    info->stored_bytes = op->variant == DIAQ_STORED ? op->stored_elems * int64_t(amp_bytes(op->dtype)) : 0;
    info->real_values = op->real_values ? 1 : 0;
    return DIAQ_OK;
}

diaq_status diaq_op_offsets(diaq_op_t op, int64_t* offsets, int64_t cap, int64_t* count) {
    clear_error();
    if (!op || !count) return fail(DIAQ_ERR_ARG, "NULL argument");
    *count = int64_t(op->offsets.size());
    if (*count > cap || (!offsets && *count)) return fail(DIAQ_ERR_ARG, "offset buffer too small");
    std::copy(op->offsets.begin(), op->offsets.end(), offsets);
    return DIAQ_OK;
}

diaq_status diaq_op_read_diagonal(diaq_op_t op, int64_t which, void* host_out, diaq_stream_t stream) {
    clear_error_device();
    DIAQ_TRY(check_op(op));
    if (op->variant != DIAQ_STORED) return fail(DIAQ_ERR_ARG, "op is on-the-fly: no stored diagonals");
    if (which < 0 || which >= int64_t(op->offsets.size())) return fail(DIAQ_ERR_ARG, "diagonal %lld out of range", (long long)which);
    if (!host_out) return fail(DIAQ_ERR_ARG, "host_out is NULL");
    const int64_t N = int64_t(1) << op->n;
    const size_t ab = amp_bytes(op->dtype);
    const char* src = static_cast<const char*>(op->d_values) + size_t(op->starts[size_t(which)]) * ab;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DIAQ_CUDA(cudaMemcpyAsync(host_out, src, size_t(dlen(N, op->offsets[size_t(which)])) * ab, cudaMemcpyDeviceToHost, s));
    DIAQ_CUDA(cudaStreamSynchronize(s));
    return DIAQ_OK;
}

diaq_status diaq_fuse(const diaq_op_t* ops, int32_t count, diaq_variant variant, diaq_stream_t stream,
                      diaq_op_t* out) {
    clear_error_device();
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ops || count < 1) return fail(DIAQ_ERR_ARG, "need at least one op");
    if (variant != DIAQ_ONTHEFLY && variant != DIAQ_STORED) return fail(DIAQ_ERR_ARG, "bad variant %d", (int)variant);
    bool raw = false;
    for (int i = 0; i < count; ++i) {
        DIAQ_TRY(check_op(ops[i]));
        if (ops[i]->n != ops[0]->n || ops[i]->dtype != ops[0]->dtype)
            return fail(DIAQ_ERR_SHAPE, "op %d is not multiplyable with op 0 (qubits or dtype differ)", i);
        raw |= ops[i]->op_class == DIAQ_CLASS_RAW;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!raw) {
        std::vector<GateDesc> ds;
        for (int i = 0; i < count; ++i) ds.push_back(ops[i]->gate);
        GateDesc f;
        DIAQ_TRY(fuse_descs(ds, &f));
        diaq_op_s* op = new (std::nothrow) diaq_op_s();
        if (!op) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
        op->n = ops[0]->n;
        op->dtype = ops[0]->dtype;
        op->variant = variant;
        op->device = ops[0]->device;
        op->gate = f;
        diaq_status st = finish_gate_op(op, nullptr, s);
        if (st != DIAQ_OK) {
            free_op_memory(op);
            delete op;
            return st;
        }
        *out = op;
        return DIAQ_OK;
    }
    // device Algorithm 1 over full-system diagonals, left to right: C = ops[i] C
    for (int i = 0; i < count; ++i)
        if (ops[i]->variant != DIAQ_STORED)
            return fail(DIAQ_ERR_UNSUPPORTED, "fusing a raw DiaQ op needs every op stored (op %d is on-the-fly)", i);
    diaq_op_s* cur = nullptr;
    for (int i = 1; i < count; ++i) {
        diaq_op_s* c = new (std::nothrow) diaq_op_s();
        if (!c) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
        c->n = ops[0]->n;
        c->dtype = ops[0]->dtype;
        c->variant = DIAQ_STORED;
        c->op_class = DIAQ_CLASS_RAW;
        c->device = ops[0]->device;
        const diaq_op_s* right = cur ? cur : ops[0];
        c->real_values = ops[i]->real_values && right->real_values;
        diaq_status st = launch_spgemm(ops[i], right, c, s);
        if (cur) {
            free_op_memory(cur);
            delete cur;
        }
        if (st != DIAQ_OK) {
            free_op_memory(c);
            delete c;
            return st;
        }
        cur = c;
    }
    if (!cur) {
        // single op: copy it
        diaq_op_s* c = new (std::nothrow) diaq_op_s();
        if (!c) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
        *c = diaq_op_s();
        c->n = ops[0]->n;
        c->dtype = ops[0]->dtype;
        c->variant = DIAQ_STORED;
        c->op_class = DIAQ_CLASS_RAW;
        c->device = ops[0]->device;
        c->offsets = ops[0]->offsets;
        c->real_values = ops[0]->real_values;
        diaq_status st = alloc_stored(c, s);
        if (st == DIAQ_OK) {
            cudaError_t e = cudaMemcpyAsync(c->d_values, ops[0]->d_values, size_t(c->stored_elems) * amp_bytes(c->dtype),
                                            cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) st = cuda_fail(e, "cudaMemcpyAsync(copy op)");
        }
        if (st != DIAQ_OK) {
            free_op_memory(c);
            delete c;
            return st;
        }
        cur = c;
    }
    *out = cur;
    return DIAQ_OK;
}

diaq_status diaq_apply(diaq_op_t op, const void* x, void* y, diaq_stream_t stream) {
    clear_error_device();
    DIAQ_TRY(check_op(op));
    if (!x || !y) return fail(DIAQ_ERR_ARG, "x or y is NULL");
    const size_t bytes = (size_t(1) << op->n) * amp_bytes(op->dtype);
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
        return fail(DIAQ_ERR_ARG, "state buffers must be 16-byte aligned");
    const bool inplace = x == y;
    if (inplace && op->variant == DIAQ_STORED) return fail(DIAQ_ERR_ARG, "stored ops cannot run in place (x == y)");
    if (!inplace && overlaps(x, y, bytes)) return fail(DIAQ_ERR_ARG, "x and y overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (inplace) {
        bool done = false;
        DIAQ_TRY(launch_inplace_skip(op, y, s, &done));
        if (done) return DIAQ_OK;
    }
    if (op->variant == DIAQ_ONTHEFLY) return launch_onthefly(op, x, y, s);
    return launch_stored(op, x, y, s);
}

diaq_status diaq_op_apply_bytes(diaq_op_t op, int32_t in_place, int64_t* bytes) {
    clear_error();
    if (!op || !bytes) return fail(DIAQ_ERR_ARG, "NULL argument");
    const int64_t N = int64_t(1) << op->n;
    const int64_t s = int64_t(amp_bytes(op->dtype));
    if (op->variant == DIAQ_STORED) {
        if (in_place) return fail(DIAQ_ERR_ARG, "stored ops cannot run in place");
        *bytes = 2 * N * s + stored_values_read(op) * s;
    } else if (in_place) {
        *bytes = inplace_bytes(op->n, op->dtype, op->gate);
    } else {
        *bytes = 2 * N * s;
    }
    return DIAQ_OK;
}

// ---------------------------------------------------------------------------
// Unitary simulation (Section II-A; per-time-step sparsity of Section III-A)
// ---------------------------------------------------------------------------
diaq_status diaq_op_diagonal_nnz(diaq_op_t op, int64_t* nnz, diaq_stream_t stream) {
    clear_error_device();
    DIAQ_TRY(check_op(op));
    if (!nnz) return fail(DIAQ_ERR_ARG, "nnz is NULL");
    if (op->variant != DIAQ_STORED) return fail(DIAQ_ERR_ARG, "op is on-the-fly: no stored diagonals");
    std::vector<int64_t> c;
    DIAQ_TRY(count_diagonal_nnz(op, &c, static_cast<cudaStream_t>(stream)));
    std::copy(c.begin(), c.end(), nnz);
    return DIAQ_OK;
}

// A stored raw op holding the diagonals of src whose count is non-zero.
static diaq_status prune_with_counts(const diaq_op_s* src, const std::vector<int64_t>& counts, cudaStream_t s,
                                     diaq_op_s** out) {
    *out = nullptr;
    diaq_op_s* c = new (std::nothrow) diaq_op_s();
    if (!c) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
    c->n = src->n;
    c->dtype = src->dtype;
    c->variant = DIAQ_STORED;
    c->op_class = DIAQ_CLASS_RAW;
    c->device = src->device;
    c->real_values = src->real_values;
    std::vector<int32_t> keep;
    for (size_t q = 0; q < src->offsets.size(); ++q)
        if (counts[q] > 0) {
            keep.push_back(int32_t(q));
            c->offsets.push_back(src->offsets[q]);
        }
    diaq_status st = alloc_stored(c, s);
    if (st == DIAQ_OK) st = launch_gather_diagonals(src, keep, c, s);
    if (st != DIAQ_OK) {
        free_op_memory(c);
        delete c;
        return st;
    }
    *out = c;
    return DIAQ_OK;
}

diaq_status diaq_op_prune(diaq_op_t op, diaq_stream_t stream, diaq_op_t* out) {
    clear_error_device();
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    DIAQ_TRY(check_op(op));
    if (op->variant != DIAQ_STORED) return fail(DIAQ_ERR_ARG, "op is on-the-fly: no stored diagonals");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int64_t> counts;
    DIAQ_TRY(count_diagonal_nnz(op, &counts, s));
    return prune_with_counts(op, counts, s, out);
}

diaq_status diaq_unitary_chain(const diaq_gate* gates, int32_t n_gates, const double* theta, int32_t n_qubits,
                               diaq_dtype dtype, int32_t prune, int64_t* n_diagonals, int64_t* nnz,
                               diaq_stream_t stream, diaq_op_t* out) {
    clear_error_device();
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!gates || n_gates < 1) return fail(DIAQ_ERR_ARG, "need at least one gate");
    if (n_qubits < 1 || n_qubits > 15) return fail(DIAQ_ERR_ARG, "unitary chain needs 1 <= n_qubits <= 15 (got %d)", n_qubits);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    diaq_op_s* U = nullptr;
    auto drop = [](diaq_op_s* p) {
        if (p) {
            free_op_memory(p);
            delete p;
        }
    };
    for (int t = 0; t < n_gates; ++t) {
        diaq_op_t g = nullptr;
        diaq_status st = diaq_build(&gates[t], n_qubits, dtype, DIAQ_STORED, theta, stream, &g);
        if (st != DIAQ_OK) {
            drop(U);
            return st;
        }
        diaq_op_s* C = nullptr;
        if (!U) {
            C = g;  // the first time step is the unitary so far
            C->op_class = DIAQ_CLASS_RAW;
        } else {
            C = new (std::nothrow) diaq_op_s();
            if (!C) {
                drop(U);
                drop(g);
                return fail(DIAQ_ERR_ALLOC, "host allocation failed");
            }
            C->n = n_qubits;
            C->dtype = dtype;
            C->variant = DIAQ_STORED;
            C->op_class = DIAQ_CLASS_RAW;
            C->device = g->device;
            C->real_values = g->real_values && U->real_values;
            st = launch_spgemm(g, U, C, s);  // C = G_t U (Algorithm 1)
            drop(U);
            drop(g);
            U = nullptr;
            if (st != DIAQ_OK) {
                drop(C);
                return st;
            }
        }
        std::vector<int64_t> counts;
        if (prune || nnz) {
            st = count_diagonal_nnz(C, &counts, s);
            if (st != DIAQ_OK) {
                drop(C);
                return st;
            }
        }
        if (prune) {
            diaq_op_s* P = nullptr;
            st = prune_with_counts(C, counts, s, &P);
            drop(C);
            if (st != DIAQ_OK) return st;
            C = P;
        }
        U = C;
        if (n_diagonals) n_diagonals[t] = int64_t(U->offsets.size());
        if (nnz) {
            int64_t z = 0;
            for (int64_t v : counts) z += v;
            nnz[t] = z;
        }
    }
    *out = U;
    return DIAQ_OK;
}

static int mem_kind(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;  // unknown: treat as pageable host
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 1;
    return 0;
}

// The slices of an op (on the fly, k <= 3) for copies that overlap it: its
// 2^(n-k) groups split into 2^b ranges by the top b non-target bits. Slice
// s holds the amplitudes whose b highest non-target bits equal s; in memory
// that is one contiguous run of 2^L amplitudes (L the lowest of those bits)
// per setting of the targets above L.
namespace {
struct Slice {
    int64_t g_begin, g_end;
    std::vector<int64_t> runs;  // first amplitude of each run
};
struct SlicePlan {
    int64_t run_len = 0;
    std::vector<Slice> slices;
};

bool plan_slices(const diaq_op_s* op, int b, SlicePlan* out) {
    if (op->variant != DIAQ_ONTHEFLY || op->op_class == DIAQ_CLASS_RAW) return false;
    const int n = op->n, k = op->gate.k;
    if (k < 1 || k > 3 || n - k < b + 1) return false;
    std::vector<int> nt, above;
    for (int q = 0; q < n; ++q) {
        bool t = false;
        for (int a = 0; a < k; ++a) t |= op->gate.targets[a] == q;
        if (!t) nt.push_back(q);
    }
    const int L = nt[size_t(n - k - b)];
    for (int a = 0; a < k; ++a)
        if (op->gate.targets[a] > L) above.push_back(op->gate.targets[a]);
    const int64_t per = (int64_t(1) << (n - k)) >> b;
    out->run_len = int64_t(1) << L;
    out->slices.assign(size_t(1) << b, Slice{});
    for (int64_t s = 0; s < (int64_t(1) << b); ++s) {
        Slice& sl = out->slices[size_t(s)];
        sl.g_begin = s * per;
        sl.g_end = sl.g_begin + per;
        int64_t base = 0;
        for (int i = 0; i < b; ++i)
            if ((s >> i) & 1) base |= int64_t(1) << nt[size_t(n - k - b + i)];
        for (int64_t c = 0; c < (int64_t(1) << above.size()); ++c) {
            int64_t st = base;
            for (size_t j = 0; j < above.size(); ++j)
                if ((c >> j) & 1) st |= int64_t(1) << above[j];
            sl.runs.push_back(st);
        }
    }
    return true;
}

// An on-the-fly op in place on groups [g0, g1) (k <= 3), or on all of them.
diaq_status run_inplace(const diaq_op_s* op, void* x, int64_t g0, int64_t g1, cudaStream_t s) {
    bool done = false;
    DIAQ_TRY(launch_inplace_skip_range(op, x, g0, g1, s, &done));
    if (done) return DIAQ_OK;
    if (op->gate.k <= 3) return launch_gate_local_range(op->n, op->dtype, op->gate, x, x, g0, g1, s);
    return launch_onthefly(op, x, x, s);
}

// Deferred scalars of a complex128 simulation. A one-qubit gate whose rows
// each have an entry of the largest magnitude sigma (RX, RY, H and the
// like: gate_scaled1_sigma) runs as V = U / sigma, one fused multiply-add
// per real component instead of two or three FP64 instructions; the stored
// state is then the true one divided by F, the product of the sigmas so far.
// The last such gate of the circuit (or one where F has fallen below 2^-400,
// so that the stored amplitudes stay far from overflow) runs as F U
// instead, which makes the stored state the true one again; every other gate
// is linear and leaves F alone.
enum SimAction { SIM_PLAIN = 0, SIM_SCALED = 1, SIM_FOLD = 2 };

struct SimStep {
    int action = SIM_PLAIN;
    GateDesc folded;  // SIM_FOLD: F U
};

static std::vector<SimStep> plan_sim_scaling(const diaq_op_t* ops, int count) {
    std::vector<SimStep> st(static_cast<size_t>(count));
    std::vector<double> sig(static_cast<size_t>(count), 0.0);
    int last = -1;
    for (int i = 0; i < count; ++i) {
        const diaq_op_s* op = ops[i];
        if (op->dtype == DIAQ_C128 && op->variant == DIAQ_ONTHEFLY && op->gate.k == 1 &&
            gate_scaled1_sigma(op->gate, &sig[size_t(i)]))
            last = i;
        else
            sig[size_t(i)] = 0.0;
    }
    double F = 1.0;
    for (int i = 0; i <= last; ++i) {
        if (sig[size_t(i)] == 0.0) continue;
        if (i == last || F < 0x1p-400) {
            SimStep& x = st[size_t(i)];
            x.action = SIM_FOLD;
            x.folded = ops[i]->gate;
            for (cplx& v : x.folded.m) v *= F;
            F = 1.0;
        } else {
            st[size_t(i)].action = SIM_SCALED;
            F *= sig[size_t(i)];
        }
    }
    return st;
}

// Runs of consecutive diagonal on-the-fly ops (plain steps) whose union of
// targets has at most DIAG_BIG_K qubits, merged by diaq_simulate into one
// pass each (k_apply_bigdiag): the table holds, for every value of the
// union's bits, the product of the ops' diagonal entries, so every changed
// amplitude takes one complex multiply for the whole run.
struct SimMerge {
    int first = 0, last = 0;  // ops [first, last]
    BigDiagArgs args{};
    size_t tab_off = 0, skip_off = 0;
};

static std::vector<SimMerge> plan_diag_merges(const diaq_op_t* ops, int lo, int hi, const std::vector<SimStep>& steps,
                                              diaq_dtype dt, std::vector<double2>* tab, std::vector<uint32_t>* skip) {
    std::vector<SimMerge> out;
    auto eligible = [&](int i) {
        return ops[i]->variant == DIAQ_ONTHEFLY && steps[size_t(i)].action == SIM_PLAIN && is_diagonal(ops[i]->gate);
    };
    for (int i = lo; i < hi;) {
        if (!eligible(i)) {
            ++i;
            continue;
        }
        uint64_t qs = 0;
        for (int a = 0; a < ops[i]->gate.k; ++a) qs |= uint64_t(1) << ops[i]->gate.targets[a];
        int j = i;
        while (j + 1 < hi && eligible(j + 1)) {
            uint64_t q2 = qs;
            for (int a = 0; a < ops[j + 1]->gate.k; ++a) q2 |= uint64_t(1) << ops[j + 1]->gate.targets[a];
            if (__builtin_popcountll(q2) > DIAG_BIG_K) break;
            qs = q2;
            ++j;
        }
        if (j == i) {
            ++i;
            continue;
        }
        SimMerge m;
        m.first = i;
        m.last = j;
        m.args.k = __builtin_popcountll(qs);
        int pos[64];
        for (int b = 0, q = 0; b < 64; ++b)
            if ((qs >> b) & 1) {
                m.args.t[q] = b;
                pos[b] = q++;
            }
        const size_t E = size_t(1) << m.args.k;
        m.tab_off = tab->size();
        m.skip_off = skip->size();
        skip->resize(skip->size() + (E + 31) / 32, 0u);
        for (size_t c = 0; c < E; ++c) {
            cplx v(1.0, 0.0);
            for (int o = i; o <= j; ++o) {
                const GateDesc& g = ops[o]->gate;
                const int D = 1 << g.k;
                int l = 0;
                for (int a = 0; a < g.k; ++a) l |= int((c >> pos[g.targets[a]]) & 1) << (g.k - 1 - a);
                v *= g.m[size_t(l) * D + l];
            }
            tab->push_back(make_double2(v.real(), v.imag()));
            const bool one = dt == DIAQ_C128 ? (v.real() == 1.0 && v.imag() == 0.0)
                                             : (float(v.real()) == 1.0f && float(v.imag()) == 0.0f);
            if (one) (*skip)[m.skip_off + c / 32] |= 1u << (c % 32);
        }
        out.push_back(m);
        i = j + 1;
    }
    return out;
}

// Two ops that diaq_simulate runs in one pass: on-the-fly, one qubit each,
// different qubits, every entry non-zero (so neither has identity rows to
// skip or structural zeros to exploit).
static bool sim_pairable(const diaq_op_s* a, const diaq_op_s* b) {
    auto dense1 = [](const diaq_op_s* o) {
        if (o->variant != DIAQ_ONTHEFLY || o->gate.k != 1 || o->gate.m.size() != 4) return false;
        for (const cplx& v : o->gate.m)
            if (v == cplx(0.0, 0.0)) return false;
        return true;
    };
    return dense1(a) && dense1(b) && a->gate.targets[0] != b->gate.targets[0];
}

static diaq_status run_inplace_step(const diaq_op_s* op, const SimStep& st, void* x, int64_t g0, int64_t g1,
                                    cudaStream_t s) {
    if (st.action == SIM_SCALED) {
        double sigma = 0.0;
        return launch_gate_scaled1_range(op->n, op->gate, x, x, g0, g1, &sigma, s);
    }
    if (st.action == SIM_FOLD) return launch_gate_local_range(op->n, op->dtype, st.folded, x, x, g0, g1, s);
    return run_inplace(op, x, g0, g1, s);
}

// Streams, events and device buffers of one diaq_simulate call, released on
// every path.
struct SimResources {
    cudaStream_t cin = nullptr, cout = nullptr;
    std::vector<cudaEvent_t> events;
    std::vector<std::pair<void*, cudaStream_t>> dev;  // stream-ordered allocations
    cudaEvent_t make(bool timing) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, timing ? cudaEventDefault : cudaEventDisableTiming) != cudaSuccess) return nullptr;
        events.push_back(e);
        return e;
    }
    ~SimResources() {
        for (auto& d : dev) cudaFreeAsync(d.first, d.second);
        for (auto& d : dev) cudaStreamSynchronize(d.second);
        if (cin) cudaStreamSynchronize(cin);
        if (cout) cudaStreamSynchronize(cout);
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        if (cin) cudaStreamDestroy(cin);
        if (cout) cudaStreamDestroy(cout);
    }
};
}  // namespace

diaq_status diaq_simulate_timed(const diaq_op_t* ops, int32_t count, const void* psi_in, void* psi_out, void* work0,
                                void* work1, diaq_stream_t stream, float* timeline_ms) {
    clear_error_device();
    if (count < 0 || (count && !ops)) return fail(DIAQ_ERR_ARG, "bad op list");
    if (!psi_in || !psi_out || !work0) return fail(DIAQ_ERR_ARG, "NULL state or work buffer");
    if (count == 0) return fail(DIAQ_ERR_ARG, "empty circuit: nothing to infer the state size from");
    const int n = ops[0]->n;
    const diaq_dtype dt = ops[0]->dtype;
    bool any_stored = false;
    for (int i = 0; i < count; ++i) {
        DIAQ_TRY(check_op(ops[i]));
        if (ops[i]->n != n || ops[i]->dtype != dt) return fail(DIAQ_ERR_SHAPE, "op %d has another size or dtype", i);
        any_stored |= ops[i]->variant == DIAQ_STORED;
    }
    if (any_stored && !work1) return fail(DIAQ_ERR_ARG, "stored ops need a second work buffer");
    const std::vector<SimStep> steps = plan_sim_scaling(ops, count);
    if (mem_kind(work0) != 1 || (work1 && mem_kind(work1) != 1)) return fail(DIAQ_ERR_ARG, "work buffers must be device memory");
    const size_t s_amp = amp_bytes(dt);
    const size_t bytes = (size_t(1) << n) * s_amp;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool in_host = !mem_kind(psi_in), out_host = !mem_kind(psi_out);
    // host copies overlap the first op (input) and the last op (output),
    // slice by slice, when those ops run in place on the fly with k <= 3
    constexpr int kSliceBits = 4;
    SlicePlan pin, pout;
    const bool pipe_in = in_host && plan_slices(ops[0], kSliceBits, &pin);
    const bool pipe_out = out_host && plan_slices(ops[count - 1], kSliceBits, &pout) && (count > 1 || pipe_in);
    SimResources R;
    const bool timing = timeline_ms != nullptr;
    cudaEvent_t t_start = nullptr, t_in = nullptr, t_compute = nullptr, t_end = nullptr;
    if (timing) {
        t_start = R.make(true);
        t_in = R.make(true);
        t_compute = R.make(true);
        t_end = R.make(true);
        if (!t_start || !t_in || !t_compute || !t_end) return fail(DIAQ_ERR_CUDA, "cudaEventCreate failed");
        DIAQ_CUDA(cudaEventRecord(t_start, s));
    }
    if (pipe_in || pipe_out) {
        cudaEvent_t e0 = R.make(false);
        if (!e0) return fail(DIAQ_ERR_CUDA, "cudaEventCreate failed");
        DIAQ_CUDA(cudaStreamCreateWithFlags(&R.cin, cudaStreamNonBlocking));
        DIAQ_CUDA(cudaStreamCreateWithFlags(&R.cout, cudaStreamNonBlocking));
        // the copies start after the work already queued on `stream`
        DIAQ_CUDA(cudaEventRecord(e0, s));
        DIAQ_CUDA(cudaStreamWaitEvent(R.cin, e0, 0));
        DIAQ_CUDA(cudaStreamWaitEvent(R.cout, e0, 0));
    }
    int first = 0, last = count;  // ops [first, last) run whole below
    bool out_sent = false;        // the output copy is already queued
    if (pipe_in) {
        const size_t run_bytes = size_t(pin.run_len) * s_amp;
        std::vector<cudaEvent_t> got(pin.slices.size());
        for (size_t j = 0; j < pin.slices.size(); ++j) {
            for (int64_t r : pin.slices[j].runs)
                DIAQ_CUDA(cudaMemcpyAsync(static_cast<char*>(work0) + size_t(r) * s_amp,
                                          static_cast<const char*>(psi_in) + size_t(r) * s_amp, run_bytes,
                                          cudaMemcpyHostToDevice, R.cin));
            got[j] = R.make(false);
            if (!got[j]) return fail(DIAQ_ERR_CUDA, "cudaEventCreate failed");
            DIAQ_CUDA(cudaEventRecord(got[j], R.cin));
        }
        if (timing) DIAQ_CUDA(cudaEventRecord(t_in, R.cin));
        const bool also_out = pipe_out && count == 1;
        const size_t out_run_bytes = size_t(pout.run_len) * s_amp;
        for (size_t j = 0; j < pin.slices.size(); ++j) {
            DIAQ_CUDA(cudaStreamWaitEvent(s, got[j], 0));
            DIAQ_TRY(run_inplace_step(ops[0], steps[0], work0, pin.slices[j].g_begin, pin.slices[j].g_end, s));
            if (also_out) {  // one op: each slice leaves as soon as it is done
                cudaEvent_t done = R.make(false);
                if (!done) return fail(DIAQ_ERR_CUDA, "cudaEventCreate failed");
                DIAQ_CUDA(cudaEventRecord(done, s));
                DIAQ_CUDA(cudaStreamWaitEvent(R.cout, done, 0));
                for (int64_t r : pout.slices[j].runs)
                    DIAQ_CUDA(cudaMemcpyAsync(static_cast<char*>(psi_out) + size_t(r) * s_amp,
                                              static_cast<const char*>(work0) + size_t(r) * s_amp, out_run_bytes,
                                              cudaMemcpyDeviceToHost, R.cout));
            }
        }
        first = 1;
        out_sent = also_out;
    } else {
        const cudaMemcpyKind kin = in_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (psi_in != work0) DIAQ_CUDA(cudaMemcpyAsync(work0, psi_in, bytes, kin, s));
        if (timing) DIAQ_CUDA(cudaEventRecord(t_in, s));
    }
    if (pipe_out && !out_sent) last = count - 1;
    // merged diagonal runs: their tables go to the device once, on `stream`
    std::vector<double2> mtab;
    std::vector<uint32_t> mskip;
    const std::vector<SimMerge> merges = plan_diag_merges(ops, first, last, steps, dt, &mtab, &mskip);
    double2* d_mtab = nullptr;
    if (!merges.empty()) {
        const size_t tb = mtab.size() * sizeof(double2), sb = mskip.size() * sizeof(uint32_t);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_mtab), tb + sb, s);
        if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(merged diagonal tables): %s", cudaGetErrorString(e));
        R.dev.push_back({d_mtab, s});
        DIAQ_CUDA(cudaMemcpyAsync(d_mtab, mtab.data(), tb, cudaMemcpyHostToDevice, s));
        DIAQ_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(d_mtab) + tb, mskip.data(), sb, cudaMemcpyHostToDevice, s));
    }
    const uint32_t* d_mskip =
        d_mtab ? reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(d_mtab) + mtab.size() * sizeof(double2))
               : nullptr;
    size_t next_merge = 0;
    void* cur = work0;
    void* other = work1;
    for (int i = first; i < last; ++i) {
        if (next_merge < merges.size() && merges[next_merge].first == i) {
            const SimMerge& m = merges[next_merge++];
            DIAQ_TRY(launch_bigdiag_inplace(n, dt, m.args, d_mtab + m.tab_off, d_mskip + m.skip_off, cur, s));
            i = m.last;
            continue;
        }
        // two consecutive one-qubit ops with no zero entry on different
        // qubits run in one pass (k_apply_pair1), each in its own form
        if (i + 1 < last && sim_pairable(ops[i], ops[i + 1])) {
            const SimStep& sa = steps[size_t(i)];
            const SimStep& sb = steps[size_t(i + 1)];
            DIAQ_TRY(launch_pair1_inplace(n, dt, sa.action == SIM_FOLD ? sa.folded : ops[i]->gate,
                                          sa.action == SIM_SCALED, sb.action == SIM_FOLD ? sb.folded : ops[i + 1]->gate,
                                          sb.action == SIM_SCALED, cur, s));
            ++i;
            continue;
        }
        if (ops[i]->variant == DIAQ_ONTHEFLY) {
            DIAQ_TRY(run_inplace_step(ops[i], steps[size_t(i)], cur, 0,
                                      ops[i]->gate.k <= 3 ? int64_t(1) << (n - ops[i]->gate.k) : 0, s));
        } else {
            DIAQ_TRY(launch_stored(ops[i], cur, other, s));
            std::swap(cur, other);
        }
    }
    if (pipe_out && !out_sent) {
        // the last op (on the fly) runs in place on the current buffer,
        // slice by slice, and each slice goes out as soon as it is done
        const size_t run_bytes = size_t(pout.run_len) * s_amp;
        for (size_t j = 0; j < pout.slices.size(); ++j) {
            DIAQ_TRY(run_inplace_step(ops[count - 1], steps[size_t(count - 1)], cur, pout.slices[j].g_begin,
                                      pout.slices[j].g_end, s));
            cudaEvent_t done = R.make(false);
            if (!done) return fail(DIAQ_ERR_CUDA, "cudaEventCreate failed");
            DIAQ_CUDA(cudaEventRecord(done, s));
            DIAQ_CUDA(cudaStreamWaitEvent(R.cout, done, 0));
            for (int64_t r : pout.slices[j].runs)
                DIAQ_CUDA(cudaMemcpyAsync(static_cast<char*>(psi_out) + size_t(r) * s_amp,
                                          static_cast<const char*>(cur) + size_t(r) * s_amp, run_bytes,
                                          cudaMemcpyDeviceToHost, R.cout));
        }
    }
    if (timing) DIAQ_CUDA(cudaEventRecord(t_compute, s));
    if (pipe_out) {
        cudaEvent_t copied = R.make(false);
        if (!copied) return fail(DIAQ_ERR_CUDA, "cudaEventCreate failed");
        DIAQ_CUDA(cudaEventRecord(copied, R.cout));
        DIAQ_CUDA(cudaStreamWaitEvent(s, copied, 0));
    } else {
        const cudaMemcpyKind kout = out_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (psi_out != cur) DIAQ_CUDA(cudaMemcpyAsync(psi_out, cur, bytes, kout, s));
    }
    if (R.cin) {  // nothing on `stream` may outlive this call's input copies
        cudaEvent_t in_done = R.make(false);
        if (!in_done) return fail(DIAQ_ERR_CUDA, "cudaEventCreate failed");
        DIAQ_CUDA(cudaEventRecord(in_done, R.cin));
        DIAQ_CUDA(cudaStreamWaitEvent(s, in_done, 0));
    }
    if (timing) DIAQ_CUDA(cudaEventRecord(t_end, s));
    DIAQ_CUDA(cudaStreamSynchronize(s));
    if (timing) {
        DIAQ_CUDA(cudaEventElapsedTime(&timeline_ms[0], t_start, t_in));
        DIAQ_CUDA(cudaEventElapsedTime(&timeline_ms[1], t_start, t_compute));
        DIAQ_CUDA(cudaEventElapsedTime(&timeline_ms[2], t_start, t_end));
    }
    return DIAQ_OK;
}

diaq_status diaq_simulate_bytes(const diaq_op_t* ops, int32_t count, int64_t* bytes) {
    clear_error();
    if (count < 0 || (count && !ops) || !bytes) return fail(DIAQ_ERR_ARG, "bad op list or NULL bytes");
    *bytes = 0;
    if (count == 0) return DIAQ_OK;
    const int n = ops[0]->n;
    const diaq_dtype dt = ops[0]->dtype;
    for (int i = 0; i < count; ++i) {
        if (!ops[i]) return fail(DIAQ_ERR_ARG, "op %d is NULL", i);
        if (ops[i]->n != n || ops[i]->dtype != dt) return fail(DIAQ_ERR_SHAPE, "op %d has another size or dtype", i);
    }
    const int64_t N = int64_t(1) << n;
    const int64_t s = int64_t(amp_bytes(dt));
    const std::vector<SimStep> steps = plan_sim_scaling(ops, count);
    std::vector<double2> tab;
    std::vector<uint32_t> skip;
    const std::vector<SimMerge> merges = plan_diag_merges(ops, 0, count, steps, dt, &tab, &skip);
    size_t next_merge = 0;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (next_merge < merges.size() && merges[next_merge].first == i) {
            const SimMerge& m = merges[next_merge++];
            const int64_t E = int64_t(1) << m.args.k;
            int64_t changed = 0;
            for (int64_t c = 0; c < E; ++c)
                if (!((skip[m.skip_off + size_t(c / 32)] >> (c % 32)) & 1)) ++changed;
            total += 2 * (N / E) * changed * s;
            i = m.last;
            continue;
        }
        if (i + 1 < count && sim_pairable(ops[i], ops[i + 1])) {
            total += 2 * N * s;
            ++i;
            continue;
        }
        int64_t b = 0;
        DIAQ_TRY(diaq_op_apply_bytes(ops[i], ops[i]->variant == DIAQ_ONTHEFLY ? 1 : 0, &b));
        total += b;
    }
    *bytes = total;
    return DIAQ_OK;
}

diaq_status diaq_simulate(const diaq_op_t* ops, int32_t count, const void* psi_in, void* psi_out, void* work0,
                          void* work1, diaq_stream_t stream) {
    return diaq_simulate_timed(ops, count, psi_in, psi_out, work0, work1, stream, nullptr);
}

static diaq_status check_state(const void* psi, int n, diaq_dtype dt) {
    if (!psi) return fail(DIAQ_ERR_ARG, "state is NULL");
    if (n < 1 || n > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_qubits = %d out of range", n);
    if (dt != DIAQ_C64 && dt != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dt);
    if (reinterpret_cast<uintptr_t>(psi) & 15) return fail(DIAQ_ERR_ARG, "state buffer must be 16-byte aligned");
    return DIAQ_OK;
}

diaq_status diaq_norm(const void* psi, int32_t n_qubits, diaq_dtype dtype, double* out, diaq_stream_t stream) {
    clear_error_device();
    DIAQ_TRY(check_state(psi, n_qubits, dtype));
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    return run_norm(psi, n_qubits, dtype, out, static_cast<cudaStream_t>(stream));
}

diaq_status diaq_expect(const void* psi, int32_t n_qubits, diaq_dtype dtype, int32_t n_terms, const uint64_t* xmask,
                        const uint64_t* zmask, const double* coeff, double* out, diaq_stream_t stream) {
    clear_error_device();
    DIAQ_TRY(check_state(psi, n_qubits, dtype));
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    if (n_terms < 0 || (n_terms && (!xmask || !zmask || !coeff))) return fail(DIAQ_ERR_ARG, "bad term arrays");
    PauliGroups pg;
    DIAQ_TRY(make_pauli_groups(n_qubits, n_terms, xmask, zmask, coeff, false, &pg));
    return run_expect(psi, n_qubits, dtype, pg, out, static_cast<cudaStream_t>(stream));
}

diaq_status diaq_apply_pauli_sum(const void* psi, void* lambda, int32_t n_qubits, diaq_dtype dtype, int32_t n_terms,
                                 const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                                 diaq_stream_t stream) {
    clear_error_device();
    DIAQ_TRY(check_state(psi, n_qubits, dtype));
    DIAQ_TRY(check_state(lambda, n_qubits, dtype));
    if (overlaps(psi, lambda, (size_t(1) << n_qubits) * amp_bytes(dtype))) return fail(DIAQ_ERR_ARG, "psi and lambda overlap");
    if (n_terms < 0 || (n_terms && (!xmask || !zmask || !coeff))) return fail(DIAQ_ERR_ARG, "bad term arrays");
    PauliGroups pg;
    DIAQ_TRY(make_pauli_groups(n_qubits, n_terms, xmask, zmask, coeff, false, &pg));
    return run_pauli_apply(psi, lambda, n_qubits, dtype, pg, static_cast<cudaStream_t>(stream));
}

diaq_status diaq_adjoint_grad(const diaq_gate* gates, int32_t n_gates, const double* theta, int32_t n_params,
                              int32_t n_terms, const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                              const void* psi0, void* work_psi, void* work_lam, int32_t n_qubits, diaq_dtype dtype,
                              double* energy, double* grad, diaq_stream_t stream) {
    clear_error_device();
    DIAQ_TRY(check_state(psi0, n_qubits, dtype));
    DIAQ_TRY(check_state(work_psi, n_qubits, dtype));
    DIAQ_TRY(check_state(work_lam, n_qubits, dtype));
    const size_t bytes = (size_t(1) << n_qubits) * amp_bytes(dtype);
    if (overlaps(work_psi, work_lam, bytes) || overlaps(psi0, work_psi, bytes) || overlaps(psi0, work_lam, bytes))
        return fail(DIAQ_ERR_ARG, "psi0, work_psi and work_lam must not overlap");
    if (n_gates < 0 || (n_gates && !gates)) return fail(DIAQ_ERR_ARG, "bad gate list");
    if (n_params < 0 || (n_params && !theta)) return fail(DIAQ_ERR_ARG, "bad parameter array");
    if (n_terms < 0 || (n_terms && (!xmask || !zmask || !coeff))) return fail(DIAQ_ERR_ARG, "bad term arrays");
    // host descriptions: forward matrices, their adjoints, generators
    std::vector<GateDesc> fwd(static_cast<size_t>(n_gates)), bwd(static_cast<size_t>(n_gates)), gen(static_cast<size_t>(n_gates));
    std::vector<int> slot(static_cast<size_t>(n_gates), -1);
    int n_slots = 0;
    for (int l = 0; l < n_gates; ++l) {
        const diaq_gate* g = &gates[l];
        if (g->param >= n_params) return fail(DIAQ_ERR_ARG, "gate %d uses parameter %d >= n_params", l, g->param);
        DIAQ_TRY(gate_desc_from(g, n_qubits, theta, &fwd[size_t(l)]));
        if (fwd[size_t(l)].k > 3) return fail(DIAQ_ERR_UNSUPPORTED, "adjoint sweep supports gates of at most 3 qubits");
        GateDesc& b = bwd[size_t(l)];
        b = fwd[size_t(l)];
        const int D = 1 << b.k;
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c) b.m[size_t(r * D + c)] = std::conj(fwd[size_t(l)].m[size_t(c * D + r)]);
        if (g->param >= 0) {
            gen[size_t(l)] = fwd[size_t(l)];
            gen[size_t(l)].m = pauli_matrix(g->gen, g->k);
            slot[size_t(l)] = n_slots++;
        }
    }
    PauliGroups pg;
    DIAQ_TRY(make_pauli_groups(n_qubits, n_terms, xmask, zmask, coeff, true, &pg));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // partial sums: energy row, then one row per parametric gate
    int P = inner_partials(n_qubits);
    for (int l = 0; l < n_gates; ++l)
        if (slot[size_t(l)] >= 0) P = std::max(P, adjoint_partials(n_qubits, dtype, fwd[size_t(l)].k));
    const int rows = 1 + n_slots;
    double* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, sizeof(double) * (size_t(rows) * P + rows), s);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMallocAsync(adjoint partials): %s", cudaGetErrorString(e));
    std::vector<double> res(static_cast<size_t>(rows));
    // the sweep; every exit below frees the partials buffer
    auto sweep = [&]() -> diaq_status {
        DIAQ_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * (size_t(rows) * P + rows), s));
        DIAQ_CUDA(cudaMemcpyAsync(work_psi, psi0, bytes, cudaMemcpyDeviceToDevice, s));
        for (int l = 0; l < n_gates; ++l)
            DIAQ_TRY(launch_gate_local(n_qubits, dtype, fwd[size_t(l)], nullptr, work_psi, work_psi, s));
        DIAQ_TRY(run_pauli_apply(work_psi, work_lam, n_qubits, dtype, pg, s));
        const int Pe = inner_partials(n_qubits);
        DIAQ_TRY(launch_inner_re(work_psi, work_lam, n_qubits, dtype, d, Pe, s));
        for (int l = n_gates - 1; l >= 0; --l) {
            const int sl = slot[size_t(l)];
            const int Pl = adjoint_partials(n_qubits, dtype, fwd[size_t(l)].k);
            DIAQ_TRY(launch_adjoint_step(n_qubits, dtype, bwd[size_t(l)], sl >= 0 ? &gen[size_t(l)] : nullptr,
                                         work_psi, work_lam, sl >= 0 ? d + size_t(1 + sl) * P : nullptr, Pl, s));
        }
        // row sums (rows have at most P used columns; unused are zero)
        DIAQ_TRY(launch_sum_rows(d, rows, P, d + size_t(rows) * P, s));
        DIAQ_CUDA(cudaMemcpyAsync(res.data(), d + size_t(rows) * P, sizeof(double) * rows, cudaMemcpyDeviceToHost, s));
        return DIAQ_OK;
    };
    const diaq_status st = sweep();
    const cudaError_t ef = cudaFreeAsync(d, s);
    const cudaError_t es = cudaStreamSynchronize(s);
    if (st != DIAQ_OK) return st;
    DIAQ_CUDA(ef);
    DIAQ_CUDA(es);
    if (energy) *energy = res[0];
    if (grad) {
        for (int p = 0; p < n_params; ++p) grad[p] = 0.0;
        for (int l = 0; l < n_gates; ++l)
            if (slot[size_t(l)] >= 0) grad[gates[l].param] += gates[l].scale * res[size_t(1 + slot[size_t(l)])];
    }
    return DIAQ_OK;
}

}  // extern "C"
