// Internal declarations shared by the host code and the CUDA kernels of
// libdiaq_gb300. Not part of the public ABI (see include/diaq.h).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "diaq.h"

// Every device and pinned allocation of the library goes through these, so
// a test can make the n-th one fail (diaq_debug_inject_alloc_failure) and
// drive each error path on the host, with no GPU fault. The real runtime
// functions are called as (cudaMalloc)(...), which the macros do not touch.
namespace diaq {
cudaError_t inj_malloc(void** p, size_t n);
cudaError_t inj_malloc_async(void** p, size_t n, cudaStream_t s);
cudaError_t inj_malloc_host(void** p, size_t n);
}  // namespace diaq
#define cudaMalloc(P, N) ::diaq::inj_malloc(reinterpret_cast<void**>(P), (N))
#define cudaMallocAsync(P, N, S) ::diaq::inj_malloc_async(reinterpret_cast<void**>(P), (N), (S))
#define cudaMallocHost(P, N) ::diaq::inj_malloc_host(reinterpret_cast<void**>(P), (N))

namespace diaq {

using cplx = std::complex<double>;

// ---------------------------------------------------------------------------
// Errors: thread-local message, status codes, CUDA checks.
// ---------------------------------------------------------------------------
diaq_status fail(diaq_status s, const char* fmt, ...);
void clear_error();
diaq_status cuda_fail(cudaError_t e, const char* what);

#define DIAQ_CUDA(expr)                                                    \
    do {                                                                   \
        cudaError_t e__ = (expr);                                          \
        if (e__ != cudaSuccess) return ::diaq::cuda_fail(e__, #expr);      \
    } while (0)

// Before a kernel launch: an error left by an earlier runtime call (ours or
// the host application's) would otherwise be reported by the launch check.
#define DIAQ_PRELAUNCH(name)                                               \
    do {                                                                   \
        cudaError_t e__ = cudaGetLastError();                              \
        if (e__ != cudaSuccess) return ::diaq::cuda_fail(e__, "an earlier CUDA call (pending before launch of " name ")"); \
    } while (0)

#define DIAQ_TRY(expr)                                                     \
    do {                                                                   \
        diaq_status s__ = (expr);                                          \
        if (s__ != DIAQ_OK) return s__;                                    \
    } while (0)

// ---------------------------------------------------------------------------
// Entry types of a local gate matrix. The kernels branch on them uniformly
// (every thread of a launch sees the same matrix), so a diagonal, permutation
// or real gate pays no FP64 work for its zero, unit or imaginary parts.
// ---------------------------------------------------------------------------
enum EntryType : uint8_t { ET_ZERO = 0, ET_ONE = 1, ET_REAL = 2, ET_IMAG = 3, ET_GENERAL = 4 };

uint8_t entry_type(cplx v);

// Host description of a gate-structured operator: k targets (targets[0] is
// the most significant local bit) and its 2^k x 2^k local matrix.
struct GateDesc {
    int k = 0;
    int targets[DIAQ_MAX_K] = {0};
    std::vector<cplx> m;  // row-major, 4^k entries
};

// Local matrix of a public gate (fixed or parametric).
diaq_status gate_desc_from(const diaq_gate* g, int n_qubits, const double* theta, GateDesc* out);
// Pauli string matrix of a parametric gate's generator on its targets.
std::vector<cplx> pauli_matrix(const char* gen, int k);
// Structural class of a local matrix.
int classify(const std::vector<cplx>& m, int k);
// Full-system offsets of a local matrix on its targets (ascending).
std::vector<int64_t> full_offsets(const GateDesc& g, const std::vector<uint8_t>* pattern);

// ---------------------------------------------------------------------------
// Ops
// ---------------------------------------------------------------------------
}  // namespace diaq

struct diaq_op_s {
    int n = 0;
    diaq_dtype dtype = DIAQ_C128;
    diaq_variant variant = DIAQ_ONTHEFLY;
    int op_class = DIAQ_CLASS_GENERAL;
    int device = 0;
    diaq::GateDesc gate;                 // valid unless op_class == RAW
    std::vector<int64_t> offsets;        // full-system diagonal indices, ascending
    // stored variant
    void* d_values = nullptr;            // concatenated diagonals (dtype)
    int64_t* d_offsets = nullptr;        // device copy of offsets
    int64_t* d_starts = nullptr;         // element start of each diagonal
    std::vector<int64_t> starts;         // host copy of d_starts
    int64_t stored_elems = 0;
    bool real_values = false;            // every stored value has imaginary part 0
    // device copy of the local matrix for k > 3 (dtype complex, then types)
    void* d_matrix = nullptr;
};

namespace diaq {

// ---------------------------------------------------------------------------
// Kernel launchers (apply.cu, reduce.cu, adjoint.cu)
// ---------------------------------------------------------------------------
inline size_t amp_bytes(diaq_dtype dt) { return dt == DIAQ_C128 ? 16 : 8; }
// SM count of the current device (cached per device ordinal).
int device_sm_count();
// In-place trade of the bit-l = 1 half of lo with the bit-l = 0 half of hi
// (two shards of n_local qubits; shard.cu).
diaq_status launch_shard_swap(void* lo, void* hi, int n_local, diaq_dtype dt, int l, cudaStream_t s);

// Launch tuning knobs, filled by the autotuner (defaults otherwise).
struct LaunchCfg {
    int threads = 256;     // threads per block
    int groups = 0;        // groups (target subspaces) per thread; 0 = default for k
};
LaunchCfg& launch_cfg(diaq_dtype dt, int k);

diaq_status launch_onthefly(const diaq_op_s* op, const void* x, void* y, cudaStream_t s);
diaq_status launch_gate_local(int n, diaq_dtype dt, const GateDesc& g, const void* d_matrix,
                              const void* x, void* y, cudaStream_t s);
diaq_status launch_stored(const diaq_op_s* op, const void* x, void* y, cudaStream_t s);
// Stored values one diaq_apply of a stored op reads: for a gate op on at
// most 3 targets only the diagonals of each row's local class
// (N/2^k x the class table's entries), else every stored value.
int64_t stored_values_read(const diaq_op_s* op);
diaq_status launch_materialise(diaq_op_s* op, cudaStream_t s);
diaq_status launch_raw_upload(diaq_op_s* op, const double* host_values, cudaStream_t s);
diaq_status launch_spgemm(const diaq_op_s* a, const diaq_op_s* b, diaq_op_s* c, cudaStream_t s);
diaq_status upload_matrix(diaq_op_s* op);

// Unitary simulation helpers (unitary.cu): per-diagonal count of values
// that are not exactly zero (synchronises s), and a gather of the stored
// diagonals keep[] of src into dst (dst offsets/starts already set).
diaq_status count_diagonal_nnz(const diaq_op_s* op, std::vector<int64_t>* nnz, cudaStream_t s);
diaq_status launch_gather_diagonals(const diaq_op_s* src, const std::vector<int32_t>& keep, diaq_op_s* dst,
                                    cudaStream_t s);

// In-place apply that reads and writes only the rows an op changes
// (inplace.cu). Sets *launched = false, and does nothing, when the op has
// no identity row or is not a k <= 3 on-the-fly gate op; the caller then
// runs the full kernel.
diaq_status launch_inplace_skip(const diaq_op_s* op, void* x, cudaStream_t s, bool* launched);
// The same on the groups [g_begin, g_end) only (a group: the 2^k amplitudes
// that share their non-target bits, numbered by those bits).
diaq_status launch_inplace_skip_range(const diaq_op_s* op, void* x, int64_t g_begin, int64_t g_end, cudaStream_t s,
                                      bool* launched);
// On-the-fly apply of a k <= 3 gate on the groups [g_begin, g_end) only.
diaq_status launch_gate_local_range(int n, diaq_dtype dt, const GateDesc& g, const void* x, void* y,
                                    int64_t g_begin, int64_t g_end, cudaStream_t s);
// Local columns read and local rows written by that kernel.
void inplace_masks(const GateDesc& g, diaq_dtype dt, uint32_t* ld_mask, uint32_t* st_mask);
// Algorithmic bytes of one in-place on-the-fly apply of g.
int64_t inplace_bytes(int n, diaq_dtype dt, const GateDesc& g);

// Diagonal ops of 4..6 qubits (diag.cu): one table lookup and one complex
// multiply per row; in place (x == y) rows whose entry is exactly 1 are
// skipped.
// Scaled form of a complex128 one-qubit gate (RX, RY, H and the like): the
// launch applies U / sigma; gate_scaled1_sigma tells whether the gate has
// the form and its sigma.
bool gate_scaled1_sigma(const GateDesc& g, double* sigma);
diaq_status launch_gate_scaled1_range(int n, const GateDesc& g, const void* x, void* y, int64_t g_begin,
                                      int64_t g_end, double* sigma, cudaStream_t s);
// One in-place pass of two one-qubit gates on different qubits (a then b),
// each in the scaled form (complex128) or general.
diaq_status launch_pair1_inplace(int n, diaq_dtype dt, const GateDesc& ga, bool sa, const GateDesc& gb, bool sb,
                                 void* x, cudaStream_t s);
// A merged run of diagonal ops (diaq_simulate): up to DIAG_BIG_K targets,
// the table index takes bit t[q] of the row as its bit q.
constexpr int DIAG_BIG_K = 11;
struct BigDiagArgs {
    int k;
    int t[DIAG_BIG_K];
};
diaq_status launch_bigdiag_inplace(int n, diaq_dtype dt, const BigDiagArgs& a, const double2* table,
                                   const uint32_t* skip, void* x, cudaStream_t s);
bool is_diagonal(const GateDesc& g);
diaq_status launch_diag(int n, diaq_dtype dt, const GateDesc& g, const void* x, void* y, cudaStream_t s);
int64_t diag_inplace_bytes(int n, diaq_dtype dt, const GateDesc& g);

// Debug bounds words, one per translation unit with checks (bounds.cuh);
// each returns the first failure recorded there (0: none; ~0: unreadable)
// and clears it when asked. In the normal build they return 0.
unsigned long long bounds_word_apply(bool clear);
unsigned long long bounds_word_inplace(bool clear);
unsigned long long bounds_word_diag(bool clear);
unsigned long long bounds_word_reduce(bool clear);
unsigned long long bounds_word_batch(bool clear);
unsigned long long bounds_word_sample(bool clear);
unsigned long long bounds_word_shard(bool clear);

// Pauli-sum terms grouped by X mask, prepared on the host.
struct PauliGroups {
    std::vector<uint64_t> xmask;         // one per group
    std::vector<int32_t> first;          // first term of each group (size groups+1)
    std::vector<uint64_t> zmask;         // per term
    std::vector<double> kappa;           // per term: c_t * i^{#Y}, interleaved complex
};
diaq_status make_pauli_groups(int n_qubits, int n_terms, const uint64_t* xm, const uint64_t* zm,
                              const double* coeff, bool real_only, PauliGroups* out);

// sum_i conj(psi[i ^ x_g]) psi[i] W_g(i) (complex, FP64) -> host out[2].
diaq_status run_expect(const void* psi, int n, diaq_dtype dt, const PauliGroups& pg, double* out,
                       cudaStream_t s);
diaq_status run_pauli_apply(const void* psi, void* lam, int n, diaq_dtype dt, const PauliGroups& pg,
                            cudaStream_t s);
diaq_status run_norm(const void* psi, int n, diaq_dtype dt, double* out, cudaStream_t s);
// The two kernels of the norm on caller-provided scratch: the block partials
// in scratch[0, norm_partials(n)) and the total in scratch[norm_partials(n)].
// diaq_norm and diaq_norm_noalloc both run exactly this (same grid, same
// per-thread order and block tree), so they return the same bits.
int norm_partials(int n);
diaq_status launch_norm(const void* psi, int n, diaq_dtype dt, double* scratch, cudaStream_t s);

// Adjoint reverse step for one gate: optional gradient partial
// Im <lam|P|psi> into partial[blockIdx] and, then, psi <- U^dag psi,
// lam <- U^dag lam in place.
diaq_status launch_adjoint_step(int n, diaq_dtype dt, const GateDesc& udag, const GateDesc* pauli,
                                void* psi, void* lam, double* partials, int n_partials,
                                cudaStream_t s);
int adjoint_partials(int n, diaq_dtype dt, int k);
diaq_status launch_sum_rows(const double* partials, int rows, int cols, double* out, cudaStream_t s);
diaq_status launch_inner_re(const void* a, const void* b, int n, diaq_dtype dt, double* partials,
                            int n_partials, cudaStream_t s);
int inner_partials(int n);

}  // namespace diaq
