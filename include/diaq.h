/*
 * diaq.h - C ABI of libdiaq_gb300, a GB300 (sm_103a) implementation of the
 * DiaQ gate-apply path of arXiv 2405.01250 ("DiaQ: Efficient State-Vector
 * Quantum Simulation").
 *
 * Conventions used by every entry point
 * -------------------------------------
 * State vectors. An n-qubit state is N = 2^n complex amplitudes stored
 * contiguously with interleaved (re, im) parts: complex64 (8 bytes per
 * amplitude) or complex128 (16 bytes). Qubit q is bit q of the basis index
 * (qubit 0 is the least significant bit). State buffers passed to the
 * device entry points are DEVICE pointers, 16-byte aligned, owned by the
 * caller; the library never frees them.
 *
 * Gates. A k-qubit gate on targets t[0..k-1] is a 2^k x 2^k complex matrix
 * M in the local basis whose most significant bit is qubit t[0]; its
 * full-system operator is the time-step unitary I_above (x) M (x) I_below of
 * Section II-C, with the factors placed on the target bits.
 *
 * DiaQ. A matrix in DiaQ form (Section IV) is a map from diagonal index d to
 * the N-|d| values of that diagonal, index d >= 0 holding A[t][t+d] and
 * d < 0 holding A[t-d][t] for t = 0 .. N-|d|-1 (the orientation of
 * Algorithm 2). Host-side value arrays are complex128, interleaved.
 *
 * Streams. diaq_stream_t is a cudaStream_t (NULL = the legacy default
 * stream). Device work is enqueued on it; entry points that return a value
 * to host memory synchronise that stream before returning.
 *
 * Errors. No entry point throws or aborts. Each returns a diaq_status; on
 * failure diaq_last_error() gives a message for the calling thread. The
 * paper's "not multiplyable" shape error (Algorithms 1 and 2) is
 * DIAQ_ERR_SHAPE. Argument checks happen before any device work, so a
 * rejected call leaves all buffers untouched.
 *
 * Ownership. diaq_op_t handles are created by diaq_build / diaq_build_diaq /
 * diaq_fuse and released by diaq_op_destroy; an op owns its device memory
 * (gate matrix, stored diagonals) on the device that was current when it was
 * built, and must be used with that device current.
 */
#ifndef DIAQ_H
#define DIAQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIAQ_MAX_K 6        /* largest gate or fused operator, in qubits */
#define DIAQ_MAX_QUBITS 34  /* largest state, in qubits */

typedef enum {
    DIAQ_OK = 0,
    DIAQ_ERR_ARG = 1,         /* invalid argument (NULL, range, aliasing) */
    DIAQ_ERR_SHAPE = 2,       /* operand shapes do not match ("not multiplyable") */
    DIAQ_ERR_ALLOC = 3,       /* device or host allocation failed */
    DIAQ_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed */
    DIAQ_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    DIAQ_ERR_BOUNDS = 6,      /* a device-side index check failed */
    DIAQ_ERR_UNSUPPORTED = 7  /* valid request outside what this build handles */
} diaq_status;

typedef enum { DIAQ_C64 = 0, DIAQ_C128 = 1 } diaq_dtype;

/* How an op multiplies: DIAQ_ONTHEFLY generates the full-system diagonals
 * from the 2^k x 2^k gate while it streams the state (Algorithm 3,
 * generalised to any target placement); DIAQ_STORED materialises them in
 * device memory and runs the DiaQ SpMV of Algorithm 2 over them. */
typedef enum { DIAQ_ONTHEFLY = 0, DIAQ_STORED = 1 } diaq_variant;

typedef void* diaq_stream_t;
typedef struct diaq_op_s* diaq_op_t;

/* A gate. For a fixed gate, m points to the 2^k x 2^k row-major complex128
 * matrix (host memory, read during the call only). A parametric gate sets
 * param >= 0 and m = NULL; it is exp(-i a/2 P) = cos(a/2) I - i sin(a/2) P
 * with a = scale * theta[param] and P the Pauli string gen (one letter from
 * "IXYZ" per target, gen[0] acting on targets[0], NUL-terminated). */
typedef struct {
    int32_t k;
    int32_t targets[DIAQ_MAX_K];
    const double* m;
    int32_t param;
    double scale;
    char gen[DIAQ_MAX_K + 2];
} diaq_gate;

/* Structural class of an op's local matrix, chosen by the builder. */
typedef enum {
    DIAQ_CLASS_GENERAL = 0,   /* dense or sparse complex */
    DIAQ_CLASS_REAL = 1,      /* all entries real */
    DIAQ_CLASS_DIAGONAL = 2,  /* only principal-diagonal entries (Section III-A) */
    DIAQ_CLASS_PERMUTATION = 3, /* one entry 1 per row and column */
    DIAQ_CLASS_MONOMIAL = 4,  /* one non-zero per row and column */
    DIAQ_CLASS_RAW = 5        /* a DiaQ matrix with no gate structure */
} diaq_class;

typedef struct {
    int32_t n_qubits;
    int32_t dtype;           /* diaq_dtype */
    int32_t variant;         /* diaq_variant */
    int32_t op_class;        /* diaq_class */
    int32_t k;               /* target count (0 for DIAQ_CLASS_RAW) */
    int32_t targets[DIAQ_MAX_K];
    int64_t n_diagonals;     /* full-system DiaQ diagonals of the op */
    int64_t stored_bytes;    /* device bytes of materialised diagonals (0 if on-the-fly) */
    int32_t real_values;     /* 1 if every entry of the op is real (imaginary part 0): gate
                                ops with a real matrix, raw ops given real values, products
                                of such ops; the stored SpMV then skips the imaginary half */
} diaq_op_info;

/* ------------------------------------------------------------------------
 * Library
 * ------------------------------------------------------------------------ */

/* Message of the last failed call on this thread ("" if none). The string
 * is owned by the library and valid until the next call on this thread. */
const char* diaq_last_error(void);

/* Version string, e.g. "diaq_gb300 0.1 (sm_103a)". */
const char* diaq_version(void);

/* ------------------------------------------------------------------------
 * Builder (host part) - Section IV (DiaQ format), Section II-C (time-step
 * unitary), Algorithm 3 (offset dIndex * dim_b of a gate diagonal).
 * ------------------------------------------------------------------------ */

/* Full-system diagonal indices of a gate on an n-qubit register, ascending:
 * every index d = sum_a (c_a - r_a) 2^{t_a} over the (row r, column c) pairs
 * of M with a non-zero entry (for a parametric gate, of I and P). Writes at
 * most cap indices to offsets (host) and the total to *count; returns
 * DIAQ_ERR_ARG if cap is too small (with *count set). No GPU needed. */
diaq_status diaq_gate_offsets(const diaq_gate* g, int32_t n_qubits, int64_t* offsets,
                              int64_t cap, int64_t* count);

/* DiaQ matrix product C = A B on the host (Algorithm 1), complex128, for
 * square matrices of order N. A and B are given as (count, indices,
 * concatenated values in index order). Where several (a, b) pairs meet on
 * one result index a+b their products are summed, and diagonals whose
 * products have no overlap are dropped (the reading of "isValid"); exact
 * zeros are kept. Two calls: with c_values == NULL it only reports
 * *c_count and *c_values_len (elements); then call again with buffers of
 * that size. No GPU needed. */
diaq_status diaq_diaq_matmul_host(int64_t N,
                                  int64_t a_count, const int64_t* a_idx, const double* a_values,
                                  int64_t b_count, const int64_t* b_idx, const double* b_values,
                                  int64_t* c_count, int64_t* c_idx, int64_t* c_values_len,
                                  double* c_values);

/* Gate fusion on the host (Section VI: spGEMM fuses consecutive gates):
 * embeds each gate in the union of their targets (union order = first
 * appearance, union[0] most significant) as a DiaQ matrix, multiplies them
 * with the accumulating product of diaq_diaq_matmul_host, and returns the
 * union targets and the dense 2^K x 2^K fused matrix (K <= DIAQ_MAX_K)
 * = M_{count-1} ... M_0. theta is read for parametric gates (may be NULL if
 * there are none). fused_m must hold 2 * 4^K doubles. No GPU needed. */
diaq_status diaq_fuse_gates_host(const diaq_gate* gates, int32_t count, const double* theta,
                                 int32_t* union_k, int32_t* union_targets, double* fused_m);

/* ------------------------------------------------------------------------
 * Ops
 * ------------------------------------------------------------------------ */

/* Build an op for gate g on an n-qubit register (1 <= n <= DIAQ_MAX_QUBITS,
 * 1 <= k <= min(n, DIAQ_MAX_K), distinct targets in [0, n)). theta is read
 * if g is parametric. DIAQ_STORED allocates sum_d (N - |d|) amplitudes of
 * device memory and fills them with a kernel on `stream`. */
diaq_status diaq_build(const diaq_gate* g, int32_t n_qubits, diaq_dtype dtype,
                       diaq_variant variant, const double* theta, diaq_stream_t stream,
                       diaq_op_t* out);

/* Build a stored op from a DiaQ matrix given on the host (Section IV):
 * count distinct indices |d| < 2^n, values concatenated in index order
 * (complex128; converted to dtype). */
diaq_status diaq_build_diaq(int32_t n_qubits, int64_t count, const int64_t* indices,
                            const double* values, diaq_dtype dtype, diaq_stream_t stream,
                            diaq_op_t* out);

/* Release an op and its device memory (NULL is accepted). Synchronises the
 * op's device before freeing. */
diaq_status diaq_op_destroy(diaq_op_t op);

diaq_status diaq_op_query(diaq_op_t op, diaq_op_info* info);

/* Full-system diagonal indices of the op, as diaq_gate_offsets. */
diaq_status diaq_op_offsets(diaq_op_t op, int64_t* offsets, int64_t cap, int64_t* count);

/* Copy stored diagonal number `which` (in index order) to host memory as
 * N-|d| amplitudes of the op's dtype; DIAQ_ERR_ARG for on-the-fly ops. */
diaq_status diaq_op_read_diagonal(diaq_op_t op, int64_t which, void* host_out, diaq_stream_t stream);

/* Fuse ops into one: out = ops[count-1] ... ops[0]. Gate-structured ops
 * are fused on the host in their union target space (diaq_fuse_gates_host;
 * the union must have at most DIAQ_MAX_K qubits, else DIAQ_ERR_UNSUPPORTED);
 * if any op is DIAQ_CLASS_RAW, the full-system DiaQ product of Algorithm 1
 * runs on the device instead and the result is stored. All ops must share
 * n_qubits and dtype (DIAQ_ERR_SHAPE otherwise). `variant` selects the
 * result's variant for gate-structured fusion. */
diaq_status diaq_fuse(const diaq_op_t* ops, int32_t count, diaq_variant variant,
                      diaq_stream_t stream, diaq_op_t* out);

/* ------------------------------------------------------------------------
 * Gate apply - the DiaQ SpMV (Algorithm 2 for stored ops; Algorithm 3,
 * generalised, for on-the-fly ops): y[i] = sum_d A_d(i) x[i + d].
 * ------------------------------------------------------------------------ */

/* y = A x on `stream`. x, y: device state vectors of the op's n_qubits and
 * dtype. y == x (in place) is allowed for on-the-fly ops only; otherwise x
 * and y must not overlap (DIAQ_ERR_ARG).
 *
 * In place, an op of k <= 3 qubits whose local matrix has identity rows
 * (row r equal to e_r exactly, e.g. a controlled phase, CZ, CNOT or SWAP;
 * Section III-A) reads only the local columns its other rows use and writes
 * only those rows: a controlled phase or CZ moves a quarter of the bytes of
 * a full pass, a CNOT or SWAP half. The result is bit-identical to the full
 * pass. diaq_op_apply_bytes reports the bytes either way. A diagonal op of
 * 4..6 qubits (e.g. a fused run of controlled phases) multiplies each row by
 * its one entry; in place it skips the rows whose entry is exactly 1.
 *
 * Stored ops: each row sums its diagonals' terms in index order. For a gate
 * op on k <= 3 targets a row reads only the diagonals its local row class
 * can use (the others hold zeros in that row). A stored zero that is read
 * is multiplied, not skipped, as in a dense product: a non-finite amplitude
 * that meets one gives NaN. */
diaq_status diaq_apply(diaq_op_t op, const void* x, void* y, diaq_stream_t stream);

/* Algorithmic HBM bytes of one diaq_apply of op into *bytes (s = bytes per
 * amplitude). Out of place (in_place = 0): 2 N s for on-the-fly ops; for
 * stored ops 2 N s plus s x the stored values the SpMV reads, which for a
 * gate op on k <= 3 targets are N / 2^k x (the diagonals each local row
 * class can use, summed over the 2^k classes): the zeros the format stores
 * where a diagonal crosses rows of another class are not read. Raw ops and
 * k > 3 read every stored value, s sum_d (N - |d|). In place (on-the-fly ops
 * only, DIAQ_ERR_ARG for stored) N / 2^k x (columns read + rows written) x s
 * when the op has identity rows (k <= 3; for a diagonal op of 4..6 qubits
 * 2 s N / 2^k x the entries that are not exactly 1), else 2 N s. Host only. */
diaq_status diaq_op_apply_bytes(diaq_op_t op, int32_t in_place, int64_t* bytes);

/* Run ops[0..count-1] in order on a state: psi_in -> psi_out. psi_in and
 * psi_out may each be host (pageable or pinned) or device pointers; host
 * data are copied in and out on `stream` inside the call. work0 and work1
 * are caller-owned device state buffers (work1 may be NULL when every op is
 * on-the-fly). On-the-fly ops run in place in work0 (with the identity-row
 * skip of diaq_apply); psi_in may be work0 itself, and psi_out the buffer
 * that ends up holding the state (work0 when every op is on-the-fly), and
 * then no copy is made. Host copies overlap the first and last ops as in
 * diaq_simulate_timed. In complex128, one-qubit on-the-fly ops whose rows
 * each hold an entry of the largest magnitude sigma (RX, RY, H and the
 * like: real diagonal, off-diagonal both real or both imaginary) run as
 * U / sigma, one fused multiply-add per real component, and the last such
 * op of the list runs as U times the product of the dropped sigmas. Two
 * consecutive one-qubit on-the-fly ops with no zero entry, on different
 * qubits, run in one pass over the state. A run
 * of consecutive diagonal on-the-fly ops whose targets span at most 11
 * qubits runs as one pass with the product of their diagonals (a table of
 * up to 2048 entries, copied to the device inside the call; rows whose
 * product is exactly 1 are not touched). The result equals the op-by-op one
 * up to rounding. Synchronises `stream` before returning. */
diaq_status diaq_simulate(const diaq_op_t* ops, int32_t count, const void* psi_in, void* psi_out,
                          void* work0, void* work1, diaq_stream_t stream);

/* diaq_simulate with the host copies overlapped and timed. When psi_in is
 * host memory and ops[0] is an on-the-fly op of k <= 3 qubits, the input is
 * copied in 16 slices (its groups split by their top 4 non-target bits, a
 * few contiguous runs each) on a second stream, and ops[0] runs on each
 * slice as soon as it has arrived; when psi_out is host memory and the last
 * op is such an op, it runs slice by slice and each finished slice is
 * copied out while the next is computed. The result is the same as
 * diaq_simulate's. timeline_ms (host, 3 floats, may be NULL) receives, from
 * the start of the call's device work, the time at which the input copy
 * was complete, the last op was done, and the output copy was complete (the
 * legs overlap). Creates and destroys two streams and a few events per
 * call; synchronises `stream`. */
diaq_status diaq_simulate_timed(const diaq_op_t* ops, int32_t count, const void* psi_in, void* psi_out,
                                void* work0, void* work1, diaq_stream_t stream, float* timeline_ms);

/* The HBM bytes diaq_simulate moves for ops on a device state (psi_in and
 * psi_out the work buffer): each merged diagonal run reads and writes the
 * rows whose product is not exactly 1 once, each one-qubit pair the state
 * once, every other op its diaq_op_apply_bytes (in place on the fly,
 * out of place stored). With host buffers the first and last ops may run
 * slice by slice outside any pair or run. Host only. */
diaq_status diaq_simulate_bytes(const diaq_op_t* ops, int32_t count, int64_t* bytes);

/* ------------------------------------------------------------------------
 * Unitary simulation - Section II-A (a circuit's unitary as the product of
 * its gate unitaries) and Section III-A (the number of diagonals and the
 * sparsity of that product after each time step, e.g. GHZ(10) stays at
 * least 99.8 % sparse). The products run on the device by Algorithm 1.
 * ------------------------------------------------------------------------ */

/* Per stored diagonal of op (in index order), the number of values that are
 * not exactly zero, into nnz (host, n_diagonals entries). DIAQ_ERR_ARG for
 * on-the-fly ops. Synchronises `stream`. */
diaq_status diaq_op_diagonal_nnz(diaq_op_t op, int64_t* nnz, diaq_stream_t stream);

/* A new stored DIAQ_CLASS_RAW op equal to op without the diagonals whose
 * values are all exactly zero. No value changes, and values that are
 * non-zero only by rounding are kept (no tolerance is applied). DIAQ_ERR_ARG
 * for on-the-fly ops. Synchronises `stream`. */
diaq_status diaq_op_prune(diaq_op_t op, diaq_stream_t stream, diaq_op_t* out);

/* The unitary U = G_{n_gates-1} ... G_0 of a circuit: each gate is built as
 * a stored op (diaq_build) and multiplied onto U on the device with the
 * accumulating DiaQ product of Algorithm 1, one time step at a time. With
 * prune != 0, diagonals that come out exactly zero are dropped after each
 * product (diaq_op_prune). After time step t, n_diagonals[t] and nnz[t]
 * (host arrays of n_gates entries, each may be NULL) receive the diagonal
 * count and the number of non-zero values of U. The result is a stored
 * DIAQ_CLASS_RAW op owned by the caller. Memory grows with the diagonals of
 * U (up to 2N - 1 of them, N^2 values for a dense unitary); the product
 * launches one grid row per result diagonal, so n_qubits <= 15. */
diaq_status diaq_unitary_chain(const diaq_gate* gates, int32_t n_gates, const double* theta, int32_t n_qubits,
                               diaq_dtype dtype, int32_t prune, int64_t* n_diagonals, int64_t* nnz,
                               diaq_stream_t stream, diaq_op_t* out);

/* ------------------------------------------------------------------------
 * Reductions (FP64 accumulation for both dtypes; deterministic for a given
 * n_qubits and dtype). The paper reads out expectation values and
 * magnetisations (Section II-B); these compute them on the device.
 * ------------------------------------------------------------------------ */

/* ||psi||^2 into *out (host). */
diaq_status diaq_norm(const void* psi, int32_t n_qubits, diaq_dtype dtype, double* out,
                      diaq_stream_t stream);

/* <psi| sum_t c_t P_t |psi> into out[0] (re), out[1] (im) (host). Term t is
 * the Pauli string with X on the bits of xmask[t] only, Z on zmask[t] only
 * and Y on both; coeff holds n_terms complex128 coefficients. n_terms may be
 * 0 (result 0). Host arrays. */
diaq_status diaq_expect(const void* psi, int32_t n_qubits, diaq_dtype dtype, int32_t n_terms,
                        const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                        double* out, diaq_stream_t stream);

/* lambda = (sum_t c_t P_t) psi on the device; lambda must not overlap psi. */
diaq_status diaq_apply_pauli_sum(const void* psi, void* lambda, int32_t n_qubits,
                                 diaq_dtype dtype, int32_t n_terms, const uint64_t* xmask,
                                 const uint64_t* zmask, const double* coeff,
                                 diaq_stream_t stream);

/* ------------------------------------------------------------------------
 * Shots - Section VII runs every benchmark for 1024 shots: basis states
 * drawn from the final state with the Born-rule probabilities.
 * ------------------------------------------------------------------------ */

/* Draw n_shots basis-state indices from psi: outcome i with probability
 * |psi_i|^2 / ||psi||^2, by the inverse of the cumulative distribution in
 * index order. Shot s takes the caller's uniform u = uniforms[s] (clamped to
 * [0, 1]; NaN counts as 0), forms r = u ||psi||^2 and returns the smallest i
 * whose running sum of |psi|^2 exceeds r; when none does (u = 1) it returns
 * the largest i of non-zero probability. An outcome of zero probability is
 * never drawn; a state of zero norm gives -1 for every shot.
 *
 * The running sums are FP64 (complex64: exact FP32 squares summed as FP32
 * pairs, about 48 bits, per 16 amplitudes) over a tree of sequential sums
 * (runs of 16 amplitudes, segs of 16 runs, tiles of 16 segs, groups of 256),
 * so where r lies within rounding of a boundary of the cumulative
 * distribution the outcome may be the neighbouring index of a plain
 * left-to-right sum; on states whose sums are exact (e.g. dyadic
 * probabilities) the outcome is exactly that of the definition.
 *
 * psi: device state (16-byte aligned). uniforms: device array of n_shots
 * doubles. out_indices: device array of n_shots int64 (8-byte aligned both).
 * 0 <= n_shots <= 2^31. Allocates about (N / 4096) x 273 doubles of device
 * scratch (the tree's running sums) on `stream` and frees it there; does
 * not synchronise. */
diaq_status diaq_sample(const void* psi, int32_t n_qubits, diaq_dtype dtype, const double* uniforms,
                        int64_t n_shots, int64_t* out_indices, diaq_stream_t stream);

/* ------------------------------------------------------------------------
 * Sharded state - a state vector larger than one device's memory is split
 * across devices (Section II-A; Section VI names the multi-node backend,
 * diaq-mpi). The 2^n amplitudes are split by the top g bits of the physical
 * basis index into 2^g shards of 2^(n-g) amplitudes: shard s holds physical
 * indices s 2^(n-g) .. (s+1) 2^(n-g) - 1. Logical qubits are mapped to
 * physical bits (0 .. n-g-1 local, n-g .. n-1 global); a gate runs in every
 * shard on its targets' physical positions once they are all local, and a
 * target on a global bit G is first exchanged with a local bit l: every
 * shard pair (s with bit G clear, s | 2^G) trades the half of s whose local
 * bit l is 1 for the half of its partner whose local bit l is 0.
 * ------------------------------------------------------------------------ */

typedef enum {
    DIAQ_SHARD_APPLY = 0,      /* run gates[gate] in every shard on local positions targets[] */
    DIAQ_SHARD_EXCHANGE = 1,   /* trade halves across global bit global_bit and local bit local_bit */
    DIAQ_SHARD_LOCAL_SWAP = 2  /* SWAP of local positions targets[0], targets[1] in every shard */
} diaq_shard_step_kind;

typedef struct {
    int32_t kind;                 /* diaq_shard_step_kind */
    int32_t gate;                 /* APPLY: index into the gate array; else -1 */
    int32_t k;                    /* APPLY: the gate's k; LOCAL_SWAP: 2 */
    int32_t targets[DIAQ_MAX_K];  /* local physical positions (targets[0] most significant, as the gate's) */
    int32_t global_bit;           /* EXCHANGE: bit of the shard index (0 .. g-1); else -1 */
    int32_t local_bit;            /* EXCHANGE: local physical bit traded with it; else -1 */
} diaq_shard_step;

/* The step list of a circuit on 2^global_bits shards, starting from the
 * identity map. Before each gate, every target held on a global bit is
 * exchanged with the local bit whose logical qubit is next used furthest
 * ahead (never one of the gate's targets). With restore != 0 the list ends
 * with exchanges and local SWAPs that return every logical qubit to its own
 * physical bit. Two calls: steps == NULL reports *n_steps; then pass cap >=
 * *n_steps entries. final_map (may be NULL, n_qubits entries) receives the
 * physical bit of each logical qubit after the last step. Every gate must
 * fit in a shard (k <= n - g; DIAQ_ERR_UNSUPPORTED otherwise);
 * 0 <= global_bits <= 16. Host only. */
diaq_status diaq_shard_schedule(const diaq_gate* gates, int32_t n_gates, int32_t n_qubits, int32_t global_bits,
                                int32_t restore, diaq_shard_step* steps, int32_t cap, int32_t* n_steps,
                                int32_t* final_map);

/* EXCHANGE between two shards in one address space, in place: the
 * amplitudes of lo_shard (the shard with global bit clear) whose local bit
 * local_bit is 1 trade places with those of hi_shard (its partner) whose
 * local bit is 0. Device buffers of 2^n_local amplitudes, not overlapping. */
diaq_status diaq_shard_swap(void* lo_shard, void* hi_shard, int32_t n_local, diaq_dtype dtype, int32_t local_bit,
                            diaq_stream_t stream);

/* EXCHANGE between ranks: buf (2^(n_local-1) amplitudes, device) receives, in
 * index order, the amplitudes of shard whose local bit local_bit equals
 * value; diaq_shard_unpack writes such a buffer back to those positions. A
 * rank whose shard has the global bit clear packs value 1 and its partner
 * value 0; they swap buffers (e.g. NCCL send/recv) and each unpacks what it
 * received with the value it packed. */
diaq_status diaq_shard_pack(const void* shard, int32_t n_local, diaq_dtype dtype, int32_t local_bit, int32_t value,
                            void* buf, diaq_stream_t stream);
diaq_status diaq_shard_unpack(const void* buf, void* shard, int32_t n_local, diaq_dtype dtype, int32_t local_bit,
                              int32_t value, diaq_stream_t stream);

/* Run a circuit on 2^global_bits shards held in this process (shards[s]:
 * device buffers of 2^(n - global_bits) amplitudes, not overlapping, on the
 * current device), in place, by the steps of diaq_shard_schedule: on-the-fly
 * ops on the local positions and diaq_shard_swap for exchanges. theta is read
 * for parametric gates. final_map as in diaq_shard_schedule (identity when
 * restore != 0). Synchronises `stream`. */
diaq_status diaq_sharded_simulate(const diaq_gate* gates, int32_t n_gates, const double* theta, int32_t n_qubits,
                                  int32_t global_bits, diaq_dtype dtype, void* const* shards, int32_t restore,
                                  int32_t* final_map, diaq_stream_t stream);

/* ||psi||^2 of a sharded state: diaq_norm of each shard, then one FP64 sum
 * over the shards in shard order. */
diaq_status diaq_sharded_norm(void* const* shards, int32_t n_qubits, int32_t global_bits, diaq_dtype dtype,
                              double* out, diaq_stream_t stream);

/* <psi| sum_t c_t P_t |psi> of a sharded state (terms as in diaq_expect, in
 * logical qubits; map: physical bit of each logical qubit, NULL for the
 * identity). X and Y letters must sit on local bits (DIAQ_ERR_UNSUPPORTED
 * otherwise: exchange the qubit first); a Z on global bit G weighs shard s by
 * (-1)^(bit G of s). Per-shard FP64 sums, then one sum over the shards. */
diaq_status diaq_sharded_expect(void* const* shards, int32_t n_qubits, int32_t global_bits, diaq_dtype dtype,
                                const int32_t* map, int32_t n_terms, const uint64_t* xmask, const uint64_t* zmask,
                                const double* coeff, double* out, diaq_stream_t stream);

/* ------------------------------------------------------------------------
 * Adjoint gradient (not in the paper; the adjoint-state method for
 * E(theta) = <psi(theta)|H|psi(theta)>, psi(theta) = U_L ... U_1 psi0).
 * ------------------------------------------------------------------------ */

/* Energy and full gradient in one forward and one reverse sweep. For a
 * parametric gate U = exp(-i a/2 P), a = scale * theta_p, the contribution
 * to dE/dtheta_p is scale * Im <lambda_l| P |psi_l>, with psi_l the state
 * after the gate and lambda_l = U_{l+1}^dag ... U_L^dag H psi_L.
 * psi0: device initial state (read only). work_psi, work_lam: caller-owned
 * device state buffers (overwritten). energy (host, may be NULL) and grad
 * (host, n_params doubles, may be NULL). The observable is as in
 * diaq_expect with real parts of coeff used (Hermitian H). */
diaq_status diaq_adjoint_grad(const diaq_gate* gates, int32_t n_gates, const double* theta,
                              int32_t n_params, int32_t n_terms, const uint64_t* xmask,
                              const uint64_t* zmask, const double* coeff, const void* psi0,
                              void* work_psi, void* work_lam, int32_t n_qubits, diaq_dtype dtype,
                              double* energy, double* grad, diaq_stream_t stream);

/* Adjoint plan: the sweep of diaq_adjoint_grad for one circuit (gates of
 * 1 or 2 qubits) recorded once as a CUDA graph and replayed per theta. The
 * plan owns its two state buffers; gate matrices are derived on the device
 * from the uploaded parameters, so no kernel argument changes between
 * replays. */
typedef struct diaq_adjoint_plan_s* diaq_adjoint_plan_t;

diaq_status diaq_adjoint_plan_create(const diaq_gate* gates, int32_t n_gates, int32_t n_params, int32_t n_terms,
                                     const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                                     int32_t n_qubits, diaq_dtype dtype, diaq_adjoint_plan_t* out);

/* Energy and gradient for theta (host, n_params). psi0 is a device state of
 * the plan's size and dtype, or NULL for |0...0>; a different psi0 pointer
 * than the previous call re-records the graph. energy / grad are host
 * outputs (may be NULL). Ordered after the work queued on `stream`;
 * synchronises before returning. */
diaq_status diaq_adjoint_plan_run(diaq_adjoint_plan_t p, const double* theta, const void* psi0, double* energy,
                                  double* grad, diaq_stream_t stream);

/* Choose how the plan sweeps. window = 0: one launch per gate (the
 * default). window = 2..5: gates are grouped into blocks acting on at most
 * `window` qubits and at most 32 gates, moving a gate only past gates on
 * disjoint qubits (so the operator and every gradient term are unchanged),
 * and one launch runs a whole block: each thread stages the 2^w amplitudes
 * of psi (and lambda) that share their other bits in shared memory and runs
 * the block's gates there, reading and writing each state once per block
 * instead of once per gate. Re-records the graph; on failure the plan falls
 * back to window 0 and the status says why. */
diaq_status diaq_adjoint_plan_set_window(diaq_adjoint_plan_t p, int32_t window);

/* As diaq_adjoint_plan_set_window, choosing also how many threads share a
 * group of the window: lanes = 1 (a thread runs the block's gates on its
 * own group) or 4 (four threads of a warp split each gate's subspaces,
 * which quadruples the threads at work and suits FP64-bound complex128
 * sweeps). lanes is ignored for window 0. */
diaq_status diaq_adjoint_plan_set_sweep(diaq_adjoint_plan_t p, int32_t window, int32_t lanes);

/* Current window and lanes, and the launches per sweep direction: window
 * blocks, or with window 0 the execution entries (gates, or gates and
 * diagonal runs when runs are on). */
diaq_status diaq_adjoint_plan_get_sweep(diaq_adjoint_plan_t p, int32_t* window, int32_t* lanes, int32_t* n_blocks);

/* Scaled rotations of the per-gate complex128 sweep (window 0; on by
 * default). A rotation U = cos(a/2) I + kappa P is applied as U / sigma,
 * sigma the larger in magnitude of cos(a/2) and kappa, whose rows need one
 * fused multiply-add per real component instead of two FP64 instructions
 * (FP64 is the bound of complex128 sweeps on this GPU); the factor
 * prod(1 / sigma) that the states then carry is tracked on the device and
 * divided out of the energy and of every gradient term. Results equal the
 * unscaled sweep up to rounding. Active only for complex128 plans whose
 * forward and reverse rotation count is at most 960 (the states grow by at
 * most sqrt(2) per rotation); on = 0 turns it off. Re-records the graph.
 * get_scaled: whether it is requested and whether it is active. */
diaq_status diaq_adjoint_plan_set_scaled(diaq_adjoint_plan_t p, int32_t on);
diaq_status diaq_adjoint_plan_get_scaled(diaq_adjoint_plan_t p, int32_t* on, int32_t* active);

/* Fused rotation pairs of the per-gate sweep (window 0; on by default): two
 * consecutive one-qubit rotations with X or Y generators on different
 * qubits run in one launch, on groups of 4 amplitudes in registers, so the
 * states are read and written once per pair; the reverse sweep takes both
 * gradient terms in it, each at its own gate's position. Re-records the
 * graph. */
diaq_status diaq_adjoint_plan_set_pairs(diaq_adjoint_plan_t p, int32_t on);
diaq_status diaq_adjoint_plan_get_pairs(diaq_adjoint_plan_t p, int32_t* on);

/* Diagonal runs of the per-gate sweep (window 0; on by default). Runs of
 * Z-type rotations (generators of I and Z letters), fixed single-qubit
 * diagonal gates and CZs - after moving the other gates that act on none of
 * a run's qubits ahead of it, which changes neither the operator nor any
 * gradient term - are applied as one diagonal operator (Section III-A:
 * such gates live on the principal diagonal, as does their product) in one
 * launch each way: a table lookup per amplitude when the run's rotations
 * share one parameter (a QAOA cost layer: the phase depends only on
 * W(i) = sum_g z_g(i)), a product of per-byte tables and the CZ sign when
 * they act on single qubits (an ansatz layer's RZs and CZ ladder). Each
 * rotation's gradient term, sum_i z_g(i) Im(conj(lambda_i) psi_i), is the
 * same anywhere inside the run. on = 0 applies every gate separately.
 * Re-records the graph. get_runs: whether runs are on, how many the circuit
 * has, and the launches per sweep direction. */
diaq_status diaq_adjoint_plan_set_runs(diaq_adjoint_plan_t p, int32_t on);
diaq_status diaq_adjoint_plan_get_runs(diaq_adjoint_plan_t p, int32_t* on, int32_t* n_runs, int32_t* n_steps);

/* Blocks of the per-gate sweep's kernels (window 0): each launch runs
 * `blocks` blocks of 256 threads over the state, grid-stride, and every
 * gradient term is summed over that many partial columns. 0 restores the
 * default, two per SM (one resident wave at the rotation kernels' register
 * counts), at most one group per thread. More blocks cost more per launch
 * (each block stages its phase tables and writes its partials). Values above
 * 64 per SM, or above one group of 2 amplitudes per thread, are clamped.
 * Re-records the graph. get_blocks: the blocks in use. */
diaq_status diaq_adjoint_plan_set_blocks(diaq_adjoint_plan_t p, int32_t blocks);
diaq_status diaq_adjoint_plan_get_blocks(diaq_adjoint_plan_t p, int32_t* blocks);

#define DIAQ_PLAN_TUNE_MAX 12

typedef struct {
    int32_t n_tried;
    int32_t window[DIAQ_PLAN_TUNE_MAX];
    int32_t lanes[DIAQ_PLAN_TUNE_MAX];
    int32_t blocks[DIAQ_PLAN_TUNE_MAX];  /* per-gate sweep blocks (window 0), else 0 */
    float ms[DIAQ_PLAN_TUNE_MAX];        /* one graph replay (energy + gradient) */
    int32_t best_window;
    int32_t best_lanes;
    int32_t best_blocks;
    float best_ms;
} diaq_plan_tuning;

/* Time the sweep per gate and window-fused with windows 3, 4 and 5 at 1 and
 * 4 lanes (`reps` graph replays each, with theta, host array of n_params)
 * and keep the fastest; when the per-gate sweep wins, also time it at 1
 * and 4 blocks per SM (diaq_adjoint_plan_set_blocks) and keep the fastest
 * of those. report may be NULL. Synchronises. */
diaq_status diaq_adjoint_plan_autotune(diaq_adjoint_plan_t p, const double* theta, int32_t reps,
                                       diaq_plan_tuning* report);

/* Current window and the number of launches per sweep (blocks, or gates
 * when window = 0); either pointer may be NULL. */
diaq_status diaq_adjoint_plan_get_window(diaq_adjoint_plan_t p, int32_t* window, int32_t* n_blocks);

diaq_status diaq_adjoint_plan_destroy(diaq_adjoint_plan_t p);

/* ------------------------------------------------------------------------
 * Autotuning and fusion planning (not in the paper; the paper fuses gates
 * with spGEMM, Section VI, but gives no rule for which to fuse).
 * ------------------------------------------------------------------------ */

#define DIAQ_APPLY_TUNE_MAX 27
#define DIAQ_FUSION_TUNE_MAX 8

typedef struct {
    int32_t n_rows;                     /* rows filled below */
    int32_t k[DIAQ_APPLY_TUNE_MAX];
    int32_t threads[DIAQ_APPLY_TUNE_MAX];
    int32_t groups[DIAQ_APPLY_TUNE_MAX];
    float ms[DIAQ_APPLY_TUNE_MAX];
    int32_t best_threads[3];            /* per k = 1, 2, 3 */
    int32_t best_groups[3];
    float best_ms[3];
} diaq_apply_tuning;

typedef struct {
    int32_t n_depths;
    int32_t ops[DIAQ_FUSION_TUNE_MAX];  /* fused ops at depth d+1 */
    float ms[DIAQ_FUSION_TUNE_MAX];     /* one pass of the circuit */
    int32_t best_depth;
} diaq_fusion_tuning;

/* Time the on-the-fly kernel for k = 1, 2, 3 (a real butterfly, a
 * controlled phase and a dense gate on the top qubits of an n_qubits state)
 * over threads per block in {64, 128, 256} x groups per thread in
 * {1, 2, 4}, using the caller's distinct device buffers x and y (contents
 * overwritten), and keep the fastest shape per (dtype, k) for all later
 * launches in this process. report may be NULL. */
diaq_status diaq_autotune_apply(int32_t n_qubits, diaq_dtype dtype, void* x, void* y, int32_t reps,
                                diaq_apply_tuning* report, diaq_stream_t stream);

/* Set the launch shape of the on-the-fly kernel for (dtype, k), k in 1..3:
 * threads a multiple of 32 in [32, 256], groups in {1, 2, 4}, or 0 for the
 * built-in default of k. Process-wide. */
diaq_status diaq_set_apply_launch(diaq_dtype dtype, int32_t k, int32_t threads, int32_t groups);

/* Group consecutive gates for fusion: a group grows while the union of its
 * targets has at most max_k qubits and it holds at most max_depth gates.
 * Writes the group index of each gate (non-decreasing, from 0) and the group
 * count. Host only. */
diaq_status diaq_plan_fusion(const diaq_gate* gates, int32_t n_gates, int32_t max_k, int32_t max_depth,
                             int32_t* group_of_gate, int32_t* n_groups);

/* Group gates for fusion, moving a gate earlier past gates it commutes
 * with (gates on disjoint qubits): each gate joins the latest group that
 * touched any of its qubits when that group stays within max_k qubits and
 * max_depth gates, else it opens a group. Writes the execution order of
 * the gates (order[pos] = gate index), the group of each position
 * (non-decreasing from 0) and the group count; the circuit's operator is
 * unchanged. Host only. */
diaq_status diaq_plan_fusion_commuting(const diaq_gate* gates, int32_t n_gates, int32_t max_k, int32_t max_depth,
                                       int32_t* order, int32_t* group_of_pos, int32_t* n_groups);

/* Group consecutive gates so that every group is either one gate that is
 * not diagonal or a run of diagonal gates (fixed matrices with zeros off the
 * diagonal, or rotations with only I and Z letters; Section III-A: such
 * gates hold their values on the principal diagonal, and so does their
 * product) whose union of targets has at most max_k qubits and which holds
 * at most max_depth gates. A run of controlled phases then fuses into one
 * diagonal op, which diaq_apply multiplies row by row, while the gates
 * between runs stay separate. Output as diaq_plan_fusion. Host only. */
diaq_status diaq_plan_fusion_diagonal(const diaq_gate* gates, int32_t n_gates, int32_t max_k, int32_t max_depth,
                                      int32_t* group_of_gate, int32_t* n_groups);

/* For each fusion depth 1..max_depth: plan (diaq_plan_fusion, or
 * diaq_plan_fusion_commuting when `commuting` is non-zero), build and fuse
 * the circuit's on-the-fly ops and time one in-place pass over the device
 * state `work` (contents overwritten); report the times and the fastest
 * depth. */
diaq_status diaq_autotune_fusion(const diaq_gate* gates, int32_t n_gates, const double* theta, int32_t n_qubits,
                                 diaq_dtype dtype, void* work, int32_t max_k, int32_t max_depth, int32_t commuting,
                                 diaq_fusion_tuning* report, diaq_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched energies and gradients (not in the paper). Many circuits of
 * uneven qubit counts run in one persistent launch replayed from a CUDA
 * graph: every circuit starts from |0...0>, applies its gates (k <= 2),
 * forms E = <psi|H|psi> and runs the adjoint sweep of diaq_adjoint_grad.
 * ------------------------------------------------------------------------ */

typedef struct diaq_batch_s* diaq_batch_t;

#define DIAQ_BATCH_TUNE_MAX 24

/* Launch shapes the autotuner timed and the one it kept (window 0: one pass
 * per gate; w > 0: the window-fused kernel of diaq_batch_set_window). */
typedef struct {
    int32_t n_tried;
    int32_t cluster[DIAQ_BATCH_TUNE_MAX];
    int32_t threads[DIAQ_BATCH_TUNE_MAX];
    int32_t window[DIAQ_BATCH_TUNE_MAX];
    int32_t lanes[DIAQ_BATCH_TUNE_MAX];
    float ms[DIAQ_BATCH_TUNE_MAX];
    int32_t best_cluster;
    int32_t best_threads;
    int32_t best_window;
    int32_t best_lanes;
    float best_ms;
} diaq_batch_tuning;

/* Build a batch of n_inst circuits (host arrays, read during the call).
 * Circuit i has n_qubits[i] in [2, 30] qubits, the gates
 * gates[gate_first[i] .. gate_first[i+1]) (1 or 2 targets; parametric gates
 * index the circuit's own parameters 0 .. param_first[i+1]-param_first[i]-1),
 * and the observable terms [term_first[i] .. term_first[i+1]) of xmask,
 * zmask, coeff (as diaq_expect; real parts used). The three *_first arrays
 * have n_inst + 1 entries and are non-decreasing. Allocates the device arena
 * (two states per circuit) and captures the launch in a CUDA graph with the
 * default shape (1 block of 256 threads per circuit team). */
diaq_status diaq_batch_create(int32_t n_inst, const int32_t* n_qubits, const int32_t* gate_first,
                              const diaq_gate* gates, const int32_t* param_first, const int32_t* term_first,
                              const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                              diaq_dtype dtype, diaq_batch_t* out);

diaq_status diaq_batch_destroy(diaq_batch_t b);

/* Choose the team shape: `cluster` blocks (1, 2, 4 or 8, one thread-block
 * cluster) of `threads` threads (a multiple of 32 in [64, 512]) per
 * circuit; recaptures the graph. */
diaq_status diaq_batch_set_launch(diaq_batch_t b, int32_t cluster, int32_t threads);

/* Energies (n_inst) and gradients (param_first[n_inst] doubles, circuit i's
 * block at param_first[i]) for the concatenated parameters theta. Host
 * arrays; energies or grads may be NULL. Replays the graph after the work
 * already queued on `stream` and synchronises before returning. */
diaq_status diaq_batch_run(diaq_batch_t b, const double* theta, double* energies, double* grads,
                           diaq_stream_t stream);

/* Choose how teams sweep. window = 0: one pass over the instance's states
 * per gate (the default). window = 2..5: gates are grouped into blocks of at
 * most `window` qubits and 32 gates, moving a gate only past gates on
 * disjoint qubits (operator and gradients unchanged); a team stages every
 * group of a block's window in shared memory, runs the block there, and
 * meets at the cluster barrier once per block. This kernel runs 128 threads
 * per block; the cluster size is kept. Recaptures the graph; on failure the
 * batch falls back to window 0 with 1 x 256 and the status says why. */
diaq_status diaq_batch_set_window(diaq_batch_t b, int32_t window);

diaq_status diaq_batch_get_window(diaq_batch_t b, int32_t* window);

/* As diaq_batch_set_window, choosing also how many threads share a group of
 * the window: 1, or 4 (four threads of a warp split each gate's subspaces).
 * lanes is ignored for window 0. */
diaq_status diaq_batch_set_sweep(diaq_batch_t b, int32_t window, int32_t lanes);

diaq_status diaq_batch_get_sweep(diaq_batch_t b, int32_t* window, int32_t* lanes);

/* Diagonal runs of the per-gate team kernel (window 0; on by default), as in
 * diaq_adjoint_plan_set_runs but in the weight form only: a run of Z-type
 * rotations that share one parameter and scale (a QAOA cost layer) is one
 * pass with a phase table indexed by W(i) = sum_g z_g(i), and its gradient
 * term sum_i W(i) Im(conj(lambda_i) psi_i). Other diagonal gates run one by
 * one. Recaptures the graph. get_runs: whether runs are on and how many the
 * batch's circuits hold. */
diaq_status diaq_batch_set_runs(diaq_batch_t b, int32_t on);
diaq_status diaq_batch_get_runs(diaq_batch_t b, int32_t* on, int32_t* n_runs);

/* Scaled rotations of the per-gate team kernel, as diaq_adjoint_plan_set_scaled
 * (complex128, window 0, every circuit within 480 parametric gates; on by
 * default); each team tracks its circuit's factor and rescales the energy
 * and the gradient terms it writes. Recaptures the graph. get_scaled:
 * requested and active. */
diaq_status diaq_batch_set_scaled(diaq_batch_t b, int32_t on);
diaq_status diaq_batch_get_scaled(diaq_batch_t b, int32_t* on, int32_t* active);

/* Time every team shape that fits - window 0 with cluster in {1,2,4,8} x
 * threads in {64,128,256}, and windows 3, 4, 5 at 1 and 4 lanes with
 * cluster in {2,8} x 128 threads - `reps` graph replays each with theta,
 * keep the fastest. report may be NULL. */
diaq_status diaq_batch_autotune(diaq_batch_t b, const double* theta, int32_t reps, diaq_batch_tuning* report,
                                diaq_stream_t stream);

/* Current shape, number of teams resident at once, and arena size. */
diaq_status diaq_batch_query(diaq_batch_t b, int32_t* cluster, int32_t* threads, int32_t* teams,
                             int64_t* arena_bytes);

/* ------------------------------------------------------------------------
 * Testing hook (not in the paper)
 * ------------------------------------------------------------------------ */

/* Make the library's after-th next device or pinned-host allocation (0: the
 * next one) fail as if memory were exhausted, once; -1 turns it off. The
 * failing call returns DIAQ_ERR_ALLOC (or the status of the step that
 * needed the memory) after releasing what it had allocated, and the library
 * stays usable. It happens on the host: no GPU work is affected.
 * Process-wide. */
diaq_status diaq_debug_inject_alloc_failure(int32_t after);

/* Debug bounds checks. The library's debug build (libdiaq_gb300_dbg.so,
 * compiled with -DDIAQ_DEBUG_BOUNDS; the normal build has no checks) checks
 * the amplitude and table indices its kernels compute before each access;
 * a failing check skips that access and records the first failure (site and
 * index) on the device.
 *
 * diaq_debug_bounds_enabled: *enabled = 1 in the debug build, 0 otherwise.
 * diaq_debug_bounds_check: reads the recorded failure (clearing it when
 * clear != 0) into *word (may be NULL; 0 when none) and returns DIAQ_OK, or
 * DIAQ_ERR_BOUNDS with the site and index in diaq_last_error(). In the
 * normal build it always returns DIAQ_OK. Call it after synchronising.
 * diaq_debug_bounds_status: the status and message for a recorded word
 * (host only, no GPU needed): bit 63 set, bits 48..62 the site, bits 0..47
 * the index. */
diaq_status diaq_debug_bounds_enabled(int32_t* enabled);
diaq_status diaq_debug_bounds_check(int32_t clear, uint64_t* word);
diaq_status diaq_debug_bounds_status(uint64_t word);

/* ------------------------------------------------------------------------
 * Allocation-free norm (the paper has no counterpart: this is a deployment
 * variant of diaq_norm).
 * ------------------------------------------------------------------------ */

/* Size, in doubles, of the fixed scratch array behind diaq_norm_noalloc
 * (32 KiB, resident on every device that loads the library until exit). */
#define DIAQ_NOALLOC_SCRATCH_DOUBLES 4096

/* ||psi||^2 into *out (host), the same value as diaq_norm, computed without
 * allocating memory: no cudaMalloc, cudaMallocAsync or cudaFree. It is for
 * callers that cannot allocate device memory - an application whose memory
 * manager owns the whole device heap, or a latency-critical loop that must
 * not pay for allocation - and keeps its partial sums in a fixed array
 * compiled into the library instead.
 *
 * It runs the same two kernels on the same grid as diaq_norm, so the two
 * return the same bits on the same device.
 *
 * Limit: the reduction uses min(ceil(N / 1024), 8 x SM count) blocks and
 * needs one double per block plus one; if that exceeds
 * DIAQ_NOALLOC_SCRATCH_DOUBLES the call returns DIAQ_ERR_UNSUPPORTED
 * (only on devices with more than 511 SMs).
 *
 * Set-up: every call looks up the array's device address in the current
 * context (cudaGetSymbolAddress, with the state's device current); the first
 * call on a device also loads the library's device code there, so make that
 * first call before any stream capture. Sharing: all calls on a device use the same
 * array, which keeps the last call's contents; every slot a call reads it
 * has written itself, so nothing needs clearing, but calls whose work
 * overlaps on the GPU (different streams, or host threads racing on one
 * device) race on the array and must be serialised by the caller.
 * Synchronises `stream` before returning. */
diaq_status diaq_norm_noalloc(const void* psi, int32_t n_qubits, diaq_dtype dtype, double* out,
                              diaq_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* DIAQ_H */
