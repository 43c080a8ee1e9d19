// Sharded state: a state vector larger than one device's memory is split
// across devices (Section II-A; Section VI names the multi-node backend,
// diaq-mpi). Here the 2^n amplitudes are split by the top g bits of the
// physical basis index into 2^g shards of 2^(n-g) amplitudes.
//
// Qubits are remapped rather than communicated gate by gate. A map sends
// each logical qubit to a physical bit: bits 0 .. n-g-1 are local (inside a
// shard), bits n-g .. n-1 global (the shard index). A gate whose targets
// are all local runs in every shard independently, on the targets'
// physical positions. A target on a global bit is first swapped with a
// local bit l: every shard pair differing in that global bit trades half
// its amplitudes (shard.cu), and the two logical qubits exchange physical
// bits. The local bit chosen is the one whose logical qubit is next needed
// furthest in the future (never one of the gate's own targets), so fewer
// exchanges follow. Optionally the schedule ends by restoring the
// identity map, with exchanges for the global bits and local SWAPs for the
// rest.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <limits>
#include <vector>

#include "internal.h"

namespace diaq {
namespace {

diaq_status check_shape(const diaq_gate* gates, int n_gates, int n_qubits, int g) {
    if (n_gates < 0 || (n_gates && !gates)) return fail(DIAQ_ERR_ARG, "bad gate array");
    if (n_qubits < 1 || n_qubits > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_qubits = %d out of range", n_qubits);
    if (g < 0 || g >= n_qubits) return fail(DIAQ_ERR_ARG, "global_bits = %d outside [0, %d)", g, n_qubits);
    if (g > 16) return fail(DIAQ_ERR_UNSUPPORTED, "global_bits = %d: at most 2^16 shards", g);
    const int n_local = n_qubits - g;
    for (int i = 0; i < n_gates; ++i) {
        const diaq_gate& q = gates[i];
        if (q.k < 1 || q.k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "gate %d: k = %d outside [1, %d]", i, q.k, DIAQ_MAX_K);
        if (q.k > n_local)
            return fail(DIAQ_ERR_UNSUPPORTED, "gate %d acts on %d qubits but a shard holds %d local qubits", i, q.k,
                        n_local);
        for (int a = 0; a < q.k; ++a) {
            if (q.targets[a] < 0 || q.targets[a] >= n_qubits)
                return fail(DIAQ_ERR_ARG, "gate %d: target %d outside [0, %d)", i, q.targets[a], n_qubits);
            for (int b = 0; b < a; ++b)
                if (q.targets[a] == q.targets[b]) return fail(DIAQ_ERR_ARG, "gate %d: repeated target", i);
        }
    }
    return DIAQ_OK;
}

struct Scheduler {
    int n, g, n_local;
    std::vector<int> phys, logi;  // logical -> physical, physical -> logical
    std::vector<diaq_shard_step> steps;
    // next_use[i][q]: first gate index >= i that uses logical qubit q
    std::vector<std::vector<int>> next_use;

    void exchange(int G, int p) {  // physical global position G with local position p
        diaq_shard_step s{};
        s.kind = DIAQ_SHARD_EXCHANGE;
        s.gate = -1;
        s.global_bit = G - n_local;
        s.local_bit = p;
        steps.push_back(s);
        const int qa = logi[G], qb = logi[p];
        logi[G] = qb;
        logi[p] = qa;
        phys[qa] = p;
        phys[qb] = G;
    }

    void local_swap(int p, int q) {
        diaq_shard_step s{};
        s.kind = DIAQ_SHARD_LOCAL_SWAP;
        s.gate = -1;
        s.k = 2;
        s.targets[0] = p;
        s.targets[1] = q;
        steps.push_back(s);
        const int qa = logi[p], qb = logi[q];
        logi[p] = qb;
        logi[q] = qa;
        phys[qa] = q;
        phys[qb] = p;
    }

    // local position to give up (its logical qubit not in `busy`): the one
    // whose qubit is next used furthest after gate index `from` - 1
    int victim(int from, const std::vector<int>& busy) {
        int best = -1, best_use = -1;
        for (int p = n_local - 1; p >= 0; --p) {
            const int q = logi[p];
            if (std::find(busy.begin(), busy.end(), q) != busy.end()) continue;
            const int use = next_use[size_t(from)][size_t(q)];
            if (use > best_use) {
                best_use = use;
                best = p;
            }
        }
        return best;
    }
};

}  // namespace
}  // namespace diaq

using namespace diaq;

extern "C" diaq_status diaq_shard_schedule(const diaq_gate* gates, int32_t n_gates, int32_t n_qubits,
                                           int32_t global_bits, int32_t restore, diaq_shard_step* steps,
                                           int32_t cap, int32_t* n_steps, int32_t* final_map) {
    clear_error();
    if (!n_steps) return fail(DIAQ_ERR_ARG, "n_steps is NULL");
    *n_steps = 0;
    DIAQ_TRY(check_shape(gates, n_gates, n_qubits, global_bits));
    Scheduler S;
    S.n = n_qubits;
    S.g = global_bits;
    S.n_local = n_qubits - global_bits;
    S.phys.resize(size_t(n_qubits));
    S.logi.resize(size_t(n_qubits));
    for (int q = 0; q < n_qubits; ++q) S.phys[size_t(q)] = S.logi[size_t(q)] = q;
    const int never = std::numeric_limits<int>::max();
    S.next_use.assign(size_t(n_gates) + 1, std::vector<int>(size_t(n_qubits), never));
    for (int i = n_gates - 1; i >= 0; --i) {
        S.next_use[size_t(i)] = S.next_use[size_t(i) + 1];
        for (int a = 0; a < gates[i].k; ++a) S.next_use[size_t(i)][size_t(gates[i].targets[a])] = i;
    }
    for (int i = 0; i < n_gates; ++i) {
        const diaq_gate& q = gates[i];
        std::vector<int> busy(q.targets, q.targets + q.k);
        for (int a = 0; a < q.k; ++a) {
            const int P = S.phys[size_t(q.targets[a])];
            if (P < S.n_local) continue;
            const int p = S.victim(i + 1, busy);
            if (p < 0) return fail(DIAQ_ERR_UNSUPPORTED, "gate %d: no local position to exchange with", i);
            S.exchange(P, p);
        }
        diaq_shard_step s{};
        s.kind = DIAQ_SHARD_APPLY;
        s.gate = i;
        s.k = q.k;
        for (int a = 0; a < q.k; ++a) s.targets[a] = S.phys[size_t(q.targets[a])];
        s.global_bit = -1;
        s.local_bit = -1;
        S.steps.push_back(s);
    }
    if (restore) {
        // global positions first: bring logical qubit G home to physical G
        for (int G = S.n_local; G < n_qubits; ++G) {
            if (S.logi[size_t(G)] == G) continue;
            int p = S.phys[size_t(G)];
            if (p >= S.n_local) {  // it sits on another global bit: make it local first
                const std::vector<int> none;
                const int l = S.victim(n_gates, none);
                S.exchange(p, l);
                p = S.phys[size_t(G)];
            }
            S.exchange(G, p);
        }
        // then the local permutation, one transposition at a time
        for (int p = 0; p < S.n_local; ++p)
            while (S.logi[size_t(p)] != p) S.local_swap(p, S.logi[size_t(p)]);
    }
    const int count = (int)S.steps.size();
    *n_steps = count;
    if (final_map)
        for (int q = 0; q < n_qubits; ++q) final_map[q] = S.phys[size_t(q)];
    if (!steps) return DIAQ_OK;
    if (cap < count) return fail(DIAQ_ERR_ARG, "steps holds %d entries, the schedule needs %d", cap, count);
    std::memcpy(steps, S.steps.data(), sizeof(diaq_shard_step) * size_t(count));
    return DIAQ_OK;
}

extern "C" diaq_status diaq_sharded_simulate(const diaq_gate* gates, int32_t n_gates, const double* theta,
                                             int32_t n_qubits, int32_t global_bits, diaq_dtype dtype,
                                             void* const* shards, int32_t restore, int32_t* final_map,
                                             diaq_stream_t stream) {
    clear_error();
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (!shards) return fail(DIAQ_ERR_ARG, "shards is NULL");
    int32_t count = 0;
    DIAQ_TRY(diaq_shard_schedule(gates, n_gates, n_qubits, global_bits, restore, nullptr, 0, &count, nullptr));
    std::vector<diaq_shard_step> steps(size_t(count) + 1);
    DIAQ_TRY(diaq_shard_schedule(gates, n_gates, n_qubits, global_bits, restore, steps.data(), count, &count,
                                 final_map));
    const int n_local = n_qubits - global_bits;
    const int S = 1 << global_bits;
    const size_t bytes = (size_t(1) << n_local) * amp_bytes(dtype);
    for (int s = 0; s < S; ++s) {
        if (!shards[s]) return fail(DIAQ_ERR_ARG, "shard %d is NULL", s);
        if (reinterpret_cast<uintptr_t>(shards[s]) & 15) return fail(DIAQ_ERR_ARG, "shard %d is not 16-byte aligned", s);
        for (int t = 0; t < s; ++t) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(shards[s]), b = reinterpret_cast<uintptr_t>(shards[t]);
            if (a < b + bytes && b < a + bytes) return fail(DIAQ_ERR_ARG, "shards %d and %d overlap", t, s);
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    static const double kSwap[32] = {1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0,
                                     0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0};
    // every op is built before the first apply and released after the last
    std::vector<diaq_op_t> ops(size_t(count), nullptr);
    auto release = [&]() {
        for (diaq_op_t o : ops)
            if (o) diaq_op_destroy(o);
    };
    for (int i = 0; i < count; ++i) {
        const diaq_shard_step& p = steps[size_t(i)];
        if (p.kind == DIAQ_SHARD_EXCHANGE) continue;
        diaq_gate lg{};
        if (p.kind == DIAQ_SHARD_APPLY) {
            lg = gates[p.gate];
        } else {
            lg.k = 2;
            lg.m = kSwap;
            lg.param = -1;
            lg.scale = 1.0;
        }
        for (int a = 0; a < p.k; ++a) lg.targets[a] = p.targets[a];
        diaq_status s = diaq_build(&lg, n_local, dtype, DIAQ_ONTHEFLY, theta, stream, &ops[size_t(i)]);
        if (s != DIAQ_OK) {
            release();
            return s;
        }
    }
    diaq_status result = DIAQ_OK;
    for (int i = 0; i < count && result == DIAQ_OK; ++i) {
        const diaq_shard_step& p = steps[size_t(i)];
        if (p.kind == DIAQ_SHARD_EXCHANGE) {
            for (int s = 0; s < S && result == DIAQ_OK; ++s)
                if (!((s >> p.global_bit) & 1))
                    result = launch_shard_swap(shards[s], shards[s | (1 << p.global_bit)], n_local, dtype, p.local_bit, st);
        } else {
            for (int s = 0; s < S && result == DIAQ_OK; ++s) result = diaq_apply(ops[size_t(i)], shards[s], shards[s], stream);
        }
    }
    if (result == DIAQ_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) result = cuda_fail(e, "cudaStreamSynchronize(sharded simulate)");
    }
    release();
    return result;
}

extern "C" diaq_status diaq_sharded_norm(void* const* shards, int32_t n_qubits, int32_t global_bits, diaq_dtype dtype,
                                         double* out, diaq_stream_t stream) {
    clear_error();
    if (!shards || !out) return fail(DIAQ_ERR_ARG, "shards or out is NULL");
    if (global_bits < 0 || global_bits >= n_qubits || global_bits > 16)
        return fail(DIAQ_ERR_ARG, "global_bits = %d out of range", global_bits);
    double total = 0.0;
    for (int s = 0; s < (1 << global_bits); ++s) {
        double v = 0.0;
        DIAQ_TRY(diaq_norm(shards[s], n_qubits - global_bits, dtype, &v, stream));
        total += v;  // one FP64 sum over the shards, in shard order
    }
    *out = total;
    return DIAQ_OK;
}

extern "C" diaq_status diaq_sharded_expect(void* const* shards, int32_t n_qubits, int32_t global_bits,
                                           diaq_dtype dtype, const int32_t* map, int32_t n_terms,
                                           const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                                           double* out, diaq_stream_t stream) {
    clear_error();
    if (!shards || !out) return fail(DIAQ_ERR_ARG, "shards or out is NULL");
    if (global_bits < 0 || global_bits >= n_qubits || global_bits > 16)
        return fail(DIAQ_ERR_ARG, "global_bits = %d out of range", global_bits);
    if (n_terms < 0 || (n_terms && (!xmask || !zmask || !coeff))) return fail(DIAQ_ERR_ARG, "bad term arrays");
    const int n_local = n_qubits - global_bits;
    std::vector<int> phys(static_cast<size_t>(n_qubits));
    for (int q = 0; q < n_qubits; ++q) {
        phys[size_t(q)] = map ? map[q] : q;
        if (phys[size_t(q)] < 0 || phys[size_t(q)] >= n_qubits) return fail(DIAQ_ERR_ARG, "map[%d] out of range", q);
        for (int r = 0; r < q; ++r)
            if (phys[size_t(r)] == phys[size_t(q)]) return fail(DIAQ_ERR_ARG, "map is not a permutation");
    }
    const uint64_t valid = (uint64_t(1) << n_qubits) - 1, local = (uint64_t(1) << n_local) - 1;
    // terms in physical bits; X or Y letters must sit on local bits
    std::vector<uint64_t> px(static_cast<size_t>(n_terms)), pz(static_cast<size_t>(n_terms));
    for (int t = 0; t < n_terms; ++t) {
        if ((xmask[t] | zmask[t]) & ~valid) return fail(DIAQ_ERR_ARG, "term %d acts on a qubit >= n_qubits", t);
        uint64_t x = 0, z = 0;
        for (int q = 0; q < n_qubits; ++q) {
            x |= ((xmask[t] >> q) & 1) << phys[size_t(q)];
            z |= ((zmask[t] >> q) & 1) << phys[size_t(q)];
        }
        if (x & ~local)
            return fail(DIAQ_ERR_UNSUPPORTED, "term %d has X or Y on a qubit held on a global bit; exchange it to a "
                                              "local bit first", t);
        px[size_t(t)] = x;
        pz[size_t(t)] = z;
    }
    // shard s: a Z on global bit G contributes (-1)^(bit G of s)
    std::vector<double> cs(size_t(2 * n_terms) + 2);
    std::vector<uint64_t> lz(size_t(n_terms) + 1);
    for (int t = 0; t < n_terms; ++t) lz[size_t(t)] = pz[size_t(t)] & local;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < (1 << global_bits); ++s) {
        for (int t = 0; t < n_terms; ++t) {
            const int sign = __builtin_popcountll((pz[size_t(t)] >> n_local) & uint64_t(s)) & 1;
            cs[size_t(2 * t)] = sign ? -coeff[2 * t] : coeff[2 * t];
            cs[size_t(2 * t + 1)] = sign ? -coeff[2 * t + 1] : coeff[2 * t + 1];
        }
        double v[2] = {0.0, 0.0};
        DIAQ_TRY(diaq_expect(shards[s], n_local, dtype, n_terms, px.data(), lz.data(), cs.data(), v, stream));
        re += v[0];
        im += v[1];
    }
    out[0] = re;
    out[1] = im;
    return DIAQ_OK;
}
