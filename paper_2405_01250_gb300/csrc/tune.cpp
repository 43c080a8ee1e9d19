// Autotuning and fusion planning for the on-the-fly gate apply.
//
//  * diaq_autotune_apply times the on-the-fly kernel for k = 1, 2, 3 over a
//    grid of launch shapes (threads per block x groups per thread) on the
//    caller's two state buffers and keeps the fastest shape per (dtype, k)
//    for every later launch in the process.
//  * diaq_plan_fusion groups consecutive gates for the DIA x DIA product
//    (Algorithm 1): a group grows while its union of targets stays within
//    max_k qubits and it holds at most max_depth gates.
//  * diaq_autotune_fusion runs a circuit once per fusion depth and reports
//    the depth with the shortest time; fusion trades passes over the state
//    for arithmetic per amplitude, which pays off only while the fused op
//    stays memory-bound (see the FP64 rate of GB300).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

using namespace diaq;

static diaq_status time_apply(int n, diaq_dtype dt, const GateDesc& g, void* x, void* y, int reps, float* ms,
                              cudaStream_t s) {
    cudaEvent_t e0, e1;
    DIAQ_CUDA(cudaEventCreate(&e0));
    DIAQ_CUDA(cudaEventCreate(&e1));
    diaq_status st = launch_gate_local(n, dt, g, nullptr, x, y, s);  // warm
    if (st == DIAQ_OK) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == DIAQ_OK; ++r) st = launch_gate_local(n, dt, g, nullptr, (r & 1) ? y : x, (r & 1) ? x : y, s);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess && st == DIAQ_OK) st = cuda_fail(e, "cudaEventSynchronize(tuning)");
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= float(reps);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// A representative gate per k on the top qubits (the stride of the largest
// offsets): k = 1 a real butterfly, k = 2 a controlled phase, k = 3 dense.
static GateDesc probe_gate(int n, int k) {
    GateDesc g;
    g.k = k;
    for (int a = 0; a < k; ++a) g.targets[a] = n - 1 - a;
    const int D = 1 << k;
    g.m.assign(size_t(D) * D, cplx(0, 0));
    if (k == 1) {
        const double h = std::sqrt(0.5);
        g.m = {h, h, h, -h};
    } else if (k == 2) {
        for (int r = 0; r < 4; ++r) g.m[size_t(r * 4 + r)] = 1.0;
        g.m[15] = cplx(std::cos(0.3), std::sin(0.3));
    } else {
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c) g.m[size_t(r * D + c)] = cplx(std::cos(0.1 * (r * D + c + 1)), std::sin(0.07 * (r + 2 * c))) / double(D);
    }
    return g;
}

extern "C" {

diaq_status diaq_autotune_apply(int32_t n_qubits, diaq_dtype dtype, void* x, void* y, int32_t reps,
                                diaq_apply_tuning* report, diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    if (!x || !y || x == y) return fail(DIAQ_ERR_ARG, "need two distinct device state buffers");
    if (n_qubits < 4 || n_qubits > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_qubits = %d outside [4, %d]", n_qubits, DIAQ_MAX_QUBITS);
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (reps < 1) reps = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int threads[] = {64, 128, 256};  // the kernel is built for at most 256
    const int groups[] = {1, 2, 4};
    int row = 0;
    for (int k = 1; k <= 3; ++k) {
        const GateDesc g = probe_gate(n_qubits, k);
        LaunchCfg& cfg = launch_cfg(dtype, k);
        const LaunchCfg saved = cfg;
        float best = 1e30f;
        LaunchCfg bestc = saved;
        for (int T : threads)
            for (int G : groups) {
                cfg.threads = T;
                cfg.groups = G;
                float ms = 0;
                diaq_status st = time_apply(n_qubits, dtype, g, x, y, reps, &ms, s);
                if (st != DIAQ_OK) {
                    cfg = saved;
                    return st;
                }
                if (report && row < DIAQ_APPLY_TUNE_MAX) {
                    report->k[row] = k;
                    report->threads[row] = T;
                    report->groups[row] = G;
                    report->ms[row] = ms;
                    ++row;
                }
                if (ms < best) {
                    best = ms;
                    bestc = cfg;
                }
            }
        cfg = bestc;
        if (report) {
            report->best_threads[k - 1] = bestc.threads;
            report->best_groups[k - 1] = bestc.groups;
            report->best_ms[k - 1] = best;
        }
    }
    if (report) report->n_rows = row;
    return DIAQ_OK;
}

diaq_status diaq_set_apply_launch(diaq_dtype dtype, int32_t k, int32_t threads, int32_t groups) {
    clear_error();
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (k < 1 || k > 3) return fail(DIAQ_ERR_ARG, "k = %d: launch shapes are tunable for k = 1..3", k);
    if (threads < 32 || threads > 256 || threads % 32)
        return fail(DIAQ_ERR_ARG, "threads = %d not a multiple of 32 in [32, 256]", threads);
    if (!(groups == 0 || groups == 1 || groups == 2 || groups == 4)) return fail(DIAQ_ERR_ARG, "groups = %d not in {0,1,2,4}", groups);
    LaunchCfg& c = launch_cfg(dtype, k);
    c.threads = threads;
    c.groups = groups;
    return DIAQ_OK;
}

diaq_status diaq_plan_fusion(const diaq_gate* gates, int32_t n_gates, int32_t max_k, int32_t max_depth,
                             int32_t* group_of_gate, int32_t* n_groups) {
    clear_error();
    if (n_gates < 0 || (n_gates && (!gates || !group_of_gate)) || !n_groups) return fail(DIAQ_ERR_ARG, "bad arrays");
    if (max_k < 1 || max_k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "max_k = %d outside [1, %d]", max_k, DIAQ_MAX_K);
    if (max_depth < 1) return fail(DIAQ_ERR_ARG, "max_depth = %d < 1", max_depth);
    int grp = -1, depth = 0;
    std::vector<int> uni;
    for (int i = 0; i < n_gates; ++i) {
        const diaq_gate& g = gates[i];
        if (g.k < 1 || g.k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "gate %d has k = %d", i, g.k);
        if (g.k > max_k) return fail(DIAQ_ERR_ARG, "gate %d (k = %d) exceeds max_k = %d", i, g.k, max_k);
        std::vector<int> u = uni;
        for (int a = 0; a < g.k; ++a)
            if (std::find(u.begin(), u.end(), g.targets[a]) == u.end()) u.push_back(g.targets[a]);
        if (grp < 0 || depth >= max_depth || int(u.size()) > max_k) {
            ++grp;
            depth = 0;
            u.assign(g.targets, g.targets + g.k);
        }
        uni = u;
        ++depth;
        group_of_gate[i] = grp;
    }
    *n_groups = grp + 1;
    return DIAQ_OK;
}

// A gate whose operator is diagonal in the computational basis: a fixed
// matrix with exact zeros off the diagonal, or a rotation whose generator
// has only I and Z letters.
static bool gate_is_diagonal(const diaq_gate& g) {
    if (g.param >= 0) {
        for (int a = 0; a < g.k; ++a)
            if (!strchr("IiZz", g.gen[a])) return false;
        return true;
    }
    if (!g.m) return false;
    const int D = 1 << g.k;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c)
            if (r != c && (g.m[2 * (r * D + c)] != 0.0 || g.m[2 * (r * D + c) + 1] != 0.0)) return false;
    return true;
}

diaq_status diaq_plan_fusion_diagonal(const diaq_gate* gates, int32_t n_gates, int32_t max_k, int32_t max_depth,
                                      int32_t* group_of_gate, int32_t* n_groups) {
    clear_error();
    if (n_gates < 0 || (n_gates && (!gates || !group_of_gate)) || !n_groups) return fail(DIAQ_ERR_ARG, "bad arrays");
    if (max_k < 1 || max_k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "max_k = %d outside [1, %d]", max_k, DIAQ_MAX_K);
    if (max_depth < 1) return fail(DIAQ_ERR_ARG, "max_depth = %d < 1", max_depth);
    int grp = -1, depth = 0;
    bool open_diag = false;  // the current group is a run of diagonal gates
    std::vector<int> uni;
    for (int i = 0; i < n_gates; ++i) {
        const diaq_gate& g = gates[i];
        if (g.k < 1 || g.k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "gate %d has k = %d", i, g.k);
        if (g.k > max_k) return fail(DIAQ_ERR_ARG, "gate %d (k = %d) exceeds max_k = %d", i, g.k, max_k);
        const bool diag = gate_is_diagonal(g);
        std::vector<int> u = uni;
        for (int a = 0; a < g.k; ++a)
            if (std::find(u.begin(), u.end(), g.targets[a]) == u.end()) u.push_back(g.targets[a]);
        if (!diag || !open_diag || depth >= max_depth || int(u.size()) > max_k) {
            ++grp;
            depth = 0;
            u.assign(g.targets, g.targets + g.k);
        }
        open_diag = diag;
        uni = u;
        ++depth;
        group_of_gate[i] = grp;
    }
    *n_groups = grp + 1;
    return DIAQ_OK;
}

diaq_status diaq_plan_fusion_commuting(const diaq_gate* gates, int32_t n_gates, int32_t max_k, int32_t max_depth,
                                       int32_t* order, int32_t* group_of_pos, int32_t* n_groups) {
    clear_error();
    if (n_gates < 0 || (n_gates && (!gates || !order || !group_of_pos)) || !n_groups)
        return fail(DIAQ_ERR_ARG, "bad arrays");
    if (max_k < 1 || max_k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "max_k = %d outside [1, %d]", max_k, DIAQ_MAX_K);
    if (max_depth < 1) return fail(DIAQ_ERR_ARG, "max_depth = %d < 1", max_depth);
    // A gate depends on the last block that touched any of its qubits; it may
    // join that block (the latest of them) if the block stays within max_k
    // qubits and max_depth gates: every block created after it touches none
    // of the gate's qubits, so the gate commutes past them unchanged.
    struct Block {
        std::vector<int> gates;
        std::vector<int> qubits;
    };
    std::vector<Block> blocks;
    std::vector<int> last;  // per qubit: last block touching it, -1 if none
    for (int i = 0; i < n_gates; ++i) {
        const diaq_gate& g = gates[i];
        if (g.k < 1 || g.k > DIAQ_MAX_K) return fail(DIAQ_ERR_ARG, "gate %d has k = %d", i, g.k);
        if (g.k > max_k) return fail(DIAQ_ERR_ARG, "gate %d (k = %d) exceeds max_k = %d", i, g.k, max_k);
        int dep = -1;
        for (int a = 0; a < g.k; ++a) {
            const int q = g.targets[a];
            if (q < 0) return fail(DIAQ_ERR_ARG, "gate %d has a negative target", i);
            if (q >= int(last.size())) last.resize(size_t(q) + 1, -1);
            dep = std::max(dep, last[size_t(q)]);
        }
        bool joined = false;
        // Blocks this gate depends on besides the latest one: one that no
        // later block has touched commutes forward past everything after
        // it, so it can merge into the latest block (their qubit sets are
        // disjoint, so the order between them does not matter).
        if (dep >= 0) {
            std::vector<int> others;
            for (int a = 0; a < g.k; ++a) {
                const int d = last[size_t(g.targets[a])];
                if (d >= 0 && d != dep && std::find(others.begin(), others.end(), d) == others.end()) others.push_back(d);
            }
            std::vector<int> u = blocks[size_t(dep)].qubits;
            size_t depth = blocks[size_t(dep)].gates.size() + 1;
            bool ok = true;
            for (int d : others) {
                const Block& A = blocks[size_t(d)];
                for (int q : A.qubits) ok &= last[size_t(q)] == d;
                for (int q : A.qubits)
                    if (std::find(u.begin(), u.end(), q) == u.end()) u.push_back(q);
                depth += A.gates.size();
            }
            for (int a = 0; a < g.k; ++a)
                if (std::find(u.begin(), u.end(), g.targets[a]) == u.end()) u.push_back(g.targets[a]);
            if (ok && !others.empty() && int(u.size()) <= max_k && int(depth) <= max_depth) {
                Block& B = blocks[size_t(dep)];
                std::vector<int> merged;
                for (int d : others) {
                    merged.insert(merged.end(), blocks[size_t(d)].gates.begin(), blocks[size_t(d)].gates.end());
                    for (int q : blocks[size_t(d)].qubits) last[size_t(q)] = dep;
                    blocks[size_t(d)].gates.clear();
                    blocks[size_t(d)].qubits.clear();
                }
                merged.insert(merged.end(), B.gates.begin(), B.gates.end());
                merged.push_back(i);
                B.gates = merged;
                B.qubits = u;
                joined = true;
            }
        }
        if (!joined && dep >= 0) {
            Block& B = blocks[size_t(dep)];
            std::vector<int> u = B.qubits;
            for (int a = 0; a < g.k; ++a)
                if (std::find(u.begin(), u.end(), g.targets[a]) == u.end()) u.push_back(g.targets[a]);
            if (int(u.size()) <= max_k && int(B.gates.size()) < max_depth) {
                B.gates.push_back(i);
                B.qubits = u;
                joined = true;
            }
        }
        if (!joined) {
            Block B;
            B.gates.push_back(i);
            B.qubits.assign(g.targets, g.targets + g.k);
            blocks.push_back(B);
            dep = int(blocks.size()) - 1;
        }
        for (int a = 0; a < g.k; ++a) last[size_t(g.targets[a])] = dep;
    }
    int pos = 0, grp = 0;
    for (size_t b = 0; b < blocks.size(); ++b) {
        if (blocks[b].gates.empty()) continue;  // merged into a later block
        for (int gi : blocks[b].gates) {
            order[pos] = gi;
            group_of_pos[pos] = grp;
            ++pos;
        }
        ++grp;
    }
    *n_groups = grp;
    return DIAQ_OK;
}

diaq_status diaq_autotune_fusion(const diaq_gate* gates, int32_t n_gates, const double* theta, int32_t n_qubits,
                                 diaq_dtype dtype, void* work, int32_t max_k, int32_t max_depth, int32_t commuting,
                                 diaq_fusion_tuning* report, diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    if (!work || !report) return fail(DIAQ_ERR_ARG, "work and report are required");
    if (max_depth < 1 || max_depth > DIAQ_FUSION_TUNE_MAX) return fail(DIAQ_ERR_ARG, "max_depth outside [1, %d]", DIAQ_FUSION_TUNE_MAX);
    if (n_gates < 1 || !gates) return fail(DIAQ_ERR_ARG, "need at least one gate");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> grp(static_cast<size_t>(n_gates)), order(static_cast<size_t>(n_gates));
    float best = 1e30f;
    int bestd = 1;
    for (int d = 1; d <= max_depth; ++d) {
        int32_t ng = 0;
        if (commuting) {
            DIAQ_TRY(diaq_plan_fusion_commuting(gates, n_gates, max_k, d, order.data(), grp.data(), &ng));
        } else {
            DIAQ_TRY(diaq_plan_fusion(gates, n_gates, max_k, d, grp.data(), &ng));
            for (int i = 0; i < n_gates; ++i) order[size_t(i)] = i;
        }
        std::vector<diaq_op_t> ops;
        diaq_status st = DIAQ_OK;
        for (int i = 0; i < n_gates && st == DIAQ_OK;) {
            int j = i;
            std::vector<diaq_op_t> part;
            while (j < n_gates && grp[size_t(j)] == grp[size_t(i)] && st == DIAQ_OK) {
                diaq_op_t o = nullptr;
                st = diaq_build(&gates[order[size_t(j)]], n_qubits, dtype, DIAQ_ONTHEFLY, theta, stream, &o);
                if (st == DIAQ_OK) part.push_back(o);
                ++j;
            }
            if (st == DIAQ_OK) {
                if (part.size() == 1) {
                    ops.push_back(part[0]);
                    part.clear();
                } else {
                    diaq_op_t f = nullptr;
                    st = diaq_fuse(part.data(), int32_t(part.size()), DIAQ_ONTHEFLY, stream, &f);
                    if (st == DIAQ_OK) ops.push_back(f);
                }
            }
            for (diaq_op_t o : part) diaq_op_destroy(o);
            i = j;
        }
        float ms = 0;
        if (st == DIAQ_OK) {
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (diaq_op_t o : ops)
                if (st == DIAQ_OK) st = launch_onthefly(o, work, work, s);  // warm
            cudaEventRecord(e0, s);
            for (diaq_op_t o : ops)
                if (st == DIAQ_OK) st = launch_onthefly(o, work, work, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        for (diaq_op_t o : ops) diaq_op_destroy(o);
        if (st != DIAQ_OK) return st;
        report->ops[d - 1] = ng;
        report->ms[d - 1] = ms;
        if (ms < best) {
            best = ms;
            bestd = d;
        }
    }
    report->n_depths = max_depth;
    report->best_depth = bestd;
    return DIAQ_OK;
}

}  // extern "C"
