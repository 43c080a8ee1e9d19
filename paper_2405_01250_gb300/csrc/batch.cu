// Batched energies and adjoint gradients: many circuits of uneven qubit
// counts in one persistent launch, replayed from a CUDA graph.
//
// Each circuit ("instance") is processed by a team of C thread blocks that
// form one thread-block cluster. A team runs the instance's whole adjoint
// computation (forward sweep, lambda = H psi with the energy, reverse sweep
// with the per-gate gradient partials) on the instance's own two state
// buffers in the arena; between gates the team meets at the hardware
// cluster barrier, so no block ever spins on a flag. Teams take instances
// from a static schedule computed on the host (largest first, round robin
// over teams), so the grid is sized to the teams that fit on the GPU at once
// and every team works until its list is done. A second small kernel sums
// the per-block partials of every instance in a fixed order.
//
// Gates have k <= 2 targets; a parametric gate is exp(-i a/2 P) with
// a = scale * theta[param] and P a Pauli string, built on the device from
// the instance's parameters so one captured graph serves every theta.

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "bounds.cuh"
#include "common.cuh"
#include "internal.h"
#include "phase.cuh"
#include "rot.cuh"
#include "win.cuh"

namespace cg = cooperative_groups;

DIAQ_BOUNDS_TU(batch)

namespace diaq {

// ---------------------------------------------------------------------------
// Device records
// ---------------------------------------------------------------------------
struct BGate {
    int32_t k;          // 1 or 2
    int32_t t[2];       // targets, t[0] most significant local bit
    int32_t param;      // -1 fixed
    int32_t pauli[2];   // generator letters 0=I 1=X 2=Y 3=Z (parametric)
    int32_t slot;       // partial-sum row of a parametric gate (instance relative), else -1
    int32_t xl;         // local X mask of the generator (parametric)
    double scale;
    RotShape rot;       // targets, offsets, Z mask and Y count (parametric)
    double re[16], im[16];  // fixed gate matrix (row-major, 2^k x 2^k)
};

// Gates that the fused pair kernels (rot2_groups) take: parametric, one
// qubit, an X or Y generator.
__host__ __device__ __forceinline__ bool pair_gate(const BGate& g) {
    return g.param >= 0 && g.k == 1 && g.xl == 1 && (g.pauli[0] == 1 || g.pauli[0] == 2);
}

// Two consecutive entries of an execution list that run as one pair.
__host__ __device__ __forceinline__ bool pair_entries(const BGate* gates, int32_t e1, int32_t e2) {
    return e1 >= 0 && e2 >= 0 && pair_gate(gates[e1]) && pair_gate(gates[e2]) && gates[e1].t[0] != gates[e2].t[0];
}

struct BInst {
    int32_t n;
    int32_t gate_begin, gate_end;
    int32_t exec_begin, exec_end;    // execution list of the per-gate kernel (gates and diagonal runs)
    int32_t exec_fwd_begin;          // the forward sweep starts here: past the leading product layer
    int32_t init_tab;                // that layer's chunk tables (product_layer), or -1: start from |0...0>
    int32_t exec_rev_begin;          // the reverse sweep stops here: the earliest entry with a gradient term
    int32_t block_begin, block_end;  // window blocks of the instance (window-fused kernel)
    int32_t param_begin, n_params;
    int32_t term_begin, term_end;
    int32_t n_slots;         // 1 (energy) + parametric gates
    int64_t psi_off, lam_off;  // amplitude offsets in the arena
    int64_t part_off;        // first partial (doubles), rows of C columns
};

// Rotation applications (forward and reverse) up to which the scaled form
// (rot_groups_s) needs no renormalisation: the stored states grow by at most
// sqrt(2) per rotation, so they, and the products of psi and lambda behind
// the energy and the gradient terms, stay below 2^960 << 2^1023.
constexpr int DIAQ_SCALED_MAX_ROT = 960;

struct BTerm {
    uint64_t x, z;
    double kr, ki;  // coefficient times i^{#Y}
    // group header, valid on the first term of each group of equal X masks
    // (lambda_tables): the group's term count, how its weight is looked up
    // (0: by the number of terms of odd parity, every coefficient equal;
    // 1: per chunk of 8 terms by their parity bits, chunk values summed),
    // its first table entry, and whether every weight is real
    int32_t gn, gmode, gtab, greal;
    // count-form groups of at least kLamClassMin terms: the terms sorted by
    // their Z mask's bits 5..7 (class k), gk[k] of class k, and gcls = 1
    int32_t gcls;
    int16_t gk[8];
};

constexpr int kLamClassMin = 4;

struct BatchArgs {
    const BInst* inst;
    const BGate* gates;
    const int32_t* exec;       // gate index, or -1 - run index
    const PhaseRun* runs;      // diagonal runs (weight form)
    const double2* ptabs;      // their phase tables: (run, direction) at (2 run + dir) PR_TAB_WEIGHT
    const void* init;          // product-layer tables of the instances (BInst::init_tab), state precision
    const BTerm* terms;
    const void* ltab;          // weight tables of the observables' term groups (lambda_tables), state precision
    int lflags;                // LAM_* flags that hold for every instance
    const int32_t* sched;      // instance ids, team-major: sched[team_first[c] .. team_first[c+1])
    const int32_t* team_first;
    const double* theta;
    void* arena;
    double* partials;
    int C;                     // blocks per team (cluster size)
    int scaled;                // rotations in the scaled form (rot_groups_s; complex128)
};

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pauli2(int letter, int r, int c, double* re, double* im) {
    // single-qubit Pauli element <r|sigma|c>
    *re = 0.0;
    *im = 0.0;
    switch (letter) {
        case 0: *re = (r == c) ? 1.0 : 0.0; break;
        case 1: *re = (r != c) ? 1.0 : 0.0; break;
        case 2: if (r != c) *im = (r == 0) ? -1.0 : 1.0; break;
        default: if (r == c) *re = (r == 0) ? 1.0 : -1.0; break;
    }
}

__device__ __forceinline__ uint8_t dev_entry_type(double re, double im) {
    if (re == 0.0 && im == 0.0) return 0;
    if (im == 0.0) return re == 1.0 ? 1 : 2;
    if (re == 0.0) return 3;
    return 4;
}

// Shared-memory gate matrices of the current step, written by thread 0.
template <typename R>
struct StepMats {
    R ure[16], uim[16];
    uint8_t uty[16];
    R pre[16], pim[16];
    uint8_t pty[16];
    int has_p;
};

// U (or U^dag when dagger) and, for parametric gates, P into smem.
template <typename R>
__device__ __noinline__ void build_step(const BGate& g, const double* theta, bool dagger, StepMats<R>* s) {
    const int D = 1 << g.k;
    double ur[16], ui[16];
    if (g.param < 0) {
        for (int e = 0; e < D * D; ++e) {
            ur[e] = g.re[e];
            ui[e] = g.im[e];
        }
    } else {
        const double a = g.scale * theta[g.param];
        double sn, cs;
        sincos(0.5 * a, &sn, &cs);
        for (int r = 0; r < D; ++r)
            for (int c = 0; c < D; ++c) {
                double pr = 1.0, pi = 0.0;
                for (int q = 0; q < g.k; ++q) {
                    double er, ei;
                    pauli2(g.pauli[q], (r >> (g.k - 1 - q)) & 1, (c >> (g.k - 1 - q)) & 1, &er, &ei);
                    const double nr = pr * er - pi * ei, ni = pr * ei + pi * er;
                    pr = nr;
                    pi = ni;
                }
                // U = cos I - i sin P
                ur[r * D + c] = (r == c ? cs : 0.0) + sn * pi;
                ui[r * D + c] = -sn * pr;
                s->pre[r * D + c] = R(pr);
                s->pim[r * D + c] = R(pi);
                s->pty[r * D + c] = dev_entry_type(pr, pi);
            }
    }
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            double vr = ur[r * D + c], vi = ui[r * D + c];
            if (dagger) {
                vr = ur[c * D + r];
                vi = -ui[c * D + r];
            }
            s->ure[r * D + c] = R(vr);
            s->uim[r * D + c] = R(vi);
            s->uty[r * D + c] = dev_entry_type(double(R(vr)), double(R(vi)));
        }
    s->has_p = g.param >= 0;
}

__device__ __forceinline__ void team_sync(int C) {
    if (C == 1) {
        __syncthreads();
    } else {
        __threadfence();
        cg::this_cluster().sync();
    }
}

// A fixed gate over the team's share of the groups, in place on psi (and,
// in the reverse sweep, lam). Each thread takes U groups per iteration (all
// loads issued before any arithmetic); the 2^k x 2^k matrix is copied into
// registers once, since the stores in the loop would otherwise force every
// entry to be reloaded.
template <typename R, int K, int U>
__device__ __noinline__ void team_fixed_u(amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam, int n,
                                          const BGate& g, const StepMats<R>& s, int64_t tid, int64_t nthreads) {
    constexpr int D = 1 << K;
    constexpr int DD = D * D;
    using A = amp_t<R>;
    int st[K];
    int64_t off[D];
    {
        int a = g.t[0], b = K == 2 ? g.t[1] : 0;
        if (K == 1) {
            st[0] = a;
        } else {
            st[0] = a < b ? a : b;
            st[K - 1] = a < b ? b : a;
        }
        for (int c = 0; c < D; ++c) {
            int64_t o = 0;
            for (int q = 0; q < K; ++q)
                if ((c >> (K - 1 - q)) & 1) o += int64_t(1) << g.t[q];
            off[c] = o;
        }
    }
    R ur[DD], ui[DD];
    uint8_t ut[DD];
#pragma unroll
    for (int e = 0; e < DD; ++e) {
        ur[e] = s.ure[e];
        ui[e] = s.uim[e];
        ut[e] = s.uty[e];
    }
    const int64_t G = int64_t(1) << (n - K);
    for (int64_t g0 = tid; g0 < G; g0 += int64_t(U) * nthreads) {
        int64_t b[U];
        A p[U][D], l[U][D];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t gi = g0 + int64_t(u) * nthreads;
            b[u] = gi < G ? insert_zeros<K>(gi, st) : int64_t(-1);
            if (b[u] >= 0 && !DIAQ_BOUNDS_OK(b[u] + off[D - 1], int64_t(1) << n, BS_WINDOW)) b[u] = -1;
            if (b[u] >= 0) {
#pragma unroll
                for (int c = 0; c < D; ++c) p[u][c] = psi[b[u] + off[c]];
                if (lam) {
#pragma unroll
                    for (int c = 0; c < D; ++c) l[u][c] = lam[b[u] + off[c]];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b[u] < 0) continue;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                A w;
                w.x = R(0);
                w.y = R(0);
                bool f = true;
#pragma unroll
                for (int c = 0; c < D; ++c) mac_typed<R>(w, f, ut[r * D + c], ur[r * D + c], ui[r * D + c], p[u][c]);
                psi[b[u] + off[r]] = w;
            }
            if (lam) {
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    A w;
                    w.x = R(0);
                    w.y = R(0);
                    bool f = true;
#pragma unroll
                    for (int c = 0; c < D; ++c) mac_typed<R>(w, f, ut[r * D + c], ur[r * D + c], ui[r * D + c], l[u][c]);
                    lam[b[u] + off[r]] = w;
                }
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void team_fixed(amp_t<R>* psi, amp_t<R>* lam, int n, const BGate& g, const StepMats<R>& s,
                                           int64_t tid, int64_t nthreads) {
    if (g.k == 1) {
        team_fixed_u<R, 1, 1>(psi, lam, n, g, s, tid, nthreads);
    } else {
        team_fixed_u<R, 2, 1>(psi, lam, n, g, s, tid, nthreads);
    }
}

// kappa for U (dagger = false) or U^dag of a rotation, from its angle:
// kappa = -i sin(a/2) i^ny, kappa' = +i sin(a/2) i^ny.
__device__ __forceinline__ void rot_angle(const BGate& g, const double* theta, bool dagger, double* cs, double* kr,
                                          double* ki) {
    double sn, c;
    sincos(0.5 * g.scale * theta[g.param], &sn, &c);
    double2 z = make_double2(0.0, dagger ? sn : -sn);  // -+ i sin
    z = mul_ipow(z, g.rot.ny);
    *cs = c;
    *kr = z.x;
    *ki = z.y;
}

// (H psi)_i for terms sorted by X mask: per group of equal masks the signed
// weight W = sum_t kappa_t (-1)^{popc((i ^ x) & z_t)} times psi[i ^ x]. W
// takes no floating-point work: it depends only on the parity bits of the
// group's terms, and is read from the group's table (lambda_tables) - by
// the number of odd parities when the coefficients are equal (a sum of ZZ
// couplings with one weight), else per chunk of 8 terms by their parity
// bits, the chunks' values summed. A real W (real coefficients, even Y
// counts) then costs two fused multiply-adds. Arithmetic in the state's
// precision.
// FL: LAM_REAL when every group's weight is real, LAM_COUNT when every group
// is looked up by its count of odd parities; with both the loop issues no
// FP64 instruction that a group does not need (branches whose FP64 work the
// compiler would predicate off, but still issue, are compiled out).
constexpr int LAM_REAL = 1;
constexpr int LAM_COUNT = 2;

template <typename R, int FL = 0>
__device__ __forceinline__ amp_t<R> pauli_lambda_elem(const amp_t<R>* psi, const BTerm* terms, const amp_t<R>* tab,
                                                      int t0, int t1, int64_t i) {
    using A = amp_t<R>;
    R lr = R(0), li = R(0);
    int t = t0;
    while (t < t1) {
        const BTerm& h = terms[t];
        const uint64_t j = uint64_t(i) ^ h.x;
        const int gn = h.gn;
        R wr, wi;
        if ((FL & LAM_COUNT) || h.gmode == 0) {
            int m = 0;
            for (int u = t; u < t + gn; ++u) m += __popcll(j & terms[u].z) & 1;
            const A w = tab[h.gtab + m];
            wr = w.x;
            wi = w.y;
        } else {
            wr = R(0);
            wi = R(0);
            for (int c = 0; 8 * c < gn; ++c) {
                int bits = 0;
                const int u1 = min(t + 8 * c + 8, t + gn);
                for (int u = t + 8 * c; u < u1; ++u) bits |= (__popcll(j & terms[u].z) & 1) << (u - t - 8 * c);
                const A w = tab[h.gtab + 256 * c + bits];
                if (c == 0) {
                    wr = w.x;
                    wi = w.y;
                } else {
                    wr += w.x;
                    wi += w.y;
                }
            }
        }
        const A pj = psi[j];
        if ((FL & LAM_REAL) || h.greal) {
            lr = fma(wr, pj.x, lr);
            li = fma(wr, pj.y, li);
        } else {
            lr = fma(wr, pj.x, fma(-wi, pj.y, lr));
            li = fma(wr, pj.y, fma(wi, pj.x, li));
        }
        t += gn;
    }
    A o;
    o.x = lr;
    o.y = li;
    return o;
}

// lam = H psi, returning this thread's share of Re <psi|lam>; FL (LAM_*)
// selects the instantiation outside the loop. Amplitudes by aligned blocks
// of 256 as in the diagonal runs: warp w of the grid (nth / 32 warps; nth a
// multiple of 32) takes blocks w, w + nth / 32, ..., its lane l the
// amplitudes l + 32 j (j = 0..7). A count-form group of at least
// kLamClassMin terms then counts its odd parities for all eight at once:
// with y = (base | l) ^ x, the parity of term u at amplitude j is
// a_u ^ parity(s & k_u) (a_u = parity(y & z_u) outside bits 5..7, k_u = bits
// 5..7 of z_u, s = j ^ bits 5..7 of x), so with D_k = n_k - 2 sum_{u in k} a_u
// the count is sum_u a_u + (sum_k D_k - WHT(D)[s]) / 2: one pass over the
// group's terms per 8 amplitudes. Other groups take one pass per amplitude.
template <typename R, int FL>
__device__ __noinline__ double lambda_share(const amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam,
                                            const BTerm* terms, const amp_t<R>* tab, int t0, int t1, int64_t N,
                                            int64_t tid, int64_t nth) {
    using A = amp_t<R>;
    Acc<R> e;
    const int lane = int(tid & 31);
    const int64_t nblk = (N + 255) >> 8;
    for (int64_t blk = tid >> 5; blk < nblk; blk += nth >> 5) {
        const int64_t base = blk << 8;
        R lr[8], li[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            lr[j] = R(0);
            li[j] = R(0);
        }
        for (int t = t0; t < t1;) {
            const BTerm& h = terms[t];
            const int gn = h.gn;
            const bool real = (FL & LAM_REAL) || h.greal;
            int m8[8];
            if (((FL & LAM_COUNT) || h.gmode == 0) && h.gcls) {
                const uint64_t ym = ((uint64_t(base) | uint64_t(lane)) ^ h.x) & ~uint64_t(0xE0);
                int D[8];
                int odd_tot = 0;
                int u = t;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    int odd = 0;
                    const int end = u + h.gk[k];
                    for (; u < end; ++u) odd += __popcll(ym & terms[u].z) & 1;
                    D[k] = h.gk[k] - 2 * odd;
                    odd_tot += odd;
                }
                const int dtot = gn - 2 * odd_tot;
#pragma unroll
                for (int hh = 1; hh < 8; hh <<= 1)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        if (!(k & hh)) {
                            const int a = D[k], b = D[k + hh];
                            D[k] = a + b;
                            D[k + hh] = a - b;
                        }
                const int xj = int((h.x >> 5) & 7);
#pragma unroll
                for (int j = 0; j < 8; ++j) m8[j] = odd_tot + ((dtot - D[j ^ xj]) >> 1);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t i = base + lane + 32 * j;
                if (i >= N) break;  // n < 8 only
                const uint64_t jx = uint64_t(i) ^ h.x;
                R wr, wi;
                if (((FL & LAM_COUNT) || h.gmode == 0) && h.gcls) {
                    const A w = tab[h.gtab + m8[j]];
                    wr = w.x;
                    wi = w.y;
                } else if ((FL & LAM_COUNT) || h.gmode == 0) {
                    int m = 0;
                    for (int v = t; v < t + gn; ++v) m += __popcll(jx & terms[v].z) & 1;
                    const A w = tab[h.gtab + m];
                    wr = w.x;
                    wi = w.y;
                } else {
                    wr = R(0);
                    wi = R(0);
                    for (int c = 0; 8 * c < gn; ++c) {
                        int bits = 0;
                        const int v1 = min(t + 8 * c + 8, t + gn);
                        for (int v = t + 8 * c; v < v1; ++v)
                            bits |= (__popcll(jx & terms[v].z) & 1) << (v - t - 8 * c);
                        const A w = tab[h.gtab + 256 * c + bits];
                        if (c == 0) {
                            wr = w.x;
                            wi = w.y;
                        } else {
                            wr += w.x;
                            wi += w.y;
                        }
                    }
                }
                const A pj = psi[jx];
                if (real) {
                    lr[j] = fma(wr, pj.x, lr[j]);
                    li[j] = fma(wr, pj.y, li[j]);
                } else {
                    lr[j] = fma(wr, pj.x, fma(-wi, pj.y, lr[j]));
                    li[j] = fma(wr, pj.y, fma(wi, pj.x, li[j]));
                }
            }
            t += gn;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t i = base + lane + 32 * j;
            if (i >= N) break;
            A o;
            o.x = lr[j];
            o.y = li[j];
            lam[i] = o;
            const A pi = psi[i];
            e.add_dot(pi.x, o.x, pi.y, o.y);
        }
    }
    return e.value();
}

template <typename R>
__device__ __forceinline__ double lambda_share_any(int fl, const amp_t<R>* psi, amp_t<R>* lam, const BTerm* terms,
                                                   const amp_t<R>* tab, int t0, int t1, int64_t N, int64_t tid,
                                                   int64_t nth) {
    switch (fl & 3) {
        case 3: return lambda_share<R, 3>(psi, lam, terms, tab, t0, t1, N, tid, nth);
        case 1: return lambda_share<R, 1>(psi, lam, terms, tab, t0, t1, N, tid, nth);
        case 2: return lambda_share<R, 2>(psi, lam, terms, tab, t0, t1, N, tid, nth);
        default: return lambda_share<R, 0>(psi, lam, terms, tab, t0, t1, N, tid, nth);
    }
}

// Amplitude i of a product state from its chunk tables: tab[c 256 + v] is
// the factor of the qubits 8c .. 8c+7 for their bit values v, the product
// taken over the chunks in order (product_layer).
template <typename R>
__device__ __forceinline__ amp_t<R> product_amp(const amp_t<R>* __restrict__ tab, int n, int64_t i) {
    amp_t<R> p = tab[i & 255];
    for (int c = 1; 8 * c < n; ++c) {
        const amp_t<R> t = tab[c * 256 + int((i >> (8 * c)) & 255)];
        const R qr = t.x, qi = t.y;
        const R tr = fma(p.x, qr, -p.y * qi);
        p.y = fma(p.x, qi, p.y * qr);
        p.x = tr;
    }
    return p;
}

// The pair of one-qubit X/Y rotations (a then b) for the team kernel:
// dispatch on the generators and the form, one group per iteration.
template <typename R, bool SC>
__device__ __forceinline__ void team_rot2(amp_t<R>* psi, amp_t<R>* lam, int n, const BGate& ga, const BGate& gb,
                                          const double* ca, const double* cb, int64_t tid, int64_t nth, double* pa,
                                          double* pb) {
    // ca, cb: (c0, c1, m1) of Rot1 for the direction
    const int qa = ga.t[0], qb = gb.t[0];
    if (ga.pauli[0] == 1) {
        const Rot1<R, 1, SC> A{R(ca[0]), R(ca[1]), ca[2] != 0.0};
        if (gb.pauli[0] == 1) {
            const Rot1<R, 1, SC> B{R(cb[0]), R(cb[1]), cb[2] != 0.0};
            rot2_groups<R, 1, 1, SC, 1>(psi, lam, n, qa, qb, A, B, tid, nth, pa, pb);
        } else {
            const Rot1<R, 2, SC> B{R(cb[0]), R(cb[1]), cb[2] != 0.0};
            rot2_groups<R, 1, 2, SC, 1>(psi, lam, n, qa, qb, A, B, tid, nth, pa, pb);
        }
    } else {
        const Rot1<R, 2, SC> A{R(ca[0]), R(ca[1]), ca[2] != 0.0};
        if (gb.pauli[0] == 1) {
            const Rot1<R, 1, SC> B{R(cb[0]), R(cb[1]), cb[2] != 0.0};
            rot2_groups<R, 2, 1, SC, 1>(psi, lam, n, qa, qb, A, B, tid, nth, pa, pb);
        } else {
            const Rot1<R, 2, SC> B{R(cb[0]), R(cb[1]), cb[2] != 0.0};
            rot2_groups<R, 2, 2, SC, 1>(psi, lam, n, qa, qb, A, B, tid, nth, pa, pb);
        }
    }
}

// Thread 0 of each team block: Rot1 coefficients (c0, c1, m1) of a pair
// member for one direction; in the scaled form also multiplies inv_s by its
// sigma.
__device__ __forceinline__ void team_rot1_coefs(const BGate& g, const double* th, bool dagger, bool scaled,
                                                double* c, double* inv_s) {
    double cs, kr, ki;
    rot_angle(g, th, dagger, &cs, &kr, &ki);
    if (scaled) {
        int m1;
        double sg;
        rot_scaled_coefs(cs, kr, ki, g.rot.ny, &m1, &c[0], &sg);
        c[1] = 0.0;
        c[2] = m1;
        *inv_s *= sg;
    } else {
        c[0] = cs;
        c[1] = g.pauli[0] == 1 ? ki : kr;  // kappa's non-zero part
        c[2] = 0.0;
    }
}

// complex64 teams take up to three consecutive one-qubit X/Y rotations on
// distinct qubits per pass (rotq_groups): one cluster barrier per tile. (The
// adjoint plan keeps pairs in complex64 too: there one launch per tile ran
// slower than one per pair.)
constexpr int kTeamTile = 3;

// Amplitudes whose loads a team thread keeps in flight in a diagonal run
// (phase_run_sweep): the team kernel runs at 128 registers (complex64 with
// four measured 3 % slower than with one: QAOA-256, 162.5 against 157.6 ms).
template <typename R>
constexpr int kTeamLoads = sizeof(R) == 4 ? 1 : 2;

// The tile of the execution list at position x (dir +1 forward, -1 backward,
// not past lim): its length and gate indices in execution order.
__device__ __forceinline__ int team_tile(const BatchArgs& a, int x, int dir, int lim, int* g) {
    int nq = 0;
    uint64_t used = 0;
    int gs[kTeamTile];
    for (int y = x; nq < kTeamTile; y += dir) {
        if (dir > 0 ? y >= lim : y < lim) break;
        const int e = a.exec[y];
        if (e < 0 || !pair_gate(a.gates[e])) break;
        const uint64_t bit = uint64_t(1) << a.gates[e].t[0];
        if (used & bit) break;
        used |= bit;
        gs[nq++] = e;
    }
    for (int j = 0; j < nq; ++j) g[j] = dir > 0 ? gs[j] : gs[nq - 1 - j];
    return nq;
}

// RotG of a tile member for one direction (thread 0 writes it to shared).
template <typename R>
__device__ __forceinline__ void team_rotg(const BGate& G, const double* th, bool dagger, RotG<R>* out, int* q) {
    double cs, kr, ki;
    rot_angle(G, th, dagger, &cs, &kr, &ki);
    const bool neg0 = (G.rot.zl & 1) != 0;
    out->a = R(cs);
    out->br[0] = R(neg0 ? -kr : kr);
    out->bi[0] = R(neg0 ? -ki : ki);
    out->br[1] = R(kr);
    out->bi[1] = R(ki);
    const double2 p0 = mul_ipow(make_double2(neg0 ? -1.0 : 1.0, 0.0), G.rot.ny);
    const double2 p1 = mul_ipow(make_double2(1.0, 0.0), G.rot.ny);
    out->pr[0] = R(p0.x);
    out->pi[0] = R(p0.y);
    out->pr[1] = R(p1.x);
    out->pi[1] = R(p1.y);
    *q = G.t[0];
}

template <typename R, int NQ>
__device__ __noinline__ void team_rotq(amp_t<R>* psi, amp_t<R>* lam, int n, const int* q, const RotG<R>* rot,
                                       int64_t tid, int64_t nth, double* part) {
    int qq[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) qq[j] = q[j];
    rotq_groups<R, NQ>(psi, lam, n, qq, rot, tid, nth, part);  // coefficients read from shared memory
}

// Phase tables of every diagonal run, both directions, once per replay:
// block (run, direction) writes its table at out + (2 run + dir) stride.
__global__ void __launch_bounds__(256) k_phase_tables(const PhaseRun* __restrict__ runs, const double* __restrict__ theta,
                                                      int n, int stride, double2* __restrict__ out) {
    const PhaseRun& r = runs[blockIdx.x];
    const bool rev = blockIdx.y != 0;
    const int E = min(phase_entries(r, n), stride);
    double2* dst = out + (int64_t(blockIdx.x) * 2 + blockIdx.y) * stride;
    for (int e = threadIdx.x; e < E; e += blockDim.x) dst[e] = phase_entry(r, theta + r.param_base, rev, e);
}

template <typename R>
__global__ void __launch_bounds__(256, 2) k_batch(const BatchArgs a) {
    using A = amp_t<R>;
    __shared__ StepMats<R> mats;
    __shared__ PhaseTables<PR_TAB_WEIGHT, R> ptab;
    __shared__ double warps[32];
    __shared__ double ang[3];
    __shared__ double sang[2];  // scaled form: m1, V's coefficient
    __shared__ double pang[6];  // a fused pair: Rot1 coefficients of both members
    __shared__ RotG<R> tg[kTeamTile];  // a complex64 tile's rotations
    __shared__ int tq[kTeamTile];
    const int C = a.C;
    const bool scaled = sizeof(R) == 8 && a.scaled != 0;
    const int rank = C == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const int team = blockIdx.x / C;
    const int64_t tid = int64_t(rank) * blockDim.x + threadIdx.x;
    const int64_t nthreads = int64_t(C) * blockDim.x;
    A* arena = reinterpret_cast<A*>(a.arena);
    for (int s = a.team_first[team]; s < a.team_first[team + 1]; ++s) {
        const BInst I = a.inst[a.sched[s]];
        A* psi = arena + I.psi_off;
        A* lam = arena + I.lam_off;
        const int64_t N = int64_t(1) << I.n;
        const double* th = a.theta + I.param_begin;
        double* part = a.partials + I.part_off;
        // scaled form: the stored states are the true ones / inv_s (thread 0
        // tracks it; the energy and every partial are multiplied by inv_s^2)
        double inv_s = 1.0;
        // |0...0>, or the state after the leading product layer directly
        for (int64_t i = tid; i < N; i += nthreads) {
            A v;
            if (I.init_tab >= 0) {
                v = product_amp<R>(reinterpret_cast<const A*>(a.init) + I.init_tab, I.n, i);
            } else {
                v.x = R(i == 0 ? 1 : 0);
                v.y = R(0);
            }
            psi[i] = v;
        }
        team_sync(C);
        // forward sweep
        for (int x = I.exec_fwd_begin; x < I.exec_end; ++x) {
            const int gi = a.exec[x];
            if (gi < 0) {  // a diagonal run: one pass with its phase table
                const PhaseRun& run = a.runs[-1 - gi];
                phase_tables_load<PR_TAB_WEIGHT>(a.ptabs + int64_t(-1 - gi) * 2 * PR_TAB_WEIGHT, 2 * run.n_rot + 1,
                                                 &ptab);
                double acc[1];
                phase_run_sweep<R, PR_WEIGHT, PR_TAB_WEIGHT, kTeamLoads<R>>(psi, nullptr, I.n, run, ptab, tid, nthreads,
                                                                         acc);
                team_sync(C);
                continue;
            }
            if constexpr (sizeof(R) == 4) {  // complex64: a tile of up to three rotations
                int tgs[kTeamTile];
                const int nq = team_tile(a, x, +1, I.exec_end, tgs);
                if (nq >= 2) {
                    if (threadIdx.x == 0)
                        for (int j = 0; j < nq; ++j) team_rotg<R>(a.gates[tgs[j]], th, false, &tg[j], &tq[j]);
                    __syncthreads();
                    double pv[kTeamTile];
                    if (nq == 3) team_rotq<R, 3>(psi, nullptr, I.n, tq, tg, tid, nthreads, pv);
                    else team_rotq<R, 2>(psi, nullptr, I.n, tq, tg, tid, nthreads, pv);
                    team_sync(C);
                    x += nq - 1;
                    continue;
                }
            }
            if (x + 1 < I.exec_end && pair_entries(a.gates, gi, a.exec[x + 1])) {  // a fused pair
                const BGate& ga = a.gates[gi];
                const BGate& gb = a.gates[a.exec[x + 1]];
                if (threadIdx.x == 0) {
                    team_rot1_coefs(ga, th, false, scaled, &pang[0], &inv_s);
                    team_rot1_coefs(gb, th, false, scaled, &pang[3], &inv_s);
                }
                __syncthreads();
                double pa, pb;
                if constexpr (sizeof(R) == 8) {
                    if (scaled) team_rot2<R, true>(psi, nullptr, I.n, ga, gb, &pang[0], &pang[3], tid, nthreads, &pa, &pb);
                    else team_rot2<R, false>(psi, nullptr, I.n, ga, gb, &pang[0], &pang[3], tid, nthreads, &pa, &pb);
                } else {
                    team_rot2<R, false>(psi, nullptr, I.n, ga, gb, &pang[0], &pang[3], tid, nthreads, &pa, &pb);
                }
                team_sync(C);
                ++x;
                continue;
            }
            const BGate& g = a.gates[gi];
            if (threadIdx.x == 0) {
                if (g.param >= 0) {
                    rot_angle(g, th, false, &ang[0], &ang[1], &ang[2]);
                    if (scaled) {
                        int m1;
                        double sg;
                        rot_scaled_coefs(ang[0], ang[1], ang[2], g.rot.ny, &m1, &sang[1], &sg);
                        sang[0] = m1;
                        inv_s *= sg;
                    }
                } else {
                    build_step<R>(g, th, false, &mats);
                }
            }
            __syncthreads();
            if (g.param >= 0) {
                if constexpr (sizeof(R) == 8) {
                    if (scaled) {
                        rot_dispatch_s<R>(g.k, g.xl, psi, nullptr, I.n, g.rot, sang[0] != 0.0, R(sang[1]), tid,
                                          nthreads);
                    } else {
                        rot_dispatch<R>(g.k, g.xl, psi, nullptr, I.n, g.rot, R(ang[0]), R(ang[1]), R(ang[2]), tid,
                                        nthreads);
                    }
                } else {
                    rot_dispatch<R>(g.k, g.xl, psi, nullptr, I.n, g.rot, R(ang[0]), R(ang[1]), R(ang[2]), tid,
                                    nthreads);
                }
            } else {
                team_fixed<R>(psi, nullptr, I.n, g, mats, tid, nthreads);
            }
            team_sync(C);
        }
        // lambda = H psi and the energy Re <psi|lambda>
        const double es = block_sum(lambda_share_any<R>(a.lflags, psi, lam, a.terms, reinterpret_cast<const A*>(a.ltab),
                                                        I.term_begin, I.term_end,
                                                        N, tid, nthreads),
                                    warps);
        if (threadIdx.x == 0) part[0 * C + rank] = scaled ? es * (inv_s * inv_s) : es;
        team_sync(C);
        // reverse sweep: partial Im <lam|P|psi>, then U^dag on psi and lam
        for (int x = I.exec_end - 1; x >= I.exec_rev_begin; --x) {
            const int gi = a.exec[x];
            if (gi < 0) {  // a diagonal run: its gradient sum, then D^dag on psi and lam
                const PhaseRun& run = a.runs[-1 - gi];
                phase_tables_load<PR_TAB_WEIGHT>(a.ptabs + (int64_t(-1 - gi) * 2 + 1) * PR_TAB_WEIGHT,
                                                 2 * run.n_rot + 1, &ptab);
                double acc[1];
                phase_run_sweep<R, PR_WEIGHT, PR_TAB_WEIGHT, kTeamLoads<R>>(psi, lam, I.n, run, ptab, tid, nthreads, acc);
                const double sum = block_sum(acc[0], warps);
                if (threadIdx.x == 0) {
                    part[int64_t(run.rot_slot[0]) * C + rank] = scaled ? sum * (inv_s * inv_s) : sum;
                    for (int g2 = 1; g2 < run.n_rot; ++g2) part[int64_t(run.rot_slot[g2]) * C + rank] = 0.0;
                }
                team_sync(C);
                continue;
            }
            if constexpr (sizeof(R) == 4) {
                int tgs[kTeamTile];
                const int nq = team_tile(a, x, -1, I.exec_rev_begin, tgs);
                if (nq >= 2) {
                    if (threadIdx.x == 0)
                        for (int j = 0; j < nq; ++j) team_rotg<R>(a.gates[tgs[j]], th, true, &tg[j], &tq[j]);
                    __syncthreads();
                    double pv[kTeamTile];
                    if (nq == 3) team_rotq<R, 3>(psi, lam, I.n, tq, tg, tid, nthreads, pv);
                    else team_rotq<R, 2>(psi, lam, I.n, tq, tg, tid, nthreads, pv);
                    for (int j = 0; j < nq; ++j) {
                        const double sj = block_sum(pv[j], warps);
                        if (threadIdx.x == 0) part[int64_t(a.gates[tgs[j]].slot) * C + rank] = sj;
                    }
                    team_sync(C);
                    x -= nq - 1;
                    continue;
                }
            }
            if (x - 1 >= I.exec_rev_begin && pair_entries(a.gates, a.exec[x - 1], gi)) {  // a fused pair (a, b)
                const BGate& ga = a.gates[a.exec[x - 1]];
                const BGate& gb = a.gates[gi];
                const double ps_b = inv_s * inv_s;  // b's partial is taken first, before b is undone
                if (threadIdx.x == 0) team_rot1_coefs(gb, th, true, scaled, &pang[3], &inv_s);
                const double ps_a = inv_s * inv_s;  // a's partial after b is undone
                if (threadIdx.x == 0) team_rot1_coefs(ga, th, true, scaled, &pang[0], &inv_s);
                __syncthreads();
                double pa, pb;
                if constexpr (sizeof(R) == 8) {
                    if (scaled) team_rot2<R, true>(psi, lam, I.n, ga, gb, &pang[0], &pang[3], tid, nthreads, &pa, &pb);
                    else team_rot2<R, false>(psi, lam, I.n, ga, gb, &pang[0], &pang[3], tid, nthreads, &pa, &pb);
                } else {
                    team_rot2<R, false>(psi, lam, I.n, ga, gb, &pang[0], &pang[3], tid, nthreads, &pa, &pb);
                }
                const double sa = block_sum(pa, warps);
                const double sb = block_sum(pb, warps);
                if (threadIdx.x == 0) {
                    part[int64_t(ga.slot) * C + rank] = scaled ? sa * ps_a : sa;
                    part[int64_t(gb.slot) * C + rank] = scaled ? sb * ps_b : sb;
                }
                team_sync(C);
                --x;
                continue;
            }
            const BGate& g = a.gates[gi];
            const double pscale = inv_s * inv_s;  // this step's partial is taken before U^dag
            if (threadIdx.x == 0) {
                if (g.param >= 0) {
                    rot_angle(g, th, true, &ang[0], &ang[1], &ang[2]);
                    if (scaled) {
                        int m1;
                        double sg;
                        rot_scaled_coefs(ang[0], ang[1], ang[2], g.rot.ny, &m1, &sang[1], &sg);
                        sang[0] = m1;
                        inv_s *= sg;
                    }
                } else {
                    build_step<R>(g, th, true, &mats);
                }
            }
            __syncthreads();
            double v = 0.0;
            if (g.param >= 0) {
                if constexpr (sizeof(R) == 8) {
                    if (scaled) {
                        v = rot_dispatch_s<R>(g.k, g.xl, psi, lam, I.n, g.rot, sang[0] != 0.0, R(sang[1]), tid,
                                              nthreads);
                    } else {
                        v = rot_dispatch<R>(g.k, g.xl, psi, lam, I.n, g.rot, R(ang[0]), R(ang[1]), R(ang[2]), tid,
                                            nthreads);
                    }
                } else {
                    v = rot_dispatch<R>(g.k, g.xl, psi, lam, I.n, g.rot, R(ang[0]), R(ang[1]), R(ang[2]), tid,
                                        nthreads);
                }
            } else {
                team_fixed<R>(psi, lam, I.n, g, mats, tid, nthreads);
            }
            if (g.slot >= 0) {
                const double sum = block_sum(v, warps);
                if (threadIdx.x == 0) part[int64_t(g.slot) * C + rank] = scaled ? sum * pscale : sum;
            }
            team_sync(C);
        }
    }
}

// Window-fused batch: the same team schedule and reductions as k_batch, but
// each team runs an instance's gates block by block (blocks of at most w
// qubits from the commutation-aware planner), staging every group of the
// window in shared memory, and meets at the cluster barrier once per block
// instead of once per gate. Block size WIN_THREADS.
template <typename R>
__device__ __forceinline__ void batch_stage(const WinBlock* __restrict__ blocks, int b, WinBlock* w,
                                            const WinGate* __restrict__ wg, const BGate* __restrict__ gates,
                                            const double* th, bool rev, WinOp<R>* ops, Acc<R>* sa) {
    const int T = blockDim.x, t = threadIdx.x;
    __syncthreads();  // the previous block's records are no longer in use
    {
        const int* src = reinterpret_cast<const int*>(blocks + b);
        int* dst = reinterpret_cast<int*>(w);
        for (int i = t; i < int(sizeof(WinBlock) / sizeof(int)); i += T) dst[i] = src[i];
    }
    __syncthreads();
    for (int i = t; i < w->count; i += T) {
        const WinGate x = wg[w->first + i];
        const BGate& G = gates[x.g];
        WinOp<R>& o = ops[i];
        o.k = G.k;
        o.b0 = x.b0;
        o.b1 = x.b1;
        o.j = G.param >= 0 ? x.j : -1;
        o.xl = G.xl;
        o.zl = G.rot.zl;
        o.ny = G.rot.ny;
        o.cs = R(0);
        o.kr = R(0);
        o.ki = R(0);
        const int Dk = 1 << G.k;
        if (G.param >= 0) {
            double cs, kr, ki;
            rot_angle(G, th, rev, &cs, &kr, &ki);
            o.cs = R(cs);
            o.kr = R(kr);
            o.ki = R(ki);
        } else {
            for (int r = 0; r < Dk; ++r)
                for (int c = 0; c < Dk; ++c) {
                    const double vr = rev ? G.re[c * Dk + r] : G.re[r * Dk + c];
                    const double vi = rev ? -G.im[c * Dk + r] : G.im[r * Dk + c];
                    o.mre[r * Dk + c] = R(vr);
                    o.mim[r * Dk + c] = R(vi);
                    o.ty[r * Dk + c] = dev_entry_type(double(R(vr)), double(R(vi)));
                }
        }
    }
    if (rev)
        for (int j = 0; j < w->np; ++j) sa[j * T + t] = Acc<R>();
    __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(WIN_THREADS) k_batch_win(const BatchArgs a, const WinBlock* __restrict__ blocks,
                                                           const WinGate* __restrict__ wg, int window) {
    using A = amp_t<R>;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double warps[32];
    __shared__ __align__(16) WinBlock w;
    const int T = WIN_THREADS, t = threadIdx.x;
    const int C = a.C;
    const int rank = C == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const int team = blockIdx.x / C;
    const int64_t tid = int64_t(rank) * T + t;
    const int64_t nthreads = int64_t(C) * T;
    const int Dmax = 1 << window;
    WinOp<R>* ops = reinterpret_cast<WinOp<R>*>(sm);
    A* sp = reinterpret_cast<A*>(sm + ((sizeof(WinOp<R>) * WIN_MAXG + 15) / 16) * 16);
    A* sl = sp + Dmax * T;
    Acc<R>* sa = reinterpret_cast<Acc<R>*>(sl + Dmax * T);
    A* cp = sp + t;
    A* cl = sl + t;
    A* arena = reinterpret_cast<A*>(a.arena);
    for (int s = a.team_first[team]; s < a.team_first[team + 1]; ++s) {
        const BInst I = a.inst[a.sched[s]];
        A* psi = arena + I.psi_off;
        A* lam = arena + I.lam_off;
        const int64_t N = int64_t(1) << I.n;
        const double* th = a.theta + I.param_begin;
        double* part = a.partials + I.part_off;
        for (int64_t i = tid; i < N; i += nthreads) {
            A v;
            v.x = R(i == 0 ? 1 : 0);
            v.y = R(0);
            psi[i] = v;
        }
        team_sync(C);
        // forward sweep, block by block
        for (int b = I.block_begin; b < I.block_end; ++b) {
            batch_stage<R>(blocks, b, &w, wg, a.gates, th, false, ops, sa);
            const int D = 1 << w.nq;
            const int64_t G = int64_t(1) << (I.n - w.nq);
            for (int64_t g = tid; g < G; g += nthreads) {
                const int64_t base = insert_zeros_rt(g, w.q, w.nq);
                const bool ok = DIAQ_BOUNDS_OK(base + w.off[D - 1], N, BS_WINDOW);
                if (ok)
                    for (int e = 0; e < D; ++e) cp[e * T] = psi[base + w.off[e]];
                for (int i = 0; i < w.count; ++i) win_apply<R>(ops[i], cp, nullptr, D, T, nullptr);
                if (ok)
                    for (int e = 0; e < D; ++e) psi[base + w.off[e]] = cp[e * T];
            }
            team_sync(C);
        }
        // lambda = H psi and the energy Re <psi|lambda>
        Acc<R> e;
        for (int64_t i = tid; i < N; i += nthreads) {
            const A o = pauli_lambda_elem<R>(psi, a.terms, reinterpret_cast<const A*>(a.ltab), I.term_begin, I.term_end, i);
            lam[i] = o;
            const A pi = psi[i];
            e.add_dot(pi.x, o.x, pi.y, o.y);
        }
        const double es = block_sum(e.value(), warps);
        if (t == 0) part[0 * C + rank] = es;
        team_sync(C);
        // reverse sweep: blocks in reverse, gates in reverse within a block
        for (int b = I.block_end - 1; b >= I.block_begin; --b) {
            batch_stage<R>(blocks, b, &w, wg, a.gates, th, true, ops, sa);
            const int D = 1 << w.nq;
            const int64_t G = int64_t(1) << (I.n - w.nq);
            for (int64_t g = tid; g < G; g += nthreads) {
                const int64_t base = insert_zeros_rt(g, w.q, w.nq);
                const bool ok = DIAQ_BOUNDS_OK(base + w.off[D - 1], N, BS_WINDOW);
                if (ok)
                    for (int e2 = 0; e2 < D; ++e2) cp[e2 * T] = psi[base + w.off[e2]];
                if (ok)
                    for (int e2 = 0; e2 < D; ++e2) cl[e2 * T] = lam[base + w.off[e2]];
                for (int i = w.count - 1; i >= 0; --i) {
                    const WinOp<R>& o = ops[i];
                    win_apply<R>(o, cp, cl, D, T, o.j >= 0 ? sa + o.j * T + t : nullptr);
                }
                if (ok)
                    for (int e2 = 0; e2 < D; ++e2) psi[base + w.off[e2]] = cp[e2 * T];
                if (ok)
                    for (int e2 = 0; e2 < D; ++e2) lam[base + w.off[e2]] = cl[e2 * T];
            }
            for (int j = 0; j < w.np; ++j) {
                const double v = block_sum(sa[j * T + t].value(), warps);
                if (t == 0) part[int64_t(w.slot[j]) * C + rank] = v;
            }
            team_sync(C);
        }
    }
}

// Dynamic shared memory of k_batch_win for a window of w qubits.
static size_t batch_win_smem(diaq_dtype dt, int w) {
    const size_t opb = dt == DIAQ_C128 ? sizeof(WinOp<double>) : sizeof(WinOp<float>);
    return ((opb * WIN_MAXG + 15) / 16) * 16 + 2 * (size_t(1) << w) * WIN_THREADS * amp_bytes(dt) +
           size_t(WIN_MAXG) * WIN_THREADS * sizeof(double);
}

// Four-lane form of k_batch_win: WIN_LANES threads of a warp share each
// group (subspaces split gate by gate, __syncwarp between gates), groups
// stored contiguously with one padding amplitude. Every thread of a block
// makes the same number of trips over the groups, so every lane reaches
// each __syncwarp.
template <typename R>
__global__ void __launch_bounds__(WIN_THREADS, 4) k_batch_win_l(const BatchArgs a, const WinBlock* __restrict__ blocks,
                                                                const WinGate* __restrict__ wg, int window) {
    using A = amp_t<R>;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double warps[32];
    __shared__ __align__(16) WinBlock w;
    constexpr int L = WIN_LANES;
    const int T = WIN_THREADS, t = threadIdx.x;
    const int GPC = T / L, gs = t / L, li = t % L;
    const int C = a.C;
    const int rank = C == 1 ? 0 : (int)cg::this_cluster().block_rank();
    const int team = blockIdx.x / C;
    const int64_t tid = int64_t(rank) * T + t;
    const int64_t nthreads = int64_t(C) * T;
    const int SDmax = (1 << window) + 1;
    WinOp<R>* ops = reinterpret_cast<WinOp<R>*>(sm);
    A* sp = reinterpret_cast<A*>(sm + ((sizeof(WinOp<R>) * WIN_MAXG + 15) / 16) * 16);
    A* sl = sp + GPC * SDmax;
    Acc<R>* sa = reinterpret_cast<Acc<R>*>(sl + GPC * SDmax);
    A* arena = reinterpret_cast<A*>(a.arena);
    for (int s = a.team_first[team]; s < a.team_first[team + 1]; ++s) {
        const BInst I = a.inst[a.sched[s]];
        A* psi = arena + I.psi_off;
        A* lam = arena + I.lam_off;
        const int64_t N = int64_t(1) << I.n;
        const double* th = a.theta + I.param_begin;
        double* part = a.partials + I.part_off;
        for (int64_t i = tid; i < N; i += nthreads) {
            A v;
            v.x = R(i == 0 ? 1 : 0);
            v.y = R(0);
            psi[i] = v;
        }
        team_sync(C);
        for (int dir = 0; dir < 2; ++dir) {
            const bool rev = dir == 1;
            if (rev) {
                // lambda = H psi and the energy Re <psi|lambda>
                Acc<R> e;
                for (int64_t i = tid; i < N; i += nthreads) {
                    const A o = pauli_lambda_elem<R>(psi, a.terms, reinterpret_cast<const A*>(a.ltab), I.term_begin, I.term_end, i);
                    lam[i] = o;
                    const A pi = psi[i];
                    e.add_dot(pi.x, o.x, pi.y, o.y);
                }
                const double es = block_sum(e.value(), warps);
                if (t == 0) part[0 * C + rank] = es;
                team_sync(C);
            }
            const int nb = I.block_end - I.block_begin;
            for (int bi = 0; bi < nb; ++bi) {
                const int b = rev ? I.block_end - 1 - bi : I.block_begin + bi;
                batch_stage<R>(blocks, b, &w, wg, a.gates, th, rev, ops, sa);
                const int D = 1 << w.nq, SD = D + 1;
                const int64_t G = int64_t(1) << (I.n - w.nq);
                A* gp = sp + gs * SD;
                A* gl = sl + gs * SD;
                for (int64_t g0 = int64_t(rank) * GPC; g0 < G; g0 += int64_t(C) * GPC) {
                    const int64_t g = g0 + gs;
                    const int64_t base = g < G ? insert_zeros_rt(g, w.q, w.nq) : 0;
                    const bool valid = g < G && DIAQ_BOUNDS_OK(base + w.off[D - 1], int64_t(1) << I.n, BS_WINDOW);
                    if (valid) {
                        for (int e2 = li; e2 < D; e2 += L) gp[e2] = psi[base + w.off[e2]];
                        if (rev)
                            for (int e2 = li; e2 < D; e2 += L) gl[e2] = lam[base + w.off[e2]];
                    }
                    __syncwarp();
                    if (!rev) {
                        for (int i = 0; i < w.count; ++i) {
                            win_apply<R, 1>(ops[i], gp, nullptr, D, 1, nullptr, li, L);
                            __syncwarp();
                        }
                    } else {
                        for (int i = w.count - 1; i >= 0; --i) {
                            const WinOp<R>& o = ops[i];
                            win_apply<R, 1>(o, gp, gl, D, 1, (valid && o.j >= 0) ? sa + o.j * T + t : nullptr, li, L);
                            __syncwarp();
                        }
                    }
                    if (valid) {
                        for (int e2 = li; e2 < D; e2 += L) psi[base + w.off[e2]] = gp[e2];
                        if (rev)
                            for (int e2 = li; e2 < D; e2 += L) lam[base + w.off[e2]] = gl[e2];
                    }
                    __syncwarp();
                }
                if (rev) {
                    for (int j = 0; j < w.np; ++j) {
                        const double v = block_sum(sa[j * T + t].value(), warps);
                        if (t == 0) part[int64_t(w.slot[j]) * C + rank] = v;
                    }
                }
                team_sync(C);
            }
        }
    }
}

static size_t batch_win_smem_lanes(diaq_dtype dt, int w) {
    const size_t opb = dt == DIAQ_C128 ? sizeof(WinOp<double>) : sizeof(WinOp<float>);
    const size_t gpc = WIN_THREADS / WIN_LANES;
    return ((opb * WIN_MAXG + 15) / 16) * 16 + 2 * gpc * ((size_t(1) << w) + 1) * amp_bytes(dt) +
           size_t(WIN_MAXG) * WIN_THREADS * sizeof(double);
}

// Per instance: energy and gradient from the partial rows, fixed order.
__global__ void k_batch_finish(const BInst* inst, const BGate* gates, const double* partials, int C, int n_inst,
                               double* energy, double* grad) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_inst) return;
    const BInst I = inst[id];
    const double* part = partials + I.part_off;
    double e = 0.0;
    for (int r = 0; r < C; ++r) e += part[r];
    energy[id] = e;
    double* g = grad + I.param_begin;
    for (int p = 0; p < I.n_params; ++p) g[p] = 0.0;
    for (int gi = I.gate_begin; gi < I.gate_end; ++gi) {
        const BGate& G = gates[gi];
        if (G.slot < 0) continue;
        double v = 0.0;
        for (int r = 0; r < C; ++r) v += part[int64_t(G.slot) * C + r];
        g[G.param] += G.scale * v;
    }
}

}  // namespace diaq

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
using namespace diaq;

struct diaq_batch_s {
    int device = 0;
    diaq_dtype dtype = DIAQ_C128;
    int n_inst = 0;
    int n_params_total = 0;
    std::vector<BInst> inst;
    std::vector<BGate> gates;
    std::vector<BTerm> terms;
    std::vector<double> work;  // per-instance work estimate (amplitude-gates)
    int64_t arena_elems = 0;
    int64_t slots_total = 0;   // sum of n_slots
    // device
    BInst* d_inst = nullptr;
    BGate* d_gates = nullptr;
    BTerm* d_terms = nullptr;
    std::vector<double2> ltab;   // lambda weight tables (lambda_tables)
    void* d_ltab = nullptr;      // in the batch's precision
    int lflags = LAM_REAL | LAM_COUNT;  // what holds for every instance
    void* d_arena = nullptr;
    double* d_theta = nullptr;
    double* d_partials = nullptr;
    double* d_out = nullptr;   // energies then grads
    int32_t* d_sched = nullptr;
    int32_t* d_team_first = nullptr;
    // pinned staging for graph replay
    double* h_theta = nullptr;
    double* h_out = nullptr;
    // launch configuration and its graph
    int C = 1, threads = 256, teams = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    // window-fused kernel (window > 0): blocks of every instance
    int window = 0;
    int lanes = 1;  // threads per group of the window-fused kernel (1 or WIN_LANES)
    WinBlock* d_blocks = nullptr;
    WinGate* d_wg = nullptr;
    // execution lists of the per-gate kernel, with or without diagonal runs
    bool runs_on = true;
    int n_runs = 0;
    std::vector<int32_t> exec_list;
    std::vector<PhaseRun> runs;
    int32_t* d_exec = nullptr;
    PhaseRun* d_runs = nullptr;
    double2* d_ptabs = nullptr;  // phase tables of the runs (k_phase_tables)
    std::vector<double2> init_tabs;  // product-layer tables of the instances (product_layer)
    void* d_init = nullptr;      // in the batch's precision
    // scaled rotations of the per-gate complex128 kernel: requested (default
    // on) and possible (every instance within the rotation bound)
    bool scaled = true;
    bool scaled_ok = false;
};


// Rotation shape of a parametric gate from its generator letters.
static void fill_rot(BGate* B) {
    const int k = B->k;
    B->xl = 0;
    B->rot.zl = 0;
    B->rot.ny = 0;
    for (int a = 0; a < k; ++a) {
        const int bit = 1 << (k - 1 - a);
        const int L = B->pauli[a];  // 0 I, 1 X, 2 Y, 3 Z
        if (L == 1 || L == 2) B->xl |= bit;
        if (L == 2 || L == 3) B->rot.zl |= bit;
        if (L == 2) B->rot.ny = (B->rot.ny + 1) & 3;
    }
    B->rot.st[0] = k == 2 ? std::min(B->t[0], B->t[1]) : B->t[0];
    B->rot.st[1] = k == 2 ? std::max(B->t[0], B->t[1]) : 0;
    for (int c = 0; c < 4; ++c) {
        int64_t o = 0;
        if (c < (1 << k))
            for (int a = 0; a < k; ++a)
                if ((c >> (k - 1 - a)) & 1) o += int64_t(1) << B->t[a];
        B->rot.off[c] = o;
    }
}

// Diagonal runs (phase.cuh) of one circuit's gates [0, n_gates): Z-type
// rotations (generators of I and Z letters), fixed single-qubit diagonal
// gates and CZs gather into a run; a gate of any other kind that acts on
// none of the run's qubits moves ahead of it (it commutes with every
// member), one that shares a qubit closes the run. A run of at least two
// gates that fits the weight form (one shared parameter and scale, no fixed
// gate) or, with chunks_ok, the chunk form (single-qubit rotations) becomes
// one step; any other run is executed gate by gate in its order. exec
// receives the execution order: gate_base + gate index, or -1 - run index
// (runs appended to *runs).
static void plan_phase_runs(const BGate* gates, int n_gates, int gate_base, bool chunks_ok, std::vector<int32_t>* exec,
                            std::vector<PhaseRun>* runs) {
    auto zrot = [](const BGate& g, uint64_t* z) {
        if (g.param < 0) return false;
        uint64_t m = 0;
        for (int a = 0; a < g.k; ++a) {
            if (g.pauli[a] != 0 && g.pauli[a] != 3) return false;
            if (g.pauli[a] == 3) m |= uint64_t(1) << g.t[a];
        }
        *z = m;
        return true;
    };
    auto fix1 = [](const BGate& g) {
        return g.param < 0 && g.k == 1 && g.re[1] == 0.0 && g.im[1] == 0.0 && g.re[2] == 0.0 && g.im[2] == 0.0;
    };
    auto cz = [](const BGate& g) {
        if (g.param >= 0 || g.k != 2) return false;
        for (int e = 0; e < 16; ++e) {
            const double want = (e == 0 || e == 5 || e == 10) ? 1.0 : (e == 15 ? -1.0 : 0.0);
            if (g.re[e] != want || g.im[e] != 0.0) return false;
        }
        return true;
    };
    std::vector<int> members;
    uint64_t run_q = 0;
    auto flush = [&]() {
        if (members.empty()) return;
        PhaseRun r = {};
        bool weight = members.size() >= 2 && int(members.size()) <= PR_MAX_ROT;
        bool chunk = chunks_ok && members.size() >= 2;
        int nr = 0;
        for (int i : members) {
            const BGate& g = gates[i];
            uint64_t z = 0;
            if (zrot(g, &z)) {
                const BGate& f = gates[members[0]];
                weight &= g.param == f.param && g.scale == f.scale && f.param >= 0;
                chunk &= __builtin_popcountll(z) == 1 && nr < PR_MAX_CROT;
                if (nr < PR_MAX_ROT) {
                    r.rot_param[nr] = g.param;
                    r.rot_scale[nr] = g.scale;
                    r.rot_z[nr] = z;
                    r.rot_slot[nr] = g.slot;
                }
                ++nr;
            } else if (fix1(g)) {
                weight = false;
                if (r.n_fix1 >= PR_MAX_FIX1) {
                    chunk = false;
                    continue;
                }
                r.fix1_q[r.n_fix1] = g.t[0];
                r.fix1_re[2 * r.n_fix1] = g.re[0];
                r.fix1_im[2 * r.n_fix1] = g.im[0];
                r.fix1_re[2 * r.n_fix1 + 1] = g.re[3];
                r.fix1_im[2 * r.n_fix1 + 1] = g.im[3];
                ++r.n_fix1;
            } else {  // a CZ
                weight = false;
                if (r.n_cz >= PR_MAX_CZ) {
                    chunk = false;
                    continue;
                }
                r.cz[r.n_cz++] = (uint64_t(1) << g.t[0]) | (uint64_t(1) << g.t[1]);
            }
        }
        r.n_rot = nr;
        weight &= nr >= 2;
        if (weight || chunk) {
            r.kind = weight ? PR_WEIGHT : PR_CHUNKS;
            // CZs inside one chunk of PR_CHUNK_BITS qubits first: their signs
            // go into that chunk's table, the others are tested per row
            std::stable_partition(r.cz, r.cz + r.n_cz, [](uint64_t m) {
                const int lo = __builtin_ctzll(m), hi = 63 - __builtin_clzll(m);
                return lo / PR_CHUNK_BITS == hi / PR_CHUNK_BITS;
            });
            r.n_cz_in = 0;
            for (int k = 0; k < r.n_cz; ++k) {
                const int lo = __builtin_ctzll(r.cz[k]), hi = 63 - __builtin_clzll(r.cz[k]);
                if (lo / PR_CHUNK_BITS == hi / PR_CHUNK_BITS) ++r.n_cz_in;
            }
            if (weight) phase_run_classes(&r);
            exec->push_back(-1 - int32_t(runs->size()));
            runs->push_back(r);
        } else {
            for (int i : members) exec->push_back(gate_base + i);
        }
        members.clear();
        run_q = 0;
    };
    for (int i = 0; i < n_gates; ++i) {
        const BGate& g = gates[i];
        uint64_t q = uint64_t(1) << g.t[0];
        if (g.k == 2) q |= uint64_t(1) << g.t[1];
        uint64_t z = 0;
        if (zrot(g, &z) || fix1(g) || cz(g)) {
            members.push_back(i);
            run_q |= q;
        } else if (members.empty() || !(q & run_q)) {
            exec->push_back(gate_base + i);
        } else {
            flush();
            exec->push_back(gate_base + i);
        }
    }
    flush();
}

// Window blocks of at most `window` qubits and WIN_MAXG gates for the gates
// [0, n_gates) of one circuit, from the commutation-aware planner (a gate
// moves only past gates on disjoint qubits). Appends the blocks and their
// gate entries; WinGate::g is gate_base + the gate's index, first is
// relative to the whole entry list.
static diaq_status make_windows(const BGate* gates, int n_gates, int gate_base, int window,
                                std::vector<WinBlock>* blocks, std::vector<WinGate>* wg) {
    if (n_gates == 0) return DIAQ_OK;
    std::vector<diaq_gate> g(static_cast<size_t>(n_gates));
    for (int i = 0; i < n_gates; ++i) {
        std::memset(&g[size_t(i)], 0, sizeof(diaq_gate));
        g[size_t(i)].k = gates[i].k;
        g[size_t(i)].targets[0] = gates[i].t[0];
        g[size_t(i)].targets[1] = gates[i].t[1];
        g[size_t(i)].param = -1;
    }
    std::vector<int32_t> order(static_cast<size_t>(n_gates)), grp(static_cast<size_t>(n_gates));
    int32_t ng = 0;
    DIAQ_TRY(diaq_plan_fusion_commuting(g.data(), n_gates, window, WIN_MAXG, order.data(), grp.data(), &ng));
    for (int pos = 0; pos < n_gates;) {
        int end = pos;
        while (end < n_gates && grp[size_t(end)] == grp[size_t(pos)]) ++end;
        WinBlock w;
        std::memset(&w, 0, sizeof(w));
        std::vector<int> qs;
        for (int i = pos; i < end; ++i) {
            const BGate& G = gates[order[size_t(i)]];
            for (int a = 0; a < G.k; ++a)
                if (std::find(qs.begin(), qs.end(), G.t[a]) == qs.end()) qs.push_back(G.t[a]);
        }
        std::sort(qs.begin(), qs.end());
        if (int(qs.size()) > WIN_MAX || end - pos > WIN_MAXG)
            return fail(DIAQ_ERR_UNSUPPORTED, "a fused block exceeds %d qubits or %d gates", WIN_MAX, WIN_MAXG);
        w.nq = int(qs.size());
        for (int a = 0; a < w.nq; ++a) w.q[a] = qs[size_t(a)];
        for (int e = 0; e < (1 << w.nq); ++e) {
            int64_t o = 0;
            for (int a = 0; a < w.nq; ++a)
                if ((e >> a) & 1) o += int64_t(1) << w.q[a];
            w.off[e] = o;
        }
        w.first = int(wg->size());
        w.count = end - pos;
        for (int i = pos; i < end; ++i) {
            const int gi = order[size_t(i)];
            const BGate& G = gates[gi];
            WinGate x;
            x.g = gate_base + gi;
            x.b0 = int(std::find(qs.begin(), qs.end(), G.t[0]) - qs.begin());
            x.b1 = G.k == 2 ? int(std::find(qs.begin(), qs.end(), G.t[1]) - qs.begin()) : 0;
            x.j = -1;
            if (G.param >= 0) {
                x.j = w.np;
                w.slot[w.np++] = G.slot;
            }
            wg->push_back(x);
        }
        blocks->push_back(w);
        pos = end;
    }
    return DIAQ_OK;
}

static void batch_free(diaq_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->d_blocks) cudaFree(b->d_blocks);
    if (b->d_wg) cudaFree(b->d_wg);
    if (b->d_exec) cudaFree(b->d_exec);
    if (b->d_runs) cudaFree(b->d_runs);
    if (b->d_ptabs) cudaFree(b->d_ptabs);
    if (b->d_init) cudaFree(b->d_init);
    for (void* p : {static_cast<void*>(b->d_inst), static_cast<void*>(b->d_gates), static_cast<void*>(b->d_terms),
                    static_cast<void*>(b->d_ltab),
                    b->d_arena, static_cast<void*>(b->d_theta), static_cast<void*>(b->d_partials),
                    static_cast<void*>(b->d_out), static_cast<void*>(b->d_sched), static_cast<void*>(b->d_team_first)})
        if (p) cudaFree(p);
    if (b->h_theta) cudaFreeHost(b->h_theta);
    if (b->h_out) cudaFreeHost(b->h_out);
}

template <typename T>
static diaq_status upload(T** d, const std::vector<T>& h) {
    const size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d), bytes);
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMalloc(%zu) for batch tables: %s", bytes, cudaGetErrorString(e));
    if (!h.empty()) DIAQ_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return DIAQ_OK;
}

// A table of complex values uploaded in the state's precision (float2 for
// complex64), so kernels read it without a conversion per amplitude.
static diaq_status upload_amps(diaq_dtype dt, const std::vector<double2>& h, void** d) {
    if (dt == DIAQ_C128) return upload(reinterpret_cast<double2**>(d), h);
    std::vector<float2> f(h.size());
    for (size_t i = 0; i < h.size(); ++i) f[i] = make_float2(float(h[i].x), float(h[i].y));
    return upload(reinterpret_cast<float2**>(d), f);
}

// The leading product layer of an execution list: the longest prefix of
// fixed one-qubit gates on distinct qubits. Applied to |0...0> they give a
// product state, amplitude i = prod_q u_q[bit q of i][0] (1 or 0 for the
// qubits outside the layer), which the kernels write directly from one
// table of 256 entries per chunk of 8 qubits (the product of that chunk's
// factors for each byte value) instead of running the layer gate by gate.
// Appends the tables to *tab and returns the layer's length (0: none).
static int product_layer(const BGate* gates, const int32_t* exec, int count, int n, std::vector<double2>* tab) {
    std::vector<int> gate_of(size_t(n), -1);
    int len = 0;
    for (; len < count; ++len) {
        const int32_t e = exec[len];
        if (e < 0) break;
        const BGate& g = gates[e];
        if (g.param >= 0 || g.k != 1 || gate_of[size_t(g.t[0])] >= 0) break;
        gate_of[size_t(g.t[0])] = e;
    }
    if (len == 0) return 0;
    const int chunks = (n + 7) / 8;
    for (int c = 0; c < chunks; ++c)
        for (int v = 0; v < 256; ++v) {
            cplx f(1.0, 0.0);
            for (int b = 0; b < 8; ++b) {
                const int q = 8 * c + b;
                const int bit = (v >> b) & 1;
                if (q >= n) {
                    if (bit) f = cplx(0.0, 0.0);
                    continue;
                }
                if (gate_of[size_t(q)] < 0) {
                    if (bit) f = cplx(0.0, 0.0);
                } else {
                    const BGate& g = gates[gate_of[size_t(q)]];
                    f *= cplx(g.re[2 * bit], g.im[2 * bit]);  // u[bit][0]: column 0, the image of |0>
                }
            }
            tab->push_back(make_double2(f.real(), f.imag()));
        }
    return len;
}

// Group headers and weight tables for the terms [t0, t1) of one observable
// (sorted by X mask; see pauli_lambda_elem), tables appended to *tab.
static int lambda_tables(std::vector<BTerm>& terms, int t0, int t1, std::vector<double2>* tab) {
    int fl = LAM_REAL | LAM_COUNT;
    for (int t = t0; t < t1;) {
        int u = t;
        while (u < t1 && terms[size_t(u)].x == terms[size_t(t)].x) ++u;
        const int gn = u - t;
        bool equal = true, real = true;
        for (int v = t; v < u; ++v) {
            equal &= terms[size_t(v)].kr == terms[size_t(t)].kr && terms[size_t(v)].ki == terms[size_t(t)].ki;
            real &= terms[size_t(v)].ki == 0.0;
        }
        int16_t gk[8] = {};
        const bool cls = equal && gn >= kLamClassMin;
        if (cls) {  // count form: the order within the group is free, so group the terms by class
            std::stable_sort(terms.begin() + t, terms.begin() + u,
                             [](const BTerm& a, const BTerm& b) { return ((a.z >> 5) & 7) < ((b.z >> 5) & 7); });
            for (int v = t; v < u; ++v) ++gk[(terms[size_t(v)].z >> 5) & 7];
        }
        BTerm& h = terms[size_t(t)];
        h.gn = gn;
        h.gtab = int32_t(tab->size());
        h.greal = real ? 1 : 0;
        h.gcls = cls ? 1 : 0;
        for (int k = 0; k < 8; ++k) h.gk[k] = gk[k];
        if (!real) fl &= ~LAM_REAL;
        if (!equal) fl &= ~LAM_COUNT;
        if (equal) {  // W = (gn - 2 m) kappa, m terms of odd parity
            h.gmode = 0;
            for (int m = 0; m <= gn; ++m) tab->push_back(make_double2(double(gn - 2 * m) * h.kr, double(gn - 2 * m) * h.ki));
        } else {  // per chunk of 8 terms: the signed sum for each parity pattern
            h.gmode = 1;
            for (int c = 0; 8 * c < gn; ++c) {
                const int len = std::min(8, gn - 8 * c);
                for (int bits = 0; bits < 256; ++bits) {
                    double wr = 0.0, wi = 0.0;
                    if (bits < (1 << len))
                        for (int e = 0; e < len; ++e) {
                            const BTerm& q = terms[size_t(t + 8 * c + e)];
                            const bool neg = (bits >> e) & 1;
                            wr += neg ? -q.kr : q.kr;
                            wi += neg ? -q.ki : q.ki;
                        }
                    tab->push_back(make_double2(wr, wi));
                }
            }
        }
        t = u;
    }
    return fl;
}

// The per-gate kernel's execution list of every instance (gates, or weight
// form diagonal runs when runs_on), instance ranges in inst, uploaded with
// the instance records.
static diaq_status batch_exec(diaq_batch_s* b) {
    b->exec_list.clear();
    b->runs.clear();
    b->init_tabs.clear();
    int first_run = 0;
    for (BInst& I : b->inst) {
        I.exec_begin = int32_t(b->exec_list.size());
        if (b->runs_on) {
            plan_phase_runs(b->gates.data() + I.gate_begin, I.gate_end - I.gate_begin, I.gate_begin, false, &b->exec_list,
                            &b->runs);
        } else {
            for (int g = I.gate_begin; g < I.gate_end; ++g) b->exec_list.push_back(g);
        }
        for (size_t r = size_t(first_run); r < b->runs.size(); ++r) b->runs[r].param_base = I.param_begin;
        first_run = int(b->runs.size());
        I.exec_end = int32_t(b->exec_list.size());
        {
            const int off = int(b->init_tabs.size());
            const int len = product_layer(b->gates.data(), b->exec_list.data() + I.exec_begin,
                                          I.exec_end - I.exec_begin, I.n, &b->init_tabs);
            I.init_tab = len > 0 ? off : -1;
            I.exec_fwd_begin = I.exec_begin + len;
        }
        // nothing below the earliest parametric entry feeds a gradient term
        I.exec_rev_begin = I.exec_end;
        for (int x = I.exec_begin; x < I.exec_end; ++x) {
            const int32_t e = b->exec_list[size_t(x)];
            if (e < 0 || b->gates[size_t(e)].param >= 0) {
                I.exec_rev_begin = x;
                break;
            }
        }
    }
    b->n_runs = int(b->runs.size());
    for (void* q : {static_cast<void*>(b->d_exec), static_cast<void*>(b->d_runs), static_cast<void*>(b->d_inst),
                    static_cast<void*>(b->d_ptabs), static_cast<void*>(b->d_init)})
        if (q) cudaFree(q);
    b->d_exec = nullptr;
    b->d_runs = nullptr;
    b->d_inst = nullptr;
    b->d_ptabs = nullptr;
    b->d_init = nullptr;
    if (b->exec_list.empty()) b->exec_list.push_back(0);
    DIAQ_TRY(upload(&b->d_exec, b->exec_list));
    DIAQ_TRY(upload_amps(b->dtype, b->init_tabs, &b->d_init));
    if (!b->runs.empty()) {
        DIAQ_TRY(upload(&b->d_runs, b->runs));
        const size_t bytes = b->runs.size() * 2 * PR_TAB_WEIGHT * sizeof(double2);
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->d_ptabs), bytes);
        if (e != cudaSuccess) {
            b->d_ptabs = nullptr;
            return fail(DIAQ_ERR_ALLOC, "cudaMalloc(%zu) for batch phase tables: %s", bytes, cudaGetErrorString(e));
        }
    }
    return upload(&b->d_inst, b->inst);
}

template <typename R>
static const void* batch_kernel() {
    return reinterpret_cast<const void*>(&k_batch<R>);
}

template <typename R>
static const void* batch_win_kernel(int lanes) {
    return lanes > 1 ? reinterpret_cast<const void*>(&k_batch_win_l<R>) : reinterpret_cast<const void*>(&k_batch_win<R>);
}

// Teams that fit on the GPU at once for cluster size C and block size T.
static diaq_status resident_teams(diaq_batch_s* b, int C, int T, int* teams) {
    const bool win = b->window > 0;
    const void* fn = win ? (b->dtype == DIAQ_C128 ? batch_win_kernel<double>(b->lanes) : batch_win_kernel<float>(b->lanes))
                         : (b->dtype == DIAQ_C128 ? batch_kernel<double>() : batch_kernel<float>());
    const size_t smem = !win ? 0 : (b->lanes > 1 ? batch_win_smem_lanes(b->dtype, b->window)
                                                 : batch_win_smem(b->dtype, b->window));
    if (win) DIAQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    if (C == 1) {
        int per_sm = 0, sms = 0;
        DIAQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, smem));
        DIAQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
        *teams = per_sm * sms;
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(T, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        DIAQ_CUDA(cudaOccupancyMaxActiveClusters(&n, fn, &cfg));
        *teams = n;
    }
    if (*teams < 1) return fail(DIAQ_ERR_UNSUPPORTED, "no team of %d blocks x %d threads fits on the device", C, T);
    return DIAQ_OK;
}

// Largest first, round robin over teams; balanced by a greedy least-loaded pick.
static void make_schedule(const diaq_batch_s* b, int teams, std::vector<int32_t>* sched, std::vector<int32_t>* first) {
    std::vector<int> order(static_cast<size_t>(b->n_inst));
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->work[size_t(x)] > b->work[size_t(y)]; });
    std::vector<std::vector<int32_t>> lists(static_cast<size_t>(teams));
    std::vector<double> load(size_t(teams), 0.0);
    for (int id : order) {
        size_t best = 0;
        for (size_t t = 1; t < load.size(); ++t)
            if (load[t] < load[best]) best = t;
        lists[best].push_back(id);
        load[best] += b->work[size_t(id)];
    }
    sched->clear();
    first->clear();
    for (auto& l : lists) {
        first->push_back(int32_t(sched->size()));
        sched->insert(sched->end(), l.begin(), l.end());
    }
    first->push_back(int32_t(sched->size()));
}

static bool batch_scaled_active(const diaq_batch_s* b) {
    return b->scaled && b->scaled_ok && b->dtype == DIAQ_C128 && b->window == 0;
}

static diaq_status launch_batch(diaq_batch_s* b, cudaStream_t s) {
    BatchArgs a;
    a.inst = b->d_inst;
    a.gates = b->d_gates;
    a.exec = b->d_exec;
    a.runs = b->d_runs;
    a.ptabs = b->d_ptabs;
    a.init = b->d_init;
    a.terms = b->d_terms;
    a.ltab = b->d_ltab;
    a.lflags = b->lflags;
    a.sched = b->d_sched;
    a.team_first = b->d_team_first;
    a.theta = b->d_theta;
    a.arena = b->d_arena;
    a.partials = b->d_partials;
    a.C = b->C;
    a.scaled = batch_scaled_active(b) ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(b->teams * b->C), 1, 1);
    cfg.blockDim = dim3(unsigned(b->threads), 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = unsigned(b->C);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = b->C > 1 ? 1 : 0;
    if (b->window > 0 && b->lanes > 1) {
        cfg.dynamicSmemBytes = batch_win_smem_lanes(b->dtype, b->window);
        const WinBlock* blk = b->d_blocks;
        const WinGate* wg = b->d_wg;
        if (b->dtype == DIAQ_C128)
            DIAQ_CUDA(cudaLaunchKernelEx(&cfg, k_batch_win_l<double>, a, blk, wg, b->window));
        else
            DIAQ_CUDA(cudaLaunchKernelEx(&cfg, k_batch_win_l<float>, a, blk, wg, b->window));
    } else if (b->window > 0) {
        cfg.dynamicSmemBytes = batch_win_smem(b->dtype, b->window);
        const WinBlock* blk = b->d_blocks;
        const WinGate* wg = b->d_wg;
        if (b->dtype == DIAQ_C128)
            DIAQ_CUDA(cudaLaunchKernelEx(&cfg, k_batch_win<double>, a, blk, wg, b->window));
        else
            DIAQ_CUDA(cudaLaunchKernelEx(&cfg, k_batch_win<float>, a, blk, wg, b->window));
    } else {
        if (b->n_runs > 0) {
            k_phase_tables<<<dim3(unsigned(b->n_runs), 2), 256, 0, s>>>(b->d_runs, b->d_theta, 0, PR_TAB_WEIGHT,
                                                                         b->d_ptabs);
            DIAQ_CUDA(cudaGetLastError());
        }
        if (b->dtype == DIAQ_C128)
            DIAQ_CUDA(cudaLaunchKernelEx(&cfg, k_batch<double>, a));
        else
            DIAQ_CUDA(cudaLaunchKernelEx(&cfg, k_batch<float>, a));
    }
    const int fb = 128;
    k_batch_finish<<<(b->n_inst + fb - 1) / fb, fb, 0, s>>>(b->d_inst, b->d_gates, b->d_partials, b->C, b->n_inst,
                                                          b->d_out, b->d_out + b->n_inst);
    DIAQ_CUDA(cudaGetLastError());
    return DIAQ_OK;
}

// Schedule for (C, threads), then capture theta upload, both kernels and the
// result download into a graph.
static diaq_status configure(diaq_batch_s* b, int C, int T, cudaStream_t s) {
    int teams = 0;
    DIAQ_TRY(resident_teams(b, C, T, &teams));
    teams = std::min(teams, b->n_inst);
    std::vector<int32_t> sched, first;
    make_schedule(b, teams, &sched, &first);
    // the old graph uses the buffers replaced below: drop it first, so a
    // failure from here on leaves no graph (diaq_batch_run then refuses)
    // rather than one that points at freed memory
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->d_sched) cudaFree(b->d_sched);
    if (b->d_team_first) cudaFree(b->d_team_first);
    b->d_sched = nullptr;
    b->d_team_first = nullptr;
    DIAQ_TRY(upload(&b->d_sched, sched));
    DIAQ_TRY(upload(&b->d_team_first, first));
    // partial rows of C columns
    if (b->d_partials) cudaFree(b->d_partials);
    b->d_partials = nullptr;
    std::vector<BInst> inst = b->inst;
    int64_t pos = 0;
    for (auto& I : inst) {
        I.part_off = pos;
        pos += int64_t(I.n_slots) * C;
    }
    cudaError_t e = cudaMalloc(&b->d_partials, size_t(std::max<int64_t>(pos, 1)) * sizeof(double));
    if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "cudaMalloc(batch partials): %s", cudaGetErrorString(e));
    DIAQ_CUDA(cudaMemcpy(b->d_inst, inst.data(), inst.size() * sizeof(BInst), cudaMemcpyHostToDevice));
    b->inst = inst;
    b->C = C;
    b->threads = T;
    b->teams = teams;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    // capture on a private stream so the caller's stream may be the legacy default
    if (!b->graph_stream) DIAQ_CUDA(cudaStreamCreateWithFlags(&b->graph_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    DIAQ_CUDA(cudaStreamBeginCapture(b->graph_stream, cudaStreamCaptureModeThreadLocal));
    diaq_status st = DIAQ_OK;
    const size_t nth = size_t(std::max(b->n_params_total, 1)) * sizeof(double);
    const size_t nout = size_t(b->n_inst + b->n_params_total) * sizeof(double);
    if (cudaMemcpyAsync(b->d_theta, b->h_theta, nth, cudaMemcpyHostToDevice, b->graph_stream) != cudaSuccess)
        st = fail(DIAQ_ERR_CUDA, "capture of the parameter upload failed");
    if (st == DIAQ_OK) st = launch_batch(b, b->graph_stream);
    if (st == DIAQ_OK && cudaMemcpyAsync(b->h_out, b->d_out, nout, cudaMemcpyDeviceToHost, b->graph_stream) != cudaSuccess)
        st = fail(DIAQ_ERR_CUDA, "capture of the result download failed");
    e = cudaStreamEndCapture(b->graph_stream, &graph);
    if (st != DIAQ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(batch)");
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(batch)");
    (void)s;
    return DIAQ_OK;
}

// Window tables for every instance (window 0 clears them); the caller
// reconfigures, which uploads the instances' block ranges.
static diaq_status batch_windows(diaq_batch_s* b, int window) {
    if (b->exec) {  // it may use the tables freed below
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->d_blocks) cudaFree(b->d_blocks);
    if (b->d_wg) cudaFree(b->d_wg);
    b->d_blocks = nullptr;
    b->d_wg = nullptr;
    b->window = 0;
    for (auto& I : b->inst) I.block_begin = I.block_end = 0;
    if (window == 0) return DIAQ_OK;
    std::vector<WinBlock> blocks;
    std::vector<WinGate> wg;
    for (auto& I : b->inst) {
        I.block_begin = int32_t(blocks.size());
        DIAQ_TRY(make_windows(b->gates.data() + I.gate_begin, I.gate_end - I.gate_begin, I.gate_begin, window,
                              &blocks, &wg));
        I.block_end = int32_t(blocks.size());
    }
    DIAQ_TRY(upload(&b->d_blocks, blocks));
    DIAQ_TRY(upload(&b->d_wg, wg));
    b->window = window;
    return DIAQ_OK;
}

static diaq_status run_graph(diaq_batch_s* b, cudaStream_t s) {
    if (!b->exec)
        return fail(DIAQ_ERR_ARG, "the batch has no launch configuration (an earlier reconfiguration failed): "
                                  "call diaq_batch_set_launch again");
    // order the replay after the caller's stream and the caller's stream after it
    cudaEvent_t ev;
    DIAQ_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    DIAQ_CUDA(cudaEventRecord(ev, s));
    DIAQ_CUDA(cudaStreamWaitEvent(b->graph_stream, ev, 0));
    DIAQ_CUDA(cudaGraphLaunch(b->exec, b->graph_stream));
    DIAQ_CUDA(cudaEventRecord(ev, b->graph_stream));
    DIAQ_CUDA(cudaStreamWaitEvent(s, ev, 0));
    DIAQ_CUDA(cudaEventSynchronize(ev));
    cudaEventDestroy(ev);
    return DIAQ_OK;
}

extern "C" {

diaq_status diaq_batch_create(int32_t n_inst, const int32_t* n_qubits, const int32_t* gate_first,
                              const diaq_gate* gates, const int32_t* param_first, const int32_t* term_first,
                              const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                              diaq_dtype dtype, diaq_batch_t* out) {
    clear_error();
    cudaGetLastError();
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_inst < 1 || !n_qubits || !gate_first || !param_first || !term_first)
        return fail(DIAQ_ERR_ARG, "need at least one instance and its index arrays");
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    diaq_batch_s* b = new (std::nothrow) diaq_batch_s();
    if (!b) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
    b->dtype = dtype;
    b->n_inst = n_inst;
    diaq_status st = DIAQ_OK;
    cudaError_t e = cudaSuccess;
    int64_t arena = 0;
    const int64_t align = 256 / int64_t(amp_bytes(dtype));
    for (int i = 0; i < n_inst && st == DIAQ_OK; ++i) {
        const int n = n_qubits[i];
        if (n < 2 || n > 30) {
            st = fail(DIAQ_ERR_ARG, "instance %d: n_qubits = %d outside [2, 30]", i, n);
            break;
        }
        if (gate_first[i + 1] < gate_first[i] || param_first[i + 1] < param_first[i] || term_first[i + 1] < term_first[i]) {
            st = fail(DIAQ_ERR_ARG, "instance %d: index arrays must be non-decreasing", i);
            break;
        }
        BInst I = {};
        I.n = n;
        I.gate_begin = int32_t(b->gates.size());
        I.param_begin = param_first[i];
        I.n_params = param_first[i + 1] - param_first[i];
        int slots = 1;
        for (int gi = gate_first[i]; gi < gate_first[i + 1]; ++gi) {
            const diaq_gate& g = gates[gi];
            if (g.k < 1 || g.k > 2) {
                st = fail(DIAQ_ERR_UNSUPPORTED, "instance %d gate %d: the batched path takes gates of 1 or 2 qubits", i, gi);
                break;
            }
            GateDesc d;
            std::vector<double> zero(size_t(std::max(I.n_params, 1)), 0.0);
            st = gate_desc_from(&g, n, zero.data(), &d);  // validates targets and generator
            if (st != DIAQ_OK) break;
            if (g.param >= I.n_params) {
                st = fail(DIAQ_ERR_ARG, "instance %d gate %d: parameter %d >= %d", i, gi, g.param, I.n_params);
                break;
            }
            BGate B = {};
            B.k = g.k;
            B.t[0] = g.targets[0];
            B.t[1] = g.k == 2 ? g.targets[1] : 0;
            B.param = g.param;
            B.scale = g.scale;
            B.slot = -1;
            if (g.param >= 0) {
                for (int q = 0; q < g.k; ++q) {
                    const char c = g.gen[q];
                    B.pauli[q] = (c == 'X' || c == 'x') ? 1 : (c == 'Y' || c == 'y') ? 2 : (c == 'Z' || c == 'z') ? 3 : 0;
                }
                B.slot = slots++;
            } else {
                for (size_t x = 0; x < d.m.size(); ++x) {
                    B.re[x] = d.m[x].real();
                    B.im[x] = d.m[x].imag();
                }
            }
            fill_rot(&B);  // targets and offsets for every gate
            b->gates.push_back(B);
        }
        if (st != DIAQ_OK) break;
        I.gate_end = int32_t(b->gates.size());
        I.term_begin = int32_t(b->terms.size());
        for (int t = term_first[i]; t < term_first[i + 1]; ++t) {
            const uint64_t valid = (uint64_t(1) << n) - 1;
            if ((xmask[t] & ~valid) || (zmask[t] & ~valid)) {
                st = fail(DIAQ_ERR_ARG, "instance %d term %d acts on a qubit >= %d", i, t, n);
                break;
            }
            BTerm T = {};
            T.x = xmask[t];
            T.z = zmask[t];
            const int ny = __builtin_popcountll(xmask[t] & zmask[t]) & 3;
            double kr = coeff[2 * t], ki = 0.0;  // Hermitian: real coefficient
            for (int r = 0; r < ny; ++r) {
                const double tr = -ki, ti = kr;
                kr = tr;
                ki = ti;
            }
            T.kr = kr;
            T.ki = ki;
            b->terms.push_back(T);
        }
        if (st != DIAQ_OK) break;
        // terms of equal X mask next to each other (the kernel sums their weights first)
        std::stable_sort(b->terms.begin() + I.term_begin, b->terms.end(),
                         [](const BTerm& u, const BTerm& v) { return u.x < v.x; });
        I.term_end = int32_t(b->terms.size());
        b->lflags &= lambda_tables(b->terms, I.term_begin, I.term_end, &b->ltab);
        I.n_slots = slots;
        I.psi_off = arena;
        arena += ((int64_t(1) << n) + align - 1) / align * align;
        I.lam_off = arena;
        arena += ((int64_t(1) << n) + align - 1) / align * align;
        b->inst.push_back(I);
        // forward + reverse touch psi once and psi, lam once per gate, plus the H psi pass
        b->work.push_back(double(int64_t(1) << n) * (3.0 * (I.gate_end - I.gate_begin) + 2.0 + (I.term_end - I.term_begin)));
        b->n_params_total = std::max(b->n_params_total, param_first[i + 1]);
    }
    b->arena_elems = arena;
    // the scaled form needs every instance's rotation applications (at most
    // two per parametric gate: forward and reverse) within the bound
    b->scaled_ok = true;
    for (const BInst& I : b->inst) b->scaled_ok &= 2 * (I.n_slots - 1) <= DIAQ_SCALED_MAX_ROT;
    // host tables validated; from here on the device is needed
    if (st == DIAQ_OK && (e = cudaGetDevice(&b->device)) != cudaSuccess) st = cuda_fail(e, "cudaGetDevice");
    if (st == DIAQ_OK) st = batch_exec(b);
    if (st == DIAQ_OK) st = upload(&b->d_gates, b->gates);
    if (st == DIAQ_OK) st = upload(&b->d_terms, b->terms);
    if (st == DIAQ_OK) st = upload_amps(b->dtype, b->ltab, &b->d_ltab);
    if (st == DIAQ_OK) {
        const size_t bytes = size_t(std::max<int64_t>(arena, 1)) * amp_bytes(dtype);
        if ((e = cudaMalloc(&b->d_arena, bytes)) != cudaSuccess)
            st = fail(DIAQ_ERR_ALLOC, "cudaMalloc of the %zu-byte state arena failed: %s", bytes, cudaGetErrorString(e));
    }
    const size_t nth = size_t(std::max(b->n_params_total, 1)) * sizeof(double);
    const size_t nout = size_t(n_inst + b->n_params_total) * sizeof(double);
    if (st == DIAQ_OK && ((e = cudaMalloc(reinterpret_cast<void**>(&b->d_theta), nth)) != cudaSuccess ||
                          (e = cudaMalloc(reinterpret_cast<void**>(&b->d_out), nout)) != cudaSuccess ||
                          (e = cudaMallocHost(reinterpret_cast<void**>(&b->h_theta), nth)) != cudaSuccess ||
                          (e = cudaMallocHost(reinterpret_cast<void**>(&b->h_out), nout)) != cudaSuccess))
        st = fail(DIAQ_ERR_ALLOC, "batch parameter/result buffers: %s", cudaGetErrorString(e));
    if (st == DIAQ_OK) {
        std::memset(b->h_theta, 0, nth);
        st = configure(b, 1, 256, nullptr);
    }
    if (st != DIAQ_OK) {
        batch_free(b);
        delete b;
        return st;
    }
    *out = b;
    return DIAQ_OK;
}

diaq_status diaq_batch_destroy(diaq_batch_t b) {
    clear_error();
    if (!b) return DIAQ_OK;
    cudaDeviceSynchronize();
    if (b->graph_stream) cudaStreamDestroy(b->graph_stream);
    batch_free(b);
    delete b;
    return DIAQ_OK;
}

diaq_status diaq_batch_set_launch(diaq_batch_t b, int32_t cluster, int32_t threads) {
    clear_error();
    cudaGetLastError();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (!(cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8))
        return fail(DIAQ_ERR_ARG, "cluster size %d not in {1, 2, 4, 8}", cluster);
    if (threads < 32 || threads > 256 || threads % 32)
        return fail(DIAQ_ERR_ARG, "threads %d not a multiple of 32 in [32, 256]", threads);
    if (b->window > 0 && threads != WIN_THREADS)
        return fail(DIAQ_ERR_ARG, "the window-fused kernel runs %d threads per block (got %d)", WIN_THREADS, threads);
    return configure(b, cluster, threads, nullptr);
}

diaq_status diaq_batch_set_runs(diaq_batch_t b, int32_t on) {
    clear_error();
    cudaGetLastError();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    DIAQ_CUDA(cudaDeviceSynchronize());
    if (b->exec) {  // it uses the lists replaced below
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->runs_on = on != 0;
    DIAQ_TRY(batch_exec(b));
    return configure(b, b->C, b->threads, nullptr);
}

diaq_status diaq_batch_set_scaled(diaq_batch_t b, int32_t on) {
    clear_error();
    cudaGetLastError();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    DIAQ_CUDA(cudaDeviceSynchronize());
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->scaled = on != 0;
    return configure(b, b->C, b->threads, nullptr);
}

diaq_status diaq_batch_get_scaled(diaq_batch_t b, int32_t* on, int32_t* active) {
    clear_error();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (on) *on = b->scaled ? 1 : 0;
    if (active) *active = batch_scaled_active(b) ? 1 : 0;
    return DIAQ_OK;
}

diaq_status diaq_batch_get_runs(diaq_batch_t b, int32_t* on, int32_t* n_runs) {
    clear_error();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (on) *on = b->runs_on ? 1 : 0;
    if (n_runs) *n_runs = b->n_runs;
    return DIAQ_OK;
}

diaq_status diaq_batch_set_window(diaq_batch_t b, int32_t window) {
    return diaq_batch_set_sweep(b, window, 1);
}

diaq_status diaq_batch_set_sweep(diaq_batch_t b, int32_t window, int32_t lanes) {
    clear_error();
    cudaGetLastError();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (window != 0 && (window < 2 || window > WIN_MAX))
        return fail(DIAQ_ERR_ARG, "window = %d: use 0 (one pass per gate) or 2..%d qubits", window, WIN_MAX);
    if (lanes != 1 && lanes != WIN_LANES)
        return fail(DIAQ_ERR_ARG, "lanes = %d: use 1 or %d threads per group", lanes, WIN_LANES);
    const int C = b->C;
    const int T = window > 0 ? WIN_THREADS : (b->window > 0 ? 256 : b->threads);
    b->lanes = window > 0 ? lanes : 1;
    diaq_status st = batch_windows(b, window);
    if (st == DIAQ_OK) st = configure(b, C, T, nullptr);
    if (st != DIAQ_OK) {
        const diaq_status first = st;
        b->lanes = 1;
        batch_windows(b, 0);
        configure(b, 1, 256, nullptr);
        return first;
    }
    return DIAQ_OK;
}

diaq_status diaq_batch_get_window(diaq_batch_t b, int32_t* window) {
    clear_error();
    if (!b || !window) return fail(DIAQ_ERR_ARG, "NULL argument");
    *window = b->window;
    return DIAQ_OK;
}

diaq_status diaq_batch_get_sweep(diaq_batch_t b, int32_t* window, int32_t* lanes) {
    clear_error();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (window) *window = b->window;
    if (lanes) *lanes = b->lanes;
    return DIAQ_OK;
}

diaq_status diaq_batch_run(diaq_batch_t b, const double* theta, double* energies, double* grads,
                           diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (b->n_params_total > 0 && !theta) return fail(DIAQ_ERR_ARG, "theta is NULL");
    for (int p = 0; p < b->n_params_total; ++p)
        if (!std::isfinite(theta[p])) return fail(DIAQ_ERR_ARG, "theta[%d] is not finite", p);
    if (b->n_params_total > 0) std::memcpy(b->h_theta, theta, sizeof(double) * size_t(b->n_params_total));
    DIAQ_TRY(run_graph(b, static_cast<cudaStream_t>(stream)));
    if (energies) std::memcpy(energies, b->h_out, sizeof(double) * size_t(b->n_inst));
    if (grads) std::memcpy(grads, b->h_out + b->n_inst, sizeof(double) * size_t(b->n_params_total));
    return DIAQ_OK;
}

diaq_status diaq_batch_autotune(diaq_batch_t b, const double* theta, int32_t reps, diaq_batch_tuning* report,
                                diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (b->n_params_total > 0 && !theta) return fail(DIAQ_ERR_ARG, "theta is NULL");
    if (reps < 1) reps = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int cls[] = {1, 2, 4, 8};
    const int ths[] = {64, 128, 256};  // k_batch is built for at most 256
    // window 0: one pass per gate; else the window-fused kernel, 1 or 4 lanes
    const int wins[] = {0, 3, 4, 5, 3, 4, 5};
    const int lns[] = {1, 1, 1, 1, WIN_LANES, WIN_LANES, WIN_LANES};
    float best = 1e30f;
    int bc = 1, bt = 256, bw = 0, bl = 1, tried = 0;
    cudaEvent_t e0, e1;
    DIAQ_CUDA(cudaEventCreate(&e0));
    DIAQ_CUDA(cudaEventCreate(&e1));
    if (b->n_params_total > 0) std::memcpy(b->h_theta, theta, sizeof(double) * size_t(b->n_params_total));
    for (int wi = 0; wi < 7; ++wi) {
      const int W = wins[wi], Ln = lns[wi];
      b->lanes = Ln;
      if (batch_windows(b, W) != DIAQ_OK) {
          clear_error();
          cudaGetLastError();
          continue;  // this window does not fit the circuits: skip it
      }
      for (int C : cls)
        for (int T : ths) {
            if (W > 0 && (T != WIN_THREADS || C == 1 || C == 4)) continue;  // fused shapes: clusters of 2 and 8
            if (configure(b, C, T, s) != DIAQ_OK) {
                clear_error();
                cudaGetLastError();
                continue;  // this shape does not fit: skip it
            }
            DIAQ_TRY(run_graph(b, s));  // warm
            DIAQ_CUDA(cudaEventRecord(e0, b->graph_stream));
            for (int r = 0; r < reps; ++r) DIAQ_CUDA(cudaGraphLaunch(b->exec, b->graph_stream));
            DIAQ_CUDA(cudaEventRecord(e1, b->graph_stream));
            DIAQ_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            DIAQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            ms /= float(reps);
            if (report && tried < DIAQ_BATCH_TUNE_MAX) {
                report->cluster[tried] = C;
                report->threads[tried] = T;
                report->window[tried] = W;
                report->lanes[tried] = Ln;
                report->ms[tried] = ms;
            }
            ++tried;
            if (ms < best) {
                best = ms;
                bc = C;
                bt = T;
                bw = W;
                bl = Ln;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!tried) return fail(DIAQ_ERR_UNSUPPORTED, "no launch shape fits");
    b->lanes = bl;
    DIAQ_TRY(batch_windows(b, bw));
    DIAQ_TRY(configure(b, bc, bt, s));
    if (report) {
        report->n_tried = std::min(tried, DIAQ_BATCH_TUNE_MAX);
        report->best_cluster = bc;
        report->best_threads = bt;
        report->best_window = bw;
        report->best_lanes = bl;
        report->best_ms = best;
    }
    return DIAQ_OK;
}

diaq_status diaq_batch_query(diaq_batch_t b, int32_t* cluster, int32_t* threads, int32_t* teams, int64_t* arena_bytes) {
    clear_error();
    if (!b) return fail(DIAQ_ERR_ARG, "batch is NULL");
    if (cluster) *cluster = b->C;
    if (threads) *threads = b->threads;
    if (teams) *teams = b->teams;
    if (arena_bytes) *arena_bytes = b->arena_elems * int64_t(amp_bytes(b->dtype));
    return DIAQ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint plan: the adjoint sweep of one circuit as a CUDA graph. Fixed
// gates are launched with their matrices in kernel parameters (they do not
// change between replays); parametric gates are Pauli rotations whose
// cos(a/2) and kappa a first kernel derives from the uploaded parameters.
// The graph (parameter upload, sweeps, reductions, result download) is
// captured once and replayed for every new theta.
// ---------------------------------------------------------------------------
namespace diaq {

struct RotAngles {
    double cs, kfr, kfi, kar, kai;  // cos(a/2), kappa of U, kappa of U^dag
    // scaled form (rot_groups_s): U = sigma V per direction
    int32_t m1;                     // 1: sigma is kappa's non-zero part, 0: sigma = cos(a/2)
    double cff, cfr;                // V's coefficient, forward and reverse
    double sgf, sgr;                // sigma, forward and reverse
};

__global__ void k_plan_angles(const BGate* gates, int n_gates, const double* theta, RotAngles* out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_gates || gates[g].param < 0) return;
    RotAngles A;
    rot_angle(gates[g], theta, false, &A.cs, &A.kfr, &A.kfi);
    rot_angle(gates[g], theta, true, &A.cs, &A.kar, &A.kai);
    int m1r = 0;  // the same form both ways: |cos| and |kappa| do not change
    rot_scaled_coefs(A.cs, A.kfr, A.kfi, gates[g].rot.ny, &A.m1, &A.cff, &A.sgf);
    rot_scaled_coefs(A.cs, A.kar, A.kai, gates[g].rot.ny, &m1r, &A.cfr, &A.sgr);
    out[g] = A;
}

// Scale bookkeeping of the scaled sweep, one thread, in sweep order. The
// stored states are the true ones times 1/prod(sigma) of the rotations
// applied so far (ScaleEvent::FWD / REV multiply inv_s by sigma). Every
// partial of a reverse step, and the energy after the forward sweep, is
// taken on states that carry the same factor 1/inv_s in psi and lambda, so
// scale[slot] = inv_s^2 turns it into the true value.
struct ScaleEvent {
    int32_t kind;  // 0 forward rotation (idx: gate), 1 energy, 2 partial slot (idx: slot), 3 reverse rotation
    int32_t idx;
};

// One block of 256 threads: thread t takes a contiguous chunk of the
// events, forms the product of its chunk's factors (all loads in flight at
// once), an exclusive product scan over the threads gives each chunk its
// starting inv_s, and each thread then writes its chunk's marks.
constexpr int kScaleThreads = 256;
constexpr int kScaleChunk = 8;  // events per thread and pass

__global__ void __launch_bounds__(kScaleThreads) k_plan_scales(const ScaleEvent* __restrict__ ev, int n_ev,
                                                               const RotAngles* __restrict__ ang, int n_slots,
                                                               double* scale) {
    __shared__ double warp_prod[kScaleThreads / 32];
    __shared__ double carry;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int s = t; s < n_slots; s += kScaleThreads) scale[s] = 1.0;
    if (t == 0) carry = 1.0;
    __syncthreads();  // marks below overwrite the defaults
    for (int base = 0; base < n_ev; base += kScaleThreads * kScaleChunk) {
        const int e0 = base + t * kScaleChunk;
        ScaleEvent x[kScaleChunk];
        double f[kScaleChunk];
#pragma unroll
        for (int c = 0; c < kScaleChunk; ++c) {
            x[c] = e0 + c < n_ev ? ev[e0 + c] : ScaleEvent{-1, -1};  // padding: no factor, no mark
            f[c] = x[c].kind == 0 ? ang[x[c].idx].sgf : (x[c].kind == 3 ? ang[x[c].idx].sgr : 1.0);
        }
        double prod = 1.0;
#pragma unroll
        for (int c = 0; c < kScaleChunk; ++c) prod *= f[c];
        // exclusive scan of the chunk products: within the warp, then over warps
        double incl = prod;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl *= v;
        }
        if (lane == 31) warp_prod[warp] = incl;
        __syncthreads();
        double before = carry;
        for (int w = 0; w < warp; ++w) before *= warp_prod[w];
        double excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = 1.0;
        double inv_s = before * excl;
#pragma unroll
        for (int c = 0; c < kScaleChunk; ++c) {
            if (x[c].kind == 1) scale[0] = inv_s * inv_s;
            else if (x[c].kind == 2) scale[x[c].idx] = inv_s * inv_s;
            inv_s *= f[c];
        }
        __syncthreads();
        if (t == kScaleThreads - 1) carry = inv_s;  // the last thread ends the pass
        __syncthreads();
    }
}

// A Pauli rotation over the whole state, forward (lam == NULL) or reverse
// with its partial. SC: the scaled form (complex128 plans; the angles carry
// the form and coefficient of each direction).
template <typename R, int K, int XL, int KT, int SC>
__global__ void __launch_bounds__(256) k_plan_rot(amp_t<R>* psi, amp_t<R>* lam, const BGate* gate,
                                                  const RotAngles* ang, int n, double* part) {
    __shared__ double warps[32];
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    const RotAngles a = *ang;
    const bool adj = lam != nullptr;  // the reverse sweep applies U^dag
    double v;
    if constexpr (SC != 0) {
        const R cf = R(adj ? a.cfr : a.cff);
        if (adj) v = rot_groups_sc<R, K, XL, (K == 1 ? 4 : (sizeof(R) == 4 ? 2 : 1)), KT>(psi, lam, n, gate->rot,
                                                                                     a.m1 != 0, cf, tid, nth);
        else v = rot_groups_sc<R, K, XL, (K == 1 ? 4 : 2), KT>(psi, nullptr, n, gate->rot, a.m1 != 0, cf, tid, nth);
    } else {
        v = rot_groups<R, K, XL, KT>(psi, lam, n, gate->rot, R(a.cs), R(adj ? a.kar : a.kfr), R(adj ? a.kai : a.kfi),
                                     tid, nth);
    }
    if (part) {
        const double s = block_sum(v, warps);
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_plan_lambda(const amp_t<R>* psi, amp_t<R>* lam, const BTerm* terms,
                                                     const void* ltab, int n_terms, int64_t N, double* part,
                                                     int lflags) {
    __shared__ double warps[32];
    const double v = lambda_share_any<R>(lflags, psi, lam, terms, reinterpret_cast<const amp_t<R>*>(ltab), 0, n_terms, N,
                                         int64_t(blockIdx.x) * blockDim.x + threadIdx.x,
                                         int64_t(gridDim.x) * blockDim.x);
    const double es = block_sum(v, warps);
    if (threadIdx.x == 0) part[blockIdx.x] = es;
}

template <typename R>
__global__ void k_plan_init(const amp_t<R>* psi0, amp_t<R>* psi, int64_t N, const void* init, int n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
        amp_t<R> v;
        if (psi0) {
            v = psi0[i];
        } else if (init) {  // the state after the leading product layer
            v = product_amp<R>(reinterpret_cast<const amp_t<R>*>(init), n, i);
        } else {
            v.x = R(i == 0 ? 1 : 0);
            v.y = R(0);
        }
        psi[i] = v;
    }
}

// Row sums of the partials, one block per row (fixed shuffle tree).
__global__ void __launch_bounds__(256) k_plan_rows(const double* __restrict__ part, int P, double* rows) {
    __shared__ double warps[32];
    const double* row = part + int64_t(blockIdx.x) * P;
    double s = 0.0;
    for (int c = threadIdx.x; c < P; c += blockDim.x) s += row[c];
    s = block_sum(s, warps);
    if (threadIdx.x == 0) rows[blockIdx.x] = s;
}

// One parametric gate's contribution to its parameter: rows[slot] times the
// gate's scale (a = scale theta).
struct FinTerm {
    int32_t slot;
    double scale;
};

// out[0] = energy, out[1 + p] = dE/dtheta_p from the row sums: one thread per
// parameter sums its gates' contributions (terms[first[p] .. first[p+1]),
// in gate order); scale (NULL: none) rescales each row of the scaled sweep.
__global__ void __launch_bounds__(256) k_plan_finish(const FinTerm* __restrict__ terms, const int32_t* __restrict__ first,
                                                     const double* __restrict__ rows, const double* __restrict__ scale,
                                                     int n_params, double* out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) out[0] = scale ? rows[0] * scale[0] : rows[0];
    for (int p = t; p < n_params; p += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int e = first[p]; e < first[p + 1]; ++e) {
            const FinTerm f = terms[e];
            v += f.scale * (scale ? rows[f.slot] * scale[f.slot] : rows[f.slot]);
        }
        out[1 + p] = v;
    }
}

// A diagonal run (phase.cuh) of the plan: forward D psi, or reverse with the
// run's gradient rows (P columns) and D^dag on psi and lambda.
template <typename R, bool REV>
__global__ void __launch_bounds__(256) k_plan_phase(amp_t<R>* psi, amp_t<R>* lam, const PhaseRun* __restrict__ run,
                                                    const double2* __restrict__ table, int n, double* part, int P) {
    __shared__ PhaseTables<PR_TAB_ALL, R> tb;
    __shared__ PhaseRun rs;
    __shared__ double warps[32];
    {
        const int* src = reinterpret_cast<const int*>(run);
        int* dst = reinterpret_cast<int*>(&rs);
        for (int i = threadIdx.x; i < int(sizeof(PhaseRun) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    phase_tables_load<PR_TAB_ALL>(table, phase_entries(rs, n), &tb);
    double acc[PR_MAX_CROT];
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    if (rs.kind == PR_WEIGHT)
        phase_run_sweep<R, PR_WEIGHT, PR_TAB_ALL>(psi, REV ? lam : nullptr, n, rs, tb, tid, nth, acc);
    else
        phase_run_sweep<R, PR_CHUNKS, PR_TAB_ALL>(psi, REV ? lam : nullptr, n, rs, tb, tid, nth, acc);
    if (!REV) return;
    if (rs.kind == PR_WEIGHT) {
        // the run's sum in the first member's row, zeros in the others' (same
        // parameter and scale, so the finish sums the same total)
        const double v = block_sum(acc[0], warps);
        if (threadIdx.x == 0) {
            part[int64_t(rs.rot_slot[0]) * P + blockIdx.x] = v;
            for (int g = 1; g < rs.n_rot; ++g) part[int64_t(rs.rot_slot[g]) * P + blockIdx.x] = 0.0;
        }
    } else {
        for (int g = 0; g < rs.n_rot; ++g) {
            const double v = block_sum(acc[g], warps);
            if (threadIdx.x == 0) part[int64_t(rs.rot_slot[g]) * P + blockIdx.x] = v;
        }
    }
}

// Reverse step of a chunk-form run (an ansatz layer's RZs and CZ ladder)
// with cheaper gradient terms. The term of a rotation on qubit q is
// sum_i (-1)^(bit q of i) t_i, t_i = Im(conj(lambda_i) psi_i). The loop
// order is phase_run_sweep's chunk form: warp v of the grid (W = 8 P warps)
// takes the aligned blocks of 256 amplitudes v, v + W, ..., its lane l the
// amplitudes 32 j + l of each. So bits 0..4 of i are the lane's, bits 5..7
// are j, and, W being a multiple of 2^(3 + z) (z = trailing zero bits of P),
// bits 8..10 are those of the warp within its block and bits 11..10+z those
// of the block index: all fixed for the thread or known per j. The thread
// therefore sums t_i per j (T_j), and for rotations on bits >= f = 11 + z
// (bits of base, fixed within a block of 256) the warp adds its block share,
// signed by that bit, once per block into shared sums. At the end, a
// Walsh-Hadamard
// butterfly over the lanes of T = sum_j T_j gives the terms for q < 5,
// signed sums of the T_j those for q = 5..7, the warps' totals signed by
// their warp bit those for q = 8..10, and the block's total signed by its
// block-index bit those for q = 11..f-1. Requires 256 threads per block.
template <typename R>
__global__ void __launch_bounds__(256, 2) k_plan_phase_rev_chunks(amp_t<R>* __restrict__ psi,
                                                               amp_t<R>* __restrict__ lam,
                                                               const PhaseRun* __restrict__ run,
                                                               const double2* __restrict__ table, int n, double* part,
                                                               int P) {
    using A = amp_t<R>;
    __shared__ PhaseTables<PR_TAB_ALL, R> tb;
    __shared__ PhaseRun rs;
    __shared__ double wt[8][9];               // per warp: sum T, lane-bit sums S_0 .. S_4, j-bit sums J_5 .. J_7
    __shared__ double wv[8][PR_MAX_CROT];     // per warp: the varying-bit sums (lane 0 adds)
    __shared__ int vq[PR_MAX_CROT];           // varying-bit rotations: their qubit
    __shared__ int vg[PR_MAX_CROT];           // ... and their index in the run
    __shared__ int nv;
    {
        const int* src = reinterpret_cast<const int*>(run);
        int* dst = reinterpret_cast<int*>(&rs);
        for (int i = threadIdx.x; i < int(sizeof(PhaseRun) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    const int64_t N = int64_t(1) << n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int f = 11 + __ffs(int(gridDim.x)) - 1;  // bits 0 .. f-1 of i are fixed or known per j
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int g = 0; g < rs.n_rot && g < PR_MAX_CROT; ++g) {
            const int q = __ffsll((long long)rs.rot_z[g]) - 1;
            if (q >= f) {
                vq[c] = q;
                vg[c] = g;
                ++c;
            }
        }
        nv = c;
    }
    for (int e = threadIdx.x; e < 8 * PR_MAX_CROT; e += blockDim.x) wv[e / PR_MAX_CROT][e % PR_MAX_CROT] = 0.0;
    phase_tables_load<PR_TAB_ALL>(table, phase_entries(rs, n), &tb);  // synchronises
    const int chunks = (n + PR_CHUNK_BITS - 1) / PR_CHUNK_BITS;
    const int n_var = nv;
    const int64_t nblk = (N + 255) >> 8;
    const int64_t W = int64_t(gridDim.x) * 8;
    Acc<R> tj[8];
    for (int64_t blk = int64_t(blockIdx.x) * 8 + warp; blk < nblk; blk += W) {
        const int64_t base = blk << 8;
        R hr = R(1), hi = R(0);  // the higher chunks' product
        for (int c = 1; c < chunks; ++c) {
            const int e = (c << 8) | int((base >> (8 * c)) & 255);
            const R qr = tb.re[e], qi = tb.im[e];
            if (c == 1) {
                hr = qr;
                hi = qi;
            } else {
                const R tr = fma(hr, qr, -hi * qi);
                hi = fma(hr, qi, hi * qr);
                hr = tr;
            }
        }
        int bneg;
        unsigned lmask;
        phase_cz_block(rs, uint64_t(base), &bneg, &lmask);
        R sb = R(0);  // this lane's share of the block: bits >= 8 of i are those of base
        auto amp = [&](int j, const A& p, const A& l) {
            const int lo = lane + 32 * j;
            const int64_t i = base + lo;
            R pr = tb.re[lo], pi = tb.im[lo];
            if (chunks > 1) {
                const R tr = fma(pr, hr, -pi * hi);
                pi = fma(pr, hi, pi * hr);
                pr = tr;
            }
            const int neg = bneg ^ (__popc(unsigned(lo) & lmask) & 1);
            const unsigned m = neg ? 0x80000000u : 0u;  // the sign by an integer flip
            A ph;
            ph.x = flip_sign(pr, m);
            ph.y = flip_sign(pi, m);
            const R t = fma(l.x, p.y, -l.y * p.x);  // Im(conj(l) p)
            tj[j].add(t);
            sb += t;
            lam[i] = cmul<R>(ph, l);
            psi[i] = cmul<R>(ph, p);
        };
        if (base + 256 <= N) {  // a whole block: V amplitudes' loads in flight together
            constexpr int V = 4;
#pragma unroll
            for (int j0 = 0; j0 < 8; j0 += V) {
                A p[V], l[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int64_t i = base + lane + 32 * (j0 + v);
                    p[v] = psi[i];
                    l[v] = lam[i];
                }
#pragma unroll
                for (int v = 0; v < V; ++v) amp(j0 + v, p[v], l[v]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t i = base + lane + 32 * j;
                if (i >= N) break;  // n < 8 only
                amp(j, psi[i], lam[i]);
            }
        }
        if (n_var > 0) {  // the warp's block share, signed per rotation into its shared sums
            double v = double(sb);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0)
                for (int u = 0; u < n_var; ++u) wv[warp][u] += ((uint64_t(base) >> vq[u]) & 1) ? -v : v;
        }
    }
    double tv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) tv[j] = tj[j].value();
    // lane butterfly: lane m ends with sum_l (-1)^popc(l & m) T_l
    double w = ((tv[0] + tv[1]) + (tv[2] + tv[3])) + ((tv[4] + tv[5]) + (tv[6] + tv[7]));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double v = __shfl_xor_sync(0xffffffffu, w, o);
        w = (lane & o) ? v - w : w + v;
    }
    if (lane == 0) wt[warp][0] = w;
#pragma unroll
    for (int q = 0; q < 5; ++q)
        if (lane == (1 << q)) wt[warp][1 + q] = w;
#pragma unroll
    for (int b = 0; b < 3; ++b) {  // q = 5 + b: sum_j (-1)^(bit b of j) T_j over the warp
        double v = 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) v += ((j >> b) & 1) ? -tv[j] : tv[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) wt[warp][6 + b] = v;
    }
    __syncthreads();
    if (threadIdx.x < rs.n_rot && threadIdx.x < PR_MAX_CROT) {
        const int g = threadIdx.x;
        const int q = __ffsll((long long)rs.rot_z[g]) - 1;
        double v = 0.0;
        if (q >= f) {
            int u = 0;
            while (vg[u] != g) ++u;
            for (int x = 0; x < 8; ++x) v += wv[x][u];
        } else if (q < 5) {
            for (int x = 0; x < 8; ++x) v += wt[x][1 + q];
        } else if (q < 8) {
            for (int x = 0; x < 8; ++x) v += wt[x][6 + q - 5];
        } else if (q < 11) {
            for (int x = 0; x < 8; ++x) v += ((x >> (q - 8)) & 1) ? -wt[x][0] : wt[x][0];
        } else {
            for (int x = 0; x < 8; ++x) v += wt[x][0];
            if ((blockIdx.x >> (q - 11)) & 1) v = -v;
        }
        part[int64_t(rs.rot_slot[g]) * P + blockIdx.x] = v;
    }
}

// Two consecutive one-qubit X/Y rotations (rot2_groups) in one launch:
// forward A then B, or reverse with both partials.
template <typename R, int GA, int GB, int SC>
__global__ void __launch_bounds__(256) k_plan_rot2(amp_t<R>* psi, amp_t<R>* lam, const BGate* ga, const BGate* gb,
                                                   const RotAngles* aa, const RotAngles* ab, int n, double* part_a,
                                                   double* part_b) {
    __shared__ double warps[32];
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = int64_t(gridDim.x) * blockDim.x;
    const bool adj = lam != nullptr;
    const RotAngles x = *aa, y = *ab;
    Rot1<R, GA, SC != 0> A;
    Rot1<R, GB, SC != 0> B;
    if (SC) {
        A.c0 = R(adj ? x.cfr : x.cff);
        A.c1 = R(0);
        A.m1 = x.m1 != 0;
        B.c0 = R(adj ? y.cfr : y.cff);
        B.c1 = R(0);
        B.m1 = y.m1 != 0;
    } else {  // kappa's non-zero part: imaginary for X, real for Y
        A.c0 = R(x.cs);
        A.c1 = R(GA == 1 ? (adj ? x.kai : x.kfi) : (adj ? x.kar : x.kfr));
        A.m1 = false;
        B.c0 = R(y.cs);
        B.c1 = R(GB == 1 ? (adj ? y.kai : y.kfi) : (adj ? y.kar : y.kfr));
        B.m1 = false;
    }
    double pa = 0.0, pb = 0.0;
    const int qa = ga->t[0], qb = gb->t[0];
    if (adj)
        rot2_groups<R, GA, GB, SC != 0, (sizeof(R) == 4 ? 2 : 1)>(psi, lam, n, qa, qb, A, B, tid, nth, &pa, &pb);
    else
        rot2_groups<R, GA, GB, SC != 0, (sizeof(R) == 4 ? 4 : 2)>(psi, nullptr, n, qa, qb, A, B, tid, nth, &pa, &pb);
    if (part_a) {
        const double sa = block_sum(pa, warps);
        const double sb = block_sum(pb, warps);
        if (threadIdx.x == 0) {
            part_a[blockIdx.x] = sa;
            part_b[blockIdx.x] = sb;
        }
    }
}


template <typename R, int SC>
static void launch_plan_rot2_sc(const BGate& a, const BGate& b, amp_t<R>* psi, amp_t<R>* lam, const BGate* da,
                                const BGate* db, const RotAngles* aa, const RotAngles* ab, int n, double* pa,
                                double* pb, int P, cudaStream_t s) {
    const int ga = a.pauli[0], gb = b.pauli[0];  // 1 X, 2 Y
    if (ga == 1 && gb == 1) k_plan_rot2<R, 1, 1, SC><<<P, 256, 0, s>>>(psi, lam, da, db, aa, ab, n, pa, pb);
    else if (ga == 1) k_plan_rot2<R, 1, 2, SC><<<P, 256, 0, s>>>(psi, lam, da, db, aa, ab, n, pa, pb);
    else if (gb == 1) k_plan_rot2<R, 2, 1, SC><<<P, 256, 0, s>>>(psi, lam, da, db, aa, ab, n, pa, pb);
    else k_plan_rot2<R, 2, 2, SC><<<P, 256, 0, s>>>(psi, lam, da, db, aa, ab, n, pa, pb);
}

template <typename R>
static void launch_plan_rot2(const BGate& a, const BGate& b, amp_t<R>* psi, amp_t<R>* lam, const BGate* da,
                             const BGate* db, const RotAngles* aa, const RotAngles* ab, int n, double* pa, double* pb,
                             int P, bool scaled, cudaStream_t s) {
    if constexpr (sizeof(R) == 8) {
        if (scaled) {
            launch_plan_rot2_sc<R, 1>(a, b, psi, lam, da, db, aa, ab, n, pa, pb, P, s);
            return;
        }
    }
    launch_plan_rot2_sc<R, 0>(a, b, psi, lam, da, db, aa, ab, n, pa, pb, P, s);
}

// kappa's form follows from the generator: imaginary for an even Y count
// (KT = 1), real for an odd one (KT = 2)
template <typename R, int KT, int SC>
static void launch_plan_rot_kt(const BGate& g, amp_t<R>* psi, amp_t<R>* lam, const BGate* dg, const RotAngles* da,
                               int n, double* part, int P, cudaStream_t s) {
    if (g.k == 1) {
        if (g.xl == 0) k_plan_rot<R, 1, 0, KT, SC><<<P, 256, 0, s>>>(psi, lam, dg, da, n, part);
        else k_plan_rot<R, 1, 1, KT, SC><<<P, 256, 0, s>>>(psi, lam, dg, da, n, part);
        return;
    }
    switch (g.xl) {
        case 0: k_plan_rot<R, 2, 0, KT, SC><<<P, 256, 0, s>>>(psi, lam, dg, da, n, part); break;
        case 1: k_plan_rot<R, 2, 1, KT, SC><<<P, 256, 0, s>>>(psi, lam, dg, da, n, part); break;
        case 2: k_plan_rot<R, 2, 2, KT, SC><<<P, 256, 0, s>>>(psi, lam, dg, da, n, part); break;
        default: k_plan_rot<R, 2, 3, KT, SC><<<P, 256, 0, s>>>(psi, lam, dg, da, n, part); break;
    }
}

// scaled: the scaled form (complex128 only)
template <typename R>
static void launch_plan_rot(const BGate& g, amp_t<R>* psi, amp_t<R>* lam, const BGate* dg, const RotAngles* da,
                            int n, double* part, int P, bool scaled, cudaStream_t s) {
    if constexpr (sizeof(R) == 8) {
        if (scaled) {
            if (g.rot.ny & 1) launch_plan_rot_kt<R, 2, 1>(g, psi, lam, dg, da, n, part, P, s);
            else launch_plan_rot_kt<R, 1, 1>(g, psi, lam, dg, da, n, part, P, s);
            return;
        }
    }
    if (g.rot.ny & 1) launch_plan_rot_kt<R, 2, 0>(g, psi, lam, dg, da, n, part, P, s);
    else launch_plan_rot_kt<R, 1, 0>(g, psi, lam, dg, da, n, part, P, s);
}

// ---------------------------------------------------------------------------
// Window-fused sweep. The gates are grouped into blocks that act on at most
// WIN_MAX qubits (the window), moving gates only past gates on disjoint
// qubits, so the circuit's operator and every gradient term are unchanged.
// One launch runs one block over the whole state: each thread takes a group
// (the 2^w amplitudes that share their bits outside the window), stages it
// in shared memory, runs the block's gates on it in order (forward) or in
// reverse order with each parametric gate's partial Im <lam|P|psi> taken
// before U^dag (reverse), and writes it back. The state is read and written
// once per block instead of once per gate.
// ---------------------------------------------------------------------------
static size_t win_smem(diaq_dtype dt, int nq, int count, int np) {
    const size_t opb = dt == DIAQ_C128 ? sizeof(WinOp<double>) : sizeof(WinOp<float>);
    const size_t ab = amp_bytes(dt);
    const size_t head = ((opb * size_t(count) + 15) / 16) * 16;
    return head + 2 * (size_t(1) << nq) * WIN_THREADS * ab + size_t(np) * WIN_THREADS * sizeof(double);
}

// Stage the block's gates for the sweep's direction (thread i < count
// writes op i) and clear the partial accumulators.
template <typename R>
__device__ __forceinline__ void plan_stage(const BGate* __restrict__ gates, const RotAngles* __restrict__ ang,
                                           const WinGate* __restrict__ wg, const WinBlock& w, bool rev,
                                           WinOp<R>* ops, Acc<R>* sa) {
    const int T = blockDim.x, t = threadIdx.x;
    for (int i = t; i < w.count; i += T) {
        const WinGate x = wg[w.first + i];
        const BGate& G = gates[x.g];
        WinOp<R>& o = ops[i];
        o.k = G.k;
        o.b0 = x.b0;
        o.b1 = x.b1;
        o.j = G.param >= 0 ? x.j : -1;
        o.xl = G.xl;
        o.zl = G.rot.zl;
        o.ny = G.rot.ny;
        o.cs = R(0);
        o.kr = R(0);
        o.ki = R(0);
        const int Dk = 1 << G.k;
        if (G.param >= 0) {
            const RotAngles a = ang[x.g];
            o.cs = R(a.cs);
            o.kr = R(rev ? a.kar : a.kfr);
            o.ki = R(rev ? a.kai : a.kfi);
        } else {
            for (int r = 0; r < Dk; ++r)
                for (int c = 0; c < Dk; ++c) {
                    const double vr = rev ? G.re[c * Dk + r] : G.re[r * Dk + c];
                    const double vi = rev ? -G.im[c * Dk + r] : G.im[r * Dk + c];
                    o.mre[r * Dk + c] = R(vr);
                    o.mim[r * Dk + c] = R(vi);
                    o.ty[r * Dk + c] = dev_entry_type(double(R(vr)), double(R(vi)));
                }
        }
    }
    for (int j = 0; j < w.np; ++j) sa[j * T + t] = Acc<R>();
    __syncthreads();
}


static size_t win_smem_lanes(diaq_dtype dt, int nq, int count, int np) {
    const size_t opb = dt == DIAQ_C128 ? sizeof(WinOp<double>) : sizeof(WinOp<float>);
    const size_t head = ((opb * size_t(count) + 15) / 16) * 16;
    const size_t gpc = WIN_THREADS / WIN_LANES;
    return head + 2 * gpc * ((size_t(1) << nq) + 1) * amp_bytes(dt) + size_t(np) * WIN_THREADS * sizeof(double);
}

template <typename R>
__global__ void __launch_bounds__(WIN_THREADS, 4) k_plan_win_l(amp_t<R>* psi, amp_t<R>* lam,
                                                               const BGate* __restrict__ gates,
                                                               const RotAngles* __restrict__ ang,
                                                               const WinGate* __restrict__ wg,
                                                               const __grid_constant__ WinBlock w, int n,
                                                               double* part, int P) {
    using A = amp_t<R>;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double warps[32];
    constexpr int L = WIN_LANES;
    const int T = WIN_THREADS, t = threadIdx.x;
    const int GPC = T / L, gs = t / L, li = t % L;
    const int D = 1 << w.nq, SD = D + 1;  // one padding amplitude per group against bank conflicts
    const bool rev = lam != nullptr;
    WinOp<R>* ops = reinterpret_cast<WinOp<R>*>(sm);
    A* sp = reinterpret_cast<A*>(sm + ((sizeof(WinOp<R>) * size_t(w.count) + 15) / 16) * 16);
    A* sl = sp + GPC * SD;
    Acc<R>* sa = reinterpret_cast<Acc<R>*>(sl + GPC * SD);
    plan_stage<R>(gates, ang, wg, w, rev, ops, sa);
    const int64_t G = int64_t(1) << (n - w.nq);
    A* gp = sp + gs * SD;
    A* gl = sl + gs * SD;
    // every thread of the block makes the same number of trips, so every
    // lane of a warp reaches each __syncwarp
    for (int64_t g0 = int64_t(blockIdx.x) * GPC; g0 < G; g0 += int64_t(gridDim.x) * GPC) {
        const int64_t g = g0 + gs;
        const int64_t base = g < G ? insert_zeros_rt(g, w.q, w.nq) : 0;
        const bool valid = g < G && DIAQ_BOUNDS_OK(base + w.off[D - 1], int64_t(1) << n, BS_WINDOW);
        if (valid) {
            for (int e = li; e < D; e += L) gp[e] = psi[base + w.off[e]];
            if (rev)
                for (int e = li; e < D; e += L) gl[e] = lam[base + w.off[e]];
        }
        __syncwarp();
        if (!rev) {
            for (int i = 0; i < w.count; ++i) {
                win_apply<R, 1>(ops[i], gp, nullptr, D, 1, nullptr, li, L);
                __syncwarp();
            }
        } else {
            for (int i = w.count - 1; i >= 0; --i) {
                const WinOp<R>& o = ops[i];
                win_apply<R, 1>(o, gp, gl, D, 1, (valid && o.j >= 0) ? sa + o.j * T + t : nullptr, li, L);
                __syncwarp();
            }
        }
        if (valid) {
            for (int e = li; e < D; e += L) psi[base + w.off[e]] = gp[e];
            if (rev)
                for (int e = li; e < D; e += L) lam[base + w.off[e]] = gl[e];
        }
        __syncwarp();
    }
    if (rev) {
        for (int j = 0; j < w.np; ++j) {
            const double v = block_sum(sa[j * T + t].value(), warps);
            if (t == 0) part[int64_t(w.slot[j]) * P + blockIdx.x] = v;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(WIN_THREADS) k_plan_win(amp_t<R>* psi, amp_t<R>* lam, const BGate* __restrict__ gates,
                                                          const RotAngles* __restrict__ ang,
                                                          const WinGate* __restrict__ wg,
                                                          const __grid_constant__ WinBlock w, int n, double* part,
                                                          int P) {
    using A = amp_t<R>;
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double warps[32];
    const int T = WIN_THREADS, t = threadIdx.x;
    const int D = 1 << w.nq;
    const bool rev = lam != nullptr;
    WinOp<R>* ops = reinterpret_cast<WinOp<R>*>(sm);
    A* sp = reinterpret_cast<A*>(sm + ((sizeof(WinOp<R>) * size_t(w.count) + 15) / 16) * 16);
    A* sl = sp + D * T;
    Acc<R>* sa = reinterpret_cast<Acc<R>*>(sl + D * T);
    // stage the block's gates in the direction of this sweep
    for (int i = t; i < w.count; i += T) {
        const WinGate x = wg[w.first + i];
        const BGate& G = gates[x.g];
        WinOp<R>& o = ops[i];
        o.k = G.k;
        o.b0 = x.b0;
        o.b1 = x.b1;
        o.j = G.param >= 0 ? x.j : -1;
        o.xl = G.xl;
        o.zl = G.rot.zl;
        o.ny = G.rot.ny;
        o.cs = R(0);
        o.kr = R(0);
        o.ki = R(0);
        const int Dk = 1 << G.k;
        if (G.param >= 0) {
            const RotAngles a = ang[x.g];
            o.cs = R(a.cs);
            o.kr = R(rev ? a.kar : a.kfr);
            o.ki = R(rev ? a.kai : a.kfi);
        } else {
            for (int r = 0; r < Dk; ++r)
                for (int c = 0; c < Dk; ++c) {
                    const double vr = rev ? G.re[c * Dk + r] : G.re[r * Dk + c];
                    const double vi = rev ? -G.im[c * Dk + r] : G.im[r * Dk + c];
                    o.mre[r * Dk + c] = R(vr);
                    o.mim[r * Dk + c] = R(vi);
                    o.ty[r * Dk + c] = dev_entry_type(double(R(vr)), double(R(vi)));
                }
        }
    }
    for (int j = 0; j < w.np; ++j) sa[j * T + t] = Acc<R>();
    __syncthreads();
    const int64_t G = int64_t(1) << (n - w.nq);
    A* cp = sp + t;
    A* cl = sl + t;
    for (int64_t g = int64_t(blockIdx.x) * T + t; g < G; g += int64_t(gridDim.x) * T) {
        const int64_t base = insert_zeros_rt(g, w.q, w.nq);
        const bool ok = DIAQ_BOUNDS_OK(base + w.off[D - 1], int64_t(1) << n, BS_WINDOW);
        if (ok)
            for (int e = 0; e < D; ++e) cp[e * T] = psi[base + w.off[e]];
        if (rev && ok)
            for (int e = 0; e < D; ++e) cl[e * T] = lam[base + w.off[e]];
        if (!rev) {
            for (int i = 0; i < w.count; ++i) win_apply<R>(ops[i], cp, nullptr, D, T, nullptr);
        } else {
            for (int i = w.count - 1; i >= 0; --i) {
                const WinOp<R>& o = ops[i];
                win_apply<R>(o, cp, cl, D, T, o.j >= 0 ? sa + o.j * T + t : nullptr);
            }
        }
        if (ok)
            for (int e = 0; e < D; ++e) psi[base + w.off[e]] = cp[e * T];
        if (rev && ok)
            for (int e = 0; e < D; ++e) lam[base + w.off[e]] = cl[e * T];
    }
    if (rev) {
        for (int j = 0; j < w.np; ++j) {
            const double v = block_sum(sa[j * T + t].value(), warps);
            if (t == 0) part[int64_t(w.slot[j]) * P + blockIdx.x] = v;
        }
    }
}

}  // namespace diaq

struct diaq_adjoint_plan_s {
    int device = 0;
    int n = 0;
    diaq_dtype dtype = DIAQ_C128;
    int n_gates = 0, n_params = 0, n_terms = 0, n_slots = 1;
    int P = 1;  // blocks of the rotation and reduction kernels (partial columns)
    int P_gate = 1;  // P of the one-launch-per-gate sweep (window-fused sweeps size their own)
    std::vector<BGate> gates;
    std::vector<GateDesc> fwd, bwd;  // fixed gates: U and U^dag
    BGate* d_gates = nullptr;
    BTerm* d_terms = nullptr;
    void* d_ltab = nullptr;      // lambda weight tables (lambda_tables), plan precision
    int lflags = 0;              // LAM_* flags of the observable
    RotAngles* d_angles = nullptr;
    void* d_psi = nullptr;
    void* d_lam = nullptr;
    double* d_theta = nullptr;
    double* d_part = nullptr;
    double* d_rows = nullptr;
    double* d_out = nullptr;
    double* h_theta = nullptr;
    double* h_out = nullptr;
    const void* psi0 = nullptr;  // captured initial-state pointer (NULL: |0...0>)
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int window = 0;                  // 0: one launch per gate; else window-fused blocks of <= window qubits
    int lanes = 1;                   // threads per group of the window-fused kernel (1 or WIN_LANES)
    std::vector<WinBlock> blocks;
    WinGate* d_wg = nullptr;
    // diagonal runs of the per-gate sweep (window 0)
    bool runs_on = true;
    std::vector<int32_t> run_order;  // gate index, or -1 - run index
    std::vector<PhaseRun> runs;
    PhaseRun* d_runs = nullptr;
    double2* d_ptabs = nullptr;  // phase tables of the runs: (run, dir) at (2 run + dir) PR_TAB_ALL
    // scaled rotations of the per-gate complex128 sweep (rot_groups_s):
    // requested (default on); active when n_events > 0
    bool scaled = true;
    bool pairs = true;               // fuse consecutive one-qubit X/Y rotations (k_plan_rot2)
    int layer_len = 0;               // leading product layer of the per-gate sweep (from |0...0>)
    void* d_init = nullptr;          // its chunk tables (product_layer), plan precision
    FinTerm* d_fin = nullptr;        // gradient terms per parameter, in gate order
    int32_t* d_fin_first = nullptr;  // n_params + 1 offsets into d_fin
    ScaleEvent* d_events = nullptr;
    int n_events = 0;
    double* d_scale = nullptr;  // n_slots rescale factors
};


static void plan_free(diaq_adjoint_plan_s* p) {
    if (p->d_init) cudaFree(p->d_init);
    p->d_init = nullptr;
    if (p->d_ptabs) cudaFree(p->d_ptabs);
    p->d_ptabs = nullptr;
    if (p->d_fin) cudaFree(p->d_fin);
    p->d_fin = nullptr;
    if (p->d_fin_first) cudaFree(p->d_fin_first);
    p->d_fin_first = nullptr;
    if (p->d_events) cudaFree(p->d_events);
    p->d_events = nullptr;
    if (p->d_scale) cudaFree(p->d_scale);
    p->d_scale = nullptr;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->d_wg) cudaFree(p->d_wg);
    p->d_wg = nullptr;
    if (p->d_runs) cudaFree(p->d_runs);
    p->d_runs = nullptr;
    for (void* q : {static_cast<void*>(p->d_gates), static_cast<void*>(p->d_terms), static_cast<void*>(p->d_ltab),
                    static_cast<void*>(p->d_angles),
                    p->d_psi, p->d_lam, static_cast<void*>(p->d_theta), static_cast<void*>(p->d_part),
                    static_cast<void*>(p->d_rows), static_cast<void*>(p->d_out)})
        if (q) cudaFree(q);
    if (p->h_theta) cudaFreeHost(p->h_theta);
    if (p->h_out) cudaFreeHost(p->h_out);
    if (p->stream) cudaStreamDestroy(p->stream);
}

// Execution order of the per-gate sweep (gate index, or -1 - run index) and
// the position of its earliest entry with a gradient term (the reverse
// sweep stops there).
static void plan_order(const diaq_adjoint_plan_s* p, std::vector<int32_t>* order, size_t* stop) {
    order->clear();
    if (p->runs_on) {
        *order = p->run_order;
    } else {
        for (int g = 0; g < p->n_gates; ++g) order->push_back(g);
    }
    *stop = order->size();
    for (size_t oi = 0; oi < order->size(); ++oi)
        if ((*order)[oi] < 0 || p->gates[size_t((*order)[oi])].param >= 0) {
            *stop = oi;
            break;
        }
}

static int plan_rotation_applications(const diaq_adjoint_plan_s* p) {
    std::vector<int32_t> order;
    size_t stop = 0;
    plan_order(p, &order, &stop);
    int count = 0;
    for (size_t oi = 0; oi < order.size(); ++oi)
        if (order[oi] >= 0 && p->gates[size_t(order[oi])].param >= 0) count += oi >= stop ? 2 : 1;
    return count;
}

// Scale events of the scaled per-gate sweep, in sweep order (uploaded
// before the graph is recorded).
static diaq_status plan_scale_events(diaq_adjoint_plan_s* p) {
    if (p->d_events) cudaFree(p->d_events);
    p->d_events = nullptr;
    p->n_events = 0;
    if (!p->scaled || p->window > 0 || p->dtype != DIAQ_C128 ||
        plan_rotation_applications(p) > DIAQ_SCALED_MAX_ROT)
        return DIAQ_OK;
    std::vector<int32_t> order;
    size_t stop = 0;
    plan_order(p, &order, &stop);
    std::vector<ScaleEvent> ev;
    for (int32_t g : order)
        if (g >= 0 && p->gates[size_t(g)].param >= 0) ev.push_back({0, g});
    ev.push_back({1, 0});
    for (size_t oi = order.size(); oi-- > stop;) {
        const int32_t g = order[oi];
        if (g < 0) {
            const PhaseRun& r = p->runs[size_t(-1 - g)];
            for (int j = 0; j < r.n_rot; ++j) ev.push_back({2, r.rot_slot[j]});
            continue;
        }
        const BGate& G = p->gates[size_t(g)];
        if (G.param < 0) continue;
        ev.push_back({2, G.slot});
        ev.push_back({3, g});
    }
    if (!p->d_scale) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p->d_scale), sizeof(double) * size_t(p->n_slots));
        if (e != cudaSuccess) {
            p->d_scale = nullptr;
            return fail(DIAQ_ERR_ALLOC, "adjoint plan scales: %s", cudaGetErrorString(e));
        }
    }
    DIAQ_TRY(upload(&p->d_events, ev));
    p->n_events = int(ev.size());
    return DIAQ_OK;
}

// The leading product layer of the per-gate sweep when it starts from
// |0...0> (uploaded before the graph is recorded).
static diaq_status plan_product_layer(diaq_adjoint_plan_s* p) {
    if (p->d_init) cudaFree(p->d_init);
    p->d_init = nullptr;
    p->layer_len = 0;
    if (p->window > 0 || p->psi0) return DIAQ_OK;
    std::vector<int32_t> order;
    size_t stop = 0;
    plan_order(p, &order, &stop);
    std::vector<double2> tab;
    const int len = product_layer(p->gates.data(), order.data(), int(order.size()), p->n, &tab);
    if (len == 0) return DIAQ_OK;
    DIAQ_TRY(upload_amps(p->dtype, tab, &p->d_init));
    p->layer_len = len;
    return DIAQ_OK;
}

template <typename R>
static diaq_status plan_record(diaq_adjoint_plan_s* p) {
    using A = amp_t<R>;
    cudaStream_t s = p->stream;
    const int64_t N = int64_t(1) << p->n;
    A* psi = static_cast<A*>(p->d_psi);
    A* lam = static_cast<A*>(p->d_lam);
    DIAQ_CUDA(cudaMemcpyAsync(p->d_theta, p->h_theta, sizeof(double) * size_t(std::max(p->n_params, 1)),
                              cudaMemcpyHostToDevice, s));
    if (p->n_gates) k_plan_angles<<<(p->n_gates + 127) / 128, 128, 0, s>>>(p->d_gates, p->n_gates, p->d_theta, p->d_angles);
    k_plan_init<R><<<p->P, 256, 0, s>>>(static_cast<const A*>(p->psi0), psi, N,
                                        p->layer_len > 0 ? p->d_init : nullptr, p->n);
    DIAQ_CUDA(cudaGetLastError());
    if (p->window > 0) {
        auto block = [&](const WinBlock& w, A* l) {
            if (p->lanes > 1)
                k_plan_win_l<R><<<p->P, WIN_THREADS, win_smem_lanes(p->dtype, w.nq, w.count, w.np), s>>>(
                    psi, l, p->d_gates, p->d_angles, p->d_wg, w, p->n, p->d_part, p->P);
            else
                k_plan_win<R><<<p->P, WIN_THREADS, win_smem(p->dtype, w.nq, w.count, w.np), s>>>(
                    psi, l, p->d_gates, p->d_angles, p->d_wg, w, p->n, p->d_part, p->P);
        };
        for (const WinBlock& w : p->blocks) block(w, nullptr);
        k_plan_lambda<R><<<p->P, 256, 0, s>>>(psi, lam, p->d_terms, p->d_ltab, p->n_terms, N, p->d_part,
                                             p->lflags);
        for (size_t b = p->blocks.size(); b-- > 0;) block(p->blocks[b], lam);
        DIAQ_CUDA(cudaGetLastError());
    } else {
        std::vector<int32_t> order;
        size_t stop = 0;
        plan_order(p, &order, &stop);
        const bool scaled = p->scaled && p->n_events > 0;
        if (scaled)
            k_plan_scales<<<1, kScaleThreads, 0, s>>>(p->d_events, p->n_events, p->d_angles, p->n_slots,
                                                      p->d_scale);
        if (p->runs_on && !p->runs.empty())
            k_phase_tables<<<dim3(unsigned(p->runs.size()), 2), 256, 0, s>>>(p->d_runs, p->d_theta, p->n, PR_TAB_ALL,
                                                                              p->d_ptabs);
        auto pairable = [&](int32_t g1, int32_t g2) {
            return p->pairs && g1 >= 0 && g2 >= 0 && pair_gate(p->gates[size_t(g1)]) &&
                   pair_gate(p->gates[size_t(g2)]) && p->gates[size_t(g1)].t[0] != p->gates[size_t(g2)].t[0];
        };
        for (size_t oi = size_t(p->layer_len); oi < order.size(); ++oi) {  // the product layer is in psi already
            const int32_t g = order[oi];
            if (g < 0) {
                k_plan_phase<R, false><<<p->P, 256, 0, s>>>(psi, nullptr, p->d_runs + (-1 - g),
                                                            p->d_ptabs + int64_t(-1 - g) * 2 * PR_TAB_ALL, p->n,
                                                            nullptr, p->P);
                continue;
            }
            if (oi + 1 < order.size() && pairable(g, order[oi + 1])) {
                const int32_t g2 = order[oi + 1];
                launch_plan_rot2<R>(p->gates[size_t(g)], p->gates[size_t(g2)], psi, nullptr, p->d_gates + g,
                                    p->d_gates + g2, p->d_angles + g, p->d_angles + g2, p->n, nullptr, nullptr, p->P,
                                    scaled, s);
                ++oi;
                continue;
            }
            const BGate& G = p->gates[size_t(g)];
            if (G.param >= 0)
                launch_plan_rot<R>(G, psi, nullptr, p->d_gates + g, p->d_angles + g, p->n, nullptr, p->P, scaled, s);
            else
                DIAQ_TRY(launch_gate_local(p->n, p->dtype, p->fwd[size_t(g)], nullptr, psi, psi, s));
        }
        k_plan_lambda<R><<<p->P, 256, 0, s>>>(psi, lam, p->d_terms, p->d_ltab, p->n_terms, N, p->d_part,
                                             p->lflags);
        // nothing below the earliest parametric entry feeds a gradient term
        for (size_t oi = order.size(); oi-- > stop;) {
            const int32_t g = order[oi];
            if (g < 0) {
                const double2* tab = p->d_ptabs + (int64_t(-1 - g) * 2 + 1) * PR_TAB_ALL;
                if (p->runs[size_t(-1 - g)].kind == PR_CHUNKS)
                    k_plan_phase_rev_chunks<R><<<p->P, 256, 0, s>>>(psi, lam, p->d_runs + (-1 - g), tab, p->n,
                                                                     p->d_part, p->P);
                else
                    k_plan_phase<R, true><<<p->P, 256, 0, s>>>(psi, lam, p->d_runs + (-1 - g), tab, p->n, p->d_part,
                                                               p->P);
                continue;
            }
            if (oi > stop && pairable(order[oi - 1], g)) {  // the pair (order[oi - 1], g), undone as one
                const int32_t g1 = order[oi - 1];
                const BGate& G1 = p->gates[size_t(g1)];
                const BGate& G2 = p->gates[size_t(g)];
                launch_plan_rot2<R>(G1, G2, psi, lam, p->d_gates + g1, p->d_gates + g, p->d_angles + g1,
                                    p->d_angles + g, p->n, p->d_part + int64_t(G1.slot) * p->P,
                                    p->d_part + int64_t(G2.slot) * p->P, p->P, scaled, s);
                --oi;
                continue;
            }
            const BGate& G = p->gates[size_t(g)];
            if (G.param >= 0) {
                launch_plan_rot<R>(G, psi, lam, p->d_gates + g, p->d_angles + g, p->n,
                                   p->d_part + int64_t(G.slot) * p->P, p->P, scaled, s);
            } else {
                DIAQ_TRY(launch_adjoint_step(p->n, p->dtype, p->bwd[size_t(g)], nullptr, psi, lam, nullptr,
                                             adjoint_partials(p->n, p->dtype, G.k), s));
            }
        }
    }
    k_plan_rows<<<p->n_slots, 256, 0, s>>>(p->d_part, p->P, p->d_rows);
    k_plan_finish<<<std::max(1, (p->n_params + 255) / 256), 256, 0, s>>>(
        p->d_fin, p->d_fin_first, p->d_rows, (p->scaled && p->window == 0 && p->n_events > 0) ? p->d_scale : nullptr,
        p->n_params, p->d_out);
    DIAQ_CUDA(cudaGetLastError());
    DIAQ_CUDA(cudaMemcpyAsync(p->h_out, p->d_out, sizeof(double) * size_t(1 + p->n_params), cudaMemcpyDeviceToHost, s));
    return DIAQ_OK;
}

// Blocks of at most `window` qubits and WIN_MAXG gates from the
// commutation-aware planner; window 0 clears them.
static diaq_status plan_windows(diaq_adjoint_plan_s* p, int window, int lanes) {
    p->blocks.clear();
    if (p->d_wg) {
        cudaFree(p->d_wg);
        p->d_wg = nullptr;
    }
    p->window = window;
    p->lanes = window > 0 ? lanes : 1;
    int P = p->P_gate;
    std::vector<WinGate> wg;
    if (window > 0 && p->n_gates > 0) {
        DIAQ_TRY(make_windows(p->gates.data(), p->n_gates, 0, window, &p->blocks, &wg));
        DIAQ_TRY(upload(&p->d_wg, wg));
        // one group per thread for the widest block, at most 4 blocks per SM
        int wmax = 1, sms = 1;
        for (const WinBlock& w : p->blocks) wmax = std::max(wmax, w.nq);
        DIAQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
        const int64_t want = (int64_t(1) << (p->n - wmax)) / (WIN_THREADS / p->lanes);
        P = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 4)));
    }
    if (P != p->P) {  // the partial rows have P columns
        double* part = nullptr;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&part), sizeof(double) * size_t(p->n_slots) * size_t(P));
        if (e != cudaSuccess) return fail(DIAQ_ERR_ALLOC, "adjoint plan partials: %s", cudaGetErrorString(e));
        cudaFree(p->d_part);
        p->d_part = part;
        p->P = P;
    }
    if (window == 0 || p->n_gates == 0) return DIAQ_OK;
    size_t most = 0;
    for (const WinBlock& w : p->blocks)
        most = std::max(most, p->lanes > 1 ? win_smem_lanes(p->dtype, w.nq, w.count, w.np)
                                           : win_smem(p->dtype, w.nq, w.count, w.np));
    const void* fn = p->lanes > 1
        ? (p->dtype == DIAQ_C128 ? reinterpret_cast<const void*>(&k_plan_win_l<double>)
                                 : reinterpret_cast<const void*>(&k_plan_win_l<float>))
        : (p->dtype == DIAQ_C128 ? reinterpret_cast<const void*>(&k_plan_win<double>)
                                 : reinterpret_cast<const void*>(&k_plan_win<float>));
    DIAQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(most)));
    return DIAQ_OK;
}

static diaq_status plan_capture(diaq_adjoint_plan_s* p) {
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    DIAQ_TRY(plan_scale_events(p));
    DIAQ_TRY(plan_product_layer(p));
    DIAQ_CUDA(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    diaq_status st = p->dtype == DIAQ_C128 ? plan_record<double>(p) : plan_record<float>(p);
    cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
    if (st != DIAQ_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture(adjoint plan)");
    e = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(adjoint plan)");
    return DIAQ_OK;
}

extern "C" {

diaq_status diaq_adjoint_plan_create(const diaq_gate* gates, int32_t n_gates, int32_t n_params, int32_t n_terms,
                                     const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                                     int32_t n_qubits, diaq_dtype dtype, diaq_adjoint_plan_t* out) {
    clear_error();
    cudaGetLastError();
    if (!out) return fail(DIAQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 2 || n_qubits > DIAQ_MAX_QUBITS) return fail(DIAQ_ERR_ARG, "n_qubits = %d out of range", n_qubits);
    if (dtype != DIAQ_C64 && dtype != DIAQ_C128) return fail(DIAQ_ERR_ARG, "bad dtype %d", (int)dtype);
    if (n_gates < 0 || (n_gates && !gates) || n_params < 0 || n_terms < 0 ||
        (n_terms && (!xmask || !zmask || !coeff)))
        return fail(DIAQ_ERR_ARG, "bad gate, parameter or term arrays");
    diaq_adjoint_plan_s* p = new (std::nothrow) diaq_adjoint_plan_s();
    if (!p) return fail(DIAQ_ERR_ALLOC, "host allocation failed");
    p->n = n_qubits;
    p->dtype = dtype;
    p->n_gates = n_gates;
    p->n_params = n_params;
    p->fwd.resize(static_cast<size_t>(n_gates));
    p->bwd.resize(static_cast<size_t>(n_gates));
    diaq_status st = DIAQ_OK;
    std::vector<double> zero(static_cast<size_t>(std::max(n_params, 1)), 0.0);
    for (int gi = 0; gi < n_gates && st == DIAQ_OK; ++gi) {
        const diaq_gate& g = gates[gi];
        if (g.k < 1 || g.k > 2) {
            st = fail(DIAQ_ERR_UNSUPPORTED, "gate %d: the adjoint plan takes gates of 1 or 2 qubits", gi);
            break;
        }
        if (g.param >= n_params) {
            st = fail(DIAQ_ERR_ARG, "gate %d uses parameter %d >= n_params", gi, g.param);
            break;
        }
        GateDesc d;
        st = gate_desc_from(&g, n_qubits, zero.data(), &d);
        if (st != DIAQ_OK) break;
        BGate B = {};
        B.k = g.k;
        B.t[0] = g.targets[0];
        B.t[1] = g.k == 2 ? g.targets[1] : 0;
        B.param = g.param;
        B.scale = g.scale;
        B.slot = -1;
        if (g.param >= 0) {
            for (int q = 0; q < g.k; ++q) {
                const char c = g.gen[q];
                B.pauli[q] = (c == 'X' || c == 'x') ? 1 : (c == 'Y' || c == 'y') ? 2 : (c == 'Z' || c == 'z') ? 3 : 0;
            }
            fill_rot(&B);
            B.slot = p->n_slots++;
        } else {
            p->fwd[size_t(gi)] = d;
            // the device record carries the matrix for the window-fused sweep
            for (size_t e = 0; e < d.m.size() && e < 16; ++e) {
                B.re[e] = d.m[e].real();
                B.im[e] = d.m[e].imag();
            }
            GateDesc u = d;
            const int D = 1 << d.k;
            for (int r = 0; r < D; ++r)
                for (int c = 0; c < D; ++c) u.m[size_t(r * D + c)] = std::conj(d.m[size_t(c * D + r)]);
            p->bwd[size_t(gi)] = u;
        }
        p->gates.push_back(B);
    }
    std::vector<BTerm> terms;
    const uint64_t valid = n_qubits >= 64 ? ~uint64_t(0) : ((uint64_t(1) << n_qubits) - 1);
    for (int t = 0; t < n_terms && st == DIAQ_OK; ++t) {
        if ((xmask[t] & ~valid) || (zmask[t] & ~valid)) {
            st = fail(DIAQ_ERR_ARG, "Pauli term %d acts on a qubit >= n_qubits", t);
            break;
        }
        BTerm T = {};
        T.x = xmask[t];
        T.z = zmask[t];
        const int ny = __builtin_popcountll(xmask[t] & zmask[t]) & 3;
        double kr = coeff[2 * t], ki = 0.0;
        for (int r = 0; r < ny; ++r) {
            const double tr = -ki, ti = kr;
            kr = tr;
            ki = ti;
        }
        T.kr = kr;
        T.ki = ki;
        terms.push_back(T);
    }
    std::stable_sort(terms.begin(), terms.end(), [](const BTerm& u, const BTerm& v) { return u.x < v.x; });
    p->n_terms = n_terms;
    std::vector<double2> ltab;
    if (st == DIAQ_OK) p->lflags = lambda_tables(terms, 0, int(terms.size()), &ltab);
    cudaError_t e = cudaSuccess;
    if (st == DIAQ_OK && (e = cudaGetDevice(&p->device)) != cudaSuccess) st = cuda_fail(e, "cudaGetDevice");
    if (st == DIAQ_OK) {
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
        // one resident wave of the rotation kernels (about 2 blocks of 256
        // per SM at their register counts); each thread loops over groups
        const int64_t want = ((int64_t(1) << n_qubits) / 2 + 255) / 256;
        p->P = int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(sms) * 2)));
        p->P_gate = p->P;
    }
    const size_t ab = amp_bytes(dtype), N = size_t(1) << n_qubits;
    if (st == DIAQ_OK) st = upload(&p->d_gates, p->gates);
    if (st == DIAQ_OK) {
        // gradient terms grouped by parameter, each group in gate order
        std::vector<int32_t> first(size_t(n_params) + 1, 0);
        for (const BGate& G : p->gates)
            if (G.slot >= 0) ++first[size_t(G.param) + 1];
        for (int q = 0; q < n_params; ++q) first[size_t(q) + 1] += first[size_t(q)];
        const size_t n_fin = size_t(first[size_t(n_params)]);
        std::vector<FinTerm> fin(n_fin);
        std::vector<int32_t> fill(first.begin(), first.end() - 1);
        for (const BGate& G : p->gates)
            if (G.slot >= 0) fin[size_t(fill[size_t(G.param)]++)] = {G.slot, G.scale};
        st = upload(&p->d_fin_first, first);
        if (st == DIAQ_OK && !fin.empty()) st = upload(&p->d_fin, fin);
    }
    if (st == DIAQ_OK) {
        plan_phase_runs(p->gates.data(), n_gates, 0, true, &p->run_order, &p->runs);
        if (!p->runs.empty()) st = upload(&p->d_runs, p->runs);
        if (st == DIAQ_OK && !p->runs.empty()) {
            const size_t bytes = p->runs.size() * 2 * PR_TAB_ALL * sizeof(double2);
            if ((e = cudaMalloc(reinterpret_cast<void**>(&p->d_ptabs), bytes)) != cudaSuccess) {
                p->d_ptabs = nullptr;
                st = fail(DIAQ_ERR_ALLOC, "adjoint plan phase tables: %s", cudaGetErrorString(e));
            }
        }
    }
    if (st == DIAQ_OK) st = upload(&p->d_terms, terms);
    if (st == DIAQ_OK) st = upload_amps(dtype, ltab, &p->d_ltab);
    if (st == DIAQ_OK &&
        ((e = cudaMalloc(reinterpret_cast<void**>(&p->d_angles), sizeof(RotAngles) * size_t(std::max(n_gates, 1)))) != cudaSuccess ||
         (e = cudaMalloc(&p->d_psi, N * ab)) != cudaSuccess || (e = cudaMalloc(&p->d_lam, N * ab)) != cudaSuccess ||
         (e = cudaMalloc(reinterpret_cast<void**>(&p->d_theta), sizeof(double) * size_t(std::max(n_params, 1)))) != cudaSuccess ||
         (e = cudaMalloc(reinterpret_cast<void**>(&p->d_part), sizeof(double) * size_t(p->n_slots) * size_t(p->P))) != cudaSuccess ||
         (e = cudaMalloc(reinterpret_cast<void**>(&p->d_rows), sizeof(double) * size_t(p->n_slots))) != cudaSuccess ||
         (e = cudaMalloc(reinterpret_cast<void**>(&p->d_out), sizeof(double) * size_t(1 + n_params))) != cudaSuccess ||
         (e = cudaMallocHost(reinterpret_cast<void**>(&p->h_theta), sizeof(double) * size_t(std::max(n_params, 1)))) != cudaSuccess ||
         (e = cudaMallocHost(reinterpret_cast<void**>(&p->h_out), sizeof(double) * size_t(1 + n_params))) != cudaSuccess))
        st = fail(DIAQ_ERR_ALLOC, "adjoint plan buffers: %s", cudaGetErrorString(e));
    if (st == DIAQ_OK) {
        std::memset(p->h_theta, 0, sizeof(double) * size_t(std::max(n_params, 1)));
        if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess)
            st = cuda_fail(e, "cudaStreamCreate(adjoint plan)");
    }
    if (st == DIAQ_OK) st = plan_capture(p);
    if (st != DIAQ_OK) {
        plan_free(p);
        delete p;
        return st;
    }
    *out = p;
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_run(diaq_adjoint_plan_t p, const double* theta, const void* psi0, double* energy,
                                  double* grad, diaq_stream_t stream) {
    clear_error();
    cudaGetLastError();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (p->n_params > 0 && !theta) return fail(DIAQ_ERR_ARG, "theta is NULL");
    for (int i = 0; i < p->n_params; ++i)
        if (!std::isfinite(theta[i])) return fail(DIAQ_ERR_ARG, "theta[%d] is not finite", i);
    if (psi0 && (reinterpret_cast<uintptr_t>(psi0) & 15)) return fail(DIAQ_ERR_ARG, "psi0 must be 16-byte aligned");
    if (psi0 != p->psi0 || !p->exec) {  // the initial-state pointer is part of the graph
        p->psi0 = psi0;
        DIAQ_TRY(plan_capture(p));
    }
    if (p->n_params) std::memcpy(p->h_theta, theta, sizeof(double) * size_t(p->n_params));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev;
    DIAQ_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    DIAQ_CUDA(cudaEventRecord(ev, s));
    DIAQ_CUDA(cudaStreamWaitEvent(p->stream, ev, 0));
    DIAQ_CUDA(cudaGraphLaunch(p->exec, p->stream));
    DIAQ_CUDA(cudaEventRecord(ev, p->stream));
    DIAQ_CUDA(cudaStreamWaitEvent(s, ev, 0));
    DIAQ_CUDA(cudaEventSynchronize(ev));
    cudaEventDestroy(ev);
    if (energy) *energy = p->h_out[0];
    if (grad)
        for (int i = 0; i < p->n_params; ++i) grad[i] = p->h_out[1 + i];
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_set_window(diaq_adjoint_plan_t p, int32_t window) {
    return diaq_adjoint_plan_set_sweep(p, window, 1);
}

diaq_status diaq_adjoint_plan_set_sweep(diaq_adjoint_plan_t p, int32_t window, int32_t lanes) {
    clear_error();
    cudaGetLastError();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (window != 0 && (window < 2 || window > WIN_MAX))
        return fail(DIAQ_ERR_ARG, "window = %d: use 0 (one launch per gate) or 2..%d qubits", window, WIN_MAX);
    if (lanes != 1 && lanes != WIN_LANES)
        return fail(DIAQ_ERR_ARG, "lanes = %d: use 1 or %d threads per group", lanes, WIN_LANES);
    int dev = -1;
    DIAQ_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(DIAQ_ERR_ARG, "plan was created on device %d but device %d is current", p->device, dev);
    DIAQ_CUDA(cudaStreamSynchronize(p->stream));
    if (p->exec) {  // it uses the tables and partials replaced below
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    diaq_status st = plan_windows(p, window, lanes);
    if (st != DIAQ_OK) {
        plan_windows(p, 0, 1);
        plan_capture(p);
        return st;
    }
    return plan_capture(p);
}

diaq_status diaq_adjoint_plan_set_runs(diaq_adjoint_plan_t p, int32_t on) {
    clear_error();
    cudaGetLastError();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    int dev = -1;
    DIAQ_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(DIAQ_ERR_ARG, "plan was created on device %d but device %d is current", p->device, dev);
    DIAQ_CUDA(cudaStreamSynchronize(p->stream));
    p->runs_on = on != 0;
    return plan_capture(p);
}

diaq_status diaq_adjoint_plan_get_runs(diaq_adjoint_plan_t p, int32_t* on, int32_t* n_runs, int32_t* n_steps) {
    clear_error();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (on) *on = p->runs_on ? 1 : 0;
    if (n_runs) *n_runs = int32_t(p->runs.size());
    if (n_steps) *n_steps = p->runs_on ? int32_t(p->run_order.size()) : p->n_gates;
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_get_sweep(diaq_adjoint_plan_t p, int32_t* window, int32_t* lanes, int32_t* n_blocks) {
    clear_error();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (window) *window = p->window;
    if (lanes) *lanes = p->lanes;
    if (n_blocks)
        *n_blocks = p->window > 0 ? int32_t(p->blocks.size())
                                  : (p->runs_on ? int32_t(p->run_order.size()) : p->n_gates);
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_set_scaled(diaq_adjoint_plan_t p, int32_t on) {
    clear_error();
    cudaGetLastError();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    int dev = -1;
    DIAQ_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(DIAQ_ERR_ARG, "plan was created on device %d but device %d is current", p->device, dev);
    DIAQ_CUDA(cudaStreamSynchronize(p->stream));
    p->scaled = on != 0;
    return plan_capture(p);
}

diaq_status diaq_adjoint_plan_set_pairs(diaq_adjoint_plan_t p, int32_t on) {
    clear_error();
    cudaGetLastError();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    int dev = -1;
    DIAQ_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(DIAQ_ERR_ARG, "plan was created on device %d but device %d is current", p->device, dev);
    DIAQ_CUDA(cudaStreamSynchronize(p->stream));
    p->pairs = on != 0;
    return plan_capture(p);
}

diaq_status diaq_adjoint_plan_get_pairs(diaq_adjoint_plan_t p, int32_t* on) {
    clear_error();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (on) *on = p->pairs ? 1 : 0;
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_get_scaled(diaq_adjoint_plan_t p, int32_t* on, int32_t* active) {
    clear_error();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (on) *on = p->scaled ? 1 : 0;
    if (active) *active = p->n_events > 0 ? 1 : 0;
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_set_blocks(diaq_adjoint_plan_t p, int32_t blocks) {
    clear_error();
    cudaGetLastError();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (blocks < 0) return fail(DIAQ_ERR_ARG, "blocks = %d: use 0 (two per SM) or a positive count", blocks);
    int dev = -1;
    DIAQ_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(DIAQ_ERR_ARG, "plan was created on device %d but device %d is current", p->device, dev);
    int sms = 1;
    DIAQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    const int64_t want = ((int64_t(1) << p->n) / 2 + 255) / 256;  // one group of 2 amplitudes per thread
    const int64_t b = blocks == 0 ? int64_t(sms) * 2 : std::min<int64_t>(blocks, int64_t(sms) * 64);
    DIAQ_CUDA(cudaStreamSynchronize(p->stream));
    if (p->exec) {  // it uses the partials replaced below
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    p->P_gate = int(std::max<int64_t>(1, std::min<int64_t>(want, b)));
    diaq_status st = plan_windows(p, p->window, p->lanes);
    if (st != DIAQ_OK) {
        plan_windows(p, 0, 1);
        plan_capture(p);
        return st;
    }
    return plan_capture(p);
}

diaq_status diaq_adjoint_plan_get_blocks(diaq_adjoint_plan_t p, int32_t* blocks) {
    clear_error();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (blocks) *blocks = p->P_gate;
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_autotune(diaq_adjoint_plan_t p, const double* theta, int32_t reps,
                                       diaq_plan_tuning* report) {
    clear_error();
    cudaGetLastError();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (p->n_params > 0 && !theta) return fail(DIAQ_ERR_ARG, "theta is NULL");
    if (reps < 1) reps = 1;
    const int wins[] = {0, 3, 4, 5, 3, 4, 5};
    const int lns[] = {1, 1, 1, 1, WIN_LANES, WIN_LANES, WIN_LANES};
    int best_w = 0, best_l = 1, best_b = p->P_gate, tried = 0;
    float best = 1e30f;
    cudaEvent_t e0, e1;
    DIAQ_CUDA(cudaEventCreate(&e0));
    DIAQ_CUDA(cudaEventCreate(&e1));
    if (p->n_params) std::memcpy(p->h_theta, theta, sizeof(double) * size_t(p->n_params));
    // one warm replay, then `reps` timed; recorded in the report, kept if fastest
    auto measure = [&](int w, int ln, int blocks) -> diaq_status {
        DIAQ_CUDA(cudaGraphLaunch(p->exec, p->stream));
        DIAQ_CUDA(cudaEventRecord(e0, p->stream));
        for (int r = 0; r < reps; ++r) DIAQ_CUDA(cudaGraphLaunch(p->exec, p->stream));
        DIAQ_CUDA(cudaEventRecord(e1, p->stream));
        DIAQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        DIAQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms /= float(reps);
        if (report && tried < DIAQ_PLAN_TUNE_MAX) {
            report->window[tried] = w;
            report->lanes[tried] = ln;
            report->blocks[tried] = blocks;
            report->ms[tried] = ms;
        }
        ++tried;
        if (ms < best) {
            best = ms;
            best_w = w;
            best_l = ln;
            if (w == 0) best_b = blocks;
        }
        return DIAQ_OK;
    };
    diaq_status st = DIAQ_OK;
    for (int c = 0; c < 7 && st == DIAQ_OK; ++c) {
        const int w = wins[c], ln = lns[c];
        if (diaq_adjoint_plan_set_sweep(p, w, ln) != DIAQ_OK) {
            clear_error();
            cudaGetLastError();
            continue;  // this window does not fit the circuit
        }
        st = measure(w, ln, w == 0 ? p->P_gate : 0);
    }
    if (st == DIAQ_OK && tried && best_w == 0) {  // the per-gate sweep at more blocks per SM
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
        if ((st = diaq_adjoint_plan_set_sweep(p, 0, 1)) == DIAQ_OK) {
            int last = p->P_gate;
            for (int m : {1, 4}) {
                if ((st = diaq_adjoint_plan_set_blocks(p, sms * m)) != DIAQ_OK) break;
                if (p->P_gate == last) continue;  // clamped to the blocks already timed
                last = p->P_gate;
                if ((st = measure(0, 1, p->P_gate)) != DIAQ_OK) break;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != DIAQ_OK) return st;
    if (!tried) return fail(DIAQ_ERR_UNSUPPORTED, "no sweep fits");
    if (best_w == 0) {
        DIAQ_TRY(diaq_adjoint_plan_set_sweep(p, 0, 1));
        DIAQ_TRY(diaq_adjoint_plan_set_blocks(p, best_b));
    } else {
        DIAQ_TRY(diaq_adjoint_plan_set_sweep(p, best_w, best_l));
    }
    if (report) {
        report->n_tried = std::min(tried, DIAQ_PLAN_TUNE_MAX);
        report->best_window = best_w;
        report->best_lanes = best_l;
        report->best_blocks = best_w == 0 ? best_b : 0;
        report->best_ms = best;
    }
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_get_window(diaq_adjoint_plan_t p, int32_t* window, int32_t* n_blocks) {
    clear_error();
    if (!p) return fail(DIAQ_ERR_ARG, "plan is NULL");
    if (window) *window = p->window;
    if (n_blocks) *n_blocks = p->window > 0 ? int32_t(p->blocks.size()) : p->n_gates;
    return DIAQ_OK;
}

diaq_status diaq_adjoint_plan_destroy(diaq_adjoint_plan_t p) {
    clear_error();
    if (!p) return DIAQ_OK;
    cudaDeviceSynchronize();
    plan_free(p);
    delete p;
    return DIAQ_OK;
}

}  // extern "C"
