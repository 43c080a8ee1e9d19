// Diagonal runs of the adjoint sweep. Z-type rotations exp(-i a/2 Z_g)
// (a generator of I and Z letters) and fixed diagonal gates hold their
// values on the principal diagonal (Section III-A), so a run of them is one
// diagonal operator, the product of their diagonals (what Algorithm 1's
// product of such DiaQ matrices gives), applied in one pass:
//   psi_i <- exp(-i sum_g a_g z_g(i) / 2) d(i) psi_i,
// z_g(i) = (-1)^popc(i & Z_g), d(i) the fixed gates' product. Every gate of
// the run commutes with every other and with each generator Z_g, so the
// gradient term of rotation g at its own position equals the one at the end
// of the run: Im <lambda|Z_g|psi> = sum_i z_g(i) Im(conj(lambda_i) psi_i),
// with the same Im(conj(lambda_i) psi_i) for every member.
//
// Two forms, chosen on the host:
//  * weight (PR_WEIGHT): every rotation shares one parameter and scale and
//    there is no fixed gate (a QAOA cost layer): the phase depends only on
//    the integer W(i) = sum_g z_g(i) in [-T, T], looked up in a table of
//    2T + 1 entries; the run's gradient term is sum_i W(i) t_i.
//  * chunks (PR_CHUNKS): every rotation acts on one qubit, fixed gates are
//    single-qubit diagonals or CZs (an ansatz layer's RZs and CZ ladder):
//    the phase is a product of one table entry per 8 qubits of i (the
//    factors of the qubits in that byte) and the CZ sign; the gradient term
//    of a rotation on qubit q is sum_i (-1)^(bit q of i) t_i.
// Tables are built per block in shared memory from theta on the device, so
// a recorded graph serves every theta.
#pragma once

#include "common.cuh"
#include "rot.cuh"

namespace diaq {

constexpr int PR_WEIGHT = 1;
constexpr int PR_CHUNKS = 2;
constexpr int PR_MAX_ROT = 48;     // rotations per run (weight form)
constexpr int PR_MAX_CROT = 24;    // rotations per run (chunk form: one accumulator each)
constexpr int PR_MAX_CZ = 64;
constexpr int PR_MAX_FIX1 = 16;
constexpr int PR_CHUNK_BITS = 8;
constexpr int PR_MAX_CHUNKS = (DIAQ_MAX_QUBITS + PR_CHUNK_BITS - 1) / PR_CHUNK_BITS;

struct PhaseRun {
    int32_t kind;                   // PR_WEIGHT or PR_CHUNKS
    int32_t n_rot;
    int32_t rot_param[PR_MAX_ROT];  // parameter index (instance-relative)
    double rot_scale[PR_MAX_ROT];   // a_g = scale * theta[param]
    uint64_t rot_z[PR_MAX_ROT];     // Z mask (chunk form: one bit)
    int32_t rot_slot[PR_MAX_ROT];   // gradient row (weight form: rot_slot[0] for the run)
    int32_t n_cz;
    int32_t n_cz_in;                // chunk form: cz[0 .. n_cz_in) lie inside one chunk (folded into its table)
    int32_t param_base;             // first parameter of the run's circuit in the theta array
    uint64_t cz[PR_MAX_CZ];         // the two bits of each CZ
    int32_t n_fix1;
    int32_t fix1_q[PR_MAX_FIX1];    // qubit of a fixed single-qubit diagonal gate
    double fix1_re[2 * PR_MAX_FIX1], fix1_im[2 * PR_MAX_FIX1];  // its entries for bit 0 and bit 1
    // weight form: the Z masks with bits 5..7 cleared, grouped by those three
    // bits (class k = bits 5..7 of the mask): class k at wz[wcls[k] .. wcls[k + 1])
    uint64_t wz[PR_MAX_ROT];
    int32_t wcls[9];
};

// Weight-form class table of a run (host): rot_z grouped by bits 5..7.
inline void phase_run_classes(PhaseRun* r) {
    int at = 0;
    for (int k = 0; k < 8; ++k) {
        r->wcls[k] = at;
        for (int g = 0; g < r->n_rot && g < PR_MAX_ROT; ++g)
            if (int((r->rot_z[g] >> 5) & 7) == k) r->wz[at++] = r->rot_z[g] & ~uint64_t(0xE0);
    }
    r->wcls[8] = at;
}

// Shared-memory tables of one run and direction: weight form entry W + T;
// chunk form entry c * 256 + v. E entries: PR_TAB_WEIGHT holds the weight
// form only, PR_TAB_ALL both forms.
constexpr int PR_TAB_WEIGHT = 2 * PR_MAX_ROT + 1;
constexpr int PR_TAB_ALL = PR_MAX_CHUNKS * 256;

// Stored in the state's precision: a complex64 sweep then converts no table
// entry per amplitude (a double-to-float conversion takes an FP64 pipe slot).
template <int E, typename T = double>
struct PhaseTables {
    T re[E];
    T im[E];
};

// Entry e of a run's table for one direction (rev: U^dag), from the
// parameters theta (the run's circuit's first parameter at theta[0]):
// weight form W + T = e; chunk form e = c * 256 + v, the product of the
// factors of the qubits in chunk c for the byte value v, times the signs
// of the CZs inside that chunk (cz[0 .. n_cz_in)).
__device__ __forceinline__ double2 phase_entry(const PhaseRun& r, const double* theta, bool rev, int e) {
    const double sg = rev ? 1.0 : -1.0;  // U = exp(-i a/2 ...), U^dag = exp(+i a/2 ...)
    double s, c;
    if (r.kind == PR_WEIGHT) {
        const double a = r.rot_scale[0] * theta[r.rot_param[0]];
        sincos(sg * 0.5 * a * double(e - r.n_rot), &s, &c);
        return make_double2(c, s);
    }
    const int ch = e >> 8, v = e & 255;
    double ang = 0.0;
    for (int g = 0; g < r.n_rot; ++g) {
        const int q = __ffsll((long long)r.rot_z[g]) - 1;
        if ((q >> 3) != ch) continue;
        const double z = ((v >> (q & 7)) & 1) ? -1.0 : 1.0;
        ang += 0.5 * r.rot_scale[g] * theta[r.rot_param[g]] * z;
    }
    sincos(sg * ang, &s, &c);
    double xr = c, xi = s;
    for (int f = 0; f < r.n_fix1; ++f) {
        const int q = r.fix1_q[f];
        if ((q >> 3) != ch) continue;
        const int b = (v >> (q & 7)) & 1;
        const double dr = r.fix1_re[2 * f + b], di = rev ? -r.fix1_im[2 * f + b] : r.fix1_im[2 * f + b];
        const double tr = xr * dr - xi * di;
        xi = xr * di + xi * dr;
        xr = tr;
    }
    int neg = 0;
    const uint64_t full = uint64_t(v) << (8 * ch);
    for (int k = 0; k < r.n_cz_in; ++k) neg ^= __popcll(full & r.cz[k]) == 2;
    return neg ? make_double2(-xr, -xi) : make_double2(xr, xi);
}

// Entries of a run's table: weight form 2T + 1, chunk form chunks x 256.
__host__ __device__ __forceinline__ int phase_entries(const PhaseRun& r, int n) {
    return r.kind == PR_WEIGHT ? 2 * r.n_rot + 1 : ((n + PR_CHUNK_BITS - 1) / PR_CHUNK_BITS) * 256;
}

// Copy a run's table, built once per replay in global memory, into the
// block's shared tables (all threads take part; synchronises).
template <int E, typename T>
__device__ __forceinline__ void phase_tables_load(const double2* __restrict__ src, int entries,
                                                  PhaseTables<E, T>* tb) {
    for (int e = threadIdx.x; e < entries && e < E; e += blockDim.x) {
        const double2 v = src[e];
        tb->re[e] = T(v.x);
        tb->im[e] = T(v.y);
    }
    __syncthreads();
}

// The sign of the CZs across chunks (those inside one chunk are in its
// table) for the aligned block of 256 amplitudes at base: a CZ on two bits
// at or above bit 8 gives the same sign to the whole block (*bneg); one with
// its low bit a below 8 flips the sign of the amplitudes with bit a set when
// its high bit is set in base, so the sign of amplitude base + lo is
// *bneg ^ parity(lo & *lmask).
__device__ __forceinline__ void phase_cz_block(const PhaseRun& r, uint64_t base, int* bneg, unsigned* lmask) {
    int b = 0;
    unsigned m = 0;
    for (int k = r.n_cz_in; k < r.n_cz; ++k) {
        const uint64_t cz = r.cz[k];
        const unsigned low = unsigned(cz & 255u);
        if (low == 0) b ^= __popcll(base & cz) == 2;
        else if (base & cz) m ^= low;
    }
    *bneg = b;
    *lmask = m;
}

template <typename R>
__device__ __forceinline__ amp_t<R> cmul(amp_t<R> a, amp_t<R> b) {
    amp_t<R> o;
    o.x = fma(a.x, b.x, -a.y * b.y);
    o.y = fma(a.x, b.y, a.y * b.x);
    return o;
}

// One run over a grid-stride share of the state. Forward
// (lam == nullptr): psi <- D psi. Reverse: the gradient terms first, then
// psi <- D^dag psi, lam <- D^dag lam (tables built for the direction).
// FORM (PR_WEIGHT or PR_CHUNKS) is the run's form, fixed at compile time so
// that no FP64 work of the other form is issued predicated off. Gradient
// terms go to acc[]: weight form acc[0] (the run's sum sum_i W(i) t_i);
// chunk form one per rotation.
// Both forms take aligned blocks of 256 amplitudes: warp w of the grid
// (nth / 32 warps; nth must be a multiple of 32) takes blocks w,
// w + nth / 32, ..., its lane l the amplitudes l + 32 j (j = 0..7) of each.
// The chunk form then forms the product of the higher chunks' table entries
// (shared by the block) once per block and lane instead of once per
// amplitude; the weight form its eight weights W as below.
// V: amplitudes whose loads are in flight together (fewer where the caller
// has fewer registers to spare).
template <typename R, int FORM, int E, int V = (sizeof(R) == 4 ? 8 : 4)>
__device__ __noinline__ void phase_run_sweep(amp_t<R>* __restrict__ psi, amp_t<R>* __restrict__ lam, int n,
                                             const PhaseRun& r, const PhaseTables<E, R>& tb, int64_t tid, int64_t nth,
                                             double* acc) {
    using A = amp_t<R>;
    constexpr bool CH = FORM == PR_CHUNKS;
    const int64_t N = int64_t(1) << n;
    Acc<R> a_w;
    Acc<R> a_c[CH ? PR_MAX_CROT : 1];
    // amplitude i (values p, l) with its phase ph (w: the weight-form W(i))
    auto finish = [&](int64_t i, A ph, int w, const A& p, const A& l) {
        if (lam) {
            const R t = fma(l.x, p.y, -l.y * p.x);  // Im(conj(l) p)
            if (!CH) {
                if constexpr (sizeof(R) == 8) {
                    a_w.s = fma(double(w), t, a_w.s);
                } else {
                    a_w.add(R(w) * t);
                }
            } else {
#pragma unroll
                for (int g = 0; g < (CH ? PR_MAX_CROT : 1); ++g) {
                    if (g >= r.n_rot) break;
                    a_c[g].add(flip_sign(t, (uint64_t(i) & r.rot_z[g]) ? 0x80000000u : 0u));
                }
            }
            lam[i] = cmul<R>(ph, l);
        }
        psi[i] = cmul<R>(ph, p);
    };
    // the eight amplitudes l + 32 j of a block; phase(j, &ph, &w) gives each
    // one's phase. In a whole block (n >= 8) the loads of V amplitudes are
    // issued before any of them is used, so their latencies overlap.
    const int lane = int(tid & 31);
    auto block8 = [&](int64_t base, auto&& phase) {
        if (base + 256 <= N) {
#pragma unroll
            for (int j0 = 0; j0 < 8; j0 += V) {
                A p[V], l[V];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int64_t i = base + lane + 32 * (j0 + v);
                    p[v] = psi[i];
                    if (lam) l[v] = lam[i];
                }
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    A ph;
                    int w;
                    phase(j0 + v, &ph, &w);
                    finish(base + lane + 32 * (j0 + v), ph, w, p[v], l[v]);
                }
            }
        } else {
            for (int j = 0; j < 8; ++j) {
                const int64_t i = base + lane + 32 * j;
                if (i >= N) break;  // n < 8 only
                A ph;
                int w;
                phase(j, &ph, &w);
                A l = {};
                if (lam) l = lam[i];
                finish(i, ph, w, psi[i], l);
            }
        }
    };
    const int64_t nblk = (N + 255) >> 8;
    if constexpr (!CH) {
        // W(i) = sum_g (-1)^popc(i & z_g). With i = x + 32 j (x = base | lane,
        // bits 5..7 clear) the sign of rotation g is (-1)^popc(x & z'_g) times
        // (-1)^popc(j & k_g), k_g = bits 5..7 of z_g, z'_g = z_g without them.
        // So the eight W of a block and lane are the Walsh-Hadamard transform
        // over j of C_k = sum over class k of (-1)^popc(x & z'_g): one pass
        // over the rotations per 8 amplitudes instead of one per amplitude.
        for (int64_t blk = tid >> 5; blk < nblk; blk += nth >> 5) {
            const int64_t base = blk << 8;
            const uint64_t x = uint64_t(base) | uint64_t(lane);
            int C[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int odd = 0;
                const int g0 = r.wcls[k], g1 = r.wcls[k + 1];
                for (int g = g0; g < g1; ++g) odd += __popcll(x & r.wz[g]) & 1;
                C[k] = (g1 - g0) - 2 * odd;
            }
#pragma unroll
            for (int h = 1; h < 8; h <<= 1)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (!(k & h)) {
                        const int a = C[k], b = C[k + h];
                        C[k] = a + b;
                        C[k + h] = a - b;
                    }
            block8(base, [&](int j, A* ph, int* w) {
                *w = C[j];
                ph->x = tb.re[C[j] + r.n_rot];
                ph->y = tb.im[C[j] + r.n_rot];
            });
        }
        acc[0] = a_w.value();
    } else {
        const int chunks = (n + PR_CHUNK_BITS - 1) / PR_CHUNK_BITS;
        for (int64_t blk = tid >> 5; blk < nblk; blk += nth >> 5) {
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
            phase_cz_block(r, uint64_t(base), &bneg, &lmask);
            block8(base, [&](int j, A* ph, int* w) {
                const int lo = lane + 32 * j;
                R pr = tb.re[lo], pi = tb.im[lo];
                if (chunks > 1) {
                    const R tr = fma(pr, hr, -pi * hi);
                    pi = fma(pr, hi, pi * hr);
                    pr = tr;
                }
                const int neg = bneg ^ (__popc(unsigned(lo) & lmask) & 1);
                const unsigned m = neg ? 0x80000000u : 0u;  // the sign by an integer flip
                ph->x = flip_sign(pr, m);
                ph->y = flip_sign(pi, m);
                *w = 0;
            });
        }
        for (int g = 0; g < r.n_rot && g < PR_MAX_CROT; ++g) acc[g] = a_c[g].value();
    }
}

}  // namespace diaq
