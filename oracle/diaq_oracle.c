/*
 * FP64 CPU oracle for the DiaQ gate-apply path (arXiv 2405.01250).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. It shares no code,
 * header, table or helper with the CUDA library; it computes every result
 * from its plain definition, slowly and obviously:
 *
 *   - a gate's action is the full-system operator of Section II-C,
 *     I_above (x) Gate (x) I_below, with the tensor factors placed on the
 *     gate's target bits, applied row by row;
 *   - a DiaQ matrix (Section IV) is a map  diagonal index -> diagonal values,
 *     where index d >= 0 holds A[t][t+d] and d < 0 holds A[t-d][t]
 *     (t = 0 .. N-|d|-1), the orientation of Algorithm 2;
 *   - a Pauli string acts on a basis state factor by factor.
 *
 * Complex numbers are interleaved (re, im) doubles. Built with
 * -ffp-contract=off so no multiply-add is fused.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Local row/column index of basis index i for a gate on targets t[0..k-1]:
 * bit (k-1-a) of the local index is bit t[a] of i (t[0] is the most
 * significant local bit). */
static int64_t local_index(int64_t i, int k, const int* t) {
    int64_t r = 0;
    for (int a = 0; a < k; ++a) r |= ((i >> t[a]) & 1) << (k - 1 - a);
    return r;
}

/* Basis index equal to i outside the targets and carrying local index c on
 * them. */
static int64_t with_local(int64_t i, int k, const int* t, int64_t c) {
    int64_t j = i;
    for (int a = 0; a < k; ++a) {
        int64_t bit = (c >> (k - 1 - a)) & 1;
        j = (j & ~((int64_t)1 << t[a])) | (bit << t[a]);
    }
    return j;
}

/*
 * y = (I_above (x) M (x) I_below) x, generalised to any target placement
 * (Section II-C): element (i, j) of the full-system operator is
 * M[local(i)][local(j)] when i and j agree outside the targets, else 0. For
 * each row i the oracle sums over the 2^k columns j that can be non-zero, in
 * ascending local column order. Out of place; y must not alias x.
 */
void oracle_apply_gate(int n, const double* x, double* y, int k, const int* t, const double* m) {
    const int64_t N = (int64_t)1 << n;
    const int64_t dim = (int64_t)1 << k;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const int64_t r = local_index(i, k, t);
        double acc_re = 0.0, acc_im = 0.0;
        for (int64_t c = 0; c < dim; ++c) {
            const int64_t j = with_local(i, k, t, c);
            const double a = m[2 * (r * dim + c)], b = m[2 * (r * dim + c) + 1];
            const double u = x[2 * j], v = x[2 * j + 1];
            acc_re += a * u - b * v;
            acc_im += a * v + b * u;
        }
        y[2 * i] = acc_re;
        y[2 * i + 1] = acc_im;
    }
}

/*
 * Full-system element A[i][j] of the gate operator above (0 when i and j
 * differ outside the targets). Writes (re, im) to out.
 */
static void gate_element(int64_t i, int64_t j, int k, const int* t, const double* m, double* out) {
    int64_t tmask = 0;
    for (int a = 0; a < k; ++a) tmask |= (int64_t)1 << t[a];
    if ((i & ~tmask) != (j & ~tmask)) { out[0] = 0.0; out[1] = 0.0; return; }
    const int64_t dim = (int64_t)1 << k;
    const int64_t r = local_index(i, k, t), c = local_index(j, k, t);
    out[0] = m[2 * (r * dim + c)];
    out[1] = m[2 * (r * dim + c) + 1];
}

/*
 * DiaQ form of a gate's full-system operator (Section IV): the sorted list of
 * diagonal indices d that hold at least one non-zero element, and for each
 * the N-|d| values A[t + max(0,-d)][t + max(0,d)], t = 0 .. N-|d|-1.
 *
 * Pass offsets == NULL to only count: returns the number of diagonals. With
 * offsets != NULL (capacity cap) fills them and returns the count. values, if
 * non-NULL, receives the diagonals back to back in offset order (interleaved
 * complex). Enumerates all N^2 elements: small n only.
 */
int64_t oracle_gate_diaq(int n, int k, const int* t, const double* m,
                         int64_t* offsets, int64_t cap, double* values) {
    const int64_t N = (int64_t)1 << n;
    char* present = (char*)calloc((size_t)(2 * N - 1), 1);
    if (!present) return -1;
    double e[2];
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            gate_element(i, j, k, t, m, e);
            if (e[0] != 0.0 || e[1] != 0.0) present[j - i + (N - 1)] = 1;
        }
    int64_t count = 0;
    for (int64_t d = -(N - 1); d <= N - 1; ++d) {
        if (!present[d + (N - 1)]) continue;
        if (offsets) {
            if (count >= cap) { free(present); return -2; }
            offsets[count] = d;
        }
        ++count;
    }
    if (offsets && values) {
        double* v = values;
        for (int64_t q = 0; q < count; ++q) {
            const int64_t d = offsets[q];
            const int64_t len = N - (d < 0 ? -d : d);
            const int64_t r0 = d < 0 ? -d : 0, c0 = d > 0 ? d : 0;
            for (int64_t s = 0; s < len; ++s) {
                gate_element(r0 + s, c0 + s, k, t, m, e);
                v[2 * s] = e[0];
                v[2 * s + 1] = e[1];
            }
            v += 2 * len;
        }
    }
    free(present);
    return count;
}

/*
 * DiaQ extraction from a dense N x N row-major complex matrix (Section IV,
 * the boxed example): same output contract as oracle_gate_diaq.
 */
int64_t oracle_dense_to_diaq(int64_t N, const double* a, int64_t* offsets, int64_t cap, double* values) {
    int64_t count = 0;
    for (int64_t d = -(N - 1); d <= N - 1; ++d) {
        const int64_t len = N - (d < 0 ? -d : d);
        const int64_t r0 = d < 0 ? -d : 0, c0 = d > 0 ? d : 0;
        int nz = 0;
        for (int64_t s = 0; s < len && !nz; ++s) {
            const int64_t idx = (r0 + s) * N + (c0 + s);
            if (a[2 * idx] != 0.0 || a[2 * idx + 1] != 0.0) nz = 1;
        }
        if (!nz) continue;
        if (offsets) {
            if (count >= cap) return -2;
            offsets[count] = d;
        }
        ++count;
    }
    if (offsets && values) {
        double* v = values;
        for (int64_t q = 0; q < count; ++q) {
            const int64_t d = offsets[q];
            const int64_t len = N - (d < 0 ? -d : d);
            const int64_t r0 = d < 0 ? -d : 0, c0 = d > 0 ? d : 0;
            for (int64_t s = 0; s < len; ++s) {
                const int64_t idx = (r0 + s) * N + (c0 + s);
                v[2 * s] = a[2 * idx];
                v[2 * s + 1] = a[2 * idx + 1];
            }
            v += 2 * len;
        }
    }
    return count;
}

/*
 * y = A x for A given in DiaQ form (Algorithm 2's result): by the definition
 * of a matrix-vector product, y[i] = sum over stored diagonals d of
 * A[i][i+d] * x[i+d] for the rows where column i+d exists. Diagonals are
 * visited in the order given. Out of place.
 */
void oracle_diaq_matvec(int64_t N, int64_t D, const int64_t* offsets, const double* values,
                        const double* x, double* y) {
    const double** base = (const double**)malloc(sizeof(double*) * (size_t)(D > 0 ? D : 1));
    const double* v = values;
    for (int64_t q = 0; q < D; ++q) {
        base[q] = v;
        v += 2 * (N - (offsets[q] < 0 ? -offsets[q] : offsets[q]));
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double acc_re = 0.0, acc_im = 0.0;
        for (int64_t q = 0; q < D; ++q) {
            const int64_t d = offsets[q];
            const int64_t j = i + d;
            if (j < 0 || j >= N) continue;
            /* A[i][i+d] sits at position min(i, j) of diagonal d */
            const int64_t s = i < j ? i : j;
            const double a = base[q][2 * s], b = base[q][2 * s + 1];
            const double u = x[2 * j], w = x[2 * j + 1];
            acc_re += a * u - b * w;
            acc_im += a * w + b * u;
        }
        y[2 * i] = acc_re;
        y[2 * i + 1] = acc_im;
    }
    free(base);
}

/*
 * Action of a Pauli string on a basis state, factor by factor: on qubit q,
 * X flips the bit, Z multiplies by -1 if the bit is 1, and Y maps |0> to
 * i|1> and |1> to -i|0>. The string is encoded by masks: bit q in xmask only
 * is X, in zmask only is Z, in both is Y. Returns the image index and writes
 * the phase (re, im).
 */
static int64_t pauli_on_basis(int n, int64_t j, uint64_t xm, uint64_t zm, double* ph) {
    double pr = 1.0, pi = 0.0;
    int64_t idx = j;
    for (int q = 0; q < n; ++q) {
        const int xb = (int)((xm >> q) & 1), zb = (int)((zm >> q) & 1);
        const int bit = (int)((j >> q) & 1);
        if (xb && !zb) {                 /* X */
            idx ^= (int64_t)1 << q;
        } else if (!xb && zb) {          /* Z */
            if (bit) { pr = -pr; pi = -pi; }
        } else if (xb && zb) {           /* Y */
            /* multiply by +i (bit 0) or -i (bit 1) */
            const double r = pr, im = pi;
            if (!bit) { pr = -im; pi = r; } else { pr = im; pi = -r; }
            idx ^= (int64_t)1 << q;
        }
    }
    ph[0] = pr;
    ph[1] = pi;
    return idx;
}

/*
 * <psi| sum_t c_t P_t |psi> with complex coefficients c_t: for every basis
 * state j, P|j> = phase * |idx>, so <psi|P|psi> = sum_j conj(psi[idx]) *
 * phase * psi[j]. Serial sums in index order (deterministic).
 * out[0], out[1] receive the real and imaginary parts.
 */
void oracle_expect(int n, const double* psi, int64_t n_terms, const uint64_t* xm, const uint64_t* zm,
                   const double* coeff, double* out) {
    const int64_t N = (int64_t)1 << n;
    double tot_re = 0.0, tot_im = 0.0;
    for (int64_t t = 0; t < n_terms; ++t) {
        double s_re = 0.0, s_im = 0.0, ph[2];
        for (int64_t j = 0; j < N; ++j) {
            const int64_t idx = pauli_on_basis(n, j, xm[t], zm[t], ph);
            /* phase * psi[j] */
            const double a = ph[0] * psi[2 * j] - ph[1] * psi[2 * j + 1];
            const double b = ph[0] * psi[2 * j + 1] + ph[1] * psi[2 * j];
            /* conj(psi[idx]) * (a + ib) */
            const double u = psi[2 * idx], v = psi[2 * idx + 1];
            s_re += u * a + v * b;
            s_im += u * b - v * a;
        }
        tot_re += coeff[2 * t] * s_re - coeff[2 * t + 1] * s_im;
        tot_im += coeff[2 * t] * s_im + coeff[2 * t + 1] * s_re;
    }
    out[0] = tot_re;
    out[1] = tot_im;
}

/* ||psi||^2 = sum_j |psi_j|^2, serial in index order. */
double oracle_norm2(int n, const double* psi) {
    const int64_t N = (int64_t)1 << n;
    double s = 0.0;
    for (int64_t j = 0; j < N; ++j) s += psi[2 * j] * psi[2 * j] + psi[2 * j + 1] * psi[2 * j + 1];
    return s;
}

/*
 * lambda = (sum_t c_t P_t) psi, by linearity term by term: each P_t sends the
 * component psi[j] |j> to phase * psi[j] |idx>. Terms are accumulated in
 * order. lambda must not alias psi.
 */
void oracle_apply_pauli_sum(int n, const double* psi, int64_t n_terms, const uint64_t* xm,
                            const uint64_t* zm, const double* coeff, double* lam) {
    const int64_t N = (int64_t)1 << n;
    memset(lam, 0, sizeof(double) * 2 * (size_t)N);
    for (int64_t t = 0; t < n_terms; ++t) {
        double ph[2];
        for (int64_t j = 0; j < N; ++j) {
            const int64_t idx = pauli_on_basis(n, j, xm[t], zm[t], ph);
            const double cr = coeff[2 * t] * ph[0] - coeff[2 * t + 1] * ph[1];
            const double ci = coeff[2 * t] * ph[1] + coeff[2 * t + 1] * ph[0];
            lam[2 * idx] += cr * psi[2 * j] - ci * psi[2 * j + 1];
            lam[2 * idx + 1] += cr * psi[2 * j + 1] + ci * psi[2 * j];
        }
    }
}

/*
 * Shots: Born-rule sampling of basis states, the measurement behind a run's
 * shots (Section VII runs every benchmark for 1024 shots). Basis state i is
 * drawn with probability |psi_i|^2 / sum_j |psi_j|^2, by the inverse of the
 * cumulative distribution in index order:
 *
 *   cdf_i = sum_{j <= i} |psi_j|^2, summed in index order, with
 *           |psi_j|^2 = re*re + im*im;
 *   r     = u * cdf_{N-1} for the shot's uniform u (clamped to [0, 1]);
 *   outcome = the smallest i with cdf_i > r, or, when no cdf_i exceeds r
 *             (u = 1), the largest i with |psi_i|^2 > 0; -1 when the state
 *             has zero norm.
 *
 * cdf is non-decreasing, so the smallest such i is found by bisection.
 */
void oracle_cdf(int n, const double* psi, double* cdf) {
    const int64_t N = (int64_t)1 << n;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        const double p = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
        s = s + p;
        cdf[i] = s;
    }
}

void oracle_sample(int n, const double* psi, int64_t shots, const double* u, int64_t* out) {
    const int64_t N = (int64_t)1 << n;
    double* cdf = (double*)malloc(sizeof(double) * (size_t)N);
    if (!cdf) {
        for (int64_t s = 0; s < shots; ++s) out[s] = -2;
        return;
    }
    oracle_cdf(n, psi, cdf);
    const double total = cdf[N - 1];
    int64_t last_pos = -1;
    for (int64_t i = N - 1; i >= 0; --i) {
        const double prev = i ? cdf[i - 1] : 0.0;
        if (cdf[i] > prev) {
            last_pos = i;
            break;
        }
    }
    for (int64_t s = 0; s < shots; ++s) {
        double v = u[s];
        if (!(v > 0.0)) v = 0.0; /* also maps NaN to 0 */
        if (v > 1.0) v = 1.0;
        const double r = v * total;
        if (!(total > 0.0)) {
            out[s] = -1;
            continue;
        }
        if (!(cdf[N - 1] > r)) {
            out[s] = last_pos;
            continue;
        }
        int64_t lo = 0, hi = N - 1; /* invariant: cdf[hi] > r */
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > r)
                hi = mid;
            else
                lo = mid + 1;
        }
        out[s] = lo;
    }
    free(cdf);
}
