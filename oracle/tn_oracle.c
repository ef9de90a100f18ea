/*
 * Reference ("oracle") implementation of sliced tensor-network contraction for random-circuit
 * amplitudes.  TEST INFRASTRUCTURE ONLY: it is plain, slow, complex128 C that is meant to be
 * checked by eye against the paper's definitions.  Only the tests, the package smoke check and
 * the benchmark's CPU-baseline leg may load it; the GPU library never calls into it and shares
 * no source with it.
 *
 * What each routine follows:
 *   orc_einsum_pair     - the pairwise contraction of Sec. 2.4, Eq. (chap2_einsum):
 *                         C[gamma] = sum over delta of A[alpha] * B[beta], with
 *                         delta = (alpha n beta) minus the labels still needed.
 *   orc_contract        - Sec. 3.1 (path of pairs, the result keeps the first operand's id) and
 *                         Sec. 3.2 (slicing: the network is cut on bonds, each cut bond is fixed
 *                         to one value per sub-task, and the sub-task results are summed).
 *   orc_statevector     - the circuit model of Sec. 2.1, simulated by applying each gate's matrix
 *                         to the full 2^n state (a second, independent reference).
 *   orc_readout         - Eq. (lxeb_2) / Eq. (lxeb_as_l2): F_l = 2^N * sum_i p(x_i) / m - 1, with
 *                         p = |amplitude|^2; also sum p^2 for the ideal-sample XEB.
 *
 * All routines return 0 on success and a negative code on bad arguments.  Labels are small
 * non-negative integers < ORC_MAX_LABEL; the dimension of every label is given by label_dim[].
 * Tensors are row-major over their label list (the last label varies fastest).
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_MAX_RANK 64
#define ORC_MAX_LABEL 65536

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int64_t prod_dims(int rank, const int *labels, const int *label_dim) {
    int64_t s = 1;
    for (int i = 0; i < rank; ++i) s *= label_dim[labels[i]];
    return s;
}

/* Position of label l in list[0..n), or -1. */
static int find_label(int n, const int *list, int l) {
    for (int i = 0; i < n; ++i)
        if (list[i] == l) return i;
    return -1;
}

/*
 * Pairwise einsum, Sec. 2.4 Eq. (chap2_einsum).  The output labels lab_c are given by the
 * caller; every label of A or B that is absent from lab_c and present in both A and B is summed
 * (delta).  A label present in A, B and C is a batch (Hadamard-product) index.  A label present
 * in only one input and absent from C is summed over that input alone.
 * For every output multi-index gamma the sum over delta runs in increasing row-major order of
 * the summed labels (the first summed label varies slowest).
 */
int orc_einsum_pair(int rank_a, const int *lab_a, const cplx *A,
                    int rank_b, const int *lab_b, const cplx *B,
                    int rank_c, const int *lab_c, cplx *C,
                    const int *label_dim) {
    if (rank_a < 0 || rank_b < 0 || rank_c < 0 || rank_a > ORC_MAX_RANK ||
        rank_b > ORC_MAX_RANK || rank_c > ORC_MAX_RANK)
        return -1;
    /* summed labels: in A or B, not in C */
    int lab_s[2 * ORC_MAX_RANK];
    int rank_s = 0;
    for (int i = 0; i < rank_a; ++i)
        if (find_label(rank_c, lab_c, lab_a[i]) < 0 && find_label(rank_s, lab_s, lab_a[i]) < 0)
            lab_s[rank_s++] = lab_a[i];
    for (int i = 0; i < rank_b; ++i)
        if (find_label(rank_c, lab_c, lab_b[i]) < 0 && find_label(rank_s, lab_s, lab_b[i]) < 0)
            lab_s[rank_s++] = lab_b[i];
    /* every output label must come from A or B */
    for (int i = 0; i < rank_c; ++i)
        if (find_label(rank_a, lab_a, lab_c[i]) < 0 && find_label(rank_b, lab_b, lab_c[i]) < 0)
            return -2;

    /* The value of each input label is read from either the output multi-index or the summed
     * multi-index: src_x[i] = (0 -> output position, 1 -> summed position), pos_x[i]. */
    int src_a[ORC_MAX_RANK], pos_a[ORC_MAX_RANK], src_b[ORC_MAX_RANK], pos_b[ORC_MAX_RANK];
    for (int i = 0; i < rank_a; ++i) {
        int p = find_label(rank_c, lab_c, lab_a[i]);
        if (p >= 0) { src_a[i] = 0; pos_a[i] = p; }
        else { src_a[i] = 1; pos_a[i] = find_label(rank_s, lab_s, lab_a[i]); }
    }
    for (int i = 0; i < rank_b; ++i) {
        int p = find_label(rank_c, lab_c, lab_b[i]);
        if (p >= 0) { src_b[i] = 0; pos_b[i] = p; }
        else { src_b[i] = 1; pos_b[i] = find_label(rank_s, lab_s, lab_b[i]); }
    }
    const int64_t size_c = prod_dims(rank_c, lab_c, label_dim);
    const int64_t size_s = prod_dims(rank_s, lab_s, label_dim);

    #pragma omp parallel for schedule(static)
    for (int64_t ic = 0; ic < size_c; ++ic) {
        int vc[ORC_MAX_RANK], vs[2 * ORC_MAX_RANK];
        /* output multi-index of ic (row-major, last label fastest) */
        int64_t r = ic;
        for (int i = rank_c - 1; i >= 0; --i) {
            int d = label_dim[lab_c[i]];
            vc[i] = (int)(r % d);
            r /= d;
        }
        cplx acc = 0.0;
        for (int64_t is = 0; is < size_s; ++is) {
            int64_t q = is;
            for (int i = rank_s - 1; i >= 0; --i) {
                int d = label_dim[lab_s[i]];
                vs[i] = (int)(q % d);
                q /= d;
            }
            int64_t oa = 0, ob = 0;
            for (int i = 0; i < rank_a; ++i)
                oa = oa * label_dim[lab_a[i]] + (src_a[i] ? vs[pos_a[i]] : vc[pos_a[i]]);
            for (int i = 0; i < rank_b; ++i)
                ob = ob * label_dim[lab_b[i]] + (src_b[i] ? vs[pos_b[i]] : vc[pos_b[i]]);
            acc += A[oa] * B[ob];
        }
        C[ic] = acc;
    }
    return 0;
}

/* Sub-tensor of T (labels lab, rank r) with label `fix` held at value v; the result has the
 * remaining labels in the same order. */
static void fix_label(int r, const int *lab, const cplx *T, int fix, int v, const int *label_dim,
                      int *out_lab, cplx *out) {
    int p = find_label(r, lab, fix);
    int64_t inner = 1;
    for (int i = p + 1; i < r; ++i) inner *= label_dim[lab[i]];
    int d = label_dim[fix];
    int64_t outer = 1;
    for (int i = 0; i < p; ++i) outer *= label_dim[lab[i]];
    for (int64_t o = 0; o < outer; ++o)
        for (int64_t in = 0; in < inner; ++in)
            out[o * inner + in] = T[(o * d + v) * inner + in];
    int k = 0;
    for (int i = 0; i < r; ++i)
        if (i != p) out_lab[k++] = lab[i];
}

typedef struct {
    int rank;
    int lab[ORC_MAX_RANK];
    cplx *data;
    int alive;
} otensor;

/*
 * Sliced contraction along a path, Sec. 3.1-3.2.
 *   tensors i = 0..num_tensors-1 with ranks[i], labels[i][], data[i][] (row-major);
 *   open_labels[0..num_open) give the output order (first = most significant);
 *   path = pairs (a, b): tensor a becomes einsum(a, b) and b is retired (Sec. 3.1);
 *   sliced_labels[j] takes digit j of the slice id (digit 0 least significant, radix = its dim);
 *   out (prod of open dims) is OVERWRITTEN with the sum over slices [slice_begin, slice_end),
 *   taken in increasing slice order.
 * Intermediate labels: the labels of a then of b that a later tensor or the output still needs.
 */
int orc_contract(int num_tensors, const int *ranks, const int *const *labels,
                 const cplx *const *data, const int *label_dim, int num_labels,
                 int num_open, const int *open_labels, int path_len, const int *path,
                 int num_sliced, const int *sliced_labels, int64_t slice_begin,
                 int64_t slice_end, cplx *out) {
    if (num_tensors <= 0 || path_len != num_tensors - 1) return -1;
    for (int i = 0; i < num_tensors; ++i) {
        if (ranks[i] < 0 || ranks[i] > ORC_MAX_RANK) return -1;
        for (int k = 0; k < ranks[i]; ++k)
            if (labels[i][k] < 0 || labels[i][k] >= num_labels) return -1;
    }
    int64_t num_slices = 1;
    for (int j = 0; j < num_sliced; ++j) num_slices *= label_dim[sliced_labels[j]];
    if (slice_begin < 0 || slice_end > num_slices || slice_begin > slice_end) return -3;
    const int64_t out_size = prod_dims(num_open, open_labels, label_dim);
    for (int64_t i = 0; i < out_size; ++i) out[i] = 0.0;

    otensor *T = (otensor *)calloc((size_t)num_tensors, sizeof(otensor));
    int *uses = (int *)calloc((size_t)num_labels, sizeof(int));
    if (!T || !uses) { free(T); free(uses); return -4; }
    int rc = 0;

    for (int64_t sigma = slice_begin; sigma < slice_end && rc == 0; ++sigma) {
        /* bind the slice: every leaf loses its sliced labels, fixed to sigma's digits */
        int digit[ORC_MAX_RANK];
        int64_t rem = sigma;
        for (int j = 0; j < num_sliced; ++j) {
            int d = label_dim[sliced_labels[j]];
            digit[j] = (int)(rem % d);
            rem /= d;
        }
        for (int i = 0; i < num_tensors; ++i) {
            int r = ranks[i];
            int lab[ORC_MAX_RANK];
            memcpy(lab, labels[i], sizeof(int) * (size_t)r);
            int64_t sz = prod_dims(r, lab, label_dim);
            cplx *cur = (cplx *)malloc(sizeof(cplx) * (size_t)sz);
            memcpy(cur, data[i], sizeof(cplx) * (size_t)sz);
            for (int j = 0; j < num_sliced; ++j) {
                if (find_label(r, lab, sliced_labels[j]) < 0) continue;
                int nlab[ORC_MAX_RANK];
                cplx *nxt = (cplx *)malloc(sizeof(cplx) * (size_t)(sz / label_dim[sliced_labels[j]]));
                fix_label(r, lab, cur, sliced_labels[j], digit[j], label_dim, nlab, nxt);
                free(cur);
                cur = nxt;
                sz /= label_dim[sliced_labels[j]];
                r -= 1;
                memcpy(lab, nlab, sizeof(int) * (size_t)r);
            }
            T[i].rank = r;
            memcpy(T[i].lab, lab, sizeof(int) * (size_t)r);
            T[i].data = cur;
            T[i].alive = 1;
        }
        /* how many live tensors (plus the output) hold each label */
        memset(uses, 0, sizeof(int) * (size_t)num_labels);
        for (int i = 0; i < num_tensors; ++i)
            for (int k = 0; k < T[i].rank; ++k) uses[T[i].lab[k]]++;
        for (int k = 0; k < num_open; ++k) uses[open_labels[k]]++;

        for (int s = 0; s < path_len; ++s) {
            int a = path[2 * s], b = path[2 * s + 1];
            if (a < 0 || b < 0 || a >= num_tensors || b >= num_tensors || a == b ||
                !T[a].alive || !T[b].alive) { rc = -5; break; }
            /* result labels: a's then b's labels still needed after this step */
            int lc[2 * ORC_MAX_RANK], rcn = 0;
            for (int k = 0; k < T[a].rank; ++k) {
                int l = T[a].lab[k];
                int in_b = find_label(T[b].rank, T[b].lab, l) >= 0;
                int others = uses[l] - 1 - (in_b ? 1 : 0);
                if (others > 0 || !in_b) lc[rcn++] = l;
            }
            for (int k = 0; k < T[b].rank; ++k) {
                int l = T[b].lab[k];
                if (find_label(T[a].rank, T[a].lab, l) < 0) lc[rcn++] = l;
            }
            if (rcn > ORC_MAX_RANK) { rc = -6; break; }
            int64_t sz = prod_dims(rcn, lc, label_dim);
            cplx *C = (cplx *)malloc(sizeof(cplx) * (size_t)sz);
            if (!C) { rc = -4; break; }
            orc_einsum_pair(T[a].rank, T[a].lab, T[a].data, T[b].rank, T[b].lab, T[b].data,
                            rcn, lc, C, label_dim);
            /* update label use counts */
            for (int k = 0; k < T[a].rank; ++k) uses[T[a].lab[k]]--;
            for (int k = 0; k < T[b].rank; ++k) uses[T[b].lab[k]]--;
            for (int k = 0; k < rcn; ++k) uses[lc[k]]++;
            free(T[a].data);
            free(T[b].data);
            T[b].data = NULL;
            T[b].alive = 0;
            T[a].rank = rcn;
            memcpy(T[a].lab, lc, sizeof(int) * (size_t)rcn);
            T[a].data = C;
        }
        if (rc == 0) {
            int root = -1;
            for (int i = 0; i < num_tensors; ++i)
                if (T[i].alive) { root = i; break; }
            if (root < 0 || T[root].rank != num_open) rc = -7;
            else {
                /* permute the root into open_labels order and add it to out */
                int perm[ORC_MAX_RANK];
                for (int k = 0; k < num_open; ++k) {
                    perm[k] = find_label(T[root].rank, T[root].lab, open_labels[k]);
                    if (perm[k] < 0) rc = -7;
                }
                if (rc == 0) {
                    for (int64_t io = 0; io < out_size; ++io) {
                        int v[ORC_MAX_RANK];
                        int64_t r = io;
                        for (int k = num_open - 1; k >= 0; --k) {
                            int d = label_dim[open_labels[k]];
                            v[k] = (int)(r % d);
                            r /= d;
                        }
                        int vr[ORC_MAX_RANK];
                        for (int k = 0; k < num_open; ++k) vr[perm[k]] = v[k];
                        int64_t off = 0;
                        for (int k = 0; k < num_open; ++k)
                            off = off * label_dim[T[root].lab[k]] + vr[k];
                        out[io] += T[root].data[off];
                    }
                }
            }
        }
        for (int i = 0; i < num_tensors; ++i) {
            free(T[i].data);
            T[i].data = NULL;
            T[i].alive = 0;
        }
    }
    free(T);
    free(uses);
    return rc;
}

/*
 * State-vector simulation (Sec. 2.1 circuit model).  n qubits, qubit 0 is the most significant
 * bit of the basis index.  gate g acts on gate_nq[g] (1 or 2) qubits gate_q[2g], gate_q[2g+1];
 * its matrix is gate_m[16g ...] row-major (2x2 uses the first 4 entries; 4x4 rows/cols are
 * 2*bit(q_first) + bit(q_second)).  state is overwritten, starting from |0...0>.
 */
int orc_statevector(int n, int num_gates, const int *gate_nq, const int *gate_q,
                    const cplx *gate_m, cplx *state) {
    if (n <= 0 || n > 34) return -1;
    const int64_t dim = (int64_t)1 << n;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) state[i] = 0.0;
    state[0] = 1.0;
    for (int g = 0; g < num_gates; ++g) {
        const cplx *M = gate_m + 16 * g;
        if (gate_nq[g] == 1) {
            int q = gate_q[2 * g];
            if (q < 0 || q >= n) return -2;
            int64_t bit = (int64_t)1 << (n - 1 - q);
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < dim; ++i) {
                if (i & bit) continue;
                cplx x0 = state[i], x1 = state[i | bit];
                state[i] = M[0] * x0 + M[1] * x1;
                state[i | bit] = M[2] * x0 + M[3] * x1;
            }
        } else if (gate_nq[g] == 2) {
            int qa = gate_q[2 * g], qb = gate_q[2 * g + 1];
            if (qa < 0 || qa >= n || qb < 0 || qb >= n || qa == qb) return -2;
            int64_t ba = (int64_t)1 << (n - 1 - qa), bb = (int64_t)1 << (n - 1 - qb);
            #pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < dim; ++i) {
                if ((i & ba) || (i & bb)) continue;
                int64_t idx[4] = {i, i | bb, i | ba, i | ba | bb};
                cplx x[4], y[4];
                for (int r = 0; r < 4; ++r) x[r] = state[idx[r]];
                for (int r = 0; r < 4; ++r) {
                    y[r] = 0.0;
                    for (int c = 0; c < 4; ++c) y[r] += M[4 * r + c] * x[c];
                }
                for (int r = 0; r < 4; ++r) state[idx[r]] = y[r];
            }
        } else {
            return -3;
        }
    }
    return 0;
}

/*
 * Readout, Eq. (lxeb_2) and Eq. (lxeb_as_l2).  For m amplitudes of an n-qubit circuit:
 *   out[0] = sum p,  out[1] = sum p^2,  out[2] = F_l = 2^n * sum p / m - 1,
 *   out[3] = 2^n * sum p^2 / sum p - 1  (XEB of ideal samples drawn from these amplitudes),
 * with p = |a|^2, summed in index order.
 */
int orc_readout(int64_t m, const cplx *amps, int n_qubits, double *out) {
    if (m <= 0 || n_qubits < 0) return -1;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double p = creal(amps[i]) * creal(amps[i]) + cimag(amps[i]) * cimag(amps[i]);
        s1 += p;
        s2 += p * p;
    }
    double D = 1.0;
    for (int i = 0; i < n_qubits; ++i) D *= 2.0;
    out[0] = s1;
    out[1] = s2;
    out[2] = D * s1 / (double)m - 1.0;
    out[3] = (s1 > 0.0) ? D * s2 / s1 - 1.0 : 0.0;
    return 0;
}
