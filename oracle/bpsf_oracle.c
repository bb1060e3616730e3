/*
 * BP-SF oracle: a plain, slow, deliberately obvious CPU implementation of the
 * decoder in "Fully Parallelized BP Decoding for Quantum LDPC Codes Can
 * Outperform BP-OSD" (Wang, Li, Mueller; arXiv 2507.00254).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the yardstick the CUDA decoder is
 * measured against.  Only the tests, the smoke check and the bench's CPU
 * baseline may load it; the decoder library never does, and the two share no
 * code, header, table or helper.
 *
 * Everything works on dense 0/1 matrices (uint8, row-major) and unpacked
 * 0/1 vectors.  No blocking, fusion or reordering beyond what the paper's
 * definitions state.  Build with -O2 -ffp-contract=off (never -ffast-math):
 * the FP32 mode relies on every add and multiply being rounded on its own.
 *
 * Readings of points the paper leaves open (all applied identically in the
 * FP64 and FP32 modes):
 *   - sign(x) is negative iff x < 0 (both zeros count as positive);
 *   - the V2C sum and the posterior sum are left folds that start at the
 *     channel LLR and add the C2V messages in ascending check index;
 *   - the normalised magnitude is one multiply alpha * min, then the sign;
 *   - damping: alpha > 0 is fixed; alpha == 0 selects the adaptive factor
 *     alpha_t = 1 - 2^-t at iteration t = 1, 2, ... of each run (the paper
 *     prints it garbled as "1 - 2^i", i the iteration), computed in double
 *     and rounded once to the mode's type;
 *   - C2V magnitudes are clamped at 2^100.  With a fixed alpha <= 1/(dv-1)
 *     messages grow at most geometrically by alpha*(dv-1) and never get
 *     near it at the workloads; with alpha_t -> 1 the clamp keeps them finite;
 *   - hard decision: e_i = 1 iff l_out_i <= 0 (Section II-B, step 4);
 *   - oscillation counters start at zero with e_prev = 0 and are updated in
 *     every iteration of the initial run (Algorithm 1);
 *   - top(|Phi|) orders bits by (flip count descending, index ascending);
 *   - trial vectors are the non-empty subsets of Phi with weight <= w_max,
 *     visited in ascending subset mask (bit j of the mask selects Phi[j]),
 *     or an explicit list of masks in list order (the sampled variant);
 *   - selection: minimum Hamming weight of the returned e xor t, ties to the
 *     earlier trial of the list (select = 0), or the earliest converged trial
 *     of the list (select = 1);
 *   - on total failure the initial run's e is returned with converged = 0.
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* GF(2) dense matrices (Appendix "Code Construction")                        */
/* ------------------------------------------------------------------------ */

/* C = A * B over GF(2); A is r x k, B is k x c. */
static void gf2_matmul(const uint8_t *A, const uint8_t *B, uint8_t *C, int r, int k, int c) {
    for (int i = 0; i < r; i++)
        for (int j = 0; j < c; j++) {
            int acc = 0;
            for (int t = 0; t < k; t++) acc ^= (A[i * k + t] & B[t * c + j]);
            C[i * c + j] = (uint8_t)acc;
        }
}

static void identity(uint8_t *I, int n) {
    memset(I, 0, (size_t)n * n);
    for (int i = 0; i < n; i++) I[i * n + i] = 1;
}

/* S_l = I_l >> 1: every row of the identity cyclically shifted right by one. */
void oracle_shift_matrix(int l, uint8_t *S) {
    uint8_t *I = malloc((size_t)l * l);
    identity(I, l);
    for (int r = 0; r < l; r++)
        for (int c = 0; c < l; c++) S[r * l + (c + 1) % l] = I[r * l + c];
    free(I);
}

/* P = M^e over GF(2) by repeated multiplication (M is n x n). */
static void gf2_power(const uint8_t *M, int n, int e, uint8_t *P) {
    uint8_t *T = malloc((size_t)n * n);
    identity(P, n);
    for (int i = 0; i < e; i++) {
        gf2_matmul(P, M, T, n, n, n);
        memcpy(P, T, (size_t)n * n);
    }
    free(T);
}

/* K = A (x) B (Kronecker product), A is a x a, B is b x b. */
static void kron(const uint8_t *A, int a, const uint8_t *B, int b, uint8_t *K) {
    int n = a * b;
    for (int i = 0; i < a; i++)
        for (int j = 0; j < a; j++)
            for (int u = 0; u < b; u++)
                for (int v = 0; v < b; v++)
                    K[(i * b + u) * n + (j * b + v)] = (uint8_t)(A[i * a + j] & B[u * b + v]);
}

/* Polynomial sum_t x^{px[t]} y^{py[t]} with x = S_l (x) I_m, y = I_l (x) S_m. */
static void bb_poly(int l, int m, int nt, const int *px, const int *py, uint8_t *out) {
    int n = l * m;
    uint8_t *Sl = malloc((size_t)l * l), *Sm = malloc((size_t)m * m);
    uint8_t *Il = malloc((size_t)l * l), *Im = malloc((size_t)m * m);
    uint8_t *x = malloc((size_t)n * n), *y = malloc((size_t)n * n);
    uint8_t *xp = malloc((size_t)n * n), *yp = malloc((size_t)n * n), *mono = malloc((size_t)n * n);
    oracle_shift_matrix(l, Sl);
    oracle_shift_matrix(m, Sm);
    identity(Il, l);
    identity(Im, m);
    kron(Sl, l, Im, m, x);
    kron(Il, l, Sm, m, y);
    memset(out, 0, (size_t)n * n);
    for (int t = 0; t < nt; t++) {
        gf2_power(x, n, px[t], xp);
        gf2_power(y, n, py[t], yp);
        gf2_matmul(xp, yp, mono, n, n, n);
        for (int i = 0; i < n * n; i++) out[i] ^= mono[i];
    }
    free(Sl); free(Sm); free(Il); free(Im); free(x); free(y); free(xp); free(yp); free(mono);
}

/*
 * Bivariate bicycle code (Appendix, "BB Codes"): A = a(x,y), B = b(x,y),
 * H_X = [A | B] and H_Z = [B^T | A^T].  hx and hz are (l m) x (2 l m).
 * With m = 1 this is the generalised bicycle code of the "GB codes" part.
 */
void oracle_bb_code(int l, int m, int na, const int *ax, const int *ay, int nb, const int *bx,
                    const int *by, uint8_t *hx, uint8_t *hz) {
    int n = l * m;
    uint8_t *A = malloc((size_t)n * n), *B = malloc((size_t)n * n);
    bb_poly(l, m, na, ax, ay, A);
    bb_poly(l, m, nb, bx, by, B);
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            hx[r * 2 * n + c] = A[r * n + c];
            hx[r * 2 * n + n + c] = B[r * n + c];
            hz[r * 2 * n + c] = B[c * n + r];
            hz[r * 2 * n + n + c] = A[c * n + r];
        }
    free(A);
    free(B);
}

/*
 * R-round phenomenological detector matrix H = [I_R (x) H0 | B_R (x) I_m0],
 * B_R lower bidiagonal (ones on the diagonal and the first subdiagonal):
 * the detector of round t compares rounds t and t-1, so a measurement error
 * in round t flips detectors t and t+1 (only t in the last round).
 * h0 is m0 x n0; out is (R m0) x (R n0 + R m0).
 */
void oracle_phenom_code(const uint8_t *h0, int m0, int n0, int R, uint8_t *out) {
    int M = R * m0, N = R * n0 + R * m0;
    uint8_t *IR = malloc((size_t)R * R), *BR = malloc((size_t)R * R), *Im = malloc((size_t)m0 * m0);
    uint8_t *left = malloc((size_t)M * R * n0), *right = malloc((size_t)M * M);
    identity(IR, R);
    identity(Im, m0);
    memset(BR, 0, (size_t)R * R);
    for (int t = 0; t < R; t++) {
        BR[t * R + t] = 1;
        if (t + 1 < R) BR[(t + 1) * R + t] = 1;
    }
    /* I_R (x) H0 for a rectangular H0, written out. */
    for (int a = 0; a < R; a++)
        for (int b = 0; b < R; b++)
            for (int u = 0; u < m0; u++)
                for (int v = 0; v < n0; v++)
                    left[(a * m0 + u) * (R * n0) + (b * n0 + v)] = (uint8_t)(IR[a * R + b] & h0[u * n0 + v]);
    kron(BR, R, Im, m0, right);
    for (int r = 0; r < M; r++) {
        memcpy(out + (size_t)r * N, left + (size_t)r * R * n0, (size_t)R * n0);
        memcpy(out + (size_t)r * N + R * n0, right + (size_t)r * M, (size_t)M);
    }
    free(IR); free(BR); free(Im); free(left); free(right);
}

/* Rank over GF(2) by Gaussian elimination on a copy. */
int oracle_gf2_rank(const uint8_t *A, int rows, int cols) {
    uint8_t *W = malloc((size_t)rows * cols);
    memcpy(W, A, (size_t)rows * cols);
    int rank = 0;
    for (int c = 0; c < cols && rank < rows; c++) {
        int piv = -1;
        for (int r = rank; r < rows; r++)
            if (W[r * cols + c]) { piv = r; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int k = 0; k < cols; k++) {
                uint8_t t = W[piv * cols + k];
                W[piv * cols + k] = W[rank * cols + k];
                W[rank * cols + k] = t;
            }
        for (int r = 0; r < rows; r++)
            if (r != rank && W[r * cols + c])
                for (int k = 0; k < cols; k++) W[r * cols + k] ^= W[rank * cols + k];
        rank++;
    }
    free(W);
    return rank;
}

/*
 * X-type logical operators: a basis of ker(H_Z) modulo rowspace(H_X).  A Z
 * residual r with H_X r = 0 is a logical error iff L_X r != 0 (Eq. MLD_quantum:
 * errors differing by a stabiliser are equivalent).  Writes up to max_k rows
 * of length n into lx and returns k.
 */
int oracle_logicals(const uint8_t *hx, int mx, const uint8_t *hz, int mz, int n, uint8_t *lx, int max_k) {
    /* Null space of H_Z from its reduced row echelon form. */
    uint8_t *W = malloc((size_t)mz * n);
    memcpy(W, hz, (size_t)mz * n);
    int *pivcol = malloc(sizeof(int) * (size_t)(mz + 1));
    int rank = 0;
    for (int c = 0; c < n && rank < mz; c++) {
        int piv = -1;
        for (int r = rank; r < mz; r++)
            if (W[r * n + c]) { piv = r; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int k = 0; k < n; k++) {
                uint8_t t = W[piv * n + k];
                W[piv * n + k] = W[rank * n + k];
                W[rank * n + k] = t;
            }
        for (int r = 0; r < mz; r++)
            if (r != rank && W[r * n + c])
                for (int k = 0; k < n; k++) W[r * n + k] ^= W[rank * n + k];
        pivcol[rank++] = c;
    }
    uint8_t *is_piv = calloc((size_t)n, 1);
    for (int r = 0; r < rank; r++) is_piv[pivcol[r]] = 1;
    /* Stack [H_X ; candidate] and keep candidates that raise the rank. */
    uint8_t *stack = malloc((size_t)(mx + n) * n);
    memcpy(stack, hx, (size_t)mx * n);
    int rows = mx, base = oracle_gf2_rank(hx, mx, n), k = 0;
    uint8_t *v = malloc((size_t)n);
    for (int f = 0; f < n && k < max_k; f++) {
        if (is_piv[f]) continue;
        memset(v, 0, (size_t)n);
        v[f] = 1; /* free variable f set, pivots solved from the RREF */
        for (int r = 0; r < rank; r++) v[pivcol[r]] = W[r * n + f];
        memcpy(stack + (size_t)rows * n, v, (size_t)n);
        int rk = oracle_gf2_rank(stack, rows + 1, n);
        if (rk > base) {
            memcpy(lx + (size_t)k * n, v, (size_t)n);
            k++;
            rows++;
            base = rk;
        }
    }
    free(W); free(pivcol); free(is_piv); free(stack); free(v);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Tanner graph (Section II-B): N(v_i) = checks of column i, N(c_j) = vars   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int M, N, nnz;
    uint8_t *H;       /* dense M x N copy */
    int *row_ptr;     /* M+1: edges of check j are row_ptr[j]..row_ptr[j+1]-1 */
    int *row_var;     /* nnz: variable of each edge (ascending within a row) */
    int *col_ptr;     /* N+1 */
    int *col_chk;     /* nnz: checks of column i in ascending order */
    int *col_edge;    /* nnz: the edge id (row-ordered) of that (check, column) pair */
    int layered;      /* 0: flooding schedule; 1: layered schedule (rows by layer) */
    int n_layers;
    int *layer_of;    /* M: layer of each row (layered schedule) */
} oracle_code;

oracle_code *oracle_code_new(const uint8_t *H, int M, int N) {
    oracle_code *c = calloc(1, sizeof(oracle_code));
    c->M = M;
    c->N = N;
    c->H = malloc((size_t)M * N);
    memcpy(c->H, H, (size_t)M * N);
    int nnz = 0;
    for (int i = 0; i < M * N; i++) nnz += H[i] ? 1 : 0;
    c->nnz = nnz;
    c->row_ptr = malloc(sizeof(int) * (size_t)(M + 1));
    c->row_var = malloc(sizeof(int) * (size_t)(nnz + 1));
    c->col_ptr = malloc(sizeof(int) * (size_t)(N + 1));
    c->col_chk = malloc(sizeof(int) * (size_t)(nnz + 1));
    c->col_edge = malloc(sizeof(int) * (size_t)(nnz + 1));
    int e = 0;
    for (int j = 0; j < M; j++) {
        c->row_ptr[j] = e;
        for (int i = 0; i < N; i++)
            if (H[j * N + i]) c->row_var[e++] = i;
    }
    c->row_ptr[M] = e;
    int f = 0;
    for (int i = 0; i < N; i++) {
        c->col_ptr[i] = f;
        for (int j = 0; j < M; j++)
            if (H[j * N + i]) {
                c->col_chk[f] = j;
                int id = -1;
                for (int g = c->row_ptr[j]; g < c->row_ptr[j + 1]; g++)
                    if (c->row_var[g] == i) id = g;
                c->col_edge[f] = id;
                f++;
            }
    }
    c->col_ptr[N] = f;
    return c;
}

void oracle_code_free(oracle_code *c) {
    if (!c) return;
    free(c->H); free(c->row_ptr); free(c->row_var); free(c->col_ptr); free(c->col_chk); free(c->col_edge);
    free(c->layer_of);
    free(c);
}

int oracle_code_nnz(const oracle_code *c) { return c->nnz; }

/* s = H e (mod 2), dense mat-vec. */
void oracle_syndrome(const oracle_code *c, const uint8_t *e, uint8_t *s) {
    for (int j = 0; j < c->M; j++) {
        int acc = 0;
        for (int i = 0; i < c->N; i++) acc ^= (c->H[j * c->N + i] & e[i]);
        s[j] = (uint8_t)acc;
    }
}

/* e H^T = s, row by row over the ones of each row. */
/*
 * Layered schedule: rows are coloured greedily in ascending order, each row
 * taking the smallest layer not used by an earlier row that shares a
 * variable with it; layers are then processed in order.  Rows of one layer
 * share no variable, so their order within the layer does not matter.
 */
void oracle_code_set_layered(oracle_code *c, int on) {
    c->layered = on ? 1 : 0;
    if (!on || c->layer_of) return;
    c->layer_of = malloc(sizeof(int) * (size_t)(c->M + 1));
    uint8_t *used = malloc((size_t)c->M + 1);
    c->n_layers = 0;
    for (int j = 0; j < c->M; j++) {
        memset(used, 0, (size_t)c->M + 1);
        for (int k = 0; k < j; k++) {
            int share = 0;
            for (int i = 0; i < c->N && !share; i++) share = c->H[(size_t)j * c->N + i] && c->H[(size_t)k * c->N + i];
            if (share) used[c->layer_of[k]] = 1;
        }
        int l = 0;
        while (used[l]) l++;
        c->layer_of[j] = l;
        if (l + 1 > c->n_layers) c->n_layers = l + 1;
    }
    free(used);
}

int oracle_code_layer(const oracle_code *c, int j) { return c->layer_of ? c->layer_of[j] : -1; }

static int satisfies(const oracle_code *c, const uint8_t *e, const uint8_t *s) {
    for (int j = 0; j < c->M; j++) {
        int acc = 0;
        for (int g = c->row_ptr[j]; g < c->row_ptr[j + 1]; g++) acc ^= e[c->row_var[g]];
        if (acc != s[j]) return 0;
    }
    return 1;
}

/* Channel LLR (Section II-B, step 1): l_ch = log((1 - p) / p), in FP64. */
void oracle_llr_f64(const double *p, int n, double *out) {
    for (int i = 0; i < n; i++) out[i] = log((1.0 - p[i]) / p[i]);
}

/* The same value rounded once to FP32. */
void oracle_llr_f32(const double *p, int n, float *out) {
    for (int i = 0; i < n; i++) out[i] = (float)log((1.0 - p[i]) / p[i]);
}

/*
 * Phi = top(flip_count, w) (Algorithm 1; Section VI suggests a partial
 * selection sort): w rounds, each taking the not-yet-chosen bit with the
 * largest count, the smaller index on ties.  Zero counts are eligible.
 */
void oracle_top(const uint16_t *flips, int N, int w, int *phi) {
    uint8_t *taken = calloc((size_t)N + 1, 1);
    for (int r = 0; r < w; r++) {
        int best = -1;
        for (int i = 0; i < N; i++) {
            if (taken[i]) continue;
            if (best < 0 || flips[i] > flips[best]) best = i;
        }
        phi[r] = best;
        if (best >= 0) taken[best] = 1;
    }
    free(taken);
}

/*
 * Trial list of Algorithm 1 as subset masks over Phi (bit j selects Phi[j]):
 * the n_masks given masks in the given order, or, when n_masks == 0, every
 * non-empty subset of weight <= w_max in ascending mask order (enumerated by
 * counting, so only for w <= 24).  Returns the count (and *out, malloc'd),
 * or -1.  The sampled variant of Section V (n_s random vectors per weight)
 * is an explicit list.
 */
static int trial_count(int w, int w_max, int n_masks) {
    if (n_masks > 0) return n_masks;
    if (w <= 0) return 0;
    if (w > 24) return -1;
    int n = 0;
    for (uint64_t m = 1; m < (1ull << w); m++)
        if (__builtin_popcountll(m) <= w_max) n++;
    return n;
}

static int trial_list(int w, int w_max, const uint64_t *masks, int n_masks, uint64_t **out) {
    int n = trial_count(w, w_max, n_masks);
    if (n < 0) return -1;
    uint64_t *l = malloc(sizeof(uint64_t) * (size_t)(n + 1));
    if (n_masks > 0) {
        memcpy(l, masks, sizeof(uint64_t) * (size_t)n);
    } else {
        int k = 0;
        for (uint64_t m = 1; w > 0 && m < (1ull << w); m++)
            if (__builtin_popcountll(m) <= w_max) l[k++] = m;
    }
    *out = l;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Normalised min-sum BP (Section II-B) with oscillation tracking            */
/* (Algorithm 1, BP_with_oscillation); one body per floating-point mode.     */
/* ------------------------------------------------------------------------ */

#define REAL double
#define SFX(name) name##_f64
#define REAL_INF ((double)INFINITY)
#define REAL_ABS fabs
#include "bp_body.inc"
#undef REAL
#undef SFX
#undef REAL_INF
#undef REAL_ABS

#define REAL float
#define SFX(name) name##_f32
#define REAL_INF ((float)INFINITY)
#define REAL_ABS fabsf
#include "bp_body.inc"
#undef REAL
#undef SFX
#undef REAL_INF
#undef REAL_ABS

/* ------------------------------------------------------------------------ */
/* Sum-product BP (FP64), used only to pin the framework on cycle-free       */
/* graphs, where it computes exact marginals.                               */
/* ------------------------------------------------------------------------ */

void oracle_bp_sumproduct(const oracle_code *c, const double *lch, const uint8_t *s, int iters, double *lout) {
    double *q = malloc(sizeof(double) * (size_t)(c->nnz + 1));
    double *r = calloc((size_t)(c->nnz + 1), sizeof(double));
    for (int t = 0; t < iters; t++) {
        for (int i = 0; i < c->N; i++)
            for (int f = c->col_ptr[i]; f < c->col_ptr[i + 1]; f++) {
                double acc = lch[i];
                for (int g = c->col_ptr[i]; g < c->col_ptr[i + 1]; g++)
                    if (g != f) acc = acc + r[c->col_edge[g]];
                q[c->col_edge[f]] = acc;
            }
        for (int j = 0; j < c->M; j++)
            for (int e = c->row_ptr[j]; e < c->row_ptr[j + 1]; e++) {
                double prod = 1.0;
                for (int g = c->row_ptr[j]; g < c->row_ptr[j + 1]; g++)
                    if (g != e) prod *= tanh(q[g] / 2.0);
                double v = 2.0 * atanh(prod);
                r[e] = s[j] ? -v : v;
            }
    }
    for (int i = 0; i < c->N; i++) {
        double acc = lch[i];
        for (int f = c->col_ptr[i]; f < c->col_ptr[i + 1]; f++) acc = acc + r[c->col_edge[f]];
        lout[i] = acc;
    }
    free(q);
    free(r);
}

/* ------------------------------------------------------------------------ */
/* Batch driver (the timed CPU baseline): shots are independent, so the     */
/* loop over shots may run on several host threads.                          */
/* ------------------------------------------------------------------------ */

/* Monotonic wall time in seconds (per-shot times of the CPU baseline; shot_s
 * of the batch drivers is nullable and changes nothing else). */
static double wall_s(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_bpsf_batch_f32(const oracle_code *c, const float *lch, int64_t n, const uint8_t *synd, int max_iter,
                           float alpha, int w, int w_max, const uint64_t *masks, int n_masks, int short_iter,
                           int select, uint8_t *e_out, uint8_t *conv, int32_t *iters, uint8_t *stage, int threads,
                           double *shot_s) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads > 0 ? threads : 1)
#else
    (void)threads;
#endif
    for (int64_t k = 0; k < n; k++) {
        int it = 0, st = 0;
        const double t0 = shot_s ? wall_s() : 0.0;
        conv[k] = (uint8_t)oracle_bpsf_f32(c, lch, synd + k * c->M, max_iter, alpha, w, w_max, masks, n_masks,
                                           short_iter, select, e_out + k * c->N, &it, &st, NULL, NULL);
        iters[k] = it;
        stage[k] = (uint8_t)st;
        if (shot_s) shot_s[k] = wall_s() - t0;
    }
}

void oracle_bpsf_batch_f64(const oracle_code *c, const double *lch, int64_t n, const uint8_t *synd, int max_iter,
                           double alpha, int w, int w_max, const uint64_t *masks, int n_masks, int short_iter,
                           int select, uint8_t *e_out, uint8_t *conv, int32_t *iters, uint8_t *stage, int threads,
                           double *shot_s) {
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 8) num_threads(threads > 0 ? threads : 1)
#else
    (void)threads;
#endif
    for (int64_t k = 0; k < n; k++) {
        int it = 0, st = 0;
        const double t0 = shot_s ? wall_s() : 0.0;
        conv[k] = (uint8_t)oracle_bpsf_f64(c, lch, synd + k * c->M, max_iter, alpha, w, w_max, masks, n_masks,
                                           short_iter, select, e_out + k * c->N, &it, &st, NULL, NULL);
        iters[k] = it;
        stage[k] = (uint8_t)st;
        if (shot_s) shot_s[k] = wall_s() - t0;
    }
}
