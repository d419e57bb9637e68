/*
 * FP64 CPU oracle for S3CMTF (sparse coupled Tucker matrix-tensor factorisation).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library.  It shares no code, header, table or helper with
 * the CUDA path, and the product path never calls it.
 *
 * Plain, slow, obviously-correct loops in double precision.  Every function cites the
 * passage of the paper it follows:
 *   Eq. (3)  row-set product over all modes but n            (Section 2.1)
 *   Eq. (4)  Tucker model, element-wise form                 (Section 2.2)
 *   Eq. (7)  objective f = f_t/2 + lambda_m f_m / 2, with the per-entry forms of
 *            f_t and f_m that follow it                      (Section 3.2)
 *   Eq. (8)  per-entry gradients                             (Section 3.2)
 *   Alg. 1   S3CMTF-naive epoch (lock-free SGD; here P = 1)  (Section 3.4)
 *   Alg. 2   compute_gradient                                (Section 3.4)
 *   Alg. 1   final QR step (U <- Q, G <- G x_n R, V <- V R^T) (Section 3.4)
 *   Def. 4 / Def. 5 / Lemma 2 / Lemma 3 / Alg. 3: intermediate data S, Collapse and the
 *            division route of S3CMTF-opt                    (Section 3.5)
 *   test RMSE                                                (Section 4.1, "Measure")
 *
 * Readings taken where the paper is silent or inconsistent (each also listed in the design
 * notes):
 *   - core regulariser per entry is lambda_reg/|Omega| * G (Eq. 8 and Alg. 2); Lemma 3 and
 *     Alg. 3 print lambda_reg * G, which contradicts the equivalence Lemma 3 claims.
 *   - rows that no train entry touches get no regulariser and no gradient (per-entry f_t).
 *   - Alg. 1 with P = 1: every tensor entry updates G with step eta_t.
 *   - eta_t = eta_0 / (1 + mu t) with t the 0-based epoch number.
 *   - S3CMTF-CP (cp = 1): the core is hyper-diagonal; its off-diagonal entries are not
 *     parameters, so every core step and the core gradient keep only the diagonal.
 *   - non-negative form (nonneg = 1; Section 5 names the projected gradient method, Lin
 *     2007, and gives no update rule): every SGD step of Alg. 1 or of the minibatch epoch
 *     is followed by the projection max(0, .) of each parameter that the step changed
 *     (the entry's rows, the core, the coupled entry's two rows); the full gradient is the
 *     plain gradient of Eq. (7).
 *   - minibatch epoch (not in the paper): all gradients of a batch at the batch-start
 *     parameters; rows take eta * (sum of their gradients) [/ their count in the batch when
 *     row_mean is set]; the core takes eta * core_scale * (mean of its per-entry gradients
 *     over the batch's tensor entries).  With batch = 1 this is Alg. 1 exactly.
 *
 * Layouts: tensor indices are structure-of-arrays, idx[n * nnz + e] (0-based); factor
 * matrices are dense row-major I_n x J_n; the core is dense with the last mode fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int N;                       /* tensor order */
    const int64_t* I;            /* [N] dimensionalities */
    const int* J;                /* [N] core dimensionalities (ranks) */
    int64_t nnz;                 /* observed (train) tensor entries */
    const int32_t* idx;          /* [N * nnz] */
    const double* x;             /* [nnz] */
    int M;                       /* number of coupled matrices */
    const int* cmode;            /* [M] coupled tensor mode, 0-based */
    const int64_t* K;            /* [M] rows of V_m (columns of Y_m) */
    const int64_t* ynnz;         /* [M] */
    const int32_t* const* yr;    /* [M][ynnz] row index j1 into I_c */
    const int32_t* const* yc;    /* [M][ynnz] column index j2 into K */
    const double* const* y;      /* [M][ynnz] */
    /* a part of a larger problem: that problem's row counts (N + M arrays: |Omega^{n,i}| for
       every tensor factor row, then |Omega_Y^{2,k}| for every coupled factor row) and its
       |Omega|, used by the regularisation terms; NULL / 0 = this data's own */
    const int64_t* const* cnt_total;
    int64_t nnz_total;
} s3o_data;

typedef struct {
    double* G;                   /* [prod J] */
    double* const* U;            /* [N][I_n * J_n] */
    double* const* V;            /* [M][K_m * J_c] */
} s3o_params;

typedef struct {
    double lr0, mu, lambda_reg, lambda_m;
    double core_scale;           /* minibatch core step multiplier */
    int64_t batch;               /* minibatch size B */
    int row_mean;                /* 0: rows take the batch sum, 1: the batch mean */
    int cp;                      /* 1: S3CMTF-CP, the core is hyper-diagonal (Section 4.2,
                                    comparison with SALS): only its diagonal is a parameter,
                                    so core steps and the core gradient keep the diagonal */
    int nonneg;                  /* 1: non-negative factorisation by projected SGD (Section 5,
                                    "Discovery"): after every step, each parameter the step
                                    changed is projected onto [0, inf), max(0, value) */
} s3o_hparams;

/* ------------------------------------------------------------------ small helpers */

/* the projection onto the non-negative orthant, element by element */
static void project_nonneg(double* v, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!(v[i] > 0.0)) v[i] = 0.0;
}

static int64_t core_size(int N, const int* J) {
    int64_t P = 1;
    for (int n = 0; n < N; ++n) P *= J[n];
    return P;
}

/* advance a multi-index (last mode fastest) */
static void odometer_next(int N, const int* J, int* j) {
    for (int n = N - 1; n >= 0; --n) {
        if (++j[n] < J[n]) return;
        j[n] = 0;
    }
}

/* S3CMTF-CP: keep only the hyper-diagonal of a core-shaped array (all ranks equal) */
static void cp_mask(int N, const int* J, const s3o_hparams* hp, double* gG) {
    if (!hp->cp) return;
    int j[8] = {0};
    const int64_t P = core_size(N, J);
    for (int64_t l = 0; l < P; ++l) {
        int diag = 1;
        for (int n = 1; n < N; ++n) diag &= j[n] == j[0];
        if (!diag) gG[l] = 0.0;
        odometer_next(N, J, j);
    }
}

/* rows a[n] = u^(n)_{i_n} of entry e */
static void entry_rows(const s3o_data* d, const s3o_params* p, int64_t e, const double** a) {
    for (int n = 0; n < d->N; ++n)
        a[n] = p->U[n] + (int64_t)d->idx[(int64_t)n * d->nnz + e] * d->J[n];
}

static double dot(const double* a, const double* b, int n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* |Omega^{n,i}| over the train entries, and |Omega_Y^{2,k}| per coupled matrix (the larger
   problem's, when the data is a part of one) */
static int64_t** tensor_counts(const s3o_data* d) {
    int64_t** c = (int64_t**)malloc(sizeof(int64_t*) * d->N);
    for (int n = 0; n < d->N; ++n) {
        c[n] = (int64_t*)calloc((size_t)d->I[n], sizeof(int64_t));
        if (d->cnt_total) memcpy(c[n], d->cnt_total[n], sizeof(int64_t) * (size_t)d->I[n]);
        else for (int64_t e = 0; e < d->nnz; ++e) c[n][d->idx[(int64_t)n * d->nnz + e]]++;
    }
    return c;
}
static int64_t** coupled_counts(const s3o_data* d) {
    int64_t** c = (int64_t**)malloc(sizeof(int64_t*) * (d->M > 0 ? d->M : 1));
    for (int m = 0; m < d->M; ++m) {
        c[m] = (int64_t*)calloc((size_t)d->K[m], sizeof(int64_t));
        if (d->cnt_total) memcpy(c[m], d->cnt_total[d->N + m], sizeof(int64_t) * (size_t)d->K[m]);
        else for (int64_t b = 0; b < d->ynnz[m]; ++b) c[m][d->yc[m][b]]++;
    }
    return c;
}
/* |Omega| of the problem the regularisers belong to */
static double omega(const s3o_data* d) { return d->nnz_total > 0 ? (double)d->nnz_total : (double)d->nnz; }
static void free_counts(int64_t** c, int n) {
    for (int k = 0; k < n; ++k) free(c[k]);
    free(c);
}

/* ------------------------------------------------------------------ Eq. (4), Eq. (3) */

/* x~ = G x {u}_alpha = sum over all core multi-indices of g_j * prod_n u^(n)_{i_n j_n} */
static double tucker_entry(int N, const int* J, const double* G, const double* const* a) {
    int j[8] = {0};
    int64_t P = core_size(N, J);
    double s = 0.0;
    for (int64_t l = 0; l < P; ++l) {
        double t = G[l];
        for (int n = 0; n < N; ++n) t *= a[n][j[n]];
        s += t;
        odometer_next(N, J, j);
    }
    return s;
}

/* [G x_{-n} {u}_alpha]_k = sum over core multi-indices with j_n = k of
   g_j * prod_{m != n} u^(m)_{i_m j_m}        (Eq. (3) applied to the core) */
static void partial_except(int N, const int* J, const double* G, const double* const* a,
                           int n, double* out) {
    int j[8] = {0};
    int64_t P = core_size(N, J);
    for (int k = 0; k < J[n]; ++k) out[k] = 0.0;
    for (int64_t l = 0; l < P; ++l) {
        double t = G[l];
        for (int m = 0; m < N; ++m)
            if (m != n) t *= a[m][j[m]];
        out[j[n]] += t;
        odometer_next(N, J, j);
    }
}

/* 1 x {u}^T_alpha: the outer product u^(1) o ... o u^(N) as a core-shaped array */
static void outer_rows(int N, const int* J, const double* const* a, double* out) {
    int j[8] = {0};
    int64_t P = core_size(N, J);
    for (int64_t l = 0; l < P; ++l) {
        double t = 1.0;
        for (int n = 0; n < N; ++n) t *= a[n][j[n]];
        out[l] = t;
        odometer_next(N, J, j);
    }
}

/* ------------------------------------------------------------------ Alg. 2 / Eq. (8) */

/* compute_gradient(alpha, x_alpha, G), the data-fit parts: x~ by Eq. (4), then
   -(x - x~) [G x_{-n} {u}_alpha] for every mode and -(x - x~) (1 x {u}^T_alpha) for the
   core.  The regularisation parts of Eq. (8) are added by add_tensor_reg.
   gu[n] has J_n values, gG has prod J values.  Returns the error x - x~. */
static double compute_gradient(const s3o_data* d, const s3o_params* p, int64_t e,
                               double* const* gu, double* gG) {
    const double* a[8];
    entry_rows(d, p, e, a);
    int N = d->N;
    const int* J = d->J;
    double xt = tucker_entry(N, J, p->G, a);
    double err = d->x[e] - xt;
    for (int n = 0; n < N; ++n) {
        partial_except(N, J, p->G, a, n, gu[n]);
        for (int k = 0; k < J[n]; ++k) gu[n][k] = -err * gu[n][k];
    }
    int64_t P = core_size(N, J);
    outer_rows(N, J, a, gG);
    for (int64_t l = 0; l < P; ++l) gG[l] = -err * gG[l];
    return err;
}

/* adds the regularisation parts of Eq. (8) for a tensor entry */
static void add_tensor_reg(const s3o_data* d, const s3o_params* p, int64_t e,
                           int64_t* const* cnt, double lambda_reg,
                           double* const* gu, double* gG) {
    for (int n = 0; n < d->N; ++n) {
        int64_t i = d->idx[(int64_t)n * d->nnz + e];
        const double* u = p->U[n] + i * d->J[n];
        double w = lambda_reg / (double)cnt[n][i];
        for (int k = 0; k < d->J[n]; ++k) gu[n][k] += w * u[k];
    }
    int64_t P = core_size(d->N, d->J);
    double w = lambda_reg / omega(d);
    for (int64_t l = 0; l < P; ++l) gG[l] += w * p->G[l];
}

/* Eq. (8), coupled-matrix rows: entry b of matrix m.  Returns the error y - y~. */
static double coupled_gradient(const s3o_data* d, const s3o_params* p, int m, int64_t b,
                               int64_t* const* cntY, double lambda_reg, double lambda_m,
                               double* gu, double* gv) {
    int c = d->cmode[m];
    int Jc = d->J[c];
    const double* u = p->U[c] + (int64_t)d->yr[m][b] * Jc;
    const double* v = p->V[m] + (int64_t)d->yc[m][b] * Jc;
    double err = d->y[m][b] - dot(u, v, Jc);
    double w = lambda_m * lambda_reg / (double)cntY[m][d->yc[m][b]];
    for (int k = 0; k < Jc; ++k) {
        gu[k] = -lambda_m * err * v[k];
        gv[k] = -lambda_m * err * u[k] + w * v[k];
    }
    return err;
}

/* ------------------------------------------------------------------ exported: O1 */

/* predictions x~ at arbitrary coordinates (idx SoA with n entries) */
void s3o_predict(const s3o_data* d, const s3o_params* p, const int32_t* idx, int64_t n,
                 double* out) {
    const double* a[8];
    for (int64_t e = 0; e < n; ++e) {
        for (int m = 0; m < d->N; ++m) a[m] = p->U[m] + (int64_t)idx[(int64_t)m * n + e] * d->J[m];
        out[e] = tucker_entry(d->N, d->J, p->G, a);
    }
}

/* the partial products G x_{-n} {u}_alpha for one coordinate, all modes: out has sum J_n */
void s3o_partials(const s3o_data* d, const s3o_params* p, const int32_t* alpha, double* out) {
    const double* a[8];
    for (int m = 0; m < d->N; ++m) a[m] = p->U[m] + (int64_t)alpha[m] * d->J[m];
    for (int n = 0; n < d->N; ++n) {
        partial_except(d->N, d->J, p->G, a, n, out);
        out += d->J[n];
    }
}

/* coupled predictions y~ = u^(c)_{j1} . v_{j2} for matrix m at n coordinates */
void s3o_predict_coupled(const s3o_data* d, const s3o_params* p, int m, const int32_t* r,
                         const int32_t* c, int64_t n, double* out) {
    int Jc = d->J[d->cmode[m]];
    for (int64_t b = 0; b < n; ++b)
        out[b] = dot(p->U[d->cmode[m]] + (int64_t)r[b] * Jc, p->V[m] + (int64_t)c[b] * Jc, Jc);
}

/* ------------------------------------------------------------------ exported: O2 */

/* f of Eq. (7) in its per-entry form (the sums that follow Eq. (7)); out[0] = f,
   out[1] = sum of squared tensor errors, out[2..2+M) = sum of squared errors of Y_m. */
void s3o_loss(const s3o_data* d, const s3o_params* p, const s3o_hparams* hp, double* out) {
    int N = d->N;
    int64_t P = core_size(N, d->J);
    int64_t** cnt = tensor_counts(d);
    int64_t** cntY = coupled_counts(d);
    double G2 = 0.0;
    for (int64_t l = 0; l < P; ++l) G2 += p->G[l] * p->G[l];
    double ft = 0.0, se = 0.0;
    const double* a[8];
    for (int64_t e = 0; e < d->nnz; ++e) {
        entry_rows(d, p, e, a);
        double err = d->x[e] - tucker_entry(N, d->J, p->G, a);
        double term = err * err + hp->lambda_reg / omega(d) * G2;
        for (int n = 0; n < N; ++n) {
            int64_t i = d->idx[(int64_t)n * d->nnz + e];
            term += hp->lambda_reg * dot(a[n], a[n], d->J[n]) / (double)cnt[n][i];
        }
        ft += term;
        se += err * err;
    }
    double f = 0.5 * ft;
    for (int m = 0; m < d->M; ++m) {
        int c = d->cmode[m];
        int Jc = d->J[c];
        double fm = 0.0, sy = 0.0;
        for (int64_t b = 0; b < d->ynnz[m]; ++b) {
            const double* u = p->U[c] + (int64_t)d->yr[m][b] * Jc;
            const double* v = p->V[m] + (int64_t)d->yc[m][b] * Jc;
            double err = d->y[m][b] - dot(u, v, Jc);
            fm += err * err + hp->lambda_reg / (double)cntY[m][d->yc[m][b]] * dot(v, v, Jc);
            sy += err * err;
        }
        f += 0.5 * hp->lambda_m * fm;
        out[2 + m] = sy;
    }
    out[0] = f;
    out[1] = se;
    free_counts(cnt, N);
    free_counts(cntY, d->M);
}

/* the same f with the regularisers summed once per parameter row instead of once per
   entry: f = 1/2 sum e^2 + lambda_reg/2 (||G||^2 + sum over rows with a train entry of
   ||u||^2) + sum_m lambda_m/2 (sum e^2 + lambda_reg sum over touched v rows ||v||^2). */
double s3o_loss_rowform(const s3o_data* d, const s3o_params* p, const s3o_hparams* hp) {
    int N = d->N;
    int64_t P = core_size(N, d->J);
    int64_t** cnt = tensor_counts(d);
    int64_t** cntY = coupled_counts(d);
    const double* a[8];
    double se = 0.0;
    for (int64_t e = 0; e < d->nnz; ++e) {
        entry_rows(d, p, e, a);
        double err = d->x[e] - tucker_entry(N, d->J, p->G, a);
        se += err * err;
    }
    double reg = 0.0;
    for (int64_t l = 0; l < P; ++l) reg += p->G[l] * p->G[l];
    for (int n = 0; n < N; ++n)
        for (int64_t i = 0; i < d->I[n]; ++i)
            if (cnt[n][i] > 0) {
                const double* u = p->U[n] + i * d->J[n];
                reg += dot(u, u, d->J[n]);
            }
    double f = 0.5 * se + 0.5 * hp->lambda_reg * reg;
    for (int m = 0; m < d->M; ++m) {
        int c = d->cmode[m];
        int Jc = d->J[c];
        double sy = 0.0, rv = 0.0;
        for (int64_t b = 0; b < d->ynnz[m]; ++b) {
            double err = d->y[m][b] - dot(p->U[c] + (int64_t)d->yr[m][b] * Jc,
                                          p->V[m] + (int64_t)d->yc[m][b] * Jc, Jc);
            sy += err * err;
        }
        for (int64_t k = 0; k < d->K[m]; ++k)
            if (cntY[m][k] > 0) {
                const double* v = p->V[m] + k * Jc;
                rv += dot(v, v, Jc);
            }
        f += 0.5 * hp->lambda_m * (sy + hp->lambda_reg * rv);
    }
    free_counts(cnt, N);
    free_counts(cntY, d->M);
    return f;
}

/* test RMSE (Section 4.1): sqrt(mean over test entries of (x - x~)^2), no clipping */
double s3o_rmse(const s3o_data* d, const s3o_params* p, const int32_t* idx, const double* x,
                int64_t n) {
    const double* a[8];
    double s = 0.0;
    for (int64_t e = 0; e < n; ++e) {
        for (int m = 0; m < d->N; ++m) a[m] = p->U[m] + (int64_t)idx[(int64_t)m * n + e] * d->J[m];
        double err = x[e] - tucker_entry(d->N, d->J, p->G, a);
        s += err * err;
    }
    return n > 0 ? sqrt(s / (double)n) : 0.0;
}

/* ------------------------------------------------------------------ exported: O3, O6 */

/* per-entry gradients of Eq. (8) for tensor entry e (Alg. 2): gu is sum J_n values
   (mode after mode), gG is prod J values.  Returns x - x~. */
double s3o_entry_gradient(const s3o_data* d, const s3o_params* p, const s3o_hparams* hp,
                          int64_t e, double* gu, double* gG) {
    int64_t** cnt = tensor_counts(d);
    double* gus[8] = {0};
    double* q = gu;
    for (int n = 0; n < d->N; ++n) { gus[n] = q; q += d->J[n]; }
    double err = compute_gradient(d, p, e, gus, gG);
    add_tensor_reg(d, p, e, cnt, hp->lambda_reg, gus, gG);
    free_counts(cnt, d->N);
    return err;
}

/* the same gradients by the S3CMTF-opt route: intermediate data S (Definition 4),
   x~ as the sum of S (Lemma 2), Collapse(S, n) (Definition 5) divided element-wise by the
   row and S divided element-wise by G (Lemma 3, Alg. 3).  Requires no zero in the rows
   or in G.  The core regulariser is lambda_reg/|Omega| (see the header). */
double s3o_entry_gradient_opt(const s3o_data* d, const s3o_params* p, const s3o_hparams* hp,
                              int64_t e, double* gu, double* gG) {
    int N = d->N;
    const int* J = d->J;
    int64_t P = core_size(N, J);
    int64_t** cnt = tensor_counts(d);
    const double* a[8];
    entry_rows(d, p, e, a);
    double* S = (double*)malloc(sizeof(double) * P);
    int j[8] = {0};
    double xt = 0.0;
    for (int64_t l = 0; l < P; ++l) {
        double s = p->G[l];
        for (int n = 0; n < N; ++n) s *= a[n][j[n]];
        S[l] = s;
        xt += s;
        odometer_next(N, J, j);
    }
    double err = d->x[e] - xt;
    double* q = gu;
    for (int n = 0; n < N; ++n) {
        int64_t i = d->idx[(int64_t)n * d->nnz + e];
        for (int k = 0; k < J[n]; ++k) q[k] = 0.0;
        memset(j, 0, sizeof(j));
        for (int64_t l = 0; l < P; ++l) {     /* Collapse(S, n) */
            q[j[n]] += S[l];
            odometer_next(N, J, j);
        }
        for (int k = 0; k < J[n]; ++k)
            q[k] = -err * q[k] / a[n][k] + hp->lambda_reg / (double)cnt[n][i] * a[n][k];
        q += J[n];
    }
    for (int64_t l = 0; l < P; ++l)
        gG[l] = -err * S[l] / p->G[l] + hp->lambda_reg / omega(d) * p->G[l];
    free(S);
    free_counts(cnt, N);
    return err;
}

/* full gradient of f = sum over train entries and coupled entries of Eq. (8).
   Outputs have the parameter shapes and are overwritten.
   w: NULL, or one weight per train entry that takes the place of -(x - x~) in that entry's
   data terms of Eq. (8) (so that a caller's upstream derivative with respect to the
   prediction x~_alpha can be propagated); the regularisation and coupled-matrix terms are
   those of Eq. (8) either way. */
void s3o_full_gradient_w(const s3o_data* d, const s3o_params* p, const s3o_hparams* hp,
                         const double* w, double* gG, double* const* gU, double* const* gV) {
    int N = d->N;
    const int* J = d->J;
    int64_t P = core_size(N, J);
    int64_t** cnt = tensor_counts(d);
    int64_t** cntY = coupled_counts(d);
    memset(gG, 0, sizeof(double) * P);
    for (int n = 0; n < N; ++n) memset(gU[n], 0, sizeof(double) * d->I[n] * J[n]);
    for (int m = 0; m < d->M; ++m) memset(gV[m], 0, sizeof(double) * d->K[m] * J[d->cmode[m]]);
    double* eg[8];
    for (int n = 0; n < N; ++n) eg[n] = (double*)malloc(sizeof(double) * J[n]);
    double* eG = (double*)malloc(sizeof(double) * P);
    for (int64_t e = 0; e < d->nnz; ++e) {
        double err = compute_gradient(d, p, e, eg, eG);
        if (w) {
            /* the data terms are -err times the partials and the outer product; rebuild them
               with the weight in place of -err */
            const double* a[8];
            entry_rows(d, p, e, a);
            for (int n = 0; n < N; ++n) {
                partial_except(N, J, p->G, a, n, eg[n]);
                for (int k = 0; k < J[n]; ++k) eg[n][k] *= w[e];
            }
            outer_rows(N, J, a, eG);
            for (int64_t l = 0; l < P; ++l) eG[l] *= w[e];
        }
        (void)err;
        add_tensor_reg(d, p, e, cnt, hp->lambda_reg, eg, eG);
        for (int n = 0; n < N; ++n) {
            int64_t i = d->idx[(int64_t)n * d->nnz + e];
            for (int k = 0; k < J[n]; ++k) gU[n][i * J[n] + k] += eg[n][k];
        }
        for (int64_t l = 0; l < P; ++l) gG[l] += eG[l];
    }
    cp_mask(N, J, hp, gG);
    for (int m = 0; m < d->M; ++m) {
        int c = d->cmode[m];
        int Jc = J[c];
        double* gu = (double*)malloc(sizeof(double) * Jc);
        double* gv = (double*)malloc(sizeof(double) * Jc);
        for (int64_t b = 0; b < d->ynnz[m]; ++b) {
            coupled_gradient(d, p, m, b, cntY, hp->lambda_reg, hp->lambda_m, gu, gv);
            for (int k = 0; k < Jc; ++k) {
                gU[c][(int64_t)d->yr[m][b] * Jc + k] += gu[k];
                gV[m][(int64_t)d->yc[m][b] * Jc + k] += gv[k];
            }
        }
        free(gu);
        free(gv);
    }
    for (int n = 0; n < N; ++n) free(eg[n]);
    free(eG);
    free_counts(cnt, N);
    free_counts(cntY, d->M);
}

void s3o_full_gradient(const s3o_data* d, const s3o_params* p, const s3o_hparams* hp,
                       double* gG, double* const* gU, double* const* gV) {
    s3o_full_gradient_w(d, p, hp, NULL, gG, gU, gV);
}

/* ------------------------------------------------------------------ exported: O4, O5 */

/* union item k -> (matrix m, entry b); returns -1 for a tensor entry */
static int union_item(const s3o_data* d, int64_t item, int64_t* b) {
    if (item < d->nnz) { *b = item; return -1; }
    item -= d->nnz;
    for (int m = 0; m < d->M; ++m) {
        if (item < d->ynnz[m]) { *b = item; return m; }
        item -= d->ynnz[m];
    }
    *b = -1;
    return -2;
}

/* eta_t of Alg. 1 */
double s3o_learning_rate(const s3o_hparams* hp, int64_t t) {
    return hp->lr0 / (1.0 + hp->mu * (double)t);
}

/* One pass of the inner loop of Alg. 1 with P = 1 (one sequential worker): visit the union
   of tensor entries and coupled entries in the given order; for a tensor entry take every
   gradient of Eq. (8) at the current parameters (Alg. 2), then update its N rows and the
   core; for a coupled entry update u^(c)_{j1} and v_{j2} from their pre-update values.
   Returns 0, or -1 on an item outside the union. */
int s3o_epoch_sequential(const s3o_data* d, s3o_params* p, const s3o_hparams* hp, int64_t t,
                         const int64_t* order, int64_t n_order) {
    int N = d->N;
    const int* J = d->J;
    int64_t P = core_size(N, J);
    double eta = s3o_learning_rate(hp, t);
    int64_t** cnt = tensor_counts(d);
    int64_t** cntY = coupled_counts(d);
    double* eg[8];
    int Jmax = 1;
    for (int n = 0; n < N; ++n) {
        eg[n] = (double*)malloc(sizeof(double) * J[n]);
        if (J[n] > Jmax) Jmax = J[n];
    }
    double* eG = (double*)malloc(sizeof(double) * P);
    double* gu = (double*)malloc(sizeof(double) * Jmax);
    double* gv = (double*)malloc(sizeof(double) * Jmax);
    int rc = 0;
    for (int64_t k = 0; k < n_order; ++k) {
        int64_t b;
        int m = union_item(d, order[k], &b);
        if (m == -2) { rc = -1; break; }
        if (m < 0) {
            compute_gradient(d, p, b, eg, eG);
            add_tensor_reg(d, p, b, cnt, hp->lambda_reg, eg, eG);
            cp_mask(N, J, hp, eG);
            for (int n = 0; n < N; ++n) {
                double* u = p->U[n] + (int64_t)d->idx[(int64_t)n * d->nnz + b] * J[n];
                for (int q = 0; q < J[n]; ++q) u[q] -= eta * eg[n][q];
                if (hp->nonneg) project_nonneg(u, J[n]);
            }
            for (int64_t l = 0; l < P; ++l) p->G[l] -= eta * eG[l];
            if (hp->nonneg) project_nonneg(p->G, P);
        } else {
            int c = d->cmode[m];
            int Jc = J[c];
            coupled_gradient(d, p, m, b, cntY, hp->lambda_reg, hp->lambda_m, gu, gv);
            double* u = p->U[c] + (int64_t)d->yr[m][b] * Jc;
            double* v = p->V[m] + (int64_t)d->yc[m][b] * Jc;
            for (int q = 0; q < Jc; ++q) {
                u[q] -= eta * gu[q];
                v[q] -= eta * gv[q];
            }
            if (hp->nonneg) {
                project_nonneg(u, Jc);
                project_nonneg(v, Jc);
            }
        }
    }
    for (int n = 0; n < N; ++n) free(eg[n]);
    free(eG);
    free(gu);
    free(gv);
    free_counts(cnt, N);
    free_counts(cntY, d->M);
    return rc;
}

/* Minibatch epoch (not in the paper; see the header): consecutive batches of hp->batch
   items of the given order; every gradient of a batch at the batch-start parameters. */
int s3o_epoch_minibatch(const s3o_data* d, s3o_params* p, const s3o_hparams* hp, int64_t t,
                        const int64_t* order, int64_t n_order) {
    int N = d->N, M = d->M;
    const int* J = d->J;
    int64_t P = core_size(N, J);
    double eta = s3o_learning_rate(hp, t);
    int64_t B = hp->batch > 0 ? hp->batch : 1;
    int64_t** cnt = tensor_counts(d);
    int64_t** cntY = coupled_counts(d);
    /* batch accumulators, one per parameter row, plus how often each row was hit */
    double* DU[8];
    int64_t* hU[8];
    double** DV = (double**)malloc(sizeof(double*) * (M > 0 ? M : 1));
    int64_t** hV = (int64_t**)malloc(sizeof(int64_t*) * (M > 0 ? M : 1));
    for (int n = 0; n < N; ++n) {
        DU[n] = (double*)calloc((size_t)(d->I[n] * J[n]), sizeof(double));
        hU[n] = (int64_t*)calloc((size_t)d->I[n], sizeof(int64_t));
    }
    for (int m = 0; m < M; ++m) {
        DV[m] = (double*)calloc((size_t)(d->K[m] * J[d->cmode[m]]), sizeof(double));
        hV[m] = (int64_t*)calloc((size_t)d->K[m], sizeof(int64_t));
    }
    double* DG = (double*)calloc((size_t)P, sizeof(double));
    double* eg[8];
    int Jmax = 1;
    for (int n = 0; n < N; ++n) {
        eg[n] = (double*)malloc(sizeof(double) * J[n]);
        if (J[n] > Jmax) Jmax = J[n];
    }
    double* eG = (double*)malloc(sizeof(double) * P);
    double* gu = (double*)malloc(sizeof(double) * Jmax);
    double* gv = (double*)malloc(sizeof(double) * Jmax);
    /* rows touched in the current batch (a row may be listed more than once) */
    int64_t cap = B * (N + 2) + 8;
    int* tf = (int*)malloc(sizeof(int) * cap);          /* factor id: n, or N + m for V_m */
    int64_t* tr = (int64_t*)malloc(sizeof(int64_t) * cap);
    int rc = 0;
    for (int64_t b0 = 0; b0 < n_order && rc == 0; b0 += B) {
        int64_t b1 = b0 + B < n_order ? b0 + B : n_order;
        int64_t nt = 0, ntouch = 0;
        for (int64_t k = b0; k < b1; ++k) {
            int64_t b;
            int m = union_item(d, order[k], &b);
            if (m == -2) { rc = -1; break; }
            if (m < 0) {
                compute_gradient(d, p, b, eg, eG);
                add_tensor_reg(d, p, b, cnt, hp->lambda_reg, eg, eG);
                for (int n = 0; n < N; ++n) {
                    int64_t i = d->idx[(int64_t)n * d->nnz + b];
                    for (int q = 0; q < J[n]; ++q) DU[n][i * J[n] + q] += eg[n][q];
                    hU[n][i]++;
                    tf[ntouch] = n; tr[ntouch++] = i;
                }
                cp_mask(N, J, hp, eG);
                for (int64_t l = 0; l < P; ++l) DG[l] += eG[l];
                nt++;
            } else {
                int c = d->cmode[m];
                int Jc = J[c];
                coupled_gradient(d, p, m, b, cntY, hp->lambda_reg, hp->lambda_m, gu, gv);
                int64_t i = d->yr[m][b], kk = d->yc[m][b];
                for (int q = 0; q < Jc; ++q) {
                    DU[c][i * Jc + q] += gu[q];
                    DV[m][kk * Jc + q] += gv[q];
                }
                hU[c][i]++;
                hV[m][kk]++;
                tf[ntouch] = c; tr[ntouch++] = i;
                tf[ntouch] = N + m; tr[ntouch++] = kk;
            }
        }
        /* apply: every touched row once (the hit count is cleared on first visit) */
        for (int64_t s = 0; s < ntouch; ++s) {
            int f = tf[s];
            int64_t i = tr[s];
            if (f < N) {
                if (hU[f][i] == 0) continue;
                double den = hp->row_mean ? (double)hU[f][i] : 1.0;
                double* u = p->U[f] + i * J[f];
                double* D = DU[f] + i * J[f];
                for (int q = 0; q < J[f]; ++q) { u[q] -= eta * D[q] / den; D[q] = 0.0; }
                if (hp->nonneg) project_nonneg(u, J[f]);
                hU[f][i] = 0;
            } else {
                int m = f - N;
                int Jc = J[d->cmode[m]];
                if (hV[m][i] == 0) continue;
                double den = hp->row_mean ? (double)hV[m][i] : 1.0;
                double* v = p->V[m] + i * Jc;
                double* D = DV[m] + i * Jc;
                for (int q = 0; q < Jc; ++q) { v[q] -= eta * D[q] / den; D[q] = 0.0; }
                if (hp->nonneg) project_nonneg(v, Jc);
                hV[m][i] = 0;
            }
        }
        if (nt > 0) {
            double w = eta * hp->core_scale / (double)nt;
            for (int64_t l = 0; l < P; ++l) { p->G[l] -= w * DG[l]; DG[l] = 0.0; }
            if (hp->nonneg) project_nonneg(p->G, P);
        }
    }
    for (int n = 0; n < N; ++n) { free(DU[n]); free(hU[n]); free(eg[n]); }
    for (int m = 0; m < M; ++m) { free(DV[m]); free(hV[m]); }
    free(DV); free(hV); free(DG); free(eG); free(gu); free(gv); free(tf); free(tr);
    free_counts(cnt, N);
    free_counts(cntY, M);
    return rc;
}

/* ------------------------------------------------------------------ final QR step
 * Algorithm 1, after the last epoch: for every mode n the thin QR decomposition
 * U^(n) = Q^(n) R^(n) (Q^(n) I_n x J_n with orthonormal columns, R^(n) J_n x J_n upper
 * triangular), U^(n) <- Q^(n), G <- G x_n R^(n); then every coupled factor
 * V_m <- V_m R^(c_m)^T.  The factorisation is unchanged: x~ = (G x_1 R^(1) ... x_N R^(N))
 * x_1 Q^(1) ... x_N Q^(N) and U^(c) V^T = Q^(c) (V R^(c)^T)^T (Section 3.4, description
 * of Algorithm 1).  The paper does not fix the signs; here diag(R^(n)) > 0, which makes
 * the thin QR of a full-column-rank matrix unique.
 *
 * Householder reflections in double precision.  R_out (optional): [N][J_n * J_n]
 * row-major.  Returns 0, or -1 when some U^(n) does not have full numerical column rank (a
 * diagonal entry of R at most 1e-7 of the largest), in which case nothing is changed. */

/* thin QR of A (rows x cols, row-major, rows >= cols) into Q (rows x cols) and R (cols x
 * cols); diag(R) >= 0.  Returns -1 if A is numerically rank deficient. */
static int householder_qr(const double* A, int64_t rows, int cols, double* Q, double* R) {
    double* W = (double*)malloc(sizeof(double) * rows * cols);     /* working copy */
    double* vs = (double*)calloc((size_t)rows * cols, sizeof(double)); /* reflectors */
    memcpy(W, A, sizeof(double) * rows * cols);
    int rc = 0;
    for (int k = 0; k < cols; ++k) {
        /* reflector v = x + sign(x_0) |x| e_0 on column k, rows k.. */
        double nrm = 0.0;
        for (int64_t i = k; i < rows; ++i) nrm += W[i * cols + k] * W[i * cols + k];
        nrm = sqrt(nrm);
        double* v = vs + (int64_t)k * rows;
        if (nrm == 0.0) { rc = -1; continue; }
        const double x0 = W[(int64_t)k * cols + k];
        const double alpha = x0 >= 0.0 ? -nrm : nrm;
        for (int64_t i = k; i < rows; ++i) v[i] = W[i * cols + k];
        v[k] -= alpha;
        double vn = 0.0;
        for (int64_t i = k; i < rows; ++i) vn += v[i] * v[i];
        vn = sqrt(vn);
        if (vn == 0.0) continue;   /* column already of the form alpha e_k */
        for (int64_t i = k; i < rows; ++i) v[i] /= vn;
        /* W[k:, k:] -= 2 v (v^T W[k:, k:]) */
        for (int c = k; c < cols; ++c) {
            double s = 0.0;
            for (int64_t i = k; i < rows; ++i) s += v[i] * W[i * cols + c];
            for (int64_t i = k; i < rows; ++i) W[i * cols + c] -= 2.0 * v[i] * s;
        }
    }
    /* R: upper triangle of W; Q = H_0 H_1 ... H_{cols-1} [I; 0] */
    for (int r = 0; r < cols; ++r)
        for (int c = 0; c < cols; ++c) R[r * cols + c] = c >= r ? W[(int64_t)r * cols + c] : 0.0;
    memset(Q, 0, sizeof(double) * rows * cols);
    for (int c = 0; c < cols; ++c) Q[(int64_t)c * cols + c] = 1.0;
    for (int k = cols - 1; k >= 0; --k) {
        const double* v = vs + (int64_t)k * rows;
        for (int c = 0; c < cols; ++c) {
            double s = 0.0;
            for (int64_t i = k; i < rows; ++i) s += v[i] * Q[i * cols + c];
            for (int64_t i = k; i < rows; ++i) Q[i * cols + c] -= 2.0 * v[i] * s;
        }
    }
    /* numerical rank: every |R_rr| above 1e-7 of the largest (what a Gram-based QR in
     * double precision can still resolve: its pivots are R_rr^2) */
    double dmax = 0.0;
    for (int r = 0; r < cols; ++r) dmax = fmax(dmax, fabs(R[r * cols + r]));
    /* signs: diag(R) >= 0 (row r of R and column r of Q flip together) */
    for (int r = 0; r < cols; ++r) {
        if (!(fabs(R[r * cols + r]) > 1e-7 * dmax)) rc = -1;
        if (R[r * cols + r] < 0.0) {
            for (int c = 0; c < cols; ++c) R[r * cols + c] = -R[r * cols + c];
            for (int64_t i = 0; i < rows; ++i) Q[i * cols + r] = -Q[i * cols + r];
        }
    }
    free(W);
    free(vs);
    return rc;
}

/* G <- G x_n R: new G[.., i, ..] = sum_j R[i][j] G[.., j, ..] (mode n, last mode fastest) */
static void core_times_matrix(int N, const int* J, double* G, int n, const double* R) {
    const int64_t P = core_size(N, J);
    int64_t inner = 1;
    for (int k = n + 1; k < N; ++k) inner *= J[k];
    const int64_t outer = P / (inner * J[n]);
    double* col = (double*)malloc(sizeof(double) * J[n]);
    for (int64_t o = 0; o < outer; ++o)
        for (int64_t s = 0; s < inner; ++s) {
            double* base = G + o * (int64_t)J[n] * inner + s;
            for (int i = 0; i < J[n]; ++i) {
                double acc = 0.0;
                for (int j = 0; j < J[n]; ++j) acc += R[i * J[n] + j] * base[(int64_t)j * inner];
                col[i] = acc;
            }
            for (int i = 0; i < J[n]; ++i) base[(int64_t)i * inner] = col[i];
        }
    free(col);
}

int s3o_finalize_qr(const s3o_data* d, s3o_params* p, double* const* R_out) {
    const int N = d->N, M = d->M;
    double** Q = (double**)malloc(sizeof(double*) * N);
    double** R = (double**)malloc(sizeof(double*) * N);
    int rc = 0;
    for (int n = 0; n < N; ++n) {
        Q[n] = (double*)malloc(sizeof(double) * d->I[n] * d->J[n]);
        R[n] = (double*)malloc(sizeof(double) * d->J[n] * d->J[n]);
        if (d->I[n] < d->J[n] || householder_qr(p->U[n], d->I[n], d->J[n], Q[n], R[n]) != 0) rc = -1;
    }
    if (rc == 0) {
        for (int n = 0; n < N; ++n) {
            memcpy(p->U[n], Q[n], sizeof(double) * d->I[n] * d->J[n]);
            core_times_matrix(N, d->J, p->G, n, R[n]);
            if (R_out && R_out[n]) memcpy(R_out[n], R[n], sizeof(double) * d->J[n] * d->J[n]);
        }
        for (int m = 0; m < M; ++m) {
            const int c = d->cmode[m], Jc = d->J[c];
            double* row = (double*)malloc(sizeof(double) * Jc);
            for (int64_t k = 0; k < d->K[m]; ++k) {
                double* v = p->V[m] + k * Jc;
                for (int i = 0; i < Jc; ++i) {   /* (V R^T)[k][i] = sum_j V[k][j] R[i][j] */
                    double acc = 0.0;
                    for (int j = 0; j < Jc; ++j) acc += v[j] * R[c][i * Jc + j];
                    row[i] = acc;
                }
                memcpy(v, row, sizeof(double) * Jc);
            }
            free(row);
        }
    }
    for (int n = 0; n < N; ++n) { free(Q[n]); free(R[n]); }
    free(Q);
    free(R);
    return rc;
}
