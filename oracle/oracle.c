/*
 * CPU oracle for the genotype PCA path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 restatement of what the GPU library computes, written from
 * the paper (Chen, Noack, Edelman, "Fast computation of the principal
 * components of genotype matrices in Julia", arXiv:1808.03374) and textbook
 * definitions.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load this code; the library never does, and the two
 * share no source.
 *
 * Matrix.  G is n samples x m SNPs with entries 0/1/2 or missing (section 1).
 * Stored SNP-major, 2 bits per entry: SNP j's codes start at byte j*stride,
 * sample i sits in byte i>>2 at bits 2*(i&3); code 3 = missing.
 * The paper leaves standardisation and missing data open (imputation is future
 * work, section 5); the reading used here: mu_j = mean of the observed codes of
 * SNP j, d_j = 1/sd_j with sd_j the population standard deviation over the
 * observed codes (d_j = 0 for a monomorphic or empty SNP), missing entries
 * mean-imputed, i.e. contribute 0 after centring.  With optional per-sample
 * weights s and per-SNP weights w:
 *     A_ij = s_i * (((double)g_ij - mu_j) * d_j * w_j)   if g_ij < 3, else 0.
 *
 * Method.  Golub-Kahan-Lanczos bidiagonalisation (section 3) with full
 * reorthogonalisation by classical Gram-Schmidt applied twice (section 3,
 * reorthogonalisation paragraph) and thick restart with ordinary Ritz vectors
 * (section 3, thick-restarting paragraph).  Convergence uses the residual-norm
 * bound of the Ritz pairs (section 3, convergence paragraph): the residual of
 * triplet i is beta_ell*|P_{ell,i}|, and the sum over the wanted triplets is the
 * ||Delta theta||_1 of Table 3.  The small projected SVD is a one-sided
 * (Hestenes) Jacobi SVD.
 *
 * Parity pins: tests compare these routines with NumPy/LAPACK on small dense
 * matrices, closed forms (column sums, Frobenius norm), the Lanczos invariants
 * and the Marchenko-Pastur law (section 2, Eqs. 4 and 5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const uint8_t *packed;
    int64_t n, m, stride;
    const double *mu, *d; /* per SNP */
    const double *s;      /* per sample weight or NULL (= 1) */
    const double *w;      /* per SNP weight or NULL (= 1) */
} orc_mat;

static inline unsigned code_at(const orc_mat *M, int64_t i, int64_t j) {
    return (M->packed[j * M->stride + (i >> 2)] >> (2 * (i & 3))) & 3u;
}

/* Entry A_ij as defined above. */
static inline double entry(const orc_mat *M, int64_t i, int64_t j) {
    unsigned c = code_at(M, i, j);
    if (c == 3u) return 0.0;
    double a = ((double)c - M->mu[j]) * M->d[j];
    if (M->w) a = a * M->w[j];
    if (M->s) a = M->s[i] * a;
    return a;
}

/* Per-SNP statistics over observed entries: count, mean, 1/(population SD).
 * var_j = (nobs*sum(g^2) - sum(g)^2) / nobs^2 with the integer numerator exact. */
void orc_colstats(const uint8_t *packed, int64_t n, int64_t m, int64_t stride,
                  double *mu, double *d, int64_t *nobs_out) {
    for (int64_t j = 0; j < m; ++j) {
        int64_t nobs = 0, s1 = 0, s2 = 0;
        for (int64_t i = 0; i < n; ++i) {
            unsigned c = (packed[j * stride + (i >> 2)] >> (2 * (i & 3))) & 3u;
            if (c == 3u) continue;
            nobs += 1;
            s1 += c;
            s2 += (int64_t)c * c;
        }
        if (nobs_out) nobs_out[j] = nobs;
        if (nobs == 0) {
            mu[j] = 0.0;
            d[j] = 0.0;
            continue;
        }
        mu[j] = (double)s1 / (double)nobs;
        double num = (double)(nobs * s2 - s1 * s1);
        double var = num / ((double)nobs * (double)nobs);
        double sd = sqrt(var);
        d[j] = sd > 0.0 ? 1.0 / sd : 0.0;
    }
}

/* Dense A, column-major n x m (A[i + j*n]). */
void orc_unpack(const orc_mat *M, double *A) {
    for (int64_t j = 0; j < M->m; ++j)
        for (int64_t i = 0; i < M->n; ++i) A[i + j * M->n] = entry(M, i, j);
}

/* y = A v: y_i = sum_j A_ij v_j, j ascending.  Threads split the samples i;
 * each y_i is still summed over j in ascending order. */
void orc_matvec(const orc_mat *M, const double *v, double *y) {
    const int64_t n = M->n, m = M->m;
#pragma omp parallel
    {
#ifdef _OPENMP
        extern int omp_get_thread_num(void);
        extern int omp_get_num_threads(void);
        int t = omp_get_thread_num(), T = omp_get_num_threads();
#else
        int t = 0, T = 1;
#endif
        int64_t i0 = n * t / T, i1 = n * (t + 1) / T;
        for (int64_t i = i0; i < i1; ++i) y[i] = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            double vj = v[j];
            for (int64_t i = i0; i < i1; ++i) y[i] += entry(M, i, j) * vj;
        }
    }
}

/* x = A^T u: x_j = sum_i A_ij u_i, i ascending. */
void orc_rmatvec(const orc_mat *M, const double *u, double *x) {
    const int64_t n = M->n, m = M->m;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m; ++j) {
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) acc += entry(M, i, j) * u[i];
        x[j] = acc;
    }
}

/* y_r = (A v)_{rows[r]} for a list of sample indices. */
void orc_matvec_rows(const orc_mat *M, const double *v, const int64_t *rows, int64_t nr, double *y) {
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nr; ++r) {
        double acc = 0.0;
        for (int64_t j = 0; j < M->m; ++j) acc += entry(M, rows[r], j) * v[j];
        y[r] = acc;
    }
}

/* x_c = (A^T u)_{cols[c]} for a list of SNP indices. */
void orc_rmatvec_cols(const orc_mat *M, const double *u, const int64_t *cols, int64_t nc, double *x) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        double acc = 0.0;
        for (int64_t i = 0; i < M->n; ++i) acc += entry(M, i, cols[c]) * u[i];
        x[c] = acc;
    }
}

/* Y = A X for k vectors at once (X m x k, Y n x k, column-major): the
 * definition y_ic = sum_j A_ij x_jc, j ascending, each product and sum
 * rounded as written -- every column equals orc_matvec of that column.  Work
 * is split over tiles of 512 samples (each task walks all SNPs for its tile,
 * so its rows of Y stay in cache); the entries of a SNP row are formed once
 * per tile and used for all k columns. */
void orc_matmat(const orc_mat *M, const double *X, int64_t k, double *Y) {
    const int64_t n = M->n, m = M->m, T = 512;
    const int64_t tiles = (n + T - 1) / T;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < tiles; ++t) {
        const int64_t i0 = t * T, i1 = i0 + T < n ? i0 + T : n, len = i1 - i0;
        double a[512];
        for (int64_t c = 0; c < k; ++c)
            for (int64_t i = i0; i < i1; ++i) Y[i + c * n] = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            for (int64_t i = 0; i < len; ++i) a[i] = entry(M, i0 + i, j);
            for (int64_t c = 0; c < k; ++c) {
                const double xj = X[j + c * m];
                double *y = Y + i0 + c * n;
                for (int64_t i = 0; i < len; ++i) y[i] += a[i] * xj;
            }
        }
    }
}

/* X = A^T U for k vectors at once (U n x k, X m x k, column-major): x_jc =
 * sum_i A_ij u_ic, i ascending -- every column equals orc_rmatvec of that
 * column.  One SNP row per task; its entries are formed once for all k. */
void orc_rmatmat(const orc_mat *M, const double *U, int64_t k, double *X) {
    const int64_t n = M->n, m = M->m;
#pragma omp parallel
    {
        double *a = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < m; ++j) {
            if (!a) continue;
            for (int64_t i = 0; i < n; ++i) a[i] = entry(M, i, j);
            for (int64_t c = 0; c < k; ++c) {
                const double *u = U + c * n;
                double acc = 0.0;
                for (int64_t i = 0; i < n; ++i) acc += a[i] * u[i];
                X[j + c * m] = acc;
            }
        }
        free(a);
    }
}

/* ------------------------------------------------------------ Jacobi SVD */

/* One-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992) of the r x c
 * column-major matrix A, r >= c.  On return A holds U*Sigma columns, sigma the
 * singular values sorted descending, U (r x c) the left vectors (zero column
 * where sigma = 0) and V (c x c) the right vectors.  Returns the sweep count,
 * or -1 if 80 sweeps did not converge. */
int orc_jacobi_svd(int64_t r, int64_t c, double *A, double *sigma, double *U, double *V) {
    const double eps = 2.220446049250313e-16;
    for (int64_t a = 0; a < c; ++a)
        for (int64_t b = 0; b < c; ++b) V[a + b * c] = (a == b) ? 1.0 : 0.0;
    int sweep, done = 0;
    for (sweep = 1; sweep <= 80 && !done; ++sweep) {
        done = 1;
        for (int64_t p = 0; p < c - 1; ++p) {
            for (int64_t q = p + 1; q < c; ++q) {
                double *ap = A + p * r, *aq = A + q * r;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t i = 0; i < r; ++i) {
                    alpha += ap[i] * ap[i];
                    beta += aq[i] * aq[i];
                    gamma += ap[i] * aq[i];
                }
                if (gamma == 0.0 || fabs(gamma) <= eps * sqrt(alpha * beta)) continue;
                done = 0;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int64_t i = 0; i < r; ++i) {
                    double x = ap[i], y = aq[i];
                    ap[i] = cs * x - sn * y;
                    aq[i] = sn * x + cs * y;
                }
                double *vp = V + p * c, *vq = V + q * c;
                for (int64_t i = 0; i < c; ++i) {
                    double x = vp[i], y = vq[i];
                    vp[i] = cs * x - sn * y;
                    vq[i] = sn * x + cs * y;
                }
            }
        }
    }
    for (int64_t b = 0; b < c; ++b) {
        double s2 = 0.0;
        for (int64_t i = 0; i < r; ++i) s2 += A[i + b * r] * A[i + b * r];
        sigma[b] = sqrt(s2);
    }
    /* selection sort, descending, moving columns of A and V along */
    for (int64_t b = 0; b < c; ++b) {
        int64_t best = b;
        for (int64_t e = b + 1; e < c; ++e)
            if (sigma[e] > sigma[best]) best = e;
        if (best != b) {
            double ts = sigma[b]; sigma[b] = sigma[best]; sigma[best] = ts;
            for (int64_t i = 0; i < r; ++i) { double t = A[i + b * r]; A[i + b * r] = A[i + best * r]; A[i + best * r] = t; }
            for (int64_t i = 0; i < c; ++i) { double t = V[i + b * c]; V[i + b * c] = V[i + best * c]; V[i + best * c] = t; }
        }
    }
    for (int64_t b = 0; b < c; ++b)
        for (int64_t i = 0; i < r; ++i) U[i + b * r] = sigma[b] > 0.0 ? A[i + b * r] / sigma[b] : 0.0;
    return done ? sweep - 1 : -1;
}

/* ------------------------------------------------------------------ GKL */

/* Philox4x32-10 (Salmon et al., SC'11), used only to draw a replacement
 * vector when the Lanczos recurrence breaks down. */
static void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1, n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

/* Uniform on (-1,1) for index i of draw number `draw` under `seed`. */
static double replacement_entry(uint64_t seed, uint32_t draw, int64_t i) {
    uint32_t c[4] = {(uint32_t)i, draw, 0x474B4C00u, (uint32_t)(i >> 32)};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return ((double)c[0] + 0.5) * (2.0 / 4294967296.0) - 1.0;
}

static double dot(int64_t len, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += a[i] * b[i];
    return s;
}

/* Classical Gram-Schmidt applied twice against the first ncols columns of W
 * (len x ncols, column-major, leading dimension len). */
static void cgs2(int64_t len, const double *W, int64_t ncols, double *x, double *coef) {
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t k = 0; k < ncols; ++k) coef[k] = dot(len, W + k * len, x);
        for (int64_t k = 0; k < ncols; ++k) {
            const double *wk = W + k * len;
            for (int64_t i = 0; i < len; ++i) x[i] -= coef[k] * wk[i];
        }
    }
}

typedef struct {
    int32_t k, ell, k_keep, maxit;
    double tol;
    uint64_t seed;
} orc_opts;

typedef struct {
    int64_t pairs;       /* A.v / A^T.u pairs applied */
    int32_t restarts;
    int32_t breakdowns;
    int32_t converged;   /* 1 if max_i r_i <= tol*sigma_1 */
    int32_t cycles;
    double max_rel_resid;/* max_{i<k} r_i / sigma_1 */
    double dtheta1;      /* sum_{i<k} r_i */
} orc_info;

/* Normalise x (length len) or, if its norm is below `floor`, replace it by a
 * fresh vector orthogonalised against W[:, :ncols]; returns the norm used as
 * the Lanczos coefficient (0 on breakdown). */
static double normalise_or_replace(int64_t len, double *x, const double *W, int64_t ncols, double *coef,
                                   double floor, uint64_t seed, uint32_t *ndraw, int32_t *nbreak) {
    double nrm = sqrt(dot(len, x, x));
    if (nrm > floor) {
        for (int64_t i = 0; i < len; ++i) x[i] /= nrm;
        return nrm;
    }
    *nbreak += 1;
    for (int tries = 0; tries < 4; ++tries) {
        uint32_t dr = (*ndraw)++;
        for (int64_t i = 0; i < len; ++i) x[i] = replacement_entry(seed, dr, i);
        cgs2(len, W, ncols, x, coef);
        double r = sqrt(dot(len, x, x));
        if (r > 0.0) {
            for (int64_t i = 0; i < len; ++i) x[i] /= r;
            break;
        }
    }
    return 0.0;
}

/* Thick-restarted GKL for the k largest singular triplets of A.
 *
 * Recurrence (0-based columns; A V = U B with B upper triangular):
 *   u_j: y = A v_j - sum_{i<j} B_ij u_i, CGS2 against u_0..u_{j-1},
 *        alpha_j = ||y||, u_j = y/alpha_j, B_jj = alpha_j;
 *   v_{j+1}: x = A^T u_j - alpha_j v_j, CGS2 against v_0..v_j,
 *        beta_j = ||x||, v_{j+1} = x/beta_j, B_{j,j+1} = beta_j.
 * After ell steps, B = P Sigma Q^T; the Ritz residual of triplet i is
 * r_i = beta_{ell-1} |P_{ell-1,i}|.  Converged when max_{i<k} r_i <= tol*sigma_0.
 * Otherwise keep k' Ritz vectors: U <- U P[:, :k'], V <- V Q[:, :k'],
 * v_{k'} <- v_ell, and B restarts as diag(sigma_0..sigma_{k'-1}) with the spike
 * column B_{i,k'} = beta_{ell-1} P_{ell-1,i}.
 *
 * Outputs: sigma (k), U (n x k), V (m x k), resid (k, may be NULL); the signs
 * follow the rule of orc_sign_fix.  Optional Ub (n x ell), Vb (m x (ell+1)) and
 * Bout (ell x ell) receive the Krylov bases and projected matrix of the last
 * cycle.  Returns 0 on convergence, 1 if maxit cycles ran out, -1 on bad
 * arguments or allocation failure. */
void orc_sign_fix(int64_t n, int64_t m, int64_t k, double *U, double *V);

int orc_gkl(const orc_mat *M, const orc_opts *o, const double *v0, double *sigma, double *U, double *V,
            double *resid, orc_info *info, double *Ub, double *Vb, double *Bout) {
    const int64_t n = M->n, m = M->m;
    const int64_t k = o->k, ell = o->ell;
    int64_t kk = o->k_keep > 0 ? o->k_keep : k + (ell - k) / 2;
    if (k < 1 || ell <= k || ell > n || ell > m || kk < k || kk >= ell) return -1;
    const double eps = 2.220446049250313e-16;

    double *Uw = calloc((size_t)(n * ell), sizeof(double));
    double *Vw = calloc((size_t)(m * (ell + 1)), sizeof(double));
    double *B = calloc((size_t)(ell * ell), sizeof(double));
    double *Bc = malloc(sizeof(double) * (size_t)(ell * ell));
    double *P = malloc(sizeof(double) * (size_t)(ell * ell));
    double *Q = malloc(sizeof(double) * (size_t)(ell * ell));
    double *sg = malloc(sizeof(double) * (size_t)ell);
    double *coef = malloc(sizeof(double) * (size_t)(ell + 1));
    double *tmp = malloc(sizeof(double) * (size_t)((n > m ? n : m) * ell));
    double *y = malloc(sizeof(double) * (size_t)(n > m ? n : m));
    if (!Uw || !Vw || !B || !Bc || !P || !Q || !sg || !coef || !tmp || !y) {
        free(Uw); free(Vw); free(B); free(Bc); free(P); free(Q); free(sg); free(coef); free(tmp); free(y);
        return -1;
    }
    orc_info inf;
    memset(&inf, 0, sizeof(inf));
    uint32_t ndraw = 0;

    /* v_0 = v0 / ||v0|| */
    {
        double nr = sqrt(dot(m, v0, v0));
        for (int64_t i = 0; i < m; ++i) Vw[i] = v0[i] / nr;
    }
    double anorm = 0.0; /* running max of alpha, beta: lower bound on ||A|| */
    int64_t j0 = 0;
    int status = 1;
    double beta_last = 0.0;
    for (int cycle = 0; cycle < o->maxit; ++cycle) {
        inf.cycles = cycle + 1;
        for (int64_t j = j0; j < ell; ++j) {
            double *uj = Uw + j * n, *vj = Vw + j * m, *vn = Vw + (j + 1) * m;
            /* u side */
            orc_matvec(M, vj, uj);
            for (int64_t i = 0; i < j; ++i)
                if (B[i + j * ell] != 0.0)
                    for (int64_t t = 0; t < n; ++t) uj[t] -= B[i + j * ell] * Uw[i * n + t];
            double pre = sqrt(dot(n, uj, uj));
            cgs2(n, Uw, j, uj, coef);
            double floor = 1e3 * eps * (anorm > pre ? anorm : pre);
            double a = normalise_or_replace(n, uj, Uw, j, coef, floor, o->seed, &ndraw, &inf.breakdowns);
            B[j + j * ell] = a;
            if (a > anorm) anorm = a;
            /* v side */
            orc_rmatvec(M, uj, vn);
            for (int64_t t = 0; t < m; ++t) vn[t] -= a * vj[t];
            pre = sqrt(dot(m, vn, vn));
            cgs2(m, Vw, j + 1, vn, coef);
            floor = 1e3 * eps * (anorm > pre ? anorm : pre);
            double b = normalise_or_replace(m, vn, Vw, j + 1, coef, floor, o->seed, &ndraw, &inf.breakdowns);
            if (j + 1 < ell) B[j + (j + 1) * ell] = b;
            else beta_last = b;
            if (b > anorm) anorm = b;
            inf.pairs += 1;
        }
        /* Ritz values and vectors of the projected matrix */
        memcpy(Bc, B, sizeof(double) * (size_t)(ell * ell));
        orc_jacobi_svd(ell, ell, Bc, sg, P, Q);
        double maxr = 0.0, sum = 0.0;
        for (int64_t i = 0; i < k; ++i) {
            double r = fabs(beta_last * P[(ell - 1) + i * ell]);
            if (resid) resid[i] = r;
            sum += r;
            if (r > maxr) maxr = r;
        }
        inf.dtheta1 = sum;
        inf.max_rel_resid = sg[0] > 0.0 ? maxr / sg[0] : 0.0;
        int conv = maxr <= o->tol * sg[0];
        if (Ub) memcpy(Ub, Uw, sizeof(double) * (size_t)(n * ell));
        if (Vb) memcpy(Vb, Vw, sizeof(double) * (size_t)(m * (ell + 1)));
        if (Bout) memcpy(Bout, B, sizeof(double) * (size_t)(ell * ell));
        if (conv || cycle == o->maxit - 1) {
            for (int64_t i = 0; i < k; ++i) sigma[i] = sg[i];
            for (int64_t c = 0; c < k; ++c) {
                for (int64_t t = 0; t < n; ++t) {
                    double s = 0.0;
                    for (int64_t l = 0; l < ell; ++l) s += Uw[l * n + t] * P[l + c * ell];
                    U[t + c * n] = s;
                }
                for (int64_t t = 0; t < m; ++t) {
                    double s = 0.0;
                    for (int64_t l = 0; l < ell; ++l) s += Vw[l * m + t] * Q[l + c * ell];
                    V[t + c * m] = s;
                }
            }
            orc_sign_fix(n, m, k, U, V);
            inf.converged = conv;
            status = conv ? 0 : 1;
            break;
        }
        /* thick restart with kk Ritz vectors */
        for (int64_t c = 0; c < kk; ++c)
            for (int64_t t = 0; t < n; ++t) {
                double s = 0.0;
                for (int64_t l = 0; l < ell; ++l) s += Uw[l * n + t] * P[l + c * ell];
                tmp[t + c * n] = s;
            }
        memcpy(Uw, tmp, sizeof(double) * (size_t)(n * kk));
        for (int64_t c = 0; c < kk; ++c)
            for (int64_t t = 0; t < m; ++t) {
                double s = 0.0;
                for (int64_t l = 0; l < ell; ++l) s += Vw[l * m + t] * Q[l + c * ell];
                tmp[t + c * m] = s;
            }
        memcpy(Vw, tmp, sizeof(double) * (size_t)(m * kk));
        memcpy(Vw + kk * m, Vw + ell * m, sizeof(double) * (size_t)m);
        memset(B, 0, sizeof(double) * (size_t)(ell * ell));
        for (int64_t i = 0; i < kk; ++i) {
            B[i + i * ell] = sg[i];
            B[i + kk * ell] = beta_last * P[(ell - 1) + i * ell];
        }
        j0 = kk;
        inf.restarts += 1;
    }
    if (info) *info = inf;
    free(Uw); free(Vw); free(B); free(Bc); free(P); free(Q); free(sg); free(coef); free(tmp); free(y);
    return status;
}

/* Sign rule for singular vector pairs: the entry of largest magnitude of each
 * v_i is made positive (first such entry on ties); u_i flips with it. */
void orc_sign_fix(int64_t n, int64_t m, int64_t k, double *U, double *V) {
    for (int64_t c = 0; c < k; ++c) {
        double *v = V + c * m, *u = U + c * n;
        int64_t best = 0;
        for (int64_t t = 1; t < m; ++t)
            if (fabs(v[t]) > fabs(v[best])) best = t;
        if (v[best] < 0.0) {
            for (int64_t t = 0; t < m; ++t) v[t] = -v[t];
            for (int64_t t = 0; t < n; ++t) u[t] = -u[t];
        }
    }
}
