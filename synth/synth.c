/*
 * Seeded synthetic inputs for the genotype-PCA path: packed genotype matrices
 * shaped like GWAS cohorts, start vectors and per-sample / per-SNP weights.
 *
 * This module draws random inputs only.  It contains none of the method's
 * arithmetic (no centring, scaling, products or decompositions), so both the
 * CPU oracle and the CUDA library can consume what it writes.
 *
 * Random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 128-bit counter is
 * permuted by ten rounds keyed by a 64-bit key.  Every draw is addressed by a
 * (stream, index...) counter, so the output does not depend on thread count.
 *
 * Genotype model.  G is n samples x m SNPs with entries in {0,1,2} (allele
 * counts, section 1 of the paper) or missing.  Each SNP j has a base allele
 * frequency p_j; each of S populations has its own frequency f_kj near p_j;
 * sample i has ancestry proportions q_i (one-hot for discrete populations,
 * Dirichlet for admixture), so its frequency at j is p_ij = sum_k q_ik f_kj and
 * G_ij ~ Binomial(2, p_ij) drawn as two Bernoulli alleles.  Each entry is
 * missing independently with probability miss_rate.
 *
 * Storage (SNP-major, 2 bits per entry): SNP j occupies `stride` bytes starting
 * at j*stride; sample i lives in byte i>>2 at bits 2*(i&3)..2*(i&3)+1.  Codes
 * 0,1,2 are allele counts and code 3 marks a missing entry.  Padding entries
 * (i >= n) are written as code 3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

typedef struct { uint32_t w[4]; } ctr4;

static inline void mulhilo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Ten Philox rounds; round r uses key + r*(W0,W1). */
ctr4 synth_philox4x32_10(ctr4 c, uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo(0xD2511F53u, c.w[0], &hi0, &lo0);
        mulhilo(0xCD9E8D57u, c.w[2], &hi1, &lo1);
        ctr4 o;
        o.w[0] = hi1 ^ c.w[1] ^ k0;
        o.w[1] = lo1;
        o.w[2] = hi0 ^ c.w[3] ^ k1;
        o.w[3] = lo0;
        c = o;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

/* Exported for the known-answer test of the generator itself. */
void synth_philox_block(const uint32_t ctr_in[4], const uint32_t key[2], uint32_t out[4]) {
    ctr4 c = {{ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]}};
    ctr4 r = synth_philox4x32_10(c, key[0], key[1]);
    memcpy(out, r.w, sizeof(r.w));
}

enum {
    ST_BASE = 1,  /* per-SNP base frequency      ctr = (j, 0, ST, draw) */
    ST_POP = 2,   /* per-(pop,SNP) perturbation  ctr = (j, k, ST, draw) */
    ST_ANC = 3,   /* per-sample ancestry         ctr = (i, k, ST, draw) */
    ST_GENO = 4,  /* per-entry genotype          ctr = (i, j, ST, 0)    */
    ST_VEC = 5,   /* free-standing vectors       ctr = (i, stream, ST, draw) */
    ST_MODEL_BLK = 6,  /* paper model: sub-block b    ctr = (b, 0, ST, draw) */
    ST_MODEL_SIG = 7,  /* paper model: entry (j, i)   ctr = (i, j, ST, 0) */
    ST_MODEL_KIN = 8   /* paper model: row copy c     ctr = (c, 0, ST, 0) */
};

static inline ctr4 draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t st, uint32_t d) {
    ctr4 c = {{a, b, st, d}};
    return synth_philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

/* 53-bit uniform in (0,1]: never returns 0 so that log() is finite. */
static inline double u53(uint32_t a, uint32_t b) {
    uint64_t x = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)x + 1.0) * (1.0 / 9007199254740992.0);
}

static double normal_from(ctr4 r) {
    double u1 = u53(r.w[0], r.w[1]);
    double u2 = u53(r.w[2], r.w[3]);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Gamma(shape, 1) by Marsaglia & Tsang (2000); shape < 1 via the U^(1/a) boost.
 * Successive attempts use successive draw indices starting at d0. */
static double gamma_draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t st, uint32_t d0, double shape) {
    double boost = 1.0;
    uint32_t d = d0;
    if (shape < 1.0) {
        ctr4 r = draw(seed, a, b, st, d++);
        boost = pow(u53(r.w[0], r.w[1]), 1.0 / shape);
        shape += 1.0;
    }
    double dd = shape - 1.0 / 3.0, cc = 1.0 / sqrt(9.0 * dd);
    for (int it = 0; it < 1000; ++it) {
        ctr4 r = draw(seed, a, b, st, d++);
        double x = normal_from(r);
        double v = 1.0 + cc * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        ctr4 r2 = draw(seed, a, b, st, d++);
        double u = u53(r2.w[0], r2.w[1]);
        if (log(u) < 0.5 * x * x + dd - dd * v + dd * log(v)) return dd * v * boost;
    }
    return dd * boost;
}

static inline double clip(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

typedef struct {
    int64_t n, m, stride;
    int32_t n_pops;        /* S >= 1 */
    int32_t admixture;     /* 0: discrete equal-size populations, 1: Dirichlet ancestry */
    int32_t base_beta;     /* 0: p_j ~ U(base_lo, base_hi); 1: p_j ~ Beta(beta_a, beta_b) clipped to [base_lo, base_hi] */
    int32_t pm_delta;      /* 1 with S == 2: f_0j = p_j + d_j, f_1j = p_j - d_j with one d_j ~ N(0, delta_sd^2) */
    double base_lo, base_hi, beta_a, beta_b;
    double delta_sd;       /* 0 gives the null model f_kj = p_j */
    double f_lo, f_hi;     /* clip range of f_kj */
    double dirichlet_alpha;
    double miss_rate;
    uint64_t seed;
} synth_params;

/* Population frequencies f (S x m, row k contiguous) and ancestry q (n x S,
 * row i contiguous).  Both are small compared with the packed matrix. */
int synth_population(const synth_params *P, double *f, double *q) {
    const int64_t n = P->n, m = P->m;
    const int S = P->n_pops;
    if (n <= 0 || m <= 0 || S <= 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < m; ++j) {
        double pj;
        if (P->base_beta) {
            double x = gamma_draw(P->seed, (uint32_t)j, 0, ST_BASE, 0, P->beta_a);
            double y = gamma_draw(P->seed, (uint32_t)j, 1, ST_BASE, 0, P->beta_b);
            pj = clip(x / (x + y), P->base_lo, P->base_hi);
        } else {
            ctr4 r = draw(P->seed, (uint32_t)j, 0, ST_BASE, 0);
            pj = P->base_lo + (P->base_hi - P->base_lo) * u53(r.w[0], r.w[1]);
        }
        if (P->pm_delta && S == 2) {
            double dj = P->delta_sd * normal_from(draw(P->seed, (uint32_t)j, 0, ST_POP, 0));
            f[0 * m + j] = clip(pj + dj, P->f_lo, P->f_hi);
            f[1 * m + j] = clip(pj - dj, P->f_lo, P->f_hi);
        } else {
            for (int k = 0; k < S; ++k) {
                double dj = P->delta_sd * normal_from(draw(P->seed, (uint32_t)j, (uint32_t)k, ST_POP, 0));
                f[(int64_t)k * m + j] = clip(pj + dj, P->f_lo, P->f_hi);
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double *qi = q + i * S;
        if (!P->admixture) {
            int pop = (int)((i * S) / n);
            for (int k = 0; k < S; ++k) qi[k] = (k == pop) ? 1.0 : 0.0;
        } else {
            double tot = 0.0;
            for (int k = 0; k < S; ++k) {
                qi[k] = gamma_draw(P->seed, (uint32_t)i, (uint32_t)k, ST_ANC, 0, P->dirichlet_alpha);
                tot += qi[k];
            }
            for (int k = 0; k < S; ++k) qi[k] /= tot;
        }
    }
    return 0;
}

/* Packed genotypes from f and q (as written by synth_population). */
int synth_pack(const synth_params *P, const double *f, const double *q, uint8_t *packed) {
    const int64_t n = P->n, m = P->m, stride = P->stride;
    const int S = P->n_pops;
    if (stride * 4 < n || stride % 16 != 0) return -1;
    const double two32 = 4294967296.0;
    const double miss_thr = P->miss_rate * two32;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < m; ++j) {
        uint8_t *row = packed + j * stride;
        memset(row, 0xFF, (size_t)stride); /* padding = code 3 */
        for (int64_t i = 0; i < n; ++i) {
            const double *qi = q + i * S;
            double pij = 0.0;
            for (int k = 0; k < S; ++k) pij += qi[k] * f[(int64_t)k * m + j];
            ctr4 r = draw(P->seed, (uint32_t)i, (uint32_t)j, ST_GENO, 0);
            unsigned code;
            if ((double)r.w[0] < miss_thr) {
                code = 3u;
            } else {
                double t = pij * two32;
                code = ((double)r.w[1] < t ? 1u : 0u) + ((double)r.w[2] < t ? 1u : 0u);
            }
            const int sh = 2 * (int)(i & 3);
            uint8_t *b = row + (i >> 2);
            *b = (uint8_t)((*b & ~(3u << sh)) | (code << sh));
        }
    }
    return 0;
}

/* Standard normal vector; stream selects an independent sequence. */
void synth_normal_vec(uint64_t seed, uint32_t stream, int64_t len, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < len; ++i) {
        ctr4 r = draw(seed, (uint32_t)i, stream, ST_VEC, (uint32_t)(i >> 32));
        out[i] = normal_from(r);
    }
}

/* Uniform vector on [lo, hi). */
void synth_uniform_vec(uint64_t seed, uint32_t stream, int64_t len, double lo, double hi, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < len; ++i) {
        ctr4 r = draw(seed, (uint32_t)i, stream, ST_VEC, 0x80000000u | (uint32_t)(i >> 32));
        out[i] = lo + (hi - lo) * (u53(r.w[0], r.w[1]) - 0x1p-53);
    }
}

/* The synthetic genotype model of section 2 (Algorithm 1) of the paper, in the
 * SNP-major packed layout: m markers (rows of the paper's matrix, SNPs here)
 * by n patients (samples).
 *  1. r sub-blocks: a marker range and a patient range, each the span between
 *     two uniform picks, set to one value k in {0, 1, 2}; later blocks overwrite
 *     earlier ones.
 *  2. "signal": nsignal draws, each setting a uniformly chosen entry to a
 *     uniform value in {0, 1, 2}.  Written per entry: an entry is hit with
 *     probability 1 - (1 - 1/(mn))^nsignal and then holds a uniform value,
 *     which is the distribution of each entry under the sequential draws.
 *  3. kinship: round(rkins m) times, a uniformly chosen marker row is replaced
 *     by a copy of another uniformly chosen row, in order.
 * No missing codes; padding samples are code 3. */
static inline uint32_t below(uint32_t x, uint32_t bound) { return (uint32_t)(((uint64_t)x * bound) >> 32); }

int synth_paper_model(int64_t n, int64_t m, int64_t stride, int32_t r, double nsignal, double rkins, uint64_t seed,
                      uint8_t *packed) {
    if (stride * 4 < n || stride % 16 != 0 || n <= 0 || m <= 0 || n > 0xFFFFFFFFLL || m > 0xFFFFFFFFLL) return -1;
    if (r < 0 || r > 4096) return -1;
    int64_t *blk = (int64_t *)malloc(sizeof(int64_t) * 5 * (size_t)(r > 0 ? r : 1));
    if (!blk) return -2;
    for (int32_t b = 0; b < r; ++b) {
        ctr4 x = draw(seed, (uint32_t)b, 0, ST_MODEL_BLK, 0);
        ctr4 y = draw(seed, (uint32_t)b, 0, ST_MODEL_BLK, 1);
        int64_t j1 = below(x.w[1], (uint32_t)m), j2 = below(x.w[2], (uint32_t)m);
        int64_t i1 = below(x.w[3], (uint32_t)n), i2 = below(y.w[0], (uint32_t)n);
        blk[5 * b + 0] = below(x.w[0], 3u);
        blk[5 * b + 1] = j1 < j2 ? j1 : j2;
        blk[5 * b + 2] = j1 < j2 ? j2 : j1;
        blk[5 * b + 3] = i1 < i2 ? i1 : i2;
        blk[5 * b + 4] = i1 < i2 ? i2 : i1;
    }
    const double mn = (double)n * (double)m;
    const double p_hit = nsignal > 0.0 ? -expm1(nsignal * log1p(-1.0 / mn)) : 0.0;
    const double hit_thr = p_hit * 4294967296.0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < m; ++j) {
        uint8_t *row = packed + j * stride;
        memset(row, 0xFF, (size_t)stride);
        for (int64_t i = 0; i < n; ++i) {
            unsigned code = 0u;
            for (int32_t b = 0; b < r; ++b)
                if (j >= blk[5 * b + 1] && j <= blk[5 * b + 2] && i >= blk[5 * b + 3] && i <= blk[5 * b + 4])
                    code = (unsigned)blk[5 * b];
            ctr4 x = draw(seed, (uint32_t)i, (uint32_t)j, ST_MODEL_SIG, 0);
            if ((double)x.w[0] < hit_thr) code = below(x.w[1], 3u);
            const int sh = 2 * (int)(i & 3);
            uint8_t *bp = row + (i >> 2);
            *bp = (uint8_t)((*bp & ~(3u << sh)) | (code << sh));
        }
    }
    const int64_t nkins = (int64_t)llround(rkins * (double)m);
    for (int64_t c = 0; c < nkins; ++c) {
        ctr4 x = draw(seed, (uint32_t)c, 0, ST_MODEL_KIN, 0);
        const int64_t dst = below(x.w[0], (uint32_t)m), src = below(x.w[1], (uint32_t)m);
        if (dst != src) memcpy(packed + dst * stride, packed + src * stride, (size_t)stride);
    }
    free(blk);
    return 0;
}
