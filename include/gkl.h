/*
 * gkl.h -- C ABI of the GB300 library for the top-k singular triplets of a
 * centred, standardised genotype matrix held 2-bit packed in GPU memory.
 *
 * Method: Golub-Kahan-Lanczos (GKL) bidiagonalisation with thick restart and
 * full (classical Gram-Schmidt applied twice, or with an adaptive second
 * pass), partial or one-sided reorthogonalisation, with a residual-norm
 * convergence test (Chen, Noack, Edelman, "Fast computation of the principal
 * components of genotype matrices in Julia", arXiv:1808.03374, section 3).
 *
 * Matrix.  G is n samples x m SNPs with entries 0, 1, 2 (allele counts) or
 * missing (section 1).  Storage is SNP-major, 2 bits per entry: the codes of
 * SNP j start at byte j*stride; sample i is in byte i>>2 at bits
 * 2*(i&3)..2*(i&3)+1; code 3 marks a missing entry.  stride is a multiple of 16
 * and >= ceil(n/4); entries i >= n inside a row must hold code 3.
 * The operator is
 *     A_ij = s_i * (g_ij - mu_j) * d_j * w_j   for observed g_ij, 0 if missing,
 * i.e. centred by the per-SNP mean mu_j, scaled by d_j (1/SD, or 0 for a
 * monomorphic SNP), with missing entries mean-imputed (the simplest imputation;
 * the paper names imputation as future work, section 5).  s (per sample) and w
 * (per SNP) are optional weights, 1 by default.
 *
 * Conventions for every entry point:
 *  - Return value: GKL_OK (0) or one of the GKL_ERR_* / GKL_NOT_CONVERGED /
 *    GKL_RANK_DEFICIENT codes.  Nothing is thrown across the ABI and no call
 *    aborts the process.  After a failure gkl_last_error() describes it.
 *  - Pointers marked (device) must be CUDA device (or managed) memory of the
 *    device that was current at gkl_init; pointers marked (host) are host
 *    memory; (host or device) accepts either.  A pointer of the wrong kind, or
 *    device memory of another GPU, is rejected with GKL_ERR_ARG.
 *  - All GPU work of a handle is ordered on the stream given to gkl_init (or
 *    gkl_set_stream).  Calls returning results in host memory synchronise that
 *    stream; gkl_matvec/gkl_rmatvec do not.
 *  - A handle is not thread-safe: one host thread at a time.
 */
#ifndef GKL_H
#define GKL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gkl_handle gkl_handle;

/* status codes */
#define GKL_OK 0
#define GKL_ERR_ARG 1        /* invalid argument (sizes, alignment, null pointer, memory kind) */
#define GKL_ERR_CUDA 2       /* a CUDA runtime call or kernel launch failed, or a kernel's bounded wait ran out */
#define GKL_ERR_NONFINITE 3  /* a Lanczos coefficient became NaN or Inf */
#define GKL_NOT_CONVERGED 4  /* maxit restart cycles ran out; outputs hold the best triplets so far */
#define GKL_ERR_GAP 5        /* gradient requested for singular values closer than min_relgap */
#define GKL_ERR_STATE 6      /* call out of order (e.g. gkl_grad before a converged gkl_svd, or after
                                gkl_set_weights changed the operator) */
#define GKL_RANK_DEFICIENT 7 /* the solve converged but A has numerical rank r < k: sigma_i for i >= r are
                                reported as 0 and gkl_info.rank = r; the outputs are otherwise complete */

/* arithmetic of the Lanczos vectors and the packed products */
#define GKL_FP64 0
#define GKL_FP32 1
/* block form (Golub-Luk-Overton block bidiagonalisation; section 5 names block
 * methods as future work): blocks of gkl_opts.block vectors, FP32 bases, FP64
 * projected matrix, full block reorthogonalisation, block products on the
 * tensor cores with each vector in 8 base-16 digits (finer than FP32), and a
 * final Rayleigh-Ritz step. */
#define GKL_BLOCK 2
/* the same with 4-digit (16-bit fixed point, the precision of a split hi+lo
 * BF16 pair) products during the iteration, 32 vectors per tensor-core pass;
 * the final Rayleigh-Ritz step and the residuals use 8 digits. */
#define GKL_BLOCK16 3

/* reorthogonalisation strategy (section 3, "choice of reorthogonalization strategy") */
#define GKL_REORTH_FULL 0     /* classical Gram-Schmidt twice against all previous vectors, every step */
#define GKL_REORTH_PARTIAL 1  /* omega-recurrence estimate of the orthogonality level; CGS2 only when it
                                 exceeds omega (and at the next step) */
#define GKL_REORTH_DGKS 2     /* full, with the second Gram-Schmidt pass only where the first removed more
                                 than half of the vector's squared norm (Daniel-Gragg-Kaufman-Stewart) */
#define GKL_REORTH_ONESIDED 3 /* one-sided: the vectors of the shorter side (u if n <= m, else v) are
                                 reorthogonalised at every step as in DGKS; the other side only when its
                                 omega-recurrence estimate exceeds omega (then also with the DGKS test) */

typedef struct gkl_opts {
    int32_t k;          /* number of singular triplets wanted, 1 <= k < ell */
    int32_t ell;        /* Krylov subspace size (restart length), k < ell <= min(n, m, 128) */
    int32_t k_keep;     /* Ritz vectors kept at a thick restart; 0 = k + (ell-k)/2 */
    int32_t reorth;     /* GKL_REORTH_*.  Block forms: FULL = two block Gram-Schmidt passes always,
                           any other value = the second pass only where the DGKS test asks for it */
    int32_t precision;  /* GKL_FP64, GKL_FP32, GKL_BLOCK or GKL_BLOCK16 */
    int32_t maxit;      /* maximum restart cycles (>= 1) */
    int32_t profile;    /* nonzero: time the packed-product kernels with CUDA events (gkl_info.ms_*) */
    int32_t block;      /* GKL_BLOCK: vectors per block, 1..32 (0 = 32); ell is rounded down to a
                           multiple of it and ell - k_keep must be one too; ignored otherwise */
    int32_t out_host;   /* nonzero: the U and V outputs of gkl_svd are host memory (the library copies
                           the results there and synchronises); zero: device memory */
    int32_t reserved0;  /* must be 0 */
    double tol;         /* converged when max_{i<k} r_i <= tol * sigma_1, r_i the Ritz residual */
    double omega;       /* PARTIAL / ONESIDED trigger level; 0 = min(1e-8 (FP64) or sqrt(eps_fp32) = 2^-12
                           (FP32), 10 tol), at least 10 unit roundoffs: the output's true residual follows the
                           orthogonality kept, about 0.1 omega sigma_1 */
    uint64_t seed;      /* counter-based generator seed for the start vector and breakdown restarts */
    const void* v0;     /* optional start vector (device, m entries of the precision's type); NULL = random */
} gkl_opts;

typedef struct gkl_info {
    int64_t matvec_pairs;  /* A.v and A^T.u pairs applied (block forms: vector pairs) */
    int32_t restarts;      /* thick restarts performed */
    int32_t cycles;        /* Lanczos cycles run (restarts + 1) */
    int32_t reorth_u;      /* steps whose u vector was reorthogonalised */
    int32_t reorth_v;      /* steps whose v vector was reorthogonalised */
    int32_t breakdowns;    /* zero Lanczos coefficients replaced by fresh vectors */
    int32_t converged;     /* 1 if the tolerance was met */
    double max_rel_resid;  /* max_{i<k} r_i / sigma_1 at exit */
    double dtheta1;        /* ||Delta theta||_1 = sum_{i<k} r_i (Table 3 of the paper) */
    double ms_total;       /* wall time of the call in milliseconds (CUDA events) */
    int64_t launches;      /* kernels launched by the call */
    int64_t n_mv;          /* A.v main-kernel launches timed (profile != 0) */
    int64_t n_rmv;         /* A^T.u main-kernel launches timed (profile != 0) */
    double ms_mv;          /* summed duration of the timed A.v main kernels */
    double ms_rmv;         /* summed duration of the timed A^T.u main kernels */
    int32_t jacobi_sweeps; /* most sweeps of the projected-matrix SVD in any cycle (+1000 if the FP64 Jacobi ran) */
    int32_t svd_fallbacks; /* cycles whose projected SVD needed the full FP64 Jacobi */
    int32_t svd_clusters;  /* ... of which because FP32 could not separate two singular values */
    int32_t rank;          /* numerical rank seen among the k values: k, or r < k with GKL_RANK_DEFICIENT */
    double ms_svd;         /* profile != 0: summed duration of the projected-SVD kernels */
    double ms_cgs;         /* profile != 0: summed duration of the reorthogonalisation kernels */
    int32_t second_u;      /* u reorthogonalisations that took a second Gram-Schmidt pass */
    int32_t second_v;      /* v reorthogonalisations that took a second pass (block forms: orthonormalisations) */
    int32_t refine_cycles; /* block forms: times the true residual after the Rayleigh-Ritz step missed tol and the
                              cycles went on with full-precision products (and a tighter estimate target) */
    int32_t reserved1;
} gkl_info;

/* Fill *o with defaults: k=10, ell=30, k_keep=0, DGKS (the adaptive second
 * pass, the paper's default), FP64, maxit=1000, profile=0, block=0,
 * out_host=0, tol=1e-10, omega=0, seed=1, v0=NULL. */
void gkl_opts_default(gkl_opts* o);

/* Per-SNP statistics of a packed matrix, computed on the GPU.
 * packed (device): m rows of stride bytes (layout above).
 * mu, scale (device, m doubles each, or NULL): mean of the observed codes and
 *   1/(population SD over the observed codes), 0 when the SD is 0 or no entry
 *   is observed (mu is then 0 too).
 * nobs (device, m int64, or NULL): observed-entry counts.
 * The integer sums are exact and mu = sum/nobs,
 *   scale = 1/sqrt((nobs*sum(g^2) - sum(g)^2) / nobs^2), each op IEEE-rounded.
 * stream: cudaStream_t or NULL for the legacy default stream.
 * Errors: GKL_ERR_ARG for n<1, m<1, stride%16, stride*4<n, misaligned packed. */
int gkl_colstats(const uint8_t* packed, int64_t n, int64_t m, int64_t stride,
                 double* mu, double* scale, int64_t* nobs, void* stream);

/* Create a handle on the current CUDA device.
 * packed (device, borrowed): not copied -- the caller keeps it alive and
 *   unchanged until gkl_destroy; must be 16-byte aligned.
 * mu, scale (host or device, m doubles each): copied in.  If both are NULL the
 *   handle computes them with gkl_colstats.
 * stream: cudaStream_t (as void*) used for all later work; NULL = default.
 * Allocates device memory for its own state (released by gkl_destroy),
 *   the largest part a list of the missing codes read by gkl_rmatvec: samples
 *   in blocks of 24,576, per (block, SNP) the missing samples' 16-bit offsets
 *   padded to a multiple of 8, about 2 bytes per missing code plus 16 bytes
 *   per (block, SNP) (4.2 GB for 2*10^9 missing codes at 200,000 x 1,000,000).
 *   It reads the packed buffer twice to build it and synchronises the stream.
 * Errors: GKL_ERR_ARG (sizes, alignment, exactly one of mu/scale NULL),
 *   GKL_ERR_CUDA (also when the tensor-core products cannot be set up). On
 *   error *h is NULL. */
int gkl_init(gkl_handle** h, const uint8_t* packed, int64_t n, int64_t m, int64_t stride,
             const double* mu, const double* scale, void* stream);

/* Change the stream used by later calls on h. */
int gkl_set_stream(gkl_handle* h, void* stream);

/* Per-sample weights s (n floats) and per-SNP weights w (m floats), host or
 * device, copied in; NULL restores weight 1 for that side.  This changes the
 * operator, so the triplets of an earlier gkl_svd no longer serve gkl_grad
 * (it returns GKL_ERR_STATE until the next converged gkl_svd). */
int gkl_set_weights(gkl_handle* h, const float* s, const float* w);

/* y = A v.  prec = GKL_FP64 (v, y double) or GKL_FP32 (float).
 * v (device, m entries), y (device, n entries); y must not alias v.
 * GKL_ERR_ARG if either is not device memory of the handle's GPU.
 * Stream-ordered; does not synchronise.  Deterministic: partial sums over SNP
 * chunks are combined in a fixed order. */
int gkl_matvec(gkl_handle* h, int prec, const void* v, void* y);

/* x = A^T u.  prec as for gkl_matvec; u (device, n entries), x (device, m);
 * GKL_ERR_ARG if either is not device memory of the handle's GPU.
 * Stream-ordered; does not synchronise.  Both precisions run on the tensor
 * cores in exact fixed point (u~ = s o u scaled by a power of two S > max|u~|
 * and rounded to 30 fractional bits for GKL_FP32, 57 for GKL_FP64; the sums are
 * exact integers, rounded once to the output type), with bounded pipeline
 * waits; a wait that runs out (never expected) is reported by the next call
 * that synchronises the stream (gkl_sync, gkl_svd, gkl_grad).
 * Deterministic. */
int gkl_rmatvec(gkl_handle* h, int prec, const void* u, void* x);

/* Block products of the block form on the tensor cores (tcgen05):
 *   transpose = 0:  Y (n x q) = A X,    X (m x q)
 *   transpose = 1:  Y (m x q) = A^T X,  X (n x q)
 * X, Y: device FP32, column-major with leading dimensions ldx, ldy (>= rows).
 * q: 1..32 vectors.  digits: 8 (each vector in 32-bit fixed point relative to
 *   its largest entry: finer than the FP32 input) or 4 (16-bit fixed point,
 *   the precision of a split hi+lo BF16 pair).  The genotypes are exact on the
 *   tensor cores and the accumulation is exact; the one rounding per entry is
 *   the fixed-point representation of the input block (|dx| <= 2^-(4 digits+1)
 *   of its largest entry) plus the final rounding to FP32.
 * Allocates its scratch per call (digit tiles, partial sums) and synchronises
 * the stream.  GKL_ERR_ARG if the tensor-core path is unavailable for this
 * handle (packed buffer not 16-byte aligned, or n > 524,000), X or Y is not
 * device memory of the handle's GPU, or arguments are out of range; GKL_ERR_CUDA on a CUDA error or a pipeline wait that ran out. */
int gkl_matmat(gkl_handle* h, int32_t transpose, int32_t q, int32_t digits, const float* X, int64_t ldx, float* Y,
               int64_t ldy);

/* y = A v, allocating no device memory (no handle needed).  The paper has no
 * counterpart: this is for callers that may not call cudaMalloc -- code whose
 * device memory is owned by a host application's own pool or arena, or loops
 * where an allocation's possible device-wide synchronisation is not allowed.
 * packed, mu, scale (device, of the current device): as for gkl_init (mu and
 *   scale are required here; gkl_colstats computes them).  No sample or SNP
 *   weights.
 * prec, v (device, m entries), y (device, n entries): as for gkl_matvec.
 * stream: cudaStream_t or NULL.
 * Scratch: a fixed 32 MiB device array inside the library, held by every GPU
 * that loads the library until the process exits.  A call needs
 * (chunks * 16*ceil(n/16) + 4*m) elements of the precision's type, chunks being
 * the SNP chunk count of the product over sample tiles of 256 words (FP64:
 * about 4 blocks per SM; FP32: the chunking, over 1 to 32 waves, that gives the
 * busiest SM the fewest rows).  On 152 SMs, n = 10,000, m = 100,000 takes 196
 * chunks in FP64 (18.9 MB) and 101 in FP32 (5.6 MB); 200,000 x 1,000,000 needs
 * more than the array holds in either precision;
 * sizes beyond 32 MiB less 256 bytes (the last 256 hold the error word of the
 * FP32 product's bounded TMA waits, which this call cannot report: it does
 * not synchronise) are rejected with GKL_ERR_ARG and a message that gives both
 * numbers.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents
 * (each call writes every element it reads, so nothing needs clearing); calls
 * that overlap on the GPU race on it and must be serialised by the caller.
 * Same results as gkl_matvec on the same inputs (same kernels).
 * Errors: GKL_ERR_ARG, GKL_ERR_CUDA; message via gkl_last_error(NULL). */
int gkl_matvec_noalloc(const uint8_t* packed, int64_t n, int64_t m, int64_t stride, const double* mu,
                       const double* scale, int prec, const void* v, void* y, void* stream);

/* Top-k singular triplets by thick-restarted GKL (section 3).
 * sigma (host, k doubles): singular values, descending.
 * U (n x k column-major, precision's type) and V (m x k): left and right
 *   singular vectors, in device memory, or in host memory when
 *   o->out_host != 0; the largest-magnitude entry of each V column is positive
 *   (first on ties) and U's column flips with it.  Either may be NULL.
 * resid (host, k doubles, or NULL): Ritz residuals r_i = beta_ell |P_{ell,i}|,
 *   an absolute error bound on sigma_i (section 3, convergence criteria).
 * info (host, or NULL): counters and the final residual level.
 * Synchronises the stream.  Returns GKL_OK, GKL_RANK_DEFICIENT (converged;
 * numerical rank r < k: sigma_i = 0 for i >= r, info->rank = r; a value counts
 * as zero when it is at most 1000 * (unit roundoff of the precision) *
 * sigma_1), GKL_NOT_CONVERGED (outputs hold the last Ritz triplets),
 * GKL_ERR_NONFINITE, GKL_ERR_ARG or GKL_ERR_CUDA.
 * The triplets (U, V, sigma) stay in the handle for gkl_scores and gkl_grad
 * (block forms: in FP32).
 * GKL_BLOCK / GKL_BLOCK16: U and V are float; for k <= 32 sigma, U, V come
 * from the final Rayleigh-Ritz step and resid holds the true residuals
 * ||A^T u_i - sigma_i v_i|| (8-digit products), otherwise the Ritz values and
 * the block residuals ||S_{s+1} P[last b rows, i]||; the convergence test uses
 * the block residuals; info->matvec_pairs counts vector pairs,
 * info->breakdowns the directions replaced by random vectors and
 * info->second_v the orthonormalisations that needed a second Gram-Schmidt
 * pass. */
int gkl_svd(gkl_handle* h, const gkl_opts* o, double* sigma, void* U, void* V,
            double* resid, gkl_info* info);

/* PC scores of the last successful gkl_svd: S = U diag(sigma) = A V_k (the
 * principal-component coordinates of the samples; section 1 of the paper).
 * S (n x k column-major, in the last solve's type: double after GKL_FP64,
 * float otherwise): device memory, or host memory when out_host != 0 (the
 * call then synchronises).  Errors: GKL_ERR_STATE (no successful solve since
 * the handle was created or its weights changed), GKL_ERR_ARG. */
int gkl_scores(gkl_handle* h, void* S, int32_t out_host);

/* Gradient of a loss L(sigma, S) on the triplets of the last converged
 * gkl_svd of h, with respect to the per-SNP weights w and per-sample weights s
 * of A = diag(s) A0 diag(w) (the paper has no differentiation; first-order
 * SVD perturbation theory).  S = U diag(sigma) = A V_k are the PC scores.
 * sigma_bar (host, k doubles, or NULL = 0): dL/dsigma_i.
 * scores_bar (device, n x k column-major in the last solve's type, or
 *   NULL = 0): dL/dS.  Each nonzero column i needs sigma_i separated from the
 *   other computed values and from the next Ritz value by min_relgap*sigma_1
 *   (else GKL_ERR_GAP); its adjoint involves a conjugate-gradient solve on the
 *   complement of V_k.
 * g_w (device, m entries) and g_s (device, n entries), either may be NULL:
 *   dL/dw and dL/ds in the last solve's type.  Weights must be nonzero.
 *   GKL_ERR_ARG if sigma_bar is not host memory, or scores_bar, g_w or g_s
 *   not device memory of the handle's GPU.
 * Synchronises the stream.  Errors: GKL_ERR_STATE (no converged solve, or the
 * weights changed since), GKL_ERR_GAP, GKL_NOT_CONVERGED (a solve did not
 * converge), GKL_ERR_ARG, GKL_ERR_CUDA (including a tensor-core product whose
 * bounded wait ran out). */
int gkl_grad(gkl_handle* h, const double* sigma_bar, const void* scores_bar, void* g_w, void* g_s,
             double min_relgap);

/* Synchronise the handle's stream and report what its kernels recorded since
 * the last synchronising call: GKL_ERR_CUDA if a CUDA error is pending or a
 * tensor-core product's bounded pipeline wait ran out (the record is then
 * cleared), else GKL_OK.  Use it after gkl_rmatvec / gkl_matvec sequences. */
int gkl_sync(gkl_handle* h);

/* Release the handle and all device memory it allocated (not `packed`). */
int gkl_destroy(gkl_handle* h);

/* Message of the last failure on h (or of the last failed gkl_init /
 * gkl_colstats / gkl_matvec_noalloc when h is NULL); never NULL. */
const char* gkl_last_error(const gkl_handle* h);

/* Library version string. */
const char* gkl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GKL_H */
