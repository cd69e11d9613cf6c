// Block form of thick-restarted GKL bidiagonalisation (Golub, Luk & Overton's
// block Lanczos bidiagonalisation, named as future work in section 5 of
// arXiv:1808.03374; the restart follows the paper's thick restart of section 3
// with a spike block in place of the spike column).
//
// Blocks of b columns, FP32 bases, FP64 projected quantities:
//   W = A V_j - U_{j-1} S_j^T            (after a restart: - U_kept C, C the spike block)
//   W <- W - U (U^T W) twice, W = U_j R_j  (orthonormalisation below)
//   Z = A^T U_j - V_j R_j^T
//   Z <- Z - V (V^T Z) twice, Z = V_{j+1} S_{j+1}
// so that A V = U T and A^T U = V T^T + V_{s+1} S_{s+1} E_s^T with T (ell x ell)
// block upper bidiagonal: R_j on the diagonal, S_{j+1}^T above it.  The SVD
// T = P Sigma Q^T gives Ritz triplets with residuals
//   || A^T u_i - sigma_i v_i || = || S_{s+1} P[last b rows, i] ||.
// A thick restart keeps k' Ritz vectors; T becomes diag(sigma_1..k') with the
// spike block C = (S_{s+1} P[last b rows, 0:k'])^T in the columns of V_{s+1}.
//
// Orthonormalisation of a block X (len x b) against a basis: CGS2, then the
// Gram matrix G = X^T X (FP32 products summed in FP64) is diagonalised in FP64
// on the host (b x b Jacobi), X <- X Z Lambda^{-1/2}; directions with
// Lambda_i <= 1e-8 Lambda_max (numerically dependent: a converged or exhausted
// subspace) are replaced by fresh counter-based random vectors; then CGS2
// again if any were replaced, and one Cholesky QR pass.  The factor R with
// X_before = X_after R is accumulated in FP64.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "epilogue.cuh"
#include "gkl_internal.cuh"

namespace gkl {

namespace {
constexpr int kGramRows = 32;   // rows per FP32 partial sum
constexpr int kMaxB = 32;       // block size limit (Gram kernel tile)
}

// ---- kernels ------------------------------------------------------------------

// part[blk][i + p j] = sum over the block's rows r of X[r + i ldx] Y[r + j ldy]
// (i < p <= 128, j < q <= 8 QC):
// FP32 products summed over 32-row chunks, the chunk sums added in FP64.  Each
// chunk is loaded into registers while the previous one is multiplied out of
// shared memory (two buffers, one barrier per chunk).  QC = 2 serves q <= 16
// without idle threads, QC = 4 q <= 32.
template <int QC>
__global__ void __launch_bounds__(256) k_gram_part(const float* __restrict__ X, int64_t ldx, int p,
                                                    const float* __restrict__ Y, int64_t ldy, int q, int64_t len,
                                                    int64_t rows_per_blk, double* __restrict__ part) {
    __shared__ float sx[2][kGramRows][129];
    __shared__ float sy[2][kGramRows][33];
    const int t = threadIdx.x, gi = t & 31, gj = t >> 5;
    const int lr = t & 31, lc = t >> 5;  // load role: row lr, columns lc + 8 k
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_blk;
    const int64_t r1 = min(len, r0 + rows_per_blk);
    double acc[4][QC];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < QC; ++c) acc[a][c] = 0.0;
    float xr[16], yr[QC];
    auto load = [&](int64_t rb) {
        const int64_t r = rb + lr;
        const bool ok = r < r1;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int c = lc + 8 * k;
            xr[k] = (ok && c < p) ? X[r + (int64_t)c * ldx] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < QC; ++k) {
            const int c = lc + 8 * k;
            yr[k] = (ok && c < q) ? Y[r + (int64_t)c * ldy] : 0.f;
        }
    };
    if (r0 < r1) load(r0);
    int buf = 0;
    for (int64_t rb = r0; rb < r1; rb += kGramRows, buf ^= 1) {
#pragma unroll
        for (int k = 0; k < 16; ++k) sx[buf][lr][lc + 8 * k] = xr[k];
#pragma unroll
        for (int k = 0; k < QC; ++k) sy[buf][lr][lc + 8 * k] = yr[k];
        __syncthreads();
        if (rb + kGramRows < r1) load(rb + kGramRows);
        float f[4][QC];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < QC; ++c) f[a][c] = 0.f;
#pragma unroll 8
        for (int rr = 0; rr < kGramRows; ++rr) {
            float xa[4], yc[QC];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = sx[buf][rr][gi + 32 * a];
#pragma unroll
            for (int c = 0; c < QC; ++c) yc[c] = sy[buf][rr][gj + 8 * c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < QC; ++c) f[a][c] = fmaf(xa[a], yc[c], f[a][c]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < QC; ++c) acc[a][c] += (double)f[a][c];
    }
    double* out = part + (int64_t)blockIdx.x * p * q;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < QC; ++c) {
            const int i = gi + 32 * a, j = gj + 8 * c;
            if (i < p && j < q) out[i + p * j] = acc[a][c];
        }
}

// out[e] = sum_blk part[blk][e] in a fixed order (deterministic): 32 elements
// per block; warp w sums blocks w, w + 8, ... (coalesced rows of 32 doubles),
// then the eight warp sums are added in warp order.
__global__ void __launch_bounds__(256) k_gram_sum(const double* __restrict__ part, int nblk, int pq,
                                                  double* __restrict__ out) {
    __shared__ double ws[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (e < pq)
        for (int b = w; b < nblk; b += 8) s += part[(int64_t)b * pq + e];
    ws[w][lane] = s;
    __syncthreads();
    if (w == 0 && e < pq) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += ws[k][lane];
        out[e] = t;
    }
}

// X[:, 0:q] <- alpha X[:, 0:q] + beta Y[:, 0:p] C  (C p x q, FP64, column-major with
// leading dimension ldc), per row.
// X and Y may be the same buffer only with alpha = 0 (X <- beta X C).  C is
// held row by row in shared memory (FP32, 32 columns) and read as float4.
__global__ void __launch_bounds__(256) k_block_axpy(float* X, int64_t ldx, int q, const float* Y,
                                                     int64_t ldy, int p, const double* __restrict__ C, int ldc,
                                                     float alpha, float beta, int64_t len) {
    __shared__ __align__(16) float sc[128 * kMaxB];
    for (int e = threadIdx.x; e < p * kMaxB; e += blockDim.x) {
        const int i = e / kMaxB, j = e % kMaxB;
        sc[e] = j < q ? (float)C[i + ldc * j] : 0.f;
    }
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < len; r += (int64_t)gridDim.x * blockDim.x) {
        float acc[kMaxB];
#pragma unroll
        for (int j = 0; j < kMaxB; ++j) acc[j] = 0.f;
        for (int i0 = 0; i0 < p; i0 += 4) {
            float y[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) y[u] = i0 + u < p ? Y[r + (int64_t)(i0 + u) * ldy] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (i0 + u >= p) break;
                const float4* cr = reinterpret_cast<const float4*>(sc + (i0 + u) * kMaxB);
#pragma unroll
                for (int j4 = 0; j4 < kMaxB / 4; ++j4) {
                    const float4 cv = cr[j4];
                    acc[4 * j4] = fmaf(y[u], cv.x, acc[4 * j4]);
                    acc[4 * j4 + 1] = fmaf(y[u], cv.y, acc[4 * j4 + 1]);
                    acc[4 * j4 + 2] = fmaf(y[u], cv.z, acc[4 * j4 + 2]);
                    acc[4 * j4 + 3] = fmaf(y[u], cv.w, acc[4 * j4 + 3]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kMaxB; ++j)
            if (j < q) {
                float* x = X + r + (int64_t)j * ldx;
                *x = (alpha == 0.f ? 0.f : alpha * *x) + beta * acc[j];
            }
    }
}

// X[:, j] <- uniform(-1, 1) from the counter-based generator, for the columns
// flagged in `cols` (bit j).
__global__ void k_block_random(float* __restrict__ X, int64_t ldx, int64_t len, uint32_t cols, uint64_t seed,
                               uint32_t draw) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < len; r += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < kMaxB; ++j)
            if (cols & (1u << j)) X[r + (int64_t)j * ldx] = (float)uniform_pm1(seed, draw + (uint32_t)j, r);
}


// Restart projection of the kept Ritz pairs, in FP64: M = T Q[:, :kk] (ell x kk)
// and Tn = P[:, :kk]^T M (kk x kk), so that A V Q_kk = (U P_kk) Tn up to the
// coupling to the discarded pairs (small when P and Q are accurate Ritz
// vectors); Tn is diagonal only when P and Q are exact.
__global__ void __launch_bounds__(128) k_tq(const double* __restrict__ T, const double* __restrict__ Q, int ell,
                                            int kk, double* __restrict__ M) {
    const int j = blockIdx.x;
    for (int r = threadIdx.x; r < ell; r += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < ell; ++c) s += T[r + (int64_t)c * ell] * Q[c + (int64_t)j * ell];
        M[r + (int64_t)j * ell] = s;
    }
}
__global__ void __launch_bounds__(128) k_ptm(const double* __restrict__ P, const double* __restrict__ M, int ell,
                                             int kk, double* __restrict__ Tn) {
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < kk; i += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < ell; ++r) s += P[r + (int64_t)i * ell] * M[r + (int64_t)j * ell];
        Tn[i + (int64_t)j * kk] = s;
    }
}

// ---- batched block products (every code decoded once for all q vectors) -------

// ---- host linear algebra (b x b, FP64) -----------------------------------------

// Symmetric eigen-decomposition by cyclic Jacobi: G = Z diag(lam) Z^T.
static void sym_eig(int q, std::vector<double> G, std::vector<double>& lam, std::vector<double>& Z) {
    Z.assign((size_t)q * q, 0.0);
    for (int i = 0; i < q; ++i) Z[i + q * i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int j = 0; j < q; ++j)
            for (int i = 0; i < q; ++i) (i == j ? dia : off) += G[i + q * j] * G[i + q * j];
        if (off <= 1e-30 * dia || off == 0.0) break;
        for (int a = 0; a < q - 1; ++a)
            for (int b = a + 1; b < q; ++b) {
                const double gab = G[a + q * b];
                if (gab == 0.0) continue;
                const double zeta = (G[b + q * b] - G[a + q * a]) / (2.0 * gab);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int k = 0; k < q; ++k) {  // G <- J^T G J
                    const double x = G[k + q * a], y = G[k + q * b];
                    G[k + q * a] = c * x - s * y;
                    G[k + q * b] = s * x + c * y;
                }
                for (int k = 0; k < q; ++k) {
                    const double x = G[a + q * k], y = G[b + q * k];
                    G[a + q * k] = c * x - s * y;
                    G[b + q * k] = s * x + c * y;
                }
                for (int k = 0; k < q; ++k) {
                    const double x = Z[k + q * a], y = Z[k + q * b];
                    Z[k + q * a] = c * x - s * y;
                    Z[k + q * b] = s * x + c * y;
                }
            }
    }
    lam.resize(q);
    for (int i = 0; i < q; ++i) lam[i] = G[i + q * i];
}

// Cholesky G = R^T R (R upper, column-major); false if not positive definite.
static bool cholesky(int q, const std::vector<double>& G, std::vector<double>& R) {
    R.assign((size_t)q * q, 0.0);
    for (int j = 0; j < q; ++j) {
        double d = G[j + q * j];
        for (int k = 0; k < j; ++k) d -= R[k + q * j] * R[k + q * j];
        if (!(d > 0.0)) return false;
        const double rjj = std::sqrt(d);
        R[j + q * j] = rjj;
        for (int i = j + 1; i < q; ++i) {
            double s = G[j + q * i];
            for (int k = 0; k < j; ++k) s -= R[k + q * j] * R[k + q * i];
            R[j + q * i] = s / rjj;
        }
    }
    return true;
}

// Inverse of an upper-triangular R (column-major).
static std::vector<double> inv_upper(int q, const std::vector<double>& R) {
    std::vector<double> X((size_t)q * q, 0.0);
    for (int j = 0; j < q; ++j) {
        X[j + q * j] = 1.0 / R[j + q * j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= j; ++k) s += R[i + q * k] * X[k + q * j];
            X[i + q * j] = -s / R[i + q * i];
        }
    }
    return X;
}

static std::vector<double> matmul(int q, const std::vector<double>& A, const std::vector<double>& B) {
    std::vector<double> C((size_t)q * q, 0.0);
    for (int j = 0; j < q; ++j)
        for (int k = 0; k < q; ++k) {
            const double b = B[k + q * j];
            if (b != 0.0)
                for (int i = 0; i < q; ++i) C[i + q * j] += A[i + q * k] * b;
        }
    return C;
}

// ---- block driver -----------------------------------------------------------------

struct BlockCtx {
    gkl_handle* h;
    cudaStream_t st;
    double* d_part;    // Gram partials
    double* d_small;   // p x q FP64 results / coefficient uploads
    void* tc_scratch;  // tensor-core products: digit tiles, partials
    int tc_digits;     // digits per vector of the tensor-core products
    int nblk_max;
    uint64_t seed;
    uint32_t draw;
    int launches;
    int deflations;
    int cgs_second;    // orthonormalisations that needed a second Gram-Schmidt pass
    int64_t products;
    // profile: CUDA events around each main tensor-core kernel (pairs), kept
    // until the solve's final synchronisation
    bool profile = false;
    bool cgs2_always = false;  // GKL_REORTH_FULL: always two Gram-Schmidt passes
    std::vector<cudaEvent_t> ev_mv, ev_rmv;
    cudaEvent_t next_event(std::vector<cudaEvent_t>& pool, size_t& used) {
        if (used == pool.size()) {
            cudaEvent_t ev = nullptr;
            cudaEventCreate(&ev);
            pool.push_back(ev);
        }
        return pool[used++];
    }
    size_t used_mv = 0, used_rmv = 0;
    ~BlockCtx() {
        for (auto* pool : {&ev_mv, &ev_rmv})
            for (cudaEvent_t ev : *pool)
                if (ev) cudaEventDestroy(ev);
    }
};

// Summed elapsed time of the recorded (begin, end) pairs; n = number of pairs.
static double sum_event_pairs(const std::vector<cudaEvent_t>& pool, size_t used, int64_t* n) {
    double ms = 0.0;
    for (size_t i = 0; i + 1 < used; i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pool[i], pool[i + 1]) == cudaSuccess) ms += t;
    }
    *n = (int64_t)(used / 2);
    return ms;
}

static int gram_blocks(const BlockCtx& c, int64_t len) {
    // two resident blocks per SM (registers), at least 256 rows each
    return (int)std::max<int64_t>(1, std::min<int64_t>(2 * (int64_t)c.h->num_sms, (len + 255) / 256));
}

// C (p x q, device FP64) = X^T Y
static cudaError_t gram(BlockCtx& c, const float* X, int64_t ldx, int p, const float* Y, int64_t ldy, int q,
                        int64_t len, double* C) {
    const int nb = gram_blocks(c, len);
    const int64_t rpb = (len + nb - 1) / nb;
    if (q <= 16)
        k_gram_part<2><<<nb, 256, 0, c.st>>>(X, ldx, p, Y, ldy, q, len, rpb, c.d_part);
    else
        k_gram_part<4><<<nb, 256, 0, c.st>>>(X, ldx, p, Y, ldy, q, len, rpb, c.d_part);
    k_gram_sum<<<(p * q + 31) / 32, 256, 0, c.st>>>(c.d_part, nb, p * q, C);
    c.launches += 2;
    return cudaGetLastError();
}

static int axpy_grid(const BlockCtx& c, int64_t len) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(4 * c.h->num_sms, (len + 255) / 256));
}

// One classical Gram-Schmidt pass X <- X - B (B^T X), B = len x nbasis; the
// coefficients are left in C (nbasis x q).
static cudaError_t cgs_pass(BlockCtx& c, float* X, int64_t ldx, int q, const float* B, int64_t ldb, int nbasis,
                            int64_t len, double* C) {
    cudaError_t e = gram(c, B, ldb, nbasis, X, ldx, q, len, C);
    if (e != cudaSuccess) return e;
    k_block_axpy<<<axpy_grid(c, len), 256, 0, c.st>>>(X, ldx, q, B, ldb, nbasis, C, nbasis, 1.f, -1.f, len);
    c.launches += 1;
    return cudaGetLastError();
}

// X <- X - B (B^T X) twice
static cudaError_t cgs2(BlockCtx& c, float* X, int64_t ldx, int q, const float* B, int64_t ldb, int nbasis,
                        int64_t len) {
    if (nbasis == 0) return cudaSuccess;
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e = cgs_pass(c, X, ldx, q, B, ldb, nbasis, len, c.d_small);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static cudaError_t upload(BlockCtx& c, const std::vector<double>& hm, double* dst) {
    return cudaMemcpyAsync(dst, hm.data(), sizeof(double) * hm.size(), cudaMemcpyHostToDevice, c.st);
}

static cudaError_t download(BlockCtx& c, const double* src, std::vector<double>& hm, size_t count) {
    hm.resize(count);
    cudaError_t e = cudaMemcpyAsync(hm.data(), src, sizeof(double) * count, cudaMemcpyDeviceToHost, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    return e;
}

// Orthonormalise X (len x q) against B (len x nb); returns R (q x q, column-major)
// with X_before = X_after R (up to the replaced directions, whose rows of R are 0).
static cudaError_t orthonormalize_once(BlockCtx& c, float* X, int64_t ldx, int q, const float* B, int64_t ldb,
                                       int nb, int64_t len, std::vector<double>& R, bool& chol_ok);

// The eigen step, replacement and Cholesky pass below are repeated (at most
// three times) while the Cholesky pass meets a matrix that is not positive
// definite in FP64 -- possible when replaced and kept directions are nearly
// dependent after the FP32 products; each repetition starts from the block the
// previous one produced, and the factors multiply.
static cudaError_t orthonormalize(BlockCtx& c, float* X, int64_t ldx, int q, const float* B, int64_t ldb, int nb,
                                  int64_t len, std::vector<double>& R) {
    R.assign((size_t)q * q, 0.0);
    for (int i = 0; i < q; ++i) R[i + (size_t)q * i] = 1.0;
    for (int attempt = 0; attempt < 3; ++attempt) {
        std::vector<double> Ri;
        bool ok = false;
        cudaError_t e = orthonormalize_once(c, X, ldx, q, B, ldb, nb, len, Ri, ok);
        if (e != cudaSuccess) return e;
        R = matmul(q, Ri, R);
        if (ok) return cudaSuccess;
    }
    return cudaErrorInvalidValue;
}

static cudaError_t orthonormalize_once(BlockCtx& c, float* X, int64_t ldx, int q, const float* B, int64_t ldb,
                                       int nb, int64_t len, std::vector<double>& R, bool& chol_ok) {
    chol_ok = false;
    // Gram-Schmidt against B, a second pass only where the first removed more
    // than half of a column's squared norm (the Daniel-Gragg-Kaufman-Stewart
    // criterion; with B orthonormal, ||x||^2 = ||x'||^2 + ||c||^2 for the
    // coefficients c of the first pass); then G = X^T X
    std::vector<double> G, lam, Z, Cf;
    double* Gd = c.d_small + GKL_MAX_ELL * kMaxB;
    cudaError_t e = cudaSuccess;
    if (nb > 0) e = cgs_pass(c, X, ldx, q, B, ldb, nb, len, c.d_small);
    if (e == cudaSuccess) e = gram(c, X, ldx, q, X, ldx, q, len, Gd);
    if (e == cudaSuccess && nb > 0) {
        Cf.resize((size_t)nb * q);
        e = cudaMemcpyAsync(Cf.data(), c.d_small, sizeof(double) * nb * q, cudaMemcpyDeviceToHost, c.st);
    }
    if (e == cudaSuccess) e = download(c, Gd, G, (size_t)q * q);
    if (e != cudaSuccess) return e;
    bool again = c.cgs2_always && nb > 0;
    for (int j = 0; j < q && nb > 0; ++j) {
        double cc = 0.0;
        for (int i = 0; i < nb; ++i) cc += Cf[i + (size_t)nb * j] * Cf[i + (size_t)nb * j];
        if (!(cc <= G[j + (size_t)q * j])) again = true;
    }
    if (again) {
        ++c.cgs_second;
        e = cgs_pass(c, X, ldx, q, B, ldb, nb, len, c.d_small);
        if (e == cudaSuccess) e = gram(c, X, ldx, q, X, ldx, q, len, Gd);
        if (e == cudaSuccess) e = download(c, Gd, G, (size_t)q * q);
        if (e != cudaSuccess) return e;
    }
    sym_eig(q, G, lam, Z);
    // descending eigenvalues, so that replaced directions come last
    std::vector<int> ord(q);
    for (int i = 0; i < q; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return lam[a] > lam[b]; });
    const double lmax = std::max(0.0, lam[ord[0]]);
    std::vector<double> M((size_t)q * q, 0.0), R1((size_t)q * q, 0.0);
    uint32_t repl = 0;
    for (int jj = 0; jj < q; ++jj) {
        const int i = ord[jj];
        if (lmax > 0.0 && lam[i] > 1e-8 * lmax) {
            const double sl = std::sqrt(lam[i]);
            for (int r = 0; r < q; ++r) {
                M[r + q * jj] = Z[r + q * i] / sl;
                R1[jj + q * r] = sl * Z[r + q * i];
            }
        } else {
            repl |= 1u << jj;
        }
    }
    e = upload(c, M, c.d_small);
    if (e != cudaSuccess) return e;
    k_block_axpy<<<axpy_grid(c, len), 256, 0, c.st>>>(X, ldx, q, X, ldx, q, c.d_small, q, 0.f, 1.f, len);
    c.launches += 1;
    if (repl) {
        k_block_random<<<axpy_grid(c, len), 256, 0, c.st>>>(X, ldx, len, repl, c.seed, c.draw);
        c.draw += kMaxB;
        c.launches += 1;
        c.deflations += __builtin_popcount(repl);
        e = cgs2(c, X, ldx, q, B, ldb, nb, len);
        if (e != cudaSuccess) return e;
    }
    // one Cholesky QR pass on the (now well-conditioned) block
    if ((e = gram(c, X, ldx, q, X, ldx, q, len, c.d_small)) != cudaSuccess) return e;
    if ((e = download(c, c.d_small, G, (size_t)q * q)) != cudaSuccess) return e;
    std::vector<double> R2;
    if (!cholesky(q, G, R2)) {  // leave X as the eigen step made it; the caller repeats
        R = R1;
        return cudaGetLastError();
    }
    const std::vector<double> R2i = inv_upper(q, R2);
    if ((e = upload(c, R2i, c.d_small)) != cudaSuccess) return e;
    k_block_axpy<<<axpy_grid(c, len), 256, 0, c.st>>>(X, ldx, q, X, ldx, q, c.d_small, q, 0.f, 1.f, len);
    c.launches += 1;
    R = matmul(q, R2, R1);
    chol_ok = true;
    return cudaGetLastError();
}

// Y[:, 0:q] = A X[:, 0:q] (forward) or A^T X (transpose) on the tensor cores, at
// most 128 / D vectors per pass.
static cudaError_t block_product(BlockCtx& c, bool transpose, const float* X, int64_t ldx, float* Y, int64_t ldy,
                                 int q) {
    gkl_handle* h = c.h;
    const int per = 128 / c.tc_digits;
    for (int c0 = 0; c0 < q; c0 += per) {
        int nl = 0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c.profile) {
            auto& pool = transpose ? c.ev_rmv : c.ev_mv;
            auto& used = transpose ? c.used_rmv : c.used_mv;
            e0 = c.next_event(pool, used);
            e1 = c.next_event(pool, used);
        }
        cudaError_t e = launch_block_product_tc(h, transpose, X + (int64_t)c0 * ldx, ldx, std::min(per, q - c0),
                                                c.tc_digits, Y + (int64_t)c0 * ldy, ldy, c.tc_scratch, &nl, e0, e1);
        if (e != cudaSuccess) return e;
        c.launches += nl;
    }
    if (!transpose) c.products += q;
    return cudaSuccess;
}

static int64_t round32(int64_t x) { return (x + 31) / 32 * 32; }

int run_block(gkl_handle* h, const gkl_opts* o, double* sigma, float* Uout, float* Vout, double* resid,
              gkl_info* info) {
    const int64_t n = h->n, m = h->m;
    const int b = o->block ? o->block : 32;
    const int k = o->k;
    if (b < 1 || b > kMaxB) return set_err(h, GKL_ERR_ARG, "block size %d outside [1, %d]", b, kMaxB);
    const int ell = o->ell / b * b;
    if (k < 1 || ell < 2 * b || ell > GKL_MAX_ELL || k >= ell || ell > std::min(n, m))
        return set_err(h, GKL_ERR_ARG, "need 1 <= k < ell, 2b <= ell <= min(n, m, %d) (ell rounded down to a multiple of b)",
                       GKL_MAX_ELL);
    int kk = o->k_keep;
    if (kk == 0) kk = std::max(k, ell - b * (int)((ell - k + 2 * b - 1) / (2 * b)));
    if (kk < k || kk >= ell || (ell - kk) % b != 0)
        return set_err(h, GKL_ERR_ARG, "k_keep must satisfy k <= k_keep < ell with ell - k_keep a multiple of b");
    if (!(o->tol > 0.0) || o->maxit < 1) return set_err(h, GKL_ERR_ARG, "tol must be > 0 and maxit >= 1");
    const int64_t ldu = round32(n), ldv = round32(m);
    const size_t ell2 = (size_t)ell * ell;
    const int nblk = 4 * h->num_sms;
    // device workspace
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off += (bytes + 255) & ~(size_t)255;
        return o2;
    };
    const size_t oU = take(sizeof(float) * ldu * ell), oU2 = take(sizeof(float) * ldu * ell);
    const size_t oV = take(sizeof(float) * ldv * (ell + b)), oV2 = take(sizeof(float) * ldv * (ell + b));
    const size_t oT = take(sizeof(double) * ell2), oP = take(sizeof(double) * 4 * ell2),
                 oQ = take(sizeof(double) * ell2), oRw = take(sizeof(double) * 8 * ell2);
    const size_t oSc = take(sizeof(DevScal)), oCo = take(sizeof(CycleOut));
    const size_t oPart = take(sizeof(double) * (size_t)nblk * GKL_MAX_ELL * kMaxB),
                 oSmall = take(sizeof(double) * 2 * GKL_MAX_ELL * kMaxB), oSigns = take(sizeof(int) * GKL_MAX_ELL);
    const size_t oOutU = take(sizeof(float) * n * k), oOutV = take(sizeof(float) * m * k);
    // products: tcgen05 with 8 digits per vector (finer than FP32), or 4 digits
    // (GKL_BLOCK16) during the iteration
    if (!block_tc_prepare(h))
        return set_err(h, GKL_ERR_ARG, "the block form needs the tensor-core products (n <= 524,000 samples)");
    const int tc_digits = o->precision == GKL_BLOCK16 ? 4 : 8;
    const size_t oBpart = take(block_tc_scratch_bytes(h, kMaxB));
    void* ws = nullptr;
    if (cudaMalloc(&ws, off) != cudaSuccess) return set_err(h, GKL_ERR_CUDA, "block workspace of %zu bytes", off);
    char* W = static_cast<char*>(ws);
    float* U = reinterpret_cast<float*>(W + oU);
    float* U2 = reinterpret_cast<float*>(W + oU2);
    float* V = reinterpret_cast<float*>(W + oV);
    float* V2 = reinterpret_cast<float*>(W + oV2);
    Sv sv{};
    sv.n = n;
    sv.m = m;
    sv.ldu = ldu;
    sv.ldv = ldv;
    sv.ell = ell;
    sv.kk = k;  // the projected SVD refines (and checks) the k wanted triplets
    sv.k = k;
    sv.prec = GKL_FP32;
    sv.fp32_only = 1;
    sv.B = reinterpret_cast<double*>(W + oT);
    sv.P = reinterpret_cast<double*>(W + oP);
    sv.Q = reinterpret_cast<double*>(W + oQ);
    sv.rw = reinterpret_cast<double*>(W + oRw);
    sv.sc = reinterpret_cast<DevScal*>(W + oSc);
    sv.co = reinterpret_cast<CycleOut*>(W + oCo);
    sv.eps_w = 5.9604644775390625e-08;
    sv.tol = o->tol;
    BlockCtx c{h,
               h->stream,
               reinterpret_cast<double*>(W + oPart),
               reinterpret_cast<double*>(W + oSmall),
               static_cast<void*>(W + oBpart),
               tc_digits,
               nblk,
               o->seed,
               0x42000000u,
               0,
               0,
               0,
               0};
    c.profile = o->profile != 0;
    c.cgs2_always = o->reorth == GKL_REORTH_FULL;
    cudaError_t e = cudaMemsetAsync(sv.sc, 0, sizeof(DevScal), c.st);
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, c.st);
    std::vector<double> T(ell2, 0.0), R, S, P, sg;
    std::vector<double> Slast;
    CycleOut* ho = h->host_out;
    int cycle = 0, restarts = 0, converged = 0, svd_fb = 0, svd_fp64 = 0, max_sweeps = 0, svd_unrefined = 0,
        svd_uncontracted = 0;
    double maxrel = 0.0, dtheta = 0.0;
    std::vector<double> res(k, 0.0);
    auto fail = [&](const char* what) {
        cudaFree(ws);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return e != cudaSuccess ? cuda_err(h, e, what) : set_err(h, GKL_ERR_CUDA, "%s", what);
    };
    // start block: V[:, 0:b] random (or v0 in column 0), orthonormalised
    if (e == cudaSuccess) {
        k_block_random<<<axpy_grid(c, m), 256, 0, c.st>>>(V, ldv, m, b == 32 ? 0xFFFFFFFFu : ((1u << b) - 1u), c.seed,
                                                          c.draw);
        c.draw += kMaxB;
        if (o->v0) e = cudaMemcpyAsync(V, o->v0, sizeof(float) * m, cudaMemcpyDeviceToDevice, c.st);
    }
    if (e == cudaSuccess) e = orthonormalize(c, V, ldv, b, nullptr, ldv, 0, m, R);
    if (e != cudaSuccess) return fail("block start");
    // output: U P[:, :k], V Q[:, :k]; for k <= 32 refined by one Rayleigh-Ritz
    // step on span(V Q[:, :k]) with FP32-grade products (W = A V_k, W^T W = Y
    // Lambda Y^T in FP64, sigma = sqrt(lambda), V = V_k Y, U = W Y / sigma),
    // whose singular values are accurate to the square of the subspace angle,
    // and the true residuals ||A^T u_i - sigma_i v_i|| from one more product
    float* Uo = reinterpret_cast<float*>(W + oOutU);
    float* Vo = reinterpret_cast<float*>(W + oOutV);
    bool true_resid = false;  // maxrel holds the true residual (else the Lanczos estimate)
    auto finalize = [&]() -> cudaError_t {
    const int digits_iter = c.tc_digits;
    c.tc_digits = 8;  // the Rayleigh-Ritz step and the residuals at full precision
    cudaError_t e = cudaSuccess;
    true_resid = false;
    if (k <= kMaxB) {
        float* Vk = V2;  // m x k (ldv)
        float* Wk = U2;  // n x k (ldu)
        std::vector<double> G, lam, Y, Rk;
        e = launch_rotate<float>(c.st, V, ldv, ell, sv.Q, ell, k, Vk, ldv, m);
        if (e == cudaSuccess) e = orthonormalize(c, Vk, ldv, k, nullptr, ldv, 0, m, Rk);
        if (e == cudaSuccess) e = block_product(c, false, Vk, ldv, Wk, ldu, k);
        if (e == cudaSuccess) e = gram(c, Wk, ldu, k, Wk, ldu, k, n, c.d_small);
        if (e == cudaSuccess) e = download(c, c.d_small, G, (size_t)k * k);
        if (e != cudaSuccess) return e;
        sym_eig(k, G, lam, Y);
        std::vector<int> ord(k);
        for (int i = 0; i < k; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](int a, int b2) { return lam[a] > lam[b2]; });
        std::vector<double> Cv((size_t)k * k), Cu((size_t)k * k), Cs((size_t)k * k, 0.0);
        for (int j = 0; j < k; ++j) {
            const double sj = std::sqrt(std::max(0.0, lam[ord[j]]));
            sg[j] = sj;
            for (int r = 0; r < k; ++r) {
                Cv[r + (size_t)k * j] = Y[r + (size_t)k * ord[j]];
                Cu[r + (size_t)k * j] = sj > 0.0 ? Y[r + (size_t)k * ord[j]] / sj : 0.0;
            }
            Cs[j + (size_t)k * j] = sj;
        }
        e = upload(c, Cv, c.d_small);
        if (e == cudaSuccess) {
            k_block_axpy<<<axpy_grid(c, m), 256, 0, c.st>>>(Vo, m, k, Vk, ldv, k, c.d_small, k, 0.f, 1.f, m);
            e = cudaStreamSynchronize(c.st);  // d_small is reused below
        }
        if (e == cudaSuccess) e = upload(c, Cu, c.d_small);
        if (e == cudaSuccess) {
            k_block_axpy<<<axpy_grid(c, n), 256, 0, c.st>>>(Uo, n, k, Wk, ldu, k, c.d_small, k, 0.f, 1.f, n);
            e = cudaStreamSynchronize(c.st);
        }
        // true residuals: Z = A^T U - V diag(sigma), r_i = ||Z_i||
        if (e == cudaSuccess) e = block_product(c, true, Uo, n, Vk, ldv, k);
        if (e == cudaSuccess) e = upload(c, Cs, c.d_small);
        if (e == cudaSuccess) {
            k_block_axpy<<<axpy_grid(c, m), 256, 0, c.st>>>(Vk, ldv, k, Vo, m, k, c.d_small, k, 1.f, -1.f, m);
            e = cudaStreamSynchronize(c.st);
        }
        if (e == cudaSuccess) e = gram(c, Vk, ldv, k, Vk, ldv, k, m, c.d_small);
        if (e == cudaSuccess) e = download(c, c.d_small, G, (size_t)k * k);
        if (e != cudaSuccess) return e;
        c.launches += 3;
        double mxr = 0.0, sumr = 0.0;
        for (int i = 0; i < k; ++i) {
            res[i] = std::sqrt(std::max(0.0, G[i + (size_t)k * i]));
            mxr = std::max(mxr, res[i]);
            sumr += res[i];
        }
        maxrel = sg[0] > 0.0 ? mxr / sg[0] : 0.0;
        dtheta = sumr;
        true_resid = true;
    } else {
        e = launch_rotate<float>(c.st, U, ldu, ell, sv.P, ell, k, Uo, n, n);
        if (e == cudaSuccess) e = launch_rotate<float>(c.st, V, ldv, ell, sv.Q, ell, k, Vo, m, m);
    }
    c.tc_digits = digits_iter;
    return e;
    };
    double est_tol = o->tol;  // target of the Lanczos estimate; halved when the true residual misses tol
    int refines = 0;
    bool fresh = false;  // this cycle starts from a single start block (cycle 0, explicit restart)
    for (cycle = 0; cycle < o->maxit; ++cycle) {
        const int c0 = cycle == 0 || fresh ? 0 : kk;
        fresh = false;
        for (int j0 = c0; j0 < ell; j0 += b) {
            float* Wb = U + (int64_t)j0 * ldu;
            cudaEventRecord(ev1, c.st);
            if ((e = block_product(c, false, V + (int64_t)j0 * ldv, ldv, Wb, ldu, b)) != cudaSuccess)
                return fail("A V block");
            if (j0 > 0) {  // W -= U[:, 0:j0] T[0:j0, j0:j0+b]
                std::vector<double> Cs((size_t)j0 * b);
                for (int cc = 0; cc < b; ++cc)
                    for (int r = 0; r < j0; ++r) Cs[r + (size_t)j0 * cc] = T[r + (size_t)ell * (j0 + cc)];
                if ((e = upload(c, Cs, c.d_small)) != cudaSuccess) return fail("coupling upload");
                k_block_axpy<<<axpy_grid(c, n), 256, 0, c.st>>>(Wb, ldu, b, U, ldu, j0, c.d_small, j0, 1.f, -1.f, n);
                c.launches += 1;
            }
            if ((e = orthonormalize(c, Wb, ldu, b, U, ldu, j0, n, R)) != cudaSuccess) return fail("U block");
            for (int cc = 0; cc < b; ++cc)
                for (int r = 0; r < b; ++r) T[(j0 + r) + (size_t)ell * (j0 + cc)] = R[r + (size_t)b * cc];
            float* Zb = V + (int64_t)(j0 + b) * ldv;
            if ((e = block_product(c, true, Wb, ldu, Zb, ldv, b)) != cudaSuccess) return fail("A^T U block");
            {  // Z -= V[:, j0:j0+b] R^T
                std::vector<double> Rt((size_t)b * b);
                for (int i = 0; i < b; ++i)
                    for (int jj = 0; jj < b; ++jj) Rt[i + (size_t)b * jj] = R[jj + (size_t)b * i];
                if ((e = upload(c, Rt, c.d_small)) != cudaSuccess) return fail("R upload");
                k_block_axpy<<<axpy_grid(c, m), 256, 0, c.st>>>(Zb, ldv, b, V + (int64_t)j0 * ldv, ldv, b,
                                                               c.d_small, b, 1.f, -1.f, m);
                c.launches += 1;
            }
            if ((e = orthonormalize(c, Zb, ldv, b, V, ldv, j0 + b, m, S)) != cudaSuccess) return fail("V block");
            if (j0 + b < ell) {
                for (int cc = 0; cc < b; ++cc)
                    for (int r = 0; r < b; ++r) T[(j0 + r) + (size_t)ell * (j0 + b + cc)] = S[cc + (size_t)b * r];
            } else {
                Slast = S;
            }
        }
        // projected SVD of T: FP32 Jacobi, FP64 refinement of the k wanted
        // triplets; where that refinement does not apply (clustered values)
        // the FP32 triplets serve the restart, and the last cycle repeats the
        // SVD with the FP64 Jacobi
        double mx = 0.0, sum = 0.0;
        std::vector<double> SP((size_t)b * ell);
        auto projected = [&](bool fp64_fallback) -> cudaError_t {
            sv.fp32_only = fp64_fallback ? 0 : 1;
            cudaError_t err = launch_small_svd(sv, c.st, 0);
            sv.fp32_only = 1;
            if (err != cudaSuccess) return err;
            c.launches += 12;
            err = cudaMemcpyAsync(ho, sv.co, sizeof(CycleOut), cudaMemcpyDeviceToHost, c.st);
            if (err == cudaSuccess)
                err = cudaMemcpyAsync(&svd_fb, &sv.sc->svd_fallback, sizeof(int), cudaMemcpyDeviceToHost, c.st);
            if (err == cudaSuccess) err = download(c, sv.P, P, ell2);
            if (err != cudaSuccess) return err;
            sg.assign(ho->sg, ho->sg + ell);
            max_sweeps = std::max(max_sweeps, ho->sweeps);
            // block residuals r_i = || S_last P[ell-b:ell, i] ||
            mx = 0.0;
            sum = 0.0;
            for (int i = 0; i < ell; ++i)
                for (int r = 0; r < b; ++r) {
                    double a = 0.0;
                    for (int t = 0; t < b; ++t) a += Slast[r + (size_t)b * t] * P[(ell - b + t) + (size_t)ell * i];
                    SP[r + (size_t)b * i] = a;
                }
            for (int i = 0; i < k; ++i) {
                double a = 0.0;
                for (int r = 0; r < b; ++r) a += SP[r + (size_t)b * i] * SP[r + (size_t)b * i];
                res[i] = std::sqrt(a);
                mx = std::max(mx, res[i]);
                sum += res[i];
            }
            maxrel = sg[0] > 0.0 ? mx / sg[0] : 0.0;
            dtheta = sum;
            converged = mx <= est_tol * sg[0] || sg[0] == 0.0;
            return cudaSuccess;
        };
        if ((e = upload(c, T, sv.B)) != cudaSuccess) return fail("T upload");
        if ((e = projected(false)) != cudaSuccess) return fail("projected SVD");
        if (svd_fb) ++svd_unrefined;
        if (ho->svd_unconverged) ++svd_uncontracted;
        if ((converged || cycle == o->maxit - 1) && svd_fb) {
            ++svd_fp64;
            if ((e = projected(true)) != cudaSuccess) return fail("projected SVD (FP64)");
        }
        if (converged || cycle == o->maxit - 1) {
            // the estimate is met (or the cycles ran out): Rayleigh-Ritz output and true residuals
            if ((e = finalize()) != cudaSuccess) return fail("Rayleigh-Ritz step");
            if (!true_resid) break;  // k > 32: the estimate decides
            if (maxrel <= o->tol || sg[0] == 0.0) {
                converged = 1;
                break;
            }
            converged = 0;
            if (cycle == o->maxit - 1) break;
            // refinement: the true residual misses tol.  After 4-digit products the kept
            // relation A V_kk = U_kk T_kk carries their rounding, which later cycles never
            // recompute: with k <= b the next cycle starts afresh (full-precision products)
            // from the top b Ritz vectors, which hold the k wanted ones.  Otherwise the cycles
            // go on from the same restart state with a tighter estimate target.
            if (c.tc_digits < 8) {
                c.tc_digits = 8;
                fresh = k <= b;
            } else {
                est_tol *= 0.5;
            }
            ++refines;
        }
        if (fresh) {  // explicit restart: V[:, 0:b] = V Q[:, 0:b], orthonormalised
            e = launch_rotate<float>(c.st, V, ldv, ell, sv.Q, ell, b, V2, ldv, m);
            if (e == cudaSuccess) e = orthonormalize(c, V2, ldv, b, nullptr, ldv, 0, m, R);
            if (e != cudaSuccess) return fail("explicit restart");
            std::swap(V, V2);
            std::fill(T.begin(), T.end(), 0.0);
            ++restarts;
            continue;
        }
        // thick restart: keep kk Ritz vectors, spike block from S_last
        e = launch_rotate<float>(c.st, U, ldu, ell, sv.P, ell, kk, U2, ldu, n);
        if (e == cudaSuccess) e = launch_rotate<float>(c.st, V, ldv, ell, sv.Q, ell, kk, V2, ldv, m);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(V2 + (int64_t)kk * ldv, sizeof(float) * ldv, V + (int64_t)ell * ldv,
                                  sizeof(float) * ldv, sizeof(float) * m, b, cudaMemcpyDeviceToDevice, c.st);
        // kept block of T: the FP64 projection P_kk^T T Q_kk (T is still in sv.B)
        double* Mtq = sv.rw + 4 * ell2;  // refinement workspace, free after the SVD
        double* Tn = sv.rw + 5 * ell2;
        std::vector<double> hTn;
        if (e == cudaSuccess) {
            k_tq<<<kk, 128, 0, c.st>>>(sv.B, sv.Q, ell, kk, Mtq);
            k_ptm<<<kk, 128, 0, c.st>>>(sv.P, Mtq, ell, kk, Tn);
            e = download(c, Tn, hTn, (size_t)kk * kk);
        }
        if (e != cudaSuccess) return fail("restart");
        c.launches += 4;
        std::swap(U, U2);
        std::swap(V, V2);
        std::fill(T.begin(), T.end(), 0.0);
        for (int i = 0; i < kk; ++i) {
            for (int j = 0; j < kk; ++j) T[i + (size_t)ell * j] = hTn[i + (size_t)kk * j];
            for (int cc = 0; cc < b; ++cc) T[i + (size_t)ell * (kk + cc)] = SP[cc + (size_t)b * i];
        }
        ++restarts;
    }
    if (e == cudaSuccess) e = launch_sign_fix<float>(c.st, Uo, n, Vo, m, k, reinterpret_cast<int*>(W + oSigns));
    // U, V out (device-to-device, or to host memory with o->out_host); the
    // triplets also stay in the handle for gkl_scores and gkl_grad
    if (e == cudaSuccess && Uout) e = cudaMemcpyAsync(Uout, Uo, sizeof(float) * n * k, cudaMemcpyDefault, c.st);
    if (e == cudaSuccess && Vout) e = cudaMemcpyAsync(Vout, Vo, sizeof(float) * m * k, cudaMemcpyDefault, c.st);
    const size_t lb = sizeof(float) * (size_t)(n + m) * k;
    if (e == cudaSuccess && h->last_bytes < lb) {
        if (h->last_U) cudaFree(h->last_U);
        h->last_U = nullptr;
        h->last_bytes = 0;
        e = cudaMalloc(&h->last_U, lb);
        if (e == cudaSuccess) h->last_bytes = lb;
    }
    if (e == cudaSuccess) {
        h->last_V = static_cast<char*>(h->last_U) + sizeof(float) * (size_t)n * k;
        e = cudaMemcpyAsync(h->last_U, Uo, sizeof(float) * n * k, cudaMemcpyDeviceToDevice, c.st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->last_V, Vo, sizeof(float) * m * k, cudaMemcpyDeviceToDevice, c.st);
    cudaEventRecord(ev1, c.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
    if (e != cudaSuccess) return fail("output");
    if (int pend = take_pending_error(h)) {
        cudaFree(ws);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return pend;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    const int rank = numerical_rank(sg.data(), k, sv.eps_w);
    for (int i = 0; i < k; ++i) {
        sigma[i] = i < rank ? sg[i] : 0.0;
        if (resid) resid[i] = res[i];
    }
    h->last_valid = converged ? 1 : 0;
    h->last_prec = GKL_FP32;
    h->last_k = k;
    for (int i = 0; i < k; ++i) h->last_sigma[i] = sigma[i];
    h->last_next = k < ell ? sg[k] : 0.0;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->matvec_pairs = c.products;
        info->restarts = restarts;
        info->cycles = cycle + 1;
        info->breakdowns = c.deflations;
        info->second_v = c.cgs_second;  // block form: orthonormalisations that needed a second CGS pass
        info->rank = rank;
        info->converged = converged;
        info->max_rel_resid = maxrel;
        info->dtheta1 = dtheta;
        info->ms_total = ms;
        info->launches = c.launches + 5;
        info->svd_fallbacks = svd_fp64;
        info->svd_clusters = svd_unrefined;  // cycles whose projected SVD could not be refined
        if (c.profile) {  // main tensor-core product kernels, summed
            info->ms_mv = sum_event_pairs(c.ev_mv, c.used_mv, &info->n_mv);
            info->ms_rmv = sum_event_pairs(c.ev_rmv, c.used_rmv, &info->n_rmv);
        }
        info->jacobi_sweeps = max_sweeps;
        info->refine_cycles = refines;
    }
    cudaFree(ws);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (!converged) return set_err(h, GKL_NOT_CONVERGED, "block form not converged after %d cycles", cycle + 1);
    if (rank < k)
        return set_err(h, GKL_RANK_DEFICIENT, "numerical rank %d < k = %d: sigma_%d.. reported as 0", rank, k,
                       rank + 1);
    return GKL_OK;
}

}  // namespace gkl
