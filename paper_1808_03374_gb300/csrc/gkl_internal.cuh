// Internal declarations shared by the translation units of libgkl.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "gkl.h"

#define GKL_MAX_ELL 128

// Diagnostic builds (-DGKL_DEBUG_SYNC_CHECKS) synchronise after each kernel of
// the product launchers and print the first one whose execution failed.
#ifdef GKL_DEBUG_SYNC_CHECKS
#include <cstdio>
#define GKL_DEBUG_SYNC(st, what)                                                              \
    do {                                                                                      \
        cudaError_t dbg_e = cudaStreamSynchronize(st);                                        \
        if (dbg_e != cudaSuccess) fprintf(stderr, "GKL_DEBUG %s: %s\n", what, cudaGetErrorString(dbg_e)); \
    } while (0)
#else
#define GKL_DEBUG_SYNC(st, what) \
    do {                         \
    } while (0)
#endif

namespace gkl {

// Scalars of one Lanczos run, resident in device memory so that the step
// sequence needs no host round trip.  Written only by single threads of
// "last blocks" (see epilogue.cuh) and read by later kernels in stream order.
struct DevScal {
    double scale_u, scale_v;  // 1/alpha_j, 1/beta_j used to normalise the new vectors
    double anorm;             // running max of the Lanczos coefficients (lower bound on ||A||)
    double beta_last;         // beta of the last step of a cycle (couples v_{ell})
    double pre;               // norm before reorthogonalisation of the current vector
    int reorth_u, reorth_v;   // reorthogonalise the current u / v vector
    int force_u, force_v;     // force reorthogonalisation at the next step (partial mode)
    int abort;                // 0, or ABORT_* -> remaining kernels of the cycle return at once
    int break_side;           // 0 = u, 1 = v
    int break_step;           // step j of the breakdown
    int n_reorth_u, n_reorth_v;
    unsigned counter;         // arrival counter of the last-block reductions (reset by the last block)
    int svd_fallback;         // projected SVD: 1 = FP32 + refinement does not apply, use FP64 Jacobi
    int n_svd_fallback;       // cycles whose projected SVD used the FP64 Jacobi
    int n_svd_cluster;        // ... of which because of clustered or tiny values
    int second_u[2];          // adaptive second Gram-Schmidt pass of the u side: {take it now, times taken}
    int second_v[2];          // ... of the v side
};

enum { ABORT_NONE = 0, ABORT_BREAKDOWN = 1, ABORT_NONFINITE = 2 };

// Result block of one cycle, copied to the host once per cycle.
struct CycleOut {
    int conv;
    int sweeps;
    int svd_cluster;          // projected SVD: refinement not applied (clustered or tiny kept values)
    int svd_unconverged;      // projected SVD: refinement applied but did not contract
    double maxrel;
    double dtheta;
    double sg[GKL_MAX_ELL];
    double resid[GKL_MAX_ELL];
};

// Solver state passed by value to the solver kernels.
struct Sv {
    int64_t n, m, ldu, ldv;
    int ell, kk, k, reorth;
    int kk_start;             // first step of the current cycle (0, or kk after a restart)
    int prec;                 // GKL_FP64 / GKL_FP32
    int fp32_only;            // projected SVD: no FP64 Jacobi fallback (block form)
    void* U;                  // n x ell (ldu), type by prec
    void* V;                  // m x (ell+1) (ldv)
    double* B;                // ell x ell, column-major
    double* muh;              // (ell+1)^2 estimates u_i^T u_k
    double* nuh;              // (ell+1)^2 estimates v_i^T v_k
    double* P;                // ell x ell left vectors of B (sorted)
    double* Q;                // ell x ell right vectors of B (sorted)
    double* rw;               // projected-SVD workspace: 8 ell^2 doubles (U0 V0 U1 V1 R S T sig)
    DevScal* sc;
    CycleOut* co;
    double* partials;         // [max blocks][GKL_MAX_ELL + 2]
    double* coef;             // [2][GKL_MAX_ELL + 2]
    double eps_w;             // unit roundoff of the working precision
    double omega;             // partial-reorthogonalisation trigger
    double tol;
    uint64_t seed;
};

}  // namespace gkl

struct gkl_handle {
    const uint8_t* packed;
    int64_t n, m, stride;
    cudaStream_t stream;
    int device;
    int num_sms;
    double* mu;      // m
    double* d;       // m
    float* s;        // n or null
    float* w;        // m or null
    // scratch for the packed products (grown on demand)
    void* scratch;
    size_t scratch_bytes;
    // solver workspace (grown on demand)
    void* ws;
    size_t ws_bytes;
    gkl::CycleOut* host_out;  // pinned
    double* aux;     // small zero-initialised device buffer: scale/sum of the tensor-core product + its counter
    // triplets of the last successful gkl_svd (for gkl_grad)
    int last_valid, last_prec, last_k;
    double last_sigma[GKL_MAX_ELL];
    double last_next;  // Ritz value k+1 of the last cycle (estimate of sigma_{k+1})
    void* last_U;      // n x k, precision's type
    void* last_V;      // m x k
    size_t last_bytes;
    void* gws;         // gradient workspace (grown on demand)
    size_t gws_bytes;
    // tensor-core (tcgen05) A^T u: 0 = not prepared, 1 = ready, -1 = unavailable
    int tc_state;
    alignas(64) unsigned char tc_map[128];  // TMA descriptor of the packed matrix (A^T u: 128 B x 128 rows, swizzled)
    alignas(64) unsigned char mv_map[128];  // TMA descriptor for A v (256 B x 32 rows, no swizzle)
    int* mv_err;     // error word of the A v kernel when the handle has no aux buffer (allocation-free product)
    int64_t* miss_off;   // list of the missing codes per (sample block, SNP): nb m + 1 offsets, built by tc_prepare
    uint16_t* miss_idx;  // their offsets in the sample block, ascending, padded to multiples of 8
    int64_t miss_nnz;    // entries of the list, padding included
    char err[512];
};

namespace gkl {

int set_err(gkl_handle* h, int code, const char* fmt, ...);
int cuda_err(gkl_handle* h, cudaError_t e, const char* what);
int ensure_scratch(gkl_handle* h, size_t bytes);

// ---- packed products (packed_ops.cu)
struct MvPlan {
    int64_t nwords;     // ceil(n/16): 32-bit words of 16 samples
    int tiles;          // sample tiles of the products
    int chunks;         // SNP chunks of A.v
    int rows_per_chunk;
    int64_t ldp;        // leading dimension of A.v partials
    size_t bytes_fp64;  // scratch bytes needed (FP64)
    // FP32 A.v (pair-table kernel): threads a block (words of a sample tile), tiles, chunks, rows a chunk
    int pair_threads, pair_tiles, pair_chunks, pair_rpc;
    int mv_chunks(bool fp32) const { return fp32 ? pair_chunks : chunks; }
};
MvPlan plan_products(const gkl_handle* h);

// Epilogue attached to the final reduction of a product: subtract earlier
// basis vectors, then reduce ||y||^2 and run the solver's last-block logic.
struct FinArgs {
    const double* bcol;  // coefficients b_r (r < nsub) to subtract: y -= sum_r b_r W[:, r]; may be null
    int nsub;
    const void* W;       // basis for the subtraction
    int64_t ldw;
    int role;            // ROLE_* (0 = plain product, no reduction)
    int j;
};

// ev0/ev1 (optional) are recorded around the main (partial-sum) kernel.
// Each launcher returns the number of kernels it enqueued through *nlaunch.
template <typename T>
cudaError_t launch_matvec(const gkl_handle* h, const T* v, T* y, void* scratch, const Sv* sv, const FinArgs* fa,
                          cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, int* nlaunch = nullptr);
template <typename T>
cudaError_t launch_rmatvec(const gkl_handle* h, const T* u, T* x, void* scratch, const Sv* sv, const FinArgs* fa,
                           cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, int* nlaunch = nullptr);
constexpr size_t kAuxBytes = 64 * 1024;
constexpr size_t kAuxErrOffset = 60 * 1024;    // int: nonzero if a tensor-core kernel's wait ran out
constexpr size_t kAuxSigmaOffset = 48 * 1024;  // GKL_MAX_ELL doubles: singular values for gkl_scores
// Synchronise the handle's stream; GKL_ERR_CUDA (message set, record cleared) if
// a tensor-core kernel's bounded wait ran out since the last check.
int take_pending_error(gkl_handle* h);
int numerical_rank(const double* sg, int k, double eps_w);
// Kind of a pointer as the library accepts it: device (or managed) memory of
// `device`, host memory (pageable, pinned or registered), or neither (device
// memory of another GPU, or an invalid pointer).
enum MemKind { MEM_BAD = 0, MEM_DEVICE = 1, MEM_HOST = 2 };
int mem_kind(const void* p, int device);
// S = U diag(sigma) (n x k, column-major) in the type of prec (GKL_FP64: double, else float)
cudaError_t launch_scores(cudaStream_t st, int prec, const void* U, const double* sigma, int64_t n, int k, void* S);
// tcgen05 A^T u (both precisions, packed_tc.cu); tc_prepare builds the TMA descriptor and the
// list of missing codes once per handle.
bool tc_prepare(gkl_handle* h);
size_t rmv_tc_scratch_bytes(const gkl_handle* h);
template <typename T>
cudaError_t launch_rmatvec_tc(const gkl_handle* h, const T* u, T* x, void* scratch, const Sv* sv, const FinArgs* fa,
                              cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch);

bool make_mv_map(const uint8_t* packed, int64_t stride, int64_t m, void* out);
cudaError_t launch_colstats(const uint8_t* packed, int64_t n, int64_t m, int64_t stride, double* mu, double* scale,
                            int64_t* nobs, cudaStream_t st);

// ---- vector kernels (solver_kernels.cu)
enum {
    ROLE_NONE = 0,
    ROLE_U_PRE = 1,
    ROLE_U_POST = 2,
    ROLE_V_PRE = 3,
    ROLE_V_POST = 4,
    ROLE_START = 5,
    ROLE_REPL_U = 6,
    ROLE_REPL_V = 7,
    ROLE_STORE = 8  // keep ||x||^2 in DevScal::pre (gradient solves)
};
enum { CGS_DOTS = 0, CGS_UPD_DOTS = 1, CGS_UPD_NORM = 2, CGS_FILL_DOTS = 3 };
int cgs_grid(int64_t len, int num_sms);

// second: null = both Gram-Schmidt passes; else the adaptive second pass (flag and count, see k_cgs)
template <typename T>
cudaError_t launch_cgs(const Sv& sv, cudaStream_t st, int mode, T* x, int64_t len, const T* W, int64_t ldw, int ncols,
                       const int* cond, int role, int j, uint32_t draw, int num_sms, int* second = nullptr);
template <typename T>
cudaError_t launch_scale(const Sv& sv, cudaStream_t st, T* x, int64_t len, const double* scale);
template <typename T>
cudaError_t launch_fill_random(const Sv& sv, cudaStream_t st, T* x, int64_t len, uint32_t draw, int check_abort);
template <typename T>
cudaError_t launch_rotate(cudaStream_t st, const T* in, int64_t ldin, int ell, const double* R, int ldr, int ncols,
                          T* out, int64_t ldout, int64_t len);
template <typename T>
cudaError_t launch_sign_fix(cudaStream_t st, T* U, int64_t n, T* V, int64_t m, int k, int* signs);
cudaError_t launch_small_svd(const Sv& sv, cudaStream_t st, int restart_ready);
// tcgen05 block products (block_tc.cu): D base-16 digits per vector, q D <= 128
bool block_tc_usable(const gkl_handle* h);
bool block_tc_prepare(gkl_handle* h);
size_t block_tc_scratch_bytes(const gkl_handle* h, int q);
// ev0/ev1 (optional) are recorded around the main tensor-core kernel.
cudaError_t launch_block_product_tc(const gkl_handle* h, bool transpose, const float* X, int64_t ldx, int q, int D,
                                    float* Y, int64_t ldy, void* scratch, int* nlaunch, cudaEvent_t ev0 = nullptr,
                                    cudaEvent_t ev1 = nullptr);
// block form (block.cu)
int run_block(gkl_handle* h, const gkl_opts* o, double* sigma, float* Uout, float* Vout, double* resid,
              gkl_info* info);
cudaError_t launch_init_state(const Sv& sv, cudaStream_t st);

// ---- Philox4x32-10 (Salmon et al., SC'11) for the start vector and breakdown restarts
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1, n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Uniform on (-1, 1) for index i of draw `draw`.
__host__ __device__ inline double uniform_pm1(uint64_t seed, uint32_t draw, int64_t i) {
    uint32_t c[4] = {(uint32_t)i, draw, 0x474B4C00u, (uint32_t)(i >> 32)};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return ((double)c[0] + 0.5) * (2.0 / 4294967296.0) - 1.0;
}

}  // namespace gkl
