// Last-block reductions and the per-step scalar logic of the Lanczos solver.
//
// Each grid-wide reduction writes one partial per block; the last block to
// arrive (arrival counter in DevScal) combines the partials in block order --
// a fixed order, so results are deterministic -- and then runs the scalar
// logic of the step (Lanczos coefficient, breakdown test, partial
// reorthogonalisation estimates).  That keeps the whole step sequence on the
// device: the host synchronises once per restart cycle.
#pragma once

#include "gkl_internal.cuh"

namespace gkl {

// All threads of a block call this after writing their partials; returns true
// in every thread of the last block to arrive.
__device__ __forceinline__ bool arrive_last(unsigned* counter) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x * gridDim.y - 1u);
    }
    __syncthreads();
    return s_last != 0;
}

__device__ __forceinline__ void release_counter(unsigned* counter) {
    if (threadIdx.x == 0) *counter = 0u;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide max of v (all threads get the result).  blockDim.x <= 1024.
__device__ inline double block_max(double v) {
    __shared__ double s_red[32];
    __shared__ double s_out;
    v = warp_max(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) s_red[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        double x = l < nw ? s_red[l] : 0.0;
        x = warp_max(x);
        if (l == 0) s_out = x;
    }
    __syncthreads();
    return s_out;
}

// ---- Lanczos coefficients -------------------------------------------------

__device__ inline void finalize_alpha(const Sv& sv, int j, double a, double pre) {
    DevScal* sc = sv.sc;
    if (!isfinite(a)) {
        sc->abort = ABORT_NONFINITE;
        sc->break_side = 0;
        sc->break_step = j;
        return;
    }
    double floor = 1e3 * sv.eps_w * fmax(sc->anorm, pre);
    if (a <= floor) {
        sv.B[j + (int64_t)j * sv.ell] = 0.0;
        sc->abort = ABORT_BREAKDOWN;
        sc->break_side = 0;
        sc->break_step = j;
        return;
    }
    sv.B[j + (int64_t)j * sv.ell] = a;
    sc->scale_u = 1.0 / a;
    sc->anorm = fmax(sc->anorm, a);
}

__device__ inline void finalize_beta(const Sv& sv, int j, double b, double pre) {
    DevScal* sc = sv.sc;
    if (!isfinite(b)) {
        sc->abort = ABORT_NONFINITE;
        sc->break_side = 1;
        sc->break_step = j;
        return;
    }
    double floor = 1e3 * sv.eps_w * fmax(sc->anorm, pre);
    double val = (b <= floor) ? 0.0 : b;
    if (j + 1 < sv.ell) sv.B[j + (int64_t)(j + 1) * sv.ell] = val;
    else sc->beta_last = val;
    if (b <= floor) {
        sc->abort = ABORT_BREAKDOWN;
        sc->break_side = 1;
        sc->break_step = j;
        return;
    }
    sc->scale_v = 1.0 / b;
    sc->anorm = fmax(sc->anorm, b);
}

// Orthogonality-level estimates for partial reorthogonalisation.  With
// A V = U B (B upper triangular) and A^T u_k = sum_l B_kl v_l for completed
// rows k, taking inner products of the two recurrences
//     alpha_j u_j = A v_j - sum_{i<j} B_ij u_i,   beta_j v_{j+1} = A^T u_j - alpha_j v_j
// with earlier vectors gives, for mu_jk ~ u_j^T u_k and nu_jk ~ v_j^T v_k:
//     alpha_j mu_jk     = sum_l B_kl nu_lj - sum_{i<j} B_ij mu_ik        (k < j)
//     beta_j  nu_{j+1,k} = sum_{i<=k} B_ik mu_ji - alpha_j nu_jk          (k <= j)
// plus a rounding term eps*(alpha_j + beta_j) of the sign of the sum
// (Simon 1984; Larsen 1998 -- the strategy section 3 of the paper cites).
// B has known structure: rows k < kk_start (kept Ritz vectors after a
// restart) hold sigma_k on the diagonal and rho_k in the spike column
// kk_start; rows k >= kk_start are bidiagonal.  The sums above therefore have
// at most two terms each, except the column kk_start (handled by a loop).
// Called by all threads of one block; returns max_k |estimate|.
__device__ inline double pro_update_u(const Sv& sv, int j, double alpha) {
    const int L = sv.ell + 1;
    const int E = sv.ell;
    const int ks = sv.kk_start;
    const double* B = sv.B;
    double bprev = j > ks ? B[(j - 1) + (int64_t)j * E] : 0.0;
    double mx = 0.0;
    for (int k = threadIdx.x; k < j; k += blockDim.x) {
        // sum_l B_kl nu_lj over row k
        double t = B[k + (int64_t)k * E] * sv.nuh[k + (int64_t)j * L];
        if (k < ks) t += B[k + (int64_t)ks * E] * sv.nuh[ks + (int64_t)j * L];
        else t += B[k + (int64_t)(k + 1) * E] * sv.nuh[(k + 1) + (int64_t)j * L];
        // sum_{i<j} B_ij mu_ik over column j
        if (j > ks) {
            t -= bprev * sv.muh[(j - 1) + (int64_t)k * L];
        } else {
            for (int i = 0; i < j; ++i) t -= B[i + (int64_t)j * E] * sv.muh[i + (int64_t)k * L];
        }
        t += copysign(sv.eps_w * (alpha + bprev), t);
        double e = t / alpha;
        sv.muh[j + (int64_t)k * L] = e;
        sv.muh[k + (int64_t)j * L] = e;
        mx = fmax(mx, fabs(e));
    }
    return block_max(mx);
}

__device__ inline double pro_update_v(const Sv& sv, int j, double beta) {
    const int L = sv.ell + 1;
    const int E = sv.ell;
    const int ks = sv.kk_start;
    const double* B = sv.B;
    double alpha = B[j + (int64_t)j * E];
    double mx = 0.0;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) {
        // sum_{i<=k} B_ik mu_ji over column k (mu_jj = 1)
        double t = B[k + (int64_t)k * E] * (k == j ? 1.0 : sv.muh[j + (int64_t)k * L]);
        if (k > ks) {
            t += B[(k - 1) + (int64_t)k * E] * sv.muh[j + (int64_t)(k - 1) * L];
        } else if (k == ks) {
            for (int i = 0; i < k; ++i) t += B[i + (int64_t)k * E] * sv.muh[j + (int64_t)i * L];
        }
        t -= alpha * sv.nuh[j + (int64_t)k * L];
        t += copysign(sv.eps_w * (alpha + beta), t);
        double e = t / beta;
        sv.nuh[(j + 1) + (int64_t)k * L] = e;
        sv.nuh[k + (int64_t)(j + 1) * L] = e;
        mx = fmax(mx, fabs(e));
    }
    return block_max(mx);
}

__device__ inline void reset_estimates(double* est, int L, int row, int upto, double eps) {
    for (int k = threadIdx.x; k < upto; k += blockDim.x) {
        est[row + (int64_t)k * L] = eps;
        est[k + (int64_t)row * L] = eps;
    }
}

// Whether the u (side 0) or v (side 1) vectors are reorthogonalised at every
// step: FULL and DGKS both sides; ONESIDED the shorter side (u if n <= m);
// PARTIAL neither (the omega-recurrence decides).
__device__ __forceinline__ bool always_reorth(const Sv& sv, int side) {
    if (sv.reorth == GKL_REORTH_FULL || sv.reorth == GKL_REORTH_DGKS) return true;
    if (sv.reorth == GKL_REORTH_ONESIDED) return side == 0 ? sv.n <= sv.m : sv.n > sv.m;
    return false;
}

// Scalar logic after ||x||^2 of the current vector is known.  Called by all
// threads of the last block.
__device__ inline void step_epilogue(const Sv& sv, int role, int j, double nrm2) {
    DevScal* sc = sv.sc;
    const double nrm = sqrt(nrm2);
    const int L = sv.ell + 1;
    __shared__ int s_do;
    switch (role) {
    case ROLE_U_PRE: {
        const int ncols = j;
        int forced = 0, trig = 0;
        if (ncols > 0) {
            if (always_reorth(sv, 0)) {
                forced = 1;
            } else {
                forced = sc->force_u || j == sv.kk_start;
                double floor = 1e3 * sv.eps_w * fmax(sc->anorm, nrm);
                if (!forced && isfinite(nrm) && nrm > floor) trig = pro_update_u(sv, j, nrm) > sv.omega;
            }
        }
        if (threadIdx.x == 0) {
            s_do = forced || trig;
            sc->pre = nrm;
            sc->reorth_u = s_do;
            sc->force_u = !always_reorth(sv, 0) && trig;
            if (s_do) sc->n_reorth_u += 1;
            else finalize_alpha(sv, j, nrm, nrm);
        }
        break;
    }
    case ROLE_U_POST:
        if (threadIdx.x == 0) finalize_alpha(sv, j, nrm, sc->pre);
        reset_estimates(sv.muh, L, j, j, sv.eps_w);
        break;
    case ROLE_V_PRE: {
        int forced = 0, trig = 0;
        if (always_reorth(sv, 1)) {
            forced = 1;
        } else {
            forced = sc->force_v || j == sv.kk_start;
            double floor = 1e3 * sv.eps_w * fmax(sc->anorm, nrm);
            if (!forced && isfinite(nrm) && nrm > floor) trig = pro_update_v(sv, j, nrm) > sv.omega;
        }
        if (threadIdx.x == 0) {
            s_do = forced || trig;
            sc->pre = nrm;
            sc->reorth_v = s_do;
            sc->force_v = !always_reorth(sv, 1) && trig;
            if (s_do) sc->n_reorth_v += 1;
            else finalize_beta(sv, j, nrm, nrm);
        }
        break;
    }
    case ROLE_V_POST:
        if (threadIdx.x == 0) finalize_beta(sv, j, nrm, sc->pre);
        reset_estimates(sv.nuh, L, j + 1, j + 1, sv.eps_w);
        break;
    case ROLE_START:
        if (threadIdx.x == 0) {
            if (!(nrm > 0.0) || !isfinite(nrm)) sc->abort = ABORT_NONFINITE;
            else sc->scale_v = 1.0 / nrm;
        }
        break;
    case ROLE_REPL_U:
        if (threadIdx.x == 0) {
            if (nrm > 0.0 && isfinite(nrm)) sc->scale_u = 1.0 / nrm;
            else sc->abort = ABORT_BREAKDOWN;
        }
        reset_estimates(sv.muh, L, j, j, sv.eps_w);
        break;
    case ROLE_REPL_V:
        if (threadIdx.x == 0) {
            if (nrm > 0.0 && isfinite(nrm)) sc->scale_v = 1.0 / nrm;
            else sc->abort = ABORT_BREAKDOWN;
        }
        reset_estimates(sv.nuh, L, j + 1, j + 1, sv.eps_w);
        break;
    case ROLE_STORE:
        if (threadIdx.x == 0) sc->pre = nrm2;
        break;
    default:
        break;
    }
}

}  // namespace gkl
