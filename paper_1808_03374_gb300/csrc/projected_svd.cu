// SVD of the small projected matrix B (ell x ell, FP64) of thick-restarted
// GKL, the Ritz residual test and the thick-restart set-up (section 3 of
// arXiv:1808.03374: thick restarting with ordinary Ritz values, residual-norm
// convergence criteria).
//
// GB300's FP64 rate is low, so the O(ell^3)-per-sweep Jacobi iteration runs in
// FP32 and FP64 accuracy is recovered by refinement built from matrix
// products (Ogita & Aishima, "Iterative refinement for singular value
// decomposition based on matrix multiplication", 2020).  Given approximate
// U, V, with R = I - U^T U, S = I - V^T V and T = U^T B V, the corrections
// U' = U (I + F), V' = V (I + G) that make U'^T U' = I, V'^T V' = I and
// U'^T B V' diagonal to first order satisfy
//     F + F^T = R,  G + G^T = S,  T_ij + s_j F_ji + s_i G_ij = 0  (i != j),
// whose solution is
//     s_i  = T_ii / (1 - (R_ii + S_ii)/2),
//     F_ij = (a s_j + b s_i) / (s_j^2 - s_i^2),  G_ij = (a s_i + b s_j) / (s_j^2 - s_i^2),
//     a = T_ij + s_j R_ij,  b = T_ji + s_j S_ij,  F_ii = R_ii/2,  G_ii = S_ii/2.
// The error of a pair is squared by each step, relative to the pair's gap; four
// steps are run, then the result is checked.  When two kept singular values are
// closer (relative to their own size) than FP32 vectors can separate, or one is
// tiny, the refinement does not apply and a full FP64 one-sided Jacobi runs
// instead (the block form keeps the FP32 triplets except at its last cycle).
#include <algorithm>

#include "epilogue.cuh"
#include "gkl_internal.cuh"

namespace gkl {

namespace {
constexpr double kClusterGap = 1e-5;   // values below this fraction of sigma_1 are "tiny" (not refinable)
constexpr double kClusterRel = 5e-6;   // gap / value below which an FP32 pair is not refinable
constexpr double kRefineCheck = 1e-10;  // largest acceptable departure after the refinement steps
}

// Residual test and restart set-up from sv.P and sv.co->sg (sorted).  All
// threads of one block.
__device__ void conv_and_restart(const Sv& sv, int restart_ready, int sweeps) {
    __shared__ int s_conv;
    const int ell = sv.ell;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double beta = sv.sc->beta_last;
        const double s0 = sv.co->sg[0];
        double maxr = 0.0, sum = 0.0;
        for (int i = 0; i < sv.k; ++i) {
            double r = fabs(beta * sv.P[(ell - 1) + i * ell]);
            sv.co->resid[i] = r;
            sum += r;
            maxr = fmax(maxr, r);
        }
        int conv = (maxr <= sv.tol * s0) || s0 == 0.0;
        sv.co->conv = conv;
        sv.co->maxrel = s0 > 0.0 ? maxr / s0 : 0.0;
        sv.co->dtheta = sum;
        sv.co->sweeps = sweeps;
        s_conv = conv;
    }
    __syncthreads();
    if (s_conv || !restart_ready) return;
    const int kk = sv.kk, L = ell + 1;
    const double beta = sv.sc->beta_last;
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        int r = t % ell, c = t / ell;
        double v = 0.0;
        if (r < kk && c == r) v = sv.co->sg[r];
        else if (r < kk && c == kk) v = beta * sv.P[(ell - 1) + r * ell];
        sv.B[t] = v;
    }
    for (int t = threadIdx.x; t < L * L; t += blockDim.x) {
        int r = t % L, c = t / L;
        double e = (r == c) ? 1.0 : sv.eps_w;
        sv.muh[t] = e;
        sv.nuh[t] = e;
    }
    if (threadIdx.x == 0) {
        sv.sc->force_u = 0;
        sv.sc->force_v = 0;
    }
}

// ---------------------------------------------------------------- FP32 Jacobi

// Round-robin parallel ordering: ell/2 disjoint column pairs per round, one
// half-warp per pair (64 pairs in flight for ell = 128).  Works on B rounded to
// FP32, columns padded with zero rows to LD = 16 RPL so that each lane holds
// RPL rows in float4 groups (vector shared-memory accesses).  Column norms are kept
// and updated by each rotation (alpha' = alpha - t gamma, beta' = beta + t
// gamma), recomputed at every sweep, so a pair costs one dot product.  Writes
// the approximate sorted triplets (U0 normalised left vectors, V0 right
// vectors, sig0) in FP64 and decides whether refinement applies.
// Rows of lane hl: groups of four, 4 hl + 64 g + i (g < RPL / 4), so that the 16
// lanes of a half-warp read 256 contiguous bytes per float4 access (no bank
// conflicts between lanes).
template <int RPL>
__device__ __forceinline__ void ld_rows(const float* col, int hl, float (&v)[RPL]) {
#pragma unroll
    for (int k = 0; k < RPL; k += 4) {
        const float4 x = *reinterpret_cast<const float4*>(col + 16 * k + 4 * hl);
        v[k] = x.x;
        v[k + 1] = x.y;
        v[k + 2] = x.z;
        v[k + 3] = x.w;
    }
}
template <int RPL>
__device__ __forceinline__ void st_rows(float* col, int hl, const float (&v)[RPL]) {
#pragma unroll
    for (int k = 0; k < RPL; k += 4)
        *reinterpret_cast<float4*>(col + 16 * k + 4 * hl) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
}

template <int RPL>
__global__ void __launch_bounds__(1024) k_svd32(Sv sv) {
    static_assert(RPL % 4 == 0, "rows per lane: whole float4");
    if (sv.sc->abort) return;
    constexpr int LD = 16 * RPL;
    extern __shared__ __align__(16) float fsm[];
    const int ell = sv.ell;
    float* W = fsm;
    float* Qm = W + ell * LD;
    __shared__ float s_nrm[GKL_MAX_ELL];
    __shared__ float s_wmax[32];
    __shared__ double s_sig[GKL_MAX_ELL];
    __shared__ int s_rank[GKL_MAX_ELL];
    for (int t = threadIdx.x; t < ell * LD; t += blockDim.x) {
        const int r = t % LD, c = t / LD;
        W[t] = r < ell ? (float)sv.B[r + c * ell] : 0.f;
        Qm[t] = r == c ? 1.f : 0.f;
    }
    __syncthreads();
    const int N = ell + (ell & 1);
    const int npairs = N / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int hl = lane & 15;
    const int p = 2 * warp + (lane >> 4);  // this half-warp's pair slot
    const float jtol = 2.f * sqrtf((float)ell) * 5.9604645e-08f;
    int sweep = 0;
    float prev = 1.f;
    for (; sweep < 40; ++sweep) {
        // exact column norms at the start of each sweep
        for (int c = warp; c < ell; c += nw) {
            float s2 = 0.f;
            for (int r = lane; r < LD; r += 32) s2 = fmaf(W[r + c * LD], W[r + c * LD], s2);
            for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            if (lane == 0) s_nrm[c] = s2;
        }
        __syncthreads();
        float mymax = 0.f;
        for (int rnd = 0; rnd < N - 1; ++rnd) {
            int a = 0, b = 0;
            bool act = p < npairs;
            if (act) {
                // round-robin pairing without integer division: (rnd +- p) mod (N - 1)
                if (p == 0) {
                    a = 0;
                    b = 1 + rnd;
                } else {
                    int x = rnd + p, y = rnd - p;
                    if (x >= N - 1) x -= N - 1;
                    if (y < 0) y += N - 1;
                    a = 1 + x;
                    b = 1 + y;
                }
                act = a < ell && b < ell;
            }
            float xa[RPL], xb[RPL];
            float ga = 0.f;
            if (act) {
                ld_rows<RPL>(W + a * LD, hl, xa);
                ld_rows<RPL>(W + b * LD, hl, xb);
#pragma unroll
                for (int k = 0; k < RPL; ++k) ga = fmaf(xa[k], xb[k], ga);
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
            if (act) {
                const float al = s_nrm[a], be = s_nrm[b];
                if (ga != 0.f && fabsf(ga) > jtol * sqrtf(al * be)) {
                    mymax = fmaxf(mymax, fabsf(ga) / sqrtf(al * be));
                    const float zeta = (be - al) / (2.f * ga);
                    const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    const float cs = 1.f / sqrtf(1.f + t * t), sn = cs * t;
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const float x = xa[k], y = xb[k];
                        xa[k] = cs * x - sn * y;
                        xb[k] = sn * x + cs * y;
                    }
                    st_rows<RPL>(W + a * LD, hl, xa);
                    st_rows<RPL>(W + b * LD, hl, xb);
                    ld_rows<RPL>(Qm + a * LD, hl, xa);
                    ld_rows<RPL>(Qm + b * LD, hl, xb);
#pragma unroll
                    for (int k = 0; k < RPL; ++k) {
                        const float x = xa[k], y = xb[k];
                        xa[k] = cs * x - sn * y;
                        xb[k] = sn * x + cs * y;
                    }
                    st_rows<RPL>(Qm + a * LD, hl, xa);
                    st_rows<RPL>(Qm + b * LD, hl, xb);
                    if (hl == 0) {
                        s_nrm[a] = al - t * ga;
                        s_nrm[b] = be + t * ga;
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mymax = fmaxf(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
        if (lane == 0) s_wmax[warp] = mymax;
        __syncthreads();
        float maxr = 0.f;
        for (int w2 = 0; w2 < nw; ++w2) maxr = fmaxf(maxr, s_wmax[w2]);
        __syncthreads();
        if (maxr == 0.f) break;  // no rotation in the sweep
        // Near convergence Jacobi is quadratic: a sweep that does not halve the
        // largest remaining |cos|, already within 2x the threshold, is at FP32
        // rounding level (the FP64 refinement that follows takes it from there).
        if (maxr < 2.f * jtol && maxr > 0.5f * prev) break;
        prev = maxr;
    }
    for (int c = warp; c < ell; c += nw) {
        double s2 = 0.0;
        for (int r = lane; r < ell; r += 32) s2 += (double)W[r + c * LD] * (double)W[r + c * LD];
        s2 = warp_sum(s2);
        if (lane == 0) s_sig[c] = sqrt(s2);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ell; c += blockDim.x) {
        int rank = 0;
        for (int e = 0; e < ell; ++e)
            if (s_sig[e] > s_sig[c] || (s_sig[e] == s_sig[c] && e < c)) ++rank;
        s_rank[c] = rank;
    }
    __syncthreads();
    double* U0 = sv.rw;
    double* V0 = U0 + ell * ell;
    double* sig0 = sv.rw + 7 * ell * ell;
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        int r = t % ell, c = t / ell;
        int dst = s_rank[c];
        double sg = s_sig[c];
        U0[r + dst * ell] = sg > 0.0 ? (double)W[r + c * LD] / sg : 0.0;
        V0[r + dst * ell] = (double)Qm[r + c * LD];
    }
    for (int c = threadIdx.x; c < ell; c += blockDim.x) sig0[s_rank[c]] = s_sig[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        // sorted values: refinement needs every gap (and the smallest value)
        // well above FP32 resolution
        // Only the kk leading triplets are used (kept Ritz vectors at a restart,
        // of which the first k are the output): their values must be
        // separated from each other and from the rest of the spectrum.
        // Clusters further down are left unrefined.
        const double top = sig0[0];
        int fb = !(top > 0.0);
        const int last = min(sv.kk, ell - 1);
        // the FP32 vectors of a pair are accurate to about eps_32 sigma / gap, so
        // the gap is measured relative to the pair's own value
        for (int i = 1; i <= last && !fb; ++i)
            if (sig0[i - 1] - sig0[i] <= kClusterRel * sig0[i - 1]) fb = 1;
        if (sig0[sv.kk - 1] <= kClusterGap * top) fb = 1;
        sv.sc->svd_fallback = fb;
        sv.co->svd_cluster = fb;
        sv.co->svd_unconverged = 0;
        if (fb) {
            sv.sc->n_svd_fallback += 1;
            sv.sc->n_svd_cluster += 1;
        }
        sv.co->sweeps = sweep;
    }
}

// R = I - U^T U, S = I - V^T V, T = U^T B V; block j computes column j.
__global__ void __launch_bounds__(128) k_ref_a(Sv sv, const double* __restrict__ U, const double* __restrict__ V) {
    if (sv.sc->abort || sv.sc->svd_fallback) return;
    const int ell = sv.ell, j = blockIdx.x;
    __shared__ double bv[GKL_MAX_ELL];
    __shared__ double uj[GKL_MAX_ELL];
    __shared__ double vj[GKL_MAX_ELL];
    double* R = sv.rw + 4 * ell * ell;
    double* S = R + ell * ell;
    double* T = S + ell * ell;
    for (int i = threadIdx.x; i < ell; i += blockDim.x) {
        uj[i] = U[i + j * ell];
        vj[i] = V[i + j * ell];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ell; i += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < ell; ++c) s += sv.B[i + c * ell] * vj[c];
        bv[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ell; i += blockDim.x) {
        const double* ui = U + i * ell;
        const double* vi = V + i * ell;
        double r = 0.0, s = 0.0, t = 0.0;
        for (int q = 0; q < ell; ++q) {
            r += ui[q] * uj[q];
            s += vi[q] * vj[q];
            t += ui[q] * bv[q];
        }
        R[i + j * ell] = (i == j ? 1.0 : 0.0) - r;
        S[i + j * ell] = (i == j ? 1.0 : 0.0) - s;
        T[i + j * ell] = t;
    }
}

// Column j of F and G, then U'[:, j] = U[:, j] + U F[:, j], V'[:, j] = V[:, j] + V G[:, j].
__global__ void __launch_bounds__(128) k_ref_b(Sv sv, const double* __restrict__ U, const double* __restrict__ V,
                                               double* __restrict__ Uo, double* __restrict__ Vo) {
    if (sv.sc->abort || sv.sc->svd_fallback) return;
    const int ell = sv.ell, j = blockIdx.x;
    const double* R = sv.rw + 4 * ell * ell;
    const double* S = R + ell * ell;
    const double* T = S + ell * ell;
    double* sig = sv.rw + 7 * ell * ell;
    __shared__ double s_s[GKL_MAX_ELL], f[GKL_MAX_ELL], g[GKL_MAX_ELL];
    for (int k = threadIdx.x; k < ell; k += blockDim.x)
        s_s[k] = T[k + k * ell] / (1.0 - 0.5 * (R[k + k * ell] + S[k + k * ell]));
    __syncthreads();
    const double sj = s_s[j];
    double top = 0.0;
    for (int k = 0; k < ell; ++k) top = fmax(top, fabs(s_s[k]));
    for (int k = threadIdx.x; k < ell; k += blockDim.x) {
        if (k == j) {
            f[k] = 0.5 * R[j + j * ell];
            g[k] = 0.5 * S[j + j * ell];
        } else if (fabs(sj - s_s[k]) <= kClusterRel * fmax(fabs(sj), fabs(s_s[k])) ||
                   fmax(fabs(sj), fabs(s_s[k])) <= kClusterGap * top) {
            // unresolved pair: too close for the FP32 vectors, or both tiny (only
            // possible outside the refined triplets, see k_svd32): leave it unrotated
            f[k] = 0.0;
            g[k] = 0.0;
        } else {
            const double sk = s_s[k];
            const double a = T[k + j * ell] + sj * R[k + j * ell];
            const double b = T[j + k * ell] + sj * S[k + j * ell];
            const double den = sj * sj - sk * sk;
            f[k] = (a * sj + b * sk) / den;
            g[k] = (a * sk + b * sj) / den;
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < ell; r += blockDim.x) {
        double u = U[r + j * ell], v = V[r + j * ell];
        for (int k = 0; k < ell; ++k) {
            u += U[r + k * ell] * f[k];
            v += V[r + k * ell] * g[k];
        }
        Uo[r + j * ell] = u;
        Vo[r + j * ell] = v;
    }
    if (threadIdx.x == 0) sig[j] = sj;
}

// Accept the refined triplets (sorted again), unless the last refinement step
// did not contract, in which case the FP64 Jacobi fallback takes over.
__global__ void __launch_bounds__(256) k_svd_final(Sv sv, const double* __restrict__ U, const double* __restrict__ V,
                                                   int restart_ready) {
    if (sv.sc->abort || sv.sc->svd_fallback) return;
    const int ell = sv.ell;
    const double* R = sv.rw + 4 * ell * ell;
    const double* S = R + ell * ell;
    const double* T = S + ell * ell;
    const double* sig = sv.rw + 7 * ell * ell;
    __shared__ double s_sig[GKL_MAX_ELL];
    __shared__ int s_rank[GKL_MAX_ELL];
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    for (int c = threadIdx.x; c < ell; c += blockDim.x) s_sig[c] = sig[c];
    __syncthreads();
    // R, S, T here were recomputed from the refined triplets: their departure
    // from (0, 0, diagonal) must be at FP64 rounding level.
    const double top = s_sig[0] > 0.0 ? s_sig[0] : 1.0;
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        int r = t % ell, c = t / ell;
        if (min(r, c) >= sv.kk) continue;  // entries among unused triplets
        double dev = fmax(fabs(R[t]), fabs(S[t]));
        if (r != c) dev = fmax(dev, fabs(T[t]) / top);
        if (!(dev <= kRefineCheck)) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) {
            sv.sc->svd_fallback = 1;
            sv.sc->n_svd_fallback += 1;
            sv.co->svd_unconverged = 1;
        }
        return;
    }
    for (int c = threadIdx.x; c < ell; c += blockDim.x) {
        int rank = 0;
        for (int e = 0; e < ell; ++e)
            if (s_sig[e] > s_sig[c] || (s_sig[e] == s_sig[c] && e < c)) ++rank;
        s_rank[c] = rank;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        int r = t % ell, c = t / ell;
        int dst = s_rank[c];
        sv.P[r + dst * ell] = U[t];
        sv.Q[r + dst * ell] = V[t];
    }
    for (int c = threadIdx.x; c < ell; c += blockDim.x) sv.co->sg[s_rank[c]] = s_sig[c];
    conv_and_restart(sv, restart_ready, sv.co->sweeps);
}

// ------------------------------------------------------------ FP64 fallback

// One-sided Jacobi SVD (Hestenes) of B in FP64, one block, round-robin pair
// order, until a sweep applies no rotation.  B Q = W, sigma_c = ||W[:,c]||,
// P[:,c] = W[:,c]/sigma_c, columns sorted by descending sigma.
__global__ void __launch_bounds__(512) k_svd64(Sv sv, int restart_ready, double* __restrict__ scratch) {
    if (sv.sc->abort || !sv.sc->svd_fallback) return;
    extern __shared__ double dsm[];
    const int ell = sv.ell;
    double* W = scratch ? scratch : dsm;
    double* Qm = W + ell * ell;
    __shared__ int s_rot;
    __shared__ double s_sig[GKL_MAX_ELL];
    __shared__ int s_rank[GKL_MAX_ELL];
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        W[t] = sv.B[t];
        Qm[t] = (t % ell == t / ell) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int N = ell + (ell & 1);
    const int npairs = N / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const double jtol = ell * 2.220446049250313e-16;
    int sweep = 0;
    for (; sweep < 60; ++sweep) {
        if (threadIdx.x == 0) s_rot = 0;
        __syncthreads();
        for (int rnd = 0; rnd < N - 1; ++rnd) {
            for (int p = warp; p < npairs; p += nw) {
                int a, b;
                if (p == 0) {
                    a = 0;
                    b = 1 + rnd % (N - 1);
                } else {
                    a = 1 + (rnd + p) % (N - 1);
                    b = 1 + (rnd + N - 1 - p) % (N - 1);
                }
                if (a >= ell || b >= ell) continue;
                double* wa = W + a * ell;
                double* wb = W + b * ell;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = lane; r < ell; r += 32) {
                    double x = wa[r], y = wb[r];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                // rotate unless the pair is orthogonal to rounding level
                if (ga == 0.0 || fabs(ga) <= jtol * sqrt(al * be)) continue;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int r = lane; r < ell; r += 32) {
                    double x = wa[r], y = wb[r];
                    wa[r] = cs * x - sn * y;
                    wb[r] = sn * x + cs * y;
                }
                double* qa = Qm + a * ell;
                double* qb = Qm + b * ell;
                for (int r = lane; r < ell; r += 32) {
                    double x = qa[r], y = qb[r];
                    qa[r] = cs * x - sn * y;
                    qb[r] = sn * x + cs * y;
                }
                if (lane == 0) s_rot = 1;
            }
            __syncthreads();
        }
        const int rot = s_rot;
        __syncthreads();
        if (!rot) break;
    }
    for (int c = warp; c < ell; c += nw) {
        double s2 = 0.0;
        for (int r = lane; r < ell; r += 32) s2 += W[r + c * ell] * W[r + c * ell];
        s2 = warp_sum(s2);
        if (lane == 0) s_sig[c] = sqrt(s2);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ell; c += blockDim.x) {
        int rank = 0;
        for (int e = 0; e < ell; ++e)
            if (s_sig[e] > s_sig[c] || (s_sig[e] == s_sig[c] && e < c)) ++rank;
        s_rank[c] = rank;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        int r = t % ell, c = t / ell;
        int dst = s_rank[c];
        double sg = s_sig[c];
        sv.P[r + dst * ell] = sg > 0.0 ? W[t] / sg : 0.0;
        sv.Q[r + dst * ell] = Qm[t];
    }
    for (int c = threadIdx.x; c < ell; c += blockDim.x) sv.co->sg[s_rank[c]] = s_sig[c];
    conv_and_restart(sv, restart_ready, 1000 + sweep);
}

// Where the refinement does not apply (clustered or tiny kept values), take the
// FP32 Jacobi triplets as they are (sorted, in sv.rw): used by the block form,
// whose bases are FP32, instead of the FP64 Jacobi.
__global__ void __launch_bounds__(256) k_svd_take32(Sv sv, int restart_ready) {
    if (sv.sc->abort || !sv.sc->svd_fallback) return;
    const int ell = sv.ell;
    const double* U0 = sv.rw;
    const double* V0 = U0 + ell * ell;
    const double* sig0 = sv.rw + 7 * ell * ell;
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        sv.P[t] = U0[t];
        sv.Q[t] = V0[t];
    }
    for (int c = threadIdx.x; c < ell; c += blockDim.x) sv.co->sg[c] = sig0[c];
    conv_and_restart(sv, restart_ready, sv.co->sweeps);
}

cudaError_t launch_small_svd(const Sv& sv, cudaStream_t st, int restart_ready) {
    const int ell = sv.ell;
    const size_t ell2 = (size_t)ell * ell;
    // FP32 Jacobi: rows per lane 4 or 8 (columns padded to 64 or 128 rows)
    const int rpl = ell <= 64 ? 4 : 8;
    const size_t smem32 = 2 * (size_t)ell * 16 * rpl * sizeof(float);
    auto kfn = rpl == 4 ? k_svd32<4> : k_svd32<8>;
    if (smem32 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32);
        if (e != cudaSuccess) return e;
    }
    kfn<<<1, 1024, smem32, st>>>(sv);
    double* U0 = sv.rw;
    double* V0 = U0 + ell2;
    double* U1 = V0 + ell2;
    double* V1 = U1 + ell2;
    // four refinement steps (quadratic: an FP32 start at a tenth of the gaps
    // reaches FP64 rounding), then the check of the result
    for (int step = 0; step < 4; ++step) {
        k_ref_a<<<ell, 128, 0, st>>>(sv, U0, V0);
        k_ref_b<<<ell, 128, 0, st>>>(sv, U0, V0, U1, V1);
        std::swap(U0, U1);
        std::swap(V0, V1);
    }
    k_ref_a<<<ell, 128, 0, st>>>(sv, U0, V0);
    k_svd_final<<<1, 256, 0, st>>>(sv, U0, V0, restart_ready);
    if (sv.fp32_only) {
        k_svd_take32<<<1, 256, 0, st>>>(sv, restart_ready);
        return cudaGetLastError();
    }
    // FP64 fallback (returns at once unless requested above)
    size_t smem = 2 * ell2 * sizeof(double);
    double* scratch = nullptr;
    if (smem > 200 * 1024) {
        scratch = sv.P + 2 * ell2;  // workspace beyond P and Q (allocated by the driver)
        smem = 0;
    } else if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_svd64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_svd64<<<1, 512, smem, st>>>(sv, restart_ready, scratch);
    return cudaGetLastError();
}

}  // namespace gkl
