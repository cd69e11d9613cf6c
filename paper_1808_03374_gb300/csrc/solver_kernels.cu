// Vector kernels of thick-restarted Golub-Kahan-Lanczos (section 3 of
// arXiv:1808.03374): classical Gram-Schmidt applied twice against a Krylov
// basis with FP64 inner products, normalisation, the thick-restart rotation
// U <- U P, V <- V Q, the sign rule of the output, and the FP64 SVD of the
// small projected matrix with the residual convergence test.
#include <algorithm>

#include "epilogue.cuh"
#include "gkl_internal.cuh"

namespace gkl {

namespace {
constexpr int kCgsThreads = 512;
constexpr int kPartStride = GKL_MAX_ELL + 2;
}

int cgs_grid(int64_t len, int num_sms) {
    int64_t g = (len + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, std::max(1, num_sms)));
}

// Deterministic block sum: each thread sums its strided subset in order, then
// a fixed shuffle tree and a fixed-order sum over warps.  All threads return it.
__device__ inline double block_sum_all(double v) {
    __shared__ double s_w[32];
    __shared__ double s_t;
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) s_w[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < nw; ++q) t += s_w[q];
        s_t = t;
    }
    __syncthreads();
    return s_t;
}

// One pass of classical Gram-Schmidt on the rows owned by this block:
//   DOTS:      c1 = W^T x
//   UPD_DOTS:  x -= W c1; c2 = W^T x
//   UPD_NORM:  x -= W c2; ||x||^2 -> step logic (role)
//   FILL_DOTS: x = fresh vector; c1 = W^T x
// W has ncols columns (leading dimension ldw).  Inner products accumulate in
// FP64; the last block adds the per-block partials in block order.
template <typename T>
__global__ void __launch_bounds__(kCgsThreads) k_cgs(Sv sv, int mode, T* __restrict__ x, int64_t len,
                                                    const T* __restrict__ W, int64_t ldw, int ncols,
                                                    const int* __restrict__ cond, int role, int j, uint32_t draw,
                                                    int64_t chunk) {
    if (sv.sc->abort) return;
    if (cond && *cond == 0) return;
    extern __shared__ unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    __shared__ double cs[kPartStride];
    const double* cin = nullptr;
    double* cout = nullptr;
    if (mode == CGS_UPD_DOTS) { cin = sv.coef; cout = sv.coef + kPartStride; }
    else if (mode == CGS_UPD_NORM) { cin = sv.coef + kPartStride; }
    else { cout = sv.coef; }
    if (cin)
        for (int t = threadIdx.x; t < ncols; t += blockDim.x) cs[t] = cin[t];
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = min(len, r0 + chunk);
    double sq = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        T xi;
        if (mode == CGS_FILL_DOTS) xi = (T)uniform_pm1(sv.seed, draw, i);
        else xi = x[i];
        if (cin) {
            T acc = (T)0;
            for (int k = 0; k < ncols; ++k) acc += W[i + (int64_t)k * ldw] * (T)cs[k];
            xi -= acc;
        }
        if (mode != CGS_DOTS) x[i] = xi;
        xs[i - r0] = xi;
        sq += (double)xi * (double)xi;
    }
    __syncthreads();
    double* part = sv.partials + (int64_t)blockIdx.x * kPartStride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t nr = r1 > r0 ? r1 - r0 : 0;
    if (mode == CGS_UPD_NORM) {
        double t = block_sum_all(sq);
        if (threadIdx.x == 0) part[0] = t;
    } else {
        for (int k = warp; k < ncols; k += nw) {
            const T* wk = W + r0 + (int64_t)k * ldw;
            double acc = 0.0;
            for (int64_t t = lane; t < nr; t += 32) acc += (double)wk[t] * (double)xs[t];
            acc = warp_sum(acc);
            if (lane == 0) part[k] = acc;
        }
    }
    if (!arrive_last(&sv.sc->counter)) return;
    const int nb = gridDim.x;
    if (mode == CGS_UPD_NORM) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) v += __ldcg(sv.partials + (int64_t)b * kPartStride);
        double tot = block_sum_all(v);
        step_epilogue(sv, role, j, tot);
    } else {
        for (int k = warp; k < ncols; k += nw) {
            double v = 0.0;
            for (int b = lane; b < nb; b += 32) v += __ldcg(sv.partials + (int64_t)b * kPartStride + k);
            v = warp_sum(v);
            if (lane == 0) cout[k] = v;
        }
    }
    __syncthreads();
    release_counter(&sv.sc->counter);
}

template <typename T>
cudaError_t launch_cgs(const Sv& sv, cudaStream_t st, int mode, T* x, int64_t len, const T* W, int64_t ldw, int ncols,
                       const int* cond, int role, int j, uint32_t draw, int num_sms) {
    int grid = cgs_grid(len, num_sms);
    int64_t chunk = (len + grid - 1) / grid;
    size_t smem = (size_t)chunk * sizeof(T);
    static bool attr_set[2] = {false, false};
    if (smem > 48 * 1024) {
        int idx = sizeof(T) == 8;
        if (!attr_set[idx]) {
            cudaFuncSetAttribute(k_cgs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr_set[idx] = true;
        }
        if (smem > 200 * 1024) return cudaErrorInvalidValue;
    }
    k_cgs<T><<<grid, kCgsThreads, smem, st>>>(sv, mode, x, len, W, ldw, ncols, cond, role, j, draw, chunk);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_scale(Sv sv, T* __restrict__ x, int64_t len, const double* __restrict__ scale) {
    if (sv.sc->abort) return;
    const T f = (T)(*scale);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

template <typename T>
cudaError_t launch_scale(const Sv& sv, cudaStream_t st, T* x, int64_t len, const double* scale) {
    int64_t blocks = std::min<int64_t>((len + 255) / 256, 4096);
    k_scale<T><<<(unsigned)blocks, 256, 0, st>>>(sv, x, len, scale);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_fill_random(Sv sv, T* __restrict__ x, int64_t len, uint32_t draw, int check_abort) {
    if (check_abort && sv.sc->abort) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (T)uniform_pm1(sv.seed, draw, i);
}

template <typename T>
cudaError_t launch_fill_random(const Sv& sv, cudaStream_t st, T* x, int64_t len, uint32_t draw, int check_abort) {
    int64_t blocks = std::min<int64_t>((len + 255) / 256, 4096);
    k_fill_random<T><<<(unsigned)blocks, 256, 0, st>>>(sv, x, len, draw, check_abort);
    return cudaGetLastError();
}

// out[:, c] = sum_l in[:, l] R[l, c] for c < ncols (rows of 32 staged in
// shared memory; in-place when out == in is safe: a block reads all of its
// rows before writing any of them).
template <typename T>
__global__ void __launch_bounds__(256) k_rotate(const T* in, int64_t ldin, int ell, const double* __restrict__ R,
                                                int ldr, int ncols, T* out, int64_t ldout, int64_t len) {
    extern __shared__ unsigned char smem_raw[];
    T* Rs = reinterpret_cast<T*>(smem_raw);  // Rs[l + c*ell]
    T* tile = Rs + ell * ncols;              // tile[l*32 + r]
    for (int t = threadIdx.x; t < ell * ncols; t += blockDim.x) {
        int l = t % ell, c = t / ell;
        Rs[t] = (T)R[l + (int64_t)c * ldr];
    }
    const int64_t nblk = (len + 31) / 32;
    for (int64_t rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
        __syncthreads();
        for (int t = threadIdx.x; t < ell * 32; t += blockDim.x) {
            int l = t >> 5, r = t & 31;
            int64_t i = rb * 32 + r;
            tile[t] = i < len ? in[i + (int64_t)l * ldin] : (T)0;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ncols * 32; t += blockDim.x) {
            int c = t >> 5, r = t & 31;
            int64_t i = rb * 32 + r;
            T acc = (T)0;
            const T* rc = Rs + (int64_t)c * ell;
            for (int l = 0; l < ell; ++l) acc += tile[l * 32 + r] * rc[l];
            if (i < len) out[i + (int64_t)c * ldout] = acc;
        }
    }
}

template <typename T>
cudaError_t launch_rotate(cudaStream_t st, const T* in, int64_t ldin, int ell, const double* R, int ldr, int ncols,
                          T* out, int64_t ldout, int64_t len) {
    size_t smem = ((size_t)ell * ncols + (size_t)ell * 32) * sizeof(T);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_rotate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int64_t blocks = std::min<int64_t>((len + 31) / 32, 1024);
    k_rotate<T><<<(unsigned)blocks, 256, smem, st>>>(in, ldin, ell, R, ldr, ncols, out, ldout, len);
    return cudaGetLastError();
}

// Sign rule: the entry of largest magnitude of each V column (first on ties)
// is made positive; the U column flips with it.
template <typename T>
__global__ void k_sign_pick(const T* __restrict__ V, int64_t m, int* __restrict__ signs) {
    const int c = blockIdx.x;
    const T* v = V + (int64_t)c * m;
    double best = -1.0;
    int64_t bi = 0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
        double a = fabs((double)v[i]);
        if (a > best) { best = a; bi = i; }
    }
    __shared__ double sb[256];
    __shared__ int64_t si[256];
    sb[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            double a = sb[threadIdx.x + o];
            int64_t ai = si[threadIdx.x + o];
            if (a > sb[threadIdx.x] || (a == sb[threadIdx.x] && ai < si[threadIdx.x])) {
                sb[threadIdx.x] = a;
                si[threadIdx.x] = ai;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) signs[c] = v[si[0]] < (T)0 ? -1 : 1;
}

template <typename T>
__global__ void k_sign_apply(T* U, int64_t n, T* V, int64_t m, int k, const int* __restrict__ signs) {
    const int64_t tot = (n + m) * k;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
        if (t < n * k) {
            int c = (int)(t / n);
            if (signs[c] < 0 && U) U[t] = -U[t];
        } else {
            int64_t q = t - n * k;
            int c = (int)(q / m);
            if (signs[c] < 0) V[q] = -V[q];
        }
    }
}

template <typename T>
cudaError_t launch_sign_fix(cudaStream_t st, T* U, int64_t n, T* V, int64_t m, int k, int* signs) {
    k_sign_pick<T><<<k, 256, 0, st>>>(V, m, signs);
    int64_t blocks = std::min<int64_t>(((n + m) * k + 255) / 256, 4096);
    k_sign_apply<T><<<(unsigned)blocks, 256, 0, st>>>(U, n, V, m, k, signs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- state

__global__ void k_init_state(Sv sv) {
    const int ell = sv.ell, L = ell + 1;
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) sv.B[t] = 0.0;
    for (int t = threadIdx.x; t < L * L; t += blockDim.x) {
        double e = (t % L == t / L) ? 1.0 : 0.0;
        sv.muh[t] = e;
        sv.nuh[t] = e;
    }
    if (threadIdx.x == 0) {
        DevScal* sc = sv.sc;
        sc->scale_u = sc->scale_v = 0.0;
        sc->anorm = 0.0;
        sc->beta_last = 0.0;
        sc->pre = 0.0;
        sc->reorth_u = sc->reorth_v = 0;
        sc->force_u = sc->force_v = 0;
        sc->abort = 0;
        sc->break_side = sc->break_step = 0;
        sc->n_reorth_u = sc->n_reorth_v = 0;
        sc->counter = 0u;
    }
}

cudaError_t launch_init_state(const Sv& sv, cudaStream_t st) {
    k_init_state<<<1, 256, 0, st>>>(sv);
    return cudaGetLastError();
}

// ------------------------------------------------------- projected SVD

// One-sided Jacobi SVD (Hestenes) of the ell x ell projected matrix B in FP64,
// one block.  Column pairs are rotated in round-robin order (ell/2 disjoint
// pairs per round, one warp per pair) until a sweep applies no rotation.
// B Q = W, sigma_c = ||W[:,c]||, P[:,c] = W[:,c]/sigma_c; columns sorted by
// descending sigma.  Then the residual test of section 3: r_i =
// beta_ell |P_{ell,i}|, converged when max_{i<k} r_i <= tol sigma_1; and,
// unless converged, B is reset for a thick restart with kk Ritz vectors:
// diag(sigma_1..sigma_kk) plus the spike column B_{i,kk} = beta_ell P_{ell,i}.
__global__ void __launch_bounds__(512) k_small_svd(Sv sv, int restart_ready, double* __restrict__ scratch) {
    if (sv.sc->abort) return;  // the cycle was cut short by a breakdown; the host resumes it
    extern __shared__ double dsm[];
    const int ell = sv.ell;
    double* W = scratch ? scratch : dsm;
    double* Qm = W + ell * ell;
    __shared__ int s_rot;
    __shared__ double s_sig[GKL_MAX_ELL];
    __shared__ int s_rank[GKL_MAX_ELL];
    __shared__ int s_conv;
    for (int t = threadIdx.x; t < ell * ell; t += blockDim.x) {
        W[t] = sv.B[t];
        Qm[t] = (t % ell == t / ell) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int N = ell + (ell & 1);
    const int npairs = N / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
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
                if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
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
        sv.co->sweeps = sweep;
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

cudaError_t launch_small_svd(const Sv& sv, cudaStream_t st, int restart_ready) {
    size_t smem = 2 * (size_t)sv.ell * sv.ell * sizeof(double);
    double* scratch = nullptr;
    if (smem > 200 * 1024) {
        scratch = sv.P + 2 * (size_t)sv.ell * sv.ell;  // workspace beyond P, Q (allocated by the driver)
        smem = 0;
    } else if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_small_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_small_svd<<<1, 512, smem, st>>>(sv, restart_ready, scratch);
    return cudaGetLastError();
}

template cudaError_t launch_cgs<float>(const Sv&, cudaStream_t, int, float*, int64_t, const float*, int64_t, int,
                                       const int*, int, int, uint32_t, int);
template cudaError_t launch_cgs<double>(const Sv&, cudaStream_t, int, double*, int64_t, const double*, int64_t, int,
                                        const int*, int, int, uint32_t, int);
template cudaError_t launch_scale<float>(const Sv&, cudaStream_t, float*, int64_t, const double*);
template cudaError_t launch_scale<double>(const Sv&, cudaStream_t, double*, int64_t, const double*);
template cudaError_t launch_fill_random<float>(const Sv&, cudaStream_t, float*, int64_t, uint32_t, int);
template cudaError_t launch_fill_random<double>(const Sv&, cudaStream_t, double*, int64_t, uint32_t, int);
template cudaError_t launch_rotate<float>(cudaStream_t, const float*, int64_t, int, const double*, int, int, float*,
                                          int64_t, int64_t);
template cudaError_t launch_rotate<double>(cudaStream_t, const double*, int64_t, int, const double*, int, int, double*,
                                           int64_t, int64_t);
template cudaError_t launch_sign_fix<float>(cudaStream_t, float*, int64_t, float*, int64_t, int, int*);
template cudaError_t launch_sign_fix<double>(cudaStream_t, double*, int64_t, double*, int64_t, int, int*);

}  // namespace gkl
