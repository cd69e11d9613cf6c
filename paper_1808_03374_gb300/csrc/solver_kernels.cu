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
//
// Adaptive second pass (second != null; second[0] = flag, second[1] = count):
// DOTS also reduces ||x||^2, and its last block asks for the second pass only
// where the first removes more than half of the squared norm, ||c1||^2 >
// ||x||^2 / 2 (for an orthonormal W, ||x - W c1||^2 = ||x||^2 - ||c1||^2, so the
// test is that of Daniel, Gragg, Kaufman and Stewart with eta = 1/sqrt(2)).
// FILL_DOTS always asks for it.  Without the flag, UPD_DOTS skips the second
// pass's inner products and UPD_NORM its update.
template <typename T>
__global__ void __launch_bounds__(kCgsThreads) k_cgs(Sv sv, int mode, T* __restrict__ x, int64_t len,
                                                    const T* __restrict__ W, int64_t ldw, int ncols,
                                                    const int* __restrict__ cond, int role, int j, uint32_t draw,
                                                    int64_t chunk, int* second) {
    if (sv.sc->abort) return;
    if (cond && *cond == 0) return;
    const bool one_pass = second != nullptr && (mode == CGS_UPD_DOTS || mode == CGS_UPD_NORM) && second[0] == 0;
    extern __shared__ unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);
    __shared__ double cs[kPartStride];
    const double* cin = nullptr;
    double* cout = nullptr;
    if (mode == CGS_UPD_DOTS) { cin = sv.coef; cout = one_pass ? nullptr : sv.coef + kPartStride; }
    else if (mode == CGS_UPD_NORM) { cin = one_pass ? nullptr : sv.coef + kPartStride; }
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
    if (mode == CGS_UPD_DOTS && one_pass) return;  // the update alone: no inner products needed
    __syncthreads();
    double* part = sv.partials + (int64_t)blockIdx.x * kPartStride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t nr = r1 > r0 ? r1 - r0 : 0;
    if (mode == CGS_UPD_NORM) {
        double t = block_sum_all(sq);
        if (threadIdx.x == 0) part[0] = t;
    } else {
        // Each lane sums its strided share in the working precision (FP32
        // products of a vector chunk are accumulated in FP32: with two
        // Gram-Schmidt passes the projections are removed far below FP32
        // rounding; FP64 FMAs are scarce on this GPU), then the lane sums are
        // combined in FP64.
        for (int k = warp; k < ncols; k += nw) {
            const T* wk = W + r0 + (int64_t)k * ldw;
            T acc_w = (T)0;
            for (int64_t t = lane; t < nr; t += 32) acc_w += wk[t] * xs[t];
            double acc = warp_sum((double)acc_w);
            if (lane == 0) part[k] = acc;
        }
        if (second && (mode == CGS_DOTS || mode == CGS_FILL_DOTS)) {
            const double t = block_sum_all(sq);
            if (threadIdx.x == 0) part[ncols] = t;
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
        if (second && (mode == CGS_DOTS || mode == CGS_FILL_DOTS)) {
            double v = 0.0;
            for (int b = threadIdx.x; b < nb; b += blockDim.x) v += __ldcg(sv.partials + (int64_t)b * kPartStride + ncols);
            const double x2 = block_sum_all(v);  // also orders the cout writes above before the read below
            if (threadIdx.x == 0) {
                double cc = 0.0;
                for (int k = 0; k < ncols; ++k) cc += cout[k] * cout[k];
                const int again = mode == CGS_FILL_DOTS || !(cc <= 0.5 * x2);
                second[0] = again;
                second[1] += again;
            }
        }
    }
    __syncthreads();
    release_counter(&sv.sc->counter);
}

template <typename T>
cudaError_t launch_cgs(const Sv& sv, cudaStream_t st, int mode, T* x, int64_t len, const T* W, int64_t ldw, int ncols,
                       const int* cond, int role, int j, uint32_t draw, int num_sms, int* second) {
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
    k_cgs<T><<<grid, kCgsThreads, smem, st>>>(sv, mode, x, len, W, ldw, ncols, cond, role, j, draw, chunk, second);
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
        sc->svd_fallback = 0;
        sc->n_svd_fallback = 0;
        sc->n_svd_cluster = 0;
        sc->second_u[0] = sc->second_u[1] = 0;
        sc->second_v[0] = sc->second_v[1] = 0;
    }
}

// PC scores S = U diag(sigma): S[i + n c] = U[i + n c] sigma_c.
template <typename T>
__global__ void k_scores(const T* __restrict__ U, const double* __restrict__ sigma, int64_t n, int k,
                         T* __restrict__ S) {
    const int64_t tot = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x)
        S[e] = (T)((double)U[e] * sigma[e / n]);
}

cudaError_t launch_scores(cudaStream_t st, int prec, const void* U, const double* sigma, int64_t n, int k, void* S) {
    const unsigned grid = (unsigned)std::min<int64_t>((n * k + 255) / 256, 4096);
    if (prec == GKL_FP64)
        k_scores<double><<<grid, 256, 0, st>>>(static_cast<const double*>(U), sigma, n, k, static_cast<double*>(S));
    else
        k_scores<float><<<grid, 256, 0, st>>>(static_cast<const float*>(U), sigma, n, k, static_cast<float*>(S));
    return cudaGetLastError();
}

cudaError_t launch_init_state(const Sv& sv, cudaStream_t st) {
    k_init_state<<<1, 256, 0, st>>>(sv);
    return cudaGetLastError();
}

template cudaError_t launch_cgs<float>(const Sv&, cudaStream_t, int, float*, int64_t, const float*, int64_t, int,
                                       const int*, int, int, uint32_t, int, int*);
template cudaError_t launch_cgs<double>(const Sv&, cudaStream_t, int, double*, int64_t, const double*, int64_t, int,
                                        const int*, int, int, uint32_t, int, int*);
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
