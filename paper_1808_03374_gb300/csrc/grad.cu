// Gradient of a loss on the top-k singular values and PC scores with respect
// to the per-SNP weights w and per-sample weights s, A = diag(s) A0 diag(w).
// The paper has no differentiation; this is first-order SVD perturbation
// theory applied to the triplets of the last gkl_svd.
//
// For L with adjoints sigma_bar (k) and S_bar (n x k, S = A V_k = U diag(sigma)):
//   d sigma_i = u_i^T dA v_i;
//   b_i = A^T s_bar_i,  x_i = sum_{l<k, l!=i} v_l (v_l^T b_i)/(sigma_i^2 - sigma_l^2) + y_i,
//   with y_i solving P (sigma_i^2 I - A^T A) P y_i = P b_i, P = I - V_k V_k^T
//   (conjugate gradients; the operator is positive definite on range(P) when
//   sigma_i > sigma_{k+1});
//   A_bar = sum_i [ (sigma_bar_i u_i + s_bar_i + A x_i) v_i^T + sigma_i u_i x_i^T ],
//   dL/dw_j = (A^T p . q)_j / w_j,  dL/ds_r = (p . A q)_r / s_r  summed over the
//   rank-one terms p q^T of A_bar -- each a packed product with an
//   element-wise epilogue.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gkl_internal.cuh"

namespace gkl {

template <typename T>
__global__ void k_axpby(T* __restrict__ y, const T* __restrict__ x, int64_t len, double a, double b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}

// g += c * q o z
template <typename T>
__global__ void k_fma_elem(T* __restrict__ g, const T* __restrict__ q, const T* __restrict__ z, int64_t len, double c) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = (T)((double)g[i] + c * (double)q[i] * (double)z[i]);
}

template <typename T>
__global__ void k_div_weights(T* __restrict__ g, const float* __restrict__ wt, int64_t len) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = (T)((double)g[i] / (double)wt[i]);
}

static unsigned blocks_for(int64_t len) { return (unsigned)std::min<int64_t>((len + 255) / 256, 2048); }

template <typename T>
struct Grad {
    gkl_handle* h;
    Sv sv;
    int64_t n, m;
    int k;
    T *U, *V;     // last triplets (n x k, m x k)
    T *X, *Pn;    // x_i (m x k), p_i (n x k)
    T *b, *r, *p, *q, *y, *tn, *tn2;
    double* R;    // k doubles: coefficients of a linear combination (device)
    double* hc;   // pinned host copy of coefficients
    int err = GKL_OK;

    int check(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return GKL_OK;
        return cuda_err(h, e, what);
    }
    int mv(const T* v, T* out) { return check(launch_matvec<T>(h, v, out, h->scratch, nullptr, nullptr), "A.v"); }
    int rmv(const T* u, T* out) { return check(launch_rmatvec<T>(h, u, out, h->scratch, nullptr, nullptr), "A^T.u"); }
    int axpby(T* yy, const T* xx, int64_t len, double a, double bb) {
        k_axpby<T><<<blocks_for(len), 256, 0, h->stream>>>(yy, xx, len, a, bb);
        return check(cudaGetLastError(), "axpby");
    }
    int fma(T* g, const T* qq, const T* z, int64_t len, double c) {
        k_fma_elem<T><<<blocks_for(len), 256, 0, h->stream>>>(g, qq, z, len, c);
        return check(cudaGetLastError(), "fma");
    }
    // c = W^T x (ncols columns, leading dimension ldw) -> host hc[0..ncols)
    int dots(const T* W, int64_t ldw, int ncols, const T* x, int64_t len) {
        int st = check(launch_cgs<T>(sv, h->stream, CGS_DOTS, const_cast<T*>(x), len, W, ldw, ncols, nullptr,
                                     ROLE_NONE, 0, 0, h->num_sms),
                       "dots");
        if (st) return st;
        st = check(cudaMemcpyAsync(hc, sv.coef, sizeof(double) * ncols, cudaMemcpyDeviceToHost, h->stream), "dots");
        if (st) return st;
        return check(cudaStreamSynchronize(h->stream), "dots");
    }
    double dot(const T* a, const T* bb, int64_t len) {
        if ((err = dots(a, len, 1, bb, len))) return 0.0;
        return hc[0];
    }
    // x <- (I - W W^T) x applied twice (CGS2); returns ||x||^2 afterwards
    double project(T* x, int64_t len, const T* W, int64_t ldw, int ncols) {
        int st;
        if ((st = check(launch_cgs<T>(sv, h->stream, CGS_DOTS, x, len, W, ldw, ncols, nullptr, ROLE_NONE, 0, 0,
                                      h->num_sms), "project")) ||
            (st = check(launch_cgs<T>(sv, h->stream, CGS_UPD_DOTS, x, len, W, ldw, ncols, nullptr, ROLE_NONE, 0, 0,
                                      h->num_sms), "project")) ||
            (st = check(launch_cgs<T>(sv, h->stream, CGS_UPD_NORM, x, len, W, ldw, ncols, nullptr, ROLE_STORE, 0, 0,
                                      h->num_sms), "project"))) {
            err = st;
            return 0.0;
        }
        double out = 0.0;
        if ((err = check(cudaMemcpyAsync(&hc[0], &sv.sc->pre, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                         "project")))
            return 0.0;
        if ((err = check(cudaStreamSynchronize(h->stream), "project"))) return 0.0;
        out = hc[0];
        return out;
    }
    // out = sum_l c_l V[:, l] with c on the host
    int combine(const double* c, T* out) {
        int st = check(cudaMemcpyAsync(R, c, sizeof(double) * k, cudaMemcpyHostToDevice, h->stream), "combine");
        if (st) return st;
        return check(launch_rotate<T>(h->stream, V, m, k, R, k, 1, out, m, m), "combine");
    }
};

template <typename T>
static int run_grad(gkl_handle* h, const double* sigma_bar, const T* Sbar, T* g_w, T* g_s, double min_relgap) {
    const int64_t n = h->n, m = h->m;
    const int k = h->last_k;
    Grad<T> G;
    G.h = h;
    G.n = n;
    G.m = m;
    G.k = k;
    G.U = static_cast<T*>(h->last_U);
    G.V = static_cast<T*>(h->last_V);
    // workspace
    const int64_t maxblk = std::max<int64_t>({(n + 255) / 256, (m + 255) / 256, 4 * (int64_t)h->num_sms}) + 8;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = (off + bytes + 255) & ~(size_t)255; return at; };
    size_t oX = take(sizeof(T) * m * k), oP = take(sizeof(T) * n * k);
    size_t ob = take(sizeof(T) * m), orr = take(sizeof(T) * m), op = take(sizeof(T) * m), oq = take(sizeof(T) * m);
    size_t oy = take(sizeof(T) * m), otn = take(sizeof(T) * n), otn2 = take(sizeof(T) * n);
    size_t oR = take(sizeof(double) * GKL_MAX_ELL), oSc = take(sizeof(DevScal));
    size_t oPart = take(sizeof(double) * maxblk * (GKL_MAX_ELL + 2)), oCoef = take(sizeof(double) * 2 * (GKL_MAX_ELL + 2));
    if (h->gws_bytes < off) {
        if (h->gws) cudaFree(h->gws);
        h->gws = nullptr;
        h->gws_bytes = 0;
        cudaError_t e = cudaMalloc(&h->gws, off);
        if (e != cudaSuccess) return cuda_err(h, e, "gradient workspace");
        h->gws_bytes = off;
    }
    MvPlan plan = plan_products(h);
    int st = ensure_scratch(h, plan.bytes_fp64);
    if (st) return st;
    char* base = static_cast<char*>(h->gws);
    G.X = reinterpret_cast<T*>(base + oX);
    G.Pn = reinterpret_cast<T*>(base + oP);
    G.b = reinterpret_cast<T*>(base + ob);
    G.r = reinterpret_cast<T*>(base + orr);
    G.p = reinterpret_cast<T*>(base + op);
    G.q = reinterpret_cast<T*>(base + oq);
    G.y = reinterpret_cast<T*>(base + oy);
    G.tn = reinterpret_cast<T*>(base + otn);
    G.tn2 = reinterpret_cast<T*>(base + otn2);
    G.R = reinterpret_cast<double*>(base + oR);
    std::vector<double> hc_store(GKL_MAX_ELL + 2);
    G.hc = hc_store.data();
    Sv& sv = G.sv;
    sv = Sv{};
    sv.n = n;
    sv.m = m;
    sv.ell = k;
    sv.k = k;
    sv.sc = reinterpret_cast<DevScal*>(base + oSc);
    sv.partials = reinterpret_cast<double*>(base + oPart);
    sv.coef = reinterpret_cast<double*>(base + oCoef);
    sv.eps_w = sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    if ((st = G.check(cudaMemsetAsync(sv.sc, 0, sizeof(DevScal), h->stream), "grad init"))) return st;
    if ((st = G.check(cudaMemsetAsync(G.X, 0, sizeof(T) * m * k, h->stream), "grad init"))) return st;

    const double* sig = h->last_sigma;
    const double s1 = sig[0];
    const double cg_tol = sizeof(T) == 8 ? 1e-12 : 1e-6;
    const int cg_maxit = 2000;

    // 1. which score columns are active, and are their singular values separated?
    std::vector<int> active(k, 0);
    if (Sbar) {
        for (int i = 0; i < k; ++i) {
            const T* si = Sbar + (int64_t)i * n;
            double nrm = G.dot(si, si, n);
            if (G.err) return G.err;
            active[i] = nrm > 0.0;
            if (!active[i]) continue;
            double gap = sig[i] - h->last_next;
            for (int l = 0; l < k; ++l)
                if (l != i) gap = std::min(gap, std::fabs(sig[i] - sig[l]));
            if (!(gap >= min_relgap * s1))
                return set_err(h, GKL_ERR_GAP,
                               "score adjoint of component %d needs relative gap %.3e, have %.3e (sigma_%d = %.6g)", i,
                               min_relgap, gap / s1, i + 1, sig[i]);
        }
    }
    // 2. x_i for the active columns
    for (int i = 0; i < k; ++i) {
        if (!active[i]) continue;
        const T* si = Sbar + (int64_t)i * n;
        T* xi = G.X + (int64_t)i * m;
        if ((st = G.rmv(si, G.b))) return st;
        if ((st = G.dots(G.V, m, k, G.b, m))) return st;
        std::vector<double> c(k, 0.0);
        const double s2 = sig[i] * sig[i];
        for (int l = 0; l < k; ++l)
            if (l != i) c[l] = G.hc[l] / (s2 - sig[l] * sig[l]);
        if ((st = G.combine(c.data(), xi))) return st;
        // CG on range(P): y solves P (s2 I - A^T A) P y = P b
        if ((st = G.axpby(G.r, G.b, m, 1.0, 0.0))) return st;
        double rr = G.project(G.r, m, G.V, m, k);
        if (G.err) return G.err;
        const double r0 = std::sqrt(rr);
        if ((st = G.check(cudaMemsetAsync(G.y, 0, sizeof(T) * m, h->stream), "cg"))) return st;
        if ((st = G.axpby(G.p, G.r, m, 1.0, 0.0))) return st;
        int it = 0;
        for (; it < cg_maxit && std::sqrt(rr) > cg_tol * r0 && r0 > 0.0; ++it) {
            if ((st = G.mv(G.p, G.tn))) return st;
            if ((st = G.rmv(G.tn, G.q))) return st;
            if ((st = G.axpby(G.q, G.p, m, s2, -1.0))) return st;  // q = s2 p - A^T A p
            G.project(G.q, m, G.V, m, k);
            if (G.err) return G.err;
            double pq = G.dot(G.p, G.q, m);
            if (G.err) return G.err;
            if (!(pq > 0.0)) return set_err(h, GKL_ERR_GAP, "gradient solve for component %d lost definiteness", i);
            const double alpha = rr / pq;
            if ((st = G.axpby(G.y, G.p, m, alpha, 1.0))) return st;
            if ((st = G.axpby(G.r, G.q, m, -alpha, 1.0))) return st;
            double rn = G.dot(G.r, G.r, m);
            if (G.err) return G.err;
            const double beta = rn / rr;
            rr = rn;
            if ((st = G.axpby(G.p, G.r, m, 1.0, beta))) return st;
        }
        if (std::sqrt(rr) > cg_tol * r0 && r0 > 0.0)
            return set_err(h, GKL_NOT_CONVERGED, "gradient solve for component %d did not converge", i);
        if ((st = G.axpby(xi, G.y, m, 1.0, 1.0))) return st;
    }
    // 3. p_i = sigma_bar_i u_i + s_bar_i + A x_i
    for (int i = 0; i < k; ++i) {
        T* pi = G.Pn + (int64_t)i * n;
        const T* ui = G.U + (int64_t)i * n;
        if (active[i]) {
            if ((st = G.mv(G.X + (int64_t)i * m, pi))) return st;
            if ((st = G.axpby(pi, Sbar + (int64_t)i * n, n, 1.0, 1.0))) return st;
            if ((st = G.axpby(pi, ui, n, sigma_bar ? sigma_bar[i] : 0.0, 1.0))) return st;
        } else {
            if ((st = G.axpby(pi, ui, n, sigma_bar ? sigma_bar[i] : 0.0, 0.0))) return st;
        }
    }
    // 4. per-weight sums over the rank-one terms (p_i v_i^T) and (sigma_i u_i x_i^T)
    if (g_w) {
        if ((st = G.check(cudaMemsetAsync(g_w, 0, sizeof(T) * m, h->stream), "g_w"))) return st;
        for (int i = 0; i < k; ++i) {
            if ((st = G.rmv(G.Pn + (int64_t)i * n, G.q))) return st;
            if ((st = G.fma(g_w, G.V + (int64_t)i * m, G.q, m, 1.0))) return st;
            if (active[i]) {
                if ((st = G.rmv(G.U + (int64_t)i * n, G.q))) return st;
                if ((st = G.fma(g_w, G.X + (int64_t)i * m, G.q, m, sig[i]))) return st;
            }
        }
        if (h->w) {
            k_div_weights<T><<<blocks_for(m), 256, 0, h->stream>>>(g_w, h->w, m);
            if ((st = G.check(cudaGetLastError(), "g_w"))) return st;
        }
    }
    if (g_s) {
        if ((st = G.check(cudaMemsetAsync(g_s, 0, sizeof(T) * n, h->stream), "g_s"))) return st;
        for (int i = 0; i < k; ++i) {
            if ((st = G.mv(G.V + (int64_t)i * m, G.tn))) return st;
            if ((st = G.fma(g_s, G.Pn + (int64_t)i * n, G.tn, n, 1.0))) return st;
            if (active[i]) {
                if ((st = G.mv(G.X + (int64_t)i * m, G.tn))) return st;
                if ((st = G.fma(g_s, G.U + (int64_t)i * n, G.tn, n, sig[i]))) return st;
            }
        }
        if (h->s) {
            k_div_weights<T><<<blocks_for(n), 256, 0, h->stream>>>(g_s, h->s, n);
            if ((st = G.check(cudaGetLastError(), "g_s"))) return st;
        }
    }
    if ((st = G.check(cudaStreamSynchronize(h->stream), "gradient"))) return st;
    return take_pending_error(h);  // a tensor-core product whose bounded wait ran out
}

}  // namespace gkl

using namespace gkl;

extern "C" int gkl_grad(gkl_handle* h, const double* sigma_bar, const void* scores_bar, void* g_w, void* g_s,
                        double min_relgap) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    if (!h->last_valid)
        return set_err(h, GKL_ERR_STATE,
                       "gkl_grad needs a converged gkl_svd on this handle, with the current weights, first");
    if (!g_w && !g_s) return set_err(h, GKL_ERR_ARG, "nothing to compute: g_w and g_s are both NULL");
    if (!(min_relgap >= 0.0)) return set_err(h, GKL_ERR_ARG, "min_relgap must be >= 0");
    for (const void* p : {scores_bar, static_cast<const void*>(g_w), static_cast<const void*>(g_s)})
        if (p && mem_kind(p, h->device) != MEM_DEVICE)
            return set_err(h, GKL_ERR_ARG, "scores_bar, g_w and g_s must be device memory of the handle's GPU");
    if (sigma_bar && mem_kind(sigma_bar, h->device) != MEM_HOST)
        return set_err(h, GKL_ERR_ARG, "sigma_bar must be host memory");
    if (h->last_prec == GKL_FP64)
        return run_grad<double>(h, sigma_bar, static_cast<const double*>(scores_bar), static_cast<double*>(g_w),
                                static_cast<double*>(g_s), min_relgap);
    return run_grad<float>(h, sigma_bar, static_cast<const float*>(scores_bar), static_cast<float*>(g_w),
                           static_cast<float*>(g_s), min_relgap);
}
