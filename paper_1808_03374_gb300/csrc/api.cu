// C ABI and host driver of the thick-restarted GKL solver.
//
// The driver enqueues the Lanczos steps of one restart cycle on the handle's
// stream without synchronising: every scalar decision of a step (Lanczos
// coefficient, partial-reorthogonalisation trigger, breakdown) is taken on the
// device by the last block of a reduction, and later kernels read it from
// device memory.  The host synchronises once per cycle, after the projected
// SVD, to read the convergence flag (section 3 of arXiv:1808.03374:
// thick restart with ordinary Ritz vectors, residual-norm convergence test).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "gkl_internal.cuh"

static thread_local char g_init_err[512] = "no error";

namespace gkl {

int set_err(gkl_handle* h, int code, const char* fmt, ...) {
    char* buf = h ? h->err : g_init_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_err(gkl_handle* h, cudaError_t e, const char* what) {
    return set_err(h, GKL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ensure_scratch(gkl_handle* h, size_t bytes) {
    if (h->scratch_bytes >= bytes) return GKL_OK;
    if (h->scratch) cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_bytes = 0;
    cudaError_t e = cudaMalloc(&h->scratch, bytes);
    if (e != cudaSuccess) return cuda_err(h, e, "scratch allocation");
    h->scratch_bytes = bytes;
    return GKL_OK;
}

// Synchronise the handle's stream and report (then clear) a bounded
// tensor-core pipeline wait that ran out since the last check.
int take_pending_error(gkl_handle* h) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "stream synchronisation");
    if (!h->aux) return GKL_OK;
    int terr = 0;
    int* ew = reinterpret_cast<int*>(reinterpret_cast<char*>(h->aux) + kAuxErrOffset);
    e = cudaMemcpyAsync(&terr, ew, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "error-word read");
    if (terr == 0) return GKL_OK;
    e = cudaMemsetAsync(ew, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err(h, e, "error-word clear");
    return set_err(h, GKL_ERR_CUDA, "tensor-core product: a bounded pipeline wait ran out (code %d)", terr);
}

static int ensure_ws(gkl_handle* h, size_t bytes) {
    if (h->ws_bytes >= bytes) return GKL_OK;
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    cudaError_t e = cudaMalloc(&h->ws, bytes);
    if (e != cudaSuccess) return cuda_err(h, e, "workspace allocation");
    h->ws_bytes = bytes;
    return GKL_OK;
}

int mem_kind(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return MEM_BAD;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return a.device == device ? MEM_DEVICE : MEM_BAD;
    return MEM_HOST;  // cudaMemoryTypeHost or cudaMemoryTypeUnregistered
}

static int current_device() {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return d;
}

// Device memory of the current device.
static bool is_device_ptr(const void* p) { return mem_kind(p, current_device()) == MEM_DEVICE; }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Numerical rank among the k leading values (descending): the count of values
// above 1000 * eps_w * sigma_1, eps_w the unit roundoff of the arithmetic.
int numerical_rank(const double* sg, int k, double eps_w) {
    const double thr = 1e3 * eps_w * (k > 0 ? sg[0] : 0.0);
    int r = 0;
    while (r < k && sg[r] > thr) ++r;
    return r;
}

// Host copy of the device scalars (read once per cycle).
struct HostState {
    DevScal sc;
};

template <typename T>
struct Driver {
    gkl_handle* h;
    Sv sv;
    T* U;
    T* V;
    int* signs;
    T* vtmp;
    int64_t n, m;
    int ell, k, kk;
    uint32_t draws = 0;
    int64_t products = 0;
    int breakdowns = 0;
    int64_t launches = 0;
    // optional CUDA-event timing of the main product kernels
    bool profile = false;
    std::vector<cudaEvent_t> ev_mv, ev_rmv, ev_svd, ev_cgs;  // pairs (begin, end)
    size_t used_mv = 0, used_rmv = 0, used_svd = 0, used_cgs = 0;
    double ms_mv = 0.0, ms_rmv = 0.0, ms_svd = 0.0, ms_cgs = 0.0;
    int64_t n_mv = 0, n_rmv = 0;

    ~Driver() {
        for (auto* pool : {&ev_mv, &ev_rmv, &ev_svd, &ev_cgs})
            for (cudaEvent_t e : *pool) cudaEventDestroy(e);
    }

    // Record the begin (end = false) or end event of a timed group.
    void mark(std::vector<cudaEvent_t>& pool, size_t& used, bool end) {
        if (!profile) return;
        if (!end) {
            cudaEvent_t b, e;
            next_pair(pool, used, &b, &e);
            if (b) cudaEventRecord(b, h->stream);
        } else if (used >= 2) {
            cudaEventRecord(pool[used - 1], h->stream);
        }
    }

    static double sum_pairs(const std::vector<cudaEvent_t>& pool, size_t used, int64_t* count) {
        double s = 0.0;
        for (size_t i = 0; i + 1 < used; i += 2) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, pool[i], pool[i + 1]) == cudaSuccess) {
                s += t;
                if (count) ++*count;
            }
        }
        return s;
    }

    int check(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return GKL_OK;
        return cuda_err(h, e, what);
    }

    // Next (begin, end) event pair of a pool, created on first use.
    void next_pair(std::vector<cudaEvent_t>& pool, size_t& used, cudaEvent_t* b, cudaEvent_t* e) {
        *b = *e = nullptr;
        if (!profile) return;
        if (used + 2 > pool.size()) {
            cudaEvent_t x, y;
            if (cudaEventCreate(&x) != cudaSuccess) return;
            if (cudaEventCreate(&y) != cudaSuccess) { cudaEventDestroy(x); return; }
            pool.push_back(x);
            pool.push_back(y);
        }
        *b = pool[used];
        *e = pool[used + 1];
        used += 2;
    }

    // Add up the event pairs recorded since the last harvest (stream synchronised).
    void harvest() {
        ms_mv += sum_pairs(ev_mv, used_mv, &n_mv);
        ms_rmv += sum_pairs(ev_rmv, used_rmv, &n_rmv);
        ms_svd += sum_pairs(ev_svd, used_svd, nullptr);
        ms_cgs += sum_pairs(ev_cgs, used_cgs, nullptr);
        cudaGetLastError();
        used_mv = used_rmv = used_svd = used_cgs = 0;
    }

    int cgs(int mode, T* x, int64_t len, const T* W, int64_t ldw, int ncols, const int* cond, int role, int j,
            uint32_t draw = 0, int* second = nullptr) {
        ++launches;
        return check(launch_cgs<T>(sv, h->stream, mode, x, len, W, ldw, ncols, cond, role, j, draw, h->num_sms, second),
                     "cgs");
    }

    // Flag and count of the adaptive second Gram-Schmidt pass of one side (DGKS
    // and ONESIDED), or null where both passes always run (FULL and PARTIAL).
    int* second_of(int side) {
        if (sv.reorth != GKL_REORTH_DGKS && sv.reorth != GKL_REORTH_ONESIDED) return nullptr;
        return side == 0 ? sv.sc->second_u : sv.sc->second_v;
    }

    int scale(T* x, int64_t len, const double* f) {
        ++launches;
        return check(launch_scale<T>(sv, h->stream, x, len, f), "scale");
    }

    int half_u(int j) {
        T* y = U + (int64_t)j * sv.ldu;
        FinArgs fa{sv.B + (int64_t)j * ell, j, U, sv.ldu, ROLE_U_PRE, j};
        cudaEvent_t e0, e1;
        next_pair(ev_mv, used_mv, &e0, &e1);
        int nl = 0;
        int st = check(launch_matvec<T>(h, V + (int64_t)j * sv.ldv, y, h->scratch, &sv, &fa, e0, e1, &nl), "A.v");
        launches += nl;
        if (st) return st;
        if (j > 0) {
            const int* cond = &sv.sc->reorth_u;
            int* sec = second_of(0);
            mark(ev_cgs, used_cgs, false);
            if ((st = cgs(CGS_DOTS, y, n, U, sv.ldu, j, cond, 0, j, 0, sec))) return st;
            if ((st = cgs(CGS_UPD_DOTS, y, n, U, sv.ldu, j, cond, 0, j, 0, sec))) return st;
            if ((st = cgs(CGS_UPD_NORM, y, n, U, sv.ldu, j, cond, ROLE_U_POST, j, 0, sec))) return st;
            mark(ev_cgs, used_cgs, true);
        }
        return scale(y, n, &sv.sc->scale_u);
    }

    int half_v(int j) {
        T* x = V + (int64_t)(j + 1) * sv.ldv;
        FinArgs fa{sv.B + j + (int64_t)j * ell, 1, V + (int64_t)j * sv.ldv, sv.ldv, ROLE_V_PRE, j};
        cudaEvent_t e0, e1;
        next_pair(ev_rmv, used_rmv, &e0, &e1);
        int nl = 0;
        int st = check(launch_rmatvec<T>(h, U + (int64_t)j * sv.ldu, x, h->scratch, &sv, &fa, e0, e1, &nl), "A^T.u");
        launches += nl;
        if (st) return st;
        const int* cond = &sv.sc->reorth_v;
        int* sec = second_of(1);
        mark(ev_cgs, used_cgs, false);
        if ((st = cgs(CGS_DOTS, x, m, V, sv.ldv, j + 1, cond, 0, j, 0, sec))) return st;
        if ((st = cgs(CGS_UPD_DOTS, x, m, V, sv.ldv, j + 1, cond, 0, j, 0, sec))) return st;
        if ((st = cgs(CGS_UPD_NORM, x, m, V, sv.ldv, j + 1, cond, ROLE_V_POST, j, 0, sec))) return st;
        mark(ev_cgs, used_cgs, true);
        return scale(x, m, &sv.sc->scale_v);
    }

    // Orthonormalise x against the first ncols columns of W with CGS2; with
    // fill, x is first replaced by a fresh counter-based random vector.
    int orthonormalise(T* x, int64_t len, const T* W, int64_t ldw, int ncols, int role, int j, bool fill,
                       const double* f) {
        int st;
        if (fill) {
            if ((st = cgs(CGS_FILL_DOTS, x, len, W, ldw, ncols, nullptr, 0, j, draws++))) return st;
        } else if ((st = cgs(CGS_DOTS, x, len, W, ldw, ncols, nullptr, 0, j))) {
            return st;
        }
        if ((st = cgs(CGS_UPD_DOTS, x, len, W, ldw, ncols, nullptr, 0, j))) return st;
        if ((st = cgs(CGS_UPD_NORM, x, len, W, ldw, ncols, nullptr, role, j))) return st;
        return scale(x, len, f);
    }

    int read_state(DevScal* out) {
        cudaError_t e = cudaMemcpyAsync(out, sv.sc, sizeof(DevScal), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        return check(e, "state read-back");
    }

    int clear_abort() {
        return check(cudaMemsetAsync(&sv.sc->abort, 0, sizeof(int), h->stream), "clear abort");
    }

    // Replace the vector of a breakdown by a fresh one orthogonal to its basis.
    int replace(int j, int side) {
        for (int attempt = 0; attempt < 4; ++attempt) {
            int st = clear_abort();
            if (st) return st;
            if (side == 0)
                st = orthonormalise(U + (int64_t)j * sv.ldu, n, U, sv.ldu, j, ROLE_REPL_U, j, true, &sv.sc->scale_u);
            else
                st = orthonormalise(V + (int64_t)(j + 1) * sv.ldv, m, V, sv.ldv, j + 1, ROLE_REPL_V, j, true,
                                    &sv.sc->scale_v);
            if (st) return st;
            DevScal hs;
            if ((st = read_state(&hs))) return st;
            if (hs.abort == ABORT_NONE) return GKL_OK;
        }
        return set_err(h, GKL_ERR_NONFINITE, "could not replace the vector after a Lanczos breakdown at step %d", j);
    }
};

template <typename T>
static int run_svd(gkl_handle* h, const gkl_opts* o, double* sigma, T* Uout, T* Vout, double* resid,
                   gkl_info* info) {
    const int64_t n = h->n, m = h->m;
    const int k = o->k, ell = o->ell;
    const int kk = o->k_keep > 0 ? o->k_keep : k + (ell - k) / 2;
    if (k < 1 || ell <= k || ell > GKL_MAX_ELL || ell > n || ell > m)
        return set_err(h, GKL_ERR_ARG, "need 1 <= k < ell <= min(n, m, %d) (k=%d ell=%d)", GKL_MAX_ELL, k, ell);
    if (kk < k || kk >= ell) return set_err(h, GKL_ERR_ARG, "need k <= k_keep < ell (k_keep=%d)", kk);
    if (o->maxit < 1 || !(o->tol >= 0.0)) return set_err(h, GKL_ERR_ARG, "need maxit >= 1 and tol >= 0");

    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        EventPair() { cudaEventCreate(&a); cudaEventCreate(&b); }
        ~EventPair() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
    } wall;
    cudaEventRecord(wall.a, h->stream);

    MvPlan plan = plan_products(h);
    int st = ensure_scratch(h, plan.bytes_fp64);
    if (st) return st;

    const int64_t ldu = (n + 31) / 32 * 32, ldv = (m + 31) / 32 * 32;
    const int L = ell + 1;
    const int64_t maxblk = std::max<int64_t>({(n + 255) / 256, (m + 255) / 256, 4 * (int64_t)h->num_sms}) + 8;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align256(off + bytes); return at; };
    size_t oU = take(sizeof(T) * ldu * ell);
    size_t oV = take(sizeof(T) * ldv * (ell + 1));
    size_t oB = take(sizeof(double) * ell * ell);
    size_t oMu = take(sizeof(double) * L * L);
    size_t oNu = take(sizeof(double) * L * L);
    size_t oPQ = take(sizeof(double) * 4 * ell * ell);  // P, Q and the FP64 Jacobi workspace
    size_t oRw = take(sizeof(double) * 8 * ell * ell);  // refinement workspace
    size_t oSc = take(sizeof(DevScal));
    size_t oCo = take(sizeof(CycleOut));
    size_t oPart = take(sizeof(double) * maxblk * (GKL_MAX_ELL + 2));
    size_t oCoef = take(sizeof(double) * 2 * (GKL_MAX_ELL + 2));
    size_t oSign = take(sizeof(int) * GKL_MAX_ELL);
    size_t oVt = take(Vout ? 0 : sizeof(T) * m * k);
    if ((st = ensure_ws(h, off))) return st;
    char* base = static_cast<char*>(h->ws);

    Driver<T> D;
    D.h = h;
    D.n = n;
    D.m = m;
    D.ell = ell;
    D.k = k;
    D.kk = kk;
    D.profile = o->profile != 0;
    D.U = reinterpret_cast<T*>(base + oU);
    D.V = reinterpret_cast<T*>(base + oV);
    D.signs = reinterpret_cast<int*>(base + oSign);
    D.vtmp = reinterpret_cast<T*>(base + oVt);
    Sv& sv = D.sv;
    sv = Sv{};
    sv.n = n;
    sv.m = m;
    sv.ldu = ldu;
    sv.ldv = ldv;
    sv.ell = ell;
    sv.kk = kk;
    sv.k = k;
    sv.reorth = o->reorth;
    sv.kk_start = 0;
    sv.prec = sizeof(T) == 8 ? GKL_FP64 : GKL_FP32;
    sv.U = D.U;
    sv.V = D.V;
    sv.B = reinterpret_cast<double*>(base + oB);
    sv.muh = reinterpret_cast<double*>(base + oMu);
    sv.nuh = reinterpret_cast<double*>(base + oNu);
    sv.P = reinterpret_cast<double*>(base + oPQ);
    sv.Q = sv.P + (size_t)ell * ell;
    sv.rw = reinterpret_cast<double*>(base + oRw);
    sv.sc = reinterpret_cast<DevScal*>(base + oSc);
    sv.co = reinterpret_cast<CycleOut*>(base + oCo);
    sv.partials = reinterpret_cast<double*>(base + oPart);
    sv.coef = reinterpret_cast<double*>(base + oCoef);
    sv.eps_w = sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    // partial / one-sided trigger level: the true residual of the output follows the
    // orthogonality kept (measured about 0.1 omega sigma_1), so the default is
    // min(1e-8 (FP64) or 2^-12 (FP32), 10 tol), and at least 10 eps_w
    sv.omega = o->omega > 0.0 ? o->omega
                              : std::min(sizeof(T) == 8 ? 1e-8 : 2.44140625e-04, std::max(10.0 * o->tol, 10.0 * sv.eps_w));
    sv.tol = o->tol;
    sv.seed = o->seed;

    D.launches += 1;
    if ((st = D.check(launch_init_state(sv, h->stream), "init"))) return st;
    // start vector v_0: given, or drawn from the counter-based generator
    T* v0 = D.V;
    if (o->v0) {
        if ((st = D.check(cudaMemcpyAsync(v0, o->v0, sizeof(T) * m, cudaMemcpyDeviceToDevice, h->stream), "v0 copy")))
            return st;
    } else {
        D.launches += 1;
        if ((st = D.check(launch_fill_random<T>(sv, h->stream, v0, m, 0xFFFFFFFFu, 0), "v0 fill"))) return st;
    }
    if ((st = D.cgs(CGS_UPD_NORM, v0, m, D.V, ldv, 0, nullptr, ROLE_START, 0))) return st;
    if ((st = D.scale(v0, m, &sv.sc->scale_v))) return st;

    CycleOut* ho = h->host_out;
    DevScal hs;
    int cycle = 0, restarts = 0, max_sweeps = 0;
    int pos_j = 0, pos_side = 0;
    bool converged = false;
    for (;;) {
        sv.kk_start = (cycle == 0) ? 0 : kk;
        const int start_j = pos_j, start_side = pos_side;
        for (int j = pos_j, side = pos_side; j < ell;) {
            st = side == 0 ? D.half_u(j) : D.half_v(j);
            if (st) return st;
            if (side == 0) side = 1;
            else { side = 0; ++j; }
        }
        D.launches += 12;  // FP32 Jacobi, 4 x 2 refinement kernels, check, final, FP64 fallback
        D.mark(D.ev_svd, D.used_svd, false);
        if ((st = D.check(launch_small_svd(sv, h->stream, 1), "projected SVD"))) return st;
        D.mark(D.ev_svd, D.used_svd, true);
        if ((st = D.check(cudaMemcpyAsync(ho, sv.co, sizeof(CycleOut), cudaMemcpyDeviceToHost, h->stream), "read")))
            return st;
        if ((st = D.read_state(&hs))) return st;
        D.harvest();
        if (hs.abort == ABORT_NONE) max_sweeps = std::max(max_sweeps, ho->sweeps);
        if (hs.abort == ABORT_NONFINITE)
            return set_err(h, GKL_ERR_NONFINITE, "non-finite Lanczos coefficient at step %d (%s side)", hs.break_step,
                           hs.break_side ? "v" : "u");
        if (hs.abort == ABORT_BREAKDOWN) {
            const int bj = hs.break_step, bs = hs.break_side;
            D.products += (bj - start_j) + (start_side == 0 ? 1 : 0);
            D.breakdowns += 1;
            if ((st = D.replace(bj, bs))) return st;
            pos_j = bs == 0 ? bj : bj + 1;
            pos_side = bs == 0 ? 1 : 0;
            continue;
        }
        D.products += (ell - start_j) - (start_side == 1 ? 1 : 0);
        converged = ho->conv != 0;
        if (converged || cycle == o->maxit - 1) break;
        // thick restart: keep kk Ritz vectors, v_kk <- v_ell
        D.launches += 2;
        if ((st = D.check(launch_rotate<T>(h->stream, D.U, ldu, ell, sv.P, ell, kk, D.U, ldu, n), "rotate U"))) return st;
        if ((st = D.check(launch_rotate<T>(h->stream, D.V, ldv, ell, sv.Q, ell, kk, D.V, ldv, m), "rotate V"))) return st;
        if ((st = D.check(cudaMemcpyAsync(D.V + (int64_t)kk * ldv, D.V + (int64_t)ell * ldv, sizeof(T) * m,
                                          cudaMemcpyDeviceToDevice, h->stream),
                          "v restart copy")))
            return st;
        if (o->reorth == GKL_REORTH_PARTIAL || (o->reorth == GKL_REORTH_ONESIDED && n <= m)) {
            // partial reorthogonalisation of the v side keeps v_ell only semi-orthogonal to V; restore it
            // against the kept vectors
            if ((st = D.orthonormalise(D.V + (int64_t)kk * ldv, m, D.V, ldv, kk, ROLE_REPL_V, kk - 1, false,
                                       &sv.sc->scale_v)))
                return st;
        }
        ++cycle;
        ++restarts;
        pos_j = kk;
        pos_side = 0;
    }
    // outputs: U_ell P[:, :k], V_ell Q[:, :k], sign rule; the triplets stay in
    // the handle for gkl_grad
    h->last_valid = 0;
    const size_t lb = sizeof(T) * (size_t)(n + m) * k;
    if (h->last_bytes < lb) {
        if (h->last_U) cudaFree(h->last_U);
        h->last_U = nullptr;
        h->last_bytes = 0;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, lb);
        if (e != cudaSuccess) return cuda_err(h, e, "output buffers");
        h->last_U = p;
        h->last_bytes = lb;
    }
    h->last_V = static_cast<char*>(h->last_U) + sizeof(T) * (size_t)n * k;
    T* Uo = static_cast<T*>(h->last_U);
    T* Vo = static_cast<T*>(h->last_V);
    D.launches += 4;
    if ((st = D.check(launch_rotate<T>(h->stream, D.U, ldu, ell, sv.P, ell, k, Uo, n, n), "U out"))) return st;
    if ((st = D.check(launch_rotate<T>(h->stream, D.V, ldv, ell, sv.Q, ell, k, Vo, m, m), "V out"))) return st;
    // One-sided reorthogonalisation leaves the vectors of the side that was not
    // reorthogonalised at every step with that basis's loss of orthogonality.
    // They are recomputed from the other side, v_i = A^T u_i (or u_i = A v_i),
    // and orthonormalised in order; the values below the numerical rank keep
    // theirs.
    const int rank0 = numerical_rank(ho->sg, k, sv.eps_w);
    if (o->reorth == GKL_REORTH_ONESIDED) {
        const bool from_u = n <= m;  // the side kept orthonormal at every step
        const int64_t len = from_u ? m : n;
        T* W = from_u ? Vo : Uo;
        for (int i = 0; i < rank0; ++i) {
            int nl = 0;
            T* dst = W + (int64_t)i * len;
            cudaError_t e = from_u ? launch_rmatvec<T>(h, Uo + (int64_t)i * n, dst, h->scratch, nullptr, nullptr,
                                                       nullptr, nullptr, &nl)
                                   : launch_matvec<T>(h, Vo + (int64_t)i * m, dst, h->scratch, nullptr, nullptr,
                                                      nullptr, nullptr, &nl);
            D.launches += nl;
            if ((st = D.check(e, "one-sided recomputation"))) return st;
            if (i == 0) {
                if ((st = D.cgs(CGS_UPD_NORM, dst, len, W, len, 0, nullptr, ROLE_START, 0))) return st;
                if ((st = D.scale(dst, len, &sv.sc->scale_v))) return st;
            } else if ((st = D.orthonormalise(dst, len, W, len, i, ROLE_START, 0, false, &sv.sc->scale_v))) {
                return st;
            }
        }
        D.products += (rank0 + 1) / 2;  // one product per vector: half a pair
    }
    if ((st = D.check(launch_sign_fix<T>(h->stream, Uo, n, Vo, m, k, D.signs), "sign"))) return st;
    // U, V out: device-to-device, or device-to-host with o->out_host
    if (Uout && (st = D.check(cudaMemcpyAsync(Uout, Uo, sizeof(T) * n * k, cudaMemcpyDefault, h->stream), "U copy")))
        return st;
    if (Vout && (st = D.check(cudaMemcpyAsync(Vout, Vo, sizeof(T) * m * k, cudaMemcpyDefault, h->stream), "V copy")))
        return st;
    cudaEventRecord(wall.b, h->stream);
    if ((st = D.check(cudaStreamSynchronize(h->stream), "final sync"))) return st;
    if ((st = take_pending_error(h))) return st;
    const int rank = numerical_rank(ho->sg, k, sv.eps_w);
    h->last_valid = converged ? 1 : 0;
    h->last_prec = sizeof(T) == 8 ? GKL_FP64 : GKL_FP32;
    h->last_k = k;
    for (int i = 0; i < k; ++i) h->last_sigma[i] = i < rank ? ho->sg[i] : 0.0;
    h->last_next = k < ell ? ho->sg[k] : 0.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, wall.a, wall.b);
    for (int i = 0; i < k; ++i) {
        sigma[i] = h->last_sigma[i];
        if (resid) resid[i] = ho->resid[i];
    }
    if (info) {
        info->matvec_pairs = D.products;
        info->restarts = restarts;
        info->cycles = cycle + 1;
        info->reorth_u = hs.n_reorth_u;
        info->reorth_v = hs.n_reorth_v;
        info->breakdowns = D.breakdowns;
        info->converged = converged ? 1 : 0;
        info->max_rel_resid = ho->maxrel;
        info->dtheta1 = ho->dtheta;
        info->ms_total = ms;
        info->launches = D.launches;
        info->n_mv = D.n_mv;
        info->n_rmv = D.n_rmv;
        info->ms_mv = D.ms_mv;
        info->ms_rmv = D.ms_rmv;
        info->jacobi_sweeps = max_sweeps;
        info->svd_fallbacks = hs.n_svd_fallback;
        info->svd_clusters = hs.n_svd_cluster;
        info->rank = rank;
        info->ms_svd = D.ms_svd;
        info->ms_cgs = D.ms_cgs;
        info->second_u = hs.second_u[1];
        info->second_v = hs.second_v[1];
    }
    if (!converged) {
        set_err(h, GKL_NOT_CONVERGED, "not converged after %d cycles (max rel. residual %.3e)", cycle + 1, ho->maxrel);
        return GKL_NOT_CONVERGED;
    }
    if (rank < k)
        return set_err(h, GKL_RANK_DEFICIENT, "numerical rank %d < k = %d: sigma_%d.. reported as 0", rank, k,
                       rank + 1);
    return GKL_OK;
}

}  // namespace gkl

using namespace gkl;

extern "C" {

const char* gkl_version(void) { return "gkl-gb300 0.1 (sm_103a)"; }

const char* gkl_last_error(const gkl_handle* h) { return h ? h->err : g_init_err; }

void gkl_opts_default(gkl_opts* o) {
    if (!o) return;
    o->k = 10;
    o->ell = 30;
    o->k_keep = 0;
    o->reorth = GKL_REORTH_DGKS;
    o->out_host = 0;
    o->reserved0 = 0;
    o->precision = GKL_FP64;
    o->maxit = 1000;
    o->profile = 0;
    o->block = 0;
    o->tol = 1e-10;
    o->omega = 0.0;
    o->seed = 1;
    o->v0 = nullptr;
}

static int check_layout(gkl_handle* h, const uint8_t* packed, int64_t n, int64_t m, int64_t stride) {
    if (!packed) return set_err(h, GKL_ERR_ARG, "packed is NULL");
    if (n < 1 || m < 1) return set_err(h, GKL_ERR_ARG, "need n >= 1 and m >= 1 (n=%lld m=%lld)", (long long)n, (long long)m);
    if (stride % 16 != 0 || stride * 4 < n)
        return set_err(h, GKL_ERR_ARG, "stride must be a multiple of 16 and >= ceil(n/4) (stride=%lld)", (long long)stride);
    if (((uintptr_t)packed & 15u) != 0) return set_err(h, GKL_ERR_ARG, "packed must be 16-byte aligned");
    if (!is_device_ptr(packed)) return set_err(h, GKL_ERR_ARG, "packed must be device memory");
    return GKL_OK;
}

int gkl_colstats(const uint8_t* packed, int64_t n, int64_t m, int64_t stride, double* mu, double* scale, int64_t* nobs,
                 void* stream) {
    int st = check_layout(nullptr, packed, n, m, stride);
    if (st) return st;
    if ((mu && !is_device_ptr(mu)) || (scale && !is_device_ptr(scale)) || (nobs && !is_device_ptr(nobs)))
        return set_err(nullptr, GKL_ERR_ARG, "outputs must be device memory");
    cudaError_t e = launch_colstats(packed, n, m, stride, mu, scale, nobs, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_err(nullptr, e, "colstats launch");
    return GKL_OK;
}

int gkl_init(gkl_handle** out, const uint8_t* packed, int64_t n, int64_t m, int64_t stride, const double* mu,
             const double* scale, void* stream) {
    if (!out) return set_err(nullptr, GKL_ERR_ARG, "handle pointer is NULL");
    *out = nullptr;
    int st = check_layout(nullptr, packed, n, m, stride);
    if (st) return st;
    if ((mu == nullptr) != (scale == nullptr)) return set_err(nullptr, GKL_ERR_ARG, "give both mu and scale, or neither");
    gkl_handle* h = new (std::nothrow) gkl_handle();
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "out of host memory");
    std::strcpy(h->err, "no error");
    h->packed = packed;
    h->n = n;
    h->m = m;
    h->stride = stride;
    h->stream = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    cudaError_t e = cudaMalloc(&h->mu, sizeof(double) * m);
    if (e == cudaSuccess) e = cudaMalloc(&h->d, sizeof(double) * m);
    if (e == cudaSuccess) e = cudaMallocHost(&h->host_out, sizeof(CycleOut));
    if (e == cudaSuccess) e = cudaMalloc(&h->aux, kAuxBytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->aux, 0, kAuxBytes, h->stream);
    if (e != cudaSuccess) {
        cuda_err(nullptr, e, "gkl_init allocation");
        gkl_destroy(h);
        return GKL_ERR_CUDA;
    }
    // the FP32 products read the packed matrix through TMA descriptors; A^T u runs on the tensor cores
    if (!make_mv_map(packed, stride, m, h->mv_map) || !tc_prepare(h)) {
        cudaGetLastError();
        set_err(nullptr, GKL_ERR_CUDA, "gkl_init: the tensor-core A^T u could not be prepared");
        gkl_destroy(h);
        return GKL_ERR_CUDA;
    }
    if (mu) {
        e = cudaMemcpyAsync(h->mu, mu, sizeof(double) * m, cudaMemcpyDefault, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->d, scale, sizeof(double) * m, cudaMemcpyDefault, h->stream);
    } else {
        e = launch_colstats(packed, n, m, stride, h->mu, h->d, nullptr, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cuda_err(nullptr, e, "gkl_init");
        gkl_destroy(h);
        return GKL_ERR_CUDA;
    }
    *out = h;
    return GKL_OK;
}

int gkl_set_stream(gkl_handle* h, void* stream) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    h->stream = (cudaStream_t)stream;
    return GKL_OK;
}

static int set_vec(gkl_handle* h, float** slot, const float* src, int64_t len, const char* what) {
    if (!src) {
        if (*slot) cudaFree(*slot);
        *slot = nullptr;
        return GKL_OK;
    }
    if (!*slot) {
        cudaError_t e = cudaMalloc(slot, sizeof(float) * len);
        if (e != cudaSuccess) return cuda_err(h, e, what);
    }
    cudaError_t e = cudaMemcpyAsync(*slot, src, sizeof(float) * len, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? GKL_OK : cuda_err(h, e, what);
}

int gkl_set_weights(gkl_handle* h, const float* s, const float* w) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    h->last_valid = 0;  // the stored triplets belong to the previous operator
    int st = set_vec(h, &h->s, s, h->n, "sample weights");
    if (st) return st;
    return set_vec(h, &h->w, w, h->m, "SNP weights");
}

int gkl_matvec(gkl_handle* h, int prec, const void* v, void* y) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    if (!v || !y || v == y) return set_err(h, GKL_ERR_ARG, "v and y must be distinct non-NULL device buffers");
    if (mem_kind(v, h->device) != MEM_DEVICE || mem_kind(y, h->device) != MEM_DEVICE)
        return set_err(h, GKL_ERR_ARG, "v and y must be device memory of the handle's GPU");
    if (prec != GKL_FP64 && prec != GKL_FP32) return set_err(h, GKL_ERR_ARG, "unknown precision %d", prec);
    MvPlan p = plan_products(h);
    int st = ensure_scratch(h, p.bytes_fp64);
    if (st) return st;
    cudaError_t e = prec == GKL_FP64
                        ? launch_matvec<double>(h, (const double*)v, (double*)y, h->scratch, nullptr, nullptr)
                        : launch_matvec<float>(h, (const float*)v, (float*)y, h->scratch, nullptr, nullptr);
    return e == cudaSuccess ? GKL_OK : cuda_err(h, e, "A.v launch");
}

int gkl_rmatvec(gkl_handle* h, int prec, const void* u, void* x) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    if (!u || !x || u == x) return set_err(h, GKL_ERR_ARG, "u and x must be distinct non-NULL device buffers");
    if (mem_kind(u, h->device) != MEM_DEVICE || mem_kind(x, h->device) != MEM_DEVICE)
        return set_err(h, GKL_ERR_ARG, "u and x must be device memory of the handle's GPU");
    if (prec != GKL_FP64 && prec != GKL_FP32) return set_err(h, GKL_ERR_ARG, "unknown precision %d", prec);
    MvPlan p = plan_products(h);
    int st = ensure_scratch(h, p.bytes_fp64);
    if (st) return st;
    cudaError_t e = prec == GKL_FP64
                        ? launch_rmatvec<double>(h, (const double*)u, (double*)x, h->scratch, nullptr, nullptr)
                        : launch_rmatvec<float>(h, (const float*)u, (float*)x, h->scratch, nullptr, nullptr);
    return e == cudaSuccess ? GKL_OK : cuda_err(h, e, "A^T.u launch");
}

int gkl_svd(gkl_handle* h, const gkl_opts* o, double* sigma, void* U, void* V, double* resid, gkl_info* info) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    if (!o) return set_err(h, GKL_ERR_ARG, "NULL options");
    if (o->reorth < GKL_REORTH_FULL || o->reorth > GKL_REORTH_ONESIDED)
        return set_err(h, GKL_ERR_ARG, "unknown reorthogonalisation mode %d", o->reorth);
    if (o->reserved0 != 0) return set_err(h, GKL_ERR_ARG, "gkl_opts.reserved0 must be 0");
    if (!sigma) return set_err(h, GKL_ERR_ARG, "sigma must not be NULL");
    if (o->v0 && mem_kind(o->v0, h->device) != MEM_DEVICE)
        return set_err(h, GKL_ERR_ARG, "v0 must be device memory of the handle's GPU");
    const int want = o->out_host ? MEM_HOST : MEM_DEVICE;
    if ((U && mem_kind(U, h->device) != want) || (V && mem_kind(V, h->device) != want))
        return set_err(h, GKL_ERR_ARG, o->out_host ? "out_host is set: U and V must be host memory"
                                                   : "U and V must be device memory of the handle's GPU");
    // a solve starts with no tensor-core wait recorded: one left over from earlier products
    // (gkl_rmatvec without gkl_sync) is reported here instead of inside this solve
    if (int pend = take_pending_error(h)) return pend;
    h->last_valid = 0;
    if (o->precision == GKL_FP64)
        return run_svd<double>(h, o, sigma, (double*)U, (double*)V, resid, info);
    if (o->precision == GKL_FP32) return run_svd<float>(h, o, sigma, (float*)U, (float*)V, resid, info);
    if (o->precision == GKL_BLOCK || o->precision == GKL_BLOCK16)
        return run_block(h, o, sigma, (float*)U, (float*)V, resid, info);
    return set_err(h, GKL_ERR_ARG, "unknown precision %d", o->precision);
}

int gkl_scores(gkl_handle* h, void* S, int32_t out_host) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    if (!h->last_valid || !h->last_U)
        return set_err(h, GKL_ERR_STATE, "gkl_scores needs a successful gkl_svd with the current weights");
    if (!S || mem_kind(S, h->device) != (out_host ? MEM_HOST : MEM_DEVICE))
        return set_err(h, GKL_ERR_ARG, out_host ? "S must be host memory (out_host set)"
                                                : "S must be device memory of the handle's GPU");
    const int k = h->last_k;
    const size_t esz = h->last_prec == GKL_FP64 ? sizeof(double) : sizeof(float);
    const size_t bytes = esz * (size_t)h->n * k;
    void* dst = S;
    if (out_host) {
        int st = ensure_scratch(h, bytes);
        if (st) return st;
        dst = h->scratch;
    }
    double* dsig = reinterpret_cast<double*>(reinterpret_cast<char*>(h->aux) + kAuxSigmaOffset);
    cudaError_t e = cudaMemcpyAsync(dsig, h->last_sigma, sizeof(double) * k, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_scores(h->stream, h->last_prec, h->last_U, dsig, h->n, k, dst);
    if (e == cudaSuccess && out_host) e = cudaMemcpyAsync(S, dst, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // dsig is read from pageable host memory
    return e == cudaSuccess ? GKL_OK : cuda_err(h, e, "scores");
}

int gkl_sync(gkl_handle* h) {
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    return take_pending_error(h);
}

int gkl_destroy(gkl_handle* h) {
    if (!h) return GKL_OK;
    if (h->mu) cudaFree(h->mu);
    if (h->d) cudaFree(h->d);
    if (h->s) cudaFree(h->s);
    if (h->w) cudaFree(h->w);
    if (h->scratch) cudaFree(h->scratch);
    if (h->ws) cudaFree(h->ws);
    if (h->host_out) cudaFreeHost(h->host_out);
    if (h->aux) cudaFree(h->aux);
    if (h->miss_off) cudaFree(h->miss_off);
    if (h->miss_idx) cudaFree(h->miss_idx);
    if (h->last_U) cudaFree(h->last_U);
    if (h->gws) cudaFree(h->gws);
    delete h;
    return GKL_OK;
}

}  // extern "C"
