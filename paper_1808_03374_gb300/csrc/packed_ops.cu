// Products with the packed, standardised genotype matrix
//     A_ij = s_i (g_ij - mu_j) d_j w_j   (g_ij observed), 0 if missing,
// read straight from the 2-bit SNP-major buffer (no unpacked or transposed
// copy).  The products y = A v and x = A^T u are the per-iteration cost of
// Golub-Kahan-Lanczos bidiagonalisation (section 3 of arXiv:1808.03374);
// mean imputation of missing codes follows from centring (section 5 names
// imputation as future work; this is its simplest form).
//
// Both products are split over (sample tile) x (SNP chunk) blocks whose
// partial sums are combined in a fixed order by a second kernel, so results
// are deterministic.
#include <algorithm>

#include "epilogue.cuh"
#include "gkl_internal.cuh"

namespace gkl {

namespace {
constexpr int kThreads = 256;   // threads per block of the product kernels
constexpr int kRowBatch = 32;   // SNP rows staged per batch
}

// ------------------------------------------------------------------ stats

// One warp per SNP row.  Bit planes lo = bit 0, hi = bit 1 of each code give
// the code counts with popcounts: code 1 = lo&~hi, code 2 = hi&~lo, code 3 = lo&hi.
__global__ void k_colstats(const uint8_t* __restrict__ packed, int64_t n, int64_t m, int64_t stride,
                           double* __restrict__ mu, double* __restrict__ scale, int64_t* __restrict__ nobs_out) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= m) return;
    const uint32_t* r = reinterpret_cast<const uint32_t*>(packed + row * stride);
    const int64_t nw = stride / 4;
    long long c1 = 0, c2 = 0, c3 = 0;
    for (int64_t t = lane; t < nw; t += 32) {
        uint32_t w = __ldg(r + t);
        uint32_t lo = w & 0x55555555u, hi = (w >> 1) & 0x55555555u;
        c1 += __popc(lo & ~hi);
        c2 += __popc(hi & ~lo);
        c3 += __popc(lo & hi);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        c2 += __shfl_xor_sync(0xffffffffu, c2, o);
        c3 += __shfl_xor_sync(0xffffffffu, c3, o);
    }
    if (lane != 0) return;
    const long long pad = stride * 4 - n;  // padding entries hold code 3
    const long long nob = n - (c3 - pad);
    const long long s1 = c1 + 2 * c2, s2 = c1 + 4 * c2;
    double mj = 0.0, dj = 0.0;
    if (nob > 0) {
        mj = (double)s1 / (double)nob;
        double num = (double)(nob * s2 - s1 * s1);
        double var = num / ((double)nob * (double)nob);
        double sd = sqrt(var);
        dj = sd > 0.0 ? 1.0 / sd : 0.0;
    }
    if (mu) mu[row] = mj;
    if (scale) scale[row] = dj;
    if (nobs_out) nobs_out[row] = nob;
}

cudaError_t launch_colstats(const uint8_t* packed, int64_t n, int64_t m, int64_t stride, double* mu, double* scale,
                            int64_t* nobs, cudaStream_t st) {
    int64_t threads = m * 32;
    unsigned blocks = (unsigned)((threads + 255) / 256);
    k_colstats<<<blocks, 256, 0, st>>>(packed, n, m, stride, mu, scale, nobs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ plan

MvPlan plan_products(const gkl_handle* h) {
    MvPlan p;
    p.nwords = (h->n + 15) / 16;
    p.tiles = (int)((p.nwords + kThreads - 1) / kThreads);
    const int target = 4 * std::max(1, h->num_sms);
    int chunks = std::max(1, target / p.tiles);
    int64_t rpc = (h->m + chunks - 1) / chunks;
    rpc = std::max<int64_t>(rpc, 64);
    rpc = (rpc + kRowBatch - 1) / kRowBatch * kRowBatch;
    p.rows_per_chunk = (int)rpc;
    p.chunks = (int)((h->m + rpc - 1) / rpc);
    p.ldp = p.nwords * 16;
    size_t mv = (size_t)p.chunks * (size_t)p.ldp + (size_t)h->m * 4;  // partials + LUT
    size_t rmv = 2 * (size_t)p.tiles * (size_t)h->m;
    size_t tc = h->aux ? rmv_mma_scratch_bytes(h) : 0;
    if (h->tc_state > 0) tc = std::max(tc, rmv_tc_scratch_bytes(h));
    p.bytes_fp64 = std::max(std::max(mv, rmv) * sizeof(double) + 256, tc);
    return p;
}

// ------------------------------------------------------------------ A v

// Per-SNP table t_j[c] = (c - mu_j) * d_j * w_j * v_j for c = 0,1,2; t_j[3] = 0
// (missing entries contribute nothing: mean imputation).
template <typename T>
__global__ void k_mv_table(int64_t m, const double* __restrict__ mu, const double* __restrict__ d,
                           const float* __restrict__ w, const T* __restrict__ v, T* __restrict__ lut) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double cw = d[j];
    if (w) cw *= (double)w[j];
    double coef = cw * (double)v[j];
    double mj = mu[j];
    lut[4 * j + 0] = (T)((0.0 - mj) * coef);
    lut[4 * j + 1] = (T)((1.0 - mj) * coef);
    lut[4 * j + 2] = (T)((2.0 - mj) * coef);
    lut[4 * j + 3] = (T)0;
}

// Partial sums over one SNP chunk: each thread owns one 32-bit word of
// every row (16 consecutive samples) and accumulates t_j[code] over the rows
// of its chunk.  Rows are read with coalesced 32-bit loads.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mv_part(const uint8_t* __restrict__ packed, int64_t stride,
                                                      int64_t nwords, int64_t m, int rpc, const T* __restrict__ lut,
                                                      T* __restrict__ part, int64_t ldp) {
    __shared__ T slut[kRowBatch * 4];
    const int64_t word = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * rpc;
    const int64_t j1 = min(m, j0 + (int64_t)rpc);
    const bool active = word < nwords;
    const int64_t wstride = stride >> 2;
    const uint32_t* base = reinterpret_cast<const uint32_t*>(packed) + (active ? word : 0);
    T acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = (T)0;
    for (int64_t jb = j0; jb < j1; jb += kRowBatch) {
        const int nr = (int)min((int64_t)kRowBatch, j1 - jb);
        __syncthreads();
        for (int t = threadIdx.x; t < nr * 4; t += kThreads) slut[t] = lut[jb * 4 + t];
        __syncthreads();
        if (!active) continue;
        for (int r = 0; r < nr; r += 8) {
            uint32_t wv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) wv[q] = (r + q < nr) ? __ldg(base + (jb + r + q) * wstride) : 0xFFFFFFFFu;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const T* L = slut + (r + q < nr ? (r + q) : 0) * 4;
                const uint32_t wq = wv[q];
                if (r + q < nr) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) acc[k] += L[(wq >> (2 * k)) & 3u];
                }
            }
        }
    }
    if (!active) return;
    T* out = part + (int64_t)blockIdx.y * ldp + word * 16;
#pragma unroll
    for (int k = 0; k < 16; ++k) out[k] = acc[k];
}

// FP32 A v partial sums with SNP-pair tables: for rows (a, b) the 16-entry
// table T[c_a + 4 c_b] = t_a[c_a] + t_b[c_b] turns two codes of one sample
// into one shared-memory lookup.  The nibble k of
//     E = (W_a & 0x33..) | ((W_b & 0x33..) << 2)   is c_a + 4 c_b of sample 2k,
//     O = ((W_a >> 2) & 0x33..) | (W_b & 0xCC..)    is c_a + 4 c_b of sample 2k+1.
// All lanes of a warp read the same 16-entry table, which spans 16 banks, so
// every lookup is a single conflict-free shared-memory wavefront.
constexpr int kPairBatch = 64;  // row pairs staged per batch (128 rows)

__global__ void __launch_bounds__(kThreads) k_mv_pair(const uint8_t* __restrict__ packed, int64_t stride,
                                                      int64_t nwords, int64_t m, int rpc,
                                                      const float* __restrict__ lut, float* __restrict__ part,
                                                      int64_t ldp) {
    __shared__ float tab[kPairBatch * 16];
    __shared__ __align__(16) float lrow[2 * kPairBatch * 4];
    static_assert(2 * kPairBatch * 4 == 2 * kThreads, "one float2 of per-SNP table rows per thread");
    const int64_t word = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * rpc;
    const int64_t j1 = min(m, j0 + (int64_t)rpc);
    const bool active = word < nwords;
    const int64_t wstride = stride >> 2;
    const uint32_t* base = reinterpret_cast<const uint32_t*>(packed) + (active ? word : 0);
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.f;
    // per-SNP table rows of a batch: thread t holds floats 2t, 2t+1 (row t/2)
    auto fetch_rows = [&](int64_t jb, int nrows) -> float2 {
        const int r = threadIdx.x >> 1;
        return r < nrows ? *reinterpret_cast<const float2*>(lut + jb * 4 + 2 * threadIdx.x) : make_float2(0.f, 0.f);
    };
    auto load_group = [&](int64_t jb, int nrows, int p0, uint32_t (&xa)[4], uint32_t (&xb)[4]) {
        const uint32_t* rp = base + (jb + 2 * p0) * wstride;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ra = 2 * (p0 + q), rb = ra + 1;
            xa[q] = (ra < nrows) ? __ldg(rp + (2 * q) * wstride) : 0xFFFFFFFFu;
            xb[q] = (rb < nrows) ? __ldg(rp + (2 * q + 1) * wstride) : 0xFFFFFFFFu;
        }
    };
    // The next batch's table rows and first group of code words are fetched
    // before the current batch is consumed, so the barriers that rebuild the
    // pair tables do not drain the memory pipeline.
    uint32_t wa[4], wb[4], na[4], nb[4];
    int64_t jb = j0;
    int nrows = (int)min((int64_t)(2 * kPairBatch), j1 - jb);
    float2 lcur = fetch_rows(jb, nrows);
    if (active && nrows > 0) load_group(jb, nrows, 0, wa, wb);
    while (jb < j1) {
        const int npairs = (nrows + 1) >> 1;
        __syncthreads();
        *reinterpret_cast<float2*>(lrow + 2 * threadIdx.x) = lcur;
        __syncthreads();
        for (int e = threadIdx.x; e < npairs * 16; e += kThreads) {
            const int p = e >> 4, ca = e & 3, cb = (e >> 2) & 3;
            const int ra = 2 * p, rb = 2 * p + 1;
            tab[e] = lrow[ra * 4 + ca] + (rb < nrows ? lrow[rb * 4 + cb] : 0.f);
        }
        __syncthreads();
        const int64_t jn = jb + 2 * kPairBatch;
        const int nrn = jn < j1 ? (int)min((int64_t)(2 * kPairBatch), j1 - jn) : 0;
        if (nrn > 0) lcur = fetch_rows(jn, nrn);
        if (active) {
            for (int p0 = 0; p0 < npairs; p0 += 4) {
                if (p0 + 4 < npairs) load_group(jb, nrows, p0 + 4, na, nb);
                else if (nrn > 0) load_group(jn, nrn, 0, na, nb);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (p0 + q >= npairs) break;
                    const char* T = reinterpret_cast<const char*>(tab + (p0 + q) * 16);
                    const uint32_t e = (wa[q] & 0x33333333u) | ((wb[q] & 0x33333333u) << 2);
                    const uint32_t o = ((wa[q] >> 2) & 0x33333333u) | (wb[q] & 0xCCCCCCCCu);
                    // byte offsets 4 * index: bytes of eL hold nibbles 0, 2, 4, 6 of e (samples
                    // 0, 4, 8, 12), bytes of eH nibbles 1, 3, 5, 7 (samples 2, 6, 10, 14); likewise
                    // for o (odd samples).  One byte-permute then yields each offset.
                    const uint32_t eL = (e << 2) & 0x3C3C3C3Cu, eH = (e >> 2) & 0x3C3C3C3Cu;
                    const uint32_t oL = (o << 2) & 0x3C3C3C3Cu, oH = (o >> 2) & 0x3C3C3C3Cu;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t sel = 0x4440u | (uint32_t)b;
                        acc[4 * b] += *reinterpret_cast<const float*>(T + __byte_perm(eL, 0u, sel));
                        acc[4 * b + 1] += *reinterpret_cast<const float*>(T + __byte_perm(oL, 0u, sel));
                        acc[4 * b + 2] += *reinterpret_cast<const float*>(T + __byte_perm(eH, 0u, sel));
                        acc[4 * b + 3] += *reinterpret_cast<const float*>(T + __byte_perm(oH, 0u, sel));
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    wa[q] = na[q];
                    wb[q] = nb[q];
                }
            }
        }
        jb = jn;
        nrows = nrn;
    }
    if (!active) return;
    float4* out = reinterpret_cast<float4*>(part + (int64_t)blockIdx.y * ldp + word * 16);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
}

__device__ inline double block_sum_to(double v, double* partials_slot) {
    __shared__ double s_red[32];
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) s_red[w] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int q = 0; q < nw; ++q) tot += s_red[q];
        *partials_slot = tot;
    }
    return tot;
}

// Runs in the last block: combine the per-block partial norms (each thread
// sums a fixed strided subset in order, then a fixed tree) and hand the total
// to the solver's step logic.
__device__ inline void finish_norm(const Sv& sv, int role, int j) {
    __shared__ double s_w[32];
    __shared__ double s_tot;
    const int nb = gridDim.x * gridDim.y;
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) t += __ldcg(sv.partials + (int64_t)b * (GKL_MAX_ELL + 2));
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += s_w[q];
        s_tot = a;
    }
    __syncthreads();
    step_epilogue(sv, role, j, s_tot);
    __syncthreads();
    release_counter(&sv.sc->counter);
}

// Final reduction of A v over SNP chunks, sample weights, optional
// subtraction of earlier basis vectors, optional norm + step logic.  A block
// takes 32 outputs at a time; its eight warps sum every eighth chunk (coalesced
// over the outputs) and the eight partial sums are added in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_mv_fin(const T* __restrict__ part, int64_t ldp, int chunks, int64_t n,
                                                const float* __restrict__ s, T* __restrict__ y, FinArgs fa, Sv sv) {
    if (fa.role != ROLE_NONE && sv.sc->abort) return;
    __shared__ double sb[GKL_MAX_ELL];
    __shared__ int sidx[GKL_MAX_ELL];
    __shared__ int snz;
    __shared__ T red[8][33];
    if (threadIdx.x == 0) {
        int c = 0;
        for (int r = 0; r < fa.nsub; ++r) {
            double b = fa.bcol[r];
            if (b != 0.0) { sb[c] = b; sidx[c] = r; ++c; }
        }
        snz = c;
    }
    __syncthreads();
    const int li = threadIdx.x & 31, g = threadIdx.x >> 5;
    const T* W = static_cast<const T*>(fa.W);
    double sq = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * 32; i0 < n; i0 += (int64_t)gridDim.x * 32) {
        const int64_t i = i0 + li;
        T acc = (T)0;
        if (i < n)
            for (int c = g; c < chunks; c += 8) acc += part[(int64_t)c * ldp + i];
        red[g][li] = acc;
        __syncthreads();
        if (g == 0 && i < n) {
            T t = red[0][li];
#pragma unroll
            for (int q = 1; q < 8; ++q) t += red[q][li];
            if (s) t *= (T)s[i];
            for (int q = 0; q < snz; ++q) t -= (T)sb[q] * W[i + (int64_t)sidx[q] * fa.ldw];
            y[i] = t;
            sq += (double)t * (double)t;
        }
        __syncthreads();
    }
    if (fa.role == ROLE_NONE) return;
    block_sum_to(sq, sv.partials + (int64_t)blockIdx.x * (GKL_MAX_ELL + 2));
    if (arrive_last(&sv.sc->counter)) finish_norm(sv, fa.role, fa.j);
}

template <typename T>
cudaError_t launch_matvec(const gkl_handle* h, const T* v, T* y, void* scratch, const Sv* sv, const FinArgs* fa,
                          cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    MvPlan p = plan_products(h);
    T* part = static_cast<T*>(scratch);
    T* lut = part + (size_t)p.chunks * (size_t)p.ldp;
    cudaStream_t st = h->stream;
    k_mv_table<T><<<(unsigned)((h->m + 255) / 256), 256, 0, st>>>(h->m, h->mu, h->d, h->w, v, lut);
    dim3 grid((unsigned)p.tiles, (unsigned)p.chunks);
    if (ev0) cudaEventRecord(ev0, st);
    if constexpr (sizeof(T) == sizeof(float))
        k_mv_pair<<<grid, kThreads, 0, st>>>(h->packed, h->stride, p.nwords, h->m, p.rows_per_chunk,
                                             reinterpret_cast<const float*>(lut), reinterpret_cast<float*>(part),
                                             p.ldp);
    else
        k_mv_part<T><<<grid, kThreads, 0, st>>>(h->packed, h->stride, p.nwords, h->m, p.rows_per_chunk, lut, part,
                                                p.ldp);
    if (ev1) cudaEventRecord(ev1, st);
    if (nlaunch) *nlaunch = 3;
    FinArgs f{};
    Sv s{};
    if (fa) f = *fa;
    if (sv) s = *sv;
    // 32 outputs per block pass; at most 4 blocks per SM (the partial-norm buffer's size)
    const int fblocks = (int)std::min<int64_t>((h->n + 31) / 32, 4 * (int64_t)h->num_sms);
    k_mv_fin<T><<<(unsigned)std::max(1, fblocks), 256, 0, st>>>(part, p.ldp, p.chunks, h->n, h->s, y, f, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ A^T u

// Partial sums for x_j = d_j w_j [ sum_obs g_ij u~_i - mu_j sum_obs u~_i ],
// u~ = s o u.  Each thread holds u~ for its 16 samples in registers and
// streams the SNP rows of its chunk; the two sums are reduced across the
// warp by shuffles and across warps in shared memory.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rmv_part(const uint8_t* __restrict__ packed, int64_t stride, int64_t n,
                                                       int64_t nwords, int64_t m, int rpc, const T* __restrict__ u,
                                                       const float* __restrict__ s, T* __restrict__ p1,
                                                       T* __restrict__ p3) {
    __shared__ T red1[kThreads / 32][kRowBatch + 1];
    __shared__ T red3[kThreads / 32][kRowBatch + 1];
    const int64_t word = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = word < nwords;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T ut[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        int64_t i = word * 16 + k;
        T val = (T)0;
        if (active && i < n) val = s ? (T)s[i] * u[i] : u[i];
        ut[k] = val;
    }
    const int64_t j0 = (int64_t)blockIdx.y * rpc;
    const int64_t j1 = min(m, j0 + (int64_t)rpc);
    const int64_t wstride = stride >> 2;
    const uint32_t* base = reinterpret_cast<const uint32_t*>(packed) + (active ? word : 0);
    for (int64_t jb = j0; jb < j1; jb += kRowBatch) {
        const int nr = (int)min((int64_t)kRowBatch, j1 - jb);
        for (int r = 0; r < nr; ++r) {
            uint32_t wq = active ? __ldg(base + (jb + r) * wstride) : 0xFFFFFFFFu;
            T a1 = (T)0, a3 = (T)0;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                uint32_t c = (wq >> (2 * k)) & 3u;
                T hv = (c == 3u) ? (T)0 : (T)c;
                T ov = (c == 3u) ? (T)0 : (T)1;
                a1 += hv * ut[k];
                a3 += ov * ut[k];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a3 += __shfl_xor_sync(0xffffffffu, a3, o);
            }
            if (lane == 0) {
                red1[wid][r] = a1;
                red3[wid][r] = a3;
            }
        }
        __syncthreads();
        if (threadIdx.x < nr) {
            T t1 = (T)0, t3 = (T)0;
#pragma unroll
            for (int q = 0; q < kThreads / 32; ++q) {
                t1 += red1[q][threadIdx.x];
                t3 += red3[q][threadIdx.x];
            }
            p1[(int64_t)blockIdx.x * m + jb + threadIdx.x] = t1;
            p3[(int64_t)blockIdx.x * m + jb + threadIdx.x] = t3;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_rmv_fin(const T* __restrict__ p1, const T* __restrict__ p3, int tiles,
                                                      int64_t m, const double* __restrict__ mu,
                                                      const double* __restrict__ d, const float* __restrict__ w,
                                                      T* __restrict__ x, FinArgs fa, Sv sv) {
    if (fa.role != ROLE_NONE && sv.sc->abort) return;
    const int64_t j = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    double sq = 0.0;
    if (j < m) {
        T s1 = (T)0, s3 = (T)0;
        for (int t = 0; t < tiles; ++t) {
            s1 += p1[(int64_t)t * m + j];
            s3 += p3[(int64_t)t * m + j];
        }
        double dw = d[j];
        if (w) dw *= (double)w[j];
        T val = (T)(dw * ((double)s1 - mu[j] * (double)s3));
        const T* W = static_cast<const T*>(fa.W);
        for (int q = 0; q < fa.nsub; ++q) val -= (T)fa.bcol[q] * W[j + (int64_t)q * fa.ldw];
        x[j] = val;
        sq = (double)val * (double)val;
    }
    if (fa.role == ROLE_NONE) return;
    block_sum_to(sq, sv.partials + (int64_t)blockIdx.x * (GKL_MAX_ELL + 2));
    if (arrive_last(&sv.sc->counter)) finish_norm(sv, fa.role, fa.j);
}

template <typename T>
cudaError_t launch_rmatvec(const gkl_handle* h, const T* u, T* x, void* scratch, const Sv* sv, const FinArgs* fa,
                           cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    if constexpr (sizeof(T) == sizeof(float)) {
        if (h->aux && h->tc_state > 0)
            return launch_rmatvec_tc(h, reinterpret_cast<const float*>(u), reinterpret_cast<float*>(x), scratch, sv,
                                     fa, ev0, ev1, nlaunch);
        if (h->aux)
            return launch_rmatvec_mma(h, reinterpret_cast<const float*>(u), reinterpret_cast<float*>(x), scratch, sv,
                                      fa, ev0, ev1, nlaunch);
    }
    MvPlan p = plan_products(h);
    T* p1 = static_cast<T*>(scratch);
    T* p3 = p1 + (size_t)p.tiles * (size_t)h->m;
    cudaStream_t st = h->stream;
    dim3 grid((unsigned)p.tiles, (unsigned)p.chunks);
    if (ev0) cudaEventRecord(ev0, st);
    k_rmv_part<T><<<grid, kThreads, 0, st>>>(h->packed, h->stride, h->n, p.nwords, h->m, p.rows_per_chunk, u, h->s, p1,
                                             p3);
    if (ev1) cudaEventRecord(ev1, st);
    if (nlaunch) *nlaunch = 2;
    FinArgs f{};
    Sv s{};
    if (fa) f = *fa;
    if (sv) s = *sv;
    k_rmv_fin<T><<<(unsigned)((h->m + kThreads - 1) / kThreads), kThreads, 0, st>>>(p1, p3, p.tiles, h->m, h->mu, h->d,
                                                                                    h->w, x, f, s);
    return cudaGetLastError();
}

template cudaError_t launch_matvec<float>(const gkl_handle*, const float*, float*, void*, const Sv*, const FinArgs*,
                                          cudaEvent_t, cudaEvent_t, int*);
template cudaError_t launch_matvec<double>(const gkl_handle*, const double*, double*, void*, const Sv*, const FinArgs*,
                                           cudaEvent_t, cudaEvent_t, int*);
template cudaError_t launch_rmatvec<float>(const gkl_handle*, const float*, float*, void*, const Sv*, const FinArgs*,
                                           cudaEvent_t, cudaEvent_t, int*);
template cudaError_t launch_rmatvec<double>(const gkl_handle*, const double*, double*, void*, const Sv*,
                                            const FinArgs*, cudaEvent_t, cudaEvent_t, int*);

}  // namespace gkl
