// Tensor-core A^T u for the FP32 path:
//     x_j = d_j w_j [ sum_{i obs} g_ij u~_i - mu_j sum_{i obs} u~_i ],  u~ = s o u
// (A as defined in gkl.h; the per-iteration product of GKL bidiagonalisation,
// section 3 of arXiv:1808.03374).
//
// The packed codes are exact small integers, so the contraction over samples
// runs on the tensor cores as an exact integer computation:
//  * u~ is written in fixed point: u~_i = S * sum_{p<7} delta_{p,i} 16^-(p+1)
//    + r_i with S = 2^e >= max|u~|, digits delta in [-16, 16] (exact in f16)
//    and |r_i| <= 2^-29 S -- finer than FP32 rounding of the inputs;
//  * codes become f16 pairs with one byte-permute: the selector
//    ((W << s) & 0x30303030) | 0x40404040 puts codes k and k+4 of a 32-bit code
//    word W into selector nibbles 1 and 3 (nibbles 0 and 2 pick a zero byte),
//    so prmt(0, table, selector) is the f16 pair (value(c_k), value(c_k+4)) with
//    the tables H(c) = c for observed codes (0 for missing) and M(c) = [c == 3];
//  * mma.sync m16n8k16 (A = 16 SNP rows x 16 samples, B = 16 samples x 8 digit
//    columns) accumulates sum_i H_ji delta_{p,i} and sum_i M_ji delta_{p,i} in
//    FP32, exactly (integers below 2^24);
//  * sum_{i obs} u~_i = sum_i u~_i - sum_{i missing} u~_i, with sum_i u~_i in FP64.
// The digit fragments are stored in the sample order that the selectors
// produce, so no data is transposed.
#include <cuda_fp16.h>

#include <algorithm>

#include "epilogue.cuh"
#include "gkl_internal.cuh"

namespace gkl {

namespace {
constexpr int kDigits = 7;               // base-16 digits of u~ (28 bits)
constexpr int kThreads = 256;            // 8 warps
constexpr int kStepSamples = 256;        // samples per warp step (64 bytes per row)
constexpr int kStepFragBytes = 4096;     // 16 MMAs x 32 lanes x 8 bytes
constexpr int kMaxStepsPerBlock = 16;    // 4096 samples, 64 KB of fragments per block
constexpr uint32_t kLutH = 0x00403C00u;  // high bytes of f16 H(c): 0, 1, 2, 0
constexpr uint32_t kLutM = 0x3C000000u;  // high bytes of f16 M(c): 0, 0, 0, 1
constexpr uint32_t kSelMask = 0x30303030u, kSelBase = 0x40404040u;
}  // namespace

struct RmvMmaPlan {
    int nb;             // sample blocks
    int steps_per_block;
    int steps;          // 256-sample steps in the row (ceil(stride/64))
    int row_groups;     // ceil(m / 16)
    int grid_y;
    size_t frag_bytes;  // digit fragments, all steps
    size_t part_bytes;  // FP64 partials: 2 * nb * m
};

static RmvMmaPlan plan_rmv_mma(const gkl_handle* h) {
    RmvMmaPlan p;
    p.steps = (int)((h->stride + 63) / 64);
    p.nb = std::max(1, (p.steps + kMaxStepsPerBlock - 1) / kMaxStepsPerBlock);
    p.steps_per_block = (p.steps + p.nb - 1) / p.nb;
    p.row_groups = (int)((h->m + 15) / 16);
    int want = std::max(1, 3 * h->num_sms / p.nb);
    p.grid_y = std::max(1, std::min(want, (p.row_groups + 7) / 8));
    p.frag_bytes = (size_t)p.steps * kStepFragBytes;
    p.part_bytes = 2 * (size_t)p.nb * (size_t)h->m * sizeof(double);
    return p;
}

size_t rmv_mma_scratch_bytes(const gkl_handle* h) {
    RmvMmaPlan p = plan_rmv_mma(h);
    return ((p.frag_bytes + 255) & ~(size_t)255) + p.part_bytes + 256;
}

// ---- digits of u~ ---------------------------------------------------------

// Pass 1: max|u~| and sum u~ (FP64), combined by the last block; the scale
// S = 2^e >= max|u~| and the sum go to dsc[0..2] = {S, 1/S, sum}.
__global__ void __launch_bounds__(256) k_u_scale(const float* __restrict__ u, const float* __restrict__ s, int64_t n,
                                                  double* __restrict__ part, unsigned* __restrict__ counter,
                                                  double* __restrict__ dsc) {
    double mx = 0.0, sm = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = (double)u[i] * (s ? (double)s[i] : 1.0);
        mx = fmax(mx, fabs(v));
        sm += v;
    }
    __shared__ double smx[32], ssm[32];
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) { smx[w] = mx; ssm[w] = sm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nw; ++q) { a = fmax(a, smx[q]); b += ssm[q]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
    if (!arrive_last(counter)) return;
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (unsigned q = 0; q < gridDim.x; ++q) {
            a = fmax(a, __ldcg(part + 2 * q));
            b += __ldcg(part + 2 * q + 1);
        }
        int e = 0;
        frexp(a, &e);                              // a = f * 2^e, f in [0.5, 1)
        double S = a > 0.0 ? ldexp(1.0, e) : 1.0;  // S >= a
        dsc[0] = S;
        dsc[1] = 1.0 / S;
        dsc[2] = b;
        *counter = 0u;
    }
}

// Pass 2: one thread per sample (padding samples get zero digits).  Sample
// r = 64 t + 16 w + k of a 256-sample step feeds lane t's code word w; code k
// sits in the pair (k_lo, k_lo + 4) with k_lo = k without its bit 2, i.e. in
// MMA u = 2 (k_lo >> 3) + ((k_lo >> 1) & 1) of that word, B register k_lo & 1,
// half (k >> 2) & 1; digit p is B column p, lane 4 p + t.
__global__ void __launch_bounds__(256) k_u_digits(const float* __restrict__ u, const float* __restrict__ s, int64_t n,
                                                   int64_t nsamp, const double* __restrict__ dsc,
                                                   uint8_t* __restrict__ frag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsamp) return;
    const int64_t step = i / kStepSamples;
    const int r = (int)(i % kStepSamples);
    const int t = r >> 6, w = (r >> 4) & 3, k = r & 15;
    const int klo = (k & 3) | (k & 8), hi = (k >> 2) & 1;
    const int uix = 2 * (klo >> 3) + ((klo >> 1) & 1), reg = klo & 1;
    uint8_t* base = frag + step * kStepFragBytes + (size_t)((w * 4 + uix) * 32 + t) * 8 + reg * 4 + hi * 2;
    double x = 0.0;
    if (i < n) x = (double)u[i] * (s ? (double)s[i] : 1.0) * dsc[1];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        int dig = 0;
        if (p < kDigits) {
            x *= 16.0;
            double rd = rint(x);
            x -= rd;
            dig = (int)rd;
        }
        *reinterpret_cast<unsigned short*>(base + (size_t)(4 * p) * 8) = __half_as_ushort(__int2half_rn(dig));
    }
}

// ---- main kernel ------------------------------------------------------------

__device__ __forceinline__ void mma_f16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                        uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pair(uint32_t lut, uint32_t sel) { return __byte_perm(0u, lut, sel); }

// Four selector words of a code word: codes (0,4 | 8,12), (1,5 | 9,13),
// (2,6 | 10,14), (3,7 | 11,15) in their low | high halves.
__device__ __forceinline__ void selectors(uint32_t W, uint32_t (&s)[4]) {
    s[0] = ((W << 4) & kSelMask) | kSelBase;
    s[1] = ((W << 2) & kSelMask) | kSelBase;
    s[2] = (W & kSelMask) | kSelBase;
    s[3] = ((W >> 2) & kSelMask) | kSelBase;
}

// Block (bx, by): sample block bx; warps stride over 16-row groups.
// Lane (g, t) owns SNP rows R+g and R+g+8 and, in each 256-sample step, the
// 16 bytes at offset 16*t of the step's 64-byte segment of those rows.
__global__ void __launch_bounds__(kThreads) k_rmv_mma(const uint8_t* __restrict__ packed, int64_t stride, int64_t m,
                                                      int steps, int steps_per_block, int row_groups,
                                                      const uint8_t* __restrict__ frag, double* __restrict__ p1,
                                                      double* __restrict__ p3, const double* __restrict__ dsc) {
    extern __shared__ __align__(16) unsigned char sfrag[];
    const int bx = blockIdx.x;
    const int st0 = bx * steps_per_block;
    const int nst = min(steps_per_block, steps - st0);
    {
        const uint4* src = reinterpret_cast<const uint4*>(frag + (size_t)st0 * kStepFragBytes);
        uint4* dst = reinterpret_cast<uint4*>(sfrag);
        const int nv = nst * kStepFragBytes / 16;
        for (int v = threadIdx.x; v < nv; v += blockDim.x) dst[v] = src[v];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const double S = dsc[0];
    const uint2* fr = reinterpret_cast<const uint2*>(sfrag) + lane;
    for (int rg = blockIdx.y * (kThreads / 32) + warp; rg < row_groups; rg += gridDim.y * (kThreads / 32)) {
        const int64_t r0 = (int64_t)rg * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < m, v1 = r1 < m;
        const uint8_t* row0 = packed + (v0 ? r0 : 0) * stride;
        const uint8_t* row1 = packed + (v1 ? r1 : 0) * stride;
        float aH[4] = {0.f, 0.f, 0.f, 0.f}, aM[4] = {0.f, 0.f, 0.f, 0.f};
        const uint4 ones = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);
        auto load = [&](int s, uint4& x0, uint4& x1) {
            const int64_t off = (int64_t)(st0 + s) * 64 + 16 * t;
            const bool in = off < stride;
            x0 = (v0 && in) ? __ldg(reinterpret_cast<const uint4*>(row0 + off)) : ones;
            x1 = (v1 && in) ? __ldg(reinterpret_cast<const uint4*>(row1 + off)) : ones;
        };
        uint4 c0, c1, n0, n1;
        load(0, c0, c1);
        for (int s = 0; s < nst; ++s) {
            if (s + 1 < nst) load(s + 1, n0, n1);
            const uint2* fs = fr + (size_t)s * (kStepFragBytes / 8);
            const uint32_t w0[4] = {c0.x, c0.y, c0.z, c0.w};
            const uint32_t w1[4] = {c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                uint32_t sa[4], sb[4];
                selectors(w0[w], sa);
                selectors(w1[w], sb);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // u = 0: codes (0,4),(1,5); 1: (2,6),(3,7); 2: (8,12),(9,13); 3: (10,14),(11,15)
                    const int lo = (u & 1) * 2, sh = (u >> 1) * 16;
                    const uint32_t ga = sa[lo] >> sh, gb = sa[lo + 1] >> sh;
                    const uint32_t ha = sb[lo] >> sh, hb = sb[lo + 1] >> sh;
                    const uint2 b = fs[(w * 4 + u) * 32];
                    mma_f16(aH, pair(kLutH, ga), pair(kLutH, ha), pair(kLutH, gb), pair(kLutH, hb), b.x, b.y);
                    mma_f16(aM, pair(kLutM, ga), pair(kLutM, ha), pair(kLutM, gb), pair(kLutM, hb), b.x, b.y);
                }
            }
            c0 = n0;
            c1 = n1;
        }
        // combine the digit columns 2t, 2t+1 across the quad: value = S sum_p D_p 16^-(p+1)
        const double f0 = ldexp(1.0, -4 * (2 * t + 1)), f1 = ldexp(1.0, -4 * (2 * t + 2));
        double h0 = (double)aH[0] * f0 + (double)aH[1] * f1, h1 = (double)aH[2] * f0 + (double)aH[3] * f1;
        double m0 = (double)aM[0] * f0 + (double)aM[1] * f1, m1 = (double)aM[2] * f0 + (double)aM[3] * f1;
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            h0 += __shfl_xor_sync(0xffffffffu, h0, o);
            h1 += __shfl_xor_sync(0xffffffffu, h1, o);
            m0 += __shfl_xor_sync(0xffffffffu, m0, o);
            m1 += __shfl_xor_sync(0xffffffffu, m1, o);
        }
        if (t == 0) {
            if (v0) {
                p1[(int64_t)bx * m + r0] = S * h0;
                p3[(int64_t)bx * m + r0] = S * m0;
            }
            if (v1) {
                p1[(int64_t)bx * m + r1] = S * h1;
                p3[(int64_t)bx * m + r1] = S * m1;
            }
        }
    }
}

// Final combination over sample blocks (fixed order), then the solver epilogue.
__global__ void __launch_bounds__(256) k_rmv_mma_fin(const double* __restrict__ p1, const double* __restrict__ p3,
                                                     int nb, int64_t m, const double* __restrict__ mu,
                                                     const double* __restrict__ d, const float* __restrict__ w,
                                                     const double* __restrict__ dsc, float* __restrict__ x, FinArgs fa,
                                                     Sv sv) {
    if (fa.role != ROLE_NONE && sv.sc->abort) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (j < m) {
        double hsum = 0.0, msum = 0.0;
        for (int b = 0; b < nb; ++b) {
            hsum += p1[(int64_t)b * m + j];
            msum += p3[(int64_t)b * m + j];
        }
        double dw = d[j];
        if (w) dw *= (double)w[j];
        const double obs = dsc[2] - msum;  // sum of u~ over observed samples
        float val = (float)(dw * (hsum - mu[j] * obs));
        const float* W = static_cast<const float*>(fa.W);
        for (int q = 0; q < fa.nsub; ++q) val -= (float)fa.bcol[q] * W[j + (int64_t)q * fa.ldw];
        x[j] = val;
        sq = (double)val * (double)val;
    }
    if (fa.role == ROLE_NONE) return;
    __shared__ double s_w[32];
    double v = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += s_w[q];
        sv.partials[(int64_t)blockIdx.x * (GKL_MAX_ELL + 2)] = a;
    }
    if (!arrive_last(&sv.sc->counter)) return;
    __shared__ double s_tot;
    double tt = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        tt += __ldcg(sv.partials + (int64_t)b * (GKL_MAX_ELL + 2));
    tt = warp_sum(tt);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = tt;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += s_w[q];
        s_tot = a;
    }
    __syncthreads();
    step_epilogue(sv, fa.role, fa.j, s_tot);
    __syncthreads();
    release_counter(&sv.sc->counter);
}

cudaError_t launch_rmatvec_mma(const gkl_handle* h, const float* u, float* x, void* scratch, const Sv* sv,
                               const FinArgs* fa, cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    const RmvMmaPlan p = plan_rmv_mma(h);
    uint8_t* frag = static_cast<uint8_t*>(scratch);
    double* p1 = reinterpret_cast<double*>(static_cast<char*>(scratch) + ((p.frag_bytes + 255) & ~(size_t)255));
    double* p3 = p1 + (size_t)p.nb * h->m;
    double* aux = h->aux;  // dsc[4] | counter | partials (zero-initialised at gkl_init)
    double* dsc = aux;
    unsigned* counter = reinterpret_cast<unsigned*>(aux + 4);
    double* part = aux + 8;
    cudaStream_t st = h->stream;
    const int sblocks = std::min(2 * h->num_sms, (int)((h->n + 255) / 256));
    k_u_scale<<<std::max(1, sblocks), 256, 0, st>>>(u, h->s, h->n, part, counter, dsc);
    const int64_t nsamp = (int64_t)p.steps * kStepSamples;
    k_u_digits<<<(unsigned)((nsamp + 255) / 256), 256, 0, st>>>(u, h->s, h->n, nsamp, dsc, frag);
    const size_t smem = (size_t)p.steps_per_block * kStepFragBytes;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_rmv_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxStepsPerBlock * kStepFragBytes);
        attr = true;
    }
    dim3 grid((unsigned)p.nb, (unsigned)p.grid_y);
    if (ev0) cudaEventRecord(ev0, st);
    k_rmv_mma<<<grid, kThreads, smem, st>>>(h->packed, h->stride, h->m, p.steps, p.steps_per_block, p.row_groups,
                                            frag, p1, p3, dsc);
    if (ev1) cudaEventRecord(ev1, st);
    FinArgs f{};
    Sv s{};
    if (fa) f = *fa;
    if (sv) s = *sv;
    k_rmv_mma_fin<<<(unsigned)((h->m + 255) / 256), 256, 0, st>>>(p1, p3, p.nb, h->m, h->mu, h->d, h->w, dsc, x, f, s);
    if (nlaunch) *nlaunch = 4;
    return cudaGetLastError();
}

}  // namespace gkl
