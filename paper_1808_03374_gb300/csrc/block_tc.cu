// Tensor-core block products for the block form of GKL bidiagonalisation
// (Golub-Luk-Overton block Lanczos, named as future work in section 5 of
// arXiv:1808.03374): X = A^T U and Y = A V for blocks of q <= 32 vectors, on
// the 5th-generation tensor cores (tcgen05, kind::f8f6f4, e4m3 operands, FP32
// accumulation in tensor memory).
//
// Fixed point.  Each vector of the block is written with D base-16 digits
// relative to a power-of-two scale S_c >= its largest entry,
//     x'_c = S_c sum_{p<D} delta_p 16^-(p+1),  delta_0 in [-16, 16], delta_p in [-8, 8],
// so |x - x'| <= 2^-(4D+1) S_c (D = 4: the 16 bits of a split hi+lo BF16 pair;
// D = 8: finer than FP32).  The q x D digit rows form the M = 128 side of the
// MMA; every product and partial sum is an integer below 2^24, so the FP32
// accumulators are exact and the digits are recombined in 64-bit integers.
//
// Genotype operand.  N = 256: 128 SNPs (or 256 samples) x two code functions
// decoded from the packed 2-bit codes by byte permutes,
//     f1(code) = g [observed] = 0, 1, 2, 0   and   f2(code) = [observed] = 1, 1, 1, 0,
// so that missing codes and the centring need no separate pass:
//   A^T U:  x_jc = d_j w_j S_c 2^-4D (sum_p 16^(D-1-p) (F1_p - mu_j F2_p))   (F_p = sum_i f(c_ij) delta_p,i)
//   A V:    y_ic = s_i S_c 2^-4D sum_p 16^(D-1-p) sum_j (f1(c_ij) delta1_p,j + f2(c_ij) delta2_p,j)
// with delta1 the digits of d_j w_j V_jc and delta2 those of -mu_j d_j w_j V_jc
// (one scale per vector covers both).
//
// Orientation ("transposed"): the digit rows are the A operand (M) and the
// decoded genotypes the B operand (N = 256), the shape at which one tcgen05.mma
// runs at full rate.  A^T U: K = samples, B K-major (the packed layout).  A V:
// K = SNPs, B MN-major (samples contiguous along N).  The sample order along
// each 16-sample group is the order the byte permutes produce (even samples,
// then odd); the digit tiles of A^T U are written in that order, and the
// epilogue of A V maps accumulator columns back to samples.
//
// Data movement: per 512-sample x 128-SNP stage one TMA box (128-byte swizzle)
// of packed codes; digit tiles by bulk copies from a buffer prepared per call in
// the shared-memory image of the operand; decoded genotypes written to shared
// memory by eight decode warps.  Warp roles: copy producer, MMA issuer, eight
// decode warps, four epilogue warps; one persistent CTA per SM.  Every wait is
// bounded; a wait that runs out sets the error word the host reads.
#include <cuda.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>

#include "gkl_internal.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"

namespace gkl {

namespace {
constexpr int kRowsT = 128;          // SNP rows per TMA box
constexpr int kStageS = 512;         // samples per TMA stage (128 bytes per row)
constexpr int kBoxBytes = 16384;     // one TMA box
constexpr int kTileBytes = 16384;    // one digit tile: 128 rows x 128 bytes
constexpr int kDecWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreadsBT = 32 * (2 + kDecWarps + kEpiWarps);  // 448
constexpr int kDec0 = 2, kEpi0 = kDec0 + kDecWarps;
constexpr uint32_t kLut1 = 0x00403800u;  // e4m3 bytes of f1: 0, 1, 2, 0
constexpr uint32_t kLut2 = 0x00383838u;  // e4m3 bytes of f2: 1, 1, 1, 0
// A^T U: rings of packed boxes (3), digit tiles (4, one per 128-sample sub-stage)
// and decoded tiles (2, 32 KB: 256 rows x 128 bytes)
constexpr int kRP = 3, kRG = 4, kRD = 2;
constexpr int kRmvTail = 4096;  // barriers, tensor-memory slot, per-tile mu and d w
constexpr int kRmvSmem = 1024 + kRP * kBoxBytes + kRG * kTileBytes + kRD * 2 * kTileBytes + kRmvTail;
// A V: rings of packed boxes (2), digit pairs (2 x 32 KB per 128-SNP stage) and
// decoded K-steps (4 x 32 KB: 2 functions x 2 halves x 8 KB)
constexpr int kVP = 2, kVG = 2, kVD = 4;
constexpr int kMvSmem = 1024 + kVP * kBoxBytes + kVG * 2 * kTileBytes + kVD * 2 * kTileBytes + 1024;
constexpr int kMaxSamplesRmv = 524000;  // |F1_p| <= 32 n < 2^24
constexpr int64_t kMaxSnpsChunk = 349000;  // |sum| <= 48 J < 2^24
}  // namespace

using tc::bar_arrive;
using tc::bar_expect_tx;
using tc::bar_init;
using tc::bar_wait;
using tc::desc_sw128;
using tc::mma_commit;
using tc::sm_addr;

// Four e4m3 bytes per function for the 16 codes of word W, in K order.
__device__ __forceinline__ void bt_decode(uint32_t W, uint4& o1, uint4& o2) {
    const uint32_t s0 = W & 0x33333333u, s1 = (W >> 2) & 0x33333333u;
    const uint32_t s0h = s0 >> 16, s1h = s1 >> 16;
    o1 = make_uint4(__byte_perm(kLut1, 0, s0), __byte_perm(kLut1, 0, s0h), __byte_perm(kLut1, 0, s1),
                    __byte_perm(kLut1, 0, s1h));
    o2 = make_uint4(__byte_perm(kLut2, 0, s0), __byte_perm(kLut2, 0, s0h), __byte_perm(kLut2, 0, s1),
                    __byte_perm(kLut2, 0, s1h));
}

// ---- per-call preparation ----------------------------------------------------

// Entries of the block in FP32: s_i U_ic (side 0); d_j w_j V_jc and -mu_j d_j w_j V_jc (side 1).
__device__ __forceinline__ float bt_xu(const float* U, int64_t ldu, int64_t i, int c, const float* s) {
    const float u = U[i + c * ldu];
    return s ? s[i] * u : u;
}
__device__ __forceinline__ float bt_xv(const float* V, int64_t ldv, int64_t j, int c, const double* d, const float* w) {
    const float dw = w ? (float)d[j] * w[j] : (float)d[j];
    return dw * V[j + c * ldv];
}
// Exponent e_c of the scale S_c = 2^e_c >= max |x| (from the FP32 bits of the max; 0 for 0).
__device__ __forceinline__ int bt_exp(int bits) {
    int e = 0;
    const float mx = __int_as_float(bits);
    if (mx > 0.f) frexpf(mx, &e);
    return e;
}

// mx[c] = bits of max |x| over rows (atomic max on the bits of non-negative floats: order-free).
__global__ void __launch_bounds__(256) k_bt_absmax(const float* __restrict__ X, int64_t ldx, int64_t len, int side,
                                                   const float* __restrict__ s, const double* __restrict__ mu,
                                                   const double* __restrict__ d, const float* __restrict__ w,
                                                   int* __restrict__ mx) {
    const int c = blockIdx.y;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        if (side == 0) {
            m = fmaxf(m, fabsf(bt_xu(X, ldx, i, c, s)));
        } else {
            const float v = bt_xv(X, ldx, i, c, d, w);
            m = fmaxf(m, fmaxf(fabsf(v), fabsf(-(float)mu[i] * v)));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
        m = fmaxf(m, red[0]);
        if (m > 0.f) atomicMax(mx + c, __float_as_int(m));
    }
}

// Balanced base-16 digits of x / S (|x| <= S = 2^e): X = rint(x 2^(4D - e)) is
// exact in FP32 (a power-of-two scaling and one rounding, |x - X 2^-4D S| <=
// 2^-(4D+1) S); digits D-1 .. 1 in [-8, 7] from the bottom, digit 0 = the rest,
// in [-16, 16].  All exact in e4m3.
__device__ __forceinline__ void bt_digits(float x, int sft, int D, int (&dg)[8]) {
    long long X = __float2ll_rn(ldexpf(x, sft));
    for (int p = D - 1; p >= 1; --p) {
        const int r = (int)((X + 8) & 15) - 8;
        dg[p] = r;
        X = (X - r) >> 4;
    }
    dg[0] = (int)X;
}
__device__ __forceinline__ uint8_t bt_e4m3(int v) {
    return (uint8_t)__nv_cvt_float_to_fp8((float)v, __NV_SATFINITE, __NV_E4M3);
}

// Digit tiles of s o U for A^T U: tile g (128 samples) row c D + p, K position
// 16 (loc / 16) + kpos(loc % 16).  The buffer is zeroed beforehand.
__global__ void __launch_bounds__(128) k_bt_digits_u(const float* __restrict__ U, int64_t ldu, int64_t n, int D,
                                                     const float* __restrict__ s, const int* __restrict__ mx,
                                                     uint8_t* __restrict__ dig) {
    const int g = blockIdx.x, c = blockIdx.y, loc = threadIdx.x;
    const int64_t i = (int64_t)g * 128 + loc;
    if (i >= n) return;
    int dg[8];
    bt_digits(bt_xu(U, ldu, i, c, s), 4 * D - bt_exp(mx[c]), D, dg);
    const int kk = 16 * (loc >> 4) + bt_kpos(loc & 15);
    uint8_t* tile = dig + (size_t)g * kTileBytes;
    for (int p = 0; p < D; ++p) tile[bt_swz(c * D + p, kk)] = bt_e4m3(dg[p]);
}

// Digit tile pairs for A V: stage t (128 SNPs) = [digits of d w V | digits of
// -mu d w V], row c D + p, K position = SNP within the stage.
__global__ void __launch_bounds__(128) k_bt_digits_v(const float* __restrict__ V, int64_t ldv, int64_t m, int D,
                                                     const double* __restrict__ mu, const double* __restrict__ d,
                                                     const float* __restrict__ w, const int* __restrict__ mx,
                                                     uint8_t* __restrict__ dig) {
    const int t = blockIdx.x, c = blockIdx.y, loc = threadIdx.x;
    const int64_t j = (int64_t)t * 128 + loc;
    if (j >= m) return;
    const int sft = 4 * D - bt_exp(mx[c]);
    const float v = bt_xv(V, ldv, j, c, d, w);
    int d1[8], d2[8];
    bt_digits(v, sft, D, d1);
    bt_digits(-(float)mu[j] * v, sft, D, d2);
    uint8_t* t1 = dig + (size_t)t * 2 * kTileBytes;
    for (int p = 0; p < D; ++p) {
        t1[bt_swz(c * D + p, loc)] = bt_e4m3(d1[p]);
        t1[kTileBytes + bt_swz(c * D + p, loc)] = bt_e4m3(d2[p]);
    }
}

// ---- X = A^T U ------------------------------------------------------------------

struct BtRmvArgs {
    const uint8_t* dig;   // nsub digit tiles
    const int* mx;        // q: bits of max |x| (scale exponents)
    const double* mu;
    const double* d;
    const float* w;
    float* X;
    int64_t ldx, m;
    int nstages, ntiles, q, D;
    int* err;
};

// Epilogue of A^T U: per tile, the digit rows' exact sums (two functions x 128
// SNPs) are scaled by 16^(D-1-p), reduce-scattered over each vector's D lanes
// (each lane then owns 16/D SNPs of every 16), and combined in FP64 with mu_j
// and d_j w_j staged in shared memory.  The four epilogue warps meet at named
// barrier 1 twice per tile; a warp whose wait ran out keeps meeting them (and
// skips its work) so that the others are never left waiting.
template <int D>
__device__ __forceinline__ void bt_rmv_epilogue(const BtRmvArgs& a, uint32_t tmem, uint32_t afull0, uint32_t aempty0,
                                                double* s_mu, double* s_dw, int warp, int lane) {
    constexpr int per = 16 / D;
    const int sub = warp & 3, r = 32 * sub + lane, et = threadIdx.x - 32 * kEpi0;
    const int c = r / D, p = r % D, sh = 4 * (D - 1 - p);
    const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
    const double Sc = c < a.q ? ldexp(1.0, bt_exp(a.mx[c]) - 4 * D) : 0.0;
    bool ok = true;
    uint32_t li = 0;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++li) {
        const uint32_t acc = li & 1u;
        {
            const int64_t j = (int64_t)tile * kRowsT + et;
            s_mu[et] = j < a.m ? a.mu[j] : 0.0;
            s_dw[et] = j < a.m ? a.d[j] * (a.w ? (double)a.w[j] : 1.0) : 0.0;
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        if (ok && !tc::bar_wait_warp(afull0 + 8u * acc, (li >> 1) & 1u)) {
            atomicCAS(a.err, 0, 20);
            ok = false;
        }
        if (ok) {
            tc::fence_after();
#pragma unroll 1
            for (int g = 0; g < 8; ++g) {
                long long z1[16], z2[16];
                bt_ld16_scaled(tmem + lane_base + 256u * acc + 16u * g, sh, z1);
                bt_ld16_scaled(tmem + lane_base + 256u * acc + 128u + 16u * g, sh, z2);
                if (g == 7) {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) bar_arrive(aempty0 + 8u * acc);
                }
                bt_reduce_scatter<D>(z1, p);
                bt_reduce_scatter<D>(z2, p);
#pragma unroll
                for (int i = 0; i < per; ++i) {
                    const int jj = 16 * g + per * p + i;
                    const int64_t j = (int64_t)tile * kRowsT + jj;
                    if (c < a.q && j < a.m)
                        a.X[j + c * a.ldx] = (float)(Sc * s_dw[jj] * ((double)z1[i] - s_mu[jj] * (double)z2[i]));
                }
            }
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
    }
}

__global__ void __launch_bounds__(kThreadsBT, 1) k_bt_rmv(const __grid_constant__ CUtensorMap tmap, BtRmvArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = sm_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sb = smem_raw + (base - raw);
    const uint32_t sP = base, sG = sP + kRP * kBoxBytes, sD = sG + kRG * kTileBytes;
    const uint32_t sBar = sD + kRD * 2 * kTileBytes;
    uint8_t* gP = sb;
    uint8_t* gD = sb + (kRP * kBoxBytes + kRG * kTileBytes);
    auto pfull = [&](int i) { return sBar + 8u * i; };
    auto pempty = [&](int i) { return sBar + 8u * (kRP + i); };
    auto gfull = [&](int i) { return sBar + 8u * (2 * kRP + i); };
    auto gempty = [&](int i) { return sBar + 8u * (2 * kRP + kRG + i); };
    auto dfull = [&](int i) { return sBar + 8u * (2 * kRP + 2 * kRG + i); };
    auto dempty = [&](int i) { return sBar + 8u * (2 * kRP + 2 * kRG + kRD + i); };
    auto afull = [&](int i) { return sBar + 8u * (2 * kRP + 2 * kRG + 2 * kRD + i); };
    auto aempty = [&](int i) { return sBar + 8u * (2 * kRP + 2 * kRG + 2 * kRD + 2 + i); };
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + (sBar - base) + 512);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tc::tmem_alloc(sm_addr(tmem_slot), 512);
    if (threadIdx.x == 32) {
        for (int i = 0; i < kRP; ++i) {
            bar_init(pfull(i), 1);
            bar_init(pempty(i), kDecWarps);
        }
        for (int i = 0; i < kRG; ++i) {
            bar_init(gfull(i), 1);
            bar_init(gempty(i), 1);
        }
        for (int i = 0; i < kRD; ++i) {
            bar_init(dfull(i), kDecWarps);
            bar_init(dempty(i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            bar_init(afull(i), 1);
            bar_init(aempty(i), kEpiWarps);
        }
        tc::bar_init_fence();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nsub = 4 * a.nstages;
    auto fail = [&](int code) { atomicCAS(a.err, 0, code); };

    if (warp == 0) {
        // ---- copies: per stage one packed box, then its four digit tiles
        if (lane == 0) {
            uint32_t ps = 0, gs = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
                for (int k = 0; k < a.nstages && ok; ++k, ++ps) {
                    const int sp = (int)(ps % kRP);
                    if (!bar_wait(pempty(sp), ((ps / kRP) & 1u) ^ 1u)) {
                        fail(11);
                        ok = false;
                        break;
                    }
                    bar_expect_tx(pfull(sp), kBoxBytes);
                    tc::tma_2d(sP + sp * kBoxBytes, &tmap, 128 * k, kRowsT * tile, pfull(sp));
                    for (int qq = 0; qq < 4; ++qq, ++gs) {
                        const int sg = (int)(gs % kRG);
                        if (!bar_wait(gempty(sg), ((gs / kRG) & 1u) ^ 1u)) {
                            fail(12);
                            ok = false;
                            break;
                        }
                        bar_expect_tx(gfull(sg), kTileBytes);
                        tc::bulk_g2s(sG + sg * kTileBytes, a.dig + (size_t)(4 * k + qq) * kTileBytes, kTileBytes,
                                     gfull(sg));
                    }
                }
            }
            // drain: every issued copy has landed before the CTA may exit
            for (uint32_t x = ps > (uint32_t)kRP ? ps - kRP : 0u; x < ps; ++x)
                if (!bar_wait(pfull((int)(x % kRP)), (x / kRP) & 1u)) fail(13);
            for (uint32_t x = gs > (uint32_t)kRG ? gs - kRG : 0u; x < gs; ++x)
                if (!bar_wait(gfull((int)(x % kRG)), (x / kRG) & 1u)) fail(14);
        }
    } else if (warp == 1) {
        // ---- MMA issuer: per 128-sample sub-stage four K-steps of 32 samples
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_e4m3(256, 0);
            uint32_t it = 0, li = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x, ++li) {
                const uint32_t acc = li & 1u;
                if (!bar_wait(aempty(acc), ((li >> 1) & 1u) ^ 1u)) {
                    fail(15);
                    break;
                }
                tc::fence_after();
                const uint32_t dcol = tmem + 256u * acc;
                for (int g = 0; g < nsub; ++g, ++it) {
                    const int sg = (int)(it % kRG), sd = (int)(it % kRD);
                    if (!bar_wait(gfull(sg), (it / kRG) & 1u) || !bar_wait(dfull(sd), (it / kRD) & 1u)) {
                        fail(16);
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint64_t ad = desc_sw128(sG + sg * kTileBytes);
                    const uint64_t bd = desc_sw128(sD + sd * 2 * kTileBytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        tc::mma_f8_ss(dcol, ad + 2 * ks, bd + 2 * ks, idesc, (g | ks) != 0);
                    mma_commit(gempty(sg));
                    mma_commit(dempty(sd));
                }
                if (ok) mma_commit(afull(acc));
            }
            if (it > 0) {  // the last commit covers every MMA issued
                const uint32_t x = it - 1;
                if (!bar_wait(dempty((int)(x % kRD)), (x / kRD) & 1u)) fail(17);
            }
        }
    } else if (warp < kEpi0) {
        // ---- decode: SNP row 32 (dw & 3) + lane, 64-sample half hh of each sub-stage
        const int dw = warp - kDec0, row = 32 * (dw & 3) + lane, hh = dw >> 2;
        uint32_t ps = 0, it = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < a.ntiles && ok; tile += gridDim.x) {
            for (int k = 0; k < a.nstages && ok; ++k, ++ps) {
                const int sp = (int)(ps % kRP);
                if (!tc::bar_wait_warp(pfull(sp), (ps / kRP) & 1u)) {
                    fail(18);
                    ok = false;
                    break;
                }
                for (int qq = 0; qq < 4; ++qq, ++it) {
                    const int sd = (int)(it % kRD);
                    const uint4 P = *reinterpret_cast<const uint4*>(gP + sp * kBoxBytes + row * 128 +
                                                                     ((((2 * qq + hh) ^ (row & 7))) << 4));
                    if (!tc::bar_wait_warp(dempty(sd), ((it / kRD) & 1u) ^ 1u)) {
                        fail(19);
                        ok = false;
                        break;
                    }
                    uint8_t* t1 = gD + sd * 2 * kTileBytes + (row >> 3) * 1024 + (row & 7) * 128;
                    const uint32_t Wv[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        uint4 o1, o2;
                        bt_decode(Wv[u], o1, o2);
                        const int ch = ((4 * hh + u) ^ (row & 7)) << 4;
                        *reinterpret_cast<uint4*>(t1 + ch) = o1;
                        *reinterpret_cast<uint4*>(t1 + kTileBytes + ch) = o2;
                    }
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) bar_arrive(dfull(sd));
                }
                __syncwarp();
                if (ok && lane == 0) bar_arrive(pempty(sp));
            }
        }
    } else {
        // ---- epilogue: lane = digit row c D + p of this warp's sub-partition
        double* s_mu = reinterpret_cast<double*>(sb + (sBar - base) + 1024);
        double* s_dw = s_mu + kRowsT;
        if (a.D == 8)
            bt_rmv_epilogue<8>(a, tmem, afull(0), aempty(0), s_mu, s_dw, warp, lane);
        else
            bt_rmv_epilogue<4>(a, tmem, afull(0), aempty(0), s_mu, s_dw, warp, lane);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

// ---- Y = A V: chunk partials -------------------------------------------------------

struct BtMvArgs {
    const uint8_t* dig;   // digit tile pairs, one per 128-SNP stage
    long long* Z;         // chunks x q x ldz partial sums (exact)
    int64_t ldz, n;
    int nblocks, nchunks, chunk_stages, nstages_m, q, D;
    int* err;
};

// Epilogue of A V: per item the 512 accumulator columns (samples in decode
// order) of each digit row, scaled and reduce-scattered over the vector's D
// lanes, are written as exact 64-bit chunk partials.
template <int D>
__device__ __forceinline__ void bt_mv_epilogue(const BtMvArgs& a, uint32_t tmem, uint32_t afull, uint32_t aempty,
                                               int warp, int lane, int nitems) {
    constexpr int per = 16 / D;
    const int sub = warp & 3, r = 32 * sub + lane;
    const int c = r / D, p = r % D, sh = 4 * (D - 1 - p);
    const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
    uint32_t li = 0;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++li) {
        const int blk = item % a.nblocks, ch = item / a.nblocks;
        if (!tc::bar_wait_warp(afull, li & 1u)) {
            atomicCAS(a.err, 0, 30);
            break;
        }
        tc::fence_after();
        long long* Zc = a.Z + ((int64_t)ch * a.q + (c < a.q ? c : 0)) * a.ldz + (int64_t)blk * kStageS;
#pragma unroll 1
        for (int g = 0; g < 32; ++g) {  // 16 columns at a time; half g / 16
            long long z[16];
            bt_ld16_scaled(tmem + lane_base + 16u * g, sh, z);
            if (g == 31) {
                tc::fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(aempty);
            }
            bt_reduce_scatter<D>(z, p);
#pragma unroll
            for (int i = 0; i < per; ++i) {
                const int col = 16 * g + per * p + i;
                const int smp = (col & ~15) + bt_sample_of_kpos(col & 15);
                if (c < a.q) Zc[smp] = z[i];
            }
        }
    }
}

__global__ void __launch_bounds__(kThreadsBT, 1) k_bt_mv(const __grid_constant__ CUtensorMap tmap, BtMvArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = sm_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sb = smem_raw + (base - raw);
    const uint32_t sP = base, sG = sP + kVP * kBoxBytes, sD = sG + kVG * 2 * kTileBytes;
    const uint32_t sBar = sD + kVD * 2 * kTileBytes;
    uint8_t* gP = sb;
    uint8_t* gD = sb + (kVP * kBoxBytes + kVG * 2 * kTileBytes);
    auto pfull = [&](int i) { return sBar + 8u * i; };
    auto pempty = [&](int i) { return sBar + 8u * (kVP + i); };
    auto gfull = [&](int i) { return sBar + 8u * (2 * kVP + i); };
    auto gempty = [&](int i) { return sBar + 8u * (2 * kVP + kVG + i); };
    auto dfull = [&](int i) { return sBar + 8u * (2 * kVP + 2 * kVG + i); };
    auto dempty = [&](int i) { return sBar + 8u * (2 * kVP + 2 * kVG + kVD + i); };
    const uint32_t afull = sBar + 8u * (2 * kVP + 2 * kVG + 2 * kVD);
    const uint32_t aempty = afull + 8u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + (sBar - base) + 512);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tc::tmem_alloc(sm_addr(tmem_slot), 512);
    if (threadIdx.x == 32) {
        for (int i = 0; i < kVP; ++i) {
            bar_init(pfull(i), 1);
            bar_init(pempty(i), kDecWarps);
        }
        for (int i = 0; i < kVG; ++i) {
            bar_init(gfull(i), 1);
            bar_init(gempty(i), 1);
        }
        for (int i = 0; i < kVD; ++i) {
            bar_init(dfull(i), kDecWarps);
            bar_init(dempty(i), 1);
        }
        bar_init(afull, 1);
        bar_init(aempty, kEpiWarps);
        tc::bar_init_fence();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nitems = a.nblocks * a.nchunks;
    auto fail = [&](int code) { atomicCAS(a.err, 0, code); };
    // items run chunk-major: the CTAs of a wave share one chunk's digit tiles
    // (in L2) and read neighbouring 128-byte pieces of the same packed rows
    auto stages_of = [&](int item, int& s0, int& ns) {
        const int ch = item / a.nblocks;
        s0 = ch * a.chunk_stages;
        ns = max(0, min(a.chunk_stages, a.nstages_m - s0));
    };

    if (warp == 0) {
        if (lane == 0) {
            uint32_t ps = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int blk = item % a.nblocks;
                int s0, ns;
                stages_of(item, s0, ns);
                for (int k = 0; k < ns; ++k, ++ps) {
                    const int sp = (int)(ps % kVP), sg = (int)(ps % kVG);
                    if (!bar_wait(pempty(sp), ((ps / kVP) & 1u) ^ 1u) ||
                        !bar_wait(gempty(sg), ((ps / kVG) & 1u) ^ 1u)) {
                        fail(21);
                        ok = false;
                        break;
                    }
                    bar_expect_tx(pfull(sp), kBoxBytes);
                    tc::tma_2d(sP + sp * kBoxBytes, &tmap, 128 * blk, kRowsT * (s0 + k), pfull(sp));
                    bar_expect_tx(gfull(sg), 2 * kTileBytes);
                    tc::bulk_g2s(sG + sg * 2 * kTileBytes, a.dig + (size_t)(s0 + k) * 2 * kTileBytes, 2 * kTileBytes,
                                 gfull(sg));
                }
            }
            for (uint32_t x = ps > (uint32_t)kVP ? ps - kVP : 0u; x < ps; ++x)
                if (!bar_wait(pfull((int)(x % kVP)), (x / kVP) & 1u)) fail(22);
            for (uint32_t x = ps > (uint32_t)kVG ? ps - kVG : 0u; x < ps; ++x)
                if (!bar_wait(gfull((int)(x % kVG)), (x / kVG) & 1u)) fail(23);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_e4m3(256, 1);
            uint32_t ps = 0, it = 0, li = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
                int s0, ns;
                stages_of(item, s0, ns);
                if (!bar_wait(aempty, (li & 1u) ^ 1u)) {
                    fail(24);
                    break;
                }
                tc::fence_after();
                for (int k = 0; k < ns && ok; ++k, ++ps) {
                    const int sg = (int)(ps % kVG);
                    if (!bar_wait(gfull(sg), (ps / kVG) & 1u)) {
                        fail(25);
                        ok = false;
                        break;
                    }
                    const uint64_t a1 = desc_sw128(sG + sg * 2 * kTileBytes);
                    const uint64_t a2 = desc_sw128(sG + sg * 2 * kTileBytes + kTileBytes);
                    for (int ks = 0; ks < 4; ++ks, ++it) {
                        const int sd = (int)(it % kVD);
                        if (!bar_wait(dfull(sd), (it / kVD) & 1u)) {
                            fail(26);
                            ok = false;
                            break;
                        }
                        tc::fence_after();
                        const uint32_t slot = sD + sd * 2 * kTileBytes;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t dcol = tmem + 256u * h;
                            const uint32_t first = (k == 0 && ks == 0) ? 0u : 1u;
                            tc::mma_f8_ss(dcol, a1 + 2 * ks, desc_sw128(slot + h * 8192, 4096, 1024), idesc, first);
                            tc::mma_f8_ss(dcol, a2 + 2 * ks, desc_sw128(slot + kTileBytes + h * 8192, 4096, 1024),
                                          idesc, 1u);
                        }
                        mma_commit(dempty(sd));
                    }
                    if (ok) mma_commit(gempty(sg));
                }
                if (ok) mma_commit(afull);
            }
            if (it > 0) {
                const uint32_t x = it - 1;
                if (!bar_wait(dempty((int)(x % kVD)), (x / kVD) & 1u)) fail(27);
            }
        }
    } else if (warp < kEpi0) {
        // ---- decode: K-step ks = SNP rows 32 ks + lane; 64 samples (16 bytes) per warp
        const int dw = warp - kDec0;
        const int h = dw >> 2, at = (dw >> 1) & 1, c0 = 4 * (dw & 1);
        uint32_t ps = 0, it = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            int s0, ns;
            stages_of(item, s0, ns);
            for (int k = 0; k < ns && ok; ++k, ++ps) {
                const int sp = (int)(ps % kVP);
                if (!tc::bar_wait_warp(pfull(sp), (ps / kVP) & 1u)) {
                    fail(28);
                    ok = false;
                    break;
                }
                for (int ks = 0; ks < 4; ++ks, ++it) {
                    const int sd = (int)(it % kVD);
                    const int row = 32 * ks + lane, g = lane >> 3, rr = lane & 7;
                    const uint4 P = *reinterpret_cast<const uint4*>(gP + sp * kBoxBytes + row * 128 +
                                                                     (((dw ^ (row & 7))) << 4));
                    if (!tc::bar_wait_warp(dempty(sd), ((it / kVD) & 1u) ^ 1u)) {
                        fail(29);
                        ok = false;
                        break;
                    }
                    uint8_t* t1 = gD + sd * 2 * kTileBytes + h * 8192 + at * 4096 + g * 1024 + rr * 128;
                    const uint32_t Wv[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        uint4 o1, o2;
                        bt_decode(Wv[u], o1, o2);
                        const int ch = ((c0 + u) ^ rr) << 4;
                        *reinterpret_cast<uint4*>(t1 + ch) = o1;
                        *reinterpret_cast<uint4*>(t1 + kTileBytes + ch) = o2;
                    }
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) bar_arrive(dfull(sd));
                }
                __syncwarp();
                if (ok && lane == 0) bar_arrive(pempty(sp));
            }
        }
    } else {
        // ---- epilogue: lane = digit row c D + p; columns = samples of the two halves
        if (a.D == 8)
            bt_mv_epilogue<8>(a, tmem, afull, aempty, warp, lane, nitems);
        else
            bt_mv_epilogue<4>(a, tmem, afull, aempty, warp, lane, nitems);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

// Y[i, c] = s_i S_c 2^-4D sum_chunk Z[chunk][c][i]
__global__ void __launch_bounds__(256) k_bt_mv_fin(const long long* __restrict__ Z, int64_t ldz, int nchunks, int64_t n,
                                                   int q, int D, const int* __restrict__ mx,
                                                   const float* __restrict__ s, float* __restrict__ Y, int64_t ldy) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * q) return;
    const int64_t i = e % n, c = e / n;
    long long t = 0;
    for (int ch = 0; ch < nchunks; ++ch) t += Z[((int64_t)ch * q + c) * ldz + i];
    double y = ldexp((double)t, bt_exp(mx[c]) - 4 * D);
    if (s) y *= (double)s[i];
    Y[i + c * ldy] = (float)y;
}

// ---- host side --------------------------------------------------------------------

namespace {
struct BtPlan {
    int nstages_n;    // 512-sample stages of the packed rows
    int nsub;         // 128-sample digit tiles (4 per stage)
    int ntiles;       // 128-SNP tiles
    int nstages_m;    // 128-SNP stages
    int nblocks;      // 512-sample blocks
    int nchunks, chunk_stages;
    int64_t ldz;
    size_t dig_u, dig_v, zbytes;
};

BtPlan plan_bt(const gkl_handle* h, int q) {
    BtPlan p;
    p.nstages_n = (int)((h->stride + 127) / 128);
    p.nsub = 4 * p.nstages_n;
    p.ntiles = (int)((h->m + kRowsT - 1) / kRowsT);
    p.nstages_m = p.ntiles;
    p.nblocks = p.nstages_n;
    p.ldz = (int64_t)p.nblocks * kStageS;
    const int sms = std::max(1, h->num_sms);
    const int min_chunks = (int)((h->m + kMaxSnpsChunk - 1) / kMaxSnpsChunk);
    int best = min_chunks;
    double best_eff = 0.0;
    for (int ch = min_chunks; ch <= std::min(p.nstages_m, min_chunks + 32); ++ch) {
        const int cs = (p.nstages_m + ch - 1) / ch, nch = (p.nstages_m + cs - 1) / cs;
        const double items = (double)p.nblocks * nch;
        const double eff = items / (std::ceil(items / sms) * sms);
        if (eff > best_eff + 0.03) {
            best_eff = eff;
            best = ch;
        }
    }
    p.chunk_stages = (p.nstages_m + best - 1) / best;
    p.nchunks = (p.nstages_m + p.chunk_stages - 1) / p.chunk_stages;
    p.dig_u = (size_t)p.nsub * kTileBytes;
    p.dig_v = (size_t)p.nstages_m * 2 * kTileBytes;
    p.zbytes = (size_t)p.nchunks * (size_t)q * (size_t)p.ldz * sizeof(long long);
    return p;
}
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

bool block_tc_usable(const gkl_handle* h) { return h->tc_state > 0 && h->n <= kMaxSamplesRmv; }

bool block_tc_prepare(gkl_handle* h) {
    if (!block_tc_usable(h)) return false;
    return cudaFuncSetAttribute(k_bt_rmv, cudaFuncAttributeMaxDynamicSharedMemorySize, kRmvSmem) == cudaSuccess &&
           cudaFuncSetAttribute(k_bt_mv, cudaFuncAttributeMaxDynamicSharedMemorySize, kMvSmem) == cudaSuccess;
}

size_t block_tc_scratch_bytes(const gkl_handle* h, int q) {
    const BtPlan p = plan_bt(h, q);
    return al256(std::max(p.dig_u, p.dig_v)) + al256(p.zbytes) + al256(sizeof(int) * 32);
}

// Y (n x q) = A X (transpose = 0) or X' (m x q) = A^T X (transpose = 1) with D
// digits per vector (q D <= 128).
cudaError_t launch_block_product_tc(const gkl_handle* h, bool transpose, const float* X, int64_t ldx, int q, int D,
                                    float* Y, int64_t ldy, void* scratch, int* nlaunch, cudaEvent_t ev0,
                                    cudaEvent_t ev1) {
    if (q < 1 || q * D > 128 || (D != 4 && D != 8)) return cudaErrorInvalidValue;
    const BtPlan p = plan_bt(h, q);
    uint8_t* dig = static_cast<uint8_t*>(scratch);
    long long* Z = reinterpret_cast<long long*>(dig + al256(std::max(p.dig_u, p.dig_v)));
    int* mx = reinterpret_cast<int*>(reinterpret_cast<char*>(Z) + al256(p.zbytes));
    int* err = reinterpret_cast<int*>(reinterpret_cast<char*>(h->aux) + kAuxErrOffset);
    cudaStream_t st = h->stream;
    alignas(64) CUtensorMap map;
    memcpy(&map, h->tc_map, sizeof(map));
    const int sms = std::max(1, h->num_sms);
    const int64_t len = transpose ? h->n : h->m;
    const unsigned sblk = (unsigned)std::max<int64_t>(1, std::min<int64_t>((2 * sms + q - 1) / q, (len + 255) / 256));
    cudaMemsetAsync(mx, 0, sizeof(int) * 32, st);
    k_bt_absmax<<<dim3(sblk, (unsigned)q), 256, 0, st>>>(X, ldx, len, transpose ? 0 : 1, h->s, h->mu, h->d, h->w, mx);
    if (transpose) {
        cudaMemsetAsync(dig, 0, p.dig_u, st);
        k_bt_digits_u<<<dim3((unsigned)p.nsub, (unsigned)q), 128, 0, st>>>(X, ldx, h->n, D, h->s, mx, dig);
        BtRmvArgs a{dig, mx, h->mu, h->d, h->w, Y, ldy, h->m, p.nstages_n, p.ntiles, q, D, err};
        if (ev0) cudaEventRecord(ev0, st);
        k_bt_rmv<<<std::min(p.ntiles, sms), kThreadsBT, kRmvSmem, st>>>(map, a);
        if (ev1) cudaEventRecord(ev1, st);
        if (nlaunch) *nlaunch = 3;
    } else {
        cudaMemsetAsync(dig, 0, p.dig_v, st);
        k_bt_digits_v<<<dim3((unsigned)p.nstages_m, (unsigned)q), 128, 0, st>>>(X, ldx, h->m, D, h->mu, h->d, h->w,
                                                                              mx, dig);
        BtMvArgs a{dig, Z, p.ldz, h->n, p.nblocks, p.nchunks, p.chunk_stages, p.nstages_m, q, D, err};
        if (ev0) cudaEventRecord(ev0, st);
        k_bt_mv<<<std::min(p.nblocks * p.nchunks, sms), kThreadsBT, kMvSmem, st>>>(map, a);
        if (ev1) cudaEventRecord(ev1, st);
        k_bt_mv_fin<<<(unsigned)((h->n * q + 255) / 256), 256, 0, st>>>(Z, p.ldz, p.nchunks, h->n, q, D, mx, h->s, Y,
                                                                        ldy);
        if (nlaunch) *nlaunch = 4;
    }
    return cudaGetLastError();
}

}  // namespace gkl

extern "C" int gkl_matmat(gkl_handle* h, int32_t transpose, int32_t q, int32_t digits, const float* X, int64_t ldx,
                          float* Y, int64_t ldy) {
    using namespace gkl;
    if (!h) return set_err(nullptr, GKL_ERR_ARG, "NULL handle");
    const int64_t rin = transpose ? h->n : h->m, rout = transpose ? h->m : h->n;
    if (!X || !Y || q < 1 || q > 32 || (digits != 4 && digits != 8) || ldx < rin || ldy < rout)
        return set_err(h, GKL_ERR_ARG, "gkl_matmat: need X, Y non-NULL, 1 <= q <= 32, digits 4 or 8, ld >= rows");
    if (mem_kind(X, h->device) != MEM_DEVICE || mem_kind(Y, h->device) != MEM_DEVICE)
        return set_err(h, GKL_ERR_ARG, "gkl_matmat: X and Y must be device memory of the handle's GPU");
    if (!block_tc_prepare(h))
        return set_err(h, GKL_ERR_ARG, "gkl_matmat: tensor-core block products unavailable for this handle");
    void* scratch = nullptr;
    const int per = 128 / digits;
    cudaError_t e = cudaMalloc(&scratch, block_tc_scratch_bytes(h, std::min<int>(per, q)));
    for (int c0 = 0; c0 < q && e == cudaSuccess; c0 += per)
        e = launch_block_product_tc(h, transpose != 0, X + (int64_t)c0 * ldx, ldx, std::min(per, q - c0), digits,
                                    Y + (int64_t)c0 * ldy, ldy, scratch, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (scratch) cudaFree(scratch);
    if (e != cudaSuccess) return cuda_err(h, e, "gkl_matmat");
    return take_pending_error(h);  // a tensor-core pipeline wait that ran out (read and cleared on h's stream)
}

