// Blackwell tensor-core A^T u (FP32 and FP64 paths):
//     x_j = d_j w_j [ sum_{i obs} g_ij u~_i - mu_j sum_{i obs} u~_i ],  u~ = s o u
// (A as defined in gkl.h; the per-step product of GKL bidiagonalisation,
// section 3 of arXiv:1808.03374).
//
// The contraction over samples is exact integer arithmetic on the
// 5th-generation tensor cores (tcgen05.mma kind::mxf4: packed e2m1 operands,
// block scales all 1.0, FP32 accumulation in tensor memory):
//  * u~ in fixed point: z_i = rint(u~_i 2^b / S), S = 2^e > max|u~|, so
//    |z_i| <= 2^b and u~'_i = S 2^-b z_i is within 2^-(b+1) S of u~_i; z_i is
//    written with D = b/3 + 1 balanced base-8 digits delta_p in [-4, 3] (all
//    exact in e2m1), z_i = sum_p delta_p,i 8^(D-1-p).  FP32: b = 30, D = 11;
//    FP64: b = 57, D = 20 -- the same MMAs, more digit rows;
//  * orientation: the D digit rows are the MMA's A operand (M = 128 lanes of
//    tensor memory, the other rows zero), the codes of 256 SNPs its B operand
//    (N = 256) and the samples its K axis: one MMA covers 256 SNPs x 64
//    samples.  A 2-bit code c read as an e2m1 nibble is the value c/2, so the
//    decode of a 32-bit word of 16 codes is two masks -- the 8 even samples
//    (W & 0x33333333) and the 8 odd ones ((W >> 2) & 0x33333333) -- and the K
//    order within each 16 samples is even samples, then odd ones (the digit
//    image is written in that order);
//  * accumulators F_p,j = sum_i (c_ij / 2) delta_p,i are multiples of 1/2
//    below 2^23 (K-ranges of at most 2,048 stages of 512 samples), so exact in
//    FP32, and X_j = sum_p 8^(D-1-p) 2 F_p,j = sum_i c_ij z_i is recombined in
//    64-bit integers (for D = 20 in two halves of 10 digits, joined in FP64);
//  * the missing code 3 counts as 3 there.  The missing codes are few (1-2%
//    of the entries) and fixed per matrix: gkl_init lists them once per SNP
//    (sample indices, ascending) and a gather kernel forms Z_j = sum of z_i
//    over the missing samples of SNP j (exact, 64-bit), so that
//    sum_{obs} g u~' = S 2^-b (X_j - 3 Z_j) and
//    sum_{obs} u~' = sum_i u~'_i - S 2^-b Z_j.  (Summing them in the decode
//    warps instead costs a divergent loop per code word: measured 44 warp
//    instructions per word, four times the MMAs' time.)
// Data movement per 512-sample stage of a 256-SNP tile: two TMA boxes of
// 128 rows x 128 bytes (128-byte swizzle) and one bulk copy of the stage's
// digit rows; the decode warps write the e2m1
// operand (two 32 KB K-chunks of 256 samples, 128-byte swizzled, K-major) to
// shared memory; one warp moves the digit rows of each K-chunk from shared to
// tensor memory.  Warp roles: 0 copies, 1 issues the MMAs, 4 writes the
// digits, 8 runs the epilogue (warps 4 and 8 own tensor-memory lanes 0-31),
// 2-3, 5-7 and 9-19 decode (one SNP row and one K-chunk per thread).  One persistent CTA per SM walks work items (tile, K-range) with
// the K-ranges of a tile consecutive, so that each row is read as one
// contiguous run.
//
// Every wait is bounded (about two seconds of clock); a wait that runs out
// sets an error word that the host reads at its next synchronising call, and
// the kernel drains its copies and frees its tensor memory before it returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "epilogue.cuh"
#include "gkl_internal.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"

namespace gkl {

namespace {
constexpr int kTile = 256;                 // SNPs per work item = MMA N
constexpr int kStageSamples = 512;         // samples per stage: 128 packed bytes per row
constexpr int kBox = 128;                  // rows per TMA box
constexpr int kBoxBytes = kBox * 128;      // 16 KB
constexpr int kStageBytes = 2 * kBoxBytes; // 32 KB of packed codes per stage
constexpr int kUnitBytes = kTile * 128;    // decoded K-chunk: 256 rows x 128 bytes (256 samples in e2m1)
constexpr int kRP = 3, kRD = 3, kRA = 3;   // ring depths: packed stages, decoded K-chunks, digit buffers
constexpr int kUnitWords = 32;
constexpr int kDigitsF32 = 11, kDigitsF64 = 20;             // tensor-memory columns of one K-chunk of digits (8 nibbles each)
constexpr int kMaxRangeStages = 2048;      // |2 F_p| <= 12 x 512 x 2048 < 2^24
constexpr int kDecodeWarps = 16;           // two groups of 8: K-chunk 0 and 1 of every stage
constexpr int kThreads = 640;              // 20 warps
constexpr int kWarpMma = 1, kWarpDigits = 4, kWarpEpi = 8;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColA = 256, kColSF = 448, kColSFA = 448, kColSFB = 480;
constexpr int kOffD = kRP * kStageBytes;
constexpr int kOffG = kOffD + kRD * kUnitBytes;
static_assert(kOffD % 1024 == 0, "decoded tiles must stay 1024-byte aligned");
// block-scaled instruction descriptor (kind::mxf4): A and B E2M1 (format 1,
// bits 7-9 and 10-12), K-major, N >> 3 at bits 17-22, scale format UE8M0
// (bit 23), M >> 4 at bits 24-28, scale-factor ids 0, K = 64 (bit 31 clear)
constexpr uint32_t kIdesc = (1u << 7) | (1u << 10) | ((uint32_t)(kTile >> 3) << 17) | (1u << 23) | ((128u >> 4) << 24);

// Fixed point with D balanced base-8 digits: z_i = rint(u~_i 2^kBits / S),
// |z_i| <= 2^kBits = 8^(D-1) (the leading digit is then -1, 0 or 1).  D = 11
// (30 bits, finer than FP32) serves the FP32 product, D = 20 (57 bits, finer
// than FP64) the FP64 one.  Digit rows 0 .. kHalf0-1 sit in tensor-memory
// lanes 0 .. kHalf0-1, the rest from lane 16 on, so that each 16-lane half
// recombines its digits in 64-bit integers without overflow (weights at most
// 8^10 on FP32 accumulators below 2^24).
template <int D>
struct Fx {
    static constexpr int kBits = 3 * (D - 1);
    static constexpr int kHalf0 = D <= 11 ? D : D / 2;
    using Z = std::conditional_t<(D <= 11), int, long long>;  // holds z_i (|z_i| <= 2^kBits)
    static constexpr int kGBytes = 2 * D * kUnitWords * 4;  // digit rows of one stage (2 K-chunks)
    static constexpr int kOffBar = kOffG + kRP * kGBytes;
    static constexpr int kSmem = 1024 + kOffBar + 1024;
    static_assert(kSmem <= 232448, "shared memory of k_rmv_tc");
    static_assert(D - kHalf0 <= 11 && kHalf0 <= 11, "weights of at most 8^10 per half");
    // digit row held by tensor-memory lane L (0..31) of the digit warp, or -1
    __host__ __device__ static constexpr int digit_of_lane(int L) {
        return L < 16 ? (L < kHalf0 ? L : -1) : (L - 16 < D - kHalf0 ? kHalf0 + L - 16 : -1);
    }
};

// decode warps: 2, 3, 5, 6, 7, 9 .. 19 -> index 0..15; index / 8 = the K-chunk of
// every stage the warp decodes, 32 (index mod 8) + lane = its SNP row
__device__ __forceinline__ int decode_index(int warp) {
    return warp < 4 ? warp - 2 : (warp < 8 ? warp - 3 : warp - 4);
}
}  // namespace

using tc::bar_arrive;
using tc::bar_expect_tx;
using tc::bar_init;
using tc::bar_wait;
using tc::bulk_g2s;
using tc::desc_sw128;
using tc::mma_commit;
using tc::sm_addr;
using tc::tma_2d;

// D (tensor memory) (+)= A (tensor memory) x B (shared memory)^T with e2m1
// operands and block scales from tensor memory.
__device__ __forceinline__ void mma_f4_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t sfa, uint32_t sfb,
                                          uint32_t acc) {
    asm volatile(
        "{.reg .pred p; setp.ne.b32 p, %5, 0; "
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], [%1], %2, %6, [%3], [%4], p;}\n" ::"r"(
            d),
        "r"(a), "l"(bdesc), "r"(sfa), "r"(sfb), "r"(acc), "r"(kIdesc));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// ---- scale of u~ ------------------------------------------------------------

// Pass 1: max|u~| and sum u~ (FP64), combined by the last block; the scale
// S = 2^e >= max|u~| and the sum go to dsc[0..2] = {S, 1/S, sum}.
template <typename T>
__global__ void __launch_bounds__(256) k_u_scale(const T* __restrict__ u, const float* __restrict__ s, int64_t n,
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

// ---- digits of u~ -------------------------------------------------------------

// e2m1 nibble of a balanced base-8 digit in [-4, 3] (index digit + 4):
// -4 -3 -2 -1 0 1 2 3  ->  0xE 0xD 0xC 0xA 0x0 0x2 0x4 0x5
__device__ __forceinline__ uint32_t e2m1_digit(int dg) {
    constexpr uint32_t lut = 0x5420ACDEu;  // nibble k = code of digit k - 4
    return (lut >> (4 * (dg + 4))) & 0xFu;
}

// One thread per tensor-memory word of a K-chunk (256 samples): the 8 samples
// at K positions 8 w .. 8 w + 7 (K position kk of sample loc in the chunk:
// 16 (loc / 16) + even/odd order within the 16, as the decode emits it).
// Writes their z values and, for every digit row p < D, the word of 8
// nibbles: image[chunk][p][w ^ 4 (p & 7)] (chunk-swizzled rows, below).
template <typename T, int D>
__global__ void __launch_bounds__(256) k_u_digits_f4(const T* __restrict__ u, const float* __restrict__ s, int64_t n,
                                                      int64_t nwords, const double* __restrict__ dsc,
                                                      uint32_t* __restrict__ image,
                                                      typename Fx<D>::Z* __restrict__ zout) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nwords) return;
    const int64_t chunk = t / kUnitWords;
    const int w = (int)(t % kUnitWords);
    const double inv = dsc[1];
    uint32_t word[D];
#pragma unroll
    for (int p = 0; p < D; ++p) word[p] = 0u;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int kk = 8 * w + e;
        const int loc = 16 * (kk >> 4) + bt_sample_of_kpos(kk & 15);
        const int64_t i = chunk * 256 + loc;
        long long z = 0;
        if (i < n) {
            const double x = (double)u[i] * (s ? (double)s[i] : 1.0) * inv;  // |x| < 1
            z = __double2ll_rn(ldexp(x, Fx<D>::kBits));
        }
        zout[i] = (typename Fx<D>::Z)z;
        long long r = z;
#pragma unroll
        for (int p = D - 1; p >= 1; --p) {
            const int dg = (int)((r + 4) & 7) - 4;
            word[p] |= e2m1_digit(dg) << (4 * e);
            r = (r - dg) >> 3;
        }
        word[0] |= e2m1_digit((int)r) << (4 * e);  // r in {-1, 0, 1}: |z| <= 8^(D-1)
    }
    // row p's 16-byte chunk c is stored at chunk c ^ (p & 7), so that the digit
    // warp's lanes (one row each) read different shared-memory banks
    uint32_t* dst = image + chunk * (D * kUnitWords);
#pragma unroll
    for (int p = 0; p < D; ++p) dst[p * kUnitWords + (w ^ ((p & 7) << 2))] = word[p];
}

// ---- main kernel ------------------------------------------------------------

struct TcArgs {
    const uint32_t* image;  // K-chunks x D x 32 digit words (k_u_digits_f4)
    int nstages, range_stages, nranges, ntiles;
    int64_t m;
    const double* dsc;      // {S, 1/S, sum u~}
    double* p1;             // nranges x m: S 2^-kBits X_j over the range
    int* err;               // set to a nonzero code if a wait ran out
};

template <int D>
__global__ void __launch_bounds__(kThreads, 1) k_rmv_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
    using F = Fx<D>;
    constexpr int kGBytes = F::kGBytes, kOffBar = F::kOffBar;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = sm_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sb = smem_raw + (base - raw);
    const uint32_t sP = base, sD = base + kOffD, sG = base + kOffG, sBar = base + kOffBar;
    auto pfull = [&](int i) { return sBar + 8u * i; };
    auto pempty = [&](int i) { return sBar + 8u * (kRP + i); };
    auto dfull = [&](int i) { return sBar + 8u * (2 * kRP + i); };
    auto dempty = [&](int i) { return sBar + 8u * (2 * kRP + kRD + i); };
    auto gfull = [&](int i) { return sBar + 8u * (2 * kRP + 2 * kRD + i); };
    auto gempty = [&](int i) { return sBar + 8u * (2 * kRP + 2 * kRD + kRA + i); };
    const uint32_t afull = sBar + 8u * (2 * kRP + 2 * kRD + 2 * kRA);
    const uint32_t aempty = afull + 8u;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + kOffBar + 512);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tc::tmem_alloc(sm_addr(tmem_slot), kTmemCols);
    if (threadIdx.x == 32) {
        for (int i = 0; i < kRP; ++i) {
            bar_init(pfull(i), 1);
            bar_init(pempty(i), kDecodeWarps + 1);  // decode warps and the digit warp
        }
        for (int i = 0; i < kRD; ++i) {
            bar_init(dfull(i), 8);
            bar_init(dempty(i), 1);
        }
        for (int i = 0; i < kRA; ++i) {
            bar_init(gfull(i), 1);
            bar_init(gempty(i), 1);
        }
        bar_init(afull, 1);
        bar_init(aempty, 1);
        tc::bar_init_fence();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp >= 4 && warp < 8) {
        // every lane: block scales 1.0 (UE8M0 127) and zero digit buffers
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        uint32_t v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0x7F7F7F7Fu;
        tmem_st32(tmem + lane_base + kColSF, v);
        tmem_st32(tmem + lane_base + kColSF + 32u, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0u;
        for (int b = 0; b < kRA; ++b) tmem_st32(tmem + lane_base + kColA + 32u * b, v);
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const int nitems = a.ntiles * a.nranges;
    auto fail = [&](int code) { atomicCAS(a.err, 0, code); };

    if (warp == 0) {
        // ---- copies: per stage two TMA boxes (256 rows x 128 bytes) and the stage's z values
        if (lane == 0) {
            uint32_t ps = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int tile = item / a.nranges, range = item % a.nranges;
                const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
                for (int k = 0; k < nst; ++k, ++ps) {
                    const int s = (int)(ps % kRP);
                    if (!bar_wait(pempty(s), ((ps / kRP) & 1u) ^ 1u)) {
                        fail(1);
                        ok = false;
                        break;
                    }
                    bar_expect_tx(pfull(s), kStageBytes + kGBytes);
                    const int x = 128 * (st0 + k);
                    tma_2d(sP + s * kStageBytes, &tmap, x, kTile * tile, pfull(s));
                    tma_2d(sP + s * kStageBytes + kBoxBytes, &tmap, x, kTile * tile + kBox, pfull(s));
                    bulk_g2s(sG + s * kGBytes, a.image + (size_t)(st0 + k) * (2 * D * kUnitWords), kGBytes, pfull(s));
                }
            }
            // drain: every issued copy has landed before the CTA may exit
            for (uint32_t q = ps > (uint32_t)kRP ? ps - kRP : 0u; q < ps; ++q)
                if (!bar_wait(pfull((int)(q % kRP)), (q / kRP) & 1u)) fail(2);
        }
    } else if (warp == kWarpMma) {
        // ---- MMA issuer: per K-chunk of 256 samples four MMAs (K = 64) into the one accumulator
        if (lane == 0) {
            uint32_t du = 0, li = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
                const int range = item % a.nranges;
                const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
                if (!bar_wait(aempty, (li & 1u) ^ 1u)) {  // the epilogue has read the previous item
                    fail(3);
                    break;
                }
                tc::fence_after();
                for (int g = 0; g < 2 * nst; ++g, ++du) {
                    const int d = (int)(du % kRD), ga = (int)(du % kRA);
                    if (!bar_wait(dfull(d), (du / kRD) & 1u) || !bar_wait(gfull(ga), (du / kRA) & 1u)) {
                        fail(4);
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    const uint64_t bd = desc_sw128(sD + d * kUnitBytes);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        mma_f4_ts(tmem, tmem + kColA + 32u * ga + 8u * ks, bd + 2 * ks, tmem + kColSFA,
                                  tmem + kColSFB, (g | ks) != 0);
                    mma_commit(dempty(d));
                    mma_commit(gempty(ga));
                }
                if (ok) mma_commit(afull);
            }
            // drain: the last commit covers every MMA issued by this thread
            if (du > 0) {
                const uint32_t q = du - 1;
                if (!bar_wait(dempty((int)(q % kRD)), (q / kRD) & 1u)) fail(5);
            }
        }
    } else if (warp == kWarpDigits) {
        // ---- digits: the D rows of each K-chunk, from the stage's shared-memory copy into
        // tensor memory (lane L holds digit row digit_of_lane(L); the other lanes zero)
        const int prow = F::digit_of_lane(lane);
        uint32_t ps = 0, du = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int range = item % a.nranges;
            const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
            for (int k = 0; k < nst && ok; ++k, ++ps) {
                const int s = (int)(ps % kRP);
                if (!tc::bar_wait_warp(pfull(s), (ps / kRP) & 1u)) {
                    fail(10);
                    ok = false;
                    break;
                }
                for (int h = 0; h < 2; ++h, ++du) {
                    const int ga = (int)(du % kRA);
                    uint32_t v[32];
                    if (prow >= 0) {
                        const uint4* src = reinterpret_cast<const uint4*>(sb + kOffG + s * kGBytes +
                                                                          (h * D + prow) * kUnitWords * 4);
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const uint4 q = src[c ^ (prow & 7)];
                            v[4 * c] = q.x;
                            v[4 * c + 1] = q.y;
                            v[4 * c + 2] = q.z;
                            v[4 * c + 3] = q.w;
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c) v[c] = 0u;
                    }
                    if (!tc::bar_wait_warp(gempty(ga), ((du / kRA) & 1u) ^ 1u)) {
                        fail(6);
                        ok = false;
                        break;
                    }
                    tc::fence_after();
                    tmem_st32(tmem + kColA + 32u * ga, v);
                    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) bar_arrive(gfull(ga));
                }
                __syncwarp();
                if (ok && lane == 0) bar_arrive(pempty(s));
            }
        }
    } else if (warp == kWarpEpi) {
        // ---- epilogue: X_j = sum_p 8^(D-1-p) 2 F_p,j, summed per 16-lane half in 64-bit
        // integers (X0 over the digits of lanes 0-15, X1 over those of lanes 16-31) and
        // recombined as X0 8^(D-kHalf0) + X1
        uint32_t li = 0;
        const double sc = ldexp(a.dsc[0], -F::kBits);
        const int p = lane & 15, dl = F::digit_of_lane(lane);
        const int sh = dl < 0 ? 0 : (lane < 16 ? 3 * (F::kHalf0 - 1 - dl) : 3 * (D - 1 - dl));
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++li) {
            const int tile = item / a.nranges, range = item % a.nranges;
            if (!tc::bar_wait_warp(afull, li & 1u)) {
                fail(7);
                break;
            }
            tc::fence_after();
#pragma unroll 1
            for (int g = 0; g < 8; ++g) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + 32u * g, r);
                if (g == 7) {
                    tc::fence_before();
                    __syncwarp();
                    if (lane == 0) bar_arrive(aempty);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    long long v[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        v[i] = dl >= 0 ? (long long)__float2int_rn(2.f * __uint_as_float(r[16 * h + i])) << sh : 0LL;
                    bt_reduce_scatter<16>(v, p);
                    double X = (double)v[0];
                    if constexpr (D > F::kHalf0) {
                        const long long x1 = shfl_xor_ll(v[0], 16);
                        X = ldexp(X, 3 * (D - F::kHalf0)) + (double)x1;
                    }
                    const int64_t j = (int64_t)tile * kTile + 32 * g + 16 * h + p;
                    if (lane < 16 && j < a.m) a.p1[(int64_t)range * a.m + j] = sc * X;
                }
            }
        }
    } else {
        // ---- decode: SNP row 32 (index mod 8) + lane of the tile, K-chunk h = index / 8 of every stage
        const int di = decode_index(warp), h = di >> 3;
        const int row = 32 * (di & 7) + lane, box = row >> 7, rr = row & 127;
        uint32_t ps = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int range = item % a.nranges;
            const int nst = min(a.range_stages, a.nstages - range * a.range_stages);
            for (int k = 0; k < nst && ok; ++k, ++ps) {
                const int s = (int)(ps % kRP);
                if (!tc::bar_wait_warp(pfull(s), (ps / kRP) & 1u)) {
                    fail(8);
                    ok = false;
                    break;
                }
                const uint8_t* prow = sb + s * kStageBytes + box * kBoxBytes + rr * 128;
                const uint32_t du = 2 * ps + (uint32_t)h;  // this K-chunk's place in the sequence of all K-chunks
                const int d = (int)(du % kRD);
                uint4 P[4];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    P[c] = *reinterpret_cast<const uint4*>(prow + (((4 * h + c) ^ (rr & 7)) << 4));
                if (!tc::bar_wait_warp(dempty(d), ((du / kRD) & 1u) ^ 1u)) {
                    fail(9);
                    ok = false;
                    break;
                }
                uint8_t* drow = sb + kOffD + d * kUnitBytes + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t W[4] = {P[c].x, P[c].y, P[c].z, P[c].w};
                    uint32_t o[8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        o[2 * q] = W[q] & 0x33333333u;             // even samples: codes 0, 2 of each byte
                        o[2 * q + 1] = (W[q] >> 2) & 0x33333333u;  // odd samples
                    }
                    *reinterpret_cast<uint4*>(drow + (((2 * c) ^ (row & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
                    *reinterpret_cast<uint4*>(drow + (((2 * c + 1) ^ (row & 7)) << 4)) =
                        make_uint4(o[4], o[5], o[6], o[7]);
                }
                tc::fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    bar_arrive(dfull(d));
                    bar_arrive(pempty(s));
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// ---- the list of missing codes and its per-product sum ------------------------
//
// The samples are cut into blocks of kMissBlock; segment (b, j) lists the
// missing samples of SNP j in block b as 16-bit offsets into the block,
// ascending, padded with kMissPad to a multiple of 8 entries (one 16-byte
// load); kMissPad is the offset of a zero slot just past the block, so the
// gather needs no test per entry.  Segments are stored block-major, off[b m + j] is the first entry of
// segment (b, j) and off[nb m] the list's length.  Per product one CTA holds
// the z values of one block in shared memory and gathers them there for a
// chunk of SNPs: the list is read once from HBM (2 bytes an entry) and the
// gathers never leave the SM.

constexpr int kMissBlock = 24576;                // samples a block: its int64 z values fill 192 KB of shared memory
constexpr uint16_t kMissPad = (uint16_t)kMissBlock;  // padding entry: the zero slot after the block's z values
constexpr int kMissSlots = kMissBlock + 16;       // z values, zero slot, padding to 16 bytes
constexpr int kMissThreads = 1024;
static_assert(kMissBlock % 16 == 0 && kMissBlock < 65536, "block of the missing-code list");

// Missing-code mask of packed word wd of a row (bit 2 s set where sample 16 wd + s has code 3),
// samples at or above n cleared.
__device__ __forceinline__ uint32_t miss_mask(const uint32_t* row, int64_t wd, int64_t n) {
    uint32_t Y = row[wd] & (row[wd] >> 1) & 0x55555555u;
    const int64_t valid = n - wd * 16;
    if (valid < 16) Y &= (1u << (2 * valid)) - 1u;
    return Y;
}

// counts[b m + j] = missing codes of SNP j in sample block b; one warp per (j, b).
__global__ void __launch_bounds__(256) k_miss_count(const uint8_t* __restrict__ packed, int64_t stride, int64_t n,
                                                     int64_t m, int nb, int* __restrict__ counts) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= m * nb) return;
    const int64_t j = gw / nb;
    const int b = (int)(gw % nb);
    const uint32_t* row = reinterpret_cast<const uint32_t*>(packed + j * stride);
    const int64_t words = (n + 15) / 16;
    const int64_t w0 = (int64_t)b * (kMissBlock / 16), w1 = min(words, w0 + kMissBlock / 16);
    int c = 0;
    for (int64_t wd = w0 + lane; wd < w1; wd += 32) c += __popc(miss_mask(row, wd, n));
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) counts[(int64_t)b * m + j] = c;
}

// Writes segment (b, j) of the list and its padding; one warp per (j, b).
__global__ void __launch_bounds__(256) k_miss_fill(const uint8_t* __restrict__ packed, int64_t stride, int64_t n,
                                                    int64_t m, int nb, const int64_t* __restrict__ off,
                                                    uint16_t* __restrict__ idx) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= m * nb) return;
    const int64_t j = gw / nb;
    const int b = (int)(gw % nb);
    const uint32_t* row = reinterpret_cast<const uint32_t*>(packed + j * stride);
    const int64_t words = (n + 15) / 16;
    const int64_t w0 = (int64_t)b * (kMissBlock / 16), w1 = min(words, w0 + kMissBlock / 16);
    const int64_t seg = (int64_t)b * m + j;
    int64_t pos = off[seg];
    const int64_t end = off[seg + 1];
    for (int64_t wb = w0; wb < w1; wb += 32) {
        const int64_t wd = wb + lane;
        uint32_t Y = wd < w1 ? miss_mask(row, wd, n) : 0u;
        const int c = __popc(Y);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int64_t q = pos + incl - c;
        while (Y) {
            const int bit = __ffs(Y) - 1;
            Y &= Y - 1u;
            if (q < end) idx[q] = (uint16_t)((wd - w0) * 16 + (bit >> 1));
            ++q;
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    for (int64_t q = pos + lane; q < end; q += 32) idx[q] = kMissPad;
}

// p3[b m + j] = S 2^-bits Z_bj, Z_bj = sum of z_i over the missing samples of
// SNP j in block b.  The sum is exact: 64-bit integers (ZT = int), or for
// 64-bit z the parts z = 2^30 hi + lo (lo in [0, 2^30)) summed apart and
// joined once in FP64.  Persistent: CTA c takes the segments [s0, s1) of the
// block-major order (one contiguous run of the list), loads the z values of
// each block its run touches into shared memory, and walks the run in batches
// of 128 segments, eight lanes a segment; the first 256 entries of a segment
// come in four 16-byte loads a lane, issued one batch ahead (the offsets two
// batches ahead) so that the loads overlap the gathers of the batch before.
struct MissSeg {
    int64_t e0, e1;  // 16-byte units of the list
};

__device__ __forceinline__ MissSeg miss_seg(const int64_t* __restrict__ off, int64_t s, int64_t a1) {
    if (s >= a1) return MissSeg{0, 0};
    return MissSeg{__ldcs(off + s) >> 3, __ldcs(off + s + 1) >> 3};
}

__device__ __forceinline__ void miss_load(const uint4* __restrict__ src, MissSeg g, int sl, uint4 (&q)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t e = g.e0 + sl + 8 * r;
        constexpr uint32_t kPad2 = (uint32_t)kMissPad * 0x10001u;
        q[r] = e < g.e1 ? __ldcs(src + e) : make_uint4(kPad2, kPad2, kPad2, kPad2);
    }
}

// Eight list entries (one 16-byte load): each offset is clamped to the zero
// slot (a corrupt offset is counted in bad and adds nothing), then its z value
// is added.
template <typename ZT>
__device__ __forceinline__ void miss_gather(uint4 q, const ZT* zs, long long& zh, long long& zl, uint32_t& bad) {
    constexpr uint32_t kPad2 = (uint32_t)kMissPad * 0x10001u;
    uint32_t wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const uint32_t cl = __vminu2(wv[c], kPad2);
        bad |= wv[c] ^ cl;
        wv[c] = cl;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t o = c & 1 ? wv[c >> 1] >> 16 : wv[c >> 1] & 0xFFFFu;
        const long long zi = (long long)zs[o];
        if constexpr (sizeof(ZT) == 4) {
            zl += zi;
        } else {
            zh += zi >> 30;
            zl += zi & ((1LL << 30) - 1);
        }
    }
}

template <typename ZT>
__global__ void __launch_bounds__(kMissThreads, 1) k_miss_sum(const int64_t* __restrict__ off,
                                                               const uint16_t* __restrict__ idx, int64_t m, int nb,
                                                               const ZT* __restrict__ z, int64_t zlen, int bits,
                                                               const double* __restrict__ dsc, double* __restrict__ p3,
                                                               int* __restrict__ err) {
    extern __shared__ __align__(16) uint8_t miss_smem[];
    ZT* zs = reinterpret_cast<ZT*>(miss_smem);
    constexpr int kGroups = kMissThreads / 8;
    const int grp = threadIdx.x >> 3, sl = threadIdx.x & 7;
    const int64_t nseg = m * nb;
    const int64_t per = (nseg + gridDim.x - 1) / gridDim.x;
    const int64_t s0 = (int64_t)blockIdx.x * per, s1 = min(nseg, s0 + per);
    const double sc = ldexp(dsc[0], -bits);
    const uint4* src = reinterpret_cast<const uint4*>(idx);
    uint32_t bad = 0u;
    for (int64_t b = s0 / m; s0 < s1 && b * m < s1; ++b) {
        const int64_t a0 = max(s0, b * m), a1 = min(s1, (b + 1) * m);
        const int64_t z0 = b * kMissBlock;
        const int cnt = (int)min((int64_t)kMissBlock, zlen - z0);
        __syncthreads();  // the previous block's gathers are done
        for (int i = threadIdx.x; i < kMissSlots; i += blockDim.x) zs[i] = i < cnt ? z[z0 + i] : (ZT)0;
        __syncthreads();
        MissSeg cur = miss_seg(off, a0 + grp, a1);
        MissSeg nxt = miss_seg(off, a0 + kGroups + grp, a1);
        uint4 q[4], qn[4];
        miss_load(src, cur, sl, q);
        for (int64_t sb = a0; sb < a1; sb += kGroups) {  // the same trip count in every lane
            const int64_t s = sb + grp;
            miss_load(src, nxt, sl, qn);                                  // batch t + 1
            const MissSeg nn = miss_seg(off, sb + 2 * kGroups + grp, a1);  // batch t + 2
            long long zh = 0, zl = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) miss_gather<ZT>(q[r], zs, zh, zl, bad);
            for (int64_t e = cur.e0 + 32 + sl; e < cur.e1; e += 8)  // entries beyond the first 256
                miss_gather<ZT>(__ldcs(src + e), zs, zh, zl, bad);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                zh += __shfl_xor_sync(0xffffffffu, zh, o);
                zl += __shfl_xor_sync(0xffffffffu, zl, o);
            }
            if (s < a1 && sl == 0) p3[s] = sc * (ldexp((double)zh, 30) + (double)zl);
            cur = nxt;
            nxt = nn;
#pragma unroll
            for (int r = 0; r < 4; ++r) q[r] = qn[r];
        }
    }
    if (bad) atomicCAS(err, 0, 51);  // an offset outside its block: clamped to the zero slot, reported
}

// ---- finishing kernel ----------------------------------------------------------

// Sums over the K-ranges (fixed order), then
//   x_j = d_j w_j [ (sum_r P1 - 3 sum_r P3) - mu_j (sum_i u~_i - sum_r P3) ]
// (P1 = S 2^-bits sum c z over the range, missing codes counted as 3; P3 = the
// missing samples' share), the subtraction of earlier basis vectors and the
// solver's norm reduction.
template <typename T>
__global__ void __launch_bounds__(256) k_rmv_tc_fin(const double* __restrict__ p1, const double* __restrict__ p3,
                                                    int nr, int nb, int64_t m, const double* __restrict__ mu,
                                                    const double* __restrict__ d, const float* __restrict__ w,
                                                    const double* __restrict__ dsc, T* __restrict__ x, FinArgs fa,
                                                    Sv sv) {
    if (fa.role != ROLE_NONE && sv.sc->abort) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (j < m) {
        double hsum = 0.0, msum = 0.0;
        for (int r = 0; r < nr; ++r) hsum += p1[(int64_t)r * m + j];
        for (int b = 0; b < nb; ++b) msum += p3[(int64_t)b * m + j];
        double dw = d[j];
        if (w) dw *= (double)w[j];
        const double obs_g = hsum - 3.0 * msum;  // sum of g u~ over the observed samples
        const double obs = dsc[2] - msum;        // sum of u~ over the observed samples
        T val = (T)(dw * (obs_g - mu[j] * obs));
        const T* W = static_cast<const T*>(fa.W);
        for (int q = 0; q < fa.nsub; ++q) val -= (T)fa.bcol[q] * W[j + (int64_t)q * fa.ldw];
        x[j] = val;
        sq = (double)val * (double)val;
    }
    if (fa.role == ROLE_NONE) return;
    __shared__ double s_w[32];
    double v = warp_sum(sq);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_w[q];
        sv.partials[(int64_t)blockIdx.x * (GKL_MAX_ELL + 2)] = t;
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
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += s_w[q];
        s_tot = t;
    }
    __syncthreads();
    step_epilogue(sv, fa.role, fa.j, s_tot);
    __syncthreads();
    release_counter(&sv.sc->counter);
}

// ---- host side --------------------------------------------------------------

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct TcPlan {
    int nstages, range_stages, nranges, ntiles, grid;
    int nb, miss_grid;  // sample blocks of the missing-code list; CTAs of its sum
    int64_t nwords;  // digit-image words of one row: K-chunks x 32
    size_t img_bytes, z_bytes, part_bytes;
};

// Work items (256-SNP tile, K-range): K-ranges of at most 2,048 stages; more
// ranges only where they even out the last wave of items over the SMs.
static TcPlan plan_tc(const gkl_handle* h) {
    TcPlan p;
    p.nstages = (int)((h->stride + 127) / 128);
    p.ntiles = (int)((h->m + kTile - 1) / kTile);
    const int sms = std::max(1, h->num_sms);
    const int nr0 = (p.nstages + kMaxRangeStages - 1) / kMaxRangeStages;
    int best = nr0;
    double best_eff = 0.0;
    for (int nr = nr0; nr <= std::min(p.nstages, nr0 + 7); ++nr) {
        const int rs = (p.nstages + nr - 1) / nr, nranges = (p.nstages + rs - 1) / rs;
        const double items = (double)p.ntiles * nranges;
        const double eff = items / (std::ceil(items / sms) * sms);
        if (eff > best_eff + 0.03) {
            best_eff = eff;
            best = nr;
        }
    }
    p.range_stages = (p.nstages + best - 1) / best;
    p.nranges = (p.nstages + p.range_stages - 1) / p.range_stages;
    p.grid = (int)std::min<int64_t>((int64_t)p.ntiles * p.nranges, sms);
    p.nwords = (int64_t)2 * p.nstages * kUnitWords;
    p.img_bytes = (size_t)2 * p.nstages * Fx<kDigitsF64>::kGBytes / 2;  // the larger digit image
    p.z_bytes = (size_t)p.nstages * kStageSamples * sizeof(long long);
    p.nb = (int)std::max<int64_t>(1, (h->n + kMissBlock - 1) / kMissBlock);
    p.miss_grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, (h->m * p.nb + 127) / 128));
    p.part_bytes = ((size_t)p.nranges + p.nb) * (size_t)h->m * sizeof(double);  // P1 per K-range, P3 per block
    return p;
}

size_t rmv_tc_scratch_bytes(const gkl_handle* h) {
    const TcPlan p = plan_tc(h);
    return al256(p.img_bytes) + al256(p.z_bytes) + p.part_bytes + 256;
}

// Prepares the tensor-core path for a handle: the TMA descriptor of the packed
// matrix (128-byte x 128-row boxes, 128-byte swizzle) and the kernel's
// shared-memory limits, and the list of missing codes.  Returns false
// (gkl_init then fails: A^T u has no other kernel) if the driver entry point
// or a step is unavailable or the packed buffer is not 16-byte aligned.
bool tc_prepare(gkl_handle* h) {
    if (h->tc_state != 0) return h->tc_state > 0;
    h->tc_state = -1;
    if ((reinterpret_cast<uintptr_t>(h->packed) & 15) != 0 || h->stride % 16 != 0) return false;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr)
        return false;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    alignas(64) CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)h->stride, (cuuint64_t)h->m};
    const cuuint64_t gstride[1] = {(cuuint64_t)h->stride};
    const cuuint32_t box[2] = {128u, (cuuint32_t)kBox};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(h->packed), gdim, gstride, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    static_assert(sizeof(CUtensorMap) == sizeof(h->tc_map), "tensor map size");
    memcpy(h->tc_map, &map, sizeof(map));
    if (cudaFuncSetAttribute(k_rmv_tc<kDigitsF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Fx<kDigitsF32>::kSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_rmv_tc<kDigitsF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Fx<kDigitsF64>::kSmem) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(k_miss_sum<int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMissSlots * (int)sizeof(int)) != cudaSuccess ||
        cudaFuncSetAttribute(k_miss_sum<long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMissSlots * (int)sizeof(long long)) != cudaSuccess)
        return false;
    // list of missing codes per (sample block, SNP), built once: counts, host prefix sum of the
    // padded counts, fill
    const int64_t m = h->m;
    const int64_t nb64 = std::max<int64_t>(1, (h->n + kMissBlock - 1) / kMissBlock);
    const int nb = (int)nb64;
    const int64_t nseg = m * nb;
    int* counts = nullptr;
    std::vector<int> hc((size_t)nseg);
    std::vector<int64_t> ho((size_t)nseg + 1);
    const unsigned wblocks = (unsigned)((nseg * 32 + 255) / 256);
    cudaError_t e = cudaMalloc(&counts, sizeof(int) * nseg);
    if (e == cudaSuccess) {
        k_miss_count<<<wblocks, 256, 0, h->stream>>>(h->packed, h->stride, h->n, m, nb, counts);
        e = cudaMemcpyAsync(hc.data(), counts, sizeof(int) * nseg, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (counts) cudaFree(counts);
    if (e != cudaSuccess) return false;
    ho[0] = 0;
    for (int64_t q = 0; q < nseg; ++q) ho[q + 1] = ho[q] + ((hc[q] + 7) & ~7);
    h->miss_nnz = ho[nseg];
    e = cudaMalloc(&h->miss_off, sizeof(int64_t) * (nseg + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->miss_idx, sizeof(uint16_t) * std::max<int64_t>(8, h->miss_nnz));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->miss_off, ho.data(), sizeof(int64_t) * (nseg + 1), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        k_miss_fill<<<wblocks, 256, 0, h->stream>>>(h->packed, h->stride, h->n, m, nb, h->miss_off, h->miss_idx);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return false;
    h->tc_state = 1;
    return true;
}

// Scale pass, digit image, the MMA kernel, the missing codes' sum and the
// finishing kernel; 11 digits for an FP32 product, 20 for an FP64 one.
template <typename T>
cudaError_t launch_rmatvec_tc(const gkl_handle* h, const T* u, T* x, void* scratch, const Sv* sv, const FinArgs* fa,
                              cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    constexpr int D = sizeof(T) == sizeof(float) ? kDigitsF32 : kDigitsF64;
    if (h->tc_state <= 0) return cudaErrorNotSupported;
    const TcPlan p = plan_tc(h);
    uint32_t* img = static_cast<uint32_t*>(scratch);
    using ZT = typename Fx<D>::Z;
    ZT* z = reinterpret_cast<ZT*>(reinterpret_cast<char*>(scratch) + al256(p.img_bytes));
    double* p1 = reinterpret_cast<double*>(reinterpret_cast<char*>(z) + al256(p.z_bytes));
    double* p3 = p1 + (size_t)p.nranges * h->m;
    double* aux = h->aux;  // dsc[4] | counter | partials of the scale pass; error word at kAuxErrOffset
    double* dsc = aux;
    unsigned* counter = reinterpret_cast<unsigned*>(aux + 4);
    double* part = aux + 8;
    int* err = reinterpret_cast<int*>(reinterpret_cast<char*>(aux) + kAuxErrOffset);
    cudaStream_t st = h->stream;
    const int sblocks = std::min(2 * h->num_sms, (int)((h->n + 255) / 256));
    GKL_DEBUG_SYNC(st, "before A^T u");
    k_u_scale<T><<<std::max(1, sblocks), 256, 0, st>>>(u, h->s, h->n, part, counter, dsc);
    GKL_DEBUG_SYNC(st, "k_u_scale");
    k_u_digits_f4<T, D><<<(unsigned)((p.nwords + 255) / 256), 256, 0, st>>>(u, h->s, h->n, p.nwords, dsc, img, z);
    GKL_DEBUG_SYNC(st, "k_u_digits_f4");
    alignas(64) CUtensorMap map;
    memcpy(&map, h->tc_map, sizeof(map));
    TcArgs a{img, p.nstages, p.range_stages, p.nranges, p.ntiles, h->m, dsc, p1, err};
    if (ev0) cudaEventRecord(ev0, st);
    k_rmv_tc<D><<<p.grid, kThreads, Fx<D>::kSmem, st>>>(map, a);
    if (ev1) cudaEventRecord(ev1, st);
    GKL_DEBUG_SYNC(st, "k_rmv_tc");
    k_miss_sum<ZT><<<(unsigned)p.miss_grid, kMissThreads, kMissSlots * sizeof(ZT), st>>>(
        h->miss_off, h->miss_idx, h->m, p.nb, z, (int64_t)p.nstages * kStageSamples, Fx<D>::kBits, dsc, p3, err);
    GKL_DEBUG_SYNC(st, "k_miss_sum");
    FinArgs f{};
    Sv s{};
    if (fa) f = *fa;
    if (sv) s = *sv;
    k_rmv_tc_fin<T><<<(unsigned)((h->m + 255) / 256), 256, 0, st>>>(p1, p3, p.nranges, p.nb, h->m, h->mu, h->d, h->w,
                                                                     dsc, x, f, s);
    GKL_DEBUG_SYNC(st, "k_rmv_tc_fin");
    if (nlaunch) *nlaunch = 5;
    return cudaGetLastError();
}

template cudaError_t launch_rmatvec_tc<float>(const gkl_handle*, const float*, float*, void*, const Sv*,
                                              const FinArgs*, cudaEvent_t, cudaEvent_t, int*);
template cudaError_t launch_rmatvec_tc<double>(const gkl_handle*, const double*, double*, void*, const Sv*,
                                               const FinArgs*, cudaEvent_t, cudaEvent_t, int*);

}  // namespace gkl
