// Blackwell tensor-core A^T u for the FP32 path:
//     x_j = d_j w_j [ sum_{i obs} g_ij u~_i - mu_j sum_{i obs} u~_i ],  u~ = s o u
// (A as defined in gkl.h; the per-step product of GKL bidiagonalisation,
// section 3 of arXiv:1808.03374).
//
// The contraction over samples is exact integer arithmetic on the 5th-generation
// tensor cores (tcgen05, kind::f8f6f4):
//  * u~ in fixed point: u~'_i = S sum_{p<7} delta_{p,i} 16^-(p+1) = S z_i 2^-28,
//    S = 2^e >= max|u~|, digits delta in [-16, 16] (exact in e4m3), z_i an
//    integer, |u~ - u~'| <= 2^-29 S;
//  * operand A (128 SNP rows x samples) is built in registers from the packed
//    codes and written to tensor memory.  Code t (bits 2t, 2t+1) of a byte is
//    read in place as e4m3: for t = 0, 2 (after one shift by 4 for t = 2) the
//    code sits in mantissa bits 0-1, H_a(c) = 1 + c/8 (bits 0x38 | c); for
//    t = 1, 3 it sits in bits 2-3 (mantissa MSB and exponent LSB), H_b(c) = 0.5,
//    0.75, 1.0, 1.5 for c = 0..3 -- affine, 0.5 + c/4, on the observed codes.
//    Five operations per 32-bit word of 16 codes;
//  * operand B = the digit matrix (K samples x N = 16 columns, 7 used) in shared
//    memory, 128-byte swizzled, K-major, the samples in the order the decode
//    produces (class a: t = 0, 2 first, then class b: t = 1, 3);
//  * eight FP32 accumulators in tensor memory (two classes x four K-step
//    residues, so that consecutive MMAs never wait on one another), each exact:
//    multiples of 1/8 below 2^21 for K-ranges of at most 64,000 samples;
//  * the missing codes are sparse and fixed per matrix: their sample indices are
//    listed once per SNP (CSR, built at the first use) and a gather kernel adds
//    the z_i of the listed samples, as exact 64-bit integers per class, to
//    Z_a and Z_b;
//  * with S_a, S_b the digit sums of the two classes,
//    sum_{obs} g u~' = S sum_p 16^-(p+1) (8 D_a[p] + 4 D_b[p]) - S sum_p 16^-(p+1) (8 S_a + 2 S_b)
//                      - S 2^-28 (3 Z_a + 4 Z_b),
//    sum_{missing} u~' = S 2^-28 (Z_a + Z_b).
// Data movement: per 512-sample stage one TMA box of 128 rows x 128 bytes
// (128-byte swizzle) brings the packed codes and one bulk copy the 8 KB digit
// tile into a shared-memory ring.  (The copy engine walks a box row by row; a
// 64-byte box width was measured at about 3 TB/s on this matrix.)  Warp roles
// per CTA: one copy producer, one MMA issuer, sixteen decode warps (four per
// TMEM sub-partition, one per 32-byte quarter of the stage) and four epilogue
// warps.  One persistent CTA per SM walks work items (128-row tile, K-range),
// the K-ranges of a tile consecutively so that each row is read as one
// contiguous run (a range-major order measured 40% slower: DRAM locality).
//
// Every wait is bounded (about two seconds of clock); a wait that runs out sets
// an error word that the host reads after the solve, and the kernel drains its
// copies and frees its tensor memory before it returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "epilogue.cuh"
#include "gkl_internal.cuh"
#include "tc_layout.cuh"
#include "tc_ptx.cuh"

namespace gkl {

namespace {
constexpr int kRows = 128;                 // SNP rows per tile = TMEM lanes = MMA M
constexpr int kStageSamples = 512;         // samples per pipeline stage
constexpr int kStageRowBytes = 128;        // packed bytes per row per stage
constexpr int kStages = 8;                 // shared-memory ring depth
constexpr int kPackedBytes = kRows * kStageRowBytes;  // 16 KB per stage
constexpr int kDigitBytes = 16 * kStageSamples;       // 8 KB: 16 digit rows x 512 samples (4 swizzle atoms)
constexpr int kAbuf = 2;                   // tensor-memory operand buffers (128 columns each)
constexpr int kDigits = 7;
constexpr int kMaxRangeStages = 125;       // 64,000 samples per K-range
constexpr int kThreads = 704;              // 22 warps
constexpr int kDecodeWarps = 16;
constexpr int kDecodeWarp0 = 2, kEpiWarp0 = kDecodeWarp0 + kDecodeWarps;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColD = 256;            // accumulators: 2 sets x 8 x 16 columns
constexpr int kBarOff = kStages * (kPackedBytes + kDigitBytes);
constexpr int kSmemBytes = 1024 + kBarOff + 1024;
// instruction descriptor: FP32 accumulate (bits 4-5 = 1), A = B = e4m3 (0), K-major
// A and B, N = 16 (bits 17-22: N >> 3), M = 128 (bits 24-28: M >> 4)
constexpr uint32_t kIdesc = (1u << 4) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
}  // namespace

// ---- PTX helpers (tc_ptx.cuh) ----------------------------------------------

using tc::bar_arrive;
using tc::bar_expect_tx;
using tc::bar_init;
using tc::bar_wait;
using tc::bulk_g2s;
using tc::desc_sw128;
using tc::mma_commit;
using tc::sm_addr;
using tc::tma_2d;
using tc::tmem_ld32;
using tc::tmem_st16;
__device__ __forceinline__ void mma_e4m3_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc) {
    tc::mma_f8_ts(d, a, bdesc, kIdesc, acc);
}
__device__ __forceinline__ void tc_fence_before() { tc::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { tc::fence_after(); }

// ---- scale of u~ -------------------------------------------------------------

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

// ---- digits of u~ -----------------------------------------------------------

// Position of sample `loc` (0..511) of a stage along the MMA's K axis.  Decode
// warp q (0..3) reads bytes 32q..32q+31 of each row: code words w = 0..7 of 16
// samples (sample 128q + 16w + 4b + t is code t of byte b).  Its operand words
// go to tensor-memory column 16q + 2w + (t >> 1) of the class-(t & 1) region
// (64 columns = 256 K bytes each), byte b of the column being K index
// 4 * column + b.
__host__ __device__ inline int tc_k_of_sample(int loc) {
    const int q = loc >> 7, w = (loc >> 4) & 7, b = (loc >> 2) & 3, t = loc & 3;
    return (t & 1) * 256 + 4 * (16 * q + 2 * w + (t >> 1)) + b;
}

// Byte offset of (digit row p, K index kk) inside a stage's 8 KB digit tile:
// four 128-byte-swizzled atoms of 16 rows x 128 K each.
__host__ __device__ inline int tc_digit_offset(int p, int kk) {
    const int atom = kk >> 7, b = kk & 127;
    return atom * 2048 + p * 128 + ((((b >> 4) ^ (p & 7))) << 4) + (b & 15);
}

// One block per stage (512 samples): digits in e4m3 into the stage's tile, z_i
// (int32) into z[], and the stage's digit sums per operand class (exact
// integers) into cs[stage][16]: [class a: p = 0..6 | class b: 8 + p].
__global__ void __launch_bounds__(512) k_u_digits_tc(const float* __restrict__ u, const float* __restrict__ s,
                                                      int64_t n, const double* __restrict__ dsc,
                                                      uint8_t* __restrict__ dig, int* __restrict__ cs,
                                                      int* __restrict__ zout) {
    const int st = blockIdx.x, loc = threadIdx.x;
    const int64_t i = (int64_t)st * kStageSamples + loc;
    double x = 0.0;
    if (i < n) x = (double)u[i] * (s ? (double)s[i] : 1.0) * dsc[1];
    uint8_t* tile = dig + (size_t)st * kDigitBytes;
    const int kk = tc_k_of_sample(loc);
    int sums[kDigits];
    int z = 0;
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        int dg = 0;
        if (p < kDigits) {
            x *= 16.0;
            const double rd = rint(x);
            x -= rd;
            dg = (int)rd;
            sums[p] = dg;
            z = 16 * z + dg;
        }
        tile[tc_digit_offset(p, kk)] = (uint8_t)__nv_cvt_float_to_fp8((float)dg, __NV_SATFINITE, __NV_E4M3);
    }
    zout[i] = z;
    // lanes of one warp alternate classes (t = loc & 3): reduce even and odd lanes separately
    __shared__ int red[16][2][kDigits];
    const int cls = loc & 1;
#pragma unroll
    for (int p = 0; p < kDigits; ++p) {
        int v = sums[p];
        for (int o = 16; o > 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((loc & 31) < 2) red[loc >> 5][cls][p] = v;
    }
    __syncthreads();
    if (loc < 2 * kDigits) {
        const int c = loc / kDigits, p = loc % kDigits;
        int t = 0;
        for (int w = 0; w < 16; ++w) t += red[w][c][p];
        cs[(size_t)st * 16 + 8 * c + p] = t;
    }
}

// ---- main kernel ------------------------------------------------------------

struct TcArgs {
    const uint8_t* dig;  // nstages x 8 KB digit tiles
    const int* cs;       // nstages x 16 digit sums per class
    int nstages, range_stages, nranges, ntiles;
    int64_t m;
    const double* dsc;   // {S, 1/S, sum u~}
    double* p1;          // nranges x m: S sum_p 16^-(p+1) (8 D_a + 4 D_b) over the range (range 0: - offsets)
    double* p3;          // nranges x m: 0 (range 0: sum u~ - sum u~'); the missing terms are added later
    int* err;            // set to a nonzero code if a wait ran out
};

__global__ void __launch_bounds__(kThreads, 1) k_rmv_tc(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = sm_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sbase = smem_raw + (base - raw);
    const uint32_t sPacked = base, sDig = base + kStages * kPackedBytes, sBar = base + kBarOff;
    auto full = [&](int s) { return sBar + 8u * s; };
    auto empty = [&](int s) { return sBar + 8u * (kStages + s); };
    auto afull = [&](int t) { return sBar + 8u * (2 * kStages + t); };
    auto aempty = [&](int t) { return sBar + 8u * (2 * kStages + kAbuf + t); };
    auto dfull = [&](int q) { return sBar + 8u * (2 * kStages + 2 * kAbuf + q); };
    auto dempty = [&](int q) { return sBar + 8u * (2 * kStages + 2 * kAbuf + 2 + q); };
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sbase + kBarOff + 384);
    double* s_csum = reinterpret_cast<double*>(sbase + kBarOff + 392);     // [2]
    long long* s_c = reinterpret_cast<long long*>(sbase + kBarOff + 512);  // [4 warps][2][kDigits]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sm_addr(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(full(s), 1);
            bar_init(empty(s), 1);
        }
        for (int t = 0; t < kAbuf; ++t) {
            bar_init(afull(t), kDecodeWarps);
            bar_init(aempty(t), 1);
        }
        for (int q = 0; q < 2; ++q) {
            bar_init(dfull(q), 1);
            bar_init(dempty(q), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nitems = a.ntiles * a.nranges;
    auto fail = [&](int code) { atomicCAS(a.err, 0, code); };

    if (warp == 0) {
        // ---- copy producer: per stage one TMA box (packed) + one bulk copy (digits)
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int tile = item / a.nranges, range = item % a.nranges;
                const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
                for (int k = 0; k < nst; ++k, ++it) {
                    const int s = (int)(it % kStages);
                    if (!bar_wait(empty(s), ((it / kStages) & 1u) ^ 1u)) {
                        fail(1);
                        ok = false;
                        break;
                    }
                    bar_expect_tx(full(s), kPackedBytes + kDigitBytes);
                    tma_2d(sPacked + s * kPackedBytes, &tmap, kStageRowBytes * (st0 + k), tile * kRows, full(s));
                    bulk_g2s(sDig + s * kDigitBytes, a.dig + (size_t)(st0 + k) * kDigitBytes, kDigitBytes, full(s));
                }
            }
            // drain: every issued copy has landed before the CTA may exit
            const uint32_t first = it > (uint32_t)kStages ? it - kStages : 0u;
            for (uint32_t q = first; q < it; ++q)
                if (!bar_wait(full((int)(q % kStages)), (q / kStages) & 1u)) fail(2);
        }
    } else if (warp == 1) {
        // ---- MMA issuer: per stage 16 MMAs (class a, b x eight 32-byte K-steps) into 8 accumulators.
        // The decode warps arrive on afull only after they have seen the stage's copies land.
        if (lane == 0) {
            uint32_t it = 0, li = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
                const int range = item % a.nranges;
                const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
                const uint32_t acc = li & 1u;
                if (!bar_wait(dempty(acc), ((li >> 1) & 1u) ^ 1u)) {
                    fail(3);
                    break;
                }
                tc_fence_after();
                const uint32_t dbase = tmem + kColD + 128u * acc;
                for (int k = 0; k < nst; ++k, ++it) {
                    const int s = (int)(it % kStages), t = (int)(it % kAbuf);
                    if (!bar_wait(afull(t), (it / kAbuf) & 1u)) {
                        fail(4);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t aA = tmem + 128u * t;
                    const uint64_t d0 = desc_sw128(sDig + s * kDigitBytes);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        // K-step i: 32 bytes = 8 columns; descriptor address in 16-byte units
                        // (+2 per 32 bytes, +128 per 2 KB atom); atoms 0-1 class a, 2-3 class b
                        const uint32_t acc_in = (k != 0) || (i >= 4);
                        const uint64_t dd = d0 + (uint64_t)(128 * (i >> 2) + 2 * (i & 3));
                        mma_e4m3_ts(dbase + 16u * (i & 3), aA + 8u * i, dd, acc_in);
                        mma_e4m3_ts(dbase + 64u + 16u * (i & 3), aA + 64u + 8u * i, dd + 256, acc_in);
                    }
                    mma_commit(aempty(t));
                    mma_commit(empty(s));
                }
                if (ok) mma_commit(dfull(acc));
            }
            // drain: the last commit covers every MMA issued by this thread
            if (it > 0) {
                const uint32_t q = it - 1;
                if (!bar_wait(empty((int)(q % kStages)), (q / kStages) & 1u)) fail(5);
            }
        }
    } else if (warp < kEpiWarp0) {
        // ---- decode: row = lane of this warp's TMEM sub-partition, 32-byte quarter q of the stage
        const int sub = warp & 3, q = (warp - kDecodeWarp0) >> 2;
        const int row = 32 * sub + lane;
        const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
        uint32_t it = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int range = item % a.nranges;
            const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
            for (int k = 0; k < nst; ++k, ++it) {
                const int s = (int)(it % kStages), t = (int)(it % kAbuf);
                if (!bar_wait(full(s), (it / kStages) & 1u)) {
                    fail(6);
                    ok = false;
                    break;
                }
                // 128-byte swizzle of the TMA tile: 16-byte chunk c of row r sits at chunk c ^ (r & 7)
                const uint8_t* rp = sbase + s * kPackedBytes + row * kStageRowBytes;
                const uint4 q0 = *reinterpret_cast<const uint4*>(rp + (((2 * q) ^ (row & 7)) << 4));
                const uint4 q1 = *reinterpret_cast<const uint4*>(rp + (((2 * q + 1) ^ (row & 7)) << 4));
                const uint32_t W[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                uint32_t ha[16], hb[16];
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const uint32_t Wv = W[w], W4 = Wv >> 4;
                    ha[2 * w] = (Wv & 0x03030303u) | 0x38383838u;
                    ha[2 * w + 1] = (W4 & 0x03030303u) | 0x38383838u;
                    hb[2 * w] = (Wv & 0x0C0C0C0Cu) | 0x30303030u;
                    hb[2 * w + 1] = (W4 & 0x0C0C0C0Cu) | 0x30303030u;
                }
                if (!bar_wait(aempty(t), ((it / kAbuf) & 1u) ^ 1u)) {
                    fail(7);
                    ok = false;
                    break;
                }
                const uint32_t col = tmem + lane_base + 128u * t + 16u * q;
                tmem_st16(col, ha);
                tmem_st16(col + 64u, hb);
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) bar_arrive(afull(t));
            }
        }
    } else {
        // ---- epilogue
        const int sub = warp & 3, et = threadIdx.x - 32 * kEpiWarp0;
        const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
        // class digit sums over all samples: s_csum[0] = sum_p 16^-(p+1) (S_a + S_b) = sum u~'/S,
        // s_csum[1] = sum_p 16^-(p+1) (8 S_a + 2 S_b), the offsets of H_a and H_b, exactly
        {
            long long c[2][kDigits];
#pragma unroll
            for (int p = 0; p < kDigits; ++p) c[0][p] = c[1][p] = 0;
            for (int st = et; st < a.nstages; st += 128)
#pragma unroll
                for (int p = 0; p < kDigits; ++p) {
                    c[0][p] += a.cs[(size_t)st * 16 + p];
                    c[1][p] += a.cs[(size_t)st * 16 + 8 + p];
                }
#pragma unroll
            for (int cl = 0; cl < 2; ++cl)
#pragma unroll
                for (int p = 0; p < kDigits; ++p) {
                    long long v = c[cl][p];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) s_c[((warp - kEpiWarp0) * 2 + cl) * kDigits + p] = v;
                }
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        if (et == 0) {
            double t0 = 0.0, t1 = 0.0;
            for (int p = kDigits - 1; p >= 0; --p) {
                long long ca = 0, cb = 0;
                for (int w = 0; w < 4; ++w) {
                    ca += s_c[(w * 2 + 0) * kDigits + p];
                    cb += s_c[(w * 2 + 1) * kDigits + p];
                }
                t0 += ldexp((double)(ca + cb), -4 * (p + 1));
                t1 += ldexp((double)(8 * ca + 2 * cb), -4 * (p + 1));
            }
            s_csum[0] = t0;
            s_csum[1] = t1;
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        const double S = a.dsc[0], usum = S * s_csum[0], hoff = S * s_csum[1];
        uint32_t li = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++li) {
            const int tile = item / a.nranges, range = item % a.nranges;
            const uint32_t acc = li & 1u;
            if (!bar_wait(dfull(acc), (li >> 1) & 1u)) {
                fail(8);
                break;
            }
            tc_fence_after();
            const int64_t j = (int64_t)tile * kRows + 32 * sub + lane;
            double hs = 0.0;
            {
                uint32_t r[32];
#pragma unroll
                for (int h = 0; h < 4; ++h) {  // accumulators 2h, 2h+1: class a (h < 2) or b
                    tmem_ld32(tmem + lane_base + kColD + 128u * acc + 32u * h, r);
                    const double wgt = h < 2 ? 8.0 : 4.0;
#pragma unroll
                    for (int p = kDigits - 1; p >= 0; --p)
                        hs += ldexp(wgt, -4 * (p + 1)) *
                              ((double)__uint_as_float(r[p]) + (double)__uint_as_float(r[16 + p]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(dempty(acc));
            if (j < a.m) {
                double P1 = S * hs, P3 = 0.0;
                if (range == 0) {
                    P1 -= hoff;                // the offsets of H_a and H_b over all samples
                    P3 += a.dsc[2] - usum;     // so that sum u~ - sum_r p3 = sum_{obs} u~'
                }
                a.p1[(int64_t)range * a.m + j] = P1;
                a.p3[(int64_t)range * a.m + j] = P3;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
    }
}

// ---- missing-code list (CSR) and the per-product gather ----------------------

// counts[j] = missing codes of SNP j among samples 0..n-1; one warp per SNP.
__global__ void __launch_bounds__(256) k_miss_count(const uint8_t* __restrict__ packed, int64_t stride, int64_t n,
                                                     int64_t m, int* __restrict__ counts) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= m) return;
    const uint32_t* row = reinterpret_cast<const uint32_t*>(packed + j * stride);
    const int64_t words = (n + 15) / 16;
    int c = 0;
    for (int64_t wd = lane; wd < words; wd += 32) {
        uint32_t Y = row[wd] & (row[wd] >> 1) & 0x55555555u;
        const int64_t valid = n - wd * 16;  // samples of this word below n
        if (valid < 16) Y &= (1u << (2 * valid)) - 1u;
        c += __popc(Y);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) counts[j] = c;
}

// idx[off[j] ..] = the missing sample indices of SNP j, ascending; one warp per SNP.
__global__ void __launch_bounds__(256) k_miss_fill(const uint8_t* __restrict__ packed, int64_t stride, int64_t n,
                                                    int64_t m, const int64_t* __restrict__ off,
                                                    uint32_t* __restrict__ idx) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= m) return;
    const uint32_t* row = reinterpret_cast<const uint32_t*>(packed + j * stride);
    const int64_t words = (n + 15) / 16;
    int64_t pos = off[j];
    for (int64_t w0 = 0; w0 < words; w0 += 32) {
        const int64_t wd = w0 + lane;
        uint32_t Y = 0;
        if (wd < words) {
            Y = row[wd] & (row[wd] >> 1) & 0x55555555u;
            const int64_t valid = n - wd * 16;
            if (valid < 16) Y &= (1u << (2 * valid)) - 1u;
        }
        const int c = __popc(Y);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        int64_t p = pos + incl - c;
        while (Y) {
            const int bit = __ffs(Y) - 1;
            Y &= Y - 1u;
            idx[p++] = (uint32_t)(wd * 16 + (bit >> 1));
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Missing terms of A^T u (no cross-block synchronisation): eight lanes per SNP
// j, four SNPs per warp, eight list entries in flight per lane (the kernel is
// bound by memory latency times the number of warp waves).  Z_a, Z_b = sums of
// z_i over the listed samples of class a (i even) and b (i odd), exact in 64-bit
// integers; p3[j] += S 2^-28 (Z_a + Z_b) and, for the operand of k_rmv_tc
// (affine in the code, so a missing code contributes 3/8 or 3/4 of z_i),
// p1[j] -= S 2^-28 (3 Z_a + 4 Z_b) (range-0 partials).
__global__ void __launch_bounds__(256) k_miss_gather(const int64_t* __restrict__ off, const uint32_t* __restrict__ idx,
                                                      int64_t m, const int* __restrict__ z,
                                                      const double* __restrict__ dsc, double* __restrict__ p1,
                                                      double* __restrict__ p3, int affine) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sl = threadIdx.x & 7;
    long long za = 0, zb = 0;
    if (j < m) {
        const int64_t e1 = off[j + 1];
        for (int64_t e = off[j] + sl; e < e1; e += 64) {
            uint32_t ii[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) ii[u] = e + 8 * u < e1 ? idx[e + 8 * u] : 0xFFFFFFFFu;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (ii[u] != 0xFFFFFFFFu) {
                    const long long v = z[ii[u]];
                    if (ii[u] & 1u)
                        zb += v;
                    else
                        za += v;
                }
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        za += __shfl_xor_sync(0xffffffffu, za, o);
        zb += __shfl_xor_sync(0xffffffffu, zb, o);
    }
    if (j < m && sl == 0 && (za | zb)) {
        const double zs = ldexp(dsc[0], -28);
        if (affine) p1[j] -= zs * (double)(3 * za + 4 * zb);
        p3[j] += zs * (double)(za + zb);
    }
}

// ---- finishing kernel ----------------------------------------------------------

// Final combination over sample blocks (fixed order), then the solver epilogue.
__global__ void __launch_bounds__(256) k_rmv_tc_fin(const double* __restrict__ p1, const double* __restrict__ p3,
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

// ---- host side --------------------------------------------------------------

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct TcPlan {
    int nstages, range_stages, nranges, ntiles, grid;
    size_t dig_bytes, cs_bytes, z_bytes, part_bytes;
};

static TcPlan plan_tc(const gkl_handle* h) {
    TcPlan p;
    p.nstages = (int)((h->stride + kStageRowBytes - 1) / kStageRowBytes);
    p.ntiles = (int)((h->m + kRows - 1) / kRows);
    const int sms = std::max(1, h->num_sms);
    const int nr0 = (p.nstages + kMaxRangeStages - 1) / kMaxRangeStages;
    // K-ranges: at most 64,000 samples each; more ranges only where they even out
    // the last wave of work items over the SMs by a few percent
    int best = nr0;
    double best_eff = 0.0;
    for (int nr = nr0; nr <= std::min(p.nstages, nr0 + 7); ++nr) {
        const int rs = (p.nstages + nr - 1) / nr, nranges = (p.nstages + rs - 1) / rs;
        const double items = (double)p.ntiles * nranges;
        const double waves = std::ceil(items / sms);
        const double eff = items / (waves * sms);
        if (eff > best_eff + 0.03) {
            best_eff = eff;
            best = nr;
        }
    }
    p.range_stages = (p.nstages + best - 1) / best;
    p.nranges = (p.nstages + p.range_stages - 1) / p.range_stages;
    p.grid = (int)std::min<int64_t>((int64_t)p.ntiles * p.nranges, sms);
    p.dig_bytes = (size_t)p.nstages * kDigitBytes;
    p.cs_bytes = (size_t)p.nstages * 16 * sizeof(int);
    p.z_bytes = (size_t)p.nstages * kStageSamples * sizeof(int);
    p.part_bytes = 2 * (size_t)p.nranges * (size_t)h->m * sizeof(double);
    return p;
}

size_t rmv_tc_scratch_bytes(const gkl_handle* h) {
    const TcPlan p = plan_tc(h);
    return p.dig_bytes + al256(p.cs_bytes) + al256(p.z_bytes) + p.part_bytes + 256;
}


// Prepares the tensor-core path for a handle: the TMA descriptor of the packed
// matrix (128-byte x 128-row boxes, 128-byte swizzle), the kernel's shared-memory
// limit and the list of missing codes per SNP.  Returns false (gkl_init then
// fails: the FP32 A^T u has no other kernel) if the driver entry point or a
// step is unavailable or the packed buffer is not 16-byte aligned.
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
    const cuuint32_t box[2] = {(cuuint32_t)kStageRowBytes, (cuuint32_t)kRows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(h->packed), gdim, gstride, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    static_assert(sizeof(CUtensorMap) == sizeof(h->tc_map), "tensor map size");
    memcpy(h->tc_map, &map, sizeof(map));
    if (cudaFuncSetAttribute(k_rmv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
        return false;
    // list of missing codes per SNP (CSR), built once: counts, host prefix sum, fill
    const int64_t m = h->m;
    int* counts = nullptr;
    std::vector<int> hc((size_t)m);
    std::vector<int64_t> ho((size_t)m + 1);
    const unsigned wblocks = (unsigned)((m * 32 + 255) / 256);
    cudaError_t e = cudaMalloc(&counts, sizeof(int) * m);
    if (e == cudaSuccess) {
        k_miss_count<<<wblocks, 256, 0, h->stream>>>(h->packed, h->stride, h->n, m, counts);
        e = cudaMemcpyAsync(hc.data(), counts, sizeof(int) * m, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (counts) cudaFree(counts);
    if (e != cudaSuccess) return false;
    ho[0] = 0;
    for (int64_t j = 0; j < m; ++j) ho[j + 1] = ho[j] + hc[j];
    h->miss_nnz = ho[m];
    e = cudaMalloc(&h->miss_off, sizeof(int64_t) * (m + 1));
    if (e == cudaSuccess) e = cudaMalloc(&h->miss_idx, sizeof(uint32_t) * std::max<int64_t>(1, h->miss_nnz));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->miss_off, ho.data(), sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        k_miss_fill<<<wblocks, 256, 0, h->stream>>>(h->packed, h->stride, h->n, m, h->miss_off, h->miss_idx);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return false;
    h->tc_state = 1;
    return true;
}

cudaError_t launch_rmatvec_tc(const gkl_handle* h, const float* u, float* x, void* scratch, const Sv* sv,
                              const FinArgs* fa, cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    const TcPlan p = plan_tc(h);
    uint8_t* dig = static_cast<uint8_t*>(scratch);
    int* cs = reinterpret_cast<int*>(dig + p.dig_bytes);
    int* z = reinterpret_cast<int*>(reinterpret_cast<char*>(cs) + ((p.cs_bytes + 255) & ~(size_t)255));
    double* p1 = reinterpret_cast<double*>(reinterpret_cast<char*>(z) + ((p.z_bytes + 255) & ~(size_t)255));
    double* p3 = p1 + (size_t)p.nranges * h->m;
    double* aux = h->aux;  // dsc[4] | counter | partials of the scale pass; error word at kAuxErrOffset
    double* dsc = aux;
    unsigned* counter = reinterpret_cast<unsigned*>(aux + 4);
    double* part = aux + 8;
    int* err = reinterpret_cast<int*>(reinterpret_cast<char*>(aux) + kAuxErrOffset);
    cudaStream_t st = h->stream;
    const int sblocks = std::min(2 * h->num_sms, (int)((h->n + 255) / 256));
    k_u_scale<<<std::max(1, sblocks), 256, 0, st>>>(u, h->s, h->n, part, counter, dsc);
    k_u_digits_tc<<<p.nstages, kStageSamples, 0, st>>>(u, h->s, h->n, dsc, dig, cs, z);
    alignas(64) CUtensorMap map;
    memcpy(&map, h->tc_map, sizeof(map));
    TcArgs a{dig, cs, p.nstages, p.range_stages, p.nranges, p.ntiles, h->m, dsc, p1, p3, err};
    if (ev0) cudaEventRecord(ev0, st);
    k_rmv_tc<<<p.grid, kThreads, kSmemBytes, st>>>(map, a);
    if (ev1) cudaEventRecord(ev1, st);
    k_miss_gather<<<(unsigned)((h->m * 8 + 255) / 256), 256, 0, st>>>(h->miss_off, h->miss_idx, h->m, z, dsc, p1,
                                                                       p3, 1);
    FinArgs f{};
    Sv s{};
    if (fa) f = *fa;
    if (sv) s = *sv;
    k_rmv_tc_fin<<<(unsigned)((h->m + 255) / 256), 256, 0, st>>>(p1, p3, p.nranges, h->m, h->mu, h->d, h->w, dsc, x,
                                                                    f, s);
    if (nlaunch) *nlaunch = 5;
    return cudaGetLastError();
}

}  // namespace gkl
