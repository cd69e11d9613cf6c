// Blackwell tensor-core A^T u for the FP32 path:
//     x_j = d_j w_j [ sum_{i obs} g_ij u~_i - mu_j sum_{i obs} u~_i ],  u~ = s o u
// (A as defined in gkl.h; the per-step product of GKL bidiagonalisation,
// section 3 of arXiv:1808.03374).
//
// The contraction over samples is exact integer arithmetic on the 5th-generation
// tensor cores (tcgen05, kind::f8f6f4):
//  * u~ in fixed point: u~'_i = S sum_{p<7} delta_{p,i} 16^-(p+1), S = 2^e >= max|u~|,
//    digits delta in [-16, 16] (exact in e4m3), |u~ - u~'| <= 2^-29 S;
//  * operand A (128 SNP rows x samples) is built in registers from the packed
//    codes and written to tensor memory: H(c) = 1 + c/8 (e4m3 bits 0x38 | c, one
//    LOP3 per four codes) and M(c) = 2^-6 [c == 3] (e4m3 bits 0x08);
//  * operand B = the digit matrix (K samples x N = 16 columns, 7 used) in shared
//    memory, 128-byte swizzled, K-major;
//  * D_H[p] = sum_i (1 + c_i/8) delta_{p,i} and D_M[p] = 2^-6 sum_{i missing} delta_{p,i}
//    accumulate in FP32 in tensor memory, exactly: every term is a multiple of
//    2^-6 and a K-range of at most 64,000 samples keeps |D| * 64 below 2^24;
//  * sum_{i obs} g_i delta_{p,i} = 8 (D_H[p] - sum_i delta_{p,i}) - 192 D_M[p] and
//    sum_{i missing} delta_{p,i} = 64 D_M[p].
// The packed tiles (128 rows x 64 bytes = 256 samples) arrive by TMA into a
// shared-memory ring; the digit tiles by bulk copy.  Warp roles per CTA: one TMA
// producer, one MMA issuer, eight decode warps (two per TMEM sub-partition, one
// per half of the 256-sample stage) and four epilogue warps.  One persistent CTA
// per SM walks work items (128-row tile, K-range).
//
// Every wait is bounded (about two seconds of clock); a wait that runs out sets
// an error word that the host reads after the solve, and the kernel drains its
// copies and frees its tensor memory before it returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>

#include "epilogue.cuh"
#include "gkl_internal.cuh"

namespace gkl {

namespace {
constexpr int kRows = 128;                 // SNP rows per tile = TMEM lanes = MMA M
constexpr int kStageSamples = 256;         // samples per pipeline stage
constexpr int kStageRowBytes = 64;         // packed bytes per row per stage
constexpr int kStages = 10;                // shared-memory ring depth
constexpr int kAbuf = 3;                   // tensor-memory operand buffers
constexpr int kPackedBytes = kRows * kStageRowBytes;  // 8 KB per stage
constexpr int kDigitBytes = 16 * kStageSamples;       // 4 KB per stage: 16 digit rows x 256 samples
constexpr int kDigits = 7;
constexpr int kMaxRangeStages = 250;       // 64,000 samples per K-range
constexpr int kThreads = 448;              // 14 warps
constexpr int kDecodeWarp0 = 2, kEpiWarp0 = 10;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColD = 384;            // accumulators: 2 x (16 H + 16 M) columns
constexpr int kBarOff = kStages * (kPackedBytes + kDigitBytes);
constexpr int kSmemBytes = 1024 + kBarOff + 512;
// instruction descriptor: FP32 accumulate (bits 4-5 = 1), A = B = e4m3 (0), K-major
// A and B, N = 16 (bits 17-22: N >> 3), M = 128 (bits 24-28: M >> 4)
constexpr uint32_t kIdesc = (1u << 4) | ((16u >> 3) << 17) | ((128u >> 4) << 24);
constexpr long long kWaitCycles = 4000000000LL;  // about two seconds at the boost clock
}  // namespace

// ---- PTX helpers ------------------------------------------------------------

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
}
// Bounded wait for the phase of parity `par` to complete.
__device__ __forceinline__ bool bar_wait(uint32_t a, uint32_t par) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p;}\n"
            : "=r"(ok)
            : "r"(a), "r"(par)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void mma_e4m3_ts(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;}\n" ::"r"(d),
        "r"(a), "l"(bdesc), "r"(kIdesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// ---- digits of u~ -----------------------------------------------------------

// Position of sample `loc` (0..255) of a stage along the MMA's K axis.  The
// decode turns a 32-bit code word (16 samples; code t of byte b is sample 4b+t)
// into four operand words H_t holding samples t, 4+t, 8+t, 12+t, so K index
// 16w + 4t + b carries sample 16w + 4b + t: a 4x4 transpose inside every
// aligned group of 16 samples.
__host__ __device__ inline int tc_k_of_sample(int loc) { return (loc & ~15) | ((loc & 3) << 2) | ((loc >> 2) & 3); }

// Byte offset of (digit row p, K index kk) inside a stage's 4 KB digit tile:
// two 128-byte-swizzled atoms of 16 rows x 128 K each.
__host__ __device__ inline int tc_digit_offset(int p, int kk) {
    const int atom = kk >> 7, b = kk & 127;
    return atom * 2048 + p * 128 + ((((b >> 4) ^ (p & 7))) << 4) + (b & 15);
}

// One block per stage (256 samples): digits in e4m3 into the stage's tile and
// the stage's digit sums (exact integers) into cs[stage][p].
__global__ void __launch_bounds__(256) k_u_digits_tc(const float* __restrict__ u, const float* __restrict__ s,
                                                      int64_t n, const double* __restrict__ dsc,
                                                      uint8_t* __restrict__ dig, int* __restrict__ cs) {
    const int st = blockIdx.x, loc = threadIdx.x;
    const int64_t i = (int64_t)st * kStageSamples + loc;
    double x = 0.0;
    if (i < n) x = (double)u[i] * (s ? (double)s[i] : 1.0) * dsc[1];
    uint8_t* tile = dig + (size_t)st * kDigitBytes;
    const int kk = tc_k_of_sample(loc);
    int sums[kDigits];
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        int dg = 0;
        if (p < kDigits) {
            x *= 16.0;
            const double rd = rint(x);
            x -= rd;
            dg = (int)rd;
            sums[p] = dg;
        }
        tile[tc_digit_offset(p, kk)] = (uint8_t)__nv_cvt_float_to_fp8((float)dg, __NV_SATFINITE, __NV_E4M3);
    }
    __shared__ int red[8][kDigits];
#pragma unroll
    for (int p = 0; p < kDigits; ++p) {
        int v = sums[p];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((loc & 31) == 0) red[loc >> 5][p] = v;
    }
    __syncthreads();
    if (loc < kDigits) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += red[w][loc];
        cs[(size_t)st * 8 + loc] = t;
    }
}

// ---- main kernel ------------------------------------------------------------

struct TcArgs {
    const uint8_t* dig;  // nstages x 4 KB digit tiles
    const int* cs;       // nstages x 8 digit sums
    int nstages, range_stages, nranges, ntiles;
    int64_t m;
    const double* dsc;   // {S, 1/S, sum u~}
    double* p1;          // nranges x m: S sum_p 16^-(p+1) sum_{i obs} g_i delta_{p,i} (range 0 carries the offset)
    double* p3;          // nranges x m: S sum_p 16^-(p+1) sum_{i missing} delta_{p,i} (+ correction in range 0)
    int* err;            // set to a nonzero code if a wait ran out
};

// Operand words of one 32-bit code word W (16 samples): H_t = 0x38 | code_t and
// M_t = 0x08 [code_t == 3] in each byte, for code positions t = 0..3.
__device__ __forceinline__ void decode_word(uint32_t W, uint32_t* H, uint32_t* M) {
    const uint32_t w2 = W >> 2, w4 = W >> 4, w6 = W >> 6;
    H[0] = (W & 0x03030303u) | 0x38383838u;
    H[1] = (w2 & 0x03030303u) | 0x38383838u;
    H[2] = (w4 & 0x03030303u) | 0x38383838u;
    H[3] = (w6 & 0x03030303u) | 0x38383838u;
    // [code_t == 3] = bit 2t & bit 2t+1 of each byte, moved to bit 3
    M[0] = (W << 3) & (W << 2) & 0x08080808u;
    M[1] = (W << 1) & W & 0x08080808u;
    M[2] = (W >> 1) & w2 & 0x08080808u;
    M[3] = (W >> 3) & w4 & 0x08080808u;
}

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
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sbase + kBarOff + 256);
    int* s_fail = reinterpret_cast<int*>(sbase + kBarOff + 260);
    double* s_csum = reinterpret_cast<double*>(sbase + kBarOff + 264);

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
            bar_init(afull(t), 8);
            bar_init(aempty(t), 1);
        }
        for (int q = 0; q < 2; ++q) {
            bar_init(dfull(q), 1);
            bar_init(dempty(q), 4);
        }
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nitems = a.ntiles * a.nranges;
    auto fail = [&](int code) {
        *s_fail = 1;
        atomicCAS(a.err, 0, code);
    };

    if (warp == 0) {
        // ---- TMA producer
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int tile = item % a.ntiles, range = item / a.ntiles;
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
        // ---- MMA issuer
        if (lane == 0) {
            uint32_t it = 0, li = 0;
            bool ok = true;
            for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++li) {
                const int range = item / a.ntiles;
                const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
                const uint32_t acc = li & 1u;
                if (!bar_wait(dempty(acc), ((li >> 1) & 1u) ^ 1u)) {
                    fail(3);
                    break;
                }
                tc_fence_after();
                const uint32_t dH = tmem + kColD + 32u * acc, dM = dH + 16u;
                for (int k = 0; k < nst; ++k, ++it) {
                    const int s = (int)(it % kStages), t = (int)(it % kAbuf);
                    if (!bar_wait(afull(t), (it / kAbuf) & 1u) || !bar_wait(full(s), (it / kStages) & 1u)) {
                        fail(4);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t aH = tmem + 128u * t, aM = aH + 64u;
                    const uint32_t bs = sDig + s * kDigitBytes;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        mma_e4m3_ts(dH, aH + 8u * q, desc_sw128(bs + (q >> 2) * 2048 + 32 * (q & 3)), (k | q) != 0);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        mma_e4m3_ts(dM, aM + 8u * q, desc_sw128(bs + (q >> 2) * 2048 + 32 * (q & 3)), (k | q) != 0);
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
        // ---- decode: row = lane of this warp's TMEM sub-partition, half of the stage
        const int sub = warp & 3, half = (warp - kDecodeWarp0) >> 2;
        const int row = 32 * sub + lane;
        const uint32_t lane_base = (uint32_t)(32 * sub) << 16;
        uint32_t it = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int range = item / a.ntiles;
            const int st0 = range * a.range_stages, nst = min(a.range_stages, a.nstages - st0);
            for (int k = 0; k < nst; ++k, ++it) {
                const int s = (int)(it % kStages), t = (int)(it % kAbuf);
                if (!bar_wait(full(s), (it / kStages) & 1u) || !bar_wait(aempty(t), ((it / kAbuf) & 1u) ^ 1u)) {
                    fail(6);
                    ok = false;
                    break;
                }
                // 64-byte swizzle of the TMA tile: chunk c of row r sits at chunk c ^ ((r >> 1) & 3)
                const uint8_t* rp = sbase + s * kPackedBytes + row * kStageRowBytes;
                const int sw = (row >> 1) & 3;
                const uint4 q0 = *reinterpret_cast<const uint4*>(rp + (((2 * half) ^ sw) << 4));
                const uint4 q1 = *reinterpret_cast<const uint4*>(rp + (((2 * half + 1) ^ sw) << 4));
                const uint32_t W[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
                uint32_t H[32], M[32];
#pragma unroll
                for (int w = 0; w < 8; ++w) decode_word(W[w], H + 4 * w, M + 4 * w);
                const uint32_t col = tmem + lane_base + 128u * t + 32u * half;
                tmem_st32(col, H);
                tmem_st32(col + 64u, M);
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
        // sum over all samples of u~' / S = sum_p 16^-(p+1) sum_i delta_{p,i}, exactly
        long long* s_c = reinterpret_cast<long long*>(sbase + kBarOff + 272);  // [4][kDigits]
        {
            long long c[kDigits] = {0, 0, 0, 0, 0, 0, 0};
            for (int st = et; st < a.nstages; st += 128)
#pragma unroll
                for (int p = 0; p < kDigits; ++p) c[p] += a.cs[(size_t)st * 8 + p];
#pragma unroll
            for (int p = 0; p < kDigits; ++p) {
                for (int o = 16; o > 0; o >>= 1) c[p] += __shfl_xor_sync(0xffffffffu, c[p], o);
                if (lane == 0) s_c[(warp - kEpiWarp0) * kDigits + p] = c[p];
            }
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        if (et == 0) {
            double t = 0.0;
            for (int p = kDigits - 1; p >= 0; --p) {
                const long long c = s_c[p] + s_c[kDigits + p] + s_c[2 * kDigits + p] + s_c[3 * kDigits + p];
                t += ldexp((double)c, -4 * (p + 1));
            }
            *s_csum = t;
        }
        asm volatile("bar.sync 1, 128;\n" ::: "memory");
        const double S = a.dsc[0], usum = S * *s_csum;
        uint32_t li = 0;
        for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++li) {
            const int tile = item % a.ntiles, range = item / a.ntiles;
            const uint32_t acc = li & 1u;
            if (!bar_wait(dfull(acc), (li >> 1) & 1u)) {
                fail(7);
                break;
            }
            tc_fence_after();
            uint32_t r[32];
            tmem_ld32(tmem + lane_base + kColD + 32u * acc, r);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(dempty(acc));
            const int64_t j = (int64_t)tile * kRows + 32 * sub + lane;
            if (j < a.m) {
                double hs = 0.0, ms = 0.0;
#pragma unroll
                for (int p = kDigits - 1; p >= 0; --p) {
                    const double f = ldexp(1.0, -4 * (p + 1));
                    const double dh = (double)__uint_as_float(r[p]), dm = (double)__uint_as_float(r[16 + p]);
                    hs += f * (8.0 * dh - 192.0 * dm);
                    ms += f * dm;
                }
                double P1 = S * hs, P3 = 64.0 * S * ms;
                if (range == 0) {
                    P1 -= 8.0 * usum;          // the offset 1 of H(c) over all samples
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

// ---- host side --------------------------------------------------------------

struct TcPlan {
    int nstages, range_stages, nranges, ntiles, grid;
    size_t dig_bytes, cs_bytes, part_bytes;
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
    p.cs_bytes = (size_t)p.nstages * 8 * sizeof(int);
    p.part_bytes = 2 * (size_t)p.nranges * (size_t)h->m * sizeof(double);
    return p;
}

size_t rmv_tc_scratch_bytes(const gkl_handle* h) {
    const TcPlan p = plan_tc(h);
    return p.dig_bytes + ((p.cs_bytes + 255) & ~(size_t)255) + p.part_bytes + 256;
}

// Builds the TMA descriptor of the packed matrix (64-byte x 128-row boxes,
// 64-byte swizzle).  Returns false if the driver entry point or the encoding is
// unavailable or the buffer is not 16-byte aligned.
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
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    static_assert(sizeof(CUtensorMap) == sizeof(h->tc_map), "tensor map size");
    memcpy(h->tc_map, &map, sizeof(map));
    if (cudaFuncSetAttribute(k_rmv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes) != cudaSuccess)
        return false;
    h->tc_state = 1;
    return true;
}

cudaError_t launch_rmatvec_tc(const gkl_handle* h, const float* u, float* x, void* scratch, const Sv* sv,
                              const FinArgs* fa, cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    const TcPlan p = plan_tc(h);
    uint8_t* dig = static_cast<uint8_t*>(scratch);
    int* cs = reinterpret_cast<int*>(dig + p.dig_bytes);
    double* p1 = reinterpret_cast<double*>(reinterpret_cast<char*>(cs) + ((p.cs_bytes + 255) & ~(size_t)255));
    double* p3 = p1 + (size_t)p.nranges * h->m;
    double* aux = h->aux;  // dsc[4] | counter | partials of the scale pass; error word at kAuxErrOffset
    double* dsc = aux;
    unsigned* counter = reinterpret_cast<unsigned*>(aux + 4);
    double* part = aux + 8;
    int* err = reinterpret_cast<int*>(reinterpret_cast<char*>(aux) + kAuxErrOffset);
    cudaStream_t st = h->stream;
    const int sblocks = std::min(2 * h->num_sms, (int)((h->n + 255) / 256));
    k_u_scale<<<std::max(1, sblocks), 256, 0, st>>>(u, h->s, h->n, part, counter, dsc);
    k_u_digits_tc<<<p.nstages, 256, 0, st>>>(u, h->s, h->n, dsc, dig, cs);
    alignas(64) CUtensorMap map;
    memcpy(&map, h->tc_map, sizeof(map));
    TcArgs a{dig, cs, p.nstages, p.range_stages, p.nranges, p.ntiles, h->m, dsc, p1, p3, err};
    if (ev0) cudaEventRecord(ev0, st);
    k_rmv_tc<<<p.grid, kThreads, kSmemBytes, st>>>(map, a);
    if (ev1) cudaEventRecord(ev1, st);
    FinArgs f{};
    Sv s{};
    if (fa) f = *fa;
    if (sv) s = *sv;
    k_rmv_mma_fin<<<(unsigned)((h->m + 255) / 256), 256, 0, st>>>(p1, p3, p.nranges, h->m, h->mu, h->d, h->w, dsc, x,
                                                                    f, s);
    if (nlaunch) *nlaunch = 4;
    return cudaGetLastError();
}

}  // namespace gkl
