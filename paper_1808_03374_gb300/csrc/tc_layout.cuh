// Layout helpers shared by the tcgen05 kernels whose genotype operand is
// decoded into shared memory: the K order of the samples of a 16-sample code
// word, the 128-byte-swizzled K-major tile layout, exact loads of FP32
// accumulators as 64-bit integers, and the reduce-scatter over digit lanes.
#pragma once

#include <stdint.h>

namespace gkl {

// Position along K of sample `s` (0..15) of a 16-sample code word: the byte
// permutes emit samples 0, 2, .., 14 then 1, 3, .., 15.
__host__ __device__ inline int bt_kpos(int s) { return (s & 1) ? 8 + (s >> 1) : (s >> 1); }
__host__ __device__ inline int bt_sample_of_kpos(int k) { return k < 8 ? 2 * k : 2 * (k - 8) + 1; }
// Byte offset of (row r, K byte kk < 128) in a 128-row, 128-byte-swizzled K-major tile.
__host__ __device__ inline int bt_swz(int r, int kk) {
    return (r >> 3) * 1024 + (r & 7) * 128 + ((((kk >> 4) ^ (r & 7))) << 4) + (kk & 15);
}

__device__ __forceinline__ long long shfl_xor_ll(long long v, int o) {
    const int lo = __shfl_xor_sync(0xffffffffu, (int)(v & 0xffffffffLL), o);
    const int hi = __shfl_xor_sync(0xffffffffu, (int)(v >> 32), o);
    return ((long long)hi << 32) | (unsigned)lo;
}

// Reduce-scatter of 16 values over the D lanes c D .. c D + D - 1 of one
// vector's digit rows (lane digit index p): on return v[0 .. 16/D) hold the
// group sums of entries (16/D) p .. (16/D) p + 16/D - 1.
template <int D>
__device__ __forceinline__ void bt_reduce_scatter(long long (&v)[16], int p) {
#pragma unroll
    for (int step = D / 2, h = 8; step >= 1; step >>= 1, h >>= 1) {
        const bool up = (p & step) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const long long send = up ? v[i] : v[i + h];
            const long long keep = up ? v[i + h] : v[i];
            v[i] = keep + shfl_xor_ll(send, step);
        }
    }
}

// 16 consecutive columns of this warp's 32 lanes, converted from the exact
// FP32 accumulator values to 64-bit integers scaled by 2^sh.
__device__ __forceinline__ void bt_ld16_scaled(uint32_t taddr, int sh, long long (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = (long long)__float2int_rn(__uint_as_float(r[i])) << sh;
}

}  // namespace gkl
