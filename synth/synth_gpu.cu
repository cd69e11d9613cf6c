/*
 * GPU twin of synth_pack (synth.c): the same packed genotype matrix, byte for
 * byte, drawn on the device so that matrices of tens of gigabytes take seconds
 * instead of minutes.  Like synth.c it draws random inputs only and holds none
 * of the PCA method's arithmetic.
 *
 * Entry (i, j): with r = Philox4x32-10 of the counter (i, j, ST_GENO, 0) under
 * the key (seed lo, seed hi),
 *   missing         iff  r0 < miss_rate * 2^32,
 *   else code = [r1 < p_ij 2^32] + [r2 < p_ij 2^32],  p_ij = sum_k q_ik f_kj
 * where synth.c forms p_ij in FP64, k ascending, each product and sum rounded
 * (no fused multiply-add).  Here:
 *  - the missing test is the integer test r0 < ceil(miss_rate * 2^32) (the
 *    host computes the ceiling; for an integer r0 the two tests agree);
 *  - p_ij is first formed in FP32 from FP32 copies of q and f.  With
 *    q_ik >= 0, sum_k q_ik = 1 and f_kj in [0, 1], its error is at most
 *    (S + 2) 2^-24 (rounding of q and f, S rounded accumulations), i.e. at most
 *    (S + 2) * 256 on the 2^32 scale, plus 256 for the rounding of p 2^32 to
 *    FP32 and 1 for the conversion to an integer.  A draw farther than twice
 *    that from the FP32 threshold is decided by it; a draw inside the margin
 *    (about one in 10^5) takes the FP64 sum exactly as synth.c writes it,
 *    with FP contraction off for this file (-fmad=false).
 * Padding entries (i >= n) are code 3, as are the bytes beyond ceil(n/4).
 */
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t o0 = hi1 ^ c[1] ^ k0, o2 = hi0 ^ c[3] ^ k1;
        c[0] = o0;
        c[1] = lo1;
        c[2] = o2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

constexpr uint32_t kStGeno = 4;  // ST_GENO of synth.c
constexpr int kMaxPops = 64;

struct PackArgs {
    int64_t n, m, words;  // words: stride / 4 (32-bit words of 16 samples per row)
    int S;
    uint64_t seed;
    uint64_t miss_int;    // r0 < miss_int  <=>  (double) r0 < miss_rate * 2^32
    const double* q64;    // n x S
    const double* f64;    // S x m
    const float* q32;
    const float* f32;
    uint32_t* out;        // m x words
    int64_t margin;       // decision margin on the 2^32 scale
};

__device__ __forceinline__ unsigned code_of(const PackArgs& a, int64_t i, int64_t j, const float* fj) {
    uint32_t c[4] = {(uint32_t)i, (uint32_t)j, kStGeno, 0u};
    philox(c, (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    if ((uint64_t)c[0] < a.miss_int) return 3u;
    const float* qi = a.q32 + i * a.S;
    float p = 0.f;
    for (int k = 0; k < a.S; ++k) p = fmaf(qi[k], fj[k], p);
    const int64_t T = (int64_t)__float2ull_rz(p * 4294967296.0f);
    unsigned code = 0u;
#pragma unroll
    for (int b = 1; b <= 2; ++b) {
        const int64_t r = (int64_t)c[b];
        if (r < T - a.margin) {
            code += 1u;
        } else if (r <= T + a.margin) {  // near the threshold: the FP64 sum of synth.c
            const double* q = a.q64 + i * a.S;
            double pij = 0.0;
            for (int k = 0; k < a.S; ++k) pij += q[k] * a.f64[(int64_t)k * a.m + j];
            const double t = pij * 4294967296.0;
            code += (double)c[b] < t ? 1u : 0u;
        }
    }
    return code;
}

// One thread per 32-bit word (16 samples) of one SNP row; grid-stride over
// (row, word) in row-major order.
__global__ void __launch_bounds__(256) k_pack(PackArgs a) {
    const int64_t total = a.m * a.words;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / a.words, w = e - j * a.words;
        float fj[kMaxPops];
        for (int k = 0; k < a.S; ++k) fj[k] = a.f32[(int64_t)k * a.m + j];
        uint32_t word = 0xFFFFFFFFu;
        const int64_t i0 = 16 * w;
        if (i0 < a.n) {
            word = 0u;
            for (int t = 0; t < 16; ++t) {
                const int64_t i = i0 + t;
                const unsigned code = i < a.n ? code_of(a, i, j, fj) : 3u;
                word |= code << (2 * t);
            }
        }
        a.out[e] = word;
    }
}

}  // namespace

extern "C" int synth_pack_gpu(int64_t n, int64_t m, int64_t stride, int32_t S, uint64_t seed, uint64_t miss_int,
                              const double* q64, const double* f64, const float* q32, const float* f32,
                              uint8_t* packed, void* stream) {
    if (n <= 0 || m <= 0 || stride % 16 != 0 || stride * 4 < n || S < 1 || S > kMaxPops) return -1;
    if (((uintptr_t)packed & 3u) != 0) return -1;
    PackArgs a;
    a.n = n;
    a.m = m;
    a.words = stride / 4;
    a.S = S;
    a.seed = seed;
    a.miss_int = miss_int;
    a.q64 = q64;
    a.f64 = f64;
    a.q32 = q32;
    a.f32 = f32;
    a.out = reinterpret_cast<uint32_t*>(packed);
    a.margin = 2 * ((int64_t)(S + 2) * 256 + 256 + 1);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_pack<<<8 * sms, 256, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
