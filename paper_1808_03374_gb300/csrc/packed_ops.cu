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
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "epilogue.cuh"
#include "gkl_internal.cuh"
#include "tc_ptx.cuh"

namespace gkl {

namespace {
constexpr int kThreads = 256;   // threads per block of the product kernels
constexpr int kRowBatch = 32;   // SNP rows staged per batch
constexpr int kMvBoxBytesHost = 256, kMvRowsHost = 16;  // TMA box of the FP32 A v kernel
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

// ------------------------------------------------------------------ TMA view for A v

// TMA descriptor of the packed matrix for the FP32 A v kernel: a 2-D uint8
// tensor (stride x m) read in boxes of 256 bytes x 16 rows, no swizzle.
// Host-only (no device memory is allocated); false if the driver entry point
// is unavailable or the descriptor is rejected.
bool make_mv_map(const uint8_t* packed, int64_t stride, int64_t m, void* out) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr) {
        cudaGetLastError();
        return false;
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t gdim[2] = {(cuuint64_t)stride, (cuuint64_t)m};
    const cuuint64_t gstride[1] = {(cuuint64_t)stride};
    const cuuint32_t box[2] = {(cuuint32_t)kMvBoxBytesHost, (cuuint32_t)kMvRowsHost};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                        const_cast<uint8_t*>(packed), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
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
    // FP32 A.v (TMA-fed pair-table kernel, CTAs of 256 words): the SNP chunking
    // that gives the busiest SM the fewest rows, every chunk at least one
    // 256-row table batch (rows a multiple of 32, two 16-row stages)
    {
        const int sms = std::max(1, h->num_sms);
        const int64_t tiles = (p.nwords + 255) / 256;
        double best = 0.0;
        for (int waves = 1; waves <= 32; ++waves) {
            int64_t chunks = std::max<int64_t>(1, (waves * (int64_t)sms + tiles - 1) / tiles);
            int64_t rpc = (h->m + chunks - 1) / chunks;
            rpc = std::max<int64_t>(rpc, 256);
            rpc = (rpc + 31) / 32 * 32;
            chunks = (h->m + rpc - 1) / rpc;
            const int64_t blocks_sm = (tiles * chunks + sms - 1) / sms;
            const double load = (double)blocks_sm * (double)rpc;
            if (best == 0.0 || load < 0.99 * best) {
                best = load;
                p.pair_threads = 256;
                p.pair_tiles = (int)tiles;
                p.pair_chunks = (int)chunks;
                p.pair_rpc = (int)rpc;
            }
        }
    }
    size_t mv = (size_t)std::max(p.chunks, p.pair_chunks) * (size_t)p.ldp + (size_t)h->m * 4;  // partials + LUT
    size_t tc = h->tc_state > 0 ? rmv_tc_scratch_bytes(h) : 0;
    p.bytes_fp64 = std::max(mv * sizeof(double) + 256, tc);
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
//
// The tables of four consecutive pairs fill one 256-byte-aligned group, so the
// shared address of a lookup is one byte-permute: byte 0 = 4 x index (from the
// code words), bytes 1-3 = the group's base; the pair within the group is the
// load's immediate offset.  Tables are built for a batch of 128 pairs (256
// rows) while the previous batch is consumed, into the other of two buffers:
// one barrier per batch.  Adjacent samples accumulate with paired FP32 adds.
constexpr int kPairBatch = 128;                  // row pairs per table batch
constexpr int kPairRows = 2 * kPairBatch;        // 256 rows
constexpr int kPairTab = kPairBatch * 16;        // floats per table buffer (8 KB)

template <int OFF>
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];\n" : "=f"(v) : "r"(a), "n"(OFF));
    return v;
}

// Four lookups (samples 4b .. 4b+3 of one pair) for b = 0..3, pair Q of the group at gb.
template <int Q>
__device__ __forceinline__ void pair_lookups(uint32_t wa, uint32_t wb, uint32_t gb, float2 (&acc)[8]) {
    const uint32_t e = (wa & 0x33333333u) | ((wb & 0x33333333u) << 2);
    const uint32_t o = ((wa >> 2) & 0x33333333u) | (wb & 0xCCCCCCCCu);
    // bytes of eL hold 4 x nibbles 0, 2, 4, 6 of e (samples 0, 4, 8, 12), bytes of
    // eH 4 x nibbles 1, 3, 5, 7 (samples 2, 6, 10, 14); likewise o (odd samples)
    const uint32_t eL = (e << 2) & 0x3C3C3C3Cu, eH = (e >> 2) & 0x3C3C3C3Cu;
    const uint32_t oL = (o << 2) & 0x3C3C3C3Cu, oH = (o >> 2) & 0x3C3C3C3Cu;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t sel = 0x7650u | (uint32_t)b;
        const float x0 = lds_f32<Q * 64>(__byte_perm(eL, gb, sel));
        const float x1 = lds_f32<Q * 64>(__byte_perm(oL, gb, sel));
        const float x2 = lds_f32<Q * 64>(__byte_perm(eH, gb, sel));
        const float x3 = lds_f32<Q * 64>(__byte_perm(oH, gb, sel));
        acc[2 * b] = __fadd2_rn(acc[2 * b], make_float2(x0, x1));
        acc[2 * b + 1] = __fadd2_rn(acc[2 * b + 1], make_float2(x2, x3));
    }
}

// The FP32 A v kernel: one CTA per (sample tile of 256 words = 4,096 samples,
// SNP chunk), 8 consumer warps (one 16-sample word per thread) and one copy
// warp.  The copy warp's lane 0 streams the tile's rows through a ring of
// shared-memory stages with TMA (16 rows x four 256-byte boxes per stage, no
// swizzle: a warp's 32 words of a row are 128 contiguous bytes, one wavefront),
// so the consumers only wait on full stages and spend their issue slots on
// table lookups.  Three CTAs share an SM (three 16 KB stages and 16 KB of
// tables each, 72 registers a thread): more warps to keep the shared-memory
// pipe that bounds the kernel busy.  Pair tables are built per 256-row batch by
// consumer threads (double-buffered; the consumers meet at a named barrier
// once per batch).
constexpr int kMvWords = 256;                  // words (16 samples each) per tile
constexpr int kMvConsumers = kMvWords;         // consumer threads
constexpr int kMvThreads = kMvConsumers + 32;  // + one copy warp
constexpr int kMvRows = 16;                    // rows per stage
constexpr int kMvBoxBytes = 256;               // box width (bytes of one row)
constexpr int kMvBoxes = kMvWords * 4 / kMvBoxBytes;
constexpr int kMvStageBytes = kMvRows * kMvWords * 4;  // 16 KB
constexpr int kMvStages = 3;
constexpr int kMvTabOff = kMvStages * kMvStageBytes;      // two table buffers of 8 KB
constexpr int kMvBarOff = kMvTabOff + 2 * kPairTab * 4;
constexpr int kMvSmem = 1024 + kMvBarOff + 256;
static_assert(kPairRows % kMvRows == 0, "a table batch covers whole stages");

__global__ void __launch_bounds__(kMvThreads, 3)
    k_mv_pair(const __grid_constant__ CUtensorMap tmap, int64_t nwords, int64_t m, int rpc,
              const float* __restrict__ lut, float* __restrict__ part, int64_t ldp, int* err) {
    extern __shared__ uint8_t mv_smem_raw[];
    const uint32_t raw = tc::sm_addr(mv_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sb = mv_smem_raw + (base - raw);
    const uint32_t sBar = base + kMvBarOff;
    auto full = [&](int s) { return sBar + 8u * s; };
    auto empty = [&](int s) { return sBar + 8u * (kMvStages + s); };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t j0 = (int64_t)blockIdx.y * rpc;
    const int64_t j1 = min(m, j0 + (int64_t)rpc);
    const int nstage = (int)((j1 - j0 + kMvRows - 1) / kMvRows);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMvStages; ++s) {
            tc::bar_init(full(s), 1);
            tc::bar_init(empty(s), kMvConsumers / 32);
        }
        tc::bar_init_fence();
    }
    __syncthreads();
    auto fail = [&](int code) {
        if (err) atomicCAS(err, 0, code);
    };

    if (warp == kMvConsumers / 32) {
        // ---- copies: rows j0 .. of this tile, four 256-byte boxes per 16-row stage
        if (lane == 0) {
            const int x0 = (int)blockIdx.x * kMvWords * 4;
            int s_it = 0;
            for (; s_it < nstage; ++s_it) {
                const int s = s_it % kMvStages;
                if (!tc::bar_wait(empty(s), ((s_it / kMvStages) & 1) ^ 1)) {
                    fail(41);
                    break;
                }
                tc::bar_expect_tx(full(s), kMvStageBytes);
                const int y = (int)(j0 + (int64_t)s_it * kMvRows);
#pragma unroll
                for (int bx = 0; bx < kMvBoxes; ++bx)
                    tc::tma_2d(base + s * kMvStageBytes + bx * kMvRows * kMvBoxBytes, &tmap, x0 + bx * kMvBoxBytes,
                               y, full(s));
            }
            // drain: every issued copy has landed before the CTA may exit
            for (int q = s_it > kMvStages ? s_it - kMvStages : 0; q < s_it; ++q)
                if (!tc::bar_wait(full(q % kMvStages), (q / kMvStages) & 1)) fail(42);
        }
        return;
    }

    // ---- consumers
    const uint32_t tb0 = base + kMvTabOff;
    float* tabs = reinterpret_cast<float*>(sb + kMvTabOff);
    const int t = threadIdx.x;
    const int64_t word = (int64_t)blockIdx.x * kMvWords + t;
    const bool active = word < nwords;
    // the table of pair p of the batch at row jb (rows jb + 2p, jb + 2p + 1) is
    // built by thread p from the two rows' 4-entry tables: one L2 round trip
    auto build = [&](int64_t jb, int buf) {
        const int p = t;
        if (p >= kPairBatch) return;
        const int64_t ra = jb + 2 * p, rb = ra + 1;
        const float4 la = ra < j1 ? __ldg(reinterpret_cast<const float4*>(lut) + ra) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 lb = rb < j1 ? __ldg(reinterpret_cast<const float4*>(lut) + rb) : make_float4(0.f, 0.f, 0.f, 0.f);
        float4* dst = reinterpret_cast<float4*>(tabs + buf * kPairTab + 16 * p);
        dst[0] = make_float4(la.x + lb.x, la.y + lb.x, la.z + lb.x, la.w + lb.x);  // c_b = 0
        dst[1] = make_float4(la.x + lb.y, la.y + lb.y, la.z + lb.y, la.w + lb.y);  // c_b = 1
        dst[2] = make_float4(la.x + lb.z, la.y + lb.z, la.z + lb.z, la.w + lb.z);  // c_b = 2
        dst[3] = make_float4(la.x + lb.w, la.y + lb.w, la.z + lb.w, la.w + lb.w);  // c_b = 3
    };
    // word t of row r of a stage: box t / 64, 4 (t mod 64) bytes into the row
    const uint32_t* wbase =
        reinterpret_cast<const uint32_t*>(sb + (t >> 6) * kMvRows * kMvBoxBytes + 4 * (t & 63));
    float2 acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
    const int nbatch = (int)((j1 - j0 + kPairRows - 1) / kPairRows);
    build(j0, 0);
    asm volatile("bar.sync 1, %0;\n" ::"n"(kMvConsumers) : "memory");
    bool ok = true;
    int s_it = 0;
    for (int i = 0; i < nbatch; ++i) {
        const int64_t jb = j0 + (int64_t)i * kPairRows;
        const uint32_t tb = tb0 + (uint32_t)(i & 1) * (kPairTab * 4);
        if (i + 1 < nbatch) build(jb + kPairRows, (i + 1) & 1);
        const int ns = min(kPairRows / kMvRows, nstage - i * (kPairRows / kMvRows));
        for (int q = 0; q < ns && ok; ++q, ++s_it) {
            const int s = s_it % kMvStages;
            if (!tc::bar_wait_warp(full(s), (s_it / kMvStages) & 1)) {
                fail(43);
                ok = false;
                break;
            }
            const uint32_t* wr = wbase + s * (kMvStageBytes / 4);
#pragma unroll
            for (int g = 0; g < kMvRows / 8; ++g) {
                uint32_t w[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) w[k] = wr[(8 * g + k) * (kMvBoxBytes / 4)];
                const uint32_t gb = tb + 256u * (uint32_t)(q * (kMvRows / 8) + g);
                pair_lookups<0>(w[0], w[1], gb, acc);
                pair_lookups<1>(w[2], w[3], gb, acc);
                pair_lookups<2>(w[4], w[5], gb, acc);
                pair_lookups<3>(w[6], w[7], gb, acc);
            }
            __syncwarp();
            if (lane == 0) tc::bar_arrive(empty(s));
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(kMvConsumers) : "memory");
    }
    if (!active || !ok) return;
    float4* out = reinterpret_cast<float4*>(part + (int64_t)blockIdx.y * ldp + word * 16);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = make_float4(acc[2 * k].x, acc[2 * k].y, acc[2 * k + 1].x, acc[2 * k + 1].y);
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
    constexpr bool fp32 = sizeof(T) == sizeof(float);
    const int chunks = p.mv_chunks(fp32);
    T* part = static_cast<T*>(scratch);
    T* lut = part + (size_t)chunks * (size_t)p.ldp;
    cudaStream_t st = h->stream;
    GKL_DEBUG_SYNC(st, "before A.v");
    k_mv_table<T><<<(unsigned)((h->m + 255) / 256), 256, 0, st>>>(h->m, h->mu, h->d, h->w, v, lut);
    GKL_DEBUG_SYNC(st, "k_mv_table");
    if (ev0) cudaEventRecord(ev0, st);
    if constexpr (fp32) {
        static std::once_flag attr;
        std::call_once(attr, [] { cudaFuncSetAttribute(k_mv_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, kMvSmem); });
        alignas(64) CUtensorMap map;
        static_assert(sizeof(CUtensorMap) == sizeof(h->mv_map), "tensor map size");
        memcpy(&map, h->mv_map, sizeof(map));
        int* err = h->aux ? reinterpret_cast<int*>(reinterpret_cast<char*>(h->aux) + kAuxErrOffset) : h->mv_err;
        k_mv_pair<<<dim3((unsigned)p.pair_tiles, (unsigned)p.pair_chunks), kMvThreads, kMvSmem, st>>>(
            map, p.nwords, h->m, p.pair_rpc, reinterpret_cast<const float*>(lut), reinterpret_cast<float*>(part), p.ldp,
            err);
    } else
        k_mv_part<T><<<dim3((unsigned)p.tiles, (unsigned)p.chunks), kThreads, 0, st>>>(
            h->packed, h->stride, p.nwords, h->m, p.rows_per_chunk, lut, part, p.ldp);
    if (ev1) cudaEventRecord(ev1, st);
    GKL_DEBUG_SYNC(st, "A.v main kernel");
    if (nlaunch) *nlaunch = 3;
    FinArgs f{};
    Sv s{};
    if (fa) f = *fa;
    if (sv) s = *sv;
    // 32 outputs per block pass; at most 4 blocks per SM (the partial-norm buffer's size)
    const int fblocks = (int)std::min<int64_t>((h->n + 31) / 32, 4 * (int64_t)h->num_sms);
    k_mv_fin<T><<<(unsigned)std::max(1, fblocks), 256, 0, st>>>(part, p.ldp, chunks, h->n, h->s, y, f, s);
    GKL_DEBUG_SYNC(st, "k_mv_fin");
    return cudaGetLastError();
}

// ------------------------------------------------------------------ A^T u

// Both precisions run the tensor-core kernel (gkl_init fails without it).
template <typename T>
cudaError_t launch_rmatvec(const gkl_handle* h, const T* u, T* x, void* scratch, const Sv* sv, const FinArgs* fa,
                           cudaEvent_t ev0, cudaEvent_t ev1, int* nlaunch) {
    return launch_rmatvec_tc<T>(h, u, x, scratch, sv, fa, ev0, ev1, nlaunch);
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
