// y = A v without allocating device memory.
//
// Some callers may not call cudaMalloc: code embedded in a larger GPU
// application that owns all device memory through its own pool or arena
// (plugins, analytics running inside another program's memory budget), and
// latency-critical loops where an allocation, which can synchronise the whole
// device, is not allowed.  gkl_init allocates (statistics, scratch), so such
// callers use this entry point instead: the caller passes every input and the
// output, and the split-sum scratch of the product lives in one file-scope
// device array of fixed size.
//
// The array is part of the library's device image: every GPU that loads the
// library holds its kStaticScratchBytes until the process exits.  All calls
// share it and it keeps the last call's contents; each call writes every
// scratch element it later reads, so nothing needs clearing between calls.
// Calls that overlap on the GPU (concurrent streams or host threads) race on
// the array and must be serialised by the caller.
//
// The FP32 product streams the matrix through TMA copies whose waits are
// bounded (about two seconds); the last 256 bytes of the array hold the word a
// wait that runs out would set.  The call does not synchronise, so such an
// event (a GPU stalled for seconds) is not reported to it: y is then
// undefined.
#include <cuda_runtime.h>

#include <mutex>

#include "gkl_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once per
// device (the host-side symbol is only a stand-in for it).
int scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return gkl::cuda_err(nullptr, e, "static scratch set-up (cudaGetSymbolAddress)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GKL_OK;
}

// Device (or managed) memory of device `dev`: memory of another GPU would turn
// into peer reads or a fault inside the kernels.
bool on_device(const void* p, int dev) { return gkl::mem_kind(p, dev) == gkl::MEM_DEVICE; }

}  // namespace

extern "C" int gkl_matvec_noalloc(const uint8_t* packed, int64_t n, int64_t m, int64_t stride, const double* mu,
                                  const double* scale, int prec, const void* v, void* y, void* stream) {
    using gkl::set_err;
    if (!packed || !mu || !scale || !v || !y || v == y)
        return set_err(nullptr, GKL_ERR_ARG, "packed, mu, scale, v and y must be non-NULL (and y must not alias v)");
    if (n < 1 || m < 1) return set_err(nullptr, GKL_ERR_ARG, "need n >= 1 and m >= 1");
    if (stride % 16 != 0 || stride * 4 < n)
        return set_err(nullptr, GKL_ERR_ARG, "stride must be a multiple of 16 and >= ceil(n/4)");
    if (((uintptr_t)packed & 15u) != 0) return set_err(nullptr, GKL_ERR_ARG, "packed must be 16-byte aligned");
    if (prec != GKL_FP64 && prec != GKL_FP32) return set_err(nullptr, GKL_ERR_ARG, "unknown precision %d", prec);

    gkl_handle h{};
    h.packed = packed;
    h.n = n;
    h.m = m;
    h.stride = stride;
    h.stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&h.device);
    if (e != cudaSuccess) return gkl::cuda_err(nullptr, e, "cudaGetDevice");
    if (h.device < 0 || h.device >= kMaxDevices) return set_err(nullptr, GKL_ERR_ARG, "device index out of range");
    const int dev = h.device;
    if (!on_device(packed, dev) || !on_device(mu, dev) || !on_device(scale, dev) || !on_device(v, dev) ||
        !on_device(y, dev))
        return set_err(nullptr, GKL_ERR_ARG, "packed, mu, scale, v and y must be device memory of the current GPU");
    e = cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, h.device);
    if (e != cudaSuccess) return gkl::cuda_err(nullptr, e, "cudaDeviceGetAttribute");
    h.mu = const_cast<double*>(mu);
    h.d = const_cast<double*>(scale);

    const gkl::MvPlan p = gkl::plan_products(&h);
    const size_t elem = prec == GKL_FP64 ? sizeof(double) : sizeof(float);
    const size_t need = ((size_t)p.mv_chunks(prec == GKL_FP32) * (size_t)p.ldp + (size_t)m * 4) * elem;
    if (need > kStaticScratchBytes - 256)
        return set_err(nullptr, GKL_ERR_ARG,
                       "gkl_matvec_noalloc: n=%lld, m=%lld needs %zu bytes of scratch, above its static maximum of "
                       "%zu bytes; use gkl_matvec",
                       (long long)n, (long long)m, need, kStaticScratchBytes - 256);
    void* scratch = nullptr;
    int st = scratch_address(h.device, &scratch);
    if (st) return st;
    if (prec == GKL_FP32) {
        if (!gkl::make_mv_map(packed, stride, m, h.mv_map))
            return set_err(nullptr, GKL_ERR_CUDA, "gkl_matvec_noalloc: TMA descriptor of the packed matrix");
        h.mv_err = reinterpret_cast<int*>(static_cast<unsigned char*>(scratch) + kStaticScratchBytes - 256);
        e = cudaMemsetAsync(h.mv_err, 0, sizeof(int), h.stream);
        if (e != cudaSuccess) return gkl::cuda_err(nullptr, e, "gkl_matvec_noalloc error word");
    }
    e = prec == GKL_FP64
            ? gkl::launch_matvec<double>(&h, (const double*)v, (double*)y, scratch, nullptr, nullptr)
            : gkl::launch_matvec<float>(&h, (const float*)v, (float*)y, scratch, nullptr, nullptr);
    if (e != cudaSuccess) return gkl::cuda_err(nullptr, e, "gkl_matvec_noalloc launch");
    return GKL_OK;
}
