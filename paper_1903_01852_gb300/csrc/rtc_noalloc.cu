// Allocation-free reconstruction + control step (rtc_reconstruct_noalloc).
//
// Some callers cannot allocate device memory once they are running: a hard
// real-time control thread must not call cudaMalloc inside its frame (the call
// can synchronise the whole device and has no latency bound), and code hosted
// inside another runtime that owns every device allocation is not allowed to
// call it at all.  This entry point lets such callers run the MVM and the
// leaky-integrator step on their own buffers: the per-column-split partial
// sums live in a fixed array compiled into this library instead of memory it
// would otherwise allocate.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "rtc_internal.h"

namespace {

// Scratch for the partial sums: nsplit x na floats.  Every GPU that loads the
// library holds these bytes until the process exits; every call shares them.
constexpr size_t kScratchFloats = RTC_NOALLOC_MAX_FLOATS;
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kWarps = 8;

// One warp per matrix row over one column split [c0, c1): 16-byte loads of the
// row and the slopes where a whole vector lies inside the split, single
// elements for the ragged end; lane sums reduced by a fixed xor butterfly.
__global__ void __launch_bounds__(kWarps * 32)
split_gemv_kernel(const float* __restrict__ M, size_t ld, int na, int ns, int split_cols,
                  const float* __restrict__ s, float* __restrict__ part) {
    const int j = blockIdx.y;
    const int r = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= na) return;
    const int c0 = j * split_cols;
    const int c1 = min(ns, c0 + split_cols);
    const float* row = M + (size_t)r * ld;
    const int nfull = (c1 - c0) >> 2;                 // whole float4 vectors in the split
    float acc = 0.f;
    for (int v = lane; v < nfull; v += 32) {
        const int c = c0 + 4 * v;
        const float4 m = __ldcs(reinterpret_cast<const float4*>(row + c));
        const float4 x = __ldg(reinterpret_cast<const float4*>(s + c));
        acc = fmaf(m.x, x.x, acc);
        acc = fmaf(m.y, x.y, acc);
        acc = fmaf(m.z, x.z, acc);
        acc = fmaf(m.w, x.w, acc);
    }
    for (int c = c0 + 4 * nfull + lane; c < c1; c += 32) acc = fmaf(row[c], s[c], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[(size_t)j * na + r] = acc;
}

// Sum of the splits in split order, row scale, q, leaky integrator.
__global__ void split_finalise_kernel(const float* __restrict__ part, int nsplit, int na,
                                      const float* __restrict__ scale, const float* __restrict__ q,
                                      const float* a_in, float* a_out, float oml, float gain) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= na) return;
    float y = 0.f;
    for (int j = 0; j < nsplit; ++j) y += part[(size_t)j * na + r];
    if (scale) y *= scale[r];
    const float w = q ? y + q[r] : y;
    a_out[r] = fmaf(gain, w, oml * a_in[r]);
}

// The scratch array's address belongs to a context: the primary context of a
// device, a driver-API context the caller made current, or the primary context
// re-created after cudaDeviceReset each have their own copy of the module.  The
// address is therefore looked up once per context, keyed by the driver's
// context id (unique for the life of the process, never reused), with that
// context current.  The two driver calls are resolved through the runtime, so
// the library needs no link against the driver library.
using CtxGetCurrentFn = int (*)(void** ctx);          // CUresult cuCtxGetCurrent(CUcontext*)
using CtxGetIdFn = int (*)(void* ctx, unsigned long long* id);  // CUresult cuCtxGetId(CUcontext, id*)

struct DriverFns {
    CtxGetCurrentFn get_current = nullptr;
    CtxGetIdFn get_id = nullptr;
};

const DriverFns& driver_fns() {
    static DriverFns fns;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fns.get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fns.get_id = reinterpret_cast<CtxGetIdFn>(p);
    });
    return fns;
}

// Id of the context current on this thread; 0 if there is none or it cannot be read.
unsigned long long current_context_id() {
    const DriverFns& d = driver_fns();
    if (!d.get_current || !d.get_id) return 0;
    void* ctx = nullptr;
    if (d.get_current(&ctx) != 0 || !ctx) return 0;
    unsigned long long id = 0;
    return d.get_id(ctx, &id) == 0 ? id : 0;
}

float* scratch_address(cudaError_t* err) {
    static std::mutex mu;
    static std::vector<std::pair<unsigned long long, float*>> addr;   // (context id, address)
    *err = cudaSuccess;
    unsigned long long id = current_context_id();
    if (id == 0) {
        // No context is current yet: the runtime's lookup below makes the current
        // device's primary context current; its id is read afterwards.
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        id = current_context_id();
        if (id == 0) { *err = cudaErrorDeviceUninitialized; return nullptr; }
    }
    std::lock_guard<std::mutex> g(mu);
    for (const auto& e : addr)
        if (e.first == id) return e.second;
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr.emplace_back(id, static_cast<float*>(p));
    return static_cast<float*>(p);
}

}  // namespace

extern "C" int rtc_reconstruct_noalloc(int32_t na, int32_t ns, const float* M, size_t ld,
                                       const float* row_scale, const float* s, const float* q,
                                       const float* a_in, float* a_out, float gain, float leak,
                                       void* stream) {
    if (na <= 0 || ns <= 0 || !M || !s || !a_in || !a_out)
        return RTC_EINVAL;
    if (ld < (size_t)ns || (ld & 3u) || (reinterpret_cast<uintptr_t>(M) & 15u) || (reinterpret_cast<uintptr_t>(s) & 15u))
        return RTC_EINVAL;
    if ((size_t)na > kScratchFloats)
        return RTC_EINVAL;   // more rows than the scratch array holds
    // Column splits: about 1024 columns each for parallelism, fewer when the
    // scratch (nsplit x na floats) would not hold them.
    int nsplit = (ns + 1023) / 1024;
    const int max_split = (int)std::min<size_t>(kScratchFloats / (size_t)na, 65535);
    if (nsplit > max_split) nsplit = max_split;
    int split_cols = (ns + nsplit - 1) / nsplit;
    split_cols = (split_cols + 3) / 4 * 4;
    nsplit = (ns + split_cols - 1) / split_cols;
    // An error left pending by the caller's own earlier work is not ours to
    // report or to clear: return without launching and leave it in place.
    if (cudaPeekAtLastError() != cudaSuccess) return RTC_ECUDA;
    cudaError_t e = cudaSuccess;
    float* part = scratch_address(&e);
    if (!part) return RTC_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (rtc::launch_kernel(split_gemv_kernel, dim3((na + kWarps - 1) / kWarps, nsplit), dim3(kWarps * 32), 0, st, M, ld, na,
                      ns, split_cols, s, part) != cudaSuccess)
        return RTC_ECUDA;
    if (rtc::launch_kernel(split_finalise_kernel, dim3((na + 255) / 256), dim3(256), 0, st, (const float*)part, nsplit, na,
                      row_scale, q, a_in, a_out, 1.0f - leak, gain) != cudaSuccess)
        return RTC_ECUDA;
    return RTC_OK;
}
