// Master of a loop split by WFS (rtc_master_*): the control law applied to the
// sum of the shards' partial reconstructions (Section 3: reconstruction nodes
// send partial DM commands to a master; Section 3.4: implicit POLC computed
// after the commands, for the next frame).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "rtc_internal.h"

using namespace rtc;

struct rtc_master {
    int dev = 0, na = 0, nshards = 0, pitch = 0;
    float gain = 0.f, leak = 0.f;
    int clip = 0;
    float amin = 0.f, amax = 0.f;
    bool has_p = false;
    int p_dtype = RTC_F32;
    cudaStream_t st = nullptr;
    cudaEvent_t ev_cmd = nullptr;
    float* d_in = nullptr;          // [nshards][pitch]
    float* d_a = nullptr;
    float* d_q = nullptr;
    float* d_cmd = nullptr;
    void* d_P = nullptr;
    BlockDev* d_pblock = nullptr;
    float* d_pscale = nullptr;
    uint64_t p_bytes = 0;
    float* h_cmd = nullptr;         // page-locked
    uint64_t last_id = 0;
    bool stepped = false;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

thread_local std::string g_master_err;

int mfail(rtc_master* m, int code, const std::string& msg) {
    if (m) m->err = msg;
    else g_master_err = msg;
    return code;
}

int mcuda(rtc_master* m, cudaError_t e, const char* where) {
    cudaGetLastError();
    return mfail(m, RTC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define MCK(m, call)                                          \
    do {                                                      \
        const cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return mcuda((m), e_, #call);  \
    } while (0)

template <typename T>
int malloc_dev(rtc_master* m, T** p, size_t bytes) {
    void* v = nullptr;
    const cudaError_t e = cudaMalloc(&v, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mfail(m, RTC_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes");
    }
    m->allocs.push_back(v);
    *p = static_cast<T*>(v);
    return RTC_OK;
}

// One thread per actuator: the shards' partials in shard order, then the POLC
// term and the leaky integrator (as the loop's fused finalisation).
__global__ void master_kernel(const float* __restrict__ in, int nshards, int pitch, int na, const float* __restrict__ q,
                              float* __restrict__ a, float* __restrict__ cmd, float oml, float gain, int clip,
                              float amin, float amax) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= na) return;
    float y = 0.f;
    for (int k = 0; k < nshards; ++k) y += in[(size_t)k * pitch + r];
    const float w = y + q[r];
    float v = fmaf(gain, w, oml * a[r]);
    if (clip) v = fminf(fmaxf(v, amin), amax);
    a[r] = v;
    cmd[r] = v;
}

void release_master(rtc_master* m) {
    if (!m) return;
    cudaSetDevice(m->dev);
    if (m->st) cudaStreamSynchronize(m->st);
    if (m->ev_cmd) cudaEventDestroy(m->ev_cmd);
    for (void* p : m->allocs) cudaFree(p);
    if (m->h_cmd) cudaFreeHost(m->h_cmd);
    if (m->st) cudaStreamDestroy(m->st);
    cudaGetLastError();
    delete m;
}

int polc(rtc_master* m) {
    if (!m->has_p) return RTC_OK;
    MCK(m, launch_gemv(m->p_dtype, m->d_P, m->d_pblock, 0, 1, m->na, m->d_a, m->d_pscale, m->d_q, 0, nullptr,
                       (long long)(m->p_bytes / std::max(m->na, 1)), false, m->st));
    return RTC_OK;
}

int create(const rtc_master_desc* d, rtc_master* m) {
    if (!d || !d->polc) return mfail(m, RTC_EINVAL, "desc and desc->polc are required");
    const rtc_polc* P = d->polc;
    if (d->na < 1 || d->na > (1 << 24)) return mfail(m, RTC_EINVAL, "na out of range");
    if (d->nshards < 1 || d->nshards > RTC_MAX_WFS) return mfail(m, RTC_EINVAL, "nshards must be in [1, RTC_MAX_WFS]");
    if (P->mode != RTC_POLC_IMPLICIT || P->D) return mfail(m, RTC_EINVAL, "the master takes implicit POLC only");
    if (P->P && P->dtype != RTC_F32 && P->dtype != RTC_BF16 && P->dtype != RTC_E4M3)
        return mfail(m, RTC_EINVAL, "bad P dtype");
    if (!std::isfinite(P->gain) || !std::isfinite(P->leak)) return mfail(m, RTC_EINVAL, "gain and leak must be finite");
    if (P->clip && !(P->amin <= P->amax)) return mfail(m, RTC_EINVAL, "clip needs amin <= amax");
    m->dev = d->device;
    m->na = d->na;
    m->nshards = d->nshards;
    m->pitch = (d->na + 3) / 4 * 4;
    m->gain = P->gain;
    m->leak = P->leak;
    m->clip = P->clip;
    m->amin = P->amin;
    m->amax = P->amax;
    m->has_p = P->P != nullptr;
    m->p_dtype = m->has_p ? P->dtype : RTC_F32;
    const size_t na = (size_t)m->na;
    if (P->a0)
        for (size_t r = 0; r < na; ++r)
            if (!std::isfinite(P->a0[r])) return mfail(m, RTC_EINVAL, "a0 not finite");
    if (m->has_p && P->row_scale)
        for (size_t r = 0; r < na; ++r)
            if (!std::isfinite(P->row_scale[r])) return mfail(m, RTC_EINVAL, "P row_scale not finite");
    if (m->has_p && m->p_dtype == RTC_F32) {
        const float* p = static_cast<const float*>(P->P);
        for (size_t i = 0; i < na * na; ++i)
            if (!std::isfinite(p[i])) return mfail(m, RTC_EINVAL, "P contains NaN or Inf");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || m->dev < 0 || m->dev >= ndev) {
        cudaGetLastError();
        return mfail(m, RTC_EINVAL, "no such CUDA device");
    }
    MCK(m, cudaSetDevice(m->dev));
    MCK(m, cudaStreamCreateWithPriority(&m->st, cudaStreamNonBlocking, -5));
    MCK(m, cudaEventCreateWithFlags(&m->ev_cmd, cudaEventDisableTiming));
    int rc = malloc_dev(m, &m->d_in, (size_t)m->nshards * m->pitch * 4);
    if (rc == RTC_OK) rc = malloc_dev(m, &m->d_a, (size_t)m->pitch * 4 + 64);
    if (rc == RTC_OK) rc = malloc_dev(m, &m->d_q, (size_t)m->pitch * 4);
    if (rc == RTC_OK) rc = malloc_dev(m, &m->d_cmd, (size_t)m->pitch * 4);
    if (rc != RTC_OK) return rc;
    MCK(m, cudaMemset(m->d_in, 0, (size_t)m->nshards * m->pitch * 4));
    MCK(m, cudaMemset(m->d_a, 0, (size_t)m->pitch * 4 + 64));
    MCK(m, cudaMemset(m->d_q, 0, (size_t)m->pitch * 4));
    if (P->a0) MCK(m, cudaMemcpy(m->d_a, P->a0, na * 4, cudaMemcpyHostToDevice));
    if (cudaMallocHost(&m->h_cmd, na * 4) != cudaSuccess) {
        cudaGetLastError();
        m->h_cmd = nullptr;
        return mfail(m, RTC_ENOMEM, "page-locked command buffer");
    }
    if (m->has_p) {
        // P as one column block [na][pitch_p], rows padded to 16 bytes with zeros
        const int V = elems_per_16B(m->p_dtype);
        BlockDev B{};
        B.ncols = m->na;
        B.pitch = (m->na + V - 1) / V * V;
        const size_t esz = dtype_size(m->p_dtype);
        m->p_bytes = na * (size_t)B.pitch * esz;
        rc = malloc_dev(m, &m->d_pblock, sizeof(BlockDev));
        if (rc == RTC_OK) rc = malloc_dev(m, &m->d_P, m->p_bytes);
        if (rc != RTC_OK) return rc;
        MCK(m, cudaMemcpy(m->d_pblock, &B, sizeof(BlockDev), cudaMemcpyHostToDevice));
        std::vector<unsigned char> rowed(m->p_bytes, 0);
        for (size_t r = 0; r < na; ++r)
            std::memcpy(rowed.data() + r * B.pitch * esz, static_cast<const unsigned char*>(P->P) + r * na * esz,
                        na * esz);
        MCK(m, cudaMemcpy(m->d_P, rowed.data(), m->p_bytes, cudaMemcpyHostToDevice));
        if (P->row_scale) {
            rc = malloc_dev(m, &m->d_pscale, na * 4);
            if (rc != RTC_OK) return rc;
            MCK(m, cudaMemcpy(m->d_pscale, P->row_scale, na * 4, cudaMemcpyHostToDevice));
        }
        rc = polc(m);                      // q = P a0 for the first frame
        if (rc != RTC_OK) return rc;
    }
    MCK(m, cudaStreamSynchronize(m->st));
    return RTC_OK;
}

}  // namespace

int rtc_master_create(const rtc_master_desc* desc, rtc_master** out) {
    if (!out) return mfail(nullptr, RTC_EINVAL, "out is NULL");
    *out = nullptr;
    rtc_master* m = new (std::nothrow) rtc_master();
    if (!m) return mfail(nullptr, RTC_ENOMEM, "host allocation failed");
    const int rc = create(desc, m);
    if (rc != RTC_OK) {
        g_master_err = m->err;
        release_master(m);
        return rc;
    }
    *out = m;
    return RTC_OK;
}

int rtc_master_input(rtc_master* m, int32_t shard, float** device_ptr) {
    if (!m || !device_ptr) return mfail(m, RTC_EINVAL, "master and device_ptr are required");
    if (shard < 0 || shard >= m->nshards) return mfail(m, RTC_EINVAL, "no such shard");
    *device_ptr = m->d_in + (size_t)shard * m->pitch;
    return RTC_OK;
}

int rtc_master_set_input(rtc_master* m, int32_t shard, const float* src, size_t n) {
    if (!m || !src) return mfail(m, RTC_EINVAL, "master and src are required");
    if (shard < 0 || shard >= m->nshards) return mfail(m, RTC_EINVAL, "no such shard");
    if (n != (size_t)m->na) return mfail(m, RTC_EINVAL, "an input holds na floats");
    MCK(m, cudaSetDevice(m->dev));
    MCK(m, cudaMemcpyAsync(m->d_in + (size_t)shard * m->pitch, src, n * 4, cudaMemcpyDefault, m->st));
    return RTC_OK;
}

int rtc_master_step(rtc_master* m, uint64_t frame_id) {
    if (!m) return mfail(nullptr, RTC_EINVAL, "master is NULL");
    if (m->stepped && frame_id <= m->last_id) return mfail(m, RTC_EORDER, "frame id not increasing");
    MCK(m, cudaSetDevice(m->dev));
    const int threads = 256;
    MCK(m, launch_kernel(master_kernel, dim3((m->na + threads - 1) / threads), dim3(threads), 0, m->st,
                         (const float*)m->d_in, m->nshards, m->pitch, m->na, (const float*)m->d_q, m->d_a, m->d_cmd,
                         1.0f - m->leak, m->gain, m->clip, m->amin, m->amax));
    MCK(m, cudaMemcpyAsync(m->h_cmd, m->d_cmd, (size_t)m->na * 4, cudaMemcpyDeviceToHost, m->st));
    MCK(m, cudaEventRecord(m->ev_cmd, m->st));
    const int rc = polc(m);                // for the next frame, after the commands
    if (rc != RTC_OK) return rc;
    m->last_id = frame_id;
    m->stepped = true;
    return RTC_OK;
}

int rtc_master_get_commands(rtc_master* m, float* out, size_t n, uint64_t* frame_id, int64_t timeout_us) {
    if (!m || !out) return mfail(m, RTC_EINVAL, "master and out are required");
    if (n < (size_t)m->na) return mfail(m, RTC_EINVAL, "out holds fewer than na floats");
    if (!m->stepped) return mfail(m, RTC_ENOENT, "no frame stepped yet");
    MCK(m, cudaSetDevice(m->dev));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(m->ev_cmd);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return mcuda(m, e, "cudaEventQuery");
        if (timeout_us >= 0 &&
            std::chrono::steady_clock::now() - t0 > std::chrono::microseconds(timeout_us))
            return mfail(m, RTC_ETIMEDOUT, "commands not ready");
        std::this_thread::yield();
    }
    std::memcpy(out, m->h_cmd, (size_t)m->na * 4);
    if (frame_id) *frame_id = m->last_id;
    return RTC_OK;
}

int rtc_master_destroy(rtc_master* m) {
    release_master(m);
    return RTC_OK;
}

const char* rtc_master_last_error(const rtc_master* m) {
    return m ? m->err.c_str() : g_master_err.c_str();
}
