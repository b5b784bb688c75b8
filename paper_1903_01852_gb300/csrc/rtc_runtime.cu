// Host runtime of the AO RTC library: loop objects, plans, streams, events,
// the page-locked command ring and the C ABI declared in include/rtc.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cerrno>
#include <unistd.h>

#include "rtc_internal.h"

using namespace rtc;

#ifndef RTC_SLOPE_ROWS_PER_THREAD
#define RTC_SLOPE_ROWS_PER_THREAD 12
#endif

namespace {

thread_local std::string g_err;

using Clock = std::chrono::steady_clock;

size_t round_up(size_t x, size_t m) { return (x + m - 1) / m * m; }

struct Slot {
    uint64_t frame_id = 0;
    uint64_t seq = 0;         // value of the slot's completion word once its commands are written
    bool used = false;        // holds a frame whose submission completed
    bool chunked = false;
    cudaEvent_t ev_start = nullptr, ev_tail = nullptr, ev_slopes = nullptr, ev_mvm = nullptr;
    cudaEvent_t ev_final = nullptr, ev_polc = nullptr, ev_tel = nullptr;
};

}  // namespace

struct rtc_loop {
    int dev = 0;
    uint32_t flags = 0;
    int na = 0, ns = 0, nwfs = 0, nrows = 0, nblk = 0, ring = 0;
    int m_dtype = RTC_F32, p_dtype = RTC_F32;
    float gain = 0.f, leak = 0.f, amin = 0.f, amax = 0.f;
    int clip = 0;
    bool has_polc = false, timing = false, telemetry = false, stage_timing = false;
    bool explicit_polc = false;     // s + D a formed before the reconstruction (RTC_POLC_EXPLICIT)
    bool partial = false;           // RTC_FLAG_PARTIAL: a shard, partial reconstruction only
    int stream_priority = 0;        // CUDA priority of the loop and camera streams
    float** d_pout = nullptr;       // device word: where else the shard writes its partial

    // host plans
    std::vector<rtc_wfs> wfs;
    std::vector<int> wfs_row0, wfs_nrows, wfs_blk0, wfs_nblk;
    std::vector<int> row_ready;     // per table row: pixel rows of its WFS needed
    std::vector<int> part_start;    // per table row (+1): first slope-kernel part of the row
    std::vector<int> blk_row_end;   // per block: end (exclusive) of its slope rows within the WFS
    std::vector<int2> norm_items;   // column blocks of globally normalised pyramids (block, WFS)
    std::vector<int> norm_item0, norm_nitems;   // per WFS: its range in norm_items
    int norm_max_pairs = 0;
    int2* d_norm_items = nullptr;
    std::vector<BlockDev> blocks_h;
    int max_cols = 0, smem_bytes = 0;
    uint64_t m_bytes = 0, p_bytes = 0, pixel_bytes = 0, device_bytes = 0;

    // device buffers
    void* d_M = nullptr;
    float* d_Mscale = nullptr;
    void* d_P = nullptr;
    float* d_Pscale = nullptr;
    BlockDev* d_blocks = nullptr;
    BlockDev* d_pblock = nullptr;
    std::vector<float*> d_dark, d_flat;
    WfsDev* d_wfs = nullptr;
    SlopeCta* d_ctas = nullptr;             // slope-kernel CTA table (row and part of each CTA)
    float* d_pscr = nullptr;                // per-part subaperture sums of split rows
    unsigned* d_row_cnt = nullptr;          // per slope row: parts finished
    unsigned* d_fin_cnt = nullptr;          // per finalisation tile: rows finished over blocks
    int nfin = 0;
    uint16_t* d_xlist = nullptr;
    float* d_ref = nullptr;
    std::vector<uint16_t*> d_frame;
    std::vector<long long> frame_pitch;     // uint16 elements
    float* d_s = nullptr;
    float* d_part = nullptr;
    float* d_a = nullptr;
    float* d_q = nullptr;
    void* d_D = nullptr;                    // explicit POLC: ns x na interaction matrix, one column block
    float* d_Dscale = nullptr;
    BlockDev* d_dblock = nullptr;
    float* d_u = nullptr;                   // explicit POLC: u = D a (ns, compact slope order)
    std::vector<void*> allocs;              // everything cudaMalloc'd, for destroy
    // guard bytes after the end of every allocation (rtc_check_guards): start, host or device
    std::vector<std::pair<unsigned char*, bool>> guards;

    // page-locked ring: per slot na commands then ns slopes
    float* h_ring = nullptr;
    float* d_ring = nullptr;
    unsigned long long* h_done = nullptr;   // page-locked completion words, one per slot
    unsigned long long* d_done = nullptr;
    unsigned long long* h_seq = nullptr;    // per slot: the value its frame writes to h_done (host-set)
    unsigned long long* d_seq = nullptr;
    unsigned long long* h_fid = nullptr;    // per slot: its frame id (host-set, read by the telemetry kernel)
    unsigned long long* d_fid = nullptr;
    unsigned long long* d_tdone = nullptr;  // per slot: GPU time its commands were complete (device)
    unsigned* d_tiles_done = nullptr;
    uint64_t frame_seq = 0;
    size_t slot_floats = 0;
    std::vector<Slot> slots;

    cudaStream_t st = nullptr, st_tel = nullptr;
    // per WFS: the stream its chunks' work runs on (cameras overlap on the device), and its join event
    std::vector<cudaStream_t> st_w;
    std::vector<cudaEvent_t> ev_w;
    cudaEvent_t ev_frame_end = nullptr;      // the loop stream's latest frame boundary

    // frame state (submitting thread)
    bool active = false;
    uint64_t cur_id = 0;
    bool have_last = false;
    uint64_t last_id = 0;
    int cur_slot = 0;
    uint64_t seq = 0;
    std::vector<int> rows_in, rows_done, blks_done;
    bool start_recorded = false;   // the frame's first chunk has recorded ev_start

    // completed-submission queue (shared with readers)
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int> pending;
    uint64_t frames_done = 0, frames_dropped = 0, frames_overrun = 0;

    // parameter double buffer (rtc_update): shadow copies, swapped at a frame boundary
    bool updatable = false;
    void* sh_M = nullptr;
    float* sh_Mscale = nullptr;
    void* sh_P = nullptr;
    float* sh_Pscale = nullptr;
    std::vector<float*> sh_dark, sh_flat;
    float* sh_ref = nullptr;
    WfsDev* sh_wfs = nullptr;
    std::vector<WfsDev> wfs_host;           // the active WFS table as last uploaded
    cudaStream_t st_up = nullptr;
    cudaEvent_t ev_swap = nullptr;
    // two page-locked staging buffers for the large uploads of rtc_update
    unsigned char* h_stage[2] = {nullptr, nullptr};
    cudaEvent_t ev_stage[2] = {nullptr, nullptr};
    bool stage_used[2] = {false, false};
    int stage_next = 0;
    bool swap_ev_valid = false;
    std::mutex upd_mu;                      // held by rtc_update; the submitting thread only try-locks it
    bool upd_pending = false;
    unsigned upd_mask = 0;                  // kUpd* bits of items waiting in the shadow buffers
    std::vector<char> upd_dark, upd_flat;   // per WFS
    std::vector<WfsDev> upd_table;          // WFS table after the swap
    bool upd_ctrl = false;
    float upd_gain = 0.f, upd_leak = 0.f, upd_amin = 0.f, upd_amax = 0.f;
    int upd_clip = 0;
    uint64_t swaps = 0;

    std::string err;
    bool broken = false;
    bool cuda_touched = false;   // false until creation first calls into CUDA
    bool plan_only = false;      // rtc_footprint: stop after planning, before any CUDA call
    uint64_t need_resident = 0, need_peak = 0;

    // telemetry circular buffer (tel_depth > 0): entries in page-locked memory written by the GPU
    long long tel_depth = 0;
    unsigned tel_streams = 0;
    int tel_decimate = 1;
    long long tel_entry_floats = 0;
    int tel_off_s = 0, tel_off_a = 0, tel_off_p = 0;
    float* h_tel = nullptr;
    float* d_tel = nullptr;
    unsigned long long* h_wcount = nullptr;   // entries published (page-locked, GPU-written)
    unsigned long long* d_wcount = nullptr;
    unsigned long long* d_telctr = nullptr;   // device counters of the telemetry kernel
    std::mutex tel_mu;                        // one reader at a time
    uint64_t tel_next = 0, tel_lost = 0;
    std::thread tel_thread;                   // rtc_telemetry_stream_start's drain thread
    std::atomic<bool> tel_streaming{false}, tel_stop{false};
    rtc_tel_stream_stats tel_stats{};

    // graph mode (RTC_FLAG_GRAPHS): per ring slot, page-locked input frames and a captured frame graph
    bool graphs = false;
    std::vector<std::vector<uint16_t*>> g_px;    // [slot][wfs] page-locked frame (host address = device address)
    std::vector<size_t> g_pitch;                 // [wfs] bytes
    std::vector<cudaGraphExec_t> g_exec;         // [slot]
    bool capturing = false;

    // pre-enqueued row chunks (RTC_FLAG_PRELAUNCH)
    bool prelaunch = false;
    unsigned long long pre_limit_ns = 0;
    unsigned pre_max_polls = 0;
    ChunkDesc* h_box = nullptr;                  // page-locked mailboxes, kBoxesPerWfs per WFS
    ChunkDesc* d_box = nullptr;                  // their device address
    ChunkDesc* d_box_mirror = nullptr;           // device memory: each settled mailbox, for the kernels
    std::vector<cudaEvent_t> ev_box;             // per mailbox: recorded after the kernels that read it
    std::vector<int> box_next;                   // per WFS: the mailbox its next pre-enqueued chunk takes
    struct PreChunk {
        bool pending = false;                    // kernels enqueued, mailbox not yet settled
        int row_begin = 0, row_end = 0;          // the rows they were enqueued for
        int upto = 0, bu = 0;                    // slope rows and column blocks done after them
        int box = 0;
        bool host_px = false;
    };
    std::vector<PreChunk> pre;                   // per WFS
    struct SeenChunk {
        int row_begin, row_end;
        bool in_place, host_px;
    };
    std::vector<std::vector<SeenChunk>> seen_prev, seen_cur;   // per WFS: chunks of the last two frames
    uint64_t pre_used = 0, pre_cancelled = 0, pre_expired = 0;
};

namespace {

constexpr int kBoxesPerWfs = 4;

enum : unsigned { kUpdM = 1u, kUpdMscale = 2u, kUpdP = 4u, kUpdPscale = 8u, kUpdTable = 16u, kUpdRef = 32u };

int capture_graphs(rtc_loop* L);

int fail(rtc_loop* L, int code, const std::string& msg) {
    if (L) L->err = msg;
    else g_err = msg;
    return code;
}

int cuda_fail(rtc_loop* L, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (L) L->broken = true;
    return fail(L, RTC_ECUDA, m);
}

#define CK(L, call)                                                    \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((L), e_, #call);       \
    } while (0)

int use_device(rtc_loop* L) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != L->dev) CK(L, cudaSetDevice(L->dev));
    return RTC_OK;
}

bool all_finite(const float* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Every allocation carries kGuardBytes of kGuardByte after its end; rtc_check_guards
// reports any that a kernel (or a copy) overwrote.
constexpr size_t kGuardBytes = 256;
constexpr size_t kStageBytes = size_t(32) << 20;   // each of the two upload staging buffers
constexpr unsigned char kGuardByte = 0xA5;

template <typename T>
int dev_alloc(rtc_loop* L, T** p, size_t bytes) {
    void* v = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = round_up(bytes, 16);
    cudaError_t e = cudaMalloc(&v, bytes + kGuardBytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(L, RTC_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    L->allocs.push_back(v);
    L->device_bytes += bytes + kGuardBytes;
    unsigned char* g = static_cast<unsigned char*>(v) + bytes;
    CK(L, cudaMemset(g, kGuardByte, kGuardBytes));
    L->guards.emplace_back(g, false);
    *p = static_cast<T*>(v);
    return RTC_OK;
}

// Page-locked, mapped host allocation with its guard bytes; *d: its device address.
int pinned_alloc(rtc_loop* L, void** h, void** d, size_t bytes, const char* what) {
    bytes = round_up(std::max<size_t>(bytes, 16), 16);
    if (cudaHostAlloc(h, bytes + kGuardBytes, cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        *h = nullptr;
        return fail(L, RTC_ENOMEM, std::string("page-locked ") + what + " of " + std::to_string(bytes) + " bytes");
    }
    unsigned char* g = static_cast<unsigned char*>(*h) + bytes;
    std::memset(g, kGuardByte, kGuardBytes);
    L->guards.emplace_back(g, true);
    CK(L, cudaHostGetDevicePointer(d, *h, 0));
    return RTC_OK;
}

#define TRY(expr)                  \
    do {                           \
        int r_ = (expr);           \
        if (r_ != RTC_OK) return r_; \
    } while (0)

void stop_stream(rtc_loop* L) {
    if (L->tel_thread.joinable()) {
        L->tel_stop = true;
        L->tel_thread.join();
    }
    L->tel_streaming = false;
}

// Settles a pending pre-enqueued chunk's mailbox with `to` (kChunkFilled after
// its fields were written, or kChunkCancelled).  Returns false if its kernels
// had already stopped waiting (the mailbox expired; they do nothing).
bool settle_prelaunched(rtc_loop* L, rtc_loop::PreChunk& p, int to) {
    p.pending = false;
    int expect = kChunkEmpty;
    if (__atomic_compare_exchange_n(&L->h_box[p.box].state, &expect, to, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST))
        return true;
    ++L->pre_expired;
    return false;
}

// Cancels every pending pre-enqueued chunk: its kernels end their wait and do
// nothing (a frame dropped or abandoned, the loop destroyed).
void cancel_prelaunched(rtc_loop* L) {
    for (auto& p : L->pre)
        if (p.pending && settle_prelaunched(L, p, kChunkCancelled)) ++L->pre_cancelled;
}

void release(rtc_loop* L) {
    if (!L) return;
    stop_stream(L);
    if (!L->cuda_touched) {
        delete L;
        return;
    }
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != L->dev) cudaSetDevice(L->dev);
    cancel_prelaunched(L);                   // pre-enqueued kernels stop waiting
    if (L->st) cudaStreamSynchronize(L->st);
    if (L->st_tel) cudaStreamSynchronize(L->st_tel);
    for (cudaStream_t w : L->st_w)
        if (w) cudaStreamSynchronize(w);
    for (cudaEvent_t e : L->ev_w)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t w : L->st_w)
        if (w) cudaStreamDestroy(w);
    for (cudaEvent_t e : L->ev_box)
        if (e) cudaEventDestroy(e);
    if (L->h_box) cudaFreeHost(L->h_box);
    if (L->ev_frame_end) cudaEventDestroy(L->ev_frame_end);
    for (auto& s : L->slots)
        for (cudaEvent_t e : {s.ev_start, s.ev_tail, s.ev_slopes, s.ev_mvm, s.ev_final, s.ev_polc, s.ev_tel})
            if (e) cudaEventDestroy(e);
    for (cudaGraphExec_t g : L->g_exec)
        if (g) cudaGraphExecDestroy(g);
    for (auto& v : L->g_px)
        for (uint16_t* p : v)
            if (p) cudaFreeHost(p);
    for (void* p : L->allocs) cudaFree(p);
    if (L->h_ring) cudaFreeHost(L->h_ring);
    if (L->h_done) cudaFreeHost(L->h_done);
    if (L->h_tel) cudaFreeHost(L->h_tel);
    if (L->st_up) cudaStreamSynchronize(L->st_up);
    if (L->ev_swap) cudaEventDestroy(L->ev_swap);
    for (int b = 0; b < 2; ++b) {
        if (L->ev_stage[b]) cudaEventDestroy(L->ev_stage[b]);
        if (L->h_stage[b]) cudaFreeHost(L->h_stage[b]);
    }
    if (L->st) cudaStreamDestroy(L->st);
    if (L->st_tel) cudaStreamDestroy(L->st_tel);
    if (L->st_up) cudaStreamDestroy(L->st_up);
    cudaGetLastError();
    delete L;
}

int check_wfs(const rtc_wfs& w, int k) {
    auto bad = [&](const char* what) {
        return fail(nullptr, RTC_EINVAL, "wfs " + std::to_string(k) + ": " + what);
    };
    if (w.width <= 0 || w.height <= 0 || w.width > 65536 || w.height > 65536) return bad("bad frame size");
    if (w.kind == RTC_WFS_SH) {
        if (w.npx <= 0 || w.nsubx <= 0 || w.nsuby <= 0 || w.ox < 0 || w.oy < 0) return bad("bad SH grid");
        if ((long long)w.ox + (long long)w.nsubx * w.npx > w.width ||
            (long long)w.oy + (long long)w.nsuby * w.npx > w.height)
            return bad("SH grid outside the frame");
        if (w.nsubx > 65535) return bad("too many subapertures across");
        if (w.nblocks < 1 || w.nblocks > w.nsuby) return bad("nblocks must be in [1, nsuby]");
        if (w.norm != RTC_NORM_LOCAL) return bad("norm applies to pyramid WFS only");
    } else if (w.kind == RTC_WFS_PYRAMID) {
        if (w.pupil <= 0) return bad("bad pupil size");
        for (int q = 0; q < 4; ++q)
            if (w.qx[q] < 0 || w.qy[q] < 0 || w.qx[q] + w.pupil > w.width || w.qy[q] + w.pupil > w.height)
                return bad("pupil image outside the frame");
        if (w.nblocks < 1 || w.nblocks > w.pupil) return bad("nblocks must be in [1, pupil]");
        if (w.norm != RTC_NORM_LOCAL && w.norm != RTC_NORM_GLOBAL) return bad("bad norm");
    } else {
        return bad("unknown kind");
    }
    return RTC_OK;
}

// Upload a row-major [rows][cols] host matrix of `dtype` into column blocks.
int upload_matrix(rtc_loop* L, int dtype, const void* host, int rows, int cols, const BlockDev* d_blocks,
                  const std::vector<BlockDev>& blocks, void* dst, bool check_finite) {
    const size_t esz = dtype_size(dtype);
    const size_t bytes = (size_t)rows * cols * esz;
    void* tmp = nullptr;
    if (bytes) {
        if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(L, RTC_ENOMEM, "temporary upload buffer of " + std::to_string(bytes) + " bytes");
        }
    }
    int rc = RTC_OK;
    int* d_bad = nullptr;
    cudaError_t e = cudaSuccess;
    int max_pitch = 0;
    for (auto& b : blocks) max_pitch = std::max(max_pitch, b.pitch);
    if (bytes) e = cudaMemcpy(tmp, host, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && check_finite && dtype == RTC_F32 && bytes) {
        e = cudaMalloc(&d_bad, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(d_bad, 0, sizeof(int));
        if (e == cudaSuccess) e = launch_check_finite(static_cast<const float*>(tmp), (size_t)rows * cols, d_bad, L->st);
        int bad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, L->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(L->st);
        if (e == cudaSuccess && bad) rc = fail(L, RTC_EINVAL, "matrix contains NaN or Inf");
    }
    if (e == cudaSuccess && rc == RTC_OK && max_pitch > 0)
        e = launch_relayout(dtype, tmp, rows, cols, d_blocks, (int)blocks.size(), max_pitch, dst, L->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(L->st);
    if (d_bad) cudaFree(d_bad);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(L, e, "matrix upload");
    return rc;
}

// The POLC product for the next frame from the current commands a: q = P a
// (implicit) or u = D a (explicit), on the loop stream.
int polc_product(rtc_loop* L, bool pdl) {
    if (L->has_polc)
        CK(L, launch_gemv(L->p_dtype, L->d_P, L->d_pblock, 0, 1, L->na, L->d_a, L->d_Pscale, L->d_q, 0, nullptr,
                          (long long)(L->p_bytes / std::max(L->na, 1)), pdl, L->st));
    else if (L->explicit_polc)
        CK(L, launch_gemv(L->p_dtype, L->d_D, L->d_dblock, 0, 1, L->ns, L->d_a, L->d_Dscale, L->d_u, 0, nullptr,
                          (long long)(L->p_bytes / std::max(L->ns, 1)), pdl, L->st));
    return RTC_OK;
}

int create_impl(const rtc_geometry* G, const rtc_calib* C, const rtc_cmat* M, const rtc_polc* P, rtc_loop* L) {
    if (!G || !M || !P) return fail(L, RTC_EINVAL, "geometry, cmat and polc are required");
    if (G->nwfs < 1 || G->nwfs > kMaxWfs || !G->wfs) return fail(L, RTC_EINVAL, "nwfs must be in [1, 16]");
    for (int k = 0; k < G->nwfs; ++k) TRY(check_wfs(G->wfs[k], k));
    if (M->dtype < RTC_F32 || M->dtype > RTC_E4M3 || !M->data || M->na < 1)
        return fail(L, RTC_EINVAL, "bad control matrix description");
    if (P->P && (P->dtype < RTC_F32 || P->dtype > RTC_E4M3)) return fail(L, RTC_EINVAL, "bad POLC dtype");
    if (P->mode != RTC_POLC_IMPLICIT && P->mode != RTC_POLC_EXPLICIT) return fail(L, RTC_EINVAL, "bad POLC mode");
    if (P->mode == RTC_POLC_EXPLICIT) {
        if (P->P) return fail(L, RTC_EINVAL, "explicit POLC takes D, not P");
        if (!P->D || P->d_dtype < RTC_F32 || P->d_dtype > RTC_E4M3)
            return fail(L, RTC_EINVAL, "explicit POLC needs D with a valid d_dtype");
    } else if (P->D) {
        return fail(L, RTC_EINVAL, "D is only used in explicit POLC mode");
    }
    if (!std::isfinite(P->gain) || !std::isfinite(P->leak)) return fail(L, RTC_EINVAL, "gain/leak not finite");
    if (P->clip && !(P->amin <= P->amax)) return fail(L, RTC_EINVAL, "clip needs amin <= amax");

    L->dev = G->device;
    L->flags = G->flags;
    L->stage_timing = (G->flags & RTC_FLAG_STAGE_TIMING) != 0;
    L->updatable = (G->flags & RTC_FLAG_UPDATABLE) != 0;
    L->timing = (G->flags & RTC_FLAG_TIMING) != 0 || L->stage_timing;
    L->telemetry = (G->flags & RTC_FLAG_TELEMETRY) != 0;
    L->ring = G->ring > 0 ? G->ring : 4;
    if (L->ring < 2 || L->ring > 1024) return fail(L, RTC_EINVAL, "ring must be in [2, 1024]");
    L->nwfs = G->nwfs;
    L->na = M->na;
    L->m_dtype = M->dtype;
    L->explicit_polc = P->mode == RTC_POLC_EXPLICIT;
    L->p_dtype = P->P ? P->dtype : L->explicit_polc ? P->d_dtype : RTC_F32;
    L->has_polc = P->P != nullptr;
    L->gain = P->gain;
    L->leak = P->leak;
    L->clip = P->clip;
    L->amin = P->amin;
    L->amax = P->amax;
    L->graphs = (G->flags & RTC_FLAG_GRAPHS) != 0;
    L->partial = (G->flags & RTC_FLAG_PARTIAL) != 0;
    if (G->priority < 0) return fail(L, RTC_EINVAL, "priority must be >= 0");
    if (L->partial && (P->P || P->D || L->explicit_polc))
        return fail(L, RTC_EINVAL, "a RTC_FLAG_PARTIAL loop takes no POLC matrix (the master applies it)");
    if (G->tel_depth < 0 || G->tel_depth > (1 << 20)) return fail(L, RTC_EINVAL, "tel_depth must be in [0, 2^20]");
    if (G->tel_decimate < 0) return fail(L, RTC_EINVAL, "tel_decimate must be >= 0");
    if (G->tel_streams & ~(RTC_TEL_SLOPES | RTC_TEL_COMMANDS | RTC_TEL_PARTIALS))
        return fail(L, RTC_EINVAL, "unknown tel_streams bits");
    L->tel_depth = G->tel_depth;
    L->tel_streams = G->tel_depth ? G->tel_streams : 0u;
    L->tel_decimate = G->tel_decimate > 0 ? G->tel_decimate : 1;
    if (L->graphs && L->updatable) return fail(L, RTC_EINVAL, "RTC_FLAG_GRAPHS and RTC_FLAG_UPDATABLE exclude each other");
    if (L->graphs && L->stage_timing)
        return fail(L, RTC_EINVAL, "RTC_FLAG_GRAPHS and RTC_FLAG_STAGE_TIMING exclude each other");
    L->prelaunch = (G->flags & RTC_FLAG_PRELAUNCH) != 0;
    if (G->prelaunch_wait_us < 0 || G->prelaunch_wait_us > 1000000)
        return fail(L, RTC_EINVAL, "prelaunch_wait_us must be in [0, 1000000]");
    if (L->prelaunch && L->timing)
        return fail(L, RTC_EINVAL, "RTC_FLAG_PRELAUNCH excludes RTC_FLAG_TIMING and RTC_FLAG_STAGE_TIMING");
    {
        const unsigned long long wait_us = G->prelaunch_wait_us > 0 ? (unsigned long long)G->prelaunch_wait_us : 10000ull;
        L->pre_limit_ns = wait_us * 1000ull;
        L->pre_max_polls = (unsigned)(16 * wait_us + 64);   // a poll (a read over the link) takes longer than 1/16 us
    }

    // ---- slope-row and block plans ------------------------------------
    const int V = elems_per_16B(L->m_dtype);
    std::vector<SlopeRow> rows;
    std::vector<uint16_t> xlist;
    std::vector<WfsDev> wdev(L->nwfs);
    int compact = 0;
    long long m_off = 0;
    int x_off = 0;
    L->wfs.assign(G->wfs, G->wfs + G->nwfs);
    for (int k = 0; k < L->nwfs; ++k) {
        const rtc_wfs& w = L->wfs[k];
        const bool sh = w.kind == RTC_WFS_SH;
        const int nr = sh ? w.nsuby : w.pupil;
        const int nc = sh ? w.nsubx : w.pupil;
        std::vector<int> units(nr);
        std::vector<std::vector<uint16_t>> row_x(nr);
        for (int i = 0; i < nr; ++i)
            for (int j = 0; j < nc; ++j)
                if (!w.valid || w.valid[(size_t)i * nc + j]) row_x[i].push_back((uint16_t)j);
        L->wfs_row0.push_back((int)rows.size());
        L->wfs_nrows.push_back(nr);
        L->wfs_blk0.push_back((int)L->blocks_h.size());
        L->wfs_nblk.push_back(w.nblocks);
        for (int b = 0; b < w.nblocks; ++b) {
            const int r0 = (int)((long long)b * nr / w.nblocks), r1 = (int)((long long)(b + 1) * nr / w.nblocks);
            BlockDev B{};
            B.m_off = m_off;
            B.x_off = x_off;
            B.c0 = compact;
            int local = 0;
            for (int i = r0; i < r1; ++i) {
                SlopeRow R{};
                R.wfs = k;
                R.row = i;
                R.unit0 = (int)xlist.size();
                R.nunits = (int)row_x[i].size();
                R.s_pad = x_off + local;
                R.s_compact = compact + local;
                rows.push_back(R);
                const int qlast = *std::max_element(w.qy, w.qy + 4);
                L->row_ready.push_back(sh ? w.oy + (i + 1) * w.npx
                                          : qlast + (w.norm == RTC_NORM_GLOBAL ? w.pupil : i + 1));
                xlist.insert(xlist.end(), row_x[i].begin(), row_x[i].end());
                local += 2 * R.nunits;
            }
            B.ncols = local;
            B.pitch = (int)round_up((size_t)local, (size_t)V);
            compact += local;
            x_off += B.pitch;
            m_off += (long long)L->na * B.pitch;
            L->blk_row_end.push_back(r1);
            L->blocks_h.push_back(B);
            L->max_cols = std::max(L->max_cols, B.ncols);
        }
        WfsDev& D = wdev[k];
        D.kind = w.kind;
        D.width = w.width;
        D.height = w.height;
        D.npx = w.npx;
        D.nsubx = w.nsubx;
        D.nsuby = w.nsuby;
        D.ox = w.ox;
        D.oy = w.oy;
        D.pupil = w.pupil;
        for (int q = 0; q < 4; ++q) { D.qx[q] = w.qx[q]; D.qy[q] = w.qy[q]; }
        D.threshold = (C && C->threshold) ? C->threshold[k] : 0.f;
        D.thresh_mode = (C && C->thresh_mode) ? C->thresh_mode[k] : RTC_THRESH_SUBTRACT;
        if (!(D.threshold >= 0.f) || !std::isfinite(D.threshold)) return fail(L, RTC_EINVAL, "threshold must be finite and >= 0");
        if (D.thresh_mode != RTC_THRESH_SUBTRACT && D.thresh_mode != RTC_THRESH_CLIP)
            return fail(L, RTC_EINVAL, "bad threshold mode");
        D.calib_pitch = (int)round_up((size_t)w.width, 4);
        D.norm = sh ? RTC_NORM_LOCAL : w.norm;
        D.gnrows = nr;
        D.gpix = 0;
        for (int i = 0; i < nr; ++i) D.gpix += (int)row_x[i].size();
        if (sh) {
            const int ws = w.nsubx * w.npx;
            const int nq = ((w.ox + ws + 3) >> 2) - (w.ox >> 2);
            D.sh_groups = std::max(1, std::min(w.npx, kSlopeThreads / nq));
            L->smem_bytes = std::max(L->smem_bytes, (int)(2 * D.sh_groups * ws * sizeof(float)));
            L->pixel_bytes += (size_t)w.nsuby * w.npx * (size_t)nq * 4 * (2 + 8);
        }
    }
    // pyramid pixel bytes: 4 pixels x (2 + 8) bytes per valid unit
    for (int k = 0; k < L->nwfs; ++k)
        if (L->wfs[k].kind == RTC_WFS_PYRAMID) {
            size_t n = 0;
            for (int r = L->wfs_row0[k]; r < L->wfs_row0[k] + L->wfs_nrows[k]; ++r) n += rows[r].nunits;
            L->pixel_bytes += n * 4 * (2 + 8);
        }
    L->nrows = (int)rows.size();
    L->nblk = (int)L->blocks_h.size();
    // Slope-kernel parts: an SH subaperture row is split by pixel rows so that no
    // thread of its CTA loads more than RTC_SLOPE_ROWS_PER_THREAD rows of one quad column.
    std::vector<SlopePart> parts;
    size_t pscr_floats = 0;
    for (int r = 0; r < L->nrows; ++r) {
        SlopeRow& R = rows[r];
        const rtc_wfs& w = L->wfs[R.wfs];
        int np = 1;
        if (w.kind == RTC_WFS_SH) {
            const int nq = ((w.ox + w.nsubx * w.npx + 3) >> 2) - (w.ox >> 2);
            const int gfull = std::max(1, kSlopeThreads / nq);
            const int rpt = RTC_SLOPE_ROWS_PER_THREAD;
            np = std::min(w.npx, std::max(1, (w.npx + rpt * gfull - 1) / (rpt * gfull)));
        }
        R.nparts = np;
        R.pscr = (int)pscr_floats;
        if (np > 1) pscr_floats += (size_t)np * R.nunits * 3;
        L->part_start.push_back((int)parts.size());
        for (int k = 0; k < np; ++k) {
            SlopePart P{};
            P.row = r;
            P.part = k;
            P.pr0 = w.kind == RTC_WFS_SH ? (k * w.npx) / np : 0;
            P.pr1 = w.kind == RTC_WFS_SH ? ((k + 1) * w.npx) / np : 0;
            parts.push_back(P);
        }
    }
    L->part_start.push_back((int)parts.size());
    // globally normalised pyramids: per-row flux sums, and their column blocks for the normalisation kernel
    L->norm_item0.assign(L->nwfs, 0);
    L->norm_nitems.assign(L->nwfs, 0);
    for (int k = 0; k < L->nwfs; ++k) {
        L->norm_item0[k] = (int)L->norm_items.size();
        if (wdev[k].norm != RTC_NORM_GLOBAL) continue;
        wdev[k].gflux = (int)pscr_floats;
        pscr_floats += (size_t)wdev[k].gnrows;
        for (int b = L->wfs_blk0[k]; b < L->wfs_blk0[k] + L->wfs_nblk[k]; ++b) {
            L->norm_items.push_back(int2{b, k});
            L->norm_max_pairs = std::max(L->norm_max_pairs, L->blocks_h[b].ncols / 2);
        }
        L->norm_nitems[k] = L->wfs_nblk[k];
    }
    L->nfin = (L->na + kFinRows - 1) / kFinRows;
    L->ns = compact;
    if (M->ns != L->ns)
        return fail(L, RTC_EINVAL, "cmat ns = " + std::to_string(M->ns) + " but the geometry has " +
                                       std::to_string(L->ns) + " slopes");
    if (L->smem_bytes > 200 * 1024) return fail(L, RTC_EINVAL, "subaperture strip too wide for shared memory");
    if (L->smem_bytes < 16) L->smem_bytes = 16;
    const int s_len = std::max(x_off, 4);
    const int VP = elems_per_16B(L->p_dtype);
    const int a_len = (int)round_up((size_t)L->na, 16);
    L->m_bytes = (uint64_t)m_off * dtype_size(L->m_dtype);

    // ---- host-side checks of the maps --------------------------------
    if (C && C->ref_slopes && !all_finite(C->ref_slopes, L->ns)) return fail(L, RTC_EINVAL, "ref_slopes not finite");
    if (M->row_scale && !all_finite(M->row_scale, L->na)) return fail(L, RTC_EINVAL, "row_scale not finite");
    if (P->P && P->row_scale && !all_finite(P->row_scale, L->na)) return fail(L, RTC_EINVAL, "P row_scale not finite");
    if (P->D && P->d_row_scale && !all_finite(P->d_row_scale, L->ns))
        return fail(L, RTC_EINVAL, "D row_scale not finite");
    if (P->a0 && !all_finite(P->a0, L->na)) return fail(L, RTC_EINVAL, "a0 not finite");
    for (int k = 0; k < L->nwfs; ++k) {
        const size_t n = (size_t)L->wfs[k].width * L->wfs[k].height;
        if (C && C->dark && C->dark[k] && !all_finite(C->dark[k], n)) return fail(L, RTC_EINVAL, "dark map not finite");
        if (C && C->flat && C->flat[k] && !all_finite(C->flat[k], n)) return fail(L, RTC_EINVAL, "flat map not finite");
    }

    // ---- HBM admission --------------------------------------------------
    size_t need = L->m_bytes + (size_t)L->na * M->ns * dtype_size(L->m_dtype);  // stored + upload temporary
    if (L->has_polc) need += (size_t)L->na * round_up(L->na, VP) * dtype_size(L->p_dtype) * 2;
    if (L->explicit_polc) need += (size_t)L->ns * round_up(L->na, VP) * dtype_size(L->p_dtype) * 2 + (size_t)L->ns * 8;
    for (auto& w : L->wfs) need += (size_t)w.height * (round_up(w.width, 4) * 8 + round_up(w.width, 8) * 2);
    need += (size_t)L->nblk * L->na * 4 + (size_t)s_len * 4 + (size_t)a_len * 8;
    if (L->updatable) {
        need += L->m_bytes;
        if (L->has_polc) need += (size_t)L->na * round_up(L->na, VP) * dtype_size(L->p_dtype);
        for (auto& w : L->wfs) need += (size_t)w.height * round_up(w.width, 4) * 8;
    }
    const size_t temporary = (size_t)L->na * M->ns * dtype_size(L->m_dtype) +
                             (L->has_polc ? (size_t)L->na * round_up(L->na, VP) * dtype_size(L->p_dtype) : 0) +
                             (L->explicit_polc ? (size_t)L->ns * round_up(L->na, VP) * dtype_size(L->p_dtype) : 0);
    L->need_peak = need;
    L->need_resident = need - temporary;
    if (L->plan_only) return RTC_OK;

    L->cuda_touched = true;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || L->dev < 0 || L->dev >= ndev) {
        cudaGetLastError();
        return fail(L, RTC_EINVAL, "no such CUDA device");
    }
    CK(L, cudaSetDevice(L->dev));
    size_t free_b = 0, total_b = 0;
    CK(L, cudaMemGetInfo(&free_b, &total_b));
    if (need + (64u << 20) > free_b)
        return fail(L, RTC_ENOMEM, "loop needs " + std::to_string(need) + " bytes of device memory, " +
                                       std::to_string(free_b) + " free");

    CK(L, configure_slopes(L->smem_bytes));
    // stream priority: the device's greatest, lowered by geometry->priority steps
    int least = 0, greatest = 0;
    CK(L, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    L->stream_priority = std::min(least, greatest + std::max(0, G->priority));
    CK(L, cudaStreamCreateWithPriority(&L->st, cudaStreamNonBlocking, L->stream_priority));
    CK(L, cudaStreamCreateWithFlags(&L->st_tel, cudaStreamNonBlocking));
    L->st_w.assign(L->nwfs, nullptr);
    L->ev_w.assign(L->nwfs, nullptr);
    for (int k = 0; k < L->nwfs; ++k) {
        CK(L, cudaStreamCreateWithPriority(&L->st_w[k], cudaStreamNonBlocking, L->stream_priority));
        CK(L, cudaEventCreateWithFlags(&L->ev_w[k], cudaEventDisableTiming));
    }
    CK(L, cudaEventCreateWithFlags(&L->ev_frame_end, cudaEventDisableTiming));
    if (L->prelaunch) {
        // the mailbox handshake is a compare-and-swap by both the CPU and the GPU on page-locked memory
        int native = 0;
        CK(L, cudaDeviceGetAttribute(&native, cudaDevAttrHostNativeAtomicSupported, L->dev));
        if (!native) return fail(L, RTC_ENOTSUP, "RTC_FLAG_PRELAUNCH needs native GPU atomics on host memory");
        const size_t nbox = (size_t)L->nwfs * kBoxesPerWfs;
        CK(L, cudaHostAlloc(reinterpret_cast<void**>(&L->h_box), nbox * sizeof(ChunkDesc), cudaHostAllocMapped));
        std::memset(static_cast<void*>(L->h_box), 0, nbox * sizeof(ChunkDesc));
        void* dv = nullptr;
        CK(L, cudaHostGetDevicePointer(&dv, L->h_box, 0));
        L->d_box = static_cast<ChunkDesc*>(dv);
        TRY(dev_alloc(L, &L->d_box_mirror, nbox * sizeof(ChunkDesc)));
        L->ev_box.assign(nbox, nullptr);
        for (cudaEvent_t& e : L->ev_box) CK(L, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        L->box_next.assign(L->nwfs, 0);
        L->pre.assign(L->nwfs, rtc_loop::PreChunk{});
        L->seen_prev.assign(L->nwfs, {});
        L->seen_cur.assign(L->nwfs, {});
    }

    // ---- device buffers ---------------------------------------------------
    TRY(dev_alloc(L, &L->d_blocks, L->blocks_h.size() * sizeof(BlockDev)));
    CK(L, cudaMemcpy(L->d_blocks, L->blocks_h.data(), L->blocks_h.size() * sizeof(BlockDev), cudaMemcpyHostToDevice));
    TRY(dev_alloc(L, &L->d_M, L->m_bytes));
    TRY(upload_matrix(L, L->m_dtype, M->data, L->na, L->ns, L->d_blocks, L->blocks_h, L->d_M, true));
    if (M->row_scale) {
        TRY(dev_alloc(L, &L->d_Mscale, (size_t)L->na * 4));
        CK(L, cudaMemcpy(L->d_Mscale, M->row_scale, (size_t)L->na * 4, cudaMemcpyHostToDevice));
    }
    if (L->has_polc) {
        BlockDev PB{};
        PB.m_off = 0;
        PB.x_off = 0;
        PB.ncols = L->na;
        PB.pitch = (int)round_up((size_t)L->na, VP);
        PB.c0 = 0;
        L->p_bytes = (uint64_t)L->na * PB.pitch * dtype_size(L->p_dtype);
        TRY(dev_alloc(L, &L->d_pblock, sizeof(BlockDev)));
        CK(L, cudaMemcpy(L->d_pblock, &PB, sizeof(BlockDev), cudaMemcpyHostToDevice));
        TRY(dev_alloc(L, &L->d_P, L->p_bytes));
        TRY(upload_matrix(L, L->p_dtype, P->P, L->na, L->na, L->d_pblock, std::vector<BlockDev>{PB}, L->d_P, true));
        if (P->row_scale) {
            TRY(dev_alloc(L, &L->d_Pscale, (size_t)L->na * 4));
            CK(L, cudaMemcpy(L->d_Pscale, P->row_scale, (size_t)L->na * 4, cudaMemcpyHostToDevice));
        }
    }
    if (L->explicit_polc) {
        BlockDev DB{};
        DB.ncols = L->na;
        DB.pitch = (int)round_up((size_t)L->na, VP);
        L->p_bytes = (uint64_t)L->ns * DB.pitch * dtype_size(L->p_dtype);
        TRY(dev_alloc(L, &L->d_dblock, sizeof(BlockDev)));
        CK(L, cudaMemcpy(L->d_dblock, &DB, sizeof(BlockDev), cudaMemcpyHostToDevice));
        TRY(dev_alloc(L, &L->d_D, L->p_bytes));
        TRY(upload_matrix(L, L->p_dtype, P->D, L->ns, L->na, L->d_dblock, std::vector<BlockDev>{DB}, L->d_D, true));
        if (P->d_row_scale) {
            TRY(dev_alloc(L, &L->d_Dscale, (size_t)L->ns * 4));
            CK(L, cudaMemcpy(L->d_Dscale, P->d_row_scale, (size_t)L->ns * 4, cudaMemcpyHostToDevice));
        }
        TRY(dev_alloc(L, &L->d_u, (size_t)L->ns * 4));
        CK(L, cudaMemset(L->d_u, 0, (size_t)L->ns * 4));
    }
    // calibration maps and frame buffers
    L->d_dark.resize(L->nwfs);
    L->d_flat.resize(L->nwfs);
    L->d_frame.resize(L->nwfs);
    L->frame_pitch.resize(L->nwfs);
    for (int k = 0; k < L->nwfs; ++k) {
        const rtc_wfs& w = L->wfs[k];
        const size_t cp = round_up(w.width, 4);
        TRY(dev_alloc(L, &L->d_dark[k], (size_t)w.height * cp * 4));
        TRY(dev_alloc(L, &L->d_flat[k], (size_t)w.height * cp * 4));
        CK(L, cudaMemset(L->d_dark[k], 0, (size_t)w.height * cp * 4));
        const float* dk = (C && C->dark) ? C->dark[k] : nullptr;
        const float* fl = (C && C->flat) ? C->flat[k] : nullptr;
        if (dk) CK(L, cudaMemcpy2D(L->d_dark[k], cp * 4, dk, (size_t)w.width * 4, (size_t)w.width * 4, w.height,
                                   cudaMemcpyHostToDevice));
        std::vector<float> ones;
        if (!fl) {
            ones.assign((size_t)w.height * cp, 1.0f);
            CK(L, cudaMemcpy(L->d_flat[k], ones.data(), ones.size() * 4, cudaMemcpyHostToDevice));
        } else {
            CK(L, cudaMemset(L->d_flat[k], 0, (size_t)w.height * cp * 4));
            CK(L, cudaMemcpy2D(L->d_flat[k], cp * 4, fl, (size_t)w.width * 4, (size_t)w.width * 4, w.height,
                               cudaMemcpyHostToDevice));
        }
        wdev[k].dark = L->d_dark[k];
        wdev[k].flat = L->d_flat[k];
        const size_t fp = round_up(w.width, 8);
        L->frame_pitch[k] = (long long)fp;
        TRY(dev_alloc(L, &L->d_frame[k], (size_t)w.height * fp * 2));
        CK(L, cudaMemset(L->d_frame[k], 0, (size_t)w.height * fp * 2));
    }
    if (L->updatable && !L->d_ref) {           // reference slopes become updatable: start from zeros
        TRY(dev_alloc(L, &L->d_ref, (size_t)L->ns * 4));
        CK(L, cudaMemset(L->d_ref, 0, (size_t)L->ns * 4));
    }
    TRY(dev_alloc(L, &L->d_wfs, wdev.size() * sizeof(WfsDev)));
    CK(L, cudaMemcpy(L->d_wfs, wdev.data(), wdev.size() * sizeof(WfsDev), cudaMemcpyHostToDevice));
    L->wfs_host = wdev;
    if (L->updatable) {
        TRY(dev_alloc(L, &L->sh_M, std::max<uint64_t>(L->m_bytes, 16)));
        CK(L, cudaMemset(L->sh_M, 0, std::max<uint64_t>(L->m_bytes, 16)));
        if (L->d_Mscale) TRY(dev_alloc(L, &L->sh_Mscale, (size_t)L->na * 4));
        if (L->has_polc) {
            TRY(dev_alloc(L, &L->sh_P, L->p_bytes));
            CK(L, cudaMemset(L->sh_P, 0, L->p_bytes));
            if (L->d_Pscale) TRY(dev_alloc(L, &L->sh_Pscale, (size_t)L->na * 4));
        }
        L->sh_dark.resize(L->nwfs);
        L->sh_flat.resize(L->nwfs);
        for (int k = 0; k < L->nwfs; ++k) {
            const size_t bytes = (size_t)L->wfs[k].height * round_up(L->wfs[k].width, 4) * 4;
            TRY(dev_alloc(L, &L->sh_dark[k], bytes));
            TRY(dev_alloc(L, &L->sh_flat[k], bytes));
            CK(L, cudaMemset(L->sh_dark[k], 0, bytes));
            CK(L, cudaMemset(L->sh_flat[k], 0, bytes));
        }
        TRY(dev_alloc(L, &L->sh_ref, (size_t)L->ns * 4));
        TRY(dev_alloc(L, &L->sh_wfs, wdev.size() * sizeof(WfsDev)));
        CK(L, cudaStreamCreateWithPriority(&L->st_up, cudaStreamNonBlocking, 0));
        CK(L, cudaEventCreateWithFlags(&L->ev_swap, cudaEventDisableTiming));
        for (int b = 0; b < 2; ++b) {
            void* dv = nullptr;
            void* hv = nullptr;
            const int rc = pinned_alloc(L, &hv, &dv, kStageBytes, "upload staging buffer");
            L->h_stage[b] = static_cast<unsigned char*>(hv);
            TRY(rc);
            CK(L, cudaEventCreateWithFlags(&L->ev_stage[b], cudaEventDisableTiming));
        }
        L->upd_dark.assign(L->nwfs, 0);
        L->upd_flat.assign(L->nwfs, 0);
    }
    {
        std::vector<SlopeCta> ctas(parts.size());
        for (size_t i = 0; i < parts.size(); ++i) {
            ctas[i].row = rows[parts[i].row];
            ctas[i].part = parts[i];
        }
        TRY(dev_alloc(L, &L->d_ctas, ctas.size() * sizeof(SlopeCta)));
        CK(L, cudaMemcpy(L->d_ctas, ctas.data(), ctas.size() * sizeof(SlopeCta), cudaMemcpyHostToDevice));
    }
    TRY(dev_alloc(L, &L->d_pscr, std::max<size_t>(pscr_floats, 4) * 4));
    TRY(dev_alloc(L, &L->d_row_cnt, (size_t)L->nrows * sizeof(unsigned)));
    CK(L, cudaMemset(L->d_row_cnt, 0, (size_t)L->nrows * sizeof(unsigned)));
    TRY(dev_alloc(L, &L->d_fin_cnt, (size_t)L->nfin * sizeof(unsigned)));
    CK(L, cudaMemset(L->d_fin_cnt, 0, (size_t)L->nfin * sizeof(unsigned)));
    if (!L->norm_items.empty()) {
        TRY(dev_alloc(L, &L->d_norm_items, L->norm_items.size() * sizeof(int2)));
        CK(L, cudaMemcpy(L->d_norm_items, L->norm_items.data(), L->norm_items.size() * sizeof(int2),
                         cudaMemcpyHostToDevice));
    }
    TRY(dev_alloc(L, &L->d_xlist, std::max<size_t>(xlist.size(), 1) * 2));
    if (!xlist.empty()) CK(L, cudaMemcpy(L->d_xlist, xlist.data(), xlist.size() * 2, cudaMemcpyHostToDevice));
    if (C && C->ref_slopes) {
        TRY(dev_alloc(L, &L->d_ref, (size_t)L->ns * 4));
        CK(L, cudaMemcpy(L->d_ref, C->ref_slopes, (size_t)L->ns * 4, cudaMemcpyHostToDevice));
    }
    TRY(dev_alloc(L, &L->d_s, (size_t)s_len * 4));
    CK(L, cudaMemset(L->d_s, 0, (size_t)s_len * 4));
    TRY(dev_alloc(L, &L->d_part, (size_t)std::max(L->nblk, 1) * L->na * 4));
    CK(L, cudaMemset(L->d_part, 0, (size_t)std::max(L->nblk, 1) * L->na * 4));
    TRY(dev_alloc(L, &L->d_a, (size_t)std::max(a_len, (int)round_up(L->na, VP)) * 4));
    CK(L, cudaMemset(L->d_a, 0, (size_t)std::max(a_len, (int)round_up(L->na, VP)) * 4));
    if (P->a0) CK(L, cudaMemcpy(L->d_a, P->a0, (size_t)L->na * 4, cudaMemcpyHostToDevice));
    TRY(dev_alloc(L, &L->d_q, (size_t)L->na * 4));
    CK(L, cudaMemset(L->d_q, 0, (size_t)L->na * 4));
    TRY(polc_product(L, false));

    // ---- page-locked ring, events -------------------------------------------
    L->slot_floats = round_up((size_t)L->na, 4) + round_up((size_t)L->ns, 4);
    {
        void *h = nullptr, *d = nullptr;
        const int rc = pinned_alloc(L, &h, &d, (size_t)L->ring * L->slot_floats * 4, "command ring");
        L->h_ring = static_cast<float*>(h);
        TRY(rc);
        std::memset(L->h_ring, 0, (size_t)L->ring * L->slot_floats * 4);
        L->d_ring = static_cast<float*>(d);
    }
    {
        void *h = nullptr, *d = nullptr;
        // per slot: completion word, its expected value, frame id; then the telemetry count
        const size_t words = 3 * (size_t)L->ring + 1;
        const int rc = pinned_alloc(L, &h, &d, words * sizeof(unsigned long long), "completion words");
        L->h_done = static_cast<unsigned long long*>(h);
        TRY(rc);
        L->h_seq = L->h_done + L->ring;
        L->h_fid = L->h_seq + L->ring;
        L->h_wcount = L->h_fid + L->ring;
        std::memset(h, 0, words * sizeof(unsigned long long));
        L->d_done = static_cast<unsigned long long*>(d);
        L->d_seq = L->d_done + L->ring;
        L->d_fid = L->d_seq + L->ring;
        L->d_wcount = L->d_fid + L->ring;
    }
    TRY(dev_alloc(L, &L->d_tdone, (size_t)L->ring * sizeof(unsigned long long)));
    CK(L, cudaMemset(L->d_tdone, 0, (size_t)L->ring * sizeof(unsigned long long)));
    if (L->tel_depth) {
        auto r4 = [](long long n) { return (n + 3) / 4 * 4; };
        long long off = 0;
        if (L->tel_streams & RTC_TEL_SLOPES) { L->tel_off_s = (int)off; off += r4(L->ns); }
        if (L->tel_streams & RTC_TEL_COMMANDS) { L->tel_off_a = (int)off; off += r4(L->na); }
        if (L->tel_streams & RTC_TEL_PARTIALS) { L->tel_off_p = (int)off; off += r4((long long)L->nwfs * L->na); }
        L->tel_entry_floats = kTelHeaderFloats + off;
        const size_t bytes = (size_t)L->tel_depth * L->tel_entry_floats * 4;
        void *h = nullptr, *d = nullptr;
        const int rc = pinned_alloc(L, &h, &d, bytes, "telemetry buffer");
        L->h_tel = static_cast<float*>(h);
        TRY(rc);
        std::memset(h, 0xff, bytes);          // no entry valid yet (index all ones)
        L->d_tel = static_cast<float*>(d);
        TRY(dev_alloc(L, &L->d_telctr, 3 * sizeof(unsigned long long)));
        CK(L, cudaMemset(L->d_telctr, 0, 3 * sizeof(unsigned long long)));
    }
    TRY(dev_alloc(L, &L->d_tiles_done, sizeof(unsigned)));
    CK(L, cudaMemset(L->d_tiles_done, 0, sizeof(unsigned)));
    TRY(dev_alloc(L, &L->d_pout, sizeof(float*)));
    CK(L, cudaMemset(L->d_pout, 0, sizeof(float*)));
    L->slots.resize(L->ring);
    const unsigned evflags = L->timing ? cudaEventDefault : cudaEventDisableTiming;
    for (auto& s : L->slots) {
        CK(L, cudaEventCreateWithFlags(&s.ev_polc, evflags));
        CK(L, cudaEventCreateWithFlags(&s.ev_tel, cudaEventDisableTiming));
        if (L->timing) {
            CK(L, cudaEventCreate(&s.ev_start));
            CK(L, cudaEventCreate(&s.ev_tail));
            CK(L, cudaEventCreate(&s.ev_final));
            CK(L, cudaEventCreate(&s.ev_slopes));
            CK(L, cudaEventCreate(&s.ev_mvm));
        }
    }
    L->rows_in.assign(L->nwfs, 0);
    L->rows_done.assign(L->nwfs, 0);
    L->blks_done.assign(L->nwfs, 0);
    CK(L, cudaStreamSynchronize(L->st));
    if (L->graphs) TRY(capture_graphs(L));
    return RTC_OK;
}

// Frame boundary: exchange the active and shadow pointers of every item a
// finished rtc_update left pending (no GPU work), and remember where the old
// buffers stop being read.  Skipped while an update is still uploading.
int apply_pending_update(rtc_loop* L) {
    if (!L->updatable) return RTC_OK;
    std::unique_lock<std::mutex> g(L->upd_mu, std::try_to_lock);
    if (!g.owns_lock() || !L->upd_pending) return RTC_OK;
    const unsigned m = L->upd_mask;
    if (m & kUpdM) std::swap(L->d_M, L->sh_M);
    if (m & kUpdMscale) std::swap(L->d_Mscale, L->sh_Mscale);
    if (m & kUpdP) std::swap(L->d_P, L->sh_P);
    if (m & kUpdPscale) std::swap(L->d_Pscale, L->sh_Pscale);
    if (m & kUpdRef) std::swap(L->d_ref, L->sh_ref);
    if (m & kUpdTable) {
        for (int k = 0; k < L->nwfs; ++k) {
            if (L->upd_dark[k]) std::swap(L->d_dark[k], L->sh_dark[k]);
            if (L->upd_flat[k]) std::swap(L->d_flat[k], L->sh_flat[k]);
        }
        std::swap(L->d_wfs, L->sh_wfs);
        L->wfs_host = L->upd_table;
    }
    if (L->upd_ctrl) {
        L->gain = L->upd_gain;
        L->leak = L->upd_leak;
        L->clip = L->upd_clip;
        L->amin = L->upd_amin;
        L->amax = L->upd_amax;
    }
    std::fill(L->upd_dark.begin(), L->upd_dark.end(), 0);
    std::fill(L->upd_flat.begin(), L->upd_flat.end(), 0);
    L->upd_mask = 0;
    L->upd_ctrl = false;
    L->upd_pending = false;
    ++L->swaps;
    CK(L, cudaEventRecord(L->ev_swap, L->st));   // frames before this point read the old buffers
    L->swap_ev_valid = true;
    return RTC_OK;
}

// Wait until the GPU no longer uses what the slot's previous frame left there:
// its commands (and the input frames of graph mode) once its POLC product has
// run; with a telemetry buffer, also its frame id, until its entry is written.
int slot_wait(rtc_loop* L, const Slot& prev, int slot) {
    if (!prev.seq) return RTC_OK;
    if (L->h_done[slot] != prev.seq) CK(L, cudaEventSynchronize(prev.ev_polc));
    if (L->tel_depth) CK(L, cudaEventSynchronize(prev.ev_tel));
    return RTC_OK;
}

// Start a frame: pick its ring slot (discarding an unread frame that still holds it,
// and waiting for the GPU to finish a frame that still uses it).
int begin_frame(rtc_loop* L, uint64_t id, bool chunked) {
    L->active = chunked;
    L->cur_id = id;
    L->cur_slot = (int)(L->seq % (uint64_t)L->ring);
    {
        Slot& prev = L->slots[L->cur_slot];
        TRY(slot_wait(L, prev, L->cur_slot));
    }
    {
        std::lock_guard<std::mutex> g(L->mu);
        auto it = std::find(L->pending.begin(), L->pending.end(), L->cur_slot);
        if (it != L->pending.end()) {
            L->pending.erase(it);
            ++L->frames_overrun;
        }
        Slot& s = L->slots[L->cur_slot];
        s.used = false;
        s.frame_id = id;
        s.chunked = chunked;
        s.seq = ++L->frame_seq;
        L->h_seq[L->cur_slot] = s.seq;
        L->h_fid[L->cur_slot] = id;
    }
    std::fill(L->rows_in.begin(), L->rows_in.end(), 0);
    std::fill(L->rows_done.begin(), L->rows_done.end(), 0);
    std::fill(L->blks_done.begin(), L->blks_done.end(), 0);
    L->start_recorded = false;
    if (L->prelaunch) {
        cancel_prelaunched(L);     // none is pending between frames; kept as a guard
        for (int k = 0; k < L->nwfs; ++k) {
            L->seen_prev[k].swap(L->seen_cur[k]);
            L->seen_cur[k].clear();
        }
    }
    return RTC_OK;
}

// Event record.  Inside a stream capture it only marks a fork/join point of the
// graph; graph launches record the slot's events again after the launch.
int record(rtc_loop* L, cudaEvent_t e, cudaStream_t st) {
    CK(L, cudaEventRecord(e, st));
    return RTC_OK;
}

TelArgs tel_args(rtc_loop* L) {
    TelArgs t{};
    t.blocks = L->d_blocks;
    t.nblk = L->nblk;
    t.na = L->na;
    t.ns = L->ns;
    t.nwfs = L->nwfs;
    for (int k = 0; k < L->nwfs; ++k) t.blk_start[k] = L->wfs_blk0[k];
    t.blk_start[L->nwfs] = L->nblk;
    t.s_pad = L->d_s;
    t.a = L->d_a;
    t.part = L->d_part;
    t.scale = L->d_Mscale;
    t.streams = L->tel_streams;
    t.off_s = L->tel_off_s;
    t.off_a = L->tel_off_a;
    t.off_p = L->tel_off_p;
    t.decimate = L->tel_decimate;
    t.depth = L->tel_depth;
    t.entry_floats = L->tel_entry_floats;
    t.ring = L->d_tel;
    t.wcount = L->d_wcount;
    t.ctr = L->d_telctr;
    t.fid = L->d_fid + L->cur_slot;
    t.t_cmd = L->d_tdone + L->cur_slot;
    return t;
}

// After the MVM (whose tail wrote the commands): POLC for the next frame and the
// telemetry copy.  Stream work only, so it can also be captured into a graph.
int enqueue_tail(rtc_loop* L) {
    Slot& s = L->slots[L->cur_slot];
    float* cmd = L->d_ring + (size_t)L->cur_slot * L->slot_floats;
    if (L->timing && !L->capturing) TRY(record(L, s.ev_final, L->st));
    TRY(polc_product(L, !L->timing));
    TRY(record(L, s.ev_polc, L->st));
    if (L->telemetry || L->tel_depth) {
        CK(L, cudaStreamWaitEvent(L->st_tel, s.ev_polc, 0));
        if (L->telemetry)
            CK(L, launch_pack_slopes(L->d_blocks, L->nblk, std::max(L->max_cols, 1), L->d_s,
                                     cmd + round_up((size_t)L->na, 4), L->st_tel));
        if (L->tel_depth) CK(L, launch_telemetry(tel_args(L), L->st_tel));
        TRY(record(L, s.ev_tel, L->st_tel));
        CK(L, cudaStreamWaitEvent(L->st, s.ev_tel, 0));   // the next frame rewrites the slopes
    } else {
        TRY(record(L, s.ev_tel, L->st));
    }
    if (!L->capturing) TRY(record(L, L->ev_frame_end, L->st));   // per-WFS streams start the next frame after it
    return RTC_OK;
}

// Make the loop stream wait for the work every per-WFS stream has queued.
int join_wfs_streams(rtc_loop* L) {
    for (int k = 0; k < L->nwfs; ++k) {
        CK(L, cudaEventRecord(L->ev_w[k], L->st_w[k]));
        CK(L, cudaStreamWaitEvent(L->st, L->ev_w[k], 0));
    }
    return RTC_OK;
}

// Host bookkeeping once a frame's work is enqueued: publish its slot to readers.
int publish_frame(rtc_loop* L) {
    Slot& s = L->slots[L->cur_slot];
    {
        std::lock_guard<std::mutex> g(L->mu);
        s.used = true;
        L->pending.push_back(L->cur_slot);
        ++L->frames_done;
    }
    L->cv.notify_all();
    L->active = false;
    L->have_last = true;
    L->last_id = L->cur_id;
    ++L->seq;
    return RTC_OK;
}

int finish_frame(rtc_loop* L) {
    TRY(enqueue_tail(L));
    return publish_frame(L);
}

FinaliseArgs fin_args(rtc_loop* L) {
    FinaliseArgs f{};
    f.enabled = 1;
    f.nblk = L->nblk;
    f.counters = L->d_fin_cnt;
    f.scale = L->d_Mscale;
    f.q = L->d_q;
    f.a = L->d_a;
    f.cmd = L->d_ring + (size_t)L->cur_slot * L->slot_floats;
    f.oml = L->explicit_polc ? 1.0f - L->leak - L->gain : 1.0f - L->leak;
    f.gain = L->gain;
    f.clip = L->clip;
    f.amin = L->amin;
    f.amax = L->amax;
    f.tiles_done = L->d_tiles_done;
    f.done_flag = L->d_done + L->cur_slot;
    f.seq = L->d_seq + L->cur_slot;
    f.t_done = L->d_tdone + L->cur_slot;
    f.partial = L->partial ? 1 : 0;
    f.pout = L->d_pout;
    return f;
}

// host_px: the pixels are read in place from page-locked host memory (a row chunk):
// the slope kernel variant with all of a thread's pixel rows in flight.
// gate: a pre-enqueued chunk's mailbox (its CTAs wait on it for the pixel address).
int slopes_rows(rtc_loop* L, int r0, int r1, const FramePtrs& fp, bool host_px, cudaStream_t st,
                const ChunkGate* gate = nullptr) {
    const int p0 = L->part_start[r0], p1 = L->part_start[r1];
    const float* pol = L->explicit_polc ? L->d_u : nullptr;
    CK(L, launch_slopes(L->d_ctas, p0, p1 - p0, L->wfs_host.data(), L->nwfs, fp, host_px, L->d_xlist, L->d_ref, pol,
                        L->d_s, L->d_pscr, L->d_row_cnt, L->smem_bytes, st, gate));
    // globally normalised pyramids whose rows all ran here (they are never split across launches)
    int i0 = -1, i1 = -1;
    for (int k = 0; k < L->nwfs; ++k)
        if (L->norm_nitems[k] && L->wfs_row0[k] >= r0 && L->wfs_row0[k] + L->wfs_nrows[k] <= r1) {
            if (i0 < 0) i0 = L->norm_item0[k];
            i1 = L->norm_item0[k] + L->norm_nitems[k];
        }
    if (i0 >= 0)
        CK(L, launch_normalise(L->d_norm_items, i0, i1 - i0, L->norm_max_pairs, L->d_blocks, L->d_wfs, L->d_pscr,
                               L->d_ref, pol, L->d_s, !L->stage_timing, st));
    return RTC_OK;
}

long long avg_row_bytes(const rtc_loop* L) {
    return (long long)(L->m_bytes / ((uint64_t)std::max(L->na, 1) * std::max(L->nblk, 1)));
}

// A dropped frame may have counted some blocks of some row tiles: once all its
// queued work is done, clear them; the next frame starts after that.
int reset_counters(rtc_loop* L) {
    cancel_prelaunched(L);
    TRY(join_wfs_streams(L));
    CK(L, cudaMemsetAsync(L->d_fin_cnt, 0, (size_t)L->nfin * sizeof(unsigned), L->st));
    CK(L, cudaEventRecord(L->ev_frame_end, L->st));
    return RTC_OK;
}

// Device address through which kernels can read p in place: device or managed
// memory, or page-locked host memory (read over the CPU-GPU link; *host is set);
// NULL for pageable memory, which must be copied.
const void* device_view(const void* p, bool* host = nullptr) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (host) *host = at.type == cudaMemoryTypeHost;
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged || at.type == cudaMemoryTypeHost)
        return at.devicePointer;
    return nullptr;
}

FramePtrs internal_frames(rtc_loop* L) {
    FramePtrs fp{};
    for (int k = 0; k < L->nwfs; ++k) {
        fp.px[k] = L->d_frame[k];
        fp.pitch[k] = L->frame_pitch[k];
    }
    return fp;
}

// Enqueues, on WFS k's camera stream, the slope and MVM kernels of its next row
// chunk as the previous frame had it (the chunk starting at the rows received so
// far, read in place), waiting on a mailbox that rtc_submit_pixels fills when
// that chunk arrives.  Nothing is enqueued when the previous frame had no such
// chunk, when the chunk completes no slope row, or when the mailbox this WFS
// takes next is still read by earlier kernels.
int prelaunch_next(rtc_loop* L, int k) {
    const rtc_wfs& w = L->wfs[k];
    if (w.kind != RTC_WFS_SH) return RTC_OK;
    const int rb = L->rows_in[k];
    const rtc_loop::SeenChunk* e = nullptr;
    for (const auto& x : L->seen_prev[k])
        if (x.row_begin == rb) e = &x;
    if (!e || !e->in_place) return RTC_OK;
    const int r0 = L->wfs_row0[k];
    const int done = L->rows_done[k];
    int upto = done;
    while (upto < L->wfs_nrows[k] && L->row_ready[r0 + upto] <= e->row_end) ++upto;
    if (upto == done) return RTC_OK;
    // the in-place conditions of submit_impl, for these rows
    if (w.oy + done * w.npx < e->row_begin) return RTC_OK;
    if (upto < w.nsuby && e->row_end > w.oy + upto * w.npx) return RTC_OK;
    const int box = k * kBoxesPerWfs + L->box_next[k];
    const cudaError_t q = cudaEventQuery(L->ev_box[box]);
    if (q == cudaErrorNotReady) return RTC_OK;
    CK(L, q);
    L->box_next[k] = (L->box_next[k] + 1) % kBoxesPerWfs;
    ChunkDesc& b = L->h_box[box];
    b.px = nullptr;
    b.pitch = 0;
    b.row0 = 0;
    __atomic_store_n(&b.state, (int)kChunkEmpty, __ATOMIC_SEQ_CST);   // before the launches below
    const ChunkGate gate{L->d_box + box, L->d_box_mirror + box, k, L->pre_max_polls, L->pre_limit_ns};
    FramePtrs fp = internal_frames(L);
    fp.px[k] = nullptr;                        // from the mailbox
    cudaStream_t sk = L->st_w[k];
    const int b0 = L->wfs_blk0[k];
    const int bd = L->blks_done[k];
    int bu = bd;
    while (bu < L->wfs_nblk[k] && L->blk_row_end[b0 + bu] <= upto) ++bu;
    rtc_loop::PreChunk& p = L->pre[k];
    p.row_begin = e->row_begin;
    p.row_end = e->row_end;
    p.upto = upto;
    p.bu = bu;
    p.box = box;
    p.host_px = e->host_px;
    TRY(slopes_rows(L, r0 + done, r0 + upto, fp, e->host_px, sk, &gate));
    p.pending = true;                          // from here on every path settles the mailbox
    if (bu > bd) {
        const FinaliseArgs fa = fin_args(L);
        CK(L, launch_gemv(L->m_dtype, L->d_M, L->d_blocks, b0 + bd, bu - bd, L->na, L->d_s, nullptr, L->d_part, L->na,
                          &fa, avg_row_bytes(L), true, sk, &L->d_box_mirror[box].state));
    }
    CK(L, cudaEventRecord(L->ev_box[box], sk));
    return RTC_OK;
}

int submit_impl(rtc_loop* L, const rtc_chunk* c) {
    if (!c || c->wfs < 0 || c->wfs >= L->nwfs || !c->px) return fail(L, RTC_EINVAL, "bad chunk");
    const rtc_wfs& w = L->wfs[c->wfs];
    if (c->row_begin < 0 || c->row_end > w.height || c->row_begin >= c->row_end)
        return fail(L, RTC_EINVAL, "bad chunk rows");
    if (c->pitch < (size_t)w.width * 2) return fail(L, RTC_EINVAL, "chunk pitch smaller than a row");
    int status = RTC_OK;
    // order checks before any state change
    if (L->active && c->frame_id != L->cur_id) {
        if (c->frame_id < L->cur_id) return fail(L, RTC_EORDER, "chunk of an older frame");
        if (c->row_begin != 0) return fail(L, RTC_EORDER, "new frame must start at row 0");
        ++L->frames_dropped;
        L->active = false;
        TRY(reset_counters(L));
        status = RTC_EDROPPED;
        L->err = "frame " + std::to_string(L->cur_id) + " was incomplete and has been dropped";
    }
    if (!L->active) {
        if (L->have_last && c->frame_id <= L->last_id) return fail(L, RTC_EORDER, "frame id not increasing");
        if (c->row_begin != 0) return fail(L, RTC_EORDER, "a frame must start at row 0");
        TRY(apply_pending_update(L));
        TRY(begin_frame(L, c->frame_id, true));
    } else if (c->row_begin != L->rows_in[c->wfs]) {
        return fail(L, RTC_EORDER, "rows of a WFS must arrive in order without gaps");
    }
    const int k = c->wfs;
    Slot& s = L->slots[L->cur_slot];
    cudaStream_t sk = L->st_w[k];              // this camera's stream
    if (L->rows_in[k] == 0) {                  // its first chunk of the frame: after the previous frame
        CK(L, cudaStreamWaitEvent(sk, L->ev_frame_end, 0));
        if (L->timing && !L->start_recorded) CK(L, cudaEventRecord(s.ev_start, sk));
        L->start_recorded = true;
    }
    // last chunk of the frame?
    bool last = true;
    for (int j = 0; j < L->nwfs; ++j) {
        const int got = j == k ? c->row_end : L->rows_in[j];
        if (got < L->wfs[j].height) last = false;
    }
    if (last && L->timing) CK(L, cudaEventRecord(s.ev_tail, sk));
    // slope rows completed by these rows
    const int r0 = L->wfs_row0[k];
    const int done = L->rows_done[k];
    int upto = done;
    while (upto < L->wfs_nrows[k] && L->row_ready[r0 + upto] <= c->row_end) ++upto;
    // Read the chunk in place when it is device-accessible, aligned, and holds
    // exactly whole subaperture rows: every row those slope rows need, and no
    // row a later chunk's subaperture row would need.  Otherwise copy it into
    // the loop's frame buffer.
    FramePtrs fp = internal_frames(L);
    bool in_place = false, host_px = false;
    if (w.kind == RTC_WFS_SH && (c->pitch & 15u) == 0 && (reinterpret_cast<uintptr_t>(c->px) & 15u) == 0 &&
        c->pitch >= round_up((size_t)w.width * 2, 16)) {
        const bool needed_here = upto == done || w.oy + done * w.npx >= c->row_begin;
        const bool no_leftover = upto >= w.nsuby || c->row_end <= w.oy + upto * w.npx;
        if (needed_here && no_leftover) {
            if (const void* dv = device_view(c->px, &host_px)) {
                in_place = true;
                fp.px[k] = static_cast<const uint16_t*>(dv);
                fp.pitch[k] = (long long)(c->pitch / 2);
                fp.row0[k] = c->row_begin;
            }
        }
    }
    if (L->prelaunch) L->seen_cur[k].push_back({c->row_begin, c->row_end, in_place, host_px});
    // the kernels of this chunk may have been enqueued already, waiting on a mailbox
    bool taken = false;
    if (L->prelaunch && L->pre[k].pending) {
        rtc_loop::PreChunk& p = L->pre[k];
        const bool match = in_place && host_px == p.host_px && c->row_begin == p.row_begin &&
                           c->row_end == p.row_end && upto == p.upto;
        if (match) {
            ChunkDesc& b = L->h_box[p.box];
            b.px = fp.px[k];
            b.pitch = fp.pitch[k];
            b.row0 = fp.row0[k];
        }
        if (settle_prelaunched(L, p, match ? kChunkFilled : kChunkCancelled)) {
            taken = match;
            if (!match) ++L->pre_cancelled;
        }
        if (taken) {
            ++L->pre_used;
            L->rows_in[k] = c->row_end;
            L->rows_done[k] = upto;
            L->blks_done[k] = p.bu;
        }
    }
    if (!taken) {
        if (!in_place)
            CK(L, cudaMemcpy2DAsync(L->d_frame[k] + (size_t)c->row_begin * L->frame_pitch[k], L->frame_pitch[k] * 2,
                                    c->px, c->pitch, (size_t)w.width * 2, c->row_end - c->row_begin, cudaMemcpyDefault,
                                    sk));
        L->rows_in[k] = c->row_end;
        const bool slopes_launched = upto > done;
        if (slopes_launched) {
            TRY(slopes_rows(L, r0 + done, r0 + upto, fp, in_place && host_px, sk));
            L->rows_done[k] = upto;
        }
        if (last && L->stage_timing) CK(L, cudaEventRecord(s.ev_slopes, sk));
        // column blocks completed by those slope rows
        const int b0 = L->wfs_blk0[k];
        int bd = L->blks_done[k];
        int bu = bd;
        while (bu < L->wfs_nblk[k] && L->blk_row_end[b0 + bu] <= L->rows_done[k]) ++bu;
        if (bu > bd) {
            const FinaliseArgs fa = fin_args(L);
            CK(L, launch_gemv(L->m_dtype, L->d_M, L->d_blocks, b0 + bd, bu - bd, L->na, L->d_s, nullptr, L->d_part,
                              L->na, &fa, avg_row_bytes(L), slopes_launched && !L->stage_timing, sk));
            L->blks_done[k] = bu;
        }
    }
    if (L->prelaunch && !last && L->rows_in[k] < w.height) TRY(prelaunch_next(L, k));
    if (last) {
        if (L->stage_timing) CK(L, cudaEventRecord(s.ev_mvm, sk));
        TRY(join_wfs_streams(L));              // POLC and telemetry follow every camera's work
        TRY(finish_frame(L));
    }
    return status;
}

// Stream work of one whole frame whose pixels are addressed by fp: slopes of
// every row, the MVM (a programmatic dependent of the slope kernel) with its
// fused finalisation, then the tail.  Shared by rtc_process_frame and the
// captured frame graphs.
int enqueue_whole_frame(rtc_loop* L, const FramePtrs& fp) {
    Slot& s = L->slots[L->cur_slot];
    if (L->timing && !L->capturing) {        // graph launches record these around the launch
        TRY(record(L, s.ev_start, L->st));
        TRY(record(L, s.ev_tail, L->st));
    }
    // Whole frames take the register-light slope kernel even from page-locked host
    // memory: their hundreds of CTAs need several per SM, and the link's bandwidth,
    // not its latency, bounds them.
    TRY(slopes_rows(L, 0, L->nrows, fp, false, L->st));
    if (L->stage_timing) TRY(record(L, s.ev_slopes, L->st));
    const FinaliseArgs fa = fin_args(L);
    CK(L, launch_gemv(L->m_dtype, L->d_M, L->d_blocks, 0, L->nblk, L->na, L->d_s, nullptr, L->d_part, L->na, &fa,
                      avg_row_bytes(L), !L->stage_timing, L->st));
    if (L->stage_timing) TRY(record(L, s.ev_mvm, L->st));
    return enqueue_tail(L);
}

// Graph mode: one set of page-locked input frames per ring slot, and the whole
// frame's stream work (slopes -> MVM -> POLC -> telemetry, with the
// programmatic-launch edges) captured once per slot into a CUDA graph.
int capture_graphs(rtc_loop* L) {
    L->g_pitch.resize(L->nwfs);
    for (int k = 0; k < L->nwfs; ++k) L->g_pitch[k] = round_up((size_t)L->wfs[k].width * 2, 16);
    L->g_px.assign(L->ring, std::vector<uint16_t*>(L->nwfs, nullptr));
    L->g_exec.assign(L->ring, nullptr);
    for (int slot = 0; slot < L->ring; ++slot) {
        FramePtrs fp{};
        for (int k = 0; k < L->nwfs; ++k) {
            void *h = nullptr, *d = nullptr;
            const size_t bytes = (size_t)L->wfs[k].height * L->g_pitch[k];
            const int rc = pinned_alloc(L, &h, &d, bytes, "input frames");
            L->g_px[slot][k] = static_cast<uint16_t*>(h);
            TRY(rc);
            std::memset(h, 0, bytes);
            fp.px[k] = static_cast<const uint16_t*>(d);
            fp.pitch[k] = (long long)(L->g_pitch[k] / 2);
        }
        L->cur_slot = slot;
        L->capturing = true;
        CK(L, cudaStreamBeginCapture(L->st, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_whole_frame(L, fp);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(L->st, &graph);
        L->capturing = false;
        if (rc != RTC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(L, e, "cudaStreamEndCapture");
        const cudaError_t ei = cudaGraphInstantiate(&L->g_exec[slot], graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) return cuda_fail(L, ei, "cudaGraphInstantiate");
    }
    L->cur_slot = 0;
    return RTC_OK;
}

// The slot the next frame will use, once the GPU is done with its previous frame.
int next_slot_free(rtc_loop* L, int* slot) {
    *slot = (int)(L->seq % (uint64_t)L->ring);
    const Slot& prev = L->slots[*slot];
    TRY(slot_wait(L, prev, *slot));
    return RTC_OK;
}

int process_impl(rtc_loop* L, uint64_t id, const uint16_t* const* px, const size_t* pitch) {
    if (!px || !pitch) return fail(L, RTC_EINVAL, "px and pitch are required");
    FramePtrs fp{};
    for (int k = 0; k < L->nwfs; ++k) {
        const rtc_wfs& w = L->wfs[k];
        if (!px[k] || (reinterpret_cast<uintptr_t>(px[k]) & 15u) || (pitch[k] & 15u) ||
            pitch[k] < round_up((size_t)w.width * 2, 16))
            return fail(L, RTC_EINVAL, "frame " + std::to_string(k) + ": pointer/pitch not 16-byte aligned or too small");
        const void* dv = device_view(px[k]);
        if (!dv) return fail(L, RTC_EINVAL, "frame " + std::to_string(k) + " is neither device nor page-locked memory");
        fp.px[k] = static_cast<const uint16_t*>(dv);
        fp.pitch[k] = (long long)(pitch[k] / 2);
        fp.row0[k] = 0;
    }
    int status = RTC_OK;
    if (L->active ? id <= L->cur_id : (L->have_last && id <= L->last_id))
        return fail(L, RTC_EORDER, "frame id not increasing");
    if (L->active) {
        ++L->frames_dropped;
        L->active = false;
        TRY(reset_counters(L));
        status = RTC_EDROPPED;
        L->err = "frame " + std::to_string(L->cur_id) + " was incomplete and has been dropped";
    }
    TRY(apply_pending_update(L));
    TRY(begin_frame(L, id, false));
    TRY(enqueue_whole_frame(L, fp));
    TRY(publish_frame(L));
    return status;
}

// Upload rows x width bytes from pageable host memory (row pitch spitch) into
// device memory (row pitch dpitch >= width, the bytes past width written as
// zeros) on the upload stream, through the loop's two page-locked staging
// buffers: this thread gathers one piece while the copy engine moves the
// previous one, and every CUDA call is a short asynchronous copy from page-locked
// memory (a pageable copy of a large matrix would be staged inside the driver,
// where it has delayed the frame thread's launches).  Rows wider than a staging
// buffer fall back to one pitched pageable copy.
int staged_upload(rtc_loop* L, void* dst, size_t dpitch, const void* src, size_t spitch, size_t width, size_t rows) {
    if (dpitch > kStageBytes) {
        CK(L, cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyHostToDevice, L->st_up));
        return RTC_OK;
    }
    const size_t per = kStageBytes / dpitch;
    for (size_t r0 = 0; r0 < rows; r0 += per) {
        const size_t n = std::min(per, rows - r0);
        const int b = L->stage_next;
        L->stage_next ^= 1;
        if (L->stage_used[b]) CK(L, cudaEventSynchronize(L->ev_stage[b]));   // its previous copy is done
        unsigned char* h = L->h_stage[b];
        const unsigned char* from = static_cast<const unsigned char*>(src) + r0 * spitch;
        for (size_t r = 0; r < n; ++r) {
            std::memcpy(h + r * dpitch, from + r * spitch, width);
            if (dpitch > width) std::memset(h + r * dpitch + width, 0, dpitch - width);
        }
        CK(L, cudaMemcpyAsync(static_cast<unsigned char*>(dst) + r0 * dpitch, h, n * dpitch, cudaMemcpyHostToDevice,
                              L->st_up));
        CK(L, cudaEventRecord(L->ev_stage[b], L->st_up));
        L->stage_used[b] = true;
    }
    return RTC_OK;
}

// Busy-poll an event until done or the deadline.
int wait_event(rtc_loop* L, cudaEvent_t ev, Clock::time_point deadline, bool forever) {
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return RTC_OK;
        if (e != cudaErrorNotReady) return cuda_fail(L, e, "cudaEventQuery");
        if (!forever && Clock::now() >= deadline) return fail(L, RTC_ETIMEDOUT, "timed out waiting for the GPU");
    }
}

// Busy-poll the slot's page-locked completion word until it holds the frame's
// sequence number or the deadline passes; every few thousand polls also ask the
// stream whether a kernel failed.
int wait_done(rtc_loop* L, int slot, uint64_t seq, Clock::time_point deadline, bool forever) {
    const volatile unsigned long long* w = L->h_done + slot;
    for (unsigned n = 1;; ++n) {
        if (*w == seq) {
            std::atomic_thread_fence(std::memory_order_acquire);
            return RTC_OK;
        }
        if ((n & 4095u) == 0) {
            const cudaError_t e = cudaStreamQuery(L->st);
            if (e != cudaSuccess && e != cudaErrorNotReady) return cuda_fail(L, e, "kernel failed");
            if (!forever && Clock::now() >= deadline) return fail(L, RTC_ETIMEDOUT, "timed out waiting for the GPU");
        }
    }
}

Clock::time_point deadline_of(int64_t us) {
    return Clock::now() + std::chrono::microseconds(us < 0 ? 0 : us);
}

int find_slot(rtc_loop* L, uint64_t frame_id) {
    std::lock_guard<std::mutex> g(L->mu);
    for (int i = 0; i < L->ring; ++i)
        if (L->slots[i].used && L->slots[i].frame_id == frame_id) return i;
    return -1;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    return ms * 1000.f;
}

}  // namespace

namespace rtc {

void loop_last_frame(const rtc_loop* L, int* slot, unsigned long long* seq) {
    const int s = (int)((L->seq + (uint64_t)L->ring - 1) % (uint64_t)L->ring);
    *slot = s;
    *seq = L->slots[s].seq;
}

bool loop_frame_done(const rtc_loop* L, int slot, unsigned long long seq) {
    const volatile unsigned long long* w = L->h_done + slot;
    return *w == seq;
}

}  // namespace rtc

extern "C" {

int rtc_create(const rtc_geometry* geometry, const rtc_calib* calib, const rtc_cmat* cmat, const rtc_polc* polc,
               rtc_loop** out) {
    if (!out) return fail(nullptr, RTC_EINVAL, "out is NULL");
    *out = nullptr;
    rtc_loop* L = new (std::nothrow) rtc_loop();
    if (!L) return fail(nullptr, RTC_ENOMEM, "host allocation failed");
    int rc = create_impl(geometry, calib, cmat, polc, L);
    if (rc != RTC_OK) {
        g_err = L->err.empty() ? g_err : L->err;
        release(L);
        return rc;
    }
    *out = L;
    return RTC_OK;
}

int rtc_destroy(rtc_loop* loop) {
    release(loop);
    return RTC_OK;
}

int rtc_submit_pixels(rtc_loop* L, const rtc_chunk* chunk) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (L->broken) return fail(L, RTC_ECUDA, "loop is in a failed state: " + L->err);
    TRY(use_device(L));
    return submit_impl(L, chunk);
}

int rtc_submit_pixels_n(rtc_loop* L, const rtc_chunk* chunks, int32_t n, int32_t* accepted) {
    if (accepted) *accepted = 0;
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (n < 0 || (n > 0 && !chunks)) return fail(L, RTC_EINVAL, "n must be >= 0 and chunks non-NULL");
    if (L->broken) return fail(L, RTC_ECUDA, "loop is in a failed state: " + L->err);
    TRY(use_device(L));
    int status = RTC_OK;
    for (int32_t i = 0; i < n; ++i) {
        const int rc = submit_impl(L, chunks + i);
        if (rc != RTC_OK && rc != RTC_EDROPPED) return rc;
        if (rc == RTC_EDROPPED) status = rc;
        if (accepted) *accepted = i + 1;
    }
    return status;
}

int rtc_process_frame(rtc_loop* L, uint64_t frame_id, const uint16_t* const* px, const size_t* pitch) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (L->broken) return fail(L, RTC_ECUDA, "loop is in a failed state: " + L->err);
    TRY(use_device(L));
    return process_impl(L, frame_id, px, pitch);
}

int rtc_next_frame_buffers(rtc_loop* L, uint16_t** px, size_t* pitch) {
    if (!L || !px || !pitch) return fail(L, RTC_EINVAL, "loop, px and pitch are required");
    if (!L->graphs) return fail(L, RTC_EINVAL, "loop created without RTC_FLAG_GRAPHS");
    TRY(use_device(L));
    int slot = 0;
    TRY(next_slot_free(L, &slot));
    for (int k = 0; k < L->nwfs; ++k) {
        px[k] = L->g_px[slot][k];
        pitch[k] = L->g_pitch[k];
    }
    return RTC_OK;
}

int rtc_submit_frame_graph(rtc_loop* L, uint64_t frame_id) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (!L->graphs) return fail(L, RTC_EINVAL, "loop created without RTC_FLAG_GRAPHS");
    if (L->broken) return fail(L, RTC_ECUDA, "loop is in a failed state: " + L->err);
    TRY(use_device(L));
    int status = RTC_OK;
    if (L->active ? frame_id <= L->cur_id : (L->have_last && frame_id <= L->last_id))
        return fail(L, RTC_EORDER, "frame id not increasing");
    if (L->active) {
        ++L->frames_dropped;
        L->active = false;
        TRY(reset_counters(L));
        status = RTC_EDROPPED;
    }
    TRY(begin_frame(L, frame_id, false));
    Slot& s = L->slots[L->cur_slot];
    if (L->timing) {                       // frame-level timing spans the whole graph launch
        CK(L, cudaEventRecord(s.ev_start, L->st));
        CK(L, cudaEventRecord(s.ev_tail, L->st));
    }
    CK(L, cudaGraphLaunch(L->g_exec[L->cur_slot], L->st));
    // the graph ends with the telemetry joined back into the loop's stream: these
    // complete when the whole frame (POLC and telemetry included) has
    if (L->timing) CK(L, cudaEventRecord(s.ev_final, L->st));
    CK(L, cudaEventRecord(s.ev_polc, L->st));
    CK(L, cudaEventRecord(s.ev_tel, L->st));
    CK(L, cudaEventRecord(L->ev_frame_end, L->st));
    TRY(publish_frame(L));
    return status;
}

int rtc_footprint(const rtc_geometry* geometry, const rtc_calib* calib, const rtc_cmat* cmat, const rtc_polc* polc,
                  uint64_t* resident_bytes, uint64_t* peak_bytes) {
    rtc_loop* L = new (std::nothrow) rtc_loop();
    if (!L) return fail(nullptr, RTC_ENOMEM, "host allocation failed");
    L->plan_only = true;
    const int rc = create_impl(geometry, calib, cmat, polc, L);
    if (rc == RTC_OK) {
        if (resident_bytes) *resident_bytes = L->need_resident;
        if (peak_bytes) *peak_bytes = L->need_peak;
    } else {
        g_err = L->err.empty() ? g_err : L->err;
    }
    release(L);
    return rc;
}

int rtc_get_commands(rtc_loop* L, float* out, size_t n, uint64_t* frame_id, int64_t timeout_us) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (!out || n != (size_t)L->na) return fail(L, RTC_EINVAL, "out must hold na floats");
    TRY(use_device(L));
    const bool forever = timeout_us < 0;
    const auto deadline = deadline_of(timeout_us);
    for (;;) {
        int slot;
        {
            std::unique_lock<std::mutex> g(L->mu);
            while (L->pending.empty()) {
                if (forever) L->cv.wait(g);
                else if (L->cv.wait_until(g, deadline) == std::cv_status::timeout && L->pending.empty())
                    return fail(L, RTC_ETIMEDOUT, "no frame pending");
            }
            slot = L->pending.front();
        }
        uint64_t seq;
        {
            std::lock_guard<std::mutex> g(L->mu);
            seq = L->slots[slot].seq;
        }
        TRY(wait_done(L, slot, seq, deadline, forever));
        std::lock_guard<std::mutex> g(L->mu);
        if (L->pending.empty() || L->pending.front() != slot) continue;   // discarded meanwhile
        L->pending.pop_front();
        std::memcpy(out, L->h_ring + (size_t)slot * L->slot_floats, (size_t)L->na * 4);
        if (frame_id) *frame_id = L->slots[slot].frame_id;
        return RTC_OK;
    }
}

int rtc_get_telemetry(rtc_loop* L, uint64_t frame_id, float* slopes, size_t ns, float* cmds, size_t na,
                      int64_t timeout_us) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (slopes && (ns != (size_t)L->ns || !L->telemetry)) return fail(L, RTC_EINVAL, "slopes need ns floats and RTC_FLAG_TELEMETRY");
    if (cmds && na != (size_t)L->na) return fail(L, RTC_EINVAL, "cmds must hold na floats");
    TRY(use_device(L));
    const int slot = find_slot(L, frame_id);
    if (slot < 0) return fail(L, RTC_ENOENT, "frame not in the ring");
    const auto deadline = deadline_of(timeout_us);
    TRY(wait_event(L, L->slots[slot].ev_tel, deadline, timeout_us < 0));
    std::lock_guard<std::mutex> g(L->mu);
    if (!L->slots[slot].used || L->slots[slot].frame_id != frame_id) return fail(L, RTC_ENOENT, "frame left the ring");
    const float* base = L->h_ring + (size_t)slot * L->slot_floats;
    if (cmds) std::memcpy(cmds, base, (size_t)L->na * 4);
    if (slopes) std::memcpy(slopes, base + round_up((size_t)L->na, 4), (size_t)L->ns * 4);
    return RTC_OK;
}

// The oldest unread entry of the telemetry buffer (caller holds tel_mu).  Sets
// no error text, so the stream thread can use it too.
int tel_read_entry(rtc_loop* L, rtc_tel_record* rec, float* slopes, float* cmds, float* partials,
                   int64_t timeout_us) {
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    const uint64_t D = (uint64_t)L->tel_depth;
    for (;;) {
        const uint64_t w = __atomic_load_n(L->h_wcount, __ATOMIC_ACQUIRE);
        if (L->tel_next >= w) {
            if (timeout_us >= 0 && Clock::now() >= deadline) return RTC_ETIMEDOUT;
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            continue;
        }
        // the writer of entry w may be active, rewriting entry w - D: entries from w - D + 1 on are intact
        if (w - L->tel_next > D - 1) {
            L->tel_lost += w - (D - 1) - L->tel_next;
            L->tel_next = w - (D - 1);
        }
        const float* e = L->h_tel + (size_t)(L->tel_next % D) * L->tel_entry_floats;
        const TelHeader* h = reinterpret_cast<const TelHeader*>(e);
        rtc_tel_record r{};
        r.index = __atomic_load_n(&h->index, __ATOMIC_ACQUIRE);
        r.frame_id = h->frame_id;
        r.t_commands_ns = h->t_commands;
        r.t_written_ns = h->t_written;
        const float* body = e + kTelHeaderFloats;
        if (slopes) std::memcpy(slopes, body + L->tel_off_s, (size_t)L->ns * 4);
        if (cmds) std::memcpy(cmds, body + L->tel_off_a, (size_t)L->na * 4);
        if (partials) std::memcpy(partials, body + L->tel_off_p, (size_t)L->nwfs * L->na * 4);
        std::atomic_thread_fence(std::memory_order_acquire);
        const uint64_t w2 = __atomic_load_n(L->h_wcount, __ATOMIC_ACQUIRE);
        if (r.index != L->tel_next || w2 - L->tel_next > D - 1) {   // rewritten while it was copied
            ++L->tel_lost;
            ++L->tel_next;
            continue;
        }
        r.lost = L->tel_lost;
        L->tel_lost = 0;
        ++L->tel_next;
        *rec = r;
        return RTC_OK;
    }
}

int rtc_telemetry_read(rtc_loop* L, rtc_tel_record* rec, float* slopes, size_t ns, float* cmds, size_t na,
                       float* partials, size_t npartials, int64_t timeout_us) {
    if (!L || !rec) return fail(L, RTC_EINVAL, "loop and rec are required");
    if (!L->tel_depth) return fail(L, RTC_EINVAL, "loop has no telemetry buffer (tel_depth 0)");
    if (L->tel_streaming) return fail(L, RTC_EINVAL, "a telemetry stream is reading the buffer");
    if (slopes && (!(L->tel_streams & RTC_TEL_SLOPES) || ns != (size_t)L->ns))
        return fail(L, RTC_EINVAL, "slopes not recorded, or ns wrong");
    if (cmds && (!(L->tel_streams & RTC_TEL_COMMANDS) || na != (size_t)L->na))
        return fail(L, RTC_EINVAL, "commands not recorded, or na wrong");
    if (partials && (!(L->tel_streams & RTC_TEL_PARTIALS) || npartials != (size_t)L->nwfs * L->na))
        return fail(L, RTC_EINVAL, "partial commands not recorded, or size not nwfs x na");
    std::lock_guard<std::mutex> g(L->tel_mu);
    const int rc = tel_read_entry(L, rec, slopes, cmds, partials, timeout_us);
    if (rc == RTC_ETIMEDOUT) return fail(L, rc, "no new telemetry entry");
    return rc;
}

int rtc_telemetry_stream_start(rtc_loop* L, int fd) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (!L->tel_depth) return fail(L, RTC_EINVAL, "loop has no telemetry buffer (tel_depth 0)");
    if (fd < 0) return fail(L, RTC_EINVAL, "bad file descriptor");
    if (L->tel_streaming || L->tel_thread.joinable()) return fail(L, RTC_EINVAL, "a telemetry stream already runs");
    L->tel_stats = rtc_tel_stream_stats{};
    L->tel_stop = false;
    L->tel_streaming = true;
    L->tel_thread = std::thread([L, fd]() {
        const bool sl = L->tel_streams & RTC_TEL_SLOPES, cm = L->tel_streams & RTC_TEL_COMMANDS,
                   pa = L->tel_streams & RTC_TEL_PARTIALS;
        const size_t nfl = (sl ? L->ns : 0) + (cm ? L->na : 0) + (pa ? (size_t)L->nwfs * L->na : 0);
        std::vector<char> buf(sizeof(rtc_tel_record) + nfl * 4);
        float* body = reinterpret_cast<float*>(buf.data() + sizeof(rtc_tel_record));
        float* ps = body;
        float* pc = ps + (sl ? L->ns : 0);
        float* pp = pc + (cm ? L->na : 0);
        for (;;) {
            const bool stopping = L->tel_stop.load();
            rtc_tel_record rec{};
            int rc;
            {
                std::lock_guard<std::mutex> g(L->tel_mu);
                rc = tel_read_entry(L, &rec, sl ? ps : nullptr, cm ? pc : nullptr, pa ? pp : nullptr,
                                    stopping ? 0 : 50000);
            }
            if (rc != RTC_OK) {
                if (stopping) break;        // everything published before the stop request is written
                continue;
            }
            L->tel_stats.lost += rec.lost;
            std::memcpy(buf.data(), &rec, sizeof(rec));
            size_t off = 0;
            while (off < buf.size()) {
                const ssize_t n = ::write(fd, buf.data() + off, buf.size() - off);
                if (n < 0) {
                    if (errno == EINTR) continue;
                    L->tel_stats.write_error = errno;
                    return;
                }
                off += (size_t)n;
            }
            ++L->tel_stats.entries;
            L->tel_stats.bytes += buf.size();
        }
    });
    return RTC_OK;
}

int rtc_telemetry_stream_stop(rtc_loop* L, rtc_tel_stream_stats* stats) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (!L->tel_thread.joinable()) return fail(L, RTC_EINVAL, "no telemetry stream runs");
    stop_stream(L);
    if (stats) *stats = L->tel_stats;
    return RTC_OK;
}

int rtc_get_timing(rtc_loop* L, uint64_t frame_id, rtc_timing* out, int64_t timeout_us) {
    if (!L || !out) return fail(L, RTC_EINVAL, "loop and out are required");
    if (!L->timing) return fail(L, RTC_EINVAL, "loop created without RTC_FLAG_TIMING");
    TRY(use_device(L));
    const int slot = find_slot(L, frame_id);
    if (slot < 0) return fail(L, RTC_ENOENT, "frame not in the ring");
    const Slot& s = L->slots[slot];
    const auto deadline = deadline_of(timeout_us);
    TRY(wait_event(L, s.ev_polc, deadline, timeout_us < 0));
    out->frame_id = frame_id;
    out->slopes_us = L->stage_timing ? elapsed(s.ev_tail, s.ev_slopes) : -1.f;
    out->mvm_us = L->stage_timing ? elapsed(s.ev_slopes, s.ev_mvm) : -1.f;
    out->final_us = 0.f;
    out->polc_us = elapsed(s.ev_final, s.ev_polc);
    out->latency_us = elapsed(s.ev_tail, s.ev_final);
    out->frame_us = elapsed(s.ev_start, s.ev_final);
    return RTC_OK;
}

int rtc_update(rtc_loop* L, const rtc_update_desc* d) {
    if (!L || !d) return fail(L, RTC_EINVAL, "loop and desc are required");
    if (!L->updatable) return fail(L, RTC_EINVAL, "loop created without RTC_FLAG_UPDATABLE");
    if ((d->P || d->P_scale) && !L->has_polc)
        return fail(L, RTC_EINVAL, L->explicit_polc ? "an explicit-POLC loop's D is fixed at creation"
                                                    : "loop has no POLC matrix");
    if (d->M_scale && !L->d_Mscale) return fail(L, RTC_EINVAL, "loop was created without control-matrix row scales");
    if (d->P_scale && !L->d_Pscale) return fail(L, RTC_EINVAL, "loop was created without POLC row scales");
    // validate everything before touching any buffer
    if (d->M && L->m_dtype == RTC_F32 && !all_finite(static_cast<const float*>(d->M), (size_t)L->na * L->ns))
        return fail(L, RTC_EINVAL, "new control matrix not finite");
    if (d->P && L->p_dtype == RTC_F32 && !all_finite(static_cast<const float*>(d->P), (size_t)L->na * L->na))
        return fail(L, RTC_EINVAL, "new POLC matrix not finite");
    if (d->M_scale && !all_finite(d->M_scale, L->na)) return fail(L, RTC_EINVAL, "new M_scale not finite");
    if (d->P_scale && !all_finite(d->P_scale, L->na)) return fail(L, RTC_EINVAL, "new P_scale not finite");
    if (d->ref_slopes && !all_finite(d->ref_slopes, L->ns)) return fail(L, RTC_EINVAL, "new ref_slopes not finite");
    for (int k = 0; k < L->nwfs; ++k) {
        const size_t n = (size_t)L->wfs[k].width * L->wfs[k].height;
        if (d->dark && d->dark[k] && !all_finite(d->dark[k], n)) return fail(L, RTC_EINVAL, "new dark not finite");
        if (d->flat && d->flat[k] && !all_finite(d->flat[k], n)) return fail(L, RTC_EINVAL, "new flat not finite");
        if (d->threshold && !(d->threshold[k] >= 0.f && std::isfinite(d->threshold[k])))
            return fail(L, RTC_EINVAL, "new threshold must be finite and >= 0");
    }
    if (d->set_control && (!std::isfinite(d->gain) || !std::isfinite(d->leak) || (d->clip && !(d->amin <= d->amax))))
        return fail(L, RTC_EINVAL, "bad control parameters");

    std::lock_guard<std::mutex> g(L->upd_mu);
    TRY(use_device(L));
    // the shadow buffers may still be read by frames issued before the last swap
    if (L->swap_ev_valid) CK(L, cudaStreamWaitEvent(L->st_up, L->ev_swap, 0));
    const size_t esz = dtype_size(L->m_dtype);
    unsigned mask = 0;
    if (d->M) {
        for (const BlockDev& B : L->blocks_h)
            if (B.ncols)
                TRY(staged_upload(L, static_cast<uint8_t*>(L->sh_M) + (size_t)B.m_off * esz, (size_t)B.pitch * esz,
                                  static_cast<const uint8_t*>(d->M) + (size_t)B.c0 * esz, (size_t)L->ns * esz,
                                  (size_t)B.ncols * esz, L->na));
        mask |= kUpdM;
    }
    if (d->M_scale) {
        CK(L, cudaMemcpyAsync(L->sh_Mscale, d->M_scale, (size_t)L->na * 4, cudaMemcpyHostToDevice, L->st_up));
        mask |= kUpdMscale;
    }
    if (d->P) {
        const size_t pe = dtype_size(L->p_dtype);
        const size_t pitch = round_up((size_t)L->na, elems_per_16B(L->p_dtype));
        TRY(staged_upload(L, L->sh_P, pitch * pe, d->P, (size_t)L->na * pe, (size_t)L->na * pe, L->na));
        mask |= kUpdP;
    }
    if (d->P_scale) {
        CK(L, cudaMemcpyAsync(L->sh_Pscale, d->P_scale, (size_t)L->na * 4, cudaMemcpyHostToDevice, L->st_up));
        mask |= kUpdPscale;
    }
    if (d->ref_slopes) {
        CK(L, cudaMemcpyAsync(L->sh_ref, d->ref_slopes, (size_t)L->ns * 4, cudaMemcpyHostToDevice, L->st_up));
        mask |= kUpdRef;
    }
    bool table = (L->upd_mask & kUpdTable) != 0;
    for (int k = 0; k < L->nwfs; ++k) {
        const rtc_wfs& w = L->wfs[k];
        const size_t cp = round_up(w.width, 4);
        if (d->dark && d->dark[k]) {
            CK(L, cudaMemcpy2DAsync(L->sh_dark[k], cp * 4, d->dark[k], (size_t)w.width * 4, (size_t)w.width * 4,
                                    w.height, cudaMemcpyHostToDevice, L->st_up));
            L->upd_dark[k] = 1;
            table = true;
        }
        if (d->flat && d->flat[k]) {
            CK(L, cudaMemcpy2DAsync(L->sh_flat[k], cp * 4, d->flat[k], (size_t)w.width * 4, (size_t)w.width * 4,
                                    w.height, cudaMemcpyHostToDevice, L->st_up));
            L->upd_flat[k] = 1;
            table = true;
        }
    }
    if (d->threshold) table = true;
    if (table) {
        // the WFS table as it will be after the swap
        std::vector<WfsDev> t = (L->upd_mask & kUpdTable) ? L->upd_table : L->wfs_host;
        for (int k = 0; k < L->nwfs; ++k) {
            t[k].dark = L->upd_dark[k] ? L->sh_dark[k] : L->d_dark[k];
            t[k].flat = L->upd_flat[k] ? L->sh_flat[k] : L->d_flat[k];
            if (d->threshold) t[k].threshold = d->threshold[k];
        }
        L->upd_table = t;
        CK(L, cudaMemcpyAsync(L->sh_wfs, L->upd_table.data(), t.size() * sizeof(WfsDev), cudaMemcpyHostToDevice,
                              L->st_up));
        mask |= kUpdTable;
    }
    CK(L, cudaStreamSynchronize(L->st_up));
    L->stage_used[0] = L->stage_used[1] = false;
    if (d->set_control) {
        L->upd_ctrl = true;
        L->upd_gain = d->gain;
        L->upd_leak = d->leak;
        L->upd_clip = d->clip;
        L->upd_amin = d->amin;
        L->upd_amax = d->amax;
    }
    L->upd_mask |= mask;
    L->upd_pending = L->upd_mask != 0 || L->upd_ctrl;
    return RTC_OK;
}

int rtc_get_state(rtc_loop* L, float* a, size_t na) {
    if (!L || !a || na != (size_t)L->na) return fail(L, RTC_EINVAL, "a must hold na floats");
    TRY(use_device(L));
    for (cudaStream_t w : L->st_w) CK(L, cudaStreamSynchronize(w));
    CK(L, cudaStreamSynchronize(L->st));
    CK(L, cudaMemcpy(a, L->d_a, na * 4, cudaMemcpyDeviceToHost));
    return RTC_OK;
}

int rtc_set_state(rtc_loop* L, const float* a, size_t na) {
    if (!L || !a || na != (size_t)L->na) return fail(L, RTC_EINVAL, "a must hold na floats");
    if (!all_finite(a, na)) return fail(L, RTC_EINVAL, "state not finite");
    TRY(use_device(L));
    for (cudaStream_t w : L->st_w) CK(L, cudaStreamSynchronize(w));
    CK(L, cudaStreamSynchronize(L->st));
    CK(L, cudaMemcpy(L->d_a, a, na * 4, cudaMemcpyHostToDevice));
    TRY(polc_product(L, false));
    CK(L, cudaStreamSynchronize(L->st));
    return RTC_OK;
}

int rtc_sync(rtc_loop* L) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    TRY(use_device(L));
    for (cudaStream_t w : L->st_w) CK(L, cudaStreamSynchronize(w));
    CK(L, cudaStreamSynchronize(L->st));
    CK(L, cudaStreamSynchronize(L->st_tel));
    return RTC_OK;
}

int rtc_check_guards(rtc_loop* L, int32_t* corrupted) {
    if (!L || !corrupted) return fail(L, RTC_EINVAL, "loop and corrupted are required");
    TRY(use_device(L));
    for (cudaStream_t w : L->st_w) CK(L, cudaStreamSynchronize(w));
    CK(L, cudaStreamSynchronize(L->st));
    CK(L, cudaStreamSynchronize(L->st_tel));
    if (L->st_up) CK(L, cudaStreamSynchronize(L->st_up));
    int bad = 0;
    unsigned char buf[kGuardBytes];
    for (const auto& g : L->guards) {
        const unsigned char* src = g.first;
        if (!g.second) {
            CK(L, cudaMemcpy(buf, g.first, kGuardBytes, cudaMemcpyDeviceToHost));
            src = buf;
        }
        for (size_t i = 0; i < kGuardBytes; ++i)
            if (src[i] != kGuardByte) {
                ++bad;
                break;
            }
    }
    *corrupted = bad;
    return RTC_OK;
}

int rtc_get_stream(rtc_loop* L, void** stream) {
    if (!L || !stream) return fail(L, RTC_EINVAL, "loop and stream are required");
    *stream = static_cast<void*>(L->st);
    return RTC_OK;
}

int rtc_set_partial_output(rtc_loop* L, float* device_ptr) {
    if (!L) return fail(nullptr, RTC_EINVAL, "loop is NULL");
    if (!L->partial) return fail(L, RTC_EINVAL, "the loop was not created with RTC_FLAG_PARTIAL");
    TRY(use_device(L));
    if (device_ptr) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, device_ptr) != cudaSuccess) {
            cudaGetLastError();
            return fail(L, RTC_EINVAL, "partial output is not device memory");
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
            return fail(L, RTC_EINVAL, "partial output is not device memory");
    }
    // frames already queued keep the pointer they read; the word is written in stream order
    for (cudaStream_t w : L->st_w) CK(L, cudaStreamSynchronize(w));
    CK(L, cudaStreamSynchronize(L->st));
    CK(L, cudaMemcpy(L->d_pout, &device_ptr, sizeof(float*), cudaMemcpyHostToDevice));
    return RTC_OK;
}

int rtc_get_info(rtc_loop* L, rtc_info* out) {
    if (!L || !out) return fail(L, RTC_EINVAL, "loop and out are required");
    out->na = L->na;
    out->ns = L->ns;
    out->nwfs = L->nwfs;
    out->nblocks = L->nblk;
    out->nrows = L->nrows;
    out->m_dtype = L->m_dtype;
    out->p_dtype = L->p_dtype;
    out->m_bytes = L->m_bytes;
    out->p_bytes = L->p_bytes;
    out->pixel_bytes = L->pixel_bytes;
    out->device_bytes = L->device_bytes;
    std::lock_guard<std::mutex> g(L->mu);
    out->frames_done = L->frames_done;
    out->frames_dropped = L->frames_dropped;
    out->frames_overrun = L->frames_overrun;
    out->swaps = L->swaps;
    out->prelaunch_used = L->pre_used;
    out->prelaunch_cancelled = L->pre_cancelled;
    out->prelaunch_expired = L->pre_expired;
    return RTC_OK;
}

const char* rtc_last_error(const rtc_loop* L) { return L ? L->err.c_str() : g_err.c_str(); }

int rtc_quantize_rows(int32_t dtype, int32_t na, int32_t ns, const float* M, size_t ld, void* codes, float* scale,
                      void* stream) {
    if ((dtype != RTC_BF16 && dtype != RTC_E4M3) || na < 0 || ns < 0 || ld < (size_t)ns)
        return fail(nullptr, RTC_EINVAL, "bad quantize arguments");
    if (na == 0) return RTC_OK;
    if (!M || !codes || !scale) return fail(nullptr, RTC_EINVAL, "NULL pointer");
    cudaError_t e = launch_quantize(dtype, na, ns, M, ld, codes, scale, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "quantize kernel");
    return RTC_OK;
}

}  // extern "C"
