// Internal device-side plans and kernel launchers of the AO RTC library.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/rtc.h"

namespace rtc {

constexpr int kMaxWfs = RTC_MAX_WFS;
constexpr int kSlopeThreads = 256;    // threads per slope-row CTA
constexpr int kGemvWarps = 8;         // warps per GEMV CTA

// Per-WFS constants read by the slope kernel.
struct WfsDev {
    int kind;                 // RTC_WFS_SH or RTC_WFS_PYRAMID
    int width, height;
    int npx, nsubx, nsuby, ox, oy;
    int pupil, qx[4], qy[4];
    float threshold;
    int thresh_mode;
    const float* dark;        // device, calib_pitch floats per row
    const float* flat;
    int calib_pitch;          // floats per calibration-map row (multiple of 4)
    int sh_groups;            // SH: row groups per CTA in the column-sum phase
    // pyramid with global normalisation (norm == RTC_NORM_GLOBAL): its slope rows
    // are always launched together, then normalised by a second kernel
    int norm;
    int gnrows;               // its slope rows
    int gpix;                 // valid pupil pixels
    int gflux;                // float offset of the per-row flux sums in the part scratch
};

// One slope row: a subaperture row (SH) or a pupil row (pyramid).
struct SlopeRow {
    int wfs;
    int row;                  // row index within its WFS
    int unit0;                // first entry of this row in the unit x-list
    int nunits;               // valid units in this row
    int s_pad;                // padded slope-buffer index of the row's first slope
    int s_compact;            // compact slope index of the row's first slope
    int nparts;               // CTAs sharing this row (split by pixel rows)
    int pscr;                 // float offset of this row's per-part sums (nparts > 1)
};

// One CTA of the slope kernel: pixel rows [pr0, pr1) of a subaperture row.
struct SlopePart {
    int row;                  // slope-row table index
    int part;                 // part index within the row
    int pr0, pr1;             // pixel rows within the subaperture (SH); unused for pyramid rows
};

// Everything one slope-kernel CTA needs from the plan, read with one set of
// 16-byte loads (the kernel is the first of a frame: a chain of dependent
// table loads would sit in its latency).
struct alignas(16) SlopeCta {
    SlopeRow row;
    SlopePart part;
};

constexpr int kFinRows = 32;  // rows per finalisation tile of the fused MVM tail

// Fused finalisation of the reconstruction MVM (enabled for the control matrix).
struct FinaliseArgs {
    int enabled;
    int nblk;                 // column blocks per frame
    unsigned* counters;       // per finalisation tile: rows done, summed over blocks
    const float* scale;       // control-matrix row scale or NULL
    const float* q;           // POLC term from the previous frame
    float* a;                 // integrator state
    float* cmd;               // commands (page-locked ring slot, mapped)
    float oml, gain;          // 1 - leak, gain
    int clip;
    float amin, amax;
    unsigned* tiles_done;     // tiles finalised this frame
    unsigned long long* done_flag;  // page-locked completion word of the ring slot, or NULL
    const unsigned long long* seq;  // page-locked word holding the value to write there (set by the
                                    // host before the launch, so a captured graph can be replayed)
    unsigned long long* t_done;     // device word of the slot: GPU global time (ns) when the commands
                                    // were complete, or NULL
    int partial;                    // shard loop (RTC_FLAG_PARTIAL): cmd gets the partial reconstruction,
                                    // no control law
    float* const* pout;             // device word: where else a shard writes it (NULL: nowhere)
};

// Mailbox of a pre-enqueued row chunk, in page-locked host memory.  The host
// writes px / pitch / row0 and then moves state from kChunkEmpty to kChunkFilled
// (or kChunkCancelled) with one compare-and-swap; a one-warp gate kernel ahead of
// the chunk's slope kernel waits a bounded time for a state other than
// kChunkEmpty and, when the time is up, moves it to kChunkExpired with the same
// compare-and-swap.  The first swap decides for both sides; the chunk's kernels
// do their work only on kChunkFilled.
enum : int { kChunkEmpty = 0, kChunkFilled = 1, kChunkCancelled = 2, kChunkExpired = 3 };
struct alignas(16) ChunkDesc {
    const uint16_t* px;       // device address of the chunk's first row
    long long pitch;          // uint16 elements
    int row0;                 // frame row of px
    int state;                // kChunk*
};
static_assert(sizeof(ChunkDesc) == 32, "chunk mailbox layout");
struct ChunkGate {
    ChunkDesc* desc;          // device address of the mailbox
    ChunkDesc* mirror;        // device memory: the settled mailbox, copied by the gate kernel for the
                              // chunk's slope and MVM kernels (whose many CTAs then read the L2, not
                              // one host cache line over the link)
    int wfs;                  // the WFS whose pixels it addresses
    unsigned max_polls;       // upper bound on the polls, whatever the clock says
    unsigned long long limit_ns;   // how long the kernel waits for the host
};

// Frame pointers for one launch; pitch in uint16 elements.  px[w] holds pixel
// row row0[w] of WFS w (row0 > 0 when only a chunk of the frame is addressed).
struct FramePtrs {
    const uint16_t* px[kMaxWfs];
    long long pitch[kMaxWfs];
    int row0[kMaxWfs];
};

// One reconstruction column block, stored as a dense [na][pitch] sub-matrix.
struct BlockDev {
    long long m_off;          // element offset of the sub-matrix
    int x_off;                // padded input-vector index of the block's first column
    int ncols;                // true columns
    int pitch;                // stored columns (multiple of 16 bytes / element size)
    int c0;                   // compact index of the block's first column
};

// Launch kernel<<<grid, block, smem, st>>>(args...) and return the launch's own
// status: an error that earlier work of the calling thread left pending is
// neither reported as this launch's nor cleared.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

size_t dtype_size(int dtype);
int elems_per_16B(int dtype);

// Opt the slope kernel in to more than 48 KB of dynamic shared memory when needed.
cudaError_t configure_slopes(int smem_bytes);

// Telemetry circular buffer (Section 3.3): one entry per recorded frame, in
// page-locked host memory written by the GPU.  An entry is a header of
// kTelHeaderFloats floats (TelHeader) and then the recorded sections.
constexpr int kTelHeaderFloats = 16;
struct TelHeader {
    unsigned long long index;       // entry number
    unsigned long long frame_id;
    unsigned long long t_commands;  // GPU global time (ns): commands complete
    unsigned long long t_written;   // GPU global time (ns): entry written
};
struct TelArgs {
    const BlockDev* blocks;
    int nblk, na, ns, nwfs;
    int blk_start[kMaxWfs + 1];     // column blocks of WFS w: [blk_start[w], blk_start[w + 1])
    const float* s_pad;             // slopes, padded block layout
    const float* a;                 // commands
    const float* part;              // unscaled per-block partial products, [nblk][na]
    const float* scale;             // control-matrix row scales or NULL
    unsigned streams;               // RTC_TEL_* sections recorded
    int off_s, off_a, off_p;        // float offsets of the sections after the header
    int decimate;                   // record every decimate-th frame that reaches telemetry
    long long depth;                // entries in the ring
    long long entry_floats;         // entry stride
    float* ring;                    // page-locked entries (device address)
    unsigned long long* wcount;     // page-locked: entries published so far
    unsigned long long* ctr;        // device: [0] frames seen, [1] entries written, [2] CTAs finished
    const unsigned long long* fid;  // page-locked: frame id of the slot
    const unsigned long long* t_cmd;  // device: the slot's command-complete time
};
cudaError_t launch_telemetry(const TelArgs& t, cudaStream_t st);

// Global pyramid normalisation over items [item0, item0 + nitems) (each a column
// block and its WFS); max_pairs bounds the slope pairs of one block.  pdl: a
// programmatic dependent of the slope kernel before it in the stream.
cudaError_t launch_normalise(const int2* items, int item0, int nitems, int max_pairs, const BlockDev* blocks,
                             const WfsDev* wfs, const float* pscr, const float* ref, const float* pol, float* s_pad,
                             bool pdl, cudaStream_t st);

// Slope kernel over the CTA table entries [cta0, cta0 + nctas).  gate: a
// pre-enqueued chunk; a one-warp kernel waits on the mailbox first, and the slope
// kernel, its programmatic dependent, takes the pixel pointer of WFS gate->wfs
// from the mailbox (and does nothing unless the host filled it).  The WFS table
// (nwfs entries, host memory) travels in the kernel parameters.  host_px: the
// variant that keeps all of a thread's pixel rows in flight, for small launches
// that read pixels in place from page-locked host memory.  Each slope is
// (measured - ref) + pol, with ref and pol (compact slope order) optional.
cudaError_t launch_slopes(const SlopeCta* ctas, int cta0, int nctas, const WfsDev* wfs, int nwfs,
                          const FramePtrs& fp, bool host_px, const uint16_t* xlist, const float* ref,
                          const float* pol, float* s_pad, float* pscr, unsigned* counters, int smem_bytes,
                          cudaStream_t st, const ChunkGate* gate = nullptr);

// GEMV over blocks [b0, b0 + nb): out[b * out_stride + r] = sum_j M_b[r][j] x[x_off_b + j],
// times out_scale[r] when out_scale is not NULL; with fin, the CTA completing the
// last block of a row tile also finalises it (a, cmd) and the last tile sets the
// completion word.  pdl: launched as a programmatic dependent of the previous
// kernel in the stream (prefetches matrix tiles into L2, then waits for it);
// avg_row_bytes sizes that prefetch.  gate_state: a pre-enqueued chunk's settled
// mailbox state (device memory), read after that wait; the launch does nothing
// unless it is kChunkFilled.
cudaError_t launch_gemv(int dtype, const void* M, const BlockDev* blocks, int b0, int nb,
                        int na, const float* x, const float* out_scale, float* out,
                        long long out_stride, const FinaliseArgs* fin, long long avg_row_bytes,
                        bool pdl, cudaStream_t st, const int* gate_state = nullptr);

// Telemetry: compact copy of the padded slope buffer, block by block.
cudaError_t launch_pack_slopes(const BlockDev* blocks, int nblk, int max_cols,
                               const float* s_pad, float* out, cudaStream_t st);

// Create-time relayout of a row-major [na][ns] matrix into column blocks (zero padding).
cudaError_t launch_relayout(int dtype, const void* src, int na, int ns, const BlockDev* blocks,
                            int nblk, int max_pitch, void* dst, cudaStream_t st);

// Per-row scaled quantisation (rtc_quantize_rows).
cudaError_t launch_quantize(int dtype, int na, int ns, const float* M, size_t ld, void* codes,
                            float* scale, cudaStream_t st);

// Finite check of a device float array; sets *bad (device int) to 1 if a NaN/Inf is found.
cudaError_t launch_check_finite(const float* x, size_t n, int* bad, cudaStream_t st);

// Loop internals used by the multi-loop server (implemented in rtc_runtime.cu).
// The ring slot and completion value of the frame submitted last.
void loop_last_frame(const rtc_loop* L, int* slot, unsigned long long* seq);
// Whether that frame's commands are written (reads its page-locked completion word).
bool loop_frame_done(const rtc_loop* L, int slot, unsigned long long seq);

}  // namespace rtc
