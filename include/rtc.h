/*
 * rtc.h - C ABI of the GB300 adaptive-optics real-time-control hot path.
 *
 * The path follows the per-frame pipeline of Jenkins, Basden & Myers,
 * "A many-core CPU prototype of an MCAO and LTAO RTC for ELT-scale
 * instruments" (arXiv 1903.01852):
 *
 *   WFS pixels (streamed in row chunks, Section 2.1-2.2)
 *     -> calibration (dark subtraction, flat field, threshold; Section 2.2)
 *     -> Shack-Hartmann centre-of-gravity or pyramid quad-difference slopes
 *        (Fig. wfs_slopes, Section 2.2; pyramid normalised locally or globally)
 *     -> reconstruction matrix-vector multiply, one partial per column block
 *        (Section 2.3; per-WFS partial DM commands summed by a master, Section 3)
 *     -> implicit (or explicit) pseudo-open-loop control term + leaky
 *        integrator (Section 3.4) -> DM commands, tagged with the camera frame
 *        number (Section 3, Fig. mcaoltao_test)
 *     -> telemetry: per-frame slope ring and an optional circular buffer of
 *        slopes, commands and per-WFS partial commands (Section 3.3); parameter
 *        changes through a double buffer (Section 3.2).
 *
 * Conventions for every entry point:
 *   - Sizes are element counts unless a name ends in "pitch" (bytes).
 *   - Every input array is owned by the caller and is copied (or, for the
 *     device-resident frame entry point, read in place) before the call
 *     returns its status; the library keeps no caller pointer after the call,
 *     except as stated for rtc_submit_pixels / rtc_process_frame.
 *   - Calls return an int status: RTC_OK (0) or a negative RTC_E* code.
 *     No C++ exception crosses the ABI.  The text of the last failure is
 *     available from rtc_last_error().
 *   - One thread submits to a loop; any thread may call rtc_get_commands,
 *     rtc_get_telemetry, rtc_get_timing, rtc_telemetry_read and rtc_update.
 *
 * Slope order (the paper does not fix one): interleaved (x, y) per valid
 * unit, units in row-major order of the subaperture grid (SH) or of the pupil
 * (pyramid), WFS after WFS in the order given at creation.  Column j of the
 * control matrix multiplies slope j.
 */
#ifndef RTC_H
#define RTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define RTC_OK         0
#define RTC_EINVAL    -1  /* bad argument: size, pointer, enum, alignment, NaN/Inf in a map */
#define RTC_ENOMEM    -2  /* device or page-locked host memory could not be had (HBM admission) */
#define RTC_ETIMEDOUT -3  /* a wait ran out before the result was ready */
#define RTC_EORDER    -4  /* chunk rejected: frame id not increasing, or rows not contiguous */
#define RTC_EDROPPED  -5  /* chunk accepted, but the previous frame was incomplete and was dropped */
#define RTC_ECUDA     -6  /* a CUDA runtime call failed; the loop should be destroyed */
#define RTC_ENOENT    -7  /* the requested frame is no longer (or not yet) in the ring */
#define RTC_ENOTSUP   -8  /* the device lacks a capability the request needs */

/* ---- enumerations ---------------------------------------------------- */
#define RTC_WFS_SH       0  /* Shack-Hartmann: centre of gravity per subaperture */
#define RTC_WFS_PYRAMID  1  /* pyramid: normalised quad difference per pupil pixel */

#define RTC_F32   0         /* IEEE binary32 */
#define RTC_BF16  1         /* bfloat16 codes (uint16 bit patterns) */
#define RTC_E4M3  2         /* FP8 E4M3 (finite-only, max 448) codes (uint8 bit patterns) */

#define RTC_THRESH_SUBTRACT 0  /* t = max(c - T, 0) */
#define RTC_THRESH_CLIP     1  /* t = c if c > T else 0 */

#define RTC_NORM_LOCAL  0   /* pyramid: divide by each pixel's own flux A+B+C+D */
#define RTC_NORM_GLOBAL 1   /* pyramid: divide by the mean flux over the valid pupil pixels */

#define RTC_POLC_IMPLICIT 0 /* q = P a added to the reconstruction (Section 3.4, implicit form) */
#define RTC_POLC_EXPLICIT 1 /* s + D a formed before the reconstruction (explicit form) */

#define RTC_FLAG_TIMING     1u /* record frame-level CUDA events (rtc_get_timing) */
#define RTC_FLAG_TELEMETRY  2u /* copy slopes of every frame to the page-locked ring */
#define RTC_FLAG_STAGE_TIMING 4u /* also time the slope and MVM kernels separately; this
                                    serialises them (no early start of the MVM) */
#define RTC_FLAG_UPDATABLE  8u /* keep shadow copies of the parameters for rtc_update
                                  (twice the matrix memory, plus 64 MiB of page-locked
                                  host memory to stage the uploads) */
#define RTC_FLAG_GRAPHS    16u /* page-locked input frames per ring slot and one captured CUDA
                                  graph per slot (rtc_next_frame_buffers, rtc_submit_frame_graph);
                                  excludes RTC_FLAG_UPDATABLE and RTC_FLAG_STAGE_TIMING */
#define RTC_FLAG_PARTIAL   32u /* a shard of a loop split by WFS (rtc_master): the loop computes
                                  only its WFS's partial reconstruction and no control law;
                                  polc->P and polc->D must be NULL */
#define RTC_FLAG_PRELAUNCH 64u /* pre-enqueue the kernels of each Shack-Hartmann row chunk when the
                                  previous chunk of its WFS is submitted (see rtc_submit_pixels);
                                  excludes RTC_FLAG_TIMING and RTC_FLAG_STAGE_TIMING; RTC_ENOTSUP on
                                  a device without native atomics on host memory */

#define RTC_MAX_WFS 16

/* Sections of a telemetry circular-buffer entry (rtc_geometry.tel_streams). */
#define RTC_TEL_SLOPES   1u /* the frame's slopes (ns floats; POL slopes in explicit-POLC mode) */
#define RTC_TEL_COMMANDS 2u /* the frame's commands (na floats) */
#define RTC_TEL_PARTIALS 4u /* per-WFS partial commands: nwfs x na floats, the reconstruction of
                               each WFS's slopes alone (what the paper's reconstruction nodes
                               send to the master, Section 3), before POLC and the integrator */

/* ---- creation-time descriptions ------------------------------------- */

/* One wavefront sensor.  Pixel frames are uint16, row-major, height x width.
 * SH: a grid of nsuby x nsubx subapertures of npx x npx pixels whose top-left
 * pixel is (ox, oy); the grid must lie inside the frame.
 * Pyramid: four pupil images of pupil x pupil pixels with top-left pixels
 * (qx[k], qy[k]) for k = A (top-left), B (top-right), C (bottom-left),
 * D (bottom-right); each must lie inside the frame.
 * valid: host uint8, row-major, nsuby x nsubx (SH) or pupil x pupil (pyramid);
 * non-zero marks a valid unit; NULL means every unit is valid.
 * nblocks: number of reconstruction column blocks this WFS's slopes are split
 * into, by whole slope rows (subaperture rows or pupil rows), as evenly as
 * possible; a block's MVM starts as soon as its pixel rows have arrived
 * (Section 2.2: centroiding starts when a row of subapertures is complete).
 * 1 <= nblocks <= number of slope rows.
 * norm (pyramid only; 0 for SH): RTC_NORM_LOCAL divides each pupil pixel's
 * quad differences by its own flux N = A+B+C+D (Fig. wfs_slopes, "relative
 * differences"); RTC_NORM_GLOBAL divides them by the mean of N over the valid
 * pupil pixels (every slope 0 when that mean is not positive).  A globally
 * normalised WFS computes its slopes, and starts its column blocks' MVM, only
 * once its whole frame has arrived, since every slope needs every pixel. */
typedef struct rtc_wfs {
    int32_t kind;
    int32_t width, height;
    int32_t nsubx, nsuby, npx, ox, oy;   /* SH only */
    int32_t pupil, qx[4], qy[4];         /* pyramid only */
    const uint8_t* valid;
    int32_t nblocks;
    int32_t norm;                        /* RTC_NORM_* (pyramid only) */
} rtc_wfs;

/* The loop's sensors and run-time options.
 * tel_depth > 0 adds a telemetry circular buffer (Section 3.3: DARC keeps
 * telemetry in circular buffers that readers drain while the loop runs) of
 * tel_depth entries in page-locked host memory, written by the GPU after each
 * recorded frame's commands, off the latency path.  Every tel_decimate-th
 * frame that completes is recorded (tel_decimate >= 1), with the sections
 * tel_streams (RTC_TEL_*, may be 0 for timing records only).  Read it with
 * rtc_telemetry_read.  0 <= tel_depth <= 1 << 20. */
typedef struct rtc_geometry {
    int32_t nwfs;                /* 1..RTC_MAX_WFS */
    const rtc_wfs* wfs;          /* host array of nwfs */
    int32_t device;              /* CUDA device ordinal */
    uint32_t flags;              /* RTC_FLAG_* */
    int32_t ring;                /* depth of the page-locked command/telemetry ring, >= 2 */
    int32_t tel_depth;           /* telemetry circular-buffer entries, 0 for none */
    uint32_t tel_streams;        /* RTC_TEL_* */
    int32_t tel_decimate;        /* record every n-th frame (0 is taken as 1) */
    int32_t priority;            /* scheduling priority of the loop's streams among the loops on
                                    its GPU: 0 (default) the highest, each step one level lower
                                    (clamped to the device's lowest); a loop with a shorter frame
                                    period given a higher priority gets the SMs first when frames
                                    of several loops are on the GPU together (rtc_server) */
    int32_t prelaunch_wait_us;   /* RTC_FLAG_PRELAUNCH: how long pre-enqueued kernels wait for their
                                    chunk before they give up, 0..1000000 (0 is taken as 10000) */
} rtc_geometry;

/* Pixel calibration (Section 2.2): c = (raw - dark) * flat, then the threshold.
 * Each map is host float32, row-major height x width of its WFS.
 * dark / flat: arrays of nwfs pointers; the array or an entry may be NULL
 * (dark 0, flat 1).  threshold: nwfs values >= 0 or NULL (0).  thresh_mode:
 * nwfs RTC_THRESH_* values or NULL (SUBTRACT).  ref_slopes: ns reference
 * slopes subtracted from the measured ones, or NULL.
 * Whether a pixel is lit (t > 0) is decided on the float32 value
 * fl(fl(raw - dark) * flat) compared with T. */
typedef struct rtc_calib {
    const float* const* dark;
    const float* const* flat;
    const float* threshold;
    const int32_t* thresh_mode;
    const float* ref_slopes;
} rtc_calib;

/* Control (reconstruction) matrix M, na x ns, host, row-major, element type
 * dtype (RTC_F32 floats, RTC_BF16 uint16 codes, RTC_E4M3 uint8 codes).
 * row_scale: host float32[na] multiplying each row (required for BF16/E4M3
 * codes produced by rtc_quantize_rows; optional for F32), or NULL.
 * ns must equal the loop's slope count.  The matrix is re-laid out into
 * column blocks in device memory; the caller's copy is not kept. */
typedef struct rtc_cmat {
    int32_t na, ns;
    int32_t dtype;
    const void* data;
    const float* row_scale;
} rtc_cmat;

/* Control law.  mode RTC_POLC_IMPLICIT (0), implicit POLC (Section 3.4):
 *   a_k = (1 - leak) a_{k-1} + gain (M s_k + q_{k-1}),  q_k = P a_k,
 * then the optional clip to [amin, amax].  q_k is computed after frame k's
 * commands are ready, for frame k+1, off the latency path.
 * P: host row-major na x na of element type dtype with optional row_scale,
 * or NULL for a plain leaky integrator (q = 0).  a0: host float32[na]
 * initial commands, or NULL for zeros.
 * mode RTC_POLC_EXPLICIT (1), the explicit form of Section 3.4: the
 * pseudo-open-loop slopes s_ol = s_k + u_{k-1} are formed first, with
 * u_k = D a_k computed after frame k's commands (off the latency path), and
 *   a_k = (1 - leak - gain) a_{k-1} + gain M s_ol,  then the optional clip.
 * D: host row-major ns x na interaction matrix of element type d_dtype with
 * optional d_row_scale (float32[ns]); required in this mode, and P must be
 * NULL.  The telemetry slopes of such a loop are s_ol.  With P = M D - I the
 * two modes give the same commands; the explicit one streams ns x na matrix
 * elements per frame for the POLC term instead of na x na. */
typedef struct rtc_polc {
    const void* P;
    int32_t dtype;
    const float* row_scale;
    float gain, leak;
    const float* a0;
    int32_t clip;
    float amin, amax;
    int32_t mode;                /* RTC_POLC_* */
    const void* D;               /* explicit mode: ns x na, or NULL */
    int32_t d_dtype;
    const float* d_row_scale;
} rtc_polc;

typedef struct rtc_loop rtc_loop;   /* opaque */

/* A control loop (Fig. ao_diag: pixel handling, reconstruction, control law;
 * Table ao_compare: the instrument configurations).  Validate the
 * description, copy every map and matrix into device memory of
 * geometry->device (admission fails with RTC_ENOMEM when they do not fit),
 * build the slope-row and column-block plans, allocate the page-locked
 * command ring and the CUDA streams and events.  On success *out is a new
 * loop; on failure *out is NULL and rtc_last_error(NULL) has the reason. */
int rtc_create(const rtc_geometry* geometry, const rtc_calib* calib,
               const rtc_cmat* cmat, const rtc_polc* polc, rtc_loop** out);

/* Wait for all work of the loop, then release everything it holds.
 * NULL is accepted.  The loop must not be used afterwards. */
int rtc_destroy(rtc_loop* loop);

/* ---- per-frame entry points ----------------------------------------- */

/* A run of whole pixel rows [row_begin, row_end) of one WFS frame.
 * px points at the first pixel of row_begin, in host memory (pageable or
 * page-locked) or device memory; rows are pitch bytes apart (pitch >=
 * 2*width).  frame_id is the camera's frame number (Section 3: it is
 * carried through to the DM command). */
typedef struct rtc_chunk {
    uint64_t frame_id;
    int32_t wfs;
    int32_t row_begin, row_end;
    const uint16_t* px;
    size_t pitch;
} rtc_chunk;

/* Pixel-stream ingest (Section 2.1-2.2).  Enqueues the copy of the rows into
 * the loop's frame buffer, the calibration + slopes of every slope row those
 * rows complete, and the MVM of every column block they complete; when the
 * last row of the last WFS of the frame arrives, also the finalisation
 * (partial sums + POLC term + integrator) that writes the commands, then the
 * POLC product for the next frame.  Returns without waiting for the GPU.
 * Rows of one WFS must arrive in order without gaps; WFS may interleave.
 * A chunk of a new (larger) frame_id while the current frame is incomplete
 * drops the current frame (its commands are never produced, the integrator
 * state is unchanged) and returns RTC_EDROPPED with the chunk accepted.
 * A smaller or repeated frame_id of a completed frame, or non-contiguous
 * rows, return RTC_EORDER and change nothing.
 * px from pageable memory may be reused when the call returns; px in
 * page-locked or device memory must stay unchanged until rtc_get_commands
 * has returned this frame.
 * RTC_FLAG_PRELAUNCH (no counterpart in the paper, whose nodes launch work
 * as pixels arrive): after a Shack-Hartmann chunk that leaves rows of its WFS
 * to come, the call also enqueues the slope and MVM kernels of that WFS's next
 * chunk as the previous frame had it (same rows, read in place), ahead of
 * its arrival.  Their CTAs wait on a page-locked mailbox for at most
 * geometry->prelaunch_wait_us; when the chunk arrives with those rows, in
 * page-locked or device memory that can be read in place, the call only writes
 * its address to the mailbox, so the GPU starts on it without a launch.
 * Otherwise (other rows, pixels that must be copied, a dropped frame, the loop
 * destroyed) the mailbox is cancelled and the kernels do nothing; if the wait
 * ran out first, they gave up the same way.  Both cases fall back to ordinary
 * launches, with the same results.  rtc_get_info counts the three outcomes.
 * Nothing is enqueued ahead for a chunk the previous frame did not have (or
 * copied), for one that completes no subaperture row, or while four earlier
 * pre-enqueued chunks of the same camera still have kernels running (a host
 * that runs ahead of the GPU): such a chunk takes ordinary launches.
 * While kernels wait, anything that waits for all work on the device
 * (cudaDeviceSynchronize, cudaFree, another loop's rtc_destroy), and this
 * loop's own rtc_sync, rtc_get_state, rtc_set_state, rtc_check_guards and
 * rtc_set_partial_output called in the middle of a frame, wait for them too:
 * until their chunk arrives, the frame is dropped or the loop destroyed, or
 * the wait runs out (and the chunk then takes ordinary launches). */
int rtc_submit_pixels(rtc_loop* loop, const rtc_chunk* chunk);

/* Several chunks in one call (no counterpart in the paper; for a host that
 * receives the rows of several cameras at once): the same as calling
 * rtc_submit_pixels on chunks[0], ..., chunks[n-1] in that order.  Stops at
 * the first chunk that fails and returns its status; *accepted (may be NULL)
 * receives the number of chunks accepted before it.  Returns RTC_EDROPPED if
 * any accepted chunk dropped a frame, else RTC_OK.  n = 0 does nothing. */
int rtc_submit_pixels_n(rtc_loop* loop, const rtc_chunk* chunks, int32_t n, int32_t* accepted);

/* Whole-frame entry point (Section 2.2's pixel handling for a whole frame at
 * once), for frames in device memory (e.g. written there by a frame grabber)
 * or in page-locked host memory (read over the CPU-GPU link): px[w] points at
 * WFS w's frame (16-byte aligned), pitch[w] is its row pitch in bytes (a
 * multiple of 16, >= 2*width rounded up to 16); pageable memory is rejected
 * with RTC_EINVAL.  The slope kernels read the frames in place; they must
 * stay unchanged until rtc_get_commands returns this frame.  Otherwise
 * behaves like submitting every row of every WFS at once. */
int rtc_process_frame(rtc_loop* loop, uint64_t frame_id,
                      const uint16_t* const* px, const size_t* pitch);

/* Graph mode (RTC_FLAG_GRAPHS): the page-locked buffers, one per WFS (px[w],
 * rows pitch[w] bytes apart, host addresses the GPU reads in place over the
 * CPU-GPU link), into which the caller writes the next frame; waits until
 * the GPU has finished the frame that last used them.  Valid until the next
 * rtc_submit_frame_graph. */
int rtc_next_frame_buffers(rtc_loop* loop, uint16_t** px, size_t* pitch);

/* Graph mode: launch the CUDA graph captured at creation for the buffers the
 * last rtc_next_frame_buffers returned (slopes, MVM with finalisation, POLC,
 * telemetry: one launch instead of four kernels and their events).  Frame-id
 * rules as rtc_process_frame. */
int rtc_submit_frame_graph(rtc_loop* loop, uint64_t frame_id);

/* The DM commands of a frame (Section 3: the master's sum of the partial
 * commands after POLC and the control law, tagged with the camera frame
 * number).  Wait (busy-polling, up to timeout_us microseconds; <0 waits
 * forever) for the oldest frame whose pixels are all submitted and whose commands have not
 * yet been returned, then copy its na commands to out (host) and its frame
 * id to *frame_id.  RTC_ETIMEDOUT leaves that frame queued.  The ring keeps
 * the last `ring` frames; older unread ones are discarded. */
int rtc_get_commands(rtc_loop* loop, float* out, size_t n, uint64_t* frame_id,
                     int64_t timeout_us);

/* Telemetry (Section 3.3): copy the slopes (ns, measured minus reference)
 * and commands (na) of frame_id, if it is still in the ring, to host
 * buffers; either pointer may be NULL.  Needs RTC_FLAG_TELEMETRY for slopes.
 * Waits up to timeout_us for that frame's GPU work. */
int rtc_get_telemetry(rtc_loop* loop, uint64_t frame_id, float* slopes, size_t ns,
                      float* cmds, size_t na, int64_t timeout_us);

/* Device times of one frame (the latency of Table ao_results, measured on the
 * GPU), from CUDA events on the loop's stream (needs RTC_FLAG_TIMING).  latency_us: for rtc_process_frame, from just before the
 * slope kernel to the end of the MVM kernel, whose tail writes the commands;
 * for chunked frames, from just before the last chunk's work.  frame_us: from
 * the frame's first submitted work to the commands.  polc_us: the POLC
 * product after the commands.  slopes_us and mvm_us (the MVM kernel with its
 * fused finalisation) need RTC_FLAG_STAGE_TIMING, else they are -1;
 * final_us is 0 (the finalisation is part of the MVM kernel).  In graph mode
 * (RTC_FLAG_GRAPHS) latency_us and frame_us span the whole graph launch, POLC
 * and telemetry included, and polc_us is about 0; RTC_FLAG_STAGE_TIMING is not
 * available there. */
typedef struct rtc_timing {
    uint64_t frame_id;
    float slopes_us, mvm_us, final_us, polc_us;
    float latency_us, frame_us;  /* frame_us: first submitted work to end of finalise */
} rtc_timing;
int rtc_get_timing(rtc_loop* loop, uint64_t frame_id, rtc_timing* out, int64_t timeout_us);

/* ---- telemetry circular buffer (Section 3.3) ------------------------------ */

/* One entry's record.  Times are the GPU's global timer in nanoseconds, so
 * differences between records are device frame times. */
typedef struct rtc_tel_record {
    uint64_t index;              /* entry number: 0, 1, 2, ... over recorded frames */
    uint64_t frame_id;
    uint64_t t_commands_ns;      /* when the frame's commands were complete */
    uint64_t t_written_ns;       /* when the entry was written */
    uint64_t lost;               /* entries overwritten before this reader reached them, since the
                                    previous successful read */
} rtc_tel_record;

/* The oldest entry not yet read, waiting up to timeout_us (< 0: forever) for
 * one to be published.  A reader that falls more than tel_depth - 1 entries
 * behind loses the oldest ones (counted in rec->lost), as with DARC's circular
 * buffers; an entry that the GPU may have been rewriting while it was copied is
 * also counted lost.  slopes (ns floats), cmds (na floats) and partials
 * (nwfs x na floats, row-major by WFS) receive the recorded sections and may
 * be NULL; a non-NULL pointer for a section the loop does not record, or a
 * wrong size, is RTC_EINVAL.  One reader at a time per loop (calls are
 * serialised).  RTC_ETIMEDOUT when nothing new was published in time;
 * RTC_EINVAL when the loop has no telemetry buffer. */
int rtc_telemetry_read(rtc_loop* loop, rtc_tel_record* rec, float* slopes, size_t ns, float* cmds, size_t na,
                       float* partials, size_t npartials, int64_t timeout_us);

/* Telemetry streaming (Section 3.3: DARC reads its circular buffers and sends
 * the telemetry on, e.g. to disk): a library thread takes over as the
 * buffer's reader and writes every entry it gets to the file descriptor fd,
 * as the rtc_tel_record (40 bytes) followed by the recorded sections in the
 * order slopes, commands, partial commands (float32).  fd stays owned by the
 * caller and must stay open until rtc_telemetry_stream_stop.  While a stream
 * runs, rtc_telemetry_read returns RTC_EINVAL.  RTC_EINVAL without a
 * telemetry buffer or when a stream already runs. */
int rtc_telemetry_stream_start(rtc_loop* loop, int fd);

typedef struct rtc_tel_stream_stats {
    uint64_t entries;            /* entries written to fd */
    uint64_t lost;               /* entries the stream lost (overwritten before it read them) */
    uint64_t bytes;              /* bytes written */
    int32_t write_error;         /* errno of the first failed write (the stream then stops), or 0 */
} rtc_tel_stream_stats;

/* Stop the stream: the thread first writes every entry already published,
 * then exits; *stats (may be NULL) receives its totals.  RTC_EINVAL when no
 * stream runs. */
int rtc_telemetry_stream_stop(rtc_loop* loop, rtc_tel_stream_stats* stats);

/* ---- parameter double buffer (Section 3.2) ----------------------------- */

/* New parameters for a running loop.  Every pointer may be NULL (unchanged);
 * shapes and element types are those given at creation.  M: host row-major
 * na x ns in the loop's matrix type, with M_scale (float32[na]) when the loop
 * was created with row scales (NULL keeps the current scales).  P / P_scale:
 * the same for the POLC matrix (loop created with implicit POLC; the D of an
 * explicit-POLC loop is fixed at creation, and a P for it is RTC_EINVAL).  dark / flat: arrays
 * of nwfs host pointers (entries may be NULL).  threshold: nwfs values or NULL.
 * ref_slopes: ns values.  set_control non-zero replaces gain, leak and the clip. */
typedef struct rtc_update_desc {
    const void* M;
    const float* M_scale;
    const void* P;
    const float* P_scale;
    const float* const* dark;
    const float* const* flat;
    const float* threshold;
    const float* ref_slopes;
    int32_t set_control;
    float gain, leak;
    int32_t clip;
    float amin, amax;
} rtc_update_desc;

/* Parameter change without stopping the loop, as DARC's double buffer
 * (Section 3.2): the new values are copied into shadow buffers on a separate
 * low-priority stream while frames keep running, then the first frame that
 * starts after this call returns uses them (the swap is a host-side pointer
 * exchange at the frame boundary, with no work added to that frame on the
 * GPU).  The matrices are gathered by the calling thread into two page-locked
 * staging buffers and copied from there, so no driver call holds a large
 * pageable copy.  The POLC term that frame uses was computed with the previous P; the
 * new P applies from that frame's own POLC product on.  Blocks the calling
 * thread (not the submitting one) until the upload is done; a second call
 * before the swap replaces the pending values.  Needs RTC_FLAG_UPDATABLE;
 * RTC_EINVAL for bad arguments or NaN/Inf values (nothing is swapped then). */
int rtc_update(rtc_loop* loop, const rtc_update_desc* desc);

/* ---- state and introspection ---------------------------------------- */

/* The control-law state (the DM commands a of the last frame, on which the
 * implicit-POLC term of Section 3.4 acts).  Wait for queued work, then copy
 * the integrator state a (na floats) out. */
int rtc_get_state(rtc_loop* loop, float* a, size_t na);
/* Wait for queued work, then set a and recompute q = P a, or u = D a in
 * explicit-POLC mode (checkpoint resume). */
int rtc_set_state(rtc_loop* loop, const float* a, size_t na);
/* Wait for all queued work of the loop. */
int rtc_sync(rtc_loop* loop);

/* Memory-safety check for tests: every device and page-locked buffer the loop
 * allocated ends in 256 guard bytes of a fixed pattern; after waiting for the
 * loop's work, *corrupted receives the number of guard regions that anything
 * (a kernel writing past a buffer, a copy) changed, 0 when all are intact. */
int rtc_check_guards(rtc_loop* loop, int32_t* corrupted);

/* The loop's CUDA stream (a cudaStream_t) in *stream, so a caller can order
 * its own work or timing events after the loop's; the loop keeps ownership. */
int rtc_get_stream(rtc_loop* loop, void** stream);

typedef struct rtc_info {
    int32_t na, ns, nwfs, nblocks, nrows;
    int32_t m_dtype, p_dtype;
    uint64_t m_bytes;          /* bytes of the stored matrix streamed per frame (incl. padding) */
    uint64_t p_bytes;          /* bytes of the stored POLC matrix (0 without POLC) */
    uint64_t pixel_bytes;      /* raw + calibration bytes read per frame by the slope kernels */
    uint64_t device_bytes;     /* device memory held by the loop */
    uint64_t frames_done, frames_dropped, frames_overrun;
    uint64_t swaps;            /* parameter swaps applied (rtc_update) */
    uint64_t prelaunch_used;       /* RTC_FLAG_PRELAUNCH: chunks whose pre-enqueued kernels ran them */
    uint64_t prelaunch_cancelled;  /* ... whose arrival did not match them (other rows, pixels to copy)
                                      or that were abandoned (frame dropped, loop destroyed) */
    uint64_t prelaunch_expired;    /* ... whose kernels stopped waiting before the chunk arrived */
} rtc_info;
int rtc_get_info(rtc_loop* loop, rtc_info* out);

/* No counterpart in the paper (DARC sizes nodes by hand): device memory a loop
 * with this description would hold once created
 * (resident_bytes) and at most during creation (peak_bytes, with the upload
 * buffers), computed from the description alone without touching the GPU;
 * this is what admission by HBM footprint uses.  Validation as rtc_create. */
int rtc_footprint(const rtc_geometry* geometry, const rtc_calib* calib, const rtc_cmat* cmat,
                  const rtc_polc* polc, uint64_t* resident_bytes, uint64_t* peak_bytes);

/* Text of the last failure on this loop, or (loop NULL) of the last failed
 * rtc_create / stateless call on the calling thread.  Never NULL. */
const char* rtc_last_error(const rtc_loop* loop);

/* ---- stateless device operations ------------------------------------ */

/* Per-row scaled quantisation of a float32 matrix in device memory (no
 * counterpart in the paper, whose matrices are float32: reduced-precision
 * storage for the memory-bound MVM of Section 2.3), for storing M or P in BF16
 * or E4M3 (halving / quartering the bytes the MVM
 * streams).  scale_r = max_j |M_rj| (BF16) or max_j |M_rj| / 448 (E4M3),
 * 1 for an all-zero row; code_rj = round-to-nearest-even of fl(M_rj/scale_r),
 * saturating at +-448 for E4M3.  M: device float32, row r at M + r*ld.
 * codes: device, row-major na x ns (uint16 for BF16, uint8 for E4M3).
 * scale: device float32[na].  stream: a cudaStream_t or NULL (legacy
 * default stream).  Asynchronous; returns RTC_EINVAL on bad arguments. */
int rtc_quantize_rows(int32_t dtype, int32_t na, int32_t ns, const float* M, size_t ld,
                      void* codes, float* scale, void* stream);

/* ---- multi-loop server ---------------------------------------------------- */

/* Several independent loops (SCAO, LTAO, MCAO ...) resident on one GPU, in the
 * spirit of the paper's several DARC instances feeding one controller
 * (Section 3), but whole loops sharing one device.  Loops are admitted by their
 * device-memory footprint (rtc_footprint) against a budget; a loop that does
 * not fit yet waits in a queue, with a private copy of its description, and is
 * created when released loops free enough memory (arrival order).  Admitted
 * loops run in graph mode (their flags gain RTC_FLAG_GRAPHS and lose
 * RTC_FLAG_UPDATABLE and the timing flags): each frame is one CUDA graph
 * launch on the loop's own stream, so frames of different loops overlap on
 * the device.  A server thread polls the completion words and records, per
 * loop, the latency from rtc_server_submit to the commands being written. */
typedef struct rtc_server rtc_server;

typedef struct rtc_server_loop_info {
    int32_t admitted;          /* 1 resident on the device, 0 waiting in the queue */
    uint64_t footprint_bytes;
    uint64_t frames;           /* latency samples recorded (since the last reset) */
    double p50_us, p99_us, p999_us, mean_us, jitter_rms_us, max_us;
} rtc_server_loop_info;

/* A server on device `device` with a device-memory budget in bytes. */
int rtc_server_create(int32_t device, uint64_t hbm_budget_bytes, rtc_server** out);
/* Stop the poller, destroy every loop, free the server.  NULL is accepted. */
int rtc_server_destroy(rtc_server* server);
/* Admit a loop (created now if it fits in the budget and nothing is queued
 * ahead of it) or queue it; *loop_id names it either way.  RTC_ENOMEM if its
 * footprint exceeds the whole budget; creation errors as rtc_create. */
int rtc_server_admit(rtc_server* server, const rtc_geometry* geometry, const rtc_calib* calib,
                     const rtc_cmat* cmat, const rtc_polc* polc, int32_t* loop_id);
/* Destroy a loop (after its queued work and any rtc_server_submit for it that
 * is in progress on another thread) or drop it from the queue, then create
 * queued loops that now fit.  The loop's handle from rtc_server_loop is
 * invalid afterwards. */
int rtc_server_release(rtc_server* server, int32_t loop_id);
/* The admitted loop's handle in *loop (NULL while queued), for
 * rtc_next_frame_buffers, rtc_get_commands, rtc_get_telemetry and the state calls. */
int rtc_server_loop(rtc_server* server, int32_t loop_id, rtc_loop** loop);
/* Launch the loop's next frame graph (rtc_submit_frame_graph) and track its
 * latency.  Different loops may be submitted from different threads; one
 * thread at a time per loop. */
int rtc_server_submit(rtc_server* server, int32_t loop_id, uint64_t frame_id);
/* Latency statistics and admission state of a loop; reset != 0 clears the samples. */
int rtc_server_stats(rtc_server* server, int32_t loop_id, int32_t reset, rtc_server_loop_info* out);
/* Bytes admitted against the budget, the budget, and loop counts. */
int rtc_server_usage(rtc_server* server, uint64_t* used_bytes, uint64_t* budget_bytes, int32_t* admitted,
                     int32_t* queued);
/* Text of the server's last failure.  Never NULL. */
const char* rtc_server_last_error(const rtc_server* server);

/* ---- per-WFS sharding (Section 3, Fig. mcaoltao_test) ---------------------
 *
 * The paper runs one reconstruction node per WFS and a master that adds the
 * nodes' partial DM commands and applies the control law.  A loop created with
 * RTC_FLAG_PARTIAL is such a node: for its WFS (their columns of the control
 * matrix, in their slope order) each frame gives the partial reconstruction
 *   y[r] = row_scale[r] * sum_j M[r][j] s[j]
 * in place of commands: rtc_get_commands returns y, and the loop's state, POLC
 * term and clip are unused.  A master holds the control law of the whole loop:
 *   a_k = (1 - leak) a_{k-1} + gain (sum_k y_k + q_{k-1}), optional clip,
 *   q_k = P a_k (implicit POLC, computed after the commands),
 * with the shards' partials added in shard order. */

/* Where a RTC_FLAG_PARTIAL loop's kernel also writes y (na floats) each frame:
 * device memory of any GPU the loop's device can write (the caller enables
 * peer access between different GPUs), typically rtc_master_input of a
 * master; NULL stops it.  Takes effect for frames submitted after the call
 * (graph mode included: the pointer is read by the kernel each frame).  The
 * caller keeps the buffer valid while frames run.  RTC_EINVAL if the loop is
 * not RTC_FLAG_PARTIAL or the pointer is not device memory. */
int rtc_set_partial_output(rtc_loop* loop, float* device_ptr);

typedef struct rtc_master rtc_master;   /* opaque */

typedef struct rtc_master_desc {
    int32_t device;              /* CUDA device of the master */
    int32_t na;                  /* actuators */
    int32_t nshards;             /* partial inputs, 1..RTC_MAX_WFS */
    const rtc_polc* polc;        /* P (na x na, optional), gain, leak, a0, clip; mode must be
                                    RTC_POLC_IMPLICIT and D NULL */
} rtc_master_desc;

/* Create a master: device buffers for nshards partial inputs of na floats
 * (zero), the state a (a0 or 0), P and q = P a0, a page-locked command buffer.
 * RTC_EINVAL for bad sizes or a non-finite P / a0; RTC_ENOMEM, RTC_ECUDA. */
int rtc_master_create(const rtc_master_desc* desc, rtc_master** out);
/* Device address of input `shard` (na floats on the master's device), for
 * rtc_set_partial_output or the caller's own copies.  Owned by the master. */
int rtc_master_input(rtc_master* master, int32_t shard, float** device_ptr);
/* Copy na floats (host or device memory) into input `shard`, ordered before
 * the next rtc_master_step (for partials that arrive from another process or
 * node).  Pageable host data is copied before the call returns. */
int rtc_master_set_input(rtc_master* master, int32_t shard, const float* src, size_t n);
/* Apply the control law to the inputs, which must hold frame frame_id's partials
 * (the caller has seen each shard's frame complete, e.g. by its
 * rtc_get_commands, or has copied them in with work ordered before this call):
 * commands, then their copy to page-locked host memory, then the POLC product
 * for the next frame, on the master's stream.  frame_id must increase
 * (RTC_EORDER otherwise).  Asynchronous. */
int rtc_master_step(rtc_master* master, uint64_t frame_id);
/* The commands of the last stepped frame (n >= na floats), waiting up to
 * timeout_us (negative: no limit) for them; RTC_ETIMEDOUT, RTC_ENOENT before
 * the first step. */
int rtc_master_get_commands(rtc_master* master, float* out, size_t n, uint64_t* frame_id, int64_t timeout_us);
/* Wait for the master's work, then release it. */
int rtc_master_destroy(rtc_master* master);
/* Text of the master's last failure (or of the last rtc_master_create failure
 * for NULL).  Never NULL. */
const char* rtc_master_last_error(const rtc_master* master);

/* ---- allocation-free reconstruction step ------------------------------ */

/* Floats in the library's fixed scratch array used by rtc_reconstruct_noalloc
 * (8 MiB on every GPU that loads the library, held until the process exits). */
#define RTC_NOALLOC_MAX_FLOATS 2097152

/* The paper has no counterpart to this entry point: it is here for callers
 * that must not allocate device memory once running, such as a hard real-time
 * control thread (cudaMalloc can synchronise the device and has no latency
 * bound) or code hosted in a framework that owns every device allocation.
 * It runs the reconstruction MVM and the leaky-integrator step of the loop on
 * the caller's buffers without allocating anything:
 *   a_out[r] = (1 - leak) a_in[r] + gain (row_scale[r] * sum_j M[r][j] s[j] + q[r])
 * M: device float32, row r at M + r*ld (16-byte aligned, ld >= ns and a
 * multiple of 4); s: device float32[ns] (16-byte aligned); row_scale and q:
 * device float32[na] or NULL (1 and 0); a_in, a_out: device float32[na], may
 * be the same buffer.  The partial sums of the column splits go to a static
 * device array of RTC_NOALLOC_MAX_FLOATS floats; na larger than that returns
 * RTC_EINVAL, as do NULL or misaligned pointers.  It runs in the context
 * current on the calling thread: the current device's primary context (the
 * CUDA runtime's default), or a driver-API context the caller created and made
 * current.  Each context has its own copy of the array, so the first call in
 * each context (and again after cudaDeviceReset, which ends the old one) looks
 * up the array's device address there; make that first call before any stream
 * capture.  Every call shares the array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it and must be serialised by the
 * caller.  Nothing in the array needs clearing: every call overwrites the part
 * it reads.  stream: a cudaStream_t or NULL; asynchronous.  Returns RTC_ECUDA,
 * without launching and without clearing it, when a CUDA error from the
 * caller's earlier work is still pending, and RTC_ECUDA if a launch fails. */
int rtc_reconstruct_noalloc(int32_t na, int32_t ns, const float* M, size_t ld,
                            const float* row_scale, const float* s, const float* q,
                            const float* a_in, float* a_out, float gain, float leak,
                            void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RTC_H */
