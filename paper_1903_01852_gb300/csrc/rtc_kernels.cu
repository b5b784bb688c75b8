// CUDA kernels of the AO real-time-control hot path (sm_103a).
//
//   slopes_kernel    calibration fused with SH centre of gravity / pyramid quad
//                    difference, one CTA per part of a slope row (Section 2.2,
//                    Fig. wfs_slopes)
//   gemv_kernel      reconstruction MVM, one partial per column block, warp per
//                    matrix row, 128-bit streaming loads (Section 2.3: the MVM
//                    is memory-bandwidth bound), with the finalisation (partial
//                    sums + POLC term + leaky integrator, Section 3 and 3.4)
//                    fused into its tail; also the POLC product P a (or D a in
//                    explicit-POLC mode)
//   normalise_kernel global normalisation of pyramid slopes by the mean flux
//   telemetry_kernel one entry of the telemetry circular buffer (Section 3.3)
//   pack / relayout / quantize / check kernels used at creation and for telemetry
#include <algorithm>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "rtc_internal.h"

namespace rtc {

size_t dtype_size(int dtype) { return dtype == RTC_F32 ? 4 : dtype == RTC_BF16 ? 2 : 1; }
int elems_per_16B(int dtype) { return int(16 / dtype_size(dtype)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch: a kernel lets the next one in its stream start
// early (launch_dependents); the next one waits (wait) before it reads anything
// the previous one writes.  Both are no-ops without the launch attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// GPU global timer in nanoseconds.
__device__ __forceinline__ unsigned long long global_time_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Release/acquire fences (lighter than the sequentially consistent __threadfence).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void fence_acq_rel_sys() { asm volatile("fence.acq_rel.sys;" ::: "memory"); }

// Prefetch of one line into L1 (no register is held for it).
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p) : "memory");
}

// Bulk prefetch of a contiguous, 16-byte aligned region into L2 (TMA engine).
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Calibration: c = (raw - dark) * flat in float32 (both operations rounded to
// nearest, never contracted), then the threshold.  A pixel is lit iff c > T.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float calibrate(unsigned raw, float dark, float flat, float T, int mode) {
    const float c = __fmul_rn(__fsub_rn(static_cast<float>(raw), dark), flat);
    if (!(c > T)) return 0.0f;
    return mode == RTC_THRESH_SUBTRACT ? __fsub_rn(c, T) : c;
}

// A slope pair as stored: (measured - reference) + pseudo-open-loop term, with
// the reference (r) and pseudo-open-loop (p) pairs already loaded.
__device__ __forceinline__ void store_pair_v(float* __restrict__ s_pad, int pad, bool has_ref, float2 r, bool has_pol,
                                             float2 p, float sx, float sy) {
    if (has_ref) { sx -= r.x; sy -= r.y; }
    if (has_pol) { sx += p.x; sy += p.y; }
    s_pad[pad] = sx;
    s_pad[pad + 1] = sy;
}

// The reference or pseudo-open-loop pair of compact slope index comp (zero when absent).
__device__ __forceinline__ float2 load_pair(const float* __restrict__ v, int comp) {
    return v ? make_float2(v[comp], v[comp + 1]) : make_float2(0.f, 0.f);
}

__device__ __forceinline__ void store_pair(float* __restrict__ s_pad, int pad, const float* __restrict__ ref,
                                           const float* __restrict__ pol, int comp, float sx, float sy) {
    store_pair_v(s_pad, pad, ref != nullptr, load_pair(ref, comp), pol != nullptr, load_pair(pol, comp), sx, sy);
}

// SH slope-row part: pixel rows [pr0, pr1) of one subaperture row.  The CTA
// first reduces each pixel column of the strip over its rows (column flux F_c
// and first moment in y), in G row groups so that narrow strips still use the
// whole CTA, four rows of loads in flight per thread; then each valid
// subaperture adds its npx columns (one thread per subaperture when that sum is
// short, one warp otherwise).  A row split in several parts (large
// subapertures) publishes per-part sums; the last part to finish adds them in
// part order and writes the slopes.  Every sum has a fixed order.  The table
// entries of each thread's (or warp's) first subaperture are loaded before the
// column sums, so they are not a dependent load at the end.
// kAllRows (row chunks read in place over the CPU-GPU link, whose latency is
// several times that of HBM): a thread first issues the loads of all its pixel
// rows (up to kRowsInFlight) and of their dark and flat maps, then calibrates
// them; the additions keep the same order, so the slopes are bit-identical to the
// other variant.  It takes ~220 registers (one CTA per SM): right for a chunk's
// few dozen CTAs, not for a whole frame's hundreds.  (Calibration loads in three
// dependent batches of four rows instead: paced latency 1-2 us longer.)
constexpr int kRowsInFlight = 12;

template <bool kAllRows>
__device__ void sh_part(const SlopePart& P, const SlopeRow& row, const WfsDev& W, const uint16_t* __restrict__ px,
                        long long pitch, int prow0, const uint16_t* __restrict__ xlist, const float* __restrict__ ref,
                        const float* __restrict__ pol, float* __restrict__ s_pad, float* __restrict__ pscr,
                        unsigned* __restrict__ counters, float* sm) {
    __shared__ int s_last;
    const int n = W.npx;
    const int ws = W.nsubx * n;                 // strip width in pixels
    const int x0 = W.ox;
    const int y0 = W.oy + row.row * n;
    const int q0 = x0 >> 2;                     // quads of 4 pixels aligned to absolute columns
    const int nq = ((x0 + ws + 3) >> 2) - q0;
    const int nr = P.pr1 - P.pr0;
    const int G = max(1, min(nr, (int)blockDim.x / nq));
    float* colF = sm;                           // [G][ws]
    float* colY = sm + G * ws;                  // [G][ws]
    const float half = 0.5f * float(n - 1);
    const float T = W.threshold;
    const int mode = W.thresh_mode;
    const bool single = row.nparts == 1;
    const bool by_thread = n * G <= 64;
    const int u_first = by_thread ? (int)threadIdx.x : (int)(threadIdx.x >> 5);
    int x_first = 0;
    float2 r_first = make_float2(0.f, 0.f), p_first = make_float2(0.f, 0.f);
    if (u_first < row.nunits) {
        x_first = xlist[row.unit0 + u_first];
        if (single) {
            r_first = load_pair(ref, row.s_compact + 2 * u_first);
            p_first = load_pair(pol, row.s_compact + 2 * u_first);
        }
    }

    for (int idx = threadIdx.x; idx < nq * G; idx += blockDim.x) {
        const int q = idx % nq;
        const int g = idx / nq;
        const int xa = (q0 + q) << 2;
        float F[4] = {0.f, 0.f, 0.f, 0.f};
        float Y[4] = {0.f, 0.f, 0.f, 0.f};
        int r = P.pr0 + g;
        if constexpr (kAllRows) {
            // every row's pixel and calibration loads issued before the first is used
            uint2 rw[kRowsInFlight];
            float4 d[kRowsInFlight], f[kRowsInFlight];
#pragma unroll
            for (int j = 0; j < kRowsInFlight; ++j) {
                const int rr = r + j * G;
                if (rr < P.pr1) {
                    const long long yy = y0 + rr;
                    rw[j] = __ldg(reinterpret_cast<const uint2*>(px + (yy - prow0) * pitch + xa));
                    d[j] = __ldg(reinterpret_cast<const float4*>(W.dark + yy * W.calib_pitch + xa));
                    f[j] = __ldg(reinterpret_cast<const float4*>(W.flat + yy * W.calib_pitch + xa));
                }
            }
#pragma unroll
            for (int j = 0; j < kRowsInFlight; ++j) {
                const int rr = r + j * G;
                if (rr < P.pr1) {
                    const uint2 q2 = rw[j];
                    const float yc = float(rr) - half;
                    const float t0 = calibrate(q2.x & 0xffffu, d[j].x, f[j].x, T, mode);
                    const float t1 = calibrate(q2.x >> 16, d[j].y, f[j].y, T, mode);
                    const float t2 = calibrate(q2.y & 0xffffu, d[j].z, f[j].z, T, mode);
                    const float t3 = calibrate(q2.y >> 16, d[j].w, f[j].w, T, mode);
                    F[0] += t0; F[1] += t1; F[2] += t2; F[3] += t3;
                    Y[0] = fmaf(t0, yc, Y[0]); Y[1] = fmaf(t1, yc, Y[1]);
                    Y[2] = fmaf(t2, yc, Y[2]); Y[3] = fmaf(t3, yc, Y[3]);
                }
            }
            r += kRowsInFlight * G;    // rows beyond (never with the default part split) go below
        }
        for (; r + 3 * G < P.pr1; r += 4 * G) {
            uint2 rw[4];
            float4 d[4], f[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long yy = y0 + r + k * G;
                rw[k] = __ldg(reinterpret_cast<const uint2*>(px + (yy - prow0) * pitch + xa));
                d[k] = __ldg(reinterpret_cast<const float4*>(W.dark + yy * W.calib_pitch + xa));
                f[k] = __ldg(reinterpret_cast<const float4*>(W.flat + yy * W.calib_pitch + xa));
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float yc = float(r + k * G) - half;
                const float t0 = calibrate(rw[k].x & 0xffffu, d[k].x, f[k].x, T, mode);
                const float t1 = calibrate(rw[k].x >> 16, d[k].y, f[k].y, T, mode);
                const float t2 = calibrate(rw[k].y & 0xffffu, d[k].z, f[k].z, T, mode);
                const float t3 = calibrate(rw[k].y >> 16, d[k].w, f[k].w, T, mode);
                F[0] += t0; F[1] += t1; F[2] += t2; F[3] += t3;
                Y[0] = fmaf(t0, yc, Y[0]); Y[1] = fmaf(t1, yc, Y[1]);
                Y[2] = fmaf(t2, yc, Y[2]); Y[3] = fmaf(t3, yc, Y[3]);
            }
        }
        for (; r < P.pr1; r += G) {
            const long long yy = y0 + r;
            const uint2 rw = __ldg(reinterpret_cast<const uint2*>(px + (yy - prow0) * pitch + xa));
            const float4 d = __ldg(reinterpret_cast<const float4*>(W.dark + yy * W.calib_pitch + xa));
            const float4 f = __ldg(reinterpret_cast<const float4*>(W.flat + yy * W.calib_pitch + xa));
            const float yc = float(r) - half;
            const float t0 = calibrate(rw.x & 0xffffu, d.x, f.x, T, mode);
            const float t1 = calibrate(rw.x >> 16, d.y, f.y, T, mode);
            const float t2 = calibrate(rw.y & 0xffffu, d.z, f.z, T, mode);
            const float t3 = calibrate(rw.y >> 16, d.w, f.w, T, mode);
            F[0] += t0; F[1] += t1; F[2] += t2; F[3] += t3;
            Y[0] = fmaf(t0, yc, Y[0]); Y[1] = fmaf(t1, yc, Y[1]);
            Y[2] = fmaf(t2, yc, Y[2]); Y[3] = fmaf(t3, yc, Y[3]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = xa + k - x0;
            if (c >= 0 && c < ws) { colF[g * ws + c] = F[k]; colY[g * ws + c] = Y[k]; }
        }
    }
    __syncthreads();

    auto emit = [&](int u, float Fs, float Xs, float Ys) {
        if (single) {
            float sx = 0.f, sy = 0.f;
            if (Fs > 0.f) { sx = Xs / Fs; sy = Ys / Fs; }
            if (u == u_first)
                store_pair_v(s_pad, row.s_pad + 2 * u, ref != nullptr, r_first, pol != nullptr, p_first, sx, sy);
            else
                store_pair(s_pad, row.s_pad + 2 * u, ref, pol, row.s_compact + 2 * u, sx, sy);
        } else {
            float* o = pscr + row.pscr + 3 * ((size_t)P.part * row.nunits + u);
            o[0] = Fs; o[1] = Xs; o[2] = Ys;
        }
    };
    if (by_thread) {
        for (int u = threadIdx.x; u < row.nunits; u += blockDim.x) {
            const int cx = (u == u_first ? x_first : xlist[row.unit0 + u]) * n;
            float Fs = 0.f, Xs = 0.f, Ys = 0.f;
            for (int k = 0; k < n; ++k) {
                float fc = 0.f, yc = 0.f;
                for (int g = 0; g < G; ++g) { fc += colF[g * ws + cx + k]; yc += colY[g * ws + cx + k]; }
                Fs += fc;
                Xs = fmaf(float(k) - half, fc, Xs);
                Ys += yc;
            }
            emit(u, Fs, Xs, Ys);
        }
    } else {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int u = warp; u < row.nunits; u += nw) {
            const int cx = (u == u_first ? x_first : xlist[row.unit0 + u]) * n;
            float Fs = 0.f, Xs = 0.f, Ys = 0.f;
            for (int p = lane; p < n * G; p += 32) {
                const int k = p % n, g = p / n;
                const float fc = colF[g * ws + cx + k];
                Fs += fc;
                Xs = fmaf(float(k) - half, fc, Xs);
                Ys += colY[g * ws + cx + k];
            }
            Fs = warp_sum(Fs);
            Xs = warp_sum(Xs);
            Ys = warp_sum(Ys);
            if (lane == 0) emit(u, Fs, Xs, Ys);
        }
    }
    if (single) return;
    // last part of the row to finish adds the parts in order (release and
    // acquire by thread 0, ordered with the other threads by the barriers)
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_acq_rel_gpu();
        const bool last = atomicAdd(&counters[P.row], 1u) == (unsigned)(row.nparts - 1);
        if (last) fence_acq_rel_gpu();
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return;
    for (int u = threadIdx.x; u < row.nunits; u += blockDim.x) {
        float Fs = 0.f, Xs = 0.f, Ys = 0.f;
        for (int k = 0; k < row.nparts; ++k) {
            const float* o = pscr + row.pscr + 3 * ((size_t)k * row.nunits + u);
            Fs += __ldcg(o);
            Xs += __ldcg(o + 1);
            Ys += __ldcg(o + 2);
        }
        float sx = 0.f, sy = 0.f;
        if (Fs > 0.f) { sx = Xs / Fs; sy = Ys / Fs; }
        store_pair(s_pad, row.s_pad + 2 * u, ref, pol, row.s_compact + 2 * u, sx, sy);
    }
    if (threadIdx.x == 0) counters[P.row] = 0u;
}

// Pyramid slope row: one thread per valid pupil pixel reads the matching pixel
// of the four pupil images A (top-left), B (top-right), C (bottom-left),
// D (bottom-right); sx = (A+C-B-D)/N, sy = (A+B-C-D)/N with N = A+B+C+D.
// With global normalisation the row stores the differences themselves and its
// flux sum (per-thread sums in unit order, then a fixed reduction over the CTA);
// normalise_kernel divides them by the mean flux once every row is done.
__device__ void pyr_row(const SlopeRow& row, const WfsDev& W, const uint16_t* __restrict__ px, long long pitch,
                        int prow0, const uint16_t* __restrict__ xlist, const float* __restrict__ ref,
                        const float* __restrict__ pol, float* __restrict__ s_pad, float* __restrict__ pscr) {
    const int i = row.row;
    const bool global = W.norm == RTC_NORM_GLOBAL;
    float flux = 0.f;
    for (int u = threadIdx.x; u < row.nunits; u += blockDim.x) {
        const int j = xlist[row.unit0 + u];
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int yy = W.qy[k] + i, xx = W.qx[k] + j;
            const size_t m = (size_t)yy * W.calib_pitch + xx;
            v[k] = calibrate(px[(long long)(yy - prow0) * pitch + xx], __ldg(W.dark + m), __ldg(W.flat + m), W.threshold,
                             W.thresh_mode);
        }
        const float N = (v[0] + v[1]) + (v[2] + v[3]);
        const float dx = (v[0] + v[2]) - (v[1] + v[3]);
        const float dy = (v[0] + v[1]) - (v[2] + v[3]);
        if (global) {
            flux += N;
            s_pad[row.s_pad + 2 * u] = dx;
            s_pad[row.s_pad + 2 * u + 1] = dy;
            continue;
        }
        float sx = 0.f, sy = 0.f;
        if (N > 0.f) { sx = dx / N; sy = dy / N; }
        store_pair(s_pad, row.s_pad + 2 * u, ref, pol, row.s_compact + 2 * u, sx, sy);
    }
    if (!global) return;
    __shared__ float s_red[kSlopeThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    flux = warp_sum(flux);
    if (lane == 0) s_red[warp] = flux;
    __syncthreads();
    if (threadIdx.x == 0) {
        float f = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) f += s_red[w];
        pscr[W.gflux + i] = f;
    }
}

// The WFS table travels in the parameters (constant bank), so a CTA's only
// global load before its pixels is its own 48-byte table entry.
struct SlopeArgs {
    const SlopeCta* ctas;
    int cta0;
    const uint16_t* xlist;
    const float* ref;
    const float* pol;
    float* s_pad;
    float* pscr;
    unsigned* counters;
    ChunkGate gate;           // desc NULL: every pixel pointer is in fp
    FramePtrs fp;
    WfsDev wfs[kMaxWfs];
};
static_assert(sizeof(SlopeCta) == 48, "slope CTA entry is three 16-byte vectors");
static_assert(sizeof(SlopeArgs) <= 4096, "slope kernel parameters");

// The wait of a pre-enqueued chunk (one thread): polls the mailbox state
// (system-scope acquire) with short sleeps until the host has moved it, at most
// limit_ns by the global timer and max_polls polls; then claims it as expired
// with a compare-and-swap, which fails if the host moved it in the meantime.
// Returns the state that both sides act on.
__device__ int chunk_gate_wait(const ChunkGate& g) {
    int* st = &g.desc->state;
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (unsigned poll = 0;; ++poll) {
        int v;
        asm volatile("ld.acquire.sys.global.b32 %0, [%1];" : "=r"(v) : "l"(st) : "memory");
        if (v != kChunkEmpty) return v;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (poll >= g.max_polls || t - t0 >= g.limit_ns) break;
        __nanosleep(32);      // a read over the link takes about a microsecond anyway
    }
    int old;
    asm volatile("atom.acq_rel.sys.global.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "l"(st), "r"(int(kChunkEmpty)), "r"(int(kChunkExpired)) : "memory");
    return old == kChunkEmpty ? int(kChunkExpired) : old;
}

// One warp that holds a pre-enqueued chunk's place on its stream until the
// mailbox is settled; the chunk's slope kernel, its programmatic dependent,
// launches when it exits.  Waiting thus occupies one warp per camera, not the
// slope kernel's CTAs (which would keep the other cameras' MVMs off the SMs).
__global__ void __launch_bounds__(32) chunk_gate_kernel(const ChunkGate g) {
    if (threadIdx.x != 0) return;
    const int state = chunk_gate_wait(g);
    if (state == kChunkFilled) {     // fields written before the host's swap
        const volatile ChunkDesc* d = g.desc;
        g.mirror->px = d->px;
        g.mirror->pitch = d->pitch;
        g.mirror->row0 = d->row0;
    }
    g.mirror->state = state;
}

template <bool kAllRows, bool kGated>
__global__ void __launch_bounds__(kSlopeThreads) slopes_kernel(const __grid_constant__ SlopeArgs a) {
    extern __shared__ float sm[];
    __shared__ ChunkDesc s_box;
    if constexpr (kGated) {
        pdl_wait();       // the gate kernel has ended: its mirror of the mailbox is written
        if (threadIdx.x == 0) {
            const ChunkDesc* d = a.gate.mirror;
            s_box.state = __ldcg(&d->state);
            if (s_box.state == kChunkFilled) {
                s_box.px = reinterpret_cast<const uint16_t*>(__ldcg(reinterpret_cast<const long long*>(&d->px)));
                s_box.pitch = __ldcg(&d->pitch);
                s_box.row0 = __ldcg(&d->row0);
            }
        }
        __syncthreads();
    }
    pdl_trigger();        // the MVM may launch now and prefetch its matrix tiles while slopes run
    if constexpr (kGated)
        if (s_box.state != kChunkFilled) return;
    union {
        int4 v[3];
        SlopeCta c;
    } e;
    const int4* src = reinterpret_cast<const int4*>(a.ctas + a.cta0 + blockIdx.x);
#pragma unroll
    for (int k = 0; k < 3; ++k) e.v[k] = __ldg(src + k);
    const SlopeRow& row = e.c.row;
    const int w = row.wfs;
    const WfsDev& W = a.wfs[w];
    const uint16_t* px = a.fp.px[w];
    long long pitch = a.fp.pitch[w];
    int prow0 = a.fp.row0[w];
    if constexpr (kGated) {
        if (w == a.gate.wfs) {
            px = s_box.px;
            pitch = s_box.pitch;
            prow0 = s_box.row0;
        }
    }
    if (W.kind == RTC_WFS_SH)
        sh_part<kAllRows>(e.c.part, row, W, px, pitch, prow0, a.xlist, a.ref, a.pol, a.s_pad, a.pscr,
                                  a.counters, sm);
    else
        pyr_row(row, W, px, pitch, prow0, a.xlist, a.ref, a.pol, a.s_pad, a.pscr);
}

// Global normalisation of pyramid slopes, a programmatic dependent of the slope
// kernel: grid.y enumerates column blocks of globally normalised WFS (items:
// block, WFS), grid.x their slope pairs.  Every CTA adds the WFS's row fluxes
// in the same fixed order (so all agree on the mean bit for bit), then divides
// its pairs by the mean flux over the valid pupil pixels.
struct NormArgs {
    const int2* items;
    int item0;
    const BlockDev* blocks;
    const WfsDev* wfs;
    const float* pscr;
    const float* ref;
    const float* pol;
    float* s_pad;
};

__global__ void __launch_bounds__(256) normalise_kernel(const __grid_constant__ NormArgs a) {
    __shared__ float s_mean;
    pdl_trigger();        // the MVM may launch and prefetch now
    pdl_wait();           // differences and row fluxes are written by the slope kernel
    const int2 it = a.items[a.item0 + blockIdx.y];
    const WfsDev& W = a.wfs[it.y];
    if (threadIdx.x < 32) {
        float f = 0.f;
        for (int r = threadIdx.x; r < W.gnrows; r += 32) f += a.pscr[W.gflux + r];
        f = warp_sum(f);
        if (threadIdx.x == 0) s_mean = f / float(W.gpix);
    }
    __syncthreads();
    const BlockDev B = a.blocks[it.x];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (B.ncols >> 1)) return;
    const float mean = s_mean;
    const float2 d = reinterpret_cast<const float2*>(a.s_pad + B.x_off)[q];
    float sx = 0.f, sy = 0.f;
    if (mean > 0.f) { sx = d.x / mean; sy = d.y / mean; }
    store_pair(a.s_pad, B.x_off + 2 * q, a.ref, a.pol, B.c0 + 2 * q, sx, sy);
}

cudaError_t launch_normalise(const int2* items, int item0, int nitems, int max_pairs, const BlockDev* blocks,
                             const WfsDev* wfs, const float* pscr, const float* ref, const float* pol, float* s_pad,
                             bool pdl, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    NormArgs a{items, item0, blocks, wfs, pscr, ref, pol, s_pad};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)std::max(1, (max_pairs + 255) / 256), (unsigned)nitems);
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, normalise_kernel, a);
}

cudaError_t configure_slopes(int smem_bytes) {
    if (smem_bytes <= 48 * 1024) return cudaSuccess;
    for (auto k : {slopes_kernel<false, false>, slopes_kernel<true, false>, slopes_kernel<false, true>,
                   slopes_kernel<true, true>}) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_slopes(const SlopeCta* ctas, int cta0, int nctas, const WfsDev* wfs, int nwfs,
                          const FramePtrs& fp, bool host_px, const uint16_t* xlist, const float* ref,
                          const float* pol, float* s_pad, float* pscr, unsigned* counters, int smem_bytes,
                          cudaStream_t st, const ChunkGate* gate) {
    if (nctas <= 0) return cudaSuccess;
    if (nwfs < 1 || nwfs > kMaxWfs) return cudaErrorInvalidValue;
    SlopeArgs a{};
    a.ctas = ctas;
    a.cta0 = cta0;
    a.xlist = xlist;
    a.ref = ref;
    a.pol = pol;
    a.s_pad = s_pad;
    a.pscr = pscr;
    a.counters = counters;
    a.fp = fp;
    std::copy(wfs, wfs + nwfs, a.wfs);
    const dim3 grid(nctas), block(kSlopeThreads);
    if (gate) {
        a.gate = *gate;
        const cudaError_t e = launch_kernel(chunk_gate_kernel, dim3(1), dim3(32), 0, st, *gate);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem_bytes;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;     // launched at the gate kernel's exit, a few us before a stream-ordered launch
        if (host_px) return cudaLaunchKernelEx(&cfg, slopes_kernel<true, true>, a);
        return cudaLaunchKernelEx(&cfg, slopes_kernel<false, true>, a);
    }
    if (host_px) return launch_kernel(slopes_kernel<true, false>, grid, block, smem_bytes, st, a);
    return launch_kernel(slopes_kernel<false, false>, grid, block, smem_bytes, st, a);
}

// ---------------------------------------------------------------------------
// GEMV: one warp per matrix row of a column block.  Each lane streams 16-byte
// vectors v = lane, lane+32, ... of the row (U of them in flight), multiplies
// by the matching input elements (read-only cache) and accumulates in float32;
// a fixed xor-butterfly reduces the 32 lane sums.  The order of every sum is
// fixed, so a block's partial does not depend on how the launch was split.
// ---------------------------------------------------------------------------
template <int DT> struct Elem;
template <> struct Elem<RTC_F32> { static constexpr int kPer16 = 4; };
template <> struct Elem<RTC_BF16> { static constexpr int kPer16 = 8; };
template <> struct Elem<RTC_E4M3> { static constexpr int kPer16 = 16; };

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

// Vectors per lane of the single-block BF16 / E4M3 products without finalisation
// (0: the MVM kernel).  E4M3 POLC, MCAO 26.6 -> 18.4 us, LTAO 20.4 -> 14.3 us (the
// same with 4); BF16 unchanged at 2 or 4 (24.5 us: 235 CTAs over 152 SMs), so off.
#ifndef RTC_GEMV_BF16_U_DEEP
#define RTC_GEMV_BF16_U_DEEP 0
#endif
#ifndef RTC_GEMV_E4M3_U_DEEP
#define RTC_GEMV_E4M3_U_DEEP 2
#endif
#ifndef RTC_GEMV_GROUP_MIN_WAVES
#define RTC_GEMV_GROUP_MIN_WAVES 2 // waves of 8 CTAs per SM a grouped launch keeps at least
#endif
// Consecutive column blocks one MVM CTA takes (its row tile of each, one fused
// finalisation for all), per storage format.  BF16 and E4M3 rows of a block are
// short (about 2.2 and 1.1 KB on MCAO), so a one-block CTA spends much of its
// life on its fixed costs; two blocks per CTA: MCAO BF16 MVM 138.9 -> 132.7 us,
// E4M3 108.1 -> 99.9 us, LTAO BF16 85.6 -> 75.4 us.  Float32 rows are long
// enough (one block: 243.2 us, two: 245.3 us).
#ifndef RTC_GEMV_GROUP_F32
#define RTC_GEMV_GROUP_F32 1
#endif
#ifndef RTC_GEMV_GROUP_BF16
#define RTC_GEMV_GROUP_BF16 2
#endif
#ifndef RTC_GEMV_GROUP_E4M3
#define RTC_GEMV_GROUP_E4M3 2
#endif

#ifndef RTC_GEMV_FFMA2_MASK
#define RTC_GEMV_FFMA2_MASK 1      // storage formats (bit 1 << dtype) that sum with packed FMAs: float32
#endif
// A lane's running sum: one float32 FMA per element in element order (float), or
// two float32 partial sums over the even and odd elements advanced with the packed
// fma.rn.f32x2 (half the FMA instructions).
using acc_pk = unsigned long long;
__device__ __forceinline__ void acc_zero(float& c) { c = 0.f; }
__device__ __forceinline__ void acc_zero(acc_pk& c) { c = 0ull; }
__device__ __forceinline__ float fma2(float a0, float a1, float b0, float b1, float c) {
    return fmaf(a1, b1, fmaf(a0, b0, c));
}
__device__ __forceinline__ acc_pk fma2(float a0, float a1, float b0, float b1, acc_pk c) {
    acc_pk a, b, d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(b0), "f"(b1));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float acc_total(float c) { return c; }
__device__ __forceinline__ float acc_total(acc_pk c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(c));
    return lo + hi;
}
template <int DT> struct AccOf {
    using type = typename std::conditional<((RTC_GEMV_FFMA2_MASK >> DT) & 1) != 0, acc_pk, float>::type;
};

template <typename A>
__device__ __forceinline__ A dot_f32(const uint4& m, const float4* x, A acc) {
    const float4 xv = __ldg(x);
    acc = fma2(__uint_as_float(m.x), __uint_as_float(m.y), xv.x, xv.y, acc);
    acc = fma2(__uint_as_float(m.z), __uint_as_float(m.w), xv.z, xv.w, acc);
    return acc;
}

template <typename A>
__device__ __forceinline__ A dot_bf16(const uint4& m, const float4* x, A acc) {
    const float4 a = __ldg(x), b = __ldg(x + 1);
    acc = fma2(bf_lo(m.x), bf_hi(m.x), a.x, a.y, acc);
    acc = fma2(bf_lo(m.y), bf_hi(m.y), a.z, a.w, acc);
    acc = fma2(bf_lo(m.z), bf_hi(m.z), b.x, b.y, acc);
    acc = fma2(bf_lo(m.w), bf_hi(m.w), b.z, b.w, acc);
    return acc;
}

__device__ __forceinline__ float2 e4m3x2(uint32_t pair16) {
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(pair16), __NV_E4M3);
    return __half22float2(*reinterpret_cast<const __half2*>(&h));
}

template <typename A>
__device__ __forceinline__ A dot_e4m3(const uint4& m, const float4* x, A acc) {
    const uint32_t w[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 xv = __ldg(x + k);
        const float2 lo = e4m3x2(w[k] & 0xffffu);
        const float2 hi = e4m3x2(w[k] >> 16);
        acc = fma2(lo.x, lo.y, xv.x, xv.y, acc);
        acc = fma2(hi.x, hi.y, xv.z, xv.w, acc);
    }
    return acc;
}

template <int DT, typename A>
__device__ __forceinline__ A dot16(const uint4& m, const float* x, int v, A acc) {
    const float4* xp = reinterpret_cast<const float4*>(x) + v * (Elem<DT>::kPer16 / 4);
    if constexpr (DT == RTC_F32) return dot_f32(m, xp, acc);
    else if constexpr (DT == RTC_BF16) return dot_bf16(m, xp, acc);
    else return dot_e4m3(m, xp, acc);
}

struct GemvArgs {
    const uint8_t* M;
    const BlockDev* blocks;
    int b0;
    int nb;                    // column blocks of the launch: b0 .. b0 + nb - 1
    int tiles;                 // row tiles per block
    int na;
    const float* x;
    const float* out_scale;
    float* out;
    long long out_stride;
    FinaliseArgs fin;
    int prefetch_ctas;         // CTAs [0, prefetch_ctas) prefetch their matrix tile into L2 before waiting
    const int* gate_state;     // a pre-enqueued chunk's mailbox state: unless kChunkFilled, do nothing
    int group;                 // column blocks per CTA (consecutive, same row tile), >= 1
};

#ifndef RTC_GEMV_F32_U
#define RTC_GEMV_F32_U 4
#endif
#ifndef RTC_GEMV_F32_RI
#define RTC_GEMV_F32_RI 1
#endif
#ifndef RTC_GEMV_BF16_U
#define RTC_GEMV_BF16_U 2
#endif
#ifndef RTC_GEMV_BF16_RI
#define RTC_GEMV_BF16_RI 4
#endif
#ifndef RTC_GEMV_E4M3_U
#define RTC_GEMV_E4M3_U 1
#endif
#ifndef RTC_GEMV_E4M3_RI
#define RTC_GEMV_E4M3_RI 4
#endif

// The master's finalisation of one tile of kFinRows rows (Section 3: sum the
// partial commands; Section 3.4: add the implicit-POLC term; leaky integrator).
// Eight thread groups each add a contiguous range of blocks in block order,
// then the eight group sums are added in group order.  The row's scale, POLC
// term and state are prefetched into L1 while the partials load.
__device__ void finalise_tile(const FinaliseArgs& f, const float* __restrict__ partial, int na, int ft) {
    __shared__ float red[kGemvWarps][32];
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int r = ft * kFinRows + lane;
    const int b0 = (seg * f.nblk) / kGemvWarps, b1 = ((seg + 1) * f.nblk) / kGemvWarps;
    if (seg == 0 && r < na) {
        if (f.scale) prefetch_l1(f.scale + r);
        prefetch_l1(f.q + r);
        prefetch_l1(f.a + r);
    }
    float y = 0.f;
    if (r < na) {
        // loads issued eight at a time, added in block order
        int b = b0;
        for (; b + 8 <= b1; b += 8) {
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldcg(partial + (size_t)(b + k) * na + r);
#pragma unroll
            for (int k = 0; k < 8; ++k) y += v[k];
        }
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = b + k < b1 ? __ldcg(partial + (size_t)(b + k) * na + r) : 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (b + k < b1) y += v[k];
    }
    red[seg][lane] = y;
    __syncthreads();
    if (seg == 0 && r < na) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kGemvWarps; ++k) t += red[k][lane];
        if (f.scale) t *= f.scale[r];
        if (f.partial) {               // a shard: its partial reconstruction, for a master to add
            f.cmd[r] = t;
            float* const po = *f.pout;
            if (po) po[r] = t;
            return;
        }
        const float w = t + f.q[r];
        float v = fmaf(f.gain, w, f.oml * f.a[r]);
        if (f.clip) v = fminf(fmaxf(v, f.amin), f.amax);
        f.a[r] = v;
        f.cmd[r] = v;
    }
}

// kGated: a pre-enqueued chunk's MVM (the check of its mailbox costs the float32
// variant two registers, so the other launches keep the kernels without it).
// kGroup: consecutive column blocks per CTA (1: one block, the loop compiles away).
template <int DT, int U, int RI, int RPW, bool kGated, int kGroup>
__device__ __forceinline__ void gemv_body(const GemvArgs& a) {
    static_assert(RPW % RI == 0 && kFinRows % (kGemvWarps * RPW) == 0, "row tiling");
    __shared__ int s_last;
    const int bg = blockIdx.x / a.tiles;
    const int tile = blockIdx.x - bg * a.tiles;
    const int g0 = bg * kGroup;                          // the CTA's blocks: [g0, g1) of the launch
    const int g1 = kGroup == 1 ? g0 + 1 : min(g0 + kGroup, a.nb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr size_t esz = 16 / Elem<DT>::kPer16;
    const int r0 = tile * kGemvWarps * RPW;
    const int rbase = r0 + warp * RPW;
    BlockDev B = a.blocks[a.b0 + g0];                    // the first block's entry, before the wait
    if (threadIdx.x == 0 && (int)blockIdx.x < a.prefetch_ctas && r0 < a.na) {
        const int rows = min(r0 + kGemvWarps * RPW, a.na) - r0;
        for (int g = g0; g < g1; ++g) {
            const BlockDev Bg = g == g0 ? B : a.blocks[a.b0 + g];
            const unsigned bytes = (unsigned)((size_t)rows * Bg.pitch * esz);
            if (bytes) prefetch_l2(a.M + (size_t)(Bg.m_off + (long long)r0 * Bg.pitch) * esz, bytes);
        }
    }
    pdl_wait();           // the input vector (slopes or commands) is written by the previous kernel
    pdl_trigger();
    if constexpr (kGated)     // written by the gate kernel, ahead of the slope kernel waited for above
        if (__ldcg(a.gate_state) != kChunkFilled) return;
#pragma unroll 1
    for (int g = g0; g < g1; ++g) {
    const int b = a.b0 + g;
    if (g != g0) B = a.blocks[b];
    const int nvec = B.pitch / Elem<DT>::kPer16;
    const float* x = a.x + B.x_off;
#pragma unroll 1
    for (int rr = 0; rr < RPW; rr += RI) {
        const uint4* mrow[RI];
        bool ok[RI];
        typename AccOf<DT>::type acc[RI];
#pragma unroll
        for (int i = 0; i < RI; ++i) {
            const int r = rbase + rr + i;
            ok[i] = r < a.na;
            mrow[i] = reinterpret_cast<const uint4*>(a.M + (size_t)(B.m_off + (long long)(ok[i] ? r : 0) * B.pitch) * esz);
            acc_zero(acc[i]);
        }
#pragma unroll 1
        for (int v0 = lane; v0 < nvec; v0 += 32 * U) {
            uint4 m[RI][U];
#pragma unroll
            for (int i = 0; i < RI; ++i)
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int v = v0 + 32 * u;
                    m[i][u] = (ok[i] && v < nvec) ? ld_stream(mrow[i] + v) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int v = v0 + 32 * u;
                if (v < nvec) {
#pragma unroll
                    for (int i = 0; i < RI; ++i) acc[i] = dot16<DT>(m[i][u], x, v, acc[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RI; ++i) {
            const float t = warp_sum(acc_total(acc[i]));
            const int r = rbase + rr + i;
            if (lane == 0 && ok[i]) a.out[(long long)b * a.out_stride + r] = a.out_scale ? t * a.out_scale[r] : t;
        }
    }
    }
    if (!a.fin.enabled) return;
    // Fused finalisation: the CTA that completes the last block of a row tile
    // (counted in rows, across launches of the same frame) finalises it.
    // Release/acquire through one thread: the barrier orders the CTA's partial
    // stores before thread 0's release fence, and its acquire fence before the
    // other threads' loads (fences are cumulative over the barrier).
    __syncthreads();
    const int ft = r0 / kFinRows;
    if (threadIdx.x == 0) {
        const int rows_here = min(r0 + kGemvWarps * RPW, a.na) - r0;
        const int ft_rows = min(kFinRows, a.na - ft * kFinRows);
        fence_acq_rel_gpu();
        const unsigned prev = atomicAdd(&a.fin.counters[ft], (unsigned)(rows_here * (g1 - g0)));
        const bool last = prev + rows_here * (g1 - g0) == (unsigned)(a.fin.nblk * ft_rows);
        if (last) fence_acq_rel_gpu();
        s_last = last;
    }
    __syncthreads();
    if (!s_last) return;
    finalise_tile(a.fin, a.out, a.na, ft);
    __syncthreads();
    if (threadIdx.x == 0) {
        a.fin.counters[ft] = 0u;
        if (a.fin.done_flag) {
            const int nfin = (a.na + kFinRows - 1) / kFinRows;
            fence_acq_rel_sys();    // this tile's commands reach the host before the tile counts as done
            if (atomicAdd(a.fin.tiles_done, 1u) == (unsigned)(nfin - 1)) {
                *a.fin.tiles_done = 0u;
                if (a.fin.t_done) *a.fin.t_done = global_time_ns();
                fence_acq_rel_sys();
                const unsigned long long seq = *reinterpret_cast<const volatile unsigned long long*>(a.fin.seq);
                *reinterpret_cast<volatile unsigned long long*>(a.fin.done_flag) = seq;
            }
        }
    }
}

template <int DT, int U, int RI, int RPW, bool kGated, int kGroup>
__global__ void __launch_bounds__(kGemvWarps * 32) gemv_kernel(const __grid_constant__ GemvArgs a) {
    gemv_body<DT, U, RI, RPW, kGated, kGroup>(a);
}

// Several column blocks per CTA, held to the resident CTAs per SM of the one-block
// kernel (the loop over blocks costs it registers otherwise).
template <int DT> struct GroupedMinCtas { static constexpr int value = 8; };
template <> struct GroupedMinCtas<RTC_BF16> { static constexpr int value = 4; };
template <> struct GroupedMinCtas<RTC_E4M3> { static constexpr int value = 5; };
template <int DT, int U, int RI, int RPW, bool kGated, int kGroup>
__global__ void __launch_bounds__(kGemvWarps * 32, GroupedMinCtas<DT>::value)
    gemv_kernel_grouped(const __grid_constant__ GemvArgs a) {
    gemv_body<DT, U, RI, RPW, kGated, kGroup>(a);
}

// A narrow format's single-block product without finalisation (the POLC product
// P a, or D a): its few hundred CTAs hold under two per SM whatever their
// registers, so each lane keeps more vectors in flight than the MVM kernels can.
template <int DT, int U, int RI, bool kGated>
__global__ void __launch_bounds__(kGemvWarps * 32, 2) gemv_kernel_deep(const __grid_constant__ GemvArgs a) {
    gemv_body<DT, U, RI, RI, kGated, 1>(a);
}

// One row per warp: the launches over a single column block (the POLC product, a
// row chunk's block) have about a thousand CTAs, and at <= 32 registers all of
// them fit in one wave of eight CTAs per SM.
template <int DT, int U, int RI, bool kGated>
__global__ void __launch_bounds__(kGemvWarps * 32, 8) gemv_kernel_1row(const __grid_constant__ GemvArgs a) {
    gemv_body<DT, U, RI, RI, kGated, 1>(a);
}

// Telemetry entry of one frame: grid.y enumerates the recorded sections (one
// slope block per y, then the commands, then one WFS's partial commands per y),
// grid.x splits each section.  Every CTA reads the frame and entry counters
// when it starts; the last CTA to finish publishes the entry (header, then the
// published count, after a system-scope fence) and advances the counters, so
// the next launch (stream-ordered) sees them.
__global__ void __launch_bounds__(256) telemetry_kernel(const __grid_constant__ TelArgs t) {
    __shared__ int s_last;
    const unsigned long long frame = t.ctr[0];
    const unsigned long long idx = t.ctr[1];
    const bool rec = frame % (unsigned long long)t.decimate == 0ull;
    if (rec) {
        float* e = t.ring + (long long)(idx % (unsigned long long)t.depth) * t.entry_floats + kTelHeaderFloats;
        const int stride = gridDim.x * blockDim.x;
        const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
        int sec = blockIdx.y;
        if (t.streams & RTC_TEL_SLOPES) {
            if (sec < t.nblk) {
                const BlockDev B = t.blocks[sec];
                for (int j = i0; j < B.ncols; j += stride) e[t.off_s + B.c0 + j] = t.s_pad[B.x_off + j];
            }
            sec -= t.nblk;
        }
        if (t.streams & RTC_TEL_COMMANDS) {
            if (sec == 0)
                for (int r = i0; r < t.na; r += stride) e[t.off_a + r] = t.a[r];
            sec -= 1;
        }
        if ((t.streams & RTC_TEL_PARTIALS) && sec >= 0 && sec < t.nwfs) {
            const int b0 = t.blk_start[sec], b1 = t.blk_start[sec + 1];
            for (int r = i0; r < t.na; r += stride) {
                float y = 0.f;
                for (int b = b0; b < b1; ++b) y += t.part[(size_t)b * t.na + r];
                if (t.scale) y *= t.scale[r];
                e[t.off_p + (size_t)sec * t.na + r] = y;
            }
        }
    }
    __threadfence_system();
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomicAdd(&t.ctr[2], 1ull) == (unsigned long long)(gridDim.x * gridDim.y) - 1ull;
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    if (rec) {
        TelHeader* h = reinterpret_cast<TelHeader*>(t.ring + (long long)(idx % (unsigned long long)t.depth) *
                                                                 t.entry_floats);
        h->index = idx;
        h->frame_id = *reinterpret_cast<const volatile unsigned long long*>(t.fid);
        h->t_commands = *t.t_cmd;
        h->t_written = global_time_ns();
        __threadfence_system();
        *reinterpret_cast<volatile unsigned long long*>(t.wcount) = idx + 1ull;
        t.ctr[1] = idx + 1ull;
    }
    t.ctr[0] = frame + 1ull;
    t.ctr[2] = 0ull;
    __threadfence_system();
}

cudaError_t launch_telemetry(const TelArgs& t, cudaStream_t st) {
    int ny = 0;
    if (t.streams & RTC_TEL_SLOPES) ny += t.nblk;
    if (t.streams & RTC_TEL_COMMANDS) ny += 1;
    if (t.streams & RTC_TEL_PARTIALS) ny += t.nwfs;
    const dim3 grid(4, (unsigned)std::max(ny, 1));
    return launch_kernel(telemetry_kernel, grid, dim3(256), 0, st, t);
}

template <typename K>
cudaError_t launch_maybe_pdl(K kernel, dim3 grid, const GemvArgs& a, bool pdl, cudaStream_t st) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kGemvWarps * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// Launches too small for RTC_GEMV_MIN_WAVES waves of 8 CTAs per SM at four rows
// per warp take fewer rows per warp.  Two waves: the ELT SCAO MVM (5316 x 8608,
// 8 blocks) runs one row per warp in 5344 CTAs, and more of them start while the
// slope kernel runs and prefetch their tiles into L2 (frame latency 43.3 against
// 45.1 us with one wave, although the MVM alone is slower: 40.6 against 36.5 us).
#ifndef RTC_GEMV_MIN_WAVES
#define RTC_GEMV_MIN_WAVES 2
#endif

template <int DT, int U, int RI, bool kG>
cudaError_t launch_gemv_t(const GemvArgs& base, int nb, long long avg_row_bytes, bool pdl, cudaStream_t st) {
    // rows per warp: as many as keep at least RTC_GEMV_MIN_WAVES waves of 8 CTAs per SM
    const int na = base.na;
    int rpw = 4;
    while (rpw > RI &&
           (long long)((na + kGemvWarps * rpw - 1) / (kGemvWarps * rpw)) * nb < RTC_GEMV_MIN_WAVES * 8LL * 152)
        rpw /= 2;
    // with packed sums two rows per warp take 34 registers (6 CTAs per SM): such
    // launches run one row per warp instead (same sums, at most 32 registers)
    constexpr bool kNoRpw2 = RI == 1 && std::is_same<typename AccOf<DT>::type, acc_pk>::value;
    if (kNoRpw2 && rpw == 2) rpw = 1;
    GemvArgs a = base;
    a.tiles = (na + kGemvWarps * rpw - 1) / (kGemvWarps * rpw);
    constexpr int kUDeep = DT == RTC_BF16 ? RTC_GEMV_BF16_U_DEEP : DT == RTC_E4M3 ? RTC_GEMV_E4M3_U_DEEP : 0;
    if constexpr (kUDeep > 0 && RI == 4) {
        if (!a.fin.enabled && nb == 1 && rpw == RI && a.tiles <= 2 * 152) {
            const long long tile_bytes = std::max(1LL, avg_row_bytes * kGemvWarps * rpw);
            a.prefetch_ctas = pdl ? (int)std::min<long long>(a.tiles, (96LL << 20) / tile_bytes) : 0;
            return launch_maybe_pdl(gemv_kernel_deep<DT, kUDeep, RI, kG>, dim3((unsigned)a.tiles), a, pdl, st);
        }
    }
    // consecutive column blocks per CTA, as many as keep that many waves
    constexpr int kMaxGroup = DT == RTC_F32 ? RTC_GEMV_GROUP_F32 : DT == RTC_BF16 ? RTC_GEMV_GROUP_BF16 : RTC_GEMV_GROUP_E4M3;
    // (one grouped instance, kMaxGroup, used when four rows per warp keep that many waves with it)
    a.group = 1;
    if (kMaxGroup > 1 && rpw >= 4 &&
        (long long)a.tiles * ((nb + kMaxGroup - 1) / kMaxGroup) >= RTC_GEMV_GROUP_MIN_WAVES * 8LL * 152)
        a.group = kMaxGroup;
    const dim3 grid((unsigned)(a.tiles * ((nb + a.group - 1) / a.group)));
    // prefetch while waiting for the producer: about 96 MB, below the L2 size
    const long long tile_bytes = std::max(1LL, avg_row_bytes * kGemvWarps * rpw * a.group);
    a.prefetch_ctas = pdl ? (int)std::min<long long>(grid.x, (96LL << 20) / tile_bytes) : 0;
    if constexpr (kMaxGroup > 1)
        if (rpw >= 4 && a.group == kMaxGroup)
            return launch_maybe_pdl(gemv_kernel_grouped<DT, U, RI, (RI > 4 ? RI : 4), kG, kMaxGroup>, grid, a, pdl, st);
    if (rpw >= 4) return launch_maybe_pdl(gemv_kernel<DT, U, RI, (RI > 4 ? RI : 4), kG, 1>, grid, a, pdl, st);
    if constexpr (!kNoRpw2)
        if (rpw >= 2) return launch_maybe_pdl(gemv_kernel<DT, U, RI, (RI > 2 ? RI : 2), kG, 1>, grid, a, pdl, st);
    if constexpr (RI == 1) return launch_maybe_pdl(gemv_kernel_1row<DT, U, 1, kG>, grid, a, pdl, st);
    else return launch_maybe_pdl(gemv_kernel<DT, U, RI, RI, kG, 1>, grid, a, pdl, st);
}

cudaError_t launch_gemv(int dtype, const void* M, const BlockDev* blocks, int b0, int nb, int na, const float* x,
                        const float* out_scale, float* out, long long out_stride, const FinaliseArgs* fin,
                        long long avg_row_bytes, bool pdl, cudaStream_t st, const int* gate_state) {
    if (nb <= 0 || na <= 0) return cudaSuccess;
    GemvArgs a{static_cast<const uint8_t*>(M), blocks, b0, nb, 0, na, x, out_scale, out, out_stride, FinaliseArgs{}, 0,
               gate_state, 1};
    if (fin) a.fin = *fin;
    if (gate_state) {
        switch (dtype) {
            case RTC_F32: return launch_gemv_t<RTC_F32, RTC_GEMV_F32_U, RTC_GEMV_F32_RI, true>(a, nb, avg_row_bytes, pdl, st);
            case RTC_BF16: return launch_gemv_t<RTC_BF16, RTC_GEMV_BF16_U, RTC_GEMV_BF16_RI, true>(a, nb, avg_row_bytes, pdl, st);
            case RTC_E4M3: return launch_gemv_t<RTC_E4M3, RTC_GEMV_E4M3_U, RTC_GEMV_E4M3_RI, true>(a, nb, avg_row_bytes, pdl, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (dtype) {
        case RTC_F32: return launch_gemv_t<RTC_F32, RTC_GEMV_F32_U, RTC_GEMV_F32_RI, false>(a, nb, avg_row_bytes, pdl, st);
        case RTC_BF16: return launch_gemv_t<RTC_BF16, RTC_GEMV_BF16_U, RTC_GEMV_BF16_RI, false>(a, nb, avg_row_bytes, pdl, st);
        case RTC_E4M3: return launch_gemv_t<RTC_E4M3, RTC_GEMV_E4M3_U, RTC_GEMV_E4M3_RI, false>(a, nb, avg_row_bytes, pdl, st);
        default: return cudaErrorInvalidValue;
    }
}

__global__ void pack_slopes_kernel(const BlockDev* __restrict__ blocks, const float* __restrict__ s_pad,
                                   float* __restrict__ out) {
    const BlockDev B = blocks[blockIdx.y];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < B.ncols; j += gridDim.x * blockDim.x)
        out[B.c0 + j] = s_pad[B.x_off + j];
}

cudaError_t launch_pack_slopes(const BlockDev* blocks, int nblk, int max_cols, const float* s_pad, float* out,
                               cudaStream_t st) {
    const dim3 grid((max_cols + 255) / 256, nblk);
    return launch_kernel(pack_slopes_kernel, grid, dim3(256), 0, st, blocks, s_pad, out);
}

// ---------------------------------------------------------------------------
// Creation-time helpers
// ---------------------------------------------------------------------------
template <typename T>
__global__ void relayout_kernel(const T* __restrict__ src, int na, int ns, const BlockDev* __restrict__ blocks,
                                T* __restrict__ dst) {
    const BlockDev B = blocks[blockIdx.y];
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)na * B.pitch;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = int(e / B.pitch), j = int(e - (long long)r * B.pitch);
        dst[B.m_off + e] = j < B.ncols ? src[(size_t)r * ns + B.c0 + j] : T(0);
    }
}

cudaError_t launch_relayout(int dtype, const void* src, int na, int ns, const BlockDev* blocks, int nblk,
                            int max_pitch, void* dst, cudaStream_t st) {
    const long long per = (long long)na * max_pitch;
    const dim3 grid((unsigned)((per + 255) / 256 < 4096 ? (per + 255) / 256 : 4096), nblk);
    switch (dtype_size(dtype)) {
        case 4:
            return launch_kernel(relayout_kernel<uint32_t>, grid, dim3(256), 0, st, (const uint32_t*)src, na, ns, blocks,
                                 (uint32_t*)dst);
        case 2:
            return launch_kernel(relayout_kernel<uint16_t>, grid, dim3(256), 0, st, (const uint16_t*)src, na, ns, blocks,
                                 (uint16_t*)dst);
        default:
            return launch_kernel(relayout_kernel<uint8_t>, grid, dim3(256), 0, st, (const uint8_t*)src, na, ns, blocks,
                                 (uint8_t*)dst);
    }
}

// One CTA per row: max |M_rj| (exact, order-free), the scale, then the codes.
__global__ void quantize_kernel(int dtype, int ns, const float* __restrict__ M, size_t ld, void* __restrict__ codes,
                                float* __restrict__ scale) {
    __shared__ float red[32];
    const int r = blockIdx.x;
    const float* row = M + (size_t)r * ld;
    float m = 0.f;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) m = fmaxf(m, fabsf(row[j]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    float s = dtype == RTC_E4M3 ? __fdiv_rn(red[0], 448.0f) : red[0];
    if (!(s > 0.f)) s = 1.0f;
    if (threadIdx.x == 0) scale[r] = s;
    if (dtype == RTC_BF16) {
        __nv_bfloat16* out = static_cast<__nv_bfloat16*>(codes) + (size_t)r * ns;
        for (int j = threadIdx.x; j < ns; j += blockDim.x) out[j] = __float2bfloat16_rn(__fdiv_rn(row[j], s));
    } else {
        __nv_fp8_storage_t* out = static_cast<__nv_fp8_storage_t*>(codes) + (size_t)r * ns;
        for (int j = threadIdx.x; j < ns; j += blockDim.x)
            out[j] = __nv_cvt_float_to_fp8(__fdiv_rn(row[j], s), __NV_SATFINITE, __NV_E4M3);
    }
}

cudaError_t launch_quantize(int dtype, int na, int ns, const float* M, size_t ld, void* codes, float* scale,
                            cudaStream_t st) {
    if (na <= 0) return cudaSuccess;
    return launch_kernel(quantize_kernel, dim3(na), dim3(256), 0, st, dtype, ns, M, ld, codes, scale);
}

__global__ void check_finite_kernel(const float* __restrict__ x, size_t n, int* bad) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) *bad = 1;
}

cudaError_t launch_check_finite(const float* x, size_t n, int* bad, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    size_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    return launch_kernel(check_finite_kernel, dim3((unsigned)g), dim3(256), 0, st, x, n, bad);
}

}  // namespace rtc
