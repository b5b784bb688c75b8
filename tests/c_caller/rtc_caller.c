/* A plain C caller of the library's C ABI (include/rtc.h), used by the tests to
 * check the boundary without the Python binding.
 *
 *   rtc_caller IN OUT
 *
 * IN (little-endian, written by the test):
 *   int32 nwfs, na, ns, nframes, nchunks, device
 *   per WFS: int32 kind, width, height, nsubx, nsuby, npx, ox, oy, pupil, qx[4], qy[4],
 *            nblocks, norm, thresh_mode; float32 threshold;
 *            uint8 valid[nsuby*nsubx or pupil*pupil]; float32 dark[h*w], flat[h*w]
 *   float32 M[na*ns]; int32 has_P; float32 P[na*na] if has_P;
 *   float32 gain, leak; int32 has_ref; float32 ref[ns] if has_ref
 *   per frame, per WFS: uint16 pixels[h*w]
 * OUT: per frame: uint64 frame id, float32 commands[na]
 *
 * Each frame is submitted as nchunks row chunks per WFS (rows split evenly, the
 * WFS interleaved chunk by chunk), frame ids 1, 2, ...  Exit status 0 on
 * success; otherwise the library's error text is printed. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "rtc.h"

static FILE* in;

static void* take(size_t bytes) {
    void* p = malloc(bytes ? bytes : 1);
    if (!p || (bytes && fread(p, 1, bytes, in) != bytes)) {
        fprintf(stderr, "short input\n");
        exit(2);
    }
    return p;
}

static int32_t take_i32(void) {
    int32_t v;
    if (fread(&v, 4, 1, in) != 1) {
        fprintf(stderr, "short input\n");
        exit(2);
    }
    return v;
}

static float take_f32(void) {
    float v;
    if (fread(&v, 4, 1, in) != 1) {
        fprintf(stderr, "short input\n");
        exit(2);
    }
    return v;
}

int main(int argc, char** argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: rtc_caller IN OUT\n");
        return 2;
    }
    in = fopen(argv[1], "rb");
    FILE* out = fopen(argv[2], "wb");
    if (!in || !out) {
        fprintf(stderr, "cannot open files\n");
        return 2;
    }
    const int32_t nwfs = take_i32(), na = take_i32(), ns = take_i32();
    const int32_t nframes = take_i32(), nchunks = take_i32(), device = take_i32();
    if (nwfs < 1 || nwfs > RTC_MAX_WFS || nchunks < 1) {
        fprintf(stderr, "bad header\n");
        return 2;
    }
    rtc_wfs wfs[RTC_MAX_WFS];
    const float* dark[RTC_MAX_WFS];
    const float* flat[RTC_MAX_WFS];
    float threshold[RTC_MAX_WFS];
    int32_t mode[RTC_MAX_WFS];
    for (int k = 0; k < nwfs; ++k) {
        rtc_wfs* w = &wfs[k];
        w->kind = take_i32();
        w->width = take_i32();
        w->height = take_i32();
        w->nsubx = take_i32();
        w->nsuby = take_i32();
        w->npx = take_i32();
        w->ox = take_i32();
        w->oy = take_i32();
        w->pupil = take_i32();
        for (int q = 0; q < 4; ++q) w->qx[q] = take_i32();
        for (int q = 0; q < 4; ++q) w->qy[q] = take_i32();
        w->nblocks = take_i32();
        w->norm = take_i32();
        mode[k] = take_i32();
        threshold[k] = take_f32();
        const size_t nv = w->kind == RTC_WFS_SH ? (size_t)w->nsubx * w->nsuby : (size_t)w->pupil * w->pupil;
        w->valid = (const uint8_t*)take(nv);
        const size_t npix = (size_t)w->width * w->height;
        dark[k] = (const float*)take(npix * 4);
        flat[k] = (const float*)take(npix * 4);
    }
    const float* M = (const float*)take((size_t)na * ns * 4);
    const int32_t has_p = take_i32();
    const float* P = has_p ? (const float*)take((size_t)na * na * 4) : NULL;
    const float gain = take_f32(), leak = take_f32();
    const int32_t has_ref = take_i32();
    const float* ref = has_ref ? (const float*)take((size_t)ns * 4) : NULL;

    rtc_geometry geo = {0};
    geo.nwfs = nwfs;
    geo.wfs = wfs;
    geo.device = device;
    geo.ring = 4;
    rtc_calib cal = {dark, flat, threshold, mode, ref};
    rtc_cmat cm = {na, ns, RTC_F32, M, NULL};
    rtc_polc pol = {0};
    pol.P = P;
    pol.dtype = RTC_F32;
    pol.gain = gain;
    pol.leak = leak;
    pol.mode = RTC_POLC_IMPLICIT;
    rtc_loop* loop = NULL;
    int rc = rtc_create(&geo, &cal, &cm, &pol, &loop);
    if (rc != RTC_OK) {
        fprintf(stderr, "rtc_create: %d %s\n", rc, rtc_last_error(NULL));
        return 1;
    }
    float* cmds = (float*)malloc((size_t)na * 4);
    for (int f = 0; f < nframes; ++f) {
        uint16_t* px[RTC_MAX_WFS];
        for (int k = 0; k < nwfs; ++k) px[k] = (uint16_t*)take((size_t)wfs[k].width * wfs[k].height * 2);
        const uint64_t id = (uint64_t)f + 1u;
        for (int c = 0; c < nchunks; ++c)
            for (int k = 0; k < nwfs; ++k) {
                const int h = wfs[k].height;
                const int r0 = (int)((long long)c * h / nchunks), r1 = (int)((long long)(c + 1) * h / nchunks);
                if (r1 <= r0) continue;
                rtc_chunk ch = {id, k, r0, r1, px[k] + (size_t)r0 * wfs[k].width, (size_t)wfs[k].width * 2};
                rc = rtc_submit_pixels(loop, &ch);
                if (rc != RTC_OK) {
                    fprintf(stderr, "rtc_submit_pixels: %d %s\n", rc, rtc_last_error(loop));
                    return 1;
                }
            }
        uint64_t got = 0;
        rc = rtc_get_commands(loop, cmds, (size_t)na, &got, 60000000);
        if (rc != RTC_OK || got != id) {
            fprintf(stderr, "rtc_get_commands: %d %s\n", rc, rtc_last_error(loop));
            return 1;
        }
        fwrite(&got, 8, 1, out);
        fwrite(cmds, 4, (size_t)na, out);
        for (int k = 0; k < nwfs; ++k) free(px[k]);
    }
    rtc_destroy(loop);
    fclose(out);
    fclose(in);
    return 0;
}
