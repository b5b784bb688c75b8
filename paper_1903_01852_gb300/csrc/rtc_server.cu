// Multi-loop server: several independent AO loops (SCAO, LTAO, MCAO ...) kept
// resident on one GPU.  Loops are admitted by their device-memory footprint
// against a budget, queued (with a private copy of their description) while
// they do not fit, and admitted in arrival order as released loops free
// memory.  Every admitted loop runs in graph mode: its frames are CUDA graph
// launches on its own stream, so frames of different loops that arrive while
// others are on the GPU overlap on the device.  A host thread polls the
// page-locked completion words and keeps each loop's latency samples
// (submission -> commands written).
//
// The paper runs one DARC instance per WFS node plus a master (Section 3);
// serving several whole loops on one device has no counterpart there.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "rtc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

size_t esize(int dtype) { return dtype == RTC_F32 ? 4 : dtype == RTC_BF16 ? 2 : 1; }

// A private copy of a loop description, for loops that wait in the queue.
struct OwnedDesc {
    std::vector<rtc_wfs> wfs;
    std::vector<std::vector<uint8_t>> valid;
    std::vector<std::vector<float>> dark, flat;
    std::vector<const float*> dark_p, flat_p;
    std::vector<float> threshold, ref, Ms, Ps, a0;
    std::vector<int32_t> mode;
    std::vector<uint8_t> M, P, D;
    std::vector<float> Ds;
    rtc_geometry g{};
    rtc_calib c{};
    rtc_cmat m{};
    rtc_polc p{};

    OwnedDesc(const rtc_geometry* G, const rtc_calib* C, const rtc_cmat* Mx, const rtc_polc* Px) {
        g = *G;
        wfs.assign(G->wfs, G->wfs + G->nwfs);
        valid.resize(G->nwfs);
        dark.resize(G->nwfs);
        flat.resize(G->nwfs);
        for (int k = 0; k < G->nwfs; ++k) {
            const rtc_wfs& w = G->wfs[k];
            const size_t nv = w.kind == RTC_WFS_SH ? (size_t)w.nsubx * w.nsuby : (size_t)w.pupil * w.pupil;
            if (w.valid) valid[k].assign(w.valid, w.valid + nv);
            const size_t np = (size_t)w.width * w.height;
            if (C && C->dark && C->dark[k]) dark[k].assign(C->dark[k], C->dark[k] + np);
            if (C && C->flat && C->flat[k]) flat[k].assign(C->flat[k], C->flat[k] + np);
        }
        if (C && C->threshold) threshold.assign(C->threshold, C->threshold + G->nwfs);
        if (C && C->thresh_mode) mode.assign(C->thresh_mode, C->thresh_mode + G->nwfs);
        if (C && C->ref_slopes) ref.assign(C->ref_slopes, C->ref_slopes + Mx->ns);
        m = *Mx;
        const size_t mb = (size_t)Mx->na * Mx->ns * esize(Mx->dtype);
        M.assign(static_cast<const uint8_t*>(Mx->data), static_cast<const uint8_t*>(Mx->data) + mb);
        if (Mx->row_scale) Ms.assign(Mx->row_scale, Mx->row_scale + Mx->na);
        p = *Px;
        if (Px->P) {
            const size_t pb = (size_t)Mx->na * Mx->na * esize(Px->dtype);
            P.assign(static_cast<const uint8_t*>(Px->P), static_cast<const uint8_t*>(Px->P) + pb);
            if (Px->row_scale) Ps.assign(Px->row_scale, Px->row_scale + Mx->na);
        }
        if (Px->D) {
            const size_t db = (size_t)Mx->ns * Mx->na * esize(Px->d_dtype);
            D.assign(static_cast<const uint8_t*>(Px->D), static_cast<const uint8_t*>(Px->D) + db);
            if (Px->d_row_scale) Ds.assign(Px->d_row_scale, Px->d_row_scale + Mx->ns);
        }
        if (Px->a0) a0.assign(Px->a0, Px->a0 + Mx->na);
        // pointers into the copies
        for (int k = 0; k < G->nwfs; ++k) wfs[k].valid = valid[k].empty() ? nullptr : valid[k].data();
        g.wfs = wfs.data();
        dark_p.resize(G->nwfs);
        flat_p.resize(G->nwfs);
        for (int k = 0; k < G->nwfs; ++k) {
            dark_p[k] = dark[k].empty() ? nullptr : dark[k].data();
            flat_p[k] = flat[k].empty() ? nullptr : flat[k].data();
        }
        c.dark = dark_p.data();
        c.flat = flat_p.data();
        c.threshold = threshold.empty() ? nullptr : threshold.data();
        c.thresh_mode = mode.empty() ? nullptr : mode.data();
        c.ref_slopes = ref.empty() ? nullptr : ref.data();
        m.data = M.data();
        m.row_scale = Ms.empty() ? nullptr : Ms.data();
        p.P = P.empty() ? nullptr : P.data();
        p.row_scale = Ps.empty() ? nullptr : Ps.data();
        p.a0 = a0.empty() ? nullptr : a0.data();
        p.D = D.empty() ? nullptr : D.data();
        p.d_row_scale = Ds.empty() ? nullptr : Ds.data();
    }
};

struct Inflight {
    int slot;
    unsigned long long seq;
    Clock::time_point t_submit;
};

struct SLoop {
    int id = 0;
    rtc_loop* L = nullptr;
    uint64_t footprint = 0;
    bool admitted = false;
    bool creating = false;
    int busy = 0;                        // submits in progress (under the server mutex)
    std::unique_ptr<OwnedDesc> desc;     // while queued
    std::deque<Inflight> inflight;
    std::vector<float> lat_us;
};

}  // namespace

struct rtc_server {
    int dev = 0;
    uint64_t budget = 0, used = 0;
    int next_id = 1;
    std::mutex mu;
    std::map<int, std::unique_ptr<SLoop>> loops;
    std::deque<int> queue;
    std::thread poller;
    std::atomic<bool> stop{false};
    std::string err;
};

namespace {

int sfail(rtc_server* S, int code, const std::string& msg) {
    if (S) S->err = msg;
    return code;
}

rtc_geometry with_graphs(const rtc_geometry* G, int dev) {
    rtc_geometry g = *G;
    g.device = dev;
    g.flags = (g.flags | RTC_FLAG_GRAPHS) & ~(RTC_FLAG_UPDATABLE | RTC_FLAG_TIMING | RTC_FLAG_STAGE_TIMING);
    return g;
}

// Completion poller: stamps the host time at which each frame's commands are written.
void poll(rtc_server* S) {
    while (!S->stop.load(std::memory_order_relaxed)) {
        bool any = false;
        {
            std::lock_guard<std::mutex> g(S->mu);
            const auto now = Clock::now();
            for (auto& kv : S->loops) {
                SLoop& l = *kv.second;
                if (!l.admitted) continue;
                while (!l.inflight.empty() && rtc::loop_frame_done(l.L, l.inflight.front().slot, l.inflight.front().seq)) {
                    l.lat_us.push_back(std::chrono::duration<float, std::micro>(now - l.inflight.front().t_submit).count());
                    l.inflight.pop_front();
                    any = true;
                }
            }
        }
        if (!any) std::this_thread::yield();
    }
}

// Create queued loops, in arrival order, while the head of the queue fits.
void admit_queued(rtc_server* S) {
    for (;;) {
        SLoop* l = nullptr;
        {
            std::lock_guard<std::mutex> g(S->mu);
            if (S->queue.empty()) return;
            auto it = S->loops.find(S->queue.front());
            if (it == S->loops.end()) {
                S->queue.pop_front();
                continue;
            }
            l = it->second.get();
            if (S->used + l->footprint > S->budget) return;
            S->used += l->footprint;
            S->queue.pop_front();
            l->creating = true;
        }
        const rtc_geometry g = with_graphs(&l->desc->g, S->dev);
        rtc_loop* L = nullptr;
        const int rc = rtc_create(&g, &l->desc->c, &l->desc->m, &l->desc->p, &L);
        std::lock_guard<std::mutex> g2(S->mu);
        l->creating = false;
        if (rc == RTC_OK) {
            l->L = L;
            l->admitted = true;
            l->desc.reset();
        } else {
            S->used -= l->footprint;      // stays queued at the front; retried on the next release
            S->queue.push_front(l->id);
            S->err = rtc_last_error(nullptr);
            return;
        }
    }
}

}  // namespace

extern "C" {

int rtc_server_create(int32_t device, uint64_t hbm_budget_bytes, rtc_server** out) {
    if (!out || hbm_budget_bytes == 0) return RTC_EINVAL;
    rtc_server* S = new (std::nothrow) rtc_server();
    if (!S) return RTC_ENOMEM;
    S->dev = device;
    S->budget = hbm_budget_bytes;
    S->poller = std::thread(poll, S);
    *out = S;
    return RTC_OK;
}

int rtc_server_destroy(rtc_server* S) {
    if (!S) return RTC_OK;
    S->stop = true;
    if (S->poller.joinable()) S->poller.join();
    for (auto& kv : S->loops)
        if (kv.second->L) rtc_destroy(kv.second->L);
    delete S;
    return RTC_OK;
}

int rtc_server_admit(rtc_server* S, const rtc_geometry* G, const rtc_calib* C, const rtc_cmat* M, const rtc_polc* P,
                     int32_t* loop_id) {
    if (!S || !G || !M || !P || !loop_id) return sfail(S, RTC_EINVAL, "server, geometry, cmat, polc and loop_id are required");
    uint64_t resident = 0, peak = 0;
    const rtc_geometry g = with_graphs(G, S->dev);
    int rc = rtc_footprint(&g, C, M, P, &resident, &peak);
    if (rc != RTC_OK) return sfail(S, rc, rtc_last_error(nullptr));
    if (resident > S->budget) return sfail(S, RTC_ENOMEM, "loop footprint exceeds the whole budget");
    auto l = std::make_unique<SLoop>();
    l->footprint = resident;
    SLoop* lp = l.get();
    bool now = false;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        l->id = S->next_id++;
        *loop_id = l->id;
        if (S->queue.empty() && S->used + resident <= S->budget) {
            S->used += resident;
            l->creating = true;
            now = true;
        } else {
            l->desc = std::make_unique<OwnedDesc>(G, C, M, P);
            S->queue.push_back(l->id);
        }
        S->loops[l->id] = std::move(l);
    }
    if (!now) return RTC_OK;
    rtc_loop* L = nullptr;
    rc = rtc_create(&g, C, M, P, &L);
    std::lock_guard<std::mutex> lk(S->mu);
    lp->creating = false;
    if (rc != RTC_OK) {
        S->used -= resident;
        S->loops.erase(lp->id);
        return sfail(S, rc, rtc_last_error(nullptr));
    }
    lp->L = L;
    lp->admitted = true;
    return RTC_OK;
}

int rtc_server_release(rtc_server* S, int32_t loop_id) {
    if (!S) return RTC_EINVAL;
    std::unique_ptr<SLoop> l;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->loops.find(loop_id);
        if (it == S->loops.end()) return sfail(S, RTC_ENOENT, "no such loop");
        if (it->second->creating) return sfail(S, RTC_EINVAL, "loop is being created");
        l = std::move(it->second);
        S->loops.erase(it);              // no new submit can find it now
        if (l->admitted) S->used -= l->footprint;
        S->queue.erase(std::remove(S->queue.begin(), S->queue.end(), loop_id), S->queue.end());
    }
    for (;;) {                           // a submit that found the loop before the erase finishes first
        {
            std::lock_guard<std::mutex> g(S->mu);
            if (l->busy == 0) break;
        }
        std::this_thread::yield();
    }
    if (l->L) rtc_destroy(l->L);     // waits for the loop's work, then frees its device memory
    admit_queued(S);
    return RTC_OK;
}

int rtc_server_loop(rtc_server* S, int32_t loop_id, rtc_loop** loop) {
    if (!S || !loop) return RTC_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->loops.find(loop_id);
    if (it == S->loops.end()) return sfail(S, RTC_ENOENT, "no such loop");
    *loop = it->second->admitted ? it->second->L : nullptr;
    return RTC_OK;
}

int rtc_server_submit(rtc_server* S, int32_t loop_id, uint64_t frame_id) {
    if (!S) return RTC_EINVAL;
    rtc_loop* L = nullptr;
    SLoop* l = nullptr;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->loops.find(loop_id);
        if (it == S->loops.end()) return sfail(S, RTC_ENOENT, "no such loop");
        if (!it->second->admitted) return sfail(S, RTC_EINVAL, "loop not admitted yet");
        l = it->second.get();
        L = l->L;
        ++l->busy;                       // rtc_server_release waits for it before destroying the loop
    }
    const auto t0 = Clock::now();
    const int rc = rtc_submit_frame_graph(L, frame_id);
    Inflight f{};
    if (rc == RTC_OK || rc == RTC_EDROPPED) rtc::loop_last_frame(L, &f.slot, &f.seq);
    f.t_submit = t0;
    std::lock_guard<std::mutex> g(S->mu);
    --l->busy;
    if (rc != RTC_OK && rc != RTC_EDROPPED) return sfail(S, rc, rtc_last_error(L));
    l->inflight.push_back(f);
    return rc;
}

int rtc_server_stats(rtc_server* S, int32_t loop_id, int32_t reset, rtc_server_loop_info* out) {
    if (!S || !out) return RTC_EINVAL;
    std::vector<float> lat;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->loops.find(loop_id);
        if (it == S->loops.end()) return sfail(S, RTC_ENOENT, "no such loop");
        SLoop& l = *it->second;
        out->admitted = l.admitted ? 1 : 0;
        out->footprint_bytes = l.footprint;
        lat = l.lat_us;
        if (reset) l.lat_us.clear();
    }
    out->frames = lat.size();
    out->p50_us = out->p99_us = out->p999_us = out->mean_us = out->jitter_rms_us = out->max_us = 0.0;
    if (lat.empty()) return RTC_OK;
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        const double k = (lat.size() - 1) * q;
        const size_t lo = (size_t)std::floor(k), hi = (size_t)std::ceil(k);
        return lat[lo] + (lat[hi] - lat[lo]) * (k - lo);
    };
    double sum = 0, sq = 0;
    for (float v : lat) sum += v;
    const double mean = sum / lat.size();
    for (float v : lat) sq += (v - mean) * (v - mean);
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    out->p999_us = pct(0.999);
    out->mean_us = mean;
    out->jitter_rms_us = std::sqrt(sq / lat.size());
    out->max_us = lat.back();
    return RTC_OK;
}

int rtc_server_usage(rtc_server* S, uint64_t* used_bytes, uint64_t* budget_bytes, int32_t* admitted, int32_t* queued) {
    if (!S) return RTC_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    if (used_bytes) *used_bytes = S->used;
    if (budget_bytes) *budget_bytes = S->budget;
    int a = 0;
    for (auto& kv : S->loops) a += kv.second->admitted ? 1 : 0;
    if (admitted) *admitted = a;
    if (queued) *queued = (int32_t)S->queue.size();
    return RTC_OK;
}

const char* rtc_server_last_error(const rtc_server* S) { return S ? S->err.c_str() : ""; }

}  // extern "C"
