// rs_serve.cu -- the serving form: a map server with continuous batching.
//
// Requests of mixed (kappa, gamma, N, resolution) arrive at any time.  A
// request is admitted while its device memory (lens list, int32 count map,
// float32 magnification map, statistics) fits the budget and a slot is
// free; then its lens field is drawn on the device and its count map
// zeroed.  Admitted requests keep lens set and partial map resident.  The
// server runs time slices: each slice is one persistent batched launch over
// a range of ray tiles of every running request chosen by rs_sched_plan
// (shortest remaining work first by default), sized to about slice_ms of
// GPU time, so a request that arrives while others run joins the next slice.
// A request whose last tiles are in a slice gets its magnification (Eq. 4)
// and statistics copy right after that slice's launch; the slice's event
// gives its completion time.  Counts are integers accumulated over tiles, so
// splitting a map over slices changes nothing: a request's map is
// bit-identical alone or in any mix.
//
// Host-side only waits: every wait on the GPU is a CUDA event wait or a
// condition-variable wait with a timeout; no device code waits on anything.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "rs_internal.cuh"

namespace rs {
namespace {

struct Req {
    int64_t ticket = 0;
    rs_request r;
    int state = RS_REQ_QUEUED;
    int err = RS_OK;
    int skips = 0;
    bool cancel = false;
    int inflight = 0;              // slices in flight that touch this request
    double t_submit = 0, t_admit = -1, t_done = -1;
    int64_t n_lens = 0;
    int64_t bytes = 0;
    double* d_lens = nullptr;
    int32_t* d_counts = nullptr;
    float* d_mu = nullptr;
    int64_t* d_stats = nullptr;
    // RS_PREC_REFINED: list counter, second-pass work counter, then the
    // ids of the rays near pixel edges
    unsigned long long* d_refine = nullptr;
    int64_t refine_cap = 0;
    int slot = -1;                 // pinned statistics slot
    int64_t stats[RS_NSTATS] = {0};
    MapDesc desc;
    float inv_navg = 0.f;
    int64_t npx = 0;
    int64_t tiles_total = 0, next_tile = 0;
    double work_per_tile = 0;
    bool unit = true;
};

struct Slice {
    cudaEvent_t ev = nullptr;
    std::vector<int64_t> touched;
    std::vector<int64_t> finishing;
};

// refined form: the ray list of a map, as rs_shoot_map sizes it
int64_t refine_capacity(const rs_request& r)
{
    return rs::refine_capacity(r.grid.n1 * r.grid.n2);
}

int64_t request_bytes(const rs_request& r, int64_t n_lens, bool refined)
{
    const int64_t npx = r.map.npix * r.map.npix;
    const int64_t a = 256;
    auto up = [&](int64_t v) { return (v + a - 1) / a * a; };
    return up(3 * n_lens * 8) + up(npx * 4) + up(npx * 4) + up(RS_NSTATS * 8) +
           (refined ? up(32 + refine_list_bytes(refine_capacity(r))) : 0);
}

}  // namespace
}  // namespace rs

using namespace rs;

struct rs_server {
    rs_server_config cfg;
    int device = 0;
    ShapeInfo si;
    std::mutex mu;
    std::condition_variable cv;      // request state changes, new work
    std::thread worker;
    bool stop = false;
    int fatal = RS_OK;
    cudaStream_t stream = nullptr;   // admission work, frees; slices of even index
    cudaStream_t stream2 = nullptr;  // slices of odd index
    cudaEvent_t admit_ev = nullptr;  // orders admission work before stream2's slices
    cudaMemPool_t pool = nullptr;
    cudaEvent_t ref_ev = nullptr;
    double t_ref = 0.0;              // server clock at ref_ev
    std::chrono::steady_clock::time_point t0;
    std::map<int64_t, Req*> reqs;
    std::deque<int64_t> queue;       // queued tickets, arrival order
    std::vector<int64_t> running;    // admitted, not finished
    std::deque<Slice> inflight;
    std::vector<cudaEvent_t> spare_events;
    int64_t* h_stats = nullptr;      // pinned, RS_NSTATS per slot
    std::vector<int> free_slots;
    int64_t next_ticket = 1;
    int64_t bytes_used = 0, peak_bytes = 0;
    int64_t n_slices = 0, n_launches = 0, n_admitted = 0, n_completed = 0, n_failed = 0,
            n_cancelled = 0;
    int inject_left = 0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace rs {
namespace {

void free_device(rs_server* S, Req* q)
{
    if (q->d_lens) cudaFreeAsync(q->d_lens, S->stream);
    if (q->d_counts) cudaFreeAsync(q->d_counts, S->stream);
    if (q->d_mu) cudaFreeAsync(q->d_mu, S->stream);
    if (q->d_stats) cudaFreeAsync(q->d_stats, S->stream);
    if (q->d_refine) cudaFreeAsync(q->d_refine, S->stream);
    q->d_refine = nullptr;
    q->d_lens = nullptr;
    q->d_counts = nullptr;
    q->d_mu = nullptr;
    q->d_stats = nullptr;
    if (q->bytes) S->bytes_used -= q->bytes;
    q->bytes = 0;
    if (q->slot >= 0) S->free_slots.push_back(q->slot);
    q->slot = -1;
}

void finish(rs_server* S, Req* q, int state, int err)
{
    q->state = state;
    q->err = err;
    if (state == RS_REQ_FAILED) ++S->n_failed;
    if (state == RS_REQ_CANCELLED) ++S->n_cancelled;
    auto it = std::find(S->running.begin(), S->running.end(), q->ticket);
    if (it != S->running.end()) S->running.erase(it);
    S->cv.notify_all();
}

// Allocate and initialise one queued request; false if the allocation failed.
bool admit_one(rs_server* S, Req* q)
{
    if (S->inject_left > 0) {          // test hook: behave as out of memory
        --S->inject_left;
        return false;
    }
    const int64_t npx = q->r.map.npix * q->r.map.npix;
    cudaError_t e = cudaSuccess;
    if (q->n_lens > 0)
        e = cudaMallocFromPoolAsync((void**)&q->d_lens, (size_t)(3 * q->n_lens) * 8, S->pool,
                                    S->stream);
    if (e == cudaSuccess)
        e = cudaMallocFromPoolAsync((void**)&q->d_counts, (size_t)npx * 4, S->pool, S->stream);
    if (e == cudaSuccess)
        e = cudaMallocFromPoolAsync((void**)&q->d_mu, (size_t)npx * 4, S->pool, S->stream);
    if (e == cudaSuccess)
        e = cudaMallocFromPoolAsync((void**)&q->d_stats, RS_NSTATS * 8, S->pool, S->stream);
    const bool refined = S->cfg.precision == RS_PREC_REFINED;
    if (e == cudaSuccess && refined) {
        q->refine_cap = refine_capacity(q->r);
        e = cudaMallocFromPoolAsync((void**)&q->d_refine, (size_t)(32 + refine_list_bytes(q->refine_cap)),
                                    S->pool, S->stream);
    }
    if (e != cudaSuccess || S->free_slots.empty()) {
        cudaGetLastError();
        const int64_t b = q->bytes;
        q->bytes = 0;
        free_device(S, q);
        q->bytes = b;
        return false;
    }
    q->slot = S->free_slots.back();
    S->free_slots.pop_back();
    S->bytes_used += q->bytes;
    S->peak_bytes = std::max(S->peak_bytes, S->bytes_used);
    int rc = launch_make_lenses(&q->r.field, q->r.seed, q->d_lens, q->n_lens, S->stream);
    if (!rc) rc = launch_fill_i32(q->d_counts, npx, 0, S->stream);
    if (!rc) rc = launch_fill_i64(q->d_stats, RS_NSTATS, 0, S->stream);
    if (!rc && refined)
        rc = cuda_fail(cudaMemsetAsync(q->d_refine, 0, 32, S->stream), "refinement counters");
    // slices run on both streams: the second one waits for this set-up too
    if (!rc) rc = cuda_fail(cudaEventRecord(S->admit_ev, S->stream), "event record");
    if (!rc) rc = cuda_fail(cudaStreamWaitEvent(S->stream2, S->admit_ev, 0), "stream wait");
    rs_options o = {S->cfg.precision, 0, S->cfg.shape, 0};
    ShapeInfo si;
    if (!rc) rc = prepare_map(&q->r.macro, q->d_lens, q->n_lens, &q->r.grid, &q->r.map, o,
                              &q->desc, &si, false);
    if (rc) {
        finish(S, q, RS_REQ_FAILED, rc);
        free_device(S, q);
        return true;
    }
    q->desc.counts = q->d_counts;
    q->desc.stats = reinterpret_cast<unsigned long long*>(q->d_stats);
    if (refined) {
        q->desc.refine_count = q->d_refine;
        q->desc.refine_ids = reinterpret_cast<int64_t*>(q->d_refine + 4);
        q->desc.refine_cap = q->refine_cap;
    }
    q->npx = npx;
    double navg = 0.0;
    rs_navg(&q->r.grid, &q->r.map, &navg);
    q->inv_navg = (float)(1.0 / navg);
    const int64_t t1 = (q->r.grid.n1 + si.tx - 1) / si.tx;
    const int64_t t2 = (q->r.grid.n2 + si.ty - 1) / si.ty;
    q->tiles_total = t1 * t2;
    q->next_tile = 0;
    // per-tile cost: the deflection sum plus about 64 interactions' worth of
    // per-ray FP64 work and binning
    q->work_per_tile = (double)si.tx * si.ty * (double)(q->n_lens + 64);
    q->unit = q->r.field.mass_model == RS_MASS_UNIT;
    q->state = RS_REQ_RUNNING;
    q->t_admit = S->now();
    ++S->n_admitted;
    S->running.push_back(q->ticket);
    return true;
}

// Finished slices: mark the requests whose last work they carried.
void complete_slices(rs_server* S, bool* progressed)
{
    while (!S->inflight.empty()) {
        Slice& sl = S->inflight.front();
        const cudaError_t e = cudaEventQuery(sl.ev);
        if (e == cudaErrorNotReady) break;
        float ms = 0.f;
        const int rc = cuda_fail(e, "slice");
        if (!rc) cudaEventElapsedTime(&ms, S->ref_ev, sl.ev);
        const double t_done = S->t_ref + ms / 1e3;
        for (int64_t t : sl.touched) {
            auto it = S->reqs.find(t);
            if (it != S->reqs.end()) --it->second->inflight;
        }
        for (int64_t t : sl.finishing) {
            auto it = S->reqs.find(t);
            if (it == S->reqs.end()) continue;
            Req* q = it->second;
            if (rc) {
                finish(S, q, RS_REQ_FAILED, rc);
                continue;
            }
            memcpy(q->stats, S->h_stats + RS_NSTATS * q->slot, sizeof q->stats);
            S->free_slots.push_back(q->slot);
            q->slot = -1;
            q->t_done = t_done;
            ++S->n_completed;
            finish(S, q, RS_REQ_DONE, RS_OK);
        }
        if (rc) S->fatal = rc;
        S->spare_events.push_back(sl.ev);
        S->inflight.pop_front();
        *progressed = true;
    }
    // cancelled requests without work in flight release their memory
    for (size_t k = 0; k < S->running.size();) {
        Req* q = S->reqs[S->running[k]];
        if (q->cancel && q->inflight == 0) {
            free_device(S, q);
            finish(S, q, RS_REQ_CANCELLED, RS_OK);
            *progressed = true;
        } else {
            ++k;
        }
    }
}

void admit_queued(rs_server* S, bool* progressed)
{
    if (S->queue.empty()) return;
    std::vector<rs_sched_queued> q(S->queue.size());
    for (size_t k = 0; k < S->queue.size(); ++k) {
        Req* r = S->reqs[S->queue[k]];
        q[k].bytes = r->bytes;
        q[k].skips = r->skips;
        q[k].pad_ = 0;
    }
    std::vector<int32_t> adm(q.size(), 0);
    rs_sched_admit(q.data(), (int)q.size(), S->bytes_used, S->cfg.hbm_budget,
                   (int)S->running.size(), S->cfg.max_active, S->cfg.max_skips, adm.data());
    std::deque<int64_t> keep;
    bool blocked = false;
    for (size_t k = 0; k < S->queue.size(); ++k) {
        Req* r = S->reqs[S->queue[k]];
        if (r->cancel) {
            finish(S, r, RS_REQ_CANCELLED, RS_OK);
            *progressed = true;
            continue;
        }
        if (adm[k] && !blocked) {
            if (admit_one(S, r)) {
                *progressed = true;
                continue;
            }
            // allocation failed: retry later, unless nothing runs that
            // could free memory
            if (S->running.empty()) {
                finish(S, r, RS_REQ_FAILED, RS_ENOMEM);
                *progressed = true;
                continue;
            }
            blocked = true;
        }
        if (!adm[k]) ++r->skips;
        keep.push_back(r->ticket);
    }
    S->queue.swap(keep);
}

// Plan and launch one slice over the running requests.
int launch_slice(rs_server* S, bool* progressed)
{
    std::vector<Req*> act;
    for (int64_t t : S->running) {
        Req* q = S->reqs[t];
        if (!q->cancel && q->next_tile < q->tiles_total) act.push_back(q);
    }
    if (act.empty()) return RS_OK;
    std::vector<rs_sched_item> items(act.size());
    for (size_t k = 0; k < act.size(); ++k)
        items[k] = rs_sched_item{act[k]->ticket, act[k]->tiles_total - act[k]->next_tile,
                                 act[k]->work_per_tile};
    const double rate = S->cfg.rate_gint > 0 ? S->cfg.rate_gint : 5000.0;
    const double budget = S->cfg.slice_ms > 0 ? S->cfg.slice_ms * rate * 1e6 : INFINITY;
    std::vector<int64_t> take(act.size(), 0);
    rs_sched_plan(items.data(), (int)items.size(), budget, S->cfg.policy, MAX_BATCH, take.data());

    std::vector<Req*> sel;
    for (size_t k = 0; k < act.size(); ++k)
        if (take[k] > 0) sel.push_back(act[k]);
    std::vector<int64_t> tk(sel.size());
    for (size_t k = 0, j = 0; k < act.size(); ++k)
        if (take[k] > 0) tk[j++] = take[k];
    // heaviest tiles first inside the launch
    std::vector<size_t> ord(sel.size());
    for (size_t k = 0; k < ord.size(); ++k) ord[k] = k;
    std::stable_sort(ord.begin(), ord.end(),
                     [&](size_t a, size_t b) { return sel[a]->n_lens > sel[b]->n_lens; });
    std::vector<MapDesc> maps;
    std::vector<char> map_unit;
    bool all_unit = true, any_unit = false;
    Slice sl;
    for (size_t k : ord) {
        Req* q = sel[k];
        MapDesc d = q->desc;
        d.tile0 = q->next_tile;
        d.tile_count = tk[k];
        q->next_tile += tk[k];
        maps.push_back(d);
        map_unit.push_back(q->unit);
        all_unit = all_unit && q->unit;
        any_unit = any_unit || q->unit;
        ++q->inflight;
        sl.touched.push_back(q->ticket);
        if (q->next_tile >= q->tiles_total) sl.finishing.push_back(q->ticket);
    }
    // consecutive slices alternate between two streams, so the next slice's
    // CTAs start on SMs freed by the tail of the previous one
    cudaStream_t st = (S->n_slices & 1) ? S->stream2 : S->stream;
    ShootExtra x = {0, nullptr, nullptr, nullptr};
    // a slice of one request runs the single-map kernel over its tile range
    // (the batched kernels index their map descriptors at run time and are
    // a few percent slower per interaction)
    auto launch = [&](const std::vector<MapDesc>& ms, bool unit) {
        const bool single = ms.size() == 1 &&
                            has_single_kernel(S->cfg.shape, S->cfg.precision, unit);
        ++S->n_launches;
        return launch_shoot(ms.data(), (int)ms.size(), x, S->cfg.shape, S->cfg.precision, unit,
                            MODE_BIN, st, 0, !single);
    };
    int rc = 0;
    if (S->cfg.precision == RS_PREC_DOUBLE_SINGLE && any_unit && !all_unit) {
        // the double-single kernels round a unit mass differently from a
        // general one (the compensated and FP32 ones multiply by m = 1, which
        // is exact): one launch per mass model, so that every request takes
        // the kernel of its single-map call
        for (bool unit : {true, false}) {
            std::vector<MapDesc> part;
            for (size_t k = 0; k < maps.size(); ++k)
                if ((bool)map_unit[k] == unit) part.push_back(maps[k]);
            if (!rc) rc = launch(part, unit);
        }
    } else {
        rc = launch(maps, all_unit);
    }
    if (!rc && !sl.finishing.empty() && !S->inflight.empty()) {
        // a finishing request may have tiles in the slice still running on
        // the other stream: its map is complete only after both
        rc = cuda_fail(cudaStreamWaitEvent(st, S->inflight.back().ev, 0), "stream wait");
    }
    if (!rc && !sl.finishing.empty() && S->cfg.precision == RS_PREC_REFINED) {
        // the refined form's second pass for the finishing requests (their
        // lists are complete now), one launch per mass model: the unit-mass
        // and the general kernel round the float-float terms differently, and
        // each request takes the kernel of its single-map call.  The first
        // request's work counter of each launch is still zero and serves it.
        for (bool unit : {true, false}) {
            std::vector<MapDesc> fin;
            unsigned long long* work = nullptr;
            for (int64_t t : sl.finishing) {
                const Req* q = S->reqs[t];
                if (q->unit != unit) continue;
                fin.push_back(q->desc);
                if (!work) work = q->d_refine + 2;
            }
            if (!rc && !fin.empty())
                rc = launch_refine(fin.data(), (int)fin.size(), work, unit, st);
        }
    }
    if (!rc && !sl.finishing.empty()) {
        std::vector<const int32_t*> c;
        std::vector<float*> m;
        std::vector<int64_t> n;
        std::vector<float> inv;
        for (int64_t t : sl.finishing) {
            Req* q = S->reqs[t];
            c.push_back(q->d_counts);
            m.push_back(q->d_mu);
            n.push_back(q->npx);
            inv.push_back(q->inv_navg);
        }
        rc = launch_magnification_batch(c.data(), m.data(), n.data(), inv.data(), (int)c.size(),
                                        st);
        for (int64_t t : sl.finishing) {
            Req* q = S->reqs[t];
            if (!rc)
                rc = cuda_fail(cudaMemcpyAsync(S->h_stats + RS_NSTATS * q->slot, q->d_stats, RS_NSTATS * 8,
                                               cudaMemcpyDeviceToHost, st),
                               "stats copy");
        }
    }
    if (S->spare_events.empty()) {
        cudaEvent_t ev;
        if (!rc) rc = cuda_fail(cudaEventCreate(&ev), "event");
        if (!rc) S->spare_events.push_back(ev);
    }
    if (!rc) {
        sl.ev = S->spare_events.back();
        S->spare_events.pop_back();
        rc = cuda_fail(cudaEventRecord(sl.ev, st), "event record");
    }
    if (rc) {
        for (int64_t t : sl.touched) {
            Req* q = S->reqs[t];
            --q->inflight;
            finish(S, q, RS_REQ_FAILED, rc);
        }
        return rc;
    }
    S->inflight.push_back(sl);
    ++S->n_slices;
    *progressed = true;
    return RS_OK;
}

// One scheduling step under the lock.
int step_locked(rs_server* S, bool* progressed)
{
    *progressed = false;
    complete_slices(S, progressed);
    admit_queued(S, progressed);
    if (S->inflight.size() < 2) {
        const int rc = launch_slice(S, progressed);
        if (rc) S->fatal = rc;
    }
    return S->fatal;
}

bool terminal(int st)
{
    return st == RS_REQ_DONE || st == RS_REQ_FAILED || st == RS_REQ_CANCELLED;
}

void worker_main(rs_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool prog = false;
        step_locked(S, &prog);
        if (S->inflight.size() >= 2 || (!prog && !S->inflight.empty())) {
            cudaEvent_t ev = S->inflight.front().ev;
            lk.unlock();
            cudaEventSynchronize(ev);
            lk.lock();
            continue;
        }
        if (!prog) S->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

void fill_result(const Req* q, rs_result* out)
{
    memset(out, 0, sizeof *out);
    out->state = q->state;
    out->error = q->err;
    if (q->state == RS_REQ_DONE) {
        out->d_mu = q->d_mu;
        out->d_counts = q->d_counts;
        memcpy(out->stats, q->stats, sizeof q->stats);
    }
    out->t_submit = q->t_submit;
    out->t_admit = q->t_admit;
    out->t_done = q->t_done;
    out->tiles_total = q->tiles_total;
    out->tiles_launched = q->next_tile;
    out->n_lens = q->n_lens;
}

}  // namespace
}  // namespace rs

extern "C" {

int rs_server_create(const rs_server_config* cfg, rs_server** out)
{
    clear_error();
    if (!cfg || !out) return fail(RS_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->hbm_budget <= 0) return fail(RS_EINVAL, "hbm_budget must be > 0");
    if (cfg->max_active < 1 || cfg->max_active > MAX_BATCH)
        return fail(RS_EINVAL, "max_active must be in 1..%d", MAX_BATCH);
    if (cfg->max_queue < 1) return fail(RS_EINVAL, "max_queue must be >= 1");
    if (cfg->policy != RS_SCHED_SRPT && cfg->policy != RS_SCHED_FIFO)
        return fail(RS_EINVAL, "policy %d unknown", cfg->policy);
    ShapeInfo si;
    int rc = shape_info(cfg->shape, cfg->precision, &si);
    if (rc) return rc;
    if (!si.batch) return fail(RS_EINVAL, "shape %d has no batched kernel", cfg->shape);
    rs_server* S = new rs_server();
    S->cfg = *cfg;
    if (S->cfg.max_skips < 0) S->cfg.max_skips = 0;
    S->si = si;
    S->inject_left = cfg->inject_alloc_failures;
    S->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&S->device);
    rc = cuda_fail(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking), "server stream");
    if (!rc)
        rc = cuda_fail(cudaStreamCreateWithFlags(&S->stream2, cudaStreamNonBlocking),
                       "server stream");
    if (!rc) rc = cuda_fail(cudaEventCreateWithFlags(&S->admit_ev, cudaEventDisableTiming), "event");
    if (!rc) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S->device;
        rc = cuda_fail(cudaMemPoolCreate(&S->pool, &props), "memory pool");
    }
    if (!rc) {
        // keep freed request memory in the pool (up to the budget) instead
        // of returning it to the driver at every synchronisation
        uint64_t thr = (uint64_t)cfg->hbm_budget;
        rc = cuda_fail(cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &thr),
                       "pool threshold");
    }
    if (!rc)
        rc = cuda_fail(cudaHostAlloc((void**)&S->h_stats, (size_t)cfg->max_active * RS_NSTATS * 8,
                                     cudaHostAllocDefault),
                       "pinned statistics");
    for (int k = cfg->max_active - 1; k >= 0; --k) S->free_slots.push_back(k);
    if (!rc) rc = cuda_fail(cudaEventCreate(&S->ref_ev), "event");
    if (!rc) rc = cuda_fail(cudaEventRecord(S->ref_ev, S->stream), "event record");
    if (!rc) rc = cuda_fail(cudaEventSynchronize(S->ref_ev), "event sync");
    S->t_ref = S->now();
    if (!rc) rc = prime_launch(cfg->shape, cfg->precision, true, true);
    if (!rc) rc = prime_launch(cfg->shape, cfg->precision, false, true);
    // single-map kernels for one-request slices, where the shape has them
    for (bool unit : {true, false})
        if (!rc && prime_launch(cfg->shape, cfg->precision, unit, false) != RS_OK) clear_error();
    if (rc) {
        rs_server_destroy(S);
        return rc;
    }
    if (cfg->threaded) S->worker = std::thread(worker_main, S);
    *out = S;
    return RS_OK;
}

int rs_server_submit(rs_server* S, const rs_request* req, int64_t* ticket)
{
    clear_error();
    if (!S || !req || !ticket) return fail(RS_EINVAL, "null argument");
    // validate everything that does not need the device buffers
    const rs_lensfield& f = req->field;
    if (f.mass_model != RS_MASS_UNIT && f.mass_model != RS_MASS_SALPETER)
        return fail(RS_EINVAL, "mass_model %d unknown", f.mass_model);
    int64_t n = req->n_lens;
    int rc;
    if (n <= 0 && (rc = rs_lens_count(f.kappa_star, f.radius, 1.0, &n))) return rc;
    rs_options o = {S->cfg.precision, 0, S->cfg.shape, 0};
    MapDesc d;
    ShapeInfo si;
    double dummy = 1.0;
    if ((rc = prepare_map(&req->macro, n > 0 ? &dummy : nullptr, n, &req->grid, &req->map, o, &d,
                          &si, false)))
        return rc;
    if (req->grid.n1 < 1 || req->grid.n2 < 1) return fail(RS_EINVAL, "empty ray grid");
    const int64_t bytes = request_bytes(*req, n, S->cfg.precision == RS_PREC_REFINED);
    if (bytes > S->cfg.hbm_budget)
        return fail(RS_ERANGE, "request needs %lld device bytes, budget is %lld",
                    (long long)bytes, (long long)S->cfg.hbm_budget);
    std::lock_guard<std::mutex> lk(S->mu);
    if ((int)S->queue.size() >= S->cfg.max_queue)
        return fail(RS_EBUSY, "queue full (%d requests)", S->cfg.max_queue);
    Req* q = new Req();
    q->ticket = S->next_ticket++;
    q->r = *req;
    q->r.n_lens = n;
    q->n_lens = n;
    q->bytes = bytes;
    q->t_submit = S->now();
    S->reqs[q->ticket] = q;
    S->queue.push_back(q->ticket);
    *ticket = q->ticket;
    S->cv.notify_all();
    return RS_OK;
}

int rs_server_step(rs_server* S, int32_t* progressed)
{
    clear_error();
    if (!S) return fail(RS_EINVAL, "null server");
    if (S->cfg.threaded) return fail(RS_EINVAL, "threaded servers step themselves");
    std::lock_guard<std::mutex> lk(S->mu);
    bool p = false;
    const int rc = step_locked(S, &p);
    if (progressed) *progressed = p ? 1 : 0;
    return rc;
}

int rs_server_poll(rs_server* S, int64_t ticket, rs_result* out)
{
    clear_error();
    if (!S || !out) return fail(RS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(RS_EINVAL, "unknown ticket %lld", (long long)ticket);
    fill_result(it->second, out);
    return RS_OK;
}

int rs_server_wait(rs_server* S, int64_t ticket, double timeout_s, rs_result* out)
{
    clear_error();
    if (!S) return fail(RS_EINVAL, "null server");
    const double deadline = S->now() + timeout_s;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return fail(RS_EINVAL, "unknown ticket %lld", (long long)ticket);
        if (terminal(it->second->state)) {
            if (out) fill_result(it->second, out);
            return RS_OK;
        }
        if (S->fatal) return fail(S->fatal, "server stopped on an error");
        if (S->now() >= deadline)
            return fail(RS_ETIMEOUT, "request %lld not finished after %.3f s", (long long)ticket,
                        timeout_s);
        if (S->cfg.threaded) {
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        } else {
            bool p = false;
            step_locked(S, &p);
            if (!p && !S->inflight.empty()) {
                cudaEvent_t ev = S->inflight.front().ev;
                lk.unlock();
                cudaEventSynchronize(ev);
                lk.lock();
            } else if (!p) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::milliseconds(1));
                lk.lock();
            }
        }
    }
}

int rs_server_cancel(rs_server* S, int64_t ticket)
{
    clear_error();
    if (!S) return fail(RS_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(RS_EINVAL, "unknown ticket %lld", (long long)ticket);
    if (!terminal(it->second->state)) it->second->cancel = true;
    S->cv.notify_all();
    return RS_OK;
}

int rs_server_release(rs_server* S, int64_t ticket)
{
    clear_error();
    if (!S) return fail(RS_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(RS_EINVAL, "unknown ticket %lld", (long long)ticket);
    Req* q = it->second;
    if (!terminal(q->state)) return fail(RS_EBUSY, "request %lld is not finished", (long long)ticket);
    free_device(S, q);
    delete q;
    S->reqs.erase(it);
    S->cv.notify_all();
    return RS_OK;
}

int rs_server_drain(rs_server* S, double timeout_s)
{
    clear_error();
    if (!S) return fail(RS_EINVAL, "null server");
    const double deadline = S->now() + timeout_s;
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        if (S->queue.empty() && S->running.empty() && S->inflight.empty()) return RS_OK;
        if (S->fatal) return fail(S->fatal, "server stopped on an error");
        if (S->now() >= deadline) return fail(RS_ETIMEOUT, "not drained after %.3f s", timeout_s);
        if (S->cfg.threaded) {
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        } else {
            bool p = false;
            step_locked(S, &p);
            if (!p && !S->inflight.empty()) {
                cudaEvent_t ev = S->inflight.front().ev;
                lk.unlock();
                cudaEventSynchronize(ev);
                lk.lock();
            } else if (!p) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::milliseconds(1));
                lk.lock();
            }
        }
    }
}

int rs_server_counters(rs_server* S, int64_t* out, int n_out)
{
    clear_error();
    if (!S || !out) return fail(RS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    const int64_t v[10] = {S->n_slices, S->n_launches, S->n_admitted, S->n_completed, S->n_failed,
                           S->n_cancelled, S->peak_bytes, S->bytes_used,
                           (int64_t)S->queue.size(), (int64_t)S->running.size()};
    for (int k = 0; k < n_out && k < 10; ++k) out[k] = v[k];
    return RS_OK;
}

double rs_server_clock(rs_server* S) { return S ? S->now() : 0.0; }

int rs_server_inject_alloc_failures(rs_server* S, int k)
{
    clear_error();
    if (!S || k < 0) return fail(RS_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(S->mu);
    S->inject_left = k;
    return RS_OK;
}

int rs_server_destroy(rs_server* S)
{
    clear_error();
    if (!S) return RS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->stream) cudaStreamSynchronize(S->stream);
    if (S->stream2) cudaStreamSynchronize(S->stream2);
    for (auto& kv : S->reqs) {
        free_device(S, kv.second);
        delete kv.second;
    }
    S->reqs.clear();
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (auto& sl : S->inflight)
        if (sl.ev) cudaEventDestroy(sl.ev);
    for (cudaEvent_t e : S->spare_events) cudaEventDestroy(e);
    if (S->ref_ev) cudaEventDestroy(S->ref_ev);
    if (S->h_stats) cudaFreeHost(S->h_stats);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->admit_ev) cudaEventDestroy(S->admit_ev);
    if (S->stream2) cudaStreamDestroy(S->stream2);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    return RS_OK;
}

}  // extern "C"
