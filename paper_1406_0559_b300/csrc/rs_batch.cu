// rs_batch.cu -- the batching form: many maps of uneven lens counts and
// sizes in one persistent launch, an autotuner for the kernel shape, and
// CUDA-graph plans that replay a whole batch with one launch call.
//
// The survey runs (Sec. 3, Table 3) are batches of independent maps; here a
// batch of up to MAX_BATCH maps goes to the GPU as one persistent kernel
// whose work items are the ray tiles of all maps, heaviest maps (most lenses
// per tile) first so that the light tiles of small maps fill the tail.  The
// per-ray arithmetic is that of rs_shoot_map for the same shape, so a map
// comes out bit-identical alone or in a batch.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "rs_internal.cuh"

namespace rs {
namespace {

// ---- batched element-wise kernels (zero fill, magnification) -------------
struct FillArgs {
    int32_t n;
    int32_t pad_;
    int32_t* counts[MAX_BATCH];
    int64_t n_el[MAX_BATCH];
    int64_t* stats[MAX_BATCH];
};

struct MagArgs {
    int32_t n;
    int32_t pad_;
    const int32_t* counts[MAX_BATCH];
    float* mu[MAX_BATCH];
    int64_t n_el[MAX_BATCH];
    float inv_navg[MAX_BATCH];
};

// blockIdx.y selects the map; blocks of x stride over its elements
__global__ void fill_batch_kernel(const __grid_constant__ FillArgs a)
{
    const int m = blockIdx.y;
    int32_t* p = a.counts[m];
    const int64_t n = a.n_el[m];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n4 = ((reinterpret_cast<uintptr_t>(p) & 15) == 0) ? n / 4 : 0;
    int4* p4 = reinterpret_cast<int4*>(p);
    for (int64_t k = t0; k < n4; k += stride) p4[k] = make_int4(0, 0, 0, 0);
    for (int64_t k = 4 * n4 + t0; k < n; k += stride) p[k] = 0;
    if (t0 < RS_NSTATS && a.stats[m]) a.stats[m][t0] = 0;
}

__global__ void magnification_batch_kernel(const __grid_constant__ MagArgs a)
{
    const int m = blockIdx.y;
    const int32_t* c = a.counts[m];
    float* mu = a.mu[m];
    const float s = a.inv_navg[m];
    const int64_t n = a.n_el[m];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool al = ((reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(mu)) & 15) == 0;
    const int64_t n4 = al ? n / 4 : 0;
    const int4* c4 = reinterpret_cast<const int4*>(c);
    float4* m4 = reinterpret_cast<float4*>(mu);
    for (int64_t k = t0; k < n4; k += stride) {
        const int4 q = __ldcs(c4 + k);
        __stcs(m4 + k, make_float4((float)q.x * s, (float)q.y * s, (float)q.z * s, (float)q.w * s));
    }
    for (int64_t k = 4 * n4 + t0; k < n; k += stride) mu[k] = (float)c[k] * s;
}

int blocks_per_map(int64_t max_el, int n_maps)
{
    // enough CTAs in total to cover every SM several times
    int64_t want = (int64_t)num_sms() * 8 / (n_maps > 0 ? n_maps : 1);
    int64_t need = (max_el / 4 + 255) / 256;
    if (want < 4) want = 4;
    if (need < 1) need = 1;
    return (int)(need < want ? need : want);
}

// ---- validated batch ------------------------------------------------------
struct Prepared {
    std::vector<MapDesc> maps;     // in launch order (heaviest first)
    std::vector<int> order;        // job index of each launch slot
    std::vector<int64_t> npx;      // pixels per map (launch order)
    std::vector<float*> mu;        // magnification outputs (launch order)
    std::vector<float> inv_navg;
    rs_options o;
    int shape;
};

// Re-raise the current error with the job index in front.
int job_fail(int rc, int job)
{
    char msg[400];
    strncpy(msg, rs_last_error(), sizeof msg - 1);
    msg[sizeof msg - 1] = 0;
    return fail(rc, "job %d: %s", job, msg);
}

int prepare_batch(const rs_job* jobs, int n_jobs, const rs_options* opt, Prepared* P,
                  bool check_ptrs)
{
    if (n_jobs < 0) return fail(RS_EINVAL, "n_jobs < 0");
    if (n_jobs > 0 && !jobs) return fail(RS_EINVAL, "jobs is NULL");
    rs_options o = {RS_PREC_COMPENSATED, 0, 0, 0};
    if (opt) o = *opt;
    P->o = o;
    P->maps.clear();
    P->order.resize(n_jobs);
    std::iota(P->order.begin(), P->order.end(), 0);
    // heaviest maps first: lens count decides the cost of one tile
    std::stable_sort(P->order.begin(), P->order.end(),
                     [&](int a, int b) { return jobs[a].n_lens > jobs[b].n_lens; });
    for (int slot = 0; slot < n_jobs; ++slot) {
        const rs_job& j = jobs[P->order[slot]];
        MapDesc d;
        ShapeInfo si;
        int rc = prepare_map(&j.macro, j.d_lens, j.n_lens, &j.grid, &j.map, o, &d, &si,
                             check_ptrs);
        if (rc) return job_fail(rc, P->order[slot]);
        if (check_ptrs) {
            if ((rc = check_device_ptr(j.d_counts, "d_counts")) ||
                (rc = check_device_ptr(j.d_stats, "d_stats")) ||
                (j.d_mu && (rc = check_device_ptr(j.d_mu, "d_mu"))))
                return job_fail(rc, P->order[slot]);
        }
        if (!j.d_counts || !j.d_stats) return fail(RS_EINVAL, "job %d: null output", P->order[slot]);
        d.counts = j.d_counts;
        d.stats = reinterpret_cast<unsigned long long*>(j.d_stats);
        P->maps.push_back(d);
        P->npx.push_back(j.map.npix * j.map.npix);
        P->mu.push_back(j.d_mu);
        float inv = 0.f;
        if (j.d_mu) {
            double navg = 0.0;
            if ((rc = rs_navg(&j.grid, &j.map, &navg)))
                return job_fail(rc, P->order[slot]);
            inv = (float)(1.0 / navg);
        }
        P->inv_navg.push_back(inv);
    }
    return RS_OK;
}

// RS_PREC_REFINED: one stream-ordered allocation holding, ahead of the
// lists, {count, count3} per map and {work, work3} per launch group (zeroed;
// *head bytes), then every map's ray list (refine_capacity); the maps'
// list pointers are set.
int alloc_refine_lists(std::vector<MapDesc>& maps, cudaStream_t s, void** scratch,
                       unsigned long long** ctr, size_t* head_bytes)
{
    const int n = (int)maps.size();
    const int n_groups = (n + MAX_BATCH - 1) / MAX_BATCH;
    std::vector<int64_t> cap(n);
    size_t lists = 0;
    for (int k = 0; k < n; ++k) {
        cap[k] = refine_capacity(maps[k].g.n1 * maps[k].g.n2);
        lists += (size_t)refine_list_bytes(cap[k]);
    }
    const size_t head = ((size_t)(2 * n + 2 * n_groups) * sizeof(unsigned long long) + 15) &
                        ~size_t(15);
    const size_t bytes = head + lists;
    if (cudaMallocAsync(scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        *scratch = nullptr;
        return fail(RS_ENOMEM, "refinement lists (%zu bytes) could not be allocated", bytes);
    }
    *ctr = static_cast<unsigned long long*>(*scratch);
    *head_bytes = head;
    char* p = static_cast<char*>(*scratch) + head;
    for (int k = 0; k < n; ++k) {
        maps[k].refine_count = *ctr + 2 * k;
        maps[k].refine_ids = reinterpret_cast<int64_t*>(p);
        maps[k].refine_cap = cap[k];
        p += refine_list_bytes(cap[k]);
    }
    return cuda_fail(cudaMemsetAsync(*ctr, 0, head, s), "refinement counters");
}

// Enqueue fills + shoot launches + magnification for a prepared batch.
// RS_PREC_REFINED: every map gets a ray list (refine_capacity) in one
// stream-ordered allocation, and one second-pass
// launch per MAX_BATCH maps runs after all first passes.
int enqueue_batch(const Prepared& P, int shape, cudaStream_t s)
{
    const int n = (int)P.maps.size();
    const bool refined = P.o.precision == RS_PREC_REFINED;
    std::vector<MapDesc> maps(P.maps);
    void* scratch = nullptr;
    unsigned long long* ctr = nullptr;      // 2 list counters per map, 2 work counters per group
    size_t head = 0;
    int rc = RS_OK;
    if (refined && n > 0) {
        rc = alloc_refine_lists(maps, s, &scratch, &ctr, &head);
        if (rc && !scratch) return rc;
    }
    for (int c0 = 0; c0 < n && !rc; c0 += MAX_BATCH) {
        const int cn = std::min(MAX_BATCH, n - c0);
        if (!P.o.accumulate) {
            FillArgs f;
            memset(&f, 0, sizeof f);
            f.n = cn;
            int64_t mx = 0;
            for (int k = 0; k < cn; ++k) {
                f.counts[k] = maps[c0 + k].counts;
                f.n_el[k] = P.npx[c0 + k];
                f.stats[k] = reinterpret_cast<int64_t*>(maps[c0 + k].stats);
                mx = std::max(mx, f.n_el[k]);
            }
            dim3 grid(blocks_per_map(mx, cn), cn);
            fill_batch_kernel<<<grid, 256, 0, s>>>(f);
            if ((rc = cuda_fail(cudaGetLastError(), "batched fill launch"))) break;
        }
        // maps that fill the GPU get their own single-map launch; the others
        // share one persistent batched launch
        ShootExtra x = {0, nullptr, nullptr, nullptr};
        std::vector<MapDesc> shared;
        shared.reserve(cn);
        for (int k = 0; k < cn && !rc; ++k) {
            const MapDesc& m = maps[c0 + k];
            if (own_launch(m, shape, P.o.precision, P.o.unit_mass != 0))
                rc = launch_shoot(&m, 1, x, shape, P.o.precision, P.o.unit_mass != 0, MODE_BIN,
                                  s, 0, false);
            else
                shared.push_back(m);
        }
        if (!rc && !shared.empty())
            rc = launch_shoot(shared.data(), (int)shared.size(), x, shape, P.o.precision,
                              P.o.unit_mass != 0, MODE_BIN, s, 0, true);
    }
    for (int c0 = 0; refined && c0 < n && !rc; c0 += MAX_BATCH)
        rc = launch_refine(maps.data() + c0, std::min(MAX_BATCH, n - c0), ctr + 2 * n + 2 * (c0 / MAX_BATCH),
                           P.o.unit_mass != 0, s);
    for (int c0 = 0; c0 < n && !rc; c0 += MAX_BATCH) {
        const int cn = std::min(MAX_BATCH, n - c0);
        MagArgs m;
        memset(&m, 0, sizeof m);
        int64_t mx = 0;
        for (int k = 0; k < cn; ++k) {
            if (!P.mu[c0 + k]) continue;
            m.counts[m.n] = maps[c0 + k].counts;
            m.mu[m.n] = P.mu[c0 + k];
            m.n_el[m.n] = P.npx[c0 + k];
            m.inv_navg[m.n] = P.inv_navg[c0 + k];
            mx = std::max(mx, m.n_el[m.n]);
            ++m.n;
        }
        if (m.n == 0) continue;
        dim3 grid(blocks_per_map(mx, m.n), m.n);
        magnification_batch_kernel<<<grid, 256, 0, s>>>(m);
        rc = cuda_fail(cudaGetLastError(), "batched magnification launch");
    }
    if (scratch) cudaFreeAsync(scratch, s);
    return rc;
}

// ---- autotuner ------------------------------------------------------------
// Key: device, precision, unit masses, log2 bucket of the mean lens count,
// log2 bucket of the mean rays per map, number of maps (log2 bucket).
typedef std::tuple<int, int, int, int, int, int> TuneKey;
std::map<TuneKey, int> g_tuned;
std::mutex g_tune_mu;

TuneKey tune_key(const rs_job* jobs, int n, const rs_options& o)
{
    int dev = 0;
    cudaGetDevice(&dev);
    double sn = 0, sr = 0;
    for (int k = 0; k < n; ++k) {
        sn += (double)jobs[k].n_lens;
        sr += (double)jobs[k].grid.n1 * (double)jobs[k].grid.n2;
    }
    const int bn = n ? (int)floor(log2(sn / n + 1.0)) : 0;
    const int br = n ? (int)floor(log2(sr / n + 1.0)) : 0;
    const int bm = (int)floor(log2((double)n + 1.0));
    return TuneKey(dev, o.precision, o.unit_mass, bn, br, bm);
}

}  // namespace

int launch_magnification_batch(const int32_t* const* counts, float* const* mu,
                               const int64_t* n_el, const float* inv_navg, int n, cudaStream_t s)
{
    int rc = RS_OK;
    for (int c0 = 0; c0 < n && !rc; c0 += MAX_BATCH) {
        MagArgs m;
        memset(&m, 0, sizeof m);
        int64_t mx = 0;
        for (int k = c0; k < n && k < c0 + MAX_BATCH; ++k) {
            m.counts[m.n] = counts[k];
            m.mu[m.n] = mu[k];
            m.n_el[m.n] = n_el[k];
            m.inv_navg[m.n] = inv_navg[k];
            mx = std::max(mx, n_el[k]);
            ++m.n;
        }
        dim3 grid(blocks_per_map(mx, m.n), m.n);
        magnification_batch_kernel<<<grid, 256, 0, s>>>(m);
        rc = cuda_fail(cudaGetLastError(), "batched magnification launch");
    }
    return rc;
}

int shoot_batch_impl(const rs_job* jobs, int n_jobs, const rs_options* opt, cudaStream_t s)
{
    Prepared P;
    int rc = prepare_batch(jobs, n_jobs, opt, &P, true);
    if (rc || n_jobs == 0) return rc;
    int shape = P.o.shape;
    if (shape == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(jobs, n_jobs, P.o));
        shape = it != g_tuned.end() ? it->second : 0;
    }
    return enqueue_batch(P, shape, s);
}

}  // namespace rs

using namespace rs;

struct rs_plan {
    Prepared P;
    int shape;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

int rs_shoot_batch(const rs_job* jobs, int n_jobs, const rs_options* opt, void* stream)
{
    clear_error();
    return shoot_batch_impl(jobs, n_jobs, opt, (cudaStream_t)stream);
}

int rs_autotune(const rs_job* jobs, int n_jobs, const rs_options* opt, int32_t* best_shape,
                float* ms_per_gint, int n_out, void* stream)
{
    clear_error();
    if (!best_shape) return fail(RS_EINVAL, "best_shape is NULL");
    Prepared P;
    int rc = prepare_batch(jobs, n_jobs, opt, &P, true);
    if (rc) return rc;
    if (n_jobs == 0) return fail(RS_EINVAL, "nothing to tune");
    cudaStream_t s = (cudaStream_t)stream;
    int cand[32];
    const int nc = batch_candidates(P.o.precision, cand, 32);
    const int tprec = P.o.precision;
    // the refined form's candidates are timed on their first pass (the
    // compensated sum, the error bound and the listing: ~97% of a map), with
    // ray lists allocated as for a batch and their counters reset per run
    std::vector<MapDesc> maps(P.maps);
    void* scratch = nullptr;
    unsigned long long* ctr = nullptr;
    size_t head = 0;
    if (tprec == RS_PREC_REFINED) {
        rc = alloc_refine_lists(maps, s, &scratch, &ctr, &head);
        if (rc) {
            if (scratch) cudaFreeAsync(scratch, s);
            return rc;
        }
    }
    // sample: the first `cap` tiles of every map, about four waves in total
    const int64_t target = (int64_t)num_sms() * 4;
    int64_t cap = target / n_jobs;
    if (cap < 1) cap = 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.f;
    int best_k = -1;
    for (int c = 0; c < nc && !rc; ++c) {
        ShapeInfo si;
        shape_info(cand[c], tprec, &si);
        double inter = 0.0;   // interactions in the sample
        for (size_t k = 0; k < maps.size(); ++k) {
            const MapDesc& d = maps[k];
            const int64_t t1 = (d.g.n1 + si.tx - 1) / si.tx;
            const int64_t t2 = (d.g.n2 + si.ty - 1) / si.ty;
            const int64_t nt = std::min(cap, t1 * t2);
            inter += (double)nt * si.tx * si.ty * (double)d.n_lens;
        }
        ShootExtra x = {0, nullptr, nullptr, nullptr};
        float ms = 0.f;
        for (int rep = 0; rep < 2 && !rc; ++rep) {   // first run warms up
            if (ctr) rc = cuda_fail(cudaMemsetAsync(ctr, 0, head, s), "refinement counters");
            for (size_t c0 = 0; c0 < maps.size() && !rc; c0 += MAX_BATCH) {
                const int cn = (int)std::min<size_t>(MAX_BATCH, maps.size() - c0);
                if (rep == 1 && c0 == 0) cudaEventRecord(e0, s);
                rc = launch_shoot(maps.data() + c0, cn, x, cand[c], tprec,
                                  P.o.unit_mass != 0, MODE_BIN, s, cap, true);
            }
        }
        if (rc) break;
        cudaEventRecord(e1, s);
        if ((rc = cuda_fail(cudaEventSynchronize(e1), "autotune timing"))) break;
        cudaEventElapsedTime(&ms, e0, e1);
        const float per_gint = (float)(ms / (inter / 1e9));
        if (ms_per_gint && c < n_out) ms_per_gint[c] = per_gint;
        if (best_k < 0 || per_gint < best) {
            best = per_gint;
            best_k = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (scratch) cudaFreeAsync(scratch, s);
    if (rc) return rc;
    *best_shape = cand[best_k];
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[tune_key(jobs, n_jobs, P.o)] = cand[best_k];
    return RS_OK;
}

int rs_tune_candidates(int precision, int32_t* shapes, int max)
{
    clear_error();
    if (!shapes || max < 1) return fail(RS_EINVAL, "bad output buffer");
    if (precision < RS_PREC_FP32 || precision > RS_PREC_REFINED)
        return fail(RS_EINVAL, "precision %d is not one of RS_PREC_*", precision);
    int tmp[64];
    const int n = batch_candidates(precision, tmp, 64);
    for (int k = 0; k < n && k < max; ++k) shapes[k] = tmp[k];
    return n;
}

int rs_plan_create(const rs_job* jobs, int n_jobs, const rs_options* opt, rs_plan** out)
{
    clear_error();
    if (!out) return fail(RS_EINVAL, "out is NULL");
    *out = nullptr;
    rs_plan* p = new rs_plan();
    p->graph = nullptr;
    p->exec = nullptr;
    int rc = prepare_batch(jobs, n_jobs, opt, &p->P, true);
    if (!rc && n_jobs == 0) rc = fail(RS_EINVAL, "empty plan");
    int shape = p->P.o.shape;
    if (!rc && shape == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(jobs, n_jobs, p->P.o));
        shape = it != g_tuned.end() ? it->second : 0;
    }
    p->shape = shape;
    cudaStream_t cs = nullptr;
    if (!rc) rc = cuda_fail(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "plan stream");
    if (!rc) {
        // resolve occupancy, SM count and kernels before capture: the
        // capture then holds only launches
        rc = prime_launch(shape, p->P.o.precision, p->P.o.unit_mass != 0, true);
        // the single-map kernel too, for maps launched on their own (not every
        // shape has one; then every map goes through the batched kernel)
        if (!rc && prime_launch(shape, p->P.o.precision, p->P.o.unit_mass != 0, false) != RS_OK)
            clear_error();
        if (!rc)
            rc = cuda_fail(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal),
                           "begin capture");
        if (!rc) {
            int erc = enqueue_batch(p->P, shape, cs);
            cudaGraph_t g = nullptr;
            int crc = cuda_fail(cudaStreamEndCapture(cs, &g), "end capture");
            rc = erc ? erc : crc;
            p->graph = g;
        }
    }
    if (!rc) rc = cuda_fail(cudaGraphInstantiate(&p->exec, p->graph, 0), "graph instantiate");
    if (cs) cudaStreamDestroy(cs);
    if (rc) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        return rc;
    }
    *out = p;
    return RS_OK;
}

int rs_plan_shape(const rs_plan* p, int32_t* shape)
{
    clear_error();
    if (!p || !shape) return fail(RS_EINVAL, "null argument");
    *shape = p->shape;
    return RS_OK;
}

int rs_plan_launch(rs_plan* p, void* stream)
{
    clear_error();
    if (!p || !p->exec) return fail(RS_EINVAL, "invalid plan");
    return cuda_fail(cudaGraphLaunch(p->exec, (cudaStream_t)stream), "graph launch");
}

int rs_plan_destroy(rs_plan* p)
{
    clear_error();
    if (!p) return RS_OK;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
    return RS_OK;
}

}  // extern "C"
