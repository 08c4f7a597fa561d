// rs_noalloc.cu -- rs_shoot_map_host_noalloc: the host-buffer map call of
// rs_shoot_map_host without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need a map:
// code running under another framework's allocator (whose accounting a
// cudaMalloc would bypass), real-time or plugin hosts that forbid
// allocation on their call path, and processes whose device memory is
// fully reserved up front.  For them this entry point keeps its device
// working set -- the lens-list copy, the int32 count map, the float32
// magnification map and the statistics -- in one file-scope __device__
// array of fixed size, so a call makes no cudaMalloc/cudaFree and no
// allocating library call.  The paper has no counterpart; this is an
// interface choice of the library.
//
// Limits: npix <= RS_NOALLOC_MAX_NPIX and n_lens <= RS_NOALLOC_MAX_LENSES
// (the array is about 10 MB and stays resident on every device that loads
// the library until the process exits).  All calls share the array: each
// call zeroes the counts and statistics it uses and overwrites the rest, but
// two calls whose work overlaps on the GPU (different streams or host
// threads at the same time) race on it and corrupt each other's maps.
#include <cuda_runtime.h>
#include <string.h>

#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

constexpr size_t kLensBytes = align_up(3ull * RS_NOALLOC_MAX_LENSES * sizeof(double));
constexpr size_t kMapPixels = (size_t)RS_NOALLOC_MAX_NPIX * RS_NOALLOC_MAX_NPIX;
constexpr size_t kCountBytes = align_up(kMapPixels * sizeof(int32_t));
constexpr size_t kMuBytes = align_up(kMapPixels * sizeof(float));
constexpr size_t kStatBytes = align_up(RS_NSTATS * sizeof(int64_t));
constexpr size_t kScratchBytes = kLensBytes + kCountBytes + kMuBytes + kStatBytes;

// The whole device working set of rs_shoot_map_host_noalloc.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch on the current device.  The symbol's
// host-side name is only a stand-in, never a device address, so the address
// is looked up on every call (cheap; nothing cached can go stale after a
// device reset reloads the module).
int scratch_on_current_device(unsigned char** out)
{
    void* p = nullptr;
    const int rc = cuda_fail(cudaGetSymbolAddress(&p, g_noalloc_scratch),
                             "cudaGetSymbolAddress(no-alloc scratch)");
    if (rc) return rc;
    *out = static_cast<unsigned char*>(p);
    return RS_OK;
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" int rs_shoot_map_host_noalloc(const rs_macro* macro, const double* h_lens,
                                         int64_t n_lens, const rs_raygrid* grid,
                                         const rs_mapspec* map, const rs_options* opt,
                                         float* h_mu, int64_t* h_stats, void* stream)
{
    clear_error();
    if (!map) return fail(RS_EINVAL, "map is NULL");
    if (map->npix > RS_NOALLOC_MAX_NPIX)
        return fail(RS_ERANGE, "npix = %lld exceeds the no-allocation limit %d",
                    (long long)map->npix, RS_NOALLOC_MAX_NPIX);
    if (n_lens > RS_NOALLOC_MAX_LENSES)
        return fail(RS_ERANGE, "n_lens = %lld exceeds the no-allocation limit %d",
                    (long long)n_lens, RS_NOALLOC_MAX_LENSES);
    if (n_lens < 0 || (n_lens > 0 && !h_lens) || !h_mu || !h_stats)
        return fail(RS_EINVAL, "null host buffer or negative n_lens");
    if (!grid) return fail(RS_EINVAL, "grid is NULL");
    if (grid->n1 < 1 || grid->n2 < 1) return fail(RS_EINVAL, "empty ray grid");

    unsigned char* base = nullptr;
    int rc = scratch_on_current_device(&base);
    if (rc) return rc;
    double* d_lens = reinterpret_cast<double*>(base);
    int32_t* d_counts = reinterpret_cast<int32_t*>(base + kLensBytes);
    float* d_mu = reinterpret_cast<float*>(base + kLensBytes + kCountBytes);
    int64_t* d_stats = reinterpret_cast<int64_t*>(base + kLensBytes + kCountBytes + kMuBytes);

    rs_options o = {RS_PREC_COMPENSATED, 0, 0, 0};
    if (opt) o = *opt;
    if (o.precision == RS_PREC_REFINED)
        return fail(RS_EINVAL, "refined precision needs a scratch list; use rs_shoot_map_host");
    o.accumulate = 0;   // the shared array holds the previous call's map
    MapDesc d;
    ShapeInfo si;
    rc = prepare_map(macro, d_lens, n_lens, grid, map, o, &d, &si, false);
    if (rc) return rc;
    double navg = 0.0;
    if ((rc = rs_navg(grid, map, &navg))) return rc;

    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npx = map->npix * map->npix;
    if (n_lens > 0)
        rc = cuda_fail(cudaMemcpyAsync(d_lens, h_lens, (size_t)(3 * n_lens) * sizeof(double),
                                       cudaMemcpyHostToDevice, s),
                       "lens upload");
    if (!rc) rc = launch_fill_i32(d_counts, npx, 0, s);
    if (!rc) rc = launch_fill_i64(d_stats, RS_NSTATS, 0, s);
    if (!rc) {
        d.counts = d_counts;
        d.stats = reinterpret_cast<unsigned long long*>(d_stats);
        ShootExtra x = {0, nullptr, nullptr, nullptr};
        rc = launch_shoot(&d, 1, x, o.shape, o.precision, o.unit_mass != 0, MODE_BIN, s);
    }
    if (!rc) rc = launch_magnification(d_counts, npx, (float)(1.0 / navg), d_mu, s);
    if (!rc)
        rc = cuda_fail(cudaMemcpyAsync(h_mu, d_mu, (size_t)npx * sizeof(float),
                                       cudaMemcpyDeviceToHost, s),
                       "map download");
    if (!rc)
        rc = cuda_fail(cudaMemcpyAsync(h_stats, d_stats, RS_NSTATS * sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, s),
                       "stats download");
    const int sync_rc = cuda_fail(cudaStreamSynchronize(s), "stream synchronise");
    return rc ? rc : sync_rc;
}
