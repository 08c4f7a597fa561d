// rs_api.cu -- the extern "C" boundary of librs_b300.so (include/rs.h).
//
// Argument checking, geometry set-up in FP64 on the host, pointer-kind
// checks (a host pointer handed to a kernel would fault the device, so it is
// rejected before any launch), and dispatch to the kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rs_internal.cuh"

namespace rs {

namespace {
thread_local char g_err[512] = "";
}

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return RS_OK;
    return fail(e == cudaErrorMemoryAllocation ? RS_ENOMEM : RS_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

void clear_error() { g_err[0] = 0; }

int num_sms()
{
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cache[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

namespace {
bool finite_pos(double v) { return isfinite(v) && v > 0.0; }
}  // namespace

// Device or managed memory?  Anything else is refused before a launch.
int check_device_ptr(const void* p, const char* name)
{
    if (!p) return fail(RS_EINVAL, "%s is NULL", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RS_EINVAL, "%s is not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(RS_EINVAL, "%s is not device memory (host pointers are not accepted here)", name);
    return RS_OK;
}

namespace {

int check_grid(const rs_raygrid* g)
{
    if (!g) return fail(RS_EINVAL, "grid is NULL");
    if (g->n1 < 0 || g->n2 < 0) return fail(RS_EINVAL, "ray counts must be >= 0");
    if (!isfinite(g->c1) || !isfinite(g->c2)) return fail(RS_EINVAL, "grid centre not finite");
    if (!finite_pos(g->half1) || !finite_pos(g->half2))
        return fail(RS_EINVAL, "grid half-widths must be finite and > 0");
    if (g->n1 > 0 && g->n2 > RS_MAX_RAYS / g->n1)
        return fail(RS_ERANGE, "n1 * n2 = %lld * %lld exceeds %lld rays per call", (long long)g->n1,
                    (long long)g->n2, (long long)RS_MAX_RAYS);
    return RS_OK;
}

int check_map(const rs_mapspec* m)
{
    if (!m) return fail(RS_EINVAL, "map is NULL");
    if (m->npix < 1 || m->npix > RS_MAX_NPIX)
        return fail(RS_ERANGE, "npix = %lld outside [1, %d]", (long long)m->npix, RS_MAX_NPIX);
    if (!isfinite(m->c1) || !isfinite(m->c2)) return fail(RS_EINVAL, "map centre not finite");
    if (!finite_pos(m->width)) return fail(RS_EINVAL, "map width must be finite and > 0");
    return RS_OK;
}

int check_macro(const rs_macro* mc)
{
    if (!mc) return fail(RS_EINVAL, "macro is NULL");
    if (!isfinite(mc->kappa_s) || !isfinite(mc->gamma))
        return fail(RS_EINVAL, "kappa_s and gamma must be finite");
    return RS_OK;
}

rs_options resolve(const rs_options* opt)
{
    rs_options o = {RS_PREC_COMPENSATED, 0, 0, 0};
    if (opt) o = *opt;
    return o;
}

int check_options(const rs_options& o)
{
    if (o.precision != RS_PREC_FP32 && o.precision != RS_PREC_COMPENSATED &&
        o.precision != RS_PREC_DOUBLE_SINGLE && o.precision != RS_PREC_REFINED)
        return fail(RS_EINVAL, "precision %d unknown", o.precision);
    if (o.unit_mass != 0 && o.unit_mass != 1) return fail(RS_EINVAL, "unit_mass must be 0 or 1");
    if (o.accumulate != 0 && o.accumulate != 1) return fail(RS_EINVAL, "accumulate must be 0 or 1");
    ShapeInfo si;
    return shape_info(o.shape, o.precision, &si);
}

}  // namespace

// Shared argument checks and geometry of one map (rs_shoot_map,
// rs_shoot_tiles, rs_shoot_batch).  check_lens: verify d_lens is device
// memory (skipped for buffers the library allocated itself).
int prepare_map(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                const rs_raygrid* grid, const rs_mapspec* map, const rs_options& o, MapDesc* d,
                ShapeInfo* si, bool check_lens)
{
    int rc;
    if ((rc = check_macro(macro)) || (rc = check_grid(grid)) || (rc = check_map(map)) ||
        (rc = check_options(o)))
        return rc;
    if (n_lens < 0 || n_lens > RS_MAX_LENSES)
        return fail(RS_ERANGE, "n_lens = %lld outside [0, %lld]", (long long)n_lens,
                    (long long)RS_MAX_LENSES);
    if (n_lens > 0 && check_lens && (rc = check_device_ptr(d_lens, "d_lens"))) return rc;
    if (n_lens > 0 && !d_lens) return fail(RS_EINVAL, "d_lens is NULL");
    shape_info(o.shape, o.precision, si);

    memset(d, 0, sizeof *d);
    Geometry& g = d->g;
    g.x0_1 = grid->c1 - grid->half1;
    g.x0_2 = grid->c2 - grid->half2;
    g.d1 = grid->n1 > 0 ? 2.0 * grid->half1 / (double)grid->n1 : 0.0;
    g.d2 = grid->n2 > 0 ? 2.0 * grid->half2 / (double)grid->n2 : 0.0;
    g.n1 = grid->n1;
    g.n2 = grid->n2;
    g.one_m_g = 1.0 - macro->gamma;
    g.one_p_g = 1.0 + macro->gamma;
    g.kappa_s = macro->kappa_s;
    g.y0_1 = map->c1 - map->width / 2.0;
    g.y0_2 = map->c2 - map->width / 2.0;
    g.inv_w = 1.0 / (map->width / (double)map->npix);
    g.npix = (int32_t)map->npix;
    // ray spacings off the 2^-12 grid need the coherent-rounding correction
    auto on_grid = [](double d) { const double v = d * 4096.0; return v == floor(v); };
    g.flags = ((grid->n1 > 0 && !on_grid(g.d1)) || (grid->n2 > 0 && !on_grid(g.d2))) ? GEO_COHERENT : 0;
    d->lx = d_lens;
    d->ly = d_lens ? d_lens + n_lens : nullptr;
    d->lm = d_lens ? d_lens + 2 * n_lens : nullptr;
    d->n_lens = (int32_t)n_lens;
    d->tiles1 = grid->n1 > 0 ? (grid->n1 + si->tx - 1) / si->tx : 0;
    return RS_OK;
}

}  // namespace rs

using namespace rs;

extern "C" {

const char* rs_version(void) { return "rs_b300 1.0 sm_103a"; }

const char* rs_last_error(void) { return g_err; }

int rs_lens_count(double kappa_star, double radius, double mean_mass, int64_t* n)
{
    clear_error();
    if (!n) return fail(RS_EINVAL, "n is NULL");
    if (!isfinite(kappa_star) || kappa_star < 0 || !isfinite(radius) || radius < 0 ||
        !finite_pos(mean_mass))
        return fail(RS_EINVAL, "kappa_star, radius >= 0 and mean_mass > 0 required");
    const double pi = 3.14159265358979323846;
    const double area = pi * radius * radius;               // disk of radius R
    const double v = kappa_star * area / (pi * mean_mass);  // Eq. 3
    if (!(v < 9.0e18)) return fail(RS_ERANGE, "lens count overflows");
    *n = (int64_t)floor(v + 0.5);
    return RS_OK;
}

int rs_navg(const rs_raygrid* grid, const rs_mapspec* map, double* navg)
{
    clear_error();
    int rc;
    if ((rc = check_grid(grid)) || (rc = check_map(map))) return rc;
    if (!navg) return fail(RS_EINVAL, "navg is NULL");
    if (grid->n1 < 1 || grid->n2 < 1) return fail(RS_EINVAL, "empty ray grid has no N_avg");
    const double d1 = 2.0 * grid->half1 / (double)grid->n1;
    const double d2 = 2.0 * grid->half2 / (double)grid->n2;
    const double w = map->width / (double)map->npix;
    *navg = (w / d1) * (w / d2);
    return RS_OK;
}

int rs_make_lenses(const rs_lensfield* f, uint64_t seed, double* d_lens, int64_t n, void* stream)
{
    clear_error();
    if (!f) return fail(RS_EINVAL, "field is NULL");
    if (n < 0 || n > RS_MAX_LENSES) return fail(RS_ERANGE, "n = %lld out of range", (long long)n);
    if (!isfinite(f->radius) || f->radius < 0) return fail(RS_EINVAL, "radius must be >= 0");
    if (f->mass_model != RS_MASS_UNIT && f->mass_model != RS_MASS_SALPETER)
        return fail(RS_EINVAL, "mass_model %d unknown", f->mass_model);
    if (f->mass_model == RS_MASS_SALPETER &&
        !(finite_pos(f->m_lo) && isfinite(f->m_hi) && f->m_hi > f->m_lo && isfinite(f->slope) &&
          f->slope != 1.0))
        return fail(RS_EINVAL, "Salpeter needs 0 < m_lo < m_hi and slope != 1");
    if (n == 0) return RS_OK;
    int rc = check_device_ptr(d_lens, "d_lens");
    if (rc) return rc;
    return launch_make_lenses(f, seed, d_lens, n, (cudaStream_t)stream);
}

int rs_tile_shape(const rs_options* opt, int64_t* tx, int64_t* ty)
{
    clear_error();
    if (!tx || !ty) return fail(RS_EINVAL, "tx/ty is NULL");
    rs_options o = resolve(opt);
    int rc = check_options(o);
    if (rc) return rc;
    ShapeInfo si;
    shape_info(o.shape, o.precision, &si);
    *tx = si.tx;
    *ty = si.ty;
    return RS_OK;
}

int rs_shape_sum(const rs_options* opt, int32_t* fold_lenses, int32_t* unroll)
{
    clear_error();
    if (!fold_lenses || !unroll) return fail(RS_EINVAL, "fold_lenses/unroll is NULL");
    rs_options o = resolve(opt);
    int rc = check_options(o);
    if (rc) return rc;
    ShapeInfo si;
    shape_info(o.shape, o.precision, &si);
    *fold_lenses = si.fold_lenses;
    *unroll = si.unroll;
    return RS_OK;
}

}  // extern "C"

namespace rs {
namespace {
// Dump mode (rs_shoot_tiles, rs_debug_rays): per-ray results of the listed
// tiles; RS_PREC_REFINED lists the rays near pixel edges with their dump
// slots and its second pass rewrites them (every ray of the tiles fits the
// list, so none keeps its compensated result).
// RS_PREC_REFINED: y_first (optional) receives every ray's first-pass image
// before the second and third passes overwrite the listed rays'.
int shoot_dump(MapDesc& d, ShootExtra x, const rs_options& o, const ShapeInfo& si, cudaStream_t s,
               double* y_first = nullptr)
{
    if (o.precision != RS_PREC_REFINED)
        return launch_shoot(&d, 1, x, o.shape, o.precision, o.unit_mass != 0, MODE_DUMP, s);
    const int64_t cap = x.n_work * si.tx * si.ty;
    void* scratch = nullptr;
    // {count, count3, work, work3}, the lists, the dump slots
    const size_t bytes = 4 * sizeof(unsigned long long) + (size_t)refine_list_bytes(cap) +
                         (size_t)cap * sizeof(int64_t);
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(RS_ENOMEM, "refinement list (%zu bytes) could not be allocated", bytes);
    }
    unsigned long long* ctr = static_cast<unsigned long long*>(scratch);
    d.refine_count = ctr;
    d.refine_ids = reinterpret_cast<int64_t*>(ctr + 4);
    d.refine_cap = cap;
    x.refine_slots = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(d.refine_ids) +
                                                refine_list_bytes(cap));
    int rc = cuda_fail(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), s), "refine counters");
    if (!rc) rc = launch_shoot(&d, 1, x, o.shape, o.precision, o.unit_mass != 0, MODE_DUMP, s);
    if (!rc && y_first)
        rc = cuda_fail(cudaMemcpyAsync(y_first, x.dump_y, (size_t)cap * 2 * sizeof(double),
                                       cudaMemcpyDeviceToDevice, s),
                       "first-pass image copy");
    if (!rc) rc = launch_refine(&d, 1, ctr + 2, o.unit_mass != 0, s, &x);
    cudaFreeAsync(scratch, s);
    return rc;
}

// The map's ray tiles [tile0, tile0 + n_tiles) (n_tiles < 0: to the end).
int shoot_map_impl(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                   const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                   int32_t* d_counts, int64_t* d_stats, void* stream, bool check_ptrs,
                   int64_t tile0 = 0, int64_t n_tiles = -1)
{
    rs_options o = resolve(opt);
    MapDesc d;
    ShapeInfo si;
    int rc = prepare_map(macro, d_lens, n_lens, grid, map, o, &d, &si, check_ptrs);
    if (rc) return rc;
    const int64_t tiles = grid->n1 > 0 && grid->n2 > 0
                              ? ((grid->n1 + si.tx - 1) / si.tx) * ((grid->n2 + si.ty - 1) / si.ty)
                              : 0;
    if (tile0 < 0 || tile0 > tiles) return fail(RS_ERANGE, "tile0 %lld outside [0, %lld]",
                                                (long long)tile0, (long long)tiles);
    if (n_tiles < 0 || n_tiles > tiles - tile0) n_tiles = tiles - tile0;
    d.tile0 = tile0;
    d.tile_count = n_tiles;
    if (check_ptrs && ((rc = check_device_ptr(d_counts, "d_counts")) ||
                       (rc = check_device_ptr(d_stats, "d_stats"))))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!o.accumulate) {
        if ((rc = launch_fill_i32(d_counts, map->npix * map->npix, 0, s))) return rc;
        if ((rc = launch_fill_i64(d_stats, RS_NSTATS, 0, s))) return rc;
    }
    d.counts = d_counts;
    d.stats = reinterpret_cast<unsigned long long*>(d_stats);
    ShootExtra x = {0, nullptr, nullptr, nullptr};
    if (n_tiles == 0) return RS_OK;
    if (o.precision != RS_PREC_REFINED)
        return launch_shoot(&d, 1, x, o.shape, o.precision, o.unit_mass != 0, MODE_BIN, s);
    // refined: the compensated pass lists the rays near pixel edges, the
    // double-single pass bins them; the list and its two counters come from
    // the stream-ordered allocator and go back to it in stream order
    const int64_t rays = std::min(grid->n1 * grid->n2, n_tiles * si.tx * si.ty);
    if (rays == 0) return RS_OK;
    const int64_t cap = refine_capacity(rays);
    void* scratch = nullptr;
    // {count, count3, work, work3}, then the lists
    const size_t bytes = 4 * sizeof(unsigned long long) + (size_t)refine_list_bytes(cap);
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(RS_ENOMEM, "refinement list (%zu bytes) could not be allocated", bytes);
    }
    unsigned long long* ctr = static_cast<unsigned long long*>(scratch);
    d.refine_count = ctr;
    d.refine_ids = reinterpret_cast<int64_t*>(ctr + 4);
    d.refine_cap = cap;
    int rc2 = cuda_fail(cudaMemsetAsync(ctr, 0, 4 * sizeof(unsigned long long), s), "refine counters");
    if (!rc2) rc2 = launch_shoot(&d, 1, x, o.shape, o.precision, o.unit_mass != 0, MODE_BIN, s);
    if (!rc2) rc2 = launch_refine(&d, 1, ctr + 2, o.unit_mass != 0, s);
    cudaFreeAsync(scratch, s);
    return rc2;
}
}  // namespace
}  // namespace rs

extern "C" {

int rs_shoot_map(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                 const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                 int32_t* d_counts, int64_t* d_stats, void* stream)
{
    clear_error();
    return shoot_map_impl(macro, d_lens, n_lens, grid, map, opt, d_counts, d_stats, stream, true);
}

int rs_shoot_map_range(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                       const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                       int64_t tile0, int64_t n_tiles, int32_t* d_counts, int64_t* d_stats,
                       int64_t* n_tiles_total, void* stream)
{
    clear_error();
    rs_options o = resolve(opt);
    o.accumulate = 1;                  // a range adds to what earlier ranges counted
    if (n_tiles_total) {
        int64_t tx = 0, ty = 0;
        int rc = rs_tile_shape(&o, &tx, &ty);
        if (rc) return rc;
        *n_tiles_total = grid && grid->n1 > 0 && grid->n2 > 0
                             ? ((grid->n1 + tx - 1) / tx) * ((grid->n2 + ty - 1) / ty)
                             : 0;
    }
    if (n_tiles < 0) return fail(RS_EINVAL, "n_tiles < 0");
    return shoot_map_impl(macro, d_lens, n_lens, grid, map, &o, d_counts, d_stats, stream, true,
                          tile0, n_tiles);
}

int rs_shoot_tiles(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                   const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                   const int64_t* d_tile_ids, int64_t n_tiles, double* d_y, int32_t* d_pix,
                   void* stream)
{
    clear_error();
    rs_options o = resolve(opt);
    MapDesc d;
    ShapeInfo si;
    int rc = prepare_map(macro, d_lens, n_lens, grid, map, o, &d, &si, true);
    if (rc) return rc;
    if (n_tiles < 0) return fail(RS_EINVAL, "n_tiles < 0");
    if (n_tiles == 0) return RS_OK;
    if ((rc = check_device_ptr(d_tile_ids, "d_tile_ids")) || (rc = check_device_ptr(d_y, "d_y")) ||
        (rc = check_device_ptr(d_pix, "d_pix")))
        return rc;
    ShootExtra x = {n_tiles, d_tile_ids, d_y, d_pix};
    return shoot_dump(d, x, o, si, (cudaStream_t)stream);
}

int rs_shoot_tiles_band(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                        const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                        const int64_t* d_tile_ids, int64_t n_tiles, float* d_band,
                        double* d_y_first, void* stream)
{
    clear_error();
    rs_options o = resolve(opt);
    if (o.precision != RS_PREC_REFINED)
        return fail(RS_EINVAL, "rs_shoot_tiles_band needs opt->precision = RS_PREC_REFINED");
    MapDesc d;
    ShapeInfo si;
    int rc = prepare_map(macro, d_lens, n_lens, grid, map, o, &d, &si, true);
    if (rc) return rc;
    if (n_tiles < 0) return fail(RS_EINVAL, "n_tiles < 0");
    if (n_tiles == 0) return RS_OK;
    if ((rc = check_device_ptr(d_tile_ids, "d_tile_ids")) || (rc = check_device_ptr(d_band, "d_band")) ||
        (d_y_first && (rc = check_device_ptr(d_y_first, "d_y_first"))))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t per = si.tx * si.ty;
    void* scratch = nullptr;
    const size_t bytes = (size_t)n_tiles * per * (2 * sizeof(double) + 2 * sizeof(int32_t));
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(RS_ENOMEM, "band scratch (%zu bytes) could not be allocated", bytes);
    }
    double* d_y = static_cast<double*>(scratch);
    int32_t* d_pix = reinterpret_cast<int32_t*>(d_y + 2 * n_tiles * per);
    ShootExtra x = {n_tiles, d_tile_ids, d_y, d_pix};
    x.dump_band = d_band;
    rc = shoot_dump(d, x, o, si, s, d_y_first);
    cudaFreeAsync(scratch, s);
    return rc;
}

int rs_debug_rays(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                  const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                  const int64_t* h_ray_ids, int64_t n, double* h_y, int32_t* h_pix, void* stream)
{
    clear_error();
    rs_options o = resolve(opt);
    MapDesc d;
    ShapeInfo si;
    int rc = prepare_map(macro, d_lens, n_lens, grid, map, o, &d, &si, true);
    if (rc) return rc;
    if (n < 0) return fail(RS_EINVAL, "n < 0");
    if (n == 0) return RS_OK;
    if (!h_ray_ids || !h_y || !h_pix) return fail(RS_EINVAL, "NULL ray list or output");
    const int64_t n1 = grid->n1, n2 = grid->n2, tx = si.tx, ty = si.ty;
    const int64_t t1 = (n1 + tx - 1) / tx;
    // the distinct tiles holding the rays, and each ray's slot in the dump
    std::vector<int64_t> tiles;
    std::vector<int64_t> slot(n);
    {
        std::vector<std::pair<int64_t, int64_t>> tk(n);
        for (int64_t k = 0; k < n; ++k) {
            const int64_t id = h_ray_ids[k];
            if (id < 0 || id >= n1 * n2)
                return fail(RS_EINVAL, "ray id %lld outside [0, %lld)", (long long)id,
                            (long long)(n1 * n2));
            const int64_t i = id % n1, j = id / n1;
            tk[k] = {(j / ty) * t1 + i / tx, k};
        }
        std::sort(tk.begin(), tk.end());
        for (int64_t k = 0; k < n; ++k) {
            if (tiles.empty() || tiles.back() != tk[k].first) tiles.push_back(tk[k].first);
            const int64_t id = h_ray_ids[tk[k].second];
            const int64_t a = (id % n1) % tx, b = (id / n1) % ty;
            slot[tk[k].second] = (int64_t)(tiles.size() - 1) * tx * ty + b * tx + a;
        }
    }
    const int64_t nt = (int64_t)tiles.size(), per = tx * ty;
    cudaStream_t s = (cudaStream_t)stream;
    void* scratch = nullptr;
    const size_t bytes = nt * sizeof(int64_t) + (size_t)nt * per * (2 * sizeof(double) +
                                                                     2 * sizeof(int32_t));
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(RS_ENOMEM, "debug scratch (%zu bytes) could not be allocated", bytes);
    }
    int64_t* d_ids = static_cast<int64_t*>(scratch);
    double* d_y = reinterpret_cast<double*>(d_ids + nt);
    int32_t* d_pix = reinterpret_cast<int32_t*>(d_y + 2 * nt * per);
    std::vector<double> y(2 * nt * per);
    std::vector<int32_t> pix(2 * nt * per);
    rc = cuda_fail(cudaMemcpyAsync(d_ids, tiles.data(), nt * sizeof(int64_t),
                                   cudaMemcpyHostToDevice, s), "tile list copy");
    if (!rc) {
        ShootExtra x = {nt, d_ids, d_y, d_pix};
        rc = shoot_dump(d, x, o, si, s);
    }
    if (!rc)
        rc = cuda_fail(cudaMemcpyAsync(y.data(), d_y, y.size() * sizeof(double),
                                       cudaMemcpyDeviceToHost, s), "result copy");
    if (!rc)
        rc = cuda_fail(cudaMemcpyAsync(pix.data(), d_pix, pix.size() * sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, s), "result copy");
    cudaFreeAsync(scratch, s);
    if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "debug sync");
    if (rc) return rc;
    for (int64_t k = 0; k < n; ++k) {
        h_y[2 * k] = y[2 * slot[k]];
        h_y[2 * k + 1] = y[2 * slot[k] + 1];
        h_pix[2 * k] = pix[2 * slot[k]];
        h_pix[2 * k + 1] = pix[2 * slot[k] + 1];
    }
    return RS_OK;
}

int rs_magnification(const int32_t* d_counts, const rs_raygrid* grid, const rs_mapspec* map,
                     float* d_mu, void* stream)
{
    clear_error();
    double navg = 0.0;
    int rc = rs_navg(grid, map, &navg);
    if (rc) return rc;
    if ((rc = check_device_ptr(d_counts, "d_counts")) || (rc = check_device_ptr(d_mu, "d_mu")))
        return rc;
    return launch_magnification(d_counts, map->npix * map->npix, (float)(1.0 / navg), d_mu,
                                (cudaStream_t)stream);
}

int rs_shoot_map_host(const rs_macro* macro, const double* h_lens, int64_t n_lens,
                      const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                      float* h_mu, int64_t* h_stats, void* stream)
{
    clear_error();
    int rc;
    if ((rc = check_macro(macro)) || (rc = check_grid(grid)) || (rc = check_map(map))) return rc;
    if (n_lens < 0 || (n_lens > 0 && !h_lens) || !h_mu || !h_stats)
        return fail(RS_EINVAL, "null host buffer or negative n_lens");
    if (grid->n1 < 1 || grid->n2 < 1) return fail(RS_EINVAL, "empty ray grid");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npx = map->npix * map->npix;
    double* d_lens = nullptr;
    int32_t* d_counts = nullptr;
    int64_t* d_stats = nullptr;
    float* d_mu = nullptr;
    cudaError_t e = cudaSuccess;
    if (n_lens > 0) e = cudaMallocAsync((void**)&d_lens, (size_t)(3 * n_lens) * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_counts, (size_t)npx * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_stats, RS_NSTATS * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_mu, (size_t)npx * sizeof(float), s);
    if (e == cudaSuccess && n_lens > 0)
        e = cudaMemcpyAsync(d_lens, h_lens, (size_t)(3 * n_lens) * sizeof(double),
                            cudaMemcpyHostToDevice, s);
    rc = cuda_fail(e, "device buffers / lens upload");
    if (!rc)
        rc = shoot_map_impl(macro, d_lens, n_lens, grid, map, opt, d_counts, d_stats, stream, false);
    double navg = 0.0;
    if (!rc) rc = rs_navg(grid, map, &navg);
    if (!rc) rc = launch_magnification(d_counts, npx, (float)(1.0 / navg), d_mu, s);
    if (!rc)
        rc = cuda_fail(cudaMemcpyAsync(h_mu, d_mu, (size_t)npx * sizeof(float),
                                       cudaMemcpyDeviceToHost, s),
                       "map download");
    if (!rc)
        rc = cuda_fail(cudaMemcpyAsync(h_stats, d_stats, RS_NSTATS * sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, s),
                       "stats download");
    if (d_mu) cudaFreeAsync(d_mu, s);
    if (d_stats) cudaFreeAsync(d_stats, s);
    if (d_counts) cudaFreeAsync(d_counts, s);
    if (d_lens) cudaFreeAsync(d_lens, s);
    const int sync_rc = cuda_fail(cudaStreamSynchronize(s), "stream synchronise");
    return rc ? rc : sync_rc;
}

}  // extern "C"
