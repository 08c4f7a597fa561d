// rs_internal.cuh -- internal declarations of the B300 ray-shooting library.
//
// Everything here is private to librs_b300.so; the public surface is
// include/rs.h.  Sec. 2.1 of Vernardos & Fluke 2014 defines the operation
// (Eq. 1 lens equation, Eq. 4 magnification).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rs.h"

namespace rs {

// ---- error reporting (thread-local last message) --------------------------
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();

// ---- FP64 geometry of one shoot call, precomputed on the host -------------
// Ray (i, j) sits at x1 = x0_1 + (i + 1/2) d1, x2 = x0_2 + (j + 1/2) d2 with
// x0 = c - half and d = 2 half / n, evaluated in exactly this order (no
// contraction) so that the FP64 ray positions are those of the definition.
struct Geometry {
    double x0_1, x0_2;      // grid corner
    double d1, d2;          // ray spacing
    int64_t n1, n2;         // rays per axis
    double one_m_g;         // 1 - gamma
    double one_p_g;         // 1 + gamma
    double kappa_s;         // smooth convergence
    double y0_1, y0_2;      // map corner
    double inv_w;           // 1 / pixel width
    int32_t npix;
    int32_t flags;          // GEO_* (fills the struct's tail padding)
};

// Geometry::flags.  GEO_COHERENT: the ray spacing is not a multiple of
// 2^-12, so rounding x_ray - x_lens to FP32 rounds the ray offset onto each
// exponent's grid coherently for all lenses of that exponent; the kernels
// then apply the per-tile first-order correction (JB0..JB1 below).
constexpr int32_t GEO_COHERENT = 1;
// Lens-offset exponents whose coherent rounding is corrected: |offset| in
// [2^JB0, 2^(JB1+1)).  A spacing that is a multiple of 2^(JB1-23) = 2^-12
// leaves every ray offset on all these grids (no correction needed).
constexpr int JB0 = 0;
constexpr int JB1 = 11;
constexpr int NJB = JB1 - JB0 + 1;

// RS_PREC_REFINED ray lists, one block of device memory per map:
//   int64 ids[cap] (rounded up to even): rays the first pass lists for the
//     second (double-single) pass;
//   float4 uv[aux]: the first pass's pixel coordinates of those rays, u and
//     v as float-float hi/lo, and float band[aux]: their bands in pixels,
//     aux = min(cap, REFINE_AUX_MAX);
//   int64 ids3[cap3]: positions in ids[] of the rays the second pass lists
//     for the third (FP64) pass.
// Dump mode appends int64 slots[cap] (the ray's dump position).  The two
// list lengths live in a separate pair of counters {count, count3}.
constexpr int64_t REFINE_AUX_MAX = int64_t(1) << 20;
__host__ __device__ __forceinline__ int64_t refine_aux_cap(int64_t cap)
{
    return cap < REFINE_AUX_MAX ? cap : REFINE_AUX_MAX;
}
__host__ __device__ __forceinline__ int64_t refine_cap3(int64_t cap)
{
    return cap / 64 > 4096 ? cap / 64 : (cap < 4096 ? cap : 4096);
}
__host__ __device__ __forceinline__ float4* refine_uv(int64_t* ids, int64_t cap)
{
    return reinterpret_cast<float4*>(ids + ((cap + 1) & ~int64_t(1)));
}
__host__ __device__ __forceinline__ float* refine_band(int64_t* ids, int64_t cap)
{
    return reinterpret_cast<float*>(refine_uv(ids, cap) + refine_aux_cap(cap));
}
__host__ __device__ __forceinline__ int64_t* refine_ids3(int64_t* ids, int64_t cap)
{
    return reinterpret_cast<int64_t*>(refine_band(ids, cap) +
                                      ((refine_aux_cap(cap) + 1) & ~int64_t(1)));
}
// Bytes of the lists of capacity cap, a multiple of 16; dump mode adds
// 8 * cap for the slots.
__host__ __device__ __forceinline__ int64_t refine_list_bytes(int64_t cap)
{
    const int64_t aux = refine_aux_cap(cap);
    const int64_t b = 8 * ((cap + 1) & ~int64_t(1)) + 16 * aux + 4 * ((aux + 1) & ~int64_t(1)) +
                      8 * refine_cap3(cap);
    return (b + 15) & ~int64_t(15);
}
// Capacity rs_shoot_map, batches and the server give a map of `rays` rays:
// every ray up to 2^22 (coarse grids, whose tiles can hold many lenses and
// then list all their rays), a sixteenth beyond.
__host__ __device__ __forceinline__ int64_t refine_capacity(int64_t rays)
{
    const int64_t all = int64_t(1) << 22;
    return rays <= all ? rays : (rays / 16 > all ? rays / 16 : all);
}

// One map of a shoot launch.
struct MapDesc {
    Geometry g;
    const double* lx;       // lens planes (device, FP64)
    const double* ly;
    const double* lm;
    int32_t n_lens;
    int32_t pad_;
    int64_t tiles1;         // ray tiles along x1 (set by the launcher)
    int64_t tile0;          // first ray tile of this launch
    int64_t tile_count;     // tiles of this launch (<= 0: all from tile0 on)
    int32_t* counts;        // bin mode: map
    unsigned long long* stats;  // bin mode: RS_NSTATS counters (RS_STAT_*)
    // RS_PREC_REFINED: ids j n1 + i of the rays whose image lies within its
    // band of a pixel edge, appended by the map kernel instead of binned
    // (dump mode: listed and written) and shot again by the second pass; the
    // list's layout is that of refine_uv / refine_band above
    int64_t* refine_ids;
    unsigned long long* refine_count;   // {rays appended, rays appended to ids3}
                                        // (either may exceed its capacity)
    int64_t refine_cap;
};

// Most maps one batched launch carries.  The whole table travels as a
// __grid_constant__ kernel parameter (no device allocation, capturable in a
// CUDA graph); MAX_BATCH descriptors stay under the 32 KB parameter limit.
constexpr int MAX_BATCH = 128;

// Everything a shoot launch needs besides the maps.
struct ShootExtra {
    int64_t n_work;           // work items: tiles of all maps, or listed tiles
    const int64_t* tile_ids;  // dump mode: tiles of map 0 to process
    double* dump_y;           // dump mode: per-ray (y1, y2)
    int32_t* dump_pix;        // dump mode: per-ray (p, q)
    // RS_PREC_REFINED dump mode: per-ray band in pixels (rs_shoot_tiles_band)
    float* dump_band;
    // unused: keeps the launch parameters' layout that the map kernel's
    // lens loop was measured with (a 24-byte shift made the compensated
    // kernel 1.2% slower through the compiler's schedule)
    int64_t reserved_[2];
    int64_t* refine_slots;    // RS_PREC_REFINED dump mode: dump slot of every listed ray
};

template <int MAXB>
struct LaunchArgs {
    int32_t n_maps;
    int32_t fold_groups;      // compensated: lens groups (of 3) per fold
    int32_t fast2sum;         // compensated: 1 = Fast2Sum fold, 0 = two-sum
    int32_t pad_;
    ShootExtra x;
    int64_t tile_begin[MAXB + 1];   // first work item of each map (prefix sums)
    MapDesc maps[MAXB];
};
static_assert(sizeof(LaunchArgs<MAX_BATCH>) <= 32764, "kernel parameter limit");

// Kernel shapes selectable through rs_options.shape.
struct ShapeInfo {
    int px;        // column pairs per thread (columns = 2 px)
    int ry;        // rows per thread
    int pair;      // 1: two of every three lenses share one reciprocal
    int fold;      // compensated: lens groups between folds
    int fold_lenses;   // compensated: lenses between folds (fold x group size)
    int unroll;    // lens groups per unrolled loop body
    int fast2sum;  // compensated: fold with Fast2Sum instead of two-sum
    int tx, ty;    // ray tile (16 threads x 2px columns, 16 threads x ry rows)
    int batch;     // 1: a multi-map kernel exists for this shape
};
int shape_info(int shape, int precision, ShapeInfo* out);

enum { MODE_BIN = 0, MODE_DUMP = 1 };

// Launch the map kernel over n_maps maps (1 <= n_maps <= MAX_BATCH; maps
// are processed in the given order, their tiles contiguous).  batched:
// use the multi-map kernel even for one map.  With tuning_cap > 0 only the
// first tuning_cap tiles of every map are shot (autotuning samples).
int launch_shoot(const MapDesc* maps, int n_maps, const ShootExtra& x, int shape, int precision,
                 bool unit_mass, int mode, cudaStream_t stream, int64_t tuning_cap = 0,
                 bool batched = false);
// RS_PREC_REFINED, second and third passes: shoot the rays listed by the map
// kernel for maps[0 .. n_maps) (min(refine_count[0], refine_cap) of each
// map's refine_ids) with the double-single sum, bin them into each map's
// counts and stats -- except those whose double-single image lies within
// its error bound of a pixel edge, which the third pass shoots in FP64 and
// bins (RS_STAT_REFINED and RS_STAT_EXACT count them; RS_STAT_OVERFLOW,
// _BAND_USE and _MAX_DELTA are set here too).  Reads the counts on the
// device (no sync).  work: two zeroed counters.  dump (one map): rewrite the
// listed rays' dump slots instead of binning.
int launch_refine(const MapDesc* maps, int n_maps, unsigned long long* work, bool unit_mass,
                  cudaStream_t stream, const ShootExtra* dump = nullptr);
// Resolve the kernel and its occupancy for a launch configuration ahead of
// time (a CUDA graph capture then holds only launches).
int prime_launch(int shape, int precision, bool unit_mass, bool batched);
// Whether a map of a batch is better launched on its own: it fills the GPU
// for at least 8 waves of tiles, and the shape has a single-map kernel.
// (The batched kernels index their map descriptors at run time and are a
// few percent slower per interaction than the single-map ones.)
bool own_launch(const MapDesc& m, int shape, int precision, bool unit_mass);
bool has_single_kernel(int shape, int precision, bool unit_mass);
int check_device_ptr(const void* p, const char* name);
int prepare_map(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                const rs_raygrid* grid, const rs_mapspec* map, const rs_options& o, MapDesc* d,
                ShapeInfo* si, bool check_lens);
// Shapes that have batched (multi-map) kernels, best first.
int batch_candidates(int precision, int* shapes, int max);
int launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s);
int launch_fill_i64(int64_t* p, int64_t n, int64_t v, cudaStream_t s);
int launch_magnification(const int32_t* counts, int64_t n, float inv_navg,
                         float* mu, cudaStream_t s);
int launch_magnification_batch(const int32_t* const* counts, float* const* mu,
                               const int64_t* n_el, const float* inv_navg, int n, cudaStream_t s);
int launch_make_lenses(const rs_lensfield* f, uint64_t seed, double* d_lens,
                       int64_t n, cudaStream_t s);

int num_sms();

// ---- own two-dimensional real FFTs of Eq. 6 (rs_fft.cu) --------------------
// n x n maps with n a multiple of 4, n/2 and n of the form 2^a 3^b 5^c and
// n <= 10240; the spectrum is stored transposed, T[k][row] for the n/2 + 1
// bins k of every row (n (n/2 + 1) complex values, as a cuFFT R2C spectrum).
struct FftPlan {
    int64_t n;
    void* tw;           // exp(2 pi i m / n), m < n, float2 (device)
};
bool fft_supported(int64_t n);
int fft_plan_create(int64_t n, FftPlan* p);
size_t fft_plan_bytes(int64_t n);   // device bytes of a plan's tables
void fft_plan_destroy(FftPlan* p);
// rows: in (n x n, int32 counts when `counts`, else float32) -> T
int fft_rows_forward(const FftPlan& p, const void* in, bool counts, float2* T, cudaStream_t s);
// columns of T: forward transform, product with K (same layout) times scale,
// inverse transform, each optional; src may be dst
int fft_columns(const FftPlan& p, const float2* src, const float2* K, float scale, bool fwd,
                bool prod, bool inv, float2* dst, cudaStream_t s);
// rows: T -> out (n x n float32), unnormalised inverse
int fft_rows_inverse(const FftPlan& p, const float2* T, float* out, cudaStream_t s);

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator: output
// k of a seed is the finaliser of seed + (k + 1) * golden gamma.  Lens fields
// and pixelFlux locations draw from it.
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                                  unsigned long long k)
{
    unsigned long long z = seed + (k + 1ull) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace rs
