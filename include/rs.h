/*
 * rs.h -- C ABI of the B300 inverse ray-shooting library (librs_b300.so).
 *
 * Direct inverse ray-shooting for quasar microlensing (Vernardos & Fluke
 * 2014, Sec. 2.1): a regular grid of light rays in the image plane is
 * deflected by N point-mass microlenses plus smooth matter and external
 * shear (Eq. 1), every ray is counted into the source-plane pixel it lands
 * in, and the magnification of a pixel is its count over the count it
 * would receive without lensing (Eq. 4).
 *
 * Conventions (every entry point):
 *   - Units: lengths in Einstein radii of the mean microlens mass (Eq. 5),
 *     masses in units of that mean mass.
 *   - Lens list: 3*n doubles in DEVICE memory, three planes of n values:
 *     x1[0..n), x2[0..n), m[0..n).  Order matters only for rounding.
 *   - Ray grid: ray (i, j), 0 <= i < n1, 0 <= j < n2, is the centre of its
 *     cell, x1 = (c1 - half1) + (i + 1/2) * (2 half1 / n1), likewise x2.
 *     Ray id = j * n1 + i.
 *   - Map: npix x npix pixels of side w = width / npix over the square
 *     centred on (c1, c2); pixel p = floor((y1 - (c1 - width/2)) / w),
 *     q likewise; pixels are half-open.  Counts are int32, row-major,
 *     row q <-> y2, column p <-> y1 (the int32 "map.bin" layout of App. B).
 *   - Device pointers are caller-owned; the library never frees them and
 *     never keeps them after the call returns.  Pointers are checked to be
 *     device (or managed) memory; a host pointer is rejected with RS_EINVAL
 *     before anything is launched.
 *   - Calls that take `stream` (a cudaStream_t, NULL = legacy default
 *     stream) only enqueue work on it and return; outputs are valid once
 *     that stream has been synchronised.  The *_host entry points are the
 *     exception: they synchronise before returning.
 *   - Return 0 (RS_OK) or a negative status; rs_last_error() then gives a
 *     message for the calling thread.  On an error nothing has been
 *     enqueued unless the status is RS_ECUDA.
 */
#ifndef RS_B300_H
#define RS_B300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RS_API __attribute__((visibility("default")))
#else
#define RS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define RS_OK        0
#define RS_EINVAL   -1   /* bad argument (null, range, host pointer, ...)   */
#define RS_ENOMEM   -2   /* a device or host allocation failed              */
#define RS_ECUDA    -3   /* a CUDA runtime call or launch failed            */
#define RS_ETIMEOUT -4   /* a bounded device-side wait gave up              */
#define RS_EBUSY    -5   /* resource in use (server slots, queue full)      */
#define RS_ERANGE   -6   /* size beyond a documented limit                  */

/* ---- enums --------------------------------------------------------------- */
#define RS_MASS_UNIT      0   /* every lens has mass 1                       */
#define RS_MASS_SALPETER  1   /* dN/dm ~ m^-slope on [m_lo, m_hi], mean 1    */

#define RS_PREC_FP32         0  /* plain FP32 running sum per ray            */
#define RS_PREC_COMPENSATED  1  /* FP32 partial sums per lens block folded    */
                                /* into a compensated (two-sum) FP32 pair     */
#define RS_PREC_DOUBLE_SINGLE 2 /* every term in float-float (hi + lo FP32),  */
                                /* ~48 bits, on the FP32 pipe; default shape  */
                                /* only; about 4-5x the cost of the above     */
#define RS_PREC_REFINED      3  /* compensated sum; every ray whose image     */
                                /* lies within its error bound (below) of a   */
                                /* pixel edge or of the map border is shot    */
                                /* again with the double-single sum before it */
                                /* is binned.  Maps, batches and the server;  */
                                /* the shapes rs_tune_candidates lists for it */

/* Error bound of the compensated (and plain FP32) sum that RS_PREC_REFINED
 * uses as each ray's refinement band, in Einstein radii (u = 2^-24):
 *
 *   B = RS_REFINE_K * RS_REFINE_CB * u * sqrt(S2)                  far field
 *     + sum_near u m_k (RS_REFINE_CL / r_k + (|x_off| + |L_off,k|) / r_k^2)
 *     + 7 u h S1                                                  systematic
 *
 * Lenses farther than 3 h from the centre of the ray's tile (h = the tile's
 * half-diagonal) form the far field.  Each FP32 rounding in a term is an
 * independent, zero-mean error bounded by u times the rounded value (the
 * probabilistic model of Higham & Mary, SIAM J. Sci. Comput. 41, 2019); a
 * term m/r carries ten of them (lens offset and dx, dy: position; dx^2, r^2,
 * the paired product, the MUFU reciprocal (2u), the back-multiply, the mass),
 * whose bounds add in quadrature to RS_REFINE_CB u m / r together with the
 * rounding of the partial sum it enters (a random walk over the up to
 * F = 48 terms between compensated folds, F/2 = 24 in squared units of
 * u m / r; with the term's own 14.5, CB^2 = 38.5 and CB = 6.2, taken as
 * 6.75).  By Hoeffding's inequality the sum exceeds
 * RS_REFINE_K times the root of the summed squared bounds with probability
 * at most 2 exp(-K^2 / 2) = 5.4e-7 per image component.
 * S2 = sum m^2 / (r_c - h)^2 and S1 = sum m / (r_c - h)^2 over the far
 * lenses, r_c measured from the tile centre.  Lenses within 3 h of the tile
 * centre (at most RS_REFINE_NEAR_CAP per tile; more and every ray of the
 * tile is recomputed) get a linear (worst-case) bound from the ray's own
 * distance r_k (RS_REFINE_CL: 12.5 for the term's own roundings at their
 * full bound, 48 for the partial-sum roundings it can inflate before the
 * next fold), with the ray's and the lens's offsets from the tile centre
 * for the rounding of those offsets.  The systematic term covers the ray
 * offset's rounding times the lensing Jacobian and the residual of the
 * coherent-rounding correction (see rs_shoot_map).  A ray is recomputed when
 * its image lies within B / w (w = pixel width) of a pixel edge. */
#define RS_REFINE_K         5.5
#define RS_REFINE_CB        6.75
#define RS_REFINE_CL        60.5
#define RS_REFINE_NEAR_CAP  64

/* Statistics of a shoot call: d_stats[RS_NSTATS] int64. */
#define RS_NSTATS          8
#define RS_STAT_IN         0   /* rays counted into the map                     */
#define RS_STAT_OUT        1   /* rays with a finite image outside the map      */
#define RS_STAT_NONFINITE  2   /* rays whose image is not finite (on a lens)    */
#define RS_STAT_REFINED    3   /* RS_PREC_REFINED: rays the second (double-     */
                               /* single) pass recomputed                       */
#define RS_STAT_EXACT      4   /* RS_PREC_REFINED: rays the third pass          */
                               /* recomputed in FP64 (those whose double-single */
                               /* image lay within its own bound of a pixel     */
                               /* edge); a subset of RS_STAT_REFINED            */
#define RS_STAT_OVERFLOW   5   /* RS_PREC_REFINED: rays that fell in their band */
                               /* but found the ray list full; they keep their  */
                               /* first-pass pixel (0 unless the list, sized   */
                               /* for every ray up to 2^22 rays and n1 n2 / 16  */
                               /* beyond, overflowed)                           */
#define RS_STAT_BAND_USE   6   /* RS_PREC_REFINED: max over the recomputed rays */
                               /* (the first 2^20 listed) of |first-pass image  */
                               /* - double-single image| / band, x 65536: an    */
                               /* a-posteriori check of the bound on a sample   */
                               /* of rays that is unbiased in their error       */
                               /* (below 65536: every sampled error was inside  */
                               /* its band)                                     */
#define RS_STAT_MAX_DELTA  7   /* RS_PREC_REFINED: the largest such difference, */
                               /* in units of 2^-32 pixel                       */

/* ---- limits ---------------------------------------------------------------- */
#define RS_MAX_NPIX      46340            /* npix^2 < 2^31                   */
#define RS_MAX_RAYS      2147483647LL     /* n1 * n2 per call (int32 counts) */
#define RS_MAX_LENSES    2147483647LL

/* ---- structs ----------------------------------------------------------- */

/* Macromodel of Eq. 1: smooth-matter convergence kappa_s and external shear
 * gamma.  The compact-object convergence kappa_* enters only through the
 * lens list (Eq. 2-3). */
typedef struct {
    double kappa_s;
    double gamma;
} rs_macro;

/* Regular ray grid in the image plane (Sec. 2.1, Fig. 1). */
typedef struct {
    double c1, c2;        /* centre                                         */
    double half1, half2;  /* half-widths of the rectangle (> 0)             */
    int64_t n1, n2;       /* rays along x1 and x2 (>= 0)                    */
} rs_raygrid;

/* Magnification map on the source plane (Sec. 2.1, Eq. 4). */
typedef struct {
    double c1, c2;        /* centre                                         */
    double width;         /* side of the square map (> 0)                   */
    int64_t npix;         /* pixels per side, 1 .. RS_MAX_NPIX              */
} rs_mapspec;

/* Lens field (Eq. 3, Fig. 1 caption, Sec. 2.5 item 2). */
typedef struct {
    double kappa_star;    /* compact-object convergence                     */
    double radius;        /* radius R of the lens disk, area A = pi R^2     */
    int32_t mass_model;   /* RS_MASS_UNIT or RS_MASS_SALPETER               */
    int32_t reserved;
    double m_lo, m_hi;    /* Salpeter mass range (before normalisation)     */
    double slope;         /* Salpeter exponent (2.35); != 1                  */
} rs_lensfield;

/* Options of a shoot call; pass NULL for the defaults
 * {RS_PREC_COMPENSATED, 0, 0, 0}. */
typedef struct {
    int32_t precision;    /* RS_PREC_FP32, _COMPENSATED, _DOUBLE_SINGLE or
                             _REFINED                                       */
    int32_t unit_mass;    /* 1: caller asserts every mass is exactly 1; the
                             mass plane is then not read                    */
    int32_t shape;        /* kernel tile shape, 0 = default (rs_tile_shape) */
    int32_t accumulate;   /* 1: add into d_counts / d_stats (no zeroing)    */
} rs_options;

/* ---- general --------------------------------------------------------------- */

/* Library version string, e.g. "rs_b300 1.0 sm_103a". */
RS_API const char* rs_version(void);

/* Message of the last failing call on this thread ("" if none). */
RS_API const char* rs_last_error(void);

/* Bounds-checked builds: librs_b300_checked.so, built beside the library
 * with RS_CHECKED (every count-map and binning-window write of the shoot
 * kernels checks its index first, skips it when out of range and counts
 * it), stands in for compute-sanitizer on small cases.  Writes the number of
 * such writes since the last call to *out, resets it and returns 1; the
 * normal library writes 0 and returns 0.  Synchronous. */
RS_API int rs_checked_violations(int64_t* out);

/* Eq. 3 with A = pi R^2: *n = round(kappa_star R^2 / mean_mass).
 * Host-only arithmetic.  RS_EINVAL for negative or non-finite inputs. */
RS_API int rs_lens_count(double kappa_star, double radius, double mean_mass, int64_t* n);

/* Eq. 4: *navg = (w / d1) (w / d2), the rays one pixel receives without
 * lensing (ray density times pixel area).  Host-only. */
RS_API int rs_navg(const rs_raygrid* grid, const rs_mapspec* map, double* navg);

/* ---- lens field ------------------------------------------------------------ */

/* Draw n lenses uniformly in the disk of radius R (r = R sqrt(u),
 * phi = 2 pi v) with unit or mean-normalised Salpeter masses, into the
 * device lens list d_lens[3n].  The random numbers are SplitMix64 outputs
 * 3k, 3k+1, 3k+2 for lens k and the given seed (counter based, so the field
 * does not depend on the launch shape).  n is usually rs_lens_count(...).
 * Fig. 1 caption (lenses in a circle of area A), Eq. 3, Sec. 2.5 item 2. */
RS_API int rs_make_lenses(const rs_lensfield* field, uint64_t seed, double* d_lens,
                   int64_t n, void* stream);

/* ---- ray shooting ------------------------------------------------------------ */

/* Shoot the whole ray grid through Eq. 1 and bin it into d_counts
 * [npix*npix] (zeroed first unless opt->accumulate).  d_stats[RS_NSTATS]
 * (device, int64; zeroed first unless opt->accumulate) receives the
 * RS_STAT_* counts: n_in + n_out + n_nonfinite = n1 n2 and the sum of
 * d_counts is n_in.
 * The FP32 forms evaluate every lens offset from an FP64 origin per ray tile;
 * where the ray spacing is not a multiple of 2^-12 (e.g. 40000 rays over
 * 60 R_E), rounding x_ray - x_lens to FP32 would round the ray's offset onto
 * the same coarse grid for every lens whose offset shares a binary exponent,
 * an error that adds up coherently over the lenses (~ kappa * ulp).  For such
 * grids the kernel sums, per tile and per exponent 0..11 of the lens offset,
 * the Jacobian of the lens terms at the tile centre, and subtracts from each
 * ray's deflection the first-order effect of its own offset's rounding on
 * that grid (lens offsets of 4096 R_E or more are not corrected).
 * RS_PREC_REFINED takes a list of up to max(4096, n1 n2 / 16) ray ids (all
 * n1 n2 rays up to 2^22 of them) plus
 * the first-pass images of the first 2^20 of them from the stream-ordered
 * allocator and releases it before return (RS_STAT_OVERFLOW counts rays
 * beyond the list).  Sec. 2.1 (Eq. 1, Eq. 4, Fig. 1). */
RS_API int rs_shoot_map(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                 const rs_raygrid* grid, const rs_mapspec* map,
                 const rs_options* opt, int32_t* d_counts, int64_t* d_stats,
                 void* stream);

/* Checkpoint and resume (Sec. 2.1's map as a sum over rays): shoot only the
 * ray tiles [tile0, tile0 + n_tiles) of the map (tiles of rs_tile_shape, in
 * its order; a range reaching past the last tile stops there) and ADD their
 * rays to d_counts and d_stats, whatever opt->accumulate says -- the caller
 * zeroes both before the first range.  A map shot as consecutive ranges that
 * cover every tile equals rs_shoot_map's bit for bit (integer counts; in
 * RS_PREC_REFINED each range runs the second and third passes over the rays
 * it listed, and RS_STAT_BAND_USE / RS_STAT_MAX_DELTA are maxima over the
 * ranges' diagnostic samples).  So a long map can stop after any range and
 * resume from (d_counts, d_stats, next tile0).  *n_tiles_total (optional,
 * host) receives the map's number of tiles.  Errors: RS_ERANGE for tile0
 * outside [0, tiles]; otherwise as rs_shoot_map. */
RS_API int rs_shoot_map_range(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                              const rs_raygrid* grid, const rs_mapspec* map,
                              const rs_options* opt, int64_t tile0, int64_t n_tiles,
                              int32_t* d_counts, int64_t* d_stats, int64_t* n_tiles_total,
                              void* stream);

/* Ray tile of the kernel that rs_shoot_map runs for these options: tiles
 * are tx x ty rays, tile t covers rays i in [tx*(t % T1), ...), j in
 * [ty*(t / T1), ...) with T1 = ceil(n1 / tx). */
RS_API int rs_tile_shape(const rs_options* opt, int64_t* tx, int64_t* ty);

/* The deflection sum of that kernel: *fold_lenses = lenses whose FP32
 * partial sum is folded into the compensated pair at a time (RS_PREC_FP32:
 * the fold interval of the shape, unused), *unroll = lens groups per
 * unrolled loop body (RS_PREC_DOUBLE_SINGLE: the compensated kernel's). */
RS_API int rs_shape_sum(const rs_options* opt, int32_t* fold_lenses, int32_t* unroll);

/* Per-ray results of the SAME kernel for a list of tiles (test and debug
 * aid): for the w-th listed tile, ray (a, b) of the tile (a < tx, b < ty)
 * writes d_y[2 r], d_y[2 r + 1] = (y1, y2) and d_pix[2 r], d_pix[2 r + 1] =
 * (p, q) at r = w*tx*ty + b*tx + a; p = q = -1 when the ray is outside the
 * map, non-finite, or beyond the grid (then y = NaN).  The arithmetic is
 * the one rs_shoot_map uses for that ray, bit for bit. */
RS_API int rs_shoot_tiles(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                   const rs_raygrid* grid, const rs_mapspec* map,
                   const rs_options* opt, const int64_t* d_tile_ids,
                   int64_t n_tiles, double* d_y, int32_t* d_pix, void* stream);

/* Refinement band of every ray of the listed tiles (test and debug aid): the
 * bound B / w, in pixels, that the first pass of RS_PREC_REFINED computes for
 * ray (a, b) of the w-th listed tile, written to d_band[w*tx*ty + b*tx + a]
 * (float32, device; 0 for rays beyond the grid; 1 where a tile holds more
 * than RS_REFINE_NEAR_CAP near lenses).  d_y_first (optional, NULL: not
 * written; float64, device, 2 per ray as rs_shoot_tiles's d_y) receives
 * every ray's image from that first pass -- the compensated sum the bound is
 * for, before the second and third passes recompute the listed rays.
 * opt->precision must be RS_PREC_REFINED.  Tiles as rs_shoot_tiles. */
RS_API int rs_shoot_tiles_band(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                               const rs_raygrid* grid, const rs_mapspec* map,
                               const rs_options* opt, const int64_t* d_tile_ids, int64_t n_tiles,
                               float* d_band, double* d_y_first, void* stream);

/* Per-ray results for an arbitrary list of rays (debug aid, the oracle's
 * per-ray interface): h_ray_ids[k] (host, int64) = j * n1 + i; writes
 * h_y[2k], h_y[2k+1] = (y1, y2) in FP64 and h_pix[2k], h_pix[2k+1] = (p, q)
 * (host; -1 and NaN as rs_shoot_tiles) from the same kernel rs_shoot_map
 * runs, bit for bit: the tiles holding the rays are shot in dump mode.
 * Device scratch from the stream-ordered allocator; synchronises `stream`.
 * RS_EINVAL for an id outside [0, n1 n2). */
RS_API int rs_debug_rays(const rs_macro* macro, const double* d_lens, int64_t n_lens,
                         const rs_raygrid* grid, const rs_mapspec* map, const rs_options* opt,
                         const int64_t* h_ray_ids, int64_t n, double* h_y, int32_t* h_pix,
                         void* stream);

/* Eq. 4: d_mu[k] = d_counts[k] / N_avg (float32), npix*npix values. */
RS_API int rs_magnification(const int32_t* d_counts, const rs_raygrid* grid,
                     const rs_mapspec* map, float* d_mu, void* stream);

/* End-to-end call with HOST buffers: copies the host lens list h_lens[3n]
 * to the device, draws nothing, shoots, converts to magnification and copies
 * the map back into h_mu[npix*npix] (float32) and h_stats[RS_NSTATS]; synchronises
 * `stream` before returning.  Device buffers are taken from the stream-
 * ordered allocator and released before return.  Pinned host memory makes
 * the copies asynchronous; pageable memory works but is slower. */
RS_API int rs_shoot_map_host(const rs_macro* macro, const double* h_lens,
                      int64_t n_lens, const rs_raygrid* grid,
                      const rs_mapspec* map, const rs_options* opt,
                      float* h_mu, int64_t* h_stats, void* stream);

/* ---- magnification probability distribution ---------------------------------- */

/* MPD of a map (Sec. 3.2.1, mpd.dat): the frequency of every magnification
 * value over the number of pixels.  Magnification values are ray counts
 * over N_avg (Eq. 4), so this is the exact histogram of the count map:
 * d_hist[c] (int64, device) = pixels with count c for c < n_bins - 1,
 * d_hist[n_bins - 1] = pixels with count >= n_bins - 1.  When d_mu is not
 * NULL the same pass also writes mu = counts / N_avg (as rs_magnification).
 * 2 <= n_bins <= 2^31.  The MPD is d_hist / npix^2. */
RS_API int rs_mpd(const int32_t* d_counts, const rs_raygrid* grid, const rs_mapspec* map,
                  float* d_mu, int64_t* d_hist, int64_t n_bins, void* stream);

/* Probability sums (Sec. 4.4, MPDs tool): for each of n_lim (1..16)
 * thresholds mu_lim, d_below[k] / d_above[k] (int64, device) = pixels with
 * mu < mu_lim / mu > mu_lim, where mu = c / N_avg is decided in FP64 as
 * c < mu_lim * N_avg.  RS_ERANGE if a threshold reaches the overflow bin.
 * The paper's macro-magnification mu_th = 1/((1-kappa)^2 - gamma^2) sets the
 * usual thresholds 0.3 mu_th and 3 mu_th. */
RS_API int rs_prob_sums(const int64_t* d_hist, int64_t n_bins, const rs_raygrid* grid,
                        const rs_mapspec* map, const double* h_mu_lim, int n_lim,
                        int64_t* d_below, int64_t* d_above, void* stream);

/* ---- map from host buffers without device allocation ------------------------ */

/* Largest map and lens list rs_shoot_map_host_noalloc accepts. */
#define RS_NOALLOC_MAX_NPIX     1024
#define RS_NOALLOC_MAX_LENSES   65536

/* rs_shoot_map_host for callers that cannot allocate device memory on their
 * call path: code running under another framework's device allocator (a
 * cudaMalloc would bypass its accounting), real-time or plugin hosts that
 * forbid allocation during a call, processes whose device memory is reserved
 * up front.  The paper has no counterpart; this is an interface choice.
 *
 * Same arguments and results as rs_shoot_map_host (host lens list in, host
 * float32 magnification map and int64 stats[RS_NSTATS] out, synchronises `stream`),
 * but the device working set (lens copy, count map, magnification map,
 * stats) lives in one fixed file-scope device array of about 10 MB that
 * every device loading the library keeps until the process exits.  No
 * cudaMalloc, cudaFree or allocating library routine is called.
 *   - Limits: npix <= RS_NOALLOC_MAX_NPIX, n_lens <= RS_NOALLOC_MAX_LENSES;
 *     larger requests return RS_ERANGE with a message.  opt->accumulate is
 *     ignored (every call starts from a zeroed map).
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     on the calling thread's current device, so nothing cached goes stale
 *     after a device reset; the first call on a device may load the
 *     library's device code there, so make it before any stream capture.
 *   - All calls share the array and it keeps the last call's contents: two
 *     calls whose work overlaps on the GPU (other streams or host threads
 *     at the same time) race and corrupt each other's results. */
RS_API int rs_shoot_map_host_noalloc(const rs_macro* macro, const double* h_lens,
                                     int64_t n_lens, const rs_raygrid* grid,
                                     const rs_mapspec* map, const rs_options* opt,
                                     float* h_mu, int64_t* h_stats, void* stream);

/* ---- batching form ------------------------------------------------------------ */

/* One map of a batch: the arguments of rs_shoot_map plus an optional
 * magnification output.  All pointers are device memory owned by the
 * caller; d_mu may be NULL (no magnification for this map). */
typedef struct {
    rs_macro macro;
    const double* d_lens;   /* 3*n_lens doubles: x1, x2, m planes          */
    int64_t n_lens;
    rs_raygrid grid;
    rs_mapspec map;
    int32_t* d_counts;      /* npix^2 int32, zeroed unless accumulate      */
    int64_t* d_stats;       /* RS_NSTATS int64, as in rs_shoot_map         */
    float* d_mu;            /* npix^2 float32 (Eq. 4) or NULL              */
} rs_job;

/* Shoot many independent maps (the survey's batches of maps, Sec. 3 and
 * Table 3) as persistent launches of up to 128 maps each, their ray tiles
 * forming one work list, maps with the most lenses first.  Then Eq. 4 for
 * every job with d_mu.  Per map the arithmetic is that of rs_shoot_map with
 * the same kernel shape, so results are bit-identical to single-map calls
 * of that shape.  opt->shape == 0 takes the shape rs_autotune chose for a
 * batch of this kind in this process, else the default.  Asynchronous on
 * `stream`; can be captured in a CUDA graph.  No allocation, except for
 * RS_PREC_REFINED: one stream-ordered allocation holding every map's ray
 * list (as rs_shoot_map), released in stream order. */
RS_API int rs_shoot_batch(const rs_job* jobs, int n_jobs, const rs_options* opt, void* stream);

/* Time every candidate shape (rs_tune_candidates; for RS_PREC_REFINED its
 * first pass, with the ray lists) on a sample of each map's ray tiles (about
 * four waves of CTAs), store the fastest for batches of this kind (device,
 * precision, mass mode, mean lens count, mean rays, number of maps), and
 * return it in *best_shape; ms_per_gint[k] (optional, n_out entries) gets
 * milliseconds per 1e9 interactions of candidate k (rs_tune_candidates
 * order).  Synchronises `stream`.  Overwrites the jobs' counts and stats. */
RS_API int rs_autotune(const rs_job* jobs, int n_jobs, const rs_options* opt,
                       int32_t* best_shape, float* ms_per_gint, int n_out, void* stream);

/* Shapes rs_autotune tries for `precision` (RS_PREC_*), in order, the
 * default first; returns how many (writes at most max).  RS_PREC_FP32 and
 * RS_PREC_COMPENSATED: every shape with batched kernels (tile sizes, rays
 * per thread, CTAs per SM, threads per CTA, lens groups per unrolled loop
 * body, fold interval; a compensated fold of 48 lenses is 4% faster than
 * the default 24 and ~1.2x its error); RS_PREC_REFINED: the shapes with
 * refined kernels (unroll 2, 4 or 8 groups, folds of 24 or 48 lenses, all
 * covered by the error bound above); RS_PREC_DOUBLE_SINGLE: the default
 * only. */
RS_API int rs_tune_candidates(int precision, int32_t* shapes, int max);

/* A batch captured once into a CUDA graph (zero fills, persistent shoot
 * launches, magnification) and replayed with one call.  The plan keeps the
 * job list; the device buffers must stay valid while the plan is used. */
typedef struct rs_plan rs_plan;
RS_API int rs_plan_create(const rs_job* jobs, int n_jobs, const rs_options* opt, rs_plan** plan);
RS_API int rs_plan_shape(const rs_plan* plan, int32_t* shape);
RS_API int rs_plan_launch(rs_plan* plan, void* stream);
RS_API int rs_plan_destroy(rs_plan* plan);

/* ---- serving form ------------------------------------------------------------- */

/* A map server with continuous batching (the "scheduler to manage the user
 * requests" of Sec. 5): requests of mixed (kappa, gamma, N, resolution)
 * arrive at any time; they are admitted while their device memory (lens
 * list + count map + magnification map, + the ray list in RS_PREC_REFINED)
 * fits the budget and a slot is free;
 * admitted requests keep their lens set and partial map on the device, and
 * the server runs time slices, each one persistent batched launch over ray
 * tiles of the running requests (shortest remaining work first by default),
 * so new requests join the next slice instead of waiting for long ones.
 * Per ray the arithmetic is that of rs_shoot_map with the same shape (where
 * the unit-mass and general-mass kernels round differently -- double-single
 * sums, the refined form's second pass -- a slice that mixes mass models
 * runs one launch per model), so a request's map is bit-identical alone or
 * in any mix. */
#define RS_SCHED_SRPT  0    /* shortest remaining work first               */
#define RS_SCHED_FIFO  1    /* arrival order                               */

#define RS_REQ_QUEUED     0
#define RS_REQ_RUNNING    1
#define RS_REQ_DONE       2
#define RS_REQ_FAILED     3
#define RS_REQ_CANCELLED  4

typedef struct {
    int64_t hbm_budget;     /* device bytes for admitted requests (> 0)      */
    double slice_ms;        /* GPU time per slice; <= 0: whole requests      */
    double rate_gint;       /* expected throughput in 1e9 interactions/s used
                               to size slices; <= 0: 5000                    */
    int32_t max_active;     /* requests resident at once, 1 .. 128           */
    int32_t max_queue;      /* queued requests before submit says RS_EBUSY   */
    int32_t policy;         /* RS_SCHED_SRPT or RS_SCHED_FIFO                */
    int32_t precision;      /* RS_PREC_*                                     */
    int32_t shape;          /* kernel shape, 0 = default                     */
    int32_t threaded;       /* 1: a host thread runs the slices; 0: the
                               caller drives them with rs_server_step        */
    int32_t max_skips;      /* admission: times a queued request may be passed
                               by later, smaller ones before it blocks them  */
    int32_t inject_alloc_failures;  /* test hook: the next k admissions fail
                               as if the device allocation failed            */
} rs_server_config;

/* A map request: macromodel, lens field drawn on the device at admission
 * (n_lens <= 0: Eq. 3), ray grid and map. */
typedef struct {
    rs_macro macro;
    rs_lensfield field;
    uint64_t seed;
    int64_t n_lens;
    rs_raygrid grid;
    rs_mapspec map;
} rs_request;

typedef struct {
    int32_t state;            /* RS_REQ_*                                     */
    int32_t error;            /* status code when RS_REQ_FAILED               */
    const float* d_mu;        /* done: device magnification map (Eq. 4),
                                 valid until rs_server_release                */
    const int32_t* d_counts;  /* done: device count map, same lifetime       */
    int64_t stats[RS_NSTATS]; /* done: the request's RS_STAT_* counts        */
    double t_submit;          /* seconds on the server clock                  */
    double t_admit;
    double t_done;            /* completion of the request's last GPU work   */
    int64_t tiles_total;
    int64_t tiles_launched;
    int64_t n_lens;
} rs_result;

typedef struct rs_server rs_server;
/* Create a server on the current device (own stream and memory pool). */
RS_API int rs_server_create(const rs_server_config* cfg, rs_server** out);
/* Queue a request; *ticket identifies it.  RS_EBUSY when the queue is full,
 * RS_ERANGE when it could never fit the memory budget. */
RS_API int rs_server_submit(rs_server* s, const rs_request* req, int64_t* ticket);
/* Non-threaded servers: one scheduling step (complete finished slices, admit,
 * launch a slice if fewer than two are in flight); *progressed = 1 if
 * anything happened. */
RS_API int rs_server_step(rs_server* s, int32_t* progressed);
RS_API int rs_server_poll(rs_server* s, int64_t ticket, rs_result* out);
/* Block until the request is done, failed or cancelled: RS_ETIMEOUT after
 * timeout_s seconds. */
RS_API int rs_server_wait(rs_server* s, int64_t ticket, double timeout_s, rs_result* out);
/* Cancel a queued or running request (its in-flight work completes first). */
RS_API int rs_server_cancel(rs_server* s, int64_t ticket);
/* Free a finished request's device memory and forget it. */
RS_API int rs_server_release(rs_server* s, int64_t ticket);
/* Wait until no request is queued or running: RS_ETIMEOUT after timeout_s. */
RS_API int rs_server_drain(rs_server* s, double timeout_s);
/* out[0..9] = slices, shoot launches, admitted, completed, failed, cancelled,
 * peak device bytes, device bytes in use, queued, running. */
RS_API int rs_server_counters(rs_server* s, int64_t* out, int n_out);
/* Seconds since the server was created (the clock of rs_result). */
RS_API double rs_server_clock(rs_server* s);
/* Test hook (host-side fault injection): the next k admissions behave as if
 * the device allocation failed.  The request stays queued while other
 * requests run (they may free memory) and fails with RS_ENOMEM otherwise. */
RS_API int rs_server_inject_alloc_failures(rs_server* s, int k);
RS_API int rs_server_destroy(rs_server* s);

/* Scheduling policy as pure host functions (no device needed).
 * rs_sched_admit: first-fit admission in queue order under the byte budget
 * and the slot limit; a request already passed max_skips times blocks those
 * behind it.  admit[k] = 1 for admitted entries; returns how many.
 * rs_sched_plan: tiles per running request for one slice of `budget`
 * interactions (policy order; every chosen request gets >= 1 tile; at most
 * max_maps requests); returns how many requests got tiles. */
typedef struct { int64_t bytes; int32_t skips; int32_t pad_; } rs_sched_queued;
typedef struct { int64_t seq; int64_t tiles_left; double work_per_tile; } rs_sched_item;
RS_API int rs_sched_admit(const rs_sched_queued* q, int n, int64_t bytes_used, int64_t budget,
                          int active, int max_active, int max_skips, int32_t* admit);
RS_API int rs_sched_plan(const rs_sched_item* items, int n, double budget, int policy,
                         int max_maps, int64_t* take);

/* ---- measurement ------------------------------------------------------------ */

/* Issue rates of the pipes the deflection sum runs on, per SM per clock,
 * from self-timed dependency chains on the current device: out[0] MUFU
 * reciprocals (rcp.approx.f32), out[1] FP32 FMA lanes, out[2] packed f32x2
 * FMA lanes (two per instruction), out[3] FP64 FMAs, out[4] the SM clock
 * seen during the FP32 run (MHz).  n_out >= 5.  Synchronous; allocates and
 * frees a few bytes of device memory.  These rates define the roofline of
 * the deflection kernel (SMs x clock x rate). */
RS_API int rs_pipe_rates(double* out, int n_out);

#ifdef __cplusplus
}
#endif
#endif /* RS_B300_H */
