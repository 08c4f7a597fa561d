/*
 * rs_oracle.h -- plain FP64 CPU oracle for direct inverse ray-shooting.
 *
 * TEST INFRASTRUCTURE ONLY.  This header and rs_oracle.c are the slow,
 * obviously-correct reference that the CUDA path is checked against.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library, and it never links against it.
 *
 * Method (Vernardos & Fluke 2014, Sec. 2.1):
 *   Eq. 1  y = diag(1-gamma, 1+gamma) x - kappa_s x - sum_i m_i (x - x_i)/|x - x_i|^2
 *   Eq. 3  N_* = kappa_* A / (pi <M>)
 *   Eq. 4  mu_ij = N_ij / N_avg
 *
 * Conventions shared by every function below (readings of the paper where it
 * is silent; each is listed with its reason in the design notes):
 *   - lengths in Einstein radii of the mean mass (Eq. 5), masses in units of
 *     the mean mass, so <M> = 1 in Eq. 3;
 *   - ray (i, j), 0 <= i < n1, 0 <= j < n2, sits at the centre of its grid
 *     cell: x1 = (c1 - h1) + (i + 1/2) * d1 with d1 = 2 h1 / n1, same for x2;
 *   - pixel p = floor((y1 - (mc1 - W/2)) / w), q likewise, w = W / npix,
 *     pixels half-open; counts are int32, row-major, row q <-> y2,
 *     column p <-> y1;
 *   - a ray with |x - x_i|^2 == 0 for some lens is singular and is excluded;
 *   - lens lists are three planes of n doubles: x1[n], x2[n], m[n].
 *
 * Parity pins: every function is checked in tests against a closed form,
 * an exact lattice count, an invariant or exact rational arithmetic, except
 * where its header comment says "parity unpinned".
 */
#ifndef RS_ORACLE_H
#define RS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double kappa_s, gamma; } orc_macro;
typedef struct { double c1, c2, h1, h2; int64_t n1, n2; } orc_grid;
typedef struct { double c1, c2, width; int64_t npix; } orc_map;

/* SplitMix64 (Steele, Lea & Flood 2014): k-th 64-bit output for a seed,
 * as a counter-based generator.  orc_u01 maps it to a double in [0, 1). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);
double orc_u01(uint64_t seed, uint64_t k);

/* Eq. 3 with A = pi R^2: N = kappa_* R^2 / <M>, rounded to nearest. */
int64_t orc_lens_count(double kappa_star, double radius, double mean_mass);

/* Lens field (Fig. 1 caption, Sec. 2.5 item 2): lens k draws u_r, u_phi, u_m
 * = outputs 3k, 3k+1, 3k+2; position r = R sqrt(u_r), phi = 2 pi u_phi;
 * mass 1 (model 0) or inverse-CDF Salpeter dN/dm ~ m^-slope on [m_lo, m_hi]
 * divided by the sample mean (model 1).  Writes x1[n], x2[n], m[n] planes
 * into lens[3n].  Returns 0, or -1 on bad arguments. */
int orc_make_lenses(double radius, int mass_model, double m_lo, double m_hi,
                    double slope, int64_t n, uint64_t seed, double* lens);

/* Deflection alpha(x) = sum_k m_k (x - x_k)/|x - x_k|^2 at k points x[2k]
 * (interleaved x1, x2), lenses in index order.  singular[k] = 1 where a lens
 * coincides with the point (alpha then NaN). */
void orc_deflection(const double* lens, int64_t n, const double* x, int64_t k,
                    double* alpha, int32_t* singular);

/* Full map (Eq. 1 + binning).  counts[npix*npix] is overwritten.
 * stats[3] = {n_in, n_out, n_singular}; n_in + n_out + n_singular = n1 n2.
 * nthreads <= 0: OpenMP default.  Returns 0, or -1 on bad arguments. */
int orc_shoot(const orc_macro* mc, const double* lens, int64_t n,
              const orc_grid* g, const orc_map* mp, int32_t* counts,
              int64_t* stats, int nthreads);

/* Same arithmetic for a list of rays ij[2k] = (i, j) pairs.  Writes
 * y[2k] (y1, y2; NaN when singular), pix[2k] (p, q; -1 when not in map) and
 * status[k] (0 in map, 1 outside or non-finite, 2 singular). */
int orc_shoot_rays(const orc_macro* mc, const double* lens, int64_t n,
                   const orc_grid* g, const orc_map* mp, const int64_t* ij,
                   int64_t k, double* y, int64_t* pix, int32_t* status,
                   int nthreads);

/* Eq. 4: mu = counts / N_avg with N_avg = (w / d1) (w / d2), the rays per
 * pixel without any lensing. */
double orc_navg(const orc_grid* g, const orc_map* mp);
void orc_magnification(const int32_t* counts, const orc_grid* g,
                       const orc_map* mp, double* mu);

/* Magnification probability distribution (Sec. 3.2.1, mpd.dat): the
 * frequency of every magnification value of a map, i.e. of every ray count
 * c (mu = c / N_avg), over the number of pixels.  hist[c] = pixels with
 * count c for c < n_bins - 1; hist[n_bins - 1] = pixels with count
 * >= n_bins - 1.  Returns 0, or -1 on bad arguments. */
int orc_count_histogram(const int32_t* counts, int64_t n, int64_t* hist, int64_t n_bins);

/* Probability sums of the MPDs tool (Sec. 4.4): for each mu_lim[k], the
 * pixels with mu < mu_lim and with mu > mu_lim, mu = c / N_avg, decided in
 * FP64 as c < mu_lim * N_avg (resp. c > mu_lim * N_avg).  Returns 0, or -1
 * when a threshold falls in the overflow bin. */
int orc_prob_sums(const int64_t* hist, int64_t n_bins, double navg, const double* mu_lim,
                  int n_lim, int64_t* below, int64_t* above);

/* ---- finite source: disc profiles and the convolution of Eq. 6 ------------
 *
 * Source profiles (Sec. 2.5 item 3: uniform disc, Gaussian disc, power law /
 * thin disc, profiles with a central brightness depression) in Einstein
 * radii, centred on the origin.  Brightness I(y1, y2), r = |y|:
 *   type 0 uniform     I = 1
 *   type 1 Gaussian    I = exp(-y1^2 / (2 sigma1^2) - y2^2 / (2 sigma2^2))
 *   type 2 power law   I = (r / r_scale)^(-index)
 *   type 3 thin disc   I = 1 / (exp(xi) - 1),
 *                      xi = (r / r_scale)^(3/4) (1 - sqrt(r_in / r))^(-1/4)
 *                      (Shakura & Sunyaev 1973 temperature profile, Planck
 *                      brightness at one wavelength; r_scale is where
 *                      h c / (lambda k T) = 1 without the inner-edge factor)
 * and I = 0 outside r_in <= r < r_out (r_out: the size at which the
 * brightness drops to zero; r_in: the central hole, 0 for none; types 2 and
 * 3 need r_in > 0).
 *
 * Binning to map pixels (Sec. 2.4): pixel (a, b) of the kernel (a: row
 * offset along y2, b: column offset along y1, -h <= a, b <= h) is sampled at
 * S x S points y1 = u1 hs, y2 = u2 hs with hs = w / (2 S) and odd integers
 * u1 = 2 (b S + s) + 1 - S, u2 = 2 (a S + t) + 1 - S, 0 <= s, t < S.  A
 * sample is inside when rho_in2 <= u1^2 + u2^2 < rho_out2, with
 * rho2 = (2 S r / w)^2 evaluated in FP64 exactly as written.  K[a][b] is the
 * sum of I over its inside samples, divided by the sum over all pixels.
 * h is the largest b >= 1 whose innermost sample, |u1| = (2b-1)S+1 and
 * |u2| = (S + 1) mod 2, has u1^2 + u2^2 < rho_out2 (h = 0 if none).  Point
 * source: if 2 r_out <= w, or the total is 0, K is the unit impulse (h = 0).
 */
typedef struct {
    int32_t type, supersample;           /* profile type 0..3, S in 1..64   */
    double r_out, r_in, sigma1, sigma2, r_scale, index;
} orc_profile;

/* Half size h of the kernel (see above), or -1 on bad arguments. */
int64_t orc_profile_half(const orc_profile* p, double w);

/* Kernel K[(2h+1)^2], row a + h, column b + h, normalised to unit sum; *raw
 * (may be NULL) receives the unnormalised sum of I over all samples.  h must
 * be orc_profile_half(p, w).  Returns 0, or -1 on bad arguments. */
int orc_profile_kernel(const orc_profile* p, double w, int64_t h, double* k, double* raw);

/* Eq. 6 as the cyclic convolution it computes on an n x n map with the
 * kernel centred on pixel (0, 0):
 *   C[q][p] = sum_{a,b=-h..h} K[a][b] M[(q - a) mod n][(p - b) mod n],
 * direct summation in FP64, kernel offsets in row order.  Needs 2h+1 <= n.
 * Returns 0, or -1 on bad arguments. */
int orc_convolve_direct(const double* m, int64_t n, const double* k, int64_t h, double* c,
                        int nthreads);

/* Same sum at cnt pixels qp[2t] = (q, p) of the map M = scale * counts. */
int orc_convolve_counts_at(const int32_t* counts, double scale, int64_t n, const double* k,
                           int64_t h, const int64_t* qp, int64_t cnt, double* out);

/* pixelFlux locations (Sec. 3.2.2): record t takes the column
 * x = (hi32(splitmix64(seed, 2t)) * npix) >> 32 and the row
 * y = (hi32(splitmix64(seed, 2t + 1)) * npix) >> 32, uniform over the map. */
void orc_pixel_locations(uint64_t seed, int64_t npix, int64_t k, int16_t* xy);

/* Histogram of values over caller-given ascending edges e[0..n_edges):
 * bin(v) = number of edges e_k <= v (so 0 = below e_0 or NaN, n_edges =
 * at or above the last edge); hist[n_edges + 1].  For the MPD of a convolved
 * map (Sec. 3.2.2, mpd.dat).  Returns 0, or -1 on bad arguments. */
int orc_value_histogram(const float* v, int64_t n, const float* edges, int64_t n_edges,
                        int64_t* hist);

/* ---- indexed maps (App. B) ------------------------------------------------
 * A count map becomes an index table -- its distinct counts in ascending
 * order -- and an indexed map in which every pixel holds the position of
 * its count in the table.  The indexed map is stored with b bits per pixel,
 * b = the fewest bits that hold every index (at least 1), packed LSB first
 * into little-endian 32-bit words: pixel t occupies bits t b .. t b + b - 1
 * of the stream (b = 16 is a plain uint16 array, b = 8 a uint8 array).
 */

/* Distinct counts of counts[n] in ascending order into table (room for n
 * entries); returns their number D, or -1 on bad arguments or a negative
 * count. */
int64_t orc_index_table(const int32_t* counts, int64_t n, int32_t* table);

/* Fewest bits that hold the indices 0 .. D-1 (1 for D <= 2). */
int orc_index_bits(int64_t distinct);

/* Words of an n-pixel map at b bits per pixel: ceil(n b / 32). */
int64_t orc_index_words(int64_t n, int bits);

/* Indexed map of counts[n] against table[D] at `bits` per pixel (>= the
 * bits D needs, <= 32) into words[orc_index_words(n, bits)].  Returns 0, or
 * -1 when a count is not in the table or on bad arguments. */
int orc_index_encode(const int32_t* counts, int64_t n, const int32_t* table, int64_t distinct,
                     int bits, uint32_t* words);

/* Counts back from an indexed map.  Returns 0, or -1 when an index is not
 * below D or on bad arguments. */
int orc_index_decode(const uint32_t* words, int64_t n, int bits, const int32_t* table,
                     int64_t distinct, int32_t* counts);

/* ---- colorbar tool (Sec. 4.6) and map previews (Sec. 3.2.1) ----------------
 * Preview sampling: an s x s sample of an n x n map takes, for sample pixel
 * (r, c), the map pixel (q, p) = (floor((2r+1) n / (2s)), floor((2c+1) n / (2s)))
 * -- the pixel under the sample's centre, no averaging of neighbours.
 * Grayscale: g = the number of the 255 ascending thresholds thr[0..255) at
 * or below the pixel's value (0..255).  Colorbar: a 256-entry RGB table
 * built from m colour stops at integer positions 0 = pos[0] <= ... <=
 * pos[m-1] = 255 by linear interpolation rounded half up in integer
 * arithmetic, lut[i] = (c_a (p_b - i) + c_b (i - p_a) + (p_b - p_a) / 2) /
 * (p_b - p_a) for the last stop pair p_a <= i < p_b with p_a < p_b (a
 * repeated position is a sharp step), and lut[255] = the last stop.  Each
 * sample pixel is then coloured lut[g] (RGBA, alpha 255).
 */
int orc_colorbar_lut(const int32_t* pos, const uint8_t* rgb, int m, uint8_t* lut);
int orc_sample_gray_counts(const int32_t* counts, int64_t n, int64_t s, const double* thr,
                           uint8_t* gray);
int orc_sample_gray_f32(const float* map, int64_t n, int64_t s, const float* thr,
                        uint8_t* gray);
void orc_colorize(const uint8_t* gray, int64_t m, const uint8_t* lut, uint8_t* rgba);

#ifdef __cplusplus
}
#endif
#endif
