/*
 * rs_conv.h -- finite-source convolution of magnification maps (librs_b300.so).
 *
 * A source larger than a map pixel is handled by convolving the map with the
 * source's brightness profile (Sec. 2.4): the profile is binned into pixels
 * of the map's pixel size, padded with zeros to the map's size, and the
 * convolution theorem gives C = F^-1[F(M) F(K)] (Eq. 6).  The products kept
 * per convolved map are its magnification probability distribution and a
 * few thousand (location, magnification) samples, pixelFlux.bin
 * (Sec. 3.2.2).  Conventions of rs.h apply (status codes, device pointers,
 * stream semantics, rs_last_error).
 *
 * Profiles (Sec. 2.5 item 3: uniform disc, Gaussian disc, power law / thin
 * disc, central brightness depression).  Lengths in Einstein radii, centred
 * on the origin, r = |y|:
 *   RS_PROFILE_UNIFORM    I = 1
 *   RS_PROFILE_GAUSSIAN   I = exp(-y1^2 / (2 sigma1^2) - y2^2 / (2 sigma2^2))
 *   RS_PROFILE_POWER_LAW  I = (r / r_scale)^(-index)
 *   RS_PROFILE_THIN_DISC  I = 1 / (exp(xi) - 1),
 *                         xi = (r / r_scale)^(3/4) (1 - sqrt(r_in / r))^(-1/4)
 *                         (Shakura-Sunyaev temperature profile seen at one
 *                         wavelength)
 * and I = 0 outside r_in <= r < r_out; r_out is the profile's size (where
 * the brightness drops to zero), r_in its central hole (0: none; power law
 * and thin disc need r_in > 0).
 *
 * Binning (Sec. 2.4, "binned in pixels of equal physical size to the map
 * pixels"): kernel pixel (a, b) -- a the row offset along y2, b the column
 * offset along y1, |a|, |b| <= h -- is sampled at the S x S points
 * y = (u1, u2) * w / (2 S) with odd-offset integers u1 = 2 (b S + s) + 1 - S,
 * u2 = 2 (a S + t) + 1 - S, 0 <= s, t < S.  A sample is inside when
 * rho_in2 <= u1^2 + u2^2 < rho_out2, rho2 = (2 S r / w)^2 in FP64 (an exact
 * integer test).  K[a][b] = sum of I over its inside samples / sum over all
 * pixels.  h is the largest b >= 1 whose innermost sample (|u1| = (2b-1)S+1,
 * |u2| = (S+1) mod 2) is inside r_out, else 0.  A point source (2 r_out <= w,
 * "smaller than a pixel") or an empty sum gives the unit impulse, h = 0.
 *
 * Convolution: cyclic on the npix x npix map with the kernel centred on
 * pixel (0, 0):  C[q][p] = sum_{a,b} K[a][b] M[(q-a) mod n][(p-b) mod n].
 * (The paper appends zeros to the kernel to reach the map's size, which is
 * this sum up to a cyclic shift by the kernel's half size.)  Pixels closer
 * than h to an edge mix in the opposite edge.  The transforms are
 * single-precision real-to-complex / complex-to-real FFTs: this library's own
 * (three passes over the map: rows, columns with the spectral product
 * between the forward and inverse column transforms, rows) when npix is a
 * multiple of 4, npix and npix/2 are products of 2, 3 and 5, and
 * npix <= 10240 -- the survey's 4096 and 10000 among them -- and cuFFT (the
 * library the paper uses) otherwise (the own path takes 16-byte aligned maps,
 * RS_EINVAL otherwise); binning, scattering, conversion, the
 * spectral product and the extraction are this library's kernels.
 * Round-off: the L2 norm of the error is bounded by about
 * 4 log2(npix^2) u ||M||_2 (u = 2^-24). 
 */
#ifndef RS_B300_CONV_H
#define RS_B300_CONV_H

#include <stddef.h>
#include <stdint.h>

#include "rs.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RS_PROFILE_UNIFORM    0
#define RS_PROFILE_GAUSSIAN   1
#define RS_PROFILE_POWER_LAW  2
#define RS_PROFILE_THIN_DISC  3

#define RS_PROFILE_MAX_SUPERSAMPLE  64
#define RS_VALUE_HIST_MAX_EDGES     4095
#define RS_PIXEL_FLUX_MAX_NPIX      32767   /* locations are int16 */

typedef struct {
    int32_t type;          /* RS_PROFILE_*                                    */
    int32_t supersample;   /* S: S x S samples per pixel, 1..64               */
    double r_out;          /* size: brightness zero at and beyond r_out (R_E) */
    double r_in;           /* central hole radius (R_E), 0 = none             */
    double sigma1, sigma2; /* Gaussian widths along y1, y2 (R_E)              */
    double r_scale;        /* power law / thin disc scale radius (R_E)        */
    double index;          /* power-law index                                 */
} rs_profile;

/* Half size h of the binned kernel for pixels of side `pixel` (R_E).  Host
 * only.  RS_EINVAL on a bad profile. */
RS_API int rs_profile_half(const rs_profile* prof, double pixel, int64_t* h);

/* The binned, unit-sum kernel into d_kernel[(2h+1)^2] (float32, device,
 * row a + h, column b + h); h must equal rs_profile_half's. */
RS_API int rs_profile_kernel(const rs_profile* prof, double pixel, float* d_kernel, int64_t h,
                             void* stream);

/* A convolver for npix x npix maps (2 <= npix <= RS_MAX_NPIX): owns the
 * kernel spectrum, a spectrum buffer, and the cuFFT plans and their work
 * area (or, on the own path, a table of the npix-th roots of unity),
 * about 2 x 4 npix (npix + 2) bytes plus the plans' work area, all allocated
 * here (RS_ENOMEM if the device has no room).  One host thread at a time per
 * convolver; calls on one convolver must be ordered (same stream, or
 * synchronised between streams). */
typedef struct rs_conv rs_conv;
RS_API int rs_conv_create(int64_t npix, rs_conv** out);
RS_API void rs_conv_destroy(rs_conv* conv);
/* Device bytes the convolver holds. */
RS_API int rs_conv_bytes(const rs_conv* conv, size_t* bytes);

/* Which transforms the convolver runs: RS_CONV_FFT_OWN (this library's,
 * for the sizes above) or RS_CONV_FFT_CUFFT. */
#define RS_CONV_FFT_OWN    1
#define RS_CONV_FFT_CUFFT  2
RS_API int rs_conv_fft_kind(const rs_conv* conv, int* kind);

/* Set the kernel from a profile (binned as above for pixel side `pixel`) or
 * from a caller's unit-sum kernel d_kernel[(2h+1)^2] (device, float32, same
 * layout; uploaded profiles).  RS_ERANGE if 2h+1 > npix. */
RS_API int rs_conv_set_profile(rs_conv* conv, const rs_profile* prof, double pixel,
                               void* stream);
RS_API int rs_conv_set_kernel(rs_conv* conv, const float* d_kernel, int64_t h, void* stream);

/* Convolve scale * counts (int32 count map, e.g. scale = 1 / N_avg of Eq. 4
 * for magnification) or a float32 map into d_out[npix^2] (float32, device).
 * d_map may be d_out.  The kernel must have been set. */
RS_API int rs_conv_apply_counts(rs_conv* conv, const int32_t* d_counts, double scale,
                                float* d_out, void* stream);
RS_API int rs_conv_apply(rs_conv* conv, const float* d_map, float* d_out, void* stream);

/* One map, several kernels (the survey convolves each map with several
 * source profiles): rs_conv_load_counts / rs_conv_load transform scale *
 * counts (or a float32 map) once and keep the spectrum on the convolver;
 * rs_conv_apply_loaded then gives the convolution with the kernel currently
 * set (rs_conv_set_profile / rs_conv_set_kernel may be called in between),
 * always through the transforms, bit-identical to rs_conv_apply_counts /
 * rs_conv_apply on the same map when those take the transform path.  The
 * first load allocates a second spectrum buffer (4 npix (npix + 2) bytes).
 * rs_conv_apply_counts / rs_conv_apply discard the loaded spectrum. */
RS_API int rs_conv_load_counts(rs_conv* conv, const int32_t* d_counts, double scale,
                               void* stream);
RS_API int rs_conv_load(rs_conv* conv, const float* d_map, void* stream);
RS_API int rs_conv_apply_loaded(rs_conv* conv, float* d_out, void* stream);

/* Kernel slots: a convolver keeps up to RS_CONV_SLOTS kernel spectra, slot 0
 * being the one rs_conv_set_profile / rs_conv_set_kernel set.  A survey loop
 * sets each profile once into its slot, then for every map loads it and
 * applies every slot (the product and the inverse transform per profile).
 * Slots 1.. take 8 npix (npix/2 + 1) bytes each, allocated on first use. */
#define RS_CONV_SLOTS 16
RS_API int rs_conv_set_profile_slot(rs_conv* conv, int slot, const rs_profile* prof,
                                    double pixel, void* stream);
RS_API int rs_conv_apply_loaded_slot(rs_conv* conv, int slot, float* d_out, void* stream);

/* pixelFlux.bin records (Sec. 3.2.2): 8 bytes each, {int16 x (column),
 * int16 y (row), float32 value}.  Locations from d_xy[2k] (device int16 x, y
 * pairs) or, when d_xy is NULL, drawn from `seed`: record t takes
 * x = (hi32(splitmix64(seed, 2t)) * npix) >> 32 and
 * y = (hi32(splitmix64(seed, 2t + 1)) * npix) >> 32 (SplitMix64 as for the
 * lens field).  A location outside the map gets the value NaN.
 * npix <= RS_PIXEL_FLUX_MAX_NPIX. */
typedef struct { int16_t x, y; float value; } rs_pixflux;
RS_API int rs_pixel_flux(const float* d_map, int64_t npix, const int16_t* d_xy, uint64_t seed,
                         int64_t k, rs_pixflux* d_records, void* stream);

/* Histogram of n float32 values over ascending edges h_edges[n_edges]
 * (host, 1..RS_VALUE_HIST_MAX_EDGES): d_hist[b] (int64, device, n_edges + 1
 * entries, overwritten) counts the values with exactly b edges at or below
 * them (bin 0 also takes NaN).  The MPD of a convolved map (mpd.dat). */
RS_API int rs_value_histogram(const float* d_v, int64_t n, const float* h_edges,
                              int64_t n_edges, int64_t* d_hist, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RS_B300_CONV_H */
