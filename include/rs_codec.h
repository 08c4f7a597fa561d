/*
 * rs_codec.h -- indexed count maps and map previews (librs_b300.so).
 *
 * Indexed maps (App. B): a count map holds far fewer distinct values than
 * its largest count, so it is stored as an index table -- the distinct counts
 * in ascending order -- and an indexed map whose pixels hold the position of
 * their count in the table, in the fewest bits that hold every position.
 * Packing: pixel t occupies bits t b .. t b + b - 1 of a stream of
 * little-endian 32-bit words, least significant bit first, so b = 16 is a
 * plain uint16 array and b = 8 a uint8 array; an n-pixel map takes
 * ceil(n b / 32) words.  Lossless: decoding gives back the counts exactly.
 *
 * Previews and the colorbar tool (Sec. 3.2.1 icon/sample images, Sec. 4.6):
 * an s x s preview of an n x n map takes for sample pixel (r, c) the map
 * pixel (floor((2r+1) n / (2s)), floor((2c+1) n / (2s))) -- the pixel under
 * the sample's centre, no averaging.  Its gray level is the number of the 255
 * ascending thresholds at or below the pixel's value (0..255; NaN -> 0), and
 * its colour is entry g of a 256-entry RGB table.  The table comes from
 * colour stops at integer positions 0 = pos[0] <= ... <= pos[m-1] = 255:
 * lut[i] = (c_a (p_b - i) + c_b (i - p_a) + floor((p_b - p_a) / 2)) /
 * (p_b - p_a) in integers for the stop pair p_a <= i < p_b (a repeated
 * position makes a sharp step), lut[255] = the last stop.  Pixels are
 * written as RGBA8 (one uint32 each, R in the low byte, alpha 255).
 *
 * Conventions of rs.h apply (status codes, device pointers, streams).
 */
#ifndef RS_B300_CODEC_H
#define RS_B300_CODEC_H

#include <stddef.h>
#include <stdint.h>

#include "rs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest count the encoder accepts: any non-negative int32 (its scratch is
 * a presence bitmap with a rank prefix, 8 bytes per 32 count values up to
 * the map's largest count). */
#define RS_INDEX_MAX_COUNT  2147483647

typedef struct {
    int64_t distinct;    /* D: distinct counts = table entries              */
    int32_t bits;        /* bits per pixel of the packed map                */
    int32_t max_count;   /* largest count of the map                        */
    int64_t words;       /* 32-bit words of the packed map, ceil(n bits/32) */
} rs_index_info;

/* Fewest bits that hold the positions 0 .. D-1 (1 for D <= 2).  Host only. */
RS_API int rs_index_bits(int64_t distinct);

/* Indexed map of d_counts[n] (device int32, all >= 0):
 * the table into d_table (device int32, room for table_cap entries) and the
 * packed map into d_words (device uint32, room for words_cap words) at
 * `bits` per pixel (0: the fewest; else at least that many, at most 32).
 * Fills *info.  Synchronises `stream` once (the table size is needed on the
 * host before packing).  Scratch of 8 bytes per 32 count values up to the
 * largest count comes from the stream-ordered allocator and is released
 * before return.  RS_ERANGE when
 * the table or the packed map does not fit, or `bits` is too few. */
RS_API int rs_index_encode(const int32_t* d_counts, int64_t n, int bits, int32_t* d_table,
                           int64_t table_cap, uint32_t* d_words, int64_t words_cap,
                           rs_index_info* info, void* stream);

/* Counts back from a packed map: d_counts[t] = d_table[index of pixel t], or
 * -1 where the index is not below `distinct` (corrupt input; nothing is
 * read out of bounds).  Asynchronous. */
RS_API int rs_index_decode(const uint32_t* d_words, int64_t n, int bits, const int32_t* d_table,
                           int64_t distinct, int32_t* d_counts, void* stream);

/* The 256 x 3 colour table from m (2..256) stops (host arrays pos[m],
 * rgb[3m]) into lut[768] (host).  Host only. */
RS_API int rs_colorbar_lut(const int32_t* pos, const uint8_t* rgb, int m, uint8_t* lut);

/* s x s preview (1 <= s <= n) of an int32 count map (thresholds: 255 host
 * doubles, compared exactly with the counts) or a float32 map (255 host
 * floats): gray levels into d_gray[s*s] (device uint8, may be NULL) and, when
 * h_lut (host, 768 bytes) is given, colours into d_rgba[s*s] (device uint32,
 * may be NULL). */
RS_API int rs_preview_counts(const int32_t* d_counts, int64_t npix, int64_t s,
                             const double* h_thr, const uint8_t* h_lut, uint8_t* d_gray,
                             uint32_t* d_rgba, void* stream);
RS_API int rs_preview_f32(const float* d_map, int64_t npix, int64_t s, const float* h_thr,
                          const uint8_t* h_lut, uint8_t* d_gray, uint32_t* d_rgba,
                          void* stream);

/* Recolour m gray levels with a new table (the colorbar tool's per-pixel
 * step): d_rgba[t] = lut[d_gray[t]]. */
RS_API int rs_colorize(const uint8_t* d_gray, int64_t m, const uint8_t* h_lut, uint32_t* d_rgba,
                       void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RS_B300_CODEC_H */
