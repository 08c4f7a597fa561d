/*
 * rs_oracle.c -- plain FP64 CPU oracle for direct inverse ray-shooting.
 *
 * TEST INFRASTRUCTURE ONLY (see rs_oracle.h).  Compiled with
 * -O2 -ffp-contract=off and no fast-math, so every expression below rounds
 * exactly as written, in the order written.  Loops run rays in row order and
 * lenses in index order; OpenMP only splits rays across threads, which does
 * not change any per-ray result (integer counts are order independent).
 */
#include "rs_oracle.h"

#include <math.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* SplitMix64, Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014: the state advances by the odd "golden gamma"
 * 0x9e3779b97f4a7c15 and each state is passed through a 64-bit finaliser
 * (the variant with multipliers 0xbf58476d1ce4e5b9 / 0x94d049bb133111eb and
 * shifts 30, 27, 31).  Output k is the finaliser of seed + (k + 1) gamma. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Top 53 bits as a double in [0, 1). */
double orc_u01(uint64_t seed, uint64_t k)
{
    return (double)(orc_splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

/* Eq. 3: N_* = kappa_* A / (pi <M>), A = pi R^2 for a disk of radius R. */
int64_t orc_lens_count(double kappa_star, double radius, double mean_mass)
{
    if (!(kappa_star >= 0.0) || !(radius >= 0.0) || !(mean_mass > 0.0))
        return -1;
    const double pi = 3.14159265358979323846;
    double area = pi * radius * radius;
    double n = kappa_star * area / (pi * mean_mass);
    return (int64_t)floor(n + 0.5);
}

int orc_make_lenses(double radius, int mass_model, double m_lo, double m_hi,
                    double slope, int64_t n, uint64_t seed, double* lens)
{
    if (n < 0 || (n > 0 && lens == NULL) || !(radius >= 0.0))
        return -1;
    if (mass_model != 0 && mass_model != 1)
        return -1;
    if (mass_model == 1 && !(m_lo > 0.0 && m_hi > m_lo && slope != 1.0))
        return -1;
    double* x1 = lens;
    double* x2 = lens + n;
    double* m = lens + 2 * n;
    const double two_pi = 6.28318530717958647692;
    for (int64_t k = 0; k < n; ++k) {
        double u_r = orc_u01(seed, 3u * (uint64_t)k);
        double u_phi = orc_u01(seed, 3u * (uint64_t)k + 1u);
        /* uniform in the disk: P(r < s) = s^2 / R^2 */
        double r = radius * sqrt(u_r);
        double phi = two_pi * u_phi;
        x1[k] = r * cos(phi);
        x2[k] = r * sin(phi);
        if (mass_model == 0) {
            m[k] = 1.0;
        } else {
            /* inverse CDF of dN/dm ~ m^-slope on [m_lo, m_hi] */
            double u_m = orc_u01(seed, 3u * (uint64_t)k + 2u);
            double e = 1.0 - slope;
            double a = pow(m_lo, e);
            double b = pow(m_hi, e);
            m[k] = pow(a + u_m * (b - a), 1.0 / e);
        }
    }
    if (mass_model == 1 && n > 0) {
        /* mean-normalise: divide by the sample mean, summed in index order */
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k)
            s += m[k];
        double mean = s / (double)n;
        for (int64_t k = 0; k < n; ++k)
            m[k] = m[k] / mean;
    }
    return 0;
}

/* Deflection sum of Eq. 1 at one point; returns 1 if singular. */
static int deflect(const double* lens, int64_t n, double x1, double x2,
                   double* a1, double* a2)
{
    const double* lx = lens;
    const double* ly = lens + n;
    const double* lm = lens + 2 * n;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double d1 = x1 - lx[k];
        double d2 = x2 - ly[k];
        double r2 = d1 * d1 + d2 * d2;
        if (r2 == 0.0)
            return 1;
        s1 += lm[k] * d1 / r2;
        s2 += lm[k] * d2 / r2;
    }
    *a1 = s1;
    *a2 = s2;
    return 0;
}

void orc_deflection(const double* lens, int64_t n, const double* x, int64_t k,
                    double* alpha, int32_t* singular)
{
    for (int64_t t = 0; t < k; ++t) {
        double a1 = 0.0, a2 = 0.0;
        int s = deflect(lens, n, x[2 * t], x[2 * t + 1], &a1, &a2);
        if (s) {
            a1 = NAN;
            a2 = NAN;
        }
        alpha[2 * t] = a1;
        alpha[2 * t + 1] = a2;
        if (singular)
            singular[t] = s;
    }
}

/* One ray: Eq. 1 then the pixel of the map.  Returns 0 in map, 1 out,
 * 2 singular. */
static int shoot_one(const orc_macro* mc, const double* lens, int64_t n,
                     const orc_grid* g, const orc_map* mp, int64_t i, int64_t j,
                     double* y1o, double* y2o, int64_t* po, int64_t* qo)
{
    double d1 = 2.0 * g->h1 / (double)g->n1;
    double d2 = 2.0 * g->h2 / (double)g->n2;
    double x1 = g->c1 - g->h1 + ((double)i + 0.5) * d1;
    double x2 = g->c2 - g->h2 + ((double)j + 0.5) * d2;
    double a1 = 0.0, a2 = 0.0;
    *po = -1;
    *qo = -1;
    if (deflect(lens, n, x1, x2, &a1, &a2)) {
        *y1o = NAN;
        *y2o = NAN;
        return 2;
    }
    /* Eq. 1, term by term */
    double y1 = (1.0 - mc->gamma) * x1 - mc->kappa_s * x1 - a1;
    double y2 = (1.0 + mc->gamma) * x2 - mc->kappa_s * x2 - a2;
    *y1o = y1;
    *y2o = y2;
    double w = mp->width / (double)mp->npix;
    double u = (y1 - (mp->c1 - mp->width / 2.0)) / w;
    double v = (y2 - (mp->c2 - mp->width / 2.0)) / w;
    if (isfinite(u) && isfinite(v) && u >= 0.0 && v >= 0.0 &&
        u < (double)mp->npix && v < (double)mp->npix) {
        *po = (int64_t)floor(u);
        *qo = (int64_t)floor(v);
        return 0;
    }
    return 1;
}

static int check_args(const double* lens, int64_t n, const orc_grid* g,
                      const orc_map* mp)
{
    if (!g || !mp || n < 0 || (n > 0 && !lens))
        return -1;
    if (g->n1 < 0 || g->n2 < 0 || mp->npix <= 0 || !(mp->width > 0.0))
        return -1;
    if ((g->n1 > 0 && !(g->h1 > 0.0)) || (g->n2 > 0 && !(g->h2 > 0.0)))
        return -1;
    return 0;
}

int orc_shoot(const orc_macro* mc, const double* lens, int64_t n,
              const orc_grid* g, const orc_map* mp, int32_t* counts,
              int64_t* stats, int nthreads)
{
    if (!mc || !counts || !stats || check_args(lens, n, g, mp))
        return -1;
    const int64_t npix = mp->npix;
    for (int64_t t = 0; t < npix * npix; ++t)
        counts[t] = 0;
    int64_t n_in = 0, n_out = 0, n_sing = 0;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) \
    reduction(+ : n_in, n_out, n_sing)
#endif
    for (int64_t j = 0; j < g->n2; ++j) {
        for (int64_t i = 0; i < g->n1; ++i) {
            double y1, y2;
            int64_t p, q;
            int s = shoot_one(mc, lens, n, g, mp, i, j, &y1, &y2, &p, &q);
            if (s == 0) {
#ifdef _OPENMP
#pragma omp atomic update
#endif
                counts[q * npix + p] += 1;
                n_in += 1;
            } else if (s == 1) {
                n_out += 1;
            } else {
                n_sing += 1;
            }
        }
    }
    stats[0] = n_in;
    stats[1] = n_out;
    stats[2] = n_sing;
    return 0;
}

int orc_shoot_rays(const orc_macro* mc, const double* lens, int64_t n,
                   const orc_grid* g, const orc_map* mp, const int64_t* ij,
                   int64_t k, double* y, int64_t* pix, int32_t* status,
                   int nthreads)
{
    if (!mc || check_args(lens, n, g, mp) || k < 0 ||
        (k > 0 && (!ij || !y || !pix || !status)))
        return -1;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
    for (int64_t t = 0; t < k; ++t) {
        int64_t i = ij[2 * t], j = ij[2 * t + 1];
        double y1, y2;
        int64_t p, q;
        status[t] = shoot_one(mc, lens, n, g, mp, i, j, &y1, &y2, &p, &q);
        y[2 * t] = y1;
        y[2 * t + 1] = y2;
        pix[2 * t] = p;
        pix[2 * t + 1] = q;
    }
    return 0;
}

/* Eq. 4: N_avg is the number of rays a pixel receives with no lensing at
 * all: ray density (1/(d1 d2)) times pixel area w^2. */
double orc_navg(const orc_grid* g, const orc_map* mp)
{
    double d1 = 2.0 * g->h1 / (double)g->n1;
    double d2 = 2.0 * g->h2 / (double)g->n2;
    double w = mp->width / (double)mp->npix;
    return (w / d1) * (w / d2);
}

void orc_magnification(const int32_t* counts, const orc_grid* g,
                       const orc_map* mp, double* mu)
{
    double navg = orc_navg(g, mp);
    int64_t total = mp->npix * mp->npix;
    for (int64_t t = 0; t < total; ++t)
        mu[t] = (double)counts[t] / navg;
}

int orc_count_histogram(const int32_t* counts, int64_t n, int64_t* hist, int64_t n_bins)
{
    if (n < 0 || n_bins < 1 || (n > 0 && !counts) || !hist)
        return -1;
    for (int64_t b = 0; b < n_bins; ++b)
        hist[b] = 0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t c = counts[t];
        if (c < 0)
            return -1;
        if (c > n_bins - 1)
            c = n_bins - 1;
        hist[c] += 1;
    }
    return 0;
}

int orc_prob_sums(const int64_t* hist, int64_t n_bins, double navg, const double* mu_lim,
                  int n_lim, int64_t* below, int64_t* above)
{
    if (!hist || n_bins < 1 || !(navg > 0.0) || n_lim < 0 ||
        (n_lim > 0 && (!mu_lim || !below || !above)))
        return -1;
    for (int k = 0; k < n_lim; ++k) {
        double thr = mu_lim[k] * navg;
        /* the overflow bin holds counts >= n_bins - 1: exact only below it */
        if (!(thr < (double)(n_bins - 1)))
            return -1;
        int64_t lo = 0, hi = 0;
        for (int64_t c = 0; c < n_bins; ++c) {
            if ((double)c < thr)
                lo += hist[c];
            else if ((double)c > thr)
                hi += hist[c];
        }
        below[k] = lo;
        above[k] = hi;
    }
    return 0;
}

/* ---- finite source (Sec. 2.4, Eq. 6; profiles of Sec. 2.5) ---------------- */

static int profile_ok(const orc_profile* p, double w)
{
    if (!p || !(w > 0.0) || p->type < 0 || p->type > 3)
        return 0;
    if (p->supersample < 1 || p->supersample > 64)
        return 0;
    if (!(p->r_out > 0.0) || !(p->r_in >= 0.0) || !(p->r_in < p->r_out))
        return 0;
    if (p->type == 1 && !(p->sigma1 > 0.0 && p->sigma2 > 0.0))
        return 0;
    if ((p->type == 2 || p->type == 3) && !(p->r_in > 0.0 && p->r_scale > 0.0))
        return 0;
    return 1;
}

static double rho2(double r, int64_t S, double w)
{
    double v = 2.0 * (double)S * r / w;
    return v * v;
}

int64_t orc_profile_half(const orc_profile* p, double w)
{
    if (!profile_ok(p, w))
        return -1;
    if (2.0 * p->r_out <= w)
        return 0;
    const int64_t S = p->supersample;
    const double out2 = rho2(p->r_out, S, w);
    const double u2min = (double)((S + 1) % 2);
    int64_t b = 1;
    for (;;) {
        double u1 = (double)((2 * b - 1) * S + 1);
        if (!(u1 * u1 + u2min * u2min < out2))
            break;
        ++b;
    }
    return b - 1;
}

/* Brightness at the sample (u1, u2) (odd-offset integers, spacing hs). */
static double brightness(const orc_profile* p, int64_t u1, int64_t u2, double hs,
                         double in2, double out2)
{
    double q = (double)(u1 * u1 + u2 * u2);
    if (!(q >= in2 && q < out2))
        return 0.0;
    double y1 = (double)u1 * hs;
    double y2 = (double)u2 * hs;
    double r = sqrt(y1 * y1 + y2 * y2);
    switch (p->type) {
    case 0:
        return 1.0;
    case 1:
        return exp(-(y1 * y1) / (2.0 * p->sigma1 * p->sigma1) -
                   (y2 * y2) / (2.0 * p->sigma2 * p->sigma2));
    case 2:
        return pow(r / p->r_scale, -p->index);
    default: {
        double xi = pow(r / p->r_scale, 0.75) * pow(1.0 - sqrt(p->r_in / r), -0.25);
        return 1.0 / expm1(xi);
    }
    }
}

int orc_profile_kernel(const orc_profile* p, double w, int64_t h, double* k, double* raw)
{
    if (!profile_ok(p, w) || !k || h != orc_profile_half(p, w))
        return -1;
    const int64_t S = p->supersample;
    const int64_t d = 2 * h + 1;
    const double hs = w / (2.0 * (double)S);
    const double in2 = rho2(p->r_in, S, w);
    const double out2 = rho2(p->r_out, S, w);
    double total = 0.0;
    if (2.0 * p->r_out > w) {
        for (int64_t a = -h; a <= h; ++a) {
            for (int64_t b = -h; b <= h; ++b) {
                double sum = 0.0;
                for (int64_t t = 0; t < S; ++t)
                    for (int64_t s = 0; s < S; ++s)
                        sum += brightness(p, 2 * (b * S + s) + 1 - S, 2 * (a * S + t) + 1 - S,
                                          hs, in2, out2);
                k[(a + h) * d + (b + h)] = sum;
                total += sum;
            }
        }
    }
    if (raw)
        *raw = total;
    if (!(total > 0.0)) {
        /* point source: unit impulse at the centre */
        for (int64_t t = 0; t < d * d; ++t)
            k[t] = 0.0;
        k[h * d + h] = 1.0;
        return 0;
    }
    for (int64_t t = 0; t < d * d; ++t)
        k[t] = k[t] / total;
    return 0;
}

static int64_t wrap(int64_t v, int64_t n)
{
    int64_t r = v % n;
    return r < 0 ? r + n : r;
}

int orc_convolve_direct(const double* m, int64_t n, const double* k, int64_t h, double* c,
                        int nthreads)
{
    if (!m || !k || !c || n < 1 || h < 0 || 2 * h + 1 > n)
        return -1;
    const int64_t d = 2 * h + 1;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
    (void)nthreads;
#endif
    for (int64_t q = 0; q < n; ++q) {
        for (int64_t p = 0; p < n; ++p) {
            double s = 0.0;
            for (int64_t a = -h; a <= h; ++a)
                for (int64_t b = -h; b <= h; ++b)
                    s += k[(a + h) * d + (b + h)] * m[wrap(q - a, n) * n + wrap(p - b, n)];
            c[q * n + p] = s;
        }
    }
    return 0;
}

int orc_convolve_counts_at(const int32_t* counts, double scale, int64_t n, const double* k,
                           int64_t h, const int64_t* qp, int64_t cnt, double* out)
{
    if (!counts || !k || n < 1 || h < 0 || 2 * h + 1 > n || cnt < 0 ||
        (cnt > 0 && (!qp || !out)))
        return -1;
    const int64_t d = 2 * h + 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t q = qp[2 * t], p = qp[2 * t + 1];
        double s = 0.0;
        for (int64_t a = -h; a <= h; ++a)
            for (int64_t b = -h; b <= h; ++b)
                s += k[(a + h) * d + (b + h)] *
                     (scale * (double)counts[wrap(q - a, n) * n + wrap(p - b, n)]);
        out[t] = s;
    }
    return 0;
}

void orc_pixel_locations(uint64_t seed, int64_t npix, int64_t k, int16_t* xy)
{
    for (int64_t t = 0; t < k; ++t) {
        uint64_t hx = orc_splitmix64(seed, 2u * (uint64_t)t) >> 32;
        uint64_t hy = orc_splitmix64(seed, 2u * (uint64_t)t + 1u) >> 32;
        xy[2 * t] = (int16_t)((hx * (uint64_t)npix) >> 32);
        xy[2 * t + 1] = (int16_t)((hy * (uint64_t)npix) >> 32);
    }
}

int orc_value_histogram(const float* v, int64_t n, const float* edges, int64_t n_edges,
                        int64_t* hist)
{
    if (n < 0 || (n > 0 && !v) || n_edges < 1 || !edges || !hist)
        return -1;
    for (int64_t e = 1; e < n_edges; ++e)
        if (!(edges[e - 1] < edges[e]))
            return -1;
    for (int64_t b = 0; b <= n_edges; ++b)
        hist[b] = 0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t b = 0;
        while (b < n_edges && edges[b] <= v[t])
            ++b;
        hist[b] += 1;
    }
    return 0;
}

/* ---- indexed maps (App. B) -------------------------------------------------- */

#include <stdlib.h>

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int64_t orc_index_table(const int32_t* counts, int64_t n, int32_t* table)
{
    if (n < 0 || (n > 0 && (!counts || !table)))
        return -1;
    for (int64_t t = 0; t < n; ++t) {
        if (counts[t] < 0)
            return -1;
        table[t] = counts[t];
    }
    qsort(table, (size_t)n, sizeof(int32_t), cmp_i32);
    int64_t d = 0;
    for (int64_t t = 0; t < n; ++t)
        if (d == 0 || table[t] != table[d - 1])
            table[d++] = table[t];
    return d;
}

int orc_index_bits(int64_t distinct)
{
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) < distinct)
        ++b;
    return b;
}

int64_t orc_index_words(int64_t n, int bits)
{
    return (n * (int64_t)bits + 31) / 32;
}

/* position of v in the ascending table, or -1 */
static int64_t find(const int32_t* table, int64_t d, int32_t v)
{
    int64_t lo = 0, hi = d;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (table[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < d && table[lo] == v) ? lo : -1;
}

int orc_index_encode(const int32_t* counts, int64_t n, const int32_t* table, int64_t distinct,
                     int bits, uint32_t* words)
{
    if (n < 0 || distinct < 1 || !table || bits < orc_index_bits(distinct) || bits > 32 ||
        (n > 0 && (!counts || !words)))
        return -1;
    int64_t nw = orc_index_words(n, bits);
    for (int64_t w = 0; w < nw; ++w)
        words[w] = 0;
    for (int64_t t = 0; t < n; ++t) {
        int64_t idx = find(table, distinct, counts[t]);
        if (idx < 0)
            return -1;
        /* bit by bit, LSB first */
        for (int k = 0; k < bits; ++k) {
            if ((idx >> k) & 1) {
                int64_t bit = t * (int64_t)bits + k;
                words[bit / 32] |= (uint32_t)1 << (bit % 32);
            }
        }
    }
    return 0;
}

int orc_index_decode(const uint32_t* words, int64_t n, int bits, const int32_t* table,
                     int64_t distinct, int32_t* counts)
{
    if (n < 0 || bits < 1 || bits > 32 || distinct < 1 || !table ||
        (n > 0 && (!words || !counts)))
        return -1;
    for (int64_t t = 0; t < n; ++t) {
        int64_t idx = 0;
        for (int k = 0; k < bits; ++k) {
            int64_t bit = t * (int64_t)bits + k;
            if ((words[bit / 32] >> (bit % 32)) & 1u)
                idx |= (int64_t)1 << k;
        }
        if (idx >= distinct)
            return -1;
        counts[t] = table[idx];
    }
    return 0;
}

/* ---- colorbar tool and previews (Sec. 4.6, Sec. 3.2.1) ----------------------- */

int orc_colorbar_lut(const int32_t* pos, const uint8_t* rgb, int m, uint8_t* lut)
{
    if (!pos || !rgb || !lut || m < 2 || pos[0] != 0 || pos[m - 1] != 255)
        return -1;
    for (int k = 1; k < m; ++k)
        if (pos[k] < pos[k - 1])
            return -1;
    for (int i = 0; i < 256; ++i) {
        int a = -1;
        for (int k = 0; k + 1 < m; ++k)
            if (pos[k] <= i && i < pos[k + 1])
                a = k;                    /* the last pair with p_a <= i < p_b */
        for (int c = 0; c < 3; ++c) {
            if (a < 0) {
                lut[3 * i + c] = rgb[3 * (m - 1) + c];
            } else {
                int pa = pos[a], pb = pos[a + 1];
                int ca = rgb[3 * a + c], cb = rgb[3 * (a + 1) + c];
                lut[3 * i + c] = (uint8_t)((ca * (pb - i) + cb * (i - pa) + (pb - pa) / 2) / (pb - pa));
            }
        }
    }
    return 0;
}

static int sample_args(int64_t n, int64_t s)
{
    return n >= 1 && s >= 1;
}

int orc_sample_gray_counts(const int32_t* counts, int64_t n, int64_t s, const double* thr,
                           uint8_t* gray)
{
    if (!counts || !thr || !gray || !sample_args(n, s))
        return -1;
    for (int64_t r = 0; r < s; ++r) {
        for (int64_t c = 0; c < s; ++c) {
            int64_t q = (2 * r + 1) * n / (2 * s);
            int64_t p = (2 * c + 1) * n / (2 * s);
            double v = (double)counts[q * n + p];
            int g = 0;
            while (g < 255 && thr[g] <= v)
                ++g;
            gray[r * s + c] = (uint8_t)g;
        }
    }
    return 0;
}

int orc_sample_gray_f32(const float* map, int64_t n, int64_t s, const float* thr, uint8_t* gray)
{
    if (!map || !thr || !gray || !sample_args(n, s))
        return -1;
    for (int64_t r = 0; r < s; ++r) {
        for (int64_t c = 0; c < s; ++c) {
            int64_t q = (2 * r + 1) * n / (2 * s);
            int64_t p = (2 * c + 1) * n / (2 * s);
            float v = map[q * n + p];
            int g = 0;
            while (g < 255 && thr[g] <= v)
                ++g;
            gray[r * s + c] = (uint8_t)g;
        }
    }
    return 0;
}

void orc_colorize(const uint8_t* gray, int64_t m, const uint8_t* lut, uint8_t* rgba)
{
    for (int64_t t = 0; t < m; ++t) {
        const uint8_t* c = lut + 3 * gray[t];
        rgba[4 * t] = c[0];
        rgba[4 * t + 1] = c[1];
        rgba[4 * t + 2] = c[2];
        rgba[4 * t + 3] = 255;
    }
}
