// rs_shoot.cu -- the inverse ray-shooting kernel (Sec. 2.1, Eq. 1 and the
// binning that feeds Eq. 4) for sm_103a.
//
// Design (B300-first; the paper's own GPU-D kernel is not followed):
//   * Persistent CTAs of 256 threads stride over ray tiles of TX x TY rays.
//     Thread (tx, ty) of the 16 x 16 arrangement owns columns tx + 16 c
//     (c < 2 PX) and rows ty + 16 r (r < RY) of the tile.
//   * FP64 only where the magnitudes need it: ray positions come from their
//     integer indices in FP64; every tile has an FP64 origin on the ray
//     lattice, and rays and lenses enter the FP32 deflection sum as offsets
//     from that origin, rounded once from FP64.  The macromodel term and the
//     final subtraction of Eq. 1 and the pixel index are FP64.
//   * Lenses are staged in shared memory in blocks of LT, double buffered,
//     as {-x, -x, -y, -y} float4s (and {m, m} float2s) so that one 16-byte
//     broadcast load feeds packed f32x2 arithmetic.  The sum runs on the
//     FP32 pipe (fma/add/mul .f32x2) and the MUFU reciprocal.
//   * Lenses go in groups of three.  With PAIR set, the first two share one
//     MUFU reciprocal: 1/a = b/(ab), 1/b = a/(ab) (Montgomery's batch
//     inversion), trading one MUFU op for three FP32 multiplies, which
//     balances the MUFU and FP32 pipes.
//   * RS_PREC_COMPENSATED: every `fold` groups (24 lenses by default; 48 in
//     the refined form's first pass) the FP32 partial sums are folded into a
//     (hi, lo) pair with Fast2Sum (or Knuth's two-sum), so the rounding of
//     the long running sum no longer grows with N.
//   * RS_PREC_REFINED: the compensated sum also lists every ray within its
//     error bound of a pixel edge (rs.h, RS_REFINE_*); refine_kernel shoots
//     the listed rays again in double-single and exact_kernel the few still
//     within that sum's bound in FP64.
//   * Binning: each ray's pixel comes from its FP64 image; counts are
//     incremented with integer atomics (order independent, so the map is
//     bit-identical run to run).
// MODE_DUMP runs the same code for a list of tiles and writes every ray's
// (y1, y2, p, q) instead of binning, so per-ray parity tests see exactly
// the arithmetic that produced the map.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr int NT = 256;          // threads per CTA
constexpr int TXT = 16;          // thread columns
constexpr int TYT = 16;          // thread rows
constexpr int LT = 768;          // lenses per shared-memory stage
static_assert(LT % 3 == 0 && LT % 4 == 0 && LT % 6 == 0 && LT % NT == 0, "stage size");
static_assert(sizeof(MapDesc) % 4 == 0, "map descriptors are copied to shared memory by 4-byte words");

// RS_CHECKED builds (librs_b300_checked.so: the bounds-checked library that
// stands in for compute-sanitizer on small cases): every count-map and
// binning-window write checks its index first; an index out of range is
// counted in g_checked_bad (read and reset by rs_checked_violations) and the
// write is skipped.  In the normal build the check is the constant true.
#ifdef RS_CHECKED
__device__ unsigned long long g_checked_bad;
__device__ __forceinline__ bool in_range(int64_t i, int64_t n)
{
    if (i >= 0 && i < n) return true;
    atomicAdd(&g_checked_bad, 1ull);
    return false;
}
#define RS_IN_RANGE(i, n) in_range((int64_t)(i), (int64_t)(n))
#else
#define RS_IN_RANGE(i, n) true
#endif

// ---- packed FP32 helpers (fma/add/mul .rn.f32x2, sm_100+) ----------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
// MUFU reciprocal (max error about 1 ulp, subnormals flushed).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 rcp2(float2 v) { return make_float2(rcp_approx(v.x), rcp_approx(v.y)); }

// Knuth two-sum of (hi, p) with the error accumulated into lo, lane-wise.
__device__ __forceinline__ void two_sum_into(float2& hi, float2& lo, float2 p)
{
    float2 s = add2(hi, p);
    float2 bb = sub2(s, hi);
    float2 e = add2(sub2(hi, sub2(s, bb)), sub2(p, bb));
    hi = s;
    lo = add2(lo, e);
}

// Dekker's Fast2Sum: exact error when |hi| >= |p| (exponent-wise), which
// holds once hi carries the accumulated deflection; otherwise the error
// estimate is inexact but the sum hi + lo stays at least as good as a
// plain FP32 sum.
__device__ __forceinline__ void fast_two_sum_into(float2& hi, float2& lo, float2 p)
{
    float2 s = add2(hi, p);
    float2 e = sub2(p, sub2(s, hi));
    hi = s;
    lo = add2(lo, e);
}

// FP64 position of ray index i: x0 + (i + 1/2) d, no contraction.
__device__ __forceinline__ double ray_pos(double x0, double d, int64_t i)
{
    return __dadd_rn(x0, __dmul_rn(__dadd_rn((double)i, 0.5), d));
}

// ---- deflection of one lens / one group of three lenses -----------------
template <int PX, int RY, bool UNIT>
__device__ __forceinline__ void lens_one(float4 L, float2 M, const float2 (&xp)[PX],
                                         const float2 (&yy)[RY], float2 (&ax)[RY][PX],
                                         float2 (&ay)[RY][PX])
{
    float2 dx[PX], dx2[PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        dx[p] = add2(xp[p], make_float2(L.x, L.y));
        dx2[p] = mul2(dx[p], dx[p]);
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        float2 dy = add2(yy[r], make_float2(L.z, L.w));
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            float2 inv = rcp2(fma2(dy, dy, dx2[p]));
            if (!UNIT) inv = mul2(inv, M);
            ax[r][p] = fma2(dx[p], inv, ax[r][p]);
            ay[r][p] = fma2(dy, inv, ay[r][p]);
        }
    }
}

// Pairing patterns: GRP lenses per group, the first 2 * NPAIR of them in
// pairs that share one reciprocal.  pair code -> (GRP, NPAIR).
__host__ __device__ constexpr int pair_grp(int pair)
{
    return pair == 2 ? 4 : pair == 3 ? 2 : pair == 4 ? 6 : 3;
}
__host__ __device__ constexpr int pair_npair(int pair) { return pair == 0 ? 0 : 1; }

template <int PX, int RY, bool UNIT, int GRP, int NPAIR>
__device__ __forceinline__ void lens_group(const float4* L, const float2* Mv,
                                           const float2 (&xp)[PX], const float2 (&yy)[RY],
                                           float2 (&ax)[RY][PX], float2 (&ay)[RY][PX])
{
    float2 dx[GRP][PX], q[GRP][PX], M[GRP];
#pragma unroll
    for (int k = 0; k < GRP; ++k) {
        const float4 Lk = L[k];
        M[k] = UNIT ? make_float2(1.f, 1.f) : Mv[k];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            dx[k][p] = add2(xp[p], make_float2(Lk.x, Lk.y));
            q[k][p] = mul2(dx[k][p], dx[k][p]);
        }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        // dy is the same for both rays of a column pair: one scalar add, the
        // pair formed by a register move (off the FMA pipe)
        float2 dy[GRP];
#pragma unroll
        for (int k = 0; k < GRP; ++k) {
            const float d = __fadd_rn(yy[r].x, L[k].z);
            dy[k] = make_float2(d, d);
        }
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            float2 rr[GRP], inv[GRP];
#pragma unroll
            for (int k = 0; k < GRP; ++k) rr[k] = fma2(dy[k], dy[k], q[k][p]);
#pragma unroll
            for (int t = 0; t < NPAIR; ++t) {
                const float2 qq = rcp2(mul2(rr[2 * t], rr[2 * t + 1]));   // 1/(a b)
                inv[2 * t] = mul2(rr[2 * t + 1], qq);                      // 1/a
                inv[2 * t + 1] = mul2(rr[2 * t], qq);                      // 1/b
            }
#pragma unroll
            for (int k = 2 * NPAIR; k < GRP; ++k) inv[k] = rcp2(rr[k]);
#pragma unroll
            for (int k = 0; k < GRP; ++k) {
                if (!UNIT) inv[k] = mul2(inv[k], M[k]);
                ax[r][p] = fma2(dx[k][p], inv[k], ax[r][p]);
                ay[r][p] = fma2(dy[k], inv[k], ay[r][p]);
            }
        }
    }
}

// ---- per-ray epilogue: Eq. 1 and the pixel index ---------------------------
// FP64 runs at 1.7 FMA/clk/SM on this part, so the per-ray part of Eq. 1 and
// of the pixel index runs in float-float on the FP32 pipe: per column and
// row the macromodel term, already shifted to the map corner and scaled to
// pixels, c = ((1-g)x1 - ks x1 - y0) / w, is computed once per tile in FP64
// (by one thread, into shared memory) and split into hi + lo FP32; per ray u = c - alpha / w with alpha = ah + al, exact to
// ~1e-14 relative (FP64 keeps the FP64 tile geometry; a pixel decision can
// differ from an FP64 evaluation only for a ray within ~1e-11 pixel of an
// edge).  With dyadic geometry and no lenses every step is exact.
struct FF {
    float h, l;
};

__device__ __forceinline__ FF split_ff(double v)
{
    FF r;
    r.h = __double2float_rn(v);
    r.l = __double2float_rn(__dsub_rn(v, (double)r.h));
    return r;
}

// s + e == a + b exactly
__device__ __forceinline__ void two_sum1(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// u = c - (ah + al) * sc as a normalised float-float uh + ul
__device__ __forceinline__ void ff_pixel_coord(FF c, float ah, float al, FF sc, float& uh,
                                               float& ul)
{
    const float ph = __fmul_rn(ah, sc.h);
    float pl = __fmaf_rn(ah, sc.h, -ph);
    pl = __fmaf_rn(ah, sc.l, pl);
    pl = __fmaf_rn(al, sc.h, pl);
    float t, e;
    two_sum1(c.h, -ph, t, e);
    e = __fadd_rn(e, __fadd_rn(c.l, -pl));
    two_sum1(t, e, uh, ul);
}

// floor(uh + ul), and 0 <= uh + ul < np
__device__ __forceinline__ int ff_floor(float uh, float ul)
{
    float f = floorf(uh);
    if (f == uh && ul < 0.f) f -= 1.f;
    return (int)f;
}
__device__ __forceinline__ bool ff_in_range(float uh, float ul, float np)
{
    const bool ge0 = uh > 0.f || (uh == 0.f && ul >= 0.f);
    const bool ltn = uh < np || (uh == np && ul < 0.f);
    return ge0 && ltn;
}

// RS_PREC_REFINED: whether the image (uh + ul, vh + vl), in pixels from the
// map corner, lies within `band` pixels of a pixel edge in either axis while
// within a pixel of the map (a finite image farther out cannot come into the
// map through an error below the band, which is at most one pixel).
__device__ __forceinline__ bool ff_near_edge(float uh, float ul, float band)
{
    // f = u - floor(uh) lies in (-ulp(uh)/2, 1 + ulp(uh)/2): u is below an
    // integer when uh is that integer and ul < 0, so the distance to the
    // nearest edge is |f| or |f - 1|
    const float f = __fadd_rn(__fsub_rn(uh, floorf(uh)), ul);   // uh - floor(uh) is exact
    return fabsf(f) < band || fabsf(__fsub_rn(f, 1.f)) < band;
}

__device__ __forceinline__ bool ff_refine(float uh, float ul, float vh, float vl, float np,
                                          float band)
{
    const bool near_map = uh > -1.f && uh < np + 1.f && vh > -1.f && vh < np + 1.f;
    return near_map && (ff_near_edge(uh, ul, band) || ff_near_edge(vh, vl, band));
}

// ---- error bound of the FP32 sums (the refined form's band) -----------------
// Per tile the map kernel gathers, while it stages the lenses, the sums the
// bound needs (rs.h, RS_REFINE_*): S2 = sum m^2 / (r_c - h)^2 and S1 = sum
// m / (r_c - h)^2 over the lenses farther than 3 h from the tile origin, and
// the lenses within 3 h themselves (at most RS_REFINE_NEAR_CAP).  They live
// in per-thread slots of dynamic shared memory (value v of thread t at
// priv[v * NTH + t], no atomics), summed over the CTA after the lens loop.
// The same slots carry the coherent-rounding correction's Jacobian sums
// (PV_J + 4 (b - JB0) + {0: d tx/d dx, 1: d ty/d dx} over lenses whose x
// offset has exponent b, {2: d tx/d dy, 3: d ty/d dy} over those whose y
// offset has it).
constexpr float U24 = 5.9604644775390625e-8f;       // 2^-24
constexpr float REF_KCB = (float)(RS_REFINE_K * RS_REFINE_CB);
constexpr float REF_CL = (float)RS_REFINE_CL;
constexpr int NEAR_CAP = RS_REFINE_NEAR_CAP;
constexpr int PV_S2 = 0, PV_S1 = 1, PV_J = 2;
constexpr int PV_ALL = PV_J + 4 * NJB;

// One staged lens at FP32 offset (xr, yr) from the tile origin (the values
// the sum uses, before negation).  Out of line: inlined into the staging
// code it changes the compiler's schedule of the lens loop (the refined map
// 0.9% slower, measured; a separate pass over the lens list before the loop
// was slower still).
template <int NTH, bool REF>
__device__ __noinline__ void field_lens(float xr, float yr, float m, bool corr, float h,
                                           float near_r2, float* priv, float4* s_near,
                                           int* s_nnear)
{
    const int t = threadIdx.x;
    const float r2 = __fmaf_rn(xr, xr, __fmul_rn(yr, yr));
    if (REF) {
        if (r2 < near_r2) {
            const int k = atomicAdd(s_nnear, 1);
            if (k < NEAR_CAP) s_near[k] = make_float4(-xr, -yr, m, sqrtf(r2));
        } else {
            // MUFU approximations (relative error ~1e-7) suffice for a bound
            const float d = __fmul_rn(r2, rsqrtf(r2)) - h;   // >= 2 h > 0
            const float i2 = __fdividef(1.f, __fmul_rn(d, d));
            priv[PV_S2 * NTH + t] += m * m * i2;
            priv[PV_S1 * NTH + t] += m * i2;
        }
    }
    if (corr) {
        const int bx = (int)((__float_as_uint(xr) >> 23) & 255u) - 127 - JB0;
        const int by = (int)((__float_as_uint(yr) >> 23) & 255u) - 127 - JB0;
        const bool okx = (unsigned)bx < (unsigned)NJB, oky = (unsigned)by < (unsigned)NJB;
        if (okx || oky) {
            // the lens terms' Jacobian at the tile origin (x = 0): with
            // d = -(xr, yr), d tx/d dx = m (yr^2 - xr^2) / r^4, d tx/d dy =
            // d ty/d dx = -2 m xr yr / r^4, d ty/d dy = -d tx/d dx
            const float i2 = __fdividef(1.f, r2);        // r2 >= 1 here
            const float i4m = m * i2 * i2;
            const float txx = (yr * yr - xr * xr) * i4m;
            const float txy = -2.f * xr * yr * i4m;
            if (okx) {
                float* q = priv + (PV_J + 4 * bx) * NTH + t;
                q[0] += txx;
                q[NTH] += txy;
            }
            if (oky) {
                float* q = priv + (PV_J + 4 * by + 2) * NTH + t;
                q[0] += txy;
                q[NTH] -= txx;
            }
        }
    }
}

// Sum the per-thread slots v < nv over the CTA into red[v] (one warp per
// value; callers put a barrier before and after).
template <int NTH>
__device__ __forceinline__ void field_reduce(const float* priv, int nv, float* red)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int v = warp; v < nv; v += NTH / 32) {
        float a = 0.f;
        for (int t = lane; t < NTH; t += 32) a += priv[v * NTH + t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) red[v] = a;
    }
}

// Coherent-rounding correction of one ray at FP32 offsets (xv, yv) from the
// tile origin: for lenses whose offset has exponent b, fl(xv + L) put the
// ray at round(xv, ulp_b) instead of xv; the deflection is corrected to
// first order with the Jacobian sums of that exponent.  Exponents with
// 2^b < 4 h are skipped (their offsets' sums can leave the exponent's range;
// the few lenses there are covered by the bound's per-term share).  Out of
// line: one copy serves every kernel variant.
__device__ __noinline__ float2 coherent_correction(const float* red, float xv, float yv, float h)
{
    float cx = 0.f, cy = 0.f;
#pragma unroll
    for (int b = 0; b < NJB; ++b) {
        const float* J = red + PV_J + 4 * b;
        const float C = __uint_as_float((unsigned)(127 + JB0 + b) << 23);   // 2^(JB0+b)
        if ((J[0] == 0.f && J[1] == 0.f && J[2] == 0.f && J[3] == 0.f) || C < 4.f * h) continue;
        const float C15 = 1.5f * C;
        const float ex = __fsub_rn(__fsub_rn(__fadd_rn(xv, C15), C15), xv);
        const float ey = __fsub_rn(__fsub_rn(__fadd_rn(yv, C15), C15), yv);
        cx = __fmaf_rn(J[0], ex, __fmaf_rn(J[2], ey, cx));
        cy = __fmaf_rn(J[1], ex, __fmaf_rn(J[3], ey, cy));
    }
    return make_float2(cx, cy);
}

// The band of one ray in pixels (rs.h): far-field and systematic parts
// per tile (base_r, in R_E), near lenses per ray.  1 pixel (every ray
// listed) when the tile held more near lenses than the list keeps.  Out of
// line, like the refined epilogue.
__device__ __noinline__ float ray_band(float base_r, const float4* s_near, int nn, bool ovf,
                                          float xv, float yv, float inv_w)
{
    if (ovf) return 1.f;
    const float xo = sqrtf(__fmaf_rn(xv, xv, __fmul_rn(yv, yv)));
    float near = 0.f;
    for (int k = 0; k < nn; ++k) {
        const float4 e = s_near[k];
        const float dx = __fadd_rn(xv, e.x), dy = __fadd_rn(yv, e.y);
        const float r2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
        if (!(r2 > 0.f)) return 1.f;
        const float ri = rsqrtf(r2);
        near = __fmaf_rn(e.z, __fmaf_rn(REF_CL, ri, (xo + e.w) * ri * ri), near);
    }
    const float b = __fmaf_rn(U24 * near, 1.01f, base_r) * inv_w + 9.3132257e-10f;   // + 2^-30
    return fminf(b, 1.f);
}

// Per-tile constants of the epilogue.
struct EpiTile {
    FF sc;      // 1 / w
    float np;   // npix
};

__device__ __forceinline__ EpiTile epi_tile(const Geometry& G)
{
    EpiTile t;
    t.sc = split_ff(G.inv_w);
    t.np = (float)G.npix;
    return t;
}

// Per column (x1) or row (x2): the macromodel term in pixels from the map
// corner, c = (((1 -+ g) x - ks x) - y0) / w, in FP64 then split.
__device__ __forceinline__ FF epi_macro(double one_mp_g, double ks, double x, double y0,
                                        double inv_w, double& m_out)
{
    m_out = __dsub_rn(__dmul_rn(one_mp_g, x), __dmul_rn(ks, x));
    return split_ff(__dmul_rn(__dsub_rn(m_out, y0), inv_w));
}

// Classify one ray: pixel (pp, qq), or -1 when it is not counted in the map;
// updates the in/out/non-finite counters of valid rays.
__device__ __forceinline__ void classify_ray(const EpiTile& T, bool valid, FF cu, FF cv, float ah,
                                             float al, float bh, float bl, int& pp, int& qq,
                                             unsigned& n_in, unsigned& n_out, unsigned& n_nf)
{
    const bool finite = isfinite(ah) && isfinite(al) && isfinite(bh) && isfinite(bl);
    float uh, ul, vh, vl;
    ff_pixel_coord(cu, ah, al, T.sc, uh, ul);
    ff_pixel_coord(cv, bh, bl, T.sc, vh, vl);
    const bool in = valid && finite && ff_in_range(uh, ul, T.np) && ff_in_range(vh, vl, T.np);
    pp = in ? ff_floor(uh, ul) : -1;
    qq = in ? ff_floor(vh, vl) : -1;
    if (valid) {
        if (in) ++n_in;
        else if (finite) ++n_out;
        else ++n_nf;
    }
}

// RS_PREC_REFINED: lists a ray near a pixel edge (warp-aggregated; every
// lane of the warp calls this together) with its first-pass pixel
// coordinates and band (the first REFINE_AUX_MAX of the list); false when it
// is not listed (not near, or the list is full).  Kept out of line also
// inside emit_ray_refined: with that arrangement the map kernel's lens loop
// was measured fastest.
__device__ __noinline__ bool refine_list(bool near, const MapDesc& M, int64_t* slots,
                                         int64_t ray_id, int64_t slot, float4 uv, float band)
{
    const unsigned m = __ballot_sync(0xffffffffu, near);
    if (!m) return false;
    const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == lead) base = atomicAdd(M.refine_count, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, lead);
    if (!near) return false;
    const unsigned long long k = base + __popc(m & ((1u << lane) - 1u));
    if (k >= (unsigned long long)M.refine_cap) return false;
    M.refine_ids[k] = ray_id;
    if ((int64_t)k < refine_aux_cap(M.refine_cap)) {
        refine_uv(M.refine_ids, M.refine_cap)[k] = uv;
        refine_band(M.refine_ids, M.refine_cap)[k] = band;
    }
    if (slot >= 0) slots[k] = slot;
    return true;
}

// One classified ray: bin mode counts pixel (pp, qq) (pp < 0: not in the
// map); dump mode writes the FP64 image y = m - a (NaN for a padding ray)
// and the pixel.  m1, m2: the FP64 macromodel terms.
template <int MODE>
__device__ __forceinline__ void write_ray(const MapDesc& M, const ShootExtra& X, int64_t w,
                                          int tile_rays, int ri_in_tile, bool valid, double m1,
                                          double m2, float ah, float al, float bh, float bl,
                                          int pp, int qq)
{
    if (MODE == MODE_BIN) {
        if (pp >= 0 && RS_IN_RANGE(pp, M.g.npix) && RS_IN_RANGE(qq, M.g.npix))
            atomicAdd(M.counts + (int64_t)qq * M.g.npix + pp, 1);
    } else {
        const int64_t ri = w * (int64_t)tile_rays + ri_in_tile;
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        const double y1 = __dsub_rn(__dsub_rn(m1, (double)ah), (double)al);
        const double y2 = __dsub_rn(__dsub_rn(m2, (double)bh), (double)bl);
        X.dump_y[2 * ri] = valid ? y1 : nan;
        X.dump_y[2 * ri + 1] = valid ? y2 : nan;
        X.dump_pix[2 * ri] = pp;
        X.dump_pix[2 * ri + 1] = qq;
    }
}

// RS_PREC_REFINED: classify_ray's steps, with the image's distance to the
// pixel edges taken from the same pixel coordinates; a ray near an edge is
// appended to the refinement list (warp-aggregated: every lane of the warp
// calls this together).  Bin mode: a listed ray is left to the second pass;
// past the list's capacity it is binned as usual.  Dump mode: it is listed
// with its dump slot and written now (the second pass overwrites it).
// Returns the ray's class: 0 in the map, 1 outside, 2 non-finite, 3 not
// counted here (padding ray, or listed in bin mode).  Out of line: inlined
// into the map kernel, it changes the compiler's schedule of the lens loop
// (1% slower per map, measured).
template <int MODE>
__device__ __noinline__ int emit_ray_refined(const MapDesc& M, const ShootExtra& X,
                                             const EpiTile& T, int64_t w, int tile_rays,
                                             int ri_in_tile, bool valid, FF cu, FF cv, double m1,
                                             double m2, float ah, float al, float bh, float bl,
                                             int64_t ray_id, float band)
{
    float uh, ul, vh, vl;
    ff_pixel_coord(cu, ah, al, T.sc, uh, ul);
    ff_pixel_coord(cv, bh, bl, T.sc, vh, vl);
    const bool finite = isfinite(ah) && isfinite(al) && isfinite(bh) && isfinite(bl);
    const int64_t slot = MODE == MODE_DUMP ? w * (int64_t)tile_rays + ri_in_tile : -1;
    if (MODE == MODE_DUMP && X.dump_band) X.dump_band[slot] = valid ? band : 0.f;
    const bool near = refine_list(valid && finite && ff_refine(uh, ul, vh, vl, T.np, band), M,
                                  X.refine_slots, ray_id, slot, make_float4(uh, ul, vh, vl),
                                  band);
    if (near && MODE == MODE_BIN) return 3;
    const bool in = valid && finite && ff_in_range(uh, ul, T.np) && ff_in_range(vh, vl, T.np);
    write_ray<MODE>(M, X, w, tile_rays, ri_in_tile, valid, m1, m2, ah, al, bh, bl,
                    in ? ff_floor(uh, ul) : -1, in ? ff_floor(vh, vl) : -1);
    return !valid ? 3 : in ? 0 : finite ? 1 : 2;
}

// Bin one ray (MODE_BIN) or write it out with its FP64 image (MODE_DUMP),
// updating the in/out/non-finite counters.  REF: the refined form's
// epilogue (emit_ray_refined).
template <int MODE, bool REF = false>
__device__ __forceinline__ void emit_ray(const MapDesc& M, const ShootExtra& X, const EpiTile& T,
                                         int64_t w, int tile_rays, int ri_in_tile, bool valid,
                                         FF cu, FF cv, double m1, double m2, float ah, float al,
                                         float bh, float bl, unsigned& n_in, unsigned& n_out,
                                         unsigned& n_nf, int64_t ray_id = 0, float band = 0.f)
{
    if (!REF) {
        int pp, qq;
        classify_ray(T, valid, cu, cv, ah, al, bh, bl, pp, qq, n_in, n_out, n_nf);
        write_ray<MODE>(M, X, w, tile_rays, ri_in_tile, valid, m1, m2, ah, al, bh, bl, pp, qq);
        return;
    }
    const int cls = emit_ray_refined<MODE>(M, X, T, w, tile_rays, ri_in_tile, valid, cu, cv, m1,
                                           m2, ah, al, bh, bl, ray_id, band);
    n_in += cls == 0;
    n_out += cls == 1;
    n_nf += cls == 2;
}

// Bin a whole ray tile.  The CTA finds the tile's footprint (bounding box of
// its in-map pixels); if it fits the shared-memory window (the lens staging
// buffer, free at this point), rays are counted there with warp-aggregated
// shared atomics and the window is flushed with one global atomic per
// non-empty pixel; otherwise each ray goes to global memory with
// warp-aggregated atomics.  Integer counts: the result does not depend on
// the path taken.  Ends with a barrier (the window is the staging buffer).
template <int NTH, int RY, int CX>
__device__ __forceinline__ void bin_tile(const int (&pix)[RY][CX], unsigned bp0, unsigned bp1,
                                         unsigned bq0, unsigned bq1, unsigned* s_box, int* win,
                                         int win_cells, int32_t* counts, int npix)
{
    const int lane = threadIdx.x & 31;
    bp0 = __reduce_min_sync(0xffffffffu, bp0);
    bp1 = __reduce_max_sync(0xffffffffu, bp1);
    bq0 = __reduce_min_sync(0xffffffffu, bq0);
    bq1 = __reduce_max_sync(0xffffffffu, bq1);
    if (threadIdx.x == 0) {
        s_box[0] = 0xffffffffu;
        s_box[1] = 0u;
        s_box[2] = 0xffffffffu;
        s_box[3] = 0u;
    }
    __syncthreads();
    if (lane == 0 && bp0 <= bp1) {
        atomicMin(s_box + 0, bp0);
        atomicMax(s_box + 1, bp1);
        atomicMin(s_box + 2, bq0);
        atomicMax(s_box + 3, bq1);
    }
    __syncthreads();
    const unsigned p0 = s_box[0], p1 = s_box[1], q0 = s_box[2], q1 = s_box[3];
    if (p0 <= p1) {
        const int bw = (int)(p1 - p0 + 1), bh = (int)(q1 - q0 + 1);
        if ((int64_t)bw * bh <= win_cells) {
            for (int k = threadIdx.x; k < bw * bh; k += NTH) win[k] = 0;
            __syncthreads();
#pragma unroll
            for (int r = 0; r < RY; ++r)
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    const int key = pix[r][c];
                    const unsigned m = __match_any_sync(0xffffffffu, key);
                    if (key >= 0 && lane == __ffs(m) - 1) {
                        const int q = key / npix, p = key - q * npix;
                        const int wi = (q - (int)q0) * bw + (p - (int)p0);
                        if (RS_IN_RANGE(wi, bw * bh)) atomicAdd(win + wi, __popc(m));
                    }
                }
            __syncthreads();
            for (int k = threadIdx.x; k < bw * bh; k += NTH) {
                const int v = win[k];
                if (v) {
                    const int dq = k / bw;
                    const int64_t gi = (int64_t)(q0 + dq) * npix + (p0 + (k - dq * bw));
                    if (RS_IN_RANGE(gi, (int64_t)npix * npix)) atomicAdd(counts + gi, v);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < RY; ++r)
#pragma unroll
                for (int c = 0; c < CX; ++c) {
                    const int key = pix[r][c];
                    const unsigned m = __match_any_sync(0xffffffffu, key);
                    if (key >= 0 && lane == __ffs(m) - 1 && RS_IN_RANGE(key, (int64_t)npix * npix))
                        atomicAdd(counts + key, (int)__popc(m));
                }
        }
    }
    __syncthreads();
}

template <int PX, int RY, int PAIR, int PREC, bool UNIT, int MODE, int MINB, int UNR, int MAXB,
          int NTH, int BIN>
__global__ void __launch_bounds__(NTH, MINB)
shoot_kernel(const __grid_constant__ LaunchArgs<MAXB> A)
{
    constexpr int CX = 2 * PX;
    constexpr int TX = TXT * CX;
    constexpr int TYTK = NTH / TXT;     // thread rows
    constexpr int LPTK = LT / NTH;      // lenses staged by each thread per stage
    static_assert(NTH % TXT == 0 && LT % NTH == 0, "thread arrangement");
    constexpr int TY = TYTK * RY;
    // the map descriptor of the current tile, copied from the kernel
    // parameters into shared memory (two buffers by tile parity) when a launch
    // carries several maps: read from there, its fields do not tie up
    // registers across the lens loop as dynamically indexed parameter loads
    // do (measured: the batched kernel 4.8% slower than the single-map one
    // with them, 1.2% with this copy)
    __shared__ __align__(16) MapDesc s_map[MAXB > 1 ? 2 : 1];
    __shared__ __align__(16) float4 s_pos[2][LT];
    __shared__ __align__(8) float2 s_m[UNIT ? 1 : 2][UNIT ? 1 : LT];
    __shared__ unsigned s_box[4];   // BIN == 1: footprint of the tile in pixels
    // Macromodel term of the epilogue per tile column (x1) and row (x2),
    // computed once per CTA in FP64 and shared by the 16 threads that use
    // each (FF; FP64 for the per-ray dump).  Two buffers by tile parity: a
    // thread may start the next tile while another still reads the terms of
    // this one.  (The rays' offsets from the tile origin stay per thread:
    // taken from shared memory they cost the lens loop 1-2%.)
    __shared__ FF s_cu[2][TX];
    __shared__ FF s_cv[2][TY];
    __shared__ double s_m1[MODE == MODE_DUMP ? 2 : 1][MODE == MODE_DUMP ? TX : 1];
    __shared__ double s_m2[MODE == MODE_DUMP ? 2 : 1][MODE == MODE_DUMP ? TY : 1];
    // error-bound and coherent-correction sums of the tile (two buffers by
    // tile parity), the near lenses (refined form), and the per-thread slots
    // (dynamic: 2 values per thread for the refined form, PV_ALL when a map
    // of the launch needs the coherent correction)
    constexpr bool REF = PREC == RS_PREC_REFINED;
    __shared__ float s_red[2][PV_ALL];
    __shared__ __align__(16) float4 s_near[REF ? 2 : 1][REF ? NEAR_CAP : 1];
    __shared__ int s_nnear[2];
    extern __shared__ __align__(16) float s_priv[];

    const int tx = threadIdx.x % TXT;
    const int ty = threadIdx.x / TXT;
    if (threadIdx.x < 2) s_nnear[threadIdx.x] = 0;
    __syncthreads();

    // in/out/non-finite counts of the map being worked on, flushed with one
    // warp reduction and three 64-bit atomics whenever the map changes
    unsigned n_in = 0, n_out = 0, n_nf = 0;
    int cur_map = -1;
    auto flush = [&]() {
        if (MODE != MODE_BIN || cur_map < 0) return;
        const unsigned s_in = __reduce_add_sync(0xffffffffu, n_in);
        const unsigned s_out = __reduce_add_sync(0xffffffffu, n_out);
        const unsigned s_nf = __reduce_add_sync(0xffffffffu, n_nf);
        if ((threadIdx.x & 31) == 0) {
            unsigned long long* st = A.maps[cur_map].stats;
            if (s_in) atomicAdd(st + 0, (unsigned long long)s_in);
            if (s_out) atomicAdd(st + 1, (unsigned long long)s_out);
            if (s_nf) atomicAdd(st + 2, (unsigned long long)s_nf);
        }
        n_in = n_out = n_nf = 0;
    };

    int pb = 1;            // buffer of the per-column / per-row terms
    EpiTile T{};           // per-map constants of the epilogue
    for (int64_t w = blockIdx.x; w < A.x.n_work; w += gridDim.x) {
        pb ^= 1;
        // map of this work item (uniform across the CTA)
        int mi = 0;
        if (MAXB > 1) {
            int lo = 0, hi = A.n_maps - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (A.tile_begin[mid] <= w) lo = mid; else hi = mid - 1;
            }
            mi = lo;
        }
        if (mi != cur_map) {
            flush();
            cur_map = mi;
            T = epi_tile(A.maps[mi].g);
        }
        const MapDesc* Mp = &A.maps[0];
        if constexpr (MAXB > 1) {
            const int* src = reinterpret_cast<const int*>(&A.maps[mi]);
            int* dst = reinterpret_cast<int*>(&s_map[MAXB > 1 ? pb : 0]);
            for (int q = threadIdx.x; q < (int)(sizeof(MapDesc) / 4); q += NTH) dst[q] = src[q];
            __syncthreads();
            Mp = &s_map[MAXB > 1 ? pb : 0];
        }
        const MapDesc& M = *Mp;
        const Geometry& G = M.g;
        const int n_lens = M.n_lens;
        const int n_stage = (n_lens + LT - 1) / LT;

        const int64_t tile = (MODE == MODE_DUMP) ? A.x.tile_ids[w]
                                                 : M.tile0 + (w - A.tile_begin[mi]);
        const int64_t tj = tile / M.tiles1;
        const int64_t ti = tile - tj * M.tiles1;
        const int64_t i0 = ti * TX;
        const int64_t j0 = tj * TY;
        // FP64 tile origin on the ray lattice
        const double o1 = ray_pos(G.x0_1, G.d1, i0 + TX / 2);
        const double o2 = ray_pos(G.x0_2, G.d2, j0 + TY / 2);
        // error-bound sums (refined form) and coherent-rounding correction
        // (ray spacing off the 2^-12 grid): per-thread slots start at zero
        const bool corr = (G.flags & GEO_COHERENT) != 0;
        const bool field = REF || corr;
        const float fh1 = (float)(G.d1 * (TX / 2)), fh2 = (float)(G.d2 * (TY / 2));
        const float h = sqrtf(__fmaf_rn(fh1, fh1, __fmul_rn(fh2, fh2)));   // tile half-diagonal
        const float near_r2 = 9.f * h * h;
        if (field) {
            const int nv = corr ? PV_ALL : PV_J;
            for (int v = 0; v < nv; ++v) s_priv[v * NTH + threadIdx.x] = 0.f;
        }

        // epilogue terms in FP64 per tile column and row, one thread each
        // (read after the tile's first barrier)
        for (int k = threadIdx.x; k < TX + TY; k += NTH) {
            double m;
            if (k < TX) {
                s_cu[pb][k] = epi_macro(G.one_m_g, G.kappa_s, ray_pos(G.x0_1, G.d1, i0 + k),
                                        G.y0_1, G.inv_w, m);
                if (MODE == MODE_DUMP) s_m1[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? k : 0] = m;
            } else {
                const int kr = k - TX;
                s_cv[pb][kr] = epi_macro(G.one_p_g, G.kappa_s, ray_pos(G.x0_2, G.d2, j0 + kr),
                                         G.y0_2, G.inv_w, m);
                if (MODE == MODE_DUMP) s_m2[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? kr : 0] = m;
            }
        }
        float2 xp[PX];
        float2 yy[RY];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            float a = __double2float_rn(__dsub_rn(ray_pos(G.x0_1, G.d1, i0 + tx + TXT * (2 * p)), o1));
            float b = __double2float_rn(__dsub_rn(ray_pos(G.x0_1, G.d1, i0 + tx + TXT * (2 * p + 1)), o1));
            xp[p] = make_float2(a, b);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            float v = __double2float_rn(__dsub_rn(ray_pos(G.x0_2, G.d2, j0 + ty + TYTK * r), o2));
            yy[r] = make_float2(v, v);
        }

        float2 ax[RY][PX], ay[RY][PX];
        float2 hx[RY][PX], lx[RY][PX], hy[RY][PX], ly[RY][PX];
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                ax[r][p] = ay[r][p] = make_float2(0.f, 0.f);
                hx[r][p] = lx[r][p] = hy[r][p] = ly[r][p] = make_float2(0.f, 0.f);
            }

        auto fold = [&]() {
            if (PREC != RS_PREC_FP32) {
#pragma unroll
                for (int r = 0; r < RY; ++r)
#pragma unroll
                    for (int p = 0; p < PX; ++p) {
                        if (A.fast2sum) {
                            fast_two_sum_into(hx[r][p], lx[r][p], ax[r][p]);
                            fast_two_sum_into(hy[r][p], ly[r][p], ay[r][p]);
                        } else {
                            two_sum_into(hx[r][p], lx[r][p], ax[r][p]);
                            two_sum_into(hy[r][p], ly[r][p], ay[r][p]);
                        }
                        ax[r][p] = ay[r][p] = make_float2(0.f, 0.f);
                    }
            }
        };

        double rx[LPTK], ryv[LPTK], rm[LPTK];
        auto load_stage = [&](int base) {
#pragma unroll
            for (int s = 0; s < LPTK; ++s) {
                const int k = base + threadIdx.x + NTH * s;
                if (k < n_lens) {
                    rx[s] = __ldg(M.lx + k);
                    ryv[s] = __ldg(M.ly + k);
                    if (!UNIT) rm[s] = __ldg(M.lm + k);
                }
            }
        };
        auto store_stage = [&](int buf, int base) {
#pragma unroll
            for (int s = 0; s < LPTK; ++s) {
                const int idx = threadIdx.x + NTH * s;
                if (base + idx < n_lens) {
                    const float xr = __double2float_rn(__dsub_rn(rx[s], o1));
                    const float yr = __double2float_rn(__dsub_rn(ryv[s], o2));
                    s_pos[buf][idx] = make_float4(-xr, -xr, -yr, -yr);
                    float m = 1.f;
                    if (!UNIT) {
                        m = __double2float_rn(rm[s]);
                        s_m[UNIT ? 0 : buf][UNIT ? 0 : idx] = make_float2(m, m);
                    }
                    if (field)
                        field_lens<NTH, REF>(xr, yr, m, corr, h, near_r2, s_priv,
                                             s_near[REF ? pb : 0], &s_nnear[pb]);
                }
            }
        };

        if (n_stage > 0) {
            load_stage(0);
            store_stage(0, 0);
            __syncthreads();
            for (int st = 0; st < n_stage; ++st) {
                const int buf = st & 1;
                const int base = st * LT;
                const bool more = st + 1 < n_stage;
                if (more) load_stage(base + LT);

                constexpr int GRP = pair_grp(PAIR);
                const int cnt = min(LT, n_lens - base);
                const int ng = cnt / GRP;
                const float4* P = s_pos[buf];
                const float2* Mv = s_m[UNIT ? 0 : buf];
                int g = 0;
                while (g < ng) {
                    const int gend = min(ng, g + A.fold_groups);
#pragma unroll UNR
                    for (; g < gend; ++g)
                        lens_group<PX, RY, UNIT, GRP, pair_npair(PAIR)>(P + GRP * g, Mv + GRP * g,
                                                                        xp, yy, ax, ay);
                    fold();
                }
                if (GRP * ng < cnt) {
#pragma unroll 1
                    for (int l = GRP * ng; l < cnt; ++l) {
                        float2 Mw = make_float2(1.f, 1.f);
                        if (!UNIT) Mw = Mv[l];
                        lens_one<PX, RY, UNIT>(P[l], Mw, xp, yy, ax, ay);
                    }
                    fold();
                }
                if (more) store_stage(buf ^ 1, base + LT);
                __syncthreads();
            }
        }

        else {
            __syncthreads();      // no lenses: the per-column terms still need it
        }

        // the tile's sums over all threads' slots; the other parity's near
        // list is reset for the next tile (its last reader passed this
        // tile's first barrier)
        if (field) {
            if (REF && threadIdx.x == 0) s_nnear[pb ^ 1] = 0;
            field_reduce<NTH>(s_priv, corr ? PV_ALL : PV_J, s_red[pb]);
            __syncthreads();
        }
        float base_r = 0.f;
        int nn = 0;
        bool novf = false;
        if (REF) {
            base_r = __fmaf_rn(REF_KCB * U24, sqrtf(s_red[pb][PV_S2]),
                               7.f * U24 * h * s_red[pb][PV_S1]);
            nn = min(s_nnear[pb], NEAR_CAP);
            novf = s_nnear[pb] > NEAR_CAP;
        }
        const float inv_wf = (float)G.inv_w;

        // ---- Eq. 1 and the pixel of every ray (macromodel part in FP64
        // per column and row, per-ray part in float-float) ---------------
        double m1[CX];
        FF cu[CX];
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            cu[c] = s_cu[pb][tx + TXT * c];
            m1[c] = MODE == MODE_DUMP ? s_m1[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? tx + TXT * c : 0] : 0.0;
        }
        // BIN == 1: pixel of every ray first (q * npix + p, or -1), then the
        // binning of the whole tile
        int pix[RY][CX];
        unsigned bp0 = 0xffffffffu, bp1 = 0u, bq0 = 0xffffffffu, bq1 = 0u;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int64_t j = j0 + ty + TYTK * r;
            const double m2 = MODE == MODE_DUMP ? s_m2[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? ty + TYTK * r : 0] : 0.0;
            const FF cv = s_cv[pb][ty + TYTK * r];
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int64_t i = i0 + tx + TXT * c;
                const bool valid = (i < G.n1) && (j < G.n2);
                const int p = c >> 1;
                const bool b = c & 1;
                float ah, al, bh, bl;
                if (PREC != RS_PREC_FP32) {
                    ah = b ? hx[r][p].y : hx[r][p].x;
                    al = b ? lx[r][p].y : lx[r][p].x;
                    bh = b ? hy[r][p].y : hy[r][p].x;
                    bl = b ? ly[r][p].y : ly[r][p].x;
                } else {
                    ah = b ? ax[r][p].y : ax[r][p].x;
                    bh = b ? ay[r][p].y : ay[r][p].x;
                    al = bl = 0.f;
                }
                const float xv = b ? xp[p].y : xp[p].x, yv = yy[r].x;
                if (corr) {
                    const float2 cc = coherent_correction(s_red[pb], xv, yv, h);
                    al = __fsub_rn(al, cc.x);
                    bl = __fsub_rn(bl, cc.y);
                }
                if (BIN == 1 && MODE == MODE_BIN) {
                    int pp, qq;
                    classify_ray(T, valid, cu[c], cv, ah, al, bh, bl, pp, qq, n_in, n_out, n_nf);
                    pix[r][c] = pp >= 0 ? qq * G.npix + pp : -1;
                    if (pp >= 0) {
                        bp0 = min(bp0, (unsigned)pp);
                        bp1 = max(bp1, (unsigned)pp);
                        bq0 = min(bq0, (unsigned)qq);
                        bq1 = max(bq1, (unsigned)qq);
                    }
                } else {
                    const float band =
                        REF ? ray_band(base_r, s_near[REF ? pb : 0], nn, novf, xv, yv, inv_wf) : 0.f;
                    emit_ray<MODE, PREC == RS_PREC_REFINED>(
                        M, A.x, T, w, TX * TY, (ty + TYTK * r) * TX + (tx + TXT * c), valid, cu[c], cv,
                        m1[c], m2, ah, al, bh, bl, n_in, n_out, n_nf, j * G.n1 + i, band);
                }
            }
        }
        if constexpr (BIN == 1 && MODE == MODE_BIN) {
            bin_tile<NTH, RY, CX>(pix, bp0, bp1, bq0, bq1, s_box,
                                  reinterpret_cast<int*>(&s_pos[0][0]), 2 * LT * 4, M.counts,
                                  G.npix);
        }
    }
    flush();
}

// ---- double-single (float-float) deflection ---------------------------------
// RS_PREC_DOUBLE_SINGLE: every term m (x - x_k)/|x - x_k|^2 is evaluated to
// about 2^-44 relative with error-free transformations on the FP32 pipe:
// Knuth's two-sum for the offsets and r^2, the FMA residual a*b - fl(a*b) for
// products (Dekker 1971), and the exact residual t = 1 - r^2 y0 of the MUFU
// reciprocal y0, so that 1/r^2 = y0 (1 + t) to second order.  Ray and lens
// offsets from the tile origin are split from FP64 into hi + lo, so no input
// is rounded to FP32.  Per ray and component the running sum is H + L: the
// term's leading product goes into H with one FMA, s = fl(H + d_h y0); the
// part of it that H took, z = s - H, is exact by Sterbenz's lemma because H
// starts at DS_OFFSET and so stays within a factor 2 of s (|term| <= H / 2
// for every lens farther than 2 / DS_OFFSET); what the rounding dropped,
// d_h y0 - z, is smaller than ulp(H) / 2 and is formed by a second FMA
// (exact to 2^-24 of itself, 2^-37 absolute) and added to L together with
// the first-order terms y0 (d_h t + d_l).  L is folded back into H every 16
// lenses and the offset is removed exactly at the end.  (A plain FP32
// partial sum would instead round at ulp of its largest term, which a lens
// next to the ray makes large.)  On B300 this costs about 28 FP32 lanes per
// interaction (4.2 interactions/clk/SM), ~25x the rate of an FP64 sum at
// 1.7 DFMA/clk/SM and ~10 FP64 operations per interaction.
constexpr int LT_DS = 512;       // lenses per shared-memory stage
constexpr float DS_OFFSET = 2048.f;   // start of the running sums (see above)
constexpr int LPT_DS = LT_DS / NT;
static_assert(LT_DS % NT == 0, "stage size");

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// s + e == a + b exactly (lane-wise)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e)
{
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

// hi + lo of a double
__device__ __forceinline__ void split_f32(double v, float& hi, float& lo)
{
    hi = __double2float_rn(v);
    lo = __double2float_rn(__dsub_rn(v, (double)hi));
}

template <int PX, int RY, bool UNIT, int MODE, int MAXB>
__global__ void __launch_bounds__(NT, 1)
shoot_kernel_ds(const __grid_constant__ LaunchArgs<MAXB> A)
{
    constexpr int CX = 2 * PX;
    constexpr int TX = TXT * CX;
    constexpr int TY = TYT * RY;
    // the current tile's map descriptor in shared memory (as shoot_kernel)
    __shared__ __align__(16) MapDesc s_map[MAXB > 1 ? 2 : 1];
    __shared__ __align__(16) float4 s_hi[2][LT_DS];   // {-xh, -xh, -yh, -yh}
    __shared__ __align__(16) float4 s_lo[2][LT_DS];   // {-xl, -xl, -yl, -yl}
    __shared__ __align__(8) float2 s_m[UNIT ? 1 : 2][UNIT ? 1 : LT_DS];   // {mh, ml}
    // epilogue terms per tile column and row, once per CTA (as in
    // shoot_kernel); two buffers by tile parity
    __shared__ FF s_cu[2][TX];
    __shared__ FF s_cv[2][TY];
    __shared__ double s_m1[MODE == MODE_DUMP ? 2 : 1][MODE == MODE_DUMP ? TX : 1];
    __shared__ double s_m2[MODE == MODE_DUMP ? 2 : 1][MODE == MODE_DUMP ? TY : 1];

    const int tx = threadIdx.x % TXT;
    const int ty = threadIdx.x / TXT;
    const float2 one2 = make_float2(1.f, 1.f);

    unsigned n_in = 0, n_out = 0, n_nf = 0;
    int cur_map = -1;
    auto flush = [&]() {
        if (MODE != MODE_BIN || cur_map < 0) return;
        const unsigned s_in = __reduce_add_sync(0xffffffffu, n_in);
        const unsigned s_out = __reduce_add_sync(0xffffffffu, n_out);
        const unsigned s_nf = __reduce_add_sync(0xffffffffu, n_nf);
        if ((threadIdx.x & 31) == 0) {
            unsigned long long* st = A.maps[cur_map].stats;
            if (s_in) atomicAdd(st + 0, (unsigned long long)s_in);
            if (s_out) atomicAdd(st + 1, (unsigned long long)s_out);
            if (s_nf) atomicAdd(st + 2, (unsigned long long)s_nf);
        }
        n_in = n_out = n_nf = 0;
    };

    int pb = 1;
    EpiTile T{};
    for (int64_t w = blockIdx.x; w < A.x.n_work; w += gridDim.x) {
        pb ^= 1;
        int mi = 0;
        if (MAXB > 1) {
            int lo = 0, hi = A.n_maps - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (A.tile_begin[mid] <= w) lo = mid; else hi = mid - 1;
            }
            mi = lo;
        }
        if (mi != cur_map) {
            flush();
            cur_map = mi;
            T = epi_tile(A.maps[mi].g);
        }
        const MapDesc* Mp = &A.maps[0];
        if constexpr (MAXB > 1) {
            const int* src = reinterpret_cast<const int*>(&A.maps[mi]);
            int* dst = reinterpret_cast<int*>(&s_map[MAXB > 1 ? pb : 0]);
            for (int q = threadIdx.x; q < (int)(sizeof(MapDesc) / 4); q += NT) dst[q] = src[q];
            __syncthreads();
            Mp = &s_map[MAXB > 1 ? pb : 0];
        }
        const MapDesc& M = *Mp;
        const Geometry& G = M.g;
        const int n_lens = M.n_lens;
        const int n_stage = (n_lens + LT_DS - 1) / LT_DS;
        const int64_t tile = (MODE == MODE_DUMP) ? A.x.tile_ids[w]
                                                 : M.tile0 + (w - A.tile_begin[mi]);
        const int64_t tj = tile / M.tiles1;
        const int64_t ti = tile - tj * M.tiles1;
        const int64_t i0 = ti * TX;
        const int64_t j0 = tj * TY;
        const double o1 = ray_pos(G.x0_1, G.d1, i0 + TX / 2);
        const double o2 = ray_pos(G.x0_2, G.d2, j0 + TY / 2);

        // epilogue terms in FP64 per tile column and row, one thread each
        // (read after the tile's first barrier)
        for (int k = threadIdx.x; k < TX + TY; k += NT) {
            double m;
            if (k < TX) {
                s_cu[pb][k] = epi_macro(G.one_m_g, G.kappa_s, ray_pos(G.x0_1, G.d1, i0 + k),
                                        G.y0_1, G.inv_w, m);
                if (MODE == MODE_DUMP) s_m1[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? k : 0] = m;
            } else {
                const int kr = k - TX;
                s_cv[pb][kr] = epi_macro(G.one_p_g, G.kappa_s, ray_pos(G.x0_2, G.d2, j0 + kr),
                                         G.y0_2, G.inv_w, m);
                if (MODE == MODE_DUMP) s_m2[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? kr : 0] = m;
            }
        }
        // ray offsets from the tile origin, hi + lo
        float2 xh[PX], xl[PX], yh[RY], yl[RY];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            float ah, al, bh, bl;
            split_f32(__dsub_rn(ray_pos(G.x0_1, G.d1, i0 + tx + TXT * (2 * p)), o1), ah, al);
            split_f32(__dsub_rn(ray_pos(G.x0_1, G.d1, i0 + tx + TXT * (2 * p + 1)), o1), bh, bl);
            xh[p] = make_float2(ah, bh);
            xl[p] = make_float2(al, bl);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            float h, l;
            split_f32(__dsub_rn(ray_pos(G.x0_2, G.d2, j0 + ty + TYT * r), o2), h, l);
            yh[r] = make_float2(h, h);
            yl[r] = make_float2(l, l);
        }

        // per ray and component: running sum H + L
        float2 Hx[RY][PX], Hy[RY][PX], Lx[RY][PX], Ly[RY][PX];
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
            for (int p = 0; p < PX; ++p)
            {
                // the running sums start at the offset DS_OFFSET (subtracted
                // exactly at the end), so that |H| >= |t| for every term of a
                // lens farther than 1/(DS_OFFSET/2) and Fast2Sum is exact
                Hx[r][p] = Hy[r][p] = make_float2(DS_OFFSET, DS_OFFSET);
                Lx[r][p] = Ly[r][p] = make_float2(0.f, 0.f);
            }

        double rx[LPT_DS], ryv[LPT_DS], rm[LPT_DS];
        auto load_stage = [&](int base) {
#pragma unroll
            for (int s = 0; s < LPT_DS; ++s) {
                const int k = base + threadIdx.x + NT * s;
                if (k < n_lens) {
                    rx[s] = __ldg(M.lx + k);
                    ryv[s] = __ldg(M.ly + k);
                    if (!UNIT) rm[s] = __ldg(M.lm + k);
                }
            }
        };
        auto store_stage = [&](int buf, int base) {
#pragma unroll
            for (int s = 0; s < LPT_DS; ++s) {
                const int idx = threadIdx.x + NT * s;
                if (base + idx < n_lens) {
                    float xhi, xlo, yhi, ylo;
                    split_f32(__dsub_rn(rx[s], o1), xhi, xlo);
                    split_f32(__dsub_rn(ryv[s], o2), yhi, ylo);
                    s_hi[buf][idx] = make_float4(-xhi, -xhi, -yhi, -yhi);
                    s_lo[buf][idx] = make_float4(-xlo, -xlo, -ylo, -ylo);
                    if (!UNIT) {
                        float mh, ml;
                        split_f32(rm[s], mh, ml);
                        s_m[UNIT ? 0 : buf][UNIT ? 0 : idx] = make_float2(mh, ml);
                    }
                }
            }
        };

        if (n_stage > 0) {
            load_stage(0);
            store_stage(0, 0);
            __syncthreads();
            for (int st = 0; st < n_stage; ++st) {
                const int buf = st & 1;
                const int base = st * LT_DS;
                const bool more = st + 1 < n_stage;
                if (more) load_stage(base + LT_DS);
                const int cnt = min(LT_DS, n_lens - base);
#pragma unroll 1
                for (int l = 0; l < cnt; ++l) {
                    const float4 Lh = s_hi[buf][l];
                    const float4 Ll = s_lo[buf][l];
                    float2 MH = one2, ML = make_float2(0.f, 0.f);
                    if (!UNIT) {
                        const float2 mm = s_m[UNIT ? 0 : buf][UNIT ? 0 : l];
                        MH = make_float2(mm.x, mm.x);
                        ML = make_float2(mm.y, mm.y);
                    }
                    // dx = x - x_k and dx^2 per column pair, hi + lo
                    float2 dxh[PX], dxl[PX], qxh[PX], qxl[PX];
#pragma unroll
                    for (int p = 0; p < PX; ++p) {
                        float2 e;
                        two_sum2(xh[p], make_float2(Lh.x, Lh.y), dxh[p], e);
                        dxl[p] = add2(e, add2(xl[p], make_float2(Ll.x, Ll.y)));
                        qxh[p] = mul2(dxh[p], dxh[p]);
                        qxl[p] = fma2(dxh[p], dxh[p], neg2(qxh[p]));
                        qxl[p] = fma2(add2(dxh[p], dxh[p]), dxl[p], qxl[p]);
                    }
#pragma unroll
                    for (int r = 0; r < RY; ++r) {
                        // dy terms are the same for both rays of a column pair:
                        // scalar arithmetic, pairs formed by register moves
                        float sh, se;
                        two_sum1(yh[r].x, Lh.z, sh, se);
                        const float sl = __fadd_rn(se, __fadd_rn(yl[r].x, Ll.z));
                        const float qh = __fmul_rn(sh, sh);
                        float ql = __fmaf_rn(sh, sh, -qh);
                        ql = __fmaf_rn(__fadd_rn(sh, sh), sl, ql);
                        const float2 dyh = make_float2(sh, sh), dyl = make_float2(sl, sl);
                        const float2 qyh = make_float2(qh, qh);
                        const float2 qyl = make_float2(ql, ql);
#pragma unroll
                        for (int p = 0; p < PX; ++p) {
                            // r^2 = dx^2 + dy^2
                            float2 r2h, r2e;
                            two_sum2(qxh[p], qyh, r2h, r2e);
                            const float2 r2l = add2(r2e, add2(qxl[p], qyl));
                            // 1/r^2 = y0 (1 + t) to second order: MUFU seed
                            // y0 and its exact residual t = 1 - r^2 y0
                            const float2 y0 = rcp2(r2h);
                            float2 t = fma2(neg2(r2h), y0, one2);
                            t = fma2(neg2(r2l), y0, t);
                            // each component d (d = dx or dy, hi + lo) adds
                            // m d / r^2 = d_h ih + lo: the hi product goes into H
                            // by an FMA, z = s - H is exact (Sterbenz: |term|
                            // <= H / 2), and the rounding d_h ih - z of that FMA,
                            // below ulp(H) / 2, is itself formed by an FMA; the
                            // lo terms are first order in the residuals
                            float2 ih = y0, dl = t;
                            if (!UNIT) {
                                ih = mul2(y0, MH);
                                const float2 rho = fma2(y0, MH, neg2(ih));
                                dl = fma2(ih, t, rho);
                                dl = fma2(ML, y0, dl);
                            }
                            auto add_term = [&](float2 dh, float2 dlo, float2& H, float2& Lo) {
                                const float2 s = fma2(dh, ih, H);
                                const float2 z = sub2(s, H);
                                Lo = add2(Lo, fma2(dh, ih, neg2(z)));
                                if (UNIT) {
                                    // lo = y0 (d_h t + d_l)
                                    Lo = fma2(y0, fma2(dh, t, dlo), Lo);
                                } else {
                                    // lo = d_h (m/r^2)_lo + d_l ih
                                    Lo = fma2(dh, dl, Lo);
                                    Lo = fma2(dlo, ih, Lo);
                                }
                                H = s;
                            };
                            add_term(dxh[p], dxl[p], Hx[r][p], Lx[r][p]);
                            add_term(dyh, dyl, Hy[r][p], Ly[r][p]);
                        }
                    }
                    if ((l & 15) == 15) {
                        // keep the low parts small: (H, L) <- Fast2Sum(H, L)
#pragma unroll
                        for (int r = 0; r < RY; ++r)
#pragma unroll
                            for (int p = 0; p < PX; ++p) {
                                float2 h = add2(Hx[r][p], Lx[r][p]);
                                Lx[r][p] = sub2(Lx[r][p], sub2(h, Hx[r][p]));
                                Hx[r][p] = h;
                                h = add2(Hy[r][p], Ly[r][p]);
                                Ly[r][p] = sub2(Ly[r][p], sub2(h, Hy[r][p]));
                                Hy[r][p] = h;
                            }
                    }
                }
                if (more) store_stage(buf ^ 1, base + LT_DS);
                __syncthreads();
            }
        } else {
            __syncthreads();      // no lenses: the per-column terms still need it
        }

        // remove the offset (exact: H lies within a factor 2 of DS_OFFSET) and
        // renormalise (H, L) with two-sum
#pragma unroll
        for (int r = 0; r < RY; ++r)
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                float2 s1, e1;
                two_sum2(sub2(Hx[r][p], make_float2(DS_OFFSET, DS_OFFSET)), Lx[r][p], s1, e1);
                Hx[r][p] = s1;
                Lx[r][p] = e1;
                two_sum2(sub2(Hy[r][p], make_float2(DS_OFFSET, DS_OFFSET)), Ly[r][p], s1, e1);
                Hy[r][p] = s1;
                Ly[r][p] = e1;
            }

        double m1[CX];
        FF cu[CX];
#pragma unroll
        for (int c = 0; c < CX; ++c) {
            cu[c] = s_cu[pb][tx + TXT * c];
            m1[c] = MODE == MODE_DUMP ? s_m1[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? tx + TXT * c : 0] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            const int64_t j = j0 + ty + TYT * r;
            const double m2 = MODE == MODE_DUMP ? s_m2[MODE == MODE_DUMP ? pb : 0][MODE == MODE_DUMP ? ty + TYT * r : 0] : 0.0;
            const FF cv = s_cv[pb][ty + TYT * r];
#pragma unroll
            for (int c = 0; c < CX; ++c) {
                const int64_t i = i0 + tx + TXT * c;
                const bool valid = (i < G.n1) && (j < G.n2);
                const int p = c >> 1;
                const bool b = c & 1;
                emit_ray<MODE>(M, A.x, T, w, TX * TY, (ty + TYT * r) * TX + (tx + TXT * c), valid,
                               cu[c], cv, m1[c], m2, b ? Hx[r][p].y : Hx[r][p].x,
                               b ? Lx[r][p].y : Lx[r][p].x, b ? Hy[r][p].y : Hy[r][p].x,
                               b ? Ly[r][p].y : Ly[r][p].x, n_in, n_out, n_nf);
            }
        }
    }
    flush();
}

// ---- RS_PREC_REFINED, second pass: the listed rays in double-single ------
// The rays the map kernel found near a pixel edge are shot again one by one
// (REF_RPT per thread, two per f32x2 lane pair) with the float-float
// arithmetic of shoot_kernel_ds, but from the origin x = 0 instead of a
// tile origin: ray and lens coordinates are split from FP64 into hi + lo,
// and dx = x - x_k comes out of a two-sum as a float-float accurate to
// ~2^-48 |x_k|, far below the FP32 rounding it replaces.  The lists of up to
// MAX_BATCH maps are cut into chunks of REF_CHUNK rays of one map each; a
// block takes one chunk at a time from a work counter (load balance without
// knowing the lists' lengths on the host), stages that map's lens list
// through shared memory, and bins its rays with the map kernel's epilogue.
constexpr int REF_NT = 128;
constexpr int REF_PAIRS = 2;                    // f32x2 ray pairs per thread
constexpr int REF_CHUNK = 2 * REF_PAIRS * REF_NT;
constexpr int REF_LT = 512;

struct RefineMap {
    Geometry g;
    const double* lx;
    const double* ly;
    const double* lm;
    int32_t n_lens;
    int32_t pad_;
    const int64_t* ids;
    const unsigned long long* count;    // {count, count3}
    int64_t cap;
    int32_t* counts;
    unsigned long long* stats;
    float eps3;                          // third-pass band in pixels
    int32_t pad2_;
};

struct RefineArgs {
    int32_t n_maps;
    int32_t pad_;
    unsigned long long* work;       // zeroed before the launch
    const int64_t* slots;           // dump mode (map 0): dump slot of every listed ray
    double* dump_y;
    int32_t* dump_pix;
    RefineMap maps[MAX_BATCH];
};
static_assert(sizeof(RefineArgs) <= 32764, "kernel parameter limit");

// one lens on one ray pair: the float-float term m d / r^2 of both
// components added to the offset running sums (as in shoot_kernel_ds)
template <bool UNIT>
__device__ __forceinline__ void refine_lens(float4 Lh, float4 Ll, float2 MH, float2 ML,
                                            float2 xh, float2 xl, float2 yh, float2 yl,
                                            float2& Hx, float2& Lx, float2& Hy, float2& Ly)
{
    const float2 one2 = make_float2(1.f, 1.f);
    float2 e, dxh, dyh;
    two_sum2(xh, make_float2(Lh.x, Lh.y), dxh, e);
    const float2 dxl = add2(e, add2(xl, make_float2(Ll.x, Ll.y)));
    two_sum2(yh, make_float2(Lh.z, Lh.w), dyh, e);
    const float2 dyl = add2(e, add2(yl, make_float2(Ll.z, Ll.w)));
    const float2 qxh = mul2(dxh, dxh);
    float2 qxl = fma2(dxh, dxh, neg2(qxh));
    qxl = fma2(add2(dxh, dxh), dxl, qxl);
    const float2 qyh = mul2(dyh, dyh);
    float2 qyl = fma2(dyh, dyh, neg2(qyh));
    qyl = fma2(add2(dyh, dyh), dyl, qyl);
    float2 r2h, r2e;
    two_sum2(qxh, qyh, r2h, r2e);
    const float2 r2l = add2(r2e, add2(qxl, qyl));
    const float2 y0 = rcp2(r2h);
    float2 t = fma2(neg2(r2h), y0, one2);
    t = fma2(neg2(r2l), y0, t);
    float2 ih = y0, dl = t;
    if (!UNIT) {
        ih = mul2(y0, MH);
        const float2 rho = fma2(y0, MH, neg2(ih));
        dl = fma2(ih, t, rho);
        dl = fma2(ML, y0, dl);
    }
    // x component
    float2 sum = fma2(dxh, ih, Hx);
    float2 z = sub2(sum, Hx);
    Lx = add2(Lx, fma2(dxh, ih, neg2(z)));
    if (UNIT) {
        Lx = fma2(y0, fma2(dxh, t, dxl), Lx);
    } else {
        Lx = fma2(dxh, dl, Lx);
        Lx = fma2(dxl, ih, Lx);
    }
    Hx = sum;
    // y component
    sum = fma2(dyh, ih, Hy);
    z = sub2(sum, Hy);
    Ly = add2(Ly, fma2(dyh, ih, neg2(z)));
    if (UNIT) {
        Ly = fma2(y0, fma2(dyh, t, dyl), Ly);
    } else {
        Ly = fma2(dyh, dl, Ly);
        Ly = fma2(dyl, ih, Ly);
    }
    Hy = sum;
}

template <bool UNIT, int MODE>
__global__ void __launch_bounds__(REF_NT, 4) refine_kernel(const __grid_constant__ RefineArgs R)
{
    __shared__ __align__(16) float4 s_hi[REF_LT];   // {-xh, -xh, -yh, -yh}
    __shared__ __align__(16) float4 s_lo[REF_LT];   // {-xl, -xl, -yl, -yl}
    __shared__ __align__(8) float2 s_m[UNIT ? 1 : REF_LT];
    __shared__ int64_t s_first[MAX_BATCH + 1];     // first chunk of every map
    __shared__ int64_t s_chunk;
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int m = 0; m < R.n_maps; ++m) {
            s_first[m] = acc;
            const int64_t listed = (int64_t)*R.maps[m].count;
            const int64_t tot = listed < R.maps[m].cap ? listed : R.maps[m].cap;
            acc += (tot + REF_CHUNK - 1) / REF_CHUNK;
        }
        s_first[R.n_maps] = acc;
    }
    __syncthreads();
    const int64_t n_chunks = s_first[R.n_maps];
    while (true) {
        if (threadIdx.x == 0) s_chunk = (int64_t)atomicAdd(R.work, 1ull);
        __syncthreads();
        const int64_t chunk = s_chunk;
        if (chunk >= n_chunks) break;
        // the chunk's map: the last one whose first chunk is at or before it
        int lo = 0, hi = R.n_maps - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= chunk) lo = mid; else hi = mid - 1;
        }
        const RefineMap& R1 = R.maps[lo];
        const Geometry& G = R1.g;
        const int64_t listed = (int64_t)*R1.count;
        const int64_t total = listed < R1.cap ? listed : R1.cap;
        const int64_t base = (chunk - s_first[lo]) * REF_CHUNK;
        const EpiTile T = epi_tile(G);
        unsigned n_in = 0, n_out = 0, n_nf = 0, n_ref = 0;
        // a-posteriori check: the first pass's error on the recomputed rays
        // (with stored images) against their bands
        float use_max = 0.f, dmax = 0.f;
        const int64_t aux = refine_aux_cap(R1.cap);
        const float4* uvs = refine_uv(const_cast<int64_t*>(R1.ids), R1.cap);
        const float* bands = refine_band(const_cast<int64_t*>(R1.ids), R1.cap);
        if (MODE == MODE_BIN && base == 0 && threadIdx.x == 0 && listed > R1.cap)
            atomicAdd(R1.stats + RS_STAT_OVERFLOW, (unsigned long long)(listed - R1.cap));
        // rays k0 + 2q and k0 + 2q + 1 form pair q
        const int64_t k0 = base + 2 * REF_PAIRS * threadIdx.x;
        int64_t id[2 * REF_PAIRS];
        double x1[2 * REF_PAIRS], x2[2 * REF_PAIRS];
        float2 xh[REF_PAIRS], xl[REF_PAIRS], yh[REF_PAIRS], yl[REF_PAIRS];
        float2 Hx[REF_PAIRS], Lx[REF_PAIRS], Hy[REF_PAIRS], Ly[REF_PAIRS];
#pragma unroll
        for (int r = 0; r < 2 * REF_PAIRS; ++r) {
            id[r] = k0 + r < total ? R1.ids[k0 + r] : (k0 < total ? R1.ids[k0] : 0);
            const int64_t i = id[r] % G.n1, j = id[r] / G.n1;
            x1[r] = ray_pos(G.x0_1, G.d1, i);
            x2[r] = ray_pos(G.x0_2, G.d2, j);
        }
#pragma unroll
        for (int q = 0; q < REF_PAIRS; ++q) {
            split_f32(x1[2 * q], xh[q].x, xl[q].x);
            split_f32(x1[2 * q + 1], xh[q].y, xl[q].y);
            split_f32(x2[2 * q], yh[q].x, yl[q].x);
            split_f32(x2[2 * q + 1], yh[q].y, yl[q].y);
            Hx[q] = Hy[q] = make_float2(DS_OFFSET, DS_OFFSET);
            Lx[q] = Ly[q] = make_float2(0.f, 0.f);
        }
        for (int l0 = 0; l0 < R1.n_lens; l0 += REF_LT) {
            const int cnt = min(REF_LT, R1.n_lens - l0);
            __syncthreads();                  // the previous stage is consumed
            for (int k = threadIdx.x; k < cnt; k += REF_NT) {
                float a, b, c, d;
                split_f32(__ldg(R1.lx + l0 + k), a, b);
                split_f32(__ldg(R1.ly + l0 + k), c, d);
                s_hi[k] = make_float4(-a, -a, -c, -c);
                s_lo[k] = make_float4(-b, -b, -d, -d);
                if (!UNIT) {
                    float mh, ml;
                    split_f32(__ldg(R1.lm + l0 + k), mh, ml);
                    s_m[UNIT ? 0 : k] = make_float2(mh, ml);
                }
            }
            __syncthreads();
            // blocks of 4 lenses, unrolled, L folded back into H after each
            // (|L| stays below 5 ulp(H) / 2: the third pass's bound); the
            // stage's last cnt % 4 lenses (fewer than 4) follow unfolded
            const int cnt4 = cnt & ~3;
#pragma unroll 1
            for (int l4 = 0; l4 < cnt4; l4 += 4) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int l = l4 + u;
                    const float4 Lh = s_hi[l];
                    const float4 Ll = s_lo[l];
                    float2 MH = make_float2(1.f, 1.f), ML = make_float2(0.f, 0.f);
                    if (!UNIT) {
                        const float2 mm = s_m[UNIT ? 0 : l];
                        MH = make_float2(mm.x, mm.x);
                        ML = make_float2(mm.y, mm.y);
                    }
#pragma unroll
                    for (int q = 0; q < REF_PAIRS; ++q)
                        refine_lens<UNIT>(Lh, Ll, MH, ML, xh[q], xl[q], yh[q], yl[q], Hx[q], Lx[q],
                                          Hy[q], Ly[q]);
                }
#pragma unroll
                for (int q = 0; q < REF_PAIRS; ++q) {
                    float2 h = add2(Hx[q], Lx[q]);
                    Lx[q] = sub2(Lx[q], sub2(h, Hx[q]));
                    Hx[q] = h;
                    h = add2(Hy[q], Ly[q]);
                    Ly[q] = sub2(Ly[q], sub2(h, Hy[q]));
                    Hy[q] = h;
                }
            }
#pragma unroll 1
            for (int l = cnt4; l < cnt; ++l) {
                const float4 Lh = s_hi[l];
                const float4 Ll = s_lo[l];
                float2 MH = make_float2(1.f, 1.f), ML = make_float2(0.f, 0.f);
                if (!UNIT) {
                    const float2 mm = s_m[UNIT ? 0 : l];
                    MH = make_float2(mm.x, mm.x);
                    ML = make_float2(mm.y, mm.y);
                }
#pragma unroll
                for (int q = 0; q < REF_PAIRS; ++q)
                    refine_lens<UNIT>(Lh, Ll, MH, ML, xh[q], xl[q], yh[q], yl[q], Hx[q], Lx[q],
                                      Hy[q], Ly[q]);
            }
        }
        int64_t* ids3 = refine_ids3(const_cast<int64_t*>(R1.ids), R1.cap);
        const int64_t cap3 = refine_cap3(R1.cap);
        unsigned n_ovf = 0;
#pragma unroll
        for (int q = 0; q < REF_PAIRS; ++q) {
            float2 ax, axl, ay, ayl;
            two_sum2(sub2(Hx[q], make_float2(DS_OFFSET, DS_OFFSET)), Lx[q], ax, axl);
            two_sum2(sub2(Hy[q], make_float2(DS_OFFSET, DS_OFFSET)), Ly[q], ay, ayl);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // every lane takes part (the third-pass list is warp-aggregated)
                const int r = 2 * q + h;
                const bool act = k0 + r < total;
                double m1, m2;
                const float ah = h ? ax.y : ax.x, al = h ? axl.y : axl.x;
                const float bh = h ? ay.y : ay.x, bl = h ? ayl.y : ayl.x;
                const FF cu = epi_macro(G.one_m_g, G.kappa_s, x1[r], G.y0_1, G.inv_w, m1);
                const FF cv = epi_macro(G.one_p_g, G.kappa_s, x2[r], G.y0_2, G.inv_w, m2);
                float uh, ul, vh, vl;
                ff_pixel_coord(cu, ah, al, T.sc, uh, ul);
                ff_pixel_coord(cv, bh, bl, T.sc, vh, vl);
                const bool finite = isfinite(ah) && isfinite(al) && isfinite(bh) && isfinite(bl);
                if (act && k0 + r < aux) {
                    const float4 c1 = uvs[k0 + r];
                    const float du = __fadd_rn(__fsub_rn(c1.x, uh), __fsub_rn(c1.y, ul));
                    const float dv = __fadd_rn(__fsub_rn(c1.z, vh), __fsub_rn(c1.w, vl));
                    const float d = fmaxf(fabsf(du), fabsf(dv));
                    if (d == d) {                  // finite images only
                        dmax = fmaxf(dmax, d);
                        use_max = fmaxf(use_max, d / bands[k0 + r]);
                    }
                }
                // rays whose double-single image lies within its error bound
                // of a pixel edge go on to the FP64 pass
                bool to3 = act && finite && ff_refine(uh, ul, vh, vl, T.np, R1.eps3);
                const unsigned m3 = __ballot_sync(0xffffffffu, to3);
                if (m3) {
                    const int lane = threadIdx.x & 31, lead = __ffs(m3) - 1;
                    unsigned long long b3 = 0;
                    if (lane == lead)
                        b3 = atomicAdd(const_cast<unsigned long long*>(R1.count) + 1,
                                       (unsigned long long)__popc(m3));
                    b3 = __shfl_sync(0xffffffffu, b3, lead);
                    const unsigned long long k3 = b3 + __popc(m3 & ((1u << lane) - 1u));
                    if (to3 && k3 < (unsigned long long)cap3) ids3[k3] = k0 + r;
                    else if (to3) {
                        to3 = false;               // list full: keeps its double-single pixel
                        ++n_ovf;
                    }
                }
                if (!act) continue;
                ++n_ref;
                if (to3 && MODE == MODE_BIN) continue;
                int pp, qq;
                classify_ray(T, true, cu, cv, ah, al, bh, bl, pp, qq, n_in, n_out, n_nf);
                if (MODE == MODE_BIN) {
                    if (pp >= 0 && RS_IN_RANGE(pp, G.npix) && RS_IN_RANGE(qq, G.npix))
                        atomicAdd(R1.counts + (int64_t)qq * G.npix + pp, 1);
                } else {
                    const int64_t ri = R.slots[k0 + r];
                    R.dump_y[2 * ri] = __dsub_rn(__dsub_rn(m1, (double)ah), (double)al);
                    R.dump_y[2 * ri + 1] = __dsub_rn(__dsub_rn(m2, (double)bh), (double)bl);
                    R.dump_pix[2 * ri] = pp;
                    R.dump_pix[2 * ri + 1] = qq;
                }
            }
        }
        if (MODE == MODE_BIN) {               // this chunk's statistics, to its map
            const unsigned s_in = __reduce_add_sync(0xffffffffu, n_in);
            const unsigned s_out = __reduce_add_sync(0xffffffffu, n_out);
            const unsigned s_nf = __reduce_add_sync(0xffffffffu, n_nf);
            const unsigned s_rf = __reduce_add_sync(0xffffffffu, n_ref);
            const unsigned s_ov = __reduce_add_sync(0xffffffffu, n_ovf);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                use_max = fmaxf(use_max, __shfl_xor_sync(0xffffffffu, use_max, o));
                dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
            }
            if ((threadIdx.x & 31) == 0) {
                if (s_in) atomicAdd(R1.stats + RS_STAT_IN, (unsigned long long)s_in);
                if (s_out) atomicAdd(R1.stats + RS_STAT_OUT, (unsigned long long)s_out);
                if (s_nf) atomicAdd(R1.stats + RS_STAT_NONFINITE, (unsigned long long)s_nf);
                if (s_rf) atomicAdd(R1.stats + RS_STAT_REFINED, (unsigned long long)s_rf);
                if (s_ov) atomicAdd(R1.stats + RS_STAT_OVERFLOW, (unsigned long long)s_ov);
                if (use_max > 0.f)
                    atomicMax(R1.stats + RS_STAT_BAND_USE,
                              (unsigned long long)fminf(use_max * 65536.f, 1.0e15f));
                if (dmax > 0.f)
                    atomicMax(R1.stats + RS_STAT_MAX_DELTA,
                              (unsigned long long)fminf(dmax * 4294967296.f, 1.0e15f));
            }
        }
        __syncthreads();                      // s_chunk is reused by the next chunk
    }
}

// ---- RS_PREC_REFINED, third pass: the rays nearest an edge in FP64 ---------
// The second pass lists the rays whose double-single image lies within that
// sum's error bound of a pixel edge; each is shot once more with Eq. 1 in
// FP64 (d = x - x_k, term d (m / r^2) with one division per lens, the
// macromodel term (1 - g) x - ks x minus the deflection, the pixel as the
// floor of (y - y0) times 1 / w).  One warp per ray: lane l sums the lenses
// l, l + 32, ... in index order and a butterfly of shuffles adds the 32
// partial sums (every lane ends with the same value), so the result differs
// from a sequential FP64 sum only by FP64 rounding.  FP64 runs at ~1.7
// operations per clock per SM on this part; the pass is cheap because the
// list is ~1e-5 of the rays.
constexpr int EX_NT = 256;

struct ExactMap {
    Geometry g;
    const double* lx;
    const double* ly;
    const double* lm;
    int32_t n_lens;
    int32_t unit;
    const int64_t* ids;          // the second pass's list (ray ids)
    const int64_t* ids3;         // positions in ids of the third pass's rays
    const unsigned long long* count;   // {count, count3}
    int64_t cap3;
    int32_t* counts;
    unsigned long long* stats;
};

struct ExactArgs {
    int32_t n_maps;
    int32_t pad_;
    unsigned long long* work;    // zeroed before the launch
    const int64_t* slots;        // dump mode (map 0): dump slot of every listed ray
    double* dump_y;
    int32_t* dump_pix;
    ExactMap maps[MAX_BATCH];
};
static_assert(sizeof(ExactArgs) <= 32764, "kernel parameter limit");

template <int MODE>
__global__ void __launch_bounds__(EX_NT) exact_kernel(const __grid_constant__ ExactArgs E)
{
    __shared__ int64_t s_first[MAX_BATCH + 1];
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int m = 0; m < E.n_maps; ++m) {
            s_first[m] = acc;
            const int64_t n3 = (int64_t)E.maps[m].count[1];
            acc += n3 < E.maps[m].cap3 ? n3 : E.maps[m].cap3;
        }
        s_first[E.n_maps] = acc;
    }
    __syncthreads();
    const int64_t total = s_first[E.n_maps];
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long gi = 0;
        if (lane == 0) gi = atomicAdd(E.work, 1ull);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if ((int64_t)gi >= total) break;
        int lo = 0, hi = E.n_maps - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_first[mid] <= (int64_t)gi) lo = mid; else hi = mid - 1;
        }
        const ExactMap& X = E.maps[lo];
        const Geometry& G = X.g;
        const int64_t k2 = X.ids3[(int64_t)gi - s_first[lo]];
        const int64_t id = X.ids[k2];
        const int64_t i = id % G.n1, j = id / G.n1;
        const double x1 = ray_pos(G.x0_1, G.d1, i);
        const double x2 = ray_pos(G.x0_2, G.d2, j);
        double s1 = 0.0, s2 = 0.0;
        bool sing = false;
        for (int k = lane; k < X.n_lens; k += 32) {
            const double d1 = __dsub_rn(x1, __ldg(X.lx + k));
            const double d2 = __dsub_rn(x2, __ldg(X.ly + k));
            const double r2 = __dadd_rn(__dmul_rn(d1, d1), __dmul_rn(d2, d2));
            sing = sing || r2 == 0.0;
            const double q = __ddiv_rn(X.unit ? 1.0 : __ldg(X.lm + k), r2);   // m / r^2
            s1 = __dadd_rn(s1, __dmul_rn(d1, q));
            s2 = __dadd_rn(s2, __dmul_rn(d2, q));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 = __dadd_rn(s1, __shfl_xor_sync(0xffffffffu, s1, o));
            s2 = __dadd_rn(s2, __shfl_xor_sync(0xffffffffu, s2, o));
        }
        sing = __any_sync(0xffffffffu, sing);
        if (lane == 0) {
            // Eq. 1 term by term, then the pixel
            const double y1 = __dsub_rn(__dsub_rn(__dmul_rn(G.one_m_g, x1), __dmul_rn(G.kappa_s, x1)), s1);
            const double y2 = __dsub_rn(__dsub_rn(__dmul_rn(G.one_p_g, x2), __dmul_rn(G.kappa_s, x2)), s2);
            const double u = __dmul_rn(__dsub_rn(y1, G.y0_1), G.inv_w);
            const double v = __dmul_rn(__dsub_rn(y2, G.y0_2), G.inv_w);
            const bool finite = !sing && isfinite(u) && isfinite(v);
            const bool in = finite && u >= 0.0 && v >= 0.0 && u < (double)G.npix && v < (double)G.npix;
            const int pp = in ? (int)floor(u) : -1, qq = in ? (int)floor(v) : -1;
            if (MODE == MODE_BIN) {
                if (in && RS_IN_RANGE(pp, G.npix) && RS_IN_RANGE(qq, G.npix))
                    atomicAdd(X.counts + (int64_t)qq * G.npix + pp, 1);
                atomicAdd(X.stats + (in ? RS_STAT_IN : finite ? RS_STAT_OUT : RS_STAT_NONFINITE), 1ull);
                atomicAdd(X.stats + RS_STAT_EXACT, 1ull);
            } else {
                const int64_t ri = E.slots[k2];
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                E.dump_y[2 * ri] = finite ? y1 : nan;
                E.dump_y[2 * ri + 1] = finite ? y2 : nan;
                E.dump_pix[2 * ri] = pp;
                E.dump_pix[2 * ri + 1] = qq;
            }
        }
    }
}

// ---- shape table and dispatch ---------------------------------------------
// px, ry: rays per thread (2 px columns x ry rows); pair: paired reciprocals;
// fold: lens groups of three between compensated folds (FP32 partial sums of
// 3 * fold lenses); f2s: fold with Fast2Sum; minb: CTAs per SM the register
// budget is sized for; unr: lens groups per unrolled loop body; full: all
// single-map variants (both precisions, general masses, per-ray dump) are
// compiled, otherwise only unit-mass map kernels (tuning candidates);
// batch: multi-map kernels (both precisions, both mass modes) exist;
// nth: threads per CTA (16 columns x nth/16 rows of threads); bin: 1 =
// tile binning through a shared-memory window with warp-aggregated atomics,
// 0 = one global atomic per ray; runr, rfold: the refined form's first pass
// on this shape (lens groups per unrolled loop body, groups between folds;
// runr = 0: no refined kernels).  The refined form's error bound (rs.h,
// RS_REFINE_*) covers FP32 partial sums of up to 48 lenses, so rfold <= 16.
// (The lens-stage size LT is not a tuning parameter: it must be a multiple
// of the group size and of the CTA's threads, so 768 for 256 threads, and
// 1536 no longer fits static shared memory; one stage barrier per 768
// lenses is 0.05% of the lens loop.)
struct Shape {
    int px, ry, pair, fold, f2s, minb, unr, full, batch, nth, bin, runr, rfold;
};
// shape ids 1..N; 0 selects the default
constexpr Shape kShapes[] = {
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0},      // 0: placeholder (default)
    {1, 4, 1, 16, 0, 2, 1, 1, 0, 256, 0, 0, 0},   // 1: 8 rays/thread, paired reciprocals, tile 32 x 64
    {2, 4, 1, 16, 0, 1, 1, 1, 0, 256, 0, 0, 0},   // 2: 16 rays/thread, paired, tile 64 x 64
    {1, 8, 1, 16, 0, 1, 1, 1, 0, 256, 0, 0, 0},   // 3: 16 rays/thread, paired, tile 32 x 128
    {1, 4, 0, 16, 0, 2, 1, 1, 0, 256, 0, 0, 0},   // 4: 8 rays/thread, one MUFU per interaction
    {2, 4, 0, 16, 0, 1, 1, 1, 0, 256, 0, 0, 0},   // 5: 16 rays/thread, one MUFU per interaction
    {2, 4, 1, 8, 0, 1, 1, 0, 0, 256, 0, 0, 0},    // 6: as 2, fold every 24 lenses
    {2, 4, 1, 4, 0, 1, 1, 0, 0, 256, 0, 0, 0},    // 7: as 2, fold every 12 lenses
    {2, 4, 1, 8, 1, 1, 1, 1, 0, 256, 0, 0, 0},    // 8: as 6 with Fast2Sum
    {2, 4, 1, 4, 1, 1, 1, 1, 0, 256, 0, 0, 0},    // 9: as 7 with Fast2Sum
    {2, 4, 1, 2, 1, 1, 1, 0, 0, 256, 0, 0, 0},    // 10: as 2, Fast2Sum every 6 lenses
    {2, 4, 0, 4, 1, 1, 1, 0, 0, 256, 0, 0, 0},    // 11: as 9 without paired reciprocals
    {2, 4, 1, 8, 1, 1, 2, 1, 1, 256, 0, 8, 16},    // 12: as 8, two groups per loop body (default); refined: 8 groups, folds of 48
    {2, 2, 1, 8, 1, 2, 1, 0, 0, 256, 0, 0, 0},    // 13: 8 rays/thread (64 x 32), 2 CTAs/SM
    {2, 2, 1, 8, 1, 2, 2, 0, 1, 256, 0, 0, 0},    // 14: as 13, two groups per loop body
    {1, 4, 1, 8, 1, 2, 2, 0, 1, 256, 0, 0, 0},    // 15: 8 rays/thread (32 x 64), unrolled
    {4, 2, 1, 8, 1, 1, 1, 0, 1, 256, 0, 0, 0},    // 16: 16 rays/thread (128 x 32)
    {2, 8, 1, 8, 1, 1, 1, 0, 0, 256, 0, 0, 0},    // 17: 32 rays/thread (64 x 128)
    {2, 2, 1, 8, 1, 3, 1, 0, 0, 256, 0, 0, 0},    // 18: as 13, 3 CTAs/SM
    {1, 4, 1, 8, 1, 3, 1, 0, 0, 256, 0, 0, 0},    // 19: 8 rays/thread, 3 CTAs/SM
    {2, 4, 1, 8, 1, 1, 2, 0, 1, 384, 0, 0, 0},    // 20: as 12 with 384 threads (64 x 96 tile)
    {1, 4, 1, 8, 1, 1, 2, 0, 1, 384, 0, 0, 0},    // 21: 8 rays/thread, 384 threads (32 x 96)
    {2, 4, 1, 8, 1, 1, 1, 0, 0, 384, 0, 0, 0},    // 22: as 20, one group per loop body
    {2, 4, 2, 6, 1, 1, 2, 0, 0, 256, 0, 0, 0},    // 23: as 12, groups of 4 with one shared reciprocal
    {2, 4, 3, 12, 1, 1, 2, 0, 0, 256, 0, 0, 0},   // 24: as 12, every two lenses share a reciprocal
    {2, 4, 4, 4, 1, 1, 1, 0, 0, 256, 0, 0, 0},    // 25: as 12, groups of 6 with one shared reciprocal
    {2, 4, 2, 6, 1, 1, 1, 0, 0, 256, 0, 0, 0},    // 26: as 23, one group per loop body
    {2, 4, 1, 8, 1, 1, 2, 1, 1, 256, 1, 0, 0},  // 27: as 12, shared-memory window binning
    {2, 4, 1, 16, 1, 1, 4, 0, 1, 256, 0, 4, 16},  // 28: as 12, folds of 48 lenses, 4 groups per body (both forms)
    {2, 4, 1, 8, 1, 1, 2, 0, 1, 256, 0, 2, 8},    // 29: as 12; refined: 2 groups per body, folds of 24
    {2, 4, 1, 16, 1, 1, 8, 0, 1, 256, 0, 8, 8},   // 30: folds of 48, 8 groups per body; refined: folds of 24
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);
constexpr int kDefaultShape = 12;

template <int MAXB>
using KernelFn = void (*)(const LaunchArgs<MAXB>);

template <int PX, int RY, int PAIR, int MINB, int UNR, bool FULL, int NTH, int BIN>
KernelFn<1> pick1(int precision, bool unit, int mode)
{
#define RS_K(P, U, MO) shoot_kernel<PX, RY, PAIR, P, U, MO, MINB, UNR, 1, NTH, BIN>
    if constexpr (!FULL) {
        if (!unit || mode != MODE_BIN) return nullptr;
        return precision == RS_PREC_FP32 ? RS_K(0, true, MODE_BIN) : RS_K(1, true, MODE_BIN);
    } else {
        if (precision == RS_PREC_FP32) {
            if (unit) return mode == MODE_BIN ? RS_K(0, true, MODE_BIN) : RS_K(0, true, MODE_DUMP);
            return mode == MODE_BIN ? RS_K(0, false, MODE_BIN) : RS_K(0, false, MODE_DUMP);
        }
        if (unit) return mode == MODE_BIN ? RS_K(1, true, MODE_BIN) : RS_K(1, true, MODE_DUMP);
        return mode == MODE_BIN ? RS_K(1, false, MODE_BIN) : RS_K(1, false, MODE_DUMP);
    }
#undef RS_K
}

template <int PX, int RY, int PAIR, int MINB, int UNR, bool BATCH, int NTH, int BIN>
KernelFn<MAX_BATCH> pickB(int precision, bool unit)
{
#define RS_K(P, U) shoot_kernel<PX, RY, PAIR, P, U, MODE_BIN, MINB, UNR, MAX_BATCH, NTH, BIN>
    if constexpr (!BATCH) {
        return nullptr;
    } else {
        if (precision == RS_PREC_FP32) return unit ? RS_K(0, true) : RS_K(0, false);
        return unit ? RS_K(1, true) : RS_K(1, false);
    }
#undef RS_K
}

// The refined form's first pass (64 x 64 tiles, paired reciprocals, Fast2Sum
// folds) with UNR lens groups per loop body; per-ray dump mode if DUMP.
template <int UNR, bool DUMP>
void pick_refined(bool unit, int mode, KernelFn<1>* k1, KernelFn<MAX_BATCH>* kb)
{
#define RS_R(U, MO, MB) shoot_kernel<2, 4, 1, RS_PREC_REFINED, U, MO, 1, UNR, MB, 256, 0>
    if (kb && mode == MODE_BIN) *kb = unit ? RS_R(true, MODE_BIN, MAX_BATCH) : RS_R(false, MODE_BIN, MAX_BATCH);
    if (k1) {
        if (mode == MODE_BIN) *k1 = unit ? RS_R(true, MODE_BIN, 1) : RS_R(false, MODE_BIN, 1);
        else if constexpr (DUMP) *k1 = unit ? RS_R(true, MODE_DUMP, 1) : RS_R(false, MODE_DUMP, 1);
    }
#undef RS_R
}

#define RS_SHAPE_B(PX, RY, PAIR, MINB, UNR, FULL, BATCH, NTH, BIN)                              \
    if (s.px == PX && s.ry == RY && s.pair == PAIR && s.minb == MINB && s.unr == UNR &&         \
        s.full == FULL && s.batch == BATCH && s.nth == NTH && s.bin == BIN) {                   \
        if (k1) *k1 = pick1<PX, RY, PAIR, MINB, UNR, FULL, NTH, BIN>(precision, unit, mode);    \
        if (kb) *kb = pickB<PX, RY, PAIR, MINB, UNR, BATCH, NTH, BIN>(precision, unit);         \
        return;                                                                                 \
    }
#define RS_SHAPE(PX, RY, PAIR, MINB, UNR, FULL, BATCH, NTH) \
    RS_SHAPE_B(PX, RY, PAIR, MINB, UNR, FULL, BATCH, NTH, 0)

void select_kernels(int shape, int precision, bool unit, int mode, KernelFn<1>* k1,
                    KernelFn<MAX_BATCH>* kb)
{
    if (k1) *k1 = nullptr;
    if (kb) *kb = nullptr;
    if (precision == RS_PREC_DOUBLE_SINGLE) {
        // one tile shape (64 x 64, 16 rays per thread) for the double-single sum
        if (shape != kDefaultShape) return;
        if (k1) {
            if (unit) *k1 = mode == MODE_BIN ? shoot_kernel_ds<2, 4, true, MODE_BIN, 1>
                                             : shoot_kernel_ds<2, 4, true, MODE_DUMP, 1>;
            else *k1 = mode == MODE_BIN ? shoot_kernel_ds<2, 4, false, MODE_BIN, 1>
                                        : shoot_kernel_ds<2, 4, false, MODE_DUMP, 1>;
        }
        if (kb) *kb = unit ? shoot_kernel_ds<2, 4, true, MODE_BIN, MAX_BATCH>
                           : shoot_kernel_ds<2, 4, false, MODE_BIN, MAX_BATCH>;
        return;
    }
    if (precision == RS_PREC_REFINED) {
        // the compensated kernel with the refinement epilogue on the shapes
        // that have one (runr); per-ray dump mode for the 8-group unroll
        switch (kShapes[shape].runr) {
        case 8: pick_refined<8, true>(unit, mode, k1, kb); break;
        case 4: pick_refined<4, false>(unit, mode, k1, kb); break;
        case 2: pick_refined<2, false>(unit, mode, k1, kb); break;
        default: break;
        }
        return;
    }
    const Shape& s = kShapes[shape];
    RS_SHAPE(1, 4, 1, 2, 1, 1, 0, 256)
    RS_SHAPE(2, 4, 1, 1, 1, 1, 0, 256)
    RS_SHAPE(1, 8, 1, 1, 1, 1, 0, 256)
    RS_SHAPE(1, 4, 0, 2, 1, 1, 0, 256)
    RS_SHAPE(2, 4, 0, 1, 1, 1, 0, 256)
    RS_SHAPE(2, 4, 1, 1, 1, 0, 0, 256)
    RS_SHAPE(2, 4, 0, 1, 1, 0, 0, 256)
    RS_SHAPE(2, 4, 1, 1, 2, 1, 1, 256)
    RS_SHAPE(2, 2, 1, 2, 1, 0, 0, 256)
    RS_SHAPE(2, 2, 1, 2, 2, 0, 1, 256)
    RS_SHAPE(1, 4, 1, 2, 2, 0, 1, 256)
    RS_SHAPE(4, 2, 1, 1, 1, 0, 1, 256)
    RS_SHAPE(2, 8, 1, 1, 1, 0, 0, 256)
    RS_SHAPE(2, 2, 1, 3, 1, 0, 0, 256)
    RS_SHAPE(1, 4, 1, 3, 1, 0, 0, 256)
    RS_SHAPE(2, 4, 1, 1, 2, 0, 1, 384)
    RS_SHAPE(1, 4, 1, 1, 2, 0, 1, 384)
    RS_SHAPE(2, 4, 1, 1, 1, 0, 0, 384)
    RS_SHAPE(2, 4, 2, 1, 2, 0, 0, 256)
    RS_SHAPE(2, 4, 3, 1, 2, 0, 0, 256)
    RS_SHAPE(2, 4, 4, 1, 1, 0, 0, 256)
    RS_SHAPE(2, 4, 2, 1, 1, 0, 0, 256)
    RS_SHAPE_B(2, 4, 1, 1, 2, 1, 1, 256, 1)
    RS_SHAPE(2, 4, 1, 1, 4, 0, 1, 256)
    RS_SHAPE(2, 4, 1, 1, 2, 0, 1, 256)
    RS_SHAPE(2, 4, 1, 1, 8, 0, 1, 256)
}
#undef RS_SHAPE
#undef RS_SHAPE_B

// Dynamic shared memory of a map-kernel launch: the per-thread slots of the
// error-bound sums (refined form) and of the coherent-rounding correction
// (any map of the launch off the 2^-12 spacing grid).
size_t field_smem(const MapDesc* maps, int n_maps, int precision, int nth)
{
    if (precision == RS_PREC_DOUBLE_SINGLE) return 0;      // float-float offsets: exact
    bool corr = false;
    for (int k = 0; k < n_maps; ++k) corr = corr || (maps[k].g.flags & GEO_COHERENT);
    if (corr) return (size_t)PV_ALL * nth * sizeof(float);
    if (precision == RS_PREC_REFINED) return (size_t)PV_J * nth * sizeof(float);
    return 0;
}
constexpr size_t FIELD_SMEM_MAX = (size_t)PV_ALL * 384 * sizeof(float);

// Resident CTAs per SM for a kernel with `dyn` bytes of dynamic shared
// memory on the current device (cached); raises the kernel's dynamic shared
// memory limit to the largest the launcher asks for on first use.
int resident_ctas(const void* fn, int nth, size_t dyn = 0)
{
    struct Entry { const void* fn; int dev; size_t dyn; int occ; };
    static Entry cache[1024];
    static int n_cache = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    for (int k = 0; k < n_cache; ++k)
        if (cache[k].fn == fn && cache[k].dev == dev && cache[k].dyn == dyn) return cache[k].occ;
    cudaFuncAttributes fa;
    int occ = 0;
    if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess &&
        fa.maxDynamicSharedSizeBytes < (int)FIELD_SMEM_MAX &&
        FIELD_SMEM_MAX + fa.sharedSizeBytes <= 227 * 1024)
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FIELD_SMEM_MAX);
    cudaGetLastError();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nth, dyn) != cudaSuccess || occ < 1)
        occ = 1;
    cudaGetLastError();
    if (n_cache < 1024) cache[n_cache++] = Entry{fn, dev, dyn, occ};
    return occ;
}

template <int MAXB>
int do_launch(KernelFn<MAXB> fn, const MapDesc* maps, int n_maps, const ShootExtra& x,
              const Shape& sh, int64_t tuning_cap, int precision, cudaStream_t stream)
{
    LaunchArgs<MAXB> a;
    memset(&a, 0, sizeof a);
    a.n_maps = n_maps;
    a.fold_groups = precision == RS_PREC_REFINED ? sh.rfold : sh.fold;
    a.fast2sum = sh.f2s;
    a.x = x;
    const int tx = TXT * 2 * sh.px, ty = (sh.nth / TXT) * sh.ry;
    int64_t acc = 0;
    for (int k = 0; k < n_maps; ++k) {
        a.maps[k] = maps[k];
        a.maps[k].tiles1 = (maps[k].g.n1 + tx - 1) / tx;
        const int64_t tiles2 = (maps[k].g.n2 + ty - 1) / ty;
        int64_t nt = maps[k].g.n1 > 0 ? a.maps[k].tiles1 * tiles2 : 0;
        nt -= maps[k].tile0;
        if (nt < 0) nt = 0;
        if (maps[k].tile_count > 0 && nt > maps[k].tile_count) nt = maps[k].tile_count;
        if (tuning_cap > 0 && nt > tuning_cap) nt = tuning_cap;
        a.tile_begin[k] = acc;
        acc += nt;
    }
    a.tile_begin[n_maps] = acc;
    if (!x.tile_ids) a.x.n_work = acc;
    if (a.x.n_work <= 0) return RS_OK;
    const size_t dyn = field_smem(maps, n_maps, precision, sh.nth);
    const int64_t cap = (int64_t)num_sms() * resident_ctas((const void*)fn, sh.nth, dyn);
    const int grid = (int)(a.x.n_work < cap ? a.x.n_work : cap);
    fn<<<grid, sh.nth, dyn, stream>>>(a);
    return cuda_fail(cudaGetLastError(), "shoot kernel launch");
}

}  // namespace

int shape_info(int shape, int precision, ShapeInfo* out)
{
    if (precision != RS_PREC_FP32 && precision != RS_PREC_COMPENSATED &&
        precision != RS_PREC_DOUBLE_SINGLE && precision != RS_PREC_REFINED)
        return fail(RS_EINVAL, "precision %d is not one of RS_PREC_*", precision);
    if (shape < 0 || shape >= kNumShapes)
        return fail(RS_EINVAL, "shape %d out of range [0, %d)", shape, kNumShapes);
    if (shape == 0) shape = kDefaultShape;
    if (precision == RS_PREC_DOUBLE_SINGLE && shape != kDefaultShape)
        return fail(RS_EINVAL, "double-single precision runs only the default shape %d",
                    kDefaultShape);
    if (precision == RS_PREC_REFINED && kShapes[shape].runr == 0)
        return fail(RS_EINVAL, "shape %d has no refined kernels", shape);
    const Shape& s = kShapes[shape];
    out->px = s.px;
    out->ry = s.ry;
    out->pair = s.pair;
    out->fold = precision == RS_PREC_REFINED ? s.rfold : s.fold;
    out->fold_lenses = out->fold * pair_grp(s.pair);
    out->unroll = precision == RS_PREC_REFINED ? s.runr : s.unr;
    out->fast2sum = s.f2s;
    out->tx = TXT * 2 * s.px;
    out->ty = (s.nth / TXT) * s.ry;
    out->batch = s.batch;
    return RS_OK;
}

int batch_candidates(int precision, int* shapes, int max)
{
    int n = 0;
    if (n < max) shapes[n++] = kDefaultShape;
    if (precision == RS_PREC_DOUBLE_SINGLE) return n;
    for (int k = 1; k < kNumShapes && n < max; ++k) {
        const bool ok = precision == RS_PREC_REFINED ? kShapes[k].runr != 0 : kShapes[k].batch != 0;
        if (ok && k != kDefaultShape) shapes[n++] = k;
    }
    return n;
}

int prime_launch(int shape, int precision, bool unit_mass, bool batched)
{
    if (shape == 0) shape = kDefaultShape;
    if (shape < 1 || shape >= kNumShapes) return fail(RS_EINVAL, "shape %d out of range", shape);
    KernelFn<1> k1 = nullptr;
    KernelFn<MAX_BATCH> kb = nullptr;
    select_kernels(shape, precision, unit_mass, MODE_BIN, &k1, &kb);
    num_sms();
    if (batched ? !kb : !k1) return fail(RS_EINVAL, "shape %d has no such kernel", shape);
    const void* fn = batched ? (const void*)kb : (const void*)k1;
    const int nth = kShapes[shape].nth;
    resident_ctas(fn, nth, 0);
    resident_ctas(fn, nth, (size_t)PV_J * nth * sizeof(float));
    resident_ctas(fn, nth, (size_t)PV_ALL * nth * sizeof(float));
    return RS_OK;
}

bool has_single_kernel(int shape, int precision, bool unit_mass)
{
    if (shape == 0) shape = kDefaultShape;
    if (shape < 1 || shape >= kNumShapes) return false;
    KernelFn<1> k1 = nullptr;
    select_kernels(shape, precision, unit_mass, MODE_BIN, &k1, nullptr);
    return k1 != nullptr;
}

bool own_launch(const MapDesc& m, int shape, int precision, bool unit_mass)
{
    if (shape == 0) shape = kDefaultShape;
    if (shape < 1 || shape >= kNumShapes) return false;
    KernelFn<1> k1 = nullptr;
    select_kernels(shape, precision, unit_mass, MODE_BIN, &k1, nullptr);
    if (!k1) return false;
    const Shape& sh = kShapes[shape];
    const int tx = TXT * 2 * sh.px, ty = (sh.nth / TXT) * sh.ry;
    if (m.g.n1 <= 0 || m.g.n2 <= 0) return false;
    int64_t nt = ((m.g.n1 + tx - 1) / tx) * ((m.g.n2 + ty - 1) / ty) - m.tile0;
    if (m.tile_count > 0 && nt > m.tile_count) nt = m.tile_count;
    const int64_t wave =
        (int64_t)num_sms() * resident_ctas((const void*)k1, sh.nth, field_smem(&m, 1, precision, sh.nth));
    return nt >= 8 * wave;
}

int launch_shoot(const MapDesc* maps, int n_maps, const ShootExtra& x, int shape, int precision,
                 bool unit_mass, int mode, cudaStream_t stream, int64_t tuning_cap, bool batched)
{
    if (shape == 0) shape = kDefaultShape;
    if (shape < 1 || shape >= kNumShapes) return fail(RS_EINVAL, "shape %d out of range", shape);
    if (n_maps < 1 || n_maps > MAX_BATCH)
        return fail(RS_EINVAL, "%d maps in one launch (1..%d)", n_maps, MAX_BATCH);
    const Shape& sh = kShapes[shape];
    if (precision == RS_PREC_REFINED) {
        bool lists = mode == MODE_BIN || (n_maps == 1 && x.refine_slots);
        for (int k = 0; k < n_maps && lists; ++k)
            lists = maps[k].refine_ids && maps[k].refine_count;
        if (!lists)
            return fail(RS_EINVAL, "refined precision needs a ray list per map (rs_shoot_map, "
                                   "rs_shoot_map_host, rs_shoot_batch)");
    }
    KernelFn<1> k1 = nullptr;
    KernelFn<MAX_BATCH> kb = nullptr;
    select_kernels(shape, precision, unit_mass, mode, &k1, &kb);
    if (n_maps == 1 && tuning_cap == 0 && !batched) {
        if (!k1)
            return fail(RS_EINVAL, "shape %d is a tuning candidate compiled only for unit-mass "
                                   "batched or map launches", shape);
        return do_launch<1>(k1, maps, 1, x, sh, 0, precision, stream);
    }
    if (!kb || mode != MODE_BIN)
        return fail(RS_EINVAL, "shape %d has no batched kernel", shape);
    return do_launch<MAX_BATCH>(kb, maps, n_maps, x, sh, tuning_cap, precision, stream);
}

int launch_refine(const MapDesc* maps, int n_maps, unsigned long long* work, bool unit_mass,
                  cudaStream_t stream, const ShootExtra* dump)
{
    if (n_maps < 1 || n_maps > MAX_BATCH || (dump && n_maps != 1))
        return fail(RS_EINVAL, "%d maps in one refinement launch", n_maps);
    RefineArgs R;
    ExactArgs E;
    memset(&R, 0, sizeof R);
    memset(&E, 0, sizeof E);
    R.n_maps = E.n_maps = n_maps;
    R.work = work;
    E.work = work + 1;
    for (int k = 0; k < n_maps; ++k) {
        const MapDesc& d = maps[k];
        RefineMap& r = R.maps[k];
        r.g = d.g;
        r.lx = d.lx;
        r.ly = d.ly;
        r.lm = d.lm;
        r.n_lens = d.n_lens;
        r.ids = d.refine_ids;
        r.count = d.refine_count;
        r.cap = d.refine_cap;
        r.counts = d.counts;
        r.stats = d.stats;
        // the second pass's error bound (Hoeffding, K = RS_REFINE_K): per
        // term, the running sum's low part L (|L| < 5 ulp(H) / 2 = 5 2^-13
        // between folds every 4 lenses) takes up to three FP32 roundings of
        // at most 5 2^-37 and the captured residual one of 2^-37, 9 2^-37 in
        // quadrature; plus 2^-36 for the split inputs and the second-order
        // reciprocal residual
        const double eps_r = RS_REFINE_K * 9.0 * ldexp(1.0, -37) * sqrt((double)(d.n_lens > 0 ? d.n_lens : 1)) +
                             ldexp(1.0, -36);
        r.eps3 = (float)(eps_r * d.g.inv_w + ldexp(1.0, -28));
        ExactMap& x = E.maps[k];
        x.g = d.g;
        x.lx = d.lx;
        x.ly = d.ly;
        x.lm = d.lm;
        x.n_lens = d.n_lens;
        x.unit = unit_mass ? 1 : 0;
        x.ids = d.refine_ids;
        x.ids3 = refine_ids3(d.refine_ids, d.refine_cap);
        x.count = d.refine_count;
        x.cap3 = refine_cap3(d.refine_cap);
        x.counts = d.counts;
        x.stats = d.stats;
    }
    void (*k)(RefineArgs);
    void (*k3)(ExactArgs);
    if (dump) {
        R.slots = E.slots = dump->refine_slots;
        R.dump_y = E.dump_y = dump->dump_y;
        R.dump_pix = E.dump_pix = dump->dump_pix;
        k = unit_mass ? refine_kernel<true, MODE_DUMP> : refine_kernel<false, MODE_DUMP>;
        k3 = exact_kernel<MODE_DUMP>;
    } else {
        k = unit_mass ? refine_kernel<true, MODE_BIN> : refine_kernel<false, MODE_BIN>;
        k3 = exact_kernel<MODE_BIN>;
    }
    const int grid = num_sms() * resident_ctas((const void*)k, REF_NT, 0);
    k<<<grid, REF_NT, 0, stream>>>(R);
    int rc = cuda_fail(cudaGetLastError(), "refine launch");
    if (rc) return rc;
    const int grid3 = num_sms() * resident_ctas((const void*)k3, EX_NT, 0);
    k3<<<grid3, EX_NT, 0, stream>>>(E);
    return cuda_fail(cudaGetLastError(), "exact pass launch");
}

}  // namespace rs

extern "C" {

int rs_checked_violations(int64_t* out)
{
    rs::clear_error();
    if (!out) return rs::fail(RS_EINVAL, "out is NULL");
#ifdef RS_CHECKED
    unsigned long long v = 0, zero = 0;
    int rc = rs::cuda_fail(cudaMemcpyFromSymbol(&v, rs::g_checked_bad, sizeof v), "checked counter");
    if (!rc) rc = rs::cuda_fail(cudaMemcpyToSymbol(rs::g_checked_bad, &zero, sizeof zero),
                                "checked counter reset");
    if (rc) return rc;
    *out = (int64_t)v;
    return 1;
#else
    *out = 0;
    return 0;
#endif
}

}  // extern "C"
