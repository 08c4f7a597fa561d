// rs_fft.cu -- the two-dimensional real FFTs of Eq. 6 (finite-source
// convolution, Sec. 2.4) as three HBM passes of shared-memory transforms.
//
// For an n x n map (n a multiple of 4, n/2 of the form 2^a 3^b 5^c, n <= 10240):
//   pass A  rows, real to complex: each CTA takes 2 rows (ROWS), packs each as n/2
//           complex values z_k = x_2k + i x_2k+1, transforms them in shared
//           memory and separates the spectra of the even and odd samples
//           (X_k = E_k + w^k O_k, w = exp(-2 pi i / n)); it writes the n/2 + 1
//           bins of its 2 rows transposed, T[k][row], 16 contiguous bytes per
//           bin (the neighbouring CTA fills the rest of the 32-byte sector
//           while it is in L2).  int32 count maps are converted to float on
//           the way in.
//   pass B  columns: each CTA takes one row of T (one column of the map's
//           spectrum, n complex values, contiguous), transforms it forward,
//           multiplies by the same row of the kernel's spectrum and the
//           scale, and transforms it back -- any of the three steps can be
//           left out (kernel spectra, loaded maps).
//   pass C  rows, complex to real: each CTA gathers its 2 rows' n/2 + 1 bins
//           from T, rebuilds the half-length complex spectrum
//           (E_k + i O_k from X_k and conj X_(n/2-k)), transforms it back and
//           writes the real rows.
// Every transform is an unnormalised in-place Cooley-Tukey FFT in shared
// memory with radices 8, 4, 2, 5, 3; the twiddles of each stage come from
// that stage's own table of block roots, and the separation's from a table
// of the n-th roots of unity, all computed in FP64 on the host.  Forward
// transforms run by decimation in frequency (natural order in,
// digit-reversed order out), inverse ones by decimation in time
// (digit-reversed in, natural out).  A butterfly reads and writes the same
// R slots, so a thread holds one butterfly at a time.  Transform lengths
// that are multiples of 256 use a padded shared-memory layout (see pix)
// that keeps their short-span stages and digit-reversed gathers off a few
// banks.  Passes A and C absorb the row transforms' digit
// reversal where they read and write the spectrum; the column spectra stay
// digit-reversed (the kernel's and the map's alike), which the product and
// the inverse column transform need no permutation for.  The transforms are
// unnormalised, so a convolution carries 1 / n^2 in the product's scale.
// HBM traffic per convolved map: pass A reads the map (4 B/px) and writes
// the spectrum (~4 B/px), pass B reads it and the kernel's spectrum and
// writes it back (~12 B/px), pass C reads it and writes the map (~8 B/px):
// ~28 B/px.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr int FFT_T = 512;          // threads per CTA of the column pass (two CTAs per SM)
constexpr int ROWS = 2;             // map rows per CTA in passes A and C (1 or 2)
constexpr int ROW_T = 512;          // threads per CTA in passes A and C
static_assert((ROWS == 1 || ROWS == 2) && 1024 % ROW_T == 0, "row pass shape");
constexpr int LD_U = 4;             // vector loads in flight per thread
constexpr int FFT_NMAX = 10240;     // largest map side of this path
constexpr int MAX_STAGES = 20;

struct FftArgs {
    int64_t n;
    int32_t L;                       // transform length of this pass
    int32_t n_st;
    int32_t radix[MAX_STAGES];
    int32_t span[MAX_STAGES];        // L / (radix[0] ... radix[s])
    const float2* tw;                // tw[m] = exp(2 pi i m / n), m < n
    const int32_t* rev;              // rows: position of frequency k after the forward transform
    const float2* tws;               // per stage s: tws[tw_off[s] + j] = exp(2 pi i j / B_s), j < span
    int32_t tw_off[MAX_STAGES];
    uint32_t m_nb[MAX_STAGES];       // divmod multipliers (see divmod) of L / radix[s]
    uint32_t m_span[MAX_STAGES];     // and of span[s]
    uint32_t m_nblk[MAX_STAGES];     // and of L / (span[s] radix[s]), blocks per row
};

// complex sums as packed f32x2 operations (one instruction for both parts;
// each lane rounds as the scalar operation would)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// -i a (forward) or +i a (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// b + mul_mi(u) and b - mul_mi(u), one scalar add or subtract per part (the
// swapped, negated operand would cost moves before a packed add)
template <bool INV>
__device__ __forceinline__ float2 add_mi(float2 b, float2 u)
{
    return INV ? make_float2(b.x - u.y, b.y + u.x) : make_float2(b.x + u.y, b.y - u.x);
}
template <bool INV>
__device__ __forceinline__ float2 sub_mi(float2 b, float2 u)
{
    return INV ? make_float2(b.x + u.y, b.y - u.x) : make_float2(b.x - u.y, b.y + u.x);
}
// a s + c and a s, lane-wise with a scalar s
__device__ __forceinline__ float2 fma2s(float2 a, float s, float2 c)
{
    return __ffma2_rn(a, make_float2(s, s), c);
}
__device__ __forceinline__ float2 mul2s(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }

// ---- DFTs of length R in registers: y_u = sum_r a_r exp(-+2 pi i r u / R)
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[2])
    {
        const float2 t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <bool INV>
struct Dft<3, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[3])
    {
        constexpr float S3 = 0.866025403784438647f;     // sin(2 pi / 3)
        const float2 s = cadd(a[1], a[2]);
        const float2 t = fma2s(s, -0.5f, a[0]);
        const float2 u = mul2s(csub(a[1], a[2]), S3);
        a[0] = cadd(a[0], s);
        a[1] = add_mi<INV>(t, u);
        a[2] = sub_mi<INV>(t, u);
    }
};

template <bool INV>
struct Dft<4, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[4])
    {
        const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        const float2 t2 = cadd(a[1], a[3]), v = csub(a[1], a[3]);
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = add_mi<INV>(t1, v);
        a[3] = sub_mi<INV>(t1, v);
    }
};

template <bool INV>
struct Dft<5, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[5])
    {
        constexpr float C1 = 0.309016994374947424f;     // cos(2 pi / 5)
        constexpr float C2 = -0.809016994374947424f;    // cos(4 pi / 5)
        constexpr float S1 = 0.951056516295153572f;     // sin(2 pi / 5)
        constexpr float S2 = 0.587785252292473129f;     // sin(4 pi / 5)
        const float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
        const float2 t3 = csub(a[1], a[4]), t4 = csub(a[2], a[3]);
        const float2 b1 = fma2s(t2, C2, fma2s(t1, C1, a[0]));
        const float2 b2 = fma2s(t2, C1, fma2s(t1, C2, a[0]));
        const float2 u1 = fma2s(t4, S2, mul2s(t3, S1));
        const float2 u2 = fma2s(t4, -S1, mul2s(t3, S2));
        a[0] = cadd(a[0], cadd(t1, t2));
        a[1] = add_mi<INV>(b1, u1);
        a[4] = sub_mi<INV>(b1, u1);
        a[2] = add_mi<INV>(b2, u2);
        a[3] = sub_mi<INV>(b2, u2);
    }
};

template <bool INV>
struct Dft<8, INV> {
    static __device__ __forceinline__ void run(float2 (&a)[8])
    {
        constexpr float H = 0.707106781186547524f;      // sqrt(2) / 2
        float2 e[4] = {a[0], a[2], a[4], a[6]};
        float2 o[4] = {a[1], a[3], a[5], a[7]};
        Dft<4, INV>::run(e);
        Dft<4, INV>::run(o);
        // w^u, w = exp(-+2 pi i / 8)
        const float2 o1 = mul2s(INV ? make_float2(o[1].x - o[1].y, o[1].x + o[1].y)
                                    : make_float2(o[1].x + o[1].y, o[1].y - o[1].x), H);
        const float2 o3 = mul2s(INV ? make_float2(o[3].x + o[3].y, o[3].y - o[3].x)
                                    : make_float2(o[3].x - o[3].y, o[3].x + o[3].y), -H);
        a[0] = cadd(e[0], o[0]);
        a[4] = csub(e[0], o[0]);
        a[1] = cadd(e[1], o1);
        a[5] = csub(e[1], o1);
        a[2] = add_mi<INV>(e[2], o[2]);
        a[6] = sub_mi<INV>(e[2], o[2]);
        a[3] = cadd(e[3], o3);
        a[7] = csub(e[3], o3);
    }
};

// q = a / b, r = a % b for 0 <= a < 2^18 and 1 <= b < 2^18 by a multiply:
// m = ceil(2^32 / b) (0 for b = 1) overestimates 1/b by less than 2^-32, so
// the high word of a m is off a / b by less than a 2^-32 < 1/b and floors to
// the exact quotient
__device__ __forceinline__ void divmod(int a, int b, uint32_t m, int& q, int& r)
{
    q = m ? (int)__umulhi((uint32_t)a, m) : a;
    r = a - q * b;
}

// Shared-memory position of element e of a transform row.  Rows whose length
// is a multiple of 256 (power-of-two map sides) are padded by 2 elements
// every 32 and 2 more every 256: their late stages (spans 4 and 1) and the
// digit-reversed gathers of the row passes would otherwise put up to 16
// lanes of a half-warp on one bank (modelled: 32 wavefronts per warp for the
// gathers at length 2048, 4 with the padding); even elements stay 16-byte
// aligned.  Other lengths are not padded.
template <bool PAD>
__device__ __forceinline__ int pix(int e)
{
    return PAD ? e + 2 * (e >> 5) + 2 * (e >> 8) : e;
}
__host__ __device__ constexpr int64_t padded_len(int64_t L, bool pad)
{
    return pad ? L + 2 * (L >> 5) + 2 * (L >> 8) : L;
}

// Vector e of ROWS rows of length L laid end to end: complex values 2e, 2e + 1
// of the concatenation (L even, so both lie in one row and one padding segment)
template <bool PAD>
__device__ __forceinline__ float4* row_vec(float2* zs, int e, int L, int Lp)
{
    const int c = 2 * e;
    if (!PAD) return reinterpret_cast<float4*>(zs + c);
    const int q = c / L;
    return reinterpret_cast<float4*>(zs + q * Lp + pix<PAD>(c - q * L));
}

// One stage of radix R, span S (= block / R), over RN sequences of
// length L (row stride ld): butterfly (block b, offset j < S) takes the R
// values at b B + j + r S.  Forward (decimation in frequency): transform,
// then output u times w_B^(-j u).  Inverse (decimation in time): input r
// times w_B^(j r), then transform.  w_B^m = tw[m n / B].
// Butterflies go to threads offset-fastest (consecutive threads take
// consecutive j of one block: unit-stride shared-memory accesses) while the
// span is at least a warp, or the block length B is even; for shorter spans
// with B odd (the radix-5 and -3 stages of 5-smooth sizes) block-fastest:
// consecutive threads take the same j of consecutive blocks, 2B words apart,
// distinct banks for every half-warp, and one broadcast twiddle, which avoids
// the bank conflicts of a warp straddling several short blocks.  (With B even
// -- power-of-two sizes -- block-fastest would put a half-warp on one bank.)
template <int R, bool INV, bool PAD, int NT, int RN>
__device__ __forceinline__ void stage(float2* z, int L, int ld, int S, const float2* tw,
                                      uint32_t m_nb, uint32_t m_S, uint32_t m_nblk)
{
    const int B = S * R;
    const int nb = L / R;                 // butterflies per row
    const bool blk_fast = S < 32 && (B & 1);
    const int nblk = L / B;               // blocks per row
    for (int g = threadIdx.x; g < RN * nb; g += NT) {
        int row, gg, blk, j;
        if (RN == 1) {
            row = 0;
            gg = g;
        } else {
            divmod(g, nb, m_nb, row, gg);
        }
        if (blk_fast) divmod(gg, nblk, m_nblk, j, blk);
        else divmod(gg, S, m_S, blk, j);
        float2* zr = z + row * ld;
        const int e0 = blk * B + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = zr[pix<PAD>(e0 + r * S)];
        // twiddles w_B^(j r): w = w_B^j from the stage's own table (consecutive
        // j, consecutive entries: one coalesced read per warp), its powers by
        // products (r - 1 roundings; a table read per power costs L1
        // bandwidth the shared-memory traffic needs)
        float2 t[R];
        if (j) {
            t[1] = __ldg(tw + j);
            if (!INV) t[1].y = -t[1].y;
#pragma unroll
            for (int r = 2; r < R; ++r) t[r] = cmul(t[r / 2], t[r - r / 2]);
        }
        if (INV && j) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], t[r]);
        }
        Dft<R, INV>::run(v);
        if (!INV && j) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], t[r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) zr[pix<PAD>(e0 + r * S)] = v[r];
    }
    __syncthreads();
}

template <bool INV, bool PAD, int NT, int RN>
__device__ __forceinline__ void stage_r(int R, float2* z, int L, int ld, int S,
                                        const float2* tw, uint32_t m_nb, uint32_t m_S,
                                        uint32_t m_nblk)
{
    switch (R) {
    case 8: stage<8, INV, PAD, NT, RN>(z, L, ld, S, tw, m_nb, m_S, m_nblk); break;
    case 4: stage<4, INV, PAD, NT, RN>(z, L, ld, S, tw, m_nb, m_S, m_nblk); break;
    case 2: stage<2, INV, PAD, NT, RN>(z, L, ld, S, tw, m_nb, m_S, m_nblk); break;
    case 5: stage<5, INV, PAD, NT, RN>(z, L, ld, S, tw, m_nb, m_S, m_nblk); break;
    default: stage<3, INV, PAD, NT, RN>(z, L, ld, S, tw, m_nb, m_S, m_nblk); break;
    }
}

// The whole transform.  Forward: stages in plan order (spans L/R1, ...);
// inverse: the same stages in reverse order.
template <bool INV, bool PAD, int NT, int RN>
__device__ void fft_smem(float2* z, int L, int ld, const FftArgs& A)
{
    if (!INV) {
        for (int s = 0; s < A.n_st; ++s)
            stage_r<false, PAD, NT, RN>(A.radix[s], z, L, ld, A.span[s], A.tws + A.tw_off[s], A.m_nb[s],
                           A.m_span[s], A.m_nblk[s]);
    } else {
        for (int s = A.n_st - 1; s >= 0; --s)
            stage_r<true, PAD, NT, RN>(A.radix[s], z, L, ld, A.span[s], A.tws + A.tw_off[s], A.m_nb[s],
                          A.m_span[s], A.m_nblk[s]);
    }
}

// ---- pass A: ROWS rows, real to complex, written transposed ----------------
template <typename IN, bool PAD>
__global__ void __launch_bounds__(ROW_T, 2 * 512 / ROW_T)
rows_fwd_kernel(const IN* __restrict__ in, const __grid_constant__ FftArgs A,
                float2* __restrict__ T)
{
    extern __shared__ __align__(16) float2 zs[];
    const int64_t n = A.n;
    const int L = A.L;                    // n / 2
    const int Lp = (int)padded_len(L, PAD);   // row stride in shared memory
    const int64_t row0 = (int64_t)blockIdx.x * ROWS;
    // pack: z_k = x_2k + i x_2k+1 (count maps converted to float, exact below
    // 2^24); the ROWS rows are contiguous, so the CTA reads n ROWS / 4
    // 16-byte vectors, LD_U in flight per thread
    {
        using V = typename std::conditional<std::is_same<IN, float>::value, float4, int4>::type;
        const V* src = reinterpret_cast<const V*>(in + row0 * n);
        const int nv = (int)(ROWS * n / 4);
        auto dst = [&](int e) -> float4* { return row_vec<PAD>(zs, e, L, Lp); };
        for (int e0 = threadIdx.x; e0 < nv; e0 += ROW_T * LD_U) {
            V v[LD_U];
#pragma unroll
            for (int u = 0; u < LD_U; ++u)
                if (e0 + u * ROW_T < nv) v[u] = __ldg(src + e0 + u * ROW_T);
#pragma unroll
            for (int u = 0; u < LD_U; ++u)
                if (e0 + u * ROW_T < nv)
                    *dst(e0 + u * ROW_T) = make_float4((float)v[u].x, (float)v[u].y, (float)v[u].z,
                                                       (float)v[u].w);
        }
    }
    __syncthreads();
    fft_smem<false, PAD, ROW_T, ROWS>(zs, L, Lp, A);
    // separate the even and odd spectra: X_k = E_k + w^k O_k for k = 0..L
    // (Z_k sits at position rev[k])
    for (int k = threadIdx.x; k <= L; k += ROW_T) {
        const int ka = __ldg(A.rev + (k == L ? 0 : k)), kb = __ldg(A.rev + (k == 0 ? 0 : L - k));
        float2 w = __ldg(A.tw + k);       // exp(+2 pi i k / n); forward takes conj
        w.y = -w.y;
        float2 x[ROWS];
#pragma unroll
        for (int q = 0; q < ROWS; ++q) {
            const float2 a = zs[q * Lp + pix<PAD>(ka)], bc = zs[q * Lp + pix<PAD>(kb)];
            const float2 b = make_float2(bc.x, -bc.y);
            const float2 e = cscale(cadd(a, b), 0.5f);
            const float2 d = csub(a, b);
            const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);     // (a - b) / (2 i)
            x[q] = cadd(e, cmul(w, o));
        }
        if constexpr (ROWS == 2)
            *reinterpret_cast<float4*>(T + (int64_t)k * n + row0) =
                make_float4(x[0].x, x[0].y, x[1].x, x[1].y);
        else
            T[(int64_t)k * n + row0] = x[0];
    }
}

// ---- pass B: one column of the spectrum (a row of T) -------------------------
constexpr int COL_FWD = 1, COL_PROD = 2, COL_INV = 4;

template <bool PAD>
__global__ void __launch_bounds__(FFT_T, 2)
cols_kernel(const float2* src, const float2* __restrict__ K, float scale, int mode,
            const __grid_constant__ FftArgs A, float2* dst)
{
    extern __shared__ __align__(16) float2 zs[];
    const int L = A.L;                    // n
    const int64_t off = (int64_t)blockIdx.x * L;
    const float4* s4 = reinterpret_cast<const float4*>(src + off);
    // vector e holds complex values 2e, 2e + 1 (one padding segment)
    auto z4 = [&](int e) -> float4* { return reinterpret_cast<float4*>(zs + pix<PAD>(2 * e)); };
    for (int e0 = threadIdx.x; e0 < L / 2; e0 += FFT_T * LD_U) {
        float4 v[LD_U];
#pragma unroll
        for (int u = 0; u < LD_U; ++u)
            if (e0 + u * FFT_T < L / 2) v[u] = s4[e0 + u * FFT_T];
#pragma unroll
        for (int u = 0; u < LD_U; ++u)
            if (e0 + u * FFT_T < L / 2) *z4(e0 + u * FFT_T) = v[u];
    }
    __syncthreads();
    if (mode & COL_FWD) fft_smem<false, PAD, FFT_T, 1>(zs, L, (int)padded_len(L, PAD), A);
    if (mode & COL_PROD) {
        const float4* k4 = reinterpret_cast<const float4*>(K + off);
        for (int e0 = threadIdx.x; e0 < L / 2; e0 += FFT_T * LD_U) {
            float4 kv[LD_U];
#pragma unroll
            for (int u = 0; u < LD_U; ++u)
                if (e0 + u * FFT_T < L / 2) kv[u] = __ldg(k4 + e0 + u * FFT_T);
#pragma unroll
            for (int u = 0; u < LD_U; ++u) {
                const int e = e0 + u * FFT_T;
                if (e < L / 2) {
                    const float4 a = *z4(e), k = kv[u];
                    *z4(e) = make_float4((a.x * k.x - a.y * k.y) * scale, (a.x * k.y + a.y * k.x) * scale,
                                         (a.z * k.z - a.w * k.w) * scale, (a.z * k.w + a.w * k.z) * scale);
                }
            }
        }
        __syncthreads();
    }
    if (mode & COL_INV) fft_smem<true, PAD, FFT_T, 1>(zs, L, (int)padded_len(L, PAD), A);
    float4* d4 = reinterpret_cast<float4*>(dst + off);
    for (int e = threadIdx.x; e < L / 2; e += FFT_T) d4[e] = *z4(e);
}

// ---- pass C: ROWS rows, complex to real -------------------------------------
template <bool PAD>
__global__ void __launch_bounds__(ROW_T, 2 * 512 / ROW_T)
rows_inv_kernel(const float2* __restrict__ T, const __grid_constant__ FftArgs A,
                float* __restrict__ out)
{
    extern __shared__ __align__(16) float2 zs[];
    const int64_t n = A.n;
    const int L = A.L;                    // n / 2
    const int Lp = (int)padded_len(L, PAD);   // row stride in shared memory
    const int64_t row0 = (int64_t)blockIdx.x * ROWS;
    // Z'_k = (X_k + conj X_(L-k)) + i w^-k (X_k - conj X_(L-k)) for k < L, by
    // pairs (k, L - k) gathered from T, stored at the digit-reversed
    // positions the inverse transform takes (k = 0 pairs with the Nyquist bin)
    // GU pairs per thread in flight: their 2 GU loads (the ROWS values of a
    // bin are adjacent in T) are issued before any is used
    constexpr int GU = 2;
    for (int k0 = threadIdx.x; k0 <= L / 2; k0 += ROW_T * GU) {
        float2 xa0[GU][ROWS], xb0[GU][ROWS];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int k = k0 + u * ROW_T;
            if (k <= L / 2) {
                const float2* ta = T + (int64_t)k * n + row0;
                const float2* tb = T + (int64_t)(L - k) * n + row0;
                if constexpr (ROWS == 2) {
                    const float4 a = *reinterpret_cast<const float4*>(ta);
                    const float4 b = *reinterpret_cast<const float4*>(tb);
                    xa0[u][0] = make_float2(a.x, a.y);
                    xa0[u][ROWS - 1] = make_float2(a.z, a.w);
                    xb0[u][0] = make_float2(b.x, b.y);
                    xb0[u][ROWS - 1] = make_float2(b.z, b.w);
                } else {
                    xa0[u][0] = *ta;
                    xb0[u][0] = *tb;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int k = k0 + u * ROW_T;
            if (k > L / 2) break;
            const int k2 = L - k;
            const float2(&xa)[ROWS] = xa0[u];
            const float2(&xb)[ROWS] = xb0[u];
            const float2 wa = __ldg(A.tw + k), wb = __ldg(A.tw + k2);   // exp(+2 pi i k / n)
            const int ra = __ldg(A.rev + k);
            const bool pair = k > 0 && k2 != k;
            const int rb = pair ? __ldg(A.rev + k2) : 0;
#pragma unroll
            for (int q = 0; q < ROWS; ++q) {
                const float2 xbc = make_float2(xb[q].x, -xb[q].y), xac = make_float2(xa[q].x, -xa[q].y);
                const float2 ea = cadd(xa[q], xbc), oa = cmul(csub(xa[q], xbc), wa);
                zs[q * Lp + pix<PAD>(ra)] = make_float2(ea.x - oa.y, ea.y + oa.x);
                if (pair) {
                    const float2 eb = cadd(xb[q], xac), ob = cmul(csub(xb[q], xac), wb);
                    zs[q * Lp + pix<PAD>(rb)] = make_float2(eb.x - ob.y, eb.y + ob.x);
                }
            }
        }
    }
    __syncthreads();
    fft_smem<true, PAD, ROW_T, ROWS>(zs, L, Lp, A);
    // the ROWS output rows are contiguous: z_k = (x_2k, x_2k+1)
    float4* o4 = reinterpret_cast<float4*>(out + row0 * n);
    for (int e = threadIdx.x; e < (int)(ROWS * n / 4); e += ROW_T)
        o4[e] = *row_vec<PAD>(zs, e, L, Lp);
}

// Radices of a length-L transform, 8s first.  A power of two 2^e with
// e = 1 (mod 3), e >= 4, ends in 4, 4 instead of 8, 2: the same number of
// shared-memory round trips, and the butterflies divide more evenly over a
// CTA's threads (length 10000: 2500 radix-4 butterflies per stage against
// 1250 radix-8 and 5000 radix-2 ones for 512 threads).
bool radices(int64_t L, int32_t* r, int32_t* n_st)
{
    int k = 0;
    int64_t m = L;
    int e = 0;
    for (int64_t t = m; t % 2 == 0; t /= 2) ++e;
    const int n8 = e % 3 == 1 && e >= 4 ? e / 3 - 1 : e / 3;
    for (int i = 0; i < n8 && k < MAX_STAGES; ++i) { r[k++] = 8; m /= 8; }
    while (m % 4 == 0 && k < MAX_STAGES) { r[k++] = 4; m /= 4; }
    while (m % 2 == 0 && k < MAX_STAGES) { r[k++] = 2; m /= 2; }
    while (m % 5 == 0 && k < MAX_STAGES) { r[k++] = 5; m /= 5; }
    while (m % 3 == 0 && k < MAX_STAGES) { r[k++] = 3; m /= 3; }
    *n_st = k;
    return m == 1;
}

// float2 entries of the stage tables of a length-L transform: sum of the
// spans L / (R1 ... Rs)
int64_t stage_tables_size(int64_t L)
{
    int32_t r[MAX_STAGES], k = 0;
    radices(L, r, &k);
    int64_t S = L, tot = 0;
    for (int s = 0; s < k; ++s) {
        S /= r[s];
        tot += S;
    }
    return tot;
}

// float2 index in the plan's table of the length-L transform's stage tables:
// after the n roots and the row digit reversal (n/2 int32 = n/4 float2)
int64_t stage_tables_base(int64_t n, int64_t L)
{
    const int64_t rows = n + n / 4;
    return L == n / 2 ? rows : rows + stage_tables_size(n / 2);
}

FftArgs args_for(const FftPlan& p, int64_t L)
{
    FftArgs a;
    memset(&a, 0, sizeof a);
    a.n = p.n;
    a.L = (int32_t)L;
    radices(L, a.radix, &a.n_st);
    int64_t S = L;
    for (int k = 0; k < a.n_st; ++k) {
        S /= a.radix[k];
        a.span[k] = (int32_t)S;
    }
    a.tw = reinterpret_cast<const float2*>(p.tw);
    a.rev = reinterpret_cast<const int32_t*>(static_cast<const float2*>(p.tw) + p.n);
    // stage tables: the row transform's (length n/2), then the column one's
    a.tws = a.tw + stage_tables_base(p.n, L);
    int32_t off = 0;
    auto magic = [](int64_t d) -> uint32_t {
        return d == 1 ? 0u : (uint32_t)(((1ull << 32) + (uint64_t)d - 1) / (uint64_t)d);
    };
    for (int k = 0; k < a.n_st; ++k) {
        a.tw_off[k] = off;
        off += a.span[k];
        a.m_nb[k] = magic(L / a.radix[k]);
        a.m_span[k] = magic(a.span[k]);
        a.m_nblk[k] = magic(L / ((int64_t)a.span[k] * a.radix[k]));
    }
    return a;
}

// The padded shared-memory layout serves transform lengths that are multiples
// of 256: their digit-reversed gathers and long-stride butterflies otherwise
// meet in a few banks
bool pads(int64_t L) { return L % 256 == 0; }

int set_smem(const void* fn, size_t bytes)
{
    return cuda_fail(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
                     "FFT shared memory");
}

}  // namespace

bool fft_supported(int64_t n)
{
    if (n < 8 || n > FFT_NMAX || n % 4) return false;
    int32_t r[MAX_STAGES], k;
    return radices(n / 2, r, &k) && radices(n, r, &k);
}

size_t fft_plan_bytes(int64_t n)
{
    return (size_t)(2 * n + n / 2 + 2 * (stage_tables_size(n / 2) + stage_tables_size(n))) *
           sizeof(float);
}

int fft_plan_create(int64_t n, FftPlan* p)
{
    memset(p, 0, sizeof *p);
    if (!fft_supported(n)) return fail(RS_EINVAL, "no own FFT for n = %lld", (long long)n);
    p->n = n;
    // n roots of unity (float2), then the digit reversal of the row transform
    // (length L = n / 2): frequency k = u1 + R1 u2 + R1 R2 u3 + ... lands at
    // position u1 L/R1 + u2 L/(R1 R2) + ... after decimation in frequency
    const int64_t L = n / 2;
    const int64_t n_stage = stage_tables_size(L) + stage_tables_size(n);
    std::vector<float> h(2 * n + L + 2 * n_stage);
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t m = 0; m < n; ++m) {
        const double a = two_pi * (double)m / (double)n;
        h[2 * m] = (float)cos(a);
        h[2 * m + 1] = (float)sin(a);
    }
    int32_t rad[MAX_STAGES], nst = 0;
    radices(L, rad, &nst);
    int32_t* rev = reinterpret_cast<int32_t*>(h.data() + 2 * n);
    for (int64_t k = 0; k < L; ++k) {
        int64_t q = k, pos = 0, S = L;
        for (int s = 0; s < nst; ++s) {
            S /= rad[s];
            pos += (q % rad[s]) * S;
            q /= rad[s];
        }
        rev[k] = (int32_t)pos;
    }
    // per transform and stage s (block B = span x radix): exp(2 pi i j / B),
    // j < span, in FP64 then rounded
    for (const int64_t len : {L, n}) {
        float* t = h.data() + 2 * stage_tables_base(n, len);
        int32_t rr[MAX_STAGES], ns = 0;
        radices(len, rr, &ns);
        int64_t S = len;
        for (int s2 = 0; s2 < ns; ++s2) {
            const int64_t B = S;
            S /= rr[s2];
            for (int64_t j = 0; j < S; ++j) {
                const double a = two_pi * (double)j / (double)B;
                *t++ = (float)cos(a);
                *t++ = (float)sin(a);
            }
        }
    }
    const size_t bytes = h.size() * sizeof(float);
    if (cudaMalloc(&p->tw, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->tw = nullptr;
        return fail(RS_ENOMEM, "FFT twiddle table");
    }
    int rc = cuda_fail(cudaMemcpy(p->tw, h.data(), bytes, cudaMemcpyHostToDevice), "twiddle upload");
    // shared memory of the largest transform each instantiation can take (a
    // padded kernel only takes lengths that are multiples of 256)
    const size_t half_u = (size_t)ROWS * (FFT_NMAX / 2) * 8, full_u = (size_t)FFT_NMAX * 8;
    const int64_t half_p = FFT_NMAX / 2 / 256 * 256, full_p = FFT_NMAX / 256 * 256;
    const size_t half_pb = (size_t)ROWS * padded_len(half_p, true) * 8;
    const size_t full_pb = (size_t)padded_len(full_p, true) * 8;
    if (!rc) rc = set_smem((const void*)rows_fwd_kernel<float, false>, half_u);
    if (!rc) rc = set_smem((const void*)rows_fwd_kernel<int32_t, false>, half_u);
    if (!rc) rc = set_smem((const void*)rows_fwd_kernel<float, true>, half_pb);
    if (!rc) rc = set_smem((const void*)rows_fwd_kernel<int32_t, true>, half_pb);
    if (!rc) rc = set_smem((const void*)rows_inv_kernel<false>, half_u);
    if (!rc) rc = set_smem((const void*)rows_inv_kernel<true>, half_pb);
    if (!rc) rc = set_smem((const void*)cols_kernel<false>, full_u);
    if (!rc) rc = set_smem((const void*)cols_kernel<true>, full_pb);
    if (rc) fft_plan_destroy(p);
    return rc;
}

void fft_plan_destroy(FftPlan* p)
{
    if (p->tw) cudaFree(p->tw);
    p->tw = nullptr;
}

int fft_rows_forward(const FftPlan& p, const void* in, bool counts, float2* T, cudaStream_t s)
{
    const FftArgs A = args_for(p, p.n / 2);
    const bool pad = pads(p.n / 2);
    const size_t smem = (size_t)ROWS * padded_len(p.n / 2, pad) * sizeof(float2);
    const unsigned grid = (unsigned)(p.n / ROWS);
    const int32_t* ic = static_cast<const int32_t*>(in);
    const float* iv = static_cast<const float*>(in);
    if (counts && pad) rows_fwd_kernel<int32_t, true><<<grid, ROW_T, smem, s>>>(ic, A, T);
    else if (counts) rows_fwd_kernel<int32_t, false><<<grid, ROW_T, smem, s>>>(ic, A, T);
    else if (pad) rows_fwd_kernel<float, true><<<grid, ROW_T, smem, s>>>(iv, A, T);
    else rows_fwd_kernel<float, false><<<grid, ROW_T, smem, s>>>(iv, A, T);
    return cuda_fail(cudaGetLastError(), "FFT row pass launch");
}

int fft_columns(const FftPlan& p, const float2* src, const float2* K, float scale, bool fwd,
                bool prod, bool inv, float2* dst, cudaStream_t s)
{
    const FftArgs A = args_for(p, p.n);
    const int mode = (fwd ? COL_FWD : 0) | (prod ? COL_PROD : 0) | (inv ? COL_INV : 0);
    const bool pad = pads(p.n);
    const size_t smem = (size_t)padded_len(p.n, pad) * sizeof(float2);
    const unsigned grid = (unsigned)(p.n / 2 + 1);
    if (pad) cols_kernel<true><<<grid, FFT_T, smem, s>>>(src, K, scale, mode, A, dst);
    else cols_kernel<false><<<grid, FFT_T, smem, s>>>(src, K, scale, mode, A, dst);
    return cuda_fail(cudaGetLastError(), "FFT column pass launch");
}

int fft_rows_inverse(const FftPlan& p, const float2* T, float* out, cudaStream_t s)
{
    const FftArgs A = args_for(p, p.n / 2);
    const bool pad = pads(p.n / 2);
    const size_t smem = (size_t)ROWS * padded_len(p.n / 2, pad) * sizeof(float2);
    const unsigned grid = (unsigned)(p.n / ROWS);
    if (pad) rows_inv_kernel<true><<<grid, ROW_T, smem, s>>>(T, A, out);
    else rows_inv_kernel<false><<<grid, ROW_T, smem, s>>>(T, A, out);
    return cuda_fail(cudaGetLastError(), "FFT inverse row pass launch");
}

}  // namespace rs
