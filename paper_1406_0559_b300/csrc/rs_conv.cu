// rs_conv.cu -- finite-source convolution of magnification maps (Sec. 2.4,
// Eq. 6), pixelFlux extraction and value histograms of convolved maps
// (Sec. 3.2.2).
//
// Per profile: the brightness profile is binned into map-sized pixels
// (S x S samples per pixel, exact integer inside test), normalised to unit
// sum in FP64, scattered around pixel (0, 0) of an npix x npix image and
// transformed once (cuFFT R2C) into the kernel spectrum F(K).
// Per map: counts -> float (exact below 2^24), R2C, the spectral product
// F(M) F(K) scaled by scale / npix^2, C2R into the caller's map.  For the
// survey's map sizes (npix a multiple of 4 with npix and npix/2 products of
// 2, 3 and 5, up to 10240: 4096 and 10000 among them) the transforms are this
// library's own (rs_fft.cu: three passes, the conversion fused into the
// first and the spectral product between the column transforms); other sizes
// use cuFFT, the library the paper uses for Eq. 6.  HBM traffic per map: the conversion
// (8 B/px), the spectral product (24 B per complex bin, n (n/2 + 1) bins) and
// the transforms.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math.h>

#include <cstring>
#include <mutex>
#include <type_traits>
#include <new>

#include "rs_internal.cuh"
#include "../../include/rs_conv.h"

struct rs_conv {
    int64_t n = 0;
    int64_t nc = 0;              // complex bins of one spectrum, n (n/2 + 1)
    int device = -1;
    bool own = false;            // this library's FFTs (rs_fft.cu); else cuFFT
    rs::FftPlan fft = {};
    cufftHandle fwd = 0, inv = 0;
    bool fwd_ok = false, inv_ok = false;
    cufftComplex* khat = nullptr;   // F(K); also scratch for the small kernel
    cufftComplex* spec = nullptr;   // working spectrum; also the kernel image
    void* work = nullptr;
    size_t work_bytes = 0;
    bool has_kernel = false;
    cufftComplex* spec2 = nullptr;  // product buffer for loaded spectra (on first use)
    cufftComplex* slot[RS_CONV_SLOTS] = {};   // kernel spectra 1.. (slot 0 is khat)
    bool slot_set[RS_CONV_SLOTS] = {};
    bool loaded = false;            // spec holds F(M) of a loaded map
    double load_scale = 1.0;        // scale of the loaded map
    int h_direct = -1;              // kernel half size when the direct path applies
    float kf[169];                  // the kernel rotated by 180 degrees, (2h+1)^2
};

namespace rs {
namespace {

// ---- profile binning -------------------------------------------------------

struct ProfParams {
    int32_t type, S;
    int64_t h;
    long long t_in, t_out;   // a sample is inside iff t_in <= u1^2 + u2^2 < t_out
    float hs;                // sample spacing unit w / (2 S)
    float c1, c2;            // 1 / (2 sigma^2) along y1, y2
    float inv_rs, neg_index, r_in;
};

__device__ __forceinline__ float brightness(const ProfParams& P, float y1, float y2)
{
    switch (P.type) {
    case RS_PROFILE_UNIFORM:
        return 1.f;
    case RS_PROFILE_GAUSSIAN:
        return expf(-(y1 * y1 * P.c1 + y2 * y2 * P.c2));
    case RS_PROFILE_POWER_LAW: {
        const float r = sqrtf(y1 * y1 + y2 * y2);
        return powf(r * P.inv_rs, P.neg_index);
    }
    default: {
        const float r = sqrtf(y1 * y1 + y2 * y2);
        const float xi = powf(r * P.inv_rs, 0.75f) * powf(1.f - sqrtf(P.r_in / r), -0.25f);
        return 1.f / expm1f(xi);
    }
    }
}

// One thread per kernel pixel: the sum of I over its inside samples (FP32
// per sample row, FP64 across rows).
__global__ void profile_raw_kernel(const __grid_constant__ ProfParams P, float* __restrict__ k)
{
    const int64_t d = 2 * P.h + 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= d * d) return;
    const long long a = idx / d - P.h;
    const long long b = idx % d - P.h;
    const long long S = P.S;
    long long u2 = 2 * (a * S) + 1 - S;
    double acc = 0.0;
    for (int t = 0; t < P.S; ++t, u2 += 2) {
        const long long v2 = u2 * u2;
        long long u1 = 2 * (b * S) + 1 - S;
        float row = 0.f;
        for (int s = 0; s < P.S; ++s, u1 += 2) {
            const long long q = u1 * u1 + v2;
            if (q >= P.t_in && q < P.t_out)
                row += brightness(P, (float)u1 * P.hs, (float)u2 * P.hs);
        }
        acc += (double)row;
    }
    k[idx] = (float)acc;
}

// One CTA: divide by the total (FP64, fixed order); an empty kernel becomes
// the unit impulse at the centre.
__global__ void __launch_bounds__(1024) normalise_kernel(float* __restrict__ k, int64_t m,
                                                         int64_t centre)
{
    __shared__ double part[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s += (double)k[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    const double total = part[0];
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x)
        k[i] = total > 0.0 ? (float)((double)k[i] / total) : (i == centre ? 1.f : 0.f);
}

// The n x n kernel image: K[a][b] at row a mod n, column b mod n, 0 elsewhere.
__global__ void scatter_kernel(const float* __restrict__ k, int64_t h, int64_t n,
                               float* __restrict__ img)
{
    const int64_t d = 2 * h + 1;
    for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
        const int64_t a = q <= h ? q : (q >= n - h ? q - n : INT64_MAX);
        float* row = img + q * n;
        for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
            const int64_t b = p <= h ? p : (p >= n - h ? p - n : INT64_MAX);
            row[p] = (a != INT64_MAX && b != INT64_MAX) ? k[(a + h) * d + (b + h)] : 0.f;
        }
    }
}

// ---- the spectral product of Eq. 6 -----------------------------------------

__device__ __forceinline__ float4 cmul2(float4 a, float4 k, float s)
{
    return make_float4((a.x * k.x - a.y * k.y) * s, (a.x * k.y + a.y * k.x) * s,
                       (a.z * k.z - a.w * k.w) * s, (a.z * k.w + a.w * k.z) * s);
}

// out[i] = spec[i] * khat[i] * s over nc complex bins (out may be spec), two
// bins per 16-byte access, four accesses in flight per thread.
__global__ void spectral_product_kernel(const float4* spec, const float4* __restrict__ khat,
                                        int64_t nc, float s, float4* out)
{
    const int64_t n2 = nc / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    constexpr int U = 4;
    int64_t i = t0;
    for (; i + (U - 1) * stride < n2; i += U * stride) {
        float4 a[U], k[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u] = __ldcs(spec + i + u * stride);
            k[u] = __ldcs(khat + i + u * stride);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) __stcs(out + i + u * stride, cmul2(a[u], k[u], s));
    }
    for (; i < n2; i += stride) __stcs(out + i, cmul2(__ldcs(spec + i), __ldcs(khat + i), s));
    if ((nc & 1) && t0 == 0) {
        const float2* sp = reinterpret_cast<const float2*>(spec);
        const float2* kp = reinterpret_cast<const float2*>(khat);
        const float2 a = sp[nc - 1], k = kp[nc - 1];
        reinterpret_cast<float2*>(out)[nc - 1] =
            make_float2((a.x * k.x - a.y * k.y) * s, (a.x * k.y + a.y * k.x) * s);
    }
}

// ---- pixelFlux and value histograms -------------------------------------------

__global__ void pixel_flux_kernel(const float* __restrict__ map, int64_t n,
                                  const short2* __restrict__ xy, unsigned long long seed,
                                  int64_t k, uint2* __restrict__ rec)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < k;
         t += (int64_t)gridDim.x * blockDim.x) {
        int x, y;
        if (xy) {
            const short2 v = xy[t];
            x = v.x;
            y = v.y;
        } else {
            const unsigned long long hx = splitmix64(seed, 2ull * (unsigned long long)t) >> 32;
            const unsigned long long hy = splitmix64(seed, 2ull * (unsigned long long)t + 1ull) >> 32;
            x = (int)((hx * (unsigned long long)n) >> 32);
            y = (int)((hy * (unsigned long long)n) >> 32);
        }
        const bool in = x >= 0 && y >= 0 && x < n && y < n;
        const float v = in ? map[(int64_t)y * n + x] : __int_as_float(0x7fc00000);
        rec[t] = make_uint2((unsigned)(unsigned short)x | ((unsigned)(unsigned short)y << 16),
                            __float_as_uint(v));
    }
}

constexpr int MAX_EDGES = RS_VALUE_HIST_MAX_EDGES;

struct EdgeArgs {
    int32_t n;
    int32_t shift;       // bucket = ordkey >> shift
    uint32_t key_lo;     // bucket of the first edge
    int32_t nkeys;       // buckets from the first edge's to the last edge's
    float e[MAX_EDGES];
};

// bin(v) = number of edges <= v.  Floats map to unsigned integers in value
// order (ordkey; -0 taken as +0).  Buckets of 2^shift consecutive keys are
// tabled from the first edge's bucket to the last edge's (at most
// HIST_TABLE buckets; shift is the smallest that fits, so for log-spaced
// edges a bucket is a small fraction of the edge spacing); entry i holds
// the number of edges below bucket key_lo + i - 1, the number inside it,
// and the first of those, between two sentinel entries that hold no edge: a
// value below the first bucket clamps onto the first (every edge above it:
// bin 0), one above the last bucket onto the last (bin n); otherwise its
// bin is the entry's count below plus one compare with the entry's edge
// when the bucket holds one edge, and a short search among the bucket's
// edges when it holds more (rare: only edges closer than a bucket share
// one).  Exact for any ascending edges.  NaN goes to bin 0.  The table is
// built once per call by table_kernel and copied into shared memory by
// every CTA, with the edges.
// The CTA's counts live in R interleaved copies of the histogram in shared
// memory (bin b of copy c at b * R + c, copy c taken by the lanes with
// lane % R == c): a smooth map puts whole warps into one or two bins, and
// one copy per lane (R = 32) keeps those atomics free of same-address
// conflicts (R = 8 or 16: at most 4- or 2-way).  The copies are summed and
// added to the global histogram at the end.
constexpr int HIST_TABLE = 8192;               // buckets (8 bytes each)
constexpr int HIST_THREADS = 1024;
constexpr size_t HIST_SMEM_MAX = 227 * 1024;

__host__ __device__ __forceinline__ unsigned ordkey_bits(unsigned b)
{
    // increasing in the value: negatives inverted, positives above them
    const unsigned neg = (unsigned)((int)b >> 31);
    return b ^ (neg | 0x80000000u);
}
__device__ __forceinline__ unsigned ordkey(float v)
{
    return ordkey_bits(__float_as_uint(v + 0.0f));          // -0 -> +0
}

// number of edges e with ordkey(e) < key (64-bit: key may be 2^32)
__device__ __forceinline__ int edges_below(const EdgeArgs& E, unsigned long long key)
{
    int lo = 0, hi = E.n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((unsigned long long)ordkey(E.e[mid]) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// T[i] = {below | inside << 16, bits of the bucket's first edge} for bucket
// key_lo + i - 1, 1 <= i <= nkeys, and two sentinels with no edge inside:
// T[0] (below every edge: bin 0) and T[nkeys + 1] (above every edge: bin n)
__global__ void table_kernel(const __grid_constant__ EdgeArgs E, uint2* __restrict__ T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > E.nkeys + 1) return;
    if (i == 0 || i == E.nkeys + 1) {
        T[i] = make_uint2(i == 0 ? 0u : (unsigned)E.n, 0u);
        return;
    }
    const unsigned long long k0 = (unsigned long long)(E.key_lo + (unsigned)(i - 1)) << E.shift;
    const int below = edges_below(E, k0);
    const int inside = edges_below(E, k0 + (1ull << E.shift)) - below;
    T[i] = make_uint2((unsigned)below | ((unsigned)inside << 16),
                      inside > 0 ? __float_as_uint(E.e[below]) : 0u);
}

template <int R>
__global__ void __launch_bounds__(HIST_THREADS, 1) value_hist_kernel(
    const float* __restrict__ v, int64_t n, const __grid_constant__ EdgeArgs E,
    const uint2* __restrict__ Tg, unsigned long long* __restrict__ hist)
{
    // dynamic shared memory: T[nkeys + 2] (uint2), edges[n], R copies of histogram[n + 1]
    extern __shared__ __align__(16) unsigned char smem[];
    const int ne = E.n, nkeys = E.nkeys, shift = E.shift;
    const int base = (int)E.key_lo - 1;          // bucket key_lo is table entry 1
    uint2* T = reinterpret_cast<uint2*>(smem);
    float* se = reinterpret_cast<float*>(smem + (size_t)(nkeys + 2) * 8);
    unsigned* sh = reinterpret_cast<unsigned*>(smem + (size_t)(nkeys + 2) * 8 + (ne * 4 + 15) / 16 * 16);
    for (int k = threadIdx.x; k < nkeys + 2; k += blockDim.x) T[k] = Tg[k];
    for (int k = threadIdx.x; k < ne; k += blockDim.x) se[k] = E.e[k];
    for (int k = threadIdx.x; k < (ne + 1) * R; k += blockDim.x) sh[k] = 0u;
    __syncthreads();
    unsigned* mine = sh + (threadIdx.x & (R - 1));
    // the bin from the table and one compare, without branches; returns
    // whether the bucket holds several edges (then `search` decides)
    // (the key shifted by at least 1 fits an int; values outside the table
    // clamp onto a sentinel, which holds no edge)
    auto entry = [&](float x) -> int {
        return min(max((int)(ordkey(x) >> shift) - base, 0), nkeys + 1);
    };
    auto fast = [&](float x, int& b) -> bool {
        const uint2 t = T[entry(x)];
        const int c = (int)(t.x >> 16);
        b = (int)(t.x & 0xffffu) + ((c != 0 && __uint_as_float(t.y) <= x) ? 1 : 0);
        const bool num = x == x;
        b = num ? b : 0;
        return c > 1 && num;
    };
    auto search = [&](float x) -> int {     // upper bound among the bucket's edges
        const uint2 t = T[entry(x)];
        int lo = (int)(t.x & 0xffffu), hi = lo + (int)(t.x >> 16);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (se[mid] <= x) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    // V values: every bin first (independent, so their table loads overlap),
    // then the rare searches, then the atomics
    auto add_v = [&](const float* x, auto vn) {
        constexpr int V = decltype(vn)::value;
        int b[V];
        bool slow = false;
#pragma unroll
        for (int k = 0; k < V; ++k) slow |= fast(x[k], b[k]);
        if (slow) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                int bb;
                if (fast(x[k], bb)) b[k] = search(x[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k) atomicAdd(mine + b[k] * R, 1u);
    };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n4 = (reinterpret_cast<uintptr_t>(v) & 15) == 0 ? n / 4 : 0;
    const float4* v4 = reinterpret_cast<const float4*>(v);
    // U float4 loads in flight per thread before any is binned
    constexpr int U = 4;
    int64_t i = t0;
    for (; i + (U - 1) * stride < n4; i += U * stride) {
        float x[4 * U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float4 w = __ldcs(v4 + i + u * stride);
            x[4 * u] = w.x;
            x[4 * u + 1] = w.y;
            x[4 * u + 2] = w.z;
            x[4 * u + 3] = w.w;
        }
        add_v(x, std::integral_constant<int, 2 * U>{});
        add_v(x + 2 * U, std::integral_constant<int, 2 * U>{});
    }
    for (; i < n4; i += stride) {
        const float4 w = __ldcs(v4 + i);
        const float x[4] = {w.x, w.y, w.z, w.w};
        add_v(x, std::integral_constant<int, 4>{});
    }
    for (int64_t j = 4 * n4 + t0; j < n; j += stride) {
        const float x[1] = {v[j]};
        add_v(x, std::integral_constant<int, 1>{});
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= ne; k += blockDim.x) {
        unsigned long long c = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) c += sh[k * R + ((r + k) & (R - 1))];   // staggered banks
        if (c) atomicAdd(hist + k, c);
    }
}

size_t hist_smem_bytes(int ne, int nkeys, int R)
{
    return (size_t)(nkeys + 2) * 8 + ((size_t)ne * 4 + 15) / 16 * 16 + (size_t)(ne + 1) * R * 4;
}

// the most histogram copies that fit (8 always do: RS_VALUE_HIST_MAX_EDGES)
int hist_copies(int ne, int nkeys)
{
    return hist_smem_bytes(ne, nkeys, 32) <= HIST_SMEM_MAX ? 32
           : hist_smem_bytes(ne, nkeys, 16) <= HIST_SMEM_MAX ? 16 : 8;
}
static_assert((size_t)(HIST_TABLE + 2) * 8 + (MAX_EDGES * 4 + 15) / 16 * 16 +
                      (size_t)(MAX_EDGES + 1) * 8 * 4 <= HIST_SMEM_MAX,
              "eight histogram copies fit for every edge count");

// Bucket tables of the value histogram: a few library-owned slots per
// device, reused in stream order.  A call takes the next slot, makes its
// stream wait for the slot's previous user, builds its table there and
// records the slot's event after the histogram -- no allocation per call,
// and calls on different streams never overwrite a table in use.
constexpr int HIST_SLOTS = 8;
constexpr int MAX_DEVICES = 64;

struct HistSlot {
    uint2* T = nullptr;
    cudaEvent_t ev = nullptr;
};

struct HistDevice {
    HistSlot slot[HIST_SLOTS];
    int next = 0;
    bool ready = false;
};

std::mutex g_hist_mu;
HistDevice g_hist[MAX_DEVICES];

// Caller holds g_hist_mu from here until the slot's event is recorded.
int hist_slot(cudaStream_t s, HistSlot** out)
{
    int dev = 0;
    int rc = cuda_fail(cudaGetDevice(&dev), "current device");
    if (rc) return rc;
    if (dev < 0 || dev >= MAX_DEVICES) return fail(RS_ERANGE, "device %d beyond %d", dev, MAX_DEVICES);
    HistDevice& d = g_hist[dev];
    if (!d.ready) {
        for (auto& sl : d.slot) {
            if (cudaMalloc(reinterpret_cast<void**>(&sl.T), (HIST_TABLE + 2) * sizeof(uint2)) !=
                    cudaSuccess ||
                cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return fail(RS_ENOMEM, "histogram table slots could not be allocated");
            }
        }
        cudaFuncSetAttribute(value_hist_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HIST_SMEM_MAX);
        cudaFuncSetAttribute(value_hist_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HIST_SMEM_MAX);
        cudaFuncSetAttribute(value_hist_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)HIST_SMEM_MAX);
        d.ready = true;
    }
    HistSlot* sl = &d.slot[d.next];
    d.next = (d.next + 1) % HIST_SLOTS;
    if ((rc = cuda_fail(cudaStreamWaitEvent(s, sl->ev, 0), "histogram slot wait"))) return rc;
    *out = sl;
    return RS_OK;
}

// ---- direct convolution for small kernels ------------------------------------
// C[q][p] = sum_{a,b} K[a][b] M[(q-a) mod n][(p-b) mod n] summed directly:
// (2h+1)^2 FMAs per pixel; faster than the FFT path while h <= DIRECT_HMAX
// (10000^2 map: 0.82 ms at h = 4 against 1.70 ms).  A CTA computes a
// 128 x 16 tile of outputs from a shared-memory copy of its input tile with
// an h-pixel halo (rows and columns wrapped cyclically); each thread
// computes 8 neighbouring outputs of a row from 16-byte loads of the input
// rows.  The kernel, rotated by 180 degrees, travels in the kernel
// parameters; each kernel row's weights are read into registers once per
// tile row.  FP32 sums of at most 169 terms.
constexpr int DIRECT_HMAX = 6;    // measured crossover with the FFT path at 10000^2: h = 7-8
constexpr int DT_W = 128, DT_H = 16, DT_OUT = 8;

struct DirectArgs {
    float kf[(2 * DIRECT_HMAX + 1) * (2 * DIRECT_HMAX + 1)];
};

template <int H, typename T>
__global__ void __launch_bounds__(256) conv_direct_kernel(const T* __restrict__ in, float scale,
                                                          int64_t n,
                                                          const __grid_constant__ DirectArgs A,
                                                          float* __restrict__ out)
{
    constexpr int D = 2 * H + 1;
    constexpr int TW = DT_W + 2 * H;
    constexpr int TWP = (TW + 3) / 4 * 4;
    constexpr int TH = DT_H + 2 * H;
    constexpr int SEG = DT_OUT + 2 * H;
    constexpr int SEG4 = (SEG + 3) / 4;
    __shared__ __align__(16) float tile[TH][TWP];
    const int64_t tiles1 = (n + DT_W - 1) / DT_W;
    const int64_t ntiles = tiles1 * ((n + DT_H - 1) / DT_H);
    const int tx = threadIdx.x % (DT_W / DT_OUT);
    const int ty = threadIdx.x / (DT_W / DT_OUT);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t q0 = (t / tiles1) * DT_H, p0 = (t % tiles1) * DT_W;
        __syncthreads();   // the previous tile has been consumed
        // tile rows by warps, columns by lanes: no division per element
        for (int i = threadIdx.x >> 5; i < TH; i += blockDim.x >> 5) {
            int64_t q = q0 - H + i;
            q = q < 0 ? q + n : (q >= n ? q - n : q);      // n > DT_H + 2H: one wrap at most
            const T* src = in + q * n;
            for (int j = threadIdx.x & 31; j < TW; j += 32) {
                int64_t p = p0 - H + j;
                p = p < 0 ? p + n : (p >= n ? p - n : p);
                tile[i][j] = (float)src[p] * scale;
            }
        }
        __syncthreads();
        float acc[DT_OUT];
#pragma unroll
        for (int j = 0; j < DT_OUT; ++j) acc[j] = 0.f;
        // rows of the kernel in a rolled loop (the fully unrolled body would
        // not fit the instruction cache); a row's weights go to registers
#pragma unroll 1
        for (int a = 0; a < D; ++a) {
            float wr[D];
#pragma unroll
            for (int b = 0; b < D; ++b) wr[b] = A.kf[a * D + b];
            float seg[4 * SEG4];
            const float4* row = reinterpret_cast<const float4*>(&tile[ty + a][tx * DT_OUT]);
#pragma unroll
            for (int k = 0; k < SEG4; ++k) {
                const float4 v = row[k];
                seg[4 * k] = v.x;
                seg[4 * k + 1] = v.y;
                seg[4 * k + 2] = v.z;
                seg[4 * k + 3] = v.w;
            }
#pragma unroll
            for (int b = 0; b < D; ++b) {
#pragma unroll
                for (int j = 0; j < DT_OUT; ++j) acc[j] = fmaf(wr[b], seg[j + b], acc[j]);
            }
        }
        const int64_t q = q0 + ty;
        if (q < n) {
#pragma unroll
            for (int j = 0; j < DT_OUT; ++j) {
                const int64_t p = p0 + tx * DT_OUT + j;
                if (p < n) out[q * n + p] = acc[j];
            }
        }
    }
}

template <typename T>
int launch_direct(int h, const T* in, float scale, int64_t n, const DirectArgs& A, float* out,
                  cudaStream_t s)
{
    const int64_t ntiles = ((n + DT_W - 1) / DT_W) * ((n + DT_H - 1) / DT_H);
    const int64_t cap = (int64_t)num_sms() * 8;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    switch (h) {
#define RS_DIRECT_CASE(H) \
    case H: conv_direct_kernel<H, T><<<grid, 256, 0, s>>>(in, scale, n, A, out); break;
        RS_DIRECT_CASE(0) RS_DIRECT_CASE(1) RS_DIRECT_CASE(2) RS_DIRECT_CASE(3)
        RS_DIRECT_CASE(4) RS_DIRECT_CASE(5) RS_DIRECT_CASE(6)
#undef RS_DIRECT_CASE
    default: return fail(RS_EINVAL, "no direct kernel for h = %d", h);
    }
    return cuda_fail(cudaGetLastError(), "direct convolution launch");
}

// ---- host helpers ----------------------------------------------------------------

int cufft_fail(cufftResult r, const char* what)
{
    if (r == CUFFT_SUCCESS) return RS_OK;
    if (r == CUFFT_ALLOC_FAILED) return fail(RS_ENOMEM, "cuFFT %s: allocation failed", what);
    return fail(RS_ECUDA, "cuFFT %s failed (cufftResult %d)", what, (int)r);
}

int check_profile(const rs_profile* p, double w)
{
    if (!p) return fail(RS_EINVAL, "profile is NULL");
    if (!(w > 0.0) || !isfinite(w)) return fail(RS_EINVAL, "pixel side must be > 0");
    if (p->type < RS_PROFILE_UNIFORM || p->type > RS_PROFILE_THIN_DISC)
        return fail(RS_EINVAL, "unknown profile type %d", p->type);
    if (p->supersample < 1 || p->supersample > RS_PROFILE_MAX_SUPERSAMPLE)
        return fail(RS_EINVAL, "supersample %d outside 1..%d", p->supersample,
                    RS_PROFILE_MAX_SUPERSAMPLE);
    if (!(p->r_out > 0.0) || !isfinite(p->r_out) || !(p->r_in >= 0.0) || !(p->r_in < p->r_out))
        return fail(RS_EINVAL, "need 0 <= r_in < r_out");
    if (p->type == RS_PROFILE_GAUSSIAN && !(p->sigma1 > 0.0 && p->sigma2 > 0.0))
        return fail(RS_EINVAL, "Gaussian profile needs sigma1, sigma2 > 0");
    if ((p->type == RS_PROFILE_POWER_LAW || p->type == RS_PROFILE_THIN_DISC) &&
        !(p->r_in > 0.0 && p->r_scale > 0.0))
        return fail(RS_EINVAL, "power-law and thin-disc profiles need r_in > 0 and r_scale > 0");
    return RS_OK;
}

double rho2(double r, int64_t S, double w)
{
    const double v = 2.0 * (double)S * r / w;
    return v * v;
}

constexpr int64_t MAX_HALF = 1 << 20;

int profile_half(const rs_profile* p, double w, int64_t* h)
{
    int rc = check_profile(p, w);
    if (rc) return rc;
    if (2.0 * p->r_out <= w) {
        *h = 0;
        return RS_OK;
    }
    const int64_t S = p->supersample;
    const double out2 = rho2(p->r_out, S, w);
    const double u2min = (double)((S + 1) % 2);
    int64_t b = 1;
    for (;; ++b) {
        const double u1 = (double)((2 * b - 1) * S + 1);
        if (!(u1 * u1 + u2min * u2min < out2)) break;
        if (b > MAX_HALF) return fail(RS_ERANGE, "profile spans more than 2^20 pixels");
    }
    *h = b - 1;
    return RS_OK;
}

int launch_profile(const rs_profile* p, double w, float* d_k, int64_t h, cudaStream_t s)
{
    int64_t want = 0;
    int rc = profile_half(p, w, &want);
    if (rc) return rc;
    if (h != want)
        return fail(RS_EINVAL, "h = %lld, the profile needs h = %lld", (long long)h,
                    (long long)want);
    const int64_t d = 2 * h + 1;
    if (2.0 * p->r_out <= w) {
        // point source: the unit impulse (normalise turns an all-zero kernel into it)
        if ((rc = cuda_fail(cudaMemsetAsync(d_k, 0, sizeof(float), s), "kernel clear")))
            return rc;
    } else {
        ProfParams P;
        P.type = p->type;
        P.S = p->supersample;
        P.h = h;
        P.t_in = (long long)ceil(rho2(p->r_in, p->supersample, w));
        P.t_out = (long long)ceil(rho2(p->r_out, p->supersample, w));
        P.hs = (float)(w / (2.0 * p->supersample));
        P.c1 = p->type == RS_PROFILE_GAUSSIAN ? (float)(1.0 / (2.0 * p->sigma1 * p->sigma1)) : 0.f;
        P.c2 = p->type == RS_PROFILE_GAUSSIAN ? (float)(1.0 / (2.0 * p->sigma2 * p->sigma2)) : 0.f;
        P.inv_rs = p->r_scale > 0.0 ? (float)(1.0 / p->r_scale) : 0.f;
        P.neg_index = (float)(-p->index);
        P.r_in = (float)p->r_in;
        const int64_t blocks = (d * d + 255) / 256;
        profile_raw_kernel<<<(unsigned)blocks, 256, 0, s>>>(P, d_k);
        if ((rc = cuda_fail(cudaGetLastError(), "profile kernel launch"))) return rc;
    }
    normalise_kernel<<<1, 1024, 0, s>>>(d_k, d * d, h * d + h);
    return cuda_fail(cudaGetLastError(), "kernel normalisation launch");
}

int check_conv(const rs_conv* c)
{
    if (!c) return fail(RS_EINVAL, "convolver is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != c->device)
        return fail(RS_EINVAL, "convolver belongs to device %d, device %d is current", c->device,
                    dev);
    return RS_OK;
}

int grid_for_n(int64_t work, int threads)
{
    int64_t need = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

// the direct path needs a map wider than a tile plus its halo
bool direct_ok(const rs_conv* c) { return c->h_direct >= 0 && c->n >= 256; }

// The spectrum of the kernel d_k (half size h) into target: the n x n
// kernel image is built in spec2 when a loaded spectrum must survive in
// spec, else in spec; d_k may live in target (it is read before the
// transform writes there).
int kernel_spectrum(rs_conv* c, const float* d_k, int64_t h, cufftComplex* target,
                    cudaStream_t s)
{
    const int64_t n = c->n;
    float* img = reinterpret_cast<float*>(c->loaded && c->spec2 ? c->spec2 : c->spec);
    if (!(c->loaded && c->spec2)) c->loaded = false;
    const unsigned rows = (unsigned)(n < (int64_t)num_sms() * 16 ? n : (int64_t)num_sms() * 16);
    scatter_kernel<<<rows, 256, 0, s>>>(d_k, h, n, img);
    int rc = cuda_fail(cudaGetLastError(), "kernel scatter launch");
    if (rc) return rc;
    if (c->own) {
        float2* t = reinterpret_cast<float2*>(target);
        if ((rc = fft_rows_forward(c->fft, img, false, t, s))) return rc;
        return fft_columns(c->fft, t, nullptr, 0.f, true, false, false, t, s);
    }
    if ((rc = cufft_fail(cufftSetStream(c->fwd, s), "set stream"))) return rc;
    return cufft_fail(cufftExecR2C(c->fwd, img, target), "R2C of the kernel");
}

int set_kernel_from_device(rs_conv* c, const float* d_k, int64_t h, cudaStream_t s)
{
    c->h_direct = -1;
    if (h <= DIRECT_HMAX) {
        // small kernel: a host copy (rotated) for the direct path; the copy to
        // pageable memory returns once the stream has reached it
        const int64_t d = 2 * h + 1;
        float k[169];
        int rc = cuda_fail(cudaMemcpyAsync(k, d_k, (size_t)(d * d) * sizeof(float),
                                           cudaMemcpyDeviceToHost, s), "kernel copy");
        if (!rc) rc = cuda_fail(cudaStreamSynchronize(s), "kernel copy sync");
        if (rc) return rc;
        for (int64_t i = 0; i < d * d; ++i) c->kf[i] = k[d * d - 1 - i];
        c->h_direct = (int)h;
    }
    int rc = kernel_spectrum(c, d_k, h, c->khat, s);
    if (rc) return rc;
    c->has_kernel = true;
    return RS_OK;
}

// own FFTs: rows (counts converted on the way in), columns with the
// spectral product between the two column transforms, rows back
int convolve_own(rs_conv* c, const void* in, bool counts, float scale, float* out, cudaStream_t s)
{
    if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15)
        return fail(RS_EINVAL, "maps must be 16-byte aligned for this size's transforms");
    float2* t = reinterpret_cast<float2*>(c->spec);
    c->loaded = false;                 // spec is overwritten
    int rc = fft_rows_forward(c->fft, in, counts, t, s);
    if (!rc) rc = fft_columns(c->fft, t, reinterpret_cast<const float2*>(c->khat), scale, true, true,
                              true, t, s);
    if (!rc) rc = fft_rows_inverse(c->fft, t, out, s);
    return rc;
}

int convolve(rs_conv* c, const float* in, float scale, float* out, cudaStream_t s)
{
    int rc;
    if (c->own) return convolve_own(c, in, false, scale, out, s);
    if ((rc = cufft_fail(cufftSetStream(c->fwd, s), "set stream")) ||
        (rc = cufft_fail(cufftSetStream(c->inv, s), "set stream")))
        return rc;
    if ((rc = cufft_fail(cufftExecR2C(c->fwd, const_cast<float*>(in), c->spec), "R2C of the map")))
        return rc;
    c->loaded = false;                 // spec is overwritten below
    spectral_product_kernel<<<grid_for_n(c->nc / 8, 256), 256, 0, s>>>(
        reinterpret_cast<const float4*>(c->spec), reinterpret_cast<const float4*>(c->khat),
        c->nc, scale, reinterpret_cast<float4*>(c->spec));
    if ((rc = cuda_fail(cudaGetLastError(), "spectral product launch"))) return rc;
    return cufft_fail(cufftExecC2R(c->inv, c->spec, out), "C2R");
}

// F(M) of a map into spec, kept for several kernels
int load_spectrum(rs_conv* c, const void* in, bool counts, cudaStream_t s)
{
    int rc;
    c->loaded = false;
    if (c->own) {
        float2* t = reinterpret_cast<float2*>(c->spec);
        if (reinterpret_cast<uintptr_t>(in) & 15)
            return fail(RS_EINVAL, "maps must be 16-byte aligned for this size's transforms");
        if ((rc = fft_rows_forward(c->fft, in, counts, t, s)) ||
            (rc = fft_columns(c->fft, t, nullptr, 0.f, true, false, false, t, s)))
            return rc;
        c->loaded = true;
        return RS_OK;
    }
    if ((rc = cufft_fail(cufftSetStream(c->fwd, s), "set stream"))) return rc;
    if ((rc = cufft_fail(cufftExecR2C(c->fwd, static_cast<float*>(const_cast<void*>(in)), c->spec),
                         "R2C of the map")))
        return rc;
    c->loaded = true;
    return RS_OK;
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" {

int rs_profile_half(const rs_profile* prof, double pixel, int64_t* h)
{
    clear_error();
    if (!h) return fail(RS_EINVAL, "h is NULL");
    return profile_half(prof, pixel, h);
}

int rs_profile_kernel(const rs_profile* prof, double pixel, float* d_kernel, int64_t h,
                      void* stream)
{
    clear_error();
    int rc = check_device_ptr(d_kernel, "d_kernel");
    if (rc) return rc;
    return launch_profile(prof, pixel, d_kernel, h, (cudaStream_t)stream);
}

int rs_conv_create(int64_t npix, rs_conv** out)
{
    clear_error();
    if (!out) return fail(RS_EINVAL, "out is NULL");
    *out = nullptr;
    if (npix < 2 || npix > RS_MAX_NPIX)
        return fail(RS_ERANGE, "npix = %lld outside [2, %d]", (long long)npix, RS_MAX_NPIX);
    rs_conv* c = new (std::nothrow) rs_conv();
    if (!c) return fail(RS_ENOMEM, "host allocation failed");
    c->n = npix;
    c->nc = npix * (npix / 2 + 1);
    cudaGetDevice(&c->device);
    int rc = RS_OK;
    long long dims[2] = {npix, npix};
    size_t w1 = 0, w2 = 0;
    const size_t spec_bytes = (size_t)c->nc * sizeof(cufftComplex);
    if (fft_supported(npix)) {
        // this library's transforms: no plans, no work area
        c->own = true;
        if ((rc = fft_plan_create(npix, &c->fft))) goto err;
        if (cudaMalloc(&c->khat, spec_bytes) != cudaSuccess ||
            cudaMalloc(&c->spec, spec_bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(RS_ENOMEM, "convolver for %lld^2 needs %.2f GB of device memory",
                      (long long)npix, 2.0 * spec_bytes / 1e9);
            goto err;
        }
        *out = c;
        return RS_OK;
    }
    if ((rc = cufft_fail(cufftCreate(&c->fwd), "plan create"))) goto err;
    c->fwd_ok = true;
    if ((rc = cufft_fail(cufftCreate(&c->inv), "plan create"))) goto err;
    c->inv_ok = true;
    if ((rc = cufft_fail(cufftSetAutoAllocation(c->fwd, 0), "auto allocation")) ||
        (rc = cufft_fail(cufftSetAutoAllocation(c->inv, 0), "auto allocation")) ||
        (rc = cufft_fail(cufftMakePlanMany64(c->fwd, 2, dims, nullptr, 1, 0, nullptr, 1, 0,
                                             CUFFT_R2C, 1, &w1), "R2C plan")) ||
        (rc = cufft_fail(cufftMakePlanMany64(c->inv, 2, dims, nullptr, 1, 0, nullptr, 1, 0,
                                             CUFFT_C2R, 1, &w2), "C2R plan")))
        goto err;
    c->work_bytes = w1 > w2 ? w1 : w2;
    if (cudaMalloc(&c->khat, spec_bytes) != cudaSuccess ||
        cudaMalloc(&c->spec, spec_bytes) != cudaSuccess ||
        (c->work_bytes && cudaMalloc(&c->work, c->work_bytes) != cudaSuccess)) {
        cudaGetLastError();
        rc = fail(RS_ENOMEM, "convolver for %lld^2 needs %.2f GB of device memory",
                  (long long)npix, (2.0 * spec_bytes + c->work_bytes) / 1e9);
        goto err;
    }
    if ((rc = cufft_fail(cufftSetWorkArea(c->fwd, c->work), "work area")) ||
        (rc = cufft_fail(cufftSetWorkArea(c->inv, c->work), "work area")))
        goto err;
    *out = c;
    return RS_OK;
err:
    rs_conv_destroy(c);
    return rc;
}

void rs_conv_destroy(rs_conv* c)
{
    if (!c) return;
    if (c->fwd_ok) cufftDestroy(c->fwd);
    if (c->inv_ok) cufftDestroy(c->inv);
    if (c->own) fft_plan_destroy(&c->fft);
    if (c->khat) cudaFree(c->khat);
    if (c->spec) cudaFree(c->spec);
    if (c->spec2) cudaFree(c->spec2);
    for (int k = 1; k < RS_CONV_SLOTS; ++k)
        if (c->slot[k]) cudaFree(c->slot[k]);
    if (c->work) cudaFree(c->work);
    delete c;
}

int rs_conv_bytes(const rs_conv* c, size_t* bytes)
{
    clear_error();
    if (!c || !bytes) return fail(RS_EINVAL, "NULL argument");
    size_t nbuf = c->spec2 ? 3 : 2;
    for (int k = 1; k < RS_CONV_SLOTS; ++k) nbuf += c->slot[k] != nullptr;
    *bytes = nbuf * (size_t)c->nc * sizeof(cufftComplex) + c->work_bytes +
             (c->own ? rs::fft_plan_bytes(c->n) : 0);
    return RS_OK;
}

int rs_conv_set_profile(rs_conv* c, const rs_profile* prof, double pixel, void* stream)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    int64_t h = 0;
    if ((rc = profile_half(prof, pixel, &h))) return rc;
    if (2 * h + 1 > c->n)
        return fail(RS_ERANGE, "profile kernel (%lld pixels wide) wider than the %lld^2 map",
                    (long long)(2 * h + 1), (long long)c->n);
    cudaStream_t s = (cudaStream_t)stream;
    c->has_kernel = false;
    float* small = reinterpret_cast<float*>(c->khat);   // (2h+1)^2 <= n (n + 2) floats
    if ((rc = launch_profile(prof, pixel, small, h, s))) return rc;
    return set_kernel_from_device(c, small, h, s);
}

int rs_conv_set_kernel(rs_conv* c, const float* d_kernel, int64_t h, void* stream)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    if ((rc = check_device_ptr(d_kernel, "d_kernel"))) return rc;
    if (h < 0 || 2 * h + 1 > c->n)
        return fail(RS_ERANGE, "kernel half size %lld does not fit the %lld^2 map", (long long)h,
                    (long long)c->n);
    c->has_kernel = false;
    return set_kernel_from_device(c, d_kernel, h, (cudaStream_t)stream);
}

int rs_conv_apply_counts(rs_conv* c, const int32_t* d_counts, double scale, float* d_out,
                         void* stream)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    if (!c->has_kernel) return fail(RS_EINVAL, "no kernel set on the convolver");
    if (!isfinite(scale)) return fail(RS_EINVAL, "scale must be finite");
    if ((rc = check_device_ptr(d_counts, "d_counts")) || (rc = check_device_ptr(d_out, "d_out")))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    c->loaded = false;
    if (direct_ok(c)) {
        DirectArgs A;
        memcpy(A.kf, c->kf, sizeof(A.kf));
        const int32_t* src = d_counts;
        if ((const void*)d_counts == (const void*)d_out) {   // in place: read a copy
            c->loaded = false;
            if ((rc = cuda_fail(cudaMemcpyAsync(c->spec, d_counts, (size_t)(c->n * c->n) * 4,
                                                cudaMemcpyDeviceToDevice, s), "input copy")))
                return rc;
            src = reinterpret_cast<const int32_t*>(c->spec);
        }
        return launch_direct<int32_t>(c->h_direct, src, (float)scale, c->n, A, d_out, s);
    }
    const float sc = (float)(scale / ((double)c->n * (double)c->n));
    if (c->own) return convolve_own(c, d_counts, true, sc, d_out, s);
    // int32 -> float, exact below 2^24; the scale rides on the spectral product
    if ((rc = launch_magnification(d_counts, c->n * c->n, 1.0f, d_out, s))) return rc;
    return convolve(c, d_out, (float)(scale / ((double)c->n * (double)c->n)), d_out, s);
}

int rs_conv_apply(rs_conv* c, const float* d_map, float* d_out, void* stream)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    if (!c->has_kernel) return fail(RS_EINVAL, "no kernel set on the convolver");
    if ((rc = check_device_ptr(d_map, "d_map")) || (rc = check_device_ptr(d_out, "d_out")))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    c->loaded = false;
    if (direct_ok(c)) {
        DirectArgs A;
        memcpy(A.kf, c->kf, sizeof(A.kf));
        const float* src = d_map;
        if (d_map == d_out) {                                 // in place: read a copy
            c->loaded = false;
            if ((rc = cuda_fail(cudaMemcpyAsync(c->spec, d_map, (size_t)(c->n * c->n) * 4,
                                                cudaMemcpyDeviceToDevice, s), "input copy")))
                return rc;
            src = reinterpret_cast<const float*>(c->spec);
        }
        return launch_direct<float>(c->h_direct, src, 1.0f, c->n, A, d_out, s);
    }
    return convolve(c, d_map, (float)(1.0 / ((double)c->n * (double)c->n)), d_out, s);
}

static int ensure_spec2(rs_conv* c)
{
    if (c->spec2) return RS_OK;
    if (cudaMalloc(&c->spec2, (size_t)c->nc * sizeof(cufftComplex)) != cudaSuccess) {
        cudaGetLastError();
        c->spec2 = nullptr;
        return fail(RS_ENOMEM, "second spectrum buffer (%.2f GB) could not be allocated",
                    (double)c->nc * sizeof(cufftComplex) / 1e9);
    }
    return RS_OK;
}

int rs_conv_load_counts(rs_conv* c, const int32_t* d_counts, double scale, void* stream)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    if (!isfinite(scale)) return fail(RS_EINVAL, "scale must be finite");
    if ((rc = check_device_ptr(d_counts, "d_counts")) || (rc = ensure_spec2(c))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->own) {
        if ((rc = load_spectrum(c, d_counts, true, s))) return rc;   // converted in the row pass
    } else {
        // int32 -> float into the second buffer (exact below 2^24), then F(M)
        float* real = reinterpret_cast<float*>(c->spec2);
        if ((rc = launch_magnification(d_counts, c->n * c->n, 1.0f, real, s))) return rc;
        if ((rc = load_spectrum(c, real, false, s))) return rc;
    }
    c->load_scale = scale;
    return RS_OK;
}

int rs_conv_load(rs_conv* c, const float* d_map, void* stream)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    if ((rc = check_device_ptr(d_map, "d_map")) || (rc = ensure_spec2(c))) return rc;
    if ((rc = load_spectrum(c, d_map, false, (cudaStream_t)stream))) return rc;
    c->load_scale = 1.0;
    return RS_OK;
}

int rs_conv_apply_loaded(rs_conv* c, float* d_out, void* stream)
{
    return rs_conv_apply_loaded_slot(c, 0, d_out, stream);
}

int rs_conv_set_profile_slot(rs_conv* c, int slot, const rs_profile* prof, double pixel,
                             void* stream)
{
    clear_error();
    if (slot == 0) return rs_conv_set_profile(c, prof, pixel, stream);
    int rc = check_conv(c);
    if (rc) return rc;
    if (slot < 1 || slot >= RS_CONV_SLOTS)
        return fail(RS_EINVAL, "slot %d outside 0..%d", slot, RS_CONV_SLOTS - 1);
    int64_t h = 0;
    if ((rc = profile_half(prof, pixel, &h))) return rc;
    if (2 * h + 1 > c->n)
        return fail(RS_ERANGE, "profile kernel (%lld pixels wide) wider than the %lld^2 map",
                    (long long)(2 * h + 1), (long long)c->n);
    if (!c->slot[slot]) {
        if (cudaMalloc(&c->slot[slot], (size_t)c->nc * sizeof(cufftComplex)) != cudaSuccess) {
            cudaGetLastError();
            c->slot[slot] = nullptr;
            return fail(RS_ENOMEM, "kernel slot %d (%.2f GB) could not be allocated", slot,
                        (double)c->nc * sizeof(cufftComplex) / 1e9);
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    c->slot_set[slot] = false;
    float* small = reinterpret_cast<float*>(c->slot[slot]);   // read before the transform
    if ((rc = launch_profile(prof, pixel, small, h, s))) return rc;
    if ((rc = kernel_spectrum(c, small, h, c->slot[slot], s))) return rc;
    c->slot_set[slot] = true;
    return RS_OK;
}

int rs_conv_apply_loaded_slot(rs_conv* c, int slot, float* d_out, void* stream)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    if (slot < 0 || slot >= RS_CONV_SLOTS)
        return fail(RS_EINVAL, "slot %d outside 0..%d", slot, RS_CONV_SLOTS - 1);
    const cufftComplex* kh = slot == 0 ? c->khat : c->slot[slot];
    if (slot == 0 ? !c->has_kernel : !c->slot_set[slot])
        return fail(RS_EINVAL, "no kernel in slot %d", slot);
    if (!c->loaded || !c->spec2) return fail(RS_EINVAL, "no map loaded on the convolver");
    if ((rc = check_device_ptr(d_out, "d_out"))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const float scale = (float)(c->load_scale / ((double)c->n * (double)c->n));
    if (c->own) {
        float2* t2 = reinterpret_cast<float2*>(c->spec2);
        if (reinterpret_cast<uintptr_t>(d_out) & 15)
            return fail(RS_EINVAL, "maps must be 16-byte aligned for this size's transforms");
        if ((rc = fft_columns(c->fft, reinterpret_cast<const float2*>(c->spec),
                              reinterpret_cast<const float2*>(kh), scale, false, true, true, t2, s)))
            return rc;
        return fft_rows_inverse(c->fft, t2, d_out, s);
    }
    spectral_product_kernel<<<grid_for_n(c->nc / 8, 256), 256, 0, s>>>(
        reinterpret_cast<const float4*>(c->spec), reinterpret_cast<const float4*>(kh), c->nc,
        scale, reinterpret_cast<float4*>(c->spec2));
    if ((rc = cuda_fail(cudaGetLastError(), "spectral product launch"))) return rc;
    if ((rc = cufft_fail(cufftSetStream(c->inv, s), "set stream"))) return rc;
    return cufft_fail(cufftExecC2R(c->inv, c->spec2, d_out), "C2R");
}

int rs_conv_fft_kind(const rs_conv* c, int* kind)
{
    clear_error();
    int rc = check_conv(c);
    if (rc) return rc;
    if (!kind) return fail(RS_EINVAL, "kind is NULL");
    *kind = c->own ? RS_CONV_FFT_OWN : RS_CONV_FFT_CUFFT;
    return RS_OK;
}

int rs_pixel_flux(const float* d_map, int64_t npix, const int16_t* d_xy, uint64_t seed,
                  int64_t k, rs_pixflux* d_records, void* stream)
{
    clear_error();
    if (npix < 1 || npix > RS_PIXEL_FLUX_MAX_NPIX)
        return fail(RS_ERANGE, "npix = %lld outside [1, %d] (int16 locations)", (long long)npix,
                    RS_PIXEL_FLUX_MAX_NPIX);
    if (k < 0) return fail(RS_EINVAL, "k < 0");
    if (k == 0) return RS_OK;
    int rc;
    if ((rc = check_device_ptr(d_map, "d_map")) || (rc = check_device_ptr(d_records, "d_records")) ||
        (d_xy && (rc = check_device_ptr(d_xy, "d_xy"))))
        return rc;
    if ((reinterpret_cast<uintptr_t>(d_records) & 7) || (reinterpret_cast<uintptr_t>(d_xy) & 3))
        return fail(RS_EINVAL, "d_records must be 8-byte and d_xy 4-byte aligned");
    pixel_flux_kernel<<<grid_for_n(k, 256), 256, 0, (cudaStream_t)stream>>>(
        d_map, npix, reinterpret_cast<const short2*>(d_xy), (unsigned long long)seed, k,
        reinterpret_cast<uint2*>(d_records));
    return cuda_fail(cudaGetLastError(), "pixel flux launch");
}

int rs_value_histogram(const float* d_v, int64_t n, const float* h_edges, int64_t n_edges,
                       int64_t* d_hist, void* stream)
{
    clear_error();
    if (!h_edges || n_edges < 1 || n_edges > MAX_EDGES)
        return fail(RS_EINVAL, "n_edges must be in 1..%d with edges given", MAX_EDGES);
    if (n < 0) return fail(RS_EINVAL, "n < 0");
    EdgeArgs local;   // passed by value: the launch copies it
    local.n = (int32_t)n_edges;
    for (int64_t i = 0; i < n_edges; ++i) {
        if (!(h_edges[i] == h_edges[i]) || (i && !(h_edges[i - 1] < h_edges[i])))
            return fail(RS_EINVAL, "edges must be ascending and not NaN (edge %lld)",
                        (long long)i);
        local.e[i] = h_edges[i];
    }
    {
        // buckets: the smallest shift that tables the first to the last edge
        // in HIST_TABLE buckets
        auto key = [](float e) {
            if (e == 0.0f) e = 0.0f;      // -0 -> +0
            uint32_t b;
            memcpy(&b, &e, 4);
            return ordkey_bits(b);
        };
        const uint32_t k0 = key(local.e[0]), k1 = key(local.e[n_edges - 1]);
        int sh = 1;                       // keys >> sh fit an int
        while (sh < 31 && (k1 >> sh) - (k0 >> sh) + 1 > (uint32_t)HIST_TABLE) ++sh;
        local.shift = sh;
        local.key_lo = k0 >> sh;
        local.nkeys = (int32_t)((k1 >> sh) - (k0 >> sh) + 1);
    }
    int rc;
    if ((rc = check_device_ptr(d_hist, "d_hist")) || (n > 0 && (rc = check_device_ptr(d_v, "d_v"))))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = launch_fill_i64(d_hist, n_edges + 1, 0, s))) return rc;
    if (n == 0) return RS_OK;
    // the bucket table, in a library-owned slot used in stream order; the
    // lock covers taking the slot, the launches and the event record
    std::lock_guard<std::mutex> lock(g_hist_mu);
    HistSlot* slot = nullptr;
    if ((rc = hist_slot(s, &slot))) return rc;
    table_kernel<<<(local.nkeys + 2 + 255) / 256, 256, 0, s>>>(local, slot->T);
    const int R = hist_copies((int)n_edges, local.nkeys);
    const size_t dyn = hist_smem_bytes((int)n_edges, local.nkeys, R);
    // one CTA of 1024 threads per SM (the copies take most of shared memory)
    int64_t want = (n / 4 + HIST_THREADS - 1) / HIST_THREADS;
    const int64_t cap = (int64_t)num_sms();
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    auto fn = R == 32 ? value_hist_kernel<32> : R == 16 ? value_hist_kernel<16> : value_hist_kernel<8>;
    fn<<<(int)want, HIST_THREADS, dyn, s>>>(d_v, n, local, slot->T,
                                           reinterpret_cast<unsigned long long*>(d_hist));
    if ((rc = cuda_fail(cudaGetLastError(), "value histogram launch"))) return rc;
    return cuda_fail(cudaEventRecord(slot->ev, s), "histogram slot record");
}

}  // extern "C"
