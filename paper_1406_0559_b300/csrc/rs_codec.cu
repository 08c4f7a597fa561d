// rs_codec.cu -- indexed count maps (App. B) and map previews / colorbar
// (Sec. 3.2.1, Sec. 4.6).
//
// Encoding: one pass finds the smallest and largest count; a bitmap with one
// bit per count value marks the values present; an exclusive scan of the
// words' popcounts gives every value its rank -- its position in the
// ascending table of distinct counts, the set bits below it -- and writes
// the table; a last pass replaces each count by its rank and packs
// the ranks, 32 pixels per thread, into exactly `bits` words per group (the
// stream is LSB first, so no two threads share a word).  Decoding unpacks a
// group per thread and looks the counts up in the table.  Integer work,
// bit-exact.  HBM: min/max 4 B/px, marking 4 B/px, packing 4 B/px + b/8 B/px;
// decoding b/8 + 4 B/px.  The bitmap and the per-word prefix (8 B per 32
// count values, 250 KB at GERLUMPH's 1e6) stay in L1/L2.
#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <utility>

#include <climits>

#include "rs_internal.cuh"
#include "../../include/rs_codec.h"

namespace rs {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr size_t SMEM_BITMAP_BYTES = 32 * 1024;   // per-CTA bitmaps up to 2^18 values
constexpr int SCAN_ITEMS = 16;
constexpr int64_t SCAN_CHUNK = (int64_t)SCAN_THREADS * SCAN_ITEMS;

__global__ void minmax_init_kernel(int* mm)
{
    mm[0] = INT_MAX;
    mm[1] = INT_MIN;
}

__global__ void __launch_bounds__(256) minmax_kernel(const int32_t* __restrict__ c, int64_t n,
                                                     int* __restrict__ mm)
{
    int lo = INT_MAX, hi = INT_MIN;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n4 = (reinterpret_cast<uintptr_t>(c) & 15) == 0 ? n / 4 : 0;
    const int4* c4 = reinterpret_cast<const int4*>(c);
    for (int64_t i = t0; i < n4; i += stride) {
        const int4 v = __ldcs(c4 + i);
        lo = min(lo, min(min(v.x, v.y), min(v.z, v.w)));
        hi = max(hi, max(max(v.x, v.y), max(v.z, v.w)));
    }
    for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
        lo = min(lo, c[i]);
        hi = max(hi, c[i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm, lo);
        atomicMax(mm + 1, hi);
    }
}

// Presence bitmap: bit v of gbits set for every count v present
// (0 <= v <= vmax).  When the bitmap fits in shared memory each CTA marks its
// own copy -- reading the word first, so that the many pixels repeating a
// marked value cost no atomic -- and ORs its non-zero words into the global
// bitmap at the end; otherwise the global words are tested and set directly.
template <bool SMEM>
__global__ void __launch_bounds__(256) mark_kernel(const int32_t* __restrict__ c, int64_t n,
                                                   int vmax, unsigned* __restrict__ gbits)
{
    extern __shared__ unsigned sbits[];
    const int nw = (vmax >> 5) + 1;
    if (SMEM) {
        for (int k = threadIdx.x; k < nw; k += blockDim.x) sbits[k] = 0u;
        __syncthreads();
    }
    unsigned* bits = SMEM ? sbits : gbits;
    auto mark = [&](int v) {
        if (v < 0 || v > vmax) return;
        const unsigned m = 1u << (v & 31);
        const unsigned cur = SMEM ? bits[v >> 5] : __ldg(bits + (v >> 5));
        if (!(cur & m)) atomicOr(bits + (v >> 5), m);
    };
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n4 = (reinterpret_cast<uintptr_t>(c) & 15) == 0 ? n / 4 : 0;
    const int4* c4 = reinterpret_cast<const int4*>(c);
    int64_t i = t0;
    for (; i + stride < n4; i += 2 * stride) {
        const int4 a = __ldcs(c4 + i), b = __ldcs(c4 + i + stride);
        mark(a.x); mark(a.y); mark(a.z); mark(a.w);
        mark(b.x); mark(b.y); mark(b.z); mark(b.w);
    }
    for (; i < n4; i += stride) {
        const int4 a = __ldcs(c4 + i);
        mark(a.x); mark(a.y); mark(a.z); mark(a.w);
    }
    for (int64_t j = 4 * n4 + t0; j < n; j += stride) mark(__ldcs(c + j));
    if (SMEM) {
        __syncthreads();
        for (int k = threadIdx.x; k < nw; k += blockDim.x)
            if (sbits[k]) atomicOr(gbits + k, sbits[k]);
    }
}

// Phase A: number of set bits in each SCAN_CHUNK-word chunk of the bitmap.
__global__ void __launch_bounds__(SCAN_THREADS) chunk_sum_kernel(const unsigned* __restrict__ f,
                                                                 int64_t len,
                                                                 int* __restrict__ part)
{
    __shared__ int red[SCAN_THREADS / 32];
    const int64_t base = blockIdx.x * SCAN_CHUNK;
    int s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k * SCAN_THREADS + threadIdx.x;
        if (i < len) s += __popc(f[i]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Phase B (one CTA): exclusive scan of the chunk sums; total into *total.
__global__ void __launch_bounds__(1024) part_scan_kernel(int* __restrict__ part, int64_t nb,
                                                         long long* __restrict__ total)
{
    __shared__ int wsum[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int64_t i = b0 + threadIdx.x;
        const int v = i < nb ? part[i] : 0;
        int x = v;   // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            int w = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if ((int)threadIdx.x >= o) w += y;
            }
            wsum[threadIdx.x] = w;   // inclusive over warps
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5;
        const long long excl = carry + (warp ? wsum[warp - 1] : 0) + (x - v);
        if (i < nb) part[i] = (int)excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Phase C: wp[w] = set bits in the words before w (exclusive scan of the
// popcounts), and the table: the value of every set bit at its rank.
__global__ void __launch_bounds__(SCAN_THREADS) rank_kernel(const unsigned* __restrict__ f,
                                                            int64_t len,
                                                            const int* __restrict__ part,
                                                            int* __restrict__ wp,
                                                            int32_t* __restrict__ table,
                                                            int64_t table_cap)
{
    __shared__ int wsum[SCAN_THREADS / 32];
    const int64_t base = blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    unsigned w[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        w[k] = i < len ? f[i] : 0u;
        s += __popc(w[k]);
    }
    int x = s;   // inclusive scan of the thread sums over the block
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < SCAN_THREADS / 32 ? wsum[threadIdx.x] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if ((int)threadIdx.x >= o) v += y;
        }
        if (threadIdx.x < SCAN_THREADS / 32) wsum[threadIdx.x] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    int r = part[blockIdx.x] + (warp ? wsum[warp - 1] : 0) + (x - s);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        const int64_t i = base + k;
        if (i < len) {
            wp[i] = r;
            unsigned m = w[k];
            int rr = r;
            while (m) {
                const int bit = __ffs(m) - 1;
                if (rr < table_cap) table[rr] = (int32_t)(i * 32 + bit);
                ++rr;
                m &= m - 1;
            }
        }
        r += __popc(w[k]);
    }
}

// Packing and unpacking: a warp takes a chunk of 1024 pixels = 32 groups of
// 32; lane g packs group g into exactly `bits` words (the stream is LSB
// first, so groups never share a word).  Counts and words go through shared
// memory so that every global access of the warp is one contiguous run:
// words sit at stride `bits` per lane with one pad word per 32.  The rank of
// a count present in the map is the number of set bitmap bits below it.
__device__ __forceinline__ int wpad(int x) { return x + (x >> 5); }

// Opt a kernel into more dynamic shared memory than the default, once per
// (device, kernel family, bit width); setting it twice is harmless.
int allow_dynamic_smem(const void* kern, int family, int bits, int bytes)
{
    static std::atomic<uint32_t> done[64][2];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    const uint32_t bit = 1u << (bits - 1);
    if (done[dev][family].load() & bit) return RS_OK;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "shared-memory attribute");
    done[dev][family].fetch_or(bit);
    return RS_OK;
}

// Packing: one kernel per bit width.  A warp loads a chunk of 1024 counts
// with coalesced 16-byte loads (lane l, load q: counts 128 q + 4 l .. + 3;
// the next chunk's loads are issued before this chunk is packed, so one
// chunk is in flight per warp while another is packed), writes them into
// its shared buffer as 32 rows of 32 (row g = group g, padded to 36 words so
// that 16-byte accesses are conflict-free), and lane g then reads its
// group's row four counts at a time, ranks them and ORs the indices into
// BITS words at constant offsets; the words leave through the same buffer
// with coalesced stores.  Only the prefetched chunk and the words are held
// in registers (not the group's 32 counts), so up to four blocks of 8 warps
// fit per SM.  The rank of a count is one lookup in a table of every rank
// 0..vmax built in shared memory by each block when vmax < PACK_SMEM_RANKS,
// else the presence bitmap and word prefix in global memory.  Counts are
// clamped to vmax (the encoder found it), so no lookup leaves its table.
// Pixels past the end pack as index 0, so the last word's unused bits are
// zero.
constexpr int DEC_WARPS = 8;
constexpr int DEC_ROW = 36;
constexpr int64_t PACK_SMEM_RANKS = 16384;    // 64 KB of shared memory

// blocks per SM the register budget is sized for: 4 (64 registers) while the
// words and the prefetched chunk fit without spilling
__host__ __device__ constexpr int pack_min_blocks(int bits, bool sr) { return sr && bits <= 20 ? 4 : 2; }

template <int BITS, bool SR>
__global__ void __launch_bounds__(32 * DEC_WARPS, pack_min_blocks(BITS, SR)) pack_kernel(
    const int32_t* __restrict__ c, int64_t n, const unsigned* __restrict__ gbits,
    const int* __restrict__ wp, int vmax, uint32_t* __restrict__ words)
{
    __shared__ __align__(16) uint32_t sb[DEC_WARPS][32 * DEC_ROW];
    extern __shared__ unsigned s_rank[];    // SR: rank of every count 0..vmax
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    auto bitmap_rank = [&](int v) -> uint32_t {
        const int q = v >> 5;
        return (uint32_t)__ldg(wp + q) + __popc(__ldg(gbits + q) & ((1u << (v & 31)) - 1u));
    };
    if (SR) {
        for (int k = threadIdx.x; k <= vmax; k += blockDim.x) s_rank[k] = bitmap_rank(k);
        __syncthreads();
    }
    auto rank = [&](int v) -> uint32_t {
        const int u = (int)min((unsigned)v, (unsigned)vmax);
        return SR ? s_rank[u] : bitmap_rank(u);
    };
    uint32_t* w = sb[wid];
    const bool vec = (reinterpret_cast<uintptr_t>(c) & 15) == 0;
    const int64_t chunks = (n + 1023) / 1024;
    const int64_t stride = (int64_t)gridDim.x * DEC_WARPS;
    // coalesced loads of a chunk: nx[q] = counts 128 q + 4 lane .. + 3
    auto load_chunk = [&](int64_t ch, int4 (&r)[8]) {
        const int64_t base = ch * 1024;
        const int m = (int)min((int64_t)1024, n - base);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int p = 128 * q + 4 * lane;
            if (vec && p + 3 < m) {
                r[q] = __ldcs(reinterpret_cast<const int4*>(c + base + p));
            } else {
                r[q].x = p < m ? __ldcs(c + base + p) : 0;
                r[q].y = p + 1 < m ? __ldcs(c + base + p + 1) : 0;
                r[q].z = p + 2 < m ? __ldcs(c + base + p + 2) : 0;
                r[q].w = p + 3 < m ? __ldcs(c + base + p + 3) : 0;
            }
        }
    };
    int4 nx[8];
    int64_t ch = blockIdx.x * (int64_t)DEC_WARPS + wid;
    if (ch < chunks) load_chunk(ch, nx);
    for (; ch < chunks; ch += stride) {
        const int64_t base = ch * 1024;
        const int m = (int)min((int64_t)1024, n - base);      // pixels in this chunk
        // counts 128 q + 4 lane + e sit in row 4 q + lane / 8, column 4 (lane % 8) + e
#pragma unroll
        for (int q = 0; q < 8; ++q)
            *reinterpret_cast<int4*>(w + (4 * q + (lane >> 3)) * DEC_ROW + 4 * (lane & 7)) = nx[q];
        __syncwarp();
        if (ch + stride < chunks) load_chunk(ch + stride, nx);
        uint32_t wr[BITS + 1];
#pragma unroll
        for (int t = 0; t <= BITS; ++t) wr[t] = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int4 u = *reinterpret_cast<const int4*>(w + lane * DEC_ROW + 4 * j);
            const int cv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t idx = rank(cv[e]);
                const int pos = (4 * j + e) * BITS, wi = pos >> 5, sh = pos & 31;
                wr[wi] |= idx << sh;
                if (sh + BITS > 32) wr[wi + 1] |= idx >> (32 - sh);
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < BITS; ++t) w[wpad(lane * BITS + t)] = wr[t];
        __syncwarp();
        const int nw = (m * BITS + 31) / 32;   // words of this chunk
        uint32_t* dst = words + ch * 32 * (int64_t)BITS;
        for (int j = lane; j < nw; j += 32) __stcs(dst + j, w[wpad(j)]);
        __syncwarp();
    }
}

using PackFn = void (*)(const int32_t*, int64_t, const unsigned*, const int*, int, uint32_t*);

template <bool SR, int... B>
constexpr std::array<PackFn, sizeof...(B)> pack_table(std::integer_sequence<int, B...>)
{
    return {{pack_kernel<B + 1, SR>...}};
}

// pack kernels by bit width (index bits - 1)
const std::array<PackFn, 32> kPackSmem = pack_table<true>(std::make_integer_sequence<int, 32>{});
const std::array<PackFn, 32> kPackGlobal = pack_table<false>(std::make_integer_sequence<int, 32>{});

// Decoding: the same chunks, one kernel per bit width (BITS is a template
// parameter, so every bit offset below is a constant).  A warp reads the
// chunk's words into its shared buffer with coalesced loads; each lane
// copies its group's BITS words into registers and cuts its 32 indices out
// of them with funnel shifts (no dependent chain); the table lookups are
// gathers from a table of up to DEC_SMEM_TABLE entries staged in shared
// memory (a gather there costs a few bank wavefronts; through L1 it costs
// one per distinct line), else from global memory; indices not below
// `distinct` give -1.  The counts go back through the same buffer,
// transposed (rows of 36 ints, so that 16-byte accesses are conflict-free),
// and leave as 16-byte coalesced stores.
constexpr int64_t DEC_SMEM_TABLE = 16384;

template <int BITS, bool TAB>
__global__ void __launch_bounds__(32 * DEC_WARPS) unpack_kernel(
    const uint32_t* __restrict__ words, int64_t n, const int32_t* __restrict__ table,
    int64_t distinct, int32_t* __restrict__ c)
{
    __shared__ __align__(16) uint32_t sb[DEC_WARPS][32 * DEC_ROW];
    extern __shared__ int s_table[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (TAB) {
        for (int64_t k = threadIdx.x; k < distinct; k += blockDim.x) s_table[k] = __ldg(table + k);
        __syncthreads();
    }
    uint32_t* w = sb[wid];
    int* v = reinterpret_cast<int*>(w);
    const bool vec = (reinterpret_cast<uintptr_t>(c) & 15) == 0;
    const int64_t chunks = (n + 1023) / 1024;
    for (int64_t ch = blockIdx.x * (int64_t)DEC_WARPS + wid; ch < chunks;
         ch += (int64_t)gridDim.x * DEC_WARPS) {
        const int64_t base = ch * 1024;
        const int m = (int)min((int64_t)1024, n - base);
        const int nw = (m * BITS + 31) / 32;
        const uint32_t* src = words + ch * 32 * (int64_t)BITS;
        for (int j = lane; j < nw; j += 32) w[wpad(j)] = __ldcs(src + j);
        __syncwarp();
        // words past nw hold stale values; the indices cut from them belong
        // to pixels past m, whose lookups stay in bounds and are not stored
        uint32_t wr[BITS + 1];
#pragma unroll
        for (int t = 0; t < BITS; ++t) wr[t] = w[wpad(lane * BITS + t)];
        wr[BITS] = 0u;
        __syncwarp();
        int val[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            constexpr uint32_t mask = BITS == 32 ? 0xffffffffu : ((1u << (BITS & 31)) - 1u);
            const int pos = k * BITS, wi = pos >> 5, sh = pos & 31;
            const uint32_t x = sh + BITS <= 32 ? (wr[wi] >> sh)
                                               : __funnelshift_r(wr[wi], wr[wi + 1], sh);
            const uint32_t idx = x & mask;
            val[k] = (int64_t)idx < distinct ? (TAB ? s_table[idx] : __ldg(table + idx)) : -1;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            *reinterpret_cast<int4*>(v + lane * DEC_ROW + 4 * q) =
                make_int4(val[4 * q], val[4 * q + 1], val[4 * q + 2], val[4 * q + 3]);
        __syncwarp();
        // pixel p of the chunk (group p / 32, member p % 32) sits at
        // v[(p / 32) * DEC_ROW + p % 32]
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int p = 128 * q + 4 * lane;
            const int4 u = *reinterpret_cast<const int4*>(v + (p >> 5) * DEC_ROW + (p & 31));
            if (vec && p + 3 < m) {
                __stcs(reinterpret_cast<int4*>(c + base + p), u);
            } else {
                if (p < m) __stcs(c + base + p, u.x);
                if (p + 1 < m) __stcs(c + base + p + 1, u.y);
                if (p + 2 < m) __stcs(c + base + p + 2, u.z);
                if (p + 3 < m) __stcs(c + base + p + 3, u.w);
            }
        }
        __syncwarp();
    }
}

using UnpackFn = void (*)(const uint32_t*, int64_t, const int32_t*, int64_t, int32_t*);

template <bool TAB, int... B>
constexpr std::array<UnpackFn, sizeof...(B)> unpack_table(std::integer_sequence<int, B...>)
{
    return {{unpack_kernel<B + 1, TAB>...}};
}

// unpack kernels by bit width (index bits - 1)
const std::array<UnpackFn, 32> kUnpackSmem = unpack_table<true>(std::make_integer_sequence<int, 32>{});
const std::array<UnpackFn, 32> kUnpackGlobal = unpack_table<false>(std::make_integer_sequence<int, 32>{});

// ---- previews ----------------------------------------------------------------

template <typename T>
struct PreviewArgs {
    T thr[256];           // 255 thresholds + NaN
    uint32_t lut[256];    // RGBA8
    int32_t has_lut, pad_;
};

template <typename M, typename T>
__global__ void __launch_bounds__(256) preview_kernel(const M* __restrict__ map, int64_t n,
                                                      int64_t s,
                                                      const __grid_constant__ PreviewArgs<T> A,
                                                      uint8_t* __restrict__ gray,
                                                      uint32_t* __restrict__ rgba)
{
    __shared__ double thr[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) thr[i] = (double)A.thr[i];
    __syncthreads();
    const int64_t total = s * s;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / s, col = t % s;
        const int64_t q = (2 * r + 1) * n / (2 * s);
        const int64_t p = (2 * col + 1) * n / (2 * s);
        const double v = (double)map[q * n + p];
        int g = 0;
#pragma unroll
        for (int k = 7; k >= 0; --k) g += thr[g + (1 << k) - 1] <= v ? (1 << k) : 0;
        if (gray) gray[t] = (uint8_t)g;
        if (rgba) rgba[t] = A.lut[g];
    }
}

__global__ void colorize_kernel(const uint8_t* __restrict__ gray, int64_t m,
                                const __grid_constant__ PreviewArgs<float> A,
                                uint32_t* __restrict__ rgba)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x)
        rgba[t] = A.lut[gray[t]];
}

int grid_cap(int64_t work, int threads, int per_sm)
{
    int64_t need = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

int build_lut(const int32_t* pos, const uint8_t* rgb, int m, uint8_t* lut)
{
    if (!pos || !rgb || !lut) return fail(RS_EINVAL, "NULL colour stops or table");
    if (m < 2 || m > 256) return fail(RS_EINVAL, "need 2..256 colour stops");
    if (pos[0] != 0 || pos[m - 1] != 255) return fail(RS_EINVAL, "stops must run from 0 to 255");
    for (int k = 1; k < m; ++k)
        if (pos[k] < pos[k - 1]) return fail(RS_EINVAL, "stop positions must not decrease");
    for (int i = 0; i < 256; ++i) {
        int a = -1;
        for (int k = 0; k + 1 < m; ++k)
            if (pos[k] <= i && i < pos[k + 1]) a = k;
        for (int ch = 0; ch < 3; ++ch) {
            if (a < 0) {
                lut[3 * i + ch] = rgb[3 * (m - 1) + ch];
                continue;
            }
            const int pa = pos[a], pb = pos[a + 1], span = pb - pa;
            const int ca = rgb[3 * a + ch], cb = rgb[3 * (a + 1) + ch];
            lut[3 * i + ch] = (uint8_t)((ca * (pb - i) + cb * (i - pa) + span / 2) / span);
        }
    }
    return RS_OK;
}

template <typename M, typename T>
int preview(const M* d_map, int64_t npix, int64_t s, const T* h_thr, const uint8_t* h_lut,
            uint8_t* d_gray, uint32_t* d_rgba, cudaStream_t st)
{
    if (npix < 1 || npix > RS_MAX_NPIX) return fail(RS_ERANGE, "npix outside [1, %d]", RS_MAX_NPIX);
    if (s < 1 || s > npix) return fail(RS_EINVAL, "preview side must be in 1..npix");
    if (!h_thr) return fail(RS_EINVAL, "thresholds are NULL");
    if (d_rgba && !h_lut) return fail(RS_EINVAL, "colours asked for without a table");
    int rc;
    if ((rc = check_device_ptr(d_map, "d_map")) || (d_gray && (rc = check_device_ptr(d_gray, "d_gray"))) ||
        (d_rgba && (rc = check_device_ptr(d_rgba, "d_rgba"))))
        return rc;
    PreviewArgs<T> A;
    for (int i = 0; i < 255; ++i) {
        if (!(h_thr[i] == h_thr[i]) || (i && !(h_thr[i - 1] < h_thr[i])))
            return fail(RS_EINVAL, "thresholds must be ascending and not NaN (%d)", i);
        A.thr[i] = h_thr[i];
    }
    A.thr[255] = (T)NAN;
    A.has_lut = h_lut != nullptr;
    A.pad_ = 0;
    for (int i = 0; i < 256; ++i)
        A.lut[i] = h_lut ? (uint32_t)h_lut[3 * i] | ((uint32_t)h_lut[3 * i + 1] << 8) |
                               ((uint32_t)h_lut[3 * i + 2] << 16) | 0xff000000u
                         : 0u;
    if (!d_gray && !d_rgba) return RS_OK;
    preview_kernel<M, T><<<grid_cap(s * s, 256, 8), 256, 0, st>>>(d_map, npix, s, A, d_gray,
                                                                    d_rgba);
    return cuda_fail(cudaGetLastError(), "preview launch");
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" {

int rs_index_bits(int64_t distinct)
{
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) < distinct) ++b;
    return b;
}

int rs_index_encode(const int32_t* d_counts, int64_t n, int bits, int32_t* d_table,
                    int64_t table_cap, uint32_t* d_words, int64_t words_cap, rs_index_info* info,
                    void* stream)
{
    clear_error();
    if (!info) return fail(RS_EINVAL, "info is NULL");
    if (n < 1) return fail(RS_EINVAL, "empty map");
    if (bits < 0 || bits > 32) return fail(RS_EINVAL, "bits must be 0 (fewest) or 1..32");
    if (table_cap < 1 || words_cap < 1) return fail(RS_EINVAL, "no room for the table or map");
    int rc;
    if ((rc = check_device_ptr(d_counts, "d_counts")) || (rc = check_device_ptr(d_table, "d_table")) ||
        (rc = check_device_ptr(d_words, "d_words")))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: min/max, total, then chunk sums and flags (grown after max is known)
    struct Small { int mm[2]; long long total; };
    Small* d_small = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&d_small), sizeof(Small), s) != cudaSuccess) {
        cudaGetLastError();
        return fail(RS_ENOMEM, "scratch allocation failed");
    }
    int* d_flags = nullptr;
    unsigned* gbits = nullptr;
    int *wp = nullptr, *part = nullptr;
    Small h{};
    int64_t len = 0, nb = 0, need_words = 0, D = 0;
    int b = 0;
    minmax_init_kernel<<<1, 1, 0, s>>>(d_small->mm);
    minmax_kernel<<<grid_cap(n / 4 + 1, 256, 8), 256, 0, s>>>(d_counts, n, d_small->mm);
    if ((rc = cuda_fail(cudaGetLastError(), "min/max launch"))) goto done;
    if ((rc = cuda_fail(cudaMemcpyAsync(&h, d_small, sizeof(Small), cudaMemcpyDeviceToHost, s),
                        "min/max copy")) ||
        (rc = cuda_fail(cudaStreamSynchronize(s), "min/max sync")))
        goto done;
    if (h.mm[0] < 0) { rc = fail(RS_EINVAL, "negative count %d in the map", h.mm[0]); goto done; }
    // scratch: presence bitmap, per-word rank prefix, chunk sums
    len = ((int64_t)h.mm[1] >> 5) + 1;                  // bitmap words
    nb = (len + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (cudaMallocAsync(reinterpret_cast<void**>(&d_flags), (size_t)(2 * len + nb) * sizeof(int),
                        s) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(RS_ENOMEM, "bitmap allocation (%lld words) failed", (long long)len);
        goto done;
    }
    gbits = reinterpret_cast<unsigned*>(d_flags);
    wp = d_flags + len;
    part = d_flags + 2 * len;
    if ((rc = launch_fill_i32(d_flags, len, 0, s))) goto done;
    if (len * sizeof(unsigned) <= SMEM_BITMAP_BYTES)
        mark_kernel<true><<<grid_cap(n / 4 + 1, 256, 8), 256, len * sizeof(unsigned), s>>>(
            d_counts, n, h.mm[1], gbits);
    else
        mark_kernel<false><<<grid_cap(n / 4 + 1, 256, 8), 256, 0, s>>>(d_counts, n, h.mm[1], gbits);
    chunk_sum_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(gbits, len, part);
    part_scan_kernel<<<1, 1024, 0, s>>>(part, nb, &d_small->total);
    rank_kernel<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(gbits, len, part, wp, d_table, table_cap);
    if ((rc = cuda_fail(cudaGetLastError(), "index table launch"))) goto done;
    if ((rc = cuda_fail(cudaMemcpyAsync(&h, d_small, sizeof(Small), cudaMemcpyDeviceToHost, s),
                        "table size copy")) ||
        (rc = cuda_fail(cudaStreamSynchronize(s), "table size sync")))
        goto done;
    D = h.total;
    b = bits ? bits : rs_index_bits(D);
    need_words = (n * (int64_t)b + 31) / 32;
    info->distinct = D;
    info->bits = b;
    info->max_count = h.mm[1];
    info->words = need_words;
    if (D > table_cap) {
        rc = fail(RS_ERANGE, "%lld distinct counts, table holds %lld", (long long)D,
                  (long long)table_cap);
        goto done;
    }
    if (b < rs_index_bits(D)) {
        rc = fail(RS_ERANGE, "%lld distinct counts need %d bits, %d asked", (long long)D,
                  rs_index_bits(D), b);
        goto done;
    }
    if (need_words > words_cap) {
        rc = fail(RS_ERANGE, "packed map needs %lld words, room for %lld", (long long)need_words,
                  (long long)words_cap);
        goto done;
    }
    {
        const bool sr = h.mm[1] < PACK_SMEM_RANKS;
        const size_t dyn = sr ? (size_t)(h.mm[1] + 1) * sizeof(unsigned) : 0;
        const PackFn kern = sr ? kPackSmem[b - 1] : kPackGlobal[b - 1];
        if (sr && (rc = allow_dynamic_smem(reinterpret_cast<const void*>(kern), 0, b,
                                           (int)(PACK_SMEM_RANKS * sizeof(unsigned)))))
            goto done;
        int per_sm = 0;
        if ((rc = cuda_fail(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,
                                                                          32 * DEC_WARPS, dyn),
                            "pack occupancy")))
            goto done;
        kern<<<grid_cap((n + 1023) / 1024, DEC_WARPS, per_sm > 0 ? per_sm : 1), 32 * DEC_WARPS,
               dyn, s>>>(d_counts, n, gbits, wp, h.mm[1], d_words);
        rc = cuda_fail(cudaGetLastError(), "pack launch");
    }
done:
    if (d_flags) cudaFreeAsync(d_flags, s);
    cudaFreeAsync(d_small, s);
    return rc;
}

int rs_index_decode(const uint32_t* d_words, int64_t n, int bits, const int32_t* d_table,
                    int64_t distinct, int32_t* d_counts, void* stream)
{
    clear_error();
    if (n < 1) return fail(RS_EINVAL, "empty map");
    if (bits < 1 || bits > 32) return fail(RS_EINVAL, "bits must be in 1..32");
    if (distinct < 1) return fail(RS_EINVAL, "empty table");
    int rc;
    if ((rc = check_device_ptr(d_words, "d_words")) || (rc = check_device_ptr(d_table, "d_table")) ||
        (rc = check_device_ptr(d_counts, "d_counts")))
        return rc;
    const bool tab = distinct <= DEC_SMEM_TABLE;
    const size_t dyn = tab ? (size_t)distinct * sizeof(int32_t) : 0;
    const UnpackFn kern = tab ? kUnpackSmem[bits - 1] : kUnpackGlobal[bits - 1];
    if (tab && (rc = allow_dynamic_smem(reinterpret_cast<const void*>(kern), 1, bits,
                                        (int)(DEC_SMEM_TABLE * sizeof(int32_t)))))
        return rc;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * DEC_WARPS, dyn);
    if (e != cudaSuccess) return cuda_fail(e, "unpack occupancy");
    kern<<<grid_cap((n + 1023) / 1024, DEC_WARPS, per_sm > 0 ? per_sm : 1), 32 * DEC_WARPS, dyn,
           (cudaStream_t)stream>>>(d_words, n, d_table, distinct, d_counts);
    return cuda_fail(cudaGetLastError(), "unpack launch");
}

int rs_colorbar_lut(const int32_t* pos, const uint8_t* rgb, int m, uint8_t* lut)
{
    clear_error();
    return build_lut(pos, rgb, m, lut);
}

int rs_preview_counts(const int32_t* d_counts, int64_t npix, int64_t s, const double* h_thr,
                      const uint8_t* h_lut, uint8_t* d_gray, uint32_t* d_rgba, void* stream)
{
    clear_error();
    // int32 counts are exact in double, so the comparisons are exact
    return preview<int32_t, double>(d_counts, npix, s, h_thr, h_lut, d_gray, d_rgba,
                                    (cudaStream_t)stream);
}

int rs_preview_f32(const float* d_map, int64_t npix, int64_t s, const float* h_thr,
                   const uint8_t* h_lut, uint8_t* d_gray, uint32_t* d_rgba, void* stream)
{
    clear_error();
    return preview<float, float>(d_map, npix, s, h_thr, h_lut, d_gray, d_rgba,
                                 (cudaStream_t)stream);
}

int rs_colorize(const uint8_t* d_gray, int64_t m, const uint8_t* h_lut, uint32_t* d_rgba,
                void* stream)
{
    clear_error();
    if (m < 0 || !h_lut) return fail(RS_EINVAL, "bad size or NULL table");
    if (m == 0) return RS_OK;
    int rc;
    if ((rc = check_device_ptr(d_gray, "d_gray")) || (rc = check_device_ptr(d_rgba, "d_rgba")))
        return rc;
    PreviewArgs<float> A;
    for (int i = 0; i < 256; ++i) {
        A.thr[i] = 0.f;
        A.lut[i] = (uint32_t)h_lut[3 * i] | ((uint32_t)h_lut[3 * i + 1] << 8) |
                   ((uint32_t)h_lut[3 * i + 2] << 16) | 0xff000000u;
    }
    A.has_lut = 1;
    A.pad_ = 0;
    colorize_kernel<<<grid_cap(m, 256, 8), 256, 0, (cudaStream_t)stream>>>(d_gray, m, A, d_rgba);
    return cuda_fail(cudaGetLastError(), "colorize launch");
}

}  // extern "C"
