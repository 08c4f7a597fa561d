// rs_mpd.cu -- magnification probability distribution and probability sums.
//
// MPD (Sec. 3.2.1, the map's mpd.dat): the frequency of every magnification
// value of a map divided by the number of pixels.  A map's magnification
// values are its ray counts over N_avg (Eq. 4), so the MPD is the exact
// histogram of the int32 count map: integer work, bit-exact.  The kernel
// reads the count map once, writes mu (Eq. 4) on the way when asked, and
// histograms the counts: counts below SBINS in a shared-memory histogram
// per CTA (flushed with one global atomic per non-empty bin), larger ones
// straight into the global histogram.  HBM-bound: 4 B/pixel read, +4 B/pixel
// written with mu.
//
// Probability sums (Sec. 4.4, MPDs tool): pixels with mu < mu_lim and with
// mu > mu_lim, from the histogram; mu = c / N_avg is compared in FP64 as
// c < mu_lim * N_avg, the threshold computed on the host.
#include <cuda_runtime.h>
#include <math.h>

#include "rs_internal.cuh"

namespace rs {
namespace {

constexpr int SBINS = 8192;      // count values histogrammed in shared memory
constexpr int MAX_LIM = 16;      // thresholds per probability-sum call

struct LimArgs {
    int32_t n;
    int32_t pad_;
    double thr[MAX_LIM];
};

__device__ __forceinline__ void count_one(int32_t c, unsigned* sh, int64_t sbins,
                                          unsigned long long* hist, int64_t n_bins)
{
    const int64_t v = c < 0 ? 0 : c;   // counts are never negative
    if (v < sbins) {
        atomicAdd(sh + v, 1u);
    } else {
        atomicAdd(hist + (v < n_bins - 1 ? v : n_bins - 1), 1ull);
    }
}

__global__ void __launch_bounds__(256) mpd_kernel(const int32_t* __restrict__ counts, int64_t n,
                                                  float inv_navg, float* __restrict__ mu,
                                                  unsigned long long* __restrict__ hist,
                                                  int64_t n_bins)
{
    __shared__ unsigned sh[SBINS];
    // shared bins hold counts 0 .. sbins-1, never the overflow bin
    const int64_t sbins = n_bins - 1 < SBINS ? n_bins - 1 : SBINS;
    for (int b = threadIdx.x; b < SBINS; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool al = ((reinterpret_cast<uintptr_t>(counts) |
                      (mu ? reinterpret_cast<uintptr_t>(mu) : 0)) & 15) == 0;
    const int64_t n4 = al ? n / 4 : 0;
    const int4* c4 = reinterpret_cast<const int4*>(counts);
    float4* m4 = reinterpret_cast<float4*>(mu);
    // four 16-byte loads in flight per thread, then stores and counting
    constexpr int U = 4;
    int64_t k = t0;
    for (; k + (U - 1) * stride < n4; k += U * stride) {
        int4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = __ldcs(c4 + k + u * stride);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (mu)
                __stcs(m4 + k + u * stride,
                       make_float4((float)q[u].x * inv_navg, (float)q[u].y * inv_navg,
                                   (float)q[u].z * inv_navg, (float)q[u].w * inv_navg));
            count_one(q[u].x, sh, sbins, hist, n_bins);
            count_one(q[u].y, sh, sbins, hist, n_bins);
            count_one(q[u].z, sh, sbins, hist, n_bins);
            count_one(q[u].w, sh, sbins, hist, n_bins);
        }
    }
    for (; k < n4; k += stride) {
        const int4 q = __ldcs(c4 + k);
        if (mu)
            __stcs(m4 + k, make_float4((float)q.x * inv_navg, (float)q.y * inv_navg,
                                       (float)q.z * inv_navg, (float)q.w * inv_navg));
        count_one(q.x, sh, sbins, hist, n_bins);
        count_one(q.y, sh, sbins, hist, n_bins);
        count_one(q.z, sh, sbins, hist, n_bins);
        count_one(q.w, sh, sbins, hist, n_bins);
    }
    for (int64_t j = 4 * n4 + t0; j < n; j += stride) {
        const int32_t c = counts[j];
        if (mu) mu[j] = (float)c * inv_navg;
        count_one(c, sh, sbins, hist, n_bins);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < sbins; b += blockDim.x)
        if (sh[b]) atomicAdd(hist + b, (unsigned long long)sh[b]);
}

// One CTA: for every threshold, the pixels below and above it.
__global__ void __launch_bounds__(1024) prob_sums_kernel(const long long* __restrict__ hist,
                                                         int64_t n_bins,
                                                         const __grid_constant__ LimArgs L,
                                                         long long* __restrict__ below,
                                                         long long* __restrict__ above)
{
    __shared__ long long red[2][32];
    for (int k = 0; k < L.n; ++k) {
        const double thr = L.thr[k];
        long long lo = 0, hi = 0;
        for (int64_t c = threadIdx.x; c < n_bins; c += blockDim.x) {
            const long long h = hist[c];
            if ((double)c < thr) lo += h;
            else if ((double)c > thr) hi += h;
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo += __shfl_down_sync(0xffffffffu, lo, o);
            hi += __shfl_down_sync(0xffffffffu, hi, o);
        }
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = lo;
            red[1][threadIdx.x >> 5] = hi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long a = 0, b = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                a += red[0][w];
                b += red[1][w];
            }
            below[k] = a;
            above[k] = b;
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" {

int rs_mpd(const int32_t* d_counts, const rs_raygrid* grid, const rs_mapspec* map, float* d_mu,
           int64_t* d_hist, int64_t n_bins, void* stream)
{
    clear_error();
    double navg = 0.0;
    int rc = rs_navg(grid, map, &navg);
    if (rc) return rc;
    if (n_bins < 2 || n_bins > (int64_t)1 << 31)
        return fail(RS_ERANGE, "n_bins = %lld outside [2, 2^31]", (long long)n_bins);
    if ((rc = check_device_ptr(d_counts, "d_counts")) || (rc = check_device_ptr(d_hist, "d_hist")) ||
        (d_mu && (rc = check_device_ptr(d_mu, "d_mu"))))
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = launch_fill_i64(d_hist, n_bins, 0, s))) return rc;
    const int64_t n = map->npix * map->npix;
    int64_t want = (n / 4 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 4;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    mpd_kernel<<<(int)want, 256, 0, s>>>(d_counts, n, (float)(1.0 / navg), d_mu,
                                         reinterpret_cast<unsigned long long*>(d_hist), n_bins);
    return cuda_fail(cudaGetLastError(), "mpd kernel launch");
}

int rs_prob_sums(const int64_t* d_hist, int64_t n_bins, const rs_raygrid* grid,
                 const rs_mapspec* map, const double* h_mu_lim, int n_lim, int64_t* d_below,
                 int64_t* d_above, void* stream)
{
    clear_error();
    double navg = 0.0;
    int rc = rs_navg(grid, map, &navg);
    if (rc) return rc;
    if (n_lim < 1 || n_lim > MAX_LIM || !h_mu_lim)
        return fail(RS_EINVAL, "n_lim must be in 1..%d with mu_lim given", MAX_LIM);
    if (n_bins < 2) return fail(RS_EINVAL, "n_bins < 2");
    LimArgs L;
    L.n = n_lim;
    L.pad_ = 0;
    for (int k = 0; k < n_lim; ++k) {
        const double thr = h_mu_lim[k] * navg;
        if (!(thr < (double)(n_bins - 1)))
            return fail(RS_ERANGE, "mu_lim[%d] * N_avg = %g reaches the overflow bin %lld", k,
                        thr, (long long)(n_bins - 1));
        L.thr[k] = thr;
    }
    for (int k = n_lim; k < MAX_LIM; ++k) L.thr[k] = 0.0;
    if ((rc = check_device_ptr(d_hist, "d_hist")) || (rc = check_device_ptr(d_below, "d_below")) ||
        (rc = check_device_ptr(d_above, "d_above")))
        return rc;
    prob_sums_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const long long*>(d_hist), n_bins, L,
        reinterpret_cast<long long*>(d_below), reinterpret_cast<long long*>(d_above));
    return cuda_fail(cudaGetLastError(), "probability sums launch");
}

}  // extern "C"
