// rs_fields.cu -- lens-field generation and element-wise map kernels.
//
//   * make_lenses: lenses uniform in a disk of area A = pi R^2 (Fig. 1
//     caption) with unit or Salpeter masses (Sec. 2.5 item 2), normalised to
//     unit mean so that Eq. 3 holds with <M> = 1.  Random numbers come from
//     SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based
//     generator: lens k takes outputs 3k, 3k+1, 3k+2 of the seed, so the
//     field does not depend on the launch shape.
//   * fill: zeroing of the count map and the statistics.
//   * magnification: Eq. 4, mu = N_ij / N_avg, an HBM-bound int32 -> f32
//     pass with 16-byte loads and stores.
#include <cuda_runtime.h>
#include <math.h>

#include "rs_internal.cuh"

namespace rs {
namespace {

// top 53 bits -> [0, 1)
__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long k)
{
    return (double)(splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void make_lenses_kernel(double radius, int model, double a, double b, double e,
                                   unsigned long long seed, double* __restrict__ x1,
                                   double* __restrict__ x2, double* __restrict__ m, int64_t n)
{
    const double two_pi = 6.28318530717958647692;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long kk = 3ull * (unsigned long long)k;
        const double r = __dmul_rn(radius, sqrt(u01(seed, kk)));
        const double phi = __dmul_rn(two_pi, u01(seed, kk + 1));
        double s, c;
        sincos(phi, &s, &c);
        x1[k] = __dmul_rn(r, c);
        x2[k] = __dmul_rn(r, s);
        if (model == RS_MASS_UNIT) {
            m[k] = 1.0;
        } else {
            // inverse CDF of dN/dm ~ m^-slope between a = m_lo^e, b = m_hi^e
            const double u = u01(seed, kk + 2);
            m[k] = pow(__dadd_rn(a, __dmul_rn(u, __dsub_rn(b, a))), 1.0 / e);
        }
    }
}

// One CTA: sum the masses in a fixed order (strided partial sums, then a
// fixed tree), divide every mass by the mean.  Deterministic for a given n.
__global__ void __launch_bounds__(1024) normalise_masses_kernel(double* __restrict__ m, int64_t n)
{
    __shared__ double part[1024];
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s = __dadd_rn(s, m[k]);
    part[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + h]);
        __syncthreads();
    }
    const double mean = __ddiv_rn(part[0], (double)n);
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) m[k] = __ddiv_rn(m[k], mean);
}

__global__ void fill_i32_kernel(int32_t* __restrict__ p, int64_t n, int32_t v)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n4 = ((reinterpret_cast<uintptr_t>(p) & 15) == 0) ? n / 4 : 0;
    int4* p4 = reinterpret_cast<int4*>(p);
    const int4 v4 = make_int4(v, v, v, v);
    for (int64_t k = t0; k < n4; k += stride) p4[k] = v4;
    for (int64_t k = 4 * n4 + t0; k < n; k += stride) p[k] = v;
}

__global__ void fill_i64_kernel(int64_t* __restrict__ p, int64_t n, int64_t v)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        p[k] = v;
}

__global__ void magnification_kernel(const int32_t* __restrict__ c, int64_t n, float inv_navg,
                                     float* __restrict__ mu)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool al = ((reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(mu)) & 15) == 0;
    const int64_t n4 = al ? n / 4 : 0;
    const int4* c4 = reinterpret_cast<const int4*>(c);
    float4* m4 = reinterpret_cast<float4*>(mu);
    // four 16-byte loads in flight per thread before the stores
    constexpr int U = 4;
    int64_t k = t0;
    for (; k + (U - 1) * stride < n4; k += U * stride) {
        int4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = __ldcs(c4 + k + u * stride);
#pragma unroll
        for (int u = 0; u < U; ++u)
            __stcs(m4 + k + u * stride,
                   make_float4((float)q[u].x * inv_navg, (float)q[u].y * inv_navg,
                               (float)q[u].z * inv_navg, (float)q[u].w * inv_navg));
    }
    for (; k < n4; k += stride) {
        const int4 q = __ldcs(c4 + k);
        __stcs(m4 + k, make_float4((float)q.x * inv_navg, (float)q.y * inv_navg,
                                   (float)q.z * inv_navg, (float)q.w * inv_navg));
    }
    for (int64_t j = 4 * n4 + t0; j < n; j += stride) mu[j] = (float)c[j] * inv_navg;
}

int grid_for(int64_t work, int per_thread, int threads)
{
    int64_t need = (work / per_thread + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 8;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

}  // namespace

int launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s)
{
    if (n <= 0) return RS_OK;
    fill_i32_kernel<<<grid_for(n, 4, 256), 256, 0, s>>>(p, n, v);
    return cuda_fail(cudaGetLastError(), "fill kernel launch");
}

int launch_fill_i64(int64_t* p, int64_t n, int64_t v, cudaStream_t s)
{
    if (n <= 0) return RS_OK;
    fill_i64_kernel<<<grid_for(n, 1, 256), 256, 0, s>>>(p, n, v);
    return cuda_fail(cudaGetLastError(), "fill kernel launch");
}

int launch_magnification(const int32_t* counts, int64_t n, float inv_navg, float* mu,
                         cudaStream_t s)
{
    if (n <= 0) return RS_OK;
    magnification_kernel<<<grid_for(n, 4, 256), 256, 0, s>>>(counts, n, inv_navg, mu);
    return cuda_fail(cudaGetLastError(), "magnification kernel launch");
}

int launch_make_lenses(const rs_lensfield* f, uint64_t seed, double* d_lens, int64_t n,
                       cudaStream_t s)
{
    if (n <= 0) return RS_OK;
    double a = 0.0, b = 0.0, e = 1.0;
    if (f->mass_model == RS_MASS_SALPETER) {
        e = 1.0 - f->slope;
        a = pow(f->m_lo, e);
        b = pow(f->m_hi, e);
    }
    make_lenses_kernel<<<grid_for(n, 1, 256), 256, 0, s>>>(
        f->radius, f->mass_model, a, b, e, (unsigned long long)seed, d_lens, d_lens + n,
        d_lens + 2 * n, n);
    int rc = cuda_fail(cudaGetLastError(), "lens kernel launch");
    if (rc) return rc;
    if (f->mass_model == RS_MASS_SALPETER) {
        normalise_masses_kernel<<<1, 1024, 0, s>>>(d_lens + 2 * n, n);
        rc = cuda_fail(cudaGetLastError(), "mass normalisation launch");
    }
    return rc;
}

}  // namespace rs
