// Device building blocks shared by the single-frame and the batched PnP
// solves: fixed-order sums of partials, the radix-select order statistic, the
// percentile/variance block and the 5-tap Gaussian tile.
#pragma once

#include <cmath>

#include "pnp_ops.cuh"

namespace mpi {

constexpr int kVecThreads = 256;
// Elements per block of the CG vector kernels (and so the number of partial
// sums of r.r): small enough that a 128 x 128 problem spreads over 32 blocks.
constexpr int kVecPerBlock = 512;
constexpr int kStatThreads = 1024;
// Values per iteration in a solve's device record (mpi_pnp_iter_info).
constexpr int kInfoCols = 4;

// Sum of `n` partials in a fixed order, computed by the whole block and
// returned to every thread (deterministic: fixed strides, fixed tree).
template <int NT>
__device__ double sum_parts(const double *__restrict__ part, int n, double *sh /* NT/32 + 1 */)
{
    double a = 0.0;
    for (int k = threadIdx.x; k < n; k += NT) a += part[k];
    a = block_sum<double, NT>(a, sh);
    if (threadIdx.x == 0) sh[NT / 32] = a;
    __syncthreads();
    const double r = sh[NT / 32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Percentile trimming and noise estimate (Sec. 3.3 and the noise estimator of
// Algorithm 1): exact order statistics by an 8-pass radix select on the
// order-preserving integer image of the FP64 values.

__device__ __forceinline__ uint64_t f64_key(double v)
{
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_f64(uint64_t k)
{
    const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

template <int NT>
__device__ double block_select(const double *__restrict__ x, int64_t N, int64_t rank,
                               unsigned *hist, unsigned long long *sh_u)
{
    uint64_t prefix = 0, mask = 0;
    int64_t krem = rank;
    const int lane = threadIdx.x & 31;
    for (int shift = 56; shift >= 0; shift -= 8) {
        for (int b = threadIdx.x; b < 256; b += NT) hist[b] = 0;
        __syncthreads();
        for (int64_t i0 = 0; i0 < N; i0 += NT) {
            const int64_t i = i0 + threadIdx.x;
            unsigned digit = 256;  // no bin
            if (i < N) {
                const uint64_t key = f64_key(x[i]);
                if ((key & mask) == prefix) digit = (unsigned)((key >> shift) & 255u);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, digit);
            if (digit < 256 && lane == __ffs(peers) - 1) atomicAdd(&hist[digit], (unsigned)__popc(peers));
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t cum = 0;
            unsigned d = 0;
            for (; d < 255; ++d) {
                if (cum + hist[d] > krem) break;
                cum += hist[d];
            }
            krem -= cum;
            sh_u[0] = prefix | ((uint64_t)d << shift);
            sh_u[1] = (unsigned long long)krem;
        }
        __syncthreads();
        prefix = sh_u[0];
        krem = (int64_t)sh_u[1];
        mask |= (uint64_t)255 << shift;
        __syncthreads();
    }
    return key_f64(prefix);
}

// Minimum over the block (order-independent), returned to every thread.
template <int NT>
__device__ __forceinline__ double block_min(double v, double *sh /* >= NT/32 + 1 */)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();  // sh may still be read by an earlier reduction
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = sh[0];
        for (int w = 1; w < NT / 32; ++w) m = fmin(m, sh[w]);
        sh[NT / 32] = m;
    }
    __syncthreads();
    const double r = sh[NT / 32];
    __syncthreads();
    return r;
}

// One block computes, for the N values x: the clip value P (the pct-th
// percentile, linear interpolation between order statistics; -inf when
// do_clip is 0), rho1 = max(x, P) rounded to R, the population variance of
// rho1 in two FP64 passes, and updates the PnP scalars: sigma, lambda = nu0
// sigma^2 on the first iteration, nu = lambda / sigma^2 (kept if sigma = 0).
// rr_part/nblk: partial sums of the final CG residual for info_row (sigma,
// nu, residual norm, clip value: kInfoCols values).
template <typename R>
__device__ void outer_stats_block(int64_t N, const double *__restrict__ x, int do_clip, double pct,
                                  bool first, double nu0, double *__restrict__ scal,
                                  const double *__restrict__ rr_part, int nblk,
                                  double *__restrict__ info_row, R *__restrict__ rho1)
{
    __shared__ unsigned hist[256];
    __shared__ unsigned long long sh_u[2];
    __shared__ double sh[kStatThreads / 32 + 1];
    double P = -INFINITY;
    if (do_clip) {
        const double h = double(N - 1) * pct / 100.0;
        const int64_t lo = (int64_t)floor(h);
        const int64_t hi = min(lo + 1, N - 1);
        const double xlo = block_select<kStatThreads>(x, N, lo, hist, sh_u);
        // The next order statistic in one pass instead of a second select:
        // x(lo + 1) is xlo itself when more than lo + 1 values are <= xlo,
        // else the smallest value above xlo (exact, order-independent).
        double xhi = xlo;
        if (hi != lo) {
            int64_t le = 0;
            double gt = INFINITY;
            for (int64_t i = threadIdx.x; i < N; i += kStatThreads) {
                const double v = x[i];
                if (v <= xlo) ++le;
                else gt = fmin(gt, v);
            }
            le = block_sum<int64_t, kStatThreads>(le, reinterpret_cast<int64_t *>(sh));
            if (threadIdx.x == 0) sh_u[0] = (unsigned long long)le;
            __syncthreads();
            le = (int64_t)sh_u[0];
            __syncthreads();
            gt = block_min<kStatThreads>(gt, sh);
            xhi = le > hi ? xlo : gt;
        }
        P = xlo + (h - double(lo)) * (xhi - xlo);
    }
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += kStatThreads) {
        const double v = fmax(x[i], P);
        rho1[i] = R(v);
        s += v;
    }
    s = block_sum<double, kStatThreads>(s, sh);
    if (threadIdx.x == 0) sh[kStatThreads / 32] = s;
    __syncthreads();
    const double mean = sh[kStatThreads / 32] / double(N);
    __syncthreads();
    double q = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += kStatThreads) {
        const double dv = fmax(x[i], P) - mean;
        q += dv * dv;
    }
    q = block_sum<double, kStatThreads>(q, sh);
    if (threadIdx.x == 0) {
        double rr = 0.0;
        for (int b = 0; b < nblk; ++b) rr += rr_part[b];
        const double sigma = sqrt(q / double(N));
        if (first) scal[kScalLambda] = nu0 * sigma * sigma;
        if (sigma > 0.0) scal[kScalNu] = scal[kScalLambda] / (sigma * sigma);
        scal[kScalSigma] = sigma;
        scal[kScalPct] = P;
        if (info_row) {
            info_row[0] = sigma;
            info_row[1] = scal[kScalNu];
            info_row[2] = sqrt(rr);
            info_row[3] = P;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Built-in denoiser: separable 5-tap Gaussian (sigma = 1 px), reflect
// boundary (d c b a | a b c d).

__device__ __forceinline__ int reflect_index(int i, int n)
{
    const int p = 2 * n;
    i %= p;
    if (i < 0) i += p;
    return i >= n ? p - 1 - i : i;
}

constexpr int kGx = 32, kGy = 8;

// One 32 x 8 output tile of the separable 5-tap Gaussian (rows first, then
// columns; reflect boundary) for tile origin (i0, j0).
template <typename R>
__device__ void gauss5_tile(const R *__restrict__ in, R *__restrict__ out, int nx, int ny, int i0,
                            int j0, R w0, R w1, R w2)
{
    __shared__ R tmp[kGy + 4][kGx];
    const R w[5] = {w2, w1, w0, w1, w2};
    const int tx = threadIdx.x % kGx, ty = threadIdx.x / kGx;
    const int i = i0 + tx;
    const int ic = min(i, nx - 1);
    for (int rr = ty; rr < kGy + 4; rr += kGy) {
        const int jr = reflect_index(j0 - 2 + rr, ny);
        const R *row = in + (int64_t)jr * nx;
        R acc = R(0);
#pragma unroll
        for (int m = -2; m <= 2; ++m) acc += w[m + 2] * row[reflect_index(ic + m, nx)];
        tmp[rr][tx] = acc;
    }
    __syncthreads();
    const int j = j0 + ty;
    if (i < nx && j < ny) {
        R acc = R(0);
#pragma unroll
        for (int m = -2; m <= 2; ++m) acc += w[m + 2] * tmp[reflect_index(j + m, ny) - (j0 - 2)][tx];
        out[(int64_t)j * nx + i] = acc;
    }
}

// 5-tap Gaussian weights exp(-m^2/2)/sum for m = 0, 1, 2.
inline void gauss5_weights(double w[3])
{
    double tot = 0.0;
    for (int m = -2; m <= 2; ++m) tot += std::exp(-0.5 * m * m);
    for (int m = 0; m <= 2; ++m) w[m] = std::exp(-0.5 * m * m) / tot;
}

}  // namespace mpi
