// Stockham autosort FFT in FP32 (float2) or FP64 (double2), shared by the
// transfer-function correction and the FFT route of the convolution C: one
// launch per radix pass
// (radices 4, 2 and every prime up to kMaxRadix, each pass a generic radix-R
// butterfly with twiddles from a per-length table), batched over the y
// dimension of the launch.
#pragma once

#include <vector>

#include "common.cuh"

namespace mpi {

constexpr int kMaxRadix = 127;
constexpr int kFftThreads = 256;

struct FftPlan {
    int64_t n = 0;
    std::vector<int> radix;  // product = n
};

// Factor n into radices; false when n has a prime factor above kMaxRadix.
bool plan_fft(int64_t n, FftPlan &p);
unsigned fft_blocks(int64_t n);
// W[m] = exp(-2 pi i m / n), m < n (device table, formed in FP64).
int fft_twiddles(int64_t n, double2 *W, cudaStream_t st);
int fft_twiddles(int64_t n, float2 *W, cudaStream_t st);
// Forward DFT of n_ch sequences of length p.n at distance `dist`: the
// transform of `a` ends in `a` (`b` is scratch of the same size).
int fft_run(const FftPlan &p, double2 *a, double2 *b, int n_ch, int64_t dist, const double2 *W,
            cudaStream_t st);
int fft_run(const FftPlan &p, float2 *a, float2 *b, int n_ch, int64_t dist, const float2 *W,
            cudaStream_t st);

// The complex type of a real type.
template <typename T> struct CxOf;
template <> struct CxOf<float> { using type = float2; };
template <> struct CxOf<double> { using type = double2; };

#ifdef __CUDACC__
// Complex value from FP64 parts, rounded to C (set-up and loads).
template <typename C>
__host__ __device__ __forceinline__ C make_cx(double re, double im);
template <>
__host__ __device__ __forceinline__ float2 make_cx<float2>(double re, double im)
{
    return make_float2(float(re), float(im));
}
template <>
__host__ __device__ __forceinline__ double2 make_cx<double2>(double re, double im)
{
    return make_double2(re, im);
}
// Complex value in the precision of its parts (no conversion).
__host__ __device__ __forceinline__ float2 cxv(float re, float im) { return make_float2(re, im); }
__host__ __device__ __forceinline__ double2 cxv(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
#endif

}  // namespace mpi
