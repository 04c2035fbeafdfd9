// Shared host/device helpers of the sm_103a MPI reconstruction library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "mpi_recon.h"

namespace mpi {

// ---------------------------------------------------------------------------
// Error reporting (host).  Every entry point returns an mpi_status; the
// reason of the last failure on this host thread is kept for
// mpi_last_error_message().
void set_error(const char *fmt, ...);
const char *last_error();

#define MPI_TRY_CUDA(expr)                                                        \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            ::mpi::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                             __FILE__, __LINE__);                                 \
            return MPI_ERR_CUDA;                                                  \
        }                                                                         \
    } while (0)

#define MPI_TRY(expr)                        \
    do {                                     \
        int st_ = (expr);                    \
        if (st_ != MPI_OK) return st_;       \
    } while (0)

// Every kernel launch of the library is followed by MPI_CHECK_LAUNCH(), which
// also counts it (mpi_kernel_launches()).
void note_launch();
void note_launches(long long n);
#define MPI_CHECK_LAUNCH()                          \
    do {                                            \
        ::mpi::note_launch();                       \
        MPI_TRY_CUDA(cudaGetLastError());           \
    } while (0)

// Optional event timing of the operator kernels (mpi_profile_enable): when
// enabled, a ProfScope records a CUDA event pair around its launch on the
// launching stream.
enum ProfClass { kProfForward = 0, kProfAdjoint = 1, kProfDbeta = 2, kProfConv = 3, kProfClasses = 4 };
class ProfScope {
  public:
    ProfScope(int cls, cudaStream_t st);
    ~ProfScope();

  private:
    int cls_;
    cudaStream_t st_;
    cudaEvent_t ev_[2];
    bool on_;
};

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Stream-ordered scratch: one cudaMallocAsync carved into aligned pieces, freed
// (stream-ordered) when the object goes out of scope.
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : stream_(s) {}
    ~Scratch() { release(); }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    // Reserve `bytes` (rounded up to 256) and return its offset.
    size_t reserve(size_t bytes) {
        size_t off = total_;
        total_ += (bytes + 255) & ~size_t(255);
        return off;
    }
    int allocate();
    template <typename T>
    T *at(size_t off) const { return reinterpret_cast<T *>(base_ + off); }
    void release();
    size_t total() const { return total_; }

  private:
    cudaStream_t stream_;
    char *base_ = nullptr;
    size_t total_ = 0;
};

int device_sm_count();

// ---------------------------------------------------------------------------
// Device helpers.

template <typename R> struct V2 { R x, y; };
template <typename R> struct V4 { R x, y, z, w; };
template <> struct alignas(8) V2<float> { float x, y; };
template <> struct alignas(16) V4<float> { float x, y, z, w; };
template <> struct alignas(16) V2<double> { double x, y; };
template <> struct alignas(16) V4<double> { double x, y, z, w; };

#ifdef __CUDACC__
// PTX approximate transcendental instructions (flush-to-zero forms).  Their
// errors are a few units in the last place of FP32; the callers' accuracy
// budget is derived with them in place.
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Fused multiply-add with the product fixed by the call (never left to the
// compiler's contraction choice), so every kernel instantiation rounds alike.
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }

// Compensated (Kahan) accumulation: sum += x with running compensation.
template <typename R>
__device__ __forceinline__ void kahan_add(R &sum, R &comp, R x)
{
    R y = x - comp;
    R t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Sum of FP32 values carried as the unevaluated pair hi + lo.  Every addition
// is Knuth's error-free TwoSum (six FP32 operations: hi + x = t + err
// exactly), the rounding errors collect in lo, so the pair holds the sum to
// about 2^-48 relative -- the accuracy of an FP64 accumulator -- while all
// the work stays on the FP32 pipe.  (GB300 executes FP64 arithmetic and the
// FP32 -> FP64 conversion at a small fraction of the FP32 rate, so summing
// millions of FP32 partials in FP64 is bound by the FP64 pipe.)  The
// explicit _rn intrinsics keep the compiler from contracting or reordering
// the transformation.
struct F2Sum {
    float hi, lo;  // value-initialise (F2Sum{}) to start at zero
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(hi, x);
        const float bp = __fsub_rn(t, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        hi = t;
        lo = __fadd_rn(lo, err);
    }
    __device__ __forceinline__ void add(const F2Sum &o)
    {
        add(o.hi);
        lo = __fadd_rn(lo, o.lo);
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

// Accumulator of a fixed-order sum of R values: the pair above for FP32
// inputs, a plain FP64 sum for FP64 inputs.  Aggregates (usable in shared
// memory): value-initialise, SumAcc<R>{}, to start at zero.
template <typename R> struct SumAcc;
template <> struct SumAcc<float> {
    F2Sum s;
    __device__ __forceinline__ void add(float x) { s.add(x); }
    __device__ __forceinline__ void add(const SumAcc &o) { s.add(o.s); }
    __device__ __forceinline__ double value() const { return s.value(); }
};
template <> struct SumAcc<double> {
    double s;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void add(const SumAcc &o) { s += o.s; }
    __device__ __forceinline__ double value() const { return s; }
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed shuffle tree, then warps in order).  All
// threads of the block must call it; the result is valid in thread 0.
template <typename R, int NT>
__device__ __forceinline__ R block_sum(R v, R *sh /* >= NT/32 */)
{
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    R t = R(0);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t += sh[w];
    }
    __syncthreads();
    return t;
}
#endif

}  // namespace mpi
