// Pipe-rate probe: the measured throughput of the instruction kinds the pair
// kernels are made of (FP32 FMA, and the MUFU/XU operations rsqrt.approx,
// ex2.approx, rcp.approx; FP64 FMA for the all-FP64 form; the packed
// two-lane FP32 FMA fma.rn.f32x2 of sm_100 and later, counted as two
// operations), in thread-operations per SM per clock.  The pair
// kernels' roofline is an issue/pipe bound, so its denominator is taken from
// this measurement on the GPU that runs them rather than from a datasheet.
//
// Every thread runs kProbeChains independent dependency chains of one
// operation (enough independent work to hide the pipe latency at full
// occupancy), so the SM's pipe, not a chain's latency, sets the rate.  Each
// block records its SM id and the SM clock (clock64) at entry and exit; the
// rate of an SM is its blocks' operations over the span from the earliest
// entry to the latest exit of its blocks, in SM clock cycles, so the result
// does not depend on the clock frequency the GPU happens to run at.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace mpi {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

template <int OP> struct ProbeType { using T = float; };
template <> struct ProbeType<MPI_PROBE_DFMA> { using T = double; };
template <> struct ProbeType<MPI_PROBE_FMA2> { using T = unsigned long long; };  // two packed f32

template <typename T> __device__ __forceinline__ T probe_init(float v) { return T(v); }
template <> __device__ __forceinline__ unsigned long long probe_init<unsigned long long>(float v)
{
    const unsigned b = __float_as_uint(v);
    return (unsigned long long)b | ((unsigned long long)b << 32);
}
template <typename T> __device__ __forceinline__ float probe_value(T v) { return float(v); }
template <> __device__ __forceinline__ float probe_value<unsigned long long>(unsigned long long v)
{
    return __uint_as_float((unsigned)v) + __uint_as_float((unsigned)(v >> 32));
}

// Every timed operation is a volatile asm statement: the compiler keeps them
// all, in program order relative to the (volatile) clock reads around the
// loop, so none is hoisted out of or sunk below the timed span.
template <int OP>
__device__ __forceinline__ typename ProbeType<OP>::T probe_op(typename ProbeType<OP>::T x)
{
    typename ProbeType<OP>::T y;
    if constexpr (OP == MPI_PROBE_FMA)
        asm volatile("fma.rn.f32 %0, %1, 0f3F7FC000, 0f3A800000;" : "=f"(y) : "f"(x));
    else if constexpr (OP == MPI_PROBE_FMA2)  // both lanes: x <- x 0.99902 + 2^-10
        asm volatile("fma.rn.f32x2 %0, %1, %2, %3;"
                     : "=l"(y)
                     : "l"(x), "l"(0x3F7FC0003F7FC000ull), "l"(0x3A8000003A800000ull));
    else if constexpr (OP == MPI_PROBE_DFMA)
        asm volatile("fma.rn.f64 %0, %1, 0d3FEFF80000000000, 0d3F50000000000000;" : "=d"(y) : "d"(x));
    else if constexpr (OP == MPI_PROBE_RSQRT)
        asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    else if constexpr (OP == MPI_PROBE_EX2)
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));  // stays in (0, 1]
    else  // x <- 1/(x + 1): an add keeps the assembler from folding rcp(rcp(x))
        asm volatile("{ .reg .f32 t; add.ftz.f32 t, %1, 0f3F800000; rcp.approx.ftz.f32 %0, t; }"
                     : "=f"(y) : "f"(x));
    return y;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads)
k_pipe_probe(int iters, float *__restrict__ sink, long long *__restrict__ rec)
{
    __shared__ unsigned long long s_t0, s_t1;
    if (threadIdx.x == 0) {
        s_t0 = ~0ull;
        s_t1 = 0ull;
    }
    __syncthreads();
    using T = typename ProbeType<OP>::T;
    T x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = probe_init<T>(0.5f + 0.001f * float((threadIdx.x + 37 * k) & 255));
    const unsigned long long t0 = (unsigned long long)clock64();
    // unrolled so that loop control is a few percent of the issued
    // instructions (FP32 FMA is issue-bound, and counts them)
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) x[k] = probe_op<OP>(x[k]);
    }
    const unsigned long long t1 = (unsigned long long)clock64();
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) acc += probe_value<T>(x[k]);
    sink[(int64_t)blockIdx.x * kProbeThreads + threadIdx.x] = acc;
    atomicMin(&s_t0, t0);
    atomicMax(&s_t1, t1);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        rec[3 * blockIdx.x] = (long long)smid;
        rec[3 * blockIdx.x + 1] = (long long)s_t0;
        rec[3 * blockIdx.x + 2] = (long long)s_t1;
    }
}

template <int OP>
static int probe_launch(unsigned blocks, int iters, float *sink, long long *rec, cudaStream_t st)
{
    k_pipe_probe<OP><<<blocks, kProbeThreads, 0, st>>>(iters, sink, rec);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

}  // namespace mpi

using namespace mpi;

extern "C" int mpi_probe_pipe_rate(int op, int blocks_per_sm, int iters, double *ops_per_clk_sm,
                                   double *ms, void *stream)
{
    if (op < MPI_PROBE_FMA || op > MPI_PROBE_FMA2 || blocks_per_sm < 1 || blocks_per_sm > 8 ||
        iters < 1 || iters > (1 << 20) || !ops_per_clk_sm) {
        set_error("invalid pipe probe arguments (op %d, blocks_per_sm %d, iters %d)", op,
                  blocks_per_sm, iters);
        return MPI_ERR_INVALID;
    }
    const cudaStream_t st = as_stream(stream);
    const unsigned blocks = (unsigned)(device_sm_count() * blocks_per_sm);
    Scratch scr(st);
    const size_t o_sink = scr.reserve(sizeof(float) * size_t(blocks) * kProbeThreads);
    const size_t o_rec = scr.reserve(sizeof(long long) * 3 * size_t(blocks));
    MPI_TRY(scr.allocate());
    float *sink = scr.at<float>(o_sink);
    long long *rec = scr.at<long long>(o_rec);
    cudaEvent_t ev[2];
    MPI_TRY_CUDA(cudaEventCreate(&ev[0]));
    MPI_TRY_CUDA(cudaEventCreate(&ev[1]));
    int rc = MPI_OK;
    MPI_TRY_CUDA(cudaEventRecord(ev[0], st));
    switch (op) {
        case MPI_PROBE_FMA: rc = probe_launch<MPI_PROBE_FMA>(blocks, iters, sink, rec, st); break;
        case MPI_PROBE_RSQRT: rc = probe_launch<MPI_PROBE_RSQRT>(blocks, iters, sink, rec, st); break;
        case MPI_PROBE_EX2: rc = probe_launch<MPI_PROBE_EX2>(blocks, iters, sink, rec, st); break;
        case MPI_PROBE_DFMA: rc = probe_launch<MPI_PROBE_DFMA>(blocks, iters, sink, rec, st); break;
        case MPI_PROBE_FMA2: rc = probe_launch<MPI_PROBE_FMA2>(blocks, iters, sink, rec, st); break;
        default: rc = probe_launch<MPI_PROBE_RCP>(blocks, iters, sink, rec, st); break;
    }
    MPI_TRY(rc);
    MPI_TRY_CUDA(cudaEventRecord(ev[1], st));
    std::vector<long long> h(3 * size_t(blocks));
    MPI_TRY_CUDA(cudaMemcpyAsync(h.data(), rec, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost, st));
    MPI_TRY_CUDA(cudaStreamSynchronize(st));
    float e_ms = 0.0f;
    MPI_TRY_CUDA(cudaEventElapsedTime(&e_ms, ev[0], ev[1]));
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (ms) *ms = e_ms;
    // Per SM: operations of its blocks over the span of their clocks.
    int max_sm = 0;
    for (unsigned b = 0; b < blocks; ++b) max_sm = std::max(max_sm, (int)h[3 * b]);
    std::vector<long long> lo(max_sm + 1, -1), hi(max_sm + 1, -1), nb(max_sm + 1, 0);
    for (unsigned b = 0; b < blocks; ++b) {
        const int s = (int)h[3 * b];
        if (s < 0) continue;
        lo[s] = (lo[s] < 0) ? h[3 * b + 1] : std::min(lo[s], h[3 * b + 1]);
        hi[s] = std::max(hi[s], h[3 * b + 2]);
        nb[s] += 1;
    }
    std::vector<double> rate;
    const double ops_per_block =
        double(kProbeThreads) * kProbeChains * double(iters) * (op == MPI_PROBE_FMA2 ? 2.0 : 1.0);
    for (int s = 0; s <= max_sm; ++s)
        if (nb[s] > 0 && hi[s] > lo[s]) rate.push_back(ops_per_block * double(nb[s]) / double(hi[s] - lo[s]));
    if (rate.empty()) {
        set_error("pipe probe recorded no SM clock spans");
        return MPI_ERR_CUDA;
    }
    std::sort(rate.begin(), rate.end());
    *ops_per_clk_sm = rate[rate.size() / 2];
    return MPI_OK;
}
