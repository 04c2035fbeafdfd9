// Pieces of the Core Stage (Eq. first:step) shared by the two- and the
// three-dimensional solves: the one-dimensional cosine weights of the
// interpolation, the binning of samples by interpolation cell (count, scan,
// stable ordering), the work units of the transpose and their ordered
// combine, and the CG solve over a Core Stage operator.  The non-template
// kernels live in grid_ops.cu behind the launchers declared here.
#pragma once

#include <algorithm>
#include <cmath>

#include "dfloat.cuh"
#include "pnp_ops.cuh"

namespace mpi {

struct AxisMap {
    double inv_h;   // 1/h
    double off;     // -p0/h - 1/2: continuous node index = p inv_h + off
    int n;
};

// Node interval and cosine weights of a position along one axis: between
// nodes k and k+1 at fraction f, node k+1 weighs (1 - cos(pi f))/2.  Outside
// the node hull the position clamps to the edge node.
template <typename R>
__device__ __forceinline__ void axis_weights(R pos, const AxisMap &a, int &k0, R &w0, R &w1)
{
    if (a.n == 1) { k0 = 0; w0 = R(1); w1 = R(0); return; }
    // The node index is formed in FP64: in FP32 its rounding (~1e-5 of a cell
    // on 100+ node grids) would already be visible in the weights.
    const double fi = double(pos) * a.inv_h + a.off;
    if (!(fi > 0.0)) { k0 = 0; w0 = R(1); w1 = R(0); return; }
    if (fi >= double(a.n - 1)) { k0 = a.n - 2; w0 = R(0); w1 = R(1); return; }
    int k = (int)floor(fi);
    k = min(k, a.n - 2);
    const R f = R(fi - double(k));
    k0 = k;
    if constexpr (sizeof(R) == 4) w1 = 0.5f * (1.0f - cospif(f));
    else w1 = 0.5 * (1.0 - cospi(f));
    w0 = R(1) - w1;
}

inline AxisMap make_axis(double p0, double h, int n)
{
    return AxisMap{1.0 / h, -p0 / h - 0.5, n};
}

constexpr int kInterpSPT = 4;     // samples per thread of the interpolation (gathers in flight)
// The transpose is organised in work units of at most kUnitLen consecutive
// entries of a cell's run of samples, so a cell where the trajectory dwells
// (thousands of samples) spreads over many units instead of keeping one
// group of lanes busy alone.  A node combines the unit sums of its adjacent
// cells in a fixed order (deterministic).
constexpr int kUnitLen = 128;
constexpr int kUnitLanes = 8;     // lanes per unit
constexpr int kUnitThreads = 256;

inline int grid_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

// count[c] += 1 for each lane's cell c (c < 0: none); lanes that hold the
// same cell add once.  All 32 lanes of the warp call it together.
__device__ __forceinline__ void warp_count_add(int *count, int c)
{
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    if (c >= 0 && int(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&count[c], __popc(peers));
}

// Binning (binning.cu).  Exclusive scan of count[0..n) into offset[0..n]
// (deterministic; tmp: cell_scan_bytes(n) of device scratch).
size_t cell_scan_bytes(int64_t n);
int cell_scan_launch(const int *count, int64_t n, int *offset, void *tmp, cudaStream_t st);
// list = the samples 0..T-1 ordered by cell_of, ascending sample index within
// a cell (a stable radix sort; tmp: cell_order_bytes(T) of device scratch,
// which also serves cell_scan_launch's scans of up to n_cells + 1 entries).
size_t cell_order_bytes(int64_t T);
int cell_order_launch(int64_t T, const int *cell_of, int n_cells, int *list, void *tmp, cudaStream_t st);

// Device scalars of one Core Stage CG solve.  A reduction's partial sums are
// added once per step, in a fixed order, by the block of the producing
// kernel that arrives last at the reduction's counter (the next kernel reads
// the finished scalar instead of every block re-adding the partials, which
// costs FP64 work quadratic in the block count).  No block waits for another.
struct CsScal {
    double rr;            // r.r of the current residual
    double alpha, beta;   // the step's coefficients
    float2 alpha_df, beta_df;  // the same as double-float pairs (double-float vectors)
    double bnorm, tol;    // ||b|| and the stop threshold on ||r|| (< 0: none)
    unsigned cnt[4];      // arrival counters of the reductions (zero between launches)
    int done;             // set once the solve has stopped
    int iters;            // CG updates performed
};
enum { kCntPq = 0, kCntRr = 1, kCntInit = 2 };

#ifdef __CUDACC__
// Called by every thread after thread 0 wrote this block's partial: true in
// the block that arrived last (which also re-arms the counter).  The partial
// is made visible device-wide before the arrival is counted; the last block
// reads the partials through L2 (cs_sum_parts).
__device__ __forceinline__ bool cs_last_block(unsigned *cnt, bool *sh_last)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(cnt, 1u);
        *sh_last = prev == gridDim.x - 1;
        if (*sh_last) {
            *cnt = 0u;
            __threadfence();
        }
    }
    __syncthreads();
    return *sh_last;
}

// Sum of n partials in a fixed order (thread strides, then a fixed tree),
// valid in thread 0.  The loads bypass L1: the partials come from other blocks.
template <int NT>
__device__ __forceinline__ double cs_sum_parts(const double *part, int n, double *sh /* >= NT/32 */)
{
    double a = 0.0;
    for (int k = threadIdx.x; k < n; k += NT) a += __ldcg(part + k);
    return block_sum<double, NT>(a, sh);
}

// After a step's <p, q> partials: pq, the stop test (stopped before, r.r or
// p.q exactly zero -- converged to round-off -- or ||r|| at or below the
// threshold) and alpha = r.r / p.q.  All threads call it.
template <int NT>
__device__ __forceinline__ void cs_finish_pq(const double *pq_part, int n, CsScal *sc, double *sh, bool *sh_last)
{
    if (!cs_last_block(&sc->cnt[kCntPq], sh_last)) return;
    const double pq = cs_sum_parts<NT>(pq_part, n, sh);
    if (threadIdx.x == 0) {
        const double rr = sc->rr;
        if (sc->done != 0 || rr == 0.0 || pq == 0.0 || (sc->tol >= 0.0 && sqrt(rr) <= sc->tol)) {
            sc->done = 1;
        } else {
            sc->alpha = rr / pq;
            sc->alpha_df = df_from_double(sc->alpha);
        }
    }
}

// Element arithmetic of the CG vectors: FP64, or double-float pairs (the
// FP32 path).  Scalars enter as FP64 or as double-float pairs.
__device__ __forceinline__ double cs_add(double a, double b) { return a + b; }
__device__ __forceinline__ df cs_add(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ double cs_axpy(double x, double a, double y) { return x + a * y; }  // x + a y
__device__ __forceinline__ df cs_axpy(df x, df a, df y) { return df_axpy(x, a, y); }
__device__ __forceinline__ double cs_scale(double x, double a) { return a * x; }
__device__ __forceinline__ df cs_scale(df x, df a) { return df_mul(x, a); }
template <typename E> __device__ __forceinline__ E cs_zero();
template <> __device__ __forceinline__ double cs_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ df cs_zero<df>() { return make_float2(0.0f, 0.0f); }
__device__ __forceinline__ double cs_neg(double a) { return -a; }
__device__ __forceinline__ df cs_neg(df a) { return df_neg(a); }
// The step's alpha / beta as the element type's scalar operand.
template <typename E> __device__ __forceinline__ E cs_alpha(const CsScal *sc);
template <> __device__ __forceinline__ double cs_alpha<double>(const CsScal *sc) { return sc->alpha; }
template <> __device__ __forceinline__ df cs_alpha<df>(const CsScal *sc) { return sc->alpha_df; }
template <typename E> __device__ __forceinline__ E cs_beta(const CsScal *sc);
template <> __device__ __forceinline__ double cs_beta<double>(const CsScal *sc) { return sc->beta; }
template <> __device__ __forceinline__ df cs_beta<df>(const CsScal *sc) { return sc->beta_df; }
// Per-thread accumulator of an inner product of element vectors.
// Sum over a block of NT threads of their double-float accumulators, on the
// FP32 pipe (a fixed butterfly per warp, then thread 0 over the warps in
// order), converted to FP64 once: the total at thread 0 (0 elsewhere); sh is
// reusable on return, as with block_sum.
template <int NT>
__device__ __forceinline__ double block_sum_f2(F2Sum v, double *sh /* >= NT/32 */)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        F2Sum t;
        t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v.add(t);
    }
    F2Sum *w = reinterpret_cast<F2Sum *>(sh);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        F2Sum s = w[0];
#pragma unroll
        for (int k = 1; k < NT / 32; ++k) s.add(w[k]);
        t = s.value();
    }
    __syncthreads();
    return t;
}

template <typename E> struct CsDot;
template <> struct CsDot<double> {
    double s;
    __device__ __forceinline__ void add(double a, double b) { s += a * b; }
    template <int NT> __device__ __forceinline__ double block_total(double *sh) const
    {
        return block_sum<double, NT>(s, sh);
    }
};
template <> struct CsDot<df> {
    F2Sum s;
    __device__ __forceinline__ void add(df a, df b) { df_dot_add(s, a, b); }
    template <int NT> __device__ __forceinline__ double block_total(double *sh) const
    {
        return block_sum_f2<NT>(s, sh);
    }
};
// An element as FP64 / from FP64 (right-hand sides and outputs).
__device__ __forceinline__ double cs_to_double(double a) { return a; }
__device__ __forceinline__ double cs_to_double(df a) { return df_to_double(a); }
template <typename E> __device__ __forceinline__ E cs_from_double(double v);
template <> __device__ __forceinline__ double cs_from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ df cs_from_double<df>(double v) { return df_from_double(v); }
// scale * s + add for a transpose sum s: FP64, or as a double-float pair
// (the error-free FP32 pair of the sum, scaled and added without rounding
// to FP64).
template <typename R>
__device__ __forceinline__ double cs_sum_scale_add(const SumAcc<R> &s, double scale, double add)
{
    return fma(s.value(), scale, add);
}
__device__ __forceinline__ df cs_sum_scale_add(const SumAcc<float> &s, df scale, df add)
{
    return df_add(df_mul(make_float2(s.s.hi, s.s.lo), scale), add);
}
// Stores an FP64 value as FP32, FP64 or a double-float pair.
__device__ __forceinline__ void cs_store(float &d, double v) { d = float(v); }
__device__ __forceinline__ void cs_store(double &d, double v) { d = v; }
__device__ __forceinline__ void cs_store(float2 &d, double v) { d = df_from_double(v); }
// An element rounded to FP32 (the operator's FP32 copy; outputs).
__device__ __forceinline__ float cs_to_float(double a) { return float(a); }
__device__ __forceinline__ float cs_to_float(df a) { return __fadd_rn(a.x, a.y); }
#endif

// The CG element type of a Core Stage in precision R: FP64 vectors for the
// FP64 path, double-float pairs for the FP32 path.
template <typename R> struct CsElem { using type = double; };
template <> struct CsElem<float> { using type = float2; };

// A host FP64 scalar as the element type's scalar operand.
inline double cs_host_scalar(double a, double *) { return a; }
inline float2 cs_host_scalar(double a, float2 *)
{
    const float hi = float(a);
    return float2{hi, float(a - double(hi))};
}

// Layouts of the FP32 copy of the CG direction an operator reads (FP32
// path), for N nodes: kP32Node4 / kP32Node2: a node's 4 / 2 components as one
// float4 / float2 (2-D); kP32Rows3x4 / kP32Rows1x4: three rows / one row of
// three components per node, each a float4 (A_{3k}, A_{3k+1}, A_{3k+2}, 0)
// (3-D).
enum P32Layout { kP32None = 0, kP32Node4, kP32Node2, kP32Rows3x4, kP32Rows1x4 };
struct P32 {
    float *buf = nullptr;
    int layout = kP32None;
    int64_t N = 0;
};

// A side stream for work of a step that is independent of its main chain:
// forked from and joined back into the step's stream with the two events
// (inside a graph capture this makes parallel branches).
struct StepFork {
    cudaStream_t side;
    cudaEvent_t fork, join;
};

// The operator of one Core Stage solve on nv unknowns (all components of all
// nodes) of element type E: FP64, or double-float pairs on the FP32 path.
// Its methods only enqueue.
template <typename E>
struct CoreStageOp {
    virtual ~CoreStageOp() = default;
    // The FP32 copy of p the operator reads (buf null: it reads p in FP64).
    // The solve keeps the copy equal to p rounded to FP32: it writes it after
    // the first direction and with every direction update.
    virtual P32 p32() const { return P32{}; }
    // q = (1/T) M^T M p + gamma Lap Lap p and the partial sums of <p, q> in
    // pq_blocks(nv) fixed blocks, finished by the producing kernel with
    // cs_finish_pq on sc.  l1, l2: work vectors of nv values.
    virtual int pq_blocks(int64_t nv) const = 0;
    virtual int step_q(const E *p, double gamma, E *q, double *pq_part, CsScal *sc, E *l1, E *l2,
                       const StepFork &fk, cudaStream_t st) = 0;
};

// CG from x = 0 on ((1/T) M^T M + gamma Lap Lap) x = b (Eq. first:step; Lap is
// symmetric, so Lap^T Lap = Lap Lap) with opts' gamma, iteration limit and
// relative tolerance; writes x (nv values of type E: double, or float2
// double-float pairs).  With a tolerance the host polls the device stop flag
// every 16 steps.  With n_iter_out (host) the stream is synchronised and the
// number of CG updates stored.
template <typename E>
int core_stage_cg(CoreStageOp<E> &op, int64_t nv, const E *b, const mpi_grid_opts &o, E *x, int *n_iter_out,
                  cudaStream_t st);

// rec[q] = rec_t[list[q]] and vs[q] = v[list[q]] (D velocity components):
// the records and velocities of the samples in list (cell) order.
template <typename Rec, typename R, int D>
__global__ void k_sort_records(int64_t T, const int *__restrict__ list, const Rec *__restrict__ rec_t,
                               const R *__restrict__ v, Rec *__restrict__ rec, R *__restrict__ vs)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < T;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = list[q];
        rec[q] = rec_t[t];
#pragma unroll
        for (int m = 0; m < D; ++m) vs[D * q + m] = v[D * t + m];
    }
}

// out[k][q] = in[k][list[q]] for the n_rows rows of a [n_rows][T] array.
template <typename R>
__global__ void k_gather_rows(int64_t T, int n_rows, const int *__restrict__ list, const R *__restrict__ in,
                              R *__restrict__ out)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < T;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = list[q];
        for (int k = 0; k < n_rows; ++k) out[(int64_t)k * T + q] = in[(int64_t)k * T + t];
    }
}

template <typename R>
int gather_rows(int64_t T, int n_rows, const int *list, const R *in, R *out, cudaStream_t st)
{
    if (T == 0) return MPI_OK;
    k_gather_rows<R><<<grid_blocks(T), 256, 0, st>>>(T, n_rows, list, in, out);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

}  // namespace mpi
