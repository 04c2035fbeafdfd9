// Batched ZeroShot-PnP (Algorithm 1 with the forward operator A) over many
// independent frames of uneven grid size and trajectory length, FP32
// operator with FP64 CG vectors and inner products.
//
// Every operator application over all frames is ONE launch of the pair
// kernel over a frame table (the work items of all frames in one grid, or one
// persistent grid pulling items from a device counter), followed by one
// batched chunk reduction.  The CG vector kernels, the percentile/variance
// step and the Gaussian denoiser are batched the same way (a block belongs to
// exactly one frame; each frame keeps its own CG and PnP scalars on the
// device).  One PnP iteration of all frames is captured once as a CUDA graph
// and replayed n_iter times.  Work-item sizes and the launch form are chosen
// by timing candidates on the first run (the autotuner), optionally cached in
// a file.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <functional>
#include <sstream>
#include <string>
#include <vector>

#include "pair_kernels.cuh"
#include "pnp_device.cuh"

namespace mpi {

int check_model(const mpi_model *m);
int check_grid(const mpi_grid_desc *g);
int check_traj(const mpi_traj *t);
ModelH to_host(const mpi_model *m);
GridH to_host(const mpi_grid_desc *g);

constexpr int kMaxBatch = MPI_BATCH_MAX_FRAMES;
using PairTab = PairBatch<float, kMaxBatch>;

// ---------------------------------------------------------------------------
// Batched kernels.

struct RedFrame {
    const float *part;
    void *out;
    const double *p;
    const double *nu;
    double *dot;
    int64_t len;
    int64_t blk0;
    int n_chunks;
};
struct RedTab {
    int n;
    RedFrame f[kMaxBatch];
};

template <typename T, int MAXN>
__device__ __forceinline__ int frame_of(const T (&f)[MAXN], int n, int64_t b)
{
    int k = 0;
#pragma unroll 1
    for (int q = 1; q < n; ++q)
        if (b >= f[q].blk0) k = q;
    return k;
}

// Chunk reduction of every frame (same arithmetic as the single-frame
// reduction): block = 32 elements of one frame.
template <typename OUT, bool CG>
__global__ void __launch_bounds__(256) k_reduce_batch(const __grid_constant__ RedTab B)
{
    __shared__ SumAcc<float> sh[8][33];
    const RedFrame &F = B.f[frame_of(B.f, B.n, blockIdx.x)];
    const int64_t b = blockIdx.x - F.blk0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = b * 32 + lane;
    SumAcc<float> acc{};
    if (e < F.len) {
#pragma unroll 8
        for (int c = w; c < F.n_chunks; c += 8) acc.add(F.part[(int64_t)c * F.len + e]);
    }
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0) {
        SumAcc<float> all{};
#pragma unroll
        for (int k = 0; k < 8; ++k) all.add(sh[k][lane]);
        double tot = all.value();
        OUT *out = reinterpret_cast<OUT *>(F.out);
        if constexpr (CG) {
            const double pe = e < F.len ? F.p[e] : 0.0;
            tot += *F.nu * pe;
            if (e < F.len) out[e] = OUT(tot);
            const double dot = warp_sum(pe * tot);
            if (lane == 0) F.dot[b] = dot;
        } else {
            if (e < F.len) out[e] = OUT(tot);
        }
    }
}

struct VecFrame {
    int64_t off, N;
    int64_t blk0;
    int nblk;
    int n_pq;
    const double *pq;
    double *rr[2];
    int *done;
    double *scal;
};
struct VecTab {
    int n;
    VecFrame f[kMaxBatch];
};

__global__ void __launch_bounds__(kVecThreads)
k_set_x_b(const __grid_constant__ VecTab B, const float *__restrict__ rho2, double *__restrict__ x)
{
    const VecFrame &F = B.f[frame_of(B.f, B.n, blockIdx.x)];
    const int64_t lb = blockIdx.x - F.blk0;
    const int64_t e0 = lb * kVecPerBlock, e1 = min(F.N, e0 + kVecPerBlock);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kVecThreads) x[F.off + e] = double(rho2[F.off + e]);
}

__global__ void __launch_bounds__(kVecThreads)
k_cg_init_b(const __grid_constant__ VecTab B, const double *__restrict__ b0, const double *__restrict__ x,
            const double *__restrict__ q, double *__restrict__ r, double *__restrict__ p)
{
    __shared__ double sh[kVecThreads / 32 + 1];
    const VecFrame &F = B.f[frame_of(B.f, B.n, blockIdx.x)];
    const int64_t lb = blockIdx.x - F.blk0;
    const double nu = F.scal[kScalNu];
    const int64_t e0 = lb * kVecPerBlock, e1 = min(F.N, e0 + kVecPerBlock);
    double acc = 0.0;
    for (int64_t e = F.off + e0 + threadIdx.x; e < F.off + e1; e += kVecThreads) {
        const double re = (b0[e] + nu * x[e]) - q[e];
        r[e] = re;
        p[e] = re;
        acc += re * re;
    }
    acc = block_sum<double, kVecThreads>(acc, sh);
    if (threadIdx.x == 0) {
        F.rr[0][lb] = acc;
        if (lb == 0) *F.done = 0;
    }
}

__global__ void __launch_bounds__(kVecThreads)
k_cg_step1_b(const __grid_constant__ VecTab B, int parity, double *__restrict__ x,
             double *__restrict__ r, const double *__restrict__ p, const double *__restrict__ q)
{
    __shared__ double sh[kVecThreads / 32 + 1];
    const VecFrame &F = B.f[frame_of(B.f, B.n, blockIdx.x)];
    const int64_t lb = blockIdx.x - F.blk0;
    const double *rr_in = F.rr[parity];
    double *rr_out = F.rr[parity ^ 1];
    const double rr = sum_parts<kVecThreads>(rr_in, F.nblk, sh);
    const double pq = sum_parts<kVecThreads>(F.pq, F.n_pq, sh);
    const bool stop = (*F.done != 0) || rr == 0.0 || pq == 0.0;
    if (stop) {
        if (threadIdx.x == 0) {
            rr_out[lb] = rr_in[lb];
            if (lb == 0) *F.done = 1;
        }
        return;
    }
    const double alpha = rr / pq;
    const int64_t e0 = lb * kVecPerBlock, e1 = min(F.N, e0 + kVecPerBlock);
    double acc = 0.0;
    for (int64_t e = F.off + e0 + threadIdx.x; e < F.off + e1; e += kVecThreads) {
        x[e] = x[e] + alpha * p[e];
        const double re = r[e] - alpha * q[e];
        r[e] = re;
        acc += re * re;
    }
    acc = block_sum<double, kVecThreads>(acc, sh);
    if (threadIdx.x == 0) rr_out[lb] = acc;
}

__global__ void __launch_bounds__(kVecThreads)
k_cg_step2_b(const __grid_constant__ VecTab B, int parity, const double *__restrict__ r,
             double *__restrict__ p)
{
    __shared__ double sh[kVecThreads / 32 + 1];
    const VecFrame &F = B.f[frame_of(B.f, B.n, blockIdx.x)];
    if (*F.done) return;
    const int64_t lb = blockIdx.x - F.blk0;
    const double ro = sum_parts<kVecThreads>(F.rr[parity], F.nblk, sh);
    const double rn = sum_parts<kVecThreads>(F.rr[parity ^ 1], F.nblk, sh);
    const double beta = rn / ro;
    const int64_t e0 = lb * kVecPerBlock, e1 = min(F.N, e0 + kVecPerBlock);
    for (int64_t e = F.off + e0 + threadIdx.x; e < F.off + e1; e += kVecThreads) p[e] = r[e] + beta * p[e];
}

struct StatTab {
    int n;
    int do_clip;
    int final_parity;
    double pct;
    VecFrame f[kMaxBatch];
    double nu0[kMaxBatch];
};

// One block per frame: percentile trimming, noise estimate and PnP scalars.
__global__ void __launch_bounds__(kStatThreads)
k_stats_b(const __grid_constant__ StatTab B, const double *__restrict__ x, float *__restrict__ rho1)
{
    const VecFrame &F = B.f[blockIdx.x];
    const bool first = F.scal[kScalIter] == 0.0;
    outer_stats_block<float>(F.N, x + F.off, B.do_clip, B.pct, first, B.nu0[blockIdx.x], F.scal,
                             F.rr[B.final_parity], F.nblk, nullptr, rho1 + F.off);
    if (threadIdx.x == 0) F.scal[kScalIter] += 1.0;
}

struct GaussFrame {
    int64_t off;
    int nx, ny;
};
struct GaussTab {
    int n;
    float w0, w1, w2;
    GaussFrame f[kMaxBatch];
};

__global__ void __launch_bounds__(kGx *kGy)
k_gauss_b(const __grid_constant__ GaussTab B, const float *__restrict__ in, float *__restrict__ out)
{
    const GaussFrame &F = B.f[blockIdx.z];
    if ((int)blockIdx.x * kGx >= F.nx || (int)blockIdx.y * kGy >= F.ny) return;  // whole block
    gauss5_tile<float>(in + F.off, out + F.off, F.nx, F.ny, blockIdx.x * kGx, blockIdx.y * kGy, B.w0,
                       B.w1, B.w2);
}

__global__ void k_init_b(const __grid_constant__ StatTab B)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < B.n) {
        double *s = B.f[f].scal;
        for (int k = 0; k < 8; ++k) s[k] = 0.0;
        s[kScalNu] = B.nu0[f];
    }
}

// ---------------------------------------------------------------------------
// Splits of one frame for a work-item budget (pairs per item).

static FwdSplit fwd_split_budget(int64_t T, int nx, int ny, int64_t budget)
{
    FwdSplit sp;
    sp.n_tiles = (int)std::max<int64_t>(1, (T + kFwdTile - 1) / kFwdTile);
    int64_t rows = budget / ((int64_t)kFwdTile * nx);
    rows = std::max<int64_t>(1, std::min<int64_t>(rows, ny));
    sp.chunk_rows = (int)rows;
    sp.n_chunks = (int)((ny + rows - 1) / rows);
    sp.rows_staged = fwd_rows_staged((int)rows, nx, sizeof(float));
    return sp;
}

static AdjSplit adj_split_budget(int64_t T, int nx, int ny, int64_t budget)
{
    AdjSplit sp;
    sp.tiles_x = (nx + kAdjTileX - 1) / kAdjTileX;
    sp.tiles_y = (ny + kAdjTileY - 1) / kAdjTileY;
    int64_t len = budget / (kAdjTileX * kAdjTileY);
    len = std::max<int64_t>(kAdjBlock, len / kAdjBlock * kAdjBlock);
    sp.chunk_len = (int)std::min<int64_t>(len, (int64_t)1 << 30);
    sp.n_chunks = (int)std::max<int64_t>(1, (T + sp.chunk_len - 1) / sp.chunk_len);
    return sp;
}

static const int64_t kBudgets[] = {1 << 20, 1 << 21, 1 << 22, 1 << 23};
static const int64_t kDefaultBudget = 1 << 21;

}  // namespace mpi

using namespace mpi;

struct mpi_batch_plan {
    int n = 0;
    int n_iter = 0, n_cg = 0;
    double clip_pct = 5.0;
    int flags = 0;
    bool diag = true;   // every frame has a diagonal G
    bool mixed = false; // some frames diagonal, some not
    std::vector<ModelH> m;
    std::vector<GridH> g;
    std::vector<int64_t> T, N, voff;
    std::vector<double> nu0;
    int64_t Ntot = 0;
    // device memory (one allocation owned by the plan)
    char *dev = nullptr;
    size_t dev_bytes = 0;
    std::vector<Geometry<float>> geo;
    std::vector<float *> fwd_part, adj_part, sA;
    std::vector<double *> pq, rr0, rr1, scal;
    std::vector<int *> done;
    double *b0 = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    float *rho1 = nullptr, *rho2 = nullptr;
    unsigned long long *queues = nullptr;  // [forward 2][adjoint 2]
    std::vector<int> nvblk, npq;
    // chosen configuration
    bool tuned = false;
    int64_t fwd_budget = kDefaultBudget, adj_budget = kDefaultBudget;
    bool fwd_persist = false, adj_persist = false;
    std::vector<FwdSplit> fs;
    std::vector<AdjSplit> as;
    int64_t fwd_items = 0, adj_items = 0;
    size_t fwd_smem = 0;
    int fwd_grid_persist = 0, adj_grid_persist = 0;
    // tables
    PairTab fwd_tab[2];  // input x / p
    PairTab adj_tab;
    RedTab red_fwd;
    RedTab red_adj[2];  // epilogue with x / p
    VecTab vec;
    StatTab stat;
    GaussTab gauss;
    int64_t vec_blocks_tot = 0;
    // graph of one PnP iteration
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_nodes = 0;
};

namespace mpi {

static int64_t frame_items_fwd(const FwdSplit &s) { return (int64_t)s.n_tiles * s.n_chunks; }
static int64_t frame_items_adj(const AdjSplit &s) { return (int64_t)s.tiles_x * s.tiles_y * s.n_chunks; }

// Splits for the given budgets (or, with MPI_BATCH_MATCH_SINGLE, exactly the
// single-frame splits) and the tables that depend on them.
static void configure(mpi_batch_plan &P, int64_t fb, int64_t ab, bool fpers, bool apers)
{
    P.fwd_budget = fb;
    P.adj_budget = ab;
    P.fwd_persist = fpers;
    P.adj_persist = apers;
    P.fs.resize(P.n);
    P.as.resize(P.n);
    const bool single = (P.flags & MPI_BATCH_MATCH_SINGLE) != 0;
    for (int f = 0; f < P.n; ++f) {
        P.fs[f] = single ? forward_split(P.T[f], P.g[f].nx, P.g[f].ny, 4, forward_target_items())
                         : fwd_split_budget(P.T[f], P.g[f].nx, P.g[f].ny, fb);
        P.as[f] = single ? adjoint_split(P.T[f], P.g[f].nx, P.g[f].ny, default_target_items(), 4)
                         : adj_split_budget(P.T[f], P.g[f].nx, P.g[f].ny, ab);
    }
    int64_t fi = 0, ai = 0;
    size_t smem = 0;
    for (int t = 0; t < 2; ++t) P.fwd_tab[t].n_frames = P.n;
    P.adj_tab.n_frames = P.n;
    for (int f = 0; f < P.n; ++f) {
        PairFrame<float> base{};
        base.rw = P.geo[f].rw;
        base.xcol = P.geo[f].xcol;
        base.yrow = P.geo[f].yrow;
        base.T = P.T[f];
        base.nx = P.g[f].nx;
        base.ny = P.g[f].ny;
        base.n_ch = P.m[f].n_ch;
        base.diag = (P.m[f].G[1] == 0.0 && P.m[f].G[2] == 0.0) ? 1 : 0;
        for (int k = 0; k < 4; ++k) base.p[k] = float(P.m[f].p[k]);
        PairFrame<float> fw = base;
        fw.item0 = fi;
        fw.part = P.fwd_part[f];
        fw.n_tiles = P.fs[f].n_tiles;
        fw.chunk = P.fs[f].chunk_rows;
        fw.rows_staged = P.fs[f].rows_staged;
        fw.near_cols = near_columns<float>(P.m[f], P.g[f]);
        P.fwd_tab[0].f[f] = fw;
        P.fwd_tab[0].f[f].in = P.x + P.voff[f];
        P.fwd_tab[1].f[f] = fw;
        P.fwd_tab[1].f[f].in = P.p + P.voff[f];
        fi += frame_items_fwd(P.fs[f]);
        smem = std::max(smem, fwd_smem_bytes(P.g[f].nx, P.fs[f].rows_staged, sizeof(float)));
        PairFrame<float> ad = base;
        ad.item0 = ai;
        ad.in = P.sA[f];
        ad.part = P.adj_part[f];
        ad.n_tiles = P.as[f].tiles_x * P.as[f].tiles_y;
        ad.tiles_x = P.as[f].tiles_x;
        ad.chunk = P.as[f].chunk_len;
        P.adj_tab.f[f] = ad;
        ai += frame_items_adj(P.as[f]);
    }
    P.fwd_items = fi;
    P.adj_items = ai;
    P.fwd_smem = smem;
    // reductions
    int64_t b = 0;
    P.red_fwd.n = P.n;
    for (int f = 0; f < P.n; ++f) {
        RedFrame &R = P.red_fwd.f[f];
        R = RedFrame{};
        R.part = P.fwd_part[f];
        R.out = P.sA[f];
        R.len = (int64_t)P.m[f].n_ch * P.T[f];
        R.n_chunks = P.fs[f].n_chunks;
        R.blk0 = b;
        b += (R.len + 31) / 32;
    }
    for (int t = 0; t < 2; ++t) {
        P.red_adj[t].n = P.n;
        int64_t bb = 0;
        for (int f = 0; f < P.n; ++f) {
            RedFrame &R = P.red_adj[t].f[f];
            R = RedFrame{};
            R.part = P.adj_part[f];
            R.out = P.q + P.voff[f];
            R.p = (t == 0 ? P.x : P.p) + P.voff[f];
            R.nu = P.scal[f] + kScalNu;
            R.dot = P.pq[f];
            R.len = P.N[f];
            R.n_chunks = P.as[f].n_chunks;
            R.blk0 = bb;
            bb += (R.len + 31) / 32;
        }
    }
}

static int64_t red_blocks(const RedTab &t)
{
    const RedFrame &L = t.f[t.n - 1];
    return L.blk0 + (L.len + 31) / 32;
}

static int persistent_grid(const void *kern, int threads, size_t smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * device_sm_count();
}

// Kernel variant for the plan's mix of diagonal / general gradients.
using FwdK = void (*)(PairTab);
using FwdPK = void (*)(PairTab, int64_t, unsigned long long *);
static FwdK fwd_kernel(const mpi_batch_plan &P)
{
    return P.mixed ? k_forward<float, double, 2, kMaxBatch>
                   : (P.diag ? k_forward<float, double, 1, kMaxBatch> : k_forward<float, double, 0, kMaxBatch>);
}
static FwdPK fwd_kernel_persistent(const mpi_batch_plan &P)
{
    return P.mixed ? k_forward_persistent<float, double, 2, kMaxBatch>
                   : (P.diag ? k_forward_persistent<float, double, 1, kMaxBatch>
                             : k_forward_persistent<float, double, 0, kMaxBatch>);
}
static FwdK adj_kernel(const mpi_batch_plan &P)
{
    return P.mixed ? k_adjoint<float, 2, false, kMaxBatch>
                   : (P.diag ? k_adjoint<float, 1, false, kMaxBatch> : k_adjoint<float, 0, false, kMaxBatch>);
}
static FwdPK adj_kernel_persistent(const mpi_batch_plan &P)
{
    return P.mixed ? k_adjoint_persistent<float, 2, false, kMaxBatch>
                   : (P.diag ? k_adjoint_persistent<float, 1, false, kMaxBatch>
                             : k_adjoint_persistent<float, 0, false, kMaxBatch>);
}

// Launch attributes that depend on the split: set outside any stream capture.
static int prepare_launch(mpi_batch_plan &P)
{
    auto kf = fwd_kernel(P);
    auto kfp = fwd_kernel_persistent(P);
    auto kap = adj_kernel_persistent(P);
    if (P.fwd_smem > 48 * 1024) {
        MPI_TRY_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.fwd_smem));
        MPI_TRY_CUDA(cudaFuncSetAttribute(kfp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P.fwd_smem));
    }
    P.fwd_grid_persist = (int)std::min<int64_t>(P.fwd_items, persistent_grid((const void *)kfp, kFwdThreads, P.fwd_smem));
    P.adj_grid_persist = (int)std::min<int64_t>(P.adj_items, persistent_grid((const void *)kap, kAdjThreads, 0));
    return MPI_OK;
}

static int launch_fwd(mpi_batch_plan &P, int which, cudaStream_t st)
{
    const PairTab &B = P.fwd_tab[which];
    {
        ProfScope prof(kProfForward, st);
        if (P.fwd_persist) {
            auto k = fwd_kernel_persistent(P);
            k<<<P.fwd_grid_persist, kFwdThreads, P.fwd_smem, st>>>(B, P.fwd_items, P.queues);
        } else {
            auto k = fwd_kernel(P);
            k<<<(unsigned)P.fwd_items, kFwdThreads, P.fwd_smem, st>>>(B);
        }
        MPI_CHECK_LAUNCH();
    }
    k_reduce_batch<float, false><<<(unsigned)red_blocks(P.red_fwd), 256, 0, st>>>(P.red_fwd);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

static int launch_adj_kernel(mpi_batch_plan &P, const PairTab &B, cudaStream_t st)
{
    ProfScope prof(kProfAdjoint, st);
    if (P.adj_persist) {
        auto k = adj_kernel_persistent(P);
        k<<<P.adj_grid_persist, kAdjThreads, 0, st>>>(B, P.adj_items, P.queues + 2);
    } else {
        auto k = adj_kernel(P);
        k<<<(unsigned)P.adj_items, kAdjThreads, 0, st>>>(B);
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// q = (A^T A + nu I) v for every frame (v = x for which = 0, p for 1).
static int apply_normal_b(mpi_batch_plan &P, int which, cudaStream_t st)
{
    MPI_TRY(launch_fwd(P, which, st));
    MPI_TRY(launch_adj_kernel(P, P.adj_tab, st));
    k_reduce_batch<double, true><<<(unsigned)red_blocks(P.red_adj[which]), 256, 0, st>>>(P.red_adj[which]);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

static int enqueue_iteration(mpi_batch_plan &P, cudaStream_t st)
{
    const unsigned vb = (unsigned)P.vec_blocks_tot;
    k_set_x_b<<<vb, kVecThreads, 0, st>>>(P.vec, P.rho2, P.x);
    MPI_CHECK_LAUNCH();
    MPI_TRY(apply_normal_b(P, 0, st));
    k_cg_init_b<<<vb, kVecThreads, 0, st>>>(P.vec, P.b0, P.x, P.q, P.r, P.p);
    MPI_CHECK_LAUNCH();
    for (int i = 0; i < P.n_cg; ++i) {
        MPI_TRY(apply_normal_b(P, 1, st));
        k_cg_step1_b<<<vb, kVecThreads, 0, st>>>(P.vec, i & 1, P.x, P.r, P.p, P.q);
        MPI_CHECK_LAUNCH();
        k_cg_step2_b<<<vb, kVecThreads, 0, st>>>(P.vec, i & 1, P.r, P.p);
        MPI_CHECK_LAUNCH();
    }
    k_stats_b<<<P.n, kStatThreads, 0, st>>>(P.stat, P.x, P.rho1);
    MPI_CHECK_LAUNCH();
    int mtx = 1, mty = 1;
    for (int f = 0; f < P.n; ++f) {
        mtx = std::max(mtx, (P.g[f].nx + kGx - 1) / kGx);
        mty = std::max(mty, (P.g[f].ny + kGy - 1) / kGy);
    }
    k_gauss_b<<<dim3(mtx, mty, P.n), kGx * kGy, 0, st>>>(P.gauss, P.rho1, P.rho2);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

static std::string tune_key(const mpi_batch_plan &P)
{
    cudaDeviceProp prop{};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::ostringstream os;
    os << prop.name << "|sm" << prop.multiProcessorCount << "|f32|" << (P.mixed ? "m" : P.diag ? "d" : "g");
    for (int f = 0; f < P.n; ++f) os << "|" << P.g[f].nx << "x" << P.g[f].ny << "x" << P.T[f] << "c" << P.m[f].n_ch;
    const size_t h = std::hash<std::string>{}(os.str());
    char buf[32];
    snprintf(buf, sizeof(buf), "%016zx", h);
    return buf;
}

static bool cache_lookup(const std::string &key, int64_t &fb, int &fp, int64_t &ab, int &ap)
{
    const char *path = getenv("MPI_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    std::ifstream in(path);
    std::string k;
    long long a, c;
    int b, d;
    while (in >> k >> a >> b >> c >> d) {
        if (k == key) {
            fb = a; fp = b; ab = c; ap = d;
            return true;
        }
    }
    return false;
}

static void cache_store(const std::string &key, int64_t fb, int fp, int64_t ab, int ap)
{
    const char *path = getenv("MPI_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    std::ofstream out(path, std::ios::app);
    out << key << " " << (long long)fb << " " << fp << " " << (long long)ab << " " << ap << "\n";
}

// Time each candidate (work-item budget x launch form) of the forward and of
// the adjoint launch over all frames on the current inputs and keep the
// fastest of each.  The candidates change only how the sums are split into
// work items, not what is summed.
static int autotune(mpi_batch_plan &P, cudaStream_t st)
{
    const std::string key = tune_key(P);
    int64_t fb, ab;
    int fp, ap;
    if (cache_lookup(key, fb, fp, ab, ap)) {
        configure(P, fb, ab, fp != 0, ap != 0);
        MPI_TRY(prepare_launch(P));
        P.tuned = true;
        return MPI_OK;
    }
    cudaEvent_t e0, e1;
    MPI_TRY_CUDA(cudaEventCreate(&e0));
    MPI_TRY_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } guard{e0, e1};
    float best_f = 1e30f, best_a = 1e30f;
    int64_t bf = kDefaultBudget, ba = kDefaultBudget;
    bool pf = false, pa = false;
    for (int64_t budget : kBudgets) {
        for (int pers = 0; pers < 2; ++pers) {
            configure(P, budget, budget, pers != 0, pers != 0);
            MPI_TRY(prepare_launch(P));
            float ms_f = 0.f, ms_a = 0.f;
            for (int rep = 0; rep < 2; ++rep) {  // first run warms up
                MPI_TRY_CUDA(cudaEventRecord(e0, st));
                MPI_TRY(launch_fwd(P, 0, st));
                MPI_TRY_CUDA(cudaEventRecord(e1, st));
                MPI_TRY_CUDA(cudaEventSynchronize(e1));
                MPI_TRY_CUDA(cudaEventElapsedTime(&ms_f, e0, e1));
                MPI_TRY_CUDA(cudaEventRecord(e0, st));
                MPI_TRY(launch_adj_kernel(P, P.adj_tab, st));
                MPI_TRY_CUDA(cudaEventRecord(e1, st));
                MPI_TRY_CUDA(cudaEventSynchronize(e1));
                MPI_TRY_CUDA(cudaEventElapsedTime(&ms_a, e0, e1));
            }
            if (ms_f < best_f) { best_f = ms_f; bf = budget; pf = pers != 0; }
            if (ms_a < best_a) { best_a = ms_a; ba = budget; pa = pers != 0; }
        }
    }
    configure(P, bf, ba, pf, pa);
    MPI_TRY(prepare_launch(P));
    cache_store(key, bf, pf ? 1 : 0, ba, pa ? 1 : 0);
    P.tuned = true;
    return MPI_OK;
}

static int capture_iteration(mpi_batch_plan &P)
{
    if (P.exec) return MPI_OK;
    if (!P.cap_stream) MPI_TRY_CUDA(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
    MPI_TRY_CUDA(cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long before = mpi_kernel_launches();
    const int st = enqueue_iteration(P, P.cap_stream);
    note_launches(before - mpi_kernel_launches());  // captured, not launched
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(P.cap_stream, &g);
    if (st != MPI_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    MPI_TRY_CUDA(ec);
    P.graph = g;
    MPI_TRY_CUDA(cudaGraphGetNodes(g, nullptr, &P.graph_nodes));
    MPI_TRY_CUDA(cudaGraphInstantiate(&P.exec, g, 0));
    return MPI_OK;
}

static void free_plan(mpi_batch_plan *P)
{
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
    if (P->dev) cudaFree(P->dev);
    delete P;
}

}  // namespace mpi

extern "C" {

int mpi_batch_plan_create(int n_frames, const mpi_model *models, const mpi_grid_desc *grids,
                          const int64_t *T, const double *nu0, const mpi_pnp_opts *opts, int flags,
                          mpi_batch_plan **plan)
{
    if (!plan) { set_error("plan is NULL"); return MPI_ERR_INVALID; }
    *plan = nullptr;
    if (n_frames < 1 || n_frames > kMaxBatch) {
        set_error("n_frames must be in [1, %d] (got %d)", kMaxBatch, n_frames);
        return n_frames > kMaxBatch ? MPI_ERR_UNSUPPORTED : MPI_ERR_INVALID;
    }
    if (!models || !grids || !T || !nu0 || !opts) { set_error("NULL plan argument"); return MPI_ERR_INVALID; }
    if (opts->op != MPI_OP_FORWARD) {
        set_error("batched plans run the forward-operator PnP only");
        return MPI_ERR_UNSUPPORTED;
    }
    if (opts->n_iter < 0 || opts->n_cg < 0 || !(opts->clip_pct <= 100.0) || std::isnan(opts->clip_pct)) {
        set_error("invalid PnP options");
        return MPI_ERR_INVALID;
    }
    mpi_batch_plan *P = new mpi_batch_plan();
    P->n = n_frames;
    P->n_iter = opts->n_iter;
    P->n_cg = opts->n_cg;
    P->clip_pct = opts->clip_pct;
    P->flags = flags;
    for (int f = 0; f < n_frames; ++f) {
        int st = check_model(&models[f]);
        if (st == MPI_OK) st = check_grid(&grids[f]);
        if (st == MPI_OK && (T[f] < 1 || T[f] >= ((int64_t)1 << 31))) {
            set_error("frame %d: T must be in [1, 2^31)", f);
            st = MPI_ERR_INVALID;
        }
        if (st == MPI_OK && !(nu0[f] >= 0.0 && std::isfinite(nu0[f]))) {
            set_error("frame %d: nu0 must be finite and >= 0", f);
            st = MPI_ERR_INVALID;
        }
        if (st != MPI_OK) {
            delete P;
            return st;
        }
        P->m.push_back(to_host(&models[f]));
        P->g.push_back(to_host(&grids[f]));
        P->T.push_back(T[f]);
        P->nu0.push_back(nu0[f]);
        P->N.push_back((int64_t)grids[f].nx * grids[f].ny);
        P->voff.push_back(P->Ntot);
        P->Ntot += P->N.back();
        if (models[f].G[1] != 0.0 || models[f].G[2] != 0.0) P->diag = false;
        else P->mixed = true;  // provisional: resolved after the loop
    }
    {
        bool any_diag = false, any_gen = false;
        for (int f = 0; f < n_frames; ++f) {
            const bool d = P->m[f].G[1] == 0.0 && P->m[f].G[2] == 0.0;
            any_diag |= d;
            any_gen |= !d;
        }
        P->mixed = any_diag && any_gen;
        P->diag = any_diag && !any_gen;
    }
    // Device memory: sized for the smallest work-item budget (most chunks).
    const int64_t bmin = kBudgets[0];
    std::vector<size_t> o_geo, o_fp, o_ap, o_sA, o_pq, o_rr0, o_rr1, o_sc;
    size_t tot = 0;
    auto take = [&](size_t b) { size_t o = tot; tot += (b + 255) & ~size_t(255); return o; };
    for (int f = 0; f < n_frames; ++f) {
        const FwdSplit fs_min = fwd_split_budget(P->T[f], P->g[f].nx, P->g[f].ny, bmin);
        const FwdSplit fs_single = forward_split(P->T[f], P->g[f].nx, P->g[f].ny, 4, forward_target_items());
        const AdjSplit as_min = adj_split_budget(P->T[f], P->g[f].nx, P->g[f].ny, bmin);
        const AdjSplit as_single = adjoint_split(P->T[f], P->g[f].nx, P->g[f].ny, default_target_items(), 4);
        const int fch = std::max(fs_min.n_chunks, fs_single.n_chunks);
        const int ach = std::max(as_min.n_chunks, as_single.n_chunks);
        o_geo.push_back(take(geometry_bytes<float>(P->T[f], P->g[f].nx, P->g[f].ny)));
        o_fp.push_back(take(sizeof(float) * size_t(fch) * P->m[f].n_ch * P->T[f]));
        o_ap.push_back(take(sizeof(float) * size_t(ach) * P->N[f]));
        o_sA.push_back(take(sizeof(float) * P->m[f].n_ch * P->T[f]));
        P->npq.push_back((int)((P->N[f] + 31) / 32));
        P->nvblk.push_back(vec_blocks(P->N[f]));
        o_pq.push_back(take(sizeof(double) * P->npq.back()));
        o_rr0.push_back(take(sizeof(double) * P->nvblk.back()));
        o_rr1.push_back(take(sizeof(double) * P->nvblk.back()));
        o_sc.push_back(take(sizeof(double) * 8 + sizeof(int) * 4));
    }
    const size_t vb = sizeof(double) * P->Ntot;
    const size_t o_b0 = take(vb), o_x = take(vb), o_r = take(vb), o_p = take(vb), o_q = take(vb);
    const size_t o_r1 = take(sizeof(float) * P->Ntot), o_r2 = take(sizeof(float) * P->Ntot);
    const size_t o_qu = take(sizeof(unsigned long long) * 4);
    if (const char *fl = getenv("MPI_FAULT")) {
        if (strcmp(fl, "alloc") == 0) {
            set_error("plan allocation of %zu bytes failed (injected by MPI_FAULT=alloc)", tot);
            delete P;
            return MPI_ERR_NOMEM;
        }
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&P->dev), tot);
    if (e != cudaSuccess) {
        set_error("plan allocation of %zu bytes failed: %s", tot, cudaGetErrorString(e));
        P->dev = nullptr;
        free_plan(P);
        return e == cudaErrorMemoryAllocation ? MPI_ERR_NOMEM : MPI_ERR_CUDA;
    }
    P->dev_bytes = tot;
    char *d = P->dev;
    for (int f = 0; f < n_frames; ++f) {
        P->geo.push_back(geometry_carve<float>(d + o_geo[f], P->T[f], P->g[f].nx, P->g[f].ny));
        P->fwd_part.push_back(reinterpret_cast<float *>(d + o_fp[f]));
        P->adj_part.push_back(reinterpret_cast<float *>(d + o_ap[f]));
        P->sA.push_back(reinterpret_cast<float *>(d + o_sA[f]));
        P->pq.push_back(reinterpret_cast<double *>(d + o_pq[f]));
        P->rr0.push_back(reinterpret_cast<double *>(d + o_rr0[f]));
        P->rr1.push_back(reinterpret_cast<double *>(d + o_rr1[f]));
        P->scal.push_back(reinterpret_cast<double *>(d + o_sc[f]));
        P->done.push_back(reinterpret_cast<int *>(d + o_sc[f] + sizeof(double) * 8));
    }
    P->b0 = reinterpret_cast<double *>(d + o_b0);
    P->x = reinterpret_cast<double *>(d + o_x);
    P->r = reinterpret_cast<double *>(d + o_r);
    P->p = reinterpret_cast<double *>(d + o_p);
    P->q = reinterpret_cast<double *>(d + o_q);
    P->rho1 = reinterpret_cast<float *>(d + o_r1);
    P->rho2 = reinterpret_cast<float *>(d + o_r2);
    P->queues = reinterpret_cast<unsigned long long *>(d + o_qu);
    if (cudaMemset(P->dev, 0, tot) != cudaSuccess) {
        set_error("plan memset failed");
        free_plan(P);
        return MPI_ERR_CUDA;
    }
    // vector/stat/gauss tables (independent of the work-item split)
    P->vec.n = n_frames;
    P->stat.n = n_frames;
    P->stat.do_clip = P->clip_pct >= 0.0 ? 1 : 0;
    P->stat.pct = P->clip_pct;
    P->stat.final_parity = P->n_cg & 1;
    P->gauss.n = n_frames;
    double w[3];
    gauss5_weights(w);
    P->gauss.w0 = float(w[0]);
    P->gauss.w1 = float(w[1]);
    P->gauss.w2 = float(w[2]);
    int64_t b = 0;
    for (int f = 0; f < n_frames; ++f) {
        VecFrame V{};
        V.off = P->voff[f];
        V.N = P->N[f];
        V.blk0 = b;
        V.nblk = P->nvblk[f];
        V.n_pq = P->npq[f];
        V.pq = P->pq[f];
        V.rr[0] = P->rr0[f];
        V.rr[1] = P->rr1[f];
        V.done = P->done[f];
        V.scal = P->scal[f];
        P->vec.f[f] = V;
        P->stat.f[f] = V;
        P->stat.nu0[f] = P->nu0[f];
        P->gauss.f[f] = GaussFrame{P->voff[f], P->g[f].nx, P->g[f].ny};
        b += V.nblk;
    }
    P->vec_blocks_tot = b;
    configure(*P, kDefaultBudget, kDefaultBudget, false, false);
    const int pst = prepare_launch(*P);
    if (pst != MPI_OK) {
        free_plan(P);
        return pst;
    }
    if (!(flags & MPI_BATCH_AUTOTUNE)) P->tuned = true;
    *plan = P;
    return MPI_OK;
}

int mpi_batch_pnp_run(mpi_batch_plan *P, const void *const *r, const void *const *v,
                      const void *const *s, void *const *rho_out, void *stream)
{
    if (!P || !r || !v || !s || !rho_out) { set_error("NULL argument"); return MPI_ERR_INVALID; }
    for (int f = 0; f < P->n; ++f)
        if (!r[f] || !v[f] || !s[f] || !rho_out[f]) {
            set_error("frame %d: NULL array", f);
            return MPI_ERR_INVALID;
        }
    const cudaStream_t st = as_stream(stream);
    for (int f = 0; f < P->n; ++f) MPI_TRY(prepare_geometry<float>(P->m[f], P->g[f], P->T[f], r[f], v[f], P->geo[f], st));
    if (!P->tuned) {
        MPI_TRY(autotune(*P, st));
        if (P->exec) {  // the split changed: recapture
            cudaGraphExecDestroy(P->exec);
            cudaGraphDestroy(P->graph);
            P->exec = nullptr;
            P->graph = nullptr;
        }
    }
    // b0 = A^T s for every frame
    PairTab Bs = P->adj_tab;
    for (int f = 0; f < P->n; ++f) Bs.f[f].in = s[f];
    MPI_TRY(launch_adj_kernel(*P, Bs, st));
    RedTab Rb = P->red_adj[0];
    for (int f = 0; f < P->n; ++f) Rb.f[f].out = P->b0 + P->voff[f];
    k_reduce_batch<double, false><<<(unsigned)red_blocks(Rb), 256, 0, st>>>(Rb);
    MPI_CHECK_LAUNCH();
    MPI_TRY_CUDA(cudaMemsetAsync(P->rho2, 0, sizeof(float) * P->Ntot, st));
    k_init_b<<<(P->n + 63) / 64, 64, 0, st>>>(P->stat);
    MPI_CHECK_LAUNCH();
    if (P->n_iter > 0) {
        MPI_TRY(capture_iteration(*P));
        for (int k = 0; k < P->n_iter; ++k) {
            MPI_TRY_CUDA(cudaGraphLaunch(P->exec, st));
            note_launches((long long)P->graph_nodes);
        }
    }
    for (int f = 0; f < P->n; ++f)
        MPI_TRY_CUDA(cudaMemcpyAsync(rho_out[f], P->rho2 + P->voff[f], sizeof(float) * P->N[f],
                                     cudaMemcpyDeviceToDevice, st));
    return MPI_OK;
}

int mpi_batch_plan_info(const mpi_batch_plan *P, mpi_batch_info *info)
{
    if (!P || !info) { set_error("NULL argument"); return MPI_ERR_INVALID; }
    info->n_frames = P->n;
    info->tuned = P->tuned ? 1 : 0;
    info->item_pairs_forward = P->fwd_budget;
    info->item_pairs_adjoint = P->adj_budget;
    info->persistent_forward = P->fwd_persist ? 1 : 0;
    info->persistent_adjoint = P->adj_persist ? 1 : 0;
    info->forward_items = P->fwd_items;
    info->adjoint_items = P->adj_items;
    info->device_bytes = (long long)P->dev_bytes;
    info->graph_nodes = (long long)P->graph_nodes;
    return MPI_OK;
}

int mpi_batch_plan_destroy(mpi_batch_plan *plan)
{
    free_plan(plan);
    return MPI_OK;
}

}  // extern "C"
