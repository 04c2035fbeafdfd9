// Core Stage (Eq. first:step): cosine interpolation of the 4-component core
// operator at the trajectory samples, its exact transpose, the replicated-
// boundary Laplacian, and the CG solve of the Euler-Lagrange equations
//   ((1/T) M^T M + gamma Lap Lap) Ahat = (1/T) M^T s.
//
// The transpose is computed without float atomics: samples are binned by the
// interpolation cell they fall in (integer counts, a scan, a fill and a
// per-cell sort by sample index give every cell a fixed sample order), and
// each node gathers from its (up to) four adjacent cells.  All of it is
// memory/latency bound.
#include <algorithm>
#include <cmath>

#include "pnp_ops.cuh"

namespace mpi {

int check_grid(const mpi_grid_desc *g);
int check_traj(const mpi_traj *t);
int check_dtype(mpi_dtype d);
GridH to_host(const mpi_grid_desc *g);

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

static AxisMap make_axis(double p0, double h, int n)
{
    return AxisMap{1.0 / h, -p0 / h - 0.5, n};
}

// s[k][t] = sum_m I[Ahat_{2k+m}](r_t) v_m(t)   (Ahat of type AT, s of type R).
// CH < 0: both channels, Ahat has 4 components, s 2 rows.  CH = k: only
// channel k, Ahat holds (A_k0, A_k1) and s one row.
template <typename R, typename AT, int CH>
__global__ void k_interp(int64_t T, const R *__restrict__ r, const R *__restrict__ v,
                         const AT *__restrict__ A, AxisMap ax, AxisMap ay, R *__restrict__ s)
{
    const int nx = ax.n;
    const int64_t N = (int64_t)ax.n * ay.n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i0, j0;
        R wx0, wx1, wy0, wy1;
        axis_weights<R>(r[2 * t], ax, i0, wx0, wx1);
        axis_weights<R>(r[2 * t + 1], ay, j0, wy0, wy1);
        const int i1 = ax.n > 1 ? i0 + 1 : i0, j1 = ay.n > 1 ? j0 + 1 : j0;
        const R vx = v[2 * t], vy = v[2 * t + 1];
        constexpr int K = CH < 0 ? 2 : 1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            R acc = R(0);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const AT *F = A + (CH < 0 ? 2 * k + m : m) * N;
                const R val = wy0 * (wx0 * R(F[(int64_t)j0 * nx + i0]) + wx1 * R(F[(int64_t)j0 * nx + i1])) +
                              wy1 * (wx0 * R(F[(int64_t)j1 * nx + i0]) + wx1 * R(F[(int64_t)j1 * nx + i1]));
                acc += val * (m == 0 ? vx : vy);
            }
            s[(int64_t)k * T + t] = acc;
        }
    }
}

// --- binning of samples by interpolation cell -------------------------------

template <typename R>
__global__ void k_cell_count(int64_t T, const R *__restrict__ r, AxisMap ax, AxisMap ay, int ncx,
                             int *__restrict__ cell_of, int *__restrict__ count)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        int i0, j0;
        R w0, w1;
        axis_weights<R>(r[2 * t], ax, i0, w0, w1);
        axis_weights<R>(r[2 * t + 1], ay, j0, w0, w1);
        const int c = j0 * ncx + i0;
        cell_of[t] = c;
        atomicAdd(&count[c], 1);
    }
}

// Exclusive scan of n ints by one block (deterministic); also copies the
// offsets to `cursor`.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
k_scan(const int *__restrict__ count, int n, int *__restrict__ offset, int *__restrict__ cursor)
{
    __shared__ int sh[kScanThreads];
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int b0 = threadIdx.x * per, b1 = min(n, b0 + per);
    int local = 0;
    for (int k = b0; k < b1; ++k) local += count[k];
    sh[threadIdx.x] = local;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const int add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    int run = sh[threadIdx.x] - local;
    for (int k = b0; k < b1; ++k) {
        offset[k] = run;
        cursor[k] = run;
        run += count[k];
    }
    if (threadIdx.x == kScanThreads - 1) offset[n] = sh[kScanThreads - 1];
}

__global__ void k_cell_fill(int64_t T, const int *__restrict__ cell_of, int *__restrict__ cursor,
                            int *__restrict__ list)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x)
        list[atomicAdd(&cursor[cell_of[t]], 1)] = (int)t;
}

// Sort each cell's sample list ascending: insertion sort for short lists,
// heap sort (O(n log n), in place) for long ones.
__global__ void k_cell_sort(int n_cells, const int *__restrict__ offset, int *__restrict__ list)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    int *a = list + offset[c];
    const int n = offset[c + 1] - offset[c];
    if (n <= 32) {
        for (int i = 1; i < n; ++i) {
            const int key = a[i];
            int j = i - 1;
            while (j >= 0 && a[j] > key) { a[j + 1] = a[j]; --j; }
            a[j + 1] = key;
        }
        return;
    }
    auto sift = [&](int root, int end) {
        while (2 * root + 1 < end) {
            int child = 2 * root + 1;
            if (child + 1 < end && a[child] < a[child + 1]) ++child;
            if (a[root] >= a[child]) return;
            const int tmp = a[root]; a[root] = a[child]; a[child] = tmp;
            root = child;
        }
    };
    for (int s = n / 2 - 1; s >= 0; --s) sift(s, n);
    for (int end = n - 1; end > 0; --end) {
        const int tmp = a[0]; a[0] = a[end]; a[end] = tmp;
        sift(0, end);
    }
}

// Ahat_{2k+m}(node) = sum over samples t of the adjacent cells of
// w_node(t) v_m(t) s_k(t).  CH = k: only channel k (s one row), output the two
// components (A_k0, A_k1).
template <typename R, typename OUT, int CH>
__global__ void k_interp_T(const R *__restrict__ r, const R *__restrict__ v, const R *__restrict__ s,
                           int64_t T, AxisMap ax, AxisMap ay, int ncx, int ncy,
                           const int *__restrict__ offset, const int *__restrict__ list,
                           OUT *__restrict__ A, double scale)
{
    const int nx = ax.n, ny = ay.n;
    const int64_t N = (int64_t)nx * ny;
    constexpr int NC = CH < 0 ? 4 : 2;
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < N;
         node += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(node % nx), j = (int)(node / nx);
        R acc[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) acc[m] = R(0);
        for (int cj = j - 1; cj <= j; ++cj) {
            if (cj < 0 || cj >= ncy) continue;
            for (int ci = i - 1; ci <= i; ++ci) {
                if (ci < 0 || ci >= ncx) continue;
                const int c = cj * ncx + ci;
                for (int q = offset[c]; q < offset[c + 1]; ++q) {
                    const int64_t t = list[q];
                    int i0, j0;
                    R wx0, wx1, wy0, wy1;
                    axis_weights<R>(r[2 * t], ax, i0, wx0, wx1);
                    axis_weights<R>(r[2 * t + 1], ay, j0, wy0, wy1);
                    const R wx = (i == i0) ? wx0 : wx1;
                    const R wy = (j == j0) ? wy0 : wy1;
                    const R w = wy * wx;
                    const R vx = v[2 * t], vy = v[2 * t + 1];
                    if constexpr (CH < 0) {
                        const R s0 = s[t], s1 = s[T + t];
                        acc[0] += w * (vx * s0);
                        acc[1] += w * (vy * s0);
                        acc[2] += w * (vx * s1);
                        acc[3] += w * (vy * s1);
                    } else {
                        const R sk = s[t];
                        acc[0] += w * (vx * sk);
                        acc[1] += w * (vy * sk);
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) A[m * N + node] = OUT(double(acc[m]) * scale);
    }
}

// Binning scratch for a trajectory on a grid.
struct Bins {
    int *cell_of, *count, *offset, *cursor, *list;
    int ncx, ncy;
};

static size_t bins_bytes(int64_t T, int nx, int ny)
{
    const size_t nc = size_t(std::max(nx - 1, 1)) * std::max(ny - 1, 1);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    return up(sizeof(int) * std::max<int64_t>(T, 1)) * 2 + up(sizeof(int) * nc) * 2 +
           up(sizeof(int) * (nc + 1));
}

static Bins bins_carve(char *p, int64_t T, int nx, int ny)
{
    Bins b;
    b.ncx = std::max(nx - 1, 1);
    b.ncy = std::max(ny - 1, 1);
    const size_t nc = size_t(b.ncx) * b.ncy;
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    b.cell_of = reinterpret_cast<int *>(p); p += up(sizeof(int) * std::max<int64_t>(T, 1));
    b.list = reinterpret_cast<int *>(p); p += up(sizeof(int) * std::max<int64_t>(T, 1));
    b.count = reinterpret_cast<int *>(p); p += up(sizeof(int) * nc);
    b.cursor = reinterpret_cast<int *>(p); p += up(sizeof(int) * nc);
    b.offset = reinterpret_cast<int *>(p);
    return b;
}

static int grid_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

template <typename R>
static int build_bins(const GridH &g, int64_t T, const R *r, const Bins &b, cudaStream_t st)
{
    const AxisMap ax = make_axis(g.x0, g.dx, g.nx), ay = make_axis(g.y0, g.dy, g.ny);
    const int nc = b.ncx * b.ncy;
    MPI_TRY_CUDA(cudaMemsetAsync(b.count, 0, sizeof(int) * nc, st));
    if (T > 0) {
        k_cell_count<R><<<grid_blocks(T), 256, 0, st>>>(T, r, ax, ay, b.ncx, b.cell_of, b.count);
        MPI_CHECK_LAUNCH();
    }
    k_scan<<<1, kScanThreads, 0, st>>>(b.count, nc, b.offset, b.cursor);
    MPI_CHECK_LAUNCH();
    if (T > 0) {
        k_cell_fill<<<grid_blocks(T), 256, 0, st>>>(T, b.cell_of, b.cursor, b.list);
        MPI_CHECK_LAUNCH();
        k_cell_sort<<<(nc + 127) / 128, 128, 0, st>>>(nc, b.offset, b.list);
        MPI_CHECK_LAUNCH();
    }
    return MPI_OK;
}

template <typename R, typename AT>
static int launch_interp(const GridH &g, int64_t T, const R *r, const R *v, const AT *A, R *s,
                         cudaStream_t st, int ch = -1)
{
    if (T == 0) return MPI_OK;
    const AxisMap ax = make_axis(g.x0, g.dx, g.nx), ay = make_axis(g.y0, g.dy, g.ny);
    if (ch < 0) k_interp<R, AT, -1><<<grid_blocks(T), 256, 0, st>>>(T, r, v, A, ax, ay, s);
    else if (ch == 0) k_interp<R, AT, 0><<<grid_blocks(T), 256, 0, st>>>(T, r, v, A, ax, ay, s);
    else k_interp<R, AT, 1><<<grid_blocks(T), 256, 0, st>>>(T, r, v, A, ax, ay, s);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename R, typename OUT>
static int launch_interp_T(const GridH &g, int64_t T, const R *r, const R *v, const R *s,
                           const Bins &b, OUT *A, double scale, cudaStream_t st, int ch = -1)
{
    const AxisMap ax = make_axis(g.x0, g.dx, g.nx), ay = make_axis(g.y0, g.dy, g.ny);
    const int64_t N = (int64_t)g.nx * g.ny;
    if (ch < 0)
        k_interp_T<R, OUT, -1><<<grid_blocks(N), 256, 0, st>>>(r, v, s, T, ax, ay, b.ncx, b.ncy, b.offset,
                                                              b.list, A, scale);
    else
        k_interp_T<R, OUT, 0><<<grid_blocks(N), 256, 0, st>>>(r, v, s, T, ax, ay, b.ncx, b.ncy, b.offset,
                                                             b.list, A, scale);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// --- Laplacian and the Core Stage operator ---------------------------------

// out_m = Lap x_m for the nc components (replicated boundary), FP64.
__global__ void k_lap(int nx, int ny, int nc, const double *__restrict__ x, double *__restrict__ out)
{
    const int64_t N = (int64_t)nx * ny;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / N, k = e % N;
        const int i = (int)(k % nx), j = (int)(k / nx);
        const double *f = x + m * N;
        const int im = i > 0 ? i - 1 : 0, ip = i < nx - 1 ? i + 1 : nx - 1;
        const int jm = j > 0 ? j - 1 : 0, jp = j < ny - 1 ? j + 1 : ny - 1;
        out[e] = f[(int64_t)j * nx + im] + f[(int64_t)j * nx + ip] + f[(int64_t)jm * nx + i] +
                 f[(int64_t)jp * nx + i] - 4.0 * f[k];
    }
}

// q = y + gamma lap2, partial sums of <p, q> (blocks of 2048 elements).
constexpr int kEpiThreads = 256, kEpiPer = 2048;
__global__ void __launch_bounds__(kEpiThreads)
k_grid_epilogue(int64_t n, const double *__restrict__ y, const double *__restrict__ lap2, double gamma,
                const double *__restrict__ p, double *__restrict__ q, double *__restrict__ dot_part)
{
    __shared__ double sh[kEpiThreads / 32];
    const int64_t e0 = (int64_t)blockIdx.x * kEpiPer, e1 = min(n, e0 + kEpiPer);
    double acc = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kEpiThreads) {
        const double qe = y[e] + gamma * lap2[e];
        q[e] = qe;
        acc += p[e] * qe;
    }
    acc = block_sum<double, kEpiThreads>(acc, sh);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = acc;
}

__global__ void k_norm_thresh(const double *__restrict__ part, int n, double tol, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0;
        for (int k = 0; k < n; ++k) a += part[k];
        out[0] = sqrt(a);
        out[1] = tol > 0.0 ? tol * sqrt(a) : -1.0;
    }
}

// Ahat and its trace (both channels: A_00 + A_11; one channel k: A_kk,
// which is component k of the stored pair (A_k0, A_k1)).
template <typename R>
__global__ void k_grid_output(int64_t N, int ch, const double *__restrict__ x, R *__restrict__ A,
                              R *__restrict__ tr)
{
    const int nc = ch < 0 ? 4 : 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int m = 0; m < nc; ++m) A[m * N + e] = R(x[m * N + e]);
        tr[e] = ch < 0 ? R(x[e] + x[3 * N + e]) : R(x[ch * N + e]);
    }
}

template <typename R>
static int grid_impl(const GridH &g, const mpi_traj *tr, const void *s_in, const mpi_grid_opts &o,
                     void *Ahat, void *trace, int *n_iter_out, cudaStream_t st)
{
    const int64_t T = tr->T;
    const int ch = o.channel - 1;  // -1: both channels; 0 / 1: that channel only
    const int nc = ch < 0 ? 4 : 2;
    const int64_t N = (int64_t)g.nx * g.ny, n4 = nc * N;
    const int nblk = vec_blocks(n4);
    const R *r = static_cast<const R *>(tr->r), *v = static_cast<const R *>(tr->v);
    const R *s = static_cast<const R *>(s_in);

    Scratch scr(st);
    const size_t o_bins = scr.reserve(bins_bytes(T, g.nx, g.ny));
    const size_t o_s = scr.reserve(sizeof(R) * (ch < 0 ? 2 : 1) * std::max<int64_t>(T, 1));
    const size_t vb = sizeof(double) * n4;
    const size_t o_b = scr.reserve(vb), o_x = scr.reserve(vb), o_r = scr.reserve(vb),
                 o_p = scr.reserve(vb), o_q = scr.reserve(vb), o_y = scr.reserve(vb),
                 o_l1 = scr.reserve(vb), o_l2 = scr.reserve(vb);
    const size_t o_parts = scr.reserve(sizeof(double) * 3 * nblk);
    const size_t o_sc = scr.reserve(sizeof(double) * 8 + sizeof(int) * 8);
    MPI_TRY(scr.allocate());
    const Bins bins = bins_carve(scr.at<char>(o_bins), T, g.nx, g.ny);
    R *s_tmp = scr.at<R>(o_s);
    double *b = scr.at<double>(o_b), *x = scr.at<double>(o_x), *rr = scr.at<double>(o_r),
           *p = scr.at<double>(o_p), *q = scr.at<double>(o_q), *y = scr.at<double>(o_y),
           *l1 = scr.at<double>(o_l1), *l2 = scr.at<double>(o_l2);
    double *pq_part = scr.at<double>(o_parts), *rr_part0 = pq_part + nblk, *rr_part1 = pq_part + 2 * nblk;
    double *scal = scr.at<double>(o_sc);
    int *done = reinterpret_cast<int *>(scal + 8), *iters = done + 1;

    MPI_TRY(build_bins<R>(g, T, r, bins, st));
    const double invT = T > 0 ? 1.0 / double(T) : 0.0;
    // b = (1/T) M^T s
    MPI_TRY((launch_interp_T<R, double>(g, T, r, v, s, bins, b, invT, st, ch)));
    MPI_TRY_CUDA(cudaMemsetAsync(x, 0, vb, st));
    MPI_TRY_CUDA(cudaMemsetAsync(q, 0, vb, st));
    MPI_TRY_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 8 + sizeof(int) * 8, st));
    // r = b, p = b, rr partials (nu = 0 from the zeroed scalar block)
    MPI_TRY(cg_init_launch(n4, b, x, q, scal, rr, p, rr_part0, done, st));
    k_norm_thresh<<<1, 32, 0, st>>>(rr_part0, nblk, o.rel_tol, scal + kScalBnorm);
    MPI_CHECK_LAUNCH();
    const double *thresh = o.rel_tol > 0.0 ? scal + kScalTol : nullptr;

    int *h_done = nullptr;
    MPI_TRY_CUDA(cudaMallocHost(reinterpret_cast<void **>(&h_done), sizeof(int)));
    struct PinnedFree {
        int *p;
        ~PinnedFree() { cudaFreeHost(p); }
    } guard{h_done};

    const int lap_grid = grid_blocks(n4);
    const int poll = 16;
    for (int it = 0; it < o.max_iter; ++it) {
        // q = (1/T) M^T M p + gamma Lap Lap p
        MPI_TRY((launch_interp<R, double>(g, T, r, v, p, s_tmp, st, ch)));
        MPI_TRY((launch_interp_T<R, double>(g, T, r, v, s_tmp, bins, y, invT, st, ch)));
        k_lap<<<lap_grid, 256, 0, st>>>(g.nx, g.ny, nc, p, l1);
        MPI_CHECK_LAUNCH();
        k_lap<<<lap_grid, 256, 0, st>>>(g.nx, g.ny, nc, l1, l2);
        MPI_CHECK_LAUNCH();
        k_grid_epilogue<<<nblk, kEpiThreads, 0, st>>>(n4, y, l2, o.gamma, p, q, pq_part);
        MPI_CHECK_LAUNCH();
        MPI_TRY(cg_step_launch(n4, x, rr, p, q, pq_part, nblk, (it & 1) ? rr_part1 : rr_part0,
                               (it & 1) ? rr_part0 : rr_part1, done, thresh, iters, st));
        if (thresh && (it + 1) % poll == 0 && it + 1 < o.max_iter) {
            MPI_TRY_CUDA(cudaMemcpyAsync(h_done, done, sizeof(int), cudaMemcpyDeviceToHost, st));
            MPI_TRY_CUDA(cudaStreamSynchronize(st));
            if (*h_done) break;
        }
    }
    const int vgrid = grid_blocks(N);
    k_grid_output<R><<<vgrid, 256, 0, st>>>(N, ch, x, static_cast<R *>(Ahat), static_cast<R *>(trace));
    MPI_CHECK_LAUNCH();
    if (n_iter_out) {
        int hi = 0;
        MPI_TRY_CUDA(cudaMemcpyAsync(h_done, iters, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPI_TRY_CUDA(cudaStreamSynchronize(st));
        hi = *h_done;
        *n_iter_out = hi;
    }
    return MPI_OK;
}

template <typename R>
static int interp_impl(const GridH &g, const mpi_traj *tr, const void *A, void *s, cudaStream_t st)
{
    return launch_interp<R, R>(g, tr->T, static_cast<const R *>(tr->r), static_cast<const R *>(tr->v),
                               static_cast<const R *>(A), static_cast<R *>(s), st);
}

template <typename R>
static int interp_T_impl(const GridH &g, const mpi_traj *tr, const void *s, void *A, cudaStream_t st)
{
    const int64_t T = tr->T;
    Scratch scr(st);
    const size_t o_bins = scr.reserve(bins_bytes(T, g.nx, g.ny));
    MPI_TRY(scr.allocate());
    const Bins bins = bins_carve(scr.at<char>(o_bins), T, g.nx, g.ny);
    MPI_TRY(build_bins<R>(g, T, static_cast<const R *>(tr->r), bins, st));
    return launch_interp_T<R, R>(g, T, static_cast<const R *>(tr->r), static_cast<const R *>(tr->v),
                                 static_cast<const R *>(s), bins, static_cast<R *>(A), 1.0, st);
}

static int check_interp_args(const mpi_grid_desc *grid, const mpi_traj *traj, mpi_dtype dtype)
{
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (traj->T >= ((int64_t)1 << 31)) {
        set_error("interpolation supports T < 2^31");
        return MPI_ERR_UNSUPPORTED;
    }
    return MPI_OK;
}

}  // namespace mpi

using namespace mpi;

extern "C" {

int mpi_interp(const mpi_grid_desc *grid, const mpi_traj *traj, mpi_dtype dtype, const void *Ahat,
               void *s, void *stream)
{
    MPI_TRY(check_interp_args(grid, traj, dtype));
    if (!Ahat || (traj->T > 0 && !s)) { set_error("Ahat or s is NULL"); return MPI_ERR_INVALID; }
    const GridH g = to_host(grid);
    return dtype == MPI_F32 ? interp_impl<float>(g, traj, Ahat, s, as_stream(stream))
                            : interp_impl<double>(g, traj, Ahat, s, as_stream(stream));
}

int mpi_interp_adjoint(const mpi_grid_desc *grid, const mpi_traj *traj, mpi_dtype dtype,
                       const void *s, void *Ahat, void *stream)
{
    MPI_TRY(check_interp_args(grid, traj, dtype));
    if (!Ahat || (traj->T > 0 && !s)) { set_error("Ahat or s is NULL"); return MPI_ERR_INVALID; }
    const GridH g = to_host(grid);
    return dtype == MPI_F32 ? interp_T_impl<float>(g, traj, s, Ahat, as_stream(stream))
                            : interp_T_impl<double>(g, traj, s, Ahat, as_stream(stream));
}

int mpi_grid(const mpi_grid_desc *grid, const mpi_traj *traj, mpi_dtype dtype, const void *s,
             const mpi_grid_opts *opts, void *Ahat, void *trace, int *n_iter_out, void *stream)
{
    MPI_TRY(check_interp_args(grid, traj, dtype));
    if (!opts || !(opts->gamma >= 0.0) || !std::isfinite(opts->gamma) || opts->max_iter < 0 ||
        std::isnan(opts->rel_tol) || opts->channel < 0 || opts->channel > 2) {
        set_error("invalid Core Stage options");
        return MPI_ERR_INVALID;
    }
    if (!Ahat || !trace || (traj->T > 0 && !s)) { set_error("s, Ahat or trace is NULL"); return MPI_ERR_INVALID; }
    const GridH g = to_host(grid);
    return dtype == MPI_F32
               ? grid_impl<float>(g, traj, s, *opts, Ahat, trace, n_iter_out, as_stream(stream))
               : grid_impl<double>(g, traj, s, *opts, Ahat, trace, n_iter_out, as_stream(stream));
}

}  // extern "C"
