// Core Stage in three dimensions (Eq. first:step with n = 3): the core
// operator at a point is the 3 x 3 matrix Ahat_km (receive channel k, velocity
// component m), measured through the tensor-product cosine interpolation
//   s_k(t) = sum_m I[Ahat_km](r_t) v_m(t),
// and recovered by CG on ((1/T) M^T M + gamma Lap Lap) Ahat = (1/T) M^T s with
// the 7-point replicated-boundary Laplacian on each component.
//
// Same organisation as the 2-D solve: interpolation records computed once per
// trajectory, samples binned by interpolation cell (a cell now has 8 corner
// nodes, a node up to 8 adjacent cells), the transpose gathered per node in
// work units of at most kUnitLen samples with an ordered combine (no float
// atomics, run-to-run identical), CG vectors and inner products in FP64.
#include "grid_common.cuh"

namespace mpi {

int check_traj(const mpi_traj *t);
int check_dtype(mpi_dtype d);
int check_grid3(const mpi_grid3_desc *g);

namespace {

struct G3 {
    int nx, ny, nz;
    double x0, y0, z0, dx, dy, dz;
    int64_t n() const { return (int64_t)nx * ny * nz; }
};

// Interpolation record of one sample: its cell (i0, j0, l0) and the upper-node
// cosine weights along x, y and z (the lower ones are 1 - w).
template <typename R>
struct InterpRec3 {
    int i0, j0, l0;
    R wx1, wy1, wz1;
};

struct Axes3 {
    AxisMap x, y, z;
};

template <typename R>
__device__ __forceinline__ InterpRec3<R> make_rec3(R px, R py, R pz, const Axes3 &a)
{
    InterpRec3<R> q;
    R w0;
    axis_weights<R>(px, a.x, q.i0, w0, q.wx1);
    axis_weights<R>(py, a.y, q.j0, w0, q.wy1);
    axis_weights<R>(pz, a.z, q.l0, w0, q.wz1);
    return q;
}

// s[k][t] = sum_m I[Ahat_{3k+m}](r_t) v_m(t).  CH < 0: all three channels
// (Ahat 9 components, s 3 rows); CH = k: channel k only (Ahat holds
// (A_k0, A_k1, A_k2), s one row).  PRE: records precomputed (rec), else formed
// from r.  kInterpSPT samples per thread, a block apart.
template <typename R, typename AT, int CH, bool PRE>
__global__ void __launch_bounds__(256)
k_interp3(int64_t T, const R *__restrict__ r, const InterpRec3<R> *__restrict__ rec,
          const R *__restrict__ v, const AT *__restrict__ A, Axes3 ax, R *__restrict__ s)
{
    const int nx = ax.x.n, ny = ax.y.n;
    const int64_t N = (int64_t)nx * ny * ax.z.n;
    constexpr int K = CH < 0 ? 3 : 1;
    const int64_t span = (int64_t)blockDim.x * kInterpSPT;
    for (int64_t base = blockIdx.x * span + threadIdx.x; base < T; base += (int64_t)gridDim.x * span) {
        InterpRec3<R> q[kInterpSPT];
        R vv[kInterpSPT][3];
#pragma unroll
        for (int u = 0; u < kInterpSPT; ++u) {
            const int64_t t = min(base + u * (int64_t)blockDim.x, T - 1);
            if constexpr (PRE) q[u] = rec[t];
            else q[u] = make_rec3<R>(r[3 * t], r[3 * t + 1], r[3 * t + 2], ax);
#pragma unroll
            for (int m = 0; m < 3; ++m) vv[u][m] = v[3 * t + m];
        }
#pragma unroll
        for (int u = 0; u < kInterpSPT; ++u) {
            const int64_t t = base + u * (int64_t)blockDim.x;
            const int i0 = q[u].i0, j0 = q[u].j0, l0 = q[u].l0;
            const int i1 = nx > 1 ? i0 + 1 : i0, j1 = ny > 1 ? j0 + 1 : j0, l1 = ax.z.n > 1 ? l0 + 1 : l0;
            const R wx1 = q[u].wx1, wy1 = q[u].wy1, wz1 = q[u].wz1;
            const R wx0 = R(1) - wx1, wy0 = R(1) - wy1, wz0 = R(1) - wz1;
            const int64_t r00 = ((int64_t)l0 * ny + j0) * nx, r01 = ((int64_t)l0 * ny + j1) * nx;
            const int64_t r10 = ((int64_t)l1 * ny + j0) * nx, r11 = ((int64_t)l1 * ny + j1) * nx;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                R acc = R(0);
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const AT *F = A + (CH < 0 ? 3 * k + m : m) * N;
                    const R lo = wy0 * (wx0 * R(F[r00 + i0]) + wx1 * R(F[r00 + i1])) +
                                 wy1 * (wx0 * R(F[r01 + i0]) + wx1 * R(F[r01 + i1]));
                    const R hi = wy0 * (wx0 * R(F[r10 + i0]) + wx1 * R(F[r10 + i1])) +
                                 wy1 * (wx0 * R(F[r11 + i0]) + wx1 * R(F[r11 + i1]));
                    acc += (wz0 * lo + wz1 * hi) * vv[u][m];
                }
                if (t < T) s[(int64_t)k * T + t] = acc;
            }
        }
    }
}

template <typename R>
__global__ void k_cell_count3(int64_t T, const R *__restrict__ r, Axes3 ax, int ncx, int ncy,
                              int *__restrict__ cell_of, int *__restrict__ count, InterpRec3<R> *__restrict__ rec)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const InterpRec3<R> q = make_rec3<R>(r[3 * t], r[3 * t + 1], r[3 * t + 2], ax);
        rec[t] = q;
        const int c = (q.l0 * ncy + q.j0) * ncx + q.i0;
        cell_of[t] = c;
        atomicAdd(&count[c], 1);
    }
}

// Calls f(cell) for the (up to) eight cells around node (i, j, l), in
// ascending cell order.
template <typename F>
__device__ __forceinline__ void for_node_cells3(int i, int j, int l, int ncx, int ncy, int ncz, F &&f)
{
    for (int cl = max(l - 1, 0); cl <= min(l, ncz - 1); ++cl)
        for (int cj = max(j - 1, 0); cj <= min(j, ncy - 1); ++cj)
            for (int ci = max(i - 1, 0); ci <= min(i, ncx - 1); ++ci) f((cl * ncy + cj) * ncx + ci);
}

__global__ void k_unit_count3(int nx, int ny, int nz, int ncx, int ncy, int ncz, const int *__restrict__ offset,
                              int *__restrict__ unit_cnt)
{
    const int N = nx * ny * nz;
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N; node += gridDim.x * blockDim.x) {
        const int i = node % nx, j = (node / nx) % ny, l = node / (nx * ny);
        int tot = 0;
        for_node_cells3(i, j, l, ncx, ncy, ncz, [&](int c) { tot += offset[c + 1] - offset[c]; });
        unit_cnt[node] = max(1, (tot + kUnitLen - 1) / kUnitLen);
    }
}

// Partial sums of one work unit: sum over its entries of w_node(t) v_m(t)
// s_k(t) (records, velocities and s in list order).  CH < 0: 9 sums; CH = k:
// channel k only (s one row), 3 sums.  n_iter: the unit bound rounded up to
// whole blocks, so every warp runs the same iterations and its shuffles see
// full warps.
template <typename R, int CH>
__global__ void __launch_bounds__(kUnitThreads)
k_interp3_T_units(const InterpRec3<R> *__restrict__ rec, const R *__restrict__ vs, const R *__restrict__ s,
                  int64_t T, int nx, int ny, int ncx, int ncy, int ncz, const int *__restrict__ offset,
                  const int *__restrict__ unit_off, const int *__restrict__ unit_node, int N, int n_iter,
                  R *__restrict__ unit_part)
{
    constexpr int NC = CH < 0 ? 9 : 3;
    constexpr int G = kUnitLanes;
    constexpr int per_block = kUnitThreads / G;
    const int sub = threadIdx.x % G;
    const int n_units = unit_off[N];
    for (int base = blockIdx.x * per_block; base < n_iter; base += gridDim.x * per_block) {
        const int w = base + (int)threadIdx.x / G;
        R acc[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) acc[m] = R(0);
        if (w < n_units) {
            const int node = unit_node[w];
            const int i = node % nx, j = (node / nx) % ny, l = node / (nx * ny);
            const int p0 = (w - unit_off[node]) * kUnitLen, p1 = p0 + kUnitLen;
            int pos = 0;
            for_node_cells3(i, j, l, ncx, ncy, ncz, [&](int c) {
                const int q_base = offset[c], cnt = offset[c + 1] - q_base;
                const int lo = max(p0, pos), hi = min(p1, pos + cnt);
#pragma unroll 2
                for (int pp = lo + sub; pp < hi; pp += G) {
                    const int q = q_base + (pp - pos);
                    const InterpRec3<R> rc = rec[q];
                    const R wx = (i == rc.i0) ? R(1) - rc.wx1 : rc.wx1;
                    const R wy = (j == rc.j0) ? R(1) - rc.wy1 : rc.wy1;
                    const R wz = (l == rc.l0) ? R(1) - rc.wz1 : rc.wz1;
                    const R wt = wz * (wy * wx);
                    const R v0 = vs[3 * q], v1 = vs[3 * q + 1], v2 = vs[3 * q + 2];
                    if constexpr (CH < 0) {
#pragma unroll
                        for (int kk = 0; kk < 3; ++kk) {
                            const R sk = wt * s[(int64_t)kk * T + q];
                            acc[3 * kk] += v0 * sk;
                            acc[3 * kk + 1] += v1 * sk;
                            acc[3 * kk + 2] += v2 * sk;
                        }
                    } else {
                        const R sk = wt * s[q];
                        acc[0] += v0 * sk;
                        acc[1] += v1 * sk;
                        acc[2] += v2 * sk;
                    }
                }
                pos += cnt;
            });
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) {
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
        }
        if (sub == 0 && w < n_units) {
#pragma unroll
            for (int m = 0; m < NC; ++m) unit_part[(int64_t)w * NC + m] = acc[m];
        }
    }
}

// out_m = Lap x_m (7-point, replicated boundary) for the nc components, FP64.
// scaled: per-axis second differences with 1/dx^2, 1/dy^2, 1/dz^2 (c).
__global__ void k_lap3(int nx, int ny, int nz, int nc, bool scaled, double3 c, const double *__restrict__ x,
                       double *__restrict__ out)
{
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e / N, k = e % N;
        const int i = (int)(k % nx), j = (int)((k / nx) % ny), l = (int)(k / ((int64_t)nx * ny));
        const double *f = x + m * N;
        const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
        const int64_t xm = i > 0 ? -sx : 0, xp = i < nx - 1 ? sx : 0;
        const int64_t ym = j > 0 ? -sy : 0, yp = j < ny - 1 ? sy : 0;
        const int64_t zm = l > 0 ? -sz : 0, zp = l < nz - 1 ? sz : 0;
        if (scaled) {
            const double c0 = f[k];
            out[e] = c.x * (f[k + xm] - 2.0 * c0 + f[k + xp]) + c.y * (f[k + ym] - 2.0 * c0 + f[k + yp]) +
                     c.z * (f[k + zm] - 2.0 * c0 + f[k + zp]);
        } else {
            out[e] = f[k + xm] + f[k + xp] + f[k + ym] + f[k + yp] + f[k + zm] + f[k + zp] - 6.0 * f[k];
        }
    }
}

// Ahat and its trace (all channels: A_00 + A_11 + A_22; channel k: A_kk,
// component k of the stored row (A_k0, A_k1, A_k2)).
template <typename R>
__global__ void k_grid3_output(int64_t N, int ch, const double *__restrict__ x, R *__restrict__ A,
                               R *__restrict__ tr)
{
    const int nc = ch < 0 ? 9 : 3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int m = 0; m < nc; ++m) A[m * N + e] = R(x[m * N + e]);
        tr[e] = ch < 0 ? R(x[e] + x[4 * N + e] + x[8 * N + e]) : R(x[ch * N + e]);
    }
}

// Binning scratch: as the 2-D one, with 3-D records and velocities.
struct Bins3 {
    int *cell_of, *count, *offset, *cursor, *list;
    void *rec_t, *rec, *vs;
    int *unit_cnt, *unit_off, *unit_cursor, *unit_node;
    void *unit_part;
    int n_units_max;
    int ncx, ncy, ncz;
};

inline size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

int units_bound3(int64_t T, int64_t N)
{
    // Every sample lies in one cell and so in the runs of at most 8 nodes.
    return (int)std::min<int64_t>(INT32_MAX, N + (8 * T + kUnitLen - 1) / kUnitLen + 1);
}

template <typename R>
size_t bins3_bytes(int64_t T, const G3 &g)
{
    const size_t nc = size_t(std::max(g.nx - 1, 1)) * std::max(g.ny - 1, 1) * std::max(g.nz - 1, 1);
    const size_t N = size_t(g.n()), U = size_t(units_bound3(T, g.n()));
    const size_t T1 = size_t(std::max<int64_t>(T, 1));
    return up256(sizeof(int) * T1) * 2 + up256(sizeof(int) * nc) * 2 + up256(sizeof(int) * (nc + 1)) +
           2 * up256(sizeof(InterpRec3<R>) * T1) + up256(3 * sizeof(R) * T1) + up256(sizeof(int) * N) * 2 +
           up256(sizeof(int) * (N + 1)) + up256(sizeof(int) * U) + up256(9 * sizeof(R) * U);
}

template <typename R>
Bins3 bins3_carve(char *p, int64_t T, const G3 &g)
{
    Bins3 b;
    b.ncx = std::max(g.nx - 1, 1);
    b.ncy = std::max(g.ny - 1, 1);
    b.ncz = std::max(g.nz - 1, 1);
    const size_t nc = size_t(b.ncx) * b.ncy * b.ncz;
    const size_t T1 = size_t(std::max<int64_t>(T, 1));
    b.cell_of = reinterpret_cast<int *>(p); p += up256(sizeof(int) * T1);
    b.list = reinterpret_cast<int *>(p); p += up256(sizeof(int) * T1);
    b.count = reinterpret_cast<int *>(p); p += up256(sizeof(int) * nc);
    b.cursor = reinterpret_cast<int *>(p); p += up256(sizeof(int) * nc);
    b.offset = reinterpret_cast<int *>(p); p += up256(sizeof(int) * (nc + 1));
    b.rec_t = p; p += up256(sizeof(InterpRec3<R>) * T1);
    b.rec = p; p += up256(sizeof(InterpRec3<R>) * T1);
    b.vs = p; p += up256(3 * sizeof(R) * T1);
    const size_t N = size_t(g.n());
    b.n_units_max = units_bound3(T, g.n());
    b.unit_cnt = reinterpret_cast<int *>(p); p += up256(sizeof(int) * N);
    b.unit_cursor = reinterpret_cast<int *>(p); p += up256(sizeof(int) * N);
    b.unit_off = reinterpret_cast<int *>(p); p += up256(sizeof(int) * (N + 1));
    b.unit_node = reinterpret_cast<int *>(p); p += up256(sizeof(int) * size_t(b.n_units_max));
    b.unit_part = p;
    return b;
}

Axes3 axes_of(const G3 &g)
{
    return Axes3{make_axis(g.x0, g.dx, g.nx), make_axis(g.y0, g.dy, g.ny), make_axis(g.z0, g.dz, g.nz)};
}

template <typename R>
int build_bins3(const G3 &g, int64_t T, const R *r, const R *v, const Bins3 &b, cudaStream_t st)
{
    const Axes3 ax = axes_of(g);
    const int nc = b.ncx * b.ncy * b.ncz;
    MPI_TRY_CUDA(cudaMemsetAsync(b.count, 0, sizeof(int) * nc, st));
    if (T > 0) {
        k_cell_count3<R><<<grid_blocks(T), 256, 0, st>>>(T, r, ax, b.ncx, b.ncy, b.cell_of, b.count,
                                                          static_cast<InterpRec3<R> *>(b.rec_t));
        MPI_CHECK_LAUNCH();
    }
    MPI_TRY(cell_scan_launch(b.count, nc, b.offset, b.cursor, st));
    if (T > 0) {
        MPI_TRY(cell_fill_launch(T, b.cell_of, b.cursor, b.list, st));
        MPI_TRY(cell_sort_launch(nc, b.offset, b.list, st));
        k_sort_records<InterpRec3<R>, R, 3><<<grid_blocks(T), 256, 0, st>>>(
            T, b.list, static_cast<const InterpRec3<R> *>(b.rec_t), v, static_cast<InterpRec3<R> *>(b.rec),
            static_cast<R *>(b.vs));
        MPI_CHECK_LAUNCH();
    }
    const int N = (int)g.n();
    k_unit_count3<<<grid_blocks(N), 256, 0, st>>>(g.nx, g.ny, g.nz, b.ncx, b.ncy, b.ncz, b.offset, b.unit_cnt);
    MPI_CHECK_LAUNCH();
    MPI_TRY(cell_scan_launch(b.unit_cnt, N, b.unit_off, b.unit_cursor, st));
    return unit_fill_launch(N, b.unit_off, b.unit_node, st);
}

template <typename R, typename AT>
int launch_interp3(const G3 &g, int64_t T, const R *r, const R *v, const AT *A, R *s, cudaStream_t st,
                   int ch = -1, const InterpRec3<R> *rec = nullptr)
{
    if (T == 0) return MPI_OK;
    const Axes3 ax = axes_of(g);
    const int blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>((T + 256 * kInterpSPT - 1) / (256 * kInterpSPT), 8192));
    if (rec) {
        if (ch < 0) k_interp3<R, AT, -1, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, s);
        else k_interp3<R, AT, 0, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, s);
    } else {
        if (ch < 0) k_interp3<R, AT, -1, false><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, s);
        else k_interp3<R, AT, 0, false><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, s);
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// s_sorted: the samples' values in list order ([rows][T]).
template <typename R, typename OUT>
int launch_interp3_T(const G3 &g, int64_t T, const R *s_sorted, const Bins3 &b, OUT *A, double scale,
                     cudaStream_t st, int ch = -1)
{
    const int N = (int)g.n();
    constexpr int per_block = kUnitThreads / kUnitLanes;
    const int n_iter = (b.n_units_max + per_block - 1) / per_block * per_block;
    const unsigned blocks = (unsigned)std::max(1, std::min(n_iter / per_block, 65535));
    const InterpRec3<R> *rec = static_cast<const InterpRec3<R> *>(b.rec);
    const R *vs = static_cast<const R *>(b.vs);
    R *part = static_cast<R *>(b.unit_part);
    if (ch < 0)
        k_interp3_T_units<R, -1><<<blocks, kUnitThreads, 0, st>>>(rec, vs, s_sorted, T, g.nx, g.ny, b.ncx, b.ncy,
                                                                  b.ncz, b.offset, b.unit_off, b.unit_node, N,
                                                                  n_iter, part);
    else
        k_interp3_T_units<R, 0><<<blocks, kUnitThreads, 0, st>>>(rec, vs, s_sorted, T, g.nx, g.ny, b.ncx, b.ncy,
                                                                 b.ncz, b.offset, b.unit_off, b.unit_node, N,
                                                                 n_iter, part);
    MPI_CHECK_LAUNCH();
    if (ch < 0) k_interp_T_combine<R, OUT, 9><<<grid_blocks(N), 256, 0, st>>>(N, b.unit_off, part, A, scale);
    else k_interp_T_combine<R, OUT, 3><<<grid_blocks(N), 256, 0, st>>>(N, b.unit_off, part, A, scale);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// The 3-D Core Stage operator: (1/T) M^T M through the binned records and
// the 7-point Laplacian of each component.
template <typename R>
struct GridOp3 final : CoreStageOp {
    const G3 &g;
    int64_t T;
    int ch, nc;
    const Bins3 &bins;
    R *s_tmp;
    R *p_r;  // FP32 path: the field rounded to R (nc N values); FP64: unused
    double invT;
    bool scaled;
    GridOp3(const G3 &g_, int64_t T_, int ch_, const Bins3 &b_, R *s_tmp_, R *p_r_, bool scaled_)
        : g(g_), T(T_), ch(ch_), nc(ch_ < 0 ? 9 : 3), bins(b_), s_tmp(s_tmp_), p_r(p_r_),
          invT(T_ > 0 ? 1.0 / double(T_) : 0.0), scaled(scaled_) {}
    int normal(const double *p, double *y, cudaStream_t st) override
    {
        const InterpRec3<R> *rec = static_cast<const InterpRec3<R> *>(bins.rec);
        const R *vs = static_cast<const R *>(bins.vs);
        if constexpr (sizeof(R) == 4) {
            const int64_t n = int64_t(nc) * g.n();
            k_round_field<R><<<grid_blocks(n), 256, 0, st>>>(n, p, p_r);
            MPI_CHECK_LAUNCH();
            MPI_TRY((launch_interp3<R, R>(g, T, nullptr, vs, p_r, s_tmp, st, ch, rec)));
        } else {
            MPI_TRY((launch_interp3<R, double>(g, T, nullptr, vs, p, s_tmp, st, ch, rec)));
        }
        return launch_interp3_T<R, double>(g, T, s_tmp, bins, y, invT, st, ch);
    }
    int lap(const double *x, double *out, cudaStream_t st) override
    {
        const double3 c = make_double3(1.0 / (g.dx * g.dx), 1.0 / (g.dy * g.dy), 1.0 / (g.dz * g.dz));
        k_lap3<<<grid_blocks(nc * g.n()), 256, 0, st>>>(g.nx, g.ny, g.nz, nc, scaled, c, x, out);
        MPI_CHECK_LAUNCH();
        return MPI_OK;
    }
};

template <typename R>
int grid3_impl(const G3 &g, const mpi_traj *tr, const void *s_in, const mpi_grid_opts &o, void *Ahat,
               void *trace, int *n_iter_out, cudaStream_t st)
{
    const int64_t T = tr->T;
    const int ch = o.channel - 1;  // -1: all channels; 0..2: that channel only
    const int nc = ch < 0 ? 9 : 3, rows = ch < 0 ? 3 : 1;
    const int64_t N = g.n(), nv = nc * N;
    const R *r = static_cast<const R *>(tr->r), *v = static_cast<const R *>(tr->v);
    const R *s = static_cast<const R *>(s_in);

    Scratch scr(st);
    const size_t o_bins = scr.reserve(bins3_bytes<R>(T, g));
    const size_t o_s = scr.reserve(sizeof(R) * rows * std::max<int64_t>(T, 1));
    const size_t o_sd = scr.reserve(sizeof(R) * rows * std::max<int64_t>(T, 1));
    const size_t o_b = scr.reserve(sizeof(double) * nv), o_x = scr.reserve(sizeof(double) * nv);
    const size_t o_pr = scr.reserve(sizeof(R) == 4 ? sizeof(R) * nv : 0);
    MPI_TRY(scr.allocate());
    const Bins3 bins = bins3_carve<R>(scr.at<char>(o_bins), T, g);
    R *s_data = scr.at<R>(o_sd);
    double *b = scr.at<double>(o_b), *x = scr.at<double>(o_x);

    MPI_TRY(build_bins3<R>(g, T, r, v, bins, st));
    MPI_TRY(gather_rows<R>(T, rows, bins.list, s, s_data, st));
    GridOp3<R> op(g, T, ch, bins, scr.at<R>(o_s), scr.at<R>(o_pr), o.lap_scaled != 0);
    MPI_TRY((launch_interp3_T<R, double>(g, T, s_data, bins, b, op.invT, st, ch)));
    MPI_TRY(core_stage_cg(op, nv, b, o, x, n_iter_out, st));
    k_grid3_output<R><<<grid_blocks(N), 256, 0, st>>>(N, ch, x, static_cast<R *>(Ahat), static_cast<R *>(trace));
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename R>
int interp3_impl(const G3 &g, const mpi_traj *tr, const void *A, void *s, cudaStream_t st)
{
    return launch_interp3<R, R>(g, tr->T, static_cast<const R *>(tr->r), static_cast<const R *>(tr->v),
                                static_cast<const R *>(A), static_cast<R *>(s), st);
}

template <typename R>
int interp3_T_impl(const G3 &g, const mpi_traj *tr, const void *s, void *A, cudaStream_t st)
{
    const int64_t T = tr->T;
    Scratch scr(st);
    const size_t o_bins = scr.reserve(bins3_bytes<R>(T, g));
    const size_t o_ss = scr.reserve(sizeof(R) * 3 * std::max<int64_t>(T, 1));
    MPI_TRY(scr.allocate());
    const Bins3 bins = bins3_carve<R>(scr.at<char>(o_bins), T, g);
    R *s_sorted = scr.at<R>(o_ss);
    MPI_TRY(build_bins3<R>(g, T, static_cast<const R *>(tr->r), static_cast<const R *>(tr->v), bins, st));
    MPI_TRY(gather_rows<R>(T, 3, bins.list, static_cast<const R *>(s), s_sorted, st));
    return launch_interp3_T<R, R>(g, T, s_sorted, bins, static_cast<R *>(A), 1.0, st);
}

int check_interp3_args(const mpi_grid3_desc *grid, const mpi_traj *traj, mpi_dtype dtype)
{
    MPI_TRY(check_grid3(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (traj->T >= ((int64_t)1 << 31)) {
        set_error("interpolation supports T < 2^31");
        return MPI_ERR_UNSUPPORTED;
    }
    if ((int64_t)grid->nx * grid->ny * grid->nz >= ((int64_t)1 << 27)) {
        set_error("the 3-D Core Stage supports grids of fewer than 2^27 nodes");
        return MPI_ERR_UNSUPPORTED;
    }
    return MPI_OK;
}

G3 to_g3(const mpi_grid3_desc *g)
{
    return G3{g->nx, g->ny, g->nz, g->x0, g->y0, g->z0, g->dx, g->dy, g->dz};
}

}  // namespace
}  // namespace mpi

using namespace mpi;

extern "C" {

int mpi_interp3(const mpi_grid3_desc *grid, const mpi_traj *traj, mpi_dtype dtype, const void *Ahat, void *s,
                void *stream)
{
    MPI_TRY(check_interp3_args(grid, traj, dtype));
    if (!Ahat || (traj->T > 0 && !s)) { set_error("Ahat or s is NULL"); return MPI_ERR_INVALID; }
    const G3 g = to_g3(grid);
    return dtype == MPI_F32 ? interp3_impl<float>(g, traj, Ahat, s, as_stream(stream))
                            : interp3_impl<double>(g, traj, Ahat, s, as_stream(stream));
}

int mpi_interp3_adjoint(const mpi_grid3_desc *grid, const mpi_traj *traj, mpi_dtype dtype, const void *s,
                        void *Ahat, void *stream)
{
    MPI_TRY(check_interp3_args(grid, traj, dtype));
    if (!Ahat || (traj->T > 0 && !s)) { set_error("Ahat or s is NULL"); return MPI_ERR_INVALID; }
    const G3 g = to_g3(grid);
    return dtype == MPI_F32 ? interp3_T_impl<float>(g, traj, s, Ahat, as_stream(stream))
                            : interp3_T_impl<double>(g, traj, s, Ahat, as_stream(stream));
}

int mpi_grid3(const mpi_grid3_desc *grid, const mpi_traj *traj, mpi_dtype dtype, const void *s,
              const mpi_grid_opts *opts, void *Ahat, void *trace, int *n_iter_out, void *stream)
{
    MPI_TRY(check_interp3_args(grid, traj, dtype));
    if (!opts || !(opts->gamma >= 0.0) || !std::isfinite(opts->gamma) || opts->max_iter < 0 ||
        std::isnan(opts->rel_tol) || opts->channel < 0 || opts->channel > 3 || opts->lap_scaled < 0 ||
        opts->lap_scaled > 1) {
        set_error("invalid Core Stage options");
        return MPI_ERR_INVALID;
    }
    if (!Ahat || !trace || (traj->T > 0 && !s)) { set_error("s, Ahat or trace is NULL"); return MPI_ERR_INVALID; }
    const G3 g = to_g3(grid);
    return dtype == MPI_F32 ? grid3_impl<float>(g, traj, s, *opts, Ahat, trace, n_iter_out, as_stream(stream))
                            : grid3_impl<double>(g, traj, s, *opts, Ahat, trace, n_iter_out, as_stream(stream));
}

}  // extern "C"
