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
#include "graph.cuh"
#include "grid_common.cuh"

namespace mpi {

int check_grid(const mpi_grid_desc *g);
int check_traj(const mpi_traj *t);
int check_dtype(mpi_dtype d);
GridH to_host(const mpi_grid_desc *g);

// Interpolation record of one sample: its cell (i0, j0) and the upper-node
// cosine weights along x and y (the lower ones are 1 - w).  Fixed for a
// trajectory, so the Core Stage computes them once per solve.
template <typename R>
struct alignas(2 * sizeof(R) + 8 > 16 ? 8 : 16) InterpRec {
    int i0, j0;
    R wx1, wy1;
};

template <typename R>
__device__ __forceinline__ InterpRec<R> make_rec(R px, R py, const AxisMap &ax, const AxisMap &ay)
{
    InterpRec<R> q;
    R w0;
    axis_weights<R>(px, ax, q.i0, w0, q.wx1);
    axis_weights<R>(py, ay, q.j0, w0, q.wy1);
    return q;
}

// s[k][t] = sum_m I[Ahat_{2k+m}](r_t) v_m(t)   (Ahat of type AT, s of type R).
// CH < 0: both channels, Ahat has 4 components, s 2 rows.  CH = k: only
// channel k, Ahat holds (A_k0, A_k1) and s one row.  PRE: the records come
// precomputed (rec), else they are formed from r.  Each thread handles
// kInterpSPT samples a block apart, so its gathers are independent.
// IL: the field is node-interleaved (A[node * NCOMP + comp], NCOMP = 4 or 2
// components of one node contiguous, 16- or 8-byte aligned), so a corner is
// one vector load; otherwise component-major (A[comp * N + node]).  The
// arithmetic is the same either way.
template <typename R, int NCOMP> struct NodeVec;
template <> struct NodeVec<float, 4> { using T = float4; };
template <> struct NodeVec<float, 2> { using T = float2; };

template <typename R, int NCOMP>
__device__ __forceinline__ void load_node(const R *__restrict__ A, int64_t node, R (&out)[NCOMP])
{
    const typename NodeVec<R, NCOMP>::T q = reinterpret_cast<const typename NodeVec<R, NCOMP>::T *>(A)[node];
    if constexpr (NCOMP == 4) { out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w; }
    else { out[0] = q.x; out[1] = q.y; }
}

template <typename R, typename AT, int CH, bool PRE, bool IL = false>
__global__ void __launch_bounds__(256)
k_interp(int64_t T, const R *__restrict__ r, const InterpRec<R> *__restrict__ rec,
         const R *__restrict__ v, const AT *__restrict__ A, AxisMap ax, AxisMap ay, R *__restrict__ s)
{
    const int nx = ax.n;
    const int64_t N = (int64_t)ax.n * ay.n;
    constexpr int K = CH < 0 ? 2 : 1;
    const int64_t span = (int64_t)blockDim.x * kInterpSPT;
    for (int64_t base = blockIdx.x * span + threadIdx.x; base < T; base += (int64_t)gridDim.x * span) {
        InterpRec<R> q[kInterpSPT];
        V2<R> vv[kInterpSPT];
#pragma unroll
        for (int u = 0; u < kInterpSPT; ++u) {
            const int64_t t = min(base + u * (int64_t)blockDim.x, T - 1);
            if constexpr (PRE) q[u] = rec[t];
            else q[u] = make_rec<R>(r[2 * t], r[2 * t + 1], ax, ay);
            vv[u] = V2<R>{v[2 * t], v[2 * t + 1]};
        }
#pragma unroll
        for (int u = 0; u < kInterpSPT; ++u) {
            const int64_t t = base + u * (int64_t)blockDim.x;
            const int i0 = q[u].i0, j0 = q[u].j0;
            const int i1 = ax.n > 1 ? i0 + 1 : i0, j1 = ay.n > 1 ? j0 + 1 : j0;
            const R wx1 = q[u].wx1, wy1 = q[u].wy1, wx0 = R(1) - wx1, wy0 = R(1) - wy1;
            if constexpr (IL) {
                constexpr int NCOMP = 2 * K;
                R f00[NCOMP], f01[NCOMP], f10[NCOMP], f11[NCOMP];  // f<row><col>
                load_node<R, NCOMP>(reinterpret_cast<const R *>(A), (int64_t)j0 * nx + i0, f00);
                load_node<R, NCOMP>(reinterpret_cast<const R *>(A), (int64_t)j0 * nx + i1, f01);
                load_node<R, NCOMP>(reinterpret_cast<const R *>(A), (int64_t)j1 * nx + i0, f10);
                load_node<R, NCOMP>(reinterpret_cast<const R *>(A), (int64_t)j1 * nx + i1, f11);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    R acc = R(0);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const int e = 2 * k + m;
                        const R val = wy0 * (wx0 * f00[e] + wx1 * f01[e]) + wy1 * (wx0 * f10[e] + wx1 * f11[e]);
                        acc += val * (m == 0 ? vv[u].x : vv[u].y);
                    }
                    if (t < T) s[(int64_t)k * T + t] = acc;
                }
            } else {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                R acc = R(0);
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const AT *F = A + (CH < 0 ? 2 * k + m : m) * N;
                    const R val = wy0 * (wx0 * R(F[(int64_t)j0 * nx + i0]) + wx1 * R(F[(int64_t)j0 * nx + i1])) +
                                  wy1 * (wx0 * R(F[(int64_t)j1 * nx + i0]) + wx1 * R(F[(int64_t)j1 * nx + i1]));
                    acc += val * (m == 0 ? vv[u].x : vv[u].y);
                }
                if (t < T) s[(int64_t)k * T + t] = acc;
            }
            }
        }
    }
}

// --- binning of samples by interpolation cell -------------------------------

template <typename R>
__global__ void k_cell_count(int64_t T, const R *__restrict__ r, AxisMap ax, AxisMap ay, int ncx,
                             int *__restrict__ cell_of, int *__restrict__ count,
                             InterpRec<R> *__restrict__ rec)
{
    // every lane of a warp runs the same iterations (warp_count_add)
    for (int64_t t0 = int64_t(blockIdx.x) * blockDim.x; t0 < T; t0 += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        int c = -1;
        if (t < T) {
            const InterpRec<R> q = make_rec<R>(r[2 * t], r[2 * t + 1], ax, ay);
            rec[t] = q;
            c = q.j0 * ncx + q.i0;
            cell_of[t] = c;
        }
        warp_count_add(count, c);
    }
}

// The transpose (Ahat_{2k+m}(node) = sum over the samples t of the node's
// adjacent cells of w_node(t) v_m(t) s_k(t)) runs by cell: each cell's run of
// samples (list order) is split into work units of at most kUnitLen entries;
// a unit reads each of its samples once and forms, for the cell's four
// corner nodes and every component, the sum of w_corner(t) v_m(t) s_k(t)
// (kUnitLanes lanes per unit, then a fixed butterfly).  A node then adds the
// unit sums of its (up to) four adjacent cells in a fixed order.  A sample is
// read once instead of once per corner node, and a cell where the trajectory
// dwells (thousands of samples) spreads over many units.

__global__ void k_cunit_count(int n_cells, const int *__restrict__ offset, int *__restrict__ cunit_cnt)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x)
        cunit_cnt[c] = (offset[c + 1] - offset[c] + kUnitLen - 1) / kUnitLen;
}

__global__ void k_cunit_fill(int n_cells, const int *__restrict__ cunit_off, int *__restrict__ unit_cell)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x)
        for (int w = cunit_off[c]; w < cunit_off[c + 1]; ++w) unit_cell[w] = c;
}

// Corner sums of one unit: for the corners (dx, dy) of the unit's cell
// (corner index dx + 2 dy) and the NC components, the sum over the unit's
// entries of w_dx w_dy v_m s_k, with rec, vs and s in list (cell) order.
// CH = k: only channel k (s one row, two components).  n_iter: the unit
// bound rounded up to whole blocks, so every warp runs the same iterations
// and its shuffles see full warps.
template <typename R, int CH>
__global__ void __launch_bounds__(kUnitThreads)
k_interp_T_cells(const InterpRec<R> *__restrict__ rec, const R *__restrict__ vs, const R *__restrict__ s,
                 int64_t T, const int *__restrict__ offset, const int *__restrict__ cunit_off,
                 const int *__restrict__ unit_cell, const int *__restrict__ n_units_dev, int n_iter,
                 R *__restrict__ unit_part)
{
    constexpr int NC = CH < 0 ? 4 : 2;
    constexpr int G = kUnitLanes;
    constexpr int per_block = kUnitThreads / G;
    const int sub = threadIdx.x % G;
    const int n_units = *n_units_dev;
    for (int base = blockIdx.x * per_block; base < n_iter; base += gridDim.x * per_block) {
        const int w = base + (int)threadIdx.x / G;
        R acc[4][NC];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < NC; ++m) acc[k][m] = R(0);
        if (w < n_units) {
            const int c = unit_cell[w];
            const int q0 = offset[c] + (w - cunit_off[c]) * kUnitLen;
            const int q1 = min(offset[c + 1], q0 + kUnitLen);
#pragma unroll 4
            for (int q = q0 + sub; q < q1; q += G) {
                const InterpRec<R> rc = rec[q];
                const R wx1 = rc.wx1, wy1 = rc.wy1, wx0 = R(1) - wx1, wy0 = R(1) - wy1;
                const R wt[4] = {wy0 * wx0, wy0 * wx1, wy1 * wx0, wy1 * wx1};
                const R vx = vs[2 * q], vy = vs[2 * q + 1];
                R pr[NC];
                if constexpr (CH < 0) {
                    const R s0 = s[q], s1 = s[T + q];
                    pr[0] = vx * s0; pr[1] = vy * s0; pr[2] = vx * s1; pr[3] = vy * s1;
                } else {
                    const R sk = s[q];
                    pr[0] = vx * sk; pr[1] = vy * sk;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int m = 0; m < NC; ++m) acc[k][m] += wt[k] * pr[m];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < NC; ++m)
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) acc[k][m] += __shfl_xor_sync(0xffffffffu, acc[k][m], o);
        if (sub == 0 && w < n_units) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int m = 0; m < NC; ++m) unit_part[((int64_t)w * 4 + k) * NC + m] = acc[k][m];
        }
    }
}

// The Core Stage's normal product by cell, M^T M p, without forming M p: the
// samples of a unit all lie in its cell, so the unit loads the cell's four
// corner nodes of the field p once, and per sample forms
//   s_k = sum_m I[p_{2k+m}](r_t) v_m(t)
// in registers (the arithmetic of k_interp) and adds w_corner v_m s_k to the
// corner sums (that of k_interp_T_cells).  The unit sums are those of the two
// kernels but for the rounding of s, which is not stored; a sample is read
// once (record and velocity) instead of gathered, stored and read again.
// IL: the field node-interleaved in R (NC components per node), else
// component-major in AT; CH = k: only channel k (two components).
template <typename R, typename AT, int CH, bool IL>
__global__ void __launch_bounds__(kUnitThreads)
k_interp_normal_cells(const InterpRec<R> *__restrict__ rec, const R *__restrict__ vs, const AT *__restrict__ A,
                      int nx, int ny, int ncx, const int *__restrict__ offset, const int *__restrict__ cunit_off,
                      const int *__restrict__ unit_cell, const int *__restrict__ n_units_dev, int n_iter,
                      R *__restrict__ unit_part)
{
    constexpr int K = CH < 0 ? 2 : 1;
    constexpr int NC = 2 * K;
    constexpr int G = kUnitLanes;
    constexpr int per_block = kUnitThreads / G;
    const int sub = threadIdx.x % G;
    const int n_units = *n_units_dev;
    const int64_t N = (int64_t)nx * ny;
    for (int base = blockIdx.x * per_block; base < n_iter; base += gridDim.x * per_block) {
        const int w = base + (int)threadIdx.x / G;
        R acc[4][NC];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < NC; ++m) acc[k][m] = R(0);
        if (w < n_units) {
            const int c = unit_cell[w];
            const int i0 = c % ncx, j0 = c / ncx;
            const int i1 = nx > 1 ? i0 + 1 : i0, j1 = ny > 1 ? j0 + 1 : j0;
            // corners: 0 = (i0, j0), 1 = (i1, j0), 2 = (i0, j1), 3 = (i1, j1)
            const int64_t nodes[4] = {(int64_t)j0 * nx + i0, (int64_t)j0 * nx + i1, (int64_t)j1 * nx + i0,
                                      (int64_t)j1 * nx + i1};
            R f[4][NC];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if constexpr (IL) {
                    load_node<R, NC>(reinterpret_cast<const R *>(A), nodes[k], f[k]);
                } else {
#pragma unroll
                    for (int e = 0; e < NC; ++e) f[k][e] = R(A[(int64_t)e * N + nodes[k]]);
                }
            }
            const int q0 = offset[c] + (w - cunit_off[c]) * kUnitLen;
            const int q1 = min(offset[c + 1], q0 + kUnitLen);
#pragma unroll 2
            for (int q = q0 + sub; q < q1; q += G) {
                const InterpRec<R> rc = rec[q];
                const R wx1 = rc.wx1, wy1 = rc.wy1, wx0 = R(1) - wx1, wy0 = R(1) - wy1;
                const R wt[4] = {wy0 * wx0, wy0 * wx1, wy1 * wx0, wy1 * wx1};
                const R vx = vs[2 * q], vy = vs[2 * q + 1];
                R pr[NC];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    R sk = R(0);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const int e = 2 * k + m;
                        const R val = wy0 * (wx0 * f[0][e] + wx1 * f[1][e]) + wy1 * (wx0 * f[2][e] + wx1 * f[3][e]);
                        sk += val * (m == 0 ? vx : vy);
                    }
                    pr[2 * k] = vx * sk;
                    pr[2 * k + 1] = vy * sk;
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int m = 0; m < NC; ++m) acc[k][m] += wt[k] * pr[m];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int m = 0; m < NC; ++m)
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) acc[k][m] += __shfl_xor_sync(0xffffffffu, acc[k][m], o);
        if (sub == 0 && w < n_units) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int m = 0; m < NC; ++m) unit_part[((int64_t)w * 4 + k) * NC + m] = acc[k][m];
        }
    }
}

// sum[m] += the unit sums of `corner` of units w0 .. w1 - 1, in unit order.
// Four units' values are loaded before they are added: the additions depend
// on one another, the loads do not, and a node beside a dense cell adds tens
// of units (one L2 round trip each when every load waits for the previous
// addition).
template <typename R, int NC>
__device__ __forceinline__ void add_unit_sums(const R *__restrict__ unit_part, int w0, int w1, int corner,
                                              SumAcc<R> (&sum)[NC])
{
    int w = w0;
    for (; w + 4 <= w1; w += 4) {
        R v[4][NC];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int m = 0; m < NC; ++m) v[u][m] = unit_part[((int64_t)(w + u) * 4 + corner) * NC + m];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int m = 0; m < NC; ++m) sum[m].add(v[u][m]);
    }
    for (; w < w1; ++w)
#pragma unroll
        for (int m = 0; m < NC; ++m) sum[m].add(unit_part[((int64_t)w * 4 + corner) * NC + m]);
}

// Ahat_m(node) = scale * the sum, over the node's adjacent cells (row-major
// cell order) and their units in order, of the unit sums of the corner the
// node is in that cell (FP32 unit sums as error-free double-float pairs).
template <typename R, typename OUT, int NC>
__global__ void k_interp_T_cell_combine(int nx, int ny, int ncx, int ncy, const int *__restrict__ cunit_off,
                                        const R *__restrict__ unit_part, OUT *__restrict__ A, double scale)
{
    const int N = nx * ny;
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N; node += gridDim.x * blockDim.x) {
        const int i = node % nx, j = node / nx;
        SumAcc<R> acc[NC] = {};
        for (int cj = j - 1; cj <= j; ++cj) {
            if (cj < 0 || cj >= ncy) continue;
            for (int ci = i - 1; ci <= i; ++ci) {
                if (ci < 0 || ci >= ncx) continue;
                const int c = cj * ncx + ci;
                const int corner = (i - ci) + 2 * (j - cj);
                add_unit_sums<R, NC>(unit_part, cunit_off[c], cunit_off[c + 1], corner, acc);
            }
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) cs_store(A[(int64_t)m * N + node], acc[m].value() * scale);
    }
}

// Binning scratch for a trajectory on a grid.
// Samples binned by interpolation cell.  list: sample indices sorted by cell
// (ascending index within a cell); offset: start of each cell's run.  rec /
// vs: the samples' interpolation records and velocities in list order, so a
// cell's samples are one contiguous run of every per-sample array (the Core
// Stage keeps its sample vectors in this order as well).
struct Bins {
    int *cell_of, *count, *offset, *list;
    void *sort_tmp;  // scratch of the ordering and the scans
    void *rec_t;  // InterpRec<R>[T], sample order (scratch of the binning)
    void *rec;    // InterpRec<R>[T], list order
    void *vs;     // R[T][2], list order
    // Work units of the transpose (see kUnitLen): per cell cunit_off[c] ..
    // cunit_off[c + 1] (cunit_off[n_cells] = the number of units); the cell
    // of each unit; 4 corners x 4 partial sums per unit.
    int *cunit_cnt, *cunit_off, *unit_cell;
    void *unit_part;
    int n_units_max;   // bound on the units (allocation)
    int n_units = -1;  // the exact count when read back to the host, else -1
    int ncx, ncy;
};

// Units of the cell runs: at most one per kUnitLen samples plus one per
// non-empty cell.
static int units_bound(int64_t T, int nx, int ny)
{
    const int64_t nc = int64_t(std::max(nx - 1, 1)) * std::max(ny - 1, 1);
    return (int)std::min<int64_t>(INT32_MAX, (T + kUnitLen - 1) / kUnitLen + std::min<int64_t>(T, nc) + 1);
}

template <typename R>
static size_t bins_bytes(int64_t T, int nx, int ny)
{
    const size_t nc = size_t(std::max(nx - 1, 1)) * std::max(ny - 1, 1);
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t U = size_t(units_bound(T, nx, ny));
    return up(sizeof(int) * std::max<int64_t>(T, 1)) * 2 + up(sizeof(int) * nc) +
           up(sizeof(int) * (nc + 1)) + up(std::max(cell_order_bytes(T), cell_scan_bytes(int64_t(nc)))) +
           2 * up(sizeof(InterpRec<R>) * std::max<int64_t>(T, 1)) + up(2 * sizeof(R) * std::max<int64_t>(T, 1)) +
           up(sizeof(int) * nc) + up(sizeof(int) * (nc + 1)) + up(sizeof(int) * U) + up(16 * sizeof(R) * U);
}

template <typename R>
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
    b.offset = reinterpret_cast<int *>(p); p += up(sizeof(int) * (nc + 1));
    b.sort_tmp = p; p += up(std::max(cell_order_bytes(T), cell_scan_bytes(int64_t(nc))));
    b.rec_t = p; p += up(sizeof(InterpRec<R>) * std::max<int64_t>(T, 1));
    b.rec = p; p += up(sizeof(InterpRec<R>) * std::max<int64_t>(T, 1));
    b.vs = p; p += up(2 * sizeof(R) * std::max<int64_t>(T, 1));
    b.n_units_max = units_bound(T, nx, ny);
    b.cunit_cnt = reinterpret_cast<int *>(p); p += up(sizeof(int) * nc);
    b.cunit_off = reinterpret_cast<int *>(p); p += up(sizeof(int) * (nc + 1));
    b.unit_cell = reinterpret_cast<int *>(p); p += up(sizeof(int) * size_t(b.n_units_max));
    b.unit_part = p;
    return b;
}

// Bins the samples, orders their records and velocities by cell and builds
// the transpose's work units.
template <typename R>
static int build_bins(const GridH &g, int64_t T, const R *r, const R *v, const Bins &b, cudaStream_t st)
{
    const AxisMap ax = make_axis(g.x0, g.dx, g.nx), ay = make_axis(g.y0, g.dy, g.ny);
    const int nc = b.ncx * b.ncy;
    MPI_TRY_CUDA(cudaMemsetAsync(b.count, 0, sizeof(int) * nc, st));
    if (T > 0) {
        k_cell_count<R><<<grid_blocks(T), 256, 0, st>>>(T, r, ax, ay, b.ncx, b.cell_of, b.count,
                                                         static_cast<InterpRec<R> *>(b.rec_t));
        MPI_CHECK_LAUNCH();
    }
    MPI_TRY(cell_scan_launch(b.count, nc, b.offset, b.sort_tmp, st));
    if (T > 0) {
        MPI_TRY(cell_order_launch(T, b.cell_of, nc, b.list, b.sort_tmp, st));
        k_sort_records<InterpRec<R>, R, 2><<<grid_blocks(T), 256, 0, st>>>(T, b.list, static_cast<const InterpRec<R> *>(b.rec_t),
                                                          v, static_cast<InterpRec<R> *>(b.rec),
                                                          static_cast<R *>(b.vs));
        MPI_CHECK_LAUNCH();
    }
    // Work units of the transpose.
    k_cunit_count<<<grid_blocks(nc), 256, 0, st>>>(nc, b.offset, b.cunit_cnt);
    MPI_CHECK_LAUNCH();
    MPI_TRY(cell_scan_launch(b.cunit_cnt, nc, b.cunit_off, b.sort_tmp, st));
    k_cunit_fill<<<grid_blocks(nc), 256, 0, st>>>(nc, b.cunit_off, b.unit_cell);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// rec (nullable): precomputed records of the samples (Core Stage).
template <typename R, typename AT>
static int launch_interp(const GridH &g, int64_t T, const R *r, const R *v, const AT *A, R *s,
                         cudaStream_t st, int ch = -1, const InterpRec<R> *rec = nullptr, bool il = false)
{
    if (T == 0) return MPI_OK;
    const AxisMap ax = make_axis(g.x0, g.dx, g.nx), ay = make_axis(g.y0, g.dy, g.ny);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((T + 256 * kInterpSPT - 1) / (256 * kInterpSPT), 8192));
    if constexpr (sizeof(AT) == 4) {
        if (il) {  // node-interleaved FP32 field, records precomputed
            if (ch < 0) k_interp<R, AT, -1, true, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
            else if (ch == 0) k_interp<R, AT, 0, true, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
            else k_interp<R, AT, 1, true, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
            MPI_CHECK_LAUNCH();
            return MPI_OK;
        }
    }
    if (rec) {
        if (ch < 0) k_interp<R, AT, -1, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
        else if (ch == 0) k_interp<R, AT, 0, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
        else k_interp<R, AT, 1, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
    } else {
        if (ch < 0) k_interp<R, AT, -1, false><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
        else if (ch == 0) k_interp<R, AT, 0, false><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
        else k_interp<R, AT, 1, false><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, ay, s);
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// The transpose's unit sums (k_interp_T_cells) into b.unit_part.
// s_sorted: the samples' values in list order ([rows][T]).
template <typename R>
static int launch_interp_T_units(int64_t T, const R *s_sorted, const Bins &b, cudaStream_t st, int ch)
{
    const int nc = b.ncx * b.ncy;
    constexpr int per_block = kUnitThreads / kUnitLanes;
    // Blocks for the exact unit count where the host has it, else for the
    // bound (every cell counted non-empty): the real count is on the device
    // and the surplus blocks exit at once.
    const int units = b.n_units >= 0 ? b.n_units : b.n_units_max;
    const int n_iter = (units + per_block - 1) / per_block * per_block;
    const unsigned blocks = (unsigned)std::max(1, std::min(n_iter / per_block, 65535));
    const InterpRec<R> *rec = static_cast<const InterpRec<R> *>(b.rec);
    const R *vs = static_cast<const R *>(b.vs);
    R *part = static_cast<R *>(b.unit_part);
    const int *n_units = b.cunit_off + nc;
    if (ch < 0)
        k_interp_T_cells<R, -1><<<blocks, kUnitThreads, 0, st>>>(rec, vs, s_sorted, T, b.offset, b.cunit_off,
                                                                 b.unit_cell, n_units, n_iter, part);
    else
        k_interp_T_cells<R, 0><<<blocks, kUnitThreads, 0, st>>>(rec, vs, s_sorted, T, b.offset, b.cunit_off,
                                                                b.unit_cell, n_units, n_iter, part);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// A = scale M^T s (all four components, or channel ch's two).
template <typename R, typename OUT>
static int launch_interp_T(const GridH &g, int64_t T, const R *s_sorted, const Bins &b, OUT *A, double scale,
                           cudaStream_t st, int ch = -1)
{
    MPI_TRY(launch_interp_T_units<R>(T, s_sorted, b, st, ch));
    const int N = g.nx * g.ny;
    const R *part = static_cast<const R *>(b.unit_part);
    if (ch < 0)
        k_interp_T_cell_combine<R, OUT, 4><<<grid_blocks(N), 256, 0, st>>>(g.nx, g.ny, b.ncx, b.ncy, b.cunit_off,
                                                                          part, A, scale);
    else
        k_interp_T_cell_combine<R, OUT, 2><<<grid_blocks(N), 256, 0, st>>>(g.nx, g.ny, b.ncx, b.ncy, b.cunit_off,
                                                                          part, A, scale);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// Unit sums of M^T M p (k_interp_normal_cells) for the Core Stage step.
template <typename R, typename AT, bool IL>
static int launch_normal_units(const GridH &g, const Bins &b, const AT *A, int ch, cudaStream_t st)
{
    const int nc = b.ncx * b.ncy;
    constexpr int per_block = kUnitThreads / kUnitLanes;
    const int units = b.n_units >= 0 ? b.n_units : b.n_units_max;
    const int n_iter = (units + per_block - 1) / per_block * per_block;
    const unsigned blocks = (unsigned)std::max(1, std::min(n_iter / per_block, 65535));
    const InterpRec<R> *rec = static_cast<const InterpRec<R> *>(b.rec);
    const R *vs = static_cast<const R *>(b.vs);
    R *part = static_cast<R *>(b.unit_part);
    const int *n_units = b.cunit_off + nc;
    if (ch < 0)
        k_interp_normal_cells<R, AT, -1, IL><<<blocks, kUnitThreads, 0, st>>>(
            rec, vs, A, g.nx, g.ny, b.ncx, b.offset, b.cunit_off, b.unit_cell, n_units, n_iter, part);
    else
        k_interp_normal_cells<R, AT, 0, IL><<<blocks, kUnitThreads, 0, st>>>(
            rec, vs, A, g.nx, g.ny, b.ncx, b.offset, b.cunit_off, b.unit_cell, n_units, n_iter, part);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// --- Laplacian and the Core Stage operator ---------------------------------

// (Lap f)(node k at i, j): 5-point, replicated boundary (a missing
// neighbour is the node itself), FP64.  scaled: per-axis second differences
// with 1/dx^2 (cx) and 1/dy^2 (cy); else the plain stencil.
__device__ __forceinline__ double lap2_at(const double *__restrict__ f, int k, int i, int j, int nx, int ny,
                                          bool scaled, double cx, double cy)
{
    const int im = i > 0 ? i - 1 : 0, ip = i < nx - 1 ? i + 1 : nx - 1;
    const int jm = j > 0 ? j - 1 : 0, jp = j < ny - 1 ? j + 1 : ny - 1;
    if (scaled) {
        const double c0 = f[k];
        return cx * (f[j * nx + im] - 2.0 * c0 + f[j * nx + ip]) + cy * (f[jm * nx + i] - 2.0 * c0 + f[jp * nx + i]);
    }
    return f[j * nx + im] + f[j * nx + ip] + f[jm * nx + i] + f[jp * nx + i] - 4.0 * f[k];
}
// The same in double-float arithmetic (cx, cy as double-float pairs).
__device__ __forceinline__ df lap2_at(const df *__restrict__ f, int k, int i, int j, int nx, int ny, bool scaled,
                                      df cx, df cy)
{
    const int im = i > 0 ? i - 1 : 0, ip = i < nx - 1 ? i + 1 : nx - 1;
    const int jm = j > 0 ? j - 1 : 0, jp = j < ny - 1 ? j + 1 : ny - 1;
    const df c0 = f[k];
    const df sx = df_add(f[j * nx + im], f[j * nx + ip]), sy = df_add(f[jm * nx + i], f[jp * nx + i]);
    if (scaled) {
        const df m2 = make_float2(-2.0f, 0.0f);
        return df_add(df_mul(df_axpy(sx, m2, c0), cx), df_mul(df_axpy(sy, m2, c0), cy));
    }
    return df_axpy(df_add(sx, sy), make_float2(-4.0f, 0.0f), c0);
}

// out_m = Lap x_m for the nc components (SCALE: w Lap x_m); E: FP64 or
// double-float elements (and scalars).
template <typename E, bool SCALE>
__global__ void k_lap(int nx, int ny, int nc, bool scaled, E cx, E cy, const E *__restrict__ x, E *__restrict__ out,
                      E w)
{
    const int N = nx * ny;  // nc N < 2^31 (grids of at most 2^28 nodes)
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc * N; e += gridDim.x * blockDim.x) {
        const int m = e / N, k = e - m * N;
        const E L = lap2_at(x + (int64_t)m * N, k, k % nx, k / nx, nx, ny, scaled, cx, cy);
        out[e] = SCALE ? cs_scale(L, w) : L;
    }
}

// One 2-D Core Stage step after the transpose's unit sums, one thread per
// node and all its components m: q = scale * (the node's combine, as
// k_interp_T_cell_combine forms it) + l2 with l2 = gamma Lap Lap p (formed
// on the side stream), written to q, and the partial sums of <p, q> over
// blocks of kQThreads consecutive nodes, finished into alpha by the last
// block.
constexpr int kQThreads = 256;
template <typename R, int NC, typename E>
__global__ void __launch_bounds__(kQThreads)
k_grid_q(int nx, int ny, int ncx, int ncy, const int *__restrict__ cunit_off, const R *__restrict__ unit_part,
         E scale, const E *__restrict__ l2, const E *__restrict__ p, E *__restrict__ q, double *__restrict__ pq_part,
         CsScal *sc)
{
    __shared__ double sh[kQThreads / 32];
    __shared__ bool last;
    const int N = nx * ny;  // <= 2^28
    const int node = blockIdx.x * kQThreads + threadIdx.x;
    CsDot<E> acc{};
    if (node < N) {
        const int i = node % nx, j = node / nx;
        SumAcc<R> sum[NC] = {};
        for (int cj = j - 1; cj <= j; ++cj) {
            if (cj < 0 || cj >= ncy) continue;
            for (int ci = i - 1; ci <= i; ++ci) {
                if (ci < 0 || ci >= ncx) continue;
                const int c = cj * ncx + ci;
                const int corner = (i - ci) + 2 * (j - cj);
                add_unit_sums<R, NC>(unit_part, cunit_off[c], cunit_off[c + 1], corner, sum);
            }
        }
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const int64_t e = (int64_t)m * N + node;
            const E qe = cs_sum_scale_add(sum[m], scale, l2[e]);
            q[e] = qe;
            acc.add(p[e], qe);
        }
    }
    const double tot = acc.template block_total<kQThreads>(sh);
    if (threadIdx.x == 0) pq_part[blockIdx.x] = tot;
    cs_finish_pq<kQThreads>(pq_part, gridDim.x, sc, sh, &last);
}

// --- Core Stage CG vector kernels -----------------------------------------
// Blocks of kCsThreads threads over kCsPer consecutive unknowns; each
// reduction is finished by its last block (CsScal), so a kernel reads its
// coefficient as one scalar.
constexpr int kCsThreads = 256, kCsPer = 2048;
inline int cs_blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + kCsPer - 1) / kCsPer); }

// r = b, p = b (x = 0), r.r, ||b|| and the stop threshold rel_tol ||b||.
// E: the element type of the vectors (double, or double-float pairs).
template <typename E>
__global__ void __launch_bounds__(kCsThreads)
k_cs_init(int64_t n, const E *__restrict__ b, E *__restrict__ r, E *__restrict__ p, double *__restrict__ rr_part,
          double rel_tol, CsScal *sc)
{
    __shared__ double sh[kCsThreads / 32];
    __shared__ bool last;
    const int64_t e0 = (int64_t)blockIdx.x * kCsPer;
    CsDot<E> acc{};
#pragma unroll
    for (int u = 0; u < kCsPer / kCsThreads; ++u) {
        const int64_t e = e0 + u * kCsThreads + threadIdx.x;
        if (e < n) {
            const E be = b[e];
            r[e] = be;
            p[e] = be;
            acc.add(be, be);
        }
    }
    const double tot = acc.template block_total<kCsThreads>(sh);
    if (threadIdx.x == 0) rr_part[blockIdx.x] = tot;
    if (!cs_last_block(&sc->cnt[kCntInit], &last)) return;
    const double rr = cs_sum_parts<kCsThreads>(rr_part, gridDim.x, sh);
    if (threadIdx.x == 0) {
        sc->rr = rr;
        sc->bnorm = sqrt(rr);
        sc->tol = rel_tol > 0.0 ? rel_tol * sqrt(rr) : -1.0;
        sc->done = 0;
        sc->iters = 0;
    }
}

// x += alpha p, r -= alpha q, the new r.r and beta = r.r(new) / r.r(old);
// counts the update.  Nothing once the solve has stopped.
template <typename E>
__global__ void __launch_bounds__(kCsThreads)
k_cs_step1(int64_t n, E *__restrict__ x, E *__restrict__ r, const E *__restrict__ p, const E *__restrict__ q,
           double *__restrict__ rr_part, CsScal *sc)
{
    __shared__ double sh[kCsThreads / 32];
    __shared__ bool last;
    constexpr int U = kCsPer / kCsThreads;
    const int64_t e0 = (int64_t)blockIdx.x * kCsPer + threadIdx.x;
    // the vectors are loaded before the stop flag is read: the flag comes
    // from the previous kernel and would otherwise add a round trip
    E xv[U], pv[U], rv[U], qv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t e = e0 + u * kCsThreads;
        const bool in = e < n;
        xv[u] = in ? x[e] : cs_zero<E>();
        pv[u] = in ? p[e] : cs_zero<E>();
        rv[u] = in ? r[e] : cs_zero<E>();
        qv[u] = in ? q[e] : cs_zero<E>();
    }
    if (sc->done) return;
    const E alpha = cs_alpha<E>(sc), nalpha = cs_neg(alpha);
    CsDot<E> acc{};
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int64_t e = e0 + u * kCsThreads;
        if (e < n) {
            x[e] = cs_axpy(xv[u], alpha, pv[u]);
            const E re = cs_axpy(rv[u], nalpha, qv[u]);
            r[e] = re;
            acc.add(re, re);
        }
    }
    const double tot = acc.template block_total<kCsThreads>(sh);
    if (threadIdx.x == 0) rr_part[blockIdx.x] = tot;
    if (!cs_last_block(&sc->cnt[kCntRr], &last)) return;
    const double rr = cs_sum_parts<kCsThreads>(rr_part, gridDim.x, sh);
    if (threadIdx.x == 0) {
        sc->beta = rr / sc->rr;
        sc->beta_df = df_from_double(sc->beta);
        sc->rr = rr;
        sc->iters += 1;
    }
}

// p = r + beta p.
template <typename E>
__global__ void __launch_bounds__(kCsThreads)
k_cs_step2(int64_t n, const E *__restrict__ r, E *__restrict__ p, const CsScal *sc)
{
    if (sc->done) return;
    const E beta = cs_beta<E>(sc);
    const int64_t e0 = (int64_t)blockIdx.x * kCsPer;
#pragma unroll
    for (int u = 0; u < kCsPer / kCsThreads; ++u) {
        const int64_t e = e0 + u * kCsThreads + threadIdx.x;
        if (e < n) p[e] = cs_axpy(r[e], beta, p[e]);
    }
}

// The FP32 copy of p in the operator's layout (P32Layout): the FP32 Core
// Stage gathers FP32 values in its interpolation (GB300 converts FP64 at a
// small fraction of the FP32 rate; a gather converting 16 or 72 values per
// sample was bound by that conversion), and the direction update writes the
// copy as it forms p.  Components per node:
template <int L>
constexpr int p32_nc()
{
    return L == kP32Node4 ? 4 : L == kP32Node2 ? 2 : L == kP32Rows3x4 ? 9 : 3;
}
template <int L>
__device__ __forceinline__ void p32_store(float *buf, int64_t node, const float *v)
{
    if constexpr (L == kP32Node4) {
        reinterpret_cast<float4 *>(buf)[node] = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (L == kP32Node2) {
        reinterpret_cast<float2 *>(buf)[node] = make_float2(v[0], v[1]);
    } else {
        constexpr int K = p32_nc<L>() / 3;
#pragma unroll
        for (int k = 0; k < K; ++k)
            reinterpret_cast<float4 *>(buf)[node * K + k] = make_float4(v[3 * k], v[3 * k + 1], v[3 * k + 2], 0.0f);
    }
}

// buf = p rounded to FP32 (one thread per node, all its components).
template <typename E, int L>
__global__ void __launch_bounds__(kCsThreads) k_cs_round(int64_t N, const E *__restrict__ p, float *buf)
{
    constexpr int NC = p32_nc<L>();
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < N;
         node += (int64_t)gridDim.x * blockDim.x) {
        float v[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) v[m] = cs_to_float(p[m * N + node]);
        p32_store<L>(buf, node, v);
    }
}

// p = r + beta p and its FP32 copy (one thread per node, all its components).
template <typename E, int L>
__global__ void __launch_bounds__(kCsThreads)
k_cs_step2_p32(int64_t N, const E *__restrict__ r, E *__restrict__ p, const CsScal *sc, float *buf)
{
    constexpr int NC = p32_nc<L>();
    for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < N;
         node += (int64_t)gridDim.x * blockDim.x) {
        E rv[NC], pv[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            rv[m] = r[m * N + node];
            pv[m] = p[m * N + node];
        }
        if (sc->done) return;  // (read after the vector loads are issued)
        const E beta = cs_beta<E>(sc);
        float v[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const E pe = cs_axpy(rv[m], beta, pv[m]);
            p[m * N + node] = pe;
            v[m] = cs_to_float(pe);
        }
        p32_store<L>(buf, node, v);
    }
}

template <typename E>
static int cs_round_launch(const P32 &d, const E *p, cudaStream_t st)
{
    const int blocks = grid_blocks(d.N);
    switch (d.layout) {
        case kP32Node4: k_cs_round<E, kP32Node4><<<blocks, kCsThreads, 0, st>>>(d.N, p, d.buf); break;
        case kP32Node2: k_cs_round<E, kP32Node2><<<blocks, kCsThreads, 0, st>>>(d.N, p, d.buf); break;
        case kP32Rows3x4: k_cs_round<E, kP32Rows3x4><<<blocks, kCsThreads, 0, st>>>(d.N, p, d.buf); break;
        default: k_cs_round<E, kP32Rows1x4><<<blocks, kCsThreads, 0, st>>>(d.N, p, d.buf); break;
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename E>
static int cs_step2_launch(const P32 &d, int64_t nv, const E *r, E *p, const CsScal *sc, cudaStream_t st)
{
    if (!d.buf) {
        k_cs_step2<E><<<cs_blocks(nv), kCsThreads, 0, st>>>(nv, r, p, sc);
    } else {
        const int blocks = grid_blocks(d.N);
        switch (d.layout) {
            case kP32Node4:
                k_cs_step2_p32<E, kP32Node4><<<blocks, kCsThreads, 0, st>>>(d.N, r, p, sc, d.buf);
                break;
            case kP32Node2:
                k_cs_step2_p32<E, kP32Node2><<<blocks, kCsThreads, 0, st>>>(d.N, r, p, sc, d.buf);
                break;
            case kP32Rows3x4:
                k_cs_step2_p32<E, kP32Rows3x4><<<blocks, kCsThreads, 0, st>>>(d.N, r, p, sc, d.buf);
                break;
            default:
                k_cs_step2_p32<E, kP32Rows1x4><<<blocks, kCsThreads, 0, st>>>(d.N, r, p, sc, d.buf);
                break;
        }
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// Ahat and its trace (both channels: A_00 + A_11; one channel k: A_kk,
// which is component k of the stored pair (A_k0, A_k1)).
template <typename R, typename E>
__global__ void k_grid_output(int64_t N, int ch, const E *__restrict__ x, R *__restrict__ A,
                              R *__restrict__ tr)
{
    const int nc = ch < 0 ? 4 : 2;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int m = 0; m < nc; ++m) A[m * N + e] = R(cs_to_double(x[m * N + e]));
        tr[e] = ch < 0 ? R(cs_to_double(cs_add(x[e], x[3 * N + e]))) : R(cs_to_double(x[ch * N + e]));
    }
}

// The 2-D Core Stage operator: (1/T) M^T M through the binned records and
// the 5-point Laplacian of each component.  A step: l2 = gamma Lap Lap p on
// the side stream (two passes) while the main chain runs M p (through the
// FP32 copy of p on the FP32 path) and the transpose's unit sums; then one
// pass forms q and the <p, q> partials (k_grid_q).  The CG vectors are FP64
// (FP64 path) or double-float pairs (FP32 path: E = float2).
template <typename R>
struct GridOp2 final : CoreStageOp<typename CsElem<R>::type> {
    using E = typename CsElem<R>::type;
    const GridH &g;
    int64_t T;
    int ch, nc;
    const Bins &bins;
    R *p_r;  // FP32 path: the FP32 copy of p, node-interleaved (nc N values); FP64: unused
    double invT;
    bool scaled;
    GridOp2(const GridH &g_, int64_t T_, int ch_, const Bins &b_, R *p_r_, bool scaled_)
        : g(g_), T(T_), ch(ch_), nc(ch_ < 0 ? 4 : 2), bins(b_), p_r(p_r_),
          invT(T_ > 0 ? 1.0 / double(T_) : 0.0), scaled(scaled_) {}
    P32 p32() const override
    {
        if constexpr (sizeof(R) == 4)
            return P32{reinterpret_cast<float *>(p_r), nc == 4 ? kP32Node4 : kP32Node2, int64_t(g.nx) * g.ny};
        return P32{};
    }
    int pq_blocks(int64_t) const override { return (int)((int64_t(g.nx) * g.ny + kQThreads - 1) / kQThreads); }
    int step_q(const E *p, double gamma, E *q, double *pq_part, CsScal *sc, E *l1, E *l2, const StepFork &fk,
               cudaStream_t st) override
    {
        E *tag = nullptr;
        const E cx = cs_host_scalar(1.0 / (g.dx * g.dx), tag), cy = cs_host_scalar(1.0 / (g.dy * g.dy), tag);
        const int lb = grid_blocks(int64_t(nc) * g.nx * g.ny);
        MPI_TRY_CUDA(cudaEventRecord(fk.fork, st));
        MPI_TRY_CUDA(cudaStreamWaitEvent(fk.side, fk.fork, 0));
        k_lap<E, false><<<lb, 256, 0, fk.side>>>(g.nx, g.ny, nc, scaled, cx, cy, p, l1, cs_host_scalar(1.0, tag));
        MPI_CHECK_LAUNCH();
        k_lap<E, true><<<lb, 256, 0, fk.side>>>(g.nx, g.ny, nc, scaled, cx, cy, l1, l2, cs_host_scalar(gamma, tag));
        MPI_CHECK_LAUNCH();
        MPI_TRY_CUDA(cudaEventRecord(fk.join, fk.side));
        // main branch: the unit sums of M^T M p, one pass over the samples
        if constexpr (sizeof(R) == 4) MPI_TRY((launch_normal_units<R, R, true>(g, bins, p_r, ch, st)));
        else MPI_TRY((launch_normal_units<R, double, false>(g, bins, reinterpret_cast<const double *>(p), ch, st)));
        MPI_TRY_CUDA(cudaStreamWaitEvent(st, fk.join, 0));
        const unsigned blocks = (unsigned)pq_blocks(0);
        const R *part = static_cast<const R *>(bins.unit_part);
        const E sc_T = cs_host_scalar(invT, tag);
        if (ch < 0)
            k_grid_q<R, 4, E><<<blocks, kQThreads, 0, st>>>(g.nx, g.ny, bins.ncx, bins.ncy, bins.cunit_off, part,
                                                           sc_T, l2, p, q, pq_part, sc);
        else
            k_grid_q<R, 2, E><<<blocks, kQThreads, 0, st>>>(g.nx, g.ny, bins.ncx, bins.ncy, bins.cunit_off, part,
                                                           sc_T, l2, p, q, pq_part, sc);
        MPI_CHECK_LAUNCH();
        return MPI_OK;
    }
};

template <typename R>
static int grid_impl(const GridH &g, const mpi_traj *tr, const void *s_in, const mpi_grid_opts &o,
                     void *Ahat, void *trace, int *n_iter_out, cudaStream_t st)
{
    const int64_t T = tr->T;
    const int ch = o.channel - 1;  // -1: both channels; 0 / 1: that channel only
    const int nc = ch < 0 ? 4 : 2, rows = ch < 0 ? 2 : 1;
    const int64_t N = (int64_t)g.nx * g.ny, n4 = nc * N;
    const R *r = static_cast<const R *>(tr->r), *v = static_cast<const R *>(tr->v);
    const R *s = static_cast<const R *>(s_in);

    Scratch scr(st);
    const size_t o_bins = scr.reserve(bins_bytes<R>(T, g.nx, g.ny));
    const size_t o_sd = scr.reserve(sizeof(R) * rows * std::max<int64_t>(T, 1));
    using E = typename CsElem<R>::type;
    const size_t o_b = scr.reserve(sizeof(E) * n4), o_x = scr.reserve(sizeof(E) * n4);
    const size_t o_pr = scr.reserve(sizeof(R) == 4 ? sizeof(R) * n4 : 0);
    MPI_TRY(scr.allocate());
    Bins bins = bins_carve<R>(scr.at<char>(o_bins), T, g.nx, g.ny);
    R *s_data = scr.at<R>(o_sd);
    E *b = scr.at<E>(o_b), *x = scr.at<E>(o_x);

    MPI_TRY(build_bins<R>(g, T, r, v, bins, st));
    // The sample vectors of the solve live in list (cell) order.
    MPI_TRY(gather_rows<R>(T, rows, bins.list, s, s_data, st));
    // The transpose runs up to thousands of times with the same units: read
    // their count once, so every launch covers exactly them.
    {
        int n_units = 0;
        MPI_TRY_CUDA(cudaMemcpyAsync(&n_units, bins.cunit_off + bins.ncx * bins.ncy, sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
        MPI_TRY_CUDA(cudaStreamSynchronize(st));
        if (n_units < 0 || n_units > bins.n_units_max) {
            set_error("Core Stage: %d work units exceed the bound %d", n_units, bins.n_units_max);
            return MPI_ERR_CUDA;
        }
        bins.n_units = n_units;
    }
    GridOp2<R> op(g, T, ch, bins, scr.at<R>(o_pr), o.lap_scaled != 0);
    // b = (1/T) M^T s
    MPI_TRY((launch_interp_T<R, E>(g, T, s_data, bins, b, op.invT, st, ch)));
    MPI_TRY(core_stage_cg<E>(op, n4, b, o, x, n_iter_out, st));
    k_grid_output<R, E><<<grid_blocks(N), 256, 0, st>>>(N, ch, x, static_cast<R *>(Ahat), static_cast<R *>(trace));
    MPI_CHECK_LAUNCH();
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
    const size_t o_bins = scr.reserve(bins_bytes<R>(T, g.nx, g.ny));
    const size_t o_ss = scr.reserve(sizeof(R) * 2 * std::max<int64_t>(T, 1));
    MPI_TRY(scr.allocate());
    const Bins bins = bins_carve<R>(scr.at<char>(o_bins), T, g.nx, g.ny);
    R *s_sorted = scr.at<R>(o_ss);
    MPI_TRY(build_bins<R>(g, T, static_cast<const R *>(tr->r), static_cast<const R *>(tr->v), bins, st));
    MPI_TRY(gather_rows<R>(T, 2, bins.list, static_cast<const R *>(s), s_sorted, st));
    return launch_interp_T<R, R>(g, T, s_sorted, bins, static_cast<R *>(A), 1.0, st);
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

template <typename E>
int core_stage_cg(CoreStageOp<E> &op, int64_t nv, const E *b, const mpi_grid_opts &o, E *x, int *n_iter_out,
                  cudaStream_t st)
{
    const int ncs = cs_blocks(nv);
    const int npq = op.pq_blocks(nv);
    const P32 p32 = op.p32();
    Scratch scr(st);
    const size_t vb = sizeof(E) * nv;
    const size_t o_r = scr.reserve(vb), o_p = scr.reserve(vb), o_q = scr.reserve(vb), o_l1 = scr.reserve(vb),
                 o_l2 = scr.reserve(vb);
    const size_t o_pq = scr.reserve(sizeof(double) * npq), o_rr = scr.reserve(sizeof(double) * ncs);
    const size_t o_sc = scr.reserve(sizeof(CsScal));
    MPI_TRY(scr.allocate());
    E *rr = scr.at<E>(o_r), *p = scr.at<E>(o_p), *q = scr.at<E>(o_q), *l1 = scr.at<E>(o_l1),
      *l2 = scr.at<E>(o_l2);
    double *pq_part = scr.at<double>(o_pq), *rr_part = scr.at<double>(o_rr);
    CsScal *sc = scr.at<CsScal>(o_sc);

    // The side stream and events of the step's fork-join (released when the
    // solve returns; the stream's work is joined into st by then).
    struct Fork {
        StepFork f{nullptr, nullptr, nullptr};
        ~Fork()
        {
            if (f.side) {
                cudaStreamSynchronize(f.side);  // (an error path may have left a fork unjoined)
                cudaStreamDestroy(f.side);
            }
            if (f.fork) cudaEventDestroy(f.fork);
            if (f.join) cudaEventDestroy(f.join);
        }
    } fk;
    MPI_TRY_CUDA(cudaStreamCreateWithFlags(&fk.f.side, cudaStreamNonBlocking));
    MPI_TRY_CUDA(cudaEventCreateWithFlags(&fk.f.fork, cudaEventDisableTiming));
    MPI_TRY_CUDA(cudaEventCreateWithFlags(&fk.f.join, cudaEventDisableTiming));

    MPI_TRY_CUDA(cudaMemsetAsync(x, 0, vb, st));
    MPI_TRY_CUDA(cudaMemsetAsync(sc, 0, sizeof(CsScal), st));
    // r = b, p = b, r.r, ||b|| and the threshold
    k_cs_init<E><<<ncs, kCsThreads, 0, st>>>(nv, b, rr, p, rr_part, o.rel_tol, sc);
    MPI_CHECK_LAUNCH();
    if (p32.buf) MPI_TRY(cs_round_launch(p32, p, st));

    int *h_done = nullptr;
    MPI_TRY_CUDA(cudaMallocHost(reinterpret_cast<void **>(&h_done), sizeof(int)));
    struct PinnedFree {
        int *p;
        ~PinnedFree() { cudaFreeHost(p); }
    } guard{h_done};
    int *done = &sc->done, *iters = &sc->iters;
    const bool thresh = o.rel_tol > 0.0;

    // One CG step: q = (1/T) M^T M p + gamma Lap Lap p, <p, q> and alpha (or
    // the stop), then the update and beta, then the new direction (and its
    // FP32 copy).
    auto enqueue_step = [&](int, cudaStream_t s) -> int {
        MPI_TRY(op.step_q(p, o.gamma, q, pq_part, sc, l1, l2, fk.f, s));
        k_cs_step1<E><<<ncs, kCsThreads, 0, s>>>(nv, x, rr, p, q, rr_part, sc);
        MPI_CHECK_LAUNCH();
        return cs_step2_launch(p32, nv, rr, p, sc, s);
    };
    auto poll_done = [&](bool &stop) -> int {
        MPI_TRY_CUDA(cudaMemcpyAsync(h_done, done, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPI_TRY_CUDA(cudaStreamSynchronize(st));
        stop = *h_done != 0;
        return MPI_OK;
    };

    // The steps are short dependent launches (latency-bound), so a run of
    // `poll` steps -- the span between two host polls of the stop flag -- is
    // captured once as a CUDA graph and replayed: the same kernels with the
    // same arguments in the same order, hence the same result.  The capture uses a
    // private stream (the caller's may be the legacy default stream, which
    // cannot be captured); the graph runs on the caller's stream.
    const int poll = 16;
    int it = 0;
    bool stop = false;
    if (o.max_iter >= 2 * poll) {
        CapturedGraph g;
        if (g.capture([&](cudaStream_t s) -> int {
                for (int k = 0; k < poll; ++k) MPI_TRY(enqueue_step(k, s));
                return MPI_OK;
            }) == MPI_OK) {
            for (; it + poll <= o.max_iter && !stop; it += poll) {
                MPI_TRY(g.launch(st));
                if (thresh && it + poll < o.max_iter) MPI_TRY(poll_done(stop));
            }
        }
    }
    for (; it < o.max_iter && !stop; ++it) {
        MPI_TRY(enqueue_step(it, st));
        if (thresh && (it + 1) % poll == 0 && it + 1 < o.max_iter) MPI_TRY(poll_done(stop));
    }
    if (n_iter_out) {
        MPI_TRY_CUDA(cudaMemcpyAsync(h_done, iters, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPI_TRY_CUDA(cudaStreamSynchronize(st));
        *n_iter_out = *h_done;
    }
    return MPI_OK;
}
template int core_stage_cg<double>(CoreStageOp<double> &, int64_t, const double *, const mpi_grid_opts &, double *,
                                   int *, cudaStream_t);
template int core_stage_cg<float2>(CoreStageOp<float2> &, int64_t, const float2 *, const mpi_grid_opts &, float2 *,
                                   int *, cudaStream_t);

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
        std::isnan(opts->rel_tol) || opts->channel < 0 || opts->channel > 2 || opts->lap_scaled < 0 ||
        opts->lap_scaled > 1) {
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
