// Core Stage in three dimensions (Eq. first:step with n = 3): the core
// operator at a point is the 3 x 3 matrix Ahat_km (receive channel k, velocity
// component m), measured through the tensor-product cosine interpolation
//   s_k(t) = sum_m I[Ahat_km](r_t) v_m(t),
// and recovered by CG on ((1/T) M^T M + gamma Lap Lap) Ahat = (1/T) M^T s with
// the 7-point replicated-boundary Laplacian on each component.
//
// Same organisation as the 2-D solve: interpolation records computed once per
// trajectory, samples binned by interpolation cell (a cell now has 8 corner
// nodes, a node up to 8 adjacent cells), the transpose summed per cell in
// work units of at most kUnitLen samples and combined per node in a fixed
// order (no float atomics, run-to-run identical), CG vectors and inner
// products in FP64.
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
// from r.  One thread per output s[k][t] (element e = k T + t): a Core Stage
// trajectory of ~10^5 samples then still fills the GPU.  IL (FP32 field,
// records precomputed): the field is node-interleaved, A4[node K + k] =
// (A_{3k}, A_{3k+1}, A_{3k+2}, 0) with K rows, so a corner's three
// components are one 16-byte load.
template <typename R, typename AT, int CH, bool PRE, bool IL = false>
__global__ void __launch_bounds__(256)
k_interp3(int64_t T, const R *__restrict__ r, const InterpRec3<R> *__restrict__ rec,
          const R *__restrict__ v, const AT *__restrict__ A, Axes3 ax, R *__restrict__ s)
{
    const int nx = ax.x.n, ny = ax.y.n;
    const int64_t N = (int64_t)nx * ny * ax.z.n;
    constexpr int K = CH < 0 ? 3 : 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < K * T;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = K == 1 ? 0 : int(e >= T) + int(e >= 2 * T);
        const int64_t t = e - k * T;
        InterpRec3<R> q;
        if constexpr (PRE) q = rec[t];
        else q = make_rec3<R>(r[3 * t], r[3 * t + 1], r[3 * t + 2], ax);
        const R vv[3] = {v[3 * t], v[3 * t + 1], v[3 * t + 2]};
        const int i0 = q.i0, j0 = q.j0, l0 = q.l0;
        const int i1 = nx > 1 ? i0 + 1 : i0, j1 = ny > 1 ? j0 + 1 : j0, l1 = ax.z.n > 1 ? l0 + 1 : l0;
        const R wx1 = q.wx1, wy1 = q.wy1, wz1 = q.wz1;
        const R wx0 = R(1) - wx1, wy0 = R(1) - wy1, wz0 = R(1) - wz1;
        const int64_t r00 = ((int64_t)l0 * ny + j0) * nx, r01 = ((int64_t)l0 * ny + j1) * nx;
        const int64_t r10 = ((int64_t)l1 * ny + j0) * nx, r11 = ((int64_t)l1 * ny + j1) * nx;
        R acc = R(0);
        if constexpr (IL) {
            const float4 *A4 = reinterpret_cast<const float4 *>(A);
            const float4 a000 = A4[(r00 + i0) * K + k], a100 = A4[(r00 + i1) * K + k];
            const float4 a010 = A4[(r01 + i0) * K + k], a110 = A4[(r01 + i1) * K + k];
            const float4 a001 = A4[(r10 + i0) * K + k], a101 = A4[(r10 + i1) * K + k];
            const float4 a011 = A4[(r11 + i0) * K + k], a111 = A4[(r11 + i1) * K + k];
            auto tri = [&](float c000, float c100, float c010, float c110, float c001, float c101, float c011,
                           float c111) {
                const R lo = wy0 * (wx0 * c000 + wx1 * c100) + wy1 * (wx0 * c010 + wx1 * c110);
                const R hi = wy0 * (wx0 * c001 + wx1 * c101) + wy1 * (wx0 * c011 + wx1 * c111);
                return wz0 * lo + wz1 * hi;
            };
            acc += tri(a000.x, a100.x, a010.x, a110.x, a001.x, a101.x, a011.x, a111.x) * vv[0];
            acc += tri(a000.y, a100.y, a010.y, a110.y, a001.y, a101.y, a011.y, a111.y) * vv[1];
            acc += tri(a000.z, a100.z, a010.z, a110.z, a001.z, a101.z, a011.z, a111.z) * vv[2];
        } else {
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const AT *F = A + (CH < 0 ? 3 * k + m : m) * N;
                const R lo = wy0 * (wx0 * R(F[r00 + i0]) + wx1 * R(F[r00 + i1])) +
                             wy1 * (wx0 * R(F[r01 + i0]) + wx1 * R(F[r01 + i1]));
                const R hi = wy0 * (wx0 * R(F[r10 + i0]) + wx1 * R(F[r10 + i1])) +
                             wy1 * (wx0 * R(F[r11 + i0]) + wx1 * R(F[r11 + i1]));
                acc += (wz0 * lo + wz1 * hi) * vv[m];
            }
        }
        s[e] = acc;
    }
}

template <typename R>
__global__ void k_cell_count3(int64_t T, const R *__restrict__ r, Axes3 ax, int ncx, int ncy,
                              int *__restrict__ cell_of, int *__restrict__ count, InterpRec3<R> *__restrict__ rec)
{
    // every lane of a warp runs the same iterations (warp_count_add)
    for (int64_t t0 = int64_t(blockIdx.x) * blockDim.x; t0 < T; t0 += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        int c = -1;
        if (t < T) {
            const InterpRec3<R> q = make_rec3<R>(r[3 * t], r[3 * t + 1], r[3 * t + 2], ax);
            rec[t] = q;
            c = (q.l0 * ncy + q.j0) * ncx + q.i0;
            cell_of[t] = c;
        }
        warp_count_add(count, c);
    }
}

// The transpose (Ahat_{3k+m}(node) = sum over the samples t of the node's
// adjacent cells of w_node(t) v_m(t) s_k(t)) runs by cell: each cell's run of
// samples (list order) is split into work units of at most kUnitLen3
// entries, one warp per unit.  Lane = 8 g + corner: the lane takes corner
// node `corner` = dx + 2 dy + 4 dz of the cell and every 4th entry from g
// (the eight corner lanes of a group read the same sample: one request per
// entry for all corners), and a fixed two-level butterfly adds the four
// groups.  The unit that completes its cell last (a per-cell arrival counter)
// adds the cell's units in order into one sum per corner and component, so a
// node combines exactly one value per adjacent cell, however many samples
// the trajectory leaves in it (a 3-D trajectory leaves most cells empty and
// piles hundreds of samples into a few).  A sample is read once instead of
// once per corner node.
#ifndef MPI_UNIT_LEN3
#define MPI_UNIT_LEN3 64
#endif
constexpr int kUnitLen3 = MPI_UNIT_LEN3;
constexpr int kT3Groups = 4;                      // entry groups per unit (lanes = 8 corners x 4)
constexpr int kT3UnitsPerBlock = kUnitThreads / 32;

__global__ void k_cunit_count3(int n_cells, const int *__restrict__ offset, int *__restrict__ cunit_cnt)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x)
        cunit_cnt[c] = (offset[c + 1] - offset[c] + kUnitLen3 - 1) / kUnitLen3;
}

__global__ void k_cunit_fill3(int n_cells, const int *__restrict__ cunit_off, int *__restrict__ unit_cell)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x)
        for (int w = cunit_off[c]; w < cunit_off[c + 1]; ++w) unit_cell[w] = c;
}

// A cell's corner sums as an unevaluated pair hi + lo (FP32: the error-free
// double-float sum of its unit sums; FP64: lo = 0).
__device__ __forceinline__ void cell_add(SumAcc<float> &a, V2<float> v) { a.s.add(F2Sum{v.x, v.y}); }
__device__ __forceinline__ void cell_add(SumAcc<double> &a, V2<double> v) { a.add(v.x); }
__device__ __forceinline__ V2<float> cell_pair(const SumAcc<float> &a) { return V2<float>{a.s.hi, a.s.lo}; }
__device__ __forceinline__ V2<double> cell_pair(const SumAcc<double> &a) { return V2<double>{a.s, 0.0}; }

// Unit sums and cell sums of the transpose: unit_part[(w 8 + corner) NC + m]
// and, at the cell's first unit u0, cell_part[(u0 8 + corner) NC + m] =
// the cell's corner-`corner` sum of w_dx w_dy w_dz v_m s_k (CH < 0: 9 sums,
// component 3k + m; CH = k: channel k only, 3 sums).  cell_cnt: zero on entry
// and on exit.
template <typename R, int CH>
__global__ void __launch_bounds__(kUnitThreads)
k_interp3_T_cells(const InterpRec3<R> *__restrict__ rec, const R *__restrict__ vs, const R *__restrict__ s,
                  int64_t T, const int *__restrict__ offset, const int *__restrict__ cunit_off,
                  const int *__restrict__ unit_cell, const int *__restrict__ n_units_dev, int n_iter,
                  R *__restrict__ unit_part, V2<R> *__restrict__ cell_part, unsigned *__restrict__ cell_cnt)
{
    constexpr int NC = CH < 0 ? 9 : 3;
    const int lane = threadIdx.x & 31, corner = lane & 7, g = lane >> 3;
    const int dx = corner & 1, dy = (corner >> 1) & 1, dz = corner >> 2;
    const int n_units = *n_units_dev;
    for (int base = blockIdx.x * kT3UnitsPerBlock; base < n_iter; base += gridDim.x * kT3UnitsPerBlock) {
        const int w = base + (int)(threadIdx.x >> 5);  // warp-uniform
        if (w >= n_units) continue;
        R acc[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) acc[m] = R(0);
        const int c = unit_cell[w];
        const int u0 = cunit_off[c], nu = cunit_off[c + 1] - u0;
        const int q0 = offset[c] + (w - u0) * kUnitLen3;
        const int q1 = min(offset[c + 1], q0 + kUnitLen3);
#pragma unroll 4
        for (int q = q0 + g; q < q1; q += kT3Groups) {
            const InterpRec3<R> rc = rec[q];
            const R wx = dx ? rc.wx1 : R(1) - rc.wx1;
            const R wy = dy ? rc.wy1 : R(1) - rc.wy1;
            const R wz = dz ? rc.wz1 : R(1) - rc.wz1;
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
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 8);
            acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], 16);
        }
        if (nu == 1) {  // the cell's only unit: its sums are the cell's
            if (g == 0) {
#pragma unroll
                for (int m = 0; m < NC; ++m) cell_part[((int64_t)u0 * 8 + corner) * NC + m] = V2<R>{acc[m], R(0)};
            }
            continue;
        }
        if (g == 0) {
#pragma unroll
            for (int m = 0; m < NC; ++m) unit_part[((int64_t)w * 8 + corner) * NC + m] = acc[m];
        }
        __threadfence();  // each lane's unit sums visible device-wide before the arrival
        __syncwarp();
        unsigned prev = 0;
        if (lane == 0) prev = atomicAdd(&cell_cnt[c], 1u);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev != unsigned(nu - 1)) continue;  // another unit of the cell finishes it
        if (lane == 0) cell_cnt[c] = 0u;
        __threadfence();
        // the four groups share the components: group g adds m = g, g + 4, ...
        for (int m = g; m < NC; m += kT3Groups) {
            SumAcc<R> a = {};
#pragma unroll 4
            for (int u = u0; u < u0 + nu; ++u) a.add(__ldcg(unit_part + ((int64_t)u * 8 + corner) * NC + m));
            cell_part[((int64_t)u0 * 8 + corner) * NC + m] = cell_pair(a);
        }
    }
}

// The combine of one node (at i, j, l), all NC components: the sums, over
// the node's adjacent non-empty cells in ascending cell order, of the cell
// sums of the corner the node is in that cell.
template <typename R, int NC>
__device__ __forceinline__ void node_combine3(int i, int j, int l, int ncx, int ncy, int ncz,
                                              const int *__restrict__ cunit_off,
                                              const V2<R> *__restrict__ cell_part, SumAcc<R> (&sum)[NC])
{
#pragma unroll
    for (int dz = 1; dz >= 0; --dz)
#pragma unroll
        for (int dy = 1; dy >= 0; --dy)
#pragma unroll
            for (int dx = 1; dx >= 0; --dx) {
                const int cl = l - dz, cj = j - dy, ci = i - dx;
                if (cl < 0 || cl >= ncz || cj < 0 || cj >= ncy || ci < 0 || ci >= ncx) continue;
                const int cc = (cl * ncy + cj) * ncx + ci;
                const int u0 = cunit_off[cc];
                if (cunit_off[cc + 1] == u0) continue;
                const V2<R> *cp = cell_part + ((int64_t)u0 * 8 + dx + 2 * dy + 4 * dz) * NC;
#pragma unroll
                for (int m = 0; m < NC; ++m) cell_add(sum[m], cp[m]);
            }
}

// Ahat_m(node) = scale * node_combine3 for all NC components.
template <typename R, typename OUT, int NC>
__global__ void k_interp3_T_cell_combine(int nx, int ny, int nz, int ncx, int ncy, int ncz,
                                         const int *__restrict__ cunit_off, const V2<R> *__restrict__ cell_part,
                                         OUT *__restrict__ A, double scale)
{
    const int N = nx * ny * nz;  // < 2^27
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N; node += gridDim.x * blockDim.x) {
        const int i = node % nx, j = (node / nx) % ny, l = node / (nx * ny);
        SumAcc<R> sum[NC] = {};
        node_combine3<R, NC>(i, j, l, ncx, ncy, ncz, cunit_off, cell_part, sum);
#pragma unroll
        for (int m = 0; m < NC; ++m) cs_store(A[(int64_t)m * N + node], sum[m].value() * scale);
    }
}

// (Lap f)(node k at i, j, l): 7-point, replicated boundary (a missing
// neighbour is the node itself), FP64.  scaled: per-axis second differences
// with 1/dx^2, 1/dy^2, 1/dz^2 (c); else the plain stencil.
template <typename E> struct Coef3 { E x, y, z; };

__device__ __forceinline__ double lap3_at(const double *__restrict__ f, int64_t k, int i, int j, int l, int nx,
                                          int ny, int nz, bool scaled, Coef3<double> c)
{
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t xm = i > 0 ? -sx : 0, xp = i < nx - 1 ? sx : 0;
    const int64_t ym = j > 0 ? -sy : 0, yp = j < ny - 1 ? sy : 0;
    const int64_t zm = l > 0 ? -sz : 0, zp = l < nz - 1 ? sz : 0;
    if (scaled) {
        const double c0 = f[k];
        return c.x * (f[k + xm] - 2.0 * c0 + f[k + xp]) + c.y * (f[k + ym] - 2.0 * c0 + f[k + yp]) +
               c.z * (f[k + zm] - 2.0 * c0 + f[k + zp]);
    }
    return f[k + xm] + f[k + xp] + f[k + ym] + f[k + yp] + f[k + zm] + f[k + zp] - 6.0 * f[k];
}
// The same in double-float arithmetic (coefficients as double-float pairs).
__device__ __forceinline__ df lap3_at(const df *__restrict__ f, int64_t k, int i, int j, int l, int nx, int ny,
                                      int nz, bool scaled, Coef3<df> c)
{
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t xm = i > 0 ? -sx : 0, xp = i < nx - 1 ? sx : 0;
    const int64_t ym = j > 0 ? -sy : 0, yp = j < ny - 1 ? sy : 0;
    const int64_t zm = l > 0 ? -sz : 0, zp = l < nz - 1 ? sz : 0;
    const df c0 = f[k];
    const df ax = df_add(f[k + xm], f[k + xp]), ay = df_add(f[k + ym], f[k + yp]), az = df_add(f[k + zm], f[k + zp]);
    if (scaled) {
        const df m2 = make_float2(-2.0f, 0.0f);
        return df_add(df_add(df_mul(df_axpy(ax, m2, c0), c.x), df_mul(df_axpy(ay, m2, c0), c.y)),
                      df_mul(df_axpy(az, m2, c0), c.z));
    }
    return df_axpy(df_add(df_add(ax, ay), az), make_float2(-6.0f, 0.0f), c0);
}

// out_m = Lap x_m for the nc components (SCALE: w Lap x_m); E: FP64 or
// double-float elements (and scalars).
template <typename E, bool SCALE>
__global__ void k_lap3(int nx, int ny, int nz, int nc, bool scaled, Coef3<E> c, const E *__restrict__ x,
                       E *__restrict__ out, E w)
{
    // nc N < 2^31 (grids of fewer than 2^27 nodes): 32-bit index arithmetic
    const int N = nx * ny * nz;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nc * N; e += gridDim.x * blockDim.x) {
        const int m = e / N, k = e - m * N;
        const int i = k % nx, j = (k / nx) % ny, l = k / (nx * ny);
        const E L = lap3_at(x + (int64_t)m * N, k, i, j, l, nx, ny, nz, scaled, c);
        out[e] = SCALE ? cs_scale(L, w) : L;
    }
}

// One Core Stage step's operator after the transpose's cell sums, one
// thread per node and all its components m: q = scale * node_combine3 + l2
// with l2 = gamma Lap Lap p (formed on the side stream), written to q, and
// the partial sums of <p, q> over blocks of kQThreads3 consecutive nodes,
// finished into alpha by the last block.  (Small blocks: a 48 x 48 x 24
// grid still spreads over about three blocks per SM.)
constexpr int kQThreads3 = 128;
template <typename R, int NC, typename E>
__global__ void __launch_bounds__(kQThreads3)
k_grid3_q(int nx, int ny, int nz, int ncx, int ncy, int ncz, const int *__restrict__ cunit_off,
          const V2<R> *__restrict__ cell_part, E scale, const E *__restrict__ l2, const E *__restrict__ p,
          E *__restrict__ q, double *__restrict__ pq_part, CsScal *sc)
{
    __shared__ double sh[kQThreads3 / 32];
    __shared__ bool last;
    const int N = nx * ny * nz;  // < 2^27
    const int node = blockIdx.x * kQThreads3 + threadIdx.x;
    CsDot<E> acc{};
    if (node < N) {
        const int i = node % nx, j = (node / nx) % ny, l = node / (nx * ny);
        SumAcc<R> sum[NC] = {};
        node_combine3<R, NC>(i, j, l, ncx, ncy, ncz, cunit_off, cell_part, sum);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            const int64_t e = (int64_t)m * N + node;
            const E qe = cs_sum_scale_add(sum[m], scale, l2[e]);
            q[e] = qe;
            acc.add(p[e], qe);
        }
    }
    const double tot = acc.template block_total<kQThreads3>(sh);
    if (threadIdx.x == 0) pq_part[blockIdx.x] = tot;
    cs_finish_pq<kQThreads3>(pq_part, gridDim.x, sc, sh, &last);
}

// Ahat and its trace (all channels: A_00 + A_11 + A_22; channel k: A_kk,
// component k of the stored row (A_k0, A_k1, A_k2)).
template <typename R, typename E>
__global__ void k_grid3_output(int64_t N, int ch, const E *__restrict__ x, R *__restrict__ A, R *__restrict__ tr)
{
    const int nc = ch < 0 ? 9 : 3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int m = 0; m < nc; ++m) A[m * N + e] = R(cs_to_double(x[m * N + e]));
        tr[e] = ch < 0 ? R(cs_to_double(cs_add(cs_add(x[e], x[4 * N + e]), x[8 * N + e])))
                       : R(cs_to_double(x[ch * N + e]));
    }
}

// Binning scratch: as the 2-D one, with 3-D records and velocities.
struct Bins3 {
    int *cell_of, *count, *offset, *list;
    void *sort_tmp;  // scratch of the ordering and the scans
    void *rec_t, *rec, *vs;
    int *cunit_cnt, *cunit_off, *unit_cell;  // transpose work units per cell
    void *unit_part;  // 8 corners x (9 or 3) sums per unit
    void *cell_part;  // V2<R>: the cell's corner sums, at its first unit's slot
    unsigned *cell_cnt;  // per-cell arrival counters of the units
    int n_units_max;  // bound on the units (allocation)
    int n_units = -1;  // the exact count when read back to the host, else -1
    int ncx, ncy, ncz;
};

inline size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Units of the cell runs: at most one per kUnitLen3 samples plus one per
// non-empty cell.
int units_bound3(int64_t T, int64_t nc)
{
    return (int)std::min<int64_t>(INT32_MAX, (T + kUnitLen3 - 1) / kUnitLen3 + std::min<int64_t>(T, nc) + 1);
}

template <typename R>
size_t bins3_bytes(int64_t T, const G3 &g)
{
    const size_t nc = size_t(std::max(g.nx - 1, 1)) * std::max(g.ny - 1, 1) * std::max(g.nz - 1, 1);
    const size_t U = size_t(units_bound3(T, int64_t(nc)));
    const size_t T1 = size_t(std::max<int64_t>(T, 1));
    return up256(sizeof(int) * T1) * 2 + up256(sizeof(int) * nc) + up256(sizeof(int) * (nc + 1)) +
           up256(std::max(cell_order_bytes(T), cell_scan_bytes(int64_t(nc)))) +
           2 * up256(sizeof(InterpRec3<R>) * T1) + up256(3 * sizeof(R) * T1) + up256(sizeof(int) * nc) +
           up256(sizeof(int) * (nc + 1)) + up256(sizeof(int) * U) + up256(8 * 9 * sizeof(R) * U) +
           up256(8 * 9 * sizeof(V2<R>) * U) + up256(sizeof(unsigned) * nc);
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
    b.offset = reinterpret_cast<int *>(p); p += up256(sizeof(int) * (nc + 1));
    b.sort_tmp = p; p += up256(std::max(cell_order_bytes(T), cell_scan_bytes(int64_t(nc))));
    b.rec_t = p; p += up256(sizeof(InterpRec3<R>) * T1);
    b.rec = p; p += up256(sizeof(InterpRec3<R>) * T1);
    b.vs = p; p += up256(3 * sizeof(R) * T1);
    b.n_units_max = units_bound3(T, int64_t(nc));
    b.cunit_cnt = reinterpret_cast<int *>(p); p += up256(sizeof(int) * nc);
    b.cunit_off = reinterpret_cast<int *>(p); p += up256(sizeof(int) * (nc + 1));
    b.unit_cell = reinterpret_cast<int *>(p); p += up256(sizeof(int) * size_t(b.n_units_max));
    b.unit_part = p; p += up256(8 * 9 * sizeof(R) * size_t(b.n_units_max));
    b.cell_part = p; p += up256(8 * 9 * sizeof(V2<R>) * size_t(b.n_units_max));
    b.cell_cnt = reinterpret_cast<unsigned *>(p);
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
    MPI_TRY_CUDA(cudaMemsetAsync(b.cell_cnt, 0, sizeof(unsigned) * nc, st));
    if (T > 0) {
        k_cell_count3<R><<<grid_blocks(T), 256, 0, st>>>(T, r, ax, b.ncx, b.ncy, b.cell_of, b.count,
                                                          static_cast<InterpRec3<R> *>(b.rec_t));
        MPI_CHECK_LAUNCH();
    }
    MPI_TRY(cell_scan_launch(b.count, nc, b.offset, b.sort_tmp, st));
    if (T > 0) {
        MPI_TRY(cell_order_launch(T, b.cell_of, nc, b.list, b.sort_tmp, st));
        k_sort_records<InterpRec3<R>, R, 3><<<grid_blocks(T), 256, 0, st>>>(
            T, b.list, static_cast<const InterpRec3<R> *>(b.rec_t), v, static_cast<InterpRec3<R> *>(b.rec),
            static_cast<R *>(b.vs));
        MPI_CHECK_LAUNCH();
    }
    // Work units of the transpose.
    k_cunit_count3<<<grid_blocks(nc), 256, 0, st>>>(nc, b.offset, b.cunit_cnt);
    MPI_CHECK_LAUNCH();
    MPI_TRY(cell_scan_launch(b.cunit_cnt, nc, b.cunit_off, b.sort_tmp, st));
    k_cunit_fill3<<<grid_blocks(nc), 256, 0, st>>>(nc, b.cunit_off, b.unit_cell);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// il: the FP32 field in the node-interleaved layout of k_round_field3_il
// (records precomputed).
template <typename R, typename AT>
int launch_interp3(const G3 &g, int64_t T, const R *r, const R *v, const AT *A, R *s, cudaStream_t st,
                   int ch = -1, const InterpRec3<R> *rec = nullptr, bool il = false)
{
    if (T == 0) return MPI_OK;
    const Axes3 ax = axes_of(g);
    const int64_t outs = (ch < 0 ? 3 : 1) * T;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((outs + 255) / 256, 16384));
    if constexpr (sizeof(AT) == 4) {
        if (il) {
            if (ch < 0) k_interp3<R, AT, -1, true, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, s);
            else k_interp3<R, AT, 0, true, true><<<blocks, 256, 0, st>>>(T, r, rec, v, A, ax, s);
            MPI_CHECK_LAUNCH();
            return MPI_OK;
        }
    }
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

// The transpose's unit sums (k_interp3_T_cells) into b.unit_part.
// s_sorted: the samples' values in list order ([rows][T]).
template <typename R>
int launch_interp3_T_units(int64_t T, const R *s_sorted, const Bins3 &b, cudaStream_t st, int ch)
{
    const int nc = b.ncx * b.ncy * b.ncz;
    constexpr int per_block = kT3UnitsPerBlock;
    // Blocks for the exact unit count where the host has it, else for the
    // bound (the real count is on the device, cunit_off[nc], and surplus
    // blocks exit at once).
    const int units = b.n_units >= 0 ? b.n_units : b.n_units_max;
    const int n_iter = (units + per_block - 1) / per_block * per_block;
    const unsigned blocks = (unsigned)std::max(1, std::min(n_iter / per_block, 65535));
    const InterpRec3<R> *rec = static_cast<const InterpRec3<R> *>(b.rec);
    const R *vs = static_cast<const R *>(b.vs);
    R *part = static_cast<R *>(b.unit_part);
    V2<R> *cpart = static_cast<V2<R> *>(b.cell_part);
    const int *n_units = b.cunit_off + nc;
    if (ch < 0)
        k_interp3_T_cells<R, -1><<<blocks, kUnitThreads, 0, st>>>(rec, vs, s_sorted, T, b.offset, b.cunit_off,
                                                                  b.unit_cell, n_units, n_iter, part, cpart,
                                                                  b.cell_cnt);
    else
        k_interp3_T_cells<R, 0><<<blocks, kUnitThreads, 0, st>>>(rec, vs, s_sorted, T, b.offset, b.cunit_off,
                                                                 b.unit_cell, n_units, n_iter, part, cpart,
                                                                 b.cell_cnt);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// A = scale M^T s (all nine components, or channel ch's three).
template <typename R, typename OUT>
int launch_interp3_T(const G3 &g, int64_t T, const R *s_sorted, const Bins3 &b, OUT *A, double scale,
                     cudaStream_t st, int ch = -1)
{
    MPI_TRY(launch_interp3_T_units<R>(T, s_sorted, b, st, ch));
    const int64_t N = g.n();
    const V2<R> *cpart = static_cast<const V2<R> *>(b.cell_part);
    if (ch < 0)
        k_interp3_T_cell_combine<R, OUT, 9><<<grid_blocks(N), 256, 0, st>>>(
            g.nx, g.ny, g.nz, b.ncx, b.ncy, b.ncz, b.cunit_off, cpart, A, scale);
    else
        k_interp3_T_cell_combine<R, OUT, 3><<<grid_blocks(N), 256, 0, st>>>(
            g.nx, g.ny, g.nz, b.ncx, b.ncy, b.ncz, b.cunit_off, cpart, A, scale);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// The 3-D Core Stage operator: (1/T) M^T M through the binned records and
// the 7-point Laplacian of each component.  A step: l2 = gamma Lap Lap p on
// the side stream (two FP64-bound passes) while the main chain runs M p
// (through the FP32 copy of p on the FP32 path) and the transpose's unit
// and cell sums; then one pass forms q and the <p, q> partials (k_grid3_q).
template <typename R>
struct GridOp3 final : CoreStageOp<typename CsElem<R>::type> {
    using E = typename CsElem<R>::type;
    const G3 &g;
    int64_t T;
    int ch, nc;
    const Bins3 &bins;
    R *s_tmp;
    float4 *p_il;  // FP32 path: the FP32 copy of p, K float4 rows per node; FP64: unused
    double invT;
    bool scaled;
    GridOp3(const G3 &g_, int64_t T_, int ch_, const Bins3 &b_, R *s_tmp_, float4 *p_il_, bool scaled_)
        : g(g_), T(T_), ch(ch_), nc(ch_ < 0 ? 9 : 3), bins(b_), s_tmp(s_tmp_), p_il(p_il_),
          invT(T_ > 0 ? 1.0 / double(T_) : 0.0), scaled(scaled_) {}
    Coef3<E> lap_coef() const
    {
        E *tag = nullptr;
        return Coef3<E>{cs_host_scalar(1.0 / (g.dx * g.dx), tag), cs_host_scalar(1.0 / (g.dy * g.dy), tag),
                        cs_host_scalar(1.0 / (g.dz * g.dz), tag)};
    }
    P32 p32() const override
    {
        if constexpr (sizeof(R) == 4)
            return P32{reinterpret_cast<float *>(p_il), ch < 0 ? kP32Rows3x4 : kP32Rows1x4, g.n()};
        return P32{};
    }
    int pq_blocks(int64_t) const override { return (int)((g.n() + kQThreads3 - 1) / kQThreads3); }
    int step_q(const E *p, double gamma, E *q, double *pq_part, CsScal *sc, E *l1, E *l2, const StepFork &fk,
               cudaStream_t st) override
    {
        E *tag = nullptr;
        const int lb = grid_blocks(nc * g.n());
        MPI_TRY_CUDA(cudaEventRecord(fk.fork, st));
        MPI_TRY_CUDA(cudaStreamWaitEvent(fk.side, fk.fork, 0));
        k_lap3<E, false><<<lb, 256, 0, fk.side>>>(g.nx, g.ny, g.nz, nc, scaled, lap_coef(), p, l1,
                                                 cs_host_scalar(1.0, tag));
        MPI_CHECK_LAUNCH();
        k_lap3<E, true><<<lb, 256, 0, fk.side>>>(g.nx, g.ny, g.nz, nc, scaled, lap_coef(), l1, l2,
                                                cs_host_scalar(gamma, tag));
        MPI_CHECK_LAUNCH();
        MPI_TRY_CUDA(cudaEventRecord(fk.join, fk.side));
        const InterpRec3<R> *rec = static_cast<const InterpRec3<R> *>(bins.rec);
        const R *vs = static_cast<const R *>(bins.vs);
        if constexpr (sizeof(R) == 4)
            MPI_TRY((launch_interp3<R, float>(g, T, nullptr, vs, reinterpret_cast<const float *>(p_il), s_tmp, st,
                                              ch, rec, true)));
        else
            MPI_TRY((launch_interp3<R, double>(g, T, nullptr, vs, reinterpret_cast<const double *>(p), s_tmp, st,
                                               ch, rec)));
        MPI_TRY(launch_interp3_T_units<R>(T, s_tmp, bins, st, ch));
        MPI_TRY_CUDA(cudaStreamWaitEvent(st, fk.join, 0));
        const unsigned blocks = (unsigned)pq_blocks(0);
        const V2<R> *cpart = static_cast<const V2<R> *>(bins.cell_part);
        const E sc_T = cs_host_scalar(invT, tag);
        if (ch < 0)
            k_grid3_q<R, 9, E><<<blocks, kQThreads3, 0, st>>>(g.nx, g.ny, g.nz, bins.ncx, bins.ncy, bins.ncz,
                                                             bins.cunit_off, cpart, sc_T, l2, p, q, pq_part, sc);
        else
            k_grid3_q<R, 3, E><<<blocks, kQThreads3, 0, st>>>(g.nx, g.ny, g.nz, bins.ncx, bins.ncy, bins.ncz,
                                                             bins.cunit_off, cpart, sc_T, l2, p, q, pq_part, sc);
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
    using E = typename CsElem<R>::type;
    const size_t o_b = scr.reserve(sizeof(E) * nv), o_x = scr.reserve(sizeof(E) * nv);
    const size_t o_pr = scr.reserve(sizeof(R) == 4 ? sizeof(float4) * rows * N : 0);
    MPI_TRY(scr.allocate());
    Bins3 bins = bins3_carve<R>(scr.at<char>(o_bins), T, g);
    R *s_data = scr.at<R>(o_sd);
    E *b = scr.at<E>(o_b), *x = scr.at<E>(o_x);

    MPI_TRY(build_bins3<R>(g, T, r, v, bins, st));
    MPI_TRY(gather_rows<R>(T, rows, bins.list, s, s_data, st));
    // The transpose runs a few thousand times with the same units: read their
    // count once, so every launch covers exactly them.
    {
        const int n_cells = bins.ncx * bins.ncy * bins.ncz;
        int n_units = 0;
        MPI_TRY_CUDA(cudaMemcpyAsync(&n_units, bins.cunit_off + n_cells, sizeof(int), cudaMemcpyDeviceToHost, st));
        MPI_TRY_CUDA(cudaStreamSynchronize(st));
        if (n_units < 0 || n_units > bins.n_units_max) {
            set_error("3-D Core Stage: %d work units exceed the bound %d", n_units, bins.n_units_max);
            return MPI_ERR_CUDA;
        }
        bins.n_units = n_units;
    }
    GridOp3<R> op(g, T, ch, bins, scr.at<R>(o_s), scr.at<float4>(o_pr), o.lap_scaled != 0);
    MPI_TRY((launch_interp3_T<R, E>(g, T, s_data, bins, b, op.invT, st, ch)));
    MPI_TRY(core_stage_cg<E>(op, nv, b, o, x, n_iter_out, st));
    k_grid3_output<R, E><<<grid_blocks(N), 256, 0, st>>>(N, ch, x, static_cast<R *>(Ahat), static_cast<R *>(trace));
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
