// Host launchers of the pair sums, the geometry preparation and the
// deterministic partial-sum reductions.
#include <algorithm>
#include <cmath>

#include "pair_kernels.cuh"

namespace mpi {

// ---------------------------------------------------------------------------
// Geometry preparation: beta G applied to sample positions/velocities and to
// voxel-centre coordinates, in FP64, rounded once to R.

template <typename R, typename IN>
__global__ void k_prepare_samples(const IN *__restrict__ r, const IN *__restrict__ v, int64_t T,
                                  double b00, double b01, double b10, double b11,
                                  V4<R> *__restrict__ rw)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double rx = double(r[2 * t]), ry = double(r[2 * t + 1]);
        const double vx = double(v[2 * t]), vy = double(v[2 * t + 1]);
        rw[t] = V4<R>{R(b00 * rx + b01 * ry), R(b10 * rx + b11 * ry),
                      R(b00 * vx + b01 * vy), R(b10 * vx + b11 * vy)};
    }
}

template <typename R>
__global__ void k_prepare_grid(int nx, int ny, double x0, double y0, double dx, double dy,
                               double b00, double b01, double b10, double b11,
                               V2<R> *__restrict__ xcol, V2<R> *__restrict__ yrow)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nx) {
        const double x = x0 + (k + 0.5) * dx;
        xcol[k] = V2<R>{R(b00 * x), R(b10 * x)};
    }
    if (k < ny) {
        const double y = y0 + (k + 0.5) * dy;
        yrow[k] = V2<R>{R(b01 * y), R(b11 * y)};
    }
}

template <typename R>
size_t geometry_bytes(int64_t T, int nx, int ny)
{
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    return up(sizeof(V4<R>) * size_t(std::max<int64_t>(T, 1))) + up(sizeof(V2<R>) * nx) +
           up(sizeof(V2<R>) * ny);
}

template <typename R>
Geometry<R> geometry_carve(void *base, int64_t T, int nx, int ny)
{
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    char *p = static_cast<char *>(base);
    Geometry<R> g;
    g.rw = reinterpret_cast<V4<R> *>(p);
    p += up(sizeof(V4<R>) * size_t(std::max<int64_t>(T, 1)));
    g.xcol = reinterpret_cast<V2<R> *>(p);
    p += up(sizeof(V2<R>) * nx);
    g.yrow = reinterpret_cast<V2<R> *>(p);
    return g;
}

template <typename R>
int prepare_geometry(const ModelH &m, const GridH &g, int64_t T, const void *r, const void *v,
                     const Geometry<R> &geo, cudaStream_t st)
{
    const double b00 = m.beta * m.G[0], b01 = m.beta * m.G[1];
    const double b10 = m.beta * m.G[2], b11 = m.beta * m.G[3];
    if (T > 0) {
        const int blocks = (int)std::min<int64_t>((T + 255) / 256, 4096);
        k_prepare_samples<R, R><<<blocks, 256, 0, st>>>(static_cast<const R *>(r),
                                                        static_cast<const R *>(v), T, b00, b01,
                                                        b10, b11, geo.rw);
        MPI_CHECK_LAUNCH();
    }
    const int n = std::max(g.nx, g.ny);
    k_prepare_grid<R><<<(n + 127) / 128, 128, 0, st>>>(g.nx, g.ny, g.x0, g.y0, g.dx, g.dy, b00,
                                                       b01, b10, b11, geo.xcol, geo.yrow);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// ---------------------------------------------------------------------------
// Work decomposition.

// Work items per operator launch: enough that the blocks' uneven costs (near
// pairs cost more than far ones) leave little idle time at the end.  The
// forward takes fewer, larger items (its row chunks also set the size of the
// partial sums it reduces): at 128 x 128 / 65 536 samples 32 per SM ran 1.2 %
// faster than 64 with half the partial sums; the adjoint keeps 64 (32 made
// the 512 x 512 adjoint 2 % slower).
#ifndef MPI_TARGET_MULT
#define MPI_TARGET_MULT 64
#endif
#ifndef MPI_TARGET_MULT_FWD
#define MPI_TARGET_MULT_FWD 32
#endif
int default_target_items() { return MPI_TARGET_MULT * device_sm_count(); }
int forward_target_items() { return MPI_TARGET_MULT_FWD * device_sm_count(); }

FwdSplit forward_split(int64_t T, int nx, int ny, int elem_bytes, int target_items)
{
    FwdSplit sp;
    sp.n_tiles = (int)std::max<int64_t>(1, (T + kFwdTile - 1) / kFwdTile);
    int want = (target_items + sp.n_tiles - 1) / sp.n_tiles;
    want = std::max(1, std::min(want, ny));
    sp.chunk_rows = (ny + want - 1) / want;
    sp.n_chunks = (ny + sp.chunk_rows - 1) / sp.chunk_rows;
    // rows staged at a time: small enough that the block's shared memory never
    // limits occupancy below the register limit
    sp.rows_staged = fwd_rows_staged(sp.chunk_rows, nx, elem_bytes);
    return sp;
}

AdjSplit adjoint_split(int64_t T, int nx, int ny, int target_items, int elem_bytes)
{
    AdjSplit sp;
    sp.tiles_x = (nx + kAdjTileX - 1) / kAdjTileX;
    sp.tiles_y = (ny + kAdjTileY - 1) / kAdjTileY;
    const int n_tiles = sp.tiles_x * sp.tiles_y;
    const int64_t blocks = std::max<int64_t>(1, (T + kAdjBlock - 1) / kAdjBlock);
    int64_t want = (target_items + n_tiles - 1) / n_tiles;
    want = std::max<int64_t>(1, std::min(want, blocks));
    const int64_t per = (blocks + want - 1) / want;  // staged blocks per chunk
    sp.chunk_len = (int)(per * kAdjBlock);
    // Small problems (a few tiles, a few staged blocks) would leave most SMs
    // idle with whole-block chunks: split the samples finer, down to 32 per
    // chunk in FP32 and 8 in FP64 (whose pair is ~10x dearer), so that there
    // are about four items per SM.
    const int64_t min_items = std::max(1, target_items / 16);
    if ((int64_t)n_tiles * blocks < min_items && T > 0) {
        const int64_t floor_len = elem_bytes == 8 ? 8 : 32;
        const int64_t chunks = (min_items + n_tiles - 1) / n_tiles;
        int64_t len = (T + chunks - 1) / chunks;
        len = (len + floor_len - 1) / floor_len * floor_len;
        sp.chunk_len = (int)std::min<int64_t>(kAdjBlock, std::max(floor_len, len));
    }
    sp.n_chunks = (int)std::max<int64_t>(1, (T + sp.chunk_len - 1) / sp.chunk_len);
    return sp;
}

// ---------------------------------------------------------------------------
// Item dispatch orders (heavy items first).

// Box of the prescaled sample positions B r_t over each `per` samples:
// (lo.x, lo.y, hi.x, hi.y).  One warp per box.
template <typename R>
__global__ void k_sample_boxes(const V4<R> *__restrict__ rw, int64_t T, int64_t per, int64_t n_box,
                               V4<R> *__restrict__ box)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= n_box) return;
    const int64_t a0 = b * per, a1 = std::min<int64_t>(T, a0 + per);
    const V4<R> q0 = rw[a0];
    R lx = q0.x, ly = q0.y, hx = q0.x, hy = q0.y;
    for (int64_t t = a0 + lane; t < a1; t += 32) {
        const V4<R> q = rw[t];
        lx = min(lx, q.x), ly = min(ly, q.y), hx = max(hx, q.x), hy = max(hy, q.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = min(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = min(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        hx = max(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = max(hy, __shfl_xor_sync(0xffffffffu, hy, o));
    }
    if (lane == 0) box[b] = V4<R>{lx, ly, hx, hy};
}

// Box of the prescaled voxel positions xcol[i] + yrow[j] over columns
// [i0, i1] and rows [j0, j1] (both maps are affine: the ends bound them).
template <typename R>
__device__ __forceinline__ V4<R> voxel_box(const V2<R> *xcol, const V2<R> *yrow, int i0, int i1,
                                           int j0, int j1)
{
    const V2<R> a = xcol[i0], b = xcol[i1], c = yrow[j0], d = yrow[j1];
    return V4<R>{min(a.x, b.x) + min(c.x, d.x), min(a.y, b.y) + min(c.y, d.y),
                 max(a.x, b.x) + max(c.x, d.x), max(a.y, b.y) + max(c.y, d.y)};
}

constexpr int kOrderThreads = 1024;

// Stable partition of the n items: heavy (sample box within the asymptotic
// radius of the voxel box) first.  ADJ selects the adjoint item layout
// (tile = 32 x kAdjTileY voxels, chunk = chunk_len samples) or the forward
// one (tile = kFwdTile samples, chunk = chunk_rows rows of all columns).
template <typename R, bool ADJ>
__global__ void __launch_bounds__(kOrderThreads)
k_item_order(int64_t n, int n_tiles, int tiles_x, int chunk, int nx, int ny,
             const V2<R> *__restrict__ xcol, const V2<R> *__restrict__ yrow,
             const V4<R> *__restrict__ sbox, int *__restrict__ order)
{
    __shared__ int s_h[32], s_l[32];
    __shared__ int s_base[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    auto heavy = [&](int64_t it) -> bool {
        const int c = (int)(it / n_tiles), tile = (int)(it % n_tiles);
        V4<R> vb, sb;
        if (ADJ) {
            const int tx = tile % tiles_x, ty = tile / tiles_x;
            const int i0 = tx * kAdjTileX, j0 = ty * kAdjTileY;
            vb = voxel_box(xcol, yrow, i0, min(nx - 1, i0 + kAdjTileX - 1), j0, min(ny - 1, j0 + kAdjTileY - 1));
            sb = sbox[c];
        } else {
            const int j0 = c * chunk;
            vb = voxel_box(xcol, yrow, 0, nx - 1, j0, min(ny - 1, j0 + chunk - 1));
            sb = sbox[tile];
        }
        const R gx = max(R(0), max(vb.x - sb.z, sb.x - vb.z));
        const R gy = max(R(0), max(vb.y - sb.w, sb.y - vb.w));
        return gx * gx + gy * gy < vfar_threshold<R, false>();
    };
    int n_heavy = 0;
    for (int64_t b = 0; b < n; b += kOrderThreads) {
        const int64_t it = b + threadIdx.x;
        n_heavy += __syncthreads_count(it < n && heavy(it));
    }
    if (threadIdx.x == 0) s_base[0] = 0, s_base[1] = n_heavy;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t b = 0; b < n; b += kOrderThreads) {
        const int64_t it = b + threadIdx.x;
        const bool valid = it < n;
        const bool hv = valid && heavy(it);
        const unsigned hb = __ballot_sync(0xffffffffu, hv), lb = __ballot_sync(0xffffffffu, valid && !hv);
        if (lane == 0) s_h[w] = __popc(hb), s_l[w] = __popc(lb);
        __syncthreads();
        int hpre = 0, lpre = 0, htot = 0, ltot = 0;
        for (int k = 0; k < kOrderThreads / 32; ++k) {
            if (k < w) hpre += s_h[k], lpre += s_l[k];
            htot += s_h[k], ltot += s_l[k];
        }
        if (hv) order[s_base[0] + hpre + __popc(hb & lt)] = (int)it;
        else if (valid) order[s_base[1] + lpre + __popc(lb & lt)] = (int)it;
        __syncthreads();
        if (threadIdx.x == 0) s_base[0] += htot, s_base[1] += ltot;
        __syncthreads();
    }
}

template <typename R>
size_t item_order_bytes(const FwdSplit *fs, const AdjSplit *as)
{
    size_t b = 4 * 256;
    if (fs) b += sizeof(int) * size_t(fs->n_tiles) * fs->n_chunks + sizeof(V4<R>) * fs->n_tiles;
    if (as) b += sizeof(int) * size_t(as->tiles_x) * as->tiles_y * as->n_chunks + sizeof(V4<R>) * as->n_chunks;
    return b;
}

template <typename R>
int prepare_item_orders(const GridH &g, int64_t T, const Geometry<R> &geo, FwdSplit *fs, AdjSplit *as,
                        void *scratch, cudaStream_t st)
{
    if (fs) fs->order = nullptr;
    if (as) as->order = nullptr;
    if (T == 0) return MPI_OK;
    char *p = static_cast<char *>(scratch);
    auto take = [&](size_t b) {
        char *q = p;
        p += (b + 255) & ~size_t(255);
        return q;
    };
    if (fs) {
        const int64_t nf = (int64_t)fs->n_tiles * fs->n_chunks;
        int *fo = reinterpret_cast<int *>(take(sizeof(int) * nf));
        V4<R> *fb = reinterpret_cast<V4<R> *>(take(sizeof(V4<R>) * fs->n_tiles));
        if (nf <= INT32_MAX) {
            k_sample_boxes<R><<<(unsigned)((int64_t(fs->n_tiles) * 32 + 255) / 256), 256, 0, st>>>(
                geo.rw, T, kFwdTile, fs->n_tiles, fb);
            MPI_CHECK_LAUNCH();
            k_item_order<R, false><<<1, kOrderThreads, 0, st>>>(nf, fs->n_tiles, 0, fs->chunk_rows, g.nx,
                                                                g.ny, geo.xcol, geo.yrow, fb, fo);
            MPI_CHECK_LAUNCH();
            fs->order = fo;
        }
    }
    if (as) {
        const int64_t na = (int64_t)as->tiles_x * as->tiles_y * as->n_chunks;
        int *ao = reinterpret_cast<int *>(take(sizeof(int) * na));
        V4<R> *ab = reinterpret_cast<V4<R> *>(take(sizeof(V4<R>) * as->n_chunks));
        if (na <= INT32_MAX) {
            k_sample_boxes<R><<<(unsigned)((int64_t(as->n_chunks) * 32 + 255) / 256), 256, 0, st>>>(
                geo.rw, T, as->chunk_len, as->n_chunks, ab);
            MPI_CHECK_LAUNCH();
            k_item_order<R, true><<<1, kOrderThreads, 0, st>>>(na, as->tiles_x * as->tiles_y, as->tiles_x,
                                                               as->chunk_len, g.nx, g.ny, geo.xcol,
                                                               geo.yrow, ab, ao);
            MPI_CHECK_LAUNCH();
            as->order = ao;
        }
    }
    return MPI_OK;
}

template size_t item_order_bytes<float>(const FwdSplit *, const AdjSplit *);
template size_t item_order_bytes<double>(const FwdSplit *, const AdjSplit *);
template int prepare_item_orders<float>(const GridH &, int64_t, const Geometry<float> &, FwdSplit *,
                                        AdjSplit *, void *, cudaStream_t);
template int prepare_item_orders<double>(const GridH &, int64_t, const Geometry<double> &, FwdSplit *,
                                         AdjSplit *, void *, cudaStream_t);

template <typename R>
size_t forward_partial_bytes(const FwdSplit &sp, int n_ch, int64_t T)
{
    return sizeof(R) * size_t(sp.n_chunks) * n_ch * size_t(std::max<int64_t>(T, 1));
}
template <typename R>
size_t adjoint_partial_bytes(const AdjSplit &sp, int nx, int ny)
{
    return sizeof(R) * size_t(sp.n_chunks) * size_t(nx) * ny;
}
size_t dbeta_partial_bytes(const AdjSplit &sp)
{
    return sizeof(double) * size_t(sp.n_chunks) * sp.tiles_x * sp.tiles_y;
}

// ---------------------------------------------------------------------------
// Reductions over chunks, in FP64 and in a fixed order.

// Sum over chunks of the partial slices part[c][e], e < len.  A block owns 32
// consecutive elements; warp w sums chunks w, w+8, ... (coalesced rows of
// 128 B), and warp 0 adds the eight warp sums in order.  FP32 partials are
// summed as error-free double-float pairs (SumAcc), FP64 ones in FP64.  With
// CG set the epilogue writes out = sum + nu * p (FP64) and the block's partial
// sum of <p, out> to dot_part[blockIdx.x].
constexpr int kRedThreads = 256;
constexpr int kRedWarps = kRedThreads / 32;

template <typename R, typename OUT, bool CG>
__global__ void __launch_bounds__(kRedThreads)
k_reduce_chunks(const R *__restrict__ part, int n_chunks, int64_t len, OUT *__restrict__ out,
                const double *__restrict__ p, const double *__restrict__ nu_dev,
                double *__restrict__ dot_part)
{
    __shared__ SumAcc<R> sh[kRedWarps][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + lane;
    SumAcc<R> acc{};
    if (e < len) {
        // Sequential sum over this warp's chunks; the unroll only lets the
        // loads run ahead (the additions keep their order).
#pragma unroll 8
        for (int c = w; c < n_chunks; c += kRedWarps) acc.add(part[(int64_t)c * len + e]);
    }
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0) {
        SumAcc<R> all{};
#pragma unroll
        for (int k = 0; k < kRedWarps; ++k) all.add(sh[k][lane]);
        double tot = all.value();
        if constexpr (CG) {
            const double pe = e < len ? p[e] : 0.0;
            tot += *nu_dev * pe;
            if (e < len) out[e] = OUT(tot);
            const double dot = warp_sum(pe * tot);
            if (lane == 0) dot_part[blockIdx.x] = dot;
        } else {
            if (e < len) out[e] = OUT(tot);
        }
    }
}

int adjoint_dot_blocks(int nx, int ny) { return (int)(((int64_t)nx * ny + 31) / 32); }
int reduce_dot_blocks(int64_t len) { return (int)((len + 31) / 32); }

static unsigned reduce_blocks(int64_t len) { return (unsigned)std::max<int64_t>(1, (len + 31) / 32); }

template <typename R, typename OUT>
int reduce_chunks(const R *part, int n_chunks, int64_t len, OUT *out, const double *cg_p,
                  const double *nu_dev, double *dot_part, cudaStream_t st)
{
    if (cg_p) {
        if constexpr (sizeof(OUT) == sizeof(double)) {
            k_reduce_chunks<R, double, true><<<reduce_blocks(len), kRedThreads, 0, st>>>(
                part, n_chunks, len, reinterpret_cast<double *>(out), cg_p, nu_dev, dot_part);
        } else {
            set_error("internal: CG epilogue needs FP64 output");
            return MPI_ERR_INVALID;
        }
    } else {
        k_reduce_chunks<R, OUT, false><<<reduce_blocks(len), kRedThreads, 0, st>>>(
            part, n_chunks, len, out, nullptr, nullptr, nullptr);
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template int reduce_chunks<float, float>(const float *, int, int64_t, float *, const double *,
                                         const double *, double *, cudaStream_t);
template int reduce_chunks<float, double>(const float *, int, int64_t, double *, const double *,
                                          const double *, double *, cudaStream_t);
template int reduce_chunks<double, double>(const double *, int, int64_t, double *, const double *,
                                           const double *, double *, cudaStream_t);

__global__ void k_sum_fixed(const double *__restrict__ part, int n, double scale,
                            double *__restrict__ out)
{
    __shared__ double sh[kRedWarps];
    double acc = 0.0;
    // fixed assignment of parts to threads, fixed tree: deterministic
    for (int k = threadIdx.x; k < n; k += kRedThreads) acc += part[k];
    acc = block_sum<double, kRedThreads>(acc, sh);
    if (threadIdx.x == 0) *out = acc * scale;
}

// ---------------------------------------------------------------------------
// Launchers.

static bool is_diag(const ModelH &m) { return m.G[1] == 0.0 && m.G[2] == 0.0; }

// Half-width (in columns) of the window around a sample that can hold a pair
// with u < near_u: sqrt(near_u) / |beta G_00 dx|, plus one for rounding.
template <typename R>
int near_columns(const ModelH &m, const GridH &g)
{
    const double pitch = std::fabs(m.beta * m.G[0] * g.dx);
    const double w = std::sqrt(double(Lang<R>::near_u)) / std::max(pitch, 1e-300);
    return (int)std::min<double>(std::ceil(w) + 1.0, (double)g.nx);
}
template int near_columns<float>(const ModelH &, const GridH &);

template <typename R>
static PairFrame<R> base_frame(const ModelH &m, const GridH &g, int64_t T, const Geometry<R> &geo)
{
    PairFrame<R> f{};
    f.rw = geo.rw;
    f.xcol = geo.xcol;
    f.yrow = geo.yrow;
    f.T = T;
    f.item0 = 0;
    f.nx = g.nx;
    f.ny = g.ny;
    f.n_ch = m.n_ch;
    for (int k = 0; k < 4; ++k) f.p[k] = R(m.p[k]);
    return f;
}

template <typename Kern>
static int set_smem(Kern k, size_t bytes)
{
    if (bytes > 48 * 1024)
        MPI_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return MPI_OK;
}

template <typename R, typename CIN, typename OUT>
int launch_forward(const ModelH &m, const GridH &g, int64_t T, const Geometry<R> &geo,
                   const FwdSplit &sp, const CIN *c, R *part, OUT *s_out, cudaStream_t st)
{
    if (T == 0) return MPI_OK;
    PairBatch<R, 1> B;
    B.n_frames = 1;
    B.f[0] = base_frame(m, g, T, geo);
    B.f[0].in = c;
    B.f[0].part = part;
    B.f[0].n_tiles = sp.n_tiles;
    B.f[0].chunk = sp.chunk_rows;
    B.f[0].rows_staged = sp.rows_staged;
    B.f[0].near_cols = near_columns<R>(m, g);
    B.f[0].order = sp.order;
    const size_t smem = fwd_smem_bytes(g.nx, sp.rows_staged, sizeof(R));
    const int64_t items = (int64_t)sp.n_tiles * sp.n_chunks;
    {
        ProfScope prof(kProfForward, st);
        if (is_diag(m)) {
            MPI_TRY(set_smem(k_forward<R, CIN, 1, 1>, smem));
            k_forward<R, CIN, 1, 1><<<(unsigned)items, kFwdThreads, smem, st>>>(B);
        } else {
            MPI_TRY(set_smem(k_forward<R, CIN, 0, 1>, smem));
            k_forward<R, CIN, 0, 1><<<(unsigned)items, kFwdThreads, smem, st>>>(B);
        }
        MPI_CHECK_LAUNCH();
    }
    const int64_t len = (int64_t)m.n_ch * T;
    k_reduce_chunks<R, OUT, false><<<reduce_blocks(len), kRedThreads, 0, st>>>(
        part, sp.n_chunks, len, s_out, nullptr, nullptr, nullptr);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename R, typename OUT>
int launch_adjoint(const ModelH &m, const GridH &g, int64_t T, const Geometry<R> &geo,
                   const AdjSplit &sp, const R *s, R *part, OUT *out, const double *cg_p,
                   const double *nu_dev, double *dot_part, cudaStream_t st)
{
    const int64_t N = (int64_t)g.nx * g.ny;
    if (T > 0) {
        PairBatch<R, 1> B;
        B.n_frames = 1;
        B.f[0] = base_frame(m, g, T, geo);
        B.f[0].in = s;
        B.f[0].part = part;
        B.f[0].n_tiles = sp.tiles_x * sp.tiles_y;
        B.f[0].tiles_x = sp.tiles_x;
        B.f[0].chunk = sp.chunk_len;
        B.f[0].order = sp.order;
        const int64_t items = (int64_t)sp.tiles_x * sp.tiles_y * sp.n_chunks;
        const bool one = sp.chunk_len <= kAdjBlock;  // one staged block per chunk
        ProfScope prof(kProfAdjoint, st);
        if (is_diag(m)) {
            if (one) k_adjoint<R, 1, false, 1, true><<<(unsigned)items, kAdjThreads, 0, st>>>(B);
            else k_adjoint<R, 1, false, 1, false><<<(unsigned)items, kAdjThreads, 0, st>>>(B);
        } else {
            if (one) k_adjoint<R, 0, false, 1, true><<<(unsigned)items, kAdjThreads, 0, st>>>(B);
            else k_adjoint<R, 0, false, 1, false><<<(unsigned)items, kAdjThreads, 0, st>>>(B);
        }
        MPI_CHECK_LAUNCH();
    } else {
        MPI_TRY_CUDA(cudaMemsetAsync(part, 0, sizeof(R) * N, st));
    }
    const int nch = T > 0 ? sp.n_chunks : 1;
    if (cg_p) {
        if constexpr (sizeof(OUT) == sizeof(double)) {
            k_reduce_chunks<R, double, true><<<reduce_blocks(N), kRedThreads, 0, st>>>(
                part, nch, N, reinterpret_cast<double *>(out), cg_p, nu_dev, dot_part);
        } else {
            set_error("internal: CG epilogue needs FP64 output");
            return MPI_ERR_INVALID;
        }
    } else {
        k_reduce_chunks<R, OUT, false><<<reduce_blocks(N), kRedThreads, 0, st>>>(
            part, nch, N, out, nullptr, nullptr, nullptr);
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename R>
int launch_dbeta(const ModelH &m, const GridH &g, int64_t T, const Geometry<R> &geo,
                 const AdjSplit &sp, const R *c, const R *gs, double *part, double *out_dev,
                 cudaStream_t st)
{
    if (T == 0) {
        MPI_TRY_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double), st));
        return MPI_OK;
    }
    PairBatch<R, 1> B;
    B.n_frames = 1;
    B.f[0] = base_frame(m, g, T, geo);
    B.f[0].in = c;
    B.f[0].in2 = gs;
    B.f[0].part = part;
    B.f[0].n_tiles = sp.tiles_x * sp.tiles_y;
    B.f[0].tiles_x = sp.tiles_x;
    B.f[0].chunk = sp.chunk_len;
    B.f[0].order = sp.order;
    const int64_t items = (int64_t)sp.tiles_x * sp.tiles_y * sp.n_chunks;
    {
        ProfScope prof(kProfDbeta, st);
        if (is_diag(m))
            k_adjoint<R, 1, true, 1><<<(unsigned)items, kAdjThreads, 0, st>>>(B);
        else
            k_adjoint<R, 0, true, 1><<<(unsigned)items, kAdjThreads, 0, st>>>(B);
        MPI_CHECK_LAUNCH();
    }
    // The kernel sums u . (beta D) with W = beta G v; divide by beta.
    k_sum_fixed<<<1, kRedThreads, 0, st>>>(part, (int)items, 1.0 / m.beta, out_dev);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// ---------------------------------------------------------------------------
// Instantiations.

template size_t geometry_bytes<float>(int64_t, int, int);
template size_t geometry_bytes<double>(int64_t, int, int);
template Geometry<float> geometry_carve<float>(void *, int64_t, int, int);
template Geometry<double> geometry_carve<double>(void *, int64_t, int, int);
template int prepare_geometry<float>(const ModelH &, const GridH &, int64_t, const void *,
                                     const void *, const Geometry<float> &, cudaStream_t);
template int prepare_geometry<double>(const ModelH &, const GridH &, int64_t, const void *,
                                      const void *, const Geometry<double> &, cudaStream_t);
template size_t forward_partial_bytes<float>(const FwdSplit &, int, int64_t);
template size_t forward_partial_bytes<double>(const FwdSplit &, int, int64_t);
template size_t adjoint_partial_bytes<float>(const AdjSplit &, int, int);
template size_t adjoint_partial_bytes<double>(const AdjSplit &, int, int);

template int launch_forward<float, float, float>(const ModelH &, const GridH &, int64_t,
                                                 const Geometry<float> &, const FwdSplit &,
                                                 const float *, float *, float *, cudaStream_t);
template int launch_forward<float, double, float>(const ModelH &, const GridH &, int64_t,
                                                  const Geometry<float> &, const FwdSplit &,
                                                  const double *, float *, float *, cudaStream_t);
template int launch_forward<double, double, double>(const ModelH &, const GridH &, int64_t,
                                                    const Geometry<double> &, const FwdSplit &,
                                                    const double *, double *, double *,
                                                    cudaStream_t);
template int launch_adjoint<float, float>(const ModelH &, const GridH &, int64_t,
                                          const Geometry<float> &, const AdjSplit &, const float *,
                                          float *, float *, const double *, const double *,
                                          double *, cudaStream_t);
template int launch_adjoint<float, double>(const ModelH &, const GridH &, int64_t,
                                           const Geometry<float> &, const AdjSplit &,
                                           const float *, float *, double *, const double *,
                                           const double *, double *, cudaStream_t);
template int launch_adjoint<double, double>(const ModelH &, const GridH &, int64_t,
                                            const Geometry<double> &, const AdjSplit &,
                                            const double *, double *, double *, const double *,
                                            const double *, double *, cudaStream_t);
template int launch_dbeta<float>(const ModelH &, const GridH &, int64_t, const Geometry<float> &,
                                 const AdjSplit &, const float *, const float *, double *,
                                 double *, cudaStream_t);
template int launch_dbeta<double>(const ModelH &, const GridH &, int64_t,
                                  const Geometry<double> &, const AdjSplit &, const double *,
                                  const double *, double *, double *, cudaStream_t);

}  // namespace mpi
