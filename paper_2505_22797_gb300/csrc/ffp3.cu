// Three-dimensional field-free point: the model of Sec. 2 with n = 3.
//
// The kernel matrix of Eq. kernel:matrix is K(y) = a I + d y y^T with the same
// scalars a = L/z, d = (L' - a)/z^2 as in two dimensions, now 3 x 3; the
// signal of Eq. core:formula is
//   s_k(t) = sum_v c_v p_k^T beta K(beta G (x_v - r_t)) G v_t
// for a 3 x 3 gradient G (the paper's standard choice is diag(-1, -1, 2)),
// r_t, v_t in R^3 and up to three receive directions p_k.  The trace kernel of
// Eq. kernel:trace carries (n - 1) = 2.
//
// Kernels:
//   k_forward3   one work item = 512 samples (4 per thread) x a chunk of
//                voxels; voxels (prescaled position + concentration) stream
//                through shared memory 512 at a time; per-chunk partials,
//                reduced in FP64 in a fixed order.
//   k_adjoint3   one work item = 1024 voxels (8 per thread) x a chunk of
//                samples; each staged sample carries (B r, B v, U = sum_k s_k
//                p_k, U.B v) so a pair costs two dot products.
//   Both test the near field once per staged pass: the gap between the
//   bounding box of the pass's prescaled voxel positions and that of the
//   samples (precomputed per 512 voxels / 256 samples) decides whether every
//   pair of the pass is in the asymptotic range (one rsqrt per pair), in the
//   closed-form range, or may need the near-FFP series.
//   k_conv3_*    the sampled trace kernel and the direct zero-padded 3-D
//                convolution (8 x 8 x 4 output tiles) for small volumes; from
//                8192 voxels (FP32) / 512 (FP64) the FFT route: the kernel
//                placed circularly on a power-of-two NZ x NY x NX grid, DFTs
//                along x, y and z as Stockham row passes with transposes in
//                between, in the call's precision.
//   k_gauss3     the built-in denoiser along one axis (5 taps, reflect).
// PnP (Algorithm 1) runs the shared driver pnp_run with a 3-D operator.
#include <algorithm>
#include <cmath>

#include "conv_ops.cuh"
#include "langevin.cuh"
#include "pnp_device.cuh"
#include "pnp_ops.cuh"

namespace mpi {

int check_traj(const mpi_traj *t);
int check_dtype(mpi_dtype d);

struct Model3H {
    double beta;
    double G[9];
    int n_ch;
    double p[9];
};
struct Grid3H {
    int nx, ny, nz;
    double x0, y0, z0, dx, dy, dz;
    __host__ __device__ int64_t n() const { return (int64_t)nx * ny * nz; }
};
struct Mat3 {
    double a[9];
};

constexpr int k3Threads = 128;
// Minimum resident blocks per SM requested for the FP32 pair kernels
// (compile-time tuning knobs; the FP64 kernels request 2).
#ifndef MPI_FWD3_MINB
#define MPI_FWD3_MINB 4
#endif
#ifndef MPI_ADJ3_MINB
#define MPI_ADJ3_MINB 4
#endif
constexpr int k3FwdS = 4;                        // samples per thread (forward)
constexpr int k3FwdTile = k3Threads * k3FwdS;    // samples per forward work item
constexpr int k3Piece = 512;                     // voxels per staged pass / per voxel box
constexpr int k3AdjV = 8;                        // voxels per thread (adjoint)
constexpr int k3AdjTile = k3Threads * k3AdjV;    // voxels per adjoint work item
constexpr int k3Batch = 256;                     // samples per staged pass / per sample box
static_assert(k3FwdTile % k3Batch == 0 && k3AdjTile % k3Piece == 0, "box tiling");

// Prepared geometry of one 3-D problem (device scratch):
//   rs[t] = B r_t, ws[t] = B v_t, vox[v] = B x_v  (B = beta G; w unused)
//   sbox / vbox: (lo, hi) of rs over each k3Batch samples / of vox over each
//   k3Piece voxels.
template <typename R>
struct Geo3 {
    V4<R> *rs, *ws, *vox, *sbox, *vbox;
};

__host__ __device__ inline int64_t n_boxes(int64_t n, int per) { return (n + per - 1) / per; }

template <typename R>
static size_t geo3_bytes(int64_t T, int64_t N)
{
    const size_t e = sizeof(V4<R>);
    return e * (2 * T + N + 2 * n_boxes(T, k3Batch) + 2 * n_boxes(N, k3Piece)) + 5 * 256;
}

template <typename R>
static Geo3<R> geo3_carve(void *base, int64_t T, int64_t N)
{
    char *p = static_cast<char *>(base);
    auto take = [&](int64_t n) {
        V4<R> *q = reinterpret_cast<V4<R> *>(p);
        p += (sizeof(V4<R>) * n + 255) & ~size_t(255);
        return q;
    };
    Geo3<R> g;
    g.rs = take(T);
    g.ws = take(T);
    g.vox = take(N);
    g.sbox = take(2 * n_boxes(T, k3Batch));
    g.vbox = take(2 * n_boxes(N, k3Piece));
    return g;
}

template <typename R, typename IN>
__global__ void k_prep3_samples(int64_t T, const IN *__restrict__ r, const IN *__restrict__ v, Mat3 B,
                                V4<R> *__restrict__ rs, V4<R> *__restrict__ ws)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double rr[3] = {double(r[3 * t]), double(r[3 * t + 1]), double(r[3 * t + 2])};
        const double vv[3] = {double(v[3 * t]), double(v[3 * t + 1]), double(v[3 * t + 2])};
        double br[3], bv[3];
        for (int q = 0; q < 3; ++q) {
            br[q] = B.a[3 * q] * rr[0] + B.a[3 * q + 1] * rr[1] + B.a[3 * q + 2] * rr[2];
            bv[q] = B.a[3 * q] * vv[0] + B.a[3 * q + 1] * vv[1] + B.a[3 * q + 2] * vv[2];
        }
        rs[t] = V4<R>{R(br[0]), R(br[1]), R(br[2]), R(0)};
        ws[t] = V4<R>{R(bv[0]), R(bv[1]), R(bv[2]), R(0)};
    }
}

template <typename R>
__global__ void k_prep3_voxels(Grid3H g, Mat3 B, V4<R> *__restrict__ vox)
{
    const int64_t N = g.n();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.nx), j = (int)((e / g.nx) % g.ny), l = (int)(e / ((int64_t)g.nx * g.ny));
        const double x[3] = {g.x0 + (i + 0.5) * g.dx, g.y0 + (j + 0.5) * g.dy, g.z0 + (l + 0.5) * g.dz};
        double bx[3];
        for (int q = 0; q < 3; ++q) bx[q] = B.a[3 * q] * x[0] + B.a[3 * q + 1] * x[1] + B.a[3 * q + 2] * x[2];
        vox[e] = V4<R>{R(bx[0]), R(bx[1]), R(bx[2]), R(0)};
    }
}

// One warp per box: lo/hi of pts[b*per, min(n, (b+1)*per)).
template <typename R>
__global__ void k_box3(const V4<R> *__restrict__ pts, int64_t n, int per, int64_t n_box,
                       V4<R> *__restrict__ box)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= n_box) return;
    const int64_t a0 = b * per, a1 = std::min<int64_t>(n, a0 + per);
    V4<R> lo = pts[a0], hi = pts[a0];
    for (int64_t e = a0 + lane; e < a1; e += 32) {
        const V4<R> q = pts[e];
        lo.x = min(lo.x, q.x), lo.y = min(lo.y, q.y), lo.z = min(lo.z, q.z);
        hi.x = max(hi.x, q.x), hi.y = max(hi.y, q.y), hi.z = max(hi.z, q.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo.x = min(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
        lo.y = min(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
        lo.z = min(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
        hi.x = max(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
        hi.y = max(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
        hi.z = max(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
    }
    if (lane == 0) {
        box[2 * b] = lo;
        box[2 * b + 1] = hi;
    }
}

template <typename R>
__device__ __forceinline__ void box_union(V4<R> &lo, V4<R> &hi, const V4<R> &l2, const V4<R> &h2)
{
    lo.x = min(lo.x, l2.x), lo.y = min(lo.y, l2.y), lo.z = min(lo.z, l2.z);
    hi.x = max(hi.x, h2.x), hi.y = max(hi.y, h2.y), hi.z = max(hi.z, h2.z);
}

// Lower bound of u = |P - Q|^2 over P in box a, Q in box b, rounded the way
// the pair loops round it (same operations, monotone in each component).
template <typename R>
__device__ __forceinline__ R box_gap2(const V4<R> &alo, const V4<R> &ahi, const V4<R> &blo,
                                      const V4<R> &bhi)
{
    const R gx = max(R(0), max(alo.x - bhi.x, blo.x - ahi.x));
    const R gy = max(R(0), max(alo.y - bhi.y, blo.y - ahi.y));
    const R gz = max(R(0), max(alo.z - bhi.z, blo.z - ahi.z));
    return fmx(gz, gz, fmx(gy, gy, gx * gx));
}

template <typename R>
__device__ __forceinline__ bool far_field(R gap2)
{
    return gap2 >= Lang<R>::near_u * R(1.0001);
}

// ---------------------------------------------------------------------------
// Forward operator.

template <typename R, typename CIN>
struct Fwd3Args {
    const V4<R> *rs, *ws, *vox, *sbox, *vbox;
    const CIN *c;
    R *part;
    int64_t T, N, chunk_len;
    int n_tiles, n_ch;
    R p[9];
};

// MODE 2: every pair of the pass in the asymptotic range (u >= vfar_u);
// 1: every pair in the closed-form range; 0: near pairs possible.
template <typename R, bool DBETA, int MODE>
__device__ __forceinline__ void lang3(R u, R &f1, R &f2)
{
    if constexpr (MODE == 2) lang_vfar<R, DBETA>(u, f1, f2);
    else if constexpr (MODE == 1) lang_far<R, DBETA>(u, f1, f2);
    else lang_checked<R, DBETA>(u, f1, f2);
}

// The asymptotic pass in packed two-lane FP32 arithmetic (f32x2, sm_100 and
// later), samples (2h, 2h + 1) of the thread in the two lanes: the same FP32
// work from half the issue slots (the pass is issue-bound in scalar form).
#ifndef MPI_FWD3_PACK
#define MPI_FWD3_PACK 1
#endif
__device__ __forceinline__ void fwd3_pass_vfar_packed(const V4<float> *sv, int cnt, const float (&Rx)[k3FwdS],
                                                      const float (&Ry)[k3FwdS], const float (&Rz)[k3FwdS],
                                                      const float (&Wx)[k3FwdS], const float (&Wy)[k3FwdS],
                                                      const float (&Wz)[k3FwdS], float (&sa)[k3FwdS],
                                                      float (&Sx)[k3FwdS], float (&Sy)[k3FwdS],
                                                      float (&Sz)[k3FwdS])
{
    constexpr int H = k3FwdS / 2;
    const float2 m1 = make_float2(-1.0f, -1.0f);
    float2 nRx[H], nRy[H], nRz[H], Wx2[H], Wy2[H], Wz2[H], sa2[H], Sx2[H], Sy2[H], Sz2[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        nRx[h] = make_float2(-Rx[2 * h], -Rx[2 * h + 1]);
        nRy[h] = make_float2(-Ry[2 * h], -Ry[2 * h + 1]);
        nRz[h] = make_float2(-Rz[2 * h], -Rz[2 * h + 1]);
        Wx2[h] = make_float2(Wx[2 * h], Wx[2 * h + 1]);
        Wy2[h] = make_float2(Wy[2 * h], Wy[2 * h + 1]);
        Wz2[h] = make_float2(Wz[2 * h], Wz[2 * h + 1]);
        sa2[h] = Sx2[h] = Sy2[h] = Sz2[h] = make_float2(0.0f, 0.0f);
    }
#pragma unroll 2
    for (int e = 0; e < cnt; ++e) {
        const V4<float> P = sv[e];
        const float2 Px = make_float2(P.x, P.x), Py = make_float2(P.y, P.y), Pz = make_float2(P.z, P.z);
        const float2 Pw = make_float2(P.w, P.w);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const float2 yx = __fadd2_rn(Px, nRx[h]), yy = __fadd2_rn(Py, nRy[h]), yz = __fadd2_rn(Pz, nRz[h]);
            const float2 u = __ffma2_rn(yz, yz, __ffma2_rn(yy, yy, __fmul2_rn(yx, yx)));
            const float2 iz = make_float2(Lang<float>::iz_vfar(u.x), Lang<float>::iz_vfar(u.y));
            const float2 iz2 = __fmul2_rn(iz, iz);
            const float2 a = __ffma2_rn(iz2, m1, iz);                  // iz - iz^2
            const float2 d = __fmul2_rn(__ffma2_rn(a, m1, iz2), iz2);  // (2 iz^2 - iz) iz^2
            const float2 yW = __ffma2_rn(yz, Wz2[h], __ffma2_rn(yy, Wy2[h], __fmul2_rn(yx, Wx2[h])));
            const float2 t = __fmul2_rn(__fmul2_rn(Pw, d), yW);
            Sx2[h] = __ffma2_rn(t, yx, Sx2[h]);
            Sy2[h] = __ffma2_rn(t, yy, Sy2[h]);
            Sz2[h] = __ffma2_rn(t, yz, Sz2[h]);
            sa2[h] = __ffma2_rn(Pw, a, sa2[h]);
        }
    }
#pragma unroll
    for (int h = 0; h < H; ++h) {
        sa[2 * h] += sa2[h].x; sa[2 * h + 1] += sa2[h].y;
        Sx[2 * h] += Sx2[h].x; Sx[2 * h + 1] += Sx2[h].y;
        Sy[2 * h] += Sy2[h].x; Sy[2 * h + 1] += Sy2[h].y;
        Sz[2 * h] += Sz2[h].x; Sz[2 * h + 1] += Sz2[h].y;
    }
}

template <typename R, int MODE>
__device__ __forceinline__ void fwd3_pass(const V4<R> *sv, int cnt, const R (&Rx)[k3FwdS],
                                          const R (&Ry)[k3FwdS], const R (&Rz)[k3FwdS],
                                          const R (&Wx)[k3FwdS], const R (&Wy)[k3FwdS],
                                          const R (&Wz)[k3FwdS], R (&sa)[k3FwdS], R (&Sx)[k3FwdS],
                                          R (&Sy)[k3FwdS], R (&Sz)[k3FwdS])
{
    if constexpr (MODE == 2 && sizeof(R) == 4 && MPI_FWD3_PACK && k3FwdS % 2 == 0) {
        fwd3_pass_vfar_packed(sv, cnt, Rx, Ry, Rz, Wx, Wy, Wz, sa, Sx, Sy, Sz);
        return;
    }
#pragma unroll 2
    for (int e = 0; e < cnt; ++e) {
        const V4<R> P = sv[e];
#pragma unroll
        for (int s = 0; s < k3FwdS; ++s) {
            const R yx = P.x - Rx[s], yy = P.y - Ry[s], yz = P.z - Rz[s];
            const R u = fmx(yz, yz, fmx(yy, yy, yx * yx));
            R a, d;
            lang3<R, false, MODE>(u, a, d);
            const R yW = fmx(yz, Wz[s], fmx(yy, Wy[s], yx * Wx[s]));
            const R t = (P.w * d) * yW;
            Sx[s] = fmx(t, yx, Sx[s]);
            Sy[s] = fmx(t, yy, Sy[s]);
            Sz[s] = fmx(t, yz, Sz[s]);
            sa[s] = fmx(P.w, a, sa[s]);
        }
    }
}

template <typename R, typename CIN>
__global__ void __launch_bounds__(k3Threads, sizeof(R) == 4 ? MPI_FWD3_MINB : 2)
k_forward3(const __grid_constant__ Fwd3Args<R, CIN> a)
{
    __shared__ V4<R> sv[k3Piece];
    const int tile = (int)(blockIdx.x % a.n_tiles);
    const int64_t chunk = blockIdx.x / a.n_tiles;
    const int64_t t0 = (int64_t)tile * k3FwdTile;
    R Rx[k3FwdS], Ry[k3FwdS], Rz[k3FwdS], Wx[k3FwdS], Wy[k3FwdS], Wz[k3FwdS];
    R sa[k3FwdS], Sx[k3FwdS], Sy[k3FwdS], Sz[k3FwdS];
#pragma unroll
    for (int s = 0; s < k3FwdS; ++s) {
        const int64_t t = std::min<int64_t>(t0 + threadIdx.x + s * k3Threads, a.T - 1);
        const V4<R> r = a.rs[t], w = a.ws[t];
        Rx[s] = r.x, Ry[s] = r.y, Rz[s] = r.z;
        Wx[s] = w.x, Wy[s] = w.y, Wz[s] = w.z;
        sa[s] = Sx[s] = Sy[s] = Sz[s] = R(0);
    }
    // bounding box of this item's samples
    const int64_t nb = n_boxes(a.T, k3Batch);
    const int64_t b0 = t0 / k3Batch;
    V4<R> slo = a.sbox[2 * b0], shi = a.sbox[2 * b0 + 1];
    for (int64_t b = b0 + 1; b < std::min<int64_t>(nb, b0 + k3FwdTile / k3Batch); ++b)
        box_union(slo, shi, a.sbox[2 * b], a.sbox[2 * b + 1]);

    const int64_t v0 = chunk * a.chunk_len, v1 = std::min<int64_t>(a.N, v0 + a.chunk_len);
    for (int64_t vp = v0; vp < v1; vp += k3Piece) {
        const int cnt = (int)std::min<int64_t>(k3Piece, v1 - vp);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += k3Threads) {
            V4<R> P = a.vox[vp + e];
            P.w = R(a.c[vp + e]);
            sv[e] = P;
        }
        __syncthreads();
        const int64_t pb = vp / k3Piece;
        const R gap2 = box_gap2(a.vbox[2 * pb], a.vbox[2 * pb + 1], slo, shi);
        if (gap2 >= vfar_threshold<R, false>())
            fwd3_pass<R, 2>(sv, cnt, Rx, Ry, Rz, Wx, Wy, Wz, sa, Sx, Sy, Sz);
        else if (far_field(gap2))
            fwd3_pass<R, 1>(sv, cnt, Rx, Ry, Rz, Wx, Wy, Wz, sa, Sx, Sy, Sz);
        else
            fwd3_pass<R, 0>(sv, cnt, Rx, Ry, Rz, Wx, Wy, Wz, sa, Sx, Sy, Sz);
    }
    // s_k = p_k^T (W sum c a + sum c d (y.W) y)
#pragma unroll
    for (int s = 0; s < k3FwdS; ++s) {
        const int64_t t = t0 + threadIdx.x + s * k3Threads;
        if (t >= a.T) continue;
        const R ox = fmx(Wx[s], sa[s], Sx[s]), oy = fmx(Wy[s], sa[s], Sy[s]), oz = fmx(Wz[s], sa[s], Sz[s]);
        for (int k = 0; k < a.n_ch; ++k)
            a.part[(chunk * a.n_ch + k) * a.T + t] = fmx(a.p[3 * k + 2], oz, fmx(a.p[3 * k + 1], oy, a.p[3 * k] * ox));
    }
}

// ---------------------------------------------------------------------------
// Adjoint operator.

template <typename R>
struct Adj3Args {
    const V4<R> *rs, *ws, *vox, *sbox, *vbox;
    const R *s;
    R *part;
    int64_t T, N, chunk_len;
    int n_vt, n_ch;
    R p[9];
};

template <typename R, int MODE>
__device__ __forceinline__ void adj3_pass(const V4<R> *sR, const V4<R> *sW, const V4<R> *sU, int cnt,
                                          const R (&Px)[k3AdjV], const R (&Py)[k3AdjV],
                                          const R (&Pz)[k3AdjV], R (&acc)[k3AdjV])
{
#pragma unroll 1
    for (int e = 0; e < cnt; ++e) {
        const V4<R> Q = sR[e], W = sW[e], U = sU[e];
#pragma unroll
        for (int m = 0; m < k3AdjV; ++m) {
            const R yx = Px[m] - Q.x, yy = Py[m] - Q.y, yz = Pz[m] - Q.z;
            const R u = fmx(yz, yz, fmx(yy, yy, yx * yx));
            const R yU = fmx(yz, U.z, fmx(yy, U.y, yx * U.x));
            const R yW = fmx(yz, W.z, fmx(yy, W.y, yx * W.x));
            // U^T K W = a (U.W) + d (y.U)(y.W)
            if constexpr (MODE == 2) {
                acc[m] = pair_acc_vfar<R, false>(u, W.w, yU * yW, acc[m]);
            } else {
                R a, d;
                lang3<R, false, MODE>(u, a, d);
                acc[m] = fmx(d * yU, yW, fmx(a, W.w, acc[m]));
            }
        }
    }
}

// The asymptotic pass in packed two-lane FP32 arithmetic, staged samples
// (2h, 2h + 1) in the two lanes (the pass is issue-bound in scalar form).
// pk: the staged samples as pairs, five float4 per pair h:
//   (-Qx, -Qy), (-Qz, Wx), (Wy, Wz), (uW, Ux), (Uy, Uz)   (each entry: even, odd sample).
#ifndef MPI_ADJ3_PACK
#define MPI_ADJ3_PACK 1
#endif
__device__ __forceinline__ void adj3_pass_vfar_packed(const float4 *pk, int npair, const float (&Px)[k3AdjV],
                                                      const float (&Py)[k3AdjV], const float (&Pz)[k3AdjV],
                                                      float (&acc)[k3AdjV])
{
    const float2 m1 = make_float2(-1.0f, -1.0f), two = make_float2(2.0f, 2.0f);
    float2 acc2[k3AdjV];
#pragma unroll
    for (int m = 0; m < k3AdjV; ++m) acc2[m] = make_float2(0.0f, 0.0f);
#pragma unroll 1
    for (int h = 0; h < npair; ++h) {
        const float4 A = pk[5 * h], B = pk[5 * h + 1], C = pk[5 * h + 2], D = pk[5 * h + 3], E = pk[5 * h + 4];
        const float2 nQx = make_float2(A.x, A.y), nQy = make_float2(A.z, A.w), nQz = make_float2(B.x, B.y);
        const float2 Wx = make_float2(B.z, B.w), Wy = make_float2(C.x, C.y), Wz = make_float2(C.z, C.w);
        const float2 uW = make_float2(D.x, D.y), Ux = make_float2(D.z, D.w);
        const float2 Uy = make_float2(E.x, E.y), Uz = make_float2(E.z, E.w);
        const float2 nuW = __fmul2_rn(uW, m1);
#pragma unroll
        for (int m = 0; m < k3AdjV; ++m) {
            const float2 yx = __fadd2_rn(make_float2(Px[m], Px[m]), nQx);
            const float2 yy = __fadd2_rn(make_float2(Py[m], Py[m]), nQy);
            const float2 yz = __fadd2_rn(make_float2(Pz[m], Pz[m]), nQz);
            const float2 u = __ffma2_rn(yz, yz, __ffma2_rn(yy, yy, __fmul2_rn(yx, yx)));
            const float2 yU = __ffma2_rn(yz, Uz, __ffma2_rn(yy, Uy, __fmul2_rn(yx, Ux)));
            const float2 yW = __ffma2_rn(yz, Wz, __ffma2_rn(yy, Wy, __fmul2_rn(yx, Wx)));
            const float2 P = __fmul2_rn(yU, yW);
            const float2 iz = make_float2(Lang<float>::iz_vfar(u.x), Lang<float>::iz_vfar(u.y));
            // iz (uW + iz (iz (2 iz - 1) P - uW)), as pair_acc_vfar
            const float2 w = __ffma2_rn(iz, __fmul2_rn(P, __ffma2_rn(iz, two, m1)), nuW);
            acc2[m] = __ffma2_rn(iz, __ffma2_rn(iz, w, uW), acc2[m]);
        }
    }
#pragma unroll
    for (int m = 0; m < k3AdjV; ++m) acc[m] += acc2[m].x + acc2[m].y;
}

template <typename R>
__global__ void __launch_bounds__(k3Threads, sizeof(R) == 4 ? MPI_ADJ3_MINB : 2)
k_adjoint3(const __grid_constant__ Adj3Args<R> a)
{
    constexpr bool PACK = sizeof(R) == 4 && MPI_ADJ3_PACK;
    __shared__ V4<R> sR[k3Batch], sW[k3Batch], sU[k3Batch];
    __shared__ float4 sPk[PACK ? 5 * (k3Batch / 2) : 1];
    const int vt = (int)(blockIdx.x % a.n_vt);
    const int64_t chunk = blockIdx.x / a.n_vt;
    const int64_t vbase = (int64_t)vt * k3AdjTile;
    R Px[k3AdjV], Py[k3AdjV], Pz[k3AdjV], acc[k3AdjV];
#pragma unroll
    for (int m = 0; m < k3AdjV; ++m) {
        const int64_t v = std::min<int64_t>(vbase + threadIdx.x + m * k3Threads, a.N - 1);
        const V4<R> P = a.vox[v];
        Px[m] = P.x, Py[m] = P.y, Pz[m] = P.z;
        acc[m] = R(0);
    }
    const int64_t npb = n_boxes(a.N, k3Piece);
    const int64_t p0 = vbase / k3Piece;
    V4<R> vlo = a.vbox[2 * p0], vhi = a.vbox[2 * p0 + 1];
    for (int64_t b = p0 + 1; b < std::min<int64_t>(npb, p0 + k3AdjTile / k3Piece); ++b)
        box_union(vlo, vhi, a.vbox[2 * b], a.vbox[2 * b + 1]);

    const int64_t tb0 = chunk * a.chunk_len, tb1 = std::min<int64_t>(a.T, tb0 + a.chunk_len);
    for (int64_t tb = tb0; tb < tb1; tb += k3Batch) {
        const int cnt = (int)std::min<int64_t>(k3Batch, tb1 - tb);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += k3Threads) {
            const int64_t t = tb + e;
            const V4<R> Q = a.rs[t], W = a.ws[t];
            R ux = R(0), uy = R(0), uz = R(0);
            for (int k = 0; k < a.n_ch; ++k) {
                const R sk = a.s[k * a.T + t];
                ux = fmx(sk, a.p[3 * k], ux);
                uy = fmx(sk, a.p[3 * k + 1], uy);
                uz = fmx(sk, a.p[3 * k + 2], uz);
            }
            const R uW = fmx(uz, W.z, fmx(uy, W.y, ux * W.x));
            sR[e] = Q;
            sW[e] = V4<R>{W.x, W.y, W.z, uW};
            sU[e] = V4<R>{ux, uy, uz, R(0)};
            if constexpr (PACK) {
                float *pb = reinterpret_cast<float *>(sPk + 5 * (e >> 1)) + (e & 1);
                const float v[10] = {-float(Q.x), -float(Q.y), -float(Q.z), float(W.x), float(W.y),
                                     float(W.z), float(uW), float(ux), float(uy), float(uz)};
#pragma unroll
                for (int j = 0; j < 10; ++j) pb[2 * j] = v[j];
                if ((e & 1) == 0 && e + 1 == cnt) {
                    // odd count: the pair's second sample contributes nothing
                    // (W and U zero) at the first one's position (u > 0)
#pragma unroll
                    for (int j = 0; j < 10; ++j) pb[2 * j + 1] = j < 3 ? v[j] : 0.0f;
                }
            }
        }
        __syncthreads();
        const int64_t sb = tb / k3Batch;
        const R gap2 = box_gap2(vlo, vhi, a.sbox[2 * sb], a.sbox[2 * sb + 1]);
        if (gap2 >= vfar_threshold<R, false>()) {
            if constexpr (PACK) adj3_pass_vfar_packed(sPk, (cnt + 1) / 2, Px, Py, Pz, acc);
            else adj3_pass<R, 2>(sR, sW, sU, cnt, Px, Py, Pz, acc);
        } else if (far_field(gap2))
            adj3_pass<R, 1>(sR, sW, sU, cnt, Px, Py, Pz, acc);
        else
            adj3_pass<R, 0>(sR, sW, sU, cnt, Px, Py, Pz, acc);
    }
#pragma unroll
    for (int m = 0; m < k3AdjV; ++m) {
        const int64_t v = vbase + threadIdx.x + m * k3Threads;
        if (v < a.N) a.part[chunk * a.N + v] = acc[m];
    }
}

// ---------------------------------------------------------------------------
// Host side of the pair operators.

struct Split3 {
    int n_tiles;        // forward: sample tiles; adjoint: voxel tiles
    int64_t chunk_len;  // forward: voxels per chunk; adjoint: samples per chunk
    int n_chunks;
};

static Split3 split3(int64_t n_tiled, int tile, int64_t n_chunked, int align, int target)
{
    Split3 s;
    s.n_tiles = (int)std::max<int64_t>(1, (n_tiled + tile - 1) / tile);
    const int64_t want = std::max<int64_t>(1, (target + s.n_tiles - 1) / s.n_tiles);
    int64_t len = (std::max<int64_t>(n_chunked, 1) + want - 1) / want;
    len = std::max<int64_t>(align, (len + align - 1) / align * align);
    s.chunk_len = len;
    s.n_chunks = (int)std::max<int64_t>(1, (n_chunked + len - 1) / len);
    return s;
}

template <typename R>
struct Op3 {
    Model3H m;
    Grid3H g;
    int64_t T = 0, N = 0;
    Geo3<R> geo{};
    Split3 fs{}, as{};
    R *fwd_part = nullptr, *adj_part = nullptr;

    size_t scratch_bytes() const
    {
        return geo3_bytes<R>(T, N) + sizeof(R) * (size_t(fs.n_chunks) * m.n_ch * T + 256) +
               sizeof(R) * (size_t(as.n_chunks) * N + 256) + 512;
    }
    void plan(const Model3H &mm, const Grid3H &gg, int64_t TT)
    {
        m = mm;
        g = gg;
        T = TT;
        N = gg.n();
        const int target = default_target_items();
        fs = split3(T, k3FwdTile, N, k3Piece, target);
        as = split3(N, k3AdjTile, T, k3Batch, target);
    }
    void carve(char *base)
    {
        geo = geo3_carve<R>(base, T, N);
        char *p = base + ((geo3_bytes<R>(T, N) + 255) & ~size_t(255));
        fwd_part = reinterpret_cast<R *>(p);
        p += (sizeof(R) * (size_t(fs.n_chunks) * m.n_ch * T + 256) + 255) & ~size_t(255);
        adj_part = reinterpret_cast<R *>(p);
    }
    Mat3 bmat() const
    {
        Mat3 B;
        for (int q = 0; q < 9; ++q) B.a[q] = m.beta * m.G[q];
        return B;
    }
    template <typename IN>
    int prepare(const IN *r, const IN *v, cudaStream_t st)
    {
        const Mat3 B = bmat();
        if (T > 0) {
            k_prep3_samples<R, IN><<<(unsigned)std::min<int64_t>((T + 255) / 256, 4096), 256, 0, st>>>(
                T, r, v, B, geo.rs, geo.ws);
            MPI_CHECK_LAUNCH();
            const int64_t nb = n_boxes(T, k3Batch);
            k_box3<R><<<(unsigned)((nb * 32 + 255) / 256), 256, 0, st>>>(geo.rs, T, k3Batch, nb, geo.sbox);
            MPI_CHECK_LAUNCH();
        }
        k_prep3_voxels<R><<<(unsigned)std::min<int64_t>((N + 255) / 256, 4096), 256, 0, st>>>(g, B, geo.vox);
        MPI_CHECK_LAUNCH();
        const int64_t np = n_boxes(N, k3Piece);
        k_box3<R><<<(unsigned)((np * 32 + 255) / 256), 256, 0, st>>>(geo.vox, N, k3Piece, np, geo.vbox);
        MPI_CHECK_LAUNCH();
        return MPI_OK;
    }
    template <typename CIN, typename OUT>
    int forward(const CIN *c, OUT *s, cudaStream_t st)
    {
        if (T == 0) return MPI_OK;
        Fwd3Args<R, CIN> a;
        a.rs = geo.rs, a.ws = geo.ws, a.vox = geo.vox, a.sbox = geo.sbox, a.vbox = geo.vbox;
        a.c = c;
        a.part = fwd_part;
        a.T = T, a.N = N, a.chunk_len = fs.chunk_len;
        a.n_tiles = fs.n_tiles, a.n_ch = m.n_ch;
        for (int q = 0; q < 9; ++q) a.p[q] = R(m.p[q]);
        {
            ProfScope prof(kProfForward, st);
            k_forward3<R, CIN><<<(unsigned)((int64_t)fs.n_tiles * fs.n_chunks), k3Threads, 0, st>>>(a);
            MPI_CHECK_LAUNCH();
        }
        return reduce_chunks<R, OUT>(fwd_part, fs.n_chunks, (int64_t)m.n_ch * T, s, nullptr, nullptr,
                                     nullptr, st);
    }
    // out = A^T s; with cg_p: out = A^T s + nu cg_p and partial sums of <cg_p, out>.
    template <typename OUT>
    int adjoint(const R *s, OUT *out, const double *cg_p, const double *nu_dev, double *dot_part,
                cudaStream_t st)
    {
        int nch = as.n_chunks;
        if (T > 0) {
            Adj3Args<R> a;
            a.rs = geo.rs, a.ws = geo.ws, a.vox = geo.vox, a.sbox = geo.sbox, a.vbox = geo.vbox;
            a.s = s;
            a.part = adj_part;
            a.T = T, a.N = N, a.chunk_len = as.chunk_len;
            a.n_vt = as.n_tiles, a.n_ch = m.n_ch;
            for (int q = 0; q < 9; ++q) a.p[q] = R(m.p[q]);
            ProfScope prof(kProfAdjoint, st);
            k_adjoint3<R><<<(unsigned)((int64_t)as.n_tiles * as.n_chunks), k3Threads, 0, st>>>(a);
            MPI_CHECK_LAUNCH();
        } else {
            MPI_TRY_CUDA(cudaMemsetAsync(adj_part, 0, sizeof(R) * N, st));
            nch = 1;
        }
        return reduce_chunks<R, OUT>(adj_part, nch, N, out, cg_p, nu_dev, dot_part, st);
    }
};

// ---------------------------------------------------------------------------
// Convolution with the 3-D sampled trace kernel.

constexpr int kC3x = 8, kC3y = 8, kC3z = 4;  // output / input tile
constexpr int kC3Kx = 2 * kC3x - 1, kC3Ky = 2 * kC3y - 1, kC3Kz = 2 * kC3z - 1;

// kernel 0: kappa_G(o) = beta tr(K(beta G o) G) = beta (a tr G + d y^T G y),
// y = beta G o (the trace kernel); kernel 1: beta tr K(beta G o) =
// beta (3 a + d |y|^2), the kernel of the gradient-weighted trace
// tr(Ahat G^-1) (positive for any G; the trace kernel of a traceless G is not).
__global__ void k_conv3_kernel_sample(Grid3H g, double beta, Mat3 G, int kernel, double *__restrict__ K)
{
    const int KX = 2 * g.nx - 1, KY = 2 * g.ny - 1, KZ = 2 * g.nz - 1;
    const int64_t n = (int64_t)KX * KY * KZ;
    const double trG = G.a[0] + G.a[4] + G.a[8];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ii = (int)(e % KX), jj = (int)((e / KX) % KY), ll = (int)(e / ((int64_t)KX * KY));
        const double o[3] = {(ii - (g.nx - 1)) * g.dx, (jj - (g.ny - 1)) * g.dy, (ll - (g.nz - 1)) * g.dz};
        double y[3];
        for (int q = 0; q < 3; ++q) y[q] = beta * (G.a[3 * q] * o[0] + G.a[3 * q + 1] * o[1] + G.a[3 * q + 2] * o[2]);
        double a, d;
        lang_checked<double, false>(y[0] * y[0] + y[1] * y[1] + y[2] * y[2], a, d);
        if (kernel == 1) {
            K[e] = beta * (3.0 * a + d * (y[0] * y[0] + y[1] * y[1] + y[2] * y[2]));
        } else {
            double yGy = 0.0;
            for (int q = 0; q < 3; ++q)
                yGy += y[q] * (G.a[3 * q] * y[0] + G.a[3 * q + 1] * y[1] + G.a[3 * q + 2] * y[2]);
            K[e] = beta * (a * trG + d * yGy);
        }
    }
}

template <typename R>
__global__ void k_round3(const double *__restrict__ in, R *__restrict__ out, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = R(in[e]);
}

static size_t conv3_kernel_bytes(const Grid3H &g, int elem)
{
    return size_t(2 * g.nx - 1) * size_t(2 * g.ny - 1) * size_t(2 * g.nz - 1) * (sizeof(double) + elem) + 512;
}

template <typename R>
static int conv3_prepare(const Model3H &m, const Grid3H &g, int kernel, void *scratch, R **K_out,
                         cudaStream_t st)
{
    const int64_t n = (int64_t)(2 * g.nx - 1) * (2 * g.ny - 1) * (2 * g.nz - 1);
    double *K64 = static_cast<double *>(scratch);
    Mat3 G;
    for (int q = 0; q < 9; ++q) G.a[q] = m.G[q];
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_conv3_kernel_sample<<<blocks, 256, 0, st>>>(g, m.beta, G, kernel, K64);
    MPI_CHECK_LAUNCH();
    if constexpr (sizeof(R) == sizeof(double)) {
        *K_out = reinterpret_cast<R *>(K64);
    } else {
        R *K = reinterpret_cast<R *>(static_cast<char *>(scratch) + ((sizeof(double) * n + 255) & ~size_t(255)));
        k_round3<R><<<blocks, 256, 0, st>>>(K64, K, n);
        MPI_CHECK_LAUNCH();
        *K_out = K;
    }
    return MPI_OK;
}

// out = C in over all voxel offsets; one 8 x 8 x 4 output tile per block,
// input walked in tiles of the same shape with the matching kernel window in
// shared memory; per-tile sums folded with compensated additions.
template <typename R, typename IN, typename OUT>
__global__ void __launch_bounds__(kC3x *kC3y *kC3z)
k_conv3_direct(int nx, int ny, int nz, const R *__restrict__ K, const IN *__restrict__ in,
               OUT *__restrict__ out)
{
    __shared__ R s_in[kC3z][kC3y][kC3x];
    __shared__ R s_k[kC3Kz][kC3Ky][kC3Kx + 1];
    const int tx = threadIdx.x % kC3x, ty = (threadIdx.x / kC3x) % kC3y, tz = threadIdx.x / (kC3x * kC3y);
    const int i0 = blockIdx.x * kC3x, j0 = blockIdx.y * kC3y, l0 = blockIdx.z * kC3z;
    const int i = i0 + tx, j = j0 + ty, l = l0 + tz;
    const int KX = 2 * nx - 1, KY = 2 * ny - 1;
    R acc = R(0), comp = R(0);
    for (int lq0 = 0; lq0 < nz; lq0 += kC3z)
        for (int jq0 = 0; jq0 < ny; jq0 += kC3y)
            for (int iq0 = 0; iq0 < nx; iq0 += kC3x) {
                __syncthreads();
                {
                    const int iq = iq0 + tx, jq = jq0 + ty, lq = lq0 + tz;
                    s_in[tz][ty][tx] = (iq < nx && jq < ny && lq < nz)
                                           ? R(in[((int64_t)lq * ny + jq) * nx + iq]) : R(0);
                }
                for (int e = threadIdx.x; e < kC3Kx * kC3Ky * kC3Kz; e += kC3x * kC3y * kC3z) {
                    const int ex = e % kC3Kx, ey = (e / kC3Kx) % kC3Ky, ez = e / (kC3Kx * kC3Ky);
                    const int oi = i0 - iq0 - (kC3x - 1) + ex;
                    const int oj = j0 - jq0 - (kC3y - 1) + ey;
                    const int ol = l0 - lq0 - (kC3z - 1) + ez;
                    const bool ok = oi > -nx && oi < nx && oj > -ny && oj < ny && ol > -nz && ol < nz;
                    s_k[ez][ey][ex] = ok ? K[((int64_t)(ol + nz - 1) * KY + (oj + ny - 1)) * KX + (oi + nx - 1)] : R(0);
                }
                __syncthreads();
                R part = R(0);
                for (int c = 0; c < kC3z; ++c)
#pragma unroll 2
                    for (int b = 0; b < kC3y; ++b)
#pragma unroll
                        for (int q = 0; q < kC3x; ++q)
                            part = fmx(s_k[tz - c + kC3z - 1][ty - b + kC3y - 1][tx - q + kC3x - 1], s_in[c][b][q], part);
                kahan_add(acc, comp, part);
            }
    if (i < nx && j < ny && l < nz) out[((int64_t)l * ny + j) * nx + i] = OUT(acc);
}

template <typename R, typename IN, typename OUT>
static int launch_conv3(const Grid3H &g, const R *K, const IN *in, OUT *out, cudaStream_t st)
{
    dim3 grid((g.nx + kC3x - 1) / kC3x, (g.ny + kC3y - 1) / kC3y, (g.nz + kC3z - 1) / kC3z);
    ProfScope prof(kProfConv, st);
    k_conv3_direct<R, IN, OUT><<<grid, kC3x * kC3y * kC3z, 0, st>>>(g.nx, g.ny, g.nz, K, in, out);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}


// --- FFT route ---------------------------------------------------------------

static int pow2_at_least(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

template <typename R>
struct Conv3Plan {
    using C2 = typename CxOf<R>::type;
    Grid3H g{};
    bool fft = false;
    const R *K = nullptr;
    int NX = 0, NY = 0, NZ = 0;
    FftPlan px, py, pz;
    C2 *WX = nullptr, *WY = nullptr, *WZ = nullptr, *Kh = nullptr, *a = nullptr, *t = nullptr;
    // Five-launch form (shared-memory transforms, conv_fft2.cu): Kh holds the
    // kernel spectrum's kx < LD, [NZ][NY][LD]; a and t the half spectra.
    bool fused = false;
    int LD = 0;
};

// The five-launch form: every transform in shared memory.
#ifndef MPI_CONV3_FUSED
#define MPI_CONV3_FUSED 1
#endif
static bool conv3_fused_fits(int NX, int NY, int NZ)
{
    return MPI_CONV3_FUSED && NX >= 4 && NY >= 4 && NZ >= 4 && NX <= 4096 && NY <= 2048 && NZ <= 2048;
}

// Kh3[kz][ky][kx] = Kh[ky][kx][kz] for kx < LD (the layout dft3 leaves, half of it).
template <typename C>
__global__ void k_conv3_kh_half(int NX, int NY, int NZ, int LD, const C *__restrict__ Kh, C *__restrict__ Kh3)
{
    const int64_t n = (int64_t)NZ * NY * LD;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e % LD), ky = (int)((e / LD) % NY), kz = (int)(e / ((int64_t)LD * NY));
        Kh3[e] = Kh[((int64_t)ky * NX + kx) * NZ + kz];
    }
}

static bool conv3_uses_fft(const Grid3H &g, int elem)
{
    // where it overtook the direct sum on GB300 (FP32 between 24x24x12 and
    // 48x48x24; FP64 already at 12x12x6)
    if (g.n() < (elem == 8 ? 512 : 8192)) return false;
    const int64_t NX = pow2_at_least(2 * g.nx - 1), NY = pow2_at_least(2 * g.ny - 1),
                  NZ = pow2_at_least(2 * g.nz - 1);
    // batch counts of the row passes run as the grid's y dimension
    return NZ * NY <= 65535 && NX * NZ <= 65535 && NY * NX <= 65535;
}

static size_t conv3_plan_bytes(const Grid3H &g, int elem)
{
    size_t b = conv3_kernel_bytes(g, elem);
    if (conv3_uses_fft(g, elem)) {
        const size_t NX = pow2_at_least(2 * g.nx - 1), NY = pow2_at_least(2 * g.ny - 1),
                     NZ = pow2_at_least(2 * g.nz - 1);
        b += 2 * size_t(elem) * (NX + NY + NZ + 3 * NX * NY * NZ) + 8 * 256;
    }
    return b;
}

template <typename C>
__global__ void k_conv3_circ(Grid3H g, int NX, int NY, int NZ, const double *__restrict__ K, C *__restrict__ kc)
{
    const int KX = 2 * g.nx - 1, KY = 2 * g.ny - 1;
    const int64_t n = (int64_t)NX * NY * NZ;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % NX), j = (int)((e / NX) % NY), l = (int)(e / ((int64_t)NX * NY));
        const int di = i < g.nx ? i : i - NX, dj = j < g.ny ? j : j - NY, dl = l < g.nz ? l : l - NZ;
        double v = 0.0;
        if (di > -g.nx && di < g.nx && dj > -g.ny && dj < g.ny && dl > -g.nz && dl < g.nz)
            v = K[((int64_t)(dl + g.nz - 1) * KY + (dj + g.ny - 1)) * KX + (di + g.nx - 1)];
        kc[e] = make_cx<C>(v, 0.0);
    }
}

template <typename IN, typename C>
__global__ void k_conv3_load(Grid3H g, int NX, int NY, int NZ, const IN *__restrict__ in, C *__restrict__ a)
{
    const int64_t n = (int64_t)NX * NY * NZ;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % NX), j = (int)((e / NX) % NY), l = (int)(e / ((int64_t)NX * NY));
        const bool inside = i < g.nx && j < g.ny && l < g.nz;
        a[e] = make_cx<C>(inside ? double(in[((int64_t)l * g.ny + j) * g.nx + i]) : 0.0, 0.0);
    }
}

template <typename OUT, typename C>
__global__ void k_conv3_crop(Grid3H g, int NX, int NY, const C *__restrict__ a, double scale, OUT *__restrict__ out)
{
    const int64_t n = g.n();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % g.nx), j = (int)((e / g.nx) % g.ny), l = (int)(e / ((int64_t)g.nx * g.ny));
        out[e] = OUT(double(a[((int64_t)l * NY + j) * NX + i].x) * scale);
    }
}

static unsigned conv3_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

// 3-D DFT of a ([NZ][NY][NX]); the result ends in a in the layout
// [NY][NX][NZ]; t is clobbered.
template <typename R>
static int dft3(const Conv3Plan<R> &P, typename Conv3Plan<R>::C2 *a, typename Conv3Plan<R>::C2 *t,
                cudaStream_t st)
{
    MPI_TRY(fft_run(P.px, a, t, P.NZ * P.NY, P.NX, P.WX, st));   // along x
    MPI_TRY(transpose_cx(P.NZ * P.NY, P.NX, a, t, st));           // t: [NX][NZ][NY]
    MPI_TRY(fft_run(P.py, t, a, P.NX * P.NZ, P.NY, P.WY, st));   // along y
    MPI_TRY(transpose_cx(P.NX * P.NZ, P.NY, t, a, st));           // a: [NY][NX][NZ]
    return fft_run(P.pz, a, t, P.NY * P.NX, P.NZ, P.WZ, st);     // along z
}

template <typename R>
static int conv3_plan_prepare(const Model3H &m, const Grid3H &g, int kernel, void *scratch, Conv3Plan<R> &P,
                              cudaStream_t st)
{
    using C2 = typename Conv3Plan<R>::C2;
    P.g = g;
    P.fft = conv3_uses_fft(g, sizeof(R));
    R *K = nullptr;
    MPI_TRY(conv3_prepare<R>(m, g, kernel, scratch, &K, st));
    P.K = K;
    if (!P.fft) return MPI_OK;
    P.NX = pow2_at_least(2 * g.nx - 1);
    P.NY = pow2_at_least(2 * g.ny - 1);
    P.NZ = pow2_at_least(2 * g.nz - 1);
    plan_fft(P.NX, P.px);
    plan_fft(P.NY, P.py);
    plan_fft(P.NZ, P.pz);
    char *p = static_cast<char *>(scratch) + ((conv3_kernel_bytes(g, sizeof(R)) + 255) & ~size_t(255));
    auto take = [&](size_t n) {
        C2 *q = reinterpret_cast<C2 *>(p);
        p += (sizeof(C2) * n + 255) & ~size_t(255);
        return q;
    };
    const int64_t n = (int64_t)P.NX * P.NY * P.NZ;
    P.WX = take(P.NX);
    P.WY = take(P.NY);
    P.WZ = take(P.NZ);
    P.Kh = take(n);
    P.a = take(n);
    P.t = take(n);
    MPI_TRY(fft_twiddles(P.NX, P.WX, st));
    MPI_TRY(fft_twiddles(P.NY, P.WY, st));
    MPI_TRY(fft_twiddles(P.NZ, P.WZ, st));
    // The sampled kernel in FP64 is the first piece of the scratch.
    k_conv3_circ<C2><<<conv3_blocks(n), 256, 0, st>>>(g, P.NX, P.NY, P.NZ, static_cast<const double *>(scratch), P.Kh);
    MPI_CHECK_LAUNCH();
    MPI_TRY(dft3(P, P.Kh, P.a, st));
    if (conv3_fused_fits(P.NX, P.NY, P.NZ)) {
        P.fused = true;
        P.LD = conv_fused_ld(P.NX, sizeof(R));
        const int64_t nh = (int64_t)P.NZ * P.NY * P.LD;
        k_conv3_kh_half<C2><<<conv3_blocks(nh), 256, 0, st>>>(P.NX, P.NY, P.NZ, P.LD, P.Kh, P.a);
        MPI_CHECK_LAUNCH();
        MPI_TRY_CUDA(cudaMemcpyAsync(P.Kh, P.a, sizeof(C2) * size_t(nh), cudaMemcpyDeviceToDevice, st));
    }
    return MPI_OK;
}

// The five-launch form of the FFT route: real rows along x in pairs to half
// spectra (the nz ny non-zero rows), the DFT along y of the ny non-zero rows
// per (z, kx group), the fused pass along z (DFT of the nz non-zero planes,
// the spectrum product, inverse DFT, nz kept), the inverse DFT along y (ny
// kept), and the inverse rows along x (cropped to nx, scaled).  The product
// spectrum is Hermitian (real input, point-symmetric kernel), so the half
// kx = 0 .. NX/2 carries it.
template <typename R, typename IN, typename OUT>
static int conv3_apply_fused(const Conv3Plan<R> &P, const IN *in, OUT *out, cudaStream_t st)
{
    using C2 = typename Conv3Plan<R>::C2;
    const Grid3H &g = P.g;
    const int64_t LD = P.LD;
    MPI_TRY((cf_rows_fwd<C2, IN>(g.nx, g.nz * g.ny, P.NX, P.LD, in, P.WX, P.a, st)));  // a: [nz][ny][LD]
    CfCols c{};
    c.LD = P.LD;
    c.mode = kCfFwd;  // along y: t = [nz][NY][LD]
    c.n = P.NY;
    c.n_in = g.ny;
    c.n_out = P.NY;
    c.n_outer = g.nz;
    c.in_outer = g.ny * LD;
    c.in_stride = LD;
    c.out_outer = P.NY * LD;
    c.out_stride = LD;
    MPI_TRY(cf_cols<C2>(c, P.a, nullptr, P.WY, P.t, st));
    c.mode = kCfFused;  // along z, outer index ky: a = [nz][NY][LD]
    c.n = P.NZ;
    c.n_in = c.n_out = g.nz;
    c.n_outer = P.NY;
    c.in_outer = c.out_outer = c.k_outer = LD;
    c.in_stride = c.out_stride = c.k_stride = P.NY * LD;
    MPI_TRY(cf_cols<C2>(c, P.t, P.Kh, P.WZ, P.a, st));
    c.mode = kCfInv;  // along y: t = [nz][ny][LD]
    c.n = P.NY;
    c.n_in = P.NY;
    c.n_out = g.ny;
    c.n_outer = g.nz;
    c.in_outer = P.NY * LD;
    c.in_stride = LD;
    c.out_outer = g.ny * LD;
    c.out_stride = LD;
    c.k_outer = c.k_stride = 0;
    MPI_TRY(cf_cols<C2>(c, P.a, nullptr, P.WY, P.t, st));
    return cf_rows_inv<C2, OUT>(g.nx, g.nz * g.ny, P.NX, P.LD, P.t, P.WX,
                                1.0 / (double(P.NX) * double(P.NY) * double(P.NZ)), out, st);
}

// out = C in (3-D), by the direct sum or the FFT route of the plan.
template <typename R, typename IN, typename OUT>
static int conv3_apply(const Conv3Plan<R> &P, const IN *in, OUT *out, cudaStream_t st)
{
    if (!P.fft) return launch_conv3<R, IN, OUT>(P.g, P.K, in, out, st);
    using C2 = typename Conv3Plan<R>::C2;
    const int64_t n = (int64_t)P.NX * P.NY * P.NZ;
    ProfScope prof(kProfConv, st);
    if (P.fused) return conv3_apply_fused<R, IN, OUT>(P, in, out, st);
    k_conv3_load<IN, C2><<<conv3_blocks(n), 256, 0, st>>>(P.g, P.NX, P.NY, P.NZ, in, P.a);
    MPI_CHECK_LAUNCH();
    MPI_TRY(dft3(P, P.a, P.t, st));
    MPI_TRY(spec_mul_conj(n, P.a, P.Kh, st));
    // DFT of the conjugated product back through the axes in reverse order.
    MPI_TRY(fft_run(P.pz, P.a, P.t, P.NY * P.NX, P.NZ, P.WZ, st));   // along z
    MPI_TRY(transpose_cx(P.NY, P.NX * P.NZ, P.a, P.t, st));           // t: [NX][NZ][NY]
    MPI_TRY(fft_run(P.py, P.t, P.a, P.NX * P.NZ, P.NY, P.WY, st));   // along y
    MPI_TRY(transpose_cx(P.NX, P.NZ * P.NY, P.t, P.a, st));           // a: [NZ][NY][NX]
    MPI_TRY(fft_run(P.px, P.a, P.t, P.NZ * P.NY, P.NX, P.WX, st));   // along x
    k_conv3_crop<OUT, C2><<<conv3_blocks(P.g.n()), 256, 0, st>>>(P.g, P.NX, P.NY, P.a, 1.0 / double(n), out);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// ---------------------------------------------------------------------------
// Built-in denoiser on a volume: the 5-tap Gaussian along x, then y, then z.

template <typename R>
__global__ void k_gauss3(const R *__restrict__ in, R *__restrict__ out, int nx, int ny, int nz, int axis,
                         R w0, R w1, R w2)
{
    const int64_t N = (int64_t)nx * ny * nz;
    const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const int64_t stride = axis == 0 ? 1 : (axis == 1 ? nx : (int64_t)nx * ny);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)((e / stride) % n);
        const int64_t base = e - (int64_t)k * stride;
        const R w[5] = {w2, w1, w0, w1, w2};
        R acc = R(0);
#pragma unroll
        for (int m = -2; m <= 2; ++m) acc = fmx(w[m + 2], in[base + (int64_t)reflect_index(k + m, n) * stride], acc);
        out[e] = acc;
    }
}

template <typename R>
static int launch_gauss3(const R *in, R *out, R *tmp, int nx, int ny, int nz, cudaStream_t st)
{
    double w[3];
    gauss5_weights(w);
    const int64_t N = (int64_t)nx * ny * nz;
    const unsigned blocks = (unsigned)std::min<int64_t>((N + 255) / 256, 8192);
    k_gauss3<R><<<blocks, 256, 0, st>>>(in, out, nx, ny, nz, 0, R(w[0]), R(w[1]), R(w[2]));
    MPI_CHECK_LAUNCH();
    k_gauss3<R><<<blocks, 256, 0, st>>>(out, tmp, nx, ny, nz, 1, R(w[0]), R(w[1]), R(w[2]));
    MPI_CHECK_LAUNCH();
    k_gauss3<R><<<blocks, 256, 0, st>>>(tmp, out, nx, ny, nz, 2, R(w[0]), R(w[1]), R(w[2]));
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// ---------------------------------------------------------------------------
// PnP (Algorithm 1) with the 3-D operators.

template <typename R>
struct PnPOp3D final : PnPOperator<R> {
    mpi_op op;
    Op3<R> A;
    Grid3H g;
    int64_t N = 0;
    Conv3Plan<R> C;
    R *sA = nullptr, *tmp1 = nullptr, *tmp2 = nullptr, *gtmp = nullptr;
    mpi_denoise3_fn den = nullptr;
    void *user = nullptr;

    int rhs(const R *data, double *b0, cudaStream_t st) override
    {
        if (op == MPI_OP_FORWARD) return A.template adjoint<double>(data, b0, nullptr, nullptr, nullptr, st);
        return conv3_apply<R, R, double>(C, data, b0, st);
    }
    int apply_normal(const double *v, double *q, const double *nu_dev, double *pq_part,
                     cudaStream_t st) override
    {
        if (op == MPI_OP_FORWARD) {
            MPI_TRY((A.template forward<double, R>(v, sA, st)));
            return A.template adjoint<double>(sA, q, v, nu_dev, pq_part, st);
        }
        MPI_TRY((conv3_apply<R, double, R>(C, v, tmp1, st)));
        MPI_TRY((conv3_apply<R, R, R>(C, tmp1, tmp2, st)));
        return axpy_dot_launch<R>(N, tmp2, v, nu_dev, q, pq_part, st);
    }
    int n_pq() const override { return op == MPI_OP_FORWARD ? reduce_dot_blocks(N) : vec_blocks(N); }
    int denoise(const R *in, R *out, const double *sigma_dev, cudaStream_t st) override
    {
        if (den) return den(in, out, g.nx, g.ny, g.nz, sizeof(R) == 4 ? MPI_F32 : MPI_F64, sigma_dev, st, user);
        return launch_gauss3<R>(in, out, gtmp, g.nx, g.ny, g.nz, st);
    }
    bool has_callback() const override { return den != nullptr; }
};

template <typename R>
static int pnp3_impl(const Model3H &m, const Grid3H &g, const mpi_traj *tr, const void *data,
                     const mpi_pnp_opts &o, mpi_denoise3_fn den, void *user, void *rho_out,
                     mpi_pnp_iter_info *info, cudaStream_t st)
{
    PnPOp3D<R> S;
    S.op = o.op;
    S.g = g;
    S.N = g.n();
    S.den = den;
    S.user = user;
    Scratch scr(st);
    size_t o_A = 0, o_sA = 0, o_K = 0, o_t1 = 0, o_t2 = 0;
    if (o.op == MPI_OP_FORWARD) {
        S.A.plan(m, g, tr->T);
        o_A = scr.reserve(S.A.scratch_bytes());
        o_sA = scr.reserve(sizeof(R) * size_t(m.n_ch) * size_t(std::max<int64_t>(tr->T, 1)));
    } else {
        o_K = scr.reserve(conv3_plan_bytes(g, sizeof(R)));
        o_t1 = scr.reserve(sizeof(R) * S.N);
        o_t2 = scr.reserve(sizeof(R) * S.N);
    }
    const size_t o_g = scr.reserve(sizeof(R) * S.N);
    MPI_TRY(scr.allocate());
    S.gtmp = scr.at<R>(o_g);
    if (o.op == MPI_OP_FORWARD) {
        S.A.carve(scr.at<char>(o_A));
        S.sA = scr.at<R>(o_sA);
        MPI_TRY(S.A.prepare(static_cast<const R *>(tr->r), static_cast<const R *>(tr->v), st));
    } else {
        MPI_TRY(conv3_plan_prepare<R>(m, g, o.kernel_component, scr.at<char>(o_K), S.C, st));
        S.tmp1 = scr.at<R>(o_t1);
        S.tmp2 = scr.at<R>(o_t2);
    }
    return pnp_run<R>(S, S.N, data, o, rho_out, info, st);
}

// ---------------------------------------------------------------------------
// Validation and entry points.

static int check_model3(const mpi_model3 *m)
{
    if (!m) { set_error("model is NULL"); return MPI_ERR_INVALID; }
    if (!(m->beta > 0.0) || !std::isfinite(m->beta)) {
        set_error("beta must be positive and finite (got %g)", m->beta);
        return MPI_ERR_INVALID;
    }
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(m->G[k])) { set_error("G has a non-finite entry"); return MPI_ERR_INVALID; }
    const double *G = m->G;
    const double det = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                       G[2] * (G[3] * G[7] - G[4] * G[6]);
    if (det == 0.0) { set_error("G is singular"); return MPI_ERR_INVALID; }
    if (m->n_ch < 1 || m->n_ch > 3) {
        set_error("n_ch must be 1, 2 or 3 (got %d)", m->n_ch);
        return MPI_ERR_INVALID;
    }
    for (int k = 0; k < 3 * m->n_ch; ++k)
        if (!std::isfinite(m->p[k])) { set_error("p has a non-finite entry"); return MPI_ERR_INVALID; }
    return MPI_OK;
}

int check_grid3(const mpi_grid3_desc *g)
{
    if (!g) { set_error("grid is NULL"); return MPI_ERR_INVALID; }
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) {
        set_error("grid must have nx, ny, nz >= 1 (got %d x %d x %d)", g->nx, g->ny, g->nz);
        return MPI_ERR_INVALID;
    }
    if ((int64_t)g->nx * g->ny * g->nz > (int64_t)1 << 28) {
        set_error("grid of %d x %d x %d voxels is larger than supported (2^28)", g->nx, g->ny, g->nz);
        return MPI_ERR_UNSUPPORTED;
    }
    const double v[6] = {g->x0, g->y0, g->z0, g->dx, g->dy, g->dz};
    for (double q : v)
        if (!std::isfinite(q)) { set_error("grid origin and spacing must be finite"); return MPI_ERR_INVALID; }
    if (g->dx == 0.0 || g->dy == 0.0 || g->dz == 0.0) {
        set_error("grid spacing must be nonzero");
        return MPI_ERR_INVALID;
    }
    return MPI_OK;
}

static Model3H to_host3(const mpi_model3 *m)
{
    Model3H h;
    h.beta = m->beta;
    for (int k = 0; k < 9; ++k) h.G[k] = m->G[k];
    h.n_ch = m->n_ch;
    for (int k = 0; k < 9; ++k) h.p[k] = k < 3 * m->n_ch ? m->p[k] : 0.0;
    return h;
}
static Grid3H to_host3(const mpi_grid3_desc *g)
{
    return Grid3H{g->nx, g->ny, g->nz, g->x0, g->y0, g->z0, g->dx, g->dy, g->dz};
}

template <typename R>
static int forward3_impl(const Model3H &m, const Grid3H &g, const mpi_traj *tr, const void *c, void *s,
                         cudaStream_t st)
{
    if (tr->T == 0) return MPI_OK;
    Op3<R> A;
    A.plan(m, g, tr->T);
    Scratch scr(st);
    const size_t o = scr.reserve(A.scratch_bytes());
    MPI_TRY(scr.allocate());
    A.carve(scr.at<char>(o));
    MPI_TRY(A.prepare(static_cast<const R *>(tr->r), static_cast<const R *>(tr->v), st));
    return A.template forward<R, R>(static_cast<const R *>(c), static_cast<R *>(s), st);
}

template <typename R>
static int adjoint3_impl(const Model3H &m, const Grid3H &g, const mpi_traj *tr, const void *s, void *c_out,
                         cudaStream_t st)
{
    Op3<R> A;
    A.plan(m, g, tr->T);
    Scratch scr(st);
    const size_t o = scr.reserve(A.scratch_bytes());
    MPI_TRY(scr.allocate());
    A.carve(scr.at<char>(o));
    MPI_TRY(A.prepare(static_cast<const R *>(tr->r), static_cast<const R *>(tr->v), st));
    return A.template adjoint<R>(static_cast<const R *>(s), static_cast<R *>(c_out), nullptr, nullptr,
                                 nullptr, st);
}

template <typename R>
static int conv3_impl(const Model3H &m, const Grid3H &g, int kernel, const void *in, void *out, cudaStream_t st)
{
    Scratch scr(st);
    const size_t o_K = scr.reserve(conv3_plan_bytes(g, sizeof(R)));
    MPI_TRY(scr.allocate());
    Conv3Plan<R> C;
    MPI_TRY(conv3_plan_prepare<R>(m, g, kernel, scr.at<char>(o_K), C, st));
    return conv3_apply<R, R, R>(C, static_cast<const R *>(in), static_cast<R *>(out), st);
}

// out = tr(Ahat G^-1) per node: sum_{k,m} Ahat[3k+m] (G^-1)_mk, in FP64.
template <typename R>
__global__ void k_weighted_trace3(int64_t N, Mat3 Gi, const R *__restrict__ A, R *__restrict__ out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int q = 0; q < 3; ++q) acc += double(A[(3 * k + q) * N + e]) * Gi.a[3 * q + k];
        out[e] = R(acc);
    }
}

static Mat3 inverse3(const double *G)
{
    const double det = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                       G[2] * (G[3] * G[7] - G[4] * G[6]);
    Mat3 I;
    I.a[0] = (G[4] * G[8] - G[5] * G[7]) / det;
    I.a[1] = (G[2] * G[7] - G[1] * G[8]) / det;
    I.a[2] = (G[1] * G[5] - G[2] * G[4]) / det;
    I.a[3] = (G[5] * G[6] - G[3] * G[8]) / det;
    I.a[4] = (G[0] * G[8] - G[2] * G[6]) / det;
    I.a[5] = (G[2] * G[3] - G[0] * G[5]) / det;
    I.a[6] = (G[3] * G[7] - G[4] * G[6]) / det;
    I.a[7] = (G[1] * G[6] - G[0] * G[7]) / det;
    I.a[8] = (G[0] * G[4] - G[1] * G[3]) / det;
    return I;
}

template <typename R>
static int weighted_trace3_impl(const Model3H &m, const Grid3H &g, const void *A, void *out, cudaStream_t st)
{
    const int64_t N = g.n();
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 8192));
    k_weighted_trace3<R><<<blocks, 256, 0, st>>>(N, inverse3(m.G), static_cast<const R *>(A), static_cast<R *>(out));
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename R>
static int gauss3_impl(const void *in, void *out, int nx, int ny, int nz, cudaStream_t st)
{
    Scratch scr(st);
    const size_t o_t = scr.reserve(sizeof(R) * (size_t)nx * ny * nz);
    MPI_TRY(scr.allocate());
    return launch_gauss3<R>(static_cast<const R *>(in), static_cast<R *>(out), scr.at<R>(o_t), nx, ny, nz, st);
}

}  // namespace mpi

using namespace mpi;

extern "C" {

int mpi_forward3(const mpi_model3 *model, const mpi_grid3_desc *grid, const mpi_traj *traj,
                 mpi_dtype dtype, const void *c, void *s, void *stream)
{
    MPI_TRY(check_model3(model));
    MPI_TRY(check_grid3(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (traj->T > 0 && (!c || !s)) { set_error("c or s is NULL"); return MPI_ERR_INVALID; }
    const Model3H m = to_host3(model);
    const Grid3H g = to_host3(grid);
    return dtype == MPI_F32 ? forward3_impl<float>(m, g, traj, c, s, as_stream(stream))
                            : forward3_impl<double>(m, g, traj, c, s, as_stream(stream));
}

int mpi_adjoint3(const mpi_model3 *model, const mpi_grid3_desc *grid, const mpi_traj *traj,
                 mpi_dtype dtype, const void *s, void *c_out, void *stream)
{
    MPI_TRY(check_model3(model));
    MPI_TRY(check_grid3(grid));
    MPI_TRY(check_traj(traj));
    MPI_TRY(check_dtype(dtype));
    if (!c_out || (traj->T > 0 && !s)) { set_error("s or c_out is NULL"); return MPI_ERR_INVALID; }
    const Model3H m = to_host3(model);
    const Grid3H g = to_host3(grid);
    return dtype == MPI_F32 ? adjoint3_impl<float>(m, g, traj, s, c_out, as_stream(stream))
                            : adjoint3_impl<double>(m, g, traj, s, c_out, as_stream(stream));
}

int mpi_conv3_kernel(const mpi_model3 *model, const mpi_grid3_desc *grid, mpi_dtype dtype, int kernel,
                     const void *in, void *out, void *stream)
{
    MPI_TRY(check_model3(model));
    MPI_TRY(check_grid3(grid));
    MPI_TRY(check_dtype(dtype));
    if (kernel != 0 && kernel != 1) { set_error("kernel must be 0 or 1 (got %d)", kernel); return MPI_ERR_INVALID; }
    if (!in || !out || in == out) { set_error("in/out NULL or aliased"); return MPI_ERR_INVALID; }
    const Model3H m = to_host3(model);
    const Grid3H g = to_host3(grid);
    return dtype == MPI_F32 ? conv3_impl<float>(m, g, kernel, in, out, as_stream(stream))
                            : conv3_impl<double>(m, g, kernel, in, out, as_stream(stream));
}

int mpi_conv3(const mpi_model3 *model, const mpi_grid3_desc *grid, mpi_dtype dtype, const void *in,
              void *out, void *stream)
{
    return mpi_conv3_kernel(model, grid, dtype, 0, in, out, stream);
}

int mpi_weighted_trace3(const mpi_model3 *model, const mpi_grid3_desc *grid, mpi_dtype dtype, const void *Ahat,
                        void *out, void *stream)
{
    MPI_TRY(check_model3(model));
    MPI_TRY(check_grid3(grid));
    MPI_TRY(check_dtype(dtype));
    if (!Ahat || !out) { set_error("Ahat or out is NULL"); return MPI_ERR_INVALID; }
    const Model3H m = to_host3(model);
    const Grid3H g = to_host3(grid);
    return dtype == MPI_F32 ? weighted_trace3_impl<float>(m, g, Ahat, out, as_stream(stream))
                            : weighted_trace3_impl<double>(m, g, Ahat, out, as_stream(stream));
}

int mpi_denoise_gaussian5_3d(const void *in, void *out, int nx, int ny, int nz, mpi_dtype dtype,
                             const double *sigma_dev, void *stream, void *user)
{
    (void)sigma_dev;
    (void)user;
    MPI_TRY(check_dtype(dtype));
    if (nx < 1 || ny < 1 || nz < 1 || !in || !out || in == out) {
        set_error("invalid denoiser arguments");
        return MPI_ERR_INVALID;
    }
    return dtype == MPI_F32 ? gauss3_impl<float>(in, out, nx, ny, nz, as_stream(stream))
                            : gauss3_impl<double>(in, out, nx, ny, nz, as_stream(stream));
}

int mpi_pnp_solve3(const mpi_model3 *model, const mpi_grid3_desc *grid, const mpi_traj *traj,
                   mpi_dtype dtype, const void *data, const mpi_pnp_opts *opts, mpi_denoise3_fn denoise,
                   void *user, void *rho_out, mpi_pnp_iter_info *info, void *stream)
{
    MPI_TRY(check_model3(model));
    MPI_TRY(check_grid3(grid));
    MPI_TRY(check_dtype(dtype));
    if (!opts) { set_error("opts is NULL"); return MPI_ERR_INVALID; }
    if (opts->op != MPI_OP_FORWARD && opts->op != MPI_OP_CONV) {
        set_error("unknown operator %d", (int)opts->op);
        return MPI_ERR_INVALID;
    }
    if (opts->op == MPI_OP_FORWARD) MPI_TRY(check_traj(traj));
    if (opts->n_iter < 0 || opts->n_cg < 0 || !(opts->nu0 >= 0.0) || !std::isfinite(opts->nu0) ||
        !(opts->clip_pct <= 100.0) || std::isnan(opts->clip_pct) || opts->kernel_component < 0 ||
        opts->kernel_component > (opts->op == MPI_OP_CONV ? 1 : 0)) {
        set_error("invalid PnP options (n_iter %d, n_cg %d, nu0 %g, clip_pct %g, kernel_component %d)",
                  opts->n_iter, opts->n_cg, opts->nu0, opts->clip_pct, opts->kernel_component);
        return MPI_ERR_INVALID;
    }
    if (!rho_out || (!data && !(opts->op == MPI_OP_FORWARD && traj->T == 0))) {
        set_error("data or rho_out is NULL");
        return MPI_ERR_INVALID;
    }
    const Model3H m = to_host3(model);
    const Grid3H g = to_host3(grid);
    return dtype == MPI_F32
               ? pnp3_impl<float>(m, g, traj, data, *opts, denoise, user, rho_out, info, as_stream(stream))
               : pnp3_impl<double>(m, g, traj, data, *opts, denoise, user, rho_out, info, as_stream(stream));
}

}  // extern "C"
