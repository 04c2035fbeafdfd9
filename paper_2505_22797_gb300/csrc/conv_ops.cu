// Convolution with the sampled trace kernel (Eq. convolution:trace,
// Eq. kernel:trace; the matrix C_h of Eq. dec:sub:tik), realised as the
// exact linear (zero-padded) convolution over all voxel offsets:
//   out[j][i] = sum_{j'i'} kappa_G(x_ij - x_i'j') in[j'][i'],
//   kappa_G(y) = beta tr(K(beta G y) G).
// The kernel is sampled once per call in FP64.  Two routes compute the same
// sum:
//  * direct (small grids): N^2 FMAs in the call's type; each block computes a
//    16 x 16 output tile and walks the input in 16 x 16 tiles staged with the
//    matching kernel window in shared memory; per-tile sums are folded with
//    compensated additions;
//  * FFT (from 64 x 64 in FP32 and 32 x 32 in FP64, where it overtakes the
//    direct sum on GB300): the kernel placed circularly on an NY x NX grid,
//    NX and NY the powers of two >= 2 nx - 1 and 2 ny - 1,
//    so the circular convolution of the zero-padded input equals the linear
//    one on the nx x ny window; 2-D DFTs in the call's precision (FP32 for
//    FP32 calls: GB300's FP64 pipe bounds FP64 passes), as row passes of the
//    Stockham FFT, a tiled transpose and row passes again; the kernel's
//    spectrum kept in
//    the transposed layout, the inverse by the conjugation identity
//    IDFT(Y) = conj(DFT(conj Y)) / n.  O(N log N) instead of N^2.  Grids whose
//    transforms fit in shared memory take the three-launch form of
//    conv_fft2.cu (real rows in pairs, half spectra, fused column pass).
#include <algorithm>

#include "conv_ops.cuh"
#include "fft.cuh"
#include "langevin.cuh"

namespace mpi {

constexpr int kConvT = 16;  // output / input tile edge

__global__ void k_conv_kernel_sample(int nx, int ny, double dx, double dy, double beta,
                                     double g00, double g01, double g10, double g11, int comp,
                                     double *__restrict__ K)
{
    const int KX = 2 * nx - 1, KY = 2 * ny - 1;
    const int64_t n = (int64_t)KX * KY;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int ii = (int)(e % KX), jj = (int)(e / KX);
        const double ox = (ii - (nx - 1)) * dx, oy = (jj - (ny - 1)) * dy;
        const double yx = beta * (g00 * ox + g01 * oy);
        const double yy = beta * (g10 * ox + g11 * oy);
        const double u = yx * yx + yy * yy;
        double a, d;
        lang_checked<double, false>(u, a, d);
        // K = a I + d y y^T;  (K G)_ab = a G_ab + d y_a (G^T y)_b
        double val;
        if (comp < 0) {  // tr(K G) = a tr G + d y^T G y
            val = a * (g00 + g11) + d * (yx * (g00 * yx + g01 * yy) + yy * (g10 * yx + g11 * yy));
        } else {
            const int ra = comp >> 1, cb = comp & 1;
            const double Gab = ra == 0 ? (cb == 0 ? g00 : g01) : (cb == 0 ? g10 : g11);
            const double ya = ra == 0 ? yx : yy;
            const double gty = cb == 0 ? g00 * yx + g10 * yy : g01 * yx + g11 * yy;
            val = a * Gab + d * ya * gty;
        }
        K[e] = beta * val;
    }
}

template <typename R>
__global__ void k_round(const double *__restrict__ in, R *__restrict__ out, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = R(in[e]);
}

size_t conv_kernel_bytes(int nx, int ny, int elem_bytes)
{
    return size_t(2 * nx - 1) * size_t(2 * ny - 1) * (sizeof(double) + elem_bytes) + 512;
}

template <typename R>
int conv_prepare_kernel(const ModelH &m, const GridH &g, void *scratch, R **K_out, cudaStream_t st,
                        int comp)
{
    const int64_t n = (int64_t)(2 * g.nx - 1) * (2 * g.ny - 1);
    double *K64 = static_cast<double *>(scratch);
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_conv_kernel_sample<<<blocks, 256, 0, st>>>(g.nx, g.ny, g.dx, g.dy, m.beta, m.G[0], m.G[1],
                                                 m.G[2], m.G[3], comp, K64);
    MPI_CHECK_LAUNCH();
    if constexpr (sizeof(R) == sizeof(double)) {
        *K_out = reinterpret_cast<R *>(K64);
    } else {
        char *p = static_cast<char *>(scratch) + ((sizeof(double) * n + 255) & ~size_t(255));
        R *K = reinterpret_cast<R *>(p);
        k_round<R><<<blocks, 256, 0, st>>>(K64, K, n);
        MPI_CHECK_LAUNCH();
        *K_out = K;
    }
    return MPI_OK;
}

// out = C in.
template <typename R, typename IN, typename OUT>
__global__ void __launch_bounds__(kConvT *kConvT)
k_conv_direct(int nx, int ny, const R *__restrict__ K, const IN *__restrict__ in,
              OUT *__restrict__ out)
{
    __shared__ R s_in[kConvT][kConvT];
    __shared__ R s_k[2 * kConvT - 1][2 * kConvT];
    const int tx = threadIdx.x % kConvT, ty = threadIdx.x / kConvT;
    const int i0 = blockIdx.x * kConvT, j0 = blockIdx.y * kConvT;
    const int i = i0 + tx, j = j0 + ty;
    const int KX = 2 * nx - 1;
    R acc = R(0), comp = R(0);
    for (int jq0 = 0; jq0 < ny; jq0 += kConvT) {
        for (int iq0 = 0; iq0 < nx; iq0 += kConvT) {
            __syncthreads();
            {
                const int iq = iq0 + tx, jq = jq0 + ty;
                s_in[ty][tx] = (iq < nx && jq < ny) ? R(in[(int64_t)jq * nx + iq]) : R(0);
            }
            // kernel window: offsets (j - jq) in [j0 - jq0 - (T-1), j0 - jq0 + (T-1)]
            for (int e = threadIdx.x; e < (2 * kConvT - 1) * (2 * kConvT - 1); e += kConvT * kConvT) {
                const int ex = e % (2 * kConvT - 1), ey = e / (2 * kConvT - 1);
                const int oi = i0 - iq0 - (kConvT - 1) + ex;  // offset i - iq
                const int oj = j0 - jq0 - (kConvT - 1) + ey;
                const bool ok = oi > -nx && oi < nx && oj > -ny && oj < ny;
                s_k[ey][ex] = ok ? K[(int64_t)(oj + ny - 1) * KX + (oi + nx - 1)] : R(0);
            }
            __syncthreads();
            R part = R(0);
#pragma unroll 4
            for (int b = 0; b < kConvT; ++b) {
                // offset index for (j - jq) = ty - b + (j0 - jq0): window row ty - b + T - 1
#pragma unroll
                for (int a = 0; a < kConvT; ++a)
                    part += s_k[ty - b + kConvT - 1][tx - a + kConvT - 1] * s_in[b][a];
            }
            kahan_add(acc, comp, part);
        }
    }
    if (i < nx && j < ny) out[(int64_t)j * nx + i] = OUT(acc);
}

template <typename R, typename IN, typename OUT>
int launch_conv(const GridH &g, const R *K, const IN *in, OUT *out, cudaStream_t st)
{
    dim3 grid((g.nx + kConvT - 1) / kConvT, (g.ny + kConvT - 1) / kConvT);
    ProfScope prof(kProfConv, st);
    k_conv_direct<R, IN, OUT><<<grid, kConvT * kConvT, 0, st>>>(g.nx, g.ny, K, in, out);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// ---------------------------------------------------------------------------
// FFT route.

// Smallest grid (voxels) for the FFT route: where it overtook the direct sum
// on GB300 (FP32: 64 x 64; FP64, whose direct sum runs on the slow FP64 pipe:
// 32 x 32).
#ifndef MPI_CONV_FFT_MIN_N
#define MPI_CONV_FFT_MIN_N 4096
#endif
#ifndef MPI_CONV_FFT_MIN_N64
#define MPI_CONV_FFT_MIN_N64 1024
#endif

// The three-launch route for the grids it fits (conv_fft2.cu); 0 keeps the
// nine-launch route everywhere.
#ifndef MPI_CONV_FUSED
#define MPI_CONV_FUSED 1
#endif

// Padded length: the power of two >= n (radix-4/2 passes only; measured on
// GB300 faster than the shortest 7-smooth length, whose radix-5/7 passes take
// the generic butterfly).
static int nice_length(int n)
{
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    return p2;
}

bool conv_uses_fft(int nx, int ny, int elem_bytes)
{
    return (int64_t)nx * ny >= (elem_bytes == 8 ? MPI_CONV_FFT_MIN_N64 : MPI_CONV_FFT_MIN_N);
}

// The sampled kernel placed circularly: kc[dj mod NY][di mod NX] = K[dj][di].
template <typename C>
__global__ void k_conv_circ(int nx, int ny, int NX, int NY, const double *__restrict__ K,
                            C *__restrict__ kc)
{
    const int KX = 2 * nx - 1;
    const int64_t n = (int64_t)NX * NY;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % NX), j = (int)(e / NX);
        const int di = i < nx ? i : i - NX, dj = j < ny ? j : j - NY;
        double v = 0.0;
        if (di > -nx && di < nx && dj > -ny && dj < ny) v = K[(int64_t)(dj + ny - 1) * KX + (di + nx - 1)];
        kc[e] = make_cx<C>(v, 0.0);
    }
}

template <typename IN, typename C>
__global__ void k_conv_load(int nx, int ny, int NX, int NY, const IN *__restrict__ in, C *__restrict__ a)
{
    const int64_t n = (int64_t)NX * NY;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % NX), j = (int)(e / NX);
        a[e] = make_cx<C>(i < nx && j < ny ? double(in[(int64_t)j * nx + i]) : 0.0, 0.0);
    }
}

// dst[c][r] = src[r][c] for a rows x cols complex matrix (32 x 32 tiles).
template <typename C>
__global__ void __launch_bounds__(32 * 8)
k_transpose_c(int rows, int cols, const C *__restrict__ src, C *__restrict__ dst)
{
    __shared__ C tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = src[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(int64_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

template <typename C>
__global__ void k_spec_mul_conj(int64_t n, C *__restrict__ t, const C *__restrict__ kh)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const C p = cmul(t[e], kh[e]);
        t[e] = cxv(p.x, -p.y);
    }
}

template <typename OUT, typename C>
__global__ void k_conv_crop(int nx, int ny, int NX, const C *__restrict__ a, double scale,
                            OUT *__restrict__ out)
{
    const int64_t n = (int64_t)nx * ny;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % nx), j = (int)(e / nx);
        out[e] = OUT(double(a[(int64_t)j * NX + i].x) * scale);
    }
}

static unsigned elem_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

template <typename C>
static int transpose_c(int rows, int cols, const C *src, C *dst, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    k_transpose_c<C><<<grid, dim3(32, 8), 0, st>>>(rows, cols, src, dst);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// 2-D DFT of a [NY][NX] (in a); result transposed, [NX][NY], in t.  a is
// clobbered (it is the ping-pong partner of the column passes).
template <typename R>
static int dft2_to_t(const ConvPlan<R> &P, typename ConvPlan<R>::C2 *a, typename ConvPlan<R>::C2 *t,
                     cudaStream_t st)
{
    MPI_TRY(fft_run(P.px, a, t, P.NY, P.NX, P.WX, st));
    MPI_TRY(transpose_c(P.NY, P.NX, a, t, st));
    return fft_run(P.py, t, a, P.NX, P.NY, P.WY, st);
}

size_t conv_plan_bytes(int nx, int ny, int elem_bytes)
{
    size_t b = conv_kernel_bytes(nx, ny, elem_bytes);
    if (conv_uses_fft(nx, ny, elem_bytes)) {
        const size_t NX = nice_length(2 * nx - 1), NY = nice_length(2 * ny - 1);
        b += 2 * size_t(elem_bytes) * (NX + NY + 3 * NX * NY) + 6 * 256;
    }
    return b;
}

template <typename R>
int conv_plan_prepare(const ModelH &m, const GridH &g, void *scratch, ConvPlan<R> &P, cudaStream_t st, int comp)
{
    P.nx = g.nx;
    P.ny = g.ny;
    P.fft = conv_uses_fft(g.nx, g.ny, sizeof(R));
    R *K = nullptr;
    MPI_TRY(conv_prepare_kernel<R>(m, g, scratch, &K, st, comp));
    P.K = K;
    if (!P.fft) return MPI_OK;
    P.NX = nice_length(2 * g.nx - 1);
    P.NY = nice_length(2 * g.ny - 1);
    plan_fft(P.NX, P.px);
    plan_fft(P.NY, P.py);
    char *p = static_cast<char *>(scratch) + ((conv_kernel_bytes(g.nx, g.ny, sizeof(R)) + 255) & ~size_t(255));
    using C2 = typename ConvPlan<R>::C2;
    auto take = [&](size_t n) {
        C2 *q = reinterpret_cast<C2 *>(p);
        p += (sizeof(C2) * n + 255) & ~size_t(255);
        return q;
    };
    const int64_t n = (int64_t)P.NX * P.NY;
    P.WX = take(P.NX);
    P.WY = take(P.NY);
    P.Kh = take(n);
    P.a = take(n);
    P.t = take(n);
    MPI_TRY(fft_twiddles(P.NX, P.WX, st));
    MPI_TRY(fft_twiddles(P.NY, P.WY, st));
    // The sampled kernel in FP64 is the first piece of the scratch.
    k_conv_circ<C2><<<elem_blocks(n), 256, 0, st>>>(g.nx, g.ny, P.NX, P.NY, static_cast<const double *>(scratch), P.a);
    MPI_CHECK_LAUNCH();
    MPI_TRY(dft2_to_t(P, P.a, P.Kh, st));
    if (MPI_CONV_FUSED && conv_fused_fits(P.NX, P.NY)) {
        P.fused = true;
        P.LD = conv_fused_ld(P.NX, sizeof(R));
        MPI_TRY(conv_fused_kernel<C2>(P.NX, P.NY, P.LD, P.Kh, P.a, st));
    }
    return MPI_OK;
}

template <typename R, typename IN, typename OUT>
int conv_apply(const ConvPlan<R> &P, const IN *in, OUT *out, cudaStream_t st)
{
    if (!P.fft) {
        GridH g{};
        g.nx = P.nx;
        g.ny = P.ny;
        return launch_conv<R, IN, OUT>(g, P.K, in, out, st);
    }
    ProfScope prof(kProfConv, st);
    if (P.fused) return conv_apply_fused<R, IN, OUT>(P, in, out, st);
    const int64_t n = (int64_t)P.NX * P.NY;
    using C2 = typename ConvPlan<R>::C2;
    k_conv_load<IN, C2><<<elem_blocks(n), 256, 0, st>>>(P.nx, P.ny, P.NX, P.NY, in, P.a);
    MPI_CHECK_LAUNCH();
    MPI_TRY(dft2_to_t(P, P.a, P.t, st));
    k_spec_mul_conj<C2><<<elem_blocks(n), 256, 0, st>>>(n, P.t, P.Kh);
    MPI_CHECK_LAUNCH();
    // DFT of the conjugated product: columns (rows of t), transpose back, rows.
    MPI_TRY(fft_run(P.py, P.t, P.a, P.NX, P.NY, P.WY, st));
    MPI_TRY(transpose_c(P.NX, P.NY, P.t, P.a, st));
    MPI_TRY(fft_run(P.px, P.a, P.t, P.NY, P.NX, P.WX, st));
    k_conv_crop<OUT, C2><<<elem_blocks((int64_t)P.nx * P.ny), 256, 0, st>>>(P.nx, P.ny, P.NX, P.a, 1.0 / double(n), out);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

int transpose_cx(int rows, int cols, const float2 *src, float2 *dst, cudaStream_t st)
{
    return transpose_c(rows, cols, src, dst, st);
}
int transpose_cx(int rows, int cols, const double2 *src, double2 *dst, cudaStream_t st)
{
    return transpose_c(rows, cols, src, dst, st);
}
template <typename C>
static int spec_mul_conj_t(int64_t n, C *t, const C *kh, cudaStream_t st)
{
    k_spec_mul_conj<C><<<elem_blocks(n), 256, 0, st>>>(n, t, kh);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}
int spec_mul_conj(int64_t n, float2 *t, const float2 *kh, cudaStream_t st) { return spec_mul_conj_t(n, t, kh, st); }
int spec_mul_conj(int64_t n, double2 *t, const double2 *kh, cudaStream_t st) { return spec_mul_conj_t(n, t, kh, st); }

template int conv_plan_prepare<float>(const ModelH &, const GridH &, void *, ConvPlan<float> &, cudaStream_t, int);
template int conv_plan_prepare<double>(const ModelH &, const GridH &, void *, ConvPlan<double> &, cudaStream_t, int);
template int conv_apply<float, float, float>(const ConvPlan<float> &, const float *, float *, cudaStream_t);
template int conv_apply<float, double, float>(const ConvPlan<float> &, const double *, float *, cudaStream_t);
template int conv_apply<float, float, double>(const ConvPlan<float> &, const float *, double *, cudaStream_t);
template int conv_apply<double, double, double>(const ConvPlan<double> &, const double *, double *, cudaStream_t);

template int conv_prepare_kernel<float>(const ModelH &, const GridH &, void *, float **, cudaStream_t, int);
template int conv_prepare_kernel<double>(const ModelH &, const GridH &, void *, double **, cudaStream_t, int);
template int launch_conv<float, float, float>(const GridH &, const float *, const float *, float *, cudaStream_t);
template int launch_conv<float, double, float>(const GridH &, const float *, const double *, float *, cudaStream_t);
template int launch_conv<float, float, double>(const GridH &, const float *, const float *, double *, cudaStream_t);
template int launch_conv<double, double, double>(const GridH &, const double *, const double *, double *, cudaStream_t);

}  // namespace mpi
