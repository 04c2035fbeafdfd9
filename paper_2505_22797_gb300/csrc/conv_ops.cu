// Convolution with the sampled trace kernel (Eq. convolution:trace,
// Eq. kernel:trace; the matrix C_h of Eq. dec:sub:tik), realised as the
// exact linear (zero-padded) convolution over all voxel offsets:
//   out[j][i] = sum_{j'i'} kappa_G(x_ij - x_i'j') in[j'][i'],
//   kappa_G(y) = beta tr(K(beta G y) G).
// The kernel is sampled once per call in FP64 and rounded to the call's type.
// The direct sum costs N^2 FMAs; each block computes a 16 x 16 output tile
// and walks the input in 16 x 16 tiles staged with the matching kernel window
// in shared memory.  Per-tile sums are folded with compensated additions.
#include <algorithm>

#include "conv_ops.cuh"
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

template int conv_prepare_kernel<float>(const ModelH &, const GridH &, void *, float **, cudaStream_t, int);
template int conv_prepare_kernel<double>(const ModelH &, const GridH &, void *, double **, cudaStream_t, int);
template int launch_conv<float, float, float>(const GridH &, const float *, const float *, float *, cudaStream_t);
template int launch_conv<float, double, float>(const GridH &, const float *, const double *, float *, cudaStream_t);
template int launch_conv<float, float, double>(const GridH &, const float *, const float *, double *, cudaStream_t);
template int launch_conv<double, double, double>(const GridH &, const double *, const double *, double *, cudaStream_t);

}  // namespace mpi
