// Internal interface of the sampled-trace-kernel convolution C.
#pragma once

#include "fft.cuh"
#include "pair_ops.cuh"

namespace mpi {

// Scratch bytes for the sampled kernel of a grid (FP64 copy + rounded copy).
size_t conv_kernel_bytes(int nx, int ny, int elem_bytes);

// Samples kappa_G on all (2ny-1) x (2nx-1) voxel offsets into `scratch`
// (conv_kernel_bytes) and returns the kernel in type R through K_out.
// comp < 0: the trace kernel; comp = 2a + b: entry (a, b) of beta K G.
template <typename R>
int conv_prepare_kernel(const ModelH &m, const GridH &g, void *scratch, R **K_out, cudaStream_t st,
                        int comp = -1);

// out = C in  (in: IN [ny][nx], out: OUT [ny][nx], must not overlap).
template <typename R, typename IN, typename OUT>
int launch_conv(const GridH &g, const R *K, const IN *in, OUT *out, cudaStream_t st);

// The operator C of one grid, by the direct sum (small grids) or by FFT
// (N >= MPI_CONV_FFT_MIN_N, DFTs in the precision R); scratch: conv_plan_bytes.
template <typename R>
struct ConvPlan {
    using C2 = typename CxOf<R>::type;
    int nx = 0, ny = 0;
    bool fft = false;
    const R *K = nullptr;  // direct route: the sampled kernel
    int NX = 0, NY = 0;    // FFT route: circular grid
    FftPlan px, py;
    C2 *WX = nullptr, *WY = nullptr, *Kh = nullptr, *a = nullptr, *t = nullptr;
    // Three-launch form (conv_fft2.cu): Kh holds the kernel spectrum's
    // columns kx < LD row-major, [NY][LD]; a and t the half spectra.
    bool fused = false;
    int LD = 0;
};
bool conv_uses_fft(int nx, int ny, int elem_bytes);
size_t conv_plan_bytes(int nx, int ny, int elem_bytes);
template <typename R>
int conv_plan_prepare(const ModelH &m, const GridH &g, void *scratch, ConvPlan<R> &P, cudaStream_t st,
                      int comp = -1);
// Building blocks of the FFT routes (2-D here, 3-D in ffp3.cu):
// dst[c][r] = src[r][c] for a rows x cols complex matrix; t = conj(t kh).
int transpose_cx(int rows, int cols, const float2 *src, float2 *dst, cudaStream_t st);
int transpose_cx(int rows, int cols, const double2 *src, double2 *dst, cudaStream_t st);
int spec_mul_conj(int64_t n, float2 *t, const float2 *kh, cudaStream_t st);
int spec_mul_conj(int64_t n, double2 *t, const double2 *kh, cudaStream_t st);

// Three-launch FFT route (conv_fft2.cu): power-of-two circular grids with
// 4 <= NX <= 4096 and 4 <= NY <= 2048 (every transform in shared memory).
bool conv_fused_fits(int NX, int NY);
// Row length of the half spectra: NX/2 + 1 rounded up to whole column groups.
int conv_fused_ld(int NX, int elem_bytes);
// Rearranges the plan's transposed kernel spectrum Kh ([NX][NY]) into the
// [NY][LD] layout of the column launch, in place (tmp: NY x LD scratch).
template <typename C>
int conv_fused_kernel(int NX, int NY, int LD, C *Kh, C *tmp, cudaStream_t st);
template <typename R, typename IN, typename OUT>
int conv_apply_fused(const ConvPlan<R> &P, const IN *in, OUT *out, cudaStream_t st);

// Pieces of the shared-memory FFT routes (conv_fft2.cu), shared by the 2-D
// and 3-D convolutions.  Row launches: n_rows real rows of nx values (row r
// at in + r nx) <-> their half spectra (row r at X + r LD, LD entries, bins
// above NX/2 zero), NX = 2^k <= 4096; the inverse extends each half by
// Hermitian symmetry, crops to nx and scales.
template <typename C, typename IN>
int cf_rows_fwd(int nx, int n_rows, int NX, int LD, const IN *in, const C *W, C *X, cudaStream_t st);
template <typename C, typename OUT>
int cf_rows_inv(int nx, int n_rows, int NX, int LD, const C *Y, const C *W, double scale, OUT *out, cudaStream_t st);
// Column launch: for every outer index o < n_outer and every group of
// adjacent kx < LD, a DFT of length n (2^k <= 2048) over the elements
// e < n_in at in + o in_outer + e in_stride + kx (zero above), written for
// e < n_out at out + o out_outer + e out_stride + kx.  mode: kCfFwd (DFT),
// kCfFused (IDFT(DFT(x) K), K at Kh + o k_outer + e k_stride + kx), kCfInv
// (IDFT); inverses unscaled.
constexpr int kCfFwd = 0, kCfFused = 1, kCfInv = 2;
struct CfCols {
    int mode = kCfFwd;
    int n = 0, n_in = 0, n_out = 0, n_outer = 0, LD = 0;
    int64_t in_outer = 0, in_stride = 0, out_outer = 0, out_stride = 0, k_outer = 0, k_stride = 0;
};
template <typename C>
int cf_cols(const CfCols &c, const C *in, const C *Kh, const C *W, C *out, cudaStream_t st);

// out = C in.  The FFT route uses the plan's buffers: one application at a
// time per plan (calls on one stream are ordered).
template <typename R, typename IN, typename OUT>
int conv_apply(const ConvPlan<R> &P, const IN *in, OUT *out, cudaStream_t st);

}  // namespace mpi
