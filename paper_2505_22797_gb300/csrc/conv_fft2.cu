// Two-dimensional FFT route of the convolution C (Eq. convolution:trace,
// Eq. kernel:trace; C_h of Eq. dec:sub:tik) in three launches that use what
// the operator's structure gives:
//  * the input is real and zero outside its ny x nx window of the NY x NX
//    circular grid, and only that window of the output is kept;
//  * the kernel's spectrum belongs to a real kernel that is even under
//    y -> -y, so the product spectrum is Hermitian and one half of its
//    columns (kx = 0 .. NX/2) determines the output.
// Launches (FP32 or FP64, DFTs in the call's precision):
//  1. rows:    pairs of real input rows as one complex sequence z = a + i b;
//              its DFT Z gives both rows' spectra, A = (Z[k] + conj Z[-k])/2,
//              B = (Z[k] - conj Z[-k])/(2i), kept for k = 0 .. NX/2 (the
//              NY - ny zero rows are not transformed);
//  2. columns: per group of adjacent kx (one 32-byte sector per row), the DFT
//              along y of the ny non-zero rows, the product with the kernel's
//              spectrum, the inverse DFT (IDFT(V) = conj(DFT(conj V))) and
//              only the ny kept rows written back;
//  3. rows:    pairs of half spectra extended by Hermitian symmetry, packed as
//              Z = A + i B; IDFT(Z) = a + i b gives both real output rows,
//              cropped to nx and scaled by 1/(NX NY).
// Every transform runs all its radix passes in shared memory (the sequences
// of a block interleaved, element e of sequence c at [e * ncols + c]), so each
// launch reads and writes global memory once.  The same sum as the nine-pass
// route (full complex grid, two transposes) up to round-off: the parts the
// three launches skip are zeros or conjugates.
#include "conv_ops.cuh"

namespace mpi {

namespace {

// Threads of a block: one radix-4 butterfly each per pass (the block's
// sequences times n/4), between kCfMinThreads and kCfMaxThreads.
constexpr int kCfMinThreads = 64;
constexpr int kCfMaxThreads = 1024;
constexpr int kCfRowThreads = 256;  // a row launch's sequences per block fill this many

// Forward DFT of 2^lg_c sequences of length n = 2^lg_n held interleaved in
// shared memory, A -> B -> A ...: Stockham passes of radix 4 (one radix-2
// pass last when lg_n is odd), twiddles W[m] = exp(-2 pi i m / n).  Returns
// the buffer holding the result.  Every thread of the block calls it.
template <typename C>
__device__ C *smem_dft(C *A, C *B, int lg_n, int lg_c, const C *__restrict__ W)
{
    const int n = 1 << lg_n;
    const int cmask = (1 << lg_c) - 1;
    C *src = A, *dst = B;
    int lg_ns = 0;
    while (lg_ns < lg_n) {
        const bool r4 = lg_n - lg_ns >= 2;
        const int Ns = 1 << lg_ns;
        if (r4) {
            const int nb = n >> 2;
            for (int b = threadIdx.x; b < (nb << lg_c); b += blockDim.x) {
                const int c = b & cmask, j = b >> lg_c;
                const int k = j & (Ns - 1);
                const int tw = k << (lg_n - lg_ns - 2);  // k n / (4 Ns)
                const int out0 = ((j >> lg_ns) << (lg_ns + 2)) + k;
                const C a0 = src[(j << lg_c) + c];
                const C a1 = cmul(src[((j + nb) << lg_c) + c], W[tw]);
                const C a2 = cmul(src[((j + 2 * nb) << lg_c) + c], W[2 * tw]);
                const C a3 = cmul(src[((j + 3 * nb) << lg_c) + c], W[3 * tw]);
                const C s02 = cxv(a0.x + a2.x, a0.y + a2.y);
                const C d02 = cxv(a0.x - a2.x, a0.y - a2.y);
                const C s13 = cxv(a1.x + a3.x, a1.y + a3.y);
                const C d13 = cxv(a1.x - a3.x, a1.y - a3.y);
                // omega_4 = -i: d13 (-i) = (d13.y, -d13.x)
                dst[(out0 << lg_c) + c] = cxv(s02.x + s13.x, s02.y + s13.y);
                dst[((out0 + Ns) << lg_c) + c] = cxv(d02.x + d13.y, d02.y - d13.x);
                dst[((out0 + 2 * Ns) << lg_c) + c] = cxv(s02.x - s13.x, s02.y - s13.y);
                dst[((out0 + 3 * Ns) << lg_c) + c] = cxv(d02.x - d13.y, d02.y + d13.x);
            }
        } else {
            const int nb = n >> 1;
            for (int b = threadIdx.x; b < (nb << lg_c); b += blockDim.x) {
                const int c = b & cmask, j = b >> lg_c;
                const int k = j & (Ns - 1);
                const int tw = k << (lg_n - lg_ns - 1);  // k n / (2 Ns)
                const int out0 = ((j >> lg_ns) << (lg_ns + 1)) + k;
                const C a = src[(j << lg_c) + c];
                const C b2 = cmul(src[((j + nb) << lg_c) + c], W[tw]);
                dst[(out0 << lg_c) + c] = cxv(a.x + b2.x, a.y + b2.y);
                dst[((out0 + Ns) << lg_c) + c] = cxv(a.x - b2.x, a.y - b2.y);
            }
        }
        __syncthreads();
        C *t = src;
        src = dst;
        dst = t;
        lg_ns += r4 ? 2 : 1;
    }
    return src;
}

// Launch 1: the half spectra X1[j][k], k < LD (k > NX/2: zero), of the input
// rows j < ny.  A block takes 2^lg_rp row pairs.
template <typename C, typename IN>
__global__ void __launch_bounds__(kCfMaxThreads)
k_cf_rows_fwd(int nx, int ny, int lg_nx, int lg_rp, int LD, const IN *__restrict__ in,
              const C *__restrict__ W, C *__restrict__ X1)
{
    using R = decltype(C{}.x);
    extern __shared__ __align__(16) unsigned char cf_smem[];
    const int NX = 1 << lg_nx, rp = 1 << lg_rp;
    C *A = reinterpret_cast<C *>(cf_smem);
    C *B = A + (NX << lg_rp);
    const int pair0 = blockIdx.x * rp;
    for (int q = threadIdx.x; q < (NX << lg_rp); q += blockDim.x) {
        const int s = q >> lg_nx, e = q & (NX - 1);
        const int ja = 2 * (pair0 + s), jb = ja + 1;
        R xa = R(0), xb = R(0);
        if (e < nx) {
            if (ja < ny) xa = R(in[(int64_t)ja * nx + e]);
            if (jb < ny) xb = R(in[(int64_t)jb * nx + e]);
        }
        A[(e << lg_rp) + s] = cxv(xa, xb);
    }
    __syncthreads();
    const C *Z = smem_dft(A, B, lg_nx, lg_rp, W);
    const int half = NX >> 1;
    for (int q = threadIdx.x; q < LD * rp; q += blockDim.x) {
        const int s = q / LD, k = q - s * LD;
        const int ja = 2 * (pair0 + s), jb = ja + 1;
        if (ja >= ny) continue;
        C a = cxv(R(0), R(0)), b = cxv(R(0), R(0));
        if (k <= half) {
            const C zk = Z[(k << lg_rp) + s];
            const C zm = Z[(((NX - k) & (NX - 1)) << lg_rp) + s];  // Z[-k]
            a = cxv(R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y));
            b = cxv(R(0.5) * (zk.y + zm.y), R(0.5) * (zm.x - zk.x));
        }
        X1[(int64_t)ja * LD + k] = a;
        if (jb < ny) X1[(int64_t)jb * LD + k] = b;
    }
}

// Launch 2: per group of 2^LG_CB adjacent kx, the column DFTs of the half
// spectra (rows j >= ny are zero), the product with the kernel's spectrum
// Kh2[ky][kx], and the inverse column DFTs kept for j < ny (unscaled):
//   Y2[j][kx] = sum_ky Kh2[ky][kx] sum_j' X1[j'][kx] W^(j' ky) W^(-j ky).
template <typename C, int LG_CB>
__global__ void __launch_bounds__(kCfMaxThreads)
k_cf_cols(int ny, int lg_ny, int LD, const C *__restrict__ X1, const C *__restrict__ Kh2,
          const C *__restrict__ W, C *__restrict__ Y2)
{
    using R = decltype(C{}.x);
    constexpr int CB = 1 << LG_CB;
    extern __shared__ __align__(16) unsigned char cf_smem[];
    const int NY = 1 << lg_ny;
    C *A = reinterpret_cast<C *>(cf_smem);
    C *B = A + (NY << LG_CB);
    const int kx0 = blockIdx.x * CB;
    for (int q = threadIdx.x; q < (NY << LG_CB); q += blockDim.x) {
        const int c = q & (CB - 1), j = q >> LG_CB;
        A[q] = j < ny ? X1[(int64_t)j * LD + kx0 + c] : cxv(R(0), R(0));
    }
    __syncthreads();
    C *F = smem_dft(A, B, lg_ny, LG_CB, W);
    C *G = F == A ? B : A;
    // conj(F Kh2), so that a second forward DFT gives the conjugated inverse
    for (int q = threadIdx.x; q < (NY << LG_CB); q += blockDim.x) {
        const int c = q & (CB - 1), ky = q >> LG_CB;
        const C p = cmul(F[q], Kh2[(int64_t)ky * LD + kx0 + c]);
        F[q] = cxv(p.x, -p.y);
    }
    __syncthreads();
    const C *H = smem_dft(F, G, lg_ny, LG_CB, W);
    for (int q = threadIdx.x; q < (ny << LG_CB); q += blockDim.x) {
        const int c = q & (CB - 1), j = q >> LG_CB;
        const C h = H[q];
        Y2[(int64_t)j * LD + kx0 + c] = cxv(h.x, -h.y);
    }
}

// Entry k of a row's full spectrum from its half (k = 0 .. half kept): the
// Hermitian extension, with the two self-conjugate bins taken real.
template <typename C>
__device__ __forceinline__ C herm_at(const C *__restrict__ row, int k, int half)
{
    using R = decltype(C{}.x);
    if (k == 0 || k == half) return cxv(row[k].x, R(0));
    if (k < half) return row[k];
    const C v = row[2 * half - k];
    return cxv(v.x, -v.y);
}

// Launch 3: pairs of rows j < ny of the product's inverse column transforms,
// Z = A + i B over the full length NX, IDFT(Z) = conj(DFT(conj Z)) = a + i b;
// out[j][i] = scale a[i] (row 2p) and scale b[i] (row 2p + 1), i < nx.
template <typename C, typename OUT>
__global__ void __launch_bounds__(kCfMaxThreads)
k_cf_rows_inv(int nx, int ny, int lg_nx, int lg_rp, int LD, const C *__restrict__ Y2,
              const C *__restrict__ W, double scale, OUT *__restrict__ out)
{
    using R = decltype(C{}.x);
    extern __shared__ __align__(16) unsigned char cf_smem[];
    const int NX = 1 << lg_nx, rp = 1 << lg_rp, half = NX >> 1;
    C *A = reinterpret_cast<C *>(cf_smem);
    C *B = A + (NX << lg_rp);
    const int pair0 = blockIdx.x * rp;
    for (int q = threadIdx.x; q < (NX << lg_rp); q += blockDim.x) {
        const int s = q >> lg_nx, k = q & (NX - 1);
        const int ja = 2 * (pair0 + s), jb = ja + 1;
        const C a = ja < ny ? herm_at(Y2 + (int64_t)ja * LD, k, half) : cxv(R(0), R(0));
        const C b = jb < ny ? herm_at(Y2 + (int64_t)jb * LD, k, half) : cxv(R(0), R(0));
        A[(k << lg_rp) + s] = cxv(a.x - b.y, -(a.y + b.x));  // conj(a + i b)
    }
    __syncthreads();
    const C *V = smem_dft(A, B, lg_nx, lg_rp, W);
    const R sc = R(scale);
    for (int q = threadIdx.x; q < nx * rp; q += blockDim.x) {
        const int s = q / nx, i = q - s * nx;
        const int ja = 2 * (pair0 + s), jb = ja + 1;
        if (ja >= ny) continue;
        const C v = V[(i << lg_rp) + s];
        out[(int64_t)ja * nx + i] = OUT(v.x * sc);
        if (jb < ny) out[(int64_t)jb * nx + i] = OUT(-v.y * sc);
    }
}

// Kh2[ky][kx] = Kh[kx][ky], kx < LD: the columns of the (transposed) kernel
// spectrum that the column launch reads, row-major.
template <typename C>
__global__ void k_cf_kh_half(int NY, int LD, const C *__restrict__ Kh, C *__restrict__ Kh2)
{
    const int64_t n = (int64_t)NY * LD;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int ky = (int)(e / LD), kx = (int)(e - (int64_t)ky * LD);
        Kh2[e] = Kh[(int64_t)kx * NY + ky];
    }
}

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Row pairs per block: enough for kCfRowThreads butterflies per pass.
int rows_lg_rp(int NX)
{
    int l = 0;
    while (((NX >> 2) << l) < kCfRowThreads) ++l;
    return l;
}

unsigned block_threads(int lg_n, int lg_c)
{
    return (unsigned)std::min(kCfMaxThreads, std::max(kCfMinThreads, (1 << (lg_n - 2)) << lg_c));
}

template <typename C>
constexpr int cols_lg_cb() { return sizeof(C) == 8 ? 2 : 1; }  // one 32-byte sector per row

template <typename K>
int allow_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024)
        MPI_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return MPI_OK;
}

}  // namespace

bool conv_fused_fits(int NX, int NY) { return NX >= 4 && NY >= 4 && NX <= 4096 && NY <= 2048; }

int conv_fused_ld(int NX, int elem_bytes)
{
    const int cb = elem_bytes == 8 ? 2 : 4;
    return (NX / 2 + 1 + cb - 1) / cb * cb;
}

template <typename C>
int conv_fused_kernel(int NX, int NY, int LD, C *Kh, C *tmp, cudaStream_t st)
{
    const int64_t n = (int64_t)NY * LD;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192));
    k_cf_kh_half<C><<<blocks, 256, 0, st>>>(NY, LD, Kh, tmp);
    MPI_CHECK_LAUNCH();
    MPI_TRY_CUDA(cudaMemcpyAsync(Kh, tmp, sizeof(C) * size_t(n), cudaMemcpyDeviceToDevice, st));
    (void)NX;
    return MPI_OK;
}

template <typename R, typename IN, typename OUT>
int conv_apply_fused(const ConvPlan<R> &P, const IN *in, OUT *out, cudaStream_t st)
{
    using C = typename ConvPlan<R>::C2;
    const int lg_nx = ilog2(P.NX), lg_ny = ilog2(P.NY);
    const int lg_rp = rows_lg_rp(P.NX);
    const int pairs = (P.ny + 1) / 2;
    const unsigned rblocks = (unsigned)((pairs + (1 << lg_rp) - 1) >> lg_rp);
    const size_t rsmem = 2 * sizeof(C) * (size_t(P.NX) << lg_rp);
    constexpr int LG_CB = cols_lg_cb<C>();
    const size_t csmem = 2 * sizeof(C) * (size_t(P.NY) << LG_CB);
    MPI_TRY(allow_smem(k_cf_rows_fwd<C, IN>, rsmem));
    MPI_TRY(allow_smem(k_cf_cols<C, LG_CB>, csmem));
    MPI_TRY(allow_smem(k_cf_rows_inv<C, OUT>, rsmem));
    const unsigned rthreads = block_threads(lg_nx, lg_rp), cthreads = block_threads(lg_ny, LG_CB);
    k_cf_rows_fwd<C, IN><<<rblocks, rthreads, rsmem, st>>>(P.nx, P.ny, lg_nx, lg_rp, P.LD, in, P.WX, P.a);
    MPI_CHECK_LAUNCH();
    k_cf_cols<C, LG_CB><<<(unsigned)(P.LD >> LG_CB), cthreads, csmem, st>>>(P.ny, lg_ny, P.LD, P.a, P.Kh, P.WY, P.t);
    MPI_CHECK_LAUNCH();
    k_cf_rows_inv<C, OUT><<<rblocks, rthreads, rsmem, st>>>(P.nx, P.ny, lg_nx, lg_rp, P.LD, P.t, P.WX,
                                                            1.0 / (double(P.NX) * double(P.NY)), out);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template int conv_fused_kernel<float2>(int, int, int, float2 *, float2 *, cudaStream_t);
template int conv_fused_kernel<double2>(int, int, int, double2 *, double2 *, cudaStream_t);
template int conv_apply_fused<float, float, float>(const ConvPlan<float> &, const float *, float *, cudaStream_t);
template int conv_apply_fused<float, double, float>(const ConvPlan<float> &, const double *, float *, cudaStream_t);
template int conv_apply_fused<float, float, double>(const ConvPlan<float> &, const float *, double *, cudaStream_t);
template int conv_apply_fused<double, double, double>(const ConvPlan<double> &, const double *, double *, cudaStream_t);

}  // namespace mpi
