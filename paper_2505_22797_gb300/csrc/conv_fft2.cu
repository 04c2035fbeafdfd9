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
constexpr int kCfPre = 4;           // kernel-spectrum elements per thread held in registers

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

// Column pass (launch 2 in 2-D; the y and z passes in 3-D): a block takes
// 2^LG_CB adjacent kx (one 32-byte sector per element) of one outer index o
// (blockIdx.x = group + n_groups o) and transforms along a column of n = 2^lg_n
// elements at distance `stride`:
//   in  element e < n_in at in  + o in_outer  + e in_stride  + kx (zero for e >= n_in),
//   out element e < n_out at out + o out_outer + e out_stride + kx,
// MODE kCfFwd:   out = DFT(in);
// MODE kCfFused: out = IDFT(DFT(in) K) (unscaled), K element e at Kh + o k_outer + e k_stride + kx;
// MODE kCfInv:   out = IDFT(in) (unscaled), by IDFT(V) = conj(DFT(conj V)).
struct CfColArgs {
    int lg_n, n_in, n_out, n_groups;
    int64_t in_outer, in_stride, out_outer, out_stride, k_outer, k_stride;
};

template <typename C, int LG_CB, int MODE>
__global__ void __launch_bounds__(kCfMaxThreads)
k_cf_cols(CfColArgs d, const C *__restrict__ in, const C *__restrict__ Kh, const C *__restrict__ W,
          C *__restrict__ out)
{
    using R = decltype(C{}.x);
    constexpr int CB = 1 << LG_CB;
    extern __shared__ __align__(16) unsigned char cf_smem[];
    const int n = 1 << d.lg_n;
    C *A = reinterpret_cast<C *>(cf_smem);
    C *B = A + (n << LG_CB);
    const int o = blockIdx.x / d.n_groups;
    const int kx0 = (blockIdx.x - o * d.n_groups) * CB;
    const C *src = in + o * d.in_outer + kx0;
    const int tot = n << LG_CB;
    // the kernel spectrum's first kCfPre elements of each thread, loaded
    // before the forward DFT so that their latency overlaps it
    const C *kc = Kh + o * d.k_outer + kx0;
    constexpr int PRE = sizeof(C) == 8 ? kCfPre : kCfPre / 2;  // FP64: within the 1024-thread register budget
    C kv[MODE == kCfFused ? PRE : 1];
    if constexpr (MODE == kCfFused) {
#pragma unroll
        for (int u = 0; u < PRE; ++u) {
            const int q = threadIdx.x + u * blockDim.x;
            if (q < tot) kv[u] = kc[(q >> LG_CB) * d.k_stride + (q & (CB - 1))];
        }
    }
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        const int c = q & (CB - 1), e = q >> LG_CB;
        C v = cxv(R(0), R(0));
        if (e < d.n_in) v = src[e * d.in_stride + c];
        if (MODE == kCfInv) v.y = -v.y;
        A[q] = v;
    }
    __syncthreads();
    C *F = smem_dft(A, B, d.lg_n, LG_CB, W);
    if constexpr (MODE == kCfFused) {
        // conj(F K), so that a second forward DFT gives the conjugated inverse
        C *G = F == A ? B : A;
#pragma unroll
        for (int u = 0; u < PRE; ++u) {
            const int q = threadIdx.x + u * blockDim.x;
            if (q < tot) {
                const C p = cmul(F[q], kv[u]);
                F[q] = cxv(p.x, -p.y);
            }
        }
        for (int q = threadIdx.x + PRE * blockDim.x; q < tot; q += blockDim.x) {
            const C p = cmul(F[q], kc[(q >> LG_CB) * d.k_stride + (q & (CB - 1))]);
            F[q] = cxv(p.x, -p.y);
        }
        __syncthreads();
        F = smem_dft(F, G, d.lg_n, LG_CB, W);
    }
    C *dst = out + o * d.out_outer + kx0;
    for (int q = threadIdx.x; q < (d.n_out << LG_CB); q += blockDim.x) {
        const int c = q & (CB - 1), e = q >> LG_CB;
        const C h = F[q];
        dst[e * d.out_stride + c] = MODE == kCfFwd ? h : cxv(h.x, -h.y);
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

template <typename C, typename IN>
int cf_rows_fwd(int nx, int n_rows, int NX, int LD, const IN *in, const C *W, C *X1, cudaStream_t st)
{
    if (n_rows <= 0) return MPI_OK;
    const int lg_nx = ilog2(NX), lg_rp = rows_lg_rp(NX);
    const unsigned blocks = (unsigned)(((n_rows + 1) / 2 + (1 << lg_rp) - 1) >> lg_rp);
    const size_t smem = 2 * sizeof(C) * (size_t(NX) << lg_rp);
    MPI_TRY(allow_smem(k_cf_rows_fwd<C, IN>, smem));
    k_cf_rows_fwd<C, IN><<<blocks, block_threads(lg_nx, lg_rp), smem, st>>>(nx, n_rows, lg_nx, lg_rp, LD, in, W, X1);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename C, typename OUT>
int cf_rows_inv(int nx, int n_rows, int NX, int LD, const C *Y, const C *W, double scale, OUT *out, cudaStream_t st)
{
    if (n_rows <= 0) return MPI_OK;
    const int lg_nx = ilog2(NX), lg_rp = rows_lg_rp(NX);
    const unsigned blocks = (unsigned)(((n_rows + 1) / 2 + (1 << lg_rp) - 1) >> lg_rp);
    const size_t smem = 2 * sizeof(C) * (size_t(NX) << lg_rp);
    MPI_TRY(allow_smem(k_cf_rows_inv<C, OUT>, smem));
    k_cf_rows_inv<C, OUT><<<blocks, block_threads(lg_nx, lg_rp), smem, st>>>(nx, n_rows, lg_nx, lg_rp, LD, Y, W, scale,
                                                                             out);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename C>
int cf_cols(const CfCols &c, const C *in, const C *Kh, const C *W, C *out, cudaStream_t st)
{
    constexpr int LG_CB = cols_lg_cb<C>();
    if (c.n_outer <= 0 || c.n_out <= 0) return MPI_OK;
    CfColArgs d{};
    d.lg_n = ilog2(c.n);
    d.n_in = c.n_in;
    d.n_out = c.n_out;
    d.n_groups = c.LD >> LG_CB;
    d.in_outer = c.in_outer;
    d.in_stride = c.in_stride;
    d.out_outer = c.out_outer;
    d.out_stride = c.out_stride;
    d.k_outer = c.k_outer;
    d.k_stride = c.k_stride;
    const unsigned blocks = (unsigned)(int64_t(d.n_groups) * c.n_outer);
    const size_t smem = 2 * sizeof(C) * (size_t(c.n) << LG_CB);
    const unsigned threads = block_threads(d.lg_n, LG_CB);
    switch (c.mode) {
        case kCfFwd:
            MPI_TRY(allow_smem(k_cf_cols<C, LG_CB, kCfFwd>, smem));
            k_cf_cols<C, LG_CB, kCfFwd><<<blocks, threads, smem, st>>>(d, in, Kh, W, out);
            break;
        case kCfFused:
            MPI_TRY(allow_smem(k_cf_cols<C, LG_CB, kCfFused>, smem));
            k_cf_cols<C, LG_CB, kCfFused><<<blocks, threads, smem, st>>>(d, in, Kh, W, out);
            break;
        default:
            MPI_TRY(allow_smem(k_cf_cols<C, LG_CB, kCfInv>, smem));
            k_cf_cols<C, LG_CB, kCfInv><<<blocks, threads, smem, st>>>(d, in, Kh, W, out);
            break;
    }
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

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
    MPI_TRY((cf_rows_fwd<C, IN>(P.nx, P.ny, P.NX, P.LD, in, P.WX, P.a, st)));
    CfCols c{};
    c.mode = kCfFused;
    c.n = P.NY;
    c.n_in = c.n_out = P.ny;
    c.n_outer = 1;
    c.LD = P.LD;
    c.in_stride = c.out_stride = c.k_stride = P.LD;
    MPI_TRY(cf_cols<C>(c, P.a, P.Kh, P.WY, P.t, st));
    return cf_rows_inv<C, OUT>(P.nx, P.ny, P.NX, P.LD, P.t, P.WX, 1.0 / (double(P.NX) * double(P.NY)), out, st);
}

template int cf_rows_fwd<float2, float>(int, int, int, int, const float *, const float2 *, float2 *, cudaStream_t);
template int cf_rows_fwd<float2, double>(int, int, int, int, const double *, const float2 *, float2 *, cudaStream_t);
template int cf_rows_fwd<double2, double>(int, int, int, int, const double *, const double2 *, double2 *,
                                          cudaStream_t);
template int cf_rows_inv<float2, float>(int, int, int, int, const float2 *, const float2 *, double, float *,
                                        cudaStream_t);
template int cf_rows_inv<float2, double>(int, int, int, int, const float2 *, const float2 *, double, double *,
                                         cudaStream_t);
template int cf_rows_inv<double2, double>(int, int, int, int, const double2 *, const double2 *, double, double *,
                                          cudaStream_t);
template int cf_cols<float2>(const CfCols &, const float2 *, const float2 *, const float2 *, float2 *, cudaStream_t);
template int cf_cols<double2>(const CfCols &, const double2 *, const double2 *, const double2 *, double2 *,
                              cudaStream_t);
template int conv_fused_kernel<float2>(int, int, int, float2 *, float2 *, cudaStream_t);
template int conv_fused_kernel<double2>(int, int, int, double2 *, double2 *, cudaStream_t);
template int conv_apply_fused<float, float, float>(const ConvPlan<float> &, const float *, float *, cudaStream_t);
template int conv_apply_fused<float, double, float>(const ConvPlan<float> &, const double *, float *, cudaStream_t);
template int conv_apply_fused<float, float, double>(const ConvPlan<float> &, const float *, double *, cudaStream_t);
template int conv_apply_fused<double, double, double>(const ConvPlan<double> &, const double *, double *, cudaStream_t);

}  // namespace mpi
