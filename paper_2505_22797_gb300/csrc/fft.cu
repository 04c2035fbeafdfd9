// Stockham autosort FFT in FP32 or FP64 (see fft.cuh).
#include <algorithm>

#include "fft.cuh"

namespace mpi {


bool plan_fft(int64_t n, FftPlan &p)
{
    p.n = n;
    p.radix.clear();
    int64_t m = n;
    while (m % 4 == 0) p.radix.push_back(4), m /= 4;
    if (m % 2 == 0) p.radix.push_back(2), m /= 2;
    for (int q = 3; q <= kMaxRadix && m > 1; q += 2)
        while (m % q == 0) p.radix.push_back(q), m /= q;
    return m == 1;
}

// W[m] = exp(-2 pi i m / n), m < n, formed in FP64 and rounded to C.
template <typename C>
__global__ void k_twiddles(int64_t n, C *__restrict__ W)
{
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * double(m) / double(n), &s, &c);
        W[m] = make_cx<C>(c, s);
    }
}

// One butterfly j (k = j mod Ns) of a Stockham pass of radix R after passes
// whose radices multiply to Ns: reads x[j + i n/R], i < R, and writes
//   y[(j/Ns) Ns R + k + q Ns] = sum_i x[j + i n/R] W^{i (k + q Ns) n/(Ns R)}.
template <typename C, typename I>
__device__ __forceinline__ void butterfly(const C *__restrict__ xc, C *__restrict__ yc, I n, int R, I Ns,
                                          const C *__restrict__ W, I j)
{
    const I nb = n / R;
    const I NsR = Ns * R;
    const I step = n / NsR;  // table stride for the NsR-th roots
    const I k = j % Ns;
    const I out0 = (j / Ns) * NsR + k;
    if (R == 2) {
        const C a = xc[j], b = cmul(xc[j + nb], W[k * step]);
        yc[out0] = cxv(a.x + b.x, a.y + b.y);
        yc[out0 + Ns] = cxv(a.x - b.x, a.y - b.y);
    } else if (R == 4) {
        const C a0 = xc[j];
        const C a1 = cmul(xc[j + nb], W[k * step]);
        const C a2 = cmul(xc[j + 2 * nb], W[2 * k * step]);
        const C a3 = cmul(xc[j + 3 * nb], W[3 * k * step]);
        const C s02 = cxv(a0.x + a2.x, a0.y + a2.y);
        const C d02 = cxv(a0.x - a2.x, a0.y - a2.y);
        const C s13 = cxv(a1.x + a3.x, a1.y + a3.y);
        const C d13 = cxv(a1.x - a3.x, a1.y - a3.y);
        // omega_4 = -i:  d13 * (-i) = (d13.y, -d13.x)
        yc[out0] = cxv(s02.x + s13.x, s02.y + s13.y);
        yc[out0 + Ns] = cxv(d02.x + d13.y, d02.y - d13.x);
        yc[out0 + 2 * Ns] = cxv(s02.x - s13.x, s02.y - s13.y);
        yc[out0 + 3 * Ns] = cxv(d02.x - d13.y, d02.y + d13.x);
    } else {
        for (int q = 0; q < R; ++q) {
            const I e = k + (I)q * Ns;  // exponent base over NsR, e < NsR
            C acc = {0, 0};
            I m = 0;                    // i e mod NsR, stepped
            for (int i = 0; i < R; ++i) {
                const C t = cmul(xc[j + i * nb], W[m * step]);
                acc.x += t.x;
                acc.y += t.y;
                m += e;
                if (m >= NsR) m -= NsR;
            }
            yc[out0 + q * Ns] = acc;
        }
    }
}

// The same butterfly for a power-of-two length with R = 2 or 4: the index
// arithmetic by shifts and masks (lg_n = log2 n, lg_ns = log2 Ns) instead of
// the divisions by runtime values above, which cost more instructions than
// the butterfly itself.  The same loads, twiddles and operations: the
// results are identical.
template <typename C>
__device__ __forceinline__ void butterfly_p2(const C *__restrict__ xc, C *__restrict__ yc, int lg_n, int R,
                                             int lg_ns, const C *__restrict__ W, int j)
{
    const int Ns = 1 << lg_ns;
    const int k = j & (Ns - 1);
    if (R == 4) {
        const int nb = 1 << (lg_n - 2);
        const int tw = k << (lg_n - lg_ns - 2);  // k n / (4 Ns)
        const int out0 = ((j >> lg_ns) << (lg_ns + 2)) + k;
        const C a0 = xc[j];
        const C a1 = cmul(xc[j + nb], W[tw]);
        const C a2 = cmul(xc[j + 2 * nb], W[2 * tw]);
        const C a3 = cmul(xc[j + 3 * nb], W[3 * tw]);
        const C s02 = cxv(a0.x + a2.x, a0.y + a2.y);
        const C d02 = cxv(a0.x - a2.x, a0.y - a2.y);
        const C s13 = cxv(a1.x + a3.x, a1.y + a3.y);
        const C d13 = cxv(a1.x - a3.x, a1.y - a3.y);
        yc[out0] = cxv(s02.x + s13.x, s02.y + s13.y);
        yc[out0 + Ns] = cxv(d02.x + d13.y, d02.y - d13.x);
        yc[out0 + 2 * Ns] = cxv(s02.x - s13.x, s02.y - s13.y);
        yc[out0 + 3 * Ns] = cxv(d02.x - d13.y, d02.y + d13.x);
    } else {
        const int nb = 1 << (lg_n - 1);
        const int tw = k << (lg_n - lg_ns - 1);  // k n / (2 Ns)
        const int out0 = ((j >> lg_ns) << (lg_ns + 1)) + k;
        const C a = xc[j], b = cmul(xc[j + nb], W[tw]);
        yc[out0] = cxv(a.x + b.x, a.y + b.y);
        yc[out0 + Ns] = cxv(a.x - b.x, a.y - b.y);
    }
}

// One Stockham pass over global memory; `dist` is the distance between
// channels (blockIdx.y).
template <typename C>
__global__ void __launch_bounds__(kFftThreads)
k_fft_pass(const C *__restrict__ x, C *__restrict__ y, int64_t n, int R, int64_t Ns,
           const C *__restrict__ W, int64_t dist)
{
    const C *xc = x + blockIdx.y * dist;
    C *yc = y + blockIdx.y * dist;
    const int64_t nb = n / R;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nb;
         j += (int64_t)gridDim.x * blockDim.x)
        butterfly<C, int64_t>(xc, yc, n, R, Ns, W, j);
}

// Every pass of a sequence in shared memory: one global read and one global
// write per 1-D transform instead of one per pass.  The first pass reads the
// sequence from global memory and the last one writes it back (a single-pass
// transform is staged through shared memory, since reading and writing the
// same global row in one pass would race); the passes between run from one
// shared buffer to the other.  A block holds `rpb` sequences of `tpr` threads
// each, so short sequences (few butterflies per pass) still keep the block's
// threads busy.
constexpr int kSmemFftMaxPasses = 24;
struct RadixList {
    int n_pass;
    int lg_n;  // log2 n when every radix is 2 or 4 (shift arithmetic), else -1
    int r[kSmemFftMaxPasses];
};

template <typename C>
__global__ void __launch_bounds__(kFftThreads)
k_fft_smem(C *__restrict__ x, int n, RadixList rl, const C *__restrict__ W, int64_t dist, int n_seq, int rpb)
{
    extern __shared__ __align__(16) unsigned char fft_smem[];
    const int tpr = blockDim.x / rpb;
    const int row = threadIdx.x / tpr, tid = threadIdx.x % tpr;
    const int seq = blockIdx.x * rpb + row;
    const bool active = row < rpb && seq < n_seq;
    C *A = reinterpret_cast<C *>(fft_smem) + (size_t)2 * n * min(row, rpb - 1);
    C *B = A + n;
    C *xc = x + (int64_t)min(seq, n_seq - 1) * dist;
    const int last = rl.n_pass - 1;
    if (last == 0) {  // one pass: stage through shared memory
        if (active)
            for (int e = tid; e < n; e += tpr) A[e] = xc[e];
        __syncthreads();
        if (active)
            for (int j = tid; j < n / rl.r[0]; j += tpr) butterfly<C, int>(A, xc, n, rl.r[0], 1, W, j);
        return;
    }
    const C *src = xc;
    C *dst = A;
    if (rl.lg_n >= 0) {
        int lg_ns = 0;
        for (int p = 0; p <= last; ++p) {
            const int R = rl.r[p];
            C *out = (p == last) ? xc : dst;
            if (active)
                for (int j = tid; j < (n >> (R == 4 ? 2 : 1)); j += tpr)
                    butterfly_p2<C>(src, out, rl.lg_n, R, lg_ns, W, j);
            __syncthreads();
            src = dst;
            dst = (dst == A) ? B : A;
            lg_ns += R == 4 ? 2 : 1;
        }
        return;
    }
    int Ns = 1;
    for (int p = 0; p <= last; ++p) {
        const int R = rl.r[p];
        C *out = (p == last) ? xc : dst;
        if (active)
            for (int j = tid; j < n / R; j += tpr) butterfly<C, int>(src, out, n, R, Ns, W, j);
        __syncthreads();
        src = dst;
        dst = (dst == A) ? B : A;
        Ns *= R;
    }
}

unsigned fft_blocks(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kFftThreads - 1) / kFftThreads, 4096)); }

// In-place in the sense of buffers: the transform of `a` ends in `a` (b is
// scratch of the same size).  n_ch channels at distance `dist`.  Sequences
// of up to 64 KB per two copies run in shared memory, longer ones pass by
// pass through global memory; both apply the same butterflies.
template <typename C>
static int fft_run_t(const FftPlan &p, C *a, C *b, int n_ch, int64_t dist, const C *W, cudaStream_t st)
{
    if (p.radix.empty()) return MPI_OK;
    const size_t smem = 2 * sizeof(C) * size_t(p.n);
    if (smem <= 64 * 1024 && (int)p.radix.size() <= kSmemFftMaxPasses) {
        RadixList rl{};
        rl.n_pass = (int)p.radix.size();
        int most = 1;  // the most butterflies of any pass
        bool p2 = true;
        for (int q = 0; q < rl.n_pass; ++q) {
            rl.r[q] = p.radix[q];
            most = std::max(most, (int)(p.n / p.radix[q]));
            p2 = p2 && (p.radix[q] == 2 || p.radix[q] == 4);
        }
        int lg = 0;
        while ((int64_t(1) << lg) < p.n) ++lg;
        rl.lg_n = p2 ? lg : -1;
        // sequences per block: as many as leave every thread a butterfly in
        // the widest pass, within the block's shared memory -- and more (a
        // thread then takes several butterflies per pass) while the blocks
        // would not all be resident at once: a 1024 x 1024 transform's 1024
        // one-row blocks exceeded the ~6 resident per SM by 112, which ran
        // alone as a second wave for a third of the launch.
        const int wave = device_sm_count() * 6;
        int rpb = 1;
        while (size_t(rpb) * 2 * smem <= 48 * 1024 && rpb * 2 <= n_ch && rpb * 2 <= kFftThreads / 32 &&
               (rpb * 2 * most <= kFftThreads || (n_ch + rpb - 1) / rpb > wave))
            rpb *= 2;
        const size_t smem_blk = smem * size_t(rpb);
        if (smem_blk > 48 * 1024)  // opt in above the default limit (set on the current device)
            MPI_TRY_CUDA(cudaFuncSetAttribute(k_fft_smem<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_blk));
        const unsigned blocks = (unsigned)((n_ch + rpb - 1) / rpb);
        k_fft_smem<C><<<blocks, kFftThreads, smem_blk, st>>>(a, (int)p.n, rl, W, dist, n_ch, rpb);
        MPI_CHECK_LAUNCH();
        return MPI_OK;
    }
    C *src = a, *dst = b;
    int64_t Ns = 1;
    for (int R : p.radix) {
        dim3 grid(fft_blocks(p.n / R), n_ch);
        k_fft_pass<C><<<grid, kFftThreads, 0, st>>>(src, dst, p.n, R, Ns, W, dist);
        MPI_CHECK_LAUNCH();
        Ns *= R;
        std::swap(src, dst);
    }
    if (src != a) MPI_TRY_CUDA(cudaMemcpyAsync(a, src, sizeof(C) * (n_ch * dist), cudaMemcpyDeviceToDevice, st));
    return MPI_OK;
}

template <typename C>
static int fft_twiddles_t(int64_t n, C *W, cudaStream_t st)
{
    k_twiddles<C><<<fft_blocks(n), kFftThreads, 0, st>>>(n, W);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

int fft_run(const FftPlan &p, double2 *a, double2 *b, int n_ch, int64_t dist, const double2 *W, cudaStream_t st)
{
    return fft_run_t(p, a, b, n_ch, dist, W, st);
}
int fft_run(const FftPlan &p, float2 *a, float2 *b, int n_ch, int64_t dist, const float2 *W, cudaStream_t st)
{
    return fft_run_t(p, a, b, n_ch, dist, W, st);
}
int fft_twiddles(int64_t n, double2 *W, cudaStream_t st) { return fft_twiddles_t(n, W, st); }
int fft_twiddles(int64_t n, float2 *W, cudaStream_t st) { return fft_twiddles_t(n, W, st); }

}  // namespace mpi
