// Transfer-function correction (Eq. core:formula:conva -> Eq. core:formula;
// the preprocessing of Sec. 3.2).  The measured signal is the model signal
// convolved in time with the receive chain's impulse response; over one
// period of T samples that is a circular convolution, so the correction is
//   s_out[k] = IDFT_T( M_k(f) DFT_T(s_raw[k])(f) / a_hat_k(f) ),
// M_k(f) = 1 where snr_k(f) >= theta_k and a_hat_k(f) != 0, else 0, on the
// T/2 + 1 non-negative bins (the negative ones mirror them: the output is
// real).
//
// The DFTs run in FP64 on the device (they are a negligible share of a
// reconstruction, and the division by a_hat amplifies round-off where
// |a_hat| is small): the Stockham FFT of fft.cu, and Bluestein's chirp-z
// algorithm (Bluestein 1970: a length-T DFT as a convolution with the chirp
// exp(-i pi m^2 / T), evaluated with power-of-two FFTs) for lengths with a
// larger prime factor.  Channels run as the y dimension of every launch.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fft.cuh"

namespace mpi {

int check_dtype(mpi_dtype d);

// ---------------------------------------------------------------------------
// Bluestein: X_k = c_k sum_m (x_m c_m) conj(c_{k-m}),  c_m = exp(-i pi m^2 / n).

__global__ void k_chirp(int64_t n, double2 *__restrict__ c)
{
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = (m * m) % (2 * n);  // exp(-i pi e / n) is 2n-periodic in e
        double s, co;
        sincospi(-double(e) / double(n), &s, &co);
        c[m] = make_double2(co, s);
    }
}

// b[m] = conj(c_m) for m < n and b[M - m] = conj(c_m) for 0 < m < n, else 0.
__global__ void k_bluestein_b(int64_t n, int64_t M, const double2 *__restrict__ c, double2 *__restrict__ b)
{
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (m < n) v = make_double2(c[m].x, -c[m].y);
        else if (M - m < n) v = make_double2(c[M - m].x, -c[M - m].y);
        b[m] = v;
    }
}

// a[ch][m] = x[ch][m] c_m (m < n), 0 up to M.
__global__ void k_bluestein_a(int64_t n, int64_t M, const double2 *__restrict__ x, int64_t xdist,
                              const double2 *__restrict__ c, double2 *__restrict__ a)
{
    const double2 *xc = x + blockIdx.y * xdist;
    double2 *ac = a + blockIdx.y * M;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x)
        ac[m] = m < n ? cmul(xc[m], c[m]) : make_double2(0.0, 0.0);
}

// a = conj(a * B)  (so that a following forward FFT gives M conj(IFFT(a B))).
__global__ void k_mul_conj(int64_t M, double2 *__restrict__ a, const double2 *__restrict__ B)
{
    double2 *ac = a + blockIdx.y * M;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M;
         m += (int64_t)gridDim.x * blockDim.x) {
        const double2 p = cmul(ac[m], B[m]);
        ac[m] = make_double2(p.x, -p.y);
    }
}

// X[ch][k] = c_k conj(a[ch][k]) / M, k < n.
__global__ void k_bluestein_out(int64_t n, int64_t M, const double2 *__restrict__ a,
                                const double2 *__restrict__ c, double2 *__restrict__ X, int64_t xdist)
{
    const double2 *ac = a + blockIdx.y * M;
    double2 *Xc = X + blockIdx.y * xdist;
    const double inv = 1.0 / double(M);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = make_double2(ac[k].x * inv, -ac[k].y * inv);
        Xc[k] = cmul(c[k], v);
    }
}

// A length-n DFT of n_ch channels (x, distance n) in place, by the Stockham
// passes or by Bluestein.
struct Dft {
    int64_t n = 0, M = 0;
    bool blue = false;
    FftPlan plan, planM;
    double2 *W = nullptr, *WM = nullptr, *chirp = nullptr, *Bq = nullptr, *work = nullptr, *work2 = nullptr;

    // Scratch bytes for n_ch channels.
    size_t bytes(int64_t nn, int n_ch)
    {
        n = nn;
        blue = !plan_fft(n, plan);
        size_t e = sizeof(double2), tot = 0;
        if (!blue) {
            tot += e * n + 256;                          // W
            tot += e * n * n_ch + 256;                   // work (ping-pong partner)
        } else {
            M = 1;
            while (M < 2 * n - 1) M <<= 1;
            plan_fft(M, planM);
            tot += e * M + 256;                          // WM
            tot += e * n + 256;                          // chirp
            tot += e * M + 256;                          // B
            tot += 2 * (e * M * n_ch + 256);             // a, work
        }
        return tot;
    }
    void carve(char *p, int n_ch)
    {
        auto take = [&](size_t b) {
            char *q = p;
            p += (b + 255) & ~size_t(255);
            return reinterpret_cast<double2 *>(q);
        };
        const size_t e = sizeof(double2);
        if (!blue) {
            W = take(e * n);
            work = take(e * n * n_ch);
        } else {
            WM = take(e * M);
            chirp = take(e * n);
            Bq = take(e * M);
            work = take(e * M * n_ch);
            work2 = take(e * M * n_ch);
        }
    }
    int prepare(cudaStream_t st)
    {
        if (!blue) return fft_twiddles(n, W, st);
        MPI_TRY(fft_twiddles(M, WM, st));
        k_chirp<<<fft_blocks(n), kFftThreads, 0, st>>>(n, chirp);
        MPI_CHECK_LAUNCH();
        k_bluestein_b<<<fft_blocks(M), kFftThreads, 0, st>>>(n, M, chirp, Bq);
        MPI_CHECK_LAUNCH();
        // B = FFT_M(b) (one channel; work2 as the ping-pong partner)
        return fft_run(planM, Bq, work2, 1, M, WM, st);
    }
    int forward(double2 *x, int n_ch, cudaStream_t st)
    {
        if (!blue) return fft_run(plan, x, work, n_ch, n, W, st);
        dim3 gM(fft_blocks(M), n_ch), gn(fft_blocks(n), n_ch);
        k_bluestein_a<<<gM, kFftThreads, 0, st>>>(n, M, x, n, chirp, work);
        MPI_CHECK_LAUNCH();
        MPI_TRY(fft_run(planM, work, work2, n_ch, M, WM, st));
        k_mul_conj<<<gM, kFftThreads, 0, st>>>(M, work, Bq);
        MPI_CHECK_LAUNCH();
        MPI_TRY(fft_run(planM, work, work2, n_ch, M, WM, st));
        k_bluestein_out<<<gn, kFftThreads, 0, st>>>(n, M, work, chirp, x, n);
        MPI_CHECK_LAUNCH();
        return MPI_OK;
    }
};

// ---------------------------------------------------------------------------

template <typename R>
__global__ void k_load_real(int64_t n, const R *__restrict__ s, double2 *__restrict__ x)
{
    const R *sc = s + blockIdx.y * n;
    double2 *xc = x + blockIdx.y * n;
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x)
        xc[m] = make_double2(double(sc[m]), 0.0);
}

struct Theta {
    double v[8];
};

// X <- conj(M X / a_hat) on all n bins (conjugated so that a forward DFT of
// the result gives n times the conjugate of the inverse DFT).
__global__ void k_spectrum(int64_t n, double2 *__restrict__ X, const double2 *__restrict__ a_hat,
                           const double *__restrict__ snr, Theta th)
{
    const int64_t F = n / 2 + 1;
    double2 *Xc = X + blockIdx.y * n;
    const double2 *ac = a_hat + blockIdx.y * F;
    const double *sc = snr ? snr + blockIdx.y * F : nullptr;
    const double theta = th.v[blockIdx.y];
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n;
         f += (int64_t)gridDim.x * blockDim.x) {
        const bool mirror = f >= F;
        const int64_t fr = mirror ? n - f : f;
        double2 a = ac[fr];
        if (mirror) a.y = -a.y;
        const double den = a.x * a.x + a.y * a.y;
        const bool keep = den > 0.0 && (!sc || sc[fr] >= theta);
        double2 y = make_double2(0.0, 0.0);
        if (keep) {
            const double2 x = Xc[f];
            // x / a = x conj(a) / |a|^2
            y = make_double2((x.x * a.x + x.y * a.y) / den, (x.y * a.x - x.x * a.y) / den);
        }
        Xc[f] = make_double2(y.x, -y.y);
    }
}

template <typename R>
__global__ void k_store_real(int64_t n, const double2 *__restrict__ x, R *__restrict__ s)
{
    const double2 *xc = x + blockIdx.y * n;
    R *sc = s + blockIdx.y * n;
    const double inv = 1.0 / double(n);
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n;
         m += (int64_t)gridDim.x * blockDim.x)
        sc[m] = R(xc[m].x * inv);  // Re(conj(FFT(conj Y)))/n = Re(IDFT(Y))
}

template <typename R>
static int transfer_impl(int n_ch, int64_t T, const void *s_raw, const double *a_hat, const double *snr,
                         const double *theta, void *s_out, cudaStream_t st)
{
    Dft dft;
    Scratch scr(st);
    const size_t o_x = scr.reserve(sizeof(double2) * T * n_ch);
    const size_t o_d = scr.reserve(dft.bytes(T, n_ch));
    MPI_TRY(scr.allocate());
    double2 *x = scr.at<double2>(o_x);
    dft.carve(scr.at<char>(o_d), n_ch);
    MPI_TRY(dft.prepare(st));
    Theta th{};
    for (int k = 0; k < n_ch; ++k) th.v[k] = snr ? theta[k] : 0.0;
    dim3 g(fft_blocks(T), n_ch);
    k_load_real<R><<<g, kFftThreads, 0, st>>>(T, static_cast<const R *>(s_raw), x);
    MPI_CHECK_LAUNCH();
    MPI_TRY(dft.forward(x, n_ch, st));
    k_spectrum<<<g, kFftThreads, 0, st>>>(T, x, reinterpret_cast<const double2 *>(a_hat), snr, th);
    MPI_CHECK_LAUNCH();
    MPI_TRY(dft.forward(x, n_ch, st));
    k_store_real<R><<<g, kFftThreads, 0, st>>>(T, x, static_cast<R *>(s_out));
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

}  // namespace mpi

using namespace mpi;

extern "C" int mpi_transfer_correct(int n_ch, int64_t T, mpi_dtype dtype, const void *s_raw,
                                    const double *a_hat, const double *snr, const double *theta,
                                    void *s_out, void *stream)
{
    MPI_TRY(check_dtype(dtype));
    if (n_ch < 1 || n_ch > 8) { set_error("n_ch must be in [1, 8] (got %d)", n_ch); return MPI_ERR_INVALID; }
    if (T < 0) { set_error("T must be >= 0"); return MPI_ERR_INVALID; }
    if (T > ((int64_t)1 << 26)) { set_error("T larger than supported (2^26)"); return MPI_ERR_UNSUPPORTED; }
    if (T == 0) return MPI_OK;
    if (!s_raw || !a_hat || !s_out) { set_error("s_raw, a_hat or s_out is NULL"); return MPI_ERR_INVALID; }
    if (snr && !theta) { set_error("snr given without theta"); return MPI_ERR_INVALID; }
    if (snr)
        for (int k = 0; k < n_ch; ++k)
            if (std::isnan(theta[k])) { set_error("theta[%d] is NaN", k); return MPI_ERR_INVALID; }
    return dtype == MPI_F32
               ? transfer_impl<float>(n_ch, T, s_raw, a_hat, snr, theta, s_out, as_stream(stream))
               : transfer_impl<double>(n_ch, T, s_raw, a_hat, snr, theta, s_out, as_stream(stream));
}
