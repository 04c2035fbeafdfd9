/*
 * mpi_recon.h -- C ABI of the GB300 (sm_103a) library for equilibrium-model
 * (Langevin) magnetic particle imaging reconstruction, after
 * "Fast Trajectory-Independent Model-Based Reconstruction Algorithm for
 * Multi-Dimensional Magnetic Particle Imaging" (Gapyak, Maerz, Weinmann).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Every array argument is DEVICE memory owned by the caller, contiguous,
 *    row-major, in the dtype named by the call (MPI_F32: float,
 *    MPI_F64: double), unless the comment says "host".
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Argument errors are detected on the host and returned before
 *    anything is enqueued.  Device-side errors surface as MPI_ERR_CUDA from
 *    this or a later call.  On error the outputs are unspecified.
 *  - The library allocates only scratch, stream-ordered on `stream`
 *    (cudaMallocAsync / cudaFreeAsync), and releases it before the call
 *    returns (plans release theirs on destroy).
 *  - No exception crosses the ABI.  mpi_last_error_message() gives a
 *    human-readable reason for the last failure on the calling host thread.
 *
 * Model (Sec. 2 of the paper)
 * ---------------------------
 *  Voxel (i, j) has centre x_ij = (x0 + (i+1/2) dx, y0 + (j+1/2) dy) and
 *  concentration c[j][i].  Grids need nx, ny >= 1.  The field-free point moves along r(t), t = 0..T-1
 *  (r[t][2], velocity v[t][2] = dr/dt per sample).  The applied field is
 *  H(x,t) = G (x - r(t)) (Sec. 2, FFP configuration).  With
 *  beta = 1/(mu0 H_sat) (Eq. hsat) the transfer-function-corrected signal on
 *  receive channel k with coil direction p_k is (Eq. core:formula)
 *      s_k(t) = sum_ij c_ij p_k^T beta K(beta G (x_ij - r_t)) G v_t,
 *  where K is the MPI kernel matrix of Eq. kernel:matrix,
 *      K(y) = L'(|y|) yy^T/|y|^2 + L(|y|)/|y| (I - yy^T/|y|^2),
 *  L(z) = coth z - 1/z the Langevin function (Eq. momentum).  The constant
 *  -mu0 m R and the minus sign of dH/dt = -G r' are dropped, as the paper's
 *  proportionality does.  Units are the caller's: G in T per length unit,
 *  positions in that length unit, beta in 1/T.
 */
#ifndef MPI_RECON_H
#define MPI_RECON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPI_OK = 0,
    MPI_ERR_INVALID = -1,     /* bad argument (checked before any launch) */
    MPI_ERR_CUDA = -2,        /* a CUDA call failed */
    MPI_ERR_NOMEM = -3,       /* scratch allocation failed */
    MPI_ERR_CALLBACK = -4,    /* the denoiser callback returned nonzero */
    MPI_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
    MPI_ERR_UNSUPPORTED = -6  /* valid but not supported (e.g. too many frames) */
} mpi_status;

typedef enum { MPI_F32 = 0, MPI_F64 = 1 } mpi_dtype;

/* Operator of the PnP data-fidelity step: the forward operator A (data are
 * samples s[n_ch][T]) or the trace-kernel convolution C_h (data are the trace
 * image u[ny][nx], Eq. dec:sub:tik). */
typedef enum { MPI_OP_FORWARD = 0, MPI_OP_CONV = 1 } mpi_op;

/* Voxel grid: nx columns, ny rows, centres (x0+(i+1/2)dx, y0+(j+1/2)dy). */
typedef struct {
    int nx, ny;
    double x0, y0, dx, dy;
} mpi_grid_desc;

/* Physics: beta = 1/(mu0 H_sat) [1/T]; G row-major 2x2 [T per length unit];
 * n_ch receive channels (1 or 2) with directions p[k*2 + m]. */
typedef struct {
    double beta;
    double G[4];
    int n_ch;
    double p[4];
} mpi_model;

/* Trajectory: T samples, r[T][2] and v[T][2] (device, dtype of the call). */
typedef struct {
    int64_t T;
    const void *r;
    const void *v;
} mpi_traj;

/* ---- Operators ---------------------------------------------------------- */

/* Forward operator A (Eq. core:formula):  s[k][t] = sum_ij c[j][i] p_k^T
 * beta K(beta G(x_ij - r_t)) G v_t.  c is [ny][nx], s is [n_ch][T].  The sum
 * over voxels is a direct (exact, untruncated) sum, reduced deterministically:
 * the same inputs give bit-identical outputs.  T == 0 is a no-op. */
int mpi_forward(const mpi_model *model, const mpi_grid_desc *grid,
                const mpi_traj *traj, mpi_dtype dtype, const void *c, void *s,
                void *stream);

/* mpi_forward without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot let a library allocate
 * device memory while they run (a scan loop with a memory budget fixed at
 * start-up, a framework that owns all device memory through its own pool, code
 * that must avoid the implicit synchronisation of cudaFree).  Same inputs,
 * outputs and results as mpi_forward; its scratch is a fixed 32 MiB array in
 * device global memory that every GPU loading the library keeps until the
 * process exits.  Problems whose scratch does not fit are rejected with
 * MPI_ERR_UNSUPPORTED before anything is enqueued: the limit is about
 * 32 MiB / (16 + 4 n_ch) bytes per sample in FP32 (1.39 million samples with
 * two channels) and half that in FP64.  The first call on a device looks up
 * the array's device address once (with that device current); make that
 * first call before any stream capture.  The address is kept for the life of
 * the process: after cudaDeviceReset on a device it no longer names the array
 * (the reset unloads the library's device image), so do not call this entry
 * point on a device that has been reset.  All calls share the array and keep
 * nothing across calls that a later call relies on; calls that overlap on the
 * GPU (other streams or host threads at the same time) race on it. */
int mpi_forward_noalloc(const mpi_model *model, const mpi_grid_desc *grid,
                        const mpi_traj *traj, mpi_dtype dtype, const void *c, void *s,
                        void *stream);

/* Adjoint A^T:  c_out[j][i] = sum_t sum_k s[k][t] p_k^T beta K(beta G(x_ij -
 * r_t)) G v_t.  Deterministic like mpi_forward.  T == 0 writes zeros. */
int mpi_adjoint(const mpi_model *model, const mpi_grid_desc *grid,
                const mpi_traj *traj, mpi_dtype dtype, const void *s, void *c_out,
                void *stream);

/* Gradient of <g, A(c; beta)> with respect to beta, written as one FP64 value
 * to the DEVICE pointer dbeta_dev.  With y = beta G(x - r), z = |y|:
 *   d/dbeta [beta K(beta G(x-r))] G v = L'(z) G v + (L''(z)/z) (y . G v) y.
 * g is [n_ch][T] (dtype of the call); c is [ny][nx]. */
int mpi_dbeta(const mpi_model *model, const mpi_grid_desc *grid,
              const mpi_traj *traj, mpi_dtype dtype, const void *c, const void *g,
              double *dbeta_dev, void *stream);

/* Convolution with the sampled trace kernel (Eq. convolution:trace,
 * Eq. kernel:trace, the matrix C_h of Eq. dec:sub:tik), read with the
 * resolution scaling and gradient of the forward model:
 *   out[j][i] = sum_{j'i'} kappa_G(x_ij - x_i'j') in[j'][i'],
 *   kappa_G(y) = beta tr(K(beta G y) G)
 * as a linear (zero-padded) convolution over all voxel offsets.  C is
 * symmetric.  in/out are [ny][nx] and must not overlap.  Grids below 4096
 * voxels (FP32) or 1024 voxels (FP64) use the direct sum in the call's
 * dtype; larger ones the FFT route
 * (circular convolution on a padded grid, DFTs in the call's precision), the
 * same operator up to round-off.  Allocates scratch (the sampled kernel; for
 * the FFT route three complex copies of the padded grid). */
int mpi_conv(const mpi_model *model, const mpi_grid_desc *grid, mpi_dtype dtype,
             const void *in, void *out, void *stream);

/* Like mpi_conv with one entry of the kernel matrix instead of its trace:
 * kappa_ab(y) = beta (K(beta G y) G)_ab, component = 2a + b (0..3).  The
 * single-channel deconvolution of Sec. 3.6 uses the diagonal entry (a, a) of
 * the measured channel.  component = -1 gives the trace kernel (mpi_conv). */
int mpi_conv_component(const mpi_model *model, const mpi_grid_desc *grid, mpi_dtype dtype,
                       int component, const void *in, void *out, void *stream);

/* Cosine interpolation of the Core Stage (Eq. first:step):
 *   s[k][t] = sum_m I[Ahat_km](r_t) v_m(t),  k = 0, 1,
 * Ahat is [4][ny][nx] (component 2k+m), s is [2][T].  Along each axis a
 * position between nodes k and k+1 at fraction f gives node k+1 the weight
 * (1 - cos(pi f))/2; nodes are the voxel centres and positions outside the
 * node hull are clamped to the edge.  mpi_interp_adjoint is the exact
 * transpose (deterministic, no float atomics). */
int mpi_interp(const mpi_grid_desc *grid, const mpi_traj *traj, mpi_dtype dtype,
               const void *Ahat, void *s, void *stream);
int mpi_interp_adjoint(const mpi_grid_desc *grid, const mpi_traj *traj,
                       mpi_dtype dtype, const void *s, void *Ahat, void *stream);

/* Binning step of the Core Stage (Eq. first:step): the samples ordered by
 * interpolation cell.  The Core Stage solves (mpi_grid, mpi_grid3,
 * mpi_interp_adjoint) order their samples this way once per call, so that a
 * cell's samples form one contiguous run and every sum over them has a fixed
 * order; this entry exposes that step on its own.
 *   list[offset[c] .. offset[c + 1]) = the samples t with cell_of[t] = c, ascending
 * cell_of: device int [T], values in [0, n_cells).  list: device int [T]
 * (must not overlap cell_of).  offset: device int [n_cells + 1], or NULL when
 * only the order is wanted; offset[n_cells] = T.  The order is that of a
 * stable sort by cell (bit-identical on every run).  0 <= T < 2^31,
 * 1 <= n_cells < 2^31, else MPI_ERR_INVALID before any launch.  Values of
 * cell_of outside [0, n_cells) leave list and offset unspecified but are
 * never used as addresses.  Allocates scratch (about 16 B per sample). */
int mpi_cell_order(int64_t T, const int *cell_of, int n_cells, int *list, int *offset, void *stream);

/* ---- Preprocessing: transfer-function correction ------------------------- */

/* The measured signal is the model signal convolved in time with the receive
 * chain's impulse response a (Eq. core:formula:conva); over one period of T
 * samples (a periodic trajectory) the convolution is circular, and the
 * correction of Sec. 3.2 divides by the transfer function in the DFT domain
 * (Eq. core:formula) and drops unreliable frequencies:
 *   s_out[k] = IDFT_T( M_k(f) DFT_T(s_raw[k])(f) / a_hat[k](f) ),
 *   M_k(f) = 1 if snr[k][f] >= theta[k] and a_hat[k](f) != 0, else 0,
 * on the F = T/2 + 1 non-negative bins f (the output is real; the negative
 * bins mirror these).  DFT_T(x)(f) = sum_t x_t exp(-2 pi i f t / T).
 * s_raw, s_out: [n_ch][T] device arrays of the call's dtype (may be the same
 * array).  a_hat: device, FP64 complex interleaved [n_ch][F][2].  snr: device
 * FP64 [n_ch][F], or NULL for no thresholding.  theta: HOST [n_ch] (read only
 * when snr is given).  1 <= n_ch <= 8, 0 <= T <= 2^26 (any length: lengths
 * with a prime factor above 127 use Bluestein's algorithm).  The DFTs run in
 * FP64 on the device.  Allocates scratch (a few complex FP64 copies). */
int mpi_transfer_correct(int n_ch, int64_t T, mpi_dtype dtype, const void *s_raw,
                         const double *a_hat, const double *snr, const double *theta,
                         void *s_out, void *stream);

/* ---- Core Stage (Eq. first:step) ---------------------------------------- */

typedef struct {
    double gamma;    /* weight of the Laplacian regulariser (paper: 1e-7) */
    int max_iter;    /* CG iteration limit (paper: 10000) */
    double rel_tol;  /* stop when ||r|| <= rel_tol ||b|| (paper: 1e-3); <= 0: run max_iter */
    int channel;     /* 0: both channels measured; 1 or 2: only channel x (k = 0) or
                        y (k = 1) measured, the partial-data setting of Sec. 3.6 */
    int lap_scaled;  /* 0: Lap is the bare stencil (gamma in stencil units); 1: the
                        Laplacian with 1/dx^2, 1/dy^2 (and 1/dz^2 in mpi_grid3) per axis,
                        which keeps one gamma valid across grid sizes */
} mpi_grid_opts;

/* Solves ((1/T) M^T M + gamma Lap^T Lap) Ahat = (1/T) M^T s by CG from
 * Ahat = 0, with M the cosine-interpolation measurement operator above and Lap
 * the 5-point Laplacian with replicated boundary on each of the 4 components.
 * s is [2][T]; outputs Ahat [4][ny][nx] and trace [ny][nx] = Ahat_00 + Ahat_11.
 * With opts->channel = k + 1 only channel k is measured: s is [1][T] (that
 * channel), the unknowns are the two components (A_k0, A_k1) of the row k,
 * Ahat is [2][ny][nx] and `trace` receives the diagonal component A_kk, the
 * input of the single-channel deconvolution (mpi_conv_component).
 * The operator runs in the call's dtype; CG vectors and inner products are
 * FP64.  With rel_tol > 0 the host polls the device-side stop flag every 16
 * CG steps (a stream synchronisation); the result is the same as stopping at
 * the first step that meets the tolerance.  If n_iter_out (HOST) is not NULL
 * the call synchronises the stream and stores the number of CG updates.
 * With opts->lap_scaled = 0, Lap is the bare stencil (no 1/h^2), so gamma is
 * in stencil units (on a grid of spacing h = dx = dy, gamma / h^4 there equals
 * gamma with lap_scaled = 1, up to rounding). */
int mpi_grid(const mpi_grid_desc *grid, const mpi_traj *traj, mpi_dtype dtype,
             const void *s, const mpi_grid_opts *opts, void *Ahat, void *trace,
             int *n_iter_out, void *stream);

/* ---- ZeroShot-PnP (Algorithm 1) ------------------------------------------ */

/* Denoiser callback: read in[ny][nx], write out[ny][nx] (device, dtype as
 * given).  sigma_dev is a DEVICE pointer to the FP64 noise level estimated for
 * this iteration.  It must only enqueue work on `stream` (no host
 * synchronisation), and return 0 on success; any other value aborts the
 * solve with MPI_ERR_CALLBACK. */
typedef int (*mpi_denoise_fn)(const void *in, void *out, int nx, int ny,
                              mpi_dtype dtype, const double *sigma_dev,
                              void *stream, void *user);

/* Built-in denoiser: separable 5-tap Gaussian (sigma = 1 px, weights
 * exp(-m^2/2)/sum, m = -2..2) with reflect boundary (d c b a | a b c d).  It
 * ignores sigma_dev.  in and out must not overlap. */
int mpi_denoise_gaussian5(const void *in, void *out, int nx, int ny, mpi_dtype dtype,
                          const double *sigma_dev, void *stream, void *user);

typedef struct {
    mpi_op op;        /* MPI_OP_FORWARD (data s[n_ch][T]) or MPI_OP_CONV (data u[ny][nx]) */
    int n_iter;       /* outer iterations (Algorithm 1 runs exactly n_iter) */
    int n_cg;         /* CG steps per data-fidelity solve (after the initial residual) */
    double nu0;       /* initial Tikhonov weight nu_0 */
    double clip_pct;  /* percentile trimming below this percentile (paper: 5); < 0 disables */
    int kernel_component; /* MPI_OP_CONV only: 0 = trace kernel; 1 + 2a + b = entry (a, b)
                             of beta K(beta G y) G (1: channel-x deconvolution, Sec. 3.6) */
} mpi_pnp_opts;

typedef struct {
    double sigma;     /* noise estimate sqrt(Var(rho1)) of this iteration */
    double nu;        /* nu_{k+1} = lambda / sigma^2 */
    double cg_resid;  /* ||r|| after the last CG step */
    double clip;      /* the percentile value rho1 was clamped to (-inf when trimming is off) */
} mpi_pnp_iter_info;

/* Algorithm 1: rho2 <- 0; for k < n_iter: rho1 <- CG(O^T O + nu_k I,
 * O^T data + nu_k rho2, x0 = rho2); rho1 <- max(rho1, P_clip(rho1));
 * sigma <- sqrt(Var rho1); lambda <- nu0 sigma^2 (k = 0); rho2 <- denoise(rho1,
 * sigma); nu <- lambda/sigma^2 (kept if sigma == 0).  Writes the last rho2 to
 * rho_out [ny][nx].  The operator runs in the call's dtype; CG vectors, inner
 * products, norms and the PnP scalars are FP64 in both precisions.  denoise
 * NULL selects mpi_denoise_gaussian5.  info (HOST, n_iter entries) is
 * optional: when given, the call synchronises the stream at the end. */
int mpi_pnp_solve(const mpi_model *model, const mpi_grid_desc *grid,
                  const mpi_traj *traj, mpi_dtype dtype, const void *data,
                  const mpi_pnp_opts *opts, mpi_denoise_fn denoise, void *user,
                  void *rho_out, mpi_pnp_iter_info *info, void *stream);

/* Sum across the processes of a sample-sharded solve: replace the `count`
 * FP64 values of the DEVICE buffer `buf` on every process by their
 * elementwise sum over all processes, ordered on `stream` (enqueue the
 * reduction on it, or complete it before returning).  Every process must
 * receive the identical sum (an NCCL all-reduce does; so does a fixed-order
 * host sum).  Returns 0 on success; nonzero aborts the solve. */
typedef int (*mpi_allreduce_fn)(double *buf, int64_t count, void *stream, void *user);

/* Algorithm 1 with O = A for ONE problem whose trajectory samples are split
 * across processes (one GPU each).  A and A^T are sums over the samples
 * (Eq. core:formula), so the samples partition the work: each process passes
 * its own contiguous slice -- traj (r, v: [T_p][2], T_p >= 0) and data
 * (s: [n_ch][T_p]) -- while model, grid, opts and the built-in or callback
 * denoiser are the same on every process.  A of an image gives this process's
 * samples with no exchange; A^T gives a partial image, which the library sums
 * across processes with `allreduce` (N = nx*ny values): once for A^T data and
 * once per CG step.  Every other step (CG vectors, inner products, trimming,
 * noise estimate, denoiser) runs replicated on the identical reduced vectors,
 * so all processes finish with the same rho_out.  One process with an
 * allreduce that does nothing computes what mpi_pnp_solve computes, up to the
 * rounding order of the CG inner products.  opts->op must be MPI_OP_FORWARD;
 * allreduce must not be NULL.  A nonzero return of allreduce (or denoise) ends
 * the call with MPI_ERR_CALLBACK.  Allocates scratch like mpi_pnp_solve plus
 * one FP64 image. */
int mpi_pnp_solve_sharded(const mpi_model *model, const mpi_grid_desc *grid,
                          const mpi_traj *traj, mpi_dtype dtype, const void *data,
                          const mpi_pnp_opts *opts, mpi_denoise_fn denoise, void *user,
                          mpi_allreduce_fn allreduce, void *comm_user, void *rho_out,
                          mpi_pnp_iter_info *info, void *stream);

/* ---- Three-dimensional field-free point (Sec. 2 with n = 3) -------------- */

/* Voxel centres x_lji = (x0 + (i+1/2)dx, y0 + (j+1/2)dy, z0 + (l+1/2)dz);
 * volumes are row-major [nz][ny][nx]. */
typedef struct {
    int nx, ny, nz;
    double x0, y0, z0;
    double dx, dy, dz;
} mpi_grid3_desc;

/* beta = 1/(mu0 H_sat) (Eq. hsat); G the 3x3 selection-field gradient,
 * row-major (the paper's standard choice is proportional to diag(-1, -1, 2));
 * p[k*3 + m] the n_ch (1..3) receive directions. */
typedef struct {
    double beta;
    double G[9];
    int n_ch;
    double p[9];
} mpi_model3;

/* Forward operator in three dimensions (Eq. core:formula with the 3x3 kernel
 * matrix of Eq. kernel:matrix):  s[k][t] = sum_lji c[l][j][i] p_k^T
 * beta K(beta G(x_lji - r_t)) G v_t.  traj->r and traj->v are [T][3] (dtype of
 * the call), c is [nz][ny][nx], s is [n_ch][T].  Exact direct sum, reduced
 * deterministically.  T == 0 is a no-op. */
int mpi_forward3(const mpi_model3 *model, const mpi_grid3_desc *grid, const mpi_traj *traj,
                 mpi_dtype dtype, const void *c, void *s, void *stream);

/* Adjoint in three dimensions: c_out[l][j][i] = sum_t sum_k s[k][t] p_k^T
 * beta K(beta G(x_lji - r_t)) G v_t.  T == 0 writes zeros. */
int mpi_adjoint3(const mpi_model3 *model, const mpi_grid3_desc *grid, const mpi_traj *traj,
                 mpi_dtype dtype, const void *s, void *c_out, void *stream);

/* out = C in with the sampled 3-D trace kernel kappa_G(y) = beta tr(K(beta G
 * y) G) (Eq. kernel:trace with n - 1 = 2), linear (zero-padded) over all
 * voxel offsets.  in and out [nz][ny][nx], must not overlap.  Volumes from
 * 8192 voxels (FP32) or 512 voxels (FP64) take the FFT route (circular
 * convolution on a padded power-of-two grid, DFTs in the call's precision):
 * the same operator up to round-off. */
int mpi_conv3(const mpi_model3 *model, const mpi_grid3_desc *grid, mpi_dtype dtype, const void *in,
              void *out, void *stream);

/* mpi_conv3 with a choice of kernel: 0 = the trace kernel above; 1 =
 * beta tr K(beta G y), the kernel of the gradient-weighted trace
 * tr(Ahat G^-1) (mpi_weighted_trace3).  For a traceless G (the physical 3-D
 * FFP gradient, proportional to diag(-1, -1, 2)) the trace kernel reduces to
 * beta d(z) y^T G y, which changes sign and has almost no mean; kernel 1 is
 * positive for any G. */
int mpi_conv3_kernel(const mpi_model3 *model, const mpi_grid3_desc *grid, mpi_dtype dtype, int kernel,
                     const void *in, void *out, void *stream);

/* out[l][j][i] = tr(Ahat G^-1) = sum_{k,m} Ahat[3k+m][l][j][i] (G^-1)_mk for the 9
 * components of mpi_grid3 (device, dtype of the call; summed in FP64).  Since
 * Ahat = beta K(beta G .) G * c, this is (beta tr K(beta G y)) * c: the input
 * of the deconvolution with mpi_conv3_kernel(kernel = 1). */
int mpi_weighted_trace3(const mpi_model3 *model, const mpi_grid3_desc *grid, mpi_dtype dtype,
                        const void *Ahat, void *out, void *stream);

/* Volume denoiser callback: as mpi_denoise_fn on [nz][ny][nx]. */
typedef int (*mpi_denoise3_fn)(const void *in, void *out, int nx, int ny, int nz, mpi_dtype dtype,
                               const double *sigma_dev, void *stream, void *user);

/* Built-in volume denoiser: the 5-tap Gaussian of mpi_denoise_gaussian5 along
 * x, then y, then z (reflect boundary).  Allocates one volume of scratch. */
int mpi_denoise_gaussian5_3d(const void *in, void *out, int nx, int ny, int nz, mpi_dtype dtype,
                             const double *sigma_dev, void *stream, void *user);

/* Algorithm 1 in three dimensions (the loop of mpi_pnp_solve) with the 3-D
 * forward operator (data s[n_ch][T]) or the 3-D convolution (data
 * u[nz][ny][nx]); opts->kernel_component selects the convolution's kernel as
 * in mpi_conv3_kernel (0 or 1; 0 with the forward operator).  denoise NULL
 * selects mpi_denoise_gaussian5_3d.  rho_out is [nz][ny][nx]. */
int mpi_pnp_solve3(const mpi_model3 *model, const mpi_grid3_desc *grid, const mpi_traj *traj,
                   mpi_dtype dtype, const void *data, const mpi_pnp_opts *opts, mpi_denoise3_fn denoise,
                   void *user, void *rho_out, mpi_pnp_iter_info *info, void *stream);

/* Core Stage in three dimensions (Eq. first:step with n = 3).  The core
 * operator at a point is the 3 x 3 matrix Ahat_km (receive channel k along
 * the coordinate axis k, velocity component m), stored [9][nz][ny][nx] with
 * component index 3k + m; I is the tensor product of the cosine interpolation
 * of mpi_interp along x, y and z (nodes at the voxel centres, positions
 * clamped to the node hull).  traj->r and traj->v are [T][3], s is [3][T]
 * (channel k, sample t):
 *   s[k][t] = sum_m I[Ahat_km](r_t) v_m(t).
 * Same conventions as mpi_interp: device pointers, dtype of the call, T < 2^31,
 * grids of fewer than 2^27 nodes; T == 0 writes nothing. */
int mpi_interp3(const mpi_grid3_desc *grid, const mpi_traj *traj, mpi_dtype dtype,
                const void *Ahat, void *s, void *stream);

/* Exact transpose of mpi_interp3: Ahat[3k+m] = sum_t w(r_t) v_m(t) s[k][t]
 * ([3][T] -> [9][nz][ny][nx]), summed in a fixed order (no atomics). */
int mpi_interp3_adjoint(const mpi_grid3_desc *grid, const mpi_traj *traj, mpi_dtype dtype,
                        const void *s, void *Ahat, void *stream);

/* Solves ((1/T) M^T M + gamma Lap^T Lap) Ahat = (1/T) M^T s by CG from
 * Ahat = 0 with M = mpi_interp3 and Lap the 7-point Laplacian with replicated
 * boundary on each of the 9 components.  opts as for mpi_grid, with channel 0
 * (all three channels: s [3][T], Ahat [9][nz][ny][nx], trace [nz][ny][nx] =
 * A_00 + A_11 + A_22) or k + 1 (only channel k = 0, 1, 2 measured: s [1][T],
 * Ahat holds the row (A_k0, A_k1, A_k2) as [3][nz][ny][nx], trace = A_kk).
 * Operator in the call's dtype, CG vectors and inner products FP64; the stop
 * test, polling, n_iter_out and the units of gamma (bare 7-point stencil)
 * behave as in mpi_grid. */
int mpi_grid3(const mpi_grid3_desc *grid, const mpi_traj *traj, mpi_dtype dtype,
              const void *s, const mpi_grid_opts *opts, void *Ahat, void *trace,
              int *n_iter_out, void *stream);

/* ---- Batched reconstructions --------------------------------------------- */

/* A plan runs Algorithm 1 with the forward operator (FP32 operator, FP64 CG
 * vectors, inner products and PnP scalars, built-in Gaussian denoiser) for up
 * to MPI_BATCH_MAX_FRAMES independent frames of different grid sizes and
 * trajectory lengths at once: every operator application over all frames is
 * one launch of the pair kernel over a frame table, the CG, percentile and
 * denoiser steps are batched the same way, and one PnP iteration of all frames
 * is captured once as a CUDA graph and replayed n_iter times.  Each frame
 * has its own model, grid, T and nu0 (host arrays of n_frames entries); opts
 * gives n_iter, n_cg and clip_pct for all frames (op must be MPI_OP_FORWARD).
 * The plan owns its device memory (cudaMalloc at create, cudaFree at
 * destroy).  Flags: MPI_BATCH_AUTOTUNE times candidate work-item sizes and
 * launch forms (one block per item, or a persistent grid pulling items from a
 * device counter) on the first run, which then synchronises the stream once;
 * the choice is cached in the file named by $MPI_AUTOTUNE_CACHE when set.
 * MPI_BATCH_MATCH_SINGLE splits every frame exactly as mpi_pnp_solve does,
 * so each frame's result is bit-identical to its single-frame solve. */
#define MPI_BATCH_MAX_FRAMES 64
#define MPI_BATCH_AUTOTUNE 1
#define MPI_BATCH_MATCH_SINGLE 2

typedef struct mpi_batch_plan mpi_batch_plan;

typedef struct {
    int n_frames;
    int tuned;                    /* the split in use is the tuned one (or was fixed) */
    long long item_pairs_forward; /* work-item budget (pairs) of the forward launch */
    long long item_pairs_adjoint;
    int persistent_forward;       /* launch form chosen: 1 = persistent grid */
    int persistent_adjoint;
    long long forward_items;      /* work items per forward / adjoint launch */
    long long adjoint_items;
    long long device_bytes;       /* device memory owned by the plan */
    long long graph_nodes;        /* kernels in the captured PnP iteration (0 before the first run) */
} mpi_batch_info;

int mpi_batch_plan_create(int n_frames, const mpi_model *models, const mpi_grid_desc *grids,
                          const int64_t *T, const double *nu0, const mpi_pnp_opts *opts,
                          int flags, mpi_batch_plan **plan);
/* r[f], v[f]: [T_f][2], s[f]: [n_ch_f][T_f], rho_out[f]: [ny_f][nx_f] (device,
 * float; host arrays of n_frames pointers).  Asynchronous on `stream` except
 * for the tuning run. */
int mpi_batch_pnp_run(mpi_batch_plan *plan, const void *const *r, const void *const *v,
                      const void *const *s, void *const *rho_out, void *stream);
int mpi_batch_plan_info(const mpi_batch_plan *plan, mpi_batch_info *info);
int mpi_batch_plan_destroy(mpi_batch_plan *plan);

/* ---- Diagnostics --------------------------------------------------------- */

const char *mpi_status_string(int status);
const char *mpi_last_error_message(void);
/* Library version as 10000*major + 100*minor + patch. */
int mpi_version(void);
/* Number of kernel launches the library has enqueued since it was loaded
 * (all streams, all devices). */
long long mpi_kernel_launches(void);

/* Event timing of the operator kernels.  While enabled, every launch of the
 * forward-operator kernel (class 0), the adjoint kernel (1), the d/dbeta
 * kernel (2) and the convolution kernel (3) is bracketed by a CUDA event pair
 * recorded on its launching stream.  mpi_profile_enable(1/0) turns it on/off
 * and resets the totals; mpi_profile_read synchronises on the recorded events
 * and returns the number of timed launches and their summed duration (ms) for
 * one class. */
int mpi_profile_enable(int enable);
int mpi_profile_read(int kernel_class, long long *launches, double *total_ms);

/* Measured instruction throughput of the GPU (no counterpart in the paper:
 * it supplies the denominator of the pair kernels' roofline, which are bound
 * by instruction issue on the FP32 and MUFU/XU pipes, not by memory).
 * Launches blocks_per_sm (1..8) blocks of 256 threads per SM on the current
 * device; every thread runs 8 independent chains of `iters` (1..2^20)
 * operations of kind `op`.  *ops_per_clk_sm receives the median over SMs of
 * the thread-operations completed per SM clock cycle (clock64 spans of the
 * SM's blocks, so independent of the clock frequency); *ms (nullable) the
 * CUDA-event time of the launch.  Allocates ~2 MB of scratch
 * (stream-ordered) and synchronises `stream`.  MPI_ERR_INVALID on arguments
 * out of range. */
#define MPI_PROBE_FMA 0   /* FP32 fma.rn */
#define MPI_PROBE_RSQRT 1 /* rsqrt.approx.ftz.f32 */
#define MPI_PROBE_EX2 2   /* ex2.approx.ftz.f32 */
#define MPI_PROBE_RCP 3   /* rcp.approx.ftz.f32 (each after an FP32 add) */
#define MPI_PROBE_DFMA 4  /* FP64 fma.rn */
#define MPI_PROBE_FMA2 5  /* fma.rn.f32x2 (two packed FP32 lanes: counted as 2 operations) */
int mpi_probe_pipe_rate(int op, int blocks_per_sm, int iters, double *ops_per_clk_sm, double *ms,
                        void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPI_RECON_H */
