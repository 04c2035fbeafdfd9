// Internal interface shared by the PnP solve and the Core Stage solve.
#pragma once

#include "pair_ops.cuh"

namespace mpi {

// Slots of the device scalar block of a solve.
constexpr int kScalNu = 0;
constexpr int kScalLambda = 1;
constexpr int kScalSigma = 2;
constexpr int kScalPct = 3;
constexpr int kScalBnorm = 4;
constexpr int kScalTol = 5;
constexpr int kScalIter = 6;  // batched solves: PnP iterations completed

int vec_blocks(int64_t n);

// r = b0 + nu x - q, p = r, per-block partial sums of r.r (vec_blocks(N)
// blocks); clears *done.
int cg_init_launch(int64_t N, const double *b0, const double *x, const double *q,
                   const double *nu_dev, double *r, double *p, double *rr_part, int *done,
                   cudaStream_t st);
// One CG update given q = A p and the n_pq partial sums of <p, q> (pq_part).  The
// partial sums of r.r alternate between rr_in and rr_out.  thresh (device,
// nullable): stop once ||r|| <= *thresh.  iters (device, nullable): counts
// the updates performed.
int cg_step_launch(int64_t N, double *x, double *r, double *p, const double *q,
                   const double *pq_part, int n_pq, const double *rr_in, double *rr_out, int *done,
                   const double *thresh, int *iters, cudaStream_t st);

template <typename R>
int launch_gauss5(const R *in, R *out, int nx, int ny, cudaStream_t st);

// q = y + nu v and vec_blocks(N) partial sums of <v, q> (the epilogue of
// operators without a fused one).
template <typename R>
int axpy_dot_launch(int64_t N, const R *y, const double *v, const double *nu_dev, double *q,
                    double *dot_part, cudaStream_t st);

// The data-fidelity operator O of one ZeroShot-PnP solve (Algorithm 1): the
// solve driver below is written against this interface, so the 2-D operators
// (A, the convolution C) and the 3-D ones share one loop.  Every method only
// enqueues on `st`.
template <typename R>
struct PnPOperator {
    virtual ~PnPOperator() = default;
    // b0 = O^T data (FP64, N values).
    virtual int rhs(const R *data, double *b0, cudaStream_t st) = 0;
    // q = (O^T O + nu I) v and `n_pq()` partial sums of <v, q> in pq_part.
    virtual int apply_normal(const double *v, double *q, const double *nu_dev, double *pq_part,
                             cudaStream_t st) = 0;
    virtual int n_pq() const = 0;
    // The denoiser step (Algorithm 1, "Denoise"): the built-in Gaussian or a
    // user callback; returns the callback's status (nonzero = failure).
    virtual int denoise(const R *in, R *out, const double *sigma_dev, cudaStream_t st) = 0;
    virtual bool has_callback() const = 0;
    // Whether apply_normal only enqueues device work (no host wait or
    // callback), so the CG of an iteration may be captured as a CUDA graph.
    virtual bool capturable() const { return true; }
};

// Algorithm 1 with operator O on N unknowns and the data of O's range (type
// R): rho_out (R, N values), optional
// per-iteration (sigma, nu, CG residual) in info.
template <typename R>
int pnp_run(PnPOperator<R> &op, int64_t N, const void *data, const mpi_pnp_opts &o, void *rho_out,
            mpi_pnp_iter_info *info, cudaStream_t st);


}  // namespace mpi
