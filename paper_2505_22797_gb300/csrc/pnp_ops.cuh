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

}  // namespace mpi
