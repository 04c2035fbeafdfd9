// ZeroShot-PnP deconvolution (Algorithm 1) on the GPU, with the forward
// operator A or the trace-kernel convolution C as the data-fidelity operator:
// CG vector kernels with deterministic FP64 inner products, the percentile
// trimming and noise estimate (one single-block kernel), the built-in 5-tap
// Gaussian denoiser, and the mpi_pnp_solve / mpi_conv /
// mpi_denoise_gaussian5 entry points.  All PnP scalars (nu, lambda, sigma,
// the CG alpha/beta) stay on the device, so a solve enqueues without any host
// synchronisation.
#include <cmath>
#include <cstring>
#include <vector>

#include "graph.cuh"
#include "conv_ops.cuh"
#include "pnp_device.cuh"

namespace mpi {

int check_model(const mpi_model *m);
int check_grid(const mpi_grid_desc *g);
int check_traj(const mpi_traj *t);
int check_dtype(mpi_dtype d);
ModelH to_host(const mpi_model *m);
GridH to_host(const mpi_grid_desc *g);

int vec_blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + kVecPerBlock - 1) / kVecPerBlock); }

template <typename R>
__global__ void k_set_x(int64_t N, const R *__restrict__ src, double *__restrict__ x)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x)
        x[e] = src ? double(src[e]) : 0.0;
}

// r = b0 + nu x - q;  p = r;  partial sums of r.r;  clears the stop flag.
__global__ void __launch_bounds__(kVecThreads)
k_cg_init(int64_t N, const double *__restrict__ b0, const double *__restrict__ x,
          const double *__restrict__ q, const double *__restrict__ nu_dev, double *__restrict__ r,
          double *__restrict__ p, double *__restrict__ rr_part, int *__restrict__ done)
{
    __shared__ double sh[kVecThreads / 32 + 1];
    const double nu = *nu_dev;
    const int64_t e0 = (int64_t)blockIdx.x * kVecPerBlock, e1 = min(N, e0 + kVecPerBlock);
    double acc = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kVecThreads) {
        const double re = (b0[e] + nu * x[e]) - q[e];
        r[e] = re;
        p[e] = re;
        acc += re * re;
    }
    acc = block_sum<double, kVecThreads>(acc, sh);
    if (threadIdx.x == 0) {
        rr_part[blockIdx.x] = acc;
        if (blockIdx.x == 0) *done = 0;
    }
}

// alpha = r.r / p.q;  x += alpha p;  r -= alpha q;  partial sums of the new r.r.
// Once r.r or p.q is exactly 0 the solve has converged to round-off: the stop
// flag is set and the remaining steps leave x, r and p untouched.  With a
// threshold (Core Stage), the solve also stops once ||r|| <= *thresh, checked
// before the update as the textbook loop does; `iters` counts the updates.
__global__ void __launch_bounds__(kVecThreads)
k_cg_step1(int64_t N, int nblk, double *__restrict__ x, double *__restrict__ r,
           const double *__restrict__ p, const double *__restrict__ q,
           const double *__restrict__ pq_part, int n_pq, const double *__restrict__ rr_in,
           double *__restrict__ rr_out, int *__restrict__ done, const double *__restrict__ thresh,
           int *__restrict__ iters)
{
    __shared__ double sh[kVecThreads / 32 + 1];
    const double rr = sum_parts<kVecThreads>(rr_in, nblk, sh);
    const double pq = sum_parts<kVecThreads>(pq_part, n_pq, sh);
    const bool stop = (*done != 0) || rr == 0.0 || pq == 0.0 || (thresh && sqrt(rr) <= *thresh);
    if (stop) {
        if (threadIdx.x == 0) {
            rr_out[blockIdx.x] = rr_in[blockIdx.x];
            if (blockIdx.x == 0) *done = 1;
        }
        return;
    }
    if (iters && blockIdx.x == 0 && threadIdx.x == 0) *iters += 1;
    const double alpha = rr / pq;
    const int64_t e0 = (int64_t)blockIdx.x * kVecPerBlock, e1 = min(N, e0 + kVecPerBlock);
    double acc = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kVecThreads) {
        x[e] = x[e] + alpha * p[e];
        const double re = r[e] - alpha * q[e];
        r[e] = re;
        acc += re * re;
    }
    acc = block_sum<double, kVecThreads>(acc, sh);
    if (threadIdx.x == 0) rr_out[blockIdx.x] = acc;
}

// beta = r.r(new) / r.r(old);  p = r + beta p.
__global__ void __launch_bounds__(kVecThreads)
k_cg_step2(int64_t N, int nblk, const double *__restrict__ r, double *__restrict__ p,
           const double *__restrict__ rr_old, const double *__restrict__ rr_new,
           const int *__restrict__ done)
{
    __shared__ double sh[kVecThreads / 32 + 1];
    if (*done) return;
    const double ro = sum_parts<kVecThreads>(rr_old, nblk, sh);
    const double rn = sum_parts<kVecThreads>(rr_new, nblk, sh);
    const double beta = rn / ro;
    const int64_t e0 = (int64_t)blockIdx.x * kVecPerBlock, e1 = min(N, e0 + kVecPerBlock);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kVecThreads) p[e] = r[e] + beta * p[e];
}

// q = y + nu v, partial sums of v.q  (epilogue for operators without a fused one).
template <typename R>
__global__ void __launch_bounds__(kVecThreads)
k_axpy_dot(int64_t N, const R *__restrict__ y, const double *__restrict__ v,
           const double *__restrict__ nu_dev, double *__restrict__ q, double *__restrict__ dot_part)
{
    __shared__ double sh[kVecThreads / 32 + 1];
    const double nu = *nu_dev;
    const int64_t e0 = (int64_t)blockIdx.x * kVecPerBlock, e1 = min(N, e0 + kVecPerBlock);
    double acc = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kVecThreads) {
        const double qe = double(y[e]) + nu * v[e];
        q[e] = qe;
        acc += v[e] * qe;
    }
    acc = block_sum<double, kVecThreads>(acc, sh);
    if (threadIdx.x == 0) dot_part[blockIdx.x] = acc;
}

template <typename R>
int axpy_dot_launch(int64_t N, const R *y, const double *v, const double *nu_dev, double *q,
                    double *dot_part, cudaStream_t st)
{
    k_axpy_dot<R><<<vec_blocks(N), kVecThreads, 0, st>>>(N, y, v, nu_dev, q, dot_part);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}
template int axpy_dot_launch<float>(int64_t, const float *, const double *, const double *, double *,
                                    double *, cudaStream_t);
template int axpy_dot_launch<double>(int64_t, const double *, const double *, const double *, double *,
                                     double *, cudaStream_t);

__global__ void k_init_scalars(double *scal, double nu0)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        scal[kScalNu] = nu0;
        scal[kScalLambda] = 0.0;
        scal[kScalSigma] = 0.0;
        scal[kScalPct] = 0.0;
    }
}

int cg_init_launch(int64_t N, const double *b0, const double *x, const double *q,
                   const double *nu_dev, double *r, double *p, double *rr_part, int *done,
                   cudaStream_t st)
{
    k_cg_init<<<vec_blocks(N), kVecThreads, 0, st>>>(N, b0, x, q, nu_dev, r, p, rr_part, done);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

int cg_step_launch(int64_t N, double *x, double *r, double *p, const double *q,
                   const double *pq_part, int n_pq, const double *rr_in, double *rr_out, int *done,
                   const double *thresh, int *iters, cudaStream_t st)
{
    const int nblk = vec_blocks(N);
    k_cg_step1<<<nblk, kVecThreads, 0, st>>>(N, nblk, x, r, p, q, pq_part, n_pq, rr_in, rr_out,
                                            done, thresh, iters);
    MPI_CHECK_LAUNCH();
    k_cg_step2<<<nblk, kVecThreads, 0, st>>>(N, nblk, r, p, rr_in, rr_out, done);
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

template <typename R>
__global__ void __launch_bounds__(kStatThreads)
k_outer_stats(int64_t N, const double *__restrict__ x, int do_clip, double pct, int k, double nu0,
              double *__restrict__ scal, const double *__restrict__ rr_part, int nblk,
              double *__restrict__ info_row, R *__restrict__ rho1)
{
    outer_stats_block<R>(N, x, do_clip, pct, k == 0, nu0, scal, rr_part, nblk, info_row, rho1);
}

template <typename R>
__global__ void __launch_bounds__(kGx *kGy)
k_gauss5(const R *__restrict__ in, R *__restrict__ out, int nx, int ny, R w0, R w1, R w2)
{
    gauss5_tile<R>(in, out, nx, ny, blockIdx.x * kGx, blockIdx.y * kGy, w0, w1, w2);
}

template <typename R>
int launch_gauss5(const R *in, R *out, int nx, int ny, cudaStream_t st)
{
    double w[3];
    gauss5_weights(w);
    dim3 grid((nx + kGx - 1) / kGx, (ny + kGy - 1) / kGy);
    k_gauss5<R><<<grid, kGx * kGy, 0, st>>>(in, out, nx, ny, R(w[0]), R(w[1]), R(w[2]));
    MPI_CHECK_LAUNCH();
    return MPI_OK;
}

// ---------------------------------------------------------------------------
// The PnP solve: one driver (pnp_run) over an operator interface.

template <typename R>
int pnp_run(PnPOperator<R> &op, int64_t N, const void *data, const mpi_pnp_opts &o, void *rho_out,
            mpi_pnp_iter_info *info, cudaStream_t st)
{
    const int nblk = vec_blocks(N);
    const int n_pq = op.n_pq();
    Scratch scr(st);
    const size_t vb = sizeof(double) * N;
    const size_t o_b0 = scr.reserve(vb), o_x = scr.reserve(vb), o_r = scr.reserve(vb),
                 o_p = scr.reserve(vb), o_q = scr.reserve(vb);
    const size_t o_pq = scr.reserve(sizeof(double) * std::max(nblk, n_pq));
    const size_t o_rr0 = scr.reserve(sizeof(double) * nblk), o_rr1 = scr.reserve(sizeof(double) * nblk);
    const size_t o_sc = scr.reserve(sizeof(double) * 8 + sizeof(int) * 4);
    const size_t o_info = scr.reserve(sizeof(double) * kInfoCols * std::max(o.n_iter, 1));
    const size_t o_r1 = scr.reserve(sizeof(R) * N), o_r2 = scr.reserve(sizeof(R) * N);
    MPI_TRY(scr.allocate());
    double *b0 = scr.at<double>(o_b0), *x = scr.at<double>(o_x), *r = scr.at<double>(o_r),
           *p = scr.at<double>(o_p), *q = scr.at<double>(o_q), *pq_part = scr.at<double>(o_pq);
    double *rr_part[2] = {scr.at<double>(o_rr0), scr.at<double>(o_rr1)};
    double *scal = scr.at<double>(o_sc), *inf = scr.at<double>(o_info);
    int *done = reinterpret_cast<int *>(scal + 8);
    R *rho1 = scr.at<R>(o_r1), *rho2 = scr.at<R>(o_r2);

    // b0 = O^T data
    MPI_TRY(op.rhs(static_cast<const R *>(data), b0, st));
    k_init_scalars<<<1, 32, 0, st>>>(scal, o.nu0);
    MPI_CHECK_LAUNCH();

    const bool fault_cb = getenv("MPI_FAULT") && strcmp(getenv("MPI_FAULT"), "callback") == 0;
    const int vgrid = (int)std::min<int64_t>((N + 255) / 256, 4096);
    // The CG of one iteration (from x = rho2): q = (O^T O + nu I) x, the
    // initial residual and n_cg steps -- the same launches with the same
    // arguments every iteration (nu is read on the device).
    auto enqueue_cg = [&](cudaStream_t s) -> int {
        MPI_TRY(op.apply_normal(x, q, scal + kScalNu, pq_part, s));
        MPI_TRY(cg_init_launch(N, b0, x, q, scal + kScalNu, r, p, rr_part[0], done, s));
        for (int i = 0; i < o.n_cg; ++i) {
            MPI_TRY(op.apply_normal(p, q, scal + kScalNu, pq_part, s));
            MPI_TRY(cg_step_launch(N, x, r, p, q, pq_part, n_pq, rr_part[i & 1], rr_part[(i + 1) & 1],
                                   done, nullptr, nullptr, s));
        }
        return MPI_OK;
    };
    // Captured once as a CUDA graph and replayed every iteration (the launches
    // are short at small sizes, where issuing them one by one is the cost);
    // not with the per-launch profiler on or an operator that calls back.
    CapturedGraph cg_graph;
    if (o.n_iter >= 2 && op.capturable() && !profile_enabled()) (void)cg_graph.capture(enqueue_cg);
    for (int k = 0; k < o.n_iter; ++k) {
        // rho1 <- CG(O^T O + nu I, O^T data + nu rho2, x0 = rho2), n_cg steps
        k_set_x<R><<<vgrid, 256, 0, st>>>(N, k == 0 ? nullptr : rho2, x);
        MPI_CHECK_LAUNCH();
        if (cg_graph.ready()) MPI_TRY(cg_graph.launch(st));
        else MPI_TRY(enqueue_cg(st));
        // trimming, sigma, lambda (k = 0), nu
        k_outer_stats<R><<<1, kStatThreads, 0, st>>>(N, x, o.clip_pct >= 0.0 ? 1 : 0, o.clip_pct, k,
                                                    o.nu0, scal, rr_part[o.n_cg & 1], nblk,
                                                    inf + kInfoCols * k, rho1);
        MPI_CHECK_LAUNCH();
        R *dst = (k == o.n_iter - 1) ? static_cast<R *>(rho_out) : rho2;
        const int rc = fault_cb ? 1 : op.denoise(rho1, dst, scal + kScalSigma, st);
        if (rc != 0) {
            if (op.has_callback() || fault_cb) {
                set_error("denoiser callback returned %d at iteration %d", rc, k);
                return MPI_ERR_CALLBACK;
            }
            return rc;
        }
    }
    if (o.n_iter == 0) MPI_TRY_CUDA(cudaMemsetAsync(rho_out, 0, sizeof(R) * N, st));
    if (info) {
        std::vector<double> h(kInfoCols * std::max(o.n_iter, 1));
        MPI_TRY_CUDA(cudaMemcpyAsync(h.data(), inf, sizeof(double) * kInfoCols * o.n_iter,
                                     cudaMemcpyDeviceToHost, st));
        MPI_TRY_CUDA(cudaStreamSynchronize(st));
        for (int k = 0; k < o.n_iter; ++k) {
            info[k].sigma = h[kInfoCols * k];
            info[k].nu = h[kInfoCols * k + 1];
            info[k].cg_resid = h[kInfoCols * k + 2];
            info[k].clip = h[kInfoCols * k + 3];
        }
    }
    return MPI_OK;
}

// The 2-D operators: A (direct pair sums over the trajectory) or C (the
// sampled-kernel convolution), and the 2-D denoiser.
template <typename R>
struct PnPOp2D final : PnPOperator<R> {
    mpi_op op;
    ModelH m;
    GridH g;
    int64_t T = 0;
    Geometry<R> geo{};
    FwdSplit fs{};
    AdjSplit as{};
    R *fwd_part = nullptr, *adj_part = nullptr, *sA = nullptr;
    ConvPlan<R> C;
    R *tmp1 = nullptr, *tmp2 = nullptr;
    int64_t N = 0;
    mpi_denoise_fn den = nullptr;
    void *user = nullptr;
    // Sample-sharded solve: this process's samples only; partial A^T images
    // are summed across processes by `ar` into `red` (FP64, N values).
    mpi_allreduce_fn ar = nullptr;
    void *ar_user = nullptr;
    double *red = nullptr;

    int reduce(double *buf, cudaStream_t st)
    {
        const int rc = ar(buf, N, st, ar_user);
        if (rc != 0) {
            set_error("allreduce callback returned %d", rc);
            return MPI_ERR_CALLBACK;
        }
        return MPI_OK;
    }
    int rhs(const R *data, double *b0, cudaStream_t st) override
    {
        if (op == MPI_OP_FORWARD) {
            MPI_TRY((launch_adjoint<R, double>(m, g, T, geo, as, data, adj_part, b0, nullptr, nullptr,
                                               nullptr, st)));
            return ar ? reduce(b0, st) : MPI_OK;
        }
        return conv_apply<R, R, double>(C, data, b0, st);
    }
    int apply_normal(const double *v, double *q, const double *nu_dev, double *pq_part,
                     cudaStream_t st) override
    {
        if (op == MPI_OP_FORWARD) {
            MPI_TRY((launch_forward<R, double, R>(m, g, T, geo, fs, v, fwd_part, sA, st)));
            if (!ar)
                return launch_adjoint<R, double>(m, g, T, geo, as, sA, adj_part, q, v, nu_dev, pq_part, st);
            // partial A^T A v of this process's samples, summed across
            // processes, then q = sum + nu v with the <v, q> partials
            MPI_TRY((launch_adjoint<R, double>(m, g, T, geo, as, sA, adj_part, red, nullptr, nullptr,
                                               nullptr, st)));
            MPI_TRY(reduce(red, st));
            return axpy_dot_launch<double>(N, red, v, nu_dev, q, pq_part, st);
        }
        MPI_TRY((conv_apply<R, double, R>(C, v, tmp1, st)));
        MPI_TRY((conv_apply<R, R, R>(C, tmp1, tmp2, st)));
        return axpy_dot_launch<R>(N, tmp2, v, nu_dev, q, pq_part, st);
    }
    int n_pq() const override
    {
        return (op == MPI_OP_FORWARD && !ar) ? adjoint_dot_blocks(g.nx, g.ny) : vec_blocks(N);
    }
    int denoise(const R *in, R *out, const double *sigma_dev, cudaStream_t st) override
    {
        if (den) return den(in, out, g.nx, g.ny, sizeof(R) == 4 ? MPI_F32 : MPI_F64, sigma_dev, st, user);
        return launch_gauss5<R>(in, out, g.nx, g.ny, st);
    }
    bool has_callback() const override { return den != nullptr; }
    bool capturable() const override { return ar == nullptr; }
};

template <typename R>
static int pnp_impl(const ModelH &m, const GridH &g, const mpi_traj *tr, const void *data,
                    const mpi_pnp_opts &o, mpi_denoise_fn den, void *user, void *rho_out,
                    mpi_pnp_iter_info *info, cudaStream_t st, mpi_allreduce_fn ar = nullptr,
                    void *ar_user = nullptr)
{
    PnPOp2D<R> S;
    S.op = o.op;
    S.m = m;
    S.g = g;
    S.T = (o.op == MPI_OP_FORWARD) ? tr->T : 0;
    S.N = (int64_t)g.nx * g.ny;
    S.den = den;
    S.user = user;
    S.ar = ar;
    S.ar_user = ar_user;
    const int target = default_target_items();

    Scratch scr(st);
    size_t o_geo = 0, o_fp = 0, o_ap = 0, o_sA = 0, o_K = 0, o_t1 = 0, o_t2 = 0, o_ord = 0, o_red = 0;
    if (ar) o_red = scr.reserve(sizeof(double) * size_t(S.N));
    if (S.op == MPI_OP_FORWARD) {
        S.fs = forward_split(S.T, g.nx, g.ny, sizeof(R), forward_target_items());
        S.as = adjoint_split(S.T, g.nx, g.ny, target, sizeof(R));
        o_geo = scr.reserve(geometry_bytes<R>(S.T, g.nx, g.ny));
        o_ord = scr.reserve(item_order_bytes<R>(&S.fs, &S.as));
        o_fp = scr.reserve(forward_partial_bytes<R>(S.fs, m.n_ch, S.T));
        o_ap = scr.reserve(adjoint_partial_bytes<R>(S.as, g.nx, g.ny));
        o_sA = scr.reserve(sizeof(R) * size_t(m.n_ch) * size_t(std::max<int64_t>(S.T, 1)));
    } else {
        o_K = scr.reserve(conv_plan_bytes(g.nx, g.ny, sizeof(R)));
        o_t1 = scr.reserve(sizeof(R) * S.N);
        o_t2 = scr.reserve(sizeof(R) * S.N);
    }
    MPI_TRY(scr.allocate());
    if (ar) S.red = scr.at<double>(o_red);
    if (S.op == MPI_OP_FORWARD) {
        S.geo = geometry_carve<R>(scr.at<char>(o_geo), S.T, g.nx, g.ny);
        S.fwd_part = scr.at<R>(o_fp);
        S.adj_part = scr.at<R>(o_ap);
        S.sA = scr.at<R>(o_sA);
        MPI_TRY(prepare_geometry<R>(m, g, S.T, tr->r, tr->v, S.geo, st));
        MPI_TRY(prepare_item_orders<R>(g, S.T, S.geo, &S.fs, &S.as, scr.at<char>(o_ord), st));
    } else {
        MPI_TRY(conv_plan_prepare<R>(m, g, scr.at<char>(o_K), S.C, st, o.kernel_component - 1));
        S.tmp1 = scr.at<R>(o_t1);
        S.tmp2 = scr.at<R>(o_t2);
    }
    return pnp_run<R>(S, S.N, data, o, rho_out, info, st);
}

template <typename R>
static int conv_impl(const ModelH &m, const GridH &g, const void *in, void *out, cudaStream_t st,
                     int comp = -1)
{
    Scratch scr(st);
    const size_t o_K = scr.reserve(conv_plan_bytes(g.nx, g.ny, sizeof(R)));
    MPI_TRY(scr.allocate());
    ConvPlan<R> C;
    MPI_TRY(conv_plan_prepare<R>(m, g, scr.at<char>(o_K), C, st, comp));
    return conv_apply<R, R, R>(C, static_cast<const R *>(in), static_cast<R *>(out), st);
}

template int launch_gauss5<float>(const float *, float *, int, int, cudaStream_t);
template int launch_gauss5<double>(const double *, double *, int, int, cudaStream_t);
template int pnp_run<float>(PnPOperator<float> &, int64_t, const void *, const mpi_pnp_opts &, void *,
                            mpi_pnp_iter_info *, cudaStream_t);
template int pnp_run<double>(PnPOperator<double> &, int64_t, const void *, const mpi_pnp_opts &, void *,
                             mpi_pnp_iter_info *, cudaStream_t);

}  // namespace mpi

using namespace mpi;

extern "C" {

int mpi_pnp_solve(const mpi_model *model, const mpi_grid_desc *grid, const mpi_traj *traj,
                  mpi_dtype dtype, const void *data, const mpi_pnp_opts *opts,
                  mpi_denoise_fn denoise, void *user, void *rho_out, mpi_pnp_iter_info *info,
                  void *stream)
{
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_dtype(dtype));
    if (!opts) { set_error("opts is NULL"); return MPI_ERR_INVALID; }
    if (opts->op != MPI_OP_FORWARD && opts->op != MPI_OP_CONV) {
        set_error("unknown operator %d", (int)opts->op);
        return MPI_ERR_INVALID;
    }
    if (opts->op == MPI_OP_FORWARD) MPI_TRY(check_traj(traj));
    if (opts->n_iter < 0 || opts->n_cg < 0 || !(opts->nu0 >= 0.0) || !std::isfinite(opts->nu0) ||
        !(opts->clip_pct <= 100.0) || std::isnan(opts->clip_pct) || opts->kernel_component < 0 ||
        opts->kernel_component > 4) {
        set_error("invalid PnP options (n_iter %d, n_cg %d, nu0 %g, clip_pct %g)", opts->n_iter,
                  opts->n_cg, opts->nu0, opts->clip_pct);
        return MPI_ERR_INVALID;
    }
    if (!rho_out || (!data && !(opts->op == MPI_OP_FORWARD && traj->T == 0))) {
        set_error("data or rho_out is NULL");
        return MPI_ERR_INVALID;
    }
    const ModelH m = to_host(model);
    const GridH g = to_host(grid);
    return dtype == MPI_F32
               ? pnp_impl<float>(m, g, traj, data, *opts, denoise, user, rho_out, info, as_stream(stream))
               : pnp_impl<double>(m, g, traj, data, *opts, denoise, user, rho_out, info, as_stream(stream));
}

int mpi_pnp_solve_sharded(const mpi_model *model, const mpi_grid_desc *grid, const mpi_traj *traj,
                          mpi_dtype dtype, const void *data, const mpi_pnp_opts *opts,
                          mpi_denoise_fn denoise, void *user, mpi_allreduce_fn allreduce,
                          void *comm_user, void *rho_out, mpi_pnp_iter_info *info, void *stream)
{
    if (!allreduce) { set_error("allreduce is NULL"); return MPI_ERR_INVALID; }
    if (!opts) { set_error("opts is NULL"); return MPI_ERR_INVALID; }
    if (opts->op != MPI_OP_FORWARD) {
        set_error("the sample-sharded solve needs opts->op = MPI_OP_FORWARD");
        return MPI_ERR_INVALID;
    }
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_dtype(dtype));
    MPI_TRY(check_traj(traj));
    if (opts->n_iter < 0 || opts->n_cg < 0 || !(opts->nu0 >= 0.0) || !std::isfinite(opts->nu0) ||
        !(opts->clip_pct <= 100.0) || std::isnan(opts->clip_pct)) {
        set_error("invalid PnP options (n_iter %d, n_cg %d, nu0 %g, clip_pct %g)", opts->n_iter,
                  opts->n_cg, opts->nu0, opts->clip_pct);
        return MPI_ERR_INVALID;
    }
    if (!rho_out || (!data && traj->T > 0)) {
        set_error("data or rho_out is NULL");
        return MPI_ERR_INVALID;
    }
    const ModelH m = to_host(model);
    const GridH g = to_host(grid);
    const cudaStream_t st = as_stream(stream);
    return dtype == MPI_F32
               ? pnp_impl<float>(m, g, traj, data, *opts, denoise, user, rho_out, info, st, allreduce, comm_user)
               : pnp_impl<double>(m, g, traj, data, *opts, denoise, user, rho_out, info, st, allreduce, comm_user);
}

int mpi_conv(const mpi_model *model, const mpi_grid_desc *grid, mpi_dtype dtype, const void *in,
             void *out, void *stream)
{
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_dtype(dtype));
    if (!in || !out || in == out) { set_error("in/out NULL or aliased"); return MPI_ERR_INVALID; }
    const ModelH m = to_host(model);
    const GridH g = to_host(grid);
    return dtype == MPI_F32 ? conv_impl<float>(m, g, in, out, as_stream(stream))
                            : conv_impl<double>(m, g, in, out, as_stream(stream));
}

int mpi_conv_component(const mpi_model *model, const mpi_grid_desc *grid, mpi_dtype dtype,
                       int component, const void *in, void *out, void *stream)
{
    MPI_TRY(check_model(model));
    MPI_TRY(check_grid(grid));
    MPI_TRY(check_dtype(dtype));
    if (component < -1 || component > 3) { set_error("component must be in [-1, 3]"); return MPI_ERR_INVALID; }
    if (!in || !out || in == out) { set_error("in/out NULL or aliased"); return MPI_ERR_INVALID; }
    const ModelH m = to_host(model);
    const GridH g = to_host(grid);
    return dtype == MPI_F32 ? conv_impl<float>(m, g, in, out, as_stream(stream), component)
                            : conv_impl<double>(m, g, in, out, as_stream(stream), component);
}

int mpi_denoise_gaussian5(const void *in, void *out, int nx, int ny, mpi_dtype dtype,
                          const double *sigma_dev, void *stream, void *user)
{
    (void)sigma_dev;
    (void)user;
    MPI_TRY(check_dtype(dtype));
    if (nx < 1 || ny < 1 || !in || !out || in == out) {
        set_error("invalid denoiser arguments");
        return MPI_ERR_INVALID;
    }
    return dtype == MPI_F32
               ? launch_gauss5<float>(static_cast<const float *>(in), static_cast<float *>(out), nx, ny, as_stream(stream))
               : launch_gauss5<double>(static_cast<const double *>(in), static_cast<double *>(out), nx, ny, as_stream(stream));
}

}  // extern "C"
