/*
 * FP64 CPU oracle for the equilibrium (Langevin) MPI operators of
 * "Fast Trajectory-Independent Model-Based Reconstruction Algorithm for
 * Multi-Dimensional MPI" (Gapyak, Maerz, Weinmann).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * Everything is IEEE double.  Loops are written in the order of the
 * definitions; the only parallelism is OpenMP over independent outputs, so
 * every output is a sequential sum and the results do not depend on the
 * thread count.
 *
 * Notation (Sec. 2 of the paper):
 *   c[j][i]     particle concentration on the voxel centres
 *               x_ij = (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy), row-major, j = row
 *   r[t][2]     FFP trajectory r(t), v[t][2] its velocity r'(t)
 *   G[2][2]     selection-field gradient (row-major), H(x,t) = G (x - r(t))
 *   beta        1 / (mu0 H_sat), so the Langevin argument is beta |H|
 *   p[k][2]     receive-coil directions, s[k][t] the signal on channel k
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int nx, ny;
    double x0, y0, dx, dy;
} og_grid;

typedef struct {
    double beta;
    double G[4];
    int n_ch;
    double p[4]; /* p[k*2 + m] */
} og_model;

/* ------------------------------------------------------------------------- */
/* Langevin function family (Eq. momentum, with L = coth z - 1/z: the "cosh"
 * printed in the paper is a typo, the Langevin function is coth z - 1/z).
 *
 *   L(z)   = coth z - 1/z
 *   L'(z)  = 1/z^2 - 1/sinh^2 z
 *   L''(z) = -2/z^3 + 2 cosh z / sinh^3 z
 *   a(z)   = L(z)/z                 (transverse eigenvalue of K, Eq. kernel:matrix)
 *   d(z)   = (L'(z) - a(z)) / z^2   (so that K(y) = a I + d y y^T)
 *   e(z)   = L''(z) / z
 *
 * Near z = 0 the closed forms cancel catastrophically, so for z < 2 the
 * oracle sums the Taylor series of coth:
 *   coth z - 1/z = sum_{n>=1} c_n z^(2n-1),  c_n = 2 (-1)^(n+1) zeta(2n) / pi^(2n)
 * (equivalently c_n = 2^(2n) B_2n / (2n)!).  Differentiating term by term:
 *   a  = sum_n c_n u^(n-1),                 L' = sum_n (2n-1) c_n u^(n-1)
 *   d  = sum_{n>=2} (2n-2) c_n u^(n-2),     e  = sum_{n>=2} (2n-1)(2n-2) c_n u^(n-2)
 * with u = z^2.  The series converges for |z| < pi; at z = 2 the ratio of
 * successive terms is 4/pi^2 ~ 0.41, so OG_NS terms reach far below 1e-16.
 */
#define OG_NS 72
#define OG_ZSER 2.0

static double og_c[OG_NS + 1];
static int og_c_ready = 0;

/* zeta(s) for even s >= 4 by direct summation plus the Euler-Maclaurin tail. */
static double og_zeta(int s)
{
    const int K = 1000;
    double acc = 0.0;
    for (int k = K; k >= 1; --k) acc += pow((double)k, -(double)s);
    double Kd = (double)K;
    /* tail sum_{k>K} k^-s ~ int_K^inf x^-s dx - K^-s/2 + s K^-(s+1)/12 */
    acc += pow(Kd, 1.0 - s) / (s - 1.0) - 0.5 * pow(Kd, -(double)s)
         + s * pow(Kd, -(double)s - 1.0) / 12.0;
    return acc;
}

static void og_init_series(void)
{
    if (og_c_ready) return;
    og_c[0] = 0.0;
    og_c[1] = 1.0 / 3.0; /* 2 zeta(2) / pi^2 = 1/3 exactly */
    for (int n = 2; n <= OG_NS; ++n) {
        double sgn = (n % 2 == 0) ? -1.0 : 1.0;
        og_c[n] = 2.0 * sgn * og_zeta(2 * n) / pow(M_PI, 2.0 * n);
    }
    og_c_ready = 1;
}

/* All six functions at one argument z >= 0. */
static void og_langevin6(double z, double *L, double *Lp, double *Lpp,
                         double *a, double *d, double *e)
{
    if (z < OG_ZSER) {
        double u = z * z;
        double sa = 0.0, sl = 0.0, sd = 0.0, se = 0.0;
        for (int n = OG_NS; n >= 1; --n) {
            sa = sa * u + og_c[n];
            sl = sl * u + (2.0 * n - 1.0) * og_c[n];
        }
        for (int n = OG_NS; n >= 2; --n) {
            sd = sd * u + (2.0 * n - 2.0) * og_c[n];
            se = se * u + (2.0 * n - 1.0) * (2.0 * n - 2.0) * og_c[n];
        }
        *a = sa; *Lp = sl; *d = sd; *e = se;
        *L = z * sa; *Lpp = z * se;
        return;
    }
    /* q = exp(-2z); coth z = (1+q)/(1-q); 1/sinh^2 z = 4q/(1-q)^2. */
    double em = expm1(-2.0 * z); /* q - 1, in (-1, 0) */
    double q = exp(-2.0 * z);
    double coth = -(2.0 + em) / em;
    double csch2 = 4.0 * q / (em * em);
    double iz = 1.0 / z;
    *L = coth - iz;
    *Lp = iz * iz - csch2;
    *Lpp = -2.0 * iz * iz * iz + 2.0 * coth * csch2;
    *a = *L * iz;
    *d = (*Lp - *a) * iz * iz;
    *e = *Lpp * iz;
}

/* Vectorised export, for the tests. */
void og_langevin(int64_t n, const double *z, double *L, double *Lp, double *Lpp,
                 double *a, double *d, double *e)
{
    og_init_series();
    for (int64_t k = 0; k < n; ++k)
        og_langevin6(z[k], &L[k], &Lp[k], &Lpp[k], &a[k], &d[k], &e[k]);
}

/* ------------------------------------------------------------------------- */
/* MPI kernel matrix (Eq. kernel:matrix):
 *   K(y) = L'(|y|) yy^T/|y|^2 + L(|y|)/|y| (I - yy^T/|y|^2) = a I + d y y^T.
 * K(0) = I/3.  Returned row-major. */
static void og_K(const double y[2], double K[4])
{
    double z = sqrt(y[0] * y[0] + y[1] * y[1]);
    double L, Lp, Lpp, a, d, e;
    og_langevin6(z, &L, &Lp, &Lpp, &a, &d, &e);
    K[0] = a + d * y[0] * y[0];
    K[1] = d * y[0] * y[1];
    K[2] = d * y[1] * y[0];
    K[3] = a + d * y[1] * y[1];
}

void og_kernel_matrix(int64_t n, const double *y, double *K)
{
    og_init_series();
    for (int64_t k = 0; k < n; ++k) og_K(&y[2 * k], &K[4 * k]);
}

static inline void og_voxel_centre(const og_grid *g, int i, int j, double x[2])
{
    x[0] = g->x0 + (i + 0.5) * g->dx;
    x[1] = g->y0 + (j + 0.5) * g->dy;
}

/* The response of one voxel at x to one trajectory sample (r, v):
 *   J w = beta K(beta G (x - r)) G v,
 * i.e. the Jacobian of H -> L(beta |H|) H/|H| at H = G(x - r), applied to
 * G r' (the time derivative of the magnetisation with the sign of
 * dH/dt = -G r' dropped together with the constant -mu0 m R, as Eq.
 * core:formula does). */
static void og_pair(const og_model *m, const double x[2], const double r[2],
                    const double v[2], double Jw[2])
{
    double dxr[2] = {x[0] - r[0], x[1] - r[1]};
    double H[2] = {m->G[0] * dxr[0] + m->G[1] * dxr[1],
                   m->G[2] * dxr[0] + m->G[3] * dxr[1]};
    double y[2] = {m->beta * H[0], m->beta * H[1]};
    double w[2] = {m->G[0] * v[0] + m->G[1] * v[1],
                   m->G[2] * v[0] + m->G[3] * v[1]};
    double K[4];
    og_K(y, K);
    Jw[0] = m->beta * (K[0] * w[0] + K[1] * w[1]);
    Jw[1] = m->beta * (K[2] * w[0] + K[3] * w[1]);
}

void og_pair_export(const og_model *m, const double *x, const double *r,
                    const double *v, double *Jw)
{
    og_init_series();
    og_pair(m, x, r, v, Jw);
}

/* ------------------------------------------------------------------------- */
/* Forward operator A (Eq. core:formula, discretised on the voxel grid):
 *   s_k(t) = sum_{j,i} c_ij p_k^T J(x_ij, t) w_t.
 * s is [n_ch][T].  Voxels are summed row-major in FP64. */
void og_forward(const og_model *m, const og_grid *g, int64_t T, const double *r,
                const double *v, const double *c, double *s)
{
    og_init_series();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < T; ++t) {
        double acc[2] = {0.0, 0.0};
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double x[2], Jw[2];
                og_voxel_centre(g, i, j, x);
                og_pair(m, x, &r[2 * t], &v[2 * t], Jw);
                double cij = c[(int64_t)j * g->nx + i];
                for (int k = 0; k < m->n_ch; ++k)
                    acc[k] += cij * (m->p[2 * k] * Jw[0] + m->p[2 * k + 1] * Jw[1]);
            }
        for (int k = 0; k < m->n_ch; ++k) s[(int64_t)k * T + t] = acc[k];
    }
}

/* Adjoint A^T at a list of voxels (all voxels when sel == NULL):
 *   g_ij = sum_t sum_k s_k(t) p_k^T J(x_ij, t) w_t, summed over t in order. */
void og_adjoint_sel(const og_model *m, const og_grid *g, int64_t T, const double *r,
                    const double *v, const double *s, int64_t n_sel,
                    const int64_t *sel, double *out)
{
    og_init_series();
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_sel; ++q) {
        int64_t idx = sel ? sel[q] : q;
        int i = (int)(idx % g->nx), j = (int)(idx / g->nx);
        double x[2];
        og_voxel_centre(g, i, j, x);
        double acc = 0.0;
        for (int64_t t = 0; t < T; ++t) {
            double Jw[2];
            og_pair(m, x, &r[2 * t], &v[2 * t], Jw);
            for (int k = 0; k < m->n_ch; ++k)
                acc += s[(int64_t)k * T + t] * (m->p[2 * k] * Jw[0] + m->p[2 * k + 1] * Jw[1]);
        }
        out[q] = acc;
    }
}

void og_adjoint(const og_model *m, const og_grid *g, int64_t T, const double *r,
                const double *v, const double *s, double *out)
{
    og_adjoint_sel(m, g, T, r, v, s, (int64_t)g->nx * g->ny, NULL, out);
}

/* d/dbeta of <gs, A(c; beta)>:
 *   sum_t sum_k gs_k(t) sum_x c_x p_k^T d/dbeta[beta K(beta y0)] w_t,
 * y0 = G(x - r_t).  Writing y = beta y0, z = |y| and using a + z a' = L',
 * 3d + z d' = L''/z:
 *   d/dbeta[beta K(beta y0)] w = L'(z) w + (L''(z)/z) (y.w) y.
 * Per-sample contributions are summed in sample order. */
void og_dbeta(const og_model *m, const og_grid *g, int64_t T, const double *r,
              const double *v, const double *c, const double *gs, double *contrib,
              double *out)
{
    og_init_series();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < T; ++t) {
        double acc = 0.0;
        const double *rt = &r[2 * t], *vt = &v[2 * t];
        double w[2] = {m->G[0] * vt[0] + m->G[1] * vt[1],
                       m->G[2] * vt[0] + m->G[3] * vt[1]};
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double x[2];
                og_voxel_centre(g, i, j, x);
                double dxr[2] = {x[0] - rt[0], x[1] - rt[1]};
                double y[2] = {m->beta * (m->G[0] * dxr[0] + m->G[1] * dxr[1]),
                               m->beta * (m->G[2] * dxr[0] + m->G[3] * dxr[1])};
                double z = sqrt(y[0] * y[0] + y[1] * y[1]);
                double L, Lp, Lpp, a, d, e;
                og_langevin6(z, &L, &Lp, &Lpp, &a, &d, &e);
                double yw = y[0] * w[0] + y[1] * w[1];
                double D[2] = {Lp * w[0] + e * yw * y[0], Lp * w[1] + e * yw * y[1]};
                double cij = c[(int64_t)j * g->nx + i];
                for (int k = 0; k < m->n_ch; ++k)
                    acc += gs[(int64_t)k * T + t] * cij * (m->p[2 * k] * D[0] + m->p[2 * k + 1] * D[1]);
            }
        contrib[t] = acc;
    }
    double tot = 0.0;
    for (int64_t t = 0; t < T; ++t) tot += contrib[t];
    *out = tot;
}

/* sum over all (voxel, sample, channel) of (p_k^T J w)^2: the squared
 * Frobenius norm of the dense matrix of A. */
double og_frob2(const og_model *m, const og_grid *g, int64_t T, const double *r,
                const double *v, double *contrib)
{
    og_init_series();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < T; ++t) {
        double acc = 0.0;
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double x[2], Jw[2];
                og_voxel_centre(g, i, j, x);
                og_pair(m, x, &r[2 * t], &v[2 * t], Jw);
                for (int k = 0; k < m->n_ch; ++k) {
                    double e = m->p[2 * k] * Jw[0] + m->p[2 * k + 1] * Jw[1];
                    acc += e * e;
                }
            }
        contrib[t] = acc;
    }
    double tot = 0.0;
    for (int64_t t = 0; t < T; ++t) tot += contrib[t];
    return tot;
}

/* ------------------------------------------------------------------------- */
/* Cosine interpolation (Eq. first:step; the scheme of the Core Stage).
 * Nodes are the voxel centres.  Along one axis, a position p falls between
 * nodes k and k+1 at fraction f in [0,1]; node k+1 gets weight
 * (1 - cos(pi f))/2 and node k the rest.  Positions outside the node hull are
 * clamped to the nearest edge node.  The 2-D scheme is the tensor product. */
static void og_axis(double p, double p0, double h, int n, int *k0, double *w0, double *w1)
{
    if (n == 1) { *k0 = 0; *w0 = 1.0; *w1 = 0.0; return; }
    double fi = (p - p0) / h - 0.5;       /* continuous node index */
    if (fi <= 0.0) { *k0 = 0; *w0 = 1.0; *w1 = 0.0; return; }
    if (fi >= n - 1) { *k0 = n - 2; *w0 = 0.0; *w1 = 1.0; return; }
    int k = (int)floor(fi);
    if (k > n - 2) k = n - 2;
    double f = fi - k;
    *k0 = k;
    *w1 = 0.5 * (1.0 - cos(M_PI * f));
    *w0 = 1.0 - *w1;
}

/* s_k(t) = sum_m I[Ahat_km](r_t) v_m(t), k = 0, 1.  Ahat is [4][ny][nx] with
 * component index 2k+m.  s is [2][T]. */
void og_interp(const og_grid *g, int64_t T, const double *r, const double *v,
               const double *Ahat, double *s)
{
    int64_t N = (int64_t)g->nx * g->ny;
    for (int64_t t = 0; t < T; ++t) {
        int i0, j0;
        double wx0, wx1, wy0, wy1;
        og_axis(r[2 * t], g->x0, g->dx, g->nx, &i0, &wx0, &wx1);
        og_axis(r[2 * t + 1], g->y0, g->dy, g->ny, &j0, &wy0, &wy1);
        int i1 = (g->nx > 1) ? i0 + 1 : i0, j1 = (g->ny > 1) ? j0 + 1 : j0;
        for (int k = 0; k < 2; ++k) {
            double acc = 0.0;
            for (int mm = 0; mm < 2; ++mm) {
                const double *F = &Ahat[(2 * k + mm) * N];
                double val = wy0 * (wx0 * F[(int64_t)j0 * g->nx + i0] + wx1 * F[(int64_t)j0 * g->nx + i1])
                           + wy1 * (wx0 * F[(int64_t)j1 * g->nx + i0] + wx1 * F[(int64_t)j1 * g->nx + i1]);
                acc += val * v[2 * t + mm];
            }
            s[(int64_t)k * T + t] = acc;
        }
    }
}

/* Exact transpose of og_interp: Ahat_km += weight * v_m(t) * s_k(t), in
 * sample order. */
void og_interp_T(const og_grid *g, int64_t T, const double *r, const double *v,
                 const double *s, double *Ahat)
{
    int64_t N = (int64_t)g->nx * g->ny;
    memset(Ahat, 0, sizeof(double) * 4 * N);
    for (int64_t t = 0; t < T; ++t) {
        int i0, j0;
        double wx0, wx1, wy0, wy1;
        og_axis(r[2 * t], g->x0, g->dx, g->nx, &i0, &wx0, &wx1);
        og_axis(r[2 * t + 1], g->y0, g->dy, g->ny, &j0, &wy0, &wy1);
        int i1 = (g->nx > 1) ? i0 + 1 : i0, j1 = (g->ny > 1) ? j0 + 1 : j0;
        for (int k = 0; k < 2; ++k)
            for (int mm = 0; mm < 2; ++mm) {
                double coef = s[(int64_t)k * T + t] * v[2 * t + mm];
                double *F = &Ahat[(2 * k + mm) * N];
                F[(int64_t)j0 * g->nx + i0] += wy0 * wx0 * coef;
                F[(int64_t)j0 * g->nx + i1] += wy0 * wx1 * coef;
                F[(int64_t)j1 * g->nx + i0] += wy1 * wx0 * coef;
                F[(int64_t)j1 * g->nx + i1] += wy1 * wx1 * coef;
            }
    }
}

/* 5-point discrete Laplacian with replicated (Neumann) boundary on one
 * [ny][nx] field: the regulariser of the Core Stage (Eq. first:step). */
void og_laplacian(const og_grid *g, const double *f, double *out)
{
    int nx = g->nx, ny = g->ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int im = i > 0 ? i - 1 : 0, ip = i < nx - 1 ? i + 1 : nx - 1;
            int jm = j > 0 ? j - 1 : 0, jp = j < ny - 1 ? j + 1 : ny - 1;
            double c0 = f[(int64_t)j * nx + i];
            out[(int64_t)j * nx + i] = f[(int64_t)j * nx + im] + f[(int64_t)j * nx + ip]
                                     + f[(int64_t)jm * nx + i] + f[(int64_t)jp * nx + i] - 4.0 * c0;
        }
}

/* ------------------------------------------------------------------------- */
/* Sampled trace kernel (Eq. convolution:trace / kernel:trace), read with the
 * resolution scaling and the gradient that multiply v in the forward model:
 *   kappa_G(y) = beta tr(K(beta G y) G),
 * sampled on all voxel offsets y = (ii dx, jj dy), |ii| < nx, |jj| < ny.
 * kern is [(2ny-1)][(2nx-1)], offset (0,0) at (ny-1, nx-1). */
/* comp < 0: the trace kernel above.  comp = 2a + b: the entry (a, b) of
 * beta K(beta G y) G instead; with only channel a measured (Sec. 3.6) the
 * deconvolution uses the (a, a) entry, the kernel of the diagonal
 * core-operator component that the single-channel Core Stage recovers. */
void og_conv_kernel_component(const og_model *m, const og_grid *g, int comp, double *kern)
{
    og_init_series();
    int KX = 2 * g->nx - 1, KY = 2 * g->ny - 1;
    for (int jj = 0; jj < KY; ++jj)
        for (int ii = 0; ii < KX; ++ii) {
            double off[2] = {(ii - (g->nx - 1)) * g->dx, (jj - (g->ny - 1)) * g->dy};
            double y[2] = {m->beta * (m->G[0] * off[0] + m->G[1] * off[1]),
                           m->beta * (m->G[2] * off[0] + m->G[3] * off[1])};
            double K[4];
            og_K(y, K);
            /* (K G)_ab = sum_c K_ac G_cb */
            double KG[4] = {K[0] * m->G[0] + K[1] * m->G[2], K[0] * m->G[1] + K[1] * m->G[3],
                            K[2] * m->G[0] + K[3] * m->G[2], K[2] * m->G[1] + K[3] * m->G[3]};
            double val = comp < 0 ? KG[0] + KG[3] : KG[comp];
            kern[(int64_t)jj * KX + ii] = m->beta * val;
        }
}

void og_conv_kernel(const og_model *m, const og_grid *g, double *kern)
{
    og_conv_kernel_component(m, g, -1, kern);
}

/* Linear (zero-padded) convolution with the sampled kernel (the matrix C_h of
 * Eq. dec:sub:tik):  out_ij = sum_{j'i'} kappa(x_ij - x_i'j') in_i'j'. */
void og_conv(const og_grid *g, const double *kern, const double *in, double *out)
{
    int nx = g->nx, ny = g->ny, KX = 2 * nx - 1;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double acc = 0.0;
            for (int jq = 0; jq < ny; ++jq)
                for (int iq = 0; iq < nx; ++iq)
                    acc += kern[(int64_t)(j - jq + ny - 1) * KX + (i - iq + nx - 1)]
                         * in[(int64_t)jq * nx + iq];
            out[(int64_t)j * nx + i] = acc;
        }
}

/* Host threads of the parallel loops (all outputs are independent, so the
   count changes no result, only the wall-clock time of a timing run). */
void og_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int og_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ========================================================================= */
/* Three-dimensional field-free point (the model of Sec. 2 with n = 3).
 *
 * The kernel matrix of Eq. kernel:matrix is stated for y in R^n; with n = 3
 * it is the 3x3 matrix K(y) = a I + d y y^T with the same scalars a, d.  The
 * signal of Eq. core:formula becomes
 *   s_k(t) = sum_{l,j,i} c_lji p_k^T beta K(beta G (x_lji - r_t)) G v_t
 * for a 3x3 gradient G (the paper's standard choice G = diag(-1, -1, 2) in
 * units of T/(mu0 m)), r_t, v_t in R^3 and up to three receive directions p_k.
 * The trace kernel of Eq. kernel:trace carries (n - 1) = 2:
 *   tr K(y) = L'(|y|) + 2 L(|y|)/|y|.
 * Voxel centres x_lji = (x0 + (i+1/2)dx, y0 + (j+1/2)dy, z0 + (l+1/2)dz);
 * arrays are [nz][ny][nx], r and v [T][3], s [n_ch][T].
 */
typedef struct {
    int nx, ny, nz;
    double x0, y0, z0, dx, dy, dz;
} og_grid3;

typedef struct {
    double beta;
    double G[9];
    int n_ch;
    double p[9]; /* p[k*3 + m] */
} og_model3;

static void og_K3(const double y[3], double K[9])
{
    double z = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    double L, Lp, Lpp, a, d, e;
    og_langevin6(z, &L, &Lp, &Lpp, &a, &d, &e);
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) K[3 * r + q] = (r == q ? a : 0.0) + d * y[r] * y[q];
}

void og_kernel_matrix3(int64_t n, const double *y, double *K)
{
    og_init_series();
    for (int64_t k = 0; k < n; ++k) og_K3(&y[3 * k], &K[9 * k]);
}

static inline void og_voxel_centre3(const og_grid3 *g, int i, int j, int l, double x[3])
{
    x[0] = g->x0 + (i + 0.5) * g->dx;
    x[1] = g->y0 + (j + 0.5) * g->dy;
    x[2] = g->z0 + (l + 0.5) * g->dz;
}

static void og_matvec3(const double M[9], const double u[3], double out[3])
{
    for (int r = 0; r < 3; ++r) out[r] = M[3 * r] * u[0] + M[3 * r + 1] * u[1] + M[3 * r + 2] * u[2];
}

/* J w = beta K(beta G (x - r)) G v, as og_pair in three dimensions. */
static void og_pair3(const og_model3 *m, const double x[3], const double r[3],
                     const double v[3], double Jw[3])
{
    double dxr[3] = {x[0] - r[0], x[1] - r[1], x[2] - r[2]};
    double H[3], w[3], K[9], Kw[3];
    og_matvec3(m->G, dxr, H);
    double y[3] = {m->beta * H[0], m->beta * H[1], m->beta * H[2]};
    og_matvec3(m->G, v, w);
    og_K3(y, K);
    og_matvec3(K, w, Kw);
    for (int q = 0; q < 3; ++q) Jw[q] = m->beta * Kw[q];
}

void og_pair3_export(const og_model3 *m, const double *x, const double *r, const double *v,
                     double *Jw)
{
    og_init_series();
    og_pair3(m, x, r, v, Jw);
}

static inline double og_pdot3(const og_model3 *m, int k, const double Jw[3])
{
    return m->p[3 * k] * Jw[0] + m->p[3 * k + 1] * Jw[1] + m->p[3 * k + 2] * Jw[2];
}

/* s_k(t) = sum over voxels (l, j, i in row-major order) of c p_k^T J w. */
void og_forward3(const og_model3 *m, const og_grid3 *g, int64_t T, const double *r,
                 const double *v, const double *c, double *s)
{
    og_init_series();
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < T; ++t) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int l = 0; l < g->nz; ++l)
            for (int j = 0; j < g->ny; ++j)
                for (int i = 0; i < g->nx; ++i) {
                    double x[3], Jw[3];
                    og_voxel_centre3(g, i, j, l, x);
                    og_pair3(m, x, &r[3 * t], &v[3 * t], Jw);
                    double cv = c[((int64_t)l * g->ny + j) * g->nx + i];
                    for (int k = 0; k < m->n_ch; ++k) acc[k] += cv * og_pdot3(m, k, Jw);
                }
        for (int k = 0; k < m->n_ch; ++k) s[(int64_t)k * T + t] = acc[k];
    }
}

/* A^T at a list of voxels (flat index (l ny + j) nx + i; all when sel == NULL). */
void og_adjoint3_sel(const og_model3 *m, const og_grid3 *g, int64_t T, const double *r,
                     const double *v, const double *s, int64_t n_sel, const int64_t *sel,
                     double *out)
{
    og_init_series();
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < n_sel; ++q) {
        int64_t idx = sel ? sel[q] : q;
        int i = (int)(idx % g->nx), j = (int)((idx / g->nx) % g->ny), l = (int)(idx / ((int64_t)g->nx * g->ny));
        double x[3];
        og_voxel_centre3(g, i, j, l, x);
        double acc = 0.0;
        for (int64_t t = 0; t < T; ++t) {
            double Jw[3];
            og_pair3(m, x, &r[3 * t], &v[3 * t], Jw);
            for (int k = 0; k < m->n_ch; ++k) acc += s[(int64_t)k * T + t] * og_pdot3(m, k, Jw);
        }
        out[q] = acc;
    }
}

void og_adjoint3(const og_model3 *m, const og_grid3 *g, int64_t T, const double *r,
                 const double *v, const double *s, double *out)
{
    og_adjoint3_sel(m, g, T, r, v, s, (int64_t)g->nx * g->ny * g->nz, NULL, out);
}

/* ||A||_F^2 = sum over (voxel, sample, channel) of (p_k^T J w)^2. */
double og_frob2_3(const og_model3 *m, const og_grid3 *g, int64_t T, const double *r,
                  const double *v)
{
    og_init_series();
    const int64_t N = (int64_t)g->nx * g->ny * g->nz;
    double tot = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : tot)
    for (int64_t idx = 0; idx < N; ++idx) {
        int i = (int)(idx % g->nx), j = (int)((idx / g->nx) % g->ny), l = (int)(idx / ((int64_t)g->nx * g->ny));
        double x[3];
        og_voxel_centre3(g, i, j, l, x);
        double acc = 0.0;
        for (int64_t t = 0; t < T; ++t) {
            double Jw[3];
            og_pair3(m, x, &r[3 * t], &v[3 * t], Jw);
            for (int k = 0; k < m->n_ch; ++k) {
                double e = og_pdot3(m, k, Jw);
                acc += e * e;
            }
        }
        tot += acc;
    }
    return tot;
}

/* Sampled trace kernel in three dimensions, kappa_G(y) = beta tr(K(beta G y) G)
 * on all voxel offsets; kern is [(2nz-1)][(2ny-1)][(2nx-1)] with offset 0 at
 * (nz-1, ny-1, nx-1).  For G = g I it is beta g (L' + 2 L/z), z = beta g |y|:
 * Eq. kernel:trace with n - 1 = 2. */
void og_conv_kernel3(const og_model3 *m, const og_grid3 *g, double *kern)
{
    og_init_series();
    int KX = 2 * g->nx - 1, KY = 2 * g->ny - 1, KZ = 2 * g->nz - 1;
    for (int ll = 0; ll < KZ; ++ll)
        for (int jj = 0; jj < KY; ++jj)
            for (int ii = 0; ii < KX; ++ii) {
                double off[3] = {(ii - (g->nx - 1)) * g->dx, (jj - (g->ny - 1)) * g->dy,
                                 (ll - (g->nz - 1)) * g->dz};
                double H[3], K[9];
                og_matvec3(m->G, off, H);
                double y[3] = {m->beta * H[0], m->beta * H[1], m->beta * H[2]};
                og_K3(y, K);
                /* tr(K G) = sum_{a,c} K_ac G_ca */
                double tr = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int q = 0; q < 3; ++q) tr += K[3 * a + q] * m->G[3 * q + a];
                kern[((int64_t)ll * KY + jj) * KX + ii] = m->beta * tr;
            }
}

/* Linear (zero-padded) 3-D convolution with the sampled kernel. */
void og_conv3(const og_grid3 *g, const double *kern, const double *in, double *out)
{
    int nx = g->nx, ny = g->ny, nz = g->nz, KX = 2 * nx - 1, KY = 2 * ny - 1;
#pragma omp parallel for schedule(static)
    for (int l = 0; l < nz; ++l)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double acc = 0.0;
                for (int lq = 0; lq < nz; ++lq)
                    for (int jq = 0; jq < ny; ++jq)
                        for (int iq = 0; iq < nx; ++iq)
                            acc += kern[((int64_t)(l - lq + nz - 1) * KY + (j - jq + ny - 1)) * KX +
                                        (i - iq + nx - 1)] *
                                   in[((int64_t)lq * ny + jq) * nx + iq];
                out[((int64_t)l * ny + j) * nx + i] = acc;
            }
}

/* ------------------------------------------------------------------------- */
/* Core Stage in three dimensions (Eq. first:step with n = 3).  The core
 * operator at a point is the n_ch x 3 matrix Ahat_km (receive channel k,
 * velocity component m); the measurement is
 *   s_k(t) = sum_m I[Ahat_km](r_t) v_m(t),
 * with I the tensor product of the one-dimensional cosine interpolation of
 * og_axis along x, y and z (nodes at the voxel centres, clamped outside the
 * node hull).  Ahat is [n_ch*3][nz][ny][nx] with component index 3k+m; s is
 * [n_ch][T]; r and v are [T][3]. */
void og_interp3(const og_grid3 *g, int n_ch, int64_t T, const double *r, const double *v,
                const double *Ahat, double *s)
{
    int64_t N = (int64_t)g->nx * g->ny * g->nz;
    for (int64_t t = 0; t < T; ++t) {
        int ix[2], iy[2], iz[2];
        double wx[2], wy[2], wz[2];
        og_axis(r[3 * t], g->x0, g->dx, g->nx, &ix[0], &wx[0], &wx[1]);
        og_axis(r[3 * t + 1], g->y0, g->dy, g->ny, &iy[0], &wy[0], &wy[1]);
        og_axis(r[3 * t + 2], g->z0, g->dz, g->nz, &iz[0], &wz[0], &wz[1]);
        ix[1] = g->nx > 1 ? ix[0] + 1 : ix[0];
        iy[1] = g->ny > 1 ? iy[0] + 1 : iy[0];
        iz[1] = g->nz > 1 ? iz[0] + 1 : iz[0];
        for (int k = 0; k < n_ch; ++k) {
            double acc = 0.0;
            for (int mm = 0; mm < 3; ++mm) {
                const double *F = &Ahat[(3 * k + mm) * N];
                double val = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a)
                            val += wz[c] * wy[b] * wx[a] *
                                   F[((int64_t)iz[c] * g->ny + iy[b]) * g->nx + ix[a]];
                acc += val * v[3 * t + mm];
            }
            s[(int64_t)k * T + t] = acc;
        }
    }
}

/* Exact transpose of og_interp3, accumulated in sample order. */
void og_interp3_T(const og_grid3 *g, int n_ch, int64_t T, const double *r, const double *v,
                  const double *s, double *Ahat)
{
    int64_t N = (int64_t)g->nx * g->ny * g->nz;
    memset(Ahat, 0, sizeof(double) * 3 * n_ch * N);
    for (int64_t t = 0; t < T; ++t) {
        int ix[2], iy[2], iz[2];
        double wx[2], wy[2], wz[2];
        og_axis(r[3 * t], g->x0, g->dx, g->nx, &ix[0], &wx[0], &wx[1]);
        og_axis(r[3 * t + 1], g->y0, g->dy, g->ny, &iy[0], &wy[0], &wy[1]);
        og_axis(r[3 * t + 2], g->z0, g->dz, g->nz, &iz[0], &wz[0], &wz[1]);
        ix[1] = g->nx > 1 ? ix[0] + 1 : ix[0];
        iy[1] = g->ny > 1 ? iy[0] + 1 : iy[0];
        iz[1] = g->nz > 1 ? iz[0] + 1 : iz[0];
        for (int k = 0; k < n_ch; ++k)
            for (int mm = 0; mm < 3; ++mm) {
                double coef = s[(int64_t)k * T + t] * v[3 * t + mm];
                double *F = &Ahat[(3 * k + mm) * N];
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a)
                            F[((int64_t)iz[c] * g->ny + iy[b]) * g->nx + ix[a]] +=
                                wz[c] * wy[b] * wx[a] * coef;
            }
    }
}

/* 7-point discrete Laplacian with replicated boundary on one [nz][ny][nx]
 * volume (the regulariser of Eq. first:step in three dimensions). */
void og_laplacian3(const og_grid3 *g, const double *f, double *out)
{
    int nx = g->nx, ny = g->ny, nz = g->nz;
    for (int l = 0; l < nz; ++l)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int im = i > 0 ? i - 1 : 0, ip = i < nx - 1 ? i + 1 : nx - 1;
                int jm = j > 0 ? j - 1 : 0, jp = j < ny - 1 ? j + 1 : ny - 1;
                int lm = l > 0 ? l - 1 : 0, lp = l < nz - 1 ? l + 1 : nz - 1;
#define OG_AT(ll, jj, ii) f[((int64_t)(ll) * ny + (jj)) * nx + (ii)]
                out[((int64_t)l * ny + j) * nx + i] =
                    OG_AT(l, j, im) + OG_AT(l, j, ip) + OG_AT(l, jm, i) + OG_AT(l, jp, i) +
                    OG_AT(lm, j, i) + OG_AT(lp, j, i) - 6.0 * OG_AT(l, j, i);
#undef OG_AT
            }
}

/* ------------------------------------------------------------------------- */
/* Grid-scaled forms (the continuous reading of Eq. first:step's regulariser
 * and of the deconvolution kernel).
 *
 * The Laplacian of a function sampled on the nodes, replicated boundary:
 *   (f(i-1) - 2 f(i) + f(i+1)) / dx^2 + (f(j-1) - 2 f(j) + f(j+1)) / dy^2
 * (and / dz^2 in three dimensions); with dx = dy = h it is the stencil of
 * og_laplacian divided by h^2. */
void og_laplacian_h(const og_grid *g, const double *f, double *out)
{
    int nx = g->nx, ny = g->ny;
    double cx = 1.0 / (g->dx * g->dx), cy = 1.0 / (g->dy * g->dy);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int im = i > 0 ? i - 1 : 0, ip = i < nx - 1 ? i + 1 : nx - 1;
            int jm = j > 0 ? j - 1 : 0, jp = j < ny - 1 ? j + 1 : ny - 1;
            double c0 = f[(int64_t)j * nx + i];
            out[(int64_t)j * nx + i] =
                cx * (f[(int64_t)j * nx + im] - 2.0 * c0 + f[(int64_t)j * nx + ip]) +
                cy * (f[(int64_t)jm * nx + i] - 2.0 * c0 + f[(int64_t)jp * nx + i]);
        }
}

void og_laplacian3_h(const og_grid3 *g, const double *f, double *out)
{
    int nx = g->nx, ny = g->ny, nz = g->nz;
    double cx = 1.0 / (g->dx * g->dx), cy = 1.0 / (g->dy * g->dy), cz = 1.0 / (g->dz * g->dz);
    for (int l = 0; l < nz; ++l)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int im = i > 0 ? i - 1 : 0, ip = i < nx - 1 ? i + 1 : nx - 1;
                int jm = j > 0 ? j - 1 : 0, jp = j < ny - 1 ? j + 1 : ny - 1;
                int lm = l > 0 ? l - 1 : 0, lp = l < nz - 1 ? l + 1 : nz - 1;
#define OG_AT(ll, jj, ii) f[((int64_t)(ll) * ny + (jj)) * nx + (ii)]
                double c0 = OG_AT(l, j, i);
                out[((int64_t)l * ny + j) * nx + i] = cx * (OG_AT(l, j, im) - 2.0 * c0 + OG_AT(l, j, ip)) +
                                                      cy * (OG_AT(l, jm, i) - 2.0 * c0 + OG_AT(l, jp, i)) +
                                                      cz * (OG_AT(lm, j, i) - 2.0 * c0 + OG_AT(lp, j, i));
#undef OG_AT
            }
}

/* The kernel of the gradient-weighted trace tr(Ahat G^-1): since
 * Ahat = beta K(beta G .) G * c, tr(Ahat G^-1) = (beta tr K(beta G y)) * c,
 * sampled on all voxel offsets like og_conv_kernel.  tr K = L' + (n-1) L/z
 * is positive, whatever the signs of G. */
void og_conv_kernel_trK(const og_model *m, const og_grid *g, double *kern)
{
    og_init_series();
    int KX = 2 * g->nx - 1, KY = 2 * g->ny - 1;
    for (int jj = 0; jj < KY; ++jj)
        for (int ii = 0; ii < KX; ++ii) {
            double off[2] = {(ii - (g->nx - 1)) * g->dx, (jj - (g->ny - 1)) * g->dy};
            double y[2] = {m->beta * (m->G[0] * off[0] + m->G[1] * off[1]),
                           m->beta * (m->G[2] * off[0] + m->G[3] * off[1])};
            double K[4];
            og_K(y, K);
            kern[(int64_t)jj * KX + ii] = m->beta * (K[0] + K[3]);
        }
}

void og_conv_kernel3_trK(const og_model3 *m, const og_grid3 *g, double *kern)
{
    og_init_series();
    int KX = 2 * g->nx - 1, KY = 2 * g->ny - 1, KZ = 2 * g->nz - 1;
    for (int ll = 0; ll < KZ; ++ll)
        for (int jj = 0; jj < KY; ++jj)
            for (int ii = 0; ii < KX; ++ii) {
                double off[3] = {(ii - (g->nx - 1)) * g->dx, (jj - (g->ny - 1)) * g->dy,
                                 (ll - (g->nz - 1)) * g->dz};
                double H[3], K[9];
                og_matvec3(m->G, off, H);
                double y[3] = {m->beta * H[0], m->beta * H[1], m->beta * H[2]};
                og_K3(y, K);
                kern[((int64_t)ll * KY + jj) * KX + ii] = m->beta * (K[0] + K[4] + K[8]);
            }
}
