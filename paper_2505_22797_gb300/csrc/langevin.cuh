// Langevin-kernel scalars for the pair evaluator, in FP32 and FP64.
//
// With L(z) = coth z - 1/z (Eq. momentum) the MPI kernel of Eq. kernel:matrix
// regroups as K(y) = a(z) I + d(z) y y^T, z = |y|, with
//     a = L(z)/z,   d = (L'(z) - a)/z^2.
// The beta-derivative of beta K(beta y0) needs
//     L'(z) = 1/z^2 - 1/sinh^2 z,   e = L''(z)/z = -2/z^4 + 2 coth z csch^2 z / z.
// All four are even in z, so they are evaluated from u = z^2.
//
// Far from the FFP the closed forms are used with q = exp(-2z):
//     coth z = (1+q)/(1-q),   csch^2 z = 4q/(1-q)^2.
// Near it they cancel catastrophically (coth z - 1/z at z = 0.01 keeps only
// ~2 correct FP32 digits), so below a switch point the Taylor series of
// coth, coth z - 1/z = sum_n c_n z^(2n-1), c_n = 2^(2n) B_2n/(2n)!, is summed
// term by term in u:
//     a  = sum_{n>=0} c_{n+1} u^n              L' = sum (2n+1) c_{n+1} u^n
//     d  = sum_{n>=0} (2n+2) c_{n+2} u^n       e  = sum (2n+2)(2n+3) c_{n+2} u^n
// The c_n below are the exact rationals of that series.
#pragma once

#include "common.cuh"

namespace mpi {

// Taylor coefficients c_n of coth z - 1/z, n = 1..14 (exact rationals).
#define MPI_C1 (1.0 / 3.0)
#define MPI_C2 (-1.0 / 45.0)
#define MPI_C3 (2.0 / 945.0)
#define MPI_C4 (-1.0 / 4725.0)
#define MPI_C5 (2.0 / 93555.0)
#define MPI_C6 (-1382.0 / 638512875.0)
#define MPI_C7 (4.0 / 18243225.0)
#define MPI_C8 (-3617.0 / 162820783125.0)
#define MPI_C9 (87734.0 / 38979295480125.0)
#define MPI_C10 (-349222.0 / 1531329465290625.0)
#define MPI_C11 (310732.0 / 13447856940643125.0)
#define MPI_C12 (-472728182.0 / 201919571963756521875.0)
#define MPI_C13 (2631724.0 / 11094481976030578125.0)
#define MPI_C14 (-13571120588.0 / 564653660170076273671875.0)

// FP32: series for u < 1 (z < 1).  Eight terms leave a truncation error of
// c_9 u^8 / a ~ 7e-9 relative in a and 1e-7 in d at u = 1; above z = 1 the
// closed form's cancellation costs at most ~5 bits.
constexpr float kNearU32 = 1.0f;
// FP64: series for u < 0.25 (z < 0.5); 14 terms reach (0.25/pi^2)^14 ~ 5e-23.
constexpr double kNearU64 = 0.25;

// Far from the FFP, q = exp(-2z) drops below the working precision and the
// closed forms reduce to their asymptotic parts (coth z -> 1, csch^2 z -> 0):
//     a = 1/z - 1/z^2,   d = (2/z^2 - 1/z)/z^2,   L' = 1/z^2,   e = -2/z^4.
// The terms dropped are about 2q relative in a, 4 z q in d, 4 z^2 q in L'
// and 4 z^3 q in e.  With z >= 12 (u >= 144) a and d lose less than 2e-9
// relative; the beta-derivative pair (L', e) uses z >= 14 (u >= 196), where
// both lose less than 8e-9: the reduced forms are exact to FP32 there.  FP64
// uses z >= 21 / 24 (dropped terms below 5e-17 / 8e-17).  One XU operation
// (rsqrt) instead of three.
constexpr float kVfarU32 = 144.0f, kVfarU32Beta = 196.0f;
constexpr double kVfarU64 = 441.0, kVfarU64Beta = 576.0;

#ifdef __CUDACC__

template <typename R> struct Lang;

template <> struct Lang<float> {
    static constexpr float near_u = kNearU32;
    static constexpr float vfar_u = kVfarU32, vfar_u_beta = kVfarU32Beta;

    // 1/z for the asymptotic forms.
    static __device__ __forceinline__ float iz_vfar(float u) { return rsqrt_approx(u); }
    // a, d for u >= vfar_u (asymptotic form, exact to FP32 there).
    static __device__ __forceinline__ void ad_vfar(float u, float &a, float &d)
    {
        const float iz = rsqrt_approx(u);
        const float iz2 = iz * iz;
        a = iz - iz2;
        d = fmaf(iz2, 2.0f, -iz) * iz2;
    }
    // L', e = L''/z for u >= vfar_u_beta.
    static __device__ __forceinline__ void le_vfar(float u, float &lp, float &e)
    {
        const float iz = rsqrt_approx(u);
        lp = iz * iz;
        e = -2.0f * lp * lp;
    }

    // a, d by the closed form (valid for u >= near_u; any u > 0 is finite).
    static __device__ __forceinline__ void ad_far(float u, float &a, float &d)
    {
        const float iz = rsqrt_approx(u);
        const float z = u * iz;
        // q4 = 4 exp(-2z) = 2^(2 - 2 z log2 e)
        const float q4 = ex2_approx(fmaf(z, -2.8853900817779268f, 2.0f));
        const float rr = rcp_approx(fmaf(q4, -0.25f, 1.0f));  // 1/(1-q)
        const float iz2 = iz * iz;
        const float qr4 = q4 * rr;                 // 4q/(1-q)
        const float coth = fmaf(qr4, 0.25f, rr);   // (1+q)/(1-q)
        a = fmaf(coth, iz, -iz2);                  // coth/z - 1/z^2
        const float lp = fmaf(-qr4, rr, iz2);      // 1/z^2 - csch^2
        d = (lp - a) * iz2;
    }
    static __device__ __forceinline__ void ad_near(float u, float &a, float &d)
    {
        a = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, float(MPI_C8), float(MPI_C7)),
            float(MPI_C6)), float(MPI_C5)), float(MPI_C4)), float(MPI_C3)), float(MPI_C2)), float(MPI_C1));
        d = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, float(16.0 * MPI_C9),
            float(14.0 * MPI_C8)), float(12.0 * MPI_C7)), float(10.0 * MPI_C6)), float(8.0 * MPI_C5)),
            float(6.0 * MPI_C4)), float(4.0 * MPI_C3)), float(2.0 * MPI_C2));
    }
    // L', e = L''/z by the closed form.
    static __device__ __forceinline__ void le_far(float u, float &lp, float &e)
    {
        const float iz = rsqrt_approx(u);
        const float z = u * iz;
        const float q4 = ex2_approx(fmaf(z, -2.8853900817779268f, 2.0f));
        const float rr = rcp_approx(fmaf(q4, -0.25f, 1.0f));
        const float iz2 = iz * iz;
        const float qr4 = q4 * rr;
        const float coth = fmaf(qr4, 0.25f, rr);
        const float csch2 = qr4 * rr;
        lp = iz2 - csch2;
        // e = (2 coth csch2 - 2/z^3)/z = 2 iz (coth csch2 - iz iz2)
        e = 2.0f * iz * fmaf(coth, csch2, -iz * iz2);
    }
    static __device__ __forceinline__ void le_near(float u, float &lp, float &e)
    {
        lp = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, float(15.0 * MPI_C8),
            float(13.0 * MPI_C7)), float(11.0 * MPI_C6)), float(9.0 * MPI_C5)), float(7.0 * MPI_C4)),
            float(5.0 * MPI_C3)), float(3.0 * MPI_C2)), float(MPI_C1));
        e = fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, fmaf(u, float(16.0 * 17.0 * MPI_C9),
            float(14.0 * 15.0 * MPI_C8)), float(12.0 * 13.0 * MPI_C7)), float(10.0 * 11.0 * MPI_C6)),
            float(8.0 * 9.0 * MPI_C5)), float(6.0 * 7.0 * MPI_C4)), float(4.0 * 5.0 * MPI_C3)),
            float(2.0 * 3.0 * MPI_C2));
    }
};

// 1/sqrt(u) in FP64 by Newton's method for f(y) = 1/y^2 - u (the classical
// inverse-square-root iteration y <- y + y (1 - u y^2)/2), started from the
// FP32 hardware estimate: each step squares the relative error (2^-22 ->
// ~2^-43 -> below FP64 rounding), with FMAs only.  Valid for u in the FP32
// normal range (the FP64 closed form uses it for u >= 1/4, the asymptotic
// form for u >= 441).
__device__ __forceinline__ double rsqrt_newton(double u)
{
    double y = double(rsqrt_approx(float(u)));
    double h = fma(-u * y, y, 1.0);
    y = fma(0.5 * y, h, y);
    h = fma(-u * y, y, 1.0);
    return fma(0.5 * y, h, y);
}

template <> struct Lang<double> {
    static constexpr double near_u = kNearU64;
    static constexpr double vfar_u = kVfarU64, vfar_u_beta = kVfarU64Beta;

    static __device__ __forceinline__ double iz_vfar(double u) { return rsqrt_newton(u); }
    static __device__ __forceinline__ void ad_vfar(double u, double &a, double &d)
    {
        const double iz = rsqrt_newton(u), iz2 = iz * iz;
        a = iz - iz2;
        d = fma(iz2, 2.0, -iz) * iz2;
    }
    static __device__ __forceinline__ void le_vfar(double u, double &lp, double &e)
    {
        const double iz = rsqrt_newton(u);
        lp = iz * iz;
        e = -2.0 * lp * lp;
    }

    // coth z and csch^2 z from q = exp(-2z) for u >= near_u: there z >= 1/2,
    // so q <= 1/e and 1 - q >= 0.63 carries no cancellation (no expm1
    // needed); one division, 1/(1 - q), serves both.
    static __device__ __forceinline__ void coth_csch2(double z, double &coth, double &csch2)
    {
        const double q = exp(-2.0 * z);
        const double r = 1.0 / (1.0 - q);
        coth = (1.0 + q) * r;
        csch2 = 4.0 * q * r * r;
    }
    static __device__ __forceinline__ void ad_far(double u, double &a, double &d)
    {
        const double iz = rsqrt_newton(u), z = u * iz, iz2 = iz * iz;
        double coth, csch2;
        coth_csch2(z, coth, csch2);
        a = coth * iz - iz2;
        d = ((iz2 - csch2) - a) * iz2;
    }
    static __device__ __forceinline__ void ad_near(double u, double &a, double &d)
    {
        a = fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u,
            fma(u, MPI_C14, MPI_C13), MPI_C12), MPI_C11), MPI_C10), MPI_C9), MPI_C8), MPI_C7),
            MPI_C6), MPI_C5), MPI_C4), MPI_C3), MPI_C2), MPI_C1);
        d = fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u,
            fma(u, 26.0 * MPI_C14, 24.0 * MPI_C13), 22.0 * MPI_C12), 20.0 * MPI_C11),
            18.0 * MPI_C10), 16.0 * MPI_C9), 14.0 * MPI_C8), 12.0 * MPI_C7), 10.0 * MPI_C6),
            8.0 * MPI_C5), 6.0 * MPI_C4), 4.0 * MPI_C3), 2.0 * MPI_C2);
    }
    static __device__ __forceinline__ void le_far(double u, double &lp, double &e)
    {
        const double iz = rsqrt_newton(u), z = u * iz, iz2 = iz * iz;
        double coth, csch2;
        coth_csch2(z, coth, csch2);
        lp = iz2 - csch2;
        e = 2.0 * iz * (coth * csch2 - iz * iz2);
    }
    static __device__ __forceinline__ void le_near(double u, double &lp, double &e)
    {
        lp = fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u,
             fma(u, 27.0 * MPI_C14, 25.0 * MPI_C13), 23.0 * MPI_C12), 21.0 * MPI_C11),
             19.0 * MPI_C10), 17.0 * MPI_C9), 15.0 * MPI_C8), 13.0 * MPI_C7), 11.0 * MPI_C6),
             9.0 * MPI_C5), 7.0 * MPI_C4), 5.0 * MPI_C3), 3.0 * MPI_C2), MPI_C1);
        e = fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u, fma(u,
            fma(u, 26.0 * 27.0 * MPI_C14, 24.0 * 25.0 * MPI_C13), 22.0 * 23.0 * MPI_C12),
            20.0 * 21.0 * MPI_C11), 18.0 * 19.0 * MPI_C10), 16.0 * 17.0 * MPI_C9),
            14.0 * 15.0 * MPI_C8), 12.0 * 13.0 * MPI_C7), 10.0 * 11.0 * MPI_C6),
            8.0 * 9.0 * MPI_C5), 6.0 * 7.0 * MPI_C4), 4.0 * 5.0 * MPI_C3), 2.0 * 3.0 * MPI_C2);
    }
};

// Per-pair selection with a per-pair branch (used where pairs near the FFP are
// possible).  For FP32 the caller guarantees warp-uniform control flow, so the
// near branch runs for the whole warp only when one of its lanes needs it.
template <typename R, bool DBETA>
__device__ __forceinline__ void lang_checked(R u, R &f1, R &f2)
{
    if constexpr (sizeof(R) == 4) {
        const bool near = u < Lang<R>::near_u;
        const R uf = near ? R(1) : u;  // keep the closed form finite
        if constexpr (DBETA) Lang<R>::le_far(uf, f1, f2);
        else Lang<R>::ad_far(uf, f1, f2);
        if (__any_sync(0xffffffffu, near)) {
            R g1, g2;
            if constexpr (DBETA) Lang<R>::le_near(u, g1, g2);
            else Lang<R>::ad_near(u, g1, g2);
            f1 = near ? g1 : f1;
            f2 = near ? g2 : f2;
        }
    } else {
        if (u < Lang<R>::near_u) {
            if constexpr (DBETA) Lang<R>::le_near(u, f1, f2);
            else Lang<R>::ad_near(u, f1, f2);
        } else {
            if constexpr (DBETA) Lang<R>::le_far(u, f1, f2);
            else Lang<R>::ad_far(u, f1, f2);
        }
    }
}

template <typename R, bool DBETA>
__device__ __forceinline__ void lang_far(R u, R &f1, R &f2)
{
    if constexpr (DBETA) Lang<R>::le_far(u, f1, f2);
    else Lang<R>::ad_far(u, f1, f2);
}

// The asymptotic form, valid for u >= vfar_threshold<R, DBETA>().
template <typename R, bool DBETA>
__device__ __forceinline__ void lang_vfar(R u, R &f1, R &f2)
{
    if constexpr (DBETA) Lang<R>::le_vfar(u, f1, f2);
    else Lang<R>::ad_vfar(u, f1, f2);
}
// acc + f1 uW + f2 P in the asymptotic range (the pair term of the adjoint
// sums), as a polynomial in iz = 1/z evaluated in nested form:
//   A^T:     (iz - iz^2) uW + iz^3 (2 iz - 1) P = iz (uW + iz (iz (2 iz - 1) P - uW)),
//   d/dbeta: iz^2 uW - 2 iz^4 P                = iz^2 (uW - 2 iz^2 P).
// Five (four) operations after P instead of the seven of forming f1 and f2
// first and then the two products.
template <typename R, bool DBETA>
__device__ __forceinline__ R pair_acc_vfar(R u, R uW, R P, R acc)
{
    const R iz = Lang<R>::iz_vfar(u);
    if constexpr (DBETA) {
        const R iz2 = iz * iz;
        return fmx(iz2, fmx(iz2 * P, R(-2), uW), acc);
    } else {
        const R w = fmx(iz, P * fmx(iz, R(2), R(-1)), -uW);
        return fmx(iz, fmx(iz, w, uW), acc);
    }
}

template <typename R, bool DBETA>
__host__ __device__ constexpr R vfar_threshold()
{
    return DBETA ? (sizeof(R) == 4 ? R(kVfarU32Beta) : R(kVfarU64Beta))
                 : (sizeof(R) == 4 ? R(kVfarU32) : R(kVfarU64));
}

#endif  // __CUDACC__

}  // namespace mpi
