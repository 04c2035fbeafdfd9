// Double-float arithmetic for the FP32 Core Stage's CG vectors.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2),
// about 48 significant bits.  The operations are built from the classical
// error-free transformations: Knuth's TwoSum (a + b = s + e exactly, six
// FP32 operations), Dekker's FastTwoSum (the same for |a| >= |b|, three) and
// the FMA form of TwoProduct (a b = p + e exactly, two).  GB300 executes FP64
// arithmetic at ~1/74 of its FP32 rate, so the Core Stage's vector updates,
// Laplacians and inner products run faster this way than in FP64 at an
// accuracy (2^-48 relative to the operands) far below the FP32 operator's.
// Scalars (alpha, beta, gamma, 1/T) stay FP64 and enter split into a
// double-float pair.
#pragma once

#include "common.cuh"

namespace mpi {

#ifdef __CUDACC__
using df = float2;  // (hi, lo)

__device__ __forceinline__ float2 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b)  // |a| >= |b| or a = 0
{
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df df_from_double(double d)
{
    const float hi = __double2float_rn(d);
    return make_float2(hi, __double2float_rn(d - double(hi)));
}
__device__ __forceinline__ double df_to_double(df a) { return double(a.x) + double(a.y); }

// a + b (the hi parts by TwoSum, the lo parts added to its error term).
__device__ __forceinline__ df df_add(df a, df b)
{
    const float2 s = df_two_sum(a.x, b.x);
    return df_fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ df df_neg(df a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a c for a double-float scalar c = (c.x, c.y).
__device__ __forceinline__ df df_mul(df a, df c)
{
    const float p = __fmul_rn(a.x, c.x);
    float e = __fmaf_rn(a.x, c.x, -p);
    e = __fmaf_rn(a.x, c.y, e);
    e = __fmaf_rn(a.y, c.x, e);
    return df_fast_two_sum(p, e);
}
// a + c b
__device__ __forceinline__ df df_axpy(df a, df c, df b) { return df_add(a, df_mul(b, c)); }

// Running sum of products for inner products: sum += a b, kept as an
// error-free FP32 pair (the products' low terms added to its error word).
__device__ __forceinline__ void df_dot_add(F2Sum &sum, df a, df b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    sum.add(p);
    sum.lo = __fadd_rn(sum.lo, e);
}
#endif

}  // namespace mpi
