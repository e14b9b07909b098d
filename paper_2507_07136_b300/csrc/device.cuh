// device.cuh -- constants, status reporting and double-float arithmetic shared by the
// sm_103a kernels of the sparse-coefficient splatting library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lsv2.h"

namespace lsv2 {

// Rasteriser constants (3DGS conventions the paper's CUDA path builds on, Sec. 3.4).
// They are float32 values; every comparison is made against exactly these numbers.
constexpr float kDilation = 0.3f;         // px^2 added to the 2D covariance diagonal
constexpr float kGuard = 1.3f;            // guard band on tan(fov/2) for the EWA Jacobian
constexpr float kDegenerateCond = 1e6f;   // tr^2 / det of the undilated 2D covariance
constexpr float kDiscFloor = 0.1f;        // floor of the eigenvalue discriminant
constexpr float kRadiusCap = 1048576.0f;  // screen radius cap (2^20 px)
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Bound of a device-side wait on another warp's progress (a pipeline stage, an accumulator):
// lsv2_set_wait_limit_ns sets it on the host (default 1 s) and every launch passes the value in
// its arguments; 0 makes a wait give up at its first unsuccessful check.  A wait that runs out
// records LSV2_ERR_TIMEOUT.
uint64_t wait_limit_ns();
constexpr uint64_t kDefaultWaitNs = 1000000000ull;
// Bound of the waits with which a CTA that gave up drains its own asynchronous work (bulk and
// tensor copies it issued, MMAs it committed) before it frees TMEM and retires.  Independent of
// the limit above: work that was issued completes on its own.
constexpr uint64_t kDrainNs = 100000000ull;

// Dot2 step (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005): add a * b to the
// unevaluated sum hi + lo with an error-free product (FMA remainder) and an error-free sum
// (TwoSum), so that the result is as accurate as one accumulated in twice the precision.
__device__ __forceinline__ void dot2_step(float a, float b, float& hi, float& lo)
{
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(se, pe));
}

// First nonzero status wins; never traps.
__device__ __forceinline__ void report(int32_t* status, int32_t code)
{
    if (status) atomicCAS(status, 0, code);
}

// 1 - 2^x for -1 <= x <= 0 from the Taylor series (2^x - 1) / x = sum_{n>=0} ln2^(n+1) x^n / (n+1)!
// taken through x^8: the first omitted term is below 1.5e-8 of the sum on the interval, and the
// Horner steps add a few ulp.  Outside [-1, 0] the result is meaningless (callers select it
// only there).
__host__ __device__ constexpr double exp2_taylor_coeff(int n)
{
    double c = 1.0;
    for (int k = 1; k <= n + 1; ++k) c *= 0.6931471805599453 / (double)k;
    return c;
}
__device__ __forceinline__ float one_minus_exp2(float x)
{
    float g = (float)exp2_taylor_coeff(8);
    g = fmaf(g, x, (float)exp2_taylor_coeff(7));
    g = fmaf(g, x, (float)exp2_taylor_coeff(6));
    g = fmaf(g, x, (float)exp2_taylor_coeff(5));
    g = fmaf(g, x, (float)exp2_taylor_coeff(4));
    g = fmaf(g, x, (float)exp2_taylor_coeff(3));
    g = fmaf(g, x, (float)exp2_taylor_coeff(2));
    g = fmaf(g, x, (float)exp2_taylor_coeff(1));
    g = fmaf(g, x, (float)exp2_taylor_coeff(0));
    return -x * g;
}

// 1 - alpha for alpha = min(0.99, o 2^p2) with p2 = power * log2(e) <= 0, without the
// cancellation of `1 - alpha` near alpha = 1 (which would multiply alpha's relative error by
// alpha / (1 - alpha) in every later transmittance): for alpha > 1/2 (hence o > 1/2, where
// 1 - o is exact, and -1 < p2 <= 0), 1 - o 2^p2 = (1 - o) + o (1 - 2^p2), a sum of two
// non-negative terms.  Branch-free: both forms are computed and one is selected.
__device__ __forceinline__ float one_minus_alpha(float alpha, float o, float p2)
{
    const float near_one = fmaf(o, one_minus_exp2(p2), 1.0f - o);
    const float r = alpha <= 0.5f ? 1.0f - alpha : near_one;
    return alpha == kAlphaMax ? 1.0f - kAlphaMax : r;
}

// ----------------------------------------------------------------------------------------
// Double-float ("double-word") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2.  Error-free transformations after Dekker (1971) and Knuth
// (TwoSum); the double-word operations follow Joldes, Muller & Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic" (ACM TOMS
// 2017): accurate DW+DW, DW*FP and DW*DW with FMA.  Every step uses explicitly rounded
// intrinsics so no contraction or reassociation can change it.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df(float a) { return {a, 0.0f}; }

__device__ __forceinline__ dfloat two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    float ap = __fsub_rn(s, bp);
    float e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
    return {s, e};
}

// Requires |a| >= |b| (or a == 0).
__device__ __forceinline__ dfloat fast_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ dfloat two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y)
{
    dfloat s = two_sum(x.hi, y.hi);
    dfloat t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    dfloat v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}

__device__ __forceinline__ dfloat df_neg(dfloat x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfloat df_sub(dfloat x, dfloat y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ dfloat df_mul_f(dfloat x, float y)
{
    dfloat c = two_prod(x.hi, y);
    float l = __fmaf_rn(x.lo, y, c.lo);
    return fast_two_sum(c.hi, l);
}

__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y)
{
    dfloat c = two_prod(x.hi, y.hi);
    float t0 = __fmul_rn(x.lo, y.lo);
    float t1 = __fmaf_rn(x.hi, y.lo, t0);
    float l2 = __fmaf_rn(x.lo, y.hi, t1);
    float l3 = __fadd_rn(c.lo, l2);
    return fast_two_sum(c.hi, l3);
}

// Quotient with one correction step: q1 = x_hi / y_hi, r = x - y q1 (in double-float),
// q2 = r_hi / y_hi.  Relative error about 2^-44.
__device__ __forceinline__ dfloat df_div(dfloat x, dfloat y)
{
    float q1 = __fdiv_rn(x.hi, y.hi);
    dfloat r = df_sub(x, df_mul_f(y, q1));
    float q2 = __fdiv_rn(r.hi, y.hi);
    return fast_two_sum(q1, q2);
}

// Square root with one correction step: s = sqrt(x_hi), then (x - s^2) / (2 s).
__device__ __forceinline__ dfloat df_sqrt(dfloat x)
{
    if (!(x.hi > 0.0f)) return df(0.0f);
    float s = __fsqrt_rn(x.hi);
    dfloat r = df_sub(x, two_prod(s, s));
    return fast_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.0f, s)));
}

// ----------------------------------------------------------------------------------------
// Evaluation of a projected Gaussian at a pixel, shared by the forward and backward splat.
//   power = -1/2 d^T Q d,  d = mean2d - pixel,  Q = conic = q1 e1 e1^T + q2 e2 e2^T.
// The conic's own entries can cancel badly for elongated footprints (terms of +-100 summing to
// -2 at 100 px along the long axis, where rounding the entries alone moves the power by 1e-5),
// so it is evaluated in its principal frame: power * log2(e) = A u^2 + B v^2 with u = e1 . d
// (stiff axis) and v = e2 . d.  The stiff axis is stored as a float pair and u is formed with
// its low part and an exact product, so its error is one rounding of u itself (needed when the
// footprint is elongated; done for every footprint, which keeps the evaluation branch-free).
// `g0` = (u_hi, v_hi, u_lo, v_lo) of the 2D mean, `ax` = (c_hi, s_hi, A, B),
// `axl` = (c_lo, s_lo, kappa, .).
__device__ __forceinline__ float eval_power2(const float4& g0, const float4& ax, const float4& axl, float pxf,
                                             float pyf)
{
    const float dx = __fadd_rn(__fsub_rn(g0.x, pxf), g0.z);
    const float dy = __fadd_rn(__fsub_rn(g0.y, pyf), g0.w);
    const float v = fmaf(ax.x, dy, -(ax.y * dx));
    // u = (c_hi + c_lo) dx + (s_hi + s_lo) dy with the product s_hi dy split exactly
    const float t = __fmul_rn(ax.y, dy);
    const float te = __fmaf_rn(ax.y, dy, -t);
    const float corr = __fmaf_rn(axl.x, dx, __fmaf_rn(axl.y, dy, te));
    const float u = __fadd_rn(__fmaf_rn(ax.x, dx, t), corr);
    return fmaf(ax.z * u, u, ax.w * v * v);
}

}  // namespace lsv2
