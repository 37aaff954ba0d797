// Double-single ("float-float") arithmetic for the refined pass.
//
// The refined pass needs its residuals, its sample values and its interface
// coefficients to about 1e-12 relative, far below FP32's 6e-8.  FP64 gives
// that, but this part runs FP64 at about 1/64 of its FP32 rate, and the
// refined pass was bound by it.  Here a value is carried as an unevaluated
// sum h + l of two floats, and every step is built from the error-free
// transformations of Knuth (two-sum: a + b = s + e exactly) and of
// Dekker with a fused multiply-add (two-prod: a b = p + e exactly), as in the
// double-word algorithms of Dekker (1971) and of Joldes, Muller and Popescu
// (2017).  Products of two error terms (about 2^-48 relative) are dropped,
// which leaves about 47 significant bits, ample for a residual that only has
// to be right to a few digits of its own size.
//
// Every operation is an explicitly rounded intrinsic (__fadd_rn, __fmul_rn,
// __fmaf_rn): the compiler never contracts or reorders them, which the
// error-free transformations depend on.
#pragma once

namespace dfs {

struct FF {
    float h, l;   // value h + l
};

__device__ __forceinline__ FF ff_from(float a) { return {a, 0.0f}; }

// FP64 -> double-single (host-prepared per-ray constants; two FP64 ops).
__device__ __forceinline__ FF ff_from_double(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }

__device__ __forceinline__ float ff_round(FF a) { return __fadd_rn(a.h, a.l); }

// a + b = s + e exactly (Knuth).
__device__ __forceinline__ FF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// a b = p + e exactly (Dekker's product with a fused multiply-add).
__device__ __forceinline__ FF two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const FF s = two_sum(a.h, b.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const FF p = two_prod(a.h, b.h);
    return {p.h, __fadd_rn(p.l, __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h)))};
}

__device__ __forceinline__ FF ff_mul_f(FF a, float b)
{
    const FF p = two_prod(a.h, b);
    return {p.h, __fmaf_rn(a.l, b, p.l)};
}

// a + w (b - a): the difference of the leading parts is exact (two-sum), its
// product with the leading part of w exact (two-prod), and the sum with a
// exact (two-sum); the dropped terms are products of two error terms.
__device__ __forceinline__ FF ff_lerp(FF a, FF b, FF w)
{
    const FF t = two_sum(b.h, -a.h);
    const float te = __fadd_rn(t.l, __fsub_rn(b.l, a.l));
    const FF p = two_prod(w.h, t.h);
    const FF c = two_sum(a.h, p.h);
    const float e = __fadd_rn(__fadd_rn(c.l, p.l), __fmaf_rn(w.h, te, __fmaf_rn(w.l, t.h, a.l)));
    return {c.h, e};
}

// n / d with d != 0.  The leading quotient q is a float estimate; the
// remainder n - q d is formed with a fused multiply-add (exact for the
// leading parts when q is within an ulp or two of n.h / d.h, and in any case
// a small number whose rounding is second order) and divided once more.
__device__ __forceinline__ FF ff_div(FF n, FF d)
{
    const float inv = __fdividef(1.0f, d.h);
    const float q = __fmul_rn(n.h, inv);
    const float rem = __fadd_rn(__fmaf_rn(-q, d.h, n.h), __fmaf_rn(-q, d.l, n.l));
    return {q, __fmul_rn(rem, inv)};
}

// p0 a + p1 b - n for floats p0, p1, n and double-single a, b, rounded to a
// float.  The leading products and their sums are exact (two-prod,
// two-sum), so a result that cancels almost all of n (a residual) keeps its
// own leading digits.
__device__ __forceinline__ float ff_dot2_minus(float p0, FF a, float p1, FF b, float n)
{
    const FF x = two_prod(p0, a.h), y = two_prod(p1, b.h);
    const FF s = two_sum(x.h, y.h);
    const FF u = two_sum(s.h, -n);
    const float tail = __fadd_rn(__fadd_rn(u.l, s.l),
                                 __fadd_rn(__fadd_rn(x.l, y.l), __fmaf_rn(p0, a.l, __fmul_rn(p1, b.l))));
    return __fadd_rn(u.h, tail);
}

}  // namespace dfs
