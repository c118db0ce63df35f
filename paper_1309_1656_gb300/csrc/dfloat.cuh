// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// single-precision numbers with |lo| <= ulp(hi)/2, giving a 48-bit
// significand (relative rounding 2^-48 ~ 3.6e-15) out of FP32 operations.
// On GB300 the FP32 pipes issue 64 times as many operations per clock as the
// FP64 pipe, so a step in double-float arithmetic, at ~10 FP32 operations
// per double-float operation, outruns the same step in FP64.
//
// The error-free transformations are Knuth's TwoSum, Dekker's Fast2Sum and
// the FMA-based product (a*b = p + e exactly with e = fma(a, b, -p)); the
// compound operations follow Dekker (1971) and the "sloppy" addition of the
// double-double literature (Hida, Li and Bailey, 2001), whose absolute error
// is bounded by ~2^-47 (|x| + |y|).  Every rounding-sensitive operation uses
// the _rn intrinsics, which the compiler never contracts into an FMA or
// reassociates.
#pragma once

#include <cuda_runtime.h>

#include "lattice.cuh"

namespace qlbm {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // Nearest double-float of a double (host side and the conversion
    // kernels; not used on the hot path).
    __host__ __device__ explicit df(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
    return df(s, e);
}

// s + e = a + b exactly if |a| >= |b| or a = 0 (Dekker's Fast2Sum).
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator+(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

__device__ __forceinline__ df operator*(df x, df y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
    return fast_two_sum(p, e);
}

// x * b for a single-precision b.
__device__ __forceinline__ df mul_f(df x, float b)
{
    const float p = __fmul_rn(x.hi, b);
    const float e = __fmaf_rn(x.lo, b, __fmaf_rn(x.hi, b, -p));
    return fast_two_sum(p, e);
}

// x * 2^k for small integer multiples that are exact (0, +-1, +-2).
__device__ __forceinline__ df scale2(df x, float s) { return df(x.hi * s, x.lo * s); }

// 1/x: the single-precision reciprocal refined by one Newton step in
// double-float, r' = r + r (1 - x r), which squares its relative error.
__device__ __forceinline__ df recip(df x)
{
    const float r = __frcp_rn(x.hi);
    const df e = df(1.0f, 0.0f) - mul_f(x, r);
    return df(r, 0.0f) + mul_f(e, r);
}

// ---------------------------------------------------------------------------
// Double-float storage: the state is two single-precision states of the
// one-vector-per-slot layout, the hi parts (b planes of float4) followed by
// the lo parts (b more planes) -- so a kernel can keep the hi parts in
// registers and re-read only the lo parts.  QuadOf<df>::V is the hi plane's
// float4; the codec knows the distance to the matching lo vector.
// ---------------------------------------------------------------------------
template <> struct QuadOf<df> { using V = float4; };

// a * b + c with one renormalisation (Dekker's product, then the sloppy
// addition of c): 15 single-precision operations instead of 7 + 11.
__device__ __forceinline__ df dfma(df a, df b, df c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    const df s = two_sum(p, c.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// The collision of `collide` in double-float arithmetic (CodecDF), in three
// pieces so that the two-pass kernel can stream the populations through the
// moment sums (df_accumulate), form the per-site coefficients
// (df_coefficients) and update a direction together with its opposite
// (df_pair):
// W' = (1 - omega) W + omega w_i P_i rho, with P_{+-} = bq + c4 t^2 +- c3 t
// for the pair's t = +-(i.j).
// A running sum of double-float terms: the hi parts are added exactly
// (TwoSum), the rounding errors and the lo parts collect in one float, and
// the pair is renormalised once when read (8 operations per term instead of
// the 11 of a renormalised addition; for b <= 19 terms the float collector
// stays within ~20 ulp of the hi sum, so its own rounding is ~1e-13 of the
// sum at worst).
struct DFAcc {
    float hi, lo;
    __device__ __forceinline__ void set(df x)
    {
        hi = x.hi;
        lo = x.lo;
    }
    __device__ __forceinline__ void add(df x)
    {
        const df s = two_sum(hi, x.hi);
        hi = s.hi;
        lo = __fadd_rn(lo, __fadd_rn(s.lo, x.lo));
    }
    __device__ __forceinline__ df value() const { return fast_two_sum(hi, lo); }
};

struct DFSums {
    DFAcc n, Sx, Sy, Sz, jxp, jxm, jyp, jym, jzp, jzm, e1, e2;
    __device__ __forceinline__ void zero()
    {
        const df z(0.f, 0.f);
        n.set(z);
        Sx.set(z);
        Sy.set(z);
        Sz.set(z);
        jxp.set(z);
        jxm.set(z);
        jyp.set(z);
        jym.set(z);
        jzp.set(z);
        jzm.set(z);
        e1.set(z);
        e2.set(z);
    }
};

// First direction contributing to a sum (component c of i equal to sign s;
// c = 3 selects |i|^2 = s); a sum starts at its first term instead of at
// zero, which saves a double-float addition per sum.
template <int D> __host__ __device__ constexpr int first_q(int c, int s)
{
    for (int q = 0; q < Lattice<D>::Q; ++q) {
        const int v = c == 0 ? cx<D>(q) : (c == 1 ? cy<D>(q) : (c == 2 ? cz<D>(q) : cnorm2<D>(q)));
        if (v == s) return q;
    }
    return -1;
}

template <int D> __device__ __forceinline__ void acc_term(DFAcc &a, df f, int q, int first)
{
    if (q == first) a.set(f);
    else a.add(f);
}

// Adds direction q's populations to the sums (q = 0, 1, ... in order).
template <int D>
__device__ __forceinline__ void df_accumulate(DFSums &a, int q, df f, df x, df y, df z)
{
    acc_term<D>(a.n, f, q, 0);
    acc_term<D>(a.Sx, x, q, 0);
    acc_term<D>(a.Sy, y, q, 0);
    acc_term<D>(a.Sz, z, q, 0);
    if (cx<D>(q) > 0) acc_term<D>(a.jxp, f, q, first_q<D>(0, 1));
    if (cx<D>(q) < 0) acc_term<D>(a.jxm, f, q, first_q<D>(0, -1));
    if (cy<D>(q) > 0) acc_term<D>(a.jyp, f, q, first_q<D>(1, 1));
    if (cy<D>(q) < 0) acc_term<D>(a.jym, f, q, first_q<D>(1, -1));
    if (cz<D>(q) > 0) acc_term<D>(a.jzp, f, q, first_q<D>(2, 1));
    if (cz<D>(q) < 0) acc_term<D>(a.jzm, f, q, first_q<D>(2, -1));
    if (cnorm2<D>(q) == 1) acc_term<D>(a.e1, f, q, first_q<D>(3, 1));
    if (cnorm2<D>(q) == 2) acc_term<D>(a.e2, f, q, first_q<D>(3, 2));
}

struct DFCoef {
    df jx, jy, jz, bq[3], omc, on, oSx, oSy, oSz;
    unsigned flag;
};

// Per-site coefficients from the moment sums n, S, J = sum_i i f_i and
// E = sum_i |i|^2 f_i (lattice units).
template <int D>
__device__ __forceinline__ DFCoef df_coefficients_of(df n, df Sx, df Sy, df Sz, df Jx, df Jy, df Jz, df E,
                                                     const Coll<df> &k)
{
    DFCoef c;
    const df rn = recip(n);
    c.jx = Jx * rn;
    c.jy = Jy * rn;
    c.jz = (D == 3) ? Jz * rn : df(0.f, 0.f);
    const df e2n = E * rn;
    const df jj = (D == 3) ? c.jx * c.jx + c.jy * c.jy + c.jz * c.jz : c.jx * c.jx + c.jy * c.jy;
    const df be = k.K * (e2n - jj);          // beta0 * eps
    const df a2 = (be - k.c) * k.inv_mc2;    // alpha2
    const df a1 = df(1.f, 0.f) - k.c * a2;   // alpha1
    const df b0 = k.c5 * jj + a1;
    const df a2K = a2 * k.K;
    c.bq[0] = b0;
    c.bq[1] = b0 + a2K;
    c.bq[2] = b0 + scale2(a2K, 2.f);
    c.omc = df(1.f, 0.f) - k.omega;
    c.on = k.omega * n;
    c.oSx = k.omega * Sx;
    c.oSy = k.omega * Sy;
    c.oSz = k.omega * Sz;
    c.flag = 0u;
    if (!(n.hi > 0.f)) c.flag |= (n.hi == n.hi) ? FLAG_NONPOSITIVE : FLAG_NONFINITE;
    if (!(fabsf(Sx.hi) + fabsf(Sy.hi) + fabsf(Sz.hi) + fabsf(be.hi) < 1e30f)) c.flag |= FLAG_NONFINITE;
    return c;
}

template <int D> __device__ __forceinline__ DFCoef df_coefficients(const DFSums &a, const Coll<df> &k)
{
    return df_coefficients_of<D>(a.n.value(), a.Sx.value(), a.Sy.value(), a.Sz.value(),
                                 a.jxp.value() - a.jxm.value(), a.jyp.value() - a.jym.value(),
                                 (D == 3) ? a.jzp.value() - a.jzm.value() : df(0.f, 0.f),
                                 a.e1.value() + scale2(a.e2.value(), 2.f), k);
}

// Updates direction q (q <= (Q-1)/2) and its opposite Q-1-q in place; for
// the rest direction (the middle index) only the first set is used.
template <int D>
__device__ __forceinline__ void df_pair(const DFCoef &c, const Coll<df> &k, int q, df &f, df &x, df &y, df &z,
                                        df &fb, df &xb, df &yb, df &zb)
{
    constexpr int Q = Lattice<D>::Q;
    const int cls = cnorm2<D>(q);
    df hp, hm;
    if (cls == 0) {
        hp = hm = k.w[0] * c.bq[0];
    } else {
        df t(0.f, 0.f);
        bool first = true;
        if (cx<D>(q)) {
            t = scale2(c.jx, (float)cx<D>(q));
            first = false;
        }
        if (cy<D>(q)) {
            t = first ? scale2(c.jy, (float)cy<D>(q)) : t + scale2(c.jy, (float)cy<D>(q));
            first = false;
        }
        if (cz<D>(q)) t = first ? scale2(c.jz, (float)cz<D>(q)) : t + scale2(c.jz, (float)cz<D>(q));
        const df A = dfma(k.c4, t * t, c.bq[cls]);
        const df B = k.c3 * t;
        hp = k.w[cls] * (A + B);
        hm = k.w[cls] * (A - B);
    }
    f = dfma(hp, c.on, c.omc * f);
    x = dfma(hp, c.oSx, c.omc * x);
    y = dfma(hp, c.oSy, c.omc * y);
    z = dfma(hp, c.oSz, c.omc * z);
    if (Q - 1 - q != q) {
        fb = dfma(hm, c.on, c.omc * fb);
        xb = dfma(hm, c.oSx, c.omc * xb);
        yb = dfma(hm, c.oSy, c.omc * yb);
        zb = dfma(hm, c.oSz, c.omc * zb);
    }
}

// Double-float storage: each value a pair of floats (8 bytes, like a
// double; 48-bit significand) in the split hi / lo layout above.  Its step
// is the two-pass kernel of twopass.cuh (df_accumulate, df_coefficients,
// df_pair); the codec itself only moves values.
struct CodecDF {
    using S = df;
    using V = QuadOf<S>::V;
    using R = df;
    static constexpr bool DEV = false;
    int64_t lo;   // float4 elements from a hi vector to its lo vector (b x plane stride)
    __device__ __forceinline__ R load(S v) const { return v; }
    __device__ __forceinline__ S store(R v) const { return v; }
    __device__ __forceinline__ void load4(const V *p, R &f, R &x, R &y, R &z) const
    {
        const float4 h = p[0], l = p[lo];
        f = df(h.x, l.x);
        x = df(h.y, l.y);
        y = df(h.z, l.z);
        z = df(h.w, l.w);
    }
    __device__ __forceinline__ void store4(V *p, R f, R x, R y, R z) const
    {
        p[0] = make_float4(f.hi, x.hi, y.hi, z.hi);
        p[lo] = make_float4(f.lo, x.lo, y.lo, z.lo);
    }
    __device__ __forceinline__ double to_double(R v, int, int) const { return v.to_double(); }
    __device__ __forceinline__ S from_double(double v, int, int) const { return df(v); }
};

}  // namespace qlbm
