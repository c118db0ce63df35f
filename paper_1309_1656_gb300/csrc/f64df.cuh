// FP64 storage, double-float arithmetic (QLBM_FP64_DF).  The populations
// are IEEE doubles in the FP64 layout, so every kernel but the step is the
// FP64 one; the step splits each double into a double-float pair, runs the
// collision of dfloat.cuh on the single-precision pipes, and rounds the
// result back to a double.  GB300 issues double-precision arithmetic at a
// small fraction of its single-precision rate (the FP64 step is bound by
// it at ~1/4 of the copy bandwidth), so the conversions are done with
// integer operations: splitting takes none of the double pipe, rounding back
// one double addition per value.
#pragma once

#include "dfloat.cuh"
#include "twopass.cuh"

namespace qlbm {

// Double-float pair of a double v, from v's bit fields alone (no double
// and no conversion instruction: the compiler would otherwise predicate a
// conversion path onto every value).  hi is v's significand rounded to 24
// bits (so |lo| <= ulp(hi)/2); lo is the remainder with its 5 lowest bits
// dropped, so |hi + lo - v| <= 2^-47 |v|.  lo is formed exactly in single
// precision: the remainder's 28 bits are placed under an explicit leading
// power of two P, and P (or 2P when hi was rounded up) is subtracted
// (Sterbenz).  Ranges: 2^-102 <= |v| < 2^128 as described; 2^-126 <= |v| <
// 2^-102 keeps hi only (error < 2^-126); smaller values give signed zero;
// larger and non-finite values give an infinity or NaN in hi (flagged by
// the step as non-finite).
__device__ __forceinline__ df df_of_double(double v)
{
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned e = (hw >> 20) & 0x7ffu;       // biased exponent (bias 1023)
    const unsigned sign = hw & 0x80000000u;
    const unsigned rb = (lw >> 28) & 1u;          // first dropped bit: round hi up
    // float exponent e - 1023 + 127; the +rb carries into the exponent when
    // the 23 kept fraction bits are all ones (up to infinity at the top)
    unsigned hb = (sign | ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29)) + rb;
    const unsigned nan = (e == 0x7ffu && ((hw & 0xfffffu) | lw)) ? 0x400000u : 0u;
    hb = e < 897u ? sign : (e > 1150u ? (sign | 0x7f800000u | nan) : hb);
    // remainder (lw mod 2^28) - rb 2^28 in units of 2^(e - 1075):
    // P = 2^(e - 1047) carries the 28 bits (top 23 kept) below it
    const unsigned pe = (e - 920u) << 23;
    const float x = __uint_as_float(pe | ((lw & 0x0fffffffu) >> 5));
    const float lo = __fsub_rn(x, __uint_as_float(pe + (rb << 23)));
    const bool has_lo = e - 921u <= 1150u - 921u;
    return df(__uint_as_float(hb), has_lo ? __uint_as_float(__float_as_uint(lo) ^ sign) : 0.f);
}

// Exact widening of a float to a double on the integer pipes (subnormal
// floats, below 2^-126, become signed zeros).
__device__ __forceinline__ double widen_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xffu;
    const unsigned ed = ef == 0u ? 0u : (ef == 0xffu ? 0x7ffu : ef + 896u);
    const unsigned m = ef == 0u ? 0u : (u & 0x7fffffu);
    return __hiloint2double((int)((u & 0x80000000u) | (ed << 20) | (m >> 3)), (int)(m << 29));
}

// widen_bits for the lo part of a pair: lo is infinite or NaN only when hi
// is, and the sum is then infinite or NaN whatever lo becomes.
__device__ __forceinline__ double widen_lo_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7fffffffu;
    const unsigned hw = a < 0x00800000u ? 0u : (a >> 3) + (896u << 20);
    return __hiloint2double((int)((u & 0x80000000u) | hw), (int)(a < 0x00800000u ? 0u : u << 29));
}

// hi + lo rounded to the nearest double (one double addition).
__device__ __forceinline__ double df_round(df a) { return __dadd_rn(widen_bits(a.hi), widen_lo_bits(a.lo)); }

__device__ __forceinline__ void load_df(const DQuad *p, df &f, df &x, df &y, df &z)
{
    double a, b, c, d;
    ldq(p, a, b, c, d);
    f = df_of_double(a);
    x = df_of_double(b);
    y = df_of_double(c);
    z = df_of_double(d);
}

// The moment sums of pass 1 in double arithmetic, straight from the stored
// doubles (about 6 double additions per population against 4 splits and
// 4-8 double-float additions; the double pipe has room for them, the
// integer pipe, which does the splits, does not).  Rounded to double-float
// once per sum for the coefficients.
struct D64Sums {
    double n, Sx, Sy, Sz, jxp, jxm, jyp, jym, jzp, jzm, e1, e2;
};

template <int D> __device__ __forceinline__ void d64_term(double &a, double v, int q, int first)
{
    a = q == first ? v : __dadd_rn(a, v);
}

template <int D>
__device__ __forceinline__ void d64_accumulate(D64Sums &a, int q, double f, double x, double y, double z)
{
    d64_term<D>(a.n, f, q, 0);
    d64_term<D>(a.Sx, x, q, 0);
    d64_term<D>(a.Sy, y, q, 0);
    d64_term<D>(a.Sz, z, q, 0);
    if (cx<D>(q) > 0) d64_term<D>(a.jxp, f, q, first_q<D>(0, 1));
    if (cx<D>(q) < 0) d64_term<D>(a.jxm, f, q, first_q<D>(0, -1));
    if (cy<D>(q) > 0) d64_term<D>(a.jyp, f, q, first_q<D>(1, 1));
    if (cy<D>(q) < 0) d64_term<D>(a.jym, f, q, first_q<D>(1, -1));
    if (cz<D>(q) > 0) d64_term<D>(a.jzp, f, q, first_q<D>(2, 1));
    if (cz<D>(q) < 0) d64_term<D>(a.jzm, f, q, first_q<D>(2, -1));
    if (cnorm2<D>(q) == 1) d64_term<D>(a.e1, f, q, first_q<D>(3, 1));
    if (cnorm2<D>(q) == 2) d64_term<D>(a.e2, f, q, first_q<D>(3, 2));
}

template <int D> __device__ __forceinline__ DFSums df_sums_of(const D64Sums &a)
{
    DFSums s;
    s.n.set(df_of_double(a.n));
    s.Sx.set(df_of_double(a.Sx));
    s.Sy.set(df_of_double(a.Sy));
    s.Sz.set(df_of_double(a.Sz));
    s.jxp.set(df_of_double(a.jxp));
    s.jxm.set(df_of_double(a.jxm));
    s.jyp.set(df_of_double(a.jyp));
    s.jym.set(df_of_double(a.jym));
    s.jzp.set(D == 3 ? df_of_double(a.jzp) : df(0.f, 0.f));
    s.jzm.set(D == 3 ? df_of_double(a.jzm) : df(0.f, 0.f));
    s.e1.set(df_of_double(a.e1));
    s.e2.set(df_of_double(a.e2));
    return s;
}

// df_pair for a direction known only at run time (lattice vector
// (ex, ey, ez), pair = it is not the rest direction): the same update with
// t = e . j formed as a full sum and the class constants picked by selects,
// so that pass 2 of the step can run as a loop (the unrolled kernel
// overflows the instruction cache).
template <int D>
__device__ __forceinline__ void df_pair_rt(const DFCoef &c, const Coll<df> &k, int ex, int ey, int ez, bool pair,
                                           df &f, df &x, df &y, df &z, df &fb, df &xb, df &yb, df &zb)
{
    const int cls = ex * ex + ey * ey + ez * ez;
    const df bq = cls == 0 ? c.bq[0] : (cls == 1 ? c.bq[1] : c.bq[2]);
    const df w = cls == 0 ? k.w[0] : (cls == 1 ? k.w[1] : k.w[2]);
    df t = scale2(c.jx, (float)ex) + scale2(c.jy, (float)ey);
    if (D == 3) t = t + scale2(c.jz, (float)ez);
    const df A = dfma(k.c4, t * t, bq);
    const df B = k.c3 * t;
    const df hp = w * (A + B);
    f = dfma(hp, c.on, c.omc * f);
    x = dfma(hp, c.oSx, c.omc * x);
    y = dfma(hp, c.oSy, c.omc * y);
    z = dfma(hp, c.oSz, c.omc * z);
    if (pair) {
        const df hm = w * (A - B);
        fb = dfma(hm, c.on, c.omc * fb);
        xb = dfma(hm, c.oSx, c.omc * xb);
        yb = dfma(hm, c.oSy, c.omc * yb);
        zb = dfma(hm, c.oSz, c.omc * zb);
    }
}

// Resident blocks of 128 per SM: the kernel keeps only the moment sums and
// the coefficients across the two passes (80-96 registers; D3Q19 at 6
// blocks ran 5 % faster than at 5 on GB300).
template <int D> constexpr int f64df_min_blocks() { return 6; }

// One AA step on FP64 storage in double-float arithmetic, in two passes:
// pass 1 streams the b populations through the moment sums (in double);
// pass 2
// re-reads each direction with its opposite (from L2 mostly), updates the
// pair and stores it.  A double's low word shares its 32-byte sector with
// the rest of the vector, so pass 2 re-reads whole values rather than
// keeping parts of them in registers; pass 2 is a loop over the pairs
// (unrolled, the kernel's code outgrows the instruction cache).  In the AA
// pattern a pair's read locations are its write locations, so the pairwise
// in-place update is race-free (as in k_step_aa_df2).
template <int D, bool ODD, bool MAG>
__global__ void __launch_bounds__(kStepBlock, f64df_min_blocks<D>())
k_step_aa_f64df(const Planes<double, Lattice<D>::Q> pl, Grid g, Coll<df> k, unsigned *__restrict__ flags)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    D64Sums a;
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        double f, x, y, z;
        ldq(pl.p[read_slot<D, ODD>(p)] + read_site<D, ODD>(g, si, p), f, x, y, z);
        d64_accumulate<D>(a, p, f, x, y, z);
    }
    const DFCoef c = df_coefficients<D>(df_sums_of<D>(a), k);
    // g.zero (0 at run time) keeps pass 2's addresses from being carried
    // over from pass 1 in registers
    SiteIdx s2 = si;
    s2.s += g.zero;
    s2.x += g.zero;
    // plane q starts q * P vectors after plane 0 (one population buffer)
    DQuad *const base = pl.p[0];
#pragma unroll 1
    for (int q = 0; q <= (Q - 1) / 2; ++q) {
        const int qb = Q - 1 - q;
        const bool pair = qb != q;
        const int ex = cx<D>(q), ey = cy<D>(q), ez = cz<D>(q);
        // read locations of populations q and qb; in the AA pattern each is
        // the other's write location
        DQuad *const rq = base + (int64_t)(ODD ? qb : q) * g.P + (ODD ? neighbour(g, s2, -ex, -ey, -ez) : s2.s);
        DQuad *const rb = base + (int64_t)(ODD ? q : qb) * g.P + (ODD ? neighbour(g, s2, ex, ey, ez) : s2.s);
        df f, x, y, z, fb, xb, yb, zb;
        load_df(rq, f, x, y, z);
        if (pair) load_df(rb, fb, xb, yb, zb);
        df_pair_rt<D>(c, k, ex, ey, ez, pair, f, x, y, z, fb, xb, yb, zb);
        if constexpr (MAG) {
            rotate_one(x, y, z, k.rot);
            if (pair) rotate_one(xb, yb, zb, k.rot);
        }
        // population q goes to slot opposite(q) at x (even) or slot q at x + e_q (odd)
        stq(rb, df_round(f), df_round(x), df_round(y), df_round(z));
        if (pair) stq(rq, df_round(fb), df_round(xb), df_round(yb), df_round(zb));
    }
    if (c.flag) atomicOr(flags, c.flag);
}

}  // namespace qlbm
