// FP64 storage, double-float arithmetic (QLBM_FP64_DF).  The populations
// are IEEE doubles in the FP64 layout, so every kernel but the step is the
// FP64 one; the step splits each double into a double-float pair, runs the
// collision of dfloat.cuh on the single-precision pipes, and rounds the
// result back to a double.  GB300 issues double-precision arithmetic at a
// small fraction of its single-precision rate (the FP64 step is bound by
// it at ~1/4 of the copy bandwidth), so the conversions are done with
// integer operations: splitting takes none of the double pipe, rounding back
// one double addition per value, and that addition is the step's only
// double-precision arithmetic.
#pragma once

#include "dfloat.cuh"
#include "step.cuh"
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

// The same split in fewer integer operations, for doubles whose biased
// exponent e is at most 1150 (|v| < 2^128) and either at least 949
// (|v| >= 2^-74) or at most 896: hi is v's significand truncated (not
// rounded) to 24 bits, and lo, the remaining 29 bits r times v's
// last-place weight 2^(e - 1075), comes from one integer-to-float
// conversion (rounded to 24 bits, the only rounding) times 2^-52 times
// hi's sign and exponent, 2^(e - 1023), all exact powers of two.  Then
// 0 <= lo / sign(v) < ulp(hi) and |hi + lo - v| <= 2^-47 |v|, as for
// df_of_double; e <= 896 gives signed zero, as df_of_double does.
__device__ __forceinline__ df df_of_double_fast(double v)
{
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned sign = hw & 0x80000000u, mag = hw & 0x7fffffffu;
    // the top 23 fraction bits under the exponent rebased from 1023 to 127
    const unsigned hb = mag < (897u << 20) ? sign : (sign | __funnelshift_l(lw, mag - (896u << 20), 3));
    const float r = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), 0x1p-52f);
    return df(__uint_as_float(hb), __fmul_rn(r, __uint_as_float(hb & 0xff800000u)));
}

// Where df_of_double_fast applies: fast_key(v) < kFastKeyLimit exactly for
// biased exponents e <= 201 or 949 <= e <= 1150.  With m the magnitude bits
// of v's high word (e in bits 20-30), min(m - (949 << 20), m) is below
// 202 << 20 iff 949 << 20 <= m < 1151 << 20 (the first term, unsigned) or
// m < 202 << 20 (the second); the warp tests the maximum over its values.
__device__ __forceinline__ unsigned fast_key(double v)
{
    const unsigned m = (unsigned)__double2hiint(v) & 0x7fffffffu;
    return min(m - (949u << 20), m);
}
constexpr unsigned kFastKeyLimit = 202u << 20;

// Exact widening of a float to a double on the integer pipes (subnormal
// floats, below 2^-126, become signed zeros).
__device__ __forceinline__ double widen_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7fffffffu;
    // exponent rebased from 127 to 1023: + 896 in the double's exponent field
    unsigned hw = (a >> 3) + (896u << 20);
    hw = a < 0x00800000u ? 0u : (a >= 0x7f800000u ? (a >> 3) | 0x7ff00000u : hw);   // infinities and NaN stay so
    return __hiloint2double((int)((u & 0x80000000u) | hw), (int)(a < 0x00800000u ? 0u : u << 29));
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

// a x + b y with each product exact to ~2^-48 (Dekker) and one TwoSum of
// the two leading parts; the result is left unnormalised (|lo| may exceed
// ulp(hi)/2 when the products nearly cancel), which the rounding to double
// (df_round, exact for any pair) and the accumulators accept as it is.
__device__ __forceinline__ df lin2(df a, df x, df b, df y)
{
    const float p1 = __fmul_rn(a.hi, x.hi);
    float e1 = __fmaf_rn(a.hi, x.hi, -p1);
    e1 = __fmaf_rn(a.hi, x.lo, __fmaf_rn(a.lo, x.hi, e1));
    const float p2 = __fmul_rn(b.hi, y.hi);
    float e2 = __fmaf_rn(b.hi, y.hi, -p2);
    e2 = __fmaf_rn(b.hi, y.lo, __fmaf_rn(b.lo, y.hi, e2));
    const df s = two_sum(p1, p2);
    return df(s.hi, __fadd_rn(s.lo, __fadd_rn(e1, e2)));
}

// a0 x0 + a1 x1 + a2 x2 with each product exact to ~2^-48 (Dekker) and two
// TwoSums of the leading parts, left unnormalised like lin2.
__device__ __forceinline__ df dot3(df a0, df x0, df a1, df x1, df a2, df x2)
{
    const float p0 = __fmul_rn(a0.hi, x0.hi), p1 = __fmul_rn(a1.hi, x1.hi), p2 = __fmul_rn(a2.hi, x2.hi);
    float e0 = __fmaf_rn(a0.hi, x0.hi, -p0), e1 = __fmaf_rn(a1.hi, x1.hi, -p1), e2 = __fmaf_rn(a2.hi, x2.hi, -p2);
    e0 = __fmaf_rn(a0.hi, x0.lo, __fmaf_rn(a0.lo, x0.hi, e0));
    e1 = __fmaf_rn(a1.hi, x1.lo, __fmaf_rn(a1.lo, x1.hi, e1));
    e2 = __fmaf_rn(a2.hi, x2.lo, __fmaf_rn(a2.lo, x2.hi, e2));
    const df s = two_sum(p0, p1), t = two_sum(s.hi, p2);
    return df(t.hi, __fadd_rn(__fadd_rn(s.lo, t.lo), __fadd_rn(e0, __fadd_rn(e1, e2))));
}

// The spin (x, y, z) rotated by the 3x3 matrix r (row-major), with dot3.
__device__ __forceinline__ void rotate_raw(df &x, df &y, df &z, const df (&r)[9])
{
    const df a = x, b = y, c = z;
    x = dot3(r[0], a, r[1], b, r[2], c);
    y = dot3(r[3], a, r[4], b, r[5], c);
    z = dot3(r[6], a, r[7], b, r[8], c);
}

// x + y without the final renormalisation (8 operations).
__device__ __forceinline__ df add_raw(df x, df y)
{
    const df s = two_sum(x.hi, y.hi);
    return df(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ df select(bool p, df a, df b) { return df(p ? a.hi : b.hi, p ? a.lo : b.lo); }

// Products of the lattice weights with the equilibrium's t and t^2
// coefficients, per class of moving direction (|i|^2 = 1, 2): the update
// of a pair then needs no multiplication by w_i.
struct F64dfConst {
    df wc3[2], wc4[2];
};

// Lattice vectors of the directions as a table in constant memory, for
// loops over directions whose index is known only at run time.
template <int D> struct DirTable {
    signed char v[Lattice<D>::Q][4];   // i_x, i_y, i_z, |i|^2
};
template <int D> constexpr DirTable<D> make_dir_table()
{
    DirTable<D> t{};
    for (int q = 0; q < Lattice<D>::Q; ++q) {
        t.v[q][0] = (signed char)cx<D>(q);
        t.v[q][1] = (signed char)cy<D>(q);
        t.v[q][2] = (signed char)cz<D>(q);
        t.v[q][3] = (signed char)cnorm2<D>(q);
    }
    return t;
}
template <int D> __constant__ DirTable<D> kDirs = make_dir_table<D>();

// The FP64_DF step keeps a site's split pairs in shared memory: Q x 4 x 8
// bytes (608 B for D3Q19, 288 B for D2Q9).  For D3Q19 one thread per site
// would leave ~10 warps resident per SM, too few to hide the step's long
// dependency chains, so there each site's work is split between two warps:
// the b directions form (b + 1)/2 groups (a direction with its opposite; the
// rest direction alone, last), warp 0 of a block takes groups [0, G0) and
// warp 1 groups [G0, (b + 1)/2), each for the same 32 consecutive sites of
// a row, which doubles the resident warps without divergence (each warp
// runs its own group range): 9 blocks (18 warps) per SM.  D2Q9 fits 24
// warps with one thread per site: there the two warps of a block take 64
// consecutive sites, all groups each.  (Keeping a group in registers to
// fit more blocks measured slower: the kernel is bound by instruction
// issue, and the extra warps did not make up for the added instructions.)
template <int D> struct F64dfSplit {
    static constexpr int Q = Lattice<D>::Q;
    static constexpr int W = D == 3 ? 2 : 1;   // warps per site
    static constexpr int NG = (Q + 1) / 2;     // direction groups
    static constexpr int G0 = W == 2 ? NG / 2 : NG;   // groups of warp 0
    static constexpr int STAGE = W == 2 ? Q : 2 * Q;   // populations staged per block
    static constexpr int SITES = 64 / W;       // sites per block of 64 threads
    static constexpr int NSUM = 18;            // floats of the 9 partial sums a warp hands over
};
constexpr int kF64dfBlock = 64;                 // two warps
template <int D> constexpr int f64df_min_blocks() { return D == 3 ? 9 : 12; }

// Neighbour indices s + e, s - e for directions known only at run time.  A
// warp's sites share one row, so where the row is away from the y (and,
// for D3Q19, z) faces the whole warp takes s +- (e_x + e_y nx + e_z nx ny)
// plus its lane's x-wrap correction (nonzero only at the row's ends);
// other rows take the per-axis offsets.
struct NbRt {
    NbOff o;
    int cxp, cxm;    // x-wrap corrections of a +x / -x step
    bool interior;   // no y or z wrapping (the same in every lane of the warp)
};
template <int D> __device__ __forceinline__ NbRt nb_rt(const Grid &g, const SiteIdx &si)
{
    NbRt n;
    n.o = nb_offsets(g, si);
    n.cxp = si.x == g.nx - 1 ? -g.nx : 0;
    n.cxm = si.x == 0 ? g.nx : 0;
    n.interior = si.y > 0 && si.y < g.ny - 1 && (D == 2 || (si.z > 0 && si.z < g.nz - 1));
    return n;
}
__device__ __forceinline__ void nb_pair_rt(const NbRt &n, const Grid &g, int s, int ex, int ey, int ez, int &sp,
                                           int &sm)
{
    if (n.interior) {
        const int d = ex + (ey + ez * g.ny) * g.nx;
        sp = s + d + (ex > 0 ? n.cxp : (ex < 0 ? n.cxm : 0));
        sm = s - d + (ex > 0 ? n.cxm : (ex < 0 ? n.cxp : 0));
    } else {
        nb_pair(n.o, s, ex, ey, ez, sp, sm);
    }
}

// Partial moment sums of the FP64_DF step, formed per direction group:
// r = f of the rest direction; a1, a2 = f_i + f_-i summed over the pairs
// with |i|^2 = 1, 2; J = sum over pairs of i (f_i - f_-i); S = sum of s_i.
// Then n = r + a1 + a2 and sum_i |i|^2 f_i = a1 + 2 a2.
struct F64dfSums {
    DFAcc r, a1, a2, jx, jy, jz, Sx, Sy, Sz;
    __device__ __forceinline__ void zero()
    {
        DFAcc *v = &r;
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i].set(df(0.f, 0.f));
    }
};

// A direction group as double-float pairs: v[0..3] = (f, s_x, s_y, s_z) of
// direction q, v[4..7] those of its opposite (zero for the rest direction).
struct DfGroup {
    df v[8];
};

// Where group q's stored vectors are: population q at x - e_q and its
// opposite at x + e_q after an even step (slots swapped), both at x after
// an odd one (the buffer after an even step holds population p in slot
// opposite(p) at x - e_p).
template <int D, bool ODD>
__device__ __forceinline__ void group_sources(const DQuad *base, const Grid &g, const NbRt &o, int s, int q,
                                              const DQuad *&pq, const DQuad *&pb)
{
    constexpr int Q = Lattice<D>::Q;
    const int qb = Q - 1 - q;
    int sp = s, sm = s;
    if (ODD) nb_pair_rt(o, g, s, kDirs<D>.v[q][0], kDirs<D>.v[q][1], kDirs<D>.v[q][2], sp, sm);
    pq = base + (int64_t)(ODD ? qb : q) * g.P + sm;
    pb = base + (int64_t)(ODD ? q : qb) * g.P + sp;
}

// Splits group q's doubles (r0, r1: direction q; b0, b1: its opposite, or
// zeros) into pairs -- the short split where the whole warp's values allow
// it (amask: the warp's active lanes) -- and adds them to the partial sums.
// q is the same in every lane, so the branches on the direction's class and
// components are taken by the warp as one.
template <int D>
__device__ __forceinline__ DfGroup split_group(int q, unsigned amask, double2 r0, double2 r1, double2 b0, double2 b1,
                                               F64dfSums &a)
{
    constexpr int Q = Lattice<D>::Q;
    const double v[8] = {r0.x, r0.y, r1.x, r1.y, b0.x, b0.y, b1.x, b1.y};
    DfGroup G;
    const unsigned key = max(max(max(fast_key(v[0]), fast_key(v[1])), max(fast_key(v[2]), fast_key(v[3]))),
                             max(max(fast_key(v[4]), fast_key(v[5])), max(fast_key(v[6]), fast_key(v[7]))));
    if (__all_sync(amask, key < kFastKeyLimit)) {
#pragma unroll
        for (int i = 0; i < 8; ++i) G.v[i] = df_of_double_fast(v[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) G.v[i] = df_of_double(v[i]);
    }
    a.Sx.add(G.v[1]);
    a.Sy.add(G.v[2]);
    a.Sz.add(G.v[3]);
    if (Q - 1 - q == q) {
        a.r.add(G.v[0]);
        return G;
    }
    a.Sx.add(G.v[5]);
    a.Sy.add(G.v[6]);
    a.Sz.add(G.v[7]);
    const df sum = add_raw(G.v[0], G.v[4]), dif = add_raw(G.v[0], -G.v[4]);
    if (kDirs<D>.v[q][3] == 1) a.a1.add(sum);
    else a.a2.add(sum);
    const int ex = kDirs<D>.v[q][0], ey = kDirs<D>.v[q][1], ez = kDirs<D>.v[q][2];
    if (ex) a.jx.add(scale2(dif, (float)ex));
    if (ey) a.jy.add(scale2(dif, (float)ey));
    if (D == 3 && ez) a.jz.add(scale2(dif, (float)ez));
    return G;
}

// Pass 1 of one warp over groups [glo, ghi) of site si, in two loops that
// both warps share (one copy of the code, so that it stays in the
// instruction cache).  The first starts the asynchronous copies of the raw
// doubles into stage[j][0 / 1] (j = 2 (group - glo) + 0 / 1; halves
// (f, s_x) and (s_y, s_z)), all before any is waited for; the second splits
// each group's values in place (a pair takes the 8 bytes of its double) and
// adds them to the partial sums.  A thread reads back only what it copied.
template <int D, bool ODD>
__device__ __forceinline__ void f64df_pass1(const DQuad *base, const Grid &g, int s, const NbRt &o, int glo,
                                            int ghi, unsigned amask, double2 (*stage)[2][32], F64dfSums &a)
{
    constexpr int Q = Lattice<D>::Q;
    const int l = threadIdx.x & 31;
#pragma unroll 1
    for (int q = glo; q < ghi; ++q) {
        const int j = 2 * (q - glo);
        const DQuad *pq, *pb;
        group_sources<D, ODD>(base, g, o, s, q, pq, pb);
        cp_async_vec<16>(&stage[j][0][l], &pq->a);
        cp_async_vec<16>(&stage[j][1][l], &pq->b);
        if (Q - 1 - q != q) {
            cp_async_vec<16>(&stage[j + 1][0][l], &pb->a);
            cp_async_vec<16>(&stage[j + 1][1][l], &pb->b);
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
#pragma unroll 1
    for (int q = glo; q < ghi; ++q) {
        const bool pair = Q - 1 - q != q;
        const int j = 2 * (q - glo);
        const double2 r0 = stage[j][0][l], r1 = stage[j][1][l];
        double2 b0 = make_double2(0.0, 0.0), b1 = b0;
        if (pair) {
            b0 = stage[j + 1][0][l];
            b1 = stage[j + 1][1][l];
        }
        const DfGroup G = split_group<D>(q, amask, r0, r1, b0, b1, a);
        reinterpret_cast<float4 *>(&stage[j][0][l])[0] = make_float4(G.v[0].hi, G.v[0].lo, G.v[1].hi, G.v[1].lo);
        reinterpret_cast<float4 *>(&stage[j][1][l])[0] = make_float4(G.v[2].hi, G.v[2].lo, G.v[3].hi, G.v[3].lo);
        if (pair) {
            reinterpret_cast<float4 *>(&stage[j + 1][0][l])[0] =
                make_float4(G.v[4].hi, G.v[4].lo, G.v[5].hi, G.v[5].lo);
            reinterpret_cast<float4 *>(&stage[j + 1][1][l])[0] =
                make_float4(G.v[6].hi, G.v[6].lo, G.v[7].hi, G.v[7].lo);
        }
    }
}

__device__ __forceinline__ void sums_to(const F64dfSums &a, float (*out)[32])
{
    const DFAcc *v = &a.r;
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        out[2 * i][l] = v[i].hi;
        out[2 * i + 1][l] = v[i].lo;
    }
}

// The block's sums of a site: a (this warp's) plus the other warp's from
// shared memory.  A rounded sum of two numbers and TwoSum's error term do
// not depend on the order of the operands, so both warps get the same sums.
__device__ __forceinline__ F64dfSums sums_combined(const F64dfSums &a, float (*other)[32])
{
    F64dfSums r;
    const DFAcc *u = &a.r;
    DFAcc *v = &r.r;
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const df s = two_sum(u[i].hi, other[2 * i][l]);
        v[i].hi = s.hi;
        v[i].lo = __fadd_rn(__fadd_rn(u[i].lo, other[2 * i + 1][l]), s.lo);
    }
    return r;
}

// What pass 2 needs of a site: u = J / n (jx, jy, jz), w_i bq for the three
// classes, 1 - omega and omega (n, S).
struct F64dfCoef {
    df jx, jy, jz, wbq0, wbq1, wbq2, omc, on, oSx, oSy, oSz;
};

template <int D>
__device__ __forceinline__ F64dfCoef f64df_coefficients(const F64dfSums &a, const Coll<df> &k, unsigned &flag)
{
    const df a1 = a.a1.value(), a2 = a.a2.value();
    const DFCoef c = df_coefficients_of<D>(a.r.value() + a1 + a2, a.Sx.value(), a.Sy.value(), a.Sz.value(),
                                           a.jx.value(), a.jy.value(), a.jz.value(), a1 + scale2(a2, 2.f), k);
    flag = c.flag;
    F64dfCoef r;
    r.jx = c.jx;
    r.jy = c.jy;
    r.jz = c.jz;
    r.wbq0 = k.w[0] * c.bq[0];
    r.wbq1 = k.w[1] * c.bq[1];
    r.wbq2 = k.w[2] * c.bq[2];
    r.omc = c.omc;
    r.on = c.on;
    r.oSx = c.oSx;
    r.oSy = c.oSy;
    r.oSz = c.oSz;
    return r;
}

// Pass 2 for group q: W' = (1 - omega) W + w_i P_+- omega (n, S) with
// w_i P_+- = (w c4 t^2 + w bq) +- w c3 t, t = i . u, for the direction and
// its opposite; the results are rounded to double (one double addition per
// value, the step's only FP64 arithmetic) and stored where the AA pattern
// puts them: population q to slot opposite(q) at x (even step) or slot q
// at x + e_q (odd), its opposite likewise.
template <int D, bool ODD, int FIELD>
__device__ __forceinline__ void update_group(int q, DfGroup &G, const F64dfCoef &c, const F64dfConst &kc,
                                             const Coll<df> &k, const df (&rs)[9], DQuad *base, const Grid &g,
                                             const NbRt &o, int s)
{
    constexpr int Q = Lattice<D>::Q;
    const int qb = Q - 1 - q;
    const bool pair = qb != q;
    const int ex = kDirs<D>.v[q][0], ey = kDirs<D>.v[q][1], ez = kDirs<D>.v[q][2];
    df hp = c.wbq0, hm;
    if (pair) {
        // t = i . u from i's one (|i|^2 = 1) or two (|i|^2 = 2) nonzero
        // components
        const bool axis = kDirs<D>.v[q][3] == 1;
        df t;
        if (axis) {
            t = scale2(select(ex != 0, c.jx, select(ey != 0, c.jy, c.jz)), (float)(ex + ey + ez));
        } else {
            const df u1 = scale2(select(ex != 0, c.jx, c.jy), (float)(ex != 0 ? ex : ey));
            const df u2 = scale2(select(ez != 0, c.jz, c.jy), (float)(ez != 0 ? ez : ey));
            t = u1 + u2;
        }
        const df A = dfma(select(axis, kc.wc4[0], kc.wc4[1]), t * t, select(axis, c.wbq1, c.wbq2));
        const df B = select(axis, kc.wc3[0], kc.wc3[1]) * t;
        hp = A + B;
        hm = A - B;
    }
    df *v = G.v;
    v[0] = lin2(c.omc, v[0], hp, c.on);
    v[1] = lin2(c.omc, v[1], hp, c.oSx);
    v[2] = lin2(c.omc, v[2], hp, c.oSy);
    v[3] = lin2(c.omc, v[3], hp, c.oSz);
    if (pair) {
        v[4] = lin2(c.omc, v[4], hm, c.on);
        v[5] = lin2(c.omc, v[5], hm, c.oSx);
        v[6] = lin2(c.omc, v[6], hm, c.oSy);
        v[7] = lin2(c.omc, v[7], hm, c.oSz);
    }
    if constexpr (FIELD != FIELD_NONE) {
        // the field term: the spins rotated by the uniform matrix or by the
        // site's own (rs)
#pragma unroll
        for (int i = 1; i < 8; ++i) v[i] = two_sum(v[i].hi, v[i].lo);
        if constexpr (FIELD == FIELD_SITE) {
            rotate_raw(v[1], v[2], v[3], rs);
            if (pair) rotate_raw(v[5], v[6], v[7], rs);
        } else {
            rotate_raw(v[1], v[2], v[3], k.rot);
            if (pair) rotate_raw(v[5], v[6], v[7], k.rot);
        }
    }
    int sp = s, sm = s;
    if (ODD) nb_pair_rt(o, g, s, ex, ey, ez, sp, sm);
    stq(base + (int64_t)(ODD ? q : qb) * g.P + sp, df_round(v[0]), df_round(v[1]), df_round(v[2]), df_round(v[3]));
    if (pair)
        stq(base + (int64_t)(ODD ? qb : q) * g.P + sm, df_round(v[4]), df_round(v[5]), df_round(v[6]),
            df_round(v[7]));
}

// One AA step on FP64 storage in double-float arithmetic.  Pass 1: each warp
// reads its groups' populations once, splits every double into its
// double-float pair (integer operations only), keeps the pairs in shared
// memory and adds them to (partial) moment sums in double-float on the FP32
// pipes; with two warps per site they exchange the partial sums through
// shared memory.  Pass 2: a loop over the groups (not unrolled: more copies
// of the code outgrow the instruction cache), each updated and stored by
// update_group.  Each value is read from and written to HBM once.  In the
// AA pattern a pair's read locations are its write locations, so the
// pairwise in-place update is race-free (as in k_step_aa_df2).
template <int D, bool ODD, int FIELD>
__global__ void __launch_bounds__(kF64dfBlock, f64df_min_blocks<D>())
k_step_aa_f64df(const Planes<double, Lattice<D>::Q> pl, Grid g, Coll<df> k, F64dfConst kc,
                unsigned *__restrict__ flags)
{
    using SP = F64dfSplit<D>;
    __shared__ double2 stage[SP::STAGE][2][32];
    __shared__ float xch[SP::W][SP::NSUM][32];   // partial sums exchanged between the warps of a site
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // site of this lane: g.nxb blocks of SP::SITES sites per row
    const int row = blockIdx.x / g.nxb;
    SiteIdx si;
    si.x = (blockIdx.x - row * g.nxb) * SP::SITES + (SP::W == 2 ? lane : (int)threadIdx.x);
    si.y = row % g.ny;
    si.z = row / g.ny;
    si.s = row * g.nx + si.x;
    const bool active = si.x < g.nx;
    const unsigned amask = __ballot_sync(0xffffffffu, active);   // every lane of the warp is present here
    // plane q starts q * P vectors after plane 0 (one population buffer)
    DQuad *const base = pl.p[0];
    const int glo = (SP::W == 2 && warp == 1) ? SP::G0 : 0, ghi = (SP::W == 2 && warp == 0) ? SP::G0 : SP::NG;
    // this warp's populations in the block's staging area
    double2(*const mine)[2][32] = stage + (SP::W == 2 ? (warp == 0 ? 0 : 2 * SP::G0) : warp * Lattice<D>::Q);
    F64dfSums a;
    a.zero();
    const NbRt o = nb_rt<D>(g, si);
    if (active) f64df_pass1<D, ODD>(base, g, si.s, o, glo, ghi, amask, mine, a);
    unsigned flag = 0u;
    if constexpr (SP::W == 2) {
        // the warps exchange their partial sums; each forms the site's
        // coefficients (the same in both)
        sums_to(a, xch[warp]);
        __syncthreads();
        if (!active) return;
        a = sums_combined(a, xch[warp ^ 1]);
    } else {
        if (!active) return;
    }
    const F64dfCoef c = f64df_coefficients<D>(a, k, flag);
    // a per-site field: the site's rotation from its unit quaternion (stored
    // as doubles), split with the integer split and formed in double-float
    // (no work on the double pipe, which the rounding back already uses)
    df rs[9];
    if constexpr (FIELD == FIELD_SITE) {
        double w, x, y, z;
        load_quat(k.qf + si.s, w, x, y, z);
        quat_rotation(df_of_double(w), df_of_double(x), df_of_double(y), df_of_double(z), rs);
    }
    // g.zero (0 at run time) keeps pass 2's addresses from being carried
    // over from pass 1 in registers
    const int s2 = si.s + g.zero;
    const float4(*const st)[2][32] = reinterpret_cast<const float4(*)[2][32]>(mine);
#pragma unroll 1
    for (int q = glo; q < ghi; ++q) {
        const int j = 2 * (q - glo);
        DfGroup G;
        const float4 a0 = st[j][0][lane], a1 = st[j][1][lane];
        G.v[0] = df(a0.x, a0.y);
        G.v[1] = df(a0.z, a0.w);
        G.v[2] = df(a1.x, a1.y);
        G.v[3] = df(a1.z, a1.w);
        if (Lattice<D>::Q - 1 - q != q) {
            const float4 b0 = st[j + 1][0][lane], b1 = st[j + 1][1][lane];
            G.v[4] = df(b0.x, b0.y);
            G.v[5] = df(b0.z, b0.w);
            G.v[6] = df(b1.x, b1.y);
            G.v[7] = df(b1.z, b1.w);
        }
        update_group<D, ODD, FIELD>(q, G, c, kc, k, rs, base, g, o, s2);
    }
    if (flag && (SP::W == 1 || warp == 0)) atomicOr(flags, flag);
}

}  // namespace qlbm
