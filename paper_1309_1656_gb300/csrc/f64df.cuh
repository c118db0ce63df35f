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

// The same split for doubles with 949 <= biased exponent e <= 1150
// (2^-74 <= |v| < 2^128) and for +-0, in fewer integer operations: hi is
// v's significand truncated (not rounded) to 24 bits, and lo, the
// remaining 29 bits r times v's last-place weight 2^(e - 1075), comes from
// one integer-to-float conversion (rounded to 24 bits, the only rounding)
// times that weight as an exact power of two.  Then 0 <= lo / sign(v) <
// ulp(hi) and |hi + lo - v| <= 2^-47 |v|, as for df_of_double.
__device__ __forceinline__ bool df_fast_range(double v)
{
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned e = (hw >> 20) & 0x7ffu;
    return e - 949u <= 1150u - 949u || ((hw & 0x7fffffffu) | lw) == 0u;
}
__device__ __forceinline__ df df_of_double_fast(double v)
{
    const unsigned hw = (unsigned)__double2hiint(v), lw = (unsigned)__double2loint(v);
    const unsigned sign = hw & 0x80000000u, mag = hw & 0x7fffffffu;
    const unsigned hb = mag == 0u ? sign : (sign | ((mag - (896u << 20)) << 3) | (lw >> 29));
    // 2^(e - 1075) as a float: exponent field e - 1075 + 127 (finite for any e;
    // lw = 0 when v = 0, so the product is then 0)
    const float w = __uint_as_float(((mag >> 20) - 948u) << 23);
    const float lo = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), w);
    return df(__uint_as_float(hb), __uint_as_float(__float_as_uint(lo) ^ sign));
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

// The FP64_DF step keeps a site's split pairs in shared memory: Q x 4 x 8
// bytes (608 B for D3Q19, 288 B for D2Q9).  For D3Q19 one thread per site
// would leave ~10 warps resident per SM, too few to hide the step's long
// dependency chains, so there each site's work is split between two warps:
// the b directions form (b + 1)/2 groups (a direction with its opposite; the
// rest direction alone, last), warp 0 of a block takes groups [0, G0) and
// warp 1 groups [G0, (b + 1)/2), each for the same 32 consecutive sites of
// a row, which doubles the resident warps without divergence (each warp
// runs its own group range).  D2Q9 fits 24 warps with one thread per site:
// there the two warps of a block take 64 consecutive sites, all groups each.
template <int D> struct F64dfSplit {
    static constexpr int Q = Lattice<D>::Q;
    static constexpr int W = D == 3 ? 2 : 1;   // warps per site
    static constexpr int NG = (Q + 1) / 2;     // direction groups
    static constexpr int G0 = W == 2 ? NG / 2 : NG;   // groups of warp 0
    // most populations one warp stages (two per group, one for the rest)
    static constexpr int MAXP = W == 1 ? Q : (2 * (NG - G0) - 1 > 2 * G0 ? 2 * (NG - G0) - 1 : 2 * G0);
    static constexpr int SITES = 64 / W;       // sites per block of 64 threads
    static constexpr int NSUM = 24;            // floats of the 12 moment sums
};
constexpr int kF64dfBlock = 64;                 // two warps
template <int D> constexpr int f64df_min_blocks() { return D == 3 ? 8 : 12; }

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

// Pass 1 of one warp, in two loops that both warps share (one copy of the
// code, so that it stays in the instruction cache).  The first starts the
// asynchronous copies of the raw doubles of the warp's populations (groups
// [glo, ghi) of site si) into stage[j][0 / 1] (j = 2 (group - glo) +
// 0 / 1; halves (f, s_x) and (s_y, s_z)), all before any is waited for.
// The second splits each value into its double-float pair, in place (a pair
// takes the 8 bytes of its double), and adds them to the partial sums.
// The momentum and energy sums are kept signed (jxp = sum i_x f,
// e1 = sum |i|^2 f; jxm, ..., e2 stay zero), so that every direction adds
// to the same sums.  A thread reads back only what it copied.
// amask: the warp's lanes that run this (sites inside the row).
template <int D, bool ODD>
__device__ __forceinline__ void f64df_pass1(const DQuad *base, const Grid &g, const SiteIdx &si, int glo, int ghi,
                                            unsigned amask, double2 (*stage)[2][32], DFSums &a)
{
    constexpr int Q = Lattice<D>::Q;
    const int np = 2 * (ghi - glo) - (2 * ghi > Q ? 1 : 0);   // the rest direction is alone
    const int l = threadIdx.x & 31;
#pragma unroll 1
    for (int j = 0; j < np; ++j) {
        const int q = glo + (j >> 1);
        const int p = (j & 1) ? Q - 1 - q : q;
        // the buffer after an even step holds population p in slot
        // opposite(p) at x - e_p
        const int slot = ODD ? Q - 1 - p : p;
        const int site = ODD ? neighbour(g, si, -kDirs<D>.v[p][0], -kDirs<D>.v[p][1], -kDirs<D>.v[p][2]) : si.s;
        const DQuad *src = base + (int64_t)slot * g.P + site;
        cp_async_vec<16>(&stage[j][0][l], &src->a);
        cp_async_vec<16>(&stage[j][1][l], &src->b);
    }
    cp_async_commit();
    cp_async_wait<0>();
#pragma unroll 1
    for (int j = 0; j < np; ++j) {
        const int q = glo + (j >> 1);
        const int p = (j & 1) ? Q - 1 - q : q;
        const double2 r0 = stage[j][0][l], r1 = stage[j][1][l];
        df F, X, Y, Z;
        // the short split where the whole warp's values allow it (the branch
        // is taken by the warp as one)
        if (__all_sync(amask, df_fast_range(r0.x) && df_fast_range(r0.y) && df_fast_range(r1.x) &&
                                        df_fast_range(r1.y))) {
            F = df_of_double_fast(r0.x);
            X = df_of_double_fast(r0.y);
            Y = df_of_double_fast(r1.x);
            Z = df_of_double_fast(r1.y);
        } else {
            F = df_of_double(r0.x);
            X = df_of_double(r0.y);
            Y = df_of_double(r1.x);
            Z = df_of_double(r1.y);
        }
        reinterpret_cast<float4 *>(&stage[j][0][l])[0] = make_float4(F.hi, F.lo, X.hi, X.lo);
        reinterpret_cast<float4 *>(&stage[j][1][l])[0] = make_float4(Y.hi, Y.lo, Z.hi, Z.lo);
        a.n.add(F);
        a.Sx.add(X);
        a.Sy.add(Y);
        a.Sz.add(Z);
        a.jxp.add(scale2(F, (float)kDirs<D>.v[p][0]));
        a.jyp.add(scale2(F, (float)kDirs<D>.v[p][1]));
        if (D == 3) a.jzp.add(scale2(F, (float)kDirs<D>.v[p][2]));
        a.e1.add(scale2(F, (float)kDirs<D>.v[p][3]));
    }
}

__device__ __forceinline__ void sums_to(const DFSums &a, float (*out)[32])
{
    const DFAcc *v = &a.n;
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        out[2 * i][l] = v[i].hi;
        out[2 * i + 1][l] = v[i].lo;
    }
}

// Both warps combine the two partial sums in the same order (warp 0's
// first), so that they form identical coefficients.
__device__ __forceinline__ DFSums sums_combined(float (*w0)[32], float (*w1)[32])
{
    DFSums a;
    DFAcc *v = &a.n;
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        const df s = two_sum(w0[2 * i][l], w1[2 * i][l]);
        v[i].hi = s.hi;
        v[i].lo = __fadd_rn(__fadd_rn(w0[2 * i + 1][l], w1[2 * i + 1][l]), s.lo);
    }
    return a;
}

// One AA step on FP64 storage in double-float arithmetic.  Pass 1 (a loop):
// each warp reads its groups' populations once, splits every double into its
// double-float pair (integer operations only), keeps the pairs in shared
// memory and adds them to (partial) moment sums in double-float on the FP32
// pipes; with two warps per site they exchange the partial sums through
// shared memory.
// Pass 2: a loop over the warp's groups (unrolled, the kernel's code
// outgrows the instruction cache) takes each direction and its opposite
// back from shared memory, updates them (df_pair_rt), rounds them to double
// (one double addition per value, the step's only FP64 arithmetic) and
// stores them.  Each value is read from and written to HBM once.  In the
// AA pattern a pair's read locations are its write locations, so the
// pairwise in-place update is race-free (as in k_step_aa_df2).
template <int D, bool ODD, bool MAG>
__global__ void __launch_bounds__(kF64dfBlock, f64df_min_blocks<D>())
k_step_aa_f64df(const Planes<double, Lattice<D>::Q> pl, Grid g, Coll<df> k, unsigned *__restrict__ flags)
{
    using SP = F64dfSplit<D>;
    constexpr int Q = Lattice<D>::Q;
    __shared__ double2 stage[2][SP::MAXP][2][32];
    __shared__ float xch[SP::W][SP::NSUM][32];
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
    DFSums a;
    a.zero();
    if (active) f64df_pass1<D, ODD>(base, g, si, glo, ghi, amask, stage[warp], a);
    if constexpr (SP::W == 2) {
        sums_to(a, xch[warp]);
        __syncthreads();
        if (!active) return;
        a = sums_combined(xch[0], xch[SP::W - 1]);
    } else {
        if (!active) return;
    }
    const DFCoef c = df_coefficients<D>(a, k);
    // g.zero (0 at run time) keeps pass 2's addresses from being carried
    // over from pass 1 in registers
    SiteIdx s2 = si;
    s2.s += g.zero;
    s2.x += g.zero;
    const float4(*const st)[2][32] = reinterpret_cast<const float4(*)[2][32]>(stage[warp]);
#pragma unroll 1
    for (int q = glo; q < ghi; ++q) {
        const int qb = Q - 1 - q;
        const bool pair = qb != q;
        const int ex = kDirs<D>.v[q][0], ey = kDirs<D>.v[q][1], ez = kDirs<D>.v[q][2];
        const int j = 2 * (q - glo);
        const float4 a0 = st[j][0][lane], a1 = st[j][1][lane];
        df f(a0.x, a0.y), x(a0.z, a0.w), y(a1.x, a1.y), z(a1.z, a1.w);
        df fb, xb, yb, zb;
        if (pair) {
            const float4 b0 = st[j + 1][0][lane], b1 = st[j + 1][1][lane];
            fb = df(b0.x, b0.y);
            xb = df(b0.z, b0.w);
            yb = df(b1.x, b1.y);
            zb = df(b1.z, b1.w);
        }
        df_pair_rt<D>(c, k, ex, ey, ez, pair, f, x, y, z, fb, xb, yb, zb);
        if constexpr (MAG) {
            rotate_one(x, y, z, k.rot);
            if (pair) rotate_one(xb, yb, zb, k.rot);
        }
        // write locations: population q goes to slot opposite(q) at x (even)
        // or slot q at x + e_q (odd); population qb likewise
        DQuad *const wq = base + (int64_t)(ODD ? q : qb) * g.P + (ODD ? neighbour(g, s2, ex, ey, ez) : s2.s);
        DQuad *const wb = base + (int64_t)(ODD ? qb : q) * g.P + (ODD ? neighbour(g, s2, -ex, -ey, -ez) : s2.s);
        stq(wq, df_round(f), df_round(x), df_round(y), df_round(z));
        if (pair) stq(wb, df_round(fb), df_round(xb), df_round(yb), df_round(zb));
    }
    if (c.flag && (SP::W == 1 || warp == 0)) atomicOr(flags, c.flag);
}

}  // namespace qlbm
