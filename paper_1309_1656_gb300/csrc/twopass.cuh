// Two-pass AA step for the double-float codec.  Holding all 4b double-float
// values of a site takes the whole register file of a thread (255 registers,
// 8 warps per SM), and with so few warps the loads and the long arithmetic
// do not overlap.  This kernel streams the populations through the moment
// sums (pass 1), keeping their hi parts (4b floats) in registers and their
// lo parts in shared memory (4b x 4 B per thread: 38.9 KB per D3Q19 block),
// forms the coefficients, then takes the lo parts of each direction
// together with its opposite back from shared memory (pass 2), updates the
// pair and stores it.  Every value is read from HBM once.  In the AA pattern the read locations of a direction
// and of its opposite are exactly the pair's two write locations (even step:
// slots q and opposite(q) at x; odd step: slot opposite(q) at x - e_q and
// slot q at x + e_q), so updating pair by pair in place is race-free within
// the thread, and across threads as in the one-pass kernel.
#pragma once

#include "dfloat.cuh"
#include "kernels.cuh"

namespace qlbm {

template <class Codec> struct TwoPass {
    static constexpr bool value = false;
};
template <> struct TwoPass<CodecDF> {
    static constexpr bool value = true;
    // Blocks of 128 per SM: D3Q19 keeps 76 hi floats per thread (128
    // registers), D2Q9 36 (96).  Re-reading whole values in pass 2 instead
    // missed in L2 for ~40 % of the re-read bytes (D3Q19).
    template <int D> static constexpr int min_blocks() { return D == 2 ? 5 : 4; }
};

// Spin rotation of the magnetic-field term for one population (see
// rotate_spins).
__device__ __forceinline__ void rotate_one(df &x, df &y, df &z, const df (&r)[9])
{
    const df a = x, b = y, c = z;
    x = r[0] * a + r[1] * b + r[2] * c;
    y = r[3] * a + r[4] * b + r[5] * c;
    z = r[6] * a + r[7] * b + r[8] * c;
}

// Location of population p of site si: slot and site index.
template <int D, bool SWAPPED>
__device__ __forceinline__ int read_slot(int p) { return SWAPPED ? opposite<D>(p) : p; }

template <int D, bool SWAPPED>
__device__ __forceinline__ int read_site(const Grid &g, const SiteIdx &si, int p)
{
    // swapped buffer: population p sits in slot opposite(p) at x - e_p
    return SWAPPED ? neighbour(g, si, -cx<D>(p), -cy<D>(p), -cz<D>(p)) : si.s;
}

template <int D, bool ODD, int FIELD>
__global__ void __launch_bounds__(kStepBlock, TwoPass<CodecDF>::min_blocks<D>())
k_step_aa_df2(const Planes<df, Lattice<D>::Q> pl, Grid g, Coll<df> k, CodecDF codec, unsigned *__restrict__ flags)
{
    constexpr int Q = Lattice<D>::Q;
    // lo parts, kept from pass 1 in shared memory (a thread reads back only
    // what it wrote: no barrier)
    __shared__ float4 lo_stage[Q][kStepBlock];
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    float hf[Q], hx[Q], hy[Q], hz[Q];   // hi parts, kept from pass 1 in registers
    DFSums a;
    a.zero();
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        const float4 *v = pl.p[read_slot<D, ODD>(p)] + read_site<D, ODD>(g, si, p);
        const float4 h = v[0], l = v[codec.lo];
        hf[p] = h.x;
        hx[p] = h.y;
        hy[p] = h.z;
        hz[p] = h.w;
        lo_stage[p][threadIdx.x] = l;
        df_accumulate<D>(a, p, df(h.x, l.x), df(h.y, l.y), df(h.z, l.z), df(h.w, l.w));
    }
    const DFCoef c = df_coefficients<D>(a, k);
    // a per-site field: the site's rotation, formed in double from its unit
    // quaternion and rounded to double-float pairs
    df rs[9];
    if constexpr (FIELD == FIELD_SITE) {
        double w, x, y, z, r[9];
        load_quat(k.qf + si.s, w, x, y, z);
        quat_rotation(w, x, y, z, r);
#pragma unroll
        for (int i = 0; i < 9; ++i) rs[i] = df(r[i]);
    }
    // g.zero (0 at run time) makes pass 2's addresses distinct expressions,
    // so the compiler re-loads the lo parts instead of keeping pass 1's.
    SiteIdx s2 = si;
    s2.s += g.zero;
    s2.x += g.zero;
#pragma unroll
    for (int q = 0; q <= (Q - 1) / 2; ++q) {
        const int qb = Q - 1 - q;
        // (index through g.zero: the compiler re-reads shared memory instead
        // of keeping pass 1's lo values in registers)
        const float4 l = lo_stage[q][threadIdx.x + g.zero];
        df f(hf[q], l.x), x(hx[q], l.y), y(hy[q], l.z), z(hz[q], l.w);
        df fb, xb, yb, zb;
        if (qb != q) {
            const float4 lb = lo_stage[qb][threadIdx.x + g.zero];
            fb = df(hf[qb], lb.x);
            xb = df(hx[qb], lb.y);
            yb = df(hy[qb], lb.z);
            zb = df(hz[qb], lb.w);
        }
        df_pair<D>(c, k, q, f, x, y, z, fb, xb, yb, zb);
        if constexpr (FIELD == FIELD_UNIFORM) {
            rotate_one(x, y, z, k.rot);
            if (qb != q) rotate_one(xb, yb, zb, k.rot);
        } else if constexpr (FIELD == FIELD_SITE) {
            rotate_one(x, y, z, rs);
            if (qb != q) rotate_one(xb, yb, zb, rs);
        }
        // population p goes to slot opposite(p) at x (even) or slot p at x + e_p (odd)
        codec.store4(pl.p[ODD ? q : qb] + (ODD ? neighbour(g, s2, cx<D>(q), cy<D>(q), cz<D>(q)) : s2.s), f, x, y,
                     z);
        if (qb != q)
            codec.store4(pl.p[ODD ? qb : q] + (ODD ? neighbour(g, s2, cx<D>(qb), cy<D>(qb), cz<D>(qb)) : s2.s), fb,
                         xb, yb, zb);
    }
    if (c.flag) atomicOr(flags, c.flag);
}

}  // namespace qlbm
