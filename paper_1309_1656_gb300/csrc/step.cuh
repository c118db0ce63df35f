// The step kernel: AA-pattern gather, fused moments + equilibrium +
// collision (the codec's), in-place streaming.  Templated on the lattice
// (D = 2: D2Q9, D = 3: D3Q19) and the storage codec.
//
// Memory layout (HBM): one population buffer of b slot planes, plane q
// holding, for every site, the vector of the four components (f, s_x, s_y,
// s_z) of slot q; plane stride P >= N vectors (padded to 64), site
// s = x + nx*(y + ny*z).  Streaming is done in
// place with the AA pattern (Bailey et al., 2009):
//   even step:  read slot q at x              -> population q at x,
//               write population q' to slot opposite(q') at x;
//   odd step:   read slot q at x + e_q        -> population opposite(q) at x,
//               write population q' to slot q' at x + e_q'.
// Each thread reads and writes the same b*4 locations, so the update is
// race-free in one buffer and every value is read once and written once per
// step (Eq. TransportStep).  After an even step the buffer is "swapped"
// (population q at x sits in slot opposite(q) at x - e_q); after an odd step
// it is back in natural order.
#pragma once

#include "lattice.cuh"

namespace qlbm {

constexpr int kStepBlock = 128;   // threads per block along x
constexpr int kRedBlock = 256;    // threads per block of the reductions

// Base pointers of the b slot planes (vectors of the four components of
// storage type S), passed by value so that every access is one multiply-add
// of a 32-bit site index onto a constant-bank pointer (keeps the b addresses
// out of registers).
template <class S, int Q> struct Planes {
    typename QuadOf<S>::V *p[Q];
};

// Site of the calling thread; false if it lies beyond the row.
struct SiteIdx {
    int x, y, z;
    int s;   // flat site index (N < 2^31)
};

__device__ __forceinline__ bool site_of_block(const Grid &g, SiteIdx &si)
{
    const int row = blockIdx.x / g.nxb;
    const int xb = blockIdx.x - row * g.nxb;
    si.x = xb * blockDim.x + threadIdx.x;
    si.y = row % g.ny;
    si.z = row / g.ny;
    si.s = row * g.nx + si.x;
    return si.x < g.nx;
}

// Flat index of site x + (dx,dy,dz), periodic.
__device__ __forceinline__ int neighbour(const Grid &g, const SiteIdx &si, int dx, int dy, int dz)
{
    const int x = wrapm(si.x + dx, g.nx);
    const int y = wrapm(si.y + dy, g.ny);
    const int z = wrapm(si.z + dz, g.nz);
    return x + g.nx * (y + g.ny * z);
}

// Offsets from a site to its periodic neighbours one step along each axis
// (x +- 1, y +- 1, z +- 1, wrapped), so that a neighbour's index is the
// site's plus one offset per nonzero component.  In loops over directions
// unrolled at compile time the selects below vanish; where the direction
// is known only at run time they are a few selects, no division and no
// multiplication.
struct NbOff {
    int xp, xm, yp, ym, zp, zm;
};
__device__ __forceinline__ void nb_offsets_yz(const Grid &g, int y, int z, NbOff &o)
{
    const int nxy = g.nx * g.ny;
    o.yp = y == g.ny - 1 ? (1 - g.ny) * g.nx : g.nx;
    o.ym = y == 0 ? (g.ny - 1) * g.nx : -g.nx;
    o.zp = z == g.nz - 1 ? (1 - g.nz) * nxy : nxy;
    o.zm = z == 0 ? (g.nz - 1) * nxy : -nxy;
}
__device__ __forceinline__ NbOff nb_offsets(const Grid &g, const SiteIdx &si)
{
    NbOff o;
    o.xp = si.x == g.nx - 1 ? 1 - g.nx : 1;
    o.xm = si.x == 0 ? g.nx - 1 : -1;
    nb_offsets_yz(g, si.y, si.z, o);
    return o;
}
__device__ __forceinline__ int nb_axis(int e, int plus, int minus) { return e > 0 ? plus : (e < 0 ? minus : 0); }
// Index of site s + e (components of e in {-1, 0, 1}).
__device__ __forceinline__ int nb_at(const NbOff &o, int s, int ex, int ey, int ez)
{
    return s + nb_axis(ex, o.xp, o.xm) + nb_axis(ey, o.yp, o.ym) + nb_axis(ez, o.zp, o.zm);
}
// Indices of s + e and s - e.
__device__ __forceinline__ void nb_pair(const NbOff &o, int s, int ex, int ey, int ez, int &sp, int &sm)
{
    sp = s + nb_axis(ex, o.xp, o.xm) + nb_axis(ey, o.yp, o.ym) + nb_axis(ez, o.zp, o.zm);
    sm = s + nb_axis(ex, o.xm, o.xp) + nb_axis(ey, o.ym, o.yp) + nb_axis(ez, o.zm, o.zp);
}

// Gathers the b populations of site si at the current time, in arithmetic
// type R.  SWAPPED selects the reading pattern of a buffer last written by
// an even step.
template <int D, class Codec, bool SWAPPED>
__device__ __forceinline__ void gather(const Planes<typename Codec::S, Lattice<D>::Q> &pl,
                                       const Grid &g, const SiteIdx &si, const Codec &codec,
                                       typename Codec::R *f, typename Codec::R *sx,
                                       typename Codec::R *sy, typename Codec::R *sz)
{
    constexpr int Q = Lattice<D>::Q;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int p = SWAPPED ? opposite<D>(q) : q;     // population held by slot q
        const int s = SWAPPED ? neighbour(g, si, cx<D>(q), cy<D>(q), cz<D>(q)) : si.s;
        codec.load4(pl.p[q] + s, f[p], sx[p], sy[p], sz[p]);
    }
}

// Minimum resident blocks of 128 per SM for the step kernels (register
// budget), by lattice.
template <int D, class Codec> constexpr int step_min_blocks()
{
    return D == 2 ? Codec::MIN_BLOCKS_2D : Codec::MIN_BLOCKS;
}

// One AA step (even: ODD = false, odd: ODD = true), fused
// moments + equilibrium + collision + streaming.
template <int D, class Codec, bool ODD, int FIELD = FIELD_NONE>
__global__ void __launch_bounds__(kStepBlock, step_min_blocks<D, Codec>())
k_step_aa(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Coll<typename Codec::R> k,
          Codec codec, unsigned *__restrict__ flags)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    R f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, ODD>(pl, g, si, codec, f, sx, sy, sz);
    const unsigned flag = Codec::template collide<D>(f, sx, sy, sz, k);
    apply_field<D, FIELD, R>(sx, sy, sz, k, si.s);
    // g.zero is 0 at run time; adding it keeps the compiler from carrying the
    // 4b load addresses (identical to the store addresses) through the
    // collision in registers.
    SiteIdx so = si;
    so.s += g.zero;
    so.x += g.zero;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        // population q goes to slot opposite(q) at x (even) or slot q at x + e_q (odd)
        const int slot = ODD ? q : opposite<D>(q);
        const int s = ODD ? neighbour(g, so, cx<D>(q), cy<D>(q), cz<D>(q)) : so.s;
        codec.store4(pl.p[slot] + s, f[q], sx[q], sy[q], sz[q]);
    }
    if (flag) atomicOr(flags, flag);
}

// Codecs whose step runs row-pipelined (k_step_aa_rows): those whose b
// vectors per site fit twice in shared memory at the step's occupancy
// (FP16: 8 bytes per vector).
template <class Codec> struct RowPipelined {
    static constexpr bool value = false;
};
template <> struct RowPipelined<CodecF16Dev> {
    static constexpr bool value = true;
};

__device__ __forceinline__ SiteIdx site_at(const Grid &g, int x, int row)
{
    SiteIdx si;
    si.x = x;
    si.y = row % g.ny;
    si.z = row / g.ny;
    si.s = row * g.nx + x;
    return si;
}

// Asynchronous global -> shared copy of one 8- or 16-byte vector
// (cp.async, completion tracked per thread by commit / wait groups).
template <int BYTES>
__device__ __forceinline__ void cp_async_vec(void *dst, const void *src)
{
    static_assert(BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("{\n\t.reg .u64 g;\n\tcvta.to.global.u64 g, %1;\n\t"
                 "cp.async.ca.shared.global [%0], [g], %2;\n\t}\n" ::"r"(d),
                 "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Starts the copies of the b stored vectors of site s (the slots an even
// step reads at x, or an odd step reads at x + e_q; o: the site's
// neighbour offsets) into dst[q * stride].
template <int D, class Codec, bool SWAPPED>
__device__ __forceinline__ void fetch_site(const Planes<typename Codec::S, Lattice<D>::Q> &pl, int s,
                                           const NbOff &o, typename QuadOf<typename Codec::S>::V *dst, int stride)
{
    using V = typename QuadOf<typename Codec::S>::V;
#pragma unroll
    for (int q = 0; q < Lattice<D>::Q; ++q) {
        const int i = SWAPPED ? nb_at(o, s, cx<D>(q), cy<D>(q), cz<D>(q)) : s;
        cp_async_vec<sizeof(V)>(dst + q * stride, pl.p[q] + i);
    }
}

// Dynamic shared memory of k_step_aa_rows: two stages of b vectors per
// thread.
template <int D, class Codec> constexpr size_t rows_smem_bytes(int block)
{
    return 2 * (size_t)Lattice<D>::Q * block * sizeof(typename QuadOf<typename Codec::S>::V);
}

// The same AA step as k_step_aa, row-pipelined: block (chunk c, group r)
// updates the sites of x-chunk c in the rpb consecutive rows
// r*rpb .. r*rpb + rpb - 1.  Each thread copies its next row's vectors into
// shared memory (cp.async) before it works on the current row, so that one
// row's loads are in flight while the previous row computes, without
// holding them in registers; a thread reads back only what it copied, so no
// block barrier is needed.  Each location is read and written by exactly
// one site update per step, so the early loads of row r + 1 never meet the
// stores of row r.
template <int D, class Codec, bool ODD, int FIELD = FIELD_NONE>
__global__ void __launch_bounds__(kStepBlock, step_min_blocks<D, Codec>())
k_step_aa_rows(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Coll<typename Codec::R> k,
               Codec codec, int rpb, unsigned *__restrict__ flags)
{
    using R = typename Codec::R;
    using V = typename QuadOf<typename Codec::S>::V;
    constexpr int Q = Lattice<D>::Q;
    extern __shared__ __align__(16) unsigned char rows_smem[];
    const int bw = blockDim.x;
    // stage t, slot q of this thread at mine[(t * Q + q) * bw]
    V *mine = reinterpret_cast<V *>(rows_smem) + threadIdx.x;
    const int grp = blockIdx.x / g.nxb;
    const int x = (blockIdx.x - grp * g.nxb) * bw + threadIdx.x;
    if (x >= g.nx) return;
    const int row0 = grp * rpb;
    const int rend = min(row0 + rpb, g.ny * g.nz);
    // the current row's coordinates and neighbour offsets, advanced row by
    // row (one division, at the start)
    SiteIdx cur = site_at(g, x, row0);
    NbOff o = nb_offsets(g, cur);
    fetch_site<D, Codec, ODD>(pl, cur.s, o, mine, bw);
    cp_async_commit();
    unsigned flag = 0;
    for (int row = row0, t = 0; row < rend; ++row, t ^= 1) {
        int ny1 = cur.y + 1, nz1 = cur.z;
        if (ny1 == g.ny) {
            ny1 = 0;
            ++nz1;
        }
        NbOff on = o;
        nb_offsets_yz(g, ny1, nz1, on);
        if (row + 1 < rend) fetch_site<D, Codec, ODD>(pl, cur.s + g.nx, on, mine + (t ^ 1) * Q * bw, bw);
        cp_async_commit();
        cp_async_wait<1>();     // this row's copies have landed
        R f[Q], sx[Q], sy[Q], sz[Q];
        const V *cv = mine + t * Q * bw;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int p = ODD ? opposite<D>(q) : q;     // population held by slot q
            codec.decode4(cv[q * bw], f[p], sx[p], sy[p], sz[p]);
        }
        flag |= Codec::template collide<D>(f, sx, sy, sz, k);
        apply_field<D, FIELD, R>(sx, sy, sz, k, cur.s);
        // store addresses recomputed from g.zero (see k_step_aa)
        const int so = cur.s + g.zero;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int slot = ODD ? q : opposite<D>(q);
            const int i = ODD ? nb_at(o, so, cx<D>(q), cy<D>(q), cz<D>(q)) : so;
            codec.store4(pl.p[slot] + i, f[q], sx[q], sy[q], sz[q]);
        }
        cur.y = ny1;
        cur.z = nz1;
        cur.s += g.nx;
        o = on;
    }
    if (flag) atomicOr(flags, flag);
}

}  // namespace qlbm
