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
template <int D, class Codec, bool ODD, bool MAG = false>
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
    if constexpr (MAG) rotate_spins<D, R>(sx, sy, sz, k.rot);
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

}  // namespace qlbm
