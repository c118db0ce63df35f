// CUDA kernels of the forward path, templated on the lattice (D = 2: D2Q9,
// D = 3: D3Q19) and the storage codec.  Instantiated once per lattice in
// kernels_d2q9.cu / kernels_d3q19.cu.
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

#include <type_traits>

#include "dfloat.cuh"
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

// One AA step (even: ODD = false, odd: ODD = true), fused
// moments + equilibrium + collision + streaming.
// Minimum resident blocks of 128 per SM for the step kernels (register
// budget), by lattice.
template <int D, class Codec> constexpr int step_min_blocks()
{
    return D == 2 ? Codec::MIN_BLOCKS_2D : Codec::MIN_BLOCKS;
}

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

// ---------------------------------------------------------------------------
// Initial equilibrium (Eq. WeqAlgo evaluated from given rho, u, eps), in
// double, stored in natural order.
// ---------------------------------------------------------------------------
struct InitConsts {
    double xi, K, c, inv_mc2, c3, c4, c5, eps0, beta0;
    double w[3];
};

template <int D>
__device__ __forceinline__ double poly_P_d(const InitConsts &ic, int q, double jx, double jy, double jz, double be)
{
    const double jj = jx * jx + jy * jy + jz * jz;
    const double a2 = (be - ic.c) * ic.inv_mc2;
    const double a1 = 1.0 - ic.c * a2;
    const double t = cx<D>(q) * jx + cy<D>(q) * jy + cz<D>(q) * jz;
    return a1 + a2 * ic.K * cnorm2<D>(q) + ic.c3 * t + ic.c4 * t * t + ic.c5 * jj;
}

template <int D, class Codec>
__global__ void __launch_bounds__(kStepBlock)
k_init_eq(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, InitConsts ic, Codec codec,
          const double *__restrict__ rho4, const double *__restrict__ u,
          const double *__restrict__ eps)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    const int64_t N = g.N, s = si.s;
    const double n = rho4[s], Sx = rho4[N + s], Sy = rho4[2 * N + s], Sz = rho4[3 * N + s];
    const double jx = u[s] / ic.xi, jy = u[N + s] / ic.xi, jz = (D == 3) ? u[2 * N + s] / ic.xi : 0.0;
    const double e = eps ? eps[s] : ic.eps0;
    const double be = ic.beta0 * e;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cls = cnorm2<D>(q);
        const double wp = ic.w[cls] * poly_P_d<D>(ic, q, jx, jy, jz, be);
        codec.store4(pl.p[q] + s, codec.load(codec.from_double(wp * n, 0, cls)),
                     codec.load(codec.from_double(wp * Sx, 1, cls)), codec.load(codec.from_double(wp * Sy, 2, cls)),
                     codec.load(codec.from_double(wp * Sz, 3, cls)));
    }
}

// ---------------------------------------------------------------------------
// State exchange in the canonical layout double [b][4][N].
// ---------------------------------------------------------------------------
template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kStepBlock)
k_get_state(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec, double *__restrict__ out)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    R f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, SWAPPED>(pl, g, si, codec, f, sx, sy, sz);
    const int64_t N = g.N;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double *o = out + (int64_t)(4 * q) * N + si.s;
        const int cls = cnorm2<D>(q);
        o[0] = codec.to_double(f[q], 0, cls);
        o[N] = codec.to_double(sx[q], 1, cls);
        o[2 * N] = codec.to_double(sy[q], 2, cls);
        o[3 * N] = codec.to_double(sz[q], 3, cls);
    }
}

template <int D, class Codec>
__global__ void __launch_bounds__(kStepBlock)
k_set_state(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec, const double *__restrict__ in)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    const int64_t N = g.N;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const double *v = in + (int64_t)(4 * q) * N + si.s;
        const int cls = cnorm2<D>(q);
        codec.store4(pl.p[q] + si.s, codec.load(codec.from_double(v[0], 0, cls)),
                     codec.load(codec.from_double(v[N], 1, cls)), codec.load(codec.from_double(v[2 * N], 2, cls)),
                     codec.load(codec.from_double(v[3 * N], 3, cls)));
    }
}

// ---------------------------------------------------------------------------
// Moments of Eq. DiscrAvr in double.
// ---------------------------------------------------------------------------
template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kStepBlock)
k_moments(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec, double xi,
          double *__restrict__ rho4, double *__restrict__ u, double *__restrict__ eps)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    R f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, SWAPPED>(pl, g, si, codec, f, sx, sy, sz);
    double fd[Q], xd[Q], yd[Q], zd[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cls = cnorm2<D>(q);
        fd[q] = codec.to_double(f[q], 0, cls);
        xd[q] = codec.to_double(sx[q], 1, cls);
        yd[q] = codec.to_double(sy[q], 2, cls);
        zd[q] = codec.to_double(sz[q], 3, cls);
    }
    const SiteMoments<D, double> m = site_moments<D, double>(fd, xd, yd, zd);
    const int64_t N = g.N, s = si.s;
    if (rho4) {
        rho4[s] = m.n;
        rho4[N + s] = m.Sx;
        rho4[2 * N + s] = m.Sy;
        rho4[3 * N + s] = m.Sz;
    }
    if (u) {
        u[s] = xi * m.jx;
        u[N + s] = xi * m.jy;
        if (D == 3) u[2 * N + s] = xi * m.jz;
    }
    if (eps) eps[s] = 0.5 * xi * xi * (m.e2n - (m.jx * m.jx + m.jy * m.jy + m.jz * m.jz));
}

// ---------------------------------------------------------------------------
// Global sums of Eqs. GlobalDensity, GlobalVelocity, GlobalTotalEnergy in
// double: per-block partials, then one block over the partials.  The launch
// shape is fixed per handle, so the result is deterministic.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double *__restrict__ out)
{
    __shared__ double sh[kRedBlock / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[warp][i] = v[i];
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
        for (int w = 0; w < kRedBlock / 32; ++w) acc += sh[w][threadIdx.x];
        out[threadIdx.x] = acc;
    }
}

template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kRedBlock)
k_conserved_partial(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec,
                    double *__restrict__ partials)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
        SiteIdx si;
        si.s = (int)s;
        si.x = (int)(s % g.nx);
        const int64_t row = s / g.nx;
        si.y = (int)(row % g.ny);
        si.z = (int)(row / g.ny);
        R f[Q], sx[Q], sy[Q], sz[Q];
        gather<D, Codec, SWAPPED>(pl, g, si, codec, f, sx, sy, sz);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int cls = cnorm2<D>(q);
            const double fq = codec.to_double(f[q], 0, cls);
            acc[0] += fq;
            acc[1] += codec.to_double(sx[q], 1, cls);
            acc[2] += codec.to_double(sy[q], 2, cls);
            acc[3] += codec.to_double(sz[q], 3, cls);
            acc[4] += cx<D>(q) * fq;
            acc[5] += cy<D>(q) * fq;
            acc[6] += cz<D>(q) * fq;
            acc[7] += cnorm2<D>(q) * fq;
        }
    }
    block_sum_store<8>(acc, partials + (int64_t)blockIdx.x * 8);
}

// Sums nparts rows of 8 partials in a fixed order; out[0..7] then scaled:
// density /N, momentum xi/N, energy xi^2/(2N).
__global__ void __launch_bounds__(kRedBlock)
k_conserved_final(const double *__restrict__ partials, int nparts, double xi, int64_t N,
                  double *__restrict__ out);

}  // namespace qlbm
