// CUDA kernels of the forward path besides the step (step.cuh): initial
// equilibrium, state exchange, moments and the conservation sums; templated
// on the lattice and the storage codec.  Instantiated once per lattice and
// codec in kernels_<lattice>_<codec>.cu.
#pragma once

#include <type_traits>

#include "dfloat.cuh"
#include "step.cuh"

namespace qlbm {

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
// Negative-definite equilibria (Sec. 3.2 end, Sec. 3.3 end): W_i^eq =
// w_i rho P_i (Eq. WeqAlgo) can have a negative eigenvalue, and the scheme
// neither clips it nor adapts tau.  This read-only diagnostic forms, from
// the current state, the moments and every P_i that the next collision uses
// and flags direction i when W_i^eq has a negative eigenvalue.  The
// eigenvalues of w_i P_i rho are w_i P_i (n +- |S|)/2 (w_i > 0), so the
// smallest is negative exactly when P_i n < |P_i| |S|.  The decision is
// taken in double whatever the storage precision.  mask[s] (if not NULL)
// receives bit i for each flagged direction; *count accumulates the number
// of flagged (site, direction) pairs (one atomic per warp).
// ---------------------------------------------------------------------------
template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kStepBlock)
k_negative_eq(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec, InitConsts ic,
              unsigned long long *__restrict__ count, unsigned *__restrict__ mask)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    unsigned m = 0u;
    if (site_of_block(g, si)) {
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
        const SiteMoments<D, double> mm = site_moments<D, double>(fd, xd, yd, zd);
        const double jj = mm.jx * mm.jx + mm.jy * mm.jy + mm.jz * mm.jz;
        const double be = ic.K * (mm.e2n - jj);
        const double normS = sqrt(mm.Sx * mm.Sx + mm.Sy * mm.Sy + mm.Sz * mm.Sz);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const double P = poly_P_d<D>(ic, q, mm.jx, mm.jy, mm.jz, be);
            if (P * mm.n < fabs(P) * normS) m |= 1u << q;
        }
        if (mask) mask[si.s] = m;
    }
    const unsigned c = __reduce_add_sync(0xffffffffu, (unsigned)__popc(m));
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
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

// Block sum of values held by lane 0 of each warp (other lanes hold 0).
template <int NV>
__device__ __forceinline__ void block_sum_lanes0(const double (&v)[NV], double *__restrict__ out)
{
    __shared__ double sh[kRedBlock / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

// Per thread, the sites' sums go into double-float accumulators on the
// FP32 pipes for single-precision and double-float storage (GB300's FP64
// pipe issues 1/64 as fast, and converting and adding every population in
// double made this reduction FP64-bound at ~10 % of HBM bandwidth): each
// site's eight sums are formed exactly in double-float (TwoSum of the
// single-precision values, or of the double-float pairs), added to the
// thread's running double-float totals, and only those totals are converted
// to double after a double-float warp sum.  The deviation codecs'
// reference part (sum over q of the fref terms, times N) is added once.
// FP64 storage sums in double.
__device__ __forceinline__ df as_df(float v) { return df(v, 0.f); }
__device__ __forceinline__ df as_df(df v) { return v; }

template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kRedBlock)
k_conserved_partial(const Planes<typename Codec::S, Lattice<D>::Q> pl, Grid g, Codec codec,
                    double *__restrict__ partials)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (std::is_same<R, double>::value) {
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
    } else {
        df tot[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) tot[k] = df(0.f, 0.f);
        for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.N; s += stride) {
            SiteIdx si;
            si.s = (int)s;
            si.x = (int)(s % g.nx);
            const int64_t row = s / g.nx;
            si.y = (int)(row % g.ny);
            si.z = (int)(row / g.ny);
            R f[Q], sx[Q], sy[Q], sz[Q];
            gather<D, Codec, SWAPPED>(pl, g, si, codec, f, sx, sy, sz);
            DFAcc a[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) a[k].set(df(0.f, 0.f));
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const df fq = as_df(f[q]);
                a[0].add(fq);
                a[1].add(as_df(sx[q]));
                a[2].add(as_df(sy[q]));
                a[3].add(as_df(sz[q]));
                if (cx<D>(q)) a[4].add(cx<D>(q) > 0 ? fq : -fq);
                if (cy<D>(q)) a[5].add(cy<D>(q) > 0 ? fq : -fq);
                if (cz<D>(q)) a[6].add(cz<D>(q) > 0 ? fq : -fq);
                if (cnorm2<D>(q)) a[7].add(scale2(fq, (float)cnorm2<D>(q)));
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) tot[k] = tot[k] + a[k].value();
        }
        // warp sum in double-float, then one conversion per warp
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            for (int o = 16; o > 0; o >>= 1) {
                const df other(__shfl_down_sync(0xffffffffu, tot[k].hi, o), __shfl_down_sync(0xffffffffu, tot[k].lo, o));
                tot[k] = tot[k] + other;
            }
            acc[k] = (threadIdx.x & 31) == 0 ? tot[k].to_double() : 0.0;
        }
        // reference part of a deviation codec (to_double(0, comp, cls) per
        // value), N times, once for the whole lattice
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double ref[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int cls = cnorm2<D>(q);
                const double r = codec.to_double(R(0), 0, cls);
                ref[0] += r;
                ref[4] += cx<D>(q) * r;
                ref[5] += cy<D>(q) * r;
                ref[6] += cz<D>(q) * r;
                ref[7] += cnorm2<D>(q) * r;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += (double)g.N * ref[k];
        }
        block_sum_lanes0<8>(acc, partials + (int64_t)blockIdx.x * 8);
        return;
    }
    block_sum_store<8>(acc, partials + (int64_t)blockIdx.x * 8);
}

// Sums nparts rows of 8 partials in a fixed order; out[0..7] then scaled:
// density /N, momentum xi/N, energy xi^2/(2N).
__global__ void __launch_bounds__(kRedBlock)
k_conserved_final(const double *__restrict__ partials, int nparts, double xi, int64_t N,
                  double *__restrict__ out);

}  // namespace qlbm
