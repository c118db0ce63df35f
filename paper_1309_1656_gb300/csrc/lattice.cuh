// Device-side lattice description and the per-site collision of the
// matrix-valued quantum lattice Boltzmann step (Mendl, Sec. 3.3).
//
// Populations are held in Pauli form (f, s) with W = (f 1 + s.sigma)/2.
// Because u and eps only depend on the traces f_i (Eq. DiscrAvr) and the
// equilibrium is W_i^eq = w_i P_i rho (Eq. WeqAlgo) with one scalar P_i per
// direction, the collision splits into
//   f_i' = (1-omega) f_i + omega w_i P_i n,    n = sum_j f_j = tr rho,
//   s_i' = (1-omega) s_i + omega w_i P_i S,    S = sum_j s_j = tr(rho sigma),
// which is Eq. CollisionStep written component-wise.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qlbm {

template <int D> struct Lattice;
template <> struct Lattice<2> { static constexpr int Q = 9; };
template <> struct Lattice<3> { static constexpr int Q = 19; };

// Position of direction q in the 3x3x3 cube of lattice vectors,
// r = (i1+1) + 3(i2+1) + 9(i3+1).  D2Q9 uses the i3 = 0 layer; D3Q19 drops
// the eight corners (Sec. 3.1).  q runs over the kept vectors in increasing r.
template <int D> __host__ __device__ constexpr int cube_index(int q)
{
    return D == 2 ? q + 9
                  : (q < 5 ? (q == 0 ? 1 : (q == 4 ? 7 : q + 2))
                           : (q < 14 ? q + 4 : (q == 14 ? 19 : (q == 18 ? 25 : q + 6))));
}
template <int D> __host__ __device__ constexpr int cx(int q) { return cube_index<D>(q) % 3 - 1; }
template <int D> __host__ __device__ constexpr int cy(int q) { return (cube_index<D>(q) / 3) % 3 - 1; }
template <int D> __host__ __device__ constexpr int cz(int q) { return cube_index<D>(q) / 9 - 1; }
template <int D> __host__ __device__ constexpr int cnorm2(int q)
{
    return cx<D>(q) * cx<D>(q) + cy<D>(q) * cy<D>(q) + cz<D>(q) * cz<D>(q);
}
template <int D> __host__ __device__ constexpr int opposite(int q) { return Lattice<D>::Q - 1 - q; }

// Per-handle collision constants in the kernel's arithmetic type.  With
// j = J/n in lattice units (u = xi j) and K = beta0 xi^2 / 2:
//   beta0 eps = K (E2/n - |j|^2),            E2 = sum_i |i|^2 f_i,
//   alpha2 = (beta0 eps - c)/(m - c^2),      alpha1 = 1 - c alpha2,
//   P_i = alpha1 + alpha2 K |i|^2 + c3 (i.j) + c4 (i.j)^2 + c5 |j|^2,
// with c3 = 2K alpha3, c4 = 4K^2 alpha4, c5 = K alpha5 (Eq. WeqAlgo).
template <typename R> struct Coll {
    R K, c, inv_mc2;
    R c3, c4, c5;
    R omega, omc;   // dt/tau and 1 - dt/tau
    R ow[3];        // omega * w for |i|^2 = 0, 1, 2
};

// Bits of the device flag word.
enum : unsigned { FLAG_NONFINITE = 1u, FLAG_NONPOSITIVE = 2u };

template <typename R> __device__ __forceinline__ R fmadd(R a, R b, R c);
template <> __device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
template <> __device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }

// Moments of Eq. DiscrAvr in lattice units: n, S, j = J/n, E2/n.
template <int D, typename R> struct SiteMoments {
    R n, Sx, Sy, Sz, jx, jy, jz, e2n;
};

template <int D, typename R>
__device__ __forceinline__ SiteMoments<D, R> site_moments(const R *f, const R *sx, const R *sy,
                                                         const R *sz)
{
    constexpr int Q = Lattice<D>::Q;
    SiteMoments<D, R> m;
    R n = R(0), Sx = R(0), Sy = R(0), Sz = R(0);
    R jxp = R(0), jxm = R(0), jyp = R(0), jym = R(0), jzp = R(0), jzm = R(0);
    R e1 = R(0), e2 = R(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        n += f[q];
        Sx += sx[q];
        Sy += sy[q];
        Sz += sz[q];
        if (cx<D>(q) > 0) jxp += f[q];
        if (cx<D>(q) < 0) jxm += f[q];
        if (cy<D>(q) > 0) jyp += f[q];
        if (cy<D>(q) < 0) jym += f[q];
        if (cz<D>(q) > 0) jzp += f[q];
        if (cz<D>(q) < 0) jzm += f[q];
        if (cnorm2<D>(q) == 1) e1 += f[q];
        if (cnorm2<D>(q) == 2) e2 += f[q];
    }
    R rn = R(1) / n;
    m.n = n;
    m.Sx = Sx;
    m.Sy = Sy;
    m.Sz = Sz;
    m.jx = (jxp - jxm) * rn;
    m.jy = (jyp - jym) * rn;
    m.jz = (D == 3) ? (jzp - jzm) * rn : R(0);
    m.e2n = (e1 + R(2) * e2) * rn;
    return m;
}

// Fused equilibrium + BGK relaxation of one site, in place on the Pauli
// components (Eqs. WeqAlgo and CollisionStep).  Returns flag bits.
template <int D, typename R>
__device__ __forceinline__ unsigned collide(R *f, R *sx, R *sy, R *sz, const Coll<R> &k)
{
    constexpr int Q = Lattice<D>::Q;
    SiteMoments<D, R> m = site_moments<D, R>(f, sx, sy, sz);
    const R jj = m.jx * m.jx + m.jy * m.jy + m.jz * m.jz;
    const R be = k.K * (m.e2n - jj);        // beta0 * eps
    const R a2 = (be - k.c) * k.inv_mc2;    // alpha2
    const R a1 = R(1) - k.c * a2;           // alpha1
    const R b0 = fmadd(k.c5, jj, a1);
    const R a2K = a2 * k.K;
    const R bq[3] = {b0, b0 + a2K, b0 + R(2) * a2K};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        R t = R(0);
        if (cx<D>(q) > 0) t += m.jx;
        if (cx<D>(q) < 0) t -= m.jx;
        if (cy<D>(q) > 0) t += m.jy;
        if (cy<D>(q) < 0) t -= m.jy;
        if (cz<D>(q) > 0) t += m.jz;
        if (cz<D>(q) < 0) t -= m.jz;
        const R P = fmadd(t, fmadd(k.c4, t, k.c3), bq[cnorm2<D>(q)]);
        const R g = k.ow[cnorm2<D>(q)] * P;
        f[q] = fmadd(g, m.n, k.omc * f[q]);
        sx[q] = fmadd(g, m.Sx, k.omc * sx[q]);
        sy[q] = fmadd(g, m.Sy, k.omc * sy[q]);
        sz[q] = fmadd(g, m.Sz, k.omc * sz[q]);
    }
    unsigned flag = 0u;
    if (!(m.n > R(0))) flag |= (m.n == m.n) ? FLAG_NONPOSITIVE : FLAG_NONFINITE;
    if (!(fabs(m.Sx) + fabs(m.Sy) + fabs(m.Sz) + fabs(be) < R(1e30))) flag |= FLAG_NONFINITE;
    return flag;
}

// Storage codecs: how a stored value becomes an arithmetic value and back.
struct CodecF64 {
    using S = double;
    using R = double;
    __device__ __forceinline__ R load(S v, int, int) const { return v; }
    __device__ __forceinline__ S store(R v, int, int) const { return v; }
};
struct CodecF32 {
    using S = float;
    using R = float;
    __device__ __forceinline__ R load(S v, int, int) const { return v; }
    __device__ __forceinline__ S store(R v, int, int) const { return v; }
};
// Half-precision deviation from a uniform reference equilibrium: the trace
// component stores f_i - fref[|i|^2], the spin components (reference 0) are
// stored as they are.
struct CodecF16Dev {
    using S = __half;
    using R = float;
    float fref[3];
    __device__ __forceinline__ R load(S v, int comp, int cls) const
    {
        return comp == 0 ? fref[cls] + __half2float(v) : __half2float(v);
    }
    __device__ __forceinline__ S store(R v, int comp, int cls) const
    {
        return __float2half_rn(comp == 0 ? v - fref[cls] : v);
    }
};

// Extent and addressing of a lattice: plane stride P (elements) separates
// the b*4 component planes of the single population buffer.
struct Grid {
    int nx, ny, nz;
    int nxb;        // blocks per x-row
    int zero;       // always 0 (see k_step_aa)
    int64_t P;      // plane stride
    int64_t N;      // sites
};

__device__ __forceinline__ int wrapm(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

}  // namespace qlbm
