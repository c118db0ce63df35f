// Reverse mode of the step (differentiation of Sec. 3.3 by the chain rule)
// and the kernels the checkpointed rollout needs.
//
// Forward map per site, in Pauli components (W = (f 1 + s.sigma)/2):
//   f_i' = f_i + omega (w_i P_i n - f_i),  s_i' = s_i + omega (w_i P_i S - s_i),
//   P_i = 1 + P1_i,  P1_i = alpha2 (K|i|^2 - c) + c3 t_i + c4 t_i^2 + c5 |j|^2,
//   t_i = i.j,  j = J/n,  alpha2 = (K (E2/n - |j|^2) - c)/(m - c^2),
// followed by streaming W^{n+1}_i(x + e_i) = W'_i(x) (Eqs. WeqAlgo,
// CollisionStep, TransportStep).  With mu_i(x) = lambda^{n+1}_i(x + e_i) the
// cotangent of W'_i(x) (streaming is a permutation), the transpose of the
// collision Jacobian is
//   lambda_s,i = (1-omega) mu_s,i + omega sum_k w_k P_k mu_s,k,
//   lambda_f,i = (1-omega) mu_f,i + nbar + i.Jbar + |i|^2 Ebar,
// where, with Pbar_k = omega w_k (n mu_f,k + S.mu_s,k),
//   G = sum_k Pbar_k (K|i_k|^2 - c),
//   jbar = sum_k Pbar_k (c3 + 2 c4 t_k) i_k + 2 j (c5 sum_k Pbar_k - K G/(m-c^2)),
//   ebar = K G/(m-c^2),
//   nbar = omega sum_k w_k P_k mu_f,k - (jbar.j + ebar E2/n)/n,
//   Jbar = jbar/n,  Ebar = ebar/n,
// and dJ/dtau gets (d omega/d tau) sum_k mu_k . (W_k^eq - W_k).
// The single-precision kernels' rounding corrections vanish in exact
// arithmetic and are not differentiated.
#pragma once

#include "kernels.cuh"

namespace qlbm {

constexpr int kAdjBlock = 128;

// Forward moments of one site in either representation (DEV: deviations
// d_i = f_i - w_i), as needed by the adjoint.
template <int D, typename R, bool DEV> struct FwdSite {
    R n, dn, Sx, Sy, Sz, jx, jy, jz, e2n, jj, a2;
};

template <int D, typename R, bool DEV>
__device__ __forceinline__ FwdSite<D, R, DEV> forward_moments(const R *f, const R *sx, const R *sy,
                                                             const R *sz, const Coll<R> &k)
{
    constexpr int Q = Lattice<D>::Q;
    FwdSite<D, R, DEV> m;
    R sn = R(0), Sx = R(0), Sy = R(0), Sz = R(0), Jx = R(0), Jy = R(0), Jz = R(0), E = R(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        sn += f[q];
        Sx += sx[q];
        Sy += sy[q];
        Sz += sz[q];
        Jx += cx<D>(q) * f[q];
        Jy += cy<D>(q) * f[q];
        Jz += cz<D>(q) * f[q];
        E += cnorm2<D>(q) * f[q];
    }
    m.dn = DEV ? sn : sn - R(1);
    m.n = DEV ? R(1) + sn : sn;
    const R rn = R(1) / m.n;
    m.Sx = Sx;
    m.Sy = Sy;
    m.Sz = Sz;
    m.jx = Jx * rn;
    m.jy = Jy * rn;
    m.jz = Jz * rn;
    m.jj = m.jx * m.jx + m.jy * m.jy + m.jz * m.jz;
    R de;   // E2/n - S2
    if (DEV) {
        de = (E - k.S2 * sn) * rn;
        m.e2n = k.S2 + de;
    } else {
        m.e2n = E * rn;
        de = m.e2n - k.S2;
    }
    // K (E2/n - |j|^2) - c = K (de - |j|^2)  (c = K S2)
    m.a2 = k.K * (de - m.jj) * k.inv_mc2;
    return m;
}

template <int D, typename R, bool DEV>
__device__ __forceinline__ R P1_of(const FwdSite<D, R, DEV> &m, const Coll<R> &k, int q)
{
    const R t = cx<D>(q) * m.jx + cy<D>(q) * m.jy + cz<D>(q) * m.jz;
    return m.a2 * (k.K * cnorm2<D>(q) - k.c) + t * (k.c3 + k.c4 * t) + k.c5 * m.jj;
}

template <typename R>
__device__ __forceinline__ double block_sum_double(double v)
{
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double acc = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += sh[w];
    return acc;
}

// One reverse step.  state: W^n in natural order; lam_in: lambda^{n+1};
// lam_out: lambda^n (natural order, arithmetic type R).  dtau_acc[block] +=
// this block's sum_k mu_k.(W^eq_k - W_k) (times d omega/d tau on the host).
template <int D, class Codec>
__global__ void __launch_bounds__(kAdjBlock)
k_adjoint(const Planes<typename Codec::S, Lattice<D>::Q> st, const Planes<typename Codec::R, Lattice<D>::Q> lin,
          const Planes<typename Codec::R, Lattice<D>::Q> lout, Grid g, Coll<typename Codec::R> k,
          Codec codec, double *__restrict__ dtau_acc)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    constexpr bool DEV = Codec::DEV;
    SiteIdx si;
    const bool active = site_of_block(g, si);
    double dtau = 0.0;
    if (active) {
        R f[Q], sx[Q], sy[Q], sz[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            f[q] = codec.load(st.p[4 * q][si.s]);
            sx[q] = codec.load(st.p[4 * q + 1][si.s]);
            sy[q] = codec.load(st.p[4 * q + 2][si.s]);
            sz[q] = codec.load(st.p[4 * q + 3][si.s]);
        }
        const FwdSite<D, R, DEV> m = forward_moments<D, R, DEV>(f, sx, sy, sz, k);
        R Af = R(0), Asx = R(0), Asy = R(0), Asz = R(0), sP = R(0), G = R(0);
        R Jbx = R(0), Jby = R(0), Jbz = R(0);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int s = neighbour(g, si, cx<D>(q), cy<D>(q), cz<D>(q));
            const R mf = lin.p[4 * q][s], mx = lin.p[4 * q + 1][s], my = lin.p[4 * q + 2][s],
                    mz = lin.p[4 * q + 3][s];
            const R w = k.w[cnorm2<D>(q)];
            const R P1 = P1_of<D, R, DEV>(m, k, q);
            const R wP = w * (R(1) + P1);
            Af += wP * mf;
            Asx += wP * mx;
            Asy += wP * my;
            Asz += wP * mz;
            const R Pbar = k.omega * w * (m.n * mf + m.Sx * mx + m.Sy * my + m.Sz * mz);
            sP += Pbar;
            G += Pbar * (k.K * cnorm2<D>(q) - k.c);
            const R t = cx<D>(q) * m.jx + cy<D>(q) * m.jy + cz<D>(q) * m.jz;
            const R T = Pbar * (k.c3 + R(2) * k.c4 * t);
            Jbx += cx<D>(q) * T;
            Jby += cy<D>(q) * T;
            Jbz += cz<D>(q) * T;
            // W^eq - W: f-part (deviation form: w ((P-1) n + dn) - d)
            const R feq_minus = DEV ? w * (P1 * m.n + m.dn) - f[q] : wP * m.n - f[q];
            dtau += (double)(mf * feq_minus + mx * (wP * m.Sx - sx[q]) + my * (wP * m.Sy - sy[q]) +
                             mz * (wP * m.Sz - sz[q]));
        }
        const R rn = R(1) / m.n;
        const R cj = R(2) * (k.c5 * sP - k.K * k.inv_mc2 * G);
        const R jbx = Jbx + cj * m.jx, jby = Jby + cj * m.jy, jbz = Jbz + cj * m.jz;
        const R ebar = k.K * k.inv_mc2 * G;
        const R nbar = k.omega * Af - (jbx * m.jx + jby * m.jy + jbz * m.jz + ebar * m.e2n) * rn;
        const R Jx = jbx * rn, Jy = jby * rn, Jz = jbz * rn, Eb = ebar * rn;
        const R omc = R(1) - k.omega;
        // second pass: mu reloaded (offset by the run-time zero so the first
        // pass's 4b values are not kept live in registers)
        SiteIdx so = si;
        so.s += g.zero;
        so.x += g.zero;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int s = neighbour(g, so, cx<D>(q), cy<D>(q), cz<D>(q));
            const R mf = lin.p[4 * q][s], mx = lin.p[4 * q + 1][s], my = lin.p[4 * q + 2][s],
                    mz = lin.p[4 * q + 3][s];
            lout.p[4 * q][so.s] = omc * mf + nbar + (cx<D>(q) * Jx + cy<D>(q) * Jy + cz<D>(q) * Jz) +
                                  cnorm2<D>(q) * Eb;
            lout.p[4 * q + 1][so.s] = omc * mx + k.omega * Asx;
            lout.p[4 * q + 2][so.s] = omc * my + k.omega * Asy;
            lout.p[4 * q + 3][so.s] = omc * mz + k.omega * Asz;
        }
    }
    const double bs = block_sum_double<R>(dtau);
    if (threadIdx.x == 0) dtau_acc[blockIdx.x] += bs;
}

// Two-buffer forward step (push): src and dst in natural order.  Used to
// recompute the states inside a checkpoint segment.
template <int D, class Codec>
__global__ void __launch_bounds__(kStepBlock, Codec::MIN_BLOCKS)
k_step_push(const Planes<typename Codec::S, Lattice<D>::Q> src, const Planes<typename Codec::S, Lattice<D>::Q> dst,
            Grid g, Coll<typename Codec::R> k, Codec codec, unsigned *__restrict__ flags)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    R f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, false>(src, g, si, codec, f, sx, sy, sz);
    unsigned flag;
    if constexpr (Codec::DEV)
        flag = collide_dev<D>(f, sx, sy, sz, k);
    else
        flag = collide<D, R>(f, sx, sy, sz, k);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int s = neighbour(g, si, cx<D>(q), cy<D>(q), cz<D>(q));
        dst.p[4 * q][s] = codec.store(f[q]);
        dst.p[4 * q + 1][s] = codec.store(sx[q]);
        dst.p[4 * q + 2][s] = codec.store(sy[q]);
        dst.p[4 * q + 3][s] = codec.store(sz[q]);
    }
    if (flag) atomicOr(flags, flag);
}

// Copy of the live (AA-ordered) buffer into natural order.
template <int D, class Codec, bool SWAPPED>
__global__ void __launch_bounds__(kStepBlock)
k_copy_natural(const Planes<typename Codec::S, Lattice<D>::Q> src, const Planes<typename Codec::S, Lattice<D>::Q> dst,
               Grid g, Codec codec)
{
    using R = typename Codec::R;
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    R f[Q], sx[Q], sy[Q], sz[Q];
    gather<D, Codec, SWAPPED>(src, g, si, codec, f, sx, sy, sz);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        dst.p[4 * q][si.s] = codec.store(f[q]);
        dst.p[4 * q + 1][si.s] = codec.store(sx[q]);
        dst.p[4 * q + 2][si.s] = codec.store(sy[q]);
        dst.p[4 * q + 3][si.s] = codec.store(sz[q]);
    }
}

// Cotangent conversion between the canonical double layout [b][4][N] and the
// internal planes of type R.
template <int D, typename R>
__global__ void __launch_bounds__(kStepBlock)
k_lam_import(const double *__restrict__ in, const Planes<R, Lattice<D>::Q> lam, Grid g)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
#pragma unroll
    for (int k = 0; k < 4 * Q; ++k) lam.p[k][si.s] = (R)in[(int64_t)k * g.N + si.s];
}

template <int D, typename R>
__global__ void __launch_bounds__(kStepBlock)
k_lam_export(const Planes<R, Lattice<D>::Q> lam, Grid g, double *__restrict__ out)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
#pragma unroll
    for (int k = 0; k < 4 * Q; ++k) out[(int64_t)k * g.N + si.s] = (double)lam.p[k][si.s];
}

// Adjoint of the equilibrium initialisation W_i = w_i P_i(u, eps) rho
// (Eq. WeqAlgo with given u and eps): gradients with respect to rho4
// (n, S), u and eps, in double.
template <int D>
__global__ void __launch_bounds__(kStepBlock)
k_init_adjoint(const double *__restrict__ lam, Grid g, InitConsts ic, const double *__restrict__ rho4,
               const double *__restrict__ u, const double *__restrict__ eps, double *__restrict__ grho4,
               double *__restrict__ gu, double *__restrict__ geps)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    const int64_t N = g.N, s = si.s;
    const double n = rho4[s], Sx = rho4[N + s], Sy = rho4[2 * N + s], Sz = rho4[3 * N + s];
    const double jx = u[s] / ic.xi, jy = u[N + s] / ic.xi, jz = (D == 3) ? u[2 * N + s] / ic.xi : 0.0;
    const double e = eps ? eps[s] : ic.eps0;
    const double be = ic.beta0 * e;
    double gn = 0, gx = 0, gy = 0, gz = 0, gjx = 0, gjy = 0, gjz = 0, gbe = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int cls = cnorm2<D>(q);
        const double w = ic.w[cls];
        const double P = poly_P_d<D>(ic, q, jx, jy, jz, be);
        const double lf = lam[(int64_t)(4 * q) * N + s], lx = lam[(int64_t)(4 * q + 1) * N + s],
                     ly = lam[(int64_t)(4 * q + 2) * N + s], lz = lam[(int64_t)(4 * q + 3) * N + s];
        gn += w * P * lf;
        gx += w * P * lx;
        gy += w * P * ly;
        gz += w * P * lz;
        const double Pb = w * (n * lf + Sx * lx + Sy * ly + Sz * lz);   // cotangent of P_q
        const double t = cx<D>(q) * jx + cy<D>(q) * jy + cz<D>(q) * jz;
        const double dPdt = ic.c3 + 2.0 * ic.c4 * t;
        gjx += Pb * (dPdt * cx<D>(q) + 2.0 * ic.c5 * jx);
        gjy += Pb * (dPdt * cy<D>(q) + 2.0 * ic.c5 * jy);
        gjz += Pb * (dPdt * cz<D>(q) + 2.0 * ic.c5 * jz);
        // P = alpha1 + alpha2 K|i|^2 + ..., alpha2 = (be - c)/(m - c^2), alpha1 = 1 - c alpha2
        gbe += Pb * ic.inv_mc2 * (ic.K * cls - ic.c);
    }
    if (grho4) {
        grho4[s] = gn;
        grho4[N + s] = gx;
        grho4[2 * N + s] = gy;
        grho4[3 * N + s] = gz;
    }
    if (gu) {
        gu[s] = gjx / ic.xi;
        gu[N + s] = gjy / ic.xi;
        if (D == 3) gu[2 * N + s] = gjz / ic.xi;
    }
    if (geps) geps[s] = gbe * ic.beta0;
}

}  // namespace qlbm
