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

// Weighted moments of a cotangent component over the directions:
// sum_i w_i v_i (1, i, |i|^2, i i^T), accumulated one direction at a time.
template <typename R> struct MuMom {
    R m0, mx, my, mz, m2, xx, yy, zz, xy, xz, yz;
    __device__ __forceinline__ void zero() { m0 = mx = my = mz = m2 = xx = yy = zz = xy = xz = yz = R(0); }
    template <int D, int q> __device__ __forceinline__ void add(R a)
    {
        constexpr int X = cx<D>(q), Y = cy<D>(q), Z = cz<D>(q);
        m0 += a;
        if (X) mx += X * a;
        if (Y) my += Y * a;
        if (Z) mz += Z * a;
        if (X * X + Y * Y + Z * Z) m2 += (X * X + Y * Y + Z * Z) * a;
        if (X) xx += a;
        if (Y) yy += a;
        if (Z) zz += a;
        if (X * Y) xy += (X * Y) * a;
        if (X * Z) xz += (X * Z) * a;
        if (Y * Z) yz += (Y * Z) * a;
    }
    // sum_i w_i v_i P_i with P_i = 1 + a2 (K|i|^2 - c) + c3 i.j + c4 (i.j)^2 + c5 |j|^2
    __device__ __forceinline__ R wP(R a2, R K, R c, R c3, R c4, R c5, R jx, R jy, R jz, R jj) const
    {
        const R quad = jx * (xx * jx + xy * jy + xz * jz) + jy * (xy * jx + yy * jy + yz * jz) +
                       jz * (xz * jx + yz * jy + zz * jz);
        return m0 * (R(1) + c5 * jj) + a2 * (K * m2 - c * m0) + c3 * (mx * jx + my * jy + mz * jz) + c4 * quad;
    }
    // (sum_i w_i v_i i i^T) j
    __device__ __forceinline__ void Mj(R jx, R jy, R jz, R &ox, R &oy, R &oz) const
    {
        ox = xx * jx + xy * jy + xz * jz;
        oy = xy * jx + yy * jy + yz * jz;
        oz = xz * jx + yz * jy + zz * jz;
    }
};

// Cotangent of the pre-rotation spins: mu_s <- R^T mu_s (the field term
// rotates the post-collision spins by R).
template <typename R>
__device__ __forceinline__ void unrotate(R &mx, R &my, R &mz, const R (&rot)[9])
{
    const R x = mx, y = my, z = mz;
    mx = rot[0] * x + rot[3] * y + rot[6] * z;
    my = rot[1] * x + rot[4] * y + rot[7] * z;
    mz = rot[2] * x + rot[5] * y + rot[8] * z;
}

template <int D, class Codec, int q, int FIELD>
__device__ __forceinline__ void adj_accumulate(const Planes<typename Codec::S, Lattice<D>::Q> &st,
                                               const Planes<typename Codec::R, Lattice<D>::Q> &lin,
                                               const Grid &g, const SiteIdx &si, const Codec &codec,
                                               const Coll<typename Codec::R> &k,
                                               const typename Codec::R (&rot)[9], typename Codec::R (&fw)[8],
                                               typename Codec::R &dot, MuMom<typename Codec::R> &A,
                                               MuMom<typename Codec::R> &Bx, MuMom<typename Codec::R> &By,
                                               MuMom<typename Codec::R> &Bz)
{
    using R = typename Codec::R;
    R f, sx, sy, sz;
    codec.load4(st.p[q] + si.s, f, sx, sy, sz);
    const int s = neighbour(g, si, cx<D>(q), cy<D>(q), cz<D>(q));
    R mf, mx, my, mz;
    ldq(lin.p[q] + s, mf, mx, my, mz);
    if constexpr (FIELD != FIELD_NONE) unrotate(mx, my, mz, rot);
    fw[0] += f;
    fw[1] += sx;
    fw[2] += sy;
    fw[3] += sz;
    if (cx<D>(q)) fw[4] += cx<D>(q) * f;
    if (cy<D>(q)) fw[5] += cy<D>(q) * f;
    if (cz<D>(q)) fw[6] += cz<D>(q) * f;
    if (cnorm2<D>(q)) fw[7] += cnorm2<D>(q) * f;
    dot += mf * f + mx * sx + my * sy + mz * sz;
    const R w = k.w[cnorm2<D>(q)];
    A.template add<D, q>(w * mf);
    Bx.template add<D, q>(w * mx);
    By.template add<D, q>(w * my);
    Bz.template add<D, q>(w * mz);
}

template <int D, class Codec, int q, int FIELD>
struct AdjLoop {
    static __device__ __forceinline__ void run(const Planes<typename Codec::S, Lattice<D>::Q> &st,
                                               const Planes<typename Codec::R, Lattice<D>::Q> &lin,
                                               const Grid &g, const SiteIdx &si, const Codec &codec,
                                               const Coll<typename Codec::R> &k,
                                               const typename Codec::R (&rot)[9], typename Codec::R (&fw)[8],
                                               typename Codec::R &dot, MuMom<typename Codec::R> &A,
                                               MuMom<typename Codec::R> &Bx, MuMom<typename Codec::R> &By,
                                               MuMom<typename Codec::R> &Bz)
    {
        adj_accumulate<D, Codec, q, FIELD>(st, lin, g, si, codec, k, rot, fw, dot, A, Bx, By, Bz);
        AdjLoop<D, Codec, q + 1, FIELD>::run(st, lin, g, si, codec, k, rot, fw, dot, A, Bx, By, Bz);
    }
};
template <int D, class Codec, int FIELD> struct AdjLoop<D, Codec, Lattice<D>::Q, FIELD> {
    static __device__ __forceinline__ void run(const Planes<typename Codec::S, Lattice<D>::Q> &,
                                               const Planes<typename Codec::R, Lattice<D>::Q> &,
                                               const Grid &, const SiteIdx &, const Codec &,
                                               const Coll<typename Codec::R> &,
                                               const typename Codec::R (&)[9], typename Codec::R (&)[8],
                                               typename Codec::R &, MuMom<typename Codec::R> &,
                                               MuMom<typename Codec::R> &, MuMom<typename Codec::R> &,
                                               MuMom<typename Codec::R> &)
    {
    }
};

// One reverse step.  state: W^n in natural order; lam_in: lambda^{n+1};
// lam_out: lambda^n (natural order, arithmetic type R).  dtau_acc[block] +=
// this block's sum_k mu_k.(W^eq_k - W_k) (times d omega/d tau on the host).
//
// Pass 1 reads W^n and mu together and folds them straight into
// accumulators: the forward moments, sum_k mu_k.W_k, and the weighted
// cotangent moments sum_k w_k mu_k (1, i_k, |i_k|^2, i_k i_k^T).  Every
// per-direction sum of the transpose above is a polynomial of degree <= 2 in
// i_k times w_k mu_k, so these moments give them once the forward moments
// are known.  Pass 2 re-reads mu (cache hits; the index carries the
// run-time zero so the compiler does not keep pass 1's values live) and
// writes lambda^n.
template <int D, class Codec, int FIELD>
__global__ void __launch_bounds__(kAdjBlock, Codec::MIN_BLOCKS)
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
        R fw[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};   // sum f, S, J, E2
        R dot = R(0);
        MuMom<R> A, Bx, By, Bz;
        A.zero();
        Bx.zero();
        By.zero();
        Bz.zero();
        // the field term's rotation at this site (the forward step rotates
        // the spins collided here; their cotangents take its transpose)
        R rot[9];
        if constexpr (FIELD != FIELD_NONE) field_rotation<FIELD>(k, si.s, rot);
        AdjLoop<D, Codec, 0, FIELD>::run(st, lin, g, si, codec, k, rot, fw, dot, A, Bx, By, Bz);
        // forward moments
        const R dn = DEV ? fw[0] : fw[0] - R(1);
        const R n = DEV ? R(1) + fw[0] : fw[0];
        const R rn = R(1) / n;
        const R Sx = fw[1], Sy = fw[2], Sz = fw[3];
        const R jx = fw[4] * rn, jy = fw[5] * rn, jz = fw[6] * rn;
        const R jj = jx * jx + jy * jy + jz * jz;
        const R de = DEV ? (fw[7] - k.S2 * fw[0]) * rn : fw[7] * rn - k.S2;   // E2/n - S2
        const R e2n = k.S2 + de;
        const R a2 = k.K * (de - jj) * k.inv_mc2;
        // sum_k w_k P_k mu_k
        const R Af = A.wP(a2, k.K, k.c, k.c3, k.c4, k.c5, jx, jy, jz, jj);
        const R Asx = Bx.wP(a2, k.K, k.c, k.c3, k.c4, k.c5, jx, jy, jz, jj);
        const R Asy = By.wP(a2, k.K, k.c, k.c3, k.c4, k.c5, jx, jy, jz, jj);
        const R Asz = Bz.wP(a2, k.K, k.c, k.c3, k.c4, k.c5, jx, jy, jz, jj);
        // Pbar_k / omega = n w_k mu_f,k + S.w_k mu_s,k  ->  its moments
        const R p0 = n * A.m0 + Sx * Bx.m0 + Sy * By.m0 + Sz * Bz.m0;
        const R p2 = n * A.m2 + Sx * Bx.m2 + Sy * By.m2 + Sz * Bz.m2;
        const R p1x = n * A.mx + Sx * Bx.mx + Sy * By.mx + Sz * Bz.mx;
        const R p1y = n * A.my + Sx * Bx.my + Sy * By.my + Sz * Bz.my;
        const R p1z = n * A.mz + Sx * Bx.mz + Sy * By.mz + Sz * Bz.mz;
        R qx, qy, qz, tx, ty, tz;
        A.Mj(jx, jy, jz, qx, qy, qz);
        qx *= n;
        qy *= n;
        qz *= n;
        Bx.Mj(jx, jy, jz, tx, ty, tz);
        qx += Sx * tx;
        qy += Sx * ty;
        qz += Sx * tz;
        By.Mj(jx, jy, jz, tx, ty, tz);
        qx += Sy * tx;
        qy += Sy * ty;
        qz += Sy * tz;
        Bz.Mj(jx, jy, jz, tx, ty, tz);
        qx += Sz * tx;
        qy += Sz * ty;
        qz += Sz * tz;
        const R sP = k.omega * p0;
        const R G = k.omega * (k.K * p2 - k.c * p0);
        const R cj = R(2) * (k.c5 * sP - k.K * k.inv_mc2 * G);
        const R jbx = k.omega * (k.c3 * p1x + R(2) * k.c4 * qx) + cj * jx;
        const R jby = k.omega * (k.c3 * p1y + R(2) * k.c4 * qy) + cj * jy;
        const R jbz = k.omega * (k.c3 * p1z + R(2) * k.c4 * qz) + cj * jz;
        const R ebar = k.K * k.inv_mc2 * G;
        const R nbar = k.omega * Af - (jbx * jx + jby * jy + jbz * jz + ebar * e2n) * rn;
        const R Jbx2 = jbx * rn, Jby2 = jby * rn, Jbz2 = jbz * rn, Eb = ebar * rn;
        const R omc = R(1) - k.omega;
        const R Sbx = k.omega * Asx, Sby = k.omega * Asy, Sbz = k.omega * Asz;
        // sum_k mu_k.(W^eq_k - W_k): f-part n Af - sum mu_f f (deviation form
        // subtracts sum w mu_f = A.m0 as well), spin part S.As - sum mu_s.s
        const R eqdot = (DEV ? (Af - A.m0) + dn * Af : n * Af) + Sx * Asx + Sy * Asy + Sz * Asz;
        dtau = (double)(eqdot - dot);
        // pass 2: lambda^n
        SiteIdx s2 = si;
        s2.s += g.zero;
        s2.x += g.zero;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int s = neighbour(g, s2, cx<D>(q), cy<D>(q), cz<D>(q));
            R mf, mx, my, mz;
            ldq(lin.p[q] + s, mf, mx, my, mz);
            if constexpr (FIELD != FIELD_NONE) unrotate(mx, my, mz, rot);
            stq(lout.p[q] + s2.s,
                omc * mf + nbar + (cx<D>(q) * Jbx2 + cy<D>(q) * Jby2 + cz<D>(q) * Jbz2) + cnorm2<D>(q) * Eb,
                omc * mx + Sbx, omc * my + Sby, omc * mz + Sbz);
        }
    }
    const double bs = block_sum_double<R>(dtau);
    if (threadIdx.x == 0) dtau_acc[blockIdx.x] += bs;
}

// Two-buffer forward step (push): src and dst in natural order.  Used to
// recompute the states inside a checkpoint segment.
template <int D, class Codec, int FIELD>
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
    const unsigned flag = Codec::template collide<D>(f, sx, sy, sz, k);
    apply_field<D, FIELD, R>(sx, sy, sz, k, si.s);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int s = neighbour(g, si, cx<D>(q), cy<D>(q), cz<D>(q));
        codec.store4(dst.p[q] + s, f[q], sx[q], sy[q], sz[q]);
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
    for (int q = 0; q < Q; ++q) codec.store4(dst.p[q] + si.s, f[q], sx[q], sy[q], sz[q]);
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
    const int64_t N = g.N;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const double *v = in + (int64_t)(4 * q) * N + si.s;
        stq(lam.p[q] + si.s, (R)v[0], (R)v[N], (R)v[2 * N], (R)v[3 * N]);
    }
}

template <int D, typename R>
__global__ void __launch_bounds__(kStepBlock)
k_lam_export(const Planes<R, Lattice<D>::Q> lam, Grid g, double *__restrict__ out)
{
    constexpr int Q = Lattice<D>::Q;
    SiteIdx si;
    if (!site_of_block(g, si)) return;
    const int64_t N = g.N;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        R a, b, c, d;
        ldq(lam.p[q] + si.s, a, b, c, d);
        double *o = out + (int64_t)(4 * q) * N + si.s;
        o[0] = (double)a;
        o[N] = (double)b;
        o[2 * N] = (double)c;
        o[3 * N] = (double)d;
    }
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
