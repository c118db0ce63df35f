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

// Per-site field of the magnetic-field term: one unit quaternion per site,
// float4 for single-precision arithmetic, two double2 (DQuad) otherwise.
struct __align__(16) DQuad {
    double2 a, b;
};
template <typename R> struct FieldOf { using V = DQuad; };
template <> struct FieldOf<float> { using V = float4; };

// Per-handle collision constants in the kernel's arithmetic type.  With
// j = J/n in lattice units (u = xi j) and K = beta0 xi^2 / 2:
//   beta0 eps = K (E2/n - |j|^2),            E2 = sum_i |i|^2 f_i,
//   alpha2 = (beta0 eps - c)/(m - c^2),      alpha1 = 1 - c alpha2,
//   P_i = alpha1 + alpha2 K |i|^2 + c3 (i.j) + c4 (i.j)^2 + c5 |j|^2,
// with c3 = 2K alpha3, c4 = 4K^2 alpha4, c5 = K alpha5 (Eq. WeqAlgo).
// g00, g01, g11 invert the Gram matrix of (1, |i|^2) under the weights and
// gj = 1 / sum_i w_i i_x^2; they project rounding residuals out of the
// single-precision equilibrium (see collide).
template <typename R> struct Coll {
    R K, c, inv_mc2;
    R c3, c4, c5;
    R omega;        // dt/tau
    R w[3];         // weights for |i|^2 = 0, 1, 2
    R g00, g01, g11, gj;
    R S2;           // sum_i w_i |i|^2 (= c / K)
    R rot[9];       // spin rotation of a uniform magnetic field (row-major), if enabled
    const typename FieldOf<R>::V *qf;   // per-site field: unit quaternion of site s at qf[s], if enabled
};

// Magnetic-field term (Sec. 5): the Vlasov commutator -i[mu sigma.B, W]
// integrated exactly over one time step is W -> U W U*,
// U = exp(-i mu dt sigma.B), i.e. every Bloch vector s_i is rotated by
// 2 mu |B| dt about B (ds/dt = 2 mu B x s).  It commutes with the
// SU(2)-covariant collision, so applying it after the BGK update is exact.
// FIELD selects the kernels' variant: none, one field for the whole
// lattice (rotation matrix in Coll::rot), or a field B(x) per site (the
// rotation of site x from the unit quaternion (cos phi, sin phi B/|B|),
// phi = mu |B(x)| dt, which the library derives from B when it is set).
enum : int { FIELD_NONE = 0, FIELD_UNIFORM = 1, FIELD_SITE = 2 };

template <int D, typename R>
__device__ __forceinline__ void rotate_spins(R *sx, R *sy, R *sz, const R (&rot)[9])
{
    constexpr int Q = Lattice<D>::Q;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const R x = sx[q], y = sy[q], z = sz[q];
        sx[q] = rot[0] * x + rot[1] * y + rot[2] * z;
        sy[q] = rot[3] * x + rot[4] * y + rot[5] * z;
        sz[q] = rot[6] * x + rot[7] * y + rot[8] * z;
    }
}

// Rotation matrix of the unit quaternion (w, x, y, z): the rotation by
// 2 acos(w) about (x, y, z).
template <typename R>
__device__ __forceinline__ void quat_rotation(R w, R x, R y, R z, R (&rot)[9])
{
    const R xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    const R wx = w * x, wy = w * y, wz = w * z;
    rot[0] = R(1) - R(2) * (yy + zz);
    rot[1] = R(2) * (xy - wz);
    rot[2] = R(2) * (xz + wy);
    rot[3] = R(2) * (xy + wz);
    rot[4] = R(1) - R(2) * (xx + zz);
    rot[5] = R(2) * (yz - wx);
    rot[6] = R(2) * (xz - wy);
    rot[7] = R(2) * (yz + wx);
    rot[8] = R(1) - R(2) * (xx + yy);
}
__device__ __forceinline__ void load_quat(const float4 *p, float &w, float &x, float &y, float &z)
{
    const float4 v = *p;
    w = v.x;
    x = v.y;
    y = v.z;
    z = v.w;
}
__device__ __forceinline__ void load_quat(const DQuad *p, double &w, double &x, double &y, double &z)
{
    const double2 a = p->a, b = p->b;
    w = a.x;
    x = a.y;
    y = b.x;
    z = b.y;
}

// The spin rotation of the field term at site s: the uniform matrix, or the
// site's own from its quaternion.
template <int FIELD, typename R>
__device__ __forceinline__ void field_rotation(const Coll<R> &k, int s, R (&rot)[9])
{
    if constexpr (FIELD == FIELD_SITE) {
        R w, x, y, z;
        load_quat(k.qf + s, w, x, y, z);
        quat_rotation(w, x, y, z, rot);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) rot[i] = k.rot[i];
    }
}

// The field term applied to the post-collision spins of site s.
template <int D, int FIELD, typename R>
__device__ __forceinline__ void apply_field(R *sx, R *sy, R *sz, const Coll<R> &k, int s)
{
    if constexpr (FIELD != FIELD_NONE) {
        R rot[9];
        field_rotation<FIELD>(k, s, rot);
        rotate_spins<D, R>(sx, sy, sz, rot);
    }
}
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

// Fused equilibrium + BGK relaxation of one site on populations held as
// they are (double precision path), in place on the Pauli components:
// Eq. WeqAlgo and Eq. CollisionStep in the paper's form W' = W + omega (W^eq - W).
// Returns flag bits.
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
        const R t = cx<D>(q) * m.jx + cy<D>(q) * m.jy + cz<D>(q) * m.jz;
        const R h = k.w[cnorm2<D>(q)] * fmadd(t, fmadd(k.c4, t, k.c3), bq[cnorm2<D>(q)]);
        f[q] = fmadd(k.omega, fmadd(h, m.n, -f[q]), f[q]);
        sx[q] = fmadd(k.omega, fmadd(h, m.Sx, -sx[q]), sx[q]);
        sy[q] = fmadd(k.omega, fmadd(h, m.Sy, -sy[q]), sy[q]);
        sz[q] = fmadd(k.omega, fmadd(h, m.Sz, -sz[q]), sz[q]);
    }
    unsigned flag = 0u;
    if (!(m.n > R(0))) flag |= (m.n == m.n) ? FLAG_NONPOSITIVE : FLAG_NONFINITE;
    if (!(fabs(m.Sx) + fabs(m.Sy) + fabs(m.Sz) + fabs(be) < R(1e30))) flag |= FLAG_NONFINITE;
    return flag;
}

// The same collision in single precision on deviations from the uniform
// reference equilibrium (n = 1, S = 0, u = 0, eps = eps0, where P_i = 1):
// d_i = f_i - w_i and s_i as they are.  Every quantity formed is a small
// fluctuation, so no digits are lost to cancellation:
//   n = 1 + dn, dn = sum d_i;   j = J/n, J = sum i d_i   (sum w_i i = 0);
//   E2/n = S2 + de, de = (dE - S2 dn)/n, dE = sum |i|^2 d_i, S2 = sum w_i |i|^2;
//   beta0 eps - c = K (de - |j|^2)                       (c = K S2);
//   P_i - 1 = -c alpha2 + alpha2 K |i|^2 + c3 t + c4 t^2 + c5 |j|^2, t = i.j;
//   g_i = f_i^eq - w_i = w_i ((P_i - 1) n + dn),   s_i^eq = w_i P_i S.
// Exact moments: in exact arithmetic sum g_i = dn, sum g_i i = J and
// sum g_i |i|^2 = dE (Sec. 3.2), so the collision conserves mass, momentum
// and energy.  Rounded constants make these sums miss by ~1e-8..1e-7 in the
// same direction at every site and step (a drift of ~1e-5 over 1000
// steps).  A first pass measures the residuals of g against the moments of
// the inputs and removes them by the weighted least-change correction
// g_i -= w_i (A + B.i + C |i|^2) (which only shifts the base coefficients
// and adds one linear term); the rest population then takes the exact mass
// and spin balance.  What remains is unbiased rounding.
// With MOM, mom receives the site's n, S_x, S_y, S_z and beta0 eps (the
// conserved moments the equilibrium was built from).
template <int D, bool MOM = false>
__device__ __forceinline__ unsigned collide_dev(float *d, float *sx, float *sy, float *sz,
                                                const Coll<float> &k, float *mom = nullptr)
{
    constexpr int Q = Lattice<D>::Q;
    constexpr int REST = (Q - 1) / 2;
    float dn = 0.f, Sx = 0.f, Sy = 0.f, Sz = 0.f;
    float jxp = 0.f, jxm = 0.f, jyp = 0.f, jym = 0.f, jzp = 0.f, jzm = 0.f, e1 = 0.f, e2 = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        dn += d[q];
        Sx += sx[q];
        Sy += sy[q];
        Sz += sz[q];
        if (cx<D>(q) > 0) jxp += d[q];
        if (cx<D>(q) < 0) jxm += d[q];
        if (cy<D>(q) > 0) jyp += d[q];
        if (cy<D>(q) < 0) jym += d[q];
        if (cz<D>(q) > 0) jzp += d[q];
        if (cz<D>(q) < 0) jzm += d[q];
        if (cnorm2<D>(q) == 1) e1 += d[q];
        if (cnorm2<D>(q) == 2) e2 += d[q];
    }
    const float n = 1.f + dn;
    const float rn = 1.f / n;
    const float Jx = jxp - jxm, Jy = jyp - jym, Jz = (D == 3) ? jzp - jzm : 0.f;
    const float dE = e1 + 2.f * e2;
    const float jx = Jx * rn, jy = Jy * rn, jz = Jz * rn;
    const float de = fmaf(-k.S2, dn, dE) * rn;
    const float jj = jx * jx + jy * jy + jz * jz;
    const float a2 = k.K * (de - jj) * k.inv_mc2;          // alpha2
    const float a2K = a2 * k.K;
    const float p0 = fmaf(k.c5, jj, -k.c * a2);            // alpha1 - 1 + alpha5 K |j|^2
    float bq[3] = {p0, p0 + a2K, p0 + 2.f * a2K};
    // residual pass
    float s0 = 0.f, s2 = 0.f, sxp = 0.f, syp = 0.f, szp = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const float t = cx<D>(q) * jx + cy<D>(q) * jy + cz<D>(q) * jz;
        const float P1 = fmaf(t, fmaf(k.c4, t, k.c3), bq[cnorm2<D>(q)]);
        const float g = k.w[cnorm2<D>(q)] * fmaf(P1, n, dn);
        s0 += g;
        if (cnorm2<D>(q) == 1) s2 += g;
        if (cnorm2<D>(q) == 2) s2 += 2.f * g;
        if (cx<D>(q) > 0) sxp += g;
        if (cx<D>(q) < 0) sxp -= g;
        if (cy<D>(q) > 0) syp += g;
        if (cy<D>(q) < 0) syp -= g;
        if (cz<D>(q) > 0) szp += g;
        if (cz<D>(q) < 0) szp -= g;
    }
    const float r0 = s0 - dn, r2 = s2 - dE;
    const float A = (k.g00 * r0 + k.g01 * r2) * rn;
    const float C = (k.g01 * r0 + k.g11 * r2) * rn;
    const float Bx = (sxp - Jx) * k.gj * rn, By = (syp - Jy) * k.gj * rn;
    const float Bz = (D == 3) ? (szp - Jz) * k.gj * rn : 0.f;
    bq[0] -= A;
    bq[1] -= A + C;
    bq[2] -= A + 2.f * C;
    float dr = 0.f, xr = 0.f, yr = 0.f, zr = 0.f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const float t = cx<D>(q) * jx + cy<D>(q) * jy + cz<D>(q) * jz;
        const float w = k.w[cnorm2<D>(q)];
        const float P1 = fmaf(t, fmaf(k.c4, t, k.c3), bq[cnorm2<D>(q)]) -
                         (cx<D>(q) * Bx + cy<D>(q) * By + cz<D>(q) * Bz);
        const float g = w * fmaf(P1, n, dn);          // f_i^eq - w_i
        const float hp = fmaf(w, P1, w);              // w_i P_i
        d[q] = fmaf(k.omega, g - d[q], d[q]);
        sx[q] = fmaf(k.omega, fmaf(hp, Sx, -sx[q]), sx[q]);
        sy[q] = fmaf(k.omega, fmaf(hp, Sy, -sy[q]), sy[q]);
        sz[q] = fmaf(k.omega, fmaf(hp, Sz, -sz[q]), sz[q]);
        if (q != REST) {
            dr += d[q];
            xr += sx[q];
            yr += sy[q];
            zr += sz[q];
        }
    }
    d[REST] = dn - dr;
    sx[REST] = Sx - xr;
    sy[REST] = Sy - yr;
    sz[REST] = Sz - zr;
    if constexpr (MOM) {
        mom[0] = n;
        mom[1] = Sx;
        mom[2] = Sy;
        mom[3] = Sz;
        mom[4] = fmaf(k.K, de - jj, k.c);   // beta0 eps = c + K (de - |j|^2)
    }
    unsigned flag = 0u;
    if (!(n > 0.f)) flag |= (n == n) ? FLAG_NONPOSITIVE : FLAG_NONFINITE;
    if (!(fabsf(Sx) + fabsf(Sy) + fabsf(Sz) + fabsf(de) < 1e30f)) flag |= FLAG_NONFINITE;
    return flag;
}

// The four components (f, s_x, s_y, s_z) of one slot at one site are stored
// together as one vector, so that each slot plane is an array of vectors and
// a warp's access to it covers 32 consecutive vectors: 512 B in single
// precision (float4, one 128-bit access per thread), 256 B in half (4
// halves, one 64-bit access), 1 KB in double (two 128-bit accesses).  A
// neighbour shift moves by whole vectors, so every access stays aligned.
template <class T> struct QuadOf;
template <> struct QuadOf<double> { using V = DQuad; };
template <> struct QuadOf<float> { using V = float4; };
template <> struct QuadOf<__half> { using V = uint2; };

__device__ __forceinline__ void ldq(const DQuad *p, double &f, double &x, double &y, double &z)
{
    const double2 a = p->a, b = p->b;
    f = a.x;
    x = a.y;
    y = b.x;
    z = b.y;
}
__device__ __forceinline__ void stq(DQuad *p, double f, double x, double y, double z)
{
    p->a = make_double2(f, x);
    p->b = make_double2(y, z);
}
__device__ __forceinline__ void ldq(const float4 *p, float &f, float &x, float &y, float &z)
{
    const float4 v = *p;
    f = v.x;
    x = v.y;
    y = v.z;
    z = v.w;
}
__device__ __forceinline__ void stq(float4 *p, float f, float x, float y, float z) { *p = make_float4(f, x, y, z); }
__device__ __forceinline__ void ldq(const uint2 *p, __half &f, __half &x, __half &y, __half &z)
{
    const uint2 v = *p;
    const __half2 a = *reinterpret_cast<const __half2 *>(&v.x), b = *reinterpret_cast<const __half2 *>(&v.y);
    f = __low2half(a);
    x = __high2half(a);
    y = __low2half(b);
    z = __high2half(b);
}
__device__ __forceinline__ void stq(uint2 *p, __half f, __half x, __half y, __half z)
{
    const __half2 a = __halves2half2(f, x), b = __halves2half2(y, z);
    uint2 v;
    v.x = *reinterpret_cast<const unsigned *>(&a);
    v.y = *reinterpret_cast<const unsigned *>(&b);
    *p = v;
}

// Storage codecs: the stored type S (vector V of four), the arithmetic type
// R, whether the kernels work on deviations d_i = f_i - w_i (DEV) or on f_i
// itself, the collision that goes with them, and the step kernel's minimum
// resident blocks per SM (register budget).  load4 / store4 move the four
// components of one slot at one site between storage and arithmetic type.
// to_double / from_double convert a stored value of component comp (0 = f,
// 1..3 = s) of a direction of class cls = |i|^2 to and from the value of
// the population itself, in double.
struct CodecF64 {
    using S = double;
    using V = QuadOf<S>::V;
    using R = double;
    static constexpr bool DEV = false;
    static constexpr int MIN_BLOCKS = 1;   // 76 doubles per site need the registers
    static constexpr int MIN_BLOCKS_2D = MIN_BLOCKS;
    template <int D> static __device__ __forceinline__ unsigned collide(R *f, R *x, R *y, R *z, const Coll<R> &k)
    {
        return qlbm::collide<D, R>(f, x, y, z, k);
    }
    __device__ __forceinline__ R load(S v) const { return v; }
    __device__ __forceinline__ S store(R v) const { return v; }
    __device__ __forceinline__ void load4(const V *p, R &f, R &x, R &y, R &z) const
    {
        S a, b, c, d;
        ldq(p, a, b, c, d);
        f = load(a);
        x = load(b);
        y = load(c);
        z = load(d);
    }
    __device__ __forceinline__ void store4(V *p, R f, R x, R y, R z) const
    {
        stq(p, store(f), store(x), store(y), store(z));
    }
    __device__ __forceinline__ double to_double(R v, int, int) const { return v; }
    __device__ __forceinline__ S from_double(double v, int, int) const { return v; }
};
struct CodecF32 {
    using S = float;
    using V = QuadOf<S>::V;
    using R = float;
    static constexpr bool DEV = true;
    static constexpr int MIN_BLOCKS = 4;   // <= 128 registers: 16 warps per SM
    static constexpr int MIN_BLOCKS_2D = MIN_BLOCKS;
    template <int D> static __device__ __forceinline__ unsigned collide(R *f, R *x, R *y, R *z, const Coll<R> &k)
    {
        return collide_dev<D>(f, x, y, z, k);
    }
    double fref[3];   // w_i by class: the reference equilibrium's traces
    __device__ __forceinline__ R load(S v) const { return v; }
    __device__ __forceinline__ S store(R v) const { return v; }
    __device__ __forceinline__ void load4(const V *p, R &f, R &x, R &y, R &z) const
    {
        S a, b, c, d;
        ldq(p, a, b, c, d);
        f = load(a);
        x = load(b);
        y = load(c);
        z = load(d);
    }
    __device__ __forceinline__ void store4(V *p, R f, R x, R y, R z) const
    {
        stq(p, store(f), store(x), store(y), store(z));
    }
    __device__ __forceinline__ double to_double(R v, int comp, int cls) const
    {
        return comp == 0 ? fref[cls] + (double)v : (double)v;
    }
    __device__ __forceinline__ S from_double(double v, int comp, int cls) const
    {
        return (float)(comp == 0 ? v - fref[cls] : v);
    }
};
struct CodecF16Dev {
    using S = __half;
    using V = QuadOf<S>::V;
    using R = float;
    static constexpr bool DEV = true;
    static constexpr int MIN_BLOCKS = 4;
    static constexpr int MIN_BLOCKS_2D = 6;   // D2Q9: 36 values per site fit in 80 registers
    template <int D> static __device__ __forceinline__ unsigned collide(R *f, R *x, R *y, R *z, const Coll<R> &k)
    {
        return collide_dev<D>(f, x, y, z, k);
    }
    double fref[3];
    __device__ __forceinline__ R load(S v) const { return __half2float(v); }
    __device__ __forceinline__ S store(R v) const { return __float2half_rn(v); }
    // pairs convert in one instruction each way (half2 <-> float2); the
    // rounding is the same round-to-nearest as __float2half_rn per value
    __device__ __forceinline__ void load4(const V *p, R &f, R &x, R &y, R &z) const { decode4(*p, f, x, y, z); }
    __device__ __forceinline__ void decode4(const V &v, R &f, R &x, R &y, R &z) const
    {
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&v.y));
        f = a.x;
        x = a.y;
        y = b.x;
        z = b.y;
    }
    __device__ __forceinline__ void store4(V *p, R f, R x, R y, R z) const
    {
        const __half2 a = __floats2half2_rn(f, x), b = __floats2half2_rn(y, z);
        uint2 v;
        v.x = *reinterpret_cast<const unsigned *>(&a);
        v.y = *reinterpret_cast<const unsigned *>(&b);
        *p = v;
    }
    __device__ __forceinline__ double to_double(R v, int comp, int cls) const
    {
        return comp == 0 ? fref[cls] + (double)v : (double)v;
    }
    __device__ __forceinline__ S from_double(double v, int comp, int cls) const
    {
        return __double2half(comp == 0 ? v - fref[cls] : v);
    }
};

// Extent and addressing of a lattice: plane stride P (vectors) separates
// the b slot planes of the single population buffer.
struct Grid {
    int nx, ny, nz;
    int nxb;        // blocks per x-row
    int zero;       // always 0 (see k_step_aa)
    int64_t P;      // plane stride (vectors of four components)
    int64_t N;      // sites
};

__device__ __forceinline__ int wrapm(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

}  // namespace qlbm
