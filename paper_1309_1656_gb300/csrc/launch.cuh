// Host launchers of the kernels for one lattice and one storage codec,
// gathered into a dispatch table (Launchers<D, Codec>::table()).  Each
// kernels_<lattice>_<codec>.cu instantiates one of them.
#pragma once

#include <type_traits>

#include "internal.h"
#include "adjoint.cuh"
#include "fdkernels.cuh"
#include "kernels.cuh"
#include "twopass.cuh"

namespace qlbm {

template <typename R> Coll<R> make_coll(const qlbm_ctx *h)
{
    const HostConsts &k = h->hc;
    const double omega = h->dt / h->tau;
    Coll<R> c;
    c.K = (R)k.K;
    c.c = (R)k.c;
    c.inv_mc2 = (R)(1.0 / (k.m - k.c * k.c));
    c.c3 = (R)(2.0 * k.K * k.alpha3);
    c.c4 = (R)(4.0 * k.K * k.K * k.alpha4);
    c.c5 = (R)(k.K * k.alpha5);
    c.omega = (R)omega;
    for (int i = 0; i < 3; ++i) c.w[i] = (R)k.w[i];
    // Gram matrix of (1, |i|^2) under the weights, and sum w i_x^2
    const int d = k.d;
    const double na = (d == 2) ? 4.0 : 6.0, nd = (d == 2) ? 4.0 : 12.0;  // axis / diagonal counts
    const double S0 = k.w[0] + na * k.w[1] + nd * k.w[2];
    const double S2 = na * k.w[1] + 2.0 * nd * k.w[2];
    const double S4 = na * k.w[1] + 4.0 * nd * k.w[2];
    const double det = S0 * S4 - S2 * S2;
    c.g00 = (R)(S4 / det);
    c.g01 = (R)(-S2 / det);
    c.g11 = (R)(S0 / det);
    const double sx2 = 2.0 * k.w[1] + ((d == 2) ? 4.0 : 8.0) * k.w[2];
    c.gj = (R)(1.0 / sx2);
    c.S2 = (R)S2;
    for (int i = 0; i < 9; ++i) c.rot[i] = (R)h->rot[i];
    c.qf = static_cast<const typename FieldOf<R>::V *>(h->qfield);
    return c;
}

// Calls f(std::integral_constant<int, FIELD>{}) for the handle's field mode
// (FIELD_NONE, FIELD_UNIFORM or FIELD_SITE), so that a launcher names each
// kernel once for all three variants.
template <class F> inline cudaError_t with_field(int mode, F &&f)
{
    switch (mode) {
    case FIELD_UNIFORM: return f(std::integral_constant<int, FIELD_UNIFORM>{});
    case FIELD_SITE: return f(std::integral_constant<int, FIELD_SITE>{});
    default: return f(std::integral_constant<int, FIELD_NONE>{});
    }
}

inline InitConsts make_init(const qlbm_ctx *h)
{
    const HostConsts &k = h->hc;
    InitConsts ic;
    ic.xi = k.xi;
    ic.K = k.K;
    ic.c = k.c;
    ic.inv_mc2 = 1.0 / (k.m - k.c * k.c);
    ic.c3 = 2.0 * k.K * k.alpha3;
    ic.c4 = 4.0 * k.K * k.K * k.alpha4;
    ic.c5 = k.K * k.alpha5;
    ic.eps0 = k.eps0;
    ic.beta0 = k.beta0;
    for (int i = 0; i < 3; ++i) ic.w[i] = k.w[i];
    return ic;
}

template <class Codec> Codec make_codec(const qlbm_ctx *h);
template <> inline CodecF64 make_codec<CodecF64>(const qlbm_ctx *) { return CodecF64{}; }
// Deviation reference: the uniform equilibrium n = 1, S = 0, u = 0,
// eps = eps0, where P_i = 1, so f_i^ref = w_i and s_i^ref = 0.
template <> inline CodecF32 make_codec<CodecF32>(const qlbm_ctx *h)
{
    CodecF32 c;
    for (int i = 0; i < 3; ++i) c.fref[i] = h->hc.w[i];
    return c;
}
template <> inline CodecF16Dev make_codec<CodecF16Dev>(const qlbm_ctx *h)
{
    CodecF16Dev c;
    for (int i = 0; i < 3; ++i) c.fref[i] = h->hc.w[i];
    return c;
}
template <> inline CodecDF make_codec<CodecDF>(const qlbm_ctx *h)
{
    CodecDF c;
    c.lo = (int64_t)h->b * h->g.P;
    return c;
}

template <int D, class Codec> struct Launchers {
    using S = typename Codec::S;
    using R = typename Codec::R;
    static constexpr int Q = Lattice<D>::Q;

    template <class T> static Planes<T, Q> planes_of(const qlbm_ctx *h, const void *base)
    {
        using V = typename QuadOf<T>::V;
        Planes<T, Q> pl;
        V *b = static_cast<V *>(const_cast<void *>(base));
        for (int q = 0; q < Q; ++q) pl.p[q] = b + (int64_t)q * h->g.P;
        return pl;
    }
    static Planes<S, Q> planes(const qlbm_ctx *h) { return planes_of<S>(h, h->pop); }

    // The step launchers (steplaunch.cuh) are compiled in translation units
    // of their own (kernels_<lattice>_<codec>_step.cu), in parallel with the
    // rest of the table.
    static cudaError_t step(qlbm_ctx *h, bool odd);
    static cudaError_t step_fd(qlbm_ctx *h, bool odd);
    static cudaError_t step_fdout(qlbm_ctx *h, bool odd, float *beta, float *mu_up, float *mu_dn, float *axis);

    static cudaError_t init_eq(qlbm_ctx *h, const double *rho4, const double *u, const double *eps)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        k_init_eq<D, Codec><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_init(h),
                                                        make_codec<Codec>(h), rho4, u, eps);
        return cudaGetLastError();
    }

    static cudaError_t get_state(qlbm_ctx *h, double *out)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        const Planes<S, Q> pl = planes(h);
        if (h->parity)
            k_get_state<D, Codec, true><<<grd, blk, 0, h->stream>>>(pl, h->g, make_codec<Codec>(h), out);
        else
            k_get_state<D, Codec, false><<<grd, blk, 0, h->stream>>>(pl, h->g, make_codec<Codec>(h), out);
        return cudaGetLastError();
    }

    static cudaError_t set_state(qlbm_ctx *h, const double *in)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        k_set_state<D, Codec><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_codec<Codec>(h), in);
        return cudaGetLastError();
    }

    static cudaError_t moments(qlbm_ctx *h, double *rho4, double *u, double *eps)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        const Planes<S, Q> pl = planes(h);
        if (h->parity)
            k_moments<D, Codec, true><<<grd, blk, 0, h->stream>>>(pl, h->g, make_codec<Codec>(h),
                                                                  h->hc.xi, rho4, u, eps);
        else
            k_moments<D, Codec, false><<<grd, blk, 0, h->stream>>>(pl, h->g, make_codec<Codec>(h),
                                                                   h->hc.xi, rho4, u, eps);
        return cudaGetLastError();
    }

    static cudaError_t conserved_partial(qlbm_ctx *h)
    {
        if (!h->red_grid) {
            // one whole wave of resident blocks (a fixed count left a
            // partial second wave); found once per handle
            int a = 0, b = 0;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_conserved_partial<D, Codec, false>,
                                                                          kRedBlock, 0);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_conserved_partial<D, Codec, true>, kRedBlock, 0);
            if (e != cudaSuccess) return e;
            const int64_t wave = (int64_t)(a < b ? a : b) * h->sms;
            h->red_grid = (int)(wave >= 1 && wave < h->nred ? wave : h->nred);
        }
        const Planes<S, Q> pl = planes(h);
        if (h->parity)
            k_conserved_partial<D, Codec, true><<<h->red_grid, kRedBlock, 0, h->stream>>>(
                pl, h->g, make_codec<Codec>(h), h->partials);
        else
            k_conserved_partial<D, Codec, false><<<h->red_grid, kRedBlock, 0, h->stream>>>(
                pl, h->g, make_codec<Codec>(h), h->partials);
        return cudaGetLastError();
    }

    static cudaError_t adjoint(qlbm_ctx *h, const void *state, const void *lam_in, void *lam_out)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        return with_field(h->mag, [&](auto fc) {
            constexpr int F = decltype(fc)::value;
            k_adjoint<D, Codec, F><<<grd, blk, 0, h->stream>>>(planes_of<S>(h, state), planes_of<R>(h, lam_in),
                                                               planes_of<R>(h, lam_out), h->g, make_coll<R>(h),
                                                               make_codec<Codec>(h), h->dtau_acc);
            return cudaGetLastError();
        });
    }

    static cudaError_t push(qlbm_ctx *h, const void *src, void *dst)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        return with_field(h->mag, [&](auto fc) {
            constexpr int F = decltype(fc)::value;
            k_step_push<D, Codec, F><<<grd, blk, 0, h->stream>>>(planes_of<S>(h, src), planes_of<S>(h, dst), h->g,
                                                                 make_coll<R>(h), make_codec<Codec>(h), h->flags);
            return cudaGetLastError();
        });
    }

    static cudaError_t copy_natural(qlbm_ctx *h, void *dst)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        if (h->parity)
            k_copy_natural<D, Codec, true><<<grd, blk, 0, h->stream>>>(planes(h), planes_of<S>(h, dst), h->g,
                                                                       make_codec<Codec>(h));
        else
            k_copy_natural<D, Codec, false><<<grd, blk, 0, h->stream>>>(planes(h), planes_of<S>(h, dst), h->g,
                                                                        make_codec<Codec>(h));
        return cudaGetLastError();
    }

    static cudaError_t lam_import(qlbm_ctx *h, const double *in, void *lam)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        k_lam_import<D, R><<<grd, blk, 0, h->stream>>>(in, planes_of<R>(h, lam), h->g);
        return cudaGetLastError();
    }

    static cudaError_t lam_export(qlbm_ctx *h, const void *lam, double *out)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        k_lam_export<D, R><<<grd, blk, 0, h->stream>>>(planes_of<R>(h, lam), h->g, out);
        return cudaGetLastError();
    }

    static cudaError_t init_adjoint(qlbm_ctx *h, const double *lam, const double *rho4, const double *u,
                                    const double *eps, double *grho4, double *gu, double *geps)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        k_init_adjoint<D><<<grd, blk, 0, h->stream>>>(lam, h->g, make_init(h), rho4, u, eps, grho4, gu, geps);
        return cudaGetLastError();
    }

    static cudaError_t fd_params(qlbm_ctx *h, double *beta, double *mu_up, double *mu_dn, double *axis)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        const FdArgs a{h->hc.beta0, h->hc.xi};
        if (h->parity)
            k_fd_params<D, Codec, true><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_codec<Codec>(h), a, beta,
                                                                    mu_up, mu_dn, axis, h->fd_fail);
        else
            k_fd_params<D, Codec, false><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_codec<Codec>(h), a, beta,
                                                                     mu_up, mu_dn, axis, h->fd_fail);
        return cudaGetLastError();
    }

    static cudaError_t fd_params_adjoint(qlbm_ctx *h, const double *gbeta, const double *gmu_up,
                                         const double *gmu_dn, const double *gaxis, double *lam)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        const FdArgs a{h->hc.beta0, h->hc.xi};
        if (h->parity)
            k_fd_params_adjoint<D, Codec, true><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_codec<Codec>(h), a,
                                                                            gbeta, gmu_up, gmu_dn, gaxis, lam);
        else
            k_fd_params_adjoint<D, Codec, false><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_codec<Codec>(h), a,
                                                                             gbeta, gmu_up, gmu_dn, gaxis, lam);
        return cudaGetLastError();
    }

    static cudaError_t init_fd(qlbm_ctx *h, const double *beta, const double *mu_up, const double *mu_dn,
                               const double *axis, const double *u)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        k_init_fd<D, Codec><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_init(h), make_codec<Codec>(h), beta,
                                                        mu_up, mu_dn, axis, u);
        return cudaGetLastError();
    }

    static cudaError_t negative_eq(qlbm_ctx *h, unsigned long long *count, unsigned *mask)
    {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        if (h->parity)
            k_negative_eq<D, Codec, true><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_codec<Codec>(h),
                                                                      make_init(h), count, mask);
        else
            k_negative_eq<D, Codec, false><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_codec<Codec>(h),
                                                                       make_init(h), count, mask);
        return cudaGetLastError();
    }

    // Entries that exist for some codecs only: named inside if constexpr, so
    // that the others never reference (and never need) their definitions.
    static constexpr auto step_fd_entry()
    {
        if constexpr (std::is_same<Codec, CodecF64>::value) return &step_fd;
        else return static_cast<decltype(&step_fd)>(nullptr);
    }
    static constexpr auto step_fdout_entry()
    {
        if constexpr (Codec::DEV) return &step_fdout;
        else return static_cast<decltype(&step_fdout)>(nullptr);
    }

    // The reverse mode (adjoint, push, cotangent import/export) exists for
    // the FP64, FP32 and FP16 codecs; double-float storage is forward only.
    static const LatticeOps *table()
    {
        if constexpr (std::is_same<Codec, CodecDF>::value) {
            static const LatticeOps t = {&step,    &init_eq,      &get_state,  &set_state,  &moments,
                                         &conserved_partial, nullptr, nullptr, &copy_natural, nullptr,
                                         nullptr, &init_adjoint, &fd_params, nullptr,
                                         &fd_params_adjoint, &init_fd, nullptr, &negative_eq};
            return &t;
        } else {
            static const LatticeOps t = {&step,    &init_eq,      &get_state,  &set_state,  &moments,
                                         &conserved_partial, &adjoint, &push, &copy_natural, &lam_import,
                                         &lam_export, &init_adjoint, &fd_params, step_fd_entry(),
                                         &fd_params_adjoint, &init_fd, step_fdout_entry(), &negative_eq};
            return &t;
        }
    }
};

}  // namespace qlbm
