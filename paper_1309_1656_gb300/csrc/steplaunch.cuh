// Definitions of the step launchers of Launchers<D, Codec> (launch.cuh):
// the fused AA step (all codecs), the FP64 step through the recovered
// Fermi-Dirac parameters, and the single-precision step with the fused FD
// solve.  Each kernels_<lattice>_<codec>_step.cu instantiates them for one
// lattice and codec, apart from the rest of the dispatch table, so that the
// heaviest kernels compile in parallel with the others.
#pragma once

#include "launch.cuh"

namespace qlbm {

template <int D, class Codec>
cudaError_t Launchers<D, Codec>::step(qlbm_ctx *h, bool odd)
{
    const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
    const Planes<S, Q> pl = planes(h);
    const Coll<R> k = make_coll<R>(h);
    const Codec codec = make_codec<Codec>(h);
    if constexpr (TwoPass<Codec>::value) {
        return with_field(h->mag, [&](auto fc) {
            constexpr int F = decltype(fc)::value;
            if (odd)
                k_step_aa_df2<D, true, F><<<grd, blk, 0, h->stream>>>(pl, h->g, k, codec, h->flags);
            else
                k_step_aa_df2<D, false, F><<<grd, blk, 0, h->stream>>>(pl, h->g, k, codec, h->flags);
            return cudaGetLastError();
        });
    } else if constexpr (RowPipelined<Codec>::value) {
        // rows per block from a sweep on GB300 (FP16): D2Q9 4096^2 gains
        // 14 % at 8, D3Q19 192^3 - 256^3 4-7 % at 4 (more rows lose to the tail)
        const int rpb = step_rows_per_block(h->g, D == 2 ? 8 : 4, step_min_blocks<D, Codec>(), h->sms);
        const dim3 grr = row_group_grid(h->g, rpb);
        const size_t sm = rows_smem_bytes<D, Codec>((int)blk.x);
        return with_field(h->mag, [&](auto fc) {
            constexpr int F = decltype(fc)::value;
            if (odd)
                k_step_aa_rows<D, Codec, true, F><<<grr, blk, sm, h->stream>>>(pl, h->g, k, codec, rpb, h->flags);
            else
                k_step_aa_rows<D, Codec, false, F><<<grr, blk, sm, h->stream>>>(pl, h->g, k, codec, rpb, h->flags);
            return cudaGetLastError();
        });
    } else {
        return with_field(h->mag, [&](auto fc) {
            constexpr int F = decltype(fc)::value;
            if (odd)
                k_step_aa<D, Codec, true, F><<<grd, blk, 0, h->stream>>>(pl, h->g, k, codec, h->flags);
            else
                k_step_aa<D, Codec, false, F><<<grd, blk, 0, h->stream>>>(pl, h->g, k, codec, h->flags);
            return cudaGetLastError();
        });
    }
    return cudaGetLastError();
}

template <int D, class Codec>
cudaError_t Launchers<D, Codec>::step_fd(qlbm_ctx *h, bool odd)
{
    if constexpr (std::is_same<Codec, CodecF64>::value) {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        const FdArgs a{h->hc.beta0, h->hc.xi};
        return with_field(h->mag, [&](auto fc) {
            constexpr int F = decltype(fc)::value;
            if (odd)
                k_step_aa_fd<D, true, F><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_coll<double>(h), a,
                                                                     h->flags);
            else
                k_step_aa_fd<D, false, F><<<grd, blk, 0, h->stream>>>(planes(h), h->g, make_coll<double>(h), a,
                                                                      h->flags);
            return cudaGetLastError();
        });
    } else {
        return cudaErrorNotSupported;
    }
}

template <int D, class Codec>
cudaError_t Launchers<D, Codec>::step_fdout(qlbm_ctx *h, bool odd, float *beta, float *mu_up, float *mu_dn,
                                          float *axis)
{
    if constexpr (Codec::DEV) {
        const dim3 blk = site_block(h->g), grd = site_grid(h->g, blk.x);
        const Planes<S, Q> pl = planes(h);
        const Coll<R> k = make_coll<R>(h);
        const Codec codec = make_codec<Codec>(h);
        const float b0 = (float)h->hc.beta0;
        return with_field(h->mag, [&](auto fc) {
            constexpr int F = decltype(fc)::value;
            if (odd)
                k_step_aa_fdout<D, Codec, true, F><<<grd, blk, 0, h->stream>>>(pl, h->g, k, codec, b0, h->flags,
                                                                               beta, mu_up, mu_dn, axis,
                                                                               h->fd_fail);
            else
                k_step_aa_fdout<D, Codec, false, F><<<grd, blk, 0, h->stream>>>(pl, h->g, k, codec, b0, h->flags,
                                                                                beta, mu_up, mu_dn, axis,
                                                                                h->fd_fail);
            return cudaGetLastError();
        });
    } else {
        return cudaErrorNotSupported;
    }
}

}  // namespace qlbm
