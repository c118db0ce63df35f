// D3Q19 (Sec. 3.1, d = 3, b = 19) step for FP64 storage in double-float arithmetic
// (QLBM_FP64_DF); the other operations of that precision are the FP64 ones
// (kernels_d3q19_fp64.cu holds its dispatch table).
#include "f64df.cuh"
#include "launch.cuh"

namespace qlbm {

template <int D> cudaError_t step_f64df(qlbm_ctx *h, bool odd)
{
    // blocks of two warps over F64dfSplit<D>::SITES consecutive sites of a
    // row, so the grid is laid out for that block width
    Grid g = h->g;
    g.nxb = (g.nx + F64dfSplit<D>::SITES - 1) / F64dfSplit<D>::SITES;
    const dim3 blk(kF64dfBlock), grd((unsigned)((int64_t)g.nxb * g.ny * g.nz));
    const Planes<double, Lattice<D>::Q> pl = Launchers<D, CodecF64>::planes(h);
    const Coll<df> k = make_coll<df>(h);
    const Coll<double> kd = make_coll<double>(h);
    F64dfConst kc;
    for (int i = 0; i < 2; ++i) {
        kc.wc3[i] = df(kd.w[i + 1] * kd.c3);
        kc.wc4[i] = df(kd.w[i + 1] * kd.c4);
    }
    return with_field(h->mag, [&](auto fc) {
        constexpr int F = decltype(fc)::value;
        if (odd) k_step_aa_f64df<D, true, F><<<grd, blk, 0, h->stream>>>(pl, g, k, kc, h->flags);
        else k_step_aa_f64df<D, false, F><<<grd, blk, 0, h->stream>>>(pl, g, k, kc, h->flags);
        return cudaGetLastError();
    });
}
template cudaError_t step_f64df<3>(qlbm_ctx *h, bool odd);

}  // namespace qlbm
