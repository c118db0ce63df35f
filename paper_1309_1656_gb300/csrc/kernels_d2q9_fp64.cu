// D2Q9 (Sec. 3.1, d = 2, b = 9) kernels for FP64 storage: the dispatch tables of FP64 storage with the
// FP64 and the double-float step, in a translation unit of its own so the instantiations
// compile in parallel.
#include "steplaunch.cuh"

namespace qlbm {
template cudaError_t Launchers<2, CodecF64>::step(qlbm_ctx *, bool);
template cudaError_t Launchers<2, CodecF64>::step_fd(qlbm_ctx *, bool);
const LatticeOps *ops_d2q9_fp64() { return Launchers<2, CodecF64>::table(); }

// FP64 storage with the double-float step: the FP64 operations, the step of
// kernels_d2q9_fp64df.cu, no reverse mode (its recorded trajectory would
// come from the FP64 step).
const LatticeOps *ops_d2q9_fp64df()
{
    static const LatticeOps t = [] {
        LatticeOps o = *Launchers<2, CodecF64>::table();
        o.step = &step_f64df<2>;
        o.adjoint = nullptr;
        o.push = nullptr;
        o.lam_import = nullptr;
        o.lam_export = nullptr;
        return o;
    }();
    return &t;
}
}  // namespace qlbm
