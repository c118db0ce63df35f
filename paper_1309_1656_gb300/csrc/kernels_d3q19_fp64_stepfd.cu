// D3Q19 (Sec. 3.1, d = 3, b = 19) launcher of the FP64 step whose equilibrium
// goes through the recovered Fermi-Dirac parameters (Eq. WeqDiscr), compiled
// apart from the rest of its dispatch table (kernels_d3q19_fp64.cu).
#include "steplaunch.cuh"

namespace qlbm {
template cudaError_t Launchers<3, CodecF64>::step_fd(qlbm_ctx *, bool);
}  // namespace qlbm
