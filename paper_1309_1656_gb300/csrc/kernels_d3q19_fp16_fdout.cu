// D3Q19 (Sec. 3.1, d = 3, b = 19) launcher of the step with the fused
// single-precision Fermi-Dirac solve for FP16 deviation storage, compiled apart from the rest of
// its dispatch table (kernels_d3q19_fp16.cu).
#include "steplaunch.cuh"

namespace qlbm {
template cudaError_t Launchers<3, CodecF16Dev>::step_fdout(qlbm_ctx *, bool, float *, float *, float *, float *);
}  // namespace qlbm
