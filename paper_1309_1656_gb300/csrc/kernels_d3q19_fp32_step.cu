// D3Q19 (Sec. 3.1, d = 3, b = 19) fused step launcher for FP32 deviation storage, compiled apart
// from the rest of its dispatch table (kernels_d3q19_fp32.cu) so that the heaviest
// kernels build in parallel.
#include "steplaunch.cuh"

namespace qlbm {
template cudaError_t Launchers<3, CodecF32>::step(qlbm_ctx *, bool);
}  // namespace qlbm
