// D2Q9 (Sec. 3.1, d = 2, b = 9) kernels for FP32 deviation storage: the dispatch table of one lattice and one
// storage codec, in a translation unit of its own so the instantiations
// compile in parallel.
#include "steplaunch.cuh"

namespace qlbm {
template cudaError_t Launchers<2, CodecF32>::step(qlbm_ctx *, bool);
template cudaError_t Launchers<2, CodecF32>::step_fdout(qlbm_ctx *, bool, float *, float *, float *, float *);
const LatticeOps *ops_d2q9_fp32() { return Launchers<2, CodecF32>::table(); }
}  // namespace qlbm
