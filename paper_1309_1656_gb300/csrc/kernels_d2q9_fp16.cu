// D2Q9 (Sec. 3.1, d = 2, b = 9) kernels for FP16 deviation storage: the dispatch table of one lattice and one
// storage codec, in a translation unit of its own so the instantiations
// compile in parallel.
#include "steplaunch.cuh"

namespace qlbm {
template cudaError_t Launchers<2, CodecF16Dev>::step(qlbm_ctx *, bool);
template cudaError_t Launchers<2, CodecF16Dev>::step_fdout(qlbm_ctx *, bool, float *, float *, float *, float *);
const LatticeOps *ops_d2q9_fp16() { return Launchers<2, CodecF16Dev>::table(); }
}  // namespace qlbm
