// D2Q9 (Sec. 3.1, d = 2, b = 9) kernels for double-float storage: the dispatch table of one lattice and one
// storage codec, in a translation unit of its own so the instantiations
// compile in parallel.
#include "steplaunch.cuh"

namespace qlbm {
template cudaError_t Launchers<2, CodecDF>::step(qlbm_ctx *, bool);
const LatticeOps *ops_d2q9_df64() { return Launchers<2, CodecDF>::table(); }
}  // namespace qlbm
