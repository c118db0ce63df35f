// D3Q19 (Sec. 3.1, d = 3, b = 19) kernels for double-float storage: the dispatch table of one lattice and one
// storage codec, in a translation unit of its own so the instantiations
// compile in parallel.
#include "launch.cuh"

namespace qlbm {
const LatticeOps *ops_d3q19_df64() { return Launchers<3, CodecDF>::table(); }
}  // namespace qlbm
