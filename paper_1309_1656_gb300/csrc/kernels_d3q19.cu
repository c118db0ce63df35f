// D3Q19 instantiation of the forward kernels (Sec. 3.1, d = 3, b = 19).
#include "launch.cuh"

namespace qlbm {
const LatticeOps *lattice_ops_d3q19(int prec) { return ops_for<3>(prec); }
}  // namespace qlbm
