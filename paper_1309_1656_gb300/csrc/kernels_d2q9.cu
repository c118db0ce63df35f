// D2Q9 instantiation of the forward kernels (Sec. 3.1, d = 2, b = 9).
#include "launch.cuh"

namespace qlbm {
const LatticeOps *lattice_ops_d2q9(int prec) { return ops_for<2>(prec); }
}  // namespace qlbm
